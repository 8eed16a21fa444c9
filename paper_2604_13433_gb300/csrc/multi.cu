// Split-row products with k right-hand sides over CSR-order PackSELL
// matrices (C = 1), for one matrix or a batch of them in one launch.
//
// The CSR-based form of the packing (each slice one row, no padding, the
// slice offsets are the row pointer) is the paper's future work for matrices
// whose rows vary too much for SELL slices (§5.1.1, §7). This kernel extends
// the split-row SpMV (variant 14) to Y = A X with X row-major [m x k] and to
// many matrices per launch:
//  * work items are tiles of consecutive rows of one matrix (at most MCT
//    words and MR_MAX rows) and single long rows, long rows first, longest
//    first; an item names its matrix, whose descriptor (arrays, vectors,
//    parameters) the warp reads when it takes the item;
//  * a warp holds a tile's words, four consecutive words per lane; the
//    columns come from a segmented prefix sum of the deltas restarting at each
//    row start (the left offset of Eq. 4 there), as in variant 14;
//  * the columns of X are taken four at a time: every word with a value
//    gathers four entries of its X row (one 16-byte load when k, ldx and X
//    allow it) and multiplies them by its value; the four products of each
//    word are summed per row with a segmented sum across the lanes, and the
//    lane holding a row's first word writes the row's four results;
//  * a long row is walked in chunks, each lane summing its own words, then a
//    butterfly reduction; once per group of four columns.
// The summation order is fixed (the same bits on every run) but is a tree:
// every entry of Y is within gamma_w * sum_j |a_ij X_jq| of the exact product
// (w stored words of the row). For k > 16 with 16-byte X and Y rows a second
// kernel, k_split_rows below, decodes each item once into a table in shared
// memory and walks its words; there a tile's rows keep the stored-order
// chain of the thread-per-row SpMV.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int MT = 128;                  // words a warp holds per chunk: four per lane
constexpr int MCT = kMultiTileWords;     // tile words at most (MT - 3: room for the aligned-down start)
constexpr int MR_MAX = kMultiTileRows;   // tile rows at most
constexpr int MW = 8;                    // warps per block
static_assert(MCT == MT - 3, "tile words must leave room for the aligned-down start");
constexpr uint32_t kAbsM = 0x80000000u;

__device__ __forceinline__ uint32_t mcomb(uint32_t a, uint32_t b) {
    return b + (a & ~(uint32_t)((int32_t)b >> 31));
}

__device__ __forceinline__ int mleft(int row, int sigma, int sig_shift, int kl) {
    const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
    return max(blk - kl, 0);
}

__device__ __forceinline__ int mout(const SplitMat &M, int row) {
    if (!M.perm_bytes) return row;
    const int blk = M.sig_shift >= 0 ? (row >> M.sig_shift) << M.sig_shift : (row / M.sigma) * M.sigma;
    return blk + (M.perm_bytes == 1 ? (int)((const uint8_t *)M.perm)[row]
                                    : (int)((const uint16_t *)M.perm)[row]);
}

__device__ __forceinline__ float mvalue(const SplitMat &M, uint32_t wd) {
    return M.fmt == PACKSELL_FMT_FP16 ? __high2float(*reinterpret_cast<const __half2 *>(&wd))
                                      : __uint_as_float(wd & M.vmask);
}

__device__ __forceinline__ uint32_t mdelta(const SplitMat &M, uint32_t wd) {
    return (wd >> 1) & ((wd & 1u) ? M.dmask : 0x7fffffffu);
}

// NV consecutive entries of a row of X or Y: NV = 4 (a group of four
// columns, one 16-byte access when VEC) or NV = 1 (k = 1, one column)
template <int NV>
struct MVec {
    float v[NV];
};

template <int NV>
__device__ __forceinline__ MVec<NV> mzero() {
    MVec<NV> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = 0.f;
    return r;
}

// entries q .. q + NV - 1 of an X row (0 past column k)
template <int NV, bool VEC>
__device__ __forceinline__ MVec<NV> mload(const float *__restrict__ xr, int q, int k) {
    MVec<NV> r;
    if constexpr (NV == 4 && VEC) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(xr));
        r.v[0] = t.x;
        r.v[1] = t.y;
        r.v[2] = t.z;
        r.v[3] = t.w;
    } else {
#pragma unroll
        for (int i = 0; i < NV; ++i) r.v[i] = q + i < k ? __ldg(xr + i) : 0.f;
    }
    return r;
}

template <int NV, bool VEC>
__device__ __forceinline__ void mstore(float *__restrict__ yr, int q, int k, const MVec<NV> &a) {
    if constexpr (NV == 4 && VEC) {
        *reinterpret_cast<float4 *>(yr) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
    } else {
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (q + i < k) yr[i] = a.v[i];
    }
}

template <int NV>
__device__ __forceinline__ void madd(MVec<NV> &a, const MVec<NV> &b) {
#pragma unroll
    for (int i = 0; i < NV; ++i) a.v[i] += b.v[i];
}

template <int NV>
__device__ __forceinline__ MVec<NV> mshfl_down(const MVec<NV> &a, int o) {
    MVec<NV> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = __shfl_down_sync(0xffffffffu, a.v[i], o);
    return r;
}

template <int NV>
__device__ __forceinline__ MVec<NV> mxor(const MVec<NV> &a, int o) {
    MVec<NV> r;
#pragma unroll
    for (int i = 0; i < NV; ++i) r.v[i] = __shfl_xor_sync(0xffffffffu, a.v[i], o);
    return r;
}

__device__ __forceinline__ uint4 mload_words(const uint32_t *__restrict__ pack, long long first,
                                             int lim, int lane) {
    const int p = 4 * lane;
    return p < lim ? __ldcs(reinterpret_cast<const uint4 *>(pack + first + p)) : make_uint4(0, 0, 0, 0);
}

// One row of more than MCT words, every group of NV columns in turn: MT
// words per chunk (four per lane), each lane summing its own words, the
// column carried across chunks, then a butterfly reduction.
template <int NV, bool VEC>
__device__ __forceinline__ void multi_long_row(const SplitMat &M, int row, long long base, int nwd,
                                               int lane) {
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0), lim = lead + nwd;
    const int io = mout(M, row);
    const int c0 = mleft(row, M.sigma, M.sig_shift, M.kl);
    for (int q0 = 0; q0 < M.k; q0 += NV) {
        uint32_t carry = (uint32_t)c0;
        MVec<NV> t = mzero<NV>();
        uint4 cur = mload_words(M.pack, a0, lim, lane);
        for (int k0 = 0; k0 < lim; k0 += MT) {
            const uint4 nxt = mload_words(M.pack, a0 + k0 + MT, lim - k0 - MT, lane);
            uint32_t wd[4] = {cur.x, cur.y, cur.z, cur.w}, cs[4], acc = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = k0 + 4 * lane + j;
                if ((unsigned)(p - lead) >= (unsigned)nwd) wd[j] = 0u;
                acc += mdelta(M, wd[j]);
                cs[j] = acc;
            }
            uint32_t inc = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            const uint32_t before = carry + inc - acc;
            carry += __shfl_sync(0xffffffffu, inc, 31);
            MVec<NV> xv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                xv[j] = ((wd[j] & 1u) && PS_IN_RANGE(before + cs[j], M.xlen))
                            ? mload<NV, VEC>(M.X + (size_t)(before + cs[j]) * M.ldx + q0, q0, M.k)
                                     : mzero<NV>();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (wd[j] & 1u) {
                    const float v = mvalue(M, wd[j]);
#pragma unroll
                    for (int i = 0; i < NV; ++i) t.v[i] = fmaf(v, xv[j].v[i], t.v[i]);
                }
            }
            cur = nxt;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) madd(t, mxor(t, o));
        if (lane == 0) mstore<NV, VEC>(M.Y + (size_t)io * M.ldy + q0, q0, M.k, t);
    }
}

// A tile of rows [r0, r0 + nrows) of nwd (<= MCT) words, four per lane in wv.
template <int NV, bool VEC>
__device__ __forceinline__ void multi_tile(const SplitMat &M, int r0, int nrows, long long base,
                                           int nwd, int lane, const uint4 &wv,
                                           uint32_t *__restrict__ s_lft, int *__restrict__ s_io,
                                           const uint32_t *__restrict__ soff) {
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0);
    reinterpret_cast<uint4 *>(s_lft)[lane] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    // row starts: kAbs | left offset and the y row; empty rows get 0
    const uint32_t a0lo = (uint32_t)a0;
    for (int kk = lane; kk < nrows; kk += 32) {
        const int r = r0 + kk;
        const uint32_t o0 = soff[kk], o1 = soff[kk + 1];
        const int io = mout(M, r);
        if (o1 != o0) {
            const int pos = (int)(o0 - a0lo);
            s_lft[pos] = kAbsM | (uint32_t)mleft(r, M.sigma, M.sig_shift, M.kl);
            s_io[pos] = io;
        } else {
            for (int q0 = 0; q0 < M.k; q0 += NV)
                mstore<NV, VEC>(M.Y + (size_t)io * M.ldy + q0, q0, M.k, mzero<NV>());
        }
    }
    __syncwarp();
    const uint4 hv = reinterpret_cast<const uint4 *>(s_lft)[lane];
    const uint32_t hl[4] = {hv.x, hv.y, hv.z, hv.w};
    uint32_t wd[4] = {wv.x, wv.y, wv.z, wv.w}, cs[4], acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int p = 4 * lane + j;
        if ((unsigned)(p - lead) >= (unsigned)nwd) wd[j] = 0u;
        acc = mcomb(acc, hl[j] + mdelta(M, wd[j]));
        cs[j] = acc;
    }
    uint32_t inc = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = mcomb(v, inc);
    }
    uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = 0u;  // the tile's first word starts a row
    uint32_t col[4];
    float val[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        col[j] = mcomb(exc, cs[j]) & ~kAbsM;
        val[j] = (wd[j] & 1u) ? mvalue(M, wd[j]) : 0.f;
    }
    uint32_t hm = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) hm |= (hl[j] >> 31) << j;
    const int fh = hm ? __ffs(hm) - 1 : 4;
    const unsigned heads = __ballot_sync(0xffffffffu, hm != 0u);
    for (int q0 = 0; q0 < M.k; q0 += NV) {
        MVec<NV> pv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            MVec<NV> xv = mzero<NV>();
            if ((wd[j] & 1u) && PS_IN_RANGE(col[j], M.xlen))
                xv = mload<NV, VEC>(M.X + (size_t)col[j] * M.ldx + q0, q0, M.k);
#pragma unroll
            for (int i = 0; i < NV; ++i) pv[j].v[i] = val[j] * xv.v[i];
        }
        // A: the lane's words before its first row start; U: A plus, while no
        // row start intervenes, the same of the lanes after it
        MVec<NV> U = mzero<NV>();
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < fh) madd(U, pv[j]);
        bool F = hm != 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const MVec<NV> v = mshfl_down(U, o);
            if (lane + o < 32 && !F) {
                madd(U, v);
                F = ((heads >> (lane + o)) & ((1u << o) - 1u)) != 0u;
            }
        }
        MVec<NV> s = mshfl_down(U, 1);
        if (lane == 31) s = mzero<NV>();
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            madd(s, pv[j]);
            if (hl[j] & kAbsM) {
                mstore<NV, VEC>(M.Y + (size_t)s_io[4 * lane + j] * M.ldy + q0, q0, M.k, s);
                s = mzero<NV>();
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void mcp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}

// the low halves of a tile's nrows + 1 row offsets into soff (one group per
// item and lane, empty for a long row)
__device__ __forceinline__ void multi_prefetch(const int64_t *__restrict__ offset, const MultiItem &d,
                                               bool live, uint32_t *soff, int lane) {
    if (live && d.meta >= 0) {
        const int nrows = d.meta >> 16;
        for (int kk = lane; kk <= nrows; kk += 32) mcp_async4(soff + kk, offset + d.r0 + kk);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ uint4 multi_first_words(const uint32_t *__restrict__ pack,
                                                   const MultiItem &d, int lane) {
    const long long a0 = d.base & ~3ll;
    const int nwd = d.meta < 0 ? -d.meta : (d.meta & 0xFFFF);
    return mload_words(pack, a0, (int)(d.base - a0) + nwd, lane);
}

// Persistent grid: warp w takes items w, w + W, ...; the next item's words
// and row offsets load while the current item is processed. A batch item's
// matrix descriptor is read when the warp takes the item (an L1 hit after
// the first item of that matrix).
template <int NV, bool VEC, bool SINGLE>
__global__ void __launch_bounds__(MW * 32)
    k_split_multi(SplitMat M0, const SplitMat *__restrict__ mats,
                  const MultiItem *__restrict__ items, int nitems) {
    __shared__ __align__(16) uint32_t s_lft[MW][MT];
    __shared__ __align__(16) int s_io[MW][MT];
    __shared__ __align__(16) uint32_t s_off[MW][2][MR_MAX + 4];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int it = gw;
    if (it >= nitems) return;
    MultiItem d = items[it];
    {
        const uint32_t *pk = SINGLE ? M0.pack : mats[d.mat].pack;
        const int64_t *of = SINGLE ? M0.offset : mats[d.mat].offset;
        const uint4 w0 = multi_first_words(pk, d, lane);
        multi_prefetch(of, d, true, s_off[wl][0], lane);
        uint4 wv = w0;  // the first item's words
        int buf = 0;
        for (; it < nitems; it += nwarps) {
            const bool has_next = it + nwarps < nitems;
            MultiItem dn{0, 0, 0, 0, 0, 0, 0};
            uint4 wn = make_uint4(0, 0, 0, 0);
            if (has_next) {
                dn = items[it + nwarps];
                const uint32_t *pn = SINGLE ? M0.pack : mats[dn.mat].pack;
                wn = multi_first_words(pn, dn, lane);
                multi_prefetch(SINGLE ? M0.offset : mats[dn.mat].offset, dn, true,
                               s_off[wl][buf ^ 1], lane);
            } else {
                multi_prefetch(nullptr, dn, false, s_off[wl][buf ^ 1], lane);
            }
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncwarp();
            const SplitMat M = SINGLE ? M0 : mats[d.mat];
            if (d.meta < 0)
                multi_long_row<NV, VEC>(M, d.r0, d.base, -d.meta, lane);
            else
                multi_tile<NV, VEC>(M, d.r0, d.meta >> 16, d.base, d.meta & 0xFFFF, lane, wv,
                                    s_lft[wl], s_io[wl], s_off[wl][buf]);
            __syncwarp();
            d = dn;
            wv = wn;
            buf ^= 1;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ---- k > 16 with 16-byte X and Y rows: words walked from a decoded table ----
// The segmented sums above re-run every scan once per group of four columns,
// and each of their gather instructions touches 32 rows of X. For wider k a
// warp decodes the item's words once into a table in shared memory (column,
// or -1 for a word without a value; value; the y row where a row starts) and
// then multiplies from it: lane (cg, h), cg = lane % KG, h = lane / KG, owns
// NQ groups of four columns, 4 cg + 4 KG i (i < NQ), of a pass of 4 KG NQ
// columns, and the RPI = 32 / KG lane groups split the tile's words into
// runs of about equal length that begin at row starts. A group walks its run
// in stored order from +0 per row, so every row of a tile gets the same fused
// multiply-adds as the thread-per-row SpMV (the same bits); one gather
// instruction fetches RPI rows of X, 16 KG contiguous bytes each. A long row
// is decoded chunk by chunk into the table; group h takes the chunk's words
// h, h + RPI, ..., and the groups' sums are added by a butterfly (a fixed
// tree: within gamma_w).
template <int NQ>
struct RowAcc {
    float4 t[NQ];
};

template <int KG, int NQ, int U>
__device__ __forceinline__ void rows_step(const SplitMat &M, const int2 (&e)[U], int qb, int cg,
                                          RowAcc<NQ> &a) {
    float4 xv[U][NQ];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int q = qb + 4 * cg + 4 * KG * i;
            if (e[u].x >= 0 && q < M.k)
                xv[u][i] = __ldg(reinterpret_cast<const float4 *>(M.X + (size_t)e[u].x * M.ldx + q));
        }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const float v = __int_as_float(e[u].y);
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int q = qb + 4 * cg + 4 * KG * i;
            if (e[u].x >= 0 && q < M.k) {
                a.t[i].x = fmaf(v, xv[u][i].x, a.t[i].x);
                a.t[i].y = fmaf(v, xv[u][i].y, a.t[i].y);
                a.t[i].z = fmaf(v, xv[u][i].z, a.t[i].z);
                a.t[i].w = fmaf(v, xv[u][i].w, a.t[i].w);
            }
        }
    }
}

template <int NQ>
__device__ __forceinline__ void rows_zero(RowAcc<NQ> &a) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) a.t[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <int KG, int NQ>
__device__ __forceinline__ void rows_store(const SplitMat &M, float *__restrict__ yr, int qb, int cg,
                                           const RowAcc<NQ> &a) {
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const int q = qb + 4 * cg + 4 * KG * i;
        if (q < M.k) *reinterpret_cast<float4 *>(yr + q) = a.t[i];
    }
}

// words of a round per lane group: four gathers in flight per lane
template <int NQ>
constexpr int rows_round() {
    return NQ >= 4 ? 1 : 4 / NQ;
}

// A tile: the words are split into RPI runs of about nwd / RPI words, each
// moved forward to the next row start, so that every row lies in one run;
// lane group h walks run h in stored order, U words (their gathers issued
// together) at a time, and writes a row's sums when the next row starts.
template <int KG, int NQ>
__device__ __forceinline__ void rows_tile(const SplitMat &M, int r0, int nrows, long long base,
                                          int nwd, int lane, const uint4 &wv,
                                          uint32_t *__restrict__ s_lft, int *__restrict__ s_io,
                                          int4 *__restrict__ s_tab, const uint32_t *__restrict__ soff) {
    constexpr int RPI = 32 / KG, U = rows_round<NQ>();
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0);
    const uint32_t a0lo = (uint32_t)a0;
    reinterpret_cast<uint4 *>(s_lft)[lane] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    // row starts: kAbs | left offset and the y row; an empty row's y is zeroed here
    for (int kk = lane; kk < nrows; kk += 32) {
        const int r = r0 + kk;
        const uint32_t o0 = soff[kk], o1 = soff[kk + 1];
        const int io = mout(M, r);
        if (o1 != o0) {
            const int pos = (int)(o0 - a0lo);
            s_lft[pos] = kAbsM | (uint32_t)mleft(r, M.sigma, M.sig_shift, M.kl);
            s_io[pos] = io;
        } else {
            for (int q = 0; q < M.k; q += 4)
                *reinterpret_cast<float4 *>(M.Y + (size_t)io * M.ldy + q) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    __syncwarp();
    const uint4 hv = reinterpret_cast<const uint4 *>(s_lft)[lane];
    const uint32_t hl[4] = {hv.x, hv.y, hv.z, hv.w};
    uint32_t wd[4] = {wv.x, wv.y, wv.z, wv.w}, cs[4], acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int p = 4 * lane + j;
        if ((unsigned)(p - lead) >= (unsigned)nwd) wd[j] = 0u;
        acc = mcomb(acc, hl[j] + mdelta(M, wd[j]));
        cs[j] = acc;
    }
    uint32_t inc = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = mcomb(v, inc);
    }
    uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = 0u;  // the tile's first word starts a row
    // table entry: column (-1: no value), value bits, y row at a row start (-1 elsewhere)
    unsigned hb[4];  // hb[j] bit l: position 4 l + j starts a row
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t col = mcomb(exc, cs[j]) & ~kAbsM;
        const bool ok = (wd[j] & 1u) && PS_IN_RANGE(col, M.xlen);
        const bool head = (hl[j] & kAbsM) != 0u;
        hb[j] = __ballot_sync(0xffffffffu, head);
        s_tab[4 * lane + j] = make_int4(ok ? (int)col : -1, ok ? __float_as_int(mvalue(M, wd[j])) : 0,
                                        head ? s_io[4 * lane + j] : -1, 0);
    }
    __syncwarp();
    // this group's run [S, E): from the first row start at or after its share
    const int cg = lane % KG, h = lane / KG;
    const int end = lead + nwd;
    auto first_start = [&](int T) {
        int best = MT;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int lmin = max(0, (T - j + 3) >> 2);
            const unsigned m = lmin >= 32 ? 0u : (hb[j] & (0xffffffffu << lmin));
            if (m) best = min(best, 4 * (__ffs(m) - 1) + j);
        }
        return min(best, end);
    };
    const int S = first_start(lead + (h * nwd) / RPI);
    const int E = h == RPI - 1 ? end : first_start(lead + ((h + 1) * nwd) / RPI);
    for (int qb = 0; qb < M.k; qb += 4 * KG * NQ) {
        RowAcc<NQ> a;
        rows_zero(a);
        int yrow = -1;
        for (int p = S; p < E; p += U) {
            int4 e[U];
            float4 xv[U][NQ];
#pragma unroll
            for (int u = 0; u < U; ++u) e[u] = p + u < E ? s_tab[p + u] : make_int4(-1, 0, -1, 0);
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int i = 0; i < NQ; ++i) {
                    const int q = qb + 4 * cg + 4 * KG * i;
                    if (e[u].x >= 0 && q < M.k)
                        xv[u][i] = __ldg(reinterpret_cast<const float4 *>(M.X + (size_t)e[u].x * M.ldx + q));
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (e[u].z >= 0) {  // a row starts: the previous one is complete
                    if (yrow >= 0) rows_store<KG, NQ>(M, M.Y + (size_t)yrow * M.ldy, qb, cg, a);
                    rows_zero(a);
                    yrow = e[u].z;
                }
                const float v = __int_as_float(e[u].y);
#pragma unroll
                for (int i = 0; i < NQ; ++i) {
                    const int q = qb + 4 * cg + 4 * KG * i;
                    if (e[u].x >= 0 && q < M.k) {
                        a.t[i].x = fmaf(v, xv[u][i].x, a.t[i].x);
                        a.t[i].y = fmaf(v, xv[u][i].y, a.t[i].y);
                        a.t[i].z = fmaf(v, xv[u][i].z, a.t[i].z);
                        a.t[i].w = fmaf(v, xv[u][i].w, a.t[i].w);
                    }
                }
            }
        }
        if (yrow >= 0) rows_store<KG, NQ>(M, M.Y + (size_t)yrow * M.ldy, qb, cg, a);
    }
    __syncwarp();
}

template <int KG, int NQ>
__device__ __forceinline__ void rows_long(const SplitMat &M, int row, long long base, int nwd,
                                          int lane, int4 *__restrict__ s_tab) {
    constexpr int RPI = 32 / KG, U = rows_round<NQ>();
    static_assert(MT % (U * RPI) == 0, "a chunk splits evenly over the lane groups");
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0), lim = lead + nwd;
    const int io = mout(M, row);
    const uint32_t c0 = (uint32_t)mleft(row, M.sigma, M.sig_shift, M.kl);
    const int cg = lane % KG, h = lane / KG;
    for (int qb = 0; qb < M.k; qb += 4 * KG * NQ) {  // the same trip count in every lane
        uint32_t carry = c0;
        RowAcc<NQ> a;
        rows_zero(a);
        uint4 cur = mload_words(M.pack, a0, lim, lane);
        for (int k0 = 0; k0 < lim; k0 += MT) {
            const uint4 nxt = mload_words(M.pack, a0 + k0 + MT, lim - k0 - MT, lane);
            uint32_t wd[4] = {cur.x, cur.y, cur.z, cur.w}, cs[4], acc = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = k0 + 4 * lane + j;
                if ((unsigned)(p - lead) >= (unsigned)nwd) wd[j] = 0u;
                acc += mdelta(M, wd[j]);
                cs[j] = acc;
            }
            uint32_t inc = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += v;
            }
            const uint32_t before = carry + inc - acc;
            carry += __shfl_sync(0xffffffffu, inc, 31);
            int2 e4[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t col = before + cs[j];
                const bool ok = (wd[j] & 1u) && PS_IN_RANGE(col, M.xlen);
                e4[j] = ok ? make_int2((int)col, __float_as_int(mvalue(M, wd[j]))) : make_int2(-1, 0);
            }
            __syncwarp();  // the previous chunk's table reads are done
#pragma unroll
            for (int j = 0; j < 4; ++j) s_tab[4 * lane + j] = make_int4(e4[j].x, e4[j].y, -1, 0);
            __syncwarp();
            for (int p = h; p < MT; p += U * RPI) {
                int2 e[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int4 t = s_tab[p + u * RPI];
                    e[u] = make_int2(t.x, t.y);
                }
                rows_step<KG, NQ, U>(M, e, qb, cg, a);
            }
            cur = nxt;
        }
#pragma unroll
        for (int o = KG; o < 32; o <<= 1) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                a.t[i].x += __shfl_xor_sync(0xffffffffu, a.t[i].x, o);
                a.t[i].y += __shfl_xor_sync(0xffffffffu, a.t[i].y, o);
                a.t[i].z += __shfl_xor_sync(0xffffffffu, a.t[i].z, o);
                a.t[i].w += __shfl_xor_sync(0xffffffffu, a.t[i].w, o);
            }
        }
        if (h == 0) rows_store<KG, NQ>(M, M.Y + (size_t)io * M.ldy, qb, cg, a);
    }
}

// Persistent grid over the same items as k_split_multi, the next item's words
// and row offsets loading while the current one is processed.
template <int KG, int NQ, bool SINGLE>
__global__ void __launch_bounds__(MW * 32, SINGLE ? 3 : 2)
    k_split_rows(SplitMat M0, const SplitMat *__restrict__ mats, const MultiItem *__restrict__ items,
                 int nitems) {
    __shared__ __align__(16) uint32_t s_lft[MW][MT];
    __shared__ __align__(16) int s_io[MW][MT];
    __shared__ __align__(16) int4 s_tab[MW][MT];
    __shared__ __align__(16) uint32_t s_off[MW][2][MR_MAX + 4];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int it = gw;
    if (it >= nitems) return;
    MultiItem d = items[it];
    {
        const uint32_t *pk = SINGLE ? M0.pack : mats[d.mat].pack;
        const int64_t *of = SINGLE ? M0.offset : mats[d.mat].offset;
        uint4 wv = multi_first_words(pk, d, lane);
        multi_prefetch(of, d, true, s_off[wl][0], lane);
        int buf = 0;
        for (; it < nitems; it += nwarps) {
            const bool has_next = it + nwarps < nitems;
            MultiItem dn{0, 0, 0, 0, 0, 0, 0};
            uint4 wn = make_uint4(0, 0, 0, 0);
            if (has_next) {
                dn = items[it + nwarps];
                const uint32_t *pn = SINGLE ? M0.pack : mats[dn.mat].pack;
                wn = multi_first_words(pn, dn, lane);
                multi_prefetch(SINGLE ? M0.offset : mats[dn.mat].offset, dn, true,
                               s_off[wl][buf ^ 1], lane);
            } else {
                multi_prefetch(nullptr, dn, false, s_off[wl][buf ^ 1], lane);
            }
            asm volatile("cp.async.wait_group 1;" ::: "memory");
            __syncwarp();
            const SplitMat M = SINGLE ? M0 : mats[d.mat];
            if (d.meta < 0)
                rows_long<KG, NQ>(M, d.r0, d.base, -d.meta, lane, s_tab[wl]);
            else
                rows_tile<KG, NQ>(M, d.r0, d.meta >> 16, d.base, d.meta & 0xFFFF, lane, wv,
                                  s_lft[wl], s_io[wl], s_tab[wl], s_off[wl][buf]);
            __syncwarp();
            d = dn;
            wv = wn;
            buf ^= 1;
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

template <int KG, int NQ, bool SINGLE>
packsell_status launch_rows_t(const SplitMat &single, const SplitMat *mats, const MultiItem *items,
                              int nitems, cudaStream_t s) {
    static std::atomic<int> cached{0};
    int blocks = cached.load(std::memory_order_relaxed);
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_split_rows<KG, NQ, SINGLE>, MW * 32,
                                                          0) != cudaSuccess)
            return fail(PACKSELL_ERR_CUDA, "split-row product: device query failed");
        blocks = sms * std::max(per, 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    blocks = std::min(blocks, (nitems + MW - 1) / MW);
    k_split_rows<KG, NQ, SINGLE><<<blocks, MW * 32, 0, s>>>(single, mats, items, nitems);
    PS_LAUNCH_CHECK("split-row product");
    return PACKSELL_OK;
}

template <bool SINGLE>
packsell_status launch_rows(const SplitMat &single, const SplitMat *mats, const MultiItem *items,
                            int nitems, int k, cudaStream_t s) {
    // eight lanes per row group (four row groups per warp): one column group
    // per lane up to k = 32, two above (passes of 64 columns)
    if (k <= 32) return launch_rows_t<8, 1, SINGLE>(single, mats, items, nitems, s);
    return launch_rows_t<8, 2, SINGLE>(single, mats, items, nitems, s);
}

template <int NV, bool VEC, bool SINGLE>
int multi_blocks() {
    static std::atomic<int> cached{0};
    int blocks = cached.load(std::memory_order_relaxed);
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_split_multi<NV, VEC, SINGLE>, MW * 32,
                                                          0) != cudaSuccess)
            return 0;
        blocks = sms * std::max(per, 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    return blocks;
}

template <int NV, bool VEC, bool SINGLE>
packsell_status launch_multi_t(const SplitMat &single, const SplitMat *mats, const MultiItem *items,
                               int nitems, cudaStream_t s) {
    int blocks = multi_blocks<NV, VEC, SINGLE>();
    if (!blocks) return fail(PACKSELL_ERR_CUDA, "split-row product: device query failed");
    blocks = std::min(blocks, (nitems + MW - 1) / MW);
    k_split_multi<NV, VEC, SINGLE><<<blocks, MW * 32, 0, s>>>(single, mats, items, nitems);
    PS_LAUNCH_CHECK("split-row product");
    return PACKSELL_OK;
}

}  // namespace

SplitMat split_mat(const Matrix &A, const float *X, int64_t ldx, float *Y, int64_t ldy, int k) {
    SplitMat M{};
    M.pack = A.pack;
    M.offset = A.offset;
    M.perm = A.p.explicit_perm ? nullptr : A.perm;
    M.perm_bytes = A.p.explicit_perm ? 0 : A.perm_bytes;
    M.X = X;
    M.Y = Y;
    M.ldx = ldx;
    M.ldy = ldy;
    M.k = k;
    M.sigma = A.p.sigma;
    M.sig_shift = (A.p.sigma & (A.p.sigma - 1)) == 0 ? __builtin_ctz((unsigned)A.p.sigma) : -1;
    M.kl = (int)std::min<int64_t>(A.p.k_left, INT32_MAX);
    M.fmt = A.p.format;
    M.dmask = (1u << A.p.D) - 1u;
    M.xlen = (int)A.m;
    M.vmask = ~((2u << A.p.D) - 1u);
    return M;
}

// Items of one C = 1 matrix from its host row offsets: consecutive rows of at
// most MCT words grouped while they hold at most MCT words and MR_MAX rows;
// a row of more words is an item of its own.
void multi_items_append(const int64_t *off, int64_t n, int mat, std::vector<MultiItem> &items) {
    auto tile = [&](int a, int b) {
        items.push_back(MultiItem{(long long)off[a], a, ((b - a) << 16) | (int)(off[b] - off[a]), mat,
                                  0, 0, 0});
    };
    int r0 = 0;
    for (int r = 0; r < (int)n; ++r) {
        const int64_t w = off[r + 1] - off[r];
        if (w > MCT) {
            if (r > r0) tile(r0, r);
            items.push_back(MultiItem{(long long)off[r], r, -(int)std::min<int64_t>(w, INT32_MAX), mat,
                                      0, 0, 0});
            r0 = r + 1;
            continue;
        }
        if (off[r + 1] - off[r0] > MCT || r + 1 - r0 > MR_MAX) {
            tile(r0, r);
            r0 = r;
        }
    }
    if ((int)n > r0) tile(r0, (int)n);
}

// long rows first, longest first (the longest serial paths start first)
void multi_items_order(std::vector<MultiItem> &items) {
    auto is_long = [](const MultiItem &a) { return a.meta < 0; };
    std::stable_partition(items.begin(), items.end(), is_long);
    const size_t nlong = (size_t)std::count_if(items.begin(), items.end(), is_long);
    std::stable_sort(items.begin(), items.begin() + nlong,
                     [](const MultiItem &a, const MultiItem &b) { return a.meta < b.meta; });
}

void multi_plan_free(Matrix &A) {
    cudaFree(A.multi_items);
    A.multi_items = nullptr;
    A.multi_nitems = 0;
}

packsell_status multi_plan(Matrix &A, cudaStream_t s) {
    multi_plan_free(A);
    if (!is_packed(A.p.format) || A.p.C != 1 || A.n == 0) return PACKSELL_OK;
    std::vector<int64_t> off((size_t)A.n + 1);
    PS_CUDA(cudaMemcpyAsync(off.data(), A.offset, sizeof(int64_t) * (A.n + 1),
                            cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    std::vector<MultiItem> items;
    items.reserve((size_t)(A.n_words / MCT + A.n / MR_MAX + 16));
    multi_items_append(off.data(), A.n, 0, items);
    multi_items_order(items);
    if (items.size() >= (size_t)INT32_MAX) return fail(PACKSELL_ERR_RANGE, "multi_plan: too many items");
    PS_CUDA(cudaMalloc(&A.multi_items, sizeof(MultiItem) * items.size()));
    PS_CUDA(cudaMemcpy(A.multi_items, items.data(), sizeof(MultiItem) * items.size(),
                       cudaMemcpyHostToDevice));
    A.multi_nitems = (int)items.size();
    return PACKSELL_OK;
}

packsell_status launch_multi(const SplitMat &single, const SplitMat *mats, const MultiItem *items,
                             int nitems, int k, bool vec, cudaStream_t s) {
    if (nitems <= 0) return PACKSELL_OK;
    const bool one = mats == nullptr;
    if (k == 1)
        return one ? launch_multi_t<1, false, true>(single, mats, items, nitems, s)
                   : launch_multi_t<1, false, false>(single, mats, items, nitems, s);
    if (vec && k > 16)  // words walked from a decoded table
        return one ? launch_rows<true>(single, mats, items, nitems, k, s)
                   : launch_rows<false>(single, mats, items, nitems, k, s);
    if (vec)
        return one ? launch_multi_t<4, true, true>(single, mats, items, nitems, s)
                   : launch_multi_t<4, true, false>(single, mats, items, nitems, s);
    return one ? launch_multi_t<4, false, true>(single, mats, items, nitems, s)
               : launch_multi_t<4, false, false>(single, mats, items, nitems, s);
}

}  // namespace packsell
