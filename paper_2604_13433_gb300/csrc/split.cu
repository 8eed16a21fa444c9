// Split-row SpMV over delta-value packing in CSR order (SpMV variant 14).
//
// A PackSELL matrix with slice height C = 1 stores each row's words one after
// another with no padding, and its slice offsets are the row pointer: the
// CSR-based form of the packing that the paper leaves as future work for
// matrices whose rows vary too much for SELL slices (§5.1.1, §7). Variant 11
// sums every row on one lane, in stored order; on power-law rows that leaves
// most lanes idle. Here all 32 lanes of a warp share the words of a tile of
// rows, whatever the row lengths:
//  * at encode time the rows are cut into items: tiles of consecutive rows of
//    at most ST - 3 words and SR_MAX rows, and single rows of more words;
//  * a warp loads a tile's words (aligned down to 16 bytes) with 16-byte
//    loads: in round u lane l holds the words at 128u + 4l .. 128u + 4l + 3;
//  * the row starts of the tile are marked in shared memory (the storage row
//    at the position of its first word, -1 elsewhere);
//  * the column of each word (Eq. 2 from the left offset of Eq. 4) is a
//    segmented prefix sum of the deltas that restarts at every row start:
//    serial over a lane's four words, then a warp scan over the lanes, then
//    carried from round to round;
//  * every word with a value gathers its x and multiplies; the products are
//    summed per row by a segmented suffix sum (serial in the lane, then across
//    lanes) whose total lands on the row's first word, and that lane writes
//    y for the row;
//  * a long row is walked ST words at a time with the column carried from
//    chunk to chunk; every lane sums its own words and a butterfly reduction
//    gives the row's total.
// The summation order is fixed, so the result is the same bits on every run,
// but it is a tree rather than the stored-order chain of fused multiply-adds:
// the rows are held to the forward error bound gamma_w * sum_j |a_ij x_j|
// (w stored words of the row), not to the thread-per-row kernels' bits.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int ST = 256;       // words a warp holds per chunk: 8 consecutive words per lane
constexpr int SCT = ST - 3;   // tile words at most (room for the aligned-down start)
constexpr int SR_MAX = 256;   // tile rows at most
constexpr int SW = 8;         // warps per block
constexpr uint32_t kAbs = 0x80000000u;  // column scan: the value is an absolute column

// Column scan operator on (absolute?, value) packed in one word: a later
// absolute column replaces what came before, a later relative delta adds to
// it (b + (a masked off when b is absolute)). Columns and their partial sums
// stay below 2^31.
__device__ __forceinline__ uint32_t col_comb(uint32_t a, uint32_t b) {
    return b + (a & ~(uint32_t)((int32_t)b >> 31));
}

// Left offset of Eq. 4 for a row (kl = k_left, at most 2^31 - 1 here: a
// larger k_left gives 0 for every row below 2^31).
__device__ __forceinline__ int split_left(int row, int sigma, int sig_shift, int kl) {
    const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
    return max(blk - kl, 0);
}

// Where row `row`'s product goes in y (through the sigma permutation when
// y is in the original order).
template <bool PERM>
__device__ __forceinline__ int split_out(int row, int sigma, int sig_shift, const void *perm,
                                         int perm_bytes) {
    if (!PERM || perm_bytes == 0) return row;
    const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
    return blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[row]
                                  : (int)((const uint16_t *)perm)[row]);
}

__device__ __forceinline__ uint4 ld_words4(const uint32_t *p) {
    return __ldcs(reinterpret_cast<const uint4 *>(p));
}

// FMT 0: the format is chosen at run time (a batch): FP16 when dc.vshift is 1
template <int FMT>
__device__ __forceinline__ float split_value(uint32_t wd, Decode dc) {
    const bool h = FMT == PACKSELL_FMT_FP16 || (FMT == 0 && dc.vshift != 0);
    if (FMT == PACKSELL_FMT_FP16) return __high2float(*reinterpret_cast<const __half2 *>(&wd));
    if (FMT == 0 && h) return __high2float(*reinterpret_cast<const __half2 *>(&wd));
    return __uint_as_float(wd & dc.vmask);
}

// delta of a word: D bits when it carries a value, 31 bits otherwise
__device__ __forceinline__ uint32_t split_delta(uint32_t wd, Decode dc) {
    return (wd >> 1) & ((wd & 1u) ? dc.dmask : 0x7fffffffu);
}

// Work item: a tile of rows [r0, r0 + nrows) holding nwd words from word
// `base` (meta = nrows << 16 | nwd), or one long row of nwd words (meta =
// -nwd). One 16-byte load gives a warp everything it needs to start.
struct __align__(16) SplitItem {
    long long base;
    int r0;
    int meta;
};

// ST words from `first` (a multiple of 4): lane l holds the 8 consecutive
// words first + 8l .. first + 8l + 7 (0 from `lim` on).
__device__ __forceinline__ void split_load(const uint32_t *__restrict__ pack, long long first,
                                           int lim, int lane, uint4 (&wv)[2]) {
    const int p = 8 * lane;
    wv[0] = p < lim ? ld_words4(pack + first + p) : make_uint4(0, 0, 0, 0);
    wv[1] = p + 4 < lim ? ld_words4(pack + first + p + 4) : make_uint4(0, 0, 0, 0);
}

template <typename Item>
__device__ __forceinline__ void split_load_item(const uint32_t *__restrict__ pack,
                                                const Item &d, int lane, uint4 (&wv)[2]) {
    const long long a0 = d.base & ~3ll;
    const int nwd = d.meta < 0 ? -d.meta : (d.meta & 0xFFFF);
    split_load(pack, a0, (int)(d.base - a0) + nwd, lane, wv);
}

__device__ __forceinline__ void unpack8(const uint4 (&wv)[2], uint32_t (&w)[8]) {
    w[0] = wv[0].x; w[1] = wv[0].y; w[2] = wv[0].z; w[3] = wv[0].w;
    w[4] = wv[1].x; w[5] = wv[1].y; w[6] = wv[1].z; w[7] = wv[1].w;
}

// One row of more than SCT words: chunks of ST words (the first one already
// loaded into cur), each lane summing its own words, the column carried
// across chunks; the next chunk's words load while the current one is
// decoded and gathered.
template <int FMT, bool PERM>
__device__ __forceinline__ void split_long_row(int row, long long base, int nwd, int sigma,
                                               int sig_shift, int k_left,
                                               const uint32_t *__restrict__ pack,
                                               const void *__restrict__ perm, int perm_bytes,
                                               Decode dc, const float *__restrict__ x,
                                               float *__restrict__ y, int lane, uint4 (&cur)[2]) {
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0), lim = lead + nwd;
    uint32_t carry = (uint32_t)split_left(row, sigma, sig_shift, k_left);
    float t = 0.f;
    for (int k0 = 0; k0 < lim; k0 += ST) {
        uint4 nxt[2];
        split_load(pack, a0 + k0 + ST, lim - k0 - ST, lane, nxt);
        uint32_t wd[8], cs[8], acc = 0;
        unpack8(cur, wd);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int p = k0 + 8 * lane + j;
            if ((unsigned)(p - lead) >= (unsigned)nwd) wd[j] = 0u;
            acc += split_delta(wd[j], dc);
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
        float xv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j)
            xv[j] = ((wd[j] & 1u) && PS_IN_RANGE(before + cs[j], dc.xlen)) ? __ldg(x + (before + cs[j]))
                                                                             : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (wd[j] & 1u) t = fmaf(split_value<FMT>(wd[j], dc), xv[j], t);
        cur[0] = nxt[0];
        cur[1] = nxt[1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) y[split_out<PERM>(row, sigma, sig_shift, perm, perm_bytes)] = t;
}

// A tile of rows [r0, r0 + nrows) with its nwd (<= SCT) words in wv. For
// each position of the tile, s_lft holds kAbs | (left offset of Eq. 4) where
// a row starts and 0 elsewhere, and s_io the row's index in y where a row
// starts: both are computed once per row, not once per word.
template <int FMT, bool PERM>
__device__ __forceinline__ void split_tile(int r0, int nrows, long long base, int nwd, int sigma,
                                           int sig_shift, int k_left,
                                           const void *__restrict__ perm, int perm_bytes,
                                           Decode dc, const float *__restrict__ x,
                                           float *__restrict__ y, int lane, const uint4 (&wv)[2],
                                           uint32_t *__restrict__ s_lft, int *__restrict__ s_io,
                                           const uint32_t *__restrict__ soff) {
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0);
    uint4 *lft4 = reinterpret_cast<uint4 *>(s_lft);
    lft4[2 * lane] = make_uint4(0, 0, 0, 0);
    lft4[2 * lane + 1] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    // mark where each row starts (the low halves of the tile's offsets were
    // copied to soff one item ahead: differences within a tile are below 2^8,
    // so they are exact modulo 2^32); an empty row's product is 0
    const uint32_t a0lo = (uint32_t)a0;
    for (int k = lane; k < nrows; k += 32) {
        const int r = r0 + k;
        const uint32_t o0 = soff[k], o1 = soff[k + 1];
        const int io = split_out<PERM>(r, sigma, sig_shift, perm, perm_bytes);
        if (o1 != o0) {
            const int pos = (int)(o0 - a0lo);
            s_lft[pos] = kAbs | (uint32_t)split_left(r, sigma, sig_shift, k_left);
            s_io[pos] = io;
        } else {
            y[io] = 0.f;
        }
    }
    __syncwarp();
    uint32_t hl[8], wd[8], cs[8], acc = 0;
    {
        const uint4 l0 = lft4[2 * lane], l1 = lft4[2 * lane + 1];
        hl[0] = l0.x; hl[1] = l0.y; hl[2] = l0.z; hl[3] = l0.w;
        hl[4] = l1.x; hl[5] = l1.y; hl[6] = l1.z; hl[7] = l1.w;
    }
    unpack8(wv, wd);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int p = 8 * lane + j;
        if ((unsigned)(p - lead) >= (unsigned)nwd) wd[j] = 0u;
        acc = col_comb(acc, hl[j] + split_delta(wd[j], dc));  // a row start: kAbs | left + d
        cs[j] = acc;
    }
    uint32_t inc = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc = col_comb(v, inc);
    }
    uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = 0u;  // the tile's first word starts a row
    // every valid word's column is now absolute (the tile's first word starts
    // a row): the flag bit is folded into the base pointer
    const float *__restrict__ xb = x - (size_t)kAbs;
    float pv[8];  // value * x of every word (0 without a value)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float xv = ((wd[j] & 1u) && PS_IN_RANGE(col_comb(exc, cs[j]) - kAbs, dc.xlen))
                             ? __ldg(xb + col_comb(exc, cs[j]))
                             : 0.f;
        pv[j] = (wd[j] & 1u) ? split_value<FMT>(wd[j], dc) * xv : 0.f;
    }
    // segmented suffix sums. A: the lane's words before its first row start
    uint32_t hm = 0;  // row starts among the lane's words
#pragma unroll
    for (int j = 0; j < 8; ++j) hm |= (hl[j] >> 31) << j;
    const int fh = hm ? __ffs(hm) - 1 : 8;
    float A = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (j < fh) A += pv[j];
    // U: A plus, while no row start intervenes, the same of the lanes after it
    const unsigned heads = __ballot_sync(0xffffffffu, hm != 0u);
    float U = A;
    bool F = hm != 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float v = __shfl_down_sync(0xffffffffu, U, o);
        if (lane + o < 32 && !F) {
            U += v;
            // heads in lanes lane + o .. lane + 2o - 1 end the run
            F = ((heads >> (lane + o)) & ((1u << o) - 1u)) != 0u;
        }
    }
    float s = __shfl_down_sync(0xffffffffu, U, 1);
    if (lane == 31) s = 0.f;
    // from the lane's end backwards: what flows in from the later lanes, then
    // each word; a row start closes its row's sum
#pragma unroll
    for (int j = 7; j >= 0; --j) {
        s += pv[j];
        if (hl[j] & kAbs) {
            y[s_io[8 * lane + j]] = s;
            s = 0.f;
        }
    }
    __syncwarp();
}

// 4-byte asynchronous global -> shared copies (cp.async), in groups
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_older() {
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // all but the newest group done
}

// Start copying the low 32 bits of a tile's nrows + 1 row offsets (int64,
// little-endian) into soff; every lane commits one group per item (empty for
// a long row) so the group counts stay equal.
template <typename Item>
__device__ __forceinline__ void split_prefetch_offsets(const Item &d, bool live,
                                                       const int64_t *__restrict__ offset,
                                                       uint32_t *soff, int lane) {
    if (live && d.meta >= 0) {
        const int nrows = d.meta >> 16;
        for (int k = lane; k <= nrows; k += 32) cp_async4(soff + k, offset + d.r0 + k);
    }
    cp_async_commit();
}

// Persistent grid: warp w takes items w, w + W, w + 2W, ... in a two-deep
// pipeline: while item k is processed, item k + 1's words (registers) and row
// offsets (shared memory, cp.async) are in flight, and item k + 2's
// descriptor; so a warp waits on one memory round trip (its gathers) per
// item rather than on the whole chain descriptor -> offsets -> words -> x.
template <int FMT, bool PERM>
__global__ void __launch_bounds__(SW * 32, 4)
    k_spmv_split(int sigma, int sig_shift, int k_left, const int64_t *__restrict__ offset,
                 const uint32_t *__restrict__ pack, const void *__restrict__ perm, int perm_bytes,
                 Decode dc, const SplitItem *__restrict__ items, int nitems,
                 const float *__restrict__ x, float *__restrict__ y) {
    __shared__ __align__(16) uint32_t s_lft[SW][ST];             // kAbs | left at row starts
    __shared__ __align__(16) int s_io[SW][ST];                   // y index at row starts
    __shared__ __align__(16) uint32_t s_off[SW][2][SR_MAX + 4];  // tile row offsets (low halves), two items
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int it = gw;
    if (it >= nitems) return;
    SplitItem d = items[it], dn{0, 0, 0};
    if (it + nwarps < nitems) dn = items[it + nwarps];
    uint4 wv[2];
    split_load_item(pack, d, lane, wv);
    split_prefetch_offsets(d, true, offset, s_off[wl][0], lane);
    int buf = 0;
    for (; it < nitems; it += nwarps) {
        const bool has_next = it + nwarps < nitems;
        SplitItem dnn{0, 0, 0};
        if (it + 2 * nwarps < nitems) dnn = items[it + 2 * nwarps];
        uint4 wn[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        if (has_next) split_load_item(pack, dn, lane, wn);
        split_prefetch_offsets(dn, has_next, offset, s_off[wl][buf ^ 1], lane);
        cp_async_wait_older();  // this item's offsets have landed (this lane's copies)
        __syncwarp();           // ... and every other lane's
        if (d.meta < 0)
            split_long_row<FMT, PERM>(d.r0, d.base, -d.meta, sigma, sig_shift, k_left, pack, perm,
                                      perm_bytes, dc, x, y, lane, wv);
        else
            split_tile<FMT, PERM>(d.r0, d.meta >> 16, d.base, d.meta & 0xFFFF, sigma, sig_shift,
                                  k_left, perm, perm_bytes, dc, x, y, lane, wv, s_lft[wl],
                                  s_io[wl], s_off[wl][buf]);
        __syncwarp();  // every lane is done with s_off[buf] before it is refilled
        d = dn;
        dn = dnn;
        wv[0] = wn[0];
        wv[1] = wn[1];
        buf ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// The same kernel over many matrices (a batched SpMV of CSR-order matrices):
// each item names its matrix, whose descriptor gives the words, offsets,
// perm, vectors, left offset and value format. A matrix's items are cut by
// the same rule as its own plan's, so each y equals variant 14's on that
// matrix alone, bit for bit. SORTED = false: every matrix has sigma = 1 (no
// sort, no perm); SORTED = true takes any sigma. The per-item matrix
// parameters live in registers (the single-matrix kernel has them as launch
// arguments), so the kernel runs three blocks per SM: at four it spills.
template <bool SORTED>
__global__ void __launch_bounds__(SW * 32, 3)
    k_spmv_split_batch(const SplitMat *__restrict__ mats, const MultiItem *__restrict__ items,
                       int nitems) {
    __shared__ __align__(16) uint32_t s_lft[SW][ST];
    __shared__ __align__(16) int s_io[SW][ST];
    __shared__ __align__(16) uint32_t s_off[SW][2][SR_MAX + 4];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int it = gw;
    if (it >= nitems) return;
    MultiItem d = items[it], dn{0, 0, 0, 0};
    if (it + nwarps < nitems) dn = items[it + nwarps];
    uint4 wv[2];
    split_load_item(mats[d.mat].pack, d, lane, wv);
    split_prefetch_offsets(d, true, mats[d.mat].offset, s_off[wl][0], lane);
    int buf = 0;
    for (; it < nitems; it += nwarps) {
        const bool has_next = it + nwarps < nitems;
        MultiItem dnn{0, 0, 0, 0};
        if (it + 2 * nwarps < nitems) dnn = items[it + 2 * nwarps];
        uint4 wn[2] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
        const SplitMat *Mn = has_next ? &mats[dn.mat] : nullptr;
        if (has_next) split_load_item(Mn->pack, dn, lane, wn);
        split_prefetch_offsets(dn, has_next, has_next ? Mn->offset : nullptr, s_off[wl][buf ^ 1],
                               lane);
        cp_async_wait_older();
        __syncwarp();
        const SplitMat &M = mats[d.mat];
        const Decode dc{M.dmask, M.vmask, M.fmt == PACKSELL_FMT_FP16 ? 1 : 0, 1.f, M.xlen};
        const int sg = SORTED ? M.sigma : 1, sh = SORTED ? M.sig_shift : 0;
        if (d.meta < 0)
            split_long_row<0, SORTED>(d.r0, d.base, -d.meta, sg, sh, M.kl, M.pack, M.perm,
                                      M.perm_bytes, dc, M.X, M.Y, lane, wv);
        else
            split_tile<0, SORTED>(d.r0, d.meta >> 16, d.base, d.meta & 0xFFFF, sg, sh, M.kl,
                                  M.perm, M.perm_bytes, dc, M.X, M.Y, lane, wv, s_lft[wl],
                                  s_io[wl], s_off[wl][buf]);
        __syncwarp();
        d = dn;
        dn = dnn;
        wv[0] = wn[0];
        wv[1] = wn[1];
        buf ^= 1;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

template <bool SORTED>
int split_batch_blocks() {
    static std::atomic<int> cached{0};
    int blocks = cached.load(std::memory_order_relaxed);
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_spmv_split_batch<SORTED>, SW * 32, 0) !=
                cudaSuccess)
            return 0;
        blocks = sms * std::max(per, 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    return blocks;
}

template <int FMT, bool PERM>
int split_blocks() {
    // persistent grid: every block resident at once (cached per process)
    static std::atomic<int> cached{0};
    int blocks = cached.load(std::memory_order_relaxed);
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_spmv_split<FMT, PERM>, SW * 32,
                                                          0) != cudaSuccess)
            return 0;
        blocks = sms * std::max(per, 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    return blocks;
}

}  // namespace

void split_plan_free(Matrix &A) {
    cudaFree(A.split_items);
    A.split_items = nullptr;
    A.split_nitems = 0;
}

// Items of variant 14 (C = 1 PackSELL matrices), built on the host from the
// row offsets: consecutive rows of at most SCT words grouped greedily while
// the group holds at most SCT words and SR_MAX rows; a row of more words is
// an item of its own. Long rows come first, longest first: they are the
// longest serial paths of the launch and start before the short tiles.
// Cut rows [0, n) with row offsets `off` into items: consecutive rows of at
// most SCT words grouped greedily while the group holds at most SCT words and
// SR_MAX rows; a row of more words is an item of its own. push(base, r0,
// meta) receives each item in row order.
template <typename Push>
static packsell_status split_cut(const int64_t *off, int n, Push push) {
    auto tile = [&](int a, int b) {
        push((long long)off[a], a, ((b - a) << 16) | (int)(off[b] - off[a]));
    };
    int r0 = 0;
    for (int r = 0; r < n; ++r) {
        const int64_t w = off[r + 1] - off[r];
        if (w > SCT) {
            if (r > r0) tile(r0, r);
            if (w >= INT32_MAX) return fail(PACKSELL_ERR_RANGE, "split-row plan: row too long");
            push((long long)off[r], r, -(int)w);
            r0 = r + 1;
            continue;
        }
        if (off[r + 1] - off[r0] > SCT || r + 1 - r0 > SR_MAX) {
            tile(r0, r);
            r0 = r;
        }
    }
    if (n > r0) tile(r0, n);
    return PACKSELL_OK;
}

// Items of variant 14 (C = 1 PackSELL matrices), built on the host from the
// row offsets by split_cut. Long rows come first, longest first: they are the
// longest serial paths of the launch and start before the short tiles.
packsell_status plan_split(Matrix &A, cudaStream_t s) {
    split_plan_free(A);
    if (!is_packed(A.p.format) || A.p.C != 1 || A.n == 0) return PACKSELL_OK;
    std::vector<int64_t> off((size_t)A.n + 1);
    PS_CUDA(cudaMemcpyAsync(off.data(), A.offset, sizeof(int64_t) * (A.n + 1),
                            cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    std::vector<SplitItem> items;
    items.reserve((size_t)(A.n_words / SCT + A.n / SR_MAX + 16));
    const packsell_status st = split_cut(off.data(), (int)A.n, [&](long long b, int r0, int meta) {
        items.push_back(SplitItem{b, r0, meta});
    });
    if (st != PACKSELL_OK) return st;
    auto is_long = [](const SplitItem &a) { return a.meta < 0; };
    std::stable_partition(items.begin(), items.end(), is_long);
    const size_t nlong = (size_t)std::count_if(items.begin(), items.end(), is_long);
    std::stable_sort(items.begin(), items.begin() + nlong,
                     [](const SplitItem &a, const SplitItem &b) { return a.meta < b.meta; });
    if (items.size() >= (size_t)INT32_MAX)
        return fail(PACKSELL_ERR_RANGE, "plan_split: too many items");
    PS_CUDA(cudaMalloc(&A.split_items, sizeof(SplitItem) * items.size()));
    PS_CUDA(cudaMemcpyAsync(A.split_items, items.data(), sizeof(SplitItem) * items.size(),
                            cudaMemcpyHostToDevice, s));
    PS_CUDA(cudaStreamSynchronize(s));
    A.split_nitems = (int)items.size();
    return PACKSELL_OK;
}

// A batch's items of matrix `mat` (n rows, row offsets `off`), by the rule of
// the matrix's own plan; the caller orders the whole list (multi_items_order).
packsell_status split_items_append(const int64_t *off, int64_t n, int mat,
                                   std::vector<MultiItem> &items) {
    return split_cut(off, (int)n, [&](long long b, int r0, int meta) {
        items.push_back(MultiItem{b, r0, meta, mat});
    });
}

packsell_status launch_split_batch(const SplitMat *mats, const MultiItem *items, int nitems,
                                   bool sorted, cudaStream_t s) {
    if (nitems <= 0) return PACKSELL_OK;
    int blocks = sorted ? split_batch_blocks<true>() : split_batch_blocks<false>();
    if (!blocks) return fail(PACKSELL_ERR_CUDA, "packsell_batch_spmv: device query failed");
    blocks = std::min(blocks, (nitems + SW - 1) / SW);
    if (sorted) k_spmv_split_batch<true><<<blocks, SW * 32, 0, s>>>(mats, items, nitems);
    else k_spmv_split_batch<false><<<blocks, SW * 32, 0, s>>>(mats, items, nitems);
    PS_LAUNCH_CHECK("packsell_batch_spmv (split rows)");
    return PACKSELL_OK;
}

packsell_status launch_split(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                             cudaStream_t s) {
    if (!A.split_items)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_spmv: variant 14 needs a PackSELL matrix with C = 1");
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    const Decode dc = make_decode(A);
    const int kl = (int)std::min<int64_t>(A.p.k_left, INT32_MAX);
    const bool h = A.p.format == PACKSELL_FMT_FP16;
    const SplitItem *it = reinterpret_cast<const SplitItem *>(A.split_items);
    // a persistent grid (fewer blocks when there are fewer items)
    const int want = (A.split_nitems + SW - 1) / SW;
    int blocks;
    if (pb) {
        blocks = h ? split_blocks<PACKSELL_FMT_FP16, true>() : split_blocks<PACKSELL_FMT_E8MY, true>();
        if (!blocks) return fail(PACKSELL_ERR_CUDA, "packsell_spmv: device query failed");
        blocks = std::min(blocks, want);
        if (h)
            k_spmv_split<PACKSELL_FMT_FP16, true><<<blocks, SW * 32, 0, s>>>(
                sg, sh, kl, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
        else
            k_spmv_split<PACKSELL_FMT_E8MY, true><<<blocks, SW * 32, 0, s>>>(
                sg, sh, kl, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
    } else {
        blocks = h ? split_blocks<PACKSELL_FMT_FP16, false>() : split_blocks<PACKSELL_FMT_E8MY, false>();
        if (!blocks) return fail(PACKSELL_ERR_CUDA, "packsell_spmv: device query failed");
        blocks = std::min(blocks, want);
        if (h)
            k_spmv_split<PACKSELL_FMT_FP16, false><<<blocks, SW * 32, 0, s>>>(
                sg, sh, kl, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
        else
            k_spmv_split<PACKSELL_FMT_E8MY, false><<<blocks, SW * 32, 0, s>>>(
                sg, sh, kl, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
    }
    PS_LAUNCH_CHECK("packsell_spmv (split rows)");
    return PACKSELL_OK;
}

}  // namespace packsell
