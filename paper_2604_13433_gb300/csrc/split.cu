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

constexpr int ST = 256;       // words a warp holds per chunk: SRD rounds of 128
constexpr int SRD = ST / 128;
constexpr int SCT = ST - 3;   // tile words at most (room for the aligned-down start)
constexpr int SR_MAX = 256;   // tile rows at most
constexpr int SW = 8;         // warps per block
constexpr uint32_t kAbs = 0x80000000u;  // column scan: the value is an absolute column

// Column scan operator on (absolute?, value) packed in one word: a later
// absolute column replaces what came before, a later relative delta adds to
// it. Columns and their partial sums stay below 2^31.
__device__ __forceinline__ uint32_t col_comb(uint32_t a, uint32_t b) { return (b & kAbs) ? b : a + b; }

__device__ __forceinline__ int split_left(int row, int sigma, int sig_shift, long long k_left) {
    const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
    return k_left < blk ? (int)(blk - k_left) : 0;
}

template <bool PERM>
__device__ __forceinline__ void split_store(int row, int sigma, int sig_shift, const void *perm,
                                            int perm_bytes, float t, float *__restrict__ y) {
    int io = row;
    if (PERM) {
        const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
        io = blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[row]
                                    : (int)((const uint16_t *)perm)[row]);
    }
    y[io] = t;
}

__device__ __forceinline__ uint4 ld_words4(const uint32_t *p) {
    return __ldcs(reinterpret_cast<const uint4 *>(p));
}

__device__ __forceinline__ uint32_t w4(const uint4 &v, int j) {
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

template <int FMT>
__device__ __forceinline__ float split_value(uint32_t wd, Decode dc) {
    if (FMT == PACKSELL_FMT_FP16) return __high2float(*reinterpret_cast<const __half2 *>(&wd));
    return __uint_as_float(wd & dc.vmask);
}

// Work item: a tile of rows [r0, r0 + nrows) holding nwd words from word
// `base` (meta = nrows << 16 | nwd), or one long row of nwd words (meta =
// -nwd). One 16-byte load gives a warp everything it needs to start.
struct __align__(16) SplitItem {
    long long base;
    int r0;
    int meta;
};

// The first ST words of an item, aligned down to 16 bytes: lane l holds the
// words at 128u + 4l .. 128u + 4l + 3 of round u (0 past the item's end).
__device__ __forceinline__ void split_load(const uint32_t *__restrict__ pack, long long base,
                                           int nwd, int lane, uint4 (&wv)[SRD]) {
    const long long a0 = base & ~3ll;
    const int lim = (int)(base - a0) + nwd;
#pragma unroll
    for (int u = 0; u < SRD; ++u) {
        const int p = 128 * u + 4 * lane;
        wv[u] = p < lim ? ld_words4(pack + a0 + p) : make_uint4(0, 0, 0, 0);
    }
}

// One row of more than SCT words: chunks of ST words (the first one already
// loaded into cur), each lane summing its own words, the column carried
// across chunks; the next chunk's words load while the current one is
// decoded and gathered.
template <int FMT, bool PERM>
__device__ __forceinline__ void split_long_row(int row, long long base, int nwd, int sigma,
                                               int sig_shift, long long k_left,
                                               const uint32_t *__restrict__ pack,
                                               const void *__restrict__ perm, int perm_bytes,
                                               Decode dc, const float *__restrict__ x,
                                               float *__restrict__ y, int lane, uint4 (&cur)[SRD]) {
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0), lim = lead + nwd;
    uint32_t carry = (uint32_t)split_left(row, sigma, sig_shift, k_left);
    float t = 0.f;
    for (int k0 = 0; k0 < lim; k0 += ST) {
        uint4 nxt[SRD];
#pragma unroll
        for (int u = 0; u < SRD; ++u) {
            const int p = k0 + ST + 128 * u + 4 * lane;
            nxt[u] = p < lim ? ld_words4(pack + a0 + p) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < SRD; ++u) {
            uint32_t wd[4], cs[4], acc = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = k0 + 128 * u + 4 * lane + j;
                wd[j] = (p >= lead && p < lim) ? w4(cur[u], j) : 0u;
                const uint32_t f = wd[j] & 1u;
                acc += (wd[j] >> 1) & (f ? dc.dmask : 0x7fffffffu);
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
            float xv[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) xv[j] = (wd[j] & 1u) ? __ldg(x + (before + cs[j])) : 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (wd[j] & 1u) t = fmaf(split_value<FMT>(wd[j], dc), xv[j], t);
        }
#pragma unroll
        for (int u = 0; u < SRD; ++u) cur[u] = nxt[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) split_store<PERM>(row, sigma, sig_shift, perm, perm_bytes, t, y);
}

// A tile of rows [r0, r0 + nrows) with its nwd (<= SCT) words in wv.
template <int FMT, bool PERM>
__device__ __forceinline__ void split_tile(int r0, int nrows, long long base, int nwd, int sigma,
                                           int sig_shift, long long k_left,
                                           const int64_t *__restrict__ offset,
                                           const void *__restrict__ perm, int perm_bytes,
                                           Decode dc, const float *__restrict__ x,
                                           float *__restrict__ y, int lane, const uint4 (&wv)[SRD],
                                           int *__restrict__ srow) {
    const long long a0 = base & ~3ll;
    const int lead = (int)(base - a0), lim = lead + nwd;
    int4 *srow4 = reinterpret_cast<int4 *>(srow);
#pragma unroll
    for (int u = 0; u < SRD; ++u) srow4[32 * u + lane] = make_int4(-1, -1, -1, -1);
    __syncwarp();
    // mark where each row starts; an empty row's product is 0
    for (int k = lane; k < nrows; k += 32) {
        const int r = r0 + k;
        const int64_t o0 = offset[r], o1 = offset[r + 1];
        if (o1 > o0) srow[(int)(o0 - a0)] = r;
        else split_store<PERM>(r, sigma, sig_shift, perm, perm_bytes, 0.f, y);
    }
    __syncwarp();
    int hr[SRD][4];    // storage row starting at the word, or -1
    float pv[SRD][4];  // value * x of every word (0 without a value)
    uint32_t carry = 0;
#pragma unroll
    for (int u = 0; u < SRD; ++u) {
        const int4 h = srow4[32 * u + lane];
        hr[u][0] = h.x;
        hr[u][1] = h.y;
        hr[u][2] = h.z;
        hr[u][3] = h.w;
        uint32_t wd[4], cs[4], acc = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int p = 128 * u + 4 * lane + j;
            wd[j] = (p >= lead && p < lim) ? w4(wv[u], j) : 0u;
            const uint32_t f = wd[j] & 1u;
            const uint32_t d = (wd[j] >> 1) & (f ? dc.dmask : 0x7fffffffu);
            const uint32_t e =
                hr[u][j] >= 0 ? kAbs | ((uint32_t)split_left(hr[u][j], sigma, sig_shift, k_left) + d) : d;
            acc = col_comb(acc, e);
            cs[j] = acc;
        }
        uint32_t inc = acc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc = col_comb(v, inc);
        }
        // the earlier rounds' state comes first (it matters up to the lane's
        // first row start)
        const uint32_t up = __shfl_up_sync(0xffffffffu, inc, 1);
        const uint32_t exc = lane == 0 ? carry : col_comb(carry, up);
        carry = col_comb(carry, __shfl_sync(0xffffffffu, inc, 31));
        float xv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t c = col_comb(exc, cs[j]) & ~kAbs;
            xv[j] = (wd[j] & 1u) ? __ldg(x + c) : 0.f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            pv[u][j] = (wd[j] & 1u) ? split_value<FMT>(wd[j], dc) * xv[j] : 0.f;
    }
    // segmented suffix sums, last round first; `in` is what flows into the
    // round's last lane from the words after it (0 past the tile's end)
    float in = 0.f;
#pragma unroll
    for (int u = SRD - 1; u >= 0; --u) {
        float seg[4], s = 0.f;
        bool hh = false;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            s += pv[u][j];
            seg[j] = s;
            if (hr[u][j] >= 0) {
                s = 0.f;
                hh = true;
            }
        }
        // U: the lane's words before its first row start plus, while no row
        // start intervenes, the same of the lanes after it
        float U = s;
        bool F = hh;
        if (lane == 31 && !F) U += in;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float v = __shfl_down_sync(0xffffffffu, U, o);
            const bool g = __shfl_down_sync(0xffffffffu, F ? 1 : 0, o) != 0;
            if (lane + o < 32 && !F) {
                U += v;
                F = g;
            }
        }
        float nxt_in = __shfl_down_sync(0xffffffffu, U, 1);
        if (lane == 31) nxt_in = in;
        in = __shfl_sync(0xffffffffu, U, 0);
        // the lane's last row start takes what flows in from the lanes after it
        bool last = true;
#pragma unroll
        for (int j = 3; j >= 0; --j) {
            if (hr[u][j] >= 0) {
                const float tot = last ? seg[j] + nxt_in : seg[j];
                last = false;
                split_store<PERM>(hr[u][j], sigma, sig_shift, perm, perm_bytes, tot, y);
            }
        }
    }
    __syncwarp();
}

// Persistent grid: warp w takes items w, w + W, ...; the next item's
// descriptor loads while the current one is processed, and its first words
// once that is done, so a warp keeps loads in flight across its items.
template <int FMT, bool PERM>
__global__ void __launch_bounds__(SW * 32)
    k_spmv_split(int sigma, int sig_shift, long long k_left, const int64_t *__restrict__ offset,
                 const uint32_t *__restrict__ pack, const void *__restrict__ perm, int perm_bytes,
                 Decode dc, const SplitItem *__restrict__ items, int nitems,
                 const float *__restrict__ x, float *__restrict__ y) {
    __shared__ __align__(16) int s_row[SW][ST];  // storage row starting at a position, or -1
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    int it = gw;
    if (it >= nitems) return;
    SplitItem d = items[it];
    uint4 wv[SRD];
    split_load(pack, d.base, d.meta < 0 ? -d.meta : (d.meta & 0xFFFF), lane, wv);
    for (; it < nitems; it += nwarps) {
        const int nit = it + nwarps;
        SplitItem dn;
        if (nit < nitems) dn = items[nit];
        if (d.meta < 0)
            split_long_row<FMT, PERM>(d.r0, d.base, -d.meta, sigma, sig_shift, k_left, pack, perm,
                                      perm_bytes, dc, x, y, lane, wv);
        else
            split_tile<FMT, PERM>(d.r0, d.meta >> 16, d.base, d.meta & 0xFFFF, sigma, sig_shift,
                                  k_left, offset, perm, perm_bytes, dc, x, y, lane, wv, s_row[wl]);
        if (nit < nitems) {
            d = dn;
            split_load(pack, d.base, d.meta < 0 ? -d.meta : (d.meta & 0xFFFF), lane, wv);
        }
    }
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
packsell_status plan_split(Matrix &A, cudaStream_t s) {
    split_plan_free(A);
    if (!is_packed(A.p.format) || A.p.C != 1 || A.n == 0) return PACKSELL_OK;
    std::vector<int64_t> off((size_t)A.n + 1);
    PS_CUDA(cudaMemcpyAsync(off.data(), A.offset, sizeof(int64_t) * (A.n + 1),
                            cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    std::vector<SplitItem> items;
    items.reserve((size_t)(A.n_words / SCT + A.n / SR_MAX + 16));
    auto tile = [&](int a, int b) {
        items.push_back(SplitItem{(long long)off[a], a, ((b - a) << 16) | (int)(off[b] - off[a])});
    };
    int r0 = 0;
    for (int r = 0; r < (int)A.n; ++r) {
        const int64_t w = off[r + 1] - off[r];
        if (w > SCT) {
            if (r > r0) tile(r0, r);
            if (w >= INT32_MAX) return fail(PACKSELL_ERR_RANGE, "plan_split: row too long");
            items.push_back(SplitItem{(long long)off[r], r, -(int)w});
            r0 = r + 1;
            continue;
        }
        if (off[r + 1] - off[r0] > SCT || r + 1 - r0 > SR_MAX) {
            tile(r0, r);
            r0 = r;
        }
    }
    if ((int)A.n > r0) tile(r0, (int)A.n);
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

packsell_status launch_split(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                             cudaStream_t s) {
    if (!A.split_items)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_spmv: variant 14 needs a PackSELL matrix with C = 1");
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    const Decode dc = make_decode(A);
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
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
        else
            k_spmv_split<PACKSELL_FMT_E8MY, true><<<blocks, SW * 32, 0, s>>>(
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
    } else {
        blocks = h ? split_blocks<PACKSELL_FMT_FP16, false>() : split_blocks<PACKSELL_FMT_E8MY, false>();
        if (!blocks) return fail(PACKSELL_ERR_CUDA, "packsell_spmv: device query failed");
        blocks = std::min(blocks, want);
        if (h)
            k_spmv_split<PACKSELL_FMT_FP16, false><<<blocks, SW * 32, 0, s>>>(
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
        else
            k_spmv_split<PACKSELL_FMT_E8MY, false><<<blocks, SW * 32, 0, s>>>(
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.split_nitems, x, y);
    }
    PS_LAUNCH_CHECK("packsell_spmv (split rows)");
    return PACKSELL_OK;
}

}  // namespace packsell
