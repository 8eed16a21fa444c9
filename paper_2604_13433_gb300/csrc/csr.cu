// Delta-value packing in CSR order: a PackSELL matrix with slice height
// C = 1 is a row-by-row word stream (each slice is one row, no padding, the
// slice offsets are the row pointer). The paper names this CSR-based form as
// the remedy for matrices whose rows vary so much that SELL slices are mostly
// padding (§5.1.1 "not suitable" matrices; §7 future work).
//
// SpMV variant 11. At encode time the rows are cut into work items: tiles of
// consecutive rows of at most CL words each, holding at most CT words and CR
// rows, and single rows of more than CL words, listed first, longest first.
// Warp w takes items w, w + W, ... (W warps in the grid):
//  * tile: the warp copies the tile's words (one contiguous run) into shared
//    memory with coalesced loads; then lane l sums rows l, l + 32 of the
//    tile from shared memory, each in stored order with fused multiply-adds,
//    gathering x for up to 16 words at once;
//  * long row: the warp walks the row CT words at a time; lane l decodes
//    words l, l + 32, ...; a warp prefix sum of the deltas gives each word's
//    column (Eq. 2) from the running column, every lane gathers its words'
//    x and writes (value, x) pairs to shared memory, and lane 0 then runs the
//    fused multiply-adds over the chunk in stored order.
// Either way every row's sum is the same chain of fmaf as the thread-per-row
// kernels, so the result is bit for bit the oracle's FP32 twin.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int CT = 256;  // words per tile (and per chunk of a long row)
constexpr int CR = 64;   // rows per tile at most
constexpr int CL = 256;  // rows of more words take the warp-cooperative path
constexpr int CW = 8;    // warps per block
constexpr int CPF = 8;   // words of a row gathered at once (most rows are short)

template <int FMT, bool PERM>
__device__ __forceinline__ void csr_store(int row, int sigma, int sig_shift, const void *perm,
                                          int perm_bytes, float t, float *__restrict__ y) {
    int io = row;
    if (PERM) {
        const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
        io = blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[row]
                                    : (int)((const uint16_t *)perm)[row]);
    }
    y[io] = t;
}

__device__ __forceinline__ int csr_left(int row, int sigma, int sig_shift, long long k_left) {
    const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
    return k_left < blk ? (int)(blk - k_left) : 0;
}

template <int FMT, bool PERM>
__global__ void __launch_bounds__(CW * 32, 4)
    k_spmv_csr(int sigma, int sig_shift, long long k_left, const int64_t *__restrict__ offset,
               const uint32_t *__restrict__ pack, const void *__restrict__ perm, int perm_bytes,
               Decode dc, const int2 *__restrict__ items, int nitems,
               const float *__restrict__ x, float *__restrict__ y) {
    __shared__ uint32_t s_w[CW][CT];            // tile words
    __shared__ __align__(16) float s_v[CW][CT];  // long rows: values
    __shared__ __align__(16) float s_x[CW][CT];  // long rows: gathered x
    __shared__ int s_ro[CW][CR + 1];  // tile row offsets (relative)
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    // warp w takes items w, w + W, ...: the plan lists the long rows first,
    // longest first, so they are dealt one per warp before the short tiles
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int it = gw; it < nitems; it += nwarps) {
        const int2 item = items[it];
        const int r0 = item.x, r1 = item.y;
        const int64_t base = offset[r0];
        const int nwd = (int)(offset[r1] - base);
        if (r1 - r0 == 1 && nwd > CL) {
            // ---- one long row, CT words per chunk ----
            uint32_t carry = (uint32_t)csr_left(r0, sigma, sig_shift, k_left);
            float t = 0.f;
            // the chunk's words are loaded one chunk ahead: the loads of
            // chunk k + 1 are in flight while chunk k is scanned, gathered
            // and summed (a warp issues in order: loads placed right before
            // their use would wait out each round trip)
            uint32_t wd[CT / 32];
#pragma unroll
            for (int u = 0; u < CT / 32; ++u)
                wd[u] = 32 * u + lane < min(CT, nwd) ? ldg_stream(pack + base + 32 * u + lane) : 0u;
            for (int k0 = 0; k0 < nwd; k0 += CT) {
                const int cnt = min(CT, nwd - k0);
                const int cn = min(CT, nwd - k0 - CT);  // next chunk (<= 0: none)
                uint32_t nx[CT / 32], c[CT / 32];
#pragma unroll
                for (int u = 0; u < CT / 32; ++u) {
                    const int k = 32 * u + lane;
                    nx[u] = k < cn ? ldg_stream(pack + base + k0 + CT + k) : 0u;
                }
#pragma unroll
                for (int u = 0; u < CT / 32; ++u) {
                    c[u] = 0u;
                    if (32 * u >= cnt) continue;  // warp-uniform: past the chunk
                    const bool f = (wd[u] & 1u) != 0u;
                    uint32_t sc = (wd[u] >> 1) & (f ? dc.dmask : 0x7fffffffu);
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t v = __shfl_up_sync(0xffffffffu, sc, o);
                        if (lane >= o) sc += v;
                    }
                    c[u] = carry + sc;  // this word's column
                    carry = __shfl_sync(0xffffffffu, c[u], 31);
                }
                float xv[CT / 32];
#pragma unroll
                for (int u = 0; u < CT / 32; ++u)
                    xv[u] = ((wd[u] & 1u) && PS_IN_RANGE(c[u], dc.xlen)) ? __ldg(x + c[u]) : 0.f;
                // a word without a value (dummy, or past the row's end) is
                // stored as the pair (-0, 0): fmaf(-0, 0, t) == t for every t
                // (including -0, infinities and NaN), so the chain below
                // needs no test and equals the one that skips such words
#pragma unroll
                for (int u = 0; u < CT / 32; ++u) {
                    if (32 * u >= cnt) continue;
                    s_v[wl][32 * u + lane] = (wd[u] & 1u) ? word_value<FMT>(wd[u], dc) : -0.f;
                    s_x[wl][32 * u + lane] = xv[u];
                }
                __syncwarp();
                if (lane == 0) {
                    const float4 *v4 = reinterpret_cast<const float4 *>(s_v[wl]);
                    const float4 *x4 = reinterpret_cast<const float4 *>(s_x[wl]);
                    const int n4 = (cnt + 3) >> 2;
#pragma unroll 4
                    for (int k = 0; k < n4; ++k) {
                        const float4 a = v4[k], b = x4[k];
                        t = fmaf(a.x, b.x, t);
                        t = fmaf(a.y, b.y, t);
                        t = fmaf(a.z, b.z, t);
                        t = fmaf(a.w, b.w, t);
                    }
                }
                __syncwarp();
#pragma unroll
                for (int u = 0; u < CT / 32; ++u) wd[u] = nx[u];
            }
            if (lane == 0) csr_store<FMT, PERM>(r0, sigma, sig_shift, perm, perm_bytes, t, y);
            continue;
        }
        // ---- a tile of rows: words to shared memory, one lane per row ----
        {
            uint32_t wd[CT / 32];
            int64_t ro[(CR + 32) / 32];
#pragma unroll
            for (int u = 0; u < CT / 32; ++u)
                wd[u] = (32 * u + lane < nwd) ? ldg_stream(pack + base + 32 * u + lane) : 0u;
#pragma unroll
            for (int u = 0; u < (CR + 32) / 32; ++u)
                ro[u] = (32 * u + lane <= r1 - r0) ? offset[r0 + 32 * u + lane] : 0;
#pragma unroll
            for (int u = 0; u < CT / 32; ++u)
                if (32 * u + lane < nwd) s_w[wl][32 * u + lane] = wd[u];
#pragma unroll
            for (int u = 0; u < (CR + 32) / 32; ++u)
                if (32 * u + lane <= r1 - r0) s_ro[wl][32 * u + lane] = (int)(ro[u] - base);
        }
        __syncwarp();
        for (int q = lane; q < r1 - r0; q += 32) {
            const int row = r0 + q;
            const int a = s_ro[wl][q], b = s_ro[wl][q + 1];
            int c = csr_left(row, sigma, sig_shift, k_left);
            float t = 0.f;
            for (int k0 = a; k0 < b; k0 += CPF) {
                uint32_t wd[CPF];
#pragma unroll
                for (int u = 0; u < CPF; ++u) wd[u] = (k0 + u < b) ? s_w[wl][k0 + u] : 0u;
                bool f[CPF];
                float xv[CPF];
#pragma unroll
                for (int u = 0; u < CPF; ++u) word_gather<FMT>(wd[u], dc, x, c, f[u], xv[u]);
#pragma unroll
                for (int u = 0; u < CPF; ++u)
                    if (f[u]) t = fmaf(word_value<FMT>(wd[u], dc), xv[u], t);
            }
            csr_store<FMT, PERM>(row, sigma, sig_shift, perm, perm_bytes, t, y);
        }
        __syncwarp();
    }
}

template <int FMT, bool PERM>
int csr_blocks() {
    // persistent grid: every block resident at once (cached per process; calls
    // from several host threads may compute it together and store the same value)
    static std::atomic<int> cached{0};
    int blocks = cached.load(std::memory_order_relaxed);
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_spmv_csr<FMT, PERM>, CW * 32, 0) !=
                cudaSuccess)
            return 0;
        blocks = sms * std::max(per, 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    return blocks;
}

}  // namespace

void csr_plan_free(Matrix &A) {
    cudaFree(A.csr_items);
    A.csr_items = nullptr;
    A.csr_nitems = 0;
}

// Items for variant 11 (C = 1 PackSELL matrices): consecutive rows of at
// most CL words are grouped greedily while they hold at most CT words and CR
// rows; a row of more than CL words is an item of its own. Built on the host
// from the row offsets.
packsell_status plan_csr(Matrix &A, cudaStream_t s) {
    csr_plan_free(A);
    if (!is_packed(A.p.format) || A.p.C != 1 || A.n == 0) return PACKSELL_OK;
    std::vector<int64_t> off((size_t)A.n + 1);
    PS_CUDA(cudaMemcpyAsync(off.data(), A.offset, sizeof(int64_t) * (A.n + 1),
                            cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    std::vector<int2> items;
    items.reserve((size_t)(A.n_words / CT + A.n / CR + 16));
    int r0 = 0;
    for (int r = 0; r < (int)A.n; ++r) {
        const int64_t w = off[r + 1] - off[r];
        if (w > CL) {  // a long row: close the tile before it, then the row alone
            if (r > r0) items.push_back(make_int2(r0, r));
            items.push_back(make_int2(r, r + 1));
            r0 = r + 1;
            continue;
        }
        if (off[r + 1] - off[r0] > CT || r + 1 - r0 > CR) {
            items.push_back(make_int2(r0, r));
            r0 = r;
        }
    }
    if ((int)A.n > r0) items.push_back(make_int2(r0, (int)A.n));
    // long rows first, longest first: they set the kernel's critical path,
    // and taken early from the queue they overlap the many short tiles
    auto is_long = [&](const int2 &a) { return a.y - a.x == 1 && off[a.y] - off[a.x] > CL; };
    std::stable_partition(items.begin(), items.end(), is_long);
    const size_t nlong = (size_t)std::count_if(items.begin(), items.end(), is_long);
    std::stable_sort(items.begin(), items.begin() + nlong, [&](const int2 &a, const int2 &b) {
        return off[a.y] - off[a.x] > off[b.y] - off[b.x];
    });
    if (items.size() >= (size_t)INT32_MAX) return fail(PACKSELL_ERR_RANGE, "plan_csr: too many items");
    PS_CUDA(cudaMalloc(&A.csr_items, sizeof(int2) * items.size()));
    PS_CUDA(cudaMemcpyAsync(A.csr_items, items.data(), sizeof(int2) * items.size(),
                            cudaMemcpyHostToDevice, s));
    PS_CUDA(cudaStreamSynchronize(s));
    A.csr_nitems = (int)items.size();
    return PACKSELL_OK;
}

packsell_status launch_csr(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                           cudaStream_t s) {
    if (!A.csr_items)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: variant 11 needs a PackSELL matrix with C = 1");
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    const Decode dc = make_decode(A);
    const bool h = A.p.format == PACKSELL_FMT_FP16;
    const int2 *it = reinterpret_cast<const int2 *>(A.csr_items);
    int blocks;
    if (pb) {
        blocks = h ? csr_blocks<PACKSELL_FMT_FP16, true>() : csr_blocks<PACKSELL_FMT_E8MY, true>();
        if (!blocks) return fail(PACKSELL_ERR_CUDA, "packsell_spmv: device query failed");
        if (h)
            k_spmv_csr<PACKSELL_FMT_FP16, true><<<blocks, CW * 32, 0, s>>>(
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.csr_nitems, x, y);
        else
            k_spmv_csr<PACKSELL_FMT_E8MY, true><<<blocks, CW * 32, 0, s>>>(
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.csr_nitems, x, y);
    } else {
        blocks = h ? csr_blocks<PACKSELL_FMT_FP16, false>() : csr_blocks<PACKSELL_FMT_E8MY, false>();
        if (!blocks) return fail(PACKSELL_ERR_CUDA, "packsell_spmv: device query failed");
        if (h)
            k_spmv_csr<PACKSELL_FMT_FP16, false><<<blocks, CW * 32, 0, s>>>(
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.csr_nitems, x, y);
        else
            k_spmv_csr<PACKSELL_FMT_E8MY, false><<<blocks, CW * 32, 0, s>>>(
                sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, dc, it, A.csr_nitems, x, y);
    }
    PS_LAUNCH_CHECK("packsell_spmv (CSR order)");
    return PACKSELL_OK;
}

}  // namespace packsell
