// SpMM, Y = A X for k right-hand sides, on PackSELL and FP32 SELL matrices
// (packsell_spmm). The paper evaluates k = 1; the lane-group mapping below
// extends its thread-per-row SpMV so that every column keeps the SpMV's
// bits.
#include <cuda_fp16.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int TPB = 256;

// SpMM, Y = A X with X row-major [m x k] (leading dimension ldx), Y [n x k].
// G lanes share a row (G = 1, 2, 4, 8, 16): they read the same words (one
// broadcast load), decode them alike, and lane sub of the group owns the
// column groups q0 + 4 sub + 4 G h (h < KV) of four consecutive columns, so
// one gather instruction fetches 32/G rows of X, 16 G contiguous bytes each
// (16-byte loads when VEC, four scalar loads otherwise). A pass covers 4 G KV
// columns; wider k takes several passes. Each column is accumulated with
// fused multiply-adds in stored order, so column q of Y equals packsell_spmv
// with x = X[:, q] bit for bit. Rounds of SPF words per row as in the
// prefetch SpMV; a row ends at its first zero word (padding follows).
constexpr int SPF = 8;

template <int KV, bool VEC>
__device__ __forceinline__ void spmm_load(const float *__restrict__ xr, int qa, int step, int k,
                                          float4 (&xv)[KV]) {
#pragma unroll
    for (int h = 0; h < KV; ++h) {
        const int q = qa + step * h;
        if (VEC) {
            xv[h] = (q < k) ? __ldg(reinterpret_cast<const float4 *>(xr + step * h))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            xv[h].x = (q < k) ? __ldg(xr + step * h) : 0.f;
            xv[h].y = (q + 1 < k) ? __ldg(xr + step * h + 1) : 0.f;
            xv[h].z = (q + 2 < k) ? __ldg(xr + step * h + 2) : 0.f;
            xv[h].w = (q + 3 < k) ? __ldg(xr + step * h + 3) : 0.f;
        }
    }
}

template <int KV>
__device__ __forceinline__ void spmm_fma(float v, const float4 (&xv)[KV], float4 (&acc)[KV]) {
#pragma unroll
    for (int h = 0; h < KV; ++h) {
        acc[h].x = fmaf(v, xv[h].x, acc[h].x);
        acc[h].y = fmaf(v, xv[h].y, acc[h].y);
        acc[h].z = fmaf(v, xv[h].z, acc[h].z);
        acc[h].w = fmaf(v, xv[h].w, acc[h].w);
    }
}

template <int KV, bool VEC>
__device__ __forceinline__ void spmm_gather(const float *__restrict__ xr, int qa, int step, int k,
                                            float v, float4 (&acc)[KV]) {
    float4 xv[KV];
    spmm_load<KV, VEC>(xr, qa, step, k, xv);
    spmm_fma<KV>(v, xv, acc);
}

template <int KV, bool VEC>
__device__ __forceinline__ void spmm_store(float *__restrict__ yr, int qa, int step, int k,
                                           const float4 (&acc)[KV]) {
#pragma unroll
    for (int h = 0; h < KV; ++h) {
        const int q = qa + step * h;
        if (VEC) {
            if (q < k) *reinterpret_cast<float4 *>(yr + step * h) = acc[h];
        } else {
            if (q < k) yr[step * h] = acc[h].x;
            if (q + 1 < k) yr[step * h + 1] = acc[h].y;
            if (q + 2 < k) yr[step * h + 2] = acc[h].z;
            if (q + 3 < k) yr[step * h + 3] = acc[h].w;
        }
    }
}

template <int FMT, int G, int KV, bool VEC, bool C32, int GB = 1>
__global__ void __launch_bounds__(TPB)
    k_spmm_packed(int n, int Cr, int sigma, long long k_left, const int64_t *__restrict__ offset,
                  const uint32_t *__restrict__ pack, const void *__restrict__ perm, int perm_bytes,
                  Decode dc, int k, const float *__restrict__ X, int64_t ldx,
                  float *__restrict__ Y, int64_t ldy) {
    const int C = C32 ? 32 : Cr;  // a constant word stride when C = 32
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(gt / G), sub = (int)(gt % G);
    if (i >= n) return;
    const int kb = i / C, l = i - kb * C;
    const int64_t s = offset[kb];
    const int w = (int)((offset[kb + 1] - s) / C);
    const uint32_t *__restrict__ pp = pack + s + l;
    const int c0 = left_offset(i, sigma, k_left);
    const int io = orig_row(i, sigma, perm, perm_bytes);
    constexpr int step = 4 * G;
    for (int q0 = 0; q0 < k; q0 += step * KV) {
        const int qa = q0 + 4 * sub;
        float4 acc[KV];
#pragma unroll
        for (int h = 0; h < KV; ++h) acc[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        int c = c0;
        for (int j0 = 0; j0 < w; j0 += SPF) {
            const int wr = w - j0;
            uint32_t wd[SPF];
#pragma unroll
            for (int u = 0; u < SPF; ++u)
                wd[u] = (u < wr) ? ldg_stream(pp + (C32 ? (j0 + u) * 32 : (int64_t)(j0 + u) * C)) : 0u;
            if (GB == 1) {
#pragma unroll
                for (int u = 0; u < SPF; ++u) {
                    const bool f = (wd[u] & 1u) != 0u;
                    c += (int)((wd[u] >> 1) & (f ? dc.dmask : 0x7fffffffu));
                    if (f && PS_IN_RANGE(c, dc.xlen))
                        spmm_gather<KV, VEC>(X + (int64_t)c * ldx + qa, qa, step, k,
                                             word_value<FMT>(wd[u], dc), acc);
                }
            } else {
                // two phases: the columns of the round first, then the X
                // gathers of GB words at a time before their multiply-adds
                // (long rows: one gather latency per GB words, not per word)
                int cc[SPF];
#pragma unroll
                for (int u = 0; u < SPF; ++u) {
                    const bool f = (wd[u] & 1u) != 0u;
                    c += (int)((wd[u] >> 1) & (f ? dc.dmask : 0x7fffffffu));
                    cc[u] = c;
                }
#pragma unroll
                for (int g0 = 0; g0 < SPF; g0 += GB) {
                    float4 xv[GB][KV];
#pragma unroll
                    for (int u = 0; u < GB; ++u) {
                        if (!PS_IN_RANGE(cc[g0 + u], dc.xlen)) wd[g0 + u] &= ~1u;  // skipped
                        if (wd[g0 + u] & 1u)
                            spmm_load<KV, VEC>(X + (int64_t)cc[g0 + u] * ldx + qa, qa, step, k, xv[u]);
                    }
#pragma unroll
                    for (int u = 0; u < GB; ++u)
                        if (wd[g0 + u] & 1u) spmm_fma<KV>(word_value<FMT>(wd[g0 + u], dc), xv[u], acc);
                }
            }
            if (wd[SPF - 1] == 0u) break;  // the row has ended
        }
        spmm_store<KV, VEC>(Y + (int64_t)io * ldy + qa, qa, step, k, acc);
    }
}

// The same lane-group SpMM for FP32 SELL: every stored slot multiplies
// (padding holds value 0), as in the SELL SpMV.
template <int G, int KV, bool VEC>
__global__ void __launch_bounds__(TPB)
    k_spmm_sell(int n, int C, int sigma, const int64_t *__restrict__ offset,
                const float *__restrict__ val, const int32_t *__restrict__ col,
                const void *__restrict__ perm, int perm_bytes, int k, const float *__restrict__ X,
                int64_t ldx, float *__restrict__ Y, int64_t ldy) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(gt / G), sub = (int)(gt % G);
    if (i >= n) return;
    const int kb = i / C, l = i - kb * C;
    const int64_t s = offset[kb];
    const int w = (int)((offset[kb + 1] - s) / C);
    const int io = orig_row(i, sigma, perm, perm_bytes);
    constexpr int step = 4 * G;
    for (int q0 = 0; q0 < k; q0 += step * KV) {
        const int qa = q0 + 4 * sub;
        float4 acc[KV];
#pragma unroll
        for (int h = 0; h < KV; ++h) acc[h] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < w; ++j) {
            const int64_t p = s + (int64_t)j * C + l;
            spmm_gather<KV, VEC>(X + (int64_t)col[p] * ldx + qa, qa, step, k, val[p], acc);
        }
        spmm_store<KV, VEC>(Y + (int64_t)io * ldy + qa, qa, step, k, acc);
    }
}

}  // namespace

template <int FMT, int G, int KV, bool VEC>
void launch_spmm_packed(const Matrix &A, const void *perm, int pb, int k, const float *X,
                        int64_t ldx, float *Y, int64_t ldy, unsigned g, cudaStream_t s) {
    constexpr int GB = KV == 1 ? 8 : 4;  // gathers in flight per lane in the two-phase form
    auto kern = A.p.C != 32 ? k_spmm_packed<FMT, G, KV, VEC, false>
                : A.max_width > 32 ? k_spmm_packed<FMT, G, KV, VEC, true, GB>  // long rows
                                   : k_spmm_packed<FMT, G, KV, VEC, true>;
    kern<<<g, TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb,
                           make_decode(A), k, X, ldx, Y, ldy);
}

template <int G, int KV, bool VEC>
void launch_spmm(const Matrix &A, const void *perm, int pb, int k, const float *X, int64_t ldx,
                 float *Y, int64_t ldy, cudaStream_t s) {
    const int64_t threads = A.n * G;
    const unsigned g = (unsigned)((threads + TPB - 1) / TPB);
    switch (A.p.format) {
        case PACKSELL_FMT_FP16:
            launch_spmm_packed<PACKSELL_FMT_FP16, G, KV, VEC>(A, perm, pb, k, X, ldx, Y, ldy, g, s);
            break;
        case PACKSELL_FMT_E8MY:
            launch_spmm_packed<PACKSELL_FMT_E8MY, G, KV, VEC>(A, perm, pb, k, X, ldx, Y, ldy, g, s);
            break;
        default:
            k_spmm_sell<G, KV, VEC><<<g, TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset,
                                                     (const float *)A.val, A.col, perm, pb, k, X,
                                                     ldx, Y, ldy);
    }
}

template <int G, int KV>
void launch_spmm_v(bool vec, const Matrix &A, const void *perm, int pb, int k, const float *X,
                   int64_t ldx, float *Y, int64_t ldy, cudaStream_t s) {
    if (vec) launch_spmm<G, KV, true>(A, perm, pb, k, X, ldx, Y, ldy, s);
    else launch_spmm<G, KV, false>(A, perm, pb, k, X, ldx, Y, ldy, s);
}

packsell_status spmm_impl(const Matrix &A, int k, const float *X, int64_t ldx, float *Y,
                          int64_t ldy, cudaStream_t s) {
    if (k < 1 || ldx < k || ldy < k)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmm: need k >= 1, ldx >= k, ldy >= k");
    if (A.p.format == PACKSELL_FMT_SELL_F64)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmm: SELL_F64 not supported");
    if (A.n == 0) return PACKSELL_OK;
    if (k == 1 && ldx == 1 && ldy == 1) return spmv_impl(A, X, Y, s);  // the tuned SpMV
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    const bool vec = k % 4 == 0 && ldx % 4 == 0 && ldy % 4 == 0 &&
                     ((uintptr_t)X & 15) == 0 && ((uintptr_t)Y & 15) == 0;
    // CSR order (C = 1): split rows, all lanes of a warp sharing a tile's words
    if (A.multi_items) {
        const packsell_status st = launch_multi(split_mat(A, X, ldx, Y, ldy, k), nullptr,
                                                (const MultiItem *)A.multi_items, A.multi_nitems, k,
                                                vec, s);
        return st;
    }
    // lanes per row and column groups per lane: one pass for k <= 128
    if (k <= 4) launch_spmm_v<1, 1>(vec, A, perm, pb, k, X, ldx, Y, ldy, s);
    else if (k <= 8) launch_spmm_v<1, 2>(vec, A, perm, pb, k, X, ldx, Y, ldy, s);
    else if (k <= 16) launch_spmm_v<2, 2>(vec, A, perm, pb, k, X, ldx, Y, ldy, s);
    else if (k <= 32) launch_spmm_v<4, 2>(vec, A, perm, pb, k, X, ldx, Y, ldy, s);
    else if (k <= 64) launch_spmm_v<8, 2>(vec, A, perm, pb, k, X, ldx, Y, ldy, s);
    else launch_spmm_v<16, 2>(vec, A, perm, pb, k, X, ldx, Y, ldy, s);
    PS_LAUNCH_CHECK("packsell_spmm");
    return PACKSELL_OK;
}

}  // namespace packsell
