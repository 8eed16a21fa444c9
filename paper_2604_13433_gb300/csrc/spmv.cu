// PackSELL and SELL products.
//
// Thread-per-row kernels (the mapping of §5.1.1): thread i owns storage row
// i; with C = 32 a warp owns a slice, so word j of all 32 rows is one
// coalesced 128-byte line (p = offset_k + j*C + l, §3/§4.4). The running
// column c starts at the left offset (Eq. 4) and adds each word's delta; a
// word with flag 1 adds value * x_c to the FP32 sum with a fused
// multiply-add, a word with flag 0 (dummy or padding) loads nothing.
#include <cuda_fp16.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int TPB = 256;
constexpr int UNROLL = 8;

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, (n + TPB - 1) / TPB); }

struct Decode {
    uint32_t dmask, vmask;
};

inline Decode make_decode(const Matrix &A) {
    Decode d;
    d.dmask = (1u << A.p.D) - 1u;
    d.vmask = ~((2u << A.p.D) - 1u);
    return d;
}

template <int FMT>
__global__ void __launch_bounds__(TPB)
    k_spmv_packed(int n, int C, int sigma, long long k_left, const int64_t *__restrict__ offset,
                  const uint32_t *__restrict__ pack, const void *__restrict__ perm, int perm_bytes,
                  Decode dc, const float *__restrict__ x, float *__restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int w = (int)((offset[k + 1] - s) / C);
    const uint32_t *pp = pack + s + l;
    int c = left_offset(i, sigma, k_left);
    float t = 0.f;
    int j = 0;
    for (; j + UNROLL <= w; j += UNROLL) {
        uint32_t wd[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) wd[u] = ldg_stream(pp + (int64_t)(j + u) * C);
        float xv[UNROLL], vv[UNROLL];
        uint32_t fl[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            uint32_t d;
            Word<FMT>::decode(wd[u], dc.dmask, dc.vmask, fl[u], d, vv[u]);
            c += (int)d;
            xv[u] = fl[u] ? __ldg(x + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            if (fl[u]) t = fmaf(vv[u], xv[u], t);
    }
    for (; j < w; ++j) {
        uint32_t f, d;
        float v;
        Word<FMT>::decode(ldg_stream(pp + (int64_t)j * C), dc.dmask, dc.vmask, f, d, v);
        c += (int)d;
        if (f) t = fmaf(v, __ldg(x + c), t);
    }
    y[orig_row(i, sigma, perm, perm_bytes)] = t;
}

// Plain SELL-C-sigma (§3): value and column streams, padding multiplies 0.
template <typename T>
__global__ void __launch_bounds__(TPB)
    k_spmv_sell(int n, int C, int sigma, const int64_t *__restrict__ offset,
                const T *__restrict__ val, const int32_t *__restrict__ col,
                const void *__restrict__ perm, int perm_bytes, const T *__restrict__ x,
                T *__restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int w = (int)((offset[k + 1] - s) / C);
    const T *vp = val + s + l;
    const int32_t *cp = col + s + l;
    T t = 0;
    int j = 0;
    for (; j + UNROLL <= w; j += UNROLL) {
        T v[UNROLL];
        int cc[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            v[u] = __ldcs(vp + (int64_t)(j + u) * C);
            cc[u] = __ldcs(cp + (int64_t)(j + u) * C);
        }
        T xv[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) xv[u] = __ldg(x + cc[u]);
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) t = fma(v[u], xv[u], t);
    }
    for (; j < w; ++j) t = fma(__ldcs(vp + (int64_t)j * C), __ldg(x + __ldcs(cp + (int64_t)j * C)), t);
    y[orig_row(i, sigma, perm, perm_bytes)] = t;
}

// SpMM, k right-hand sides in chunks of KT accumulators per thread.
template <int FMT, int KT>
__global__ void __launch_bounds__(TPB)
    k_spmm_packed(int n, int C, int sigma, long long k_left, const int64_t *__restrict__ offset,
                  const uint32_t *__restrict__ pack, const void *__restrict__ perm, int perm_bytes,
                  Decode dc, int k, const float *__restrict__ X, int64_t ldx,
                  float *__restrict__ Y, int64_t ldy) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int kb = i / C, l = i - kb * C;
    int64_t s = offset[kb];
    int w = (int)((offset[kb + 1] - s) / C);
    const uint32_t *pp = pack + s + l;
    int io = orig_row(i, sigma, perm, perm_bytes);
    int c0 = left_offset(i, sigma, k_left);
    for (int r0 = 0; r0 < k; r0 += KT) {
        float acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q] = 0.f;
        int c = c0;
        for (int j = 0; j < w; ++j) {
            uint32_t f, d;
            float v;
            Word<FMT>::decode(ldg_stream(pp + (int64_t)j * C), dc.dmask, dc.vmask, f, d, v);
            c += (int)d;
            if (f) {
                const float *xr = X + (int64_t)c * ldx + r0;
#pragma unroll
                for (int q = 0; q < KT; ++q)
                    if (r0 + q < k) acc[q] = fmaf(v, __ldg(xr + q), acc[q]);
            }
        }
        float *yr = Y + (int64_t)io * ldy + r0;
#pragma unroll
        for (int q = 0; q < KT; ++q)
            if (r0 + q < k) yr[q] = acc[q];
    }
}

template <int KT>
__global__ void __launch_bounds__(TPB)
    k_spmm_sell(int n, int C, int sigma, const int64_t *__restrict__ offset,
                const float *__restrict__ val, const int32_t *__restrict__ col,
                const void *__restrict__ perm, int perm_bytes, int k, const float *__restrict__ X,
                int64_t ldx, float *__restrict__ Y, int64_t ldy) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int kb = i / C, l = i - kb * C;
    int64_t s = offset[kb];
    int w = (int)((offset[kb + 1] - s) / C);
    int io = orig_row(i, sigma, perm, perm_bytes);
    for (int r0 = 0; r0 < k; r0 += KT) {
        float acc[KT];
#pragma unroll
        for (int q = 0; q < KT; ++q) acc[q] = 0.f;
        for (int j = 0; j < w; ++j) {
            float v = val[s + (int64_t)j * C + l];
            const float *xr = X + (int64_t)col[s + (int64_t)j * C + l] * ldx + r0;
#pragma unroll
            for (int q = 0; q < KT; ++q)
                if (r0 + q < k) acc[q] = fmaf(v, __ldg(xr + q), acc[q]);
        }
        float *yr = Y + (int64_t)io * ldy + r0;
#pragma unroll
        for (int q = 0; q < KT; ++q)
            if (r0 + q < k) yr[q] = acc[q];
    }
}

// dx += A^T dy by atomic adds from each stored value.
template <int FMT>
__global__ void __launch_bounds__(TPB)
    k_spmv_t_packed(int n, int C, int sigma, long long k_left, const int64_t *__restrict__ offset,
                    const uint32_t *__restrict__ pack, const void *__restrict__ perm,
                    int perm_bytes, Decode dc, const float *__restrict__ dy, float *dx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int w = (int)((offset[k + 1] - s) / C);
    float g = dy[orig_row(i, sigma, perm, perm_bytes)];
    int c = left_offset(i, sigma, k_left);
    for (int j = 0; j < w; ++j) {
        uint32_t f, d;
        float v;
        Word<FMT>::decode(pack[s + (int64_t)j * C + l], dc.dmask, dc.vmask, f, d, v);
        c += (int)d;
        if (f && g != 0.f) atomicAdd(dx + c, v * g);
    }
}

__global__ void __launch_bounds__(TPB)
    k_spmv_t_sell(int n, int C, int sigma, const int64_t *__restrict__ offset,
                  const float *__restrict__ val, const int32_t *__restrict__ col,
                  const void *__restrict__ perm, int perm_bytes, const float *__restrict__ dy,
                  float *dx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int w = (int)((offset[k + 1] - s) / C);
    float g = dy[orig_row(i, sigma, perm, perm_bytes)];
    if (g == 0.f) return;
    for (int j = 0; j < w; ++j) {
        float v = val[s + (int64_t)j * C + l];
        if (v != 0.f) atomicAdd(dx + col[s + (int64_t)j * C + l], v * g);
    }
}

// out[q] = alpha * u_i * v_c for the q-th stored nonzero (CSR order).
template <int FMT>
__global__ void __launch_bounds__(TPB)
    k_pattern_outer_packed(int n, int C, int sigma, long long k_left,
                           const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
                           const void *__restrict__ perm, int perm_bytes, Decode dc,
                           const int64_t *__restrict__ rowptr, float alpha,
                           const float *__restrict__ u, const float *__restrict__ v,
                           float *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int w = (int)((offset[k + 1] - s) / C);
    int io = orig_row(i, sigma, perm, perm_bytes);
    float a = alpha * u[io];
    int64_t q = rowptr[io];
    int c = left_offset(i, sigma, k_left);
    for (int j = 0; j < w; ++j) {
        uint32_t f, d;
        float val;
        Word<FMT>::decode(pack[s + (int64_t)j * C + l], dc.dmask, dc.vmask, f, d, val);
        c += (int)d;
        if (f) out[q++] = a * v[c];
    }
}

__global__ void __launch_bounds__(TPB)
    k_pattern_outer_sell(int n, int C, int sigma, const int64_t *__restrict__ offset,
                         const int32_t *__restrict__ col, const void *__restrict__ perm,
                         int perm_bytes, const int64_t *__restrict__ rowptr, float alpha,
                         const float *__restrict__ u, const float *__restrict__ v,
                         float *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int io = orig_row(i, sigma, perm, perm_bytes);
    float a = alpha * u[io];
    int64_t q0 = rowptr[io], len = rowptr[io + 1] - q0;
    for (int64_t j = 0; j < len; ++j) out[q0 + j] = a * v[col[s + j * C + l]];
}

}  // namespace

packsell_status spmv_impl(const Matrix &A, const float *x, float *y, cudaStream_t s) {
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    int g = grid_for(A.n);
    switch (A.p.format) {
        case PACKSELL_FMT_FP16:
            k_spmv_packed<PACKSELL_FMT_FP16><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
            break;
        case PACKSELL_FMT_E8MY:
            k_spmv_packed<PACKSELL_FMT_E8MY><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
            break;
        case PACKSELL_FMT_SELL_F32:
            k_spmv_sell<float><<<g, TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset,
                                                 (const float *)A.val, A.col, perm, pb, x, y);
            break;
        default:
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: SELL_F64 needs packsell_spmv_f64");
    }
    PS_LAUNCH_CHECK("packsell_spmv");
    return PACKSELL_OK;
}

packsell_status spmv_f64_impl(const Matrix &A, const double *x, double *y, cudaStream_t s) {
    if (A.p.format != PACKSELL_FMT_SELL_F64)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_f64: matrix is not SELL_F64");
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    k_spmv_sell<double><<<grid_for(A.n), TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset,
                                                      (const double *)A.val, A.col, perm, pb, x, y);
    PS_LAUNCH_CHECK("packsell_spmv_f64");
    return PACKSELL_OK;
}

packsell_status spmm_impl(const Matrix &A, int k, const float *X, int64_t ldx, float *Y,
                          int64_t ldy, cudaStream_t s) {
    if (k < 1 || ldx < k || ldy < k)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmm: need k >= 1, ldx >= k, ldy >= k");
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    int g = grid_for(A.n);
    constexpr int KT = 16;
    switch (A.p.format) {
        case PACKSELL_FMT_FP16:
            k_spmm_packed<PACKSELL_FMT_FP16, KT><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A),
                k, X, ldx, Y, ldy);
            break;
        case PACKSELL_FMT_E8MY:
            k_spmm_packed<PACKSELL_FMT_E8MY, KT><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A),
                k, X, ldx, Y, ldy);
            break;
        case PACKSELL_FMT_SELL_F32:
            k_spmm_sell<KT><<<g, TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset,
                                              (const float *)A.val, A.col, perm, pb, k, X, ldx, Y,
                                              ldy);
            break;
        default:
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmm: SELL_F64 not supported");
    }
    PS_LAUNCH_CHECK("packsell_spmm");
    return PACKSELL_OK;
}

packsell_status spmv_t_impl(const Matrix &A, const float *dy, float *dx, cudaStream_t s) {
    if (A.m > 0) PS_CUDA(cudaMemsetAsync(dx, 0, sizeof(float) * A.m, s));
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    int g = grid_for(A.n);
    switch (A.p.format) {
        case PACKSELL_FMT_FP16:
            k_spmv_t_packed<PACKSELL_FMT_FP16><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), dy, dx);
            break;
        case PACKSELL_FMT_E8MY:
            k_spmv_t_packed<PACKSELL_FMT_E8MY><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), dy, dx);
            break;
        case PACKSELL_FMT_SELL_F32:
            k_spmv_t_sell<<<g, TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset,
                                            (const float *)A.val, A.col, perm, pb, dy, dx);
            break;
        default:
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_transpose: SELL_F64 not supported");
    }
    PS_LAUNCH_CHECK("packsell_spmv_transpose");
    return PACKSELL_OK;
}

packsell_status pattern_outer_impl(const Matrix &A, float alpha, const float *u, const float *v,
                                   float *out, cudaStream_t s) {
    if (!A.rowptr)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_pattern_outer: matrix was encoded without keep_rowptr");
    if (A.n == 0 || A.nnz == 0) return PACKSELL_OK;
    const void *perm = A.perm;  // rows are addressed in original order here
    int pb = A.perm_bytes;
    int g = grid_for(A.n);
    switch (A.p.format) {
        case PACKSELL_FMT_FP16:
            k_pattern_outer_packed<PACKSELL_FMT_FP16><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A),
                A.rowptr, alpha, u, v, out);
            break;
        case PACKSELL_FMT_E8MY:
            k_pattern_outer_packed<PACKSELL_FMT_E8MY><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A),
                A.rowptr, alpha, u, v, out);
            break;
        default:
            k_pattern_outer_sell<<<g, TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset, A.col, perm,
                                                   pb, A.rowptr, alpha, u, v, out);
            break;
    }
    PS_LAUNCH_CHECK("packsell_pattern_outer");
    return PACKSELL_OK;
}

}  // namespace packsell
