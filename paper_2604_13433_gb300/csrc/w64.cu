// Products on 64-bit PackSELL words (PACKSELL_FMT_W64_E11MY; W = 64, one of
// §4.2.1's word sizes): bit 0 flag, bits 1..D delta, bits D+1..63 an E11MY
// value (a binary64 pattern whose low D + 1 bits are zero); a word with flag
// 0 carries a 63-bit delta (a dummy) or is padding (0). x, y and the
// accumulation are FP64, so the format serves as the FP64 operator of the
// solvers (the outer iteration of §5.2.2 and the outer FGMRES of §5.2.1) at
// 8 bytes per stored element instead of plain SELL's 12.
//
// One thread per row; the words of a round go out before any x gather, and
// each real word is one fused multiply-add in stored order from +0 (the
// chain the oracle's FP64 product fixes). Launched with programmatic
// dependent launch: the first round's words load before the wait on the
// previous kernel of the stream, x and y after it.
#include <algorithm>

#include "device.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace packsell {
namespace {

constexpr int TPB = 256;
constexpr int WU = 4;  // words per round (8 and 16 measured slower on the 27-point matrix)

template <bool DOT>
__device__ __forceinline__ void w64_rows(int n, int C, int sigma, long long k_left, int D,
                                         const int64_t *__restrict__ offset,
                                         const unsigned long long *__restrict__ pack,
                                         const void *__restrict__ perm, int perm_bytes,
                                         const double *__restrict__ x, double *__restrict__ y,
                                         const double *__restrict__ b, Red red, int xlen) {
    if (DOT) grid_dep_sync();  // the reducing form waits before it starts
    else grid_dep_launch();    // one pass over the rows: signal at block start
    if (DOT && red.sc->done) return;  // solver converged: idle (grid-uniform)
    // a decoded delta, and every column, stays below 2^31 (columns are int32 and
    // a dummy's delta is at most a column gap), so the delta comes from the low
    // half of the word; the value's upper 32 bits are the word's own
    const uint32_t dmask = (1u << D) - 1u;
    const uint32_t vmask_lo = (uint32_t)~((2ull << D) - 1ull);
    double d1 = 0.0, d2 = 0.0;
    const int stride = DOT ? gridDim.x * blockDim.x : n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int k = i / C, l = i - k * C;
        const int64_t s = offset[k];
        const int w = (int)((offset[k + 1] - s) / C);
        const unsigned long long *pp = pack + s + l;
        int c = left_offset(i, sigma, k_left);
        double t = 0.0;
        if (!DOT && w == 0) grid_dep_wait();
        for (int j0 = 0; j0 < w; j0 += WU) {
            unsigned long long wd[WU];
#pragma unroll
            for (int u = 0; u < WU; ++u)
                wd[u] = j0 + u < w ? __ldcs(pp + (int64_t)(j0 + u) * C) : 0ull;
            if (!DOT) grid_dep_wait();  // returns at once after the first round
            bool f[WU];
            double xv[WU];
#pragma unroll
            for (int u = 0; u < WU; ++u) {
                const uint32_t lo = (uint32_t)wd[u];
                f[u] = (lo & 1u) != 0u;
                c += (int)((lo >> 1) & (f[u] ? dmask : 0x7fffffffu));
                xv[u] = (f[u] && PS_IN_RANGE(c, xlen)) ? __ldg(x + c) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < WU; ++u)
                if (f[u])
                    t = fma(__hiloint2double((int)(wd[u] >> 32), (int)((uint32_t)wd[u] & vmask_lo)),
                            xv[u], t);
        }
        const int io = orig_row(i, sigma, perm, perm_bytes);
        y[io] = t;
        if (DOT) {
            d1 = fma(x[io], t, d1);
            if (b) d2 = fma(x[io], b[io], d2);
        }
    }
    if (DOT) reduce_publish(red, d1, d2);
}

__global__ void __launch_bounds__(TPB)
    k_spmv_w64(int n, int C, int sigma, long long k_left, int D, const int64_t *__restrict__ offset,
               const unsigned long long *__restrict__ pack, const void *__restrict__ perm,
               int perm_bytes, const double *__restrict__ x, double *__restrict__ y, int xlen) {
    w64_rows<false>(n, C, sigma, k_left, D, offset, pack, perm, perm_bytes, x, y, nullptr, Red{},
                    xlen);
}

// The reducing form (y = A x, then x.y and, with b, x.b into the solver's
// deterministic reduction), on a fixed grid of four blocks per SM.
__global__ void __launch_bounds__(TPB, 4)
    k_spmv_w64_dot(int n, int C, int sigma, long long k_left, int D,
                   const int64_t *__restrict__ offset, const unsigned long long *__restrict__ pack,
                   const void *__restrict__ perm, int perm_bytes, const double *__restrict__ x,
                   double *__restrict__ y, const double *__restrict__ b, Red red, int xlen) {
    w64_rows<true>(n, C, sigma, k_left, D, offset, pack, perm, perm_bytes, x, y, b, red, xlen);
}

// 1 / a_ii of a square matrix (1 where the diagonal is absent or 0).
__global__ void __launch_bounds__(TPB)
    k_inv_diag_w64(int n, int C, int sigma, long long k_left, int D,
                   const int64_t *__restrict__ offset, const unsigned long long *__restrict__ pack,
                   const void *__restrict__ perm, int perm_bytes, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long dmask = (1ull << D) - 1ull;
    const unsigned long long vmask = ~((2ull << D) - 1ull);
    const int k = i / C, l = i - k * C;
    const int64_t s = offset[k];
    const int w = (int)((offset[k + 1] - s) / C);
    const int io = orig_row(i, sigma, perm, perm_bytes);
    long long c = left_offset(i, sigma, k_left);
    double d = 0.0;
    for (int j = 0; j < w; ++j) {
        const unsigned long long wd = pack[s + (int64_t)j * C + l];
        const bool f = (wd & 1ull) != 0ull;
        c += (long long)((wd >> 1) & (f ? dmask : 0x7fffffffffffffffull));
        if (f && c == io) d = __longlong_as_double((long long)(wd & vmask));
    }
    out[io] = d != 0.0 ? 1.0 / d : 1.0;
}

inline unsigned rows_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TPB - 1) / TPB); }

}  // namespace

packsell_status spmv_w64_impl(const Matrix &A, const double *x, double *y, cudaStream_t s) {
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    const int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    const cudaError_t e = launch_pdl(k_spmv_w64, rows_grid(A.n), TPB, s, (int)A.n, A.p.C,
                                     A.p.sigma, (long long)A.p.k_left, A.p.D,
                                     (const int64_t *)A.offset,
                                     (const unsigned long long *)A.pack64, perm, pb, x, y,
                                     (int)A.m);
    if (e != cudaSuccess) return cuda_fail(e, "packsell_spmv_f64 (64-bit words)");
    PS_LAUNCH_CHECK("packsell_spmv_f64 (64-bit words)");
    return PACKSELL_OK;
}

packsell_status spmv_dot_w64(const Matrix &A, const double *x, double *y, const double *b,
                             const Red &red, unsigned grid, cudaStream_t s) {
    const cudaError_t e = launch_pdl(k_spmv_w64_dot, grid, TPB, s, (int)A.n, A.p.C, A.p.sigma,
                                     (long long)A.p.k_left, A.p.D, (const int64_t *)A.offset,
                                     (const unsigned long long *)A.pack64,
                                     (const void *)A.perm, A.perm_bytes, x, y, b, red,
                                     (int)A.m);
    if (e != cudaSuccess) return cuda_fail(e, "spmv_dot_f64 (64-bit words)");
    PS_LAUNCH_CHECK("spmv_dot_f64 (64-bit words)");
    return PACKSELL_OK;
}

packsell_status inv_diag_w64(const Matrix &A, double *out, cudaStream_t s) {
    if (A.n == 0) return PACKSELL_OK;
    k_inv_diag_w64<<<rows_grid(A.n), TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma,
                                                  (long long)A.p.k_left, A.p.D, A.offset,
                                                  (const unsigned long long *)A.pack64, A.perm,
                                                  A.perm_bytes, out);
    PS_LAUNCH_CHECK("packsell_inv_diag (64-bit words)");
    return PACKSELL_OK;
}

}  // namespace packsell
