// SpMV with binary16 vectors, the paper's FP16 SpMV configuration (§5.1.1:
// x and y in FP16): x_c is read as binary16 and widened exactly to FP32, each
// row is summed with FP32 fused multiply-adds in stored order (the same chain
// as packsell_spmv with x widened), and y_i is rounded to binary16 (nearest,
// ties to even). Thread-per-row with the words of a round loaded at once
// (rounds fitted to the widest slice), for PackSELL matrices with C = 32.
#include <cuda_fp16.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int TPB = 256;

template <int FMT, int PF, bool PERM>
__global__ void __launch_bounds__(TPB)
    k_spmv_x16(int n, int sigma, int sig_shift, long long k_left,
               const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
               const void *__restrict__ perm, int perm_bytes, Decode dc,
               const __half *__restrict__ x, __half *__restrict__ y) {
    grid_dep_launch();  // one pass over the rows: signal at block start
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = i >> 5;
    const int64_t s = offset[k];
    const int w = (int)((offset[k + 1] - s) >> 5);
    const uint32_t *__restrict__ pp = pack + s + (i & 31);
    const int blk = sig_shift >= 0 ? (i >> sig_shift) << sig_shift : (i / sigma) * sigma;
    int c = (k_left < blk) ? (int)(blk - k_left) : 0;
    float t = 0.f;
    if (w <= 0) grid_dep_wait();
    for (int j0 = 0; j0 < w; j0 += PF) {
        const int wr = w - j0;
        uint32_t wd[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) wd[u] = (u < wr) ? ldg_stream(pp + (j0 + u) * 32) : 0u;
        // the first round's words load before the wait; x and y after it
        if (j0 == 0) grid_dep_wait();
        bool f[PF];
        float xv[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            f[u] = (wd[u] & 1u) != 0u;
            c += (int)((wd[u] >> 1) & (f[u] ? dc.dmask : 0x7fffffffu));
            if (f[u]) xv[u] = PS_IN_RANGE(c, dc.xlen) ? __half2float(__ldg(x + c)) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (f[u]) t = fmaf(word_value<FMT>(wd[u], dc), xv[u], t);
    }
    int io = i;
    if (PERM) io = blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[i]
                                          : (int)((const uint16_t *)perm)[i]);
    y[io] = __float2half_rn(t);
}

template <int FMT, int PF>
cudaError_t launch_x16(const Matrix &A, const void *perm, int pb, const __half *x, __half *y,
                       cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    const unsigned g = (unsigned)((A.n + TPB - 1) / TPB);
    return launch_pdl(pb ? k_spmv_x16<FMT, PF, true> : k_spmv_x16<FMT, PF, false>, g, TPB, s,
                      (int)A.n, sg, sh, A.p.k_left, (const int64_t *)A.offset,
                      (const uint32_t *)A.pack, perm, pb, make_decode(A), x, y);
}

template <int FMT>
cudaError_t launch_x16_pf(const Matrix &A, const void *perm, int pb, const __half *x, __half *y,
                          cudaStream_t s) {
    const int w = A.max_width;
    if (w <= 8) return launch_x16<FMT, 8>(A, perm, pb, x, y, s);
    if (w <= 12) return launch_x16<FMT, 12>(A, perm, pb, x, y, s);
    return launch_x16<FMT, 16>(A, perm, pb, x, y, s);
}

}  // namespace

packsell_status spmv_x16_impl(const Matrix &A, const uint16_t *x, uint16_t *y, cudaStream_t s) {
    if (!is_packed(A.p.format) || A.p.C != 32)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_spmv_x16: needs a PackSELL matrix with C = 32");
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    const int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    const __half *xh = reinterpret_cast<const __half *>(x);
    __half *yh = reinterpret_cast<__half *>(y);
    const cudaError_t e = A.p.format == PACKSELL_FMT_FP16
                              ? launch_x16_pf<PACKSELL_FMT_FP16>(A, perm, pb, xh, yh, s)
                              : launch_x16_pf<PACKSELL_FMT_E8MY>(A, perm, pb, xh, yh, s);
    if (e != cudaSuccess) return cuda_fail(e, "packsell_spmv_x16");
    PS_LAUNCH_CHECK("packsell_spmv_x16");
    return PACKSELL_OK;
}

}  // namespace packsell
