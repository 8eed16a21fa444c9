// SpMV on 16-bit PackSELL words (PACKSELL_FMT_W16_E4M3; W = 16, D = 7,
// §4.2.1's other word sizes): bit 0 flag, bits 1..7 delta, bits 8..15 an FP8
// E4M3 value; a dummy's delta field is 15 bits. Thread-per-row with the words
// of a round loaded at once (16-bit cache-streaming loads, rounds fitted to
// the widest slice, a constant word stride for C = 32), FP32 fused
// multiply-adds in stored order: the same chain as the 32-bit words'
// kernels, on the E4M3 values widened exactly to FP32. Launched with
// programmatic dependent launch.
#include <cuda_fp16.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int TPB = 256;

// The E4M3 value of a 16-bit word (code in bits 8..15), exactly: E4M3 and
// binary16 differ in exponent bias by 8 and in fraction width, so the code's
// 7 magnitude bits placed at binary16 bits 7..13 (sign at bit 15) give a
// binary16 number equal to the E4M3 value times 2^-8, normal and subnormal
// codes alike; the product by 2^8 is exact.
__device__ __forceinline__ float w16_value(uint32_t w) {
    const unsigned short h = (unsigned short)((w & 0x8000u) | ((w >> 1) & 0x3F80u));
    return __half2float(__ushort_as_half(h)) * 256.0f;
}

template <int PF, int MINB, bool PERM, bool C32>
__global__ void __launch_bounds__(TPB, MINB)
    k_spmv_w16(int n, int Cr, int sigma, int sig_shift, long long k_left,
               const int64_t *__restrict__ offset, const uint16_t *__restrict__ pack,
               const void *__restrict__ perm, int perm_bytes, const float *__restrict__ x,
               float *__restrict__ y, int xlen) {
    const int C = C32 ? 32 : Cr;  // a constant word stride when C = 32
    grid_dep_launch();  // one pass over the rows: signal at block start
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k = i / C, l = i - k * C;
    const int64_t s = offset[k];
    const int w = (int)((offset[k + 1] - s) / C);
    const unsigned short *__restrict__ pp = reinterpret_cast<const unsigned short *>(pack) + s + l;
    const int blk = sig_shift >= 0 ? (i >> sig_shift) << sig_shift : (i / sigma) * sigma;
    int c = (k_left < blk) ? (int)(blk - k_left) : 0;
    float t = 0.f;
    if (w <= 0) grid_dep_wait();
    for (int j0 = 0; j0 < w; j0 += PF) {
        const int wr = w - j0;
        uint32_t wd[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u)
            wd[u] = (u < wr) ? (uint32_t)__ldcs(pp + (C32 ? (j0 + u) * 32 : (int64_t)(j0 + u) * C)) : 0u;
        // the first round's words load before the wait; x and y after it
        if (j0 == 0) grid_dep_wait();
        bool f[PF];
        float xv[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            f[u] = (wd[u] & 1u) != 0u;
            c += (int)((wd[u] >> 1) & (f[u] ? 0x7Fu : 0x7FFFu));
            if (f[u]) xv[u] = PS_IN_RANGE(c, xlen) ? __ldg(x + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (f[u]) t = fmaf(w16_value(wd[u]), xv[u], t);
    }
    int io = i;
    if (PERM) io = blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[i]
                                          : (int)((const uint16_t *)perm)[i]);
    y[io] = t;
}

template <int PF, int MINB>
cudaError_t launch_w16(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    const unsigned g = (unsigned)((A.n + TPB - 1) / TPB);
    const bool c32 = A.p.C == 32;
    // other slice heights keep 64-bit word offsets: fewer blocks per SM
    auto kern = pb ? (c32 ? k_spmv_w16<PF, MINB, true, true> : k_spmv_w16<PF, 3, true, false>)
                   : (c32 ? k_spmv_w16<PF, MINB, false, true> : k_spmv_w16<PF, 3, false, false>);
    return launch_pdl(kern, g, TPB, s, (int)A.n, A.p.C, sg, sh, A.p.k_left,
                      (const int64_t *)A.offset, (const uint16_t *)A.pack16, perm, pb, x, y,
                      (int)A.m);
}

}  // namespace

packsell_status spmv_w16_impl(const Matrix &A, const float *x, float *y, cudaStream_t s) {
    if (!is_w16(A.p.format) || !A.pack16)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: not a 16-bit-word matrix");
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    const int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    const int w = A.max_width;
    const cudaError_t e = w <= 8    ? launch_w16<8, 6>(A, perm, pb, x, y, s)
                          : w <= 12 ? launch_w16<12, 5>(A, perm, pb, x, y, s)
                                    : launch_w16<16, 5>(A, perm, pb, x, y, s);
    if (e != cudaSuccess) return cuda_fail(e, "packsell_spmv (16-bit words)");
    PS_LAUNCH_CHECK("packsell_spmv (16-bit words)");
    return PACKSELL_OK;
}

}  // namespace packsell
