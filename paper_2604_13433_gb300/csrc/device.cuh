// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "internal.h"

namespace packsell {

// Record the first error seen by any thread (code and index).
__device__ __forceinline__ void dev_fail(DevStatus *st, int code, long long index) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = index;
}

// Left offset of Eq. 4: the same for every row of a block of sigma rows, so it
// can be computed from the storage row index.
__device__ __forceinline__ int left_offset(int i, int sigma, long long k_left) {
    long long b = (long long)(i / sigma) * sigma;
    return (k_left < b) ? (int)(b - k_left) : 0;
}

// Original row of storage row i (§3): block base + perm.
__device__ __forceinline__ int orig_row(int i, int sigma, const void *perm, int perm_bytes) {
    if (perm_bytes == 0) return i;
    int b = (i / sigma) * sigma;
    int q = (perm_bytes == 1) ? (int)((const uint8_t *)perm)[i] : (int)((const uint16_t *)perm)[i];
    return b + q;
}

// Decoded word: flag, delta and value. The delta field is D bits wide when the
// flag is set and 31 bits wide otherwise (§4.2.1); the value is the upper
// 31 - D bits read as FP16 (bits 16..31) or as an FP32 pattern (E8MY).
template <int FMT>
struct Word {
    __device__ __forceinline__ static void decode(uint32_t w, uint32_t dmask, uint32_t vmask,
                                                  uint32_t &flag, uint32_t &delta, float &v) {
        flag = w & 1u;
        delta = (w >> 1) & (flag ? dmask : 0x7fffffffu);
        if (FMT == PACKSELL_FMT_FP16) {
            v = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
        } else {
            v = __uint_as_float(w & vmask);
        }
    }
};

__device__ __forceinline__ uint32_t ldg_stream(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

}  // namespace packsell
