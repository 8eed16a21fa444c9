// Device helpers shared by the library's kernels.
#pragma once

#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#include <utility>

#include "internal.h"

namespace packsell {

// Record the first error seen by any thread (code and index).
__device__ __forceinline__ void dev_fail(DevStatus *st, int code, long long index) {
    if (atomicCAS(&st->code, 0, code) == 0) st->index = index;
}

// ---- the bounds-check build (compiled with -DPACKSELL_CHECKS) ----
// Every x (or X row) gather at a column decoded from the words, and every
// write the decoded words steer (the transpose's scatter, the pattern
// product's output), first checks its index against the array's length; an
// index out of range skips the access and is counted, with the first such
// index kept. Each translation unit has its own counters (a device variable
// per unit, since the library is not built for relocatable device code);
// packsell_check_status sums them through the readers that the units
// register at load time. The regular build compiles every check to `true`.
#ifdef PACKSELL_CHECKS
namespace {
__device__ unsigned long long g_checks[2];  // out-of-range accesses; first index

__device__ __forceinline__ bool check_in_range(long long i, long long len) {
    if (i >= 0 && i < len) return true;
    if (atomicAdd(&g_checks[0], 1ull) == 0ull) g_checks[1] = (unsigned long long)i;
    return false;
}

// read and clear this unit's counters (host; the current device)
cudaError_t read_checks_here(unsigned long long *count, long long *first) {
    unsigned long long h[2] = {0ull, 0ull};
    cudaError_t e = cudaMemcpyFromSymbol(h, g_checks, sizeof h);
    if (e != cudaSuccess) return e;
    *count = h[0];
    *first = (long long)h[1];
    const unsigned long long z[2] = {0ull, 0ull};
    return cudaMemcpyToSymbol(g_checks, z, sizeof z);
}

struct ChecksRegistrar {
    ChecksRegistrar() { register_checks_reader(&read_checks_here); }
};
ChecksRegistrar g_checks_registrar;
}  // namespace
#define PS_IN_RANGE(i, len) ::packsell::check_in_range((long long)(i), (long long)(len))
#else
#define PS_IN_RANGE(i, len) true
#endif

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
// Fixed point: the V-bit two's-complement field (an arithmetic shift
// sign-extends it) times the matrix's 2^s; exact, since |q| < 2^24.
template <int FMT>
struct Word {
    __device__ __forceinline__ static void decode(uint32_t w, uint32_t dmask, uint32_t vmask,
                                                  uint32_t &flag, uint32_t &delta, float &v,
                                                  int vshift = 0, float vscale = 1.f) {
        flag = w & 1u;
        delta = (w >> 1) & (flag ? dmask : 0x7fffffffu);
        if (FMT == PACKSELL_FMT_FP16) {
            v = __half2float(__ushort_as_half((unsigned short)(w >> 16)));
        } else if (FMT == PACKSELL_FMT_FIXED) {
            v = (float)((int32_t)w >> vshift) * vscale;
        } else {
            v = __uint_as_float(w & vmask);
        }
    }
};

// Masks of a matrix's word layout: delta bits (flag 1) and value bits; for
// fixed point the shift of the value field and the matrix's scale 2^s; the
// length of x (m: what the bounds-check build checks columns against).
struct Decode {
    uint32_t dmask, vmask;
    int vshift;
    float vscale;
    int xlen;
};

inline Decode make_decode(const Matrix &A) {
    Decode d;
    d.dmask = (1u << A.p.D) - 1u;
    d.vmask = ~((2u << A.p.D) - 1u);
    d.vshift = A.p.D + 1;
    d.vscale = ldexpf(1.0f, A.value_exp);
    d.xlen = (int)A.m;
    return d;
}

// One word: add its delta to c; if it carries a value, gather x_c.
template <int FMT>
__device__ __forceinline__ void word_gather(uint32_t wd, Decode dc, const float *__restrict__ x,
                                            int &c, bool &f, float &xv) {
    f = (wd & 1u) != 0u;
    c += (int)((wd >> 1) & (f ? dc.dmask : 0x7fffffffu));
    if (f) xv = PS_IN_RANGE(c, dc.xlen) ? __ldg(x + c) : 0.f;
}

// The value a word carries (FP16 in the upper half, or E8MY bits).
template <int FMT>
__device__ __forceinline__ float word_value(uint32_t wd, Decode dc) {
    if (FMT == PACKSELL_FMT_FP16) return __high2float(*reinterpret_cast<const __half2 *>(&wd));
    if (FMT == PACKSELL_FMT_FIXED) return (float)((int32_t)wd >> dc.vshift) * dc.vscale;
    return __uint_as_float(wd & dc.vmask);
}

// A word of the packed stream is read once: a cache-streaming load (evict
// first) keeps the words from taking L1 and L2 lines from the x gathers
// (with plain loads the words evict x and the gathers fall through to L2).
__device__ __forceinline__ uint32_t ldg_stream(const uint32_t *p) { return __ldcs(p); }

// ---- programmatic dependent launch (sm_90 and later) ----
// A kernel launched by launch_pdl may be scheduled while the previous kernel
// of its stream drains. grid_dep_sync first waits until that kernel has
// completed and its memory is visible (at once when there is none), then
// lets the next kernel of the stream be scheduled once every block of this
// grid has passed the same point (or exited). Signalling only after the
// wait keeps at most one kernel waiting ahead: signalled at block start, a
// chain of persistent-grid solver kernels queued up on the SMs and slowed the
// one running. The product kernels read only the matrix (complete when
// encode or import returns, never written by a product) before the call,
// and x, y and solver state after it.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dep_sync() {
    grid_dep_wait();
    grid_dep_launch();
}
// A grid that covers the rows once (more blocks than fit at a time) may
// signal at block start instead: its dependents can then only be scheduled
// once its last wave has started.

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s,
                       Args &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---- mbarrier and bulk-copy (TMA engine) primitives, inline PTX ----
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// make mbarrier initialisation visible to the async proxy
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes to the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned) completing `bytes` transactions on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}" : "=r"(ok) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity: at most `limit` polls;
// false if it ran out. The kernels' waits for data take the limit set by
// packsell_set_wait_limit (kWaitLimit by default); the drain of copies
// already issued, before a kernel that gave up returns, always takes
// kWaitLimit, so that every copy lands before the block's shared memory is
// released.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t limit = kWaitLimit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

}  // namespace packsell
