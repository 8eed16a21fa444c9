// PackSELL / SELL encoder on the device.
//
// Steps (§4.1-§4.3, §3), each a kernel on the caller's stream:
//   1. check the CSR (row pointer, sorted in-range columns) and take the
//      lower bandwidth k_left = max(0, max_ij (i - j)) used by Eq. 4;
//   2. quantise every value into its word's value field (§4.2.2);
//   3. count stored words per row: nonzeros plus one dummy before every
//      nonzero whose delta (Eq. 2, first delta from Eq. 4) needs more than D
//      bits (§4.3);
//   4. sort rows by stored words, descending and stable, inside blocks of
//      sigma rows (§3, §4.3) -> perm;
//   5. slice widths (max over C rows) and their exclusive scan -> offset;
//   6. (host reads the word total once) scatter words column-major per slice,
//      zero words as padding.
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

constexpr int TPB = 256;

inline int blocks_for(int64_t n, int tpb = TPB) {
    int64_t b = (n + tpb - 1) / tpb;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 30));
}

__global__ void k_check_rows(int n, int64_t m, int64_t nnz, const int64_t *__restrict__ rowptr,
                             const int32_t *__restrict__ col, unsigned long long *kl,
                             DevStatus *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        if (rowptr[0] != 0) dev_fail(st, PACKSELL_ERR_INVALID_ARG, -1);
        if (rowptr[n] != nnz) dev_fail(st, PACKSELL_ERR_INVALID_ARG, -2);
    }
    unsigned dmax = 0;  // this row's i - (first column), if positive
    if (i < n) {
        int64_t a = rowptr[i], b = rowptr[i + 1];
        if (a < 0 || b < a || b > nnz) {
            dev_fail(st, PACKSELL_ERR_INVALID_ARG, i);
        } else {
            int prev = -1;
            bool ok = true;
            for (int64_t p = a; p < b; ++p) {
                int c = col[p];
                if (c < 0 || (int64_t)c >= m) {
                    dev_fail(st, PACKSELL_ERR_RANGE, p);
                    ok = false;
                    break;
                }
                if (c <= prev) {
                    dev_fail(st, PACKSELL_ERR_UNSORTED, p);
                    ok = false;
                    break;
                }
                prev = c;
            }
            if (ok && b > a && i > col[a]) dmax = (unsigned)(i - col[a]);
        }
    }
    // one atomic per warp: millions of atomics on one address serialise
    dmax = __reduce_max_sync(0xffffffffu, dmax);
    if ((threadIdx.x & 31) == 0 && dmax) atomicMax(kl, (unsigned long long)dmax);
}

// FP16 value field: binary16 in bits 16..31, round to nearest even.
template <typename T>
__device__ __forceinline__ int field_fp16(T v, uint32_t &field) {
    if (!isfinite(v)) return PACKSELL_ERR_NONFINITE;
    __half h = (sizeof(T) == 4) ? __float2half_rn((float)v) : __double2half((double)v);
    if (__hisinf(h)) return PACKSELL_ERR_RANGE;
    field = (uint32_t)__half_as_ushort(h) << 16;
    return 0;
}

// E8MY value field from an FP32 value: round half away from zero at bit D+1
// of the FP32 pattern by adding half a step to the magnitude and clearing
// the low D+1 bits (a carry moves into the exponent on its own).
__device__ __forceinline__ int field_e8my(float v, int D, uint32_t &field) {
    uint32_t b = __float_as_uint(v);
    uint32_t mag = b & 0x7fffffffu;
    if (mag >= 0x7f800000u) return PACKSELL_ERR_NONFINITE;
    uint32_t r = (mag + (1u << D)) & ~((2u << D) - 1u);
    if (r >= 0x7f800000u) return PACKSELL_ERR_RANGE;
    field = (b & 0x80000000u) | r;
    return 0;
}

// E8MY value field from an FP64 value, rounded once from the double: the
// step is 2^(e - 23 + D) for v in [2^(e-1), 2^e), with e held at FP32's
// smallest normal binade below it; v / step is rounded half away from zero.
__device__ __forceinline__ int field_e8my(double v, int D, uint32_t &field) {
    if (!isfinite(v)) return PACKSELL_ERR_NONFINITE;
    if (v == 0.0) {
        field = signbit(v) ? 0x80000000u : 0u;
        return 0;
    }
    int e;
    frexp(v, &e);
    if (e < -125) e = -125;
    if (e > 129) return PACKSELL_ERR_RANGE;
    double step = ldexp(1.0, e - 23 + D);
    double r = round(v / step) * step;
    if (fabs(r) >= 0x1p128) return PACKSELL_ERR_RANGE;
    field = __float_as_uint((float)r) & ~((2u << D) - 1u);
    return 0;
}

// FP8 E4M3 code (16-bit words) with the hardware conversion, round to
// nearest even from the input precision. Saturation is only a fallback: a
// magnitude above 464 (halfway from 448, the largest finite value, to the
// next step) would round past 448 and is reported as out of range.
template <typename T>
__device__ __forceinline__ int field_e4m3(T v, uint32_t &field) {
    if (!isfinite(v)) return PACKSELL_ERR_NONFINITE;
    if (fabs((double)v) > 464.0) return PACKSELL_ERR_RANGE;
    field = (sizeof(T) == 4) ? (uint32_t)__nv_cvt_float_to_fp8((float)v, __NV_SATFINITE, __NV_E4M3)
                             : (uint32_t)__nv_cvt_double_to_fp8((double)v, __NV_SATFINITE, __NV_E4M3);
    return 0;
}

// Fixed-point value field: q = v / 2^s rounded half away from zero (exact
// scaling and rounding in double), as a V = 31 - D bit two's-complement
// integer in bits D+1..31; |q| above 2^(V-1) - 1 is out of range.
template <typename T>
__device__ __forceinline__ int field_fixed(T v, int D, int s, uint32_t &field) {
    if (!isfinite(v)) return PACKSELL_ERR_NONFINITE;
    const int V = 31 - D;
    const double q = round(ldexp((double)v, -s));
    if (fabs(q) > ldexp(1.0, V - 1) - 1.0) return PACKSELL_ERR_RANGE;
    const uint32_t bits = (uint32_t)((unsigned long long)(long long)q & ((1ull << V) - 1ull));
    field = bits << (D + 1);
    return 0;
}

// the largest finite |v| (as the bits of a non-negative double, which order
// as integers)
template <typename T>
__global__ void k_absmax(int64_t nnz, const T *__restrict__ val, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs((double)val[p]);
        if (isfinite(a)) m = max(m, (unsigned long long)__double_as_longlong(a));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

template <typename T>
__global__ void k_quantize(int64_t nnz, const T *__restrict__ val, int fmt, int D,
                           uint32_t *__restrict__ field, DevStatus *st, int s = 0) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        uint32_t f = 0;
        int err = (fmt == PACKSELL_FMT_FP16) ? field_fp16(val[p], f)
                  : (fmt == PACKSELL_FMT_W16_E4M3) ? field_e4m3(val[p], f)
                  : (fmt == PACKSELL_FMT_FIXED)    ? field_fixed(val[p], D, s, f)
                                                   : field_e8my(val[p], D, f);
        if (err) dev_fail(st, err, p);
        field[p] = f;
    }
}

// E11MY field of a 64-bit word (the value bits D+1..63): the binary64
// pattern of v with half a unit of the D + 1 dropped bits added to its
// magnitude, then those bits cleared (round half away from zero, subnormals
// on the grid of the smallest normal binade); an all-ones exponent after the
// rounding is out of range.
template <typename T>
__device__ __forceinline__ int field_e11my(T v, int D, unsigned long long &field) {
    const double d = (double)v;
    if (!isfinite(d)) return PACKSELL_ERR_NONFINITE;
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned long long sign = b & 0x8000000000000000ull;
    unsigned long long mag = b & 0x7fffffffffffffffull;
    mag = (mag + (1ull << D)) & ~((2ull << D) - 1ull);
    if ((mag >> 52) == 0x7ffull) return PACKSELL_ERR_RANGE;
    field = sign | mag;
    return 0;
}

template <typename T>
__global__ void k_quantize64(int64_t nnz, const T *__restrict__ val, int D,
                             unsigned long long *__restrict__ field, DevStatus *st) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long f = 0;
        const int err = field_e11my(val[p], D, f);
        if (err) dev_fail(st, err, p);
        field[p] = f;
    }
}

__device__ __forceinline__ long long resolve_k_left(long long user, const unsigned long long *kl) {
    return user >= 0 ? user : (long long)*kl;
}

// Stored words per original row; for SELL (packed = 0) just the row length.
__global__ void k_count_words(int n, const int64_t *__restrict__ rowptr,
                              const int32_t *__restrict__ col, int sigma, long long k_left_user,
                              const unsigned long long *kl, int D, int packed, int W,
                              int32_t *__restrict__ words, unsigned long long *total,
                              DevStatus *st) {
    // a malformed row pointer (found by k_check_rows) must not be walked
    if (st->code != 0) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    long long cnt = 0;
    if (i < n) {
        int64_t a = rowptr[i], b = rowptr[i + 1];
        cnt = b - a;
        if (packed) {
            long long prev = left_offset(i, sigma, resolve_k_left(k_left_user, kl));
            long long lim = 1ll << D;
            // a dummy's delta field: W - 1 bits
            const long long dmax = W >= 64 ? 0x7fffffffffffffffll : (1ll << (W - 1)) - 1;
            for (int64_t p = a; p < b; ++p) {
                long long d = (long long)col[p] - prev;
                if (d < 0) {
                    dev_fail(st, PACKSELL_ERR_INVALID_ARG, p);
                    break;
                }
                // dummies while the delta does not fit in D bits, each taking
                // at most dmax of it (one dummy with 32-bit words)
                while (d >= lim) {
                    d -= d < dmax ? d : dmax;
                    ++cnt;
                }
                prev = col[p];
            }
        }
        if (cnt > 0x7fffffffll) {
            dev_fail(st, PACKSELL_ERR_RANGE, i);
            cnt = 0;
        }
        words[i] = (int32_t)cnt;
    }
    // warp-reduce the word total, one atomic per warp
    unsigned long long v = (unsigned long long)cnt;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// Stable descending sort by stored words inside each block of sigma rows:
// rank(t) = #{u : w_u > w_t} + #{u < t : w_u == w_t}. Storage row b0 + rank
// holds original row b0 + t, recorded as perm[b0 + rank] = t (§3).
constexpr int SORT_TILE = 4096;

__global__ void k_sigma_sort(int n, int sigma, const int32_t *__restrict__ words, void *perm,
                             int perm_bytes, int32_t *__restrict__ words_st) {
    __shared__ int32_t tile[SORT_TILE];
    int64_t b0 = (int64_t)blockIdx.x * sigma;
    int len = (int)((n - b0 < sigma) ? (n - b0) : sigma);
    for (int tb = 0; tb < len; tb += blockDim.x) {
        int t = tb + threadIdx.x;
        int key = (t < len) ? words[b0 + t] : 0;
        int rank = 0;
        for (int ub = 0; ub < len; ub += SORT_TILE) {
            int cnt = (len - ub < SORT_TILE) ? (len - ub) : SORT_TILE;
            __syncthreads();
            for (int u = threadIdx.x; u < cnt; u += blockDim.x) tile[u] = words[b0 + ub + u];
            __syncthreads();
            if (t < len) {
                for (int u = 0; u < cnt; ++u) {
                    int ku = tile[u];
                    rank += (ku > key) | ((ku == key) & (ub + u < t));
                }
            }
        }
        if (t < len) {
            int64_t dst = b0 + rank;
            words_st[dst] = key;
            if (perm_bytes == 1) ((uint8_t *)perm)[dst] = (uint8_t)t;
            else if (perm_bytes == 2) ((uint16_t *)perm)[dst] = (uint16_t)t;
        }
    }
}

__global__ void k_copy_words(int n, const int32_t *__restrict__ w, int32_t *__restrict__ o) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) o[i] = w[i];
}

__global__ void k_slice_widths(int64_t S, int n, int C, const int32_t *__restrict__ words_st,
                               int64_t *__restrict__ slice_words, int *max_width) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= S) return;
    int w = 0;
    int64_t r0 = k * C, r1 = (r0 + C < n) ? r0 + C : n;
    for (int64_t r = r0; r < r1; ++r) w = max(w, words_st[r]);
    slice_words[k] = (int64_t)C * w;
    atomicMax(max_width, w);
}

// ---- exclusive scan of int64 (3 phases, recursive on the block sums) ----
constexpr int SCAN_TPB = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_CHUNK = SCAN_TPB * SCAN_ITEMS;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *warp_sums,
                                                          long long &total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        long long s = (lane < nw) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) warp_sums[lane] = s;  // inclusive warp prefix
    }
    __syncthreads();
    long long before = (wid > 0) ? warp_sums[wid - 1] : 0;
    total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + inc - v;
}

__global__ void k_scan_block_sums(int64_t S, const int64_t *__restrict__ in,
                                  int64_t *__restrict__ sums) {
    __shared__ long long ws[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    long long v = 0;
    for (int q = 0; q < SCAN_ITEMS; ++q)
        if (base + q < S) v += in[base + q];
    long long total;
    block_exclusive_scan(v, ws, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// out[i] = carry[block] + exclusive prefix inside the block; out[S] = total.
__global__ void k_scan_apply(int64_t S, const int64_t *__restrict__ in,
                             const int64_t *__restrict__ carry, int64_t *__restrict__ out) {
    __shared__ long long ws[32];
    int64_t base = (int64_t)blockIdx.x * SCAN_CHUNK + (int64_t)threadIdx.x * SCAN_ITEMS;
    long long v[SCAN_ITEMS], s = 0;
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        v[q] = (base + q < S) ? in[base + q] : 0;
        s += v[q];
    }
    long long total;
    long long pre = block_exclusive_scan(s, ws, total) + (carry ? carry[blockIdx.x] : 0);
    for (int q = 0; q < SCAN_ITEMS; ++q) {
        if (base + q < S) out[base + q] = pre;
        pre += v[q];
    }
    if (base < S && base + SCAN_ITEMS >= S) out[S] = pre;  // thread holding the last item
}

packsell_status scan_exclusive(const int64_t *in, int64_t *out, int64_t S, cudaStream_t s) {
    if (S <= 0) {
        PS_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return PACKSELL_OK;
    }
    int64_t B = (S + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (B == 1) {
        k_scan_apply<<<1, SCAN_TPB, 0, s>>>(S, in, nullptr, out);
        PS_LAUNCH_CHECK("k_scan_apply");
        return PACKSELL_OK;
    }
    int64_t *sums = nullptr, *carry = nullptr;
    PS_CUDA(cudaMallocAsync((void **)&sums, sizeof(int64_t) * B, s));
    PS_CUDA(cudaMallocAsync((void **)&carry, sizeof(int64_t) * (B + 1), s));
    k_scan_block_sums<<<(unsigned)B, SCAN_TPB, 0, s>>>(S, in, sums);
    PS_LAUNCH_CHECK("k_scan_block_sums");
    packsell_status st = scan_exclusive(sums, carry, B, s);
    if (st != PACKSELL_OK) return st;
    k_scan_apply<<<(unsigned)B, SCAN_TPB, 0, s>>>(S, in, carry, out);
    PS_LAUNCH_CHECK("k_scan_apply");
    PS_CUDA(cudaFreeAsync(sums, s));
    PS_CUDA(cudaFreeAsync(carry, s));
    return PACKSELL_OK;
}

// Scatter one storage row per thread into the column-major slice layout:
// word j of storage row i sits at offset[k] + j*C + l (k = i / C, l = i % C).
// Threads past n (phantom rows of the last slice) write padding only.
__global__ void k_scatter_packed(int n, int64_t rows_total, int C, int sigma, long long k_left_user,
                                 const unsigned long long *kl, int D,
                                 const int64_t *__restrict__ rowptr,
                                 const int32_t *__restrict__ col,
                                 const uint32_t *__restrict__ field, const void *perm,
                                 int perm_bytes, const int64_t *__restrict__ offset,
                                 uint32_t *__restrict__ pack) {
    int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ii >= rows_total) return;
    int i = (int)ii;
    int64_t k = ii / C;
    int l = (int)(ii - k * C);
    int64_t s = offset[k];
    int64_t w = (offset[k + 1] - s) / C;
    uint32_t *dst = pack + s + l;
    int64_t j = 0;
    if (i < n) {
        int r = orig_row(i, sigma, perm, perm_bytes);
        long long prev = left_offset(i, sigma, resolve_k_left(k_left_user, kl));
        long long lim = 1ll << D;
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) {
            long long d = (long long)col[p] - prev;
            if (d >= lim) {
                dst[j * C] = (uint32_t)d << 1;  // dummy: flag 0, 31-bit delta
                ++j;
                d = 0;
            }
            dst[j * C] = field[p] | ((uint32_t)d << 1) | 1u;
            ++j;
            prev = col[p];
        }
    }
    for (; j < w; ++j) dst[j * C] = 0u;
}

// 64-bit words: field | (d << 1) | 1 with a value, (d << 1) for a dummy (63
// delta bits: one dummy covers any gap), 0 for padding.
__global__ void k_scatter_w64(int n, int64_t rows_total, int C, int sigma, long long k_left_user,
                              const unsigned long long *kl, int D,
                              const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                              const unsigned long long *__restrict__ field, const void *perm,
                              int perm_bytes, const int64_t *__restrict__ offset,
                              unsigned long long *__restrict__ pack) {
    int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ii >= rows_total) return;
    int i = (int)ii;
    int64_t k = ii / C;
    int l = (int)(ii - k * C);
    int64_t s = offset[k];
    int64_t w = (offset[k + 1] - s) / C;
    unsigned long long *dst = pack + s + l;
    int64_t j = 0;
    if (i < n) {
        int r = orig_row(i, sigma, perm, perm_bytes);
        long long prev = left_offset(i, sigma, resolve_k_left(k_left_user, kl));
        const long long lim = 1ll << D;
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) {
            long long d = (long long)col[p] - prev;
            if (d >= lim) {
                dst[j * C] = (unsigned long long)d << 1;
                ++j;
                d = 0;
            }
            dst[j * C] = field[p] | ((unsigned long long)d << 1) | 1ull;
            ++j;
            prev = col[p];
        }
    }
    for (; j < w; ++j) dst[j * C] = 0ull;
}

// 16-bit words: (code << 8) | (d << 1) | 1 with a value, (q << 1) for a
// dummy of q < 2^15, 0 for padding; dummies while the delta is 2^7 or more.
__global__ void k_scatter_w16(int n, int64_t rows_total, int C, int sigma, long long k_left_user,
                              const unsigned long long *kl, const int64_t *__restrict__ rowptr,
                              const int32_t *__restrict__ col, const uint32_t *__restrict__ code,
                              const void *perm, int perm_bytes, const int64_t *__restrict__ offset,
                              uint16_t *__restrict__ pack) {
    int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ii >= rows_total) return;
    int i = (int)ii;
    int64_t k = ii / C;
    int l = (int)(ii - k * C);
    int64_t s = offset[k];
    int64_t w = (offset[k + 1] - s) / C;
    uint16_t *dst = pack + s + l;
    int64_t j = 0;
    if (i < n) {
        int r = orig_row(i, sigma, perm, perm_bytes);
        long long prev = left_offset(i, sigma, resolve_k_left(k_left_user, kl));
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p) {
            long long d = (long long)col[p] - prev;
            while (d >= 128) {
                const long long q = d < 32767 ? d : 32767;
                dst[j * C] = (uint16_t)(q << 1);
                ++j;
                d -= q;
            }
            dst[j * C] = (uint16_t)((code[p] << 8) | ((uint32_t)d << 1) | 1u);
            ++j;
            prev = col[p];
        }
    }
    for (; j < w; ++j) dst[j * C] = 0;
}

template <typename TO, typename TI>
__global__ void k_scatter_sell(int n, int64_t rows_total, int C, int sigma,
                               const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                               const TI *__restrict__ val_in, const void *perm, int perm_bytes,
                               const int64_t *__restrict__ offset, TO *__restrict__ val,
                               int32_t *__restrict__ colo) {
    int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ii >= rows_total) return;
    int i = (int)ii;
    int64_t k = ii / C;
    int l = (int)(ii - k * C);
    int64_t s = offset[k];
    int64_t w = (offset[k + 1] - s) / C;
    int64_t j = 0;
    int last = 0;
    if (i < n) {
        int r = orig_row(i, sigma, perm, perm_bytes);
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p, ++j) {
            val[s + j * C + l] = (TO)val_in[p];
            last = col[p];
            colo[s + j * C + l] = last;
        }
    }
    for (; j < w; ++j) {  // padding: zero value at a valid column
        val[s + j * C + l] = (TO)0;
        colo[s + j * C + l] = last;
    }
}

// FP16 SELL (§3 layout, binary16 values): the value of each stored nonzero is
// the upper half of its FP16 field; padding slots hold column -1.
__global__ void k_scatter_sell16(int n, int64_t rows_total, int C, int sigma,
                                 const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                 const uint32_t *__restrict__ field, const void *perm, int perm_bytes,
                                 const int64_t *__restrict__ offset, uint16_t *__restrict__ val,
                                 int32_t *__restrict__ colo) {
    int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ii >= rows_total) return;
    int i = (int)ii;
    int64_t k = ii / C;
    int l = (int)(ii - k * C);
    int64_t s = offset[k];
    int64_t w = (offset[k + 1] - s) / C;
    int64_t j = 0;
    if (i < n) {
        int r = orig_row(i, sigma, perm, perm_bytes);
        for (int64_t p = rowptr[r]; p < rowptr[r + 1]; ++p, ++j) {
            val[s + j * C + l] = (uint16_t)(field[p] >> 16);
            colo[s + j * C + l] = col[p];
        }
    }
    for (; j < w; ++j) {
        val[s + j * C + l] = 0;
        colo[s + j * C + l] = -1;
    }
}

// The fixed-point exponent: the smallest s with (2^(V-1) - 1) * 2^s >= M
// (0 for M = 0), V = 31 - D.
int fixed_exponent(double M, int D) {
    const int V = 31 - D;
    if (!(M > 0.0)) return 0;
    const double top = ldexp(1.0, V - 1) - 1.0;
    int sx = ilogb(M) - (V - 1);
    while (ldexp(top, sx) < M) ++sx;
    while (ldexp(top, sx - 1) >= M) --sx;
    return sx;
}

const char *status_text(int code) {
    switch (code) {
        case PACKSELL_ERR_INVALID_ARG: return "invalid row pointer or k_left below the bandwidth";
        case PACKSELL_ERR_UNSORTED: return "columns not strictly increasing";
        case PACKSELL_ERR_NONFINITE: return "non-finite value";
        case PACKSELL_ERR_RANGE: return "column out of range or value overflows the format";
        default: return "error";
    }
}

struct Temps {
    cudaStream_t s;
    void *ptrs[16] = {};
    int n = 0;
    explicit Temps(cudaStream_t st) : s(st) {}
    template <typename T>
    cudaError_t get(T **p, size_t bytes) {
        cudaError_t e = cudaMallocAsync((void **)p, std::max<size_t>(bytes, 16), s);
        if (e == cudaSuccess) ptrs[n++] = *p;
        return e;
    }
    ~Temps() {
        for (int i = 0; i < n; ++i) cudaFreeAsync(ptrs[i], s);
    }
};

void free_matrix_arrays(Matrix *A) {
    cudaFree(A->pack);
    cudaFree(A->pack16);
    cudaFree(A->pack64);
    cudaFree(A->val);
    cudaFree(A->col);
    cudaFree(A->offset);
    cudaFree(A->perm);
    cudaFree(A->rowptr);
    cudaFree(A->status);
    for (int v = 0; v < Matrix::kBulkVariants; ++v) cudaFree(A->part[v]);
    stage_free(*A);
    csr_plan_free(*A);
    split_plan_free(*A);
    multi_plan_free(*A);
}

}  // namespace

packsell_status encode_impl(const packsell_params &p, int64_t n, int64_t m, int64_t nnz,
                            const int64_t *rowptr, const int32_t *col, const void *val,
                            int val_is_f64, cudaStream_t s, Matrix **out) {
    const int fmt = p.format;
    if (!out) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: out is NULL");
    *out = nullptr;
    if (!is_packed(fmt) && !is_sell(fmt) && !is_w16(fmt) && !is_sell16(fmt) && !is_fixed(fmt) &&
        !is_w64(fmt))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: unknown format");
    if (p.C < 1 || p.C > 1024) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: C must be in [1, 1024]");
    if (p.sigma < 1 || p.sigma > 65536)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: sigma must be in [1, 65536]");
    if (fmt == PACKSELL_FMT_FP16 && p.D != 15)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: FP16 needs D = 15");
    if (fmt == PACKSELL_FMT_E8MY && (p.D < 1 || p.D > 22))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: E8MY needs D in [1, 22]");
    // fixed point: V = 31 - D <= 25 bits, so every q converts to FP32 exactly
    if (is_fixed(fmt) && (p.D < 6 || p.D > 22))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: FIXED needs D in [6, 22]");
    if (is_w16(fmt) && p.D != 7)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: W16_E4M3 needs D = 7");
    // 64-bit words: columns stay below 2^31, so more delta bits buy nothing
    if (is_w64(fmt) && (p.D < 1 || p.D > 31))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: W64_E11MY needs D in [1, 31]");
    if (n < 0 || m < 0 || nnz < 0 || n >= (1ll << 31) || m >= (1ll << 31))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: n and m must be in [0, 2^31)");
    if (!rowptr || (nnz > 0 && (!col || !val)))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: NULL array");
    if (p.k_left < -1) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: k_left < -1");

    // delta-value words
    const bool packed = is_packed(fmt) || is_w16(fmt) || is_fixed(fmt) || is_w64(fmt);
    const int D = packed ? p.D : 31;
    const int W = is_w16(fmt) ? 16 : is_w64(fmt) ? 64 : 32;
    const int64_t S = (n + p.C - 1) / p.C;
    const int perm_bytes = (p.sigma == 1) ? 0 : (p.sigma <= 256 ? 1 : 2);

    Matrix *A = new Matrix();
    A->n = n;
    A->m = m;
    A->nnz = nnz;
    A->p = p;
    A->n_slices = S;
    A->perm_bytes = perm_bytes;
    cudaGetDevice(&A->device);
    auto bail = [&](packsell_status st) {
        free_matrix_arrays(A);
        delete A;
        return st;
    };

    {
        Temps T(s);
        DevStatus *st = nullptr;
        unsigned long long *kl = nullptr, *total = nullptr;
        int *maxw = nullptr;
        uint32_t *field = nullptr;
        unsigned long long *field64 = nullptr;  // E11MY fields of 64-bit words
        int32_t *words = nullptr, *words_st = nullptr;
        int64_t *slice_words = nullptr;
        cudaError_t e = cudaSuccess;
        if ((e = T.get(&st, sizeof(DevStatus))) || (e = T.get(&kl, 8)) || (e = T.get(&total, 8)) ||
            (e = T.get(&maxw, 4)) || (e = T.get(&words, 4 * (size_t)n)) ||
            (e = T.get(&words_st, 4 * (size_t)n)) || (e = T.get(&slice_words, 8 * (size_t)S)) ||
            (((packed && !is_w64(fmt)) || is_sell16(fmt)) && (e = T.get(&field, 4 * (size_t)nnz))) ||
            (is_w64(fmt) && (e = T.get(&field64, 8 * (size_t)nnz))))
            return bail(e == cudaErrorMemoryAllocation
                            ? fail(PACKSELL_ERR_NO_MEMORY, "packsell_encode: temporaries")
                            : cuda_fail(e, "cudaMallocAsync"));
        if ((e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s)) || (e = cudaMemsetAsync(kl, 0, 8, s)) ||
            (e = cudaMemsetAsync(total, 0, 8, s)) || (e = cudaMemsetAsync(maxw, 0, 4, s)))
            return bail(cuda_fail(e, "packsell_encode: cudaMemsetAsync"));
        if (cudaMalloc(&A->offset, sizeof(int64_t) * (S + 1)) != cudaSuccess ||
            (perm_bytes && cudaMalloc(&A->perm, (size_t)perm_bytes * n) != cudaSuccess) ||
            (p.keep_rowptr && cudaMalloc(&A->rowptr, sizeof(int64_t) * (n + 1)) != cudaSuccess))
            return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_encode: matrix arrays"));

        k_check_rows<<<blocks_for(n), TPB, 0, s>>>((int)n, m, nnz, rowptr, col, kl, st);
        if (is_fixed(fmt) && nnz > 0) {
            // fixed point: the exponent from the largest magnitude first
            unsigned long long *amax = nullptr, hmax = 0;
            if ((e = T.get(&amax, 8)) || (e = cudaMemsetAsync(amax, 0, 8, s)))
                return bail(cuda_fail(e, "packsell_encode: fixed-point scale"));
            const int qb0 = std::min(blocks_for(nnz), 152 * 64);
            if (val_is_f64) k_absmax<double><<<qb0, TPB, 0, s>>>(nnz, (const double *)val, amax);
            else k_absmax<float><<<qb0, TPB, 0, s>>>(nnz, (const float *)val, amax);
            if ((e = cudaMemcpyAsync(&hmax, amax, 8, cudaMemcpyDeviceToHost, s)) ||
                (e = cudaStreamSynchronize(s)))
                return bail(cuda_fail(e, "packsell_encode: fixed-point scale"));
            double M;
            memcpy(&M, &hmax, sizeof M);
            A->value_exp = fixed_exponent(M, p.D);
        }
        if (is_w64(fmt) && nnz > 0) {
            const int qb = std::min(blocks_for(nnz), 152 * 64);
            if (val_is_f64)
                k_quantize64<double><<<qb, TPB, 0, s>>>(nnz, (const double *)val, D, field64, st);
            else
                k_quantize64<float><<<qb, TPB, 0, s>>>(nnz, (const float *)val, D, field64, st);
        } else if ((packed || is_sell16(fmt)) && nnz > 0) {
            int qb = blocks_for(nnz);
            qb = std::min(qb, 152 * 64);
            // FP16 SELL takes the FP16 quantiser of the packed format
            const int qf = is_sell16(fmt) ? PACKSELL_FMT_FP16 : fmt, qd = is_sell16(fmt) ? 15 : D;
            if (val_is_f64)
                k_quantize<double><<<qb, TPB, 0, s>>>(nnz, (const double *)val, qf, qd, field, st,
                                                      A->value_exp);
            else
                k_quantize<float><<<qb, TPB, 0, s>>>(nnz, (const float *)val, qf, qd, field, st,
                                                     A->value_exp);
        }
        if (n > 0) {
            k_count_words<<<blocks_for(n), TPB, 0, s>>>((int)n, rowptr, col, p.sigma, p.k_left, kl,
                                                       D, packed ? 1 : 0, W, words, total, st);
            if (p.sigma > 1) {
                int64_t nb = (n + p.sigma - 1) / p.sigma;
                int tpb = std::min(1024, ((std::min(p.sigma, 1024) + 31) / 32) * 32);
                k_sigma_sort<<<(unsigned)nb, tpb, 0, s>>>((int)n, p.sigma, words, A->perm,
                                                          perm_bytes, words_st);
            } else {
                k_copy_words<<<blocks_for(n), TPB, 0, s>>>((int)n, words, words_st);
            }
            k_slice_widths<<<blocks_for(S), TPB, 0, s>>>(S, (int)n, p.C, words_st, slice_words,
                                                        maxw);
        }
        PS_LAUNCH_CHECK("packsell_encode: kernels");
        packsell_status sst = scan_exclusive(slice_words, A->offset, S, s);
        if (sst != PACKSELL_OK) return bail(sst);
        if (p.keep_rowptr && (e = cudaMemcpyAsync(A->rowptr, rowptr, sizeof(int64_t) * (n + 1),
                                                  cudaMemcpyDeviceToDevice, s)))
            return bail(cuda_fail(e, "packsell_encode: row pointer copy"));

        DevStatus hst{};
        unsigned long long hkl = 0, htotal = 0;
        int hmaxw = 0;
        int64_t nw = 0;
        if ((e = cudaMemcpyAsync(&hst, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(&hkl, kl, 8, cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(&htotal, total, 8, cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(&hmaxw, maxw, 4, cudaMemcpyDeviceToHost, s)) ||
            (e = cudaMemcpyAsync(&nw, A->offset + S, 8, cudaMemcpyDeviceToHost, s)))
            return bail(cuda_fail(e, "packsell_encode: read-back"));
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "packsell_encode: synchronize"));
        if (hst.code != 0)
            return bail(fail((packsell_status)hst.code,
                             std::string("packsell_encode: ") + status_text(hst.code) +
                                 " (index " + std::to_string(hst.index) + ")"));
        A->p.k_left = p.k_left >= 0 ? p.k_left : (int64_t)hkl;
        A->n_words = nw;
        A->n_dummies = packed ? (int64_t)htotal - nnz : 0;
        A->n_pad = nw - (int64_t)htotal;
        A->max_width = hmaxw;

        if (is_w64(fmt)) {
            if (cudaMalloc(&A->pack64, sizeof(uint64_t) * std::max<int64_t>(nw, 1)) != cudaSuccess)
                return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_encode: word array"));
            int64_t rows_total = S * p.C;
            if (rows_total > 0)
                k_scatter_w64<<<blocks_for(rows_total), TPB, 0, s>>>(
                    (int)n, rows_total, p.C, p.sigma, A->p.k_left, kl, D, rowptr, col, field64,
                    A->perm, perm_bytes, A->offset, (unsigned long long *)A->pack64);
        } else if (is_w16(fmt)) {
            if (cudaMalloc(&A->pack16, sizeof(uint16_t) * std::max<int64_t>(nw, 1)) != cudaSuccess)
                return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_encode: word array"));
            int64_t rows_total = S * p.C;
            if (rows_total > 0)
                k_scatter_w16<<<blocks_for(rows_total), TPB, 0, s>>>(
                    (int)n, rows_total, p.C, p.sigma, A->p.k_left, kl, rowptr, col, field,
                    A->perm, perm_bytes, A->offset, A->pack16);
        } else if (packed) {
            // kWordTail spare words: a 16-byte vector load that starts at the
            // last words of the array stays inside the allocation
            if (cudaMalloc(&A->pack, sizeof(uint32_t) * (nw + kWordTail)) != cudaSuccess)
                return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_encode: word array"));
            int64_t rows_total = S * p.C;
            if (rows_total > 0)
                k_scatter_packed<<<blocks_for(rows_total), TPB, 0, s>>>(
                    (int)n, rows_total, p.C, p.sigma, A->p.k_left, kl, D, rowptr, col, field,
                    A->perm, perm_bytes, A->offset, A->pack);
        } else if (is_sell16(fmt)) {
            if (cudaMalloc(&A->val, 2 * std::max<int64_t>(nw, 1)) != cudaSuccess ||
                cudaMalloc(&A->col, 4 * std::max<int64_t>(nw, 1)) != cudaSuccess)
                return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_encode: value arrays"));
            int64_t rows_total = S * p.C;
            if (rows_total > 0)
                k_scatter_sell16<<<blocks_for(rows_total), TPB, 0, s>>>(
                    (int)n, rows_total, p.C, p.sigma, rowptr, col, field, A->perm, perm_bytes,
                    A->offset, (uint16_t *)A->val, A->col);
        } else {
            size_t vb = fmt == PACKSELL_FMT_SELL_F64 ? 8 : 4;
            if (cudaMalloc(&A->val, vb * std::max<int64_t>(nw, 1)) != cudaSuccess ||
                cudaMalloc(&A->col, 4 * std::max<int64_t>(nw, 1)) != cudaSuccess)
                return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_encode: value arrays"));
            int64_t rows_total = S * p.C;
            if (rows_total > 0) {
                int g = blocks_for(rows_total);
                if (fmt == PACKSELL_FMT_SELL_F64) {
                    if (val_is_f64)
                        k_scatter_sell<double, double><<<g, TPB, 0, s>>>(
                            (int)n, rows_total, p.C, p.sigma, rowptr, col, (const double *)val,
                            A->perm, perm_bytes, A->offset, (double *)A->val, A->col);
                    else
                        k_scatter_sell<double, float><<<g, TPB, 0, s>>>(
                            (int)n, rows_total, p.C, p.sigma, rowptr, col, (const float *)val,
                            A->perm, perm_bytes, A->offset, (double *)A->val, A->col);
                } else {
                    if (val_is_f64)
                        k_scatter_sell<float, double><<<g, TPB, 0, s>>>(
                            (int)n, rows_total, p.C, p.sigma, rowptr, col, (const double *)val,
                            A->perm, perm_bytes, A->offset, (float *)A->val, A->col);
                    else
                        k_scatter_sell<float, float><<<g, TPB, 0, s>>>(
                            (int)n, rows_total, p.C, p.sigma, rowptr, col, (const float *)val,
                            A->perm, perm_bytes, A->offset, (float *)A->val, A->col);
                }
            }
        }
        PS_LAUNCH_CHECK("packsell_encode: scatter");
        packsell_status pst = plan_spmv(*A, s);
        if (pst != PACKSELL_OK) return bail(pst);
        // the matrix is complete on return: products may read its words
        // before they wait on the previous kernel of their stream
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return bail(cuda_fail(e, "packsell_encode: synchronize"));
        // Temps are released (stream-ordered) here; they outlive the scatter.
    }
    *out = A;
    return PACKSELL_OK;
}

packsell_status scan_i64(const int64_t *in, int64_t *out, int64_t S, cudaStream_t s) {
    return scan_exclusive(in, out, S, s);
}

void destroy_matrix(Matrix *A) {
    if (!A) return;
    free_matrix_arrays(A);
    delete A;
}

// ---- validation of imported matrices ----
namespace {
// What k_validate decodes: 32-bit words (FP16, E8MY, fixed point), 16- or
// 64-bit words, or the column array of plain SELL (FP16 SELL pads with
// column -1).
enum ValidateKind { kValWords32 = 0, kValWords16 = 1, kValCols = 2, kValCols16 = 3, kValWords64 = 4 };

template <int KIND>
__global__ void k_validate(int n, int64_t m, int C, int sigma, long long k_left, int D,
                           const int64_t *__restrict__ offset, const void *__restrict__ words,
                           const int32_t *__restrict__ colv, const void *perm, int perm_bytes,
                           unsigned long long *count, DevStatus *st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (perm_bytes) {
        int q = perm_bytes == 1 ? ((const uint8_t *)perm)[i] : ((const uint16_t *)perm)[i];
        int b = (i / sigma) * sigma;
        if (q >= sigma || b + q >= n) {
            dev_fail(st, PACKSELL_ERR_CORRUPT, i);
            return;
        }
    }
    int64_t k = i / C;
    int l = i - (int)(k * C);
    int64_t s = offset[k], e = offset[k + 1];
    if (s < 0 || e < s || (e - s) % C) {
        dev_fail(st, PACKSELL_ERR_CORRUPT, i);
        return;
    }
    int64_t w = (e - s) / C;
    unsigned long long cnt = 0;
    if (KIND == kValWords32 || KIND == kValWords16 || KIND == kValWords64) {
        // flag 1: D delta bits; flag 0 (dummy, padding): the rest of the word
        const unsigned long long dmask = (1ull << D) - 1ull;
        const unsigned long long wide = KIND == kValWords64   ? 0x7fffffffffffffffull
                                        : KIND == kValWords32 ? 0x7fffffffull
                                                              : 0x7fffull;
        long long c = left_offset(i, sigma, k_left);
        for (int64_t j = 0; j < w; ++j) {
            const int64_t at = s + j * C + l;
            const unsigned long long wd =
                KIND == kValWords64   ? ((const unsigned long long *)words)[at]
                : KIND == kValWords32 ? (unsigned long long)((const uint32_t *)words)[at]
                                      : (unsigned long long)((const uint16_t *)words)[at];
            const unsigned long long flag = wd & 1ull;
            const unsigned long long delta = (wd >> 1) & (flag ? dmask : wide);
            // a column past m (or a delta that would overflow the sum) is corrupt
            if (wd != 0ull && (delta >= (unsigned long long)m || (c += (long long)delta) >= m)) {
                dev_fail(st, PACKSELL_ERR_CORRUPT, at);
                return;
            }
            cnt += flag;
        }
    } else {
        bool pad = false;
        for (int64_t j = 0; j < w; ++j) {
            const int c = colv[s + j * C + l];
            // FP16 SELL: a row's slots after its first -1 are all -1 (the
            // product stops at the first); nonpadding slots are counted
            const bool bad = KIND == kValCols16 ? (c >= m || c < -1 || (pad && c != -1))
                                                : (c < 0 || c >= m);
            if (bad) {
                dev_fail(st, PACKSELL_ERR_CORRUPT, s + j * C + l);
                return;
            }
            if (KIND == kValCols16) {
                pad = c < 0;
                cnt += !pad;
            }
        }
    }
    if (cnt) atomicAdd(count, cnt);
}
}  // namespace

packsell_status validate_impl(const Matrix &A, cudaStream_t s, const char *what) {
    Temps T(s);
    DevStatus *st = nullptr;
    unsigned long long *cnt = nullptr;
    PS_CUDA(T.get(&st, sizeof(DevStatus)));
    PS_CUDA(T.get(&cnt, 8));
    PS_CUDA(cudaMemsetAsync(st, 0, sizeof(DevStatus), s));
    PS_CUDA(cudaMemsetAsync(cnt, 0, 8, s));
    const int fmt = A.p.format;
    const bool counted = !is_sell(fmt);  // every format but plain SELL counts its values
    if (A.n > 0) {
        int g = blocks_for(A.n);
        if (is_packed(fmt) || is_fixed(fmt))
            k_validate<kValWords32><<<g, TPB, 0, s>>>((int)A.n, A.m, A.p.C, A.p.sigma, A.p.k_left,
                                                      A.p.D, A.offset, A.pack, nullptr, A.perm,
                                                      A.perm_bytes, cnt, st);
        else if (is_w64(fmt))
            k_validate<kValWords64><<<g, TPB, 0, s>>>((int)A.n, A.m, A.p.C, A.p.sigma, A.p.k_left,
                                                      A.p.D, A.offset, A.pack64, nullptr, A.perm,
                                                      A.perm_bytes, cnt, st);
        else if (is_w16(fmt))
            k_validate<kValWords16><<<g, TPB, 0, s>>>((int)A.n, A.m, A.p.C, A.p.sigma, A.p.k_left,
                                                      A.p.D, A.offset, A.pack16, nullptr, A.perm,
                                                      A.perm_bytes, cnt, st);
        else if (is_sell16(fmt))
            k_validate<kValCols16><<<g, TPB, 0, s>>>((int)A.n, A.m, A.p.C, A.p.sigma, A.p.k_left,
                                                     31, A.offset, nullptr, A.col, A.perm,
                                                     A.perm_bytes, cnt, st);
        else
            k_validate<kValCols><<<g, TPB, 0, s>>>((int)A.n, A.m, A.p.C, A.p.sigma, A.p.k_left, 31,
                                                   A.offset, nullptr, A.col, A.perm, A.perm_bytes,
                                                   cnt, st);
        PS_LAUNCH_CHECK("k_validate");
    }
    DevStatus hst{};
    unsigned long long hc = 0;
    PS_CUDA(cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaMemcpyAsync(&hc, cnt, 8, cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaStreamSynchronize(s));
    if (hst.code)
        return fail(PACKSELL_ERR_CORRUPT, std::string(what) +
                                              ": bad word, column or perm at index " +
                                              std::to_string(hst.index));
    if (counted && (int64_t)hc != A.nnz)
        return fail(PACKSELL_ERR_CORRUPT, std::string(what) + ": value words do not match nnz");
    return PACKSELL_OK;
}

// Storage position -> original row (§3): the inverse of the sigma-block sort.
__global__ void k_storage_rows(int n, int sigma, const void *perm, int perm_bytes,
                               int32_t *__restrict__ rows) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        rows[i] = orig_row(i, sigma, perm, perm_bytes);
}

// ---- quantisation on its own, and the quantisation error of a format ----
namespace {

// Per row: s_err = sum |a_ij - q(a_ij)|, s_q = sum |q(a_ij)|, s_a = sum |a_ij|
// in double, then the maxima over the rows (non-negative doubles order as
// their bit patterns, so the maxima are atomicMax on the patterns). A value
// the format cannot hold sets `bad`.
template <typename T>
__global__ void k_format_error(int n, const int64_t *__restrict__ rowptr, const T *__restrict__ val,
                               int fmt, int D, unsigned long long *out, int *bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double se = 0.0, sq = 0.0, sa = 0.0;
    unsigned long long len = 0;
    if (i < n) {
        const int64_t a = rowptr[i], b = rowptr[i + 1];
        len = (unsigned long long)(b - a);
        for (int64_t p = a; p < b; ++p) {
            const T v = val[p];
            uint32_t f = 0;
            const int err = fmt == PACKSELL_FMT_FP16 ? field_fp16(v, f) : field_e8my(v, D, f);
            if (err) {
                atomicExch(bad, err);
                continue;
            }
            const double q = fmt == PACKSELL_FMT_FP16
                                 ? (double)__half2float(__ushort_as_half((unsigned short)(f >> 16)))
                                 : (double)__uint_as_float(f);
            se += fabs((double)v - q);
            sq += fabs(q);
            sa += fabs((double)v);
        }
    }
    unsigned long long e = __double_as_longlong(se), q = __double_as_longlong(sq),
                       aa = __double_as_longlong(sa);
    // a warp's maxima in full 64-bit precision: a shuffle reduction
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
        q = max(q, __shfl_xor_sync(0xffffffffu, q, o));
        aa = max(aa, __shfl_xor_sync(0xffffffffu, aa, o));
        len = max(len, __shfl_xor_sync(0xffffffffu, len, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, e);
        atomicMax(out + 1, q);
        atomicMax(out + 2, aa);
        atomicMax(out + 3, len);
    }
}

}  // namespace

packsell_status quantize_impl(int fmt, int D, int64_t n, const void *val, int is64, uint32_t *field,
                              int64_t *bad_index, cudaStream_t s) {
    if (bad_index) *bad_index = -1;
    if (!(fmt == PACKSELL_FMT_FP16 && D == 15) && !(fmt == PACKSELL_FMT_E8MY && D >= 1 && D <= 22) &&
        !(fmt == PACKSELL_FMT_W16_E4M3 && D == 7))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_quantize: bad format or D");
    if (n == 0) return PACKSELL_OK;
    DevStatus *st = nullptr;
    PS_CUDA(cudaMallocAsync(&st, sizeof(DevStatus), s));
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    const int qb = (int)std::min<int64_t>((n + TPB - 1) / TPB, 152 * 32);
    if (e == cudaSuccess) {
        if (is64) k_quantize<double><<<qb, TPB, 0, s>>>(n, (const double *)val, fmt, D, field, st);
        else k_quantize<float><<<qb, TPB, 0, s>>>(n, (const float *)val, fmt, D, field, st);
        e = cudaGetLastError();
    }
    DevStatus h{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(st, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "packsell_quantize");
    if (h.code) {
        if (bad_index) *bad_index = h.index;
        return fail((packsell_status)h.code, "packsell_quantize: value " + std::to_string(h.index) +
                                                 (h.code == PACKSELL_ERR_RANGE ? " overflows the format"
                                                                               : " is not finite"));
    }
    return PACKSELL_OK;
}

packsell_status format_error_impl(int64_t n, const int64_t *rowptr, const void *val, int is64,
                                  int fmt, int D, cudaStream_t s, double out[3], int64_t *max_len,
                                  int *bad) {
    out[0] = out[1] = out[2] = 0.0;
    *max_len = 0;
    *bad = 0;
    if (n == 0) return PACKSELL_OK;
    unsigned long long *d = nullptr;
    PS_CUDA(cudaMallocAsync(&d, 4 * sizeof(unsigned long long) + sizeof(int), s));
    int *dbad = reinterpret_cast<int *>(d + 4);
    cudaError_t e = cudaMemsetAsync(d, 0, 4 * sizeof(unsigned long long) + sizeof(int), s);
    if (e == cudaSuccess) {
        if (is64)
            k_format_error<double><<<blocks_for(n), TPB, 0, s>>>((int)n, rowptr, (const double *)val,
                                                                  fmt, D, d, dbad);
        else
            k_format_error<float><<<blocks_for(n), TPB, 0, s>>>((int)n, rowptr, (const float *)val,
                                                                 fmt, D, d, dbad);
        e = cudaGetLastError();
    }
    unsigned long long h[4] = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "packsell_tune_format: quantisation error");
    for (int k = 0; k < 3; ++k) {
        double v;
        memcpy(&v, &h[k], sizeof v);
        out[k] = v;
    }
    *max_len = (int64_t)h[3];
    return PACKSELL_OK;
}

packsell_status storage_rows_impl(const Matrix &A, int32_t *rows, cudaStream_t s) {
    if (A.n == 0) return PACKSELL_OK;
    const int blocks = (int)std::min<int64_t>((A.n + 255) / 256, 4096);
    k_storage_rows<<<blocks, 256, 0, s>>>((int)A.n, A.p.sigma, A.perm, A.perm_bytes, rows);
    PS_LAUNCH_CHECK("packsell_storage_rows");
    return PACKSELL_OK;
}

}  // namespace packsell
