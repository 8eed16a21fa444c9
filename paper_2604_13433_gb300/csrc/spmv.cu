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
#include <atomic>

#include "device.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace packsell {
namespace {

constexpr int TPB = 256;
constexpr int UNROLL = 8;

inline int grid_for(int64_t n) { return (int)std::max<int64_t>(1, (n + TPB - 1) / TPB); }

// Words per prefetch round for a matrix whose widest slice has w words: the
// smallest of 8, 10, 12, 16 that holds w (16 for wider slices).
inline int round_words(int w) { return w <= 8 ? 8 : w <= 10 ? 10 : w <= 12 ? 12 : 16; }

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
    bool live = true;  // false once a zero (padding) word ends the row
    for (; live && j + UNROLL <= w; j += UNROLL) {
        uint32_t wd[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) wd[u] = ldg_stream(pp + (int64_t)(j + u) * C);
        float xv[UNROLL], vv[UNROLL];
        uint32_t fl[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            uint32_t d;
            Word<FMT>::decode(wd[u], dc.dmask, dc.vmask, fl[u], d, vv[u], dc.vshift, dc.vscale);
            c += (int)d;
            xv[u] = (fl[u] && PS_IN_RANGE(c, dc.xlen)) ? __ldg(x + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            if (fl[u]) t = fmaf(vv[u], xv[u], t);
        live = wd[UNROLL - 1] != 0u;
    }
    for (; live && j < w; ++j) {
        uint32_t f, d;
        float v;
        const uint32_t wj = ldg_stream(pp + (int64_t)j * C);
        if (wj == 0u) break;
        Word<FMT>::decode(wj, dc.dmask, dc.vmask, f, d, v, dc.vshift, dc.vscale);
        c += (int)d;
        if (f && PS_IN_RANGE(c, dc.xlen)) t = fmaf(v, __ldg(x + c), t);
    }
    y[orig_row(i, sigma, perm, perm_bytes)] = t;
}

// Thread-per-row SpMV with row register prefetch: each thread first issues
// the loads of up to PF words of its row at once (L1-bypassing loads
// predicated on j < w), then decodes them, issues their x
// gathers, and finally runs the fused multiply-adds in stored order. A row of
// up to PF words costs one memory round trip for its words and one for its
// gathers. Words past the row's slice width are taken as 0 (padding).
// One row of the prefetch kernels: returns the sum, sets the output index
// (PERM: rows are written through the sigma permutation).
template <int FMT, int PF, int C, bool PERM = true, bool EXIT = false, bool PDL = false>
__device__ __forceinline__ float prefetch_row(int i, int sigma, int sig_shift, long long k_left,
                                              const int64_t *__restrict__ offset,
                                              const uint32_t *__restrict__ pack,
                                              const void *__restrict__ perm, int perm_bytes,
                                              Decode dc, const float *__restrict__ x, int &io) {
    const int k = i / C, l = i - k * C;
    const int64_t s = offset[k];
    const int w = (int)((offset[k + 1] - s) / C);
    const uint32_t *__restrict__ pp = pack + s + l;
    const int blk = sig_shift >= 0 ? (i >> sig_shift) << sig_shift : (i / sigma) * sigma;
    int c = (k_left < blk) ? (int)(blk - k_left) : 0;
    float t = 0.f;
    if (PDL && w <= 0) grid_dep_wait();
    for (int j0 = 0; j0 < w; j0 += PF) {
        const int wr = w - j0;
        // loads predicated on the width; a word past it acts as padding
        uint32_t wd[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) wd[u] = (u < wr) ? ldg_stream(pp + (j0 + u) * C) : 0u;
        // PDL: the matrix is complete before any product runs, so the first
        // round's words (and the offsets) load while the previous kernel of
        // the stream finishes; x and y are touched only after the wait
        if (PDL && j0 == 0) grid_dep_wait();
        bool f[PF];
        float xv[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) word_gather<FMT>(wd[u], dc, x, c, f[u], xv[u]);
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (f[u]) t = fmaf(word_value<FMT>(wd[u], dc), xv[u], t);
        // EXIT: a zero word is padding (real words have flag 1, dummies a
        // nonzero delta), and padding runs to the slice's end: the row is
        // done, and the lane stops loading, so on slices of uneven rows the
        // warp's later loads fetch only the sectors of rows still running
        if (EXIT && wd[PF - 1] == 0u) break;
    }
    io = i;
    if (PERM) {
        if (perm_bytes == 1) io = blk + (int)((const uint8_t *)perm)[i];
        else if (perm_bytes == 2) io = blk + (int)((const uint16_t *)perm)[i];
    }
    return t;
}

// One row per thread; the reducing form (DOT) runs on the fixed solver grid
// and strides over rows (warps stay on whole slices) so that its reduction
// is deterministic.
template <int FMT, int PF, int C, int MINB, bool DOT = false, bool PERM = true,
          bool EXIT = false, bool PDL = false>
__global__ void __launch_bounds__(TPB, MINB)
    k_spmv_prefetch(int n, int sigma, int sig_shift, long long k_left,
                    const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
                    const void *__restrict__ perm, int perm_bytes, Decode dc,
                    const float *__restrict__ x, float *__restrict__ y, Red red = Red{}) {
    if (!DOT) {
        if (PDL) grid_dep_launch();  // one pass over the rows: signal at block start
        const int i = blockIdx.x * blockDim.x + threadIdx.x;
        if (i >= n) return;
        int io;
        const float t = prefetch_row<FMT, PF, C, PERM, EXIT, PDL>(
            i, sigma, sig_shift, k_left, offset, pack, perm, perm_bytes, dc, x, io);
        y[io] = t;
        return;
    }
    if (red.sc->done) return;  // solver converged: idle (grid-uniform)
    float d1 = 0.f;  // per-thread sum in FP32; block and grid sums in FP64
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int io;
        const float t = prefetch_row<FMT, PF, C, PERM>(i, sigma, sig_shift, k_left, offset, pack,
                                                       perm, perm_bytes, dc, x, io);
        y[io] = t;
        d1 = fmaf(x[io], t, d1);
    }
    reduce_publish(red, (double)d1, 0.0);
}

// Pipelined persistent SpMV for short rows (variant 12, and the solver's
// fused SpMV + dot when every row fits one round): each thread walks rows
// i, i + stride, ... (stride a multiple of 32, so a warp stays on whole
// slices) and loads the next row's words, and the slice offsets of the row
// after it, before it decodes and gathers the current row: the word loads
// of one row overlap the gathers of the previous one. Every slice must fit
// one round (width <= PF <= 16). Same bits as the thread-per-row kernels.
template <int FMT, int PF>
__device__ __forceinline__ void pipe_round(const uint32_t (&wd)[PF], Decode dc,
                                           const float *__restrict__ x, int &c, float &t) {
    bool f[PF];
    float xv[PF];
#pragma unroll
    for (int u = 0; u < PF; ++u) word_gather<FMT>(wd[u], dc, x, c, f[u], xv[u]);
#pragma unroll
    for (int u = 0; u < PF; ++u)
        if (f[u]) t = fmaf(word_value<FMT>(wd[u], dc), xv[u], t);
}

// PDL (launched by launch_pdl): the first row's words and the next row's
// offsets load before the wait; the solver state, x and y after it.
template <int FMT, int PF, int MINB, bool DOT, bool PERM, bool PDL = false>
__global__ void __launch_bounds__(TPB, MINB)
    k_spmv_pipe(int n, int sigma, int sig_shift, long long k_left,
                const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
                const void *__restrict__ perm, int perm_bytes, Decode dc,
                const float *__restrict__ x, float *__restrict__ y, Red red = Red{}) {
    if (!PDL && DOT && red.sc->done) return;  // solver converged: idle (grid-uniform)
    float d1 = 0.f;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cur[PF];
    int in = i + stride;
    int64_t sn = 0, en = 0;
    if (i < n) {
        const int64_t s = offset[i >> 5];
        const int w = (int)((offset[(i >> 5) + 1] - s) >> 5);
#pragma unroll
        for (int u = 0; u < PF; ++u) cur[u] = (u < w) ? ldg_stream(pack + s + (i & 31) + u * 32) : 0u;
        if (in < n) {
            sn = offset[in >> 5];
            en = offset[(in >> 5) + 1];
        }
    }
    if (PDL) {
        grid_dep_sync();
        if (DOT && red.sc->done) return;  // every thread, as above
    }
    if (i < n) {
        while (true) {
            const int wn = (int)((en - sn) >> 5);
            uint32_t nxt[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u)
                nxt[u] = (in < n && u < wn) ? ldg_stream(pack + sn + (in & 31) + u * 32) : 0u;
            const int in2 = in + stride;
            int64_t sn2 = 0, en2 = 0;
            if (in2 < n) {
                sn2 = offset[in2 >> 5];
                en2 = offset[(in2 >> 5) + 1];
            }
            const int blk = sig_shift >= 0 ? (i >> sig_shift) << sig_shift : (i / sigma) * sigma;
            int c = (k_left < blk) ? (int)(blk - k_left) : 0;
            float t = 0.f;
            pipe_round<FMT, PF>(cur, dc, x, c, t);
            int io = i;
            if (PERM) io = blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[i]
                                                  : (int)((const uint16_t *)perm)[i]);
            y[io] = t;
            if (DOT) d1 = fmaf(x[io], t, d1);
            if (in >= n) break;
            i = in;
#pragma unroll
            for (int u = 0; u < PF; ++u) cur[u] = nxt[u];
            in = in2;
            sn = sn2;
            en = en2;
        }
    }
    if (DOT) reduce_publish(red, (double)d1, 0.0);
}

// The same pipelined structure over FP32 SELL (C = 32, every slice within PF
// slots) fused with sum_i x_i y_i: the solver's inner product with an FP32
// SELL matrix, so that the FP32-SELL inner solve is compared with the
// PackSELL one on kernels of the same form. Each thread loads the next row's
// values and columns before it gathers the current row; a row multiplies
// exactly its slice's w slots in stored order (the bits of k_spmv_sell).
template <int PF, int MINB, bool PERM>
__global__ void __launch_bounds__(TPB, MINB)
    k_sell_pipe_dot(int n, int sigma, int sig_shift, const int64_t *__restrict__ offset,
                    const float *__restrict__ val, const int32_t *__restrict__ col,
                    const void *__restrict__ perm, int perm_bytes, const float *__restrict__ x,
                    float *__restrict__ y, Red red) {
    float d1 = 0.f;
    const int stride = gridDim.x * blockDim.x;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float cv[PF];
    int cc[PF], w = 0;
    int in = i + stride;
    int64_t sn = 0, en = 0;
    if (i < n) {
        const int64_t s = offset[i >> 5];
        w = (int)((offset[(i >> 5) + 1] - s) >> 5);
#pragma unroll
        for (int u = 0; u < PF; ++u) {
            cv[u] = u < w ? __ldcs(val + s + (i & 31) + u * 32) : 0.f;
            cc[u] = u < w ? __ldcs(col + s + (i & 31) + u * 32) : 0;
        }
        if (in < n) {
            sn = offset[in >> 5];
            en = offset[(in >> 5) + 1];
        }
    }
    // the matrix is complete before any solve: its words load before the wait
    grid_dep_sync();
    if (red.sc->done) return;  // solver converged: idle (grid-uniform)
    if (i < n) {
        while (true) {
            const int wn = (int)((en - sn) >> 5);
            float nv[PF];
            int nc[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const bool ok = in < n && u < wn;
                nv[u] = ok ? __ldcs(val + sn + (in & 31) + u * 32) : 0.f;
                nc[u] = ok ? __ldcs(col + sn + (in & 31) + u * 32) : 0;
            }
            const int in2 = in + stride;
            int64_t sn2 = 0, en2 = 0;
            if (in2 < n) {
                sn2 = offset[in2 >> 5];
                en2 = offset[(in2 >> 5) + 1];
            }
            float xv[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) xv[u] = u < w ? __ldg(x + cc[u]) : 0.f;
            float t = 0.f;
#pragma unroll
            for (int u = 0; u < PF; ++u)
                if (u < w) t = fmaf(cv[u], xv[u], t);
            int io = i;
            if (PERM) {
                const int blk = sig_shift >= 0 ? (i >> sig_shift) << sig_shift : (i / sigma) * sigma;
                io = blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[i]
                                            : (int)((const uint16_t *)perm)[i]);
            }
            y[io] = t;
            d1 = fmaf(x[io], t, d1);
            if (in >= n) break;
            i = in;
            w = wn;
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                cv[u] = nv[u];
                cc[u] = nc[u];
            }
            in = in2;
            sn = sn2;
            en = en2;
        }
    }
    reduce_publish(red, (double)d1, 0.0);
}

// Dual-row persistent SpMV: every thread handles two rows per loop trip, row
// i (slice k) and row i + stride (another slice), in lockstep: the word loads
// of both rows are issued before either is decoded, then both rows' gathers,
// then both fused multiply-add chains. Twice the bytes in flight per thread
// of the one-row prefetch kernel, on a persistent grid (the reducing form
// runs on the fixed solver grid). PF words of each row per round.
template <int FMT, int PF, int MINB, bool DOT = false>
__global__ void __launch_bounds__(TPB, MINB)
    k_spmv_dual(int n, int sigma, int sig_shift, long long k_left,
                const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
                const void *__restrict__ perm, int perm_bytes, Decode dc,
                const float *__restrict__ x, float *__restrict__ y, Red red = Red{}) {
    if (DOT && red.sc->done) return;  // solver converged: idle (grid-uniform)
    float d1 = 0.f;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += 2 * stride) {
        const int i1 = i0 + stride;
        const bool has1 = i1 < n;
        const int k0 = i0 >> 5, k1 = i1 >> 5;
        const int64_t s0 = offset[k0];
        const int w0 = (int)((offset[k0 + 1] - s0) >> 5);
        const int64_t s1 = has1 ? offset[k1] : 0;
        const int w1 = has1 ? (int)((offset[k1 + 1] - s1) >> 5) : 0;
        const uint32_t *__restrict__ p0 = pack + s0 + (i0 & 31);
        const uint32_t *__restrict__ p1 = pack + s1 + (i1 & 31);
        const int b0 = sig_shift >= 0 ? (i0 >> sig_shift) << sig_shift : (i0 / sigma) * sigma;
        const int b1 = sig_shift >= 0 ? (i1 >> sig_shift) << sig_shift : (i1 / sigma) * sigma;
        int c0 = (k_left < b0) ? (int)(b0 - k_left) : 0;
        int c1 = (k_left < b1) ? (int)(b1 - k_left) : 0;
        float t0 = 0.f, t1 = 0.f;
        const int wm = w0 > w1 ? w0 : w1;
        for (int j0 = 0; j0 < wm; j0 += PF) {
            const int r0 = w0 - j0, r1 = w1 - j0;
            uint32_t a[PF], b[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) a[u] = (u < r0) ? ldg_stream(p0 + (j0 + u) * 32) : 0u;
#pragma unroll
            for (int u = 0; u < PF; ++u) b[u] = (u < r1) ? ldg_stream(p1 + (j0 + u) * 32) : 0u;
            bool fa[PF], fb[PF];
            float xa[PF], xb[PF];
#pragma unroll
            for (int u = 0; u < PF; ++u) word_gather<FMT>(a[u], dc, x, c0, fa[u], xa[u]);
#pragma unroll
            for (int u = 0; u < PF; ++u) word_gather<FMT>(b[u], dc, x, c1, fb[u], xb[u]);
#pragma unroll
            for (int u = 0; u < PF; ++u)
                if (fa[u]) t0 = fmaf(word_value<FMT>(a[u], dc), xa[u], t0);
#pragma unroll
            for (int u = 0; u < PF; ++u)
                if (fb[u]) t1 = fmaf(word_value<FMT>(b[u], dc), xb[u], t1);
        }
        int o0 = i0, o1 = i1;
        if (perm_bytes == 1) {
            o0 = b0 + (int)((const uint8_t *)perm)[i0];
            if (has1) o1 = b1 + (int)((const uint8_t *)perm)[i1];
        } else if (perm_bytes == 2) {
            o0 = b0 + (int)((const uint16_t *)perm)[i0];
            if (has1) o1 = b1 + (int)((const uint16_t *)perm)[i1];
        }
        y[o0] = t0;
        if (has1) y[o1] = t1;
        if (DOT) {
            d1 = fmaf(x[o0], t0, d1);
            if (has1) d1 = fmaf(x[o1], t1, d1);
        }
    }
    if (DOT) reduce_publish(red, (double)d1, 0.0);
}

template <int FMT, int PF, int MINB>
packsell_status launch_dual(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                            cudaStream_t s) {
    // persistent grid: every block resident at once (cached per process; calls
    // from several host threads may compute it together and store the same value)
    static std::atomic<int> cached{0};
    int blocks = cached.load(std::memory_order_relaxed);
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        PS_CUDA(cudaGetDevice(&dev));
        PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_spmv_dual<FMT, PF, MINB>, TPB, 0));
        blocks = sms * (per > 0 ? per : 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    k_spmv_dual<FMT, PF, MINB><<<blocks, TPB, 0, s>>>((int)A.n, sg, sh, A.p.k_left, A.offset,
                                                      A.pack, perm, pb, make_decode(A), x, y);
    PS_LAUNCH_CHECK("packsell_spmv (dual)");
    return PACKSELL_OK;
}

template <int FMT, int PF, int MINB, bool EXIT>
void launch_prefetch_e(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                       cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sig_shift = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    if (pb)  // the permuted form needs a few more registers: one block fewer per SM
        k_spmv_prefetch<FMT, PF, 32, MINB - 1, false, true, EXIT><<<grid_for(A.n), TPB, 0, s>>>(
            (int)A.n, sg, sig_shift, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
    else
        k_spmv_prefetch<FMT, PF, 32, MINB, false, false, EXIT><<<grid_for(A.n), TPB, 0, s>>>(
            (int)A.n, sg, sig_shift, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
}

template <int FMT, int PF, int MINB>
packsell_status launch_prefetch(const Matrix &A, const void *perm, int pb, const float *x,
                                float *y, cudaStream_t s) {
    // rows stop at their first padding word only where padding is a real
    // share of the stored words (more than 1/8): elsewhere the test costs
    // more than it saves
    if (A.n_pad * 8 > A.n_words)
        launch_prefetch_e<FMT, PF, MINB, true>(A, perm, pb, x, y, s);
    else
        launch_prefetch_e<FMT, PF, MINB, false>(A, perm, pb, x, y, s);
    PS_LAUNCH_CHECK("packsell_spmv (prefetch)");
    return PACKSELL_OK;
}

// Variant 13: the kernel of variant 5 (rows run to the slice width) launched
// with programmatic stream serialisation, so that its blocks are scheduled
// while the previous kernel of the stream drains and load their first words
// before they wait for it.
template <int FMT, int PF, int MINB>
packsell_status launch_prefetch_pdl(const Matrix &A, const void *perm, int pb, const float *x,
                                    float *y, cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    const unsigned g = (unsigned)grid_for(A.n);
    const int n = (int)A.n;
    const long long kl = A.p.k_left;
    const int64_t *offset = A.offset;
    const uint32_t *pack = A.pack;
    const Decode dc = make_decode(A);
    const cudaError_t e =
        pb ? launch_pdl(k_spmv_prefetch<FMT, PF, 32, MINB - 1, false, true, false, true>, g, TPB, s, n,
                        sg, sh, kl, offset, pack, perm, pb, dc, x, y, Red{})
           : launch_pdl(k_spmv_prefetch<FMT, PF, 32, MINB, false, false, false, true>, g, TPB, s, n, sg,
                        sh, kl, offset, pack, perm, pb, dc, x, y, Red{});
    if (e != cudaSuccess) return cuda_fail(e, "packsell_spmv (variant 13)");
    PS_LAUNCH_CHECK("packsell_spmv (variant 13)");
    return PACKSELL_OK;
}

// variant 13 with its round size fitted to the widest slice (as variant 5)
template <int FMT>
packsell_status prefetch_pdl_rounds(int pf, const Matrix &A, const void *perm, int pb,
                                    const float *x, float *y, cudaStream_t s) {
    if (pf == 8) return launch_prefetch_pdl<FMT, 8, 6>(A, perm, pb, x, y, s);
    if (pf == 10) return launch_prefetch_pdl<FMT, 10, 6>(A, perm, pb, x, y, s);
    if (pf == 12) return launch_prefetch_pdl<FMT, 12, 5>(A, perm, pb, x, y, s);
    return launch_prefetch_pdl<FMT, 16, 5>(A, perm, pb, x, y, s);
}

template <int FMT, int PF, int MINB, bool PERM>
int pipe_blocks() {
    // persistent grid: every block resident at once (cached as in launch_dual)
    static std::atomic<int> cached{0};
    int blocks = cached.load(std::memory_order_relaxed);
    if (!blocks) {
        int dev = 0, sms = 0, per = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per, k_spmv_pipe<FMT, PF, MINB, false, PERM>, TPB, 0) != cudaSuccess)
            return 0;
        blocks = sms * std::max(per, 1);
        cached.store(blocks, std::memory_order_relaxed);
    }
    return blocks;
}

template <int FMT, int PF, int MINB>
packsell_status launch_pipe(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                            cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    const int blocks = pb ? pipe_blocks<FMT, PF, MINB, true>() : pipe_blocks<FMT, PF, MINB, false>();
    if (!blocks) return fail(PACKSELL_ERR_CUDA, "packsell_spmv (pipelined): device query failed");
    if (pb)
        k_spmv_pipe<FMT, PF, MINB, false, true><<<blocks, TPB, 0, s>>>(
            (int)A.n, sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
    else
        k_spmv_pipe<FMT, PF, MINB, false, false><<<blocks, TPB, 0, s>>>(
            (int)A.n, sg, sh, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
    PS_LAUNCH_CHECK("packsell_spmv (pipelined)");
    return PACKSELL_OK;
}

// Bulk-staged PackSELL SpMV (C = 32).
//
// Warp gw owns the contiguous slices [part[gw], part[gw+1]): one contiguous
// run of words (a "stream"), which it copies into a circular shared-memory
// ring of NS chunks of SW words with cp.async.bulk (TMA engine); chunk g of
// the stream lands in ring words [(g*SW) & MASK, ...) and completes on
// mbarrier g % NS. Lane 0 keeps up to NS chunks in flight; the whole warp
// waits on a chunk's mbarrier (bounded) before reading it, and lane 0
// re-issues a slot once the warp has moved past its chunk. Bytes in flight
// per warp are up to NS * SW * 4, independent of registers.
//
// Lane l decodes row l of each slice; its word j sits at stream position
// s0 + 32 j + l, i.e. ring[(s0 + 32 j + l) & MASK]: 32 consecutive words per
// column, one bank per lane. A slice is processed in one pass once all chunks
// it touches have landed (slices up to (NS-1)*SW/32 columns wide); wider
// slices are processed chunk by chunk. Rows are summed in stored order with
// one fused multiply-add per value word, so the result equals the
// thread-per-row kernel's bits (a word without a value adds 0 * 0, which
// leaves a sum that starts at +0 unchanged).
template <int NS, int SW>
struct BulkRing {
    static constexpr int RING = NS * SW;
    static_assert((SW & (SW - 1)) == 0 && SW % 32 == 0, "SW: power of two, whole columns");
    // ring word of stream position q: chunk q / SW sits in slot (q / SW) % NS
    __device__ static __forceinline__ int at(int q) { return ((q / SW) % NS) * SW + (q & (SW - 1)); }
};

template <int NS, int SW>
__device__ __forceinline__ int bulk_issue(int lane, int next, int lim, int total,
                                          const uint32_t *__restrict__ src, uint32_t *ring,
                                          uint64_t *bar, uint64_t pol) {
    if (lane == 0) {
        for (int g = next; g < lim; ++g) {
            const int q = g % NS;
            const int w0 = g * SW;
            const int cnt = total - w0 < SW ? total - w0 : SW;
            const uint32_t bytes = (uint32_t)cnt * 4u;
            mbar_expect_tx(&bar[q], bytes);
            bulk_g2s(ring + q * SW, src + w0, bytes, &bar[q], pol);
        }
    }
    return lim > next ? lim : next;
}

// Accumulate columns [j0, j1) of one row from ring words at p + 32 j (the
// caller's ring base already includes the lane): full groups of 8 with all
// loads and gathers first, then the group's fused multiply-adds in order,
// and a word-at-a-time tail.
struct RowState {
    int c;
    float t;
};

template <int FMT>
__device__ __forceinline__ RowState row_run(const uint32_t *ring, int p, int j0, int j1, Decode dc,
                                            const float *__restrict__ x, RowState r) {
    int c = r.c;
    float t = r.t;
    int j = j0;
    for (; j + 8 <= j1; j += 8) {
        uint32_t wd[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) wd[u] = ring[p + 32 * (j + u)];
        bool f[8];
        float xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) word_gather<FMT>(wd[u], dc, x, c, f[u], xv[u]);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (f[u]) t = fmaf(word_value<FMT>(wd[u], dc), xv[u], t);
    }
    for (; j < j1; ++j) {
        const uint32_t wd = ring[p + 32 * j];
        bool f;
        float xv;
        word_gather<FMT>(wd, dc, x, c, f, xv);
        if (f) t = fmaf(word_value<FMT>(wd, dc), xv, t);
    }
    return RowState{c, t};
}

// The run above as a real call (fewer registers in the caller) or inlined.
template <int FMT>
__device__ __noinline__ RowState row_run_call(const uint32_t *ring, int p, int j0, int j1,
                                              Decode dc, const float *__restrict__ x, RowState r) {
    return row_run<FMT>(ring, p, j0, j1, dc, x, r);
}

template <int FMT, bool INL>
__device__ __forceinline__ RowState bulk_row_run(const uint32_t *ring, int p, int j0, int j1,
                                                 Decode dc, const float *__restrict__ x,
                                                 RowState r) {
    return INL ? row_run<FMT>(ring, p, j0, j1, dc, x, r) : row_run_call<FMT>(ring, p, j0, j1, dc, x, r);
}

template <int FMT, int NW, int NS, int SW, int MINB, bool INL>
__global__ void __launch_bounds__(NW * 32, MINB)
    k_spmv_bulk(int n, int sigma, int sig_shift, long long k_left,
                const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
                const void *__restrict__ perm, int perm_bytes, Decode dc,
                const float *__restrict__ x, float *__restrict__ y,
                const int32_t *__restrict__ part, DevStatus *st, uint32_t wait_limit) {
    using R = BulkRing<NS, SW>;
    extern __shared__ __align__(128) uint32_t ring_all[];
    __shared__ __align__(8) uint64_t bars[NW][NS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NW + warp;
    const int k0 = part[gw], k1 = part[gw + 1];
    if (k0 >= k1) return;  // warp-uniform
    uint32_t *ring = ring_all + warp * R::RING;
    uint64_t *bar = bars[warp];
    const int64_t base = offset[k0];
    const int total = (int)(offset[k1] - base);  // words of this warp's stream
    const uint32_t *src = pack + base;
    const int nchunks = (total + SW - 1) / SW;
    const uint64_t pol = policy_evict_first();
    if (lane == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncwarp();
    int issued = bulk_issue<NS, SW>(lane, 0, NS < nchunks ? NS : nchunks, total, src, ring, bar, pol);
    int waited = 0;    // chunks [0, waited) have landed
    int released = 0;  // chunks [0, released) are consumed

    // wait for chunks up to and including g (in order); false on timeout
    auto wait_upto = [&](int g) -> bool {
        for (; waited <= g; ++waited) {
            bool ok = mbar_wait(&bar[waited % NS], (uint32_t)((waited / NS) & 1), wait_limit);
            if (!__all_sync(0xffffffffu, ok)) return false;
        }
        return true;
    };
    // the warp no longer reads chunks below g: refill their slots
    auto release_below = [&](int g) {
        if (g > released) {
            released = g;
            __syncwarp();
            if (lane == 0) fence_proxy_async_smem();
            const int lim = released + NS < nchunks ? released + NS : nchunks;
            issued = bulk_issue<NS, SW>(lane, issued, lim, total, src, ring, bar, pol);
        }
    };

    for (int kb = k0; kb < k1; kb += 32) {
        const int nk = (k1 - kb < 32) ? (k1 - kb) : 32;
        const int o_lo = (lane < nk) ? (int)(offset[kb + lane] - base) : 0;
        const int o_hi = (lane < nk) ? (int)(offset[kb + lane + 1] - base) : 0;
        for (int q = 0; q < nk; ++q) {
            const int s0 = __shfl_sync(0xffffffffu, o_lo, q);
            const int s1 = __shfl_sync(0xffffffffu, o_hi, q);
            const int w = (s1 - s0) >> 5;
            const int row = (kb + q) * 32 + lane;
            const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
            RowState rs{(k_left < blk) ? (int)(blk - k_left) : 0, 0.f};
            int yo = row;
            if (perm_bytes == 1) yo = blk + (int)((const uint8_t *)perm)[min(row, n - 1)];
            else if (perm_bytes == 2) yo = blk + (int)((const uint16_t *)perm)[min(row, n - 1)];
            if (w > 0) {
                if (s1 - s0 <= (NS - 1) * SW) {
                    // whole slice resident at once; a slice that runs past the
                    // ring's last word continues at ring word 0
                    if (!wait_upto((s1 - 1) / SW)) goto timeout;
                    const int r0 = R::at(s0);
                    const int room = (R::RING - r0) >> 5;  // columns before the ring's end
                    if (w <= room) {
                        rs = bulk_row_run<FMT, INL>(ring, r0 + lane, 0, w, dc, x, rs);
                    } else {
                        rs = bulk_row_run<FMT, INL>(ring, r0 + lane, 0, room, dc, x, rs);
                        rs = bulk_row_run<FMT, INL>(ring, lane - 32 * room, room, w, dc, x, rs);
                    }
                    release_below(s1 / SW);
                } else {
                    // wide slice: one chunk at a time
                    int j = 0;
                    while (j < w) {
                        const int pos = s0 + 32 * j;
                        const int g = pos / SW;
                        if (!wait_upto(g)) goto timeout;
                        const int jend = min(w, j + (((g + 1) * SW - pos) >> 5));
                        rs = bulk_row_run<FMT, INL>(ring, R::at(pos) + lane - 32 * j, j, jend, dc, x, rs);
                        j = jend;
                        release_below(s0 + 32 * j < s1 ? (s0 + 32 * j) / SW : s1 / SW);
                    }
                }
            }
            if (row < n) y[yo] = rs.t;
        }
    }
    return;
timeout:
    if (lane == 0) dev_fail(st, PACKSELL_ERR_TIMEOUT, gw);
    // let every copy already issued land before the block's shared memory goes
    for (int g = waited; g < issued; ++g) mbar_wait(&bar[g % NS], (uint32_t)((g / NS) & 1));
}

// Bulk kernel configurations (warps per block, chunks per warp, words per
// chunk), selected as SpMV variants 2, 3 and 4.
struct BulkCfg {
    int nw, ns, sw;
    size_t smem() const { return sizeof(uint32_t) * (size_t)nw * ns * sw; }
};
constexpr BulkCfg kBulkCfg[3] = {{8, 3, 512}, {4, 3, 512}, {8, 2, 1024}};

template <int FMT, int V>
struct BulkKernel;
// MINB: blocks per SM that the configuration's shared memory allows, so
// the register budget matches the occupancy the ring sizes permit
#define PS_BULK_KERNEL(V, NW, NS, SW, MINB, INL)                                        \
    template <int FMT>                                                                  \
    struct BulkKernel<FMT, V> {                                                         \
        static constexpr auto fn = k_spmv_bulk<FMT, NW, NS, SW, MINB, INL>;             \
    };
PS_BULK_KERNEL(0, 8, 3, 512, 4, false)
PS_BULK_KERNEL(1, 4, 3, 512, 9, false)
PS_BULK_KERNEL(2, 8, 2, 1024, 3, true)
#undef PS_BULK_KERNEL

// part[g] = first slice whose word offset reaches g * N_w / G, g = 0..G.
__global__ void k_partition(int64_t S, const int64_t *__restrict__ offset, int G,
                            int32_t *__restrict__ part) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > G) return;
    int64_t total = offset[S];
    int64_t target = (int64_t)((__int128)total * g / G);
    int64_t lo = 0, hi = S;  // first k in [0, S] with offset[k] >= target
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (offset[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    part[g] = (int32_t)(g == G ? S : lo);
}

template <int FMT>
void *bulk_fn(int v) {
    switch (v) {
        case 0: return (void *)BulkKernel<FMT, 0>::fn;
        case 1: return (void *)BulkKernel<FMT, 1>::fn;
        default: return (void *)BulkKernel<FMT, 2>::fn;
    }
}

template <int FMT>
packsell_status launch_bulk(const Matrix &A, int v, const void *perm, int pb, const float *x,
                            float *y, cudaStream_t s) {
    const int sg = A.p.sigma;
    int sig_shift = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    int n = (int)A.n;
    long long kl = A.p.k_left;
    Decode dc = make_decode(A);
    const int32_t *part = A.part[v];
    DevStatus *st = A.status;
    const BulkCfg &cf = kBulkCfg[v];
    int sigma = sg;
    const int64_t *offset = A.offset;
    const uint32_t *pack = A.pack;
    uint32_t wl = data_wait_limit();
    void *kargs[] = {&n, &sigma, &sig_shift, &kl, (void *)&offset, (void *)&pack, (void *)&perm,
                     &pb, &dc, (void *)&x, (void *)&y, (void *)&part, (void *)&st, &wl};
    PS_CUDA(cudaLaunchKernel(bulk_fn<FMT>(v), dim3(A.part_blocks[v]), dim3(cf.nw * 32), kargs,
                             cf.smem(), s));
    return PACKSELL_OK;
}

// Plain SELL-C-sigma (§3): value and column streams, padding multiplies 0.
// With DOT the kernel also reduces sum_i x_i y_i and sum_i x_i b_i over the
// output rows (square matrices, original order).
// PDL (launched by launch_pdl): in the single pass the first round of values
// and columns loads before the grid waits for the previous kernel of the
// stream; the reducing form waits first.
template <typename T, bool DOT, bool PDL>
__device__ __forceinline__ void sell_rows(int n, int C, int sigma,
                                          const int64_t *__restrict__ offset,
                                          const T *__restrict__ val,
                                          const int32_t *__restrict__ col,
                                          const void *__restrict__ perm, int perm_bytes,
                                          const T *__restrict__ x, T *__restrict__ y,
                                          const T *__restrict__ b, Red red) {
    if (DOT && PDL) grid_dep_sync();  // the reducing form waits before it starts
    if (!DOT && PDL) grid_dep_launch();  // one pass over the rows: signal at block start
    if (DOT && red.sc->done) return;  // solver converged: idle (grid-uniform)
    T d1 = 0, d2 = 0;  // per-thread sums in T; block and grid sums in FP64
    const int stride = DOT ? gridDim.x * blockDim.x : n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int k = i / C, l = i - k * C;
        const int64_t s = offset[k];
        const int w = (int)((offset[k + 1] - s) / C);
        const T *vp = val + s + l;
        const int32_t *cp = col + s + l;
        T t = 0;
        int j = 0;
        if (PDL && !DOT && w < UNROLL) grid_dep_wait();
        for (; j + UNROLL <= w; j += UNROLL) {
            T v[UNROLL];
            int cc[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                v[u] = __ldcs(vp + (int64_t)(j + u) * C);
                cc[u] = __ldcs(cp + (int64_t)(j + u) * C);
            }
            // every round (returns at once after the first): a wait in the
            // first round alone makes the compiler peel it (34 -> 62 registers)
            if (PDL && !DOT) grid_dep_wait();
            T xv[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) xv[u] = __ldg(x + cc[u]);
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) t = fma(v[u], xv[u], t);
        }
        for (; j < w; ++j) t = fma(__ldcs(vp + (int64_t)j * C), __ldg(x + __ldcs(cp + (int64_t)j * C)), t);
        const int io = orig_row(i, sigma, perm, perm_bytes);
        y[io] = t;
        if (DOT) {
            d1 = fma(x[io], t, d1);
            if (b) d2 = fma(x[io], b[io], d2);
        }
    }
    if (DOT) reduce_publish(red, (double)d1, (double)d2);
}

template <typename T, bool DOT = false, bool PDL = false>
__global__ void __launch_bounds__(TPB)
    k_spmv_sell(int n, int C, int sigma, const int64_t *__restrict__ offset,
                const T *__restrict__ val, const int32_t *__restrict__ col,
                const void *__restrict__ perm, int perm_bytes, const T *__restrict__ x,
                T *__restrict__ y, const T *__restrict__ b = nullptr, Red red = Red{}) {
    sell_rows<T, DOT, PDL>(n, C, sigma, offset, val, col, perm, perm_bytes, x, y, b, red);
}

// The FP64 reducing form (FP64 PCG and the outer loop of IO-CG) with a
// register budget of four blocks per SM: left to itself the compiler fits
// it in 32 registers and spills.
__global__ void __launch_bounds__(TPB, 4)
    k_spmv_sell_dot64(int n, int C, int sigma, const int64_t *__restrict__ offset,
                      const double *__restrict__ val, const int32_t *__restrict__ col,
                      const void *__restrict__ perm, int perm_bytes, const double *__restrict__ x,
                      double *__restrict__ y, const double *__restrict__ b, Red red) {
    sell_rows<double, true, true>(n, C, sigma, offset, val, col, perm, perm_bytes, x, y, b, red);
}

// FP16 SELL (binary16 values, int32 columns, padding at column -1): one
// thread per row, each nonzero one fused multiply-add in stored order; the
// padding slots, trailing each row, add nothing, so a row's sum is the chain
// of the FP16 PackSELL kernels over the same values. The loads of a round of
// UNROLL slots go out before any is used, as in the FP32 SELL kernel, and the
// launch is programmatic (values and columns load before the wait on the
// previous kernel of the stream; x and y after it).
template <int U, bool C32>
__global__ void __launch_bounds__(TPB)
    k_spmv_sell16(int n, int Cr, int sigma, const int64_t *__restrict__ offset,
                  const uint16_t *__restrict__ val, const int32_t *__restrict__ col,
                  const void *__restrict__ perm, int perm_bytes, const float *__restrict__ x,
                  float *__restrict__ y) {
    const int C = C32 ? 32 : Cr;  // a constant slot stride when C = 32
    grid_dep_launch();  // one pass over the rows: signal at block start
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) {
        grid_dep_wait();
        return;
    }
    const int k = i / C, l = i - k * C;
    const int64_t s = offset[k];
    const int w = (int)((offset[k + 1] - s) / C);
    const uint16_t *vp = val + s + l;
    const int32_t *cp = col + s + l;
    float t = 0.f;
    bool waited = false;
    for (int j = 0; j < w; j += U) {
        uint16_t v[U];
        int cc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = j + u < w;
            v[u] = ok ? __ldcs(vp + (int64_t)(j + u) * C) : (uint16_t)0;
            cc[u] = ok ? __ldcs(cp + (int64_t)(j + u) * C) : -1;
        }
        if (!waited) {
            grid_dep_wait();
            waited = true;
        }
        float xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) xv[u] = cc[u] >= 0 ? __ldg(x + cc[u]) : 0.f;
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (cc[u] >= 0) t = fmaf(__half2float(__ushort_as_half(v[u])), xv[u], t);
        if (cc[U - 1] < 0) break;  // padding: the row has ended
    }
    if (!waited) grid_dep_wait();
    y[orig_row(i, sigma, perm, perm_bytes)] = t;
}

// Thread-per-row PackSELL SpMV fused with sum_i x_i y_i (solver use, any C),
// on a fixed grid striding over rows.
template <int FMT>
__global__ void __launch_bounds__(TPB)
    k_spmv_packed_dot(int n, int C, int sigma, long long k_left,
                      const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
                      const void *__restrict__ perm, int perm_bytes, Decode dc,
                      const float *__restrict__ x, float *__restrict__ y, Red red) {
    if (red.sc->done) return;  // solver converged: idle (grid-uniform)
    float d1 = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int k = i / C, l = i - k * C;
        const int64_t s = offset[k];
        const int w = (int)((offset[k + 1] - s) / C);
        int c = left_offset(i, sigma, k_left);
        float t = 0.f;
        for (int j = 0; j < w; ++j) {
            bool f;
            float xv;
            const uint32_t wd = ldg_stream(pack + s + (int64_t)j * C + l);
            word_gather<FMT>(wd, dc, x, c, f, xv);
            if (f) t = fmaf(word_value<FMT>(wd, dc), xv, t);
        }
        const int io = orig_row(i, sigma, perm, perm_bytes);
        y[io] = t;
        d1 = fmaf(x[io], t, d1);
    }
    reduce_publish(red, (double)d1, 0.0);
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
        if (f && g != 0.f && PS_IN_RANGE(c, dc.xlen)) atomicAdd(dx + c, v * g);
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
        if (f && PS_IN_RANGE(c, dc.xlen) && PS_IN_RANGE(q, rowptr[io + 1])) out[q] = a * v[c];
        q += f;
    }
}

template <typename T>
__global__ void __launch_bounds__(TPB)
    k_pattern_outer_sell(int n, int C, int sigma, const int64_t *__restrict__ offset,
                         const int32_t *__restrict__ col, const void *__restrict__ perm,
                         int perm_bytes, const int64_t *__restrict__ rowptr, T alpha,
                         const T *__restrict__ u, const T *__restrict__ v,
                         T *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int io = orig_row(i, sigma, perm, perm_bytes);
    T a = alpha * u[io];
    int64_t q0 = rowptr[io], len = rowptr[io + 1] - q0;
    for (int64_t j = 0; j < len; ++j) out[q0 + j] = a * v[col[s + j * C + l]];
}

}  // namespace

// Polls of the staged kernels' waits for data (packsell_set_wait_limit).
static std::atomic<uint32_t> g_wait_limit{kWaitLimit};
uint32_t data_wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }
void set_data_wait_limit(uint32_t limit) { g_wait_limit.store(limit, std::memory_order_relaxed); }

// Launch plan of the bulk-staged kernels: for each configuration a
// persistent grid of as many blocks as fit on the device, and the per-warp
// slice partition balanced by words. Variant 0 then runs configuration 0.
packsell_status plan_spmv(Matrix &A, cudaStream_t s) {
    if (!A.status) {
        PS_CUDA(cudaMalloc(&A.status, sizeof(DevStatus)));
        PS_CUDA(cudaMemsetAsync(A.status, 0, sizeof(DevStatus), s));
    }
    A.auto_variant = 1;
    if (is_packed(A.p.format) && A.p.C == 1 && A.n > 0 && A.n < INT32_MAX) {
        packsell_status st = plan_csr(A, s);
        if (st != PACKSELL_OK) return st;
        st = plan_split(A, s);
        if (st != PACKSELL_OK) return st;
        st = multi_plan(A, s);
        if (st != PACKSELL_OK) return st;
        // untuned default for CSR order: the split-row kernel (all lanes busy
        // on rows of any length); variant 11 keeps the stored-order chain
        if (A.split_items) A.auto_variant = 14;
        else if (A.csr_items) A.auto_variant = 11;
        return PACKSELL_OK;
    }
    // fixed point in slices of 32 rows: the row-prefetch kernel (variant 13)
    if (is_fixed(A.p.format) && A.p.C == 32 && A.n > 0) A.auto_variant = 13;
    // the bulk kernel indexes a warp's words with 32-bit integers
    if (!is_packed(A.p.format) || A.p.C != 32 || A.n == 0 || A.n_words >= (1ll << 31) - 4096)
        return PACKSELL_OK;
    int dev = 0, sms = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int v = 0; v < Matrix::kBulkVariants; ++v) {
        const BulkCfg &cf = kBulkCfg[v];
        void *fn = A.p.format == PACKSELL_FMT_FP16 ? bulk_fn<PACKSELL_FMT_FP16>(v)
                                                   : bulk_fn<PACKSELL_FMT_E8MY>(v);
        PS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cf.smem()));
        int per_sm = 0;
        PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, cf.nw * 32, cf.smem()));
        if (per_sm < 1) continue;
        const int blocks = sms * per_sm, G = blocks * cf.nw;
        if (A.part[v]) cudaFree(A.part[v]);
        A.part[v] = nullptr;
        PS_CUDA(cudaMalloc(&A.part[v], sizeof(int32_t) * (G + 1)));
        k_partition<<<(G + 1 + 255) / 256, 256, 0, s>>>(A.n_slices, A.offset, G, A.part[v]);
        PS_LAUNCH_CHECK("k_partition");
        A.part_blocks[v] = blocks;
        A.part_warps[v] = G;
    }
    // untuned default (variant 0), by matrix shape: every slice within one
    // round -> the pipelined kernel; padding above 1/8 of the words (uneven
    // rows) -> the TMA-staged variant 4; otherwise -> variant 13
    if (A.max_width <= 16) A.auto_variant = 12;
    else if (A.n_pad * 8 > A.n_words && A.part[2]) A.auto_variant = 4;
    else A.auto_variant = 13;
    return plan_stage(A, s);
}

packsell_status spmv_impl(const Matrix &A, const float *x, float *y, cudaStream_t s) {
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    int g = grid_for(A.n);
    const int var = A.variant == 0 ? A.auto_variant : A.variant;
    if (var == 11 && is_packed(A.p.format)) return launch_csr(A, perm, pb, x, y, s);
    if (var == 14 && is_packed(A.p.format)) return launch_split(A, perm, pb, x, y, s);
    if (var == 12 && is_packed(A.p.format)) {
        if (A.p.C != 32 || A.max_width > 16)
            return fail(PACKSELL_ERR_INVALID_ARG,
                        "packsell_spmv: variant 12 needs C = 32 and slices of at most 16 words");
        const bool h = A.p.format == PACKSELL_FMT_FP16;
        const int pf = round_words(A.max_width);
        if (pf == 8)
            return h ? launch_pipe<PACKSELL_FMT_FP16, 8, 5>(A, perm, pb, x, y, s)
                     : launch_pipe<PACKSELL_FMT_E8MY, 8, 5>(A, perm, pb, x, y, s);
        if (pf == 10)
            return h ? launch_pipe<PACKSELL_FMT_FP16, 10, 4>(A, perm, pb, x, y, s)
                     : launch_pipe<PACKSELL_FMT_E8MY, 10, 4>(A, perm, pb, x, y, s);
        if (pf == 12)
            return h ? launch_pipe<PACKSELL_FMT_FP16, 12, 4>(A, perm, pb, x, y, s)
                     : launch_pipe<PACKSELL_FMT_E8MY, 12, 4>(A, perm, pb, x, y, s);
        return h ? launch_pipe<PACKSELL_FMT_FP16, 16, 3>(A, perm, pb, x, y, s)
                 : launch_pipe<PACKSELL_FMT_E8MY, 16, 3>(A, perm, pb, x, y, s);
    }
    if ((var == 9 || var == 10) && is_packed(A.p.format))
        return launch_stage(A, var - 9, perm, pb, x, y, s);
    if ((var == 7 || var == 8) && is_packed(A.p.format)) {
        if (A.p.C != 32)
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: the dual-row variants need C = 32");
        const bool h = A.p.format == PACKSELL_FMT_FP16;
        if (var == 7) {
            const int pf = std::min(12, round_words(A.max_width));
            if (pf == 8)
                return h ? launch_dual<PACKSELL_FMT_FP16, 8, 5>(A, perm, pb, x, y, s)
                         : launch_dual<PACKSELL_FMT_E8MY, 8, 5>(A, perm, pb, x, y, s);
            if (pf == 10)
                return h ? launch_dual<PACKSELL_FMT_FP16, 10, 4>(A, perm, pb, x, y, s)
                         : launch_dual<PACKSELL_FMT_E8MY, 10, 4>(A, perm, pb, x, y, s);
            return h ? launch_dual<PACKSELL_FMT_FP16, 12, 4>(A, perm, pb, x, y, s)
                     : launch_dual<PACKSELL_FMT_E8MY, 12, 4>(A, perm, pb, x, y, s);
        }
        return h ? launch_dual<PACKSELL_FMT_FP16, 16, 3>(A, perm, pb, x, y, s)
                 : launch_dual<PACKSELL_FMT_E8MY, 16, 3>(A, perm, pb, x, y, s);
    }
    if (var == 13 && (is_packed(A.p.format) || is_fixed(A.p.format))) {
        if (A.p.C != 32)
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: variant 13 needs C = 32");
        const int pf = round_words(A.max_width);
        switch (A.p.format) {
            case PACKSELL_FMT_FP16: return prefetch_pdl_rounds<PACKSELL_FMT_FP16>(pf, A, perm, pb, x, y, s);
            case PACKSELL_FMT_E8MY: return prefetch_pdl_rounds<PACKSELL_FMT_E8MY>(pf, A, perm, pb, x, y, s);
            default: return prefetch_pdl_rounds<PACKSELL_FMT_FIXED>(pf, A, perm, pb, x, y, s);
        }
    }
    if ((var == 5 || var == 6) && is_packed(A.p.format)) {
        if (A.p.C != 32)
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: the prefetch variants need C = 32");
        const bool h = A.p.format == PACKSELL_FMT_FP16;
        if (var == 6)
            return h ? launch_prefetch<PACKSELL_FMT_FP16, 32, 4>(A, perm, pb, x, y, s)
                     : launch_prefetch<PACKSELL_FMT_E8MY, 32, 4>(A, perm, pb, x, y, s);
        // round size fitted to the widest slice: decoded slots past a row's
        // width are wasted work, which dominates on short rows
        const int pf = round_words(A.max_width);
        if (pf == 8)
            return h ? launch_prefetch<PACKSELL_FMT_FP16, 8, 6>(A, perm, pb, x, y, s)
                     : launch_prefetch<PACKSELL_FMT_E8MY, 8, 6>(A, perm, pb, x, y, s);
        if (pf == 10)
            return h ? launch_prefetch<PACKSELL_FMT_FP16, 10, 6>(A, perm, pb, x, y, s)
                     : launch_prefetch<PACKSELL_FMT_E8MY, 10, 6>(A, perm, pb, x, y, s);
        if (pf == 12)
            return h ? launch_prefetch<PACKSELL_FMT_FP16, 12, 5>(A, perm, pb, x, y, s)
                     : launch_prefetch<PACKSELL_FMT_E8MY, 12, 5>(A, perm, pb, x, y, s);
        return h ? launch_prefetch<PACKSELL_FMT_FP16, 16, 5>(A, perm, pb, x, y, s)
                 : launch_prefetch<PACKSELL_FMT_E8MY, 16, 5>(A, perm, pb, x, y, s);
    }
    if (var >= 2 && var <= 4 && is_packed(A.p.format)) {
        const int v = var - 2;
        if (v >= Matrix::kBulkVariants || !A.part[v])
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: bulk-staged variant unavailable");
        return A.p.format == PACKSELL_FMT_FP16 ? launch_bulk<PACKSELL_FMT_FP16>(A, v, perm, pb, x, y, s)
                                               : launch_bulk<PACKSELL_FMT_E8MY>(A, v, perm, pb, x, y, s);
    }
    switch (A.p.format) {
        case PACKSELL_FMT_FP16:
            k_spmv_packed<PACKSELL_FMT_FP16><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
            break;
        case PACKSELL_FMT_E8MY:
            k_spmv_packed<PACKSELL_FMT_E8MY><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
            break;
        case PACKSELL_FMT_SELL_F32: {
            const cudaError_t e = launch_pdl(k_spmv_sell<float, false, true>, (unsigned)g, TPB, s,
                                             (int)A.n, A.p.C, A.p.sigma, (const int64_t *)A.offset,
                                             (const float *)A.val, (const int32_t *)A.col, perm,
                                             pb, x, y, (const float *)nullptr, Red{});
            if (e != cudaSuccess) return cuda_fail(e, "packsell_spmv (SELL)");
            break;
        }
        case PACKSELL_FMT_FIXED:
            k_spmv_packed<PACKSELL_FMT_FIXED><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y);
            break;
        case PACKSELL_FMT_SELL_F16: {
            // rounds of 16 slots where rows are longer than 8 (as the PackSELL
            // row-prefetch kernel), a constant slot stride when C = 32
            const bool wide = A.max_width > 8, c32 = A.p.C == 32;
            auto k = wide ? (c32 ? k_spmv_sell16<16, true> : k_spmv_sell16<16, false>)
                          : (c32 ? k_spmv_sell16<8, true> : k_spmv_sell16<8, false>);
            const cudaError_t e = launch_pdl(k, (unsigned)g, TPB, s, (int)A.n, A.p.C,
                                             A.p.sigma, (const int64_t *)A.offset,
                                             (const uint16_t *)A.val, (const int32_t *)A.col, perm,
                                             pb, x, y);
            if (e != cudaSuccess) return cuda_fail(e, "packsell_spmv (FP16 SELL)");
            break;
        }
        default:
            return fail(PACKSELL_ERR_INVALID_ARG,
                        "packsell_spmv: SELL_F64 and W64_E11MY need packsell_spmv_f64");
    }
    PS_LAUNCH_CHECK("packsell_spmv");
    return PACKSELL_OK;
}

packsell_status spmv_f64_impl(const Matrix &A, const double *x, double *y, cudaStream_t s) {
    if (is_w64(A.p.format)) return spmv_w64_impl(A, x, y, s);
    if (A.p.format != PACKSELL_FMT_SELL_F64)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_spmv_f64: matrix is neither SELL_F64 nor W64_E11MY");
    if (A.n == 0) return PACKSELL_OK;
    const void *perm = A.p.explicit_perm ? nullptr : A.perm;
    int pb = A.p.explicit_perm ? 0 : A.perm_bytes;
    k_spmv_sell<double><<<grid_for(A.n), TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset,
                                                      (const double *)A.val, A.col, perm, pb, x, y);
    PS_LAUNCH_CHECK("packsell_spmv_f64");
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
            if (A.p.format != PACKSELL_FMT_SELL_F32)
                return fail(PACKSELL_ERR_INVALID_ARG,
                            "packsell_pattern_outer: SELL_F64 needs packsell_pattern_outer_f64");
            k_pattern_outer_sell<float><<<g, TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset, A.col,
                                                          perm, pb, A.rowptr, alpha, u, v, out);
            break;
    }
    PS_LAUNCH_CHECK("packsell_pattern_outer");
    return PACKSELL_OK;
}

// ---- fused SpMV + dot launchers for the solvers (square, original order) ----
// Reducing kernels run on fixed grids of at most 8 blocks per SM (the size of
// the partial-sum buffers); each kernel's grid depends only on the device.
int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        sms = 160;  // no device yet: size for a large part
    }
    return std::max(1, sms);
}

int reduce_blocks() { return device_sms() * 8; }

// persistent grid of a reducing kernel: resident blocks, at most 8 per SM
template <typename K>
int dot_grid(K kern) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, TPB, 0) != cudaSuccess) {
        cudaGetLastError();
        per = 4;
    }
    return device_sms() * std::min(8, std::max(1, per));
}

template <int FMT, int PF, int MINB>
void launch_prefetch_dot(const Matrix &A, const float *x, float *y, const Red &red,
                         cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    if (A.perm_bytes) {
        auto k = k_spmv_prefetch<FMT, PF, 32, MINB - 1, true, true>;
        k<<<dot_grid(k), TPB, 0, s>>>((int)A.n, sg, sh, A.p.k_left, A.offset, A.pack, A.perm,
                                      A.perm_bytes, make_decode(A), x, y, red);
    } else {
        auto k = k_spmv_prefetch<FMT, PF, 32, MINB, true, false>;
        k<<<dot_grid(k), TPB, 0, s>>>((int)A.n, sg, sh, A.p.k_left, A.offset, A.pack, A.perm, 0,
                                      make_decode(A), x, y, red);
    }
}

template <int FMT, int PF, int MINB>
cudaError_t launch_pipe_dot(const Matrix &A, const float *x, float *y, const Red &red,
                            cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    if (A.perm_bytes) {
        auto k = k_spmv_pipe<FMT, PF, MINB, true, true, true>;
        return launch_pdl(k, (unsigned)dot_grid(k), TPB, s, (int)A.n, sg, sh, A.p.k_left,
                          (const int64_t *)A.offset, (const uint32_t *)A.pack,
                          (const void *)A.perm, A.perm_bytes, make_decode(A), x, y, red);
    }
    auto k = k_spmv_pipe<FMT, PF, MINB, true, false, true>;
    return launch_pdl(k, (unsigned)dot_grid(k), TPB, s, (int)A.n, sg, sh, A.p.k_left,
                      (const int64_t *)A.offset, (const uint32_t *)A.pack, (const void *)A.perm, 0,
                      make_decode(A), x, y, red);
}

template <int PF, int MINB>
cudaError_t launch_sell_pipe_dot(const Matrix &A, const float *x, float *y, const Red &red,
                                 cudaStream_t s) {
    const int sg = A.p.sigma;
    const int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    if (A.perm_bytes) {
        auto k = k_sell_pipe_dot<PF, MINB, true>;
        return launch_pdl(k, (unsigned)dot_grid(k), TPB, s, (int)A.n, sg, sh, (const int64_t *)A.offset,
                          (const float *)A.val, (const int32_t *)A.col, (const void *)A.perm,
                          A.perm_bytes, x, y, red);
    }
    auto k = k_sell_pipe_dot<PF, MINB, false>;
    return launch_pdl(k, (unsigned)dot_grid(k), TPB, s, (int)A.n, sg, sh, (const int64_t *)A.offset,
                      (const float *)A.val, (const int32_t *)A.col, (const void *)A.perm, 0, x, y,
                      red);
}

int spmv_dot_blocks(const Matrix &) { return reduce_blocks(); }

packsell_status spmv_dot_f32(const Matrix &A, const float *x, float *y, const Red &red,
                             cudaStream_t s) {
    const int g = device_sms() * 4;
    const void *perm = A.perm;
    const int pb = A.perm_bytes;
    if (A.p.format == PACKSELL_FMT_SELL_F32 && A.p.C == 32 && A.max_width <= 16) {
        // short rows: the pipelined form (the PackSELL inner solve's structure)
        const int pf = round_words(A.max_width);
        const cudaError_t e = pf == 8    ? launch_sell_pipe_dot<8, 4>(A, x, y, red, s)
                              : pf == 10 ? launch_sell_pipe_dot<10, 3>(A, x, y, red, s)
                              : pf == 12 ? launch_sell_pipe_dot<12, 3>(A, x, y, red, s)
                                         : launch_sell_pipe_dot<16, 2>(A, x, y, red, s);
        if (e != cudaSuccess) return cuda_fail(e, "spmv_dot_f32 (SELL, pipelined)");
    } else if (A.p.format == PACKSELL_FMT_SELL_F32) {
        const cudaError_t e = launch_pdl(k_spmv_sell<float, true, true>, (unsigned)g, TPB, s,
                                         (int)A.n, A.p.C, A.p.sigma, (const int64_t *)A.offset,
                                         (const float *)A.val, (const int32_t *)A.col, perm, pb,
                                         x, y, (const float *)nullptr, red);
        if (e != cudaSuccess) return cuda_fail(e, "spmv_dot_f32 (SELL)");
    } else if (A.p.C == 32 && A.max_width <= 16) {
        // every row fits one round: the pipelined kernel loads the next
        // row's words while the current row is gathered
        const bool h = A.p.format == PACKSELL_FMT_FP16;
        const int pf = round_words(A.max_width);
        cudaError_t e;
        if (pf == 8)
            e = h ? launch_pipe_dot<PACKSELL_FMT_FP16, 8, 5>(A, x, y, red, s)
                  : launch_pipe_dot<PACKSELL_FMT_E8MY, 8, 5>(A, x, y, red, s);
        else if (pf == 10)
            e = h ? launch_pipe_dot<PACKSELL_FMT_FP16, 10, 6>(A, x, y, red, s)
                  : launch_pipe_dot<PACKSELL_FMT_E8MY, 10, 6>(A, x, y, red, s);
        else if (pf == 12)
            e = h ? launch_pipe_dot<PACKSELL_FMT_FP16, 12, 4>(A, x, y, red, s)
                  : launch_pipe_dot<PACKSELL_FMT_E8MY, 12, 4>(A, x, y, red, s);
        else
            e = h ? launch_pipe_dot<PACKSELL_FMT_FP16, 16, 3>(A, x, y, red, s)
                  : launch_pipe_dot<PACKSELL_FMT_E8MY, 16, 3>(A, x, y, red, s);
        if (e != cudaSuccess) return cuda_fail(e, "spmv_dot_f32 (pipelined)");
    } else if (A.p.C == 32) {
        // row-prefetch kernel, rounds fitted to the widest slice
        const bool h = A.p.format == PACKSELL_FMT_FP16;
        const int pf = round_words(A.max_width);
        if (pf == 8) {
            if (h) launch_prefetch_dot<PACKSELL_FMT_FP16, 8, 6>(A, x, y, red, s);
            else launch_prefetch_dot<PACKSELL_FMT_E8MY, 8, 6>(A, x, y, red, s);
        } else if (pf == 10) {
            if (h) launch_prefetch_dot<PACKSELL_FMT_FP16, 10, 6>(A, x, y, red, s);
            else launch_prefetch_dot<PACKSELL_FMT_E8MY, 10, 6>(A, x, y, red, s);
        } else if (pf == 12) {
            if (h) launch_prefetch_dot<PACKSELL_FMT_FP16, 12, 5>(A, x, y, red, s);
            else launch_prefetch_dot<PACKSELL_FMT_E8MY, 12, 5>(A, x, y, red, s);
        } else {
            if (h) launch_prefetch_dot<PACKSELL_FMT_FP16, 16, 5>(A, x, y, red, s);
            else launch_prefetch_dot<PACKSELL_FMT_E8MY, 16, 5>(A, x, y, red, s);
        }
    } else {
        if (A.p.format == PACKSELL_FMT_FP16)
            k_spmv_packed_dot<PACKSELL_FMT_FP16><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y, red);
        else
            k_spmv_packed_dot<PACKSELL_FMT_E8MY><<<g, TPB, 0, s>>>(
                (int)A.n, A.p.C, A.p.sigma, A.p.k_left, A.offset, A.pack, perm, pb, make_decode(A), x, y, red);
    }
    PS_LAUNCH_CHECK("spmv_dot_f32");
    return PACKSELL_OK;
}

packsell_status spmv_dot_f64(const Matrix &A, const double *x, double *y, const double *b,
                             const Red &red, cudaStream_t s) {
    if (is_w64(A.p.format)) return spmv_dot_w64(A, x, y, b, red, (unsigned)(device_sms() * 4), s);
    const cudaError_t e = launch_pdl(k_spmv_sell_dot64, (unsigned)(device_sms() * 4),
                                     TPB, s, (int)A.n, A.p.C, A.p.sigma, (const int64_t *)A.offset,
                                     (const double *)A.val, (const int32_t *)A.col,
                                     (const void *)A.perm, A.perm_bytes, x, y, b, red);
    if (e != cudaSuccess) return cuda_fail(e, "spmv_dot_f64");
    PS_LAUNCH_CHECK("spmv_dot_f64");
    return PACKSELL_OK;
}

packsell_status pattern_outer_f64_impl(const Matrix &A, double alpha, const double *u,
                                       const double *v, double *out, cudaStream_t s) {
    if (A.p.format != PACKSELL_FMT_SELL_F64)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pattern_outer_f64: matrix is not SELL_F64");
    if (!A.rowptr)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_pattern_outer_f64: matrix was encoded without keep_rowptr");
    if (A.n == 0 || A.nnz == 0) return PACKSELL_OK;
    k_pattern_outer_sell<double><<<grid_for(A.n), TPB, 0, s>>>(
        (int)A.n, A.p.C, A.p.sigma, A.offset, A.col, A.perm, A.perm_bytes, A.rowptr, alpha, u, v, out);
    PS_LAUNCH_CHECK("packsell_pattern_outer_f64");
    return PACKSELL_OK;
}

namespace {
// 1 / a_ii of a square SELL_F64 matrix (1 where the diagonal is absent or 0)
__global__ void __launch_bounds__(TPB)
    k_inv_diag(int n, int C, int sigma, const int64_t *__restrict__ offset,
               const double *__restrict__ val, const int32_t *__restrict__ col,
               const void *__restrict__ perm, int perm_bytes, double *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = i / C, l = i - k * C;
    int64_t s = offset[k];
    int w = (int)((offset[k + 1] - s) / C);
    int io = orig_row(i, sigma, perm, perm_bytes);
    double d = 0.0;
    for (int j = 0; j < w; ++j) {
        const int64_t p = s + (int64_t)j * C + l;
        if (col[p] == io && val[p] != 0.0) d = val[p];
    }
    out[io] = d != 0.0 ? 1.0 / d : 1.0;
}
}  // namespace

packsell_status inv_diag_impl(const Matrix &A, double *out, cudaStream_t s) {
    if (!is_f64_op(A.p.format) || A.n != A.m)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_inv_diag: needs a square SELL_F64 or W64_E11MY matrix");
    if (is_w64(A.p.format)) return inv_diag_w64(A, out, s);
    if (A.n == 0) return PACKSELL_OK;
    k_inv_diag<<<grid_for(A.n), TPB, 0, s>>>((int)A.n, A.p.C, A.p.sigma, A.offset,
                                             (const double *)A.val, A.col, A.perm, A.perm_bytes, out);
    PS_LAUNCH_CHECK("packsell_inv_diag");
    return PACKSELL_OK;
}

}  // namespace packsell
