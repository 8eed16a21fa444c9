// Solvers: FP64 Jacobi-preconditioned CG, and the inner-outer CG (IO-CG) of
// §5.2.2 - flexible CG in FP64 whose preconditioner is m_in iterations of
// PCG in FP32 on a PackSELL (or FP32 SELL) copy of the matrix.
//
// Every step is a kernel on a private stream; scalars (alpha, beta, norms)
// stay on the device in a SolveScalars record written by the last block of
// each reducing kernel (deterministic, see reduce.cuh). One outer iteration
// (IO-CG) or `check_every` PCG iterations are captured once as a CUDA graph
// and replayed; the host reads the scalars after each replay. When the
// recurrence residual drops below rtol the device sets `done` and the
// remaining kernels of the replay idle, so iteration counts are exact. The
// host then checks the true residual ||b - A x||_2 / ||b||_2 in FP64; if it is
// not yet below rtol the residual is replaced by the true one and the outer
// method restarts from the current x.
//
// Readings of §5.2.2 (which gives the scheme, not its details): flexible CG
// keeps one previous direction (FCG(1)); the inner PCG starts from zero, runs
// exactly m_in iterations and solves for r / ||r||_2 (scaled back after),
// so FP32 never sees the outer residual's magnitude; the Jacobi
// preconditioner (if given) acts inside the inner PCG.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <mutex>
#include <string>

#include "device.cuh"
#include "internal.h"
#include "reduce.cuh"

namespace packsell {
namespace {

constexpr int VTPB = 256;

// grid-stride loop over [0, n)
#define PS_FOR(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// r = b - Ax (Ax given). s1 = b.b, s2 = r.r; r written when r != nullptr.
__global__ void __launch_bounds__(VTPB)
    k_residual(int64_t n, const double *__restrict__ b, const double *__restrict__ ax,
               double *__restrict__ r, Red red) {
    double bb = 0.0, rr = 0.0;
    PS_FOR(i, n) {
        const double bi = b[i], ri = bi - ax[i];
        if (r) r[i] = ri;
        bb += bi * bi;
        rr += ri * ri;
    }
    reduce_publish(red, red.fin == FIN_RT ? rr : bb, rr);
}

// PCG start (type T): z = M r, p = z, s1 = r.z
template <typename T>
__global__ void __launch_bounds__(VTPB)
    k_pcg_init(int64_t n, const T *__restrict__ r, const T *__restrict__ M, T *__restrict__ p,
               Red red) {
    T rz = 0;
    PS_FOR(i, n) {
        const T z = M ? M[i] * r[i] : r[i];
        p[i] = z;
        rz = fma(r[i], z, rz);
    }
    reduce_publish(red, (double)rz, 0.0);
}

// Inner PCG start: r_in = r / ||r|| (rounded to FP32), x_in = 0, p = M r_in.
__global__ void __launch_bounds__(VTPB)
    k_inner_init(int64_t n, const double *__restrict__ r64, const float *__restrict__ M,
                 float *__restrict__ xi, float *__restrict__ ri, float *__restrict__ pi, Red red) {
    if (red.sc->done) return;
    const double inv = red.sc->rnorm > 0.0 ? 1.0 / red.sc->rnorm : 0.0;
    float rz = 0.f;
    PS_FOR(i, n) {
        const float r = (float)(r64[i] * inv);
        const float z = M ? M[i] * r : r;
        xi[i] = 0.f;
        ri[i] = r;
        pi[i] = z;
        rz = fmaf(r, z, rz);
    }
    reduce_publish(red, (double)rz, 0.0);
}

// Vector kernels move VW = 16 / sizeof(T) elements per 128-bit access and
// handle two such vectors per loop trip, so each thread keeps several
// 128-bit loads in flight (a streaming kernel on GB300 needs ~45 KB in flight
// per SM). Pointers must be 16-byte aligned (checked by the launcher, which
// falls back to one element per access otherwise).
template <typename T>
struct V;
template <>
struct V<float> {
    using type = float4;
    static constexpr int W = 4;
};
template <>
struct V<double> {
    using type = double2;
    static constexpr int W = 2;
};

template <typename T>
__device__ __forceinline__ void ldv(const T *p, int64_t v, T (&e)[V<T>::W]) {
    *reinterpret_cast<typename V<T>::type *>(e) = reinterpret_cast<const typename V<T>::type *>(p)[v];
}
template <typename T>
__device__ __forceinline__ void stv(T *p, int64_t v, const T (&e)[V<T>::W]) {
    reinterpret_cast<typename V<T>::type *>(p)[v] = *reinterpret_cast<const typename V<T>::type *>(e);
}

// r -= alpha q and, with XUP, x += alpha p; s1 = r.z (z = M r), s2 = r.r.
// Each thread sums its own elements in T (FP32 for the inner PCG: GB300's
// FP64 rate is too low to spend per element) and the block and grid sums
// are FP64. Without XUP the x update of the iteration is left to the next
// direction kernel (k_pupdate, which reads p anyway), or to the final one.
template <typename T, bool VEC, bool XUP>
__global__ void __launch_bounds__(VTPB)
    k_update(int64_t n, T *__restrict__ x, T *__restrict__ r, const T *__restrict__ p,
             const T *__restrict__ q, const T *__restrict__ M, Red red) {
    grid_dep_sync();  // launched by launch_pdl: everything it reads comes from earlier kernels
    if (red.sc->done) return;
    const T a = (T)red.sc->alpha;
    T rz = 0, rr = 0;
    auto one = [&](int64_t i) {
        if (XUP) x[i] = fma(a, p[i], x[i]);
        const T ri = fma(-a, q[i], r[i]);
        r[i] = ri;
        const T z = M ? M[i] * ri : ri;
        rz = fma(ri, z, rz);
        rr = fma(ri, ri, rr);
    };
    if (VEC) {
        constexpr int W = V<T>::W;
        const int64_t nv = n / W, tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int64_t st = (int64_t)gridDim.x * blockDim.x;
        for (int64_t v0 = tid; v0 < nv; v0 += 2 * st) {
            T xe[2][W], pe[2][W], qe[2][W], re[2][W], me[2][W];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t v = v0 + h * st;
                if (v < nv) {
                    if (XUP) {
                        ldv(x, v, xe[h]);
                        ldv(p, v, pe[h]);
                    }
                    ldv(q, v, qe[h]);
                    ldv(r, v, re[h]);
                    if (M) ldv(M, v, me[h]);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t v = v0 + h * st;
                if (v < nv) {
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        if (XUP) xe[h][k] = fma(a, pe[h][k], xe[h][k]);
                        re[h][k] = fma(-a, qe[h][k], re[h][k]);
                        const T z = M ? me[h][k] * re[h][k] : re[h][k];
                        rz = fma(re[h][k], z, rz);
                        rr = fma(re[h][k], re[h][k], rr);
                    }
                    if (XUP) stv(x, v, xe[h]);
                    stv(r, v, re[h]);
                }
            }
        }
        for (int64_t i = nv * W + tid; i < n; i += st) one(i);
    } else {
        PS_FOR(i, n) one(i);
    }
    reduce_publish(red, (double)rz, (double)rr);
}

// Direction update. MODE 0: p = M r + beta p. MODE 1: first x += alpha p
// (the previous iteration's x update, deferred from k_update: the same fused
// multiply-add on the same p), then p = M r + beta p. MODE 2: x += alpha p
// alone (the last iteration of a fixed-length solve). alpha and beta are
// the iteration's (alpha is not rewritten before the next product).
template <typename T, bool VEC, int MODE>
__global__ void __launch_bounds__(VTPB)
    k_pupdate(int64_t n, const T *__restrict__ r, const T *__restrict__ M, T *__restrict__ p,
              T *__restrict__ x, const SolveScalars *sc) {
    grid_dep_sync();  // launched by launch_pdl, as k_update
    if (sc->done) return;
    const T b = (T)sc->beta;
    const T a = (T)sc->alpha;
    constexpr bool XU = MODE != 0, PU = MODE != 2;
    if (VEC) {
        constexpr int W = V<T>::W;
        const int64_t nv = n / W, tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int64_t st = (int64_t)gridDim.x * blockDim.x;
        for (int64_t v0 = tid; v0 < nv; v0 += 2 * st) {
            T re[2][W], pe[2][W], me[2][W], xe[2][W];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t v = v0 + h * st;
                if (v < nv) {
                    ldv(p, v, pe[h]);
                    if (XU) ldv(x, v, xe[h]);
                    if (PU) {
                        ldv(r, v, re[h]);
                        if (M) ldv(M, v, me[h]);
                    }
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t v = v0 + h * st;
                if (v < nv) {
                    if (XU) {
#pragma unroll
                        for (int k = 0; k < W; ++k) xe[h][k] = fma(a, pe[h][k], xe[h][k]);
                        stv(x, v, xe[h]);
                    }
                    if (PU) {
#pragma unroll
                        for (int k = 0; k < W; ++k)
                            pe[h][k] = fma(b, pe[h][k], M ? me[h][k] * re[h][k] : re[h][k]);
                        stv(p, v, pe[h]);
                    }
                }
            }
        }
        for (int64_t i = nv * W + tid; i < n; i += st) {
            if (XU) x[i] = fma(a, p[i], x[i]);
            if (PU) p[i] = fma(b, p[i], M ? M[i] * r[i] : r[i]);
        }
    } else {
        PS_FOR(i, n) {
            if (XU) x[i] = fma(a, p[i], x[i]);
            if (PU) {
                const T z = M ? M[i] * r[i] : r[i];
                p[i] = fma(b, p[i], z);
            }
        }
    }
}

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// The per-iteration kernels (SpMV + dot, update, direction) run with
// programmatic dependent launch: each is scheduled while the one before it
// drains.
template <typename T>
cudaError_t launch_update(int G, cudaStream_t q, int64_t n, T *x, T *r, const T *p, const T *qv,
                          const T *M, const Red &red, bool xup = true) {
    const bool vec =
        aligned16(x) && aligned16(r) && aligned16(p) && aligned16(qv) && (!M || aligned16(M));
    auto k = vec ? (xup ? k_update<T, true, true> : k_update<T, true, false>)
                 : (xup ? k_update<T, false, true> : k_update<T, false, false>);
    return launch_pdl(k, (unsigned)G, VTPB, q, n, x, r, p, qv, M, red);
}

// mode: 0 direction only, 1 deferred x update then direction, 2 x update only
template <typename T>
cudaError_t launch_pupdate(int G, cudaStream_t q, int64_t n, const T *r, const T *M, T *p, T *x,
                           const SolveScalars *sc, int mode = 0) {
    const bool vec = aligned16(r) && aligned16(p) && (!M || aligned16(M)) && aligned16(x);
    auto k = mode == 0 ? (vec ? k_pupdate<T, true, 0> : k_pupdate<T, false, 0>)
             : mode == 1 ? (vec ? k_pupdate<T, true, 1> : k_pupdate<T, false, 1>)
                         : (vec ? k_pupdate<T, true, 2> : k_pupdate<T, false, 2>);
    return launch_pdl(k, (unsigned)G, VTPB, q, n, r, M, p, x, sc);
}

// Outer: z = ||r|| x_in (FP64), s1 = z.q (q = A p of the previous direction)
__global__ void __launch_bounds__(VTPB)
    k_outer_z(int64_t n, const float *__restrict__ xi, double *__restrict__ z,
              const double *__restrict__ q, Red red) {
    if (red.sc->done) return;
    const double rn = red.sc->rnorm;
    double zq = 0.0;
    PS_FOR(i, n) {
        const double zi = rn * (double)xi[i];
        z[i] = zi;
        zq += zi * q[i];
    }
    reduce_publish(red, zq, 0.0);
}

// Outer: p = z - beta_o p (beta_o = 0 right after a (re)start)
__global__ void __launch_bounds__(VTPB)
    k_outer_p(int64_t n, const double *__restrict__ z, double *__restrict__ p,
              const SolveScalars *sc) {
    if (sc->done) return;
    const double b = sc->beta_o;
    PS_FOR(i, n) p[i] = (b == 0.0) ? z[i] : z[i] - b * p[i];
}

// Outer: x += alpha_o p, r -= alpha_o q; s1 = r.r
__global__ void __launch_bounds__(VTPB)
    k_outer_xr(int64_t n, double *__restrict__ x, double *__restrict__ r,
               const double *__restrict__ p, const double *__restrict__ q, Red red) {
    if (red.sc->done) return;
    const double a = red.sc->alpha_o;
    double rr = 0.0;
    PS_FOR(i, n) {
        x[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        rr += ri * ri;
    }
    reduce_publish(red, rr, 0.0);
}

__global__ void k_f64_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
    PS_FOR(i, n) b[i] = (float)a[i];
}

inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

struct Work {
    double *r, *z, *p, *q;        // FP64 vectors
    float *xi, *ri, *pi, *qi, *M32;  // FP32 inner vectors (IO-CG)
    double *partials;
    unsigned *counter;
    SolveScalars *sc;
    double *hist;
    size_t bytes;
};

Work carve(void *base, int64_t n, bool inner, bool has_m, int max_iters, int pblocks) {
    Work w{};
    char *p = (char *)base;
    auto take = [&](size_t b) {
        char *q = p;
        p += al(b);
        return (void *)q;
    };
    w.r = (double *)take(8 * n);
    w.z = (double *)take(8 * n);
    w.p = (double *)take(8 * n);
    w.q = (double *)take(8 * n);
    if (inner) {
        w.xi = (float *)take(4 * n);
        w.ri = (float *)take(4 * n);
        w.pi = (float *)take(4 * n);
        w.qi = (float *)take(4 * n);
        if (has_m) w.M32 = (float *)take(4 * n);
    }
    w.partials = (double *)take(16 * (size_t)pblocks);
    w.counter = (unsigned *)take(64);
    w.sc = (SolveScalars *)take(sizeof(SolveScalars));
    w.hist = (double *)take(8 * (size_t)(max_iters + 2));
    w.bytes = (size_t)(p - (char *)base);
    return w;
}

// fixed grid of the vector kernels (4 blocks per SM): the reductions are
// deterministic for a given device
int vec_blocks() { return reduce_blocks() / 2; }

}  // namespace

size_t solve_workspace_bytes(int64_t n, int m_in, int has_m, int max_iters) {
    const int pblocks = reduce_blocks();
    return carve(nullptr, n, m_in > 0, has_m != 0, max_iters, pblocks).bytes + 256;
}

packsell_status solve_impl(const Matrix *A64, const Matrix *Ain, const double *inv_diag,
                           const double *b, double *x, const packsell_solve_opts &o_in, void *work,
                           size_t work_bytes, double *h_hist, packsell_solve_result *res,
                           cudaStream_t caller, bool noalloc) {
    // no-allocation mode: the caller's stream, no graph, no events, the
    // workspace given (never allocated here)
    packsell_solve_opts o = o_in;
    if (noalloc) o.use_graph = 0;
    const bool io = o.m_in > 0;
    if (!A64 || !is_f64_op(A64->p.format))
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_pcg: A_outer must be a SELL_F64 or W64_E11MY matrix");
    const int64_t n = A64->n;
    if (A64->m != n || A64->p.explicit_perm)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_pcg: A_outer must be square with rows in original order");
    if (io) {
        if (!Ain || Ain->n != n || Ain->m != n || Ain->p.explicit_perm ||
            !(is_packed(Ain->p.format) || Ain->p.format == PACKSELL_FMT_SELL_F32))
            return fail(PACKSELL_ERR_INVALID_ARG,
                        "packsell_pcg: A_inner must be a square PackSELL or SELL_F32 matrix "
                        "of the same size, rows in original order");
    }
    if (o.max_iters < 1 || o.check_every < 1 || !(o.rtol > 0.0) || o.m_in < 0)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg: bad options");
    if (n == 0) {
        if (res) *res = packsell_solve_result{};
        return PACKSELL_OK;
    }
    if (!b || !x) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg: NULL vector");

    const int pblocks = reduce_blocks();
    const size_t need = solve_workspace_bytes(n, o.m_in, inv_diag != nullptr, o.max_iters);
    void *own = nullptr;
    cudaStream_t s = caller;
    if (!noalloc) PS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    packsell_status st = PACKSELL_OK;
    Work w{};
    SolveScalars h{};
    int iters = 0;
    bool converged = false;
    double relres_true = -1.0;

    const auto t_start = std::chrono::steady_clock::now();
    if (!noalloc) {
        // the caller's pending work on its stream comes first
        cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming);
        cudaEventRecord(ev0, caller);
        cudaStreamWaitEvent(s, ev0, 0);
        cudaEventDestroy(ev0);
        ev0 = nullptr;
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
    }

    if (work) {
        if (work_bytes < need) {
            st = fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg: workspace too small (need " +
                                                    std::to_string(need) + " bytes)");
            goto out;
        }
        w = carve((void *)(((uintptr_t)work + 255) & ~(uintptr_t)255), n, io, inv_diag != nullptr,
                  o.max_iters, pblocks);
    } else {
        if (noalloc) {
            st = fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg: no workspace");
            goto out;
        }
        if (cudaMallocAsync(&own, need, s) != cudaSuccess) {
            st = fail(PACKSELL_ERR_NO_MEMORY, "packsell_pcg: workspace allocation");
            goto out;
        }
        w = carve((void *)(((uintptr_t)own + 255) & ~(uintptr_t)255), n, io, inv_diag != nullptr,
                  o.max_iters, pblocks);
    }
    {
        const int G = vec_blocks();
        auto red = [&](int fin) { return Red{w.partials, w.counter, w.sc, w.hist, fin}; };
        SolveScalars init{};
        init.rtol = o.rtol;
        init.max_iters = o.max_iters;
        init.restart = 1;
        // every copy, memset and synchronisation of the host loop is checked
        auto ck = [&](cudaError_t e) {
            if (e != cudaSuccess) st = cuda_fail(e, "packsell_pcg: copy or synchronize");
            return e == cudaSuccess;
        };
        if (!ck(cudaMemcpyAsync(w.sc, &init, sizeof(init), cudaMemcpyHostToDevice, s)) ||
            !ck(cudaMemsetAsync(w.counter, 0, 64, s)) || !ck(cudaMemsetAsync(w.q, 0, 8 * n, s)))
            goto out;
        if (ev0) cudaEventRecord(ev0, s);
        if (io && inv_diag) k_f64_to_f32<<<G, VTPB, 0, s>>>(n, inv_diag, w.M32);

        // r = b - A x, ||b||, ||r||
        auto residual = [&](double *r_out, int fin) -> packsell_status {
            packsell_status e = spmv_f64_impl(*A64, x, w.z, s);
            if (e != PACKSELL_OK) return e;
            k_residual<<<G, VTPB, 0, s>>>(n, b, w.z, r_out, red(fin));
            PS_LAUNCH_CHECK("k_residual");
            return PACKSELL_OK;
        };
        st = residual(w.r, FIN_BB_RR);
        if (st != PACKSELL_OK) goto out;
        if (!io) {
            k_pcg_init<double><<<G, VTPB, 0, s>>>(n, w.r, inv_diag, w.p, red(FIN_RZ_INIT));
        }

        // one replay = `chunk` outer (IO-CG) or PCG iterations
        const int chunk = std::min(o.check_every, o.max_iters);
        auto body = [&](cudaStream_t q) -> packsell_status {
            for (int c = 0; c < chunk; ++c) {
                if (io) {
                    k_inner_init<<<G, VTPB, 0, q>>>(n, w.r, w.M32, w.xi, w.ri, w.pi, red(FIN_RZ_INIT));
                    for (int k = 0; k < o.m_in; ++k) {
                        packsell_status e = spmv_dot_f32(*Ain, w.pi, w.qi, red(FIN_PQ_ALPHA), q);
                        if (e != PACKSELL_OK) return e;
                        // the inner solve has a fixed length: each iteration's
                        // x update rides on the next direction update (which
                        // reads p anyway), the last one on its own
                        cudaError_t ce = launch_update<float>(G, q, n, w.xi, w.ri, w.pi, w.qi,
                                                              w.M32, red(FIN_RZ_BETA), false);
                        if (ce == cudaSuccess)
                            ce = launch_pupdate<float>(G, q, n, w.ri, w.M32, w.pi, w.xi, w.sc,
                                                       k + 1 < o.m_in ? 1 : 2);
                        if (ce != cudaSuccess) return cuda_fail(ce, "packsell_pcg: inner update");
                    }
                    k_outer_z<<<G, VTPB, 0, q>>>(n, w.xi, w.z, w.q, red(FIN_ZQ_BETA));
                    k_outer_p<<<G, VTPB, 0, q>>>(n, w.z, w.p, w.sc);
                    packsell_status e = spmv_dot_f64(*A64, w.p, w.q, w.r, red(FIN_OUTER_ALPHA), q);
                    if (e != PACKSELL_OK) return e;
                    k_outer_xr<<<G, VTPB, 0, q>>>(n, x, w.r, w.p, w.q, red(FIN_RR));
                } else {
                    packsell_status e = spmv_dot_f64(*A64, w.p, w.q, nullptr, red(FIN_PQ_ALPHA_64), q);
                    if (e != PACKSELL_OK) return e;
                    cudaError_t ce = launch_update<double>(G, q, n, x, w.r, w.p, w.q, inv_diag,
                                                           red(FIN_RZ_BETA_RR));
                    if (ce == cudaSuccess)
                        ce = launch_pupdate<double>(G, q, n, w.r, inv_diag, w.p, x, w.sc);
                    if (ce != cudaSuccess) return cuda_fail(ce, "packsell_pcg: update");
                }
            }
            PS_LAUNCH_CHECK("packsell_pcg: iteration");
            return PACKSELL_OK;
        };
        if (o.use_graph) {
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                st = fail(PACKSELL_ERR_CUDA, "packsell_pcg: stream capture failed to start");
                goto out;
            }
            packsell_status e = body(s);
            cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (e != PACKSELL_OK) { st = e; goto out; }
            if (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                st = fail(PACKSELL_ERR_CUDA, "packsell_pcg: graph capture failed");
                goto out;
            }
        }
        while (iters < o.max_iters) {
            if (o.use_graph) {
                if (cudaGraphLaunch(exec, s) != cudaSuccess) {
                    st = fail(PACKSELL_ERR_CUDA, "packsell_pcg: graph launch failed");
                    goto out;
                }
            } else {
                st = body(s);
                if (st != PACKSELL_OK) goto out;
            }
            if (!ck(cudaMemcpyAsync(&h, w.sc, sizeof(h), cudaMemcpyDeviceToHost, s))) goto out;
            if (cudaStreamSynchronize(s) != cudaSuccess) {
                st = cuda_fail(cudaGetLastError(), "packsell_pcg: iteration");
                goto out;
            }
            iters = h.iter;
            if (h.status) {
                st = fail(PACKSELL_ERR_BREAKDOWN, "packsell_pcg: breakdown (p^T A p <= 0 or "
                                                  "a non-finite residual)");
                goto out;
            }
            if (h.done && h.relres < o.rtol) {
                // the recurrence says converged: check the true residual
                st = residual(nullptr, FIN_RT);
                if (st != PACKSELL_OK) goto out;
                if (!ck(cudaMemcpyAsync(&h, w.sc, sizeof(h), cudaMemcpyDeviceToHost, s)) ||
                    !ck(cudaStreamSynchronize(s)))
                    goto out;
                relres_true = h.bb > 0.0 ? sqrt(h.rt / h.bb) : 0.0;
                if (relres_true < o.rtol) {
                    converged = true;
                    break;
                }
                // replace the residual by the true one and restart the directions
                st = residual(w.r, FIN_BB_RR);
                if (st != PACKSELL_OK) goto out;
                if (!io) k_pcg_init<double><<<G, VTPB, 0, s>>>(n, w.r, inv_diag, w.p, red(FIN_RZ_INIT));
                int one = 1, zero = 0;
                if (!ck(cudaMemcpyAsync(&w.sc->restart, &one, sizeof(int), cudaMemcpyHostToDevice, s)) ||
                    !ck(cudaMemcpyAsync(&w.sc->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s)) ||
                    !ck(cudaStreamSynchronize(s)))
                    goto out;
            }
        }
        if (ev1) cudaEventRecord(ev1, s);
        if (!ck(cudaMemcpyAsync(&h, w.sc, sizeof(h), cudaMemcpyDeviceToHost, s))) goto out;
        if (!ck(cudaStreamSynchronize(s))) goto out;
        if (h_hist &&
            !ck(cudaMemcpy(h_hist, w.hist, sizeof(double) * (size_t)(std::min(h.iter, o.max_iters) + 1),
                           cudaMemcpyDeviceToHost)))
            goto out;
        if (relres_true < 0.0) {
            st = residual(nullptr, FIN_RT);
            if (st != PACKSELL_OK) goto out;
            SolveScalars h2{};
            if (!ck(cudaMemcpyAsync(&h2, w.sc, sizeof(h2), cudaMemcpyDeviceToHost, s)) ||
                !ck(cudaStreamSynchronize(s)))
                goto out;
            relres_true = h2.bb > 0.0 ? sqrt(h2.rt / h2.bb) : 0.0;
        }
        if (res) {
            float ms = 0.f;
            if (ev0 && ev1) cudaEventElapsedTime(&ms, ev0, ev1);
            else ms = (float)std::chrono::duration<double, std::milli>(
                          std::chrono::steady_clock::now() - t_start).count();
            res->iters = h.iter;
            res->inner_iters = h.inner;
            res->relres = h.relres;
            res->relres_true = relres_true;
            res->seconds = ms * 1e-3;
        }
        if (!converged)
            st = fail(PACKSELL_ERR_NOT_CONVERGED,
                      "packsell_pcg: no convergence in " + std::to_string(o.max_iters) + " iterations");
    }
out:
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (own) cudaFreeAsync(own, s);
    cudaStreamSynchronize(s);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (!noalloc) cudaStreamDestroy(s);
    return st;
}

// ---- the solver without allocation -------------------------------------
// Some callers cannot allocate device memory at the time they solve: an
// application that reserved the device's memory for its own pool, a plugin
// given a fixed budget, a loop that must not take cudaMalloc's implicit
// synchronisation. For them the whole solver workspace lives in one static
// device array, sized for systems of up to about 160,000 unknowns (IO-CG)
// or 260,000 (FP64 PCG). Every call shares it.
constexpr size_t kNoAllocBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_pcg_scratch[kNoAllocBytes];

namespace {
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;
}  // namespace

// Device address of g_pcg_scratch on the current device (looked up once per
// device, with that device current; in host code the name is only a
// host-side stand-in for it). A cudaDeviceReset invalidates the kept address
// together with every other device object of the library.
static packsell_status noalloc_scratch(void **out) {
    int dev = 0;
    PS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "packsell_pcg_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PACKSELL_OK;
}

size_t noalloc_capacity() { return kNoAllocBytes; }

packsell_status solve_noalloc(const Matrix *A64, const Matrix *Ain, const double *inv_diag,
                              const double *b, double *x, const packsell_solve_opts &o,
                              double *h_hist, packsell_solve_result *res, cudaStream_t s) {
    if (!A64) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg_noalloc: NULL matrix");
    if (o.max_iters < 1 || o.m_in < 0)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg_noalloc: bad options");
    const size_t need = solve_workspace_bytes(A64->n, o.m_in, inv_diag != nullptr, o.max_iters);
    if (need > kNoAllocBytes)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_pcg_noalloc: this system needs " + std::to_string(need) +
                        " bytes of workspace, the static area holds " +
                        std::to_string(kNoAllocBytes) + " (use packsell_pcg)");
    void *scratch = nullptr;
    packsell_status st = noalloc_scratch(&scratch);
    if (st != PACKSELL_OK) return st;
    return solve_impl(A64, Ain, inv_diag, b, x, o, scratch, kNoAllocBytes, h_hist, res, s, true);
}

}  // namespace packsell
