// F3R: the nested Krylov solver of §5.2.1 (FGMRES, FGMRES, FGMRES and an
// innermost preconditioned Richardson), with the FP16 SpMV of the two inner
// layers as PackSELL FP16 or FP16 SELL, or every layer in FP64.
//
// Layer 1 is restarted flexible GMRES in double precision on the FP64
// operator; its preconditioner is layer 2, m2 iterations of flexible GMRES
// from zero on the FP32 (or FP64) operator; layer 2's preconditioner is layer
// 3, m3 iterations of flexible GMRES from zero on the FP16 operator; layer 3's
// preconditioner is layer 4, m4 steps of Richardson z <- z + omega (r - A z)
// from z = 0 on the FP16 operator (Jacobi preconditioning is the identity on
// the symmetrically scaled matrices of §5.2). Every layer builds its Krylov
// basis with classical Gram-Schmidt: the dot products of a step are one
// deterministic reduction (block partials summed in block order, in double
// precision), the update of the new vector is done in the layer's arithmetic
// (double for the FP64 layers; FP32 for the FP32 layers of FP16-F3R, whose
// per-thread partial sums are FP32 as well, since on GB300 the FP64 pipe
// and not memory would bound those kernels), and the Hessenberg matrix, its
// Givens rotations and the small least-squares solve stay on the device in
// double precision.
// Layers 2-4 run a fixed number of steps (no convergence test); layer 1
// reads its residual estimate |g_{j+1}| after every step and confirms
// convergence on the true residual b - A x in FP64.
//
// The two inner SpMVs of the FP16 layers are the only kernels that differ
// between PackSELL-F3R and FP16-SELL-F3R, and both sum every row as the
// same chain of fused multiply-adds over the same FP16 values: the two
// solvers produce the same iterates, bit for bit (the paper's observation
// that they converge identically).
#include <cuda_fp16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace packsell {

int device_sms();

namespace {

constexpr int FT = 256;  // threads per block of the vector kernels

inline int fgrid(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)device_sms() * 4, (n + FT - 1) / FT));
}

// block-wide sum of a double (fixed tree), result in thread 0
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    __syncthreads();
    return t;
}

// Arnoldi state of one layer (double, device): H column-major (m+1) x m,
// Givens cosines and sines, right-hand side g (m+1), solution y (m), and
// scal = {beta = ||rhs||, 1 / (last norm), |g_{j+1}|}
struct Hess {
    double *H, *cs, *sn, *g, *y, *scal;
    int m;
};

// The reducing kernels below end with the step that needs the whole
// reduction: each block writes its partial, and the block that arrives last
// (an atomic counter, back at 0 when it is done) adds the partials in block
// order and finishes, so no one-block kernel follows. Called by every thread
// after thread 0 has written the block's partial; true in the last block
// once every partial is visible.
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x * gridDim.y - 1u;
        if (last) *counter = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// sum of the G partials at p, in block order (the whole block; thread 0 has it)
__device__ __forceinline__ double partial_sum(const double *p, int G, double *sh) {
    double s = 0.0;
    for (int b = threadIdx.x; b < G; b += FT) s += ((const volatile double *)p)[b];
    return block_sum(s, sh);
}

// beta = ||rhs|| from the partials; g = beta e_1; scal[1] = 1 / beta
__device__ __forceinline__ void begin_finish(int G, const double *part, Hess h, double *sh) {
    const double s = partial_sum(part, G, sh);
    if (threadIdx.x == 0) {
        const double beta = sqrt(s);
        h.scal[0] = beta;
        h.scal[1] = beta > 0.0 ? 1.0 / beta : 0.0;
        h.scal[2] = beta;
        for (int i = 0; i <= h.m; ++i) h.g[i] = 0.0;
        h.g[0] = beta;
    }
}

// partial sums of v.v per block; the last block sets up the layer (begin_finish)
template <typename T>
__global__ void __launch_bounds__(FT) k_norm2_begin(int64_t n, const T *__restrict__ v,
                                                    double *__restrict__ part, unsigned *counter,
                                                    Hess h) {
    __shared__ double sh[FT / 32];
    double s = 0.0;
    if constexpr (std::is_same<T, float>::value) {  // an FP32 layer: FP32 thread partials
        float sf = 0.f;
        for (int64_t i = blockIdx.x * (int64_t)FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
            sf = fmaf(v[i], v[i], sf);
        s = (double)sf;
    } else {
        for (int64_t i = blockIdx.x * (int64_t)FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT) {
            const double a = (double)v[i];
            s = fma(a, a, s);
        }
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (last_block(counter)) begin_finish(gridDim.x, part, h, sh);
}

// partial sums of w.v_i for the cnt basis vectors v_i (blockIdx.y = i); the
// last block sets h[i][j] = the sum of the partials of w.v_i, in block order
template <typename T>
__global__ void __launch_bounds__(FT) k_mdot(int64_t n, const T *__restrict__ V,
                                             const T *__restrict__ w, double *__restrict__ part,
                                             unsigned *counter, Hess h, int j) {
    __shared__ double sh[FT / 32];
    const T *__restrict__ v = V + (int64_t)blockIdx.y * n;
    double s = 0.0;
    if constexpr (std::is_same<T, float>::value) {
        float sf = 0.f;
        for (int64_t i = blockIdx.x * (int64_t)FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
            sf = fmaf(w[i], v[i], sf);
        s = (double)sf;
    } else {
        for (int64_t i = blockIdx.x * (int64_t)FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
            s = fma((double)w[i], (double)v[i], s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
    if (!last_block(counter)) return;
    const int G = gridDim.x;
    for (int i = 0; i < (int)gridDim.y; ++i) {
        const double t = partial_sum(part + (int64_t)i * G, G, sh);
        if (threadIdx.x == 0) h.H[i + (int64_t)j * (h.m + 1)] = t;
    }
}

// out = (TO)(in * scal[k])
template <typename TI, typename TO>
__global__ void __launch_bounds__(FT) k_scale(int64_t n, const TI *__restrict__ in, TO *__restrict__ out,
                                              const double *__restrict__ scal) {
    const double s = *scal;
    if constexpr (std::is_same<TI, float>::value && std::is_same<TO, float>::value) {
        const float sf = (float)s;
        for (int64_t i = blockIdx.x * (int64_t)FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
            out[i] = in[i] * sf;
    } else {
        for (int64_t i = blockIdx.x * (int64_t)FT + threadIdx.x; i < n; i += (int64_t)gridDim.x * FT)
            out[i] = (TO)((double)in[i] * s);
    }
}

// h[j+1][j] = ||w||; the earlier Givens rotations on column j, a new one
// that zeroes h[j+1][j]; g updated; scal[1] = 1 / h[j+1][j], scal[2] = |g[j+1]|
__device__ __forceinline__ void arnoldi_finish(int G, const double *part, Hess h, int j, double *sh) {
    const double s = partial_sum(part, G, sh);
    if (threadIdx.x != 0) return;
    const int ld = h.m + 1;
    double *col = h.H + (int64_t)j * ld;
    const double hn = sqrt(s);
    col[j + 1] = hn;
    for (int k = 0; k < j; ++k) {
        const double a = col[k], b = col[k + 1];
        col[k] = h.cs[k] * a + h.sn[k] * b;
        col[k + 1] = -h.sn[k] * a + h.cs[k] * b;
    }
    const double a = col[j], b = col[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, sn = r > 0.0 ? b / r : 0.0;
    h.cs[j] = c;
    h.sn[j] = sn;
    col[j] = r;
    col[j + 1] = 0.0;
    h.g[j + 1] = -sn * h.g[j];
    h.g[j] = c * h.g[j];
    h.scal[1] = hn > 0.0 ? 1.0 / hn : 0.0;
    h.scal[2] = fabs(h.g[j + 1]);
}

// w = w - sum_i h[i][j] v_i (in double, rounded once to T); partials of w.w;
// the last block closes the Arnoldi step (arnoldi_finish)
template <typename T>
__global__ void __launch_bounds__(FT) k_orth(int64_t n, const T *__restrict__ V, int cnt, Hess h, int j,
                                             T *__restrict__ w, double *__restrict__ part,
                                             unsigned *counter) {
    __shared__ double sh[FT / 32];
    __shared__ double hc[64];
    __shared__ float hf[64];
    for (int i = threadIdx.x; i < cnt; i += FT) {
        hc[i] = h.H[i + (int64_t)j * (h.m + 1)];
        hf[i] = (float)hc[i];
    }
    __syncthreads();
    double s = 0.0;
    if constexpr (std::is_same<T, float>::value) {
        float sf = 0.f;
        for (int64_t e = blockIdx.x * (int64_t)FT + threadIdx.x; e < n; e += (int64_t)gridDim.x * FT) {
            float a = w[e];
            for (int i = 0; i < cnt; ++i) a = fmaf(-hf[i], V[(int64_t)i * n + e], a);
            w[e] = a;
            sf = fmaf(a, a, sf);
        }
        s = (double)sf;
    } else {
        for (int64_t e = blockIdx.x * (int64_t)FT + threadIdx.x; e < n; e += (int64_t)gridDim.x * FT) {
            double a = (double)w[e];
            for (int i = 0; i < cnt; ++i) a -= hc[i] * (double)V[(int64_t)i * n + e];
            const T r = (T)a;
            w[e] = r;
            s = fma((double)r, (double)r, s);
        }
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (last_block(counter)) arnoldi_finish(gridDim.x, part, h, j, sh);
}

// y = R^-1 g over the first k columns (R the rotated Hessenberg matrix)
__global__ void k_backsolve(Hess h, int k) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int ld = h.m + 1;
    for (int i = k - 1; i >= 0; --i) {
        double t = h.g[i];
        for (int c = i + 1; c < k; ++c) t -= h.H[i + (int64_t)c * ld] * h.y[c];
        const double d = h.H[i + (int64_t)i * ld];
        h.y[i] = d != 0.0 ? t / d : 0.0;
    }
}

// out = (ACC ? out : 0) + sum_{j<k} y_j z_j (in double, rounded once)
template <typename TZ, typename TO, bool ACC>
__global__ void __launch_bounds__(FT) k_combine(int64_t n, const TZ *__restrict__ Z, int k,
                                                const double *__restrict__ y, TO *__restrict__ out) {
    __shared__ double ys[64];
    __shared__ float yf[64];
    for (int i = threadIdx.x; i < k; i += FT) {
        ys[i] = y[i];
        yf[i] = (float)y[i];
    }
    __syncthreads();
    if constexpr (std::is_same<TZ, float>::value && std::is_same<TO, float>::value) {
        for (int64_t e = blockIdx.x * (int64_t)FT + threadIdx.x; e < n; e += (int64_t)gridDim.x * FT) {
            float a = ACC ? out[e] : 0.f;
            for (int j = 0; j < k; ++j) a = fmaf(yf[j], Z[(int64_t)j * n + e], a);
            out[e] = a;
        }
    } else {
        for (int64_t e = blockIdx.x * (int64_t)FT + threadIdx.x; e < n; e += (int64_t)gridDim.x * FT) {
            double a = ACC ? (double)out[e] : 0.0;
            for (int j = 0; j < k; ++j) a += ys[j] * (double)Z[(int64_t)j * n + e];
            out[e] = (TO)a;
        }
    }
}

// Richardson: z = omega r (first step) or z = z + omega (r - t)
template <typename T>
__global__ void __launch_bounds__(FT) k_rich(int64_t n, T *__restrict__ z, const T *__restrict__ r,
                                             const T *__restrict__ t, float omega, int first) {
    for (int64_t e = blockIdx.x * (int64_t)FT + threadIdx.x; e < n; e += (int64_t)gridDim.x * FT)
        z[e] = first ? (T)(omega * r[e]) : (T)(z[e] + omega * (r[e] - t[e]));
}

// r = b - A x (x, r, b double) and the partials of r.r; the last block sets
// up layer 1 from r (begin_finish: beta = ||r||, v_0 scale)
__global__ void __launch_bounds__(FT) k_resid(int64_t n, const double *__restrict__ b,
                                              const double *__restrict__ ax, double *__restrict__ r,
                                              double *__restrict__ part, unsigned *counter, Hess h) {
    __shared__ double sh[FT / 32];
    double s = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)FT + threadIdx.x; e < n; e += (int64_t)gridDim.x * FT) {
        const double v = b[e] - ax[e];
        r[e] = v;
        s = fma(v, v, s);
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
    if (last_block(counter)) begin_finish(gridDim.x, part, h, sh);
}

// one product of a layer: double vectors on the FP64 formats (SELL_F64,
// 64-bit words), float vectors on the others
packsell_status layer_spmv(const Matrix &A, const double *x, double *y, cudaStream_t s) {
    return spmv_f64_impl(A, x, y, s);
}
packsell_status layer_spmv(const Matrix &A, const float *x, float *y, cudaStream_t s) {
    return spmv_impl(A, x, y, s);
}

// device memory of the solve, in one allocation
struct Pool {
    char *base = nullptr, *cur = nullptr;
    size_t left = 0;
    template <typename T>
    T *take(size_t count) {
        size_t b = (count * sizeof(T) + 255) & ~(size_t)255;
        if (b > left) return nullptr;
        T *p = reinterpret_cast<T *>(cur);
        cur += b;
        left -= b;
        return p;
    }
};

template <typename T>
struct Layer {
    int m = 0;
    T *V = nullptr;  // (m + 1) basis vectors
    T *Z = nullptr;  // m preconditioned vectors
    Hess h{};
};

template <typename T>
bool make_layer(Pool &P, Layer<T> &L, int m, int64_t n) {
    L.m = m;
    L.V = P.take<T>((size_t)(m + 1) * n);
    L.Z = P.take<T>((size_t)m * n);
    L.h.m = m;
    L.h.H = P.take<double>((size_t)(m + 1) * m);
    L.h.cs = P.take<double>(m);
    L.h.sn = P.take<double>(m);
    L.h.g = P.take<double>(m + 1);
    L.h.y = P.take<double>(m);
    L.h.scal = P.take<double>(4);
    return L.V && L.Z && L.h.H && L.h.cs && L.h.sn && L.h.g && L.h.y && L.h.scal;
}

template <typename TI>
struct F3R {
    const Matrix *A1, *A2, *A3;
    int64_t n;
    int G;
    double *part;  // G * 64 partials
    unsigned *counter;  // blocks of the running reduction that have finished (0 between launches)
    Layer<double> L1;
    Layer<TI> L2, L3;
    TI *rt = nullptr;  // the product of a Richardson step (the iterate is layer 3's z_j)
    int m4;
    float omega;
    cudaStream_t s;

    // layer 4: z = Richardson(r), m4 steps from z = 0
    packsell_status richardson(const TI *r, TI *z) {
        k_rich<TI><<<G, FT, 0, s>>>(n, z, r, (const TI *)nullptr, omega, 1);
        for (int k = 1; k < m4; ++k) {
            packsell_status st = layer_spmv(*A3, z, rt, s);
            if (st != PACKSELL_OK) return st;
            k_rich<TI><<<G, FT, 0, s>>>(n, z, r, rt, omega, 0);
        }
        PS_LAUNCH_CHECK("f3r: Richardson");
        return PACKSELL_OK;
    }

    // one Arnoldi step j of layer L on operator A: w = A z_j, orthogonalise
    // against v_0..v_j, normalise into v_{j+1}
    template <typename T>
    packsell_status arnoldi(Layer<T> &L, const Matrix &A, int j) {
        T *w = L.V + (int64_t)(j + 1) * n;
        packsell_status st = layer_spmv(A, L.Z + (int64_t)j * n, w, s);
        if (st != PACKSELL_OK) return st;
        const int cnt = j + 1;
        k_mdot<T><<<dim3(G, cnt), FT, 0, s>>>(n, L.V, w, part, counter, L.h, j);
        k_orth<T><<<G, FT, 0, s>>>(n, L.V, cnt, L.h, j, w, part, counter);
        k_scale<T, T><<<G, FT, 0, s>>>(n, w, w, L.h.scal + 1);
        PS_LAUNCH_CHECK("f3r: Arnoldi step");
        return PACKSELL_OK;
    }

    // v_0 = rhs / ||rhs|| (converted to T), g = ||rhs|| e_1
    template <typename T, typename TR>
    void begin(Layer<T> &L, const TR *rhs) {
        k_norm2_begin<TR><<<G, FT, 0, s>>>(n, rhs, part, counter, L.h);
        k_scale<TR, T><<<G, FT, 0, s>>>(n, rhs, L.V, L.h.scal + 1);
    }

    // layer 3: m3 steps of FGMRES from zero on A3, preconditioned by layer 4
    packsell_status layer3(const TI *rhs, TI *out) {
        begin(L3, rhs);
        for (int j = 0; j < L3.m; ++j) {
            packsell_status st = richardson(L3.V + (int64_t)j * n, L3.Z + (int64_t)j * n);
            if (st == PACKSELL_OK) st = arnoldi(L3, *A3, j);
            if (st != PACKSELL_OK) return st;
        }
        k_backsolve<<<1, 32, 0, s>>>(L3.h, L3.m);
        k_combine<TI, TI, false><<<G, FT, 0, s>>>(n, L3.Z, L3.m, L3.h.y, out);
        PS_LAUNCH_CHECK("f3r: layer 3");
        return PACKSELL_OK;
    }

    // layer 2: m2 steps of FGMRES from zero on A2, preconditioned by layer 3
    packsell_status layer2(const double *rhs, double *out) {
        begin(L2, rhs);
        for (int j = 0; j < L2.m; ++j) {
            packsell_status st = layer3(L2.V + (int64_t)j * n, L2.Z + (int64_t)j * n);
            if (st == PACKSELL_OK) st = arnoldi(L2, *A2, j);
            if (st != PACKSELL_OK) return st;
        }
        k_backsolve<<<1, 32, 0, s>>>(L2.h, L2.m);
        k_combine<TI, double, false><<<G, FT, 0, s>>>(n, L2.Z, L2.m, L2.h.y, out);
        PS_LAUNCH_CHECK("f3r: layer 2");
        return PACKSELL_OK;
    }
};

template <typename TI>
packsell_status run_f3r(const Matrix &A1, const Matrix &A2, const Matrix &A3, const double *b,
                        double *x, const packsell_f3r_opts &o, packsell_solve_result *res,
                        cudaStream_t caller) {
    const int64_t n = A1.n;
    cudaStream_t s = nullptr;
    PS_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *mem = nullptr;
    packsell_status st = PACKSELL_OK;
    int iters = 0, steps = 0;
    double relres = 1.0, relres_true = -1.0;
    bool converged = false;
    const int G = fgrid(n);
    F3R<TI> F{};
    Pool P;
    {
        cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming);
        cudaEventRecord(ev0, caller);
        cudaStreamWaitEvent(s, ev0, 0);  // the caller's pending work first
        cudaEventDestroy(ev0);
        ev0 = nullptr;
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
    }
    const size_t need =
        sizeof(double) * ((size_t)(2 * o.m1 + 1) * n + 5 * (size_t)n + 64 * (size_t)G +
                          (size_t)(o.m1 + 1) * o.m1 + 8 * (size_t)o.m1 + 16) +
        sizeof(TI) * ((size_t)(2 * o.m2 + 1) * n + (size_t)(2 * o.m3 + 1) * n + 2 * (size_t)n) +
        sizeof(double) * ((size_t)(o.m2 + 1) * o.m2 + (size_t)(o.m3 + 1) * o.m3 + 8 * (size_t)(o.m2 + o.m3) + 32) +
        256 * 40;
    double *r = nullptr, *ax = nullptr, *zt = nullptr, *prhs = nullptr, *pout = nullptr;
    double nb = 0.0;
    if (cudaMallocAsync(&mem, need, s) != cudaSuccess) {
        st = fail(PACKSELL_ERR_NO_MEMORY, "packsell_f3r: workspace allocation");
        goto out;
    }
    P.base = P.cur = (char *)mem;
    P.left = need;
    F.A1 = &A1;
    F.A2 = &A2;
    F.A3 = &A3;
    F.n = n;
    F.G = G;
    F.m4 = o.m4;
    F.omega = (float)o.omega;
    F.s = s;
    F.part = P.take<double>(64 * (size_t)G);
    F.counter = P.take<unsigned>(1);
    r = P.take<double>(n);
    ax = P.take<double>(n);
    zt = P.take<double>(n);
    prhs = P.take<double>(n);
    pout = P.take<double>(n);
    F.rt = P.take<TI>(n);
    if (!F.part || !F.counter || !r || !ax || !zt || !prhs || !pout || !F.rt || !make_layer(P, F.L1, o.m1, n) ||
        !make_layer(P, F.L2, o.m2, n) || !make_layer(P, F.L3, o.m3, n)) {
        st = fail(PACKSELL_ERR_NO_MEMORY, "packsell_f3r: workspace carving");
        goto out;
    }
    {
        auto ck = [&](cudaError_t e) {
            if (e != cudaSuccess) st = cuda_fail(e, "packsell_f3r");
            return e == cudaSuccess;
        };
        auto true_residual = [&](double *rr) -> packsell_status {
            packsell_status e = spmv_f64_impl(A1, x, ax, s);
            if (e != PACKSELL_OK) return e;
            k_resid<<<G, FT, 0, s>>>(n, b, ax, r, F.part, F.counter, F.L1.h);  // beta = ||r||, v_0 scale
            PS_LAUNCH_CHECK("f3r: residual");
            double sc[3];
            if (!ck(cudaMemcpyAsync(sc, F.L1.h.scal, sizeof(sc), cudaMemcpyDeviceToHost, s)) ||
                !ck(cudaStreamSynchronize(s)))
                return st;
            *rr = sc[0];
            return PACKSELL_OK;
        };
        // ||b||
        if (!ck(cudaMemsetAsync(F.counter, 0, sizeof(unsigned), s))) goto out;
        k_norm2_begin<double><<<G, FT, 0, s>>>(n, b, F.part, F.counter, F.L1.h);
        double sc[3];
        if (!ck(cudaMemcpyAsync(sc, F.L1.h.scal, sizeof(sc), cudaMemcpyDeviceToHost, s)) ||
            !ck(cudaStreamSynchronize(s)))
            goto out;
        nb = sc[0];
        // layers 2-4 (the preconditioner of an outer step) as one CUDA graph:
        // a fixed sequence of some hundreds of kernels with no host step,
        // replayed on the fixed buffers prhs -> pout
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = fail(PACKSELL_ERR_CUDA, "packsell_f3r: stream capture failed to start");
            goto out;
        }
        {
            const packsell_status cst = F.layer2(prhs, pout);
            const cudaError_t ce = cudaStreamEndCapture(s, &graph);
            if (cst != PACKSELL_OK) {
                st = cst;
                goto out;
            }
            if (ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                st = fail(PACKSELL_ERR_CUDA, "packsell_f3r: graph capture failed");
                goto out;
            }
        }
        if (nb == 0.0) {
            if (!ck(cudaMemsetAsync(x, 0, sizeof(double) * n, s))) goto out;
            relres = relres_true = 0.0;
            converged = true;
            goto done;
        }
        cudaEventRecord(ev0, s);
        while (iters < o.max_iters && !converged) {
            // restart cycle: r = b - A x, v_0 = r / ||r||
            double rn = 0.0;
            st = true_residual(&rn);
            if (st != PACKSELL_OK) goto out;
            relres = rn / nb;
            if (relres < o.rtol) {
                relres_true = relres;
                converged = true;
                break;
            }
            k_scale<double, double><<<G, FT, 0, s>>>(n, r, F.L1.V, F.L1.h.scal + 1);
            int k = 0;
            for (; k < o.m1 && iters < o.max_iters; ++k) {
                if (!ck(cudaMemcpyAsync(prhs, F.L1.V + (int64_t)k * n, sizeof(double) * n,
                                        cudaMemcpyDeviceToDevice, s)) ||
                    !ck(cudaGraphLaunch(exec, s)) ||
                    !ck(cudaMemcpyAsync(F.L1.Z + (int64_t)k * n, pout, sizeof(double) * n,
                                        cudaMemcpyDeviceToDevice, s)))
                    goto out;
                st = F.arnoldi(F.L1, A1, k);
                if (st != PACKSELL_OK) goto out;
                ++iters;
                if (!ck(cudaMemcpyAsync(sc, F.L1.h.scal, sizeof(sc), cudaMemcpyDeviceToHost, s)) ||
                    !ck(cudaStreamSynchronize(s)))
                    goto out;
                relres = sc[2] / nb;
                if (!std::isfinite(relres)) {
                    st = fail(PACKSELL_ERR_BREAKDOWN, "packsell_f3r: non-finite residual");
                    goto out;
                }
                if (relres < o.rtol) {
                    ++k;
                    break;
                }
            }
            // x += sum_j y_j z_j over the cycle's k steps
            k_backsolve<<<1, 32, 0, s>>>(F.L1.h, k);
            k_combine<double, double, true><<<G, FT, 0, s>>>(n, F.L1.Z, k, F.L1.h.y, x);
            PS_LAUNCH_CHECK("f3r: update");
            ++steps;
            if (relres < o.rtol) {
                double rt = 0.0;
                st = true_residual(&rt);
                if (st != PACKSELL_OK) goto out;
                relres_true = rt / nb;
                if (relres_true < o.rtol) converged = true;
                // otherwise the next cycle restarts from the true residual
            }
        }
        cudaEventRecord(ev1, s);
        if (!ck(cudaStreamSynchronize(s))) goto out;
        if (relres_true < 0.0) {
            double rt = 0.0;
            st = true_residual(&rt);
            if (st != PACKSELL_OK) goto out;
            relres_true = rt / nb;
        }
    }
done:
    if (res) {
        float ms = 0.f;
        if (ev0 && ev1 && cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) ms = 0.f;
        res->iters = iters;
        res->inner_iters = iters * o.m2 * o.m3;
        res->relres = relres;
        res->relres_true = relres_true;
        res->seconds = ms * 1e-3;
    }
    if (!converged)
        st = fail(PACKSELL_ERR_NOT_CONVERGED,
                  "packsell_f3r: no convergence in " + std::to_string(o.max_iters) + " outer iterations");
out:
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (mem) cudaFreeAsync(mem, s);
    cudaStreamSynchronize(s);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    cudaStreamDestroy(s);
    (void)steps;
    (void)zt;
    return st;
}

}  // namespace

packsell_status f3r_impl(const Matrix *A1, const Matrix *A2, const Matrix *A3, const double *b,
                         double *x, const packsell_f3r_opts &o, packsell_solve_result *res,
                         cudaStream_t s) {
    if (!A1 || !A2 || !A3) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_f3r: NULL matrix");
    const int64_t n = A1->n;
    auto square = [&](const Matrix *A) { return A->n == n && A->m == n && !A->p.explicit_perm; };
    if (!is_f64_op(A1->p.format) || !square(A1) || !square(A2) || !square(A3))
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_f3r: A_outer must be SELL_F64 or W64_E11MY; all three square, of "
                    "one size, rows in original order");
    const bool all64 = is_f64_op(A2->p.format) && is_f64_op(A3->p.format);
    const bool mixed = A2->p.format == PACKSELL_FMT_SELL_F32 &&
                       (A3->p.format == PACKSELL_FMT_FP16 || A3->p.format == PACKSELL_FMT_SELL_F16 ||
                        A3->p.format == PACKSELL_FMT_E8MY);
    if (!all64 && !mixed)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_f3r: layers 2-4 need FP64 matrices (FP64-F3R) or SELL_F32 and a "
                    "PackSELL / FP16 SELL matrix (FP16-F3R)");
    if (o.m1 < 1 || o.m1 > 60 || o.m2 < 1 || o.m2 > 60 || o.m3 < 1 || o.m3 > 60 || o.m4 < 1 ||
        o.max_iters < 1 || !(o.rtol > 0.0) || !(o.omega > 0.0))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_f3r: bad options");
    if (n == 0) {
        if (res) *res = packsell_solve_result{};
        return PACKSELL_OK;
    }
    if (!b || !x) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_f3r: NULL vector");
    return all64 ? run_f3r<double>(*A1, *A2, *A3, b, x, o, res, s)
                 : run_f3r<float>(*A1, *A2, *A3, b, x, o, res, s);
}

}  // namespace packsell
