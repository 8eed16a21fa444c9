// Deterministic device reductions and the solver's device-resident scalars.
//
// A reducing kernel runs on a fixed grid; every block reduces its threads'
// contributions in a fixed tree, writes one partial per block, and the last
// block to finish (found with an atomic counter) adds the partials in block
// order and runs a "finish" step on the solver scalars (alpha, beta, norms).
// The result depends only on the grid size, never on block timing, so a
// solve is bitwise reproducible run to run on the same device.
#pragma once

#include <stdint.h>

#include "internal.h"

namespace packsell {

// Scalars of the solvers, all in double precision, kept on the device so the
// iteration never round-trips through the host.
struct SolveScalars {
    double rz, pq, alpha, beta;            // PCG (inner, or the FP64 baseline)
    double rr, bb, relres, rnorm;          // residual norms; rnorm = ||r||_2
    double zq, pq_o, pr_o, alpha_o, beta_o;  // outer flexible CG
    double rt;                             // ||b - A x||_2^2 of a true-residual check
    double rtol;                           // target relative residual
    int max_iters;                         // iteration cap (outer for IO-CG)
    int done;                              // below rtol or at the cap: later kernels idle
    int restart;                           // outer: next direction ignores the previous one
    int status;                            // PACKSELL_ERR_BREAKDOWN when set
    int iter;                              // outer iterations completed
    int inner;                             // inner iterations completed
};

enum Finish {
    FIN_NONE = 0,
    FIN_PQ_ALPHA,     // s1 = p.q        -> alpha = rz / pq (inner PCG: p.q <= 0 stalls it)
    FIN_PQ_ALPHA_64,  // as FIN_PQ_ALPHA, p.q <= 0 is a breakdown (FP64 PCG)
    FIN_RZ_INIT,      // s1 = r.z        -> rz
    FIN_RZ_BETA,      // s1 = r.z (new)  -> beta = rz_new / rz, rz = rz_new
    FIN_RZ_BETA_RR,   // as FIN_RZ_BETA, s2 = r.r -> relres (FP64 PCG iteration)
    FIN_ZQ_BETA,      // s1 = z.q        -> beta_o = zq / pq_o (0 after a restart)
    FIN_OUTER_ALPHA,  // s1 = p.q, s2 = p.r -> alpha_o = pr / pq
    FIN_RR,           // s1 = r.r        -> relres, rnorm; counts an outer iteration
    FIN_RR_PCG,       // s1 = r.r        -> relres (FP64 PCG, counted per iteration)
    FIN_BB_RR,        // s1 = b.b, s2 = r.r -> bb, rr, relres, rnorm
    FIN_RT            // s1 = ||b - A x||^2 -> rt
};

struct Red {
    double *partials;   // 2 doubles per block
    unsigned *counter;  // 0 between launches
    SolveScalars *sc;
    double *hist;       // optional relres history (indexed by outer iteration)
    int fin;
};

__device__ __forceinline__ void finish(const Red &r, double s1, double s2) {
    SolveScalars *sc = r.sc;
    switch (r.fin) {
        case FIN_PQ_ALPHA:
            sc->pq = s1;
            sc->alpha = (s1 > 0.0 && sc->rz > 0.0) ? sc->rz / s1 : 0.0;
            if (!isfinite(s1)) sc->status = PACKSELL_ERR_BREAKDOWN;
            sc->inner += 1;
            break;
        case FIN_PQ_ALPHA_64:
            sc->pq = s1;
            if (!(s1 > 0.0)) {
                sc->status = PACKSELL_ERR_BREAKDOWN;
                sc->alpha = 0.0;
            } else {
                sc->alpha = sc->rz / s1;
            }
            break;
        case FIN_RZ_INIT:
            sc->rz = s1;
            break;
        case FIN_RZ_BETA:
            sc->beta = (sc->rz > 0.0) ? s1 / sc->rz : 0.0;
            sc->rz = s1;
            break;
        case FIN_RZ_BETA_RR:
            sc->beta = (sc->rz > 0.0) ? s1 / sc->rz : 0.0;
            sc->rz = s1;
            sc->rr = s2;
            sc->rnorm = sqrt(s2);
            sc->relres = sc->bb > 0.0 ? sqrt(s2 / sc->bb) : 0.0;
            if (!isfinite(sc->relres)) sc->status = PACKSELL_ERR_BREAKDOWN;
            if (r.hist) r.hist[sc->iter + 1] = sc->relres;
            sc->iter += 1;
            if (sc->relres < sc->rtol || sc->iter >= sc->max_iters) sc->done = 1;
            break;
        case FIN_ZQ_BETA:
            sc->zq = s1;
            sc->beta_o = (sc->restart || !(sc->pq_o > 0.0)) ? 0.0 : s1 / sc->pq_o;
            sc->restart = 0;
            break;
        case FIN_OUTER_ALPHA:
            sc->pq_o = s1;
            sc->pr_o = s2;
            if (!(s1 > 0.0)) {
                sc->status = PACKSELL_ERR_BREAKDOWN;
                sc->alpha_o = 0.0;
            } else {
                sc->alpha_o = s2 / s1;
            }
            break;
        case FIN_RR:
        case FIN_RR_PCG:
            sc->rr = s1;
            sc->rnorm = sqrt(s1);
            sc->relres = sc->bb > 0.0 ? sqrt(s1 / sc->bb) : 0.0;
            if (!isfinite(sc->relres)) sc->status = PACKSELL_ERR_BREAKDOWN;
            if (r.hist) r.hist[sc->iter + 1] = sc->relres;
            sc->iter += 1;
            if (sc->relres < sc->rtol || sc->iter >= sc->max_iters) sc->done = 1;
            break;
        case FIN_BB_RR:
            sc->bb = s1;
            sc->rr = s2;
            sc->rnorm = sqrt(s2);
            sc->relres = s1 > 0.0 ? sqrt(s2 / s1) : 0.0;
            if (r.hist) r.hist[sc->iter] = sc->relres;
            sc->done = sc->relres < sc->rtol;
            break;
        case FIN_RT:
            sc->rt = s1;
            break;
        default:
            break;
    }
}

// Sum (v1, v2) over the block (blockDim.x a multiple of 32, at most 1024).
__device__ __forceinline__ void block_sum2(double &v1, double &v2) {
    __shared__ double s1[32], s2[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        v1 += __shfl_down_sync(0xffffffffu, v1, o);
        v2 += __shfl_down_sync(0xffffffffu, v2, o);
    }
    __syncthreads();  // the arrays may still be read by a previous call
    if (lane == 0) {
        s1[wid] = v1;
        s2[wid] = v2;
    }
    __syncthreads();
    if (wid == 0) {
        v1 = lane < nw ? s1[lane] : 0.0;
        v2 = lane < nw ? s2[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            v1 += __shfl_down_sync(0xffffffffu, v1, o);
            v2 += __shfl_down_sync(0xffffffffu, v2, o);
        }
    }
}

// Every thread of every block calls this once with its contributions.
__device__ __forceinline__ void reduce_publish(const Red &r, double v1, double v2) {
    __shared__ bool last;
    block_sum2(v1, v2);
    if (threadIdx.x == 0) {
        r.partials[2 * blockIdx.x] = v1;
        r.partials[2 * blockIdx.x + 1] = v2;
        __threadfence();
        last = atomicAdd(r.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) {
        a += ((volatile double *)r.partials)[2 * q];
        b += ((volatile double *)r.partials)[2 * q + 1];
    }
    block_sum2(a, b);
    if (threadIdx.x == 0) {
        finish(r, a, b);
        *r.counter = 0u;
    }
}

}  // namespace packsell
