// Stage-planned TMA SpMV (C = 32), variants 9 and 10.
//
// At plan time every warp's contiguous run of slices (the same word-balanced
// partition as the bulk kernels) is cut into stages: consecutive whole slices
// up to SW words, or SW-word pieces (whole columns) of a slice that is larger
// than a stage. A stage is one contiguous run of words, copied into a
// shared-memory slot by one cp.async.bulk (TMA engine) that completes on the
// slot's mbarrier; lane 0 keeps NS stages in flight. The consumer waits once
// per stage and walks its slices without any wrap or chunk test: lane l
// decodes row l of each slice (one bank per lane), issuing all gathers of a
// round of up to PF words before the round's fused multiply-adds. Rows are
// summed in stored order, so results equal every other variant's bits.
// All waits are bounded; a timeout is recorded in the matrix's status word,
// the copies already issued are allowed to land, and the warp returns.
#include <cuda_fp16.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"

namespace packsell {
namespace {

// ---- plan: stage boundaries per warp ----------------------------------------
// Boundaries are word offsets relative to the warp's first word; warp g's
// list sb[sptr[g] .. sptr[g+1]) holds (stages + 1) entries, 0 first, the
// warp's word count last.
template <bool FILL>
__global__ void k_stage_plan(int G, const int32_t *__restrict__ part,
                             const int64_t *__restrict__ offset, int SW,
                             int64_t *__restrict__ count, const int64_t *__restrict__ sptr,
                             int32_t *__restrict__ sb) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const int k0 = part[g], k1 = part[g + 1];
    const int64_t base = k0 < k1 ? offset[k0] : 0;
    int64_t nb = 0;  // boundaries written after the leading 0
    int32_t *out = FILL ? sb + sptr[g] : nullptr;
    if (FILL) out[0] = 0;
    auto emit = [&](int64_t b) {
        ++nb;
        if (FILL) out[nb] = (int32_t)b;
    };
    int64_t cur_lo = 0, cur_hi = 0;
    for (int k = k0; k < k1; ++k) {
        const int64_t lo = offset[k] - base, hi = offset[k + 1] - base;
        if (hi == lo) continue;
        if (hi - lo <= SW) {
            if (hi - cur_lo > SW) {
                emit(lo);
                cur_lo = lo;
            }
            cur_hi = hi;
        } else {
            if (cur_hi > cur_lo) {
                emit(lo);
                cur_lo = lo;
            }
            for (int64_t b = lo + SW; b < hi; b += SW) {
                emit(b);
                cur_lo = b;
            }
            cur_hi = hi;
        }
    }
    if (cur_hi > cur_lo) emit(cur_hi);  // closes the last stage at the warp's word count
    if (!FILL) count[g] = nb + 1;       // entries of the list
}

// ---- the kernel ---------------------------------------------------------------
template <int FMT, int PF>
__device__ __forceinline__ void stage_run(const uint32_t *rs, int ncol, Decode dc,
                                          const float *__restrict__ x, int &c, float &t) {
    for (int j0 = 0; j0 < ncol; j0 += PF) {
        const int r = ncol - j0;
        uint32_t wd[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) wd[u] = (u < r) ? rs[(j0 + u) * 32] : 0u;
        bool f[PF];
        float xv[PF];
#pragma unroll
        for (int u = 0; u < PF; ++u) word_gather<FMT>(wd[u], dc, x, c, f[u], xv[u]);
#pragma unroll
        for (int u = 0; u < PF; ++u)
            if (f[u]) t = fmaf(word_value<FMT>(wd[u], dc), xv[u], t);
    }
}

template <int FMT, int NW, int NS, int SW, int PF, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB)
    k_spmv_stage(int n, int sigma, int sig_shift, long long k_left,
                 const int64_t *__restrict__ offset, const uint32_t *__restrict__ pack,
                 const void *__restrict__ perm, int perm_bytes, Decode dc,
                 const float *__restrict__ x, float *__restrict__ y,
                 const int32_t *__restrict__ part, const int64_t *__restrict__ sptr,
                 const int32_t *__restrict__ sbnd, DevStatus *st, uint32_t wait_limit) {
    static_assert((NS & (NS - 1)) == 0, "NS: power of two");
    extern __shared__ __align__(128) uint32_t ring_all[];
    __shared__ __align__(8) uint64_t bars[NW][NS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * NW + warp;
    const int k0 = part[gw], k1 = part[gw + 1];
    if (k0 >= k1) return;  // warp-uniform
    uint32_t *ring = ring_all + warp * NS * SW;
    uint64_t *bar = bars[warp];
    const int64_t base = offset[k0];
    const uint32_t *src = pack + base;
    const int32_t *B = sbnd + sptr[gw];
    const int nst = (int)(sptr[gw + 1] - sptr[gw]) - 1;
    const uint64_t pol = policy_evict_first();
    if (lane == 0) {
        for (int q = 0; q < NS; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncwarp();

    // stage boundaries, 32 at a time in lanes; out-of-batch ones read directly
    int gb = 0;
    int32_t bl = (lane <= nst) ? B[lane] : 0;
    auto bound = [&](int i) -> int {
        const int d = i - gb;
        const int v = __shfl_sync(0xffffffffu, bl, d & 31);
        return (d >= 0 && d < 32) ? v : B[i];
    };
    auto issue = [&](int g) {
        const int lo = bound(g), hi = bound(g + 1);
        if (lane == 0) {
            uint64_t *b = &bar[g & (NS - 1)];
            const uint32_t bytes = (uint32_t)(hi - lo) * 4u;
            mbar_expect_tx(b, bytes);
            bulk_g2s(ring + (g & (NS - 1)) * SW, src + lo, bytes, b, pol);
        }
    };
    int issued = 0;
    for (; issued < NS && issued < nst; ++issued) issue(issued);

    // slice offsets, 32 at a time in lanes
    int kb = k0;
    int64_t o_lo = (kb + lane < k1) ? offset[kb + lane] - base : 0;
    int64_t o_hi = (kb + lane < k1) ? offset[kb + lane + 1] - base : 0;
    int k = k0, j = 0, s0 = 0, w = 0, row = 0, yo = 0, c = 0;
    float t = 0.f;
    auto setup = [&]() {  // state of slice k (uniform), row of this lane
        if (k - kb >= 32) {
            kb = k;
            o_lo = (kb + lane < k1) ? offset[kb + lane] - base : 0;
            o_hi = (kb + lane < k1) ? offset[kb + lane + 1] - base : 0;
        }
        const int q = k - kb;
        s0 = (int)__shfl_sync(0xffffffffu, o_lo, q);
        w = ((int)__shfl_sync(0xffffffffu, o_hi, q) - s0) >> 5;
        j = 0;
        row = k * 32 + lane;
        const int blk = sig_shift >= 0 ? (row >> sig_shift) << sig_shift : (row / sigma) * sigma;
        c = (k_left < blk) ? (int)(blk - k_left) : 0;
        yo = row;
        if (perm_bytes && row < n)
            yo = blk + (perm_bytes == 1 ? (int)((const uint8_t *)perm)[row]
                                        : (int)((const uint16_t *)perm)[row]);
        t = 0.f;
    };
    setup();
    for (int g = 0; g < nst; ++g) {
        if (g - gb >= 32) {  // next 32 boundaries
            gb = g;
            bl = (gb + lane <= nst) ? B[gb + lane] : 0;
        }
        if (!__all_sync(0xffffffffu,
                        mbar_wait(&bar[g & (NS - 1)], (uint32_t)((g / NS) & 1), wait_limit))) {
            if (lane == 0) dev_fail(st, PACKSELL_ERR_TIMEOUT, gw);
            for (int h = g; h < issued; ++h) mbar_wait(&bar[h & (NS - 1)], (uint32_t)((h / NS) & 1));
            return;
        }
        const int lo = bound(g), hi = bound(g + 1);
        const uint32_t *rs = ring + (g & (NS - 1)) * SW - lo + lane;  // rs[p]: word p of the stream
        while (k < k1) {
            const int pos = s0 + 32 * j;
            if (w > 0 && pos >= hi) break;  // the slice goes on in a later stage
            const int ncol = min(w - j, (hi - pos) >> 5);
            if (ncol > 0) stage_run<FMT, PF>(rs + pos, ncol, dc, x, c, t);
            j += ncol;
            if (j < w) break;
            if (row < n) y[yo] = t;
            ++k;
            if (k < k1) setup();
        }
        __syncwarp();
        if (lane == 0) fence_proxy_async_smem();
        if (issued < nst) issue(issued++);
    }
    while (k < k1) {  // empty slices after the warp's last word
        if (row < n) y[yo] = t;
        ++k;
        if (k < k1) setup();
    }
}

struct StageCfg {
    int nw, ns, sw;
    size_t smem() const { return sizeof(uint32_t) * (size_t)nw * ns * sw; }
};
constexpr StageCfg kStageCfg[2] = {{8, 2, 1024}, {8, 2, 512}};

template <int FMT, int V>
struct StageKernel;
template <int FMT>
struct StageKernel<FMT, 0> {
    static constexpr auto fn = k_spmv_stage<FMT, 8, 2, 1024, 16, 3>;
};
template <int FMT>
struct StageKernel<FMT, 1> {
    static constexpr auto fn = k_spmv_stage<FMT, 8, 2, 512, 12, 5>;
};

template <int FMT>
void *stage_fn(int v) {
    return v == 0 ? (void *)StageKernel<FMT, 0>::fn : (void *)StageKernel<FMT, 1>::fn;
}

__global__ void k_stage_partition(int64_t S, const int64_t *__restrict__ offset, int G,
                                  int32_t *__restrict__ part) {
    int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > G) return;
    int64_t total = offset[S];
    int64_t target = (int64_t)((__int128)total * g / G);
    int64_t lo = 0, hi = S;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (offset[mid] >= target) hi = mid;
        else lo = mid + 1;
    }
    part[g] = (int32_t)(g == G ? S : lo);
}

}  // namespace

void stage_free(Matrix &A) {
    for (int v = 0; v < Matrix::kStageVariants; ++v) {
        cudaFree(A.stage[v].part);
        cudaFree(A.stage[v].sptr);
        cudaFree(A.stage[v].sb);
        A.stage[v] = StagePlan{};
    }
}

packsell_status plan_stage(Matrix &A, cudaStream_t s) {
    stage_free(A);
    if (!is_packed(A.p.format) || A.p.C != 32 || A.n == 0 || A.n_words >= (1ll << 31) - 4096)
        return PACKSELL_OK;
    int dev = 0, sms = 0;
    PS_CUDA(cudaGetDevice(&dev));
    PS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (int v = 0; v < Matrix::kStageVariants; ++v) {
        const StageCfg &cf = kStageCfg[v];
        void *fn = A.p.format == PACKSELL_FMT_FP16 ? stage_fn<PACKSELL_FMT_FP16>(v)
                                                   : stage_fn<PACKSELL_FMT_E8MY>(v);
        PS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cf.smem()));
        int per = 0;
        PS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, cf.nw * 32, cf.smem()));
        if (per < 1) continue;
        StagePlan &P = A.stage[v];
        P.blocks = sms * per;
        const int G = P.blocks * cf.nw;
        P.warps = G;
        int64_t *cnt = nullptr;
        PS_CUDA(cudaMalloc(&P.part, sizeof(int32_t) * (G + 1)));
        PS_CUDA(cudaMalloc(&P.sptr, sizeof(int64_t) * (G + 1)));
        PS_CUDA(cudaMallocAsync(&cnt, sizeof(int64_t) * G, s));
        k_stage_partition<<<(G + 256) / 256, 256, 0, s>>>(A.n_slices, A.offset, G, P.part);
        k_stage_plan<false><<<(G + 255) / 256, 256, 0, s>>>(G, P.part, A.offset, cf.sw, cnt, nullptr, nullptr);
        packsell_status e = scan_i64(cnt, P.sptr, G, s);
        if (e != PACKSELL_OK) return e;
        int64_t total = 0;
        PS_CUDA(cudaMemcpyAsync(&total, P.sptr + G, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PS_CUDA(cudaStreamSynchronize(s));
        PS_CUDA(cudaMalloc(&P.sb, sizeof(int32_t) * std::max<int64_t>(total, 1)));
        k_stage_plan<true><<<(G + 255) / 256, 256, 0, s>>>(G, P.part, A.offset, cf.sw, nullptr, P.sptr, P.sb);
        PS_CUDA(cudaFreeAsync(cnt, s));
        PS_LAUNCH_CHECK("plan_stage");
    }
    return PACKSELL_OK;
}

packsell_status launch_stage(const Matrix &A, int v, const void *perm, int pb, const float *x,
                             float *y, cudaStream_t s) {
    const StagePlan &P = A.stage[v];
    if (!P.part) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: stage variant unavailable");
    const StageCfg &cf = kStageCfg[v];
    int n = (int)A.n, sg = A.p.sigma;
    int sh = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
    long long kl = A.p.k_left;
    Decode dc = make_decode(A);
    const int64_t *offset = A.offset;
    const uint32_t *pack = A.pack;
    const int32_t *part = P.part, *sb = P.sb;
    const int64_t *sptr = P.sptr;
    DevStatus *st = A.status;
    uint32_t wl = data_wait_limit();
    void *args[] = {&n, &sg, &sh, &kl, (void *)&offset, (void *)&pack, (void *)&perm, &pb, &dc,
                    (void *)&x, (void *)&y, (void *)&part, (void *)&sptr, (void *)&sb, (void *)&st,
                    &wl};
    void *fn = A.p.format == PACKSELL_FMT_FP16 ? stage_fn<PACKSELL_FMT_FP16>(v)
                                               : stage_fn<PACKSELL_FMT_E8MY>(v);
    PS_CUDA(cudaLaunchKernel(fn, dim3(P.blocks), dim3(cf.nw * 32), args, cf.smem(), s));
    return PACKSELL_OK;
}

}  // namespace packsell
