// Batched PackSELL products: many matrices of uneven sizes per launch.
// A plan holds, on the device, one descriptor per matrix (its word, offset and
// perm arrays, parameters and bound vectors) and work lists:
//  * matrices with C = 32: items (matrix, slice range) of roughly equal word
//    counts; warps take items round-robin and lane l of a warp computes row l
//    of each slice of its item (thread-per-row, stored order, fused
//    multiply-adds: the same bits as packsell_spmv on each matrix alone);
//  * matrices with C = 1 (CSR order): split-row items (tiles of rows and
//    single long rows, long rows first) in one persistent launch for all of
//    them: a batched SpMV takes the items and kernel of variant 14 (each y
//    the bits of variant 14 on its matrix alone), a batched SpMM those of
//    multi.cu with k right-hand sides.
#include <cuda_fp16.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace packsell {

struct BatchMat {
    const uint32_t *pack;
    const int64_t *offset;
    const void *perm;
    const float *x;
    float *y;
    long long k_left;
    int n, m, sigma, sig_shift, perm_bytes, fmt;
    uint32_t dmask, vmask;
};

struct BatchItem {
    int mat, k0, k1, pad;
};

struct Batch {
    int count = 0;
    int nitems = 0;
    int blocks = 0;
    BatchMat *d_mats = nullptr;
    BatchItem *d_items = nullptr;
    std::vector<BatchMat> h_mats;
    int64_t words = 0, rows = 0, bytes = 0;
    // CSR-order (C = 1) matrices: split-row descriptors and items
    int k = 1;       // right-hand sides (1: a batched SpMV plan)
    bool vec = false;  // every X and Y allows 16-byte accesses
    SplitMat *d_smats = nullptr;
    MultiItem *d_mitems = nullptr;
    int n_mitems = 0;
    bool split1 = false;  // the items are variant 14's (one right-hand side)
    bool sorted = false;  // a CSR-order matrix has sigma > 1
};

namespace {

constexpr int BTPB = 256;
constexpr int BPF = 16;  // words of a row loaded per round

template <int FMT>
__device__ __forceinline__ float row_dot(const BatchMat &M, int row, int64_t s, int w) {
    const uint32_t *__restrict__ pp = M.pack + s + (row & 31);
    const int blk = M.sig_shift >= 0 ? (row >> M.sig_shift) << M.sig_shift : (row / M.sigma) * M.sigma;
    int c = (M.k_left < blk) ? (int)(blk - M.k_left) : 0;
    float t = 0.f;
    for (int j0 = 0; j0 < w; j0 += BPF) {
        const int wr = w - j0;
        uint32_t wd[BPF];
#pragma unroll
        for (int u = 0; u < BPF; ++u) wd[u] = (u < wr) ? ldg_stream(pp + (j0 + u) * 32) : 0u;
        bool f[BPF];
        float xv[BPF];
#pragma unroll
        for (int u = 0; u < BPF; ++u) {
            f[u] = (wd[u] & 1u) != 0u;
            c += (int)((wd[u] >> 1) & (f[u] ? M.dmask : 0x7fffffffu));
            if (f[u]) xv[u] = PS_IN_RANGE(c, M.m) ? __ldg(M.x + c) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < BPF; ++u) {
            if (f[u]) {
                const float v = FMT == PACKSELL_FMT_FP16
                                    ? __high2float(*reinterpret_cast<const __half2 *>(&wd[u]))
                                    : __uint_as_float(wd[u] & M.vmask);
                t = fmaf(v, xv[u], t);
            }
        }
        if (wd[BPF - 1] == 0u) break;  // padding: the row has ended
    }
    return t;
}

__global__ void __launch_bounds__(BTPB)
    k_spmv_batched(const BatchMat *__restrict__ mats, const BatchItem *__restrict__ items,
                   int nitems) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int it = gw; it < nitems; it += nw) {
        const BatchItem item = items[it];
        const BatchMat M = mats[item.mat];
        for (int k = item.k0; k < item.k1; ++k) {
            const int64_t s = M.offset[k];
            const int w = (int)((M.offset[k + 1] - s) >> 5);
            const int row = k * 32 + lane;
            const float t = (M.fmt == PACKSELL_FMT_FP16) ? row_dot<PACKSELL_FMT_FP16>(M, row, s, w)
                                                         : row_dot<PACKSELL_FMT_E8MY>(M, row, s, w);
            if (row < M.n) {
                int io = row;
                if (M.perm_bytes) {
                    const int blk = M.sig_shift >= 0 ? (row >> M.sig_shift) << M.sig_shift
                                                     : (row / M.sigma) * M.sigma;
                    io = blk + (M.perm_bytes == 1 ? (int)((const uint8_t *)M.perm)[row]
                                                  : (int)((const uint16_t *)M.perm)[row]);
                }
                M.y[io] = t;
            }
        }
    }
}

}  // namespace

void batch_free(Batch *B) {
    if (!B) return;
    cudaFree(B->d_mats);
    cudaFree(B->d_items);
    cudaFree(B->d_smats);
    cudaFree(B->d_mitems);
    delete B;
}

// Upload the split-row part of a plan: descriptors (one per matrix, C = 32
// matrices included but never referenced) and items.
static packsell_status upload_split(Batch *B, const std::vector<SplitMat> &smats,
                                    std::vector<MultiItem> &mitems, cudaStream_t s) {
    if (mitems.empty()) return PACKSELL_OK;
    multi_items_order(mitems);
    if (mitems.size() >= (size_t)INT32_MAX)
        return fail(PACKSELL_ERR_RANGE, "packsell_batch_create: too many items");
    if (cudaMalloc(&B->d_smats, sizeof(SplitMat) * smats.size()) != cudaSuccess ||
        cudaMalloc(&B->d_mitems, sizeof(MultiItem) * mitems.size()) != cudaSuccess)
        return fail(PACKSELL_ERR_NO_MEMORY, "packsell_batch_create: plan arrays");
    cudaError_t e = cudaMemcpyAsync(B->d_smats, smats.data(), sizeof(SplitMat) * smats.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_mitems, mitems.data(), sizeof(MultiItem) * mitems.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "packsell_batch_create: plan copy");
    B->n_mitems = (int)mitems.size();
    return PACKSELL_OK;
}

packsell_status batch_create(int count, const Matrix *const *A, const float *const *x,
                             float *const *y, cudaStream_t s, Batch **out) {
    *out = nullptr;
    if (count < 1) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create: count < 1");
    Batch *B = new Batch();
    B->count = count;
    B->h_mats.resize(count);
    std::vector<BatchItem> items;
    std::vector<int64_t> offs;
    std::vector<SplitMat> smats(count);
    std::vector<MultiItem> mitems;
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_spmv_batched, BTPB, 0) != cudaSuccess) {
        batch_free(B);
        return fail(PACKSELL_ERR_CUDA, "packsell_batch_create: device query failed");
    }
    B->blocks = sms * std::max(per, 1);
    const int64_t warps = (int64_t)B->blocks * (BTPB / 32);
    int64_t total_words = 0;
    for (int i = 0; i < count; ++i) {
        const Matrix *m = A[i];
        if (!m || !is_packed(m->p.format) || (m->p.C != 32 && m->p.C != 1)) {
            batch_free(B);
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create: matrix " + std::to_string(i) +
                                                      " is not a PackSELL matrix with C = 32 or C = 1");
        }
        if ((m->m > 0 && !x[i]) || (m->n > 0 && !y[i])) {
            batch_free(B);
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create: NULL vector for matrix " +
                                                      std::to_string(i));
        }
        if (m->p.C == 32) total_words += m->n_words;
    }
    // items of about total / (8 * warps) words (at least 2048), whole slices
    const int64_t target = std::max<int64_t>(2048, total_words / std::max<int64_t>(1, 8 * warps));
    for (int i = 0; i < count; ++i) {
        const Matrix *m = A[i];
        const int sg = m->p.sigma;
        BatchMat d{};
        d.pack = m->pack;
        d.offset = m->offset;
        d.perm = m->p.explicit_perm ? nullptr : m->perm;
        d.perm_bytes = m->p.explicit_perm ? 0 : m->perm_bytes;
        d.x = x[i];
        d.y = y[i];
        d.k_left = m->p.k_left;
        d.n = (int)m->n;
        d.m = (int)m->m;
        d.sigma = sg;
        d.sig_shift = (sg & (sg - 1)) == 0 ? __builtin_ctz((unsigned)sg) : -1;
        d.fmt = m->p.format;
        d.dmask = (1u << m->p.D) - 1u;
        d.vmask = ~((2u << m->p.D) - 1u);
        B->h_mats[i] = d;
        smats[i] = split_mat(*m, x[i], 1, y[i], 1, 1);
        B->words += m->n_words;
        B->rows += m->n;
        B->bytes += 4 * m->n_words + 8 * (m->n_slices + 1) + (int64_t)d.perm_bytes * m->n + 4 * m->m +
                    4 * m->n;
        if (m->n == 0) continue;
        offs.resize(m->n_slices + 1);
        if (cudaMemcpy(offs.data(), m->offset, 8 * (m->n_slices + 1), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            batch_free(B);
            return fail(PACKSELL_ERR_CUDA, "packsell_batch_create: reading offsets");
        }
        if (m->p.C == 1) {
            B->sorted = B->sorted || m->p.sigma > 1;
            const packsell_status st = split_items_append(offs.data(), m->n, i, mitems);
            if (st != PACKSELL_OK) {
                batch_free(B);
                return st;
            }
            continue;
        }
        int k0 = 0;
        for (int k = 0; k < m->n_slices; ++k) {
            if (offs[k + 1] - offs[k0] >= target || k + 1 == m->n_slices) {
                items.push_back(BatchItem{i, k0, k + 1, 0});
                k0 = k + 1;
            }
        }
    }
    B->nitems = (int)items.size();
    if (cudaMalloc(&B->d_mats, sizeof(BatchMat) * count) != cudaSuccess ||
        cudaMalloc(&B->d_items, sizeof(BatchItem) * std::max<size_t>(1, items.size())) != cudaSuccess) {
        batch_free(B);
        return fail(PACKSELL_ERR_NO_MEMORY, "packsell_batch_create: plan arrays");
    }
    cudaError_t e = cudaMemcpyAsync(B->d_mats, B->h_mats.data(), sizeof(BatchMat) * count,
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(B->d_items, items.data(), sizeof(BatchItem) * items.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        batch_free(B);
        return cuda_fail(e, "packsell_batch_create: plan copy");
    }
    B->split1 = true;
    const packsell_status st = upload_split(B, smats, mitems, s);
    if (st != PACKSELL_OK) {
        batch_free(B);
        return st;
    }
    *out = B;
    return PACKSELL_OK;
}

packsell_status batch_create_mm(int count, const Matrix *const *A, int k, const float *const *X,
                                const int64_t *ldx, float *const *Y, const int64_t *ldy,
                                cudaStream_t s, Batch **out) {
    *out = nullptr;
    if (count < 1 || k < 1)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create_spmm: count < 1 or k < 1");
    Batch *B = new Batch();
    B->count = count;
    B->k = k;
    std::vector<SplitMat> smats(count);
    std::vector<MultiItem> mitems;
    std::vector<int64_t> offs;
    std::vector<std::vector<int64_t>> offs_all;  // row offsets of the matrices with rows
    bool vec = k % 4 == 0;
    // one right-hand side in contiguous vectors: the SpMV items and kernel
    bool split1 = k == 1;
    for (int i = 0; i < count; ++i) {
        const Matrix *m = A[i];
        const int64_t lx = ldx ? ldx[i] : k, ly = ldy ? ldy[i] : k;
        if (!m || !is_packed(m->p.format) || m->p.C != 1) {
            batch_free(B);
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create_spmm: matrix " +
                                                      std::to_string(i) +
                                                      " is not a PackSELL matrix with C = 1");
        }
        if ((m->m > 0 && !X[i]) || (m->n > 0 && !Y[i]) || lx < k || ly < k) {
            batch_free(B);
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create_spmm: NULL block or "
                                                  "leading dimension below k for matrix " +
                                                      std::to_string(i));
        }
        vec = vec && lx % 4 == 0 && ly % 4 == 0 && ((uintptr_t)X[i] & 15) == 0 &&
              ((uintptr_t)Y[i] & 15) == 0;
        split1 = split1 && lx == 1 && ly == 1;
        B->sorted = B->sorted || m->p.sigma > 1;
        smats[i] = split_mat(*m, X[i], lx, Y[i], ly, k);
        B->words += m->n_words;
        B->rows += m->n;
        B->bytes += 4 * m->n_words + 8 * (m->n_slices + 1) +
                    (int64_t)(m->p.explicit_perm ? 0 : m->perm_bytes) * m->n + 4 * (int64_t)k * (m->m + m->n);
        if (m->n == 0) continue;
        offs.resize(m->n_slices + 1);
        if (cudaMemcpy(offs.data(), m->offset, 8 * (m->n_slices + 1), cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
            batch_free(B);
            return fail(PACKSELL_ERR_CUDA, "packsell_batch_create_spmm: reading offsets");
        }
        offs_all.push_back(offs);
    }
    B->vec = vec;
    B->split1 = split1;
    for (int i = 0, j = 0; i < count; ++i) {
        if (A[i]->n == 0) continue;
        const std::vector<int64_t> &o = offs_all[j++];
        if (split1) {
            const packsell_status st = split_items_append(o.data(), A[i]->n, i, mitems);
            if (st != PACKSELL_OK) {
                batch_free(B);
                return st;
            }
        } else {
            multi_items_append(o.data(), A[i]->n, i, mitems);
        }
    }
    const packsell_status st = upload_split(B, smats, mitems, s);
    if (st != PACKSELL_OK) {
        batch_free(B);
        return st;
    }
    *out = B;
    return PACKSELL_OK;
}

void batch_stats(const Batch &B, int64_t *words, int64_t *bytes, int32_t *items) {
    if (words) *words = B.words;
    if (bytes) *bytes = B.bytes;
    if (items) *items = B.nitems + B.n_mitems;
}

packsell_status batch_spmv(const Batch &B, cudaStream_t s) {
    if (!B.d_mats)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_batch_spmv: a plan from packsell_batch_create_spmm (use packsell_batch_spmm)");
    if (B.nitems > 0) {
        k_spmv_batched<<<B.blocks, BTPB, 0, s>>>(B.d_mats, B.d_items, B.nitems);
        PS_LAUNCH_CHECK("packsell_batch_spmv");
    }
    return launch_split_batch(B.d_smats, B.d_mitems, B.n_mitems, B.sorted, s);
}

packsell_status batch_spmm(const Batch &B, cudaStream_t s) {
    if (B.d_mats)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_spmm: the plan is a batched SpMV plan");
    if (B.split1) return launch_split_batch(B.d_smats, B.d_mitems, B.n_mitems, B.sorted, s);
    return launch_multi(SplitMat{}, B.d_smats, B.d_mitems, B.n_mitems, B.k, B.vec, s);
}

}  // namespace packsell
