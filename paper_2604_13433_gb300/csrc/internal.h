// Internal declarations of the PackSELL CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "packsell.h"

namespace packsell {

// Device status word written by kernels that validate input. The first
// kernel to find a problem records its code and the offending index.
struct DevStatus {
    int code;      // packsell_status, 0 = fine
    int pad;
    long long index;
};

// Stage plan of a stage-planned SpMV configuration (stage.cu).
struct StagePlan {
    int32_t *part = nullptr;  // warps + 1 slice boundaries
    int64_t *sptr = nullptr;  // warps + 1 starts of each warp's boundary list
    int32_t *sb = nullptr;    // boundary lists (relative word offsets)
    int blocks = 0, warps = 0;
};

struct Matrix {
    int64_t n = 0, m = 0, nnz = 0;
    packsell_params p{};
    int64_t n_slices = 0, n_words = 0, n_dummies = 0, n_pad = 0;
    int32_t max_width = 0;
    int32_t perm_bytes = 0;
    int32_t value_exp = 0;  // FIXED: value = q * 2^value_exp
    int device = 0;
    // device arrays
    uint32_t *pack = nullptr;  // PackSELL words
    uint16_t *pack16 = nullptr;  // 16-bit words (PACKSELL_FMT_W16_E4M3)
    uint64_t *pack64 = nullptr;  // 64-bit words (PACKSELL_FMT_W64_E11MY)
    void *val = nullptr;       // SELL values (float / double)
    int32_t *col = nullptr;    // SELL columns
    int64_t *offset = nullptr; // n_slices + 1
    void *perm = nullptr;      // n entries of perm_bytes
    int64_t *rowptr = nullptr; // optional copy of the CSR row pointer
    DevStatus *status = nullptr; // device status word of the SpMV kernels
    // SpMV launch plan: the variant in use and, for each bulk-staged
    // configuration, the per-warp slice partition of a persistent grid
    static constexpr int kBulkVariants = 3;
    int variant = 0;       // 0 auto, 1 thread-per-row, 2.. bulk-staged configs
    int auto_variant = 1;  // what variant 0 runs (set by the plan or the tuner)
    int32_t *part[kBulkVariants] = {};  // part_warps + 1 slice boundaries
    int part_warps[kBulkVariants] = {};
    int part_blocks[kBulkVariants] = {};
    static constexpr int kStageVariants = 2;  // variants 9, 10
    StagePlan stage[kStageVariants];
    // variant 11 (C = 1): work items (first row, last row + 1) of the
    // CSR-order kernel, as int2 pairs
    void *csr_items = nullptr;
    int csr_nitems = 0;
    // variant 14 (C = 1): work items of the split-row kernel
    void *split_items = nullptr;
    int split_nitems = 0;
    // C = 1: work items of the split-row SpMM (multi.cu)
    void *multi_items = nullptr;
    int multi_nitems = 0;
};

// Spare words allocated after a matrix's packed word array (never read as
// data): 16-byte vector loads of the last words stay inside the allocation.
constexpr int64_t kWordTail = 4;

inline bool is_packed(int fmt) { return fmt == PACKSELL_FMT_FP16 || fmt == PACKSELL_FMT_E8MY; }
inline bool is_sell(int fmt) { return fmt == PACKSELL_FMT_SELL_F32 || fmt == PACKSELL_FMT_SELL_F64; }
inline bool is_w16(int fmt) { return fmt == PACKSELL_FMT_W16_E4M3; }
inline bool is_sell16(int fmt) { return fmt == PACKSELL_FMT_SELL_F16; }
inline bool is_fixed(int fmt) { return fmt == PACKSELL_FMT_FIXED; }
inline bool is_w64(int fmt) { return fmt == PACKSELL_FMT_W64_E11MY; }
// the formats whose products are FP64 (packsell_spmv_f64)
inline bool is_f64_op(int fmt) { return fmt == PACKSELL_FMT_SELL_F64 || is_w64(fmt); }

// bounds-check build: each translation unit registers a reader of its
// counters (out-of-range accesses, first index; read and cleared)
using ChecksReader = cudaError_t (*)(unsigned long long *count, long long *first);
void register_checks_reader(ChecksReader r);

// thread-local error message
packsell_status fail(packsell_status st, const std::string &msg);
packsell_status cuda_fail(cudaError_t e, const char *where);
void clear_error();

int64_t matrix_bytes(const Matrix &A);

// encode.cu
packsell_status encode_impl(const packsell_params &p, int64_t n, int64_t m, int64_t nnz,
                            const int64_t *rowptr, const int32_t *col, const void *val,
                            int val_is_f64, cudaStream_t s, Matrix **out);
packsell_status validate_impl(const Matrix &A, cudaStream_t s, const char *what);
void destroy_matrix(Matrix *A);
packsell_status scan_i64(const int64_t *in, int64_t *out, int64_t S, cudaStream_t s);
packsell_status quantize_impl(int fmt, int D, int64_t n, const void *val, int is64, uint32_t *field,
                              int64_t *bad_index, cudaStream_t s);
// max_i sum_j |a_ij - q(a_ij)|, max_i sum_j |q(a_ij)|, max_i sum_j |a_ij| for a
// format (out[0..2]), the longest row, and a nonzero *bad if a value does
// not fit the format
packsell_status format_error_impl(int64_t n, const int64_t *rowptr, const void *val, int is64,
                                  int fmt, int D, cudaStream_t s, double out[3], int64_t *max_len,
                                  int *bad);

// stage.cu
packsell_status plan_stage(Matrix &A, cudaStream_t s);
void stage_free(Matrix &A);

// w16.cu
packsell_status spmv_w16_impl(const Matrix &A, const float *x, float *y, cudaStream_t s);

// half_io.cu
packsell_status spmv_x16_impl(const Matrix &A, const uint16_t *x, uint16_t *y, cudaStream_t s);

// csr.cu
packsell_status plan_csr(Matrix &A, cudaStream_t s);
void csr_plan_free(Matrix &A);
packsell_status launch_csr(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                           cudaStream_t s);
// multi.cu: split-row products with k right-hand sides over CSR-order
// (C = 1) PackSELL matrices, one matrix or a batch in one launch
constexpr int kMultiTileWords = 125;  // words of a tile at most
constexpr int kMultiTileRows = 128;   // rows of a tile at most
struct SplitMat {  // one matrix of a split-row product and its vectors
    const uint32_t *pack;
    const int64_t *offset;
    const void *perm;  // NULL: y in storage order
    const float *X;    // [m x k], row-major, leading dimension ldx
    float *Y;          // [n x k], row-major, leading dimension ldy
    long long ldx, ldy;
    int k, sigma, sig_shift, kl, perm_bytes, fmt;
    uint32_t dmask, vmask;
    int xlen;  // rows of X (m)
};
struct __align__(16) MultiItem {  // a tile (meta = rows << 16 | words) or a long row (meta = -words)
    long long base;
    int r0;
    int meta;
    int mat;
    int pad0, pad1, pad2;
};
SplitMat split_mat(const Matrix &A, const float *X, int64_t ldx, float *Y, int64_t ldy, int k);
void multi_items_append(const int64_t *off, int64_t n, int mat, std::vector<MultiItem> &items);
void multi_items_order(std::vector<MultiItem> &items);
packsell_status multi_plan(Matrix &A, cudaStream_t s);
void multi_plan_free(Matrix &A);
packsell_status launch_multi(const SplitMat &single, const SplitMat *mats, const MultiItem *items,
                             int nitems, int k, bool vec, cudaStream_t s);

// split.cu
packsell_status plan_split(Matrix &A, cudaStream_t s);
void split_plan_free(Matrix &A);
packsell_status split_items_append(const int64_t *off, int64_t n, int mat,
                                   std::vector<MultiItem> &items);
packsell_status launch_split_batch(const SplitMat *mats, const MultiItem *items, int nitems,
                                   bool sorted, cudaStream_t s);
packsell_status launch_split(const Matrix &A, const void *perm, int pb, const float *x, float *y,
                             cudaStream_t s);

packsell_status launch_stage(const Matrix &A, int v, const void *perm, int pb, const float *x,
                             float *y, cudaStream_t s);

// spmv.cu
constexpr uint32_t kWaitLimit = 1u << 24;  // default polls of a bounded mbarrier wait
uint32_t data_wait_limit();
void set_data_wait_limit(uint32_t limit);
packsell_status plan_spmv(Matrix &A, cudaStream_t s);
packsell_status spmv_impl(const Matrix &A, const float *x, float *y, cudaStream_t s);
packsell_status spmv_f64_impl(const Matrix &A, const double *x, double *y, cudaStream_t s);
packsell_status spmm_impl(const Matrix &A, int k, const float *X, int64_t ldx, float *Y,
                          int64_t ldy, cudaStream_t s);
packsell_status spmv_t_impl(const Matrix &A, const float *dy, float *dx, cudaStream_t s);
packsell_status pattern_outer_impl(const Matrix &A, float alpha, const float *u, const float *v,
                                   float *out, cudaStream_t s);
packsell_status inv_diag_impl(const Matrix &A, double *out, cudaStream_t s);
packsell_status storage_rows_impl(const Matrix &A, int32_t *rows, cudaStream_t s);
packsell_status pattern_outer_f64_impl(const Matrix &A, double alpha, const double *u,
                                       const double *v, double *out, cudaStream_t s);

// batch.cu
struct Batch;
packsell_status batch_create(int count, const Matrix *const *A, const float *const *x,
                             float *const *y, cudaStream_t s, Batch **out);
packsell_status batch_spmv(const Batch &B, cudaStream_t s);
packsell_status batch_create_mm(int count, const Matrix *const *A, int k, const float *const *X,
                                const int64_t *ldx, float *const *Y, const int64_t *ldy,
                                cudaStream_t s, Batch **out);
packsell_status batch_spmm(const Batch &B, cudaStream_t s);
void batch_free(Batch *B);
void batch_stats(const Batch &B, int64_t *words, int64_t *bytes, int32_t *items);

// solve.cu
size_t solve_workspace_bytes(int64_t n, int m_in, int has_m, int max_iters);
packsell_status solve_impl(const Matrix *A64, const Matrix *Ain, const double *inv_diag,
                           const double *b, double *x, const packsell_solve_opts &o, void *work,
                           size_t work_bytes, double *h_hist, packsell_solve_result *res,
                           cudaStream_t caller, bool noalloc = false);
packsell_status solve_noalloc(const Matrix *A64, const Matrix *Ain, const double *inv_diag,
                              const double *b, double *x, const packsell_solve_opts &o,
                              double *h_hist, packsell_solve_result *res, cudaStream_t s);
size_t noalloc_capacity();

// f3r.cu
packsell_status f3r_impl(const Matrix *A1, const Matrix *A2, const Matrix *A3, const double *b,
                         double *x, const packsell_f3r_opts &o, packsell_solve_result *res,
                         cudaStream_t s);

// solver support (spmv.cu): SpMV fused with a deterministic dot reduction
struct Red;
int reduce_blocks();
int spmv_dot_blocks(const Matrix &A);
packsell_status spmv_dot_f32(const Matrix &A, const float *x, float *y, const Red &red,
                             cudaStream_t s);
packsell_status spmv_dot_f64(const Matrix &A, const double *x, double *y, const double *b,
                             const Red &red, cudaStream_t s);

// w64.cu: products on 64-bit words
packsell_status spmv_w64_impl(const Matrix &A, const double *x, double *y, cudaStream_t s);
packsell_status spmv_dot_w64(const Matrix &A, const double *x, double *y, const double *b,
                             const Red &red, unsigned grid, cudaStream_t s);
packsell_status inv_diag_w64(const Matrix &A, double *out, cudaStream_t s);

}  // namespace packsell

#define PS_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return packsell::cuda_fail(e_, #call);   \
    } while (0)

#define PS_LAUNCH_CHECK(where)                                          \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return packsell::cuda_fail(e_, where);   \
    } while (0)
