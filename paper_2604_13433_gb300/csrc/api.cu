// C ABI entry points: argument checks, error text, matrix lifetime, export.
#include <cuda_runtime.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.h"

namespace packsell {

static thread_local std::string g_last_error;

packsell_status fail(packsell_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

packsell_status cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PACKSELL_ERR_NO_MEMORY : PACKSELL_ERR_CUDA;
}

void clear_error() { g_last_error.clear(); }

int64_t matrix_bytes(const Matrix &A) {
    int64_t b = 8 * (A.n_slices + 1) + (int64_t)A.perm_bytes * A.n;
    if (is_w16(A.p.format)) b += 2 * A.n_words;
    else if (is_w64(A.p.format)) b += 8 * A.n_words;
    else if (is_sell16(A.p.format)) b += 6 * A.n_words;
    else if (is_packed(A.p.format) || is_fixed(A.p.format)) b += 4 * A.n_words;
    else b += (A.p.format == PACKSELL_FMT_SELL_F64 ? 12 : 8) * A.n_words;
    if (A.rowptr) b += 8 * (A.n + 1);
    return b;
}

void destroy_matrix(Matrix *A);

// Readers of the bounds-check counters, one per translation unit (registered
// while the library loads; empty in the regular build).
static std::vector<ChecksReader> &checks_readers() {
    static std::vector<ChecksReader> r;
    return r;
}

void register_checks_reader(ChecksReader r) { checks_readers().push_back(r); }

// Sum and clear every unit's counters: PACKSELL_ERR_CHECK if any access was
// skipped, else OK.
static packsell_status read_checks() {
    unsigned long long total = 0;
    long long first = -1;
    for (ChecksReader r : checks_readers()) {
        unsigned long long c = 0;
        long long f = 0;
        PS_CUDA(r(&c, &f));
        if (c && first < 0) first = f;
        total += c;
    }
    if (total)
        return fail(PACKSELL_ERR_CHECK, "packsell_check_status: " + std::to_string(total) +
                                            " out-of-range accesses skipped (first index " +
                                            std::to_string(first) + ")");
    return PACKSELL_OK;
}

// The SpMV of a matrix: 16-bit words have their own kernel.
packsell_status spmv_route(const Matrix &A, const float *x, float *y, cudaStream_t s) {
    return is_w16(A.p.format) ? spmv_w16_impl(A, x, y, s) : spmv_impl(A, x, y, s);
}

// Calls that take neither 16-bit words nor FP16 SELL.
packsell_status no_w16(const Matrix &A, const char *what) {
    if (is_w16(A.p.format))
        return fail(PACKSELL_ERR_INVALID_ARG, std::string(what) + ": not available for 16-bit words");
    if (is_sell16(A.p.format))
        return fail(PACKSELL_ERR_INVALID_ARG, std::string(what) + ": not available for FP16 SELL");
    if (is_fixed(A.p.format))
        return fail(PACKSELL_ERR_INVALID_ARG, std::string(what) + ": not available for fixed point");
    if (is_w64(A.p.format))
        return fail(PACKSELL_ERR_INVALID_ARG,
                    std::string(what) + ": not available for 64-bit words (FP64 products only)");
    return PACKSELL_OK;
}

}  // namespace packsell

using namespace packsell;

namespace {
constexpr uint64_t kMagic = 0x324C4C4553434B50ull;  // "PKCSELL2"

struct BlobHeader {
    uint64_t magic;
    int64_t n, m, nnz;
    packsell_params p;
    int64_t n_slices, n_words, n_dummies, n_pad;
    int32_t max_width, perm_bytes;
    int32_t value_exp, reserved;  // fixed point's 2^s; 0
};

// Bytes per stored word of each format in the blob: the word, or value and
// column of plain SELL.
inline size_t blob_word_bytes(int fmt) {
    if (is_w16(fmt)) return 2;
    if (is_w64(fmt)) return 8;
    if (is_packed(fmt) || is_fixed(fmt)) return 4;
    if (is_sell16(fmt)) return 6;
    return fmt == PACKSELL_FMT_SELL_F64 ? 12 : 8;
}

inline cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

inline const Matrix *M(const packsell_matrix *A) { return reinterpret_cast<const Matrix *>(A); }
}  // namespace

extern "C" {

void packsell_params_default(packsell_params *p) {
    if (!p) return;
    p->C = 32;
    p->sigma = 256;
    p->D = 15;
    p->format = PACKSELL_FMT_FP16;
    p->explicit_perm = 0;
    p->keep_rowptr = 0;
    p->k_left = -1;
}

const char *packsell_version(void) { return "packsell-gb300 0.1 (sm_103a)"; }

int32_t packsell_checks_build(void) {
#ifdef PACKSELL_CHECKS
    return 1;
#else
    return 0;
#endif
}

const char *packsell_last_error(void) { return g_last_error.c_str(); }

packsell_status packsell_encode(const packsell_params *params, int64_t n, int64_t m, int64_t nnz,
                                const int64_t *rowptr, const int32_t *col, const void *val,
                                int32_t val_is_f64, void *stream, packsell_matrix **out) {
    clear_error();
    if (!params) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_encode: params is NULL");
    Matrix *A = nullptr;
    packsell_status st = encode_impl(*params, n, m, nnz, rowptr, col, val, val_is_f64,
                                     as_stream(stream), &A);
    if (out) *out = reinterpret_cast<packsell_matrix *>(A);
    return st;
}

packsell_status packsell_destroy(packsell_matrix *A) {
    clear_error();
    if (!A) return PACKSELL_OK;
    cudaDeviceSynchronize();
    destroy_matrix(reinterpret_cast<Matrix *>(A));
    return PACKSELL_OK;
}

packsell_status packsell_get_info(const packsell_matrix *Ah, packsell_info *info) {
    clear_error();
    if (!Ah || !info) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_get_info: NULL argument");
    const Matrix &A = *M(Ah);
    memset(info, 0, sizeof(*info));
    info->n = A.n;
    info->m = A.m;
    info->nnz = A.nnz;
    info->params = A.p;
    info->n_slices = A.n_slices;
    info->n_words = A.n_words;
    info->n_dummies = A.n_dummies;
    info->n_pad = A.n_pad;
    info->max_width = A.max_width;
    info->perm_bytes = A.perm_bytes;
    info->bytes = matrix_bytes(A);
    info->pack = A.pack;
    info->val = A.val;
    info->col = A.col;
    info->offset = A.offset;
    info->perm = A.perm;
    info->value_exp = A.value_exp;
    return PACKSELL_OK;
}

packsell_status packsell_export(const packsell_matrix *Ah, void *h_blob, size_t *bytes,
                                void *stream) {
    clear_error();
    if (!Ah || !bytes) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_export: NULL argument");
    const Matrix &A = *M(Ah);
    const size_t vb = blob_word_bytes(A.p.format);
    size_t need = sizeof(BlobHeader) + 8 * (A.n_slices + 1) + (size_t)A.perm_bytes * A.n +
                  vb * (size_t)A.n_words;
    if (!h_blob) {
        *bytes = need;
        return PACKSELL_OK;
    }
    if (*bytes < need) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_export: blob too small");
    BlobHeader h{};
    h.magic = kMagic;
    h.n = A.n;
    h.m = A.m;
    h.nnz = A.nnz;
    h.p = A.p;
    h.p.keep_rowptr = 0;
    h.n_slices = A.n_slices;
    h.n_words = A.n_words;
    h.n_dummies = A.n_dummies;
    h.n_pad = A.n_pad;
    h.max_width = A.max_width;
    h.perm_bytes = A.perm_bytes;
    h.value_exp = A.value_exp;
    char *dst = (char *)h_blob;
    memcpy(dst, &h, sizeof(h));
    dst += sizeof(h);
    cudaStream_t s = as_stream(stream);
    PS_CUDA(cudaMemcpyAsync(dst, A.offset, 8 * (A.n_slices + 1), cudaMemcpyDeviceToHost, s));
    dst += 8 * (A.n_slices + 1);
    if (A.perm_bytes) {
        PS_CUDA(cudaMemcpyAsync(dst, A.perm, (size_t)A.perm_bytes * A.n, cudaMemcpyDeviceToHost, s));
        dst += (size_t)A.perm_bytes * A.n;
    }
    if (is_w16(A.p.format)) {
        PS_CUDA(cudaMemcpyAsync(dst, A.pack16, 2 * (size_t)A.n_words, cudaMemcpyDeviceToHost, s));
    } else if (is_w64(A.p.format)) {
        PS_CUDA(cudaMemcpyAsync(dst, A.pack64, 8 * (size_t)A.n_words, cudaMemcpyDeviceToHost, s));
    } else if (is_packed(A.p.format) || is_fixed(A.p.format)) {
        PS_CUDA(cudaMemcpyAsync(dst, A.pack, 4 * (size_t)A.n_words, cudaMemcpyDeviceToHost, s));
    } else {
        const size_t eb = vb - 4;
        PS_CUDA(cudaMemcpyAsync(dst, A.val, eb * (size_t)A.n_words, cudaMemcpyDeviceToHost, s));
        dst += eb * (size_t)A.n_words;
        PS_CUDA(cudaMemcpyAsync(dst, A.col, 4 * (size_t)A.n_words, cudaMemcpyDeviceToHost, s));
    }
    PS_CUDA(cudaStreamSynchronize(s));
    *bytes = need;
    return PACKSELL_OK;
}

packsell_status packsell_import(const void *h_blob, size_t bytes, void *stream,
                                packsell_matrix **out) {
    clear_error();
    if (!h_blob || !out || bytes < sizeof(BlobHeader))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_import: bad arguments");
    *out = nullptr;
    BlobHeader h;
    memcpy(&h, h_blob, sizeof(h));
    const packsell_params &p = h.p;
    const bool fmt_ok = is_packed(p.format) || is_sell(p.format) || is_w16(p.format) ||
                        is_sell16(p.format) || is_fixed(p.format) || is_w64(p.format);
    // delta bits each word format accepts (packsell_encode's own ranges)
    const bool d_ok = is_packed(p.format)  ? (p.D >= 1 && p.D <= 22)
                      : is_fixed(p.format) ? (p.D >= 6 && p.D <= 22)
                      : is_w16(p.format)   ? p.D == 7
                      : is_w64(p.format)   ? (p.D >= 1 && p.D <= 31)
                                           : true;
    if (h.magic != kMagic || !fmt_ok || !d_ok || h.n < 0 || h.n >= (1ll << 31) || h.m < 0 ||
        h.m >= (1ll << 31) || p.C < 1 || p.C > 1024 || p.sigma < 1 || p.sigma > 65536 ||
        h.n_slices != (h.n + p.C - 1) / p.C || h.n_words < 0 ||
        h.perm_bytes != (p.sigma == 1 ? 0 : (p.sigma <= 256 ? 1 : 2)) || p.k_left < 0 ||
        (is_fixed(p.format) ? (h.value_exp < -1100 || h.value_exp > 1100) : h.value_exp != 0))
        return fail(PACKSELL_ERR_CORRUPT, "packsell_import: bad header");
    const size_t vb = blob_word_bytes(p.format);
    size_t need = sizeof(BlobHeader) + 8 * (h.n_slices + 1) + (size_t)h.perm_bytes * h.n +
                  vb * (size_t)h.n_words;
    if (bytes < need) return fail(PACKSELL_ERR_CORRUPT, "packsell_import: blob truncated");
    const char *src = (const char *)h_blob + sizeof(h);
    const int64_t *offs = (const int64_t *)src;
    if (offs[0] != 0 || offs[h.n_slices] != h.n_words)
        return fail(PACKSELL_ERR_CORRUPT, "packsell_import: offsets do not match the word count");
    int64_t widest = 0;
    for (int64_t k = 0; k < h.n_slices; ++k) {
        if (offs[k + 1] < offs[k] || (offs[k + 1] - offs[k]) % p.C)
            return fail(PACKSELL_ERR_CORRUPT, "packsell_import: offsets not C-aligned");
        widest = std::max<int64_t>(widest, (offs[k + 1] - offs[k]) / p.C);
    }
    // kernels size their rounds by the widest slice: it must be the offsets' own
    if (widest != h.max_width)
        return fail(PACKSELL_ERR_CORRUPT, "packsell_import: widest slice does not match the offsets");

    Matrix *A = new Matrix();
    A->n = h.n;
    A->m = h.m;
    A->nnz = h.nnz;
    A->p = p;
    A->p.keep_rowptr = 0;
    A->n_slices = h.n_slices;
    A->n_words = h.n_words;
    A->n_dummies = h.n_dummies;
    A->n_pad = h.n_pad;
    A->max_width = h.max_width;
    A->perm_bytes = h.perm_bytes;
    A->value_exp = h.value_exp;
    cudaGetDevice(&A->device);
    cudaStream_t s = as_stream(stream);
    auto bail = [&](packsell_status st) {
        destroy_matrix(A);
        return st;
    };
    if (cudaMalloc(&A->offset, 8 * (h.n_slices + 1)) != cudaSuccess ||
        (h.perm_bytes && cudaMalloc(&A->perm, (size_t)h.perm_bytes * h.n) != cudaSuccess))
        return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_import: allocation"));
    if (cudaMemcpyAsync(A->offset, src, 8 * (h.n_slices + 1), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail(fail(PACKSELL_ERR_CUDA, "packsell_import: copy"));
    src += 8 * (h.n_slices + 1);
    if (h.perm_bytes) {
        if (cudaMemcpyAsync(A->perm, src, (size_t)h.perm_bytes * h.n, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return bail(fail(PACKSELL_ERR_CUDA, "packsell_import: copy"));
        src += (size_t)h.perm_bytes * h.n;
    }
    size_t nw = (size_t)std::max<int64_t>(h.n_words, 1);
    if (is_w64(p.format)) {
        if (cudaMalloc(&A->pack64, 8 * nw) != cudaSuccess)
            return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_import: allocation"));
        if (cudaMemcpyAsync(A->pack64, src, 8 * (size_t)h.n_words, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return bail(fail(PACKSELL_ERR_CUDA, "packsell_import: copy"));
    } else if (is_w16(p.format)) {
        if (cudaMalloc(&A->pack16, 2 * nw) != cudaSuccess)
            return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_import: allocation"));
        if (cudaMemcpyAsync(A->pack16, src, 2 * (size_t)h.n_words, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return bail(fail(PACKSELL_ERR_CUDA, "packsell_import: copy"));
    } else if (is_packed(p.format) || is_fixed(p.format)) {
        if (cudaMalloc(&A->pack, 4 * (nw + kWordTail)) != cudaSuccess)
            return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_import: allocation"));
        if (cudaMemcpyAsync(A->pack, src, 4 * (size_t)h.n_words, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return bail(fail(PACKSELL_ERR_CUDA, "packsell_import: copy"));
    } else {
        const size_t eb = vb - 4;
        if (cudaMalloc(&A->val, eb * nw) != cudaSuccess || cudaMalloc(&A->col, 4 * nw) != cudaSuccess)
            return bail(fail(PACKSELL_ERR_NO_MEMORY, "packsell_import: allocation"));
        if (cudaMemcpyAsync(A->val, src, eb * (size_t)h.n_words, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(A->col, src + eb * (size_t)h.n_words, 4 * (size_t)h.n_words,
                            cudaMemcpyHostToDevice, s) != cudaSuccess)
            return bail(fail(PACKSELL_ERR_CUDA, "packsell_import: copy"));
    }
    packsell_status st = validate_impl(*A, s, "packsell_import");
    if (st != PACKSELL_OK) return bail(st);
    st = plan_spmv(*A, s);
    if (st != PACKSELL_OK) return bail(st);
    *out = reinterpret_cast<packsell_matrix *>(A);
    return PACKSELL_OK;
}

packsell_status packsell_set_spmv_variant(packsell_matrix *A, int32_t variant) {
    clear_error();
    if (!A || variant < 0 || variant > PACKSELL_SPMV_VARIANTS)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_set_spmv_variant: bad argument");
    Matrix *m = reinterpret_cast<Matrix *>(A);
    if (variant == 11 || variant == 14) {
        if (!(variant == 11 ? m->csr_items : m->split_items))
            return fail(PACKSELL_ERR_INVALID_ARG, "packsell_set_spmv_variant: variant " +
                                                      std::to_string(variant) +
                                                      " needs a PackSELL matrix with C = 1");
        m->variant = variant;
        return PACKSELL_OK;
    }
    if (variant >= 2 && variant <= 4 && !m->part[variant - 2])
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_set_spmv_variant: bulk-staged needs a PackSELL matrix with C = 32");
    const bool fixed13 = variant == 13 && is_fixed(m->p.format);  // fixed point runs variant 13 too
    if (variant >= 5 && ((!is_packed(m->p.format) && !fixed13) || m->p.C != 32))
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_set_spmv_variant: variants 5-10, 12 and 13 need a PackSELL matrix with C = 32");
    if (variant == 12 && m->max_width > 16)
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_set_spmv_variant: variant 12 needs slices of at most 16 words");
    if (variant >= 9 && variant <= 10 && !m->stage[variant - 9].part)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_set_spmv_variant: stage plan unavailable");
    m->variant = variant;
    return PACKSELL_OK;
}

namespace packsell {
// Time every SpMV variant available for the matrix (`reps` launches each
// after three untimed ones, CUDA events on `s`); the fastest in *best_var.
static packsell_status tune_variants(Matrix *m, const float *x, float *y, int reps, float *h_times,
                                     cudaStream_t s, int *best_var, float *best_ms_out) {
    const int nvar = PACKSELL_SPMV_VARIANTS;
    if (h_times)
        for (int v = 0; v < nvar; ++v) h_times[v] = 0.f;
    cudaEvent_t e0, e1;
    PS_CUDA(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(PACKSELL_ERR_CUDA, "packsell_tune_spmv: event");
    }
    const int keep = m->variant;
    int best = m->auto_variant;
    float best_ms = 0.f;
    packsell_status st = PACKSELL_OK;
    for (int var = 1; var <= nvar && st == PACKSELL_OK; ++var) {
        // fixed point: the thread-per-row kernel and variant 13
        if (var >= 2 && !is_packed(m->p.format) && !(is_fixed(m->p.format) && var == 13)) continue;
        if (var == 11 && !m->csr_items) continue;
        if (var == 14 && !m->split_items) continue;
        if (((var >= 5 && var <= 10) || var == 12 || var == 13) && m->p.C != 32) continue;
        if (var == 12 && m->max_width > 16) continue;
        if (var >= 9 && var <= 10 && !m->stage[var - 9].part) continue;
        if (var >= 2 && var <= 4 && !m->part[var - 2]) continue;
        m->variant = var;
        for (int r = 0; r < 3 && st == PACKSELL_OK; ++r) st = spmv_route(*m, x, y, s);
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == PACKSELL_OK; ++r) st = spmv_route(*m, x, y, s);
        cudaEventRecord(e1, s);
        if (st != PACKSELL_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fail(PACKSELL_ERR_CUDA, "packsell_tune_spmv: timing failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        if (h_times) h_times[var - 1] = ms;
        if (best_ms == 0.f || ms < best_ms) {
            best_ms = ms;
            best = var;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    m->variant = keep;
    if (st == PACKSELL_OK) {
        m->auto_variant = best;
        if (best_var) *best_var = best;
        if (best_ms_out) *best_ms_out = best_ms;
    }
    return st;
}
}  // namespace packsell

packsell_status packsell_tune_spmv(packsell_matrix *A, const float *x, float *y, int32_t reps,
                                   float *h_times, void *stream) {
    clear_error();
    if (!A || (M(A)->m > 0 && !x) || (M(A)->n > 0 && !y) || reps < 1)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_tune_spmv: bad argument");
    if (is_f64_op(M(A)->p.format))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_tune_spmv: FP64 matrices have one product");
    return tune_variants(reinterpret_cast<Matrix *>(A), x, y, reps, h_times, as_stream(stream),
                         nullptr, nullptr);
}

packsell_status packsell_quantize(int32_t format, int32_t D, int64_t n, const void *val,
                                  int32_t val_is_f64, uint32_t *field, int64_t *h_bad_index,
                                  void *stream) {
    clear_error();
    if (n < 0 || (n > 0 && (!val || !field)))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_quantize: bad argument");
    return quantize_impl(format, D, n, val, val_is_f64, field, h_bad_index, as_stream(stream));
}

packsell_status packsell_tune_format(int64_t n, int64_t m, int64_t nnz, const int64_t *rowptr,
                                     const int32_t *col, const void *val, int32_t val_is_f64,
                                     double max_error, const float *x, float *y, int32_t reps,
                                     packsell_params *best, packsell_format_trial *h_trials,
                                     int32_t max_trials, int32_t *n_trials, void *stream) {
    clear_error();
    if (n < 1 || m < 1 || nnz < 0 || !rowptr || (nnz > 0 && (!col || !val)) || !x || !y ||
        !best || reps < 1 || !(max_error > 0.0) || (max_trials > 0 && !h_trials) || max_trials < 0)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_tune_format: bad argument");
    cudaStream_t s = as_stream(stream);
    // value formats, most value bits last; layouts of §3 (SELL-C-sigma) and CSR order
    struct Fmt { int fmt, D; };
    const Fmt fmts[] = {{PACKSELL_FMT_FP16, 15}, {PACKSELL_FMT_E8MY, 15}, {PACKSELL_FMT_E8MY, 11},
                        {PACKSELL_FMT_E8MY, 7},  {PACKSELL_FMT_E8MY, 3},  {PACKSELL_FMT_E8MY, 1}};
    struct Lay { int C, sigma; };
    const Lay lays[] = {{32, 256}, {32, 65536}, {1, 1}};
    const double u = 0x1p-24;
    double err[6];
    bool ok[6];
    for (int f = 0; f < 6; ++f) {
        double e[3];
        int64_t maxlen = 0;
        int bad = 0;
        const packsell_status st = format_error_impl(n, rowptr, val, val_is_f64, fmts[f].fmt, fmts[f].D,
                                                     s, e, &maxlen, &bad);
        if (st != PACKSELL_OK) return st;
        // |y_hat - A x|_i <= (sum_j |a_ij - q(a_ij)| + gamma_w sum_j |q(a_ij)|) ||x||_inf with
        // w <= 2 nnz_i stored words (one dummy per nonzero at most, 32-bit words)
        const double w = 2.0 * (double)std::max<int64_t>(maxlen, 1);
        const double gw = w * u / (1.0 - w * u);
        err[f] = e[2] > 0.0 ? (e[0] + gw * e[1]) / e[2] : 0.0;
        ok[f] = bad == 0 && err[f] <= max_error;
    }
    int count = 0, best_i = -1;
    double best_ms = 0.0;
    packsell_params bp{};
    for (const Lay &L : lays) {
        for (int f = 0; f < 6; ++f) {
            packsell_params p;
            packsell_params_default(&p);
            p.C = L.C;
            p.sigma = L.sigma;
            p.D = fmts[f].D;
            p.format = fmts[f].fmt;
            packsell_format_trial t{};
            t.params = p;
            t.error = err[f];
            t.admissible = ok[f] ? 1 : 0;
            if (ok[f]) {
                Matrix *Am = nullptr;
                packsell_status st = encode_impl(p, n, m, nnz, rowptr, col, val, val_is_f64, s, &Am);
                if (st != PACKSELL_OK) return st;
                int var = 0;
                float ms = 0.f;
                st = tune_variants(Am, x, y, reps, nullptr, s, &var, &ms);
                t.variant = var;
                t.ms = ms;
                t.n_words = Am->n_words;
                t.bytes = 4.0 * (double)Am->n_words + 8.0 * (double)(Am->n_slices + 1) +
                          (double)Am->perm_bytes * (double)n + 4.0 * (double)(m + n);
                cudaStreamSynchronize(s);
                destroy_matrix(Am);
                if (st != PACKSELL_OK) return st;
                if (best_i < 0 || ms < best_ms) {
                    best_i = count;
                    best_ms = ms;
                    bp = p;
                }
            }
            if (count < max_trials) h_trials[count] = t;
            ++count;
        }
    }
    if (n_trials) *n_trials = std::min(count, max_trials);
    if (best_i < 0)
        return fail(PACKSELL_ERR_RANGE, "packsell_tune_format: no format meets the error ceiling "
                                        "(the finest, E8M21, bounds it by " +
                                            std::to_string(err[5]) + ")");
    *best = bp;
    return PACKSELL_OK;
}

packsell_status packsell_set_wait_limit(int64_t polls) {
    clear_error();
    set_data_wait_limit(polls < 0 ? kWaitLimit
                                  : (uint32_t)std::min<int64_t>(polls, (int64_t)UINT32_MAX));
    return PACKSELL_OK;
}

packsell_status packsell_validate(const packsell_matrix *A, void *stream) {
    clear_error();
    if (!A) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_validate: NULL matrix");
    return validate_impl(*M(A), as_stream(stream), "packsell_validate");
}

packsell_status packsell_check_status(const packsell_matrix *A, void *stream) {
    clear_error();
    if (!A) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_check_status: NULL matrix");
    const Matrix *m = M(A);
    if (!m->status) return PACKSELL_OK;
    DevStatus h{};
    cudaStream_t s = as_stream(stream);
    PS_CUDA(cudaMemcpyAsync(&h, m->status, sizeof(h), cudaMemcpyDeviceToHost, s));
    PS_CUDA(cudaMemsetAsync(m->status, 0, sizeof(DevStatus), s));
    PS_CUDA(cudaStreamSynchronize(s));
    if (h.code)
        return fail((packsell_status)h.code,
                    "packsell_check_status: a bounded wait ran out in warp " + std::to_string(h.index));
    return read_checks();
}

packsell_status packsell_spmv(const packsell_matrix *A, const float *x, float *y, void *stream) {
    clear_error();
    if (!A || (M(A)->m > 0 && !x) || (M(A)->n > 0 && !y))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv: NULL argument");
    return spmv_route(*M(A), x, y, as_stream(stream));
}

packsell_status packsell_spmv_f64(const packsell_matrix *A, const double *x, double *y,
                                  void *stream) {
    clear_error();
    if (!A || (M(A)->m > 0 && !x) || (M(A)->n > 0 && !y))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_f64: NULL argument");
    return spmv_f64_impl(*M(A), x, y, as_stream(stream));
}

packsell_status packsell_spmm(const packsell_matrix *A, int32_t k, const float *X, int64_t ldx,
                              float *Y, int64_t ldy, void *stream) {
    clear_error();
    if (!A || (M(A)->m > 0 && !X) || (M(A)->n > 0 && !Y))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmm: NULL argument");
    if (no_w16(*M(A), "packsell_spmm") != PACKSELL_OK) return PACKSELL_ERR_INVALID_ARG;
    return spmm_impl(*M(A), k, X, ldx, Y, ldy, as_stream(stream));
}

packsell_status packsell_spmv_transpose(const packsell_matrix *A, const float *dy, float *dx,
                                        void *stream) {
    clear_error();
    if (!A || (M(A)->n > 0 && !dy) || (M(A)->m > 0 && !dx))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_transpose: NULL argument");
    if (no_w16(*M(A), "packsell_spmv_transpose") != PACKSELL_OK) return PACKSELL_ERR_INVALID_ARG;
    return spmv_t_impl(*M(A), dy, dx, as_stream(stream));
}

packsell_status packsell_pattern_outer(const packsell_matrix *A, float alpha, const float *u,
                                       const float *v, float *out, void *stream) {
    clear_error();
    if (!A || (M(A)->nnz > 0 && (!u || !v || !out)))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pattern_outer: NULL argument");
    if (no_w16(*M(A), "packsell_pattern_outer") != PACKSELL_OK) return PACKSELL_ERR_INVALID_ARG;
    return pattern_outer_impl(*M(A), alpha, u, v, out, as_stream(stream));
}

packsell_status packsell_spmv_backward(const packsell_matrix *A, const float *x, const float *dy,
                                       float *dx, float *dval, void *stream) {
    clear_error();
    if (!A || (M(A)->n > 0 && !dy) || (dval && M(A)->m > 0 && !x))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_backward: NULL argument");
    if (no_w16(*M(A), "packsell_spmv_backward") != PACKSELL_OK) return PACKSELL_ERR_INVALID_ARG;
    if (dval && !M(A)->rowptr)  // checked before dx is written
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_spmv_backward: dval needs a matrix encoded with keep_rowptr");
    cudaStream_t s = as_stream(stream);
    if (dx) {
        const packsell_status st = spmv_t_impl(*M(A), dy, dx, s);
        if (st != PACKSELL_OK) return st;
    }
    if (dval) return pattern_outer_impl(*M(A), 1.0f, dy, x, dval, s);
    return PACKSELL_OK;
}

packsell_status packsell_inv_diag(const packsell_matrix *A, double *out, void *stream) {
    clear_error();
    if (!A || (M(A)->n > 0 && !out)) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_inv_diag: NULL argument");
    return inv_diag_impl(*M(A), out, as_stream(stream));
}

packsell_status packsell_spmv_host(const packsell_matrix *A, const float *h_x, float *h_y,
                                   float *d_x, float *d_y, void *stream) {
    clear_error();
    if (!A) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_host: NULL matrix");
    const Matrix &m = *M(A);
    if ((m.m > 0 && (!h_x || !d_x)) || (m.n > 0 && (!h_y || !d_y)))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_host: NULL buffer");
    if (is_f64_op(m.p.format))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_host: FP64 matrices need packsell_spmv_f64");
    cudaStream_t s = as_stream(stream);
    if (m.m > 0)
        PS_CUDA(cudaMemcpyAsync(d_x, h_x, sizeof(float) * (size_t)m.m, cudaMemcpyHostToDevice, s));
    const packsell_status st = spmv_route(m, d_x, d_y, s);
    if (st != PACKSELL_OK) return st;
    if (m.n > 0)
        PS_CUDA(cudaMemcpyAsync(h_y, d_y, sizeof(float) * (size_t)m.n, cudaMemcpyDeviceToHost, s));
    return PACKSELL_OK;
}

packsell_status packsell_spmv_x16(const packsell_matrix *A, const uint16_t *x, uint16_t *y,
                                  void *stream) {
    clear_error();
    if (!A || (M(A)->m > 0 && !x) || (M(A)->n > 0 && !y))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_spmv_x16: NULL argument");
    return spmv_x16_impl(*M(A), x, y, as_stream(stream));
}

packsell_status packsell_storage_rows(const packsell_matrix *A, int32_t *rows, void *stream) {
    clear_error();
    if (!A || (M(A)->n > 0 && !rows))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_storage_rows: NULL argument");
    return storage_rows_impl(*M(A), rows, as_stream(stream));
}

packsell_status packsell_pattern_outer_f64(const packsell_matrix *A, double alpha,
                                           const double *u, const double *v, double *out,
                                           void *stream) {
    clear_error();
    if (!A || (M(A)->nnz > 0 && (!u || !v || !out)))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pattern_outer_f64: NULL argument");
    return pattern_outer_f64_impl(*M(A), alpha, u, v, out, as_stream(stream));
}

packsell_status packsell_batch_create(int32_t count, const packsell_matrix *const *A,
                                      const float *const *x, float *const *y, void *stream,
                                      packsell_batch **out) {
    clear_error();
    if (!out || !A || !x || !y || count < 1)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create: bad argument");
    *out = nullptr;
    Batch *B = nullptr;
    packsell_status st = batch_create(count, reinterpret_cast<const Matrix *const *>(A), x, y,
                                      as_stream(stream), &B);
    *out = reinterpret_cast<packsell_batch *>(B);
    return st;
}

packsell_status packsell_batch_spmv(const packsell_batch *B, void *stream) {
    clear_error();
    if (!B) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_spmv: NULL plan");
    return batch_spmv(*reinterpret_cast<const Batch *>(B), as_stream(stream));
}

packsell_status packsell_batch_create_spmm(int32_t count, const packsell_matrix *const *A, int32_t k,
                                           const float *const *X, const int64_t *ldx,
                                           float *const *Y, const int64_t *ldy, void *stream,
                                           packsell_batch **out) {
    clear_error();
    if (!out || count < 1 || !A || !X || !Y)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_create_spmm: bad argument");
    Batch *B = nullptr;
    packsell_status st = batch_create_mm(count, reinterpret_cast<const Matrix *const *>(A), k, X, ldx,
                                         Y, ldy, as_stream(stream), &B);
    *out = reinterpret_cast<packsell_batch *>(B);
    return st;
}

packsell_status packsell_batch_spmm(const packsell_batch *B, void *stream) {
    clear_error();
    if (!B) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_spmm: NULL plan");
    return batch_spmm(*reinterpret_cast<const Batch *>(B), as_stream(stream));
}

packsell_status packsell_batch_info(const packsell_batch *B, int64_t *words, int64_t *bytes,
                                    int32_t *items) {
    clear_error();
    if (!B) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_batch_info: NULL plan");
    batch_stats(*reinterpret_cast<const Batch *>(B), words, bytes, items);
    return PACKSELL_OK;
}

packsell_status packsell_batch_destroy(packsell_batch *B) {
    clear_error();
    if (B) {
        cudaDeviceSynchronize();
        batch_free(reinterpret_cast<Batch *>(B));
    }
    return PACKSELL_OK;
}

size_t packsell_pcg_workspace_bytes(int64_t n, int32_t m_in, int32_t has_diag, int32_t max_iters) {
    if (n < 0 || m_in < 0 || max_iters < 0) return 0;
    return solve_workspace_bytes(n, m_in, has_diag, max_iters);
}

packsell_status packsell_pcg(const packsell_matrix *A_outer, const packsell_matrix *A_inner,
                             const double *inv_diag, const double *b, double *x,
                             const packsell_solve_opts *opts, void *work, size_t work_bytes,
                             double *h_hist, packsell_solve_result *result, void *stream) {
    clear_error();
    if (!A_outer || !opts) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg: NULL argument");
    return solve_impl(M(A_outer), A_inner ? M(A_inner) : nullptr, inv_diag, b, x, *opts, work,
                      work_bytes, h_hist, result, as_stream(stream));
}

packsell_status packsell_pcg_backward(const packsell_matrix *A_outer,
                                      const packsell_matrix *A_inner, const double *inv_diag,
                                      const double *x, const double *dL_dx, double *dL_db,
                                      double *dL_dA, const packsell_solve_opts *opts, void *work,
                                      size_t work_bytes, packsell_solve_result *result,
                                      void *stream) {
    clear_error();
    if (!A_outer || !opts || (M(A_outer)->n > 0 && (!x || !dL_dx || !dL_db)))
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg_backward: NULL argument");
    const Matrix &Ao = *M(A_outer);
    if (dL_dA && (Ao.p.format != PACKSELL_FMT_SELL_F64 || !Ao.rowptr))
        return fail(PACKSELL_ERR_INVALID_ARG,
                    "packsell_pcg_backward: dL_dA needs a SELL_F64 A_outer encoded with keep_rowptr");
    cudaStream_t s = as_stream(stream);
    if (Ao.n > 0) PS_CUDA(cudaMemsetAsync(dL_db, 0, sizeof(double) * (size_t)Ao.n, s));
    packsell_status st = solve_impl(&Ao, A_inner ? M(A_inner) : nullptr, inv_diag, dL_dx, dL_db,
                                    *opts, work, work_bytes, nullptr, result, s);
    if (st != PACKSELL_OK || !dL_dA) return st;
    return pattern_outer_f64_impl(Ao, -1.0, dL_db, x, dL_dA, s);
}

packsell_status packsell_pcg_noalloc(const packsell_matrix *A_outer,
                                     const packsell_matrix *A_inner, const double *inv_diag,
                                     const double *b, double *x,
                                     const packsell_solve_opts *opts, double *h_hist,
                                     packsell_solve_result *result, void *stream) {
    clear_error();
    if (!A_outer || !opts) return fail(PACKSELL_ERR_INVALID_ARG, "packsell_pcg_noalloc: NULL argument");
    return solve_noalloc(M(A_outer), A_inner ? M(A_inner) : nullptr, inv_diag, b, x, *opts,
                         h_hist, result, as_stream(stream));
}

}  // extern "C"

void packsell_f3r_opts_default(packsell_f3r_opts *o) {
    if (!o) return;
    o->rtol = 1e-9;
    o->m1 = 30;
    o->m2 = 8;
    o->m3 = 4;
    o->m4 = 2;
    o->max_iters = 300;
    o->omega = 1.0;
}

packsell_status packsell_f3r(const packsell_matrix *A_outer, const packsell_matrix *A_mid,
                             const packsell_matrix *A_low, const double *b, double *x,
                             const packsell_f3r_opts *opts, packsell_solve_result *result,
                             void *stream) {
    clear_error();
    if (!A_outer || !A_mid || !A_low || !opts)
        return fail(PACKSELL_ERR_INVALID_ARG, "packsell_f3r: NULL argument");
    return f3r_impl(M(A_outer), M(A_mid), M(A_low), b, x, *opts, result, as_stream(stream));
}
