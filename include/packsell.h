/*
 * packsell.h - C ABI of the PackSELL library for GB300 (sm_103a).
 *
 * PackSELL (arXiv 2604.13433) is sliced ELLPACK in which every 32-bit word
 * packs a delta-encoded column index and a matrix value:
 *   bit 0 (flag) = 1: bits 1..D hold the delta, bits D+1..31 hold the value
 *                     (V = 31 - D bits; W = V + D + 1 = 32, §4.2.1);
 *   bit 0 (flag) = 0: bits 1..31 hold the delta and there is no value
 *                     (a dummy, inserted before any nonzero whose delta does
 *                     not fit in D bits, or padding when the word is 0, §4.3).
 * Column indices are deltas from the previous nonzero of the row; the first
 * one is taken from the left offset of Eq. 4, which depends only on the block
 * of sigma rows the row belongs to (§4.1, §4.3). Rows are grouped into slices
 * of C rows stored column-major and padded to the slice's widest row; rows
 * are sorted by stored-word count inside blocks of sigma rows (SELL-C-sigma,
 * §3), the in-block permutation kept in `perm`.
 *
 * Conventions for every entry point:
 *  - Pointers are DEVICE pointers unless the name starts with h_ (host).
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream). Calls are
 *    asynchronous on it unless the comment says the call synchronises.
 *  - The caller owns every vector it passes; the library owns the device
 *    buffers inside a packsell_matrix until packsell_destroy.
 *  - Every call returns a packsell_status. On failure nothing is written to
 *    outputs except where stated, and packsell_last_error() describes it.
 *    No C++ exception crosses this boundary.
 *  - Index types: row and column counts below 2^31, nonzero and word counts
 *    in int64.
 *  - Inputs and outputs of one call must not overlap (x and y of a product,
 *    X and Y of packsell_spmm, the solver's b and x).
 *  - A matrix is read-only to the products, which may run on several
 *    streams at once. packsell_set_spmv_variant and packsell_tune_spmv change
 *    it and must not overlap other calls on the same matrix; kernels that
 *    report through the matrix's device status word share that word.
 *  - Some products (SpMV variant 13, FP32 SELL, 16-bit words, binary16
 *    vectors) are launched with programmatic dependent launch: they start
 *    while the previous kernel of the stream drains and read the matrix
 *    before they wait for it; x, y and every other buffer are touched only
 *    after it has completed. A matrix is complete when packsell_encode or
 *    packsell_import returns, and the caller must not write its arrays.
 */
#ifndef PACKSELL_H
#define PACKSELL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PACKSELL_VERSION_MAJOR 0
#define PACKSELL_VERSION_MINOR 1

typedef enum packsell_status {
    PACKSELL_OK = 0,
    PACKSELL_ERR_INVALID_ARG = 1,   /* bad size, parameter or pointer */
    PACKSELL_ERR_UNSORTED = 2,      /* CSR columns not strictly increasing in a row */
    PACKSELL_ERR_NONFINITE = 3,     /* a matrix value is Inf or NaN */
    PACKSELL_ERR_RANGE = 4,         /* value overflows the format, or column out of range */
    PACKSELL_ERR_CUDA = 5,          /* a CUDA runtime call failed */
    PACKSELL_ERR_NOT_CONVERGED = 6, /* solver hit its iteration limit */
    PACKSELL_ERR_BREAKDOWN = 7,     /* solver: p^T A p <= 0 or a non-finite residual */
    PACKSELL_ERR_NO_MEMORY = 8,     /* device allocation failed */
    PACKSELL_ERR_CORRUPT = 9,       /* imported data fails validation */
    PACKSELL_ERR_TIMEOUT = 10,      /* a kernel's bounded wait ran out (see
                                       packsell_check_status) */
    PACKSELL_ERR_CHECK = 11         /* bounds-check build only: a decoded index was
                                       out of range (see packsell_check_status) */
} packsell_status;

/* Value formats.
 * FP16  : IEEE binary16 in bits 16..31, round to nearest even; needs D = 15
 *         (§4.2.2, the paper's FP16 configuration).
 * E8MY  : 1 sign, 8 exponent, Y = 22 - D mantissa bits: an FP32 bit pattern
 *         with the low D+1 bits clear, rounded half away from zero on its
 *         grid (§4.2.2); D in [1, 22].
 * SELL_F32 / SELL_F64 : plain SELL-C-sigma (§3) with separate FP32 / FP64
 *         value and int32 column arrays: the baseline format and the FP64
 *         outer operator of the mixed-precision solver. D is ignored.
 * W16_E4M3: 16-bit words (W = 16, one of the other word sizes of §4.2.1):
 *         bit 0 flag, bits 1..7 delta (D = 7, needs D = 7), bits 8..15 an
 *         FP8 E4M3 value (OCP: 4 exponent bits, bias 7, 3 fraction bits,
 *         largest finite 448, round to nearest even; a value that rounds
 *         past 448 is PACKSELL_ERR_RANGE). A dummy holds a 15-bit delta, so a
 *         gap of 2^15 or more takes several dummies (each takes
 *         min(remaining delta, 2^15 - 1)). n_words counts 16-bit words.
 *         Supported by packsell_encode, packsell_spmv (one thread-per-row
 *         kernel; packsell_set_spmv_variant/tune_spmv see variant 1 only),
 *         packsell_spmv_host, packsell_get_info, packsell_storage_rows and
 *         packsell_export and packsell_import (2-byte words);
 *         the other calls return PACKSELL_ERR_INVALID_ARG for it.
 * FIXED : fixed point, an integer value format (§4.2.1 allows any V-bit
 *         format, integer ones included): bits D+1..31 hold a two's-
 *         complement integer q of V = 31 - D bits and the value is q * 2^s,
 *         with one exponent s for the matrix (packsell_info.value_exp): the
 *         smallest s with (2^(V-1) - 1) * 2^s >= max |a_ij|; q = a_ij / 2^s
 *         rounded half away from zero. Integer-valued matrices (stencils with
 *         integer coefficients) are exact. D in [6, 22] (V <= 25 bits, so
 *         every q converts to FP32 exactly). Supported by
 *         packsell_encode, packsell_spmv (the thread-per-row variant 1 and,
 *         with C = 32, variant 13, the default there; both summing the decoded values q * 2^s in
 *         stored order: the bits of the FP32 twin of the decoded matrix;
 *         packsell_tune_spmv times the two), packsell_spmv_host, packsell_get_info,
 *         packsell_storage_rows, packsell_export and packsell_import (the
 *         blob carries s); the other calls return PACKSELL_ERR_INVALID_ARG.
 * SELL_F16: plain SELL-C-sigma (§3) with binary16 values (round to nearest
 *         even, as FP16 PackSELL) in a uint16 array and int32 columns, 48
 *         bits per stored element: the FP16 SELL the paper compares
 *         PackSELL with (§5.1.1) and the FP16 operator of FP16-F3R (§5.2.1).
 *         Padding slots hold column -1 and add nothing, so a row's sum is the
 *         chain of the FP16 PackSELL kernels over the same values: the same
 *         bits. Supported by packsell_encode, packsell_spmv (one
 *         thread-per-row kernel), packsell_get_info, packsell_storage_rows,
 *         packsell_export, packsell_import and packsell_f3r; the other calls
 *         return PACKSELL_ERR_INVALID_ARG.
 * W64_E11MY: 64-bit words (W = 64, another word size of §4.2.1; V = 63 - D):
 *         bit 0 flag, bits 1..D delta, bits D+1..63 an E11MY value, i.e. a
 *         binary64 pattern (1 sign, 11 exponent bits, Y = 51 - D mantissa
 *         bits) with the low D+1 bits clear, rounded half away from zero on
 *         its grid (E8MY's rule carried over to binary64; a value that
 *         rounds past the largest finite double is PACKSELL_ERR_RANGE). A
 *         dummy holds a 63-bit delta, so one dummy covers any gap: the word
 *         counts, perm and offsets are those of 32-bit words with the same D.
 *         D in [1, 31]; n_words counts 64-bit words. The products are FP64
 *         (x, y and accumulation): the FP64 operator of the solvers at 8
 *         bytes per stored element (SELL_F64 takes 12). Supported by
 *         packsell_encode, packsell_spmv_f64, packsell_inv_diag,
 *         packsell_pcg and packsell_pcg_noalloc (as A_outer), packsell_f3r
 *         (as A_outer, and as A_mid and A_low of FP64-F3R),
 *         packsell_get_info, packsell_storage_rows, packsell_export and
 *         packsell_import; the other calls return PACKSELL_ERR_INVALID_ARG.
 */
typedef enum packsell_format {
    PACKSELL_FMT_FP16 = 1,
    PACKSELL_FMT_E8MY = 2,
    PACKSELL_FMT_SELL_F32 = 3,
    PACKSELL_FMT_SELL_F64 = 4,
    PACKSELL_FMT_W16_E4M3 = 5,
    PACKSELL_FMT_SELL_F16 = 6,
    PACKSELL_FMT_FIXED = 7,
    PACKSELL_FMT_W64_E11MY = 8
} packsell_format;

typedef struct packsell_params {
    int32_t C;             /* slice height in rows, 1..1024 (32 = one warp) */
    int32_t sigma;         /* sort block in rows, 1..65536 (1 = no sorting) */
    int32_t D;             /* delta bits (see packsell_format) */
    int32_t format;        /* a packsell_format */
    int32_t explicit_perm; /* 1: y is written in storage (sorted) row order,
                              0: y is written in the original row order */
    int32_t keep_rowptr;   /* 1: keep a copy of the CSR row pointer, needed to
                              write matrix gradients in CSR order */
    int64_t k_left;        /* lower bandwidth used in Eq. 4; -1 computes it */
} packsell_params;

/* Defaults (the parameters of §4.2-§4.3; C = 32, sigma = 256 and FP16 with
 * D = 15 are the paper's FP16 configuration, §5.1.1): C = 32, sigma = 256,
 * D = 15, FP16, implicit permutation,
 * keep_rowptr = 0, k_left = -1. */
void packsell_params_default(packsell_params *p);

typedef struct packsell_matrix packsell_matrix; /* opaque */

typedef struct packsell_info {
    int64_t n, m, nnz;
    packsell_params params; /* k_left filled in with the value used */
    int64_t n_slices;       /* ceil(n / C) */
    int64_t n_words;        /* stored words (PackSELL) or elements (SELL) */
    int64_t n_dummies;      /* dummy words (0 for SELL) */
    int64_t n_pad;          /* padding words, phantom rows of the last slice included */
    int32_t max_width;      /* widest slice, in words per row */
    int32_t perm_bytes;     /* bytes per perm entry: 0 (sigma = 1), 1 or 2 */
    int64_t bytes;          /* device bytes the matrix holds (all arrays) */
    /* device arrays (read-only views for tests and tools) */
    const uint32_t *pack;   /* 32-bit PackSELL words; NULL for SELL formats and for 16- and
                               64-bit words (packsell_export copies those) */
    const void *val;        /* SELL values (float or double), NULL for PackSELL */
    const int32_t *col;     /* SELL columns, NULL for PackSELL */
    const int64_t *offset;  /* n_slices + 1 word offsets of the slices */
    const void *perm;       /* n entries of perm_bytes, NULL when sigma = 1 */
    int32_t value_exp;      /* FIXED: the matrix exponent s (value = q * 2^s); 0 otherwise */
} packsell_info;

const char *packsell_version(void);

/* 1 when the library is the bounds-check build (compiled with
 * -DPACKSELL_CHECKS: libpacksell_checks.so), 0 otherwise. In that build
 * every gather of x (or a row of X) at a column decoded from the words, and
 * every write the decoded words steer (the transpose's scatter, the pattern
 * product's output), first checks its index against the array's length;
 * an index out of range skips the access and is counted, and
 * packsell_check_status reports the count. Plain SELL columns are stored,
 * not decoded, and are checked at encode and import instead. */
int32_t packsell_checks_build(void);

/* Message for the last failing call on this thread ("" if none). */
const char *packsell_last_error(void);

/* ---------------------------------------------------------------------- */
/* Encoding (§4.1 Eq. 2, §4.2, §4.3 Eq. 4, §3 sigma sort)                   */
/* ---------------------------------------------------------------------- */

/* Encode an n x m CSR matrix into PackSELL (or SELL) on the device.
 *   rowptr : int64 [n + 1], rowptr[0] = 0, rowptr[n] = nnz
 *   col    : int32 [nnz], strictly increasing within each row, in [0, m)
 *   val    : [nnz] float (val_is_f64 = 0) or double (val_is_f64 = 1)
 * Every step runs in CUDA kernels on `stream`: validation, lower bandwidth,
 * quantisation, word counts with dummies, the stable sigma sort (descending
 * stored words), slice widths, offsets, scatter. The call SYNCHRONISES the
 * stream (to size the word array, and at the end: the matrix is complete
 * when the call returns). Temporaries are stream-ordered
 * allocations freed before return. On success *out owns new device buffers.
 * Errors: INVALID_ARG (parameters, k_left below the bandwidth), UNSORTED,
 * RANGE (column out of range, value overflows the format), NONFINITE,
 * NO_MEMORY, CUDA. The encoded words are bit-identical to the paper's
 * definition for the same parameters. */
packsell_status packsell_encode(const packsell_params *params, int64_t n, int64_t m,
                                int64_t nnz, const int64_t *rowptr, const int32_t *col,
                                const void *val, int32_t val_is_f64, void *stream,
                                packsell_matrix **out);

/* Locality reordering before encoding (host arrays, host code; no device is
 * needed). §4.3 spends a dummy word wherever two consecutive columns of a
 * row are 2^D or more apart; the paper names a locality-improving ordering as
 * the way to fewer dummies and leaves it to future work (§7). Grouping rows
 * of similar length into the same slices also cuts SELL padding at small
 * sigma.
 *
 * packsell_reorder_rcm: reverse Cuthill-McKee order of the symmetrised
 * pattern A + A^T of a square CSR matrix (rowptr int64 [n+1], col int32
 * [nnz]; diagonal and duplicate entries ignored). Each connected component
 * starts from a pseudo-peripheral vertex (George-Liu search from a vertex of
 * least degree); a breadth-first search appends every vertex's unvisited
 * neighbours in increasing degree, ties by index; the order is reversed.
 * perm: int32 [n], out: perm[k] = the original row placed at position k.
 * Errors: INVALID_ARG (NULL, n out of range, bad rowptr), RANGE (a column
 * outside [0, n)), NO_MEMORY (host). */
packsell_status packsell_reorder_rcm(int64_t n, const int64_t *rowptr, const int32_t *col,
                                     int32_t *perm);

/* The reordering of §7's future work applied (§4.3 dummies depend on the
 * column order). B = P A P^T on host CSR arrays: row k of B is row perm[k] of A, column j
 * becomes inv(perm)[j], columns sorted within each row; values (float, or
 * double with val_is_f64 = 1) move with them. val and out_val are both NULL
 * (pattern only) or both set. out_rowptr int64 [n+1], out_col int32 [nnz],
 * out_val [nnz]. Solving with B: b_new = b[perm], x = x_new scattered back
 * (x[perm[k]] = x_new[k]). Errors: INVALID_ARG (NULL, perm not a
 * permutation), RANGE (a column outside [0, n)), NO_MEMORY (host). */
packsell_status packsell_permute_csr(int64_t n, const int64_t *rowptr, const int32_t *col,
                                     const void *val, int32_t val_is_f64, const int32_t *perm,
                                     int64_t *out_rowptr, int32_t *out_col, void *out_val);

/* Free the matrix (synchronises the device first). NULL is accepted.
 * Housekeeping with no counterpart in the paper. */
packsell_status packsell_destroy(packsell_matrix *A);

packsell_status packsell_get_info(const packsell_matrix *A, packsell_info *info);

/* Serialise the stored arrays of §4.3 (no counterpart in the paper) to a
 * host blob, for every format: a 112-byte header (magic "PKCSELL2"; n, m,
 * nnz; packsell_params; n_slices, n_words, n_dummies, n_pad; max_width,
 * perm_bytes, value_exp, 0), the n_slices + 1 offsets (int64), perm
 * (perm_bytes per row), then the words (uint32, or uint16 for W16_E4M3) or
 * the values (float, double or binary16) followed by the columns (int32).
 * With h_blob == NULL only *bytes is set. Synchronises `stream`. */
packsell_status packsell_export(const packsell_matrix *A, void *h_blob, size_t *bytes,
                                void *stream);

/* Rebuild a matrix (§4.3's arrays) from packsell_export's blob. The blob is validated on the
 * device (every row decoded, columns checked against m, value words, or the
 * FP16 SELL slots that are not padding, counted against nnz) before the call
 * returns; a bad blob gives CORRUPT and no matrix. Synchronises `stream`. */
packsell_status packsell_import(const void *h_blob, size_t bytes, void *stream,
                                packsell_matrix **out);

/* ---------------------------------------------------------------------- */
/* Products (§4.4 PackSELL SpMV; §3 SELL SpMV)                              */
/* ---------------------------------------------------------------------- */

/* y = A x (Eq. 1) by the §4.4 algorithm. x: float [m], y: float [n]
 * (original order, or storage order with explicit_perm). FP32
 * accumulation; variants 1-13 sum each row as one chain of fused
 * multiply-adds in stored order; variant 14 (CSR order, split rows) sums a
 * row in a fixed tree order. Every variant gives the same bits from run to
 * run. Words with flag 0 (dummies, padding) read no x and add nothing. Works
 * for PackSELL and SELL_F32 matrices. No allocation. */
packsell_status packsell_spmv(const packsell_matrix *A, const float *x, float *y,
                              void *stream);

/* y = A x (Eq. 1, the §4.4 algorithm) from and to host memory: enqueues on
 * `stream` the copy of h_x (float [m], host; pinned memory lets the copy run
 * asynchronously) into the
 * caller's device buffer d_x, packsell_spmv(A, d_x, d_y), and the copy of
 * d_y (float [n], device) into h_y (host). The caller owns all four buffers
 * and must keep them until the stream reaches the end of the call; h_y is
 * valid after the stream is synchronised. One cudaMemcpyAsync per copy; no
 * allocation. Errors: INVALID_ARG on a NULL buffer, CUDA if a copy cannot be
 * enqueued. */
packsell_status packsell_spmv_host(const packsell_matrix *A, const float *h_x, float *h_y,
                                   float *d_x, float *d_y, void *stream);

/* y = A x with binary16 vectors: the paper's FP16 SpMV configuration (§5.1.1,
 * x and y in FP16). x: uint16 [m], binary16 bit patterns, widened exactly to
 * FP32; each row is summed with FP32 fused multiply-adds in stored order (the
 * chain of packsell_spmv with x widened); y: uint16 [n], the sums rounded to
 * binary16 (nearest, ties to even), in the original row order (storage order
 * with explicit_perm). PackSELL matrices with C = 32. Errors: INVALID_ARG.
 * No allocation. */
packsell_status packsell_spmv_x16(const packsell_matrix *A, const uint16_t *x, uint16_t *y,
                                  void *stream);

/* y = A x in double for a SELL_F64 matrix (§3's SELL-C-sigma; the FP64
 * operator of §5.2.2's outer iteration) or a W64_E11MY matrix (§4.4's
 * algorithm on 64-bit words: one thread per row, one FP64 fused multiply-add
 * per real word in stored order from +0). x: double [m], y: double [n]
 * (original order, or storage order with explicit_perm). No allocation. */
packsell_status packsell_spmv_f64(const packsell_matrix *A, const double *x, double *y,
                                  void *stream);

/* Y = A X for k right-hand sides (an extension: the paper evaluates k = 1).
 * X: float, row-major [m x k] with leading dimension ldx >= k; Y: float,
 * row-major [n x k] with ldy >= k (rows in storage order with explicit_perm).
 * C > 1 (and SELL_F32): a group of 1-16 lanes shares each row (more for
 * wider k); the words are decoded once per lane and every real word feeds
 * the row's k columns with fused multiply-adds in stored order, so column q
 * of Y equals the thread-per-row packsell_spmv with x = X[:, q] bit for bit.
 * C = 1 PackSELL (CSR order): the split-row kernel (all lanes of a warp
 * share a tile's words, four columns at a time, segmented sums across the
 * lanes): every entry within gamma_w * sum_j |a_ij X_jq| of the exact
 * product, the same bits on every run. k = 1 with ldx = ldy = 1 runs the
 * SpMV itself. 16-byte X/Y loads need k, ldx, ldy divisible by 4 and
 * 16-byte aligned X and Y; other layouts take scalar loads. PackSELL and
 * SELL_F32 matrices. Errors: INVALID_ARG (k < 1, ld < k, SELL_F64). No
 * allocation. */
packsell_status packsell_spmm(const packsell_matrix *A, int32_t k, const float *X,
                              int64_t ldx, float *Y, int64_t ldy, void *stream);

/* Number of SpMV kernel variants (1..PACKSELL_SPMV_VARIANTS). */
#define PACKSELL_SPMV_VARIANTS 14

/* SpMV kernel variants (1-13 compute the same bits; 14 rounds differently):
 *   0 auto: the tuner's choice once packsell_tune_spmv has run, else by
 *     shape: 14 for C = 1 PackSELL; for C = 32 PackSELL 12 when every slice
 *     holds at most 16 words, 4 when padding exceeds 1/8 of the stored
 *     words, otherwise 13; 1 for everything else,
 *   1 thread-per-row with direct loads (the paper's mapping, §5.1.1),
 *   2, 3, 4 bulk-staged: every warp streams its contiguous range of slices
 *     through a circular ring of shared-memory chunks filled by
 *     cp.async.bulk (TMA engine) and completed on mbarriers; the three differ
 *     in warps per block, chunks per warp and chunk size (8/4/2 KB, 4/4/2 KB,
 *     8/2/4 KB). Bulk variants need a PackSELL matrix with C = 32;
 *   5, 6 thread-per-row with row register prefetch: the words of a round
 *     are loaded at once before any is decoded; 5 sizes the round to the
 *     widest slice (8, 10, 12 or 16 words), 6 uses 32 (PackSELL, C = 32);
 *   7, 8 dual-row persistent: each thread loads two rows (from two slices)
 *     together, rounds of 8-12 words fitted to the widest slice (7) or 16
 *     (8) (PackSELL, C = 32);
 *   9, 10 stage-planned TMA: at encode time each warp's slices are cut into
 *     stages of whole slices (at most 4 KB (9) or 2 KB (10)); one
 *     cp.async.bulk per stage into a double-buffered shared-memory slot with
 *     an mbarrier; the consumer waits once per stage (PackSELL, C = 32).
 *  11 CSR order (PackSELL with C = 1: each slice is one row, the words of the
 *     rows lie one after another with no padding, the delta-value packing in
 *     CSR order that §7 leaves as future work for matrices too irregular for
 *     SELL). At encode time the rows are cut into tiles of at most 256 words
 *     and 64 rows, and rows of more than 256 words become items of their own.
 *     A warp copies a tile's words to shared memory with coalesced loads and
 *     its lanes sum one row each; a long row is walked 256 words at a time
 *     with a warp prefix sum of the deltas for the columns, parallel gathers
 *     and one in-order chain of fused multiply-adds. Same bits as variant 1.
 *  12 pipelined persistent (PackSELL, C = 32): each thread walks rows i,
 *     i + stride, ... and loads the next row's words (and the slice offsets
 *     of the row after it) before it decodes and gathers the current row, so
 *     the word loads of one row overlap the gathers of the previous one; one
 *     round per row, fitted to the widest slice as in 5, so every slice must
 *     hold at most 16 words. For short rows (the solver's 7-point matrices);
 *     the solver's fused SpMV + dot uses it for such matrices.
 *  13 variant 5 (rows run to the slice width) launched with programmatic
 *     dependent launch: its blocks are scheduled while the previous kernel
 *     of the stream drains, load the offsets and their first round of words,
 *     and only then wait for that kernel to complete before they read x or
 *     write y. Safe because a matrix is complete when packsell_encode or
 *     packsell_import returns and no product writes it (PackSELL, C = 32).
 *  14 split rows in CSR order (PackSELL with C = 1; the future-work form of
 *     §7 as variant 11): at encode time the rows are cut into tiles of at
 *     most 253 words and 256 rows, and longer rows become items of their
 *     own. All 32 lanes of a warp share a tile's words (16-byte loads, four
 *     words per lane per round): the columns (Eq. 2 from the left offset of
 *     Eq. 4) are a segmented prefix sum of the deltas restarting at each row
 *     start, and the products are summed per row by a segmented sum across
 *     the lanes; a long row is walked 256 words at a time, each lane summing
 *     its words, then a butterfly reduction. The order is fixed (the same
 *     bits on every run) but is a tree, not the stored-order chain: each row
 *     is within gamma_w * sum_j |a_ij x_j| of the exact product (w stored
 *     words of the row). The plan's default for C = 1 PackSELL matrices. */
packsell_status packsell_set_spmv_variant(packsell_matrix *A, int32_t variant);

/* Autotune the SpMV variant (the §4.4 product in several kernel mappings;
 * no counterpart in the paper) for this matrix: time every available variant
 * (`reps` launches each after a warm-up, CUDA events on `stream`) on the
 * caller's x [m] and y [n], and make variant 0 run the fastest. Writes y.
 * Synchronises `stream`. If h_times is not NULL it receives the average
 * milliseconds per launch of variants 1..PACKSELL_SPMV_VARIANTS (0 where
 * unavailable). */
packsell_status packsell_tune_spmv(packsell_matrix *A, const float *x, float *y, int32_t reps,
                                   float *h_times, void *stream);

/* The value quantiser of §4.2.2 on its own (step one of the encoder): field[p]
 * = the value field of val[p] in `format` with D delta bits, as it sits in a
 * word's upper bits (FP16: the binary16 pattern << 16, round to nearest
 * even, D = 15; E8MY: the FP32 pattern rounded half away from zero with the
 * low D + 1 bits clear, D in [1, 22]; W16_E4M3: the FP8 E4M3 code, D = 7).
 * val: float [n] (val_is_f64 = 0) or double [n] (1), device; field: uint32
 * [n], device. SYNCHRONISES `stream`. Errors: INVALID_ARG (format, D),
 * RANGE (a value rounds past the format's largest), NONFINITE (Inf or NaN);
 * on those *h_bad_index (nullable, host) receives the first offending index
 * found and the fields are unspecified. */
packsell_status packsell_quantize(int32_t format, int32_t D, int64_t n, const void *val,
                                  int32_t val_is_f64, uint32_t *field, int64_t *h_bad_index,
                                  void *stream);

/* One candidate of packsell_tune_format. */
typedef struct packsell_format_trial {
    packsell_params params; /* C, sigma, D, format tried (implicit permutation) */
    double error;       /* bound on the SpMV backward error of §5.1.2 with this value format */
    int32_t admissible; /* 1: every value fits and error <= the ceiling (then timed) */
    int32_t variant;    /* fastest SpMV variant (0: not timed) */
    int64_t n_words;    /* stored words (0: not timed) */
    double bytes;       /* algorithmic bytes of one SpMV (0: not timed) */
    double ms;          /* milliseconds per SpMV with that variant (0: not timed) */
} packsell_format_trial;

/* Autotuner of the format's knobs (the paper leaves them to the user: slice
 * height and sort block of §3, delta/value split D and value format of
 * §4.2-§4.3, whose accuracy §5.1.2 measures as a backward error). For a CSR
 * matrix (device arrays as packsell_encode) and a backward-error ceiling:
 *  1. for each value format - FP16 (D = 15) and E8MY with D = 15, 11, 7, 3,
 *     1 (E8M7 .. E8M21) - a kernel bounds the backward error
 *     ||y - A x||_inf / (||A||_inf ||x||_inf) of an SpMV with it by
 *     (max_i sum_j |a_ij - q(a_ij)| + gamma_w max_i sum_j |q(a_ij)|) /
 *     max_i sum_j |a_ij|, w = twice the longest row (each nonzero takes at
 *     most one dummy), gamma_w = w u / (1 - w u), u = 2^-24;
 *  2. every format within the ceiling is encoded in each layout - C = 32
 *     with sigma = 256 and sigma = 65,536, and C = 1 (CSR order) - and its
 *     SpMV variants timed as packsell_tune_spmv does (on the caller's x [m]
 *     and y [n], `reps` launches each; y is overwritten);
 *  3. *best = the parameters of the fastest (implicit permutation, k_left
 *     computed), to pass to packsell_encode.
 * h_trials (host, max_trials entries, nullable when max_trials = 0) receives
 * every candidate in the order above (18 at most), *n_trials (nullable)
 * their count. SYNCHRONISES `stream`; allocates and frees each candidate.
 * Errors: INVALID_ARG, RANGE (no format within the ceiling), and those of
 * packsell_encode. */
packsell_status packsell_tune_format(int64_t n, int64_t m, int64_t nnz, const int64_t *rowptr,
                                     const int32_t *col, const void *val, int32_t val_is_f64,
                                     double max_error, const float *x, float *y, int32_t reps,
                                     packsell_params *best, packsell_format_trial *h_trials,
                                     int32_t max_trials, int32_t *n_trials, void *stream);

/* Diagnostics (no counterpart in the paper): the number of polls after
 * which the TMA-staged SpMV variants (2-4, 9, 10) give up waiting for a
 * chunk of words to land in shared memory; polls < 0 restores the default
 * (2^24). A kernel that gives up records PACKSELL_ERR_TIMEOUT in the
 * matrix's status word (packsell_check_status), skips the rest of its rows
 * (their y entries are left as they were), and before it returns waits -
 * with the default limit, whatever is set here - for every copy it has
 * issued. polls = 0 makes every such wait give up at once: the way to
 * exercise that path. Applies to later launches in the process, on every
 * device; not to be changed while SpMVs of those variants run. */
packsell_status packsell_set_wait_limit(int64_t polls);

/* Housekeeping (no counterpart in the paper): read and clear the matrix's
 * device status word (synchronises `stream`).
 * Returns PACKSELL_ERR_TIMEOUT if a kernel's bounded wait on a shared-memory
 * stage ran out since the last check (the kernel then skipped the rest of
 * its work). In the bounds-check build (packsell_checks_build) it also reads
 * and clears the out-of-range counters of the current device - kept for the
 * whole library, not per matrix - and returns PACKSELL_ERR_CHECK, with the
 * count and the first index in the message, if any access was skipped since
 * the last check. Else PACKSELL_OK. */
packsell_status packsell_check_status(const packsell_matrix *A, void *stream);

/* Housekeeping (no counterpart in the paper): decode the whole matrix on the
 * device and check it against the record kept at encode time - every slice
 * offset C-aligned and increasing, every perm entry inside its sigma block,
 * every column (Eq. 2 from Eq. 4's left offset) below m, and the words with
 * a value (or the FP16 SELL slots that are not padding) counting nnz.
 * packsell_import runs the same check on every blob. Reads the matrix only;
 * synchronises `stream`. Returns CORRUPT (with the first bad index in the
 * message) or OK. */
packsell_status packsell_validate(const packsell_matrix *A, void *stream);

/* ---------------------------------------------------------------------- */
/* Batched SpMV: many matrices, one persistent launch                       */
/* ---------------------------------------------------------------------- */
/* The paper runs one matrix per launch; batching many small or uneven
 * matrices into one launch is this library's extension of §4.4. */

typedef struct packsell_batch packsell_batch; /* opaque plan */

/* Many §4.4 products in one launch per layout (the paper runs one matrix at
 * a time). Build a plan for y_i = A_i x_i, i < count. A: host array of
 * PackSELL matrices with C = 32 or C = 1 (FP16 and E8MY, sigma and the
 * permutation mode may be mixed); x, y: host arrays of device pointers (x_i
 * float [m_i], y_i float [n_i]) bound to the plan. The plan uploads one
 * descriptor per matrix and work lists:
 *  - C = 32 matrices: (matrix, slice range) items of about equal word counts,
 *    taken round-robin by the warps of one persistent launch, one thread per
 *    row (each row's sum is the bits of packsell_spmv);
 *  - C = 1 matrices (CSR order, §7's future work): the items of the
 *    split-row kernel of packsell_spmm (tiles of at most 125 words and 128
 *    rows, rows of more words on their own, long rows first), taken by the
 *    warps of a second persistent launch; every row within gamma_w * sum_j
 *    |a_ij x_j| of the exact product, the same bits on every run.
 * Reads each matrix's offsets (SYNCHRONISES `stream`). The matrices and
 * vectors must outlive the plan. */
packsell_status packsell_batch_create(int32_t count, const packsell_matrix *const *A,
                                      const float *const *x, float *const *y, void *stream,
                                      packsell_batch **out);

/* Every y_i = A_i x_i (§4.4) of a plan from packsell_batch_create: one
 * launch for the C = 32 matrices and one for the C = 1 matrices
 * (asynchronous; no allocation, so it can be captured in a CUDA graph).
 * Errors: INVALID_ARG for a plan from packsell_batch_create_spmm. */
packsell_status packsell_batch_spmv(const packsell_batch *B, void *stream);

/* Many products with k right-hand sides (Y_i = A_i X_i; the paper evaluates
 * k = 1 on one matrix at a time) in one launch. A: host array of `count`
 * PackSELL matrices with C = 1 (CSR order); X, Y: host arrays of device
 * pointers, X_i float row-major [m_i x k] with leading dimension ldx[i] >= k,
 * Y_i float [n_i x k] with ldy[i] >= k (rows in storage order with
 * explicit_perm); ldx, ldy: host arrays, or NULL for k. The plan holds the
 * split-row items of every matrix (see packsell_batch_create); one
 * persistent launch takes them all, each tile computing four columns at a
 * time (16-byte X and Y accesses when k and every leading dimension are
 * multiples of 4 and every block is 16-byte aligned). Every entry of Y_i is
 * within gamma_w * sum_j |a_ij X_jq| of the exact product. Reads each
 * matrix's offsets (SYNCHRONISES `stream`). Errors: INVALID_ARG (k < 1, a
 * matrix that is not PackSELL with C = 1, a NULL block, ld < k), NO_MEMORY,
 * CUDA. */
packsell_status packsell_batch_create_spmm(int32_t count, const packsell_matrix *const *A, int32_t k,
                                           const float *const *X, const int64_t *ldx,
                                           float *const *Y, const int64_t *ldy, void *stream,
                                           packsell_batch **out);

/* Run a plan from packsell_batch_create_spmm (asynchronous, one launch, no
 * allocation). Errors: INVALID_ARG for a plan from packsell_batch_create. */
packsell_status packsell_batch_spmm(const packsell_batch *B, void *stream);

/* Work-list statistics of a batch plan (no counterpart in the paper): total
 * stored words, algorithmic bytes of one launch (words, offsets, perm, x and
 * y once), number of work items. */
packsell_status packsell_batch_info(const packsell_batch *B, int64_t *words, int64_t *bytes,
                                    int32_t *items);

packsell_status packsell_batch_destroy(packsell_batch *B);

/* ---------------------------------------------------------------------- */
/* Backward (adjoint) products                                              */
/* ---------------------------------------------------------------------- */

/* The adjoint of Eq. 1 over the §4.3 layout: dx = A^T dy (float [m]),
 * written from the packed layout with atomic adds:
 * the result is overwritten (not accumulated) and its rounding depends on
 * the order of the adds. */
packsell_status packsell_spmv_transpose(const packsell_matrix *A, const float *dy,
                                        float *dx, void *stream);

/* The gradient of Eq. 1 with respect to the stored values: out[q] =
 * alpha * u_i * v_j for every stored nonzero a_ij, with q its CSR
 * position. u: float [n] (original row order), v: float [m], out: float
 * [nnz]. This is dL/dA on the pattern for y = A x (u = dL/dy, v = x,
 * alpha = 1) and for x = A^-1 b (u = adjoint solution, v = x, alpha = -1).
 * Needs a matrix encoded with keep_rowptr = 1. */
packsell_status packsell_pattern_outer(const packsell_matrix *A, float alpha, const float *u,
                                       const float *v, float *out, void *stream);

/* As packsell_pattern_outer, for the §5.2.2 solve: out[q] = alpha * u_i *
 * v_j in double for a SELL_F64 matrix encoded with
 * keep_rowptr = 1 (u: double [n], v: double [m], out: double [nnz], CSR
 * order): dL/dA on the pattern of x = A^-1 b is pattern_outer(-1, lam, x)
 * with lam the adjoint solution of A^T lam = dL/dx. */
packsell_status packsell_pattern_outer_f64(const packsell_matrix *A, double alpha,
                                           const double *u, const double *v, double *out,
                                           void *stream);

/* Backward of y = A x (the adjoint of the §4.4 product; the paper
 * differentiates nothing). Given x (float [m]) and dy = dL/dy (float [n]),
 * both in original order:
 *   dx   : NULL (skipped) or float [m], out: A^T dy, overwritten, with
 *          atomic adds as in packsell_spmv_transpose
 *   dval : NULL (skipped) or float [nnz], out: dL/da_ij = dy_i x_j at the
 *          CSR position of a_ij (needs keep_rowptr = 1; gradient through
 *          the quantiser taken as the identity)
 * Asynchronous on `stream`. Errors: those of packsell_spmv_transpose and
 * packsell_pattern_outer, which it runs. */
packsell_status packsell_spmv_backward(const packsell_matrix *A, const float *x, const float *dy,
                                       float *dx, float *dval, void *stream);


/* ---------------------------------------------------------------------- */
/* Solvers (§5.2.2): FP64 PCG and the mixed-precision inner-outer CG        */
/* ---------------------------------------------------------------------- */

typedef struct packsell_solve_opts {
    double rtol;         /* stop when ||b - A x||_2 / ||b||_2 < rtol, checked on the
                            true residual in FP64 */
    int32_t m_in;        /* inner FP32 PCG iterations per outer step (IO-CG);
                            0 = plain FP64 Jacobi PCG on A_outer */
    int32_t max_iters;   /* outer iterations (PCG iterations when m_in = 0) */
    int32_t check_every; /* iterations per graph replay between host checks; the
                            device idles once converged, so counts stay exact */
    int32_t use_graph;   /* 1: replay the iteration body as a captured CUDA graph */
} packsell_solve_opts;

typedef struct packsell_solve_result {
    int32_t iters;       /* outer (or PCG) iterations done */
    int32_t inner_iters; /* inner iterations done (IO-CG) */
    double relres;       /* recurrence residual ||r|| / ||b|| at exit */
    double relres_true;  /* true residual ||b - A x|| / ||b|| at exit (FP64) */
    double seconds;      /* device time of the solve (CUDA events) */
} packsell_solve_result;

/* The Jacobi preconditioner of §5.2 (diagonal scaling): out[i] = 1 / a_ii
 * (double [n]) for a square SELL_F64 or W64_E11MY matrix, in the
 * original row order: the Jacobi preconditioner of packsell_pcg. Rows whose
 * diagonal is missing or zero get 1. */
packsell_status packsell_inv_diag(const packsell_matrix *A, double *out, void *stream);

/* rows[i] = the original row stored at storage position i (int32 [n], device),
 * i.e. (i / sigma) * sigma + perm[i] with the sigma-block sort of §3 / §4.3.
 * With explicit_perm, packsell_spmv writes y[i] for that row, so
 * y_orig[rows[i]] = y[i]; with sigma = 1 rows[i] = i. Works for every format
 * and either perm mode. Errors: INVALID_ARG on a NULL argument. */
packsell_status packsell_storage_rows(const packsell_matrix *A, int32_t *rows, void *stream);

/* Device workspace bytes the §5.2.2 solvers (packsell_pcg) need for n unknowns (has_diag: a Jacobi
 * preconditioner is passed). */
size_t packsell_pcg_workspace_bytes(int64_t n, int32_t m_in, int32_t has_diag,
                                    int32_t max_iters);

/* Solve A x = b for SPD A (§5.2.2: FP64 PCG, or the inner-outer CG).
 *   A_outer : SELL_F64 or W64_E11MY matrix (square, implicit permutation): the FP64
 *             operator of the outer iteration and of the residual check
 *   A_inner : PackSELL (FP16 / E8MY) or SELL_F32 copy of the same matrix for
 *             the inner FP32 PCG (ignored when m_in = 0)
 *   inv_diag: NULL or double [n], the Jacobi preconditioner 1 / a_ii
 *   b       : double [n]; x: double [n], the initial guess on entry, the
 *             solution on exit
 *   work    : device workspace of at least packsell_pcg_workspace_bytes, or
 *             NULL to let the call allocate (stream-ordered) and free it
 *   h_hist  : NULL or host double [max_iters + 1]: recurrence residual after
 *             each outer (PCG) iteration, entry 0 the initial one
 * IO-CG: flexible CG (one previous direction) in FP64; its preconditioner is
 * m_in PCG iterations in FP32 from zero on r / ||r||_2 with A_inner. Outer
 * dot products are FP64 throughout; inner ones sum each thread's elements in
 * FP32 and combine the partial sums in FP64 (deterministically). The
 * residual is replaced by the true one if the recurrence claims convergence
 * before b - A x does.
 * Runs on a private stream after the caller's pending work; SYNCHRONISES.
 * Returns NOT_CONVERGED after max_iters (x holds the last iterate),
 * BREAKDOWN on p^T A p <= 0 or a non-finite residual. */
packsell_status packsell_pcg(const packsell_matrix *A_outer, const packsell_matrix *A_inner,
                             const double *inv_diag, const double *b, double *x,
                             const packsell_solve_opts *opts, void *work, size_t work_bytes,
                             double *h_hist, packsell_solve_result *result, void *stream);

/* Backward of the §5.2.2 solve x = A^-1 b for SPD A: the adjoint solve A lam = dL/dx (A is
 * symmetric, so A^T = A), with the operators and options of packsell_pcg,
 * from lam = 0; then dL/db = lam and dL/da_ij = -lam_i x_j on the pattern.
 *   x      : double [n], the forward solution
 *   dL_dx  : double [n]
 *   dL_db  : double [n], out: lam
 *   dL_dA  : NULL (skipped) or double [nnz], out in CSR order (A_outer
 *            encoded with keep_rowptr = 1), written on `stream` after the
 *            solve
 * Other arguments as packsell_pcg. The solve SYNCHRONISES; its status is
 * returned (NOT_CONVERGED leaves the last iterate in dL_db and skips dL_dA). */
packsell_status packsell_pcg_backward(const packsell_matrix *A_outer,
                                      const packsell_matrix *A_inner, const double *inv_diag,
                                      const double *x, const double *dL_dx, double *dL_db,
                                      double *dL_dA, const packsell_solve_opts *opts, void *work,
                                      size_t work_bytes, packsell_solve_result *result,
                                      void *stream);

/* packsell_pcg without any device allocation. The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory when
 * they solve - an application that reserved the device's memory up front
 * for its own pool, where a cudaMalloc would fail or fragment that pool;
 * a plugin handed a fixed memory budget by its host; a latency-bound loop
 * that must not take cudaMalloc's or cudaFree's implicit synchronisation.
 * It takes the same arguments as packsell_pcg minus the workspace: the
 * workspace comes from one static device array of 8 MiB in the library
 * (enough for about 160,000 unknowns with IO-CG and 260,000 with FP64 PCG;
 * every GPU that loads the library holds it until the process exits). A
 * system whose workspace would not fit (packsell_pcg_workspace_bytes >
 * 8 MiB) is rejected with PACKSELL_ERR_INVALID_ARG and a message giving
 * both sizes.
 * - It allocates nothing: no cudaMalloc/cudaFree, no stream, event or graph;
 *   it runs directly on `stream`, reads the solver's scalars back to the
 *   host as it iterates, and synchronises `stream` before returning
 *   (result->seconds is host wall time).
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and keeps it for later
 *   calls on that device. A cudaDeviceReset invalidates the kept address, as it does every
 *   matrix of the library: do not call the library on a device after
 *   resetting it.
 * - All calls share the array and every call re-initialises what must start
 *   from zero, so results do not depend on earlier calls; but calls that
 *   overlap on the GPU (other threads or streams) race on it: serialise them. */
packsell_status packsell_pcg_noalloc(const packsell_matrix *A_outer,
                                     const packsell_matrix *A_inner, const double *inv_diag,
                                     const double *b, double *x,
                                     const packsell_solve_opts *opts, double *h_hist,
                                     packsell_solve_result *result, void *stream);

/* ---------------------------------------------------------------------- */
/* F3R: the nested Krylov solver of §5.2.1                                 */
/* ---------------------------------------------------------------------- */

typedef struct packsell_f3r_opts {
    double rtol;        /* stop when ||b - A x||_2 / ||b||_2 < rtol (true residual, FP64) */
    int32_t m1;         /* restart length of the outer FGMRES (layer 1), 1..60 */
    int32_t m2;         /* FGMRES steps of layer 2 per application, 1..60 */
    int32_t m3;         /* FGMRES steps of layer 3 per application, 1..60 */
    int32_t m4;         /* Richardson steps of layer 4 per application, >= 1 */
    int32_t max_iters;  /* outer FGMRES steps at most */
    double omega;       /* Richardson damping, > 0 */
} packsell_f3r_opts;

/* Defaults: rtol = 1e-9 (the paper's criterion, §5.2), m1 = 30, m2 = 8,
 * m3 = 4, m4 = 2, max_iters = 300, omega = 1. The paper takes F3R's own
 * defaults from the work that defines it and does not print them; these are
 * this library's choices. */
void packsell_f3r_opts_default(packsell_f3r_opts *o);

/* Solve A x = b with F3R (§5.2.1): FGMRES(m1) in FP64 on A_outer (restarted,
 * x the initial guess on entry, the solution on exit), preconditioned by
 * m2 steps of FGMRES on A_mid from zero, preconditioned by m3 steps of FGMRES
 * on A_low from zero, preconditioned by m4 Richardson steps z <- z + omega
 * (r - A_low z) from z = 0 (the Jacobi preconditioner is the identity on
 * the symmetrically scaled matrices of §5.2: scale A beforehand).
 * Configurations:
 *  - FP16-F3R: A_mid SELL_F32 (layer 2 in FP32) and A_low a PackSELL FP16
 *    (or E8MY) or an FP16 SELL matrix (layers 3 and 4: FP32 vectors, the
 *    FP16 SpMV of the paper);
 *  - FP64-F3R: A_mid and A_low SELL_F64 or W64_E11MY (every layer in FP64).
 * A_outer is SELL_F64 or W64_E11MY; all three square, of the same size, rows in original
 * order (any C and sigma). Krylov bases by classical Gram-Schmidt in each
 * layer's arithmetic: FP64 layers in double; FP32 layers in FP32, with the
 * dot products' per-thread partials in FP32 and their block and grid sums in
 * FP64 (deterministic: block order); Hessenberg matrices, Givens rotations
 * and least-squares solves in FP64 on the device. The outer residual estimate is read after every
 * outer step; convergence is confirmed on the true FP64 residual (a cycle
 * restarts from it otherwise). FP16-F3R with a PackSELL FP16 A_low and with
 * the FP16 SELL copy of the same matrix runs the same arithmetic: the same
 * iterates, bit for bit.
 * b, x: double [n], device. result (nullable): iters = outer steps,
 * inner_iters = layer-3 steps (iters * m2 * m3), relres = the last outer
 * estimate, relres_true, seconds (device time). Allocates its workspace
 * (stream-ordered) and SYNCHRONISES. Errors: INVALID_ARG, NO_MEMORY, CUDA,
 * NOT_CONVERGED (x holds the last iterate), BREAKDOWN (non-finite residual). */
packsell_status packsell_f3r(const packsell_matrix *A_outer, const packsell_matrix *A_mid,
                             const packsell_matrix *A_low, const double *b, double *x,
                             const packsell_f3r_opts *opts, packsell_solve_result *result,
                             void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PACKSELL_H */
