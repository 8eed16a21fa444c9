/*
 * PackSELL oracle: a plain, slow, obviously correct CPU implementation of what
 * the PackSELL format and its SpMV compute (arXiv 2604.13433).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's compute path may link,
 * load or call this file; only the tests, the smoke check and the bench's CPU
 * baseline do. It shares no code, header, table or helper with the CUDA
 * library: every routine here is written from the paper's text.
 *
 * Precision: integer and bit work is exact. Values are handled in double
 * precision except the FP32 "twin" SpMV, which fixes FP32 fused multiply-add
 * in stored order on purpose. Build with -ffp-contract=off (no implicit FMA).
 *
 * Readings of the paper taken here where it is silent (each is listed with its
 * reason in the design notes):
 *  - E8MY below FP32's normal range: the rounding grid stays at the spacing
 *    of the smallest normal binade (the paper's ldexpf would underflow).
 *  - Padding and dummy words contribute nothing (no x load, no multiply).
 *  - Stable sort inside sigma blocks: equal word counts keep original order.
 *  - Columns must be strictly increasing inside a row.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_UNSORTED = 2, ORC_ERR_NONFINITE = 3,
       ORC_ERR_RANGE = 4 };
enum { ORC_FMT_FP16 = 1, ORC_FMT_E8MY = 2, ORC_FMT_FIXED = 7, ORC_FMT_W64_E11MY = 8 };

/* ------------------------------------------------------------------------ */
/* Value formats (§4.2.2)                                                     */
/* ------------------------------------------------------------------------ */

/* IEEE 754 binary16 from a real value, round to nearest, ties to even.
 * Written from the binary16 definition: 1 sign, 5 exponent bits (bias 15),
 * 10 fraction bits; subnormals have spacing 2^-24; largest finite 65504.
 * Returns ORC_OK, ORC_ERR_NONFINITE (input inf/nan) or ORC_ERR_RANGE
 * (rounds past 65504). */
int orc_f16_bits(double v, uint16_t *out)
{
    if (isnan(v) || isinf(v)) return ORC_ERR_NONFINITE;
    uint16_t sign = signbit(v) ? 0x8000u : 0u;
    double a = fabs(v);
    if (a == 0.0) { *out = sign; return ORC_OK; }
    int ex;
    (void)frexp(a, &ex); /* a = f * 2^ex, f in [0.5, 1): binade [2^(ex-1), 2^ex) */
    int e = ex - 1;      /* a in [2^e, 2^(e+1)) */
    double q = (e < -14) ? ldexp(1.0, -24) : ldexp(1.0, e - 10); /* spacing */
    double r = a / q;    /* exact: division by a power of two */
    double fl = floor(r);
    double rem = r - fl;
    if (rem > 0.5 || (rem == 0.5 && fmod(fl, 2.0) != 0.0)) fl += 1.0;
    double res = fl * q;
    if (res > 65504.0) return ORC_ERR_RANGE;
    uint16_t bits;
    if (res < ldexp(1.0, -14)) {
        bits = (uint16_t)fl; /* subnormal: count of 2^-24 (0 .. 1023) */
    } else {
        int rex;
        (void)frexp(res, &rex);
        int E = rex - 1;                        /* res in [2^E, 2^(E+1)) */
        double frac = res / ldexp(1.0, E) - 1.0; /* in [0, 1) */
        bits = (uint16_t)(((E + 15) << 10) | (uint16_t)(frac * 1024.0));
    }
    *out = (uint16_t)(sign | bits);
    return ORC_OK;
}

/* Real value of a binary16 bit pattern. */
double orc_f16_value(uint16_t h)
{
    int s = (h >> 15) & 1, E = (h >> 10) & 0x1f, F = h & 0x3ff;
    double mag;
    if (E == 0) mag = ldexp((double)F, -24);
    else if (E == 31) mag = F ? NAN : INFINITY;
    else mag = ldexp(1.0 + F / 1024.0, E - 15);
    return s ? -mag : mag;
}

static uint32_t f32_bits(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }
static float f32_from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }

/* E8MY bits (1 sign, 8 exponent, Y = 22 - D mantissa bits, FP32 layout with
 * the low D + 1 bits clear), following the paper's steps (§4.2.2): take the
 * binary exponent of v, set the rounding unit to 2^(exp - 24 + D + 1), round
 * v / unit to the nearest integer with halves away from zero, scale back,
 * reinterpret as FP32 bits and clear the low D + 1 bits.
 * Reading where the paper is silent: below FP32's normal range the exponent is
 * held at that of the smallest normal binade, so the unit stays 2^(D + 1)
 * FP32 subnormal steps. Returns ORC_OK, ORC_ERR_NONFINITE or ORC_ERR_RANGE. */
int orc_e8my_bits(double v, int D, uint32_t *out)
{
    if (D < 1 || D > 22) return ORC_ERR_ARG;
    if (isnan(v) || isinf(v)) return ORC_ERR_NONFINITE;
    if (v == 0.0) { *out = signbit(v) ? 0x80000000u : 0u; return ORC_OK; }
    int ex;
    (void)frexp(v, &ex);
    if (ex < -125) ex = -125;
    double unit = ldexp(1.0, ex - 24 + D + 1);
    double r = round(v / unit) * unit; /* round(): halves away from zero */
    if (fabs(r) >= ldexp(1.0, 128)) return ORC_ERR_RANGE;
    float rf = (float)r;
    if ((double)rf != r) return ORC_ERR_RANGE; /* cannot happen on the grid */
    uint32_t b = f32_bits(rf);
    b = (b >> (D + 1)) << (D + 1);
    *out = b;
    return ORC_OK;
}

/* E11MY bits (1 sign, 11 exponent, Y = 51 - D mantissa bits, binary64 layout
 * with the low D + 1 bits zero): the value format of 64-bit words (W = 64,
 * V = 63 - D), E8MY's rule (§4.2.2) carried over to binary64: round half away
 * from zero on the grid 2^(e - 53 + D + 1), e the binade of v, the grid of
 * the smallest normal binade below it. D in [1, 31]. */
static uint64_t f64_bits(double v)
{
    uint64_t b;
    memcpy(&b, &v, sizeof b);
    return b;
}

int orc_e11my_bits(double v, int D, uint64_t *out)
{
    if (D < 1 || D > 31) return ORC_ERR_ARG;
    if (isnan(v) || isinf(v)) return ORC_ERR_NONFINITE;
    if (v == 0.0) { *out = signbit(v) ? 0x8000000000000000ull : 0ull; return ORC_OK; }
    int ex;
    (void)frexp(v, &ex); /* |v| in [2^(ex-1), 2^ex) */
    if (ex < -1021) ex = -1021;
    const double unit = ldexp(1.0, ex - 53 + D + 1);
    const double r = round(v / unit) * unit; /* both steps exact; round(): halves away */
    if (isinf(r)) return ORC_ERR_RANGE;
    uint64_t b = f64_bits(r);
    b = (b >> (D + 1)) << (D + 1);
    *out = b;
    return ORC_OK;
}

double orc_e11my_value(uint64_t bits)
{
    double v;
    memcpy(&v, &bits, sizeof v);
    return v;
}

/* Fixed point, an integer value format (§4.2.1 allows any V-bit format,
 * integer formats included): the V = 31 - D value bits hold a two's-
 * complement integer q and the value is q * 2^s, with one exponent s for the
 * whole matrix. s is the smallest integer with (2^(V-1) - 1) * 2^s >= M, M the
 * largest |a_ij| (s = 0 when M = 0), so every value rounds to an integer of at
 * most 2^(V-1) - 1 in magnitude. Written from that definition with exact
 * power-of-two scaling in double. */
int orc_fixed_exponent(double M, int D)
{
    const int V = 31 - D;
    if (D < 1 || D > 22) return 0;
    if (!(M > 0.0)) return 0;
    const double top = ldexp(1.0, V - 1) - 1.0;  /* largest magnitude of q */
    int s = ilogb(M) - (V - 1);
    while (ldexp(top, s) < M) ++s;
    while (ldexp(top, s - 1) >= M) --s;
    return s;
}

/* Value field of v in fixed point with exponent s: q = v / 2^s rounded half
 * away from zero (round()), placed as a V-bit two's-complement integer in
 * bits D+1..31. Returns ORC_OK, ORC_ERR_NONFINITE, or ORC_ERR_RANGE when |q|
 * exceeds 2^(V-1) - 1. */
int orc_fixed_bits(double v, int D, int s, uint32_t *out)
{
    if (D < 1 || D > 22) return ORC_ERR_ARG;
    if (isnan(v) || isinf(v)) return ORC_ERR_NONFINITE;
    const int V = 31 - D;
    const double q = round(ldexp(v, -s));
    if (fabs(q) > ldexp(1.0, V - 1) - 1.0) return ORC_ERR_RANGE;
    const int64_t qi = (int64_t)q;
    const uint32_t bits = (uint32_t)((uint64_t)qi & ((1ull << V) - 1ull));
    *out = bits << (D + 1);
    return ORC_OK;
}

/* The value of a fixed-point field: the sign-extended V-bit integer times 2^s. */
double orc_fixed_value(uint32_t field, int D, int s)
{
    const int V = 31 - D;
    int64_t q = (int64_t)(field >> (D + 1));
    if (q >= (1ll << (V - 1))) q -= (1ll << V);
    return ldexp((double)q, s);
}

/* Fixed-point quantisation of nnz values: the exponent from the largest
 * magnitude, then every field and its value. Returns the first error with its
 * index in *bad. */
int orc_quantize_fixed(int64_t nnz, const double *val, int32_t D, uint32_t *field, double *deq,
                       int32_t *s_out, int64_t *bad)
{
    *bad = -1;
    double M = 0.0;
    for (int64_t p = 0; p < nnz; ++p) {
        if (isnan(val[p]) || isinf(val[p])) { *bad = p; return ORC_ERR_NONFINITE; }
        if (fabs(val[p]) > M) M = fabs(val[p]);
    }
    const int s = orc_fixed_exponent(M, D);
    *s_out = s;
    for (int64_t p = 0; p < nnz; ++p) {
        int st = orc_fixed_bits(val[p], D, s, &field[p]);
        if (st) { *bad = p; return st; }
        deq[p] = orc_fixed_value(field[p], D, s);
    }
    return ORC_OK;
}

/* Upper-V-bit value field for format fmt (FP16 needs D = 15). */
int orc_value_field(double v, int fmt, int D, uint32_t *field)
{
    if (fmt == ORC_FMT_FP16) {
        if (D != 15) return ORC_ERR_ARG;
        uint16_t h;
        int st = orc_f16_bits(v, &h);
        if (st) return st;
        *field = (uint32_t)h << 16;
        return ORC_OK;
    }
    if (fmt == ORC_FMT_E8MY) return orc_e8my_bits(v, D, field);
    return ORC_ERR_ARG;
}

/* The working-precision value a field stands for. */
double orc_field_value(uint32_t field, int fmt)
{
    if (fmt == ORC_FMT_FP16) return orc_f16_value((uint16_t)(field >> 16));
    return (double)f32_from_bits(field);
}

/* ------------------------------------------------------------------------ */
/* Words (§4.2.1): bit 0 is the flag.                                         */
/*   flag 1: bits 1..D hold the delta, bits D+1..31 the value.                */
/*   flag 0: bits 1..31 hold the delta; there is no value.                    */
/* ------------------------------------------------------------------------ */
/* FP8 E4M3 (the OCP 8-bit floating-point format): 1 sign bit, 4 exponent bits
 * (bias 7), 3 fraction bits; subnormals have spacing 2^-9; the code S.1111.111
 * is NaN and there are no infinities, so the largest finite value is
 * 1.75 * 2^8 = 448. Round to nearest, ties to even, from the definition:
 * scale the magnitude to an integer grid of the binade (exact in double) and
 * round it with nearbyint (the default rounding mode is to nearest even).
 * Returns ORC_OK, ORC_ERR_NONFINITE (input inf/nan) or ORC_ERR_RANGE (rounds
 * past 448). This is the value format of the 16-bit words (W = 16, D = 7,
 * V = 8), one of the other word sizes the paper names (§4.2.1). */
int orc_e4m3_bits(double v, uint8_t *out)
{
    if (!isfinite(v)) return ORC_ERR_NONFINITE;
    uint8_t s = signbit(v) ? 0x80 : 0x00;
    double a = fabs(v);
    if (a == 0.0) { *out = s; return ORC_OK; }
    if (a < ldexp(1.0, -6)) {                  /* subnormal range: unit 2^-9 */
        double q = nearbyint(a / ldexp(1.0, -9));  /* 0 .. 8 */
        *out = (uint8_t)(s | (uint8_t)q);       /* q = 8 is the smallest normal, 0x08 */
        return ORC_OK;
    }
    int e;
    frexp(a, &e);                               /* a = f * 2^e, f in [0.5, 1) */
    e -= 1;                                     /* a in [2^e, 2^(e+1)) */
    double q = nearbyint(a / ldexp(1.0, e - 3)); /* 8 .. 16 */
    if (q == 16.0) { q = 8.0; e += 1; }
    int E = e + 7;
    int M = (int)q - 8;
    if (E > 15 || (E == 15 && M == 7)) return ORC_ERR_RANGE;
    *out = (uint8_t)(s | (uint8_t)(E << 3) | (uint8_t)M);
    return ORC_OK;
}

/* The value of an E4M3 code (NaN for S.1111.111). */
double orc_e4m3_value(uint8_t c)
{
    int E = (c >> 3) & 15, M = c & 7;
    double sgn = (c & 0x80) ? -1.0 : 1.0;
    if (E == 15 && M == 7) return NAN;
    if (E == 0) return sgn * ldexp((double)M, -9);
    return sgn * ldexp(1.0 + M / 8.0, E - 7);
}

uint32_t orc_word_value(uint32_t field, uint32_t delta) { return field | (delta << 1) | 1u; }
uint32_t orc_word_dummy(uint32_t delta) { return delta << 1; }

/* Split a word into (flag, delta, value field). */
void orc_unpack(uint32_t w, int D, uint32_t *flag, uint32_t *delta, uint32_t *field)
{
    if (w & 1u) {
        *flag = 1;
        *delta = (w >> 1) & ((1u << D) - 1u);
        *field = w & ~((1u << (D + 1)) - 1u);
    } else {
        *flag = 0;
        *delta = w >> 1;
        *field = 0;
    }
}

/* ------------------------------------------------------------------------ */
/* Encoding (§4.1 delta encoding, §4.3 alignment, dummies, permutation)       */
/* ------------------------------------------------------------------------ */

/* Lower bandwidth k_left = max(0, max over nonzeros a_ij of i - j). */
int64_t orc_lower_bandwidth(int64_t n, const int64_t *rowptr, const int32_t *col)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (i - col[p] > k) k = i - col[p];
    return k;
}

/* Left offset of Eq. 4: uniform inside each block of sigma rows. */
int64_t orc_left_offset(int64_t i, int64_t sigma, int64_t k_left)
{
    int64_t b = (i / sigma) * sigma;
    return (k_left < b) ? b - k_left : 0;
}

/* Check the CSR: columns in [0, m), strictly increasing inside each row. */
int orc_check_csr(int64_t n, int64_t m, const int64_t *rowptr, const int32_t *col)
{
    if (rowptr[0] != 0) return ORC_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) {
        if (rowptr[i + 1] < rowptr[i]) return ORC_ERR_ARG;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            if (col[p] < 0 || col[p] >= m) return ORC_ERR_RANGE;
            if (p > rowptr[i] && col[p] <= col[p - 1]) return ORC_ERR_UNSORTED;
        }
    }
    return ORC_OK;
}

/* Stored words of original row i with W-bit words: its nonzeros plus the
 * dummies before every nonzero whose delta (Eq. 2, first delta taken from the
 * left offset) does not fit in D bits. A dummy's delta field has W - 1 bits
 * (§4.2.1): while the remaining delta is 2^D or more, a dummy takes
 * min(delta, 2^(W-1) - 1) of it. With W = 32 (columns below 2^31) that is one
 * dummy carrying the whole delta, the real word then carrying 0 (§4.3).
 * Returns -1 if a delta would be negative. */
int64_t orc_row_words_w(int64_t i, const int64_t *rowptr, const int32_t *col, int64_t sigma,
                        int64_t k_left, int D, int W, int64_t *dummies)
{
    int64_t prev = orc_left_offset(i, sigma, k_left), words = 0;
    const int64_t dmax = W == 64 ? INT64_MAX : ((int64_t)1 << (W - 1)) - 1;
    *dummies = 0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int64_t d = (int64_t)col[p] - prev;
        if (d < 0) return -1;
        while (d >= ((int64_t)1 << D)) {
            d -= (d < dmax ? d : dmax);
            ++words;
            ++*dummies;
        }
        ++words;
        prev = col[p];
    }
    return words;
}

int64_t orc_row_words(int64_t i, const int64_t *rowptr, const int32_t *col, int64_t sigma,
                      int64_t k_left, int D, int64_t *dummies)
{
    return orc_row_words_w(i, rowptr, col, sigma, k_left, D, 32, dummies);
}

typedef struct { int64_t key; int64_t idx; } orc_kv;

static int orc_kv_cmp(const void *a, const void *b)
{
    const orc_kv *x = (const orc_kv *)a, *y = (const orc_kv *)b;
    if (x->key != y->key) return (x->key > y->key) ? -1 : 1; /* descending words */
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);        /* stable */
}

/* Plan: word counts, sigma permutation, slice offsets.
 *   words[n]         stored words per ORIGINAL row
 *   perm[n]          for STORAGE row i, original row = floor(i/sigma)*sigma + perm[i]
 *   offset[S+1]      S = ceil(n / C) slices, offset[k+1] - offset[k] = C * w_k
 *   stats[4]         k_left used, total words, dummies, padding words
 * k_left_in < 0 computes the lower bandwidth. */
int orc_encode_plan_w(int64_t n, int64_t m, const int64_t *rowptr, const int32_t *col,
                      int32_t C, int32_t sigma, int32_t D, int32_t W, int64_t k_left_in,
                      int64_t *words, int32_t *perm, int64_t *offset, int64_t *stats)
{
    if (n < 0 || m < 0 || m >= ((int64_t)1 << 31) || C < 1 || sigma < 1 || D < 1 ||
        D > (W == 64 ? 31 : W - 2) || (W != 16 && W != 32 && W != 64))
        return ORC_ERR_ARG;
    int st = orc_check_csr(n, m, rowptr, col);
    if (st) return st;
    int64_t k_left = k_left_in < 0 ? orc_lower_bandwidth(n, rowptr, col) : k_left_in;
    int64_t dummies = 0, nnz = rowptr[n];
    for (int64_t i = 0; i < n; ++i) {
        int64_t dm;
        words[i] = orc_row_words_w(i, rowptr, col, sigma, k_left, D, W, &dm);
        if (words[i] < 0) return ORC_ERR_ARG; /* k_left smaller than the bandwidth */
        dummies += dm;
    }
    orc_kv *kv = (orc_kv *)malloc(sizeof(orc_kv) * (size_t)(sigma > 0 ? sigma : 1));
    if (!kv) return ORC_ERR_ARG;
    for (int64_t b0 = 0; b0 < n; b0 += sigma) {
        int64_t len = (n - b0 < sigma) ? n - b0 : sigma;
        for (int64_t t = 0; t < len; ++t) { kv[t].key = words[b0 + t]; kv[t].idx = t; }
        qsort(kv, (size_t)len, sizeof(orc_kv), orc_kv_cmp);
        for (int64_t t = 0; t < len; ++t) perm[b0 + t] = (int32_t)kv[t].idx;
    }
    free(kv);
    int64_t S = (n + C - 1) / C;
    offset[0] = 0;
    for (int64_t k = 0; k < S; ++k) {
        int64_t w = 0;
        for (int64_t i = k * C; i < (k + 1) * C && i < n; ++i) {
            int64_t orig = (i / sigma) * sigma + perm[i];
            if (words[orig] > w) w = words[orig];
        }
        offset[k + 1] = offset[k] + (int64_t)C * w;
    }
    stats[0] = k_left;
    stats[1] = offset[S];
    stats[2] = dummies;
    stats[3] = offset[S] - nnz - dummies; /* padding, phantom rows included */
    return ORC_OK;
}

int orc_encode_plan(int64_t n, int64_t m, const int64_t *rowptr, const int32_t *col,
                    int32_t C, int32_t sigma, int32_t D, int64_t k_left_in,
                    int64_t *words, int32_t *perm, int64_t *offset, int64_t *stats)
{
    if (D > 22) return ORC_ERR_ARG;
    return orc_encode_plan_w(n, m, rowptr, col, C, sigma, D, 32, k_left_in, words, perm, offset,
                             stats);
}

/* Fill pack[offset[S]] given the plan. field[nnz] holds each nonzero's value
 * field (from orc_value_field) in CSR order. */
int orc_encode_fill(int64_t n, const int64_t *rowptr, const int32_t *col, const uint32_t *field,
                    int32_t C, int32_t sigma, int32_t D, int64_t k_left, const int32_t *perm,
                    const int64_t *offset, uint32_t *pack)
{
    int64_t S = (n + C - 1) / C;
    memset(pack, 0, sizeof(uint32_t) * (size_t)offset[S]); /* padding words are 0 */
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C, orig = (i / sigma) * sigma + perm[i];
        int64_t prev = orc_left_offset(i, sigma, k_left), j = 0;
        for (int64_t p = rowptr[orig]; p < rowptr[orig + 1]; ++p) {
            int64_t d = (int64_t)col[p] - prev;
            if (d < 0) return ORC_ERR_ARG;
            if (d >= ((int64_t)1 << D)) {
                pack[offset[k] + j * C + l] = orc_word_dummy((uint32_t)d);
                ++j;
                d = 0;
            }
            pack[offset[k] + j * C + l] = orc_word_value(field[p], (uint32_t)d);
            ++j;
            prev = col[p];
        }
        if (offset[k] + j * C > offset[k + 1]) return ORC_ERR_ARG;
    }
    return ORC_OK;
}

/* Decode back to CSR in ORIGINAL row order: counts[n] real words per row,
 * then col_out/field_out at out_rowptr positions (caller passes the rowptr it
 * expects; the function reports a mismatch in counts through the return). */
int orc_decode(int64_t n, int32_t C, int32_t sigma, int32_t D, int64_t k_left,
               const int32_t *perm, const int64_t *offset, const uint32_t *pack,
               const int64_t *rowptr, int32_t *col_out, uint32_t *field_out, int64_t *counts)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C, orig = (i / sigma) * sigma + perm[i];
        int64_t w = (offset[k + 1] - offset[k]) / C;
        int64_t c = orc_left_offset(i, sigma, k_left), q = rowptr[orig], cnt = 0;
        for (int64_t j = 0; j < w; ++j) {
            uint32_t flag, delta, fld;
            orc_unpack(pack[offset[k] + j * C + l], D, &flag, &delta, &fld);
            c += delta;
            if (flag) {
                if (q < rowptr[orig + 1]) { col_out[q] = (int32_t)c; field_out[q] = fld; }
                ++q;
                ++cnt;
            }
        }
        counts[orig] = cnt;
    }
    return ORC_OK;
}

/* 64-bit words (W = 64, §4.2.1 with V = 63 - D): a word with a value is
 * field | (d << 1) | 1, the field an E11MY pattern whose low D + 1 bits are
 * zero; a dummy is (d << 1) with flag 0 (63 delta bits, so one dummy covers any
 * gap); padding is 0. Same slice layout and plan as the 32-bit words
 * (orc_encode_plan_w with W = 64). */
int orc_encode64_fill(int64_t n, const int64_t *rowptr, const int32_t *col, const uint64_t *field,
                      int32_t C, int32_t sigma, int32_t D, int64_t k_left, const int32_t *perm,
                      const int64_t *offset, uint64_t *pack)
{
    int64_t S = (n + C - 1) / C;
    memset(pack, 0, sizeof(uint64_t) * (size_t)offset[S]);
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C, orig = (i / sigma) * sigma + perm[i];
        int64_t prev = orc_left_offset(i, sigma, k_left), j = 0;
        for (int64_t p = rowptr[orig]; p < rowptr[orig + 1]; ++p) {
            int64_t d = (int64_t)col[p] - prev;
            if (d < 0) return ORC_ERR_ARG;
            if (d >= ((int64_t)1 << D)) {
                pack[offset[k] + j * C + l] = (uint64_t)d << 1;
                ++j;
                d = 0;
            }
            pack[offset[k] + j * C + l] = field[p] | ((uint64_t)d << 1) | 1u;
            ++j;
            prev = col[p];
        }
        if (offset[k] + j * C > offset[k + 1]) return ORC_ERR_ARG;
    }
    return ORC_OK;
}

/* 64-bit words back to CSR in original row order (as orc_decode). */
int orc_decode64(int64_t n, int32_t C, int32_t sigma, int32_t D, int64_t k_left,
                 const int32_t *perm, const int64_t *offset, const uint64_t *pack,
                 const int64_t *rowptr, int32_t *col_out, uint64_t *field_out, int64_t *counts)
{
    const uint64_t low = ((uint64_t)2 << D) - 1; /* flag and delta bits */
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C, orig = (i / sigma) * sigma + perm[i];
        int64_t w = (offset[k + 1] - offset[k]) / C;
        int64_t c = orc_left_offset(i, sigma, k_left), q = rowptr[orig], cnt = 0;
        for (int64_t j = 0; j < w; ++j) {
            const uint64_t wd = pack[offset[k] + j * C + l];
            if (wd & 1u) {
                c += (int64_t)((wd >> 1) & (((uint64_t)1 << D) - 1));
                if (q < rowptr[orig + 1]) { col_out[q] = (int32_t)c; field_out[q] = wd & ~low; }
                ++q;
                ++cnt;
            } else {
                c += (int64_t)(wd >> 1);
            }
        }
        counts[orig] = cnt;
    }
    return ORC_OK;
}

/* y = A x by the §4.4 algorithm over 64-bit words in double: per storage row,
 * walk the slice's words, add every delta to the column, and for a word with
 * a value add v * x_c with one fused multiply-add (fma(), correctly rounded),
 * starting from +0, in stored order. y in original row order, or storage
 * order with explicit_order. */
void orc_packsell64_spmv_f64(int64_t n, int32_t C, int32_t sigma, int32_t D, int64_t k_left,
                             const int32_t *perm, const int64_t *offset, const uint64_t *pack,
                             const double *x, double *y, int explicit_order)
{
    const uint64_t low = ((uint64_t)2 << D) - 1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C;
        int64_t w = (offset[k + 1] - offset[k]) / C;
        int64_t c = orc_left_offset(i, sigma, k_left);
        double t = 0.0;
        for (int64_t j = 0; j < w; ++j) {
            const uint64_t wd = pack[offset[k] + j * C + l];
            if (wd & 1u) {
                c += (int64_t)((wd >> 1) & (((uint64_t)1 << D) - 1));
                t = fma(orc_e11my_value(wd & ~low), x[c], t);
            } else {
                c += (int64_t)(wd >> 1);
            }
        }
        y[explicit_order ? i : (i / sigma) * sigma + perm[i]] = t;
    }
}

/* y = A x in double, one fused multiply-add per nonzero in column order from
 * +0: the result of one thread walking one row's 64-bit words. */
void orc_csr_spmv_fma_f64(int64_t n, const int64_t *rowptr, const int32_t *col,
                          const double *val, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) t = fma(val[p], x[col[p]], t);
        y[i] = t;
    }
}

/* 16-bit words (W = 16, D = 7): a word with a value is (code << 8) | (d << 1)
 * | 1 with the E4M3 code in bits 8..15; a dummy is (q << 1), q < 2^15; padding
 * is 0. Same slice layout and plan as the 32-bit words (orc_encode_plan_w with
 * W = 16). codes[nnz]: each nonzero's E4M3 code in CSR order. */
int orc_encode16_fill(int64_t n, const int64_t *rowptr, const int32_t *col, const uint8_t *codes,
                      int32_t C, int32_t sigma, int64_t k_left, const int32_t *perm,
                      const int64_t *offset, uint16_t *pack)
{
    const int D = 7;
    const int64_t dmax = 32767;
    int64_t S = (n + C - 1) / C;
    memset(pack, 0, sizeof(uint16_t) * (size_t)offset[S]);
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C, orig = (i / sigma) * sigma + perm[i];
        int64_t prev = orc_left_offset(i, sigma, k_left), j = 0;
        for (int64_t p = rowptr[orig]; p < rowptr[orig + 1]; ++p) {
            int64_t d = (int64_t)col[p] - prev;
            if (d < 0) return ORC_ERR_ARG;
            while (d >= ((int64_t)1 << D)) {
                int64_t q = d < dmax ? d : dmax;
                pack[offset[k] + j * C + l] = (uint16_t)(q << 1);
                ++j;
                d -= q;
            }
            pack[offset[k] + j * C + l] = (uint16_t)(((uint32_t)codes[p] << 8) | ((uint32_t)d << 1) | 1u);
            ++j;
            prev = col[p];
        }
        if (offset[k] + j * C > offset[k + 1]) return ORC_ERR_ARG;
    }
    return ORC_OK;
}

/* Decode 16-bit words back to CSR in original row order (as orc_decode). */
int orc_decode16(int64_t n, int32_t C, int32_t sigma, int64_t k_left, const int32_t *perm,
                 const int64_t *offset, const uint16_t *pack, const int64_t *rowptr,
                 int32_t *col_out, uint8_t *code_out, int64_t *counts)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C, orig = (i / sigma) * sigma + perm[i];
        int64_t w = (offset[k + 1] - offset[k]) / C;
        int64_t c = orc_left_offset(i, sigma, k_left), q = rowptr[orig], cnt = 0;
        for (int64_t j = 0; j < w; ++j) {
            uint16_t word = pack[offset[k] + j * C + l];
            if (word & 1u) {
                c += (word >> 1) & 0x7Fu;
                if (q < rowptr[orig + 1]) { col_out[q] = (int32_t)c; code_out[q] = (uint8_t)(word >> 8); }
                ++q;
                ++cnt;
            } else {
                c += (word >> 1) & 0x7FFFu;
            }
        }
        counts[orig] = cnt;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SpMV                                                                       */
/* ------------------------------------------------------------------------ */

/* y = A x in double over CSR (y_i = sum_j a_ij x_j, CSR order). */
void orc_csr_spmv_f64(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                      const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double t = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) t += val[p] * x[col[p]];
        y[i] = t;
    }
}

/* y = A x in single precision with one fused multiply-add per nonzero in CSR
 * (= stored) order, starting from +0. This is exactly what a thread that owns
 * one row and walks its packed words in order computes. */
void orc_csr_spmv_fma_f32(int64_t n, const int64_t *rowptr, const int32_t *col,
                          const float *val, const float *x, float *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        float t = 0.0f;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) t = fmaf(val[p], x[col[p]], t);
        y[i] = t;
    }
}

/* dx = A^T dy in double. */
void orc_csr_spmv_t_f64(int64_t n, int64_t m, const int64_t *rowptr, const int32_t *col,
                        const double *val, const double *dy, double *dx)
{
    for (int64_t j = 0; j < m; ++j) dx[j] = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) dx[col[p]] += val[p] * dy[i];
}

/* Y = A X in double, X row-major [m x k] (leading dimension ldx), Y [n x k]. */
void orc_csr_spmm_f64(int64_t n, int64_t k, const int64_t *rowptr, const int32_t *col,
                      const double *val, const double *X, int64_t ldx, double *Y, int64_t ldy)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t r = 0; r < k; ++r) Y[i * ldy + r] = 0.0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
            for (int64_t r = 0; r < k; ++r) Y[i * ldy + r] += val[p] * X[(int64_t)col[p] * ldx + r];
    }
}

/* The paper's PackSELL SpMV algorithm (§4.4) run over packed words, in double:
 * for each storage row i, c starts at the left offset, every word adds its
 * delta to c, and every word that carries a value adds value * x_c.
 * explicit_order != 0 writes y in storage order, else in original order. */
void orc_packsell_spmv_f64(int64_t n, int32_t C, int32_t sigma, int32_t D, int32_t fmt,
                           int64_t k_left, const int32_t *perm, const int64_t *offset,
                           const uint32_t *pack, const double *x, double *y, int explicit_order,
                           int32_t value_exp)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = i / C, l = i % C;
        int64_t iout = explicit_order ? i : (i / sigma) * sigma + perm[i];
        int64_t s = offset[k], w = (offset[k + 1] - s) / C;
        int64_t c = orc_left_offset(i, sigma, k_left);
        double t = 0.0;
        for (int64_t j = 0; j < w; ++j) {
            uint32_t flag, delta, fld;
            orc_unpack(pack[s + j * C + l], D, &flag, &delta, &fld);
            c += delta;
            if (flag)
                t += (fmt == ORC_FMT_FIXED ? orc_fixed_value(fld, D, value_exp)
                                           : orc_field_value(fld, fmt)) * x[c];
        }
        y[iout] = t;
    }
}

/* Quantize nnz values into value fields and their working-precision values.
 * Returns the first error, with its index in *bad (or -1). */
int orc_quantize(int64_t nnz, const double *val, int32_t fmt, int32_t D, uint32_t *field,
                 double *deq, int64_t *bad)
{
    *bad = -1;
    for (int64_t p = 0; p < nnz; ++p) {
        int st = orc_value_field(val[p], fmt, D, &field[p]);
        if (st) { *bad = p; return st; }
        deq[p] = orc_field_value(field[p], fmt);
    }
    return ORC_OK;
}

/* E11MY fields (binary64 patterns) and their values of nnz values. */
int orc_quantize_e11my(int64_t nnz, const double *val, int32_t D, uint64_t *field, double *deq,
                       int64_t *bad)
{
    *bad = -1;
    for (int64_t p = 0; p < nnz; ++p) {
        int st = orc_e11my_bits(val[p], D, &field[p]);
        if (st) { *bad = p; return st; }
        deq[p] = orc_e11my_value(field[p]);
    }
    return ORC_OK;
}

/* Set the number of threads of the OpenMP loops above (timing of the host
 * baseline on one core and on all cores; no effect without OpenMP). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Number of threads the OpenMP loops above use (1 without OpenMP). */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
