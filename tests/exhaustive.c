/*
 * Exhaustive sweeps over FP32 bit patterns for the quantizer pins and the
 * GPU quantizer parity test. Test code: compiled by the tests themselves
 * (gcc, OpenMP), never by the library.
 *
 * The oracle's quantizer (orc_value_field) is passed in as a function pointer,
 * so the arithmetic under test stays in the oracle; this file holds only
 * - two routes of its own that reach the same results by a different path
 *   (integer arithmetic on the FP32 bits), used to pin the oracle, and
 * - loops that compare the oracle with those routes or with fields computed
 *   on the GPU, counting mismatches and remembering the first one.
 */
#include <stdint.h>
#include <string.h>

typedef int (*field_fn)(double v, int fmt, int D, uint32_t *field);

enum { OK = 0, ERR_NONFINITE = 3, ERR_RANGE = 4 };
enum { FMT_FP16 = 1, FMT_E8MY = 2 };

static float from_bits(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }

/* E8MY by integer rounding: adding half a grid step (2^D units of the last
 * place) to the magnitude bits and clearing the low D + 1 bits rounds half
 * away from zero; a carry out of the fraction moves into the exponent by
 * itself, and the result overflows when it reaches the Inf pattern. */
static int route_e8my(uint32_t b, int D, uint32_t *out)
{
    const uint32_t mag = b & 0x7FFFFFFFu;
    if (mag >= 0x7F800000u) return ERR_NONFINITE;
    const uint64_t r = ((uint64_t)mag + (1ull << D)) & ~((2ull << D) - 1ull);
    if (r >= 0x7F800000ull) return ERR_RANGE;
    *out = (b & 0x80000000u) | (uint32_t)r;
    return OK;
}

/* binary16 by integer rounding on the FP32 fields. An FP32 value with biased
 * exponent e and significand M (implicit bit included) is M * 2^(e - 150);
 * in units of binary16's step for the same binade it is M >> s with s = 13 for
 * binary16 normals (e >= 113) and s = 126 - e below (subnormal step 2^-24).
 * Round the shifted-out bits to nearest, ties to even. The binary16 pattern
 * is then (e - 112) << 10 plus the rounded fraction for normals, where a
 * carry into bit 10 steps the exponent; results at or above 0x7C00 overflow. */
static int route_f16(uint32_t b, uint32_t *out)
{
    const uint32_t sign = (b >> 16) & 0x8000u;
    const uint32_t e = (b >> 23) & 0xFFu, f = b & 0x7FFFFFu;
    if (e == 0xFFu) return ERR_NONFINITE;
    uint32_t h;
    if (e >= 113) {
        const uint32_t keep = f >> 13, rest = f & 0x1FFFu;
        h = ((e - 112) << 10) + keep;
        if (rest > 0x1000u || (rest == 0x1000u && (keep & 1u))) h += 1;
        if (h >= 0x7C00u) return ERR_RANGE;
    } else {
        const uint64_t M = e ? (f | 0x800000u) : f;      /* FP32 subnormals: no implicit bit */
        const int s = e ? 126 - (int)e : 125;            /* e = 0 has the scale of e = 1 */
        if (s >= 64) {
            h = 0;
        } else {
            const uint64_t keep = M >> s, rest = M & ((1ull << s) - 1ull), half = 1ull << (s - 1);
            h = (uint32_t)keep;
            if (rest > half || (rest == half && (keep & 1u))) h += 1;
        }
    }
    *out = (sign | h) << 16;
    return OK;
}

/* Patterns [lo, hi): oracle against the integer route of format fmt.
 * Non-finite inputs must give ERR_NONFINITE on both sides, overflow
 * ERR_RANGE on both sides, everything else the same field.
 * Returns the number of mismatches; *first_bad = the smallest one (or ~0). */
int64_t sweep_route(field_fn orc, int fmt, int D, uint64_t lo, uint64_t hi, uint64_t *first_bad)
{
    int64_t bad = 0;
    uint64_t first = ~0ull;
#pragma omp parallel for schedule(static, 1 << 16) reduction(+ : bad) reduction(min : first)
    for (int64_t i = (int64_t)lo; i < (int64_t)hi; ++i) {
        const uint32_t b = (uint32_t)i;
        uint32_t fo = 0, fr = 0;
        const int so = orc((double)from_bits(b), fmt, D, &fo);
        const int sr = fmt == FMT_FP16 ? route_f16(b, &fr) : route_e8my(b, D, &fr);
        if (so != sr || (so == OK && fo != fr)) {
            ++bad;
            if ((uint64_t)i < first) first = (uint64_t)i;
        }
    }
    *first_bad = first;
    return bad;
}

/* Patterns lo + i, i < n: oracle field against dev[i], a field the GPU
 * computed for the same pattern (the caller passes only patterns the GPU
 * quantised without error). Returns the number of mismatches. */
int64_t compare_fields(field_fn orc, int fmt, int D, uint64_t lo, int64_t n, const uint32_t *dev,
                       uint64_t *first_bad)
{
    int64_t bad = 0;
    uint64_t first = ~0ull;
#pragma omp parallel for schedule(static, 1 << 16) reduction(+ : bad) reduction(min : first)
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t b = (uint32_t)(lo + (uint64_t)i);
        uint32_t fo = 0;
        const int so = orc((double)from_bits(b), fmt, D, &fo);
        if (so != OK || fo != dev[i]) {
            ++bad;
            if (lo + (uint64_t)i < first) first = lo + (uint64_t)i;
        }
    }
    *first_bad = first;
    return bad;
}
