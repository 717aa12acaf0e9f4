// decomp.h -- closed-form index arithmetic of OpenFFT's decomposition
// (Duy & Ozaki, Sec. 2, Eqs. 1-9), usable from host and device code.
//
// An "ordering" is one of abc = [Na][Nb][Nc], cab = [Nc][Na][Nb],
// cba = [Nc][Nb][Na] (slowest first).  For ordering dims (D0, D1, D2):
//   Eq. 2  f(r) = floor(D0 r / P) D1 D2       if P <= D0        (slabs)
//               = floor(D0 D1 r / P) D2       if D0 < P <= D0 D1 (pencils)
// Every box is a whole number of rows of length D2, so the decomposition is
// described by row boundaries rb(r) = f(r) / D2 = floor(M r / P) * U with
// (M, U) = (D0, D1) for slabs and (D0 D1, 1) for pencils.  The owner of row
// q is the closed-form inverse floor(((q/U) + 1) P - 1) / M).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define DHD __host__ __device__ __forceinline__
#else
#define DHD inline
#endif

namespace ofg {

enum Layout { ABC = 0, CAB = 1, CBA = 2 };

struct Ordering {
    int64_t D0, D1, D2;   // dims, slowest first
    int64_t M, U;         // rows are grouped in units of U; M units in total
    int64_t P;
    int degree;           // 1 = slabs, 2 = pencils, -1 undefined
};

DHD Ordering make_ordering(int64_t D0, int64_t D1, int64_t D2, int64_t P)
{
    Ordering o;
    o.D0 = D0; o.D1 = D1; o.D2 = D2; o.P = P;
    if (P <= D0) { o.degree = 1; o.M = D0; o.U = D1; }
    else if (P <= D0 * D1) { o.degree = 2; o.M = D0 * D1; o.U = 1; }
    else { o.degree = -1; o.M = 1; o.U = 1; }
    return o;
}

DHD Ordering ordering_of(int layout, int64_t Na, int64_t Nb, int64_t Nc, int64_t P)
{
    if (layout == ABC) return make_ordering(Na, Nb, Nc, P);
    if (layout == CAB) return make_ordering(Nc, Na, Nb, P);
    return make_ordering(Nc, Nb, Na, P);
}

// First row of rank r (r = 0..P); rank r owns rows [row_begin(r), row_begin(r+1)).
DHD int64_t row_begin(const Ordering& o, int64_t r) { return ((o.M * r) / o.P) * o.U; }

// Eq. 2 / Eqs. 3-4: first 1-D index of rank r.
DHD int64_t box_begin(const Ordering& o, int64_t r) { return row_begin(o, r) * o.D2; }

// Rank owning row q (closed-form inverse of row_begin).
DHD int64_t row_owner(const Ordering& o, int64_t q)
{
    int64_t u = q / o.U;
    return ((u + 1) * o.P - 1) / o.M;
}

DHD int64_t clamp0(int64_t v, int64_t hi) { return v < 0 ? 0 : (v > hi ? hi : v); }

// |[Q0, Q1) intersect [lo, hi)|
DHD int64_t overlap(int64_t Q0, int64_t Q1, int64_t lo, int64_t hi)
{
    int64_t a = Q0 > lo ? Q0 : lo;
    int64_t b = Q1 < hi ? Q1 : hi;
    return b > a ? b - a : 0;
}

// #{q in [0, Q) : q mod m < a}
DHD int64_t count_mod_below(int64_t Q, int64_t m, int64_t a)
{
    int64_t rem = Q % m;
    return (Q / m) * a + (rem < a ? rem : a);
}

// ---------------------------------------------------------------------------
// Transposes.  Each is described from the SOURCE ordering's point of view:
// a source row q (length Ls) holds elements e = 0..Ls-1; the element goes to
// destination row dq(q, e) whose owner is the receiving rank.  For each
// transpose the destination row of element e is an affine function of e with
// unit slope inside a "block" of source rows, which gives closed forms for
// counts and for positions inside a send segment (ascending source index).
//
//   R1  abc -> cab : src row q = a Nb + b (elements c), dst row c Na + a
//   R2  cab -> cba : src row q = c Na + a (elements b), dst row c Nb + b
//   R2' cba -> cab : src row q = c Nb + b (elements a), dst row c Na + a
//   R1' cab -> abc : src row q = c Na + a (elements b), dst row a Nb + b
// ---------------------------------------------------------------------------

struct Transpose {
    int which;                 // 1, 2, -2, -1
    int64_t Na, Nb, Nc;
    Ordering src, dst;
};

DHD Transpose make_transpose(int which, int64_t Na, int64_t Nb, int64_t Nc, int64_t P)
{
    Transpose t;
    t.which = which; t.Na = Na; t.Nb = Nb; t.Nc = Nc;
    int sl = which == 1 ? ABC : (which == 2 ? CAB : (which == -2 ? CBA : CAB));
    int dl = which == 1 ? CAB : (which == 2 ? CBA : (which == -2 ? CAB : ABC));
    t.src = ordering_of(sl, Na, Nb, Nc, P);
    t.dst = ordering_of(dl, Na, Nb, Nc, P);
    return t;
}

// Destination 1-D index of source element (row q, element e).
DHD int64_t dest_index(const Transpose& t, int64_t q, int64_t e)
{
    switch (t.which) {
    case 1: { int64_t a = q / t.Nb, b = q - a * t.Nb; return ((e * t.Na + a) * t.Nb) + b; }
    case 2: { int64_t c = q / t.Na, a = q - c * t.Na; return ((c * t.Nb + e) * t.Na) + a; }
    case -2: { int64_t c = q / t.Nb, b = q - c * t.Nb; return ((c * t.Na + e) * t.Nb) + b; }
    default: { int64_t c = q / t.Na, a = q - c * t.Na; return ((a * t.Nb + e) * t.Nc) + c; }
    }
}

// Inverse: destination 1-D index y -> (source row, element).
DHD void source_of(const Transpose& t, int64_t y, int64_t* q, int64_t* e)
{
    switch (t.which) {
    case 1: {   // y in cab: (c, a, b)
        int64_t b = y % t.Nb, ca = y / t.Nb, a = ca % t.Na, c = ca / t.Na;
        *q = a * t.Nb + b; *e = c; return; }
    case 2: {   // y in cba: (c, b, a)
        int64_t a = y % t.Na, cb = y / t.Na, b = cb % t.Nb, c = cb / t.Nb;
        *q = c * t.Na + a; *e = b; return; }
    case -2: {  // y in cab: (c, a, b)
        int64_t b = y % t.Nb, ca = y / t.Nb, a = ca % t.Na, c = ca / t.Na;
        *q = c * t.Nb + b; *e = a; return; }
    default: {  // y in abc: (a, b, c)
        int64_t c = y % t.Nc, ab = y / t.Nc, b = ab % t.Nb, a = ab / t.Nb;
        *q = c * t.Na + a; *e = b; return; }
    }
}

// For destination rank s with rows [Q0, Q1) and a source row q: the elements
// of row q that go to s form the contiguous range [e_lo, e_lo + cnt).
// `w` is the number of elements per source row.
DHD void row_range(const Transpose& t, int64_t q, int64_t Q0, int64_t Q1,
                   int64_t* e_lo, int64_t* cnt)
{
    switch (t.which) {
    case 1: {   // dst row = e Na + a, e in [0, Nc): stride Na
        int64_t a = q / t.Nb;
        int64_t lo = Q0 - a <= 0 ? 0 : (Q0 - a + t.Na - 1) / t.Na;
        int64_t hi = Q1 - a <= 0 ? 0 : (Q1 - a + t.Na - 1) / t.Na;
        if (hi > t.Nc) hi = t.Nc;
        if (lo > hi) lo = hi;
        *e_lo = lo; *cnt = hi - lo; return; }
    case 2: {   // dst row = c Nb + e, e in [0, Nb)
        int64_t c = q / t.Na;
        int64_t lo = Q0 - c * t.Nb, hi = Q1 - c * t.Nb;
        lo = clamp0(lo, t.Nb); hi = clamp0(hi, t.Nb);
        *e_lo = lo; *cnt = hi > lo ? hi - lo : 0; return; }
    case -2: {  // dst row = c Na + e, e in [0, Na)
        int64_t c = q / t.Nb;
        int64_t lo = Q0 - c * t.Na, hi = Q1 - c * t.Na;
        lo = clamp0(lo, t.Na); hi = clamp0(hi, t.Na);
        *e_lo = lo; *cnt = hi > lo ? hi - lo : 0; return; }
    default: {  // dst row = a Nb + e, e in [0, Nb)
        int64_t a = q % t.Na;
        int64_t lo = Q0 - a * t.Nb, hi = Q1 - a * t.Nb;
        lo = clamp0(lo, t.Nb); hi = clamp0(hi, t.Nb);
        *e_lo = lo; *cnt = hi > lo ? hi - lo : 0; return; }
    }
}

// F(q) = sum over source rows q' < q of (elements of q' going to rows [Q0,Q1)).
DHD int64_t prefix_to(const Transpose& t, int64_t q, int64_t Q0, int64_t Q1)
{
    switch (t.which) {
    case 1: {   // per-row count depends on a = q / Nb; H(a) = #{y in [Q0,Q1): y mod Na < a}
        int64_t a = q / t.Nb, rem = q - a * t.Nb;
        int64_t Ha = count_mod_below(Q1, t.Na, a) - count_mod_below(Q0, t.Na, a);
        int64_t Ha1 = count_mod_below(Q1, t.Na, a + 1) - count_mod_below(Q0, t.Na, a + 1);
        return t.Nb * Ha + rem * (Ha1 - Ha); }
    case 2: {   // per-row count depends on c = q / Na: |[Q0,Q1) n [c Nb, (c+1) Nb)|
        int64_t c = q / t.Na, rem = q - c * t.Na;
        return t.Na * overlap(Q0, Q1, 0, c * t.Nb) + rem * overlap(Q0, Q1, c * t.Nb, (c + 1) * t.Nb); }
    case -2: {  // per-row count depends on c = q / Nb: |[Q0,Q1) n [c Na, (c+1) Na)|
        int64_t c = q / t.Nb, rem = q - c * t.Nb;
        return t.Nb * overlap(Q0, Q1, 0, c * t.Na) + rem * overlap(Q0, Q1, c * t.Na, (c + 1) * t.Na); }
    default: {  // per-row count depends on a = q mod Na: |[Q0,Q1) n [a Nb, (a+1) Nb)|
        int64_t c = q / t.Na, a = q - c * t.Na;
        return c * overlap(Q0, Q1, 0, t.Na * t.Nb) + overlap(Q0, Q1, 0, a * t.Nb); }
    }
}

// Count of elements sent by source rank r to destination rank s (Sec. 4.1 volume).
DHD int64_t pair_count(const Transpose& t, int64_t r, int64_t s)
{
    int64_t R0 = row_begin(t.src, r), R1 = row_begin(t.src, r + 1);
    int64_t Q0 = row_begin(t.dst, s), Q1 = row_begin(t.dst, s + 1);
    return prefix_to(t, R1, Q0, Q1) - prefix_to(t, R0, Q0, Q1);
}

// Elements per source row.
DHD int64_t row_len(const Transpose& t) { return t.src.D2; }
// Elements per destination row.
DHD int64_t dst_row_len(const Transpose& t) { return t.dst.D2; }

}  // namespace ofg
