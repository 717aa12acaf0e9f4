/*
 * oracle.c -- plain, slow FP64 reference of OpenFFT's 3-D C2C method.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU
 * baseline leg of bench.py load this library.  It shares no code, header,
 * table or helper with the CUDA path in paper_1501_07350_gb300/, and the
 * product path never loads it.
 *
 * What each part follows (Duy & Ozaki, "Performance Tuning of a Parallel 3-D
 * FFT Package OpenFFT"):
 *   - Eq. 1       row-major map of a 3-D point to a 1-D index;
 *   - Eq. 2       the partition function f(N1,N2,N3,Np,myid);
 *   - Eqs. 3-4    block distribution x^s = f(id), x^e = f(id+1)-1;
 *   - Eqs. 5-7    translation of x^s / x^e back to 3-D coordinates;
 *   - Eqs. 8-9    the 2-D (pencil) form taken when N1 < Np <= N1*N2;
 *   - Sec. 2      transpose order abc -> cab -> cba;
 *   - Sec. 3.1.1  execution: per rank copy a line out, 1-D FFT, copy back;
 *                 pack a send buffer per destination, communicate, unpack
 *                 and merge into the next decomposition.
 *
 * Readings where the paper is silent:
 *   - stage s transforms the fastest axis of its ordering: c in abc, b in
 *     cab, a in cba (each rank owns complete lines of that axis);
 *   - the degree (1-D or 2-D) is chosen per ordering from its own leading
 *     dimensions; Np > N1*N2 is undefined by Eq. 2 and is rejected;
 *   - forward = exp(-2 pi i ...), unnormalised; backward = exp(+2 pi i ...)
 *     with a final division by N, input in cba order, output in abc order,
 *     axes transformed a, b, c;
 *   - inside a send segment, elements are kept in ascending source index;
 *   - real transforms (future work in the paper): the real abc array is
 *     decomposed with (Na, Nb, Nc), the complex half arrays of the later
 *     stages with Nc replaced by Nc/2 + 1; the inverse keeps the real part of
 *     the inverse DFT of the half spectrum extended by Hermitian symmetry
 *     along c.
 *
 * Arithmetic: plain double, no compensated sums, so the FFT error grows like
 * u*log(n).  Twiddles are evaluated in long double and rounded once.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { double re, im; } cplx;

static const long double PI_L = 3.141592653589793238462643383279502884L;

/* ---------------------------------------------------------------- Eq. 2 -- */

/* Start offset of process `id` in the 1-D order of an (N1,N2,N3) ordering.
 * Returns -1 where Eq. 2 is undefined (Np > N1*N2 or bad arguments). */
int64_t oracle_f(int64_t N1, int64_t N2, int64_t N3, int64_t Np, int64_t id)
{
    if (N1 < 1 || N2 < 1 || N3 < 1 || Np < 1 || id < 0 || id > Np) return -1;
    if (Np <= N1) return ((N1 * id) / Np) * N2 * N3;           /* 1-D slabs   */
    if (Np <= N1 * N2) return ((N1 * N2 * id) / Np) * N3;      /* 2-D pencils */
    return -1;
}

/* Eqs. 3-4 for all ranks: xs[id] = f(id) for id = 0..Np (so x^e = xs[id+1]-1). */
int oracle_boundaries(int64_t N1, int64_t N2, int64_t N3, int64_t Np, int64_t* xs)
{
    for (int64_t id = 0; id <= Np; ++id) {
        xs[id] = oracle_f(N1, N2, N3, Np, id);
        if (xs[id] < 0) return -1;
    }
    return 0;
}

/* Eqs. 5-7: 1-D index -> (a,b,c) coordinates of the (N1,N2,N3) ordering. */
void oracle_to3d(int64_t N1, int64_t N2, int64_t N3, int64_t x, int64_t abc[3])
{
    (void)N1;
    int64_t a = x / (N2 * N3);
    int64_t b = (x - a * N2 * N3) / N3;
    int64_t c = x - a * N2 * N3 - b * N3;
    abc[0] = a; abc[1] = b; abc[2] = c;
}

/* Box of rank `id`: x^s, x^e (Eqs. 3-4) and their 3-D coordinates (Eqs. 5-7). */
int oracle_box(int64_t N1, int64_t N2, int64_t N3, int64_t Np, int64_t id,
               int64_t* xs, int64_t* xe, int64_t start3[3], int64_t end3[3])
{
    int64_t s = oracle_f(N1, N2, N3, Np, id);
    int64_t e = oracle_f(N1, N2, N3, Np, id + 1);
    if (s < 0 || e < 0) return -1;
    *xs = s;
    *xe = e - 1;
    oracle_to3d(N1, N2, N3, s, start3);
    if (e - 1 >= s) oracle_to3d(N1, N2, N3, e - 1, end3);
    else { end3[0] = end3[1] = end3[2] = -1; }   /* empty box */
    return 0;
}

/* Degree of an ordering: 1 = slabs (Np <= N1), 2 = pencils, -1 undefined. */
int oracle_degree(int64_t N1, int64_t N2, int64_t Np)
{
    if (Np <= N1) return 1;
    if (Np <= N1 * N2) return 2;
    return -1;
}

/* ------------------------------------------------------------ orderings -- */

/* Layout codes: 0 = abc, 1 = cab, 2 = cba (slowest axis first).  axis[i] is
 * the original axis (0=a, 1=b, 2=c) that is the i-th dimension of the layout. */
static void layout_axes(int layout, int axis[3])
{
    static const int tab[3][3] = {{0, 1, 2}, {2, 0, 1}, {2, 1, 0}};
    axis[0] = tab[layout][0]; axis[1] = tab[layout][1]; axis[2] = tab[layout][2];
}

static void layout_dims(int layout, const int64_t n[3], int64_t D[3])
{
    int axis[3];
    layout_axes(layout, axis);
    D[0] = n[axis[0]]; D[1] = n[axis[1]]; D[2] = n[axis[2]];
}

/* Eq. 1 applied to the layout: point (v[0]=a, v[1]=b, v[2]=c) -> 1-D index. */
static int64_t layout_index(int layout, const int64_t n[3], const int64_t v[3])
{
    int axis[3]; int64_t D[3];
    layout_axes(layout, axis);
    layout_dims(layout, n, D);
    return (v[axis[0]] * D[1] + v[axis[1]]) * D[2] + v[axis[2]];
}

/* 1-D index in the layout -> point (a,b,c), by Eqs. 5-7. */
static void layout_point(int layout, const int64_t n[3], int64_t x, int64_t v[3])
{
    int axis[3]; int64_t D[3], d[3];
    layout_axes(layout, axis);
    layout_dims(layout, n, D);
    oracle_to3d(D[0], D[1], D[2], x, d);
    v[axis[0]] = d[0]; v[axis[1]] = d[1]; v[axis[2]] = d[2];
}

/* Owner of 1-D index y: the rank whose [x^s, x^e] holds it, by bisection over
 * the ascending boundaries xs[0..Np]. */
static int64_t owner_of(const int64_t* xs, int64_t Np, int64_t y)
{
    int64_t lo = 0, hi = Np - 1;           /* invariant: xs[lo] <= y < xs[hi+1] */
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (xs[mid] <= y) lo = mid; else hi = mid - 1;
    }
    return lo;
}

/* ------------------------------------------------------- 1-D FFT engine -- */

/* Table W[e] = exp(sign * 2 pi i e / n), e = 0..n-1, in long double, rounded. */
static cplx* make_table(int64_t n, int sign)
{
    cplx* W = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    for (int64_t e = 0; e < n; ++e) {
        long double ang = 2.0L * PI_L * (long double)e / (long double)n;
        W[e].re = (double)cosl(ang);
        W[e].im = (double)((long double)sign * sinl(ang));
    }
    return W;
}

static inline cplx cmul(cplx a, cplx b)
{
    cplx r;
    r.re = a.re * b.re - a.im * b.im;
    r.im = a.re * b.im + a.im * b.re;
    return r;
}

static int is_prime(int64_t n)
{
    if (n < 2) return 0;
    for (int64_t p = 2; p * p <= n; ++p) if (n % p == 0) return 0;
    return 1;
}

/* Radix of one decimation-in-time split: 4, then 2, 3, 5, else the smallest
 * prime factor; 0 means "take the direct DFT" (n <= 5 or n prime). */
static int64_t choose_radix(int64_t n)
{
    if (n <= 5 || is_prime(n)) return 0;
    if (n % 4 == 0) return 4;
    if (n % 2 == 0) return 2;
    if (n % 3 == 0) return 3;
    if (n % 5 == 0) return 5;
    for (int64_t p = 7; p <= n; ++p) if (n % p == 0) return p;
    return 0;
}

/* y[0..n) = DFT_n of x[0], x[stride], ...; W is the table of length Wn, and
 * W_n^e = W[e * (Wn / n)].  Recursive decimation in time:
 *   X[k + q m] = sum_j W_r^{j q} (W_n^{j k} Y_j[k]),   n = r m,
 * where Y_j is the m-point DFT of the subsequence x[j + r t]. */
static void fft_rec(int64_t n, const cplx* x, int64_t stride, cplx* y,
                    const cplx* W, int64_t Wn)
{
    int64_t step = Wn / n;
    if (n == 1) { y[0] = x[0]; return; }
    int64_t r = choose_radix(n);
    if (r == 0) {                                      /* direct DFT */
        for (int64_t k = 0; k < n; ++k) {
            cplx acc = {0.0, 0.0};
            for (int64_t j = 0; j < n; ++j) {
                cplx t = cmul(x[j * stride], W[((j * k) % n) * step]);
                acc.re += t.re; acc.im += t.im;
            }
            y[k] = acc;
        }
        return;
    }
    int64_t m = n / r;
    for (int64_t j = 0; j < r; ++j)
        fft_rec(m, x + j * stride, stride * r, y + j * m, W, Wn);
    cplx* t = (cplx*)malloc(sizeof(cplx) * (size_t)(2 * r));
    cplx* z = t + r;
    for (int64_t k = 0; k < m; ++k) {
        for (int64_t j = 0; j < r; ++j)
            t[j] = cmul(y[j * m + k], W[((j * k) % n) * step]);
        for (int64_t q = 0; q < r; ++q) {
            cplx acc = {0.0, 0.0};
            for (int64_t j = 0; j < r; ++j) {
                /* W_r^{jq} = W_n^{jq m} */
                cplx u = cmul(t[j], W[(((j * q) % r) * m) * step]);
                acc.re += u.re; acc.im += u.im;
            }
            z[q] = acc;
        }
        for (int64_t q = 0; q < r; ++q) y[k + q * m] = z[q];
    }
    free(t);
}

/* Unnormalised 1-D DFT of length n with exponent sign `sign` (-1 forward). */
void oracle_fft1d(int64_t n, const cplx* x, cplx* y, int sign)
{
    cplx* W = make_table(n, sign);
    fft_rec(n, x, 1, y, W, n);
    free(W);
}

/* Brute-force O(n^2) DFT, long double accumulation (pins oracle_fft1d). */
void oracle_dft1d_brute(int64_t n, const cplx* x, cplx* y, int sign)
{
    for (int64_t k = 0; k < n; ++k) {
        long double sr = 0.0L, si = 0.0L;
        for (int64_t j = 0; j < n; ++j) {
            long double ang = 2.0L * PI_L * (long double)((j * k) % n) / (long double)n;
            long double c = cosl(ang), s = (long double)sign * sinl(ang);
            sr += (long double)x[j].re * c - (long double)x[j].im * s;
            si += (long double)x[j].re * s + (long double)x[j].im * c;
        }
        y[k].re = (double)sr; y[k].im = (double)si;
    }
}

/* Brute-force O(N^2) 3-D DFT on A[a][b][c] (abc order), output X[ka][kb][kc]
 * in the same order, long double accumulation.  Phase index is reduced
 * exactly in integers: t = (a ka mod Na) N/Na + (b kb mod Nb) N/Nb + ... */
void oracle_dft3d_brute(int64_t Na, int64_t Nb, int64_t Nc, const cplx* A, cplx* X, int sign)
{
    int64_t N = Na * Nb * Nc;
    for (int64_t ka = 0; ka < Na; ++ka)
    for (int64_t kb = 0; kb < Nb; ++kb)
    for (int64_t kc = 0; kc < Nc; ++kc) {
        long double sr = 0.0L, si = 0.0L;
        for (int64_t a = 0; a < Na; ++a)
        for (int64_t b = 0; b < Nb; ++b)
        for (int64_t c = 0; c < Nc; ++c) {
            int64_t t = ((a * ka) % Na) * (N / Na) + ((b * kb) % Nb) * (N / Nb)
                      + ((c * kc) % Nc) * (N / Nc);
            t %= N;
            long double ang = 2.0L * PI_L * (long double)t / (long double)N;
            long double cr = cosl(ang), ci = (long double)sign * sinl(ang);
            const cplx v = A[(a * Nb + b) * Nc + c];
            sr += (long double)v.re * cr - (long double)v.im * ci;
            si += (long double)v.re * ci + (long double)v.im * cr;
        }
        X[(ka * Nb + kb) * Nc + kc].re = (double)sr;
        X[(ka * Nb + kb) * Nc + kc].im = (double)si;
    }
}

/* One output line of the 3-D DFT by its definition, summed axis by axis:
 *   X[ka,kb,kc] = sum_a W_a^{a ka} sum_b W_b^{b kb} sum_c W_c^{c kc} A[a,b,c],
 * for all ka at fixed (kb,kc).  O(N) work, used to sample full-size outputs. */
void oracle_dft3d_line(int64_t Na, int64_t Nb, int64_t Nc, const cplx* A, int sign,
                       int64_t kb, int64_t kc, cplx* line)
{
    cplx* Wa = make_table(Na, sign);
    cplx* Wb = make_table(Nb, sign);
    cplx* Wc = make_table(Nc, sign);
    cplx* s = (cplx*)malloc(sizeof(cplx) * (size_t)Na);
    for (int64_t a = 0; a < Na; ++a) {
        cplx sb = {0.0, 0.0};
        for (int64_t b = 0; b < Nb; ++b) {
            cplx sc = {0.0, 0.0};
            const cplx* row = A + (a * Nb + b) * Nc;
            for (int64_t c = 0; c < Nc; ++c) {
                cplx t = cmul(row[c], Wc[(c * kc) % Nc]);
                sc.re += t.re; sc.im += t.im;
            }
            cplx t = cmul(sc, Wb[(b * kb) % Nb]);
            sb.re += t.re; sb.im += t.im;
        }
        s[a] = sb;
    }
    for (int64_t ka = 0; ka < Na; ++ka) {
        cplx acc = {0.0, 0.0};
        for (int64_t a = 0; a < Na; ++a) {
            cplx t = cmul(s[a], Wa[(a * ka) % Na]);
            acc.re += t.re; acc.im += t.im;
        }
        line[ka] = acc;
    }
    free(Wa); free(Wb); free(Wc); free(s);
}

/* ------------------------------------------------- redistribution steps -- */

/* Steps (4)-(6) of the execution flow for one transpose, literally:
 * every source rank r packs, in ascending source index, the (destination
 * index, value) pairs of its box into one segment per destination rank s;
 * the segments are communicated (copied into the receive buffer of s, in
 * order of source rank); every destination rank unpacks its receive buffer
 * into its box of the next ordering.  C[r*Np+s] receives the element count
 * of segment (r, s).  Returns 0, or -1 on an undefined decomposition / an
 * element that would land outside the receiver's box. */
static int redistribute(int src_layout, int dst_layout, const int64_t n[3], int64_t Np,
                        const cplx* src, cplx* dst, int64_t* C)
{
    int64_t Ds[3], Dd[3];
    layout_dims(src_layout, n, Ds);
    layout_dims(dst_layout, n, Dd);
    int64_t N = n[0] * n[1] * n[2];
    int64_t* xs_src = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    int64_t* xs_dst = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    if (oracle_boundaries(Ds[0], Ds[1], Ds[2], Np, xs_src) ||
        oracle_boundaries(Dd[0], Dd[1], Dd[2], Np, xs_dst)) {
        free(xs_src); free(xs_dst);
        return -1;
    }
    int64_t* cnt = (int64_t*)calloc((size_t)(Np * Np), sizeof(int64_t));
    /* count: which destination each source element goes to */
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t x = xs_src[r]; x < xs_src[r + 1]; ++x) {
            int64_t v[3];
            layout_point(src_layout, n, x, v);
            int64_t y = layout_index(dst_layout, n, v);
            cnt[r * Np + owner_of(xs_dst, Np, y)] += 1;
        }
    /* send displacements: rank r's send buffer spans [xs_src[r], xs_src[r+1]) */
    int64_t* sdispl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np * Np));
    int64_t* rdispl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np * Np));
    for (int64_t r = 0; r < Np; ++r) {
        int64_t off = xs_src[r];
        for (int64_t s = 0; s < Np; ++s) { sdispl[r * Np + s] = off; off += cnt[r * Np + s]; }
    }
    /* receive displacements: rank s's receive buffer spans [xs_dst[s], xs_dst[s+1]) */
    for (int64_t s = 0; s < Np; ++s) {
        int64_t off = xs_dst[s];
        for (int64_t r = 0; r < Np; ++r) { rdispl[s * Np + r] = off; off += cnt[r * Np + s]; }
    }
    /* (4) pack */
    int64_t* sidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    cplx* sval = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    int64_t* fill = (int64_t*)calloc((size_t)(Np * Np), sizeof(int64_t));
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t x = xs_src[r]; x < xs_src[r + 1]; ++x) {
            int64_t v[3];
            layout_point(src_layout, n, x, v);
            int64_t y = layout_index(dst_layout, n, v);
            int64_t s = owner_of(xs_dst, Np, y);
            int64_t pos = sdispl[r * Np + s] + fill[r * Np + s]++;
            sidx[pos] = y;
            sval[pos] = src[x];
        }
    /* (5) communicate */
    int64_t* ridx = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    cplx* rval = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    for (int64_t s = 0; s < Np; ++s)
        for (int64_t r = 0; r < Np; ++r) {
            int64_t len = cnt[r * Np + s];
            memcpy(ridx + rdispl[s * Np + r], sidx + sdispl[r * Np + s], sizeof(int64_t) * (size_t)len);
            memcpy(rval + rdispl[s * Np + r], sval + sdispl[r * Np + s], sizeof(cplx) * (size_t)len);
        }
    /* (6) unpack into the receiver's box */
    int bad = 0;
    for (int64_t s = 0; s < Np; ++s)
        for (int64_t p = xs_dst[s]; p < xs_dst[s + 1]; ++p) {
            int64_t y = ridx[p];
            if (y < xs_dst[s] || y >= xs_dst[s + 1]) { bad = 1; continue; }
            dst[y] = rval[p];
        }
    if (C) memcpy(C, cnt, sizeof(int64_t) * (size_t)(Np * Np));
    free(xs_src); free(xs_dst); free(cnt); free(sdispl); free(rdispl);
    free(sidx); free(sval); free(fill); free(ridx); free(rval);
    return bad ? -1 : 0;
}

/* Transpose alone.  which: 1 = abc->cab, 2 = cab->cba, -2 = cba->cab,
 * -1 = cab->abc.  C (Np*Np, may be NULL) receives the count matrix. */
int oracle_redistribute(int64_t Na, int64_t Nb, int64_t Nc, int64_t Np, int which,
                        const cplx* src, cplx* dst, int64_t* C)
{
    const int64_t n[3] = {Na, Nb, Nc};
    switch (which) {
    case 1:  return redistribute(0, 1, n, Np, src, dst, C);
    case 2:  return redistribute(1, 2, n, Np, src, dst, C);
    case -2: return redistribute(2, 1, n, Np, src, dst, C);
    case -1: return redistribute(1, 0, n, Np, src, dst, C);
    default: return -1;
    }
}

/* Steps (1)-(3): every rank copies each complete line of the fastest axis of
 * its box into a line buffer, transforms it, and copies it back. */
static int transform_stage(int layout, const int64_t n[3], int64_t Np, cplx* data, int sign)
{
    int64_t D[3];
    layout_dims(layout, n, D);
    int64_t* xs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    if (oracle_boundaries(D[0], D[1], D[2], Np, xs)) { free(xs); return -1; }
    int64_t len = D[2];
    cplx* W = make_table(len, sign);
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)len);
    cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)len);
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t x = xs[r]; x < xs[r + 1]; x += len) {        /* box = whole lines */
            memcpy(buf, data + x, sizeof(cplx) * (size_t)len);    /* (1) */
            fft_rec(len, buf, 1, res, W, len);                    /* (2) */
            memcpy(data + x, res, sizeof(cplx) * (size_t)len);    /* (3) */
        }
    free(W); free(buf); free(res); free(xs);
    return 0;
}

/* ---------------------------------------------- real transforms (R2C) -- */

/* A real 3-D transform keeps the kc <= Nc/2 half of the spectrum: the rest
 * follows from X[-ka,-kb,-kc] = conj X[ka,kb,kc].  The paper names real
 * transforms as future work only.  Reading taken: the real abc array is
 * decomposed by Eqs. 2-9 with (Na, Nb, Nc) and the complex arrays of the
 * later stages by the same equations with Nc replaced by Nch = Nc/2 + 1
 * (integer division): cab (Nch, Na, Nb), cba (Nch, Nb, Na).  Rank boxes are
 * whole c-lines in both the real array and the half array, so a rank keeps
 * the same lines across the first stage. */

/* Stage 1, forward: every rank copies each real c-line of its box into a
 * complex line buffer (imaginary parts 0), takes the 1-D DFT and keeps
 * frequencies 0..Nch-1 as that line of the half array [Na][Nb][Nch]. */
static int real_stage_forward(int64_t Na, int64_t Nb, int64_t Nc, int64_t Np, const double* x, cplx* half)
{
    const int64_t Nch = Nc / 2 + 1;
    int64_t* xs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    if (oracle_boundaries(Na, Nb, Nc, Np, xs)) { free(xs); return -1; }
    cplx* W = make_table(Nc, -1);
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)Nc);
    cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)Nc);
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t xx = xs[r]; xx < xs[r + 1]; xx += Nc) {
            const int64_t l = xx / Nc;                             /* line (a, b) */
            for (int64_t i = 0; i < Nc; ++i) { buf[i].re = x[xx + i]; buf[i].im = 0.0; }
            fft_rec(Nc, buf, 1, res, W, Nc);
            memcpy(half + l * Nch, res, sizeof(cplx) * (size_t)Nch);
        }
    free(W); free(buf); free(res); free(xs);
    return 0;
}

/* Last stage of the inverse: each c-line of the half array [Na][Nb][Nch] is
 * extended to the full spectrum, Z[k] = conj Z[Nc - k] for k >= Nch; the
 * inverse DFT is taken and its real part kept (so only the real parts of
 * Z[0] and, for even Nc, of Z[Nc/2] count). */
static int real_stage_backward(int64_t Na, int64_t Nb, int64_t Nc, int64_t Np, const cplx* half, double* x)
{
    const int64_t Nch = Nc / 2 + 1;
    int64_t* xs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    if (oracle_boundaries(Na, Nb, Nc, Np, xs)) { free(xs); return -1; }
    cplx* W = make_table(Nc, 1);
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)Nc);
    cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)Nc);
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t xx = xs[r]; xx < xs[r + 1]; xx += Nc) {
            const int64_t l = xx / Nc;
            for (int64_t k = 0; k < Nc; ++k) {
                if (k < Nch) buf[k] = half[l * Nch + k];
                else { buf[k].re = half[l * Nch + Nc - k].re; buf[k].im = -half[l * Nch + Nc - k].im; }
            }
            fft_rec(Nc, buf, 1, res, W, Nc);
            for (int64_t i = 0; i < Nc; ++i) x[xx + i] = res[i].re;
        }
    free(W); free(buf); free(res); free(xs);
    return 0;
}

/* Real 3-D transform under the decomposition.
 *   dir = -1: in = real abc array (Na*Nb*Nc doubles), out = half spectrum in
 *             cba order [Nch][Nb][Na]; stages c (real), b, a.
 *   dir = +1: in = half spectrum in cba order, out = real abc array divided
 *             by N = Na*Nb*Nc; stages a, b, c (real).
 * C1, C2 (may be NULL): count matrices of the two transposes of the half
 * array. */
int oracle_rfft3d(int64_t Na, int64_t Nb, int64_t Nc, int64_t Np, int dir,
                  const void* in, void* out, int64_t* C1, int64_t* C2)
{
    const int64_t Nch = Nc / 2 + 1;
    const int64_t nh[3] = {Na, Nb, Nch};
    const int64_t M = Na * Nb * Nch, N = Na * Nb * Nc;
    if (dir != -1 && dir != 1) return -1;
    cplx* t0 = (cplx*)malloc(sizeof(cplx) * (size_t)M);
    cplx* t1 = (cplx*)malloc(sizeof(cplx) * (size_t)M);
    int rc = 0;
    if (dir == -1) {
        rc |= real_stage_forward(Na, Nb, Nc, Np, (const double*)in, t0);   /* along c, real */
        rc |= redistribute(0, 1, nh, Np, t0, t1, C1);                     /* abc -> cab    */
        rc |= transform_stage(1, nh, Np, t1, -1);                         /* along b       */
        rc |= redistribute(1, 2, nh, Np, t1, t0, C2);                     /* cab -> cba    */
        rc |= transform_stage(2, nh, Np, t0, -1);                         /* along a       */
        memcpy(out, t0, sizeof(cplx) * (size_t)M);
    } else {
        memcpy(t0, in, sizeof(cplx) * (size_t)M);
        rc |= transform_stage(2, nh, Np, t0, 1);                          /* along a       */
        rc |= redistribute(2, 1, nh, Np, t0, t1, C1);                     /* cba -> cab    */
        rc |= transform_stage(1, nh, Np, t1, 1);                          /* along b       */
        rc |= redistribute(1, 0, nh, Np, t1, t0, C2);                     /* cab -> abc    */
        double* x = (double*)out;
        rc |= real_stage_backward(Na, Nb, Nc, Np, t0, x);                 /* along c, real */
        for (int64_t i = 0; i < N; ++i) x[i] /= (double)N;
    }
    free(t0); free(t1);
    return rc ? -1 : 0;
}

/* Full 3-D C2C transform under the decomposition.
 *   dir = -1 (forward): in = abc order, out = cba order; stages c, b, a.
 *   dir = +1 (backward): in = cba order, out = abc order; stages a, b, c,
 *                        then division by N.
 * C1 / C2 (Np*Np each, may be NULL) receive the count matrices of the first
 * and second transpose of this direction.  Returns 0 or -1. */
int oracle_fft3d(int64_t Na, int64_t Nb, int64_t Nc, int64_t Np, int dir,
                 const cplx* in, cplx* out, int64_t* C1, int64_t* C2)
{
    const int64_t n[3] = {Na, Nb, Nc};
    int64_t N = Na * Nb * Nc;
    if (dir != -1 && dir != 1) return -1;
    cplx* t0 = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    cplx* t1 = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    memcpy(t0, in, sizeof(cplx) * (size_t)N);
    int rc = 0;
    if (dir == -1) {
        rc |= transform_stage(0, n, Np, t0, -1);             /* along c in abc */
        rc |= redistribute(0, 1, n, Np, t0, t1, C1);         /* abc -> cab     */
        rc |= transform_stage(1, n, Np, t1, -1);             /* along b in cab */
        rc |= redistribute(1, 2, n, Np, t1, t0, C2);         /* cab -> cba     */
        rc |= transform_stage(2, n, Np, t0, -1);             /* along a in cba */
        memcpy(out, t0, sizeof(cplx) * (size_t)N);
    } else {
        rc |= transform_stage(2, n, Np, t0, 1);              /* along a in cba */
        rc |= redistribute(2, 1, n, Np, t0, t1, C1);         /* cba -> cab     */
        rc |= transform_stage(1, n, Np, t1, 1);              /* along b in cab */
        rc |= redistribute(1, 0, n, Np, t1, t0, C2);         /* cab -> abc     */
        rc |= transform_stage(0, n, Np, t0, 1);              /* along c in abc */
        for (int64_t i = 0; i < N; ++i) {
            out[i].re = t0[i].re / (double)N;
            out[i].im = t0[i].im / (double)N;
        }
    }
    free(t0); free(t1);
    return rc ? -1 : 0;
}

/* ============================================= D-dimensional transforms == */

/* The paper cites 4-D and 5-D transforms under the same decomposition (Sec. 1)
 * without giving their transpose orders.  Reading taken (generalising the
 * 3-D order abc -> cab -> cba of Sec. 2): for A[N_1]...[N_D] (axis d_D
 * fastest), ordering s = 1..D is
 *     (d_D, d_{D-1}, ..., d_{D-s+2}, d_1, d_2, ..., d_{D-s+1}),
 * i.e. each transpose moves the axis just transformed (the fastest) behind
 * the axes moved before it.  Stage s transforms the fastest axis of
 * ordering s; the forward result is left in ordering D (d_D ... d_1, i.e.
 * the reversed axes); the backward transform runs the orderings in reverse
 * and divides by N.  Each ordering is decomposed by Eqs. 2-9 with
 * (N1, N2, N3) = (its first dimension, its second, the product of the
 * rest): the row-wise 1-D translation of Eq. 1 with the trailing axes
 * collapsed, so every rank holds whole lines of the fastest axis. */

#define ORACLE_MAX_DIMS 8

/* axes[j] = the original axis (0 = d_1) at position j of ordering s */
static void nd_axes(int D, int s, int axes[])
{
    int k = 0;
    for (int i = 0; i < s - 1; ++i) axes[k++] = D - 1 - i;
    for (int i = 0; i < D - s + 1; ++i) axes[k++] = i;
}

/* Eqs. 2-4 of ordering s: boundaries xs[0..Np] (returns -1 if undefined) */
static int nd_boundaries(int D, const int64_t* n, int s, int64_t Np, int64_t* xs)
{
    int axes[ORACLE_MAX_DIMS];
    nd_axes(D, s, axes);
    int64_t rest = 1;
    for (int j = 2; j < D; ++j) rest *= n[axes[j]];
    return oracle_boundaries(n[axes[0]], n[axes[1]], rest, Np, xs);
}

/* Eq. 1 in ordering s: coordinates v (per original axis) -> 1-D index */
static int64_t nd_index(int D, const int64_t* n, int s, const int64_t* v)
{
    int axes[ORACLE_MAX_DIMS];
    nd_axes(D, s, axes);
    int64_t x = 0;
    for (int j = 0; j < D; ++j) x = x * n[axes[j]] + v[axes[j]];
    return x;
}

/* the inverse: 1-D index of ordering s -> coordinates */
static void nd_point(int D, const int64_t* n, int s, int64_t x, int64_t* v)
{
    int axes[ORACLE_MAX_DIMS];
    nd_axes(D, s, axes);
    for (int j = D - 1; j >= 0; --j) {
        v[axes[j]] = x % n[axes[j]];
        x /= n[axes[j]];
    }
}

/* Steps (1)-(3) in ordering s: every rank transforms the complete lines of
 * the fastest axis of its box. */
static int nd_transform_stage(int D, const int64_t* n, int s, int64_t Np, cplx* data, int sign)
{
    int axes[ORACLE_MAX_DIMS];
    nd_axes(D, s, axes);
    int64_t* xs = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    if (nd_boundaries(D, n, s, Np, xs)) { free(xs); return -1; }
    int64_t len = n[axes[D - 1]];
    cplx* W = make_table(len, sign);
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)len);
    cplx* res = (cplx*)malloc(sizeof(cplx) * (size_t)len);
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t x = xs[r]; x < xs[r + 1]; x += len) {
            memcpy(buf, data + x, sizeof(cplx) * (size_t)len);
            fft_rec(len, buf, 1, res, W, len);
            memcpy(data + x, res, sizeof(cplx) * (size_t)len);
        }
    free(W); free(buf); free(res); free(xs);
    return 0;
}

/* Steps (4)-(6) from ordering s_src to ordering s_dst, literally: pack per
 * destination rank in ascending source index, communicate in order of
 * source rank, unpack.  C[r*Np+s] receives the counts. */
static int nd_redistribute(int D, const int64_t* n, int s_src, int s_dst, int64_t Np,
                           const cplx* src, cplx* dst, int64_t* C)
{
    int64_t N = 1;
    for (int j = 0; j < D; ++j) N *= n[j];
    int64_t* xs_src = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    int64_t* xs_dst = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np + 1));
    if (nd_boundaries(D, n, s_src, Np, xs_src) || nd_boundaries(D, n, s_dst, Np, xs_dst)) {
        free(xs_src); free(xs_dst);
        return -1;
    }
    int64_t* cnt = (int64_t*)calloc((size_t)(Np * Np), sizeof(int64_t));
    int64_t v[ORACLE_MAX_DIMS];
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t x = xs_src[r]; x < xs_src[r + 1]; ++x) {
            nd_point(D, n, s_src, x, v);
            cnt[r * Np + owner_of(xs_dst, Np, nd_index(D, n, s_dst, v))] += 1;
        }
    int64_t* sdispl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np * Np));
    int64_t* rdispl = (int64_t*)malloc(sizeof(int64_t) * (size_t)(Np * Np));
    for (int64_t r = 0; r < Np; ++r) {
        int64_t off = xs_src[r];
        for (int64_t s = 0; s < Np; ++s) { sdispl[r * Np + s] = off; off += cnt[r * Np + s]; }
    }
    for (int64_t s = 0; s < Np; ++s) {
        int64_t off = xs_dst[s];
        for (int64_t r = 0; r < Np; ++r) { rdispl[s * Np + r] = off; off += cnt[r * Np + s]; }
    }
    /* (4) pack */
    int64_t* sidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    cplx* sval = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    int64_t* fill = (int64_t*)calloc((size_t)(Np * Np), sizeof(int64_t));
    for (int64_t r = 0; r < Np; ++r)
        for (int64_t x = xs_src[r]; x < xs_src[r + 1]; ++x) {
            nd_point(D, n, s_src, x, v);
            int64_t y = nd_index(D, n, s_dst, v);
            int64_t s = owner_of(xs_dst, Np, y);
            int64_t pos = sdispl[r * Np + s] + fill[r * Np + s]++;
            sidx[pos] = y;
            sval[pos] = src[x];
        }
    /* (5) communicate */
    int64_t* ridx = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    cplx* rval = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    for (int64_t s = 0; s < Np; ++s)
        for (int64_t r = 0; r < Np; ++r) {
            int64_t len = cnt[r * Np + s];
            memcpy(ridx + rdispl[s * Np + r], sidx + sdispl[r * Np + s], sizeof(int64_t) * (size_t)len);
            memcpy(rval + rdispl[s * Np + r], sval + sdispl[r * Np + s], sizeof(cplx) * (size_t)len);
        }
    /* (6) unpack */
    int bad = 0;
    for (int64_t s = 0; s < Np; ++s)
        for (int64_t p = xs_dst[s]; p < xs_dst[s + 1]; ++p) {
            int64_t y = ridx[p];
            if (y < xs_dst[s] || y >= xs_dst[s + 1]) { bad = 1; continue; }
            dst[y] = rval[p];
        }
    if (C) memcpy(C, cnt, sizeof(int64_t) * (size_t)(Np * Np));
    free(xs_src); free(xs_dst); free(cnt); free(sdispl); free(rdispl);
    free(sidx); free(sval); free(fill); free(ridx); free(rval);
    return bad ? -1 : 0;
}

/* Eqs. 2-4 of ordering s (1..D) of a D-dimensional array: xs[0..Np]. */
int oracle_nd_boundaries(int D, const int64_t* n, int s, int64_t Np, int64_t* xs)
{
    if (D < 2 || D > ORACLE_MAX_DIMS || s < 1 || s > D) return -1;
    return nd_boundaries(D, n, s, Np, xs);
}

/* One transpose alone: ordering s -> s + 1 (step > 0) or s + 1 -> s. */
int oracle_nd_redistribute(int D, const int64_t* n, int64_t Np, int s, int forward,
                           const cplx* src, cplx* dst, int64_t* C)
{
    if (D < 3 || D > ORACLE_MAX_DIMS || s < 1 || s >= D) return -1;
    return forward ? nd_redistribute(D, n, s, s + 1, Np, src, dst, C)
                   : nd_redistribute(D, n, s + 1, s, Np, src, dst, C);
}

/* The whole D-dimensional transform under the decomposition over Np ranks.
 * dir = -1: A in ordering 1 (the array as given), result in ordering D;
 * dir = +1: A in ordering D, result in ordering 1, divided by N. */
int oracle_fftnd(int D, const int64_t* n, int64_t Np, int dir, const cplx* in, cplx* out)
{
    if (D < 3 || D > ORACLE_MAX_DIMS || (dir != -1 && dir != 1)) return -1;
    int64_t N = 1;
    for (int j = 0; j < D; ++j) N *= n[j];
    cplx* t0 = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    cplx* t1 = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    memcpy(t0, in, sizeof(cplx) * (size_t)N);
    int rc = 0;
    if (dir == -1) {
        for (int s = 1; s <= D; ++s) {
            rc |= nd_transform_stage(D, n, s, Np, t0, -1);
            if (s < D) {
                rc |= nd_redistribute(D, n, s, s + 1, Np, t0, t1, NULL);
                cplx* t = t0; t0 = t1; t1 = t;
            }
        }
        memcpy(out, t0, sizeof(cplx) * (size_t)N);
    } else {
        for (int s = D; s >= 1; --s) {
            rc |= nd_transform_stage(D, n, s, Np, t0, 1);
            if (s > 1) {
                rc |= nd_redistribute(D, n, s, s - 1, Np, t0, t1, NULL);
                cplx* t = t0; t0 = t1; t1 = t;
            }
        }
        const double count = (double)N;
        for (int64_t i = 0; i < N; ++i) {
            out[i].re = t0[i].re / count;
            out[i].im = t0[i].im / count;
        }
    }
    free(t0); free(t1);
    return rc ? -1 : 0;
}
