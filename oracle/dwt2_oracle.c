/* dwt2_oracle.c -- plain, slow CPU oracle for the 2-D DWT by lifting.
 *
 * TEST INFRASTRUCTURE ONLY: it is called by the tests, the smoke check and the benchmark's
 * CPU-baseline leg, never by the product path.  It shares no code with the CUDA library.
 *
 * Arithmetic: the float wavelets in double (fp64); the reversible CDF 5/3 in exact int64 with
 * an explicit floor division (never C truncation).  Every routine works on plain arrays with
 * loops written the way the paper states the steps; nothing is blocked, fused or reordered.
 *
 * Sources, by routine:
 *   line_step_*        one 1-D lifting step of Eq. 2 (Sec. 2): predict d += P(s), update s += U(d)
 *   sep_level_*        separable 2-D lifting, steps P, P*, U, U* per lifting pair (Eq. 3)
 *   nonsep_*           spatial predict / spatial update steps of the non-separable scheme (Eq. 5)
 *   *_inverse_*        the same steps undone in reverse order (the inverse of each matrix)
 *   *_adj_*            the transpose of each step, applied in reverse order
 *   orc_forward etc.   the multi-level (Mallat) recursion on LL cited in Sec. 2
 * Readings where the paper is silent (wavelet constants, 9/7 normalisation, integer rounding,
 * boundary handling, length-1 axes) are stated next to the code that takes them.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "dwt2_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------
 * Wavelet constants.  The paper evaluates CDF 5/3 (Sec. 1, Sec. 4) without printing its
 * coefficients and claims the schemes hold for any wavelet (Sec. 1, Sec. 5).
 *   CDF 5/3: P(z) = -1/2 (1 + z), U(z) = 1/4 (1 + z^-1), no scaling.
 *   CDF 9/7: the Daubechies-Sweldens factorisation into two lifting pairs (the lifting
 *            factorisation of Eq. 2), followed by scaling low-pass by 1/K and high-pass by K/2,
 *            which gives the low-pass a DC gain of 1 and the high-pass a Nyquist gain of 1.
 *   Reversible CDF 5/3: d = x_o - floor((x_e + x_e') / 2), s = x_e + floor((d' + d + 2) / 4).
 *   Deslauriers-Dubuc 9/7 and 13/7 (interpolating wavelets, no scaling): the predict is the
 *            cubic interpolation of the odd sample from its four even neighbours,
 *            d[m] = x[2m+1] - (9/16 (s[m] + s[m+1]) - 1/16 (s[m-1] + s[m+2])), so the high
 *            pass vanishes on cubics; the update is half the predict's transpose,
 *            s[m] += 1/4 (d[m-1] + d[m]) for 9/7 (two vanishing moments of the low pass at
 *            Nyquist) and s[m] += 9/32 (d[m-1] + d[m]) - 1/32 (d[m-2] + d[m+1]) for 13/7 (four).
 *            Each step has an inner tap pair (distance 1 in the interleaved signal) and an outer
 *            one (distance 3); the CDF wavelets have no outer pair.
 * ---------------------------------------------------------------------------------------- */
static const double C53_P = -0.5;
static const double C53_U = 0.25;
static const double C97_ALPHA = -1.586134342059924;
static const double C97_BETA = -0.052980118572961;
static const double C97_GAMMA = 0.882911075530934;
static const double C97_DELTA = 0.443506852043971;
static const double C97_K = 1.230174104914001;

typedef struct {
    int npairs;
    double p[2], u[2];   /* inner tap pair of each predict / update */
    double p3[2], u3[2]; /* outer tap pair (0 for the CDF wavelets) */
} lifting_t;

static int get_lifting(int wavelet, lifting_t* L) {
    L->p3[0] = L->p3[1] = L->u3[0] = L->u3[1] = 0.0;
    switch (wavelet) {
    case ORC_CDF53_INT: /* coefficients only used for their structure; arithmetic is integer */
    case ORC_CDF53:
        L->npairs = 1;
        L->p[0] = C53_P;
        L->u[0] = C53_U;
        return 0;
    case ORC_CDF97:
        L->npairs = 2;
        L->p[0] = C97_ALPHA;
        L->u[0] = C97_BETA;
        L->p[1] = C97_GAMMA;
        L->u[1] = C97_DELTA;
        return 0;
    case ORC_DD97:
    case ORC_DD137:
        L->npairs = 1;
        L->p[0] = -9.0 / 16.0;
        L->p3[0] = 1.0 / 16.0;
        L->u[0] = wavelet == ORC_DD97 ? 0.25 : 9.0 / 32.0;
        L->u3[0] = wavelet == ORC_DD97 ? 0.0 : -1.0 / 32.0;
        return 0;
    default:
        return -1;
    }
}

/* Scale of one axis after the lifting pairs (CDF 9/7 only): even (low) samples 1/K, odd (high)
 * samples K/2.  An axis of length 1 is passed through and therefore not scaled. */
static double axis_scale(int wavelet, long n, long parity) {
    if (wavelet != ORC_CDF97 || n < 2) return 1.0;
    return parity ? C97_K / 2.0 : 1.0 / C97_K;
}

/* floor(a / b) for b > 0, written out (C '/' truncates toward zero). */
static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b, r = a % b;
    return (r < 0) ? q - 1 : q;
}

/* Whole-sample symmetric reflection of one index just outside [0, n): x[-1] = x[1],
 * x[n] = x[n-2].  Valid for -1 <= i <= n and n >= 2. */
static long refl1(long i, long n) {
    if (i < 0) return -i;
    if (i >= n) return 2 * (n - 1) - i;
    return i;
}

/* Whole-sample symmetric extension of any index: the signal repeated with period 2n-2 and
 * mirrored about samples 0 and n-1 (repeated reflection, for signals shorter than the
 * extension). */
static long refl_any(long i, long n) {
    if (n == 1) return 0;
    long p = 2 * n - 2;
    i %= p;
    if (i < 0) i += p;
    return i >= n ? p - i : i;
}

/* ------------------------------------------------------------------------------------------
 * One 1-D lifting step (Eq. 2) on the line v[0], v[s], ..., v[(n-1)s].
 * parity 1 = predict: every odd sample i gets coef * (v[i-1] + v[i+1]);
 * parity 0 = update:  every even sample i gets coef * (v[i-1] + v[i+1]).
 * mirror = 1: neighbours outside the line are the whole-sample reflections (refl1).
 * mirror = 0: samples with a neighbour outside the line are left unchanged (used on a signal
 *             that has already been extended far enough).
 * A line of length 1 has no odd sample and passes through.
 * ---------------------------------------------------------------------------------------- */
static void line_step_f(double* v, long n, long s, int parity, double coef, double coef3,
                        int mirror) {
    if (n < 2) return;
    for (long i = parity; i < n; i += 2) {
        long l = i - 1, r = i + 1;
        if (coef3 == 0.0) {
            if (!mirror && (l < 0 || r >= n)) continue;
            l = refl1(l, n);
            r = refl1(r, n);
            v[i * s] += coef * (v[l * s] + v[r * s]);
        } else {
            /* the outer pair at distance 3 (Deslauriers-Dubuc): reflections of any depth */
            long l3 = i - 3, r3 = i + 3;
            if (!mirror && (l3 < 0 || r3 >= n)) continue;
            v[i * s] += coef * (v[refl_any(l, n) * s] + v[refl_any(r, n) * s]) +
                        coef3 * (v[refl_any(l3, n) * s] + v[refl_any(r3, n) * s]);
        }
    }
}

/* Integer step: predict v[i] -= floor((v[i-1] + v[i+1]) / 2),
 *               update  v[i] += floor((v[i-1] + v[i+1] + 2) / 4);
 * sign = -1 undoes the step (same floor expression, opposite sign). */
static void line_step_i(int64_t* v, long n, long s, int parity, int sign, int mirror) {
    if (n < 2) return;
    for (long i = parity; i < n; i += 2) {
        long l = i - 1, r = i + 1;
        if (!mirror && (l < 0 || r >= n)) continue;
        l = refl1(l, n);
        r = refl1(r, n);
        if (parity)
            v[i * s] -= sign * floor_div(v[l * s] + v[r * s], 2);
        else
            v[i * s] += sign * floor_div(v[l * s] + v[r * s] + 2, 4);
    }
}

/* Transpose of line_step_f: the step reads v[l], v[r] and adds to v[i]; its transpose adds
 * coef * g[i] to g[l] and to g[r] and leaves g[i] alone (a mirrored tap read twice adds twice). */
static void line_step_adj_f(double* g, long n, long s, int parity, double coef) {
    if (n < 2) return;
    for (long i = parity; i < n; i += 2) {
        long l = refl1(i - 1, n), r = refl1(i + 1, n);
        g[l * s] += coef * g[i * s];
        g[r * s] += coef * g[i * s];
    }
}

/* A step along every row (horizontal, the paper's P / U) or every column (vertical, P* / U*).
 * The lines of one step are independent (a line step reads and writes its own line only), so
 * with more than one thread (orc_set_threads) they are shared out among the threads; each line
 * is still computed by one thread in the same order, so the results do not depend on it. */
enum { AX_ROWS = 0, AX_COLS = 1 };

static void plane_step_f(double* x, long H, long W, int axis, int parity, double coef,
                         double coef3, int mirror) {
    if (axis == AX_ROWS) {
#pragma omp parallel for schedule(static)
        for (long r = 0; r < H; ++r) line_step_f(x + r * W, W, 1, parity, coef, coef3, mirror);
    } else {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < W; ++c) line_step_f(x + c, H, W, parity, coef, coef3, mirror);
    }
}

static void plane_step_i(int64_t* x, long H, long W, int axis, int parity, int sign, int mirror) {
    if (axis == AX_ROWS) {
#pragma omp parallel for schedule(static)
        for (long r = 0; r < H; ++r) line_step_i(x + r * W, W, 1, parity, sign, mirror);
    } else {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < W; ++c) line_step_i(x + c, H, W, parity, sign, mirror);
    }
}

static void plane_step_adj_f(double* g, long H, long W, int axis, int parity, double coef) {
    if (axis == AX_ROWS) {
#pragma omp parallel for schedule(static)
        for (long r = 0; r < H; ++r) line_step_adj_f(g + r * W, W, 1, parity, coef);
    } else {
#pragma omp parallel for schedule(static)
        for (long c = 0; c < W; ++c) line_step_adj_f(g + c, H, W, parity, coef);
    }
}

/* ------------------------------------------------------------------------------------------
 * The ordered list of 2-D lifting steps of one level for a separable scheme.
 * ORC_SEP_EQ3: per lifting pair the four matrices of Eq. 3, rightmost first: P (rows),
 *              P* (columns), U (rows), U* (columns).
 * ORC_SEP_ROWS / ORC_SEP_COLS: the complete 1-D lifting along one axis, then the other
 *              (Sec. 2 notes that horizontal and vertical steps may be interleaved freely).
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int axis, parity;
    double coef, coef3; /* inner and outer tap pair */
} step2d_t;

static int level_steps(int wavelet, int scheme, step2d_t* st) {
    lifting_t L;
    if (get_lifting(wavelet, &L)) return -1;
    int n = 0;
    if (scheme == ORC_SEP_EQ3) {
        for (int k = 0; k < L.npairs; ++k) {
            st[n++] = (step2d_t){AX_ROWS, 1, L.p[k], L.p3[k]};
            st[n++] = (step2d_t){AX_COLS, 1, L.p[k], L.p3[k]};
            st[n++] = (step2d_t){AX_ROWS, 0, L.u[k], L.u3[k]};
            st[n++] = (step2d_t){AX_COLS, 0, L.u[k], L.u3[k]};
        }
    } else if (scheme == ORC_SEP_ROWS || scheme == ORC_SEP_COLS) {
        int first = scheme == ORC_SEP_ROWS ? AX_ROWS : AX_COLS;
        for (int pass = 0; pass < 2; ++pass) {
            int axis = pass == 0 ? first : 1 - first;
            for (int k = 0; k < L.npairs; ++k) {
                st[n++] = (step2d_t){axis, 1, L.p[k], L.p3[k]};
                st[n++] = (step2d_t){axis, 0, L.u[k], L.u3[k]};
            }
        }
    } else {
        return -1;
    }
    return n;
}

/* Band geometry of one level of an h x w plane. */
typedef struct {
    long ner, ndr, nec, ndc; /* even / odd row counts, even / odd column counts */
} geom_t;

static geom_t geom_of(long h, long w) {
    geom_t g = {(h + 1) / 2, h / 2, (w + 1) / 2, w / 2};
    return g;
}

/* Split an interleaved plane into LL, HL, LH, HH (the quad of Sec. 2), applying the 9/7
 * scaling of each axis; join is the exact reverse (dividing by the scaling). */
static void split_f(const double* x, long h, long w, int wavelet, double* LL, double* HL,
                    double* LH, double* HH) {
    geom_t g = geom_of(h, w);
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) {
            double v = x[r * w + c] * axis_scale(wavelet, h, r & 1) * axis_scale(wavelet, w, c & 1);
            long n = r / 2, m = c / 2;
            if (!(r & 1) && !(c & 1)) LL[n * g.nec + m] = v;
            if (!(r & 1) && (c & 1)) HL[n * g.ndc + m] = v;
            if ((r & 1) && !(c & 1)) LH[n * g.nec + m] = v;
            if ((r & 1) && (c & 1)) HH[n * g.ndc + m] = v;
        }
}

static void join_f(const double* LL, const double* HL, const double* LH, const double* HH, long h,
                   long w, int wavelet, int divide, double* x) {
    geom_t g = geom_of(h, w);
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) {
            long n = r / 2, m = c / 2;
            double v;
            if (!(r & 1) && !(c & 1)) v = LL[n * g.nec + m];
            else if (!(r & 1)) v = HL[n * g.ndc + m];
            else if (!(c & 1)) v = LH[n * g.nec + m];
            else v = HH[n * g.ndc + m];
            double s = axis_scale(wavelet, h, r & 1) * axis_scale(wavelet, w, c & 1);
            x[r * w + c] = divide ? v / s : v * s;
        }
}

static void split_i(const int64_t* x, long h, long w, int64_t* LL, int64_t* HL, int64_t* LH,
                    int64_t* HH) {
    geom_t g = geom_of(h, w);
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) {
            int64_t v = x[r * w + c];
            long n = r / 2, m = c / 2;
            if (!(r & 1) && !(c & 1)) LL[n * g.nec + m] = v;
            if (!(r & 1) && (c & 1)) HL[n * g.ndc + m] = v;
            if ((r & 1) && !(c & 1)) LH[n * g.nec + m] = v;
            if ((r & 1) && (c & 1)) HH[n * g.ndc + m] = v;
        }
}

static void join_i(const int64_t* LL, const int64_t* HL, const int64_t* LH, const int64_t* HH,
                   long h, long w, int64_t* x) {
    geom_t g = geom_of(h, w);
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) {
            long n = r / 2, m = c / 2;
            if (!(r & 1) && !(c & 1)) x[r * w + c] = LL[n * g.nec + m];
            else if (!(r & 1)) x[r * w + c] = HL[n * g.ndc + m];
            else if (!(c & 1)) x[r * w + c] = LH[n * g.nec + m];
            else x[r * w + c] = HH[n * g.ndc + m];
        }
}

/* ------------------------------------------------------------------------------------------
 * Separable level, forward (Eq. 3), in place on an interleaved h x w plane.
 * extension_form = 1: extend by 8 samples of whole-sample symmetric extension on each side of
 * every axis longer than 1 (8 is even, so sample parity is kept, and exceeds the reach of the
 * longest wavelet: 4 samples for CDF 9/7, 6 for Deslauriers-Dubuc 13/7), lift with no boundary
 * rule, crop.
 * ---------------------------------------------------------------------------------------- */
#define EXT 8

static int sep_level_fwd_f(double* x, long h, long w, int wavelet, int scheme, int ext) {
    step2d_t st[16];
    int ns = level_steps(wavelet, scheme, st);
    if (ns < 0) return -1;
    if (!ext) {
        for (int k = 0; k < ns; ++k)
            plane_step_f(x, h, w, st[k].axis, st[k].parity, st[k].coef, st[k].coef3, 1);
        return 0;
    }
    long eh = h > 1 ? EXT : 0, ew = w > 1 ? EXT : 0;
    long H2 = h + 2 * eh, W2 = w + 2 * ew;
    double* y = (double*)malloc(sizeof(double) * H2 * W2);
    if (!y) return -2;
    for (long r = 0; r < H2; ++r)
        for (long c = 0; c < W2; ++c)
            y[r * W2 + c] = x[refl_any(r - eh, h) * w + refl_any(c - ew, w)];
    for (int k = 0; k < ns; ++k)
        plane_step_f(y, H2, W2, st[k].axis, st[k].parity, st[k].coef, st[k].coef3, 0);
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) x[r * w + c] = y[(r + eh) * W2 + (c + ew)];
    free(y);
    return 0;
}

static int sep_level_fwd_i(int64_t* x, long h, long w, int scheme, int ext) {
    step2d_t st[16];
    int ns = level_steps(ORC_CDF53_INT, scheme, st);
    if (ns < 0) return -1;
    if (!ext) {
        for (int k = 0; k < ns; ++k) plane_step_i(x, h, w, st[k].axis, st[k].parity, +1, 1);
        return 0;
    }
    long eh = h > 1 ? EXT : 0, ew = w > 1 ? EXT : 0;
    long H2 = h + 2 * eh, W2 = w + 2 * ew;
    int64_t* y = (int64_t*)malloc(sizeof(int64_t) * H2 * W2);
    if (!y) return -2;
    for (long r = 0; r < H2; ++r)
        for (long c = 0; c < W2; ++c)
            y[r * W2 + c] = x[refl_any(r - eh, h) * w + refl_any(c - ew, w)];
    for (int k = 0; k < ns; ++k) plane_step_i(y, H2, W2, st[k].axis, st[k].parity, +1, 0);
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) x[r * w + c] = y[(r + eh) * W2 + (c + ew)];
    free(y);
    return 0;
}

/* Separable level, inverse: the steps of the forward list in reverse order, each undone. */
static int sep_level_inv_f(double* x, long h, long w, int wavelet, int scheme) {
    step2d_t st[16];
    int ns = level_steps(wavelet, scheme, st);
    if (ns < 0) return -1;
    for (int k = ns - 1; k >= 0; --k)
        plane_step_f(x, h, w, st[k].axis, st[k].parity, -st[k].coef, -st[k].coef3, 1);
    return 0;
}

static int sep_level_inv_i(int64_t* x, long h, long w, int scheme) {
    step2d_t st[16];
    int ns = level_steps(ORC_CDF53_INT, scheme, st);
    if (ns < 0) return -1;
    for (int k = ns - 1; k >= 0; --k) plane_step_i(x, h, w, st[k].axis, st[k].parity, -1, 1);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Non-separable lifting (Sec. 3, Eq. 5), on the four polyphase components
 *   a = LL (ner x nec), b = HL (ner x ndc), c = LH (ndr x nec), e = HH (ndr x ndc).
 * Spatial predict  [1 0 0 0; P 1 0 0; P* 0 1 0; PP* P* P 1] and
 * spatial update   [1 U U* UU*; 0 1 0 U*; 0 0 1 U; 0 0 0 1], where P acts along rows
 * (HL[n][m] gets p (a[n][m] + a[n][m+1])), P* along columns, and PP*, UU* are their tensor
 * products.  Boundaries: the whole-sample reflection expressed on polyphase indices --
 *   a predict reading even index m+1 past the end reads index ne-1      (pr),
 *   an update reading odd index m-1 = -1 reads index 0                  (ul),
 *   an update reading odd index m = nd (odd length) reads index nd-1    (ur).
 * ---------------------------------------------------------------------------------------- */
static long pr_(long m, long ne) { return m + 1 < ne ? m + 1 : ne - 1; }
static long ul_(long m) { return m > 0 ? m - 1 : 0; }
static long ur_(long m, long nd) { return m < nd ? m : nd - 1; }

typedef struct {
    geom_t g;
    double *a, *b, *c, *e;
} quad_f_t;

typedef struct {
    geom_t g;
    int64_t *a, *b, *c, *e;
} quad_i_t;

#define A_(q, n, m) (q)->a[(n) * (q)->g.nec + (m)]
#define B_(q, n, m) (q)->b[(n) * (q)->g.ndc + (m)]
#define C_(q, n, m) (q)->c[(n) * (q)->g.nec + (m)]
#define E_(q, n, m) (q)->e[(n) * (q)->g.ndc + (m)]

static double* dup_f(const double* p, long n) {
    double* q = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (q && n > 0) memcpy(q, p, sizeof(double) * n);
    return q;
}

static int64_t* dup_i(const int64_t* p, long n) {
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    if (q && n > 0) memcpy(q, p, sizeof(int64_t) * n);
    return q;
}

/* Spatial predict, float (Eq. 5, right matrix).  Reads the components before the step
 * (copies), writes b, c, e; a is unchanged ("predict is responsible for HH", Sec. 3). */
static void nonsep_predict_f(quad_f_t* q, double p) {
    geom_t g = q->g;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.ndc; ++m)
            B_(q, n, m) = B_(&o, n, m) + p * (A_(&o, n, m) + A_(&o, n, pr_(m, g.nec)));
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.nec; ++m)
            C_(q, n, m) = C_(&o, n, m) + p * (A_(&o, n, m) + A_(&o, pr_(n, g.ner), m));
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) {
            long m1 = pr_(m, g.nec), n1 = pr_(n, g.ner);
            E_(q, n, m) = E_(&o, n, m) + p * (C_(&o, n, m) + C_(&o, n, m1)) +
                          p * (B_(&o, n, m) + B_(&o, n1, m)) +
                          p * p * (A_(&o, n, m) + A_(&o, n, m1) + A_(&o, n1, m) + A_(&o, n1, m1));
        }
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* Spatial update, float (Eq. 5, left matrix); e is unchanged ("update is responsible for LL"). */
static void nonsep_update_f(quad_f_t* q, double u) {
    geom_t g = q->g;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.nec; ++m) {
            double v = A_(&o, n, m);
            long ml = ul_(m), mr = ur_(m, g.ndc), nl = ul_(n), nr = ur_(n, g.ndr);
            if (g.ndc) v += u * (B_(&o, n, ml) + B_(&o, n, mr));
            if (g.ndr) v += u * (C_(&o, nl, m) + C_(&o, nr, m));
            if (g.ndr && g.ndc)
                v += u * u * (E_(&o, nl, ml) + E_(&o, nl, mr) + E_(&o, nr, ml) + E_(&o, nr, mr));
            A_(q, n, m) = v;
        }
    if (g.ndr)
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.ndc; ++m)
                B_(q, n, m) = B_(&o, n, m) + u * (E_(&o, ul_(n), m) + E_(&o, ur_(n, g.ndr), m));
    if (g.ndc)
        for (long n = 0; n < g.ndr; ++n)
            for (long m = 0; m < g.nec; ++m)
                C_(q, n, m) = C_(&o, n, m) + u * (E_(&o, n, ul_(m)) + E_(&o, n, ur_(m, g.ndc)));
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* Inverse spatial update: [1 -U -U* UU*; 0 1 0 -U*; 0 0 1 -U; 0 0 0 1]. */
static void nonsep_update_inv_f(quad_f_t* q, double u) {
    geom_t g = q->g;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.nec; ++m) {
            double v = A_(&o, n, m);
            long ml = ul_(m), mr = ur_(m, g.ndc), nl = ul_(n), nr = ur_(n, g.ndr);
            if (g.ndc) v -= u * (B_(&o, n, ml) + B_(&o, n, mr));
            if (g.ndr) v -= u * (C_(&o, nl, m) + C_(&o, nr, m));
            if (g.ndr && g.ndc)
                v += u * u * (E_(&o, nl, ml) + E_(&o, nl, mr) + E_(&o, nr, ml) + E_(&o, nr, mr));
            A_(q, n, m) = v;
        }
    if (g.ndr)
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.ndc; ++m)
                B_(q, n, m) = B_(&o, n, m) - u * (E_(&o, ul_(n), m) + E_(&o, ur_(n, g.ndr), m));
    if (g.ndc)
        for (long n = 0; n < g.ndr; ++n)
            for (long m = 0; m < g.nec; ++m)
                C_(q, n, m) = C_(&o, n, m) - u * (E_(&o, n, ul_(m)) + E_(&o, n, ur_(m, g.ndc)));
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* Inverse spatial predict: [1 0 0 0; -P 1 0 0; -P* 0 1 0; PP* -P* -P 1]. */
static void nonsep_predict_inv_f(quad_f_t* q, double p) {
    geom_t g = q->g;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.ndc; ++m)
            B_(q, n, m) = B_(&o, n, m) - p * (A_(&o, n, m) + A_(&o, n, pr_(m, g.nec)));
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.nec; ++m)
            C_(q, n, m) = C_(&o, n, m) - p * (A_(&o, n, m) + A_(&o, pr_(n, g.ner), m));
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) {
            long m1 = pr_(m, g.nec), n1 = pr_(n, g.ner);
            E_(q, n, m) = E_(&o, n, m) - p * (B_(&o, n, m) + B_(&o, n1, m)) -
                          p * (C_(&o, n, m) + C_(&o, n, m1)) +
                          p * p * (A_(&o, n, m) + A_(&o, n, m1) + A_(&o, n1, m) + A_(&o, n1, m1));
        }
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* Integer spatial predict.  Sec. 2 allows the horizontal and vertical steps of Eq. 3 to be
 * interleaved in any order, which holds in exact arithmetic but not once every step floors.
 * The fused step therefore reproduces the floors of Eq. 3's order P (rows) then P* (columns):
 *   hl(n,m) = b - floor((a + a[n][m+1]) / 2)             P on HL
 *   t       = e - floor((c + c[n][m+1]) / 2)             P on HH
 *   LH      = c - floor((a + a[n+1][m]) / 2)             P* on LH
 *   HH      = t - floor((hl(n,m) + hl(n+1,m)) / 2)       P* on HH, reading P's HL result
 * all from the values before the step. */
static void nonsep_predict_i(quad_i_t* q) {
    geom_t g = q->g;
    quad_i_t o = {g, dup_i(q->a, g.ner * g.nec), dup_i(q->b, g.ner * g.ndc),
                  dup_i(q->c, g.ndr * g.nec), dup_i(q->e, g.ndr * g.ndc)};
#define HLP(n, m) (B_(&o, n, m) - floor_div(A_(&o, n, m) + A_(&o, n, pr_(m, g.nec)), 2))
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.ndc; ++m) B_(q, n, m) = HLP(n, m);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.nec; ++m)
            C_(q, n, m) = C_(&o, n, m) - floor_div(A_(&o, n, m) + A_(&o, pr_(n, g.ner), m), 2);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) {
            int64_t t = E_(&o, n, m) - floor_div(C_(&o, n, m) + C_(&o, n, pr_(m, g.nec)), 2);
            E_(q, n, m) = t - floor_div(HLP(n, m) + HLP(pr_(n, g.ner), m), 2);
        }
#undef HLP
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* Integer spatial update, reproducing Eq. 3's U (rows) then U* (columns):
 *   lh(n,m) = c + floor((e[n][m-1] + e[n][m] + 2) / 4)          U on LH
 *   t       = a + floor((b[n][m-1] + b[n][m] + 2) / 4)          U on LL
 *   LL      = t + floor((lh(n-1,m) + lh(n,m) + 2) / 4)          U* on LL, reading U's LH result
 *   HL      = b + floor((e[n-1][m] + e[n][m] + 2) / 4)          U* on HL                     */
static void nonsep_update_i(quad_i_t* q) {
    geom_t g = q->g;
    quad_i_t o = {g, dup_i(q->a, g.ner * g.nec), dup_i(q->b, g.ner * g.ndc),
                  dup_i(q->c, g.ndr * g.nec), dup_i(q->e, g.ndr * g.ndc)};
#define LHU(n, m)                                                                                \
    (C_(&o, n, m) +                                                                              \
     (g.ndc ? floor_div(E_(&o, n, ul_(m)) + E_(&o, n, ur_(m, g.ndc)) + 2, 4) : 0))
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.nec; ++m) {
            int64_t t = A_(&o, n, m);
            if (g.ndc) t += floor_div(B_(&o, n, ul_(m)) + B_(&o, n, ur_(m, g.ndc)) + 2, 4);
            if (g.ndr) t += floor_div(LHU(ul_(n), m) + LHU(ur_(n, g.ndr), m) + 2, 4);
            A_(q, n, m) = t;
        }
    if (g.ndr)
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.ndc; ++m)
                B_(q, n, m) = B_(&o, n, m) +
                              floor_div(E_(&o, ul_(n), m) + E_(&o, ur_(n, g.ndr), m) + 2, 4);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.nec; ++m) C_(q, n, m) = LHU(n, m);
#undef LHU
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* Inverse integer spatial update: undo U* then U, same floor expressions, subtracted:
 *   hl = b - floor((e[n-1][m] + e[n][m] + 2) / 4)               undo U* on HL
 *   t  = a - floor((c[n-1][m] + c[n][m] + 2) / 4)               undo U* on LL (c = stored LH)
 *   LH = c - floor((e[n][m-1] + e[n][m] + 2) / 4)               undo U on LH
 *   LL = t - floor((hl(n,m-1) + hl(n,m) + 2) / 4)               undo U on LL, reading hl   */
static void nonsep_update_inv_i(quad_i_t* q) {
    geom_t g = q->g;
    quad_i_t o = {g, dup_i(q->a, g.ner * g.nec), dup_i(q->b, g.ner * g.ndc),
                  dup_i(q->c, g.ndr * g.nec), dup_i(q->e, g.ndr * g.ndc)};
#define HLU(n, m)                                                                                \
    (B_(&o, n, m) -                                                                              \
     (g.ndr ? floor_div(E_(&o, ul_(n), m) + E_(&o, ur_(n, g.ndr), m) + 2, 4) : 0))
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.nec; ++m) {
            int64_t t = A_(&o, n, m);
            if (g.ndr) t -= floor_div(C_(&o, ul_(n), m) + C_(&o, ur_(n, g.ndr), m) + 2, 4);
            if (g.ndc) t -= floor_div(HLU(n, ul_(m)) + HLU(n, ur_(m, g.ndc)) + 2, 4);
            A_(q, n, m) = t;
        }
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.ndc; ++m) B_(q, n, m) = HLU(n, m);
    if (g.ndc)
        for (long n = 0; n < g.ndr; ++n)
            for (long m = 0; m < g.nec; ++m)
                C_(q, n, m) = C_(&o, n, m) -
                              floor_div(E_(&o, n, ul_(m)) + E_(&o, n, ur_(m, g.ndc)) + 2, 4);
#undef HLU
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* Inverse integer spatial predict: undo P* then P:
 *   LH' = c + floor((a + a[n+1][m]) / 2)                          undo P* on LH
 *   t   = e + floor((b + b[n+1][m]) / 2)                          undo P* on HH (b = P's HL)
 *   HL' = b + floor((a + a[n][m+1]) / 2)                          undo P on HL
 *   HH' = t + floor((LH'(n,m) + LH'(n,m+1)) / 2)                  undo P on HH, reading LH' */
static void nonsep_predict_inv_i(quad_i_t* q) {
    geom_t g = q->g;
    quad_i_t o = {g, dup_i(q->a, g.ner * g.nec), dup_i(q->b, g.ner * g.ndc),
                  dup_i(q->c, g.ndr * g.nec), dup_i(q->e, g.ndr * g.ndc)};
#define LHR(n, m) (C_(&o, n, m) + floor_div(A_(&o, n, m) + A_(&o, pr_(n, g.ner), m), 2))
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.ndc; ++m)
            B_(q, n, m) = B_(&o, n, m) + floor_div(A_(&o, n, m) + A_(&o, n, pr_(m, g.nec)), 2);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.nec; ++m) C_(q, n, m) = LHR(n, m);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) {
            int64_t t = E_(&o, n, m) + floor_div(B_(&o, n, m) + B_(&o, pr_(n, g.ner), m), 2);
            E_(q, n, m) = t + floor_div(LHR(n, m) + LHR(n, pr_(m, g.nec)), 2);
        }
#undef LHR
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* 9/7 scaling of the four components (per axis: low 1/K, high K/2; length-1 axes unscaled). */
static void scale_quad_f(quad_f_t* q, long h, long w, int wavelet, int divide) {
    geom_t g = q->g;
    double s[4] = {axis_scale(wavelet, h, 0) * axis_scale(wavelet, w, 0),
                   axis_scale(wavelet, h, 0) * axis_scale(wavelet, w, 1),
                   axis_scale(wavelet, h, 1) * axis_scale(wavelet, w, 0),
                   axis_scale(wavelet, h, 1) * axis_scale(wavelet, w, 1)};
    double* arr[4] = {q->a, q->b, q->c, q->e};
    long cnt[4] = {g.ner * g.nec, g.ner * g.ndc, g.ndr * g.nec, g.ndr * g.ndc};
    for (int k = 0; k < 4; ++k)
        for (long i = 0; i < cnt[k]; ++i) arr[k][i] = divide ? arr[k][i] / s[k] : arr[k][i] * s[k];
}

/* ------------------------------------------------------------------------------------------
 * The spatial steps of Eq. 5 for lifting steps with more taps (the Deslauriers-Dubuc wavelets):
 * the same matrices, with P, P*, U, U* and the products PP*, UU* written as tap lists.  P reads
 * the even samples m + off of an odd sample m (offsets 0, +1 and, with the outer pair, -1, +2);
 * U reads the odd samples m + off of an even sample m (offsets -1, 0 and -2, +1).  The
 * whole-sample extension of an axis of length len, stated on band indices: even position 2k
 * is band index refl(2k) / 2, odd position 2k + 1 is (refl(2k + 1) - 1) / 2.  sign = -1 undoes
 * the step (the same matrix entries with the off-diagonal blocks negated and the product
 * term kept, as in the two-tap inverses above).
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    int n;
    long off[4];
    double c[4];
} taps_t;

static taps_t predict_taps(double p, double p3) {
    taps_t t = {2, {0, 1, 0, 0}, {p, p, 0.0, 0.0}};
    if (p3 != 0.0) {
        t.n = 4;
        t.off[2] = -1;
        t.off[3] = 2;
        t.c[2] = t.c[3] = p3;
    }
    return t;
}

static taps_t update_taps(double u, double u3) {
    taps_t t = {2, {-1, 0, 0, 0}, {u, u, 0.0, 0.0}};
    if (u3 != 0.0) {
        t.n = 4;
        t.off[2] = -2;
        t.off[3] = 1;
        t.c[2] = t.c[3] = u3;
    }
    return t;
}

static long ev_(long k, long len) { return refl_any(2 * k, len) / 2; }
static long od_(long k, long len) { return (refl_any(2 * k + 1, len) - 1) / 2; }

static void nonsep_predict_taps_f(quad_f_t* q, taps_t P, double sign) {
    geom_t g = q->g;
    long h = g.ner + g.ndr, w = g.nec + g.ndc;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.ndc; ++m) {
            double v = 0.0;
            for (int k = 0; k < P.n; ++k) v += P.c[k] * A_(&o, n, ev_(m + P.off[k], w));
            B_(q, n, m) = B_(&o, n, m) + sign * v;
        }
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.nec; ++m) {
            double v = 0.0;
            for (int k = 0; k < P.n; ++k) v += P.c[k] * A_(&o, ev_(n + P.off[k], h), m);
            C_(q, n, m) = C_(&o, n, m) + sign * v;
        }
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) {
            double vh = 0.0, vv = 0.0, va = 0.0;
            for (int k = 0; k < P.n; ++k) {
                vh += P.c[k] * C_(&o, n, ev_(m + P.off[k], w)); /* P  (LH) */
                vv += P.c[k] * B_(&o, ev_(n + P.off[k], h), m); /* P* (HL) */
                for (int l = 0; l < P.n; ++l)                    /* P* P (LL) */
                    va += P.c[k] * P.c[l] * A_(&o, ev_(n + P.off[k], h), ev_(m + P.off[l], w));
            }
            E_(q, n, m) = E_(&o, n, m) + sign * (vh + vv) + va;
        }
    free(o.a); free(o.b); free(o.c); free(o.e);
}

static void nonsep_update_taps_f(quad_f_t* q, taps_t U, double sign) {
    geom_t g = q->g;
    long h = g.ner + g.ndr, w = g.nec + g.ndc;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.nec; ++m) {
            double vh = 0.0, vv = 0.0, va = 0.0;
            for (int k = 0; k < U.n; ++k) {
                if (g.ndc) vh += U.c[k] * B_(&o, n, od_(m + U.off[k], w)); /* U  (HL) */
                if (g.ndr) vv += U.c[k] * C_(&o, od_(n + U.off[k], h), m); /* U* (LH) */
                if (g.ndr && g.ndc)                                         /* U* U (HH) */
                    for (int l = 0; l < U.n; ++l)
                        va += U.c[k] * U.c[l] *
                              E_(&o, od_(n + U.off[k], h), od_(m + U.off[l], w));
            }
            A_(q, n, m) = A_(&o, n, m) + sign * (vh + vv) + va;
        }
    if (g.ndr)
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.ndc; ++m) {
                double v = 0.0;
                for (int k = 0; k < U.n; ++k) v += U.c[k] * E_(&o, od_(n + U.off[k], h), m);
                B_(q, n, m) = B_(&o, n, m) + sign * v;
            }
    if (g.ndc)
        for (long n = 0; n < g.ndr; ++n)
            for (long m = 0; m < g.nec; ++m) {
                double v = 0.0;
                for (int k = 0; k < U.n; ++k) v += U.c[k] * E_(&o, n, od_(m + U.off[k], w));
                C_(q, n, m) = C_(&o, n, m) + sign * v;
            }
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* ------------------------------------------------------------------------------------------
 * Adapted non-separable scheme (Sec. 3, Fig. 3).  With P = P0 + P1, P0 = p (the constant
 * monomial) and P1 = p z, the spatial predict matrix of Eq. 5 factors as
 * M_P(P) = M_P(P1) M_P(P0): every factor is one of the commuting 1-D steps d += P0 s,
 * d += P1 s along rows and columns.  Likewise M_U(U) = M_U(U1) M_U(U0) with U0 = u, U1 = u z^-1.
 * The M(P0), M(U0) factors read only the quad itself ("constants ... never access the results
 * belonging to extraneous cores"); the M(P1), M(U1) factors keep the non-separable form with
 * the neighbour at m+1 / n+1 (predict) or m-1 / n-1 (update).  On the symmetric extension the
 * "own" sample of an update at the right end of an odd-length axis is the mirrored one, so the
 * constant part reads index ur(m) and the neighbour part ul(m), as the plain update does.
 * ---------------------------------------------------------------------------------------- */

/* M_P(P0) = [1 0 0 0; p 1 0 0; p 0 1 0; p^2 p p 1] on each quad (reads the quad only), computed,
 * as Sec. 3 computes the constant parts, with the separable scheme: the horizontal step
 * b += p a, e += p c, then the vertical step c += p a, e += p b (b as the horizontal step left
 * it).  Multiplied out, e gains p c + p b + p^2 a: the matrix above. */
static void adapted_predict_local_f(quad_f_t* q, double p) {
    geom_t g = q->g;
    for (long n = 0; n < g.ner; ++n) /* horizontal */
        for (long m = 0; m < g.ndc; ++m) B_(q, n, m) += p * A_(q, n, m);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) E_(q, n, m) += p * C_(q, n, m);
    for (long n = 0; n < g.ndr; ++n) /* vertical */
        for (long m = 0; m < g.nec; ++m) C_(q, n, m) += p * A_(q, n, m);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) E_(q, n, m) += p * B_(q, n, m);
}

/* M_P(P1): [1 0 0 0; pz 1 0 0; pz_n 0 1 0; p^2 z z_n, pz_n, pz, 1] (neighbours m+1, n+1). */
static void adapted_predict_fused_f(quad_f_t* q, double p) {
    geom_t g = q->g;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.ndc; ++m)
            B_(q, n, m) = B_(&o, n, m) + p * A_(&o, n, pr_(m, g.nec));
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.nec; ++m)
            C_(q, n, m) = C_(&o, n, m) + p * A_(&o, pr_(n, g.ner), m);
    for (long n = 0; n < g.ndr; ++n)
        for (long m = 0; m < g.ndc; ++m) {
            long m1 = pr_(m, g.nec), n1 = pr_(n, g.ner);
            E_(q, n, m) = E_(&o, n, m) + p * p * A_(&o, n1, m1) + p * B_(&o, n1, m) +
                          p * C_(&o, n, m1);
        }
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* M_U(U0) = [1 u u u^2; 0 1 0 u; 0 0 1 u; 0 0 0 1] on each quad (own samples of the extension),
 * with the separable scheme: the horizontal step a += u b, c += u e, then the vertical step
 * a += u c, b += u e (c as the horizontal step left it).  Multiplied out, a gains
 * u b + u c + u^2 e: the matrix above.  The "own" sample of the last quad of an odd-length axis
 * is the mirrored one (ur_). */
static void adapted_update_local_f(quad_f_t* q, double u) {
    geom_t g = q->g;
    if (g.ndc) { /* horizontal */
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.nec; ++m) A_(q, n, m) += u * B_(q, n, ur_(m, g.ndc));
        for (long n = 0; n < g.ndr; ++n)
            for (long m = 0; m < g.nec; ++m) C_(q, n, m) += u * E_(q, n, ur_(m, g.ndc));
    }
    if (g.ndr) { /* vertical */
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.nec; ++m) A_(q, n, m) += u * C_(q, ur_(n, g.ndr), m);
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.ndc; ++m) B_(q, n, m) += u * E_(q, ur_(n, g.ndr), m);
    }
}

/* M_U(U1): [1 uz^-1 uz_n^-1 u^2 z^-1 z_n^-1; 0 1 0 uz_n^-1; 0 0 1 uz^-1; 0 0 0 1]. */
static void adapted_update_fused_f(quad_f_t* q, double u) {
    geom_t g = q->g;
    quad_f_t o = {g, dup_f(q->a, g.ner * g.nec), dup_f(q->b, g.ner * g.ndc),
                  dup_f(q->c, g.ndr * g.nec), dup_f(q->e, g.ndr * g.ndc)};
    for (long n = 0; n < g.ner; ++n)
        for (long m = 0; m < g.nec; ++m) {
            double v = A_(&o, n, m);
            long ml = ul_(m), nl = ul_(n);
            if (g.ndc) v += u * B_(&o, n, ml);
            if (g.ndr) v += u * C_(&o, nl, m);
            if (g.ndr && g.ndc) v += u * u * E_(&o, nl, ml);
            A_(q, n, m) = v;
        }
    if (g.ndr)
        for (long n = 0; n < g.ner; ++n)
            for (long m = 0; m < g.ndc; ++m) B_(q, n, m) = B_(&o, n, m) + u * E_(&o, ul_(n), m);
    if (g.ndc)
        for (long n = 0; n < g.ndr; ++n)
            for (long m = 0; m < g.nec; ++m) C_(q, n, m) = C_(&o, n, m) + u * E_(&o, n, ul_(m));
    free(o.a); free(o.b); free(o.c); free(o.e);
}

/* The k-th step of one adapted level: local predict, fused predict, local update, fused
 * update, for each lifting pair in turn. */
static void adapted_step_f(quad_f_t* q, const lifting_t* L, int k) {
    const int pair = k / 4;
    switch (k % 4) {
    case 0: adapted_predict_local_f(q, L->p[pair]); break;
    case 1: adapted_predict_fused_f(q, L->p[pair]); break;
    case 2: adapted_update_local_f(q, L->u[pair]); break;
    default: adapted_update_fused_f(q, L->u[pair]); break;
    }
}

/* ------------------------------------------------------------------------------------------
 * One level in each direction, for every scheme.  x is the interleaved h x w plane of LL_{j-1};
 * the four outputs are dense band arrays.
 * ---------------------------------------------------------------------------------------- */
static int level_fwd_f(const double* x, long h, long w, int wavelet, int scheme, int ext,
                       double* LL, double* HL, double* LH, double* HH) {
    if (scheme == ORC_ADAPTED) {
        lifting_t L;
        if (get_lifting(wavelet, &L)) return -1;
        quad_f_t q = {geom_of(h, w), LL, HL, LH, HH};
        split_f(x, h, w, ORC_CDF53, LL, HL, LH, HH); /* plain split, no scaling */
        for (int k = 0; k < 4 * L.npairs; ++k) adapted_step_f(&q, &L, k);
        scale_quad_f(&q, h, w, wavelet, 0);
        return 0;
    }
    if (scheme == ORC_NONSEP_EQ5) {
        lifting_t L;
        if (get_lifting(wavelet, &L)) return -1;
        quad_f_t q = {geom_of(h, w), LL, HL, LH, HH};
        split_f(x, h, w, ORC_CDF53, LL, HL, LH, HH); /* plain split, no scaling */
        for (int k = 0; k < L.npairs; ++k) {
            if (L.p3[k] != 0.0 || L.u3[k] != 0.0) {
                nonsep_predict_taps_f(&q, predict_taps(L.p[k], L.p3[k]), 1.0);
                nonsep_update_taps_f(&q, update_taps(L.u[k], L.u3[k]), 1.0);
            } else {
                nonsep_predict_f(&q, L.p[k]);
                nonsep_update_f(&q, L.u[k]);
            }
        }
        scale_quad_f(&q, h, w, wavelet, 0);
        return 0;
    }
    double* t = dup_f(x, h * w);
    if (!t) return -2;
    int rc = sep_level_fwd_f(t, h, w, wavelet, scheme, ext);
    if (!rc) split_f(t, h, w, wavelet, LL, HL, LH, HH);
    free(t);
    return rc;
}

static int level_fwd_i(const int64_t* x, long h, long w, int scheme, int ext, int64_t* LL,
                       int64_t* HL, int64_t* LH, int64_t* HH) {
    if (scheme == ORC_NONSEP_EQ5) {
        quad_i_t q = {geom_of(h, w), LL, HL, LH, HH};
        split_i(x, h, w, LL, HL, LH, HH);
        nonsep_predict_i(&q);
        nonsep_update_i(&q);
        return 0;
    }
    int64_t* t = dup_i(x, h * w);
    if (!t) return -2;
    int rc = sep_level_fwd_i(t, h, w, scheme, ext);
    if (!rc) split_i(t, h, w, LL, HL, LH, HH);
    free(t);
    return rc;
}

static int level_inv_f(const double* LL, const double* HL, const double* LH, const double* HH,
                       long h, long w, int wavelet, int scheme, double* x) {
    if (scheme == ORC_NONSEP_EQ5) {
        lifting_t L;
        if (get_lifting(wavelet, &L)) return -1;
        geom_t g = geom_of(h, w);
        quad_f_t q = {g, dup_f(LL, g.ner * g.nec), dup_f(HL, g.ner * g.ndc),
                      dup_f(LH, g.ndr * g.nec), dup_f(HH, g.ndr * g.ndc)};
        scale_quad_f(&q, h, w, wavelet, 1);
        for (int k = L.npairs - 1; k >= 0; --k) {
            if (L.p3[k] != 0.0 || L.u3[k] != 0.0) {
                nonsep_update_taps_f(&q, update_taps(L.u[k], L.u3[k]), -1.0);
                nonsep_predict_taps_f(&q, predict_taps(L.p[k], L.p3[k]), -1.0);
            } else {
                nonsep_update_inv_f(&q, L.u[k]);
                nonsep_predict_inv_f(&q, L.p[k]);
            }
        }
        join_f(q.a, q.b, q.c, q.e, h, w, ORC_CDF53, 0, x);
        free(q.a); free(q.b); free(q.c); free(q.e);
        return 0;
    }
    join_f(LL, HL, LH, HH, h, w, wavelet, 1, x);
    return sep_level_inv_f(x, h, w, wavelet, scheme);
}

static int level_inv_i(const int64_t* LL, const int64_t* HL, const int64_t* LH,
                       const int64_t* HH, long h, long w, int scheme, int64_t* x) {
    if (scheme == ORC_NONSEP_EQ5) {
        geom_t g = geom_of(h, w);
        quad_i_t q = {g, dup_i(LL, g.ner * g.nec), dup_i(HL, g.ner * g.ndc),
                      dup_i(LH, g.ndr * g.nec), dup_i(HH, g.ndr * g.ndc)};
        nonsep_update_inv_i(&q);
        nonsep_predict_inv_i(&q);
        join_i(q.a, q.b, q.c, q.e, h, w, x);
        free(q.a); free(q.b); free(q.c); free(q.e);
        return 0;
    }
    join_i(LL, HL, LH, HH, h, w, x);
    return sep_level_inv_i(x, h, w, scheme);
}

/* Adjoint of one forward level: W_j = split . scale . (steps s_1 .. s_n), so
 * W_j^T = (s_1^T .. s_n^T applied last-first) . scale . join. */
static int level_fwd_adj_f(const double* gLL, const double* gHL, const double* gLH,
                           const double* gHH, long h, long w, int wavelet, double* gx) {
    step2d_t st[16];
    int ns = level_steps(wavelet, ORC_SEP_EQ3, st);
    if (ns < 0) return -1;
    join_f(gLL, gHL, gLH, gHH, h, w, wavelet, 0, gx);
    for (int k = ns - 1; k >= 0; --k)
        plane_step_adj_f(gx, h, w, st[k].axis, st[k].parity, st[k].coef);
    return 0;
}

/* Adjoint of one inverse level: W_j^-1 = (undo s_n .. undo s_1) . unscale . join, so
 * W_j^-T = split . unscale . (undo s_1)^T .. (undo s_n)^T, applied first-to-last. */
static int level_inv_adj_f(const double* gx_in, long h, long w, int wavelet, double* gLL,
                           double* gHL, double* gLH, double* gHH) {
    step2d_t st[16];
    int ns = level_steps(wavelet, ORC_SEP_EQ3, st);
    if (ns < 0) return -1;
    double* g = dup_f(gx_in, h * w);
    if (!g) return -2;
    for (int k = 0; k < ns; ++k)
        plane_step_adj_f(g, h, w, st[k].axis, st[k].parity, -st[k].coef);
    /* split with the inverse scale: multiply by 1 / scale */
    geom_t gg = geom_of(h, w);
    for (long r = 0; r < h; ++r)
        for (long c = 0; c < w; ++c) {
            double v = g[r * w + c] / (axis_scale(wavelet, h, r & 1) * axis_scale(wavelet, w, c & 1));
            long n = r / 2, m = c / 2;
            if (!(r & 1) && !(c & 1)) gLL[n * gg.nec + m] = v;
            if (!(r & 1) && (c & 1)) gHL[n * gg.ndc + m] = v;
            if ((r & 1) && !(c & 1)) gLH[n * gg.nec + m] = v;
            if ((r & 1) && (c & 1)) gHH[n * gg.ndc + m] = v;
        }
    free(g);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Multi-level layout: level j maps an h_{j-1} x w_{j-1} LL plane (h_0 = H, w_0 = W) to
 * bands of ceil/floor halves.  The band list is LL_J, then HL_J, LH_J, HH_J, ..., HL_1, LH_1,
 * HH_1, each dense.
 * ---------------------------------------------------------------------------------------- */
/* Threads for the line loops of the separable steps (1 = the plain sequential oracle, the
 * default).  Returns the count in effect (1 when built without OpenMP). */
int orc_set_threads(int n) {
#ifdef _OPENMP
    omp_set_num_threads(n < 1 ? 1 : n);
    return n < 1 ? 1 : n;
#else
    (void)n;
    return 1;
#endif
}

int orc_max_levels(int H, int W) {
    long n = H > W ? H : W;
    int L = 0;
    while (n > 1) {
        n = (n + 1) / 2;
        ++L;
    }
    return L < 1 ? 1 : L;
}

typedef struct {
    long h[33], w[33];      /* LL plane size entering level j+1 (index j = 0..J) */
    int64_t off_ll;         /* offset of LL_J */
    int64_t off[33][3];     /* offsets of HL_j, LH_j, HH_j */
    int64_t total;
} layout_t;

static int make_layout(int H, int W, int levels, layout_t* Lo) {
    if (H < 1 || W < 1 || levels < 1 || levels > orc_max_levels(H, W) || levels > 32) return -1;
    Lo->h[0] = H;
    Lo->w[0] = W;
    for (int j = 1; j <= levels; ++j) {
        Lo->h[j] = (Lo->h[j - 1] + 1) / 2;
        Lo->w[j] = (Lo->w[j - 1] + 1) / 2;
    }
    int64_t o = 0;
    Lo->off_ll = o;
    o += (int64_t)Lo->h[levels] * Lo->w[levels];
    for (int j = levels; j >= 1; --j) {
        geom_t g = geom_of(Lo->h[j - 1], Lo->w[j - 1]);
        Lo->off[j][0] = o;
        o += g.ner * g.ndc;
        Lo->off[j][1] = o;
        o += g.ndr * g.nec;
        Lo->off[j][2] = o;
        o += g.ndr * g.ndc;
    }
    Lo->total = o;
    return 0;
}

int64_t orc_coeff_count(int H, int W, int levels) {
    layout_t Lo;
    if (make_layout(H, W, levels, &Lo)) return -1;
    return Lo.total;
}

static int valid_scheme(int wavelet, int scheme) {
    if (wavelet < ORC_CDF53_INT || wavelet > ORC_DD137) return 0;
    return scheme >= ORC_SEP_EQ3 && scheme <= ORC_NONSEP_EQ5;
}

/* The adjoints, the adapted scheme and the step-by-step entry points are stated for the CDF
 * wavelets (two-tap steps). */
static int is_cdf(int wavelet) { return wavelet >= ORC_CDF53_INT && wavelet <= ORC_CDF97; }

/* The adapted scheme is defined for the float wavelets' forward transform (its constant /
 * neighbour split of a floor term would change the integer result). */
static int valid_forward_scheme(int wavelet, int scheme) {
    if (scheme == ORC_ADAPTED) return wavelet == ORC_CDF53 || wavelet == ORC_CDF97;
    return valid_scheme(wavelet, scheme);
}

int orc_forward(const void* img, int H, int W, int wavelet, int levels, int scheme,
                int extension_form, void* out) {
    layout_t Lo;
    if (!img || !out || !valid_forward_scheme(wavelet, scheme) || make_layout(H, W, levels, &Lo))
        return -1;
    if (extension_form && (scheme == ORC_NONSEP_EQ5 || scheme == ORC_ADAPTED)) return -1;
    long n0 = (long)H * W;
    if (wavelet == ORC_CDF53_INT) {
        int64_t* cur = dup_i((const int64_t*)img, n0);
        int64_t* o = (int64_t*)out;
        for (int j = 1; j <= levels; ++j) {
            long h = Lo.h[j - 1], w = Lo.w[j - 1];
            int64_t* ll = (int64_t*)malloc(sizeof(int64_t) * Lo.h[j] * Lo.w[j]);
            int rc = level_fwd_i(cur, h, w, scheme, extension_form, ll, o + Lo.off[j][0],
                                 o + Lo.off[j][1], o + Lo.off[j][2]);
            free(cur);
            cur = ll;
            if (rc) { free(cur); return rc; }
        }
        memcpy(o + Lo.off_ll, cur, sizeof(int64_t) * Lo.h[levels] * Lo.w[levels]);
        free(cur);
    } else {
        double* cur = dup_f((const double*)img, n0);
        double* o = (double*)out;
        for (int j = 1; j <= levels; ++j) {
            long h = Lo.h[j - 1], w = Lo.w[j - 1];
            double* ll = (double*)malloc(sizeof(double) * Lo.h[j] * Lo.w[j]);
            int rc = level_fwd_f(cur, h, w, wavelet, scheme, extension_form, ll,
                                 o + Lo.off[j][0], o + Lo.off[j][1], o + Lo.off[j][2]);
            free(cur);
            cur = ll;
            if (rc) { free(cur); return rc; }
        }
        memcpy(o + Lo.off_ll, cur, sizeof(double) * Lo.h[levels] * Lo.w[levels]);
        free(cur);
    }
    return 0;
}

int orc_inverse(const void* coeffs, int H, int W, int wavelet, int levels, int scheme,
                void* img) {
    layout_t Lo;
    if (!img || !coeffs || !valid_scheme(wavelet, scheme) || make_layout(H, W, levels, &Lo))
        return -1;
    if (wavelet == ORC_CDF53_INT) {
        const int64_t* c = (const int64_t*)coeffs;
        int64_t* cur = dup_i(c + Lo.off_ll, Lo.h[levels] * Lo.w[levels]);
        for (int j = levels; j >= 1; --j) {
            long h = Lo.h[j - 1], w = Lo.w[j - 1];
            int64_t* x = (int64_t*)malloc(sizeof(int64_t) * h * w);
            int rc = level_inv_i(cur, c + Lo.off[j][0], c + Lo.off[j][1], c + Lo.off[j][2], h,
                                 w, scheme, x);
            free(cur);
            cur = x;
            if (rc) { free(cur); return rc; }
        }
        memcpy(img, cur, sizeof(int64_t) * (long)H * W);
        free(cur);
    } else {
        const double* c = (const double*)coeffs;
        double* cur = dup_f(c + Lo.off_ll, Lo.h[levels] * Lo.w[levels]);
        for (int j = levels; j >= 1; --j) {
            long h = Lo.h[j - 1], w = Lo.w[j - 1];
            double* x = (double*)malloc(sizeof(double) * h * w);
            int rc = level_inv_f(cur, c + Lo.off[j][0], c + Lo.off[j][1], c + Lo.off[j][2], h,
                                 w, wavelet, scheme, x);
            free(cur);
            cur = x;
            if (rc) { free(cur); return rc; }
        }
        memcpy(img, cur, sizeof(double) * (long)H * W);
        free(cur);
    }
    return 0;
}

/* W = level_J . ... . level_1, so W^T applies level_J^T first, down to level_1^T. */
int orc_forward_adjoint(const double* g_coeffs, int H, int W, int wavelet, int levels,
                        double* g_img) {
    layout_t Lo;
    if (!g_coeffs || !g_img || wavelet == ORC_CDF53_INT || !is_cdf(wavelet) ||
        make_layout(H, W, levels, &Lo))
        return -1;
    double* cur = dup_f(g_coeffs + Lo.off_ll, Lo.h[levels] * Lo.w[levels]);
    for (int j = levels; j >= 1; --j) {
        long h = Lo.h[j - 1], w = Lo.w[j - 1];
        double* x = (double*)malloc(sizeof(double) * h * w);
        int rc = level_fwd_adj_f(cur, g_coeffs + Lo.off[j][0], g_coeffs + Lo.off[j][1],
                                 g_coeffs + Lo.off[j][2], h, w, wavelet, x);
        free(cur);
        cur = x;
        if (rc) { free(cur); return rc; }
    }
    memcpy(g_img, cur, sizeof(double) * (long)H * W);
    free(cur);
    return 0;
}

/* W^-1 = level_1^-1 . ... . level_J^-1, so W^-T applies level_1^-T first, up to level_J^-T. */
int orc_inverse_adjoint(const double* g_img, int H, int W, int wavelet, int levels,
                        double* g_coeffs) {
    layout_t Lo;
    if (!g_coeffs || !g_img || wavelet == ORC_CDF53_INT || !is_cdf(wavelet) ||
        make_layout(H, W, levels, &Lo))
        return -1;
    double* cur = dup_f(g_img, (long)H * W);
    for (int j = 1; j <= levels; ++j) {
        long h = Lo.h[j - 1], w = Lo.w[j - 1];
        double* ll = (double*)malloc(sizeof(double) * Lo.h[j] * Lo.w[j]);
        int rc = level_inv_adj_f(cur, h, w, wavelet, ll, g_coeffs + Lo.off[j][0],
                                 g_coeffs + Lo.off[j][1], g_coeffs + Lo.off[j][2]);
        free(cur);
        cur = ll;
        if (rc) { free(cur); return rc; }
    }
    memcpy(g_coeffs + Lo.off_ll, cur, sizeof(double) * Lo.h[levels] * Lo.w[levels]);
    free(cur);
    return 0;
}

int orc_nonsep_steps(const double* img, int H, int W, int wavelet, int nsteps, double* out) {
    lifting_t L;
    if (!img || !out || H < 1 || W < 1 || wavelet == ORC_CDF53_INT || !is_cdf(wavelet) ||
        get_lifting(wavelet, &L) ||
        nsteps < 0 || nsteps > 2 * L.npairs)
        return -1;
    geom_t g = geom_of(H, W);
    double* a = out;
    double* b = a + g.ner * g.nec;
    double* c = b + g.ner * g.ndc;
    double* e = c + g.ndr * g.nec;
    quad_f_t q = {g, a, b, c, e};
    split_f(img, H, W, ORC_CDF53, a, b, c, e);
    for (int k = 0; k < nsteps; ++k) {
        if (k % 2 == 0) nonsep_predict_f(&q, L.p[k / 2]);
        else nonsep_update_f(&q, L.u[k / 2]);
    }
    return 0;
}

int orc_adapted_steps(const double* img, int H, int W, int wavelet, int nsteps, double* out) {
    lifting_t L;
    if (!img || !out || H < 1 || W < 1 || wavelet == ORC_CDF53_INT || !is_cdf(wavelet) ||
        get_lifting(wavelet, &L) ||
        nsteps < 0 || nsteps > 4 * L.npairs)
        return -1;
    geom_t g = geom_of(H, W);
    double* a = out;
    double* b = a + g.ner * g.nec;
    double* c = b + g.ner * g.ndc;
    double* e = c + g.ndr * g.nec;
    quad_f_t q = {g, a, b, c, e};
    split_f(img, H, W, ORC_CDF53, a, b, c, e);
    for (int k = 0; k < nsteps; ++k) adapted_step_f(&q, &L, k);
    return 0;
}

int orc_adapted_apply(double* abce, int H, int W, int wavelet, int k0, int k1) {
    lifting_t L;
    if (!abce || H < 1 || W < 1 || wavelet == ORC_CDF53_INT || !is_cdf(wavelet) ||
        get_lifting(wavelet, &L) ||
        k0 < 0 || k1 < k0 || k1 > 4 * L.npairs)
        return -1;
    geom_t g = geom_of(H, W);
    double* a = abce;
    double* b = a + g.ner * g.nec;
    double* c = b + g.ner * g.ndc;
    double* e = c + g.ndr * g.nec;
    quad_f_t q = {g, a, b, c, e};
    for (int k = k0; k < k1; ++k) adapted_step_f(&q, &L, k);
    return 0;
}
