// dwt2_lifting.cuh -- the lifting arithmetic of one decomposition level, as row-streaming stages.
//
// Data model: a lane owns kQ adjacent polyphase quads (q = 0 .. kQ-1) of one quad row,
//   a = LL = x[2n][2m], b = HL = x[2n][2m+1], c = LH = x[2n+1][2m], e = HH = x[2n+1][2m+1]
// (the quad [LL, HL, LH, HH] of Sec. 2).  Horizontal neighbours (quad m +/- 1) come from the
// adjacent lane by warp shuffle; vertical neighbours (quad row n +/- 1) are the rows pushed
// before / after, kept in registers.  Rows are pushed top to bottom; a stage that reads the row
// below returns its result one push late (lag 1).
//
// Boundaries are not handled here: the loaders feed the whole-sample symmetric extension of
// the plane (mirrored rows and columns), on which lifting needs no boundary rule.
//
// Wavelets: P(z) = p (1 + z) reads quad m and m + 1 (row n and n + 1 for P*); U(z) = u (1 + z^-1)
// reads m - 1 and m (n - 1 and n for U*).
#pragma once

#include <type_traits>

#include "dwt2_device.cuh"

namespace dwt2 {

constexpr int kQ = 2;  // polyphase quads per lane (adjacent along a row)

enum Wavelet { WV_CDF53_INT = 0, WV_CDF53 = 1, WV_CDF97 = 2, WV_DD97 = 3, WV_DD137 = 4 };
// The Deslauriers-Dubuc (interpolating) wavelets: their predict has four taps, and so does the
// 13/7's update.
__host__ __device__ constexpr bool is_dd(int wv) { return wv == WV_DD97 || wv == WV_DD137; }
enum Mode {
    MODE_NONSEP = 0,
    MODE_SEP = 1,
    MODE_ROWS = 2,
    MODE_COLS = 3,
    MODE_ADJ_INV = 4,
    MODE_ADAPTED = 5,
    MODE_CONV = 6
};

// CDF 9/7 lifting constants and the per-axis normalisation (low * 1/K, high * K/2).
constexpr float k97Alpha = -1.586134342059924f;
constexpr float k97Beta = -0.052980118572961f;
constexpr float k97Gamma = 0.882911075530934f;
constexpr float k97Delta = 0.443506852043971f;
constexpr float k97K = 1.230174104914001f;
constexpr float k97Low = 1.0f / k97K;
constexpr float k97High = k97K / 2.0f;
// 2-D band scales of a 9/7 level (per axis low 1/K, high K/2)
constexpr float k97sLL = k97Low * k97Low;
constexpr float k97sHL = k97Low * k97High;
constexpr float k97sLH = k97High * k97Low;
constexpr float k97sHH = k97High * k97High;

template <typename C>
struct QRow {
    C a[kQ], b[kQ], c[kQ], e[kQ];
};

template <typename C>
__device__ __forceinline__ void zero_row(QRow<C>& r) {
#pragma unroll
    for (int q = 0; q < kQ; ++q) r.a[q] = r.b[q] = r.c[q] = r.e[q] = C(0);
}

// =============================================================================================
// One lifting term.  Float: p (s0 + s1) and u (d0 + d1).  Reversible integer CDF 5/3: the
// predict term is -floor((s0 + s1) / 2) and the update term floor((d0 + d1 + 2) / 4), both by
// arithmetic shift (floor for negative values too).
// =============================================================================================
template <typename C>
__device__ __forceinline__ C step_p(C s0, C s1, float p) {
    if constexpr (std::is_same<C, int32_t>::value) {  // integer: -floor((s0 + s1) / 2)
        return -((s0 + s1) >> 1);
    } else {
        return p * (s0 + s1);
    }
}
template <typename C>
__device__ __forceinline__ C step_u(C d0, C d1, float u) {
    if constexpr (std::is_same<C, int32_t>::value) {  // integer: floor((d0 + d1 + 2) / 4)
        return (d0 + d1 + 2) >> 2;
    } else {
        return u * (d0 + d1);
    }
}

// Packed fp32: a lane's two quads (kQ == 2) take the same arithmetic, so the inverse float
// stages evaluate both at once with the f32x2 instructions (one add and one fma per term for the
// pair instead of per quad); x + w (s0 + s1) rounds exactly as the scalar fused form.  Measured on
// GB300: the 9/7 inverse 1.9% faster; the forward stages 1.6% and (after the predict was
// rescheduled) 4.4% slower packed, so they stay scalar.
template <typename C>
constexpr bool kPacked = std::is_same<C, float>::value && kQ == 2;
__device__ __forceinline__ float2 v2(const float (&v)[kQ]) { return make_float2(v[0], v[1]); }
__device__ __forceinline__ void put2(float (&v)[kQ], float2 x) {
    v[0] = x.x;
    v[1] = x.y;
}
__device__ __forceinline__ float2 lift2(float2 x, float2 s0, float2 s1, float2 w) {
    return __ffma2_rn(w, __fadd2_rn(s0, s1), x);
}

// Band scaling of a row (packed: one f32x2 multiply per band for the lane's two quads); used by
// the inverse.
__device__ __forceinline__ void scale_row(QRow<float>& r, float sa, float sb, float sc, float se) {
    if constexpr (kQ == 2) {
        put2(r.a, __fmul2_rn(v2(r.a), make_float2(sa, sa)));
        put2(r.b, __fmul2_rn(v2(r.b), make_float2(sb, sb)));
        put2(r.c, __fmul2_rn(v2(r.c), make_float2(sc, sc)));
        put2(r.e, __fmul2_rn(v2(r.e), make_float2(se, se)));
    } else {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.a[q] *= sa;
            r.b[q] *= sb;
            r.c[q] *= sc;
            r.e[q] *= se;
        }
    }
}

// Adds v to every component of a float row (the DC level shift of the first forward level and
// of the last inverse level); integer rows are never shifted.  Packed, also in the scalar
// forward stages: on GB300 the 9/7 forward with the shift measured 0.1410 ms with these four
// f32x2 adds per row against 0.1427 ms with eight scalar ones (0.1385 ms without the shift).
template <typename C>
__device__ __forceinline__ void add_row(QRow<C>& r, float v) {
    if constexpr (kPacked<C>) {
        const float2 w = make_float2(v, v);
        put2(r.a, __fadd2_rn(v2(r.a), w));
        put2(r.b, __fadd2_rn(v2(r.b), w));
        put2(r.c, __fadd2_rn(v2(r.c), w));
        put2(r.e, __fadd2_rn(v2(r.e), w));
    } else if constexpr (std::is_same<C, float>::value) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.a[q] += v;
            r.b[q] += v;
            r.c[q] += v;
            r.e[q] += v;
        }
    }
}
// The same on the LL component only (the shift of LL_J entering the inverse).
template <typename C>
__device__ __forceinline__ void add_ll(QRow<C>& r, float v) {
    if constexpr (kPacked<C>) {
        put2(r.a, __fadd2_rn(v2(r.a), make_float2(v, v)));
    } else if constexpr (std::is_same<C, float>::value) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) r.a[q] += v;
    }
}

// =============================================================================================
// Non-separable scheme (Sec. 3, Eq. 5).
//
// Each fused step reads only the values before the step (one synchronisation point per step).
// The tensor-product entries PP* and UU* are evaluated as the product of their 1-D factors
// (P* applied to P's result, U* to U's), recomputed from the step's inputs: it is the same
// linear map, and in fp32 it avoids the large cancelling p^2 (a + a[m+1] + a[n+1] + ...) sum of
// the expanded form (about two bits better for CDF 9/7).  For the integer wavelet this order is
// forced: Sec. 2 lets horizontal and vertical steps interleave freely, which holds in exact
// arithmetic only, so the fused steps reproduce the floors of Eq. 3's order P, P*, U, U*.
// =============================================================================================

// Spatial predict [1 0 0 0; P 1 0 0; P* 0 1 0; PP* P* P 1]:
//   hl  = b + P(a)             = b + p (a + a[m+1])
//   LH  = c + P*(a)            = c + p (a + a[n+1])
//   HH  = e + P(c) + P*(hl)    = e + p (c + c[m+1]) + p (hl + hl[n+1])
//       ( = e + P(c) + P*(b) + PP*(a) )
// LL is unchanged ("the predict step is completely responsible for HH", Sec. 3).
// Every term reads values from before the step only.  push(y) consumes quad row n + 1 and
// returns row n (lag 1).  The terms of a row that need nothing from the next row -- hl and the
// partial sum t = e + P(c) -- are evaluated when the row arrives, so the state carried to the
// next push is (a, hl, c, t): the same operations as at output time, one value fewer per quad
// to carry than (a, c, e, hl, c[m+1]).
template <typename C>
struct PredictNS {
    float p;
    QRow<C> x;  // row n: a, hl (in b), c, t (in e)
    __device__ __forceinline__ void init(float p_) {
        p = p_;
        zero_row(x);
    }
    __device__ __forceinline__ void push(const QRow<C>& y, QRow<C>& o) {
        C yar[kQ], ycr[kQ];
        right_of(y.a, yar);
        right_of(y.c, ycr);
        QRow<C> n;  // row n + 1: a, hl, c, t
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            n.a[q] = y.a[q];
            n.b[q] = y.b[q] + step_p(y.a[q], yar[q], p);
            n.c[q] = y.c[q];
            n.e[q] = y.e[q] + step_p(y.c[q], ycr[q], p);
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            o.a[q] = x.a[q];
            o.b[q] = x.b[q];
            o.c[q] = x.c[q] + step_p(x.a[q], n.a[q], p);
            o.e[q] = x.e[q] + step_p(x.b[q], n.b[q], p);
        }
        x = n;
    }
};

// Spatial update [1 U U* UU*; 0 1 0 U*; 0 0 1 U; 0 0 0 1]:
//   lh  = c + U(e)             = c + u (e[m-1] + e)
//   LL  = a + U(b) + U*(lh)    = a + u (b[m-1] + b) + u (lh[n-1] + lh)
//       ( = a + U(b) + U*(c) + UU*(e) )
//   HL  = b + U*(e)            = b + u (e[n-1] + e)
//   LH  = lh
// HH is unchanged ("the update step is responsible for LL").  In place, lag 0.
template <typename C>
struct UpdateNS {
    float u;
    C plh[kQ], pe[kQ];  // row n - 1: lh, e
    __device__ __forceinline__ void init(float u_) {
        u = u_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) plh[q] = pe[q] = C(0);
    }
    __device__ __forceinline__ void push(QRow<C>& r) {
        C bl[kQ], el[kQ];
        left_of(r.b, bl);
        left_of(r.e, el);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const C lh = r.c[q] + step_u(el[q], r.e[q], u);
            const C t = r.a[q] + step_u(bl[q], r.b[q], u);
            const C a = t + step_u(plh[q], lh, u);
            const C b = r.b[q] + step_u(pe[q], r.e[q], u);
            plh[q] = lh;
            pe[q] = r.e[q];
            r.a[q] = a;
            r.b[q] = b;
            r.c[q] = lh;
        }
    }
};

// Inverse spatial update [1 -U -U* UU*; 0 1 0 -U*; 0 0 1 -U; 0 0 0 1], evaluated as the
// forward update's terms undone in reverse order (same terms, subtracted):
//   hl = HL - u (e[n-1] + e);  t = LL - u (LH[n-1] + LH);  c = LH - u (e[m-1] + e);
//   a  = t - u (hl[m-1] + hl).   Lag 0.
template <typename C>
struct InvUpdateNS {
    float u;
    C pc[kQ], pe[kQ];  // row n - 1: stored LH, e
    __device__ __forceinline__ void init(float u_) {
        u = u_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) pc[q] = pe[q] = C(0);
    }
    __device__ __forceinline__ void push(QRow<C>& r) {
        C el[kQ], hl[kQ], hll[kQ];
        left_of(r.e, el);
        if constexpr (kPacked<C>) {
            const float2 w = make_float2(-u, -u);
            const float2 e = v2(r.e), c = v2(r.c);
            const float2 h = lift2(v2(r.b), v2(pe), e, w);
            put2(hl, h);
            left_of(hl, hll);
            const float2 t = lift2(v2(r.a), v2(pc), c, w);
            put2(r.c, lift2(c, v2(el), e, w));
            put2(r.a, lift2(t, v2(hll), h, w));
            put2(r.b, h);
            put2(pc, c);
            put2(pe, e);
            return;
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) hl[q] = r.b[q] - step_u(pe[q], r.e[q], u);
        left_of(hl, hll);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const C t = r.a[q] - step_u(pc[q], r.c[q], u);
            const C c = r.c[q] - step_u(el[q], r.e[q], u);
            const C a = t - step_u(hll[q], hl[q], u);
            pc[q] = r.c[q];
            pe[q] = r.e[q];
            r.a[q] = a;
            r.b[q] = hl[q];
            r.c[q] = c;
        }
    }
};

// Inverse spatial predict [1 0 0 0; -P 1 0 0; -P* 0 1 0; PP* -P* -P 1], as the forward terms
// undone in reverse order:
//   c = LH - p (a + a[n+1]);  t = HH - p (HL + HL[n+1]);  b = HL - p (a + a[m+1]);
//   e = t - p (c + c[m+1]).   Lag 1.
template <typename C>
struct InvPredictNS {
    float p;
    QRow<C> x;
    C xar[kQ];
    __device__ __forceinline__ void init(float p_) {
        p = p_;
        zero_row(x);
#pragma unroll
        for (int q = 0; q < kQ; ++q) xar[q] = C(0);
    }
    __device__ __forceinline__ void push(const QRow<C>& y, QRow<C>& o) {
        C c[kQ], cr[kQ];
        if constexpr (kPacked<C>) {
            const float2 w = make_float2(-p, -p);
            const float2 c2 = lift2(v2(x.c), v2(x.a), v2(y.a), w);
            put2(c, c2);
            right_of(c, cr);
            const float2 t = lift2(v2(x.e), v2(x.b), v2(y.b), w);
            put2(o.b, lift2(v2(x.b), v2(x.a), v2(xar), w));
            put2(o.e, lift2(t, c2, v2(cr), w));
            put2(o.c, c2);
#pragma unroll
            for (int q = 0; q < kQ; ++q) o.a[q] = x.a[q];
            x = y;
            right_of(y.a, xar);
            return;
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) c[q] = x.c[q] - step_p(x.a[q], y.a[q], p);
        right_of(c, cr);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const C t = x.e[q] - step_p(x.b[q], y.b[q], p);
            o.a[q] = x.a[q];
            o.b[q] = x.b[q] - step_p(x.a[q], xar[q], p);
            o.c[q] = c[q];
            o.e[q] = t - step_p(c[q], cr[q], p);
        }
        x = y;
        right_of(y.a, xar);
    }
};

// =============================================================================================
// Adapted non-separable scheme (Sec. 3, Fig. 3), float wavelets.  P = P0 + P1 with P0 = p (the
// constant monomial) and P1 = p z, U = U0 + U1 with U0 = u and U1 = u z^-1; each spatial step
// of Eq. 5 is evaluated as a local step with the constants (no other quad is read), then the
// fused step with P1 / U1:
//   M_P(P) = M_P(P1) M_P(P0),  M_P(P0) = [1 0 0 0; p 1 0 0; p 0 1 0; p^2 p p 1],
//   M_U(U) = M_U(U1) M_U(U0),  M_U(U0) = [1 u u u^2; 0 1 0 u; 0 0 1 u; 0 0 0 1].
// Sec. 3 evaluates the constant parts with the separable scheme, which has the fewest
// operations: the local steps are a horizontal then a vertical 1-D step, 4 FMAs per quad
// instead of the 5 of the multiplied-out matrix.  The fused steps are evaluated in the factored
// form of the plain scheme (the P1* / U1* term applied to P1's / U1's result), also 4 FMAs.
// The same linear map as the plain scheme; fp32 rounding differs.
// =============================================================================================

// Local predict on arrival (separable: b' = b + p a, t = e + p c, then c' = c + p a,
// e' = t + p b'), then the fused P1 step, factored like PredictNS (lag 1):
//   hl = b' + p a[m+1],  LH = c' + p a[n+1],  HH = (e' + p c'[m+1]) + p hl[n+1]
//      ( = e' + p^2 a[n+1][m+1] + p b'[n+1] + p c'[m+1] ).
// State carried to the next push: row n's a, hl, c', and e' + p c'[m+1].
struct AdaptedPredict {
    float p;
    QRow<float> x;  // row n: a, hl (in b), c', t (in e)
    __device__ __forceinline__ void init(float p_) {
        p = p_;
        zero_row(x);
    }
    __device__ __forceinline__ void push(const QRow<float>& y, QRow<float>& o) {
        QRow<float> n;  // row n + 1: a, hl, c', t
        float lb[kQ], le[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {  // local step, horizontal then vertical
            lb[q] = fmaf(p, y.a[q], y.b[q]);
            le[q] = fmaf(p, y.c[q], y.e[q]);
            n.c[q] = fmaf(p, y.a[q], y.c[q]);
            le[q] = fmaf(p, lb[q], le[q]);
        }
        float yar[kQ], ycr[kQ];
        right_of(y.a, yar);
        right_of(n.c, ycr);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            n.a[q] = y.a[q];
            n.b[q] = fmaf(p, yar[q], lb[q]);
            n.e[q] = fmaf(p, ycr[q], le[q]);
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            o.a[q] = x.a[q];
            o.b[q] = x.b[q];
            o.c[q] = fmaf(p, n.a[q], x.c[q]);
            o.e[q] = fmaf(p, n.b[q], x.e[q]);
        }
        x = n;
    }
};

// Local update (separable: a1 = a + u b, c' = c + u e, then a' = a1 + u c', b' = b + u e), then
// the fused U1 step, factored like UpdateNS, both on the row as it arrives (lag 0):
//   LH = c' + u e[m-1],  LL = a' + u b'[m-1] + u LH[n-1],  HL = b' + u e[n-1]
//      ( LL = a' + u b'[m-1] + u c'[n-1] + u^2 e[n-1][m-1] ).
struct AdaptedUpdate {
    float u;
    float plh[kQ], pe[kQ];  // row n - 1: LH, e
    __device__ __forceinline__ void init(float u_) {
        u = u_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) plh[q] = pe[q] = 0.f;
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        float a[kQ], b[kQ], c[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {  // local step, horizontal then vertical
            a[q] = fmaf(u, r.b[q], r.a[q]);
            c[q] = fmaf(u, r.e[q], r.c[q]);
            a[q] = fmaf(u, c[q], a[q]);
            b[q] = fmaf(u, r.e[q], r.b[q]);
        }
        float bl[kQ], el[kQ];
        left_of(b, bl);
        left_of(r.e, el);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const float lh = fmaf(u, el[q], c[q]);
            r.a[q] = fmaf(u, plh[q], fmaf(u, bl[q], a[q]));
            r.b[q] = fmaf(u, pe[q], b[q]);
            r.c[q] = lh;
            plh[q] = lh;
            pe[q] = r.e[q];
        }
    }
};

// =============================================================================================
// Separable convolution (Eq. 4), float wavelets: N^H, the whole 1-D analysis along rows as one
// filtering step, then N^V along columns, each followed by the subsampling.  The analysis
// filters are the impulse responses of the 1-D lifting steps above (with the per-axis 9/7
// scaling), evaluated at compile time: low taps -kL..kL around the even sample, high taps
// -kH..kH around the odd one.  They are symmetric, so the whole-sample symmetric extension the
// loaders supply is the boundary rule here too.
// =============================================================================================
template <int WV>
struct ConvTaps {
    static constexpr int kL = WV == WV_CDF97 ? 4 : 2;
    static constexpr int kH = WV == WV_CDF97 ? 3 : 1;
    float lo[2 * kL + 1] = {};
    float hi[2 * kH + 1] = {};
};

template <int WV>
constexpr ConvTaps<WV> conv_taps() {
    ConvTaps<WV> t{};
    constexpr int kN = 16, kN0 = 4;  // half-length of the probe signal, observed output index
    constexpr int kPairs = WV == WV_CDF97 ? 2 : 1;
    const double P[2] = {WV == WV_CDF97 ? double(k97Alpha) : -0.5, double(k97Gamma)};
    const double U[2] = {WV == WV_CDF97 ? double(k97Beta) : 0.25, double(k97Delta)};
    for (int k = 2 * kN0 - t.kL; k <= 2 * kN0 + 1 + t.kH; ++k) {
        double sv[kN] = {}, dv[kN] = {};  // even / odd samples of the unit impulse at k
        if (k % 2 == 0) sv[k / 2] = 1.0;
        else dv[k / 2] = 1.0;
        for (int j = 0; j < kPairs; ++j) {
            for (int i = 0; i + 1 < kN; ++i) dv[i] += P[j] * (sv[i] + sv[i + 1]);
            for (int i = kN - 1; i >= 1; --i) sv[i] += U[j] * (dv[i - 1] + dv[i]);
        }
        const double ls = WV == WV_CDF97 ? double(k97Low) : 1.0;
        const double hs = WV == WV_CDF97 ? double(k97High) : 1.0;
        const int tl = k - 2 * kN0, th = k - 2 * kN0 - 1;
        if (tl >= -t.kL && tl <= t.kL) t.lo[tl + t.kL] = float(ls * sv[kN0]);
        if (th >= -t.kH && th <= t.kH) t.hi[th + t.kH] = float(hs * dv[kN0]);
    }
    return t;
}

// Vertical step N^V over the horizontally filtered quad rows (a: low column of row 2n, b: high
// column of row 2n, c: low column of row 2n + 1, e: high column of row 2n + 1).  Keeps a window
// of 2 kLag + 1 quad rows; push(row n + kLag) returns output quad row n (LL, HL, LH, HH).
template <int WV>
struct ConvV {
    static constexpr int kL = ConvTaps<WV>::kL, kH = ConvTaps<WV>::kH;
    static constexpr int kLag = (kL + 1) / 2;
    static constexpr int kWin = 2 * kLag + 1;
    QRow<float> w[kWin];
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int j = 0; j < kWin; ++j) zero_row(w[j]);
    }
    // pixel row 2n + t of the low (hi = false) or high column of quad q
    __device__ __forceinline__ float pix(int t, bool high, int q) const {
        const int j = kLag + (t >= 0 ? t / 2 : -((1 - t) / 2));
        const bool odd = (t & 1) != 0;
        return high ? (odd ? w[j].e[q] : w[j].b[q]) : (odd ? w[j].c[q] : w[j].a[q]);
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        constexpr ConvTaps<WV> T = conv_taps<WV>();
#pragma unroll
        for (int j = 0; j + 1 < kWin; ++j) w[j] = w[j + 1];
        w[kWin - 1] = r;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            float ll = 0.f, hl = 0.f, lh = 0.f, hh = 0.f;
#pragma unroll
            for (int t = -kL; t <= kL; ++t) {
                ll = fmaf(T.lo[t + kL], pix(t, false, q), ll);
                hl = fmaf(T.lo[t + kL], pix(t, true, q), hl);
            }
#pragma unroll
            for (int t = -kH; t <= kH; ++t) {
                lh = fmaf(T.hi[t + kH], pix(t + 1, false, q), lh);
                hh = fmaf(T.hi[t + kH], pix(t + 1, true, q), hh);
            }
            r.a[q] = ll;
            r.b[q] = hl;
            r.c[q] = lh;
            r.e[q] = hh;
        }
    }
};

// =============================================================================================
// Separable lifting (Eq. 3) evaluated in the same single pass: the four steps P, P*, U, U* one
// after the other, each reading the previous step's result.  The comparator of the paper's
// separable scheme on the same data path.
// =============================================================================================
// P (rows) then P* (columns); lag 1.
template <typename C>
struct PredictSep {
    float p;
    QRow<C> x;
    __device__ __forceinline__ void init(float p_) {
        p = p_;
        zero_row(x);
    }
    __device__ __forceinline__ void push(QRow<C> y, QRow<C>& o) {
        C ar[kQ], cr[kQ];
        right_of(y.a, ar);
        right_of(y.c, cr);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {  // P on the new row
            y.b[q] += step_p(y.a[q], ar[q], p);
            y.e[q] += step_p(y.c[q], cr[q], p);
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {  // P* on the row above, now that its lower neighbour is known
            o.a[q] = x.a[q];
            o.b[q] = x.b[q];
            o.c[q] = x.c[q] + step_p(x.a[q], y.a[q], p);
            o.e[q] = x.e[q] + step_p(x.b[q], y.b[q], p);
        }
        x = y;
    }
};

// U (rows) then U* (columns); lag 0.
template <typename C>
struct UpdateSep {
    float u;
    C pc[kQ], pe[kQ];
    __device__ __forceinline__ void init(float u_) {
        u = u_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) pc[q] = pe[q] = C(0);
    }
    __device__ __forceinline__ void push(QRow<C>& r) {
        C bl[kQ], el[kQ];
        left_of(r.b, bl);
        left_of(r.e, el);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {  // U
            r.a[q] += step_u(bl[q], r.b[q], u);
            r.c[q] += step_u(el[q], r.e[q], u);
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {  // U*
            r.a[q] += step_u(pc[q], r.c[q], u);
            r.b[q] += step_u(pe[q], r.e[q], u);
            pc[q] = r.c[q];
            pe[q] = r.e[q];
        }
    }
};

// Row-only pass (all horizontal steps of all pairs, then the horizontal scaling); lag 0.
template <typename C, int WV>
__device__ __forceinline__ void rows_only(QRow<C>& r) {
    constexpr int npairs = WV == WV_CDF97 ? 2 : 1;
    const float ps[kQ] = {WV == WV_CDF97 ? k97Alpha : -0.5f, k97Gamma};
    const float us[kQ] = {WV == WV_CDF97 ? k97Beta : 0.25f, k97Delta};
#pragma unroll
    for (int k = 0; k < npairs; ++k) {
        C ar[kQ], cr[kQ], bl[kQ], el[kQ];
        right_of(r.a, ar);
        right_of(r.c, cr);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.b[q] += step_p(r.a[q], ar[q], ps[k]);
            r.e[q] += step_p(r.c[q], cr[q], ps[k]);
        }
        left_of(r.b, bl);
        left_of(r.e, el);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.a[q] += step_u(bl[q], r.b[q], us[k]);
            r.c[q] += step_u(el[q], r.e[q], us[k]);
        }
    }
    if constexpr (WV == WV_CDF97) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.a[q] *= k97Low;
            r.c[q] *= k97Low;
            r.b[q] *= k97High;
            r.e[q] *= k97High;
        }
    }
}

// Column-only steps: P* (lag 1) and U* (lag 0).
template <typename C>
struct PredictCol {
    float p;
    QRow<C> x;
    __device__ __forceinline__ void init(float p_) {
        p = p_;
        zero_row(x);
    }
    __device__ __forceinline__ void push(const QRow<C>& y, QRow<C>& o) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            o.a[q] = x.a[q];
            o.b[q] = x.b[q];
            o.c[q] = x.c[q] + step_p(x.a[q], y.a[q], p);
            o.e[q] = x.e[q] + step_p(x.b[q], y.b[q], p);
        }
        x = y;
    }
};
template <typename C>
struct UpdateCol {
    float u;
    C pc[kQ], pe[kQ];
    __device__ __forceinline__ void init(float u_) {
        u = u_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) pc[q] = pe[q] = C(0);
    }
    __device__ __forceinline__ void push(QRow<C>& r) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.a[q] += step_u(pc[q], r.c[q], u);
            r.b[q] += step_u(pe[q], r.e[q], u);
            pc[q] = r.c[q];
            pe[q] = r.e[q];
        }
    }
};

// =============================================================================================
// Adjoints (transposes) of the fused steps, for gradients.  The forward level is
// W = S . U_K P_K ... U_1 P_1 (P = P* after P along rows, U = U* after U), so
//   W^T    = P_1^T U_1^T ... P_K^T U_K^T S           (applied right to left),
//   W^-T   = S^-1 U_K^-T P_K^-T ... U_1^-T P_1^-T,   with P^-1 = P(-p), U^-1 = U(-u).
// The transpose of a step with the in-step symmetric reflection is not a reflected step: a
// mirrored tap that read a sample twice now adds twice into it, and nothing is read from beyond
// the edge.  In gather form on one axis of length N (ne even, nd odd samples):
//   transposed predict, into even sample k:  p (w_own g_d[k] + w_left g_d[k-1])
//       w_own  = [0 <= k < nd] (1 + [nd == ne and k == ne - 1]),  w_left = [1 <= k <= nd]
//   transposed update, into odd sample k:    u (w_own g_s[k] + w_right g_s[k+1])
//       w_own  = [0 <= k < nd] (1 + [k == 0]),
//       w_right = [0 <= k < nd] ([k + 1 < ne] + [nd < ne and k == nd - 1])
// Values outside the plane enter only with weight 0 (the loaders supply zeros there).
// =============================================================================================
struct AxisLen {
    int ne, nd;
};
__device__ __forceinline__ float tp_own(int k, AxisLen a) {
    return (k >= 0 && k < a.nd) ? ((a.nd == a.ne && k == a.ne - 1) ? 2.f : 1.f) : 0.f;
}
__device__ __forceinline__ float tp_left(int k, AxisLen a) { return (k >= 1 && k <= a.nd) ? 1.f : 0.f; }
__device__ __forceinline__ float tu_own(int k, AxisLen a) {
    return (k >= 0 && k < a.nd) ? (k == 0 ? 2.f : 1.f) : 0.f;
}
__device__ __forceinline__ float tu_right(int k, AxisLen a) {
    return (k >= 0 && k < a.nd)
               ? float(k + 1 < a.ne ? 1 : 0) + float(a.nd < a.ne && k == a.nd - 1 ? 1 : 0)
               : 0.f;
}

// Per-lane horizontal weights of the lane's kQ quads (quad columns m0 .. m0 + kQ - 1).  ones:
// every weight of every lane of the warp is 1 (a warp away from the plane's left and right
// edges), so its rows away from the top and bottom edges can take the steps without weights.
struct LaneW {
    float p_own[kQ], p_left[kQ], u_own[kQ], u_right[kQ];
    bool ones;
    __device__ __forceinline__ void init(int m0, AxisLen cols) {
        bool one = true;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            p_own[q] = tp_own(m0 + q, cols);
            p_left[q] = tp_left(m0 + q, cols);
            u_own[q] = tu_own(m0 + q, cols);
            u_right[q] = tu_right(m0 + q, cols);
            one = one && p_own[q] == 1.f && p_left[q] == 1.f && u_own[q] == 1.f &&
                  u_right[q] == 1.f;
        }
        ones = __all_sync(0xffffffffu, one);
    }
};
// Rows n of an axis whose transposed-step weights are all 1 (tp_own, tp_left, tu_own, tu_right),
// with a margin of kPairs rows for the pipelines' row offsets.
__device__ __forceinline__ bool interior_row(int n, AxisLen rows, int margin) {
    return n >= 1 + margin && n + margin < rows.nd - 1;
}

// Transpose of the fused update: U*^T (into g_c from g_a, into g_e from g_b; reads row n + 1),
// then U^T (into g_b from g_a, into g_e from the new g_c; reads quad m + 1).  Predict-shaped,
// lag 1: push(row n + 1) returns row n.
struct AdjUpdate {
    float u;
    QRow<float> x;
    int xn;
    float xar[kQ];
    __device__ __forceinline__ void init(float u_) {
        u = u_;
        zero_row(x);
        xn = -1 << 20;
#pragma unroll
        for (int q = 0; q < kQ; ++q) xar[q] = 0.f;
    }
    template <bool kFast = false>
    __device__ __forceinline__ void push(const QRow<float>& y, int yn, QRow<float>& o,
                                         const LaneW& hw, AxisLen rows) {
        if constexpr (kFast) {  // all weights 1: the bits the general form gives with them
            float gc[kQ], gcr[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) gc[q] = fmaf(u, x.a[q], fmaf(u, y.a[q], x.c[q]));
            right_of(gc, gcr);
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const float ge = fmaf(u, x.b[q], fmaf(u, y.b[q], x.e[q]));
                o.a[q] = x.a[q];
                o.b[q] = x.b[q] + u * (x.a[q] + xar[q]);
                o.c[q] = gc[q];
                o.e[q] = ge + u * (gc[q] + gcr[q]);
            }
            x = y;
            xn = yn;
            right_of(y.a, xar);
            return;
        }
        // the step's constant folded into the row weights: two FMAs per vertical term, as in
        // the forward steps.  (Folding it into the lane weights too would hold their products
        // in registers for the whole loop: 8 more, one CTA per SM fewer.)
        const float wo = u * tu_own(xn, rows), wr = u * tu_right(xn, rows);
        float gc[kQ], gcr[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) gc[q] = fmaf(wo, x.a[q], fmaf(wr, y.a[q], x.c[q]));
        right_of(gc, gcr);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const float ge = fmaf(wo, x.b[q], fmaf(wr, y.b[q], x.e[q]));
            o.a[q] = x.a[q];
            o.b[q] = x.b[q] + u * (hw.u_own[q] * x.a[q] + hw.u_right[q] * xar[q]);
            o.c[q] = gc[q];
            o.e[q] = ge + u * (hw.u_own[q] * gc[q] + hw.u_right[q] * gcr[q]);
        }
        x = y;
        xn = yn;
        right_of(y.a, xar);
    }
};

// Transpose of the fused predict: P*^T (into g_a from g_c, into g_b from g_e; reads row n - 1),
// then P^T (into g_a from the new g_b, into g_c from g_e; reads quad m - 1).  Update-shaped,
// lag 0, in place.
struct AdjPredict {
    float p;
    float pc[kQ], pe[kQ];  // row n - 1: g_c, g_e entering this step
    __device__ __forceinline__ void init(float p_) {
        p = p_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) pc[q] = pe[q] = 0.f;
    }
    template <bool kFast = false>
    __device__ __forceinline__ void push(QRow<float>& r, int n, const LaneW& hw, AxisLen rows) {
        if constexpr (kFast) {  // all weights 1
            float ga[kQ], gb[kQ], gbl[kQ], gel[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                ga[q] = fmaf(p, r.c[q], fmaf(p, pc[q], r.a[q]));
                gb[q] = fmaf(p, r.e[q], fmaf(p, pe[q], r.b[q]));
            }
            left_of(gb, gbl);
            left_of(r.e, gel);
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const float gc = r.c[q] + p * (r.e[q] + gel[q]);
                pc[q] = r.c[q];
                pe[q] = r.e[q];
                r.a[q] = ga[q] + p * (gb[q] + gbl[q]);
                r.b[q] = gb[q];
                r.c[q] = gc;
            }
            return;
        }
        const float wo = p * tp_own(n, rows), wl = p * tp_left(n, rows);
        float ga[kQ], gb[kQ], gbl[kQ], gel[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            ga[q] = fmaf(wo, r.c[q], fmaf(wl, pc[q], r.a[q]));
            gb[q] = fmaf(wo, r.e[q], fmaf(wl, pe[q], r.b[q]));
        }
        left_of(gb, gbl);
        left_of(r.e, gel);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            const float gc = r.c[q] + p * (hw.p_own[q] * r.e[q] + hw.p_left[q] * gel[q]);
            pc[q] = r.c[q];
            pe[q] = r.e[q];
            r.a[q] = ga[q] + p * (hw.p_own[q] * gb[q] + hw.p_left[q] * gbl[q]);
            r.b[q] = gb[q];
            r.c[q] = gc;
        }
    }
};

// Adjoint pipelines.  AdjFwdPipe = W^T (band gradients in, plane gradient out; the data flow of
// the inverse kernel).  AdjInvPipe = W^-T (plane gradient in, band gradients out; the data flow
// of the forward kernel).  Both lag kPairs rows.  The scale factors come from the host (an axis
// of length 1 is not scaled).
struct Scale4 {
    float ll, hl, lh, hh;
};

template <int WV>
struct AdjFwdPipe {
    static constexpr int kPairs = WV == WV_CDF97 ? 2 : 1;
    static constexpr int kLag = kPairs;
    using C = float;
    AdjUpdate tu[kPairs];
    AdjPredict tp[kPairs];
    __device__ __forceinline__ void init() {
        const float P[2] = {WV == WV_CDF97 ? k97Alpha : -0.5f, k97Gamma};
        const float U[2] = {WV == WV_CDF97 ? k97Beta : 0.25f, k97Delta};
#pragma unroll
        for (int k = 0; k < kPairs; ++k) {  // pairs in reverse order
            tu[k].init(U[kPairs - 1 - k]);
            tp[k].init(P[kPairs - 1 - k]);
        }
    }
    __device__ __forceinline__ void push(QRow<float>& r, int n, const LaneW& hw, AxisLen rows,
                                         const Scale4& s) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.a[q] *= s.ll;
            r.b[q] *= s.hl;
            r.c[q] *= s.lh;
            r.e[q] *= s.hh;
        }
        // rows n - kPairs .. n take part in this push; away from every edge no weight is needed
        if (hw.ones && interior_row(n, rows, kPairs)) {
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                QRow<float> t;
                tu[k].template push<true>(r, n - k, t, hw, rows);
                tp[k].template push<true>(t, n - k - 1, hw, rows);
                r = t;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                QRow<float> t;
                tu[k].push(r, n - k, t, hw, rows);
                tp[k].push(t, n - k - 1, hw, rows);
                r = t;
            }
        }
    }
};

template <int WV>
struct AdjInvPipe {
    static constexpr int kPairs = WV == WV_CDF97 ? 2 : 1;
    static constexpr int kLag = kPairs;
    using C = float;
    AdjPredict tp[kPairs];
    AdjUpdate tu[kPairs];
    __device__ __forceinline__ void init() {
        const float P[2] = {WV == WV_CDF97 ? k97Alpha : -0.5f, k97Gamma};
        const float U[2] = {WV == WV_CDF97 ? k97Beta : 0.25f, k97Delta};
#pragma unroll
        for (int k = 0; k < kPairs; ++k) {  // pairs in forward order, negated coefficients
            tp[k].init(-P[k]);
            tu[k].init(-U[k]);
        }
    }
    __device__ __forceinline__ void push(QRow<float>& r, int n, const LaneW& hw, AxisLen rows,
                                         const Scale4& inv_s) {
        if (hw.ones && interior_row(n, rows, kPairs)) {
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                QRow<float> t;
                tp[k].template push<true>(r, n - k, hw, rows);
                tu[k].template push<true>(r, n - k, t, hw, rows);
                r = t;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                QRow<float> t;
                tp[k].push(r, n - k, hw, rows);
                tu[k].push(r, n - k, t, hw, rows);
                r = t;
            }
        }
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            r.a[q] *= inv_s.ll;
            r.b[q] *= inv_s.hl;
            r.c[q] *= inv_s.lh;
            r.e[q] *= inv_s.hh;
        }
    }
};

// =============================================================================================
// One forward level as a pipeline: push a raw (extended) quad row, get back the finished row
// kLag pushes earlier, in place.
// =============================================================================================
template <int WV, int MODE>
struct FwdPipe;

// reversible integer 5/3
template <int MODE>
struct FwdPipe<WV_CDF53_INT, MODE> {
    static constexpr int kLag = MODE == MODE_ROWS ? 0 : 1;
    using C = int32_t;
    PredictNS<int32_t> pn;
    UpdateNS<int32_t> un;
    PredictSep<int32_t> ps;
    UpdateSep<int32_t> us;
    PredictCol<int32_t> pcol;
    UpdateCol<int32_t> ucol;
    __device__ __forceinline__ void init(float = -0.f) {  // integer levels take no shift
        if constexpr (MODE == MODE_NONSEP) { pn.init(0.f); un.init(0.f); }
        if constexpr (MODE == MODE_SEP) { ps.init(0.f); us.init(0.f); }
        if constexpr (MODE == MODE_COLS) { pcol.init(0.f); ucol.init(0.f); }
    }
    __device__ __forceinline__ void push(QRow<int32_t>& r) {
        QRow<int32_t> t;
        if constexpr (MODE == MODE_NONSEP) { pn.push(r, t); un.push(t); r = t; }
        if constexpr (MODE == MODE_SEP) { ps.push(r, t); us.push(t); r = t; }
        if constexpr (MODE == MODE_ROWS) { rows_only<int32_t, WV_CDF53_INT>(r); }
        if constexpr (MODE == MODE_COLS) { pcol.push(r, t); ucol.push(t); r = t; }
    }
};

// float 5/3 and 9/7
template <int WV, int MODE>
struct FwdPipe {
    static constexpr int kPairs = WV == WV_CDF97 ? 2 : 1;
    static constexpr int kLag = MODE == MODE_ROWS ? 0 : kPairs;
    using C = float;
    PredictNS<float> pn[kPairs];
    UpdateNS<float> un[kPairs];
    PredictSep<float> ps[kPairs];
    UpdateSep<float> us[kPairs];
    PredictCol<float> pcol[kPairs];
    UpdateCol<float> ucol[kPairs];
    AdaptedPredict pa[kPairs];
    AdaptedUpdate ua[kPairs];
    ConvV<WV> cv;
    float ll_add;  // added to the finished LL (the DC level shift at the last level, else -0)
    static_assert(MODE != MODE_CONV || ConvV<WV>::kLag == kPairs, "lag of the convolution");
    __device__ __forceinline__ void init(float ll_add_ = -0.f) {
        ll_add = ll_add_;
        if constexpr (MODE == MODE_CONV) cv.init();
        const float P[kQ] = {WV == WV_CDF97 ? k97Alpha : -0.5f, k97Gamma};
        const float U[kQ] = {WV == WV_CDF97 ? k97Beta : 0.25f, k97Delta};
#pragma unroll
        for (int k = 0; k < kPairs; ++k) {
            if constexpr (MODE == MODE_NONSEP) { pn[k].init(P[k]); un[k].init(U[k]); }
            if constexpr (MODE == MODE_SEP) { ps[k].init(P[k]); us[k].init(U[k]); }
            if constexpr (MODE == MODE_COLS) { pcol[k].init(P[k]); ucol[k].init(U[k]); }
            if constexpr (MODE == MODE_ADAPTED) { pa[k].init(P[k]); ua[k].init(U[k]); }
        }
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        if constexpr (MODE == MODE_ROWS) {
            rows_only<float, WV>(r);
            return;
        } else if constexpr (MODE == MODE_CONV) {
            cv.push(r);  // the taps include the scaling
            return;
        } else {
#pragma unroll
            for (int k = 0; k < kPairs; ++k) {
                QRow<float> t;
                if constexpr (MODE == MODE_NONSEP) { pn[k].push(r, t); un[k].push(t); }
                if constexpr (MODE == MODE_SEP) { ps[k].push(r, t); us[k].push(t); }
                if constexpr (MODE == MODE_COLS) { pcol[k].push(r, t); ucol[k].push(t); }
                if constexpr (MODE == MODE_ADAPTED) { pa[k].push(r, t); ua[k].push(t); }
                r = t;
            }
            if constexpr (WV == WV_CDF97) {
                // per axis: low * 1/K, high * K/2 (COLS: vertical axis only)
                constexpr float sLL = MODE == MODE_COLS ? k97Low : k97sLL;
                constexpr float sHL = MODE == MODE_COLS ? k97Low : k97sHL;
                constexpr float sLH = MODE == MODE_COLS ? k97High : k97sLH;
                constexpr float sHH = MODE == MODE_COLS ? k97High : k97sHH;
#pragma unroll
                for (int q = 0; q < kQ; ++q) {
                    r.a[q] = fmaf(r.a[q], sLL, ll_add);
                    r.b[q] *= sHL;
                    r.c[q] *= sLH;
                    r.e[q] *= sHH;
                }
            } else {
#pragma unroll
                for (int q = 0; q < kQ; ++q) r.a[q] += ll_add;
            }
        }
    }
};

// One inverse level: push an (extended) quad row of the four bands, get back the reconstructed
// quad row kLag pushes earlier.
template <int WV>
struct InvPipe {
    static constexpr int kPairs = WV == WV_CDF97 ? 2 : 1;
    static constexpr int kLag = kPairs;
    using C = float;
    InvUpdateNS<float> iu[kPairs];
    InvPredictNS<float> ip[kPairs];
    __device__ __forceinline__ void init() {
        const float P[kQ] = {WV == WV_CDF97 ? k97Alpha : -0.5f, k97Gamma};
        const float U[kQ] = {WV == WV_CDF97 ? k97Beta : 0.25f, k97Delta};
#pragma unroll
        for (int k = 0; k < kPairs; ++k) {
            iu[k].init(U[kPairs - 1 - k]);
            ip[k].init(P[kPairs - 1 - k]);
        }
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        if constexpr (WV == WV_CDF97) {
            constexpr float sLL = 1.0f / (k97Low * k97Low);
            constexpr float sHL = 1.0f / (k97Low * k97High);
            constexpr float sHH = 1.0f / (k97High * k97High);
            scale_row(r, sLL, sHL, sHL, sHH);
        }
#pragma unroll
        for (int k = 0; k < kPairs; ++k) {
            QRow<float> t;
            iu[k].push(r);
            ip[k].push(r, t);
            r = t;
        }
    }
};

template <>
struct InvPipe<WV_CDF53_INT> {
    static constexpr int kLag = 1;
    using C = int32_t;
    InvUpdateNS<int32_t> iu;
    InvPredictNS<int32_t> ip;
    __device__ __forceinline__ void init() {
        iu.init(0.f);
        ip.init(0.f);
    }
    __device__ __forceinline__ void push(QRow<int32_t>& r) {
        QRow<int32_t> t;
        iu.push(r);
        ip.push(r, t);
        r = t;
    }
};

// =============================================================================================
// Four-tap lifting steps: the Deslauriers-Dubuc 9/7 and 13/7 (Sec. 1 and Sec. 5 hold the schemes
// for any wavelet).  The predict of an odd sample reads its even neighbours at m, m+1 (inner
// pair, weight p0) and m-1, m+2 (outer pair, p1): the cubic interpolation, p0 = -9/16,
// p1 = 1/16.  The update of an even sample reads its odd neighbours at m-1, m (u0) and m-2, m+1
// (u1): 1/4, 0 for 9/7 and 9/32, -1/32 for 13/7.  No scaling.  The spatial steps are those of
// Eq. 5 with these P, P*, U, U*, evaluated in the factored form of the two-tap steps above
// (HH += P*(HL after P) + P(LH); LL += U(HL) + U*(LH after U)).  A level of the 13/7 reaches
// three quads each way, so its warp windows keep two halo lanes on each side (a narrower output
// window, halo_q); the 9/7, with the two-tap update, reaches two, as the CDF wavelets do.
// =============================================================================================
constexpr float kDDp0 = -9.0f / 16.0f;
constexpr float kDDp1 = 1.0f / 16.0f;
constexpr float kDD137u0 = 9.0f / 32.0f;
constexpr float kDD137u1 = -1.0f / 32.0f;

// v at quad m + K (K = 1, 2) and m - K of each of a lane's kQ quads (K <= kQ).
template <int K, typename C>
__device__ __forceinline__ void right_k(const C (&v)[kQ], C (&r)[kQ]) {
#pragma unroll
    for (int q = 0; q < kQ; ++q)
        r[q] = q + K < kQ ? v[q + K] : __shfl_down_sync(kFull, v[q + K - kQ], 1);
}
template <int K, typename C>
__device__ __forceinline__ void left_k(const C (&v)[kQ], C (&l)[kQ]) {
#pragma unroll
    for (int q = 0; q < kQ; ++q)
        l[q] = q - K >= 0 ? v[q - K] : __shfl_up_sync(kFull, v[q - K + kQ], 1);
}

// v at quads m + 1 and m + 2 (or m - 1 and m - 2) of each of a lane's two quads, taking the
// shuffle the two share once: 2 shuffles instead of 3.
template <typename C>
__device__ __forceinline__ void right_12(const C (&v)[kQ], C (&r1)[kQ], C (&r2)[kQ]) {
    static_assert(kQ == 2, "two quads per lane");
    const C s = __shfl_down_sync(kFull, v[0], 1);  // quad m + 2 of quad 0, m + 1 of quad 1
    r1[0] = v[1];
    r1[1] = s;
    r2[0] = s;
    r2[1] = __shfl_down_sync(kFull, v[1], 1);
}
template <typename C>
__device__ __forceinline__ void left_12(const C (&v)[kQ], C (&l1)[kQ], C (&l2)[kQ]) {
    static_assert(kQ == 2, "two quads per lane");
    const C s = __shfl_up_sync(kFull, v[1], 1);  // quad m - 1 of quad 0, m - 2 of quad 1
    l1[0] = s;
    l1[1] = v[0];
    l2[0] = __shfl_up_sync(kFull, v[0], 1);
    l2[1] = s;
}

// P along a row: p0 (v[m] + v[m+1]) + p1 (v[m-1] + v[m+2]).  kShared takes the neighbours with
// right_12 (3 shuffles instead of 4, the same values).  The 13/7 inverse steps use it; in the
// 13/7 forward, whose registers are capped for 4 CTAs per SM, it spilled (level 1 111 -> 129 us).
template <bool kShared = false>
__device__ __forceinline__ void predict_h4(const float (&v)[kQ], float p0, float p1,
                                           float (&o)[kQ]) {
    float r1[kQ], r2[kQ], l1[kQ];
    if constexpr (kShared) {
        right_12(v, r1, r2);
    } else {
        right_k<1>(v, r1);
        right_k<2>(v, r2);
    }
    left_k<1>(v, l1);
#pragma unroll
    for (int q = 0; q < kQ; ++q) o[q] = fmaf(p0, v[q] + r1[q], p1 * (l1[q] + r2[q]));
}
// U along a row: u0 (v[m-1] + v[m]) + u1 (v[m-2] + v[m+1]).  kShared as in predict_h4.
template <bool kShared = false>
__device__ __forceinline__ void update_h4(const float (&v)[kQ], float u0, float u1,
                                          float (&o)[kQ]) {
    float l1[kQ], l2[kQ], r1[kQ];
    if constexpr (kShared) {
        left_12(v, l1, l2);
    } else {
        left_k<1>(v, l1);
        left_k<2>(v, l2);
    }
    right_k<1>(v, r1);
#pragma unroll
    for (int q = 0; q < kQ; ++q) o[q] = fmaf(u0, l1[q] + v[q], u1 * (l2[q] + r1[q]));
}
// A vertical four-tap term from four rows: w0 (x0 + x1) + w1 (xm + x2).
__device__ __forceinline__ float tap4(float x0, float x1, float xm, float x2, float w0, float w1) {
    return fmaf(w0, x0 + x1, w1 * (xm + x2));
}

// Spatial predict with a four-tap P.  push(row n + 2) returns row n (lag 2).
struct PredictNS4 {
    float a[3][kQ], b[3][kQ];  // rows n-1, n, n+1: LL and HL after the horizontal step
    float c[2][kQ], t[2][kQ];  // rows n, n+1: LH and HH + P(LH)
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            a[0][q] = a[1][q] = a[2][q] = b[0][q] = b[1][q] = b[2][q] = 0.f;
            c[0][q] = c[1][q] = t[0][q] = t[1][q] = 0.f;
        }
    }
    __device__ __forceinline__ void push(const QRow<float>& y, QRow<float>& o) {
        float pa[kQ], pc[kQ], yb[kQ], yt[kQ];
        predict_h4(y.a, kDDp0, kDDp1, pa);
        predict_h4(y.c, kDDp0, kDDp1, pc);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            yb[q] = y.b[q] + pa[q];
            yt[q] = y.e[q] + pc[q];
            o.a[q] = a[1][q];
            o.b[q] = b[1][q];
            o.c[q] = c[0][q] + tap4(a[1][q], a[2][q], a[0][q], y.a[q], kDDp0, kDDp1);
            o.e[q] = t[0][q] + tap4(b[1][q], b[2][q], b[0][q], yb[q], kDDp0, kDDp1);
            a[0][q] = a[1][q];
            a[1][q] = a[2][q];
            a[2][q] = y.a[q];
            b[0][q] = b[1][q];
            b[1][q] = b[2][q];
            b[2][q] = yb[q];
            c[0][q] = c[1][q];
            c[1][q] = y.c[q];
            t[0][q] = t[1][q];
            t[1][q] = yt[q];
        }
    }
};

// Spatial update with a four-tap U.  push(row i + 1) returns row i (lag 1).
struct UpdateNS4 {
    float u0, u1;
    float l[3][kQ], e[3][kQ];  // rows i-2, i-1, i: LH + U(HH), and HH
    float ta[kQ], hb[kQ];      // row i: LL + U(HL), and HL
    __device__ __forceinline__ void init(float u0_, float u1_) {
        u0 = u0_;
        u1 = u1_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            l[0][q] = l[1][q] = l[2][q] = e[0][q] = e[1][q] = e[2][q] = 0.f;
            ta[q] = hb[q] = 0.f;
        }
    }
    __device__ __forceinline__ void push(const QRow<float>& x, QRow<float>& o) {
        float ue[kQ], ub[kQ], xl[kQ], xt[kQ];
        update_h4(x.e, u0, u1, ue);
        update_h4(x.b, u0, u1, ub);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            xl[q] = x.c[q] + ue[q];
            xt[q] = x.a[q] + ub[q];
            o.a[q] = ta[q] + tap4(l[1][q], l[2][q], l[0][q], xl[q], u0, u1);
            o.b[q] = hb[q] + tap4(e[1][q], e[2][q], e[0][q], x.e[q], u0, u1);
            o.c[q] = l[2][q];
            o.e[q] = e[2][q];
            l[0][q] = l[1][q];
            l[1][q] = l[2][q];
            l[2][q] = xl[q];
            e[0][q] = e[1][q];
            e[1][q] = e[2][q];
            e[2][q] = x.e[q];
            ta[q] = xt[q];
            hb[q] = x.b[q];
        }
    }
};

// Undoes UpdateNS4.  push(row i + 1) returns row i (lag 1).  kShared as in InvPredictNS4.
template <bool kShared>
struct InvUpdateNS4 {
    float u0, u1;
    float c[3][kQ], e[3][kQ];  // rows i-2, i-1, i: stored LH and HH
    float a1[kQ], b1[kQ];      // row i: stored LL and HL
    __device__ __forceinline__ void init(float u0_, float u1_) {
        u0 = u0_;
        u1 = u1_;
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            c[0][q] = c[1][q] = c[2][q] = e[0][q] = e[1][q] = e[2][q] = 0.f;
            a1[q] = b1[q] = 0.f;
        }
    }
    __device__ __forceinline__ void push(const QRow<float>& x, QRow<float>& o) {
        float hl[kQ], uh[kQ], ue[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            hl[q] = b1[q] - tap4(e[1][q], e[2][q], e[0][q], x.e[q], u0, u1);
        update_h4<kShared>(hl, u0, u1, uh);
        update_h4<kShared>(e[2], u0, u1, ue);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            o.a[q] = a1[q] - tap4(c[1][q], c[2][q], c[0][q], x.c[q], u0, u1) - uh[q];
            o.b[q] = hl[q];
            o.c[q] = c[2][q] - ue[q];
            o.e[q] = e[2][q];
            c[0][q] = c[1][q];
            c[1][q] = c[2][q];
            c[2][q] = x.c[q];
            e[0][q] = e[1][q];
            e[1][q] = e[2][q];
            e[2][q] = x.e[q];
            a1[q] = x.a[q];
            b1[q] = x.b[q];
        }
    }
};

// Undoes PredictNS4.  push(row i + 2) returns row i (lag 2).  kShared: the horizontal
// neighbours with one shuffle fewer (predict_h4, update_h4), the same values.  Measured on
// GB300, 8192^2, 5 levels, with it in both inverse steps: the 13/7 inverse with fp32 bands
// 167.4 -> 164.3-165.3 us, but with bf16 bands 179.7 -> 181.7 us (a 4-byte spill under the
// 96-register bound), and the 9/7 inverse, whose update is the two-tap one, 141.2 -> 143.0 us.
// So only the 13/7 inverse with 32-bit bands takes it (InvPipeOf).
template <bool kShared>
struct InvPredictNS4 {
    float a[3][kQ], b[3][kQ];  // rows i-1, i, i+1: LL and stored HL
    float c[2][kQ], e[2][kQ];  // rows i, i+1: stored LH and HH
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            a[0][q] = a[1][q] = a[2][q] = b[0][q] = b[1][q] = b[2][q] = 0.f;
            c[0][q] = c[1][q] = e[0][q] = e[1][q] = 0.f;
        }
    }
    __device__ __forceinline__ void push(const QRow<float>& y, QRow<float>& o) {
        float lh[kQ], pa[kQ], pl[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            lh[q] = c[0][q] - tap4(a[1][q], a[2][q], a[0][q], y.a[q], kDDp0, kDDp1);
        predict_h4<kShared>(a[1], kDDp0, kDDp1, pa);
        predict_h4<kShared>(lh, kDDp0, kDDp1, pl);
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            o.a[q] = a[1][q];
            o.b[q] = b[1][q] - pa[q];
            o.c[q] = lh[q];
            o.e[q] = e[0][q] - tap4(b[1][q], b[2][q], b[0][q], y.b[q], kDDp0, kDDp1) - pl[q];
            a[0][q] = a[1][q];
            a[1][q] = a[2][q];
            a[2][q] = y.a[q];
            b[0][q] = b[1][q];
            b[1][q] = b[2][q];
            b[2][q] = y.b[q];
            c[0][q] = c[1][q];
            c[1][q] = y.c[q];
            e[0][q] = e[1][q];
            e[1][q] = y.e[q];
        }
    }
};

// The two-pass separable comparator for the four-tap wavelets: the row pass applies P then U
// along each pixel row (lag 0); the column pass applies P* (lag 2) then U* (lag 1 with four taps,
// lag 0 with two, the existing UpdateCol) along the columns.
template <int WV>
__device__ __forceinline__ void rows_only_dd(QRow<float>& r) {
    float pa[kQ], pc[kQ], ub[kQ], ue[kQ];
    predict_h4(r.a, kDDp0, kDDp1, pa);
    predict_h4(r.c, kDDp0, kDDp1, pc);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        r.b[q] += pa[q];
        r.e[q] += pc[q];
    }
    const float u0 = WV == WV_DD97 ? 0.25f : kDD137u0;
    const float u1 = WV == WV_DD97 ? 0.f : kDD137u1;
    update_h4(r.b, u0, u1, ub);
    update_h4(r.e, u0, u1, ue);
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        r.a[q] += ub[q];
        r.c[q] += ue[q];
    }
}

// P* along the columns with four taps: push(row n + 2) returns row n (lag 2).
struct PredictCol4 {
    float a[3][kQ], b[3][kQ];  // rows n-1, n, n+1: the even pixel rows (LL, HL positions)
    float c[2][kQ], e[2][kQ];  // rows n, n+1: the odd pixel rows
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            a[0][q] = a[1][q] = a[2][q] = b[0][q] = b[1][q] = b[2][q] = 0.f;
            c[0][q] = c[1][q] = e[0][q] = e[1][q] = 0.f;
        }
    }
    __device__ __forceinline__ void push(const QRow<float>& y, QRow<float>& o) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            o.a[q] = a[1][q];
            o.b[q] = b[1][q];
            o.c[q] = c[0][q] + tap4(a[1][q], a[2][q], a[0][q], y.a[q], kDDp0, kDDp1);
            o.e[q] = e[0][q] + tap4(b[1][q], b[2][q], b[0][q], y.b[q], kDDp0, kDDp1);
            a[0][q] = a[1][q];
            a[1][q] = a[2][q];
            a[2][q] = y.a[q];
            b[0][q] = b[1][q];
            b[1][q] = b[2][q];
            b[2][q] = y.b[q];
            c[0][q] = c[1][q];
            c[1][q] = y.c[q];
            e[0][q] = e[1][q];
            e[1][q] = y.e[q];
        }
    }
};

// U* along the columns with four taps: push(row i + 1) returns row i (lag 1).
struct UpdateCol4 {
    float c[3][kQ], e[3][kQ];  // rows i-2, i-1, i: the odd pixel rows after P*
    float a1[kQ], b1[kQ];      // row i: the even pixel rows
    __device__ __forceinline__ void init() {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            c[0][q] = c[1][q] = c[2][q] = e[0][q] = e[1][q] = e[2][q] = 0.f;
            a1[q] = b1[q] = 0.f;
        }
    }
    __device__ __forceinline__ void push(const QRow<float>& x, QRow<float>& o) {
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
            o.a[q] = a1[q] + tap4(c[1][q], c[2][q], c[0][q], x.c[q], kDD137u0, kDD137u1);
            o.b[q] = b1[q] + tap4(e[1][q], e[2][q], e[0][q], x.e[q], kDD137u0, kDD137u1);
            o.c[q] = c[2][q];
            o.e[q] = e[2][q];
            c[0][q] = c[1][q];
            c[1][q] = c[2][q];
            c[2][q] = x.c[q];
            e[0][q] = e[1][q];
            e[1][q] = e[2][q];
            e[2][q] = x.e[q];
            a1[q] = x.a[q];
            b1[q] = x.b[q];
        }
    }
};

// One Deslauriers-Dubuc level (the non-separable scheme only).  9/7: the four-tap predict and
// the two-tap update (lag 2); 13/7: both four-tap (lag 3).
template <int MODE>
struct FwdPipe<WV_DD97, MODE> {
    static_assert(MODE == MODE_NONSEP || MODE == MODE_ROWS || MODE == MODE_COLS,
                  "the Deslauriers-Dubuc wavelets have the fused scheme and the two-pass one");
    static constexpr int kLag = MODE == MODE_ROWS ? 0 : 2;
    using C = float;
    PredictNS4 pn;
    UpdateNS<float> un;
    PredictCol4 pcol;
    UpdateCol<float> ucol;
    float ll_add;
    __device__ __forceinline__ void init(float ll_add_ = -0.f) {
        ll_add = ll_add_;
        if constexpr (MODE == MODE_NONSEP) { pn.init(); un.init(0.25f); }
        if constexpr (MODE == MODE_COLS) { pcol.init(); ucol.init(0.25f); }
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        if constexpr (MODE == MODE_ROWS) {
            rows_only_dd<WV_DD97>(r);
            return;
        } else {
            QRow<float> t;
            if constexpr (MODE == MODE_NONSEP) { pn.push(r, t); un.push(t); }
            if constexpr (MODE == MODE_COLS) { pcol.push(r, t); ucol.push(t); }
#pragma unroll
            for (int q = 0; q < kQ; ++q) t.a[q] += ll_add;
            r = t;
        }
    }
};

template <int MODE>
struct FwdPipe<WV_DD137, MODE> {
    static_assert(MODE == MODE_NONSEP || MODE == MODE_ROWS || MODE == MODE_COLS,
                  "the Deslauriers-Dubuc wavelets have the fused scheme and the two-pass one");
    static constexpr int kLag = MODE == MODE_ROWS ? 0 : 3;
    using C = float;
    PredictNS4 pn;
    UpdateNS4 un;
    PredictCol4 pcol;
    UpdateCol4 ucol;
    float ll_add;
    __device__ __forceinline__ void init(float ll_add_ = -0.f) {
        ll_add = ll_add_;
        if constexpr (MODE == MODE_NONSEP) { pn.init(); un.init(kDD137u0, kDD137u1); }
        if constexpr (MODE == MODE_COLS) { pcol.init(); ucol.init(); }
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        if constexpr (MODE == MODE_ROWS) {
            rows_only_dd<WV_DD137>(r);
            return;
        } else {
            QRow<float> t, o;
            if constexpr (MODE == MODE_NONSEP) { pn.push(r, t); un.push(t, o); }
            if constexpr (MODE == MODE_COLS) { pcol.push(r, t); ucol.push(t, o); }
#pragma unroll
            for (int q = 0; q < kQ; ++q) o.a[q] += ll_add;
            r = o;
        }
    }
};

template <>
struct InvPipe<WV_DD97> {
    static constexpr int kLag = 2;
    using C = float;
    InvUpdateNS<float> iu;
    InvPredictNS4<false> ip;
    __device__ __forceinline__ void init() {
        iu.init(0.25f);
        ip.init();
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        QRow<float> t;
        iu.push(r);
        ip.push(r, t);
        r = t;
    }
};

template <bool kShared>
struct InvPipeDD137 {
    static constexpr int kLag = 3;
    using C = float;
    InvUpdateNS4<kShared> iu;
    InvPredictNS4<kShared> ip;
    __device__ __forceinline__ void init() {
        iu.init(kDD137u0, kDD137u1);
        ip.init();
    }
    __device__ __forceinline__ void push(QRow<float>& r) {
        QRow<float> t, o;
        iu.push(r, t);
        ip.push(t, o);
        r = o;
    }
};

template <>
struct InvPipe<WV_DD137> : InvPipeDD137<false> {};

// The inverse pipeline of the streaming kernel whose band planes are of type TB: InvPipe, but
// the 13/7 with 32-bit bands takes the shared-shuffle steps (see InvPredictNS4).  Both forms give
// the same bits.
template <int WV, typename TB>
struct InvPipeOf {
    using type = InvPipe<WV>;
};
template <typename TB>
struct InvPipeOf<WV_DD137, TB> {
    using type = InvPipeDD137<sizeof(TB) == 4>;
};

}  // namespace dwt2
