// Device arithmetic of the poroelastic displacement discontinuity kernels
// (influence coefficients of paper Eqs. 2.3-2.5), GB300 path.
//
// Everything is written in the global (x, y) frame for a source placed at
// the origin and a target at z = (x, y):
//
//  * pot_kernel: point source given by its potency (Pxx, Pyy, Pxy) = ds *
//    sym(D (x) n) of a DD vector D across normal n, plus a fluid source q ds.
//    Used for the far field (M2L between Chebyshev nodes, Gauss points of
//    distant elements).  Terms:
//      - drained elastic stress, a homogeneous degree -2 rational function,
//      - poroelastic transient: stress 2G(grad grad psi - I lap psi) of the
//        potential psi = K2 [a(z) g(r^2) + tr(P) Ein(u)], u = r^2/(4 c t),
//        a(z) = (Pyy - Pxx)(x^2 - y^2) - 4 Pxy x y,  g = (1 - F(u))/r^2,
//        F(u) = (1 - e^-u)/u; the Ein term is the diffusion of the point
//        dilatation that the crack opening volume puts at the source,
//      - pore pressure -(alpha/S) Ce [a P(2,u)/r^4 - tr(P) e^-u/(4ct)],
//        P(2,u) = 1 - (1+u) e^-u,
//      - fluid source: p = q E1(u)/(4 pi kappa),
//        sigma = -eta q/(4 pi kappa) [2 F n n + (E1 - F) I].
//  * disl_field: a DD held on the half line starting at the origin (a
//    poroelastic edge dislocation).  A constant-DD element [y1, y2] is
//    disl(x - y1) - disl(x - y2) exactly, at all times and distances, its own
//    midpoint included (the delta lines of the point dilatation cancel along
//    the half line, so the transient needs only e^-u).
//
// All transient functions are evaluated without cancellation: series below
// u = 1, closed forms above.
#pragma once
#include <cuda_runtime.h>
#include "internal.h"

#define DEV __device__ __forceinline__

template <class T> DEV T dexp(T x);
template <> DEV float dexp<float>(float x) { return expf(x); }
template <> DEV double dexp<double>(double x) { return exp(x); }
template <class T> DEV T dlog(T x);
template <> DEV float dlog<float>(float x) { return logf(x); }
template <> DEV double dlog<double>(double x) { return log(x); }

template <class T> struct Prec;
template <> struct Prec<float> { static constexpr int NS = 11; static constexpr int NE = 16; static constexpr int NC = 10; };
template <> struct Prec<double> { static constexpr int NS = 22; static constexpr int NE = 40; static constexpr int NC = 60; };

// e^-u, F, F', F'' with F(u) = (1 - e^-u)/u.
// Above U_BIG e^-u is below the rounding of the algebraic tails (1/u)
template <class T> struct Big;
template <> struct Big<float> { static constexpr float U = 30.f; };
template <> struct Big<double> { static constexpr double U = 70.0; };

// The series branches (u < 1) are rare on the hot path (they serve pairs
// closer than ~2 sqrt(ct)) and long once unrolled, so they live out of line
// and the hot kernels keep a small instruction footprint.
template <class T> struct Tri { T a, b, c; };
template <class T> struct Quad { T a, b, c, d; };

// F = sum (-u)^k/(k+1)!, F' = sum (k+1)(-1)^(k+1) u^k/(k+2)!,
// F'' = sum (k+1)(k+2)(-1)^k u^k/(k+3)!   (Horner, highest term first)
template <class T>
__device__ __noinline__ Tri<T> f_series(T u) {
    T a = 0, b = 0, c = 0;
#pragma unroll
    for (int k = Prec<T>::NS; k >= 0; --k) {
        T f1 = 1, f2 = 1, f3 = 1;
#pragma unroll
        for (int j = 2; j <= k + 1; ++j) f1 *= T(j);
        f2 = f1 * T(k + 2);
        f3 = f2 * T(k + 3);
        T sg = (k & 1) ? T(-1) : T(1);
        a = a * u + sg / f1;
        b = b * u - sg * T(k + 1) / f2;
        c = c * u + sg * T((k + 1) * (k + 2)) / f3;
    }
    return Tri<T>{a, b, c};
}

template <class T>
DEV void f_funcs(T u, T iu, T &e, T &F0, T &F1, T &F2) {
    if (u > Big<T>::U) {
        e = T(0);
        F0 = iu;
        F1 = -iu * iu;
        F2 = T(2) * iu * iu * iu;
        return;
    }
    e = dexp<T>(-u);
    if (u < T(1)) {
        Tri<T> r = f_series<T>(u);
        F0 = r.a; F1 = r.b; F2 = r.c;
    } else {
        F0 = (T(1) - e) * iu;
        F1 = (e - F0) * iu;
        F2 = -(e + T(2) * F1) * iu;
    }
}

// Remainders of F, F', F'' beyond their large-u forms 1/u, -1/u^2, 2/u^3
// (exponentially small, u >= 1): F = 1/u + F0r, F' = -1/u^2 + F1r,
// F'' = 2/u^3 + F2r with F0r = -e/u, F1r = e (1/u + 1/u^2),
// F2r = -e/u - 2 F1r/u.  A transient written with these in place of F,
// F', F'' (ghat, P2h likewise below) is the part of one side of a time
// window that is not a polynomial in c t: the polynomial parts of the two
// sides are subtracted in closed form instead (no cancellation).
template <class T>
DEV void f_rem(T u, T iu, T &e, T &F0, T &F1, T &F2) {
    e = u > Big<T>::U ? T(0) : dexp<T>(-u);
    F0 = -e * iu;
    F1 = e * iu * (T(1) + iu);
    F2 = -e * iu - T(2) * F1 * iu;
}
// ghat = 1/u - 1/u^2 + g0r, ghat' = -1/u^2 + 2/u^3 + g1r,
// ghat'' = 2/u^3 - 6/u^4 + g2r, P2h = 1/u^2 + p2r
template <class T>
DEV void g_rem(T u, T iu, T e, T F0, T F1, T F2, T &g0, T &g1, T &g2, T &p2h) {
    g0 = -F0 * iu;
    g1 = -(F1 + g0) * iu;
    g2 = -(F2 + T(2) * g1) * iu;
    p2h = -(T(1) + u) * e * iu * iu;
}

// ghat = (1 - F)/u and its two derivatives; P2h = P(2,u)/u^2.
// ghat = sum (-1)^k u^k/(k+2)!, ghat' = sum_{k>=1} (-1)^k k u^(k-1)/(k+2)!,
// ghat'' = sum_{k>=2} (-1)^k k(k-1) u^(k-2)/(k+2)!,
// P2h = sum_{k>=2} (-1)^k (k-1) u^(k-2)/k!
template <class T>
__device__ __noinline__ Quad<T> g_series(T u) {
    T a = 0, b = 0, c = 0, d = 0;
#pragma unroll
    for (int k = Prec<T>::NS + 2; k >= 0; --k) {
        T fk = 1;
#pragma unroll
        for (int j = 2; j <= k; ++j) fk *= T(j);
        T fk2 = fk * T(k + 1) * T(k + 2);
        T sg = (k & 1) ? T(-1) : T(1);
        a = a * u + sg / fk2;
        if (k >= 1) b = b * u + sg * T(k) / fk2;
        if (k >= 2) c = c * u + sg * T(k * (k - 1)) / fk2;
        if (k >= 2) d = d * u + sg * T(k - 1) / fk;
    }
    return Quad<T>{a, b, c, d};
}

template <class T>
DEV void g_funcs(T u, T iu, T e, T F0, T F1, T F2, T &g0, T &g1, T &g2, T &p2h) {
    if (u < T(1)) {
        Quad<T> r = g_series<T>(u);
        g0 = r.a; g1 = r.b; g2 = r.c; p2h = r.d;
    } else {
        g0 = (T(1) - F0) * iu;
        g1 = -(F1 + g0) * iu;
        g2 = -(F2 + T(2) * g1) * iu;
        p2h = (T(1) - (T(1) + u) * e) * iu * iu;
    }
}

// Exponential integral E1(u), u > 0: Ein series minus log below 2.5,
// continued fraction (even contraction, bottom-up) above.
template <class T>
DEV T e1(T u) {
    if (u < T(2.5)) {
        T s = 0;
#pragma unroll
        for (int k = Prec<T>::NE; k >= 1; --k) {
            T fk = 1;
#pragma unroll
            for (int j = 2; j <= k; ++j) fk *= T(j);
            T sg = (k & 1) ? T(1) : T(-1);
            s = s * u + sg / (T(k) * fk);
        }
        s *= u;   // Ein(u)
        return s - dlog<T>(u) - T(0.57721566490153286061);
    }
    if (u > Big<T>::U) return T(0);
    T f = u + T(2 * Prec<T>::NC + 1);
#pragma unroll
    for (int k = Prec<T>::NC; k >= 1; --k) f = u + T(2 * k - 1) - T(k * k) / f;
    return dexp<T>(-u) / f;
}

// FP32: Ein series below 1; for 1 <= u <= 30, E1 = e^-u/u * h(1/u) with
// h(t) = u e^u E1(u) as a degree-12 Chebyshev series in
// x = 2 (t - 1/30)/(1 - 1/30) - 1 (Clenshaw; coefficients from
// csrc/fit_e1.py, relative error < 3e-7); 0 above 30.
__constant__ float c_e1cheb[13] = {7.479364044e-01f, -1.782856521e-01f, 3.253978214e-02f, -7.307559064e-03f,
                                   1.867943905e-03f, -5.230081780e-04f, 1.568588335e-04f, -4.967373770e-05f,
                                   1.644605689e-05f, -5.651932686e-06f, 2.005327778e-06f, -7.314854142e-07f,
                                   2.734071549e-07f};
static __device__ __noinline__ float e1f_series(float u) {
    float s = 0.f;
#pragma unroll
    for (int k = 10; k >= 1; --k) {
        float fk = 1.f;
#pragma unroll
        for (int j = 2; j <= k; ++j) fk *= (float)j;
        s = s * u + ((k & 1) ? 1.f : -1.f) / ((float)k * fk);
    }
    return s * u - __logf(u) - 0.5772156649f;
}
DEV float e1f(float u, float iu) {
    if (u < 1.f) return e1f_series(u);
    if (u > 30.f) return 0.f;
    float x = (iu - 1.f / 30.f) * (2.f / (1.f - 1.f / 30.f)) - 1.f;
    float b1 = 0.f, b2 = 0.f;
#pragma unroll
    for (int k = 12; k >= 1; --k) {
        float t = 2.f * x * b1 - b2 + c_e1cheb[k];
        b2 = b1;
        b1 = t;
    }
    return __expf(-u) * iu * (x * b1 - b2 + c_e1cheb[0]);
}
template <class T> DEV T e1x(T u, T iu) { return e1<T>(u); }
template <> DEV float e1x<float>(float u, float iu) { return e1f(u, iu); }

// ---------------------------------------------------------------------------
// point kernel, potency form
// ---------------------------------------------------------------------------
// g0c = 1/(4ct), ct4 = 4ct, ir2 = 1/r^2 (precomputed by the caller).
// REM: only the remainder beyond the polynomial large-u form (u >= 1).
template <class T, bool REM = false>
DEV void pot_transient(const KConst<T> &k, T x, T y, T ir2, T Pxx, T Pyy, T Pxy, T q, T g0c, T ct4, T s,
                       T acc[4]) {
    T x2 = x * x, y2 = y * y, xy = x * y, r2 = x2 + y2;
    T u = r2 * g0c, iu = ct4 * ir2;
    T e, F0, F1, F2, gh0, gh1, gh2, p2h;
    if (REM) {
        f_rem<T>(u, iu, e, F0, F1, F2);
        g_rem<T>(u, iu, e, F0, F1, F2, gh0, gh1, gh2, p2h);
    } else {
        f_funcs<T>(u, iu, e, F0, F1, F2);
        g_funcs<T>(u, iu, e, F0, F1, F2, gh0, gh1, gh2, p2h);
    }
    T dP = Pyy - Pxx, trP = Pxx + Pyy;
    T a = dP * (x2 - y2) - T(4) * Pxy * xy;
    T ax = T(2) * dP * x - T(4) * Pxy * y;
    T ay = -T(2) * dP * y - T(4) * Pxy * x;
    T axx = T(2) * dP, axy = -T(4) * Pxy;
    T g = g0c * gh0, g1 = g0c * g0c * gh1, g2 = g0c * g0c * g0c * gh2;
    T m0a = T(2) * g0c * F0 * trP, m0b = T(4) * g0c * g0c * F1 * trP;
    T pxx = axx * g + T(4) * ax * x * g1 + T(2) * a * g1 + T(4) * a * x2 * g2 + m0a + m0b * x2;
    T pyy = -axx * g + T(4) * ay * y * g1 + T(2) * a * g1 + T(4) * a * y2 * g2 + m0a + m0b * y2;
    T pxy = axy * g + T(2) * (ax * y + ay * x) * g1 + T(4) * a * xy * g2 + m0b * xy;
    T sk = s * k.K2 * k.G2;
    acc[0] -= sk * pyy;                         // 2G (psi_xx - lap psi) = -2G psi_yy
    acc[1] -= sk * pxx;
    acc[2] += sk * pxy;
    acc[3] -= s * k.aS * k.Ce * (a * g0c * g0c * p2h - trP * g0c * e);
    if (q != T(0)) {
        T E1 = e1x<T>(u, iu);
        T pre = s * q * k.i4pk;
        T nn = T(2) * F0 * ir2;
        acc[0] -= pre * k.eta * (nn * x2 + E1 - F0);
        acc[1] -= pre * k.eta * (nn * y2 + E1 - F0);
        acc[2] -= pre * k.eta * (nn * xy);
        acc[3] += pre * E1;
    }
}

// The part of a time window (t_lo > 0) of the point kernel that is
// polynomial in c t at large u: the t-free terms of the two sides cancel,
// what is left is linear in d4ct = 4c (t_hi - t_lo):
//   d4ct * 6 G2 K2 / r^8 * (Q, -Q, -2 R, 0)
//   + fluid source: -eta q/(4 pi kappa) d4ct / r^4 * (x^2-y^2, y^2-x^2, 2xy, 0)
// with Q = (Pxx-Pyy)(x^4 - 6x^2y^2 + y^4) + 8 Pxy xy (x^2-y^2),
//      R = Pxy (x^4 - 6x^2y^2 + y^4) - 2 (Pxx-Pyy) xy (x^2-y^2).
template <class T>
DEV void pot_asym(const KConst<T> &k, T x, T y, T Pxx, T Pyy, T Pxy, T q, T d4ct, T acc[4]) {
    T x2 = x * x, y2 = y * y, xy = x * y;
    T ir2 = T(1) / (x2 + y2), ir4 = ir2 * ir2;
    T d = x2 - y2, dPm = Pxx - Pyy;
    T c4 = d * d - T(4) * x2 * y2, s4 = T(4) * xy * d;
    T f = T(6) * k.G2 * k.K2 * d4ct * ir4 * ir4;
    T Q = dPm * c4 + T(2) * Pxy * s4, R = Pxy * c4 - T(0.5) * dPm * s4;
    T fq = -k.eta * k.i4pk * q * d4ct * ir4;
    acc[0] += f * Q + fq * d;
    acc[1] -= f * Q + fq * d;
    acc[2] += fq * T(2) * xy - T(2) * f * R;
}

// Time element (t_lo > 0) with u >= 1 on both sides (the hi side has the
// smaller u): the polynomial parts of the two sides in closed form, plus
// each side's exponentially small remainder.  Evaluated side by side, the
// two sides' common t-free term (the undrained - drained difference) would
// cancel and take the small window difference with it.  (Kernels that only
// see windows starting at 0 instantiate with t_lo known to be 0, which
// removes this branch from their code.)
template <class T>
DEV Quad<T> pot_window_rem(KConst<T> k, T x, T y, T Pxx, T Pyy, T Pxy, T q, Win<T> w) {
    const T r2 = x * x + y * y, ir2 = T(1) / r2;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    pot_asym<T>(k, x, y, Pxx, Pyy, Pxy, q, T(4) * (w.ct_hi - w.ct_lo), acc);
    if (r2 * w.g_hi <= Big<T>::U) {
        pot_transient<T, true>(k, x, y, ir2, Pxx, Pyy, Pxy, q, w.g_hi, T(4) * w.ct_hi, T(1), acc);
        pot_transient<T, true>(k, x, y, ir2, Pxx, Pyy, Pxy, q, w.g_lo, T(4) * w.ct_lo, T(-1), acc);
    }
    return Quad<T>{acc[0], acc[1], acc[2], acc[3]};
}

template <class T>
DEV void pot_kernel(const KConst<T> &k, T x, T y, T Pxx, T Pyy, T Pxy, T q, const Win<T> &w,
                    T acc[4]) {
    T ir2 = T(1) / (x * x + y * y);
    if (w.ct_lo > T(0) && (x * x + y * y) * w.g_hi >= T(1)) {
        const Quad<T> r = pot_window_rem<T>(k, x, y, Pxx, Pyy, Pxy, q, w);
        acc[0] += r.a; acc[1] += r.b; acc[2] += r.c; acc[3] += r.d;
        return;
    }
    if (w.elastic) {
        T x2 = x * x, y2 = y * y, xy = x * y;
        T C = k.Cel * ir2 * ir2 * ir2;
        T A1 = x2 * x2, B1 = y2 * y2, Cm = x2 * y2;
        acc[0] -= C * (Pxx * (T(3) * A1 - T(6) * Cm - B1) + Pyy * (-A1 + T(6) * Cm - B1) +
                       Pxy * xy * (T(12) * x2 - T(4) * y2));
        acc[1] += C * (Pxx * (A1 - T(6) * Cm + B1) + Pyy * (A1 + T(6) * Cm - T(3) * B1) +
                       Pxy * xy * (T(4) * x2 - T(12) * y2));
        acc[2] += C * (Pxx * xy * (-T(6) * x2 + T(2) * y2) + T(2) * Pxy * (A1 - T(6) * Cm + B1) +
                       Pyy * xy * (T(2) * x2 - T(6) * y2));
    }
    const int sides = w.ct_lo > T(0) ? 2 : 1;
#pragma unroll 1
    for (int sd = 0; sd < sides; ++sd)
        pot_transient<T>(k, x, y, ir2, Pxx, Pyy, Pxy, q, sd ? w.g_lo : w.g_hi, T(4) * (sd ? w.ct_lo : w.ct_hi),
                         sd ? T(-1) : T(1), acc);
}

// Point kernel where u = r^2/(4ct) > Big<float>::U on every side of the
// window, so that e^-u and E1(u) vanish in FP32 (the general path above
// takes the same branches).  Expanding pot_kernel + pot_transient with
// F = 1/u, F' = -1/u^2, F'' = 2/u^3, E1 = 0 gives exactly
//   drained elastic + transient
//     = [elastic window] * (undrained elastic: C_el -> C_el + 2 G2 K2,
//                           pressure aS Ce ((Pxx-Pyy)(x^2-y^2) + 4 Pxy x y)/r^4)
//       + d4ct * 6 G2 K2 / r^8 * ( Q, -Q, -2 R, 0 )
//       + fluid source: -eta q/(4 pi kappa) d4ct / r^4 * (x^2-y^2, y^2-x^2, 2xy, 0)
// with Q = (Pxx-Pyy)(x^4 - 6x^2y^2 + y^4) + 8 Pxy xy (x^2-y^2),
//      R = Pxy (x^4 - 6x^2y^2 + y^4) - 2 (Pxx-Pyy) xy (x^2-y^2),
// d4ct = 4c (t_hi - t_lo) (t_lo = 0 for the elastic window): the t-free
// transient terms of the two sides cancel in a time element.
//
// Evaluated in complex form: with z = x + i y, the potency written as its
// trace Tr = Pxx + Pyy and Pi = (Pxx - Pyy) + 2 i Pxy, and conj(Pi) z^2,
// conj(Pi) z^4 the only angular factors, the elastic stresses are
//   sxx + syy = -2 C Re(conj(Pi) z^2) / r^4,
//   syy - sxx =  2 C (Tr Re(z^2) / r^4 + Re(conj(Pi) z^4) / r^6),
//   sxy       = -  C (Tr Im(z^2) / r^4 + Im(conj(Pi) z^4) / r^6),
// the pressure is aS Ce Re(conj(Pi) z^2) / r^4, and Q = Re(conj(Pi) z^4),
// -2 R = Im(conj(Pi) z^4) (the same expansion regrouped; checked against the
// Cartesian form above to 1e-14 in FP64).  Constants below: ce = C (0 in a
// time element), pc = aS Ce (0 in a time element), fa0 = 6 G2 K2 d4ct,
// fq0 = -eta d4ct / (4 pi kappa).
//
// Exact integral of this large-u point kernel over a straight source element (half-length
// a, unit tangent t = tx + i ty, target at z = zx + i zy from the element's
// midpoint, s over [-a, a]): with D = z^2 - a^2 t^2,
//   int (z - s t)^-2 ds = 2a / D,
//   int (z - s t)^-4 ds = 2a (z^2 + a^2 t^2 / 3) / D^3,
//   int conj(z - s t) (z - s t)^-3 ds = 2a (|z|^2 - a^2) / D^2
// (the last after writing conj(z - s t) = conj(z) - conj(t)^2 (z - (z - s t))),
// and the complex-form terms above are Re/Im of Pi or Tr times these
// (Re(conj(Pi) z^2) / r^4 = Re(Pi / z^2), conj(Pi) z^4 / r^6 = conj(Pi conj(z) / z^3),
// conj(Pi) z^4 / r^8 = conj(Pi / z^4), z^2 / r^4 = conj(1 / z^2)).  Valid
// where u > Big along the whole element; exact at any distance there, and
// free of the cancellation of an end-point difference (checked against a
// 60-point Gauss rule of the point kernel to 5e-14 in FP64 from 1.3 a outward).
// a2t2 = a^2 t^2 (complex), a2 = a^2, ta = 2a; acc += the element's field.
template <class T> DEV T rcp_fast(T x);
template <> DEV float rcp_fast<float>(float x) { return __fdividef(1.f, x); }
template <> DEV double rcp_fast<double>(double x) { return 1.0 / x; }
template <class T>
DEV void elem_bigu(T zx, T zy, T a2tr, T a2ti, T a2, T ta, T Pd, T P2, T Tr, T q, T ce, T pc, T fa0, T fq0,
                   T acc[4]) {
    const T z2r = zx * zx - zy * zy, z2i = T(2) * zx * zy, zz = zx * zx + zy * zy;
    const T dr = z2r - a2tr, di = z2i - a2ti;
    const T inv = rcp_fast<T>(dr * dr + di * di);
    const T ir = dr * inv, ii = -di * inv;                             // 1 / D
    const T jr = ir * ir - ii * ii, ji = T(2) * ir * ii;               // 1 / D^2
    const T kr = jr * ir - ji * ii, ki = jr * ii + ji * ir;            // 1 / D^3
    const T i2r = ta * ir, i2i = ta * ii;
    const T m = ta * (zz - a2);
    const T imr = m * jr, imi = m * ji;
    const T er = a2tr * (T(1) / T(3)) + z2r, ei = a2ti * (T(1) / T(3)) + z2i;
    const T i4r = ta * (er * kr - ei * ki), i4i = ta * (er * ki + ei * kr);
    const T A = Pd * i2r - P2 * i2i;                                   // Re(Pi I2)
    const T rv = Pd * imr - P2 * imi, iv = -(Pd * imi + P2 * imr);     // (Re, -Im)(Pi IM)
    const T q4 = Pd * i4r - P2 * i4i, r4 = -(Pd * i4i + P2 * i4r);     // (Re, -Im)(Pi I4)
    const T s = ce * A;
    const T dv = ce * (Tr * i2r + rv);
    const T sxy = ce * (Tr * i2i - iv);
    const T fq = fq0 * q;
    const T t0 = fa0 * q4 + fq * i2r;
    acc[0] += -s - dv + t0;
    acc[1] += -s + dv - t0;
    acc[2] += sxy + fa0 * r4 - fq * i2i;
    acc[3] += pc * A;
}

// ---------------------------------------------------------------------------
// half-line DD (edge dislocation), DD vector (Dx, Dy)
// ---------------------------------------------------------------------------
// REM: only the remainder beyond the polynomial large-u form (u >= 1; the
// pressure's 1 - e^-u = u F becomes -e^-u)
template <class T, bool REM = false>
DEV void disl_transient(const KConst<T> &k, T zx, T zy, T ir2, T Dx, T Dy, T g0c, T ct4, T s, T acc[4]) {
    T r2 = zx * zx + zy * zy;
    T beta = T(2) * g0c;                        // 1/(2ct)
    T u = r2 * g0c, iu = ct4 * ir2;
    T e, F0, F1, F2;
    if (REM) f_rem<T>(u, iu, e, F0, F1, F2);
    else f_funcs<T>(u, iu, e, F0, F1, F2);
    T V1 = F0 + F1, V2 = F1 + F2;
    T l = Dx * zy - Dy * zx, lx = -Dy, ly = Dx;
    T cm = -k.K2 * beta;
    T lb = l * beta * V2;
    T pxx = cm * (T(2) * lx * zx * V1 + lb * zx * zx + l * V1);
    T pyy = cm * (T(2) * ly * zy * V1 + lb * zy * zy + l * V1);
    T pxy = cm * ((lx * zy + ly * zx) * V1 + lb * zx * zy);
    T sk = s * k.G2;
    acc[0] -= sk * pyy;
    acc[1] -= sk * pxx;
    acc[2] += sk * pxy;
    acc[3] -= s * k.aS * k.Ce * l * ir2 * (u * F0);      // 1 - e^-u = u F(u)
}

// u >= 1 on both sides of a time element (the hi side has the smaller u).
// Written with the large-u forms of the transient functions (F0 = 1/u,
// F1 = -1/u^2, F2 = 2/u^3, e^-u = 0), each side is the same t-independent
// term (the undrained - drained difference) plus a term linear in 4ct/r^2;
// the former cancels exactly between the sides, and evaluated side by side
// it would cost ~log10(u) digits.  What is left of the polynomial part,
// written out: 2 G2 K2 (4 ct_hi - 4 ct_lo) / r^4 times the dislocation's
// angular factors (the pressure terms cancel); then each side's
// exponentially small remainder (zero beyond u = Big).
template <class T>
DEV Quad<T> disl_window_rem(KConst<T> k, T zx, T zy, T Dx, T Dy, Win<T> w, T s) {
    const T r2 = zx * zx + zy * zy, ir2 = T(1) / r2;
    T acc[4] = {T(0), T(0), T(0), T(0)};
    const T l = Dx * zy - Dy * zx;
    const T f = s * T(8) * k.G2 * k.K2 * (w.ct_hi - w.ct_lo) * ir2 * ir2;
    acc[0] -= f * (T(2) * Dx * zy + l - T(4) * l * zy * zy * ir2);
    acc[1] -= f * (l - T(2) * Dy * zx - T(4) * l * zx * zx * ir2);
    acc[2] += f * (Dx * zx - Dy * zy - T(4) * l * zx * zy * ir2);
    if (r2 * w.g_hi <= Big<T>::U) {
        disl_transient<T, true>(k, zx, zy, ir2, Dx, Dy, w.g_hi, T(4) * w.ct_hi, s, acc);
        disl_transient<T, true>(k, zx, zy, ir2, Dx, Dy, w.g_lo, T(4) * w.ct_lo, -s, acc);
    }
    return Quad<T>{acc[0], acc[1], acc[2], acc[3]};
}

template <class T>
DEV void disl_field(const KConst<T> &k, T zx, T zy, T Dx, T Dy, const Win<T> &w, T s, T acc[4]) {
    T ir2 = T(1) / (zx * zx + zy * zy);
    if (w.elastic) {
        T x2 = zx * zx, y2 = zy * zy;
        T C = s * k.Cel * ir2 * ir2;
        acc[0] += C * (Dx * zy * (T(3) * x2 + y2) - Dy * zx * (x2 - y2));
        acc[1] -= C * (Dx * zy * (x2 - y2) + Dy * zx * (x2 + T(3) * y2));
        acc[2] -= C * (x2 - y2) * (Dx * zx + Dy * zy);
    }
    const int sides = w.ct_lo > T(0) ? 2 : 1;
    if (sides == 2 && (zx * zx + zy * zy) * w.g_hi >= T(1)) {
        const Quad<T> r = disl_window_rem<T>(k, zx, zy, Dx, Dy, w, s);
        acc[0] += r.a; acc[1] += r.b; acc[2] += r.c; acc[3] += r.d;
        return;
    }
#pragma unroll 1
    for (int sd = 0; sd < sides; ++sd)
        disl_transient<T>(k, zx, zy, ir2, Dx, Dy, sd ? w.g_lo : w.g_hi, T(4) * (sd ? w.ct_lo : w.ct_hi),
                          sd ? -s : s, acc);
}

// rotate a global (sxx, syy, sxy) into the target frame: (sigma_s, sigma_n)
template <class T>
DEV void to_local(T tx, T ty, const T g[4], T &ss, T &sn) {
    T nx = -ty, ny = tx;
    sn = g[0] * nx * nx + T(2) * g[2] * nx * ny + g[1] * ny * ny;
    ss = g[0] * tx * nx + g[2] * (tx * ny + ty * nx) + g[1] * ty * ny;
}

// ---------------------------------------------------------------------------
// an element on its own midpoint (FP64): dislocation pair at +-a t plus the
// closed-form fluid-source integrals along the line
// ---------------------------------------------------------------------------
__device__ inline void self_field(const KConst<double> &k, const Win<double> &w, double a, double tx, double ty,
                           double Ds, double Dn, double Dq, double out[3]) {
    double nx = -ty, ny = tx;
    double Dx = Ds * tx + Dn * nx, Dy = Ds * ty + Dn * ny;
    double g[4] = {0, 0, 0, 0};
    disl_field<double>(k, a * tx, a * ty, Dx, Dy, w, 1.0, g);      // target - start = a t
    disl_field<double>(k, -a * tx, -a * ty, Dx, Dy, w, -1.0, g);   // target - end   = -a t
    double ss, sn;
    to_local<double>(tx, ty, g, ss, sn);
    double p = g[3];
    // fluid source on its own element: closed forms along the line,
    // int E1(s^2/4ct) ds and int F(s^2/4ct) ds over [-a, a]
    if (Dq != 0.0) {
        for (int side = 0; side < 2; ++side) {
            double ct = side == 0 ? w.ct_hi : w.ct_lo;
            if (ct <= 0.0) continue;
            double sg = side == 0 ? 1.0 : -1.0;
            double s4 = sqrt(4.0 * ct), A = a / s4;
            double sp = 1.7724538509055160273 * erf(A);
            double IE1 = 2.0 * s4 * (A * e1<double>(A * A) + sp);
            double IF = 2.0 * s4 * (sp - (-expm1(-A * A)) / A);
            sn += sg * (-k.eta * k.i4pk * Dq * (IE1 - IF));
            p += sg * k.i4pk * Dq * IE1;
        }
    }
    out[0] = ss; out[1] = sn; out[2] = p;
}

