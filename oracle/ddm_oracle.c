/*
 * FP64 CPU oracle for the fully coupled poroelastic displacement discontinuity
 * method (constant spatial elements, constant temporal elements).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, imports or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA path.
 *
 * What it computes (paper sections cited by equation):
 *   - the influence coefficients A_ij of Eqs. (2.3)-(2.5): stress (sigma_s,
 *     sigma_n) and pore pressure p at an element midpoint caused by a unit
 *     shear DD, normal DD or fluid source held on another element over a time
 *     element.  The paper delegates the closed forms to the poroelastic DDM
 *     literature; here they are built from their definition:
 *       * drained elastic part: Somigliana integral of the plane-strain Kelvin
 *         solution contracted with the moment tensor of the DD,
 *       * poroelastic part: u = u_drained + grad(psi) with
 *         lap(psi) = (eta/G) p and the pore pressure solving the diffusion
 *         equation driven by the drained dilatation (Biot / Rice-Cleary
 *         plane strain),
 *       * fluid source: continuous line source, p = Q/(4 pi kappa) E1(u),
 *     with second derivatives taken exactly by hyper-dual arithmetic,
 *   - element integrals by adaptive Gauss-Legendre quadrature along the
 *     source element; the target's own element is the Hadamard finite part
 *     of the (hypersingular) drained elastic kernel plus regular quadrature
 *     of the smooth transient remainder,
 *   - the dense influence matrix A(t) (step-on response at time t), and the
 *     field at arbitrary points (for pins).
 *
 * Conventions (a reading; the paper states none): SI units, tension-positive
 * stress, D = u(+) - u(-) with the + face on the side the unit normal points
 * to, the normal is the tangent rotated by +90 degrees, D_n > 0 opens the
 * crack.  Unknowns are [Ds(N), Dn(N), Dq(N)]; rows are [sigma_s, sigma_n, p]
 * at element midpoints in each element's own (s, n) frame.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC -o libddm_oracle.so ddm_oracle.c -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define PI 3.14159265358979323846
#define EULER_GAMMA 0.57721566490153286061

/* ------------------------------------------------------------------------ */
/* material                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    double G, nu, nu_u, B, perm, visc;      /* inputs */
    double lam, alpha, eta, M, S, kappa, c, kpsi;
} mat_t;

/* Biot / Rice-Cleary constants from (G, nu, nu_u, B, k, mu). */
static void mat_init(mat_t *m, const double in[6]) {
    m->G = in[0]; m->nu = in[1]; m->nu_u = in[2]; m->B = in[3];
    m->perm = in[4]; m->visc = in[5];
    double G = m->G, nu = m->nu, nuu = m->nu_u, B = m->B;
    m->lam = 2.0 * G * nu / (1.0 - 2.0 * nu);
    m->alpha = 3.0 * (nuu - nu) / (B * (1.0 - 2.0 * nu) * (1.0 + nuu));
    m->eta = m->alpha * (1.0 - 2.0 * nu) / (2.0 * (1.0 - nu));
    m->M = 2.0 * G * (nuu - nu) / (m->alpha * m->alpha * (1.0 - 2.0 * nuu) * (1.0 - 2.0 * nu));
    m->S = m->alpha * m->eta / G + 1.0 / m->M;         /* storage at constant drained strain */
    m->kappa = m->perm / m->visc;                        /* mobility k/mu */
    m->c = m->kappa / m->S;                              /* diffusivity */
    m->kpsi = m->alpha * m->eta / (G * m->S);            /* dimensionless coupling */
}

void orc_constants(const double in[6], double out[8]) {
    mat_t m; mat_init(&m, in);
    out[0] = m.alpha; out[1] = m.eta; out[2] = m.M; out[3] = m.S;
    out[4] = m.kappa; out[5] = m.c; out[6] = m.kpsi; out[7] = m.lam;
}

/* ------------------------------------------------------------------------ */
/* special functions                                                         */
/* ------------------------------------------------------------------------ */
/* Ein(u) = int_0^u (1-e^-v)/v dv, power series (entire function). */
static double ein_series(double u) {
    double s = 0.0, term = 1.0;
    for (int k = 1; k < 200; ++k) {
        term *= -u / k;                 /* (-u)^k / k! */
        double add = -term / k;
        s += add;
        if (fabs(add) < 1e-18 * fabs(s)) break;
    }
    return s;
}
/* E1(u) for u >= 2 by the continued fraction
 * E1(u) = e^-u / (u+1 - 1/(u+3 - 4/(u+5 - ...))), evaluated bottom-up with a
 * depth that is doubled until two successive values agree. */
static double e1_cf(double u) {
    double prev = 0.0;
    for (int depth = 16; depth <= 4096; depth *= 2) {
        double f = u + 2.0 * depth + 1.0;
        for (int k = depth; k >= 1; --k) f = u + 2.0 * k - 1.0 - (double)k * k / f;
        double v = exp(-u) / f;
        if (depth > 16 && fabs(v - prev) <= 1e-16 * fabs(v)) return v;
        prev = v;
    }
    return prev;
}
double orc_e1(double u) {
    if (u <= 0.0) return INFINITY;
    if (u < 2.0) return ein_series(u) - log(u) - EULER_GAMMA;
    return e1_cf(u);
}
double orc_ein(double u) {
    if (u < 2.0) return ein_series(u);
    return orc_e1(u) + log(u) + EULER_GAMMA;
}
/* F(u) = (1 - e^-u)/u and its first two derivatives (series near 0). */
static void Ffun(double u, double *F0, double *F1, double *F2) {
    if (u < 0.5) {
        /* F = sum (-u)^k/(k+1)!, F' = sum_k (k+1)(-1)^(k+1) u^k/(k+2)!,
           F'' = sum_k (k+1)(k+2)(-1)^k u^k/(k+3)! */
        double a = 0, b = 0, c = 0, pk = 1.0;           /* pk = u^k */
        double f1 = 1.0, f2 = 2.0, f3 = 6.0;            /* (k+1)!, (k+2)!, (k+3)! */
        for (int k = 0; k < 30; ++k) {
            double sg = (k & 1) ? -1.0 : 1.0;
            a += sg * pk / f1;
            b += -sg * (k + 1) * pk / f2;
            c += sg * (k + 1) * (k + 2) * pk / f3;
            pk *= u; f1 *= (k + 2); f2 *= (k + 3); f3 *= (k + 4);
        }
        *F0 = a; *F1 = b; *F2 = c;
    } else {
        double e = exp(-u);
        *F0 = (1.0 - e) / u;
        *F1 = (e - *F0) / u;
        *F2 = -(e + 2.0 * (*F1)) / u;
    }
}

/* ------------------------------------------------------------------------ */
/* hyper-dual numbers: value, d/de1, d/de2, d2/de1de2                         */
/* ------------------------------------------------------------------------ */
typedef struct { double v, a, b, ab; } hd;
static hd H(double v) { hd r = {v, 0, 0, 0}; return r; }
static hd hadd(hd x, hd y) { hd r = {x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab}; return r; }
static hd hsub(hd x, hd y) { hd r = {x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab}; return r; }
static hd hmul(hd x, hd y) {
    hd r = {x.v * y.v, x.v * y.a + x.a * y.v, x.v * y.b + x.b * y.v,
            x.v * y.ab + x.a * y.b + x.b * y.a + x.ab * y.v};
    return r;
}
static hd hscale(hd x, double s) { hd r = {x.v * s, x.a * s, x.b * s, x.ab * s}; return r; }
/* apply a scalar function with value f0 and derivatives f1, f2 */
static hd hfun(hd x, double f0, double f1, double f2) {
    hd r = {f0, f1 * x.a, f1 * x.b, f1 * x.ab + f2 * x.a * x.b};
    return r;
}
static hd hinv(hd x) { double i = 1.0 / x.v; return hfun(x, i, -i * i, 2.0 * i * i * i); }
static hd hdiv(hd x, hd y) { return hmul(x, hinv(y)); }
static hd hlog(hd x) { return hfun(x, log(x.v), 1.0 / x.v, -1.0 / (x.v * x.v)); }
static hd hexpneg(hd x) { double e = exp(-x.v); return hfun(x, e, -e, e); }   /* e^-x */
static hd hF(hd u) { double a, b, c; Ffun(u.v, &a, &b, &c); return hfun(u, a, b, c); }
/* 1 - F(u) without cancellation: series sum_{k>=1} (-1)^(k+1) u^k/(k+1)! near 0 */
static hd hOneMinusF(hd u) {
    double a, b, c, g;
    Ffun(u.v, &a, &b, &c);
    if (u.v < 0.5) {
        double term = 1.0, fk = 1.0;
        g = 0.0;
        for (int k = 1; k < 30; ++k) {
            term *= u.v; fk *= (k + 1);
            g += ((k & 1) ? 1.0 : -1.0) * term / fk;
        }
    } else {
        g = 1.0 - a;
    }
    return hfun(u, g, -b, -c);
}
static hd hE1(hd u) {
    double e = exp(-u.v);
    return hfun(u, orc_e1(u.v), -e / u.v, e * (1.0 + u.v) / (u.v * u.v));
}
static hd hEin(hd u) { double a, b, c; Ffun(u.v, &a, &b, &c); return hfun(u, orc_ein(u.v), a, b); }

/* ------------------------------------------------------------------------ */
/* point kernels (response at z = x - y, step-on at time 0, observed at t)   */
/* ------------------------------------------------------------------------ */
/* Plane-strain Kelvin displacement G_ip(z) for a unit force along p. */
static void kelvin(const mat_t *m, hd zx, hd zy, hd Gm[2][2]) {
    hd r2 = hadd(hmul(zx, zx), hmul(zy, zy));
    hd lnr = hscale(hlog(r2), 0.5);
    double pre = 1.0 / (8.0 * PI * m->G * (1.0 - m->nu));
    hd z[2] = {zx, zy};
    for (int i = 0; i < 2; ++i)
        for (int p = 0; p < 2; ++p) {
            hd t = hdiv(hmul(z[i], z[p]), r2);
            if (i == p) t = hsub(t, hscale(lnr, 3.0 - 4.0 * m->nu));
            Gm[i][p] = hscale(t, pre);
        }
}

/* Second derivatives d_j d_q G_ip(z) -> d2G[i][p][q][j]. */
static void kelvin_d2(const mat_t *m, double zx, double zy, double d2G[2][2][2][2]) {
    for (int q = 0; q < 2; ++q)
        for (int j = 0; j < 2; ++j) {
            hd X = {zx, q == 0 ? 1.0 : 0.0, j == 0 ? 1.0 : 0.0, 0.0};
            hd Y = {zy, q == 1 ? 1.0 : 0.0, j == 1 ? 1.0 : 0.0, 0.0};
            hd Gm[2][2];
            kelvin(m, X, Y, Gm);
            for (int i = 0; i < 2; ++i)
                for (int p = 0; p < 2; ++p) d2G[i][p][q][j] = Gm[i][p].ab;
        }
}

/* Moment tensor (per unit element length) of a DD vector D across a surface
 * with unit normal n in the drained medium. */
static void moment(const mat_t *m, const double D[2], const double n[2], double Mt[2][2]) {
    double dn = D[0] * n[0] + D[1] * n[1];
    for (int p = 0; p < 2; ++p)
        for (int q = 0; q < 2; ++q)
            Mt[p][q] = (p == q ? m->lam * dn : 0.0) + m->G * (D[p] * n[q] + D[q] * n[p]);
}

/* Drained elastic stress at z from a point DD (D, n): u_i = -M_pq d_q G_ip. */
static void elastic_dd(const mat_t *m, double zx, double zy, const double D[2], const double n[2],
                       double sig[3]) {
    double d2G[2][2][2][2], Mt[2][2], gu[2][2];
    kelvin_d2(m, zx, zy, d2G);
    moment(m, D, n, Mt);
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double s = 0.0;
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) s -= Mt[p][q] * d2G[i][p][q][j];
            gu[i][j] = s;                          /* du_i/dx_j */
        }
    double exx = gu[0][0], eyy = gu[1][1], exy = 0.5 * (gu[0][1] + gu[1][0]);
    double tr = exx + eyy;
    sig[0] = m->lam * tr + 2.0 * m->G * exx;
    sig[1] = m->lam * tr + 2.0 * m->G * eyy;
    sig[2] = 2.0 * m->G * exy;
}

/* Regular (principal value) drained dilatation of a point DD:
 * div u = -M_pq d_q d_i G_ip with d_i G_ip = -(1-2nu)/(4 pi G (1-nu)) z_p/r^2. */
static hd eps_reg(const mat_t *m, hd zx, hd zy, const double Mt[2][2]) {
    hd r2 = hadd(hmul(zx, zx), hmul(zy, zy));
    hd r4 = hmul(r2, r2);
    double pre = (1.0 - 2.0 * m->nu) / (4.0 * PI * m->G * (1.0 - m->nu));
    double trM = Mt[0][0] + Mt[1][1];
    hd zMz = hadd(hadd(hscale(hmul(zx, zx), Mt[0][0]), hscale(hmul(zy, zy), Mt[1][1])),
                  hscale(hmul(zx, zy), 2.0 * Mt[0][1]));
    /* M_pq d_q (z_p / r^2) = trM / r^2 - 2 zMz / r^4 */
    hd v = hsub(hdiv(H(trM), r2), hscale(hdiv(zMz, r4), 2.0));
    return hscale(v, pre);
}

/* Displacement potential psi of the poroelastic correction of a point DD:
 *   psi = (kpsi/4) r^2 eps_reg (1 - F(u)) - (kpsi Vd / (4 pi)) Ein(u),
 * with Vd = -(1-2nu)(D.n)/(2(1-nu)) the point dilatation that the drained
 * solution puts at the source (fixed by the undrained limit t -> 0+). */
static hd psi_dd(const mat_t *m, hd zx, hd zy, double t, const double Mt[2][2], double dn) {
    hd r2 = hadd(hmul(zx, zx), hmul(zy, zy));
    hd u = hscale(r2, 1.0 / (4.0 * m->c * t));
    hd e = eps_reg(m, zx, zy, Mt);
    hd one_minus_F = hOneMinusF(u);
    hd p2 = hscale(hmul(hmul(r2, e), one_minus_F), 0.25 * m->kpsi);
    double Vd = -(1.0 - 2.0 * m->nu) * dn / (2.0 * (1.0 - m->nu));
    hd p0 = hscale(hEin(u), -m->kpsi * Vd / (4.0 * PI));
    return hadd(p2, p0);
}

/* Displacement potential of a continuous point fluid source of unit rate:
 * radial displacement u_r = (eta/(4 pi kappa G)) (2ct/r)[u E1 + 1 - e^-u], so
 * psi = (eta c t / (4 pi kappa G)) [u E1(u) + 1 - e^-u + Ein(u)]. */
static hd psi_q(const mat_t *m, hd zx, hd zy, double t) {
    hd r2 = hadd(hmul(zx, zx), hmul(zy, zy));
    hd u = hscale(r2, 1.0 / (4.0 * m->c * t));
    hd h = hadd(hadd(hmul(u, hE1(u)), hsub(H(1.0), hexpneg(u))), hEin(u));
    return hscale(h, m->eta * m->c * t / (4.0 * PI * m->kappa * m->G));
}

/* Stress 2G (d_i d_j psi - delta_ij lap psi) of a displacement potential. */
typedef hd (*psi_fn)(const mat_t *, hd, hd, double, const double[2][2], double);
static void psi_stress_dd(const mat_t *m, double zx, double zy, double t, const double Mt[2][2],
                          double dn, double sig[3]) {
    double d[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = i; j < 2; ++j) {
            hd X = {zx, i == 0 ? 1.0 : 0.0, j == 0 ? 1.0 : 0.0, 0.0};
            hd Y = {zy, i == 1 ? 1.0 : 0.0, j == 1 ? 1.0 : 0.0, 0.0};
            d[i][j] = psi_dd(m, X, Y, t, Mt, dn).ab;
        }
    double lap = d[0][0] + d[1][1];
    sig[0] = 2.0 * m->G * (d[0][0] - lap);
    sig[1] = 2.0 * m->G * (d[1][1] - lap);
    sig[2] = 2.0 * m->G * d[0][1];
}
static void psi_stress_q(const mat_t *m, double zx, double zy, double t, double sig[3]) {
    double d[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = i; j < 2; ++j) {
            hd X = {zx, i == 0 ? 1.0 : 0.0, j == 0 ? 1.0 : 0.0, 0.0};
            hd Y = {zy, i == 1 ? 1.0 : 0.0, j == 1 ? 1.0 : 0.0, 0.0};
            d[i][j] = psi_q(m, X, Y, t).ab;
        }
    double lap = d[0][0] + d[1][1];
    sig[0] = 2.0 * m->G * (d[0][0] - lap);
    sig[1] = 2.0 * m->G * (d[1][1] - lap);
    sig[2] = 2.0 * m->G * d[0][1];
}

/* Pore pressure of a point DD: the diffusion of the (regular + point)
 * drained dilatation, p = -(alpha/S)[eps_reg P(2,u) + Vd e^-u/(4 pi c t)]. */
static double p_dd(const mat_t *m, double zx, double zy, double t, const double Mt[2][2], double dn) {
    hd e = eps_reg(m, H(zx), H(zy), Mt);
    double r2 = zx * zx + zy * zy, u = r2 / (4.0 * m->c * t);
    double P2 = (u < 1e-3) ? u * u * (0.5 - u / 3.0 + u * u / 8.0) : 1.0 - (1.0 + u) * exp(-u);
    double Vd = -(1.0 - 2.0 * m->nu) * dn / (2.0 * (1.0 - m->nu));
    return -(m->alpha / m->S) * (e.v * P2 + Vd * exp(-u) / (4.0 * PI * m->c * t));
}
static double p_q(const mat_t *m, double zx, double zy, double t) {
    double u = (zx * zx + zy * zy) / (4.0 * m->c * t);
    return orc_e1(u) / (4.0 * PI * m->kappa);
}

/* Full point kernel.  src: 0 -> unit DD vector D (global) with normal n,
 * 1 -> unit fluid source.  part: bit 1 = drained elastic, bit 2 = transient.
 * out = (sxx, syy, sxy, p).  t <= 0 returns zeros (no response before the
 * source is switched on). */
static void point_kernel(const mat_t *m, double zx, double zy, double t, int src, const double D[2],
                         const double n[2], int part, double out[4]) {
    out[0] = out[1] = out[2] = out[3] = 0.0;
    if (t <= 0.0) return;
    double s[3];
    if (src == 0) {
        double Mt[2][2];
        moment(m, D, n, Mt);
        double dn = D[0] * n[0] + D[1] * n[1];
        if (part & 1) {
            elastic_dd(m, zx, zy, D, n, s);
            out[0] += s[0]; out[1] += s[1]; out[2] += s[2];
        }
        if (part & 2) {
            psi_stress_dd(m, zx, zy, t, Mt, dn, s);
            out[0] += s[0]; out[1] += s[1]; out[2] += s[2];
            out[3] += p_dd(m, zx, zy, t, Mt, dn);
        }
    } else {
        if (part & 2) {     /* the fluid source has no drained-elastic part */
            psi_stress_q(m, zx, zy, t, s);
            out[0] += s[0]; out[1] += s[1]; out[2] += s[2];
            out[3] += p_q(m, zx, zy, t);
        }
    }
}

/* exported for pins: kernel of a point DD (D, n) plus a fluid source Q */
void orc_point_kernel(const double in[6], double zx, double zy, double t, double Dx, double Dy,
                      double nx, double ny, double Q, int part, double out[4]) {
    mat_t m; mat_init(&m, in);
    double D[2] = {Dx, Dy}, n[2] = {nx, ny}, a[4], b[4];
    point_kernel(&m, zx, zy, t, 0, D, n, part, a);
    point_kernel(&m, zx, zy, t, 1, D, n, part, b);
    for (int k = 0; k < 4; ++k) out[k] = a[k] + Q * b[k];
}

/* ------------------------------------------------------------------------ */
/* adaptive Gauss-Legendre quadrature of a vector integrand                  */
/* ------------------------------------------------------------------------ */
#define NGL 10
static double gl_x[NGL], gl_w[NGL];
static int gl_ready = 0;
/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n. */
static void gl_init(void) {
    if (gl_ready) return;
    for (int i = 0; i < NGL; ++i) {
        double x = cos(PI * (i + 0.75) / (NGL + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= NGL; ++k) { double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            dp = NGL * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

#define NV 12          /* 3 source types x 4 outputs */
typedef struct {
    const mat_t *m;
    double tx, ty;          /* target point */
    double y1x, y1y, sx, sy; /* source start point and unit tangent */
    double nx, ny;          /* source normal */
    double t;
    int part;
    double len;             /* element length (bisection stops at 1e-12 len) */
    int self;               /* target is the element midpoint: z = (len/2 - s) t */
} integ_ctx;

static void integrand(const integ_ctx *c, double s, double out[NV]) {
    double zx, zy;
    if (c->self) {               /* exact offset from the midpoint, never 0 at a node */
        zx = (0.5 * c->len - s) * c->sx; zy = (0.5 * c->len - s) * c->sy;
    } else {
        zx = c->tx - (c->y1x + s * c->sx); zy = c->ty - (c->y1y + s * c->sy);
    }
    double n[2] = {c->nx, c->ny};
    double Ds[2] = {c->sx, c->sy}, Dn[2] = {c->nx, c->ny};
    point_kernel(c->m, zx, zy, c->t, 0, Ds, n, c->part, out + 0);
    point_kernel(c->m, zx, zy, c->t, 0, Dn, n, c->part, out + 4);
    point_kernel(c->m, zx, zy, c->t, 1, Dn, n, c->part, out + 8);
}
static void gl_rule(const integ_ctx *c, double a, double b, double out[NV]) {
    double h = 0.5 * (b - a), mid = 0.5 * (a + b), f[NV];
    for (int k = 0; k < NV; ++k) out[k] = 0.0;
    for (int i = 0; i < NGL; ++i) {
        integrand(c, mid + h * gl_x[i], f);
        for (int k = 0; k < NV; ++k) out[k] += h * gl_w[i] * f[k];
    }
}
/* recursive bisection: accept when the two-half estimate agrees with the
 * whole-interval estimate within a tolerance proportional to the interval's
 * share of the element (per source type, relative to its scale), floored at
 * rounding level so that only a branch running into a singular point goes
 * deep (bounded by the depth limit). */
static void adapt(const integ_ctx *c, double a, double b, const double whole[NV], const double scale[3],
                  double tol_per_len, int depth, double out[NV]) {
    double m = 0.5 * (a + b), L[NV], R[NV];
    gl_rule(c, a, m, L);
    gl_rule(c, m, b, R);
    int ok = 1;
    for (int k = 0; k < NV; ++k) {
        double lim = fmax(tol_per_len * (b - a), 1e-15) * scale[k / 4];
        if (fabs(L[k] + R[k] - whole[k]) > lim) { ok = 0; break; }
    }
    if (ok || depth > 55 || (b - a) < 1e-12 * c->len) {
        for (int k = 0; k < NV; ++k) out[k] = L[k] + R[k];
        return;
    }
    double oL[NV], oR[NV];
    adapt(c, a, m, L, scale, tol_per_len, depth + 1, oL);
    adapt(c, m, b, R, scale, tol_per_len, depth + 1, oR);
    for (int k = 0; k < NV; ++k) out[k] = oL[k] + oR[k];
}
static void integrate(const integ_ctx *c, double a, double b, const double *scale_floor, double out[NV]) {
    double whole[NV], scale[3];
    gl_rule(c, a, b, whole);
    /* scale from a refined first estimate so a near-singular start does not
       shrink it */
    double L[NV], R[NV];
    gl_rule(c, a, 0.5 * (a + b), L);
    gl_rule(c, 0.5 * (a + b), b, R);
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int k = 0; k < 4; ++k) {
            s = fmax(s, fabs(whole[4 * j + k]));
            s = fmax(s, fabs(L[4 * j + k] + R[4 * j + k]));
        }
        if (scale_floor) s = fmax(s, scale_floor[j]);
        scale[j] = s > 0.0 ? s : 1e-300;
    }
    adapt(c, a, b, whole, scale, 1e-13 / (b - a), 0, out);
}

/* ------------------------------------------------------------------------ */
/* element influence                                                         */
/* ------------------------------------------------------------------------ */
/* Global field (sxx, syy, sxy, p) at point (px, py) from unit Ds, Dn, Dq on
 * element (x0,y0)-(x1,y1), step-on response at time t.  self != 0 means the
 * point is the element's own midpoint. */
static void element_field(const mat_t *m, double px, double py, double x0, double y0, double x1,
                          double y1, double t, int self, double out[NV]) {
    gl_init();
    for (int k = 0; k < NV; ++k) out[k] = 0.0;
    if (t <= 0.0) return;
    double L = hypot(x1 - x0, y1 - y0);
    integ_ctx c = {m, px, py, x0, y0, (x1 - x0) / L, (y1 - y0) / L, 0, 0, t, 3, L, self};
    c.nx = -c.sy; c.ny = c.sx;
    if (!self) {
        integrate(&c, 0.0, L, NULL, out);
        return;
    }
    /* own element.  Drained elastic part: Hadamard finite part.  On the
       element line the kernel is homogeneous of degree -2 and even,
       K(tau s) = K(s)/tau^2, and f.p. int_{-a}^{a} dtau/tau^2 = -2/a. */
    double a = 0.5 * L, sv[3], el[NV] = {0};
    double n[2] = {c.nx, c.ny}, Ds[2] = {c.sx, c.sy}, Dn[2] = {c.nx, c.ny};
    elastic_dd(m, c.sx, c.sy, Ds, n, sv);
    for (int k = 0; k < 3; ++k) el[k] = -2.0 / a * sv[k];
    elastic_dd(m, c.sx, c.sy, Dn, n, sv);
    for (int k = 0; k < 3; ++k) el[4 + k] = -2.0 / a * sv[k];
    /* transient parts are regular (the fluid-source pressure has an
       integrable log singularity at the midpoint, reached by bisection toward
       the split point); tolerance relative to the full self coefficient */
    double floor3[3] = {0, 0, 0};
    for (int k = 0; k < 4; ++k) { floor3[0] = fmax(floor3[0], fabs(el[k])); floor3[1] = fmax(floor3[1], fabs(el[4 + k])); }
    double A[NV], Bv[NV];
    c.part = 2;
    integrate(&c, 0.0, 0.5 * L, floor3, A);
    integrate(&c, 0.5 * L, L, floor3, Bv);
    for (int k = 0; k < NV; ++k) out[k] = A[k] + Bv[k] + el[k];
}

/* rotate (sxx, syy, sxy) into the frame (t, n) of a target element */
static void to_local(double tx, double ty, const double g[4], double *ss, double *sn, double *p) {
    double nx = -ty, ny = tx;
    *sn = g[0] * nx * nx + 2.0 * g[2] * nx * ny + g[1] * ny * ny;
    *ss = g[0] * tx * nx + g[2] * (tx * ny + ty * nx) + g[1] * ty * ny;
    *p = g[3];
}

/* 3x3 block: rows (sigma_s, sigma_n, p) at target element i's midpoint,
 * columns (Ds, Dn, Dq) of source element j. */
static void block(const mat_t *m, const double *xy, int64_t N, int64_t i, int64_t j, double t,
                  double out[3][3]) {
    const double *X0 = xy, *Y0 = xy + N, *X1 = xy + 2 * N, *Y1 = xy + 3 * N;
    double px = 0.5 * (X0[i] + X1[i]), py = 0.5 * (Y0[i] + Y1[i]);
    double Li = hypot(X1[i] - X0[i], Y1[i] - Y0[i]);
    double tx = (X1[i] - X0[i]) / Li, ty = (Y1[i] - Y0[i]) / Li;
    double f[NV];
    element_field(m, px, py, X0[j], Y0[j], X1[j], Y1[j], t, i == j, f);
    for (int col = 0; col < 3; ++col) {
        double ss, sn, p;
        to_local(tx, ty, f + 4 * col, &ss, &sn, &p);
        out[0][col] = ss; out[1][col] = sn; out[2][col] = p;
    }
}

/* Rows `rows[0..nrows)` (indices into the 3N unknowns/equations) of the
 * dense influence matrix A(t), written row-major to A (nrows x 3N). */
void orc_assemble_rows(const double in[6], const double *xy, int64_t N, double t,
                       const int64_t *rows, int64_t nrows, double *A) {
    mat_t m; mat_init(&m, in);
    gl_init();
    /* group requested rows by target element so each block is computed once */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t row = rows[r], i = row % N, comp = row / N;
        int first = 1;
        for (int64_t q = 0; q < r; ++q) if (rows[q] % N == i) { first = 0; break; }
        if (!first) continue;
        for (int64_t j = 0; j < N; ++j) {
            double b[3][3];
            block(&m, xy, N, i, j, t, b);
            for (int64_t q = r; q < nrows; ++q) {
                if (rows[q] % N != i) continue;
                int c2 = (int)(rows[q] / N);
                for (int col = 0; col < 3; ++col) A[q * 3 * N + col * N + j] = b[c2][col];
            }
        }
        (void)comp;
    }
}

/* Full dense influence matrix A(t), row-major 3N x 3N. */
void orc_assemble(const double in[6], const double *xy, int64_t N, double t, double *A) {
    mat_t m; mat_init(&m, in);
    gl_init();
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            double b[3][3];
            block(&m, xy, N, i, j, t, b);
            for (int r = 0; r < 3; ++r)
                for (int col = 0; col < 3; ++col) A[(r * N + i) * 3 * N + col * N + j] = b[r][col];
        }
}

/* Global field (sxx, syy, sxy, p) at arbitrary points from element sources
 * D = [Ds, Dn, Dq] (3N), step-on response at time t.  Points must not lie on
 * an element unless flagged in on_elem (index of that element, or -1 for a
 * point lying on no element; -1 everywhere is the usual case). */
void orc_field(const double in[6], const double *xy, int64_t N, double t, const double *D,
               const double *pts, int64_t npts, const int64_t *on_elem, double *out) {
    mat_t m; mat_init(&m, in);
    gl_init();
    const double *X0 = xy, *Y0 = xy + N, *X1 = xy + 2 * N, *Y1 = xy + 3 * N;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < npts; ++q) {
        double acc[4] = {0, 0, 0, 0};
        for (int64_t j = 0; j < N; ++j) {
            double f[NV];
            element_field(&m, pts[2 * q], pts[2 * q + 1], X0[j], Y0[j], X1[j], Y1[j], t,
                          on_elem && on_elem[q] == j, f);
            for (int k = 0; k < 4; ++k) acc[k] += f[k] * D[j] + f[4 + k] * D[N + j] + f[8 + k] * D[2 * N + j];
        }
        for (int k = 0; k < 4; ++k) out[4 * q + k] = acc[k];
    }
}

/* Single element field, exported for pins (12 values: 3 sources x 4 outputs). */
void orc_element_field(const double in[6], double px, double py, double x0, double y0, double x1,
                       double y1, double t, int self, double out[12]) {
    mat_t m; mat_init(&m, in);
    element_field(&m, px, py, x0, y0, x1, y1, t, self, out);
}

int orc_num_threads(void) {
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
