"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself:
closed forms (Sneddon/Griffith crack opening, K_I = p sqrt(pi a)), the field
equations (equilibrium, compatibility, diffusion), conservation of fluid
mass, the undrained/drained limits, values printed in the paper, library
special functions, and geometric invariances.  CPU only."""
import json
import math
import os

import numpy as np
import pytest
import scipy.special as sc

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
MAT = (6e9, 0.2, 0.33, 0.8, 1e-18, 1e-3)        # G, nu, nu_u, B, k, mu (single-crack case)


def crack(N=200, a=1.0, angle=0.0, x0=0.0, y0=0.0):
    xs = np.linspace(-a, a, N + 1)
    c, s = math.cos(angle), math.sin(angle)
    return np.array([x0 + c * xs[:-1], y0 + s * xs[:-1], x0 + c * xs[1:], y0 + s * xs[1:]]), \
        0.5 * (xs[:-1] + xs[1:])


# ----------------------------------------------------------------------------
# special functions and constants
# ----------------------------------------------------------------------------
def test_e1_ein_against_scipy():
    for u in [1e-8, 1e-3, 0.1, 0.7, 1.5, 1.999, 2.0, 2.5, 7.0, 30.0, 200.0]:
        ref = sc.exp1(u)
        assert abs(oracle.e1(u) / ref - 1) < 1e-13, u
        if u > 1e-3:   # Ein from scipy via E1 + ln u + gamma (exact enough away from 0)
            assert abs(oracle.ein(u) / (ref + math.log(u) + np.euler_gamma) - 1) < 1e-12, u
    # Ein near 0 against its defining integral
    from scipy.integrate import quad
    for u in [1e-6, 1e-2, 0.5]:
        v, _ = quad(lambda s: -np.expm1(-s) / s, 0, u, epsabs=0, epsrel=1e-13)
        assert abs(oracle.ein(u) / v - 1) < 1e-12


def test_diffusivity_closed_form():
    """c from the Detournay-Cheng closed form in (k/mu, B, G, nu, nu_u)."""
    G, nu, nuu, B, k, mu = MAT
    kap = k / mu
    c_ref = 2 * kap * B ** 2 * G * (1 - nu) * (1 + nuu) ** 2 / (9 * (1 - nuu) * (nuu - nu))
    assert abs(oracle.constants(MAT)["c"] / c_ref - 1) < 1e-13


def test_biot_alpha_matches_paper_table():
    """Table 1 prints alpha = 0.449 for Westerly granite (3 digits)."""
    g = json.load(open(os.path.join(HERE, "golden", "westerly_granite.json")))
    a = oracle.constants((g["G"], g["nu"], g["nu_u"], g["B"], g["perm"], 1e-3))["alpha"]
    assert abs(a - g["alpha"]) < 0.0025


# ----------------------------------------------------------------------------
# point kernels satisfy the field equations
# ----------------------------------------------------------------------------
def _fields(z, t, src):
    if src == "dd":
        return oracle.point_kernel(MAT, z, t, D=(0.3, -0.8), n=(0.6, 0.8))
    return oracle.point_kernel(MAT, z, t, Q=1e-12)


@pytest.mark.parametrize("src", ["dd", "q"])
@pytest.mark.parametrize("z,t", [((0.13, -0.21), 200.0), ((0.02, 0.05), 50.0), ((1.3, 0.4), 5e4)])
def test_point_kernel_field_equations(src, z, t):
    c = oracle.constants(MAT)
    G, lam, alpha, M, kap = MAT[0], c["lam"], c["alpha"], c["M"], c["kappa"]
    r = math.hypot(*z)
    h = 2e-3 * r

    def F(x, y, tt=t):
        return _fields((x, y), tt, src)

    def d(fn, ax, x, y, hh=h):   # 4th-order central difference
        if ax == 0:
            return (-fn(x + 2 * hh, y) + 8 * fn(x + hh, y) - 8 * fn(x - hh, y) + fn(x - 2 * hh, y)) / (12 * hh)
        return (-fn(x, y + 2 * hh) + 8 * fn(x, y + hh) - 8 * fn(x, y - hh) + fn(x, y - 2 * hh)) / (12 * hh)

    x, y = z
    s0 = F(x, y)
    scale = np.max(np.abs(s0[:3])) / r
    dx, dy = d(F, 0, x, y), d(F, 1, x, y)
    # equilibrium of total stress
    assert abs(dx[0] + dy[2]) < 1e-6 * scale
    assert abs(dx[2] + dy[1]) < 1e-6 * scale

    def strain(x, y):
        s = F(x, y)
        e = (s[0] + s[1] + 2 * alpha * s[3]) / (2 * (lam + G))
        return np.array([(s[0] - lam * e + alpha * s[3]) / (2 * G),
                         (s[1] - lam * e + alpha * s[3]) / (2 * G), s[2] / (2 * G), e, s[3]])

    # compatibility of the strain derived from stress and pore pressure
    hc = 2e-3 * r
    exx_yy = (strain(x, y + hc)[0] - 2 * strain(x, y)[0] + strain(x, y - hc)[0]) / hc ** 2
    eyy_xx = (strain(x + hc, y)[1] - 2 * strain(x, y)[1] + strain(x - hc, y)[1]) / hc ** 2
    exy_xy = (strain(x + hc, y + hc)[2] - strain(x + hc, y - hc)[2] - strain(x - hc, y + hc)[2]
              + strain(x - hc, y - hc)[2]) / (4 * hc ** 2)
    emag = np.max(np.abs(strain(x, y)[:3])) / r ** 2
    assert abs(exx_yy + eyy_xx - 2 * exy_xy) < 3e-4 * emag
    # fluid mass: d(zeta)/dt = kappa lap(p), zeta = alpha eps + p/M
    ht = 1e-4 * t

    def zeta(tt):
        s = F(x, y, tt)
        e = (s[0] + s[1] + 2 * alpha * s[3]) / (2 * (lam + G))
        return alpha * e + s[3] / M

    zt = (zeta(t + ht) - zeta(t - ht)) / (2 * ht)
    p = lambda a, b: F(a, b)[3]
    lap = (p(x + h, y) + p(x - h, y) + p(x, y + h) + p(x, y - h) - 4 * p(x, y)) / h ** 2
    assert abs(zt - kap * lap) < 2e-4 * max(abs(zt), abs(kap * lap))


def test_point_kernel_limits():
    """t -> 0+: the response is the undrained elastic one (nu -> nu_u);
    t -> inf: the drained one (transient part -> 0)."""
    z = (0.4, -0.25)
    und = list(MAT)
    und[1] = MAT[2]
    for D, n in [((1.0, 0.0), (0.0, 1.0)), ((0.3, 0.7), (0.6, 0.8))]:
        early = oracle.point_kernel(MAT, z, 1e-9, D=D, n=n)
        el_u = oracle.point_kernel(und, z, 1e-9, D=D, n=n, part=1)
        assert np.allclose(early[:3], el_u[:3], rtol=1e-9, atol=1e-9 * np.abs(el_u).max())
        late = oracle.point_kernel(MAT, z, 1e14, D=D, n=n, part=2)
        el_d = oracle.point_kernel(MAT, z, 1e14, D=D, n=n, part=1)
        assert np.max(np.abs(late)) < 1e-6 * np.max(np.abs(el_d))


def test_fluid_source_mass_balance():
    """Fluid content of a constant element source integrates to q L t
    (S p integrated over the plane; kernel normalisation 1/(4 pi kappa))."""
    c = oracle.constants(MAT)
    t = 100.0
    L = 0.02
    Rd = math.sqrt(4 * c["c"] * t)
    xy = np.array([[-L / 2], [0.0], [L / 2], [0.0]])
    D = np.array([0.0, 0.0, 1e-9])
    # polar grid around the element centre (log-spaced radius)
    rs = np.geomspace(1e-2 * Rd, 12 * Rd, 60)
    th = np.linspace(0, 2 * np.pi, 24, endpoint=False) + 0.01
    R, T = np.meshgrid(rs, th, indexing="ij")
    pts = np.stack([R * np.cos(T), R * np.sin(T)], -1).reshape(-1, 2)
    p = oracle.field(MAT, xy, D, t, pts)[:, 3].reshape(R.shape)
    ring = p.mean(axis=1) * 2 * np.pi * rs
    total = c["S"] * np.trapezoid(ring, rs)
    assert abs(total / (L * 1e-9 * t) - 1) < 5e-3


# ----------------------------------------------------------------------------
# element integration
# ----------------------------------------------------------------------------
def test_self_term_is_limit_of_adjacent_field():
    """The element's own coefficient (Hadamard finite part of the drained
    kernel + regular transient) equals the limit of the field at points
    approaching the midpoint from either face."""
    y0, y1 = (0.0, 0.0), (0.02, 0.0)
    for t in [10.0, 1e4]:
        f_self = oracle.element_field(MAT, (0.01, 0.0), y0, y1, t, True)
        lims = []
        for side in (+1, -1):
            eps = np.array([4e-5, 2e-5, 1e-5])
            vals = np.array([oracle.element_field(MAT, (0.01, side * e), y0, y1, t) for e in eps])
            # Richardson on the two finest values (field is smooth in eps, O(eps))
            lims.append(2 * vals[2] - vals[1])
        for lim in lims:
            for src in (0, 1):                # DD columns: stresses and p
                scale = np.abs(f_self[src]).max()
                assert np.allclose(lim[src], f_self[src], atol=2e-3 * scale)


def test_element_quadrature_against_composite_rule():
    """Adaptive element integrals equal a plain composite trapezoid-free
    Gauss rule with many panels for well-separated targets."""
    from numpy.polynomial.legendre import leggauss
    xg, wg = leggauss(8)
    y0, y1 = np.array([0.1, -0.05]), np.array([0.13, -0.01])
    L = np.linalg.norm(y1 - y0)
    tv = (y1 - y0) / L
    nv = np.array([-tv[1], tv[0]])
    target = np.array([0.16, 0.03])
    t = 30.0
    ref = np.zeros((3, 4))
    panels = 64
    for k in range(panels):
        a, b = k * L / panels, (k + 1) * L / panels
        for xi, wi in zip(xg, wg):
            s = 0.5 * (a + b) + 0.5 * (b - a) * xi
            z = target - (y0 + s * tv)
            w = 0.5 * (b - a) * wi
            ref[0] += w * oracle.point_kernel(MAT, z, t, D=tv, n=nv)
            ref[1] += w * oracle.point_kernel(MAT, z, t, D=nv, n=nv)
            ref[2] += w * oracle.point_kernel(MAT, z, t, Q=1.0)
    got = oracle.element_field(MAT, target, y0, y1, t)
    for r in range(3):
        assert np.allclose(got[r], ref[r], rtol=1e-10, atol=1e-10 * np.abs(ref[r]).max())


def test_rotation_and_translation_invariance():
    """Local-frame coefficients do not depend on where the crack pair sits or
    how it is oriented (catches transposed indices / frame mistakes)."""
    def pair(angle, shift):
        c, s = math.cos(angle), math.sin(angle)
        base = np.array([[0.0, 0.0, 0.05, 0.0], [0.02, 0.07, 0.06, 0.1]])  # two elements
        out = np.zeros((4, 2))
        for e in range(2):
            for k in range(2):
                x, y = base[e, 2 * k], base[e, 2 * k + 1]
                out[2 * k, e] = c * x - s * y + shift[0]
                out[2 * k + 1, e] = s * x + c * y + shift[1]
        return out
    A0 = oracle.assemble(MAT, pair(0.0, (0, 0)), 20.0)
    A1 = oracle.assemble(MAT, pair(1.1, (3.0, -7.0)), 20.0)
    assert np.allclose(A0, A1, rtol=1e-9, atol=1e-9 * np.abs(A0).max())


# ----------------------------------------------------------------------------
# closed-form crack solutions
# ----------------------------------------------------------------------------
def _opening_check(t, nu_eff, drained):
    N, a, p = 200, 1.0, 1e6
    xy, xm = crack(N, a)
    A = oracle.assemble(MAT, xy, t)
    b = oracle.rhs(xy, p_f=p, system="impermeable")
    x = oracle.solve(A, b, N, "impermeable")
    Dn = x[N:2 * N]
    w = 2 * (1 - nu_eff) * p / MAT[0] * np.sqrt(a * a - xm ** 2)
    mid = np.abs(xm) <= 0.8 * a
    assert np.max(np.abs(Dn[mid] / w[mid] - 1)) < 0.01
    assert abs(Dn[N // 2] / w[N // 2] - 1) < 0.005
    assert np.max(np.abs(x[:N])) < 1e-12 * np.max(np.abs(Dn))
    KI, _ = oracle.sif(MAT, xy, x, [0, N - 1], drained=drained)
    assert np.all(np.abs(KI / (p * math.sqrt(math.pi * a)) - 1) < 0.02)


def test_sneddon_drained_limit():
    _opening_check(1e12, MAT[1], True)


def test_sneddon_undrained_limit():
    _opening_check(1e-4, MAT[2], False)


def test_shear_crack_inclined_drained():
    """Inclined crack under uniform far-field shear (drained): sliding
    profile Ds = 2(1-nu) tau/G sqrt(a^2-x^2) and K_II = tau sqrt(pi a)."""
    N, a, angle = 120, 1.0, 0.6
    xy, xm = crack(N, a, angle, x0=3.0, y0=-2.0)
    A = oracle.assemble(MAT, xy, 1e12)
    tau = 2e6
    b = np.zeros(3 * N)
    b[:N] = -tau                                  # induced shear cancels the applied one
    x = oracle.solve(A, b, N, "impermeable")
    Ds = x[:N]
    w = 2 * (1 - MAT[1]) * tau / MAT[0] * np.sqrt(a * a - xm ** 2)
    mid = np.abs(xm) <= 0.8 * a
    assert np.max(np.abs(Ds[mid] / w[mid] - 1)) < 0.012
    _, KII = oracle.sif(MAT, xy, x, [0, N - 1])
    assert np.all(np.abs(np.abs(KII) / (tau * math.sqrt(math.pi * a)) - 1) < 0.02)


def test_olson_factor_matches_paper():
    g = json.load(open(os.path.join(HERE, "golden", "olson_sif.json")))
    N = 4
    xy, _ = crack(N)
    x = np.zeros(3 * N)
    x[N] = 1e-4
    KI, _ = oracle.sif(MAT, xy, x, [0])
    G, nu = MAT[0], MAT[1]
    E = 2 * G * (1 + nu)
    a = 0.25
    assert abs(KI[0] - g["factor"] * E / (4 * (1 - nu * nu)) * math.sqrt(math.pi / (2 * a)) * 1e-4) < 1e-6


# ----------------------------------------------------------------------------
# time marching
# ----------------------------------------------------------------------------
def test_history_telescopes_for_constant_history():
    """With the same D on every time element, the history sum plus the
    current-step product equals the step-on response A(t_h) D (Eqs. 2.3-2.5
    with constant temporal elements)."""
    xy, _ = crack(12, 0.5)
    N = 12
    rng = np.random.default_rng(1)
    D = rng.standard_normal(3 * N) * np.r_[np.full(2 * N, 1e-4), np.full(N, 1e-9)]
    times = np.array([0.0, 7.0, 19.0, 40.0, 71.0])      # non-uniform steps, H = 3 past steps
    hist = np.array([D, D, D])
    lhs = oracle.history(MAT, xy, hist, times) + oracle.matvec(MAT, xy, D, 0.0, times[-1] - times[-2])
    rhs = oracle.matvec(MAT, xy, D, 0.0, times[-1])
    assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-10 * np.abs(rhs).max())


def test_march_matches_single_solve_for_one_step():
    xy, _ = crack(16, 0.5)
    N = 16
    b = oracle.rhs(xy, sigma_H=3e6, sigma_h=2e6, p_f=5e6, p0=1e6)
    x1 = oracle.march(MAT, xy, [0.0, 10.0], [b])[0]
    x2 = oracle.solve(oracle.assemble(MAT, xy, 10.0), b, N)
    assert np.allclose(x1, x2, rtol=1e-12)


# ----------------------------------------------------------------------------
# far-field loads resolved on inclined cracks, and the RATE system
# ----------------------------------------------------------------------------
def _resolved(angle, sigma_H, sigma_h):
    """Cauchy resolution of the far field diag(sigma_H, sigma_h)
    (compression positive) on a crack with tangent (cos, sin) and normal
    (-sin, cos): compressive normal stress and tension-positive shear."""
    s, c = math.sin(angle), math.cos(angle)
    return sigma_H * s * s + sigma_h * c * c, (sigma_H - sigma_h) * s * c


def _profile(nu_eff, load, xm, a):
    return 2 * (1 - nu_eff) * load / MAT[0] * np.sqrt(a * a - xm ** 2)


@pytest.mark.parametrize("angle", [0.3, 0.9, 2.2])
def test_far_field_on_inclined_crack_drained(angle):
    """oracle.rhs under sigma_H != sigma_h plus p_f (paper Sec. 4 far-field
    transform) on an inclined crack, drained limit: the opening follows
    Sneddon with the net load p_f - sigma_nn, the sliding follows the shear
    analogue with the resolved shear (sign included), and Eq. 2.6 gives
    K_I = (p_f - sigma_nn) sqrt(pi a), K_II = tau sqrt(pi a)."""
    N, a = 120, 1.0
    sH, sh, pf = 3e6, 2e6, 5e6
    xy, xm = crack(N, a, angle, x0=3.0, y0=-2.0)
    A = oracle.assemble(MAT, xy, 1e12)
    x = oracle.solve(A, oracle.rhs(xy, sigma_H=sH, sigma_h=sh, p_f=pf, system="impermeable"), N, "impermeable")
    snn, tau = _resolved(angle, sH, sh)
    mid = np.abs(xm) <= 0.8 * a
    wn, ws = _profile(MAT[1], pf - snn, xm, a), _profile(MAT[1], tau, xm, a)
    assert np.max(np.abs(x[N:2 * N][mid] / wn[mid] - 1)) < 0.012
    assert np.max(np.abs(x[:N][mid] / ws[mid] - 1)) < 0.012
    KI, KII = oracle.sif(MAT, xy, x, [0, N - 1])
    assert np.all(np.abs(KI / ((pf - snn) * math.sqrt(math.pi * a)) - 1) < 0.02)
    assert np.all(np.abs(KII / (tau * math.sqrt(math.pi * a)) - 1) < 0.02)


def test_rate_system_drained_reduces_to_sneddon():
    """RATE system (rows sigma_s and sigma_n + p, D_q prescribed) with
    D_q = 0 in the drained limit: the DDs induce no pore pressure, so the
    solution is Sneddon's with the net load p0 - sigma_nn and the shear
    analogue with the resolved shear."""
    N, a, angle = 120, 1.0, 0.7
    sH, sh, p0 = 3e6, 2e6, 6e6
    xy, xm = crack(N, a, angle)
    A = oracle.assemble(MAT, xy, 1e12)
    x = oracle.solve(A, oracle.rhs(xy, sigma_H=sH, sigma_h=sh, p0=p0, system="rate"), N, "rate", Dq=0.0)
    snn, tau = _resolved(angle, sH, sh)
    mid = np.abs(xm) <= 0.8 * a
    assert np.max(np.abs(x[N:2 * N][mid] / _profile(MAT[1], p0 - snn, xm, a)[mid] - 1)) < 0.012
    assert np.max(np.abs(x[:N][mid] / _profile(MAT[1], tau, xm, a)[mid] - 1)) < 0.012
    assert np.all(x[2 * N:] == 0.0)


def test_rate_system_undrained_skempton():
    """RATE system with D_q = 0 in the undrained limit.  On the faces of a
    uniformly pressurised Griffith crack both in-plane stresses equal -p_net
    (Westergaard), so Skempton's undrained pore pressure in plane strain is
    p = -B (1 + nu_u)(sigma_xx + sigma_yy) / 3 = 2 B (1 + nu_u) p_net / 3 and
    the row sigma_n + p = -(1 - 2 B (1 + nu_u) / 3) p_net.  The opening is
    then Sneddon's with nu_u and p_net = (p0 - sigma_nn) / (1 - 2B(1+nu_u)/3);
    a system that dropped the pressure row would be 3.4 times too stiff."""
    N, a, angle = 120, 1.0, 0.7
    G, nu, nuu, B = MAT[:4]
    sH, sh, p0 = 3e6, 2e6, 6e6
    xy, xm = crack(N, a, angle)
    A = oracle.assemble(MAT, xy, 1e-4)
    x = oracle.solve(A, oracle.rhs(xy, sigma_H=sH, sigma_h=sh, p0=p0, system="rate"), N, "rate", Dq=0.0)
    snn, tau = _resolved(angle, sH, sh)
    skempton = 1 - 2 * B * (1 + nuu) / 3
    pnet = (p0 - snn) / skempton
    mid = np.abs(xm) <= 0.8 * a
    assert np.max(np.abs(x[N:2 * N][mid] / _profile(nuu, pnet, xm, a)[mid] - 1)) < 0.012
    assert np.max(np.abs(x[:N][mid] / _profile(nuu, tau, xm, a)[mid] - 1)) < 0.012
    p_mid = (A @ x)[2 * N + N // 2]
    assert abs(p_mid / (2 * B * (1 + nuu) / 3 * pnet) - 1) < 1e-4


@pytest.mark.parametrize("system", ["rate", "impermeable"])
def test_two_unknown_systems_satisfy_their_rows(system):
    """With a non-zero prescribed D_q at a finite time, the returned 3N
    vector satisfies the system's own rows of the full product A x:
    sigma_s = b_s and sigma_n (+ p for RATE) = b_n; the prescribed D_q is
    returned unchanged."""
    N = 40
    xy, _ = crack(N, 0.5, 0.4)
    A = oracle.assemble(MAT, xy, 30.0)
    rng = np.random.default_rng(7)
    Dq = 1e-6 * (1 + rng.random(N))
    b = oracle.rhs(xy, sigma_H=3e6, sigma_h=2e6, p_f=5e6, p0=1e6, system=system)
    x = oracle.solve(A, b, N, system, Dq=Dq)
    y = A @ x
    assert np.array_equal(x[2 * N:], Dq)
    row_n = y[N:2 * N] + (y[2 * N:] if system == "rate" else 0.0)
    scale = np.abs(b[:2 * N]).max()
    assert np.abs(y[:N] - b[:N]).max() < 1e-9 * scale
    assert np.abs(row_n - b[N:2 * N]).max() < 1e-9 * scale


def test_rate_march_satisfies_rows_with_history():
    """Two time steps of the RATE system (paper Sec. 4 marching; rows sigma_s
    and sigma_n + p with the fluid source prescribed): at the second step the
    solutions satisfy the system's rows of the complete equations, every time
    element included, i.e. the pressure part of the history term enters the
    sigma_n + p row."""
    N = 30
    xy, _ = crack(N, 0.5, 0.3)
    times = np.array([0.0, 40.0, 90.0])
    b = oracle.rhs(xy, sigma_H=3e6, sigma_h=2e6, p0=1e6, system="rate")
    dq = [np.full(N, 2e-9), np.full(N, 3e-9)]
    sols = oracle.march(MAT, xy, times, [b, b], system="rate", Dq_steps=dq)
    A = lambda t: oracle.assemble(MAT, xy, t)
    y = (A(90.0) - A(50.0)) @ sols[0] + A(50.0) @ sols[1]
    row_n = y[N:2 * N] + y[2 * N:]
    scale = np.abs(b[:2 * N]).max()
    assert np.abs(y[:N] - b[:N]).max() < 1e-9 * scale
    assert np.abs(row_n - b[N:2 * N]).max() < 1e-9 * scale


# ---------------------------------------------------------------------------
# growth step (reading of the propagation check): maximum tangential stress
# ---------------------------------------------------------------------------
def test_kink_special_cases():
    th, keq = oracle.kink([2.0, 0.0, 0.0], [0.0, 1.0, -1.0])
    assert th[0] == 0.0 and keq[0] == 2.0                                  # pure mode I: straight, K_eq = K_I
    assert abs(th[1] - (-2.0 * math.atan(1.0 / math.sqrt(2.0)))) < 1e-14   # pure mode II: -70.53 degrees
    assert abs(th[1] - math.radians(-70.528779)) < 1e-7
    assert abs(keq[1] - 2.0 / math.sqrt(3.0)) < 1e-13                      # K_eq = (2 / sqrt 3) K_II
    assert abs(th[2] + th[1]) < 1e-14 and abs(keq[2] - keq[1]) < 1e-13     # K_II -> -K_II mirrors the kink


def test_kink_maximises_the_hoop_stress():
    """theta_c is the maximiser over (-pi, pi) of the hoop-stress factor
    cos(t/2)(K_I cos^2(t/2) - 1.5 K_II sin t), found by brute force."""
    rng = np.random.default_rng(5)
    t = np.linspace(-math.pi + 1e-6, math.pi - 1e-6, 400001)
    for KI, KII in zip(rng.uniform(0.0, 2.0, 20), rng.uniform(-2.0, 2.0, 20)):
        s = np.cos(t / 2) * (KI * np.cos(t / 2) ** 2 - 1.5 * KII * np.sin(t))
        th, keq = oracle.kink(KI, KII)
        assert abs(t[np.argmax(s)] - th) < 1e-4
        assert abs(s.max() - keq) < 1e-8 * max(1.0, abs(keq))


def test_grow_straight_mode_one():
    """A straight crack along x with pure opening at its tips grows straight
    on at both ends by one element of the tip element's length."""
    xy, _ = crack(10, 1.0)
    N = xy.shape[1]
    D = np.zeros(3 * N)
    D[N:2 * N] = 1e-3                                          # opening only
    tips, ends = np.array([0, N - 1]), np.array([0, 1])
    g, t2, e2, th, keq = oracle.grow(MAT, xy, D, tips, ends, 0.0)
    assert g.shape[1] == N + 2 and list(t2) == [N, N + 1] and list(e2) == [1, 1]
    L = xy[2, 0] - xy[0, 0]
    assert np.allclose(g[:, N], [xy[0, 0], 0.0, xy[0, 0] - L, 0.0], atol=1e-15)
    assert np.allclose(g[:, N + 1], [xy[2, N - 1], 0.0, xy[2, N - 1] + L, 0.0], atol=1e-15)
    # a toughness above K_eq stops the growth
    g, t2, _, _, _ = oracle.grow(MAT, xy, D, tips, ends, 1.01 * keq.max())
    assert g.shape[1] == N and list(t2) == [0, N - 1]


def test_grow_turns_toward_the_largest_compression():
    """A pressurised crack at 45 degrees under sigma_H (x) > sigma_h (y),
    drained: the opening works against the smaller compression, so the
    kinks at both tips turn the fracture toward the x axis (the sign of K_II
    in the tip frame and the direction of the kink, checked by physics)."""
    xy, _ = crack(40, 1.0, angle=math.pi / 4)
    N = xy.shape[1]
    loads = dict(sigma_H=20e6, sigma_h=10e6, p_f=25e6, p0=0.0)
    D = oracle.solve(oracle.assemble(MAT, xy, 1e12), oracle.rhs(xy, system="impermeable", **loads), N,
                     "impermeable")
    g, _, _, th, keq = oracle.grow(MAT, xy, D, [0, N - 1], [0, 1], 0.0)
    assert g.shape[1] == N + 2
    for j in (N, N + 1):
        d = g[2:, j] - g[:2, j]
        assert abs(d[1]) / abs(d[0]) < 0.9              # closer to the x axis than 45 degrees
    assert th[0] * th[1] > 0 and abs(abs(th[0]) - abs(th[1])) < 1e-6   # point-symmetric kinks
