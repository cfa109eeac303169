"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: exactness on polynomials, the
convergence order, the paper's worked HMF example, closed forms (slab field, waterbag dispersion
relation), a library route (numpy FFT) or a trivially exact case (integer shifts = np.roll).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1206_3229_gb300 import inputs as I
from conftest import read_golden


def grid_of(w: I.Workload) -> O.Grid:
    return O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic,
                  w.p_periodic, w.dt, w.eps, w.G)


# ----------------------------------------------------------------------------- Eq. (findif)
@pytest.mark.parametrize("q", range(0, 10))
def test_fd2_exact_for_polynomials_up_to_degree_9(q):
    """The 9-point eighth-order stencil differentiates x^q (q <= 9) exactly (interior nodes)."""
    n, du = 40, 0.05
    x = (np.arange(n) - n // 2) * du
    f = x ** q
    d2 = O.fd2(f, periodic=False, du=du)
    exact = q * (q - 1) * x ** (q - 2) if q >= 2 else np.zeros(n)
    inner = slice(4, n - 4)
    scale = max(1.0, np.abs(f).max() / du ** 2)
    assert np.max(np.abs(d2[inner] - exact[inner])) <= 1e-11 * scale


def test_fd2_not_exact_for_degree_10():
    """Degree 10 is the first failure: sum_m c_m m^10 = -1152 gives error -(1152/10!) * 10! h^8."""
    n, du = 40, 0.05
    x = (np.arange(n) - n // 2) * du
    d2 = O.fd2(x ** 10, periodic=False, du=du)
    exact = 90 * x ** 8
    err = d2[4:n - 4] - exact[4:n - 4]
    # f^(10) = 10!, leading error term = (sum c_m m^10 / 10!) h^8 f^(10) = -1152 h^8 (constant).
    assert np.allclose(err, -1152 * du ** 8, rtol=1e-4, atol=0)


def test_fd2_eighth_order_on_sin():
    """Periodic sin(kx): the error against -k^2 sin(kx) falls by 2^8 per halving of h."""
    errs = []
    for n in (16, 32, 64):
        L = 2 * math.pi
        x = np.arange(n) * (L / n)
        d2 = O.fd2(np.sin(x), periodic=True, du=L / n)
        errs.append(np.max(np.abs(d2 + np.sin(x))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 0.9 * 256 <= r1 <= 1.1 * 256 and 0.9 * 256 <= r2 <= 1.1 * 256, errs


# ----------------------------------------------------------------------------- Eqs. (splinegen, splinecoeffs)
@pytest.mark.parametrize("s", [0.37, -2.81, 5.5, -0.999, 0.0001])
def test_spline_reproduces_cubics(s):
    """FD f'' is exact on cubics and the NR cubic is then the cubic itself: exact reproduction."""
    n, du = 64, 0.1
    x = np.arange(n) * du
    a, b, c, d = 0.3, -1.2, 0.7, 0.25
    f = a + b * x + c * x ** 2 + d * x ** 3
    out = O.spline_shift(f, periodic=False, du=du, s=s)
    foot = x - s * du
    exact = a + b * foot + c * foot ** 2 + d * foot ** 3
    m = int(math.ceil(abs(s))) + 6
    assert np.max(np.abs(out[m:n - m] - exact[m:n - m])) <= 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("s", [3, -2, 17, 0])
def test_integer_shift_is_roll(s):
    """An integer displacement gives beta = 0: the new line is the old one moved by s cells."""
    rng = np.random.default_rng(7)
    f = rng.uniform(-1, 1, 48)
    out = O.spline_shift(f, periodic=True, du=0.3, s=float(s))
    assert np.array_equal(out, np.roll(f, s))


@pytest.mark.parametrize("s", [0.42, -3.7, 9.13])
def test_periodic_equals_tiled_zero_extended(s):
    """Periodic wrap must agree with the zero-extended line of three copies, in the middle copy."""
    rng = np.random.default_rng(11)
    n = 32
    f = rng.uniform(0, 1, n)
    per = O.spline_shift(f, periodic=True, du=0.2, s=s)
    tiled = O.spline_shift(np.tile(f, 3), periodic=False, du=0.2, s=s)
    assert np.max(np.abs(per - tiled[n:2 * n])) <= 1e-14 * f.max()


def test_zero_outside_reading_uses_zero_second_derivative():
    """Reading: on a non-periodic axis f = 0 and f'' = 0 at nodes outside the grid.

    Node 0 of a line holding a single 1 at node 0, moved by s = 0.5: foot at y = -0.5, k = -1,
    alpha = beta = 1/2; f_{-1} = 0 and f''_{-1} = 0, so the value is beta*1 + delta*f''_0 with
    f''_0 = c_0/du^2 and delta = (beta^3 - beta) du^2/6.
    """
    n, du = 16, 0.5
    f = np.zeros(n)
    f[0] = 1.0
    out = O.spline_shift(f, periodic=False, du=du, s=0.5)
    beta = 0.5
    expect = beta + (beta ** 3 - beta) / 6.0 * (-205.0 / 72.0)
    assert abs(out[0] - expect) <= 1e-15


def test_spline_is_fourth_order_on_smooth_data():
    """Interpolation error of a smooth periodic line shrinks ~h^4 (the spline's order)."""
    errs = []
    for n in (32, 64, 128):
        L = 2 * math.pi
        x = np.arange(n) * (L / n)
        f = np.exp(np.sin(x))
        s = 0.3
        out = O.spline_shift(f, periodic=True, du=L / n, s=s)
        errs.append(np.max(np.abs(out - np.exp(np.sin(x - s * L / n)))))
    assert errs[0] / errs[1] > 12 and errs[1] / errs[2] > 12, errs


# ----------------------------------------------------------------------------- Sec. 3 split, free streaming
def test_free_streaming_integer_cells_is_exact():
    """F = 0 and dp*(dt/2)/dx = 1: each step moves row j by exactly 2(j - np/2) cells."""
    nx, npp = 64, 32
    dx = 2 * math.pi / nx
    dp = 1.0 / 32
    dt = 2 * dx / dp
    g = O.Grid("free", nx, npp, -math.pi, math.pi, -(npp // 2) * dp, (npp // 2) * dp, True, False, dt)
    rng = np.random.default_rng(3)
    f0 = rng.uniform(0, 1, (npp, nx))
    f, _ = O.run(g, f0, 3, with_moments=False)
    expect = np.stack([np.roll(f0[j], 3 * 2 * (j - npp // 2)) for j in range(npp)])
    assert np.max(np.abs(f - expect)) <= 1e-14 * f0.max()


def test_free_streaming_smooth_matches_characteristics():
    """Smooth f0(x) g(p) streamed for t: f(x, p, t) = f0(x - p t) g(p), to the spline's accuracy."""
    errs = []
    for n in (64, 128):
        g = O.Grid("free", n, 32, -math.pi, math.pi, -1.0, 1.0, True, False, 0.05)
        x = g.xmin + np.arange(n) * g.dx
        p = g.pmin + np.arange(32) * g.dp
        f0 = np.exp(np.cos(x))[None, :] * np.exp(-p ** 2)[:, None]
        steps = 20
        f, _ = O.run(g, f0, steps, with_moments=False)
        t = steps * g.dt
        exact = np.exp(np.cos(x[None, :] - p[:, None] * t)) * np.exp(-p ** 2)[:, None]
        errs.append(np.max(np.abs(f - exact)))
    assert errs[0] < 1e-3 and errs[0] / errs[1] > 8, errs


def test_p_shift_direction_follows_force():
    """Eq. (step3): f^(II)(p) = f^(I)(p - F dt), so a positive force moves structures to larger p."""
    g = O.Grid("free", 16, 64, -1.0, 1.0, -2.0, 2.0, True, False, 0.1)
    p = g.pmin + np.arange(64) * g.dp
    f = np.repeat(np.exp(-((p - 0.0) / 0.2) ** 2)[:, None], 16, axis=1)
    s_col = np.full(16, 4.0)  # +4 cells
    out = O.advect_p(g, f, s_col)
    assert np.argmax(out[:, 0]) == np.argmax(f[:, 0]) + 4


# ----------------------------------------------------------------------------- HMF (Sec. 2, 4.2)
def test_hmf_paper_waterbag_moments():
    """Paper Sec. 4.2: waterbag of width 2.262 in theta, |p| <= 1.766 -> M = 0.8, e = 0.7."""
    gd = read_golden("hmf_waterbag_paper.txt")
    a, p0, pmax = float(gd["theta_width"]), float(gd["p0"]), float(gd["pmax"])
    res = {}
    for n in (256, 512):
        w = I.Workload("paper_hmf", "hmf", n, n, -math.pi, math.pi, -pmax, pmax, True, False,
                       float(gd["dt"]), 1, init="box", x0=a / 2, p0=p0)
        m = O.moments(grid_of(w), I.initial_state(w))
        res[n] = (math.hypot(m["Mx"], m["My"]), m["energy"])
    for n, (M, e) in res.items():
        tol = 16.0 / n  # O(dtheta, dp) from where the box edges fall on the grid
        assert abs(M - float(gd["M"])) <= tol and abs(e - float(gd["e"])) <= tol, (n, M, e)
    # and the closed forms behind the quoted numbers: M = 2 sin(a/2)/a, e = p0^2/6 + (1 - M^2)/2
    Mc = 2 * math.sin(a / 2) / a
    assert abs(Mc - 0.8) < 1e-3 and abs(p0 ** 2 / 6 + (1 - Mc ** 2) / 2 - 0.7) < 1e-3


def test_hmf_potential_energy_identity():
    """HMF: 1/2 dx^2 sum_ik (1 - cos(x_i - x_k)) rho_i rho_k = (mass^2 - Mx^2 - My^2)/2."""
    w = I.HMF_256.resized(64)
    m = O.moments(grid_of(w), I.initial_state(w))
    assert abs(m["potential"] - 0.5 * (m["mass"] ** 2 - m["Mx"] ** 2 - m["My"] ** 2)) <= 1e-13


def _hmf_homog(U, amp, n=64, npp=128, pmax=2.0, dt=0.05):
    w = I.Workload("hmf_homog", "hmf", n, npp, -math.pi, math.pi, -pmax, pmax, True, False, dt, 0,
                   init="mode", x0=math.pi, p0=math.sqrt(6 * (U - 0.5)), mode_amp=amp)
    return w, grid_of(w)


def test_hmf_homogeneous_stable_waterbag_is_stationary():
    """U = 0.7 > 7/12, no perturbation: M = 0 to rounding, F = 0, so f does not change."""
    w, g = _hmf_homog(0.7, 0.0)
    f0 = I.initial_state(w)
    f, _ = O.run(g, f0, 200, with_moments=False)
    assert np.max(np.abs(f - f0)) <= 1e-13 * f0.max()


def test_hmf_stable_waterbag_mode_does_not_grow():
    """U = 0.7: the waterbag dispersion relation w^2 = 6U - 7/2 > 0 has no growing root."""
    w, g = _hmf_homog(0.7, 1e-6)
    f0 = I.initial_state(w)
    M0 = math.hypot(*(O.moments(g, f0)[k] for k in ("Mx", "My")))
    _, hist = O.run(g, f0, 400)
    M = np.hypot(hist[:, 2], hist[:, 3])
    assert M.max() <= 10 * M0


def test_hmf_unstable_waterbag_growth_rate():
    """U = 0.55 < 7/12: |M| grows at gamma = sqrt(1/2 - p0^2) (p0^2 = 3<p^2> of the discrete f0).

    Linearising Eqs. (vlasoveq, hmfmeanforce, mxmydef) about a homogeneous waterbag gives
    omega^2 = p0^2 - 1/2, i.e. gamma = sqrt(7/2 - 6U) = sqrt(0.2) for the continuous waterbag.
    """
    w, g = _hmf_homog(0.55, 1e-6, n=64, npp=512, pmax=2.0, dt=0.05)
    f0 = I.initial_state(w)
    p = g.pmin + np.arange(g.np) * g.dp
    p2 = np.sum(f0 * (p ** 2)[:, None]) * g.dx * g.dp
    gamma_th = math.sqrt(0.5 - 3 * p2)
    _, hist = O.run(g, f0, 420)
    M = np.hypot(hist[:, 2], hist[:, 3])
    t = hist[:, 0]
    sel = (M > 1e-5) & (M < 1e-3)
    assert sel.sum() > 20
    gamma = np.polyfit(t[sel], np.log(M[sel]), 1)[0]
    assert abs(gamma - gamma_th) <= 0.05 * gamma_th, (gamma, gamma_th)


# ----------------------------------------------------------------------------- ring (Eq. ringpot)
def _ring_grid(n, eps):
    return O.Grid("ring", n, 16, -math.pi, math.pi, -1.0, 1.0, True, False, 0.05, eps=eps)


def test_ring_force_matches_fft_convolution():
    g = _ring_grid(128, 0.01)
    rng = np.random.default_rng(5)
    rho = rng.uniform(0, 1, g.nx)
    F = O.force(g, rho)
    u = np.arange(g.nx) * g.dx
    q = 1 - np.cos(u) + g.eps
    dV = np.sin(u) / (2 * math.sqrt(2) * q ** 1.5)
    Ffft = -g.dx * np.real(np.fft.ifft(np.fft.fft(dV) * np.fft.fft(rho)))
    assert np.max(np.abs(F - Ffft)) <= 1e-12 * np.abs(F).max()


def test_ring_force_antisymmetric_for_symmetric_density():
    g = _ring_grid(128, 0.01)
    th = g.xmin + np.arange(g.nx) * g.dx
    rho = np.exp(np.cos(th))            # symmetric about theta = 0 (node nx/2)
    F = O.force(g, rho)
    i = np.arange(1, g.nx // 2)
    c = g.nx // 2
    assert np.max(np.abs(F[c + i] + F[c - i])) <= 1e-12 * np.abs(F).max()
    assert abs(F[c]) <= 1e-12 * np.abs(F).max()


def test_ring_force_large_eps_tends_to_hmf():
    """Eq. (ringpot) for eps >> 1: V ~ const + (1 - cos)/(2 sqrt2 eps^{3/2}), the HMF potential."""
    th_n = 64
    rho = 1 + 0.3 * np.cos(np.arange(th_n) * 2 * math.pi / th_n - 0.4)
    hmf = O.force(O.Grid("hmf", th_n, 16, -math.pi, math.pi, -1, 1, True, False, 0.1), rho)
    errs = []
    for eps in (1e2, 1e3):
        Fr = O.force(_ring_grid(th_n, eps), rho) * 2 * math.sqrt(2) * eps ** 1.5
        errs.append(np.max(np.abs(Fr - hmf)) / np.abs(hmf).max())
    assert errs[1] < errs[0] and errs[1] < 3e-3, errs


def _f_with_density(g: O.Grid, rho: np.ndarray) -> np.ndarray:
    """A state whose density dp * sum_j f[j, i] is rho (every row the same)."""
    return np.tile(rho / (g.np * g.dp), (g.np, 1))


def _ring_V_integrals(eps: float):
    """Closed forms of int_{-pi}^{pi} V(u) du and int_{-pi}^{pi} V(u) cos u du for Eq. (ringpot).

    With 1 - cos u = 2 sin^2(u/2) and t = u/2 both reduce to complete elliptic integrals of the
    parameter m = -2/eps:  int V = -(2 sqrt2 / sqrt eps) K(m),  and since cos u = 1 - 2 sin^2 t,
    int V cos u = -(2 sqrt2 / sqrt eps) [K(m) - (2/n)(E(m) - K(m))] with n = 2/eps."""
    sp = pytest.importorskip("scipy.special")
    n = 2.0 / eps
    K, E = sp.ellipk(-n), sp.ellipe(-n)
    c = -2.0 * math.sqrt(2.0) / math.sqrt(eps)
    return c * K, c * (K - (2.0 / n) * (E - K))


@pytest.mark.parametrize("eps,n", [(0.01, 256), (0.1, 128), (1.0, 64)])
def test_ring_potential_of_uniform_density_is_an_elliptic_integral(eps, n):
    """U = 1/2 int int V(x - x') rho rho' for rho = m/(2 pi): U = m^2/(4 pi) int V.  V is analytic
    on the circle for eps > 0, so the rectangle rule of the oracle converges geometrically (rate
    exp(-N sqrt(2 eps))) and the closed form holds to rounding."""
    g = _ring_grid(n, eps)
    mass = 0.7
    rho = np.full(n, mass / (2 * math.pi))
    U = O.moments(g, _f_with_density(g, rho))["potential"]
    intV, _ = _ring_V_integrals(eps)
    exact = mass ** 2 / (4 * math.pi) * intV
    assert U < 0
    assert abs(U - exact) <= 1e-12 * abs(exact), (U, exact)


@pytest.mark.parametrize("a", [0.3, 0.9])
def test_ring_potential_of_a_cosine_mode(a):
    """rho = c (1 + a cos theta): by the Fourier series of V, int int V rho rho' =
    c^2 [2 pi int V + pi a^2 int V cos u]; this fixes the k = +-1 harmonic of V as well."""
    eps, n = 0.05, 256
    g = _ring_grid(n, eps)
    c = 0.4
    th = g.xmin + np.arange(n) * g.dx
    rho = c * (1 + a * np.cos(th))
    U = O.moments(g, _f_with_density(g, rho))["potential"]
    intV, intVc = _ring_V_integrals(eps)
    exact = 0.5 * c * c * (2 * math.pi * intV + math.pi * a * a * intVc)
    assert abs(U - exact) <= 1e-12 * abs(exact), (U, exact)


def test_ring_potential_large_eps_tends_to_hmf():
    """For eps >> 1, V = -1/sqrt(2 eps) + (1 - cos u)/(2 sqrt2 eps^{3/2}) + O(eps^{-5/2}), so
    (U_ring + mass^2/(2 sqrt(2 eps))) * 2 sqrt2 eps^{3/2} tends to the HMF potential (the oracle's
    HMF potential is pinned separately)."""
    n = 64
    th = -math.pi + np.arange(n) * 2 * math.pi / n
    rho = 1 + 0.3 * np.cos(th - 0.4) + 0.1 * np.sin(2 * th)
    gh = O.Grid("hmf", n, 16, -math.pi, math.pi, -1, 1, True, False, 0.1)
    mh = O.moments(gh, _f_with_density(gh, rho))
    errs = []
    for eps in (1e2, 1e3, 1e4):
        g = _ring_grid(n, eps)
        m = O.moments(g, _f_with_density(g, rho))
        scaled = (m["potential"] + m["mass"] ** 2 / (2 * math.sqrt(2 * eps))) * 2 * math.sqrt(2) * eps ** 1.5
        errs.append(abs(scaled - mh["potential"]) / abs(mh["potential"]))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-3, errs
    assert 5 < errs[0] / errs[1] < 20, errs      # error O(1/eps)


# ----------------------------------------------------------------------------- sheet (Eq. sheetpot)
def test_sheet_field_of_uniform_slab():
    """rho = 1/2 on |x| < 1: E = -2 pi G x inside, -/+ 2 pi G outside; U = 2 pi G / 3."""
    n = 512
    g = O.Grid("sheet", n, 16, -4.0, 4.0, -1.0, 1.0, False, False, 0.02, G=1.0)
    x = g.xmin + (np.arange(n)) * g.dx
    rho = np.where(np.abs(x) < 1, 0.5, 0.0)
    F = O.force(g, rho)
    inside = np.abs(x) < 0.9
    outside = np.abs(x) > 1.1
    assert np.max(np.abs(F[inside] + 2 * math.pi * x[inside])) <= 4 * math.pi * g.dx
    assert np.max(np.abs(F[outside] + 2 * math.pi * np.sign(x[outside]))) <= 4 * math.pi * g.dx
    errs = []
    for nn in (512, 1024):
        gg = O.Grid("sheet", nn, 16, -4.0, 4.0, -1.0, 1.0, False, False, 0.02, G=1.0)
        xx = gg.xmin + np.arange(nn) * gg.dx
        f = np.zeros((gg.np, nn))
        f[gg.np // 2] = np.where(np.abs(xx) < 1, 0.5, 0.0) / gg.dp
        errs.append(abs(O.moments(gg, f)["potential"] - 2 * math.pi / 3) / (2 * math.pi / 3))
    assert errs[0] <= 3 * g.dx and 1.6 <= errs[0] / errs[1] <= 2.4, errs  # first order in dx


# ----------------------------------------------------------------------------- conservation over runs
def test_config1_mass_and_energy_drift():
    """HMF 256^2, 200 steps: mass is conserved to rounding; energy drift is small (Table 1 scale)."""
    w = I.HMF_256
    g = grid_of(w)
    f0 = I.initial_state(w)
    m0 = O.moments(g, f0)
    _, hist = O.run(g, f0, w.steps)
    assert np.max(np.abs(hist[:, 1] - m0["mass"])) <= 1e-12
    assert np.max(np.abs(hist[:, 6] - m0["energy"])) / abs(m0["energy"]) <= 1e-2


# ----------------------------------------------------------------------------- the input generator
def test_splitmix64_published_vectors():
    gd = read_golden("splitmix64_vectors.txt")
    for key, seed in (("seed0", 0), ("seed1234567", 1234567)):
        want = [int(v, 16) for v in gd[key].split()]
        got = I.splitmix64(seed, np.arange(1, len(want) + 1))
        assert [int(v) for v in got] == want


# ------------------------------------------------------------------------------------- Casimirs
def _gauss(nx, np_, sx, sp, L=12.0, P=12.0):
    g = O.Grid("free", nx, np_, -L / 2, L / 2, -P / 2, P / 2, True, True, 0.1)
    x = g.xmin + (g.xmax - g.xmin) / nx * np.arange(nx)
    p = g.pmin + (g.pmax - g.pmin) / np_ * np.arange(np_)
    f = np.exp(-0.5 * (x[None, :] / sx) ** 2 - 0.5 * (p[:, None] / sp) ** 2) / (2 * math.pi * sx * sp)
    return g, f


def test_entropy_and_l2_of_a_gaussian_match_their_closed_forms():
    """Differential entropy of a 2-D normal density, 1 + ln(2 pi sx sp), and its integral of f^2,
    1 / (4 pi sx sp): the rectangle rule converges spectrally for a resolved, decayed Gaussian."""
    sx, sp = 0.9, 1.3
    g, f = _gauss(192, 256, sx, sp, 24.0, 24.0)
    assert O.entropy(g, f) == pytest.approx(1.0 + math.log(2 * math.pi * sx * sp), abs=1e-10)
    assert O.moments(g, f)["l2"] == pytest.approx(1.0 / (4 * math.pi * sx * sp), abs=1e-10)


def test_entropy_scaling_identity_and_negative_cells():
    """S[lambda f] = lambda S[f] - lambda ln(lambda) M[f]; nodes with f <= 0 add nothing to S."""
    g, f = _gauss(128, 96, 0.7, 1.1)
    M = O.moments(g, f)["mass"]
    for lam in (0.25, 3.0):
        assert O.entropy(g, lam * f) == pytest.approx(lam * O.entropy(g, f) - lam * math.log(lam) * M, rel=1e-12)
    h = f.copy()
    h[::7, ::5] = -1e-3   # spline undershoot
    mask = h > 0
    assert O.entropy(g, h) == pytest.approx(O.entropy(g, np.where(mask, f, 0.0)), rel=1e-14)


def test_entropy_is_conserved_by_integer_free_streaming_and_maximal_for_the_box():
    """An integer-cell x-shift permutes nodes (the method is exact there): every Casimir is conserved.
    Among densities of equal mass on the same support the uniform one has the largest entropy."""
    w = I.HMF_256.resized(64, 64)
    g = grid_of(w)
    rng = np.random.default_rng(3)
    f = rng.uniform(0.1, 1.0, (64, 64))
    s = np.round(rng.uniform(-9, 9, 64))
    assert O.entropy(g, O.advect_x(g, f, s)) == pytest.approx(O.entropy(g, f), rel=1e-13)
    box = np.full_like(f, f.mean())
    assert O.entropy(g, box) > O.entropy(g, f)


# ----------------------------------------------------------------------------- global spline (Eq. tridiagsys)
# The comparison method of Tables 1-2.  Pinned against an independent cubic-spline library (SciPy's
# CubicSpline: periodic end conditions, and natural end conditions on the knots -1..n with zero
# data there), against the closed-form symbol of the cyclic system, and by exact integer shifts.

def _scipy_spline_shift(f, periodic, du, s):
    interpolate = pytest.importorskip("scipy.interpolate")
    n = f.size
    x = np.arange(n) * du
    if periodic:
        cs = interpolate.CubicSpline(np.append(x, n * du), np.append(f, f[0]), bc_type="periodic")
        return cs(np.mod(x - s * du, n * du))
    xe = np.arange(-1, n + 1) * du
    cs = interpolate.CubicSpline(xe, np.concatenate([[0.0], f, [0.0]]), bc_type="natural")
    y = x - s * du
    return np.where((y >= -du) & (y <= n * du), cs(np.clip(y, -du, n * du)), 0.0)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("s", [0.3, -2.7, 5.25, -0.999, 17.5])
def test_gs_shift_matches_library_cubic_spline(periodic, s):
    rng = np.random.default_rng(11)
    n = 96
    du = 0.07
    f = rng.standard_normal(n)
    got = O.spline_shift(f, periodic, du, s, spline="gs")
    ref = _scipy_spline_shift(f, periodic, du, s)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.abs(f).max()


@pytest.mark.parametrize("q", [1, 3, 10, 31])
def test_gs_second_derivative_symbol_on_periodic_modes(q):
    """cos(q x) on n periodic nodes: the cyclic system gives f'' = lambda f with
    lambda = (6/du^2)(2 cos th - 2)/(4 + 2 cos th), th = q du (Fourier symbol of Eq. tridiagsys)."""
    n = 128
    du = 2 * math.pi / n
    x = np.arange(n) * du
    th = q * du
    lam = 6.0 / du**2 * (2 * math.cos(th) - 2) / (4 + 2 * math.cos(th))
    for f in (np.cos(q * x), np.sin(q * x)):
        got = O.gs2(f, True, du)
        assert np.max(np.abs(got - lam * f)) <= 1e-12 * abs(lam)


def test_gs_tends_to_the_exact_second_derivative_and_differs_from_fd():
    """Smooth periodic data: the spline's nodal f'' is second-order accurate (symbol -k^2 (1 + th^2/12)),
    Eq. findif eighth-order: two different f'' whose errors shrink at their own rates."""
    errs_gs, errs_fd = [], []
    for n in (16, 32):
        du = 2 * math.pi / n
        x = np.arange(n) * du
        f = np.sin(x)
        errs_gs.append(np.max(np.abs(O.gs2(f, True, du) + f)))
        errs_fd.append(np.max(np.abs(O.fd2(f, True, du) + f)))
    assert 3.8 < errs_gs[0] / errs_gs[1] < 4.2    # O(du^2)
    assert errs_fd[0] / errs_fd[1] > 200           # O(du^8)


def test_gs_free_streaming_integer_cells_is_exact():
    """Integer shifts reproduce the data exactly for the global spline too (beta = 0)."""
    nx, npp = 64, 32
    dx = 2 * math.pi / nx
    dp = 1.0 / 32
    dt = 2 * dx / dp
    g = O.Grid("free", nx, npp, -math.pi, math.pi, -(npp // 2) * dp, (npp // 2) * dp, True, False, dt,
               spline="gs")
    rng = np.random.default_rng(4)
    f0 = rng.uniform(0, 1, (npp, nx))
    f, _ = O.run(g, f0, 3, with_moments=False)
    expect = np.stack([np.roll(f0[j], 3 * 2 * (j - npp // 2)) for j in range(npp)])
    assert np.max(np.abs(f - expect)) <= 1e-13 * f0.max()


def test_gs_run_conserves_mass_on_the_paper_waterbag():
    """HMF 256^2, 200 steps with the global spline: mass to rounding, energy drift of Table 1 size."""
    w = I.HMF_256
    g = O.Grid(w.model, w.nx, w.np, w.xmin, w.xmax, w.pmin, w.pmax, w.x_periodic, w.p_periodic,
               w.dt, w.eps, w.G, spline="gs")
    f0 = I.initial_state(w)
    m0 = O.moments(g, f0)
    _, hist = O.run(g, f0, w.steps)
    assert np.max(np.abs(hist[:, 1] - m0["mass"])) <= 1e-12
    assert np.max(np.abs(hist[:, 6] - m0["energy"])) / abs(m0["energy"]) <= 1e-2
