"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, an independent quadrature rule, a library FFT, brute
force on tiny inputs.  The planted-mistake tests at the end show that a
plausible slip in the oracle (a sign, a dropped factor, an index) makes at
least one of these checks fail.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy import special

import oracle as O
import workloads as W


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# --------------------------------------------------------------------------- parameters

def test_oversampled_length_definition():
    # M_sigma = 2 ceil(ceil(sigma M)/2) (Algorithm 2.1), values by hand
    assert O.oversampled_length(256, 2.0) == 512
    assert O.oversampled_length(20, 2.0) == 40
    assert O.oversampled_length(100, 1.1) == 110
    assert O.oversampled_length(100, 1.25) == 126     # ceil(125) = 125 -> 2*ceil(62.5) = 126
    assert O.oversampled_length(101 * 2, 1.5) == 304  # 303 -> 304


# --------------------------------------------------------------------------- windows

@pytest.mark.parametrize("kind", ["sinh", "ckb"])
def test_window_class_phi_mL(kind):
    """Phi_{m,L} (Section 3): even, support [-m/L, m/L], phi(0) = 1, values in
    [0, 1], non-increasing on [0, inf)."""
    L, m = 128, 6
    w = O.Window(kind, L, m, O.default_beta("shannon", m, 2.0))
    x = np.linspace(0, 1.5 * m / L, 2001)
    v = w.phi(x)
    assert v[0] == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_array_equal(w.phi(-x), v)
    assert np.all(v[x >= m / L] == 0.0)
    assert np.all((v >= 0) & (v <= 1))
    assert np.all(np.diff(v) <= 1e-15)
    # derivative: central differences away from the edge
    xs = np.linspace(0.05, 0.95, 7) * m / L
    h = 1e-7 / L
    fd = (w.phi(xs + h) - w.phi(xs - h)) / (2 * h)
    np.testing.assert_allclose(w.dphi(xs), fd, rtol=1e-6, atol=1e-6 * L)


def test_sinc_and_derivative():
    z = np.array([0.0, 1e-9, 1e-3, 0.5, 3.0, -7.25, np.pi])
    np.testing.assert_allclose(O.sinc(z), np.where(z == 0, 1, np.sin(z) / np.where(z == 0, 1, z)),
                               rtol=1e-15, atol=1e-16)
    # derivative vs the full power series sinc'(z) = sum_{n>=1} (-1)^n 2n z^(2n-1)/(2n+1)!
    from math import factorial
    zz = np.array([1e-9, 1e-3, 0.0099, 0.0101, 0.5, 3.0, -3.7])
    ser = np.array([sum((-1) ** n * 2 * n * float(v) ** (2 * n - 1) / factorial(2 * n + 1)
                        for n in range(1, 40)) for v in zz])
    np.testing.assert_allclose(O.dsinc(zz), ser, rtol=1e-12, atol=1e-18)
    assert O.dsinc(np.array([0.0]))[0] == 0.0


# --------------------------------------------------------------------------- step 0a

def _gl_theta_rule(L, m, beta, v, panels=64, order=20):
    """Independent rule: substitute L x = m sin(theta) (smooth integrand,
    Gauss-Legendre on uniform theta panels)."""
    t, wt = np.polynomial.legendre.leggauss(order)
    edges = np.linspace(0.0, np.pi / 2, panels + 1)
    total = np.zeros_like(v, dtype=np.float64)
    for a, b in zip(edges[:-1], edges[1:]):
        th = 0.5 * (b - a) * t + 0.5 * (a + b)
        x = (m / L) * np.sin(th)
        jac = (m / L) * np.cos(th) * 0.5 * (b - a)
        phi = np.sinh(beta * np.cos(th)) / np.sinh(beta)
        ker = O.sinc(L * np.pi * x) * phi
        total += np.sum(2.0 * ker[None, :] * np.cos(2 * np.pi * np.outer(v, x)) * (wt * jac)[None, :], axis=1)
    return total


@pytest.mark.parametrize("m", [3, 6, 9])
def test_psi_hat_vs_independent_rule(m):
    L = 256
    beta = O.default_beta("shannon", m, 2.0)
    w = O.Window("sinh", L, m, beta)
    v = np.arange(-64, 64, 7, dtype=np.float64)
    q = O.window_transform(w, v)
    ref = _gl_theta_rule(L, m, beta, v)
    assert np.max(np.abs(q - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_psi_hat_sine_integral_closed_form():
    """phi == 1 on the support: 2 int_0^{m/L} sinc(L pi x) cos(2 pi v x) dx
    = (Si(pi (L+2v) m/L) + Si(pi (L-2v) m/L)) / (L pi)."""
    L, m = 64, 5
    w = O.Window("table", L, m, 0.0, tuple([1.0] * 4097))
    v = np.array([0.0, 1.0, 7.5, 16.0, 31.0, 40.0])
    q = O.window_transform(w, v, with_sinc=True)
    si = lambda z: special.sici(z)[0]
    ref = (si(np.pi * (L + 2 * v) * m / L) + si(np.pi * (L - 2 * v) * m / L)) / (L * np.pi)
    np.testing.assert_allclose(q, ref, rtol=0, atol=1e-16)


def test_phi_hat_bessel_closed_form():
    """Classical sinh window: int_{-1}^{1} sinh(beta sqrt(1-t^2)) e^{-i w t} dt
    = pi beta I1(sqrt(beta^2 - w^2))/sqrt(beta^2 - w^2) (J1 for |w| > beta)."""
    L, m = 64, 5
    beta = O.default_beta("classic", m, 2.0)
    w = O.Window("sinh", L, m, beta)
    v = np.array([0.0, 3.0, 10.0, 16.0, 40.0, 60.0])
    q = O.window_transform(w, v, with_sinc=False)
    om = 2 * np.pi * v * m / L
    ref = []
    for o in om:
        if abs(o) < beta:
            r = np.sqrt(beta**2 - o**2)
            ref.append(np.pi * beta * special.i1(r) / r)
        else:
            r = np.sqrt(o**2 - beta**2)
            ref.append(np.pi * beta * special.j1(r) / r)
    ref = (m / L) * np.array(ref) / np.sinh(beta)
    assert np.max(np.abs(q - ref)) <= 1e-14 * np.max(np.abs(ref))


@pytest.mark.parametrize("kind", ["sinh", "ckb"])
def test_L_psi_hat_close_to_one(kind):
    """Section 5: |I_L| psi_hat(k) ~ 1 for k in I_M (numerical observation)."""
    p = O.make_plan(1, 256, 2.0, 8, window=kind)
    fac = O.precorrection_factors(p)[0]     # 1/(L psi_hat)
    assert np.max(np.abs(1.0 / fac - 1.0)) < 1e-3


def test_quadrature_refinement_converged():
    p = O.make_plan(1, 128, 2.0, 7)
    w = p.windows[0]
    k = np.arange(-64, 64, dtype=np.float64)
    a = O.window_transform(p, k)
    # the same integral split into twice as many panels (halves of sinc periods)
    from scipy import integrate
    b = np.zeros_like(k)
    for n in range(2 * w.m):
        val, _ = integrate.quad_vec(lambda x: 2 * w.phi(x) * O.sinc(w.L * np.pi * x) * np.cos(2 * np.pi * k * x),
                                    n / (2 * w.L), (n + 1) / (2 * w.L), epsabs=1e-17, epsrel=1e-15, norm="max")
        b += val
    assert np.max(np.abs(a - b)) <= 1e-15 * np.max(np.abs(a))


# --------------------------------------------------------------------------- step 2

def test_idft_vs_bruteforce_and_fft():
    rng = np.random.default_rng(7)
    # tiny 2-D and 3-D: non-separable brute force
    for Ms, Ls in [((4, 6), (8, 12)), ((2, 4, 4), (4, 8, 8))]:
        d = len(Ms)
        p = O.Plan(d, Ms, Ls, 1, "shannon", ())
        th = rng.standard_normal((1,) + Ms) + 1j * rng.standard_normal((1,) + Ms)
        got = O.step2_idft(p, th)[0]
        ref = np.zeros(Ls, dtype=complex)
        for ell in np.ndindex(*Ls):
            lv = np.array(ell) - np.array(Ls) // 2
            s = 0
            for k in np.ndindex(*Ms):
                kv = np.array(k) - np.array(Ms) // 2
                s += th[(0,) + k] * np.exp(2j * np.pi * np.sum(kv * lv / np.array(Ls)))
            ref[ell] = s / np.prod(Ls)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)
    # moderate 2-D: library FFT on the zero-padded array
    Ms, Ls = (32, 16), (64, 32)
    p = O.Plan(2, Ms, Ls, 1, "shannon", ())
    th = rng.standard_normal((1,) + Ms) + 1j * rng.standard_normal((1,) + Ms)
    pad = np.zeros(Ls, dtype=complex)
    pad[(Ls[0] - Ms[0]) // 2:(Ls[0] + Ms[0]) // 2, (Ls[1] - Ms[1]) // 2:(Ls[1] + Ms[1]) // 2] = th[0]
    ref = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(pad)))
    np.testing.assert_allclose(O.step2_idft(p, th)[0], ref, rtol=0, atol=1e-15)


# --------------------------------------------------------------------------- step 3

@pytest.mark.parametrize("d", [1, 2, 3])
def test_interpolation_property(d):
    """R_{phi,m} f (k/L) = f(k/L) (Section 3): nodes on grid points return
    the grid value exactly (the other taps have sinc = 0)."""
    M = {1: 64, 2: 32, 3: 16}[d]
    p = O.make_plan(d, M, 2.0, 4)
    rng = np.random.default_rng(1)
    grid = rng.standard_normal((1,) + p.L) + 1j * rng.standard_normal((1,) + p.L)
    idx = rng.integers(0, p.L[0], size=(50, d))
    x = (idx - p.L[0] // 2) / p.L[0]
    f = O.step3_short_sums(p, grid, x)
    ref = grid[0][tuple(idx.T)]
    np.testing.assert_allclose(f[0], ref, rtol=1e-15, atol=1e-15)


def fejer(M, x):
    """sum_{k in I_M} (1 - |2k/M|) e^{2 pi i k x} = (2/M) sin^2(pi M x/2)/sin^2(pi x)
    (Fejer kernel of order M/2; the k = -M/2 term vanishes)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sin(np.pi * x)
    safe = np.where(np.abs(s) < 1e-300, 1.0, s)
    return np.where(np.abs(s) < 1e-300, M / 2.0, (2.0 / M) * np.sin(np.pi * M * x / 2) ** 2 / safe**2)


def test_ndft_vs_fejer_closed_form():
    M = 64
    x = np.linspace(-0.5, 0.49, 301).reshape(-1, 1)
    f = O.ndft(W.triangle(M, 1)[None].astype(complex), x)[0]
    np.testing.assert_allclose(f, fejer(M, x[:, 0]), rtol=0, atol=1e-12)
    # 2-D: tensor product of Fejer kernels
    x2 = np.random.default_rng(2).uniform(-0.5, 0.5, (200, 2))
    f2 = O.ndft(W.triangle(16, 2)[None].astype(complex), x2)[0]
    np.testing.assert_allclose(f2, fejer(16, x2[:, 0]) * fejer(16, x2[:, 1]), rtol=0, atol=1e-12)


def test_triangle_closed_forms_c1():
    """C1 (d=1, M=256, L=512, m=8): forward on feasible nodes equals the Fejer
    closed form to window-error level, and the gap to (M/2) sinc^2(pi M x/2)
    is the closed-form quadrature gap (2/M) sin^2(pi M x/2)[1/sin^2(pi x) - 1/(pi x)^2]."""
    M, m = 256, 8
    p = O.make_plan(1, M, 2.0, m)
    x = W.nodes_feasible(1000, 1, m, 512, dtype=np.float64)
    f = O.forward(p, W.triangle(M, 1)[None].astype(complex), x)[0]
    xx = x[:, 0]
    fej = fejer(M, xx)
    assert np.max(np.abs(f - fej)) <= 1e-6 * (M / 2)
    gap = (2.0 / M) * np.sin(np.pi * M * xx / 2) ** 2 * (1 / np.sin(np.pi * xx) ** 2 - 1 / (np.pi * xx) ** 2)
    sinc2 = (M / 2) * O.sinc(np.pi * M * xx / 2) ** 2
    np.testing.assert_allclose(fej - sinc2, gap, rtol=1e-9, atol=1e-12)
    assert np.max(np.abs((f - sinc2) - gap)) <= 1e-6 * (M / 2)
    # imaginary part vanishes: real even data with fhat(-M/2) = 0
    assert np.max(np.abs(np.imag(O.forward(p, W.triangle(M, 1)[None].astype(complex), x)))) < 1e-12


@pytest.mark.parametrize("d,method,tol", [(1, "shannon", 1e-6), (2, "shannon", 2e-6),
                                          (1, "classic", 1e-12), (2, "classic", 1e-12)])
def test_ndft_limit(d, method, tol):
    """Eqs. 5.1/5.2: on feasible nodes both methods approximate the
    trigonometric sum; error at m = 8 vs the brute-force NDFT."""
    M = {1: 64, 2: 32}[d]
    m = 8
    p = O.make_plan(d, M, 2.0, m, method=method)
    x = W.nodes_feasible(1500, d, m, 2 * M, dtype=np.float64, seed=11)
    fh = W.fhat_gaussian(M, d, dtype=np.complex128)
    assert rel_l2(O.forward(p, fh, x), O.ndft(fh, x)) < tol


def test_decay_in_m():
    """The Shannon method's error vs the NDFT decreases monotonically in m,
    log-linearly with slope near -beta/m = -pi (1 - 1/sigma) (the paper's
    bounds are referenced, not printed: only the decay is checked)."""
    errs = []
    for m in range(2, 11):
        p = O.make_plan(1, 64, 2.0, m)
        x = W.nodes_feasible(1500, 1, m, 128, dtype=np.float64, seed=3)
        fh = W.fhat_gaussian(64, 1, dtype=np.complex128)
        errs.append(rel_l2(O.forward(p, fh, x), O.ndft(fh, x)))
    errs = np.array(errs)
    assert np.all(np.diff(np.log(errs)) < 0)
    slope = np.polyfit(np.arange(2, 11), np.log(errs), 1)[0]
    assert -2.2 < slope < -1.2, slope


def test_default_beta_near_optimum():
    m = 6
    base = O.default_beta("shannon", m, 2.0)
    x = W.nodes_feasible(1500, 1, m, 128, dtype=np.float64, seed=3)
    fh = W.fhat_gaussian(64, 1, dtype=np.complex128)
    ref = O.ndft(fh, x)
    errs = {}
    for fac in [0.7, 0.85, 1.0, 1.15, 1.3]:
        p = O.make_plan(1, 64, 2.0, m, beta=base * fac)
        errs[fac] = rel_l2(O.forward(p, fh, x), ref)
    assert errs[1.0] <= 3.0 * min(errs.values())


# --------------------------------------------------------------------------- adjoint and matrix form

@pytest.mark.parametrize("d,method", [(1, "shannon"), (2, "shannon"), (3, "shannon"),
                                      (1, "classic"), (2, "classic"), (3, "classic")])
def test_adjoint_identity(d, method):
    """<A fhat, g> = <fhat, A^H g> (Eq. 4.11 and its transpose)."""
    M = {1: 32, 2: 16, 3: 8}[d]
    p = O.make_plan(d, M, 2.0, 3, method=method)
    x = W.nodes_uniform(300, d, dtype=np.float64, seed=5)
    fh = W.fhat_gaussian(M, d, batch=2, dtype=np.complex128)
    g = W.adjoint_input(300, batch=2, dtype=np.complex128)
    fac = O.precorrection_factors(p)
    lhs = np.vdot(g, O.forward(p, fh, x, fac))
    rhs = np.vdot(O.adjoint(p, g, x, fac), fh)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("d,method", [(1, "shannon"), (2, "shannon"), (1, "classic"), (2, "classic")])
def test_dense_matrix_form(d, method):
    """f = Psi F D_psihat fhat (Eq. 4.11) with the matrices built entry by
    entry, and hat{h} = (Psi F D)^H g."""
    M = {1: 8, 2: 4}[d]
    p = O.make_plan(d, M, 2.0, 2, method=method)
    x = W.nodes_uniform(5, d, dtype=np.float64, seed=9)
    fh = W.fhat_gaussian(M, d, dtype=np.complex128)
    g = W.adjoint_input(5, dtype=np.complex128)
    fac = O.precorrection_factors(p)
    Psi, F, D = O.dense_matrices(p, x, fac)
    A = Psi @ F @ D
    np.testing.assert_allclose(O.forward(p, fh, x, fac)[0], A @ fh.reshape(-1), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(O.adjoint(p, g, x, fac).reshape(-1), A.conj().T @ g[0], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("d,method", [(1, "shannon"), (2, "shannon"), (3, "shannon"),
                                      (1, "classic"), (2, "classic"), (3, "classic")])
def test_adjoint_short_sums_at_points(d, method):
    """Psi^T g evaluated straight from its definition at selected grid points
    equals the scattered (bincount) form at those points, including points
    on the grid's edges (zero extension, resp. the periodic wrap of
    Algorithm 2.1) and nodes on both domain edges."""
    M = {1: 32, 2: 16, 3: 8}[d]
    p = O.make_plan(d, M, 2.0, 3, method=method)
    x = W.nodes_uniform(400, d, dtype=np.float64, seed=15)
    x = np.concatenate([x, np.full((2, d), -0.5), np.full((2, d), np.nextafter(0.5, 0.0))])
    g = W.adjoint_input(x.shape[0], batch=2, dtype=np.complex128)
    full = O.adjoint_short_sums(p, g, x).reshape(2, -1)
    rng = np.random.default_rng(3)
    cells = rng.integers(0, p.L[0], size=(40, d))
    cells = np.concatenate([cells, np.zeros((1, d), np.int64), np.full((1, d), p.L[0] - 1)])
    flat = np.ravel_multi_index(tuple(cells.T), p.L)
    np.testing.assert_allclose(O.adjoint_short_sums_at(p, g, x, cells), full[:, flat], rtol=1e-13, atol=1e-14)


def test_ndft_adjoint_is_transpose():
    x = W.nodes_uniform(40, 2, dtype=np.float64)
    fh = W.fhat_gaussian(8, 2, dtype=np.complex128)
    g = W.adjoint_input(40, dtype=np.complex128)
    lhs = np.vdot(g, O.ndft(fh, x))
    rhs = np.vdot(O.ndft_adjoint(g, x, 8), fh)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# --------------------------------------------------------------------------- node derivative

@pytest.mark.parametrize("d,method", [(1, "shannon"), (2, "shannon"), (2, "classic")])
def test_node_derivative_finite_differences(d, method):
    """Central differences with one Richardson step (h, h/2) in FP64."""
    M = {1: 32, 2: 16}[d]
    p = O.make_plan(d, M, 2.0, 4, method=method)
    x = W.nodes_uniform(20, d, dtype=np.float64, seed=13)
    fh = W.fhat_gaussian(M, d, dtype=np.complex128)
    fac = O.precorrection_factors(p)
    der = O.node_derivative(p, fh, x, fac)[0]
    grid = O.grid_samples(p, fh, fac)
    for t in range(d):
        e = np.zeros(d)
        e[t] = 1.0

        def cd(h):
            return (O.step3_short_sums(p, grid, x + h * e) - O.step3_short_sums(p, grid, x - h * e))[0] / (2 * h)
        h = 1e-4 / p.L[0]
        rich = (4 * cd(h / 2) - cd(h)) / 3
        np.testing.assert_allclose(der[:, t], rich, rtol=1e-7, atol=1e-7 * np.abs(der).max())


def test_node_grad_contraction():
    p = O.make_plan(2, 8, 2.0, 2)
    x = W.nodes_uniform(10, 2, dtype=np.float64)
    fh = W.fhat_gaussian(8, 2, batch=3, dtype=np.complex128)
    gf = W.adjoint_input(10, batch=3, dtype=np.complex128)
    der = O.node_derivative(p, fh, x)
    gx = O.node_grad(p, fh, x, gf)
    # directional derivative of the real functional Re<gf, f(x)> along v
    v = W.fd_directions(10, 2)
    h = 1e-6
    fp = O.forward(p, fh, x + h * v)
    fm = O.forward(p, fh, x - h * v)
    dir_fd = np.real(np.vdot(gf, (fp - fm) / (2 * h)))
    assert abs(np.sum(gx * v) - dir_fd) <= 1e-6 * abs(dir_fd) + 1e-9
    assert der.shape == (3, 10, 2)


# --------------------------------------------------------------------------- binning keys

def test_bin_nodes_invariants():
    L, T = (64, 32), (16, 8)
    x = W.nodes_uniform(3000, 2, dtype=np.float32)
    key, perm, off, ok = O.bin_nodes(x, L, T)
    assert ok
    # perm sorts (key, j) lexicographically
    ks = key[perm]
    assert np.all((np.diff(ks) > 0) | ((np.diff(ks) == 0) & (np.diff(perm) > 0)))
    # each node lies in its cell, checked in exact rational arithmetic
    nt = (L[0] // T[0], L[1] // T[1])
    for j in range(0, 3000, 37):
        kk = int(key[j])
        tile, local = divmod(kk, T[0] * T[1])
        c0, c1 = divmod(tile, nt[1])
        r0, r1 = divmod(local, T[1])
        for t, (c, r) in enumerate([(c0, r0), (c1, r1)]):
            i = c * T[t] + r - L[t] // 2
            xv = Fraction(float(x[j, t]))
            assert Fraction(i, L[t]) <= xv < Fraction(i + 1, L[t])
    # tile offsets: counts per tile
    tiles = key // (T[0] * T[1])
    assert off[0] == 0 and off[-1] == 3000
    np.testing.assert_array_equal(np.diff(off), np.bincount(tiles, minlength=nt[0] * nt[1]))
    # domain violations are reported
    bad = x.copy()
    bad[5, 1] = np.float32(0.5)
    assert not O.bin_nodes(bad, L, T)[3]
    bad[5, 1] = np.nan
    assert not O.bin_nodes(bad, L, T)[3]


# --------------------------------------------------------------------------- learned window invariants

def test_learned_table_class_constraints():
    params = O.mlp_init()
    tab = O.learned_table(params)
    assert tab[0] == pytest.approx(1.0, abs=1e-15) and tab[-1] == 0.0
    w = O.Window("table", 64, 4, 0.0, tuple(tab))
    x = np.linspace(-4 / 64, 4 / 64, 101)
    np.testing.assert_allclose(w.phi(x), w.phi(-x), rtol=0, atol=0)
    # Catmull-Rom reproduces quadratics exactly in the interior; a cubic's
    # error is O(h^3) (tangent error h^2 f'''/6 times h)
    u = np.arange(4097) / 4096
    uu = np.linspace(0.01, 0.99, 333)
    quad = 0.3 - 0.7 * u + 1.1 * u**2
    np.testing.assert_allclose(O.catmull_rom(quad, uu), 0.3 - 0.7 * uu + 1.1 * uu**2, rtol=0, atol=1e-14)
    cub = u**3
    err = np.max(np.abs(O.catmull_rom(cub, uu) - uu**3))
    assert 0 < err < (1 / 4096) ** 3


# --------------------------------------------------------------------------- planted mistakes

def _pin_results():
    """A compact battery of the pins above; returns {name: passed}."""
    out = {}
    # NDFT limit on complex data, d=2 with unequal M (catches axis/sign slips)
    p = O.make_plan(2, (32, 16), 2.0, 6)
    x = W.nodes_feasible(200, 2, 6, 32, dtype=np.float64, seed=21)
    fh = W.fhat_gaussian((32, 16), dtype=np.complex128)
    fac = O.precorrection_factors(p)
    out["ndft_limit"] = rel_l2(O.forward(p, fh, x, fac), O.ndft(fh, x)) < 5e-5
    # adjoint identity
    g = W.adjoint_input(200, dtype=np.complex128)
    lhs = np.vdot(g, O.forward(p, fh, x, fac))
    rhs = np.vdot(O.adjoint(p, g, x, fac), fh)
    out["adjoint"] = abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # interpolation property
    p1 = O.make_plan(1, 32, 2.0, 4)
    rng = np.random.default_rng(1)
    grid = rng.standard_normal((1, 64)) + 1j * rng.standard_normal((1, 64))
    idx = rng.integers(0, 64, size=(20, 1))
    out["interp"] = np.allclose(O.step3_short_sums(p1, grid, (idx - 32) / 64)[0], grid[0, idx[:, 0]],
                                rtol=1e-14, atol=1e-14)
    # L psi_hat ~ 1
    p8 = O.make_plan(1, 64, 2.0, 8)
    out["Lpsihat"] = np.max(np.abs(1.0 / O.precorrection_factors(p8)[0] - 1.0)) < 1e-4
    return out


def test_pins_pass_unmodified():
    assert all(_pin_results().values())


def _mutant_fourier_conj(M, L):
    k = np.arange(-M // 2, M // 2, dtype=np.int64)
    ell = np.arange(-L // 2, L // 2, dtype=np.int64)
    r = np.mod(np.outer(ell, k), L).astype(np.float64)
    return np.exp(-2j * np.pi * r / L)                    # planted: wrong exponent sign


def _mutant_step2_no_norm(plan, theta_hat):
    out = np.asarray(theta_hat, dtype=np.complex128)
    for t in range(plan.d):
        out = O.nfft_oracle._apply_along(out, O.fourier_matrix(plan.M[t], plan.L[t]), t + 1)
    return out                                              # planted: dropped 1/|I_L|


def _mutant_fourier_shifted_k(M, L):
    k = np.arange(-M // 2 + 1, M // 2 + 1, dtype=np.int64)  # planted: centred index off by one
    ell = np.arange(-L // 2, L // 2, dtype=np.int64)
    r = np.mod(np.outer(ell, k), L).astype(np.float64)
    return np.exp(2j * np.pi * r / L)


_orig_tap_ranges = O.nfft_oracle.tap_ranges


def _mutant_tap_shift(plan, x, t):
    ell, member, store = _orig_tap_ranges(plan, x, t)
    L = plan.L[t]
    ell = ell + 1                                           # planted: off-by-one tap index
    member = (ell <= (L * x[:, t])[:, None] + plan.m) & (ell >= -L // 2) & (ell < L // 2)
    store = np.where(member, ell + L // 2, 0)
    return ell, member, store


def _mutant_kernel_no_pi(self, t, x):
    w = self.windows[t]
    return O.sinc(w.L * np.asarray(x, dtype=np.float64)) * w.phi(x)   # planted: sinc(Lx) for sinc(L pi x)


_orig_adjoint_idft = O.nfft_oracle.adjoint_idft


def _mutant_adjoint_transpose(plan, u):
    out = np.asarray(u, dtype=np.complex128)
    for t in range(plan.d):
        out = O.nfft_oracle._apply_along(out, O.fourier_matrix(plan.M[t], plan.L[t]).T, t + 1)  # planted: no conj
    return out


_orig_wt = O.nfft_oracle.window_transform


def _mutant_drop_panel(plan_or_window, v, t=0, with_sinc=None):
    full = _orig_wt(plan_or_window, v, t, with_sinc)
    # planted: a dropped term (the first sinc lobe's panel is doubled instead of integrated once)
    w = plan_or_window.windows[t] if isinstance(plan_or_window, O.Plan) else plan_or_window
    from scipy import integrate
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    first, _ = integrate.quad_vec(lambda x: 2 * w.phi(x) * O.sinc(w.L * np.pi * x) * np.cos(2 * np.pi * v * x),
                                  0.0, 1.0 / w.L, norm="max")
    return full + 0.001 * first


@pytest.mark.parametrize("target,mutant", [
    ("fourier_matrix", _mutant_fourier_conj),
    ("step2_idft", _mutant_step2_no_norm),
    ("fourier_matrix", _mutant_fourier_shifted_k),
    ("tap_ranges", _mutant_tap_shift),
    ("adjoint_idft", _mutant_adjoint_transpose),
    ("window_transform", _mutant_drop_panel),
])
def test_planted_mistake_is_caught(monkeypatch, target, mutant):
    monkeypatch.setattr(O.nfft_oracle, target, mutant)
    res = _pin_results()
    assert not all(res.values()), res


def test_planted_kernel_mistake_is_caught(monkeypatch):
    monkeypatch.setattr(O.Plan, "kernel", _mutant_kernel_no_pi)
    res = _pin_results()
    assert not all(res.values()), res


# --------------------------------------------------------------------------- learned-window oracle pieces

def test_mlp_backward_finite_differences():
    params = O.mlp_init()
    s = np.linspace(0, 1, 37) ** 2
    up = np.cos(7 * s) + 0.3
    g = O.mlp_backward(params, s, up)
    rng = np.random.default_rng(0)
    for name in ["W1", "b1", "W2", "b2", "W3", "b3"]:
        d = rng.standard_normal(params[name].shape)
        h = 1e-6
        pp = {k: v.copy() for k, v in params.items()}
        pm = {k: v.copy() for k, v in params.items()}
        pp[name] += h * d
        pm[name] -= h * d
        fd = (np.dot(up, O.mlp_forward(pp, s)) - np.dot(up, O.mlp_forward(pm, s))) / (2 * h)
        assert abs(np.sum(g[name] * d) - fd) <= 1e-7 * max(1.0, abs(fd)), name


def test_learned_table_grad_finite_differences():
    params = O.mlp_init()
    n = 64
    w = np.sin(np.arange(n + 1) * 0.37)
    g = O.learned_table_grad(params, w, n)
    d = np.random.default_rng(1).standard_normal(params["W2"].shape)
    h = 1e-6
    pp = {k: v.copy() for k, v in params.items()}
    pm = {k: v.copy() for k, v in params.items()}
    pp["W2"] += h * d
    pm["W2"] -= h * d
    fd = (np.dot(w, O.learned_table(pp, n)) - np.dot(w, O.learned_table(pm, n))) / (2 * h)
    assert abs(np.sum(g["W2"] * d) - fd) <= 1e-7 * max(1.0, abs(fd))


def test_window_loss_zero_at_target():
    p = O.make_plan(1, 32, 2.0, 3)
    x = W.nodes_feasible(100, 1, 3, 64, dtype=np.float64)
    fh = W.fhat_gaussian(32, 1, dtype=np.complex128)
    y = O.forward(p, fh, x)
    assert O.window_loss(p, fh, x, y) < 1e-28
    assert O.window_loss(p, fh, x, O.ndft(fh, x)) > 0
