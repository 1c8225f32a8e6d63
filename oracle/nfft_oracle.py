"""FP64 oracle: Algorithm 4.2, its adjoint, Algorithm 2.1, the NDFT, node
binning and node derivatives, written plainly in numpy/scipy.

TEST INFRASTRUCTURE ONLY -- see the package docstring.  Nothing here is
blocked, fused or reordered beyond what the paper's definitions state; a
library routine (matmul/tensordot, adaptive quadrature, a stable sort)
serves as a step where noted.

Conventions (the paper leaves storage unspecified, Section 1):
  * arrays over I_M and I_L are centred and row-major, dim 0 slowest:
    element k sits at index k + M/2 (resp. l + L/2);
  * a leading batch axis B is always present: fhat (B, M_0..M_{d-1}),
    f and g (B, N);
  * nodes x have shape (N, d).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy import integrate, special

__all__ = [
    "oversampled_length", "default_beta", "Window", "Plan", "make_plan",
    "sinc", "dsinc", "window_transform", "precorrection_factors",
    "fourier_matrix", "step1_precorrect", "mlp_backward", "learned_table_grad", "window_loss", "step2_idft", "step3_short_sums",
    "forward", "grid_samples", "adjoint", "adjoint_short_sums", "adjoint_short_sums_at",
    "adjoint_idft", "ndft", "ndft_adjoint", "node_derivative", "node_grad",
    "bin_nodes", "tap_ranges", "dense_matrices", "mlp_init", "mlp_forward",
    "learned_table", "catmull_rom",
]


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------

def oversampled_length(M: int, sigma: float) -> int:
    """M_sigma = 2 * ceil(ceil(sigma*M) / 2) (Algorithm 2.1 input).

    The product sigma*M is rounded down by 1e-9 before the ceiling so that
    e.g. sigma = 1.1, M = 100 gives 110 and not 112 through FP noise."""
    s = math.ceil(sigma * M - 1e-9)
    return 2 * math.ceil(s / 2)


def default_beta(method: str, m: int, sigma: float) -> float:
    """Window shape parameter (the paper only says "certain beta > 0",
    Remark 3.1).

    Reading: for the regularized Shannon formula, beta = pi*m*lambda/(1+lambda)
    with L = (1+lambda)M, i.e. pi*m*(1 - 1/sigma); for the classical NFFT's
    sinh window, beta = 2*pi*m*(1 - 1/(2 sigma)).  Both come from the
    authors' cited window studies, not from the paper's text; a beta sweep
    in the tests checks that the Shannon value sits near the error minimum."""
    if method == "shannon":
        return math.pi * m * (1.0 - 1.0 / sigma)
    if method == "classic":
        return 2.0 * math.pi * m * (1.0 - 1.0 / (2.0 * sigma))
    raise ValueError(method)


# ---------------------------------------------------------------------------
# Windows (Section 3, Remark 3.1) and the regularized sinc (Eq. 4.2)
# ---------------------------------------------------------------------------

def catmull_rom(values: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Evaluate a table v_i = g(i/n), i = 0..n, on u in [0, 1] by cubic
    Catmull-Rom interpolation.

    Reading for the tabulated window (the paper has none): the ghost values
    are v_{-1} = v_1 (even symmetry about u = 0) and
    v_{n+1} = 2 v_n - v_{n-1} (linear extension past the support edge).
    On the interval [u_i, u_{i+1}] with t = n*u - i the interpolant is
    1/2 [2p1 + (p2 - p0) t + (2p0 - 5p1 + 4p2 - p3) t^2 + (3p1 - p0 - 3p2 + p3) t^3]
    with p0..p3 = v_{i-1}, v_i, v_{i+1}, v_{i+2}."""
    v = np.asarray(values, dtype=np.float64)
    n = v.size - 1
    ext = np.concatenate([[v[1]], v, [2.0 * v[n] - v[n - 1]]])  # ext[j] = v_{j-1}
    u = np.asarray(u, dtype=np.float64)
    s = np.clip(u, 0.0, 1.0) * n
    i = np.minimum(np.floor(s).astype(np.int64), n - 1)
    t = s - i
    p0, p1, p2, p3 = ext[i], ext[i + 1], ext[i + 2], ext[i + 3]
    return 0.5 * (2.0 * p1 + (p2 - p0) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t
                  + (3.0 * p1 - p0 - 3.0 * p2 + p3) * t * t * t)


def _catmull_rom_deriv(values: np.ndarray, u: np.ndarray) -> np.ndarray:
    """d/du of :func:`catmull_rom` (same ghost values)."""
    v = np.asarray(values, dtype=np.float64)
    n = v.size - 1
    ext = np.concatenate([[v[1]], v, [2.0 * v[n] - v[n - 1]]])
    u = np.asarray(u, dtype=np.float64)
    s = np.clip(u, 0.0, 1.0) * n
    i = np.minimum(np.floor(s).astype(np.int64), n - 1)
    t = s - i
    p0, p1, p2, p3 = ext[i], ext[i + 1], ext[i + 2], ext[i + 3]
    dt = 0.5 * ((p2 - p0) + 2.0 * (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t
                + 3.0 * (3.0 * p1 - p0 - 3.0 * p2 + p3) * t * t)
    return dt * n


@dataclass(frozen=True)
class Window:
    """One-dimensional window phi in Phi_{m,L} (Section 3): even, supported
    on [-m/L, m/L], phi(0) = 1, non-increasing on [0, inf).

    kind 'sinh'  : Eq. 3.4, sinh(beta*sqrt(1-(Lx/m)^2)) / sinh(beta);
    kind 'ckb'   : continuous Kaiser-Bessel, (I0(beta*sqrt(.)) - 1)/(I0(beta) - 1);
    kind 'table' : tabulated values on u = |Lx|/m in [0, 1] (learned window),
                   Catmull-Rom interpolated (see :func:`catmull_rom`).
    L is the grid length of this dimension (L = M_sigma for Algorithm 2.1)."""
    kind: str
    L: int
    m: int
    beta: float
    table: tuple | None = None

    def _s(self, x):
        # sqrt(1 - (Lx/m)^2) inside the support, NaN-free outside
        r = self.L * np.asarray(x, dtype=np.float64) / self.m
        inside = np.abs(r) < 1.0
        s = np.sqrt(np.where(inside, (1.0 - r) * (1.0 + r), 0.0))
        return r, s, inside

    def phi(self, x):
        r, s, inside = self._s(x)
        if self.kind == "sinh":
            val = np.sinh(self.beta * s) / np.sinh(self.beta)
        elif self.kind == "ckb":
            val = (special.i0(self.beta * s) - 1.0) / (special.i0(self.beta) - 1.0)
        elif self.kind == "table":
            val = catmull_rom(np.asarray(self.table), np.abs(r))
        else:
            raise ValueError(self.kind)
        return np.where(inside, val, 0.0)

    def dphi(self, x):
        """phi'(x); zero on |Lx| >= m (reading: the derivative's infinite
        limit at the support edge is multiplied by a vanishing sinc, the
        product contributes nothing there)."""
        r, s, inside = self._s(x)
        safe_s = np.where(inside & (s > 0), s, 1.0)
        ds_dx = -(self.L / self.m) * r / safe_s          # d/dx sqrt(1-(Lx/m)^2)
        if self.kind == "sinh":
            val = self.beta * np.cosh(self.beta * s) * ds_dx / np.sinh(self.beta)
        elif self.kind == "ckb":
            val = self.beta * special.i1(self.beta * s) * ds_dx / (special.i0(self.beta) - 1.0)
        elif self.kind == "table":
            val = (_catmull_rom_deriv(np.asarray(self.table), np.abs(r))
                   * np.sign(r) * (self.L / self.m))
        else:
            raise ValueError(self.kind)
        return np.where(inside & (s > 0), val, 0.0)


def sinc(z):
    """sinc(z) = sin(z)/z, sinc(0) = 1 (Section 3)."""
    z = np.asarray(z, dtype=np.float64)
    zs = np.where(z == 0.0, 1.0, z)
    return np.where(z == 0.0, 1.0, np.sin(zs) / zs)


def dsinc(z):
    """sinc'(z) = (cos z - sinc z)/z, with the Taylor series
    -z/3 + z^3/30 - z^5/840 + z^7/45360 for |z| < 0.1, where the closed form
    cancels (relative error ~ eps/z^2) and the series' first dropped term
    z^9/3991680 is below 1e-14 relative."""
    z = np.asarray(z, dtype=np.float64)
    small = np.abs(z) < 0.1
    zs = np.where(small, 1.0, z)
    far = (np.cos(zs) - np.sin(zs) / zs) / zs
    near = -z / 3.0 + z**3 / 30.0 - z**5 / 840.0 + z**7 / 45360.0
    return np.where(small, near, far)


@dataclass(frozen=True)
class Plan:
    """Parameters of one transform.

    method 'shannon': Algorithm 4.2, kernel psi(x) = sinc(L pi x) phi(x)
                      (Eq. 4.2), non-periodic short sums with zero extension
                      outside I_L;
    method 'classic': Algorithm 2.1, kernel = periodized phi_m.
    """
    d: int
    M: tuple
    L: tuple
    m: int
    method: str
    windows: tuple = field(compare=False)

    @property
    def size_L(self) -> int:
        return int(np.prod(self.L))

    def kernel(self, t: int, x):
        """The 1-D short-sum kernel of dimension t evaluated at x."""
        w = self.windows[t]
        if self.method == "shannon":
            return sinc(w.L * np.pi * np.asarray(x, dtype=np.float64)) * w.phi(x)
        return w.phi(x)

    def dkernel(self, t: int, x):
        w = self.windows[t]
        x = np.asarray(x, dtype=np.float64)
        if self.method == "shannon":
            z = w.L * np.pi * x
            return w.L * np.pi * dsinc(z) * w.phi(x) + sinc(z) * w.dphi(x)
        return w.dphi(x)


def make_plan(d: int, M, sigma: float, m: int, method: str = "shannon",
              window: str = "sinh", beta: float | None = None,
              table=None) -> Plan:
    Ms = tuple(int(v) for v in (M if np.ndim(M) else (M,) * d))
    if len(Ms) != d:
        raise ValueError("M must have d entries")
    Ls = tuple(oversampled_length(Mt, sigma) for Mt in Ms)
    if beta is None:
        beta = default_beta(method, m, sigma)
    tab = None if table is None else tuple(float(v) for v in np.asarray(table))
    wins = tuple(Window(window, Lt, m, float(beta), tab) for Lt in Ls)
    return Plan(d, Ms, Ls, m, method, wins)


# ---------------------------------------------------------------------------
# Step 0a: Fourier transform of the kernel (Eq. 3.1 convention)
# ---------------------------------------------------------------------------

def window_transform(plan_or_window, v, t: int = 0, with_sinc: bool | None = None):
    """hat{psi}(v) = int psi(x) e^{-2 pi i v x} dx = 2 int_0^{m/L} psi(x) cos(2 pi v x) dx.

    psi is real and even, so the transform is real.  For the Shannon method
    the kernel is sinc(L pi x) phi(x) (Eq. 4.2, step 0a of Algorithm 4.2); for
    the classical NFFT it is phi alone (step 0a of Algorithm 2.1; the Fourier
    coefficient of the periodized window equals hat{phi}(k) because
    supp phi lies inside [-1/2, 1/2]).

    Rule: scipy's adaptive Gauss-Kronrod (quad_vec, vectorised over v) on the
    panels [n/L, (n+1)/L], n = 0..m-1, whose ends are the sinc's zeros; the
    square-root edge behaviour at m/L is resolved by adaptive bisection."""
    if isinstance(plan_or_window, Plan):
        w = plan_or_window.windows[t]
        if with_sinc is None:
            with_sinc = plan_or_window.method == "shannon"
    else:
        w = plan_or_window
        with_sinc = True if with_sinc is None else with_sinc
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))

    def integrand(x):
        k = w.phi(x) * (sinc(w.L * np.pi * x) if with_sinc else 1.0)
        return 2.0 * k * np.cos(2.0 * np.pi * v * x)

    total = np.zeros_like(v)
    for n in range(w.m):
        val, _err = integrate.quad_vec(integrand, n / w.L, (n + 1) / w.L,
                                       epsabs=1e-17, epsrel=1e-15, norm="max",
                                       limit=20000)
        total += val
    return total


def precorrection_factors(plan: Plan):
    """Per-dimension factors d_t(k) = 1 / (L_t hat{psi}_t(k)), k in I_{M_t}.

    Their tensor product is the diagonal of D_psihat = diag(1/(|I_L| psi_hat(k)))
    of Eq. 4.9 (resp. D of Eq. 2.2 for the classical NFFT), reading the
    multivariate window as a tensor product."""
    out = []
    for t in range(plan.d):
        k = np.arange(-plan.M[t] // 2, plan.M[t] // 2, dtype=np.float64)
        out.append(1.0 / (plan.L[t] * window_transform(plan, k, t)))
    return out


# ---------------------------------------------------------------------------
# Steps 1 and 2: precorrection and the oversampled inverse DFT
# ---------------------------------------------------------------------------

def fourier_matrix(M: int, L: int) -> np.ndarray:
    """F of Eq. 2.3 for one dimension: F[l, k] = exp(2 pi i k l / L),
    rows l in I_L, columns k in I_M (centred).  The exponent's integer k*l is
    reduced mod L exactly before the angle is formed."""
    k = np.arange(-M // 2, M // 2, dtype=np.int64)
    ell = np.arange(-L // 2, L // 2, dtype=np.int64)
    r = np.mod(np.outer(ell, k), L).astype(np.float64)
    ang = 2.0 * np.pi * r / L
    return np.cos(ang) + 1j * np.sin(ang)


def _apply_along(a: np.ndarray, mat: np.ndarray, axis: int) -> np.ndarray:
    """Contract ``mat`` (n_out x n_in) with axis ``axis`` of ``a``."""
    out = np.tensordot(mat, a, axes=([1], [axis]))
    return np.moveaxis(out, 0, axis)


def step1_precorrect(plan: Plan, fhat: np.ndarray, factors=None) -> np.ndarray:
    """Step 1 of Algorithm 4.2: theta_hat(k) = fhat(k) / psi_hat(k) on I_M
    (zero on I_L minus I_M is implicit: step 2 only sums over I_M)."""
    fhat = np.asarray(fhat, dtype=np.complex128)
    factors = precorrection_factors(plan) if factors is None else factors
    out = fhat.copy()
    for t in range(plan.d):
        # 1/psi_hat_t(k) = L_t * d_t(k)
        shape = [1] * (plan.d + 1)
        shape[t + 1] = plan.M[t]
        out = out * (plan.L[t] * factors[t]).reshape(shape)
    return out


def step2_idft(plan: Plan, theta_hat: np.ndarray) -> np.ndarray:
    """Step 2 of Algorithm 4.2: vartheta_l = 1/|I_L| sum_{k in I_M} theta_hat(k) e^{2 pi i k l / L},
    l in I_L, as a direct separable DFT (one dense contraction per axis)."""
    out = np.asarray(theta_hat, dtype=np.complex128)
    for t in range(plan.d):
        out = _apply_along(out, fourier_matrix(plan.M[t], plan.L[t]), t + 1)
    return out / plan.size_L


def grid_samples(plan: Plan, fhat: np.ndarray, factors=None) -> np.ndarray:
    """Steps 1 and 2: the equispaced approximations vartheta_l ~ f(l/L) of Eq. 4.7,
    shape (B, L_0, ..., L_{d-1})."""
    return step2_idft(plan, step1_precorrect(plan, fhat, factors))


# ---------------------------------------------------------------------------
# Step 3: short sums over J_{L,m}(x) (Eq. 4.8)
# ---------------------------------------------------------------------------

def tap_ranges(plan: Plan, x: np.ndarray, t: int):
    """For dimension t: the 2m+1 candidate indices l = ceil(L x - m) + o,
    o = 0..2m, the membership mask of the closed set {l : -m + Lx <= l <= m + Lx}
    (Eq. 4.8; for the classical NFFT, Eq. 2.5 before wrapping), and the
    centred storage index of each member.

    Shannon method: members outside I_L carry no sample (zero extension,
    the first form of the sum before Eq. 4.8).  Classical NFFT: the index
    wraps modulo L (periodized window)."""
    L = plan.L[t]
    m = plan.m
    lx = L * np.asarray(x[:, t], dtype=np.float64)        # exact for L = 2^p
    lo = np.ceil(lx - m).astype(np.int64)
    ell = lo[:, None] + np.arange(2 * m + 1, dtype=np.int64)[None, :]
    member = ell <= (lx + m)[:, None]
    if plan.method == "shannon":
        member &= (ell >= -L // 2) & (ell < L // 2)
        store = ell + L // 2
    else:
        store = np.mod(ell + L // 2, L)
    store = np.where(member, store, 0)
    return ell, member, store


def _tap_weights(plan: Plan, x: np.ndarray, t: int):
    ell, member, store = tap_ranges(plan, x, t)
    L = plan.L[t]
    # x_t - l/L evaluated as (L x_t - l)/L: both terms exact for L = 2^p
    u = (L * np.asarray(x[:, t], dtype=np.float64)[:, None] - ell) / L
    w = np.where(member, plan.kernel(t, u), 0.0)
    dw = np.where(member, plan.dkernel(t, u), 0.0)
    return store, w, dw


def _gather_tensor(grid_b: np.ndarray, stores):
    """grid_b[store_0[:, o0], store_1[:, o1], ...] broadcast to (n, K, ..., K)."""
    d = len(stores)
    idx = []
    for t, s in enumerate(stores):
        shape = [s.shape[0]] + [1] * d
        shape[t + 1] = s.shape[1]
        idx.append(s.reshape(shape))
    return grid_b[tuple(idx)]


def _weight_tensor(ws):
    d = len(ws)
    out = None
    for t, w in enumerate(ws):
        shape = [w.shape[0]] + [1] * d
        shape[t + 1] = w.shape[1]
        wt = w.reshape(shape)
        out = wt if out is None else out * wt
    return out


def _chunks(n: int, plan: Plan):
    step = max(1, int(4_000_000 // (2 * plan.m + 1) ** plan.d))
    for a in range(0, n, step):
        yield a, min(n, a + step)


def step3_short_sums(plan: Plan, grid: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Step 3 of Algorithm 4.2 (or of Algorithm 2.1 for method 'classic'):
    f_j = sum_{l in J_{L,m}(x_j)} vartheta_l psi(x_j - l/L), where
    psi(x) = prod_t psi_t(x_t).  Returns shape (B, N)."""
    grid = np.asarray(grid, dtype=np.complex128)
    x = np.asarray(x, dtype=np.float64)
    B, N = grid.shape[0], x.shape[0]
    f = np.zeros((B, N), dtype=np.complex128)
    for a, b in _chunks(N, plan):
        xs = x[a:b]
        per_dim = [_tap_weights(plan, xs, t) for t in range(plan.d)]
        weights = _weight_tensor([p[1] for p in per_dim])
        axes = tuple(range(1, plan.d + 1))
        for bi in range(B):
            vals = _gather_tensor(grid[bi], [p[0] for p in per_dim])
            f[bi, a:b] = np.sum(vals * weights, axis=axes)
    return f


def forward(plan: Plan, fhat: np.ndarray, x: np.ndarray, factors=None) -> np.ndarray:
    """Algorithm 4.2 (or 2.1): f = Psi F D_psihat fhat (Eq. 4.11), shape (B, N)."""
    return step3_short_sums(plan, grid_samples(plan, fhat, factors), x)


# ---------------------------------------------------------------------------
# Adjoint: D_psihat F^H Psi^T (transpose of Eq. 4.11; not stated in the paper)
# ---------------------------------------------------------------------------

def adjoint_short_sums(plan: Plan, g: np.ndarray, x: np.ndarray) -> np.ndarray:
    """u = Psi^T g: u_l = sum_j g_j psi(x_j - l/L), shape (B, L_0, ..., L_{d-1})."""
    g = np.asarray(g, dtype=np.complex128)
    x = np.asarray(x, dtype=np.float64)
    B, N = g.shape
    size = plan.size_L
    u = np.zeros((B, size), dtype=np.complex128)
    for a, b in _chunks(N, plan):
        xs = x[a:b]
        per_dim = [_tap_weights(plan, xs, t) for t in range(plan.d)]
        weights = _weight_tensor([p[1] for p in per_dim])
        flat = np.zeros(weights.shape, dtype=np.int64)
        stride = 1
        for t in reversed(range(plan.d)):
            s = per_dim[t][0]
            shape = [s.shape[0]] + [1] * plan.d
            shape[t + 1] = s.shape[1]
            flat = flat + s.reshape(shape) * stride
            stride *= plan.L[t]
        flat = flat.reshape(-1)
        for bi in range(B):
            contrib = (g[bi, a:b].reshape((-1,) + (1,) * plan.d) * weights).reshape(-1)
            u[bi] += np.bincount(flat, weights=contrib.real, minlength=size)
            u[bi] += 1j * np.bincount(flat, weights=contrib.imag, minlength=size)
    return u.reshape((B,) + tuple(plan.L))


def adjoint_short_sums_at(plan: Plan, g: np.ndarray, x: np.ndarray, cells) -> np.ndarray:
    """u_l = sum_j g_j psi(x_j - l/L) (Psi^T g, the transpose of the short
    sums of Eq. 4.8) at the listed grid points only, straight from the
    definition: for every listed l (storage indices, shape (n_cells, d)) and
    every node, the product of the d one-dimensional kernels at
    x_{j,t} - l_t/L_t, taken where |L_t x_{j,t} - l_t| <= m in every
    dimension.  For Algorithm 2.1 the index difference is reduced modulo L_t
    to its nearest image (periodized window).  Returns shape (B, n_cells).

    Equal to adjoint_short_sums at those points; it needs only the nodes
    whose taps reach them, so large node sets can be checked on a few cells."""
    g = np.asarray(g, dtype=np.complex128)
    x = np.asarray(x, dtype=np.float64)
    cells = np.asarray(cells, dtype=np.int64).reshape(-1, plan.d)
    out = np.zeros((g.shape[0], cells.shape[0]), dtype=np.complex128)
    for c, cell in enumerate(cells):
        w = np.ones(x.shape[0], dtype=np.float64)
        for t in range(plan.d):
            L = plan.L[t]
            ell = int(cell[t]) - L // 2                   # l_t in I_L
            delta = L * x[:, t] - ell                     # L x - l, exact for L = 2^p
            if plan.method == "classic":
                delta = delta - L * np.round(delta / L)
            inside = np.abs(delta) <= plan.m
            w = w * np.where(inside, plan.kernel(t, delta / L), 0.0)
        out[:, c] = g @ w
    return out


def adjoint_idft(plan: Plan, u: np.ndarray) -> np.ndarray:
    """F^H u: h(k) = sum_{l in I_L} e^{-2 pi i k l / L} u_l, k in I_M (no normalisation)."""
    out = np.asarray(u, dtype=np.complex128)
    for t in range(plan.d):
        out = _apply_along(out, fourier_matrix(plan.M[t], plan.L[t]).conj().T, t + 1)
    return out


def adjoint(plan: Plan, g: np.ndarray, x: np.ndarray, factors=None) -> np.ndarray:
    """hat{h} = D_psihat F^H Psi^T g, shape (B, M_0, ..., M_{d-1}).

    D_psihat is real (psi real and even gives a real psi_hat) and Psi is real,
    so the adjoint of Eq. 4.11 is D_psihat F^H Psi^T."""
    factors = precorrection_factors(plan) if factors is None else factors
    h = adjoint_idft(plan, adjoint_short_sums(plan, g, x))
    for t in range(plan.d):
        shape = [1] * (plan.d + 1)
        shape[t + 1] = plan.M[t]
        h = h * factors[t].reshape(shape)
    return h


# ---------------------------------------------------------------------------
# The trigonometric sums themselves (Eq. 2.1) by brute force
# ---------------------------------------------------------------------------

def ndft(fhat: np.ndarray, x: np.ndarray) -> np.ndarray:
    """f(x_j) = sum_{k in I_M} fhat_k e^{2 pi i k x_j} (Eq. 2.1), shape (B, N).

    Computed as the separable product of 1-D exponentials, dimension by
    dimension (the exponential of a sum is the product of exponentials)."""
    fhat = np.asarray(fhat, dtype=np.complex128)
    x = np.asarray(x, dtype=np.float64)
    B = fhat.shape[0]
    d = x.shape[1]
    Ms = fhat.shape[1:]
    out = np.zeros((B, x.shape[0]), dtype=np.complex128)
    step = max(1, (1 << 22) // max(1, int(np.prod(Ms[:-1]))) // B)

    def expo(xt, Mt):
        k = np.arange(-Mt // 2, Mt // 2, dtype=np.float64)
        return np.exp(2j * np.pi * np.outer(xt, k))                   # (n, M_t)

    for a in range(0, x.shape[0], step):
        xs = x[a:a + step]
        # last dimension first: (B, M_0..M_{d-2}, n) -> (B, n, M_0..M_{d-2})
        cur = np.tensordot(fhat, expo(xs[:, d - 1], Ms[d - 1]), axes=([d], [1]))
        cur = np.moveaxis(cur, -1, 1)
        for t in reversed(range(d - 1)):
            cur = np.einsum("bj...k,jk->bj...", cur, expo(xs[:, t], Ms[t]))
        out[:, a:a + step] = cur
    return out


def ndft_adjoint(g: np.ndarray, x: np.ndarray, M) -> np.ndarray:
    """hat{h}_k = sum_j g_j e^{-2 pi i k x_j}, shape (B, M_0, ..., M_{d-1})."""
    g = np.asarray(g, dtype=np.complex128)
    x = np.asarray(x, dtype=np.float64)
    d = x.shape[1]
    Ms = tuple(M) if np.ndim(M) else (M,) * d
    es = []
    for t in range(d):
        k = np.arange(-Ms[t] // 2, Ms[t] // 2, dtype=np.float64)
        es.append(np.exp(-2j * np.pi * np.outer(x[:, t], k)))
    letters = "pqr"[:d]
    expr = "bj," + ",".join("j" + c for c in letters) + "->b" + letters
    return np.einsum(expr, g, *es)


# ---------------------------------------------------------------------------
# Node derivative (the forward map differentiated with respect to x_j)
# ---------------------------------------------------------------------------

def node_derivative(plan: Plan, fhat: np.ndarray, x: np.ndarray, factors=None) -> np.ndarray:
    """df_j / dx_{j,t} = sum_l vartheta_l psi_t'(x_t - l_t/L_t) prod_{s != t} psi_s(x_s - l_s/L_s),
    shape (B, N, d).  Taps with |L x_t - l_t| >= m contribute nothing."""
    grid = grid_samples(plan, fhat, factors)
    x = np.asarray(x, dtype=np.float64)
    B, N = grid.shape[0], x.shape[0]
    out = np.zeros((B, N, plan.d), dtype=np.complex128)
    for a, b in _chunks(N, plan):
        xs = x[a:b]
        per_dim = [_tap_weights(plan, xs, t) for t in range(plan.d)]
        axes = tuple(range(1, plan.d + 1))
        for t in range(plan.d):
            ws = [p[2] if s == t else p[1] for s, p in enumerate(per_dim)]
            weights = _weight_tensor(ws)
            for bi in range(B):
                vals = _gather_tensor(grid[bi], [p[0] for p in per_dim])
                out[bi, a:b, t] = np.sum(vals * weights, axis=axes)
    return out


def node_grad(plan: Plan, fhat: np.ndarray, x: np.ndarray, grad_f: np.ndarray,
              factors=None) -> np.ndarray:
    """Vector-Jacobian product for real nodes and complex outputs:
    grad_x[j, t] = sum_b Re(conj(grad_f[b, j]) * df_{b,j}/dx_{j,t}), shape (N, d)."""
    der = node_derivative(plan, fhat, x, factors)
    gf = np.asarray(grad_f, dtype=np.complex128)
    return np.sum(np.real(np.conj(gf)[:, :, None] * der), axis=0)


# ---------------------------------------------------------------------------
# Node binning (implementation device; integer results)
# ---------------------------------------------------------------------------

def bin_nodes(x: np.ndarray, L, tile):
    """Cell keys, stable permutation and tile offsets for nodes x.

    For each node and dimension: i_t = floor(L_t * x_t) + L_t/2 in [0, L_t),
    with the product L_t * x_t rounded once in the nodes' own precision
    (float32 nodes: float32 product).  With tile shape T (T_t | L_t):
    c_t = i_t div T_t (tile coordinate), r_t = i_t mod T_t (cell in tile);
    key = lin(c) * prod(T) + lin(r), row-major, dim 0 slowest.  The
    permutation sorts by (key, j) -- stable in j.  tile_off has one entry
    per tile plus one: the start of each tile's run in sorted order.

    Returns (key, perm, tile_off, domain_ok) with domain_ok False if some
    coordinate is outside [-1/2, 1/2) or NaN."""
    x = np.asarray(x)
    N, d = x.shape
    Ls = tuple(L) if np.ndim(L) else (L,) * d
    Ts = tuple(tile) if np.ndim(tile) else (tile,) * d
    ok = bool(np.all((x >= -0.5) & (x < 0.5)))
    dt = x.dtype.type
    lin_c = np.zeros(N, dtype=np.int64)
    lin_r = np.zeros(N, dtype=np.int64)
    for t in range(d):
        prod = (dt(Ls[t]) * x[:, t]).astype(x.dtype)     # one rounding in x's precision
        prod = np.where(np.isfinite(prod), prod, 0)
        i = np.floor(prod).astype(np.int64) + Ls[t] // 2
        i = np.clip(i, 0, Ls[t] - 1)
        c, r = i // Ts[t], i % Ts[t]
        lin_c = lin_c * (Ls[t] // Ts[t]) + c
        lin_r = lin_r * Ts[t] + r
    cells_per_tile = int(np.prod(Ts))
    key = lin_c * cells_per_tile + lin_r
    perm = np.argsort(key, kind="stable")
    n_tiles = int(np.prod([Ls[t] // Ts[t] for t in range(d)]))
    counts = np.bincount(lin_c, minlength=n_tiles)
    tile_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return key, perm.astype(np.int64), tile_off, ok


# ---------------------------------------------------------------------------
# Dense matrices of Eqs. 4.9-4.11 (tiny sizes only)
# ---------------------------------------------------------------------------

def dense_matrices(plan: Plan, x: np.ndarray, factors=None):
    """Explicit Psi (N x |I_L|), F (|I_L| x |I_M|) and D_psihat (diagonal) of
    Eqs. 4.9-4.11 for d = 1..3, built entry by entry from their definitions
    (Psi_{j,l} = psi(x_j - l/L) restricted to |L x_t - l_t| <= m)."""
    factors = precorrection_factors(plan) if factors is None else factors
    x = np.asarray(x, dtype=np.float64)
    grids = np.meshgrid(*[np.arange(-Lt // 2, Lt // 2) for Lt in plan.L], indexing="ij")
    ells = np.stack([g.reshape(-1) for g in grids], axis=1)          # (|I_L|, d)
    Psi = np.ones((x.shape[0], ells.shape[0]))
    for t in range(plan.d):
        Lt = plan.L[t]
        delta = Lt * x[:, t][:, None] - ells[:, t][None, :]
        if plan.method == "classic":
            delta = delta - Lt * np.round(delta / Lt)                 # periodize
        inside = np.abs(delta) <= plan.m
        Psi *= np.where(inside, plan.kernel(t, delta / Lt), 0.0)
    F = np.ones((ells.shape[0], 1), dtype=np.complex128)
    kgrids = np.meshgrid(*[np.arange(-Mt // 2, Mt // 2) for Mt in plan.M], indexing="ij")
    ks = np.stack([g.reshape(-1) for g in kgrids], axis=1)
    F = np.exp(2j * np.pi * np.sum(ells[:, None, :] * ks[None, :, :] / np.array(plan.L), axis=2))
    dvec = np.ones(ks.shape[0])
    for t in range(plan.d):
        dvec = dvec * factors[t][ks[:, t] + plan.M[t] // 2]
    return Psi, F, np.diag(dvec)


# ---------------------------------------------------------------------------
# Learned window: MLP phi_theta and its table (parity unpinned beyond the
# invariants the tests check: evenness, phi(0) = 1, phi(m/L) = 0)
# ---------------------------------------------------------------------------

def mlp_init(hidden: int = 64, seed: int = 4):
    """Parameters of the 1 -> hidden -> hidden -> 1 tanh MLP (float64)."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((hidden, 1)) * 1.0,
        "b1": rng.standard_normal(hidden) * 0.5,
        "W2": rng.standard_normal((hidden, hidden)) / np.sqrt(hidden),
        "b2": np.zeros(hidden),
        "W3": rng.standard_normal((1, hidden)) * 0.01,
        "b3": np.zeros(1),
    }


def mlp_forward(params, s: np.ndarray) -> np.ndarray:
    """g(s) = W3 tanh(W2 tanh(W1 s + b1) + b2) + b3 for scalar inputs s."""
    s = np.asarray(s, dtype=np.float64).reshape(-1, 1)
    h1 = np.tanh(s @ params["W1"].T + params["b1"])
    h2 = np.tanh(h1 @ params["W2"].T + params["b2"])
    return (h2 @ params["W3"].T + params["b3"]).reshape(-1)


def learned_table(params, n: int = 4096) -> np.ndarray:
    """Window table v_i = phi_theta(u_i), u_i = i/n, i = 0..n, with
    phi_theta(u) = (1 - u^2) exp(g(u^2) - g(0)) -- even, phi(0) = 1 and zero
    at the support edge by construction (the class Phi_{m,L}, Section 3;
    monotonicity is checked, not enforced)."""
    u = np.arange(n + 1, dtype=np.float64) / n
    g = mlp_forward(params, u * u)
    g0 = mlp_forward(params, np.zeros(1))[0]
    return (1.0 - u * u) * np.exp(g - g0)


def mlp_backward(params, s: np.ndarray, upstream: np.ndarray):
    """Gradient of sum_i upstream_i * g(s_i) with respect to the MLP
    parameters (plain backpropagation in FP64)."""
    s = np.asarray(s, dtype=np.float64).reshape(-1, 1)
    up = np.asarray(upstream, dtype=np.float64).reshape(-1, 1)
    z1 = s @ params["W1"].T + params["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.tanh(z2)
    grads = {"W3": up.T @ h2, "b3": up.sum(axis=0)}
    d2 = (up @ params["W3"]) * (1.0 - h2 * h2)
    grads["W2"] = d2.T @ h1
    grads["b2"] = d2.sum(axis=0)
    d1 = (d2 @ params["W2"]) * (1.0 - h1 * h1)
    grads["W1"] = d1.T @ s
    grads["b1"] = d1.sum(axis=0)
    return grads


def learned_table_grad(params, dE_dv: np.ndarray, n: int = 4096):
    """Chain rule from a gradient with respect to the table values
    v_i = (1 - u_i^2) exp(g(u_i^2) - g(0)) to the MLP parameters."""
    u = np.arange(n + 1, dtype=np.float64) / n
    v = learned_table(params, n)
    up = np.asarray(dE_dv, dtype=np.float64) * v          # d v_i / d g(u_i^2) = v_i
    grads = mlp_backward(params, u * u, up)
    g0 = mlp_backward(params, np.zeros(1), np.array([-np.sum(up)]))   # d v_i / d g(0) = -v_i
    return {k: grads[k] + g0[k] for k in grads}


def window_loss(plan: Plan, fhat: np.ndarray, x: np.ndarray, y: np.ndarray, factors=None) -> float:
    """E = ||f - y||^2 / ||y||^2 with f the forward transform of ``plan``
    (the objective of the learned window; y is the trigonometric sum)."""
    f = forward(plan, fhat, x, factors)
    y = np.asarray(y, dtype=np.complex128)
    return float(np.sum(np.abs(f - y) ** 2) / np.sum(np.abs(y) ** 2))
