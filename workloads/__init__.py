"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module draws random numbers and lays out node geometry only; it holds
none of the transform's arithmetic (no window, no precorrection, no Fourier
sums).  Every array it returns is host memory (numpy).  Floating-point inputs
for single-precision plans are generated in float64, rounded once to float32,
and handed to both sides in that rounded form, so that errors measure the
arithmetic of the transform and not the rounding of its inputs.

Seeds (one stream per role): 0 nodes, 1 Fourier data, 2 adjoint input,
3 finite-difference directions, 4 training data, 5 held-out data.

Workloads (the paper's experiments are all synthetic, Section 5):
  * uniform nodes in [-1/2, 1/2)^d;
  * radial spokes in d=3 (2^13 spokes of 2^10 samples, golden-ratio
    directions, 1e-4 Gaussian jitter) -- density grows like 1/r^2;
  * scaled Chebyshev nodes of Example 5.1 (Eq. 5.6);
  * Fourier data: the triangle 1-|2k/M| (Example 5.1 up to scale) and
    complex N(0,1) samples times the triangle envelope.
"""
from __future__ import annotations

import numpy as np

SEED_NODES = 0
SEED_FHAT = 1
SEED_ADJ = 2
SEED_FD = 3
SEED_TRAIN = 4
SEED_HELDOUT = 5

_HALF_BELOW = {
    np.float32: np.nextafter(np.float32(0.5), np.float32(0.0)),
    np.float64: np.nextafter(0.5, 0.0),
}


def _clamp_half_open(x: np.ndarray, dtype) -> np.ndarray:
    """Cast to ``dtype`` and keep every coordinate inside [-1/2, 1/2)."""
    x = x.astype(dtype)
    hi = _HALF_BELOW[np.dtype(dtype).type]
    np.clip(x, dtype(-0.5), hi, out=x)
    return x


def nodes_uniform(n: int, d: int, seed: int = SEED_NODES, dtype=np.float32) -> np.ndarray:
    """n nodes i.i.d. uniform in [-1/2, 1/2)^d, shape (n, d), row-major."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5, 0.5, size=(n, d))
    return _clamp_half_open(x, dtype)


def nodes_feasible(n: int, d: int, m: int, L: int, seed: int = SEED_NODES,
                   dtype=np.float32) -> np.ndarray:
    """n nodes i.i.d. uniform in [-1/2 + m/L, 1/2 - m/L)^d (the feasible
    domain of the procedure, Section 4)."""
    rng = np.random.default_rng(seed)
    a = 0.5 - m / L
    x = rng.uniform(-a, a, size=(n, d)).astype(dtype)
    x = np.clip(x, dtype(-a), np.nextafter(dtype(a), dtype(0)))
    return x


def spoke_directions(n_spokes: int) -> np.ndarray:
    """Unit vectors on a Fibonacci sphere: z_s = 1 - (2s+1)/S, azimuth
    advancing by the golden angle 2*pi/phi^2 per spoke."""
    s = np.arange(n_spokes, dtype=np.float64)
    z = 1.0 - (2.0 * s + 1.0) / n_spokes
    golden = (1.0 + np.sqrt(5.0)) / 2.0
    az = s * (2.0 * np.pi / golden**2)
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([r * np.cos(az), r * np.sin(az), z], axis=1)


def nodes_spokes(n_spokes: int = 1 << 13, per_spoke: int = 1 << 10,
                 jitter: float = 1e-4, seed: int = SEED_NODES,
                 dtype=np.float32) -> np.ndarray:
    """Radial-spoke nodes in d=3, shape (n_spokes*per_spoke, 3).

    Radius r ~ U[-1/2, 1/2) i.i.d. per sample, x = r*u_s + jitter*N(0, I),
    clamped to [-1/2, 1/2).  Nodes are ordered spoke by spoke."""
    rng = np.random.default_rng(seed)
    u = spoke_directions(n_spokes)
    r = rng.uniform(-0.5, 0.5, size=(n_spokes, per_spoke, 1))
    x = r * u[:, None, :] + jitter * rng.standard_normal((n_spokes, per_spoke, 3))
    return _clamp_half_open(x.reshape(-1, 3), dtype)


def nodes_chebyshev(n: int, m: int, L: int, dtype=np.float64) -> np.ndarray:
    """Scaled Chebyshev nodes of Example 5.1: cos((j-1)pi/n) * (1/2 - m/L),
    j = 1..n, shape (n, 1).  The first node equals 1/2 - m/L; it is kept
    (its only tap beyond the grid carries a zero window value)."""
    j = np.arange(n, dtype=np.float64)
    x = np.cos(j * np.pi / n) * (0.5 - m / L)
    return x.astype(dtype).reshape(n, 1)


def frequencies(M: int) -> np.ndarray:
    """The index set I_M = [-M/2, M/2) in centred order."""
    return np.arange(-M // 2, M // 2)


def triangle(M, d: int | None = None) -> np.ndarray:
    """Real triangle data prod_t (1 - |2 k_t / M_t|), k in I_M, centred
    row-major (dim 0 slowest).  M is an int (with d) or a tuple."""
    Ms = (M,) * d if d is not None else tuple(M)
    out = np.ones((), dtype=np.float64)
    for Mt in Ms:
        k = frequencies(Mt).astype(np.float64)
        out = np.multiply.outer(out, 1.0 - np.abs(2.0 * k / Mt))
    return out


def fhat_gaussian(M, d: int | None = None, batch: int = 1, seed: int = SEED_FHAT,
                  envelope: bool = True, dtype=np.complex64) -> np.ndarray:
    """Complex data (N(0,1) + i N(0,1)) times the triangle envelope (or no
    envelope), shape (batch, M_0, ..., M_{d-1})."""
    Ms = (M,) * d if d is not None else tuple(M)
    rng = np.random.default_rng(seed)
    shape = (batch,) + Ms
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if envelope:
        z = z * triangle(Ms)[None]
    return z.astype(dtype)


def adjoint_input(n: int, batch: int = 1, seed: int = SEED_ADJ,
                  dtype=np.complex64) -> np.ndarray:
    """Complex N(0,1) values at the nodes, shape (batch, n)."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((batch, n)) + 1j * rng.standard_normal((batch, n))
    return z.astype(dtype)


def fd_directions(n: int, d: int, seed: int = SEED_FD) -> np.ndarray:
    """Unit-norm random directions for directional finite differences."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, d))
    return v / np.linalg.norm(v)


def feasible_mask(x: np.ndarray, m: int, L) -> np.ndarray:
    """Nodes inside [-1/2 + m/L, 1/2 - m/L)^d (per dimension L_t)."""
    Ls = np.broadcast_to(np.asarray(L, dtype=np.float64), (x.shape[1],))
    a = 0.5 - m / Ls
    return np.all((x >= -a) & (x < a), axis=1)
