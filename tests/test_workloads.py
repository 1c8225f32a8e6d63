"""The seeded input generators (module `workloads`): every recipe the tests
and the benchmark rely on, checked against its stated definition (no GPU)."""
import numpy as np
import pytest

import workloads as W


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_uniform_nodes_range_seed_and_single_rounding(dtype):
    x = W.nodes_uniform(20000, 3, seed=7, dtype=dtype)
    assert x.shape == (20000, 3) and x.dtype == dtype
    assert np.all(x >= -0.5) and np.all(x < 0.5)
    np.testing.assert_array_equal(x, W.nodes_uniform(20000, 3, seed=7, dtype=dtype))
    assert not np.array_equal(x, W.nodes_uniform(20000, 3, seed=8, dtype=dtype))
    # FP32 nodes are the FP64 draw rounded once
    x64 = W.nodes_uniform(20000, 3, seed=7, dtype=np.float64)
    np.testing.assert_array_equal(W.nodes_uniform(20000, 3, seed=7, dtype=np.float32), x64.astype(np.float32))
    # uniform: each coordinate's mean and variance near 0 and 1/12
    assert np.all(np.abs(x64.mean(axis=0)) < 0.01)
    assert np.all(np.abs(x64.var(axis=0) - 1 / 12) < 0.003)


@pytest.mark.parametrize("m,L", [(4, 64), (8, 512)])
def test_feasible_nodes_lie_in_the_feasible_domain(m, L):
    x = W.nodes_feasible(5000, 2, m, L, seed=3, dtype=np.float32)
    assert np.all(W.feasible_mask(x, m, L))
    a = 0.5 - m / L
    assert np.all(x >= np.float32(-a)) and np.all(x < np.float32(a))
    # a node on the feasible boundary is outside the half-open domain
    edge = np.array([[a, 0.0], [-a, 0.0]])
    np.testing.assert_array_equal(W.feasible_mask(edge, m, L), [False, True])


def test_spoke_directions_fibonacci_sphere():
    S = 64
    u = W.spoke_directions(S)
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(u[:, 2], 1.0 - (2.0 * np.arange(S) + 1.0) / S, rtol=0, atol=1e-15)
    golden = (1.0 + np.sqrt(5.0)) / 2.0
    az = np.arctan2(u[:, 1], u[:, 0])
    step = np.angle(np.exp(1j * (az[1:] - az[:-1])))
    np.testing.assert_allclose(step, np.angle(np.exp(1j * 2.0 * np.pi / golden**2)), rtol=0, atol=1e-12)


def test_spoke_nodes_lie_on_their_spokes():
    S, P, jitter = 32, 256, 1e-4
    x = W.nodes_spokes(n_spokes=S, per_spoke=P, jitter=jitter, seed=1, dtype=np.float64)
    assert x.shape == (S * P, 3)
    assert np.all(x >= -0.5) and np.all(x < 0.5)
    u = W.spoke_directions(S)
    xs = x.reshape(S, P, 3)
    r = np.einsum("spk,sk->sp", xs, u)                    # coordinate along the spoke
    dist = np.linalg.norm(xs - r[..., None] * u[:, None, :], axis=2)
    assert np.all(np.abs(r) <= 0.5 + 6 * jitter)         # radius U[-1/2, 1/2) plus jitter
    assert np.max(dist) < 6 * jitter                       # Gaussian jitter off the line
    assert abs(np.std(dist) - jitter * np.sqrt(2 - np.pi / 2)) < 0.2 * jitter   # 2-d radial spread


def test_chebyshev_nodes_of_example_5_1():
    M, m = 100, 5
    L = 2 * M
    x = W.nodes_chebyshev(M // 2, m, L)
    assert x.shape == (M // 2, 1)
    j = np.arange(1, M // 2 + 1)
    np.testing.assert_allclose(x[:, 0], np.cos((j - 1) * np.pi / (M // 2)) * (0.5 - m / L), rtol=0, atol=1e-16)
    assert x[0, 0] == 0.5 - m / L


def test_triangle_and_fourier_data():
    M = 16
    t = W.triangle(M, 2)
    k = W.frequencies(M)
    assert k[0] == -M // 2 and k[-1] == M // 2 - 1
    np.testing.assert_array_equal(t, np.multiply.outer(1 - np.abs(2 * k / M), 1 - np.abs(2 * k / M)))
    assert np.all(t[0, :] == 0) and t[M // 2, M // 2] == 1.0
    fh = W.fhat_gaussian(M, 2, batch=3, seed=4, dtype=np.complex128)
    assert fh.shape == (3, M, M)
    assert np.all(fh[:, 0, :] == 0) and np.all(fh[:, :, 0] == 0)   # the envelope's zero at k = -M/2
    np.testing.assert_array_equal(fh, W.fhat_gaussian(M, 2, batch=3, seed=4, dtype=np.complex128))
    z = W.fhat_gaussian(64, 2, batch=8, seed=5, envelope=False, dtype=np.complex128)
    assert abs(np.mean(np.abs(z) ** 2) - 2.0) < 0.05          # N(0,1) + i N(0,1)
    g = W.adjoint_input(50000, batch=2, seed=6, dtype=np.complex128)
    assert g.shape == (2, 50000) and abs(np.mean(np.abs(g) ** 2) - 2.0) < 0.05
    v = W.fd_directions(100, 3, seed=7)
    assert v.shape == (100, 3) and abs(np.linalg.norm(v) - 1.0) < 1e-14
