"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

Element-by-element comparisons at sizes the oracle finishes in seconds but
that span several tiles, several work items per tile and ragged tails;
integer binning results bit for bit.  Tolerances (relative l2 over all
outputs and batch entries): 1e-12 for FP64 plans, 1e-5 for FP32 plans.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import oracle_plan, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nb = pytest.importorskip("paper_2502_07155_gb300")

TOL = {"f64": 1e-12, "f32": 1e-5, "f32c": 1e-5}
RDT = {"f64": np.float64, "f32": np.float32, "f32c": np.float32}
CDT = {"f64": np.complex128, "f32": np.complex64, "f32c": np.complex64}

# (d, M, m, N, nodes_per_item): several tiles, several items per tile, ragged tails
SHAPES = {
    1: (256, 8, 1000, 64),
    2: (64, 6, 3000, 128),
    3: (32, 4, 3000, 256),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_07155_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def make(d, prec, method="shannon", window="sinh", batch=1, m=None, M=None, N=None, table=None, seed=0,
         npi=None, factors=False):
    M0, m0, N0, npi0 = SHAPES[d]
    M = M or M0
    m = m or m0
    N = N if N is not None else N0
    plan = nb.Plan(d, M, 2.0, m, window=window, precision=prec, method=method, batch=batch, table=table,
                   nodes_per_item=npi or npi0, factors=factors)
    x = W.nodes_uniform(N, d, seed=seed, dtype=RDT[prec])
    plan.set_nodes(to_dev(x))
    return plan, x


# --------------------------------------------------------------------------- step 0a

@pytest.mark.parametrize("method", ["shannon", "classic"])
@pytest.mark.parametrize("window", ["sinh", "ckb"])
def test_precorrection_factors(method, window):
    plan = nb.Plan(2, (64, 32), 2.0, 5, window=window, method=method, precision="f64")
    op = oracle_plan(plan)
    ref = O.precorrection_factors(op)
    for t in range(2):
        got = plan.factors(t)
        assert np.max(np.abs(got - ref[t]) / np.abs(ref[t])) < 1e-13


def test_precorrection_factors_table_window():
    tab = O.learned_table(O.mlp_init())
    plan = nb.Plan(1, 128, 2.0, 4, window="table", table=tab, precision="f64")
    op = oracle_plan(plan, table=tab)
    ref = O.precorrection_factors(op)[0]
    assert np.max(np.abs(plan.factors(0) - ref) / np.abs(ref)) < 1e-10


# --------------------------------------------------------------------------- binning

@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_binning_bit_exact(d, prec):
    plan, x = make(d, prec)
    # adversarial extras: duplicates, grid points, both edges of the domain
    L = plan.L[0]
    extra = np.concatenate([x[:50], np.full((7, d), -0.5), (np.arange(7 * d).reshape(7, d) % L - L // 2) / L,
                            np.full((3, d), np.nextafter(RDT[prec](0.5), RDT[prec](0)))]).astype(RDT[prec])
    xs = np.concatenate([x, extra]).astype(RDT[prec])
    plan.set_nodes(to_dev(xs))
    keys, perm, off = plan.binning()
    info = plan.info()
    rk, rp, roff, ok = O.bin_nodes(xs, plan.L, info["tile"][:d])
    assert ok
    np.testing.assert_array_equal(perm.astype(np.int64), rp)
    np.testing.assert_array_equal(keys.astype(np.int64), rk[rp])
    np.testing.assert_array_equal(off.astype(np.int64), roff)


@pytest.mark.parametrize("bad", [0.5, -0.5000001, np.nan, np.inf])
def test_binning_domain_error(bad):
    plan, x = make(2, "f32")
    x = x.copy()
    x[17, 1] = bad
    with pytest.raises(nb.NfftblError) as e:
        plan.set_nodes(to_dev(x))
    assert e.value.name == "EDOMAIN"
    with pytest.raises(nb.NfftblError) as e2:
        plan.forward(to_dev(W.fhat_gaussian(64, 2, dtype=np.complex64)))
    assert e2.value.name == "ESTATE"


# --------------------------------------------------------------------------- forward / adjoint

CASES = [(d, prec, method) for d in (1, 2, 3) for prec in ("f64", "f32", "f32c") for method in ("shannon", "classic")]


@pytest.mark.parametrize("d,prec,method", CASES)
def test_forward_parity(d, prec, method):
    batch = 2
    plan, x = make(d, prec, method=method, batch=batch)
    fh = W.fhat_gaussian(plan.M, batch=batch, dtype=CDT[prec])
    f = to_host(plan.forward(to_dev(fh)))
    plan.sync()
    op = oracle_plan(plan)
    ref = O.forward(op, fh, x)
    assert rel_l2(f, ref) < TOL[prec]
    # the grid after steps 1-2 (Eq. 4.7)
    assert rel_l2(plan.grid(), O.grid_samples(op, fh)) < TOL[prec]


@pytest.mark.parametrize("d,prec,method", CASES)
def test_adjoint_parity(d, prec, method):
    batch = 2
    plan, x = make(d, prec, method=method, batch=batch)
    g = W.adjoint_input(x.shape[0], batch=batch, dtype=CDT[prec])
    fh = to_host(plan.adjoint(to_dev(g)))
    plan.sync()
    ref = O.adjoint(oracle_plan(plan), g, x)
    assert rel_l2(fh, ref) < TOL[prec]


FACTOR_CASES = [(d, prec, method, window) for d in (1, 2, 3) for prec in ("f64", "f32")
                for method, window in (("shannon", "sinh"), ("classic", "sinh"), ("shannon", "table"),
                                       ("shannon", "ckb"))]


@pytest.mark.parametrize("d,prec,method,window", FACTOR_CASES)
def test_stored_factors_match_evaluated(d, prec, method, window):
    """Step 0b in tensor-product form: with the window factors stored by
    set_nodes (factors=True) and evaluated in every transform (default),
    forward and adjoint agree with the oracle, and with each other to the
    rounding of the plan precision."""
    batch = 2
    table = O.learned_table(O.mlp_init()) if window == "table" else None
    outs = {}
    for factors in (True, False):
        plan, x = make(d, prec, method=method, window=window, batch=batch, table=table, factors=factors)
        fh = W.fhat_gaussian(plan.M, batch=batch, dtype=CDT[prec])
        g = W.adjoint_input(x.shape[0], batch=batch, dtype=CDT[prec])
        outs[factors] = (to_host(plan.forward(to_dev(fh))), to_host(plan.adjoint(to_dev(g))))
        plan.sync()
    op = oracle_plan(plan, table=table)
    for factors in (True, False):
        assert rel_l2(outs[factors][0], O.forward(op, fh, x)) < TOL[prec]
        assert rel_l2(outs[factors][1], O.adjoint(op, g, x)) < TOL[prec]
    agree = 1e-14 if prec == "f64" else 1e-6
    assert rel_l2(outs[True][0], outs[False][0]) < agree
    assert rel_l2(outs[True][1], outs[False][1]) < agree


GENERAL_L = [
    (1, 20, 5, "f64", "shannon"),            # L = 40 = 2^3 5
    (1, 20, 5, "f32", "classic"),
    (1, 100, 5, "f64", "shannon"),           # L = 200 = 2^3 5^2
    (2, (20, 24), 4, "f64", "shannon"),      # L = (40, 48 = 2^4 3)
    (2, (20, 24), 4, "f32", "classic"),
    (2, (30, 36), 3, "f32", "shannon"),      # L = (60 = 2^2 3 5, 72 = 2^3 3^2)
    (3, (12, 10, 18), 3, "f64", "shannon"),  # L = (24, 20, 36)
    (3, 12, 3, "f32", "classic"),
]


@pytest.mark.parametrize("d,M,m,prec,method", GENERAL_L)
def test_general_L_parity(d, M, m, prec, method):
    """sigma = 2 with M_t not a power of two: L_t = 2^a 3^b 5^c (mixed-radix
    FFT passes, power-of-two tiles dividing L_t).  Binning bit-exact; grid
    (Eq. 4.7), forward and adjoint against the oracle."""
    batch = 2
    plan = nb.Plan(d, M, 2.0, m, precision=prec, method=method, batch=batch)
    assert any(L & (L - 1) for L in plan.L)
    x = W.nodes_uniform(2000, d, dtype=RDT[prec], seed=4)
    plan.set_nodes(to_dev(x))
    keys, perm, off = plan.binning()
    rk, rp, roff, ok = O.bin_nodes(x, plan.L, plan.info()["tile"][:d])
    assert ok
    np.testing.assert_array_equal(perm.astype(np.int64), rp)
    np.testing.assert_array_equal(off.astype(np.int64), roff)
    op = oracle_plan(plan)
    fh = W.fhat_gaussian(plan.M, batch=batch, dtype=CDT[prec])
    f = to_host(plan.forward(to_dev(fh)))
    assert rel_l2(plan.grid(), O.grid_samples(op, fh)) < TOL[prec]
    assert rel_l2(f, O.forward(op, fh, x)) < TOL[prec]
    g = W.adjoint_input(x.shape[0], batch=batch, dtype=CDT[prec])
    h = to_host(plan.adjoint(to_dev(g)))
    plan.sync()
    assert rel_l2(h, O.adjoint(op, g, x)) < TOL[prec]


@pytest.mark.parametrize("d,prec,method", [(1, "f64", "shannon"), (2, "f64", "shannon"), (2, "f32", "classic"),
                                           (3, "f32", "shannon")])
def test_without_precorrection(d, prec, method):
    """precorrect=False: D = I (Section 5's approximation |I_L| psi_hat ~ 1,
    so 1/(|I_L| psi_hat) ~ 1): factors 1, forward and adjoint against the
    oracle run with the same factors, and close to the precorrected result
    (D_psihat differs from I by the window's ripple in the pass band)."""
    batch = 2
    M0, m0, N0, npi0 = SHAPES[d]
    plan = nb.Plan(d, M0, 2.0, m0, precision=prec, method=method, batch=batch, precorrect=False)
    x = W.nodes_uniform(N0, d, dtype=RDT[prec], seed=6)
    plan.set_nodes(to_dev(x))
    for t in range(d):
        np.testing.assert_array_equal(plan.factors(t), np.ones(plan.M[t]))
    op = oracle_plan(plan)
    fac = [np.ones(plan.M[t]) for t in range(d)]
    fh = W.fhat_gaussian(plan.M, batch=batch, dtype=CDT[prec])
    g = W.adjoint_input(N0, batch=batch, dtype=CDT[prec])
    f = to_host(plan.forward(to_dev(fh)))
    assert rel_l2(f, O.forward(op, fh, x, fac)) < TOL[prec]
    assert rel_l2(to_host(plan.adjoint(to_dev(g))), O.adjoint(op, g, x, fac)) < TOL[prec]
    # for the Shannon method D_psihat differs from I by the pass-band ripple of
    # psi_hat only (the classical window's L phi_hat is not close to 1)
    if method == "shannon":
        assert rel_l2(f, O.forward(op, fh, x)) < 1e-2


def test_general_L_rejects_other_primes():
    with pytest.raises(nb.NfftblError) as e:
        nb.Plan(1, 14, 2.0, 3)        # L = 28 = 2^2 7
    assert e.value.name == "EUNSUPPORTED"


@pytest.mark.parametrize("d", [1, 2, 3])
def test_adjoint_identity_gpu(d):
    """<A fhat, g> = <fhat, A^H g> with both sides from the GPU (FP64)."""
    plan, x = make(d, "f64", batch=1)
    fh = W.fhat_gaussian(plan.M, dtype=np.complex128)
    g = W.adjoint_input(x.shape[0], dtype=np.complex128)
    f = to_host(plan.forward(to_dev(fh)))
    h = to_host(plan.adjoint(to_dev(g)))
    lhs = np.vdot(g, f)
    rhs = np.vdot(h, fh)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("d,prec", [(1, "f64"), (2, "f64"), (3, "f64"), (2, "f32"), (3, "f32")])
def test_interpolation_property_gpu(d, prec):
    """Nodes on grid points return the grid values (Section 3, the sinc taps
    vanish): FP64 to rounding, FP32 to one rounding of phi(0)."""
    plan, _ = make(d, prec)
    L = plan.L[0]
    rng = np.random.default_rng(3)
    idx = rng.integers(0, L, size=(500, d))
    x = ((idx - L // 2) / L).astype(RDT[prec])
    plan.set_nodes(to_dev(x))
    fh = W.fhat_gaussian(plan.M, dtype=CDT[prec])
    f = to_host(plan.forward(to_dev(fh)))[0]
    grid = plan.grid()[0]
    ref = grid[tuple(idx.T)]
    tol = 1e-15 if prec == "f64" else 3e-7
    assert np.max(np.abs(f - ref)) <= tol * np.max(np.abs(grid))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_empty_and_single_node(prec):
    plan, _ = make(2, prec, N=0)
    fh = W.fhat_gaussian(plan.M, dtype=CDT[prec])
    f = plan.forward(to_dev(fh))
    assert f.shape == (1, 0)
    h = to_host(plan.adjoint(to_dev(np.zeros((1, 0), dtype=CDT[prec]))))
    assert np.all(h == 0)
    plan.set_nodes(to_dev(np.array([[0.1234, -0.377]], dtype=RDT[prec])))
    f1 = to_host(plan.forward(to_dev(fh)))
    ref = O.forward(oracle_plan(plan), fh, np.array([[0.1234, -0.377]], dtype=RDT[prec]))
    assert rel_l2(f1, ref) < TOL[prec]
    plan.sync()


@pytest.mark.parametrize("window", ["ckb", "table"])
def test_other_windows_forward(window):
    tab = O.learned_table(O.mlp_init()) if window == "table" else None
    plan = nb.Plan(2, 64, 2.0, 5, window=window, table=tab, precision="f64")
    x = W.nodes_uniform(2000, 2, dtype=np.float64)
    plan.set_nodes(to_dev(x))
    fh = W.fhat_gaussian(64, 2, dtype=np.complex128)
    f = to_host(plan.forward(to_dev(fh)))
    ref = O.forward(oracle_plan(plan, table=tab), fh, x)
    assert rel_l2(f, ref) < (1e-12 if window == "ckb" else 1e-9)


# --------------------------------------------------------------------------- node derivative

@pytest.mark.parametrize("d,prec,method", [(1, "f64", "shannon"), (2, "f64", "shannon"), (3, "f64", "shannon"),
                                           (2, "f64", "classic"), (2, "f32", "shannon"), (3, "f32", "shannon")])
def test_node_grad_parity(d, prec, method):
    batch = 2
    plan, x = make(d, prec, method=method, batch=batch, N=800)
    fh = W.fhat_gaussian(plan.M, batch=batch, dtype=CDT[prec])
    gf = W.adjoint_input(x.shape[0], batch=batch, dtype=CDT[prec])
    gx = to_host(plan.node_grad(to_dev(fh), to_dev(gf)))
    plan.sync()
    ref = O.node_grad(oracle_plan(plan), fh, x, gf)
    assert rel_l2(gx, ref) < TOL[prec]


# --------------------------------------------------------------------------- launch accounting

def test_kernel_launch_count_grows():
    plan, _ = make(2, "f32")
    n0 = plan.kernel_launches()
    plan.forward(to_dev(W.fhat_gaussian(plan.M, dtype=np.complex64)))
    plan.sync()
    assert plan.kernel_launches() == n0 + 3     # two FFT passes + interpolation


# --------------------------------------------------------------------------- adjoint: exactness and dense cells

@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_adjoint_bitwise_deterministic(prec):
    """Fixed-point box accumulation and the ordered flush make the adjoint
    independent of scheduling: repeated calls agree bit for bit."""
    plan, x = make(3, prec, batch=2, N=5000)
    g = to_dev(W.adjoint_input(x.shape[0], batch=2, dtype=CDT[prec]))
    h1 = to_host(plan.adjoint(g))
    h2 = to_host(plan.adjoint(g))
    np.testing.assert_array_equal(h1, h2)


def clustered_nodes(n, d, dtype, seed=7):
    """Most nodes in a few cells near the origin (long same-cell runs, many
    work items per tile), the rest uniform: the radial-spoke centre in
    miniature."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5, 0.5, size=(n, d))
    k = int(0.8 * n)
    x[:k] = rng.normal(0.0, 2e-3, size=(k, d))
    return np.clip(x, -0.5, np.nextafter(0.5, 0)).astype(dtype)


@pytest.mark.parametrize("d,prec,method", [(2, "f32", "shannon"), (3, "f32", "shannon"), (2, "f64", "shannon"),
                                           (3, "f64", "classic"), (1, "f32", "shannon")])
def test_adjoint_dense_cells(d, prec, method):
    M = {1: 256, 2: 64, 3: 32}[d]
    m = {1: 8, 2: 6, 3: 4}[d]
    plan = nb.Plan(d, M, 2.0, m, precision=prec, method=method, batch=1, nodes_per_item=256)
    x = clustered_nodes(6000, d, RDT[prec])
    plan.set_nodes(to_dev(x))
    assert plan.info()["n_work"] > plan.info()["n_tiles"] // 8   # several items in the dense tiles
    g = W.adjoint_input(x.shape[0], dtype=CDT[prec])
    h = to_host(plan.adjoint(to_dev(g)))
    ref = O.adjoint(oracle_plan(plan), g, x)
    assert rel_l2(h, ref) < TOL[prec]
    f = to_host(plan.forward(to_dev(W.fhat_gaussian(plan.M, dtype=CDT[prec]))))
    assert np.all(np.isfinite(f))


# --------------------------------------------------------------------------- truncation m chosen at run time

# Truncations outside the compile-time set {2, ..., 8} (m = 9 .. 12) run the
# kernels that take m as an argument (tap arrays of length 24, loops bounded
# by 2m); the m = 7 cases run the compiled 2m = 14 kernels (odd m).
RUNTIME_M = [
    (1, 256, 12, "f64", "shannon", "sinh", False),
    (1, 256, 9, "f32", "classic", "sinh", False),
    (2, 64, 7, "f32", "shannon", "sinh", False),
    (2, 64, 10, "f64", "classic", "sinh", False),
    (2, 64, 7, "f64", "shannon", "ckb", False),
    (2, 64, 11, "f32", "shannon", "sinh", True),      # stored window factors
    (3, 32, 7, "f32", "shannon", "sinh", False),
    (3, 32, 9, "f32", "classic", "sinh", False),
    (3, 32, 7, "f64", "classic", "sinh", True),
]


@pytest.mark.parametrize("d,M,m,prec,method,window,factors", RUNTIME_M)
def test_runtime_m_parity(d, M, m, prec, method, window, factors):
    """Forward, adjoint (Eq. 4.11 and its transpose) and the node gradient
    against the oracle for truncations without a compiled kernel; batch 2 and
    small work items so that several items share a tile."""
    batch, N = 2, 1500
    plan = nb.Plan(d, M, 2.0, m, window=window, precision=prec, method=method, batch=batch,
                   nodes_per_item=96, factors=factors)
    x = W.nodes_uniform(N, d, dtype=RDT[prec], seed=5)
    plan.set_nodes(to_dev(x))
    op = oracle_plan(plan)
    fh = W.fhat_gaussian(plan.M, batch=batch, dtype=CDT[prec])
    g = W.adjoint_input(N, batch=batch, dtype=CDT[prec])
    f = to_host(plan.forward(to_dev(fh)))
    assert rel_l2(f, O.forward(op, fh, x)) < TOL[prec]
    h = to_host(plan.adjoint(to_dev(g)))
    plan.sync()
    assert rel_l2(h, O.adjoint(op, g, x)) < TOL[prec]
    gx = to_host(plan.node_grad(to_dev(fh), to_dev(g)))
    plan.sync()
    assert rel_l2(gx, O.node_grad(op, fh, x, g)) < TOL[prec]


@pytest.mark.parametrize("prec,m", [("f64", 9), ("f32", 10)])
def test_runtime_m_box_too_large_is_a_plan_error(prec, m):
    """d = 3 with a truncation whose smallest spreading box and node tables
    exceed the shared memory of one block: plan creation fails with
    EUNSUPPORTED instead of launching (FP64 supports m <= 8 at d = 3, FP32
    m <= 9)."""
    with pytest.raises(nb.NfftblError) as e:
        nb.Plan(3, 32, 2.0, m, precision=prec)
    assert e.value.name == "EUNSUPPORTED"


def test_strided_fft_pass_covers_every_line():
    """L = 90 (M = 60, sigma = 1.5) with a batch of 32: the pass over
    dimension 0 has 32 x 90 strided lines, enough for several lines per
    block; the lines per block must divide the inner extent 90 so that no
    column is left out.  Grid, forward and adjoint against the oracle."""
    batch = 32
    plan = nb.Plan(2, 60, 1.5, 4, precision="f64", batch=batch)
    assert tuple(plan.L) == (90, 90)
    x = W.nodes_uniform(500, 2, dtype=np.float64, seed=8)
    plan.set_nodes(to_dev(x))
    op = oracle_plan(plan)
    fh = W.fhat_gaussian(plan.M, batch=batch, dtype=np.complex128)
    f = to_host(plan.forward(to_dev(fh)))
    assert rel_l2(plan.grid(), O.grid_samples(op, fh)) < TOL["f64"]
    assert rel_l2(f, O.forward(op, fh, x)) < TOL["f64"]
    g = W.adjoint_input(500, batch=batch, dtype=np.complex128)
    h = to_host(plan.adjoint(to_dev(g)))
    plan.sync()
    assert rel_l2(h, O.adjoint(op, g, x)) < TOL["f64"]


@pytest.mark.parametrize("d,batch,prec", [(2, 8, "f32"), (2, 7, "f64"), (3, 5, "f32"), (3, 4, "f64")])
def test_batch_larger_than_one_shared_memory_group(d, batch, prec):
    """More batch entries than boxes fit in shared memory at once (6 at
    d = 2, 3 at d = 3 for these shapes): the interpolation stages the tile's
    boxes group by group with a ragged last group, the spreading groups its
    boxes likewise.  Forward, adjoint and node gradient against the oracle."""
    plan, x = make(d, prec, batch=batch)
    op = oracle_plan(plan)
    fh = W.fhat_gaussian(plan.M, batch=batch, dtype=CDT[prec], seed=21)
    g = W.adjoint_input(x.shape[0], batch=batch, dtype=CDT[prec], seed=22)
    assert rel_l2(to_host(plan.forward(to_dev(fh))), O.forward(op, fh, x)) < TOL[prec]
    assert rel_l2(to_host(plan.adjoint(to_dev(g))), O.adjoint(op, g, x)) < TOL[prec]
    gx = to_host(plan.node_grad(to_dev(fh), to_dev(g)))
    plan.sync()
    assert rel_l2(gx, O.node_grad(op, fh, x, g)) < TOL[prec]


# --------------------------------------------------------------------------- polynomial tap weights

@pytest.mark.parametrize("d,m,method,window", [(1, 8, "shannon", "sinh"), (2, 6, "shannon", "sinh"),
                                               (2, 4, "classic", "sinh"), (2, 5, "shannon", "ckb"),
                                               (3, 4, "shannon", "sinh"), (2, 3, "shannon", "table")])
def test_polynomial_weights_match_closed_form(d, m, method, window):
    """FP32 plans made with weights='poly' fit one polynomial per tap; the
    fit is kept only within 3e-7 of the largest weight.  The forward and
    adjoint transforms with the polynomials agree with the closed-form
    weights (the default) and with the oracle at the FP32 tolerance."""
    M = SHAPES[d][0]
    tab = O.learned_table(O.mlp_init()) if window == "table" else None
    x = W.nodes_uniform(2000, d, dtype=np.float32, seed=12)
    fh = W.fhat_gaussian(M, d, batch=1, dtype=np.complex64, seed=13)
    g = W.adjoint_input(2000, batch=1, dtype=np.complex64, seed=14)
    res = {}
    for wts in ("poly", "closed"):
        plan = nb.Plan(d, M, 2.0, m, window=window, precision="f32", method=method, table=tab, weights=wts)
        info = plan.info()
        if wts == "poly":
            assert info["poly_weights"] == 1 and 0 < info["poly_err"] <= 3e-7, info
        else:
            assert info["poly_weights"] == 0
        plan.set_nodes(to_dev(x))
        res[wts] = (to_host(plan.forward(to_dev(fh))), to_host(plan.adjoint(to_dev(g))))
        plan.sync()
        op = oracle_plan(plan, table=tab)
    for k in range(2):
        assert rel_l2(res["poly"][k], res["closed"][k]) < 2e-6
    assert rel_l2(res["poly"][0], O.forward(op, fh, x)) < TOL["f32"]
    assert rel_l2(res["poly"][1], O.adjoint(op, g, x)) < TOL["f32"]
