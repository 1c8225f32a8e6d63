"""The d = 3 FP32 spreading on the tensor cores (single-batch plans) against
the oracle's transposed short sums (Eq. 4.11 transposed) and against the
column-owner kernel that batched plans run: every closed-form weight kind,
truncations with one to five M tiles, both accumulator segment lengths
(8 stages with two alternating accumulators at m <= 6, 32 stages with one
accumulator at m >= 7), on clustered nodes whose dense tiles hold work
items of up to 1024 nodes (many stages and segments per item)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import oracle_plan, rel_l2, to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nb = pytest.importorskip("paper_2502_07155_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_07155_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def clustered(n, seed=11, L=64):
    """80 % of the nodes around the centre of one grid cell (cell 4 of each
    dimension's upper half: inside one 8^3 tile, whose items then hold 1024
    nodes each), the rest uniform."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-0.5, 0.5, size=(n, 3))
    k = int(0.8 * n)
    x[:k] = rng.normal(4.5 / L, 2e-3, size=(k, 3))
    return np.clip(x, -0.5, np.nextafter(0.5, 0)).astype(np.float32)


CASES = [(8, "shannon", "sinh"), (7, "classic", "sinh"), (4, "shannon", "table"), (6, "shannon", "sinh"),
         (2, "shannon", "sinh")]


@pytest.mark.parametrize("m,method,window", CASES)
def test_tensor_spreading_parity(m, method, window):
    M, N = 32, 4000
    tab = O.learned_table(O.mlp_init()) if window == "table" else None
    x = clustered(N)
    g = W.adjoint_input(N, dtype=np.complex64)
    g2 = np.concatenate([g, W.adjoint_input(N, dtype=np.complex64, seed=5)], axis=0)

    plan = nb.Plan(3, M, 2.0, m, window=window, table=tab, precision="f32", method=method, batch=1)
    plan.set_nodes(to_dev(x))
    _, _, off = plan.binning()
    assert np.diff(off.astype(np.int64)).max() > 2048         # items of 1024 nodes: many stages and segments
    n0 = plan.kernel_launches()
    h = to_host(plan.adjoint(to_dev(g)))
    plan.sync()
    n_tensor = plan.kernel_launches() - n0

    # the batched plan runs the column-owner kernel (an independent implementation)
    plan2 = nb.Plan(3, M, 2.0, m, window=window, table=tab, precision="f32", method=method, batch=2)
    plan2.set_nodes(to_dev(x))
    n0 = plan2.kernel_launches()
    h2 = to_host(plan2.adjoint(to_dev(g2)))
    plan2.sync()
    assert n_tensor == plan2.kernel_launches() - n0 + 1        # + the input gather into sorted order

    ref = O.adjoint(oracle_plan(plan, table=tab), g, x)
    assert rel_l2(h, ref) < 1e-5
    assert rel_l2(h[0], h2[0]) < 5e-6
    plan.close()
    plan2.close()


def test_tensor_spreading_bitwise_deterministic():
    """A fixed MMA issue order and fixed segment readouts: repeated calls
    agree bit for bit."""
    plan = nb.Plan(3, 32, 2.0, 8, precision="f32", batch=1)
    x = clustered(4000, seed=3)
    plan.set_nodes(to_dev(x))
    g = to_dev(W.adjoint_input(x.shape[0], dtype=np.complex64))
    h1 = to_host(plan.adjoint(g))
    h2 = to_host(plan.adjoint(g))
    np.testing.assert_array_equal(h1, h2)
    plan.close()
