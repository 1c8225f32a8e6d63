"""Host-buffer entry points (nfftbl_forward_host / nfftbl_adjoint_host /
nfftbl_join): the same maps as the device calls (Eq. 4.11 and its
transpose), so the results must equal the device calls' bit for bit, for
page-locked and for pageable host buffers, with several calls in flight
before one sync (the staging buffers are reused, ordered by events)."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nb = pytest.importorskip("paper_2502_07155_gb300")

SHAPE = {1: (256, 8), 2: (64, 6), 3: (32, 4)}
N = 3000


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_07155_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _plan(d, prec, method="shannon", batch=2):
    M, m = SHAPE[d]
    plan = nb.Plan(d, M, 2.0, m, precision=prec, method=method, batch=batch)
    x = W.nodes_uniform(N, d, seed=3, dtype=np.float64 if prec == "f64" else np.float32)
    plan.set_nodes(to_dev(x))
    return plan


@pytest.mark.parametrize("d,prec,method", [(1, "f64", "shannon"), (2, "f32", "shannon"), (2, "f64", "classic"),
                                           (3, "f32", "shannon")])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_calls_equal_device_calls(d, prec, method, pinned):
    plan = _plan(d, prec, method)
    cdt = np.complex128 if prec == "f64" else np.complex64
    steps = 3
    fh = [W.fhat_gaussian(plan.M, batch=2, dtype=cdt, seed=10 + k) for k in range(steps)]
    g = [W.adjoint_input(N, batch=2, dtype=cdt, seed=20 + k) for k in range(steps)]
    ref_f = [to_host(plan.forward(to_dev(a))) for a in fh]
    ref_h = [to_host(plan.adjoint(to_dev(b))) for b in g]
    plan.sync()
    if pinned:
        fh_in = [torch.from_numpy(a).pin_memory() for a in fh]
        g_in = [torch.from_numpy(b).pin_memory() for b in g]
        outs = [(plan.forward_host(fh_in[k]), plan.adjoint_host(g_in[k])) for k in range(steps)]
    else:
        outs = []
        for k in range(steps):
            f_out = np.empty((2, N), dtype=cdt)
            h_out = np.empty((2,) + tuple(plan.M), dtype=cdt)
            plan.forward_host(fh[k], out=f_out)
            plan.adjoint_host(g[k], out=h_out)
            outs.append((f_out, h_out))
    plan.sync()
    for k in range(steps):
        f_out, h_out = (np.asarray(o) for o in outs[k])
        np.testing.assert_array_equal(f_out, ref_f[k])
        np.testing.assert_array_equal(h_out, ref_h[k])


def test_join_orders_the_plan_stream_after_downloads():
    plan = _plan(2, "f32")
    fh = W.fhat_gaussian(plan.M, batch=2, dtype=np.complex64, seed=5)
    ref = to_host(plan.forward(to_dev(fh)))
    plan.sync()
    out = plan.forward_host(torch.from_numpy(fh).pin_memory())
    plan.join()
    ev = torch.cuda.Event()
    ev.record(torch.cuda.current_stream())
    ev.synchronize()
    np.testing.assert_array_equal(out.numpy(), ref)


def test_host_calls_reject_device_tensors_and_bad_shapes():
    plan = _plan(2, "f32")
    fh = W.fhat_gaussian(plan.M, batch=2, dtype=np.complex64)
    with pytest.raises(TypeError):
        plan.forward_host(to_dev(fh))
    with pytest.raises(ValueError):
        plan.forward_host(fh[:1])
    with pytest.raises(TypeError):
        plan.adjoint_host(np.zeros((2, N), dtype=np.complex128))


def test_host_calls_without_nodes_and_with_growing_node_count():
    """N = 0 (nothing to download for the forward, zeros from the adjoint),
    then node sets of growing size: the staging buffers grow with N."""
    plan = nb.Plan(2, 64, 2.0, 6, precision="f32")
    plan.set_nodes(to_dev(np.zeros((0, 2), dtype=np.float32)))
    fh = W.fhat_gaussian(plan.M, dtype=np.complex64)
    f = plan.forward_host(torch.from_numpy(fh).pin_memory())
    h = plan.adjoint_host(torch.zeros((1, 0), dtype=torch.complex64))
    plan.sync()
    assert tuple(f.shape) == (1, 0)
    assert np.all(h.numpy() == 0)
    for n in (100, 5000):
        x = W.nodes_uniform(n, 2, seed=n)
        plan.set_nodes(to_dev(x))
        g = W.adjoint_input(n, dtype=np.complex64)
        ref_f = to_host(plan.forward(to_dev(fh)))
        ref_h = to_host(plan.adjoint(to_dev(g)))
        plan.sync()
        f = plan.forward_host(torch.from_numpy(fh).pin_memory())
        h = plan.adjoint_host(torch.from_numpy(g).pin_memory())
        plan.sync()
        np.testing.assert_array_equal(f.numpy(), ref_f)
        np.testing.assert_array_equal(h.numpy(), ref_h)
