"""nfftbl_grid_noalloc: the equispaced samples of steps 1-2 computed without
any device allocation inside the library.

Callers that cannot allocate device memory through the library (code that
runs under a framework owning the memory pool or its allocator hooks, a host
that only hands out its own buffers) cannot create a plan, since nfftbl_plan
allocates.  This entry point takes only the caller's input and output
buffers and keeps its intermediates in a fixed 16 MiB device array.  Its
result must equal the grid a plan holds after nfftbl_forward, and the
oracle's equispaced samples, on consecutive calls that reuse the same array
(the second call with unchanged parameters reuses the window factors the
first one left there).

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
nb = pytest.importorskip("paper_2502_07155_gb300")

TOL_F32 = 1e-5   # the FP32 parity tolerance of the other GPU tests


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2502_07155_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def call_noalloc(fhat, sigma, m, grid):
    """Call the C-ABI entry point directly (no Python-side allocation)."""
    lib = nb.lib()
    d = fhat.dim() - 1
    Ms = [int(v) for v in fhat.shape[1:]]
    Marr = (ctypes.c_int * 3)(*(Ms + [0] * (3 - d)))
    st = lib.nfftbl_grid_noalloc(d, Marr, float(sigma), int(m), 0.0, int(fhat.shape[0]),
                                 ctypes.c_void_p(fhat.data_ptr()), ctypes.c_void_p(grid.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("d,M,m,batch", [(1, 256, 8, 2), (2, (64, 32), 6, 2), (3, 16, 4, 1),
                                         (1, 60, 5, 3), (2, (48, 40), 4, 2)])
def test_grid_noalloc_matches_forward_twice(d, M, m, batch):
    """Two calls in a row against nfftbl_forward's grid and against the
    oracle (L = 120, 96 x 80 are of the form 2^a 3^b 5^c, not powers of
    two)."""
    plan = nb.Plan(d, M, 2.0, m, precision="f32", batch=batch)
    op = O.make_plan(d, plan.M, 2.0, m, beta=plan.beta)
    x = W.nodes_uniform(500, d, dtype=np.float32)
    plan.set_nodes(torch.from_numpy(x).cuda())
    grid = torch.empty((batch,) + plan.L, dtype=torch.complex64, device="cuda")
    for call, seed in enumerate((11, 12)):      # two calls in a row, same scratch
        fh = torch.from_numpy(W.fhat_gaussian(plan.M, batch=batch, seed=seed, dtype=np.complex64)).cuda()
        plan.forward(fh)
        ref = plan.grid()
        grid.fill_(float("nan"))
        assert call_noalloc(fh, 2.0, m, grid) == 0, nb.lib().nfftbl_plan_error()
        torch.cuda.synchronize()
        got = grid.cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}: output not fully written"
        assert rel_l2(got, ref) < TOL_F32, f"call {call}"
        assert rel_l2(got, O.grid_samples(op, fh.cpu().numpy())) < TOL_F32, f"call {call} vs oracle"
    plan.close()


def test_grid_noalloc_parameters_change_between_calls():
    """A call with other parameters between two equal ones: the window
    factors in the shared array are recomputed when the parameters change
    and match the oracle on every call."""
    outs = []
    for M, m in [((64, 32), 6), ((64, 32), 5), ((64, 32), 6)]:
        fh_np = W.fhat_gaussian(M, batch=1, seed=31, dtype=np.complex64)
        fh = torch.from_numpy(fh_np).cuda()
        grid = torch.full((1, 128, 64), float("nan"), dtype=torch.complex64, device="cuda")
        assert call_noalloc(fh, 2.0, m, grid) == 0, nb.lib().nfftbl_plan_error()
        torch.cuda.synchronize()
        got = grid.cpu().numpy()
        op = O.make_plan(2, M, 2.0, m)
        assert rel_l2(got, O.grid_samples(op, fh_np)) < TOL_F32
        outs.append(got)
    np.testing.assert_array_equal(outs[0], outs[2])


def test_grid_noalloc_rejects_oversize():
    fh = torch.zeros((1, 2048, 2048), dtype=torch.complex64, device="cuda")
    grid = torch.zeros((1, 1), dtype=torch.complex64, device="cuda")
    st = call_noalloc(fh, 2.0, 6, grid)
    assert nb.STATUS[st] == "EINVAL"
    msg = nb.lib().nfftbl_plan_error().decode()
    assert "16 MiB" in msg and "bytes of scratch" in msg


def test_grid_noalloc_rejects_batch_overflow():
    """A batch whose scratch size would overflow 64 bits is rejected before
    anything is launched (the pointers are never read)."""
    lib = nb.lib()
    Marr = (ctypes.c_int * 3)(2048, 2048, 2048)   # B * 2048^2 * 4096 * 8 bytes wraps 64 bits for B = 2^31 - 1
    st = lib.nfftbl_grid_noalloc(3, Marr, 2.0, 6, 0.0, 2**31 - 1, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                 ctypes.c_void_p(0))
    assert nb.STATUS[st] == "EINVAL"
    assert "bytes of scratch" in lib.nfftbl_plan_error().decode()


def test_grid_noalloc_rejects_other_primes():
    """L = 2 * 7 * 8 = 112 is not of the form 2^a 3^b 5^c."""
    fh = torch.zeros((1, 56), dtype=torch.complex64, device="cuda")
    grid = torch.zeros((1, 112), dtype=torch.complex64, device="cuda")
    assert nb.STATUS[call_noalloc(fh, 2.0, 4, grid)] == "EUNSUPPORTED"
