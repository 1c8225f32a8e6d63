"""The bounded device wait's timeout path, made to run out on purpose
without faulting the device: the interpolation's tile waits are armed with
nothing to complete them (nfftbl_set_wait_limit with stall_next), so every
wait gives up after the (short) limit, the kernel returns, and the next
nfftbl_sync reports ETIMEOUT.  The plan keeps working afterwards, with the
default limit restored as well as with a short one."""
import time

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


@pytest.mark.parametrize("d,prec", [(2, "f32"), (3, "f32"), (3, "f64")])
def test_wait_runs_out_and_plan_recovers(d, prec):
    M, m = {2: (64, 6), 3: (32, 7)}[d]   # (d = 3 FP32, m = 7: the two-buffer interpolation)
    N = 3000
    rdt, cdt = (np.float64, np.complex128) if prec == "f64" else (np.float32, np.complex64)
    plan = nb.Plan(d, M, 2.0, m, precision=prec)
    x = W.nodes_uniform(N, d, dtype=rdt)
    fh = W.fhat_gaussian(M, d, dtype=cdt)
    plan.set_nodes(to_dev(x))
    ref = O.forward(oracle_plan(plan), fh, x)
    fh_d = to_dev(fh)

    plan.set_wait_limit(1_000_000, stall_next=True)          # 1 ms
    t0 = time.perf_counter()
    plan.forward(fh_d)
    with pytest.raises(nb.NfftblError) as e:
        plan.sync()
    assert e.value.name == "ETIMEOUT"
    assert time.perf_counter() - t0 < 30.0                   # gave up, did not hang

    # the word is cleared and the context is usable: same plan, short limit kept
    f = to_host(plan.forward(fh_d))
    plan.sync()
    assert rel_l2(f, ref) < (1e-12 if prec == "f64" else 1e-5)
    # default limit restored
    plan.set_wait_limit(0)
    f = to_host(plan.forward(fh_d))
    plan.sync()
    assert rel_l2(f, ref) < (1e-12 if prec == "f64" else 1e-5)
    plan.close()


def test_wait_limit_out_of_range_is_einval():
    plan = nb.Plan(2, 64, 2.0, 6, precision="f32")
    with pytest.raises(nb.NfftblError) as e:
        plan.set_wait_limit(-5)
    assert e.value.name == "EINVAL"
    plan.close()
