"""Helpers shared by the GPU parity tests: oracle plans mirroring a GPU plan,
host/device conversion and error norms."""
import numpy as np

import oracle as O


def rel_l2(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.linalg.norm((got - ref).ravel()) / max(np.linalg.norm(ref.ravel()), 1e-300))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def to_host(t):
    return t.detach().cpu().numpy()


def oracle_plan(gpu_plan, table=None):
    """The oracle plan with the same d, M, L, m, method, window and beta as a
    GPU plan (beta read back from the library so that both use one value).
    The tests use sigma = L/M exactly."""
    info = gpu_plan.info()
    d = info["d"]
    method = "shannon" if info["method"] == 0 else "classic"
    window = {0: "sinh", 1: "ckb", 2: "table"}[info["window"]]
    sigma = info["L"][0] / info["M"][0]
    return O.make_plan(d, info["M"][:d], sigma, info["m"], method=method, window=window,
                       beta=info["beta"], table=table)
