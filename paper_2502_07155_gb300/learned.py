"""Training driver for the learned window (tabulated MLP window phi_theta).

Every arithmetic step of a training iteration runs in the library's kernels
(C-ABI): the MLP forward and table (nfftbl_mlp_table), psi_hat of the table
by quadrature (nfftbl_set_window_table), the transform, its loss and the
gradient with respect to the table (nfftbl_window_loss_grad), the MLP
backward with BF16 tensor-core products (nfftbl_mlp_backward) and Adam
(nfftbl_adam_step).  This module allocates the device buffers and loops.

Window: phi_theta(u) = (1 - u^2) exp(g(u^2) - g(0)) on u = |Lx|/m, an even
window with phi(0) = 1 and phi(1) = 0 (the class Phi_{m,L} of Section 3);
tabulated at table_len = 4097 points and interpolated by Catmull-Rom
inside the short-sum kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Plan, lib, NfftblError, STATUS

HIDDEN = 64


def init_params(hidden: int = HIDDEN, seed: int = 4) -> np.ndarray:
    """Seeded initial parameters in the C-ABI layout (W1, b1, W2, b2, W3, b3).
    The output layer starts small, so the first window is close to 1 - u^2."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal(hidden) * 1.0
    b1 = rng.standard_normal(hidden) * 0.5
    W2 = rng.standard_normal((hidden, hidden)) / np.sqrt(hidden)
    b2 = np.zeros(hidden)
    W3 = rng.standard_normal(hidden) * 0.01
    b3 = np.zeros(1)
    return np.concatenate([W1, b1, W2.reshape(-1), b2, W3, b3]).astype(np.float32)


def params_to_dict(p: np.ndarray, hidden: int = HIDDEN) -> dict:
    """Split a flat parameter vector into named arrays (float64)."""
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in [("W1", (hidden, 1)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
                        ("W3", (1, hidden)), ("b3", (1,))]:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def _check(st: int, what: str):
    if st != 0:
        raise NfftblError(st, what)


class WindowTrainer:
    """Trains phi_theta for one plan shape (d, M, sigma, m) on fixed nodes,
    Fourier data and targets (the trigonometric sums at the nodes)."""

    def __init__(self, d: int, M, m: int, sigma: float = 2.0, table_len: int = 4097, batch: int = 1,
                 params: np.ndarray | None = None, lr: float = 3e-3):
        import torch
        self.torch = torch
        self.lib = lib()
        self.table_len = table_len
        self.count = int(self.lib.nfftbl_mlp_param_count(HIDDEN))
        p0 = init_params() if params is None else np.asarray(params, dtype=np.float32)
        dev = torch.device("cuda")
        self.params = torch.from_numpy(p0.copy()).to(dev)
        self.grad = torch.zeros(self.count, dtype=torch.float32, device=dev)
        self.m1 = torch.zeros_like(self.grad)
        self.m2 = torch.zeros_like(self.grad)
        self.table = torch.zeros(table_len, dtype=torch.float64, device=dev)
        self.act = torch.zeros(table_len * (2 * HIDDEN + 1), dtype=torch.float32, device=dev)
        self.scratch = torch.zeros(int(self.lib.nfftbl_mlp_scratch_floats(HIDDEN, table_len)), dtype=torch.float32,
                                   device=dev)
        self.grad_table = torch.zeros(table_len, dtype=torch.float64, device=dev)
        self.loss = torch.zeros(3, dtype=torch.float64, device=dev)
        self.lr = lr
        self.steps = 0
        self._make_table()
        self.plan = Plan(d, M, sigma, m, window="table", table=self.table.cpu().numpy(), precision="f32",
                         batch=batch)

    def _ptr(self, t):
        return ctypes.c_void_p(t.data_ptr())

    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def _make_table(self):
        _check(self.lib.nfftbl_mlp_table(self._ptr(self.params), HIDDEN, self.table_len, self._ptr(self.table),
                                         self._ptr(self.act), self._stream()), "nfftbl_mlp_table")

    def set_data(self, x, fhat, y):
        """Training nodes (N, d) float32, Fourier data (B, M..) complex64 and
        targets (B, N) complex64, all CUDA tensors."""
        self.plan.set_nodes(x)
        self.fhat = fhat.contiguous()
        self.y = y.contiguous()

    def loss_and_grads(self):
        """Refresh the table from the MLP, then the loss, dE/d(table) and dE/d(params)."""
        self._make_table()
        self.plan.set_window_table(self.table)
        self.plan.window_loss_grad(self.fhat, self.y, self.grad_table, self.loss)
        _check(self.lib.nfftbl_mlp_backward(self._ptr(self.params), HIDDEN, self.table_len, self._ptr(self.act),
                                            self._ptr(self.table), self._ptr(self.grad_table),
                                            self._ptr(self.scratch), self._ptr(self.grad), self._stream()),
               "nfftbl_mlp_backward")

    def step(self, lr: float | None = None):
        self.loss_and_grads()
        self.steps += 1
        _check(self.lib.nfftbl_adam_step(self._ptr(self.params), self._ptr(self.grad), self._ptr(self.m1),
                                         self._ptr(self.m2), self.count, self.steps,
                                         float(self.lr if lr is None else lr), 0.9, 0.999, 1e-8, self._stream()),
               "nfftbl_adam_step")

    def train(self, steps: int, lr_final: float | None = None, log_every: int = 0):
        """Adam with a cosine-decayed learning rate; returns the loss history
        read back every log_every steps (0: only the last)."""
        hist = []
        lr0 = self.lr
        lr1 = lr0 * 0.05 if lr_final is None else lr_final
        for i in range(steps):
            lr = lr1 + 0.5 * (lr0 - lr1) * (1 + np.cos(np.pi * i / max(1, steps)))
            self.step(lr)
            if log_every and (i % log_every == 0):
                hist.append((i, float(self.loss[0].item())))
        self.loss_and_grads()
        hist.append((steps, float(self.loss[0].item())))
        return hist

    def table_host(self) -> np.ndarray:
        self._make_table()
        return self.table.cpu().numpy()
