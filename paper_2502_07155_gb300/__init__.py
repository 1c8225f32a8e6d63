"""GB300-native NFFT for bandlimited functions (Kircheis & Potts).

Python binding of the C-ABI library ``libnfftbl.so`` (``include/nfftbl.h``).
This module only marshals arguments: every step of every transform runs in
the library's CUDA kernels.  PyTorch supplies device memory and streams.
There is no CPU fallback: if the library is missing or no GPU is present,
constructing a :class:`Plan` raises.

    import torch, paper_2502_07155_gb300 as nb
    plan = nb.Plan(d=2, M=256, sigma=2.0, m=8)            # Algorithm 4.2, FP32
    plan.set_nodes(x)                                      # (N, 2) float32, cuda
    f = plan.forward(fhat)                                 # (B, 256, 256) -> (B, N)
    g = plan.adjoint(f)                                    # (B, N) -> (B, 256, 256)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

__all__ = ["Plan", "NfftblError", "lib", "library_path", "STATUS", "oversampled_length"]

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libnfftbl.so")

STATUS = {0: "OK", 1: "EINVAL", 2: "EDOMAIN", 3: "EUNSUPPORTED", 4: "ENOMEM", 5: "ECUDA",
          6: "ESTATE", 7: "ETIMEOUT", 8: "EINTERNAL"}
_WINDOWS = {"sinh": 0, "ckb": 1, "table": 2}
_PRECISIONS = {"f64": 0, "f32": 1, "f32c": 2}
_METHODS = {"shannon": 0, "classic": 1}

EXPORTED = [
    "nfftbl_default_opts", "nfftbl_plan", "nfftbl_set_stream", "nfftbl_set_nodes", "nfftbl_forward",
    "nfftbl_adjoint", "nfftbl_node_grad", "nfftbl_sync", "nfftbl_destroy", "nfftbl_last_error",
    "nfftbl_plan_error", "nfftbl_get_info", "nfftbl_get_factors", "nfftbl_get_binning", "nfftbl_get_grid",
    "nfftbl_grid_ptr", "nfftbl_interp_grid", "nfftbl_spread_grid", "nfftbl_kernel_launches",
    "nfftbl_kernel_timing", "nfftbl_kernel_times", "nfftbl_grid_noalloc",
    "nfftbl_set_window_table", "nfftbl_window_loss_grad", "nfftbl_mlp_table", "nfftbl_mlp_backward",
    "nfftbl_mlp_param_count", "nfftbl_mlp_scratch_floats", "nfftbl_adam_step", "nfftbl_window_transform",
    "nfftbl_forward_host", "nfftbl_adjoint_host", "nfftbl_join", "nfftbl_set_wait_limit",
]
KERNEL_CLASSES = ("fft", "interp", "spread", "grad", "bin", "flush")


class NfftblError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("method", ctypes.c_int), ("beta", ctypes.c_double),
                ("batch", ctypes.c_int), ("table", ctypes.POINTER(ctypes.c_double)),
                ("table_len", ctypes.c_int), ("tile", ctypes.c_int * 3), ("nodes_per_item", ctypes.c_int),
                ("factors", ctypes.c_int), ("precorrect", ctypes.c_int), ("weights", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("M", ctypes.c_int * 3), ("L", ctypes.c_int * 3), ("m", ctypes.c_int),
                ("precision", ctypes.c_int), ("method", ctypes.c_int), ("window", ctypes.c_int),
                ("batch", ctypes.c_int), ("beta", ctypes.c_double), ("tile", ctypes.c_int * 3),
                ("n_nodes", ctypes.c_int64), ("n_tiles", ctypes.c_int64), ("n_work", ctypes.c_int64),
                ("key_bits", ctypes.c_int), ("poly_weights", ctypes.c_int), ("poly_err", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libnfftbl.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(library_path):
        raise RuntimeError(f"{library_path} is missing: build it with paper_2502_07155_gb300.build.build()")
    L = ctypes.CDLL(library_path)
    P = ctypes.c_void_p
    st = ctypes.c_int
    L.nfftbl_default_opts.argtypes = [ctypes.POINTER(_Opts)]
    L.nfftbl_default_opts.restype = None
    L.nfftbl_plan.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_double,
                              ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Opts)]
    L.nfftbl_plan.restype = st
    L.nfftbl_set_stream.argtypes = [P, P]
    L.nfftbl_set_stream.restype = st
    L.nfftbl_set_nodes.argtypes = [P, ctypes.c_int64, P]
    L.nfftbl_set_nodes.restype = st
    for name in ("nfftbl_forward", "nfftbl_adjoint", "nfftbl_forward_host", "nfftbl_adjoint_host"):
        getattr(L, name).argtypes = [P, P, P]
        getattr(L, name).restype = st
    L.nfftbl_join.argtypes = [P]
    L.nfftbl_join.restype = st
    L.nfftbl_node_grad.argtypes = [P, P, P, P]
    L.nfftbl_node_grad.restype = st
    L.nfftbl_set_wait_limit.argtypes = [P, ctypes.c_int64, ctypes.c_int]
    L.nfftbl_set_wait_limit.restype = st
    L.nfftbl_sync.argtypes = [P]
    L.nfftbl_sync.restype = st
    L.nfftbl_destroy.argtypes = [P]
    L.nfftbl_destroy.restype = st
    L.nfftbl_last_error.argtypes = [P]
    L.nfftbl_last_error.restype = ctypes.c_char_p
    L.nfftbl_plan_error.argtypes = []
    L.nfftbl_plan_error.restype = ctypes.c_char_p
    L.nfftbl_get_info.argtypes = [P, ctypes.POINTER(_Info)]
    L.nfftbl_get_info.restype = st
    L.nfftbl_get_factors.argtypes = [P, ctypes.c_int, P]
    L.nfftbl_get_factors.restype = st
    L.nfftbl_get_binning.argtypes = [P, P, P, P]
    L.nfftbl_get_binning.restype = st
    L.nfftbl_get_grid.argtypes = [P, P]
    L.nfftbl_get_grid.restype = st
    L.nfftbl_grid_ptr.argtypes = [P, ctypes.POINTER(P)]
    L.nfftbl_grid_ptr.restype = st
    L.nfftbl_interp_grid.argtypes = [P, P]
    L.nfftbl_interp_grid.restype = st
    L.nfftbl_window_transform.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P]
    L.nfftbl_window_transform.restype = st
    L.nfftbl_spread_grid.argtypes = [P, P]
    L.nfftbl_spread_grid.restype = st
    L.nfftbl_kernel_launches.argtypes = [P]
    L.nfftbl_kernel_launches.restype = ctypes.c_int64
    L.nfftbl_kernel_timing.argtypes = [P, ctypes.c_int]
    L.nfftbl_kernel_timing.restype = st
    L.nfftbl_kernel_times.argtypes = [P, P, P]
    L.nfftbl_kernel_times.restype = st
    L.nfftbl_grid_noalloc.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, P, P, P]
    L.nfftbl_grid_noalloc.restype = st
    L.nfftbl_set_window_table.argtypes = [P, P, ctypes.c_int]
    L.nfftbl_set_window_table.restype = st
    L.nfftbl_window_loss_grad.argtypes = [P, P, P, P, P]
    L.nfftbl_window_loss_grad.restype = st
    L.nfftbl_mlp_table.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P]
    L.nfftbl_mlp_table.restype = st
    L.nfftbl_mlp_backward.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, P, P, P, P]
    L.nfftbl_mlp_backward.restype = st
    L.nfftbl_mlp_param_count.argtypes = [ctypes.c_int]
    L.nfftbl_mlp_param_count.restype = ctypes.c_int64
    L.nfftbl_mlp_scratch_floats.argtypes = [ctypes.c_int, ctypes.c_int]
    L.nfftbl_mlp_scratch_floats.restype = ctypes.c_int64
    L.nfftbl_adam_step.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, P]
    L.nfftbl_adam_step.restype = st
    _lib = L
    return L


def oversampled_length(M: int, sigma: float) -> int:
    """L = 2 ceil(ceil(sigma M)/2) (the library computes the same; mirrored
    here only to size output tensors)."""
    import math
    s = math.ceil(sigma * M - 1e-9)
    return 2 * ((s + 1) // 2)


def _torch():
    import torch
    return torch


class Plan:
    """One transform configuration with its device state (C-ABI nfftbl_plan_t).

    Arguments follow ``nfftbl_plan``: ``d``, ``M`` (int or d ints),
    ``sigma``, ``m``, ``window`` ('sinh' | 'ckb' | 'table'), and the options
    ``precision`` ('f32' | 'f32c' | 'f64'), ``method`` ('shannon' |
    'classic'), ``beta`` (None = default), ``batch``, ``table`` (values on
    u in [0, 1] for the table window), ``tile``, ``nodes_per_item``,
    ``factors`` (keep the d x 2m window factors per node from set_nodes),
    ``precorrect`` (False: D = I, Section 5's approximation |I_L| psi_hat ~ 1),
    ``weights`` ('closed': the window's closed form, the default; 'poly':
    per-tap polynomial weights in the FP32 spreading where they are accurate).
    """

    def __init__(self, d: int, M, sigma: float = 2.0, m: int = 6, window: str = "sinh",
                 precision: str = "f32", method: str = "shannon", beta: float | None = None,
                 batch: int = 1, table=None, tile=None, nodes_per_item: int | None = None,
                 factors: bool = False, precorrect: bool = True, weights: str = "closed"):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("nfftbl needs a CUDA device; there is no CPU fallback")
        self._lib = lib()
        Ms = [int(M)] * d if np.ndim(M) == 0 else [int(v) for v in M]
        self.d = d
        self.M = tuple(Ms)
        self.precision = precision
        self.method = method
        self.batch = batch
        o = _Opts()
        self._lib.nfftbl_default_opts(ctypes.byref(o))
        o.precision = _PRECISIONS[precision]
        o.method = _METHODS[method]
        o.beta = 0.0 if beta is None else float(beta)
        o.batch = int(batch)
        self._table = None
        if table is not None:
            self._table = np.ascontiguousarray(np.asarray(table, dtype=np.float64))
            o.table = self._table.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            o.table_len = self._table.size
        if tile is not None:
            for t, v in enumerate(tile):
                o.tile[t] = int(v)
        if nodes_per_item:
            o.nodes_per_item = int(nodes_per_item)
        o.factors = 1 if factors else 0
        o.precorrect = 1 if precorrect else 0
        o.weights = {"closed": 0, "poly": 1}[weights]
        Marr = (ctypes.c_int * 3)(*(Ms + [0] * (3 - d)))
        h = ctypes.c_void_p()
        st = self._lib.nfftbl_plan(ctypes.byref(h), d, Marr, float(sigma), int(m), _WINDOWS[window], ctypes.byref(o))
        if st != 0:
            raise NfftblError(st, self._lib.nfftbl_plan_error().decode())
        self._h = h
        info = self.info()
        self.L = tuple(info["L"][:d])
        self.m = m
        self.beta = info["beta"]
        self.n_nodes = -1
        self._rdtype = torch.float64 if precision == "f64" else torch.float32
        self._cdtype = torch.complex128 if precision == "f64" else torch.complex64

    # ------------------------------------------------------------------ helpers
    def _check(self, st: int):
        if st != 0:
            raise NfftblError(st, self._lib.nfftbl_last_error(self._h).decode())

    def _stream(self):
        torch = _torch()
        self._lib.nfftbl_set_stream(self._h, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    def _dev(self, t, dtype, shape=None, name="tensor"):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype:
            raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return ctypes.c_void_p(t.data_ptr())

    def _host(self, t, shape, name):
        """Data pointer of a contiguous host array of the plan's complex dtype:
        a CPU torch tensor (page-locked for asynchronous copies) or a numpy
        array."""
        torch = _torch()
        if isinstance(t, np.ndarray):
            want = np.complex128 if self.precision == "f64" else np.complex64
            if t.dtype != want:
                raise TypeError(f"{name} must have dtype {np.dtype(want)}, got {t.dtype}")
            if tuple(t.shape) != tuple(shape):
                raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
            if not t.flags.c_contiguous:
                raise ValueError(f"{name} must be C-contiguous")
            return ctypes.c_void_p(t.ctypes.data)
        if not isinstance(t, torch.Tensor) or t.is_cuda:
            raise TypeError(f"{name} must be a CPU tensor or a numpy array")
        if t.dtype != self._cdtype:
            raise TypeError(f"{name} must have dtype {self._cdtype}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return ctypes.c_void_p(t.data_ptr())

    @property
    def handle(self):
        return self._h

    # ------------------------------------------------------------------ API
    def set_nodes(self, x):
        """Nodes x: (N, d) CUDA tensor, float32 (f32 plans) or float64 (f64)."""
        if x.dim() != 2 or x.shape[1] != self.d:
            raise ValueError(f"x must have shape (N, {self.d})")
        ptr = self._dev(x, self._rdtype, name="x")
        self._stream()
        self._check(self._lib.nfftbl_set_nodes(self._h, int(x.shape[0]), ptr))
        self.n_nodes = int(x.shape[0])
        return self

    def forward(self, fhat, out=None):
        """f = Psi F D fhat: (B, M_0, .., M_{d-1}) -> (B, N) complex."""
        torch = _torch()
        fh = self._dev(fhat, self._cdtype, (self.batch,) + self.M, "fhat")
        if out is None:
            out = torch.empty((self.batch, max(self.n_nodes, 0)), dtype=self._cdtype, device=fhat.device)
        po = self._dev(out, self._cdtype, (self.batch, max(self.n_nodes, 0)), "out")
        self._stream()
        self._check(self._lib.nfftbl_forward(self._h, fh, po))
        return out

    def adjoint(self, f, out=None):
        """fhat = D F^H Psi^T f: (B, N) -> (B, M_0, .., M_{d-1}) complex."""
        torch = _torch()
        pf = self._dev(f, self._cdtype, (self.batch, max(self.n_nodes, 0)), "f")
        if out is None:
            out = torch.empty((self.batch,) + self.M, dtype=self._cdtype, device=f.device)
        po = self._dev(out, self._cdtype, (self.batch,) + self.M, "out")
        self._stream()
        self._check(self._lib.nfftbl_adjoint(self._h, pf, po))
        return out

    def forward_host(self, fhat, out=None):
        """forward() with host input and output (CPU tensors or numpy arrays;
        page-locked tensors give asynchronous copies that overlap other calls'
        transforms).  Asynchronous: the caller keeps fhat and out alive and
        reads out after sync() (or after work on the plan stream that follows
        join())."""
        torch = _torch()
        pi = self._host(fhat, (self.batch,) + self.M, "fhat")
        if out is None:
            out = torch.empty((self.batch, max(self.n_nodes, 0)), dtype=self._cdtype, pin_memory=True)
        po = self._host(out, (self.batch, max(self.n_nodes, 0)), "out")
        self._stream()
        self._check(self._lib.nfftbl_forward_host(self._h, pi, po))
        return out

    def adjoint_host(self, f, out=None):
        """adjoint() with host input and output; see forward_host."""
        torch = _torch()
        pi = self._host(f, (self.batch, max(self.n_nodes, 0)), "f")
        if out is None:
            out = torch.empty((self.batch,) + self.M, dtype=self._cdtype, pin_memory=True)
        po = self._host(out, (self.batch,) + self.M, "out")
        self._stream()
        self._check(self._lib.nfftbl_adjoint_host(self._h, pi, po))
        return out

    def join(self):
        """Order later work on the plan stream after the host-buffer calls'
        downloads (no host blocking)."""
        self._stream()
        self._check(self._lib.nfftbl_join(self._h))

    def node_grad(self, fhat, grad_f, out=None):
        """grad_x[j, t] = sum_b Re(conj(grad_f[b, j]) d f_{b,j} / d x_{j,t}), shape (N, d)."""
        torch = _torch()
        fh = self._dev(fhat, self._cdtype, (self.batch,) + self.M, "fhat")
        gf = self._dev(grad_f, self._cdtype, (self.batch, max(self.n_nodes, 0)), "grad_f")
        if out is None:
            out = torch.empty((max(self.n_nodes, 0), self.d), dtype=self._rdtype, device=fhat.device)
        po = self._dev(out, self._rdtype, (max(self.n_nodes, 0), self.d), "out")
        self._stream()
        self._check(self._lib.nfftbl_node_grad(self._h, fh, gf, po))
        return out

    def interp_grid(self, out=None):
        """Step 3 alone on the plan's current grid: (B, N)."""
        torch = _torch()
        if out is None:
            out = torch.empty((self.batch, max(self.n_nodes, 0)), dtype=self._cdtype, device="cuda")
        po = self._dev(out, self._cdtype, (self.batch, max(self.n_nodes, 0)), "out")
        self._stream()
        self._check(self._lib.nfftbl_interp_grid(self._h, po))
        return out

    def window_transform(self, v, t: int = 0):
        """psi_hat(v) (phi_hat for the classical method) of dimension t at the
        real frequencies v (a float64 CUDA tensor), by the plan's quadrature."""
        torch = _torch()
        v = v.to(device="cuda", dtype=torch.float64).contiguous()
        out = torch.empty_like(v)
        self._stream()
        self._check(self._lib.nfftbl_window_transform(self._h, int(t), ctypes.c_void_p(v.data_ptr()), v.numel(),
                                                      ctypes.c_void_p(out.data_ptr())))
        return out

    def spread_grid(self, f):
        """Transposed step 3 into the plan's grid (cleared first)."""
        pf = self._dev(f, self._cdtype, (self.batch, max(self.n_nodes, 0)), "f")
        self._stream()
        self._check(self._lib.nfftbl_spread_grid(self._h, pf))

    def grid_tensor(self):
        """A torch view of the plan's grid (B, L_0, .., L_{d-1}) (no copy; valid
        while the plan lives)."""
        torch = _torch()
        p = ctypes.c_void_p()
        self._check(self._lib.nfftbl_grid_ptr(self._h, ctypes.byref(p)))
        n = self.batch * int(np.prod(self.L))
        es = 16 if self.precision == "f64" else 8
        # wrap the raw device pointer through the CUDA array interface
        holder = _DevicePtr(p.value, n * es, self._cdtype)
        t = torch.as_tensor(holder, device="cuda")
        return t.view((self.batch,) + self.L)

    def sync(self):
        self._check(self._lib.nfftbl_sync(self._h))

    def set_wait_limit(self, limit_ns: int = 0, stall_next: bool = False):
        """Limit of the bounded tile-copy waits in ns (0: the default 2 s);
        stall_next arms the next interpolation's waits with nothing to
        complete them (a test of the timeout path)."""
        self._check(self._lib.nfftbl_set_wait_limit(self._h, int(limit_ns), 1 if stall_next else 0))

    def info(self) -> dict:
        inf = _Info()
        self._check(self._lib.nfftbl_get_info(self._h, ctypes.byref(inf)))
        return {"d": inf.d, "M": list(inf.M), "L": list(inf.L), "m": inf.m, "precision": inf.precision,
                "method": inf.method, "window": inf.window, "batch": inf.batch, "beta": inf.beta,
                "tile": list(inf.tile), "n_nodes": inf.n_nodes, "n_tiles": inf.n_tiles, "n_work": inf.n_work,
                "key_bits": inf.key_bits, "poly_weights": inf.poly_weights, "poly_err": inf.poly_err}

    def factors(self, t: int) -> np.ndarray:
        """d_t(k) = 1/(L_t psi_hat_t(k)), k in I_{M_t} (host copy)."""
        out = np.empty(self.M[t], dtype=np.float64)
        self._check(self._lib.nfftbl_get_factors(self._h, t, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def binning(self):
        """(keys, perm, tile_off) as uint32 host arrays."""
        n = max(self.n_nodes, 0)
        info = self.info()
        keys = np.empty(n, dtype=np.uint32)
        perm = np.empty(n, dtype=np.uint32)
        off = np.empty(info["n_tiles"] + 1, dtype=np.uint32)
        self._check(self._lib.nfftbl_get_binning(self._h, keys.ctypes.data_as(ctypes.c_void_p),
                                                 perm.ctypes.data_as(ctypes.c_void_p),
                                                 off.ctypes.data_as(ctypes.c_void_p)))
        return keys, perm, off

    def grid(self) -> np.ndarray:
        """Host copy of the grid, (B, L_0, .., L_{d-1}) complex."""
        dt = np.complex128 if self.precision == "f64" else np.complex64
        out = np.empty((self.batch,) + self.L, dtype=dt)
        self._check(self._lib.nfftbl_get_grid(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_window_table(self, table_dev):
        """Replace the table window by a (len,) float64 CUDA tensor."""
        t = self._dev(table_dev, _torch().float64, name="table")
        self._stream()
        self._check(self._lib.nfftbl_set_window_table(self._h, t, int(table_dev.numel())))

    def window_loss_grad(self, fhat, y, grad_table, loss):
        """E = ||f - y||^2/||y||^2 and dE/d(table) into the given float64 CUDA
        tensors (grad_table: (len,), loss: (3,) = E, num, den)."""
        torch = _torch()
        fh = self._dev(fhat, self._cdtype, (self.batch,) + self.M, "fhat")
        yy = self._dev(y, self._cdtype, (self.batch, max(self.n_nodes, 0)), "y")
        gt = self._dev(grad_table, torch.float64, name="grad_table")
        ls = self._dev(loss, torch.float64, (3,), "loss")
        self._stream()
        self._check(self._lib.nfftbl_window_loss_grad(self._h, fh, yy, gt, ls))

    def kernel_launches(self) -> int:
        return int(self._lib.nfftbl_kernel_launches(self._h))

    def kernel_timing(self, enable: bool = True):
        """Record CUDA events around each later kernel launch (resets sums)."""
        self._check(self._lib.nfftbl_kernel_timing(self._h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """{class: (total_ms, launches)} since the last call; resets."""
        ms = np.zeros(len(KERNEL_CLASSES), dtype=np.float64)
        cnt = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
        self._check(self._lib.nfftbl_kernel_times(self._h, ms.ctypes.data_as(ctypes.c_void_p),
                                                  cnt.ctypes.data_as(ctypes.c_void_p)))
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.nfftbl_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_noalloc(fhat, sigma: float, m: int, grid=None, beta: float | None = None):
    """Steps 1-2 without any device allocation inside the library
    (C-ABI nfftbl_grid_noalloc): fhat (B, M_0, .., M_{d-1}) complex64 CUDA
    tensor -> grid (B, L_0, .., L_{d-1}) complex64.  For callers that cannot
    allocate device memory through the library; pass ``grid`` to supply the
    output buffer as well.  Calls that overlap on the GPU share one fixed
    scratch array and must be serialised."""
    torch = _torch()
    L_ = lib()
    d = fhat.dim() - 1
    Ms = [int(v) for v in fhat.shape[1:]]
    Ls = [oversampled_length(v, sigma) for v in Ms]
    if fhat.dtype != torch.complex64 or not fhat.is_cuda or not fhat.is_contiguous():
        raise TypeError("fhat must be a contiguous complex64 CUDA tensor")
    if grid is None:
        grid = torch.empty([fhat.shape[0]] + Ls, dtype=torch.complex64, device=fhat.device)
    Marr = (ctypes.c_int * 3)(*(Ms + [0] * (3 - d)))
    st = L_.nfftbl_grid_noalloc(d, Marr, float(sigma), int(m), 0.0 if beta is None else float(beta),
                                int(fhat.shape[0]), ctypes.c_void_p(fhat.data_ptr()),
                                ctypes.c_void_p(grid.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise NfftblError(st, L_.nfftbl_plan_error().decode())
    return grid


class _DevicePtr:
    """Minimal __cuda_array_interface__ wrapper around a library-owned buffer."""

    def __init__(self, ptr: int, nbytes: int, cdtype):
        torch = _torch()
        self._ptr = ptr
        typestr = "<c16" if cdtype == torch.complex128 else "<c8"
        es = 16 if cdtype == torch.complex128 else 8
        self.__cuda_array_interface__ = {"shape": (nbytes // es,), "typestr": typestr,
                                         "data": (ptr, False), "version": 2, "strides": None}
