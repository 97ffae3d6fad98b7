"""ctypes binding of libbf.so (include/bf.h): argument marshalling only.

Every computation runs in the CUDA library; torch tensors provide device memory and the
current CUDA stream.  Importing this module loads the library and raises if it is missing
(build it with ``python -m paper_1509_02468_gb300.build``): there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbf.so")

BF_OK, BF_EINVAL, BF_ECUDA, BF_EBREAKDOWN, BF_ENONFINITE, BF_ETIMEOUT, BF_ENOMEM = 0, -1, -2, -3, -4, -5, -6
F32, F64 = 0, 1
WINDOWS = {"square": 0, "cross": 1}
WEIGHT_MODES = {"onthefly": 0, "stored_f32": 1, "stored_bf16": 2}
OPS = {"W": 0, "L": 1, "DINV_W": 2, "D": 3, "NSYM": 4, "NDIAGL": 5}
PRECONDS = {"jacobi": 0, "identity": 1, "net": 2, "spd": 3}
BETAS = {"flexible": 0, "printed": 1}
PENCILS = {"D": 0, "I": 1}
GRAMS = {"fp32": 0, "bf16": 1, "bf16x3": 2, "bf16x6": 3}
STATUS = {0: "ran", 1: "converged", 2: "breakdown"}


class BFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libbf error {code}: {msg}")
        self.code = code


class bf_params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("window", ctypes.c_int32), ("weight_mode", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("sigma_s", ctypes.c_double), ("sigma_r", ctypes.c_double)]


class bf_guided_params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("radius", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("eps", ctypes.c_double)]


class bf_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("restarts", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rnorm", ctypes.c_double), ("ref", ctypes.c_double)]


class bf_cg_opts(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("shift", ctypes.c_double), ("tol", ctypes.c_double),
                ("hist", ctypes.c_void_p), ("net", ctypes.c_void_p), ("spd", ctypes.c_void_p)]


class bf_lobpcg_opts(ctypes.Structure):
    _fields_ = [("pencil", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("constrain_e", ctypes.c_int32), ("gram", ctypes.c_int32),
                ("tol", ctypes.c_double), ("theta_hist", ctypes.c_void_p),
                ("net", ctypes.c_void_p), ("spd", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_1509_02468_gb300.build`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "bf_weights": [ctypes.POINTER(bf_params), vp, ctypes.POINTER(vp), vp],
        "bf_guided_graph": [ctypes.POINTER(bf_guided_params), vp, ctypes.POINTER(vp), vp],
        "bf_graph_free": [vp],
        "bf_graph_update": [vp, vp, vp],
        "bf_graph_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32),
                          ctypes.POINTER(ctypes.c_int32)],
        "bf_graph_degree": [vp, vp, vp],
        "bf_graph_export_weights": [vp, vp, vp],
        "bf_apply": [vp, i32, vp, i64, i32, vp, i64, dp, vp],
        "bf_simple_filter": [vp, vp, i32, vp, vp],
        "bf_reguided_filter": [vp, vp, i32, vp, vp],
        "cg_filter": [vp, vp, i32, ctypes.POINTER(bf_cg_opts), vp, ctypes.POINTER(bf_info), vp],
        "lobpcg_filter": [vp, vp, i64, i32, i32, ctypes.POINTER(bf_lobpcg_opts), vp, dp, dp, vp,
                          ctypes.POINTER(bf_info), vp],
        "bf_rayleigh_ritz": [vp, i32, i32, i32, vp, vp, vp, vp, vp],
        "cg_filter_noalloc": [vp, vp, i32, ctypes.POINTER(bf_cg_opts), vp, ctypes.POINTER(bf_info), vp],
        "cg_refine": [vp, vp, vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(bf_cg_opts), i32, i32, vp,
                      ctypes.POINTER(bf_info), vp],
        "bf_shifted_residual": [vp, vp, vp, ctypes.c_double, vp, vp],
        "bf_net_nweights": [],
        "bf_net_create": [vp, ctypes.POINTER(vp)],
        "bf_net_free": [vp],
        "bf_net_weights": [vp, vp, i32],
        "bf_net_apply": [vp, vp, vp, i64, i32, vp, i64, vp],
        "bf_net_zero_grad": [vp, vp],
        "bf_net_accumulate": [vp, vp, vp, vp, vp],
        "bf_net_grad": [vp, vp, vp, vp],
        "bf_net_adam": [vp, ctypes.c_float, ctypes.c_float, vp],
        "bf_spd_create": [i32, vp, ctypes.POINTER(vp)],
        "bf_spd_free": [vp],
        "bf_spd_size": [vp],
        "bf_spd_weights": [vp, vp],
        "bf_spd_apply": [vp, vp, vp, i64, i32, vp, i64, vp],
        "bf_spd_zero_grad": [vp, vp],
        "bf_spd_accumulate": [vp, vp, ctypes.c_double, vp, vp, vp],
        "bf_spd_grad": [vp, vp, vp, vp],
        "bf_spd_adam": [vp, ctypes.c_float, ctypes.c_float, vp],
        "bf_gram_tc_test": [vp, vp, vp, vp, vp, vp, vp, i32, i32, i64, i32, vp, vp],
        "bf_wait_test": [i32, i32, vp],
        "bf_batch_create": [vp, i32, ctypes.POINTER(vp)],
        "bf_batch_free": [vp],
        "bf_batch_cg": [vp, vp, vp, i32, ctypes.POINTER(bf_cg_opts), vp, vp],
        "bf_batch_tune": [vp, vp, vp, i32, vp, vp],
        "bf_batch_cg_persistent": [vp, vp, vp, i32, ctypes.POINTER(bf_cg_opts), vp, vp],
        "bf_batch_barrier_test": [vp, vp, vp, i32, vp],
        "bf_batch_lobpcg": [vp, vp, i32, i32, ctypes.POINTER(bf_lobpcg_opts), vp, vp, i32, vp, vp],
        "bf_batch_tiles": [vp, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.bf_last_error.argtypes = []
    lib.bf_last_error.restype = ctypes.c_char_p
    lib.bf_launch_count.argtypes = []
    lib.bf_launch_count.restype = ctypes.c_uint64
    return lib


_lib = _load()


def lib():
    return _lib


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(_lib.bf_launch_count())


def _check(rc):
    if rc != BF_OK:
        raise BFError(rc, _lib.bf_last_error().decode())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


@dataclass
class Info:
    iters: int
    status: str
    restarts: int
    rnorm: float
    ref: float


def _info(i: bf_info) -> Info:
    return Info(i.iters, STATUS.get(i.status, str(i.status)), i.restarts, i.rnorm, i.ref)


class Graph:
    """A bf_graph handle (device buffers owned by the library)."""

    def __init__(self, handle, params, shape, dtype, device):
        self.handle = handle
        self.params = params
        self.shape = shape
        self.n = shape[0] * shape[1]
        self.dtype = dtype
        self.device = device

    def free(self):
        if self.handle:
            _lib.bf_graph_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def taps(self):
        t = ctypes.c_int32()
        _check(_lib.bf_graph_info(self.handle, None, ctypes.byref(t), None))
        return t.value


def bf_weights(guide: torch.Tensor, radius: int, sigma_s: float, sigma_r: float,
               window: str = "square", weight_mode: str = "onthefly", stream=None) -> Graph:
    """Graph of Section 2 from a 1D signal (shape (n,)) or an image (shape (ny, nx))."""
    if not guide.is_cuda or guide.dtype not in (torch.float32, torch.float64):
        raise ValueError("guide must be a float32/float64 CUDA tensor")
    guide = guide.contiguous()
    if guide.dim() == 1:
        ndim, ny, nx = 1, 1, guide.shape[0]
    elif guide.dim() == 2:
        ndim, ny, nx = 2, guide.shape[0], guide.shape[1]
    else:
        raise ValueError("guide must be 1D or 2D")
    p = bf_params(ndim=ndim, radius=radius, nx=nx, ny=ny, window=WINDOWS[window],
                  weight_mode=WEIGHT_MODES[weight_mode],
                  dtype=F64 if guide.dtype == torch.float64 else F32, reserved=0,
                  sigma_s=float(sigma_s), sigma_r=float(sigma_r))
    h = ctypes.c_void_p()
    _check(_lib.bf_weights(ctypes.byref(p), _ptr(guide), ctypes.byref(h), _stream(stream)))
    return Graph(h, p, (ny, nx), guide.dtype, guide.device)


def guided_graph(guide: torch.Tensor, radius: int, eps: float, stream=None) -> Graph:
    """The guided filter's graph of Section 3 (bf_guided_graph): Algorithm 1 as the
    operator D^-1 Wt, Wt of Eq. 6, from a 1D signal (shape (n,)) or an image (ny, nx)."""
    if not guide.is_cuda or guide.dtype not in (torch.float32, torch.float64):
        raise ValueError("guide must be a float32/float64 CUDA tensor")
    guide = guide.contiguous()
    if guide.dim() == 1:
        ndim, ny, nx = 1, 1, guide.shape[0]
    elif guide.dim() == 2:
        ndim, ny, nx = 2, guide.shape[0], guide.shape[1]
    else:
        raise ValueError("guide must be 1D or 2D")
    p = bf_guided_params(ndim=ndim, radius=radius, nx=nx, ny=ny,
                         dtype=F64 if guide.dtype == torch.float64 else F32, reserved=0,
                         eps=float(eps))
    h = ctypes.c_void_p()
    _check(_lib.bf_guided_graph(ctypes.byref(p), _ptr(guide), ctypes.byref(h), _stream(stream)))
    return Graph(h, p, (ny, nx), guide.dtype, guide.device)


def graph_update(g: Graph, guide: torch.Tensor, stream=None) -> Graph:
    """Recompute g for a new guide of the same shape and dtype (bf_graph_update): the same
    work as bf_weights into the graph's own buffers, no device allocation."""
    if not guide.is_cuda or guide.dtype != g.dtype or guide.device != g.device:
        raise ValueError("guide must be a CUDA tensor of the graph's dtype and device")
    guide = guide.contiguous()
    if tuple(guide.shape) != (tuple(g.shape) if guide.dim() == 2 else (g.n,)):
        raise ValueError("guide must have the graph's shape")
    _check(_lib.bf_graph_update(g.handle, _ptr(guide), _stream(stream)))
    return g


def graph_degree(g: Graph, stream=None) -> torch.Tensor:
    d = torch.empty(g.n, dtype=g.dtype, device=g.device)
    _check(_lib.bf_graph_degree(g.handle, _ptr(d), _stream(stream)))
    return d


def graph_export_weights(g: Graph, stream=None) -> torch.Tensor:
    out = torch.empty((g.n, g.taps), dtype=g.dtype, device=g.device)
    _check(_lib.bf_graph_export_weights(g.handle, _ptr(out), _stream(stream)))
    return out


def _as_block(X: torch.Tensor):
    if X.dim() == 1:
        return X.view(-1, 1), 1
    return X, X.shape[1]


def bf_apply(g: Graph, op: str, X: torch.Tensor, Y: torch.Tensor | None = None,
             dots: bool = False, stream=None):
    """Y = op X for X of shape (n,) or (n, k) (row stride may exceed k)."""
    Xb, k = _as_block(X)
    if Xb.stride(1) != 1:
        raise ValueError("X columns must be contiguous")
    if Y is None:
        Y = torch.empty_like(X, memory_format=torch.contiguous_format)
    Yb, _ = _as_block(Y)
    d = torch.empty(k, dtype=torch.float64, device=X.device) if dots else None
    _check(_lib.bf_apply(g.handle, OPS[op], _ptr(Xb), Xb.stride(0), k, _ptr(Yb), Yb.stride(0),
                         _ptr(d), _stream(stream)))
    return (Y, d) if dots else Y


def bf_simple_filter(g: Graph, x0: torch.Tensor, iters: int, out=None, stream=None):
    out = torch.empty_like(x0) if out is None else out
    _check(_lib.bf_simple_filter(g.handle, _ptr(x0), iters, _ptr(out), _stream(stream)))
    return out


def reguided_filter(g: Graph, x0: torch.Tensor, iters: int, out=None, stream=None):
    """iters steps of the nonlinear BF iteration (bf_reguided_filter): each step guides
    Eq. 2 by the current iterate.  g is overwritten with the graph of the last guide."""
    if not x0.is_cuda or x0.dtype != g.dtype or x0.numel() != g.n or not x0.is_contiguous():
        raise ValueError("x0 must be a contiguous CUDA tensor of the graph's dtype and size")
    out = torch.empty_like(x0) if out is None else out
    _check(_lib.bf_reguided_filter(g.handle, _ptr(x0), iters, _ptr(out), _stream(stream)))
    return out


def cg_filter(g: Graph, x0: torch.Tensor, kmax: int, precond: str = "jacobi",
              beta: str = "flexible", shift: float = 0.0, tol: float = 0.0,
              hist: bool = False, out=None, sync: bool = True, stream=None, net: "Net | None" = None,
              spd: "Spd | None" = None):
    """Algorithm 2.  Returns (x, info, hist) -- info None unless sync, hist None unless asked.
    precond="net" uses the learned preconditioner `net`, precond="spd" the learned SPD one."""
    out = torch.empty_like(x0) if out is None else out
    h = torch.full((2 * max(kmax, 1),), float("nan"), dtype=torch.float64, device=x0.device) if hist else None
    o = bf_cg_opts(precond=PRECONDS[precond], beta=BETAS[beta], shift=shift, tol=tol,
                   hist=h.data_ptr() if h is not None else None,
                   net=net.handle if net is not None else None,
                   spd=spd.handle if spd is not None else None)
    info = bf_info() if sync else None
    _check(_lib.cg_filter(g.handle, _ptr(x0), kmax, ctypes.byref(o), _ptr(out),
                          ctypes.byref(info) if info is not None else None, _stream(stream)))
    return out, (_info(info) if info is not None else None), h


def cg_filter_noalloc(g: Graph, x0: torch.Tensor, kmax: int, precond: str = "jacobi",
                      beta: str = "flexible", shift: float = 0.0, tol: float = 0.0,
                      out=None, sync: bool = True, stream=None):
    """cg_filter with its scratch in the library's static device array (no allocation by
    the library; n <= 262144).  Returns (x, info)."""
    out = torch.empty_like(x0) if out is None else out
    o = bf_cg_opts(precond=PRECONDS[precond], beta=BETAS[beta], shift=shift, tol=tol, hist=None)
    info = bf_info() if sync else None
    _check(_lib.cg_filter_noalloc(g.handle, _ptr(x0), kmax, ctypes.byref(o), _ptr(out),
                                  ctypes.byref(info) if info is not None else None,
                                  _stream(stream)))
    return out, (_info(info) if info is not None else None)


def shifted_residual(g: Graph, x0: torch.Tensor, x: torch.Tensor, shift: float, out=None, stream=None):
    """r = shift (x0 - x) - L x (bf_shifted_residual)."""
    out = torch.empty_like(x) if out is None else out
    _check(_lib.bf_shifted_residual(g.handle, _ptr(x0), _ptr(x), shift, _ptr(out), _stream(stream)))
    return out


def cg_refine(g64: Graph, g32: Graph, x0: torch.Tensor, shift: float, tol: float, precond: str = "jacobi",
              inner_tol: float = 1e-3, inner_kmax: int = 3000, outer_max: int = 30, net: "Net | None" = None,
              out=None, stream=None, spd: "Spd | None" = None):
    """(L + shift I) x = shift x0 to a true relative residual tol (cg_refine: FP64 residuals
    on g64, FP32 inner CG on g32).  x0: float64 CUDA tensor.  Returns (x, info)."""
    if x0.dtype != torch.float64:
        raise ValueError("x0 must be float64")
    out = torch.empty_like(x0) if out is None else out
    o = bf_cg_opts(precond=PRECONDS[precond], beta=BETAS["flexible"], shift=shift, tol=inner_tol, hist=None,
                   net=net.handle if net is not None else None, spd=spd.handle if spd is not None else None)
    info = bf_info()
    _check(_lib.cg_refine(g64.handle, g32.handle, _ptr(x0), shift, tol, ctypes.byref(o), inner_kmax, outer_max,
                          _ptr(out), ctypes.byref(info), _stream(stream)))
    return out, _info(info)


def lobpcg_filter(g: Graph, X0: torch.Tensor, kmax: int, pencil: str = "D",
                  precond: str = "jacobi", constrain: bool = False, tol: float = 0.0,
                  want_X: bool = True, want_y: bool = True, theta_hist: bool = False,
                  sync: bool = True, stream=None, net: "Net | None" = None, gram: str = "fp32",
                  spd: "Spd | None" = None):
    """Algorithm 3 on a block X0 of shape (n, k).  gram: "fp32" | "bf16" | "bf16x3" (tensor cores).  Returns a dict with X, theta, resid, y,
    theta_hist and info (entries None when not requested)."""
    Xb, k = _as_block(X0)
    dev = X0.device
    X = torch.empty((g.n, k), dtype=X0.dtype, device=dev) if want_X else None
    y = torch.empty(g.n, dtype=X0.dtype, device=dev) if want_y else None
    theta = torch.empty(k, dtype=torch.float64, device=dev)
    resid = torch.empty(k, dtype=torch.float64, device=dev)
    th = torch.full(((kmax + 1) * k,), float("nan"), dtype=torch.float64, device=dev) if theta_hist else None
    o = bf_lobpcg_opts(pencil=PENCILS[pencil], precond=PRECONDS[precond],
                       constrain_e=int(constrain), gram=GRAMS[gram], tol=tol,
                       theta_hist=th.data_ptr() if th is not None else None,
                       net=net.handle if net is not None else None,
                       spd=spd.handle if spd is not None else None)
    info = bf_info() if sync else None
    _check(_lib.lobpcg_filter(g.handle, _ptr(Xb), Xb.stride(0), k, kmax, ctypes.byref(o),
                              _ptr(X), _ptr(theta), _ptr(resid), _ptr(y),
                              ctypes.byref(info) if info is not None else None, _stream(stream)))
    return {"X": X, "theta": theta, "resid": resid, "y": y,
            "theta_hist": th.view(kmax + 1, k) if th is not None else None,
            "info": _info(info) if info is not None else None}


def rayleigh_ritz(GA: torch.Tensor, GB: torch.Tensor, k: int, m_nop: int = 0,
                  want_cp: bool = False, stream=None):
    """The LOBPCG Rayleigh-Ritz step on the GPU (include/bf_testing.h).  Returns
    (C, theta, Cp or None, status, restarts)."""
    m = GA.shape[0]
    dev = GA.device
    G = torch.stack([GA, GB]).to(torch.float64).contiguous()
    C = torch.empty((m, k), dtype=torch.float64, device=dev)
    Cp = torch.empty((m, k), dtype=torch.float64, device=dev) if want_cp else None
    theta = torch.empty(k, dtype=torch.float64, device=dev)
    flags = torch.zeros(2, dtype=torch.int32, device=dev)
    _check(_lib.bf_rayleigh_ritz(_ptr(G), m, k, m_nop, _ptr(C), _ptr(Cp), _ptr(theta),
                                 _ptr(flags), _stream(stream)))
    f = flags.cpu().tolist()
    return C, theta, Cp, f[0], f[1]


class Net:
    """The learned preconditioner (bf_net): a 3-layer 3 x 3 conv net, weights in FP32 and
    applied rounded to BF16.  `weights` is a flat float32 array of nweights() values or the
    list [W1 (16,3,3,3), W2 (16,16,3,3), W3 (1,16,3,3)]."""

    def __init__(self, weights):
        import numpy as np
        if isinstance(weights, (list, tuple)):
            weights = np.concatenate([np.asarray(w, np.float32).ravel() for w in weights])
        w = np.ascontiguousarray(np.asarray(weights, np.float32).ravel())
        if w.size != nweights():
            raise ValueError(f"expected {nweights()} weights, got {w.size}")
        h = ctypes.c_void_p()
        _check(_lib.bf_net_create(w.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self.handle = h.value

    def free(self):
        if getattr(self, "handle", None):
            _lib.bf_net_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def weights(self, rounded: bool = False):
        """Flat float32 numpy copy of the master (or BF16-rounded) weights."""
        import numpy as np
        w = np.empty(nweights(), np.float32)
        _check(_lib.bf_net_weights(self.handle, w.ctypes.data_as(ctypes.c_void_p), int(rounded)))
        return w

    def apply(self, g: Graph, R: torch.Tensor, out=None, stream=None):
        """Z = T(R) column by column; R is (n,) or (n, k)."""
        Rb, k = _as_block(R)
        Z = torch.empty_like(Rb) if out is None else out
        _check(_lib.bf_net_apply(self.handle, g.handle, _ptr(Rb), Rb.stride(0), k, _ptr(Z),
                                 Z.stride(0), _stream(stream)))
        return Z.view_as(R) if R.dim() == 1 else Z

    def zero_grad(self, stream=None):
        _check(_lib.bf_net_zero_grad(self.handle, _stream(stream)))

    def accumulate(self, g: Graph, r: torch.Tensor, z: torch.Tensor, stream=None):
        _check(_lib.bf_net_accumulate(self.handle, g.handle, _ptr(r), _ptr(z), _stream(stream)))

    def grad(self, stream=None):
        """(flat float32 gradient, loss) accumulated since the last reset."""
        import numpy as np
        gr = np.empty(nweights(), np.float32)
        loss = ctypes.c_double()
        _check(_lib.bf_net_grad(self.handle, gr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss),
                                _stream(stream)))
        return gr, loss.value

    def adam(self, lr: float, scale: float = 1.0, stream=None):
        _check(_lib.bf_net_adam(self.handle, ctypes.c_float(lr), ctypes.c_float(scale), _stream(stream)))


def nweights() -> int:
    return int(_lib.bf_net_nweights())


class Spd:
    """The learned symmetric positive definite preconditioner (bf_spd):
    T r = D^-1/2 (u + K^T K u), u = D^-1/2 r, K a (2h+1) x (2h+1) correlation kernel
    (float32, row-major taps; None: zero, i.e. Jacobi)."""

    def __init__(self, half: int, K=None):
        import numpy as np
        h = ctypes.c_void_p()
        if K is not None:
            Kc = np.ascontiguousarray(np.asarray(K, np.float32).reshape(-1))
            if Kc.size != (2 * half + 1) ** 2:
                raise ValueError(f"K must have {(2 * half + 1) ** 2} taps")
            _check(_lib.bf_spd_create(half, Kc.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        else:
            _check(_lib.bf_spd_create(half, None, ctypes.byref(h)))
        self.half = half
        self.handle = h.value

    def free(self):
        if getattr(self, "handle", None):
            _lib.bf_spd_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def kernel(self):
        """K as a (2h+1, 2h+1) float32 numpy array."""
        import numpy as np
        ks = 2 * self.half + 1
        K = np.empty(ks * ks, np.float32)
        _check(_lib.bf_spd_weights(self.handle, K.ctypes.data_as(ctypes.c_void_p)))
        return K.reshape(ks, ks)

    def apply(self, g: Graph, R: torch.Tensor, out=None, stream=None):
        """Z = T R column by column; R is (n,) or (n, k)."""
        Rb, k = _as_block(R)
        Z = torch.empty_like(Rb) if out is None else out
        _check(_lib.bf_spd_apply(self.handle, g.handle, _ptr(Rb), Rb.stride(0), k, _ptr(Z), Z.stride(0),
                                 _stream(stream)))
        return Z.view_as(R) if R.dim() == 1 else Z

    def zero_grad(self, stream=None):
        _check(_lib.bf_spd_zero_grad(self.handle, _stream(stream)))

    def accumulate(self, g: Graph, shift: float, r: torch.Tensor, z: torch.Tensor, stream=None):
        _check(_lib.bf_spd_accumulate(self.handle, g.handle, float(shift), _ptr(r), _ptr(z), _stream(stream)))

    def grad(self, stream=None):
        """(gradient as a (2h+1, 2h+1) float64 array, loss) accumulated since the last reset."""
        import numpy as np
        ks = 2 * self.half + 1
        gr = np.empty(ks * ks, np.float64)
        loss = ctypes.c_double()
        _check(_lib.bf_spd_grad(self.handle, gr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss),
                                _stream(stream)))
        return gr.reshape(ks, ks), loss.value

    def adam(self, lr: float, scale: float = 1.0, stream=None):
        _check(_lib.bf_spd_adam(self.handle, ctypes.c_float(lr), ctypes.c_float(scale), _stream(stream)))


class Batch:
    """Batched CG over many graphs (bf_batch): one work list per window shape, one CUDA
    graph per (kmax, options)."""

    def __init__(self, graphs):
        self.graphs = list(graphs)              # the batch keeps pointers to them
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.handle for g in self.graphs])
        h = ctypes.c_void_p()
        _check(_lib.bf_batch_create(arr, len(self.graphs), ctypes.byref(h)))
        self.handle = h.value

    def free(self):
        if getattr(self, "handle", None):
            _lib.bf_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @staticmethod
    def _ptrs(ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def cg(self, x0s, kmax: int, precond: str = "jacobi", beta: str = "flexible", shift: float = 0.0,
           tol: float = 0.0, outs=None, sync: bool = True, stream=None):
        """Returns (outs, infos) -- infos None unless sync."""
        outs = [torch.empty_like(x) for x in x0s] if outs is None else outs
        o = bf_cg_opts(precond=PRECONDS[precond], beta=BETAS[beta], shift=shift, tol=tol, hist=None, net=None)
        infos = (bf_info * len(x0s))() if sync else None
        _check(_lib.bf_batch_cg(self.handle, self._ptrs(x0s), self._ptrs(outs), kmax, ctypes.byref(o),
                                infos, _stream(stream)))
        return outs, ([_info(i) for i in infos] if infos is not None else None)

    def cg_persistent(self, x0s, kmax: int, precond: str = "jacobi", beta: str = "flexible",
                      shift: float = 0.0, tol: float = 0.0, outs=None, stream=None):
        """The same run in one persistent cooperative launch (bf_batch_cg_persistent);
        synchronises.  Returns (outs, infos)."""
        outs = [torch.empty_like(x) for x in x0s] if outs is None else outs
        o = bf_cg_opts(precond=PRECONDS[precond], beta=BETAS[beta], shift=shift, tol=tol, hist=None, net=None)
        infos = (bf_info * len(x0s))()
        _check(_lib.bf_batch_cg_persistent(self.handle, self._ptrs(x0s), self._ptrs(outs), kmax, ctypes.byref(o),
                                           infos, _stream(stream)))
        return outs, [_info(i) for i in infos]

    def barrier_test(self, x0s, kmax: int = 2, outs=None, stream=None):
        """Persistent run with one CTA that never reaches the first grid barrier
        (include/bf_testing.h): raises BFError(BF_ETIMEOUT)."""
        outs = [torch.empty_like(x) for x in x0s] if outs is None else outs
        _check(_lib.bf_batch_barrier_test(self.handle, self._ptrs(x0s), self._ptrs(outs), kmax, _stream(stream)))

    def lobpcg(self, X0s, kmax: int, nstreams: int = 32, pencil: str = "D", precond: str = "jacobi",
               constrain: bool = False, gram: str = "fp32", sync: bool = True, stream=None):
        """Algorithm 3 on every instance (bf_batch_lobpcg); X0s: list of (n_i, k) float32 blocks.
        Returns (thetas, ys, infos) -- infos None unless sync."""
        k = X0s[0].shape[1]
        thetas = [torch.empty(k, dtype=torch.float64, device=X.device) for X in X0s]
        ys = [torch.empty(X.shape[0], dtype=X.dtype, device=X.device) for X in X0s]
        o = bf_lobpcg_opts(pencil=PENCILS[pencil], precond=PRECONDS[precond], constrain_e=int(constrain),
                           gram=GRAMS[gram], tol=0.0, theta_hist=None, net=None)
        infos = (bf_info * len(X0s))() if sync else None
        _check(_lib.bf_batch_lobpcg(self.handle, self._ptrs(X0s), k, kmax, ctypes.byref(o), self._ptrs(thetas),
                                    self._ptrs(ys), nstreams, infos, _stream(stream)))
        if sync:
            torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return thetas, ys, ([_info(i) for i in infos] if infos is not None else None)

    def tune(self, x0s, iters: int = 5, outs=None, stream=None):
        """Autotune the image tile shape; returns the timings (ms) of the three candidates."""
        outs = [torch.empty_like(x) for x in x0s] if outs is None else outs
        ms = (ctypes.c_float * 3)()
        _check(_lib.bf_batch_tune(self.handle, self._ptrs(x0s), self._ptrs(outs), iters, ms, _stream(stream)))
        return list(ms)

    def tiles(self):
        t, v = ctypes.c_int64(), ctypes.c_int32()
        _check(_lib.bf_batch_tiles(self.handle, ctypes.byref(t), ctypes.byref(v)))
        return t.value, v.value


def wait_test(iters: int, arrive: bool, stream=None):
    """The library's bounded device wait on a barrier of its own (include/bf_testing.h):
    returns normally when thread 0 arrives, raises BFError(BF_ETIMEOUT) when nothing does."""
    _check(_lib.bf_wait_test(int(iters), int(bool(arrive)), _stream(stream)))


def gram_tc(S_blocks, AS_blocks, b=None, split: bool = False, stream=None, mode: str | None = None):
    """Tensor-core Gram (include/bf_testing.h): returns (S^T AS, S^T B S) as float64 tensors
    for lists of 1..3 pixel-major float32 blocks of shape (n, k).  mode: "bf16", "bf16x3"
    or "bf16x6" (default: "bf16x3" if split else "bf16")."""
    nblk = len(S_blocks)
    n, k = S_blocks[0].shape
    m = nblk * k
    mode = mode or ("bf16x3" if split else "bf16")
    G = torch.empty((2, m, m), dtype=torch.float64, device=S_blocks[0].device)
    Sp = [_ptr(x) for x in S_blocks] + [None] * (3 - nblk)
    Ap = [_ptr(x) for x in AS_blocks] + [None] * (3 - nblk)
    _check(_lib.bf_gram_tc_test(*Sp, *Ap, _ptr(b), nblk, k, n, GRAMS[mode], _ptr(G), _stream(stream)))
    return G[0], G[1]
