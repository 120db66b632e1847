"""Python binding of libptn.so (the C ABI in include/ptn.h).

Argument marshalling only: every step of a solve runs in the CUDA library.  Device
arrays are torch tensors (float64, contiguous, on the solver's device); the stream is
torch's current stream unless given.  ``load()`` raises if the library is missing --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PTN_LIB selects another build of the library (e.g. one with user models linked in)
LIB_PATH = os.environ.get("PTN_LIB") or os.path.join(_HERE, "_build", "libptn.so")

PTN_FP64, PTN_FP32_FP64SOLVE, PTN_FP32 = 0, 1, 2
METHOD_IP, METHOD_ADMM = 0, 1
PTN_ERR_INVALID_ARG, PTN_ERR_CUDA = -1, -6
STATUS = {0: "ok", -1: "invalid argument", -2: "infeasible start", -3: "not converged",
          -4: "numerical failure", -5: "device wait timed out", -6: "CUDA error"}

EXPORTS = ["ptn_default_options", "ptn_solver_create", "ptn_solver_destroy", "ptn_last_error",
           "ptn_set_options", "ptn_solve_ip", "ptn_solve_admm", "ptn_solve_batch", "ptn_adjoint",
           "ptn_num_rows", "ptn_version", "ptn_solve_ip_static", "ptn_batch_prepare",
           "ptn_solve_batch_async", "ptn_model_dims", "ptn_adjoint_checkpointed", "ptn_set_reference",
           "ptn_arith_check"]

_P = C.POINTER(C.c_double)


class Problem(C.Structure):
    _fields_ = [("model", C.c_int), ("nx", C.c_int), ("nu", C.c_int), ("integrator", C.c_int),
                ("dt", C.c_double), ("prm", C.c_double * 8),
                ("A", _P), ("B", _P), ("W", _P), ("Q", _P), ("R", _P), ("Qf", _P),
                ("xref", _P), ("uref", _P), ("xlo", _P), ("xhi", _P), ("ulo", _P), ("uhi", _P)]


_OPT_INTS = ["precision", "max_newton", "max_outer", "ls_count", "admm_fixed_iters", "roll_max_iter",
             "block_threads", "grid_min_T", "grid_steps_per_thread", "polish_after",
             "cluster_max_blocks", "sequential", "costate_mode", "update_mode"]
_OPT_DBLS = ["mu0", "zeta", "mu_final", "tol_inner", "tol_final", "rho", "admm_tol", "alpha0",
             "alpha_min", "alpha_max", "ls_beta", "armijo_c1", "armijo_eps", "roll_tol", "polish",
             "armijo_eps32"]


_OPT_TAIL = ["fp64_finish", "pad_opt"]


class Options(C.Structure):
    _fields_ = [(k, C.c_int) for k in _OPT_INTS] + [(k, C.c_double) for k in _OPT_DBLS] + \
               [(k, C.c_int) for k in _OPT_TAIL]


class Info(C.Structure):
    _fields_ = [(k, C.c_int) for k in ["status", "newton_iters", "outer_iters", "ls_rejects",
                                       "factor_fails", "roll_fails", "roll_iters", "ls_evals",
                                       "exact_passes", "finish_iters"]] + \
               [(k, C.c_double) for k in ["mu", "alpha", "r_stat", "r_dyn", "r_feas", "r_kkt", "J",
                                          "J_c", "r_p", "r_d"]] + \
               [("cycles", C.c_longlong * 7)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "cycles"}
        d["cycles"] = list(self.cycles)
        return d


_lib = None


def _open(path: str):
    if not os.path.exists(path):
        raise OSError(f"libptn.so not found at {path}: run paper_2409_20027_gb300.build.build()")
    return C.CDLL(path)


def load(path: str = LIB_PATH):
    """Load libptn.so; raises OSError when it has not been built (no CPU fallback)."""
    global _lib
    if _lib is None:
        lib = _open(path)
        vp, ip = C.c_void_p, C.POINTER(C.c_int)
        lib.ptn_default_options.argtypes = [C.POINTER(Options)]
        lib.ptn_solver_create.argtypes = [C.POINTER(Problem), C.POINTER(Options), C.c_int, C.c_int, C.POINTER(vp)]
        lib.ptn_solver_destroy.argtypes = [vp]
        lib.ptn_last_error.argtypes = [vp]
        lib.ptn_last_error.restype = C.c_char_p
        lib.ptn_set_options.argtypes = [vp, C.POINTER(Options)]
        lib.ptn_solve_ip.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp, C.POINTER(Info), vp]
        lib.ptn_solve_admm.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp, vp, vp, C.POINTER(Info), vp]
        lib.ptn_solve_batch.argtypes = [vp, C.c_int, C.c_int, ip, C.POINTER(C.c_double), vp, vp, vp, vp, vp, vp,
                                         C.POINTER(Info), vp]
        lib.ptn_adjoint.argtypes = [vp, C.c_int, ip, vp, vp, vp, vp, C.c_double, C.c_double, vp, vp, vp, vp,
                                    vp, vp, vp, vp]
        lib.ptn_adjoint_checkpointed.argtypes = [vp, C.c_int, C.c_int, vp, vp, vp, vp, C.c_double, C.c_double, vp,
                                                 vp, vp, vp, vp, vp, vp, vp]
        lib.ptn_set_reference.argtypes = [vp, vp, vp]
        lib.ptn_num_rows.argtypes = [vp]
        lib.ptn_solve_ip_static.argtypes = [C.POINTER(Problem), C.POINTER(Options), vp, vp, C.c_int, vp, vp, vp,
                                            C.POINTER(Info), C.c_char_p, C.c_int, vp]
        lib.ptn_batch_prepare.argtypes = [vp, C.c_int, C.c_int, ip, C.POINTER(C.c_double), vp]
        lib.ptn_solve_batch_async.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.ptn_model_dims.argtypes = [C.c_int, ip, ip]
        lib.ptn_arith_check.argtypes = [C.c_int, vp, vp, vp, vp, vp, vp, vp]
        lib.ptn_version.restype = C.c_char_p
        _lib = lib
    return _lib


def default_options(**kw) -> Options:
    o = Options()
    load().ptn_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class PtnError(RuntimeError):
    pass


def _dptr(t):
    """Device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _check_buf(t, numel, name, min_only=False):
    """Refuse a buffer that the kernel would read or write out of bounds, or that lives on
    another device than the current one (None passes: the argument is optional)."""
    if t is None:
        return
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{torch.cuda.current_device()}")
    n = t.numel()
    if n < numel if min_only else n != numel:
        raise ValueError(f"{name} has {n} elements, expected {numel}")


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Solver:
    """A solver handle for one problem (model, weights, bounds), owning its workspace."""

    def __init__(self, prob, max_T: int, max_batch: int = 1, options: Options | None = None, **opt):
        lib = load()
        self._keep = []
        P = Problem()
        P.model, P.nx, P.nu, P.integrator = int(prob.model), int(prob.nx), int(prob.nu), int(prob.integrator)
        P.dt = float(prob.dt)
        prm = np.zeros(8)
        prm[:len(prob.prm)] = prob.prm
        for i in range(8):
            P.prm[i] = prm[i]
        for name in ["A", "B", "W", "Q", "R", "Qf", "xref", "uref", "xlo", "xhi", "ulo", "uhi"]:
            v = getattr(prob, name, None)
            if v is None:
                setattr(P, name, None)
            else:
                a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel())
                self._keep.append(a)
                setattr(P, name, a.ctypes.data_as(_P))
        self.options = options if options is not None else default_options(**opt)
        h = C.c_void_p()
        rc = lib.ptn_solver_create(C.byref(P), C.byref(self.options), int(max_T), int(max_batch), C.byref(h))
        self._h = h
        if rc != 0:
            msg = lib.ptn_last_error(h).decode() if h.value else ""
            lib.ptn_solver_destroy(h)
            self._h = C.c_void_p()
            raise PtnError(f"ptn_solver_create failed ({rc}): {msg}")
        self.nx, self.nu = P.nx, P.nu
        self.nw = lib.ptn_num_rows(h)
        self.prob = prob

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().ptn_solver_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        rc = load().ptn_set_options(self._h, C.byref(self.options))
        if rc != 0:
            raise PtnError(self.last_error())

    def set_reference(self, xref_traj=None, uref_traj=None):
        """Time-varying targets for the following solves (ptn_set_reference): contiguous
        float64 CUDA tensors laid out like the state / control outputs of those solves, or
        None.  The solver keeps references to the tensors."""
        for a in (xref_traj, uref_traj):
            if a is not None and (not a.is_cuda or a.dtype.itemsize != 8 or not a.is_contiguous()):
                raise ValueError("targets must be contiguous float64 CUDA tensors")
        self._refs = (xref_traj, uref_traj)
        rc = load().ptn_set_reference(self._h, _dptr(xref_traj), _dptr(uref_traj))
        if rc != 0:
            raise PtnError(self.last_error())

    def last_error(self) -> str:
        return load().ptn_last_error(self._h).decode()

    def _out(self, rows, cols, like):
        import torch
        return torch.empty((rows, cols), dtype=torch.float64, device=like.device)

    def solve_ip(self, x0, T: int, u_init=None, x_out=None, u_out=None, lam_out=None, stream=None):
        """IP solve (Sec. II-B).  Returns (x, u, lam, info dict)."""
        x_out = self._out(T + 1, self.nx, x0) if x_out is None else x_out
        u_out = self._out(T, self.nu, x0) if u_out is None else u_out
        lam_out = self._out(T + 1, self.nx, x0) if lam_out is None else lam_out
        _check_solve_bufs(T, self.nx, self.nu, x0, u_init, x_out, u_out, lam_out)
        info = Info()
        rc = load().ptn_solve_ip(self._h, _dptr(x0), _dptr(u_init), int(T), _dptr(x_out), _dptr(u_out),
                                 _dptr(lam_out), C.byref(info), _stream(stream))
        self._raise_unsolved(rc, "ptn_solve_ip")
        return x_out, u_out, lam_out, info.as_dict()

    def _raise_unsolved(self, rc, name):
        # refused before any solve ran (argument checks, CUDA errors): no report was written
        if rc in (PTN_ERR_INVALID_ARG, PTN_ERR_CUDA):
            raise PtnError(f"{name}: {self.last_error()} ({rc})")

    def solve_admm(self, x0, T: int, u_init=None, stream=None, with_zv=False):
        """ADMM solve (Sec. II-C).  Returns (x, u, lam, info) or with z, v."""
        x = self._out(T + 1, self.nx, x0)
        u = self._out(T, self.nu, x0)
        lam = self._out(T + 1, self.nx, x0)
        z = self._out(T, max(self.nw, 1), x0) if with_zv else None
        v = self._out(T, max(self.nw, 1), x0) if with_zv else None
        info = Info()
        rc = load().ptn_solve_admm(self._h, _dptr(x0), _dptr(u_init), int(T), _dptr(x), _dptr(u), _dptr(lam),
                                   _dptr(z), _dptr(v), C.byref(info), _stream(stream))
        self._raise_unsolved(rc, "ptn_solve_admm")
        if with_zv:
            return x, u, lam, z, v, info.as_dict()
        return x, u, lam, info.as_dict()

    def solve_batch(self, x0, T_b, xref=None, u_init=None, method: int = METHOD_IP, x_out=None, u_out=None,
                    lam_out=None, stream=None, dt_b=None):
        """B instances in one launch.  x0: (B, nx) CUDA tensor, T_b: int sequence, dt_b:
        optional per-instance time steps (stage weights scaled by dt_b / prob.dt).
        Returns (x, u, lam, infos) with concatenated trajectories."""
        Tb = np.ascontiguousarray(np.asarray(T_b, dtype=np.int32))
        B = len(Tb)
        dtb = None if dt_b is None else np.ascontiguousarray(np.asarray(dt_b, dtype=np.float64))
        if dtb is not None and dtb.shape != (B,):
            raise ValueError("dt_b must have one entry per instance")
        S = int(Tb.sum())
        x_out = self._out(S + B, self.nx, x0) if x_out is None else x_out
        u_out = self._out(S, self.nu, x0) if u_out is None else u_out
        lam_out = self._out(S + B, self.nx, x0) if lam_out is None else lam_out
        infos = (Info * B)()
        rc = load().ptn_solve_batch(self._h, int(method), B, Tb.ctypes.data_as(C.POINTER(C.c_int)),
                                    None if dtb is None else dtb.ctypes.data_as(C.POINTER(C.c_double)), _dptr(x0),
                                    _dptr(xref), _dptr(u_init), _dptr(x_out), _dptr(u_out), _dptr(lam_out), infos,
                                    _stream(stream))
        self._raise_unsolved(rc, "ptn_solve_batch")
        return x_out, u_out, lam_out, [i.as_dict() for i in infos]

    def prepare_batch(self, T_b, method: int = METHOD_IP, dt_b=None, stream=None):
        """Fix a batch layout (horizons, time steps, method) and its launch shape for
        solve_batch_async; synchronises the stream.  Raises PtnError on invalid input."""
        self._prepared = None
        Tb = np.ascontiguousarray(np.asarray(T_b, dtype=np.int32))
        B = len(Tb)
        dtb = None if dt_b is None else np.ascontiguousarray(np.asarray(dt_b, dtype=np.float64))
        if dtb is not None and dtb.shape != (B,):
            raise ValueError("dt_b must have one entry per instance")
        rc = load().ptn_batch_prepare(self._h, int(method), B, Tb.ctypes.data_as(C.POINTER(C.c_int)),
                                      None if dtb is None else dtb.ctypes.data_as(C.POINTER(C.c_double)),
                                      _stream(stream))
        if rc != 0:
            raise PtnError(f"ptn_batch_prepare: {self.last_error()} ({rc})")
        self._prepared = (B, int(Tb.sum()))

    def new_info_buffer(self, B: int, device="cuda"):
        """Device buffer for B ptn_info records (solve_batch_async's info_dev)."""
        import torch
        return torch.zeros(B * C.sizeof(Info), dtype=torch.uint8, device=device)

    def solve_batch_async(self, x0, xref=None, u_init=None, x_out=None, u_out=None, lam_out=None,
                          info_dev=None, stream=None):
        """Enqueue a solve of the prepared batch without waiting (graph-capturable: kernel
        launches only).  Outputs are allocated when not given (inside a capture they come
        from the graph's pool).  Returns (x, u, lam, info_dev); decode info_dev with
        infos_from_device once the stream has passed the solve."""
        if getattr(self, "_prepared", None) is None:
            raise PtnError("no batch prepared (prepare_batch)")
        B, S = self._prepared
        x_out = self._out(S + B, self.nx, x0) if x_out is None else x_out
        u_out = self._out(S, self.nu, x0) if u_out is None else u_out
        lam_out = self._out(S + B, self.nx, x0) if lam_out is None else lam_out
        info_dev = self.new_info_buffer(B, x0.device) if info_dev is None else info_dev
        if info_dev.numel() < B * C.sizeof(Info) or not info_dev.is_cuda or not info_dev.is_contiguous():
            raise ValueError("info_dev must be a contiguous CUDA buffer of B ptn_info records")
        rc = load().ptn_solve_batch_async(self._h, _dptr(x0), _dptr(xref), _dptr(u_init), _dptr(x_out),
                                          _dptr(u_out), _dptr(lam_out), C.c_void_p(info_dev.data_ptr()),
                                          _stream(stream))
        if rc != 0:
            raise PtnError(f"ptn_solve_batch_async: {self.last_error()} ({rc})")
        return x_out, u_out, lam_out, info_dev

    def adjoint(self, T_b, x0, x_star, u_star, mu: float, gJ: float = 1.0, gx=None, gu=None, xref=None,
                stream=None):
        """Gradients of gJ J* + <gx, x*> + <gu, u*> w.r.t. x0, diag Q, diag R, diag Qf, prm."""
        import torch
        Tb = np.ascontiguousarray(np.asarray(T_b, dtype=np.int32))
        B = len(Tb)
        dev = x_star.device
        out = {k: torch.zeros((B, c), dtype=torch.float64, device=dev)
               for k, c in [("x0", self.nx), ("Qd", self.nx), ("Rd", self.nu), ("Qfd", self.nx), ("prm", 8)]}
        rc = load().ptn_adjoint(self._h, B, Tb.ctypes.data_as(C.POINTER(C.c_int)), _dptr(x0), _dptr(xref),
                                _dptr(x_star), _dptr(u_star), float(mu), float(gJ), _dptr(gx), _dptr(gu),
                                _dptr(out["x0"]), _dptr(out["Qd"]), _dptr(out["Rd"]), _dptr(out["Qfd"]),
                                _dptr(out["prm"]), _stream(stream))
        if rc != 0:
            raise PtnError(f"ptn_adjoint failed ({rc}): {self.last_error()}")
        return out

    def adjoint_checkpointed(self, T: int, seg_len: int, x0, x_star, u_star, mu: float, gJ: float = 1.0, gx=None,
                             gu=None, xref=None, stream=None):
        """adjoint() of one instance whose horizon T may exceed the workspace: segments of
        seg_len steps, linearisations recomputed from the trajectory in each sweep."""
        import torch
        dev = x_star.device
        out = {k: torch.zeros((1, c), dtype=torch.float64, device=dev)
               for k, c in [("x0", self.nx), ("Qd", self.nx), ("Rd", self.nu), ("Qfd", self.nx), ("prm", 8)]}
        for a, rows, cols in [(x_star, T + 1, self.nx), (u_star, T, self.nu), (gx, T + 1, self.nx), (gu, T, self.nu)]:
            if a is not None and (a.numel() != rows * cols or not a.is_contiguous() or a.device != dev):
                raise ValueError("x_star, u_star, gx, gu: contiguous (T+1) x nx / T x nu on the solver's device")
        rc = load().ptn_adjoint_checkpointed(self._h, int(T), int(seg_len), _dptr(x0), _dptr(xref), _dptr(x_star),
                                             _dptr(u_star), float(mu), float(gJ), _dptr(gx), _dptr(gu),
                                             _dptr(out["x0"]), _dptr(out["Qd"]), _dptr(out["Rd"]),
                                             _dptr(out["Qfd"]), _dptr(out["prm"]), _stream(stream))
        if rc != 0:
            raise PtnError(f"ptn_adjoint_checkpointed failed ({rc}): {self.last_error()}")
        return out


def model_dims(model: int):
    """(nx, nu) of a model id known to the loaded library (built-in or user-registered),
    or None."""
    nx, nu = C.c_int(), C.c_int()
    rc = load().ptn_model_dims(int(model), C.byref(nx), C.byref(nu))
    return (nx.value, nu.value) if rc == 0 else None


def arith_check(p=None, f=None, d=None, stream=None):
    """ptn_arith_check: the kernels' pivot reciprocal of p (FP64), FP32 -> FP64 widening of
    f and FP64 -> FP32 rounding of d, each a 1-D contiguous CUDA tensor (or None).  Returns
    (rcp, f2d, d2f), None where the input was None; synchronises the stream."""
    import torch
    ns = {len(t) for t in (p, f, d) if t is not None}
    if len(ns) != 1:
        raise ValueError("give at least one input; all inputs have the same length")
    n = ns.pop()
    for t, dt, name in ((p, torch.float64, "p"), (f, torch.float32, "f"), (d, torch.float64, "d")):
        if t is not None and (not t.is_cuda or t.dtype != dt or not t.is_contiguous() or t.dim() != 1):
            raise ValueError(f"{name}: a 1-D contiguous CUDA {dt} tensor")
    out = lambda t, dt: None if t is None else torch.empty(n, dtype=dt, device=t.device)
    rcp, f2d, d2f = out(p, torch.float64), out(f, torch.float64), out(d, torch.float32)
    ptr = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    rc = load().ptn_arith_check(n, ptr(p), ptr(rcp), ptr(f), ptr(f2d), ptr(d), ptr(d2f), _stream(stream))
    if rc != 0:
        raise PtnError(f"ptn_arith_check failed ({rc})")
    torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    return rcp, f2d, d2f


def infos_from_device(info_dev, B: int):
    """Decode B ptn_info records from a device (or host) byte buffer into dicts (copies to
    the host, so it waits for the work that writes them)."""
    raw = info_dev[: B * C.sizeof(Info)].cpu().numpy().tobytes()
    return [r.as_dict() for r in (Info * B).from_buffer_copy(raw)]


def status_view(info_dev, B: int):
    """(B, 2) int32 device view of the status and Newton-iteration fields of the records."""
    import torch
    return info_dev[: B * C.sizeof(Info)].view(-1).view(torch.int32).reshape(B, -1)[:, :2]


def _check_solve_bufs(T, nx, nu, x0, u_init, x_out, u_out, lam_out):
    """Sizes and device of a single solve's buffers (x0: nx, u_init: T*nu, x_out and
    lam_out: (T+1)*nx, u_out: T*nu)."""
    T = int(T)
    if T < 1:
        return  # the library reports the invalid horizon
    _check_buf(x0, nx, "x0")
    _check_buf(u_init, T * nu, "u_init")
    _check_buf(x_out, (T + 1) * nx, "x_out")
    _check_buf(u_out, T * nu, "u_out")
    _check_buf(lam_out, (T + 1) * nx, "lam_out")


def _make_problem(prob):
    """ptn_problem record for `prob`; returns (record, arrays it points into)."""
    keep = []
    P = Problem()
    P.model, P.nx, P.nu, P.integrator = int(prob.model), int(prob.nx), int(prob.nu), int(prob.integrator)
    P.dt = float(prob.dt)
    prm = np.zeros(8)
    prm[:len(prob.prm)] = prob.prm
    for i in range(8):
        P.prm[i] = prm[i]
    for name in ["A", "B", "W", "Q", "R", "Qf", "xref", "uref", "xlo", "xhi", "ulo", "uhi"]:
        v = getattr(prob, name, None)
        if v is None:
            setattr(P, name, None)
        else:
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64).ravel())
            keep.append(a)
            setattr(P, name, a.ctypes.data_as(_P))
    return P, keep


def solve_ip_static(prob, x0, T: int, u_init=None, x_out=None, u_out=None, lam_out=None,
                    options: Options | None = None, stream=None, **opt):
    """ptn_solve_ip_static: one IP solve with no handle and no device allocation by the
    library (workspace in a fixed 4 MiB device array shared by all calls on a device).
    Output tensors are allocated here unless given.  Returns (x, u, lam, info); raises
    PtnError for invalid arguments and CUDA errors, like a handle's create would."""
    lib = load()
    P, keep = _make_problem(prob)
    o = options if options is not None else default_options(**opt)
    nx, nu = int(prob.nx), int(prob.nu)
    import torch
    mk = lambda r, c: torch.empty((r, c), dtype=torch.float64, device=x0.device)
    x_out = mk(T + 1, nx) if x_out is None else x_out
    u_out = mk(T, nu) if u_out is None else u_out
    lam_out = mk(T + 1, nx) if lam_out is None else lam_out
    _check_solve_bufs(T, nx, nu, x0, u_init, x_out, u_out, lam_out)
    info = Info()
    err = C.create_string_buffer(512)
    rc = lib.ptn_solve_ip_static(C.byref(P), C.byref(o), _dptr(x0), _dptr(u_init), int(T), _dptr(x_out),
                                 _dptr(u_out), _dptr(lam_out), C.byref(info), err, 512, _stream(stream))
    del keep
    if rc in (PTN_ERR_INVALID_ARG, PTN_ERR_CUDA):
        raise PtnError(f"ptn_solve_ip_static failed ({rc}): {err.value.decode()}")
    return x_out, u_out, lam_out, info.as_dict()


def theta_of(prob):
    """Parameter vector [diag Q, diag R, diag Qf, prm (8)] of a problem, as the adjoint
    orders its gradients."""
    prm = np.zeros(8)
    prm[:len(prob.prm)] = prob.prm
    return np.concatenate([np.diag(np.asarray(prob.Q, dtype=np.float64)),
                           np.diag(np.asarray(prob.R, dtype=np.float64).reshape(prob.nu, prob.nu)),
                           np.diag(np.asarray(prob.Qf, dtype=np.float64)), prm])


def _solve_ip_function():
    import torch

    class SolveIP(torch.autograd.Function):
        """Batched IP solve with gradients from ptn_adjoint (Sec. II-B solution, KKT adjoint).

        forward(x0 (B, nx), theta, solver, T_b, xref) -> (x*, u*, J*): concatenated
        trajectories as in solve_batch and J* (B,), the barrier objective at mu_final.
        theta must equal theta_of(solver.prob) (the solver's own parameters; anything
        else raises ValueError); it is an input only so that autograd can route
        d loss / d theta to it."""

        @staticmethod
        def forward(ctx, x0, theta, solver, T_b, xref):
            want = theta_of(solver.prob)
            got = theta.detach().to("cpu", torch.float64).reshape(-1).numpy()
            if got.shape != want.shape or not np.array_equal(got, want):
                raise ValueError("theta must equal theta_of(solver.prob): the solve and its gradients use the "
                                 "solver's own parameters; build a Solver for other parameters")
            x, u, _, infos = solver.solve_batch(x0.detach().contiguous(), T_b, xref=xref)
            bad = [(i, f["status"]) for i, f in enumerate(infos) if f["status"] != 0]
            if bad:
                raise PtnError(f"solve failed for instances {bad}: {solver.last_error()}")
            J = torch.tensor([f["J_c"] for f in infos], dtype=torch.float64, device=x0.device)
            ctx.solver, ctx.T_b, ctx.xref, ctx.mu = solver, list(T_b), xref, infos[0]["mu"]
            ctx.save_for_backward(x0.detach(), x, u)
            return x, u, J

        @staticmethod
        def backward(ctx, gx, gu, gJ):
            x0, x, u = ctx.saved_tensors
            s = ctx.solver
            B = len(ctx.T_b)
            # the adjoint is linear in (gJ, gx, gu): one call for the trajectory part and,
            # since gJ differs per instance, one envelope call with gJ = 1 scaled per row
            lin = s.adjoint(ctx.T_b, x0, x, u, ctx.mu, 0.0,
                            None if gx is None else gx.contiguous(), None if gu is None else gu.contiguous(),
                            xref=ctx.xref) if (gx is not None or gu is not None) else None
            env = s.adjoint(ctx.T_b, x0, x, u, ctx.mu, 1.0, xref=ctx.xref) if gJ is not None else None
            tot = {}
            for k in ["x0", "Qd", "Rd", "Qfd", "prm"]:
                v = torch.zeros_like((lin or env)[k])
                if lin is not None:
                    v = v + lin[k]
                if env is not None:
                    v = v + gJ.reshape(B, 1) * env[k]
                tot[k] = v
            g_theta = torch.cat([tot["Qd"], tot["Rd"], tot["Qfd"], tot["prm"]], dim=1).sum(0)
            return tot["x0"], g_theta, None, None, None

    return SolveIP


_SOLVE_IP = None


def solve_ip_autograd(solver, x0, T_b, theta=None, xref=None):
    """Differentiable batched IP solve: (x*, u*, J*) with gradients to x0 and theta."""
    global _SOLVE_IP
    import torch
    if _SOLVE_IP is None:
        _SOLVE_IP = _solve_ip_function()
    if theta is None:
        theta = torch.tensor(theta_of(solver.prob), dtype=torch.float64, device=x0.device)
    return _SOLVE_IP.apply(x0, theta, solver, T_b, xref)
