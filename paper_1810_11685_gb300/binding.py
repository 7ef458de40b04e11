"""ctypes binding of ``include/qpat.h`` (argument marshalling only).

Every function here converts torch tensors to raw device pointers and calls
the entry point of the same name in ``libqpat.so``; all arithmetic runs in
the library's CUDA kernels.  Outputs are allocated with torch on the tensor's
device, and each call enqueues on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_PKG)
_LIB_PATH = os.path.join(_PKG, "libqpat.so")
_HEADER = os.path.join(_ROOT, "include", "qpat.h")

STATUS = {0: "QPAT_OK", 1: "QPAT_EINVAL", 2: "QPAT_EUNSTABLE", 3: "QPAT_ENONFINITE",
          4: "QPAT_ENOCONV", 5: "QPAT_ETIMEOUT", 6: "QPAT_ENOMEM", 7: "QPAT_ECUDA"}
FP64, FP32 = 0, 1
# internal pass ids of the propagation kernels (csrc/qpat_internal.h, enum Phase)
PHASES = {"F_R1": 0, "F_R2": 1, "F_R3": 2, "F_R3L": 3, "F_C1": 10, "F_C2": 11, "F_C3": 12,
          "A_R1": 20, "A_R1L": 21, "A_R3": 22, "A_R5": 23, "A_C2": 30, "A_C4": 31, "A_C6": 32}


class QpatError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class qpat_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 2), ("pml", ctypes.c_int), ("dx", ctypes.c_double),
                ("dt", ctypes.c_double), ("nt", ctypes.c_int), ("c_ref", ctypes.c_double),
                ("pml_alpha", ctypes.c_double), ("y", ctypes.c_double), ("lossless", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("gamma_d", ctypes.c_double),
                ("pcg_max_iter", ctypes.c_int), ("pcg_tol", ctypes.c_double),
                ("generic_fft", ctypes.c_int), ("no_graphs", ctypes.c_int), ("n2", ctypes.c_int),
                ("da_jacobi", ctypes.c_int)]


class qpat_medium(ctypes.Structure):
    _fields_ = [("c", ctypes.c_void_p), ("rho", ctypes.c_void_p), ("alpha0_db", ctypes.c_void_p),
                ("kappa", ctypes.c_void_p)]


class qpat_group_shape(ctypes.Structure):
    _fields_ = [("multi", ctypes.c_int), ("row_block", ctypes.c_int), ("col_block", ctypes.c_int),
                ("largest_first", ctypes.c_int)]


class qpat_ld_params(ctypes.Structure):
    _fields_ = [("k_max", ctypes.c_int), ("i_max", ctypes.c_int), ("i_m", ctypes.c_int),
                ("tol_in", ctypes.c_double), ("tol_out", ctypes.c_double), ("gamma", ctypes.c_double),
                ("beta", ctypes.c_double), ("tv_edge", ctypes.c_double), ("tv_max_iter", ctypes.c_int),
                ("tv_tol", ctypes.c_double), ("method", ctypes.c_int), ("kp_max", ctypes.c_int),
                ("tol_med", ctypes.c_double), ("lbfgs_m", ctypes.c_int), ("j_max", ctypes.c_int),
                ("ls_max", ctypes.c_int), ("c1", ctypes.c_double), ("c2", ctypes.c_double),
                ("tau", ctypes.c_double), ("rho", ctypes.c_double), ("nu", ctypes.c_double),
                ("lower", ctypes.c_double), ("upper", ctypes.c_double)]


class qpat_ld_info(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int), ("inner_total", ctypes.c_int), ("sub_total", ctypes.c_int),
                ("tv_iters", ctypes.c_longlong),
                ("products", ctypes.c_longlong), ("eps_first", ctypes.c_double), ("eps_last", ctypes.c_double),
                ("seconds", ctypes.c_double * 3)]


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load libqpat.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "qpat_create": [ctypes.POINTER(qpat_config), ctypes.POINTER(qpat_medium), vp, i, i, vp,
                        ctypes.POINTER(vp)],
        "qpat_destroy": [vp],
        "qpat_set_stream": [vp, vp],
        "qpat_get_sizes": [vp, ctypes.POINTER(ll)],
        "qpat_sync": [vp],
        "qpat_acoustic_forward": [vp, i, vp, vp],
        "qpat_acoustic_adjoint": [vp, i, vp, vp],
        "qpat_da_solve": [vp, i, vp, ctypes.c_uint, vp],
        "qpat_forward": [vp, i, vp, ctypes.c_uint, vp, vp],
        "qpat_jvp": [vp, i, vp, vp, vp, ctypes.c_uint, vp],
        "qpat_vjp": [vp, i, vp, vp, vp, ctypes.c_uint, vp],
        "qpat_dot": [vp, i, ll, vp, vp, ctypes.POINTER(d)],
        "qpat_get_stats": [vp, ctypes.POINTER(ll)],
        "qpat_ckpt_bytes": [vp, i, i, ctypes.POINTER(ll)],
        "qpat_group_create": [i, vp, ctypes.POINTER(vp)],
        "qpat_group_destroy": [vp],
        "qpat_group_propagate": [vp, i, vp, vp, vp, vp],
        "qpat_group_jvp": [vp, vp, vp, vp, vp, ctypes.c_uint, vp, vp],
        "qpat_autotune": [vp, i, i, ctypes.POINTER(i)],
        "qpat_group_set_shape": [vp, ctypes.POINTER(qpat_group_shape)],
        "qpat_group_get_shape": [vp, ctypes.POINTER(qpat_group_shape), ctypes.POINTER(i), vp],
        "qpat_group_tune": [vp, vp, i, vp, ctypes.POINTER(qpat_group_shape), ctypes.POINTER(d),
                            ctypes.POINTER(i)],
        "qpat_acoustic_forward_ckpt": [vp, i, vp, vp, i, vp],
        "qpat_acoustic_resume": [vp, i, vp, i, i, vp],
        "qpat_profile": [vp, i],
        "qpat_profile_read": [vp, ctypes.POINTER(d), ctypes.POINTER(ll)],
        "qpat_ld_solve": [vp, i, vp, vp, vp, vp, ctypes.POINTER(qpat_ld_params), ctypes.POINTER(qpat_ld_info),
                          ctypes.POINTER(d), ctypes.POINTER(i)],
        "qpat_tv_apply": [vp, vp, d, d, d, vp, vp],
        "qpat_set_kappa": [vp, vp],
        "qpat_jvp_kappa": [vp, i, vp, vp, vp, ctypes.c_uint, vp],
        "qpat_vjp_kappa": [vp, i, vp, vp, vp, ctypes.c_uint, vp],
        "qpat_jvp_medium": [vp, vp, vp, vp, vp],
        "qpat_vjp_medium": [vp, vp, vp, vp, vp],
        "qpat_set_medium_checkpoints": [vp, i],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.qpat_last_error.argtypes = [vp]
    lib.qpat_last_error.restype = ctypes.c_char_p
    lib.qpat_barrier_check.argtypes = [i, i, i, d, vp, ctypes.POINTER(i)]
    lib.qpat_barrier_check.restype = ctypes.c_int
    lib.qpat_dot_noalloc.argtypes = [i, i, ll, vp, vp, vp, vp]
    lib.qpat_dot_noalloc.restype = ctypes.c_int
    lib.qpat_noalloc_last_error.argtypes = []
    lib.qpat_noalloc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def exported_symbols():
    """Names of every entry point declared in include/qpat.h."""
    text = open(_HEADER).read()
    return sorted(set(re.findall(r"\b(qpat_[a-z_0-9]+)\s*\(", text)))


def _check(ctx_ptr, status):
    if status != 0:
        msg = load().qpat_last_error(ctx_ptr) if ctx_ptr else b""
        raise QpatError(status, (msg or b"").decode())


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _host(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Context:
    """Owns a ``qpat_ctx``: medium, sensors, grid and workspace on one GPU."""

    def __init__(self, c, rho, alpha0_db, kappa, sensors, *, dx, dt, nt, pml, y=1.5, lossless=False,
                 precision="fp32", max_batch=1, c_ref=0.0, pml_alpha=0.0, gamma_d=0.0,
                 pcg_max_iter=0, pcg_tol=0.0, generic_fft=False, no_graphs=False,
                 da_precond="multigrid", device=None):
        import torch
        lib = load()
        c = _host(c)
        rho = _host(rho)
        kappa = _host(kappa)
        self.dim = c.ndim
        sensors = _host(sensors).reshape(-1, self.dim)
        self.grid_shape = c.shape
        self.interior_shape = kappa.shape
        self.ny, self.nx = c.shape[-2], c.shape[-1]
        self.n0, self.n1 = kappa.shape[-1], kappa.shape[-2]
        cfg = qpat_config()
        cfg.n[0], cfg.n[1] = self.n0, self.n1
        cfg.n2 = kappa.shape[0] if self.dim == 3 else 0
        cfg.pml, cfg.dx, cfg.dt, cfg.nt = int(pml), float(dx), float(dt), int(nt)
        cfg.c_ref, cfg.pml_alpha, cfg.y = float(c_ref), float(pml_alpha), float(y)
        cfg.lossless, cfg.max_batch = int(bool(lossless)), int(max_batch)
        cfg.gamma_d, cfg.pcg_max_iter, cfg.pcg_tol = float(gamma_d), int(pcg_max_iter), float(pcg_tol)
        cfg.generic_fft = int(bool(generic_fft))
        cfg.no_graphs = int(bool(no_graphs))
        if da_precond not in ("multigrid", "jacobi"):
            raise ValueError(f"da_precond must be 'multigrid' or 'jacobi', not {da_precond!r}")
        cfg.da_jacobi = int(da_precond == "jacobi")
        keep = [c, rho, kappa, sensors]
        al = None
        if not lossless:
            al = _host(alpha0_db)
            keep.append(al)
        med = qpat_medium(c.ctypes.data, rho.ctypes.data, None if al is None else al.ctypes.data,
                          kappa.ctypes.data)
        self.precision = precision
        self.dtype = torch.float32 if precision == "fp32" else torch.float64
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.nt, self.ns, self.max_batch = int(nt), sensors.shape[0], int(max_batch)
        self.N = int(np.prod(self.interior_shape))
        self.dx = float(dx)
        out = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream().cuda_stream
            st = lib.qpat_create(ctypes.byref(cfg), ctypes.byref(med), sensors.ctypes.data,
                                 sensors.shape[0], FP32 if precision == "fp32" else FP64,
                                 ctypes.c_void_p(stream), ctypes.byref(out))
        if st != 0:
            raise QpatError(st, "qpat_create failed (details on stderr)")
        self._ptr = out
        self._lib = lib

    # -- plumbing ---------------------------------------------------------
    def _stream(self):
        import torch
        _check(self._ptr, self._lib.qpat_set_stream(self._ptr, ctypes.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)))

    def _empty(self, *shape, dtype=None):
        import torch
        return torch.empty(*shape, dtype=dtype or self.dtype, device=self.device)

    def _in(self, t, dtype, shape_tail):
        import torch
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError("expected a CUDA tensor")
        if t.dtype != dtype:
            raise TypeError(f"expected {dtype}, got {t.dtype}")
        t = t.contiguous()
        if t.dim() == len(shape_tail):
            t = t.unsqueeze(0)
        if tuple(t.shape[1:]) != tuple(shape_tail):
            raise ValueError(f"expected trailing shape {shape_tail}, got {tuple(t.shape)}")
        return t

    @staticmethod
    def _one(t, name):
        """The single problem of a [1][...] tensor (entry points without a batch)."""
        if t.shape[0] != 1:
            raise ValueError(f"{name}: this entry point takes one problem, got a batch of {t.shape[0]}")
        return t[0]

    def close(self):
        if getattr(self, "_ptr", None):
            self._lib.qpat_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self):
        arr = (ctypes.c_longlong * 6)()
        _check(self._ptr, self._lib.qpat_get_sizes(self._ptr, arr))
        return list(arr)

    def sync(self):
        _check(self._ptr, self._lib.qpat_sync(self._ptr))

    def stats(self):
        arr = (ctypes.c_longlong * 3)()
        _check(self._ptr, self._lib.qpat_get_stats(self._ptr, arr))
        return {"launches": arr[0], "profiled": arr[1], "pcg_iterations": arr[2]}

    def profile(self, phase):
        """Bracket every launch of pass ``phase`` (name or id; None = off) with CUDA events."""
        pid = -1 if phase is None else (PHASES[phase] if isinstance(phase, str) else int(phase))
        _check(self._ptr, self._lib.qpat_profile(self._ptr, pid))

    def profile_read(self):
        """(summed device ms, launches) of the profiled pass; resets the profiler."""
        ms = ctypes.c_double()
        n = ctypes.c_longlong()
        _check(self._ptr, self._lib.qpat_profile_read(self._ptr, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    # -- entry points ----------------------------------------------------
    def acoustic_forward(self, p0, out=None):
        p0 = self._in(p0, self.dtype, self.interior_shape)
        B = p0.shape[0]
        out = self._empty(B, self.nt, self.ns) if out is None else out
        self._stream()
        _check(self._ptr, self._lib.qpat_acoustic_forward(self._ptr, B, _ptr(p0), _ptr(out)))
        return out

    def acoustic_adjoint(self, data, out=None):
        data = self._in(data, self.dtype, (self.nt, self.ns))
        B = data.shape[0]
        out = self._empty(B, *self.interior_shape) if out is None else out
        self._stream()
        _check(self._ptr, self._lib.qpat_acoustic_adjoint(self._ptr, B, _ptr(data), _ptr(out)))
        return out

    def ckpt_bytes(self, batch, K):
        n = ctypes.c_longlong()
        _check(self._ptr, self._lib.qpat_ckpt_bytes(self._ptr, int(batch), int(K), ctypes.byref(n)))
        return n.value

    def acoustic_forward_ckpt(self, p0, K, out=None):
        """H_a that also stores the forward state every K loop iterations;
        returns (data, checkpoint buffer)."""
        import torch
        p0 = self._in(p0, self.dtype, self.interior_shape)
        B = p0.shape[0]
        out = self._empty(B, self.nt, self.ns) if out is None else out
        ck = torch.empty(self.ckpt_bytes(B, K), dtype=torch.uint8, device=self.device)
        self._stream()
        _check(self._ptr, self._lib.qpat_acoustic_forward_ckpt(self._ptr, B, _ptr(p0), _ptr(out), int(K), _ptr(ck)))
        return out, ck

    def acoustic_resume(self, ckpt, K, m, batch, out=None):
        """Continue H_a from checkpoint m: fills samples (m+1)K .. nt-1 of ``out``."""
        out = self._empty(batch, self.nt, self.ns).zero_() if out is None else out
        self._stream()
        _check(self._ptr, self._lib.qpat_acoustic_resume(self._ptr, int(batch), _ptr(ckpt), int(K), int(m), _ptr(out)))
        return out

    def autotune(self, batch=1, steps=40):
        """Pick specialised vs generic passes per axis by timing; returns
        {"fast_rows": bool, "fast_cols": bool}."""
        ch = ctypes.c_int()
        self._stream()
        _check(self._ptr, self._lib.qpat_autotune(self._ptr, int(batch), int(steps), ctypes.byref(ch)))
        return {"fast_rows": bool(ch.value & 1), "fast_cols": bool(ch.value & 2)}

    def da_solve(self, mu, illum):
        import torch
        mu = self._in(mu, torch.float64, self.interior_shape)
        out = self._empty(mu.shape[0], *self.interior_shape, dtype=torch.float64)
        self._stream()
        _check(self._ptr, self._lib.qpat_da_solve(self._ptr, mu.shape[0], _ptr(mu), int(illum), _ptr(out)))
        return out

    def forward(self, mu, illum, return_phi=False):
        import torch
        mu = self._in(mu, torch.float64, self.interior_shape)
        B = mu.shape[0]
        out = self._empty(B, self.nt, self.ns)
        phi = self._empty(B, *self.interior_shape, dtype=torch.float64) if return_phi else None
        self._stream()
        _check(self._ptr, self._lib.qpat_forward(self._ptr, B, _ptr(mu), int(illum), _ptr(out), _ptr(phi)))
        return (out, phi) if return_phi else out

    def jvp(self, mu, dmu, illum, phi0=None):
        import torch
        mu = self._in(mu, torch.float64, self.interior_shape)
        dmu = self._in(dmu, torch.float64, self.interior_shape)
        if phi0 is not None:
            phi0 = self._in(phi0, torch.float64, self.interior_shape)
        B = dmu.shape[0]
        out = self._empty(B, self.nt, self.ns)
        self._stream()
        _check(self._ptr, self._lib.qpat_jvp(self._ptr, B, _ptr(mu), _ptr(phi0), _ptr(dmu), int(illum), _ptr(out)))
        return out

    def vjp(self, mu, w, illum, phi0=None):
        import torch
        mu = self._in(mu, torch.float64, self.interior_shape)
        w = self._in(w, self.dtype, (self.nt, self.ns))
        if phi0 is not None:
            phi0 = self._in(phi0, torch.float64, self.interior_shape)
        B = w.shape[0]
        out = self._empty(B, *self.interior_shape, dtype=torch.float64)
        self._stream()
        _check(self._ptr, self._lib.qpat_vjp(self._ptr, B, _ptr(mu), _ptr(phi0), _ptr(w), int(illum), _ptr(out)))
        return out

    def ld_solve(self, data, illums, mu0, kappa0=None, k_max=10, i_max=30, i_m=5, tol_in=0.0, tol_out=None,
                 gamma=1e-6, beta=2e-5, tv_edge=0.0, tv_max_iter=0, tv_tol=0.0, method="ld", kp_max=20,
                 tol_med=1e-3, lbfgs_m=5, j_max=10, ls_max=20, c1=1e-4, c2=0.9, tau=0.25, rho=1.0, nu=1e-3,
                 lower=1e-3, upper=1e3):
        """qpat_ld_solve: returns (mu, eps history, inner iterations per outer
        iteration, info dict), or ((kappa, mu), ...) when kappa0 is given
        (simultaneous reconstruction).  data: [nq][nt][ns] in the context
        precision; mu0, kappa0: FP64 interior fields (initial guesses).
        method: "ld" (Algorithm 5) or "pdipm" (Algorithm 6, with kp_max and
        tol_med), or "admm" (Algorithms 1-3, with lbfgs_m, j_max, ls_max,
        c1, c2, tau, rho, nu and the box [lower, upper] on Xbar; inner = L-BFGS
        iterations per ADMM iteration)."""
        import torch
        nq = len(illums)
        data = data.contiguous()
        if data.dtype != self.dtype or tuple(data.shape) != (nq, self.nt, self.ns) or data.device.type != "cuda":
            raise TypeError("data must be a CUDA tensor [nq][nt][ns] of the context precision")
        mu = self._in(mu0, torch.float64, self.interior_shape).clone()
        kappa = None if kappa0 is None else self._in(kappa0, torch.float64, self.interior_shape).clone()
        methods = {"ld": 0, "pdipm": 1, "admm": 2}
        if method not in methods:
            raise ValueError("method must be 'ld', 'pdipm' or 'admm'")
        if tol_out is None:
            tol_out = 1e-2 if method == "admm" else 1e-3
        prm = qpat_ld_params(k_max, i_max, i_m, tol_in, tol_out, gamma, beta, tv_edge, tv_max_iter, tv_tol,
                             methods[method], kp_max, tol_med, lbfgs_m, j_max, ls_max, c1, c2, tau, rho, nu,
                             lower, upper)
        info = qpat_ld_info()
        eps = (ctypes.c_double * (max(k_max, 1) + 1))()
        inner = (ctypes.c_int * max(k_max, 1))()
        ill = (ctypes.c_uint * nq)(*[int(q) for q in illums])
        self._stream()
        _check(self._ptr, self._lib.qpat_ld_solve(self._ptr, nq, ill, _ptr(data), _ptr(mu), _ptr(kappa),
                                                  ctypes.byref(prm), ctypes.byref(info), eps, inner))
        k = info.outer
        out = {f: getattr(info, f) for f, _ in qpat_ld_info._fields_}
        out["seconds"] = {"acoustic": info.seconds[0], "optical": info.seconds[1], "tv": info.seconds[2]}
        coeffs = mu[0] if kappa is None else (kappa[0], mu[0])
        return coeffs, list(eps)[:k + 1], list(inner)[:k], out

    def tv_apply(self, xbar, u, edge, beta, gamma):
        """qpat_tv_apply: M_gamma[xbar] u (FP64 interior fields)."""
        import torch
        xbar = self._in(xbar, torch.float64, self.interior_shape)
        u = self._in(u, torch.float64, self.interior_shape)
        out = torch.empty_like(u)
        self._stream()
        _check(self._ptr, self._lib.qpat_tv_apply(self._ptr, _ptr(xbar), float(edge), float(beta), float(gamma),
                                                  _ptr(u), _ptr(out)))
        return out[0]

    def set_kappa(self, kappa):
        """qpat_set_kappa: new optical diffusion (FP64 interior field)."""
        import torch
        kappa = self._in(kappa, torch.float64, self.interior_shape)
        self._stream()
        _check(self._ptr, self._lib.qpat_set_kappa(self._ptr, _ptr(kappa)))

    def jvp_kappa(self, mu, dkappa, illum, phi0=None):
        """qpat_jvp_kappa: H_a J_o dkappa."""
        import torch
        mu = self._in(mu, torch.float64, self.interior_shape)
        dkappa = self._in(dkappa, torch.float64, self.interior_shape)
        if phi0 is not None:
            phi0 = self._in(phi0, torch.float64, self.interior_shape)
        B = dkappa.shape[0]
        out = self._empty(B, self.nt, self.ns)
        self._stream()
        _check(self._ptr, self._lib.qpat_jvp_kappa(self._ptr, B, _ptr(mu), _ptr(phi0), _ptr(dkappa), int(illum),
                                                   _ptr(out)))
        return out

    def vjp_kappa(self, mu, w, illum, phi0=None):
        """qpat_vjp_kappa: J_o^* H_a^*(w) in kappa."""
        import torch
        mu = self._in(mu, torch.float64, self.interior_shape)
        w = self._in(w, self.dtype, (self.nt, self.ns))
        if phi0 is not None:
            phi0 = self._in(phi0, torch.float64, self.interior_shape)
        B = w.shape[0]
        out = self._empty(B, *self.interior_shape, dtype=torch.float64)
        self._stream()
        _check(self._ptr, self._lib.qpat_vjp_kappa(self._ptr, B, _ptr(mu), _ptr(phi0), _ptr(w), int(illum),
                                                   _ptr(out)))
        return out

    def jvp_medium(self, p0, dc=None, drho=None):
        """qpat_jvp_medium: J_c dc + J_rho drho at the interior initial
        pressure p0 (2D contexts; the sweep in the context precision, the
        buffers FP64); dc, drho on the full grid."""
        import torch
        p0 = self._one(self._in(p0, torch.float64, self.interior_shape), "p0")
        dc = None if dc is None else self._one(self._in(dc, torch.float64, self.grid_shape), "dc")
        drho = None if drho is None else self._one(self._in(drho, torch.float64, self.grid_shape), "drho")
        out = self._empty(self.nt, self.ns, dtype=torch.float64)
        self._stream()
        _check(self._ptr, self._lib.qpat_jvp_medium(self._ptr, _ptr(p0), _ptr(dc), _ptr(drho), _ptr(out)))
        return out

    def set_medium_checkpoints(self, K=0):
        """qpat_set_medium_checkpoints: checkpoint interval of vjp_medium (0: automatic)."""
        _check(self._ptr, self._lib.qpat_set_medium_checkpoints(self._ptr, int(K)))

    def vjp_medium(self, p0, w):
        """qpat_vjp_medium: (J_c^T w, J_rho^T w) on the full grid."""
        import torch
        p0 = self._one(self._in(p0, torch.float64, self.interior_shape), "p0")
        w = self._one(self._in(w, torch.float64, (self.nt, self.ns)), "w")
        g_c = self._empty(*self.grid_shape, dtype=torch.float64)
        g_rho = self._empty(*self.grid_shape, dtype=torch.float64)
        self._stream()
        _check(self._ptr, self._lib.qpat_vjp_medium(self._ptr, _ptr(p0), _ptr(w), _ptr(g_c), _ptr(g_rho)))
        return g_c, g_rho

    def dot(self, a, b):
        a = a.contiguous()
        b = b.contiguous()
        if a.dtype != self.dtype or b.dtype != self.dtype or a.shape != b.shape:
            raise TypeError("dot wants two tensors of the context precision and equal shape")
        B = a.shape[0] if a.dim() > 1 else 1
        L = a.numel() // B
        out = (ctypes.c_double * B)()
        self._stream()
        _check(self._ptr, self._lib.qpat_dot(self._ptr, B, L, _ptr(a), _ptr(b), out))
        return list(out)


class Group:
    """Several contexts (e.g. the uneven grids of a Newton inner loop)
    propagated concurrently in one captured CUDA graph (``qpat_group_*``)."""

    def __init__(self, ctxs):
        self._lib = load()
        self.ctxs = list(ctxs)
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c._ptr.value for c in self.ctxs])
        out = ctypes.c_void_p()
        _check(None, self._lib.qpat_group_create(len(self.ctxs), arr, ctypes.byref(out)))
        self._ptr = out

    def close(self):
        if getattr(self, "_ptr", None):
            self._lib.qpat_group_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _run(self, dir_, ins, outs):
        import torch
        n = len(self.ctxs)
        batches = (ctypes.c_int * n)(*[0 if t is None else t.shape[0] for t in ins])
        pin = (ctypes.c_void_p * n)(*[_ptr(t) for t in ins])
        pout = (ctypes.c_void_p * n)(*[_ptr(t) for t in outs])
        st = self._lib.qpat_group_propagate(self._ptr, dir_, batches, pin, pout,
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != 0:
            raise QpatError(st, self._lib.qpat_last_error(self.ctxs[0]._ptr).decode())
        return outs

    SHAPE_KEYS = ("multi", "row_block", "col_block", "largest_first")

    def set_shape(self, multi=1, row_block=144, col_block=576, largest_first=1):
        """qpat_group_set_shape (see include/qpat.h)."""
        sh = qpat_group_shape(int(multi), int(row_block), int(col_block), int(largest_first))
        _check(None, self._lib.qpat_group_set_shape(self._ptr, ctypes.byref(sh)))

    def shape(self, batches=None):
        """(shape dict, multi_ready) for members with work in ``batches``."""
        sh = qpat_group_shape()
        ready = ctypes.c_int()
        arr = None if batches is None else (ctypes.c_int * len(self.ctxs))(*[int(b) for b in batches])
        _check(None, self._lib.qpat_group_get_shape(self._ptr, ctypes.byref(sh), ctypes.byref(ready), arr))
        return {k: getattr(sh, k) for k in self.SHAPE_KEYS}, bool(ready.value)

    def tune(self, batches, steps=10):
        """qpat_group_tune: returns (best shape dict, [(shape dict, ms), ...])."""
        import torch
        n = len(self.ctxs)
        arr = (ctypes.c_int * n)(*[int(b) for b in batches])
        best = qpat_group_shape()
        ms = (ctypes.c_double * 16)()
        nc = ctypes.c_int()
        st = self._lib.qpat_group_tune(self._ptr, arr, int(steps),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                       ctypes.byref(best), ms, ctypes.byref(nc))
        if st != 0:
            raise QpatError(st, self._lib.qpat_last_error(self.ctxs[0]._ptr).decode())
        shapes = [(0, 144, 576, 1)] + [(1, rb, cb, lf) for rb in (144, 288) for cb in (288, 576) for lf in (1, 0)]
        cands = [(dict(zip(self.SHAPE_KEYS, sh)), ms[k]) for k, sh in enumerate(shapes[:nc.value])]
        return {k: getattr(best, k) for k in self.SHAPE_KEYS}, cands

    def acoustic_forward(self, p0s, outs=None):
        """H_a of every member: p0s[i] is [B_i][n1][n0] (or None to skip);
        outs[i] (optional) the [B_i][nt][ns] output."""
        ins = [None if p is None else c._in(p, c.dtype, c.interior_shape) for c, p in zip(self.ctxs, p0s)]
        if outs is None:
            outs = [None if p is None else c._empty(p.shape[0], c.nt, c.ns) for c, p in zip(self.ctxs, ins)]
        return self._run(0, ins, outs)

    def acoustic_adjoint(self, datas):
        ins = [None if d is None else c._in(d, c.dtype, (c.nt, c.ns)) for c, d in zip(self.ctxs, datas)]
        outs = [None if d is None else c._empty(d.shape[0], *c.interior_shape) for c, d in zip(self.ctxs, ins)]
        return self._run(1, ins, outs)

    def jvp(self, mus, dmus, illum, phi0s=None):
        import torch
        n = len(self.ctxs)
        mus = [c._in(m, torch.float64, c.interior_shape) for c, m in zip(self.ctxs, mus)]
        dmus = [c._in(d, torch.float64, c.interior_shape) for c, d in zip(self.ctxs, dmus)]
        phis = [None] * n if phi0s is None else [c._in(p, torch.float64, c.interior_shape) for c, p in zip(self.ctxs, phi0s)]
        outs = [c._empty(d.shape[0], c.nt, c.ns) for c, d in zip(self.ctxs, dmus)]
        arr = lambda ts: (ctypes.c_void_p * n)(*[_ptr(t) for t in ts])
        batches = (ctypes.c_int * n)(*[d.shape[0] for d in dmus])
        st = self._lib.qpat_group_jvp(self._ptr, batches, arr(mus), arr(phis) if phi0s is not None else None,
                                      arr(dmus), int(illum), arr(outs),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if st != 0:
            raise QpatError(st, self._lib.qpat_last_error(self.ctxs[0]._ptr).decode())
        return outs


# C-ABI-named wrappers -------------------------------------------------------
def qpat_create(*args, **kw) -> Context:
    return Context(*args, **kw)


def qpat_destroy(ctx: Context):
    ctx.close()


def qpat_acoustic_forward(ctx: Context, p0, out=None):
    return ctx.acoustic_forward(p0, out)


def qpat_acoustic_adjoint(ctx: Context, data, out=None):
    return ctx.acoustic_adjoint(data, out)


def qpat_da_solve(ctx: Context, mu, illum):
    return ctx.da_solve(mu, illum)


def qpat_forward(ctx: Context, mu, illum, return_phi=False):
    return ctx.forward(mu, illum, return_phi)


def qpat_jvp(ctx: Context, mu, dmu, illum, phi0=None):
    return ctx.jvp(mu, dmu, illum, phi0)


def qpat_vjp(ctx: Context, mu, w, illum, phi0=None):
    return ctx.vjp(mu, w, illum, phi0)


def qpat_dot(ctx: Context, a, b):
    return ctx.dot(a, b)


def qpat_dot_noalloc(a, b, out=None):
    """<a_b, b_b> in FP64 without any device allocation inside the library
    (``out``: a preallocated CUDA float64 tensor of shape [batch]; the
    caller owns every buffer).  a, b: CUDA float32/float64 [batch][len]."""
    import torch
    lib = load()
    for name, t in (("a", a), ("b", b)):
        if not isinstance(t, torch.Tensor) or t.device.type != "cuda":
            raise TypeError(f"qpat_dot_noalloc: {name} must be a CUDA tensor")
        if t.dtype not in (torch.float32, torch.float64):
            raise TypeError(f"qpat_dot_noalloc: {name} must be float32 or float64, not {t.dtype}")
    if a.dtype != b.dtype or a.shape != b.shape or a.dim() != 2:
        raise ValueError("qpat_dot_noalloc wants two [batch][len] tensors of one dtype and shape")
    if a.device != b.device:
        raise ValueError("qpat_dot_noalloc: a and b must be on one device")
    a = a.contiguous()
    b = b.contiguous()
    if out is None:
        out = torch.empty(a.shape[0], dtype=torch.float64, device=a.device)
    elif (not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or out.device != a.device
          or out.numel() != a.shape[0] or not out.is_contiguous()):
        raise ValueError("qpat_dot_noalloc: out must be a contiguous float64 tensor of `batch` elements "
                         "on the device of a and b")
    prec = FP32 if a.dtype == torch.float32 else FP64
    # the library looks up its scratch and launches on the current device
    with torch.cuda.device(a.device):
        st = lib.qpat_dot_noalloc(prec, a.shape[0], a.shape[1], _ptr(a), _ptr(b), _ptr(out),
                                  ctypes.c_void_p(torch.cuda.current_stream(a.device).cuda_stream))
    if st != 0:
        raise QpatError(st, lib.qpat_noalloc_last_error().decode())
    return out


def qpat_barrier_check(blocks, rounds=4, absent=0, limit_s=1.0):
    """Run the bounded grid barrier's check kernel on the current device and
    stream; returns the status code (0 = QPAT_OK, 5 = QPAT_ETIMEOUT)."""
    import torch
    st = ctypes.c_int()
    load().qpat_barrier_check(int(blocks), int(rounds), int(absent), float(limit_s),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream), ctypes.byref(st))
    return st.value


def qpat_ld_solve(ctx: Context, data, illums, mu0, kappa0=None, **params):
    return ctx.ld_solve(data, illums, mu0, kappa0, **params)


def qpat_tv_apply(ctx: Context, xbar, edge, beta, gamma, u):
    return ctx.tv_apply(xbar, u, edge, beta, gamma)


def qpat_set_kappa(ctx: Context, kappa):
    ctx.set_kappa(kappa)


def qpat_jvp_kappa(ctx: Context, mu, dkappa, illum, phi0=None):
    return ctx.jvp_kappa(mu, dkappa, illum, phi0)


def qpat_vjp_kappa(ctx: Context, mu, w, illum, phi0=None):
    return ctx.vjp_kappa(mu, w, illum, phi0)


def qpat_jvp_medium(ctx: Context, p0, dc=None, drho=None):
    return ctx.jvp_medium(p0, dc, drho)


def qpat_vjp_medium(ctx: Context, p0, w):
    return ctx.vjp_medium(p0, w)


def qpat_sync(ctx: Context):
    ctx.sync()


def qpat_get_sizes(ctx: Context):
    return ctx.sizes()


def context_from_workload(w, precision="fp32", max_batch=1, nt=None, **kw) -> Context:
    """Context for a ``phantoms.Workload`` (medium, sensors, dt from its recipe)."""
    import phantoms
    c, rho, alpha = phantoms.acoustic_medium(w)
    dt = phantoms.time_step(w, c)
    return Context(c, rho, alpha, phantoms.optical_diffusion(w), phantoms.sensor_positions(w),
                   dx=w.dx, dt=dt, nt=w.nt if nt is None else nt, pml=w.pml, y=w.y, lossless=w.lossless,
                   precision=precision, max_batch=max_batch, **kw)
