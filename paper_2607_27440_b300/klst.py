"""Thin Python binding over the C ABI of ``include/klst.h`` (argument marshalling only).

Device memory and streams come from PyTorch; every step of the eigensolve runs in
the CUDA library ``libklst.so``.  There is no CPU fallback: if the library or a
CUDA device is missing, the calls raise.
"""
import ctypes
import os

import numpy as np

from . import build as _build

c_int32, c_int64, c_double, c_void_p, c_uint64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64

KLST_OK, KLST_EINVAL, KLST_ENOMEM, KLST_ESINGULAR, KLST_ENOCONV, KLST_EREFINE, KLST_ETIMEOUT, KLST_ECUDA = 0, -1, -2, -3, -4, -5, -6, -7
FP64, MIXED, DF64 = 0, 1, 2
CONV_REL, CONV_RESID = 0, 1
ARITH_F64, ARITH_DF64 = 0, 1
JD_PREC_FULL, JD_PREC_BLOCK = 0, 1
BASES = {"tanh": 0, "mott_smith": 1, "gilbarg_paolucci": 2}


class PencilDesc(ctypes.Structure):
    _fields_ = [("nx", c_int32), ("qx", c_int32), ("qy", c_int32), ("map_L", c_double), ("map_sinf", c_double),
                ("mach", c_double), ("gamma", c_double), ("visc_s", c_double), ("re_delta", c_double),
                ("beta", c_double), ("width", c_double), ("base", c_int32), ("noneq", c_int32),
                ("conservative", c_int32)]


class EigsOpts(ctypes.Structure):
    _fields_ = [("nev", c_int32), ("ncv", c_int32), ("max_restarts", c_int32), ("max_refine", c_int32),
                ("tol", c_double), ("refine_tol", c_double), ("v0", c_void_p), ("seed", c_uint64),
                ("conv", c_int32), ("est_out", c_void_p), ("keep", c_int32),
                ("arith", c_int32)]


class EigsInfo(ctypes.Structure):
    _fields_ = [("nconv", c_int32), ("restarts", c_int32), ("applies", c_int32), ("refine_sweeps", c_int32),
                ("t_factor_ms", c_double), ("t_eigs_ms", c_double), ("max_resid", c_double),
                ("max_refine_resid", c_double), ("t_apply_ms", c_double), ("t_orth_ms", c_double),
                ("t_restart_ms", c_double), ("t_schur_ms", c_double),
                ("reorths", c_int32), ("schur_sweeps", c_int32), ("schur_swaps", c_int32),
                ("schur_rotations", c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class JdOpts(ctypes.Structure):
    _fields_ = [("nev", c_int32), ("ncv", c_int32), ("kmin", c_int32), ("max_outer", c_int32), ("tol", c_double),
                ("gmres_m", c_int32), ("gmres_max", c_int32), ("gmres_rtol", c_double), ("gmres_atol", c_double),
                ("precond", c_int32), ("v0", c_void_p), ("seed", c_uint64)]


class JdInfo(ctypes.Structure):
    _fields_ = [("nconv", c_int32), ("outer", c_int32), ("inner", c_int32), ("restarts", c_int32),
                ("applies_op", c_int64), ("applies_prec", c_int64), ("t_ms", c_double), ("max_resid", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BgkOpts(ctypes.Structure):
    _fields_ = [("max_steps", c_int32), ("cfl", c_double), ("dt", c_double), ("tol", c_double),
                ("check_every", c_int32), ("recentre_every", c_int32), ("recentre_tol", c_double),
                ("start", c_int32)]


class BgkInfo(ctypes.Structure):
    _fields_ = [("steps", c_int32), ("recentres", c_int32), ("resid", c_double), ("centre", c_double),
                ("dt", c_double), ("t_ms", c_double), ("newton_avg", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GpCase(ctypes.Structure):
    _fields_ = [("mach", c_double), ("re", c_double), ("visc_s", c_double), ("prandtl", c_double)]


class GpOpts(ctypes.Structure):
    _fields_ = [("step", c_double), ("eps", c_double), ("max_steps", c_int32)]


class GpResult(ctypes.Structure):
    _fields_ = [("delta", c_double), ("x_shock", c_double), ("x_up", c_double), ("lambda_s", c_double),
                ("steps", c_int32), ("status", c_int32)]


class KlstError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} [{code}]")
        self.code = code


_lib = None

EXPORTS = {
    "klst_status_string": (ctypes.c_char_p, [c_int32]),
    "klst_last_error": (ctypes.c_char_p, []),
    "klst_launch_count": (ctypes.c_ulonglong, []),
    "klst_prof_enable": (None, [c_int32]),
    "klst_prof_reset": (None, []),
    "klst_prof_entry": (c_int32, [c_int32, ctypes.c_char_p, c_int32, ctypes.POINTER(c_double),
                                  ctypes.POINTER(c_int64)]),
    "klst_build_pencil": (c_int32, [ctypes.POINTER(PencilDesc), c_void_p, ctypes.POINTER(c_void_p)]),
    "klst_build_pencil_base": (c_int32, [ctypes.POINTER(PencilDesc), c_void_p, c_void_p, c_void_p,
                                         ctypes.POINTER(c_void_p)]),
    "klst_gp_shock": (c_int32, [c_void_p, c_int32, ctypes.POINTER(GpOpts), ctypes.POINTER(c_double), c_int32,
                                c_void_p, c_void_p, c_void_p]),
    "klst_bgk_base_flow": (c_int32, [ctypes.POINTER(PencilDesc), ctypes.POINTER(BgkOpts), c_void_p, c_void_p,
                                     ctypes.POINTER(BgkInfo), c_void_p]),
    "klst_pencil_destroy": (None, [c_void_p]),
    "klst_pencil_dims": (c_int32, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_int32),
                                   ctypes.POINTER(c_int32), ctypes.POINTER(c_int64)]),
    "klst_pencil_tables": (c_int32, [c_void_p] + [c_void_p] * 9),
    "klst_export_dense": (c_int32, [c_void_p, c_double, c_double, c_void_p, c_void_p]),
    "klst_apply_pencil": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "klst_apply_pencil_noalloc": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "klst_apply_pencil_noalloc_capacity": (ctypes.c_size_t, []),
    "klst_base_noneq": (c_int32, [c_void_p, c_void_p]),
    "klst_eigvec_macro": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "klst_factor_shift": (c_int32, [c_void_p, c_double, c_double, c_int32, c_void_p, ctypes.POINTER(c_void_p)]),
    "klst_factor_destroy": (None, [c_void_p]),
    "klst_factor_info": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "klst_factor_inverse_info": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "klst_apply_shift_invert": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "klst_jd_eigs": (c_int32, [c_void_p, ctypes.POINTER(JdOpts), c_void_p, c_void_p, c_void_p,
                               ctypes.POINTER(JdInfo), c_void_p]),
    "klst_factor_set_refine": (c_int32, [c_void_p, c_int32, c_double]),
    "klst_factor_check": (c_int32, [c_void_p, c_void_p]),
    "klst_debug_fail_alloc_after": (None, [c_int64]),
    "klst_eigs": (c_int32, [c_void_p, ctypes.POINTER(EigsOpts), c_void_p, c_void_p, c_void_p,
                            ctypes.POINTER(EigsInfo), c_void_p]),
    "klst_batch_eigs": (c_int32, [c_int32, c_void_p, c_void_p, c_int32, ctypes.POINTER(EigsOpts), c_int32,
                                  c_void_p, c_void_p, c_void_p, c_void_p]),
    "klst_solve_footprint": (c_int64, [ctypes.POINTER(PencilDesc), c_int32, ctypes.POINTER(EigsOpts)]),
    "klst_gemm_f64_tc": (c_int32, [c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int64, c_int32, c_int32, c_int32,
                                   c_void_p]),
    "klst_server_create": (c_int32, [c_int64, c_int32, ctypes.POINTER(c_void_p)]),
    "klst_server_submit": (c_int32, [c_void_p, ctypes.POINTER(PencilDesc), c_double, c_double, c_int32,
                                     ctypes.POINTER(EigsOpts), ctypes.POINTER(c_uint64)]),
    "klst_server_poll": (c_int32, [c_void_p, c_uint64, c_int32, ctypes.POINTER(c_int32), c_void_p, c_void_p,
                                   ctypes.POINTER(EigsInfo), ctypes.POINTER(c_double)]),
    "klst_server_stats": (c_int32, [c_void_p, ctypes.POINTER(c_int32), ctypes.POINTER(c_int32),
                                    ctypes.POINTER(c_int64)]),
    "klst_server_destroy": (None, [c_void_p]),
}


def prof_enable(on=True):
    """Record CUDA events around each named kernel group on its launching stream."""
    load().klst_prof_enable(1 if on else 0)


def prof_reset():
    load().klst_prof_reset()


def prof_read():
    """{group: (total_ms, calls)} accumulated since the last prof_reset (waits for the events)."""
    lib = load()
    out = {}
    count = lib.klst_prof_entry(-1, None, 0, None, None)
    buf = ctypes.create_string_buffer(64)
    for i in range(count):
        ms, calls = c_double(0), c_int64(0)
        lib.klst_prof_entry(i, buf, 64, ctypes.byref(ms), ctypes.byref(calls))
        out[buf.value.decode()] = (ms.value, calls.value)
    return out


def lib_path():
    return _build.LIB


def load(build_if_stale=True):
    """Load libklst.so (building it in-tree first when missing or older than its sources)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not built: {_build.LIB}")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code):
    if code != KLST_OK:
        lib = load()
        raise KlstError(code, f"{lib.klst_status_string(code).decode()}: {lib.klst_last_error().decode()}")


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the kLST library has no CPU path")
    return torch


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_void_p(s.cuda_stream)


def make_desc(spec):
    g = spec if isinstance(spec, dict) else spec.as_dict()
    return PencilDesc(nx=g["nx"], qx=g["qx"], qy=g["qy"], map_L=g["map_L"], map_sinf=g["map_sinf"], mach=g["mach"],
                      gamma=g["gamma"], visc_s=g["visc_s"], re_delta=g["re_delta"], beta=g["beta"], width=g["width"],
                      base=BASES[g["base"]], noneq=int(g["noneq"]), conservative=int(g["conservative"]))


def _ptr(t):
    return c_void_p(t.data_ptr())


def _check_in(x, n, name="x"):
    """x must be a CUDA complex128 tensor of shape (n,) or (nrhs, n); returns it contiguous."""
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.dtype != torch.complex128 or x.device.type != "cuda":
        raise ValueError(f"{name} must be a complex128 CUDA tensor")
    if x.dim() not in (1, 2) or x.shape[-1] != n or x.numel() == 0:
        raise ValueError(f"{name} must have shape (n,) or (nrhs, n) with n = {n}, got {tuple(x.shape)}")
    return x.contiguous()


def _check_out(out, x, name="out"):
    """A caller-supplied output must match x exactly and not overlap it: the kernels write n * nrhs
    complex128 values through its pointer."""
    torch = _torch()
    if not isinstance(out, torch.Tensor) or out.dtype != torch.complex128:
        raise ValueError(f"{name} must be a complex128 tensor")
    if out.device != x.device:
        raise ValueError(f"{name} is on {out.device}, x on {x.device}")
    if tuple(out.shape) != tuple(x.shape) or not out.is_contiguous():
        raise ValueError(f"{name} must be contiguous with shape {tuple(x.shape)}, got {tuple(out.shape)}")
    nb = x.numel() * 16
    if out.data_ptr() < x.data_ptr() + nb and x.data_ptr() < out.data_ptr() + nb:
        raise ValueError(f"{name} may not overlap x")
    return out


class Pencil:
    """Device-resident kLST pencil (klst_build_pencil)."""

    def __init__(self, spec, stream=None, base=None):
        """``base``: optional (g_c, h_c) float64 CUDA tensors of shape (Nx, Nxi) in node order (e.g. from
        bgk_base_flow), used in place of the synthetic base flow (klst_build_pencil_base)."""
        lib = load()
        torch = _torch()
        self.spec = spec
        self._desc = make_desc(spec)
        h = c_void_p()
        if base is None:
            _check(lib.klst_build_pencil(ctypes.byref(self._desc), _stream(stream), ctypes.byref(h)))
        else:
            shape = (spec.nx, spec.nxi)
            gb = []
            for a in base:
                if (not isinstance(a, torch.Tensor) or a.dtype != torch.float64 or a.device.type != "cuda"
                        or tuple(a.shape) != shape):
                    raise ValueError(f"base arrays must be float64 CUDA tensors of shape {shape}")
                gb.append(a.contiguous())
            _check(lib.klst_build_pencil_base(ctypes.byref(self._desc), _ptr(gb[0]), _ptr(gb[1]), _stream(stream),
                                              ctypes.byref(h)))
        self.handle = h
        n, nx, nxi, fp = c_int64(), c_int32(), c_int32(), c_int64()
        _check(lib.klst_pencil_dims(h, ctypes.byref(n), ctypes.byref(nx), ctypes.byref(nxi), ctypes.byref(fp)))
        self.n, self.nx, self.nxi, self.footprint = n.value, nx.value, nxi.value, fp.value

    def close(self):
        if getattr(self, "handle", None):
            load().klst_pencil_destroy(self.handle)
            self.handle = None

    __del__ = close

    def tables(self):
        nx, nxi = self.nx, self.nxi
        out = dict(x=np.zeros(nx), Dx=np.zeros((nx, nx)), xi_x=np.zeros(nxi), xi_y=np.zeros(nxi), W=np.zeros(nxi),
                   nu=np.zeros(nx), G=np.zeros((nxi, 2, 4, nx)), w=np.zeros((nxi, 2, 4, nx)),
                   bc=np.zeros((nx, nxi), dtype=np.uint8))
        args = [out[k].ctypes.data_as(c_void_p) for k in ("x", "Dx", "xi_x", "xi_y", "W", "nu", "G", "w", "bc")]
        _check(load().klst_pencil_tables(self.handle, *args))
        return out

    def export_dense(self, sigma=0.0):
        n = self.n
        A = np.zeros((n, n), dtype=np.complex128)
        B = np.zeros(n)
        sigma = complex(sigma)
        _check(load().klst_export_dense(self.handle, sigma.real, sigma.imag, A.ctypes.data_as(c_void_p),
                                        B.ctypes.data_as(c_void_p)))
        return A, B

    def apply(self, x, omega=None, stream=None):
        """(A - omega_r B) x_r for x of shape (nrhs, n) (or (n,)), complex128 on the device."""
        torch = _torch()
        x = _check_in(x, self.n)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = torch.empty_like(x)
        om = None
        if omega is not None:
            om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, dtype=np.complex128), (nrhs,)))
        _check(load().klst_apply_pencil(self.handle, _ptr(x), _ptr(y), nrhs,
                                        om.ctypes.data_as(c_void_p) if om is not None else None, _stream(stream)))
        return y

    def apply_noalloc(self, x, omega=None, out=None, stream=None):
        """Same as ``apply`` through klst_apply_pencil_noalloc (fixed device scratch, no allocation).

        ``out`` lets a caller that cannot allocate pass its own output buffer.
        """
        torch = _torch()
        x = _check_in(x, self.n)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = torch.empty_like(x) if out is None else _check_out(out, x)
        om = None
        if omega is not None:
            om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega, dtype=np.complex128), (nrhs,)))
        _check(load().klst_apply_pencil_noalloc(self.handle, _ptr(x), _ptr(y), nrhs,
                                                om.ctypes.data_as(c_void_p) if om is not None else None,
                                                _stream(stream)))
        return y

    def base_noneq(self):
        """E_neq(x_j) of the base flow (Eq. L2norm), float64 (nx,)."""
        out = np.zeros(self.nx)
        _check(load().klst_base_noneq(self.handle, out.ctypes.data_as(c_void_p)))
        return out

    def eigvec_macro(self, vecs, stream=None):
        """(rho^, u^, v^, E^) per point for vectors of shape (nvec, n) or (n,): complex (nvec, 4, nx), and
        max_x |U^| per vector (Eq. Unormpert)."""
        vecs = _check_in(vecs, self.n, "vecs")
        nvec = 1 if vecs.dim() == 1 else vecs.shape[0]
        m = np.zeros((nvec, 4, self.nx), dtype=np.complex128)
        um = np.zeros(nvec)
        _check(load().klst_eigvec_macro(self.handle, _ptr(vecs), nvec, m.ctypes.data_as(c_void_p),
                                        um.ctypes.data_as(c_void_p), _stream(stream)))
        return m, um

    def factor(self, sigma, precision=FP64, stream=None):
        return Factor(self, sigma, precision, stream)


class Factor:
    """Shifted factorisation of a pencil (klst_factor_shift)."""

    def __init__(self, pencil, sigma, precision=FP64, stream=None):
        lib = load()
        self.pencil = pencil
        self.sigma = complex(sigma)
        self.precision = precision
        h = c_void_p()
        _check(lib.klst_factor_shift(pencil.handle, self.sigma.real, self.sigma.imag, precision, _stream(stream),
                                     ctypes.byref(h)))
        self.handle = h
        fp, tms = c_int64(), c_double()
        _check(lib.klst_factor_info(h, None, None, None, ctypes.byref(fp), ctypes.byref(tms)))
        self.footprint, self.t_factor_ms = fp.value, tms.value

    def close(self):
        if getattr(self, "handle", None):
            load().klst_factor_destroy(self.handle)
            self.handle = None

    __del__ = close

    def inverse_info(self):
        """klst_factor_inverse_info: {"method": 1 tensor-core Newton-Schulz | 0 float64 Gauss-Jordan,
        "steps", "fallback", "resid"}."""
        m, st, fb, r = c_int32(), c_int32(), c_int32(), c_double()
        _check(load().klst_factor_inverse_info(self.handle, ctypes.byref(m), ctypes.byref(st), ctypes.byref(fb),
                                               ctypes.byref(r)))
        return {"method": m.value, "steps": st.value, "fallback": fb.value, "resid": r.value}

    def set_refine(self, max_refine, refine_tol):
        _check(load().klst_factor_set_refine(self.handle, max_refine, refine_tol))

    def check(self, stream=None):
        """klst_factor_check: KLST_EREFINE if an apply since the last check missed refine_tol, else KLST_OK."""
        return load().klst_factor_check(self.handle, _stream(stream))

    def apply(self, x, out=None, stream=None):
        """y = (A - sigma B)^{-1} B x for x of shape (nrhs, n) or (n,), complex128 on the device."""
        torch = _torch()
        x = _check_in(x, self.pencil.n)
        nrhs = 1 if x.dim() == 1 else x.shape[0]
        y = torch.empty_like(x) if out is None else _check_out(out, x)
        _check(load().klst_apply_shift_invert(self.handle, _ptr(x), _ptr(y), nrhs, _stream(stream)))
        return y

    def eigs(self, nev, ncv, tol=1e-12, max_restarts=200, max_refine=4, refine_tol=1e-12, v0=None, seed=0,
             vectors=False, stream=None, check=True, conv=CONV_REL, keep=0, arith=ARITH_F64):
        """Krylov-Schur shift-invert eigensolve; returns (omega[nev], vecs (nev, n) or None, resid[nev], info).

        info carries the klst_eigs_info fields plus ``status`` and ``ritz_est`` (final Ritz estimates).
        """
        torch = _torch()
        n = self.pencil.n
        ev = np.zeros(2 * nev)
        res = np.zeros(nev)
        vec = torch.empty((nev, n), dtype=torch.complex128, device="cuda") if vectors else None
        if v0 is not None:
            v0 = _check_in(v0, n, "v0")
            if v0.dim() != 1:
                raise ValueError("v0 must be one vector of length n")
        est = np.zeros(nev)
        opts = EigsOpts(nev=nev, ncv=ncv, max_restarts=max_restarts, max_refine=max_refine, tol=tol,
                        refine_tol=refine_tol, v0=v0.data_ptr() if v0 is not None else None, seed=seed, conv=conv,
                        est_out=est.ctypes.data, keep=keep, arith=arith)
        info = EigsInfo()
        code = load().klst_eigs(self.handle, ctypes.byref(opts), ev.ctypes.data_as(c_void_p),
                                _ptr(vec) if vec is not None else None, res.ctypes.data_as(c_void_p),
                                ctypes.byref(info), _stream(stream))
        if check:
            _check(code)
        omega = ev[0::2] + 1j * ev[1::2]
        d = info.as_dict()
        d["status"] = code
        d["ritz_est"] = est
        return omega, vec, res, d


    def jd_eigs(self, nev, ncv=40, kmin=6, tol=1e-10, max_outer=2000, gmres_m=30, gmres_max=200, gmres_rtol=1e-6,
                gmres_atol=1e-12, precond=JD_PREC_FULL, v0=None, seed=0, vectors=False, stream=None, check=True):
        """klst_jd_eigs: Jacobi-Davidson with harmonic Ritz extraction; returns (omega[nconv],
        vecs (nconv, n) or None, resid[nconv], info) with info = the klst_jd_info fields plus ``status``."""
        torch = _torch()
        n = self.pencil.n
        ev = np.zeros(2 * nev)
        res = np.zeros(nev)
        vec = torch.empty((nev, n), dtype=torch.complex128, device="cuda") if vectors else None
        if v0 is not None:
            v0 = _check_in(v0, n, "v0")
            if v0.dim() != 1:
                raise ValueError("v0 must be one vector of length n")
        opts = JdOpts(nev=nev, ncv=ncv, kmin=kmin, max_outer=max_outer, tol=tol, gmres_m=gmres_m,
                      gmres_max=gmres_max, gmres_rtol=gmres_rtol, gmres_atol=gmres_atol, precond=precond,
                      v0=v0.data_ptr() if v0 is not None else None, seed=seed)
        info = JdInfo()
        code = load().klst_jd_eigs(self.handle, ctypes.byref(opts), ev.ctypes.data_as(c_void_p),
                                   _ptr(vec) if vec is not None else None, res.ctypes.data_as(c_void_p),
                                   ctypes.byref(info), _stream(stream))
        if check:
            _check(code)
        k = info.nconv
        d = info.as_dict()
        d["status"] = code
        return (ev[0:2 * k:2] + 1j * ev[1:2 * k:2], vec[:k] if vec is not None else None, res[:k], d)


BGK_STARTS = {"mott_smith": 0, "gilbarg_paolucci": 1}


def bgk_base_flow(spec, max_steps=20000, cfl=0.5, dt=0.0, tol=0.0, check_every=100, recentre_every=0,
                  recentre_tol=0.25, start="mott_smith", stream=None):
    """klst_bgk_base_flow: the BE-BGK steady shock on the pencil's grid; returns (g, h, info) with g, h
    float64 CUDA tensors of shape (Nx, Nxi) in node order (j = 0 downstream).  start: 'mott_smith' or
    'gilbarg_paolucci' (the continuum profile's local Maxwellian)."""
    lib = load()
    torch = _torch()
    d = make_desc(spec)
    g = torch.empty((spec.nx, spec.nxi), dtype=torch.float64, device="cuda")
    h = torch.empty_like(g)
    o = BgkOpts(max_steps=max_steps, cfl=cfl, dt=dt, tol=tol, check_every=check_every,
                recentre_every=recentre_every, recentre_tol=recentre_tol, start=BGK_STARTS[start])
    info = BgkInfo()
    _check(lib.klst_bgk_base_flow(ctypes.byref(d), ctypes.byref(o), _ptr(g), _ptr(h), ctypes.byref(info),
                                  _stream(stream)))
    return g, h, info.as_dict()


def gp_shock(mach, re=1.0, visc_s=0.5, prandtl=1.0, x=None, step=0.0, eps=0.0, max_steps=0, stream=None):
    """klst_gp_shock over a batch of cases (mach, re, visc_s, prandtl broadcast to one length).
    Returns (res, prof): res a dict of numpy arrays (delta, x_shock, x_up, lambda_s, steps, status) and
    prof a float64 CUDA tensor (3, ncases, len(x)) of rho, u, T at the points x (measured from the
    steepest point), or None without x.  With re = 1, res["delta"] is the self-consistent Re_Delta."""
    lib = load()
    torch = _torch()
    cols = np.broadcast_arrays(*[np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (mach, re, visc_s, prandtl)])
    n = cols[0].size
    cases = (GpCase * n)(*[GpCase(*(float(c.flat[i]) for c in cols)) for i in range(n)])
    res = (GpResult * n)()
    xs = None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float64).ravel())
    npts = 0 if xs is None else xs.size
    prof = torch.empty((3, n, npts), dtype=torch.float64, device="cuda") if npts else None
    o = GpOpts(step=step, eps=eps, max_steps=max_steps)
    _check(lib.klst_gp_shock(cases, n, ctypes.byref(o),
                             None if xs is None else xs.ctypes.data_as(ctypes.POINTER(c_double)), npts,
                             _ptr(prof) if prof is not None else None, res, _stream(stream)))
    out = {k: np.array([getattr(r, k) for r in res]) for k, _ in GpResult._fields_}
    return out, prof


def _opts(nev, ncv, tol=1e-12, max_restarts=200, max_refine=4, refine_tol=1e-12, seed=0, conv=CONV_REL, keep=0,
          arith=ARITH_F64):
    return EigsOpts(nev=nev, ncv=ncv, max_restarts=max_restarts, max_refine=max_refine, tol=tol,
                    refine_tol=refine_tol, v0=None, seed=seed, conv=conv, est_out=None, keep=keep, arith=arith)


def batch_eigs(specs, sigmas, nev, ncv, precision=FP64, nworkers=0, **kw):
    """klst_batch_eigs over a list of pencil specs and shifts; returns (omega (P, nev), resid (P, nev), status (P,), infos)."""
    lib = load()
    _torch()
    P = len(specs)
    descs = (PencilDesc * P)(*[make_desc(s) for s in specs])
    sig = np.ascontiguousarray(np.asarray(sigmas, dtype=np.complex128))
    ev = np.zeros((P, 2 * nev))
    res = np.zeros((P, nev))
    st = np.zeros(P, dtype=np.int32)
    infos = (EigsInfo * P)()
    opts = _opts(nev, ncv, **kw)
    code = lib.klst_batch_eigs(P, ctypes.cast(descs, c_void_p), sig.ctypes.data_as(c_void_p), precision,
                               ctypes.byref(opts), nworkers, ev.ctypes.data_as(c_void_p),
                               res.ctypes.data_as(c_void_p), st.ctypes.data_as(c_void_p), ctypes.cast(infos, c_void_p))
    if code == KLST_EINVAL:  # rejected before any pencil ran: status_host was not written
        _check(code)
    return ev[:, 0::2] + 1j * ev[:, 1::2], res, st, [i.as_dict() for i in infos]


def gemm_f64_tc(A, B, stream=None):
    """C = A @ B (float64 CUDA tensors, 2-D) through klst_gemm_f64_tc (float64 accuracy on tensor cores)."""
    torch = _torch()
    for t, nm in ((A, "A"), (B, "B")):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or t.device.type != "cuda" or t.dim() != 2:
            raise ValueError(f"{nm} must be a 2-D float64 CUDA tensor")
    M, K = A.shape
    K2, N = B.shape
    if K2 != K:
        raise ValueError("inner dimensions differ")
    At = A.t().contiguous()  # column-major M x K: the transpose's row-major storage
    Bt = B.t().contiguous()
    C = torch.empty((N, M), dtype=torch.float64, device=A.device)  # column-major M x N
    _check(load().klst_gemm_f64_tc(_ptr(At), M, _ptr(Bt), K, _ptr(C), M, M, N, K, _stream(stream)))
    return C.t()


def fail_alloc_after(n):
    """klst_debug_fail_alloc_after: the n-th next device allocation of the library fails (n < 0: off)."""
    load().klst_debug_fail_alloc_after(int(n))


def solve_footprint(spec, nev, ncv, precision=FP64, **kw):
    """Device bytes klst_server admits a request by (klst_solve_footprint)."""
    d = make_desc(spec)
    o = _opts(nev, ncv, **kw)
    b = load().klst_solve_footprint(ctypes.byref(d), precision, ctypes.byref(o))
    if b < 0:
        _check(int(b))
    return int(b)


class Server:
    """klst_server_*: footprint-admitted, concurrently running eigensolve requests."""

    def __init__(self, hbm_budget_bytes, max_slots):
        lib = load()
        _torch()
        h = c_void_p()
        _check(lib.klst_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(h)))
        self.handle = h
        self._nev = {}

    def submit(self, spec, sigma, nev, ncv, precision=FP64, **kw):
        d = make_desc(spec)
        o = _opts(nev, ncv, **kw)
        t = c_uint64()
        sigma = complex(sigma)
        _check(load().klst_server_submit(self.handle, ctypes.byref(d), sigma.real, sigma.imag, precision,
                                         ctypes.byref(o), ctypes.byref(t)))
        self._nev[t.value] = nev
        return t.value

    def poll(self, ticket, wait=False):
        """Returns None while running, else (omega, resid, info, latency_ms, status)."""
        nev = self._nev[ticket]
        done = c_int32()
        ev = np.zeros(2 * nev)
        res = np.zeros(nev)
        info = EigsInfo()
        lat = c_double()
        code = load().klst_server_poll(self.handle, ticket, 1 if wait else 0, ctypes.byref(done),
                                       ev.ctypes.data_as(c_void_p), res.ctypes.data_as(c_void_p), ctypes.byref(info),
                                       ctypes.byref(lat))
        if not done.value:
            if code != KLST_OK:
                _check(code)
            return None
        del self._nev[ticket]
        return ev[0::2] + 1j * ev[1::2], res, info.as_dict(), lat.value, code

    def stats(self):
        q, r, b = c_int32(), c_int32(), c_int64()
        _check(load().klst_server_stats(self.handle, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
        return q.value, r.value, b.value

    def close(self):
        if getattr(self, "handle", None):
            load().klst_server_destroy(self.handle)
            self.handle = None

    __del__ = close
