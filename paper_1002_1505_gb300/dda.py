"""Thin Python binding of the C-ABI library libdda.so (ctypes, argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the library's CUDA kernels (or,
for set-up, in its host C++).  Device buffers are torch tensors on the
context's device; their data pointers and torch's current stream are passed
through.  If the library is missing, importing this module raises: there is
no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("DDA_LIB", os.path.join(_HERE, "libdda.so"))

DDA_OK, DDA_EINVAL, DDA_ENOMEM, DDA_ECUDA, DDA_ENOCONV, DDA_ETIMEOUT, DDA_ESTATE, DDA_EUNSUPPORTED = range(8)
DDA_C64, DDA_C128, DDA_C128DF = 1, 2, 3  # DDA_C128DF: complex128 vectors, double-float arithmetic
SHAPES = {"ELLIPSOID": 1, "RCTGLPRSM": 2, "CYLINDER1": 3, "HEX_PRISM": 4}
PRESCRIPTIONS = {"CM": 1, "LATTDR": 2, "GKDLDR": 3}
SOLVERS = {"BICGSTAB": 1, "CCG": 2, "BICGSTAB2": 3, "COCG": 4, "QMRCS": 5}
PRECONDS = {"NONE": 0, "JACOBI": 1}
PRECISIONS = {"C64": 1, "C128": 2, "MIXED": 3}
STATUS_NAMES = ["DDA_OK", "DDA_EINVAL", "DDA_ENOMEM", "DDA_ECUDA", "DDA_ENOCONV", "DDA_ETIMEOUT", "DDA_ESTATE",
                "DDA_EUNSUPPORTED"]


class DDAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class dda_solve_opts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("inner_tol", ctypes.c_double), ("timeout_ms", ctypes.c_double),
                ("warm_start", ctypes.c_int), ("check_every", ctypes.c_int), ("normal_eq", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("precond", ctypes.c_int), ("phi_reuse", ctypes.c_int)]


class dda_solve_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("matvecs", ctypes.c_int), ("outer", ctypes.c_int),
                ("converged", ctypes.c_int), ("true_rel_resid", ctypes.c_double),
                ("normal_eq_ratio", ctypes.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdda.so not built at {LIB_PATH}: run paper_1002_1505_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "dda_create": (I, [ctypes.POINTER(P), I, P]),
        "dda_destroy": (None, [P]),
        "dda_last_error": (ctypes.c_char_p, [P]),
        "dda_set_stream": (I, [P, P]),
        "dda_setup_shape": (I, [P, I, P, I, P, P]),
        "dda_setup_target": (I, [P, P, P, I64, P, P, P]),
        "dda_setup_target_aniso": (I, [P, P, P, I64, P, P, P]),
        "dda_setup_target_anifrm": (I, [P, P, P, I64, P, P, P, P]),
        "dda_get_sites": (I, [P, P, P]),
        "dda_get_box": (I, [P, P, P]),
        "dda_set_incident": (I, [P, D, P, I, P, I]),
        "dda_kd_from_x": (I, [P, D, P, P]),
        "dda_set_periodicity": (I, [P, D, D, D]),
        "dda_orientation_average": (I, [P, I, I, P, I64, P]),
        "dda_nrhs": (I, [P]),
        "dda_get_incidence": (I, [P, P, P]),
        "dda_incident_field": (I, [P, P, I]),
        "dda_build_green_fft": (I, [P, P]),
        "dda_set_polarizability": (I, [P, I, P, I]),
        "dda_get_inv_alpha": (I, [P, P]),
        "dda_matvec": (I, [P, P, P, I, I]),
        "dda_solve": (I, [P, P, P, P]),
        "dda_cross_sections": (I, [P, P, P, P, I, P]),
        "dda_version": (ctypes.c_char_p, []),
        "dda_kernel_launches": (ctypes.c_ulonglong, []),
        "dda_selftest_bulk_wait": (I, [I, P]),
        "dda_probe_tc_dft": (I, [I, I64, I, P]),
        "dda_angular_averages": (I, [P, P, D, P, P]),
        "dda_force_torque": (I, [P, P, D, P, P]),
        "dda_near_field": (I, [P, P, P, I64, P, P]),
        "dda_periodic_scattering": (I, [P, P, I, P, P, P, P]),
        "dda_orientation_grid": (I, [P, I, P, I, P, I, P, P]),
        "dda_profile_matvec": (I, [P, I, I, I, P, P]),
        "dda_matvec_noalloc": (I, [P, P, P, I, I]),
        "dda_schedule_info": (I, [P, I, P]),
        "dda_solve_batch": (I, [P, I, P, P, P, P]),
        "dda_unet_create": (I, [ctypes.POINTER(P), I, P, I, I, P, ctypes.c_uint64]),
        "dda_unet_destroy": (None, [P]),
        "dda_unet_check_fault": (I, [P]),
        "dda_unet_last_error": (ctypes.c_char_p, [P]),
        "dda_unet_nparams": (I64, [P]),
        "dda_unet_get_params": (I, [P, P, I]),
        "dda_unet_set_params": (I, [P, P]),
        "dda_unet_forward": (I, [P, P, P, I, P]),
        "dda_unet_loss_grad": (I, [P, P, P, P, I, P, ctypes.POINTER(D)]),
        "dda_unet_adamw": (I, [P, D, D, D, D, D]),
        "dda_unet_features": (I, [P, P, P, P]),
        "dda_unet_targets": (I, [P, P, P, P, P, P, I]),
        "dda_unet_warm_start": (I, [P, P, P, P, I, P]),
        "dda_unet_forward_train": (I, [P, P, P, I, P]),
        "dda_unet_mse": (I, [P, P, P, P, I, P, D, P, ctypes.POINTER(D)]),
        "dda_unet_backward": (I, [P, P, I, P]),
        "dda_unet_residual_grad": (I, [P, P, P, P, D, P, ctypes.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class Context:
    """Owns one dda_ctx.  device < 0 gives a host-only context (set-up and getters only)."""

    def __init__(self, device: int = 0, stream=None):
        self._h = ctypes.c_void_p()
        s = 0 if device < 0 else _stream_handle(stream)
        st = LIB.dda_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(s))
        if st != DDA_OK:
            raise DDAError(st, "dda_create failed")
        self.device = device
        self.n = 0
        self.box = (0, 0, 0)
        self.nrhs = 0
        self.iorth = 0
        self.kd = 0.0
        self._periodic_2d = False   # both periods set (a new target makes it finite again)

    def close(self):
        if self._h:
            LIB.dda_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != DDA_OK:
            raise DDAError(st, LIB.dda_last_error(self._h).decode())

    # ---------------------------------------------------------------- set-up
    def dda_setup_shape(self, shape: str, shpar: Sequence[float]):
        self._periodic_2d = False
        sp = np.ascontiguousarray(shpar, dtype=np.float64)
        n = ctypes.c_int64()
        box = np.zeros(3, dtype=np.int32)
        self._check(LIB.dda_setup_shape(self._h, SHAPES[shape.upper()], _ptr(sp), len(sp), ctypes.byref(n), _ptr(box)))
        self.n = int(n.value)
        self.box = tuple(int(v) for v in box)
        return self.n, self.box

    def dda_setup_target(self, ixyz, icomp=None, origin=(0.0, 0.0, 0.0), a1=None, a2=None):
        """icomp: None, N 1-based compositions, or N x 3 (one per axis: anisotropic materials)."""
        self._periodic_2d = False
        ij = np.ascontiguousarray(ixyz, dtype=np.int32)
        ic = None if icomp is None else np.ascontiguousarray(icomp, dtype=np.int32)
        fn = LIB.dda_setup_target
        if ic is not None and ic.ndim == 2:
            fn = LIB.dda_setup_target_aniso
        org = np.ascontiguousarray(origin, dtype=np.float64)
        a1v = None if a1 is None else np.ascontiguousarray(a1, dtype=np.float64)
        a2v = None if a2 is None else np.ascontiguousarray(a2, dtype=np.float64)
        self._check(fn(self._h, _ptr(ij), None if ic is None else _ptr(ic), ij.shape[0], _ptr(org),
                                         None if a1v is None else _ptr(a1v), None if a2v is None else _ptr(a2v)))
        self.n, self.box = self.dda_get_box()

    def dda_setup_target_anifrm(self, ixyz, icomp3, df_angles, origin=(0.0, 0.0, 0.0), a1=None, a2=None):
        """Site list with per-axis compositions (N x 3, 1-based) and per-site Dielectric-Frame angles
        (N x 3: theta_DF, phi_DF, beta_DF, radians): the guide's ANIFRMFIL target."""
        self._periodic_2d = False
        ij = np.ascontiguousarray(ixyz, dtype=np.int32)
        ic = np.ascontiguousarray(icomp3, dtype=np.int32)
        an = np.ascontiguousarray(df_angles, dtype=np.float64)
        org = np.ascontiguousarray(origin, dtype=np.float64)
        a1v = None if a1 is None else np.ascontiguousarray(a1, dtype=np.float64)
        a2v = None if a2 is None else np.ascontiguousarray(a2, dtype=np.float64)
        self._check(LIB.dda_setup_target_anifrm(self._h, _ptr(ij), _ptr(ic), ij.shape[0], _ptr(org),
                                                None if a1v is None else _ptr(a1v),
                                                None if a2v is None else _ptr(a2v), _ptr(an)))
        self.n, self.box = self.dda_get_box()

    def dda_get_box(self):
        """(N, (box_x, box_y, box_z)) of the current target."""
        n = np.zeros(1, dtype=np.int64)
        box = np.zeros(3, dtype=np.int32)
        self._check(LIB.dda_get_box(self._h, _ptr(n), _ptr(box)))
        return int(n[0]), tuple(int(v) for v in box)

    def dda_get_sites(self):
        out = np.zeros((self.n, 3), dtype=np.int32)
        org = np.zeros(3, dtype=np.float64)
        self._check(LIB.dda_get_sites(self._h, _ptr(out), _ptr(org)))
        return out, org

    def dda_set_periodicity(self, py: float, pz: float, gamma: float = 0.01):
        """Repeat the target with periods py (y_TF) and pz (z_TF), 0 = none; gamma = interaction cutoff."""
        self._check(LIB.dda_set_periodicity(self._h, float(py), float(pz), float(gamma)))
        self._periodic_2d = py > 0 and pz > 0

    def dda_kd_from_x(self, x: float):
        """(kd, a_eff / d) for size parameter x of the current target."""
        kd = ctypes.c_double()
        aeff = ctypes.c_double()
        st = LIB.dda_kd_from_x(self._h, float(x), ctypes.byref(kd), ctypes.byref(aeff))
        if st != DDA_OK:
            raise DDAError(st, "dda_kd_from_x failed (needs a target and x > 0)")
        return float(kd.value), float(aeff.value)

    def dda_set_incident(self, kd: float, orientations, e01_lf=((0, 0), (1, 0), (0, 0)), iorth: int = 2):
        ori = np.ascontiguousarray(orientations, dtype=np.float64).reshape(-1, 3)
        e = np.ascontiguousarray(e01_lf, dtype=np.float64).reshape(6)
        self._check(LIB.dda_set_incident(self._h, float(kd), _ptr(ori), ori.shape[0], _ptr(e), int(iorth)))
        self.nrhs = LIB.dda_nrhs(self._h)
        self.iorth = iorth
        self.kd = float(kd)
        return self.nrhs

    def dda_get_incidence(self):
        k = np.zeros((self.nrhs, 3))
        e = np.zeros((self.nrhs, 6))
        self._check(LIB.dda_get_incidence(self._h, _ptr(k), _ptr(e)))
        return k, e[:, 0::2] + 1j * e[:, 1::2]

    def dda_build_green_fft(self, pad: Optional[Sequence[int]] = None):
        p = None if pad is None else np.ascontiguousarray(pad, dtype=np.int32)
        self._check(LIB.dda_build_green_fft(self._h, None if p is None else _ptr(p)))

    def dda_set_polarizability(self, prescription: str, m):
        ms = np.atleast_1d(np.asarray(m, dtype=np.complex128))
        arr = np.ascontiguousarray(np.stack([ms.real, ms.imag], axis=1))
        self._check(LIB.dda_set_polarizability(self._h, PRESCRIPTIONS[prescription.upper()], _ptr(arr), len(ms)))
        self.ncomp = len(ms)

    def dda_get_inv_alpha(self):
        out = np.zeros((self.nrhs, self.ncomp, 3, 2))
        self._check(LIB.dda_get_inv_alpha(self._h, _ptr(out)))
        return out[..., 0] + 1j * out[..., 1]

    # ---------------------------------------------------------------- device work
    def _dev_check(self, t, dtype_code):
        import torch
        want = torch.complex64 if dtype_code == DDA_C64 else torch.complex128  # C128 and C128DF
        if not t.is_cuda or t.dtype != want or not t.is_contiguous():
            raise DDAError(DDA_EINVAL, f"expected a contiguous {want} CUDA tensor")

    def dda_incident_field(self, e, dtype=DDA_C128):
        self._dev_check(e, dtype)
        self._check(LIB.dda_incident_field(self._h, ctypes.c_void_p(e.data_ptr()), dtype))

    def dda_matvec(self, p, ap, nrhs: Optional[int] = None, double_float: bool = False):
        """ap = A p (dtype of p); double_float=True computes a complex128 product in
        double-float arithmetic (DDA_C128DF)."""
        import torch
        dt = DDA_C64 if p.dtype == torch.complex64 else DDA_C128
        if double_float:
            if dt != DDA_C128:
                raise DDAError(DDA_EINVAL, "the double-float product takes complex128 vectors")
            dt = DDA_C128DF
        self._dev_check(p, dt)
        self._dev_check(ap, dt)
        nr = self.nrhs if nrhs is None else nrhs
        self._check(LIB.dda_matvec(self._h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(ap.data_ptr()), nr, dt))

    def dda_matvec_noalloc(self, p, ap, nrhs: Optional[int] = None):
        """Same product as dda_matvec, using the library's fixed 32 MiB scratch (no allocation)."""
        import torch
        dt = DDA_C64 if p.dtype == torch.complex64 else DDA_C128
        self._dev_check(p, dt)
        self._dev_check(ap, dt)
        nr = self.nrhs if nrhs is None else nrhs
        self._check(LIB.dda_matvec_noalloc(self._h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(ap.data_ptr()),
                                           nr, dt))

    def dda_solve(self, p, solver="BICGSTAB", precision="MIXED", tol=1e-5, maxit=1000, inner_tol=0.0,
                  timeout_ms=0.0, warm_start=False, check_every=8, normal_eq=False, use_graph=True,
                  raise_on_noconv=True, precond="NONE", phi_reuse=False):
        """Solve A P = E_inc; p is a complex128 [nrhs,3,N] CUDA tensor (guess if warm_start, solution out)."""
        self._dev_check(p, DDA_C128)
        o = dda_solve_opts(SOLVERS[solver.upper()], PRECISIONS[precision.upper()], tol, maxit, inner_tol,
                           timeout_ms, int(bool(warm_start)), check_every, int(bool(normal_eq)), int(bool(use_graph)),
                           PRECONDS[precond.upper()], int(bool(phi_reuse)))
        rep = (dda_solve_report * self.nrhs)()
        st = LIB.dda_solve(self._h, ctypes.byref(o), ctypes.c_void_p(p.data_ptr()), rep)
        reports = [{k: getattr(r, k) for k, _ in dda_solve_report._fields_} for r in rep]
        if st != DDA_OK and (raise_on_noconv or st not in (DDA_ENOCONV, DDA_ETIMEOUT)):
            self._check(st)
        return reports, st

    def dda_angular_averages(self, p, eta=0.5):
        """(out [nrhs, 6] = Qsca_int, <cos>, <cos^2>, <n>_LF xyz; number of directions) for solved P."""
        self._dev_check(p, DDA_C128)
        out = np.zeros((self.nrhs, 6))
        nd = np.zeros(1, dtype=np.int32)
        self._check(LIB.dda_angular_averages(self._h, ctypes.c_void_p(p.data_ptr()), float(eta), _ptr(out), _ptr(nd)))
        return out, int(nd[0])

    def dda_force_torque(self, p, eta=0.5):
        """(Q_pr [nrhs, 3], Q_Gamma [nrhs, 3], number of directions), Target-Frame components."""
        self._dev_check(p, DDA_C128)
        out = np.zeros((self.nrhs, 6))
        nd = np.zeros(1, dtype=np.int32)
        self._check(LIB.dda_force_torque(self._h, ctypes.c_void_p(p.data_ptr()), float(eta), _ptr(out), _ptr(nd)))
        return out[:, :3].copy(), out[:, 3:].copy(), int(nd[0])

    def dda_near_field(self, p, points, want_b=True):
        """(E [nrhs, npts, 3], B [nrhs, npts, 3] or None) complex, at TF points (npts, 3), lattice units."""
        self._dev_check(p, DDA_C128)
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
        e = np.zeros((self.nrhs, pts.shape[0], 6))
        b = np.zeros((self.nrhs, pts.shape[0], 6)) if want_b else None
        self._check(LIB.dda_near_field(self._h, ctypes.c_void_p(p.data_ptr()), _ptr(pts), pts.shape[0], _ptr(e),
                                       None if b is None else _ptr(b)))
        to_c = lambda a: a[..., 0::2] + 1j * a[..., 1::2]
        return to_c(e), (None if b is None else to_c(b))

    def dda_periodic_scattering(self, p, spec, mueller=True, tr=None):
        """Orders of a periodic target: spec (n, 2) = (M, N) (doubly periodic) or (M, zeta) (singly).
        Returns (dirs [n, 2, 3], Mueller [n_ori, n, 2, 4, 4] or None, T/R [nrhs, n, 2] or None);
        tr defaults to True for doubly periodic targets."""
        self._dev_check(p, DDA_C128)
        sp = np.ascontiguousarray(spec, dtype=np.float64).reshape(-1, 2)
        n = sp.shape[0]
        dirs = np.zeros((n, 2, 3))
        m = np.zeros((self.nrhs // self.iorth, n, 2, 16)) if mueller else None
        if tr is None:
            tr = self._periodic_2d
        t = np.zeros((self.nrhs, n, 2)) if tr else None
        self._check(LIB.dda_periodic_scattering(self._h, ctypes.c_void_p(p.data_ptr()), n, _ptr(sp), _ptr(dirs),
                                                None if m is None else _ptr(m), None if t is None else _ptr(t)))
        return dirs, (None if m is None else m.reshape(-1, n, 2, 4, 4)), t

    def dda_cross_sections(self, p, dirs=None):
        """Returns (Q array [nrhs,4] = Qext,Qabs,Qsca,Qpha, Mueller [n_ori,ndir,4,4] or None)."""
        self._dev_check(p, DDA_C128)
        q = np.zeros((self.nrhs, 4))
        if dirs is not None and len(dirs):
            d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 2)
            m = np.zeros((self.nrhs // self.iorth, d.shape[0], 16))
            self._check(LIB.dda_cross_sections(self._h, ctypes.c_void_p(p.data_ptr()), _ptr(q), _ptr(d), d.shape[0],
                                               _ptr(m)))
            return q, m.reshape(-1, d.shape[0], 4, 4)
        self._check(LIB.dda_cross_sections(self._h, ctypes.c_void_p(p.data_ptr()), _ptr(q), None, 0, None))
        return q, None


class UNet:
    """The learned warm start's 3-D U-Net (library-owned parameters and kernels)."""

    def __init__(self, device: int = 0, stream=None, cin: int = 9, cout: int = 6, ch=(12, 24, 32, 48), seed: int = 0):
        self._h = ctypes.c_void_p()
        chv = np.ascontiguousarray(ch, dtype=np.int32)
        st = LIB.dda_unet_create(ctypes.byref(self._h), int(device), ctypes.c_void_p(_stream_handle(stream)),
                                 int(cin), int(cout), _ptr(chv), ctypes.c_uint64(seed))
        if st != DDA_OK:
            raise DDAError(st, "dda_unet_create failed")
        self.cin, self.cout, self.ch = cin, cout, tuple(ch)
        self._keep = chv

    def close(self):
        if self._h:
            LIB.dda_unet_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != DDA_OK:
            raise DDAError(st, LIB.dda_unet_last_error(self._h).decode())

    def dda_unet_check_fault(self):
        """Raise if a tcgen05 convolution's bounded wait gave up since the last check."""
        self._check(LIB.dda_unet_check_fault(self._h))

    @property
    def nparams(self) -> int:
        return int(LIB.dda_unet_nparams(self._h))

    def dda_unet_get_params(self, which: int = 0) -> np.ndarray:
        out = np.zeros(self.nparams, dtype=np.float32)
        self._check(LIB.dda_unet_get_params(self._h, _ptr(out), int(which)))
        return out

    def dda_unet_set_params(self, theta):
        arr = np.ascontiguousarray(theta, dtype=np.float32)
        self._check(LIB.dda_unet_set_params(self._h, _ptr(arr)))

    @staticmethod
    def _dims(dims):
        return np.ascontiguousarray(dims, dtype=np.int32)

    def dda_unet_forward(self, x, y, dims):
        d = self._dims(dims)
        self._check(LIB.dda_unet_forward(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                         int(x.shape[0]), _ptr(d)))

    def dda_unet_loss_grad(self, x, t, mask, dims) -> float:
        d = self._dims(dims)
        loss = ctypes.c_double()
        self._check(LIB.dda_unet_loss_grad(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                           ctypes.c_void_p(mask.data_ptr()), int(x.shape[0]), _ptr(d),
                                           ctypes.byref(loss)))
        return float(loss.value)

    def dda_unet_forward_train(self, x, y, dims):
        d = self._dims(dims)
        self._check(LIB.dda_unet_forward_train(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                               int(x.shape[0]), _ptr(d)))

    def dda_unet_mse(self, y, t, mask, gy, dims, weight=1.0) -> float:
        d = self._dims(dims)
        loss = ctypes.c_double()
        self._check(LIB.dda_unet_mse(self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                     ctypes.c_void_p(mask.data_ptr()), int(y.shape[0]), _ptr(d), float(weight),
                                     ctypes.c_void_p(gy.data_ptr()), ctypes.byref(loss)))
        return float(loss.value)

    def dda_unet_backward(self, gy, dims):
        d = self._dims(dims)
        self._check(LIB.dda_unet_backward(self._h, ctypes.c_void_p(gy.data_ptr()), int(gy.shape[0]), _ptr(d)))

    def dda_unet_adamw(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
        self._check(LIB.dda_unet_adamw(self._h, float(lr), float(beta1), float(beta2), float(eps), float(wd)))


def dda_unet_features(ctx: "Context", x, dims, offset=None):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    o = None if offset is None else np.ascontiguousarray(offset, dtype=np.int32)
    ctx._check(LIB.dda_unet_features(ctx._h, ctypes.c_void_p(x.data_ptr()), _ptr(d), None if o is None else _ptr(o)))


def dda_unet_targets(ctx: "Context", p, t, mask, dims, offset=None, residual=False):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    o = None if offset is None else np.ascontiguousarray(offset, dtype=np.int32)
    ctx._check(LIB.dda_unet_targets(ctx._h, ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                    ctypes.c_void_p(mask.data_ptr()), _ptr(d), None if o is None else _ptr(o),
                                    int(bool(residual))))


def dda_unet_warm_start(ctx: "Context", y, dims, p, offset=None, residual=False):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    o = None if offset is None else np.ascontiguousarray(offset, dtype=np.int32)
    ctx._check(LIB.dda_unet_warm_start(ctx._h, ctypes.c_void_p(y.data_ptr()), _ptr(d), None if o is None else _ptr(o),
                                       int(bool(residual)), ctypes.c_void_p(p.data_ptr())))


def dda_unet_residual_grad(ctx: "Context", y, gy, dims, weight=1.0, offset=None) -> float:
    """Adds weight * sum_b |E_b - A P0_b|^2/|E_b|^2 (P0 = alpha (E_inc + y)) to the returned loss and its gradient to gy."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    o = None if offset is None else np.ascontiguousarray(offset, dtype=np.int32)
    loss = ctypes.c_double()
    ctx._check(LIB.dda_unet_residual_grad(ctx._h, ctypes.c_void_p(y.data_ptr()), _ptr(d), None if o is None else _ptr(o),
                                          float(weight), ctypes.c_void_p(gy.data_ptr()), ctypes.byref(loss)))
    return float(loss.value)


def dda_orientation_grid(beta_deg, nbeta, theta_deg, ntheta, phi_deg, nphi):
    """(orientations [n, 3] radians (beta, Theta, Phi), weights [n]) of the guide's orientation sampling."""
    n = int(nbeta) * int(ntheta) * int(nphi)
    ori = np.zeros((n, 3))
    w = np.zeros(n)
    b = np.ascontiguousarray(beta_deg, dtype=np.float64)
    t = np.ascontiguousarray(theta_deg, dtype=np.float64)
    f = np.ascontiguousarray(phi_deg, dtype=np.float64)
    st = LIB.dda_orientation_grid(_ptr(b), int(nbeta), _ptr(t), int(ntheta), _ptr(f), int(nphi), _ptr(ori), _ptr(w))
    if st != DDA_OK:
        raise DDAError(st, "dda_orientation_grid failed")
    return ori, w


def dda_orientation_average(q, w, iorth: int = 2):
    """Weighted average over orientations of per-RHS results q [n_ori * iorth, ...]; returns [iorth, ...]."""
    wv = np.ascontiguousarray(w, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    tail = q.shape[1:] if q.shape[0] == len(wv) * iorth else q.shape[2:]
    nval = int(np.prod(tail)) if len(tail) else 1
    out = np.zeros((iorth,) + tuple(tail))
    st = LIB.dda_orientation_average(_ptr(wv), len(wv), int(iorth), _ptr(q), nval, _ptr(out))
    if st != DDA_OK:
        raise DDAError(st, "dda_orientation_average failed")
    return out


orientation_average = dda_orientation_average


def dda_selftest_bulk_wait(device: int = 0) -> bool:
    """True when the library's bounded bulk-copy wait gives up by itself on a barrier that never completes."""
    out = np.zeros(1, dtype=np.int32)
    st = LIB.dda_selftest_bulk_wait(int(device), _ptr(out))
    if st != DDA_OK:
        raise DDAError(st, "dda_selftest_bulk_wait failed")
    return bool(out[0])


def dda_probe_tc_dft(device: int = 0, nvec: int = 1 << 21, reps: int = 256):
    """{fp32_ms, tensor_ms, fp32_err, tensor_err} of `reps` DFT-8 stages on nvec vectors (measurement probe)."""
    out = np.zeros(4)
    st = LIB.dda_probe_tc_dft(int(device), int(nvec), int(reps), _ptr(out))
    if st != DDA_OK:
        raise DDAError(st, "dda_probe_tc_dft failed")
    return {"fp32_ms": out[0], "tensor_ms": out[1], "fp32_err": out[2], "tensor_err": out[3]}


def dda_kernel_launches() -> int:
    return int(LIB.dda_kernel_launches())


def dda_profile_matvec(ctx: "Context", nrhs: int, dtype: int = DDA_C64, iters: int = 20):
    """Mean ms of each pass of the product (3 or 5 passes), CUDA events on the context's stream."""
    ms = np.zeros(5)
    npass = ctypes.c_int()
    ctx._check(LIB.dda_profile_matvec(ctx._h, int(nrhs), int(dtype), int(iters), _ptr(ms), ctypes.byref(npass)))
    return ms[:npass.value]


def dda_schedule_info(ctx: "Context", dtype: int = DDA_C64):
    """(passes, fast, plane_threads, tuned_nrhs, ctas_per_plane, x_tile_rows, bulk_staged, x_components_per_cta,
    z_register_fused)."""
    info = np.zeros(12, dtype=np.int32)
    ctx._check(LIB.dda_schedule_info(ctx._h, int(dtype), _ptr(info)))
    return tuple(int(v) for v in info[:9])


def dda_solve_batch(ctxs, ps, solver="BICGSTAB", precision="MIXED", tol=1e-5, maxit=1000, inner_tol=0.0,
                    timeout_ms=0.0, check_every=8, normal_eq=False, precond="NONE", phi_reuse=False):
    """Solve several contexts concurrently; ps[i] complex128 [nrhs_i,3,N_i] CUDA tensors.

    Returns (list of per-context report lists, list of statuses, overall status)."""
    n = len(ctxs)
    for c, p in zip(ctxs, ps):
        c._dev_check(p, DDA_C128)
    o = dda_solve_opts(SOLVERS[solver.upper()], PRECISIONS[precision.upper()], tol, maxit, inner_tol, timeout_ms,
                       0, check_every, int(bool(normal_eq)), 1, PRECONDS[precond.upper()], int(bool(phi_reuse)))
    handles = (ctypes.c_void_p * n)(*[c._h.value for c in ctxs])
    bufs = (ctypes.c_void_p * n)(*[p.data_ptr() for p in ps])
    rep_arrays = [(dda_solve_report * c.nrhs)() for c in ctxs]
    reps = (ctypes.c_void_p * n)(*[ctypes.cast(r, ctypes.c_void_p).value for r in rep_arrays])
    sts = (ctypes.c_int * n)(*([-1] * n))
    overall = LIB.dda_solve_batch(handles, n, ctypes.byref(o), bufs, reps, sts)
    out = [[{k: getattr(r, k) for k, _ in dda_solve_report._fields_} for r in ra] for ra in rep_arrays]
    return out, list(sts), overall


def dda_version() -> str:
    return LIB.dda_version().decode()


def setup_workload(ctx: Context, w, pad=None):
    """Target, incidence, Green tensor and polarizability for a workload description."""
    ctx.dda_setup_shape(w.shape, w.shpar)
    kd, _ = ctx.dda_kd_from_x(w.x)
    ctx.dda_set_incident(kd, w.orientations, [[c[0], c[1]] for c in w.e01], w.iorth)
    if ctx.device >= 0:
        ctx.dda_build_green_fft(pad if pad is not None else w.pad)
    ctx.dda_set_polarizability(w.prescription, w.m)
    return kd
