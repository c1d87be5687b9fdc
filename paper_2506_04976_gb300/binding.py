"""ctypes binding of the C ABI in include/pet_gb300.h (argument marshalling only).

Every compute step runs in the CUDA library ``_build/libpetgb300.so``.  Importing this
module loads the library and raises if it is missing: there is no CPU fallback.
Tensors passed in must be contiguous CUDA tensors of the stated dtype; work is
enqueued on torch's current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpetgb300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"CUDA library {LIB_PATH} is missing; build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")

_lib = C.CDLL(LIB_PATH)

PET_Y_U16, PET_Y_U32, PET_Y_F32 = 0, 1, 2
SGD, SAGA, SVRG = 0, 1, 2
STEP_CONST, STEP_VANISH, STEP_ALG1, STEP_BB, STEP_ALG2 = 0, 1, 2, 3, 4
SAMPLE_PERM, SAMPLE_REPLACE, SAMPLE_HM, SAMPLE_COFACTOR, SAMPLE_IMPORTANCE = 0, 1, 2, 3, 4
GRAD_DETERMINISTIC, OBJ_ONLY = 1, 2

STATUS = {0: "PET_OK", 1: "PET_ERR_ARG", 2: "PET_ERR_SHAPE", 3: "PET_ERR_INFEASIBLE",
          4: "PET_ERR_TIMEOUT", 5: "PET_ERR_CUDA", 6: "PET_ERR_UNSUPPORTED",
          7: "PET_ERR_STATE", 8: "PET_ERR_NOMEM"}


class PetError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} "
                         f"({_lib.pet_status_str(status).decode()})")


class Geometry(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("nrad", C.c_int), ("nview", C.c_int), ("nplane", C.c_int), ("ntof", C.c_int),
        ("drad", C.c_double), ("rdet", C.c_double),
        ("z1", C.POINTER(C.c_double)), ("z2", C.POINTER(C.c_double)),
        ("tof_sigma", C.c_double), ("tof_bin", C.c_double),
        ("nsubsets", C.c_int),
        ("res_fwhm", C.c_double),
    ]


class RdpParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("gamma", C.c_float), ("eps", C.c_float), ("scale", C.c_float),
        ("kappa", C.c_void_p),
    ]


class SolverOpts(C.Structure):
    _fields_ = [
        ("algo", C.c_int), ("omega", C.c_int), ("step_rule", C.c_int),
        ("tau0", C.c_double), ("eta", C.c_double),
        ("precond_kind", C.c_int), ("alpha", C.c_double), ("delta_rel", C.c_double),
        ("pc_iters", C.POINTER(C.c_longlong)), ("n_pc", C.c_int),
        ("beta", C.c_float), ("gamma", C.c_float), ("eps", C.c_float),
        ("kappa", C.c_void_p),
        ("seed", C.c_ulonglong),
        ("order", C.POINTER(C.c_int)), ("norder", C.c_longlong),
        ("use_graph", C.c_int), ("deterministic", C.c_int),
        ("sampling", C.c_int), ("low_memory", C.c_int), ("bb_until", C.c_longlong),
    ]


_vp = C.c_void_p
_sigs = {
    "pet_status_str": (C.c_char_p, [C.c_int]),
    "pet_plan_create": (C.c_int, [C.POINTER(Geometry), C.POINTER(_vp)]),
    "pet_plan_destroy": (None, [_vp]),
    "pet_plan_set_data": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp, _vp]),
    "pet_plan_set_counts": (C.c_int, [_vp, _vp, C.c_int, _vp]),
    "pet_copy_to_device": (C.c_int, [_vp, _vp, C.c_size_t, C.c_int, _vp]),
    "pet_subset_size": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int)]),
    "pet_plan_mult": (_vp, [_vp]),
    "pet_plan_sensitivity": (_vp, [_vp, C.c_int]),
    "pet_plan_check": (C.c_int, [_vp, _vp]),
    "pet_plan_set_grad_shape": (C.c_int, [_vp, C.c_int, C.c_int]),
    "pet_plan_autotune": (C.c_int, [_vp, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pet_plan_set_rdp_tile": (C.c_int, [_vp, C.c_int]),
    "pet_forward": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    "pet_back": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int, _vp]),
    "pet_objective_grad": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.POINTER(RdpParams), C.c_int, _vp]),
    "pet_em_update": (C.c_int, [_vp, C.c_int, _vp, _vp]),
    "pet_ratio": (C.c_int, [_vp, C.c_int, _vp, _vp, _vp, C.c_int, _vp]),
    "pet_rdp": (C.c_int, [C.POINTER(RdpParams), _vp, _vp, _vp, _vp, C.c_int, _vp]),
    "pet_precond": (C.c_int, [_vp, _vp, _vp, C.c_float, C.c_float, _vp, _vp]),
    "pet_nrmse": (C.c_int, [_vp, _vp, _vp, _vp, C.c_size_t, _vp, _vp]),
    "pet_solver_create": (C.c_int, [_vp, C.POINTER(SolverOpts), C.POINTER(_vp)]),
    "pet_solver_destroy": (None, [_vp]),
    "pet_solver_set_image": (C.c_int, [_vp, _vp, _vp]),
    "pet_solver_image": (_vp, [_vp]),
    "pet_solver_run": (C.c_int, [_vp, C.c_longlong, _vp]),
    "pet_solver_taus": (C.c_longlong, [_vp, C.POINTER(C.c_double), C.c_longlong]),
    "pet_solver_iteration": (C.c_longlong, [_vp]),
    "pet_solver_subsets": (C.c_longlong, [_vp, C.POINTER(C.c_int), C.c_longlong]),
    "pet_solver_profile": (C.c_int, [_vp, C.c_int]),
    "pet_launch_count": (C.c_longlong, []),
    "pet_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, C.POINTER(_vp)]),
    "pet_batch_destroy": (None, [_vp]),
    "pet_batch_run": (C.c_int, [_vp, C.c_longlong, _vp]),
    "pet_batch_set_grad_shape": (C.c_int, [_vp, C.c_int, C.c_int]),
    "pet_batch_autotune": (C.c_int, [_vp, _vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pet_solver_kernel_time": (C.c_int, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _ck(status, where):
    if status != 0:
        raise PetError(status, where)


def _stream():
    return _vp(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype=torch.float32, numel=None):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return _vp(t.data_ptr())


_YT = {torch.int16: PET_Y_U16, torch.uint16: PET_Y_U16, torch.int32: PET_Y_U32,
       torch.uint32: PET_Y_U32, torch.float32: PET_Y_F32}


def rdp_params(shape, spacing, gamma, eps, scale, kappa=None):
    nz, ny, nx = shape
    return RdpParams(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]),
                     float(gamma), float(eps), float(scale),
                     _vp(kappa.data_ptr()) if kappa is not None else None)


class Plan:
    """A projector plan (pet_plan) for one scanner geometry and image grid."""

    def __init__(self, geom, nsubsets):
        self._z1 = np.ascontiguousarray(geom["z1"], np.float64)
        self._z2 = np.ascontiguousarray(geom["z2"], np.float64)
        self.geom = dict(geom)
        self.nsub = int(nsubsets)
        T = int(geom.get("ntof", 1))
        self.T = T if T > 1 else 1
        g = Geometry(int(geom["nx"]), int(geom["ny"]), int(geom["nz"]),
                     float(geom["dx"]), float(geom["dy"]), float(geom["dz"]),
                     int(geom["nrad"]), int(geom["nview"]), len(self._z1), T,
                     float(geom["drad"]), float(geom["rdet"]),
                     self._z1.ctypes.data_as(C.POINTER(C.c_double)),
                     self._z2.ctypes.data_as(C.POINTER(C.c_double)),
                     float(geom.get("tof_sigma", 1.0)), float(geom.get("tof_bin", 1.0)),
                     self.nsub, float(geom.get("res_fwhm", 0.0)))
        h = _vp()
        _ck(_lib.pet_plan_create(C.byref(g), C.byref(h)), "pet_plan_create")
        self._h = h
        self.img_shape = (g.nz, g.ny, g.nx)
        self.N = g.nz * g.ny * g.nx
        self.lor_shape = (g.nview, g.nplane, g.nrad)
        self.sino_shape = (g.nview, g.nplane, g.nrad, self.T)
        self.spacing = (g.dx, g.dy, g.dz)
        self._keep = []

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.pet_plan_destroy(h)
            self._h = None

    def subset_views(self, s):
        n = C.c_int()
        _ck(_lib.pet_subset_size(self._h, int(s), C.byref(n)), "pet_subset_size")
        return n.value

    def subset_shape(self, s):
        return (self.subset_views(s),) + self.sino_shape[1:]

    def set_data(self, y, r, mu=None, sens=None):
        """y: counts (uint16 / int32 / float32) and r: float32, both (V,P,R,T) on the GPU."""
        if y.dtype not in _YT:
            raise ValueError("y must be uint16, int32/uint32 or float32")
        nbin = int(np.prod(self.sino_shape))
        _ck(_lib.pet_plan_set_data(self._h, _ptr(y, None, nbin), _YT[y.dtype], _ptr(r, numel=nbin),
                                   _ptr(mu, numel=self.N) if mu is not None else None,
                                   _ptr(sens, numel=nbin // self.T) if sens is not None else None,
                                   _stream()), "pet_plan_set_data")
        self._keep = [y, r]

    def set_counts(self, y, r):
        """Rebinds counts and background only (the next frame on the same scanner and
        attenuation map): no device work, the factors and sensitivities are kept."""
        if y.dtype not in _YT:
            raise ValueError("y must be uint16, int32/uint32 or float32")
        nbin = int(np.prod(self.sino_shape))
        _ck(_lib.pet_plan_set_counts(self._h, _ptr(y, None, nbin), _YT[y.dtype], _ptr(r, numel=nbin)),
            "pet_plan_set_counts")
        self._keep = [y, r]

    def mult(self):
        p = _lib.pet_plan_mult(self._h)
        return _wrap(p, self.lor_shape)

    def sensitivity(self, s=-1):
        return _wrap(_lib.pet_plan_sensitivity(self._h, int(s)), self.img_shape)

    def set_grad_shape(self, planes_per_thread=0, parts=0):
        _ck(_lib.pet_plan_set_grad_shape(self._h, int(planes_per_thread), int(parts)),
            "pet_plan_set_grad_shape")

    def set_rdp_tile(self, slices=0):
        """RDP stencil tile of the plan's prior evaluations: 2, 4 or 8 slices (0: default)."""
        _ck(_lib.pet_plan_set_rdp_tile(self._h, int(slices)), "pet_plan_set_rdp_tile")

    def autotune(self):
        """Times the fused-gradient launch shapes and the RDP stencil tiles and keeps the
        fastest; returns the gradient's shape."""
        k, sp = C.c_int(), C.c_int()
        _ck(_lib.pet_plan_autotune(self._h, _stream(), C.byref(k), C.byref(sp)), "pet_plan_autotune")
        return k.value, sp.value

    def check(self):
        _ck(_lib.pet_plan_check(self._h, _stream()), "pet_plan_check")

    def forward(self, x, s=-1, out=None):
        shp = self.subset_shape(s) if s >= 0 else self.sino_shape
        out = torch.empty(shp, device=x.device, dtype=torch.float32) if out is None else out
        _ck(_lib.pet_forward(self._h, int(s), _ptr(x, numel=self.N), _ptr(out, numel=int(np.prod(shp))),
                             _stream()), "pet_forward")
        return out

    def back(self, q, s=-1, deterministic=False, out=None):
        shp = self.subset_shape(s) if s >= 0 else self.sino_shape
        out = torch.empty(self.img_shape, device=q.device, dtype=torch.float32) if out is None else out
        _ck(_lib.pet_back(self._h, int(s), _ptr(q, numel=int(np.prod(shp))), _ptr(out, numel=self.N),
                          int(bool(deterministic)), _stream()), "pet_back")
        return out

    def objective_grad(self, x, s=-1, prior=None, deterministic=False, obj_only=False, g=None,
                       want_obj=True):
        """(f_s(x) as a 0-d float64 CUDA tensor, gradient) with prior = (beta_scale, gamma, eps[, kappa])."""
        g = None if obj_only else (torch.empty(self.img_shape, device=x.device) if g is None else g)
        obj = torch.zeros((), device=x.device, dtype=torch.float64) if want_obj else None
        rp = None
        if prior is not None:
            scale, gamma, eps = prior[:3]
            kappa = prior[3] if len(prior) > 3 else None
            rp = C.byref(rdp_params(self.img_shape, self.spacing, gamma, eps, scale, kappa))
        flags = (GRAD_DETERMINISTIC if deterministic else 0) | (OBJ_ONLY if obj_only else 0)
        _ck(_lib.pet_objective_grad(self._h, int(s), _ptr(x, numel=self.N),
                                    _ptr(g, numel=self.N) if g is not None else None,
                                    _ptr(obj, torch.float64) if obj is not None else None,
                                    rp, flags, _stream()), "pet_objective_grad")
        return obj, g

    def ratio(self, ax, s=-1, want_q=True, want_obj=True):
        """(sum of KL terms as a 0-d float64 tensor, q = 1 - y/(ax + r)) from ax = A_s x."""
        shp = self.subset_shape(s) if s >= 0 else self.sino_shape
        q = torch.empty(shp, device=ax.device) if want_q else None
        obj = torch.zeros((), device=ax.device, dtype=torch.float64) if want_obj else None
        _ck(_lib.pet_ratio(self._h, int(s), _ptr(ax, numel=int(np.prod(shp))),
                           _ptr(q) if q is not None else None,
                           _ptr(obj, torch.float64) if obj is not None else None, 0, _stream()),
            "pet_ratio")
        return obj, q

    def em_update(self, x, s):
        _ck(_lib.pet_em_update(self._h, int(s), _ptr(x, numel=self.N), _stream()), "pet_em_update")
        return x

    def precond(self, x, hdiag_betaS=None, alpha=1.0, delta_rel=1e-6, out=None):
        out = torch.empty_like(x) if out is None else out
        _ck(_lib.pet_precond(self._h, _ptr(x, numel=self.N),
                             _ptr(hdiag_betaS, numel=self.N) if hdiag_betaS is not None else None,
                             float(alpha), float(delta_rel), _ptr(out, numel=self.N), _stream()),
            "pet_precond")
        return out


def launch_count():
    """Kernels launched by the library so far (graph replays count their kernel nodes)."""
    return _lib.pet_launch_count()


def copy_to_device(dst, src, max_blocks=0):
    """Kernel copy of a pinned host tensor into a CUDA tensor of the same dtype and size
    (pet_copy_to_device) on the current stream; max_blocks bounds its grid (0: four
    blocks per SM)."""
    if not (dst.is_cuda and dst.is_contiguous()):
        raise ValueError("dst: expected a contiguous CUDA tensor")
    if src.is_cuda or not src.is_contiguous() or not src.is_pinned():
        raise ValueError("src: expected a contiguous pinned host tensor")
    if src.dtype != dst.dtype or src.numel() != dst.numel():
        raise ValueError("src and dst differ in dtype or size")
    _ck(_lib.pet_copy_to_device(_vp(dst.data_ptr()), _vp(src.data_ptr()), src.numel() * src.element_size(),
                                int(max_blocks), _stream()), "pet_copy_to_device")


def _wrap(ptr, shape):
    """Device buffer owned by the library -> a torch view (no copy, no ownership)."""
    if not ptr:
        raise PetError(1, "null buffer")
    n = int(np.prod(shape))

    class _Iface:
        __cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (ptr, False),
                                    "version": 3, "strides": None}

    return torch.as_tensor(_Iface(), device="cuda")


RDP_ACC_GRAD, RDP_ACC_VAL = 1, 2


def rdp(x, spacing, gamma, eps, scale=1.0, kappa=None, want_grad=True, want_hdiag=True,
        want_val=True, grad_out=None, accumulate=False, val_out=None, accumulate_val=False):
    """(scale*S(x), scale*grad S, scale*diag Hess S) of eq. 3 on the GPU.  accumulate adds
    the gradient into grad_out; accumulate_val adds scale*S into val_out (a 0-d float64
    CUDA tensor) instead of overwriting it."""
    g = (torch.empty_like(x) if grad_out is None else grad_out) if want_grad else None
    h = torch.empty_like(x) if want_hdiag else None
    v = (torch.zeros((), device=x.device, dtype=torch.float64) if val_out is None else val_out) \
        if want_val else None
    p = rdp_params(tuple(x.shape), spacing, gamma, eps, scale, kappa)
    flags = (RDP_ACC_GRAD if accumulate else 0) | (RDP_ACC_VAL if accumulate_val else 0)
    _ck(_lib.pet_rdp(C.byref(p), _ptr(x), _ptr(g) if g is not None else None,
                     _ptr(h) if h is not None else None, _ptr(v, torch.float64) if v is not None else None,
                     flags, _stream()), "pet_rdp")
    return v, g, h


def nrmse(x, ref, mask, bg):
    out = torch.zeros((), device=x.device, dtype=torch.float64)
    _ck(_lib.pet_nrmse(_ptr(x), _ptr(ref), _ptr(mask, torch.uint8), _ptr(bg, torch.uint8),
                       x.numel(), _ptr(out, torch.float64), _stream()), "pet_nrmse")
    return out


class Solver:
    """Preconditioned SGD / SAGA / SVRG (eq. 6-9, Algorithm 1) on a Plan."""

    def __init__(self, plan: Plan, *, algo=SVRG, omega=2, step_rule=STEP_VANISH, tau0=1.0, eta=0.02,
                 precond_kind=1, alpha=1.0, delta_rel=1e-6, pc_iters=(0,), beta=0.1, gamma=2.0,
                 eps=1e-3, kappa=None, seed=0, order=None, use_graph=True, deterministic=False,
                 sampling=SAMPLE_PERM, low_memory=False, bb_until=0):
        self.plan = plan
        self._pc = np.ascontiguousarray(pc_iters, np.int64)
        self._order = np.ascontiguousarray(order, np.int32) if order is not None else None
        self._kappa = kappa
        o = SolverOpts(algo, omega, step_rule, tau0, eta, precond_kind, alpha, delta_rel,
                       self._pc.ctypes.data_as(C.POINTER(C.c_longlong)), len(self._pc),
                       beta, gamma, eps, _vp(kappa.data_ptr()) if kappa is not None else None,
                       seed,
                       self._order.ctypes.data_as(C.POINTER(C.c_int)) if self._order is not None else None,
                       len(self._order) if self._order is not None else 0,
                       int(bool(use_graph)), int(bool(deterministic)), int(sampling), int(bool(low_memory)),
                       int(bb_until))
        h = _vp()
        _ck(_lib.pet_solver_create(plan._h, C.byref(o), C.byref(h)), "pet_solver_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.pet_solver_destroy(h)
            self._h = None

    def set_image(self, x):
        _ck(_lib.pet_solver_set_image(self._h, _ptr(x, numel=self.plan.N), _stream()),
            "pet_solver_set_image")

    def run(self, niter):
        _ck(_lib.pet_solver_run(self._h, int(niter), _stream()), "pet_solver_run")

    def image(self):
        return _wrap(_lib.pet_solver_image(self._h), self.plan.img_shape)

    @property
    def k(self):
        return _lib.pet_solver_iteration(self._h)

    def profile(self, enable=True):
        _ck(_lib.pet_solver_profile(self._h, int(bool(enable))), "pet_solver_profile")

    def kernel_time(self):
        """(total ms, launches) of the fused subset-gradient kernel since the last call."""
        ms, n = C.c_double(), C.c_longlong()
        _ck(_lib.pet_solver_kernel_time(self._h, C.byref(ms), C.byref(n)), "pet_solver_kernel_time")
        return ms.value, n.value

    def taus(self):
        torch.cuda.current_stream().synchronize()
        n = self.k
        buf = (C.c_double * max(n, 1))()
        c = _lib.pet_solver_taus(self._h, buf, n)
        return np.array(buf[:c])

    def subsets(self):
        """Subset used by each iteration so far (-1 at SVRG snapshot refreshes)."""
        torch.cuda.current_stream().synchronize()
        n = self.k
        buf = (C.c_int * max(n, 1))()
        c = _lib.pet_solver_subsets(self._h, buf, n)
        return np.array(buf[:c], dtype=np.int32)


class Batch:
    """Independent reconstructions advanced together (pet_batch_*)."""

    def __init__(self, solvers, iters_per_graph=8):
        self.solvers = list(solvers)
        arr = (_vp * len(self.solvers))(*[sv._h for sv in self.solvers])
        h = _vp()
        _ck(_lib.pet_batch_create(arr, len(self.solvers), int(iters_per_graph), C.byref(h)), "pet_batch_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.pet_batch_destroy(h)
            self._h = None

    def run(self, niter):
        _ck(_lib.pet_batch_run(self._h, int(niter), _stream()), "pet_batch_run")

    def set_grad_shape(self, planes_per_thread, parts):
        _ck(_lib.pet_batch_set_grad_shape(self._h, int(planes_per_thread), int(parts)), "pet_batch_set_grad_shape")

    def autotune(self):
        k, sp = C.c_int(), C.c_int()
        _ck(_lib.pet_batch_autotune(self._h, _stream(), C.byref(k), C.byref(sp)), "pet_batch_autotune")
        return k.value, sp.value
