"""FP64 CPU oracle for the subset-gradient path of RDP-regularised PET reconstruction.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may load this package; the product library never does.  The C
source (``pet_oracle.c``) shares nothing with the CUDA library.  This wrapper converts
numpy arrays to pointers and back; all arithmetic is in the C file.

Paper sections followed: forward model and KL data term (Sec. 1.1-1.2, eq. 1-2), RDP
(eq. 3, Appendix A.1), subset objective (eq. 5), preconditioned proximal stochastic
gradient step (eq. 6), SAGA (eq. 7), SVRG (eq. 9, Algorithm 1), preconditioners
(Sec. 2.3, eq. 8), stepsizes (Sec. 2.2, Table 1), sampling (Sec. 2.4), OSEM
initialisation and NRMSE (Sec. 3.1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pet_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

STEP_CONST, STEP_VANISH, STEP_ALG1, STEP_BB, STEP_ALG2 = 0, 1, 2, 3, 4
SGD, SAGA, SVRG = 0, 1, 2
SAMPLE_PERM, SAMPLE_REPLACE, SAMPLE_HM, SAMPLE_COFACTOR, SAMPLE_IMPORTANCE = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Geom(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("nrad", C.c_int), ("nview", C.c_int), ("nplane", C.c_int), ("ntof", C.c_int),
        ("drad", C.c_double), ("rdet", C.c_double),
        ("z1", C.POINTER(C.c_double)), ("z2", C.POINTER(C.c_double)),
        ("tof_sigma", C.c_double), ("tof_bin", C.c_double),
        ("res_fwhm", C.c_double),
    ]


class _Opts(C.Structure):
    _fields_ = [
        ("algo", C.c_int), ("nsub", C.c_int), ("niter", C.c_long), ("omega", C.c_int),
        ("step_rule", C.c_int), ("tau0", C.c_double), ("eta", C.c_double),
        ("precond_kind", C.c_int), ("alpha", C.c_double), ("delta_rel", C.c_double),
        ("pc_iters", C.POINTER(C.c_long)), ("n_pc", C.c_int),
        ("beta", C.c_double), ("gamma", C.c_double), ("eps", C.c_double),
        ("kappa", C.POINTER(C.c_double)),
        ("order", C.POINTER(C.c_int)),
        ("sampling", C.c_int), ("sample_seed", C.c_uint64),
        ("subsets_out", C.POINTER(C.c_int)), ("bb_until", C.c_long),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.o_kl_term.restype = C.c_double
        _lib.o_tof_weight.restype = C.c_double
        _lib.o_data_grad.restype = C.c_double
        _lib.o_data_grad_views.restype = C.c_double
        _lib.o_rdp.restype = C.c_double
        _lib.o_nrmse.restype = C.c_double
        _lib.o_step_alg1.restype = C.c_double
        _lib.o_step_alg2.restype = C.c_double
        _lib.o_splitmix64.restype = C.c_uint64
        _lib.o_splitmix64_at.restype = C.c_uint64
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Geometry:
    """Holds a C geometry struct plus the arrays it points to.

    ``geom`` is a mapping with keys nx, ny, nz, dx, dy, dz, nrad, nview, drad, rdet,
    z1, z2 (per-plane endpoint axial positions, mm), ntof, tof_sigma, tof_bin and
    optionally res_fwhm (image-space Gaussian resolution model, mm; default none).
    """

    def __init__(self, geom):
        self.z1 = _f64(geom["z1"])
        self.z2 = _f64(geom["z2"])
        self.ntof = int(geom.get("ntof", 1))
        self.s = _Geom(int(geom["nx"]), int(geom["ny"]), int(geom["nz"]),
                       float(geom["dx"]), float(geom["dy"]), float(geom["dz"]),
                       int(geom["nrad"]), int(geom["nview"]), len(self.z1), self.ntof,
                       float(geom["drad"]), float(geom["rdet"]), _d(self.z1), _d(self.z2),
                       float(geom.get("tof_sigma", 1.0)), float(geom.get("tof_bin", 1.0)),
                       float(geom.get("res_fwhm", 0.0)))
        g = self.s
        self.img_shape = (g.nz, g.ny, g.nx)
        self.T = self.ntof if self.ntof > 1 else 1
        self.sino_shape = (g.nview, g.nplane, g.nrad, self.T)
        self.lor_shape = (g.nview, g.nplane, g.nrad)

    @property
    def ref(self):
        return C.byref(self.s)


def gauss_filter(x, spacing, fwhm):
    """G x: separable Gaussian of the given FWHM (mm), zero outside the image."""
    x = _f64(x)
    out = np.empty_like(x)
    nz, ny, nx = x.shape
    lib().o_gauss_filter(nx, ny, nz, C.c_double(spacing[0]), C.c_double(spacing[1]), C.c_double(spacing[2]),
                         C.c_double(fwhm), _d(x), _d(out))
    return out


def subset_views(nview, nsub, s):
    out = np.zeros(nview, np.int32)
    c = lib().o_subset_views(nview, nsub, s, _i(out))
    return out[:c].copy()


def driving_axis(G: Geometry, v: int) -> int:
    return lib().o_driving_axis(G.ref, v)


def lor_entries(G: Geometry, v, p, r):
    """Joseph row of LOR (v,p,r): (voxel indices, weights in mm, positions t in mm)."""
    me = 4 * max(G.s.nx, G.s.ny, G.s.nz) + 4
    vox = np.zeros(me, np.int32)
    wt = np.zeros(me)
    tp = np.zeros(me)
    ne = lib().o_lor_entries(G.ref, v, p, r, _i(vox), _d(wt), _d(tp))
    if ne < 0:
        raise ValueError("axial axis would drive this LOR")
    return vox[:ne].copy(), wt[:ne].copy(), tp[:ne].copy()


def tof_weight(G: Geometry, b, t):
    return lib().o_tof_weight(G.ref, int(b), C.c_double(t))


def project(G: Geometry, x, views=None):
    """Geometric projection P x (no multiplicative factors) over ``views``."""
    views = np.arange(G.s.nview, dtype=np.int32) if views is None else np.asarray(views, np.int32)
    x = _f64(x)
    out = np.zeros((len(views), G.s.nplane, G.s.nrad, G.T))
    if lib().o_project(G.ref, _i(views), len(views), _d(x), _d(out)) != 0:
        raise ValueError("axial axis would drive a LOR")
    return out


def project_lors(G: Geometry, x, vpr):
    """Geometric projection of listed LORs; vpr is an (L, 3) int array of (view, plane, radial)."""
    vpr = np.ascontiguousarray(vpr, np.int32)
    x = _f64(x)
    out = np.zeros((len(vpr), G.T))
    if lib().o_project_lors(G.ref, _i(vpr), len(vpr), _d(x), _d(out)) != 0:
        raise ValueError("axial axis would drive a LOR")
    return out


def backproject(G: Geometry, q, views=None):
    views = np.arange(G.s.nview, dtype=np.int32) if views is None else np.asarray(views, np.int32)
    q = _f64(q)
    out = np.zeros(G.img_shape)
    if lib().o_backproject(G.ref, _i(views), len(views), _d(q), _d(out)) != 0:
        raise ValueError("axial axis would drive a LOR")
    return out


def multiplicative(G: Geometry, mu=None, sens=None):
    """m = sens * exp(-P mu) per LOR, shape (V, P, R)."""
    m = np.zeros(G.lor_shape)
    mu_keep = _f64(mu) if mu is not None else None
    sens_keep = _f64(sens) if sens is not None else None
    if lib().o_multiplicative(G.ref, _d(mu_keep) if mu_keep is not None else None,
                              _d(sens_keep) if sens_keep is not None else None, _d(m)) != 0:
        raise ValueError("axial axis would drive a LOR")
    return m


def kl_term(s, t):
    return lib().o_kl_term(C.c_double(s), C.c_double(t))


def data_grad(G: Geometry, nsub, s, x, m, r, y, want_grad=True):
    """(D_s(x), grad D_s(x)) for subset s (s=-1: all views)."""
    x, m, r, y = _f64(x), _f64(m), _f64(r), _f64(y)
    g = np.zeros(G.img_shape) if want_grad else None
    val = lib().o_data_grad(G.ref, nsub, s, _d(x), _d(m), _d(r), _d(y), _d(g) if want_grad else None)
    return val, g


def data_grad_views(G: Geometry, views, x, m_c, r_c, y_c, want_grad=True):
    """(D(x), grad D(x)) over the listed views with compact data: m_c (nv, P, R), r_c and
    y_c (nv, P, R, T) for those views in order (P, R, T of G's plane list)."""
    views = np.ascontiguousarray(views, np.int32)
    x, m_c, r_c, y_c = _f64(x), _f64(m_c), _f64(r_c), _f64(y_c)
    nv = len(views)
    if m_c.size != nv * G.s.nplane * G.s.nrad or r_c.size != m_c.size * G.T or y_c.size != r_c.size:
        raise ValueError("compact data do not match the views and the geometry")
    g = np.zeros(G.img_shape) if want_grad else None
    val = lib().o_data_grad_views(G.ref, _i(views), nv, _d(x), _d(m_c), _d(r_c), _d(y_c),
                                  _d(g) if want_grad else None)
    if not np.isfinite(val) and np.all(np.isfinite(r_c)):
        raise ValueError("axial axis would drive a LOR, or infeasible data")
    return val, g


def sensitivity(G: Geometry, nsub, s, m):
    m = _f64(m)
    out = np.zeros(G.img_shape)
    lib().o_sensitivity(G.ref, nsub, s, _d(m), _d(out))
    return out


def rdp(x, spacing, gamma, eps, kappa=None):
    """(S(x), grad S(x), diag Hess S(x)) for a (nz, ny, nx) image."""
    x = _f64(x)
    nz, ny, nx = x.shape
    grad = np.zeros_like(x)
    hd = np.zeros_like(x)
    kap = _f64(kappa) if kappa is not None else None
    S = lib().o_rdp(nx, ny, nz, C.c_double(spacing[0]), C.c_double(spacing[1]),
                    C.c_double(spacing[2]), C.c_double(gamma), C.c_double(eps),
                    _d(kap) if kap is not None else None,
                    _d(x), _d(grad), _d(hd))
    return S, grad, hd


def precond(x, sens, hdiag_betaS=None, alpha=1.0, delta=0.0, kind=1):
    x, sens = _f64(x), _f64(sens)
    h = _f64(hdiag_betaS) if hdiag_betaS is not None else np.zeros_like(x)
    D = np.zeros_like(x)
    lib().o_precond(C.c_size_t(x.size), kind, _d(x), _d(sens), _d(h), C.c_double(alpha),
                    C.c_double(delta), _d(D))
    return D


def splitmix64_stream(seed, count):
    st = C.c_uint64(seed)
    return [lib().o_splitmix64(C.byref(st)) for _ in range(count)]


def subset_order(seed, nsub, niter, kind=SAMPLE_PERM):
    """Subset per iteration under a sampling rule of Sec. 2.4 (not importance)."""
    out = np.zeros(niter, np.int32)
    if kind == SAMPLE_PERM:
        lib().o_subset_order(C.c_uint64(seed), nsub, niter, _i(out))
    elif lib().o_subset_order_kind(kind, C.c_uint64(seed), nsub, niter, _i(out)) != 0:
        raise ValueError(f"no precomputed order for sampling rule {kind}")
    return out


def splitmix64_at(seed, k):
    return lib().o_splitmix64_at(C.c_uint64(seed), C.c_long(k))


def cofactor_generators(n):
    out = np.zeros(max(n, 1), np.int32)
    c = lib().o_cofactor_generators(n, _i(out))
    return out[:c].copy()


def draw_index(p, u):
    p = _f64(p)
    return lib().o_draw_index(_d(p), len(p), C.c_double(u))


def step_alg1(k):
    return lib().o_step_alg1(C.c_long(k))


def step_alg2(k, nsub, tau_bb):
    return lib().o_step_alg2(C.c_long(k), nsub, C.c_double(tau_bb))


def solve(G: Geometry, x0, m, r, y, sens, *, algo, nsub, niter, order, omega=2,
          step_rule=STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1, alpha=1.0,
          delta_rel=1e-6, pc_iters=(0,), beta=0.1, gamma=2.0, eps=1e-3, kappa=None,
          snap_every=0, sampling=SAMPLE_PERM, sample_seed=0, subsets_out=None, bb_until=0):
    """Runs SGD/SAGA/SVRG (eq. 6-9, Algorithm 1) from x0; returns (x, taus, snaps).
    With sampling=SAMPLE_IMPORTANCE (SVRG) the subsets are drawn inside from
    sample_seed and `order` is ignored; subsets_out (int32 array of length niter, may
    be None) receives the subset of every iteration (-1 at snapshot refreshes).  bb_until
    > 0 recomputes the BB step only at refreshes k <= bb_until (Table 1: epochs 2, 4, 6)."""
    x = _f64(x0).copy()
    m, r, y, sens = _f64(m), _f64(r), _f64(y), _f64(sens)
    order = np.ascontiguousarray(order, np.int32)
    pcs = np.ascontiguousarray(pc_iters, np.int64)
    kap = _f64(kappa) if kappa is not None else None
    o = _Opts(algo, nsub, niter, omega, step_rule, tau0, eta, precond_kind, alpha, delta_rel,
              pcs.ctypes.data_as(C.POINTER(C.c_long)), len(pcs), beta, gamma, eps,
              _d(kap) if kap is not None else None, _i(order), sampling, C.c_uint64(sample_seed),
              _i(subsets_out) if subsets_out is not None else None, C.c_long(bb_until))
    taus = np.zeros(niter)
    nsnap = niter // snap_every if snap_every > 0 else 0
    snaps = np.zeros((max(nsnap, 1),) + x.shape)
    lib().o_solve(G.ref, C.byref(o), _d(m), _d(r), _d(y), _d(sens), _d(x), _d(taus),
                  _d(snaps) if nsnap else None, C.c_long(snap_every))
    return x, taus, snaps[:nsnap]


def em_update(G: Geometry, nsub, s, m, r, y, x):
    """One OSEM sub-iteration on subset s (MLEM when nsub == 1); returns the new x."""
    x = _f64(x).copy()
    m, r, y = _f64(m), _f64(r), _f64(y)
    lib().o_em_update(G.ref, nsub, s, _d(m), _d(r), _d(y), _d(x))
    return x


def nrmse(x, ref, mask, bg):
    x, ref = _f64(x), _f64(ref)
    mask = np.ascontiguousarray(mask, np.uint8)
    bg = np.ascontiguousarray(bg, np.uint8)
    return lib().o_nrmse(C.c_size_t(x.size), _d(x), _d(ref),
                         mask.ctypes.data_as(C.POINTER(C.c_ubyte)),
                         bg.ctypes.data_as(C.POINTER(C.c_ubyte)))
