"""The image-space resolution model (Sec. 3.1, a 4 mm Gaussian; system matrix P G) in
the CUDA operators and solver against the FP64 oracle with the same model.

Tolerances as for the operators without the model (the separable FP32 passes add
~1e-7 relative): projections and backprojections 1e-5 relative L2 per view / image,
gradients against the scale of A^T 1, solver trajectories 1e-4 relative L2."""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, torch.float32)


class Case:
    def __init__(self, name, **over):
        from paper_2506_04976_gb300 import binding as pet
        self.p = synth.make_problem(name, 4, **over)
        self.g = dict(self.p["geom"], res_fwhm=4.0)
        self.n = self.p["nsub"]
        self.plan = pet.Plan(self.g, self.n)
        self.mu32 = self.p["mu"].astype(np.float32)
        self.sens32 = self.p["sens"].astype(np.float32)
        self.plan.set_data(torch.from_numpy(self.p["y"].astype(np.int32)).to(DEV), _t(self.p["r"]),
                           _t(self.mu32), _t(self.sens32))
        self.G = O.Geometry(self.g)
        self.m = O.multiplicative(self.G, self.mu32, self.sens32)
        self.x = np.maximum(self.p["x_true"], 0.05 * self.p["x_true"].max()).astype(np.float32)
        self.xt = _t(self.x)


_C = {}


def case(key):
    if key not in _C:
        spec = {"c1": ("c1", {}), "3d": ("c2", dict(nx=40, nz=23, nrad=70, nview=36, nsub=6)),
                "tof": ("c3", dict(nx=40, nz=23, nrad=70, nview=36, nsub=6))}[key]
        _C[key] = Case(spec[0], **spec[1])
    return _C[key]


def _close(gpu, ref, rel_l2=1e-5, rel_el=1e-4, abs_frac=1e-5):
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    d = np.abs(gpu - ref)
    assert np.linalg.norm(d) <= rel_l2 * np.linalg.norm(ref)
    assert (d <= rel_el * np.abs(ref) + abs_frac * np.abs(ref).max()).all(), d.max()


@pytest.mark.parametrize("key", ["c1", "3d", "tof"])
def test_forward_and_back_with_resolution_model(key):
    c = case(key)
    s = 1
    views = O.subset_views(c.g["nview"], c.n, s)
    ax = c.plan.forward(c.xt, s).cpu().numpy()
    ref = c.m[views][..., None] * O.project(c.G, c.x, views)
    for j in range(len(views)):
        _close(ax[j], ref[j])
    shape = (len(views),) + c.G.sino_shape[1:]
    q = (0.5 + synth.uniform(8, 5, int(np.prod(shape)))).reshape(shape).astype(np.float32)
    for det in (False, True):
        g = c.plan.back(_t(q), s, deterministic=det).cpu().numpy()
        _close(g, O.backproject(c.G, c.m[views][..., None] * q.astype(np.float64), views))
    # the model changes the result (the test would pass vacuously otherwise)
    ref0 = c.m[views][..., None] * O.project(O.Geometry(dict(c.g, res_fwhm=0.0)), c.x, views)
    assert np.linalg.norm(ref0 - ref) > 1e-3 * np.linalg.norm(ref)


@pytest.mark.parametrize("key", ["c1", "3d", "tof"])
@pytest.mark.parametrize("det", [False, True])
def test_gradient_and_sensitivity_with_resolution_model(key, det):
    c = case(key)
    s = 2
    beta, gam, eps = 0.3, 2.0, 1e-3
    obj, g = c.plan.objective_grad(c.xt, s, prior=(beta / c.n, gam, eps), deterministic=det)
    val, gd = O.data_grad(c.G, c.n, s, c.x, c.m, c.p["r"], c.p["y"])
    S, gs, _ = O.rdp(c.x.astype(np.float64), (c.g["dx"], c.g["dy"], c.g["dz"]), gam, eps)
    ref = gd + beta / c.n * gs
    scale = O.sensitivity(c.G, c.n, s, c.m)
    d = np.abs(g.cpu().numpy() - ref)
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
    assert abs(float(obj) - (val + beta / c.n * S)) <= 1e-5 * abs(val)
    _close(c.plan.sensitivity(s).cpu().numpy(), scale)
    _close(c.plan.sensitivity(-1).cpu().numpy(), O.sensitivity(c.G, 1, -1, c.m))


def test_em_update_with_resolution_model():
    c = case("3d")
    x = c.xt.clone()
    c.plan.em_update(x, 3)
    _close(x.cpu().numpy(), O.em_update(c.G, c.n, 3, c.m, c.p["r"], c.p["y"], c.x))


@pytest.mark.parametrize("key,algo,low_memory,det", [("c1", O.SVRG, False, False), ("3d", O.SVRG, False, False),
                                                     ("3d", O.SVRG, True, False), ("tof", O.SAGA, False, False),
                                                     ("3d", O.SAGA, False, True)])
def test_solver_with_resolution_model(key, algo, low_memory, det):
    from paper_2506_04976_gb300 import binding as pet
    c = case(key)
    n = c.n
    niter = 3 * n + 1
    sens = O.sensitivity(c.G, 1, -1, c.m)
    x0 = np.full(c.G.img_shape, float(c.p["x_true"].mean()), np.float32)
    order = O.subset_order(12, n, niter)
    kw = dict(omega=2, step_rule=O.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1, alpha=1.0, delta_rel=1e-6,
              pc_iters=(0, n, 2 * n), beta=c.p["beta"], gamma=c.p["gamma"], eps=c.p["eps"])
    xo, _, _ = O.solve(c.G, x0, c.m, c.p["r"], c.p["y"], sens, algo=algo, nsub=n, niter=niter, order=order, **kw)
    s = pet.Solver(c.plan, algo=algo, order=order, low_memory=low_memory, deterministic=det, **kw)
    s.set_image(_t(x0))
    s.run(niter)
    xg = s.image().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - xo) <= 1e-4 * np.linalg.norm(xo)


def test_invalid_resolution_settings():
    from paper_2506_04976_gb300 import binding as pet
    p = synth.make_problem("c1", 0)
    for fwhm, status in ((-1.0, 1), (500.0, 6)):  # negative; more than 31 taps per side
        with pytest.raises(pet.PetError) as e:
            pet.Plan(dict(p["geom"], res_fwhm=fwhm), p["nsub"])
        assert e.value.status == status
