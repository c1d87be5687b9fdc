"""GPU parity of each operator against the FP64 oracle on the same seeded inputs.

Tolerances (derived from FP32 arithmetic):
  * projections, backprojections, sensitivities, attenuation factors: relative L2 error
    per view / per image <= 1e-5 and elementwise |d| <= 1e-4 |ref| + 1e-5 max|ref|;
  * gradients of the KL term (a difference of two positive backprojections): errors
    measured against the scale of A^T 1, in L2 (1e-5 of ||A_s^T 1||) and per voxel
    (1e-4 (A_s^T 1)_j + 1e-6 max A_s^T 1, which also bounds entries near zero);
  * RDP: max-norm relative 1e-5 (gradient), elementwise 1e-5 (Hessian diagonal),
    1e-5 (value); KL objective 1e-5 relative;
  * sums of many FP32 atomics: adjointness within 1e-5 relative.
"""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _pet():
    from paper_2506_04976_gb300 import binding
    return binding


def _t(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dt)


def _y_tensor(y):
    return torch.from_numpy(y.astype(np.int32)).to(DEV)


class Case:
    def __init__(self, name, **over):
        self.p = synth.make_problem(name, 0, **over)
        self.g = self.p["geom"]
        self.n = self.p["nsub"]
        pet = _pet()
        self.plan = pet.Plan(self.g, self.n)
        self.mu32 = self.p["mu"].astype(np.float32)
        self.sens32 = self.p["sens"].astype(np.float32)
        self.y = _y_tensor(self.p["y"])
        self.r = _t(self.p["r"])
        self.plan.set_data(self.y, self.r, _t(self.mu32), _t(self.sens32))
        self.G = O.Geometry(self.g)
        self.m = O.multiplicative(self.G, self.mu32, self.sens32)
        self.x = np.maximum(self.p["x_true"], 0.05 * self.p["x_true"].max()).astype(np.float32)
        self.xt = _t(self.x)


_CASES = {}


def case(key):
    if key not in _CASES:
        specs = {
            "c1": ("c1", {}),
            "3d": ("c2", dict(nx=40, nz=23, nrad=70, nview=36, nsub=6)),
            # TOF bins over the 362 mm FOV diagonal with sigma 24.8 mm: 11 bins of 33 mm
            # (a sample meets at most 6 bins), 13 of 28 mm (7) and 5 of 73 mm (4) run the
            # windowed TOF kernel; 25 bins of 15 mm (11) the kernels with per-edge weights
            "tof": ("c3", dict(nx=40, nz=23, nrad=70, nview=36, nsub=6)),
            "tof13": ("c3", dict(nx=40, nz=23, nrad=70, nview=36, nsub=6, ntof=13)),
            "tof5": ("c3", dict(nx=40, nz=23, nrad=70, nview=36, nsub=6, ntof=5)),
            "tof25": ("c3", dict(nx=40, nz=23, nrad=70, nview=36, nsub=6, ntof=25)),
        }
        name, over = specs[key]
        _CASES[key] = Case(name, **over)
    return _CASES[key]


def _close(gpu, ref, rel_l2=1e-5, rel_el=1e-4, abs_frac=1e-5):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.abs(gpu - ref)
    l2 = np.linalg.norm(d) / max(np.linalg.norm(ref), 1e-300)
    el = (d > rel_el * np.abs(ref) + abs_frac * np.abs(ref).max()).sum()
    assert l2 <= rel_l2, f"relative L2 error {l2:.3e}"
    assert el == 0, f"{el} elements beyond tolerance (max abs err {d.max():.3e})"
    return l2


@pytest.mark.parametrize("key", ["c1", "3d", "tof"])
def test_multiplicative_factors(key):
    c = case(key)
    m_gpu = c.plan.mult().cpu().numpy()
    _close(m_gpu, c.m)


@pytest.mark.parametrize("key", ["c1", "3d", "tof", "tof13", "tof5", "tof25"])
@pytest.mark.parametrize("subset", [0, 3])
def test_forward_projection(key, subset):
    c = case(key)
    ax = c.plan.forward(c.xt, subset).cpu().numpy()
    views = O.subset_views(c.g["nview"], c.n, subset)
    ref = c.m[views][..., None] * O.project(c.G, c.x, views)
    for j in range(len(views)):  # per projection view
        _close(ax[j], ref[j])


@pytest.mark.parametrize("key", ["c1", "3d", "tof", "tof13", "tof25"])
@pytest.mark.parametrize("det", [False, True])
def test_back_projection(key, det):
    c = case(key)
    s = 2
    views = O.subset_views(c.g["nview"], c.n, s)
    shape = (len(views),) + c.G.sino_shape[1:]
    q = (0.5 + synth.uniform(3, 5, int(np.prod(shape)))).reshape(shape).astype(np.float32)
    g = c.plan.back(_t(q), s, deterministic=det).cpu().numpy()
    ref = O.backproject(c.G, c.m[views][..., None] * q.astype(np.float64), views)
    _close(g, ref)


@pytest.mark.parametrize("key", ["c1", "tof"])
def test_deterministic_backprojection_is_reproducible(key):
    c = case(key)
    shape = c.plan.subset_shape(1)
    q = _t((0.5 + synth.uniform(4, 5, int(np.prod(shape)))).reshape(shape))
    a = c.plan.back(q, 1, deterministic=True).cpu().numpy()
    b = c.plan.back(q, 1, deterministic=True).cpu().numpy()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("key", ["c1", "3d", "tof"])
def test_sensitivity_images(key):
    c = case(key)
    _close(c.plan.sensitivity(-1).cpu().numpy(), O.sensitivity(c.G, 1, -1, c.m))
    _close(c.plan.sensitivity(1).cpu().numpy(), O.sensitivity(c.G, c.n, 1, c.m))


@pytest.mark.parametrize("key", ["c1", "3d", "tof", "tof13", "tof5", "tof25"])
@pytest.mark.parametrize("det", [False, True])
def test_subset_objective_and_gradient(key, det):
    c = case(key)
    s = 1
    beta, gam, eps = 0.3, 2.0, 1e-3
    obj, g = c.plan.objective_grad(c.xt, s, prior=(beta / c.n, gam, eps), deterministic=det)
    g = g.cpu().numpy()
    val, gd = O.data_grad(c.G, c.n, s, c.x, c.m, c.p["r"], c.p["y"])
    S, gs, _ = O.rdp(c.x.astype(np.float64), (c.g["dx"], c.g["dy"], c.g["dz"]), gam, eps)
    ref = gd + beta / c.n * gs
    scale = O.sensitivity(c.G, c.n, s, c.m)
    d = np.abs(g - ref)
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
    assert d.max() <= 1e-4 * scale.max()
    assert np.all(d <= 1e-4 * scale + 1e-6 * scale.max())  # per voxel, small entries included
    f = val + beta / c.n * S
    assert abs(float(obj) - f) <= 1e-5 * abs(f)
    c.plan.check()


@pytest.mark.parametrize("key", ["c1", "tof", "tof25"])
def test_objective_only_matches(key):
    c = case(key)
    o1, _ = c.plan.objective_grad(c.xt, 0)
    o2, g2 = c.plan.objective_grad(c.xt, 0, obj_only=True)
    assert g2 is None
    assert abs(float(o1) - float(o2)) <= 1e-12 * abs(float(o1))


def test_gpu_adjointness_full_size_c2():
    """<A_s x, q> = <x, A_s^T q> at the full 3D non-TOF size (a property at any size)."""
    p = synth.make_problem("c2", 0)
    pet = _pet()
    plan = pet.Plan(p["geom"], p["nsub"])
    plan.set_data(_y_tensor(p["y"]), _t(p["r"]), _t(p["mu"]), _t(p["sens"]))
    gen = torch.Generator(device=DEV).manual_seed(7)
    x = torch.rand(plan.img_shape, device=DEV, generator=gen)
    for s in (0, 11, 20):
        q = torch.rand(plan.subset_shape(s), device=DEV, generator=gen)
        ax = plan.forward(x, s)
        for det in (False, True):
            atq = plan.back(q, s, deterministic=det)
            lhs = torch.dot(ax.double().ravel(), q.double().ravel()).item()
            rhs = torch.dot(x.double().ravel(), atq.double().ravel()).item()
            assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_full_size_c2_sampled_rows_and_subset_gradient():
    """Full 3D non-TOF workload: sampled projection rows and one whole subset gradient
    against the oracle."""
    p = synth.make_problem("c2", 0)
    pet = _pet()
    g = p["geom"]
    plan = pet.Plan(g, p["nsub"])
    mu32, sens32 = p["mu"].astype(np.float32), p["sens"].astype(np.float32)
    plan.set_data(_y_tensor(p["y"]), _t(p["r"]), _t(mu32), _t(sens32))
    G = O.Geometry(g)
    x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
    xt = _t(x)
    s = 5
    views = O.subset_views(g["nview"], p["nsub"], s)
    ax = plan.forward(xt, s).cpu().numpy()
    rng = np.random.default_rng(0)
    jv = rng.integers(0, len(views), 200)
    pp = rng.integers(0, len(g["z1"]), 200)
    rr = rng.integers(0, g["nrad"], 200)
    vpr = np.stack([views[jv], pp, rr], 1)
    m = O.multiplicative(G, mu32, sens32)
    ref = m[vpr[:, 0], vpr[:, 1], vpr[:, 2]][:, None] * O.project_lors(G, x, vpr)
    got = ax[jv, pp, rr]
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    _, gg = plan.objective_grad(xt, s)
    _, gd = O.data_grad(G, p["nsub"], s, x, m, p["r"], p["y"])
    scale = O.sensitivity(G, p["nsub"], s, m)
    d = np.abs(gg.cpu().numpy() - gd)
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
    assert np.all(d <= 1e-4 * scale + 1e-6 * scale.max())  # per voxel, small entries included


def test_full_size_c3_sampled_tof_lors_and_subset_gradient():
    """Full 3D TOF workload (11 TOF bins, 1e6 counts; data generated on the device) in
    the autotuned launch shape: sampled TOF LORs and one whole subset gradient and
    objective against the oracle, which receives the same data copied to the host."""
    p = synth.make_problem_device("c3", 0, device=DEV)
    pet = _pet()
    g = p["geom"]
    plan = pet.Plan(g, p["nsub"])
    mu32 = p["mu"].astype(np.float32)
    plan.set_data(p["y"], p["r"], _t(mu32), p["sens"])
    plan.autotune()
    sens32 = p["sens"].cpu().numpy()
    y = p["y"].cpu().numpy()
    p = dict(p, y=y.view(np.uint16) if y.dtype == np.int16 else y, r=p["r"].cpu().numpy())
    assert plan.sino_shape == (168, 109, 250, 11)
    G = O.Geometry(g)
    m = O.multiplicative(G, mu32, sens32)
    x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
    xt = _t(x)
    s = 13
    views = O.subset_views(g["nview"], p["nsub"], s)
    ax = plan.forward(xt, s).cpu().numpy()
    rng = np.random.default_rng(1)
    jv = rng.integers(0, len(views), 200)
    pp = rng.integers(0, len(g["z1"]), 200)
    rr = rng.integers(0, g["nrad"], 200)
    vpr = np.stack([views[jv], pp, rr], 1)
    ref = m[vpr[:, 0], vpr[:, 1], vpr[:, 2]][:, None] * O.project_lors(G, x, vpr)
    got = ax[jv, pp, rr]
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    obj, gg = plan.objective_grad(xt, s)
    val, gd = O.data_grad(G, p["nsub"], s, x, m, p["r"], p["y"])
    scale = O.sensitivity(G, p["nsub"], s, m)
    d = np.abs(gg.cpu().numpy() - gd)
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
    assert np.all(d <= 1e-4 * scale + 1e-6 * scale.max())  # per voxel, small entries included
    assert abs(float(obj) - val) <= 1e-5 * abs(val)


@pytest.mark.parametrize("shape,kappa", [((1, 37, 45), False), ((11, 19, 70), False), ((11, 19, 70), True)])
def test_rdp_parity(shape, kappa):
    rng = np.random.default_rng(1)
    x = rng.uniform(0.0, 3.0, shape).astype(np.float32)
    x[x < 0.3] = 0.0  # exact zeros: d = 0 and s = 0 pairs
    k = rng.uniform(0.5, 1.5, shape).astype(np.float32) if kappa else None
    sp, gam, eps, beta = (2.0, 2.0, 2.8), 2.0, 1e-3, 0.7
    pet = _pet()
    v, gr, h = pet.rdp(_t(x), sp, gam, eps, beta, _t(k) if kappa else None)
    S, gs, hs = O.rdp(x.astype(np.float64), sp, gam, eps, k.astype(np.float64) if kappa else None)
    assert np.abs(gr.cpu().numpy() - beta * gs).max() <= 1e-5 * np.abs(beta * gs).max()
    hg = h.cpu().numpy()
    assert np.all(np.abs(hg - beta * hs) <= 1e-5 * np.abs(beta * hs) + 1e-7 * np.abs(beta * hs).max())
    assert abs(float(v) - beta * S) <= 1e-5 * abs(beta * S)


def test_rdp_constant_image_gpu():
    pet = _pet()
    x = torch.full((5, 17, 33), 1.7, device=DEV)
    v, g, h = pet.rdp(x, (2.0, 2.0, 2.8), 2.0, 1e-3, 1.0)
    assert float(v) == 0.0 and float(g.abs().max()) == 0.0


@pytest.mark.parametrize("key", ["c1", "3d"])
@pytest.mark.parametrize("kind", [0, 1])
def test_preconditioner(key, kind):
    c = case(key)
    beta, gam, eps = 0.4, 2.0, 1e-3
    pet = _pet()
    _, _, h = pet.rdp(c.xt, (c.g["dx"], c.g["dy"], c.g["dz"]), gam, eps, beta)
    D = c.plan.precond(c.xt, h if kind else None, 1.0, 1e-6).cpu().numpy()
    x64 = c.x.astype(np.float64)
    _, _, hs = O.rdp(x64, (c.g["dx"], c.g["dy"], c.g["dz"]), gam, eps)
    ref = O.precond(x64, O.sensitivity(c.G, 1, -1, c.m), beta * hs, 1.0, 1e-6 * x64.max(), kind=kind)
    assert np.all(np.abs(D - ref) <= 2e-5 * np.abs(ref) + 1e-7 * np.abs(ref).max())


@pytest.mark.parametrize("key", ["c1", "tof", "tof25"])
def test_em_update(key):
    c = case(key)
    x = c.xt.clone()
    c.plan.em_update(x, 2)
    ref = O.em_update(c.G, c.n, 2, c.m, c.p["r"], c.p["y"], c.x)
    _close(x.cpu().numpy(), ref)


def test_nrmse_gpu_vs_oracle():
    c = case("c1")
    pet = _pet()
    ref = c.x * 1.01 + 0.001
    val = pet.nrmse(c.xt, _t(ref), _t(c.p["mask"], torch.uint8), _t(c.p["bg"], torch.uint8))
    o = O.nrmse(c.x, ref.astype(np.float32), c.p["mask"], c.p["bg"])
    assert abs(float(val) - o) <= 1e-9 * o


def test_infeasible_data_reported():
    """ybar = 0 where y > 0 (zero image, zero background) gives PET_ERR_INFEASIBLE."""
    g = case("c1").g
    pet = _pet()
    plan = pet.Plan(g, 6)
    shape = plan.sino_shape
    y = torch.ones(shape, device=DEV, dtype=torch.int32)
    r = torch.zeros(shape, device=DEV)
    plan.set_data(y, r)
    x = torch.zeros(plan.img_shape, device=DEV)
    plan.objective_grad(x, 0)
    with pytest.raises(pet.PetError) as e:
        plan.check()
    assert e.value.status == 3
    plan.check()  # cleared


def test_argument_errors():
    pet = _pet()
    c = case("c1")
    with pytest.raises(pet.PetError) as e:
        c.plan.forward(c.xt, 99)
    assert e.value.status == 1
    g = dict(c.g)
    g["rdet"] = 10.0  # radial bins beyond the detector radius
    with pytest.raises(pet.PetError) as e:
        pet.Plan(g, 6)
    assert e.value.status == 2


def test_y_zero_and_zero_image():
    """y = 0 everywhere: the KL term reduces to sum(ybar) and its gradient to A^T 1."""
    c = case("3d")
    pet = _pet()
    plan = pet.Plan(c.g, c.n)
    y = torch.zeros(plan.sino_shape, device=DEV, dtype=torch.int32)
    plan.set_data(y, c.r, _t(c.mu32), _t(c.sens32))
    obj, g = plan.objective_grad(c.xt, 0)
    sens = O.sensitivity(c.G, c.n, 0, c.m)
    _close(g.cpu().numpy(), sens)
    views = O.subset_views(c.g["nview"], c.n, 0)
    ref = (c.m[views][..., None] * O.project(c.G, c.x, views)).sum() + c.p["r"][views].astype(np.float64).sum()
    assert abs(float(obj) - ref) <= 1e-5 * ref


@pytest.mark.parametrize("key", ["3d", "tof"])
def test_set_counts_rebinds_counts_and_background(key):
    """A second frame bound with set_counts gives the oracle's objective and gradient of
    that frame's counts and background with the first frame's factors m (Sec. 1.1)."""
    c = case(key)
    rng = np.random.default_rng(7)
    y2 = rng.poisson(1.5 * c.p["y"].astype(np.float64) + 0.2).astype(np.int32)
    r2 = (0.7 * c.p["r"].astype(np.float64) + 0.01).astype(np.float32)
    y2d, r2d = _y_tensor(y2), _t(r2)
    try:
        c.plan.set_counts(y2d, r2d)
        s = 2
        obj, g = c.plan.objective_grad(c.xt, s)
        g = g.cpu().numpy()
        val, gd = O.data_grad(c.G, c.n, s, c.x, c.m, r2, y2)
        scale = O.sensitivity(c.G, c.n, s, c.m)
        d = np.abs(g - gd)
        assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
        assert np.all(d <= 1e-4 * scale + 1e-6 * scale.max())
        assert abs(float(obj) - val) <= 1e-5 * abs(val)
        assert np.allclose(c.plan.sensitivity(s).cpu().numpy(), scale, rtol=1e-4, atol=1e-5 * scale.max())
    finally:
        c.plan.set_counts(c.y, c.r)


def test_set_counts_needs_bound_data():
    pet = _pet()
    plan = pet.Plan(case("c1").g, 6)
    y = torch.zeros(plan.sino_shape, device=DEV, dtype=torch.int32)
    with pytest.raises(pet.PetError) as e:
        plan.set_counts(y, torch.zeros(plan.sino_shape, device=DEV))
    assert e.value.status == 7


@pytest.mark.parametrize("key", ["c1", "3d", "tof", "tof13", "tof5", "tof25"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 2), (1, 4), (1, 8), (1, 16), (2, 1), (2, 2), (2, 4), (2, 8), (2, 16),
                                   (4, 1), (4, 2), (4, 4), (4, 8), (4, 16)])
def test_grad_launch_shapes(key, shape):
    """Every launch shape of the fused gradient (planes per thread x parts per LOR)
    gives the oracle's subset objective and gradient."""
    c = case(key)
    k, parts = shape
    windowed = key in ("tof", "tof13", "tof5")
    if c.plan.T > 1 and (k > (4 if windowed else 1) or parts > (8 if windowed else 4)):
        pytest.skip("not a launch shape of this TOF kernel")
    c.plan.set_grad_shape(k, parts)
    try:
        s = 3
        obj, g = c.plan.objective_grad(c.xt, s)
        val, gd = O.data_grad(c.G, c.n, s, c.x, c.m, c.p["r"], c.p["y"])
        scale = O.sensitivity(c.G, c.n, s, c.m)
        d = np.abs(g.cpu().numpy() - gd)
        assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
        assert d.max() <= 1e-4 * scale.max()
        assert abs(float(obj) - val) <= 1e-5 * abs(val)
        # EM mode shares the kernel
        x = c.xt.clone()
        c.plan.em_update(x, 2)
        _close(x.cpu().numpy(), O.em_update(c.G, c.n, 2, c.m, c.p["r"], c.p["y"], c.x))
    finally:
        c.plan.set_grad_shape(0, 0)


@pytest.mark.parametrize("slices", [2, 4, 8])
def test_rdp_tiles_in_the_subset_objective(slices):
    """Every RDP stencil tile (slices per block) gives the oracle's prior share of the
    subset objective and gradient (eq. 5)."""
    c = case("3d")
    c.plan.set_rdp_tile(slices)
    try:
        s, beta, gam, eps = 2, 0.3, 2.0, 1e-3
        obj, g = c.plan.objective_grad(c.xt, s, prior=(beta / c.n, gam, eps))
        val, gd = O.data_grad(c.G, c.n, s, c.x, c.m, c.p["r"], c.p["y"])
        S, gs, _ = O.rdp(c.x.astype(np.float64), (c.g["dx"], c.g["dy"], c.g["dz"]), gam, eps)
        scale = O.sensitivity(c.G, c.n, s, c.m)
        d = np.abs(g.cpu().numpy() - (gd + beta / c.n * gs))
        assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
        f = val + beta / c.n * S
        assert abs(float(obj) - f) <= 1e-5 * abs(f)
    finally:
        c.plan.set_rdp_tile(0)


def test_autotune_keeps_parity():
    c = case("3d")
    k, parts = c.plan.autotune()
    assert k in (1, 2, 4) and parts in (1, 2, 4, 8, 16)
    _, g = c.plan.objective_grad(c.xt, 1)
    _, gd = O.data_grad(c.G, c.n, 1, c.x, c.m, c.p["r"], c.p["y"])
    scale = O.sensitivity(c.G, c.n, 1, c.m)
    assert np.linalg.norm(g.cpu().numpy() - gd) <= 1e-5 * np.linalg.norm(scale)
    c.plan.set_grad_shape(0, 0)
