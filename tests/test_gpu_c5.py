"""The large TOF workload at full size (215x215x71 image; 357 radial x 224 views x 1293
planes x 13 TOF bins = 1.34 G bins; uint16 counts; 25 uneven subsets): sampled TOF LORs
against the oracle, adjointness of one subset, and one whole subset gradient."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
_S = {}


def c5():
    if not _S:
        from paper_2506_04976_gb300 import binding as pet
        t0 = time.time()
        p = synth.make_problem_device("c5", 0, device=DEV)
        t1 = time.time()
        plan = pet.Plan(p["geom"], p["nsub"])
        mu = torch.from_numpy(p["mu"].astype(np.float32)).to(DEV)
        plan.set_data(p["y"], p["r"], mu, p["sens"])
        torch.cuda.synchronize()
        _S.update(p=p, plan=plan, mu=mu, gen_s=t1 - t0, setup_s=time.time() - t1)
    return _S


def test_c5_shapes_and_uneven_subsets():
    S = c5()
    p, plan = S["p"], S["plan"]
    assert plan.sino_shape == (224, 1293, 357, 13)
    sizes = [plan.subset_views(s) for s in range(25)]
    assert sizes.count(9) == 24 and sizes.count(8) == 1
    assert p["y"].dtype == torch.int16  # uint16 counts


def test_c5_sampled_tof_lors_against_oracle():
    S = c5()
    p, plan = S["p"], S["plan"]
    g = p["geom"]
    s = 7
    x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
    ax = plan.forward(torch.from_numpy(x).to(DEV), s)
    views = O.subset_views(g["nview"], p["nsub"], s)
    rng = np.random.default_rng(3)
    jv = rng.integers(0, len(views), 64)
    pp = rng.integers(0, len(g["z1"]), 64)
    rr = rng.integers(60, g["nrad"] - 60, 64)  # LORs through the object
    vpr = np.stack([views[jv], pp, rr], 1)
    got = ax[torch.from_numpy(jv).to(DEV), torch.from_numpy(pp).to(DEV), torch.from_numpy(rr).to(DEV)].cpu().numpy()
    G = O.Geometry(g)
    g1 = dict(g, ntof=1)
    sens = p["sens"][torch.from_numpy(vpr[:, 0]).to(DEV), torch.from_numpy(vpr[:, 1]).to(DEV),
                     torch.from_numpy(vpr[:, 2]).to(DEV)].double().cpu().numpy()
    # m = sens exp(-P mu) for the sampled LORs (the oracle's attenuation model, Sec. 1.1)
    m = sens * np.exp(-O.project_lors(O.Geometry(g1), p["mu"].astype(np.float32), vpr)[:, 0])
    ref = m[:, None] * O.project_lors(G, x, vpr)
    assert np.all(np.abs(got - ref) <= 1e-4 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    assert np.linalg.norm(got - ref) <= 1e-5 * np.linalg.norm(ref)


def test_c5_adjointness_one_subset():
    S = c5()
    plan = S["plan"]
    gen = torch.Generator(device=DEV).manual_seed(3)
    x = torch.rand(plan.img_shape, device=DEV, generator=gen)
    s = 24  # the 8-view subset
    q = torch.rand(plan.subset_shape(s), device=DEV, generator=gen)
    ax = plan.forward(x, s)
    lhs = torch.dot(ax.double().ravel(), q.double().ravel()).item()
    for det in (False, True):
        atq = plan.back(q, s, deterministic=det)
        rhs = torch.dot(x.double().ravel(), atq.double().ravel()).item()
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_c5_subset_gradient_finite_and_feasible():
    S = c5()
    p, plan = S["p"], S["plan"]
    x = torch.from_numpy(np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)).to(DEV)
    obj, g = plan.objective_grad(x, 3, prior=(p["beta"] / p["nsub"], p["gamma"], p["eps"]))
    torch.cuda.synchronize()
    plan.check()
    assert torch.isfinite(g).all() and np.isfinite(float(obj))
    # the gradient of a subset term is bounded by its sensitivity (q <= m per bin)
    assert float(g.max()) <= float(plan.sensitivity(3).max()) * 1.0001 + p["beta"]
