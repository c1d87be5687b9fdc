"""Ragged sizes: an odd image (37 x 37 x 19 voxels, 25 planes with oblique ones), an odd sinogram (53 radial bins x 26
views, n = 4 subsets of 7, 7, 6 and 6 views) so that every tiled kernel (32-wide transposes
and update tiles, 32 x 8 x 4 RDP tiles, warp-wide LOR groups) ends in a partial tile.
Operators, the RDP and a solver trajectory against the FP64 oracle, with the tolerances
of the other parity tests."""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

_C = {}


def case():
    if "c" not in _C:
        from paper_2506_04976_gb300 import binding as pet
        p = synth.make_problem("c2", 7, nx=37, nz=19, nrad=53, nview=26, nsub=4)
        g = p["geom"]
        plan = pet.Plan(g, p["nsub"])
        mu32, sens32 = p["mu"].astype(np.float32), p["sens"].astype(np.float32)
        plan.set_data(torch.from_numpy(p["y"].astype(np.int32)).to(DEV), torch.from_numpy(p["r"]).to(DEV),
                      torch.from_numpy(mu32).to(DEV), torch.from_numpy(sens32).to(DEV))
        G = O.Geometry(g)
        m = O.multiplicative(G, mu32, sens32)
        x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
        _C["c"] = (p, plan, G, m, x)
    return _C["c"]


def _close(gpu, ref, rel_l2=1e-5, rel_el=1e-4, abs_frac=1e-5):
    gpu, ref = np.asarray(gpu, np.float64), np.asarray(ref, np.float64)
    d = np.abs(gpu - ref)
    assert np.linalg.norm(d) <= rel_l2 * np.linalg.norm(ref)
    assert (d <= rel_el * np.abs(ref) + abs_frac * np.abs(ref).max()).all(), d.max()


@pytest.mark.parametrize("s", [0, 3])
def test_ragged_operators(s):
    p, plan, G, m, x = case()
    n = p["nsub"]
    views = O.subset_views(p["geom"]["nview"], n, s)
    xt = torch.from_numpy(x).to(DEV)
    ax = plan.forward(xt, s).cpu().numpy()
    ref = m[views][..., None] * O.project(G, x, views)
    for j in range(len(views)):
        _close(ax[j], ref[j])
    obj, g = plan.objective_grad(xt, s)
    val, gd = O.data_grad(G, n, s, x, m, p["r"], p["y"])
    scale = O.sensitivity(G, n, s, m)
    assert np.linalg.norm(g.cpu().numpy() - gd) <= 1e-5 * np.linalg.norm(scale)
    assert abs(float(obj) - val) <= 1e-5 * abs(val)
    _close(plan.sensitivity(s).cpu().numpy(), scale)


def test_ragged_rdp():
    from paper_2506_04976_gb300 import binding as pet
    p, plan, G, m, x = case()
    sp = (p["geom"]["dx"], p["geom"]["dy"], p["geom"]["dz"])
    val, gs, hs = pet.rdp(torch.from_numpy(x).to(DEV), sp, p["gamma"], p["eps"])
    S, gso, hso = O.rdp(x.astype(np.float64), sp, p["gamma"], p["eps"])
    gs = gs.cpu().numpy()
    assert np.abs(gs - gso).max() <= 1e-5 * np.abs(gso).max()
    _close(hs.cpu().numpy(), hso)
    assert abs(float(val) - S) <= 1e-5 * abs(S)


@pytest.mark.parametrize("algo", [O.SVRG, O.SAGA])
def test_ragged_solver(algo):
    from paper_2506_04976_gb300 import binding as pet
    p, plan, G, m, x = case()
    n = p["nsub"]
    niter = 3 * n + 1
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.full(G.img_shape, float(p["x_true"].mean()), np.float32)
    order = O.subset_order(3, n, niter)
    kw = dict(omega=2, step_rule=O.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1, alpha=1.0, delta_rel=1e-6,
              pc_iters=(0, n, 2 * n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
    xo, _, _ = O.solve(G, x0, m, p["r"], p["y"], sens, algo=algo, nsub=n, niter=niter, order=order, **kw)
    s = pet.Solver(plan, algo=algo, order=order, **kw)
    s.set_image(torch.from_numpy(x0).to(DEV))
    s.run(niter)
    xg = s.image().cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - xo) <= 1e-4 * np.linalg.norm(xo)
