"""The subset objective as a torch.autograd.Function (eq. 5): its backward (the
backprojection kernel plus the RDP gradient kernel) against the FP64 oracle gradient and
against central finite differences (h = 1e-3 relative) of its own forward, in the fused,
recompute and store modes.

FD tolerance: the forward value is an FP64 sum of FP32 per-bin terms; between x + h e_j
and x - h e_j only the LORs through voxel j change, so the FD noise is ~1e-7 of those
LORs' terms over 2h, far below the 1e-2 |g_j| + 1e-3 max|g| bound used here."""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

_C = {}


def setup(key):
    if key not in _C:
        from paper_2506_04976_gb300 import binding as pet
        if key == "c1":
            p = synth.make_problem("c1", 2)
        elif key == "3d":
            p = synth.make_problem("c2", 2, nx=32, nz=13, nrad=56, nview=24, nsub=4)
        elif key == "tof":
            p = synth.make_problem("c3", 2, nx=32, nz=13, nrad=56, nview=24, nsub=4)
        else:  # the full-size TOF workload
            p = synth.make_problem("c3", 0)
        plan = pet.Plan(p["geom"], p["nsub"])
        mu32, sens32 = p["mu"].astype(np.float32), p["sens"].astype(np.float32)
        y = p["y"].view(np.int16) if p["y"].dtype == np.uint16 else p["y"].astype(np.int32)
        plan.set_data(torch.from_numpy(y).to(DEV), torch.from_numpy(p["r"]).to(DEV),
                      torch.from_numpy(mu32).to(DEV), torch.from_numpy(sens32).to(DEV))
        x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
        _C[key] = (p, plan, mu32, sens32, x)
    return _C[key]


def _obj(plan, x, s, beta, mode, p):
    from paper_2506_04976_gb300.autograd import subset_objective
    return subset_objective(x, plan, s, beta=beta, gamma=p["gamma"], eps=p["eps"], mode=mode)


@pytest.mark.parametrize("key", ["c1", "3d", "tof"])
@pytest.mark.parametrize("mode", ["fused", "recompute", "store"])
def test_backward_matches_oracle_gradient(key, mode):
    p, plan, mu32, sens32, x = setup(key)
    beta, s = 0.5, 1
    xt = torch.from_numpy(x).to(DEV).requires_grad_(True)
    f = _obj(plan, xt, s, beta, mode, p)
    if mode == "recompute":  # nothing sinogram-sized is kept for the backward
        assert all(t.numel() <= plan.N for t in f.grad_fn.saved_tensors)
    f.backward()
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, mu32, sens32)
    val, gd = O.data_grad(G, p["nsub"], s, x, m, p["r"], p["y"])
    S, gs, _ = O.rdp(x.astype(np.float64), (p["geom"]["dx"], p["geom"]["dy"], p["geom"]["dz"]), p["gamma"], p["eps"])
    ref = gd + beta / p["nsub"] * gs
    scale = O.sensitivity(G, p["nsub"], s, m)
    d = np.abs(xt.grad.cpu().numpy() - ref)
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
    assert abs(float(f.detach()) - (val + beta / p["nsub"] * S)) <= 1e-5 * abs(val)


def test_modes_agree_and_scale_with_grad_output():
    p, plan, _, _, x = setup("tof")
    grads = []
    for mode in ("fused", "recompute", "store"):
        xt = torch.from_numpy(x).to(DEV).requires_grad_(True)
        (3.0 * _obj(plan, xt, 2, 0.5, mode, p)).backward()
        grads.append(xt.grad.cpu().numpy())
    for gr in grads[1:]:
        assert np.linalg.norm(gr - grads[0]) <= 1e-5 * np.linalg.norm(grads[0])
    xt = torch.from_numpy(x).to(DEV).requires_grad_(True)
    _obj(plan, xt, 2, 0.5, "fused", p).backward()
    g1 = 3.0 * xt.grad.cpu().numpy()  # separate run: atomics sum in a different order
    assert np.linalg.norm(grads[0] - g1) <= 1e-5 * np.linalg.norm(g1)


@pytest.mark.parametrize("key", ["tof", "c3full"])
def test_central_differences_64_voxels(key):
    p, plan, _, _, x = setup(key)
    beta, s = 0.5, 3
    mode = "recompute"
    xt = torch.from_numpy(x).to(DEV).requires_grad_(True)
    _obj(plan, xt, s, beta, mode, p).backward()
    g = xt.grad.cpu().numpy().ravel()
    rng = np.random.default_rng(5)
    idx = rng.choice(x.size, 64, replace=False)
    xf = x.ravel()
    for j in idx:
        h = 1e-3 * max(float(xf[j]), 1e-3)
        xp, xm = xf.copy(), xf.copy()
        xp[j] += h
        xm[j] -= h
        with torch.no_grad():
            fp = float(_obj(plan, torch.from_numpy(xp.reshape(x.shape)).to(DEV), s, beta, mode, p))
            fm = float(_obj(plan, torch.from_numpy(xm.reshape(x.shape)).to(DEV), s, beta, mode, p))
        # the perturbation as actually stored in FP32
        hh = (np.float64(np.float32(xp[j])) - np.float64(np.float32(xm[j]))) / 2
        fd = (fp - fm) / (2 * hh)
        assert abs(fd - g[j]) <= 1e-2 * abs(g[j]) + 1e-3 * np.abs(g).max(), (j, fd, g[j])
