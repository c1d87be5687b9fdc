"""Plane groups of the windowed TOF kernel.  When the planes of every group lie a whole
number of slices apart (ring pitch = 2 slices here) the persistent kernel takes one floor
and one axial weight per sample for the whole group; at a fractional offset (ring pitch
1.5 slices) every plane evaluates its own axial position.  Both against the FP64 oracle
(eq. 5 with the KL data term of Sec. 1.2), with 2 and 4 planes per thread and with one
and two parts per LOR, at the tolerances of the other subset-gradient tests."""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth
from tests.geoms import geom3d, rand_img, rand_sino

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

_P = {}


def _problem(pitch_slices):
    if pitch_slices not in _P:
        from paper_2506_04976_gb300 import binding as pet
        # 7 TOF bins of 10 mm, sigma 8 mm: a sample meets at most 6 bins (windowed kernel)
        g = geom3d(n=24, nz=9, nrad=32, nview=12, d=2.0, dz=2.0, ntof=7, tof_sigma=8.0, tof_bin=10.0)
        g["z1"], g["z2"] = synth.planes_span1(5, pitch_slices * g["dz"])
        n = 3
        plan = pet.Plan(g, n)
        G = O.Geometry(g)
        shape = (g["nview"], len(g["z1"]), g["nrad"], g["ntof"])
        rng = np.random.default_rng(17)
        y = rng.poisson(3.0 * rand_sino(g, 3)).astype(np.int32).reshape(shape)
        r = (0.2 * rand_sino(g, 4)).astype(np.float32).reshape(shape)
        plan.set_data(torch.from_numpy(y).to(DEV), torch.from_numpy(r).to(DEV))
        m = O.multiplicative(G, np.zeros(G.img_shape, np.float32), np.ones(shape[:3], np.float32))
        x = rand_img(g, 5, 0.1, 1.0).astype(np.float32)
        _P[pitch_slices] = (g, n, plan, G, m, x, y, r)
    return _P[pitch_slices]


@pytest.mark.parametrize("pitch_slices", [2.0, 1.5])
@pytest.mark.parametrize("grad_shape", [(2, 1), (4, 1), (2, 2)])
def test_tof_plane_groups_against_oracle(pitch_slices, grad_shape):
    g, n, plan, G, m, x, y, r = _problem(pitch_slices)
    plan.set_grad_shape(*grad_shape)
    xt = torch.from_numpy(x).to(DEV)
    for s in range(n):
        obj, gg = plan.objective_grad(xt, s)
        val, gd = O.data_grad(G, n, s, x, m, r, y)
        scale = O.sensitivity(G, n, s, m)
        d = np.abs(gg.cpu().numpy() - gd)
        assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale), s
        assert np.all(d <= 1e-4 * scale + 1e-6 * scale.max()), s
        assert abs(float(obj) - val) <= 1e-5 * abs(val), s
    plan.check()
