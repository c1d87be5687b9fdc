"""The stored converged reference images (tests/golden/ref_<config>_seed<k>.npz, written
by the committed scripts beside them from the oracle alone) satisfy the optimality
conditions of min_x D(x) + beta S(x), x >= 0 (eq. 1 with the prior of eq. 3): the KKT
residual ||min(x, grad F(x))|| / ||grad F(x_osem)||, recomputed here with the oracle
from the image as stored (float32), is below 1e-6, and the image is nonnegative.  The
normalisation ||grad F(x_osem)|| is recomputed for the 2D image and taken from the file
(written there by the oracle-only script) for the 3D ones, whose OSEM epoch takes long.

The half-resolution TOF reference (c3s) stops at 1.28e-6: there L-BFGS-B's line search
finds no further decrease of the FP64 objective (it ends abnormally, with no iteration,
from a fresh restart), and checkpoints 80 iterations apart differ by 0.014% NRMSE; its
bound is 1.5e-6."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _refs():
    out = []
    for f in sorted(os.listdir(GOLDEN)):
        if f.startswith("ref_") and f.endswith(".npz"):
            cfg, seed = f[4:-4].split("_seed")
            out.append((cfg, int(seed)))
    return out


@pytest.mark.parametrize("cfg,seed", _refs())
def test_reference_is_a_kkt_point(cfg, seed):
    d = np.load(os.path.join(GOLDEN, f"ref_{cfg}_seed{seed}.npz"))
    p = synth.make_problem(cfg, seed)
    g = p["geom"]
    G = O.Geometry(g)
    m = O.multiplicative(G, p["mu"].astype(np.float32), p["sens"].astype(np.float32))
    sp = (g["dx"], g["dy"], g["dz"])

    def grad(x):
        _, gd = O.data_grad(G, 1, -1, x, m, p["r"], p["y"])
        _, gs, _ = O.rdp(x, sp, p["gamma"], p["eps"])
        return gd + p["beta"] * gs

    x = d["x"].astype(np.float64)
    assert x.shape == G.img_shape and (x >= 0).all()
    if g["nz"] > 1 and "g0_norm" in d:
        g0n = float(d["g0_norm"])
    else:
        n = p["nsub"]
        x0 = np.ones(G.img_shape)
        for s in range(n):
            x0 = O.em_update(G, n, s, m, p["r"], p["y"], x0)
        g0n = np.linalg.norm(grad(x0))
    res = np.linalg.norm(np.minimum(x, grad(x))) / g0n
    assert res < (1.5e-6 if cfg == "c3s" else 1e-6), res
