"""Writes a converged reference image with L-BFGS-B, the way Sec. 3.1 obtains its
references (preconditioned L-BFGS-B on the full objective), for the time-to-1%-NRMSE
measurement on the 3D workloads, where the stochastic run of make_reference.py converges
too slowly in FP64 on the host.

Calls only the FP64 oracle (oracle/) and the seeded input generator.  The objective is
    F(x) = sum_j d(A_j x + r_j, y_j) + beta S(x),   x >= 0,
with the data term and its gradient summed over W view subsets evaluated in W worker
processes (the data term partitions over subsets) and the RDP in the main process.  The
variables are scaled, x = d z with d = sqrt(harmonic preconditioner at the start image)
(eq. 8), and z >= 0 is kept by L-BFGS-B's bounds.  The start image is one OSEM epoch.
Every `--check` iterations the KKT residual ||min(x, grad F(x))|| / ||grad F(x0)|| is
recorded and the image saved (float32) to tests/golden/ref_<config>_seed<k>.npz.

    python tests/golden/make_reference_lbfgs.py c2 0 [--workers 7] [--maxiter 600]
        [--init file.npz] [--out file.npz]

--init restarts from an image this script wrote, with the variable scaling recomputed
there (the KKT normalisation always refers to the OSEM start image and is stored with
the result as g0_norm); --out writes elsewhere
than tests/golden, e.g. while the run is still far from converged.
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2506_04976_gb300 import synth  # noqa: E402

_W = {}


def _init(config, seed, nworkers):
    sys.path.insert(0, ROOT)
    p = synth.make_problem(config, seed)
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, p["mu"].astype(np.float32), p["sens"].astype(np.float32))
    _W.update(p=p, G=G, m=m, W=nworkers)


def _data_part(args):
    w, x = args
    p, G, m, W = _W["p"], _W["G"], _W["m"], _W["W"]
    val, g = O.data_grad(G, W, w, x, m, p["r"], p["y"])
    return val, g


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config")
    ap.add_argument("seed", type=int)
    ap.add_argument("--workers", type=int, default=7)
    ap.add_argument("--maxiter", type=int, default=600)
    ap.add_argument("--check", type=int, default=20)
    ap.add_argument("--out", default=None)
    ap.add_argument("--init", default=None)
    a = ap.parse_args()
    from scipy.optimize import minimize

    p = synth.make_problem(a.config, a.seed)
    g = p["geom"]
    G = O.Geometry(g)
    m = O.multiplicative(G, p["mu"].astype(np.float32), p["sens"].astype(np.float32))
    sp = (g["dx"], g["dy"], g["dz"])
    n, beta = p["nsub"], p["beta"]
    out = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"ref_{a.config}_seed{a.seed}.npz")

    x = np.ones(G.img_shape)
    for s in range(n):  # one OSEM epoch (Sec. 3.1)
        x = O.em_update(G, n, s, m, p["r"], p["y"], x)
    sens = O.sensitivity(G, 1, -1, m)
    xs = np.load(a.init)["x"].astype(np.float64) if a.init else x  # scaling from the start image
    _, _, H = O.rdp(xs, sp, p["gamma"], p["eps"])
    D = O.precond(xs, sens, beta * H, 1.0, 1e-6 * xs.max(), kind=1)
    d = np.sqrt(np.maximum(D, 1e-12 * D.max()))

    ctx = mp.get_context("spawn")
    pool = ctx.Pool(a.workers, initializer=_init, initargs=(a.config, a.seed, a.workers))
    shape = G.img_shape
    evals = [0]

    def fg(x):
        parts = pool.map(_data_part, [(w, x) for w in range(a.workers)])
        val = sum(v for v, _ in parts)
        grad = sum(gg for _, gg in parts)
        S, gs, _ = O.rdp(x, sp, p["gamma"], p["eps"])
        evals[0] += 1
        return val + beta * S, grad + beta * gs

    F0, g0 = fg(x)
    g0n = np.linalg.norm(g0)
    it0 = 0
    if a.init:
        prev = np.load(a.init)
        assert str(prev["config"]) == a.config and int(prev["seed"]) == a.seed
        x, it0 = prev["x"].astype(np.float64), int(prev["epochs"])
    t0 = time.time()
    state = {"it": it0, "kkt": np.inf}

    def fun(z):
        xx = (d * z.reshape(shape))
        F, gr = fg(xx)
        state["last"] = (xx, gr)
        return F, (d * gr).ravel()

    def callback(zk):
        state["it"] += 1
        if state["it"] % a.check == 0:
            xx = d * zk.reshape(shape)
            _, gr = fg(xx)
            res = np.linalg.norm(np.minimum(xx, gr)) / g0n
            state["kkt"] = res
            print(f"iter {state['it']} evals {evals[0]} kkt {res:.3e} ({time.time() - t0:.0f} s)", flush=True)
            np.savez_compressed(out, x=xx.astype(np.float32), kkt=res, epochs=state["it"], config=a.config,
                                seed=a.seed, method="lbfgsb", g0_norm=g0n)

    z0 = (x / d).ravel()
    minimize(fun, z0, jac=True, method="L-BFGS-B", bounds=[(0, None)] * z0.size, callback=callback,
             options=dict(maxiter=a.maxiter, maxfun=4 * a.maxiter, maxcor=20, ftol=1e-16, gtol=1e-12))
    pool.close()
    print("wrote", out, "kkt", state["kkt"])


if __name__ == "__main__":
    main()
