"""Writes converged reference images for the time-to-1%-NRMSE measurement.

Calls only the FP64 oracle (oracle/) and the seeded input generator: preconditioned SVRG
(eq. 9, Algorithm 1, harmonic preconditioner of eq. 8, constant unit step) from one OSEM
epoch (Sec. 3.1), run in chunks until the KKT residual of
    min_x  sum_i f_i(x) + indicator(x >= 0)
measured as ||min(x, grad f(x))|| / ||grad f(x0)||, falls below the target.  The image is
stored as float32 with the residual reached, in tests/golden/ref_<config>_seed<k>.npz.

    python tests/golden/make_reference.py c1 0 [--kkt 1e-6] [--max-epochs 4000] [--tau 1.0]

A smaller constant step (--tau) keeps the iteration stable on the low-count 3D workloads,
where a unit step makes the KKT residual oscillate between chunks.  --out writes elsewhere
than tests/golden (for comparing step sizes); --resume continues from a file it wrote.
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2506_04976_gb300 import synth  # noqa: E402


def full_grad(G, p, m, x):
    _, gd = O.data_grad(G, 1, -1, x, m, p["r"], p["y"])
    sp = (p["geom"]["dx"], p["geom"]["dy"], p["geom"]["dz"])
    _, gs, _ = O.rdp(x, sp, p["gamma"], p["eps"])
    return gd + p["beta"] * gs


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config")
    ap.add_argument("seed", type=int)
    ap.add_argument("--kkt", type=float, default=1e-6)
    ap.add_argument("--max-epochs", type=int, default=4000)
    ap.add_argument("--chunk", type=int, default=20, help="epochs between KKT checks")
    ap.add_argument("--tau", type=float, default=1.0, help="constant SVRG step")
    ap.add_argument("--out", default=None)
    ap.add_argument("--resume", default=None, help="npz written by this script to continue from")
    a = ap.parse_args()
    p = synth.make_problem(a.config, a.seed)
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, p["mu"].astype(np.float32), p["sens"].astype(np.float32))
    n = p["nsub"]
    sens = O.sensitivity(G, 1, -1, m)
    x = np.ones(G.img_shape)
    for s in range(n):  # one OSEM epoch
        x = O.em_update(G, n, s, m, p["r"], p["y"], x)
    g0 = np.linalg.norm(full_grad(G, p, m, x))
    epochs, res = 0, np.inf
    if a.resume:
        prev = np.load(a.resume)
        assert str(prev["config"]) == a.config and int(prev["seed"]) == a.seed
        x, epochs = prev["x"].astype(np.float64), int(prev["epochs"])
    t0 = time.time()
    out = a.out or os.path.join(os.path.dirname(os.path.abspath(__file__)), f"ref_{a.config}_seed{a.seed}.npz")
    seed = 1000 + a.seed
    while epochs < a.max_epochs:
        niter = a.chunk * n
        order = O.subset_order(seed + epochs, n, niter)
        x, _, _ = O.solve(G, x, m, p["r"], p["y"], sens, algo=O.SVRG, nsub=n, niter=niter, order=order,
                          omega=2, step_rule=O.STEP_CONST, tau0=a.tau, precond_kind=1, alpha=1.0,
                          delta_rel=1e-6, pc_iters=(0,), beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
        epochs += a.chunk
        res = np.linalg.norm(np.minimum(x, full_grad(G, p, m, x))) / g0
        print(f"epochs {epochs} kkt {res:.3e} ({time.time() - t0:.0f} s)", flush=True)
        np.savez_compressed(out, x=x.astype(np.float32), kkt=res, epochs=epochs,
                            config=a.config, seed=a.seed, tau=a.tau)
        if res < a.kkt:
            break
    print("wrote", out, "kkt", res)


if __name__ == "__main__":
    main()
