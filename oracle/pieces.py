"""The FP64 oracle split over host processes, for workloads whose subsets are too large
for one core (the brain-scale TOF sinogram: 4.15 M LORs x 13 TOF bins per subset).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the tests and the CPU-baseline
leg of the benchmark use it; the product library never does.  Nothing here adds
arithmetic of its own: a large set of LORs is cut into pieces (one view and a run of
planes each), every piece is evaluated by the oracle's functions on a geometry whose
plane list holds only that run, and the pieces' images and values are added.  The
multiplicative factors m = sens exp(-P mu) (Sec. 1.1) are formed per piece from the
oracle's own non-TOF projection of mu.

Processes are started with "spawn", so a parent that has already initialised CUDA can
use this safely.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_W = {}


def _init(geom, x, mu):
    _W.update(geom=geom, x=x, mu=mu)


def _piece_geoms(v, p0, p1):
    from . import Geometry
    g = _W["geom"]
    gk = dict(g, z1=np.asarray(g["z1"])[p0:p1], z2=np.asarray(g["z2"])[p0:p1])
    return Geometry(gk), Geometry(dict(gk, ntof=1))


def _mult(G1, v, sens):
    from . import project
    m = np.asarray(sens, np.float64)
    if _W["mu"] is not None:
        m = m * np.exp(-project(G1, _W["mu"], [v])[0, :, :, 0])
    return m


def _group(tasks):
    """Runs a list of pieces in this worker and returns the summed results and the
    worker's compute time (s)."""
    import time
    from . import backproject, data_grad_views, project
    t0 = time.perf_counter()
    val, img, sino = 0.0, None, []
    for op, v, p0, p1, sens, a, b in tasks:
        G, G1 = _piece_geoms(v, p0, p1)
        m = _mult(G1, v, sens)
        if op == "fwd":  # m P x of the piece, [P][R][T]
            sino.append((p0, m[..., None] * project(G, _W["x"], [v])[0]))
        elif op == "back":  # P^T (m q) of the piece
            gk = backproject(G, (m[..., None] * np.asarray(a, np.float64))[None], [v])
            img = gk if img is None else img + gk
        else:  # data term and gradient of the piece, a = r, b = y
            vk, gk = data_grad_views(G, [v], _W["x"], m[None], np.asarray(a)[None], np.asarray(b)[None])
            val += vk
            img = gk if img is None else img + gk
    return val, img, sino, time.perf_counter() - t0


def _pool_run(geom, x, mu, tasks, workers):
    workers = max(1, min(workers or os.cpu_count() or 1, len(tasks)))
    groups = [tasks[i::workers] for i in range(workers)]
    ctx = mp.get_context("spawn")
    geom = {k: (np.asarray(v) if k in ("z1", "z2") else v) for k, v in geom.items()}
    x = None if x is None else np.ascontiguousarray(x)
    mu = None if mu is None else np.ascontiguousarray(mu)
    with ctx.Pool(workers, initializer=_init, initargs=(geom, x, mu)) as pool:
        return pool.map(_group, groups)


def _chunks(nplane, chunk):
    return [(p0, min(nplane, p0 + chunk)) for p0 in range(0, nplane, chunk)]


def forward_view(geom, v, x, mu, sens_v, workers=None, chunk=64):
    """A x for every LOR of view v (all planes): [P][R][T], with A = m P (Sec. 1.1)."""
    P = len(geom["z1"])
    tasks = [("fwd", v, p0, p1, sens_v[p0:p1], None, None) for p0, p1 in _chunks(P, chunk)]
    out = None
    for _, _, sino, _ in _pool_run(geom, x, mu, tasks, workers):
        for p0, s in sino:
            if out is None:
                out = np.zeros((P,) + s.shape[1:])
            out[p0:p0 + s.shape[0]] = s
    return out


def back_views(geom, views, q_c, mu, sens_c, workers=None, chunk=64):
    """A^T q for a sinogram q_c [j][P][R][T] over the listed views (A = m P); sens_c holds
    their sensitivities [j][P][R]."""
    P = len(geom["z1"])
    tasks = [("back", int(v), p0, p1, sens_c[j][p0:p1], q_c[j][p0:p1], None)
             for j, v in enumerate(views) for p0, p1 in _chunks(P, chunk)]
    return sum(r[1] for r in _pool_run(geom, None, mu, tasks, workers) if r[1] is not None)


def back_view(geom, v, q_v, mu, sens_v, workers=None, chunk=64):
    """A^T q for a sinogram q_v [P][R][T] of view v alone (A = m P)."""
    return back_views(geom, [v], [q_v], mu, [sens_v], workers, chunk)


def data_grad_subset(geom, views, x, mu, sens_c, r_c, y_c, workers=None, chunk=96, timing=None):
    """(D_s(x), grad D_s(x)) of eq. 5 over the listed views, data in compact layout:
    sens_c (nv, P, R), r_c and y_c (nv, P, R, T).  timing (a dict, optional) receives
    the slowest worker's compute time ("seconds", process start-up excluded) and the
    number of worker processes ("workers")."""
    P = len(geom["z1"])
    tasks = [("grad", int(v), p0, p1, sens_c[j][p0:p1], r_c[j][p0:p1], y_c[j][p0:p1])
             for j, v in enumerate(views) for p0, p1 in _chunks(P, chunk)]
    res = _pool_run(geom, x, mu, tasks, workers)
    if timing is not None:
        timing["seconds"] = max(r[3] for r in res)
        timing["workers"] = len(res)
    return sum(r[0] for r in res), sum(r[1] for r in res if r[1] is not None)
