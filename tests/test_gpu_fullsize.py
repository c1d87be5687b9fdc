"""Full-size solver trajectories against the FP64 oracle.

c2 (128x128x47 image, 250 radial x 168 views x 109 planes, 21 subsets): two epochs of
ALG1 of Table 1 (SVRG, Algorithm 1, with the harmonic preconditioner of eq. 8 and the
piecewise steps 3 / 2 / ...) from one OSEM epoch (Sec. 3.1), with the same subset order
on both sides.  The OSEM start image comes from the oracle, cast to float32, so both
runs start from identical values.  Bounds: 1e-4 relative L2 over the phantom support
(the NRMSE mask) and, per voxel of that mask, 1e-4 |x_ref| + 1e-5 max x_ref.

c4 (32 instances of uneven image and sinogram sizes, betas, count levels and subset
counts, as generated by synth.batch_specs): SAGA advanced by the batched driver equals
every instance run alone (within 1e-5, or within twice the difference between two single
runs where the atomics' order alone moves a low-count instance further), and the
smallest instance equals the oracle's trajectory."""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _device_data(pet, p):
    plan = pet.Plan(p["geom"], p["nsub"])
    mu32, sens32 = p["mu"].astype(np.float32), p["sens"].astype(np.float32)
    y = p["y"].view(np.int16) if p["y"].dtype == np.uint16 else p["y"].astype(np.int32)
    keep = [torch.from_numpy(y).to(DEV), torch.from_numpy(p["r"]).to(DEV), torch.from_numpy(mu32).to(DEV),
            torch.from_numpy(sens32).to(DEV)]
    plan.set_data(*keep)
    plan._test_keep = keep
    return plan, mu32, sens32


def test_c2_alg1_two_epochs_against_oracle():
    from paper_2506_04976_gb300 import binding as pet
    from paper_2506_04976_gb300.presets import petric_solver_kwargs
    p = synth.make_problem("c2", 0)
    n = p["nsub"]
    plan, mu32, sens32 = _device_data(pet, p)
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, mu32, sens32)
    x = np.ones(G.img_shape)
    for s in range(n):  # one OSEM epoch from a uniform image
        x = O.em_update(G, n, s, m, p["r"], p["y"], x)
    x0 = x.astype(np.float32)
    niter = 2 * n
    order = O.subset_order(2024, n, niter)
    kw = petric_solver_kwargs("ALG1", n)
    okw = dict(omega=kw["omega"], step_rule=O.STEP_ALG1, tau0=kw["tau0"], precond_kind=1, alpha=kw["alpha"],
               delta_rel=1e-6, pc_iters=kw["pc_iters"], beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
    xo, taus_o, _ = O.solve(G, x0, m, p["r"], p["y"], O.sensitivity(G, 1, -1, m), algo=O.SVRG, nsub=n,
                            niter=niter, order=order, **okw)
    solver = pet.Solver(plan, beta=p["beta"], gamma=p["gamma"], eps=p["eps"], order=order,
                        **dict(kw, delta_rel=1e-6))
    solver.set_image(torch.from_numpy(x0).to(DEV))
    solver.run(niter)
    torch.cuda.synchronize()
    xg = solver.image().cpu().numpy().astype(np.float64)
    assert np.allclose(solver.taus(), taus_o, rtol=1e-7)
    mask = p["mask"].astype(bool)
    d = np.abs(xg - xo)[mask]
    ref = xo[mask]
    assert np.linalg.norm(d) <= 1e-4 * np.linalg.norm(ref)
    assert np.all(d <= 1e-4 * np.abs(ref) + 1e-5 * ref.max())
    assert np.linalg.norm(xg - xo) <= 1e-4 * np.linalg.norm(xo)


def _c4_problems():
    from tests.geoms import make_spec_problem
    specs = synth.batch_specs(0, 32)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        return pool.map(make_spec_problem, [(100 + i, sp) for i, sp in enumerate(specs)])


def _saga(pet, p, plan, x0, seed):
    n = p["nsub"]
    s = pet.Solver(plan, algo=pet.SAGA, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1,
                   pc_iters=(0, n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"], seed=seed)
    s.set_image(torch.from_numpy(x0).to(DEV))
    return s


def test_c4_batch_of_32_matches_single_runs_and_oracle():
    from paper_2506_04976_gb300 import binding as pet
    probs = _c4_problems()
    inst = []
    for p in probs:
        plan, mu32, sens32 = _device_data(pet, p)
        x0 = np.full(plan.img_shape, float(p["x_true"].mean()), np.float32)
        inst.append((p, plan, mu32, sens32, x0))
    E = 8
    niter = 3 * E + 5  # plain windows (preconditioner updates), graph windows and a tail
    solvers = [_saga(pet, p, plan, x0, 500 + i) for i, (p, plan, _, _, x0) in enumerate(inst)]
    b = pet.Batch(solvers, iters_per_graph=E)
    b.set_grad_shape(2, 1)
    b.run(niter)
    torch.cuda.synchronize()
    xb = [s.image().cpu().numpy().astype(np.float64) for s in solvers]
    taus_b = [s.taus() for s in solvers]
    subs_b = [s.subsets() for s in solvers]
    del b, solvers
    for i, (p, plan, _, _, x0) in enumerate(inst):
        plan.set_grad_shape(2, 1)  # the batch's launch shape: only the atomics' order differs
        s1 = _saga(pet, p, plan, x0, 500 + i)
        s1.run(niter)
        torch.cuda.synchronize()
        x1 = s1.image().cpu().numpy().astype(np.float64)
        # the FP32 atomics add in a different order in every run, batched or not: the
        # bound is 1e-5 or, where a second single run differs from the first by more
        # (low-count instances amplify the rounding over the iterations), twice that
        # run-to-run difference
        s2 = _saga(pet, p, plan, x0, 500 + i)
        s2.run(niter)
        torch.cuda.synchronize()
        d_ss = np.linalg.norm(s2.image().cpu().numpy().astype(np.float64) - x1)
        assert np.linalg.norm(xb[i] - x1) <= max(1e-5 * np.linalg.norm(x1), 2.0 * d_ss), i
        assert np.array_equal(taus_b[i], s1.taus()) and np.array_equal(subs_b[i], s1.subsets()), i
        assert np.array_equal(subs_b[i], O.subset_order(500 + i, p["nsub"], niter)), i
        del s1, s2
    i = min(range(len(inst)), key=lambda k: inst[k][1].N * len(inst[k][0]["geom"]["z1"]))
    p, plan, mu32, sens32, x0 = inst[i]
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, mu32, sens32)
    n = p["nsub"]
    xo, _, _ = O.solve(G, x0, m, p["r"], p["y"], O.sensitivity(G, 1, -1, m), algo=O.SAGA, nsub=n, niter=niter,
                       order=O.subset_order(500 + i, n, niter), step_rule=O.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1,
                       pc_iters=(0, n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
    assert np.linalg.norm(xb[i] - xo) <= 1e-4 * np.linalg.norm(xo)
