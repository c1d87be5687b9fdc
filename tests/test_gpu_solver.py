"""GPU SGD / SAGA / SVRG trajectories (eq. 6-9, Algorithm 1) against the FP64 oracle
run with the same subset order, stepsize rule and preconditioner schedule.

Tolerance: the reconstructed image after several epochs within 1e-4 relative L2 of
the oracle's (FP32 arithmetic along a contractive iteration); stepsizes of the
deterministic rules equal to FP32 rounding; BB stepsizes within 1e-3 relative (a ratio
of FP64 dot products of differences of FP32 images)."""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

_P = {}


def problem(key):
    if key not in _P:
        if key == "c1":
            p = synth.make_problem("c1", 1)
        elif key == "3d":
            p = synth.make_problem("c2", 1, nx=32, nz=13, nrad=56, nview=24, nsub=4)
        else:
            p = synth.make_problem("c3", 1, nx=28, nz=9, nrad=48, nview=20, nsub=4)
        from paper_2506_04976_gb300 import binding as pet
        g = p["geom"]
        plan = pet.Plan(g, p["nsub"])
        mu32, sens32 = p["mu"].astype(np.float32), p["sens"].astype(np.float32)
        plan.set_data(torch.from_numpy(p["y"].astype(np.int32)).to(DEV), torch.from_numpy(p["r"]).to(DEV),
                      torch.from_numpy(mu32).to(DEV), torch.from_numpy(sens32).to(DEV))
        G = O.Geometry(g)
        m = O.multiplicative(G, mu32, sens32)
        sens = O.sensitivity(G, 1, -1, m)
        x0 = np.full(G.img_shape, float(p["x_true"].mean()), np.float32)
        _P[key] = (p, plan, G, m, sens, x0)
    return _P[key]


def _run_both(key, algo, niter, step_rule=O.STEP_VANISH, tau0=1.0, use_graph=True, beta=None,
              pc_iters=None, deterministic=False, precond_kind=1):
    from paper_2506_04976_gb300 import binding as pet
    p, plan, G, m, sens, x0 = problem(key)
    n = p["nsub"]
    beta = p["beta"] if beta is None else beta
    pc = (0, n, 2 * n) if pc_iters is None else pc_iters
    order = O.subset_order(99, n, niter)
    kw = dict(omega=2, step_rule=step_rule, tau0=tau0, eta=0.02, precond_kind=precond_kind, alpha=1.0,
              delta_rel=1e-6, pc_iters=pc, beta=beta, gamma=p["gamma"], eps=p["eps"])
    xo, taus_o, _ = O.solve(G, x0, m, p["r"], p["y"], sens, algo=algo, nsub=n, niter=niter, order=order, **kw)
    s = pet.Solver(plan, algo=algo, order=order, use_graph=use_graph, deterministic=deterministic, **kw)
    s.set_image(torch.from_numpy(x0).to(DEV))
    s.run(niter)
    torch.cuda.synchronize()
    xg = s.image().cpu().numpy().astype(np.float64)
    return xg, xo, s.taus(), taus_o, s


@pytest.mark.parametrize("key", ["c1", "3d", "tof"])
@pytest.mark.parametrize("algo", [O.SVRG, O.SAGA, O.SGD])
def test_trajectory_matches_oracle(key, algo):
    p = problem(key)[0]
    niter = 3 * p["nsub"] + 2  # crosses epoch boundaries, graph and plain iterations
    xg, xo, tg, to, _ = _run_both(key, algo, niter)
    rel = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert rel <= 1e-4, rel
    assert np.allclose(tg, to, rtol=1e-6)
    assert (xg >= 0).all()


@pytest.mark.parametrize("rule", [O.STEP_BB, O.STEP_ALG2, O.STEP_ALG1, O.STEP_CONST])
def test_stepsize_rules(rule):
    p = problem("c1")[0]
    n = p["nsub"]
    niter = 5 * n
    xg, xo, tg, to, _ = _run_both("c1", O.SVRG, niter, step_rule=rule, tau0=0.5)
    assert np.allclose(tg, to, rtol=1e-3)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-4


def test_mlem_preconditioner_path():
    xg, xo, tg, to, _ = _run_both("3d", O.SVRG, 10, precond_kind=0)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-4


def test_graph_and_plain_agree():
    p = problem("3d")[0]
    niter = 2 * p["nsub"]
    a, _, ta, _, _ = _run_both("3d", O.SVRG, niter, use_graph=True)
    b, _, tb, _, _ = _run_both("3d", O.SVRG, niter, use_graph=False)
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= 1e-5
    assert np.array_equal(ta, tb)


def test_deterministic_solver_is_bitwise_reproducible():
    p = problem("c1")[0]
    niter = 2 * p["nsub"] + 1
    a, xo, _, _, _ = _run_both("c1", O.SVRG, niter, deterministic=True)
    b, _, _, _, _ = _run_both("c1", O.SVRG, niter, deterministic=True)
    assert np.array_equal(a, b)
    assert np.linalg.norm(a - xo) / np.linalg.norm(xo) <= 1e-4


def test_seeded_order_matches_oracle_generator():
    """Without an explicit order the solver draws splitmix64 Fisher-Yates permutations
    per epoch from its seed, the same definition as the oracle's generator."""
    from paper_2506_04976_gb300 import binding as pet
    p, plan, G, m, sens, x0 = problem("c1")
    n = p["nsub"]
    niter = 2 * n + 3
    kw = dict(omega=2, step_rule=O.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1, alpha=1.0,
              delta_rel=1e-6, pc_iters=(0,), beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
    s = pet.Solver(plan, algo=O.SAGA, seed=12345, **kw)
    s.set_image(torch.from_numpy(x0).to(DEV))
    s.run(niter)
    xg = s.image().cpu().numpy()
    xo, _, _ = O.solve(G, x0, m, p["r"], p["y"], sens, algo=O.SAGA, nsub=n, niter=niter,
                       order=O.subset_order(12345, n, niter), **kw)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-4


def test_profile_and_launch_counter():
    from paper_2506_04976_gb300 import binding as pet
    p, plan, G, m, sens, x0 = problem("c1")
    n = p["nsub"]
    s = pet.Solver(plan, algo=O.SVRG, beta=p["beta"], pc_iters=(0,))
    s.set_image(torch.from_numpy(x0).to(DEV))
    s.profile(True)
    c0 = pet.launch_count()
    s.run(2 * n)
    torch.cuda.synchronize()
    ms, launches = s.kernel_time()
    assert launches == 3 * n - 1 and ms > 0
    assert pet.launch_count() - c0 > 3 * n
