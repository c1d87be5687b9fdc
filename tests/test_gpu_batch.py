"""Batched instances (uneven sizes, betas, count levels and subset counts) advanced by
one launch per phase: each instance's result equals the same solver run alone (up to
the atomics' summation order) and, for one instance, the FP64 oracle's trajectory.  With
SVRG every snapshot refresh (and every preconditioner update) makes its instance run
that window alone while the others stay batched."""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"

SPECS = [
    dict(name="c1", nx=48, nrad=72, nview=60, nsub=6, beta=0.05, counts=3e5),
    dict(name="c2", nx=32, nz=9, nrad=64, nview=28, nsub=7, beta=0.5, counts=2e6),
    dict(name="c1", nx=40, nrad=80, nview=40, nsub=8, beta=0.2, counts=1e6),
    dict(name="c2", nx=24, nz=5, nrad=48, nview=30, nsub=5, beta=0.01, counts=1e7),
]


def _instances():
    from paper_2506_04976_gb300 import binding as pet
    out = []
    for i, sp in enumerate(SPECS):
        sp = dict(sp)
        name = sp.pop("name")
        p = synth.make_problem(name, 10 + i, **sp)
        plan = pet.Plan(p["geom"], p["nsub"])
        mu32, sens32 = p["mu"].astype(np.float32), p["sens"].astype(np.float32)
        plan.set_data(torch.from_numpy(p["y"].astype(np.int32)).to(DEV), torch.from_numpy(p["r"]).to(DEV),
                      torch.from_numpy(mu32).to(DEV), torch.from_numpy(sens32).to(DEV))
        x0 = np.full(plan.img_shape, float(p["x_true"].mean()), np.float32)
        out.append((p, plan, mu32, sens32, x0))
    return out


def _solver(pet, p, plan, x0, seed, algo, step_rule=None):
    n = p["nsub"]
    s = pet.Solver(plan, algo=algo, step_rule=pet.STEP_VANISH if step_rule is None else step_rule, tau0=1.0,
                   eta=0.02, precond_kind=1, pc_iters=(0, n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"],
                   seed=seed)
    s.set_image(torch.from_numpy(x0).to(DEV))
    return s


@pytest.mark.parametrize("algo", ["saga", "sgd", "svrg", "svrg_bb"])
def test_batch_matches_single_runs_and_oracle(algo):
    from paper_2506_04976_gb300 import binding as pet
    A = {"saga": pet.SAGA, "sgd": pet.SGD}.get(algo, pet.SVRG)
    rule = pet.STEP_BB if algo == "svrg_bb" else pet.STEP_VANISH
    inst = _instances()
    E, niter = 4, 3 * 4 + 19  # graph epochs, plain windows (preconditioner updates) and a tail
    if algo == "svrg":
        niter = 2 * 16 + 11  # several snapshot refreshes of every instance
    elif algo == "svrg_bb":
        # one BB step per instance (computed at its second refresh, k = 2n <= 16): a BB step
        # is a ratio of dot products of differences of nearly equal images, so later steps
        # amplify the atomics' rounding differences between the two runs
        niter = 2 * 8 + 2
    solvers = [_solver(pet, p, plan, x0, 100 + i, A, rule) for i, (p, plan, _, _, x0) in enumerate(inst)]
    b = pet.Batch(solvers, iters_per_graph=E)
    b.run(niter)
    torch.cuda.synchronize()
    xb = [s.image().cpu().numpy().astype(np.float64) for s in solvers]
    taus_b = [s.taus() for s in solvers]
    del b
    for i, (p, plan, mu32, sens32, x0) in enumerate(inst):
        s1 = _solver(pet, p, plan, x0, 100 + i, A, rule)
        s1.run(niter)
        torch.cuda.synchronize()
        x1 = s1.image().cpu().numpy().astype(np.float64)
        assert np.linalg.norm(xb[i] - x1) <= 1e-5 * np.linalg.norm(x1), i
        if rule == pet.STEP_BB:  # BB steps: ratios of FP64 dot products of FP32 images
            assert np.allclose(taus_b[i], s1.taus(), rtol=1e-5)
        else:
            assert np.array_equal(taus_b[i], s1.taus())
    # instance 1 (3D) against the oracle with the same subset order
    p, plan, mu32, sens32, x0 = inst[1]
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, mu32, sens32)
    n = p["nsub"]
    xo, _, _ = O.solve(G, x0, m, p["r"], p["y"], O.sensitivity(G, 1, -1, m), algo=A, nsub=n, niter=niter,
                       order=O.subset_order(101, n, niter), step_rule=rule, tau0=1.0, eta=0.02,
                       precond_kind=1, pc_iters=(0, n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
    assert np.linalg.norm(xb[1] - xo) <= 1e-4 * np.linalg.norm(xo)


def test_batch_with_kappa_weighted_priors():
    """Instances with a kappa image (eq. 3 weights) mixed with plain ones: each equals its
    solver run alone, and the kappa-weighted 3D instance equals the oracle's trajectory."""
    from paper_2506_04976_gb300 import binding as pet
    inst = _instances()
    kap = {}
    for i in (1, 2):
        shape = inst[i][1].img_shape
        kap[i] = (0.5 + synth.random_image_like(inst[i][0]["geom"], 40 + i)).astype(np.float32).reshape(shape)
    E, niter = 4, 3 * 4 + 7

    def make(i, p, plan, x0):
        n = p["nsub"]
        kt = torch.from_numpy(kap[i]).to(DEV) if i in kap else None
        s = pet.Solver(plan, algo=pet.SAGA, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1,
                       pc_iters=(0, n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"], kappa=kt, seed=300 + i)
        s._test_kappa = kt
        s.set_image(torch.from_numpy(x0).to(DEV))
        return s

    solvers = [make(i, p, plan, x0) for i, (p, plan, _, _, x0) in enumerate(inst)]
    b = pet.Batch(solvers, iters_per_graph=E)
    b.set_grad_shape(2, 1)
    b.run(niter)
    torch.cuda.synchronize()
    xb = [s.image().cpu().numpy().astype(np.float64) for s in solvers]
    del b, solvers
    for i, (p, plan, _, _, x0) in enumerate(inst):
        plan.set_grad_shape(2, 1)
        s1 = make(i, p, plan, x0)
        s1.run(niter)
        torch.cuda.synchronize()
        x1 = s1.image().cpu().numpy().astype(np.float64)
        assert np.linalg.norm(xb[i] - x1) <= 1e-5 * np.linalg.norm(x1), i
        del s1
    p, plan, mu32, sens32, x0 = inst[1]
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, mu32, sens32)
    n = p["nsub"]
    xo, _, _ = O.solve(G, x0, m, p["r"], p["y"], O.sensitivity(G, 1, -1, m), algo=O.SAGA, nsub=n, niter=niter,
                       order=O.subset_order(301, n, niter), step_rule=O.STEP_VANISH, tau0=1.0, eta=0.02,
                       precond_kind=1, pc_iters=(0, n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"],
                       kappa=kap[1].astype(np.float64))
    assert np.linalg.norm(xb[1] - xo) <= 1e-4 * np.linalg.norm(xo)


def test_batch_autotune_and_shapes():
    from paper_2506_04976_gb300 import binding as pet
    inst = _instances()
    results = []
    for shape in ("auto", (1, 1), (4, 4), (2, 8)):
        solvers = [_solver(pet, p, plan, x0, 200 + i, pet.SAGA) for i, (p, plan, _, _, x0) in enumerate(inst)]
        b = pet.Batch(solvers, iters_per_graph=5)
        if shape == "auto":
            k, sp = b.autotune()
            assert k in (1, 2, 4) and sp in (1, 2, 4, 8)
        else:
            b.set_grad_shape(*shape)
        b.run(2 * 5 + 8)
        torch.cuda.synchronize()
        results.append([s.image().cpu().numpy().astype(np.float64) for s in solvers])
        del b, solvers
    for other in results[1:]:
        for a, c in zip(results[0], other):
            assert np.linalg.norm(a - c) <= 1e-5 * np.linalg.norm(a)


def test_batch_rejects_shared_plans_and_mixed_algorithms():
    from paper_2506_04976_gb300 import binding as pet
    inst = _instances()
    p, plan, _, _, x0 = inst[0]
    s1 = _solver(pet, p, plan, x0, 1, pet.SAGA)
    s2 = _solver(pet, p, plan, x0, 2, pet.SAGA)
    with pytest.raises(pet.PetError):
        pet.Batch([s1, s2])
    p2, plan2, _, _, x02 = inst[1]
    s3 = _solver(pet, p2, plan2, x02, 3, pet.SGD)
    with pytest.raises(pet.PetError):
        pet.Batch([s1, s3])


def test_batch_runs_unbatched_options_alone():
    """A TOF plan, the deterministic backprojector and the table-free SVRG have no batched
    form: inside a batch they run alone in every window and give the results of the same
    solvers run on their own, while the other instances stay batched."""
    from paper_2506_04976_gb300 import binding as pet
    inst = _instances()
    pt = synth.make_problem("c3", 21, nx=24, nz=7, nrad=40, nview=24, nsub=4)
    plan_t = pet.Plan(pt["geom"], pt["nsub"])
    plan_t.set_data(torch.from_numpy(pt["y"].astype(np.int32)).to(DEV), torch.from_numpy(pt["r"]).to(DEV),
                    torch.from_numpy(pt["mu"].astype(np.float32)).to(DEV),
                    torch.from_numpy(pt["sens"].astype(np.float32)).to(DEV))
    x0t = np.full(plan_t.img_shape, float(pt["x_true"].mean()), np.float32)
    cases = [(inst[0][0], inst[0][1], inst[0][4], {}), (inst[1][0], inst[1][1], inst[1][4], {}),
             (inst[2][0], inst[2][1], inst[2][4], dict(deterministic=True)), (pt, plan_t, x0t, {}),
             (inst[3][0], inst[3][1], inst[3][4], dict(low_memory=True))]

    def make(i, p, plan, x0, extra):
        n = p["nsub"]
        s = pet.Solver(plan, algo=pet.SVRG, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1,
                       pc_iters=(0, n), beta=p["beta"], gamma=p["gamma"], eps=p["eps"], seed=400 + i, **extra)
        s.set_image(torch.from_numpy(x0).to(DEV))
        return s

    niter = 3 * 4 + 6
    solvers = [make(i, *c) for i, c in enumerate(cases)]
    b = pet.Batch(solvers, iters_per_graph=4)
    b.set_grad_shape(2, 1)
    b.run(niter)
    torch.cuda.synchronize()
    xb = [s.image().cpu().numpy().astype(np.float64) for s in solvers]
    del b, solvers
    for i, (p, plan, x0, extra) in enumerate(cases):
        plan.set_grad_shape(2, 1)
        s1 = make(i, p, plan, x0, extra)
        s1.run(niter)
        torch.cuda.synchronize()
        x1 = s1.image().cpu().numpy().astype(np.float64)
        if extra.get("deterministic"):
            assert np.array_equal(xb[i], x1), i  # the voxel-driven gather has a fixed order
        else:
            assert np.linalg.norm(xb[i] - x1) <= 1e-5 * np.linalg.norm(x1), i


def test_c4_specs_shape():
    sp = synth.batch_specs(0, 32)
    assert len(sp) == 32
    for s in sp:
        assert 96 <= s["nx"] <= 192 and s["nx"] % 8 == 0
        assert 8 <= s["nsub"] <= 28 and s["nview"] % s["nsub"] == 0
        assert s["nrad"] == round(1.95 * s["nx"])
        assert 0.01 <= s["beta"] <= 1 and 1e5 <= s["counts"] <= 1e8
