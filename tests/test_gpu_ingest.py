"""Ingest of a frame's data: the kernel copy from page-locked host memory is bit-exact
(ragged sizes and a 16-byte tail included), refuses pageable or misaligned sources, and a
plan rebound to a second frame with pet_plan_set_counts reads the copied data."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("nbytes", [16, 17, 4096 + 5, 1_000_003, (3 << 20) + 48])
@pytest.mark.parametrize("max_blocks", [0, 1, 3])
def test_copy_to_device_is_bit_exact(nbytes, max_blocks):
    from paper_2506_04976_gb300 import binding as pet
    rng = np.random.default_rng(nbytes)
    host = torch.from_numpy(rng.integers(0, 256, nbytes, dtype=np.uint8)).pin_memory()
    dev = torch.zeros(nbytes, dtype=torch.uint8, device=DEV)
    pet.copy_to_device(dev, host, max_blocks)
    torch.cuda.synchronize()
    assert torch.equal(dev.cpu(), host)


def test_copy_to_device_rejects_bad_sources():
    from paper_2506_04976_gb300 import binding as pet
    dev = torch.zeros(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(ValueError):
        pet.copy_to_device(dev, torch.zeros(64, dtype=torch.uint8))  # pageable
    host = torch.zeros(80, dtype=torch.uint8).pin_memory()
    with pytest.raises(pet.PetError) as e:
        pet.copy_to_device(dev, host[1:65])  # 1 byte past a 16-byte boundary
    assert e.value.status == 1
    with pytest.raises(pet.PetError) as e:
        pet.copy_to_device(dev, host[:64], -1)
    assert e.value.status == 1


def test_second_frame_through_ingest_and_set_counts():
    import oracle as O
    from paper_2506_04976_gb300 import binding as pet, synth
    p = synth.make_problem("c2", 0, nx=40, nz=23, nrad=70, nview=36, nsub=6)
    plan = pet.Plan(p["geom"], 6)
    mu32, sens32 = p["mu"].astype(np.float32), p["sens"].astype(np.float32)
    y1 = torch.from_numpy(p["y"].astype(np.int32)).to(DEV)
    r1 = torch.from_numpy(p["r"]).to(DEV)
    plan.set_data(y1, r1, torch.from_numpy(mu32).to(DEV), torch.from_numpy(sens32).to(DEV))
    rng = np.random.default_rng(3)
    y2 = rng.poisson(0.8 * p["y"].astype(np.float64) + 0.3).astype(np.int32)
    r2 = (1.3 * p["r"].astype(np.float64)).astype(np.float32)
    y2h, r2h = torch.from_numpy(y2).pin_memory(), torch.from_numpy(r2).pin_memory()
    y2d, r2d = torch.empty_like(y1), torch.empty_like(r1)
    pet.copy_to_device(y2d, y2h)
    pet.copy_to_device(r2d, r2h)
    plan.set_counts(y2d, r2d)
    x = np.maximum(p["x_true"], 0.05 * p["x_true"].max()).astype(np.float32)
    obj, g = plan.objective_grad(torch.from_numpy(x).to(DEV), 4)
    G = O.Geometry(p["geom"])
    m = O.multiplicative(G, mu32, sens32)
    val, gd = O.data_grad(G, 6, 4, x, m, r2, y2)
    scale = O.sensitivity(G, 6, 4, m)
    d = np.abs(g.cpu().numpy() - gd)
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(scale)
    assert np.all(d <= 1e-4 * scale + 1e-6 * scale.max())
    assert abs(float(obj) - val) <= 1e-5 * abs(val)


def test_solver_follows_set_counts_between_runs():
    """A solver restarted after pet_plan_set_counts reconstructs the new frame: its graph-
    replayed SVRG epochs equal those of a solver on a plan bound to that frame from the
    start (same launch shape and subset order; only the atomics' order differs)."""
    from paper_2506_04976_gb300 import binding as pet, synth
    p = synth.make_problem("c2", 0, nx=40, nz=23, nrad=70, nview=36, nsub=6)
    mu = torch.from_numpy(p["mu"].astype(np.float32)).to(DEV)
    sens = torch.from_numpy(p["sens"].astype(np.float32)).to(DEV)
    y1 = torch.from_numpy(p["y"].astype(np.int32)).to(DEV)
    r1 = torch.from_numpy(p["r"]).to(DEV)
    rng = np.random.default_rng(11)
    y2 = torch.from_numpy(rng.poisson(1.7 * p["y"].astype(np.float64) + 0.1).astype(np.int32)).to(DEV)
    r2 = torch.from_numpy((0.8 * p["r"].astype(np.float64)).astype(np.float32)).to(DEV)
    x0 = torch.full(tuple(p["x_true"].shape), float(p["x_true"].mean()), device=DEV)
    kw = dict(algo=pet.SVRG, step_rule=pet.STEP_VANISH, tau0=1.0, eta=0.02, precond_kind=1, pc_iters=(0, 6),
              beta=p["beta"], gamma=p["gamma"], eps=p["eps"], seed=5, use_graph=True)
    a = pet.Plan(p["geom"], 6)
    a.set_data(y1, r1, mu, sens)
    a.set_grad_shape(2, 1)
    sa = pet.Solver(a, **kw)
    sa.set_image(x0)
    sa.run(18)
    a.set_counts(y2, r2)
    sa.set_image(x0)
    sa.run(24)
    b = pet.Plan(p["geom"], 6)
    b.set_data(y2, r2, mu, sens)
    b.set_grad_shape(2, 1)
    sb = pet.Solver(b, **kw)
    sb.set_image(x0)
    sb.run(24)
    torch.cuda.synchronize()
    xa, xb = sa.image().cpu().numpy().astype(np.float64), sb.image().cpu().numpy().astype(np.float64)
    assert np.array_equal(sa.subsets(), sb.subsets())
    assert np.linalg.norm(xa - xb) <= 1e-5 * np.linalg.norm(xb)
