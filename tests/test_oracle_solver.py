"""Pins of the oracle's iterative methods (eq. 6-9, Algorithm 1, Table 1, Sec. 2.4,
Sec. 3.1) against special cases with known answers: the MLEM identity, monotone
likelihood, fixed points at consistent data, reductions at n = 1, unbiasedness of the
estimators, KKT conditions at convergence, the stepsize table and the published
splitmix64 output."""
import numpy as np
import pytest

import oracle as O
from paper_2506_04976_gb300 import synth
from tests.geoms import geom2d, geom3d, rand_img, rand_sino


def _data(g, seed=0, consistent=False):
    G = O.Geometry(g)
    xt = rand_img(g, seed, 0.5, 2.0)
    m = 0.5 + 0.5 * rand_sino(g, seed + 1, 0, 1)[..., 0]
    r = rand_sino(g, seed + 2, 0.1, 0.3)
    ybar = m[..., None] * O.project(G, xt) + r
    y = ybar if consistent else np.floor(ybar + rand_sino(g, seed + 3, 0, 1))
    return G, xt, m, r, y


def test_splitmix64_published_outputs():
    assert O.splitmix64_stream(0, 1)[0] == 0xE220A8397B1DCDAF
    assert O.splitmix64_stream(1234567, 5) == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_subset_order_is_a_permutation_each_epoch():
    order = O.subset_order(42, 7, 70)
    for e in range(10):
        assert sorted(order[7 * e:7 * e + 7].tolist()) == list(range(7))
    assert not np.array_equal(order[:7], order[7:14])


def test_table1_alg1_and_alg2():
    vals = {0: 3, 9: 3, 10: 2, 99: 2, 100: 1.5, 199: 1.5, 200: 1, 299: 1, 300: 0.5, 5000: 0.5}
    for k, v in vals.items():
        assert O.step_alg1(k) == v
    n = 25
    assert O.step_alg2(9, n, 10.0) == 3.0 and O.step_alg2(9, n, 0.4) == 0.4
    assert O.step_alg2(10, n, 10.0) == 2.2 and O.step_alg2(2 * n - 1, n, 10.0) == 2.2
    assert O.step_alg2(2 * n, n, 10.0) == 1.0 and O.step_alg2(2 * n, n, 0.7) == 0.7


@pytest.mark.parametrize("tof", [1, 4])
def test_preconditioned_gd_step_equals_mlem(tof):
    """beta = 0, delta = 0, tau = 1, n = 1 and D_MLEM: one step of eq. 6 is exactly the
    MLEM update x A^T(y/ybar) / A^T 1 (Sec. 2.3)."""
    g = geom3d(6, 3, 9, 6, ntof=tof, tof_sigma=6.0, tof_bin=8.0)
    G, xt, m, r, y = _data(g)
    x0 = np.ones(G.img_shape)
    sens = O.sensitivity(G, 1, -1, m)
    x_gd, _, _ = O.solve(G, x0, m, r, y, sens, algo=O.SGD, nsub=1, niter=1, order=[0],
                         step_rule=O.STEP_CONST, tau0=1.0, precond_kind=0, delta_rel=0.0,
                         beta=0.0)
    x_em = O.em_update(G, 1, 0, m, r, y, x0)
    assert np.allclose(x_gd, x_em, rtol=1e-12, atol=1e-14)


def test_mlem_likelihood_monotone():
    g = geom2d(10, 14, 12)
    G, xt, m, r, y = _data(g, 1)
    x = np.ones(G.img_shape)
    prev = np.inf
    for it in range(50):
        val, _ = O.data_grad(G, 1, -1, x, m, r, y, want_grad=False)
        assert val <= prev * (1 + 1e-13)
        prev = val
        x = O.em_update(G, 1, 0, m, r, y, x)


def test_em_fixed_point_at_consistent_data():
    g = geom3d(6, 3, 9, 6)
    G, xt, m, r, y = _data(g, 2, consistent=True)
    for s in range(3):
        assert np.allclose(O.em_update(G, 3, s, m, r, y, xt), xt, rtol=1e-12)


def test_n1_svrg_saga_sgd_equal_projected_gd():
    g = geom2d(8, 12, 10)
    G, xt, m, r, y = _data(g, 3)
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.full(G.img_shape, 1.0)
    kw = dict(nsub=1, niter=6, order=np.zeros(6, np.int32), step_rule=O.STEP_CONST, tau0=0.8,
              precond_kind=1, beta=0.05, pc_iters=(0, 2))
    xs = [O.solve(G, x0, m, r, y, sens, algo=a, **kw)[0] for a in (O.SGD, O.SAGA, O.SVRG)]
    # plain projected GD with the same preconditioner schedule, composed from pinned parts
    x = x0.copy()
    for k in range(6):
        if k in (0, 2):
            _, _, H = O.rdp(x, (g["dx"], g["dy"], g["dz"]), 2.0, 1e-3)
            D = O.precond(x, sens, 0.05 * H, 1.0, 1e-6 * x.max(), kind=1)
        _, gd = O.data_grad(G, 1, -1, x, m, r, y)
        _, gs, _ = O.rdp(x, (g["dx"], g["dy"], g["dz"]), 2.0, 1e-3)
        x = np.maximum(0.0, x - 0.8 * D * (gd + 0.05 * gs))
    for xa in xs:
        assert np.allclose(xa, x, rtol=1e-11, atol=1e-13)


def test_vanishing_step_rule_hand_values():
    """Sec. 2.2's vanishing rule tau_k = tau0 / (1 + eta k / n), k the 0-based update
    index over all epochs: hand-computed values at n = 6, eta = 0.02, tau0 = 1.5 (k
    instead of k/n, k + 1 instead of k, or a dropped tau0 each fail one of them)."""
    g = geom2d(8, 12, 12)
    G, xt, m, r, y = _data(g, 6)
    sens = O.sensitivity(G, 1, -1, m)
    n, niter = 6, 601
    _, taus, _ = O.solve(G, np.full(G.img_shape, 1.0), m, r, y, sens, algo=O.SGD, nsub=n, niter=niter,
                         order=O.subset_order(5, n, niter), step_rule=O.STEP_VANISH, tau0=1.5, eta=0.02,
                         precond_kind=0, beta=0.0, pc_iters=(0,))
    hand = {0: 1.5, 5: 1.4754098360655739, 6: 1.4705882352941176, 12: 1.4423076923076923, 600: 0.5}
    for k, v in hand.items():
        assert taus[k] == pytest.approx(v, rel=1e-15), k


def test_vanishing_step_drives_the_updates():
    """The recorded vanishing steps are the ones the iterates use: three SGD updates
    (n = 2, eta = 0.4, tau0 = 1.5: steps 1.5, 1.25, 1.5/1.4 by hand) composed from the
    pinned data gradient, RDP and preconditioner parts."""
    g = geom2d(8, 12, 12)
    G, xt, m, r, y = _data(g, 7)
    n, beta = 2, 0.05
    sp = (g["dx"], g["dy"], g["dz"])
    sens = O.sensitivity(G, 1, -1, m)
    order = np.array([1, 0, 0], np.int32)
    x0 = np.full(G.img_shape, 1.0)
    xs, taus, _ = O.solve(G, x0, m, r, y, sens, algo=O.SGD, nsub=n, niter=3, order=order,
                          step_rule=O.STEP_VANISH, tau0=1.5, eta=0.4, precond_kind=0, beta=beta,
                          pc_iters=(0,))
    steps = (1.5, 1.25, 1.0714285714285714)
    assert np.allclose(taus, steps, rtol=1e-15)
    x = x0.copy()
    D = O.precond(x, sens, None, 1.0, 1e-6 * x.max(), kind=0)
    for k, i in enumerate(order):
        _, gd = O.data_grad(G, n, int(i), x, m, r, y)
        _, gs, _ = O.rdp(x, sp, 2.0, 1e-3)
        x = np.maximum(0.0, x - steps[k] * D * (n * gd + beta * gs))
    assert np.allclose(xs, x, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("algo", [O.SGD, O.SAGA, O.SVRG])
def test_estimators_unbiased_second_iteration(algo):
    """With no clipping by the prox, averaging iteration 2 over the subset drawn equals
    one full preconditioned gradient step from x^1 (E_i of the SGD, SAGA and SVRG
    estimators is the full gradient; a wrong n factor or a dropped table term fails)."""
    g = geom2d(8, 12, 12)
    G, xt, m, r, y = _data(g, 4)
    n = 4
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.full(G.img_shape, 1.5)
    kw = dict(nsub=n, niter=2, step_rule=O.STEP_CONST, tau0=0.01, precond_kind=1,
              beta=0.1, pc_iters=(0,), omega=2)
    x2s = []
    for i in range(n):
        x2, _, _ = O.solve(G, x0, m, r, y, sens, algo=algo, order=[0, i], **kw)
        x2s.append(x2)
    x1, _, _ = O.solve(G, x0, m, r, y, sens, algo=algo, order=[0, 0], **dict(kw, niter=1))
    assert (np.array(x2s) > 0).all()
    _, _, H = O.rdp(x0, (g["dx"], g["dy"], g["dz"]), 2.0, 1e-3)
    D = O.precond(x0, sens, 0.1 * H, 1.0, 1e-6 * x0.max(), kind=1)
    _, gd = O.data_grad(G, 1, -1, x1, m, r, y)
    _, gs, _ = O.rdp(x1, (g["dx"], g["dy"], g["dz"]), 2.0, 1e-3)
    expect = x1 - 0.01 * D * (gd + 0.1 * gs)
    assert np.allclose(np.mean(x2s, 0), expect, rtol=1e-11, atol=1e-13)


def test_svrg_converges_to_kkt_point():
    """SVRG with the harmonic preconditioner reaches a point satisfying the KKT
    conditions of min sum_i f_i + indicator(x >= 0): grad_j = 0 where x_j > 0 and
    grad_j >= 0 where x_j = 0, measured as ||min(x, grad)|| / ||grad(x0)||."""
    g = geom2d(12, 16, 12)
    G, xt, m, r, y = _data(g, 5)
    n, beta = 3, 0.2
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.ones(G.img_shape)
    niter = 600
    x, taus, _ = O.solve(G, x0, m, r, y, sens, algo=O.SVRG, nsub=n, niter=niter,
                         order=O.subset_order(7, n, niter), step_rule=O.STEP_CONST, tau0=1.0,
                         precond_kind=1, beta=beta, pc_iters=(0, n, 2 * n))

    def full_grad(z):
        _, gd = O.data_grad(G, 1, -1, z, m, r, y)
        _, gs, _ = O.rdp(z, (g["dx"], g["dy"], g["dz"]), 2.0, 1e-3)
        return gd + beta * gs

    g0 = full_grad(x0)
    res = np.linalg.norm(np.minimum(x, full_grad(x))) / np.linalg.norm(g0)
    assert res < 1e-6


def test_bb_step_is_secant_ratio():
    """Short BB step (Sec. 2.2) at the second SVRG refresh: p^T q / q^T D q of the
    snapshot and full-gradient differences in the preconditioner's metric (D computed
    here independently from the start image); before that the start value is used."""
    g = geom2d(8, 12, 8)
    G, xt, m, r, y = _data(g, 6)
    n = 2
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.ones(G.img_shape)
    niter = 9
    order = O.subset_order(3, n, niter)
    kw = dict(algo=O.SVRG, nsub=n, niter=niter, order=order, tau0=0.5, precond_kind=1,
              beta=0.1, pc_iters=(0,), omega=2)
    x, taus, snaps = O.solve(G, x0, m, r, y, sens, step_rule=O.STEP_BB, snap_every=1, **kw)
    assert np.all(taus[:4] == 0.5)

    def full_grad(z):
        _, gd = O.data_grad(G, 1, -1, z, m, r, y)
        _, gs, _ = O.rdp(z, (g["dx"], g["dy"], g["dz"]), 2.0, 1e-3)
        return gd + 0.1 * gs

    p = snaps[3] - x0  # snapshot at k = 4 is x after iteration 3
    q = full_grad(snaps[3]) - full_grad(x0)
    _, _, H = O.rdp(x0, (g["dx"], g["dy"], g["dz"]), 2.0, 1e-3)
    D = O.precond(x0, sens, 0.1 * H, 1.0, 1e-6 * x0.max(), kind=1)
    assert taus[4] == pytest.approx(float((p * q).sum() / (q * D * q).sum()), rel=1e-10)
    assert np.all(taus[4:8] == taus[4])


def test_bb_step_is_dimensionless():
    """The BB step multiplies D grad, like the Table 1 steps it is capped against: on the
    2D workload it is of order one, where the ratio p'q / q'q (units of image / gradient)
    is three orders of magnitude smaller."""
    p = synth.make_problem("c1", 0)
    G = O.Geometry(p["geom"])
    n = p["nsub"]
    m = O.multiplicative(G, p["mu"].astype(np.float32), p["sens"].astype(np.float32))
    sens = O.sensitivity(G, 1, -1, m)
    x = np.ones(G.img_shape)
    for s in range(n):
        x = O.em_update(G, n, s, m, p["r"], p["y"], x)
    niter = 2 * n + 1
    _, taus, _ = O.solve(G, x, m, p["r"], p["y"], sens, algo=O.SVRG, nsub=n, niter=niter,
                         order=O.subset_order(1, n, niter), step_rule=O.STEP_BB, tau0=1.0, precond_kind=1,
                         pc_iters=(0,), beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
    assert 0.05 < taus[2 * n] < 20.0


def test_nrmse_definition():
    x = np.arange(1.0, 7.0)
    ref = x.copy()
    mask = np.ones(6, np.uint8)
    bg = np.array([1, 1, 0, 0, 0, 0], np.uint8)
    assert O.nrmse(x, ref, mask, bg) == 0.0
    assert O.nrmse(x + 0.3, ref, mask, bg) == pytest.approx(0.3 / 1.5, rel=1e-14)


def test_generated_problem_counts_and_shapes():
    p = synth.make_problem("c1", 0)
    assert p["y"].shape == (90, 1, 96, 1)
    assert abs(int(p["y"].sum()) - 1e5) < 5 * np.sqrt(1e5)
    assert abs(p["r"].sum() / 1e5 - 0.1) < 1e-6
    p2 = synth.make_problem("c2", 0, nx=32, nz=23, nrad=64, nview=42)
    assert len(p2["geom"]["z1"]) == 23 + 2 * (23 - 16)
    z1, z2 = synth.planes_span3_segments(24, 5.6)
    assert len(z1) == 109
    z1, z2 = synth.planes_span1(36, 4.0, 1293)
    assert len(z1) == 1293 and np.abs(z1 - z2).max() <= 34 * 4.0 + 1e-9


def test_study_workloads_are_half_resolution_versions():
    """c2s / c2s16 / c3s keep c2's and c3's physics at half the sizes; only c2s16 changes
    the prior strength (16 instead of 4 at 1e7 counts), only c3s carries TOF bins."""
    for name, T, beta in (("c2s", 1, 4 * 2e-4 * 1e7 / 3e7), ("c2s16", 1, 16 * 2e-4 * 1e7 / 3e7),
                          ("c3s", 11, 4 * 2e-4 * 1e6 / 3e7)):
        prm = synth._setup(name, 0)
        g = prm["geom"]
        assert (g["nx"], g["ny"], g["nz"], g["nrad"], g["nview"], g["ntof"]) == (64, 64, 23, 125, 84, T)
        assert len(g["z1"]) == 23 + 2 * (23 - 16) and prm["nsub"] == 21
        assert abs(prm["beta"] - beta) <= 1e-12 * beta
        assert abs(g["dx"] - 4.0) < 1e-12 and abs(g["drad"] - 4.0) < 1e-12
    assert synth._setup("c3s", 0)["geom"]["tof_bin"] == synth._setup("c3", 0)["geom"]["tof_bin"] == 33.0


def test_variance_reduced_estimators_vanish_at_the_minimiser():
    """At the converged image x* (the stored 2D reference, KKT residual ~1e-7) the SVRG and
    SAGA estimators equal grad J(x*), which is ~0 on the support: their iterates stay at x*
    (up to the projection onto x >= 0), while plain SGD, whose estimator n grad f_i(x*) is
    not zero, moves away (eq. 7, eq. 9 vs eq. 6)."""
    import os
    d = np.load(os.path.join(os.path.dirname(__file__), "golden", "ref_c1_seed0.npz"))
    p = synth.make_problem("c1", 0)
    G = O.Geometry(p["geom"])
    n = p["nsub"]
    m = O.multiplicative(G, p["mu"].astype(np.float32), p["sens"].astype(np.float32))
    sens = O.sensitivity(G, 1, -1, m)
    xs = d["x"].astype(np.float64)
    niter = 2 * n + 1
    kw = dict(nsub=n, niter=niter, order=O.subset_order(5, n, niter), step_rule=O.STEP_CONST, tau0=1.0,
              precond_kind=1, pc_iters=(0,), beta=p["beta"], gamma=p["gamma"], eps=p["eps"])
    moved = {}
    for algo in (O.SGD, O.SAGA, O.SVRG):
        x, _, _ = O.solve(G, xs, m, p["r"], p["y"], sens, algo=algo, **kw)
        moved[algo] = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert moved[O.SVRG] < 1e-5 and moved[O.SAGA] < 1e-5  # ~7e-8: the reference's own residual
    assert moved[O.SGD] > 1e-2


def test_bb_step_frozen_after_bb_until():
    """Table 1 computes the BB step of ALG2/ALG3 at the ends of epochs 2, 4 and 6 only:
    with bb_until the step of later refreshes keeps the last value, while without it a
    new secant ratio is taken at every refresh."""
    g = geom2d(8, 12, 8)
    G, xt, m, r, y = _data(g, 6)
    n = 2
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.ones(G.img_shape)
    niter = 13
    kw = dict(algo=O.SVRG, nsub=n, niter=niter, order=O.subset_order(3, n, niter), tau0=0.5, precond_kind=1,
              beta=0.1, pc_iters=(0,), omega=2, step_rule=O.STEP_BB)
    _, t_all, _ = O.solve(G, x0, m, r, y, sens, **kw)
    _, t_frz, _ = O.solve(G, x0, m, r, y, sens, bb_until=4, **kw)
    assert np.array_equal(t_all[:8], t_frz[:8])          # refreshes at k = 0, 4 are the same
    assert np.all(t_frz[8:] == t_frz[4])                  # k = 8, 12: frozen at the k = 4 value
    assert t_all[8] != t_all[4] and t_all[12] != t_all[8]  # recomputed without the limit
