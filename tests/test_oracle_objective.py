"""Pins of the oracle's KL data term, RDP (eq. 3 and Appendix A.1) and
preconditioners (Sec. 2.3, eq. 8): hand-computed values, finite differences,
invariants and the inequalities the paper states."""
import math

import numpy as np
import pytest

import oracle as O
from tests.geoms import geom2d, geom3d, rand_img, rand_sino


# ------------------------------------------------------------------ KL (Sec. 1.2)
def test_kl_hand_values_and_cases():
    assert O.kl_term(2.0, 1.0) == pytest.approx(1.0 - math.log(2.0), abs=1e-15)
    assert O.kl_term(3.0, 3.0) == 0.0
    assert O.kl_term(1.5, 0.0) == 1.5
    assert O.kl_term(0.0, 0.0) == 0.0
    assert math.isinf(O.kl_term(0.0, 1.0))
    assert math.isinf(O.kl_term(-1.0, 0.0))
    rng = np.random.default_rng(0)
    for s, t in rng.uniform(0.01, 10, (200, 2)):
        assert O.kl_term(s, t) >= 0.0


def _problem(g, seed=0):
    G = O.Geometry(g)
    x = rand_img(g, seed, 0.5, 2.0)
    m = 0.5 + 0.5 * rand_sino(g, seed + 1, 0, 1)[..., 0]
    r = rand_sino(g, seed + 2, 0.1, 0.3)
    y = np.floor(3 * rand_sino(g, seed + 3, 0, 2))
    return G, x, m, r, y


@pytest.mark.parametrize("tof", [1, 5])
def test_data_gradient_vanishes_at_consistent_data(tof):
    g = geom3d(6, 3, 9, 6, ntof=tof, tof_sigma=6.0, tof_bin=8.0)
    G, x, m, r, _ = _problem(g)
    ybar = m[..., None] * O.project(G, x) + r
    val, grad = O.data_grad(G, 1, -1, x, m, r, ybar)
    assert abs(val) < 1e-12 * ybar.sum()
    assert np.abs(grad).max() < 1e-12 * O.sensitivity(G, 1, -1, m).max()


@pytest.mark.parametrize("tof", [1, 5])
def test_data_gradient_finite_differences(tof):
    g = geom3d(6, 3, 9, 6, ntof=tof, tof_sigma=6.0, tof_bin=8.0)
    G, x, m, r, y = _problem(g, 3)
    for s in (-1, 1):
        _, grad = O.data_grad(G, 3, s, x, m, r, y)
        rng = np.random.default_rng(1)
        for idx in rng.integers(0, x.size, 12):
            h = 1e-5
            xp, xm = x.copy().ravel(), x.copy().ravel()
            xp[idx] += h
            xm[idx] -= h
            fp, _ = O.data_grad(G, 3, s, xp.reshape(x.shape), m, r, y, want_grad=False)
            fm, _ = O.data_grad(G, 3, s, xm.reshape(x.shape), m, r, y, want_grad=False)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - grad.ravel()[idx]) < 1e-6 * (1 + abs(fd))


def test_subsets_partition_the_data_term():
    g = geom2d(8, 12, 12)
    G, x, m, r, y = _problem(g, 4)
    full, gfull = O.data_grad(G, 1, -1, x, m, r, y)
    parts = [O.data_grad(G, 5, s, x, m, r, y) for s in range(5)]
    assert abs(sum(p[0] for p in parts) - full) < 1e-12 * abs(full)
    assert np.allclose(sum(p[1] for p in parts), gfull, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("tof", [1, 5])
def test_compact_view_pieces_add_up_to_the_subset_data_term(tof):
    """The compact-data form over pieces (one view and a run of planes each) adds up to the
    subset's data term and gradient (eq. 5), and its gradient matches central finite
    differences of its own value."""
    g = geom3d(6, 3, 9, 6, ntof=tof, tof_sigma=6.0, tof_bin=8.0)
    G, x, m, r, y = _problem(g, 5)
    nsub, s = 2, 1
    val, grad = O.data_grad(G, nsub, s, x, m, r, y)
    P = len(g["z1"])
    tot, gsum = 0.0, np.zeros_like(grad)
    for v in O.subset_views(g["nview"], nsub, s):
        for p0, p1 in ((0, 2), (2, P)):
            gk = dict(g, z1=g["z1"][p0:p1], z2=g["z2"][p0:p1])
            vk, gr = O.data_grad_views(O.Geometry(gk), [v], x, m[v:v + 1, p0:p1], r[v:v + 1, p0:p1],
                                       y[v:v + 1, p0:p1])
            tot += vk
            gsum += gr
    assert abs(tot - val) <= 1e-12 * abs(val)
    assert np.allclose(gsum, grad, rtol=1e-12, atol=1e-12 * np.abs(grad).max())
    Gk = O.Geometry(dict(g, z1=g["z1"][1:3], z2=g["z2"][1:3]))
    v = 2
    args = (m[v:v + 1, 1:3], r[v:v + 1, 1:3], y[v:v + 1, 1:3])
    _, gk = O.data_grad_views(Gk, [v], x, *args)
    rng = np.random.default_rng(2)
    for idx in rng.integers(0, x.size, 8):
        h = 1e-5
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[idx] += h
        xm[idx] -= h
        fp, _ = O.data_grad_views(Gk, [v], xp.reshape(x.shape), *args, want_grad=False)
        fm, _ = O.data_grad_views(Gk, [v], xm.reshape(x.shape), *args, want_grad=False)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - gk.ravel()[idx]) < 1e-6 * (1 + abs(fd))


def test_process_pieces_reproduce_the_oracle():
    """oracle.pieces (the oracle split over spawned processes, one view and a run of planes
    per piece) gives the single-process oracle's subset data term, gradient, forward
    projection and backprojection of one view."""
    from oracle import pieces
    g = geom3d(6, 3, 9, 6, ntof=4, tof_sigma=6.0, tof_bin=8.0)
    G = O.Geometry(g)
    x = rand_img(g, 8, 0.5, 2.0)
    mu = rand_img(g, 9, 0.0, 0.01)
    sens = rand_sino(g, 10, 0.8, 1.2)[..., 0]
    r = rand_sino(g, 11, 0.1, 0.3)
    y = np.floor(rand_sino(g, 12, 0.0, 3.0))
    m = O.multiplicative(G, mu, sens)
    nsub, s = 3, 2
    views = O.subset_views(g["nview"], nsub, s)
    val, grad = O.data_grad(G, nsub, s, x, m, r, y)
    pv, pg = pieces.data_grad_subset(g, views, x, mu, sens[views], r[views], y[views], workers=2, chunk=2)
    assert abs(pv - val) <= 1e-12 * abs(val)
    assert np.allclose(pg, grad, rtol=1e-12, atol=1e-12 * np.abs(grad).max())
    v = int(views[1])
    fwd = pieces.forward_view(g, v, x, mu, sens[v], workers=2, chunk=2)
    assert np.allclose(fwd, m[v][..., None] * O.project(G, x, [v])[0], rtol=1e-12, atol=0)
    q = rand_sino(g, 13, -1.0, 1.0)[v]
    bk = pieces.back_view(g, v, q, mu, sens[v], workers=2, chunk=2)
    assert np.allclose(bk, O.backproject(G, (m[v][..., None] * q)[None], [v]), rtol=1e-12,
                       atol=1e-13 * np.abs(bk).max())


@pytest.mark.parametrize("tof", [1, 4])
def test_empty_bins_without_background(tof):
    """Bins with y = 0 and ybar = 0 (LORs that miss the object, no background): the KL
    term d(s, 0) = s of Sec. 1.2 is 0 there and its derivative is 1, so with a zero image,
    zero background and no counts the data term vanishes and its gradient is A^T 1; the
    EM update leaves the zero image at zero."""
    g = geom3d(6, 3, 9, 6, ntof=tof, tof_sigma=6.0, tof_bin=8.0)
    G = O.Geometry(g)
    m = 0.5 + 0.5 * rand_sino(g, 14, 0, 1)[..., 0]
    z = np.zeros(G.sino_shape)
    x = np.zeros(G.img_shape)
    val, grad = O.data_grad(G, 3, 1, x, m, z, z)
    assert val == 0.0 and np.isfinite(grad).all()
    assert np.allclose(grad, O.sensitivity(G, 3, 1, m), rtol=1e-14, atol=0)
    views = O.subset_views(g["nview"], 3, 1)
    vv, gv = O.data_grad_views(G, views, x, m[views], z[views], z[views])
    assert vv == 0.0 and np.allclose(gv, grad, rtol=1e-14, atol=0)
    assert np.array_equal(O.em_update(G, 3, 1, m, z, z, x), x)


def test_sensitivity_is_backprojection_of_ones():
    g = geom3d(6, 3, 9, 6, ntof=4, tof_sigma=6.0, tof_bin=8.0)
    G, x, m, _, _ = _problem(g)
    sens = O.sensitivity(G, 1, -1, m)
    ones = np.ones(G.sino_shape)
    assert np.allclose(sens, O.backproject(G, m[..., None] * ones), rtol=1e-14)
    # <A x, 1> = <x, A^T 1>
    lhs = (m[..., None] * O.project(G, x)).sum()
    assert abs(lhs - (x * sens).sum()) < 1e-12 * lhs


# ------------------------------------------------------------------ RDP (eq. 3)
def test_rdp_two_voxel_hand_values():
    """x = (3, 1), gamma = 2, eps = 0, unit weight: S = d^2/phi = 4/8; dS/dx0 =
    d(2 phi - d - gamma|d|)/phi^2 = 20/64; d2S/dx0^2 = 2 (2 x1)^2/phi^3 = 8/512."""
    x = np.array([[[3.0, 1.0]]])
    S, g, H = O.rdp(x, (1.0, 2.0, 2.0), 2.0, 0.0)
    assert S == pytest.approx(0.5, abs=1e-15)
    assert g[0, 0, 0] == pytest.approx(20 / 64, abs=1e-15)
    # at x1: d = -2, same phi = 8: -2 (16 - (-2 + 4)) / 64 = -28/64 (S depends on the sum,
    # so the two partials are not negatives of each other)
    assert g[0, 0, 1] == pytest.approx(-28 / 64, abs=1e-15)
    assert H[0, 0, 0] == pytest.approx(8 / 512, abs=1e-15)
    # d2S/dx1^2 = 2 (s - d' + eps)^2 / phi^3 with d' = x1 - x0 = -2: 2*36/512
    assert H[0, 0, 1] == pytest.approx(72 / 512, abs=1e-15)


def test_rdp_constant_image_is_flat():
    x = np.full((4, 5, 6), 2.5)
    S, g, H = O.rdp(x, (2.0, 2.0, 2.8), 2.0, 1e-3)
    assert S == 0.0 and np.all(g == 0.0)
    assert np.all(H > 0)


@pytest.mark.parametrize("shape", [(1, 7, 6), (4, 5, 6)])
def test_rdp_gradient_and_hessian_finite_differences(shape):
    rng = np.random.default_rng(2)
    x = rng.uniform(0.1, 3.0, shape)
    kappa = rng.uniform(0.5, 1.5, shape)
    sp, gam, eps = (2.0, 2.0, 2.8), 2.0, 1e-2
    S, g, H = O.rdp(x, sp, gam, eps, kappa)
    for idx in rng.integers(0, x.size, 15):
        h = 1e-5
        xp, xm = x.copy().ravel(), x.copy().ravel()
        xp[idx] += h
        xm[idx] -= h
        Sp, gp, _ = O.rdp(xp.reshape(shape), sp, gam, eps, kappa)
        Sm, gm, _ = O.rdp(xm.reshape(shape), sp, gam, eps, kappa)
        assert abs((Sp - Sm) / (2 * h) - g.ravel()[idx]) < 1e-7 * (1 + abs(g.ravel()[idx]))
        assert abs((gp.ravel()[idx] - gm.ravel()[idx]) / (2 * h) - H.ravel()[idx]) < 1e-6 * (
            1 + abs(H.ravel()[idx]))
        # double FD of S for the Hessian diagonal
        S0 = S
        d2 = (Sp - 2 * S0 + Sm) / h ** 2
        assert abs(d2 - H.ravel()[idx]) < 2e-3 * (1 + abs(H.ravel()[idx]))


def test_rdp_euler_identity_eps0():
    """With eps = 0 the prior is 1-homogeneous, so <grad S(x), x> = S(x)."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0.1, 3.0, (3, 6, 7))
    S, g, _ = O.rdp(x, (2.0, 2.0, 2.8), 2.0, 0.0)
    assert abs((g * x).sum() - S) < 1e-12 * S


def test_rdp_axis_flip_symmetry():
    rng = np.random.default_rng(4)
    x = rng.uniform(0.1, 3.0, (3, 6, 7))
    S, g, H = O.rdp(x, (2.0, 2.0, 2.8), 2.0, 1e-3)
    for ax in range(3):
        Sf, gf, Hf = O.rdp(np.flip(x, ax).copy(), (2.0, 2.0, 2.8), 2.0, 1e-3)
        assert abs(Sf - S) < 1e-12 * S
        assert np.allclose(np.flip(gf, ax), g, rtol=1e-12, atol=1e-14)
        assert np.allclose(np.flip(Hf, ax), H, rtol=1e-12, atol=1e-14)


def test_rdp_tv_limit():
    """phi(s, d) ~ |d|/gamma when s << gamma |d| (Sec. 1.2); for a nonnegative image
    s >= |d|, so the limit needs a large gamma."""
    x = np.array([[[1e-6, 50.0]]])
    gam = 100.0
    S, _, _ = O.rdp(x, (1.0, 1.0, 1.0), gam, 0.0)
    assert abs(S - 50.0 / gam) / (50.0 / gam) < 0.02


def test_rdp_weights_2d_neighbourhood():
    """nz = 1 leaves the 8 in-plane neighbours: a single bright voxel in a zero image
    with gamma=0 and a negligible eps gives S = sum_j w_j x^2/x = x * (4 + 4/sqrt 2);
    in 3D the 26 neighbours give 6 + 12/sqrt 2 + 8/sqrt 3."""
    x = np.zeros((1, 5, 5))
    x[0, 2, 2] = 3.0
    S, _, _ = O.rdp(x, (1.0, 1.0, 1.0), 0.0, 1e-13)
    assert S == pytest.approx(3.0 * (4 + 4 / math.sqrt(2)), rel=1e-12)
    x3 = np.zeros((3, 3, 3))
    x3[1, 1, 1] = 1.0
    S3, _, _ = O.rdp(x3, (1.0, 1.0, 1.0), 0.0, 1e-13)
    assert S3 == pytest.approx(6 + 12 / math.sqrt(2) + 8 / math.sqrt(3), rel=1e-12)


# ------------------------------------------------------------------ preconditioners
def test_precond_beta0_is_mlem_and_bounds():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 3, 200)
    sens = rng.uniform(0.5, 2, 200)
    H = rng.uniform(0.01, 5, 200)
    delta = 1e-3
    Dm = O.precond(x, sens, None, 1.0, delta, kind=0)
    assert np.allclose(Dm, (x + delta) / sens, rtol=1e-15)
    assert np.array_equal(O.precond(x, sens, np.zeros(200), 1.0, delta, kind=1), Dm)
    for alpha in (0.5, 1.0, 3.0):
        Dh = O.precond(x, sens, H, alpha, delta, kind=1)
        # eq. 8: D <= min(D_MLEM, alpha^-1 D_betaS), D_betaS = 1/H
        assert np.all(Dh <= Dm * (1 + 1e-15))
        assert np.all(Dh <= 1.0 / (alpha * H) * (1 + 1e-15))
        # harmonic form: 1/D = 1/D_MLEM + alpha/D_betaS
        assert np.allclose(1 / Dh, 1 / Dm + alpha * H, rtol=1e-13)
