"""Pins of the oracle's geometry, Joseph projector and TOF model against facts the
mathematics fixes: adjointness, exact line integrals of constant and linear images,
the dense-matrix transpose, chords through a uniform cylinder, TOF partition of unity
and textbook normal-distribution probabilities."""
import math

import numpy as np
import pytest

import oracle as O
from tests.geoms import geom2d, geom3d, rand_img, rand_sino


def _ip(a, b):
    return float(np.dot(np.ravel(a), np.ravel(b)))


@pytest.mark.parametrize("kind", ["2d", "3d", "3d_tof"])
def test_adjointness(kind):
    g = {"2d": geom2d(9, 13, 11), "3d": geom3d(7, 5, 11, 9),
         "3d_tof": geom3d(7, 5, 11, 9, ntof=5, tof_sigma=6.0, tof_bin=8.0)}[kind]
    G = O.Geometry(g)
    x = rand_img(g, 1)
    y = rand_sino(g, 2)
    lhs = _ip(O.project(G, x), y)
    rhs = _ip(x, O.backproject(G, y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_dense_matrix_transpose_8x8():
    """Column j of A = P e_j, row l of A^T-applied = P^T e_l: the two must agree exactly."""
    for g in (geom2d(8, 12, 8), geom3d(8, 3, 10, 6)):
        G = O.Geometry(g)
        N = g["nx"] * g["ny"] * g["nz"]
        cols = []
        for j in range(N):
            e = np.zeros(N)
            e[j] = 1.0
            cols.append(O.project(G, e.reshape(G.img_shape)).ravel())
        A = np.stack(cols, 1)
        M = A.shape[0]
        rows = []
        for l in range(M):
            e = np.zeros(M)
            e[l] = 1.0
            rows.append(O.backproject(G, e.reshape(G.sino_shape)).ravel())
        AT = np.stack(rows, 1)
        assert np.array_equal(A.T, AT)
        assert (A >= 0).all() and A.sum() > 0


def test_row_through_voxel_centres_is_column_sum():
    """View 0 (phi=0) drives along y; a radial offset landing on voxel column centre
    ix makes the row exactly dy * e_{(iy, ix)} for every iy."""
    g = geom2d(8, 16, 4, d=2.0, drad=2.0)
    G = O.Geometry(g)
    # radial bin r sits at s = (r - 7.5)*2 = -7, -5, ..., voxel centres at (ix-3.5)*2
    for r in range(16):
        s = (r - 7.5) * 2.0
        ix = s / 2.0 + 3.5
        if not (0 <= ix <= 7) or ix != int(ix):
            continue
        vox, wt, _ = O.lor_entries(G, 0, 0, r)
        assert sorted(vox.tolist()) == [iy * 8 + int(ix) for iy in range(8)]
        assert np.allclose(wt, 2.0, rtol=0, atol=1e-12)


def test_constant_and_linear_images_interior_rays():
    """For rays whose transverse coordinate stays inside the grid on every plane, Joseph
    integrates a constant image to c * N_k * step and, because linear interpolation is
    exact for linear functions, a transverse ramp to step * sum of the ramp at the
    intersection points."""
    g = geom2d(16, 9, 12, d=2.0, drad=1.5, rdet=200.0)
    G = O.Geometry(g)
    n = 16
    ctr = (np.arange(n) - 7.5) * 2.0
    X = np.broadcast_to(ctr[None, :], (n, n))
    Y = np.broadcast_to(ctr[:, None], (n, n))
    const = np.full((1, n, n), 3.0)
    checked = 0
    for v in range(12):
        k = O.driving_axis(G, v)
        phi = v * math.pi / 12
        for r in range(9):
            s = (r - 4.0) * 1.5
            u = np.array([-math.sin(phi), math.cos(phi)])
            m = s * np.array([math.cos(phi), math.sin(phi)])
            # intersection with every driving-axis voxel-centre line
            lam = (ctr - m[k]) / u[k]
            pts = m[None, :] + lam[:, None] * u[None, :]
            trans = pts[:, 1 - k]
            if trans.min() < ctr[0] or trans.max() > ctr[-1]:
                continue
            step = 2.0 / abs(u[k])
            ramp = (0.7 * X - 0.3 * Y + 5.0)[None]
            p_const = O.project(G, const, [v])[0, 0, r, 0]
            p_ramp = O.project(G, ramp, [v])[0, 0, r, 0]
            exact_ramp = step * np.sum(0.7 * pts[:, 0] - 0.3 * pts[:, 1] + 5.0)
            assert abs(p_const - 3.0 * n * step) < 1e-9
            assert abs(p_ramp - exact_ramp) < 1e-9 * abs(exact_ramp)
            checked += 1
    assert checked > 20


def test_uniform_cylinder_chords():
    """A uniform cylinder of radius rho and value c: the line integral along an LOR at
    radial offset s is 2 c sqrt(rho^2 - s^2) / cos(theta), theta the axial obliquity.
    The voxelised cylinder agrees within a voxelisation bound O(voxel size)."""
    n, nz, d, dz = 64, 9, 1.0, 2.0
    g = geom3d(n, nz, 41, 8, d=d, dz=dz, drad=1.0, rdet=120.0)
    G = O.Geometry(g)
    rho, c = 20.0, 1.0
    xc = (np.arange(n) - (n - 1) / 2) * d
    X, Y = np.meshgrid(xc, xc)
    img = np.zeros((nz, n, n))
    img[:, X ** 2 + Y ** 2 <= rho ** 2] = c
    proj = O.project(G, img)[..., 0]
    z1, z2 = g["z1"], g["z2"]
    checked = 0
    for p in range(len(z1)):
        # chord must stay inside the axial extent of the image over the cylinder
        if max(abs(z1[p]), abs(z2[p])) > (nz - 1) / 2 * dz - 2.5:
            continue
        for r in range(41):
            s = r - 20.0
            if abs(s) > rho - 3.0:
                continue
            h = math.sqrt(120.0 ** 2 - s ** 2)
            cos_t = 2 * h / math.sqrt(4 * h * h + (z2[p] - z1[p]) ** 2)
            exact = 2 * c * math.sqrt(rho ** 2 - s ** 2) / cos_t
            for v in range(8):
                assert abs(proj[v, p, r] - exact) < 1.5 * d * c / cos_t
                checked += 1
    assert checked > 100


def test_tof_weight_textbook_values():
    """Bin of width 2 sigma centred on the emission point holds P(|Z|<1)/P(|Z|<3)."""
    g = geom3d(4, 1, 4, 4, ntof=1, tof_sigma=10.0, tof_bin=20.0)
    g["ntof"] = 1
    G = O.Geometry(g)
    G.s.ntof = 1  # one bin centred at 0
    w = O.tof_weight(G, 0, 0.0)
    p1, p3 = 0.6826894921370859, 0.9973002039367398  # normal 1- and 3-sigma masses
    assert abs(w - p1 / p3) < 1e-13
    # far beyond 3 sigma + half bin: exactly zero
    assert O.tof_weight(G, 0, 41.0) == 0.0


def test_tof_partition_of_unity_and_nontof_sum():
    g = geom3d(8, 3, 10, 6, ntof=9, tof_sigma=5.0, tof_bin=8.0)
    G = O.Geometry(g)
    T, w = 9, 8.0
    for t in np.linspace(-T * w / 2 + 3 * 5.0, T * w / 2 - 3 * 5.0, 37):
        s = sum(O.tof_weight(G, b, t) for b in range(T))
        assert abs(s - 1.0) < 1e-14
    # symmetry w_b(t) = w_{T-1-b}(-t)
    for t in (-7.3, 0.0, 2.2, 19.9):
        for b in range(T):
            assert abs(O.tof_weight(G, b, t) - O.tof_weight(G, T - 1 - b, -t)) < 1e-15
    # summing TOF bins recovers the non-TOF projection when the bins cover the image
    x = rand_img(g, 5)
    pt = O.project(G, x).sum(-1)
    g1 = dict(g, ntof=1)
    pn = O.project(O.Geometry(g1), x)[..., 0]
    assert np.allclose(pt, pn, rtol=1e-12, atol=1e-12)


def test_tof_centroid_of_point_source():
    """A point source on the LOR midplane away from the TOF range ends: the TOF
    profile is symmetric about the source position along the LOR."""
    g = geom2d(15, 15, 4, d=2.0, drad=2.0)
    g.update(ntof=11, tof_sigma=4.0, tof_bin=3.0)
    G = O.Geometry(g)
    img = np.zeros((1, 15, 15))
    img[0, 7, 7] = 1.0  # centre voxel at the origin
    prof = O.project(G, img)[0, 0, 7]  # view 0, central radial bin passes the origin
    assert prof.sum() > 0
    c = (np.arange(11) - 5) * 3.0
    centroid = (prof * c).sum() / prof.sum()
    assert abs(centroid) < 1e-12
    assert np.allclose(prof, prof[::-1], rtol=1e-12, atol=1e-15)


def test_attenuation_factor_of_water_disk():
    """m = exp(-P mu) for a uniform disk: exp(-mu * chord) within the voxelisation bound."""
    n, d = 64, 2.0
    g = geom2d(n, 31, 6, d=d, drad=4.0, rdet=300.0)
    G = O.Geometry(g)
    xc = (np.arange(n) - (n - 1) / 2) * d
    X, Y = np.meshgrid(xc, xc)
    mu_val, rho = 0.0096, 50.0
    mu = np.where(X ** 2 + Y ** 2 <= rho ** 2, mu_val, 0.0)[None]
    m = O.multiplicative(G, mu, None)
    for r in range(31):
        s = (r - 15) * 4.0
        if abs(s) > rho - 4:
            continue
        ex = math.exp(-2 * mu_val * math.sqrt(rho ** 2 - s ** 2))
        assert np.all(np.abs(m[:, 0, r] - ex) < 2 * d * mu_val * ex)
    sens = np.full(G.lor_shape, 0.5)
    assert np.allclose(O.multiplicative(G, mu, sens), 0.5 * m, rtol=1e-15)


def test_subset_views_every_nth():
    assert O.subset_views(10, 3, 1).tolist() == [1, 4, 7]
    assert O.subset_views(224, 25, 24).tolist() == [24, 49, 74, 99, 124, 149, 174, 199]
    sizes = [len(O.subset_views(224, 25, s)) for s in range(25)]
    assert sizes.count(9) == 24 and sizes.count(8) == 1


def test_driving_axis_rule():
    g = geom2d(8, 8, 8)
    G = O.Geometry(g)
    # 45 degrees (v=2 of 8) drives along x, 0 and 135+ drive along y
    assert [O.driving_axis(G, v) for v in range(8)] == [1, 1, 0, 0, 0, 0, 0, 1]
