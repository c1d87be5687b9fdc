"""Pins of the oracle's image-space resolution model (Sec. 3.1: a 4 mm isotropic Gaussian
kernel models the limited spatial resolution; the system matrix becomes P G).

The kernel is checked against what a Gaussian of the given FWHM must satisfy: the
response at half the FWHM is half the peak (which pins sigma = FWHM / (2 sqrt(2 ln 2))),
unit mass, the variance of a normal truncated after ceil(3 sigma / delta) taps, symmetry and separability;
G is its own adjoint with zero padding; the projector with the model stays the exact
transpose of its backprojector; attenuation factors ignore the model."""
import math

import numpy as np
import pytest

import oracle as O
from tests.geoms import geom2d, geom3d, rand_img, rand_sino


def _delta(shape, at):
    x = np.zeros(shape)
    x[at] = 1.0
    return x


def test_half_maximum_at_half_fwhm():
    # FWHM 4 mm sampled every 0.5 mm: the tap at 2 mm is exactly half the centre tap
    y = O.gauss_filter(_delta((1, 1, 61), (0, 0, 30)), (0.5, 1e3, 1e3), 4.0)[0, 0]
    assert y[34] / y[30] == pytest.approx(0.5, rel=1e-12)
    assert y[26] / y[30] == pytest.approx(0.5, rel=1e-12)


def test_mass_variance_and_truncation():
    fwhm, d = 4.0, 0.25
    sigma = fwhm / (2 * math.sqrt(2 * math.log(2)))
    y = O.gauss_filter(_delta((1, 1, 201), (0, 0, 100)), (d, 1e3, 1e3), fwhm)[0, 0]  # no blur across y
    k = (np.arange(201) - 100) * d
    assert y.sum() == pytest.approx(1.0, abs=1e-14)
    # R = ceil(3 sigma / d) taps per side: a normal truncated at t = (R + 1/2) d / sigma
    # (midpoint rule) has variance sigma^2 (1 - 2 t phi(t) / (2 Phi(t) - 1))
    R = math.ceil(3 * sigma / d)
    t = (R + 0.5) * d / sigma
    phit = math.exp(-t * t / 2) / math.sqrt(2 * math.pi)
    Phit = 0.5 * (1 + math.erf(t / math.sqrt(2)))
    var = sigma ** 2 * (1 - 2 * t * phit / (2 * Phit - 1))
    assert float((y * k * k).sum()) == pytest.approx(var, rel=1e-3)
    assert (y[np.abs(np.arange(201) - 100) > R] == 0).all() and (y[np.abs(np.arange(201) - 100) <= R] > 0).all()


def test_point_response_is_separable_and_symmetric():
    shape = (9, 15, 15)
    sp = (2.0, 2.0, 2.8)
    y = O.gauss_filter(_delta(shape, (4, 7, 7)), sp, 4.0)
    ax = y[4, 7, :] / y[4, 7, 7]
    ay = y[4, :, 7] / y[4, 7, 7]
    az = y[:, 7, 7] / y[4, 7, 7]
    assert np.allclose(y / y[4, 7, 7], az[:, None, None] * ay[None, :, None] * ax[None, None, :], rtol=1e-12)
    assert np.allclose(ax, ax[::-1]) and np.allclose(az, az[::-1]) and np.allclose(ax, ay)
    assert y.sum() == pytest.approx(1.0, abs=1e-14)
    # the coarser axial spacing samples the same Gaussian: ratio of the first taps
    sigma = 4.0 / (2 * math.sqrt(2 * math.log(2)))
    assert az[5] == pytest.approx(math.exp(-2.8 ** 2 / (2 * sigma ** 2)), rel=1e-12)


def test_self_adjoint_with_zero_padding():
    rng = np.random.default_rng(1)
    for shape, sp in (((7, 11, 13), (2.0, 2.0, 2.8)), ((1, 12, 12), (2.0, 2.0, 2.0))):
        a, b = rng.random(shape), rng.random(shape)
        Ga, Gb = O.gauss_filter(a, sp, 4.0), O.gauss_filter(b, sp, 4.0)
        assert float((Ga * b).sum()) == pytest.approx(float((a * Gb).sum()), rel=1e-13)
        # zero padding: mass leaks only through the boundary
        assert Ga.sum() <= a.sum() + 1e-12


def test_zero_fwhm_is_identity_and_2d_has_no_axial_blur():
    rng = np.random.default_rng(2)
    a = rng.random((5, 6, 7))
    assert np.array_equal(O.gauss_filter(a, (2, 2, 2), 0.0), a)
    y = O.gauss_filter(_delta((1, 21, 21), (0, 10, 10)), (2.0, 2.0, 2.0), 4.0)
    assert y.sum() == pytest.approx(1.0, abs=1e-14)  # nothing lost to a missing axial neighbour


@pytest.mark.parametrize("kind", ["2d", "3d", "tof"])
def test_projector_with_resolution_model_is_adjoint(kind):
    g = geom2d(10, 14, 12) if kind == "2d" else geom3d(8, 5, 12, 10, ntof=(5 if kind == "tof" else 1))
    g = dict(g, res_fwhm=4.0)
    G = O.Geometry(g)
    x = rand_img(g, 3)
    y = rand_sino(g, 4)
    views = np.arange(g["nview"], dtype=np.int32)
    Ax = O.project(G, x)
    Aty = O.backproject(G, y)
    assert float((Ax * y).sum()) == pytest.approx(float((x * Aty).sum()), rel=1e-12)
    # P G x = P (G x): the model acts on the image only
    G0 = O.Geometry(dict(g, res_fwhm=0.0))
    sp = (g["dx"], g["dy"], g["dz"])
    assert np.allclose(Ax, O.project(G0, O.gauss_filter(x, sp, 4.0)), rtol=1e-12, atol=1e-14)
    assert np.allclose(Aty, O.gauss_filter(O.backproject(G0, y), sp, 4.0), rtol=1e-12, atol=1e-14)
    del views


def test_attenuation_factors_ignore_the_resolution_model():
    g = geom3d(8, 5, 12, 10)
    rng = np.random.default_rng(5)
    mu = 0.01 * rng.random((g["nz"], g["ny"], g["nx"]))
    m1 = O.multiplicative(O.Geometry(dict(g, res_fwhm=4.0)), mu, None)
    m0 = O.multiplicative(O.Geometry(g), mu, None)
    assert np.array_equal(m0, m1)
