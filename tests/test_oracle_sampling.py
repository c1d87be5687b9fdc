"""Pins of the oracle's subset sampling rules (Sec. 2.4): Herman-Meyer order against
bit reversal and hand-derived mixed-radix values, cofactor order against the group of
units of Z_n and a hand-worked n = 10 case, sampling with replacement against the
published splitmix64 outputs and a chi-square bound, the importance draw against
brute-force inverse-CDF rules, and importance-sampled SVRG against the unbiasedness of
its estimator."""
import math

import numpy as np
import pytest

import oracle as O
from tests.geoms import geom2d, rand_img, rand_sino


def _bitrev(j, bits):
    return int(format(j, f"0{bits}b")[::-1], 2) if bits else 0


@pytest.mark.parametrize("bits", [0, 1, 2, 3, 4, 5])
def test_herman_meyer_powers_of_two_are_bit_reversal(bits):
    n = 1 << bits
    assert O.subset_order(0, n, n, O.SAMPLE_HM).tolist() == [_bitrev(j, bits) for j in range(n)]


def test_herman_meyer_hand_values_and_primes():
    # n = 6 = 2 * 3: digit d1 (base 2) weighs 3, d2 (base 3) weighs 1
    assert O.subset_order(0, 6, 6, O.SAMPLE_HM).tolist() == [0, 3, 1, 4, 2, 5]
    # n = 12 = 2 * 2 * 3: weights 6, 3, 1
    assert O.subset_order(0, 12, 12, O.SAMPLE_HM).tolist() == [0, 6, 3, 9, 1, 7, 4, 10, 2, 8, 5, 11]
    for p in (2, 3, 5, 7, 13, 23):  # one prime factor: the identity
        assert O.subset_order(0, p, p, O.SAMPLE_HM).tolist() == list(range(p))


def test_herman_meyer_is_a_permutation_repeated_every_epoch():
    for n in range(1, 41):
        o = O.subset_order(0, n, 3 * n, O.SAMPLE_HM)
        assert sorted(o[:n].tolist()) == list(range(n))
        assert np.array_equal(o[:n], o[n:2 * n]) and np.array_equal(o[:n], o[2 * n:])


def test_cofactor_generators_are_the_units_ranked_by_distance():
    for n in range(1, 41):
        gens = O.cofactor_generators(n).tolist()
        assert sorted(gens) == [g for g in range(1, n) if math.gcd(g, n) == 1]
        d = [min(abs(g - 0.3 * n), abs(g - 0.7 * n)) for g in gens]
        assert all(d[i] <= d[i + 1] + 1e-12 for i in range(len(d) - 1))
    # n = 10: units 1, 3, 7, 9; 0.3 n = 3 and 0.7 n = 7 are units themselves
    assert O.cofactor_generators(10).tolist() == [3, 7, 1, 9]


def test_cofactor_order_hand_worked_and_permutations():
    o = O.subset_order(0, 10, 50, O.SAMPLE_COFACTOR).tolist()
    assert o[:10] == [0, 3, 6, 9, 2, 5, 8, 1, 4, 7]      # generator 3
    assert o[10:20] == [0, 7, 4, 1, 8, 5, 2, 9, 6, 3]    # generator 7
    assert o[20:30] == list(range(10))                   # generator 1
    assert o[30:40] == [0, 9, 8, 7, 6, 5, 4, 3, 2, 1]    # generator 9
    assert o[40:50] == o[:10]                            # list exhausted: start again
    for n in (2, 5, 12, 21, 25, 27, 28):
        oo = O.subset_order(0, n, 6 * n, O.SAMPLE_COFACTOR)
        for e in range(6):
            assert sorted(oo[e * n:(e + 1) * n].tolist()) == list(range(n))
    assert O.subset_order(0, 1, 4, O.SAMPLE_COFACTOR).tolist() == [0, 0, 0, 0]


def test_with_replacement_uses_the_published_stream():
    pub = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    for n in (7, 21, 25):
        assert O.subset_order(1234567, n, 5, O.SAMPLE_REPLACE).tolist() == [((z >> 32) * n) >> 32 for z in pub]
    assert [O.splitmix64_at(1234567, k) for k in range(5)] == pub
    assert O.splitmix64_at(0, 0) == 0xE220A8397B1DCDAF


def test_with_replacement_is_uniform():
    n, draws = 21, 210000
    o = O.subset_order(99, n, draws, O.SAMPLE_REPLACE)
    cnt = np.bincount(o, minlength=n)
    chi2 = float(((cnt - draws / n) ** 2 / (draws / n)).sum())
    assert chi2 < 60.0  # 20 degrees of freedom: P(chi2 > 60) < 1e-5
    # with replacement: some epoch-sized window repeats a subset (a permutation never does)
    assert any(len(set(o[i:i + n].tolist())) < n for i in range(0, 10 * n, n))


def test_draw_index_inverse_cdf():
    rng = np.random.default_rng(3)
    for n in (1, 2, 7, 25):
        p = np.full(n, 1.0 / n)
        for u in rng.random(200):
            assert O.draw_index(p, u) == min(int(math.floor(u * n)), n - 1)
    p = np.array([0.2, 0.0, 0.5, 0.3])
    assert O.draw_index(p, 0.0) == 0 and O.draw_index(p, 0.19999) == 0
    assert O.draw_index(p, 0.2) == 2 and O.draw_index(p, 0.69999) == 2
    assert O.draw_index(p, 0.7) == 3 and O.draw_index(p, 1.0) == 3  # u above the sum: last nonzero
    us = rng.random(40000)
    freq = np.bincount([O.draw_index(p, u) for u in us], minlength=4) / len(us)
    assert np.allclose(freq, p, atol=0.01) and freq[1] == 0


def _data(g, seed=0):
    G = O.Geometry(g)
    xt = rand_img(g, seed, 0.5, 2.0)
    m = 0.5 + 0.5 * rand_sino(g, seed + 1, 0, 1)[..., 0]
    r = rand_sino(g, seed + 2, 0.1, 0.3)
    y = np.floor(m[..., None] * O.project(G, xt) + r + rand_sino(g, seed + 3, 0, 1))
    return G, xt, m, r, y


def test_importance_svrg_estimator_is_unbiased():
    """Iteration 1 after the refresh, averaged over the subset drawn with the
    probabilities p_i = ||grad f_i(x0)|| / sum_j ||grad f_j(x0)|| (computed here from the
    oracle's data gradient and RDP), equals one full preconditioned gradient step from
    x1: the estimator (1/p_i)(grad f_i(x1) - grad f_i(x0)) + grad f(x0) is unbiased.
    A weight of n instead of 1/p_i, or probabilities from the wrong image, fails."""
    g = geom2d(8, 12, 12)
    G, xt, m, r, y = _data(g, 4)
    n, beta, tau = 4, 0.1, 0.01
    sp = (g["dx"], g["dy"], g["dz"])
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.full(G.img_shape, 1.5)
    _, gs0, _ = O.rdp(x0, sp, 2.0, 1e-3)
    nrm = np.array([np.linalg.norm(O.data_grad(G, n, i, x0, m, r, y)[1] + beta / n * gs0) for i in range(n)])
    p = nrm / nrm.sum()
    assert p.max() / p.min() > 1.02  # the test needs unequal probabilities
    kw = dict(algo=O.SVRG, nsub=n, niter=2, order=[0, 0], step_rule=O.STEP_CONST, tau0=tau, precond_kind=1,
              beta=beta, pc_iters=(0,), omega=2, sampling=O.SAMPLE_IMPORTANCE)
    x2 = {}
    for seed in range(400):
        subs = np.zeros(2, np.int32)
        xs, _, _ = O.solve(G, x0, m, r, y, sens, sample_seed=seed, subsets_out=subs, **kw)
        u = (O.splitmix64_at(seed, 1) >> 11) / 2.0 ** 53
        assert subs[0] == -1 and subs[1] == O.draw_index(p, u)
        x2.setdefault(int(subs[1]), xs)
        if len(x2) == n:
            break
    assert len(x2) == n
    x1, _, _ = O.solve(G, x0, m, r, y, sens, **dict(kw, niter=1))
    assert all((v > 0).all() for v in x2.values())
    _, _, H = O.rdp(x0, sp, 2.0, 1e-3)
    D = O.precond(x0, sens, beta * H, 1.0, 1e-6 * x0.max(), kind=1)
    _, gd = O.data_grad(G, 1, -1, x1, m, r, y)
    _, gs, _ = O.rdp(x1, sp, 2.0, 1e-3)
    expect = x1 - tau * D * (gd + beta * gs)
    mean = sum(p[i] * x2[i] for i in range(n))
    assert np.allclose(mean, expect, rtol=1e-11, atol=1e-13)


def test_importance_with_one_subset_is_plain_svrg():
    g = geom2d(8, 12, 12)
    G, xt, m, r, y = _data(g, 5)
    sens = O.sensitivity(G, 1, -1, m)
    x0 = np.full(G.img_shape, 1.0)
    kw = dict(algo=O.SVRG, nsub=1, niter=6, order=[0] * 6, step_rule=O.STEP_CONST, tau0=0.5,
              precond_kind=1, beta=0.1, pc_iters=(0,), omega=2)
    a, _, _ = O.solve(G, x0, m, r, y, sens, **kw)
    b, _, _ = O.solve(G, x0, m, r, y, sens, sampling=O.SAMPLE_IMPORTANCE, sample_seed=7, **kw)
    assert np.array_equal(a, b)
