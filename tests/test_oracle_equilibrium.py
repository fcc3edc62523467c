"""Pins of the oracle's lattice and entropic equilibrium (Sec. 2, Eq. feq_min)
against facts the paper and the mathematics fix, independent of the oracle's
own formulas."""
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d3q27_weights.txt")


def test_weights_match_golden_table(orc):
    c, w = orc.lattice()
    rows = [ln.split() for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    for name, c2, count, frac in rows:
        sel = (c ** 2).sum(1) == int(c2)
        assert sel.sum() == int(count), name
        assert np.allclose(w[sel], float(Fraction(frac)), rtol=0, atol=1e-16), name
    assert abs(w.sum() - 1.0) < 1e-15


def test_lattice_index_and_opposites(orc):
    c, _ = orc.lattice()
    for i in range(27):
        assert i == 9 * (c[i, 0] + 1) + 3 * (c[i, 1] + 1) + (c[i, 2] + 1)
        assert np.array_equal(c[26 - i], -c[i])


def test_lattice_isotropy_cs2_one_third(orc):
    """Second and fourth moments of the weights are isotropic with c_s^2 = 1/3
    (Sec. 2: c_s = 1/sqrt(3))."""
    c, w = orc.lattice()
    d = np.eye(3)
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, d / 3, atol=1e-15)
    M4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(M4, iso, atol=1e-15)


def _random_rho_u(rng, n, umax=0.2):
    return 1.0 + 0.2 * (rng.random(n) - 0.5), umax * (2 * rng.random((n, 3)) - 1)


def test_feq_conserves_mass_and_momentum(orc):
    c, _ = orc.lattice()
    rng = np.random.default_rng(11)
    rho, u = _random_rho_u(rng, 200)
    for r, uu in zip(rho, u):
        f = orc.feq(r, uu)
        assert abs(f.sum() - r) < 2e-15
        assert np.allclose(c.T @ f, r * uu, rtol=0, atol=2e-15)
        assert (f > 0).all()


def test_feq_log_is_affine_in_velocity(orc):
    """Lagrange condition of Eq. (feq_min): ln(f_i/W_i) = a + b.c_i."""
    c, w = orc.lattice()
    rng = np.random.default_rng(12)
    A = np.hstack([np.ones((27, 1)), c.astype(float)])
    for r, uu in zip(*_random_rho_u(rng, 50, 0.3)):
        y = np.log(orc.feq(r, uu) / w)
        coef, *_ = np.linalg.lstsq(A, y, rcond=None)
        assert np.abs(A @ coef - y).max() < 1e-13


def _entropy_minimiser_newton(w, c, rho, u):
    """Independent route to Eq. (feq_min): the minimiser has the form
    f_i = W_i exp(l0 + l.c_i); solve the four moment equations for (l0, l) by
    Newton's method on the convex dual."""
    lam = np.zeros(4)
    A = np.hstack([np.ones((27, 1)), c.astype(float)])
    target = np.concatenate([[rho], rho * np.asarray(u)])
    for _ in range(100):
        f = w * np.exp(A @ lam)
        res = A.T @ f - target
        if np.abs(res).max() < 1e-16:
            break
        J = A.T @ (f[:, None] * A)
        lam -= np.linalg.solve(J, res)
    return w * np.exp(A @ lam)


def test_feq_equals_numerical_entropy_minimiser(orc):
    c, w = orc.lattice()
    rng = np.random.default_rng(13)
    for r, uu in zip(*_random_rho_u(rng, 40, 0.3)):
        ref = _entropy_minimiser_newton(w, c, r, uu)
        assert np.allclose(orc.feq(r, uu), ref, rtol=1e-13, atol=0)


def test_feq_is_entropy_minimum_under_constraints(orc):
    """Brute force: any perturbation that keeps rho and j raises H."""
    c, _ = orc.lattice()
    rng = np.random.default_rng(14)
    A = np.hstack([np.ones((27, 1)), c.astype(float)])
    # basis of the null space of the moment map
    _, _, vt = np.linalg.svd(A.T)
    null = vt[4:]
    f0 = orc.feq(1.03, [0.07, -0.05, 0.11])
    H0 = orc.entropy(f0)
    for _ in range(200):
        d = null.T @ rng.standard_normal(23)
        d *= 1e-3 * f0.min() / np.abs(d).max()
        assert orc.entropy(f0 + d) > H0


def test_feq_at_rest_is_weights(orc):
    _, w = orc.lattice()
    assert np.allclose(orc.feq(1.0, [0, 0, 0]), w, rtol=0, atol=1e-17)
    assert np.allclose(orc.feq(2.5, [0, 0, 0]), 2.5 * w, rtol=1e-15)


@pytest.mark.parametrize("u", [0.02, 0.05, 0.1])
def test_feq_second_moment_departs_at_fourth_order(orc, u):
    """The exact equilibrium reproduces rho (c_s^2 + u^2) in the second moment
    up to O(u^4), which distinguishes it from the second-order polynomial."""
    c, _ = orc.lattice()
    f = orc.feq(1.0, [u, 0, 0])
    Pxx = (c[:, 0] ** 2 * f).sum()
    dev = Pxx - (1 / 3 + u * u)
    assert abs(dev) < 2 * u ** 4
    assert abs(dev) > 0.1 * u ** 4
