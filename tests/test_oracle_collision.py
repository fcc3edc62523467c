"""Pins of the oracle's KBC collision (Sec. 2, Eqs. kineticEq, kbc_relax,
gamma_min and the analytic stabilizer) against conservation, the moment
structure of the split, the entropy condition and the LBGK special cases."""
import itertools

import numpy as np
import pytest


def _random_state(orc, rng, amp=0.02):
    rho = 1 + 0.02 * (rng.random() - 0.5)
    u = 0.1 * (2 * rng.random(3) - 1)
    fe = orc.feq(rho, u)
    return fe * (1 + amp * rng.standard_normal(27))


def _moment_matrix(c):
    """All 27 natural moments M_pqr = sum f cx^p cy^q cz^r, p,q,r in {0,1,2}."""
    rows = [np.prod([c[:, a] ** e for a, e in enumerate(pqr)], axis=0)
            for pqr in itertools.product(range(3), repeat=3)]
    return np.array(rows, dtype=float), list(itertools.product(range(3), repeat=3))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_collision_conserves_mass_and_momentum(orc, mode):
    c, _ = orc.lattice()
    rng = np.random.default_rng(21 + mode)
    for _ in range(100):
        f = _random_state(orc, rng)
        out, _ = orc.collide(f, 0.97, mode)
        assert abs(out.sum() - f.sum()) < 2e-15
        assert np.allclose(c.T @ out, c.T @ f, rtol=0, atol=2e-15)


def test_shear_part_carries_exactly_the_deviatoric_moments(orc):
    """ds has the deviatoric second moments of df and no other natural moment;
    dh has every natural moment of df except those."""
    c, _ = orc.lattice()
    M, idx = _moment_matrix(c)
    rng = np.random.default_rng(22)
    for _ in range(50):
        f = _random_state(orc, rng, 0.05)
        fe, ds, dh = orc.kbc_split(f)
        df = f - fe
        P = np.einsum("ia,ib,i->ab", c, c, df)
        dev = P - np.eye(3) * np.trace(P) / 3
        mds, mdh, mdf = M @ ds, M @ dh, M @ df
        for k, (p, q, r) in enumerate(idx):
            if p + q + r == 2:
                a = [ax for ax, e in enumerate((p, q, r)) for _ in range(e)]
                assert abs(mds[k] - dev[a[0], a[1]]) < 1e-16
            else:
                assert abs(mds[k]) < 1e-16
        # dh keeps df's trace and every moment of order != 2
        for k, (p, q, r) in enumerate(idx):
            if p + q + r != 2:
                assert abs(mdh[k] - mdf[k]) < 1e-16
        Ph = np.einsum("ia,ib,i->ab", c, c, dh)
        assert np.allclose(Ph, np.eye(3) * np.trace(P) / 3, atol=1e-16)


def test_kbc_split_face_edge_table(orc):
    """For a single deviatoric moment the shear part is the tensor-product dual
    function: faces get (2 N_xz - N_yz)/6, (-N_xz + 2 N_yz)/6, (-N_xz - N_yz)/6
    on +-x, +-y, +-z, and the rest, edges and corners get 0."""
    c, w = orc.lattice()
    fe = orc.feq(1.0, [0, 0, 0])
    # perturbation with only M200 - M002 != 0 among second moments: +e on +-x faces,
    # -e on +-z faces (keeps mass, momentum, trace)
    e = 1e-4
    d = np.zeros(27)
    for i in range(27):
        if tuple(c[i]) in [(1, 0, 0), (-1, 0, 0)]:
            d[i] = e
        if tuple(c[i]) in [(0, 0, 1), (0, 0, -1)]:
            d[i] = -e
    _, ds, dh = orc.kbc_split(fe + d)
    # second moments: M200 = 2e, M002 = -2e -> N_xz = 4e, N_yz = 2e
    nxz, nyz = 4 * e, 2 * e
    for i in range(27):
        t = tuple(c[i])
        if t in [(1, 0, 0), (-1, 0, 0)]:
            assert abs(ds[i] - (2 * nxz - nyz) / 6) < 1e-12 * e
        elif t in [(0, 1, 0), (0, -1, 0)]:
            assert abs(ds[i] - (-nxz + 2 * nyz) / 6) < 1e-12 * e
        elif t in [(0, 0, 1), (0, 0, -1)]:
            assert abs(ds[i] - (-nxz - nyz) / 6) < 1e-12 * e
        else:
            assert abs(ds[i]) < 1e-12 * e


def test_lbgk_mode_is_bgk_with_twice_beta(orc):
    rng = np.random.default_rng(23)
    for beta in [0.6, 0.9, 0.999]:
        f = _random_state(orc, rng)
        rho = f.sum()
        c, _ = orc.lattice()
        u = c.T @ f / rho
        ref = f - 2 * beta * (f - orc.feq(rho, u))
        out, g = orc.collide(f, beta, 2)
        assert g == 2.0
        assert np.allclose(out, ref, rtol=1e-12, atol=0)


A0 = lambda x: 1.0 - x * x
A1 = lambda x: 0.5 * x
A2 = lambda x: 0.5 * (3 * x * x - 2)


def test_pure_shear_perturbation_lands_in_s(orc):
    """A perturbation built from the deviatoric dual functions is assigned
    entirely to the shear part (dh at round-off)."""
    c, _ = orc.lattice()
    fe = orc.feq(1.01, [0.03, -0.02, 0.04])
    rng = np.random.default_rng(24)
    for _ in range(20):
        nxz, nyz, pxy, pxz, pyz = 1e-4 * rng.standard_normal(5)
        dxx, dyy, dzz = (2 * nxz - nyz) / 3, (-nxz + 2 * nyz) / 3, (-nxz - nyz) / 3
        p = np.array([dxx * A2(a) * A0(b) * A0(z) + dyy * A0(a) * A2(b) * A0(z)
                      + dzz * A0(a) * A0(b) * A2(z) + pxy * A1(a) * A1(b) * A0(z)
                      + pxz * A1(a) * A0(b) * A1(z) + pyz * A0(a) * A1(b) * A1(z)
                      for a, b, z in c])
        _, ds, dh = orc.kbc_split(fe + p)
        assert np.abs(dh).max() < 1e-10 * np.abs(p).max()
        assert np.allclose(ds, p, rtol=0, atol=1e-10 * np.abs(p).max())


def test_no_shear_nonequilibrium_relaxes_h_fully(orc):
    """With ds = 0 the analytic stabilizer is g = 1/beta, so b g = 1 and the
    higher moments relax fully: f' = f - dh = f^eq."""
    c, _ = orc.lattice()
    fe = orc.feq(0.99, [-0.02, 0.05, 0.01])
    rng = np.random.default_rng(28)
    for beta in [0.7, 0.95, 0.999]:
        m = 1e-4 * rng.standard_normal(4)
        # third- and fourth-order natural moments only (M210, M111, M220, M222)
        p = np.array([m[0] * A2(a) * A1(b) * A0(z) + m[1] * A1(a) * A1(b) * A1(z)
                      + m[2] * A2(a) * A2(b) * A0(z) + m[3] * A2(a) * A2(b) * A2(z)
                      for a, b, z in c])
        f = fe + p
        _, ds, dh = orc.kbc_split(f)
        assert np.abs(ds).max() < 1e-10 * np.abs(p).max()
        out, g = orc.collide(f, beta, 0)
        assert g == pytest.approx(1 / beta, rel=1e-8)
        assert np.allclose(out, fe, rtol=0, atol=1e-9 * np.abs(p).max())


def test_beta_one_half_returns_equilibrium(orc):
    """beta = 1/2 gives g = 1/b - (2 - 1/b) r = 2 for every ratio r, so
    f' = f - (ds + dh) = f^eq."""
    c, _ = orc.lattice()
    rng = np.random.default_rng(25)
    for _ in range(30):
        f = _random_state(orc, rng, 0.05)
        out, g = orc.collide(f, 0.5, 0)
        assert g == pytest.approx(2.0, abs=1e-14)
        rho = f.sum()
        assert np.allclose(out, orc.feq(rho, c.T @ f / rho), rtol=1e-14, atol=0)


def test_exact_stabilizer_solves_entropy_condition(orc):
    """The exact g zeroes Eq. (gamma_min) and minimises H(f'(g)) on a scan."""
    rng = np.random.default_rng(26)
    beta = 0.98
    for _ in range(20):
        f = _random_state(orc, rng, 0.03)
        fe, ds, dh = orc.kbc_split(f)
        g = orc.gamma_exact(ds, dh, fe, beta)
        scale = np.abs(dh).sum() * 10
        assert abs(orc.gamma_residual(ds, dh, fe, beta, g)) < 1e-15 * scale + 1e-18
        Hg = orc.entropy(f - beta * (2 * ds + g * dh))
        for gg in g + np.linspace(-0.5, 0.5, 41):
            fp = f - beta * (2 * ds + gg * dh)
            if (fp > 0).all():
                assert orc.entropy(fp) >= Hg - 1e-15
        out, g2 = orc.collide(f, beta, 1)
        assert g2 == g


def test_analytic_stabilizer_converges_to_exact(orc):
    """The analytic g is the root of Eq. (gamma_min) with the logarithm
    expanded to first order in the deviations (ds, dh)/f^eq; the next order
    of the expansion is smaller by one power of the deviation, so along a
    fixed perturbation direction scaled by eps, g_analytic - g_exact = C eps
    + O(eps^2): the fitted order over eps = 1e-3 ... 1e-5 is 1 and the error
    over eps settles to a constant.  A wrong factor or sign in the analytic
    formula leaves an O(1) error and fails both."""
    rng = np.random.default_rng(27)
    beta = 0.99
    fe0 = orc.feq(1.0, [0.04, 0.02, -0.03])
    eps_l = np.array([1e-3, 3e-4, 1e-4, 3e-5, 1e-5])
    for _ in range(10):
        d = rng.standard_normal(27)
        errs = []
        for eps in eps_l:
            f = fe0 * (1 + eps * d)
            fe, ds, dh = orc.kbc_split(f)
            _, ga = orc.collide(f, beta, 0)
            errs.append(abs(ga - orc.gamma_exact(ds, dh, fe, beta)))
        errs = np.array(errs)
        slope = np.polyfit(np.log(eps_l), np.log(errs), 1)[0]
        assert abs(slope - 1.0) < 0.05
        c = errs / eps_l
        assert abs(c[-1] - c[-2]) < 0.02 * c[-1]
        assert errs[-1] < 1e-4
