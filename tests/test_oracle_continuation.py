"""Pins of the oracle pieces that the parameter continuation of Sec. 4 needs:
domains of any edge length, d GL / d mu, and the energy (Eq. discr energy)."""
import numpy as np
import pytest

import gl_inputs as gi

BH3 = gi.WORKLOADS["cube128"][3]


@pytest.mark.parametrize("dim,N,field", [(2, 17, (0.0, 0.0, 1.0)), (3, 7, BH3)])
def test_edge_length_scaling(oracle_mod, dim, N, field):
    """Scaling the domain by L: the link phases of A = (mu/2) bhat x x grow by L^2
    (theta_L(mu) = theta_1(mu L^2)), alpha by L^(d-2) (cotangents are scale-free,
    Kuhn tetrahedra scale with length) and |V| by L^d, so K-hat_L(mu) =
    L^(d-2) K-hat_1(mu L^2) and K_L(mu) = K_1(mu L^2) / L^2."""
    L, mu = 10.0, 0.37
    mL = oracle_mod.Mesh(dim, N, mu, field, edge=L)
    m1 = oracle_mod.Mesh(dim, N, mu * L * L, field)
    rpL, ciL, vL = mL.khat_csr()
    rp1, ci1, v1 = m1.khat_csr()
    np.testing.assert_array_equal(rpL, rp1)
    np.testing.assert_array_equal(ciL, ci1)
    np.testing.assert_allclose(vL, L ** (dim - 2) * v1, rtol=1e-12, atol=1e-12 * np.abs(vL).max())
    np.testing.assert_allclose(mL.volumes(), L ** dim * m1.volumes(), rtol=1e-15)
    assert mL.volumes().sum() == pytest.approx(L ** dim, rel=1e-13)
    x = mL.nodes()
    assert x.min() == pytest.approx(-L / 2) and x[:, :dim].max() == pytest.approx(L / 2)


@pytest.mark.parametrize("dim,N,field,edge", [(2, 21, (0.0, 0.0, 1.0), 10.0), (3, 7, BH3, 3.0)])
def test_dmu_central_difference(oracle_mod, dim, N, field, edge):
    """d GL / d mu against the central difference (GL(mu + e) - GL(mu - e)) / 2e
    of two independently assembled meshes (error O(e^2))."""
    mu, eps = 0.41, 1e-5
    psi = gi.disk(N ** dim, 3)
    d = oracle_mod.Mesh(dim, N, mu, field, edge=edge).residual_dmu(psi)
    fd = (oracle_mod.Mesh(dim, N, mu + eps, field, edge=edge).residual(psi)
          - oracle_mod.Mesh(dim, N, mu - eps, field, edge=edge).residual(psi)) / (2 * eps)
    assert np.linalg.norm(d - fd) <= 1e-7 * np.linalg.norm(d), np.linalg.norm(d - fd) / np.linalg.norm(d)
    # a gauge offset a0 does not enter d K / d mu beyond the phases it shifts:
    # at psi = 1 and mu = 0 the derivative is i D^-1 sum_k alpha theta1 (a discrete divergence of A_1)
    m0 = oracle_mod.Mesh(dim, N, 0.0, field, edge=edge)
    d0 = m0.residual_dmu(np.ones(m0.n, complex))
    assert np.abs(d0.real).max() <= 1e-14 * max(1.0, np.abs(d0).max())


def test_dmu_is_orthogonal_to_the_gauge_direction(oracle_mod):
    """<i psi, GL(psi)>_R = 0 for every psi and mu (phase invariance, Sec. 2), so its mu
    derivative <i psi, d GL / d mu>_R vanishes: the bordered continuation system
    stays consistent although J(psi)(i psi) = i GL(psi) is singular at solutions."""
    m = oracle_mod.Mesh(2, 19, 0.6, edge=6.0)
    psi = gi.disk(m.n, 8)
    d = m.residual_dmu(psi)
    assert abs(m.inner_r(1j * psi, d)) <= 1e-12 * np.sqrt(m.inner_r(d, d) * m.inner_r(psi, psi))
    assert abs(m.inner_r(1j * psi, m.residual(psi))) <= 1e-12 * np.sqrt(m.inner_r(psi, psi)) * \
        np.sqrt(m.inner_r(m.residual(psi), m.residual(psi)))


@pytest.mark.parametrize("dim,edge", [(2, 10.0), (3, 4.0)])
def test_energy_of_the_homogeneous_state(oracle_mod, dim, edge):
    """psi = 1 without field: F_1 = 0 and F_2 = sum |V| (-1 + 1/2) = -|Omega| / 2, so
    the energy per unit volume is -1/2 (the start of Fig. 4's energy curve)."""
    N = 9
    m = oracle_mod.Mesh(dim, N, 0.0, edge=edge)
    F = m.energy(np.ones(m.n, complex))
    assert F == pytest.approx(-0.5 * edge ** dim, rel=1e-13)
    # a constant phase changes nothing; with a field, psi = 1 costs kinetic energy
    assert m.energy(np.exp(0.7j) * np.ones(m.n)) == pytest.approx(F, rel=1e-13)
    mf = oracle_mod.Mesh(dim, N, 0.5, edge=edge)
    assert mf.energy(np.ones(m.n, complex)) > F


def test_oracle_continuation_reproduces_fig4(oracle_mod):
    """The oracle's pseudo-arclength continuation on the edge-10 square (33 x 33,
    from psi = 1 at mu = 0): it starts at F/|Omega| = -1/2, folds back first near
    mu = 0.30 (Fig. 4's swallow tail), MINRES needs more iterations past the fold,
    and where the curve first reaches mu = 0.47 after the fold 2F/|Omega| matches
    the paper's printed -0.47 (tests/golden/fig4_continuation_states.txt)."""
    import os

    from oracle import continuation as ocont

    N = 33
    pts, psi, mu = ocont.continuation(2, N, 10.0, np.ones(N * N, complex), 0.0, ds=0.1, ds_max=0.3, max_steps=15,
                                      mu_max=1.2)
    mus = np.array([p["mu"] for p in pts])
    F = np.array([p["energy"] for p in pts])
    its = np.array([p["iters_last"] for p in pts])
    assert F[0] == pytest.approx(-0.5, abs=1e-14) and all(p["gl_norm"] <= 1e-9 for p in pts)
    fold = next(k for k in range(1, len(mus) - 1) if (mus[k] - mus[k - 1]) * (mus[k + 1] - mus[k]) < 0)
    assert 0.29 <= mus[fold] <= 0.32, mus
    assert np.all(np.diff(F[: fold + 1]) > 0)
    assert np.median(its[fold + 1:]) > np.median(its[1:fold])
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig4_continuation_states.txt")) as f:
        mu_p, F_p = [tuple(map(float, ln.split())) for ln in f if ln.strip() and not ln.startswith("#")][0]
    k = next(k for k in range(fold, len(mus) - 1) if (mus[k] - mu_p) * (mus[k + 1] - mu_p) <= 0)
    w = (mu_p - mus[k]) / (mus[k + 1] - mus[k])
    assert abs(2.0 * ((1 - w) * F[k] + w * F[k + 1]) - F_p) <= 0.01


def test_bordered_step_solves_the_bordered_system(oracle_mod):
    """The corrector's block elimination (two MINRES solves with J and a scalar
    border equation) against a dense solve of the realified bordered system
    [J, dGL/dmu; t^T W, t_mu] (dpsi, dmu) = -(GL, n), W the |V|/|Omega| weights
    of the arclength row, on a 5 x 5 mesh."""
    from oracle import continuation as ocont

    N, edge, mu = 5, 4.0, 0.6
    m = oracle_mod.Mesh(2, N, mu, edge=edge)
    n, vol_tot = m.n, edge ** 2
    psi = gi.psi_noisy_one(n, 11, amplitude=0.3)
    g = np.random.default_rng(12)
    t_psi = g.standard_normal(n) + 1j * g.standard_normal(n)
    t_mu, ncond = 0.7, 0.05
    r = m.residual(psi)
    dpsi, dmu, ia, ic = ocont.bordered_step(m, psi, t_psi, t_mu, ncond, r, vol_tot, tol=1e-13, maxit=2000,
                                            max_coarse=4)
    assert ia.converged and ic.converged
    Jr = m.jacobian_dense_real(psi)
    gm = m.residual_dmu(psi)
    vol = m.volumes()
    A = np.zeros((2 * n + 1, 2 * n + 1))
    A[:2 * n, :2 * n] = Jr
    A[:2 * n, 2 * n] = np.concatenate([gm.real, gm.imag])
    # <t, x>_R / |Omega| = sum |V| (Re t Re x + Im t Im x) / |Omega|
    A[2 * n, :2 * n] = np.concatenate([vol * t_psi.real, vol * t_psi.imag]) / vol_tot
    A[2 * n, 2 * n] = t_mu
    rhs = -np.concatenate([r.real, r.imag, [ncond]])
    sol = np.linalg.solve(A, rhs)
    ref = sol[:n] + 1j * sol[n:2 * n]
    assert np.linalg.norm(dpsi - ref) <= 1e-8 * np.linalg.norm(ref)
    assert dmu == pytest.approx(sol[2 * n], rel=1e-8, abs=1e-12)
