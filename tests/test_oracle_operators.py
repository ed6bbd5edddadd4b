"""Pins of the oracle's nonlinear operators (Eq. discr ginla, the discrete
Jacobian, Eq. discr energy) against the paper's identities and finite differences."""
import numpy as np
import pytest

import gl_inputs as gi

BH3 = gi.WORKLOADS["cube128"][3]


def mesh(oracle_mod, dim, N=7, mu=1.7):
    return oracle_mod.Mesh(dim, N, mu, BH3 if dim == 3 else (0, 0, 1))


@pytest.mark.parametrize("dim", [2, 3])
def test_energy_gradient_is_gl(oracle_mod, dim):
    """d/dt F(psi + t phi) at t = 0 equals 2 <phi, GL(psi)>_R (Euler-Lagrange, Sec. 3)."""
    m = mesh(oracle_mod, dim)
    psi, phi = gi.disk(m.n, 1), gi.complex_normal(m.n, 2)
    eps = 1e-5
    fd = (m.energy(psi + eps * phi) - m.energy(psi - eps * phi)) / (2 * eps)
    assert fd == pytest.approx(2 * m.inner_r(phi, m.residual(psi)), rel=1e-8)


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobian_is_derivative_of_gl(oracle_mod, dim):
    """J(psi) phi = d/de GL(psi + e phi) (Eq. Newton system / Eq. jacobian); central
    differences converge at second order."""
    m = mesh(oracle_mod, dim)
    psi, phi = gi.disk(m.n, 3), gi.complex_normal(m.n, 4)
    J = m.jacobian(psi, phi)
    errs = []
    for eps in (1e-2, 5e-3):
        fd = (m.residual(psi + eps * phi) - m.residual(psi - eps * phi)) / (2 * eps)
        errs.append(np.abs(fd - J).max())
    assert errs[1] < 0.3 * errs[0] and errs[1] < 1e-3 * np.abs(J).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobian_self_adjoint_in_real_inner_product(oracle_mod, dim):
    """<chi, J phi>_R = <J chi, phi>_R (Lemma j self-adjoint, discrete form)."""
    m = mesh(oracle_mod, dim)
    psi = gi.disk(m.n, 5)
    for s in range(3):
        chi, phi = gi.complex_normal(m.n, 10 + s), gi.complex_normal(m.n, 20 + s)
        a, b = m.inner_r(chi, m.jacobian(psi, phi)), m.inner_r(m.jacobian(psi, chi), phi)
        assert a == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobian_i_psi_identity(oracle_mod, dim):
    """J(psi)(i psi) = i GL(psi) for every psi, which gives J(psi_s)(i psi_s) = 0 at
    solutions (Eq. jacobian nullspace)."""
    m = mesh(oracle_mod, dim)
    psi = gi.disk(m.n, 6)
    np.testing.assert_allclose(m.jacobian(psi, 1j * psi), 1j * m.residual(psi), atol=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_gauge_invariance_of_gl(oracle_mod, dim):
    """GL(e^{i chi} psi) = e^{i chi} GL(psi) for constant chi (Sec. 2)."""
    m = mesh(oracle_mod, dim)
    psi = gi.disk(m.n, 7)
    ph = np.exp(0.83j)
    np.testing.assert_allclose(m.residual(ph * psi), ph * m.residual(psi), atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_realified_jacobian_symmetric(oracle_mod, dim):
    """The 2n x 2n real matrix of J times diag(D, D) is symmetric (Remark rmk:isometry
    with the D-weighted inner product), and the realified inner product equals <.,.>_R."""
    m = mesh(oracle_mod, dim, N=5)
    psi = gi.disk(m.n, 8)
    Jr = m.jacobian_dense_real(psi)
    D2 = np.concatenate([m.volumes()] * 2)
    S = D2[:, None] * Jr
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    x, y = gi.complex_normal(m.n, 1), gi.complex_normal(m.n, 2)
    xr, yr = np.concatenate([x.real, x.imag]), np.concatenate([y.real, y.imag])
    assert np.dot(D2 * xr, yr) == pytest.approx(m.inner_r(x, y), rel=1e-13)
    # the realified matrix applied to [Re phi; Im phi] is J phi
    phi = gi.complex_normal(m.n, 3)
    y = Jr @ np.concatenate([phi.real, phi.imag])
    np.testing.assert_allclose(y[: m.n] + 1j * y[m.n:], m.jacobian(psi, phi), atol=1e-12)


def test_jacobian_nullspace_at_newton_solution(oracle_mod):
    """Newton from psi = 1 + noise converges quadratically to a GL solution, where
    i psi spans a kernel direction of J (Eq. jacobian nullspace)."""
    m = oracle_mod.Mesh(2, 12, 2.0)
    psi = gi.psi_noisy_one(m.n, 2)
    norms = []
    for _ in range(8):
        psi_next, gn, info = m.newton_step(psi, tol=1e-12)
        norms.append(gn)
        if gn < 1e-9:
            # psi already solves GL to rounding; the next right-hand side would be
            # noise in the near-kernel direction i psi (Sec. 3), so stop here
            break
        assert info.converged
        psi = psi_next
    assert norms[-1] < 1e-9
    # quadratic convergence: each error at most a modest constant times the square of the last
    for a, b in zip(norms[1:-1], norms[2:]):
        assert b < 5 * a * a + 1e-12
    Jip = m.jacobian(psi, 1j * psi)
    assert np.abs(Jip).max() < 1e-8
