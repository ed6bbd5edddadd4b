"""Pins of the FP64 warm-start network oracle (``oracle/warmstart.py``).

The network is the project's own definition (the paper has no learned part); it
is pinned by
* central differences of its loss against the analytic backward pass,
* hand-built weight settings for which the network reduces to closed forms tied
  to independently pinned operators: the Jacobi guess b / diag(K) and the
  magnetic Jacobi operator S = I - diag(K)^-1 K (K from the C oracle's kinetic
  apply, Eq. (10)),
* the loss at the exact solution (dense direct solve) and at zero,
* Adam's closed-form steps under a constant gradient.
"""
import numpy as np
import pytest

import gl_inputs as gi
from oracle import warmstart as ws

C = ws.C


def small_case(oracle_mod, dim=2, N=6, mu=1.0, seed=3):
    bhat = (0.0, 0.0, 1.0) if dim == 2 else tuple(np.ones(3) / np.sqrt(3))
    m = oracle_mod.Mesh(dim, N, mu, bhat)
    g = ws.Graph(m)
    psi = gi.disk(m.n, seed)
    b = gi.complex_normal(m.n, seed + 1)
    return m, g, psi, b


def kinetic_diag(m):
    """K_ii from the C oracle's K apply on unit vectors (independent of khat_csr)."""
    d = np.zeros(m.n)
    for i in range(m.n):
        e = np.zeros(m.n, np.complex128)
        e[i] = 1.0
        d[i] = m.kinetic(e)[i].real
    return d


def set_identity_tail(theta, first_layer):
    """Layers 1..3 pass channels 0..3 through; the head returns
    (h0 - h1) + i (h2 - h3).  Layer 0 is set by first_layer(W0)."""
    Ws, U = ws.split(theta)
    theta[:] = 0.0
    first_layer(Ws[0])
    for W in Ws[1:]:
        for c in range(4):
            W[c, c] = 1.0
    U[0, 0], U[0, 1], U[1, 2], U[1, 3] = 1.0, -1.0, 1.0, -1.0
    return theta


@pytest.mark.parametrize("dim,N", [(2, 6), (3, 4)])
def test_gradient_central_differences(oracle_mod, dim, N):
    m, g, psi, b = small_case(oracle_mod, dim, N)
    theta = gi.warmstart_init(5).astype(np.float64)
    L, grad = ws.loss_and_grad(theta, g, psi, b)
    assert 0 < L
    rng = gi.rng(9)
    Ws, U = ws.split(np.arange(ws.NPARAM))
    blocks = [w for w in Ws] + [U]
    checked = 0
    for blk in blocks:
        idx = blk.ravel()
        gmax = np.max(np.abs(grad[idx]))
        assert gmax > 0
        pick = rng.choice(idx, size=8, replace=False)
        for j in pick:
            h = 1e-6
            tp, tm = theta.copy(), theta.copy()
            tp[j] += h
            tm[j] -= h
            Lp, _ = ws.loss_and_grad(tp, g, psi, b)
            Lm, _ = ws.loss_and_grad(tm, g, psi, b)
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - grad[j]) <= 1e-6 * gmax + 1e-6 * abs(grad[j]), (j, fd, grad[j], gmax)
            checked += 1
    assert checked == 8 * 5
    # rows 63 of the W^l feed only the constant channel: exactly zero gradient
    for W in Ws:
        assert np.all(grad[W[C - 1]] == 0.0)


def test_identity_network_is_jacobi_guess(oracle_mod):
    m, g, psi, b = small_case(oracle_mod)

    def first(W0):
        W0[0, 0], W0[1, 0], W0[2, 1], W0[3, 1] = 1.0, -1.0, 1.0, -1.0

    theta = set_identity_tail(np.zeros(ws.NPARAM), first)
    x0 = ws.predict(theta, g, psi, b)
    np.testing.assert_allclose(x0, b / kinetic_diag(m), rtol=1e-13, atol=0)


@pytest.mark.parametrize("dim,N,mu", [(2, 6, 1.0), (3, 4, 2.0)])
def test_aggregation_is_magnetic_jacobi(oracle_mod, dim, N, mu):
    """Layer 0 taking the aggregated pair (S b^) gives x0 = (S b) / K_ii with
    S b = b - (K b) / K_ii, K from the C oracle (Eq. (10))."""
    m, g, psi, b = small_case(oracle_mod, dim, N, mu)

    def first(W0):
        W0[0, C], W0[1, C], W0[2, C + 1], W0[3, C + 1] = 1.0, -1.0, 1.0, -1.0

    theta = set_identity_tail(np.zeros(ws.NPARAM), first)
    kd = kinetic_diag(m)
    expect = (b - m.kinetic(b) / kd) / kd
    np.testing.assert_allclose(ws.predict(theta, g, psi, b), expect, rtol=0, atol=1e-12 * np.max(np.abs(expect)))


def test_aggregation_averages_constants_without_field(oracle_mod):
    m = oracle_mod.Mesh(3, 5, 0.0)
    g = ws.Graph(m)
    h = np.zeros((m.n, C))
    h[:, 0] = 2.5
    h[:, 1] = -1.0
    s = g.aggregate(h)
    np.testing.assert_allclose(s[:, 0], 2.5, rtol=1e-14)
    np.testing.assert_allclose(s[:, 1], -1.0, rtol=1e-14)


def test_aggregation_adjoint(oracle_mod):
    m, g, psi, b = small_case(oracle_mod, 3, 4, 1.3)
    rng = gi.rng(4)
    u = rng.standard_normal((m.n, C))
    v = rng.standard_normal((m.n, C))
    assert abs(np.sum(v * g.aggregate(u)) - np.sum(g.aggregate_adjoint(v) * u)) <= 1e-12 * np.sum(np.abs(u)) * np.sum(np.abs(v)) / m.n


def test_loss_at_solution_and_zero(oracle_mod):
    m, g, psi, b = small_case(oracle_mod)
    bhat = b / g.dnorm(b)
    assert abs(ws.loss(g, psi, bhat, np.zeros(m.n, np.complex128)) - 1.0) < 1e-14
    xs = m.dense_solve(psi, bhat)
    assert ws.loss(g, psi, bhat, xs) < 1e-20


def test_scale_equivariance(oracle_mod):
    m, g, psi, b = small_case(oracle_mod)
    theta = gi.warmstart_init(2).astype(np.float64)
    x1 = ws.predict(theta, g, psi, b)
    x2 = ws.predict(theta, g, psi, 7.25 * b)
    np.testing.assert_allclose(x2, 7.25 * x1, rtol=1e-12)


def test_adam_constant_gradient_closed_form():
    """Under a constant gradient the bias-corrected moments equal g and g^2
    exactly, so every step moves by -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 0.01, 1e-8
    expect = th.copy()
    for t in range(1, 6):
        th, m, v = ws.adam_step(th, g, m, v, t, lr, eps=eps)
        expect = expect - lr * g / (np.abs(g) + eps)
        np.testing.assert_allclose(th, expect, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- the hint
@pytest.mark.parametrize("dim,N", [(2, 6), (3, 4)])
def test_gradient_central_differences_with_hint(oracle_mod, dim, N):
    """With a hint the network sees two more input channels (the normalised hint)
    and the residual the hint's multiple leaves; the backward pass still matches
    central differences, including the weights reading the hint channels."""
    m, g, psi, b = small_case(oracle_mod, dim, N)
    hint = gi.complex_normal(m.n, 21)
    theta = gi.warmstart_init(6).astype(np.float64)
    L, grad = ws.loss_and_grad(theta, g, psi, b, hint)
    Ws, _ = ws.split(np.arange(ws.NPARAM))
    rng = gi.rng(10)
    # layer 0's columns 6, 7 read the hint pair (and 64 + 6, 64 + 7 its aggregate)
    cols = [Ws[0][:, 6], Ws[0][:, 7], Ws[0][:, C + 6], Ws[0][:, C + 7]]
    idx = np.concatenate([c[:C - 1] for c in cols])
    gmax = np.max(np.abs(grad))
    assert np.max(np.abs(grad[idx])) > 1e-3 * gmax
    for j in rng.choice(idx, size=12, replace=False):
        h = 1e-6
        tp, tm = theta.copy(), theta.copy()
        tp[j] += h
        tm[j] -= h
        fd = (ws.loss_and_grad(tp, g, psi, b, hint)[0] - ws.loss_and_grad(tm, g, psi, b, hint)[0]) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-6 * gmax + 1e-6 * abs(grad[j]), (j, fd, grad[j])
    # without the hint channels' signal (a hint of zero) those weights get no gradient
    _, g0 = ws.loss_and_grad(theta, g, psi, b, np.zeros(m.n, complex))
    assert np.all(g0[idx] == 0.0)


def test_hint_multiple_is_minimal_residual(oracle_mod):
    """With the network's head at zero the guess is alpha a, and alpha minimises
    ||b - J (t a)||_D over t (checked against a fine scan); a hint that solves the
    system exactly is returned as it is (alpha = 1, zero residual)."""
    m, g, psi, b = small_case(oracle_mod)
    theta = np.zeros(ws.NPARAM)
    a = gi.complex_normal(m.n, 22)
    x0 = ws.predict(theta, g, psi, b, a)
    alpha = x0[0] / a[0]
    np.testing.assert_allclose(x0, alpha * a, rtol=1e-12, atol=0)
    assert abs(alpha.imag) <= 1e-14 * abs(alpha)
    res = lambda t: g.dnorm(b - m.jacobian(psi, t * a))  # noqa: E731
    ts = alpha.real + np.linspace(-1e-3, 1e-3, 41) * (1 + abs(alpha.real))
    assert res(alpha.real) <= min(res(t) for t in ts) * (1 + 1e-12)
    # the exact solution as hint
    xs = m.dense_solve(psi, b)
    x0 = ws.predict(theta, g, psi, b, xs)
    assert g.dnorm(b - m.jacobian(psi, x0)) <= 1e-9 * g.dnorm(b)
    # no hint is the original form; a zero hint changes nothing either
    theta = gi.warmstart_init(7).astype(np.float64)
    np.testing.assert_array_equal(ws.predict(theta, g, psi, b, np.zeros(m.n, complex)),
                                  ws.predict(theta, g, psi, b))
