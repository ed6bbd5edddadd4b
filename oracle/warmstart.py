"""FP64 oracle of the learned warm start for the Jacobian solve.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports this module.

The paper has no learned component; the network below is the project's own
definition, stated here in full so that the CUDA kernels can be checked against
it.  It predicts the initial guess of the Newton-system solve J(psi) x = b
(Sec. 3, Eq. (16)) as

    x0 = ||b||_D * ( y(psi, b / ||b||_D) / K_ii ),       ||b||_D^2 = sum_i |V_i| |b_i|^2,

which is scale-equivariant because the solve is linear in b.  K_ii is the
diagonal of K = D^-1 K-hat (Eq. (10), Remark 2.3), so the identity network gives
the Jacobi guess b / diag(K).

With a hint a (a vector the caller expects to resemble the solution, e.g. the
same Newton step's correction at the previous field strength of a
continuation), the guess is that vector's best multiple plus the network's
correction for what it leaves:

    alpha = <J a, b>_R / <J a, J a>_R  (0 when J a = 0),   r = b - alpha J a,
    x0 = alpha a + ||r||_D * ( y(psi, r / ||r||_D, a / ||a||_D) / K_ii ),

where alpha minimises ||b - J (alpha a)||_D; without a hint a = 0, alpha = 0 and
r = b (the form above).

Network (4 layers of 64 real channels = 32 complex channel pairs):

* input h^0_i = [Re r^_i, Im r^_i, Re psi_i, Im psi_i, |psi_i|^2, 0, Re a^_i,
  Im a^_i, 0, ..., 0, 1] with r^ = r / ||r||_D and a^ = a / ||a||_D (zeros
  without a hint; the hint is the complex channel pair (6, 7); channel 63 is the
  constant 1 in every layer; it carries the biases).
* twisted aggregation, acting on each complex channel pair (2c, 2c + 1):
      (S u)_i = sum_{k != i} w_ik u_k,    w_ik = -K-hat_ik / K-hat_ii,
  i.e. S = I - diag(K-hat)^-1 K-hat, the magnetic Jacobi operator: the edge
  coefficients alpha_ik and phases exp(-i theta_ik) of Eq. (10), normalised per row.
* layer l = 0..3:  a^l_i = [h^l_i ; (S h^l)_i]  (128),  z^l_i = W^l a^l_i  (64),
  h^{l+1}_i = relu(z^l_i) with channel 63 reset to 1.
* head: y_i = U h^4_i  (2 -> one complex number per node).

Parameters, one flat float vector: W^0..W^3 (64 x 128 each, row-major: out x in),
then U (2 x 64).  Rows 63 of the W^l only feed the discarded channel 63.

Training loss of one sample (psi, b[, a]):  L = ||r^ - J(psi) x^||_D^2  with
x^ = y / K_ii, which is ||b - J x0||_D^2 / ||r||_D^2 -- the squared true-Jacobian
residual of the predicted guess relative to what the hint leaves (without a
hint: to ||b||_D, the quantity the zero-guess fallback tests).  For a triple (psi, b, x*) with J x* = b it equals
||J (x^ - x*/||b||_D)||_D^2.

J(psi) phi = K phi + (-1 + 2|psi|^2) phi + psi^2 conj(phi) is the Jacobian of
Eq. (16), taken from the plain-C oracle (``glref_jacobian_apply``).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

C = 64          # channels per layer
CIN = 2 * C     # [h, S h]
LAYERS = 4
NPARAM = LAYERS * C * CIN + 2 * C


def split(theta):
    """Views of the flat parameter vector: ([W^0..W^3], U)."""
    theta = np.asarray(theta)
    Ws = [theta[l * C * CIN:(l + 1) * C * CIN].reshape(C, CIN) for l in range(LAYERS)]
    U = theta[LAYERS * C * CIN:].reshape(2, C)
    return Ws, U


class Graph:
    """Per-mesh data the network needs: the twisted aggregation S (complex CSR),
    K_ii = K-hat_ii / |V_i|, |V_i|, and the oracle mesh for J."""

    def __init__(self, mesh):
        rp, ci, v = mesh.khat_csr()
        n = mesh.n
        Kh = sp.csr_matrix((v, ci, rp), shape=(n, n))
        d = np.real(Kh.diagonal())
        off = Kh - sp.diags(Kh.diagonal())
        self.S = sp.csr_matrix(-sp.diags(1.0 / d) @ off)   # w_ik = -K-hat_ik / K-hat_ii
        self.SH = sp.csr_matrix(self.S.conj().T)            # Euclidean adjoint on complex pairs
        self.vol = mesh.volumes()
        self.kdiag = d / self.vol                           # K_ii
        self.mesh = mesh
        self.n = n

    def aggregate(self, h):
        """S applied to every complex channel pair of h (n x 64 real)."""
        z = h[:, 0::2] + 1j * h[:, 1::2]
        s = self.S @ z
        out = np.empty_like(h)
        out[:, 0::2], out[:, 1::2] = s.real, s.imag
        return out

    def aggregate_adjoint(self, g):
        z = g[:, 0::2] + 1j * g[:, 1::2]
        s = self.SH @ z
        out = np.empty_like(g)
        out[:, 0::2], out[:, 1::2] = s.real, s.imag
        return out

    def dnorm(self, x) -> float:
        return float(np.sqrt(np.sum(self.vol * np.abs(x) ** 2)))


def features(g: Graph, psi, bhat, ahat=None):
    h = np.zeros((g.n, C))
    h[:, 0], h[:, 1] = bhat.real, bhat.imag
    h[:, 2], h[:, 3] = psi.real, psi.imag
    h[:, 4] = np.abs(psi) ** 2
    if ahat is not None:
        h[:, 6], h[:, 7] = ahat.real, ahat.imag
    h[:, C - 1] = 1.0
    return h


def inner_r(g: Graph, x, y) -> float:
    return float(np.sum(g.vol * np.real(np.conj(x) * y)))


def hint_split(g: Graph, psi, b, hint):
    """(alpha, r, a^): the hint's minimal-residual multiple, the residual it leaves,
    and the normalised hint (alpha = 0, r = b, a^ = None without a hint)."""
    if hint is None:
        return 0.0, b, None
    an = g.dnorm(hint)
    if an == 0:
        return 0.0, b, np.zeros(g.n, complex)
    q = g.mesh.jacobian(psi, hint)
    qq = inner_r(g, q, q)
    alpha = inner_r(g, q, b) / qq if qq > 0 else 0.0
    return alpha, b - alpha * q, hint / an


def forward(theta, g: Graph, psi, b, hint=None):
    """Returns (xhat, cache): xhat = y / K_ii for r^ = r / ||r||_D, r the residual
    the hint's multiple leaves (r = b without a hint)."""
    Ws, U = split(theta)
    alpha, r, ahat = hint_split(g, psi, b, hint)
    bn = g.dnorm(r)
    bhat = r / bn
    h = features(g, psi, bhat, ahat)
    hs, As = [h], []
    for W in Ws:
        a = np.concatenate([h, g.aggregate(h)], axis=1)
        z = a @ W.T
        h = np.maximum(z, 0.0)
        h[:, C - 1] = 1.0
        As.append(a)
        hs.append(h)
    y = hs[-1] @ U.T
    xhat = (y[:, 0] + 1j * y[:, 1]) / g.kdiag
    return xhat, dict(bn=bn, bhat=bhat, hs=hs, As=As, alpha=alpha)


def predict(theta, g: Graph, psi, b, hint=None):
    """x0 = alpha a + ||r||_D * xhat (x0 = ||b||_D * xhat without a hint)."""
    xhat, cache = forward(theta, g, psi, b, hint)
    x0 = cache["bn"] * xhat
    if hint is not None:
        x0 = x0 + cache["alpha"] * hint
    return x0


def loss(g: Graph, psi, bhat, xhat) -> float:
    r = bhat - g.mesh.jacobian(psi, xhat)
    return float(np.sum(g.vol * np.abs(r) ** 2))


def loss_and_grad(theta, g: Graph, psi, b, hint=None):
    """L and dL/dtheta (flat, same layout as theta) for one sample."""
    Ws, U = split(theta)
    xhat, cache = forward(theta, g, psi, b, hint)
    bhat, hs, As = cache["bhat"], cache["hs"], cache["As"]
    r = bhat - g.mesh.jacobian(psi, xhat)
    L = float(np.sum(g.vol * np.abs(r) ** 2))
    # J is self-adjoint in <x, y>_R = Re sum |V| conj(x) y (Sec. 3), so the
    # Euclidean gradient of L with respect to (Re x^, Im x^) is -2 |V| J r.
    gx = -2.0 * g.vol * g.mesh.jacobian(psi, r)
    gy = gx / g.kdiag
    dy = np.stack([gy.real, gy.imag], axis=1)          # n x 2
    dU = dy.T @ hs[-1]
    dh = dy @ U
    dWs = [None] * LAYERS
    for l in range(LAYERS - 1, -1, -1):
        dz = dh * (hs[l + 1] > 0.0)
        dz[:, C - 1] = 0.0                              # channel 63 is a constant
        dWs[l] = dz.T @ As[l]
        if l > 0:
            da = dz @ Ws[l]
            dh = da[:, :C] + g.aggregate_adjoint(da[:, C:])
    grad = np.concatenate([w.ravel() for w in dWs] + [dU.ravel()])
    return L, grad


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, Algorithm 1) with bias correction; t >= 1.
    Returns the new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
