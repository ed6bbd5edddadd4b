"""Pins of the oracle's discretisation (Section 3 of the paper) against closed
forms, brute force and the paper's identities."""
import itertools
import math

import numpy as np
import pytest

import gl_inputs as gi


def rand_simplex(dim, g):
    while True:
        p = g.standard_normal((dim + 1, dim))
        e = p[1:] - p[0]
        if abs(np.linalg.det(e)) > 0.2:
            return p


def simplex_vol(p):
    e = p[1:] - p[0]
    return abs(np.linalg.det(e)) / math.factorial(len(e))


@pytest.mark.parametrize("dim", [2, 3])
def test_corollary_identity_random_simplices(oracle_mod, dim):
    """Cor. 'simplex': |S| ||u||^2 = sum_edges alpha_ij |<e_ij, u>|^2 for all u in C^d."""
    g = gi.rng(10 + dim)
    for _ in range(25):
        p = rand_simplex(dim, g)
        al = oracle_mod.simplex_alpha(dim, p)
        edges = [(a, b) for a in range(dim + 1) for b in range(a + 1, dim + 1)]
        for _ in range(4):
            u = g.standard_normal(dim) + 1j * g.standard_normal(dim)
            lhs = simplex_vol(p) * np.vdot(u, u).real
            terms = [al[s] * abs(np.dot(p[b] - p[a], u)) ** 2 for s, (a, b) in enumerate(edges)]
            # M alpha = b is solved in FP64; its condition number is ~1e3 for these simplices
            assert abs(lhs - sum(terms)) <= 1e-10 * sum(abs(t) for t in terms)


def test_cotangent_formula_matches_linear_system(oracle_mod):
    """Remark after Cor. 'simplex': for triangles the M alpha = b solution is 1/2 cot(opposite angle)."""
    g = gi.rng(3)
    for _ in range(50):
        p = rand_simplex(2, g)
        a1 = oracle_mod.simplex_alpha(2, p, "linsys")
        a2 = oracle_mod.simplex_alpha(2, p, "cot")
        np.testing.assert_allclose(a1, a2, rtol=1e-11, atol=1e-12)


def test_unique_alpha_kuhn_tet(oracle_mod):
    """The edge-basis lemma makes alpha unique; for a Kuhn tetrahedron of a cube of
    side h it is h/6 on the three axis edges and 0 on the diagonals."""
    h = 0.25
    p = np.array([[0, 0, 0], [h, 0, 0], [h, h, 0], [h, h, h]], float)
    al = oracle_mod.simplex_alpha(3, p)
    # edge order (0,1),(0,2),(0,3),(1,2),(1,3),(2,3): axis edges are (0,1),(1,2),(2,3)
    np.testing.assert_allclose(al, [h / 6, 0, 0, h / 6, 0, h / 6], atol=1e-15)


def test_edges_2d_closed_form(oracle_mod):
    """Right-isosceles triangles: legs get 1/2 per triangle, the hypotenuse 0 (dropped);
    an interior axis edge is in 2 triangles (alpha = 1), a boundary one in 1 (1/2)."""
    N = 9
    m = oracle_mod.Mesh(2, N, 1.3)
    ej, ek, al, th = m.edges()
    assert m.nedges == 2 * N * (N - 1)
    for a, b, v in zip(ej, ek, al):
        ia, ja, ib, jb = a % N, a // N, b % N, b // N
        assert abs(ia - ib) + abs(ja - jb) == 1
        if ja == jb:
            boundary = ja in (0, N - 1)
        else:
            boundary = ia in (0, N - 1)
        assert v == pytest.approx(0.5 if boundary else 1.0, abs=1e-14)
    assert np.all(np.diff(ej.astype(np.int64) * m.n + ek) > 0), "edges must be sorted lexicographically"


def test_edges_3d_count_tets(oracle_mod):
    """3D: alpha_jk = (h/6) x (number of Kuhn tetrahedra that contain edge jk as an
    axis edge), counted by brute force over all cells."""
    N = 5
    h = 1.0 / (N - 1)
    m = oracle_mod.Mesh(3, N, 0.7, gi.WORKLOADS["cube128"][3])
    ej, ek, al, th = m.edges()
    count = {}
    nid = lambda i, j, k: i + N * (j + N * k)
    for i, j, k in itertools.product(range(N - 1), repeat=3):
        for perm in itertools.permutations(range(3)):
            c = [i, j, k]
            prev = nid(*c)
            for ax in perm:
                c[ax] += 1
                cur = nid(*c)
                key = (min(prev, cur), max(prev, cur))
                count[key] = count.get(key, 0) + 1
                prev = cur
    assert m.nedges == len(count) == 3 * N * N * (N - 1)
    for a, b, v in zip(ej, ek, al):
        assert v == pytest.approx(h / 6 * count[(a, b)], rel=1e-12)


@pytest.mark.parametrize("dim,N", [(2, 5), (3, 4)])
def test_control_volumes_brute_force(oracle_mod, dim, N):
    """|V_j| is the measure of the points of the domain nearer to x_j than to any
    other node (the Voronoi region, Sec. 3), estimated on a fine sample grid."""
    m = oracle_mod.Mesh(dim, N, 1.0)
    x = m.nodes()[:, :dim]
    vol = m.volumes()
    assert vol.sum() == pytest.approx(1.0, abs=1e-14)
    M = 64 if dim == 2 else 24  # multiples of 2 (N - 1): sample cells nest in the Voronoi cells
    s = (np.arange(M) + 0.5) / M - 0.5
    pts = np.stack(np.meshgrid(*([s] * dim), indexing="ij"), -1).reshape(-1, dim)
    d = ((pts[:, None, :] - x[None, :, :]) ** 2).sum(-1)
    owner = d.argmin(1)
    est = np.bincount(owner, minlength=m.n) / len(pts)
    np.testing.assert_allclose(vol, est, atol=1e-12)


def test_phase_closed_form_and_quadrature(oracle_mod):
    """theta_jk = integral of A from x_j to x_k; for A = (mu/2) bhat x x this is
    (mu/2) bhat . (x_j x x_k); check against that and a 5-point Gauss-Legendre rule."""
    mu = 1.7
    bh = np.array([0.3, -0.5, 0.8])
    bh /= np.linalg.norm(bh)
    m = oracle_mod.Mesh(3, 4, mu, bh)
    x = m.nodes()
    ej, ek, al, th = m.edges()
    closed = 0.5 * mu * np.einsum("i,ei->e", bh, np.cross(x[ej], x[ek]))
    np.testing.assert_allclose(th, closed, atol=1e-15)
    gx, gw = np.polynomial.legendre.leggauss(5)
    quad = np.zeros(len(ej))
    for t, w in zip(gx, gw):
        pt = x[ej] + 0.5 * (t + 1) * (x[ek] - x[ej])
        A = 0.5 * mu * np.cross(bh, pt)
        quad += 0.5 * w * np.einsum("ei,ei->e", A, x[ek] - x[ej])
    np.testing.assert_allclose(th, quad, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_pure_gauge_null_vector(oracle_mod, dim):
    """With a constant potential A = c (no field), psi_j = exp(i c.x_j) is a pure
    gauge and K psi = 0 exactly; the opposite phase sign is not in the kernel.
    This fixes the sign reading of the link variables (Eq. link variable)."""
    c = np.array([0.9, -1.4, 0.6])
    m = oracle_mod.Mesh(dim, 6, 0.0, (0, 0, 1), c)
    x = m.nodes()
    psi = np.exp(1j * x @ c)
    assert np.abs(m.kinetic(psi)).max() < 1e-11
    assert np.abs(m.kinetic(np.conj(psi))).max() > 1.0


@pytest.mark.parametrize("dim", [2, 3])
def test_gauge_covariance_of_K(oracle_mod, dim):
    """A -> A + grad chi with psi -> exp(i chi) psi (chi = c.x) leaves the physics
    unchanged: K(A + c)(e^{i c.x} psi) = e^{i c.x} K(A) psi."""
    c = np.array([0.4, 1.1, -0.3])
    bh = gi.WORKLOADS["cube128"][3]
    m0 = oracle_mod.Mesh(dim, 6, 2.0, bh)
    m1 = oracle_mod.Mesh(dim, 6, 2.0, bh, c)
    ph = np.exp(1j * m0.nodes() @ c)
    psi = gi.disk(m0.n, 7)
    np.testing.assert_allclose(m1.kinetic(ph * psi), ph * m0.kinetic(psi), atol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_field_is_neumann_laplacian(oracle_mod, dim):
    """A = 0: K-hat is the alpha-weighted graph Laplacian with constant null vector
    (the Neumann Laplacian, Sec. 3 and Eq. lambda0 cont)."""
    m = oracle_mod.Mesh(dim, 6, 0.0)
    K = m.khat_dense()
    assert np.abs(K.imag).max() == 0
    assert np.abs(K @ np.ones(m.n)).max() < 1e-13
    ej, ek, al, th = m.edges()
    L = np.zeros((m.n, m.n))
    for a, b, v in zip(ej, ek, al):
        L[a, a] += v
        L[b, b] += v
        L[a, b] -= v
        L[b, a] -= v
    np.testing.assert_allclose(K.real, L, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_khat_hermitian_psd_and_posdef_identity(oracle_mod, dim):
    """K-hat is Hermitian and positive semidefinite, with
    <psi, K psi>_D = sum_edges alpha |psi_j - U psi_k|^2 (Eq. posdef)."""
    m = oracle_mod.Mesh(dim, 6, 1.5, gi.WORKLOADS["cube128"][3])
    K = m.khat_dense()
    assert np.abs(K - K.conj().T).max() == 0
    assert np.linalg.eigvalsh(K).min() > -1e-12
    ej, ek, al, th = m.edges()
    for seed in range(3):
        psi = gi.complex_normal(m.n, 20 + seed)
        lhs = np.vdot(psi, K @ psi)
        rhs = np.sum(al * np.abs(psi[ej] - np.exp(-1j * th) * psi[ek]) ** 2)
        assert abs(lhs.imag) < 1e-12 * abs(rhs)
        assert lhs.real == pytest.approx(rhs, rel=1e-12)
        # K = D^-1 K-hat is self-adjoint in the discrete inner product (Lemma, Sec. 3)
        phi = gi.complex_normal(m.n, 40 + seed)
        vol = m.volumes()
        a = np.vdot(vol * phi, m.kinetic(psi))
        b = np.vdot(vol * m.kinetic(phi), psi)
        assert abs(a - b) < 1e-12 * abs(a)


def test_smallest_eigenvalue_estimate(oracle_mod):
    """Eq. (smallest lambda): <1, K 1>_D / <1, 1>_D = |Omega|^-1 sum alpha |2 sin(arg U / 2)|^2
    exactly, and it tends to |Omega|^-1 int |A|^2 = mu^2/24 on the unit square/cube
    (Eq. lambda0 cont) as h -> 0."""
    mu = 1.3
    errs = []
    for N in (9, 17, 33, 65):
        m = oracle_mod.Mesh(2, N, mu)
        vol = m.volumes()
        one = np.ones(m.n, complex)
        rq = np.vdot(vol, m.kinetic(one)).real / vol.sum()
        ej, ek, al, th = m.edges()
        assert rq == pytest.approx(np.sum(al * (2 * np.sin(th / 2)) ** 2) / vol.sum(), rel=1e-12)
        errs.append(abs(rq - mu ** 2 / 24))
    assert errs[-1] < 0.02 * mu ** 2 / 24
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    m = oracle_mod.Mesh(3, 33, mu, gi.WORKLOADS["cube128"][3])
    vol = m.volumes()
    rq = np.vdot(vol, m.kinetic(np.ones(m.n, complex))).real
    assert rq == pytest.approx(mu ** 2 / 24, rel=0.05)


@pytest.mark.parametrize("dim", [2, 3])
def test_kinetic_operator_consistent_with_pde(oracle_mod, dim):
    """At interior nodes K psi approximates (-i grad - A)^2 psi; for psi = exp(i k.x)
    and divergence-free A this is |k - A(x)|^2 psi.  The error must fall like h^2,
    which fixes the sign convention of the phases against the PDE (Eq. GL)."""
    k = np.array([1.3, -0.7, 0.4])[:dim]
    mu = 3.0
    bh = np.array([0.0, 0.0, 1.0]) if dim == 2 else np.array(gi.WORKLOADS["cube128"][3])
    errs = []
    for N in ((17, 33, 65) if dim == 2 else (9, 17, 33)):
        m = oracle_mod.Mesh(dim, N, mu, bh)
        x = m.nodes()
        psi = np.exp(1j * x[:, :dim] @ k)
        A = 0.5 * mu * np.cross(bh, x)[:, :dim]
        exact = np.sum((k - A) ** 2, axis=1) * psi
        inner = np.all(np.abs(x[:, :dim]) < 0.5 - 1e-9, axis=1)
        errs.append(np.abs(m.kinetic(psi) - exact)[inner].max())
    rate = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rate > 1.6) and rate[-1] > 1.8, (errs, rate)
