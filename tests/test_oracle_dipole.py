"""Pins of the dipole potential A_d (Sec. 4): the edge phases against an
independent adaptive quadrature, Stokes' theorem on the lattice faces against
the flux of the dipole field B = (3 (m . r^) r^ - m) / |r|^3, the zero-field
limit, and the shape of Fig. 3's "cube in A_d" panel."""
import os

import numpy as np
import pytest
import scipy.integrate as si

X0_3D, X0_2D, MOM = (0.0, 0.0, 6.0), (0.0, 0.0, 1.0), (0.0, 0.0, 1.0)
L3 = 10.0 / np.sqrt(3.0)  # cube of circumradius 5
L2 = 10.0 / np.sqrt(2.0)  # square of circumradius 5


def a_dipole(x, x0, m):
    r = np.asarray(x) - np.asarray(x0)
    return np.cross(m, r) / np.linalg.norm(r) ** 3


def b_dipole(x, x0, m):
    r = np.asarray(x) - np.asarray(x0)
    d = np.linalg.norm(r)
    rh = r / d
    return (3.0 * np.dot(m, rh) * rh - np.asarray(m)) / d ** 3


@pytest.mark.parametrize("dim,N,L,x0", [(3, 6, L3, X0_3D), (2, 9, L2, X0_2D)])
def test_edge_phases_against_adaptive_quadrature(oracle_mod, dim, N, L, x0):
    m = oracle_mod.Mesh(dim, N, 1.0, edge=L, dipole=(x0, MOM))
    x = m.nodes()
    ej, ek, _, theta = m.edges()
    g = np.random.default_rng(3)
    for e in g.choice(len(ej), 40, replace=False):
        xa, xb = x[ej[e]], x[ek[e]]
        d = xb - xa
        ref, _ = si.quad(lambda t: float(np.dot(a_dipole(xa + t * d, x0, MOM), d)), 0.0, 1.0, epsabs=1e-15,
                         epsrel=1e-13)
        assert abs(m.edge_integral1(xa, xb) - ref) <= 1e-12 * max(abs(ref), 1e-3 * np.linalg.norm(d) / 9.0)
        assert theta[e] == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_stokes_on_lattice_faces(oracle_mod):
    """The phases around a face of the cube lattice add up to the flux of
    B = curl A_d through it (a wrong sign, a wrong cross product or a dropped
    1/|r|^3 factor breaks it)."""
    N = 5
    m = oracle_mod.Mesh(3, N, 1.0, edge=L3, dipole=(X0_3D, MOM))
    h = L3 / (N - 1)
    lo = -L3 / 2
    g = np.random.default_rng(4)
    for _ in range(6):
        i, j, k = g.integers(0, N - 1, 3)
        axis = int(g.integers(0, 3))
        c = np.array([lo + i * h, lo + j * h, lo + k * h])
        u, v = [a for a in range(3) if a != axis]
        eu, ev = np.eye(3)[u] * h, np.eye(3)[v] * h
        loop = [c, c + eu, c + eu + ev, c + ev]
        circ = sum(m.edge_integral1(loop[q], loop[(q + 1) % 4]) for q in range(4))
        n = np.cross(eu, ev) / h ** 2
        flux, _ = si.dblquad(lambda s, t: float(np.dot(b_dipole(c + t * eu + s * ev, X0_3D, MOM), n)) * h * h,
                             0.0, 1.0, 0.0, 1.0, epsabs=1e-14, epsrel=1e-12)
        assert circ == pytest.approx(flux, rel=1e-10, abs=1e-14)


def test_zero_field_limit(oracle_mod):
    """At mu = 0 the dipole mesh is the field-free mesh: same K-hat bit for bit."""
    a = oracle_mod.Mesh(3, 6, 0.0, edge=L3, dipole=(X0_3D, MOM))
    b = oracle_mod.Mesh(3, 6, 0.0, edge=L3)
    for u, w in zip(a.khat_csr(), b.khat_csr()):
        np.testing.assert_array_equal(u, w)


def read_fig3_ad():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig3_cube_ad_iterations.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, *vals = line.split()
                rows[name] = [int(x) for x in vals]
    return rows


def test_fig3_cube_in_dipole_shape(oracle_mod):
    """Fig. 3, cube in A_d (psi = 1, tol 1e-11): the unpreconditioned counts grow
    with the mesh, R_1's stay flat at about the paper's (29-32 from 2n = 6750 on),
    R_inf's are flat and lowest."""
    fig = read_fig3_ad()
    its = {"unprec": [], "R1": [], "Rinf": []}
    for N in (10, 15):
        m = oracle_mod.Mesh(3, N, 1.0, edge=L3, dipole=(X0_3D, MOM))
        assert 2 * m.n in fig["dims"]
        one = np.ones(m.n, complex)
        its["unprec"].append(m.solve(one, one, tol=1e-11, cycles=0, maxit=3000)[1].iters)
        its["R1"].append(m.solve(one, one, tol=1e-11, max_coarse=64)[1].iters)
        its["Rinf"].append(m.solve(one, one, tol=1e-11, max_coarse=64, cycles=oracle_mod.CYCLES_INF)[1].iters)
    assert its["unprec"][1] > 1.3 * its["unprec"][0]
    assert abs(its["R1"][1] - its["R1"][0]) <= 2 and abs(its["R1"][1] - fig["R1"][2]) <= 4
    assert abs(its["Rinf"][1] - its["Rinf"][0]) <= 1 and max(its["Rinf"]) < min(its["R1"])


@pytest.mark.parametrize("dim,N,L,x0", [(3, 6, L3, X0_3D), (2, 9, L2, X0_2D)])
def test_dmu_on_dipole_meshes(oracle_mod, dim, N, L, x0):
    """d GL / d mu on a dipole mesh (phase per unit mu from the quadrature) against
    the central difference of two independently assembled meshes."""
    mu, eps = 0.9, 1e-5
    psi = np.ones(N ** dim, complex) + 0.2 * np.exp(1j * np.arange(N ** dim))
    d = oracle_mod.Mesh(dim, N, mu, edge=L, dipole=(x0, MOM)).residual_dmu(psi)
    fd = (oracle_mod.Mesh(dim, N, mu + eps, edge=L, dipole=(x0, MOM)).residual(psi)
          - oracle_mod.Mesh(dim, N, mu - eps, edge=L, dipole=(x0, MOM)).residual(psi)) / (2 * eps)
    assert np.linalg.norm(d - fd) <= 1e-7 * np.linalg.norm(d)
