"""The oracle's assembly on general simplicial meshes (glref_mesh_create_simplicial;
the paper's Delaunay meshes of its six test domains, Sec. 4), pinned to:

* the tetrahedron coefficients in closed form (|e_kl| cot(theta_kl) / 6): the
  corollary's identity |S| |u|^2 = sum_e alpha_e <e, u>^2 on random tetrahedra,
  and the linear-system solution of the structured path on well-shaped ones;
* the structured assembly: the Kuhn lattice fed in as a list of simplices gives
  K-hat bit for bit in 2D and to 4e-16 of its largest entry in 3D (the closed
  form against the linear system), the control volumes h^d 2^-b to rounding (2D;
  3D at interior nodes: at the cube's boundary the Kuhn split is not well-centred
  and the circumcentric dual differs from the lattice Voronoi cell);
* the Voronoi regions of an equilateral triangulation: regular hexagons of area
  (sqrt 3 / 2) h^2 at interior nodes (a well-centred Delaunay mesh, where the dual
  of the coefficients is exactly the Voronoi diagram);
* the control volumes tile the mesh: sum |V| = sum of the simplex volumes, every
  |V| > 0 on the Delaunay meshes of the six domains;
* K-hat Hermitian and, without field, K-hat 1 = 0 (the coefficients sum to the
  diagonal);
* the R_1-preconditioned MINRES iteration counts stay flat as the disc's mesh is
  refined (Sec. 4, Fig. 2).
"""
import itertools
import math

import numpy as np
import pytest

import gl_inputs as gi


def kuhn_simplices(dim, N):
    nid = lambda i, j, k: i + N * (j + N * k)  # noqa: E731
    out = []
    if dim == 2:
        for j in range(N - 1):
            for i in range(N - 1):
                out.append([nid(i, j, 0), nid(i + 1, j, 0), nid(i + 1, j + 1, 0)])
                out.append([nid(i, j, 0), nid(i + 1, j + 1, 0), nid(i, j + 1, 0)])
    else:
        for k in range(N - 1):
            for j in range(N - 1):
                for i in range(N - 1):
                    for perm in itertools.permutations(range(3)):
                        c = [i, j, k]
                        v = [nid(*c)]
                        for a in perm:
                            c[a] += 1
                            v.append(nid(*c))
                        out.append(v)
    return np.array(out)


def test_dihedral_coefficients(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(20):
        p = rng.standard_normal((4, 3))
        a = oracle_mod.simplex_alpha(3, p, method="dihedral")
        vol = abs(np.linalg.det(p[1:] - p[0])) / 6
        edges = [(i, j) for i in range(4) for j in range(i + 1, 4)]
        S = sum(a[k] * np.outer(p[j] - p[i], p[j] - p[i]) for k, (i, j) in enumerate(edges))
        assert np.abs(S - vol * np.eye(3)).max() <= 1e-12 * max(1.0, vol)
    # a well-shaped tetrahedron: the structured path's linear system agrees
    p = np.array([[0.0, 0, 0], [1.0, 0.1, 0], [0.2, 1.0, 0.1], [0.1, 0.2, 1.1]])
    np.testing.assert_allclose(oracle_mod.simplex_alpha(3, p, method="dihedral"),
                               oracle_mod.simplex_alpha(3, p, method="linsys"), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("dim,N", [(2, 9), (3, 6)])
def test_kuhn_lattice_as_simplices(oracle_mod, dim, N):
    bh = (0.0, 0.0, 1.0) if dim == 2 else tuple(np.array([0.3, 0.4, 0.866]) / np.linalg.norm([0.3, 0.4, 0.866]))
    ms = oracle_mod.Mesh(dim, N, 1.3, bh, edge=2.0)
    mg = oracle_mod.Mesh.from_simplices(dim, ms.nodes(), kuhn_simplices(dim, N), 1.3, bhat=bh)
    rp, ci, v = ms.khat_csr()
    rp2, ci2, v2 = mg.khat_csr()
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    if dim == 2:
        assert np.array_equal(v, v2)  # the same cotangent formula
    else:
        # the dihedral closed form against the structured path's linear system
        assert np.abs(v - v2).max() <= 4e-16 * np.abs(v).max()
    vs, vg = ms.volumes(), mg.volumes()
    assert vg.sum() == pytest.approx(2.0 ** dim, rel=1e-14)
    if dim == 2:
        np.testing.assert_allclose(vg, vs, rtol=4e-16 * 4, atol=0)
    else:
        x = ms.nodes()
        interior = np.all(np.abs(x) < 1.0 - 1e-9, axis=1)
        np.testing.assert_allclose(vg[interior], vs[interior], rtol=4e-15, atol=0)


def test_equilateral_voronoi_hexagons(oracle_mod):
    h = 0.5
    pts = [(i * h + 0.5 * h * (j % 2), j * h * math.sqrt(3) / 2) for j in range(12) for i in range(12)]
    pts = np.array(pts)
    from scipy.spatial import Delaunay

    tri = Delaunay(pts)
    m = oracle_mod.Mesh.from_simplices(2, pts, tri.simplices, 0.7)
    vol = m.volumes()
    # interior nodes: all six lattice neighbours present
    x = pts
    interior = [(i, j) for j in range(2, 10) for i in range(2, 10)]
    ids = [j * 12 + i for i, j in interior]
    np.testing.assert_allclose(vol[ids], math.sqrt(3) / 2 * h * h, rtol=1e-13)
    assert len(x) == 144


@pytest.mark.parametrize("name,h", [("tri", 0.6), ("sq", 0.6), ("circ", 0.6), ("tet", 1.2), ("cube", 1.0),
                                    ("ball", 1.2)])
def test_domain_meshes_volumes_and_khat(oracle_mod, name, h):
    dim, x, s = gi.delaunay_domain(name, h, seed=3)
    m = oracle_mod.Mesh.from_simplices(dim, x, s, 1.0)
    vol = m.volumes()
    e = x[s[:, 1:], :dim] - x[s[:, :1], :dim]
    meshvol = np.abs(np.linalg.det(e)).sum() / math.factorial(dim)
    assert vol.sum() == pytest.approx(meshvol, rel=1e-12)
    assert vol.min() > 0
    Kd = m.khat_dense()
    assert np.abs(Kd - Kd.conj().T).max() <= 1e-14 * np.abs(Kd).max()
    m0 = oracle_mod.Mesh.from_simplices(dim, x, s, 0.0)
    K0 = m0.khat_dense()
    assert np.abs(K0.imag).max() == 0.0
    assert np.abs(K0 @ np.ones(m0.n)).max() <= 1e-13 * np.abs(K0).max()
    assert np.linalg.eigvalsh(K0).min() >= -1e-12 * np.abs(K0).max()


def test_disc_iterations_flat(oracle_mod):
    counts = []
    for h in (0.5, 0.35, 0.25):
        dim, x, s = gi.delaunay_domain("circ", h, seed=2)
        m = oracle_mod.Mesh.from_simplices(dim, x, s, 1.0)
        psi = np.ones(m.n, complex)
        b = gi.complex_normal(m.n, 5)
        _, info = m.solve(psi, b, max_coarse=64, tol=1e-10)
        assert info.converged and info.true_relres <= 1e-10
        counts.append(info.iters)
    assert max(counts) - min(counts) <= 4, counts
