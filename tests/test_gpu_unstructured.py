"""General simplicial meshes on the GPU (gl_mesh_create_simplicial): the Delaunay
meshes of the paper's six test domains (Sec. 4: triangle, square, disc,
tetrahedron, cube, ball of circumradius 5), assembled on the device and compared
with the oracle's assembly of the same simplices (K-hat structure bit-exact,
values and control volumes to rounding), the finest-level colouring (the same
round-based smallest-last colours as the oracle's), and solves: every solve
reaches the FP64 true residual 1e-10 measured with the oracle's Jacobian, with
the oracle's iteration count (+-1 in FP64, a few more with the FP32 V-cycle),
in the uniform field and in the
dipole field; the counts stay flat as the disc's mesh is refined (Sec. 4,
Fig. 2)."""
import numpy as np
import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
DOMAINS = [("tri", 0.3), ("sq", 0.3), ("circ", 0.3), ("tet", 0.8), ("cube", 0.7), ("ball", 0.9)]
DIPOLE = {2: ((0.0, 0.0, 1.0), (0.0, 0.0, 1.0)), 3: ((0.0, 0.0, 6.0), (0.0, 0.0, 1.0))}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def true_relres(om, psi, b, x):
    vol = om.volumes()
    r = b - om.jacobian(psi, x)
    return float(np.sqrt(np.sum(vol * np.abs(r) ** 2) / np.sum(vol * np.abs(b) ** 2)))


@pytest.mark.parametrize("field", ["uniform", "dipole"])
@pytest.mark.parametrize("name,h", DOMAINS)
def test_assembly_matches_oracle(oracle_mod, name, h, field):
    dim, x, s = gi.delaunay_domain(name, h, seed=4)
    dip = DIPOLE[dim] if field == "dipole" else None
    om = oracle_mod.Mesh.from_simplices(dim, x, s, 0.8, dipole=dip)
    m = gl.gl_mesh_create_simplicial(dim, x, s, 0.8, dipole=dip)
    try:
        rp, ci, v = gl.gl_mesh_khat(m)
        orp, oci, ov = om.khat_csr()
        assert np.array_equal(rp, orp) and np.array_equal(ci, oci)
        assert np.abs(v - ov).max() <= 1e-13 * np.abs(ov).max()
        vol = torch.zeros(om.n, dtype=torch.float64, device=DEV)
        n, _ = gl.gl_mesh_info(m, vol)
        assert n == om.n
        np.testing.assert_allclose(vol.cpu().numpy(), om.volumes(), rtol=1e-13, atol=0)
    finally:
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("name,h", DOMAINS)
def test_colours_and_solves_match_oracle(oracle_mod, name, h):
    dim, x, s = gi.delaunay_domain(name, h, seed=5)
    om = oracle_mod.Mesh.from_simplices(dim, x, s, 1.0)
    m = gl.gl_mesh_create_simplicial(dim, x, s, 1.0)
    n = om.n
    psi, b = np.ones(n, complex), gi.complex_normal(n, 6)
    try:
        P = oracle_mod.Precond(om, psi, max_coarse=64)
        G = gl.gl_precond_setup(m, dev(psi), gl.options(max_coarse=64))
        try:
            ocol = P.colors(0)
            gcol = gl.gl_precond_level_colors(G, 0)
            assert np.array_equal(gcol, ocol)
            rp, ci, _ = om.khat_csr()
            rows = np.repeat(np.arange(n), np.diff(rp))
            off = ci != rows
            assert not np.any(gcol[rows[off]] == gcol[ci[off]])  # a proper colouring
        finally:
            gl.gl_precond_destroy(G)
        _, oinfo = om.solve(psi, b, max_coarse=64, tol=1e-10)
        # the FP32 V-cycle costs a few iterations (its rounding makes R_1 vary slightly
        # between applications, which MINRES's recurrence assumes away)
        for prec, slack in ((gl.GL_FP64, 1), (gl.GL_MIXED_PRECOND, 6)):
            xg = torch.zeros(n, dtype=torch.complex128, device=DEV)
            st, info = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), xg, gl.options(max_coarse=64, precision=prec))
            assert st == 0 and info.converged, (name, prec, info.as_dict())
            assert true_relres(om, psi, b, xg.cpu().numpy()) <= 1.01e-10
            assert abs(info.iters - oinfo.iters) <= slack, (name, prec, info.iters, oinfo.iters)
            assert info.lattice_stencil == 0 and info.df_jacobian == 0
    finally:
        gl.gl_mesh_destroy(m)


def test_disc_counts_flat_and_bad_input():
    counts = []
    for h in (0.4, 0.2, 0.1, 0.05):
        dim, x, s = gi.delaunay_domain("circ", h, seed=7)
        m = gl.gl_mesh_create_simplicial(dim, x, s, 1.0)
        try:
            n = x.shape[0]
            xg = torch.zeros(n, dtype=torch.complex128, device=DEV)
            st, info = gl.gl_jacobian_solve(m, dev(np.ones(n, complex)), None, dev(gi.complex_normal(n, 8)), xg,
                                            gl.options())
            assert st == 0 and info.converged and info.true_relres <= 1.01e-10
            counts.append(info.iters)
        finally:
            gl.gl_mesh_destroy(m)
    print(f"disc, h = 0.4 ... 0.05 ({[len(gi.delaunay_domain('circ', h, seed=7)[1]) for h in (0.4, 0.2, 0.1, 0.05)]} "
          f"nodes): iterations {counts}")
    assert max(counts) <= 2 * min(counts) + 2, counts
    dim, x, s = gi.delaunay_domain("sq", 1.0, seed=1)
    bad = s.copy()
    bad[0, 0] = x.shape[0]
    with pytest.raises(gl.GLError):
        gl.gl_mesh_create_simplicial(dim, x, bad, 1.0)
    flat = s.copy()
    flat[0, 1] = flat[0, 0]
    with pytest.raises(gl.GLError):
        gl.gl_mesh_create_simplicial(dim, x, flat, 1.0)


SIZES = {"tri": (0.5, 0.25, 0.125), "sq": (0.5, 0.25, 0.125), "circ": (0.5, 0.25, 0.125),
         "tet": (1.0, 0.6, 0.4), "cube": (1.0, 0.6, 0.4), "ball": (1.0, 0.6, 0.4)}


@pytest.mark.parametrize("field", ["A_z", "A_d"])
@pytest.mark.parametrize("name", list(SIZES))
def test_fig2_fig3_counts_on_delaunay_domains(name, field):
    """Figs. 2-3 in the paper's setting on Delaunay meshes of its domains: psi = 1,
    right-hand side 1, phi_0 = 0, tol 1e-11, mu = 1, A_z or A_d (dipole at
    (0,0,1) in 2D, (0,0,6) in 3D), R_1 and R_inf, three refinements.  The counts
    stay bounded as n grows (max <= 2 min + 2; R_inf's do not grow by more than 3,
    and fall on the finer, more regular meshes) and R_inf takes no more
    iterations than R_1.  They are printed."""
    r1, rinf, ns = [], [], []
    for h in SIZES[name]:
        dim, x, s = gi.delaunay_domain(name, h, seed=9)
        dip = DIPOLE[dim] if field == "A_d" else None
        m = gl.gl_mesh_create_simplicial(dim, x, s, 1.0, dipole=dip)
        try:
            n = x.shape[0]
            psi = torch.ones(n, dtype=torch.complex128, device=DEV)
            b = torch.ones(n, dtype=torch.complex128, device=DEV)
            its = []
            for k in (1, gl.GL_CYCLES_INF):
                xg = torch.zeros_like(b)
                st, info = gl.gl_jacobian_solve(m, psi, None, b, xg, gl.options(tol=1e-11, cycles=k, max_coarse=64))
                assert st == 0 and info.converged, (name, field, h, k, info.as_dict())
                its.append(info.iters)
            r1.append(its[0])
            rinf.append(its[1])
            ns.append(2 * n)
        finally:
            gl.gl_mesh_destroy(m)
    print(f"{name} {field}: real dimension {ns}: R_1 {r1}, R_inf {rinf}")
    assert max(r1) <= 2 * min(r1) + 2, r1
    assert max(rinf) <= 2 * min(rinf) + 2 and rinf[-1] <= rinf[0] + 3, rinf
    assert all(a >= b for a, b in zip(r1, rinf)), (r1, rinf)


@pytest.mark.parametrize("precision", [gl.GL_FP64, gl.GL_MIXED_PRECOND])
def test_batch_of_unstructured_meshes(oracle_mod, precision):
    """Meshes of three domains in one batched launch: every instance reaches the
    true residual 1e-10 with the oracle's Jacobian, as its single solve does."""
    cases = [gi.delaunay_domain(name, h, seed=10) for name, h in (("tri", 0.3), ("circ", 0.3), ("tet", 0.8))]
    meshes = [gl.gl_mesh_create_simplicial(dim, x, s, 0.9) for dim, x, s in cases]
    try:
        psis = [dev(gi.psi_noisy_one(x.shape[0], 20 + k)) for k, (_, x, _) in enumerate(cases)]
        bs = [dev(gi.complex_normal(x.shape[0], 30 + k)) for k, (_, x, _) in enumerate(cases)]
        xs = [torch.zeros_like(b) for b in bs]
        opts = gl.options(precision=precision, max_coarse=64)
        st, infos = gl.gl_batch_solve(meshes, psis, bs, xs, opts)
        assert st == 0
        for k, (dim, x, s) in enumerate(cases):
            om = oracle_mod.Mesh.from_simplices(dim, x, s, 0.9)
            assert infos[k].converged
            assert true_relres(om, psis[k].cpu().numpy(), bs[k].cpu().numpy(), xs[k].cpu().numpy()) <= 1.01e-10
            x1 = torch.zeros_like(bs[k])
            st1, info1 = gl.gl_jacobian_solve(meshes[k], psis[k], None, bs[k], x1, opts)
            assert st1 == 0 and abs(info1.iters - infos[k].iters) <= (1 if precision == gl.GL_FP64 else 3)
    finally:
        for m in meshes:
            gl.gl_mesh_destroy(m)
