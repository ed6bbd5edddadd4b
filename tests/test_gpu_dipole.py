"""The dipole potential A_d on the GPU (Sec. 4): assembly against the oracle,
the stored stencil chosen automatically (the lattice tables do not hold for a
field that varies along the edges), and Fig. 3's cube-in-A_d panel."""
import os

import numpy as np
import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
MOM = (0.0, 0.0, 1.0)
L3, X3 = 10.0 / np.sqrt(3.0), (0.0, 0.0, 6.0)
L2, X2 = 10.0 / np.sqrt(2.0), (0.0, 0.0, 1.0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim,N,L,x0", [(3, 9, L3, X3), (2, 17, L2, X2)])
def test_dipole_mesh_matches_oracle(oracle_mod, dim, N, L, x0):
    om = oracle_mod.Mesh(dim, N, 0.8, edge=L, dipole=(x0, MOM))
    m = gl.gl_mesh_create_dipole(dim, N, L, 0.8, x0, MOM)
    try:
        rp, ci, v = gl.gl_mesh_khat(m)
        orp, oci, ov = om.khat_csr()
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(ci, oci)
        np.testing.assert_allclose(v, ov, rtol=0, atol=1e-13 * np.abs(ov).max())
        psi = gi.disk(om.n, 5)
        d = torch.zeros(om.n, dtype=torch.complex128, device=DEV)
        gl.gl_residual_dmu(m, dev(psi), d)
        od = om.residual_dmu(psi)
        np.testing.assert_allclose(d.cpu().numpy(), od, rtol=0, atol=1e-12 * np.abs(od).max())
        assert gl.gl_energy(m, dev(psi)) == pytest.approx(om.energy(psi), rel=1e-12)
        # mu scales A_d: the mesh moved to mu = 1.3 equals the oracle's at 1.3
        gl.gl_mesh_set_mu(m, 1.3)
        om2 = oracle_mod.Mesh(dim, N, 1.3, edge=L, dipole=(x0, MOM))
        np.testing.assert_allclose(gl.gl_mesh_khat(m)[2], om2.khat_csr()[2], rtol=0, atol=1e-13 * np.abs(ov).max())
    finally:
        gl.gl_mesh_destroy(m)


def test_dipole_uses_the_stored_stencil(oracle_mod):
    N = 16
    om = oracle_mod.Mesh(3, N, 1.0, edge=L3, dipole=(X3, MOM))
    m = gl.gl_mesh_create_dipole(3, N, L3, 1.0, X3, MOM)
    try:
        psi, b = gi.psi_noisy_one(om.n, 6), gi.complex_normal(om.n, 7)
        x = torch.zeros(om.n, dtype=torch.complex128, device=DEV)
        st, info = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x,
                                        gl.options(max_coarse=64, precision=gl.GL_MIXED_PRECOND))
        assert st == 0 and info.converged
        assert info.lattice_stencil == 0 and info.df_jacobian == 0
        xo, _ = om.solve(psi, b, max_coarse=64, tol=1e-12)
        assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-7 * np.linalg.norm(xo)
    finally:
        gl.gl_mesh_destroy(m)
    with pytest.raises(gl.GLError):
        gl.gl_mesh_create_dipole(3, 8, L3, 1.0, (0.0, 0.0, 1.0), MOM)  # inside the cube


def read_fig3_ad():
    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig3_cube_ad_iterations.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, *vals = line.split()
                rows[name] = [int(x) for x in vals]
    return rows


def test_fig3_cube_in_dipole_on_gpu(oracle_mod):
    """Fig. 3, cube in A_d (psi = 1, phi_0 = 0, tol 1e-11) at the paper's sizes
    2n = 2000 ... 85750: R_1 counts stay in a band independent of the size (the
    paper's run 22-32; here 25-35, the lowest where the hierarchy gains a
    level), R_inf counts are flat and below R_1's, and the oracle agrees within
    one where it runs in seconds."""
    fig = read_fig3_ad()
    r1, rinf = [], []
    for N, dims in zip((10, 15, 20, 25, 30, 35), fig["dims"][1:]):
        assert 2 * N ** 3 == dims
        m = gl.gl_mesh_create_dipole(3, N, L3, 1.0, X3, MOM)
        try:
            one = torch.ones(N ** 3, dtype=torch.complex128, device=DEV)
            its = []
            for k in (1, gl.GL_CYCLES_INF):
                x = torch.zeros_like(one)
                st, info = gl.gl_jacobian_solve(m, one, None, one, x, gl.options(tol=1e-11, cycles=k, max_coarse=64))
                assert st == 0 and info.converged
                its.append(info.iters)
            r1.append(its[0])
            rinf.append(its[1])
            if N <= 15:
                om = oracle_mod.Mesh(3, N, 1.0, edge=L3, dipole=(X3, MOM))
                o1 = np.ones(om.n, complex)
                assert abs(om.solve(o1, o1, tol=1e-11, max_coarse=64)[1].iters - its[0]) <= 1
        finally:
            gl.gl_mesh_destroy(m)
    print(f"Fig. 3 cube in A_d: R_1 {r1} (paper {fig['R1'][1:7]}); R_inf {rinf} (paper {fig['Rinf'][1:7]})")
    assert 20 <= min(r1) and max(r1) <= 40 and max(rinf) - min(rinf) <= 2
    assert all(a < b for a, b in zip(rinf, r1))
    assert abs(np.median(r1) - np.median(fig["R1"][2:7])) <= 4
