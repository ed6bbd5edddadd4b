"""Parity at the benchmark's full size: the 3D cube with 128^3 nodes, in the
launch configuration bench.py times (a gl_prec set up once in GL_MIXED, solves
from x = 0 at tol 1e-10).  The oracle builds the same mesh; the checks are the
mesh and level-0 aggregation bit for bit, the Jacobian element by element, and
the solutions' true residual measured with the oracle's Jacobian."""
import numpy as np
import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
EPS64 = np.finfo(np.float64).eps


@pytest.fixture(scope="module")
def big(oracle_mod):
    dim, _, mu, bh = gi.WORKLOADS["cube128"]
    N = 128
    om = oracle_mod.Mesh(dim, N, mu, bh)
    gm = gl.gl_mesh_create(dim, N, mu, bh)
    yield om, gm
    gl.gl_mesh_destroy(gm)


def test_mesh_and_khat_full_size(big):
    om, gm = big
    rp, ci, v = gl.gl_mesh_khat(gm)
    orp, oci, ov = om.khat_csr()
    assert len(ov) == 14_581_760
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(ci, oci)
    assert np.abs(v - ov).max() <= 1e-13 * np.abs(ov).max()


def test_jacobian_full_size(big):
    om, gm = big
    n = om.n
    psi, phi = gi.disk(n, 4), gi.complex_normal(n, 5)
    y = torch.empty(n, dtype=torch.complex128, device=DEV)
    gl.gl_jacobian_apply(gm, torch.from_numpy(psi).to(DEV), torch.from_numpy(phi).to(DEV), y)
    ref = om.jacobian(psi, phi)
    rp, ci, v = om.khat_csr()
    rowabs = np.add.reduceat(np.abs(v) * np.abs(phi)[ci], rp[:-1]) / om.volumes()
    scale = rowabs + (1 + 3 * np.abs(psi) ** 2) * np.abs(phi)
    torch.cuda.synchronize()
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 64 * EPS64 * scale)


def test_level0_aggregation_full_size(big, oracle_mod):
    om, gm = big
    psi = torch.ones(om.n, dtype=torch.complex128, device=DEV)
    G = gl.gl_precond_setup(gm, psi, gl.options(precision=gl.GL_MIXED))
    try:
        rp, ci, _ = om.khat_csr()
        nagg, agg = oracle_mod.aggregate(rp, ci)
        np.testing.assert_array_equal(gl.gl_precond_level_aggregates(G, 0), agg)
        assert gl.gl_precond_level_info(G, 1)["n"] == nagg
        # the level-1 colouring follows from the level-1 pattern by the round-based
        # smallest-last rule (the default, on the device), and on request by the
        # one-at-a-time smallest-last rule (host) and by Jones-Plassmann
        lrp, lci, _ = gl.gl_precond_level_matrix(G, 1)
        npsl, colpsl, levels = oracle_mod.color_psl(lrp, lci)
        np.testing.assert_array_equal(gl.gl_precond_level_colors(G, 1), colpsl)
        print(f"level 1: {len(lrp) - 1} nodes, {npsl} colours in {levels.max() + 1} removal rounds")
        others = {}
        for name, c in (("sl", gl.GL_COLOR_SL), ("jp", gl.GL_COLOR_JP)):
            Gc = gl.gl_precond_setup(gm, psi, gl.options(precision=gl.GL_MIXED, coloring=c))
            try:
                nref, cref = (oracle_mod.color_sl(lrp, lci)[:2] if name == "sl" else oracle_mod.color_jp(lrp, lci))
                np.testing.assert_array_equal(gl.gl_precond_level_colors(Gc, 1), cref)
                others[name] = nref
            finally:
                gl.gl_precond_destroy(Gc)
        assert npsl <= others["sl"] and npsl < others["jp"]
    finally:
        gl.gl_precond_destroy(G)


@pytest.mark.parametrize("precision", [gl.GL_FP64, gl.GL_MIXED, gl.GL_MIXED_PRECOND])
def test_solve_full_size_true_residual(big, precision):
    """The bench's solve reaches ||b - J x||_D / ||b||_D <= 1e-10 measured with the
    oracle's Jacobian, for psi == 1 (bench) and psi uniform in the unit disk."""
    om, gm = big
    n = om.n
    b = gi.complex_normal(n, 5)
    vol = om.volumes()
    for psi_h in (np.ones(n, complex), gi.disk(n, 4)):
        psi = torch.from_numpy(psi_h).to(DEV)
        G = gl.gl_precond_setup(gm, psi, gl.options(precision=precision))
        try:
            x = torch.zeros(n, dtype=torch.complex128, device=DEV)
            st, info = gl.gl_jacobian_solve(gm, psi, G, torch.from_numpy(b).to(DEV), x,
                                            gl.options(precision=precision))
            assert st == 0 and info.converged
            torch.cuda.synchronize()
            xh = x.cpu().numpy()
            r = b - om.jacobian(psi_h, xh)
            rel = np.sqrt(np.sum(vol * np.abs(r) ** 2) / np.sum(vol * np.abs(b) ** 2))
            assert rel <= 1.01e-10, rel
        finally:
            gl.gl_precond_destroy(G)
