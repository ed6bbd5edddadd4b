"""Parameter continuation in mu on the GPU (Sec. 4, Fig. 4): domains of any
edge length, the in-place change of mu, the energy and d GL / d mu against the
oracle, and the pseudo-arclength driver against the oracle's restatement
(``oracle/continuation.py``) step by step."""
import numpy as np
import pytest

import gl_inputs as gi
from oracle import continuation as ocont

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
BH3 = gi.WORKLOADS["cube128"][3]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,N,edge,mu,field", [(2, 33, 10.0, 0.3, (0.0, 0.0, 1.0)), (3, 9, 3.0, 0.8, BH3)])
def test_edge_mesh_energy_dmu(oracle_mod, dim, N, edge, mu, field):
    om = oracle_mod.Mesh(dim, N, mu, field, edge=edge)
    m = gl.gl_mesh_create(dim, N, mu, field, edge=edge)
    try:
        rp, ci, v = gl.gl_mesh_khat(m)
        orp, oci, ov = om.khat_csr()
        np.testing.assert_array_equal(rp, orp)
        np.testing.assert_array_equal(ci, oci)
        np.testing.assert_allclose(v, ov, rtol=0, atol=1e-13 * np.abs(ov).max())
        psi = gi.disk(om.n, 4)
        F = gl.gl_energy(m, dev(psi))
        assert F == pytest.approx(om.energy(psi), rel=1e-12)
        d = torch.zeros(om.n, dtype=torch.complex128, device=DEV)
        gl.gl_residual_dmu(m, dev(psi), d)
        od = om.residual_dmu(psi)
        np.testing.assert_allclose(d.cpu().numpy(), od, rtol=0, atol=1e-12 * np.abs(od).max())
    finally:
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("precision", [gl.GL_FP64, gl.GL_MIXED_PRECOND])
def test_set_mu_matches_a_fresh_mesh(oracle_mod, precision):
    """gl_mesh_set_mu(0.2 -> 0.7) gives the operator of a mesh made at 0.7 (to the
    last bits of the phase), solves on it match the oracle at 0.7, and a
    preconditioner from before the change is refused."""
    N, edge = 40, 10.0
    om = oracle_mod.Mesh(2, N, 0.7, edge=edge)
    m = gl.gl_mesh_create(2, N, 0.2, edge=edge)
    psi, b = gi.disk(om.n, 5), gi.complex_normal(om.n, 6)
    opts = gl.options(max_coarse=64, precision=precision)
    try:
        G_old = gl.gl_precond_setup(m, dev(psi), opts)
        x = torch.zeros(om.n, dtype=torch.complex128, device=DEV)
        gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x, opts)  # builds the FP32 copies at 0.2
        gl.gl_mesh_set_mu(m, 0.7)
        rp, ci, v = gl.gl_mesh_khat(m)
        np.testing.assert_allclose(v, om.khat_csr()[2], rtol=0, atol=1e-14 * np.abs(v).max())
        r = torch.zeros_like(x)
        gl.gl_residual(m, dev(psi), r)
        np.testing.assert_allclose(r.cpu().numpy(), om.residual(psi), rtol=0, atol=1e-12 * np.abs(om.residual(psi)).max())
        x.zero_()
        st, info = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x, opts)
        assert st == 0 and info.converged
        xo, _ = om.solve(psi, b, max_coarse=64, tol=1e-12)
        assert rel(x.cpu().numpy(), xo) <= 1e-7
        if precision == gl.GL_MIXED_PRECOND:
            assert info.lattice_stencil == 1 and info.df_jacobian == 1
        with pytest.raises(gl.GLError):
            gl.gl_jacobian_solve(m, dev(psi), G_old, dev(b), x, opts)
        gl.gl_precond_destroy(G_old)
    finally:
        gl.gl_mesh_destroy(m)


def test_continuation_matches_oracle(oracle_mod):
    """The first steps of the continuation on the edge-10 square from psi = 1 at
    mu = 0 (Fig. 4's setting on a 33 x 33 mesh): every accepted point (mu, energy,
    Newton steps) equals the oracle's; the fold near mu = 0.30 appears in both."""
    N, edge, steps = 33, 10.0, 10
    kw = dict(ds=0.1, ds_max=0.3, max_steps=steps, mu_max=1.2, newton_tol=1e-9, newton_maxit=8)
    opts_o = dict(kw, linear_tol=1e-8, max_coarse=512)
    pts_o, psi_o, mu_o = ocont.continuation(2, N, edge, np.ones(N * N, complex), 0.0, **opts_o)
    m = gl.gl_mesh_create(2, N, 0.0, edge=edge)
    try:
        psi = torch.ones(N * N, dtype=torch.complex128, device=DEV)
        co = gl.cont_options(**kw, solver=dict(tol=1e-8, max_coarse=512))
        st, pts = gl.gl_continuation(m, psi, co, max_points=64)
        assert st == 0
        assert len(pts) == len(pts_o) == steps + 1
        before_fold = True
        for k, (p, q) in enumerate(zip(pts, pts_o)):
            print(f"{k:2d} mu {p['mu']:.6f} ({q['mu']:.6f}) F {p['energy']:.6f} ({q['energy']:.6f}) newton "
                  f"{p['newton_steps']} ({q['newton']}) last {p['iters_last']} ({q['iters_last']})")
            assert p["newton_steps"] == q["newton"] and p["retries"] == q["retries"]
            assert p["mu"] == pytest.approx(q["mu"], abs=1e-7)
            assert p["energy"] == pytest.approx(q["energy"], abs=1e-7)
            # strictly before the turning point: mu rises into the point and out of it
            rises_out = k + 1 < len(pts) and pts[k + 1]["mu"] > p["mu"]
            before_fold = before_fold and (k == 0 or p["mu"] > pts[k - 1]["mu"]) and rises_out
            # the last Newton step solves for a correction of GL already near its
            # rounding level; before the fold J is definite there and the counts
            # agree; at the turning point J is nearly singular and past it indefinite,
            # and there that count is rounding noise
            if before_fold:
                assert abs(p["iters_last"] - q["iters_last"]) <= max(2, 0.1 * q["iters_last"])
        mus = np.array([p["mu"] for p in pts])
        turn = int(np.argmax(np.diff(mus) < 0))
        assert turn > 0 and 0.27 <= mus[turn] <= 0.33, mus
        assert rel(psi.cpu().numpy(), psi_o) <= 1e-6
    finally:
        gl.gl_mesh_destroy(m)


def read_fig4():
    import os

    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig4_continuation_states.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                mu, F = line.split()
                rows.append((float(mu), float(F)))
    return rows


def test_continuation_fig4_shape():
    """Fig. 4 on a 201 x 201 mesh of the edge-10 square, 80 steps: the energy per
    unit volume starts at -1/2 and rises, the curve folds back (swallow tail)
    near mu = 0.30 and again further on (vortices entering), and past the first
    fold, where the Jacobian gains an unstable eigenvalue, MINRES needs more
    iterations than before it; near mu = 0.8 several times as many."""
    N, edge = 201, 10.0
    m = gl.gl_mesh_create(2, N, 0.0, edge=edge)
    try:
        psi = torch.ones(N * N, dtype=torch.complex128, device=DEV)
        co = gl.cont_options(ds=0.1, ds_max=0.3, max_steps=80, mu_max=1.0, solver=dict(tol=1e-8))
        st, pts = gl.gl_continuation(m, psi, co, max_points=128)
        assert st == 0
        for k, p in enumerate(pts):
            print(f"{k:2d} mu {p['mu']:.4f} F {p['energy']:.5f} newton {p['newton_steps']} last {p['iters_last']} "
                  f"total {p['iters_total']} setup {p['setup_ms']:.1f} ms solve {p['solve_ms']:.1f} ms")
        mus = np.array([p["mu"] for p in pts])
        F = np.array([p["energy"] for p in pts])
        assert F[0] == pytest.approx(-0.5, abs=1e-12)
        assert np.all(np.diff(F[: int(np.argmax(np.diff(mus) < 0)) + 1]) > 0)
        turn = int(np.argmax(np.diff(mus) < 0))
        assert turn > 0 and 0.25 <= mus[turn] <= 0.35, mus
        its = np.array([p["iters_last"] for p in pts])
        assert np.median(its[turn + 2:]) > np.median(its[1:turn])
        folds = int(np.sum(np.diff(np.sign(np.diff(mus))) != 0))
        assert folds >= 2 and len(pts) == 81
        late = its[(mus > 0.7) & (np.arange(len(mus)) > turn)]
        assert late.size and late.max() >= 3 * np.median(its[1:turn])
        # the states printed in Fig. 4: where the curve first reaches mu = 0.47 (0.93)
        # after its first fold, 2 F / |Omega| = -0.47 (-0.12), to the printed digits
        first_fold = next(k for k in range(1, len(mus) - 1) if (mus[k] - mus[k - 1]) * (mus[k + 1] - mus[k]) < 0)
        for mu_p, F_p in read_fig4():
            k = next(k for k in range(first_fold, len(mus) - 1) if (mus[k] - mu_p) * (mus[k + 1] - mu_p) <= 0)
            w = (mu_p - mus[k]) / (mus[k + 1] - mus[k])
            F_here = 2.0 * ((1 - w) * F[k] + w * F[k + 1])
            print(f"Fig. 4 state: mu {mu_p}: 2F/|Omega| = {F_here:.4f} (paper {F_p})")
            assert abs(F_here - F_p) <= 0.01
    finally:
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("autotune", [0, 1])
def test_setup_like_reuses_the_symbolic_hierarchy(autotune):
    """A setup for a new psi and mu that takes over an earlier preconditioner's
    aggregates, colours and kernel choices gives the same hierarchy as a full
    setup (aggregates, colours and level matrices bit for bit) and the same
    solve (bit for bit when neither setup times kernels)."""
    import time

    N = 24
    bh = gi.WORKLOADS["cube128"][3]
    m = gl.gl_mesh_create(3, N, 0.4, bh, edge=4.0)
    n = N ** 3
    opts = gl.options(max_coarse=64, autotune=autotune, precision=gl.GL_MIXED_PRECOND)
    psi1, psi2 = dev(gi.disk(n, 1)), dev(gi.psi_noisy_one(n, 2))
    b = dev(gi.complex_normal(n, 3))
    G1 = gl.gl_precond_setup(m, psi1, opts)
    try:
        gl.gl_mesh_set_mu(m, 0.9)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G2 = gl.gl_precond_setup_like(m, psi2, G1, opts)
        t1 = time.perf_counter()
        G3 = gl.gl_precond_setup(m, psi2, opts)
        t2 = time.perf_counter()
        try:
            nl = gl.gl_precond_levels(G3)
            assert gl.gl_precond_levels(G2) == nl >= 3
            for lv in range(nl):
                for a, c in zip(gl.gl_precond_level_matrix(G2, lv), gl.gl_precond_level_matrix(G3, lv)):
                    np.testing.assert_array_equal(a, c)
                np.testing.assert_array_equal(gl.gl_precond_level_colors(G2, lv), gl.gl_precond_level_colors(G3, lv))
                if lv + 1 < nl:
                    np.testing.assert_array_equal(gl.gl_precond_level_aggregates(G2, lv),
                                                  gl.gl_precond_level_aggregates(G3, lv))
            xs = []
            for G in (G2, G3):
                x = torch.zeros(n, dtype=torch.complex128, device=DEV)
                st, info = gl.gl_jacobian_solve(m, psi2, G, b, x, opts)
                assert st == 0 and info.converged
                xs.append(x.cpu().numpy())
            if autotune == 0:
                np.testing.assert_array_equal(xs[0], xs[1])
            else:
                assert rel(xs[0], xs[1]) <= 1e-8
            print(f"autotune {autotune}: setup taking over {1e3 * (t1 - t0):.1f} ms, full {1e3 * (t2 - t1):.1f} ms")
        finally:
            gl.gl_precond_destroy(G2)
            gl.gl_precond_destroy(G3)
    finally:
        gl.gl_precond_destroy(G1)
        gl.gl_mesh_destroy(m)


def test_resume_from_checkpoint(tmp_path):
    """A continuation stopped after a few points, saved (mu, psi, the points so
    far) and reloaded, restarts from exactly the saved state on a mesh made from
    the saved description, and continues."""
    from paper_1204_5125_gb300 import state

    N, edge = 33, 10.0
    kw = dict(ds=0.1, ds_max=0.3, mu_max=1.2, newton_tol=1e-9, newton_maxit=8, solver=dict(tol=1e-8, max_coarse=512))
    m = gl.gl_mesh_create(2, N, 0.0, edge=edge)
    try:
        psi = torch.ones(N * N, dtype=torch.complex128, device=DEV)
        st, pts = gl.gl_continuation(m, psi, gl.cont_options(max_steps=4, **kw), max_points=16)
        assert st == 0 and len(pts) == 5
        state.save_state(str(tmp_path), dim=2, N=N, mu=pts[-1]["mu"], psi=psi, edge=edge, points=pts)
    finally:
        gl.gl_mesh_destroy(m)
    s = state.load_state(str(tmp_path))
    assert s["points"][-1]["mu"] == pts[-1]["mu"]
    m = gl.gl_mesh_create(2, s["N"], s["mu"], edge=s["edge"])
    try:
        psi2 = torch.from_numpy(s["psi"]).to(DEV)
        vol = torch.zeros(N * N, dtype=torch.float64, device=DEV)
        gl.gl_mesh_info(m, vol)
        # the points carry F / |Omega|
        assert float(gl.gl_energy(m, psi2)) / float(vol.sum()) == pytest.approx(pts[-1]["energy"], rel=1e-12)
        st, more = gl.gl_continuation(m, psi2, gl.cont_options(max_steps=3, **kw), max_points=16)
        assert st == 0 and len(more) == 4
        assert more[0]["mu"] == pytest.approx(pts[-1]["mu"], abs=1e-14)
        assert more[0]["energy"] == pytest.approx(pts[-1]["energy"], rel=1e-12)
        assert all(p["newton_steps"] <= 8 for p in more)
    finally:
        gl.gl_mesh_destroy(m)
