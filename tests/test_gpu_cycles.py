"""R_k for k > 1 and R_10 ~ R_inf (Eq. prec1, prec2), and the cost measure of
Fig. 1 (matrix-vector-product equivalents), on the GPU.

Fig. 1's setting on a smaller square: psi == b == 1, field along z, k in
{1, 2, 5, 10}.  Checked: the cost model equals the oracle's count exactly;
iteration counts match the oracle's within one and fall with k; the cost in
matvec equivalents and the measured GPU time are lowest for k = 1 (the
paper's conclusion); the preconditioning residual after k cycles equals the
oracle's."""
import numpy as np
import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("dim,N,mc", [(2, 45, 32), (3, 13, 24), (2, 9, 128)])  # the last: one level
def test_cost_model_matches_oracle(oracle_mod, dim, N, mc):
    om = oracle_mod.Mesh(dim, N, 1.0)
    psi = gi.disk(om.n, 7)
    P = oracle_mod.Precond(om, psi, max_coarse=mc)
    m = gl.gl_mesh_create(dim, N, 1.0)
    G = gl.gl_precond_setup(m, dev(psi), gl.options(max_coarse=mc))
    try:
        for k in (1, 2, 10):
            assert gl.gl_precond_cost(G, k) == pytest.approx(P.cost(k), rel=1e-14)
    finally:
        gl.gl_precond_destroy(G)
        gl.gl_mesh_destroy(m)


def test_fig1_cycles_on_gpu(oracle_mod):
    N, mu = 257, 1.0
    om = oracle_mod.Mesh(2, N, mu)
    n = om.n
    psi = np.ones(n, np.complex128)
    b = np.ones(n, np.complex128)
    m = gl.gl_mesh_create(2, N, mu)
    res = {}
    try:
        for k in (1, 2, 5, 10):
            opts = gl.options(cycles=k, max_coarse=512)
            G = gl.gl_precond_setup(m, dev(psi), opts)
            try:
                x = torch.zeros(n, dtype=torch.complex128, device=DEV)
                gl.gl_jacobian_solve(m, dev(psi), G, dev(b), x, opts)  # warm-up (graph capture)
                times = []
                for _ in range(3):
                    x.zero_()
                    st, info = gl.gl_jacobian_solve(m, dev(psi), G, dev(b), x, opts)
                    assert st == 0 and info.converged
                    times.append(info.solve_ms)
                _, oinfo = om.solve(psi, b, cycles=k, max_coarse=512, tol=1e-10)
                # R_k applies agree to ~4e-14; with R_10 the oracle stops at a true
                # residual of 9.99e-11, a borderline the GPU's rounding lands just
                # above, and the true residual then needs three more iterations
                slack = 1 if k <= 5 else 3
                assert abs(info.iters - oinfo.iters) <= slack, (k, info.iters, oinfo.iters)
                res[k] = (info.iters, info.matvec_equiv, min(times), gl.gl_precond_cost(G, 1))
            finally:
                gl.gl_precond_destroy(G)
        for k, (it, mv, ms, vc) in res.items():
            print(f"k={k:2d}: {it:3d} iterations, {mv:7.1f} matvec equivalents (V-cycle = {vc:.2f}), {ms:.2f} ms")
        its = [res[k][0] for k in (1, 2, 5, 10)]
        assert all(a >= b for a, b in zip(its, its[1:])) and its[0] > its[-1]
        assert min(res, key=lambda k: res[k][1]) == 1
        assert min(res, key=lambda k: res[k][2]) == 1
    finally:
        gl.gl_mesh_destroy(m)


def test_rk_residual_matches_oracle(oracle_mod):
    """k V-cycles of the GPU reduce the preconditioning residual of
    (K-hat + 2 D|psi|^2) z = D v exactly as the oracle's do, and more cycles
    reduce it further.  (With these SA parameters one V-cycle contracts by about
    0.45 in 2D, so R_10 leaves ~2e-4 here: not the near-exact inverse the paper's
    PyAMG V-cycle gave after ten cycles.)"""
    N, mu = 129, 1.0
    om = oracle_mod.Mesh(2, N, mu)
    n = om.n
    psi = gi.psi_noisy_one(n, 9)
    v = gi.complex_normal(n, 10)
    vol = om.volumes()
    m = gl.gl_mesh_create(2, N, mu)
    prev = np.inf
    try:
        for k in (1, 2, 10):
            G = gl.gl_precond_setup(m, dev(psi), gl.options(cycles=k, max_coarse=512))
            try:
                z = torch.zeros(n, dtype=torch.complex128, device=DEV)
                gl.gl_precond_apply(G, dev(v), z)
            finally:
                gl.gl_precond_destroy(G)
            zh = z.cpu().numpy()
            zo = oracle_mod.Precond(om, psi, cycles=k, max_coarse=512).apply(v)
            r = v - (om.kinetic(zh) + 2 * np.abs(psi) ** 2 * zh)  # D^-1 (D v - P-hat z)
            ro = v - (om.kinetic(zo) + 2 * np.abs(psi) ** 2 * zo)
            rel = np.sqrt(np.sum(vol * np.abs(r) ** 2) / np.sum(vol * np.abs(v) ** 2))
            relo = np.sqrt(np.sum(vol * np.abs(ro) ** 2) / np.sum(vol * np.abs(v) ** 2))
            print(f"R_{k} residual {rel:.3e} (oracle {relo:.3e})")
            assert rel == pytest.approx(relo, rel=1e-6)
            assert rel < prev
            prev = rel
        assert prev < 1e-3
    finally:
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("dim,N,mc", [(2, 65, 64), (3, 17, 64)])
def test_rinf_apply(oracle_mod, dim, N, mc):
    """R_inf = P^-1 D (Eq. prec1): the GPU's cycled V-cycle against a sparse
    direct solve of K-hat + 2 D|psi|^2 and against the oracle's R_inf; the
    device loop runs the same number of cycles as the oracle (within one, the
    stopping test sits at 1e-12 where rounding may move it)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    field = (0.0, 0.0, 1.0) if dim == 2 else gi.WORKLOADS["cube128"][3]
    om = oracle_mod.Mesh(dim, N, 1.0, field)
    n = om.n
    psi = gi.psi_noisy_one(n, 5)
    v = gi.complex_normal(n, 6)
    vol = om.volumes()
    rp, ci, kv = om.khat_csr()
    Ph = sp.csr_matrix((kv, ci, rp), shape=(n, n)) + sp.diags(2.0 * vol * np.abs(psi) ** 2)
    exact = spl.spsolve(sp.csc_matrix(Ph), vol * v)
    zo, ko = oracle_mod.Precond(om, psi, cycles=oracle_mod.CYCLES_INF, max_coarse=mc).apply_count(v)
    dn = lambda x: np.sqrt(np.sum(vol * np.abs(x) ** 2))  # noqa: E731
    m = gl.gl_mesh_create(dim, N, 1.0, field)
    G = gl.gl_precond_setup(m, dev(psi), gl.options(cycles=gl.GL_CYCLES_INF, max_coarse=mc))
    try:
        z = torch.zeros(n, dtype=torch.complex128, device=DEV)
        gl.gl_precond_apply(G, dev(v), z)
        zg = z.cpu().numpy()
        print(f"R_inf: oracle {ko} cycles; error vs direct solve GPU {dn(zg - exact) / dn(exact):.2e}, "
              f"oracle {dn(zo - exact) / dn(exact):.2e}")
        assert dn(zg - exact) <= 1e-10 * dn(exact)
        assert dn(zg - zo) <= 1e-10 * dn(zo)
        # the same input gives the same output; a zero input gives zero
        z2 = torch.zeros_like(z)
        gl.gl_precond_apply(G, dev(v), z2)
        assert torch.equal(z, z2)
        gl.gl_precond_apply(G, torch.zeros_like(z), z2)
        assert not bool(torch.any(z2 != 0))
    finally:
        gl.gl_precond_destroy(G)
        gl.gl_mesh_destroy(m)


def test_rinf_solve(oracle_mod):
    """MINRES with R_inf on the Fig. 1 setting (psi = b = 1): iterations equal the
    oracle's within one and are at most those of R_10; the cycles per
    application and the matvec equivalents come from the device counters, and
    R_1 stays the cheapest (Fig. 1's conclusion)."""
    N, mu = 129, 1.0
    om = oracle_mod.Mesh(2, N, mu)
    n = om.n
    psi = np.ones(n, np.complex128)
    b = np.ones(n, np.complex128)
    m = gl.gl_mesh_create(2, N, mu)
    res = {}
    try:
        for k in (1, 10, gl.GL_CYCLES_INF):
            opts = gl.options(cycles=k, max_coarse=512)
            x = torch.zeros(n, dtype=torch.complex128, device=DEV)
            st, info = gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x, opts)
            assert st == 0 and info.converged
            res[k] = info
        _, oinfo = om.solve(psi, b, cycles=oracle_mod.CYCLES_INF, max_coarse=512, tol=1e-10)
        inf = res[gl.GL_CYCLES_INF]
        print(f"R_inf: {inf.iters} iterations (oracle {oinfo.iters}), {inf.cycles_per_apply:.1f} cycles per "
              f"application, {inf.matvec_equiv:.0f} matvec equivalents; R_10 {res[10].iters} iterations, "
              f"{res[10].matvec_equiv:.0f}; R_1 {res[1].iters}, {res[1].matvec_equiv:.0f}")
        assert abs(inf.iters - oinfo.iters) <= 1
        assert inf.iters <= res[10].iters
        assert 10 < inf.cycles_per_apply < 200
        assert res[1].cycles_per_apply == 1 and res[10].cycles_per_apply == 10
        # the counters: matvec_equiv = (iters + 1) + (cycles applied) x (V-cycle + residual),
        # cycles applied = applications x cycles_per_apply, one application per
        # iteration plus the initial one (a whole number within [iters, iters + 2])
        G = gl.gl_precond_setup(m, dev(psi), gl.options(max_coarse=512))
        try:
            per = gl.gl_precond_cost(G, 1) + 1.0
        finally:
            gl.gl_precond_destroy(G)
        applies = (inf.matvec_equiv - (inf.iters + 1)) / (inf.cycles_per_apply * per)
        assert abs(applies - round(applies)) < 1e-6 and inf.iters <= round(applies) <= inf.iters + 2, applies
        assert res[1].matvec_equiv < res[10].matvec_equiv < inf.matvec_equiv
        # FP32 forms reject R_inf
        with pytest.raises(gl.GLError):
            x = torch.zeros(n, dtype=torch.complex128, device=DEV)
            gl.gl_jacobian_solve(m, dev(psi), None, dev(b), x,
                                 gl.options(cycles=gl.GL_CYCLES_INF, precision=gl.GL_MIXED_PRECOND))
    finally:
        gl.gl_mesh_destroy(m)


def read_fig3():
    import os

    rows = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig3_cube_az_iterations.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, *vals = line.split()
                rows[name] = [int(v) for v in vals]
    return rows


def test_fig3_cube_rinf_on_gpu(oracle_mod):
    """Fig. 3 in the paper's own setting: the cube of circumradius 5 (edge
    10/sqrt3) in A_z, psi = 1, phi_0 = 0, tol 1e-11, on meshes whose real
    dimension 2n matches the paper's points from 2000 to 85750.  R_inf's counts
    are flat (the paper: 10 at every size; here 13: a different mesh family and
    stopping test, the spectrum of R_inf J is the same operator's), R_1's are
    flat too (the paper: 18-19) and above R_inf's; the oracle agrees within one
    where it runs in seconds."""
    fig = read_fig3()
    L = 10.0 / np.sqrt(3.0)
    rinf, r1 = [], []
    for N, dims in zip((10, 15, 20, 25, 30, 35), fig["dims"][1:]):
        assert 2 * N ** 3 == dims
        m = gl.gl_mesh_create(3, N, 1.0, (0.0, 0.0, 1.0), edge=L)
        try:
            n = N ** 3
            psi = torch.ones(n, dtype=torch.complex128, device=DEV)
            b = torch.ones(n, dtype=torch.complex128, device=DEV)
            its = []
            for k in (gl.GL_CYCLES_INF, 1):
                x = torch.zeros_like(b)
                st, info = gl.gl_jacobian_solve(m, psi, None, b, x, gl.options(tol=1e-11, cycles=k, max_coarse=64))
                assert st == 0 and info.converged
                its.append(info.iters)
            rinf.append(its[0])
            r1.append(its[1])
            if N <= 15:
                om = oracle_mod.Mesh(3, N, 1.0, (0.0, 0.0, 1.0), edge=L)
                ones = np.ones(n, complex)
                _, oi = om.solve(ones, ones, tol=1e-11, max_coarse=64, cycles=oracle_mod.CYCLES_INF)
                assert abs(oi.iters - its[0]) <= 1, (N, oi.iters, its[0])
        finally:
            gl.gl_mesh_destroy(m)
    print(f"Fig. 3 cube: 2n {fig['dims'][1:]}; R_inf {rinf} (paper {fig['Rinf'][1:]}); R_1 {r1} (paper {fig['R1'][1:]})")
    assert max(rinf) - min(rinf) <= 1 and abs(np.median(rinf) - np.median(fig["Rinf"][1:])) <= 4
    assert max(r1) - min(r1) <= 3 and all(a < b for a, b in zip(rinf, r1))
