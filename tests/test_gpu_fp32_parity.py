"""Element-level parity of the reduced-precision kernels the headline solve runs
(GL_MIXED_PRECOND on meshes with an even number of nodes per side) with the
FP64 oracle:

* the FP32 V-cycle R_1 (lattice-stencil finest sweeps and residual, FP32 coarse
  sweeps, restriction and prolongation, FP64 coarsest solve) against the
  oracle's R_1 (Eq. prec2) on the same hierarchy;
* the double-FP32 Jacobian apply (about 48 significant bits) against the
  oracle's J(psi) applied to the same FP32-rounded vector (Sec. 3).

Bounds, from the arithmetic:
* FP32 V-cycle: each entry of z passes through O(10^2) FP32 roundings of unit
  roundoff u32 = 2^-24 (about 4 sweeps and 3 transfers per level, each summing
  a few tens of products), and the smoothing and coarse correction are
  contractions, so for R_1 ||z32 - z||_D <= 2^8 u32 ||z||_D (= 1.5e-5).  R_k
  with k >= 2 forms the finest residual r = v - P-hat z between cycles in FP32:
  its entries are differences of terms as large as the row magnitude sum times
  |z|, while ||r|| is about 0.13 ||v|| (the V-cycle's contraction), so r carries
  an error up to 2^4 times larger relative to itself, which the next cycle
  passes on: bound 2^12 u32 (= 2.4e-4).  The measured errors are printed (R_1:
  2 to 5 u32; R_2: 100 to 800 u32 on these meshes).
* double-FP32 Jacobian: a row is formed from hi + lo pairs with error-free
  transformations (about 48 bits), so |y - y_ref| <= 2^-44 |row|, with |row| the
  row's magnitude sum sum_k |K_ik||phi_k| + (1 + 3|psi_i|^2)|phi_i|, against
  64 eps64 = 2^-46 |row| for the FP64 apply.
"""
import numpy as np
import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

BH3 = gi.WORKLOADS["cube128"][3]
DEV = torch.device("cuda:0")
U32 = 2.0 ** -24
# even N (the lattice stencil needs it); N^dim is not a multiple of 256, so every
# kernel has a ragged tail, and each case spans several CTAs
EVEN = [(2, 50), (2, 96), (3, 18), (3, 24), (3, 26)]


def bhat(dim):
    return BH3 if dim == 3 else (0.0, 0.0, 1.0)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def dnorm(vol, z):
    return float(np.sqrt(np.sum(vol * np.abs(z) ** 2)))


@pytest.mark.parametrize("dim,N", EVEN, ids=lambda p: str(p))
@pytest.mark.parametrize("cycles", [1, 2])
def test_fp32_vcycle_matches_oracle_r1(oracle_mod, dim, N, cycles):
    om = oracle_mod.Mesh(dim, N, 1.0, bhat(dim))
    m = gl.gl_mesh_create(dim, N, 1.0, bhat(dim))
    n = om.n
    psi, v = gi.disk(n, 31), gi.complex_normal(n, 32)
    opts = dict(max_coarse=24, cycles=cycles)
    P = oracle_mod.Precond(om, psi, **opts)
    G = gl.gl_precond_setup(m, dev(psi), gl.options(precision=gl.GL_MIXED_PRECOND, **opts))
    try:
        z = torch.empty(n, dtype=torch.complex128, device=DEV)
        gl.gl_precond_apply_precision(G, dev(v), z, gl.GL_MIXED_PRECOND)
        # the FP32 V-cycle sees v rounded to FP32: compare with the oracle's R_1 of that vector
        v32 = v.astype(np.complex64).astype(np.complex128)
        ref = P.apply(v32)
        vol = om.volumes()
        err = dnorm(vol, host(z) - ref) / dnorm(vol, ref)
        print(f"{dim}d N={N} R_{cycles}: ||z32 - z||_D / ||z||_D = {err:.2e} ({err / U32:.1f} u32)")
        assert err <= (2 ** 8 if cycles == 1 else 2 ** 12) * U32
        # the lattice stencil took the finest level (even N)
        x = torch.zeros(n, dtype=torch.complex128, device=DEV)
        st, info = gl.gl_jacobian_solve(m, dev(psi), G, dev(v), x,
                                        gl.options(precision=gl.GL_MIXED_PRECOND, **opts))
        assert st == 0 and info.lattice_stencil == 1
    finally:
        gl.gl_precond_destroy(G)
        gl.gl_mesh_destroy(m)


# meshes whose coarsest level (max_coarse 4096, two levels) has 1294 and 1661
# nodes: rows longer than a block's threads with a ragged tail
LARGE_COARSEST = [(2, 96), (3, 26)]


@pytest.mark.parametrize("dim,N", LARGE_COARSEST, ids=lambda p: str(p))
def test_fp32_vcycle_large_coarsest_matches_oracle(oracle_mod, dim, N):
    """The FP32 V-cycle with the double-FP32 coarsest product on a coarsest level
    of the benchmark's size class: against the oracle's R_1 at the FP32
    V-cycle's bound, and against the same V-cycle with the FP64 coarsest
    product, which differs only where the FP32 roundings of a 48-bit and a
    53-bit value of the same product differ (a few u32)."""
    om = oracle_mod.Mesh(dim, N, 1.0, bhat(dim))
    m = gl.gl_mesh_create(dim, N, 1.0, bhat(dim))
    n = om.n
    psi, v = gi.disk(n, 31), gi.complex_normal(n, 32)
    P = oracle_mod.Precond(om, psi, max_coarse=4096)
    Gs = [gl.gl_precond_setup(m, dev(psi), gl.options(precision=gl.GL_MIXED_PRECOND, max_coarse=4096,
                                                      coarse_df=df)) for df in (1, 0)]
    try:
        nc = gl.gl_precond_level_info(Gs[0], 1)["n"]
        assert gl.gl_precond_levels(Gs[0]) == 2 and nc > 1024 and nc % 32 != 0
        zs = []
        for G in Gs:
            z = torch.empty(n, dtype=torch.complex128, device=DEV)
            gl.gl_precond_apply_precision(G, dev(v), z, gl.GL_MIXED_PRECOND)
            zs.append(host(z))
        ref = P.apply(v.astype(np.complex64).astype(np.complex128))
        vol = om.volumes()
        err = dnorm(vol, zs[0] - ref) / dnorm(vol, ref)
        dif = dnorm(vol, zs[0] - zs[1]) / dnorm(vol, zs[1])
        print(f"{dim}d N={N} coarsest {nc}: vs oracle {err / U32:.1f} u32, vs FP64 coarsest product {dif / U32:.2f} u32")
        assert err <= 2 ** 8 * U32
        assert dif <= 4 * U32
    finally:
        for G in Gs:
            gl.gl_precond_destroy(G)
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("dim,N", EVEN, ids=lambda p: str(p))
def test_double_fp32_jacobian_matches_oracle(oracle_mod, dim, N):
    om = oracle_mod.Mesh(dim, N, 1.0, bhat(dim))
    m = gl.gl_mesh_create(dim, N, 1.0, bhat(dim))
    n = om.n
    try:
        psi = gi.disk(n, 33)
        phi = gi.complex_normal(n, 34).astype(np.complex64).astype(np.complex128)
        y = torch.empty(n, dtype=torch.complex128, device=DEV)
        gl.gl_jacobian_apply(m, dev(psi), dev(phi), y, precision=gl.GL_MIXED_PRECOND)
        ref = om.jacobian(psi, phi)
        rp, ci, v = om.khat_csr()
        a = np.abs(v)
        ap = np.abs(phi)
        vol = om.volumes()
        row = np.add.reduceat(a * ap[ci], rp[:-1]) / vol + (1 + 3 * np.abs(psi) ** 2) * ap
        rel = np.abs(host(y) - ref) / row
        print(f"{dim}d N={N}: max |y - y_ref| / |row| = {rel.max():.2e} (2^{np.log2(rel.max()):.1f})")
        assert rel.max() <= 2.0 ** -44
        # the degenerate case without field: K's null vector phi = 1, where K phi
        # cancels entirely (the table phases are exactly 1)
        m0 = gl.gl_mesh_create(dim, N, 0.0, bhat(dim))
        om0 = oracle_mod.Mesh(dim, N, 0.0, bhat(dim))
        try:
            one = np.ones(n, np.complex128)
            gl.gl_jacobian_apply(m0, dev(psi), dev(one), y, precision=gl.GL_MIXED_PRECOND)
            ref0 = om0.jacobian(psi, one)
            rp0, ci0, v0 = om0.khat_csr()
            row0 = np.add.reduceat(np.abs(v0), rp0[:-1]) / om0.volumes() + (1 + 3 * np.abs(psi) ** 2)
            assert (np.abs(host(y) - ref0) / row0).max() <= 2.0 ** -44
        finally:
            gl.gl_mesh_destroy(m0)
    finally:
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("dim,N", EVEN, ids=lambda p: str(p))
def test_fp64_lattice_jacobian_matches_oracle(oracle_mod, dim, N):
    """The FP64 Jacobian from the lattice tables (matrix-free; gl_jacobian_apply with
    GL_APPLY_FP64_TABLES, and MINRES's FP64 apply with options.lattice = 2) against
    the oracle's J, element by element at 64 eps64 of the row's magnitude sum; an
    FP64 solve with lattice = 2 reports that it ran from the tables, with lattice =
    1 from the stored K; the two solves (to 1e-10) agree within one iteration and
    1e-8 in the solution."""
    om = oracle_mod.Mesh(dim, N, 1.0, bhat(dim))
    m = gl.gl_mesh_create(dim, N, 1.0, bhat(dim))
    n = om.n
    try:
        psi, phi = gi.disk(n, 37), gi.complex_normal(n, 38)
        y = torch.empty(n, dtype=torch.complex128, device=DEV)
        gl.gl_jacobian_apply(m, dev(psi), dev(phi), y, precision=gl.GL_APPLY_FP64_TABLES)
        ref = om.jacobian(psi, phi)
        rp, ci, v = om.khat_csr()
        row = np.add.reduceat(np.abs(v) * np.abs(phi)[ci], rp[:-1]) / om.volumes() + \
            (1 + 3 * np.abs(psi) ** 2) * np.abs(phi)
        rel = np.abs(host(y) - ref) / row
        print(f"{dim}d N={N}: FP64 lattice J, max |y - y_ref| / |row| = {rel.max():.2e} eps64 x "
              f"{rel.max() / 2.0 ** -52:.1f}")
        assert rel.max() <= 64 * 2.0 ** -52
        b = dev(gi.complex_normal(n, 39))
        xs, infos = [], []
        for lat in (2, 1):
            x = torch.zeros(n, dtype=torch.complex128, device=DEV)
            st, info = gl.gl_jacobian_solve(m, dev(psi), None, b, x, gl.options(max_coarse=64, lattice=lat))
            assert st == 0 and info.converged
            xs.append(x)
            infos.append(info)
        assert infos[0].jacobian_tables == 1 and infos[1].jacobian_tables == 0
        assert abs(infos[0].iters - infos[1].iters) <= 1
        assert float(torch.linalg.norm(xs[0] - xs[1]) / torch.linalg.norm(xs[1])) <= 1e-8
    finally:
        gl.gl_mesh_destroy(m)


def test_double_fp32_jacobian_needs_even_n():
    m = gl.gl_mesh_create(2, 17, 1.0)
    try:
        x = torch.ones(17 * 17, dtype=torch.complex128, device=DEV)
        y = torch.empty_like(x)
        with pytest.raises(gl.GLError):
            gl.gl_jacobian_apply(m, x, x, y, precision=gl.GL_MIXED_PRECOND)
        with pytest.raises(gl.GLError):
            gl.gl_jacobian_apply(m, x, x, y, precision=gl.GL_APPLY_FP64_TABLES)
        # an odd-N mesh has no lattice stencil: the FP64 solve streams the stored K
        b = dev(gi.complex_normal(17 * 17, 40))
        z = torch.zeros_like(b)
        st, info = gl.gl_jacobian_solve(m, x, None, b, z, gl.options(max_coarse=64, lattice=2))
        assert st == 0 and info.jacobian_tables == 0
    finally:
        gl.gl_mesh_destroy(m)


@pytest.mark.parametrize("precision", [gl.GL_FP64, gl.GL_MIXED_PRECOND], ids=["fp64", "fp32vc"])
def test_flag_and_grid_sweeps_bit_identical(precision):
    """The neighbour-flag sweep and the grid-barrier sweep give every row the same
    inputs in the same order: for the same lanes per row (autotune off) their
    preconditioner outputs agree bit for bit."""
    N = 48
    m = gl.gl_mesh_create(3, N, 1.0, BH3)
    n = N ** 3
    psi, v = dev(gi.disk(n, 35)), dev(gi.complex_normal(n, 36))
    zs = []
    try:
        for sync in (1, 2):
            G = gl.gl_precond_setup(m, psi, gl.options(max_coarse=256, sweep_sync=sync, autotune=0,
                                                       cluster_sweeps=0, precision=precision))
            try:
                # level 1 runs the asked-for synchronisation on several CTAs
                sw = gl.gl_precond_level_sweep(G, 1, precision)
                assert sw["sync"] == sync - 1, sw
                if sync == 2:
                    assert sw["ctas"] >= 4, sw
                z = torch.empty_like(psi)
                gl.gl_precond_apply_precision(G, v, z, precision)
                torch.cuda.synchronize()
                zs.append(z)
            finally:
                gl.gl_precond_destroy(G)
        assert torch.equal(zs[0], zs[1])
    finally:
        gl.gl_mesh_destroy(m)
