"""Mesh independence of the R_1-preconditioned MINRES iteration counts on the GPU
(Sec. 4, Fig. 3: the counts stay bounded as the mesh is refined), at the sizes
of the benchmark's sweep: 2D squares N = 32 ... 1024 (mu = 1 along z) and 3D
cubes N = 16 ... 128 (mu = 1 along (1,1,1)/sqrt 3), psi = 1 (the paper's
setting), right-hand side complex normal (seed 5), tol 1e-10, x0 = 0, the
default hierarchy (coarsening down to 512 nodes), in FP64 and with the FP32
V-cycle.  Every solve must reach the FP64 true residual 1e-10.  The counts rise
where the hierarchy gains a level (a V-cycle with one more multicoloured level
contracts a little less) and are otherwise flat: over a 1000-fold growth of n
they stay below twice the smallest count plus two, and the three largest 2D
meshes (same depth) agree within two.  Measured on one GB300 (FP64): squares
15, 19, 18, 25, 26, 26; cubes 14, 18, 18, 25.  The counts are printed."""
import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
FAMILIES = {
    "square": (2, [32, 64, 128, 256, 512, 1024], (0.0, 0.0, 1.0)),
    "cube": (3, [16, 32, 64, 128], gi.WORKLOADS["cube128"][3]),
}


@pytest.mark.parametrize("precision", [gl.GL_FP64, gl.GL_MIXED_PRECOND], ids=["fp64", "fp32vc"])
@pytest.mark.parametrize("family", list(FAMILIES))
def test_iteration_counts_flat_in_n(family, precision):
    dim, sizes, bh = FAMILIES[family]
    counts = []
    for N in sizes:
        n = N ** dim
        m = gl.gl_mesh_create(dim, N, 1.0, bh)
        try:
            psi = torch.ones(n, dtype=torch.complex128, device=DEV)
            b = torch.from_numpy(gi.complex_normal(n, 5)).to(DEV)
            x = torch.zeros_like(b)
            st, info = gl.gl_jacobian_solve(m, psi, None, b, x, gl.options(precision=precision))
            assert st == 0 and info.converged and info.true_relres <= 1.01e-10, (N, info.as_dict())
            counts.append(info.iters)
        finally:
            gl.gl_mesh_destroy(m)
    print(f"{family} precision {precision}: N {sizes} -> iterations {counts}")
    assert max(counts) <= 2 * min(counts) + 2, counts
    if family == "square":
        assert max(counts[-3:]) - min(counts[-3:]) <= 2, counts
