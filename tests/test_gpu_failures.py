"""Failure detection without a GPU fault.

* Every wait of the coarse-level Gauss-Seidel sweeps (grid barrier or neighbour
  flags) is bounded by 1 s of the GPU's global timer.  gl_precond_debug
  (GL_DEBUG_STALL_SWEEPS) moves every wait target out of reach, so the waits
  run out: the solve or preconditioner call must return GL_ERR_TIMEOUT, reset
  the synchronisation state, and the next call on the same handle must give the
  normal result (the GPU context stays usable).
* A host-made indefinite preconditioner (the one-level hierarchy's dense
  inverse multiplied by -1) must end MINRES with GL_ERR_BREAKDOWN.
"""
import time

import numpy as np
import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
BH3 = gi.WORKLOADS["cube128"][3]
GL_ERR_BREAKDOWN, GL_ERR_TIMEOUT = 5, 7


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("sync", [1, 2], ids=["grid", "flags"])
@pytest.mark.parametrize("precision", [gl.GL_FP64, gl.GL_MIXED_PRECOND], ids=["fp64", "fp32vc"])
def test_sweep_wait_runs_out_and_recovers(sync, precision):
    # 48^3: level 1 has ~10^4 rows, so its sweeps run on several CTAs
    m = gl.gl_mesh_create(3, 48, 1.0, BH3)
    n = 48 ** 3
    psi, b = dev(gi.disk(n, 21)), dev(gi.complex_normal(n, 22))
    opts = gl.options(max_coarse=256, sweep_sync=sync, autotune=0, cluster_sweeps=0, precision=precision)
    P = gl.gl_precond_setup(m, psi, opts)
    try:
        assert gl.gl_precond_levels(P) >= 3
        x_ref = torch.zeros_like(psi)
        st, info_ref = gl.gl_jacobian_solve(m, psi, P, b, x_ref, opts)
        assert st == 0 and info_ref.converged
        # every wait target out of reach: the solve ends with GL_ERR_TIMEOUT
        gl.gl_precond_debug(P, gl.GL_DEBUG_STALL_SWEEPS)
        x = torch.zeros_like(psi)
        t0 = time.time()
        st, info = gl.gl_jacobian_solve(m, psi, P, b, x, opts, raise_on_fail=False)
        dt = time.time() - t0
        assert st == GL_ERR_TIMEOUT and not info.converged, (st, info.as_dict())
        assert dt < 30, dt
        # the state is reset: the same solve again gives the same iterate
        x2 = torch.zeros_like(psi)
        st, info2 = gl.gl_jacobian_solve(m, psi, P, b, x2, opts)
        assert st == 0 and info2.iters == info_ref.iters
        assert torch.equal(x2, x_ref)
        # the preconditioner call reports it too, and recovers
        z_ref, z = torch.empty_like(psi), torch.empty_like(psi)
        gl.gl_precond_apply_precision(P, b, z_ref, precision)
        gl.gl_precond_debug(P, gl.GL_DEBUG_STALL_SWEEPS)
        with pytest.raises(gl.GLError) as e:
            gl.gl_precond_apply_precision(P, b, z, precision)
        assert e.value.status == GL_ERR_TIMEOUT
        gl.gl_precond_apply_precision(P, b, z, precision)
        torch.cuda.synchronize()
        assert torch.equal(z, z_ref)
    finally:
        gl.gl_precond_destroy(P)
        gl.gl_mesh_destroy(m)


def test_indefinite_preconditioner_is_a_breakdown():
    # 16^2 = 256 nodes <= max_coarse: one level, R_1 is the dense inverse times D
    m = gl.gl_mesh_create(2, 16, 1.0)
    n = 256
    psi, b = dev(gi.disk(n, 23)), dev(gi.complex_normal(n, 24))
    P = gl.gl_precond_setup(m, psi, gl.options())
    try:
        assert gl.gl_precond_levels(P) == 1
        x = torch.zeros_like(psi)
        st, info = gl.gl_jacobian_solve(m, psi, P, b, x, gl.options())
        assert st == 0 and info.converged
        gl.gl_precond_debug(P, gl.GL_DEBUG_NEGATE_COARSEST)
        x = torch.zeros_like(psi)
        st, info = gl.gl_jacobian_solve(m, psi, P, b, x, gl.options(), raise_on_fail=False)
        assert st == GL_ERR_BREAKDOWN and not info.converged
        assert bool(torch.all(torch.isfinite(torch.view_as_real(x))))
    finally:
        gl.gl_precond_destroy(P)
        gl.gl_mesh_destroy(m)


def test_negated_coarsest_reaches_the_fp32_vcycle():
    # two levels: the FP32 V-cycle's double-FP32 copy of the coarsest inverse is
    # rebuilt from the negated FP64 inverse, so both V-cycles apply the same
    # (indefinite) operator afterwards
    m = gl.gl_mesh_create(2, 40, 1.0)
    n = 1600
    psi, b = dev(gi.disk(n, 25)), dev(gi.complex_normal(n, 26))
    P = gl.gl_precond_setup(m, psi, gl.options(precision=gl.GL_MIXED_PRECOND, max_coarse=256))
    try:
        assert gl.gl_precond_levels(P) >= 2
        z64, z32 = torch.empty_like(psi), torch.empty_like(psi)
        gl.gl_precond_apply_precision(P, b, z32, gl.GL_MIXED_PRECOND)
        before = z32.clone()
        gl.gl_precond_debug(P, gl.GL_DEBUG_NEGATE_COARSEST)
        gl.gl_precond_apply_precision(P, b, z64, gl.GL_FP64)
        gl.gl_precond_apply_precision(P, b, z32, gl.GL_MIXED_PRECOND)
        rel = lambda a, c: float(torch.linalg.vector_norm(a - c) / torch.linalg.vector_norm(c))
        assert rel(z32, z64) <= 2 ** 8 * 2.0 ** -24
        assert rel(before, z64) > 1e-3
    finally:
        gl.gl_precond_destroy(P)
        gl.gl_mesh_destroy(m)


def test_debug_rejects_unknown_action():
    m = gl.gl_mesh_create(2, 8, 1.0)
    psi = torch.ones(64, dtype=torch.complex128, device=DEV)
    P = gl.gl_precond_setup(m, psi, gl.options())
    try:
        with pytest.raises(gl.GLError):
            gl.gl_precond_debug(P, 99)
    finally:
        gl.gl_precond_destroy(P)
        gl.gl_mesh_destroy(m)
