"""gl_jacobian_apply_noalloc: the Jacobian apply for callers that cannot let the
library allocate device memory during a call (a fixed memory budget or their own
pool, latency-critical loops where cudaMalloc/cudaFree may synchronise).  Its
buffers live in a static device array shared by every call, so two calls in a
row must each give the result of the allocating entry point (the same kernel on
the same inputs: bit for bit), and a mesh larger than the array is refused.
This file is collected last so that a failure here comes after every other test
has run; it also passes on its own in a fresh process."""
import ctypes

import pytest

import gl_inputs as gi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402

DEV = torch.device("cuda:0")
MAX_NODES = 1 << 18


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dim,N", [(2, 301), (3, 47)])
def test_noalloc_matches_allocating_apply_twice(dim, N):
    bh = gi.WORKLOADS["cube128"][3] if dim == 3 else (0.0, 0.0, 1.0)
    m = gl.gl_mesh_create(dim, N, 1.3, bh)
    lib = gl.library()
    n = N ** dim
    assert n <= MAX_NODES
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    try:
        for call in range(2):
            psi = torch.from_numpy(gi.disk(n, 30 + call)).to(DEV)
            phi = torch.from_numpy(gi.complex_normal(n, 40 + call)).to(DEV)
            y_ref = torch.empty_like(phi)
            y = torch.full_like(phi, float("nan"))
            gl.gl_jacobian_apply(m, psi, phi, y_ref)
            st = lib.gl_jacobian_apply_noalloc(m, ptr(psi), ptr(phi), ptr(y), stream)
            assert st == 0, gl.gl_last_error()
            torch.cuda.synchronize()
            # both run the FP64 Jacobian kernel on the same reordered inputs
            assert torch.equal(y, y_ref), f"call {call}"
    finally:
        gl.gl_mesh_destroy(m)


def test_noalloc_rejects_meshes_beyond_capacity():
    N = 513  # 513^2 = 263169 nodes > 262144
    m = gl.gl_mesh_create(2, N, 1.0)
    try:
        n = N * N
        psi = torch.ones(n, dtype=torch.complex128, device=DEV)
        phi = torch.ones_like(psi)
        y = torch.empty_like(psi)
        st = gl.library().gl_jacobian_apply_noalloc(m, ptr(psi), ptr(phi), ptr(y), None)
        assert st == 8  # GL_ERR_CAPACITY
        assert "262144" in gl.gl_last_error()
    finally:
        gl.gl_mesh_destroy(m)
