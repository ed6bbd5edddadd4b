"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
entry point declared in include/gl.h (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "gl.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"GL_API\s+(?:gl_status|const char \*)\s*(gl_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("gl_mesh_create", "gl_residual", "gl_jacobian_apply", "gl_precond_setup", "gl_precond_apply",
                 "gl_jacobian_solve", "gl_newton_step", "gl_batch_solve", "gl_last_error"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    from paper_1204_5125_gb300 import EXPORTED, build

    path = build.build()
    lib = ctypes.CDLL(path)
    syms = declared_symbols()
    assert sorted(EXPORTED) == syms, "binding and header disagree"
    for name in syms:
        assert hasattr(lib, name), name


def test_options_default_and_errors_without_gpu():
    """Calls that touch no device memory work on a CPU-only host."""
    import paper_1204_5125_gb300 as gl

    o = gl.gl_options_default()
    assert o.tol == 1e-10 and o.cycles == 1 and o.max_coarse == 512 and o.precision == gl.GL_FP64
    lib = gl.library()
    assert lib.gl_mesh_destroy(None) == 0
    assert lib.gl_precond_levels(None, None) == 1  # GL_ERR_ARG
    assert "NULL" in gl.gl_last_error()
