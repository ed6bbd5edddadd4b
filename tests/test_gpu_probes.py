"""The measurement probes behind the rooflines: the FMA peaks (FP32 faster than
FP64 on this part) and the latencies that bound a phase of the coarse-level
sweeps (a release/acquire hand-off between CTAs on different SMs, a dependent L2
load, a store followed by a GPU-scope fence).  Checked for plausibility: finite,
positive, ordered, and far below the 1 s bound of every wait."""
import math

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_1204_5125_gb300 as gl  # noqa: E402


def test_fma_peaks():
    f64 = gl.gl_measure_fma_peak(gl.GL_FP64)
    f32 = gl.gl_measure_fma_peak(gl.GL_MIXED)
    print(f"FMA peaks: FP64 {f64:.0f} GFLOP/s, FP32 {f32:.0f} GFLOP/s")
    assert math.isfinite(f64) and math.isfinite(f32) and 0 < f64 < f32


def test_sync_latency():
    lat = gl.gl_measure_sync_latency()
    print("latencies (ns):", {k: round(v, 1) for k, v in lat.items()})
    for v in lat.values():
        assert math.isfinite(v) and v > 0
    assert lat["handoff_ns"] <= lat["handoff_max_ns"] < 1e5
    assert lat["l2_load_ns"] < 1e4 and lat["fence_ns"] < 1e5
