"""Checkpoint / resume of a continuation state (host side, no GPU): the files
round-trip bit for bit, are little-endian regardless of the input's byte order,
and a wrong size is refused."""
import json
import os

import numpy as np
import pytest

from paper_1204_5125_gb300 import state


def test_round_trip(tmp_path):
    rng = np.random.default_rng(3)
    n = 5 ** 3
    psi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    params = rng.standard_normal(1000).astype(np.float32)
    pts = [{"mu": 0.0, "energy": -0.5}, {"mu": 0.1, "energy": -0.49}]
    state.save_state(str(tmp_path), dim=3, N=5, mu=0.1, psi=psi, edge=10.0, bhat=(0.0, 0.0, 1.0),
                     ws_params=params, points=pts)
    s = state.load_state(str(tmp_path))
    assert s["dim"] == 3 and s["N"] == 5 and s["edge"] == 10.0 and s["mu"] == 0.1
    assert np.array_equal(s["psi"], psi) and np.array_equal(s["params"], params)
    assert s["points"] == pts
    # the binary is little-endian complex128: re, im interleaved
    raw = np.fromfile(os.path.join(tmp_path, "psi.bin"), dtype="<f8")
    assert np.array_equal(raw[0::2], psi.real) and np.array_equal(raw[1::2], psi.imag)


def test_big_endian_input_is_written_little_endian(tmp_path):
    psi = np.arange(16, dtype=">c16") * (1 + 2j)
    state.save_state(str(tmp_path), dim=2, N=4, mu=0.3, psi=psi)
    s = state.load_state(str(tmp_path))
    assert np.array_equal(s["psi"], psi.astype(np.complex128)) and s["params"] is None


def test_wrong_sizes_are_refused(tmp_path):
    with pytest.raises(ValueError):
        state.save_state(str(tmp_path), dim=2, N=4, mu=0.0, psi=np.ones(15, complex))
    state.save_state(str(tmp_path), dim=2, N=4, mu=0.0, psi=np.ones(16, complex))
    with open(os.path.join(tmp_path, "meta.json")) as f:
        meta = json.load(f)
    meta["n"] = 17
    with open(os.path.join(tmp_path, "meta.json"), "w") as f:
        json.dump(meta, f)
    with pytest.raises(ValueError):
        state.load_state(str(tmp_path))
