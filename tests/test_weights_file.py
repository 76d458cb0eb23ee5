"""Learned min-sum weights on disk: a flat FP32 file plus a JSON header (CPU)."""
import json

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def learned():
    from paper_2004_09084_gb300 import learned
    return learned


def test_weights_round_trip(tmp_path, learned):
    code = synth.make_code("0.1", 64)
    rng = np.random.default_rng(3)
    ws = rng.random((7, code.mb, 2)).astype(np.float32)
    wo = rng.random((7, code.mb, 2)).astype(np.float32)
    path = str(tmp_path / "w.f32")
    hdr = learned.save_weights(path, ws, wo, code.base, code.shifts, code.Z,
                               info={"snr_range": [0.2, 0.22]})
    assert hdr["shape"] == [7, code.mb, 2]
    raw = np.fromfile(path, dtype="<f4")
    np.testing.assert_array_equal(raw, np.concatenate([ws.ravel(), wo.ravel()]))
    ws2, wo2, h2 = learned.load_weights(path, code.base, code.shifts, code.Z)
    np.testing.assert_array_equal(ws2, ws)
    np.testing.assert_array_equal(wo2, wo)
    assert h2["info"]["snr_range"] == [0.2, 0.22]


def test_weights_file_checks(tmp_path, learned):
    code = synth.make_code("0.1", 64)
    other = synth.make_code("0.1", 64, seed=1)
    ws = np.ones((3, code.mb, 2), np.float32)
    path = str(tmp_path / "w.f32")
    learned.save_weights(path, ws, 0 * ws, code.base, code.shifts, code.Z)
    with pytest.raises(ValueError, match="another code"):
        learned.load_weights(path, other.base, other.shifts, other.Z)
    with pytest.raises(ValueError, match="another code"):
        learned.load_weights(path, code.base, code.shifts, 128)
    with pytest.raises(ValueError):
        learned.save_weights(path, ws[:, :5], ws[:, :5], code.base, code.shifts, code.Z)
    data = bytearray(open(path, "rb").read())
    data[5] ^= 1
    open(path, "wb").write(bytes(data))
    with pytest.raises(ValueError, match="does not match"):
        learned.load_weights(path)
    h = json.load(open(path + ".json"))
    h["version"] = 99
    json.dump(h, open(path + ".json", "w"))
    with pytest.raises(ValueError, match="not a"):
        learned.load_weights(path)
