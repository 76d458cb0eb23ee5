"""The debug build (every index the kernels gather or scatter is checked)
decodes small cases of every row path with both kernels and records no
violation; its results equal the release build's.

The debug library is built and loaded in a child process
(QCMET_DEBUG_BUILD=1): one process loads one build of the library.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# cases: (name, code, frames, iterations, options); the codes take every row
# path: degree <= 4 rows (split, pipelined, paired), degree 5..16 (lane pairs),
# an empty row, an unconnected column, a degree-1 check, odd and even Z
CHILD = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2004_09084_gb300 as q
assert q.library_path().endswith("libqcmet_debug.so"), q.library_path()
out = {}
data = np.load(sys.argv[2], allow_pickle=True)
for key in sorted(k[:-5] for k in data.files if k.endswith("_base")):
    base, shifts, Z = data[key + "_base"], data[key + "_shifts"], int(data[key + "_Z"])
    llr, syn, T = data[key + "_llr"], data[key + "_syn"], int(data[key + "_T"])
    qc = q.Code(base, shifts, Z)
    d_llr, d_syn = torch.from_numpy(llr).cuda(), torch.from_numpy(syn).cuda()
    for kernel in ("frame", "group"):
        for msg in ("fp32", "fp16"):
            h, p, ok = q.decode(qc, d_llr, d_syn, T, kernel=kernel, msg=msg)
            torch.cuda.synchronize()
            out[f"{key}/{kernel}/{msg}"] = [int(q.debug_checks()), p.cpu().numpy().tolist()]
    h, p, ok, it = q.decode_early_stop(qc, d_llr, d_syn, T, 1)
    out[f"{key}/early"] = [int(q.debug_checks()), p.cpu().numpy().tolist()]
print(json.dumps(out))
"""


def cases():
    rng = np.random.default_rng(21)
    out = {}
    c = synth.make_code("0.1", 64)
    out["rate0.1_Z64"] = (c.base, c.shifts, 64)
    c = synth.make_code("0.05", 33)
    out["rate0.05_Z33"] = (c.base, c.shifts, 33)
    base = np.zeros((6, 18), np.int8)
    for l in range(6):
        base[l, rng.choice(18, int(rng.integers(1, 17)), replace=False)] = 1
    out["random_deg1_16_Z37"] = (base, np.where(base == 1, rng.integers(0, 37, base.shape), 0), 37)
    base = np.array([[1, 1, 1, 0, 1, 0], [1, 1, 0, 0, 0, 1], [0, 0, 0, 0, 0, 0],
                     [0, 0, 1, 0, 0, 0]], np.int8)
    out["degenerate_Z30"] = (base, np.where(base == 1, rng.integers(0, 30, base.shape), 0), 30)
    return out


def test_debug_build_checks_every_index_and_finds_none(q, tmp_path):
    arrays = {}
    expected = {}
    for key, (base, shifts, Z) in cases().items():
        code = synth.Code(base=np.asarray(base, np.int8), shifts=np.asarray(shifts, np.int32), Z=Z)
        rng = np.random.default_rng(len(key))
        x = rng.integers(0, 2, size=(6, code.n), dtype=np.uint8)
        llr = ((1.0 - 2.0 * x) * 1.5 + rng.normal(0, 1.5, size=x.shape)).astype(np.float32)
        syn = synth.syndrome(code, x)
        T = 4
        arrays.update({key + "_base": code.base, key + "_shifts": code.shifts, key + "_Z": Z,
                       key + "_llr": llr, key + "_syn": syn, key + "_T": T})
        qc = q.Code(code.base, code.shifts, code.Z)
        d_llr, d_syn = torch.from_numpy(llr).cuda(), torch.from_numpy(syn).cuda()
        for kernel in ("frame", "group"):
            for msg in ("fp32", "fp16"):
                _, p, _ = q.decode(qc, d_llr, d_syn, T, kernel=kernel, msg=msg)
                expected[f"{key}/{kernel}/{msg}"] = p.cpu().numpy()
        _, p, _, _ = q.decode_early_stop(qc, d_llr, d_syn, T, 1)
        expected[f"{key}/early"] = p.cpu().numpy()
    path = str(tmp_path / "cases.npz")
    np.savez(path, **arrays)
    env = dict(os.environ, QCMET_DEBUG_BUILD="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, path], capture_output=True, text=True,
                       env=env, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    assert set(got) == set(expected)
    for name, (bits, post) in got.items():
        assert bits == 0, f"{name}: index-check bits {bits:#x}"
        np.testing.assert_array_equal(np.asarray(post, np.float32), expected[name], err_msg=name)


NVTX_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_2004_09084_gb300 as q, synth
code = synth.make_code("0.1", 64)
fr = synth.make_frames(code, 6, 0.161)
qc = q.Code(code.base, code.shifts, code.Z)
_, p, _ = q.decode(qc, torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda(), 5)
np.save(sys.argv[2], p.cpu().numpy())
"""


def test_nvtx_ranges_change_no_result(q, tmp_path):
    # QCMET_NVTX=1 (read once per process) pushes host ranges around each call
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 6, 0.161)
    qc = q.Code(code.base, code.shifts, code.Z)
    _, p, _ = q.decode(qc, torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda(), 5)
    out = str(tmp_path / "p.npy")
    r = subprocess.run([sys.executable, "-c", NVTX_CHILD, ROOT, out], capture_output=True,
                       text=True, env=dict(os.environ, QCMET_NVTX="1"), timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    np.testing.assert_array_equal(np.load(out), p.cpu().numpy())


@pytest.fixture(scope="module")
def q():
    import paper_2004_09084_gb300 as q
    assert torch.cuda.is_available()
    return q
