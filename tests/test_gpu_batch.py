"""Mixed batches: frames of several codes in one graph-captured launch.

Every candidate configuration the autotuner may choose gives the same
arithmetic per frame, so a batch must reproduce, bit for bit, the decode of
each frame with its own code through qcmet_decode.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_2004_09084_gb300 as q
    assert torch.cuda.is_available()
    return q


def mixed(q, counts):
    """counts: list of (rate, Z, frames) -> list of (qcode, llr[n], syn[m], x) per frame."""
    out = []
    for j, (rate, Z, K) in enumerate(counts):
        code = synth.make_code(rate, Z)
        qc = q.Code(code.base, code.shifts, code.Z)
        fr = synth.make_frames(code, K, synth.RATE_SNR[rate] + 0.1, first=1000 * j)
        for k in range(K):
            out.append((qc, torch.from_numpy(fr.llr[k]).cuda(), torch.from_numpy(fr.syn[k]).cuda(),
                        fr.x[k]))
    order = np.random.default_rng(5).permutation(len(out))   # interleave the codes
    return [out[i] for i in order]


@pytest.mark.parametrize("msg", ["fp32", "fp16"])
@pytest.mark.parametrize("autotune", [0, 1, 2])
def test_batch_equals_per_code_decoding(q, msg, autotune):
    frames = mixed(q, [("0.1", 40, 5), ("0.05", 64, 4), ("0.02", 16, 6), ("0.1", 128, 3)])
    T = 12
    b = q.Batch([(c, l, s) for c, l, s, _ in frames], T, msg=msg, autotune=autotune)
    b.run()
    torch.cuda.synchronize()
    cfg = b.config()
    # autotuned: frame kernel (2 block sizes) and grouped kernel (5 cluster
    # sizes), each x 2 schedules x 2 orders, and one concurrent launch per code
    # x 2 schedules; 0: the grouped kernel, clusters of 4; 2: one launch per code
    assert cfg["candidates"] == {0: 1, 1: 30, 2: 1}[autotune]
    assert cfg["kernel"] in (1, 2)
    if autotune == 0:
        assert cfg["kernel"] == 2 and cfg["cluster_size"] == 4 and cfg["per_code_launches"] == 0
    if autotune == 2:
        assert cfg["kernel"] == 2 and cfg["per_code_launches"] == 4
    for k, (qc, llr, syn, x) in enumerate(frames):
        h, p, ok = q.decode(qc, llr[None].contiguous(), syn[None].contiguous(), T, msg=msg)
        torch.cuda.synchronize()
        assert torch.equal(b.hard[k], h[0]), k
        assert torch.equal(b.post[k], p[0]), k
        assert b.ok[k][0].item() == ok[0].item()


def test_batch_replays_and_sees_new_inputs(q):
    frames = mixed(q, [("0.1", 64, 3), ("0.05", 32, 3)])
    T = 8
    b = q.Batch([(c, l, s) for c, l, s, _ in frames], T, autotune=False)
    b.run()
    torch.cuda.synchronize()
    first = [p.clone() for p in b.post]
    b.run()
    torch.cuda.synchronize()
    for a, c in zip(first, b.post):
        assert torch.equal(a, c)
    # new data in the same input buffers
    for qc, llr, syn, _ in frames:
        llr.neg_()
    b.run()
    torch.cuda.synchronize()
    for k, (qc, llr, syn, x) in enumerate(frames):
        _, p, _ = q.decode(qc, llr[None].contiguous(), syn[None].contiguous(), T)
        torch.cuda.synchronize()
        assert torch.equal(b.post[k], p[0])


def test_batch_arguments(q):
    import ctypes
    h = ctypes.c_void_p()
    assert q.lib.qcmet_batch_create(None, 0, 5, 0, 0, None, ctypes.byref(h)) == q.ERR_INVALID_ARG
    arr = (q.Frame * 1)()
    assert q.lib.qcmet_batch_create(arr, 1, 5, 0, 0, None, ctypes.byref(h)) == q.ERR_INVALID_ARG
    q.lib.qcmet_batch_destroy(None)
