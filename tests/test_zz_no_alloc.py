"""qcmet_decode_noalloc: decoding for callers that cannot allocate device memory.

The entry point keeps its scratch in a fixed array of device memory that the
library defines, so a caller that must not call cudaMalloc (for instance one
whose host application owns all device memory) can still decode.  These tests
call it through the C ABI and compare it with qcmet_decode on the same inputs,
twice in a row, since every call reuses the same array.

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LLR_TOL = 1e-4   # the relative posterior tolerance of the other GPU tests


@pytest.fixture(scope="module")
def q():
    import paper_2004_09084_gb300 as q
    assert torch.cuda.is_available()
    return q


def _outputs(K, n):
    return (torch.empty((K, n), dtype=torch.uint8, device="cuda"),
            torch.empty((K, n), dtype=torch.float32, device="cuda"),
            torch.empty((K,), dtype=torch.uint8, device="cuda"))


def _noalloc(q, qc, llr, syn, T, out):
    hard, post, ok = out
    stream = torch.cuda.current_stream().cuda_stream
    return q.lib.qcmet_decode_noalloc(qc.handle, llr.data_ptr(), syn.data_ptr(), llr.shape[0], T,
                                      hard.data_ptr(), post.data_ptr(), ok.data_ptr(), stream)


@pytest.mark.parametrize("Z,K,T", [(64, 16, 20), (12500, 2, 3)])
def test_noalloc_matches_the_allocating_entry_point_twice_in_a_row(q, Z, K, T):
    code = synth.make_code("0.1", Z)
    qc = q.Code(code.base, code.shifts, code.Z)
    for call in range(2):
        fr = synth.make_frames(code, K, 0.161, first=100 * call)
        llr = torch.from_numpy(fr.llr).cuda()
        syn = torch.from_numpy(fr.syn).cuda()
        ref_hard, ref_post, ref_ok = q.decode(qc, llr, syn, T)
        out = _outputs(K, code.n)
        assert _noalloc(q, qc, llr, syn, T, out) == q.OK, q.lib.qcmet_last_error()
        torch.cuda.synchronize()
        hard, post, ok = (t.cpu().numpy() for t in out)
        rp = ref_post.cpu().numpy().astype(np.float64)
        err = np.abs(post.astype(np.float64) - rp) / np.maximum(np.abs(rp), 1.0)
        assert err.max() <= LLR_TOL, f"call {call}: max relative LLR difference {err.max():.3g}"
        np.testing.assert_array_equal(hard, ref_hard.cpu().numpy())
        np.testing.assert_array_equal(ok, ref_ok.cpu().numpy())


def test_noalloc_rejects_work_beyond_its_scratch(q):
    code = synth.make_code("0.1", 12500)
    qc = q.Code(code.base, code.shifts, code.Z)
    K = 3   # 3 x 230 slots x 12512 x 4 B exceeds the 32 MiB array
    llr = torch.zeros((K, code.n), dtype=torch.float32, device="cuda")
    syn = torch.zeros((K, code.m), dtype=torch.uint8, device="cuda")
    out = _outputs(K, code.n)
    assert _noalloc(q, qc, llr, syn, 2, out) == q.ERR_INVALID_ARG
    msg = q.lib.qcmet_last_error().decode()
    assert "bytes" in msg and "qcmet_decode_noalloc" in msg


def test_noalloc_requires_llr_post(q):
    code = synth.make_code("0.1", 64)
    qc = q.Code(code.base, code.shifts, code.Z)
    llr = torch.zeros((1, code.n), dtype=torch.float32, device="cuda")
    syn = torch.zeros((1, code.m), dtype=torch.uint8, device="cuda")
    hard, _, ok = _outputs(1, code.n)
    st = q.lib.qcmet_decode_noalloc(qc.handle, llr.data_ptr(), syn.data_ptr(), 1, 2,
                                    hard.data_ptr(), None, ok.data_ptr(), None)
    assert st == q.ERR_INVALID_ARG
