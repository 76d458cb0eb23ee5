"""qcmet_decode_noalloc: decoding for callers that cannot allocate device memory.

Some callers must not call cudaMalloc: a plug-in whose host application owns
all device memory through its own pool, or a pipeline that cannot accept the
device-wide synchronisation an allocation implies.  The entry point keeps its
scratch in a fixed array of device memory that the library defines, so such a
caller can still decode.  These tests call it through the C ABI:

* its results equal qcmet_decode's bit for bit (the same kernel on the same
  inputs), on two calls in a row, since every call reuses the same array;
* against the FP64 oracle, its posteriors over the first five iterations are
  within the tolerance of the other GPU parity tests;
* on a handle that never ran qcmet_decode it gives correct results and the
  device's free memory does not change across the call.

This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LLR_TOL = 1e-4   # the relative posterior tolerance of the other GPU parity tests


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


def _syndrome_ok(code, hard, syn):
    return np.all(synth.syndrome(code, hard) == syn, axis=1).astype(np.uint8)


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
        # the same kernel, launch shape and arithmetic: identical results
        np.testing.assert_array_equal(post, ref_post.cpu().numpy())
        np.testing.assert_array_equal(hard, ref_hard.cpu().numpy())
        np.testing.assert_array_equal(ok, ref_ok.cpu().numpy())
        np.testing.assert_array_equal(ok, _syndrome_ok(code, hard, fr.syn))


@pytest.mark.parametrize("T", [1, 3, 5])
def test_noalloc_matches_the_oracle(q, T):
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 8, 0.161, first=500)
    qc = q.Code(code.base, code.shifts, code.Z)
    out = _outputs(8, code.n)
    llr = torch.from_numpy(fr.llr).cuda()
    syn = torch.from_numpy(fr.syn).cuda()
    assert _noalloc(q, qc, llr, syn, T, out) == q.OK, q.lib.qcmet_last_error()
    torch.cuda.synchronize()
    hard, post, ok = (t.cpu().numpy() for t in out)
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T, nthreads=8)
    err = np.abs(post.astype(np.float64) - rp) / np.maximum(np.abs(rp), 1.0)
    assert err.max() <= LLR_TOL, f"T={T}: max relative LLR error {err.max():.3g}"
    np.testing.assert_array_equal(ok, _syndrome_ok(code, hard, fr.syn))


def test_noalloc_on_a_fresh_handle_allocates_nothing(q):
    code = synth.make_code("0.05", 40)
    fr = synth.make_frames(code, 5, 0.3, first=700)
    llr = torch.from_numpy(fr.llr).cuda()
    syn = torch.from_numpy(fr.syn).cuda()
    out = _outputs(5, code.n)
    # CUDA loads the library's device code (and with it the static array) at
    # the library's first launch on the device: let one call do that first
    warm = q.Code(code.base, code.shifts, code.Z)
    assert _noalloc(q, warm, llr, syn, 1, out) == q.OK, q.lib.qcmet_last_error()
    torch.cuda.synchronize()
    # a handle that never ran qcmet_decode: no device state of its own
    qc = q.Code(code.base, code.shifts, code.Z)
    torch_before = torch.cuda.memory_allocated()
    free_before, _ = torch.cuda.mem_get_info()
    assert _noalloc(q, qc, llr, syn, 6, out) == q.OK, q.lib.qcmet_last_error()
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == torch_before
    assert free_after == free_before, f"free device memory changed by {free_before - free_after} B"
    hard, post, ok = (t.cpu().numpy() for t in out)
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 6)
    err = np.abs(post.astype(np.float64) - rp) / np.maximum(np.abs(rp), 1.0)
    assert err.max() <= LLR_TOL
    np.testing.assert_array_equal(ok, _syndrome_ok(code, hard, fr.syn))
    # and the allocating entry point on the same handle afterwards agrees
    h2, p2, ok2 = q.decode(qc, llr, syn, 6)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(post, p2.cpu().numpy())
    np.testing.assert_array_equal(ok, ok2.cpu().numpy())


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
