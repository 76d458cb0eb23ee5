"""GPU parity: the CUDA decoder (through the C ABI) against the FP64 oracle.

Bars (the FP32 decoder): posterior LLRs within 1e-4 * max(|L_ref|, 1) over
iterations 1-5; the ok flag equal to [H c = s] recomputed from the GPU's own
hard decisions; at 50 iterations at least 99.99% of hard decisions and 99% of
frame outcomes equal to the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth
from tests import helpers

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LLR_TOL = 1e-4


@pytest.fixture(scope="module")
def q():
    from paper_2004_09084_gb300 import build
    build.build()
    import paper_2004_09084_gb300 as q
    assert torch.cuda.is_available()
    return q


def gpu_decode(q, code, llr, syn, T, merge="exact", msg="fp32", threads=0, want_post=True,
               kernel="auto"):
    qc = code if isinstance(code, q.Code) else q.Code(code.base, code.shifts, code.Z, merge=merge)
    d_llr = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    d_syn = torch.from_numpy(np.ascontiguousarray(syn)).cuda()
    h, p, ok = q.decode(qc, d_llr, d_syn, T, msg=msg, threads=threads, want_post=want_post,
                        kernel=kernel)
    torch.cuda.synchronize()
    return h.cpu().numpy(), (p.cpu().numpy() if p is not None else None), ok.cpu().numpy()


def rel_err(a, ref):
    return np.abs(a.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1.0)


def syndrome_ok(code, hard, syn):
    return np.all(synth.syndrome(code, hard) == syn, axis=1).astype(np.uint8)


# --------------------------------------------------------------------------
# Small workload: rate 0.1, Z = 64, SNR 0.161

@pytest.fixture(scope="module")
def small():
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 16, 0.161)
    return code, fr


@pytest.mark.parametrize("kernel", ["frame", "group"])
@pytest.mark.parametrize("T", [1, 2, 3, 4, 5])
def test_llr_parity_first_five_iterations(q, small, T, kernel):
    code, fr = small
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, T, kernel=kernel)
    rh, rp, rok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T, nthreads=8)
    err = rel_err(p, rp)
    assert err.max() <= LLR_TOL, f"max relative LLR error {err.max():.3g}"
    confident = np.abs(rp) > 1e-3
    np.testing.assert_array_equal(h[confident], rh[confident])
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))


@pytest.mark.parametrize("kernel", ["frame", "group"])
def test_fifty_iterations_hard_decisions_and_frame_outcomes(q, small, kernel):
    code, fr = small
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 50, kernel=kernel)
    rh, rp, rok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 50, nthreads=8)
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))     # bit-exact flag
    agree = np.mean(h == rh)
    assert agree >= 0.9999, f"hard-decision agreement {agree:.6f}"
    assert np.mean(ok == rok) >= 0.99


def test_noiseless_frames_decode(q):
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 4, 0.161, noiseless=True)
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 1)
    np.testing.assert_array_equal(h, fr.x)
    np.testing.assert_array_equal(ok, np.ones(4, np.uint8))


def test_zero_iterations_return_the_channel(q, small):
    code, fr = small
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 0)
    np.testing.assert_array_equal(p, fr.llr)
    np.testing.assert_array_equal(h, (fr.llr < 0).astype(np.uint8))
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))


def test_coset_symmetry_is_exact_on_gpu(q, small):
    code, fr = small
    rng = np.random.default_rng(4)
    x0 = rng.integers(0, 2, size=fr.x.shape, dtype=np.uint8)
    flip = (1.0 - 2.0 * x0).astype(np.float32)
    _, p, _ = gpu_decode(q, code, fr.llr, fr.syn, 7)
    _, p2, _ = gpu_decode(q, code, fr.llr * flip, fr.syn ^ synth.syndrome(code, x0), 7)
    np.testing.assert_array_equal(p2, p * flip)


# --------------------------------------------------------------------------
# Several thread-block passes with a ragged tail; more frames than SMs

def test_parity_with_ragged_z(q):
    code = synth.make_code("0.1", 2500)     # the paper's expansion factor; 2500 = 2 * 1024 + 452
    fr = synth.make_frames(code, 3, 0.161)
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 3)
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 3, nthreads=3)
    assert rel_err(p, rp).max() <= LLR_TOL


def test_more_frames_than_ctas(q):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    code = synth.make_code("0.1", 8)
    fr = synth.make_frames(code, sms + 9, 0.161)
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 4)
    rh, rp, rok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 4, nthreads=8)
    assert rel_err(p, rp).max() <= LLR_TOL
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))


@pytest.mark.parametrize("threads", [32, 96, 256, 1024])
def test_block_size_does_not_change_results(q, small, threads):
    # the frame kernel's block size (the grouped kernel sizes its own blocks)
    code, fr = small
    ref = gpu_decode(q, code, fr.llr, fr.syn, 5, kernel="frame")
    got = gpu_decode(q, code, fr.llr, fr.syn, 5, threads=threads, kernel="frame")
    for a, b in zip(ref, got):
        np.testing.assert_array_equal(a, b)


# --------------------------------------------------------------------------
# Code shapes: high-degree rows (lane-pair path), degenerate blocks

def random_code(seed, mb, nb, Z, min_deg, max_deg):
    rng = np.random.default_rng(seed)
    base = np.zeros((mb, nb), np.int8)
    for l in range(mb):
        d = int(rng.integers(min_deg, max_deg + 1))
        base[l, rng.choice(nb, d, replace=False)] = 1
    shifts = np.where(base == 1, rng.integers(0, Z, size=base.shape), 0).astype(np.int32)
    return synth.Code(base=base, shifts=shifts, Z=Z)


@pytest.mark.parametrize("seed,lo,hi", [(0, 9, 12), (1, 13, 16), (2, 1, 16), (3, 2, 8)])
def test_parity_for_row_degrees_up_to_the_limit(q, seed, lo, hi):
    code = random_code(seed, 6, 18, 37, lo, hi)
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 2, size=(3, code.n), dtype=np.uint8)
    llr = ((1.0 - 2.0 * x) * 2.0 + rng.normal(0, 2.0, size=x.shape)).astype(np.float32)
    syn = synth.syndrome(code, x)
    for merge in ("none", "exact"):
        h, p, ok = gpu_decode(q, code, llr, syn, 3, merge=merge)
        _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, llr, syn, 3)
        assert rel_err(p, rp).max() <= LLR_TOL
        np.testing.assert_array_equal(ok, syndrome_ok(code, h, syn))


def test_degenerate_blocks(q):
    # column 3 unconnected, row 2 empty (its checks only test s_m), row 3 a
    # single circulant (degree-1 check), columns 4 and 5 of degree one
    base = np.array([[1, 1, 1, 0, 1, 0],
                     [1, 1, 0, 0, 0, 1],
                     [0, 0, 0, 0, 0, 0],
                     [0, 0, 1, 0, 0, 0]], np.int8)
    Z = 33
    rng = np.random.default_rng(8)
    shifts = np.where(base == 1, rng.integers(0, Z, size=base.shape), 0).astype(np.int32)
    code = synth.Code(base=base, shifts=shifts, Z=Z)
    x = rng.integers(0, 2, size=(2, code.n), dtype=np.uint8)
    llr = ((1.0 - 2.0 * x) + rng.normal(0, 1.0, size=x.shape)).astype(np.float32)
    syn = synth.syndrome(code, x)
    syn[1, 2 * Z + 5] ^= 1          # an empty check with s_m = 1 can never be satisfied
    for T in (0, 1, 4):
        h, p, ok = gpu_decode(q, code, llr, syn, T)
        rh, rp, rok = oracle.decode(base, shifts, Z, llr, syn, T)
        assert rel_err(p, rp).max() <= LLR_TOL
        np.testing.assert_array_equal(ok, syndrome_ok(code, h, syn))
        assert ok[1] == 0
        np.testing.assert_array_equal(p[:, 3 * Z:4 * Z], llr[:, 3 * Z:4 * Z])


# --------------------------------------------------------------------------
# Schedules (Results, Eqs. (m)-(m2))

def test_exact_merge_is_bit_identical_to_base_order(q, small):
    code, fr = small
    a = gpu_decode(q, code, fr.llr, fr.syn, 6, merge="none")
    b = gpu_decode(q, code, fr.llr, fr.syn, 6, merge="exact")
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_greedy_merge_matches_the_oracle_in_the_same_order(q, small):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z, merge="greedy")
    rows, layers = qc.schedule()
    assert len(layers) < 54
    h, p, ok = gpu_decode(q, qc, fr.llr, fr.syn, 4)
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 4, order=rows,
                             nthreads=8)
    assert rel_err(p, rp).max() <= LLR_TOL


# --------------------------------------------------------------------------
# Entry points and error paths

def test_without_llr_post_the_outputs_are_unchanged(q, small):
    code, fr = small
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 5)
    h2, p2, ok2 = gpu_decode(q, code, fr.llr, fr.syn, 5, want_post=False)
    assert p2 is None
    np.testing.assert_array_equal(h, h2)
    np.testing.assert_array_equal(ok, ok2)


def test_host_entry_point_matches_device_entry_point(q, small):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok = gpu_decode(q, qc, fr.llr, fr.syn, 5)
    h2, p2, ok2 = q.decode_host(qc, fr.llr, fr.syn, 5)
    np.testing.assert_array_equal(h, h2)
    np.testing.assert_array_equal(p, p2)
    np.testing.assert_array_equal(ok, ok2)
    h3, p3, ok3 = q.decode_host(qc, fr.llr, fr.syn, 5, want_post=False)
    assert p3 is None
    np.testing.assert_array_equal(h, h3)


def test_misaligned_pointer_is_rejected(q, small):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    buf = torch.from_numpy(np.concatenate([np.zeros(1, np.float32), fr.llr[0]])).cuda()
    syn = torch.from_numpy(fr.syn[:1]).cuda()
    hard = torch.empty((1, code.n), dtype=torch.uint8, device="cuda")
    ok = torch.empty((1,), dtype=torch.uint8, device="cuda")
    st = q.lib.qcmet_decode(qc.handle, buf.data_ptr() + 4, syn.data_ptr(), 1, 3,
                            hard.data_ptr(), None, ok.data_ptr(), None)
    assert st == q.ERR_ALIGNMENT
    assert b"aligned" in q.lib.qcmet_last_error()


def test_invalid_sizes_are_rejected(q, small):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    d = torch.zeros((1, code.n), dtype=torch.float32, device="cuda")
    s = torch.zeros((1, code.m), dtype=torch.uint8, device="cuda")
    h = torch.zeros((1, code.n), dtype=torch.uint8, device="cuda")
    o = torch.zeros((1,), dtype=torch.uint8, device="cuda")
    args = (qc.handle, d.data_ptr(), s.data_ptr())
    assert q.lib.qcmet_decode(*args, -1, 3, h.data_ptr(), None, o.data_ptr(), None) == q.ERR_INVALID_ARG
    assert q.lib.qcmet_decode(*args, 1, -1, h.data_ptr(), None, o.data_ptr(), None) == q.ERR_INVALID_ARG
    assert q.lib.qcmet_decode(*args, 0, 3, None, None, None, None) == q.OK      # K = 0: no-op
    with pytest.raises(q.QcmetError):
        q.decode(qc, d, s, 3, threads=48)


# --------------------------------------------------------------------------
# Full size: Z = 12500 (n = 10^6), 128 frames, the configuration bench.py times

@pytest.fixture(scope="module")
def full():
    code = synth.make_code("0.1", 12500)
    fr = synth.make_frames(code, 128, 0.161)
    return code, fr


def test_full_size_llr_parity_on_sampled_frames(q, full):
    code, fr = full
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 2)
    pick = [0, 77]
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr[pick], fr.syn[pick], 2,
                             nthreads=2)
    assert rel_err(p[pick], rp).max() <= LLR_TOL


def test_full_size_fixed_iterations_properties(q, full):
    code, fr = full
    h, p, ok = gpu_decode(q, code, fr.llr, fr.syn, 100)
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))
    np.testing.assert_array_equal(h, (p < 0).astype(np.uint8))
    assert np.all(np.isfinite(p))
    # decoding a coset-shifted copy negates exactly the shifted posteriors
    x0 = fr.x[::-1].copy()
    flip = (1.0 - 2.0 * x0).astype(np.float32)
    _, p2, ok2 = gpu_decode(q, code, fr.llr * flip, fr.syn ^ synth.syndrome(code, x0), 100)
    # exact up to a q that is exactly 0 (its check then sends +-Phi(30) ~ 2e-13 either way)
    np.testing.assert_allclose(p2, p * flip, rtol=1.2e-7, atol=1e-9)
    np.testing.assert_array_equal(ok2, ok)


def test_host_entry_point_at_full_size(q, full):
    # the host-buffer entry point at the bench size equals the device entry point
    code, fr = full
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok = q.decode(qc, torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda(), 3)
    torch.cuda.synchronize()
    h2, p2, ok2 = q.decode_host(qc, fr.llr, fr.syn, 3)
    np.testing.assert_array_equal(h2, h.cpu().numpy())
    np.testing.assert_array_equal(p2, p.cpu().numpy())
    np.testing.assert_array_equal(ok2, ok.cpu().numpy())
    h3, p3, ok3 = q.decode_host(qc, fr.llr, fr.syn, 3, want_post=False, l2_persist=True)
    assert p3 is None
    np.testing.assert_array_equal(h3, h2)
    np.testing.assert_array_equal(ok3, ok2)


def test_block_size_does_not_change_results_at_full_size(q, full):
    # one warp per frame against the default 1024 threads: per check the
    # arithmetic is the same, so the results are identical
    code, fr = full
    qc = q.Code(code.base, code.shifts, code.Z)
    d_llr = torch.from_numpy(fr.llr[:6]).cuda()
    d_syn = torch.from_numpy(fr.syn[:6]).cuda()
    h, p, ok = q.decode(qc, d_llr, d_syn, 3, threads=1024, kernel="frame")
    h2, p2, ok2 = q.decode(qc, d_llr, d_syn, 3, threads=32, kernel="frame")
    torch.cuda.synchronize()
    assert torch.equal(p, p2) and torch.equal(h, h2) and torch.equal(ok, ok2)


def test_l2_persist_window_changes_no_result(q, full):
    # the option only attaches an L2 access-policy window to the launch
    code, fr = full
    qc = q.Code(code.base, code.shifts, code.Z)
    d_llr = torch.from_numpy(fr.llr[:40]).cuda()
    d_syn = torch.from_numpy(fr.syn[:40]).cuda()
    h, p, ok = q.decode(qc, d_llr, d_syn, 6, kernel="frame")
    h2, p2, ok2 = q.decode(qc, d_llr, d_syn, 6, l2_persist=True, kernel="frame")
    torch.cuda.synchronize()
    assert torch.equal(h, h2) and torch.equal(p, p2) and torch.equal(ok, ok2)
    # the grouped kernel accepts and ignores the option; its results are the same
    h4, p4, ok4 = q.decode(qc, d_llr, d_syn, 6, l2_persist=True, kernel="group")
    torch.cuda.synchronize()
    assert torch.equal(h, h4) and torch.equal(p, p4) and torch.equal(ok, ok4)
    h3, p3, ok3 = q.decode_host(qc, fr.llr[:3], fr.syn[:3], 6, l2_persist=True)
    np.testing.assert_array_equal(h3, h[:3].cpu().numpy())
    np.testing.assert_array_equal(p3, p[:3].cpu().numpy())


def _persisting_l2_limit():
    # the context's cudaLimitPersistingL2CacheSize, read through the CUDA runtime
    import ctypes
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so.13"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    else:
        pytest.skip("CUDA runtime library not found")
    v = ctypes.c_size_t(0)
    assert rt.cudaDeviceGetLimit(ctypes.byref(v), 0x06) == 0  # cudaLimitPersistingL2CacheSize
    return v.value


def test_windowed_decode_gives_l2_back_to_later_decodes(q, full):
    # A frame-kernel decode under the persisting window raises the context's
    # persisting-L2 limit; the next decode without a window puts it back, so
    # the part of L2 set aside does not stay lost to the grouped kernel (with
    # it set aside, grouped decodes of these frames ran about a quarter slower).
    code, fr = full
    qc = q.Code(code.base, code.shifts, code.Z)
    d_llr = torch.from_numpy(fr.llr).cuda()
    d_syn = torch.from_numpy(fr.syn).cuda()
    q.decode(qc, d_llr, d_syn, 2, kernel="group")
    torch.cuda.synchronize()
    before = _persisting_l2_limit()
    h, p, ok = q.decode(qc, d_llr, d_syn, 2, l2_persist=True, kernel="frame")
    torch.cuda.synchronize()
    assert _persisting_l2_limit() >= before
    h2, p2, ok2 = q.decode(qc, d_llr, d_syn, 2, kernel="group")
    torch.cuda.synchronize()
    # back to the value found (the driver keeps the limit in steps of a few KiB)
    assert abs(_persisting_l2_limit() - before) <= 1 << 20
    assert torch.equal(h, h2) and torch.equal(p, p2) and torch.equal(ok, ok2)


def test_maximum_size_frames(q):
    # The largest frame the boundary accepts, n = 4 Z = 2^31 - 4 (Z = 2^29 - 1,
    # odd, so rows end in a ragged pass), two frames so that frame offsets pass
    # 2^31 elements, one core-and-degree-1 row and one all-core row.  After one
    # layered iteration a posterior depends only on its depth-2 neighbourhood,
    # so sampled posteriors are recomputed exactly with the oracle's check
    # rule; the ok flags are checked against H c = s recomputed with torch.
    Z = (1 << 29) - 1
    base = np.array([[1, 1, 1, 1], [1, 0, 1, 1]], dtype=np.int8)
    rng = np.random.default_rng(11)
    shifts = (rng.integers(0, Z, size=base.shape) * base).astype(np.int32)
    shifts[0, 2] = Z - 1                     # a shift that wraps at once
    K, n, m = 2, 4 * Z, 2 * Z
    qc = q.Code(base, shifts, Z)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    llr = torch.randn((K, n), generator=gen, device="cuda")
    syn = torch.randint(0, 2, (K, m), generator=gen, device="cuda", dtype=torch.uint8)
    # frame 1: a codeword x with s = H x, received strongly, so that it decodes (ok = 1)
    x = torch.randint(0, 2, (n,), generator=gen, device="cuda", dtype=torch.uint8)
    xv = x.view(4, Z)
    for l in range(2):
        acc = torch.zeros(Z, dtype=torch.uint8, device="cuda")
        for c in range(4):
            if base[l, c]:
                acc ^= torch.roll(xv[c], -int(shifts[l, c]))
        syn[1, l * Z:(l + 1) * Z] = acc
    llr[1] = 4.0 * (1.0 - 2.0 * x.float()) + 0.5 * llr[1]
    del x, xv, acc
    hard, post, ok = q.decode(qc, llr, syn, 1)
    torch.cuda.synchronize()
    assert int(ok[1]) == 1

    # H c = s per frame, from the GPU's hard decisions (torch ops, not the decoder)
    for f in range(K):
        hv = hard[f].view(4, Z)
        good = True
        for l in range(2):
            acc = syn[f, l * Z:(l + 1) * Z].clone()
            for c in range(4):
                if base[l, c]:
                    acc ^= torch.roll(hv[c], -int(shifts[l, c]))
            good = good and not bool(acc.any())
        assert int(ok[f]) == int(good)
        del hv

    def ch(f, c, j):
        return float(llr[f, c * Z + j])

    def row_msgs(f, l, i, L):
        # messages of check (l, i) given the posteriors L(c, j) of its variables
        cols = [c for c in range(4) if base[l, c]]
        js = [(i + int(shifts[l, c])) % Z for c in cols]
        qv = np.array([L(c, j) for c, j in zip(cols, js)])
        r = oracle.check_update(qv, int(syn[f, l * Z + i]) & 1)
        return dict(zip(zip(cols, js), qv + r))

    def after_row0(f, c, j):
        if not base[0, c]:
            return ch(f, c, j)
        i0 = (j - int(shifts[0, c])) % Z
        return row_msgs(f, 0, i0, lambda cc, jj: ch(f, cc, jj))[(c, j)]

    def after_row1(f, c, j):
        if not base[1, c]:
            return after_row0(f, c, j)
        i1 = (j - int(shifts[1, c])) % Z
        return row_msgs(f, 1, i1, lambda cc, jj: after_row0(f, cc, jj))[(c, j)]

    picks = [(c, j) for c in range(4) for j in (0, 1, Z - 2, Z - 1)]
    picks += [(int(c), int(j)) for c, j in zip(rng.integers(0, 4, 48), rng.integers(0, Z, 48))]
    for f in range(K):
        for c, j in picks:
            want = after_row1(f, c, j)
            got = float(post[f, c * Z + j])
            assert abs(got - want) <= 1e-4 * max(abs(want), 1.0), (f, c, j, got, want)
            assert int(hard[f, c * Z + j]) == int(got < 0.0)
    del llr, syn, hard, post, ok
    torch.cuda.empty_cache()


# --------------------------------------------------------------------------
# Early termination (Discussion, Table tabearly)

@pytest.fixture(scope="module")
def converging():
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 24, 0.3)       # most frames decode within a few iterations
    return code, fr


@pytest.mark.parametrize("every", [1, 4])
def test_early_stop_matches_the_oracle(q, converging, every):
    code, fr = converging
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok, it = q.decode_early_stop(qc, torch.from_numpy(fr.llr).cuda(),
                                       torch.from_numpy(fr.syn).cuda(), 30, every)
    torch.cuda.synchronize()
    h, p, ok, it = h.cpu().numpy(), p.cpu().numpy(), ok.cpu().numpy(), it.cpu().numpy()
    rh, rp, rok, rit = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 30,
                                     early_every=every, return_iters=True, nthreads=8)
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))
    same = it == rit
    assert np.mean(same) >= 0.95 and np.any(it < 30)
    assert rel_err(p[same], rp[same]).max() <= 10 * LLR_TOL
    assert np.all((it % every == 0) | (it == 30))


def test_early_stop_equals_a_fixed_decode_of_that_many_iterations(q, converging):
    code, fr = converging
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok, it = q.decode_early_stop(qc, torch.from_numpy(fr.llr).cuda(),
                                       torch.from_numpy(fr.syn).cuda(), 25, 2)
    torch.cuda.synchronize()
    p, ok, it = p.cpu().numpy(), ok.cpu().numpy(), it.cpu().numpy()
    for T in sorted(set(it.tolist())):
        sel = np.flatnonzero(it == T)
        hh, pp, oo = gpu_decode(q, qc, fr.llr[sel], fr.syn[sel], int(T))
        np.testing.assert_array_equal(p[sel], pp)
        np.testing.assert_array_equal(ok[sel], oo)
        if T < 25:
            assert np.all(oo == 1)


def test_early_stop_arguments(q, small):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    d = torch.zeros((1, code.n), dtype=torch.float32, device="cuda")
    s = torch.zeros((1, code.m), dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QcmetError):
        q.decode_early_stop(qc, d, s, 10, 0)
    h, p, ok, it = q.decode_early_stop(qc, d[:1] + 1.0, s, 0, 1)   # no iteration: channel decision
    torch.cuda.synchronize()
    assert it.item() == 0 and ok.item() == 1


# --------------------------------------------------------------------------
# 16-bit message storage (FP32 arithmetic and posteriors)
#
# The oracle rounds every stored message to the same format (IEEE round to
# nearest even).  FP32 and FP64 messages can straddle a rounding midpoint, so
# a stored message may differ by one unit in the last place of the 16-bit
# format, about 2^(1-p) |r| for a p-bit significand; such differences add up
# over iterations.  Bound: T * 2^(2-p) relative (floor 1).

@pytest.mark.parametrize("kernel", ["frame", "group"])
@pytest.mark.parametrize("msg,p,fmt", [("fp16", 11, oracle.MSG_FP16), ("bf16", 8, oracle.MSG_BF16)])
def test_16bit_messages_match_the_oracle_with_rounded_messages(q, small, msg, p, fmt, kernel):
    code, fr = small
    for T in (1, 3, 5):
        h, pg, ok = gpu_decode(q, code, fr.llr, fr.syn, T, msg=msg, kernel=kernel)
        _, rp, rok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T,
                                   msg_fmt=fmt, nthreads=8)
        err = rel_err(pg, rp)
        assert err.max() <= T * 2.0 ** (2 - p), f"T={T}: {err.max():.3g}"
        assert np.mean(h == (rp < 0)) >= 0.999
        np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))


# Frame outcomes of the 16-bit formats against the oracle (with messages rounded
# the same way) at an SNR where about half of the frames decode:
# test_gpu_oracle_outcomes.py.
