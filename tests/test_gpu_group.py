"""The grouped decode kernel (frames interleaved four at a time, a cluster of
thread blocks per group) against the FP64 oracle and against the per-frame
kernel.

Both kernels evaluate the same arithmetic per check and frame in the same
order, so their results must be identical bit for bit, whatever the cluster
size, frame count (including a partial last group) or message format; against
the oracle the bars of the other parity tests apply (posteriors within
1e-4 * max(|L|, 1) over iterations 1-5, ok = [H c = s] exactly).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LLR_TOL = 1e-4


@pytest.fixture(scope="module")
def q():
    import paper_2004_09084_gb300 as q
    assert torch.cuda.is_available()
    return q


def run(q, qc, llr, syn, T, **kw):
    h, p, ok = q.decode(qc, torch.from_numpy(np.ascontiguousarray(llr)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(syn)).cuda(), T, **kw)
    torch.cuda.synchronize()
    return h.cpu().numpy(), (p.cpu().numpy() if p is not None else None), ok.cpu().numpy()


def rel_err(a, ref):
    return np.abs(a.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1.0)


def syndrome_ok(code, hard, syn):
    return np.all(synth.syndrome(code, hard) == syn, axis=1).astype(np.uint8)


def assert_same(a, b):
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


@pytest.fixture(scope="module")
def small():
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 16, 0.161)
    return code, fr


@pytest.mark.parametrize("T", [1, 2, 3, 4, 5])
def test_group_kernel_matches_the_oracle(q, small, T):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok = run(q, qc, fr.llr, fr.syn, T, kernel="group")
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T, nthreads=8)
    err = rel_err(p, rp)
    assert err.max() <= LLR_TOL, f"T={T}: {err.max():.3g}"
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))
    np.testing.assert_array_equal(h, (p < 0).astype(np.uint8))


@pytest.mark.parametrize("K", [1, 4, 7, 16])
@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
def test_group_kernel_is_bit_identical_to_the_frame_kernel(q, small, K, cluster):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    ref = run(q, qc, fr.llr[:K], fr.syn[:K], 6, kernel="frame")
    got = run(q, qc, fr.llr[:K], fr.syn[:K], 6, kernel="group", cluster=cluster)
    assert_same(ref, got)


@pytest.mark.parametrize("msg", ["fp16", "bf16"])
def test_group_kernel_16bit_messages_are_bit_identical(q, small, msg):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    ref = run(q, qc, fr.llr[:9], fr.syn[:9], 5, kernel="frame", msg=msg)
    got = run(q, qc, fr.llr[:9], fr.syn[:9], 5, kernel="group", msg=msg)
    assert_same(ref, got)


def test_group_kernel_ragged_z_and_many_groups(q):
    # Z = 2500 (the paper's expansion factor): ranges of 625 checks per block
    # at cluster size 4, several rounds with a ragged tail; 41 frames = 10
    # full groups and one of a single frame
    code = synth.make_code("0.1", 2500)
    fr = synth.make_frames(code, 41, 0.161, first=300)
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok = run(q, qc, fr.llr, fr.syn, 3, kernel="group", cluster=4)
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr[::8], fr.syn[::8], 3,
                             nthreads=6)
    assert rel_err(p[::8], rp).max() <= LLR_TOL
    np.testing.assert_array_equal(ok, syndrome_ok(code, h, fr.syn))
    assert_same((h, p, ok), run(q, qc, fr.llr, fr.syn, 3, kernel="frame"))


def random_code(seed, mb, nb, Z, min_deg, max_deg):
    rng = np.random.default_rng(seed)
    base = np.zeros((mb, nb), np.int8)
    for l in range(mb):
        d = int(rng.integers(min_deg, max_deg + 1))
        base[l, rng.choice(nb, d, replace=False)] = 1
    shifts = np.where(base == 1, rng.integers(0, Z, size=base.shape), 0).astype(np.int32)
    return synth.Code(base=base, shifts=shifts, Z=Z)


@pytest.mark.parametrize("seed,lo,hi", [(0, 9, 12), (1, 13, 16), (2, 1, 16), (3, 2, 8)])
def test_group_kernel_row_degrees_up_to_the_limit(q, seed, lo, hi):
    code = random_code(seed, 6, 18, 37, lo, hi)
    rng = np.random.default_rng(seed)
    x = rng.integers(0, 2, size=(6, code.n), dtype=np.uint8)
    llr = ((1.0 - 2.0 * x) * 2.0 + rng.normal(0, 2.0, size=x.shape)).astype(np.float32)
    syn = synth.syndrome(code, x)
    for merge in ("none", "exact"):
        qc = q.Code(code.base, code.shifts, code.Z, merge=merge)
        h, p, ok = run(q, qc, llr, syn, 3, kernel="group", cluster=2)
        _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, llr, syn, 3)
        assert rel_err(p, rp).max() <= LLR_TOL
        np.testing.assert_array_equal(ok, syndrome_ok(code, h, syn))
        assert_same((h, p, ok), run(q, qc, llr, syn, 3, kernel="frame"))


def test_group_kernel_degenerate_blocks(q):
    # column 3 unconnected, row 2 empty, row 3 a degree-1 check, columns 4 and 5 of degree one
    base = np.array([[1, 1, 1, 0, 1, 0],
                     [1, 1, 0, 0, 0, 1],
                     [0, 0, 0, 0, 0, 0],
                     [0, 0, 1, 0, 0, 0]], np.int8)
    Z = 33
    rng = np.random.default_rng(8)
    shifts = np.where(base == 1, rng.integers(0, Z, size=base.shape), 0).astype(np.int32)
    code = synth.Code(base=base, shifts=shifts, Z=Z)
    x = rng.integers(0, 2, size=(6, code.n), dtype=np.uint8)
    llr = ((1.0 - 2.0 * x) + rng.normal(0, 1.0, size=x.shape)).astype(np.float32)
    syn = synth.syndrome(code, x)
    syn[5, 2 * Z + 5] ^= 1          # an empty check with s_m = 1 can never be satisfied
    qc = q.Code(base, shifts, Z)
    for T in (0, 1, 4):
        h, p, ok = run(q, qc, llr, syn, T, kernel="group", cluster=2)
        rh, rp, rok = oracle.decode(base, shifts, Z, llr, syn, T)
        assert rel_err(p, rp).max() <= LLR_TOL
        np.testing.assert_array_equal(ok, syndrome_ok(code, h, syn))
        assert ok[5] == 0
        np.testing.assert_array_equal(p[:, 3 * Z:4 * Z], llr[:, 3 * Z:4 * Z])


def test_group_kernel_without_llr_post_and_from_host(q, small):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok = run(q, qc, fr.llr, fr.syn, 5, kernel="group")
    h2, p2, ok2 = run(q, qc, fr.llr, fr.syn, 5, kernel="group", want_post=False)
    assert p2 is None
    np.testing.assert_array_equal(h, h2)
    np.testing.assert_array_equal(ok, ok2)
    h3, p3, ok3 = q.decode_host(qc, fr.llr, fr.syn, 5, kernel="group")
    assert_same((h, p, ok), (h3, p3, ok3))


def test_group_kernel_rejects_what_it_does_not_serve(q, small):
    code, fr = small
    qc = q.Code(code.base, code.shifts, code.Z)
    d = torch.from_numpy(fr.llr).cuda()
    s = torch.from_numpy(fr.syn).cuda()
    with pytest.raises(q.QcmetError) as e:
        q.decode_early_stop(qc, d, s, 10, 1, kernel="group")
    assert e.value.status == q.ERR_UNSUPPORTED
    for bad in (17, -1):
        with pytest.raises(q.QcmetError) as e:
            q.decode(qc, d, s, 3, kernel="group", cluster=bad)
        assert e.value.status == q.ERR_INVALID_ARG


# --------------------------------------------------------------------------
# Full size (Z = 12500, n = 10^6): the bench's code

def test_group_kernel_full_size(q):
    code = synth.make_code("0.1", 12500)
    fr = synth.make_frames(code, 6, 0.161, first=40)
    qc = q.Code(code.base, code.shifts, code.Z)
    h, p, ok = run(q, qc, fr.llr, fr.syn, 2, kernel="group")
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr[[0, 5]], fr.syn[[0, 5]], 2,
                             nthreads=2)
    assert rel_err(p[[0, 5]], rp).max() <= LLR_TOL
    assert_same((h, p, ok), run(q, qc, fr.llr, fr.syn, 2, kernel="frame"))
    for cluster in (1, 8):
        assert_same((h, p, ok), run(q, qc, fr.llr, fr.syn, 2, kernel="group", cluster=cluster))


# --------------------------------------------------------------------------
# Launch shapes: any cluster size up to 16 and two groups per cluster (the
# cluster's blocks split the two groups' checks, so one block may hold checks
# of both) give the per-frame kernel's results bit for bit.

@pytest.mark.parametrize("rate,Z,K,cluster,groups", [
    ("0.1", 1250, 16, 3, 2),     # two groups per cluster, blocks straddle the groups
    ("0.1", 1250, 12, 5, 2),     # three groups: the last cluster holds one
    ("0.05", 1000, 9, 4, 2),     # a partial last group (one frame)
    ("0.02", 777, 8, 7, 2),      # Z with no factor of 2
    ("0.1", 1250, 8, 9, 1),      # a non-portable cluster size, one group per cluster
    ("0.1", 1250, 4, 16, 1),     # the largest cluster
    ("0.05", 1000, 24, 6, 0),    # automatic groups per cluster
])
def test_launch_shapes_are_bit_identical_to_the_frame_kernel(q, rate, Z, K, cluster, groups):
    code = synth.make_code(rate, Z)
    fr = synth.make_frames(code, K, synth.RATE_SNR[rate] + 0.05, first=900)
    qc = q.Code(code.base, code.shifts, code.Z)
    try:
        plan = q.group_plan(qc, K, cluster=cluster, groups=groups)
    except q.QcmetError as e:
        assert e.status == q.ERR_UNSUPPORTED
        pytest.skip(f"cluster size {cluster} cannot be scheduled on this device")
    if groups:
        assert plan["groups_per_cluster"] == groups
    assert plan["cluster_size"] == cluster
    for msg in ("fp32", "fp16"):
        for T in (1, 8):
            ref = run(q, qc, fr.llr, fr.syn, T, kernel="frame", msg=msg)
            got = run(q, qc, fr.llr, fr.syn, T, kernel="group", cluster=cluster, groups=groups,
                      msg=msg)
            assert_same(got, ref)


def test_group_plan_spreads_frames_over_the_device(q):
    code = synth.make_code("0.1", 12500)
    qc = q.Code(code.base, code.shifts, code.Z)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    for K in (4, 16, 64, 128):
        p = q.group_plan(qc, K)
        groups = (K + 3) // 4
        assert p["clusters"] == -(-groups // p["groups_per_cluster"])
        assert p["blocks"] == p["clusters"] * p["cluster_size"]
        assert p["clusters"] <= p["active_clusters"], p      # one wave
        # a group of four frames is split over several SMs when SMs are free
        assert p["blocks"] >= min(sms // 2, 8 * groups), p
    with pytest.raises(q.QcmetError) as e:
        q.group_plan(qc, 8, groups=3)
    assert e.value.status == q.ERR_INVALID_ARG
