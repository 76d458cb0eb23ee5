"""Pins of the FP64 oracle to results fixed by the paper or by mathematics.

None of these compare the oracle with itself: each checks it against a brute
force, a closed form, a value printed in arXiv 2004.09084, or an invariant
that a dropped term, a wrong sign or index, or a transposed operand breaks.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from tests import helpers

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------
# Phi (Methods, step 2): Phi(x) = -ln tanh(x/2), Phi = Phi^{-1}

def test_phi_closed_forms():
    # (e^x + 1)/(e^x - 1) = 2 at x = ln 3, so Phi(ln 3) = ln 2 and, by
    # self-inversion, Phi(ln 2) = ln 3.
    assert oracle.phi(math.log(3.0)) == pytest.approx(math.log(2.0), rel=1e-15)
    assert oracle.phi(math.log(2.0)) == pytest.approx(math.log(3.0), rel=1e-15)


def test_phi_matches_definition_where_it_is_well_conditioned():
    for x in np.linspace(0.05, 12.0, 97):
        ref = -math.log(math.tanh(x / 2.0))
        assert oracle.phi(x) == pytest.approx(ref, rel=1e-12)


def test_phi_is_an_involution_on_the_clipping_interval():
    lo, hi = oracle.clip_min(), oracle.clip_max()
    assert hi == 30.0
    # the lower clip is Phi(30), so Phi maps [lo, hi] onto itself
    assert lo == pytest.approx(2.0 * math.atanh(math.exp(-30.0)), rel=1e-14)
    for x in np.geomspace(lo, hi, 200):
        assert oracle.phi(oracle.phi(x)) == pytest.approx(x, rel=1e-11)


def test_phi_clipping():
    lo, hi = oracle.clip_min(), oracle.clip_max()
    assert oracle.phi(0.0) == pytest.approx(hi, rel=1e-12)
    assert oracle.phi(1e-300) == pytest.approx(hi, rel=1e-12)
    assert oracle.phi(1e6) == pytest.approx(lo, rel=1e-12)


# --------------------------------------------------------------------------
# One check node (Methods, step 2, with the syndrome sign)

@pytest.mark.parametrize("d", [2, 3, 4, 5, 7, 10])
@pytest.mark.parametrize("s", [0, 1])
def test_check_update_equals_bruteforce_extrinsic(d, s):
    rng = np.random.default_rng(100 * d + s)
    for _ in range(4):
        q = rng.normal(0.0, 3.0, size=d)
        got = oracle.check_update(q, s)
        ref = helpers.check_message_bruteforce(q, s)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12)


def test_degree_two_check_passes_the_other_message_through():
    # Phi(Phi(|q|)) = |q|: a degree-2 check forwards the other message (flipped by s)
    rng = np.random.default_rng(7)
    for _ in range(50):
        q = rng.uniform(-29.0, 29.0, size=2)
        for s in (0, 1):
            r = oracle.check_update(q, s)
            sign = -1.0 if s else 1.0
            assert r[0] == pytest.approx(sign * q[1], rel=1e-11)
            assert r[1] == pytest.approx(sign * q[0], rel=1e-11)


@pytest.mark.parametrize("d", [3, 4, 6, 10])
def test_phi_rule_equals_tanh_product_rule(d):
    rng = np.random.default_rng(d)
    for _ in range(20):
        q = rng.normal(0.0, 4.0, size=d)
        got = oracle.check_update(q, 0)
        t = np.tanh(q / 2.0)
        ref = np.array([2.0 * np.arctanh(np.prod(np.delete(t, j))) for j in range(d)])
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-13)


def test_syndrome_bit_negates_every_message():
    rng = np.random.default_rng(3)
    q = rng.normal(0, 2, size=6)
    np.testing.assert_array_equal(oracle.check_update(q, 1), -oracle.check_update(q, 0))


def test_degree_one_check_saturates():
    # empty exclusive set: the clipped Phi of an empty sum is the upper clip
    r0 = oracle.check_update([0.7], 0)
    r1 = oracle.check_update([0.7], 1)
    assert r0[0] == pytest.approx(30.0, rel=1e-12)
    assert r1[0] == pytest.approx(-30.0, rel=1e-12)


def test_message_magnitudes_stay_in_the_clipping_interval():
    lo, hi = oracle.clip_min(), oracle.clip_max()
    rng = np.random.default_rng(11)
    for _ in range(200):
        d = int(rng.integers(2, 11))
        q = rng.normal(0, 40, size=d) * rng.choice([1e-9, 1.0, 10.0], size=d)
        r = np.abs(oracle.check_update(q, 0))
        assert np.all(r >= lo * (1 - 1e-12)) and np.all(r <= hi * (1 + 1e-12))


# --------------------------------------------------------------------------
# The circulant convention (Results, after Eq. (m))

def test_circulant_expansion_follows_right_shift_convention():
    expected = helpers.read_matrix_file("circulant_Z4_shift1.txt")
    np.testing.assert_array_equal(helpers.circulant(4, 1), expected)


def test_generator_syndrome_uses_the_same_convention():
    code = synth.make_code("0.1", 8)
    x = np.random.default_rng(0).integers(0, 2, size=(3, code.n), dtype=np.uint8)
    H = helpers.expand_dense(code.base, code.shifts, code.Z)
    np.testing.assert_array_equal(synth.syndrome(code, x), helpers.syndrome_dense(H, x))


# --------------------------------------------------------------------------
# Whole decoder against exact marginals on cycle-free codes

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("Z", [1, 2])
def test_layered_bp_is_exact_on_cycle_free_codes(seed, Z):
    base, shifts = helpers.tree_code(seed, Z)
    H = helpers.expand_dense(base, shifts, Z)
    m, n = H.shape
    if n > 18:
        pytest.skip("too many variables for enumeration")
    rng = np.random.default_rng(1000 + seed)
    x = rng.integers(0, 2, size=n, dtype=np.uint8)
    s = helpers.syndrome_dense(H, x[None])[0]
    llr = (2.0 * ((1.0 - 2.0 * x) + rng.normal(0, 1.2, size=n)) / 1.44).astype(np.float32)
    hard, post, ok = oracle.decode(base, shifts, Z, llr[None], s[None], iterations=12)
    ref = helpers.exact_app(H, llr, s)
    assert np.max(np.abs(ref)) < 25.0       # no clipping in play
    np.testing.assert_allclose(post[0], ref, rtol=1e-9, atol=1e-9)
    np.testing.assert_array_equal(hard[0], (ref < 0).astype(np.uint8))


def test_bp_on_a_tree_is_exact_with_any_row_order():
    base, shifts = helpers.tree_code(4, 2)
    H = helpers.expand_dense(base, shifts, 2)
    n = H.shape[1]
    rng = np.random.default_rng(5)
    x = rng.integers(0, 2, size=n, dtype=np.uint8)
    s = helpers.syndrome_dense(H, x[None])[0]
    llr = (2.0 * ((1.0 - 2.0 * x) + rng.normal(0, 1.0, size=n))).astype(np.float32)
    ref = helpers.exact_app(H, llr, s)
    order = np.arange(base.shape[0])[::-1]
    _, post, _ = oracle.decode(base, shifts, 2, llr[None], s[None], 12, order=order)
    np.testing.assert_allclose(post[0], ref, rtol=1e-9, atol=1e-9)


# --------------------------------------------------------------------------
# Invariants on the synthetic QC-MET code

@pytest.fixture(scope="module")
def small_case():
    code = synth.make_code("0.1", 16)
    fr = synth.make_frames(code, 3, 0.161)
    return code, fr


def test_noiseless_input_decodes_in_one_iteration():
    code = synth.make_code("0.1", 16)
    fr = synth.make_frames(code, 3, 0.161, noiseless=True)
    hard, post, ok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 1)
    np.testing.assert_array_equal(hard, fr.x)
    np.testing.assert_array_equal(ok, [1, 1, 1])


def test_zero_iterations_return_the_channel(small_case):
    code, fr = small_case
    hard, post, ok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 0)
    np.testing.assert_array_equal(post, fr.llr.astype(np.float64))
    np.testing.assert_array_equal(hard, (fr.llr < 0).astype(np.uint8))


def test_ok_flag_is_the_syndrome_test(small_case):
    code, fr = small_case
    H = helpers.expand_dense(code.base, code.shifts, code.Z)
    for T in (1, 3, 10):
        hard, _, ok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T)
        recomputed = np.all(helpers.syndrome_dense(H, hard) == fr.syn, axis=1)
        np.testing.assert_array_equal(ok.astype(bool), recomputed)


def test_coset_symmetry_is_exact(small_case):
    # decoding (llr * (1 - 2 x0), s ^ H x0) negates exactly the posteriors of x0's ones
    code, fr = small_case
    rng = np.random.default_rng(9)
    x0 = rng.integers(0, 2, size=(3, code.n), dtype=np.uint8)
    flip = (1.0 - 2.0 * x0).astype(np.float32)
    _, post, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 6)
    _, post2, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr * flip,
                                fr.syn ^ synth.syndrome(code, x0), 6)
    np.testing.assert_array_equal(post2, post * flip.astype(np.float64))


def test_quasi_cyclic_decoder_equals_plain_matrix_decoder(small_case):
    # Expanding every circulant by hand and decoding the result as a Z = 1 code,
    # one check per layer in layer order, must give identical numbers: the Z
    # checks of one base row touch disjoint variables.
    code, fr = small_case
    H = helpers.expand_dense(code.base, code.shifts, code.Z)
    _, post, ok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 4)
    _, post1, ok1 = oracle.decode(H.astype(np.int8), np.zeros(H.shape, np.int32), 1,
                                  fr.llr, fr.syn, 4)
    np.testing.assert_array_equal(post1, post)
    np.testing.assert_array_equal(ok1, ok)


def test_tanh_rule_decoder_matches_phi_rule_decoder(small_case):
    code, fr = small_case
    _, post, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 3)
    _, post_t, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 3,
                                 rule=oracle.RULE_TANH)
    err = np.abs(post_t - post) / np.maximum(np.abs(post), 1.0)
    assert err.max() < 1e-6


def test_reordering_rows_with_disjoint_columns_is_exact():
    # Eq. (m1): rows 0 and 1 share no column, so swapping them inside one
    # iteration leaves every number unchanged.
    base = np.array([[1, 0, 0], [0, 1, 1], [1, 1, 1]], dtype=np.int8)
    shifts = np.array([[1, 0, 0], [0, 2, 1], [2, 0, 0]], dtype=np.int32)
    Z = 5
    H = helpers.expand_dense(base, shifts, Z)
    rng = np.random.default_rng(2)
    x = rng.integers(0, 2, size=(2, 15), dtype=np.uint8)
    s = helpers.syndrome_dense(H, x)
    llr = rng.normal(1.0, 2.0, size=(2, 15)).astype(np.float32)
    _, a, _ = oracle.decode(base, shifts, Z, llr, s, 5, order=[0, 1, 2])
    _, b, _ = oracle.decode(base, shifts, Z, llr, s, 5, order=[1, 0, 2])
    np.testing.assert_array_equal(a, b)
    _, c, _ = oracle.decode(base, shifts, Z, llr, s, 5, order=[0, 2, 1])
    assert not np.array_equal(a, c)     # a reorder across related rows is not exact


def test_threads_do_not_change_results(small_case):
    code, fr = small_case
    a = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 3, nthreads=1)
    b = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 3, nthreads=3)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


# --------------------------------------------------------------------------
# Message storage rounding (FP16 / BF16 variants)

def test_fp16_rounding_matches_ieee_half():
    rng = np.random.default_rng(4)
    xs = np.concatenate([rng.normal(0, 8, 500), rng.normal(0, 1e-5, 200),
                         np.geomspace(1e-9, 30, 100)])
    for x in xs:
        assert oracle.round_msg(x, oracle.MSG_FP16) == float(np.float16(x))


def test_bf16_rounding_ties_to_even_and_keeps_8_bits():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties go to the even one (1)
    assert oracle.round_msg(1.0 + 2.0 ** -8, oracle.MSG_BF16) == 1.0
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 and 1 + 2^-6: even is 1 + 2^-6
    assert oracle.round_msg(1.0 + 3 * 2.0 ** -8, oracle.MSG_BF16) == 1.0 + 2.0 ** -6
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    xs = rng.normal(0, 8, 1000).astype(np.float32)      # float32 inputs: one rounding only
    ref = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_msg(float(x), oracle.MSG_BF16) for x in xs])
    np.testing.assert_array_equal(got, ref)


def test_exact_storage_format_is_identity():
    for x in (0.3, -17.25, 1e-11):
        assert oracle.round_msg(x, oracle.MSG_EXACT) == x


# --------------------------------------------------------------------------
# Min-sum rule (learned variant)

def test_minsum_with_unit_weights_is_plain_minsum():
    code = synth.make_code("0.1", 8)
    fr = synth.make_frames(code, 2, 0.3)
    T = 2
    ws = np.ones((T, code.mb, 2))
    wo = np.zeros((T, code.mb, 2))
    _, post, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T,
                               rule=oracle.RULE_MINSUM, w_scale=ws, w_offset=wo)
    # hand-rolled plain min-sum on the dense matrix, one check at a time, layer order
    H = helpers.expand_dense(code.base, code.shifts, code.Z)
    for k in range(2):
        L = fr.llr[k].astype(np.float64).copy()
        R = np.zeros(H.shape)
        for _ in range(T):
            for mrow in range(H.shape[0]):
                vs = np.flatnonzero(H[mrow])
                q = L[vs] - R[mrow, vs]
                r = np.empty_like(q)
                for j in range(len(vs)):
                    o = np.delete(q, j)
                    r[j] = (-1.0 if fr.syn[k, mrow] else 1.0) * np.prod(np.where(o < 0, -1.0, 1.0)) \
                        * min(np.min(np.abs(o)), 30.0)
                R[mrow, vs] = r
                L[vs] = q + r
        np.testing.assert_allclose(post[k], L, rtol=1e-12, atol=1e-12)


def test_minsum_offset_and_scale():
    # one degree-3 check: |r_j| = max(scale * min_{k != j} |q_k| - offset, 0)
    base = np.array([[1, 1, 1]], dtype=np.int8)
    shifts = np.zeros((1, 3), np.int32)
    llr = np.array([[2.0, -3.0, 0.5]], dtype=np.float32)
    s = np.array([[1]], dtype=np.uint8)
    ws = np.full((1, 1, 2), 0.75)
    wo = np.full((1, 1, 2), 0.25)
    _, post, _ = oracle.decode(base, shifts, 1, llr, s, 1, rule=oracle.RULE_MINSUM,
                               w_scale=ws, w_offset=wo)
    # edge 0: others (-3, 0.5): sign -1 * s-flip -1 = +1, mag max(0.75*0.5-0.25, 0) = 0.125
    # edge 1: others (2, 0.5): sign +1 * -1 = -1, mag 0.125
    # edge 2: others (2, -3): sign -1 * -1 = +1, mag max(0.75*2-0.25,0) = 1.25
    np.testing.assert_allclose(post[0], [2.125, -3.125, 1.75], rtol=1e-15)


def test_minsum_message_clip():
    # |r| is clipped to 30, the sum-product rule's clip: with unit weights a
    # degree-3 check over (50, 60, -70) sends min(60, 30), min(50, 30), min(50, 30)
    base = np.array([[1, 1, 1]], dtype=np.int8)
    shifts = np.zeros((1, 3), np.int32)
    llr = np.array([[50.0, 60.0, -70.0]], dtype=np.float32)
    s = np.array([[0]], dtype=np.uint8)
    ws = np.ones((1, 1, 2))
    wo = np.zeros((1, 1, 2))
    _, post, _ = oracle.decode(base, shifts, 1, llr, s, 1, rule=oracle.RULE_MINSUM,
                               w_scale=ws, w_offset=wo)
    # edge 0: others (60, -70) -> -30; edge 1: others (50, -70) -> -30; edge 2: (50, 60) -> +30
    np.testing.assert_array_equal(post[0], [20.0, 30.0, -40.0])
    # offset below the clip: 1.0 * 60 - 35 = 25 < 30 for edge 0
    wo = np.full((1, 1, 2), 35.0)
    _, post, _ = oracle.decode(base, shifts, 1, llr, s, 1, rule=oracle.RULE_MINSUM,
                               w_scale=ws, w_offset=wo)
    np.testing.assert_array_equal(post[0], [25.0, 45.0, -55.0])


# --------------------------------------------------------------------------
# The SNR convention, pinned by the efficiencies printed in Table tab1

def test_efficiency_reproduces_table_tab1():
    tab = helpers.read_table("table_tab1.txt")
    for rate, snr, beta_pct, *_ in tab:
        assert 100.0 * synth.efficiency(rate, snr) == pytest.approx(beta_pct, abs=0.006)


def test_throughput_times_latency_is_one_megabit():
    # Table tab1: Mbit/s x "latency per iteration" = 1.00 in every column, so the
    # printed latency is the decode wall time divided by the 128 codewords, and
    # the speed is K * n / wall time.
    tab = helpers.read_table("table_tab1.txt")
    for *_, latency, mbit in tab:
        assert latency * mbit == pytest.approx(1.0, abs=0.003)


def test_channel_llr_convention():
    code = synth.make_code("0.1", 4)
    fr = synth.make_frames(code, 1, 0.25, noiseless=True)
    # noiseless R = 1 - 2x, sigma^2 = 1/SNR = 4: L = 2R/sigma^2 = +-0.5
    np.testing.assert_allclose(fr.llr[0], 0.5 * (1.0 - 2.0 * fr.x[0]))


# --------------------------------------------------------------------------
# Early termination (Discussion, Table tabearly)

def test_early_termination_stops_at_the_first_passing_check_and_changes_nothing_else():
    code = synth.make_code("0.1", 16)
    fr = synth.make_frames(code, 12, 0.3)
    T = 30
    for every in (1, 3):
        h, p, ok, it = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T,
                                     early_every=every, return_iters=True)
        H = helpers.expand_dense(code.base, code.shifts, code.Z)
        for k in range(12):
            # a stopped frame equals a fixed-iteration decode of exactly that many iterations
            hk, pk, okk = oracle.decode(code.base, code.shifts, code.Z, fr.llr[k:k + 1],
                                        fr.syn[k:k + 1], int(it[k]))
            np.testing.assert_array_equal(p[k], pk[0])
            assert ok[k] == okk[0]
            assert it[k] % every == 0 or it[k] == T
            # it stopped at the first checked iteration whose hard decision satisfies H c = s
            for t in range(every, int(it[k]), every):
                ht, _, okt = oracle.decode(code.base, code.shifts, code.Z, fr.llr[k:k + 1],
                                           fr.syn[k:k + 1], t)
                assert okt[0] == 0
            if it[k] < T:
                assert ok[k] == 1
                assert np.all(helpers.syndrome_dense(H, h[k:k + 1])[0] == fr.syn[k])
        assert np.any(it < T)          # at SNR 0.3 most frames converge early


def test_early_termination_off_is_the_fixed_schedule():
    code = synth.make_code("0.1", 8)
    fr = synth.make_frames(code, 3, 0.3)
    a = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 7)
    b = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, 7, early_every=0,
                      return_iters=True)
    for u, v in zip(a, b[:3]):
        np.testing.assert_array_equal(u, v)
    np.testing.assert_array_equal(b[3], [7, 7, 7])


# --------------------------------------------------------------------------
# Learned min-sum: loss and its gradient (the training target of the learned variant)

def _minsum_case(Z=4, K=2, T=3, seed=0, snr=0.3):
    code = synth.make_code("0.1", Z)
    fr = synth.make_frames(code, K, snr)
    rng = np.random.default_rng(seed)
    ws = 0.7 + 0.3 * rng.random((T, code.mb, 2))
    wo = 0.3 * rng.random((T, code.mb, 2))
    return code, fr, T, ws, wo


def test_minsum_gradient_matches_central_differences():
    code, fr, T, ws, wo = _minsum_case()
    loss, gs, go = oracle.minsum_train(code.base, code.shifts, code.Z, fr.llr, fr.syn, fr.x, T,
                                       ws, wo)
    rng = np.random.default_rng(1)
    eps = 1e-6
    picks = [tuple(rng.integers(0, s) for s in ws.shape) for _ in range(12)]
    picks += [(0, 0, 0), (T - 1, 1, 0), (1, 5, 1)]
    for idx in picks:
        for which in ("scale", "offset"):
            def f(delta):
                a, b = ws.copy(), wo.copy()
                (a if which == "scale" else b)[idx] += delta
                return oracle.minsum_train(code.base, code.shifts, code.Z, fr.llr, fr.syn, fr.x,
                                           T, a, b)[0].sum()
            fd = (f(eps) - f(-eps)) / (2 * eps)
            an = (gs if which == "scale" else go)[idx]
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-9), (which, idx)


def test_minsum_gradient_with_the_message_clip_active():
    # Core columns carry confident correct LLRs (magnitude 50) and degree-1
    # columns confident wrong ones (45): checks send messages at the clip
    # (|r| = 30) both ways, and the posteriors they reach stay wrong or small,
    # so the loss depends on those messages while the clip holds them fixed.
    code, fr, T, _, _ = _minsum_case(snr=0.3)
    Z = code.Z
    deg = np.repeat(code.base.sum(axis=0), Z)
    sx = 1.0 - 2.0 * fr.x
    llr = np.where(deg > 1, 50.0 * sx, -45.0 * sx).astype(np.float32)
    rng = np.random.default_rng(3)
    ws = 0.9 + 0.2 * rng.random((T, code.mb, 2))
    wo = 0.1 * rng.random((T, code.mb, 2))
    loss, gs, go = oracle.minsum_train(code.base, code.shifts, code.Z, llr, fr.syn, fr.x, T,
                                       ws, wo)
    eps = 1e-6
    worst = 0.0
    for idx in np.ndindex(ws.shape):
        for which in ("scale", "offset"):
            def f(delta):
                a, b = ws.copy(), wo.copy()
                (a if which == "scale" else b)[idx] += delta
                return oracle.minsum_train(code.base, code.shifts, code.Z, llr, fr.syn, fr.x,
                                           T, a, b)[0].sum()
            fd = (f(eps) - f(-eps)) / (2 * eps)
            an = (gs if which == "scale" else go)[idx]
            worst = max(worst, abs(an - fd))
            # the loss sum is O(100): central differences carry ~1e-8 of rounding;
            # a gradient taken through a clipped message would be off by ~1e-2
            assert an == pytest.approx(fd, rel=1e-5, abs=1e-6), (which, idx)
    assert np.abs(gs).max() > 1e-3 and np.abs(go).max() > 1e-3   # the loss is not saturated


def test_minsum_loss_is_the_mean_cross_entropy_of_the_decoder_posteriors():
    code, fr, T, ws, wo = _minsum_case(T=2)
    loss, _, _ = oracle.minsum_train(code.base, code.shifts, code.Z, fr.llr, fr.syn, fr.x, T,
                                     ws, wo)
    sgx = 1.0 - 2.0 * fr.x.astype(np.float64)
    terms = []
    for t in (1, 2):
        _, post, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, t,
                                   rule=oracle.RULE_MINSUM, w_scale=ws, w_offset=wo)
        terms.append(np.logaddexp(0.0, -sgx * post).mean(axis=1))
    np.testing.assert_allclose(loss, np.mean(terms, axis=0), rtol=1e-12)
