"""GPU learned offset/scaled min-sum: forward, loss and hand-written backward
against the FP64 oracle, the autograd wrapper, and what training gains.

Min-sum passes the selected minimum |q| straight through, so the rounding
difference between the FP32 kernels and the FP64 oracle is not damped the way
the tanh rule damps it: on the rate-0.1 code it grows about tenfold per
iteration (measured on GB300: 3e-6 after one iteration, 3e-5 after two, 4e-4
after three).  Once the trajectories part, different argmin and max(., 0)
choices change the piecewise-linear gradient.  The element-wise bars therefore
apply where the trajectories coincide (one or two iterations); longer runs are
compared in distribution (hard decisions, loss, gradient direction).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import paper_2004_09084_gb300 as q
    assert torch.cuda.is_available()
    return q


@pytest.fixture(scope="module")
def learned(q):
    from paper_2004_09084_gb300 import learned
    return learned


def weights(code, T, seed=0):
    rng = np.random.default_rng(seed)
    ws = (0.7 + 0.3 * rng.random((T, code.mb, 2))).astype(np.float32)
    wo = (0.3 * rng.random((T, code.mb, 2))).astype(np.float32)
    return ws, wo


def rel_err(a, ref):
    return np.abs(a.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1.0)


@pytest.mark.parametrize("Z,K", [(64, 8), (2500, 2)])
def test_learned_decode_matches_the_oracle(q, learned, Z, K):
    code = synth.make_code("0.1", Z)
    fr = synth.make_frames(code, K, 0.2)
    qc = q.Code(code.base, code.shifts, code.Z)
    for T in (1, 2):
        ws, wo = weights(code, T)
        h, p, ok = learned.decode(qc, torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda(),
                                  torch.from_numpy(ws).cuda(), torch.from_numpy(wo).cuda())
        torch.cuda.synchronize()
        _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T,
                                 rule=oracle.RULE_MINSUM, w_scale=ws.astype(np.float64),
                                 w_offset=wo.astype(np.float64), nthreads=8)
        assert rel_err(p.cpu().numpy(), rp).max() <= 1e-4
        hh = h.cpu().numpy()
        want = np.all(synth.syndrome(code, hh) == fr.syn, axis=1).astype(np.uint8)
        np.testing.assert_array_equal(ok.cpu().numpy(), want)


@pytest.mark.parametrize("seed,lo,hi", [(0, 1, 4), (1, 5, 10), (2, 11, 16)])
def test_learned_decode_for_row_degrees_up_to_the_limit(q, learned, seed, lo, hi):
    # every row path of the min-sum rule: one thread per check (degree <= 4),
    # two lanes per check with the loads issued together (5..10) or gathered
    # as used (11..16)
    rng = np.random.default_rng(seed)
    mb, nb, Z = 6, 18, 37
    base = np.zeros((mb, nb), np.int8)
    for l in range(mb):
        base[l, rng.choice(nb, int(rng.integers(lo, hi + 1)), replace=False)] = 1
    shifts = np.where(base == 1, rng.integers(0, Z, size=base.shape), 0).astype(np.int32)
    code = synth.Code(base=base, shifts=shifts, Z=Z)
    x = rng.integers(0, 2, size=(3, code.n), dtype=np.uint8)
    llr = ((1.0 - 2.0 * x) * 2.0 + rng.normal(0, 2.0, size=x.shape)).astype(np.float32)
    syn = synth.syndrome(code, x)
    qc = q.Code(code.base, code.shifts, code.Z)
    T = 1
    ws, wo = weights(code, T, seed=seed)
    h, p, ok = learned.decode(qc, torch.from_numpy(llr).cuda(), torch.from_numpy(syn).cuda(),
                              torch.from_numpy(ws).cuda(), torch.from_numpy(wo).cuda())
    torch.cuda.synchronize()
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, llr, syn, T, rule=oracle.RULE_MINSUM,
                             w_scale=ws.astype(np.float64), w_offset=wo.astype(np.float64))
    assert rel_err(p.cpu().numpy(), rp).max() <= 1e-4


def test_learned_decode_agrees_in_distribution_over_more_iterations(q, learned):
    # at an SNR where min-sum converges, both reach the same decisions
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 16, 0.35)
    qc = q.Code(code.base, code.shifts, code.Z)
    T = 10
    ws, wo = weights(code, T)
    h, p, ok = learned.decode(qc, torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda(),
                              torch.from_numpy(ws).cuda(), torch.from_numpy(wo).cuda())
    torch.cuda.synchronize()
    rh, rp, rok = oracle.decode(code.base, code.shifts, code.Z, fr.llr, fr.syn, T,
                                rule=oracle.RULE_MINSUM, w_scale=ws.astype(np.float64),
                                w_offset=wo.astype(np.float64), nthreads=8)
    assert np.mean(h.cpu().numpy() == rh) >= 0.99
    assert np.mean(ok.cpu().numpy() == rok) >= 0.9


@pytest.mark.parametrize("Z,K,T,bar", [(64, 6, 1, 2e-3), (64, 6, 2, 2e-3), (64, 6, 4, 5e-2),
                                       (12500, 1, 2, 1e-2)])
def test_loss_and_gradient_match_the_oracle(q, learned, Z, K, T, bar):
    code = synth.make_code("0.1", Z)
    fr = synth.make_frames(code, K, 0.18)
    qc = q.Code(code.base, code.shifts, code.Z)
    ws, wo = weights(code, T, seed=3)
    d = dict(llr=torch.from_numpy(fr.llr).cuda(), syn=torch.from_numpy(fr.syn).cuda(),
             bits=torch.from_numpy(fr.x).cuda())
    tws = torch.from_numpy(ws).cuda().requires_grad_()
    two = torch.from_numpy(wo).cuda().requires_grad_()
    loss = learned.minsum_loss(tws, two, qc, d["llr"], d["syn"], d["bits"])
    loss.sum().backward()
    torch.cuda.synchronize()
    rl, rgs, rgo = oracle.minsum_train(code.base, code.shifts, code.Z, fr.llr, fr.syn, fr.x, T,
                                       ws.astype(np.float64), wo.astype(np.float64))
    np.testing.assert_allclose(loss.detach().cpu().numpy(), rl, rtol=1e-4)
    for g, rg in ((tws.grad, rgs), (two.grad, rgo)):
        g = g.cpu().numpy().astype(np.float64).ravel()
        rg = rg.ravel()
        rel = np.linalg.norm(g - rg) / np.linalg.norm(rg)
        cos = float(g @ rg / (np.linalg.norm(g) * np.linalg.norm(rg)))
        assert rel <= bar and cos >= 0.999, (rel, cos)


def test_message_clip_matches_the_oracle(q, learned):
    # confident correct core LLRs (50) and confident wrong degree-1 LLRs (45):
    # messages sit at the clip |r| = 30 in both directions; decode, loss and
    # gradient follow the oracle, and nothing overflows
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 4, 0.3)
    deg = np.repeat(code.base.sum(axis=0), code.Z)
    sx = 1.0 - 2.0 * fr.x
    llr = np.where(deg > 1, 50.0 * sx, -45.0 * sx).astype(np.float32)
    qc = q.Code(code.base, code.shifts, code.Z)
    T = 2
    ws = np.full((T, code.mb, 2), 1.0, np.float32)
    wo = np.full((T, code.mb, 2), 0.125, np.float32)
    d_llr, d_syn = torch.from_numpy(llr).cuda(), torch.from_numpy(fr.syn).cuda()
    h, p, ok = learned.decode(qc, d_llr, d_syn, torch.from_numpy(ws).cuda(), torch.from_numpy(wo).cuda())
    torch.cuda.synchronize()
    _, rp, _ = oracle.decode(code.base, code.shifts, code.Z, llr, fr.syn, T, rule=oracle.RULE_MINSUM,
                             w_scale=ws.astype(np.float64), w_offset=wo.astype(np.float64))
    assert np.abs(rp).max() > 100.0              # large posteriors: the clip is active
    assert rel_err(p.cpu().numpy(), rp).max() <= 1e-5
    tws = torch.from_numpy(ws).cuda().requires_grad_()
    two = torch.from_numpy(wo).cuda().requires_grad_()
    loss = learned.minsum_loss(tws, two, qc, d_llr, d_syn, torch.from_numpy(fr.x).cuda())
    loss.sum().backward()
    torch.cuda.synchronize()
    rl, rgs, rgo = oracle.minsum_train(code.base, code.shifts, code.Z, llr, fr.syn, fr.x, T,
                                       ws.astype(np.float64), wo.astype(np.float64))
    np.testing.assert_allclose(loss.detach().cpu().numpy(), rl, rtol=1e-4)
    for g, rg in ((tws.grad, rgs), (two.grad, rgo)):
        g = g.cpu().numpy().astype(np.float64).ravel()
        assert np.all(np.isfinite(g))
        rel = np.linalg.norm(g - rg.ravel()) / np.linalg.norm(rg)
        assert rel <= 2e-3, rel


def test_thirty_iterations_stay_finite(q, learned):
    # The clip keeps the forward finite even for unscaled min-sum.  The exact
    # gradient of 30 unrolled unscaled iterations is itself beyond the FP32
    # range here (the FP64 oracle gives |dL/dw| ~ 1e42 at scale 1, ~1e13 at
    # 0.5 and ~1e-3 at 0.25 on the Z = 64 code), so training starts from small
    # scales; from scale 0.25 the FP32 backward stays finite.
    code = synth.make_code("0.1", 2500)
    fr = synth.make_frames(code, 4, 0.161)
    qc = q.Code(code.base, code.shifts, code.Z)
    d = dict(llr=torch.from_numpy(fr.llr).cuda(), syn=torch.from_numpy(fr.syn).cuda(),
             bits=torch.from_numpy(fr.x).cuda())
    ws, wo = learned.init_weights(qc, 30)
    _, p, _ = learned.decode(qc, d["llr"], d["syn"], ws, wo)
    assert bool(torch.isfinite(p).all())
    ws, wo = learned.init_weights(qc, 30, scale=0.25)
    ws.requires_grad_()
    wo.requires_grad_()
    learned.minsum_loss(ws, wo, qc, d["llr"], d["syn"], d["bits"]).mean().backward()
    assert bool(torch.isfinite(ws.grad).all()) and bool(torch.isfinite(wo.grad).all())


def test_autograd_mean_scales_the_gradient(q, learned):
    code = synth.make_code("0.1", 64)
    fr = synth.make_frames(code, 4, 0.2)
    qc = q.Code(code.base, code.shifts, code.Z)
    ws, wo = weights(code, 3)
    args = (qc, torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda(),
            torch.from_numpy(fr.x).cuda())
    a = torch.from_numpy(ws).cuda().requires_grad_()
    b = torch.from_numpy(wo).cuda().requires_grad_()
    learned.minsum_loss(a, b, *args).sum().backward()
    ga, gb = a.grad.clone(), b.grad.clone()
    a.grad = None
    b.grad = None
    learned.minsum_loss(a, b, *args).mean().backward()
    torch.testing.assert_close(a.grad * 4, ga)
    torch.testing.assert_close(b.grad * 4, gb)


def test_backward_needs_a_forward(q):
    code = synth.make_code("0.1", 16)
    qc = q.Code(code.base, code.shifts, code.Z)
    g = torch.zeros((2, code.mb, 2), dtype=torch.float32, device="cuda")
    assert q.lib.qcmet_minsum_backward(qc.handle, g.data_ptr(), g.data_ptr(), None) == q.ERR_INVALID_ARG


def test_training_improves_on_plain_minsum(q, learned):
    # Training the scales and offsets on decoder-generated frames must beat
    # plain min-sum (scale 1, offset 0) on held-out frames.
    code = synth.make_code("0.1", 64)
    qc = q.Code(code.base, code.shifts, code.Z)
    T = 10
    gen = torch.Generator(device="cuda")
    gen.manual_seed(1234)
    ws, wo = learned.init_weights(qc, T)
    ws.requires_grad_()
    wo.requires_grad_()
    opt = torch.optim.Adam([ws, wo], lr=0.02)
    for _ in range(150):
        llr, syn, x = learned.make_batch(qc, 64, 0.2, 0.3, gen)
        opt.zero_grad()
        learned.minsum_loss(ws, wo, qc, llr, syn, x).mean().backward()
        opt.step()
    gen.manual_seed(99)
    llr, syn, x = learned.make_batch(qc, 512, 0.25, 0.25, gen)
    base_s, base_o = learned.init_weights(qc, T)

    def ber(s, o):
        h, _, _ = learned.decode(qc, llr, syn, s, o)
        return (h != x).float().mean().item()
    trained, plain = ber(ws, wo), ber(base_s, base_o)
    assert trained < 0.8 * plain, (trained, plain)


@pytest.mark.parametrize("Z,T", [(64, 6), (37, 4)])
def test_grouped_minsum_equals_the_frame_kernel(q, learned, Z, T):
    # qcmet_minsum_decode takes the grouped kernel for four frames or more and
    # the frame kernel for fewer; the two evaluate the rule identically
    code = synth.make_code("0.1", Z)
    fr = synth.make_frames(code, 8, 0.2, first=900)
    qc = q.Code(code.base, code.shifts, code.Z)
    ws, wo = weights(code, T, seed=5)
    ws, wo = torch.from_numpy(ws).cuda(), torch.from_numpy(wo).cuda()
    llr, syn = torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda()
    h, p, ok = learned.decode(qc, llr, syn, ws, wo)
    for k in range(0, 8, 2):
        h2, p2, ok2 = learned.decode(qc, llr[k:k + 2].contiguous(), syn[k:k + 2].contiguous(), ws, wo)
        torch.cuda.synchronize()
        assert torch.equal(p[k:k + 2], p2) and torch.equal(h[k:k + 2], h2) and torch.equal(ok[k:k + 2], ok2)


def test_grouped_minsum_with_two_groups_per_cluster(q, learned):
    # 192 frames of the full-size code: the launch chooser gives a cluster two
    # groups when that leaves fewer checks per SM; frames of both groups of a
    # cluster (blocks that straddle them included) equal the frame kernel's
    code = synth.make_code("0.1", 12500)
    qc = q.Code(code.base, code.shifts, code.Z)
    plan = q.group_plan(qc, 192)
    if plan["groups_per_cluster"] != 2:
        pytest.skip(f"the chooser keeps one group per cluster on this device: {plan}")
    T = 3
    fr = synth.make_frames(code, 192, 0.2, first=1200)
    ws, wo = weights(code, T, seed=6)
    ws, wo = torch.from_numpy(ws).cuda(), torch.from_numpy(wo).cuda()
    llr, syn = torch.from_numpy(fr.llr).cuda(), torch.from_numpy(fr.syn).cuda()
    h, p, ok = learned.decode(qc, llr, syn, ws, wo)
    for k in (0, 4, 6, 186, 190):
        h2, p2, ok2 = learned.decode(qc, llr[k:k + 2].contiguous(), syn[k:k + 2].contiguous(), ws, wo)
        torch.cuda.synchronize()
        assert torch.equal(p[k:k + 2], p2) and torch.equal(h[k:k + 2], h2) and torch.equal(ok[k:k + 2], ok2)
