"""Batched (level-merged, graph-replayed) evaluation: bit-exact against the
per-request plain evaluator and the oracle, with requests from several
client key sets in one batch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from oracle import circuit, evaluate, fixedpoint as fx, gsw  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import image_2d, signal_1d  # noqa: E402

REQS = [(8, 1, 8, 4), (4, 1, 6, 2), (2, 4, 8, 3), (16, 1, 8, 4), (4, 1, 6, 2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


def _inputs(sp, reqs):
    """Per-request signals, key sets (request index mod 3) and device ciphertexts."""
    cw = sf.ct_words(sp)
    keys = {ks: sf.keygen(sp, 100 + ks) for ks in range(3)}
    pubs = {ks: torch.from_numpy(k.public().view(np.int32)).cuda() for ks, k in keys.items()}
    cts, sigs = [], []
    for r, (N1, N2, F, f) in enumerate(reqs):
        re_, im_ = signal_1d(N1 * N2, -1, 1, r) if N2 == 1 else image_2d(N1, N2, r)
        d = torch.empty((N1 * N2 * 2 * F, cw), dtype=torch.int32, device="cuda")
        sf.encrypt_bits_device(sp, pubs[r % 3], re_, im_, F, f, 7 + r, d)
        cts.append(d)
        sigs.append((re_, im_))
    return keys, cts, sigs


def _single(sp, req, d_in, flags=0):
    plan = sf.Plan(sp, *req, flags=flags)
    out = torch.empty((plan.info["outputs"], plan.info["ct_words"]), dtype=torch.int32, device="cuda")
    scr = torch.empty(max(1, plan.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    plan.eval_fft(d_in, out, scr)
    plan.check()
    return out


@pytest.mark.parametrize("pset,flags", [("P0", 0), ("P2", 0), ("P2", sf.PLAN_INT_KERNEL)])
def test_batch_equals_per_request_plans(pset, flags):
    sp = sf.param_set(pset)
    keys, cts, _ = _inputs(sp, REQS)
    batch = sf.Batch(sp, REQS, flags)
    info = batch.info
    assert info["inputs"] == sum(len(c) for c in cts)
    d_in = torch.cat(cts)
    out = torch.empty((info["outputs"], info["ct_words"]), dtype=torch.int32, device="cuda")
    scr = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for _ in range(2):                       # capture, then replay
            out.fill_(-1)
            batch.eval(d_in, out, scr, stream)
            batch.check(stream)
            for r, req in enumerate(REQS):
                want = _single(sp, req, cts[r], flags)
                got = out[batch.out_off[r]:batch.out_off[r] + len(want)]
                assert torch.equal(got, want), (r, req)


def test_batch_graph_replay_equals_plain_launches():
    sp = sf.param_set("P2")
    _, cts, _ = _inputs(sp, REQS[:3])
    d_in = torch.cat(cts)
    res = []
    stream = torch.cuda.Stream()
    for flags in (0, sf.BATCH_NO_GRAPH):
        b = sf.Batch(sp, REQS[:3], flags)
        out = torch.zeros((b.info["outputs"], b.info["ct_words"]), dtype=torch.int32, device="cuda")
        scr = torch.empty(max(1, b.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
        with torch.cuda.stream(stream):
            b.eval(d_in, out, scr, stream)
            b.check(stream)
        res.append(out)
    assert torch.equal(res[0], res[1])


def test_batch_request_matches_oracle_and_decrypts():
    """One request of a mixed-key batch against the oracle's ciphertexts."""
    sp = sf.param_set("P2")
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    reqs = [(4, 1, 6, 2), (8, 1, 8, 4)]
    keys, cts, sigs = _inputs(sp, reqs)
    b = sf.Batch(sp, reqs)
    d_in = torch.cat(cts)
    out = torch.empty((b.info["outputs"], b.info["ct_words"]), dtype=torch.int32, device="cuda")
    scr = torch.empty(max(1, b.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.eval(d_in, out, scr, stream)
        b.check(stream)
    r = 1
    N, _, F, f = reqs[r]
    re_, im_ = sigs[r]
    ko = gsw.Keys(p, 100 + r % 3)
    c = circuit.fft_circuit(N, 1, F, f)
    ins = []
    for k in range(N):
        for part, x in enumerate((re_[k], im_[k])):
            for bit_i, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                ins.append(gsw.encrypt(ko, bit, 7 + r, (2 * k + part) * F + bit_i))
    want = evaluate.eval_encrypted(c, p, ins)
    got = out[b.out_off[r]:b.out_off[r] + len(want)].cpu().numpy().view(np.uint32)
    assert np.array_equal(got.reshape(want.shape), want)
    W = (p.n + 1) * p.L
    rows = got.reshape(len(want), -1)[:, (p.ell - 1) * W:p.ell * W]
    _, _, raw = sf.decrypt(keys[r % 3], rows, W, N, F, f)
    q = [fx.quantize(x, F, f) for x in re_]
    er, ei = fx.fft_int(q, [0] * N, F, f)
    assert list(raw) == [v for k in range(N) for v in (er[k], ei[k])]


@pytest.mark.parametrize("pset", ["P0", "P2"])
def test_pipelined_host_evaluation(pset):
    """Five steps through two device buffer sets with the copies on their own
    streams: every step's host output equals the batch's device-path result
    for that step's inputs (different inputs per step, one repeated)."""
    sp = sf.param_set(pset)
    reqs = REQS[:3]
    batch = sf.Batch(sp, reqs)
    info = batch.info
    cw = info["ct_words"]
    keys = sf.keygen(sp, 5)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    steps_in = []
    for s in range(3):   # different plaintexts and randomness per step
        cts = []
        for r, (N1, N2, F, f) in enumerate(reqs):
            re_, im_ = signal_1d(N1 * N2, -1, 1, 10 * s + r) if N2 == 1 else image_2d(N1, N2, 10 * s + r)
            d = torch.empty((N1 * N2 * 2 * F, cw), dtype=torch.int32, device="cuda")
            sf.encrypt_bits_device(sp, pub, re_, im_, F, f, 50 + 10 * s + r, d)
            cts.append(d)
        steps_in.append(cts)
    h_ins = [torch.cat(c).cpu().pin_memory() for c in steps_in]
    order = [0, 1, 2, 0, 1]
    stream = torch.cuda.Stream()
    d_ins = [torch.empty((info["inputs"], cw), dtype=torch.int32, device="cuda") for _ in range(2)]
    d_outs = [torch.empty((info["outputs"], cw), dtype=torch.int32, device="cuda") for _ in range(2)]
    scr = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    h_outs = [torch.empty((info["outputs"], cw), dtype=torch.int32).pin_memory() for _ in order]
    batch.eval_host_pipelined([h_ins[i] for i in order], h_outs, d_ins, d_outs, scr, stream)
    # reference: the device path, one step at a time
    ref_out = torch.empty((info["outputs"], cw), dtype=torch.int32, device="cuda")
    for i, h_out in zip(order, h_outs):
        with torch.cuda.stream(stream):
            batch.eval(h_ins[i].cuda(), ref_out, scr, stream)
        batch.check(stream)
        torch.cuda.synchronize()
        assert torch.equal(h_out, ref_out.cpu())


PERSIST_REQS = [(16, 1, 16, 8), (8, 1, 8, 4), (4, 4, 8, 3), (32, 1, 16, 8), (8, 8, 16, 8),
                (64, 1, 16, 8), (4, 1, 6, 2)]


@pytest.mark.parametrize("pset,graph", [("P2", True), ("P2", False), ("P0", True)])
def test_persistent_batch_equals_level_by_level(pset, graph):
    """One persistent launch across all levels (gates claimed in program
    order, levels overlapping by one) against the level-by-level batch on the
    same inputs: identical ciphertexts, on three evaluations in a row (the
    epochs of the gates' done flags advance); at ell 128 and at the toy
    parameters (Ng 64)."""
    sp = sf.param_set(pset)
    _, cts, _ = _inputs(sp, PERSIST_REQS)
    d_in = torch.cat(cts)
    stream = torch.cuda.Stream()
    ref_b = sf.Batch(sp, PERSIST_REQS)
    ref = torch.empty((ref_b.info["outputs"], ref_b.info["ct_words"]), dtype=torch.int32, device="cuda")
    scr = torch.empty(max(1, ref_b.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        ref_b.eval(d_in, ref, scr, stream)
        ref_b.check(stream)
    pb = sf.Batch(sp, PERSIST_REQS, sf.BATCH_PERSISTENT | (0 if graph else sf.BATCH_NO_GRAPH))
    assert pb.info["gate_kernel"] == sf.KERNEL_SM and pb.info["products"] == ref_b.info["products"]
    pscr = torch.empty(max(1, pb.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    for _ in range(3):
        out = torch.full_like(ref, -1)
        with torch.cuda.stream(stream):
            pb.eval(d_in, out, pscr, stream)
            pb.check(stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_persistent_batch_across_the_epoch_wrap():
    """The run counter that the gates' done flags are compared with is 32
    bits; across its wrap the flags are cleared, so that the runs on either
    side of it still wait for their producers: identical outputs each time."""
    sp = sf.param_set("P2")
    reqs = PERSIST_REQS[:4]
    _, cts, _ = _inputs(sp, reqs)
    d_in = torch.cat(cts)
    stream = torch.cuda.Stream()
    ref_b = sf.Batch(sp, reqs)
    ref = torch.empty((ref_b.info["outputs"], ref_b.info["ct_words"]), dtype=torch.int32, device="cuda")
    scr = torch.empty(max(1, ref_b.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        ref_b.eval(d_in, ref, scr, stream)
        ref_b.check(stream)
    pb = sf.Batch(sp, reqs, sf.BATCH_PERSISTENT)
    pscr = torch.empty(max(1, pb.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    pb.set_epoch(0xFFFFFFFD, stream)
    for _ in range(4):   # epochs 0xFFFFFFFE, 0xFFFFFFFF, then 1 (flags cleared), 2
        out = torch.full_like(ref, -1)
        with torch.cuda.stream(stream):
            pb.eval(d_in, out, pscr, stream)
            pb.check(stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    with pytest.raises(sf.SfftError):   # the hook is for persistent batches only
        ref_b.set_epoch(1, stream)


def test_persistent_batch_request_matches_oracle():
    sp = sf.param_set("P2")
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    reqs = [(8, 1, 8, 4), (16, 1, 8, 4), (4, 1, 6, 2)]
    keys, cts, sigs = _inputs(sp, reqs)
    b = sf.Batch(sp, reqs, sf.BATCH_PERSISTENT)
    d_in = torch.cat(cts)
    out = torch.empty((b.info["outputs"], b.info["ct_words"]), dtype=torch.int32, device="cuda")
    scr = torch.empty(max(1, b.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.eval(d_in, out, scr, stream)
        b.check(stream)
    r = 0
    N, _, F, f = reqs[r]
    re_, im_ = sigs[r]
    ko = gsw.Keys(p, 100 + r % 3)
    ins = []
    for k in range(N):
        for part, x in enumerate((re_[k], im_[k])):
            for bit_i, bit in enumerate(fx.to_bits(fx.quantize(x, F, f), F)):
                ins.append(gsw.encrypt(ko, bit, 7 + r, (2 * k + part) * F + bit_i))
    want = evaluate.eval_encrypted(circuit.fft_circuit(N, 1, F, f), p, ins)
    got = out[b.out_off[r]:b.out_off[r] + len(want)].cpu().numpy().view(np.uint32)
    assert np.array_equal(got.reshape(want.shape), want)


def test_persistent_batch_rejects_unsupported_forms():
    with pytest.raises(sf.SfftError):   # general tensor-core kernel (Ng > 256)
        sf.Batch(sf.param_set("P1", 224), [(8, 1, 8, 4)], sf.BATCH_PERSISTENT)
    with pytest.raises(sf.SfftError):   # linear (exclusive-carry) gates
        sf.Batch(sf.param_set("P2"), [(8, 1, 8, 4)], sf.BATCH_PERSISTENT | sf.PLAN_XCARRY)


def test_full_c4_batch_equals_plain_path_persistent_form_and_oracle():
    """The 256-request batch workload (the bench's batch256_p2 inputs: N 16 to
    128, 16- and 24-bit words, four key sets) evaluated as one graph-replayed
    batch: every request's ciphertexts equal its own plan's (the plain path)
    and the persistent form's; the smallest request also equals the oracle's
    encrypted evaluation."""
    from synthetic import batch_requests
    sp = sf.param_set("P2")
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    cw = sf.ct_words(sp)
    reqs = batch_requests(count=256, seed=4, key_sets=4)
    dims = [(r.N1, r.N2, r.F, r.f) for r in reqs]
    pubs = {ks: torch.from_numpy(sf.keygen(sp, 1000 + ks).public().view(np.int32)).cuda()
            for ks in range(4)}
    b = sf.Batch(sp, dims)
    d_in = torch.empty((b.info["inputs"], cw), dtype=torch.int32, device="cuda")
    for i, r in enumerate(reqs):
        n = r.N1 * r.N2 * 2 * r.F
        sf.encrypt_bits_device(sp, pubs[r.key_set], r.re, r.im, r.F, r.f, r.seed,
                               d_in[b.in_off[i]:b.in_off[i] + n])
    out = torch.empty((b.info["outputs"], cw), dtype=torch.int32, device="cuda")
    pb = sf.Batch(sp, dims, sf.BATCH_PERSISTENT)
    assert list(pb.in_off) == list(b.in_off) and list(pb.out_off) == list(b.out_off)
    scr = torch.empty(max(b.info["scratch_bytes"], pb.info["scratch_bytes"]) // 4 + 1,
                      dtype=torch.int32, device="cuda")
    pout = torch.full_like(out, -1)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        b.eval(d_in, out, scr, stream)
        b.check(stream)
        pb.eval(d_in, pout, scr, stream)
        pb.check(stream)
    torch.cuda.synchronize()
    assert torch.equal(pout, out)
    for i, r in enumerate(reqs):
        n = r.N1 * r.N2 * 2 * r.F
        want = _single(sp, dims[i], d_in[b.in_off[i]:b.in_off[i] + n])
        assert torch.equal(out[b.out_off[i]:b.out_off[i] + len(want)], want), (i, dims[i])
    i = min(range(len(reqs)), key=lambda k: (reqs[k].N1 * reqs[k].F, k))
    r = reqs[i]
    ko = gsw.Keys(p, 1000 + r.key_set)
    ins = []
    for k in range(r.N1):
        for part, x in enumerate((r.re[k], r.im[k])):
            for bit_i, bit in enumerate(fx.to_bits(fx.quantize(x, r.F, r.f), r.F)):
                ins.append(gsw.encrypt(ko, bit, r.seed, (2 * k + part) * r.F + bit_i))
    want = evaluate.eval_encrypted(circuit.fft_circuit(r.N1, 1, r.F, r.f), p, ins)
    got = out[b.out_off[i]:b.out_off[i] + len(want)].cpu().numpy().view(np.uint32)
    assert np.array_equal(got.reshape(want.shape), want)
