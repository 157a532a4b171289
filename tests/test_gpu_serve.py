"""Serving loop: continuous batching keeps every result identical to the same
request evaluated alone (bit for bit), whatever else shares its launches."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1611_08769_gb300 as sf  # noqa: E402
from paper_1611_08769_gb300 import build as sfbuild  # noqa: E402
from synthetic import image_2d, signal_1d  # noqa: E402

SHAPES = [(8, 1, 8, 4), (4, 1, 6, 2), (2, 4, 8, 3), (16, 1, 8, 4), (4, 4, 8, 3), (8, 1, 6, 2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sfbuild.build()


def _request_inputs(sp, shape, key_set, seed):
    N1, N2, F, f = shape
    keys = sf.keygen(sp, 300 + key_set)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    re_, im_ = signal_1d(N1 * N2, -1, 1, seed) if N2 == 1 else image_2d(N1, N2, seed)
    d = torch.empty((N1 * N2 * 2 * F, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, pub, re_, im_, F, f, seed, d)
    return d


def _alone(sp, shape, d_in):
    plan = sf.Plan(sp, *shape)
    out = torch.empty((plan.info["outputs"], plan.info["ct_words"]), dtype=torch.int32, device="cuda")
    scr = torch.empty(max(1, plan.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    plan.eval_fft(d_in, out, scr)
    plan.check()
    return out.cpu()


@pytest.mark.parametrize("pset,budget_kb", [("P0", 1024), ("P2", 90 * 1024)])
def test_served_results_equal_alone(pset, budget_kb):
    """Budgets hold only a few requests at once, so later ones queue for memory."""
    sp = sf.param_set(pset)
    reqs = []
    for k in range(12):
        shape = SHAPES[k % len(SHAPES)]
        d_in = _request_inputs(sp, shape, k % 4, 50 + k)
        h_in = d_in.cpu().pin_memory()
        h_out = torch.zeros((shape[0] * shape[1] * 2 * shape[2], sf.ct_words(sp)),
                            dtype=torch.int32).pin_memory()
        reqs.append((shape, d_in, h_in, h_out))
    srv = sf.Server(sp, budget_kb << 10, max_active=8)
    try:
        tickets = []
        for k, (shape, _, h_in, h_out) in enumerate(reqs):
            tickets.append(srv.submit(shape, h_in, h_out))
            if k == 5:
                time.sleep(0.05)          # the second half arrives while the first runs
        lat = [srv.wait(t) for t in tickets]
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == len(reqs)
    assert all(x > 0 for x in lat)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for shape, d_in, _, h_out in reqs:
        assert torch.equal(h_out, _alone(sp, shape, d_in)), shape


def test_request_beyond_budget_is_rejected():
    sp = sf.param_set("P2")
    srv = sf.Server(sp, 120 << 20, max_active=4)
    try:
        big = np.zeros((64 * 2 * 16, sf.ct_words(sp)), dtype=np.uint32)
        out = np.zeros_like(big)
        with pytest.raises(sf.SfftError):
            srv.submit((64, 1, 16, 8), big, out)     # 16,970 ciphertexts = 139 MB > the arena
        with pytest.raises(sf.SfftError):
            srv.wait(12345, timeout_ms=10)          # unknown ticket
    finally:
        srv.close()


def test_served_request_matches_oracle():
    """One request served in a mix of others (different shapes and client
    keys, a budget that makes later requests wait, one large request that
    the admission lets smaller ones pass) is compared ciphertext for
    ciphertext with the oracle's encrypted evaluation of the same circuit on
    the same encryptions (toy noise-free parameters)."""
    from oracle import circuit, evaluate, fixedpoint as fx, gsw
    sp = sf.param_set("P0")
    p = gsw.Params(sp.n, sp.ell, sp.m, sp.chi)
    shape = (8, 1, 8, 4)
    key_seed, enc_seed = 77, 13
    re_, im_ = signal_1d(8, -1, 1, 5)
    keys = sf.keygen(sp, key_seed)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    d_in = torch.empty((8 * 2 * 8, sf.ct_words(sp)), dtype=torch.int32, device="cuda")
    sf.encrypt_bits_device(sp, pub, re_, im_, 8, 4, enc_seed, d_in)
    target = (shape, d_in.cpu().pin_memory(), torch.zeros((8 * 2 * 8, sf.ct_words(sp)), dtype=torch.int32).pin_memory())
    mix = [((16, 16, 12, 2), None)] + [(SHAPES[k % len(SHAPES)], None) for k in range(8)]
    others = []
    for k, (sh, _) in enumerate(mix):
        di = _request_inputs(sp, sh, k % 3, 90 + k)
        others.append((sh, di.cpu().pin_memory(),
                       torch.zeros((sh[0] * sh[1] * 2 * sh[2], sf.ct_words(sp)), dtype=torch.int32).pin_memory()))
    # 23 MB: the 16 x 16 image (21.6 MB of ciphertexts) fits only once the
    # first small requests have left, and the later small ones pass it
    srv = sf.Server(sp, 23 << 20, max_active=8)
    try:
        tickets = [srv.submit(sh, hi, ho) for sh, hi, ho in others[1:4]]
        tickets.append(srv.submit(*others[0]))
        t_target = srv.submit(*target)
        tickets += [srv.submit(sh, hi, ho) for sh, hi, ho in others[4:]]
        srv.wait(t_target)
        for t in tickets:
            srv.wait(t)
    finally:
        srv.close()
    got = target[2].numpy().view(np.uint32).reshape(-1, p.Ng, p.n + 1, p.L)
    ko = gsw.Keys(p, key_seed)
    c = circuit.fft_circuit(*shape)
    cts = []
    for k in range(8):
        for part, x in enumerate((re_[k], im_[k])):
            for b, bit in enumerate(fx.to_bits(fx.quantize(x, 8, 4), 8)):
                cts.append(gsw.encrypt(ko, bit, enc_seed, (2 * k + part) * 8 + b))
    want = evaluate.eval_encrypted(c, p, cts)
    assert np.array_equal(got, want)
