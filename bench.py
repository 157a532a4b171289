"""Benchmark of the encrypted FFT on GB300 (one JSON line on rank 0).

Default workload (fft64_16bit_noisy): 1-D encrypted FFT, N = 64, 16-bit
two's-complement fixed point (8 integer, 8 fraction bits), real inputs uniform
in [-8, 8), imaginary part 0, one request, under the noisy leveled GSW
parameters (n = 1, chi = 1, m = Ng, ell = the smallest multiple of 32 whose
static noise bound stays below q/4: 1056). One step = one evaluation of the
whole FFT circuit on the device (every gate of every level), inputs resident
in HBM. `value` is the batched form (level program replayed as one CUDA
graph); the plain level-by-level evaluator is timed beside it.

Other workloads (--config): fft8_8bit_toy (toy noise-free parameters),
fft16x16_image_noisy (2-D row-column FFT of a 16 x 16 image, 10.6 words),
batch256_p2 (256 independent 1-D FFTs, N in {16..128}, F in {16, 24}, four
client key sets, one graph-replayed level-merged batch; noise-free ell 128),
fft64_16bit_xcarry (the default workload built with exclusive-carry full
adders, a circuit variant: fewer products, its own smaller ell),
fft8_8bit_nand (8-point 8-bit FFT built from NAND gates only, the paper's
literal gate construction, at its own smallest ell), fft64_16bit_enctw_xcarry
(the default workload with encrypted twiddles and the encrypted-operand
multiplier, exclusive-carry adders), fft64_16bit_enctw (the same with the
paper's adders, ell 1440), refresh32_noisy (refresh by homomorphic
decryption of 32 ciphertexts at the default workload's ell; metric:
refreshed ciphertexts/s).

The default run (no --config) adds two blocks measured on the same box
after the headline: "batch" (batch256_p2, the level-merged batch of 256
requests replayed as a graph against the plain per-request evaluator, with
its roofline and the autotuned ring depth of the small-ciphertext kernel) and
"serve" (serve_p2: Poisson arrivals at 0.8x the measured closed-burst
capacity into the continuous-batching server, p50/p99 latency); --no-extra
skips them.

Keys beyond the base contract:
  roofline      the gate-product kernel against its peak (tensor or ALU)
  cpu_baseline  the CPU oracle on a bounded prefix of the same circuit
  e2e           same metric through the host-buffer C ABI call (H2D of the
                input ciphertexts and D2H of the outputs timed every step)
  plain         the plain level-by-level evaluator on the same workload
  gates_per_s   ciphertext products per second
Multi-GPU (torchrun): every rank runs an independent replica (one request's
FFT does not shard); value = FFTs/s summed over ranks.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Integer-pipe rates measured on this GPU by the library's microbenchmark
# (sfft_measure_int_peak: add.u32, lop3, mad.lo, popc; ops/s), filled once
# per process by int_peaks(); the integer kernel's roofline is taken against
# the measured add rate.
_INT_PEAKS = {}


def int_peaks(sf):
    if not _INT_PEAKS:
        for name in sf.INT_PEAK_OPS:
            _INT_PEAKS[name] = sf.measure_int_peak(name)
    return dict(_INT_PEAKS)

DEFAULT_CONFIG = "fft64_16bit_noisy"

CONFIGS = {
    # single-request FFTs: (N1, N2, F, f, lo, hi, parameter set)
    "fft64_16bit_noisy": dict(kind="fft", N1=64, N2=1, F=16, f=8, lo=-8.0, hi=8.0, pset="P1"),
    "fft8_8bit_toy": dict(kind="fft", N1=8, N2=1, F=8, f=4, lo=-1.0, hi=1.0, pset="P0"),
    "fft16x16_image_noisy": dict(kind="fft", N1=16, N2=16, F=16, f=6, lo=None, hi=None, pset="P1"),
    "fft64_16bit_p2": dict(kind="fft", N1=64, N2=1, F=16, f=8, lo=-8.0, hi=8.0, pset="P2"),
    # circuit variant: exclusive-carry full adders (linear carry gates, smaller ell)
    "fft64_16bit_xcarry": dict(kind="fft", N1=64, N2=1, F=16, f=8, lo=-8.0, hi=8.0, pset="P1",
                               xcarry=True),
    # the paper's literal NAND-only gates
    "fft8_8bit_nand": dict(kind="fft", N1=8, N2=1, F=8, f=4, lo=-1.0, hi=1.0, pset="P1",
                           nand=True),
    # encrypted twiddles (encrypted-operand Wallace multiplier), exclusive-carry adders
    "fft64_16bit_enctw_xcarry": dict(kind="fft", N1=64, N2=1, F=16, f=8, lo=-8.0, hi=8.0,
                                     pset="P1", xcarry=True, enc_twiddle=True),
    # encrypted twiddles with the paper's adders (ell 1440, 288 digit columns)
    "fft64_16bit_enctw": dict(kind="fft", N1=64, N2=1, F=16, f=8, lo=-8.0, hi=8.0,
                              pset="P1", enc_twiddle=True),
    # refresh of 32 ciphertexts at the ell of the 64-point 16-bit workload
    "refresh32_noisy": dict(kind="refresh", count=32, pset="P1", ell_of=(64, 1, 16, 8)),
    "batch256_p2": dict(kind="batch", count=256, pset="P2", key_sets=4),
    "serve_p2": dict(kind="serve", pset="P2", key_sets=8, requests=400, calib=48),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=DEFAULT_CONFIG, choices=sorted(CONFIGS))
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="budget of the bounded oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain evaluator")
    ap.add_argument("--mode", default="fft", choices=["fft", "gates"],
                    help="fft: the workload (default); gates: one level of independent random "
                         "gates at the workload's parameters")
    ap.add_argument("--gates", type=int, default=128, help="gates per level in --mode gates")
    ap.add_argument("--kernel", default="auto", choices=["auto", "int", "tc", "sm"],
                    help="gate kernel: automatic, integer ALU, general tensor-core, "
                         "small-ciphertext tensor-core")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving HBM admission budget")
    ap.add_argument("--requests", type=int, default=0, help="serving: requests in the trace")
    ap.add_argument("--no-extra", action="store_true",
                    help="default workload only: skip the batch and serve blocks")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests of the serve block of the default run")
    return ap.parse_args()


class ClockSampler:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 4 + k and s[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def max_over_ranks(x, world, device):
    """The largest of every rank's x (the slowest replica times the job)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, ms, world):
    """Whole-job units per second: every rank runs its own replica of the
    workload in ms (the maximum over ranks)."""
    return world * units_per_rank * 1000.0 / ms


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "of measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "of fallback"


# DRAM bytes (read + write) per product of the tensor-core gate kernel, from an
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of one launch over
# a 512-gate level at n = 1, ell = 1056, inputs larger than L2), keyed by
# (n, ell). The algorithmic bytes of a product at these parameters are 3.07 MB:
# the expanded B operand once, the A and B rows, the two output rows.
TC_DRAM_BYTES_PER_PRODUCT = {(1, 1056): 3.101e6}
# The same for the small-ciphertext kernel (k_gate_sm), from an ncu capture of
# one launch over a 40,000-gate level of half adders at n = 1, ell = 128 (1.31
# GB, larger than L2): 656.4 MB read + 608.4 MB written. Half adders write two
# outputs; an FFT level mixes in single-output gates, so this figure is an
# upper estimate for FFT levels.
SM_DRAM_BYTES_PER_PRODUCT = {(1, 128): 31620.0}


def expand_bytes_per_product(params):
    """Algorithmic bytes of k_expand_b per product: B' read once (Ng rows of
    (n+1) ell bits) and its tensor-core image written once (per 128-row K
    step two atoms of (n+1) ceil16(ceil(ell / 11)) digit rows x 128 bytes)."""
    Ng = (params.n + 1) * params.ell
    ndpad = (params.n + 1) * ((-(-params.ell // 11) + 15) // 16 * 16)
    return Ng * Ng // 8 + -(-Ng // 128) * ndpad * 256


def roofline(params, gate_kernel, gate_ms, launches, gates_timed, tc_columns=0, expand_ms=None):
    """Roofline of the dominant kernel (the gate product) from CUDA-event times.

    Integer kernel: unit = one product = Ng^2 (n+1) L 32-bit limb additions,
    against the measured add rate. Tensor-core kernel: unit = one product =
    the scope table's algorithmic contraction, 2 Ng^2 (n+1) ell / 8 flops (the
    bits times byte digits of B'), against the measured dense bf16 rate
    (kind::f16 runs fp16 at the bf16 rate); the sustained figure, since the
    kernel runs inside a long step. The kernel computes the same sums with
    11-bit digits, fewer flops: `executed` gives its own MMA flops (2 Ng^2 C,
    C = (n+1) ceil(ell / 11) digit columns per row) against the same peak.
    With the tensor-core path, `expand` gives the B expansion (k_expand_b,
    HBM-bound) against the measured copy rate from its own events.
    """
    Ng, L = (params.n + 1) * params.ell, params.ell // 32
    W = (params.n + 1) * L
    avg_launch_ms = gate_ms / max(1, launches)
    sec = gate_ms / 1000.0 if gate_ms > 0 else float("inf")
    if gate_kernel == 3:
        # small-ciphertext kernel: HBM-bound; algorithmic bytes per product =
        # two ciphertexts read and one written, 3 Ng^2 / 8
        peaks, src = measured_peaks()
        bpp = 3.0 * Ng * Ng / 8
        achieved = bpp * gates_timed / sec / 1e9
        hbm = float(peaks["hbm_gbs"])
        cols = tc_columns or (params.n + 1) * params.ell // 8
        ncols = (cols + 15) // 16 * 16
        flops = 2.0 * Ng * Ng * ncols * gates_timed / sec / 1e12
        tpk = float(peaks["bf16_tflops_sustained"])
        per = SM_DRAM_BYTES_PER_PRODUCT.get((params.n, params.ell))
        return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm,
                "traffic": per * gates_timed / max(1, launches) if per else None,
                "traffic_unit": "bytes per launch", "kernel": "k_gate_sm",
                "avg_launch_ms": avg_launch_ms, "bytes_per_product": bpp,
                "peak_source": f"hbm_gbs {src}",
                "tensor": {"achieved": flops, "peak": tpk, "unit": "TFLOP/s", "frac": flops / tpk,
                           "flops_per_product": 2.0 * Ng * Ng * ncols,
                           "peak_source": f"bf16_tflops_sustained {src}"}}
    if gate_kernel == 2:
        peaks, src = measured_peaks()
        cols = tc_columns or (params.n + 1) * -(-params.ell // 11)
        fpp = 2.0 * Ng * Ng * (params.n + 1) * params.ell / 8
        achieved = fpp * gates_timed / sec / 1e12
        executed = 2.0 * Ng * Ng * cols * gates_timed / sec / 1e12
        peak = float(peaks["bf16_tflops_sustained"])
        per = TC_DRAM_BYTES_PER_PRODUCT.get((params.n, params.ell))
        traffic = per * gates_timed / max(1, launches) if per else None
        out = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
               "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
               "kernel": "k_gate_tc", "avg_launch_ms": avg_launch_ms,
               "flops_per_product": fpp,
               "flops_definition": "2 Ng^2 (n+1) ell / 8 per product (bits x byte digits of B')",
               "peak_source": f"bf16_tflops_sustained {src}",
               "executed": {"achieved": executed, "frac": executed / peak,
                            "flops_per_product": 2.0 * Ng * Ng * cols,
                            "definition": "the kernel's MMA flops: 2 Ng^2 x digit columns "
                                          "(11-bit digits)"}}
        if expand_ms:
            xb = expand_bytes_per_product(params)
            xa = xb * gates_timed / (expand_ms / 1000.0) / 1e9
            hbm = float(peaks["hbm_gbs"])
            out["expand"] = {"kernel": "k_expand_b", "bound": "hbm", "achieved": xa, "peak": hbm,
                             "unit": "GB/s", "frac": xa / hbm, "bytes_per_product": xb,
                             "avg_launch_ms": expand_ms / max(1, launches),
                             "peak_source": f"hbm_gbs {src}"}
        return out
    ops = float(Ng) * Ng * (params.n + 1) * L * gates_timed
    achieved = ops / sec
    peak = _INT_PEAKS.get("iadd3")
    if not peak:
        raise RuntimeError("integer peak not measured (call int_peaks first)")
    return {"bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "Tops/s (32-bit limb adds)", "frac": achieved / peak, "traffic": None,
            "kernel": "k_gate_generic", "avg_launch_ms": avg_launch_ms,
            "peak_source": "measured on this GPU: add.u32 rate (sfft_measure_int_peak)"}


def variant_of(cfg):
    """Circuit variant switches of a config (keyword arguments of min_ell and
    the oracle's fft_circuit)."""
    c = CONFIGS[cfg]
    return {k: bool(c.get(k, False)) for k in ("xcarry", "nand", "enc_twiddle")}


def kernel_flags(sf, kernel):
    """Plan flags of --kernel (auto and sm: the library's choice)."""
    return {"int": sf.PLAN_INT_KERNEL, "tc": sf.PLAN_TC_KERNEL}.get(kernel, 0)


def flags_of(sf, cfg):
    v = variant_of(cfg)
    return ((sf.PLAN_XCARRY if v["xcarry"] else 0) | (sf.PLAN_NAND if v["nand"] else 0)
            | (sf.PLAN_ENC_TWIDDLE if v["enc_twiddle"] else 0))


# The fixed parameter sets of the workloads, (n, ell, m, chi); P1 takes the
# smallest safe ell of its circuit (chi = 1, m = Ng).
PSETS = {"P0": (1, 32, 64, 0), "P2": (1, 128, 256, 0)}


def workload_items(cfg):
    """[(dims, re, im, key_set, enc_seed)] of a config: seeded synthetic
    signals only (no scheme code)."""
    from synthetic import batch_requests, image_2d, serving_trace, signal_1d
    c = CONFIGS[cfg]
    if c["kind"] == "batch":
        reqs = batch_requests(count=c["count"], seed=4, key_sets=c["key_sets"])
        return [((r.N1, r.N2, r.F, r.f), r.re, r.im, r.key_set, i) for i, r in enumerate(reqs)]
    if c["kind"] == "serve":   # a sample of the serving trace's requests
        trace = serving_trace(16, 1.0, seed=6, key_sets=c["key_sets"])
        return [((r.N1, r.N2, r.F, r.f), r.re, r.im, r.key_set, r.seed) for r in trace]
    dims = (c["N1"], c["N2"], c["F"], c["f"])
    if c["N2"] == 1:
        re_, im_ = signal_1d(c["N1"], c["lo"], c["hi"], seed=0)
    else:
        re_, im_ = image_2d(c["N1"], c["N2"], seed=0)
    return [(dims, re_, im_, 0, 0)]


def _p1_dims(cfg, items):
    c = CONFIGS[cfg]
    return [c["ell_of"]] if c["kind"] == "refresh" else sorted({d for d, *_ in items})


def product_params(sf, cfg, items=()):
    """Parameters of a config from the library (its own smallest ell for P1)."""
    c = CONFIGS[cfg]
    if c["pset"] != "P1":
        return sf.Params(*PSETS[c["pset"]][:2], PSETS[c["pset"]][2], PSETS[c["pset"]][3])
    var = {} if c["kind"] == "refresh" else variant_of(cfg)
    ell = max(sf.min_ell(*d, n=1, chi=1, **var) for d in _p1_dims(cfg, items))
    return sf.param_set("P1", ell)


def oracle_params(cfg, items=()):
    """Parameters of a config from the oracle alone (oracle.noise.smallest_ell
    over the oracle's own circuits for P1): what the reference arm and the CPU
    baseline run, independent of the library."""
    from oracle import circuit, gsw, noise
    c = CONFIGS[cfg]
    if c["pset"] != "P1":
        return gsw.Params(*PSETS[c["pset"]])
    var = {} if c["kind"] == "refresh" else variant_of(cfg)
    ell = max(noise.smallest_ell(circuit.fft_circuit(*d, **var), 1, 1) for d in _p1_dims(cfg, items))
    return gsw.Params(1, ell, 2 * ell, 1)


def fft_inputs(twiddles, dims, re_, im_, enc_twiddle):
    """(re, im) values encrypted for one request: the signal, then (with
    encrypted twiddles) the twiddle table W_M^k, M = max(N1, N2), as exact
    fixed-point values; twiddles(M, f) gives the quantised (wr, wi) lists."""
    N1, N2, F, f = dims
    if not enc_twiddle:
        return list(re_), list(im_)
    wr, wi = twiddles(max(N1, N2), f)
    return (list(re_) + [w / 2 ** f for w in wr],
            list(im_) + [w / 2 ** f for w in wi])


def product_twiddles(sf):
    def tw(M, f):
        wr, wi = sf.twiddles(M, f)
        return wr.tolist(), wi.tolist()
    return tw


def oracle_twiddles(M, f):
    from oracle import circuit
    tw = circuit.twiddles(M, f)
    return [w[0] for w in tw], [w[1] for w in tw]


def workload(sf, cfg):
    """(params, items) of a single-request, batch or serving config for the
    library's arm."""
    items = workload_items(cfg)
    return product_params(sf, cfg, items), items


def oracle_gate_prefix(c, p, input_bit, budget_s):
    """Times the oracle's gates of circuit c in order until budget_s of gate
    time is spent. Inputs are encrypted on first use (untimed); input_bit(w)
    gives the plaintext bit of input wire w. Returns (gates done, seconds)."""
    from oracle import circuit, gsw
    keys = gsw.Keys(p, 0)
    cts = {}
    zero, one = gsw.zero_ct(p), gsw.one_ct(p)

    def get(w):
        if w == circuit.ZERO:
            return zero
        if w == circuit.ONE:
            return one
        if w not in cts:
            cts[w] = gsw.encrypt(keys, input_bit(w), 0, w)
        return cts[w]

    done, dt = 0, 0.0
    for op, a, b, o in c.gates:
        A, B = (b, a) if (b is not None and c.d(b) > c.d(a)) else (a, b)
        xa, xb = get(A), None if B is None else get(B)
        t1 = time.perf_counter()
        cts[o] = gsw.gate(p, xa, xb, gsw.GATE_CODES[op])
        dt += time.perf_counter() - t1
        done += 1
        if dt > budget_s:
            break
    return done, dt


def cpu_oracle_sample(params, items, budget_s, variant=None):
    """Oracle on a bounded prefix of the first request's circuit.

    Returns (FFTs/s, gates/s, description). FFT time is the per-gate time
    times the mean oracle gate count of the workload's distinct FFT shapes."""
    from oracle import circuit, fixedpoint as fx, gsw
    variant = variant or {}
    p = gsw.Params(params.n, params.ell, params.m, params.chi)
    (N1, N2, F, f), re_, im_, _, _ = items[0]
    c = circuit.fft_circuit(N1, N2, F, f, **variant)
    re_all, im_all = fft_inputs(oracle_twiddles, (N1, N2, F, f), re_, im_,
                                variant.get("enc_twiddle", False))

    def input_bit(w):   # wire (sample * 2 + part) * F + bit, twiddles after the signal
        sample, rem = divmod(w, 2 * F)
        part, bit = divmod(rem, F)
        x = re_all[sample] if part == 0 else im_all[sample]
        return fx.to_bits(fx.quantize(x, F, f), F)[bit]

    done, dt = oracle_gate_prefix(c, p, input_bit, budget_s)
    per_gate = dt / done
    shapes = sorted({d for d, *_ in items})
    sizes = {d: (len(c.gates) if d == (N1, N2, F, f) else
                 len(circuit.fft_circuit(*d, **variant).gates)) for d in shapes}
    mean_gates = sum(sizes[d] for d, *_ in items) / len(items)
    fft_s = per_gate * mean_gates
    detail = (f"first {done} of {len(c.gates)} oracle gates (each logical gate evaluated separately) "
              f"of the {N1}x{N2} F={F} circuit at the same parameters, {dt:.1f} s; FFT time "
              f"extrapolated to {fft_s:.1f} s from the mean oracle gate count {mean_gates:.0f}")
    return 1.0 / fft_s, done / dt, detail


def cpu_refresh_sample(params, count, budget_s, xcarry=False):
    """Oracle on a bounded prefix of one refresh circuit (the worst-case
    selection: every key ciphertext selected). Returns (refreshes/s, gates/s,
    description); the time per refresh is extrapolated from the per-gate time."""
    from oracle import gsw, refresh
    p = gsw.Params(params.n, params.ell, params.m, params.chi)
    c = refresh.refresh_circuit(p, [None], xcarry=xcarry)
    done, dt = oracle_gate_prefix(c, p, lambda w: w % 2, budget_s)
    per = dt / done * len(c.gates)
    detail = (f"first {done} of {len(c.gates)} oracle gates of one refresh circuit (every key "
              f"ciphertext selected) at the same parameters, {dt:.1f} s; time per refreshed "
              f"ciphertext extrapolated to {per:.1f} s")
    return 1.0 / per, done / dt, detail


def run_reference(args, rank, world):
    if rank != 0:
        return
    budget = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    vals = []
    detail = ""
    if CONFIGS[args.config]["kind"] == "refresh":
        params, count = oracle_params(args.config), CONFIGS[args.config]["count"]
        metric, unit = "refreshed ciphertexts/s", "ct/s"
        cfg = refresh_config_json(args.config, params, count)
        sample = lambda: cpu_refresh_sample(params, count, budget,  # noqa: E731
                                            variant_of(args.config)["xcarry"])
    else:
        items = workload_items(args.config)
        params = oracle_params(args.config, items)
        metric, unit = "encrypted FFTs/s", "FFT/s"
        cfg = config_json(args.config, params, items)
        sample = lambda: cpu_oracle_sample(params, items, budget,  # noqa: E731
                                           variant_of(args.config))
    for s in range(args.warmup + args.steps):
        fps, gps, detail = sample()
        if s >= args.warmup:
            vals.append(fps)
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": metric, "value": v, "unit": unit,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / v, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": v, "unit": unit, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": detail},
            "e2e": {"value": v, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


CIRCUIT_NOTES = {
    "xcarry": "exclusive-carry full adders (variant; carries are linear gates)",
    "nand": "every gate built of GSW NAND gates (the paper's literal construction)",
    "enc_twiddle": "twiddles encrypted (inputs after the signal), encrypted-operand multiplier",
}


def config_json(cfg, params, items):
    out = {"workload": cfg, "n": params.n, "ell": params.ell, "m": params.m, "chi": params.chi,
           "requests": len(items)}
    notes = [CIRCUIT_NOTES[k] for k, on in variant_of(cfg).items() if on]
    if notes:
        out["circuit"] = "; ".join(notes)
    if len(items) == 1:
        (N1, N2, F, f), *_ = items[0]
        out.update({"N1": N1, "N2": N2, "F": F, "f": f})
    else:
        out["key_sets"] = len({it[3] for it in items})
    return out


def refresh_config_json(cfg, params, count):
    out = {"workload": cfg, "n": params.n, "ell": params.ell, "m": params.m, "chi": params.chi,
           "refreshed_per_step": count,
           "circuit": "homomorphic decryption of row ell - 1: Wallace sum of the top "
                      "ceil(log2(n ell + 1)) + 3 bits of n ell + 1 selected key ciphertexts"}
    notes = [CIRCUIT_NOTES[k] for k, on in variant_of(cfg).items() if on]
    if notes:
        out["circuit"] += "; " + "; ".join(notes)
    return out


def run_refresh(args):
    """Refresh of `count` ciphertexts per step (rank 0; replicas elsewhere)."""
    import torch

    import paper_1611_08769_gb300 as sf
    from paper_1611_08769_gb300 import build as sfbuild
    sfbuild.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(local)
    params, count = product_params(sf, args.config), CONFIGS[args.config]["count"]
    flags = kernel_flags(sf, args.kernel) | flags_of(sf, args.config)
    cw = sf.ct_words(params)
    keys = sf.keygen(params, 3000)
    pub = torch.from_numpy(keys.public().view(np.int32)).cuda()
    kb = keys.key_bits()
    d_bk = torch.empty((len(kb), cw), dtype=torch.int32, device="cuda")
    sf.encrypt_raw_bits_device(params, pub, kb, 11, d_bk)
    rng = np.random.default_rng(12)
    src_bits = rng.integers(0, 2, size=count).astype(np.uint8)
    d_src = torch.empty((count, cw), dtype=torch.int32, device="cuda")
    sf.encrypt_raw_bits_device(params, pub, src_bits, 13, d_src)
    plan = sf.Plan.refresher(params, count, flags)
    info = plan.info
    if info["gate_kernel"] == sf.KERNEL_INT:
        int_peaks(sf)
    d_out = torch.empty((count, cw), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    run = lambda: plan.refresh(d_bk, d_src, d_out, scratch, stream)  # noqa: E731
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            run()
        plan.check(stream)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        n0 = sf.lib().sfft_launch_count()
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                run()
            ev1.record(stream)
            torch.cuda.synchronize()
        launches_timed = sf.lib().sfft_launch_count() - n0
        ms = ev0.elapsed_time(ev1) / args.steps
        plan.check(stream)
        plan.set_timing(True)
        run()
        gate_ms, expand_ms, launches, gates_timed = plan.timing()
        plan.set_timing(False)
        # end to end: sources from pinned host memory, refreshed ciphertexts back
        h_src = d_src.cpu().pin_memory()
        h_out = torch.empty((count, cw), dtype=torch.int32).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            d_src.copy_(h_src, non_blocking=True)
            run()
            h_out.copy_(d_out, non_blocking=True)
            stream.synchronize()
        e2e_ms = (time.perf_counter() - t0) * 1000.0 / args.steps
    # the refreshed bits decrypt to the sources
    rows = d_out.view(count, -1)[:, (params.ell - 1) * (params.n + 1) * params.ell // 32:
                                 params.ell * (params.n + 1) * params.ell // 32]
    raw = sf.decrypt(keys, rows.cpu().numpy().view(np.uint32), (params.n + 1) * params.ell // 32,
                     count // 4, 2, 0)[2]   # 2-bit words: ciphertext i is bit i % 2 of word i // 2
    ok = [(int(raw[i // 2]) >> (i % 2)) & 1 for i in range(count // 4 * 4)] == \
        [int(b) for b in src_bits[:count // 4 * 4]]
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        oparams = oracle_params(args.config)   # the oracle's own ell (equal to the library's)
        v, gps, detail = cpu_refresh_sample(oparams, count, args.cpu_seconds,
                                            variant_of(args.config)["xcarry"])
        cpu = {"value": v, "unit": "ct/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": detail, "gates_per_s": gps, "oracle_ell": oparams.ell,
               "oracle_ell_equals_library": oparams.ell == params.ell}
    if rank != 0:
        return
    cfg = refresh_config_json(args.config, params, count)
    cfg.update({"products_per_step": info["products"], "levels": info["levels"],
                "l2": f"bootstrapping key {len(kb) * cw * 4 / 1e9:.2f} GB (> L2 129 MB)",
                "sources": "fresh encryptions of seeded random bits",
                "decrypts_to_sources": ok})
    line = {
        "metric": "refreshed ciphertexts/s", "value": count * 1000.0 / ms, "unit": "ct/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": cfg,
        "gates_per_s": info["products"] * 1000.0 / ms,
        "roofline": roofline(params, info["gate_kernel"], gate_ms, launches, gates_timed,
                             info["tc_columns"], expand_ms),
        "cpu_baseline": cpu,
        "e2e": {"value": count * 1000.0 / e2e_ms, "unit": "ct/s",
                "h2d_bytes_per_step": count * cw * 4, "d2h_bytes_per_step": count * cw * 4},
        "gpu_launches": launches_timed,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_gates(args):
    """One level of `--gates` random products at the workload's parameters."""
    import torch

    import paper_1611_08769_gb300 as sf
    from paper_1611_08769_gb300 import build as sfbuild
    sfbuild.build()
    params, _ = workload(sf, args.config)
    cw = sf.ct_words(params)
    G = args.gates
    gen = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randint(-2**31, 2**31 - 1, (G, cw), dtype=torch.int32, device="cuda", generator=gen)
    B = torch.randint(-2**31, 2**31 - 1, (G, cw), dtype=torch.int32, device="cuda", generator=gen)
    O0, O1 = torch.empty_like(A), torch.empty_like(A)
    code0 = [sf.pack_code(0, 1, 1, -2)] * G
    code1 = [sf.pack_code(0, 0, 0, 1)] * G
    flags = [2 if g % 3 else 3 for g in range(G)]   # every third A operand complemented
    kern = {"auto": 0, "int": 1, "tc": 2, "sm": 3}[args.kernel]
    for _ in range(args.warmup):
        sf.gate_level(params, A, B, O0, O1, code0, code1, flags, kernel=kern)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(args.steps):
        ev0.record()
        sf.gate_level(params, A, B, O0, O1, code0, code1, flags, kernel=kern)
        ev1.record()
        torch.cuda.synchronize()
        ms.append(ev0.elapsed_time(ev1))
    t = statistics.median(ms)
    info = sf.circuit_info(params, 2, 1, 4, 1)
    gk = kern if kern else info["gate_kernel"]
    if gk == 1:
        int_peaks(sf)
    print(json.dumps({"mode": "gates", "gates": G, "ms_per_level": t, "gates_per_s": G / t * 1e3,
                      "config": {"workload": args.config, "n": params.n, "ell": params.ell},
                      "note": "includes the test hook's descriptor upload, allocation and sync",
                      "roofline": roofline(params, gk, t, 1, G, info["tc_columns"])}), flush=True)


def run_serve(args, config=None, requests=0, emit=True):
    """Poisson arrivals into the continuous-batching server (rank 0 only);
    returns the JSON line (printed when emit)."""
    import torch

    import paper_1611_08769_gb300 as sf
    from paper_1611_08769_gb300 import build as sfbuild
    from synthetic import serving_trace
    sfbuild.build()
    config = config or args.config
    c = CONFIGS[config]
    params = product_params(sf, config)
    cw = sf.ct_words(params)
    count = requests or args.requests or c["requests"]
    # one encrypted input per distinct (shape, key set); outputs rotate per shape
    probe = serving_trace(count + c["calib"], 1.0, seed=5, key_sets=c["key_sets"])
    keys = {ks: sf.keygen(params, 2000 + ks) for ks in range(c["key_sets"])}
    pubs = {ks: torch.from_numpy(k.public().view(np.int32)).cuda() for ks, k in keys.items()}
    inputs, outputs = {}, {}
    # shapes and key sets of a trace do not depend on its rate
    for r in probe + serving_trace(count, 1.0, seed=6, key_sets=c["key_sets"]):
        shape = (r.N1, r.N2, r.F, r.f)
        if (shape, r.key_set) not in inputs:
            n = r.N1 * r.N2 * 2 * r.F
            d = torch.empty((n, cw), dtype=torch.int32, device="cuda")
            sf.encrypt_bits_device(params, pubs[r.key_set], r.re, r.im, r.F, r.f, r.seed, d)
            inputs[(shape, r.key_set)] = d.cpu().pin_memory()
            del d
        if shape not in outputs:
            outputs[shape] = [torch.empty((r.N1 * r.N2 * 2 * r.F, cw), dtype=torch.int32).pin_memory()
                              for _ in range(4)]
    products = {s: sf.circuit_info(params, *s)["products"] for s in outputs}
    srv = sf.Server(params, int(args.budget_gb * (1 << 30)), max_active=64)
    rot = {}

    def submit(r):
        shape = (r.N1, r.N2, r.F, r.f)
        k = rot.get(shape, 0)
        rot[shape] = k + 1
        return srv.submit(shape, inputs[(shape, r.key_set)], outputs[shape][k % 4])

    # every shape's circuit compiled before the clock starts (a server's
    # warm-up, like loading a model), then the capacity: a closed burst of
    # the same mix, on the same server as the timed trace
    t0 = time.perf_counter()
    for shape in outputs:
        srv.prepare(shape)
    prepare_s = time.perf_counter() - t0
    burst = probe[:c["calib"]]
    t0 = time.perf_counter()
    tickets = [submit(r) for r in burst]
    for t in tickets:
        srv.wait(t)
    cap = len(burst) / (time.perf_counter() - t0)
    rate = 0.8 * cap
    trace = serving_trace(count, rate, seed=6, key_sets=c["key_sets"])
    st0 = srv.stats()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        t0 = time.perf_counter()
        tickets = []
        for r in trace:
            now = time.perf_counter() - t0
            if r.arrival_s > now:
                time.sleep(r.arrival_s - now)
            tickets.append(submit(r))
        lat = [srv.wait(t) for t in tickets]
        wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    served_prod = sum(products[(r.N1, r.N2, r.F, r.f)] for r in trace)
    by_shape = {}
    for r, x in zip(trace, lat):
        by_shape.setdefault("%dx%d F%d" % (r.N1, r.N2, r.F), []).append(x)
    per_shape = {k: {"requests": len(v), "p50_ms": float(np.percentile(v, 50)),
                     "p99_ms": float(np.percentile(v, 99))} for k, v in sorted(by_shape.items())}
    line = {
        "metric": "encrypted FFTs/s served", "value": len(trace) / wall, "unit": "FFT/s",
        "n_gpus": 1, "steps": len(trace), "warmup": len(burst), "ms_per_step": wall * 1000 / len(trace),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": config, "n": params.n, "ell": params.ell, "chi": params.chi,
                   "requests": len(trace), "key_sets": c["key_sets"],
                   "arrival_rate_per_s": rate, "capacity_closed_burst_per_s": cap,
                   "hbm_budget_gb": args.budget_gb, "max_active": 64,
                   "mix": "75% 1-D N in {8..256} 8.8, 25% 2-D 8x8/16x16/32x32 at log2(pixels)+2 "
                          "integer bits, F = 16"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(max(lat)), "by_shape": per_shape,
                       "note": "submit to completion, per request of the timed trace"},
        "gates_per_s": served_prod / wall,
        "server": {"ticks": st["ticks"] - st0["ticks"], "tick_gates": st["tick_gates"] - st0["tick_gates"],
                   "peak_active": st["peak_active"], "prepare_s": prepare_s,
                   "admission": "arrival order; a request that does not fit may be passed by up to "
                                "16 later ones that do"},
        "e2e": {"value": len(trace) / wall, "unit": "FFT/s",
                "note": "served end to end: host ciphertexts in, host ciphertexts out"},
        "clocks": clk.summary(),
    }
    if emit:
        print(json.dumps(line), flush=True)
    return line


def run_fft(args, config, steps, warmup, world, rank, local, cpu_leg=True, plain_leg=True):
    """One FFT or batch workload on this rank's GPU: the batched form (graph
    replay) timed, per-launch kernel events, the plain evaluator, the host
    pipeline and (rank 0, one GPU) the CPU oracle baseline. Returns the JSON
    line on rank 0, None elsewhere."""
    import torch
    import torch.distributed as dist

    import paper_1611_08769_gb300 as sf
    from paper_1611_08769_gb300 import build as sfbuild

    sfbuild.build()
    params, items = workload(sf, config)
    flags = kernel_flags(sf, args.kernel) | flags_of(sf, config)
    enc_tw = variant_of(config)["enc_twiddle"]
    cw = sf.ct_words(params)
    reqs = [d for d, *_ in items]

    # client side: one key pair per key set, inputs encrypted on the device
    keys = {ks: sf.keygen(params, 1000 + ks) for ks in sorted({it[3] for it in items})}
    pubs = {ks: torch.from_numpy(k.public().view(np.int32)).cuda() for ks, k in keys.items()}
    batch = sf.Batch(params, reqs, flags)
    info = batch.info
    if info["gate_kernel"] == sf.KERNEL_INT:
        int_peaks(sf)
    tuned = None
    if info["gate_kernel"] == sf.KERNEL_SM:   # ring depth of the small-ciphertext kernel
        depth, us = sf.autotune_small(params, 20000, 3)
        tuned = {"ring_depth": depth, "ns_per_gate_by_depth": {k: round(v * 1000, 2) for k, v in us.items()},
                 "level": "20000 random half-adder products"}
    d_in = torch.empty((info["inputs"], cw), dtype=torch.int32, device="cuda")
    for r, ((N1, N2, F, f), re_, im_, ks, seed) in enumerate(items):
        re_all, im_all = fft_inputs(product_twiddles(sf), (N1, N2, F, f), re_, im_, enc_tw)
        n = len(re_all) * 2 * F
        sf.encrypt_bits_device(params, pubs[ks], re_all, im_all, F, f, seed,
                               d_in[batch.in_off[r]:batch.in_off[r] + n])
    d_out = torch.empty((info["outputs"], cw), dtype=torch.int32, device="cuda")
    scratch = torch.empty(max(1, info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, steps):
        barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return ev0.elapsed_time(ev1) / steps

    # batched form (graph replay): the headline
    run_b = lambda: batch.eval(d_in, d_out, scratch, stream)  # noqa: E731
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            run_b()
        batch.check(stream)
        with ClockSampler(local) as clk:
            ms = timed(run_b, steps)
        batch.check(stream)
    ms = max_over_ranks(ms, world, "cuda")
    fft_per_s = replica_throughput(len(items), ms, world)

    # kernel timing (per-launch events; graph replay is bypassed while timing)
    batch.set_timing(True)
    n0 = sf.lib().sfft_launch_count()
    with torch.cuda.stream(stream):
        run_b()
    kernels_per_step = sf.lib().sfft_launch_count() - n0
    gate_ms, expand_ms, launches, gates_timed = batch.timing()
    batch.set_timing(False)

    # the persistent form (one launch across levels) on the same inputs, where
    # the small-ciphertext kernel runs a circuit without linear gates
    persistent = None
    if info["gate_kernel"] == sf.KERNEL_SM and not variant_of(config)["xcarry"]:
        pbatch = sf.Batch(params, reqs, flags | sf.BATCH_PERSISTENT)
        pscr = torch.empty(max(1, pbatch.info["scratch_bytes"] // 4), dtype=torch.int32, device="cuda")
        p_out = torch.empty_like(d_out)
        run_pb = lambda: pbatch.eval(d_in, p_out, pscr, stream)  # noqa: E731
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                run_pb()
            pbatch.check(stream)
            pms = timed(run_pb, steps)
            pbatch.check(stream)
            run_b()
        torch.cuda.synchronize()
        persistent = {"ms_per_step": pms, "value": len(items) * 1000.0 / pms, "unit": "FFT/s",
                      "launches_per_step": 3, "scratch_bytes": pbatch.info["scratch_bytes"],
                      "speedup_vs_level_launches": ms / pms,
                      "outputs_equal_level_by_level": bool(torch.equal(p_out, d_out))}
        del pbatch, pscr, p_out

    # plain level-by-level evaluator on the same workload (per-request plans)
    plain = None
    if plain_leg:
        plans = [sf.Plan(params, *d, flags) for d in reqs]
        pscr = torch.empty(max(1, max(p.info["scratch_bytes"] for p in plans) // 4),
                           dtype=torch.int32, device="cuda")

        def run_p():
            for r, p in enumerate(plans):
                p.eval_fft(d_in[batch.in_off[r]:], d_out[batch.out_off[r]:], pscr, stream)
        with torch.cuda.stream(stream):
            for _ in range(min(1, warmup)):
                run_p()
            pms = timed(run_p, max(1, steps))
        plain = {"ms_per_step": pms, "value": len(items) * 1000.0 / pms, "unit": "FFT/s",
                 "launches_per_step": sum(p.info["levels"] + 1 for p in plans),
                 "speedup_of_batched": pms / ms}
        del plans

    # end to end through the C ABI with host buffers: every step copies its
    # inputs from pinned host memory and its outputs back, double-buffered so
    # that step i's copies overlap steps i - 1 and i + 1
    h_in = d_in.cpu().pin_memory()
    h_outs = [torch.empty(d_out.shape, dtype=d_out.dtype).pin_memory() for _ in range(2)]
    d_in2 = torch.empty_like(d_in)
    d_out2 = torch.empty_like(d_out)
    pipe = lambda n: batch.eval_host_pipelined(  # noqa: E731
        [h_in] * n, [h_outs[i % 2] for i in range(n)], [d_in, d_in2], [d_out, d_out2], scratch,
        stream)
    with torch.cuda.stream(stream):
        pipe(2)   # warm-up: both buffer sets' graphs
        barrier()
        t0 = time.perf_counter()
        pipe(steps)
        e2e_ms = (time.perf_counter() - t0) * 1000.0 / steps
        barrier()
    e2e_ms = max_over_ranks(e2e_ms, world, "cuda")

    cpu = None
    if rank == 0 and world == 1 and cpu_leg:
        oparams = oracle_params(config, items)   # the oracle's own ell
        fps, gps, detail = cpu_oracle_sample(oparams, items, args.cpu_seconds, variant_of(config))
        cpu = {"value": fps, "unit": "FFT/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": detail, "gates_per_s": gps, "oracle_ell": oparams.ell,
               "oracle_ell_equals_library": oparams.ell == params.ell}

    if rank == 0:
        cfg = config_json(config, params, items)
        if tuned:
            cfg["autotune"] = tuned
        cfg.update({"products_per_step": info["products"], "levels": info["levels"],
                    "evaluator": "level-merged program replayed as one CUDA graph",
                    "l2": f"inputs {info['inputs'] * cw * 4 / 1e9:.2f} GB (> L2 129 MB)"
                          if info["inputs"] * cw * 4 > 129e6 else
                          f"inputs {info['inputs'] * cw * 4 / 1e6:.1f} MB (< L2; scratch "
                          f"{info['scratch_bytes'] / 1e9:.2f} GB of intermediates streamed)"})
        line = {
            "metric": "encrypted FFTs/s", "value": fft_per_s, "unit": "FFT/s", "n_gpus": world,
            "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": cfg,
            "gates_per_s": world * info["products"] * 1000.0 / ms,
            "roofline": roofline(params, info["gate_kernel"], gate_ms, launches, gates_timed,
                                 info["tc_columns"], expand_ms),
            "plain": plain,
            "persistent": persistent,
            "cpu_baseline": cpu,
            "e2e": {"value": world * len(items) * 1000.0 / e2e_ms, "unit": "FFT/s",
                    "h2d_bytes_per_step": info["inputs"] * cw * 4,
                    "d2h_bytes_per_step": info["outputs"] * cw * 4,
                    "api": "sfft_batch_eval_host_pipelined (copies overlapped with the "
                           "neighbouring steps)"},
            "gpu_launches": steps * kernels_per_step,
            "clocks": clk.summary(),
        }
        return line
    return None


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "gates":
        return run_gates(args)
    if CONFIGS[args.config]["kind"] == "serve":
        return run_serve(args) if rank == 0 else None
    if CONFIGS[args.config]["kind"] == "refresh":
        return run_refresh(args)

    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    line = run_fft(args, args.config, args.steps, args.warmup, world, rank, local,
                   cpu_leg=not args.no_cpu_baseline, plain_leg=not args.no_plain)
    if rank == 0 and world == 1 and args.config == DEFAULT_CONFIG and not args.no_extra:
        # the baseline metric's other forms on the same box: batched vs plain
        # on the 256-request batch, one narrow program, and the
        # continuous-batching server
        torch.cuda.empty_cache()
        b = run_fft(args, "batch256_p2", 3, 2, 1, 0, local, cpu_leg=False, plain_leg=True)
        line["batch"] = {k: b[k] for k in ("metric", "value", "unit", "ms_per_step", "gates_per_s",
                                           "config", "roofline", "plain", "persistent", "e2e",
                                           "gpu_launches", "clocks")}
        torch.cuda.empty_cache()
        # a narrow program: one 64-point FFT at ell 128, level by level and as
        # one persistent launch (where the one-launch form pays)
        nb = run_fft(args, "fft64_16bit_p2", 10, 3, 1, 0, local, cpu_leg=False, plain_leg=False)
        line["narrow"] = {k: nb[k] for k in ("metric", "value", "unit", "ms_per_step", "gates_per_s",
                                             "config", "persistent", "gpu_launches", "clocks")}
        torch.cuda.empty_cache()
        srv = run_serve(args, "serve_p2", requests=args.serve_requests, emit=False)
        line["serve"] = {k: srv[k] for k in ("metric", "value", "unit", "config", "latency_ms",
                                             "gates_per_s", "server", "clocks")}
        import paper_1611_08769_gb300 as sf
        with ClockSampler(local) as clk:
            pk = int_peaks(sf)
        line["int_peaks"] = {"unit": "Tops/s", **{k: v / 1e12 for k, v in pk.items()},
                             "how": "8 independent chains per thread of one 32-bit op, all SMs at "
                                    "full occupancy, CUDA events (popc: popc + xor per step)",
                             "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
