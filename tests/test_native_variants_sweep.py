"""Sweep of small FFT circuits over every combination of the circuit variants
(paper gates / exclusive carry / NAND-only, plaintext / encrypted twiddles) and
shapes (1-D, square and non-square 2-D): the native compiler's device program,
run in plaintext with its slots, fix-ups and adjusted coefficients, equals the
oracle's independent circuit on random input bits; product counts, depth and
the static noise bound agree. CPU only."""
import itertools
import random

import numpy as np
import pytest

from oracle import circuit, evaluate, noise

SHAPES = [(2, 1, 4, 1), (4, 1, 6, 2), (2, 2, 4, 1), (4, 2, 6, 2), (2, 4, 6, 3)]
VARIANTS = [{}, {"xcarry": True}, {"nand": True}]


@pytest.mark.parametrize("shape,variant,enc", [
    (s, v, e) for s, v, e in itertools.product(SHAPES, VARIANTS, (False, True))])
def test_native_program_equals_oracle(shape, variant, enc):
    import paper_1611_08769_gb300 as sf
    N1, N2, F, f = shape
    if enc and f > F - 2:
        pytest.skip("encrypted twiddles need f <= F - 2")
    sp = sf.param_set("P0")
    c = circuit.fft_circuit(N1, N2, F, f, enc_twiddle=enc, **variant)
    st = circuit.stats(c)
    info = sf.circuit_info(sp, N1, N2, F, f, enc_twiddle=enc, **variant)
    assert info["inputs"] == len(c.inputs) and info["outputs"] == len(c.outputs)
    assert info["products"] == st["products"]
    # levels = multiplicative depth; with exclusive carries a linear gate that
    # reads another linear gate's output (through constant folding) runs one
    # level later, so there can be more levels than the depth
    if variant.get("xcarry"):
        assert info["levels"] >= st["depth"]
    else:
        assert info["levels"] == st["depth"]
    ell = sf.min_ell(N1, N2, F, f, 1, 1, enc_twiddle=enc, **variant)
    assert ell == noise.smallest_ell(c, 1, 1)
    rng = random.Random(hash((shape, tuple(variant), enc)) & 0xFFFF)
    for _ in range(4):
        bits = [rng.randint(0, 1) for _ in range(len(c.inputs))]
        got = sf.program_eval_plain(sp, N1, N2, F, f, np.array(bits, np.uint8), enc_twiddle=enc,
                                    **variant)
        assert list(got) == evaluate.eval_plain(c, bits)
