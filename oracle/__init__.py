"""CPU oracle for the encrypted FFT (test infrastructure only).

This package is the plain, slow, obviously-correct CPU statement of what the
GPU library computes: the GSW'13 scheme the paper uses (Sec. 3), the gate
circuit built from it (Sec. 4: gates, half/full adders, ripple adders and
subtractors, Wallace constant multiplier, fixed-point butterflies, radix-2
FFT) and the plaintext fixed-point FFT it must agree with (Sec. 4, Sec. 5).

It is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path, and the CUDA path never calls it.

Modules
-------
prng        counter-based SplitMix64 streams (randomness layout; paper silent)
gsw         GSW'13 KeyGen/Enc/Dec/gates, compressed form and literal N x N form
circuit     canonical gate netlist: HA, FA, ADD, SUB, Wallace MUL, butterfly, FFT
fixedpoint  quantisation, twiddles, closed-form integer FFT, FP64 DFT, Thm 2 bound
noise       static worst-case noise bound and the measured noise of a ciphertext
evaluate    plaintext and encrypted evaluation of a circuit
refresh     ciphertext refresh by homomorphic decryption (bootstrapping key,
            truncated phase sum, refresh circuit, closed form)

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (see tests/test_oracle_*.py); none is
"parity unpinned".
"""
