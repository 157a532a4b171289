"""ctypes declarations of the C ABI in include/sfft.h (argument marshalling only).

Loading fails loudly when the in-tree library is missing: there is no
Python or CPU fallback for any call.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsfft.so")

c_u32, c_u64, c_i32, c_i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
c_void_p, c_double_p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
c_u32_p, c_u16_p, c_u8_p, c_i64_p = (ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint16),
                                     ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(ctypes.c_int64))


class sfft_params(ctypes.Structure):
    _fields_ = [("n", c_u32), ("ell", c_u32), ("m", c_u32), ("chi", c_u32)]


class sfft_plan_info(ctypes.Structure):
    _fields_ = [("inputs", c_u64), ("outputs", c_u64), ("gates_and", c_u64), ("gates_xor", c_u64),
                ("gates_or", c_u64), ("gates_not", c_u64), ("products", c_u64), ("levels", c_u64),
                ("max_level_width", c_u64), ("scratch_slots", c_u64), ("scratch_bytes", c_u64),
                ("ct_words", c_u64), ("noise_bits", c_u32), ("noise_ok", c_u32),
                ("gate_kernel", c_u32), ("tc_columns", c_u32), ("gates_xadd", c_u64)]


P = ctypes.POINTER
# name: (restype, argtypes)
SIGNATURES = {
    "sfft_last_error": (ctypes.c_char_p, []),
    "sfft_version": (ctypes.c_char_p, []),
    "sfft_launch_count": (c_u64, []),
    "sfft_ct_words": (c_u64, [P(sfft_params)]),
    "sfft_keygen": (c_i32, [P(sfft_params), c_u64, P(c_void_p)]),
    "sfft_keys_free": (None, [c_void_p]),
    "sfft_keys_public": (c_i32, [c_void_p, c_u32_p, c_u64]),
    "sfft_encrypt_bits": (c_i32, [c_void_p, c_double_p, c_double_p, c_u64, c_u32, c_u32, c_u64,
                                  c_u32_p]),
    "sfft_encrypt_bits_device": (c_i32, [P(sfft_params), c_void_p, c_double_p, c_double_p, c_u64,
                                         c_u32, c_u32, c_u64, c_void_p, c_void_p]),
    "sfft_decrypt": (c_i32, [c_void_p, c_u32_p, c_u64, c_u64, c_u32, c_u32, c_double_p,
                             c_double_p, c_i64_p]),
    "sfft_gather_dec_rows": (c_i32, [P(sfft_params), c_void_p, c_u64, c_void_p, c_void_p]),
    "sfft_min_ell": (c_u32, [c_u32, c_u32, c_u32, c_u32, c_u32, c_u32, c_u32]),
    "sfft_plan_create": (c_i32, [P(sfft_params), c_u32, c_u32, c_u32, c_u32, c_u32, P(c_void_p)]),
    "sfft_plan_info_get": (c_i32, [c_void_p, P(sfft_plan_info)]),
    "sfft_plan_free": (None, [c_void_p]),
    "sfft_eval_fft": (c_i32, [c_void_p, c_void_p, c_void_p, c_void_p, c_u64, c_void_p]),
    "sfft_eval_fft_host": (c_i32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                   c_u64, c_void_p]),
    "sfft_eval_fft_noalloc": (c_i32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "sfft_noalloc_scratch_bytes": (c_u64, []),
    "sfft_plan_set_timing": (c_i32, [c_void_p, ctypes.c_int]),
    "sfft_plan_timing": (c_i32, [c_void_p, c_double_p, c_double_p, P(c_u64), P(c_u64)]),
    "sfft_circuit_info": (c_i32, [P(sfft_params), c_u32, c_u32, c_u32, c_u32, c_u32,
                                  P(sfft_plan_info)]),
    "sfft_program_eval_plain": (c_i32, [P(sfft_params), c_u32, c_u32, c_u32, c_u32, c_u32, c_u8_p,
                                        c_u8_p]),
    "sfft_program_gates": (c_i32, [P(sfft_params), c_u32, c_u32, c_u32, c_u32, c_u32, c_void_p, c_u64,
                                   P(c_u64)]),
    "sfft_word_plan_create": (c_i32, [P(sfft_params), c_u32, c_u64, c_u32, c_u32, c_u32,
                                      P(c_void_p)]),
    "sfft_word_min_ell": (c_u32, [c_u32, c_u32, c_u32, c_u32, c_u32, c_u32]),
    "sfft_word_circuit_info": (c_i32, [P(sfft_params), c_u32, c_u64, c_u32, c_u32, c_u32,
                                       P(sfft_plan_info)]),
    "sfft_word_program_eval_plain": (c_i32, [P(sfft_params), c_u32, c_u64, c_u32, c_u32, c_u32,
                                             c_u8_p, c_u8_p]),
    "sfft_twiddles": (c_i32, [c_u32, c_u32, c_i64_p, c_i64_p]),
    "sfft_encrypt_raw_bits_device": (c_i32, [P(sfft_params), c_void_p, c_u8_p, c_u64, c_u64,
                                             c_void_p, c_void_p]),
    "sfft_key_bits": (c_i32, [c_void_p, c_u8_p, c_u64]),
    "sfft_refresh_plan_create": (c_i32, [P(sfft_params), c_u64, c_u32, P(c_void_p)]),
    "sfft_refresh_min_ell": (c_u32, [c_u32, c_u32, c_u32]),
    "sfft_refresh": (c_i32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_u64, c_void_p]),
    "sfft_refresh_circuit_info": (c_i32, [P(sfft_params), c_u64, c_u32, P(sfft_plan_info)]),
    "sfft_refresh_eval_plain": (c_i32, [P(sfft_params), c_u64, c_u32, c_u8_p, c_u32_p, c_u8_p]),
    "sfft_eval_levels": (c_i32, [c_void_p, c_u32, c_u32, c_void_p, c_void_p, c_void_p, c_u64, c_void_p]),
    "sfft_plan_level": (c_i32, [c_void_p, c_u32, c_u32_p, c_u32_p, c_u8_p, c_u64, P(c_u64), P(c_u64)]),
    "sfft_measure_int_peak": (c_i32, [c_u32, c_u32, c_double_p]),
    "sfft_autotune_small": (c_i32, [P(sfft_params), c_u64, c_u32, c_u32_p, c_double_p]),
    "sfft_small_kernel_set_slots": (c_i32, [c_u32, c_u32]),
    "sfft_gate_level_withheld": (c_i32, [P(sfft_params), c_void_p, c_void_p, c_void_p, c_u16_p,
                                         c_u8_p, c_u64, c_u32, c_void_p]),
    "sfft_gate_level": (c_i32, [P(sfft_params), c_void_p, c_void_p, c_void_p, c_void_p, c_u16_p,
                                c_u16_p, c_u8_p, c_u64, c_u32, c_void_p]),
    "sfft_plan_check": (c_i32, [c_void_p, c_void_p]),
    "sfft_batch_create": (c_i32, [P(sfft_params), c_void_p, c_u32, c_u32, P(c_void_p)]),
    "sfft_batch_info_get": (c_i32, [c_void_p, P(sfft_plan_info)]),
    "sfft_batch_offsets": (c_i32, [c_void_p, P(c_u64), P(c_u64)]),
    "sfft_batch_eval": (c_i32, [c_void_p, c_void_p, c_void_p, c_void_p, c_u64, c_void_p]),
    "sfft_batch_check": (c_i32, [c_void_p, c_void_p]),
    "sfft_batch_set_epoch": (c_i32, [c_void_p, c_u32, c_void_p]),
    "sfft_batch_eval_host_pipelined": (c_i32, [c_void_p, P(c_void_p), P(c_void_p), c_u32,
                                               P(c_void_p), P(c_void_p), c_void_p, c_u64,
                                               c_void_p]),
    "sfft_batch_eval_host": (c_i32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                    c_u64, c_void_p]),
    "sfft_batch_set_timing": (c_i32, [c_void_p, ctypes.c_int]),
    "sfft_batch_timing": (c_i32, [c_void_p, c_double_p, c_double_p, P(c_u64), P(c_u64)]),
    "sfft_batch_free": (None, [c_void_p]),
}


class sfft_request(ctypes.Structure):
    _fields_ = [("N1", c_u32), ("N2", c_u32), ("F", c_u32), ("f", c_u32)]


class sfft_server_stats(ctypes.Structure):
    _fields_ = [("completed", c_u64), ("queued", c_u64), ("active", c_u64), ("ticks", c_u64),
                ("tick_gates", c_u64), ("peak_active", c_u64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double)]


SIGNATURES.update({
    "sfft_server_create": (c_i32, [P(sfft_params), c_u64, c_u32, c_u32, P(c_void_p)]),
    "sfft_server_submit": (c_i32, [c_void_p, P(sfft_request), c_void_p, c_void_p, P(c_u64)]),
    "sfft_server_prepare": (c_i32, [c_void_p, P(sfft_request)]),
    "sfft_server_wait": (c_i32, [c_void_p, c_u64, c_u32, c_double_p]),
    "sfft_server_get_stats": (c_i32, [c_void_p, P(sfft_server_stats)]),
    "sfft_server_free": (None, [c_void_p]),
})

_lib = None


def lib():
    """The loaded library with every declared signature bound."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"native library missing: {LIB_PATH} "
                              "(build it with paper_1611_08769_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class SfftError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sfft error {code}: {msg}")
        self.code = code


def check(rc):
    if rc != 0:
        raise SfftError(rc, lib().sfft_last_error().decode())
    return rc
