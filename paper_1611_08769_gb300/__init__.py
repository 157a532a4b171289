"""GB300-native encrypted FFT (GSW'13 gate circuits on sm_103a).

Thin Python binding over the C ABI in ``include/sfft.h``; every step of the
computation runs in the native library's CUDA kernels. PyTorch supplies
device memory and streams only.

Client calls (host): ``keygen``, ``encrypt_bits``, ``decrypt``.
Server calls (device): ``Plan`` (``sfft_plan_create``) with ``eval_fft`` /
``eval_fft_host``, ``encrypt_bits_device``, ``gather_dec_rows``,
``gate_level`` (single-level test hook).
"""
import ctypes

import numpy as np

from . import native
from .native import SfftError, check, lib, sfft_params, sfft_plan_info

PLAN_ALLOW_NOISY = 1
PLAN_INT_KERNEL = 2
PLAN_XCARRY = 8   # circuit variant: exclusive-carry full adders (sfft.h SFFT_PLAN_XCARRY)
PLAN_NAND = 16    # circuit variant: every gate built of NAND gates (sfft.h SFFT_PLAN_NAND)
PLAN_ENC_TWIDDLE = 32   # FFT twiddles as encrypted inputs (sfft.h SFFT_PLAN_ENC_TWIDDLE)
PLAN_TC_KERNEL = 64     # the general tensor-core kernel where the small one applies
WORD_ADD, WORD_SUB, WORD_MUL = 1, 2, 3   # word circuits (sfft.h SFFT_WORD_*)
KERNEL_AUTO, KERNEL_INT, KERNEL_TC, KERNEL_SM = 0, 1, 2, 3

__all__ = ["Params", "Keys", "Plan", "keygen", "encrypt_bits", "encrypt_bits_device", "decrypt",
           "gather_dec_rows", "min_ell", "gate_level", "ct_words", "SfftError", "version",
           "word_min_ell", "word_circuit_info", "twiddles", "refresh_min_ell",
           "refresh_circuit_info", "refresh_eval_plain", "encrypt_raw_bits_device"]

PARAM_SETS = {
    # toy, noise-free (chi = 0): exact decryption at any depth; insecure by construction
    "P0": (1, 32, 64, 0),
    # noise-free multi-limb throughput set
    "P2": (1, 128, 256, 0),
}


def Params(n, ell, m=None, chi=0):
    """GSW parameters; m defaults to Ng = (n+1) ell."""
    return sfft_params(n, ell, (n + 1) * ell if m is None else m, chi)


def param_set(name, ell=None):
    """'P0', 'P2', or 'P1' (chi = 1, m = Ng, ell given -- see min_ell)."""
    if name == "P1":
        return Params(1, ell, None, 1)
    n, e, m, chi = PARAM_SETS[name]
    return Params(n, e, m, chi)


def version():
    return lib().sfft_version().decode()


def ct_words(p):
    return int(lib().sfft_ct_words(ctypes.byref(p)))


def _dptr(t):
    return ctypes.c_void_p(0 if t is None else int(t.data_ptr()))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(0)
    return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Keys:
    """Secret/public key pair of one client (host-owned)."""

    def __init__(self, params, seed):
        self.params = params
        h = ctypes.c_void_p()
        check(lib().sfft_keygen(ctypes.byref(params), seed, ctypes.byref(h)))
        self._h = h

    def public(self):
        p = self.params
        out = np.zeros(p.m * (p.n + 1) * (p.ell // 32), dtype=np.uint32)
        check(lib().sfft_keys_public(self._h, out.ctypes.data_as(native.c_u32_p), out.size))
        return out

    def key_bits(self):
        """The n ell + 1 bits a bootstrapping key encrypts (sfft_key_bits)."""
        p = self.params
        out = np.zeros(p.n * p.ell + 1, dtype=np.uint8)
        check(lib().sfft_key_bits(self._h, out.ctypes.data_as(native.c_u8_p), out.size))
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().sfft_keys_free(h)
            self._h = None


def keygen(params, seed):
    return Keys(params, seed)


def encrypt_bits(keys, re, im, F, f, enc_seed):
    """Host encryption of a fixed-point signal -> uint32 array (2 F count, ct_words)."""
    re = _f64(re)
    im = None if im is None else _f64(im)
    cw = ct_words(keys.params)
    out = np.zeros((len(re) * 2 * F, cw), dtype=np.uint32)
    check(lib().sfft_encrypt_bits(keys._h, re.ctypes.data_as(native.c_double_p),
                                  None if im is None else im.ctypes.data_as(native.c_double_p),
                                  len(re), F, f, enc_seed, out.ctypes.data_as(native.c_u32_p)))
    return out


def encrypt_bits_device(params, d_pub, re, im, F, f, enc_seed, d_out, stream=None):
    """GPU encryption into the device tensor d_out (2 F count ciphertexts)."""
    re = _f64(re)
    im = None if im is None else _f64(im)
    check(lib().sfft_encrypt_bits_device(
        ctypes.byref(params), _dptr(d_pub), re.ctypes.data_as(native.c_double_p),
        None if im is None else im.ctypes.data_as(native.c_double_p), len(re), F, f, enc_seed,
        _dptr(d_out), _stream(stream)))


def encrypt_raw_bits_device(params, d_pub, bits, enc_seed, d_out, stream=None):
    """GPU encryption of arbitrary bits, ciphertext c = bits[c] (sfft_encrypt_raw_bits_device)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    check(lib().sfft_encrypt_raw_bits_device(ctypes.byref(params), _dptr(d_pub),
                                             bits.ctypes.data_as(native.c_u8_p), bits.size,
                                             enc_seed, _dptr(d_out), _stream(stream)))


def decrypt(keys, rows, row_stride_words, count, F, f):
    """Host decryption; returns (re, im, raw) numpy arrays."""
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    re = np.zeros(count)
    im = np.zeros(count)
    raw = np.zeros(2 * count, dtype=np.int64)
    check(lib().sfft_decrypt(keys._h, rows.ctypes.data_as(native.c_u32_p), row_stride_words,
                             count, F, f, re.ctypes.data_as(native.c_double_p),
                             im.ctypes.data_as(native.c_double_p), raw.ctypes.data_as(native.c_i64_p)))
    return re, im, raw


def gather_dec_rows(params, d_ct, n_ct, d_rows, stream=None):
    check(lib().sfft_gather_dec_rows(ctypes.byref(params), _dptr(d_ct), n_ct, _dptr(d_rows),
                                     _stream(stream)))


def _variant(xcarry, nand, enc_twiddle=False):
    return ((PLAN_XCARRY if xcarry else 0) | (PLAN_NAND if nand else 0)
            | (PLAN_ENC_TWIDDLE if enc_twiddle else 0))


def _info_dict(info):
    return {k: getattr(info, k) for k, _ in sfft_plan_info._fields_}


def min_ell(N1, N2, F, f, n=1, chi=1, xcarry=False, nand=False, enc_twiddle=False):
    return int(lib().sfft_min_ell(N1, N2, F, f, n, chi, _variant(xcarry, nand, enc_twiddle)))


def circuit_info(params, N1, N2, F, f, xcarry=False, nand=False, enc_twiddle=False):
    """Host-only statistics of the compiled FFT circuit (sfft_circuit_info)."""
    info = sfft_plan_info()
    check(lib().sfft_circuit_info(ctypes.byref(params), N1, N2, F, f,
                                  _variant(xcarry, nand, enc_twiddle), ctypes.byref(info)))
    return _info_dict(info)


def program_eval_plain(params, N1, N2, F, f, in_bits, xcarry=False, nand=False, enc_twiddle=False):
    """Host-only plaintext run of the compiled device program (sfft_program_eval_plain)."""
    flags = _variant(xcarry, nand, enc_twiddle)
    in_bits = np.ascontiguousarray(in_bits, dtype=np.uint8)
    out = np.zeros(circuit_info(params, N1, N2, F, f, xcarry, nand, enc_twiddle)["outputs"],
                   dtype=np.uint8)
    check(lib().sfft_program_eval_plain(ctypes.byref(params), N1, N2, F, f, flags,
                                        in_bits.ctypes.data_as(native.c_u8_p),
                                        out.ctypes.data_as(native.c_u8_p)))
    return out


# one sfft_gate_record (include/sfft.h)
GATE_RECORD = np.dtype([("a", "<u4"), ("b", "<u4"), ("o0", "<u4"), ("o1", "<u4"), ("code", "<u4"),
                        ("flags", "<u4"), ("level", "<u4"), ("dep_a", "<u4"), ("dep_b", "<u4")])


def program_gates(params, N1, N2, F, f, flags=0):
    """Host-only listing of the compiled FFT program, one GATE_RECORD per gate
    in program order (sfft_program_gates); flags as for sfft_program_gates."""
    n = ctypes.c_uint64(0)
    check(lib().sfft_program_gates(ctypes.byref(params), N1, N2, F, f, flags, None, 0, ctypes.byref(n)))
    out = np.zeros(n.value, dtype=GATE_RECORD)
    check(lib().sfft_program_gates(ctypes.byref(params), N1, N2, F, f, flags,
                                   ctypes.c_void_p(out.ctypes.data), n.value, ctypes.byref(n)))
    return out


def word_min_ell(op, F, f, n=1, chi=1, xcarry=False, nand=False):
    return int(lib().sfft_word_min_ell(op, F, f, n, chi, _variant(xcarry, nand)))


def word_circuit_info(params, op, count, F, f, xcarry=False, nand=False):
    """Host-only statistics of a word circuit (sfft_word_circuit_info)."""
    info = sfft_plan_info()
    check(lib().sfft_word_circuit_info(ctypes.byref(params), op, count, F, f,
                                       _variant(xcarry, nand), ctypes.byref(info)))
    return _info_dict(info)


def word_program_eval_plain(params, op, count, F, f, in_bits, xcarry=False, nand=False):
    """Host-only plaintext run of a word circuit's device program."""
    in_bits = np.ascontiguousarray(in_bits, dtype=np.uint8)
    out = np.zeros(count * F, dtype=np.uint8)
    check(lib().sfft_word_program_eval_plain(ctypes.byref(params), op, count, F, f,
                                             _variant(xcarry, nand),
                                             in_bits.ctypes.data_as(native.c_u8_p),
                                             out.ctypes.data_as(native.c_u8_p)))
    return out


def refresh_min_ell(n=1, chi=1, xcarry=False, nand=False):
    return int(lib().sfft_refresh_min_ell(n, chi, _variant(xcarry, nand)))


def refresh_circuit_info(params, count, xcarry=False, nand=False):
    """Host-only statistics of a refresh program (sfft_refresh_circuit_info)."""
    info = sfft_plan_info()
    check(lib().sfft_refresh_circuit_info(ctypes.byref(params), count, _variant(xcarry, nand),
                                          ctypes.byref(info)))
    return _info_dict(info)


def refresh_eval_plain(params, key_bits, rows, xcarry=False, nand=False):
    """Host-only plaintext run of a refresh program: rows = (count, (n+1) ell/32)
    uint32 rows ell - 1 of the refreshed ciphertexts; returns count bits."""
    rows = np.ascontiguousarray(rows, dtype=np.uint32)
    count = rows.shape[0]
    key_bits = np.ascontiguousarray(key_bits, dtype=np.uint8)
    out = np.zeros(count, dtype=np.uint8)
    check(lib().sfft_refresh_eval_plain(ctypes.byref(params), count, _variant(xcarry, nand),
                                        key_bits.ctypes.data_as(native.c_u8_p),
                                        rows.ctypes.data_as(native.c_u32_p),
                                        out.ctypes.data_as(native.c_u8_p)))
    return out


def twiddles(M, f):
    """Quantised twiddles W_M^k, k < M/2, as two int64 arrays (sfft_twiddles)."""
    wr = np.zeros(M // 2, dtype=np.int64)
    wi = np.zeros(M // 2, dtype=np.int64)
    check(lib().sfft_twiddles(M, f, wr.ctypes.data_as(native.c_i64_p),
                              wi.ctypes.data_as(native.c_i64_p)))
    return wr, wi


class Plan:
    """Compiled FFT circuit resident on the device (sfft_plan_create)."""

    def __init__(self, params, N1, N2, F, f, flags=0):
        self.params = params
        self.N1, self.N2, self.F, self.f = N1, N2, F, f
        h = ctypes.c_void_p()
        check(lib().sfft_plan_create(ctypes.byref(params), N1, N2, F, f, flags, ctypes.byref(h)))
        self._h = h
        info = sfft_plan_info()
        check(lib().sfft_plan_info_get(h, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in sfft_plan_info._fields_}

    @classmethod
    def words(cls, params, op, count, F, f, flags=0):
        """count word operations (sfft_word_plan_create); evaluated like an FFT plan."""
        self = cls.__new__(cls)
        self.params = params
        self.N1 = self.N2 = None
        self.F, self.f = F, f
        h = ctypes.c_void_p()
        check(lib().sfft_word_plan_create(ctypes.byref(params), op, count, F, f, flags,
                                          ctypes.byref(h)))
        self._h = h
        info = sfft_plan_info()
        check(lib().sfft_plan_info_get(h, ctypes.byref(info)))
        self.info = _info_dict(info)
        return self

    @classmethod
    def refresher(cls, params, count, flags=0):
        """Refresh of count ciphertexts (sfft_refresh_plan_create); run with refresh()."""
        self = cls.__new__(cls)
        self.params = params
        self.N1 = self.N2 = self.F = self.f = None
        h = ctypes.c_void_p()
        check(lib().sfft_refresh_plan_create(ctypes.byref(params), count, flags, ctypes.byref(h)))
        self._h = h
        info = sfft_plan_info()
        check(lib().sfft_plan_info_get(h, ctypes.byref(info)))
        self.info = _info_dict(info)
        return self

    def refresh(self, d_bk, d_src, d_out, d_scratch, stream=None):
        nbytes = 0 if d_scratch is None else d_scratch.numel() * d_scratch.element_size()
        check(lib().sfft_refresh(self._h, _dptr(d_bk), _dptr(d_src), _dptr(d_out),
                                 _dptr(d_scratch), nbytes, _stream(stream)))

    def eval_fft(self, d_in, d_out, d_scratch, stream=None):
        nbytes = 0 if d_scratch is None else d_scratch.numel() * d_scratch.element_size()
        check(lib().sfft_eval_fft(self._h, _dptr(d_in), _dptr(d_out), _dptr(d_scratch), nbytes,
                                  _stream(stream)))

    def eval_levels(self, l0, l1, d_in, d_out, d_scratch, stream=None):
        """Levels [l0, l1) of the program (sfft_eval_levels, a test hook)."""
        nbytes = 0 if d_scratch is None else d_scratch.numel() * d_scratch.element_size()
        check(lib().sfft_eval_levels(self._h, l0, l1, _dptr(d_in), _dptr(d_out), _dptr(d_scratch),
                                     nbytes, _stream(stream)))

    def level(self, level):
        """Gates of one level (sfft_plan_level): (desc (n, 4) uint32 references
        A, B, output 0, output 1; code (n,) uint32; flags (n,) uint8; products)."""
        n, npr = ctypes.c_uint64(0), ctypes.c_uint64(0)
        check(lib().sfft_plan_level(self._h, level, None, None, None, 0, ctypes.byref(n),
                                    ctypes.byref(npr)))
        desc = np.zeros((max(1, n.value), 4), dtype=np.uint32)
        code = np.zeros(max(1, n.value), dtype=np.uint32)
        flags = np.zeros(max(1, n.value), dtype=np.uint8)
        check(lib().sfft_plan_level(self._h, level, desc.ctypes.data_as(native.c_u32_p),
                                    code.ctypes.data_as(native.c_u32_p),
                                    flags.ctypes.data_as(native.c_u8_p), n.value, ctypes.byref(n),
                                    ctypes.byref(npr)))
        return desc[:n.value], code[:n.value], flags[:n.value], int(npr.value)

    def eval_fft_host(self, h_in, h_out, d_in, d_out, d_scratch, stream=None):
        nbytes = 0 if d_scratch is None else d_scratch.numel() * d_scratch.element_size()
        check(lib().sfft_eval_fft_host(self._h, _dptr(h_in), _dptr(h_out), _dptr(d_in),
                                       _dptr(d_out), _dptr(d_scratch), nbytes, _stream(stream)))

    def check(self, stream=None):
        """sfft_plan_check: raises SfftError (ETIMEOUT) if a device wait ran out."""
        check(lib().sfft_plan_check(self._h, _stream(stream)))

    def eval_fft_noalloc(self, d_in, d_out, stream=None):
        """sfft_eval_fft_noalloc: scratch in the library's fixed device array."""
        check(lib().sfft_eval_fft_noalloc(self._h, _dptr(d_in), _dptr(d_out), _stream(stream)))

    def set_timing(self, on):
        check(lib().sfft_plan_set_timing(self._h, 1 if on else 0))

    def timing(self):
        """(gate-kernel ms, B-expansion ms, levels launched, products) since the last read."""
        ms, xms = ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_uint64()
        g = ctypes.c_uint64()
        check(lib().sfft_plan_timing(self._h, ctypes.byref(ms), ctypes.byref(xms), ctypes.byref(n),
                                     ctypes.byref(g)))
        return ms.value, xms.value, n.value, g.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().sfft_plan_free(h)
            self._h = None


BATCH_NO_GRAPH = 4
BATCH_PERSISTENT = 128   # one persistent launch across levels (sfft.h SFFT_BATCH_PERSISTENT)


class Batch:
    """Many FFT requests evaluated level-merged (sfft_batch_create), graph-replayed."""

    def __init__(self, params, requests, flags=0):
        self.params = params
        self.requests = [tuple(r) for r in requests]
        arr = (native.sfft_request * len(self.requests))(*[native.sfft_request(*r) for r in self.requests])
        h = ctypes.c_void_p()
        check(lib().sfft_batch_create(ctypes.byref(params), arr, len(self.requests), flags,
                                      ctypes.byref(h)))
        self._h = h
        info = sfft_plan_info()
        check(lib().sfft_batch_info_get(h, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in sfft_plan_info._fields_}
        n = len(self.requests)
        i_off = (ctypes.c_uint64 * n)()
        o_off = (ctypes.c_uint64 * n)()
        check(lib().sfft_batch_offsets(h, i_off, o_off))
        self.in_off, self.out_off = list(i_off), list(o_off)

    def eval(self, d_in, d_out, d_scratch, stream=None):
        nbytes = 0 if d_scratch is None else d_scratch.numel() * d_scratch.element_size()
        check(lib().sfft_batch_eval(self._h, _dptr(d_in), _dptr(d_out), _dptr(d_scratch), nbytes,
                                    _stream(stream)))

    def eval_host(self, h_in, h_out, d_in, d_out, d_scratch, stream=None):
        nbytes = 0 if d_scratch is None else d_scratch.numel() * d_scratch.element_size()
        check(lib().sfft_batch_eval_host(self._h, _dptr(h_in), _dptr(h_out), _dptr(d_in),
                                         _dptr(d_out), _dptr(d_scratch), nbytes, _stream(stream)))

    def eval_host_pipelined(self, h_ins, h_outs, d_ins, d_outs, d_scratch, stream):
        """sfft_batch_eval_host_pipelined: len(h_ins) steps through two device
        buffer sets (d_ins, d_outs: two tensors each), copies overlapped."""
        n = len(h_ins)
        if len(h_outs) != n or len(d_ins) != 2 or len(d_outs) != 2:
            raise ValueError("need one output per input and two device buffer sets")
        arr = lambda ts: (ctypes.c_void_p * len(ts))(*[int(t.data_ptr()) for t in ts])  # noqa: E731
        nbytes = 0 if d_scratch is None else d_scratch.numel() * d_scratch.element_size()
        check(lib().sfft_batch_eval_host_pipelined(self._h, arr(h_ins), arr(h_outs), n, arr(d_ins),
                                                   arr(d_outs), _dptr(d_scratch), nbytes,
                                                   _stream(stream)))

    def check(self, stream=None):
        check(lib().sfft_batch_check(self._h, _stream(stream)))

    def set_epoch(self, epoch, stream=None):
        """Test hook: the persistent form's run counter (sfft_batch_set_epoch)."""
        check(lib().sfft_batch_set_epoch(self._h, epoch, _stream(stream)))

    def set_timing(self, on):
        check(lib().sfft_batch_set_timing(self._h, 1 if on else 0))

    def timing(self):
        """(gate-kernel ms, B-expansion ms, levels launched, products) since the last read."""
        ms, xms = ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_uint64()
        g = ctypes.c_uint64()
        check(lib().sfft_batch_timing(self._h, ctypes.byref(ms), ctypes.byref(xms), ctypes.byref(n),
                                      ctypes.byref(g)))
        return ms.value, xms.value, n.value, g.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().sfft_batch_free(h)
            self._h = None


def _hptr(a):
    """Host pointer of a numpy array or a CPU torch tensor."""
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    return ctypes.c_void_p(int(a.data_ptr()))


class Server:
    """Continuous-batching encrypted-FFT server (sfft_server_create)."""

    def __init__(self, params, hbm_budget_bytes, max_active=64, flags=0):
        self.params = params
        h = ctypes.c_void_p()
        check(lib().sfft_server_create(ctypes.byref(params), int(hbm_budget_bytes), max_active, flags,
                                       ctypes.byref(h)))
        self._h = h
        self._held = {}

    def prepare(self, request):
        """Compile a request shape ahead of its first submission (sfft_server_prepare)."""
        req = native.sfft_request(*request)
        check(lib().sfft_server_prepare(self._h, ctypes.byref(req)))

    def submit(self, request, h_in, h_out):
        """Queue one request; h_in / h_out stay referenced until wait()."""
        t = ctypes.c_uint64()
        req = native.sfft_request(*request)
        check(lib().sfft_server_submit(self._h, ctypes.byref(req), _hptr(h_in), _hptr(h_out),
                                       ctypes.byref(t)))
        self._held[t.value] = (h_in, h_out)
        return t.value

    def wait(self, ticket, timeout_ms=600000):
        lat = ctypes.c_double()
        check(lib().sfft_server_wait(self._h, ticket, timeout_ms, ctypes.byref(lat)))
        self._held.pop(ticket, None)
        return lat.value

    def stats(self):
        st = native.sfft_server_stats()
        check(lib().sfft_server_get_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in native.sfft_server_stats._fields_}

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().sfft_server_free(h)
            self._h = None
        self._held.clear()

    def __del__(self):
        self.close()


def gate_level(params, d_a, d_b, d_out0, d_out1, code0, code1, flags, stream=None, kernel=0):
    code0 = np.ascontiguousarray(code0, dtype=np.uint16)
    code1 = np.ascontiguousarray(code1, dtype=np.uint16)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    check(lib().sfft_gate_level(ctypes.byref(params), _dptr(d_a), _dptr(d_b), _dptr(d_out0),
                                _dptr(d_out1), code0.ctypes.data_as(native.c_u16_p),
                                code1.ctypes.data_as(native.c_u16_p),
                                flags.ctypes.data_as(native.c_u8_p), len(code0), kernel,
                                _stream(stream)))


INT_PEAK_OPS = ("iadd3", "lop3", "imad", "popc")


def measure_int_peak(op, iters=4096):
    """Measured integer-pipe rate of the current GPU (sfft_measure_int_peak),
    operations per second; op is an index into INT_PEAK_OPS or its name."""
    if isinstance(op, str):
        op = INT_PEAK_OPS.index(op)
    v = ctypes.c_double(0)
    check(lib().sfft_measure_int_peak(op, iters, ctypes.byref(v)))
    return float(v.value)


def autotune_small(params, n_gates=20000, reps=3):
    """Autotuner of the small-ciphertext kernel (sfft_autotune_small): returns
    (chosen ring depth, {depth: microseconds per gate})."""
    best = ctypes.c_uint32(0)
    us = (ctypes.c_double * 8)()
    check(lib().sfft_autotune_small(ctypes.byref(params), n_gates, reps, ctypes.byref(best), us))
    return int(best.value), {k + 1: float(us[k]) for k in range(8) if us[k] > 0}


def small_kernel_set_slots(ell, nslots):
    """Ring depth of the small-ciphertext kernel at ell (0: the default)."""
    check(lib().sfft_small_kernel_set_slots(ell, nslots))


def gate_level_withheld(params, d_a, d_b, d_out0, code0, flags, step, stream=None):
    """Failure-detection test hook (sfft_gate_level_withheld): raises SfftError
    with code SFFT_ETIMEOUT once the kernel's bounded waits have run out."""
    code0 = np.ascontiguousarray(code0, dtype=np.uint16)
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    check(lib().sfft_gate_level_withheld(ctypes.byref(params), _dptr(d_a), _dptr(d_b),
                                         _dptr(d_out0), code0.ctypes.data_as(native.c_u16_p),
                                         flags.ctypes.data_as(native.c_u8_p), len(code0), step,
                                         _stream(stream)))


def pack_code(c0, c1, c2, c3):
    return (c0 & 15) | ((c1 & 15) << 4) | ((c2 & 15) << 8) | ((c3 & 15) << 12)
