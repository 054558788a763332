"""Thin Python binding of libhe.so (include/he.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all arithmetic runs in the
library's CUDA kernels.  Device buffers are torch tensors (dtype int64 used as a container for
uint64 residues) on the current CUDA device; host arrays are numpy.  There is no CPU fallback:
if the library is missing or fails to load, `lib()` raises.
"""
import ctypes
import os

import numpy as np

HE_OK, HE_EINVAL, HE_ENOMEM, HE_ENOKEY, HE_ECUDA, HE_ETIMEOUT = 0, -1, -2, -3, -4, -5
HE_COEFF, HE_NTT = 0, 1
HE_DP_DOT, HE_DP_SHIFT, HE_DP_SHIFT_EXT, HE_CP_CP, HE_DP_DP = 0, 1, 2, 3, 4
HE_ROW_SWAP = 0x7FFFFFFF
HE_TUNE_TAP_TILE, HE_TUNE_TAP_ARITH, HE_TUNE_NTT_SPLIT, HE_TUNE_NTT_RADIX, HE_TUNE_LIMB_GROUPS = 0, 1, 2, 3, 4
HE_TUNE_BCONV_FUSED = 5
HE_TUNE_REPORT_LEN = 16
HE_RELIN_KEY = -0x80000000

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhe.so")


class HeParams(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_uint32), ("n_q", ctypes.c_uint32), ("q_bits", ctypes.c_uint32),
                ("n_p", ctypes.c_uint32), ("p_bits", ctypes.c_uint32), ("alpha", ctypes.c_uint32),
                ("t", ctypes.c_uint64)]


class HeCt(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n_polys", ctypes.c_uint32),
                ("n_limbs", ctypes.c_uint32), ("domain", ctypes.c_int32)]


class HeLayout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("I_c", "I_h", "I_w", "d", "stride", "pad", "r", "O_c", "pack", "modswitch")]


class HeNet(ctypes.Structure):
    _fields_ = [("conv", HeLayout), ("m1", ctypes.c_int32), ("m2", ctypes.c_int32)]


class HeMcConv(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("C_in", "H", "W", "d", "pad", "r", "O_c")]


class HeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_P = ctypes.c_void_p
_U64P = ctypes.POINTER(ctypes.c_uint64)
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_CTP = ctypes.POINTER(HeCt)
_SIGS = {
    "he_ctx_create": ([ctypes.POINTER(HeParams), _P, ctypes.POINTER(_P)], ctypes.c_int),
    "he_ctx_destroy": ([_P], None),
    "he_last_error": ([_P], ctypes.c_char_p),
    "he_set_stream": ([_P, _P], ctypes.c_int),
    "he_get_moduli": ([_P, _U64P, ctypes.c_int], ctypes.c_int),
    "he_op_counts": ([_P, _U64P], None),
    "he_reset_op_counts": ([_P], None),
    "he_launch_count": ([_P], ctypes.c_uint64),
    "he_set_phase_timing": ([_P, ctypes.c_int], ctypes.c_int),
    "he_phase_times": ([_P, ctypes.POINTER(ctypes.c_double), _U64P], ctypes.c_int),
    "he_gaussian_table": ([_U64P], None),
    "he_keygen_secret": ([_P, ctypes.c_uint64, _I64P], ctypes.c_int),
    "he_keygen_galois": ([_P, _I64P, ctypes.c_uint64, _I32P, ctypes.c_int], ctypes.c_int),
    "he_export_galois": ([_P, ctypes.c_int32, _U64P], ctypes.c_int),
    "he_load_keys": ([_P, _U64P, _I32P, ctypes.c_int], ctypes.c_int),
    "he_encrypt": ([_P, _I64P, _I64P, ctypes.c_uint64, _CTP], ctypes.c_int),
    "he_decrypt": ([_P, _I64P, _CTP, _I64P], ctypes.c_int),
    "he_to_ntt": ([_P, _CTP], ctypes.c_int),
    "he_to_coeff": ([_P, _CTP], ctypes.c_int),
    "he_encode": ([_P, _I64P, _P], ctypes.c_int),
    "he_rotate": ([_P, _CTP, ctypes.c_int32, _CTP], ctypes.c_int),
    "he_rotate_noalloc": ([_P, _CTP, ctypes.c_int32, _CTP], ctypes.c_int),
    "he_rotate_batch": ([_P, _CTP, ctypes.c_int, ctypes.c_int32, _CTP], ctypes.c_int),
    "he_automorphism": ([_P, _CTP, ctypes.c_int, ctypes.c_int32, _CTP], ctypes.c_int),
    "he_rotate_hoisted": ([_P, _CTP, _I32P, ctypes.c_int, _CTP], ctypes.c_int),
    "he_rotate_hoisted_batch": ([_P, _CTP, ctypes.c_int, _I32P, ctypes.c_int, _CTP], ctypes.c_int),
    "he_mul_plain_acc": ([_P, _CTP, _P, ctypes.c_int, _CTP], ctypes.c_int),
    "he_add": ([_P, _CTP, _CTP, _CTP], ctypes.c_int),
    "he_rescale": ([_P, _CTP, _CTP], ctypes.c_int),
    "he_multiply": ([_P, _CTP, _CTP, _CTP], ctypes.c_int),
    "he_multiply_batch": ([_P, _CTP, _CTP, ctypes.c_int, _CTP], ctypes.c_int),
    "he_fc_layer_batch": ([_P, _CTP, ctypes.c_int, _I32P, _I32P, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, _CTP], ctypes.c_int),
    "he_combine_batch": ([_P, _CTP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _CTP], ctypes.c_int),
    "he_net_required_steps": ([_P, ctypes.POINTER(HeNet), _I32P, ctypes.c_int], ctypes.c_int),
    "he_autotune": ([_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "he_probe_int_mac": ([_P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "he_probe_int_ops": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int], ctypes.c_int),
    "he_probe_mem": ([_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int], ctypes.c_int),
    "he_check": ([_P], ctypes.c_int),
    "he_tune_set": ([_P, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "he_tune_get": ([_P, ctypes.c_int, _I32P], ctypes.c_int),
    "he_set_wait_report": ([_P, ctypes.c_int], ctypes.c_int),
    "he_mc_conv_batch": ([_P, _CTP, ctypes.c_int, _I32P, _I32P, ctypes.POINTER(HeMcConv), _CTP],
                         ctypes.c_int),
    "he_rotate_sum_batch": ([_P, _CTP, ctypes.c_int, _I32P, ctypes.c_int], ctypes.c_int),
    "he_fc_mc_batch": ([_P, _CTP, ctypes.c_int, ctypes.c_int, _I32P, _I32P, _I32P, ctypes.c_int,
                        ctypes.c_int, ctypes.c_int, _CTP], ctypes.c_int),
    "he_deep_required_steps": ([_P, ctypes.POINTER(HeMcConv), ctypes.c_int, ctypes.c_int, _I32P,
                                ctypes.c_int], ctypes.c_int),
    "he_deep_batch": ([_P, _CTP, ctypes.c_int, ctypes.POINTER(HeMcConv), ctypes.c_int,
                       ctypes.POINTER(_I32P), ctypes.POINTER(_I32P), _I32P, ctypes.c_int, _CTP],
                      ctypes.c_int),
    "he_net_batch": ([_P, _CTP, ctypes.c_int, _I32P, _I32P, _I32P, _I32P, ctypes.POINTER(HeNet),
                      _CTP], ctypes.c_int),
    "he_ffconv_layer": ([_P, _CTP, _I32P, _I32P, ctypes.POINTER(HeLayout), _CTP], ctypes.c_int),
    "he_ffconv_layer_batch": ([_P, _CTP, ctypes.c_int, _I32P, _I32P, ctypes.POINTER(HeLayout), _CTP],
                              ctypes.c_int),
    "he_ffconv_required_steps": ([_P, ctypes.POINTER(HeLayout), _I32P, ctypes.c_int], ctypes.c_int),
    "he_ffconv_plan": ([_P, _I32P, _I32P, ctypes.POINTER(HeLayout), _I32P], ctypes.c_int),
    "he_ffconv_layer_planned": ([_P, ctypes.c_int32, _CTP, ctypes.c_int, _CTP], ctypes.c_int),
    "he_ffconv_plan_free": ([_P, ctypes.c_int32], ctypes.c_int),
    "he_ffconv_graph_create": ([_P, ctypes.c_int32, _CTP, ctypes.c_int, _CTP, ctypes.c_int, _I32P],
                               ctypes.c_int),
    "he_graph_launch": ([_P, ctypes.c_int32], ctypes.c_int),
    "he_graph_begin": ([_P, ctypes.c_int], ctypes.c_int),
    "he_graph_end": ([_P, _I32P], ctypes.c_int),
    "he_graph_free": ([_P, ctypes.c_int32], ctypes.c_int),
    "he_ntt": ([_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
}
_lib = None


def lib():
    """Load libhe.so (build it first with __graft_entry__.build() or build_ext.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


def _i64(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_I64P)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_I32P)


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(_U64P)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: the library has no CPU path")
    return torch


class Context:
    """An he_ctx plus the marshalling helpers; methods are named after the C entry points."""

    def __init__(self, log_n, n_q, n_p, alpha, t=65537, q_bits=50, p_bits=60, stream=None):
        torch = _torch()
        self.N = 1 << log_n
        self.L, self.K, self.alpha = n_q, n_p, alpha
        self.dnum = -(-n_q // alpha)
        self._graph_refs = {}                     # graph id -> the tensors it reads / writes
        prm = HeParams(log_n, n_q, q_bits, n_p, p_bits, alpha, t)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _P()
        rc = lib().he_ctx_create(ctypes.byref(prm), ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(h))
        if rc != HE_OK:
            raise HeError(rc, "he_ctx_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().he_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc, what):
        if rc != HE_OK:
            raise HeError(rc, f"{what}: {lib().he_last_error(self.h).decode()}")

    # ---- buffers
    def new_ct(self, level=None, count=None):
        torch = _torch()
        lv = self.L if level is None else level
        shape = (2, lv, self.N) if count is None else (count, 2, lv, self.N)
        with torch.cuda.stream(self.stream):      # ordered before the library's work on it
            return torch.zeros(shape, dtype=torch.int64, device="cuda")

    @staticmethod
    def ct_struct(t, domain=HE_NTT):
        return HeCt(t.data_ptr(), 2, t.shape[-2], domain)

    def ct_array(self, ts, domain=HE_NTT):
        if isinstance(ts, CtBatch):
            return ts.arr
        arr = (HeCt * len(ts))()
        for i, t in enumerate(ts):
            arr[i] = self.ct_struct(t, domain)
        return arr

    def ct_batch(self, ts, domain=HE_NTT):
        """Ciphertext tensors marshalled once, for repeated calls on the same list."""
        return CtBatch(self, ts, domain)

    def to_numpy(self, t):
        self.stream.synchronize()                  # the library may still be writing t
        return t.detach().cpu().numpy().view(np.uint64)

    def from_numpy(self, a):
        torch = _torch()
        with torch.cuda.stream(self.stream):
            return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()

    # ---- context
    def he_get_moduli(self):
        out = np.zeros(64, dtype=np.uint64)
        n = lib().he_get_moduli(self.h, out.ctypes.data_as(_U64P), 64)
        return [int(x) for x in out[:n]]

    def he_op_counts(self):
        out = np.zeros(4, dtype=np.uint64)
        lib().he_op_counts(self.h, out.ctypes.data_as(_U64P))
        return {"mulpc": int(out[0]), "addcc": int(out[1]), "rot": int(out[2]), "ks": int(out[3])}

    def he_launch_count(self):
        return int(lib().he_launch_count(self.h))

    PHASES = ("encode", "modup", "taps", "moddown", "rotate", "restore", "multiply")

    def he_set_phase_timing(self, enable):
        self._ck(lib().he_set_phase_timing(self.h, int(enable)), "he_set_phase_timing")

    def he_phase_times(self):
        """{phase: (milliseconds, spans)} summed since the last call (synchronises the stream)."""
        ms = (ctypes.c_double * 8)()
        calls = np.zeros(8, dtype=np.uint64)
        self._ck(lib().he_phase_times(self.h, ms, calls.ctypes.data_as(_U64P)), "he_phase_times")
        return {name: (ms[i], int(calls[i])) for i, name in enumerate(self.PHASES)}

    def he_reset_op_counts(self):
        lib().he_reset_op_counts(self.h)

    # ---- client side
    def he_keygen_secret(self, seed):
        out = np.zeros(self.N, dtype=np.int64)
        self._ck(lib().he_keygen_secret(self.h, seed, out.ctypes.data_as(_I64P)), "he_keygen_secret")
        return out

    def he_keygen_galois(self, sk, seed, steps):
        sk, psk = _i64(sk)
        st, pst = _i32(steps)
        self._ck(lib().he_keygen_galois(self.h, psk, seed, pst, len(st)), "he_keygen_galois")

    def key_words(self):
        return self.dnum * 2 * (self.L + self.K) * self.N

    def he_export_galois(self, step):
        out = np.zeros(self.key_words(), dtype=np.uint64)
        self._ck(lib().he_export_galois(self.h, step, out.ctypes.data_as(_U64P)), "he_export_galois")
        return out.reshape(self.dnum, 2, self.L + self.K, self.N)

    def he_load_keys(self, blob, steps):
        b, pb = _u64(blob)
        st, pst = _i32(steps)
        self._ck(lib().he_load_keys(self.h, pb, pst, len(st)), "he_load_keys")

    def he_encrypt(self, sk, slots, seed, domain=HE_NTT, out=None):
        out = self.new_ct() if out is None else out
        sk, psk = _i64(sk)
        sl, psl = _i64(slots)
        c = self.ct_struct(out, domain)
        self._ck(lib().he_encrypt(self.h, psk, psl, seed, ctypes.byref(c)), "he_encrypt")
        return out

    def he_decrypt(self, sk, ct, domain=HE_NTT):
        sk, psk = _i64(sk)
        out = np.zeros(self.N, dtype=np.int64)
        c = self.ct_struct(ct, domain)
        self._ck(lib().he_decrypt(self.h, psk, ctypes.byref(c), out.ctypes.data_as(_I64P)), "he_decrypt")
        return out

    # ---- evaluation
    def he_to_ntt(self, ct):
        c = self.ct_struct(ct, HE_COEFF)
        self._ck(lib().he_to_ntt(self.h, ctypes.byref(c)), "he_to_ntt")
        return ct

    def he_to_coeff(self, ct):
        c = self.ct_struct(ct, HE_NTT)
        self._ck(lib().he_to_coeff(self.h, ctypes.byref(c)), "he_to_coeff")
        return ct

    def he_encode(self, slots):
        torch = _torch()
        with torch.cuda.stream(self.stream):
            out = torch.zeros((self.L, self.N), dtype=torch.int64, device="cuda")
        sl, psl = _i64(slots)
        self._ck(lib().he_encode(self.h, psl, ctypes.c_void_p(out.data_ptr())), "he_encode")
        return out

    def he_rotate(self, ct, step, out=None):
        out = self.new_ct() if out is None else out
        a, b = self.ct_struct(ct), self.ct_struct(out)
        self._ck(lib().he_rotate(self.h, ctypes.byref(a), step, ctypes.byref(b)), "he_rotate")
        return out

    def he_rotate_noalloc(self, ct, step, out):
        """he_rotate for callers that cannot allocate device memory: the library's scratch is
        a fixed static device array, and `out` must be supplied by the caller."""
        a, b = self.ct_struct(ct), self.ct_struct(out)
        self._ck(lib().he_rotate_noalloc(self.h, ctypes.byref(a), step, ctypes.byref(b)),
                 "he_rotate_noalloc")
        return out

    def he_rotate_batch(self, cts, step, outs=None):
        outs = [self.new_ct() for _ in cts] if outs is None else outs
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        self._ck(lib().he_rotate_batch(self.h, ia, len(cts), step, oa), "he_rotate_batch")
        return outs

    def he_automorphism(self, cts, step, outs=None):
        outs = [self.new_ct() for _ in cts] if outs is None else outs
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        self._ck(lib().he_automorphism(self.h, ia, len(cts), step, oa), "he_automorphism")
        return outs

    def he_rotate_hoisted(self, ct, steps, outs=None):
        outs = [self.new_ct() for _ in steps] if outs is None else outs
        a = self.ct_struct(ct)
        st, pst = _i32(steps)
        oa = self.ct_array(outs)
        self._ck(lib().he_rotate_hoisted(self.h, ctypes.byref(a), pst, len(st), oa), "he_rotate_hoisted")
        return outs

    def he_rotate_hoisted_batch(self, cts, steps, outs=None):
        """outs[i * h + s]: cts[i] rotated by steps[s] (one ModUp per ciphertext)."""
        outs = [self.new_ct() for _ in range(len(cts) * len(steps))] if outs is None else outs
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        st, pst = _i32(steps)
        self._ck(lib().he_rotate_hoisted_batch(self.h, ia, len(cts), pst, len(st), oa),
                 "he_rotate_hoisted_batch")
        return outs

    def he_mul_plain_acc(self, cts, pts, acc):
        ia = self.ct_array(cts)
        c = self.ct_struct(acc)
        self._ck(lib().he_mul_plain_acc(self.h, ia, ctypes.c_void_p(pts.data_ptr()), len(cts),
                                        ctypes.byref(c)), "he_mul_plain_acc")
        return acc

    def he_add(self, a, b, out=None, domain=HE_NTT):
        out = self.new_ct(level=a.shape[-2]) if out is None else out
        x, y, z = self.ct_struct(a, domain), self.ct_struct(b, domain), self.ct_struct(out, domain)
        self._ck(lib().he_add(self.h, ctypes.byref(x), ctypes.byref(y), ctypes.byref(z)), "he_add")
        return out

    def he_multiply(self, a, b, out=None):
        out = self.new_ct() if out is None else out
        x, y, z = self.ct_struct(a), self.ct_struct(b), self.ct_struct(out)
        self._ck(lib().he_multiply(self.h, ctypes.byref(x), ctypes.byref(y), ctypes.byref(z)),
                 "he_multiply")
        return out

    def he_multiply_batch(self, a, b, outs=None):
        outs = [self.new_ct() for _ in a] if outs is None else outs
        x, y, z = self.ct_array(a), self.ct_array(b), self.ct_array(outs)
        self._ck(lib().he_multiply_batch(self.h, x, y, len(a), z), "he_multiply_batch")
        return outs

    def he_fc_layer_batch(self, cts, F, pos, period, outs=None):
        outs = [self.new_ct() for _ in cts] if outs is None else outs
        f, pf = _i32(F)
        ps, pp = _i32(pos)
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        self._ck(lib().he_fc_layer_batch(self.h, ia, len(cts), pf, pp, len(ps), f.shape[0], period,
                                         oa), "he_fc_layer_batch")
        return outs

    def he_combine_batch(self, cts, n_ch, block, outs=None):
        """cts: [B][n_ch] ciphertexts flattened image-major."""
        B = len(cts) // n_ch
        outs = [self.new_ct() for _ in range(B)] if outs is None else outs
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        self._ck(lib().he_combine_batch(self.h, ia, B, n_ch, block, oa), "he_combine_batch")
        return outs

    @staticmethod
    def net(lay, m1, m2):
        return HeNet(lay, m1, m2)

    def he_net_required_steps(self, net):
        out = np.zeros(8192, dtype=np.int32)
        n = lib().he_net_required_steps(self.h, ctypes.byref(net), out.ctypes.data_as(_I32P), 8192)
        if n < 0:
            raise HeError(n, "he_net_required_steps: shape does not fit the ring")
        return [int(x) for x in out[:n]]

    def he_net_batch(self, cts_in, W1, W2, F1, F2, net, outs=None):
        """cts_in: B ciphertexts (B * K Im2Col columns for HE_CP_CP)."""
        B = len(cts_in)
        if net.conv.pack == HE_CP_CP:
            B //= net.conv.d * net.conv.d * net.conv.I_c
        outs = [self.new_ct() for _ in range(B)] if outs is None else outs
        ia, oa = self.ct_array(cts_in), self.ct_array(outs)
        w1, pw1 = _i32(W1)
        w2, pw2 = _i32(W2)
        f1, pf1 = _i32(F1)
        f2, pf2 = _i32(F2)
        self._ck(lib().he_net_batch(self.h, ia, B, pw1, pw2, pf1, pf2, ctypes.byref(net), oa),
                 "he_net_batch")
        return outs

    def he_autotune(self, batch, force_tile=0):
        """Tune the NTT split and the tap kernel's tile and arithmetic by timing (force_tile
        128 / 256 only sets the tile).  Returns the report as a dict: tap-kernel ms per launch
        by (tile, arithmetic), the NTT ms and split, and the choices."""
        ms = (ctypes.c_double * HE_TUNE_REPORT_LEN)()
        self._ck(lib().he_autotune(self.h, batch, force_tile, ms), "he_autotune")
        return {"tap_ms": {"128_chains": ms[0], "128_columns": ms[1], "256_chains": ms[2],
                           "256_columns": ms[3], "128_products": ms[8]},
                "ntt_ms": ms[4], "ntt_log2_n1": int(ms[5]), "ntt_radix": int(ms[9]),
                "conversion_ms": {"1": ms[10], "2": ms[11], "4": ms[12]},
                "limb_groups": int(ms[13]), "tap_tile": int(ms[6]),
                "bconv_ms": {"separate": ms[14], "fused": ms[15]},
                "bconv": ("separate", "fused")[self.he_tune_get(HE_TUNE_BCONV_FUSED)],
                "tap_arith": ("chains", "columns", "products")[int(ms[7])]}

    def he_tune_set(self, knob, value):
        self._ck(lib().he_tune_set(self.h, knob, int(value)), "he_tune_set")

    def he_tune_get(self, knob):
        v = (ctypes.c_int32 * 1)()
        self._ck(lib().he_tune_get(self.h, knob, v), "he_tune_get")
        return int(v[0])

    def he_probe_int_mac(self):
        """Measured 64 x 64 -> 128-bit products/s: (carry chain, 32-bit column sums)."""
        out = (ctypes.c_double * 2)()
        self._ck(lib().he_probe_int_mac(self.h, out), "he_probe_int_mac")
        return float(out[0]), float(out[1])

    def he_check(self):
        """Wait for the stream; raise HeError (HE_ETIMEOUT) if a bounded device wait ran out
        since the last check, or HE_ECUDA if a kernel failed."""
        self._ck(lib().he_check(self.h), "he_check")

    def he_set_wait_report(self, polls):
        """Test hook: polls before the tap kernel reports a stage wait (-1: the default)."""
        self._ck(lib().he_set_wait_report(self.h, int(polls)), "he_set_wait_report")

    def he_probe_int_ops(self):
        """Rates per second: carry-chain, column and Karatsuba products; mad.lo / mad.hi /
        mad.wide.u32 instructions; products of the 64-bit add-with-carry residue form."""
        out = (ctypes.c_double * 7)()
        self._ck(lib().he_probe_int_ops(self.h, out, 7), "he_probe_int_ops")
        return dict(zip(("chain", "columns", "karatsuba", "mad_lo", "mad_hi", "mad_wide",
                         "chain_wide"), (float(v) for v in out)))

    def he_probe_mem(self):
        """Read GB/s of an L2-resident buffer and of an HBM-sized one."""
        out = (ctypes.c_double * 2)()
        self._ck(lib().he_probe_mem(self.h, out, 2), "he_probe_mem")
        return {"l2_read_gbs": float(out[0]), "hbm_read_gbs": float(out[1])}

    # ---- deeper networks (several ciphertexts per tensor)
    @staticmethod
    def mc_conv(C_in, H, W, d, r, O_c):
        """Stride-1 same convolution; r = 0 (or None) for the unfactorized layer."""
        return HeMcConv(C_in, H, W, d, (d - 1) // 2, int(r or 0), O_c)

    def mc_cts(self, channels, H, W):
        """Ciphertexts holding `channels` maps of H x W in the block layout."""
        bk = 1 << max(0, (H * W - 1).bit_length())
        g = (self.N // 2) // bk
        return -(-channels // g)

    def he_mc_conv_batch(self, cts, W1, W2, conv, outs=None):
        n_in = self.mc_cts(conv.C_in, conv.H, conv.W)
        B = len(cts) // n_in
        n_out = self.mc_cts(conv.O_c, conv.H, conv.W)
        outs = [self.new_ct() for _ in range(B * n_out)] if outs is None else outs
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        w1, pw1 = _i32(W1)
        if W2 is None:
            pw2 = None
        else:
            w2, pw2 = _i32(W2)
        self._ck(lib().he_mc_conv_batch(self.h, ia, B, pw1, pw2, ctypes.byref(conv), oa),
                 "he_mc_conv_batch")
        return outs

    def he_rotate_sum_batch(self, cts, steps):
        st, pst = _i32(steps)
        arr = self.ct_array(cts)
        self._ck(lib().he_rotate_sum_batch(self.h, arr, len(cts), pst, len(st)), "he_rotate_sum_batch")
        return cts

    def he_fc_mc_batch(self, cts, n_ct, F, ct_of, pos, period, outs=None):
        B = len(cts) // n_ct
        outs = [self.new_ct() for _ in range(B)] if outs is None else outs
        f, pf = _i32(F)
        co, pco = _i32(ct_of)
        ps, pps = _i32(pos)
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        self._ck(lib().he_fc_mc_batch(self.h, ia, B, n_ct, pf, pco, pps, len(ps), f.shape[0], period,
                                      oa), "he_fc_mc_batch")
        return outs

    def he_deep_required_steps(self, convs, n_cls):
        arr = (HeMcConv * len(convs))(*convs)
        out = np.zeros(8192, dtype=np.int32)
        n = lib().he_deep_required_steps(self.h, arr, len(convs), n_cls, out.ctypes.data_as(_I32P), 8192)
        if n < 0:
            raise HeError(n, "he_deep_required_steps: shape does not fit the ring")
        return [int(x) for x in out[:n]]

    def he_deep_batch(self, cts, convs, W1s, W2s, F, outs=None):
        n_in = self.mc_cts(convs[0].C_in, convs[0].H, convs[0].W)
        B = len(cts) // n_in
        outs = [self.new_ct() for _ in range(B)] if outs is None else outs
        keep = [_i32(w) for w in W1s]
        keep2 = [None if w is None else _i32(w) for w in W2s]
        p1 = (_I32P * len(convs))(*[k[1] for k in keep])
        p2 = (_I32P * len(convs))(*[(k[1] if k is not None else _I32P()) for k in keep2])
        f, pf = _i32(F)
        arr = (HeMcConv * len(convs))(*convs)
        ia, oa = self.ct_array(cts), self.ct_array(outs)
        self._ck(lib().he_deep_batch(self.h, ia, B, arr, len(convs), p1, p2, pf, f.shape[0], oa),
                 "he_deep_batch")
        return outs

    def he_rescale(self, ct, out=None):
        out = self.new_ct(level=ct.shape[-2] - 1) if out is None else out
        a, b = self.ct_struct(ct), self.ct_struct(out)
        self._ck(lib().he_rescale(self.h, ctypes.byref(a), ctypes.byref(b)), "he_rescale")
        return out

    @staticmethod
    def layout(I_c, I_h, I_w, d, stride, pad, r, O_c, pack="dp_shift", modswitch=False):
        packs = {"dp_dot": HE_DP_DOT, "dp_shift": HE_DP_SHIFT, "dp_shift_ext": HE_DP_SHIFT_EXT,
                 "cp_cp": HE_CP_CP, "dp_dp": HE_DP_DP}
        return HeLayout(I_c, I_h, I_w, d, stride, pad, r, O_c, packs[pack], int(bool(modswitch)))

    def he_ffconv_required_steps(self, lay):
        out = np.zeros(4096, dtype=np.int32)
        n = lib().he_ffconv_required_steps(self.h, ctypes.byref(lay), out.ctypes.data_as(_I32P), 4096)
        if n < 0:
            raise HeError(n, "he_ffconv_required_steps: layout does not fit the ring")
        return [int(x) for x in out[:n]]

    def he_ffconv_layer_batch(self, cts_in, W1, W2, lay, outs=None):
        """cts_in: B ciphertexts, or for HE_CP_CP B * K Im2Col column ciphertexts."""
        B = len(cts_in)
        if lay.pack == HE_CP_CP:
            B //= lay.d * lay.d * lay.I_c
        lv = self.L - 1 if lay.modswitch else self.L
        outs = [self.new_ct(level=lv) for _ in range(B * lay.O_c)] if outs is None else outs
        ia, oa = self.ct_array(cts_in), self.ct_array(outs)
        w1, pw1 = _i32(W1)
        w2, pw2 = _i32(W2)
        self._ck(lib().he_ffconv_layer_batch(self.h, ia, B, pw1, pw2, ctypes.byref(lay), oa),
                 "he_ffconv_layer_batch")
        return outs

    def he_ffconv_plan(self, W1, W2, lay):
        w1, pw1 = _i32(W1)
        w2, pw2 = _i32(W2)
        pid = (ctypes.c_int32 * 1)()
        self._ck(lib().he_ffconv_plan(self.h, pw1, pw2, ctypes.byref(lay), pid), "he_ffconv_plan")
        return int(pid[0])

    def he_ffconv_layer_planned(self, plan, cts_in, lay, outs=None):
        """lay: the plan's layout (for the output count); cts_in as for he_ffconv_layer_batch."""
        B = len(cts_in)
        if lay.pack == HE_CP_CP:
            B //= lay.d * lay.d * lay.I_c
        lv = self.L - 1 if lay.modswitch else self.L
        outs = [self.new_ct(level=lv) for _ in range(B * lay.O_c)] if outs is None else outs
        ia, oa = self.ct_array(cts_in), self.ct_array(outs)
        self._ck(lib().he_ffconv_layer_planned(self.h, plan, ia, B, oa), "he_ffconv_layer_planned")
        return outs

    def he_ffconv_plan_free(self, plan):
        self._ck(lib().he_ffconv_plan_free(self.h, plan), "he_ffconv_plan_free")

    def he_ffconv_graph_create(self, plan, cts_in, lay, outs=None, share_scratch=False):
        """Captures the planned layer on these buffers; returns (graph id, outs).  The
        tensors stay referenced here until he_graph_free, since the graph reads and writes
        them in place at every he_graph_launch."""
        B = len(cts_in)
        if lay.pack == HE_CP_CP:
            B //= lay.d * lay.d * lay.I_c
        lv = self.L - 1 if lay.modswitch else self.L
        outs = [self.new_ct(level=lv) for _ in range(B * lay.O_c)] if outs is None else outs
        ia, oa = self.ct_array(cts_in), self.ct_array(outs)
        gid = (ctypes.c_int32 * 1)()
        self._ck(lib().he_ffconv_graph_create(self.h, plan, ia, B, oa, int(bool(share_scratch)), gid),
                 "he_ffconv_graph_create")
        self._graph_refs[int(gid[0])] = (list(cts_in), list(outs))
        return int(gid[0]), outs

    def he_graph_begin(self, share_scratch=False):
        """Start recording the calls that follow on this context (see he_graph_end)."""
        self._ck(lib().he_graph_begin(self.h, int(bool(share_scratch))), "he_graph_begin")

    def he_graph_end(self, keep=()):
        """Finish the recording; returns the graph id.  `keep`: tensors the recorded calls
        read or write, held here until he_graph_free."""
        gid = (ctypes.c_int32 * 1)()
        self._ck(lib().he_graph_end(self.h, gid), "he_graph_end")
        self._graph_refs[int(gid[0])] = list(keep)
        return int(gid[0])

    def he_graph_launch(self, graph):
        self._ck(lib().he_graph_launch(self.h, graph), "he_graph_launch")

    def he_graph_free(self, graph):
        self._ck(lib().he_graph_free(self.h, graph), "he_graph_free")
        self._graph_refs.pop(graph, None)

    def he_ffconv_layer(self, ct_in, W1, W2, lay, outs=None):
        lv = self.L - 1 if lay.modswitch else self.L
        outs = [self.new_ct(level=lv) for _ in range(lay.O_c)] if outs is None else outs
        a = self.ct_struct(ct_in)
        oa = self.ct_array(outs)
        w1, pw1 = _i32(W1)
        w2, pw2 = _i32(W2)
        self._ck(lib().he_ffconv_layer(self.h, ctypes.byref(a), pw1, pw2, ctypes.byref(lay), oa),
                 "he_ffconv_layer")
        return outs

    def he_ntt(self, data, n_items, n_limbs, inverse=False):
        self._ck(lib().he_ntt(self.h, ctypes.c_void_p(data.data_ptr()), n_items, n_limbs, int(inverse)),
                 "he_ntt")
        return data


class CtBatch:
    """A list of ciphertext tensors with its C-ABI struct array built once; accepted wherever a
    list of ciphertexts is.  The tensors are kept alive by it."""

    def __init__(self, ctx, ts, domain=HE_NTT):
        self.ts = list(ts)
        self.arr = (HeCt * len(self.ts))()
        for i, t in enumerate(self.ts):
            self.arr[i] = ctx.ct_struct(t, domain)

    def __len__(self):
        return len(self.ts)

    def __getitem__(self, i):
        return self.ts[i]

    def __iter__(self):
        return iter(self.ts)


def he_gaussian_table():
    out = np.zeros(20, dtype=np.uint64)
    lib().he_gaussian_table(out.ctypes.data_as(_U64P))
    return [int(x) for x in out]
