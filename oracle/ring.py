"""Thin ctypes wrapper over oracle/ring.c (exact Z_q and Z_q[X]/(X^n+1) arithmetic).

Test infrastructure: the independent CPU oracle.  All arrays are numpy uint64, C-contiguous.
"""
import ctypes

import numpy as np

from .build import build

_U64P = ctypes.POINTER(ctypes.c_uint64)
_I64P = ctypes.POINTER(ctypes.c_int64)
_u64 = ctypes.c_uint64
_i64 = ctypes.c_int64
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    sig = {
        "orc_powmod": ([_u64, _u64, _u64], _u64),
        "orc_vec_add": ([_U64P, _U64P, _U64P, _i64, _u64], None),
        "orc_vec_sub": ([_U64P, _U64P, _U64P, _i64, _u64], None),
        "orc_vec_mul": ([_U64P, _U64P, _U64P, _i64, _u64], None),
        "orc_vec_mul_scalar": ([_U64P, _u64, _U64P, _i64, _u64], None),
        "orc_vec_mac_scalar": ([_U64P, _U64P, _u64, _U64P, _i64, _u64], None),
        "orc_vec_reduce": ([_U64P, _U64P, _i64, _u64], None),
        "orc_vec_from_signed": ([_I64P, _U64P, _i64, _u64], None),
        "orc_negacyclic_schoolbook": ([_U64P, _U64P, _U64P, _i64, _u64], None),
        "orc_negacyclic_coeff": ([_U64P, _U64P, _i64, _u64, _i64], _u64),
        "orc_negacyclic_eval": ([_U64P, _U64P, _i64, _u64, _u64], None),
        "orc_negacyclic_interp": ([_U64P, _U64P, _i64, _u64, _u64], None),
        "orc_negacyclic_mul": ([_U64P, _U64P, _U64P, _i64, _u64, _u64], None),
        "orc_uniform_mod": ([_U64P, _U64P, _u64, _i64, _U64P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _u(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(_U64P)


def _out(n):
    o = np.empty(n, dtype=np.uint64)
    return o, o.ctypes.data_as(_U64P)


def vadd(a, b, q):
    a, pa = _u(a); b, pb = _u(b); o, po = _out(a.size)
    _load().orc_vec_add(pa, pb, po, a.size, q)
    return o.reshape(a.shape)


def vsub(a, b, q):
    a, pa = _u(a); b, pb = _u(b); o, po = _out(a.size)
    _load().orc_vec_sub(pa, pb, po, a.size, q)
    return o.reshape(a.shape)


def vmul(a, b, q):
    a, pa = _u(a); b, pb = _u(b); o, po = _out(a.size)
    _load().orc_vec_mul(pa, pb, po, a.size, q)
    return o.reshape(a.shape)


def vmul_scalar(a, s, q):
    a, pa = _u(a); o, po = _out(a.size)
    _load().orc_vec_mul_scalar(pa, int(s) % q, po, a.size, q)
    return o.reshape(a.shape)


def vmac_scalar(acc, a, s, q):
    """(acc + a * s) mod q."""
    acc, pc = _u(acc); a, pa = _u(a); o, po = _out(a.size)
    _load().orc_vec_mac_scalar(pc, pa, int(s) % q, po, a.size, q)
    return o.reshape(a.shape)


def vreduce(a, q):
    a, pa = _u(a); o, po = _out(a.size)
    _load().orc_vec_reduce(pa, po, a.size, q)
    return o.reshape(a.shape)


def from_signed(a, q):
    """Signed int64 array -> residues in [0, q)."""
    a = np.ascontiguousarray(a, dtype=np.int64)
    o, po = _out(a.size)
    _load().orc_vec_from_signed(a.ctypes.data_as(_I64P), po, a.size, q)
    return o.reshape(a.shape)


def polymul_schoolbook(a, b, q):
    a, pa = _u(a); b, pb = _u(b); o, po = _out(a.size)
    _load().orc_negacyclic_schoolbook(pa, pb, po, a.size, q)
    return o


def polymul_coeff(a, b, q, k):
    """Coefficient k of a*b in Z_q[X]/(X^n+1), straight from the definition."""
    a, pa = _u(a); b, pb = _u(b)
    return int(_load().orc_negacyclic_coeff(pa, pb, a.size, q, k))


def neg_eval(a, q, psi):
    a, pa = _u(a); o, po = _out(a.size)
    _load().orc_negacyclic_eval(pa, po, a.size, q, psi)
    return o


def neg_interp(v, q, psi):
    v, pv = _u(v); o, po = _out(v.size)
    _load().orc_negacyclic_interp(pv, po, v.size, q, psi)
    return o


def polymul(a, b, q, psi):
    a, pa = _u(a); b, pb = _u(b); o, po = _out(a.size)
    _load().orc_negacyclic_mul(pa, pb, po, a.size, q, psi)
    return o


def uniform_mod(hi, lo, q):
    hi, ph = _u(hi); lo, pl = _u(lo); o, po = _out(hi.size)
    _load().orc_uniform_mod(ph, pl, q, hi.size, po)
    return o
