"""CPU oracle for the symplectic minimum distance -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
import this package.  The GPU library never does: it shares no code with it.

Two independent computations of d = min{ wt_s(c) : c in C, c != 0 } with
wt_s(a, b) = #{i : a_i != 0 or b_i != 0} (Section 2, definitions):

* :func:`bruteforce` -- every codeword once (Gray-code walk over a basis).
* :func:`bz` -- Algorithm 3 (Saved_isometry): (a, b) -> (a, b, a + b), plain
  binary Brouwer-Zimmermann for the Hamming weight (Section 2.1), d = d_H / 2.

Inputs use the library's layout: ``field=2`` -> uint8 array (K, 2n) of bits
(x | z); ``field=4`` -> uint8 array (K, n) of F4 symbols v = a + 2b meaning
a + alpha*b.  ``n_stab`` > 0 takes the minimum over C minus the span of the
first ``n_stab`` rows (the modified algorithm's check, Section 2.1).
"""
import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, EINCOMPLETE, EZERO = 0, -1, -5, -6


class OracleResult(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("lower", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("n_gamma", ctypes.c_int32), ("k_eff", ctypes.c_int32),
                ("complete", ctypes.c_int32), ("codewords", ctypes.c_uint64),
                ("seconds", ctypes.c_double), ("threads", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        L.oracle_bruteforce.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), u8p,
                                        ctypes.POINTER(ctypes.c_uint64)]
        L.oracle_bruteforce.restype = ctypes.c_int
        L.oracle_bz.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_double, ctypes.POINTER(OracleResult),
                                u8p, ctypes.POINTER(ctypes.c_int32), ctypes.c_int,
                                ctypes.POINTER(ctypes.c_int)]
        L.oracle_bz.restype = ctypes.c_int
        L.oracle_iso_weight.argtypes = [u8p, ctypes.c_int]
        L.oracle_iso_weight.restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed with code %d" % (what, code))
        self.code = code


def _prep(gen, field):
    g = np.ascontiguousarray(np.asarray(gen, dtype=np.uint8))
    if g.ndim != 2:
        raise ValueError("generator must be 2-D")
    K = g.shape[0]
    n = g.shape[1] // 2 if field == 2 else g.shape[1]
    return g, n, K


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def bruteforce(gen, field=2, n_stab=0, threads=0, want_wdist=False):
    """Returns (d, witness[2n], wdist or None); wdist[w] counts codewords of weight w."""
    g, n, K = _prep(gen, field)
    d = ctypes.c_int(0)
    wit = np.zeros(2 * n, dtype=np.uint8)
    wd = np.zeros(n + 1, dtype=np.uint64) if want_wdist else None
    rc = lib().oracle_bruteforce(_ptr(g), n, K, field, n_stab, threads, ctypes.byref(d),
                                 _ptr(wit),
                                 wd.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
                                 if wd is not None else None)
    if rc != OK:
        raise OracleError(rc, "oracle_bruteforce")
    return d.value, wit, wd


def bz(gen, field=2, n_stab=0, threads=0, time_budget=0.0, ltrace_cap=0, allow_incomplete=False):
    """Algorithm 3 + plain Brouwer-Zimmermann.  Returns a dict with d, lower, rounds,
    n_gamma, k_eff, complete, codewords, seconds, threads, witness, ltrace."""
    g, n, K = _prep(gen, field)
    res = OracleResult()
    wit = np.zeros(2 * n, dtype=np.uint8)
    lt = (ctypes.c_int32 * max(ltrace_cap, 1))()
    ln = ctypes.c_int(0)
    rc = lib().oracle_bz(_ptr(g), n, K, field, n_stab, threads, float(time_budget),
                         ctypes.byref(res), _ptr(wit), lt if ltrace_cap else None,
                         ltrace_cap, ctypes.byref(ln))
    if rc != OK and not (allow_incomplete and rc == EINCOMPLETE):
        raise OracleError(rc, "oracle_bz")
    out = {f: getattr(res, f) for f, _ in OracleResult._fields_ if f != "pad"}
    out["witness"] = wit
    out["ltrace"] = [lt[i] for i in range(ln.value)]
    out["status"] = rc
    return out


def iso_weight(row, n):
    r = np.ascontiguousarray(np.asarray(row, dtype=np.uint8))
    return lib().oracle_iso_weight(_ptr(r), n)
