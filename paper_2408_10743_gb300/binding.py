"""ctypes binding of libdist (include/dist.h): the same entry points, argument
marshalling only.  All computation happens inside the library; there is no
Python or CPU fallback -- if libdist.so cannot be built or loaded, or no CUDA
device is present, the calls raise.

Streams: pass a ``torch.cuda.Stream`` (or its integer handle) as ``stream``;
None selects the stream owned by the code object.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

DIST_F2, DIST_F4 = 2, 4
DIST_OK = 0
DIST_EINVAL, DIST_ENOMEM, DIST_ECUDA, DIST_ETIMEOUT = -1, -2, -3, -4
DIST_EINCOMPLETE, DIST_EZERO, DIST_EBUSY, DIST_EINTERNAL, DIST_ERANGE = -5, -6, -7, -8, -9


class DistResult(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("lower", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("k_eff", ctypes.c_int32), ("n_gamma", ctypes.c_int32),
                ("status", ctypes.c_int32), ("codewords", ctypes.c_uint64),
                ("seconds", ctypes.c_double), ("witness", ctypes.c_uint8 * 256),
                ("coeffs", ctypes.c_uint8 * 256), ("gpu_seconds", ctypes.c_double),
                ("launches", ctypes.c_uint64)]


# The same layout as a numpy structured dtype: an array of dist_result viewed
# without copying (Batch.wait_array).
RESULT_DTYPE = np.dtype({
    "names": [f for f, _ in DistResult._fields_],
    "formats": [{"witness": (np.uint8, 256), "coeffs": (np.uint8, 256), "codewords": np.uint64,
                 "launches": np.uint64, "seconds": np.float64, "gpu_seconds": np.float64}.get(f, np.int32)
                for f, _ in DistResult._fields_],
    "offsets": [getattr(DistResult, f).offset for f, _ in DistResult._fields_],
    "itemsize": ctypes.sizeof(DistResult)})


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_gamma_built", ctypes.c_int32), ("n_gamma_used", ctypes.c_int32),
                ("k_eff", ctypes.c_int32), ("s_rank", ctypes.c_int32),
                ("d_est", ctypes.c_int32), ("u0", ctypes.c_int32),
                ("order", ctypes.c_int32 * 16), ("a", ctypes.c_int32 * 16),
                ("b", ctypes.c_int32 * 16), ("f", ctypes.c_int32 * 16)]


class IntpeakResult(ctypes.Structure):
    _fields_ = [("mix_per_s", ctypes.c_double), ("popc_per_s", ctypes.c_double),
                ("lop3_per_s", ctypes.c_double), ("sm_mhz", ctypes.c_double),
                ("sms", ctypes.c_int32), ("blocks", ctypes.c_int32)]


class Tuning(ctypes.Structure):
    _fields_ = [("chunks_per_warp", ctypes.c_int32), ("lane_cap_log2", ctypes.c_int32),
                ("lane_floor_log2", ctypes.c_int32),
                ("codewords_per_s", ctypes.c_double)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("slice_ms", ctypes.c_double), ("max_resident_bytes", ctypes.c_uint64),
                ("time_limit_s", ctypes.c_double)]


class BatchStats(ctypes.Structure):
    _fields_ = [("slices", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("codes_done", ctypes.c_uint64), ("active", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64),
                ("gpu_seconds", ctypes.c_double), ("plan_seconds", ctypes.c_double),
                ("post_seconds", ctypes.c_double)]


# name -> (restype, argtypes); mirrors include/dist.h
_U8P = ctypes.POINTER(ctypes.c_uint8)
_VP = ctypes.c_void_p
SIGNATURES = {
    "dist_init": (ctypes.c_int, [ctypes.POINTER(_VP), _U8P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "dist_init_many": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_U8P),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "dist_set_exclude": (ctypes.c_int, [_VP, ctypes.c_int]),
    "dist_solve": (ctypes.c_int, [_VP, ctypes.POINTER(DistResult), _VP]),
    "dist_solve_bounded": (ctypes.c_int, [_VP, ctypes.POINTER(DistResult), _VP, ctypes.c_double]),
    "dist_free": (ctypes.c_int, [_VP]),
    "dist_solve_isometry": (ctypes.c_int, [_VP, ctypes.POINTER(DistResult), _VP]),
    "dist_plan_info_get": (ctypes.c_int, [_U8P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.POINTER(PlanInfo)]),
    "dist_plan_unit": (ctypes.c_int, [_U8P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, _U8P, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    "dist_intpeak": (ctypes.c_int, [ctypes.POINTER(IntpeakResult), ctypes.c_int, _VP]),
    "dist_normalizer": (ctypes.c_int, [_U8P, ctypes.c_int, ctypes.c_int, _U8P, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    "dist_init_stabilizer": (ctypes.c_int, [ctypes.POINTER(_VP), _U8P, ctypes.c_int, ctypes.c_int]),
    "dist_solve_noalloc": (ctypes.c_int, [_U8P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(DistResult), _VP]),
    "dist_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(BatchOpts)]),
    "dist_batch_submit": (ctypes.c_int, [_VP, ctypes.POINTER(_VP), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "dist_batch_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(DistResult)]),
    "dist_batch_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(DistResult),
                                       ctypes.c_double]),
    "dist_batch_wait_any": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_uint64)]),
    "dist_batch_stats": (ctypes.c_int, [_VP, ctypes.POINTER(BatchStats)]),
    "dist_batch_destroy": (ctypes.c_int, [_VP]),
    "dist_set_tuning": (ctypes.c_int, [ctypes.POINTER(Tuning)]),
    "dist_get_tuning": (ctypes.c_int, [ctypes.POINTER(Tuning)]),
    "dist_autotune": (ctypes.c_int, [ctypes.POINTER(Tuning), ctypes.c_double]),
    "dist_set_plan_search": (ctypes.c_int, [ctypes.c_int]),
    "dist_get_plan_search": (ctypes.c_int, []),
    "dist_set_gamma_limit": (ctypes.c_int, [ctypes.c_int]),
    "dist_get_gamma_limit": (ctypes.c_int, []),
    "dist_set_event_timing": (ctypes.c_int, [ctypes.c_int]),
    "dist_get_event_timing": (ctypes.c_int, []),
    "dist_set_iso_walk": (ctypes.c_int, [ctypes.c_int]),
    "dist_get_iso_walk": (ctypes.c_int, []),
    "dist_autotune_codes": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_double,
                                           ctypes.POINTER(Tuning)]),
    "dist_version": (ctypes.c_char_p, []),
    "dist_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libdist.so (compiling it first if the sources changed)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libdist.so is missing: the CUDA library did not build")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


class DistError(RuntimeError):
    def __init__(self, code: int, what: str):
        msg = lib().dist_strerror(code).decode()
        super().__init__("%s: %s (%d)" % (what, msg, code))
        self.code = code


def _check(code: int, what: str, ok=(DIST_OK,)) -> int:
    if code not in ok:
        raise DistError(code, what)
    return code


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def _as_gen(generator, field):
    g = np.ascontiguousarray(np.asarray(generator, dtype=np.uint8))
    if g.ndim != 2:
        raise ValueError("generator must be a 2-D array")
    K = g.shape[0]
    n = g.shape[1] // 2 if field == DIST_F2 else g.shape[1]
    return g, n, K


def _ptr(a):
    return a.ctypes.data_as(_U8P)


# --- entry points with the C names --------------------------------------------------

def dist_init(generator, n, K, field):
    h = _VP()
    g = np.ascontiguousarray(np.asarray(generator, dtype=np.uint8))
    _check(lib().dist_init(ctypes.byref(h), _ptr(g), n, K, field), "dist_init")
    return h


def dist_init_many(generators, field=None):
    """dist_init of many codes in one call.  generators: a list of 2-D arrays
    (field: one value or a list, DIST_F2 by default).  Returns (handles,
    statuses): a handle per code (None where its status is an error)."""
    count = len(generators)
    fields = [DIST_F2] * count if field is None else (list(field) if isinstance(field, (list, tuple)) else [field] * count)
    arrs, ns, Ks = [], [], []
    for g, f in zip(generators, fields):
        a, n, K = _as_gen(g, f)
        arrs.append(a)
        ns.append(n)
        Ks.append(K)
    ptrs = (_U8P * max(count, 1))(*[_ptr(a) for a in arrs])
    c_n = (ctypes.c_int * max(count, 1))(*ns)
    c_K = (ctypes.c_int * max(count, 1))(*Ks)
    c_f = (ctypes.c_int * max(count, 1))(*fields)
    c_st = (ctypes.c_int * max(count, 1))()
    hs = (_VP * max(count, 1))()
    rc = lib().dist_init_many(hs, count, ptrs, c_n, c_K, c_f, c_st)
    if rc == DIST_EINVAL and count and all(c_st[i] == 0 for i in range(count)):
        _check(rc, "dist_init_many")
    handles = [_VP(hs[i]) if hs[i] else None for i in range(count)]
    return handles, [int(c_st[i]) for i in range(count)]


def dist_set_exclude(handle, n_stab):
    return _check(lib().dist_set_exclude(handle, n_stab), "dist_set_exclude")


def _as_stab(stabilizers):
    s = np.ascontiguousarray(np.asarray(stabilizers, dtype=np.uint8))
    if s.ndim != 2 or s.shape[1] % 2:
        raise ValueError("stabilizers must be a 2-D array of rows (x | z)")
    return s, s.shape[1] // 2, s.shape[0]


def dist_normalizer(stabilizers):
    """Normalizer matrix of a qubit stabilizer code: (rows, n_stab), the first
    n_stab rows a basis of S (host only)."""
    s, n, m = _as_stab(stabilizers)
    out = np.zeros((2 * n, 2 * n), dtype=np.uint8)
    K, ns = ctypes.c_int(), ctypes.c_int()
    _check(lib().dist_normalizer(_ptr(s), n, m, _ptr(out), ctypes.byref(K), ctypes.byref(ns)),
           "dist_normalizer")
    return out[:K.value].copy(), ns.value


def dist_init_stabilizer(stabilizers):
    s, n, m = _as_stab(stabilizers)
    h = _VP()
    _check(lib().dist_init_stabilizer(ctypes.byref(h), _ptr(s), n, m), "dist_init_stabilizer")
    return h


def dist_solve(handle, stream=None, ok=(DIST_OK,)):
    r = DistResult()
    _check(lib().dist_solve(handle, ctypes.byref(r), _stream_handle(stream)), "dist_solve", ok)
    return r


def dist_solve_bounded(handle, time_limit_s, stream=None):
    r = DistResult()
    _check(lib().dist_solve_bounded(handle, ctypes.byref(r), _stream_handle(stream),
                                    float(time_limit_s)),
           "dist_solve_bounded", ok=(DIST_OK, DIST_EINCOMPLETE))
    return r


def dist_solve_isometry(handle, stream=None):
    r = DistResult()
    _check(lib().dist_solve_isometry(handle, ctypes.byref(r), _stream_handle(stream)), "dist_solve_isometry")
    return r


def dist_free(handle):
    return _check(lib().dist_free(handle), "dist_free")


def dist_plan_info_get(generator, field=DIST_F2, n_stab=0) -> PlanInfo:
    g, n, K = _as_gen(generator, field)
    info = PlanInfo()
    _check(lib().dist_plan_info_get(_ptr(g), n, K, field, n_stab, ctypes.byref(info)),
           "dist_plan_info_get")
    return info


def dist_plan_unit(generator, gamma, unit, rep, field=DIST_F2):
    g, n, K = _as_gen(generator, field)
    out = np.zeros(2 * n, dtype=np.uint8)
    q = ctypes.c_int(0)
    kind = ctypes.c_int(0)
    _check(lib().dist_plan_unit(_ptr(g), n, K, field, gamma, unit, rep, _ptr(out),
                                ctypes.byref(q), ctypes.byref(kind)), "dist_plan_unit")
    return out, q.value, kind.value


def dist_intpeak(iters=4096, stream=None) -> IntpeakResult:
    r = IntpeakResult()
    _check(lib().dist_intpeak(ctypes.byref(r), iters, _stream_handle(stream)), "dist_intpeak")
    return r


def dist_solve_noalloc(generator, field=DIST_F2, n_stab=0, stream=None) -> DistResult:
    """Solve without any device allocation: all device scratch lives in the
    library's fixed static array (see include/dist.h).  Calls share that array,
    so calls whose GPU work overlaps must be serialized by the caller."""
    g, n, K = _as_gen(generator, field)
    r = DistResult()
    _check(lib().dist_solve_noalloc(_ptr(g), n, K, field, n_stab, ctypes.byref(r),
                                    _stream_handle(stream)), "dist_solve_noalloc")
    return r


def dist_batch_create(max_active=0, slice_ms=0.0, max_resident_bytes=0, time_limit_s=0.0):
    h = _VP()
    o = BatchOpts(max_active, 0, float(slice_ms), int(max_resident_bytes), float(time_limit_s))
    _check(lib().dist_batch_create(ctypes.byref(h), ctypes.byref(o)), "dist_batch_create")
    return h


def dist_batch_submit(batch, handles):
    arr = (_VP * len(handles))(*[h.value if isinstance(h, _VP) else h for h in handles])
    t = ctypes.c_uint64(0)
    _check(lib().dist_batch_submit(batch, arr, len(handles), ctypes.byref(t)), "dist_batch_submit")
    return t.value


def dist_batch_poll(batch, ticket, count):
    """Results of a finished ticket, or None while it is running."""
    res = (DistResult * count)()
    rc = lib().dist_batch_poll(batch, ticket, res)
    if rc == DIST_EBUSY:
        return None
    _check(rc, "dist_batch_poll")
    return list(res)


def dist_batch_wait(batch, ticket, count, timeout_s=0.0, as_array=False):
    res = (DistResult * count)()
    _check(lib().dist_batch_wait(batch, ticket, res, float(timeout_s)), "dist_batch_wait")
    return np.frombuffer(res, dtype=RESULT_DTYPE) if as_array else list(res)


def dist_batch_wait_any(batch, timeout_s=0.0):
    """Id of a finished ticket (each reported once), or None on timeout."""
    t = ctypes.c_uint64(0)
    rc = lib().dist_batch_wait_any(batch, float(timeout_s), ctypes.byref(t))
    if rc == DIST_ETIMEOUT:
        return None
    _check(rc, "dist_batch_wait_any")
    return t.value


def dist_batch_stats(batch) -> dict:
    s = BatchStats()
    _check(lib().dist_batch_stats(batch, ctypes.byref(s)), "dist_batch_stats")
    return {f: getattr(s, f) for f, _ in BatchStats._fields_}


def dist_batch_destroy(batch):
    return _check(lib().dist_batch_destroy(batch), "dist_batch_destroy")


def dist_set_tuning(chunks_per_warp=0, lane_cap_log2=0, lane_floor_log2=0):
    t = Tuning(chunks_per_warp, lane_cap_log2, lane_floor_log2, 0.0)
    return _check(lib().dist_set_tuning(ctypes.byref(t)), "dist_set_tuning")


def dist_set_plan_search(trials):
    return _check(lib().dist_set_plan_search(int(trials)), "dist_set_plan_search")


def dist_get_plan_search() -> int:
    return lib().dist_get_plan_search()


def dist_set_gamma_limit(m):
    return _check(lib().dist_set_gamma_limit(int(m)), "dist_set_gamma_limit")


def dist_get_gamma_limit() -> int:
    return lib().dist_get_gamma_limit()


def dist_set_event_timing(on):
    return _check(lib().dist_set_event_timing(1 if on else 0), "dist_set_event_timing")


def dist_get_event_timing() -> int:
    return lib().dist_get_event_timing()


def dist_set_iso_walk(mode):
    """Walk of dist_solve_isometry on rounds r >= 2: 0 automatic, 1 the split
    walk wherever it applies (r <= 8), 2 never the split walk."""
    return _check(lib().dist_set_iso_walk(int(mode)), "dist_set_iso_walk")


def dist_get_iso_walk() -> int:
    return lib().dist_get_iso_walk()


def dist_get_tuning() -> dict:
    t = Tuning()
    _check(lib().dist_get_tuning(ctypes.byref(t)), "dist_get_tuning")
    return {"chunks_per_warp": t.chunks_per_warp, "lane_cap_log2": t.lane_cap_log2,
            "lane_floor_log2": t.lane_floor_log2}


def dist_autotune(budget_s=10.0) -> dict:
    """Times calibration solves over a grid of chunk settings on the current
    device and applies the fastest; returns it with its codewords/s."""
    t = Tuning()
    _check(lib().dist_autotune(ctypes.byref(t), float(budget_s)), "dist_autotune")
    return {"chunks_per_warp": t.chunks_per_warp, "lane_cap_log2": t.lane_cap_log2,
            "lane_floor_log2": t.lane_floor_log2, "codewords_per_s": t.codewords_per_s}


def dist_autotune_codes(codes, budget_s=10.0) -> dict:
    """The autotuner's search timed on the given Code objects."""
    arr = (_VP * len(codes))(*[c._h for c in codes])
    t = Tuning()
    _check(lib().dist_autotune_codes(arr, len(codes), float(budget_s), ctypes.byref(t)),
           "dist_autotune_codes")
    return {"chunks_per_warp": t.chunks_per_warp, "lane_cap_log2": t.lane_cap_log2,
            "lane_floor_log2": t.lane_floor_log2, "codewords_per_s": t.codewords_per_s}


def dist_version() -> str:
    return lib().dist_version().decode()


def dist_strerror(code: int) -> str:
    return lib().dist_strerror(code).decode()


# --- convenience wrapper ---------------------------------------------------------------

def result_dict(r: DistResult, n: int, K: int, field: int) -> dict:
    wlen = 2 * n if field == DIST_F2 else n
    return {"d": r.d, "lower": r.lower, "rounds": r.rounds, "k_eff": r.k_eff,
            "n_gamma": r.n_gamma, "status": r.status, "codewords": int(r.codewords),
            "seconds": r.seconds, "gpu_seconds": r.gpu_seconds, "launches": int(r.launches),
            "witness": np.frombuffer(bytes(r.witness), dtype=np.uint8)[:wlen].copy(),
            "coeffs": np.frombuffer(bytes(r.coeffs), dtype=np.uint8)[:K].copy()}


class Code:
    """One code on the current CUDA device (owns a dist_code)."""

    def __init__(self, generator, field=DIST_F2):
        g, n, K = _as_gen(generator, field)
        self.n, self.K, self.field = n, K, field
        self._h = dist_init(g, n, K, field)

    @classmethod
    def many(cls, generators, field=DIST_F2):
        """Codes for a list of generator matrices, initialised together
        (dist_init_many: planning on the library's host threads, one device
        allocation).  Raises DistError for the first code that fails, after
        releasing the others."""
        handles, statuses = dist_init_many(generators, field)
        bad = [i for i, st in enumerate(statuses) if st != 0]
        if bad:
            for h in handles:
                if h is not None:
                    dist_free(h)
            _check(statuses[bad[0]], "dist_init_many (code %d)" % bad[0])
        codes = []
        for g, h in zip(generators, handles):
            self = cls.__new__(cls)
            _, self.n, self.K = _as_gen(g, field)
            self.field = field
            self._h = h
            codes.append(self)
        return codes

    @classmethod
    def from_stabilizers(cls, stabilizers):
        """The normalizer code of a qubit stabilizer code, with S excluded:
        solve() returns d(Q).  The code's rows are those of dist_normalizer
        (a basis of S first), which is what the returned coefficients index."""
        gen, n_stab = dist_normalizer(stabilizers)
        self = cls.__new__(cls)
        self.n, self.K, self.field = gen.shape[1] // 2, gen.shape[0], DIST_F2
        self.n_stab = n_stab
        self._h = dist_init_stabilizer(stabilizers)
        return self

    def set_exclude(self, n_stab: int):
        dist_set_exclude(self._h, n_stab)

    def solve(self, stream=None, time_limit_s: float = 0.0) -> dict:
        if time_limit_s > 0:
            r = dist_solve_bounded(self._h, time_limit_s, stream)
        else:
            r = dist_solve(self._h, stream)
        return result_dict(r, self.n, self.K, self.field)

    def solve_isometry(self, stream=None) -> dict:
        """The same distance by the isometry method (Algorithm 3) on the GPU."""
        return result_dict(dist_solve_isometry(self._h, stream), self.n, self.K, self.field)

    def close(self):
        if self._h:
            dist_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quantum_distance(stabilizers, stream=None) -> dict:
    """d(Q) of a qubit stabilizer code from its stabilizer generators."""
    with Code.from_stabilizers(stabilizers) as c:
        return c.solve(stream)


def distance(generator, field=DIST_F2, n_stab=0, stream=None) -> dict:
    """Certified symplectic minimum distance of one code (convenience)."""
    with Code(generator, field) as c:
        if n_stab:
            c.set_exclude(n_stab)
        return c.solve(stream)


class Batch:
    """Many codes on one device: batched launches with continuous admission.
    ``submit`` returns a ticket; ``wait``/``poll`` return one result dict per
    code (``seconds`` = latency from submission).  Codes stay owned by the
    batch until their ticket is collected."""

    def __init__(self, max_active=0, slice_ms=0.0, max_resident_bytes=0, time_limit_s=0.0):
        self._h = dist_batch_create(max_active, slice_ms, max_resident_bytes, time_limit_s)
        self._tickets = {}

    def submit(self, codes):
        codes = list(codes)
        t = dist_batch_submit(self._h, [c._h for c in codes])
        self._tickets[t] = codes
        return t

    def _finish(self, t, res):
        codes = self._tickets.pop(t)
        return [result_dict(r, c.n, c.K, c.field) for r, c in zip(res, codes)]

    def poll(self, ticket):
        res = dist_batch_poll(self._h, ticket, len(self._tickets[ticket]))
        return None if res is None else self._finish(ticket, res)

    def wait(self, ticket, timeout_s=0.0):
        return self._finish(ticket, dist_batch_wait(self._h, ticket, len(self._tickets[ticket]),
                                                    timeout_s))

    def wait_array(self, ticket, timeout_s=0.0):
        """As wait, but all results as one numpy structured array (fields of
        dist_result; witness and coeffs as 256-byte rows) without per-code
        Python objects."""
        n = len(self._tickets[ticket])
        res = dist_batch_wait(self._h, ticket, n, timeout_s, as_array=True)
        self._tickets.pop(ticket)
        return res

    def wait_any(self, timeout_s=0.0):
        """Id of a finished ticket (collect it with poll), or None on timeout."""
        return dist_batch_wait_any(self._h, timeout_s)

    def stats(self):
        return dist_batch_stats(self._h)

    def close(self):
        if self._h:
            dist_batch_destroy(self._h)
            self._h = None
            self._tickets.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
