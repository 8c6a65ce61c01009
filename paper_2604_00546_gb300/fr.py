"""Python binding of the C ABI in include/fr.h (argument marshalling only).

Every computation runs in libfr.so (CUDA kernels for sm_103a and the host
client code). If the library is missing or fails to load, importing the
binding raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FR_OK = 0
FR_ERR_INVALID_ARG = 1
FR_ERR_HBM_BUDGET = 2
FR_ERR_CUDA = 3
FR_ERR_TIMEOUT = 4
FR_ERR_LEVEL = 5
FR_ERR_FORMAT = 6
FR_ERR_INTERNAL = 7
FR_ERR_UNSUPPORTED = 8

FR_MODE_SCORES, FR_MODE_IDENTIFY, FR_MODE_MEMBERSHIP = 0, 1, 2
(FR_KEYS_ONDEMAND, FR_KEYS_CPU_BSGS, FR_KEYS_HYDIA_DG, FR_KEYS_TBS_ONLINE, FR_KEYS_TBS_TOTAL,
 FR_KEYS_TBE_TOTAL) = range(6)

EXPORTED = [
    "fr_setup", "fr_required_rotations", "fr_rotation_set", "fr_rotation_count", "fr_keygen", "fr_load_keys",
    "fr_load_db", "fr_encrypt_db", "fr_load_db_encrypted", "fr_db_info", "fr_encrypt", "fr_encrypt_slots", "fr_match", "fr_match_batch", "fr_match_multi", "fr_set_db_tier", "fr_decrypt", "fr_ct_export", "fr_ct_import",
    "fr_ct_info", "fr_ct_upload", "fr_rotate", "fr_rotate_hoisted", "fr_rotate_noalloc", "fr_rescale", "fr_mul_relin", "fr_add",
    "fr_chebyshev", "fr_rotate_sum", "fr_membership_reduce", "fr_sync", "fr_profile", "fr_profile_read", "fr_profile_only", "fr_launch_count", "fr_butterfly_peak", "fr_fp64_peak", "fr_ntt_time", "fr_use_graphs", "fr_inject_alloc_failure", "fr_ntt_tuning", "fr_ntt_set_shapes",
    "fr_ctx_primes", "fr_ctx_info", "fr_work_level", "fr_cheb_coeffs", "fr_cheb_coeffs_lo", "fr_free_ct", "fr_free_cts", "fr_free_keys", "fr_free_db",
    "fr_free", "fr_last_error", "fr_serve_start", "fr_serve_stop", "fr_match_submit", "fr_match_poll",
    "fr_serve_stats", "fr_serve_plan",
]


class ServeParams(C.Structure):
    _fields_ = [("max_batch", C.c_uint32), ("slots", C.c_uint32), ("hbm_budget_bytes", C.c_uint64)]


class FrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"fr status {status}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [
        ("log_n", C.c_uint32), ("n_q", C.c_uint32), ("q_bits", C.POINTER(C.c_uint32)), ("n_p", C.c_uint32),
        ("p_bits", C.POINTER(C.c_uint32)), ("dnum", C.c_uint32), ("scale_bits", C.c_uint32), ("ell", C.c_uint32),
        ("n1", C.c_uint32), ("schedule", C.c_uint32), ("cheb_degree", C.c_uint32), ("threshold", C.c_double),
        ("hbm_budget_bytes", C.c_uint64), ("device", C.c_int), ("cuda_stream", C.c_void_p),
        ("db_tier", C.c_uint32), ("level_mode", C.c_uint32), ("sum_radix", C.c_uint32),
        ("hoist_giants", C.c_uint32), ("comparator", C.c_uint32), ("hoist_babies", C.c_uint32),
        ("hoist_sum", C.c_uint32),
    ]


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfr.so (building it first if needed); raise if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libfr.so is not built; run paper_2604_00546_gb300.build.build()")
    L = C.CDLL(_build.LIB)
    vp, st = C.c_void_p, C.c_int
    u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
    f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
    f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
    i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
    sig = {
        "fr_setup": (st, [C.POINTER(Params), C.POINTER(vp)]),
        "fr_required_rotations": (st, [vp, C.c_int, i32p, C.c_size_t, C.POINTER(C.c_size_t)]),
        "fr_rotation_set": (st, [C.c_uint32, C.c_uint32, C.c_uint32, C.c_int, C.c_int, i32p, C.c_size_t,
                                 C.POINTER(C.c_size_t)]),
        "fr_rotation_count": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32]),
        "fr_keygen": (st, [vp, i32p, C.c_size_t, C.c_uint64, C.POINTER(vp)]),
        "fr_load_keys": (st, [vp, vp]),
        "fr_load_db": (st, [vp, f32p, C.c_size_t, C.c_size_t, C.POINTER(vp)]),
        "fr_encrypt_db": (st, [vp, vp, f32p, C.c_size_t, C.c_size_t, C.c_int, C.c_uint32, C.c_uint64, u64p,
                               C.c_size_t]),
        "fr_load_db_encrypted": (st, [vp, u64p, C.c_size_t, C.c_size_t, C.c_uint32, C.c_int, C.POINTER(vp)]),
        "fr_db_info": (st, [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]),
        "fr_encrypt": (st, [vp, vp, f64p, C.c_size_t, C.c_uint64, C.POINTER(vp)]),
        "fr_encrypt_slots": (st, [vp, vp, f64p, C.c_size_t, C.c_uint64, C.POINTER(vp)]),
        "fr_match": (st, [vp, vp, vp, C.c_int, C.POINTER(C.POINTER(vp)), C.POINTER(C.c_size_t)]),
        "fr_match_batch": (st, [vp, vp, C.POINTER(vp), C.c_size_t, C.c_int, C.POINTER(C.POINTER(vp)),
                                C.POINTER(C.c_size_t)]),
        "fr_set_db_tier": (st, [vp, C.c_uint32]),
        "fr_match_multi": (st, [vp, C.POINTER(vp), C.POINTER(vp), C.c_size_t, C.c_int, C.POINTER(C.POINTER(vp)),
                                C.POINTER(C.c_size_t)]),
        "fr_decrypt": (st, [vp, vp, vp, f64p, C.c_size_t]),
        "fr_ct_export": (st, [vp, u64p, C.c_size_t, C.POINTER(C.c_uint32), C.POINTER(C.c_double)]),
        "fr_ct_import": (st, [vp, u64p, C.c_uint32, C.c_double, C.POINTER(vp)]),
        "fr_ct_info": (st, [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_int)]),
        "fr_ct_upload": (st, [vp, vp]),
        "fr_rotate": (st, [vp, vp, C.c_int32, C.POINTER(vp)]),
        "fr_rotate_hoisted": (st, [vp, vp, i32p, C.c_size_t, C.POINTER(vp)]),
        "fr_rotate_noalloc": (st, [vp, C.c_void_p, C.c_uint32, C.c_int32, C.c_void_p]),
        "fr_rescale": (st, [vp, vp, C.POINTER(vp)]),
        "fr_mul_relin": (st, [vp, vp, vp, C.POINTER(vp)]),
        "fr_add": (st, [vp, vp, vp, C.POINTER(vp)]),
        "fr_chebyshev": (st, [vp, vp, C.POINTER(vp)]),
        "fr_rotate_sum": (st, [vp, vp, C.POINTER(vp)]),
        "fr_membership_reduce": (st, [vp, C.POINTER(vp), C.c_size_t, C.POINTER(vp)]),
        "fr_sync": (st, [vp]),
        "fr_profile": (st, [vp, C.c_int]),
        "fr_profile_only": (st, [vp, C.c_char_p]),
        "fr_profile_read": (st, [vp, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_uint64),
                                 C.POINTER(C.c_uint64)]),
        "fr_launch_count": (C.c_uint64, [vp]),
        "fr_butterfly_peak": (st, [C.c_int, C.POINTER(C.c_double)]),
        "fr_ntt_time": (st, [vp, C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "fr_fp64_peak": (st, [C.c_int, C.POINTER(C.c_double)]),
        "fr_use_graphs": (st, [vp, C.c_int]),
        "fr_inject_alloc_failure": (st, [vp, C.c_int64]),
        "fr_ntt_tuning": (st, [vp, np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS"), f64p]),
        "fr_ntt_set_shapes": (st, [vp, np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")]),
        "fr_ctx_primes": (st, [vp, u64p, C.c_size_t, C.POINTER(C.c_size_t)]),
        "fr_ctx_info": (st, [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                             C.POINTER(C.c_uint64)]),
        "fr_cheb_coeffs": (st, [C.c_uint32, C.c_double, f64p]),
        "fr_cheb_coeffs_lo": (st, [C.c_uint32, C.c_double, C.c_double, f64p]),
        "fr_work_level": (C.c_uint32, [vp]),
        "fr_free_ct": (None, [vp]),
        "fr_free_cts": (None, [C.POINTER(vp), C.c_size_t]),
        "fr_free_keys": (None, [vp]),
        "fr_free_db": (None, [vp]),
        "fr_free": (None, [vp]),
        "fr_last_error": (C.c_char_p, []),
        "fr_serve_start": (st, [vp, C.POINTER(ServeParams)]),
        "fr_serve_stop": (st, [vp]),
        "fr_match_submit": (st, [vp, vp, vp, C.c_int, C.POINTER(C.c_uint64)]),
        "fr_match_poll": (st, [vp, C.c_uint64, C.c_int, C.POINTER(C.POINTER(vp)), C.POINTER(C.c_size_t),
                               C.POINTER(C.c_double)]),
        "fr_serve_stats": (st, [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                                C.POINTER(C.c_uint64)]),
        "fr_serve_plan": (st, [np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS"), C.c_size_t, C.c_uint32,
                               C.c_uint64, C.c_uint64, C.c_uint64,
                               np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS"), C.POINTER(C.c_size_t)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status):
    if status != FR_OK:
        raise FrError(status, (_lib.fr_last_error() or b"").decode())


# ---------------------------------------------------------------------------
# object layer
# ---------------------------------------------------------------------------
class _Handle:
    """A library object owned by a context. The context is freed only after every object it owns
    (a finaliser order Python does not guarantee for objects collected in one reference cycle)."""

    def _register(self, ctx, h):
        self.ctx = ctx
        self.h = h
        self._live = True
        ctx._live += 1

    def _release(self, free_fn):
        if not getattr(self, "_live", False):
            return
        self._live = False
        try:
            if self.h is not None and self.h.value and _lib is not None and self.ctx.h is not None:
                free_fn(self.h)
        finally:
            self.h = None
            self.ctx._dep_freed()


class Ciphertext(_Handle):
    """Library-owned ciphertext handle."""

    def __init__(self, ctx, handle):
        self._register(ctx, C.c_void_p(handle) if not isinstance(handle, C.c_void_p) else handle)

    def __del__(self):
        try:
            self._release(_lib.fr_free_ct)
        except Exception:
            pass

    def info(self):
        lvl, dev = C.c_uint32(), C.c_int()
        _check(_lib.fr_ct_info(self.h, C.byref(lvl), C.byref(dev)))
        return lvl.value, bool(dev.value)

    @property
    def level(self):
        return self.info()[0]

    def export(self):
        lvl = self.level
        buf = np.empty((2, lvl + 1, self.ctx.N), dtype=np.uint64)
        out_l, sc = C.c_uint32(), C.c_double()
        _check(_lib.fr_ct_export(self.h, buf, buf.size, C.byref(out_l), C.byref(sc)))
        return buf

    def upload(self):
        _check(_lib.fr_ct_upload(self.ctx.h, self.h))
        return self


class Context:
    """fr_ctx: parameters, primes, device tables."""

    def __init__(self, log_n, q_bits, p_bits, dnum, scale_bits, ell, n1, cheb_degree=0, threshold=0.5,
                 hbm_budget_bytes=0, device=0, cuda_stream=None, schedule=0, level_mode=0, db_tier=0, sum_radix=0,
                 hoist_giants=0, comparator=0, hoist_babies=0, hoist_sum=0):
        L = load()
        self._qb = (C.c_uint32 * len(q_bits))(*q_bits)
        self._pb = (C.c_uint32 * len(p_bits))(*p_bits)
        self.params = Params(log_n, len(q_bits), self._qb, len(p_bits), self._pb, dnum, scale_bits, ell, n1,
                             schedule, cheb_degree, threshold, hbm_budget_bytes, device,
                             C.c_void_p(cuda_stream) if cuda_stream else None, db_tier, level_mode, sum_radix,
                             int(hoist_giants), int(comparator), int(hoist_babies), int(hoist_sum))
        h = C.c_void_p()
        self._live = 0          # library objects of this context still alive
        self._closing = False
        _check(L.fr_setup(C.byref(self.params), C.byref(h)))
        self.h = h
        self.N = 1 << log_n
        self.n = self.N // 2
        self.ell = ell
        self.n1 = n1
        self.nq = len(q_bits)
        self.top = self.nq - 1
        self.work_level = int(L.fr_work_level(self.h))

    def close(self):
        """Free the context once every object it owns is freed (now, if none is left)."""
        self._closing = True
        if getattr(self, "_live", 0) == 0:
            self._free_now()

    def _dep_freed(self):
        self._live -= 1
        if self._closing and self._live == 0:
            self._free_now()

    def _free_now(self):
        if getattr(self, "h", None) is not None and self.h.value:
            _lib.fr_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def primes(self):
        out = np.zeros(64, dtype=np.uint64)
        n = C.c_size_t()
        _check(_lib.fr_ctx_primes(self.h, out, 64, C.byref(n)))
        return [int(x) for x in out[: n.value]]

    def info(self):
        a, b, d, r = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_uint64()
        _check(_lib.fr_ctx_info(self.h, C.byref(a), C.byref(b), C.byref(d), C.byref(r)))
        return dict(n_slots=a.value, top_level=b.value, n_digits=d.value, resident_bytes=r.value)

    def required_rotations(self, mode):
        out = np.zeros(4096, dtype=np.int32)
        n = C.c_size_t()
        _check(_lib.fr_required_rotations(self.h, int(mode), out, out.size, C.byref(n)))
        return [int(x) for x in out[: n.value]]

    def keygen(self, rotations, seed):
        r = np.ascontiguousarray(rotations, dtype=np.int32)
        h = C.c_void_p()
        _check(_lib.fr_keygen(self.h, r, len(r), int(seed), C.byref(h)))
        return Keys(self, h)

    def load_keys(self, keys):
        _check(_lib.fr_load_keys(self.h, keys.h))

    def load_db(self, templates, tier=None):
        """Upload a template database; tier (0 auto, 1, 2, 3) sets the storage tier for this
        and later loads."""
        if tier is not None:
            _check(_lib.fr_set_db_tier(self.h, int(tier)))
        T = np.ascontiguousarray(templates, dtype=np.float32)
        h = C.c_void_p()
        _check(_lib.fr_load_db(self.h, T, T.shape[0], T.shape[1], C.byref(h)))
        return Database(self, h, T.shape[0])

    def encrypt_db(self, keys, templates, level=None, seed=0, prerotate=True):
        """Enroller side: the G*ell encrypted diagonals of the templates, [G][ell][2][level+1][N]
        (export format), at `level` (default: the working level); pre-rotated by the enroller
        (prerotate) or plain, for the server to pre-rotate at load."""
        T = np.ascontiguousarray(templates, dtype=np.float32)
        K, ell = T.shape
        level = self.work_level if level is None else int(level)
        G = -(-K // self.n)
        out = np.empty((G, ell, 2, level + 1, self.N), dtype=np.uint64)
        _check(_lib.fr_encrypt_db(self.h, keys.h, T, K, ell, 1 if prerotate else 0, level, int(seed), out, out.size))
        return out

    def load_db_encrypted(self, cts, K, prerotated=True):
        """Server side: a database (storage tier 4) of the encrypted diagonals from encrypt_db."""
        E = np.ascontiguousarray(cts, dtype=np.uint64)
        h = C.c_void_p()
        _check(_lib.fr_load_db_encrypted(self.h, E, int(K), E.shape[1], E.shape[3] - 1, 1 if prerotated else 0,
                                         C.byref(h)))
        return Database(self, h, int(K))

    def encrypt(self, keys, q, seed):
        q = np.ascontiguousarray(q, dtype=np.float64)
        h = C.c_void_p()
        _check(_lib.fr_encrypt(self.h, keys.h, q, q.size, int(seed), C.byref(h)))
        return Ciphertext(self, h)

    def encrypt_slots(self, keys, z, seed):
        z = np.ascontiguousarray(z, dtype=np.float64)
        h = C.c_void_p()
        _check(_lib.fr_encrypt_slots(self.h, keys.h, z, z.size, int(seed), C.byref(h)))
        return Ciphertext(self, h)

    def import_ct(self, words, level, scale=None):
        w = np.ascontiguousarray(words, dtype=np.uint64).reshape(-1)
        h = C.c_void_p()
        sc = float(scale) if scale is not None else float(2.0 ** self.params.scale_bits)
        _check(_lib.fr_ct_import(self.h, w, int(level), sc, C.byref(h)))
        return Ciphertext(self, h)

    def decrypt(self, keys, ct, n=None):
        n = self.n if n is None else n
        out = np.empty(n, dtype=np.float64)
        _check(_lib.fr_decrypt(self.h, keys.h, ct.h, out, n))
        return out

    def match(self, db, query, mode):
        arr = C.POINTER(C.c_void_p)()
        n = C.c_size_t()
        _check(_lib.fr_match(self.h, db.h, query.h, int(mode), C.byref(arr), C.byref(n)))
        cts = [Ciphertext(self, C.c_void_p(arr[i])) for i in range(n.value)]
        # release only the array (the handles are owned by the Ciphertext objects)
        _lib.fr_free_cts(arr, 0)
        return cts

    def match_batch(self, db, queries, mode):
        """One pass over several queries; returns one list of output ciphertexts per query."""
        arr = C.POINTER(C.c_void_p)()
        n = C.c_size_t()
        hs = (C.c_void_p * len(queries))(*[q.h.value for q in queries])
        _check(_lib.fr_match_batch(self.h, db.h, hs, len(queries), int(mode), C.byref(arr), C.byref(n)))
        cts = [Ciphertext(self, C.c_void_p(arr[i])) for i in range(n.value)]
        _lib.fr_free_cts(arr, 0)
        per = n.value // len(queries)
        return [cts[i * per:(i + 1) * per] for i in range(len(queries))]

    def ntt_tuning(self):
        """Tile shape chosen per NTT batch bucket and the tuner's times (us, bucket x shape)."""
        shapes = np.zeros(4, dtype=np.uint32)
        us = np.zeros(24, dtype=np.float64)
        _check(_lib.fr_ntt_tuning(self.h, shapes, us))
        return dict(buckets=["<=4", "<=16", "<=64", ">64"], shapes=[int(x) for x in shapes],
                    us=us.reshape(4, 6).round(2).tolist())

    def ntt_time(self, npolys, level=None, reps=5):
        """(forward us, inverse us) of one batched NTT of npolys limb-polynomials."""
        f, i = C.c_double(), C.c_double()
        lvl = self.work_level if level is None else int(level)
        _check(_lib.fr_ntt_time(self.h, int(npolys), lvl, int(reps), C.byref(f), C.byref(i)))
        return f.value, i.value

    def ntt_set_shapes(self, shapes):
        _check(_lib.fr_ntt_set_shapes(self.h, np.ascontiguousarray(shapes, dtype=np.uint32)))

    def inject_alloc_failure(self, after):
        """Make the after-th device allocation from now fail (FR_ERR_HBM_BUDGET); -1: off."""
        _check(_lib.fr_inject_alloc_failure(self.h, int(after)))

    def use_graphs(self, on=True):
        """Replay matches as CUDA graphs (default) or launch every kernel per call."""
        _check(_lib.fr_use_graphs(self.h, 1 if on else 0))

    # -- serving loop (continuous batching) ------------------------------------------
    def serve_start(self, max_batch=8, slots=2, hbm_budget_bytes=0):
        p = ServeParams(int(max_batch), int(slots), int(hbm_budget_bytes))
        _check(_lib.fr_serve_start(self.h, C.byref(p)))

    def serve_stop(self):
        _check(_lib.fr_serve_stop(self.h))

    def submit(self, db, query, mode):
        """Queue a match request; returns its ticket."""
        t = C.c_uint64()
        _check(_lib.fr_match_submit(self.h, db.h, query.h, int(mode), C.byref(t)))
        return t.value

    def poll(self, ticket, block_ms=-1, with_latency=False):
        """Outputs of a ticket (list of ciphertexts), or None when not finished within block_ms;
        with_latency: (outputs, submit-to-device-completion milliseconds)."""
        arr = C.POINTER(C.c_void_p)()
        n = C.c_size_t()
        lat = C.c_double()
        st = _lib.fr_match_poll(self.h, C.c_uint64(ticket), int(block_ms), C.byref(arr), C.byref(n), C.byref(lat))
        if st == FR_ERR_TIMEOUT:
            return None
        _check(st)
        cts = [Ciphertext(self, C.c_void_p(arr[i])) for i in range(n.value)]
        _lib.fr_free_cts(arr, 0)
        return (cts, lat.value) if with_latency else cts

    def serve_stats(self):
        a, b, p, m = C.c_uint64(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(_lib.fr_serve_stats(self.h, C.byref(a), C.byref(b), C.byref(p), C.byref(m)))
        return dict(completed=a.value, batches=b.value, outstanding=p.value, max_concurrent_batches=m.value)

    def match_multi(self, dbs, queries, mode):
        """Query b against database dbs[b], all in one pass; one list of outputs per query."""
        arr = C.POINTER(C.c_void_p)()
        n = C.c_size_t()
        hq = (C.c_void_p * len(queries))(*[q.h.value for q in queries])
        hd = (C.c_void_p * len(dbs))(*[d.h.value for d in dbs])
        _check(_lib.fr_match_multi(self.h, hd, hq, len(queries), int(mode), C.byref(arr), C.byref(n)))
        cts = [Ciphertext(self, C.c_void_p(arr[i])) for i in range(n.value)]
        _lib.fr_free_cts(arr, 0)
        out, i = [], 0
        for d in dbs:
            k = 1 if int(mode) == FR_MODE_MEMBERSHIP else d.info()["groups"]
            out.append(cts[i:i + k])
            i += k
        return out

    def _unary(self, fn, ct):
        h = C.c_void_p()
        _check(fn(self.h, ct.h, C.byref(h)))
        return Ciphertext(self, h)

    def rotate(self, ct, k):
        h = C.c_void_p()
        _check(_lib.fr_rotate(self.h, ct.h, int(k), C.byref(h)))
        return Ciphertext(self, h)

    def rotate_hoisted(self, ct, ks):
        ks = np.ascontiguousarray(ks, dtype=np.int32)
        hs = (C.c_void_p * len(ks))()
        _check(_lib.fr_rotate_hoisted(self.h, ct.h, ks, len(ks), C.cast(hs, C.POINTER(C.c_void_p))))
        return [Ciphertext(self, C.c_void_p(hs[i])) for i in range(len(ks))]

    def rotate_noalloc(self, d_in, level, k, d_out):
        """Rotation without allocation on caller-owned device buffers (raw addresses)."""
        _check(_lib.fr_rotate_noalloc(self.h, C.c_void_p(d_in), int(level), int(k), C.c_void_p(d_out)))

    def rescale(self, ct):
        return self._unary(_lib.fr_rescale, ct)

    def chebyshev(self, ct):
        return self._unary(_lib.fr_chebyshev, ct)

    def rotate_sum(self, ct):
        return self._unary(_lib.fr_rotate_sum, ct)

    def membership_reduce(self, parts):
        """Mod-q sum of threshold ciphertexts (one level), then RotateAndSum: the membership
        result of the groups the parts came from."""
        hs = (C.c_void_p * len(parts))(*[p.h.value for p in parts])
        h = C.c_void_p()
        _check(_lib.fr_membership_reduce(self.h, hs, len(parts), C.byref(h)))
        return Ciphertext(self, h)

    def mul_relin(self, a, b):
        h = C.c_void_p()
        _check(_lib.fr_mul_relin(self.h, a.h, b.h, C.byref(h)))
        return Ciphertext(self, h)

    def add(self, a, b):
        h = C.c_void_p()
        _check(_lib.fr_add(self.h, a.h, b.h, C.byref(h)))
        return Ciphertext(self, h)

    def sync(self):
        _check(_lib.fr_sync(self.h))

    def profile(self, enable):
        _check(_lib.fr_profile(self.h, 1 if enable else 0))

    def profile_only(self, prefix=""):
        _check(_lib.fr_profile_only(self.h, (prefix or "").encode()))

    def profile_read(self, region):
        ms, n, b = C.c_double(), C.c_uint64(), C.c_uint64()
        _check(_lib.fr_profile_read(self.h, region.encode(), C.byref(ms), C.byref(n), C.byref(b)))
        return ms.value, n.value, b.value

    def launch_count(self):
        return int(_lib.fr_launch_count(self.h))


class Keys(_Handle):
    def __init__(self, ctx, h):
        self._register(ctx, h)

    def __del__(self):
        try:
            self._release(_lib.fr_free_keys)
        except Exception:
            pass


class Database(_Handle):
    def __init__(self, ctx, h, K):
        self._register(ctx, h)
        self.K = K

    def info(self):
        t, g, b, sc = C.c_uint32(), C.c_uint64(), C.c_uint64(), C.c_uint32()
        _check(_lib.fr_db_info(self.h, C.byref(t), C.byref(g), C.byref(b), C.byref(sc)))
        return dict(tier=t.value, groups=g.value, bytes=b.value, schedule=sc.value)

    def __del__(self):
        try:
            self._release(_lib.fr_free_db)
        except Exception:
            pass


# ---------------------------------------------------------------------------
# host-only functions
# ---------------------------------------------------------------------------
def rotation_set(ell, n1, slots, which, membership=False):
    L = load()
    out = np.zeros(1 << 16, dtype=np.int32)
    n = C.c_size_t()
    _check(L.fr_rotation_set(int(ell), int(n1), int(slots), int(which), 1 if membership else 0, out, out.size,
                             C.byref(n)))
    return [int(x) for x in out[: n.value]]


def serve_plan(classes, max_batch, avail_bytes, ws_base, ws_per_query):
    """The serving loop's batch planner (host only): indices of the next batch."""
    cls = np.ascontiguousarray(classes, dtype=np.uint32)
    out = np.zeros(max(1, int(max_batch)), dtype=np.uint32)
    n = C.c_size_t()
    _check(load().fr_serve_plan(cls, len(cls), int(max_batch), int(avail_bytes), int(ws_base), int(ws_per_query),
                                out, C.byref(n)))
    return [int(x) for x in out[: n.value]]


def butterfly_peak(device=0):
    v = C.c_double()
    _check(load().fr_butterfly_peak(int(device), C.byref(v)))
    return v.value


def fp64_peak(device=0):
    """Measured FP64 operations per second (register-only fused multiply-adds)."""
    L = load()
    v = C.c_double()
    _check(L.fr_fp64_peak(int(device), C.byref(v)))
    return v.value


def rotation_count(ell, n1, groups, schedule=0):
    return int(load().fr_rotation_count(int(ell), int(n1), int(groups), int(schedule)))


def cheb_coeffs(n, tau, low=0.0):
    """Interpolant at the n + 1 Chebyshev nodes of 1 for x >= tau, `low` below (-1: sign)."""
    out = np.empty(n + 1, dtype=np.float64)
    _check(load().fr_cheb_coeffs_lo(int(n), float(tau), float(low), out))
    return out
