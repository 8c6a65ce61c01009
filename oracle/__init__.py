"""CPU oracle for the encrypted face-matching hot path (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
``--impl reference`` legs may import this package. The product package
(``paper_2604_00546_gb300``) never imports it. This module is argument
marshalling only: every step of the oracle runs in ``ckks_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libckks_oracle.so")
_lock = threading.Lock()
_lib = None

u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
i8p = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    vp = C.c_void_p
    L.or_setup.restype = vp
    L.or_setup.argtypes = [C.c_int, i32p, C.c_int, i32p, C.c_int, C.c_int, C.c_int]
    L.or_free.argtypes = [vp]
    L.or_dstart.restype = C.c_int
    L.or_dstart.argtypes = [vp, C.c_int]
    for f in ("or_n", "or_nq", "or_np", "or_alpha", "or_ndig"):
        getattr(L, f).restype = C.c_int
        getattr(L, f).argtypes = [vp]
    L.or_prime.restype = C.c_uint64
    L.or_prime.argtypes = [vp, C.c_int]
    L.or_psi.restype = C.c_uint64
    L.or_psi.argtypes = [vp, C.c_int]
    L.or_is_prime.restype = C.c_int
    L.or_is_prime.argtypes = [C.c_uint64]
    L.or_gen_primes.restype = C.c_int
    L.or_gen_primes.argtypes = [C.c_int, i32p, C.c_int, u64p]
    L.or_ntt_fwd.argtypes = [vp, C.c_int, u64p]
    L.or_ntt_inv.argtypes = [vp, C.c_int, u64p]
    L.or_automorph_coef.argtypes = [vp, C.c_uint64, C.c_int, u64p, u64p]
    L.or_automorph_eval.argtypes = [vp, C.c_uint64, u64p, u64p]
    L.or_galois.restype = C.c_uint64
    L.or_galois.argtypes = [vp, C.c_long]
    L.or_chacha20_block.argtypes = [u32p, C.c_uint32, u32p, u8p]
    L.or_sample_ternary.argtypes = [C.c_uint64, C.c_uint64, C.c_int, i8p]
    L.or_sample_cbd.argtypes = [C.c_uint64, C.c_uint64, C.c_int, i32p]
    L.or_sample_uniform.argtypes = [C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint64, C.c_int, u64p]
    L.or_encode_coeffs.argtypes = [vp, f64p, C.c_int, i64p]
    L.or_encode.argtypes = [vp, f64p, C.c_int, C.c_int, u64p]
    L.or_decode_coeffs.argtypes = [vp, i64p, C.c_double, f64p]
    L.or_keygen.restype = vp
    L.or_keygen.argtypes = [vp, C.c_uint64]
    L.or_free_keys.argtypes = [vp]
    L.or_secret.argtypes = [vp, C.c_int, i8p]
    L.or_make_evk.argtypes = [vp, vp, C.c_int, C.c_uint64, u64p]
    L.or_encrypt.argtypes = [vp, vp, f64p, C.c_uint64, u64p]
    L.or_decrypt_coeffs.argtypes = [vp, vp, u64p, C.c_int, i64p]
    L.or_decrypt.argtypes = [vp, vp, u64p, C.c_int, C.c_double, f64p]
    L.or_decrypt_values.argtypes = [vp, vp, u64p, C.c_int, f64p]
    L.or_hoisted_rotate.argtypes = [vp, vp, u64p, C.c_int, np.ctypeslib.ndpointer(np.int64), C.c_int, u64p]
    L.or_rotate.argtypes = [vp, vp, u64p, C.c_int, C.c_long, u64p]
    L.or_rescale.argtypes = [vp, u64p, C.c_int, u64p]
    L.or_drop.argtypes = [vp, u64p, C.c_int, C.c_int, u64p]
    L.or_add.argtypes = [vp, u64p, u64p, C.c_int, u64p]
    L.or_mul_relin.argtypes = [vp, vp, u64p, u64p, C.c_int, u64p]
    L.or_cheb_coeffs.argtypes = [C.c_int, C.c_double, f64p]
    L.or_cheb_coeffs_lo.argtypes = [C.c_int, C.c_double, C.c_double, f64p]
    L.or_f4_eval.restype = C.c_int
    L.or_f4_eval.argtypes = [vp, vp, u64p, C.c_int, u64p]
    L.or_comparator_eval.restype = C.c_int
    L.or_comparator_eval.argtypes = [vp, vp, u64p, C.c_int, C.c_int, C.c_double, C.c_int, u64p]
    L.or_ps_split.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.or_cheb_ps_eval_fp64.restype = C.c_double
    L.or_cheb_ps_eval_fp64.argtypes = [f64p, C.c_int, C.c_double]
    L.or_cheb_eval.restype = C.c_int
    L.or_cheb_eval.argtypes = [vp, vp, u64p, C.c_int, C.c_int, C.c_double, u64p]
    L.or_rotate_sum.argtypes = [vp, vp, u64p, C.c_int, C.c_int]
    L.or_diag_slots.argtypes = [f32p, C.c_long, C.c_int, C.c_int, C.c_long, C.c_int, C.c_long, f64p]
    L.or_bsgs_scores.restype = C.c_int
    L.or_bsgs_scores.argtypes = [vp, vp, u64p, C.c_int, f32p, C.c_long, C.c_int, C.c_int, u64p]
    L.or_bsgs_scores_range.restype = C.c_int
    L.or_bsgs_scores_range.argtypes = [vp, vp, u64p, C.c_int, f32p, C.c_long, C.c_int, C.c_int, C.c_int, C.c_int,
                                       u64p]
    L.or_giant_step.restype = C.c_int
    L.or_giant_step.argtypes = [vp, u64p, C.c_int, C.c_int, f32p, C.c_long, C.c_int, C.c_long, C.c_int, u64p]
    L.or_diag_scores.restype = C.c_int
    L.or_diag_scores.argtypes = [vp, vp, u64p, f32p, C.c_long, C.c_int, u64p]
    L.or_match.restype = C.c_int
    L.or_match.argtypes = [vp, vp, u64p, C.c_int, f32p, C.c_long, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                           C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, u64p, C.POINTER(C.c_int)]
    L.or_bsgs_scores_pq.restype = C.c_int
    L.or_bsgs_scores_pq.argtypes = [vp, vp, u64p, C.c_int, f32p, C.c_long, C.c_int, C.c_int, C.c_int, C.c_int, u64p]
    L.or_bsgs_scores_hoisted.restype = C.c_int
    L.or_bsgs_scores_hoisted.argtypes = [vp, vp, u64p, C.c_int, f32p, C.c_long, C.c_int, C.c_int, u64p]
    L.or_table_scores.restype = C.c_int
    L.or_table_scores.argtypes = [vp, vp, u64p, C.c_int, f32p, C.c_long, C.c_int, C.c_int, u64p]
    L.or_encrypt_db.argtypes = [vp, vp, f32p, C.c_long, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, u64p]
    L.or_prerotate_db.argtypes = [vp, vp, u64p, C.c_int, C.c_long, C.c_int, C.c_int, C.c_int, u64p]
    L.or_enc_giant_step.restype = C.c_int
    L.or_enc_giant_step.argtypes = [vp, vp, u64p, C.c_int, C.c_int, u64p, C.c_int, C.c_int, C.c_int, u64p]
    L.or_enc_bsgs_scores.restype = C.c_int
    L.or_enc_bsgs_scores.argtypes = [vp, vp, u64p, C.c_int, u64p, C.c_int, C.c_long, C.c_int, C.c_int, C.c_int,
                                     u64p]
    L.or_match_enc.restype = C.c_int
    L.or_match_enc.argtypes = [vp, vp, u64p, C.c_int, u64p, C.c_int, C.c_long, C.c_int, C.c_int, C.c_int, C.c_int,
                               C.c_double, C.c_int, C.c_int, C.c_int, u64p, C.POINTER(C.c_int)]
    L.or_rotate_sum_radix.restype = C.c_int
    L.or_rotate_sum_radix.argtypes = [vp, vp, u64p, C.c_int, C.c_int, C.c_int]
    L.or_rotate_sum_hoisted.restype = C.c_int
    L.or_rotate_sum_hoisted.argtypes = [vp, vp, u64p, C.c_int, C.c_int, C.c_int]
    L.or_set_threads.argtypes = [C.c_int]
    L.or_get_threads.restype = C.c_int


# ---------------------------------------------------------------------------
# thin object wrappers
# ---------------------------------------------------------------------------
MODE_SCORES, MODE_IDENTIFY, MODE_MEMBERSHIP = 0, 1, 2


class Ctx:
    """Oracle CKKS context: primes, NTT tables, slot order."""

    def __init__(self, log_n, q_bits, p_bits, dnum, scale_bits):
        self.L = lib()
        qb = np.asarray(q_bits, dtype=np.int32)
        pb = np.asarray(p_bits, dtype=np.int32)
        h = self.L.or_setup(int(log_n), qb, len(qb), pb, len(pb), int(dnum), int(scale_bits))
        if not h:
            raise ValueError("oracle setup failed")
        self.h = h
        self.log_n = int(log_n)
        self.N = 1 << self.log_n
        self.n = self.N // 2
        self.nq = len(qb)
        self.np_ = len(pb)
        self.scale_bits = int(scale_bits)
        self.alpha = self.L.or_alpha(h)
        self.ndig = self.L.or_ndig(h)
        self.dstart = [self.L.or_dstart(h, d) for d in range(self.ndig + 1)]
        self.primes = [int(self.L.or_prime(h, i)) for i in range(self.nq + self.np_)]

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.or_free(self.h)
        except Exception:
            pass

    @property
    def top(self):
        return self.nq - 1

    def ct_shape(self, level):
        return (2, level + 1, self.N)

    def psi(self, i):
        return int(self.L.or_psi(self.h, i))

    def ntt_fwd(self, i, a):
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        self.L.or_ntt_fwd(self.h, i, a)
        return a

    def ntt_inv(self, i, a):
        a = np.ascontiguousarray(a, dtype=np.uint64).copy()
        self.L.or_ntt_inv(self.h, i, a)
        return a

    def galois(self, k):
        return int(self.L.or_galois(self.h, int(k)))

    def automorph_coef(self, g, i, a):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(a)
        self.L.or_automorph_coef(self.h, int(g), int(i), a, out)
        return out

    def automorph_eval(self, g, a):
        a = np.ascontiguousarray(a, dtype=np.uint64)
        out = np.empty_like(a)
        self.L.or_automorph_eval(self.h, int(g), a, out)
        return out

    def encode_coeffs(self, z, scale_bits=None):
        z = np.ascontiguousarray(z, dtype=np.float64)
        assert z.shape == (self.n,)
        m = np.empty(self.N, dtype=np.int64)
        self.L.or_encode_coeffs(self.h, z, self.scale_bits if scale_bits is None else scale_bits, m)
        return m

    def encode(self, z, level=None, scale_bits=None):
        level = self.top if level is None else level
        z = np.ascontiguousarray(z, dtype=np.float64)
        out = np.empty((level + 1, self.N), dtype=np.uint64)
        self.L.or_encode(self.h, z, level, self.scale_bits if scale_bits is None else scale_bits, out)
        return out

    def decode_coeffs(self, x, scale):
        x = np.ascontiguousarray(x, dtype=np.int64)
        z = np.empty(self.n, dtype=np.float64)
        self.L.or_decode_coeffs(self.h, x, float(scale), z)
        return z

    def keygen(self, seed):
        return Keys(self, seed)

    def rescale(self, ct, level):
        ct = np.ascontiguousarray(ct, dtype=np.uint64)
        out = np.empty((2, level, self.N), dtype=np.uint64)
        self.L.or_rescale(self.h, ct, level, out)
        return out

    def add(self, a, b, level):
        out = np.empty((2, level + 1, self.N), dtype=np.uint64)
        self.L.or_add(self.h, np.ascontiguousarray(a), np.ascontiguousarray(b), level, out)
        return out

    def drop(self, ct, level, level2):
        tmp = np.ascontiguousarray(ct, dtype=np.uint64).copy()
        self.L.or_drop(self.h, tmp, level, level2, tmp)
        return tmp.reshape(-1)[: 2 * (level2 + 1) * self.N].reshape(2, level2 + 1, self.N).copy()


class Keys:
    """Oracle secret/public keys; key-switching keys are generated on demand from the seed."""

    def __init__(self, ctx: Ctx, seed: int):
        self.ctx = ctx
        self.L = ctx.L
        self.h = self.L.or_keygen(ctx.h, int(seed))
        self.seed = int(seed)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.L.or_free_keys(self.h)
        except Exception:
            pass

    def secret(self):
        s = np.empty(self.ctx.N, dtype=np.int8)
        self.L.or_secret(self.h, self.ctx.N, s)
        return s

    def make_evk(self, relin, g):
        c = self.ctx
        beta = c.ndig
        out = np.empty((beta, 2, c.nq + c.np_, c.N), dtype=np.uint64)
        self.L.or_make_evk(c.h, self.h, int(relin), int(g), out)
        return out

    def encrypt(self, z, seed):
        c = self.ctx
        z = np.ascontiguousarray(z, dtype=np.float64)
        assert z.shape == (c.n,)
        out = np.empty((2, c.nq, c.N), dtype=np.uint64)
        self.L.or_encrypt(c.h, self.h, z, int(seed), out)
        return out

    def decrypt_coeffs(self, ct, level):
        x = np.empty(self.ctx.N, dtype=np.int64)
        self.L.or_decrypt_coeffs(self.ctx.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, x)
        return x

    def decrypt_values(self, ct, level):
        x = np.empty(self.ctx.N, dtype=np.float64)
        self.L.or_decrypt_values(self.ctx.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, x)
        return x

    def decrypt(self, ct, level, scale=None):
        c = self.ctx
        scale = float(2.0 ** c.scale_bits) if scale is None else float(scale)
        z = np.empty(c.n, dtype=np.float64)
        self.L.or_decrypt(c.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, scale, z)
        return z

    def rotate(self, ct, level, k):
        out = np.empty((2, level + 1, self.ctx.N), dtype=np.uint64)
        self.L.or_rotate(self.ctx.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, int(k), out)
        return out

    def hoisted_rotate(self, ct, level, ks):
        ks = np.asarray(ks, dtype=np.int64)
        out = np.empty((len(ks), 2, level + 1, self.ctx.N), dtype=np.uint64)
        self.L.or_hoisted_rotate(self.ctx.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, ks,
                                 len(ks), out)
        return out

    def mul_relin(self, a, b, level):
        out = np.empty((2, level + 1, self.ctx.N), dtype=np.uint64)
        self.L.or_mul_relin(self.ctx.h, self.h, np.ascontiguousarray(a, dtype=np.uint64),
                            np.ascontiguousarray(b, dtype=np.uint64), level, out)
        return out

    def cheb_eval(self, ct, level, n, tau):
        d1, d2 = ps_split(n)
        out = np.empty((2, level - d2 + 1, self.ctx.N), dtype=np.uint64)
        r = self.L.or_cheb_eval(self.ctx.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, int(n),
                                float(tau), out)
        if r < 0:
            raise ValueError("unsupported Chebyshev degree / level")
        return out

    def f4_eval(self, ct, level):
        """(1 + f_4(y)) / 2 of the ct y at `level`, at level - 4 (hybrid comparator's second part)."""
        out = np.empty((2, level - 3, self.ctx.N), dtype=np.uint64)
        if self.L.or_f4_eval(self.ctx.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, out) < 0:
            raise ValueError("level too low")
        return out

    def comparator_eval(self, ct, level, n, tau, comparator):
        """Threshold of the match: comparator 0 = cheb_eval; 1 = hybrid (depth d2 + 4)."""
        d1, d2 = ps_split(n)
        dep = d2 + (4 if comparator == 1 else 0)
        out = np.empty((2, level - dep + 1, self.ctx.N), dtype=np.uint64)
        r = self.L.or_comparator_eval(self.ctx.h, self.h, np.ascontiguousarray(ct, dtype=np.uint64), level, int(n),
                                      float(tau), int(comparator), out)
        if r < 0:
            raise ValueError("unsupported comparator / level")
        return out

    def rotate_sum(self, ct, level, steps, radix=2, hoist=False):
        """RotateAndSum over 2^steps slots, in radix `radix` (2: one rotation per step); hoist: the
        rotations of each step are summed before one ModDown."""
        x = np.ascontiguousarray(ct, dtype=np.uint64).copy()
        if hoist:
            if self.L.or_rotate_sum_hoisted(self.ctx.h, self.h, x, level, int(steps), int(radix)) < 0:
                raise ValueError("radix must be a power of two")
        elif radix == 2:
            self.L.or_rotate_sum(self.ctx.h, self.h, x, level, int(steps))
        elif self.L.or_rotate_sum_radix(self.ctx.h, self.h, x, level, int(steps), int(radix)) < 0:
            raise ValueError("radix must be a power of two")
        return x

    def bsgs_scores_pq(self, qct, T, ell, n1, level=None, hoist=False, pq=True):
        """Scores at level-1 with the baby steps kept in Q_l u P (pq) or not; hoist: giant steps
        sharing one ModDown per group."""
        c = self.ctx
        L = c.top if level is None else int(level)
        T = np.ascontiguousarray(T, dtype=np.float32)
        K = T.shape[0]
        G = (K + c.n - 1) // c.n
        out = np.empty((G, 2, L, c.N), dtype=np.uint64)
        r = self.L.or_bsgs_scores_pq(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), L, T, K, ell, n1,
                                     1 if pq else 0, 1 if hoist else 0, out)
        if r < 0:
            raise ValueError("bad parameters")
        return out

    def bsgs_scores(self, qct, T, ell, n1, level=None, hoist=False):
        """Scores at level-1 of a query ct at `level` (default: the top level); hoist: the giant
        steps of a group share one ModDown."""
        c = self.ctx
        level = c.top if level is None else level
        T = np.ascontiguousarray(T, dtype=np.float32)
        K = T.shape[0]
        G = (K + c.n - 1) // c.n
        out = np.empty((G, 2, level, c.N), dtype=np.uint64)
        fn = self.L.or_bsgs_scores_hoisted if hoist else self.L.or_bsgs_scores
        r = fn(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), level, T, K, ell, n1, out)
        if r < 0:
            raise ValueError("bad BSGS parameters")
        return out

    def table_scores(self, qct, T, ell, n1, level=None):
        """Scores at level-1 by the rotated-query table of Algorithm 1 (BSGS-Diagonal)."""
        c = self.ctx
        level = c.top if level is None else level
        T = np.ascontiguousarray(T, dtype=np.float32)
        K = T.shape[0]
        G = (K + c.n - 1) // c.n
        out = np.empty((G, 2, level, c.N), dtype=np.uint64)
        r = self.L.or_table_scores(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), level, T, K, ell, n1,
                                   out)
        if r < 0:
            raise ValueError("bad BSGS parameters")
        return out

    def bsgs_scores_range(self, qct, T, ell, n1, j0, j1, level=None):
        """Scores restricted to giant steps j0 <= j < j1 (a bounded sample of the BSGS work)."""
        c = self.ctx
        level = c.top if level is None else level
        T = np.ascontiguousarray(T, dtype=np.float32)
        K = T.shape[0]
        G = (K + c.n - 1) // c.n
        out = np.empty((G, 2, level, c.N), dtype=np.uint64)
        r = self.L.or_bsgs_scores_range(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), level, T, K, ell,
                                        n1, int(j0), int(j1), out)
        if r < 0:
            raise ValueError("bad BSGS parameters")
        return out

    def giant_step(self, babies_eval, n1, T, ell, g, j):
        """One giant step (diagonal encodes, MAC, rescale) on evaluation-form babies [n1][2][L+1][N]."""
        c = self.ctx
        T = np.ascontiguousarray(T, dtype=np.float32)
        level = babies_eval.shape[2] - 1
        P = np.empty((2, level, c.N), dtype=np.uint64)
        r = self.L.or_giant_step(c.h, np.ascontiguousarray(babies_eval, dtype=np.uint64), int(level), int(n1), T,
                                 T.shape[0], int(ell), int(g), int(j), P)
        if r < 0:
            raise ValueError("bad giant step")
        return P

    def diag_scores(self, qct, T, ell):
        c = self.ctx
        T = np.ascontiguousarray(T, dtype=np.float32)
        K = T.shape[0]
        G = (K + c.n - 1) // c.n
        out = np.empty((G, 2, c.top, c.N), dtype=np.uint64)
        r = self.L.or_diag_scores(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), T, K, ell, out)
        if r < 0:
            raise ValueError("bad parameters")
        return out

    def match(self, qct, T, ell, n1, mode, cheb_n=59, tau=0.5, level=None, schedule=0, sum_radix=2, hoist=False,
              comparator=0, babies_pq=False, hoist_sum=False):
        """Full match of a top-level query ct, computed at working level `level` (default: top);
        schedule 0: on-demand BSGS with pre-rotated diagonals, 1: rotated-query table;
        comparator 0: the step interpolant (the paper's GPU path), 1: the hybrid comparator;
        babies_pq: the baby steps stay in Q_l u P (one ModDown per giant step); hoist_sum: the
        rotations of each RotateAndSum step share one ModDown."""
        c = self.ctx
        lq = c.top if level is None else int(level)
        T = np.ascontiguousarray(T, dtype=np.float32)
        K = T.shape[0]
        G = (K + c.n - 1) // c.n
        cnt = 1 if mode == MODE_MEMBERSHIP else G
        out = np.zeros(cnt * 2 * c.top * c.N, dtype=np.uint64)   # large enough for any output level
        lvl = C.c_int(0)
        r = self.L.or_match(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), lq, T, K, ell, n1, mode,
                            int(cheb_n), float(tau), int(comparator), int(schedule), int(sum_radix),
                            1 if hoist else 0, 1 if babies_pq else 0, 1 if hoist_sum else 0, out, C.byref(lvl))
        if r < 0:
            raise ValueError("match failed")
        level = lvl.value
        w = 2 * (level + 1) * c.N          # output ciphertexts are packed back to back
        return out[: cnt * w].reshape(cnt, 2, level + 1, c.N).copy(), level

    # -- encrypted database (enroller-side pre-rotation, lazy relinearisation) ------------
    def encrypt_db(self, T, ell, n1, seed, level=None, prerotate=True):
        """The G*ell encrypted diagonals [G][ell][2][level+1][N] (coefficient form), pre-rotated
        by the enroller (prerotate) or plain (for the server's pre-rotation)."""
        c = self.ctx
        level = c.top if level is None else int(level)
        T = np.ascontiguousarray(T, dtype=np.float32)
        K = T.shape[0]
        G = (K + c.n - 1) // c.n
        out = np.empty((G, ell, 2, level + 1, c.N), dtype=np.uint64)
        self.L.or_encrypt_db(c.h, self.h, T, K, ell, n1, 1 if prerotate else 0, int(seed), level, out)
        return out

    def prerotate_db(self, E, n1, level):
        """Server-side pre-rotation of plain encrypted diagonals E, at `level`."""
        c = self.ctx
        E = np.ascontiguousarray(E, dtype=np.uint64)
        G, ell, el = E.shape[0], E.shape[1], E.shape[3] - 1
        out = np.empty((G, ell, 2, level + 1, c.N), dtype=np.uint64)
        self.L.or_prerotate_db(c.h, self.h, E, el, G, ell, n1, int(level), out)
        return out

    def enc_scores(self, qct, E, n1, level=None, hoist=False):
        """Scores at level-1 of a query ct at `level` (default: top) against encrypted diagonals E."""
        c = self.ctx
        level = c.top if level is None else level
        E = np.ascontiguousarray(E, dtype=np.uint64)
        G, ell, el = E.shape[0], E.shape[1], E.shape[3] - 1
        out = np.empty((G, 2, level, c.N), dtype=np.uint64)
        r = self.L.or_enc_bsgs_scores(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), level, E, el, G, ell,
                                      n1, 1 if hoist else 0, out)
        if r < 0:
            raise ValueError("bad arguments")
        return out

    def match_enc(self, qct, E, K, n1, mode, cheb_n=59, tau=0.5, level=None, sum_radix=2, hoist=False,
                  hoist_sum=False):
        """Full match of a top-level query ct against encrypted diagonals E, at working level
        `level` (default: top); returns (outputs, their level)."""
        c = self.ctx
        lq = c.top if level is None else int(level)
        E = np.ascontiguousarray(E, dtype=np.uint64)
        G, ell, el = E.shape[0], E.shape[1], E.shape[3] - 1
        cnt = 1 if mode == MODE_MEMBERSHIP else G
        out = np.zeros(cnt * 2 * c.top * c.N, dtype=np.uint64)
        lvl = C.c_int(0)
        r = self.L.or_match_enc(c.h, self.h, np.ascontiguousarray(qct, dtype=np.uint64), lq, E, el, int(K), ell,
                                n1, mode, int(cheb_n), float(tau), int(sum_radix), 1 if hoist else 0,
                                1 if hoist_sum else 0, out, C.byref(lvl))
        if r < 0:
            raise ValueError("match failed")
        level = lvl.value
        w = 2 * (level + 1) * c.N
        return out[: cnt * w].reshape(cnt, 2, level + 1, c.N).copy(), level


# ---------------------------------------------------------------------------
# free functions
# ---------------------------------------------------------------------------
def gen_primes(log_n, bits):
    b = np.asarray(bits, dtype=np.int32)
    out = np.zeros(len(b), dtype=np.uint64)
    r = lib().or_gen_primes(int(log_n), b, len(b), out)
    if r != 0:
        raise ValueError("prime generation failed")
    return [int(x) for x in out]


def is_prime(n):
    return bool(lib().or_is_prime(int(n)))


def chacha20_block(key_words, counter, nonce_words):
    out = np.zeros(64, dtype=np.uint8)
    lib().or_chacha20_block(np.asarray(key_words, dtype=np.uint32), int(counter),
                            np.asarray(nonce_words, dtype=np.uint32), out)
    return out


def sample_ternary(seed, obj, n):
    out = np.empty(n, dtype=np.int8)
    lib().or_sample_ternary(int(seed), int(obj), int(n), out)
    return out


def sample_cbd(seed, obj, n):
    out = np.empty(n, dtype=np.int32)
    lib().or_sample_cbd(int(seed), int(obj), int(n), out)
    return out


def sample_uniform(seed, obj, limb, q, n):
    out = np.empty(n, dtype=np.uint64)
    lib().or_sample_uniform(int(seed), int(obj), int(limb), int(q), int(n), out)
    return out


def cheb_coeffs(n, tau, low=0.0):
    """Chebyshev interpolant at the n + 1 nodes of f = 1 for x >= tau, `low` below."""
    out = np.empty(n + 1, dtype=np.float64)
    lib().or_cheb_coeffs_lo(int(n), float(tau), float(low), out)
    return out


def ps_split(n):
    d1, d2 = C.c_int(0), C.c_int(0)
    lib().or_ps_split(int(n), C.byref(d1), C.byref(d2))
    return d1.value, d2.value


def cheb_ps_eval_fp64(coeffs_padded, x):
    cf = np.ascontiguousarray(coeffs_padded, dtype=np.float64)
    return float(lib().or_cheb_ps_eval_fp64(cf, len(cf), float(x)))


def diag_slots(T, ell, slots, k, d, shift):
    T = np.ascontiguousarray(T, dtype=np.float32)
    z = np.empty(slots, dtype=np.float64)
    lib().or_diag_slots(T, T.shape[0], int(ell), int(slots), int(k), int(d), int(shift), z)
    return z


def set_threads(t):
    lib().or_set_threads(int(t))


def get_threads():
    return int(lib().or_get_threads())
