"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds input generation only (no homomorphic arithmetic); the
oracle tests and the CUDA path both draw their inputs from here. Templates
are L2-normalised Gaussian embeddings of dimension ell (ArcFace-like, the
paper's ell = 512); the query and its planted near-duplicates follow the
configurations below.
"""
from __future__ import annotations

import numpy as np

# CKKS parameter sets
CONFIGS = {
    # tiny: N=2^12, Q = 60/40/40, P = 3 x 60, dnum 1, Delta 2^40, K=64, ell=64, n1=8, scores only
    "tiny": dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60, 60, 60], dnum=1, scale_bits=40, ell=64, n1=8,
                 cheb_degree=0, threshold=0.5, K=64, mode=0, seed=1),
    # mid-size parity case: several NTT tiles, two template groups with a ragged tail, full threshold
    "mid": dict(log_n=13, q_bits=[60] + [45] * 8, p_bits=[60, 60, 60], dnum=3, scale_bits=45, ell=64, n1=8,
                cheb_degree=59, threshold=0.5, K=5000, mode=2, seed=6),
    # deeper chain than the threshold needs: the match runs at a lower working level
    "deep": dict(log_n=13, q_bits=[60] + [45] * 11, p_bits=[60, 60, 60], dnum=4, scale_bits=45, ell=64, n1=8,
                 cheb_degree=59, threshold=0.5, K=5000, mode=2, seed=7, level_mode=1),
    # mid-size case deep enough for the hybrid comparator (degree 59 + f_4: 10 levels, working level 12)
    "mid_hybrid": dict(log_n=13, q_bits=[60] + [45] * 13, p_bits=[60, 60, 60], dnum=4, scale_bits=45, ell=64, n1=8,
                       cheb_degree=59, threshold=0.5, K=5000, mode=2, seed=8, level_mode=1, duplicates=6),
    # membership at the headline size: N=2^16, Q = 60 + 24 x 50, P = 4 x 60, dnum 6, Delta 2^50,
    # K = 2^15 templates of ell = 512, 32 near-duplicates at cosine 0.8, degree-59 threshold
    "membership": dict(log_n=16, q_bits=[60] + [50] * 24, p_bits=[60] * 4, dnum=6, scale_bits=50, ell=512, n1=32,
                       cheb_degree=59, threshold=0.5, K=1 << 15, mode=2, seed=2, duplicates=32),
    # identification at scale: K = 2^20 (32 groups)
    "identify": dict(log_n=16, q_bits=[60] + [50] * 24, p_bits=[60] * 4, dnum=6, scale_bits=50, ell=512, n1=32,
                     cheb_degree=59, threshold=0.5, K=1 << 20, mode=1, seed=3, duplicates=32),
}

DATASET_SEED = 0xF00D0000
KEY_SEED = 0xC0FFEE00
ENC_SEED = 0xE0C00000


def ctx_params(cfg, level_mode=None):
    c = CONFIGS[cfg] if isinstance(cfg, str) else cfg
    p = {k: c[k] for k in ("log_n", "q_bits", "p_bits", "dnum", "scale_bits", "ell", "n1", "cheb_degree",
                           "threshold")}
    p["level_mode"] = c.get("level_mode", 0) if level_mode is None else level_mode
    return p


def work_level(cfg, level_mode=None, comparator=0):
    """Working level of the match: the top level, or 2 + d2 (capped) in level mode 1, with 4
    levels more for the hybrid comparator (comparator 1)."""
    c = CONFIGS[cfg] if isinstance(cfg, str) else cfg
    lm = c.get("level_mode", 0) if level_mode is None else level_mode
    top = len(c["q_bits"]) - 1
    if lm == 0:
        return top
    d2 = 0
    if c["cheb_degree"]:
        n = c["cheb_degree"]
        best = None
        for d1 in range(1, n + 2):
            b = 1
            while d1 * 2 ** (b - 1) < n:
                b += 1
            if best is None or d1 + b < best[0] or (d1 + b == best[0] and d1 > best[1]):
                best = (d1 + b, d1, b)
        d2 = best[2] + (4 if comparator == 1 else 0)
    return min(top, 2 + d2)


def templates(K, ell, seed):
    """K x ell float32 rows: g ~ N(0, I) in float64, divided by its norm, cast to float32."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((K, ell))
    g /= np.linalg.norm(g, axis=1, keepdims=True)
    return g.astype(np.float32)


def unit(rng, ell):
    v = rng.standard_normal(ell)
    return v / np.linalg.norm(v)


def plant_duplicates(T, q, count, cosine, rng):
    """Overwrite `count` seeded rows with 0.8 q + 0.6 u (u a unit vector orthogonal to q)."""
    K, ell = T.shape
    idx = rng.choice(K, size=min(count, K), replace=False)
    s = np.sqrt(max(0.0, 1.0 - cosine * cosine))
    for i in idx:
        u = rng.standard_normal(ell)
        u -= (u @ q) * q
        u /= np.linalg.norm(u)
        T[i] = (cosine * q + s * u).astype(np.float32)
    return np.sort(idx)


def workload(cfg, K=None):
    """(templates float32 [K, ell], query float64 [ell], planted indices) of a configuration."""
    c = CONFIGS[cfg] if isinstance(cfg, str) else cfg
    K = c["K"] if K is None else K
    ell = c["ell"]
    seed = DATASET_SEED + c["seed"]
    T = templates(K, ell, seed)
    rng = np.random.default_rng(seed + 1)
    if c.get("duplicates"):
        q = unit(rng, ell)
        planted = plant_duplicates(T, q, c["duplicates"], 0.8, rng)
    else:
        q = T[0].astype(np.float64) + 0.1 * rng.standard_normal(ell)
        q /= np.linalg.norm(q)
        planted = np.array([0])
    return T, q, planted


def key_seed(cfg):
    c = CONFIGS[cfg] if isinstance(cfg, str) else cfg
    return KEY_SEED + c["seed"]


def enc_seed(cfg, request=0):
    c = CONFIGS[cfg] if isinstance(cfg, str) else cfg
    return ENC_SEED + c["seed"] + request


# Serving loop: Poisson arrivals against 8 resident databases. The six listed database
# sizes are assigned to the 8 databases cyclically (db d has K = SERVING_SIZES[d mod 6]).
SERVING_SIZES = [1 << 12, 1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18]
SERVING_DBS = 8
SERVING_SEED = 0x5E7E0000


def serving_databases(ell=512):
    """Template sets of the 8 serving databases (seeded Gaussian, L2-normalised, float32)."""
    return [templates(SERVING_SIZES[d % len(SERVING_SIZES)], ell, SERVING_SEED + d) for d in range(SERVING_DBS)]


def serving_requests(duration_s=60.0, rate=20.0, membership_share=0.7, n_queries=16, seed=SERVING_SEED):
    """Request stream: arrival times (Poisson process of `rate` per second over duration_s),
    mode (membership with probability membership_share, else identification), database
    index (uniform over the 8) and query index (uniform over a pool of n_queries)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        mode = 2 if rng.random() < membership_share else 1
        out.append((t, mode, int(rng.integers(SERVING_DBS)), int(rng.integers(n_queries))))
    return out


def serving_queries(n_queries=16, ell=512, seed=SERVING_SEED + 100):
    rng = np.random.default_rng(seed)
    return [unit(rng, ell) for _ in range(n_queries)]


# Batched launches: 64 queries against 64 databases of uneven sizes, K_d = round(2^U(10, 17)).
MULTI_SEED = 0x3A7C0000


def multi_sizes(n=64, seed=MULTI_SEED):
    rng = np.random.default_rng(seed)
    return [int(round(2.0 ** rng.uniform(10, 17))) for _ in range(n)]


def multi_database(d, K, ell=512, seed=MULTI_SEED):
    return templates(K, ell, seed + 1 + d)

