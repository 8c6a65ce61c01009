"""GPU parity: every homomorphic primitive and the full match, through the C ABI,
bit-exact against the CPU oracle on the same seeds, plus decrypted-value checks.

Sizes: 'tiny' (N=2^12, 3 limbs, K=64) and 'mid' (N=2^13, 9 limbs, 3 digits,
K=5000 -> two template groups with a ragged tail, degree-59 threshold).
"""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


class Env:
    def __init__(self, cfg, extra_rots=()):
        c = W.CONFIGS[cfg]
        self.cfg = c
        self.ctx = fr.Context(device=0, **W.ctx_params(cfg))
        mode = c["mode"]
        rots = sorted(set(self.ctx.required_rotations(fr.FR_MODE_MEMBERSHIP if mode == 2 else mode)) | set(extra_rots))
        self.keys = self.ctx.keygen(rots, W.key_seed(cfg))
        self.ctx.load_keys(self.keys)
        self.oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
        self.ok = self.oc.keygen(W.key_seed(cfg))
        self.T, self.q, self.planted = W.workload(cfg)
        self.zq = np.tile(self.q, self.oc.n // c["ell"])
        self.qct = self.ctx.encrypt(self.keys, self.q, W.enc_seed(cfg))
        self.oq = self.ok.encrypt(self.zq, W.enc_seed(cfg))
        self.L = self.oc.top


@pytest.fixture(scope="module")
def tiny():
    return Env("tiny", extra_rots=[3, 5, 64, 2047, 100])


@pytest.fixture(scope="module")
def mid():
    return Env("mid", extra_rots=[3])


@pytest.fixture(scope="module")
def deep():
    return Env("deep")


def dev_copy(env, words, level):
    ct = env.ctx.import_ct(words, level)
    ct.upload()
    return ct


def test_encrypt_matches_oracle(tiny):
    assert np.array_equal(tiny.qct.export(), tiny.oq)


def test_upload_export_round_trip(tiny):
    ct = dev_copy(tiny, tiny.oq, tiny.L)
    assert ct.info() == (tiny.L, True)
    assert np.array_equal(ct.export(), tiny.oq)


@pytest.mark.parametrize("env_name", ["tiny", "mid"])
def test_rescale_matches_oracle(env_name, request):
    env = request.getfixturevalue(env_name)
    ct = dev_copy(env, env.oq, env.L)
    r = env.ctx.rescale(ct)
    assert r.level == env.L - 1
    assert np.array_equal(r.export(), env.oc.rescale(env.oq, env.L))


@pytest.mark.parametrize("k", [1, 3, 5, 64, 2047])
def test_rotate_matches_oracle(tiny, k):
    ct = dev_copy(tiny, tiny.oq, tiny.L)
    got = tiny.ctx.rotate(ct, k).export()
    assert np.array_equal(got, tiny.ok.rotate(tiny.oq, tiny.L, k))


def test_rotate_lower_level_matches_oracle(tiny):
    low = tiny.oc.rescale(tiny.oq, tiny.L)
    ct = dev_copy(tiny, low, tiny.L - 1)
    assert np.array_equal(tiny.ctx.rotate(ct, 100).export(), tiny.ok.rotate(low, tiny.L - 1, 100))


def test_rotate_mid_matches_oracle(mid):
    ct = dev_copy(mid, mid.oq, mid.L)
    assert np.array_equal(mid.ctx.rotate(ct, 3).export(), mid.ok.rotate(mid.oq, mid.L, 3))


def test_hoisted_rotations_match_oracle(tiny):
    ks = [1, 2, 3, 7]
    ct = dev_copy(tiny, tiny.oq, tiny.L)
    outs = tiny.ctx.rotate_hoisted(ct, ks)
    ref = tiny.ok.hoisted_rotate(tiny.oq, tiny.L, ks)
    for i in range(len(ks)):
        assert np.array_equal(outs[i].export(), ref[i]), ks[i]


@pytest.mark.parametrize("env_name", ["tiny", "mid"])
def test_mul_relin_matches_oracle(env_name, request):
    env = request.getfixturevalue(env_name)
    rng = np.random.default_rng(3)
    z2 = rng.uniform(-1, 1, env.oc.n)
    o2 = env.ok.encrypt(z2, 77)
    a = dev_copy(env, env.oq, env.L)
    b = dev_copy(env, o2, env.L)
    got = env.ctx.mul_relin(a, b).export()
    assert np.array_equal(got, env.ok.mul_relin(env.oq, o2, env.L))


def test_add_matches_oracle(tiny):
    a = dev_copy(tiny, tiny.oq, tiny.L)
    assert np.array_equal(tiny.ctx.add(a, a).export(), tiny.oc.add(tiny.oq, tiny.oq, tiny.L))


def test_match_scores_tiny(tiny):
    db = tiny.ctx.load_db(tiny.T)
    out = tiny.ctx.match(db, tiny.qct, fr.FR_MODE_SCORES)
    assert len(out) == 1
    ref = tiny.ok.bsgs_scores(tiny.oq, tiny.T, tiny.cfg["ell"], tiny.cfg["n1"])
    assert np.array_equal(out[0].export(), ref[0])
    dec = tiny.ctx.decrypt(tiny.keys, out[0])
    s = tiny.T.astype(np.float64) @ tiny.q
    assert np.abs(dec[: len(s)] - s).max() < 1e-4
    assert np.abs(dec[len(s):]).max() < 1e-4


def test_match_with_device_resident_query(tiny):
    db = tiny.ctx.load_db(tiny.T)
    q = tiny.ctx.encrypt(tiny.keys, tiny.q, W.enc_seed("tiny"))
    q.upload()
    out = tiny.ctx.match(db, q, fr.FR_MODE_SCORES)
    ref = tiny.ok.bsgs_scores(tiny.oq, tiny.T, tiny.cfg["ell"], tiny.cfg["n1"])
    assert np.array_equal(out[0].export(), ref[0])


def test_chebyshev_matches_oracle(mid):
    # Chebyshev of a fresh encryption of scores-like values at level L-1
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, mid.oc.n)
    o = mid.oc.drop(mid.ok.encrypt(z, 31), mid.L, mid.L - 1)
    ct = dev_copy(mid, o, mid.L - 1)
    got = mid.ctx.chebyshev(ct)
    ref = mid.ok.cheb_eval(o, mid.L - 1, 59, 0.5)
    assert np.array_equal(got.export(), ref)
    p = np.polynomial.chebyshev.chebval(z, oracle.cheb_coeffs(59, 0.5))
    assert np.abs(mid.ctx.decrypt(mid.keys, got) - p).max() < 1e-2


def test_rotate_sum_matches_oracle(mid):
    o = mid.oc.drop(mid.oq, mid.L, 2)
    ct = dev_copy(mid, o, 2)
    got = mid.ctx.rotate_sum(ct).export()
    steps = int(np.log2(mid.oc.n))
    assert np.array_equal(got, mid.ok.rotate_sum(o, 2, steps))


def test_match_scores_mid_two_groups(mid):
    db = mid.ctx.load_db(mid.T)
    out = mid.ctx.match(db, mid.qct, fr.FR_MODE_SCORES)
    assert len(out) == 2
    ref = mid.ok.bsgs_scores(mid.oq, mid.T, mid.cfg["ell"], mid.cfg["n1"])
    for g in range(2):
        assert np.array_equal(out[g].export(), ref[g]), g
    s = mid.T.astype(np.float64) @ mid.q
    dec = np.concatenate([mid.ctx.decrypt(mid.keys, o) for o in out])
    assert np.abs(dec[: len(s)] - s).max() < 1e-4


@pytest.mark.parametrize("mode", [fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_match_threshold_modes_mid(mid, mode):
    db = mid.ctx.load_db(mid.T)
    out = mid.ctx.match(db, mid.qct, mode)
    ref, lvl = mid.ok.match(mid.oq, mid.T, mid.cfg["ell"], mid.cfg["n1"], mode, 59, 0.5)
    assert len(out) == len(ref)
    for g in range(len(out)):
        assert out[g].level == lvl
        assert np.array_equal(out[g].export(), ref[g]), g
    s = mid.T.astype(np.float64) @ mid.q
    n = mid.oc.n
    G = len(s) // n + 1
    sp = np.zeros(G * n)
    sp[: len(s)] = s
    p = np.polynomial.chebyshev.chebval(sp, oracle.cheb_coeffs(59, 0.5))
    if mode == fr.FR_MODE_IDENTIFY:
        dec = np.concatenate([mid.ctx.decrypt(mid.keys, o) for o in out])
        assert np.abs(dec - p).max() < 1e-2
        far = np.abs(s - 0.5) > 0.02
        assert np.array_equal((dec[: len(s)] >= 0.5)[far], (s >= 0.5)[far])
    else:
        dec = mid.ctx.decrypt(mid.keys, out[0])
        assert abs(dec[0] - p.sum()) < 1e-2


@pytest.mark.parametrize("mode", [fr.FR_MODE_SCORES, fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_match_at_working_level_deep(deep, mode):
    """level_mode 1: the top-level query (11) is dropped to level 8 before the BSGS product."""
    assert deep.ctx.work_level == 8 == W.work_level("deep")
    db = deep.ctx.load_db(deep.T)
    out = deep.ctx.match(db, deep.qct, mode)
    ref, lvl = deep.ok.match(deep.oq, deep.T, deep.cfg["ell"], deep.cfg["n1"], mode, 59, 0.5, level=8)
    assert len(out) == len(ref)
    for g in range(len(out)):
        assert out[g].level == lvl
        assert np.array_equal(out[g].export(), ref[g]), g
    s = deep.T.astype(np.float64) @ deep.q
    if mode == fr.FR_MODE_SCORES:
        dec = np.concatenate([deep.ctx.decrypt(deep.keys, o) for o in out])
        assert np.abs(dec[: len(s)] - s).max() < 1e-4
    elif mode == fr.FR_MODE_MEMBERSHIP:
        n = deep.oc.n
        sp = np.zeros(((len(s) + n - 1) // n) * n)
        sp[: len(s)] = s
        p = np.polynomial.chebyshev.chebval(sp, oracle.cheb_coeffs(59, 0.5))
        assert abs(deep.ctx.decrypt(deep.keys, out[0])[0] - p.sum()) < 1e-2


def test_match_graph_replay_bit_exact(mid):
    """fr_match runs eagerly the first time, is captured as a CUDA graph the second
    time and replayed afterwards; every call must equal the oracle."""
    db = mid.ctx.load_db(mid.T)
    rng = np.random.default_rng(21)
    for call in range(4):
        q = rng.standard_normal(mid.cfg["ell"])
        q /= np.linalg.norm(q)
        seed = 1000 + call
        qct = mid.ctx.encrypt(mid.keys, q, seed)
        if call % 2:
            qct.upload()
        out = mid.ctx.match(db, qct, fr.FR_MODE_MEMBERSHIP)
        oq = mid.ok.encrypt(np.tile(q, mid.oc.n // mid.cfg["ell"]), seed)
        ref, lvl = mid.ok.match(oq, mid.T, mid.cfg["ell"], mid.cfg["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5)
        assert np.array_equal(out[0].export(), ref[0]), call


@pytest.mark.parametrize("mode", [fr.FR_MODE_SCORES, fr.FR_MODE_MEMBERSHIP])
def test_per_query_encoding_tier_matches_stored_diagonals(mode):
    """Tier C (2): only the FP32 templates stay in HBM and every query encodes the pre-rotated
    diagonals of each group on the device; tier B (3): their rounded integer coefficients stay
    and every query forms residues and NTTs. Each equals the stored-diagonal tier and the
    oracle, bit for bit (two groups, ragged tail)."""
    c = W.CONFIGS["mid"]
    T, q, _ = W.workload("mid")
    outs = []
    for tier in (1, 2, 3):
        ctx = fr.Context(device=0, db_tier=tier, **W.ctx_params("mid"))
        keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
        ctx.load_keys(keys)
        db = ctx.load_db(T)
        assert db.info()["tier"] == tier and db.info()["groups"] == 2
        qct = ctx.encrypt(keys, q, W.enc_seed("mid"))
        outs.append([o.export() for o in ctx.match(db, qct, mode)])
        outs.append([o.export() for o in ctx.match(db, qct, mode)])   # second call: graph capture
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed("mid"))
    oq = ok.encrypt(np.tile(q, oc.n // c["ell"]), W.enc_seed("mid"))
    ref, _ = ok.match(oq, T, c["ell"], c["n1"], mode, 59, 0.5)
    for o in outs:
        assert len(o) == len(ref)
        for g in range(len(ref)):
            assert np.array_equal(o[g], ref[g])


@pytest.mark.parametrize("mode", [fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_match_batch_equals_oracle_per_query(mid, mode):
    """fr_match_batch: three queries in one pass (shared ModUp groups, key-grouped inner
    products, one MAC pass); each query's outputs equal the oracle's; the second call
    replays the captured graph."""
    db = mid.ctx.load_db(mid.T)
    rng = np.random.default_rng(33)
    qs, refs = [], []
    for b in range(3):
        q = rng.standard_normal(mid.cfg["ell"])
        q /= np.linalg.norm(q)
        qs.append(mid.ctx.encrypt(mid.keys, q, 2000 + b))
        oq = mid.ok.encrypt(np.tile(q, mid.oc.n // mid.cfg["ell"]), 2000 + b)
        refs.append(mid.ok.match(oq, mid.T, mid.cfg["ell"], mid.cfg["n1"], mode, 59, 0.5)[0])
    for call in range(2):
        outs = mid.ctx.match_batch(db, qs, mode)
        assert len(outs) == 3
        for b in range(3):
            assert len(outs[b]) == len(refs[b])
            for g in range(len(refs[b])):
                assert np.array_equal(outs[b][g].export(), refs[b][g]), (call, b, g)
