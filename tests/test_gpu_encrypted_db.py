"""GPU parity of the encrypted-database match (storage tier 4; the paper's setting, with the
diagonals pre-rotated by the enroller, Section 5.3.3, or by the server at load, Section 5.3,
and lazy relinearisation).

The enroller's ciphertexts come from the library's host code and must equal the oracle's bit
for bit. Every match output (scores, identification, membership) must equal the oracle's
encrypted-database match bit for bit, eagerly and replayed as a CUDA graph. Batched and
multi-database calls must give each query's single-call outputs. At the headline size
(N = 2^16, K = 2^15, ell = 512, level 8) the scores must decrypt to the FP64 inner products.
"""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


class Env:
    def __init__(self, cfg, enroll_level=None, server_prerotation=False, hoist=False):
        c = W.CONFIGS[cfg]
        self.c = c
        self.hoist = hoist
        self.ctx = fr.Context(device=0, hoist_giants=1 if hoist else 0, **W.ctx_params(cfg))
        rots = self.ctx.required_rotations(fr.FR_MODE_MEMBERSHIP)
        if server_prerotation:   # the negative giant steps -j n1
            rots = sorted(set(rots) | set(fr.rotation_set(c["ell"], c["n1"], self.ctx.n, fr.FR_KEYS_TBS_TOTAL, True)))
        self.keys = self.ctx.keygen(rots, W.key_seed(cfg))
        self.ctx.load_keys(self.keys)
        self.oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
        self.ok = self.oc.keygen(W.key_seed(cfg))
        self.T, self.q, _ = W.workload(cfg)
        self.lq = self.ctx.work_level
        self.el = self.lq if enroll_level is None else enroll_level
        pre = not server_prerotation
        self.E = self.ctx.encrypt_db(self.keys, self.T, level=self.el, seed=0xE1000, prerotate=pre)
        self.db = self.ctx.load_db_encrypted(self.E, len(self.T), prerotated=pre)
        # what the server holds, per the oracle: the enroller's ciphertexts, or the oracle's
        # server-side pre-rotation of the plain ones
        self.E_server = self.E if pre else self.ok.prerotate_db(self.E, c["n1"], self.lq)
        self.qct = self.ctx.encrypt(self.keys, self.q, W.enc_seed(cfg))
        self.oq = self.ok.encrypt(np.tile(self.q, self.oc.n // c["ell"]), W.enc_seed(cfg))


@pytest.fixture(scope="module")
def mid():
    return Env("mid")


@pytest.fixture(scope="module")
def tbs():
    # plain encrypted diagonals, pre-rotated by the server at load with the negative giant keys
    return Env("mid", server_prerotation=True)


@pytest.fixture(scope="module")
def hoisted():
    # giant steps sharing one ModDown per group
    return Env("mid", hoist=True)


@pytest.fixture(scope="module")
def deep():
    # enrolled at the top level; the server keeps the limbs of its lower working level
    return Env("deep", enroll_level=len(W.CONFIGS["deep"]["q_bits"]) - 1)


def test_enrollment_matches_oracle(mid):
    ref = mid.ok.encrypt_db(mid.T, mid.c["ell"], mid.c["n1"], 0xE1000, level=mid.el)
    assert np.array_equal(mid.E, ref)
    assert mid.db.info()["tier"] == 4 and mid.db.info()["schedule"] == 0


def test_plain_enrollment_matches_oracle(tbs):
    ref = tbs.ok.encrypt_db(tbs.T, tbs.c["ell"], tbs.c["n1"], 0xE1000, level=tbs.el, prerotate=False)
    assert np.array_equal(tbs.E, ref)


@pytest.mark.parametrize("env_name", ["mid", "deep", "tbs", "hoisted"])
@pytest.mark.parametrize("mode", [fr.FR_MODE_SCORES, fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_match_matches_oracle(env_name, mode, request):
    env = request.getfixturevalue(env_name)
    ref, lvl = env.ok.match_enc(env.oq, env.E_server, len(env.T), env.c["n1"], mode, env.c["cheb_degree"],
                                env.c["threshold"], level=env.lq, hoist=env.hoist)
    for call in range(2):   # eager, then the captured graph
        outs = env.ctx.match(env.db, env.qct, mode)
        assert len(outs) == ref.shape[0]
        for g, o in enumerate(outs):
            assert o.level == lvl
            assert np.array_equal(o.export(), ref[g]), (call, g)


def test_scores_decrypt(mid):
    S = mid.ctx.match(mid.db, mid.qct, fr.FR_MODE_SCORES)
    s = mid.T.astype(np.float64) @ mid.q
    n = mid.ctx.n
    got = np.concatenate([mid.ctx.decrypt(mid.keys, o) for o in S])
    assert np.abs(got[:len(s)] - s).max() < 1e-4
    assert np.abs(got[len(s):]).max() < 1e-4
    assert len(S) == -(-len(s) // n)


def test_batch_and_multi_equal_single_calls(mid):
    ctx, keys = mid.ctx, mid.keys
    rng = np.random.default_rng(8)
    qs = []
    for i in range(3):
        v = rng.standard_normal(mid.c["ell"])
        qs.append(ctx.encrypt(keys, v / np.linalg.norm(v), 900 + i))
    single = [[o.export() for o in ctx.match(mid.db, q, fr.FR_MODE_IDENTIFY)] for q in qs]
    batch = ctx.match_batch(mid.db, qs, fr.FR_MODE_IDENTIFY)
    for b in range(3):
        assert all(np.array_equal(o.export(), r) for o, r in zip(batch[b], single[b]))
    # mixed with a plaintext database of another size in one pass
    Tp = W.templates(700, mid.c["ell"], W.DATASET_SEED + 77)
    dbp = ctx.load_db(Tp)
    alone = [o.export() for o in ctx.match(dbp, qs[1], fr.FR_MODE_IDENTIFY)]
    for call in range(2):
        outs = ctx.match_multi([mid.db, dbp, mid.db], qs, fr.FR_MODE_IDENTIFY)
        assert all(np.array_equal(o.export(), r) for o, r in zip(outs[0], single[0]))
        assert all(np.array_equal(o.export(), r) for o, r in zip(outs[1], alone))
        assert all(np.array_equal(o.export(), r) for o, r in zip(outs[2], single[2]))


def test_refusals(mid):
    ctx = mid.ctx
    with pytest.raises(fr.FrError) as e:
        ctx.load_db_encrypted(mid.E[:, :, :, :mid.lq], len(mid.T))     # below the working level
    assert e.value.status == fr.FR_ERR_LEVEL
    bad = mid.E.copy()
    bad[0, 3, 1, 2, 17] = ctx.primes()[2]
    with pytest.raises(fr.FrError) as e:
        ctx.load_db_encrypted(bad, len(mid.T))
    assert e.value.status == fr.FR_ERR_FORMAT
    with pytest.raises(fr.FrError) as e:
        ctx.encrypt_db(mid.keys, mid.T[:, :32])
    assert e.value.status == fr.FR_ERR_INVALID_ARG
    with pytest.raises(fr.FrError) as e:     # server-side pre-rotation without the negative giant keys
        ctx.load_db_encrypted(mid.E, len(mid.T), prerotated=False)
    assert e.value.status == fr.FR_ERR_INVALID_ARG


def test_headline_size_scores_decrypt():
    """N = 2^16, K = 2^15 templates of ell = 512 (one group), 32 near-duplicates, level 8:
    the encrypted database's scores decrypt to the FP64 inner products and the threshold
    separates the near-duplicates."""
    cfg = "membership"
    c = W.CONFIGS[cfg]
    ctx = fr.Context(device=0, **W.ctx_params(cfg, level_mode=1))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
    ctx.load_keys(keys)
    T, q, planted = W.workload(cfg)
    E = ctx.encrypt_db(keys, T, seed=0xE2000)
    db = ctx.load_db_encrypted(E, len(T))
    del E
    qct = ctx.encrypt(keys, q, W.enc_seed(cfg))
    s = T.astype(np.float64) @ q
    got = ctx.decrypt(keys, ctx.match(db, qct, fr.FR_MODE_SCORES)[0])
    assert np.abs(got - s).max() < 1e-4
    ident = ctx.decrypt(keys, ctx.match(db, qct, fr.FR_MODE_IDENTIFY)[0])
    far = np.abs(s - c["threshold"]) > 0.02
    assert np.array_equal((ident >= 0.5)[far], (s >= c["threshold"])[far])
    assert set(np.flatnonzero(ident >= 0.5)) >= set(int(i) for i in planted)


def test_serving_loop_with_encrypted_database(mid):
    """Requests against an encrypted database through fr_match_submit / fr_match_poll give the
    outputs of fr_match."""
    ctx, keys = mid.ctx, mid.keys
    qs = [ctx.encrypt(keys, mid.q, 700 + i) for i in range(3)]
    ref = [[o.export() for o in ctx.match(mid.db, q, fr.FR_MODE_IDENTIFY)] for q in qs]
    ctx.serve_start(max_batch=4, slots=2)
    try:
        tickets = [ctx.submit(mid.db, q, fr.FR_MODE_IDENTIFY) for q in qs]
        for t, r in zip(tickets, ref):
            outs = ctx.poll(t)
            assert all(np.array_equal(o.export(), x) for o, x in zip(outs, r))
    finally:
        ctx.serve_stop()
