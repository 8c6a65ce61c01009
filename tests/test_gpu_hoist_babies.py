"""GPU parity of the baby steps kept in Q_l u P (fr_params.hoist_babies, double hoisting of the
baby steps): every output bit-exact against the oracle's or_bsgs_scores_pq / match(babies_pq)
for scores, identification and membership, with one ModDown per giant step fused with its
rescale; with the giant steps sharing one ModDown too; for one query, a batch, a multi-database
pass; for the three plaintext storage tiers; and at the headline size. Encrypted databases
refuse the flag."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 1], ids=["giants-plain", "giants-hoisted"])
def env(request):
    c = W.CONFIGS["mid"]
    ctx = fr.Context(device=0, hoist_babies=1, hoist_giants=request.param, **W.ctx_params("mid"))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
    ctx.load_keys(keys)
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed("mid"))
    T, q, _ = W.workload("mid")
    return dict(c=c, ctx=ctx, keys=keys, oc=oc, ok=ok, T=T, q=q, db=ctx.load_db(T, tier=1),
                hoist=bool(request.param))


def oracle_query(env, seed):
    return env["ok"].encrypt(np.tile(env["q"], env["oc"].n // env["c"]["ell"]), seed)


@pytest.mark.parametrize("mode", [fr.FR_MODE_SCORES, fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_match_matches_oracle(env, mode):
    c, ctx = env["c"], env["ctx"]
    seed = W.enc_seed("mid", 5)
    qct = ctx.encrypt(env["keys"], env["q"], seed)
    ref, lvl = env["ok"].match(oracle_query(env, seed), env["T"], c["ell"], c["n1"], mode, 59, 0.5,
                               hoist=env["hoist"], babies_pq=True)
    for call in range(2):   # eager, then the captured graph
        outs = ctx.match(env["db"], qct, mode)
        assert len(outs) == ref.shape[0]
        for g, o in enumerate(outs):
            assert o.level == lvl
            assert np.array_equal(o.export(), ref[g]), (call, g)


def test_scores_decrypt_to_matvec(env):
    c, ctx = env["c"], env["ctx"]
    qct = ctx.encrypt(env["keys"], env["q"], 4242)
    outs = ctx.match(env["db"], qct, fr.FR_MODE_SCORES)
    got = np.concatenate([ctx.decrypt(env["keys"], o) for o in outs])[: len(env["T"])]
    assert np.abs(got - env["T"].astype(np.float64) @ env["q"]).max() < 1e-4


def test_batch_multi_and_tiers_match_oracle(env):
    c, ctx = env["c"], env["ctx"]
    seeds = [W.enc_seed("mid", 10 + i) for i in range(3)]
    qs = [ctx.encrypt(env["keys"], env["q"], s) for s in seeds]
    refs = [env["ok"].match(oracle_query(env, s), env["T"], c["ell"], c["n1"], fr.FR_MODE_IDENTIFY, 59, 0.5,
                            hoist=env["hoist"], babies_pq=True)[0] for s in seeds]
    batch = ctx.match_batch(env["db"], qs, fr.FR_MODE_IDENTIFY)
    for b in range(3):
        assert all(np.array_equal(o.export(), r) for o, r in zip(batch[b], refs[b])), b
    T2 = W.templates(700, c["ell"], W.DATASET_SEED + 91)
    db2 = ctx.load_db(T2, tier=1)
    ref2 = env["ok"].match(oracle_query(env, seeds[1]), T2, c["ell"], c["n1"], fr.FR_MODE_IDENTIFY, 59, 0.5,
                           hoist=env["hoist"], babies_pq=True)[0]
    outs = ctx.match_multi([env["db"], db2, env["db"]], qs, fr.FR_MODE_IDENTIFY)
    assert all(np.array_equal(o.export(), r) for o, r in zip(outs[0], refs[0]))
    assert all(np.array_equal(o.export(), r) for o, r in zip(outs[1], ref2))
    assert all(np.array_equal(o.export(), r) for o, r in zip(outs[2], refs[2]))
    # the per-query encoded tiers (templates resident; integer coefficients resident)
    for tier in (2, 3):
        dbt = ctx.load_db(env["T"], tier=tier)
        got = ctx.match(dbt, qs[0], fr.FR_MODE_IDENTIFY)
        assert all(np.array_equal(o.export(), r) for o, r in zip(got, refs[0])), tier
    ctx.load_db(T2, tier=0)   # back to the automatic tier for later loads


def test_encrypted_database_refuses_hoisted_babies(env):
    c, ctx = env["c"], env["ctx"]
    T = W.templates(300, c["ell"], W.DATASET_SEED + 92)
    E = ctx.encrypt_db(env["keys"], T, seed=0xE7000)
    db = ctx.load_db_encrypted(E, len(T))
    with pytest.raises(fr.FrError) as e:
        ctx.match(db, ctx.encrypt(env["keys"], env["q"], 4243), fr.FR_MODE_SCORES)
    assert e.value.status == fr.FR_ERR_UNSUPPORTED


def test_membership_full_size_bit_exact():
    """The headline membership (N = 2^16, K = 2^15, working level 8, giant steps sharing one
    ModDown, RotateAndSum in radix 4) with the baby steps in Q_l u P: bit-exact with the oracle
    and within the membership tolerance of the FP64 sum."""
    cfg = "membership"
    c = W.CONFIGS[cfg]
    ctx = fr.Context(device=0, hoist_babies=1, hoist_giants=1, sum_radix=4, **W.ctx_params(cfg, level_mode=1))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
    ctx.load_keys(keys)
    T, q, _ = W.workload(cfg)
    db = ctx.load_db(T)
    qct = ctx.encrypt(keys, q, W.enc_seed(cfg))
    outs = [ctx.match(db, qct, fr.FR_MODE_MEMBERSHIP)[0] for _ in range(2)]
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed(cfg))
    oq = ok.encrypt(np.tile(q, oc.n // c["ell"]), W.enc_seed(cfg))
    ref, lvl = ok.match(oq, T, c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5, level=ctx.work_level, sum_radix=4,
                        hoist=True, babies_pq=True)
    for o in outs:
        assert o.level == lvl and np.array_equal(o.export(), ref[0])
    s = T.astype(np.float64) @ q
    p = np.polynomial.chebyshev.chebval(s, fr.cheb_coeffs(59, 0.5))
    assert abs(ctx.decrypt(keys, outs[0])[0] - p.sum()) < 1e-2
