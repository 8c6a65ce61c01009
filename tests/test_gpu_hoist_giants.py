"""GPU parity of the giant steps sharing one ModDown per (query, group) (fr_params.hoist_giants,
double hoisting): bit-exact against the oracle's hoisted giant steps for scores,
identification and membership, one query, a batch, and a multi-database pass; with one giant
step the outputs equal the unhoisted ones."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    c = W.CONFIGS["mid"]
    ctx = fr.Context(device=0, hoist_giants=1, **W.ctx_params("mid"))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
    ctx.load_keys(keys)
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed("mid"))
    T, q, _ = W.workload("mid")
    return dict(c=c, ctx=ctx, keys=keys, oc=oc, ok=ok, T=T, q=q, db=ctx.load_db(T))


def oracle_query(env, seed):
    return env["ok"].encrypt(np.tile(env["q"], env["oc"].n // env["c"]["ell"]), seed)


@pytest.mark.parametrize("mode", [fr.FR_MODE_SCORES, fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_match_matches_oracle(env, mode):
    c, ctx = env["c"], env["ctx"]
    seed = W.enc_seed("mid", 5)
    qct = ctx.encrypt(env["keys"], env["q"], seed)
    ref, lvl = env["ok"].match(oracle_query(env, seed), env["T"], c["ell"], c["n1"], mode, 59, 0.5, hoist=True)
    for call in range(2):   # eager, then the captured graph
        outs = ctx.match(env["db"], qct, mode)
        assert len(outs) == ref.shape[0]
        for g, o in enumerate(outs):
            assert o.level == lvl
            assert np.array_equal(o.export(), ref[g]), (call, g)


def test_batch_and_multi_match_oracle(env):
    c, ctx = env["c"], env["ctx"]
    seeds = [W.enc_seed("mid", 10 + i) for i in range(3)]
    qs = [ctx.encrypt(env["keys"], env["q"], s) for s in seeds]
    refs = [env["ok"].match(oracle_query(env, s), env["T"], c["ell"], c["n1"], fr.FR_MODE_IDENTIFY, 59, 0.5,
                            hoist=True)[0] for s in seeds]
    batch = ctx.match_batch(env["db"], qs, fr.FR_MODE_IDENTIFY)
    for b in range(3):
        assert all(np.array_equal(o.export(), r) for o, r in zip(batch[b], refs[b]))
    T2 = W.templates(700, c["ell"], W.DATASET_SEED + 91)
    db2 = ctx.load_db(T2)
    ref2 = env["ok"].match(oracle_query(env, seeds[1]), T2, c["ell"], c["n1"], fr.FR_MODE_IDENTIFY, 59, 0.5,
                           hoist=True)[0]
    outs = ctx.match_multi([env["db"], db2, env["db"]], qs, fr.FR_MODE_IDENTIFY)
    assert all(np.array_equal(o.export(), r) for o, r in zip(outs[0], refs[0]))
    assert all(np.array_equal(o.export(), r) for o, r in zip(outs[1], ref2))
    assert all(np.array_equal(o.export(), r) for o, r in zip(outs[2], refs[2]))


def test_one_giant_step_equals_unhoisted():
    c = dict(W.CONFIGS["mid"], n1=32)           # ell = 64: n2 = 2, one giant rotation
    outs = []
    for h in (0, 1):
        ctx = fr.Context(device=0, hoist_giants=h, **W.ctx_params(c))
        keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_SCORES), W.key_seed("mid"))
        ctx.load_keys(keys)
        T, q, _ = W.workload("mid")
        db = ctx.load_db(T)
        outs.append([o.export() for o in ctx.match(db, ctx.encrypt(keys, q, 77), fr.FR_MODE_SCORES)])
    assert all(np.array_equal(a, b) for a, b in zip(outs[0], outs[1]))
