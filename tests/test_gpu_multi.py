"""GPU tests of fr_match_multi (configuration "batched launches"): queries against databases
of uneven sizes and storage tiers in one pass. Each query's outputs must equal fr_match on
that query and database alone, bit for bit, on the eager first call and on the replayed graph;
one pair is also checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    c = W.CONFIGS["mid"]   # N = 2^13: 4096 slots per group
    ctx = fr.Context(device=0, **W.ctx_params("mid"))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
    ctx.load_keys(keys)
    sizes = [(100, 1), (4096, 2), (5000, 3), (9000, 1), (300, 3)]   # (K, tier): G = 1, 1, 2, 3, 1
    Ts = [W.templates(K, c["ell"], W.DATASET_SEED + 300 + i) for i, (K, _) in enumerate(sizes)]
    dbs = [ctx.load_db(T, tier=t) for T, (_, t) in zip(Ts, sizes)]
    ctx.load_db(Ts[0][:1], tier=0)   # back to auto for later loads
    rng = np.random.default_rng(41)
    qv = []
    for i in range(6):
        v = rng.standard_normal(c["ell"])
        qv.append(v / np.linalg.norm(v))
    return dict(c=c, ctx=ctx, keys=keys, Ts=Ts, dbs=dbs, qv=qv)


def pairs(env):
    # 6 queries: the five databases and the 9000-template one again
    return [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (5, 3)]


@pytest.mark.parametrize("mode", [fr.FR_MODE_SCORES, fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_multi_equals_each_pair_alone(env, mode):
    ctx, keys = env["ctx"], env["keys"]
    pr = pairs(env)
    assert [d.info()["tier"] for d in env["dbs"]] == [1, 2, 3, 1, 3]
    ref = []
    for qi, di in pr:
        ct = ctx.encrypt(keys, env["qv"][qi], 4000 + qi)
        ref.append([o.export() for o in ctx.match(env["dbs"][di], ct, mode)])
    for call in range(2):
        qs = [ctx.encrypt(keys, env["qv"][qi], 4000 + qi) for qi, _ in pr]
        outs = ctx.match_multi([env["dbs"][di] for _, di in pr], qs, mode)
        assert len(outs) == len(pr)
        for b in range(len(pr)):
            assert len(outs[b]) == len(ref[b])
            for g in range(len(ref[b])):
                assert np.array_equal(outs[b][g].export(), ref[b][g]), (call, b, g)


def test_multi_pair_matches_oracle(env):
    c, ctx, keys = env["c"], env["ctx"], env["keys"]
    qi, di = 5, 3
    outs = ctx.match_multi([env["dbs"][2], env["dbs"][di]],
                           [ctx.encrypt(keys, env["qv"][0], 77), ctx.encrypt(keys, env["qv"][qi], 78)],
                           fr.FR_MODE_MEMBERSHIP)
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed("mid"))
    oq = ok.encrypt(np.tile(env["qv"][qi], oc.n // c["ell"]), 78)
    ref, _ = ok.match(oq, env["Ts"][di], c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5)
    assert np.array_equal(outs[1][0].export(), ref[0])


def test_graph_cache_eviction_keeps_results(env):
    """More distinct database lists than the per-context graph cache holds (16): every list is
    matched twice (eager, then captured), the least used graphs are dropped, and a list whose
    graph was dropped still gives the same outputs when it comes back."""
    ctx, keys, dbs = env["ctx"], env["keys"], env["dbs"]
    combos = [(i, j) for i in range(len(dbs)) for j in range(len(dbs)) if i != j]   # 20 lists
    q = [ctx.encrypt(keys, env["qv"][0], 91), ctx.encrypt(keys, env["qv"][1], 92)]
    first = {}
    for i, j in combos:
        for _ in range(2):
            outs = ctx.match_multi([dbs[i], dbs[j]], q, fr.FR_MODE_SCORES)
            got = [[o.export() for o in out] for out in outs]
            if (i, j) in first:
                assert all(np.array_equal(a, b) for x, y in zip(got, first[(i, j)]) for a, b in zip(x, y))
            first[(i, j)] = got
    for i, j in combos[:3]:   # dropped by now
        outs = ctx.match_multi([dbs[i], dbs[j]], q, fr.FR_MODE_SCORES)
        got = [[o.export() for o in out] for out in outs]
        assert all(np.array_equal(a, b) for x, y in zip(got, first[(i, j)]) for a, b in zip(x, y))
