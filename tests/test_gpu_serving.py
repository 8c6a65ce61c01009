"""GPU tests of the serving loop (continuous batching through fr_match_submit /
fr_match_poll): a mix of membership, identification and score requests against two
resident databases, host and device queries, submitted while earlier batches run. Each
result must equal the same query matched alone by fr_match, bit for bit, and the first
ones also the oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    c = W.CONFIGS["mid"]
    ctx = fr.Context(device=0, **W.ctx_params("mid"))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
    ctx.load_keys(keys)
    T, q, _ = W.workload("mid")
    T2 = W.templates(1500, c["ell"], W.DATASET_SEED + 55)
    dbs = [ctx.load_db(T), ctx.load_db(T2)]
    rng = np.random.default_rng(77)
    queries = []
    for r in range(6):
        v = rng.standard_normal(c["ell"])
        v /= np.linalg.norm(v)
        queries.append((v, 3000 + r))
    return dict(c=c, ctx=ctx, keys=keys, Ts=[T, T2], dbs=dbs, queries=queries)


def requests(env):
    modes = [fr.FR_MODE_MEMBERSHIP, fr.FR_MODE_IDENTIFY, fr.FR_MODE_SCORES]
    out = []
    for i in range(14):
        out.append((i % 2, modes[(i // 2) % 3], i % len(env["queries"]), i % 3 == 0))
    return out


def alone(env, d, mode, qi):
    v, seed = env["queries"][qi]
    ct = env["ctx"].encrypt(env["keys"], v, seed)
    return [o.export() for o in env["ctx"].match(env["dbs"][d], ct, mode)]


@pytest.mark.parametrize("max_batch,slots", [(4, 2), (8, 3), (1, 1)])
def test_results_equal_alone_and_in_the_mix(env, max_batch, slots):
    ctx = env["ctx"]
    reqs = requests(env)
    ref = [alone(env, d, m, qi) for d, m, qi, _ in reqs]
    ctx.serve_start(max_batch=max_batch, slots=slots)
    try:
        cts = []
        tickets = []
        for d, m, qi, on_dev in reqs:
            v, seed = env["queries"][qi]
            ct = ctx.encrypt(env["keys"], v, seed)
            if on_dev:
                ct.upload()
            cts.append(ct)
            tickets.append(ctx.submit(env["dbs"][d], ct, m))
        del cts   # the loop keeps what it needs
        for i, t in enumerate(reversed(tickets)):
            got, lat = ctx.poll(t, -1, with_latency=True)
            j = len(tickets) - 1 - i
            assert len(got) == len(ref[j])
            assert lat > 0
            for g in range(len(got)):
                assert np.array_equal(got[g].export(), ref[j][g]), (j, g)
        st = ctx.serve_stats()
        assert st["completed"] == len(reqs) and st["outstanding"] == 0
        assert st["batches"] <= len(reqs)
        if max_batch == 1:
            assert st["batches"] == len(reqs)
    finally:
        ctx.serve_stop()


def test_mix_matches_oracle_and_ticket_rules(env):
    ctx, c = env["ctx"], env["c"]
    v, seed = env["queries"][0]
    ctx.serve_start(max_batch=4, slots=2)
    try:
        t1 = ctx.submit(env["dbs"][0], ctx.encrypt(env["keys"], v, seed), fr.FR_MODE_MEMBERSHIP)
        t2 = ctx.submit(env["dbs"][1], ctx.encrypt(env["keys"], v, seed), fr.FR_MODE_IDENTIFY)
        out1 = ctx.poll(t1)
        out2 = ctx.poll(t2)
        with pytest.raises(fr.FrError) as e:
            ctx.poll(t1, 0)               # consumed
        assert e.value.status == fr.FR_ERR_INVALID_ARG
        with pytest.raises(fr.FrError):
            ctx.poll(123456789, 0)        # never issued
    finally:
        ctx.serve_stop()
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed("mid"))
    oq = ok.encrypt(np.tile(v, oc.n // c["ell"]), seed)
    ref1, _ = ok.match(oq, env["Ts"][0], c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5)
    ref2, _ = ok.match(oq, env["Ts"][1], c["ell"], c["n1"], fr.FR_MODE_IDENTIFY, 59, 0.5)
    assert np.array_equal(out1[0].export(), ref1[0])
    assert len(out2) == len(ref2)
    for g in range(len(ref2)):
        assert np.array_equal(out2[g].export(), ref2[g])


def test_tight_budget_runs_requests_one_by_one(env):
    """A budget below one request's workspace: each batch runs alone once nothing else is
    in flight; results are unchanged."""
    ctx = env["ctx"]
    v, seed = env["queries"][1]
    ref = alone(env, 0, fr.FR_MODE_MEMBERSHIP, 1)
    ctx.serve_start(max_batch=8, slots=2, hbm_budget_bytes=1)
    try:
        ts = [ctx.submit(env["dbs"][0], ctx.encrypt(env["keys"], v, seed), fr.FR_MODE_MEMBERSHIP) for _ in range(4)]
        for t in ts:
            assert np.array_equal(ctx.poll(t)[0].export(), ref[0])
        st = ctx.serve_stats()
        assert st["batches"] == 4 and st["max_concurrent_batches"] == 1
    finally:
        ctx.serve_stop()
