"""GPU test of the block-sharded match: a database split along group boundaries, each shard
matched on its own (as one rank of a multi-GPU job would), the per-group outputs passed through
the export format (as the exchange between ranks does) and reduced with fr_membership_reduce.
Identification must give the whole database's per-group outputs, and membership the whole
database's membership ciphertext, bit for bit."""
import numpy as np
import pytest

from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import shard
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    c = W.CONFIGS["mid"]   # N = 2^13: 4096 templates per group
    ctx = fr.Context(device=0, **W.ctx_params("mid"))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
    ctx.load_keys(keys)
    T = W.templates(9000, c["ell"], W.DATASET_SEED + 500)     # 3 groups, the last one ragged
    rng = np.random.default_rng(5)
    q = rng.standard_normal(c["ell"])
    return dict(c=c, ctx=ctx, keys=keys, T=T, full=ctx.load_db(T), q=q / np.linalg.norm(q))


@pytest.mark.parametrize("world", [2, 3, 4])
def test_shards_reduce_to_whole_database(env, world):
    ctx, keys, T = env["ctx"], env["keys"], env["T"]
    slots = ctx.n
    qct = ctx.encrypt(keys, env["q"], 321)
    full_id = [o.export() for o in ctx.match(env["full"], qct, fr.FR_MODE_IDENTIFY)]
    full_mem = ctx.match(env["full"], qct, fr.FR_MODE_MEMBERSHIP)[0].export()
    parts = []
    for r in range(world):
        Ts, (g0, g1) = shard.template_shard(T, slots, world, r)
        if g1 == g0:
            continue
        db = ctx.load_db(Ts)
        outs = shard.sharded_match(ctx, db, qct, fr.FR_MODE_IDENTIFY)
        assert len(outs) == g1 - g0
        for g, o in zip(range(g0, g1), outs):
            w = o.export()
            assert np.array_equal(w, full_id[g]), (r, g)
            parts.append(ctx.import_ct(w, w.shape[1] - 1))     # through the exchange format
    assert len(parts) == len(full_id)
    got = ctx.membership_reduce(parts).export()
    assert np.array_equal(got, full_mem)
    rev = ctx.membership_reduce(parts[::-1]).export()          # the sum is order-free
    assert np.array_equal(rev, full_mem)


def test_one_shard_is_the_plain_match(env):
    ctx, keys = env["ctx"], env["keys"]
    qct = ctx.encrypt(keys, env["q"], 322)
    got = shard.sharded_match(ctx, env["full"], qct, fr.FR_MODE_MEMBERSHIP)[0].export()
    assert np.array_equal(got, ctx.match(env["full"], qct, fr.FR_MODE_MEMBERSHIP)[0].export())


def test_reduce_refusals(env):
    ctx, keys = env["ctx"], env["keys"]
    qct = ctx.encrypt(keys, env["q"], 323)
    outs = ctx.match(env["full"], qct, fr.FR_MODE_IDENTIFY)
    with pytest.raises(fr.FrError) as e:
        ctx.membership_reduce([])
    assert e.value.status == fr.FR_ERR_INVALID_ARG
    with pytest.raises(fr.FrError) as e:
        ctx.membership_reduce([outs[0], ctx.rescale(outs[1])])
    assert e.value.status == fr.FR_ERR_LEVEL
