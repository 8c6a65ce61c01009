"""GPU parity of RotateAndSum in radix r (fr_params.sum_radix): each step adds the r-1
rotations by t s of the running sum, hoisted over one ModUp; with fr_params.hoist_sum the
rotations of a step also share one ModDown. Bit-exact against the oracle's radix-r
RotateAndSum (plain or with one ModDown per step), alone and inside the membership match (one
query and a batch); the rotation-key set follows the radix."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def make(radix, hoist_sum=0):
    c = W.CONFIGS["mid"]
    ctx = fr.Context(device=0, sum_radix=radix, hoist_sum=hoist_sum, **W.ctx_params("mid"))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
    ctx.load_keys(keys)
    return c, ctx, keys


@pytest.fixture(scope="module")
def oc():
    c = W.CONFIGS["mid"]
    o = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    return o, o.keygen(W.key_seed("mid"))


def test_key_set_follows_radix():
    _, ctx, _ = make(8)
    rots = set(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP))
    n = ctx.n                                   # 4096 slots = 8^4
    want = {t * s for s in (1, 8, 64, 512) for t in range(1, 8)}
    # the babies 1..7 and the giants 8..56 are radix-8 steps themselves
    assert rots == want
    _, ctx2, _ = make(0)
    assert {1 << t for t in range(12)} <= set(ctx2.required_rotations(fr.FR_MODE_MEMBERSHIP))
    with pytest.raises(fr.FrError):
        fr.Context(device=0, sum_radix=6, **W.ctx_params("mid"))
    assert n == 4096


@pytest.mark.parametrize("radix", [4, 8, 32])
def test_rotate_sum_matches_oracle(oc, radix):
    o, ok = oc
    _, ctx, keys = make(radix)
    rng = np.random.default_rng(radix)
    z = rng.uniform(-1, 1, o.n) / o.n
    ct = ok.encrypt(z, 40 + radix)
    lvl = 2
    low = o.drop(ct, o.top, lvl)
    got = ctx.rotate_sum(ctx.import_ct(low, lvl)).export()
    ref = ok.rotate_sum(low, lvl, int(np.log2(o.n)), radix=radix)
    assert np.array_equal(got, ref)
    assert np.abs(ok.decrypt(ref, lvl) - z.sum()).max() < 1e-5


@pytest.mark.parametrize("radix", [8, 64])
def test_membership_matches_oracle(oc, radix):
    o, ok = oc
    c, ctx, keys = make(radix)
    T, q, _ = W.workload("mid")
    db = ctx.load_db(T)
    qs = [ctx.encrypt(keys, q, W.enc_seed("mid", i)) for i in range(2)]
    refs = []
    for i in range(2):
        oq = ok.encrypt(np.tile(q, o.n // c["ell"]), W.enc_seed("mid", i))
        ref, lvl = ok.match(oq, T, c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5, sum_radix=radix)
        refs.append(ref[0])
    for call in range(2):   # eager, then the captured graph
        got = ctx.match(db, qs[0], fr.FR_MODE_MEMBERSHIP)[0].export()
        assert np.array_equal(got, refs[0]), call
    batch = ctx.match_batch(db, qs, fr.FR_MODE_MEMBERSHIP)
    for i in range(2):
        assert np.array_equal(batch[i][0].export(), refs[i])


@pytest.mark.parametrize("radix", [2, 4, 32])
def test_rotate_sum_one_moddown_per_step_matches_oracle(oc, radix):
    o, ok = oc
    _, ctx, keys = make(radix, hoist_sum=1)
    rng = np.random.default_rng(100 + radix)
    z = rng.uniform(-1, 1, o.n) / o.n
    ct = ok.encrypt(z, 60 + radix)
    lvl = 2
    low = o.drop(ct, o.top, lvl)
    got = ctx.rotate_sum(ctx.import_ct(low, lvl)).export()
    ref = ok.rotate_sum(low, lvl, int(np.log2(o.n)), radix=radix, hoist=True)
    assert np.array_equal(got, ref)
    assert np.abs(ok.decrypt(ref, lvl) - z.sum()).max() < 1e-5


def test_membership_one_moddown_per_sum_step_matches_oracle(oc):
    o, ok = oc
    c, ctx, keys = make(8, hoist_sum=1)
    T, q, _ = W.workload("mid")
    db = ctx.load_db(T)
    qs = [ctx.encrypt(keys, q, W.enc_seed("mid", i)) for i in range(2)]
    refs = []
    for i in range(2):
        oq = ok.encrypt(np.tile(q, o.n // c["ell"]), W.enc_seed("mid", i))
        ref, lvl = ok.match(oq, T, c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5, sum_radix=8, hoist_sum=True)
        refs.append(ref[0])
    for call in range(2):   # eager, then the captured graph
        got = ctx.match(db, qs[0], fr.FR_MODE_MEMBERSHIP)[0].export()
        assert np.array_equal(got, refs[0]), call
    batch = ctx.match_batch(db, qs, fr.FR_MODE_MEMBERSHIP)
    for i in range(2):
        assert np.array_equal(batch[i][0].export(), refs[i])
