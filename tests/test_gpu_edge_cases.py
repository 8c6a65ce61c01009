"""Edge cases of the match on the GPU, bit-exact against the oracle where a result exists:
a single template; exactly one full group of N/2 slots and one more row (a second group
holding one template); n1 not dividing ell (a partial last giant step) under both schedules;
and the API's refusals (empty database, bad batch sizes, wrong level, unknown mode, objects
of another context)."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C = W.CONFIGS["tiny"]   # N = 2^12 (2048 slots), ell = 64, n1 = 8, scores only


def make(n1=None, schedule=0):
    prm = W.ctx_params("tiny")
    if n1 is not None:
        prm["n1"] = n1
    ctx = fr.Context(device=0, schedule=schedule, **prm)
    n1v = prm["n1"]
    rots = sorted(set(list(range(1, n1v)) + [n1v * j for j in range(1, (C["ell"] + n1v - 1) // n1v)]))
    keys = ctx.keygen(rots, W.key_seed("tiny"))
    ctx.load_keys(keys)
    return ctx, keys


@pytest.fixture(scope="module")
def orc():
    oc = oracle.Ctx(C["log_n"], C["q_bits"], C["p_bits"], C["dnum"], C["scale_bits"])
    return oc, oc.keygen(W.key_seed("tiny"))


def query(seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(C["ell"])
    return q / np.linalg.norm(q)


def check_scores(ctx, keys, orc, T, n1, seed, schedule=0):
    oc, ok = orc
    q = query(seed)
    db = ctx.load_db(T)
    out = ctx.match(db, ctx.encrypt(keys, q, seed), fr.FR_MODE_SCORES)
    oq = ok.encrypt(np.tile(q, oc.n // C["ell"]), seed)
    ref = (ok.table_scores if schedule == 1 else ok.bsgs_scores)(oq, T, C["ell"], n1)
    assert len(out) == len(ref)
    for g in range(len(ref)):
        assert np.array_equal(out[g].export(), ref[g]), g
    s = T.astype(np.float64) @ q
    dec = np.concatenate([ctx.decrypt(keys, o) for o in out])
    assert np.abs(dec[: len(s)] - s).max() < 1e-4
    if len(dec) > len(s):
        assert np.abs(dec[len(s):]).max() < 1e-4   # padding rows score 0


def test_single_template(orc):
    ctx, keys = make()
    check_scores(ctx, keys, orc, W.templates(1, C["ell"], 11), C["n1"], 101)


@pytest.mark.parametrize("K", [2048, 2049])
def test_full_group_and_one_more_row(orc, K):
    ctx, keys = make()
    check_scores(ctx, keys, orc, W.templates(K, C["ell"], 12), C["n1"], 102)


@pytest.mark.parametrize("schedule", [0, 1])
def test_n1_not_dividing_ell(orc, schedule):
    # ell = 64, n1 = 5: n2 = 13 giant steps, the last one with 4 diagonals
    ctx, keys = make(n1=5, schedule=schedule)
    check_scores(ctx, keys, orc, W.templates(300, C["ell"], 13), 5, 103, schedule)


def test_refusals():
    ctx, keys = make()
    other, okeys = make()
    T = W.templates(100, C["ell"], 14)
    with pytest.raises(fr.FrError) as e:
        ctx.load_db(np.zeros((0, C["ell"]), dtype=np.float32))
    assert e.value.status == fr.FR_ERR_INVALID_ARG
    db = ctx.load_db(T)
    q = ctx.encrypt(keys, query(5), 5)
    with pytest.raises(fr.FrError) as e:
        ctx.match_batch(db, [], fr.FR_MODE_SCORES)
    assert e.value.status == fr.FR_ERR_INVALID_ARG
    with pytest.raises(fr.FrError) as e:
        ctx.match_batch(db, [q] * 65, fr.FR_MODE_SCORES)
    assert e.value.status == fr.FR_ERR_INVALID_ARG
    with pytest.raises(fr.FrError) as e:
        ctx.match(db, ctx.rescale(q.upload()), fr.FR_MODE_SCORES)
    assert e.value.status == fr.FR_ERR_LEVEL
    with pytest.raises(fr.FrError) as e:
        ctx.match(db, q, 7)
    assert e.value.status == fr.FR_ERR_INVALID_ARG
    with pytest.raises(fr.FrError) as e:
        ctx.match(other.load_db(T), q, fr.FR_MODE_SCORES)
    assert e.value.status == fr.FR_ERR_INVALID_ARG
    # a context without a Chebyshev degree refuses the threshold modes
    with pytest.raises(fr.FrError) as e:
        ctx.match(db, q, fr.FR_MODE_MEMBERSHIP)
    assert e.value.status == fr.FR_ERR_INVALID_ARG


def test_profile_only_times_one_region_class(orc):
    # a profiled match with a region filter times that class only (and the whole replay); the
    # outputs are the same bits as unprofiled
    ctx, keys = make()
    T = W.templates(300, C["ell"], 15)
    db = ctx.load_db(T)
    q = ctx.encrypt(keys, query(6), 6)
    ref = [o.export() for o in ctx.match(db, q, fr.FR_MODE_SCORES)]
    for only in ("ntt", "ip", ""):
        ctx.profile_only(only)
        ctx.profile(True)
        out = ctx.match(db, q, fr.FR_MODE_SCORES)
        ms_ntt, n_ntt, _ = ctx.profile_read("ntt")
        ms_ip, n_ip, _ = ctx.profile_read("ip")
        ms_match, n_match, _ = ctx.profile_read("match")
        ctx.profile(False)
        assert len(out) == len(ref) and all(np.array_equal(o.export(), r) for o, r in zip(out, ref))
        assert n_match == 1 and ms_match > 0
        assert (n_ntt > 0) == (only in ("ntt", ""))
        assert (n_ip > 0) == (only in ("ip", ""))
        assert ms_ntt + ms_ip <= ms_match
    ctx.profile_only("")


def test_stage_profile_keeps_both_chebyshev_streams():
    # a membership match profiled by stages only runs the Chebyshev branches on their two
    # streams, one profiled by region class on one stream; every form gives the unprofiled bits
    cfg = "mid"
    ctx = fr.Context(device=0, **W.ctx_params(cfg))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
    ctx.load_keys(keys)
    T, q, _ = W.workload(cfg)
    db = ctx.load_db(T)
    qct = ctx.encrypt(keys, q, W.enc_seed(cfg))
    ref = ctx.match(db, qct, fr.FR_MODE_MEMBERSHIP)[0].export()
    for only in ("stage:", ""):
        ctx.profile_only(only)
        ctx.profile(True)
        out = ctx.match(db, qct, fr.FR_MODE_MEMBERSHIP)[0].export()
        ms_cheb, n_cheb, _ = ctx.profile_read("stage:cheb")
        ms_match, n_match, _ = ctx.profile_read("match")
        n_ntt = ctx.profile_read("ntt")[1]
        ctx.profile(False)
        assert np.array_equal(out, ref)
        assert n_cheb == 1 and 0 < ms_cheb <= ms_match
        assert (n_ntt > 0) == (only == "")
    ctx.profile_only("")
