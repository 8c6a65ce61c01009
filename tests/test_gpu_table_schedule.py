"""GPU parity of the rotated-query table schedule (Algorithm 1, BSGS-Diagonal): all ell
rotations of the query are built once (babies hoisted over one ModUp of the query, giant
rotations of each baby hoisted over one ModUp of that baby), then every template group
is one sum of ell products with the plain diagonals and one rescale. Outputs are compared
bit for bit with the oracle's table schedule, at the top level and at the working level,
with stored and per-query-encoded diagonals, on the first (eager) and second (captured
graph) call."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def setup(cfg, schedule, tier=0, K=None, level_mode=None):
    c = W.CONFIGS[cfg]
    ctx = fr.Context(device=0, schedule=schedule, db_tier=tier, **W.ctx_params(cfg, level_mode=level_mode))
    mode = fr.FR_MODE_MEMBERSHIP if c["mode"] == 2 else c["mode"]
    keys = ctx.keygen(ctx.required_rotations(mode), W.key_seed(cfg))
    ctx.load_keys(keys)
    T, q, _ = W.workload(cfg)
    if K is not None:
        T = W.templates(K, c["ell"], W.DATASET_SEED + 99)
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed(cfg))
    qct = ctx.encrypt(keys, q, W.enc_seed(cfg))
    oq = ok.encrypt(np.tile(q, oc.n // c["ell"]), W.enc_seed(cfg))
    return c, ctx, keys, T, q, oc, ok, qct, oq


def test_table_scores_tiny():
    c, ctx, keys, T, q, oc, ok, qct, oq = setup("tiny", 1)
    db = ctx.load_db(T)
    assert db.info()["schedule"] == 1
    ref = ok.table_scores(oq, T, c["ell"], c["n1"])
    for _ in range(2):
        out = ctx.match(db, qct, fr.FR_MODE_SCORES)
        assert np.array_equal(out[0].export(), ref[0])
    s = T.astype(np.float64) @ q
    assert np.abs(ctx.decrypt(keys, out[0])[: len(s)] - s).max() < 1e-4


@pytest.mark.parametrize("tier", [1, 2, 3])
def test_table_scores_and_membership_mid(tier):
    """Two groups with a ragged tail; tier 2 encodes the plain diagonals per query, tier 3
    expands their stored integer coefficients per query."""
    c, ctx, keys, T, q, oc, ok, qct, oq = setup("mid", 1, tier=tier)
    db = ctx.load_db(T)
    assert db.info()["schedule"] == 1 and db.info()["tier"] == tier and db.info()["groups"] == 2
    ref = ok.table_scores(oq, T, c["ell"], c["n1"])
    refm, lvl = ok.match(oq, T, c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5, schedule=1)
    for _ in range(2):
        out = ctx.match(db, qct, fr.FR_MODE_SCORES)
        for g in range(2):
            assert np.array_equal(out[g].export(), ref[g]), g
        m = ctx.match(db, qct, fr.FR_MODE_MEMBERSHIP)
        assert m[0].level == lvl
        assert np.array_equal(m[0].export(), refm[0])


def test_table_identification_at_working_level_deep():
    c, ctx, keys, T, q, oc, ok, qct, oq = setup("deep", 1)
    db = ctx.load_db(T)
    ref, lvl = ok.match(oq, T, c["ell"], c["n1"], fr.FR_MODE_IDENTIFY, 59, 0.5, level=8, schedule=1)
    out = ctx.match(db, qct, fr.FR_MODE_IDENTIFY)
    assert len(out) == len(ref)
    for g in range(len(ref)):
        assert out[g].level == lvl
        assert np.array_equal(out[g].export(), ref[g]), g


def test_auto_schedule_picks_by_rotation_count():
    """Auto (2): on demand while ell - n1 >= G (n2 - 1), the table beyond. tiny: ell = 64,
    n1 = 8, n2 = 8, N/2 = 2048 slots: G = 1 -> on demand; G = 9 -> table (56 < 63)."""
    c, ctx, keys, T, q, oc, ok, qct, oq = setup("tiny", 2)
    assert ctx.load_db(T).info()["schedule"] == 0
    T9 = W.templates(9 * 2048 - 100, c["ell"], W.DATASET_SEED + 77)
    db9 = ctx.load_db(T9)
    assert db9.info()["schedule"] == 1 and db9.info()["groups"] == 9
    out = ctx.match(db9, qct, fr.FR_MODE_SCORES)
    ref = ok.table_scores(oq, T9, c["ell"], c["n1"])
    assert len(out) == 9
    for g in range(9):
        assert np.array_equal(out[g].export(), ref[g]), g
