"""Identification at full size: K=2^20 templates (32 groups of 2^15 slots), N=2^16 at the
working level, degree-59 threshold, diagonals encoded per query on the device (tier C).

Checks that hold at any size:
- every group's output ciphertext equals, bit for bit, the output of matching that group's
  2^15 templates alone (the groups share only the hoisted baby steps);
- every decrypted slot is within 1e-2 of the FP64 threshold polynomial of its score;
- decisions agree with (s >= 0.5) outside the 0.02 margin, and every planted duplicate is found.
The 2^15-template match itself is checked bit for bit against the oracle in
test_gpu_fullsize.py."""
import numpy as np
import pytest

from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    c = W.CONFIGS["identify"]
    ctx = fr.Context(device=0, db_tier=2, **W.ctx_params("identify", level_mode=1))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_IDENTIFY), W.key_seed("identify"))
    ctx.load_keys(keys)
    T, q, planted = W.workload("identify")
    db = ctx.load_db(T)
    qct = ctx.encrypt(keys, q, W.enc_seed("identify"))
    out = ctx.match(db, qct, fr.FR_MODE_IDENTIFY)
    return dict(c=c, ctx=ctx, keys=keys, T=T, q=q, planted=planted, db=db, qct=qct, out=out)


def test_tier_and_group_count(env):
    info = env["db"].info()
    assert info["tier"] == 2 and info["groups"] == 32 and len(env["out"]) == 32


@pytest.mark.parametrize("g", [0, 17, 31])
def test_group_equals_its_templates_alone(env, g):
    n = 1 << 15
    sub = env["ctx"].load_db(np.ascontiguousarray(env["T"][g * n:(g + 1) * n]))
    alone = env["ctx"].match(sub, env["qct"], fr.FR_MODE_IDENTIFY)
    assert len(alone) == 1
    assert np.array_equal(alone[0].export(), env["out"][g].export())


def test_decisions_over_all_slots(env):
    c, T, q = env["c"], env["T"], env["q"]
    s = T.astype(np.float64) @ q
    p = np.polynomial.chebyshev.chebval(s, fr.cheb_coeffs(c["cheb_degree"], c["threshold"]))
    dec = np.concatenate([env["ctx"].decrypt(env["keys"], o) for o in env["out"]])[: len(s)]
    assert np.abs(dec - p).max() < 1e-2
    far = np.abs(s - 0.5) > 0.02
    assert np.array_equal((dec >= 0.5)[far], (s >= 0.5)[far])
    assert set(env["planted"].tolist()).issubset(set(np.nonzero(dec >= 0.5)[0].tolist()))
