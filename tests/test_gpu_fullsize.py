"""Full-size GPU checks at the headline parameters (N=2^16, 25 Q limbs + 4 P
limbs, 6 digits, K=2^15 templates of ell=512, n1=32, degree-59 threshold), in
the launch configuration bench.py times.

- scores ciphertext bit-exact against the oracle (the oracle computes the whole
  BSGS product: 31 hoisted baby rotations, 512 diagonal encodes, 15 giant
  rotations);
- membership and identification outputs decrypted against the FP64 reference
  (a property that holds at any size: |p(s) - decrypted| < 1e-2, decisions
  agree outside a 0.02 margin, membership sum within 1e-2).
"""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CFG = "membership"


@pytest.fixture(scope="module", params=[0, 1], ids=["full_chain", "working_level"])
def env(request):
    c = W.CONFIGS[CFG]
    ctx = fr.Context(device=0, **W.ctx_params(CFG, level_mode=request.param))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(CFG))
    ctx.load_keys(keys)
    T, q, planted = W.workload(CFG)
    db = ctx.load_db(T)
    qct = ctx.encrypt(keys, q, W.enc_seed(CFG))
    s = T.astype(np.float64) @ q
    p = np.polynomial.chebyshev.chebval(s, fr.cheb_coeffs(c["cheb_degree"], c["threshold"]))
    return dict(c=c, ctx=ctx, keys=keys, T=T, q=q, planted=planted, db=db, qct=qct, s=s, p=p,
                lq=ctx.work_level)


def test_scores_bit_exact_vs_oracle(env):
    c = env["c"]
    out = env["ctx"].match(env["db"], env["qct"], fr.FR_MODE_SCORES)
    got = out[0].export()
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed(CFG))
    oq = ok.encrypt(np.tile(env["q"], oc.n // c["ell"]), W.enc_seed(CFG))
    assert np.array_equal(env["qct"].export(), oq)
    lq = env["lq"]
    ref = ok.bsgs_scores(oc.drop(oq, oc.top, lq), env["T"], c["ell"], c["n1"], level=lq)
    assert np.array_equal(got, ref[0])
    dec = env["ctx"].decrypt(env["keys"], out[0])
    assert np.abs(dec - env["s"]).max() < 1e-4


def test_identification_decisions(env):
    out = env["ctx"].match(env["db"], env["qct"], fr.FR_MODE_IDENTIFY)
    assert len(out) == 1
    dec = env["ctx"].decrypt(env["keys"], out[0])
    s, p = env["s"], env["p"]
    assert np.abs(dec - p).max() < 1e-2
    far = np.abs(s - 0.5) > 0.02
    assert np.array_equal((dec >= 0.5)[far], (s >= 0.5)[far])
    found = np.nonzero(dec >= 0.5)[0]
    assert set(env["planted"]).issubset(set(found))


def test_membership_sum(env):
    out = env["ctx"].match(env["db"], env["qct"], fr.FR_MODE_MEMBERSHIP)
    assert len(out) == 1 and out[0].level == env["lq"] - 1 - 6
    dec = env["ctx"].decrypt(env["keys"], out[0])
    assert abs(dec[0] - env["p"].sum()) < 1e-2
    assert np.abs(dec - env["p"].sum()).max() < 1e-2


def test_repeat_is_deterministic(env):
    a = env["ctx"].match(env["db"], env["qct"], fr.FR_MODE_MEMBERSHIP)[0].export()
    b = env["ctx"].match(env["db"], env["qct"], fr.FR_MODE_MEMBERSHIP)[0].export()
    assert np.array_equal(a, b)
