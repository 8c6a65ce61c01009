"""The membership match at full size in the configuration bench.py times: N = 2^16, 25 Q limbs +
4 P limbs, 6 digits, K = 2^15 templates of ell = 512, n1 = 32, degree-59 threshold, working level
8, baby steps kept in Q_l u P, giant steps sharing one ModDown per group, RotateAndSum in radix 4
with one ModDown per step.
The membership ciphertext must equal the oracle's match in the same configuration bit for bit, and
decrypt to the FP64 membership sum."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CFG = "membership"


def test_membership_bit_exact_in_bench_configuration():
    c = W.CONFIGS[CFG]
    ctx = fr.Context(device=0, hoist_babies=1, hoist_giants=1, sum_radix=4, hoist_sum=1,
                     **W.ctx_params(CFG, level_mode=1))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(CFG))
    ctx.load_keys(keys)
    T, q, _ = W.workload(CFG)
    db = ctx.load_db(T)
    qct = ctx.encrypt(keys, q, W.enc_seed(CFG))
    outs = [ctx.match(db, qct, fr.FR_MODE_MEMBERSHIP)[0] for _ in range(2)]   # eager, then the graph
    got = [o.export() for o in outs]
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed(CFG))
    oq = ok.encrypt(np.tile(q, oc.n // c["ell"]), W.enc_seed(CFG))
    ref, lvl = ok.match(oq, T, c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, c["cheb_degree"], c["threshold"],
                        level=ctx.work_level, sum_radix=4, hoist=True, babies_pq=True, hoist_sum=True)
    assert outs[0].level == lvl
    for g in got:
        assert np.array_equal(g, ref[0])
    s = T.astype(np.float64) @ q
    p = np.polynomial.chebyshev.chebval(s, fr.cheb_coeffs(c["cheb_degree"], c["threshold"]))
    assert abs(ctx.decrypt(keys, outs[0])[0] - p.sum()) < 1e-2
