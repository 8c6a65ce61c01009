"""The hybrid comparator (comparator = 1; Section "HyDia": a Chebyshev approximation followed by
the fixed-degree polynomial f_4 of Cheon et al. 2020) on the GPU, through the C ABI, bit-exact
against the CPU oracle: the threshold alone, identification and membership at a mid size
(N = 2^13, 14 limbs, K = 5000 in two groups with a ragged tail), and the membership match at the
headline size (N = 2^16, K = 2^15, working level 12), whose decrypted value is the count of the
32 planted matches."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def f4_closed(y):
    from math import comb
    return sum(comb(2 * i, i) / 4.0 ** i * y * (1 - y * y) ** i for i in range(5))


def hybrid_fp64(s, n, tau):
    y = np.polynomial.chebyshev.chebval(s, fr.cheb_coeffs(n, tau, low=-1.0))
    return (1 + f4_closed(y)) / 2


class Env:
    def __init__(self, cfg):
        c = W.CONFIGS[cfg]
        self.c = c
        self.ctx = fr.Context(device=0, comparator=1, **W.ctx_params(cfg))
        self.keys = self.ctx.keygen(self.ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
        self.ctx.load_keys(self.keys)
        self.oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
        self.ok = self.oc.keygen(W.key_seed(cfg))
        self.T, self.q, self.planted = W.workload(cfg)
        self.qct = self.ctx.encrypt(self.keys, self.q, W.enc_seed(cfg))
        self.oq = self.ok.encrypt(np.tile(self.q, self.oc.n // c["ell"]), W.enc_seed(cfg))
        self.L = self.ctx.work_level
        self.db = self.ctx.load_db(self.T)


@pytest.fixture(scope="module")
def mid():
    return Env("mid_hybrid")


def test_hybrid_working_level(mid):
    d1, d2 = oracle.ps_split(59)
    assert mid.L == W.work_level("mid_hybrid", comparator=1) == 2 + d2 + 4


def test_hybrid_threshold_matches_oracle(mid):
    rng = np.random.default_rng(5)
    z = rng.uniform(-1, 1, mid.oc.n)
    lvl = mid.L - 1
    o = mid.oc.drop(mid.ok.encrypt(z, 44), mid.oc.top, lvl)
    ct = mid.ctx.import_ct(o, lvl).upload()
    out = mid.ctx.chebyshev(ct)
    assert out.level == lvl - 10
    ref = mid.ok.comparator_eval(o, lvl, 59, 0.5, 1)
    assert np.array_equal(out.export(), ref)
    assert np.abs(mid.ctx.decrypt(mid.keys, out) - hybrid_fp64(z, 59, 0.5)).max() < 1e-2


@pytest.mark.parametrize("mode", [fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_hybrid_match_matches_oracle(mid, mode):
    outs = [mid.ctx.match(mid.db, mid.qct, mode) for _ in range(2)]   # eager, then the graph
    ref, lvl = mid.ok.match(mid.oq, mid.T, mid.c["ell"], mid.c["n1"], mode, 59, 0.5, level=mid.L, comparator=1)
    assert outs[0][0].level == lvl == mid.L - 1 - 10
    for out in outs:
        assert len(out) == len(ref)
        for g in range(len(ref)):
            assert np.array_equal(out[g].export(), ref[g]), g
    K = len(mid.T)
    s = mid.T.astype(np.float64) @ mid.q
    n = mid.oc.n
    sp = np.zeros(((K + n - 1) // n) * n)
    sp[:K] = s
    h = hybrid_fp64(sp, 59, 0.5)
    if mode == fr.FR_MODE_MEMBERSHIP:
        m = mid.ctx.decrypt(mid.keys, outs[0][0])[0]
        assert abs(m - h.sum()) < 1e-2
        far = np.abs(s - 0.5) > 0.02
        assert np.all(far) and abs(m - (s >= 0.5).sum()) < 0.1
    else:
        dec = np.concatenate([mid.ctx.decrypt(mid.keys, o) for o in outs[0]])
        assert np.abs(dec - h).max() < 1e-2


def test_hybrid_membership_full_size_is_a_count():
    """Headline size with the hybrid comparator: bit-exact with the oracle; the decrypted sum is
    the number of planted matches (32) within 0.5, non-matches contributing almost nothing."""
    cfg = "membership"
    c = W.CONFIGS[cfg]
    ctx = fr.Context(device=0, comparator=1, hoist_giants=1, sum_radix=4, **W.ctx_params(cfg, level_mode=1))
    assert ctx.work_level == 12
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed(cfg))
    ctx.load_keys(keys)
    T, q, planted = W.workload(cfg)
    db = ctx.load_db(T)
    qct = ctx.encrypt(keys, q, W.enc_seed(cfg))
    outs = [ctx.match(db, qct, fr.FR_MODE_MEMBERSHIP)[0] for _ in range(2)]
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed(cfg))
    oq = ok.encrypt(np.tile(q, oc.n // c["ell"]), W.enc_seed(cfg))
    ref, lvl = ok.match(oq, T, c["ell"], c["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5, level=12, sum_radix=4, hoist=True,
                        comparator=1)
    assert outs[0].level == lvl == 1
    for o in outs:
        assert np.array_equal(o.export(), ref[0])
    m = ctx.decrypt(keys, outs[0])[0]
    s = T.astype(np.float64) @ q
    assert abs(m - hybrid_fp64(s, 59, 0.5).sum()) < 1e-2
    assert abs(m - len(planted)) < 0.5
