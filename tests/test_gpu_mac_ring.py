"""GPU parity of the persistent diagonal MAC (k_mac_ring, batches of 2 to 4 queries against one
database): at N = 2^13 with ell = 512 and n1 = 32 (n2 = 16 giant steps, the tiling the headline
uses), two template groups with a ragged tail, the scores of batches of 3, 4 and 6 queries (the
last split 4 + 2) and of one query (k_mac), with the baby steps in Q_l or in Q_l u P, bit-exact
against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu

C = dict(log_n=13, q_bits=[60] + [45] * 4, p_bits=[60, 60, 60], dnum=2, scale_bits=45, ell=512, n1=32,
         cheb_degree=0, threshold=0.5)
K = 5000


@pytest.fixture(scope="module")
def orc():
    oc = oracle.Ctx(C["log_n"], C["q_bits"], C["p_bits"], C["dnum"], C["scale_bits"])
    return oc, oc.keygen(0x5EED0A11)


def query(seed):
    rng = np.random.default_rng(seed)
    q = rng.standard_normal(C["ell"])
    return q / np.linalg.norm(q)


@pytest.mark.parametrize("pq", [0, 1], ids=["babies-Q", "babies-QP"])
def test_ring_mac_scores_match_oracle(orc, pq):
    oc, ok = orc
    ctx = fr.Context(device=0, hoist_babies=pq, **C)
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_SCORES), 0x5EED0A11)
    ctx.load_keys(keys)
    T = W.templates(K, C["ell"], 21)
    db = ctx.load_db(T)
    seeds = [700 + i for i in range(6)]
    qv = [query(s) for s in seeds]
    refs = []
    for q, s in zip(qv, seeds):
        oq = ok.encrypt(np.tile(q, oc.n // C["ell"]), s)
        refs.append(ok.bsgs_scores_pq(oq, T, C["ell"], C["n1"], pq=bool(pq)) if pq else
                    ok.bsgs_scores(oq, T, C["ell"], C["n1"]))
    cts = [ctx.encrypt(keys, q, s) for q, s in zip(qv, seeds)]
    out = ctx.match(db, cts[0], fr.FR_MODE_SCORES)
    assert all(np.array_equal(o.export(), r) for o, r in zip(out, refs[0])) and len(out) == len(refs[0])
    for nb in (3, 4, 6):
        outs = ctx.match_batch(db, cts[:nb], fr.FR_MODE_SCORES)
        for b in range(nb):
            assert len(outs[b]) == len(refs[b])
            for g, o in enumerate(outs[b]):
                assert np.array_equal(o.export(), refs[b][g]), (nb, b, g)
    s = T.astype(np.float64) @ qv[0]
    dec = np.concatenate([ctx.decrypt(keys, o) for o in out])[:K]
    assert np.abs(dec - s).max() < 1e-4
