"""GPU parity at every supported ring size (N = 2^10 .. 2^16; the paper's own ring is 2^15):
each NTT size has its own kernel instantiation and tile shape, so rotation, rescale, ct x ct
product and a two-group score match are checked bit for bit against the oracle at each size,
on a small prime chain (Q = 60/45/45, P = 60/60, one prime per digit)."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu

QB, PB, DNUM, SB = [60, 45, 45], [60, 60], 3, 45


@pytest.mark.parametrize("log_n", [10, 11, 14, 15, 16])
def test_ring_size_parity(log_n):
    ell, n1 = 64, 8
    ctx = fr.Context(device=0, log_n=log_n, q_bits=QB, p_bits=PB, dnum=DNUM, scale_bits=SB, ell=ell, n1=n1)
    n = ctx.n
    rots = sorted(set(ctx.required_rotations(fr.FR_MODE_SCORES)) | {5, n - 1})
    seed = 0x51E0 + log_n
    keys = ctx.keygen(rots, seed)
    ctx.load_keys(keys)
    oc = oracle.Ctx(log_n, QB, PB, DNUM, SB)
    ok = oc.keygen(seed)
    assert ctx.primes() == oc.primes
    rng = np.random.default_rng(log_n)
    z = rng.uniform(-1, 1, n)
    oq = ok.encrypt(z, 7)
    top = oc.top
    ct = ctx.import_ct(oq, top).upload()
    assert np.array_equal(ctx.encrypt_slots(keys, z, 7).export(), oq)
    for k in (1, 5, n - 1):
        assert np.array_equal(ctx.rotate(ct, k).export(), ok.rotate(oq, top, k)), k
    assert np.array_equal(ctx.rescale(ct).export(), oc.rescale(oq, top))
    ob = ok.encrypt(rng.uniform(-1, 1, n), 8)
    cb = ctx.import_ct(ob, top).upload()
    assert np.array_equal(ctx.mul_relin(ct, cb).export(), ok.mul_relin(oq, ob, top))
    # two template groups, the second ragged
    K = n + 37
    T = W.templates(K, ell, 0x7E00 + log_n)
    qv = rng.standard_normal(ell)
    qv /= np.linalg.norm(qv)
    db = ctx.load_db(T)
    got = ctx.match(db, ctx.encrypt(keys, qv, 9), fr.FR_MODE_SCORES)
    ref, lvl = ok.match(ok.encrypt(np.tile(qv, n // ell), 9), T, ell, n1, fr.FR_MODE_SCORES)
    assert len(got) == 2 == ref.shape[0]
    for g in range(2):
        assert got[g].level == lvl
        assert np.array_equal(got[g].export(), ref[g]), g
    s = np.concatenate([ctx.decrypt(keys, o) for o in got])
    assert np.abs(s[:K] - T.astype(np.float64) @ qv).max() < 1e-4


@pytest.mark.parametrize("pattern", ["max", "zero_max", "near_top"])
def test_extreme_residues(pattern):
    """Residues at the ends of their range (q - 1, 0, values just below q for the 60-bit
    primes) through the NTT, the key switch, the rescale and the ct x ct product: the lazy
    reductions must still land on the oracle's bits."""
    log_n = 12
    ctx = fr.Context(device=0, log_n=log_n, q_bits=QB, p_bits=PB, dnum=DNUM, scale_bits=SB, ell=64, n1=8)
    keys = ctx.keygen([1, 3], 0xED6E)
    ctx.load_keys(keys)
    oc = oracle.Ctx(log_n, QB, PB, DNUM, SB)
    ok = oc.keygen(0xED6E)
    N, top = oc.N, oc.top
    q = np.array(oc.primes[: top + 1], dtype=np.uint64)
    w = np.empty((2, top + 1, N), dtype=np.uint64)
    rng = np.random.default_rng(3)
    for i in range(top + 1):
        if pattern == "max":
            w[:, i] = q[i] - np.uint64(1)
        elif pattern == "zero_max":
            w[:, i] = np.where(rng.random((2, N)) < 0.5, np.uint64(0), q[i] - np.uint64(1))
        else:
            w[:, i] = q[i] - rng.integers(1, 1 << 10, (2, N)).astype(np.uint64)
    ct = ctx.import_ct(w, top).upload()
    assert np.array_equal(ct.export(), w)
    for k in (1, 3):
        assert np.array_equal(ctx.rotate(ct, k).export(), ok.rotate(w, top, k)), k
    assert np.array_equal(ctx.rescale(ct).export(), oc.rescale(w, top))
    assert np.array_equal(ctx.mul_relin(ct, ct).export(), ok.mul_relin(w, w, top))
