"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a printed
value of the paper (tests/golden), a published test vector, a closed form,
brute force on tiny inputs, or an invariant. All run on the CPU.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# config-1 parameters: N=2^12, Q = 60/40/40, P = 3 x 60 (reading R2), dnum = 1, Delta = 2^40
P1 = dict(log_n=12, q_bits=[60, 40, 40], p_bits=[60, 60, 60], dnum=1, scale_bits=40)


@pytest.fixture(scope="module")
def c1():
    return oracle.Ctx(**P1)


@pytest.fixture(scope="module")
def k1(c1):
    return c1.keygen(0xC0FFEE01)


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                key, val = line.split(None, 1)
                vals[key] = val.strip()
    return vals


def brev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2)


def rhaz(x):
    """round half away from zero"""
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


# ---------------------------------------------------------------------------
# generator of randomness: ChaCha20 (RFC 8439)
# ---------------------------------------------------------------------------
def test_chacha20_rfc8439_vector():
    g = read_golden("chacha20_rfc8439_block.txt")
    key = bytes.fromhex(g["key"])
    nonce = bytes.fromhex(g["nonce"])
    kw = np.frombuffer(key, dtype="<u4").astype(np.uint32)
    nw = np.frombuffer(nonce, dtype="<u4").astype(np.uint32)
    out = oracle.chacha20_block(kw, int(g["counter"]), nw)
    assert out.tobytes().hex() == g["block"]


def test_chacha20_matches_independent_library():
    crypt = pytest.importorskip("cryptography.hazmat.primitives.ciphers")
    rng = np.random.default_rng(5)
    for _ in range(4):
        key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
        nonce = rng.integers(0, 256, 12, dtype=np.uint8).tobytes()
        ctr = int(rng.integers(0, 2**31))
        enc = crypt.Cipher(crypt.algorithms.ChaCha20(key, ctr.to_bytes(4, "little") + nonce), mode=None).encryptor()
        ref = enc.update(bytes(64))
        out = oracle.chacha20_block(np.frombuffer(key, "<u4").astype(np.uint32), ctr,
                                    np.frombuffer(nonce, "<u4").astype(np.uint32))
        assert out.tobytes() == ref


def test_samplers_distributions():
    n = 1 << 15
    t = oracle.sample_ternary(11, 1, n)
    assert set(np.unique(t)) <= {-1, 0, 1}
    frac = [(t == v).mean() for v in (-1, 0, 1)]
    assert max(abs(f - 1 / 3) for f in frac) < 0.02
    e = oracle.sample_cbd(11, 3, n)
    assert np.abs(e).max() <= 21 and abs(e.mean()) < 0.1 and abs(e.var() - 10.5) < 0.6
    q = (1 << 50) - 1234567
    u = oracle.sample_uniform(11, 2, 4, q, n)
    assert u.max() < q and abs(u.astype(np.float64).mean() / q - 0.5) < 0.02
    # distinct objects / limbs give distinct streams
    assert not np.array_equal(u, oracle.sample_uniform(11, 2, 5, q, n))


# ---------------------------------------------------------------------------
# primes and roots (reading R1)
# ---------------------------------------------------------------------------
def test_primes_config1_and_config2():
    sympy = pytest.importorskip("sympy")
    for log_n, qb, pb in [(12, [60, 40, 40], [60, 60, 60]), (16, [60] + [50] * 24, [60] * 4)]:
        ps = oracle.gen_primes(log_n, qb + pb)
        M = 2 << log_n
        assert len(set(ps)) == len(ps)
        for p, b in zip(ps, qb + pb):
            assert sympy.isprime(p) and p % M == 1 and p.bit_length() == b
        # "largest-first per bit size": every prime = 1 mod 2N of that size above the
        # smallest chosen one is chosen, and they appear in descending order
        for b in set(qb + pb):
            chosen = [p for p, bb in zip(ps, qb + pb) if bb == b]
            assert chosen == sorted(chosen, reverse=True)
            c = ((1 << b) - 1) // M * M + 1
            above = []
            while c >= min(chosen):
                if sympy.isprime(c):
                    above.append(c)
                c -= M
            assert above == chosen


def test_psi_is_primitive_root_from_smallest_generator(c1):
    sympy = pytest.importorskip("sympy")
    N = c1.N
    for i, q in enumerate(c1.primes):
        psi = c1.psi(i)
        g = int(sympy.primitive_root(q))
        assert psi == pow(g, (q - 1) // (2 * N), q)
        assert pow(psi, N, q) == q - 1


# ---------------------------------------------------------------------------
# NTT: evaluation at psi^(2 brev(k) + 1), pinned by O(N^2) evaluation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("log_n", [3, 4, 6])
def test_ntt_is_evaluation_at_odd_powers(log_n):
    c = oracle.Ctx(log_n, [30], [31], 1, 20)
    N, q, psi = c.N, c.primes[0], c.psi(0)
    rng = np.random.default_rng(log_n)
    a = [int(x) for x in rng.integers(0, q, N)]
    A = c.ntt_fwd(0, np.array(a, dtype=np.uint64))
    for k in range(N):
        e = 2 * brev(k, log_n) + 1
        ref = sum(a[j] * pow(psi, e * j, q) for j in range(N)) % q
        assert int(A[k]) == ref
    assert [int(x) for x in c.ntt_inv(0, A)] == a


def test_ntt_negacyclic_convolution_schoolbook():
    log_n = 8
    c = oracle.Ctx(log_n, [40], [41], 1, 20)
    N, q = c.N, c.primes[0]
    rng = np.random.default_rng(3)
    a = [int(x) for x in rng.integers(0, q, N)]
    b = [int(x) for x in rng.integers(0, q, N)]
    ref = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                ref[k] = (ref[k] + a[i] * b[j]) % q
            else:
                ref[k - N] = (ref[k - N] - a[i] * b[j]) % q
    A = c.ntt_fwd(0, np.array(a, dtype=np.uint64))
    B = c.ntt_fwd(0, np.array(b, dtype=np.uint64))
    C = np.array([(int(x) * int(y)) % q for x, y in zip(A, B)], dtype=np.uint64)
    assert [int(x) for x in c.ntt_inv(0, C)] == ref


def test_automorphism_coef_and_eval_agree(c1):
    rng = np.random.default_rng(2)
    q = c1.primes[1]
    N = c1.N
    a = rng.integers(0, q, N).astype(np.uint64)
    for k in (1, 3, 17, -5):
        g = c1.galois(k)
        assert g == pow(5, k % (N // 2), 2 * N)
        # plain restatement of a(X) -> a(X^g)
        ref = np.zeros(N, dtype=object)
        for j in range(N):
            e = (j * g) % (2 * N)
            if e < N:
                ref[e] = int(a[j])
            else:
                ref[e - N] = (q - int(a[j])) % q
        got = c1.automorph_coef(g, 1, a)
        assert [int(x) for x in got] == list(ref)
        assert np.array_equal(c1.ntt_fwd(1, got), c1.automorph_eval(g, c1.ntt_fwd(1, a)))


# ---------------------------------------------------------------------------
# Encoding: inverse canonical embedding over the 5^j slot order (reading R5)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("log_n", [5, 8, 10])
def test_encode_matches_quadratic_definition(log_n):
    c = oracle.Ctx(log_n, [50], [51], 1, 40)
    N, n, M = c.N, c.N // 2, 2 * c.N
    rng = np.random.default_rng(log_n)
    z = rng.uniform(-1, 1, n)
    g = np.array([pow(5, j, M) for j in range(n)], dtype=np.int64)
    cc = np.arange(N, dtype=np.int64)
    ang = 2 * np.pi * ((g[:, None] * cc[None, :]) % M) / M
    m_def = (z[:, None] * np.cos(ang)).sum(axis=0) / n * 2.0 ** 40
    ref = rhaz(m_def)
    got = c.encode_coeffs(z).astype(np.float64)
    bad = np.nonzero(got != ref)[0]
    near_tie = np.abs(np.abs(m_def - np.trunc(m_def)) - 0.5) < 1e-2
    assert np.all(near_tie[bad]) and np.all(np.abs(got - ref) <= 1)
    assert len(bad) <= max(2, N // 256)


def test_encode_decode_round_trip(c1):
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, c1.n)
    m = c1.encode_coeffs(z)
    assert np.abs(c1.decode_coeffs(m, 2.0 ** 40) - z).max() < 1e-9


def test_galois_5k_is_left_rotation_of_slots(c1):
    """decode(sigma_{5^k}(encode(z))) = z rotated left by k (Eq. equ:diag's Rot_i direction)."""
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, c1.n)
    m = c1.encode_coeffs(z)
    N = c1.N
    for k in (1, 2, 7, 100):
        g = pow(5, k, 2 * N)
        out = np.zeros(N, dtype=np.int64)
        for j in range(N):
            e = (j * g) % (2 * N)
            if e < N:
                out[e] = m[j]
            else:
                out[e - N] = -m[j]
        assert np.abs(c1.decode_coeffs(out, 2.0 ** 40) - np.roll(z, -k)).max() < 1e-9


# ---------------------------------------------------------------------------
# Keys, encryption, key switching, rescale, products
# ---------------------------------------------------------------------------
def test_encrypt_decrypt(c1, k1):
    rng = np.random.default_rng(6)
    z = rng.uniform(-1, 1, c1.n)
    ct = k1.encrypt(z, 0xE0C00001)
    assert ct.shape == (2, 3, c1.N) and all(int(ct[:, i].max()) < c1.primes[i] for i in range(3))
    assert np.abs(k1.decrypt(ct, 2) - z).max() < 1e-6
    # same seed -> same ciphertext; other seed -> other ciphertext
    assert np.array_equal(ct, k1.encrypt(z, 0xE0C00001))
    assert not np.array_equal(ct, k1.encrypt(z, 0xE0C00002))


def _small_centered(v, q):
    v = int(v) % q
    return v - q if v > q // 2 else v


def test_evk_structure(c1, k1):
    """evk_d0 + evk_d1 * s = e_d + [P]_{q_i} s' on the digit's limbs (hybrid key switching key)."""
    s = k1.secret().astype(np.int64)
    N = c1.N
    g = c1.galois(3)
    evk = k1.make_evk(0, g)
    T = c1.nq + c1.np_
    P = 1
    for p in c1.primes[c1.nq:]:
        P *= p
    for d in range(c1.ndig):
        lo, hi = c1.dstart[d], c1.dstart[d + 1]
        for i in range(T):
            q = c1.primes[i]
            se = c1.ntt_fwd(i, (s % q).astype(np.uint64))
            sp = c1.automorph_eval(g, se)
            b = evk[d, 0, i].astype(object)
            a = evk[d, 1, i].astype(object)
            val = (b + a * se.astype(object)) % q
            if lo <= i < hi:
                val = (val - (P % q) * sp.astype(object)) % q
            e = c1.ntt_inv(i, np.array(val, dtype=np.uint64))
            ec = np.array([_small_centered(x, q) for x in e])
            assert np.abs(ec).max() <= 21


def test_rotation_decrypts_to_left_rotation(c1, k1):
    rng = np.random.default_rng(7)
    z = rng.uniform(-1, 1, c1.n)
    ct = k1.encrypt(z, 99)
    for k in (1, 5, 64, c1.n - 1):
        r = k1.rotate(ct, 2, k)
        assert np.abs(k1.decrypt(r, 2) - np.roll(z, -k)).max() < 1e-6
    ct1 = c1.drop(ct, 2, 1)
    assert np.abs(k1.decrypt(k1.rotate(ct1, 1, 9), 1) - np.roll(z, -9)).max() < 1e-6


def test_hoisted_equals_individual_rotations(c1, k1):
    rng = np.random.default_rng(8)
    ct = k1.encrypt(rng.uniform(-1, 1, c1.n), 5)
    ks = [0, 1, 2, 7]
    H = k1.hoisted_rotate(ct, 2, ks)
    for i, k in enumerate(ks):
        assert np.array_equal(H[i], k1.rotate(ct, 2, k))


def test_rescale_is_rounded_division_by_last_prime(c1):
    """Exact CRT check: output = (x - v) / q_l with v the centered residue mod q_l."""
    rng = np.random.default_rng(9)
    qs = c1.primes[:3]
    Q = qs[0] * qs[1] * qs[2]
    N = 64
    ct = np.zeros((2, 3, c1.N), dtype=np.uint64)
    xs = [int(v) for v in rng.integers(0, 2 ** 62, N)]
    xs = [(x * 977 + 12345) % Q for x in xs]
    for j, x in enumerate(xs):
        for i in range(3):
            ct[0, i, j] = x % qs[i]
            ct[1, i, j] = (x * 3) % qs[i]
    out = c1.rescale(ct, 2)
    ql = qs[2]
    for t, mult in ((0, 1), (1, 3)):
        for j, x0 in enumerate(xs):
            x = (x0 * mult) % Q
            v = x % ql
            v = v - ql if v > (ql - 1) // 2 else v
            y = (x - v) // ql
            assert (x - v) % ql == 0
            for i in range(2):
                assert int(out[t, i, j]) == y % qs[i]


def test_mul_relin_rescale(c1, k1):
    rng = np.random.default_rng(10)
    z1, z2 = rng.uniform(-1, 1, c1.n), rng.uniform(-1, 1, c1.n)
    a, b = k1.encrypt(z1, 1), k1.encrypt(z2, 2)
    m = c1.rescale(k1.mul_relin(a, b, 2), 2)
    assert np.abs(k1.decrypt(m, 1) - z1 * z2).max() < 1e-6


def test_rotate_sum_gives_total_in_every_slot(c1, k1):
    rng = np.random.default_rng(11)
    z = rng.uniform(-1, 1, c1.n) / c1.n
    ct = k1.encrypt(z, 3)
    steps = int(np.log2(c1.n))
    r = k1.rotate_sum(ct, 2, steps)
    assert np.abs(k1.decrypt(r, 2) - z.sum()).max() < 1e-5
    # radix r: hoisted rotations by t s, t < r, per step; the same total, other key-switch noise
    for radix in (4, 8, 32):
        rr = k1.rotate_sum(ct, 2, steps, radix=radix)
        assert np.abs(k1.decrypt(rr, 2) - z.sum()).max() < 1e-5
        assert not np.array_equal(rr, r)
    # one radix-4 step over 4 slots is x + Rot_1(x) + Rot_2(x) + Rot_3(x), hoisted rotations
    # being the individual ones (reading R6b)
    x = ct.copy()
    for t in (1, 2, 3):
        x = c1.add(x, k1.rotate(ct, 2, t), 2)
    assert np.array_equal(k1.rotate_sum(ct, 2, 2, radix=4), x)
    # partial sums: 8 slots in radix 4 = one radix-4 step (s = 1) and one radix-2 step (s = 4)
    y = k1.rotate_sum(ct, 2, 2, radix=4)
    y = c1.add(y, k1.rotate(y, 2, 4), 2)
    assert np.array_equal(k1.rotate_sum(ct, 2, 3, radix=4), y)


def test_rotate_sum_hoisted_one_moddown_per_step(c1, k1):
    """RotateAndSum with the rotations of each step summed before one ModDown: the total in
    every slot; with one rotation per step (radix 2) the radix-2 form bit for bit; the steps
    are those of the radix form (a radix-4 step over 4 slots, then a plain rotation by 4)."""
    rng = np.random.default_rng(12)
    z = rng.uniform(-1, 1, c1.n) / c1.n
    ct = k1.encrypt(z, 5)
    steps = int(np.log2(c1.n))
    assert np.array_equal(k1.rotate_sum(ct, 2, steps, radix=2, hoist=True), k1.rotate_sum(ct, 2, steps))
    for radix in (4, 8, 32):
        h = k1.rotate_sum(ct, 2, steps, radix=radix, hoist=True)
        plain = k1.rotate_sum(ct, 2, steps, radix=radix)
        assert np.abs(k1.decrypt(h, 2) - z.sum()).max() < 1e-5
        assert not np.array_equal(h, plain)
        # the ModDown of a sum and the sum of the ModDowns differ by key-switch rounding only
        assert np.abs(k1.decrypt(h, 2) - k1.decrypt(plain, 2)).max() < 1e-5
    y = k1.rotate_sum(ct, 2, 2, radix=4, hoist=True)
    y = c1.add(y, k1.rotate(y, 2, 4), 2)
    assert np.array_equal(k1.rotate_sum(ct, 2, 3, radix=4, hoist=True), y)


# ---------------------------------------------------------------------------
# Matrix-vector product: diagonal method and BSGS (Eq. equ:diag, Eq. equ:diagbsgs-grouped,
# Eq. eq:prerotation), checked against the FP64 matvec and against each other
# ---------------------------------------------------------------------------
def _templates(K, ell, seed):
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((K, ell))
    T /= np.linalg.norm(T, axis=1, keepdims=True)
    return T.astype(np.float32)


def test_diag_slots_is_hydia_packing():
    ell, slots = 8, 32
    T = _templates(50, ell, 1)
    for k, d, shift in [(0, 0, 0), (0, 3, 0), (1, 5, 16), (0, 7, 8)]:
        z = oracle.diag_slots(T, ell, slots, k, d, shift)
        for x in range(slots):
            y = (x - shift) % slots
            b, r = divmod(y, ell)
            row = (k * (slots // ell) + b) * ell + r
            ref = T[row, (r + d) % ell] if row < len(T) else 0.0
            assert z[x] == np.float64(ref)


def test_bsgs_and_diagonal_match_plain_matvec(c1, k1):
    K, ell = 64, 64
    T = _templates(K, ell, 0xF00D0001)
    rng = np.random.default_rng(12)
    q = T[0].astype(np.float64) + 0.1 * rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k1.encrypt(np.tile(q, c1.n // ell), 13)
    ref = T.astype(np.float64) @ q
    for n1 in (8, 5, 64):
        S = k1.bsgs_scores(qct, T, ell, n1)
        got = k1.decrypt(S[0], 1)
        assert np.abs(got[:K] - ref).max() < 1e-4
        assert np.abs(got[K:]).max() < 1e-4        # padding rows score 0
    D = k1.diag_scores(qct, T, ell)
    assert np.abs(k1.decrypt(D[0], 1)[:K] - ref).max() < 1e-4
    # n1 = l is HyDia-DG (no giant steps): the same computation as the naive diagonal method
    assert np.array_equal(k1.bsgs_scores(qct, T, ell, ell), D)


def test_bsgs_special_cases(c1, k1):
    ell = 32
    T = _templates(200, ell, 3)
    # one-hot query picks column c of the templates
    for col in (0, 5, 31):
        q = np.zeros(ell)
        q[col] = 1.0
        qct = k1.encrypt(np.tile(q, c1.n // ell), 40 + col)
        got = k1.decrypt(k1.bsgs_scores(qct, T, ell, 4)[0], 1)
        assert np.abs(got[:200] - T[:, col]).max() < 1e-4
    # K = l: one square, the textbook diagonal method of Eq. equ:diag
    Tsq = _templates(ell, ell, 4)
    q = np.linalg.norm(Tsq[1]) * Tsq[1].astype(np.float64)
    qct = k1.encrypt(np.tile(q, c1.n // ell), 7)
    got = k1.decrypt(k1.bsgs_scores(qct, Tsq, ell, 8)[0], 1)
    assert np.abs(got[:ell] - Tsq.astype(np.float64) @ q).max() < 1e-4


def test_giant_steps_with_one_moddown(c1, k1):
    """Double hoisting of the giant steps (one ModDown per group over the summed inner
    products): the FP64 matvec again; with a single giant rotation (n2 = 2) it is the rotation
    itself, bit for bit; with more, other bits (ModDown is linear only up to its rounding)."""
    K, ell = 64, 64
    T = _templates(K, ell, 0xF00D0009)
    rng = np.random.default_rng(22)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k1.encrypt(np.tile(q, c1.n // ell), 24)
    ref = T.astype(np.float64) @ q
    for n1 in (8, 5):
        S = k1.bsgs_scores(qct, T, ell, n1, hoist=True)
        got = k1.decrypt(S[0], 1)
        assert np.abs(got[:K] - ref).max() < 1e-4 and np.abs(got[K:]).max() < 1e-4
        assert not np.array_equal(S, k1.bsgs_scores(qct, T, ell, n1))
    assert np.array_equal(k1.bsgs_scores(qct, T, ell, 32, hoist=True), k1.bsgs_scores(qct, T, ell, 32))
    assert np.array_equal(k1.bsgs_scores(qct, T, ell, 64, hoist=True), k1.bsgs_scores(qct, T, ell, 64))


def test_baby_steps_in_extended_basis(c1, k1):
    """Baby steps kept in Q_l u P, one ModDown per giant step (double hoisting of the baby steps):
    the FP64 matvec again, with and without the giant steps sharing one ModDown; with n1 = 1 the
    only baby is P q, whose ModDown is q exactly, so the scores equal the plain schedule bit for
    bit; with more babies the bits differ (ModDown is linear only up to its rounding)."""
    K, ell = 64, 64
    T = _templates(K, ell, 0xF00D000A)
    rng = np.random.default_rng(23)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k1.encrypt(np.tile(q, c1.n // ell), 25)
    ref = T.astype(np.float64) @ q
    for n1 in (8, 5, 64):
        for hoist in (False, True):
            S = k1.bsgs_scores_pq(qct, T, ell, n1, hoist=hoist)
            got = k1.decrypt(S[0], 1)
            assert np.abs(got[:K] - ref).max() < 1e-4 and np.abs(got[K:]).max() < 1e-4
            assert not np.array_equal(S, k1.bsgs_scores(qct, T, ell, n1, hoist=hoist))
    assert np.array_equal(k1.bsgs_scores_pq(qct, T, ell, 1), k1.bsgs_scores(qct, T, ell, 1))
    assert np.array_equal(k1.bsgs_scores_pq(qct, T, ell, 8, pq=False), k1.bsgs_scores(qct, T, ell, 8))


def test_table_schedule_matches_plain_matvec(c1, k1):
    """Algorithm 1 (rotated-query table): decrypts to the FP64 matvec for any n1; with
    n1 = l (babies only) or n1 = 1 (giant rotations of q only) every table entry is one
    hoisted rotation of q, so the scores are bit-identical to the naive diagonal method."""
    K, ell = 64, 64
    T = _templates(K, ell, 0xF00D0007)
    rng = np.random.default_rng(21)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k1.encrypt(np.tile(q, c1.n // ell), 23)
    ref = T.astype(np.float64) @ q
    for n1 in (8, 5):
        S = k1.table_scores(qct, T, ell, n1)
        got = k1.decrypt(S[0], 1)
        assert np.abs(got[:K] - ref).max() < 1e-4
        assert np.abs(got[K:]).max() < 1e-4
        # a different composition of rotations than the on-demand schedule: same values, other noise
        assert not np.array_equal(S, k1.bsgs_scores(qct, T, ell, n1))
    D = k1.diag_scores(qct, T, ell)
    assert np.array_equal(k1.table_scores(qct, T, ell, ell), D)
    assert np.array_equal(k1.table_scores(qct, T, ell, 1), D)


def test_table_schedule_multi_group():
    c = oracle.Ctx(10, [60, 40, 40], [60, 60, 60], 1, 40)
    k = c.keygen(78)
    ell = 16
    K = 2 * c.n + 37
    T = _templates(K, ell, 6)
    rng = np.random.default_rng(1)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k.encrypt(np.tile(q, c.n // ell), 3)
    S = k.table_scores(qct, T, ell, 4)
    assert S.shape[0] == 3
    ref = T.astype(np.float64) @ q
    got = np.concatenate([k.decrypt(S[g], 1) for g in range(3)])
    assert np.abs(got[:K] - ref).max() < 1e-4 and np.abs(got[K:]).max() < 1e-4


def test_multi_group_packing():
    """K > numSlots: G = ceil(K / numSlots) groups (Fig. 1), score of row t in slot t mod numSlots of group t div numSlots."""
    c = oracle.Ctx(10, [60, 40, 40], [60, 60, 60], 1, 40)
    k = c.keygen(77)
    ell = 16
    K = 2 * c.n + 100
    T = _templates(K, ell, 5)
    rng = np.random.default_rng(0)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k.encrypt(np.tile(q, c.n // ell), 2)
    S = k.bsgs_scores(qct, T, ell, 4)
    assert S.shape[0] == 3
    ref = T.astype(np.float64) @ q
    got = np.concatenate([k.decrypt(S[g], 1) for g in range(3)])
    assert np.abs(got[:K] - ref).max() < 1e-4 and np.abs(got[K:]).max() < 1e-4
    Sh = k.bsgs_scores(qct, T, ell, 4, hoist=True)       # one ModDown per group
    got = np.concatenate([k.decrypt(Sh[g], 1) for g in range(3)])
    assert np.abs(got[:K] - ref).max() < 1e-4 and np.abs(got[K:]).max() < 1e-4


# ---------------------------------------------------------------------------
# Chebyshev threshold (Eq. eq:cheb-sign, Paterson-Stockmeyer paragraph)
# ---------------------------------------------------------------------------
def test_ps_split_printed_values():
    g = read_golden("paper_counts.txt")
    assert oracle.ps_split(13) == (int(g["ps_d1_n13"]), int(g["ps_d2_n13"]))
    assert oracle.ps_split(59) == (2, 6)
    assert oracle.ps_split(27) == (2, 5)
    # rule itself: minimal d1 + d2 with d1 * 2^(d2-1) >= n, ties to larger d1
    for n in range(2, 130):
        d1, d2 = oracle.ps_split(n)
        assert d1 * 2 ** (d2 - 1) >= n
        for a in range(1, n + 2):
            for b in range(1, 12):
                if a * 2 ** (b - 1) >= n:
                    assert a + b > d1 + d2 or (a + b == d1 + d2 and a <= d1)


@pytest.mark.parametrize("n", [13, 27, 59])
def test_chebyshev_coefficients_interpolate_step(n):
    tau = 0.5
    cf = oracle.cheb_coeffs(n, tau)
    theta = np.pi * (np.arange(n + 1) + 0.5) / (n + 1)
    xj = np.cos(theta)
    fj = (xj >= tau).astype(np.float64)
    # interpolation property: p(x_j) = f(x_j) at the n+1 Chebyshev nodes
    V = np.cos(np.outer(np.arange(n + 1) * 1.0, theta)).T
    assert np.abs(V @ cf - fj).max() < 1e-12
    # PS recursion (Chebyshev division) == closed form == Clenshaw on a grid
    d1, d2 = oracle.ps_split(n)
    pad = np.zeros(d1 * 2 ** (d2 - 1))
    pad[: n + 1] = cf
    xs = np.linspace(-1, 1, 41)
    closed = np.array([np.sum(cf * np.cos(np.arange(n + 1) * np.arccos(x))) for x in xs])
    clen = np.polynomial.chebyshev.chebval(xs, cf)
    ps = np.array([oracle.cheb_ps_eval_fp64(pad, x) for x in xs])
    assert np.abs(closed - clen).max() < 1e-12 and np.abs(ps - clen).max() < 1e-12


def test_chebyshev_decision_margin():
    """(p(s) >= 0.5) == (s >= 0.5) for |s - 0.5| > 0.02 at degree 59 (reading R12)."""
    cf = oracle.cheb_coeffs(59, 0.5)
    xs = np.linspace(-1, 1, 200001)
    p = np.polynomial.chebyshev.chebval(xs, cf)
    far = np.abs(xs - 0.5) > 0.02
    assert np.all((p[far] >= 0.5) == (xs[far] >= 0.5))


def test_homomorphic_chebyshev_matches_fp64():
    c = oracle.Ctx(11, [60] + [40] * 8, [60, 60, 60], 3, 40)
    k = c.keygen(21)
    rng = np.random.default_rng(13)
    z = rng.uniform(-1, 1, c.n)
    ct = k.encrypt(z, 4)
    for n in (13, 59):
        d1, d2 = oracle.ps_split(n)
        out = k.cheb_eval(ct, c.top, n, 0.5)
        got = k.decrypt(out, c.top - d2)
        ref = np.polynomial.chebyshev.chebval(z, oracle.cheb_coeffs(n, 0.5))
        assert np.abs(got - ref).max() < 1e-3, n


# ---------------------------------------------------------------------------
# Hybrid comparator (Section "HyDia": lower-depth Chebyshev + Cheon et al. 2020's fixed
# polynomial; reading R27)
# ---------------------------------------------------------------------------
def f4_closed(y):
    """f_4(y) = sum_{i=0}^{4} C(2i, i) 4^-i y (1 - y^2)^i (Cheon, Kim, Kim 2020), the closed form."""
    from math import comb
    return sum(comb(2 * i, i) / 4.0 ** i * y * (1 - y * y) ** i for i in range(5))


def test_f4_closed_form_properties():
    """f_4 is odd, f_4(+-1) = +-1, f_4'(y) = (315/128)(1 - y^2)^4, and |f_4| <= 1 on [-1, 1]."""
    ys = np.linspace(-1, 1, 2001)
    assert np.abs(f4_closed(-ys) + f4_closed(ys)).max() < 1e-14
    assert abs(f4_closed(1.0) - 1.0) < 1e-15
    h = 1e-6
    d = (f4_closed(ys[1:-1] + h) - f4_closed(ys[1:-1] - h)) / (2 * h)
    assert np.abs(d - 315.0 / 128.0 * (1 - ys[1:-1] ** 2) ** 4).max() < 1e-7
    assert np.abs(f4_closed(ys)).max() <= 1.0 + 1e-15


def test_sign_interpolant_is_twice_step_minus_one():
    """The sign(x - tau) interpolant is 2 (step interpolant) - T_0, since the interpolation is
    linear in the sampled function; and it interpolates sign at the nodes."""
    for n in (13, 59):
        st = oracle.cheb_coeffs(n, 0.5)
        sg = oracle.cheb_coeffs(n, 0.5, low=-1.0)
        ref = 2 * st
        ref[0] -= 1.0
        assert np.abs(sg - ref).max() < 1e-12
        theta = np.pi * (np.arange(n + 1) + 0.5) / (n + 1)
        xj = np.cos(theta)
        assert np.abs(np.polynomial.chebyshev.chebval(xj, sg) - np.where(xj >= 0.5, 1.0, -1.0)).max() < 1e-11


def test_homomorphic_f4_matches_closed_form():
    c = oracle.Ctx(11, [60] + [40] * 8, [60, 60, 60], 3, 40)
    k = c.keygen(23)
    rng = np.random.default_rng(17)
    z = rng.uniform(-1.02, 1.02, c.n)
    ct = k.encrypt(z, 6)
    out = k.f4_eval(ct, c.top)
    got = k.decrypt(out, c.top - 4)
    assert np.abs(got - (1 + f4_closed(z)) / 2).max() < 1e-4


def test_homomorphic_hybrid_comparator_matches_fp64_and_depth():
    c = oracle.Ctx(11, [60] + [40] * 9, [60, 60, 60], 4, 40)
    k = c.keygen(29)
    rng = np.random.default_rng(19)
    z = rng.uniform(-1, 1, c.n)
    ct = k.encrypt(z, 7)
    n = 13
    d1, d2 = oracle.ps_split(n)
    out = k.comparator_eval(ct, c.top, n, 0.5, 1)
    assert out.shape[1] == c.top - d2 - 4 + 1
    y = np.polynomial.chebyshev.chebval(z, oracle.cheb_coeffs(n, 0.5, low=-1.0))
    got = k.decrypt(out, c.top - d2 - 4)
    assert np.abs(got - (1 + f4_closed(y)) / 2).max() < 1e-3
    # comparator 0 is the plain Chebyshev evaluation, bit for bit
    assert np.array_equal(k.comparator_eval(ct, c.top, n, 0.5, 0), k.cheb_eval(ct, c.top, n, 0.5))


def test_hybrid_comparator_makes_membership_a_count():
    """On the headline workload's FP64 scores (K = 2^15, 32 planted at cosine 0.8), the hybrid's
    per-slot values sum to the number of matches within 0.5 (non-matches contribute < 0.5 in
    all), where the plain degree-59 step interpolant adds about 12.8; decisions agree outside
    the 0.02 margin and the error there is below 0.015 (reading R27)."""
    from paper_2604_00546_gb300 import workloads as W
    T, q, planted = W.workload("membership")
    s = T.astype(np.float64) @ q
    sg = oracle.cheb_coeffs(59, 0.5, low=-1.0)
    h = (1 + f4_closed(np.polynomial.chebyshev.chebval(s, sg))) / 2
    match = s >= 0.5
    assert match.sum() == len(planted)
    assert abs(h[~match].sum()) < 0.5 and abs(h.sum() - len(planted)) < 0.5
    plain = np.polynomial.chebyshev.chebval(s, oracle.cheb_coeffs(59, 0.5))
    assert plain[~match].sum() > 10
    xs = np.linspace(-1, 1, 200001)
    hx = (1 + f4_closed(np.polynomial.chebyshev.chebval(xs, sg))) / 2
    far = np.abs(xs - 0.5) > 0.02
    assert np.all((hx[far] >= 0.5) == (xs[far] >= 0.5))
    assert np.abs(hx[far] - (xs[far] >= 0.5)).max() < 0.015


# ---------------------------------------------------------------------------
# Full pipeline, small: identification and membership (Algorithms 5 and 6)
# ---------------------------------------------------------------------------
def test_match_modes_small():
    c = oracle.Ctx(11, [60] + [40] * 8, [60, 60, 60], 3, 40)
    k = c.keygen(31)
    ell = 32
    K = 700
    T = _templates(K, ell, 7)
    q = T[3].astype(np.float64)
    # plant near-duplicates at cosine 0.8
    rng = np.random.default_rng(14)
    for idx in (10, 200, 650):
        u = rng.standard_normal(ell)
        u -= (u @ q) * q
        u /= np.linalg.norm(u)
        T[idx] = (0.8 * q + 0.6 * u).astype(np.float32)
    qct = k.encrypt(np.tile(q, c.n // ell), 9)
    s = T.astype(np.float64) @ q
    cf = oracle.cheb_coeffs(59, 0.5)
    p = np.polynomial.chebyshev.chebval(np.concatenate([s, np.zeros(c.n - K)]), cf)
    ident, lvl = k.match(qct, T, ell, 4, oracle.MODE_IDENTIFY, 59, 0.5)
    assert lvl == c.top - 1 - 6
    got = k.decrypt(ident[0], lvl)
    assert np.abs(got - p).max() < 1e-2
    far = np.abs(s - 0.5) > 0.02
    assert np.array_equal((got[:K] >= 0.5)[far], (s >= 0.5)[far])
    memb, lvl2 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5)
    m = k.decrypt(memb[0], lvl2)
    assert abs(m[0] - p.sum()) < 1e-2 and np.abs(m - p.sum()).max() < 1e-2
    # the table schedule (Algorithm 1) feeds the same threshold and sum
    memt, lvl3 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5, schedule=1)
    assert lvl3 == lvl2
    mt = k.decrypt(memt[0], lvl3)
    assert np.abs(mt - p.sum()).max() < 1e-2
    # RotateAndSum in radix 8 (hoisted rotations per step): the same sum
    memr, lvl4 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5, sum_radix=8)
    assert lvl4 == lvl2 and not np.array_equal(memr, memb)
    assert np.abs(k.decrypt(memr[0], lvl4) - p.sum()).max() < 1e-2
    # giant steps sharing one ModDown per group: the same sum
    memh, lvl5 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5, hoist=True)
    assert lvl5 == lvl2 and not np.array_equal(memh, memb)
    assert np.abs(k.decrypt(memh[0], lvl5) - p.sum()).max() < 1e-2
    # baby steps kept in Q_l u P: the same sum
    memq, lvl6 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5, hoist=True, babies_pq=True)
    assert lvl6 == lvl2 and not np.array_equal(memq, memh)
    assert np.abs(k.decrypt(memq[0], lvl6) - p.sum()).max() < 1e-2
    # RotateAndSum steps sharing one ModDown: the same sum
    mems, lvl7 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5, sum_radix=8, hoist_sum=True)
    assert lvl7 == lvl2 and not np.array_equal(mems, memr)
    assert np.abs(k.decrypt(mems[0], lvl7) - p.sum()).max() < 1e-2


def test_match_hybrid_comparator_small():
    """The hybrid comparator in the match: 4 more levels, each slot (1 + f_4(p_sign(s))) / 2,
    and the membership sum is the count of the rows at or above the threshold."""
    c = oracle.Ctx(11, [60] + [40] * 12, [60, 60, 60], 4, 40)
    k = c.keygen(37)
    ell, K = 32, 700
    T = _templates(K, ell, 9)
    q = T[5].astype(np.float64)
    rng = np.random.default_rng(16)
    for idx in (11, 300, 640):
        u = rng.standard_normal(ell)
        u -= (u @ q) * q
        u /= np.linalg.norm(u)
        T[idx] = (0.8 * q + 0.6 * u).astype(np.float32)
    T[5] = (0.3 * q + np.sqrt(1 - 0.09) * u).astype(np.float32)   # the query's own row off the threshold
    qct = k.encrypt(np.tile(q, c.n // ell), 10)
    s = np.concatenate([T.astype(np.float64) @ q, np.zeros(c.n - K)])
    y = np.polynomial.chebyshev.chebval(s, oracle.cheb_coeffs(59, 0.5, low=-1.0))
    h = (1 + f4_closed(y)) / 2
    lq = 12
    ident, lvl = k.match(qct, T, ell, 4, oracle.MODE_IDENTIFY, 59, 0.5, level=lq, comparator=1)
    assert lvl == lq - 1 - 6 - 4
    assert np.abs(k.decrypt(ident[0], lvl) - h).max() < 1e-2
    memb, lvl2 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5, level=lq, comparator=1)
    assert lvl2 == lvl
    m = k.decrypt(memb[0], lvl2)
    # at ell = 32 some random rows also score above 0.5; no score falls inside the margin, so
    # the sum is the count of rows at or above the threshold
    assert np.all(np.abs(s - 0.5) > 0.02)
    assert abs(m[0] - h.sum()) < 1e-2 and abs(m[0] - (s >= 0.5).sum()) < 0.05


# ---------------------------------------------------------------------------
# Decryption range and the working level
# ---------------------------------------------------------------------------
def test_decrypt_crt_two_limbs_beyond_first_prime():
    """Values above q0 / (2 Delta) decrypt exactly from limbs 0 and 1 (centered CRT)."""
    c = oracle.Ctx(10, [40, 40, 40], [60, 60], 1, 30)
    k = c.keygen(3)
    rng = np.random.default_rng(2)
    z = 2500.0 + rng.uniform(-1, 1, c.n)     # constant term 2500 Delta > q0 / 2
    ct = k.encrypt(z, 4)
    assert np.abs(k.decrypt(ct, 2) - z).max() < 1e-4
    assert np.abs(k.decrypt(c.drop(ct, 2, 1), 1) - z).max() < 1e-4
    assert np.abs(k.decrypt(c.drop(ct, 2, 0), 0) - z).max() > 100      # one limb wraps


def test_match_at_working_level_consistent():
    c = oracle.Ctx(11, [60] + [40] * 10, [60, 60, 60], 4, 40)
    k = c.keygen(41)
    ell, K = 32, 900
    T = _templates(K, ell, 8)
    rng = np.random.default_rng(15)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k.encrypt(np.tile(q, c.n // ell), 5)
    lq = 8
    out, lvl = k.match(qct, T, ell, 4, oracle.MODE_SCORES, 59, 0.5, level=lq)
    assert lvl == lq - 1
    ref = k.bsgs_scores(c.drop(qct, c.top, lq), T, ell, 4, level=lq)
    assert np.array_equal(out, ref)
    assert np.abs(k.decrypt(out[0], lvl)[:K] - T.astype(np.float64) @ q).max() < 1e-4
    memb, lvl2 = k.match(qct, T, ell, 4, oracle.MODE_MEMBERSHIP, 59, 0.5, level=lq)
    assert lvl2 == 1
    s = np.concatenate([T.astype(np.float64) @ q, np.zeros(c.n - K)])
    p = np.polynomial.chebyshev.chebval(s, oracle.cheb_coeffs(59, 0.5))
    assert abs(k.decrypt(memb[0], 1)[0] - p.sum()) < 1e-2


# ---------------------------------------------------------------------------
# Encrypted database (enroller-side pre-rotation, Section 5.3.3; lazy relinearisation)
# ---------------------------------------------------------------------------
def test_encrypted_db_decrypts_to_prerotated_diagonals():
    """Enrollment: each ciphertext decrypts to its diagonal rotated by -j n1 slots (Eq.
    eq:prerotation applied to the plaintext), read straight from the templates."""
    c = oracle.Ctx(10, [60, 40, 40], [60, 60, 60], 1, 40)
    k = c.keygen(90)
    ell, n1, K = 16, 4, c.n + 70           # two groups, the second ragged
    T = _templates(K, ell, 9)
    E = k.encrypt_db(T, ell, n1, 500, level=1)
    assert E.shape == (2, ell, 2, 2, c.N)
    B = c.n // ell
    for g, d in [(0, 0), (0, 5), (1, 11), (1, 15)]:
        z = k.decrypt(E[g, d], 1)
        shift = (d // n1) * n1
        for x in range(0, c.n, 37):
            y = (x - shift) % c.n
            b, r = divmod(y, ell)
            row = (g * B + b) * ell + r
            ref = float(T[row, (r + d) % ell]) if row < K else 0.0
            assert abs(z[x] - ref) < 1e-6
    # the enroller encrypts at the top level and drops limbs: the low limbs are the top-level ones
    top = k.encrypt_db(T[:c.n], ell, n1, 500)
    assert np.array_equal(c.drop(top[0, 7], c.top, 1), E[0, 7])


def test_encrypted_db_trivial_encryption_is_plaintext_path():
    """With trivial encryptions (m, 0) of the pre-rotated diagonals, the c1 parts of the
    tensor products and d2 vanish, the relinearisation adds KS(0) = 0, and the encrypted-database
    scores equal the plaintext-database scores bit for bit."""
    c = oracle.Ctx(10, [60, 40, 40], [60, 60, 60], 1, 40)
    k = c.keygen(91)
    ell, n1, K = 16, 4, c.n + 70
    T = _templates(K, ell, 10)
    rng = np.random.default_rng(3)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k.encrypt(np.tile(q, c.n // ell), 6)
    G = 2
    E = np.zeros((G, ell, 2, c.top + 1, c.N), dtype=np.uint64)
    for g in range(G):
        for d in range(ell):
            E[g, d, 0] = c.encode(oracle.diag_slots(T, ell, c.n, g, d, (d // n1) * n1))
    got = k.enc_scores(qct, E, n1)
    assert np.array_equal(got, k.bsgs_scores(qct, T, ell, n1))
    # the same with the giant steps sharing one ModDown
    assert np.array_equal(k.enc_scores(qct, E, n1, hoist=True), k.bsgs_scores(qct, T, ell, n1, hoist=True))


def test_encrypted_db_scores_and_match():
    """Real encryptions: scores decrypt to the FP64 inner products; the threshold and the
    membership sum follow them as in the plaintext-database match."""
    c = oracle.Ctx(11, [60] + [40] * 8, [60, 60, 60], 3, 40)
    k = c.keygen(92)
    ell, n1, K = 32, 4, 700
    T = _templates(K, ell, 11)
    q = T[3].astype(np.float64)
    rng = np.random.default_rng(16)
    for idx in (10, 650):
        u = rng.standard_normal(ell)
        u -= (u @ q) * q
        u /= np.linalg.norm(u)
        T[idx] = (0.8 * q + 0.6 * u).astype(np.float32)
    qct = k.encrypt(np.tile(q, c.n // ell), 9)
    lq = 7
    E = k.encrypt_db(T, ell, n1, 600, level=lq)
    s = T.astype(np.float64) @ q
    S, lvl = k.match_enc(qct, E, K, n1, oracle.MODE_SCORES, level=lq)
    assert lvl == lq - 1
    got = k.decrypt(S[0], lvl)
    assert np.abs(got[:K] - s).max() < 1e-4 and np.abs(got[K:]).max() < 1e-4
    # not the plaintext path's bits (another product), the same values
    Sp, _ = k.match(qct, T, ell, n1, oracle.MODE_SCORES, level=lq)
    assert not np.array_equal(S, Sp)
    p = np.polynomial.chebyshev.chebval(np.concatenate([s, np.zeros(c.n - K)]), oracle.cheb_coeffs(59, 0.5))
    ident, l1 = k.match_enc(qct, E, K, n1, oracle.MODE_IDENTIFY, level=lq)
    assert l1 == lq - 1 - 6
    gi = k.decrypt(ident[0], l1)
    assert np.abs(gi - p).max() < 1e-2
    far = np.abs(s - 0.5) > 0.02
    assert np.array_equal((gi[:K] >= 0.5)[far], (s >= 0.5)[far])
    memb, l2 = k.match_enc(qct, E, K, n1, oracle.MODE_MEMBERSHIP, level=lq)
    assert l2 == l1
    assert np.abs(k.decrypt(memb[0], l2) - p.sum()).max() < 1e-2


def test_server_prerotation_of_encrypted_diagonals():
    """Server-side pre-rotation (the GPU variant of Section 5.3 that rotates encrypted diagonals
    at load with negative giant-step keys): the rotated ciphertexts decrypt to the same
    pre-rotated diagonals the enroller variant encrypts, and the match decrypts to the FP64
    inner products; the bits differ from the enroller variant (key-switch noise)."""
    c = oracle.Ctx(10, [60, 40, 40], [60, 60, 60], 1, 40)
    k = c.keygen(93)
    ell, n1, K = 16, 4, c.n + 70
    T = _templates(K, ell, 12)
    plain = k.encrypt_db(T, ell, n1, 700, prerotate=False)
    pre = k.prerotate_db(plain, n1, 2)
    tbe = k.encrypt_db(T, ell, n1, 700, level=2)
    for g, d in [(0, 2), (0, 9), (1, 14)]:
        zp = k.decrypt(plain[g, d], c.top)
        z = k.decrypt(pre[g, d], 2)
        assert np.abs(z - k.decrypt(tbe[g, d], 2)).max() < 1e-6
        assert np.abs(z - np.roll(zp, (d // n1) * n1)).max() < 1e-6      # Rot_{-j n1}: slot x <- x - j n1
        if d >= n1:
            assert not np.array_equal(pre[g, d], tbe[g, d])
        else:
            assert np.array_equal(pre[g, d], tbe[g, d])
    rng = np.random.default_rng(4)
    q = rng.standard_normal(ell)
    q /= np.linalg.norm(q)
    qct = k.encrypt(np.tile(q, c.n // ell), 8)
    S = k.enc_scores(qct, pre, n1, level=2)
    got = np.concatenate([k.decrypt(S[g], 1) for g in range(2)])
    s = T.astype(np.float64) @ q
    assert np.abs(got[:K] - s).max() < 1e-4 and np.abs(got[K:]).max() < 1e-4
