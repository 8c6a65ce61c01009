"""CPU tests of libfr.so: exported symbols, host client code (bit-exact with the
oracle on the same seeds), rotation-set and rotation-count bookkeeping against
the values printed in the paper. No GPU is needed."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split(None, 1)
                vals[k] = int(v)
    return vals


def header_functions():
    src = open(os.path.join(ROOT, "include", "fr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = fr.load()
    names = header_functions()
    assert len(names) >= 30
    for n in names:
        assert hasattr(L, n), n
    assert sorted(fr.EXPORTED) == names


def test_setup_without_gpu_fails_loudly():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(fr.FrError) as e:
        fr.Context(device=0, **W.ctx_params("tiny"))
    assert e.value.status == fr.FR_ERR_CUDA


@pytest.mark.parametrize("cfg", ["tiny", "mid"])
def test_client_primes_keys_and_encryption_match_oracle(cfg):
    c = W.CONFIGS[cfg]
    ctx = fr.Context(device=-1, **W.ctx_params(cfg))
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    assert ctx.primes() == oc.primes
    assert ctx.info()["n_digits"] == oc.ndig
    keys = ctx.keygen([1, 2], W.key_seed(cfg))
    ok = oc.keygen(W.key_seed(cfg))
    T, q, _ = W.workload(cfg)
    ct = ctx.encrypt(keys, q, W.enc_seed(cfg))
    ref = ok.encrypt(np.tile(q, oc.n // c["ell"]), W.enc_seed(cfg))
    assert np.array_equal(ct.export(), ref)
    # decryption by the library of the oracle's ciphertext
    imp = ctx.import_ct(ref, oc.top)
    z = ctx.decrypt(keys, imp)
    assert np.abs(z - np.tile(q, oc.n // c["ell"])).max() < 1e-6


@pytest.mark.parametrize("level", [2, 8])
def test_enroller_encrypted_diagonals_match_oracle(level):
    """Encrypted-database enrollment (host code of the library): the pre-rotated diagonals of a
    two-group database, encrypted at `level`, equal the oracle's bit for bit."""
    c = W.CONFIGS["mid"]
    ctx = fr.Context(device=-1, **W.ctx_params("mid"))
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    keys = ctx.keygen([1], W.key_seed("mid"))
    ok = oc.keygen(W.key_seed("mid"))
    T = W.templates(ctx.n + 300, c["ell"], W.DATASET_SEED + 90)
    E = ctx.encrypt_db(keys, T, level=level, seed=0xABC)
    assert E.shape == (2, c["ell"], 2, level + 1, oc.N)
    assert np.array_equal(E, ok.encrypt_db(T, c["ell"], c["n1"], 0xABC, level=level))
    P = ctx.encrypt_db(keys, T, level=level, seed=0xABC, prerotate=False)     # plain diagonals
    assert np.array_equal(P, ok.encrypt_db(T, c["ell"], c["n1"], 0xABC, level=level, prerotate=False))
    assert np.array_equal(P[:, :c["n1"]], E[:, :c["n1"]]) and not np.array_equal(P, E)
    with pytest.raises(fr.FrError) as e:
        ctx.encrypt_db(keys, T, level=len(c["q_bits"]))
    assert e.value.status == fr.FR_ERR_LEVEL


def test_import_rejects_unreduced_words():
    c = W.CONFIGS["tiny"]
    ctx = fr.Context(device=-1, **W.ctx_params("tiny"))
    w = np.zeros((2, 3, 1 << c["log_n"]), dtype=np.uint64)
    w[1, 2, 7] = np.uint64(ctx.primes()[2])
    with pytest.raises(fr.FrError) as e:
        ctx.import_ct(w, 2)
    assert e.value.status == fr.FR_ERR_FORMAT


def test_device_calls_on_client_context_fail():
    ctx = fr.Context(device=-1, **W.ctx_params("tiny"))
    keys = ctx.keygen([1], 5)
    ct = ctx.encrypt(keys, np.ones(64) / 8, 9)
    with pytest.raises(fr.FrError) as e:
        ctx.rotate(ct, 1)
    assert e.value.status == fr.FR_ERR_CUDA


@pytest.mark.parametrize("n", [13, 27, 59])
def test_chebyshev_coefficients_bit_identical_to_oracle(n):
    a = fr.cheb_coeffs(n, 0.5)
    b = oracle.cheb_coeffs(n, 0.5)
    assert a.tobytes() == b.tobytes()


def test_rotation_sets_reproduce_paper_key_counts():
    g = read_golden("paper_counts.txt")
    ell, n1, slots = 512, 23, 1 << 14
    assert len(fr.rotation_set(ell, n1, slots, fr.FR_KEYS_CPU_BSGS)) == g["keys_cpu_bsgs_l512_n1_23"]
    hydia = fr.rotation_set(ell, n1, slots, fr.FR_KEYS_HYDIA_DG)
    assert len(hydia) == g["keys_dg_total"]
    assert len([k for k in hydia if k < ell]) == g["keys_hydia_l512"]
    assert len(fr.rotation_set(ell, n1, slots, fr.FR_KEYS_TBS_ONLINE)) == g["keys_tbs_online"]
    assert len(fr.rotation_set(ell, n1, slots, fr.FR_KEYS_TBS_TOTAL)) == g["keys_tbs_total"]
    assert len(fr.rotation_set(ell, n1, slots, fr.FR_KEYS_TBE_TOTAL)) == g["keys_tbe_total"]
    # this library's on-demand set at the headline parameters: 31 baby + 15 giant (+ 6 extra powers of two)
    assert len(fr.rotation_set(512, 32, 1 << 15, fr.FR_KEYS_ONDEMAND, False)) == 46
    assert len(fr.rotation_set(512, 32, 1 << 15, fr.FR_KEYS_ONDEMAND, True)) == 52


def test_rotation_counts_reproduce_paper_table():
    g = read_golden("paper_counts.txt")
    for G, key in [(1, "rot_textbook_G1"), (4, "rot_textbook_G4"), (16, "rot_textbook_G16"),
                   (32, "rot_textbook_G32"), (64, "rot_textbook_G64")]:
        assert fr.rotation_count(512, 23, G, 0) == g[key]
    assert fr.rotation_count(512, 23, 64, 1) == g["rot_bsgs_diagonal"]


def test_required_rotations_of_context():
    ctx = fr.Context(device=-1, **W.ctx_params("membership"))
    s = ctx.required_rotations(fr.FR_MODE_SCORES)
    assert s == list(range(1, 32)) + [32 * j for j in range(1, 16)]
    m = ctx.required_rotations(fr.FR_MODE_MEMBERSHIP)
    assert set(m) == set(s) | {1 << t for t in range(15)}


def test_client_decrypt_crt_matches_oracle():
    params = dict(log_n=10, q_bits=[40, 40, 40], p_bits=[60, 60], dnum=1, scale_bits=30, ell=32, n1=4)
    ctx = fr.Context(device=-1, **params)
    oc = oracle.Ctx(10, [40, 40, 40], [60, 60], 1, 30)
    ok = oc.keygen(3)
    keys = ctx.keygen([], 3)
    rng = np.random.default_rng(2)
    z = 2500.0 + rng.uniform(-1, 1, oc.n)
    ct = ok.encrypt(z, 4)
    for lvl in (2, 1):
        w = oc.drop(ct, 2, lvl)
        got = ctx.decrypt(keys, ctx.import_ct(w, lvl))
        assert np.abs(got - z).max() < 1e-4
        assert got.tobytes() == ok.decrypt(w, lvl).tobytes()


def test_work_level_of_contexts():
    for cfg, lm, expect in [("membership", 0, 24), ("membership", 1, 8), ("tiny", 1, 2), ("deep", 1, 8),
                            ("mid", 1, 8)]:
        ctx = fr.Context(device=-1, **W.ctx_params(cfg, level_mode=lm))
        assert ctx.work_level == expect == W.work_level(cfg, lm)


def test_radix_rotation_key_set_and_parameter_checks():
    """RotateAndSum in radix r needs the keys t s (t < r, s = 1, r, r^2, ...) instead of the
    powers of two; the parameters are checked by fr_setup on the host."""
    base = W.ctx_params("mid")
    ctx8 = fr.Context(device=-1, sum_radix=8, **base)
    assert set(ctx8.required_rotations(fr.FR_MODE_MEMBERSHIP)) == {t * s for s in (1, 8, 64, 512) for t in range(1, 8)}
    ctx4 = fr.Context(device=-1, sum_radix=4, **base)
    r4 = set(ctx4.required_rotations(fr.FR_MODE_MEMBERSHIP))
    assert {t * 4 ** e for e in range(6) for t in (1, 2, 3)} <= r4 and 2048 in r4     # 4096 = 4^6: six steps
    ctx2 = fr.Context(device=-1, **base)
    assert {1 << t for t in range(12)} <= set(ctx2.required_rotations(fr.FR_MODE_MEMBERSHIP))
    # identification needs no slot sum: the same keys for every radix
    assert ctx8.required_rotations(fr.FR_MODE_IDENTIFY) == ctx2.required_rotations(fr.FR_MODE_IDENTIFY)
    for bad in (dict(sum_radix=6), dict(sum_radix=128), dict(hoist_giants=2)):
        with pytest.raises(fr.FrError) as e:
            fr.Context(device=-1, **base, **bad)
        assert e.value.status == fr.FR_ERR_INVALID_ARG
    ctx2.inject_alloc_failure(3)      # host-side setting; no device allocation on a client context
    ctx2.inject_alloc_failure(-1)
