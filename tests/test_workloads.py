"""The seeded synthetic inputs (CPU): shapes, norms and planted structure of every workload the
tests and the bench use, so that a change to the recipe shows up here rather than as a moved
benchmark number."""
import numpy as np

from paper_2604_00546_gb300 import workloads as W


def test_templates_are_unit_rows_and_seeded():
    T = W.templates(1000, 512, 7)
    assert T.shape == (1000, 512) and T.dtype == np.float32
    assert np.abs(np.linalg.norm(T.astype(np.float64), axis=1) - 1.0).max() < 1e-6
    assert np.array_equal(T, W.templates(1000, 512, 7))
    assert not np.array_equal(T, W.templates(1000, 512, 8))


def test_membership_workload_plants_32_duplicates_at_cosine_08():
    T, q, planted = W.workload("membership")
    assert T.shape == (1 << 15, 512) and q.shape == (512,)
    assert abs(np.linalg.norm(q) - 1.0) < 1e-12
    assert len(planted) == 32 and len(set(planted.tolist())) == 32
    s = T.astype(np.float64) @ q
    assert np.abs(s[planted] - 0.8).max() < 1e-6           # float32 rows
    others = np.setdiff1d(np.arange(len(T)), planted)
    assert np.abs(s[others]).max() < 0.3                  # random unit vectors in 512 dimensions
    assert (s >= 0.5).sum() == 32


def test_identify_workload_size_and_groups():
    c = W.CONFIGS["identify"]
    assert c["K"] == 1 << 20 and -(-c["K"] // (1 << (c["log_n"] - 1))) == 32


def test_serving_stream():
    reqs = W.serving_requests()
    t = np.array([r[0] for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < 60.0
    assert 1000 < len(reqs) < 1400                       # Poisson, mean 1200
    mem = np.mean([r[1] == 2 for r in reqs])
    assert 0.65 < mem < 0.75
    assert {r[2] for r in reqs} == set(range(8))
    sizes = [len(T) for T in W.serving_databases(ell=8)]
    assert sizes == [1 << 12, 1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18, 1 << 12, 1 << 14]


def test_multi_sizes_log_uniform():
    K = W.multi_sizes()
    assert len(K) == 64 and min(K) >= 1 << 10 and max(K) <= 1 << 17
    lk = np.log2(K)
    assert 12.5 < lk.mean() < 14.5                       # U(10, 17) has mean 13.5


def test_work_level_rule():
    # 2 + d2 with the degree-59 split (d1, d2) = (2, 6), capped at the top level
    assert W.work_level("membership", 1) == 8
    assert W.work_level("membership", 0) == 24
    assert W.work_level("deep", 1) == 8
