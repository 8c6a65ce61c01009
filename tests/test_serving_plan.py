"""CPU tests of the serving loop's batch planner (fr_serve_plan): the next batch serves the
oldest request's class, in arrival order, at most max_batch requests, rounded down to a
power of two and halved until its workspace fits the HBM still free."""
import pytest

from paper_2604_00546_gb300 import fr

GB = 1 << 30


def test_oldest_class_in_arrival_order():
    cls = [3, 1, 3, 3, 2, 3, 3, 1, 3]
    assert fr.serve_plan(cls, 8, 100 * GB, GB, GB) == [0, 2, 3, 5]  # 6 of class 3 -> 4
    assert fr.serve_plan(cls, 2, 100 * GB, GB, GB) == [0, 2]
    assert fr.serve_plan([1, 2, 2, 2], 8, 100 * GB, 0, GB) == [0]


def test_power_of_two_and_cap():
    assert len(fr.serve_plan([0] * 7, 8, 100 * GB, 0, GB)) == 4
    assert len(fr.serve_plan([0] * 8, 8, 100 * GB, 0, GB)) == 8
    assert len(fr.serve_plan([0] * 30, 16, 100 * GB, 0, GB)) == 16
    assert len(fr.serve_plan([0] * 3, 1, 100 * GB, 0, GB)) == 1


def test_admission_by_free_memory():
    # base 2 GB + 3 GB per query, 14 GB free: 8 -> 4 (14 GB) fits exactly
    assert len(fr.serve_plan([0] * 8, 8, 14 * GB, 2 * GB, 3 * GB)) == 4
    assert len(fr.serve_plan([0] * 8, 8, 13 * GB, 2 * GB, 3 * GB)) == 2
    assert len(fr.serve_plan([0] * 8, 8, 5 * GB, 2 * GB, 3 * GB)) == 1
    assert fr.serve_plan([0] * 8, 8, 4 * GB, 2 * GB, 3 * GB) == []   # nothing fits: wait


def test_empty_queue():
    assert fr.serve_plan([], 8, GB, 0, 1) == []


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_plan_properties_random(seed):
    import random
    rng = random.Random(seed)
    for _ in range(200):
        n = rng.randint(1, 40)
        cls = [rng.randint(0, 3) for _ in range(n)]
        mb = rng.choice([1, 2, 4, 8, 16, 64])
        base, per = rng.randint(0, 4) * GB, rng.randint(1, 4) * GB
        avail = rng.randint(0, 80) * GB
        got = fr.serve_plan(cls, mb, avail, base, per)
        B = len(got)
        same = [i for i in range(n) if cls[i] == cls[0]]
        if B:
            assert got == same[:B]                         # oldest class, arrival order
            assert B & (B - 1) == 0 and B <= mb            # power of two within the cap
            assert base + B * per <= avail                 # fits
        # maximal: doubling would break the cap, the class size or the budget
        B2 = max(1, 2 * B)
        assert B2 > mb or B2 > len(same) or base + B2 * per > avail
