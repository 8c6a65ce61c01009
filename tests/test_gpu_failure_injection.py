"""Error paths under injected device-allocation failures (host-side injection through
fr_inject_alloc_failure; nothing faults on the device): a match whose n-th allocation fails
returns FR_ERR_HBM_BUDGET wherever the failure lands (key switch, MAC, the two-stream threshold,
graph capture, output), and the context then matches again with the same bits."""
import numpy as np
import pytest

from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    ctx = fr.Context(device=0, **W.ctx_params("mid"))
    keys = ctx.keygen(ctx.required_rotations(fr.FR_MODE_MEMBERSHIP), W.key_seed("mid"))
    ctx.load_keys(keys)
    T, q, _ = W.workload("mid")
    return dict(ctx=ctx, keys=keys, db=ctx.load_db(T), q=q)


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("mode", [fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_allocation_failures_leave_context_usable(env, graphs, mode):
    ctx, db = env["ctx"], env["db"]
    ctx.use_graphs(graphs)
    qct = ctx.encrypt(env["keys"], env["q"], 55)
    ref = [o.export() for o in ctx.match(db, qct, mode)]
    failures = 0
    try:
        for after in (0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233, 377):
            ctx.inject_alloc_failure(after)
            try:
                got = [o.export() for o in ctx.match(db, qct, mode)]
                assert all(np.array_equal(a, b) for a, b in zip(got, ref))   # fewer allocations than `after`
            except fr.FrError as e:
                assert e.status == fr.FR_ERR_HBM_BUDGET, e
                failures += 1
            finally:
                ctx.inject_alloc_failure(-1)
            again = [o.export() for o in ctx.match(db, qct, mode)]
            assert all(np.array_equal(a, b) for a, b in zip(again, ref)), after
    finally:
        ctx.use_graphs(True)
    assert failures >= (2 if graphs else 3)   # replayed graphs allocate only their outputs


def test_batch_allocation_failure(env):
    ctx, db = env["ctx"], env["db"]
    ctx.use_graphs(False)   # every call allocates its whole workspace
    try:
        qs = [ctx.encrypt(env["keys"], env["q"], 60 + i) for i in range(2)]
        ref = [[o.export() for o in out] for out in ctx.match_batch(db, qs, fr.FR_MODE_MEMBERSHIP)]
        for after in (4, 40):
            ctx.inject_alloc_failure(after)
            try:
                with pytest.raises(fr.FrError):
                    ctx.match_batch(db, qs, fr.FR_MODE_MEMBERSHIP)
            finally:
                ctx.inject_alloc_failure(-1)
            got = [[o.export() for o in out] for out in ctx.match_batch(db, qs, fr.FR_MODE_MEMBERSHIP)]
            assert all(np.array_equal(a, b) for x, y in zip(got, ref) for a, b in zip(x, y))
    finally:
        ctx.use_graphs(True)
