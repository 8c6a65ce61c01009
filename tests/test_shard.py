"""Block-sharded matching (the multi-process form of Algorithms 5 and 6) on the CPU.

Template groups are split across gloo ranks. Each rank's per-group outputs come from the oracle,
standing in for one GPU's library calls. The exchange and reduction logic of shard.py (the path
`bench.py --shard` runs: query broadcast as a tensor, per-group ciphertexts sent to rank 0 with
point-to-point tensor transfers, mod-q sum and RotateAndSum there) must then reproduce the
single-process oracle result bit for bit, for identification (groups gathered in order) and
membership, at world sizes 2 and 4. A rank that holds no group is covered too.
"""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import shard
from paper_2604_00546_gb300 import workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

# N = 2^12 (2048 slots per group), the mid chain, K = 5000: three groups, the last one ragged
CFG = dict(log_n=12, q_bits=[60] + [45] * 8, p_bits=[60] * 3, dnum=3, scale_bits=45, ell=64, n1=8, K=5000)
KEY_SEED, ENC_SEED, T_SEED = 0x5EED01, 0x5EED02, 0x5EED03


def test_group_range_covers_groups_once():
    for G in range(0, 11):
        for world in range(1, 6):
            rs = [shard.group_range(G, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == G
            assert all(rs[r][1] == rs[r + 1][0] for r in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1 and sizes == sorted(sizes, reverse=True)
    with pytest.raises(ValueError):
        shard.group_range(3, 2, 2)


def test_identification_database_splits_evenly():
    """The 32 groups of the K = 2^20 database over 1..8 ranks: every group once, sizes within one."""
    T = np.zeros((1 << 20, 1), dtype=np.float32)
    for world in range(1, 9):
        parts = [shard.template_shard(T, 1 << 15, world, r) for r in range(world)]
        assert sum(p.shape[0] for p, _ in parts) == 1 << 20
        sizes = [g1 - g0 for _, (g0, g1) in parts]
        assert sum(sizes) == 32 and max(sizes) - min(sizes) <= 1


def test_template_shards_rejoin():
    T = W.templates(5000, 64, 7)
    for world in (1, 2, 3, 4):
        parts = [shard.template_shard(T, 2048, world, r) for r in range(world)]
        assert np.array_equal(np.concatenate([p for p, _ in parts]), T)
        for p, (g0, g1) in parts:
            assert p.shape[0] == min(g1 * 2048, 5000) - min(g0 * 2048, 5000)


class _Ct:
    """Ciphertext stand-in: exported words [2][level+1][N]."""

    def __init__(self, words):
        self.w = np.ascontiguousarray(words, dtype=np.uint64)

    def export(self):
        return self.w


class OracleEngine:
    """The oracle behind the engine methods shard.py calls (one GPU's library, on the CPU)."""

    def __init__(self):
        self.oc = oracle.Ctx(CFG["log_n"], CFG["q_bits"], CFG["p_bits"], CFG["dnum"], CFG["scale_bits"])
        self.ok = self.oc.keygen(KEY_SEED)

    def encrypt(self, q):
        return _Ct(self.ok.encrypt(np.tile(q, self.oc.n // CFG["ell"]), ENC_SEED))

    def match(self, db, query, mode):
        out, _ = self.ok.match(query.w, db, CFG["ell"], CFG["n1"], mode, 59, 0.5)
        return [_Ct(x) for x in out]

    def import_ct(self, words, level):
        assert words.shape[1] == level + 1
        return _Ct(words)

    def membership_reduce(self, parts):
        lvl = parts[0].w.shape[1] - 1
        s = parts[0].w
        for p in parts[1:]:
            s = self.oc.add(s, p.w, lvl)
        return _Ct(self.ok.rotate_sum(s, lvl, CFG["log_n"] - 1))


def _query():
    rng = np.random.default_rng(11)
    q = rng.standard_normal(CFG["ell"])
    return q / np.linalg.norm(q)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        oracle.set_threads(2)
        eng = OracleEngine()
        T = W.templates(CFG["K"], CFG["ell"], T_SEED)
        Ts, (g0, g1) = shard.template_shard(T, 1 << (CFG["log_n"] - 1), ws, rank)
        query = shard.share_query(eng, eng.encrypt(_query()) if rank == 0 else None, dist)
        res = shard.sharded_match(eng, Ts if g1 > g0 else None, query, mode, dist)
        q.put((rank, None if res is None else [r.export() for r in res]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 4])   # 3 groups: split 2 + 1, and 1 + 1 + 1 + none
@pytest.mark.parametrize("mode", [fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP])
def test_sharded_equals_single_process(ws, mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, ws, port, mode, q)) for r in range(ws)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=300) for _ in range(ws))
    for p in ps:
        p.join(60)
        assert p.exitcode == 0
    assert all(res[r] is None for r in range(1, ws))
    eng = OracleEngine()
    T = W.templates(CFG["K"], CFG["ell"], T_SEED)
    ref, _ = eng.ok.match(eng.encrypt(_query()).w, T, CFG["ell"], CFG["n1"], mode, 59, 0.5)
    got = res[0]
    assert len(got) == ref.shape[0] == (1 if mode == fr.FR_MODE_MEMBERSHIP else 3)
    for g in range(len(got)):
        assert np.array_equal(got[g], ref[g]), g


def test_one_process_needs_no_collective():
    eng = OracleEngine()
    T = W.templates(CFG["K"], CFG["ell"], T_SEED)[:2048]    # one group
    qct = eng.encrypt(_query())
    got = shard.sharded_match(eng, T, shard.share_query(eng, qct), fr.FR_MODE_MEMBERSHIP)
    ref, _ = eng.ok.match(qct.w, T, CFG["ell"], CFG["n1"], fr.FR_MODE_MEMBERSHIP, 59, 0.5)
    assert np.array_equal(got[0].export(), ref[0])
    with pytest.raises(ValueError):
        shard.sharded_match(eng, None, qct, fr.FR_MODE_MEMBERSHIP)
