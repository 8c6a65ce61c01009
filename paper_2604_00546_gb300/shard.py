"""Block-sharded matching across processes, one GPU each (the multi-GPU form of Algorithms 5
and 6).

The HyDia packing (Section 3, Fig. 1) puts numSlots = N/2 templates in one group, and every
group is matched on its own: the scores, the threshold and the per-group outputs of group k
depend only on templates [k numSlots, (k+1) numSlots). So a database splits along group
boundaries. Rank r loads the templates of a contiguous range of groups and matches the same
query against them.

- Identification (Algorithm 6) needs no exchange. The destination rank gathers every rank's
  per-group threshold ciphertexts in group order.
- Membership (Algorithm 5) needs one exchange. Every rank runs identification on its groups.
  The destination rank gathers the per-group ciphertexts and calls `membership_reduce`
  (`fr_membership_reduce`): a mod-q sum, then RotateAndSum. That equals the single-process
  membership bit for bit, because a sum mod q is exact and independent of the order of its
  terms.

Ciphertexts cross processes in the library's export format: coefficient form,
[2][level+1][N] uint64, packed into one int64 tensor per rank and moved with tensor
collectives (broadcast of the query, point-to-point send/recv of the per-group outputs to the
destination rank). Over NCCL the tensors live on the rank's GPU (the current CUDA device); over
gloo on the host. No kernel of the library ever reads another rank's memory.

The engine is any object with the `fr.Context` methods used here: match, import_ct and
membership_reduce. Outputs expose `export()`.
"""
from __future__ import annotations

import numpy as np

from . import fr


def group_range(G: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous range [g0, g1) of the G groups held by `rank`. Ranks differ by at most one
    group, and the lower ranks take the extra ones."""
    if world < 1 or not 0 <= rank < world or G < 0:
        raise ValueError("bad world size, rank or group count")
    base, extra = divmod(G, world)
    g0 = rank * base + min(rank, extra)
    return g0, g0 + base + (1 if rank < extra else 0)


def template_shard(T: np.ndarray, slots: int, world: int, rank: int):
    """The rows of T (K x ell) that fall in `rank`'s groups, and the range (g0, g1). A group
    holds `slots` templates; the last group of the database may be ragged."""
    K = int(T.shape[0])
    G = -(-K // slots)
    g0, g1 = group_range(G, world, rank)
    return T[g0 * slots:min(g1 * slots, K)], (g0, g1)


def _coll_device(dist):
    """Where collective tensors live: the current CUDA device for NCCL, the host otherwise."""
    import torch
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def _to_tensor(words, device):
    import torch
    flat = np.ascontiguousarray(words, dtype=np.uint64).reshape(-1).view(np.int64)
    return torch.from_numpy(flat).to(device)


def _to_words(t, shape):
    return t.cpu().numpy().view(np.uint64).reshape(shape)


def share_query(engine, query, dist=None, src: int = 0):
    """The query ciphertext on every rank. `src` passes its handle and exports it; the other
    ranks pass None and import what src broadcasts (a shape header, then the words)."""
    if dist is None or dist.get_world_size() == 1:
        return query
    import torch
    dev = _coll_device(dist)
    rank = dist.get_rank()
    w = query.export() if rank == src else None
    hdr = torch.tensor(list(w.shape) if w is not None else [0, 0, 0], dtype=torch.int64, device=dev)
    dist.broadcast(hdr, src=src)
    shape = tuple(int(x) for x in hdr.tolist())
    buf = _to_tensor(w, dev) if w is not None else torch.empty(int(np.prod(shape)), dtype=torch.int64, device=dev)
    dist.broadcast(buf, src=src)
    if rank == src:
        return query
    return engine.import_ct(_to_words(buf, shape), shape[1] - 1)


def sharded_match(engine, db, query, mode: int, dist=None, dst: int = 0):
    """Match `query` against a database split across the ranks of `dist` (torch.distributed,
    initialised; None for one process).

    db is this rank's shard (from template_shard), or None if the rank holds no group. Every rank
    passes the same query. On `dst` the result is a list of ciphertexts: the scores or threshold
    outputs of all groups in group order (FR_MODE_SCORES, FR_MODE_IDENTIFY), or the single
    membership ciphertext (FR_MODE_MEMBERSHIP). Other ranks return None.
    """
    if mode not in (fr.FR_MODE_SCORES, fr.FR_MODE_IDENTIFY, fr.FR_MODE_MEMBERSHIP):
        raise ValueError("unknown mode")
    local = fr.FR_MODE_IDENTIFY if mode == fr.FR_MODE_MEMBERSHIP else mode
    outs = list(engine.match(db, query, local)) if db is not None else []
    world = 1 if dist is None else dist.get_world_size()
    rank = 0 if dist is None else dist.get_rank()
    if world == 1:
        parts = outs
    else:
        import torch
        dev = _coll_device(dist)
        if rank != dst:
            # header (count, limbs, N), then every output's words in group order
            words = [o.export() for o in outs]
            shape = words[0].shape if words else (2, 0, 0)
            hdr = torch.tensor([len(words), shape[1], shape[2]], dtype=torch.int64, device=dev)
            dist.send(hdr, dst=dst)
            if words:
                dist.send(_to_tensor(np.stack(words), dev), dst=dst)
            return None
        parts = []
        for r in range(world):
            if r == dst:
                parts.extend(outs)
                continue
            hdr = torch.empty(3, dtype=torch.int64, device=dev)
            dist.recv(hdr, src=r)
            n, limbs, N = (int(x) for x in hdr.tolist())
            if n == 0:
                continue
            buf = torch.empty(n * 2 * limbs * N, dtype=torch.int64, device=dev)
            dist.recv(buf, src=r)
            words = _to_words(buf, (n, 2, limbs, N))
            parts.extend(engine.import_ct(words[i], limbs - 1) for i in range(n))
    if mode != fr.FR_MODE_MEMBERSHIP:
        return parts
    if not parts:
        raise ValueError("no rank holds a group of the database")
    return [engine.membership_reduce(parts)]
