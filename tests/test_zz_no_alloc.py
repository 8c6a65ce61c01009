"""fr_rotate_noalloc: the rotation for callers that cannot allocate device memory
while they run. Its temporaries live in a fixed device array inside the
library; the caller passes device buffers for input and output. The test
compares it bit for bit with the CPU oracle's rotation of the same ciphertext
under the same keys (tiny ring) and with fr_rotate (which allocates its
temporaries), two calls in a row, and checks that refused calls (level above the
loaded keys, working set beyond the fixed array) fail with their status.
This file is collected last so that a failure here cannot hide another one."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run(cfg, level_mode, ks, check_oracle=False):
    torch = pytest.importorskip("torch")
    ctx = fr.Context(device=0, **W.ctx_params(cfg, level_mode=level_mode))
    keys = ctx.keygen(sorted(set(ks)), W.key_seed(cfg))
    ctx.load_keys(keys)
    rng = np.random.default_rng(11)
    z = rng.uniform(-1, 1, ctx.n)
    ct = ctx.encrypt_slots(keys, z, 5)
    words = ct.export()
    lvl = ctx.work_level
    words = np.ascontiguousarray(np.stack([words[0, : lvl + 1], words[1, : lvl + 1]]))
    ref_ct = ctx.import_ct(words, lvl).upload()
    d_in = torch.from_numpy(words.view(np.int64)).to("cuda:0")
    ok = None
    if check_oracle:
        c = W.CONFIGS[cfg]
        oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
        ok = oc.keygen(W.key_seed(cfg))
    for k in ks:
        ref = ctx.rotate(ref_ct, k).export()
        if ok is not None:
            assert np.array_equal(ref, ok.rotate(words, lvl, k)), k
        for _ in range(2):  # two calls in a row share the scratch array
            d_out = torch.zeros_like(d_in)
            ctx.sync()
            ctx.rotate_noalloc(d_in.data_ptr(), lvl, k, d_out.data_ptr())
            ctx.sync()
            got = d_out.cpu().numpy().view(np.uint64)
            assert np.array_equal(got, ref), k
            if ok is not None:
                assert np.array_equal(got, ok.rotate(words, lvl, k)), k
    # the rotated slots are the left rotation of z
    d_out = torch.zeros_like(d_in)
    ctx.rotate_noalloc(d_in.data_ptr(), lvl, ks[0], d_out.data_ptr())
    ctx.sync()
    dec = ctx.decrypt(keys, ctx.import_ct(d_out.cpu().numpy().view(np.uint64), lvl))
    assert np.abs(dec - np.roll(z, -ks[0])).max() < 1e-4
    return ctx, d_in


def test_noalloc_rotation_matches_oracle_and_fr_rotate_small():
    _run("tiny", 0, [1, 5, 2047], check_oracle=True)


def test_noalloc_rotation_matches_fr_rotate_headline_working_level():
    torch = pytest.importorskip("torch")
    ctx, d_in = _run("membership", 1, [3, 32])
    # a level above the loaded keys is refused before anything is enqueued: the output
    # buffer keeps its contents
    lvl = ctx.work_level + 1
    buf = torch.zeros(2 * (lvl + 1) * ctx.N, dtype=torch.int64, device="cuda:0")
    out = torch.full_like(buf, 7)
    with pytest.raises(fr.FrError) as e:
        ctx.rotate_noalloc(buf.data_ptr(), lvl, 3, out.data_ptr())
    assert e.value.status == fr.FR_ERR_LEVEL
    ctx.sync()
    assert bool((out == 7).all())


def test_noalloc_rotation_rejects_working_set_beyond_the_array():
    # keys for the whole chain (two rotations only): at N=2^16, level 24 needs more scratch
    # than the fixed array holds and is refused with a clear error
    torch = pytest.importorskip("torch")
    ctx = fr.Context(device=0, **W.ctx_params("membership", level_mode=0))
    keys = ctx.keygen([3], W.key_seed("membership"))
    ctx.load_keys(keys)
    buf = torch.zeros(2 * 25 * ctx.N, dtype=torch.int64, device="cuda:0")
    out = torch.zeros_like(buf)
    with pytest.raises(fr.FrError) as e:
        ctx.rotate_noalloc(buf.data_ptr(), 24, 3, out.data_ptr())
    assert e.value.status == fr.FR_ERR_INVALID_ARG and "scratch" in str(e.value)
