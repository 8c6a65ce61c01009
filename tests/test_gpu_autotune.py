"""GPU tests of the NTT tile-shape autotuner: fr_setup times every shape (four radix-8
two-pass tile shapes, the single-launch cluster kernel and the radix-16 two-pass kernels) per
batch bucket at N=2^16 and keeps the fastest; every shape gives the same transforms, so a rotation at
N=2^16 (which runs inverse and forward NTTs of several batch sizes) is bit-identical to the
oracle under each forced shape."""
import numpy as np
import pytest

import oracle
from paper_2604_00546_gb300 import fr
from paper_2604_00546_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    c = W.CONFIGS["membership"]
    ctx = fr.Context(device=0, **W.ctx_params("membership", level_mode=1))
    keys = ctx.keygen(list(range(1, 9)), W.key_seed("membership"))
    ctx.load_keys(keys)
    oc = oracle.Ctx(c["log_n"], c["q_bits"], c["p_bits"], c["dnum"], c["scale_bits"])
    ok = oc.keygen(W.key_seed("membership"))
    rng = np.random.default_rng(9)
    z = rng.uniform(-1, 1, oc.n)
    top = oc.top
    ct = ok.encrypt(z, 55)
    lvl = ctx.work_level
    low = oc.drop(ct, top, lvl)
    ref = ok.hoisted_rotate(low, lvl, list(range(1, 9)))
    ref_rot = {k: ref[k - 1] for k in range(1, 9)}
    return dict(ctx=ctx, ok=ok, oc=oc, low=low, lvl=lvl, ref_rot=ref_rot, ref_rs=oc.rescale(low, lvl))


def test_tuner_picks_the_fastest_measured_shape(big):
    t = big["ctx"].ntt_tuning()
    us = np.array(t["us"])
    assert us.shape == (4, 6) and (us[:, :4] > 0).all()
    for b in range(4):
        avail = np.where(us[b] > 0, us[b], np.inf)
        sh = t["shapes"][b]
        # the default shape stays unless another is the fastest by at least 3%
        if sh == 0:
            assert avail[1:].min() >= 0.97 * avail[0] or avail[1:].min() >= avail[0]
        else:
            assert avail[sh] == avail.min() and avail[sh] < 0.97 * avail[0]


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5])
def test_every_shape_is_bit_exact(big, shape):
    ctx = big["ctx"]
    saved = ctx.ntt_tuning()["shapes"]
    try:
        ctx.ntt_set_shapes([shape] * 4)
        ct = ctx.import_ct(big["low"], big["lvl"])
        ct.upload()
        # hoisted rotations: batches of 9, 30, 16 and 144 limb-polynomials; rescale: 2 and 16
        ks = list(range(1, 9))
        outs = ctx.rotate_hoisted(ct, ks)
        for k, o in zip(ks, outs):
            assert np.array_equal(o.export(), big["ref_rot"][k]), k
        assert np.array_equal(ctx.rescale(ct).export(), big["ref_rs"])
    finally:
        ctx.ntt_set_shapes(saved)


def test_measured_peaks_are_plausible():
    """The register-only ceilings the bench divides by: the NTT butterfly (64-bit integer
    pipes) and the FP64 fused multiply-add (the encoder's FFT). Both well above zero and
    below what any GB300 could do (2070 MHz x 152 SMs bounds them)."""
    bfly = fr.butterfly_peak(0)
    fp64 = fr.fp64_peak(0)
    assert 1e11 < bfly < 1e13
    assert 1e11 < fp64 < 1e13
