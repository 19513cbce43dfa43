"""GPU parity of the Gaussian-set codec (Sec. 4, quantisation and
compression) with the oracle: bit-exact codes, Morton order and delta
streams at several position widths (one- and two-word Morton keys, ties),
decoded parameters equal to the oracle's decode, the full 500k-Gaussian
microscopy set, LZMA containers interchangeable with the oracle's, rendering
of decoded sets, serving an encoded set, and argument checks."""
import numpy as np
import pytest
import torch

import oracle
from oracle import codec as oc
from paper_2603_20611_b300 import binding as B
from paper_2603_20611_b300 import synth
from tests.gpu_util import assert_forward_close, dev_set, np32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return B.Context(0)


def _u16(t):
    return t.cpu().numpy().view(np.uint16)


def _check_encode(ctx, g, bits):
    hdr, streams, order = B.gp_encode(ctx, dev_set(g), bits)
    h_ref, s_ref, o_ref = oc.encode(g.mu, g.scale, g.quat, g.alpha, bits=bits)
    assert hdr.n == g.n and hdr.pos_bits == bits
    assert np.array_equal(np.array(hdr.lo[:], np.float32), h_ref["lo"])
    assert np.array_equal(np.array(hdr.hi[:], np.float32), h_ref["hi"])
    assert hdr.log_s_min == pytest.approx(h_ref["L0"], rel=1e-15, abs=1e-15)
    assert hdr.log_s_max == pytest.approx(h_ref["L1"], rel=1e-15, abs=1e-15)
    np.testing.assert_array_equal(order.cpu().numpy(), o_ref)
    np.testing.assert_array_equal(_u16(streams), s_ref)
    return hdr, streams


@pytest.mark.parametrize("bits", [3, 8, 10, 14, 15])
def test_encode_is_bit_exact(ctx, bits):
    g = synth.small(seed=400 + bits, n=3001, extent=(64, 48, 32))
    _check_encode(ctx, g, bits)


def test_scale_codes_at_their_thresholds(ctx):
    """Scales placed on the fp32 values around the codec's double-precision
    thresholds exp(L0 + (k - 1/2) D) (the float nearest each one and its two
    neighbours): the device's codes, decided without double arithmetic, equal
    the oracle's double comparisons."""
    g = synth.small(seed=430, n=3000, extent=(64, 64, 32))
    s = g.scale.astype(np.float32).copy()
    lo, hi = np.float32(0.25), np.float32(12.0)
    s[0, 0], s[1, 1] = lo, hi  # fixes L0 and L1
    L0, L1 = float(np.log(np.float64(lo))), float(np.log(np.float64(hi)))
    th = oc.scale_thresholds(L0, L1)
    rng = np.random.default_rng(5)
    ks = rng.choice(th.size, 900, replace=False)
    f = th[ks].astype(np.float32)
    cand = np.concatenate([f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(0))])
    cand = np.clip(cand, lo, hi)
    flat = s.reshape(-1)
    flat[10:10 + cand.size] = cand  # after the two fixed entries (flat indices 0 and 4)
    g2 = synth.GaussianSet(g.mu, flat.reshape(s.shape), g.quat, g.alpha, g.extent)
    _check_encode(ctx, g2, 12)


def test_decode_matches_oracle(ctx):
    g = synth.small(seed=420, n=2500, extent=(64, 64, 32))
    hdr, streams = _check_encode(ctx, g, 14)
    gs = B.gp_decode(ctx, hdr, streams)
    h_ref = {"n": hdr.n, "bits": 14, "lo": np.array(hdr.lo[:], np.float32), "hi": np.array(hdr.hi[:], np.float32),
             "L0": hdr.log_s_min, "L1": hdr.log_s_max}
    mu, s, q, a = oc.decode(h_ref, _u16(streams))
    assert np.array_equal(gs.mu.cpu().numpy(), mu)
    assert np.array_equal(gs.quat.cpu().numpy(), q)
    assert np.array_equal(gs.alpha.cpu().numpy(), a)
    # the scale is exp() of the log-domain code in double on each side: equal up to 1 ulp of fp32
    ds = np.abs(gs.scale.cpu().numpy().astype(np.float64) - s) / np.spacing(s)
    assert ds.max() <= 1.0


def test_full_microscopy_set(ctx):
    g = synth.microscopy()
    hdr, streams = _check_encode(ctx, g, 14)
    blob = B.encode_bytes(ctx, dev_set(g))
    assert len(blob) < 22 * g.n  # LZMA shrinks the 22-byte-per-Gaussian streams
    h2, s2 = oc.unpack(blob)  # the product's container is the oracle's container
    np.testing.assert_array_equal(s2, _u16(streams))


def test_containers_interchange_and_render(ctx):
    g = synth.small(seed=430, n=2000, extent=(64, 64, 32))
    h_ref, s_ref, _ = oc.encode(g.mu, g.scale, g.quat, g.alpha, bits=14)
    hdr, gs = B.decode_bytes(ctx, oc.pack(h_ref, s_ref))
    z = synth.slice_positions(range(0, 32, 3))
    I_dec = B.gp_render_slices(ctx, gs, z, 64, 64, 2.0)
    mu, s, q, a = (np32(t) for t in (gs.mu, gs.scale, gs.quat, gs.alpha))
    assert_forward_close(np32(I_dec), oracle.render(mu, s, q, a, z, 64, 64, 2.0), "decoded set")
    # and the decoded set renders like the original (quantisation noise only)
    I0 = oracle.render(g.mu, g.scale, g.quat, g.alpha, z, 64, 64, 2.0)
    psnr = 10 * np.log10(I0.max() ** 2 / np.mean((np32(I_dec) - I0) ** 2))
    assert psnr > 40.0, psnr


def test_serving_an_encoded_set(ctx):
    g = synth.small(seed=440, n=3000, extent=(96, 96, 48))
    hdr, streams, _ = B.gp_encode(ctx, dev_set(g), 14)
    gs = B.gp_decode(ctx, hdr, streams)
    srv = B.Server(ctx, workers=2)
    sid = srv.load_encoded(hdr, streams)
    out = torch.empty(2, 96, 96, device="cuda")
    z = np.array([10.5, 30.25], np.float32)
    t = srv.submit(B.GP_REQ_STACK, sid, out, z=z, H=96, W=96, sigma_z=2.0)
    for _ in range(600):
        r = srv.poll(t, timeout_ms=100)
        if r is not None:
            break
    assert r["status"] == B.GP_OK
    assert torch.equal(out, B.gp_render_slices(ctx, gs, z, 96, 96, 2.0))
    srv.close()


def test_bad_arguments(ctx):
    g = synth.small(seed=450, n=50, extent=(16, 16, 16))
    gs = dev_set(g)
    for bits in (0, 16):
        with pytest.raises(B.GPError):
            B.gp_encode(ctx, gs, bits)
    gs.scale[3, 1] = 0.0
    with pytest.raises(B.GPError) as ei:
        B.gp_encode(ctx, gs, 14)
    assert ei.value.status == B.GP_ERR_ARG
