"""Pins of the codec oracle (Sec. 4, quantisation and compression) against
textbook facts: Morton keys of known points and the Z-order of a 2 x 2 x 2
grid, round-trip error within half a quantisation step for every attribute,
quaternion sign folding (q and -q are the same rotation), zigzag / delta
inverses, the stable Morton order, and the LZMA container round trip."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import codec
from paper_2603_20611_b300 import synth


def test_morton_keys_of_known_points():
    c = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [2, 0, 0], [3, 0, 0], [0, 0, 2], [5, 3, 6]])
    k = codec.morton(c, 4)
    # key bit 3 j + a is bit j of axis a
    assert list(k[:7]) == [1, 2, 4, 7, 8, 9, 32]
    ref = 0
    for j in range(4):
        for a in range(3):
            ref |= ((int(c[7, a]) >> j) & 1) << (3 * j + a)
    assert int(k[7]) == ref


def test_z_order_of_a_cube():
    g = np.array([[x, y, z] for z in range(2) for y in range(2) for x in range(2)])
    rng = np.random.Generator(np.random.PCG64(0))
    perm = rng.permutation(8)
    order = np.argsort(codec.morton(g[perm], 1), kind="stable")
    assert [tuple(v) for v in g[perm][order]] == [tuple(v) for v in g]  # x fastest, then y, then z


def test_round_trip_within_half_a_step():
    g = synth.small(seed=5, n=3000, extent=(64, 48, 32))
    hdr, streams, order = codec.encode(g.mu, g.scale, g.quat, g.alpha, bits=14)
    mu, s, q, a = codec.decode(hdr, streams)
    mu0, s0, q0, a0 = (np.asarray(x, np.float64)[order] for x in (g.mu, g.scale, g.quat, g.alpha))
    step = (hdr["hi"].astype(np.float64) - hdr["lo"]) / (2 ** 14 - 1)
    assert np.all(np.abs(mu - mu0) <= 0.5 * step * (1 + 1e-4) + 1e-5)
    D = (hdr["L1"] - hdr["L0"]) / 4095
    assert np.all(np.abs(np.log(s.astype(np.float64)) - np.log(s0)) <= 0.5 * D * (1 + 1e-4) + 1e-6)
    assert np.all(np.abs(a - np.clip(a0, 0, 1)) <= 0.5 / 4095 + 1e-6)
    qn = q0 / np.linalg.norm(q0, axis=1, keepdims=True)
    qn = np.where(qn[:, :1] < 0, -qn, qn)
    assert np.all(q[:, 0] >= 0) and np.all(np.abs(q - qn) <= 0.5 / 2047.5 + 1e-6)
    # the folded quaternion is the same rotation
    R0 = Rotation.from_quat(np.c_[q0[:, 1:], q0[:, 0]]).as_matrix()
    R1 = Rotation.from_quat(np.c_[qn[:, 1:], qn[:, 0]]).as_matrix()
    np.testing.assert_allclose(R1, R0, atol=1e-12)


def test_order_is_the_stable_morton_order():
    g = synth.small(seed=6, n=500, extent=(16, 16, 16))
    hdr, streams, order = codec.encode(g.mu, g.scale, g.quat, g.alpha, bits=3)  # coarse: many equal keys
    pc, _, _ = codec.position_codes(g.mu, 3)
    keys = codec.morton(pc, 3)
    assert np.all(np.diff(keys[order].astype(np.int64)) >= 0)
    for kk in np.unique(keys):  # equal keys keep their input order
        idx = order[keys[order] == kk]
        assert np.all(np.diff(idx) > 0)


def test_zigzag_and_delta_inverses():
    d = np.array([0, 1, -1, 2, -2, 16383, -16383])
    assert list(codec.zigzag(d)) == [0, 2, 1, 4, 3, 32766, 32765]
    np.testing.assert_array_equal(codec.unzigzag(codec.zigzag(d)), d)


def test_lzma_container_round_trip():
    g = synth.small(seed=7, n=2000, extent=(64, 64, 32))
    hdr, streams, _ = codec.encode(g.mu, g.scale, g.quat, g.alpha)
    blob = codec.pack(hdr, streams)
    h2, s2 = codec.unpack(blob)
    np.testing.assert_array_equal(s2, streams)
    assert h2["n"] == hdr["n"] and h2["L0"] == hdr["L0"] and np.array_equal(h2["lo"], hdr["lo"])
    assert len(blob) < 22 * g.n  # smaller than the raw 16-bit streams


def test_bits_are_validated():
    g = synth.small(seed=8, n=10, extent=(8, 8, 8))
    with pytest.raises(ValueError):
        codec.encode(g.mu, g.scale, g.quat, g.alpha, bits=16)
