"""Oracle of the Gaussian-set codec (Sec. 4: "Quantization and compression"):
Morton (Z-order) sort, quantisation, per-attribute delta streams; LZMA on the
host.

TEST INFRASTRUCTURE ONLY (imported by tests/ and nothing in the product).

The paper fixes the steps and bit widths (positions normalised to the scene's
bounding box at typically 14 bits per axis; intensities as 12-bit integers in
[0, 1]; scales log-transformed, then 12 bits; quaternions on the positive
half-sphere at 12 bits per component; Morton order; delta coding; LZMA).  It
prints no rounding rule or container, so these readings are written here and
the device codec follows them exactly.  Every integer decision is taken in
fp32 with each operation rounded separately (numpy float32), except the
scale codes, which compare the float scale with double-precision thresholds:

* position axis k: d = hi - lo, inv = (2^B - 1) / d, code = clamp(floor((mu -
  lo) * inv + 0.5), 0, 2^B - 1); decode lo + code * (d / (2^B - 1));
* scale: L0 = ln(min s), L1 = ln(max s) over all 3n scales (double),
  D = (L1 - L0) / 4095; code = number of k in 1..4095 with s >= exp(L0 + (k -
  1/2) D) (round to nearest in the log domain); decode exp(L0 + code D);
* intensity: code = clamp(floor(clamp(alpha, 0, 1) * 4095 + 0.5), 0, 4095);
  decode code / 4095;
* quaternion: q / |q| (|q|^2 summed w, x, y, z in order), negated when w < 0
  (the same rotation); code = clamp(floor((c + 1) * 2047.5 + 0.5), 0, 4095);
  decode code / 2047.5 - 1;
* Morton key: bit 3 j + a of the key is bit j of the position code of axis a
  (x = 0, y = 1, z = 2); Gaussians are ordered by a stable sort on the key;
* streams (11, in the order x y z s0 s1 s2 qw qx qy qz alpha): first code,
  then differences of consecutive codes in Morton order, zigzag-mapped
  (d >= 0 -> 2 d, d < 0 -> -2 d - 1) to uint16 (B <= 15).
"""
from __future__ import annotations

import lzma
import struct

import numpy as np

F = np.float32
N_STREAMS = 11


def _q_affine(v, lo, inv, top):
    t = (F(v) - F(lo)).astype(F) * F(inv)
    t = (t.astype(F) + F(0.5)).astype(F)
    return np.clip(np.floor(t), 0, top).astype(np.int64)


def position_codes(mu, bits):
    mu = np.asarray(mu, F)
    top = (1 << bits) - 1
    lo = mu.min(axis=0).astype(F)
    hi = mu.max(axis=0).astype(F)
    codes = np.zeros(mu.shape, np.int64)
    for k in range(3):
        d = F(hi[k] - lo[k])
        if d > 0:
            inv = F(F(top) / d)
            codes[:, k] = _q_affine(mu[:, k], lo[k], inv, top)
    return codes, lo, hi


def scale_thresholds(L0, L1):
    D = (L1 - L0) / 4095.0
    k = np.arange(1, 4096, dtype=np.float64)
    return np.exp(L0 + (k - 0.5) * D)


def scale_codes(scale):
    s = np.asarray(scale, F)
    L0 = float(np.log(np.float64(s.min())))
    L1 = float(np.log(np.float64(s.max())))
    if L1 == L0:
        return np.zeros(s.shape, np.int64), L0, L1
    th = scale_thresholds(L0, L1)
    return np.searchsorted(th, s.astype(np.float64), side="right").astype(np.int64), L0, L1


def alpha_codes(alpha):
    a = np.clip(np.asarray(alpha, F), F(0), F(1)).astype(F)
    t = (a * F(4095)).astype(F)
    return np.clip(np.floor((t + F(0.5)).astype(F)), 0, 4095).astype(np.int64)


def quat_codes(quat):
    q = np.asarray(quat, F)
    n2 = (q[:, 0] * q[:, 0]).astype(F)
    for k in (1, 2, 3):
        n2 = (n2 + (q[:, k] * q[:, k]).astype(F)).astype(F)
    nrm = np.sqrt(n2).astype(F)
    safe = np.where(nrm > 0, nrm, F(1)).astype(F)
    c = np.where(nrm[:, None] > 0, (q / safe[:, None]).astype(F), F(0)).astype(F)
    c = np.where(c[:, :1] < 0, -c, c).astype(F)
    t = ((c + F(1)).astype(F) * F(2047.5)).astype(F)
    return np.clip(np.floor((t + F(0.5)).astype(F)), 0, 4095).astype(np.int64)


def morton(codes, bits):
    key = np.zeros(codes.shape[0], np.uint64)
    for j in range(bits):
        for a in range(3):
            key |= ((codes[:, a].astype(np.uint64) >> np.uint64(j)) & np.uint64(1)) << np.uint64(3 * j + a)
    return key


def zigzag(d):
    d = np.asarray(d, np.int64)
    return np.where(d >= 0, 2 * d, -2 * d - 1)


def unzigzag(z):
    z = np.asarray(z, np.int64)
    return np.where(z % 2 == 0, z // 2, -(z + 1) // 2)


def encode(mu, scale, quat, alpha, bits=14):
    """(header dict, streams uint16 [11, n], order [n]): order[i] is the input
    index of the i-th encoded Gaussian."""
    if not 1 <= bits <= 15:
        raise ValueError("bits must be in 1..15")
    pc, lo, hi = position_codes(mu, bits)
    sc, L0, L1 = scale_codes(scale)
    qc = quat_codes(quat)
    ac = alpha_codes(alpha)
    order = np.argsort(morton(pc, bits), kind="stable")
    all_codes = np.concatenate([pc, sc, qc, ac[:, None]], axis=1)[order]  # [n, 11]
    d = np.diff(all_codes, axis=0, prepend=np.zeros((1, N_STREAMS), np.int64))
    streams = zigzag(d).T.astype(np.uint16)
    header = {"n": int(np.asarray(alpha).shape[0]), "bits": bits, "lo": lo, "hi": hi, "L0": L0, "L1": L1}
    return header, streams, order


def decode(header, streams):
    """(mu, scale, quat, alpha) float32 in the encoded (Morton) order."""
    codes = np.cumsum(unzigzag(np.asarray(streams, np.int64)), axis=1).T  # [n, 11]
    bits = header["bits"]
    top = F((1 << bits) - 1)
    lo, hi = np.asarray(header["lo"], F), np.asarray(header["hi"], F)
    mu = np.empty((codes.shape[0], 3), F)
    for k in range(3):
        step = F(F(hi[k] - lo[k]) / top)
        mu[:, k] = (lo[k] + (codes[:, k].astype(F) * step).astype(F)).astype(F)
    L0, L1 = header["L0"], header["L1"]
    D = (L1 - L0) / 4095.0
    scale = np.exp(L0 + codes[:, 3:6].astype(np.float64) * D).astype(F)
    quat = ((codes[:, 6:10].astype(F) / F(2047.5)).astype(F) - F(1)).astype(F)
    alpha = (codes[:, 10].astype(F) / F(4095)).astype(F)
    return mu, scale, quat, alpha


_HDR = struct.Struct("<qi3f3f2d")


def pack(header, streams) -> bytes:
    """Container: header then the 11 streams (uint16 little-endian), LZMA-compressed."""
    raw = _HDR.pack(header["n"], header["bits"], *[float(x) for x in header["lo"]],
                    *[float(x) for x in header["hi"]], header["L0"], header["L1"])
    return lzma.compress(raw + np.ascontiguousarray(streams, "<u2").tobytes())


def unpack(blob: bytes):
    raw = lzma.decompress(blob)
    n, bits, lx, ly, lz, hx, hy, hz, L0, L1 = _HDR.unpack_from(raw)
    streams = np.frombuffer(raw, "<u2", offset=_HDR.size).reshape(N_STREAMS, n)
    return ({"n": n, "bits": bits, "lo": np.array([lx, ly, lz], F), "hi": np.array([hx, hy, hz], F),
             "L0": L0, "L1": L1}, streams)
