"""Helpers shared by the GPU parity tests (no arithmetic of the operator here)."""
import numpy as np
import torch

from paper_2603_20611_b300 import binding as B

# Parity bars (the operator's stated tolerances): forward relative L2 <= 1e-5 and
# max abs <= 1e-4 of the oracle's peak; gradients relative L2 <= 1e-3 per group.
FWD_REL_L2 = 1e-5
FWD_MAX_ABS_FRAC = 1e-4
GRAD_REL_L2 = 1e-3


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def assert_forward_close(gpu, ref, what=""):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    peak = float(np.abs(ref).max()) if ref.size else 0.0
    r = rel_l2(gpu, ref)
    m = float(np.abs(gpu - ref).max()) if ref.size else 0.0
    assert r <= FWD_REL_L2, f"{what}: forward rel L2 {r:.3e} > {FWD_REL_L2}"
    assert m <= FWD_MAX_ABS_FRAC * max(peak, 1e-30), f"{what}: max abs {m:.3e} > 1e-4 * peak {peak:.3e}"


def assert_grads_close(gpu, ref, what="", tol=GRAD_REL_L2):
    names = ("mu", "scale", "quat", "alpha")
    for name, g, r in zip(names, gpu, ref):
        g = g.detach().cpu().numpy() if isinstance(g, torch.Tensor) else g
        e = rel_l2(g, r)
        assert e <= tol, f"{what}: d{name} rel L2 {e:.3e} > {tol}"


def dev_set(g, scale_mod=1.0):
    return B.GaussianSet.from_numpy(g, "cuda", scale_mod)


def np32(t):
    return t.detach().cpu().numpy().astype(np.float64)
