"""FP64 oracle of the fit loop's parameter update.

TEST INFRASTRUCTURE ONLY (imported by tests/ and nothing in the product).

The paper trains with Adam (Kingma & Ba 2015) for 30k iterations, with initial
learning rates 6e-4 (position), 2e-2 (opacity / intensity), 2e-3 (scale) and
1e-3 (rotation), each decaying exponentially to 0.1 of its initial value
(Sec. 5.1, implementation details).  Written here from those definitions:

* Adam, one step t = 1, 2, ... for a parameter theta with gradient g:
      m <- b1 m + (1 - b1) g,     v <- b2 v + (1 - b2) g^2,
      theta <- theta - lr_t * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps);
* the schedule: lr_t = lr_0 * r^(k / K) with k = t - 1 clipped to [0, K],
  r = 0.1 the final ratio and K the number of iterations (so the first step
  uses lr_0 and step K + 1 onward uses r lr_0);
* the parameterisation (readings, not printed in the paper): the scale and the
  intensity are optimised as log s and logit alpha -- the Gaussian-splatting
  pipeline the paper says it follows -- so their gradients are
  g_log_s = g_s * s and g_logit = g_alpha * alpha (1 - alpha); positions and
  quaternions are optimised as they are; the position rate is relative to the
  scene extent (multiplied by `extent`).
"""
from __future__ import annotations

import numpy as np

PAPER_LR = {"mu": 6e-4, "scale": 2e-3, "quat": 1e-3, "alpha": 2e-2}
GROUPS = ("mu", "scale", "quat", "alpha")


def lr_at(lr0: float, t: int, total: int, final_ratio: float = 0.1) -> float:
    k = min(max(t - 1, 0), total)
    return lr0 * final_ratio ** (k / total)


def adam_update(theta, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """One Adam step (Algorithm 1 of Kingma & Ba) in FP64; returns (theta, m, v)."""
    theta = np.asarray(theta, np.float64)
    g = np.asarray(g, np.float64)
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def logit(a):
    a = np.clip(np.asarray(a, np.float64), 1e-6, 1.0 - 1e-6)
    return np.log(a) - np.log1p(-a)


class FitState:
    """Optimiser state of one Gaussian set: raw parameters, first and second moments."""

    def __init__(self, mu, scale, quat, alpha, log_scale_logit_alpha=True):
        self.act = bool(log_scale_logit_alpha)
        self.raw = {"mu": np.array(mu, np.float64), "quat": np.array(quat, np.float64),
                    "scale": np.log(np.asarray(scale, np.float64)) if self.act else np.array(scale, np.float64),
                    "alpha": logit(alpha) if self.act else np.array(alpha, np.float64)}
        self.m = {k: np.zeros_like(v) for k, v in self.raw.items()}
        self.v = {k: np.zeros_like(v) for k, v in self.raw.items()}

    def params(self):
        """The parameters the renderer takes (scale and intensity activated)."""
        if self.act:
            s = np.exp(self.raw["scale"])
            a = 1.0 / (1.0 + np.exp(-self.raw["alpha"]))
        else:
            s, a = self.raw["scale"], self.raw["alpha"]
        return self.raw["mu"], s, self.raw["quat"], a

    def step(self, grads, t, lrs=PAPER_LR, total=30000, final_ratio=0.1, extent=1.0, beta1=0.9, beta2=0.999,
             eps=1e-15):
        """Applies one update given dL/d(mu, scale, quat, alpha) of the rendered parameters."""
        _, s, _, a = self.params()
        g = dict(zip(GROUPS, (np.asarray(x, np.float64) for x in grads)))
        if self.act:
            g["scale"] = g["scale"] * s
            g["alpha"] = g["alpha"] * a * (1.0 - a)
        for k in GROUPS:
            lr = lr_at(lrs[k] * (extent if k == "mu" else 1.0), t, total, final_ratio)
            self.raw[k], self.m[k], self.v[k] = adam_update(self.raw[k], g[k].reshape(self.raw[k].shape),
                                                            self.m[k], self.v[k], t, lr, beta1, beta2, eps)
        return self.params()


__all__ = ["PAPER_LR", "GROUPS", "lr_at", "adam_update", "logit", "FitState"]
