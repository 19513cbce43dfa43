"""Derives the coefficients of the rasterisers' exp2 polynomials.

2^x = 2^n * 2^f with n = round(x) and f = x - n in [-1/2, 1/2]; 2^f is
approximated by a polynomial p(f) with p(0) = 1 exactly, chosen to minimise
the maximum RELATIVE error |p(f) / 2^f - 1| on [-1/2, 1/2] by the Remez
exchange algorithm (equioscillation at deg + 1 points once the constant term
is fixed).  The coefficients are then rounded to fp32 and the error of the
rounded polynomial, evaluated by Horner's rule in fp32 arithmetic (emulated
with numpy float32, separate multiply and add roundings), is reported.

Two degrees: 6 (GP_EXP2_C*, about 2 ulp: the forward's pixels, which the
images need to fp32 accuracy) and 4 (GP_EXP2G_C*, 3.6e-6 relative: the
exponentials the backward recomputes, whose gradients are held to 1e-3).

Run: python exp2_poly.py   (prints the C initialisers used in gp_common.cuh)
"""
import numpy as np

DEG = 6
LO, HI = -0.5, 0.5


def remez(deg=DEG, iters=30):
    # unknowns: c1..c_deg and the levelled error E; p(f) = 1 + sum c_k f^k
    k = np.arange(1, deg + 1)
    m = deg + 1  # number of reference points
    x = 0.5 * (LO + HI) + 0.5 * (HI - LO) * np.cos(np.pi * np.arange(m)[::-1] / (m - 1))
    g = np.linspace(LO, HI, 200001)
    for _ in range(iters):
        t = np.exp2(x)
        # p(x_i) / t_i - 1 = (-1)^i E  ->  sum c_k x_i^k - (-1)^i E t_i = t_i - 1
        A = np.zeros((m, deg + 1))
        A[:, :deg] = x[:, None] ** k[None, :]
        A[:, deg] = -((-1.0) ** np.arange(m)) * t
        sol = np.linalg.solve(A, t - 1.0)
        c = sol[:deg]
        err = (1.0 + (g[:, None] ** k[None, :]) @ c) / np.exp2(g) - 1.0
        # new reference: alternating extrema of the error curve
        idx = [0]
        for i in range(1, len(g) - 1):
            if (err[i] - err[i - 1]) * (err[i + 1] - err[i]) <= 0:
                idx.append(i)
        idx.append(len(g) - 1)
        pts = []
        for i in idx:
            if pts and np.sign(err[i]) == np.sign(err[pts[-1]]):
                if abs(err[i]) > abs(err[pts[-1]]):
                    pts[-1] = i
            else:
                pts.append(i)
        while len(pts) > m:
            if abs(err[pts[0]]) < abs(err[pts[-1]]):
                pts.pop(0)
            else:
                pts.pop()
        if len(pts) == m:
            x = g[np.array(pts)]
    return c, float(np.max(np.abs(err)))


def horner_f32(c32, f):
    f = f.astype(np.float32)
    p = np.full_like(f, c32[-1])
    for ck in c32[-2::-1]:
        p = (p * f + np.float32(ck)).astype(np.float32)
    p = (p * f + np.float32(1.0)).astype(np.float32)
    return p


if __name__ == "__main__":
    for deg, name in ((DEG, "GP_EXP2_C"), (4, "GP_EXP2G_C")):
        c, e = remez(deg)
        c32 = c.astype(np.float32)
        g = np.linspace(LO, HI, 2000001)
        rel = horner_f32(c32, g).astype(np.float64) / np.exp2(g) - 1.0
        print(f"// degree {deg}, levelled relative error {e:.3e}, fp32 Horner max rel err "
              f"{np.max(np.abs(rel)):.3e} ({np.max(np.abs(rel)) / 2**-24:.2f} ulp of 2^-24)")
        for i, ck in enumerate(c32, start=1):
            print(f"#define {name}{i} {float(ck)!r}f")
