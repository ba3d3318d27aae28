"""Derive the polynomial coefficients of the library's Box-Muller kernels.

    python paper_2310_19925_b300/csrc/fit_boxmuller.py

This is a development tool; the build does not run it.  It prints the
float32 coefficients used in include/orand_device.cuh together with their
worst-case errors.  The method is the textbook one (argument reduction plus a
near-minimax polynomial; Cody & Waite 1980, Muller 2016 "Elementary
Functions", ch. 3):

  * log:  u1 = 2^e * f with f in [sqrt(2)/2, sqrt(2)), g = f - 1 (exact),
          ln(1+g) = g + g^2 * PL(g), PL ~ (ln(1+g) - g) / g^2.
  * sinpi/cospi on r in [-1/4, 1/4], t = r^2:
          sin(pi r) = r * (PI_HI + (PI_LO + t * QS(t))), evaluated as
          fma(r, PI_HI, r * (PI_LO + t * QS(t))) so that the leading term
          pi r is rounded once (pi = PI_HI + PI_LO, both float32);
          cos(pi r) = 1 + t * QC(t), evaluated as fma(t, QC(t), 1).

Each polynomial is a weighted least-squares fit on Chebyshev nodes.  The
weights come from Lawson's iteration, which drives the fit towards the
minimax (equioscillating) relative error.  The coefficients are then rounded
to float32, and the worst error is measured in float64 over a dense grid.
"""
import numpy as np


def cheb_nodes(a, b, n):
    k = np.arange(n)
    return 0.5 * (a + b) + 0.5 * (b - a) * np.cos(np.pi * (k + 0.5) / n)


def lawson_fit(x, y, deg, iters=200):
    """Polynomial coefficients c[0..deg] (lowest first) approximately
    minimising max |(p(x) - y) / y| via Lawson's reweighted least squares."""
    V = np.vander(x, deg + 1, increasing=True)
    w = np.ones_like(x) / len(x)
    scale = 1.0 / np.abs(y)
    c = None
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * (sw * scale)[:, None], y * sw * scale, rcond=None)
        err = np.abs(V @ c - y) * scale
        w = w * err
        w /= w.sum()
    return c


def horner(c, x):
    acc = np.zeros_like(x) + c[-1]
    for ci in c[-2::-1]:
        acc = acc * x + ci
    return acc


def fit_log():
    lo, hi = np.sqrt(0.5) - 1.0, np.sqrt(2.0) - 1.0
    g = cheb_nodes(lo, hi, 4000)
    g = g[np.abs(g) > 1e-6]
    y = (np.log1p(g) - g) / g ** 2
    c = np.float32(lawson_fit(g, y, 8)).astype(np.float64)
    gg = np.linspace(lo, hi, 200001)
    gg = gg[np.abs(gg) > 1e-9]
    yy = (np.log1p(gg) - gg) / gg ** 2
    rel = np.max(np.abs(horner(c, gg) - yy) / np.abs(yy))
    return c, rel


PI_HI = float(np.float32(np.pi))
PI_LO = float(np.float32(np.pi - PI_HI))


def fit_sinpi():
    """QS(t) ~ (sin(pi sqrt t) / sqrt t - pi) / t on t in (0, 1/16]."""
    t = cheb_nodes(0.0, 1.0 / 16, 2000)
    r = np.sqrt(t)
    y = (np.sin(np.pi * r) / r - np.pi) / t
    c = np.float32(lawson_fit(t, y, 3)).astype(np.float64)
    tt = np.linspace(1e-9, 1.0 / 16, 200001)
    yy = (np.sin(np.pi * np.sqrt(tt)) / np.sqrt(tt) - np.pi) / tt
    return c, np.max(np.abs(horner(c, tt) - yy) / np.abs(yy))


def fit_cospi():
    """QC(t) ~ (cos(pi sqrt t) - 1) / t on t in (0, 1/16]."""
    t = cheb_nodes(0.0, 1.0 / 16, 2000)
    y = (np.cos(np.pi * np.sqrt(t)) - 1.0) / t
    c = np.float32(lawson_fit(t, y, 4)).astype(np.float64)
    tt = np.linspace(1e-9, 1.0 / 16, 200001)
    yy = (np.cos(np.pi * np.sqrt(tt)) - 1.0) / tt
    return c, np.max(np.abs(horner(c, tt) - yy) / np.abs(yy))


if __name__ == "__main__":
    print("PI_HI = %r (%#010x), PI_LO = %r (%#010x)" % (np.float32(PI_HI), np.float32(PI_HI).view(np.uint32),
                                                     np.float32(PI_LO), np.float32(PI_LO).view(np.uint32)))
    for name, fn in [("PL (log)", fit_log), ("QS (sinpi)", fit_sinpi), ("QC (cospi)", fit_cospi)]:
        c, rel = fn()
        print("%s: max relative error %.3g (%.2f ulp of 2^-24)" % (name, rel, rel * 2 ** 24))
        for i, ci in enumerate(c):
            print("  c%d = %s  (%.9e)" % (i, np.float32(ci).view(np.uint32).__format__("#010x"), np.float32(ci)))
