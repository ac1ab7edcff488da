"""Coefficients of the encode kernel's polynomial phasors.

A share of the encode's unit phasors exp(i 2 pi f), |f| <= 1/2 turn, is
evaluated on the FMA pipe instead of the MUFU unit: exp(i x) with x = pi f,
|x| <= pi/2, from polynomials for sin x and cos x, then squared as a complex
number (the double angle).  This script fits those polynomials:

    sin x ~ x (a0 + a1 x^2 + a2 x^4 + a3 x^6 + a4 x^8)
    cos x ~ b0 + b1 x^2 + b2 x^4 + b3 x^6 + b4 x^8

near-minimax in absolute error on [0, pi/2], by Lawson's algorithm
(iteratively reweighted least squares: the weights are multiplied by the
current absolute error, which drives the fit towards equal-ripple).  Five
terms each reach 3.3e-9 (sin) and 4.7e-8 (cos) in exact arithmetic, and about
1.5e-7 both when evaluated in float32 by Horner's rule, no worse than the
Taylor polynomials of six and seven terms they replace (2.0e-7, 1.2e-7).

Run it to print the coefficients written into csrc/encode.cu and the float32
evaluation errors:  python -m paper_2408_09066_gb300.phasor_poly
"""
import numpy as np


def lawson(basis, target, iters: int = 300):
    """Near-minimax coefficients of sum_k c_k basis_k ~ target on the grid."""
    A = np.stack(basis, 1)
    w = np.full(A.shape[0], 1.0 / A.shape[0])
    c = None
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], target * sw, rcond=None)
        err = np.abs(A @ c - target)
        w = w * err
        w /= w.sum()
    return c, float(np.abs(A @ c - target).max())


def fit(terms: int = 5, points: int = 20001):
    x = np.linspace(0.0, np.pi / 2, points)
    x2 = x * x
    a, ea = lawson([x * x2 ** k for k in range(terms)], np.sin(x))
    b, eb = lawson([x2 ** k for k in range(terms)], np.cos(x))
    return a, ea, b, eb


def horner_f32(coeffs, z):
    r = np.float32(coeffs[-1]) * np.ones_like(z)
    for c in coeffs[-2::-1]:
        r = (r * z + np.float32(c)).astype(np.float32)
    return r


def main():
    a, ea, b, eb = fit()
    xf = np.linspace(-np.pi / 2, np.pi / 2, 200001).astype(np.float32)
    z = (xf * xf).astype(np.float32)
    s = (horner_f32([np.float32(v) for v in a], z) * xf).astype(np.float32)
    c = horner_f32([np.float32(v) for v in b], z)
    x64 = xf.astype(np.float64)
    print("sin:", ", ".join("%.9e" % v for v in a), "| max error %.2e, float32 %.2e"
          % (ea, np.abs(s - np.sin(x64)).max()))
    print("cos:", ", ".join("%.9e" % v for v in b), "| max error %.2e, float32 %.2e"
          % (eb, np.abs(c - np.cos(x64)).max()))


if __name__ == "__main__":
    main()
