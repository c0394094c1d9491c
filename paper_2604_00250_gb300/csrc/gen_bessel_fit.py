"""Writes bessel_fit.h: float32 approximations of the modified Bessel functions
that the Rician NLL (Eq. 9) and its gradient need.

For z < ZS the kernels sum the power series (A&S 9.6.10)
    I0(z) = sum_k t^k / (k!)^2,   I1(z) = (z/2) sum_k t^k / (k! (k+1)!),   t = z^2/4,
with NSER terms. For z >= ZS they evaluate two smooth functions of x = ZS / z in (0, 1]:
    PA(x) = sqrt(2 pi z) i0e(z)            -> log i0e(z) = log PA - log(2 pi z) / 2
    PB(x) = z (1 - I1(z) / I0(z))          -> Q(z) = 1 - I1/I0 = PB / z
as degree-DEG polynomials fitted here by relative least squares on Chebyshev-spaced
nodes against scipy.special.i0e / i1e (Cephes, float64). Q is obtained directly, never
as 1 - I1/I0, so it keeps relative accuracy where I1/I0 -> 1.

Run: python gen_bessel_fit.py > bessel_fit.h
"""
import math

import numpy as np
import scipy.special as sp

ZS = 4.0
DEG = 12
NSER = 12


def fit(fun):
    xs = 0.5 * (1 - np.cos(np.linspace(0, np.pi, 4000)))
    xs = xs[xs > 1e-7]
    y = fun(ZS / xs)
    V = np.vander(xs, DEG + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V / y[:, None], np.ones_like(y), rcond=None)
    return c


def pa(z):
    return np.sqrt(2 * np.pi * z) * sp.i0e(z)


def pb(z):
    return z * (1 - sp.i1e(z) / sp.i0e(z))


def arr(name, vals):
    body = ", ".join(f"{float(v):.9e}f" for v in vals)
    return f"__device__ __constant__ float {name}[{len(vals)}] = {{{body}}};"


def arr2(name, xs, ys):
    """Two tables interleaved as float2 {x_k, y_k}: the two Horner chains that share an argument
    then run as one packed f32x2 chain."""
    body = ", ".join(f"{{{float(x):.9e}f, {float(y):.9e}f}}" for x, y in zip(xs, ys))
    return f"__device__ __constant__ float2 {name}[{len(xs)}] = {{{body}}};"


def main():
    ca = fit(pa)
    cb = fit(pb)
    s0 = [1.0 / math.factorial(k) ** 2 for k in range(NSER)]
    s1 = [1.0 / (math.factorial(k) * math.factorial(k + 1)) for k in range(NSER)]
    print("/* Generated by gen_bessel_fit.py -- do not edit. */")
    print("#pragma once")
    print(f"#define PRISM_BESSEL_ZS {ZS:.1f}f")
    print(f"#define PRISM_BESSEL_DEG {DEG}")
    print(f"#define PRISM_BESSEL_NSER {NSER}")
    print(arr("k_bessel_pa", ca))
    print(arr("k_bessel_pb", cb))
    print(arr("k_bessel_s0", s0))
    print(arr("k_bessel_s1", s1))
    print(arr2("k_bessel_pba", cb, ca))
    print(arr2("k_bessel_s01", s0, s1))


if __name__ == "__main__":
    main()
