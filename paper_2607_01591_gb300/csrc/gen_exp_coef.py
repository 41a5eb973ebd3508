"""Generate the coefficients of the library's FP32 evaluation of F(tau) = 1 - exp(-tau).

Method (our own design, not a copy of any math library): write tau = n ln2 + r with n the
nearest integer to tau/ln2, so |r| <= ln2/2. Then exp(-tau) = 2^-n (1 - P(r)) with
P(r) = 1 - exp(-r) = r + r^2 H(r), and

    F(tau) = (1 - 2^-n) + 2^-n P(r),

which for n = 0 is exactly P(tau) (no cancellation for small tau). H(r) = (P(r) - r)/r^2 is
smooth; it is approximated by the degree-4 polynomial interpolating H at the 5 Chebyshev nodes of
[-ln2/2, ln2/2] (near-minimax), with coefficients rounded to FP32. Running this script rewrites
exp_f32_coef.h next to it and prints the FP64 error of the approximation of H and of P.
"""
import math
import os

import numpy as np

A = math.log(2.0) / 2.0
DEG = 4


def H(r):
    r = np.asarray(r, dtype=np.float64)
    out = np.empty_like(r)
    small = np.abs(r) < 1e-3
    rs = r[small]
    # series of (1 - e^-r - r)/r^2 = -1/2 + r/6 - r^2/24 + r^3/120 - r^4/720 + r^5/5040
    out[small] = -0.5 + rs / 6 - rs ** 2 / 24 + rs ** 3 / 120 - rs ** 4 / 720 + rs ** 5 / 5040
    rb = r[~small]
    out[~small] = (-np.expm1(-rb) - rb) / rb ** 2
    return out


def main():
    k = np.arange(DEG + 1)
    nodes = A * np.cos((2 * k + 1) * np.pi / (2 * (DEG + 1)))
    V = np.vander(nodes, DEG + 1, increasing=True)
    c = np.linalg.solve(V, H(nodes))
    c32 = c.astype(np.float32)
    r = np.linspace(-A, A, 200001)
    h_err = np.abs(np.polynomial.polynomial.polyval(r, c32.astype(np.float64)) - H(r)).max()
    P = -np.expm1(-r)
    Papprox = r + r * r * np.polynomial.polynomial.polyval(r, c32.astype(np.float64))
    nz = r != 0
    p_rel = (np.abs(Papprox - P)[nz] / np.abs(P[nz])).max()
    print(f"max |H error| = {h_err:.3e}, max relative P error (FP64 evaluation) = {p_rel:.3e}")
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "exp_f32_coef.h")
    with open(out, "w") as f:
        f.write("// Generated by gen_exp_coef.py: H(r) ~ c0 + c1 r + c2 r^2 + c3 r^3 + c4 r^4 on\n")
        f.write("// [-ln2/2, ln2/2], H(r) = (1 - exp(-r) - r)/r^2 (Chebyshev-node interpolation).\n")
        f.write(f"// FP64 max |H err| {h_err:.3e}; max relative error of r + r^2 H(r): {p_rel:.3e}\n")
        f.write("#pragma once\n")
        for i, v in enumerate(c32):
            f.write(f"#define MOC_EXP_H{i} ({float(v):.9e}f)\n")
    print("wrote", out)


if __name__ == "__main__":
    main()
