// Generated by gen_exp_coef.py: H(r) ~ c0 + c1 r + c2 r^2 + c3 r^3 + c4 r^4 on
// [-ln2/2, ln2/2], H(r) = (1 - exp(-r) - r)/r^2 (Chebyshev-node interpolation).
// FP64 max |H err| 6.656e-08; max relative error of r + r^2 H(r): 2.345e-08
#pragma once
#define MOC_EXP_H0 (-5.000000000e-01f)
#define MOC_EXP_H1 (1.666657776e-01f)
#define MOC_EXP_H2 (-4.166655615e-02f)
#define MOC_EXP_H3 (8.363173343e-03f)
#define MOC_EXP_H4 (-1.392617589e-03f)
