"""CPU checks of the arithmetic that two mixed-precision kernels rely on, against plain FP64 numpy.

1. Difference form of the lowest imaginary-grid columns of the W table: with M = Pi(i xi) - Pi(0), which has the
   closed form 4 xi^2 sum_ia B_ia B_ia^T / (D_ia (D_ia^2 + xi^2)), eps(i xi) = eps(0) - M and therefore
   eps(i xi)^-1 - eps(0)^-1 = eps(i xi)^-1 M eps(0)^-1, so W(i xi) - W(0) = y_xi^T M y_0 with y = eps^-1 b.
2. Double-float multiply-add (FP32 pairs): the exact-product and TwoSum steps of the refinement residual GEMMs,
   emulated here step by step in float32 (an FMA is emulated by its exact float64 value rounded once to float32,
   which is what a fused multiply-add returns for these operands), reach close to 48-bit accuracy on a long,
   cancelling dot product, where plain float32 accumulation stays near 24 bits.
"""
import math

import numpy as np

from oracle import gw_oracle as O
from paper_2107_10423_gb300 import synth


def test_difference_form_of_the_w_table():
    s = synth.water_cluster(2, 7)
    B = s.b_ia()
    D = O.pair_energies(s.eps, s.n_occ)
    Bn = s.b_nm()[0]                       # rows b_m of the first target
    P0 = O.pi_imag(s.eps, s.n_occ, B, 0.0)
    eps0_inv = np.linalg.inv(np.eye(P0.shape[0]) - P0)
    for xi in (4.4e-5, 2.3e-4, 3e-3):
        M = (B * (4.0 * xi * xi / (D * (D * D + xi * xi)))) @ B.T
        Pg = O.pi_imag(s.eps, s.n_occ, B, xi)
        assert np.abs(M - (Pg - P0)).max() < 1e-12 * np.abs(P0).max()
        epsg_inv = np.linalg.inv(np.eye(P0.shape[0]) - Pg)
        for b in Bn[:5]:
            direct = O.w_corr(Pg, b) - O.w_corr(P0, b)
            form = (epsg_inv @ b) @ M @ (eps0_inv @ b)
            # the difference is O(xi^2); the form keeps its relative accuracy
            assert abs(form - direct) <= 1e-9 * abs(O.w_corr(P0, b)) + 1e-6 * abs(form), (xi, form, direct)


def _f32(x):
    return np.float32(x)


def _fma32(a, b, c):
    """float32 fused multiply-add: the float64 value of a*b + c is exact here or within one float64 rounding,
    then rounded once to float32."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _df_dot(x, y):
    xh = x.astype(np.float32)
    xl = (x - xh.astype(np.float64)).astype(np.float32)
    yh = y.astype(np.float32)
    yl = (y - yh.astype(np.float64)).astype(np.float32)
    sh, sl = np.float32(0.0), np.float32(0.0)
    for ah, al, bh, bl in zip(xh, xl, yh, yl):
        ph = _f32(ah * bh)
        pe = _fma32(ah, bh, -ph)
        pe = _fma32(ah, bl, pe)
        pe = _fma32(al, bh, pe)
        t = _f32(sh + ph)
        v = _f32(t - sh)
        e = _f32(_f32(sh - _f32(t - v)) + _f32(ph - v))
        sl = _f32(sl + _f32(e + pe))
        sh = t
    return np.float64(sh) + np.float64(sl)


def test_double_float_dot_product_accuracy():
    rng = np.random.default_rng(5)
    n = 4096
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    y[n // 2:] = -y[: n // 2] * (x[: n // 2] / x[n // 2:])      # strong cancellation: the sum is tiny
    y[0] += 1e-3
    terms = x * y
    exact = math.fsum(terms)
    scale = float(np.abs(terms).sum())
    err_df = abs(_df_dot(x, y) - exact) / scale
    acc32 = np.float32(0.0)
    for a, b in zip(x.astype(np.float32), y.astype(np.float32)):
        acc32 = _fma32(a, b, acc32)
    err_32 = abs(float(acc32) - exact) / scale
    print(f"relative to sum|x_i y_i|: double-float {err_df:.2e}, float32 {err_32:.2e}")
    assert err_df < 2.0 ** -44, err_df
    assert err_32 > 2.0 ** -30, err_32      # the plain FP32 sum is far worse: the pair arithmetic is what helps
