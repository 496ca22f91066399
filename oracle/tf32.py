"""TF32 split products: the error model of the mixed path's tensor-core
products (TEST INFRASTRUCTURE; only the tests may import it).

The mixed path multiplies FP32 blocks on the tensor cores with the 3xTF32
split product.  TF32 keeps 10 explicit mantissa bits (11 significant bits)
and the FP32 exponent.  Each FP32 value is split as
    x_hi = tf32(x),   x_lo = tf32(x - x_hi)
(x - x_hi is exact in FP32), and
    X Y^T ~ X_hi Y_hi^T + X_hi Y_lo^T + X_lo Y_hi^T,
dropping X_lo Y_lo^T, which is below FP32 rounding.  Rounding to TF32 is to
nearest with ties away from zero (the reading taken of "3xTF32": PTX
cvt.rna.tf32.f32).

Here the three partial products are formed in float64, where the product of
two 11-bit significands is exact and sums of up to 2^31 such terms of
comparable size lose nothing that matters at FP32 level, so the result is the
split product itself without the accumulation error of the hardware.
"""
import numpy as np


def tf32_rna(a):
    """Round FP32 values to TF32: add half a TF32 unit in the last place to the
    magnitude bits and clear the 13 bits below it (nearest, ties away from
    zero; the sign bit is untouched)."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    sign = u & 0x80000000
    mag = ((u & 0x7FFFFFFF) + 0x1000) & 0x7FFFE000
    return (sign | mag).astype(np.uint32).view(np.float32)


def split(a):
    """(x_hi, x_lo) with x_hi = tf32(x), x_lo = tf32(x - x_hi), both FP32."""
    a = np.asarray(a, dtype=np.float32)
    hi = tf32_rna(a)
    lo = tf32_rna((a - hi).astype(np.float32))
    return hi, lo


def product_3xtf32(X, Y):
    """The split product X Y^T ~ X_hi Y_hi^T + X_hi Y_lo^T + X_lo Y_hi^T of FP32
    matrices X [.., n, k], Y [.., m, k], formed in float64."""
    Xh, Xl = (v.astype(np.float64) for v in split(X))
    Yh, Yl = (v.astype(np.float64) for v in split(Y))
    mm = lambda A, B: np.einsum("...ik,...jk->...ij", A, B)
    return mm(Xh, Yh) + mm(Xh, Yl) + mm(Xl, Yh)
