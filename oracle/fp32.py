"""Exact IEEE-754 binary32 emulation for the oracle's integer-valued decisions.

TEST INFRASTRUCTURE ONLY: nothing on the product path imports this module.

Two decisions of the method are integers decided by floating point: whether a
Gaussian's 3-sigma circle touches a tile (Sec. 3.2, the tile-circle test that
defines S_j) and which K Gaussians rank first at a pixel (Sec. 3.2, top-K by
Gaussian value). The CUDA path takes both decisions in binary32 with every
operation rounded once (round-to-nearest-even), in the operation order fixed by
the library's header. The oracle therefore takes the same decisions in the same
precision, through the helpers below, and computes every *value* in float64.

numpy's float32 add, subtract, multiply and divide are single IEEE operations
(one rounding each), so they are used as they are. numpy has no fused
multiply-add; `fma32` provides one with a single rounding, built from the
round-to-odd theorem (Boldo and Melquiond, "Emulation of FMA and correctly
rounded sums: proved algorithms using rounding to odd", IEEE TC 2008): a sum
rounded to odd in a format with at least p+2 bits of precision, then rounded to
nearest in precision p, equals the exact sum rounded to nearest in precision p.
float64 has 53 >= 24 + 2 bits.
"""
import numpy as np

F32 = np.float32
F64 = np.float64


def f32(x):
    """Round to binary32 (round-to-nearest-even), as an ndarray of float32."""
    return np.asarray(x).astype(F32)


def _two_sum(a, b):
    """Knuth's TwoSum in float64: s = fl(a+b) and e with a + b = s + e exactly."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def fma32(a, b, c):
    """a*b + c rounded once to binary32, for binary32 inputs.

    The product of two binary32 significands (24 bits each) is exact in
    float64. The float64 sum s = fl(p + c) and its exact error e come from
    TwoSum; the exact sum is then rounded to odd in float64 (s itself when e is
    zero or s's last bit is already odd, else the float64 neighbour of s on
    e's side, which then has an odd last bit), and that value is rounded to
    nearest binary32.
    """
    a = np.asarray(a, dtype=F32).astype(F64)
    b = np.asarray(b, dtype=F32).astype(F64)
    c = np.asarray(c, dtype=F32).astype(F64)
    p = a * b
    s, e = _two_sum(p, c)
    s = np.asarray(s, dtype=F64)
    e = np.asarray(e, dtype=F64)
    odd = (s.view(np.uint64) & np.uint64(1)) == np.uint64(1)
    toward = np.where(e > 0, np.inf, -np.inf)
    neighbour = np.nextafter(s, toward)
    ro = np.where((e == 0) | odd, s, neighbour)
    return ro.astype(F32)
