"""Rounding of binary64 values into the value sets of the sketch number
formats.  ORACLE: test infrastructure only.

The paper computes in binary64 throughout (MATLAB, Sec. 8).  The precision
forms of this library store the tensor and the tensor-core side of the DRMs in a
narrower format; the DRM *is* the rounded matrix, so the oracle rounds the same
way and then computes exactly.  Definition used (IEEE-754 round to nearest,
ties to even, at p significand bits, with gradual underflow at exponent emin):

    q(x) = sign(x) * rint(|x| / 2^(e - p + 1)) * 2^(e - p + 1),
    e = max(floor(log2 |x|), emin)

fp32: p = 24, emin = -126, overflow -> inf.
bf16: p = 8,  emin = -126, overflow -> inf.
e4m3: p = 4,  emin = -6,   largest finite 448, overflow saturates to +-448
      (OCP FP8 E4M3 has no infinity; saturation is this library's reading).
"""
import numpy as np

FORMATS = {
    "f64": None,
    "f32": (24, -126, float(np.finfo(np.float32).max), "inf"),
    "bf16": (8, -126, float.fromhex("0x1.fep127"), "inf"),
    "e4m3": (4, -6, 448.0, "sat"),
}


def round_to(x, fmt):
    """Round binary64 array x to the value set of fmt (RNE), returned as f64."""
    x = np.asarray(x, dtype=np.float64)
    spec = FORMATS[fmt]
    if spec is None:
        return x.copy()
    p, emin, vmax, overflow = spec
    a = np.abs(x)
    _, fe = np.frexp(a)                     # a = m 2^fe, m in [0.5, 1)
    e = np.maximum(fe.astype(np.int64) - 1, emin)
    scale_exp = e - (p - 1)
    q = np.rint(np.ldexp(a, -scale_exp))    # exact scaling, then RNE
    r = np.ldexp(q, scale_exp)
    r = np.where(a == 0.0, 0.0, r)
    if overflow == "inf":
        r = np.where(r > vmax, np.inf, r)
    else:
        r = np.minimum(r, vmax)
    return np.copysign(r, x)


def eps_of(fmt):
    """Unit roundoff 2^-p of a format (binary64: 2^-53)."""
    return {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "bf16": 2.0 ** -8, "e4m3": 2.0 ** -4}[fmt]


# ---------------------------------------------------------------------------
# Precision forms of the first-level pass (the tensor's storage formats)
# ---------------------------------------------------------------------------
# BF16x2 split: a binary32 tensor A is carried as two bfloat16 tensors,
#   hi = bf16(A),  lo = bf16(A - hi)   (A - hi is exact in binary32),
# and the pass multiplies both by the same bfloat16 DRM block, so the tensor it
# sketches is hi + lo (|A - (hi + lo)| <= 2^-17 |A| away from A, normal range).
#
# FP8 E4M3 with one binary32 scale per 128 x 128 tile of the pass matrix M
# (rows = the root's left-group modes, columns = the rest):
#   s = max|tile| / 448 (binary32 division; s = 1 for an all-zero tile),
#   q = e4m3(A / s)     (binary32 division, then nearest-even, saturating),
# and the pass multiplies the dequantised tile  bf16(f32(q * s))  on the
# bfloat16 tensor cores: the tensor it sketches is that dequantised matrix.

E4M3_MAX = 448.0
TILE = 128


def split_bf16x2(A):
    """(hi, lo) of a binary32-valued array, both bfloat16 values as f64."""
    A = np.asarray(A, dtype=np.float64)
    hi = round_to(A, "bf16")
    lo = round_to(A - hi, "bf16")
    return hi, lo


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fp8_tile_quantize(M):
    """Per-tile E4M3 quantisation of a 2-D binary32-valued matrix M.
    Returns (q, scales): q the E4M3 values (f64 array, M's shape), scales the
    binary32 scale of each 128 x 128 tile (f64 array [row tiles][col tiles])."""
    M32 = _f32(M)
    rows, cols = M32.shape
    nrt, nct = -(-rows // TILE), -(-cols // TILE)
    scales = np.zeros((nrt, nct))
    q = np.zeros(M32.shape)
    for bi in range(nrt):
        for bj in range(nct):
            t = M32[bi * TILE:(bi + 1) * TILE, bj * TILE:(bj + 1) * TILE]
            mx = np.float32(np.max(np.abs(t))) if t.size else np.float32(0)
            s = np.float32(1.0) if mx == 0 else np.float32(mx / np.float32(E4M3_MAX))
            scales[bi, bj] = float(s)
            q[bi * TILE:(bi + 1) * TILE, bj * TILE:(bj + 1) * TILE] = round_to(
                (t / s).astype(np.float64), "e4m3")
    return q, scales


def fp8_dequantize_bf16(q, scales):
    """bf16(f32(q * s)) per tile: the matrix the E4M3 pass sketches."""
    q = np.asarray(q, dtype=np.float64)
    rows, cols = q.shape
    s = np.repeat(np.repeat(np.asarray(scales, dtype=np.float64), TILE, 0), TILE, 1)[:rows, :cols]
    prod = (_f32(q) * _f32(s)).astype(np.float64)     # one binary32 rounding
    return round_to(prod, "bf16")


def e4m3_encode(v):
    """E4M3 bytes (uint8) of E4M3 values (sign, 4-bit exponent bias 7, 3-bit
    mantissa; exponent field 0 = subnormals 2^-6 * m/8)."""
    v = np.asarray(v, dtype=np.float64)
    sign = np.signbit(v).astype(np.uint8) << 7
    a = np.abs(v)
    out = np.zeros(a.shape, dtype=np.uint8)
    sub = a < 2.0 ** -6
    m_sub = np.rint(a / 2.0 ** -9).astype(np.int64)
    _, fe = np.frexp(np.where(sub, 1.0, a))
    e = fe.astype(np.int64) - 1
    m_norm = np.rint((np.where(sub, 1.0, a) / np.ldexp(1.0, e) - 1.0) * 8).astype(np.int64)
    code = np.where(sub, m_sub, ((e + 7) << 3) | m_norm)
    out[...] = code.astype(np.uint8)
    return out | sign


def e4m3_decode(b):
    """E4M3 values (f64) of bytes; the code 0x7f / 0xff is NaN."""
    b = np.asarray(b, dtype=np.uint8).astype(np.int64)
    s = np.where(b & 0x80, -1.0, 1.0)
    e = (b >> 3) & 0xF
    m = b & 0x7
    v = np.where(e == 0, m / 8.0 * 2.0 ** -6, (1 + m / 8.0) * np.ldexp(1.0, e - 7))
    v = np.where((e == 15) & (m == 7), np.nan, v)
    return s * v
