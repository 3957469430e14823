"""Rounding of binary64 values into the value sets of the sketch number
formats.  ORACLE: test infrastructure only.

The paper computes in binary64 throughout (MATLAB, Sec. 8).  The precision
forms of this build store the tensor and the tensor-core side of the DRMs in a
narrower format; the DRM *is* the rounded matrix, so the oracle rounds the same
way and then computes exactly.  Definition used (IEEE-754 round to nearest,
ties to even, at p significand bits, with gradual underflow at exponent emin):

    q(x) = sign(x) * rint(|x| / 2^(e - p + 1)) * 2^(e - p + 1),
    e = max(floor(log2 |x|), emin)

fp32: p = 24, emin = -126, overflow -> inf.
bf16: p = 8,  emin = -126, overflow -> inf.
e4m3: p = 4,  emin = -6,   largest finite 448, overflow saturates to +-448
      (OCP FP8 E4M3 has no infinity; saturation is this build's reading).
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
