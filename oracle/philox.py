"""Philox4x32-10 and the Gaussian transform that draws the DRMs.  ORACLE: test
infrastructure only.

The paper draws Gaussian dimension reduction matrices (Sec. 4, eq. (sketch);
Sec. 7, per-mode factors X_i, Y_i) with MATLAB ``randn``.  This build needs the
host and the device to draw bit-identical matrices, so the draw is defined
here from published methods only:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): 10 rounds of the Philox S-box with multipliers
  0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
  Pinned by the Random123 known-answer vectors in tests/golden/philox_kat.txt.
* Two 53-bit uniforms per call: u1 = (top53(w0:w1) + 1) * 2^-53 in (0, 1],
  u2 = top53(w2:w3) * 2^-53 in [0, 1).
* Box-Muller (Box & Muller 1958): z0 = R cos(2 pi u2), z1 = R sin(2 pi u2),
  R = sqrt(-2 ln u1).  ln, sin and cos are evaluated here from their Taylor /
  atanh series with separately rounded IEEE-754 binary64 +, -, *, / and sqrt
  only (no fused multiply-add), so any IEEE machine evaluating the same
  operation sequence gets the same bits.

Counter layout (this library's own): element (i, j) of a factor of kind K with
identifier ID takes counter (i, j >> 1, (K << 24) | ID, 0) and key
(seed mod 2^32, seed >> 32); even j takes z0, odd j takes z1.  An element's
value therefore does not depend on the matrix width, so a DRM with r columns
is the first r columns of one with more (the paper's single r, Sec. 7, read
per node).
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)

# factor kinds (the third counter word's top byte)
KIND_X = 1    # per-mode right factor X_mu (n_mu x r)          Sec. 7
KIND_Y = 2    # per-mode left factor Y_mu (n_mu x (r + p))      Sec. 7
KIND_XT = 3   # STTNN right factor on a contracted group (s_s x r)   Sec. 5
KIND_DX = 4   # unstructured Gaussian X_{l,k} (oracle only)     eq. (sketch)
KIND_DY = 5   # unstructured Gaussian Y_{l,k} (oracle only)     eq. (sketch)

# binary64 constants: the nearest doubles to ln 2, sqrt 2 and pi / 4
LN2 = 0.6931471805599453
SQRT2 = 1.4142135623730951
PI_4 = 0.7853981633974483
LN_TERMS = 11     # atanh series terms: z^(2k) / (2k + 1), k = 0..11
SIN_TERMS = 8     # sin series to psi^17 / 17!
COS_TERMS = 9     # cos series to psi^18 / 18!


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit counters (held in uint64).

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
    the key is advanced by the Weyl increments between rounds.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK32
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for _ in range(10):
        p0 = m0 * c0          # < 2^64: exact in uint64
        p1 = m1 * c2
        n0 = (p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0)
        n1 = p1 & _MASK32
        n2 = (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1)
        n3 = p0 & _MASK32
        c0, c1, c2, c3 = n0, n1, n2, n3
        k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def uniforms(w0, w1, w2, w3):
    """Two binary64 uniforms from one Philox output: u1 in (0,1], u2 in [0,1)."""
    hi = (w0 << np.uint64(32)) | w1
    lo = (w2 << np.uint64(32)) | w3
    s = 2.0 ** -53
    u1 = ((hi >> np.uint64(11)).astype(np.float64) + 1.0) * s
    u2 = (lo >> np.uint64(11)).astype(np.float64) * s
    return u1, u2


def ln_series(u):
    """Natural log of u in (0, 1] from u = m 2^e, m in [sqrt2/2, sqrt2], and
    ln m = 2 atanh z = 2 sum_k z^(2k+1) / (2k+1), z = (m - 1) / (m + 1)."""
    u = np.asarray(u, dtype=np.float64)
    fm, fe = np.frexp(u)                  # u = fm 2^fe, fm in [0.5, 1): exact
    m = fm * 2.0                          # exact
    e = (fe - 1).astype(np.float64)
    big = m > SQRT2
    m = np.where(big, m * 0.5, m)         # exact
    e = np.where(big, e + 1.0, e)
    z = (m - 1.0) / (m + 1.0)
    z2 = z * z
    p = np.full_like(z, 1.0 / (2 * LN_TERMS + 1))
    for k in range(LN_TERMS - 1, -1, -1):
        p = p * z2
        p = p + 1.0 / (2 * k + 1)
    t = z * p
    lnm = t + t
    return e * LN2 + lnm


def _sin_cos_octant(psi):
    """sin and cos of psi in [0, pi/4] from nested Taylor series."""
    x2 = psi * psi
    s = np.ones_like(psi)
    for k in range(SIN_TERMS, 0, -1):
        q = x2 * s
        q = q / float((2 * k) * (2 * k + 1))
        s = 1.0 - q
    s = psi * s
    c = np.ones_like(psi)
    for k in range(COS_TERMS, 0, -1):
        q = x2 * c
        q = q / float((2 * k - 1) * (2 * k))
        c = 1.0 - q
    return s, c


def sincos_2pi(u):
    """(sin 2 pi u, cos 2 pi u) for u in [0, 1), with exact octant reduction
    t = 8u, k = floor t, f = t - k, psi = (f or 1 - f) * pi/4."""
    u = np.asarray(u, dtype=np.float64)
    t = u * 8.0
    k = np.floor(t)
    f = t - k
    k = k.astype(np.int64)
    odd = (k & 1) == 1
    g = np.where(odd, 1.0 - f, f)
    psi = g * PI_4
    s, c = _sin_cos_octant(psi)
    # theta = k pi/4 + f pi/4; per octant (sin theta, cos theta):
    # 0:(s,c) 1:(c,s) 2:(c,-s) 3:(s,-c) 4:(-s,-c) 5:(-c,-s) 6:(-c,s) 7:(-s,c)
    sin_t = np.select([k == 0, k == 1, k == 2, k == 3, k == 4, k == 5, k == 6, k == 7],
                      [s, c, c, s, -s, -c, -c, -s])
    cos_t = np.select([k == 0, k == 1, k == 2, k == 3, k == 4, k == 5, k == 6, k == 7],
                      [c, s, -s, -c, -c, -s, s, c])
    return sin_t, cos_t


def box_muller(u1, u2):
    """(z0, z1) = R (cos 2 pi u2, sin 2 pi u2), R = sqrt(-2 ln u1)."""
    r = np.sqrt(ln_series(u1) * -2.0)
    s, c = sincos_2pi(u2)
    return r * c, r * s


def gaussian_matrix(seed, kind, ident, rows, cols):
    """rows x cols binary64 N(0,1) matrix for factor (kind, ident) of a seed."""
    rows, cols = int(rows), int(cols)
    if rows == 0 or cols == 0:
        return np.zeros((rows, cols))
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    i = np.arange(rows, dtype=np.uint64)[:, None]
    j = np.arange(cols, dtype=np.uint64)[None, :]
    c0 = np.broadcast_to(i, (rows, cols))
    c1 = np.broadcast_to(j >> np.uint64(1), (rows, cols))
    c2 = np.uint64((int(kind) << 24) | (int(ident) & 0xFFFFFF))
    w = philox4x32_10(c0, c1, np.full((rows, cols), c2, dtype=np.uint64),
                      np.zeros((rows, cols), dtype=np.uint64),
                      seed & 0xFFFFFFFF, seed >> 32)
    u1, u2 = uniforms(*w)
    z0, z1 = box_muller(u1, u2)
    even = (np.arange(cols) % 2 == 0)[None, :]
    return np.where(even, z0, z1)
