"""CPU emulation of FP32-pair ("double-single") arithmetic, step for step as
the GPU's outer residual evaluates the relative form of M u (test helper).

A pair is hi + lo with two float32 values.  Products are split exactly with
a fused multiply-add (emulated here in float64, where the product of two
float32 values is exact), sums of leading parts with Knuth's TwoSum, and the
trailing parts are accumulated in plain float32 (no renormalisation between
steps, one Fast2Sum at the end of each contraction).  A float64 operand enters
as hi = its significand rounded to 24 bits and lo = the remainder rounded to
float32.
"""
import numpy as np

F32 = np.float32
F64 = np.float64


def fma(a, b, c):
    """float32 a*b + c with one rounding (the product is exact in float64; the
    float64 sum can differ from a true fused operation by a double rounding,
    which is far below what these tests resolve)."""
    return (a.astype(F64) * b.astype(F64) + c.astype(F64)).astype(F32)


def two_sum(a, b):
    """s + e == a + b exactly, s = fl(a + b)."""
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    e = ((a - (s - bb).astype(F32)).astype(F32) + (b - bb).astype(F32)).astype(F32)
    return s, e


def fast_two_sum(a, b):
    """s + e == a + b for |a| >= |b|."""
    s = (a + b).astype(F32)
    return s, (b - (s - a).astype(F32)).astype(F32)


def split64(d):
    """float64 -> (hi, lo): hi = d rounded to 24 significand bits (to nearest,
    ties away from zero: the magnitude's bits plus half a unit, truncated), lo =
    d - hi rounded to float32.  |d| below 2^-126 gives (0, 0)."""
    d = np.asarray(d, dtype=F64)
    bits = (d.view(np.int64) + np.int64(1 << 28)) & ~np.int64((1 << 29) - 1)
    hi = bits.view(F64)
    tiny = np.abs(d) < 2.0 ** -126
    hi = np.where(tiny, 0.0, hi)
    lo = np.where(tiny, 0.0, d - hi)
    return hi.astype(F32), lo.astype(F32)


def mul_acc(wh, wl, xh, xl, sh, sl):
    """(sh, sl) += (wh, wl) (xh, xl): exact leading product, TwoSum into sh,
    every error term into sl."""
    p = (wh * xh).astype(F32)
    e = fma(wh, xh, -p)
    e = fma(wh, xl, e)
    e = fma(wl, xh, e)
    s, t = two_sum(sh, p)
    return s, (sl + (t + e).astype(F32)).astype(F32)


def mul_first(wh, wl, xh, xl):
    """(wh, wl) (xh, xl) as a pair (the first term of a sum)."""
    p = (wh * xh).astype(F32)
    e = fma(wh, xh, -p)
    e = fma(wh, xl, e)
    return p, fma(wl, xh, e)


def extension_delta(wx, wy, wz, dh, dl):
    """delta = sum of w_x w_y w_z d over the 4^d stencil in pair arithmetic.
    w*: (hi, lo) of the 1-D weights, each (N, 4); d: (N, nz, 4, 4) as [z][y][x]
    (nz = 1 in 2-D, wz None).  Order: y for each (z, x), then z, then x."""
    nz = dh.shape[1]
    qh = ql = None
    for c in range(nz):
        ph, pl = mul_first(wy[0][:, 0:1], wy[1][:, 0:1], dh[:, c, 0, :], dl[:, c, 0, :])
        for b in range(1, 4):
            ph, pl = mul_acc(wy[0][:, b:b + 1], wy[1][:, b:b + 1], dh[:, c, b, :], dl[:, c, b, :], ph, pl)
        if wz is None:
            qh, ql = ph, pl
        elif c == 0:
            qh, ql = mul_first(wz[0][:, 0:1], wz[1][:, 0:1], ph, pl)
        else:
            qh, ql = mul_acc(wz[0][:, c:c + 1], wz[1][:, c:c + 1], ph, pl, qh, ql)
    sh, sl = mul_first(wx[0][:, 0], wx[1][:, 0], qh[:, 0], ql[:, 0])
    for a in range(1, 4):
        sh, sl = mul_acc(wx[0][:, a], wx[1][:, a], qh[:, a], ql[:, a], sh, sl)
    return fast_two_sum(sh, sl)


def to64(h, l):
    return h.astype(F64) + l.astype(F64)


def pair_mul(ah, al, bh, bl):
    """(ah, al) (bh, bl) as a normalised pair."""
    p = (ah * bh).astype(F32)
    e = fma(ah, bh, -p)
    e = fma(ah, bl, e)
    e = fma(al, bh, e)
    return fast_two_sum(p, e)


def pair_add(ah, al, bh, bl):
    """(ah, al) + (bh, bl) as a normalised pair."""
    s, t = two_sum(ah, bh)
    return fast_two_sum(s, (t + (al + bl).astype(F32)).astype(F32))


def residual(u_i, f_i, c, ref_i, dh_i, dl_i, ref_k, dh_k, dl_k, inv_h2, gamma):
    """r_i = f_i - c u_i + M u_i with
    M u_i = S / dx^2 + gamma ((ref_i - u_i) + delta_i),
    S = sum_k (ref_k - ref_i) + (delta_k - delta_i) in pair arithmetic
    (ref float32, delta pairs; k over the 2d neighbours, axis 1 of *_k);
    1/dx^2 and gamma enter as pairs, ref_i - u_i is formed in float64."""
    sh = np.zeros(u_i.shape, F32)
    sl = np.zeros(u_i.shape, F32)
    for q in range(ref_k.shape[1]):
        ah, al = two_sum(ref_k[:, q], -ref_i)
        bh, bl = two_sum(dh_k[:, q], -dh_i)
        ch, cl = two_sum(ah, bh)
        sh, t = two_sum(sh, ch)
        sl = (sl + ((al + bl).astype(F32) + (cl + t).astype(F32)).astype(F32)).astype(F32)
        sl = (sl + (dl_k[:, q] - dl_i).astype(F32)).astype(F32)
    Sh, Sl = fast_two_sum(sh, sl)
    ih, il = split64(np.full(u_i.shape, inv_h2))
    gh, gl = split64(np.full(u_i.shape, gamma))
    lh, ll = pair_mul(Sh, Sl, ih, il)
    eh, el = split64(ref_i.astype(F64) - u_i)
    th, tl = pair_add(eh, el, dh_i, dl_i)
    th, tl = pair_mul(th, tl, gh, gl)
    mh, ml = pair_add(lh, ll, th, tl)
    return (f_i - c * u_i) + to64(mh, ml)
