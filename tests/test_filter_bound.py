"""CPU check of the certification rule of the FP32 segment / triangle filter
that the traversal kernels apply before any FP64 replay (the two-stage error
bound described in csrc/rsi_internal.cuh, for the definition of Sec. 2).

A float32 emulation of that filter runs on adversarial inputs: crossings
within 1e-9 .. 1e-3 (relative) of an edge, a vertex or a segment end,
segments nearly parallel to the plane, and coordinates over many binades.
Every decision it certifies (miss or hit) must equal the FP64 definition's,
and for certified hits the (t, u, v) error bound it reports must cover the
definition's values.  The emulation rounds every operation separately (no
FMA contraction except where the filter itself calls fmaf), one of the
evaluation orders the bound is derived for.  CPU only."""
import numpy as np
import pytest

from _adversarial import adversarial

F = np.float32
U = 2.0 ** -24
K = F(2.0 ** -17)
ETA = F(2.0 ** -100)
LO, HI = F(2.0 ** -30), F(2.0 ** 30)


def fmaf(a, b, c):
    """float32 fused multiply-add (one rounding up to double rounding at
    ties, which only matters at the last bit of a bound with slack)."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def maxabs(x):
    return np.maximum(np.maximum(np.abs(x[:, 0]), np.abs(x[:, 1])), np.abs(x[:, 2]))


def cross(x, y):
    return np.stack([x[:, 1] * y[:, 2] - x[:, 2] * y[:, 1],
                     x[:, 2] * y[:, 0] - x[:, 0] * y[:, 2],
                     x[:, 0] * y[:, 1] - x[:, 1] * y[:, 0]], axis=1)


def dot(x, y):
    return (x[:, 0] * y[:, 0] + x[:, 1] * y[:, 1]) + x[:, 2] * y[:, 2]


def filter32(a, b, v0, v1, v2, shrink=1.0):
    """Returns (res, t, u, v, err): res 0 miss, 1 hit, 2 undecided.
    `shrink` < 1 scales both stages' bound constants down (a planted
    mistake, to show that the inputs catch an undersized bound)."""
    with np.errstate(all="ignore"):
        e1, e2 = v1 - v0, v2 - v0
        m1, m2 = maxabs(e1), maxabs(e2)
        d = b - a
        md = maxabs(d)
        s = a - v0
        ms = maxabs(s)
        mhi = np.maximum(np.maximum(m1, m2), ms)
        mlo = np.minimum(np.minimum(m1, m2), np.where(ms == 0, F(1), ms))
        undecidable = ~((md >= LO) & (md <= HI)) | (mhi > HI) | (mlo < LO)
        p = cross(d, e2)
        det = dot(e1, p)
        q = cross(s, e1)
        nu, nv, nt = dot(s, p), dot(d, q), dot(e2, q)
        adet = np.abs(det)
        sg = np.where(det < 0, F(-1), F(1))
        nu, nv, nt = nu * sg, nv * sg, nt * sg
        w = (adet - nu) - nv
        r = adet - nt
        # stage 1
        Pde, Pse = md * m2, ms * m1
        Mdet, MU, MV, MT = m1 * Pde, ms * Pde, md * Pse, m2 * Pse
        k = F(K * shrink)
        Bdet, BU, BV, BT = (fmaf(k, x, ETA) for x in (Mdet, MU, MV, MT))
        Bw = fmaf(k, (Mdet + MU) + MV, ETA)
        Br = fmaf(k, Mdet + MT, ETA)
        s1 = adet > Bdet
        rej1 = s1 & ((nu < -BU) | (nv < -BV) | (nt < -BT) | (w < -Bw) | (r < -Br))
        acc1 = s1 & ~rej1 & (nu > BU) & (nv > BV) & (nt > BT) & (w > Bw) & (r > Br)
        # stage 2
        g = F(11 * U * shrink)
        ad, a1, a2, asv = np.abs(d), np.abs(e1), np.abs(e2), np.abs(s)
        Px = ad[:, 1] * a2[:, 2] + ad[:, 2] * a2[:, 1]
        Py = ad[:, 2] * a2[:, 0] + ad[:, 0] * a2[:, 2]
        Pz = ad[:, 0] * a2[:, 1] + ad[:, 1] * a2[:, 0]
        Qx = asv[:, 1] * a1[:, 2] + asv[:, 2] * a1[:, 1]
        Qy = asv[:, 2] * a1[:, 0] + asv[:, 0] * a1[:, 2]
        Qz = asv[:, 0] * a1[:, 1] + asv[:, 1] * a1[:, 0]
        Bdet2 = fmaf(g, (a1[:, 0] * Px + a1[:, 1] * Py) + a1[:, 2] * Pz, ETA)
        BU2 = fmaf(g, (asv[:, 0] * Px + asv[:, 1] * Py) + asv[:, 2] * Pz, ETA)
        BV2 = fmaf(g, (ad[:, 0] * Qx + ad[:, 1] * Qy) + ad[:, 2] * Qz, ETA)
        BT2 = fmaf(g, (a2[:, 0] * Qx + a2[:, 1] * Qy) + a2[:, 2] * Qz, ETA)
        Bw2 = fmaf(F(2.01 * U), (adet + np.abs(nu)) + np.abs(nv), (Bdet2 + BU2) + BV2)
        Br2 = fmaf(F(1.01 * U), adet + np.abs(nt), Bdet2 + BT2)
        s2 = adet > Bdet2
        rej2 = s2 & ((nu < -BU2) | (nv < -BV2) | (nt < -BT2) | (w < -Bw2) | (r < -Br2))
        acc2 = s2 & ~rej2 & (nu > BU2) & (nv > BV2) & (nt > BT2) & (w > Bw2) & (r > Br2)
        res = np.full(a.shape[0], 2, np.int8)
        st2 = ~rej1 & ~acc1
        res[st2 & acc2] = 1
        res[st2 & rej2] = 0
        res[acc1] = 1
        res[rej1] = 0
        res[(m1 == 0) | (m2 == 0)] = 0      # an exactly zero edge: det = 0 in FP64
        res[undecidable & ~((m1 == 0) | (m2 == 0))] = 2
        # error bounds of the deciding stage
        Bd = np.where(acc1, Bdet, Bdet2)
        Bu_ = np.where(acc1, BU, BU2)
        Bv_ = np.where(acc1, BV, BV2)
        Bt_ = np.where(acc1, BT, BT2)
        inv = F(1) / adet
        t, u, v = nt * inv, nu * inv, nv * inv
        den = F(1) / (adet - Bd)
        eT, eU, eV = fmaf(t, Bd, Bt_) * den, fmaf(u, Bd, Bu_) * den, fmaf(v, Bd, Bv_) * den
        err = np.maximum(np.maximum(eT, eU), eV) * F(1.001) + F(2.0 ** -22)
    return res, t, u, v, err


def definition64(a, b, v0, v1, v2):
    """The FP64 definition of Sec. 2 in its operation order."""
    a, b, v0, v1, v2 = (x.astype(np.float64) for x in (a, b, v0, v1, v2))
    d, e1, e2, s = b - a, v1 - v0, v2 - v0, a - v0
    p = cross(d, e2)
    det = dot(e1, p)
    q = cross(s, e1)
    nu, nv, nt = dot(s, p), dot(d, q), dot(e2, q)
    sg = np.where(det < 0, -1.0, 1.0)
    det, nu, nv, nt = det * sg, nu * sg, nv * sg, nt * sg
    hit = (det > 0) & (nu >= 0) & (nv >= 0) & (nu + nv <= det) & (nt >= 0) & (nt <= det)
    with np.errstate(all="ignore"):
        return hit, nt / det, nu / det, nv / det


@pytest.mark.parametrize("seed", range(4))
def test_certified_decisions_match_the_definition(seed):
    rng = np.random.default_rng(100 + seed)
    a, b, v0, v1, v2 = adversarial(rng, 500_000)
    res, t, u, v, err = filter32(a, b, v0, v1, v2)
    hit, t64, u64, v64 = definition64(a, b, v0, v1, v2)
    cert = res != 2
    # the filter must decide most cases and leave the hardest to FP64
    assert 0.5 < cert.mean() < 1.0
    wrong = cert & ((res == 1) != hit)
    assert not wrong.any(), \
        f"{int(wrong.sum())} certified decisions differ, first {np.argmax(wrong)}"
    h = res == 1
    with np.errstate(invalid="ignore"):
        for name, x, x64 in (("t", t, t64), ("u", u, u64), ("v", v, v64)):
            off = h & (np.abs(x.astype(np.float64) - x64) > err.astype(np.float64))
            assert not off.any(), f"{name}: {int(off.sum())} certified hits outside their bound"


def test_adversarial_inputs_catch_an_undersized_bound():
    """The same inputs against the filter with both stages' constants cut
    by 2^9: it then certifies wrong decisions, so the check above is not
    vacuous."""
    rng = np.random.default_rng(100)
    a, b, v0, v1, v2 = adversarial(rng, 500_000)
    res, *_ = filter32(a, b, v0, v1, v2, shrink=2.0 ** -9)
    hit = definition64(a, b, v0, v1, v2)[0]
    assert ((res != 2) & ((res == 1) != hit)).sum() > 0
