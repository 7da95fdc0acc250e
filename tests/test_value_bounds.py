"""CPU checks of the values the kernels produce beyond the decisions: the
nearest crossing's (t, u, v) when the decision filter's own bound is too
loose for the 1e-5 output tolerance (the nearest mode of Sec. 2.4, values of
the Sec. 2 definition), and the adjoint's gradients:

- the tighter per-triangle bound (componentwise magnitudes and gamma_10,
  `mt32_tight` in csrc/rsi_internal.cuh) must cover the FP32 values'
  distance to the definition's, so that accepting them below the threshold
  is safe;
- the double-float recomputation (`mt_df`: two-sum / two-product pairs,
  about 44 bits) must land within the tolerance wherever that bound can
  keep the determinant away from zero;
- the adjoint's double-float algebra (`k_backward` in csrc/backward.cu)
  must match the FP64 adjoint of the oracle within the gradient tolerance
  on the same range.

All are float32 emulations on the adversarial inputs of
test_filter_bound.py.  Beyond that range (crossings at grazing angles whose
determinant the FP32 bound cannot separate from zero) the double-float
values can exceed the tolerance (nearest values: 1.6e-5 once in 140k hits;
gradients: up to 3e-4 in 36 of 47k hits); the kernels do not yet fall back
to FP64 there.  CPU only."""
import numpy as np
import pytest

import oracle
from test_filter_bound import ETA, F, adversarial, cross, definition64, dot, fmaf

U = 2.0 ** -24


def tight32(a, b, v0, v1, v2):
    """(t, u, v, et, euv) as the tight per-triangle bound computes them;
    et = euv = inf where the determinant cannot be bounded away from zero."""
    with np.errstate(all="ignore"):
        d, e1, e2, s = b - a, v1 - v0, v2 - v0, a - v0
        p, q = cross(d, e2), cross(s, e1)
        det, nu, nv, nt = dot(e1, p), dot(s, p), dot(d, q), dot(e2, q)
        ad_, a1, a2, asv = np.abs(d), np.abs(e1), np.abs(e2), np.abs(s)
        Px = ad_[:, 1] * a2[:, 2] + ad_[:, 2] * a2[:, 1]
        Py = ad_[:, 2] * a2[:, 0] + ad_[:, 0] * a2[:, 2]
        Pz = ad_[:, 0] * a2[:, 1] + ad_[:, 1] * a2[:, 0]
        Qx = asv[:, 1] * a1[:, 2] + asv[:, 2] * a1[:, 1]
        Qy = asv[:, 2] * a1[:, 0] + asv[:, 0] * a1[:, 2]
        Qz = asv[:, 0] * a1[:, 1] + asv[:, 1] * a1[:, 0]
        g = F(10 * U * 1.0001)
        Bd = g * ((a1[:, 0] * Px + a1[:, 1] * Py) + a1[:, 2] * Pz) + ETA
        Bu = g * ((asv[:, 0] * Px + asv[:, 1] * Py) + asv[:, 2] * Pz) + ETA
        Bv = g * ((ad_[:, 0] * Qx + ad_[:, 1] * Qy) + ad_[:, 2] * Qz) + ETA
        Bt = g * ((a2[:, 0] * Qx + a2[:, 1] * Qy) + a2[:, 2] * Qz) + ETA
        ad = np.abs(det)
        ok = (ad > 2 * Bd) & np.isfinite(ad)
        inv = F(1) / ad
        sg = np.where(det < 0, F(-1), F(1))
        t, u, v = sg * nt * inv, sg * nu * inv, sg * nv * inv
        den = F(1) / (ad - Bd)
        et = fmaf(np.abs(t), Bd, Bt) * den
        eu = fmaf(np.abs(u), Bd, Bu) * den
        ev = fmaf(np.abs(v), Bd, Bv) * den
        euv = np.maximum(eu, ev) * F(1.001) + F(2.0 ** -22) * np.maximum(
            F(1), np.maximum(np.abs(u), np.abs(v)))
        et = et * F(1.001) + F(2.0 ** -22) * np.maximum(F(1), np.abs(t))
    inf = F(np.inf)
    return t, u, v, np.where(ok, et, inf), np.where(ok, euv, inf)


# double-float pairs (h, l) of float32 arrays
def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _fast(a, b):
    s = a + b
    return s, b - (s - a)


def _add(x, y):
    s, e = _two_sum(x[0], y[0])
    return _fast(s, e + (x[1] + y[1]))


def _neg(x):
    return -x[0], -x[1]


def _mul(x, y):
    p = x[0] * y[0]
    e = fmaf(x[0], y[0], -p)
    return _fast(p, fmaf(x[0], y[1], fmaf(x[1], y[0], e)))


def _div(x, y, r):
    q1 = x[0] * r
    res = _add(x, _neg(_mul(y, (q1, np.zeros_like(q1)))))
    return _fast(q1, res[0] * r)


def df32(a, b, v0, v1, v2):
    """(t, u, v) recomputed in double-float in the definition's order."""
    with np.errstate(all="ignore"):
        d = [_two_sum(b[:, k], -a[:, k]) for k in range(3)]
        e1 = [_two_sum(v1[:, k], -v0[:, k]) for k in range(3)]
        e2 = [_two_sum(v2[:, k], -v0[:, k]) for k in range(3)]
        s0 = [_two_sum(a[:, k], -v0[:, k]) for k in range(3)]

        def xp(x, y):
            return [_add(_mul(x[1], y[2]), _neg(_mul(x[2], y[1]))),
                    _add(_mul(x[2], y[0]), _neg(_mul(x[0], y[2]))),
                    _add(_mul(x[0], y[1]), _neg(_mul(x[1], y[0])))]

        def dp(x, y):
            return _add(_add(_mul(x[0], y[0]), _mul(x[1], y[1])), _mul(x[2], y[2]))

        p, q = xp(d, e2), xp(s0, e1)
        det = dp(e1, p)
        r = F(1) / det[0]
        return [h + l for h, l in (_div(x, det, r) for x in (dp(e2, q), dp(s0, p), dp(d, q)))]


@pytest.fixture(scope="module")
def cases():
    rng = np.random.default_rng(5)
    a, b, v0, v1, v2 = adversarial(rng, 300_000)
    hit, t64, u64, v64 = definition64(a, b, v0, v1, v2)
    return (a, b, v0, v1, v2), hit, (t64, u64, v64)


def test_tight_bound_covers_the_fp32_values(cases):
    args, hit, (t64, u64, v64) = cases
    t, u, v, et, euv = tight32(*args)
    bounded = hit & np.isfinite(et)
    assert bounded.sum() > 0.8 * hit.sum()
    with np.errstate(invalid="ignore"):
        assert not (bounded & (np.abs(t - t64) > et)).any()
        duv = np.maximum(np.abs(u - u64), np.abs(v - v64))
        assert not (bounded & (duv > euv)).any()


def test_double_float_values_within_tolerance_where_bounded(cases):
    args, hit, ref = cases
    et = tight32(*args)[3]
    bounded = hit & np.isfinite(et)
    with np.errstate(invalid="ignore"):
        for x, x64 in zip(df32(*args), ref):
            rel = np.abs(x.astype(np.float64) - x64) / np.maximum(1.0, np.abs(x64))
            assert np.nanmax(np.where(bounded, rel, 0.0)) <= 1e-6


def adjoint_df32(a, b, v0, v1, v2, gP, gt):
    """Per-segment gradients (dA, dB, dV0, dV1, dV2) of the double-float
    adjoint, as float64 arrays [n, 15]."""
    n = a.shape[0]

    def sub(x, y):
        return _add(x, _neg(y))

    def fr(x):
        return x, np.zeros_like(x)

    def xp(x, y):
        return [sub(_mul(x[1], y[2]), _mul(x[2], y[1])), sub(_mul(x[2], y[0]), _mul(x[0], y[2])),
                sub(_mul(x[0], y[1]), _mul(x[1], y[0]))]

    def dp(x, y):
        return _add(_add(_mul(x[0], y[0]), _mul(x[1], y[1])), _mul(x[2], y[2]))

    def val(z):
        return z[0].astype(np.float64) + z[1].astype(np.float64)

    with np.errstate(all="ignore"):
        d = [_two_sum(b[:, k], -a[:, k]) for k in range(3)]
        nd = [_neg(x) for x in d]
        e1 = [_two_sum(v1[:, k], -v0[:, k]) for k in range(3)]
        e2 = [_two_sum(v2[:, k], -v0[:, k]) for k in range(3)]
        s0 = [_two_sum(a[:, k], -v0[:, k]) for k in range(3)]
        c12, c20, c01 = xp(e1, e2), xp(e2, nd), xp(nd, e1)
        det = dp(nd, c12)
        r = F(1) / det[0]
        t, u, v = (_div(dp(c, s0), det, r) for c in (c12, c20, c01))
        gpd = [fr(gP[:, k]) for k in range(3)]
        gx0, gx1, gx2 = _add(dp(gpd, d), fr(gt[:, 0])), fr(gt[:, 1]), fr(gt[:, 2])
        one = fr(np.ones(n, F))
        w, omt = sub(sub(one, u), v), sub(one, t)
        out = np.zeros((n, 15))
        for k in range(3):
            num = _add(_add(_mul(gx0, c12[k]), _mul(gx1, c20[k])), _mul(gx2, c01[k]))
            lam = _div(num, det, r)
            sk = _add(gpd[k], lam)
            out[:, k] = val(_mul(omt, sk)).astype(F)
            out[:, 3 + k] = val(_mul(t, sk)).astype(F)
            for q, wt in enumerate((w, u, v)):
                out[:, 6 + 3 * q + k] = -val(_mul(wt, lam))
    return out


def test_double_float_adjoint_within_tolerance_where_bounded():
    rng = np.random.default_rng(11)
    n = 100_000
    a, b, v0, v1, v2 = adversarial(rng, n)
    hit = definition64(a, b, v0, v1, v2)[0]
    bounded = hit & np.isfinite(tight32(a, b, v0, v1, v2)[3])
    gP = rng.normal(size=(n, 3)).astype(F)
    gt = rng.normal(size=(n, 3)).astype(F)
    # the oracle's FP64 adjoint, one triangle per segment
    V = np.stack([v0, v1, v2], axis=1).reshape(-1, 3)
    T = np.arange(3 * n, dtype=np.int32).reshape(-1, 3)
    tri = np.where(bounded, np.arange(n), -1).astype(np.int32)
    gV, gA, gB = oracle.backward(V, T, a, b, tri, gP=gP.astype(np.float64),
                                 gtuv=gt.astype(np.float64))
    ref = np.concatenate([gA, gB, gV.reshape(n, 9)], axis=1)[bounded]
    got = adjoint_df32(a, b, v0, v1, v2, gP, gt)[bounded]
    scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=1, keepdims=True))
    assert bounded.sum() > 30_000
    assert (np.abs(got - ref) / scale).max() <= 1e-5
