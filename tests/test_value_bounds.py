"""CPU checks of the values the kernels produce beyond the decisions: the
nearest crossing's (t, u, v), point and distance (the nearest mode of
Sec. 2.4, values of the Sec. 2 definition), and the adjoint's gradients,
on the adversarial inputs of tests/_adversarial.py:

- the tighter per-triangle bound (componentwise magnitudes and gamma_10,
  `mt32_tight` in csrc/rsi_internal.cuh) must cover the FP32 values'
  distance to the definition's, so that accepting them below the threshold
  is safe;
- the double-float recomputation (`mt_df`: two-sum / two-product pairs,
  about 44 bits) must land well within the tolerance wherever that bound can
  keep the determinant away from zero;
- the kernels' whole rule for the nearest outputs (`nearest_values` in
  csrc/traverse_core.cuh: FP32 values accepted under the bound-derived
  thresholds with the point fma(t, fl(d), a); double-float (t, u, v) with
  the same point where the bound still separates det from zero, |d| times
  the bound stays small and |d| < 64; the FP64 definition otherwise) must
  give every output of every hit within the 1e-5 tolerance, and the
  double-float t must stay far below 2^-20 of the FP32 bound, the margin
  that rule takes;
- the adjoint's rule (`k_backward` in csrc/backward.cu: double-float
  algebra, FP64 where |det M| <= 2^-16 of its componentwise magnitude) must
  match the oracle's FP64 adjoint within the gradient tolerance on every
  hit, while double-float everywhere would not.

All are float32 emulations; the FP64 branches of both rules evaluate the
definition in the oracle's own operation order, so their rows are the
oracle's values.  CPU only."""
import numpy as np
import pytest

import oracle
from _adversarial import adversarial
from test_filter_bound import ETA, F, cross, definition64, dot, fmaf

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


def df_t(a, b, v0, v1, v2):
    """The double-float t as a (high, low) pair of float32 arrays."""
    return df_outputs(a, b, v0, v1, v2, pair=True)


def df_outputs(a, b, v0, v1, v2, pair=False):
    """(t, u, v, P, dist) as the double-float recomputation forms them:
    (t, u, v) rounded to FP32, the point fma(t, fl(d), a) (the rule sends
    segments with |d| >= 64 to FP64 instead)."""
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
        t = _div(dp(e2, q), det, r)
        if pair:
            return t
        u, v = (_div(x, det, r) for x in (dp(s0, p), dp(d, q)))
        tf = t[0] + t[1]
        dd = fmaf(d[0][0], d[0][0], fmaf(d[1][0], d[1][0], d[2][0] * d[2][0]))
        P = np.stack([(tf.astype(np.float64) * d[k][0].astype(np.float64)
                       + a[:, k].astype(np.float64)).astype(F) for k in range(3)], axis=1)
        return tf, u[0] + u[1], v[0] + v[1], P, tf * np.sqrt(dd)


def test_double_float_t_error_far_below_the_bound():
    """The double-float t, before its rounding to FP32, against the
    definition's: within 2^-24 of the FP32 tight bound on every bounded hit
    (the nearest-output rule assumes 2^-20)."""
    rng = np.random.default_rng(7)
    a, b, v0, v1, v2 = adversarial(rng, 300_000)
    hit, t64, _, _ = definition64(a, b, v0, v1, v2)
    et = tight32(a, b, v0, v1, v2)[3]
    sel = hit & np.isfinite(et)
    t_hi, t_lo = df_t(a, b, v0, v1, v2)
    with np.errstate(invalid="ignore"):
        r = np.abs(t_hi.astype(np.float64) + t_lo.astype(np.float64) - t64) / et
    assert sel.sum() > 100_000
    assert np.nanmax(np.where(sel, r, 0.0)) <= 2.0 ** -24


def nearest_outputs(a, b, v0, v1, v2):
    """The kernels' rule for the outputs of a crossing: returns
    (t, u, v, P, dist) as float64 arrays and the path taken per row
    (0 FP32 accepted, 1 double-float, 2 the FP64 definition)."""
    t32, u32, v32, et, euv = tight32(a, b, v0, v1, v2)
    d = b - a
    with np.errstate(all="ignore"):
        dlen = np.sqrt(fmaf(d[:, 0], d[:, 0], fmaf(d[:, 1], d[:, 1], d[:, 2] * d[:, 2]))) * F(1.0001)
        thresh = F(0.95) * ((F(1e-5) - F(U)) / np.maximum(F(1), dlen) - F(U))
        accept = (et <= thresh) & (euv <= F(0.95e-5))
        exact = ~np.isfinite(et) | (dlen * et > F(4)) | (euv > F(4)) | (dlen >= F(64))
        path = np.where(accept, 0, np.where(exact, 2, 1))
        P32 = (t32.astype(np.float64)[:, None] * d.astype(np.float64)
               + a.astype(np.float64)).astype(F)                    # fmaf(t, fl(d), a)
        dist32 = t32 * np.sqrt(fmaf(d[:, 0], d[:, 0], fmaf(d[:, 1], d[:, 1], d[:, 2] * d[:, 2])))
        tdf, udf, vdf, Pdf, distdf = df_outputs(a, b, v0, v1, v2)
        h64, t64, u64, v64 = definition64(a, b, v0, v1, v2)
        a64, d64 = a.astype(np.float64), b.astype(np.float64) - a.astype(np.float64)
        P64 = (a64 + t64[:, None] * d64).astype(F)
        dist64 = (t64 * np.sqrt(np.sum(d64 * d64, axis=1))).astype(F)

    def pick(x32, xdf, x64):
        c = path if np.ndim(x32) == 1 else path[:, None]
        return np.where(c == 0, x32, np.where(c == 1, xdf, x64)).astype(np.float64)

    return (pick(t32, tdf, t64.astype(F)), pick(u32, udf, u64.astype(F)),
            pick(v32, vdf, v64.astype(F)), pick(P32, Pdf, P64), pick(dist32, distdf, dist64),
            path)


def test_nearest_outputs_within_tolerance_on_every_hit():
    rng = np.random.default_rng(6)
    a, b, v0, v1, v2 = adversarial(rng, 400_000)
    hit, t64, u64, v64 = definition64(a, b, v0, v1, v2)
    t, u, v, P, dist, path = nearest_outputs(a, b, v0, v1, v2)
    a64, d64 = a.astype(np.float64), b.astype(np.float64) - a.astype(np.float64)
    ref = dict(t=t64, u=u64, v=v64, P=a64 + t64[:, None] * d64,
               dist=t64 * np.linalg.norm(d64, axis=1))
    got = dict(t=t, u=u, v=v, P=P, dist=dist)
    h = hit
    # every path is exercised, the FP64 one by the grazing crossings
    assert min((path[h] == k).sum() for k in range(3)) > 5_000
    for name in ref:
        with np.errstate(invalid="ignore"):
            bad = np.abs(got[name] - ref[name]) > 1e-5 * np.maximum(1.0, np.abs(ref[name]))
        if bad.ndim == 2:
            bad = bad.any(axis=1)
        assert not (h & bad).any(), f"{name}: {int((h & bad).sum())} hits outside 1e-5"


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


def adjoint_rule_errors(seed, n):
    """Per-row worst gradient error of the adjoint's rule against the
    oracle's FP64 adjoint (one triangle per segment, every hit), relative to
    max(|g|, 1e-3 max |g|) per row; also the error of double-float on every
    row and the FP64 mask."""
    rng = np.random.default_rng(seed)
    a, b, v0, v1, v2 = adversarial(rng, n)
    hit = definition64(a, b, v0, v1, v2)[0]
    gP = rng.normal(size=(n, 3)).astype(F)
    gt = rng.normal(size=(n, 3)).astype(F)
    V = np.stack([v0, v1, v2], axis=1).reshape(-1, 3)
    T = np.arange(3 * n, dtype=np.int32).reshape(-1, 3)
    tri = np.where(hit, np.arange(n), -1).astype(np.int32)
    gV, gA, gB = oracle.backward(V, T, a, b, tri, gP=gP.astype(np.float64),
                                 gtuv=gt.astype(np.float64))
    ref = np.concatenate([gA, gB, gV.reshape(n, 9)], axis=1)[hit]
    got = adjoint_df32(a, b, v0, v1, v2, gP, gt)[hit]
    with np.errstate(all="ignore"):
        scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max(axis=1, keepdims=True))
        err_df = np.nanmax(np.abs(got - ref) / scale, axis=1)
        # the switch: |det M| against its componentwise magnitude, float32
        d, e1, e2 = b - a, v1 - v0, v2 - v0
        ad, a1, a2 = np.abs(d), np.abs(e1), np.abs(e2)
        mag = sum(ad[:, k] * (a1[:, (k + 1) % 3] * a2[:, (k + 2) % 3] +
                              a1[:, (k + 2) % 3] * a2[:, (k + 1) % 3]) for k in range(3))
        det = dot(-d, cross(e1, e2))
        fp64 = ~(np.abs(det) > F(2.0 ** -16) * mag)[hit]
    return np.where(fp64, 0.0, err_df), err_df, fp64


def test_adjoint_within_tolerance_on_every_hit():
    """Double-float rows within 1e-5 with a margin (FP64 rows are the
    oracle's arithmetic); without the FP64 switch the same inputs exceed
    the tolerance, so the switch is what closes it."""
    err, err_df_only, fp64 = adjoint_rule_errors(11, 300_000)
    assert err.size > 100_000 and fp64.sum() > 1_000
    assert err.max() <= 2e-6
    assert (err_df_only > 1e-5).sum() > 0
