"""CPU check that the traversal's segment / box test is conservative: it
never rejects a box that the exact segment a + s (b - a), s in [0, 1],
touches (a rejected box would hide its triangles from the Moller-Trumbore
test of Sec. 2).  A float32 emulation of the test as csrc/rsi_internal.cuh
performs it (entry and exit parameters (face - a) * (1/d) per axis, the face
chosen by the sign of 1/d, 1/d from an approximate reciprocal within 1 ulp,
the exit scaled by 1 + 2^-18; a padded box-overlap test when some
0 < |d_i| < 2^-60) runs on boxes built around a point of the segment that is
known exactly (rational arithmetic), down to zero-width boxes whose faces
pass through that point, and on segments with zero direction components.
CPU only."""
from fractions import Fraction

import numpy as np
import pytest

F = np.float32
SLACK = F(1 + 2.0 ** -18)
TINY = F(2.0 ** -60)


def slab32(a, b, lo, hi, rcp_ulp, slack=SLACK):
    """The box test on float32 inputs; rcp_ulp in {-1, 0, 1} moves each
    reciprocal by that many ulps (the approximate reciprocal's error);
    `slack` is the exit's scale factor."""
    with np.errstate(all="ignore"):
        d = b - a
        inv = F(1) / d
        inv = np.where(rcp_ulp > 0, np.nextafter(inv, F(np.inf)),
                       np.where(rcp_ulp < 0, np.nextafter(inv, F(-np.inf)), inv)).astype(F)
        inv = np.where(np.isinf(F(1) / d), F(1) / d, inv)     # 1/0 stays +-inf
        neg = inv < 0
        near = np.where(neg, hi, lo)
        far = np.where(neg, lo, hi)
        tn = (near - a) * inv
        tf = (far - a) * inv
        tn = np.fmax(np.fmax(tn[:, 0], tn[:, 1]), np.fmax(tn[:, 2], F(0)))
        tf = np.fmin(np.fmin(tf[:, 0], tf[:, 1]), np.fmin(tf[:, 2], F(1)))
        hit = tn <= tf * F(slack)
        # segments with a tiny nonzero direction component: padded overlap
        ad = np.abs(d)
        tiny = np.any((ad > 0) & (ad < TINY), axis=1)
        bb = a + d
        pad = (np.abs(a) + np.abs(bb)) * F(2.0 ** -21) + F(2.0 ** -140)
        ov = ~np.any((np.fmax(a, bb) + pad < lo) | (np.fmin(a, bb) - pad > hi), axis=1)
    return np.where(tiny, ov, hit)


def down32(x):
    f = F(float(x))
    return f if Fraction(float(f)) <= x else np.nextafter(f, F(-np.inf))


def up32(x):
    f = F(float(x))
    return f if Fraction(float(f)) >= x else np.nextafter(f, F(np.inf))


def touching_cases(rng, n):
    """Segments over many binades (some with zero or tiny direction
    components) and boxes that contain an exactly known point of them."""
    A = np.empty((n, 3), F)
    B = np.empty((n, 3), F)
    LO = np.empty((n, 3), F)
    HI = np.empty((n, 3), F)
    for i in range(n):
        scale = 2.0 ** rng.uniform(-20, 20)
        a = (rng.normal(size=3) * scale).astype(F)
        b = (a + rng.normal(size=3) * scale * 2.0 ** rng.uniform(-12, 2)).astype(F)
        kind = rng.integers(0, 5)
        if kind == 1:                       # a zero direction component
            k = rng.integers(0, 3)
            b[k] = a[k]
        elif kind == 2:                     # tiny coordinates, tiny components
            a = (rng.normal(size=3) * 2.0 ** -64).astype(F)
            b = (a + rng.normal(size=3) * 2.0 ** -66).astype(F)
        s = rng.choice([Fraction(0), Fraction(1), Fraction(int(rng.integers(0, 1025)), 1024)])
        X = [Fraction(float(a[k])) + s * (Fraction(float(b[k])) - Fraction(float(a[k])))
             for k in range(3)]
        for k in range(3):
            lo, hi = down32(X[k]), up32(X[k])
            if kind != 3:                   # kind 3: the tightest box around X
                span = float(abs(b[k] - a[k])) + float(abs(a[k])) * 1e-3
                lo = F(lo - span * rng.choice([0.0, 1e-6, 0.3]))
                hi = F(hi + span * rng.choice([0.0, 1e-6, 0.3]))
                lo = min(lo, down32(X[k]))
                hi = max(hi, up32(X[k]))
            LO[i, k], HI[i, k] = lo, hi
        A[i], B[i] = a, b
    return A, B, LO, HI


@pytest.mark.parametrize("seed", range(3))
def test_boxes_touched_by_the_exact_segment_are_never_rejected(seed):
    rng = np.random.default_rng(200 + seed)
    A, B, LO, HI = touching_cases(rng, 20_000)
    for ulp in (-1, 0, 1):
        hit = slab32(A, B, LO, HI, np.full(A.shape, ulp))
        miss = np.nonzero(~hit)[0]
        assert miss.size == 0, \
            f"rcp {ulp:+d} ulp: {miss.size} touched boxes rejected, first {miss[:3]}"


def test_without_the_slack_touched_boxes_are_lost():
    """A planted mistake: with the exit not scaled (or scaled by only
    1 + 2^-22) the same boxes are rejected, so the check above is not
    vacuous."""
    rng = np.random.default_rng(200)
    A, B, LO, HI = touching_cases(rng, 20_000)
    for slack in (1.0, 1 + 2.0 ** -22):
        assert (~slab32(A, B, LO, HI, np.full(A.shape, 1), slack=slack)).sum() > 0


def test_the_test_still_culls():
    """Boxes beside the segment are rejected (the check above is not met by
    a test that accepts everything)."""
    rng = np.random.default_rng(7)
    n = 20_000
    a = rng.normal(size=(n, 3)).astype(F)
    b = (a + rng.normal(size=(n, 3))).astype(F)
    off = np.abs(a - b).max(axis=1, keepdims=True) + np.abs(a).max(axis=1, keepdims=True) + 1
    lo = (np.maximum(a, b) + off).astype(F)       # entirely beyond both ends on every axis
    hi = (lo + 1).astype(F)
    assert not slab32(a, b, lo, hi, np.zeros((n, 3))).any()
