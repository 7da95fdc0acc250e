"""Pins for the oracle's FP64 adjoint of the nearest hit (triangle held fixed):
closed forms on the unit triangle, FP64 central finite differences, and
translation invariance.  CPU only."""
import numpy as np
import pytest

from paper_2209_02878_gb300 import synth

from _golden import load_backward_cases


def test_closed_form_unit_triangle(orc):
    # plane z=0 through v0=(0,0,0), v1=(1,0,0), v2=(0,1,0); vertical segment at
    # (x,y) from az to bz: t = -az/(bz-az), P = (x, y, 0), u = x, v = y.
    x, y, az, bz = 0.25, 0.125, -1.0, 3.0
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    T = np.array([[0, 1, 2]], np.int32)
    A = np.array([[x, y, az]], np.float32)
    B = np.array([[x, y, bz]], np.float32)
    t = -az / (bz - az)
    tri = np.array([0], np.int32)
    # dP_x / da_x = 1 - t, dP_x / db_x = t; the plane does not move with a, b
    gV, gA, gB = orc.backward(V, T, A, B, tri, gP=np.array([[1.0, 0, 0]]))
    assert np.allclose(gA[0], [1 - t, 0, 0], atol=1e-15)
    assert np.allclose(gB[0], [t, 0, 0], atol=1e-15)
    # P_z follows the plane height w z0 + u z1 + v z2 at (x, y)
    gV, gA, gB = orc.backward(V, T, A, B, tri, gP=np.array([[0, 0, 1.0]]))
    assert np.allclose(gV[:, 2], [1 - x - y, x, y], atol=1e-15)
    assert np.allclose(gA[0], 0, atol=1e-15) and np.allclose(gB[0], 0, atol=1e-15)
    # dt / da_z = -bz/(bz-az)^2, dt / db_z = az/(bz-az)^2
    gV, gA, gB = orc.backward(V, T, A, B, tri, gtuv=np.array([[1.0, 0, 0]]))
    assert np.isclose(gA[0, 2], -bz / (bz - az) ** 2, rtol=1e-14)
    assert np.isclose(gB[0, 2], az / (bz - az) ** 2, rtol=1e-14)
    # du / dv1_x: moving v1 along x stretches e1, u = x / v1x -> -x
    gV, gA, gB = orc.backward(V, T, A, B, tri, gtuv=np.array([[0, 1.0, 0]]))
    assert np.isclose(gV[1, 0], -x, rtol=1e-14)
    # moving a along x with b fixed moves P_x = u by (1-t) per unit
    assert np.isclose(gA[0, 0], 1 - t, rtol=1e-14)
    assert np.isclose(gB[0, 0], t, rtol=1e-14)


@pytest.mark.parametrize("case", load_backward_cases(), ids=lambda c: c["name"])
def test_golden_backward_cases(orc, case):
    """tests/golden/backward_hand_cases.txt: every gradient component of a
    combined loss on P and (t, u, v), derived by hand (dyadic, so FP64 holds
    them to the last bit up to the rounding of its few divisions)."""
    gV, gA, gB = orc.backward(case["V"], case["T"], case["A"], case["B"],
                              np.array([0], np.int32), gP=case["gP"], gtuv=case["gtuv"])
    np.testing.assert_allclose(gA, case["gA"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(gB, case["gB"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(gV, case["gV"], rtol=1e-14, atol=1e-14)


def _problem(seed=0, G=33, n=4000):
    rng = np.random.default_rng(seed)
    mesh = synth.heightfield(G, rng)
    xy = rng.uniform(0.05, 0.95, size=(n, 2))
    dxy = rng.normal(0, 0.05, size=(n, 2))
    A = np.c_[xy, -np.ones(n)].astype(np.float32)
    B = np.c_[xy + dxy, np.ones(n)].astype(np.float32)
    W = rng.normal(size=(n, 3))
    Wt = rng.normal(size=(n, 3))
    return mesh, A, B, W, Wt


def test_adjoint_matches_central_differences(orc):
    mesh, A, B, W, Wt = _problem()
    o = orc.brute(mesh.V, mesh.T, A, B)
    tri = np.where(o["neardeg"] == 0, o["tri"], -1).astype(np.int32)
    assert (tri >= 0).mean() > 0.9
    gV, gA, gB = orc.backward(mesh.V, mesh.T, A, B, tri, gP=W, gtuv=Wt)
    V64, A64, B64 = mesh.V.astype(np.float64), A.astype(np.float64), B.astype(np.float64)

    def loss(Vx, Ax, Bx, idx):
        r = orc.eval_fixed(Vx, mesh.T, Ax[idx], Bx[idx], tri[idx])
        return float(np.sum(r[:, 3:] * W[idx]) + np.sum(r[:, :3] * Wt[idx]))

    rng = np.random.default_rng(1)
    used = np.unique(mesh.T[tri[tri >= 0]])
    checks = 0
    # vertex coordinates (only segments whose triangle uses the vertex move)
    for vtx in rng.choice(used, 60, replace=False):
        seg_idx = np.nonzero(np.any(mesh.T[np.maximum(tri, 0)] == vtx, axis=1) & (tri >= 0))[0]
        for k in range(3):
            h = 1e-6 * max(1.0, abs(V64[vtx, k]))
            Vp, Vm = V64.copy(), V64.copy()
            Vp[vtx, k] += h
            Vm[vtx, k] -= h
            fd = (loss(Vp, A64, B64, seg_idx) - loss(Vm, A64, B64, seg_idx)) / (2 * h)
            assert abs(fd - gV[vtx, k]) <= 1e-6 * max(1.0, abs(gV[vtx, k])), (vtx, k)
            checks += 1
    # segment endpoints
    for i in rng.choice(np.nonzero(tri >= 0)[0], 60, replace=False):
        for which, G_ in ((A64, gA), (B64, gB)):
            for k in range(3):
                h = 1e-6 * max(1.0, abs(which[i, k]))
                orig = which[i, k]
                which[i, k] = orig + h
                lp = loss(V64, A64, B64, [i])
                which[i, k] = orig - h
                lm = loss(V64, A64, B64, [i])
                which[i, k] = orig
                fd = (lp - lm) / (2 * h)
                assert abs(fd - G_[i, k]) <= 1e-6 * max(1.0, abs(G_[i, k])), (i, k)
                checks += 1
    assert checks == 60 * 3 + 60 * 6


def test_translation_invariance_and_misses(orc):
    mesh, A, B, W, Wt = _problem(seed=2, n=500)
    o = orc.brute(mesh.V, mesh.T, A, B)
    tri = o["tri"].astype(np.int32)
    tri[::7] = -1                                   # some misses
    gV, gA, gB = orc.backward(mesh.V, mesh.T, A, B, tri, gP=W, gtuv=Wt)
    # t, u, v do not change when everything translates: total = sum of gP
    total = gV.sum(0) + gA.sum(0) + gB.sum(0)
    assert np.allclose(total, W[tri >= 0].sum(0), rtol=1e-10, atol=1e-10)
    assert np.all(gA[tri < 0] == 0) and np.all(gB[tri < 0] == 0)
    untouched = np.setdiff1d(np.arange(mesh.n_vert), mesh.T[tri[tri >= 0]].ravel())
    assert np.all(gV[untouched] == 0)
