"""The oracle's pins catch plausible mistakes: each mutant below copies
oracle/rsi_oracle.c with one deliberate error (an open interval, a dropped
sign normalisation, swapped or mis-indexed operands, a wrong tie rule, a
wrong Morton bit order, quantisation scale or split rule, a wrong adjoint
weight), compiles it on the CPU and runs the hand-derived fixtures of
tests/golden/ against it; every mutant must fail at least one of them, and
the unmodified source must pass all.  CPU only."""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from _golden import load_backward_cases, load_inside_case, load_lbvh_case, load_mt_cases

MUTANTS = {
    "open t interval": [("(nt >= 0) && (nt <= det);", "(nt >= 0) && (nt < det);")],
    "open u + v edge": [("(nu + nv <= det)", "(nu + nv < det)")],
    "open u edge": [("(det > 0) && (nu >= 0)", "(det > 0) && (nu > 0)")],
    "no sign normalisation": [("    if (det < 0) {\n        det = -det;",
                               "    if (0) {\n        det = -det;")],
    "p = e2 x d": [("cross3(d, e2, p);", "cross3(e2, d, p);")],
    "s0 from v1": [("    sub3(a, v0, s0);\n    cross3(s0, e1, q);",
                    "    sub3(a, v1, s0);\n    cross3(s0, e1, q);")],
    "u and v swapped": [("        s->bu = r.nu / r.det;\n        s->bv = r.nv / r.det;",
                         "        s->bu = r.nv / r.det;\n        s->bv = r.nu / r.det;")],
    "tie to the higher index": [("(t == s->bt && j < s->best)", "(t == s->bt && j > s->best)")],
    "dist without |d|": [("s->bt * sqrt(dot3(d, d)) : 0.0;", "s->bt : 0.0;")],
    "point from b": [("? a[k] + s->bt * d[k] : 0.0;", "? b[k] + s->bt * d[k] : 0.0;")],
    "Morton x and z swapped": [("c |= ((x >> k) & 1u) << (3 * k + 2);",
                                "c |= ((z >> k) & 1u) << (3 * k + 2);"),
                               ("c |= ((z >> k) & 1u) << (3 * k);",
                                "c |= ((x >> k) & 1u) << (3 * k);")],
    "quantisation scale 1023": [("height_axis ? 32768.0f : 1024.0f;",
                                 "height_axis ? 32768.0f : 1023.0f;")],
    "split after the last equal prefix": [("if (clz64(K[f] ^ K[k]) > dfl) g = k;",
                                           "if (clz64(K[f] ^ K[k]) >= dfl) g = k;")],
    "adjoint end weights swapped": [("gA[3 * i + k] = (1.0 - t) * (gpk + lam[k]);",
                                     "gA[3 * i + k] = t * (gpk + lam[k]);")],
    "adjoint v1 weight v": [("gV[3 * i1 + k] += -u * lam[k];", "gV[3 * i1 + k] += -v * lam[k];")],
}


def golden_failures(orc):
    """Names of the golden checks that `orc` (the oracle module, bound to
    some build of rsi_oracle.c) fails."""
    bad = []
    for c in load_mt_cases():
        o = orc.brute(c["V"], c["T"], c["A"], c["B"])
        ok = (o["flag"][0], o["count"][0], o["tri"][0]) == (c["flag"], c["count"], c["tri"])
        if ok and "tuv" in c:
            ok = (list(o["tuv"][0]) == list(c["tuv"]) and list(o["point"][0]) == list(c["point"])
                  and o["dist"][0] == c["dist"])
        if not ok:
            bad.append("mt:" + c["name"])
    for c in load_backward_cases():
        gV, gA, gB = orc.backward(c["V"], c["T"], c["A"], c["B"], np.array([0], np.int32),
                                  gP=c["gP"], gtuv=c["gtuv"])
        if not all(np.allclose(g, w, rtol=1e-14, atol=1e-14)
                   for g, w in ((gA, c["gA"]), (gB, c["gB"]), (gV, c["gV"]))):
            bad.append("backward:" + c["name"])
    c = load_lbvh_case()
    o = orc.lbvh(c["V"], c["T"])
    if not (list(o["codes"]) == c["codes"] and list(o["order"]) == c["order"]
            and list(o["left"]) == c["left"] and list(o["right"]) == c["right"]
            and o["range"].tolist() == c["range"]
            and all(o["nbox"][k].tolist() == c[f"nbox{k}"] for k in (0, 3, 4))):
        bad.append("lbvh")
    c = load_inside_case()
    u = np.array([0.31, 0.57, 0.76])
    B = (c["P"] + 10.0 * u / np.linalg.norm(u)).astype(np.float32)
    if not np.array_equal(orc.brute(c["V"], c["T"], c["P"], B)["count"] % 2, c["inside"]):
        bad.append("cube parity")
    return bad


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(os.path.dirname(oracle.__file__), "rsi_oracle.c")) as fh:
        return fh.read()


def _build(src, path):
    with open(path + ".c", "w") as fh:
        fh.write(src)
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                    "-std=c11", "-o", path + ".so", path + ".c", "-lm"],
                   check=True, capture_output=True)
    return oracle._bind(C.CDLL(path + ".so"))


def _with_lib(lib):
    """Run the golden checks with the oracle module bound to `lib`."""
    oracle._get()  # the shipped build first, so that it is restored below
    saved = oracle._lib
    oracle._lib = lib
    try:
        return golden_failures(oracle)
    finally:
        oracle._lib = saved


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc is needed to build the mutants")
def test_unmodified_source_passes(source, tmp_path):
    assert _with_lib(_build(source, str(tmp_path / "orc_ref"))) == []


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc is needed to build the mutants")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(source, tmp_path, name):
    src = source
    for old, new in MUTANTS[name]:
        assert src.count(old) == 1, f"{name}: the snippet to mutate must occur once"
        src = src.replace(old, new)
    bad = _with_lib(_build(src, str(tmp_path / "orc_mut")))
    assert bad, f"mutant '{name}' passes every golden check"
