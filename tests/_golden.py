"""Reader of the text fixtures under tests/golden/ (hand-derived expected
values; each file states its derivation and the passage it follows)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _vecs(text, dtype):
    return np.array([[float(x) for x in v.split(",")] for v in text.split()], dtype)


def load_mt_cases(name="mt_hand_cases.txt"):
    """One dict per case: name, V float32 [nV,3], T int32 [nT,3], A, B
    float32 [1,3], flag, count, tri, and for hits tuv, point, dist."""
    cases = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fields = [f.strip() for f in line.split(";")]
            c = {"name": fields[0]}
            for f in fields[1:]:
                key, val = f.split("=", 1)
                c[key] = val
            case = {"name": c["name"],
                    "V": _vecs(c["V"], np.float32),
                    "T": _vecs(c["T"], np.float64).astype(np.int32),
                    "A": _vecs(c["a"], np.float32),
                    "B": _vecs(c["b"], np.float32),
                    "flag": int(c["flag"]), "count": int(c["count"]), "tri": int(c["tri"])}
            if "tuv" in c:
                case["tuv"] = np.array([float(x) for x in c["tuv"].split(",")])
                case["point"] = np.array([float(x) for x in c["point"].split(",")])
                case["dist"] = float(c["dist"])
            cases.append(case)
    return cases


def load_backward_cases(name="backward_hand_cases.txt"):
    """One dict per case: name, V, T, A, B as for load_mt_cases, gP and gtuv
    float64 [1,3], and the expected gA, gB [1,3] and gV [nV,3]."""
    cases = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fields = [f.strip() for f in line.split(";")]
            c = dict(f.split("=", 1) for f in fields[1:])
            cases.append({"name": fields[0],
                          "V": _vecs(c["V"], np.float32),
                          "T": _vecs(c["T"], np.float64).astype(np.int32),
                          "A": _vecs(c["a"], np.float32), "B": _vecs(c["b"], np.float32),
                          "gP": _vecs(c["gP"], np.float64), "gtuv": _vecs(c["gtuv"], np.float64),
                          "gA": _vecs(c["gA"], np.float64), "gB": _vecs(c["gB"], np.float64),
                          "gV": _vecs(c["gV"], np.float64)})
    return cases


def load_lbvh_case(name="lbvh_hand_case.txt"):
    """The hand-worked build: a point mesh (V, T: degenerate triangles whose
    corners coincide, so each centroid is its point) and the expected
    bounds, per-triangle codes, order, left / right children, ranges and
    three internal boxes."""
    c = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=", 1)
                c[k] = v
    P = _vecs(c["points"], np.float32)
    out = {"V": np.repeat(P, 3, axis=0),
           "T": np.arange(3 * len(P), dtype=np.int32).reshape(-1, 3),
           "bounds": [float(x) for x in c["bounds"].split(",")],
           "codes": [int(x) for x in c["codes"].split()],
           "order": [int(x) for x in c["order"].split()],
           "left": [int(x) for x in c["left"].split()],
           "right": [int(x) for x in c["right"].split()],
           "range": [[int(x) for x in r.split(",")] for r in c["range"].split()]}
    for k in ("nbox0", "nbox3", "nbox4"):
        out[k] = [float(x) for x in c[k].split(",")]
    return out


def load_inside_case(name="cube_inside_cases.txt"):
    """The closed cube: V float32 [8,3], T int32 [12,3], points P float32
    [n,3] and the expected inside flags uint8 [n]."""
    c = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=", 1)
                c[k] = v
    return {"V": _vecs(c["V"], np.float32),
            "T": _vecs(c["T"], np.float64).astype(np.int32),
            "P": _vecs(c["P"], np.float32),
            "inside": np.array([int(x) for x in c["inside"].split()], np.uint8)}
