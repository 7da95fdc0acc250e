"""Autotuner front end: runs rsi_autotune (the timing loop lives in the
library) and keeps a JSON cache keyed by (GPU name, mode, N_t bucket, N_r
bucket), so a workload class is tuned once per GPU model; and
rsi_autotune_height_axis, which picks the build's Morton axes for a mesh."""
from __future__ import annotations

import ctypes as C
import json
import math
import os

import torch

from . import _abi
from . import _mode, _rsi_output, _alloc_outputs, _stream, _vp

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "rsi_gb300", "tune.json")


def bucket(n: int) -> int:
    """Power-of-two bucket of a size."""
    return 0 if n <= 0 else int(math.log2(n))


def cache_key(mode, n_tri: int, n_seg: int, device=None) -> str:
    name = torch.cuda.get_device_name(device)
    return f"{name}|{mode}|t{bucket(n_tri)}|r{bucket(n_seg)}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def autotune_height_axis(bvh, V, T, A, B, mode="bool", launch=None, reps=5, stream=None):
    """Time the traversal of these segments over trees built with each
    Morton code (height_axis 0: x, y, z; 1, 2, 3: that axis left out) and
    leave bvh built with the fastest.  Returns (best axis, {axis: ms})."""
    from . import _launch
    lib = _abi.load()
    m = _mode(mode)
    n = int(A.shape[0])
    o = _alloc_outputs(m, n, A.device, False, None)
    ro = _rsi_output(o)
    lo = _launch(launch, n, A.device)
    ms = (C.c_float * 4)()
    best = C.c_int32()
    with torch.cuda.device(A.device):
        _abi.check(lib.rsi_autotune_height_axis(bvh._h, _vp(V), _vp(T), _vp(A), _vp(B), n, m,
                                                C.byref(ro), C.byref(lo), int(reps),
                                                _stream(stream), ms, C.byref(best)),
                   "rsi_autotune_height_axis")
    bvh.height_axis = best.value
    return best.value, {a: float(ms[a]) for a in range(4)}


def autotune(bvh, V, T, A, B, mode="bool", block_sizes=(64, 128, 256, 512),
             stack_depths=(8, 32, 64), smem_nodes=(-1, 255, 511, 1023), leaf_sizes=(1, 2, 4),
             reps=5, cache: str | None = DEFAULT_CACHE, stream=None, try_packet=True):
    """Time every combination (the handle is rebuilt per leaf size) and
    return (best launch options dict, best leaf size, table of entries).
    With try_packet, the warp-cooperative traversal (launch option `packet`,
    faster when the segments are coherent) is timed against the winner too.
    The handle is left built with the best leaf size."""
    lib = _abi.load()
    m = _mode(mode)
    key = cache_key(m, bvh.nT, int(A.shape[0]), A.device)
    if cache:
        hit = _load(cache).get(key)
        if hit:  # the caller rebuilds with hit["leaf_size"] if it differs
            return hit["launch"], hit["leaf_size"], hit.get("table", [])
    o = _alloc_outputs(m, int(A.shape[0]), A.device, False, None)
    ro = _rsi_output(o)

    def arr(xs):
        return (C.c_int32 * len(xs))(*xs), len(xs)

    bs, nbs = arr(block_sizes)
    sd, nsd = arr(stack_depths)
    sm, nsm = arr(smem_nodes)
    ls, nls = arr(leaf_sizes)
    cap = nbs * nsd * nsm * nls
    table = (_abi.rsi_tune_entry * cap)()
    n_written = C.c_int32()
    best = _abi.rsi_launch_opts()
    best_leaf = C.c_int32()
    with torch.cuda.device(A.device):
        _abi.check(lib.rsi_autotune(bvh._h, _vp(V), _vp(T), _vp(A), _vp(B), int(A.shape[0]), m,
                                    C.byref(ro), bs, nbs, sd, nsd, sm, nsm, ls, nls, int(reps),
                                    _stream(stream), table, cap, C.byref(n_written),
                                    C.byref(best), C.byref(best_leaf)), "rsi_autotune")
    rows = [dict(block_size=t.block_size, stack_depth=t.stack_depth, smem_nodes=t.smem_nodes,
                 leaf_size=t.leaf_size, ms=t.ms) for t in table[:n_written.value]]
    launch = dict(block_size=best.block_size, stack_depth=best.stack_depth,
                  smem_nodes=best.smem_nodes)
    bvh.leaf_size = best_leaf.value
    if try_packet:
        s = stream if stream is not None else torch.cuda.current_stream()

        def median_ms(lo):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            bvh.intersect(A, B, m, launch=lo, out=o, stream=s)  # warm-up
            ms = []
            for _ in range(max(1, int(reps))):
                e0.record(s)
                bvh.intersect(A, B, m, launch=lo, out=o, stream=s)
                e1.record(s)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            return sorted(ms)[len(ms) // 2]

        t_best, t_packet = median_ms(launch), median_ms({"packet": 1})
        rows.append(dict(packet=1, leaf_size=best_leaf.value, ms=t_packet))
        if t_packet < t_best:
            launch = {"packet": 1}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = _load(cache)
        data[key] = dict(launch=launch, leaf_size=best_leaf.value, table=rows)
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return launch, best_leaf.value, rows


def autotune_batch(items, block_sizes=(64, 128, 256), stack_depths=(32, 64),
                   leaf_sizes=(1, 2, 4), reps=3, cache: str | None = DEFAULT_CACHE,
                   stream=None):
    """Tune the batched launch: for each leaf size (a multi-mesh build) and
    launch configuration, time `reps` persistent traversals of the whole batch
    with CUDA events and return (best launch dict, best leaf size, table).
    `items` as for Batch: (V, T, A, B, mode) tuples of CUDA tensors."""
    from . import Batch
    n_tri = sum(int(t[1].shape[0]) for t in items)
    n_seg = sum(int(t[2].shape[0]) for t in items)
    key = cache_key("batch%d" % len(items), n_tri, n_seg, items[0][0].device)
    if cache:
        hit = _load(cache).get(key)
        if hit:
            return hit["launch"], hit["leaf_size"], hit.get("table", [])
    s = stream if stream is not None else torch.cuda.current_stream()
    rows = []
    with torch.cuda.stream(s):
        for leaf in leaf_sizes:
            for bs in block_sizes:
                for sd in stack_depths:
                    launch = dict(block_size=bs, stack_depth=sd)
                    b = Batch(items, leaf_size=leaf, launch=launch, stream=s)
                    b.build(stream=s)
                    b.intersect(stream=s)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    ms = []
                    for _ in range(reps):
                        e0.record(s)
                        b.intersect(stream=s)
                        e1.record(s)
                        e1.synchronize()
                        ms.append(e0.elapsed_time(e1))
                    b.close()
                    rows.append(dict(block_size=bs, stack_depth=sd, leaf_size=leaf,
                                     ms=sorted(ms)[len(ms) // 2]))
    best = min(rows, key=lambda r: r["ms"])
    launch = dict(block_size=best["block_size"], stack_depth=best["stack_depth"])
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        data = _load(cache)
        data[key] = dict(launch=launch, leaf_size=best["leaf_size"], table=rows)
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return launch, best["leaf_size"], rows
