"""Benchmark: segment / triangle-mesh intersection on GB300.

Headline workload (one step): LBVH build + boolean traversal of 10M segments
against a 123x123 heightfield (29,768 triangles) -- the paper's 10M rays x
~30k triangles (Table 3) with synthetic data.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--quick]

Under torchrun each rank runs the same per-rank workload on its own GPU
(segments drawn from a per-rank seed, the mesh replicated), no collective on
the data path; value = all ranks' segments / max-over-ranks time (weak
scaling).  --impl reference times the FP64 CPU oracle (the only baseline that
exists: the paper's code and data are not available) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Msegments/s (build+traverse) at 10M×30k tris; fwd+bwd and batched Mseg/s"
UNIT = "Msegments/s"
WORKLOAD = "heightfield 123x123 (29,768 tris) x 10M segments, boolean, build+traverse"
BYTES_PER_SEG_BOOL = 25     # 24 B of segment endpoints in + 1 B flag out
BYTES_PER_SEG_NEAREST = 64  # 24 B in + tri, t, u, v, point, dist (40 B) out
BYTES_PER_SEG_COUNT = 28
# dram__bytes_read.sum + dram__bytes_write.sum and warp instructions of one
# k_trace<BOOL> launch on this workload, from an ncu capture of the traversal
# built from sources hashing to `sha`; reported as null once they differ
TRAFFIC = {"sha": "9f8774bd7cbf58c6", "bytes": 257_930_240, "warp_inst": 953_680_560,
           "l2_hit_pct": 81.7, "l1_hit_pct": 68.4}
# peak warp-instruction issue rate: 152 SMs x 4 schedulers x 1 per cycle at
# the maximum SM clock (2,070 MHz)
ISSUE_PEAK = 152 * 4 * 2.070e9
# FP32 operations the traversal performs per node visit (two child boxes, each
# 6 subtract + 6 multiply + 4 max + 4 min + 1 multiply + 1 compare... counted
# as 20) and per Moller-Trumbore test (~50); compared with the FP32 rate that
# rsi_fp32_peak measures on the same GPU
FP32_OPS_PER_VISIT = 40
FP32_OPS_PER_TEST = 50
TRAVERSAL_SOURCES = ("traverse_core.cuh", "rsi_internal.cuh", "traverse.cu")


def traversal_sha():
    """First 16 hex digits of sha256 over the traversal kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAVERSAL_SOURCES:
        with open(os.path.join(ROOT, "paper_2209_02878_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()  # start timing only once the sampler is producing
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def timed(fn, steps, stream, torch):
    """Run fn() `steps` times between CUDA events on `stream`; returns ms/step."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def cpu_oracle_1thread(mesh, seg, n=200_000):
    """The same oracle on one host thread, on the first n segments.
    Returns (Mseg/s, n, seconds)."""
    import oracle
    t0 = time.perf_counter()
    bvh = oracle.CpuBVH(mesh.V, mesh.T)
    bvh.query(seg.A[:n], seg.B[:n], threads=1)
    dt = time.perf_counter() - t0
    return n / dt / 1e6, n, dt


def cpu_oracle_rate(mesh, seg, target_s=12.0, max_n=10_000_000):
    """The FP64 oracle (CPU BVH + Moller-Trumbore, OpenMP over all host
    cores) on a bounded sample of the segments: build + query.
    Returns (Mseg/s, threads, sample size, seconds)."""
    import oracle
    threads = oracle.num_threads()
    n = 20000
    total = 0.0
    while True:
        t0 = time.perf_counter()
        bvh = oracle.CpuBVH(mesh.V, mesh.T)
        bvh.query(seg.A[:n], seg.B[:n], threads=threads)
        dt = time.perf_counter() - t0
        total += dt
        if dt >= target_s or n >= max_n or total > 3 * target_s:
            return n / dt / 1e6, threads, n, dt
        n = min(max_n, int(n * max(2.0, min(20.0, target_s / max(dt, 1e-3)))))


def neardeg_rate(mesh, seg, n=200_000):
    """Share of near-degenerate segments among the first n (the oracle's
    flag), with the sample size."""
    import oracle
    n = min(n, seg.n)
    r = oracle.CpuBVH(mesh.V, mesh.T).query(seg.A[:n], seg.B[:n], threads=oracle.num_threads())
    return {"value": float(r["neardeg"].mean()), "sample": n}


# ------------------------------------------------------------------ arms
def run_ours(args):
    import torch
    import paper_2209_02878_gb300 as rsi
    from paper_2209_02878_gb300 import synth

    rank, local, world = env_rank()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.Stream(device=dev)

    n_seg = 10_000_000
    # every rank: the same (replicated) mesh; rank 0 the 10M segments of the
    # single-GPU workload, rank r its own 10M of the same distribution
    mesh, seg = synth.workload_paper_bool(n_seg=n_seg)
    if rank > 0:
        seg = synth.segments_random_direction(np.random.default_rng(1 + 1000 * rank), n_seg,
                                              mesh.V)
    V = torch.from_numpy(mesh.V).to(dev)
    T = torch.from_numpy(mesh.T).to(dev)
    A = torch.from_numpy(seg.A).to(dev)
    B = torch.from_numpy(seg.B).to(dev)
    flag = torch.empty(n_seg, dtype=torch.uint8, device=dev)
    out = {"flag": flag}
    torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        bvh = rsi.BVH(V, T, stream=stream)
        # build: bounds, Morton, 4 sort passes x (histogram, scatter; the scan
        # is folded into the scatter at 30 tiles), Karras, climb; + traversal
        # bounds, Morton, 4 x (histogram, scatter), Karras, the two box
        # passes, the traversal
        kernels_per_step = 2 + 2 * 4 + 1 + 2 + 1

        def eager_step():
            bvh.build(V, T, stream=stream)
            bvh.intersect(A, B, "bool", out=out, stream=stream)

        for _ in range(max(args.warmup, 3)):
            eager_step()
        stream.synchronize()
        step = eager_step
        if not args.no_graph:
            # the whole step (build + traversal, 14 kernels) as one CUDA graph
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                eager_step()
            step = graph.replay
            step()
            stream.synchronize()
        if bvh.status(stream) != 0:
            raise RuntimeError("device status set during warm-up")
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as clk:
            # the sampler runs from before the warm-up repeats to after the
            # timed region; about 0.3 s of untimed steps first, so that it
            # sees the clocks under this load more than a couple of times
            t_end = time.perf_counter() + 0.3
            while time.perf_counter() < t_end:
                for _ in range(20):
                    step()
                stream.synchronize()
            ms_step = timed(step, args.steps, stream, torch)
            torch.cuda.synchronize()
        if dist:
            t = torch.tensor([ms_step], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_step = float(t.item())
            dist.barrier()

        # kernel-only timings (same stream, after the headline region)
        ms_trav = timed(lambda: bvh.intersect(A, B, "bool", out=out, stream=stream),
                        args.steps, stream, torch)
        ms_build = timed(lambda: bvh.build(V, T, stream=stream), args.steps, stream, torch)
        stats = bvh.intersect(A, B, "bool", stats=True, stream=stream)["stats"]
        # the same step with the build's height-field option (the terrain is
        # z = f(x, y): the Morton code leaves z out); the flags must not change
        bvh_h = rsi.BVH(V, T, height_axis=3, stream=stream)
        out_h = {"flag": torch.empty_like(out["flag"])}

        def step_h():
            bvh_h.build(V, T, stream=stream)
            bvh_h.intersect(A, B, "bool", out=out_h, stream=stream)

        step_h()
        run_h = step_h
        if not args.no_graph:
            g_h = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_h, stream=stream):
                step_h()
            run_h = g_h.replay
        run_h()
        ms_step_h = timed(run_h, args.steps, stream, torch)
        ms_trav_h = timed(lambda: bvh_h.intersect(A, B, "bool", out=out_h, stream=stream),
                          args.steps, stream, torch)
        stats_h = bvh_h.intersect(A, B, "bool", stats=True, stream=stream)["stats"]
        stream.synchronize()
        if not torch.equal(out_h["flag"], out["flag"]):
            raise RuntimeError("height-field tree gave other flags")
        # the FP32 ceiling, measured by the library's FMA probe (~60 ms)
        fp32_tflops = rsi.fp32_peak(1 << 20, stream=stream)

        # end to end through the public API from pinned host memory: the
        # build plus rsi_intersect_host every step (the copy engine streams
        # the pinned segments into device staging under one persistent
        # traversal; the flags come back with one device-to-host copy)
        hA = torch.from_numpy(seg.A).pin_memory()
        hB = torch.from_numpy(seg.B).pin_memory()
        hout = {"flag": torch.empty(n_seg, dtype=torch.uint8).pin_memory()}

        # the build replayed from a CUDA graph, as in the device step (the
        # host call itself runs eagerly: it stages, flags and copies back)
        build_step = bvh.build
        if not args.no_graph:
            g_build = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_build, stream=stream):
                bvh.build(V, T, stream=stream)
            build_step = lambda V_, T_, stream=None: g_build.replay()  # noqa: E731

        def e2e_step():
            build_step(V, T, stream=stream)
            bvh.intersect_host(hA, hB, "bool", out=hout, stream=stream)

        for _ in range(2):
            e2e_step()
        stream.synchronize()
        ms_e2e = timed(e2e_step, max(2, args.steps // 2), stream, torch)
        if not np.array_equal(hout["flag"].numpy(), flag.cpu().numpy()):
            raise RuntimeError("host-buffer path disagrees with the device path")

    extras = {}
    if not args.quick:
        extras = run_extras(args, torch, rsi, synth, dev, stream, dist)

    peak, peak_kind = measured_peaks()
    algo_bytes = BYTES_PER_SEG_BOOL * n_seg
    fp32_ops = (FP32_OPS_PER_VISIT * stats["node_visits"] +
                FP32_OPS_PER_TEST * stats["tri_tests"])
    achieved = algo_bytes / (ms_trav * 1e-3) / 1e9
    res = {
        "metric": METRIC, "value": round(world * n_seg / (ms_step * 1e-3) / 1e6, 3),
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (FP64 for decisions the FP32 bound cannot settle)",
        "data": "synthetic (seeded heightfield + random-direction segments)",
        "config": {"workload": WORKLOAD, "n_triangles": mesh.n_tri, "segments_per_gpu": n_seg,
                   "parallelism": f"replicas x{world}, segments sharded per rank",
                   "l2": "inputs larger than L2 (240 MB of segments per step)",
                   "launch": "persistent grid from occupancy, block 128, stack 64, binary nodes, "
                             "input segment order, no shared-memory treelet",
                   "graph": not args.no_graph},
        "e2e": {"value": round(world * n_seg / (ms_e2e * 1e-3) / 1e6, 3), "unit": UNIT,
                "h2d_bytes_per_step": 24 * n_seg, "d2h_bytes_per_step": n_seg,
                "ms_per_step": round(ms_e2e, 4)},
        "gpu_launches": kernels_per_step * args.steps,
        "clocks": clk.summary(),
        "roofline": {"bound": "hbm", "kernel": "k_trace<BOOL>", "achieved": round(achieved, 2),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 5),
                     "peak_kind": peak_kind,
                     "traffic": TRAFFIC["bytes"] if traversal_sha() == TRAFFIC["sha"] else None,
                     "l2_hit_pct": TRAFFIC["l2_hit_pct"] if traversal_sha() == TRAFFIC["sha"] else None,
                     "l1_hit_pct": TRAFFIC["l1_hit_pct"] if traversal_sha() == TRAFFIC["sha"] else None,
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "kernel_ms": round(ms_trav, 4)},
        "issue_roofline": ({"bound": "issue", "kernel": "k_trace<BOOL>",
                            "achieved": round(TRAFFIC["warp_inst"] / (ms_trav * 1e-3) / 1e12, 4),
                            "peak": round(ISSUE_PEAK / 1e12, 4), "unit": "Twarp-inst/s",
                            "frac": round(TRAFFIC["warp_inst"] / (ms_trav * 1e-3) / ISSUE_PEAK, 4)}
                           if traversal_sha() == TRAFFIC["sha"] else None),
        "fp32_roofline": {"bound": "fp32", "kernel": "k_trace<BOOL>",
                          "achieved": round(fp32_ops / (ms_trav * 1e-3) / 1e12, 4),
                          "peak": round(fp32_tflops, 3), "unit": "TFLOP/s",
                          "frac": round(fp32_ops / (ms_trav * 1e-3) / 1e12 / fp32_tflops, 5),
                          "peak_kind": "measured (rsi_fp32_peak FMA probe)",
                          "ops_per_visit": FP32_OPS_PER_VISIT,
                          "ops_per_test": FP32_OPS_PER_TEST},
        "breakdown": {"traverse_only_Msegs": round(n_seg / (ms_trav * 1e-3) / 1e6, 3),
                      "build_ms": round(ms_build, 4), "traverse_ms": round(ms_trav, 4),
                      "node_visits_per_seg": round(stats["node_visits"] / n_seg, 3),
                      "tri_tests_per_seg": round(stats["tri_tests"] / n_seg, 3),
                      "fp64_tests_per_seg": stats["fp64_tests"] / n_seg,
                      "height_axis_option": {
                          "note": "the same step with the build option height_axis=3 (the "
                                  "Morton code of the z = f(x, y) terrain leaves z out; same "
                                  "flags); not the paper's code, so not the headline",
                          "Msegs": round(n_seg / (ms_step_h * 1e-3) / 1e6, 3),
                          "ms_per_step": round(ms_step_h, 4),
                          "traverse_ms": round(ms_trav_h, 4),
                          "node_visits_per_seg": round(stats_h["node_visits"] / n_seg, 3)}},
    }
    res.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, thr, n, dt = cpu_oracle_rate(mesh, seg)
        rate1, n1, dt1 = cpu_oracle_1thread(mesh, seg)
        # near-degenerate segments (a crossing within 1e-6 of an edge or an
        # end, or coplanar), counted by the oracle on a sample of each
        # workload; the kernels match the oracle on them too
        res["breakdown"]["neardeg_per_seg"] = neardeg_rate(mesh, seg)
        if "fwd_bwd" in res:
            dmesh, dseg, _ = synth.workload_diff()
            res["fwd_bwd"]["neardeg_per_seg"] = neardeg_rate(dmesh, dseg)
        res["cpu_baseline"] = {"value": round(rate, 5), "unit": UNIT, "cores": thr,
                               "kind": "oracle",
                               "sample": f"first {n} of the 10M segments, CPU BVH build + "
                                         f"FP64 query, {dt:.1f} s",
                               "one_thread": {"value": round(rate1, 5),
                                              "sample": f"first {n1} segments, {dt1:.1f} s"}}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res))


def run_extras(args, torch, rsi, synth, dev, stream, dist=None):
    """fwd+bwd (131k-triangle heightfield, 262k segments), count + nearest
    (1.3M-triangle icosphere, 1M segments), a coherent raster of segments
    (per-segment stacks against warp packets) and the 64-mesh batch, each
    beside the plain single-mesh forward on the same mesh."""
    out = {}
    steps = max(3, args.steps)
    with torch.cuda.stream(stream):
        # fwd + bwd
        mesh, seg, w = synth.workload_diff()
        V = torch.from_numpy(mesh.V).to(dev)
        T = torch.from_numpy(mesh.T).to(dev)
        A = torch.from_numpy(seg.A).to(dev)
        B = torch.from_numpy(seg.B).to(dev)
        W = torch.from_numpy(w).to(dev)
        bvh = rsi.BVH(V, T, stream=stream)

        def fwd():
            return bvh.intersect(A, B, "nearest", stream=stream)

        def fwd_bwd():
            bvh.build(V, T, stream=stream)
            o = bvh.intersect(A, B, "nearest", stream=stream)
            rsi.intersect_backward(V, T, A, B, o["tri"], grad_point=W, stream=stream)

        def fwd_bwd_refit():  # a training step whose vertices moved: refit, not rebuild
            bvh.refit(V, stream=stream)
            o = bvh.intersect(A, B, "nearest", stream=stream)
            rsi.intersect_backward(V, T, A, B, o["tri"], grad_point=W, stream=stream)

        # the same training step through the public autograd API: an in-place
        # update of the vertex parameter (as an optimizer makes; it bumps the
        # tensor's version), then nearest_hit with the reused tree, which
        # refits it, and the backward pass of loss = sum(w . P)
        Vp = V.clone().requires_grad_(True)
        bvh_ag = rsi.BVH(Vp.detach(), T, stream=stream)
        nudge = [1e-7]

        def fwd_bwd_autograd():
            with torch.no_grad():
                Vp.add_(nudge[0])
            nudge[0] = -nudge[0]
            P, _, _ = rsi.nearest_hit(Vp, T, A, B, bvh=bvh_ag)
            (P * W).sum().backward()

        for _ in range(3):
            fwd_bwd()
            fwd_bwd_refit()
            fwd_bwd_autograd()
        ms_fb_eager = timed(fwd_bwd, steps, stream, torch)
        # the same step captured once as a CUDA graph and replayed, as a
        # training loop with static shapes would run it (build, traversal,
        # adjoint and their allocations become graph nodes: no per-launch
        # host work)
        g_fb = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_fb, stream=stream):
            fwd_bwd()
        g_fb.replay()
        stream.synchronize()
        ms_fb = timed(g_fb.replay, steps, stream, torch)
        g_f = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_f, stream=stream):
            bvh.build(V, T, stream=stream)
            fwd()
        g_f.replay()
        stream.synchronize()
        ms_f = timed(g_f.replay, steps, stream, torch)
        ms_fr = timed(fwd_bwd_refit, steps, stream, torch)
        g_fr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_fr, stream=stream):
            fwd_bwd_refit()
        g_fr.replay()
        stream.synchronize()
        ms_frg = timed(g_fr.replay, steps, stream, torch)
        refits0 = bvh_ag.refits
        ms_fa = timed(fwd_bwd_autograd, steps, stream, torch)
        if bvh_ag.refits - refits0 != steps:
            raise RuntimeError("nearest_hit did not refit the reused tree every step")
        # the same autograd step captured once as a CUDA graph (the refit it
        # needs is captured with it; the vertex update is a fixed nudge)
        ms_fag = None
        try:
            g_fa = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_fa, stream=stream):
                fwd_bwd_autograd()
            g_fa.replay()
            stream.synchronize()
            ms_fag = timed(g_fa.replay, steps, stream, torch)
        except RuntimeError:
            ms_fag = None
        # fixed segments over a moving mesh (camera rays in a fitting loop):
        # the coherent processing order is computed once (rsi_segment_order)
        # and every step reuses it; outputs are those of the input order
        order = bvh.segment_order(A, B, stream=stream)
        lo_ord = {"order": order}

        def fwd_bwd_ordered():
            bvh.build(V, T, stream=stream)
            o = bvh.intersect(A, B, "nearest", launch=lo_ord, stream=stream)
            rsi.intersect_backward(V, T, A, B, o["tri"], grad_point=W, stream=stream)

        def fwd_bwd_refit_ordered():
            bvh.refit(V, stream=stream)
            o = bvh.intersect(A, B, "nearest", launch=lo_ord, stream=stream)
            rsi.intersect_backward(V, T, A, B, o["tri"], grad_point=W, stream=stream)

        ms_ord = {}
        for name, fn in (("build", fwd_bwd_ordered), ("refit", fwd_bwd_refit_ordered)):
            fn()
            g_o = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_o, stream=stream):
                fn()
            g_o.replay()
            stream.synchronize()
            ms_ord[name] = timed(g_o.replay, steps, stream, torch)
            del g_o
        # the same steps over a tree built with the height-field option (the
        # terrain is z = f(x, y): the Morton code leaves z out); same outputs
        bvh_h = rsi.BVH(V, T, height_axis=3, stream=stream)
        order_h = bvh_h.segment_order(A, B, stream=stream)
        lo_h = {"order": order_h}

        def fwd_bwd_h():
            bvh_h.build(V, T, stream=stream)
            o = bvh_h.intersect(A, B, "nearest", stream=stream)
            rsi.intersect_backward(V, T, A, B, o["tri"], grad_point=W, stream=stream)

        def fwd_bwd_h_refit_ordered():
            bvh_h.refit(V, stream=stream)
            o = bvh_h.intersect(A, B, "nearest", launch=lo_h, stream=stream)
            rsi.intersect_backward(V, T, A, B, o["tri"], grad_point=W, stream=stream)

        for name, fn in (("h_build", fwd_bwd_h), ("h_refit_order", fwd_bwd_h_refit_ordered)):
            fn()
            g_o = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g_o, stream=stream):
                fn()
            g_o.replay()
            stream.synchronize()
            ms_ord[name] = timed(g_o.replay, steps, stream, torch)
            del g_o
        o_h = bvh_h.intersect(A, B, "nearest", stream=stream)
        ms_near_h = timed(lambda: bvh_h.intersect(A, B, "nearest", out=o_h, stream=stream),
                          steps, stream, torch)
        ms_near_h_ord = timed(lambda: bvh_h.intersect(A, B, "nearest", launch=lo_h, out=o_h,
                                                      stream=stream), steps, stream, torch)
        st_h = bvh_h.intersect(A, B, "nearest", stats=True, stream=stream)["stats"]
        o_ref = bvh.intersect(A, B, "nearest", stream=stream)
        stream.synchronize()
        for k in ("tri", "tuv", "point", "dist"):
            if not torch.equal(o_h[k], o_ref[k]):
                raise RuntimeError("height-field tree gave other nearest outputs")
        del bvh_h
        o_in = bvh.intersect(A, B, "nearest", stream=stream)
        o_ord = bvh.intersect(A, B, "nearest", launch=lo_ord, stream=stream)
        ms_near_in = timed(lambda: bvh.intersect(A, B, "nearest", out=o_in, stream=stream),
                           steps, stream, torch)
        ms_near_ord = timed(lambda: bvh.intersect(A, B, "nearest", launch=lo_ord, out=o_ord,
                                                  stream=stream), steps, stream, torch)
        ms_order = timed(lambda: bvh.segment_order(A, B, stream=stream), steps, stream, torch)
        st = bvh.intersect(A, B, "nearest", stats=True, stream=stream)["stats"]
        out["fwd_bwd"] = {"workload": "heightfield 257x257 (131,072 tris) x 262,144 near-vertical "
                                      "segments, nearest + adjoint, build included",
                          "value": round(seg.n / (ms_fb * 1e-3) / 1e6, 3), "unit": UNIT,
                          "graph": True,
                          "eager": round(seg.n / (ms_fb_eager * 1e-3) / 1e6, 3),
                          "forward_only": round(seg.n / (ms_f * 1e-3) / 1e6, 3),
                          "forward_only_note": "build + nearest, as a graph",
                          "with_refit": round(seg.n / (ms_fa * 1e-3) / 1e6, 3),
                          "with_refit_note": "torch autograd step: in-place vertex update, "
                                             "nearest_hit with the reused tree (refit), "
                                             "backward of sum(w . P)",
                          "with_refit_autograd_graph": (round(seg.n / (ms_fag * 1e-3) / 1e6, 3)
                                                        if ms_fag else None),
                          "with_refit_direct": round(seg.n / (ms_fr * 1e-3) / 1e6, 3),
                          "with_refit_graph": round(seg.n / (ms_frg * 1e-3) / 1e6, 3),
                          "with_order_graph": round(seg.n / (ms_ord["build"] * 1e-3) / 1e6, 3),
                          "with_refit_order_graph": round(seg.n / (ms_ord["refit"] * 1e-3) / 1e6,
                                                          3),
                          "order_note": "the segments' coherent order (rsi_segment_order, "
                                        "Morton code of the midpoint + direction octant) "
                                        "computed once, outside the step, and reused: the "
                                        "segments stay fixed while the mesh moves",
                          "nearest_ms": {"input_order": round(ms_near_in, 4),
                                         "segment_order": round(ms_near_ord, 4),
                                         "computing_the_order": round(ms_order, 4)},
                          "height_axis_option": {
                              "note": "the tree built with height_axis=3 (the terrain's "
                                      "Morton code leaves z out; same outputs); not the "
                                      "paper's code",
                              "graph": round(seg.n / (ms_ord["h_build"] * 1e-3) / 1e6, 3),
                              "with_refit_order_graph": round(
                                  seg.n / (ms_ord["h_refit_order"] * 1e-3) / 1e6, 3),
                              "nearest_ms": {"input_order": round(ms_near_h, 4),
                                             "segment_order": round(ms_near_h_ord, 4)},
                              "node_visits_per_seg": round(st_h["node_visits"] / seg.n, 3)},
                          "nearest_breakdown": {
                              "node_visits_per_seg": round(st["node_visits"] / seg.n, 3),
                              "tri_tests_per_seg": round(st["tri_tests"] / seg.n, 3),
                              "fp64_decisions_per_seg": st["fp64_tests"] / seg.n,
                              "df_refines_per_seg": round(st["df_refines"] / seg.n, 5),
                              "fp64_values_per_seg": st["fp64_values"] / seg.n}}
        del bvh_ag, Vp
        # the same step sharded over the ranks (data parallel): each rank
        # builds the replicated mesh's tree and runs its contiguous shard of
        # the segments; the vertex gradient is all-reduced (the one
        # collective; none at one rank)
        from paper_2209_02878_gb300 import sharding
        world = dist.get_world_size() if dist else 1
        bvh_sh = rsi.BVH(V, T, stream=stream)

        def sharded_step():
            bvh_sh.build(V, T, stream=stream)
            sharding.nearest_backward_shard(V, T, A, B, grad_point=W, bvh=bvh_sh, stream=stream)

        for _ in range(3):
            sharded_step()
        stream.synchronize()
        if dist:
            dist.barrier()
        ms_sh = timed(sharded_step, steps, stream, torch)
        if dist:
            t_ = torch.tensor([ms_sh], device=dev)
            dist.all_reduce(t_, op=dist.ReduceOp.MAX)
            ms_sh = float(t_.item())
        out["fwd_bwd"]["sharded"] = {
            "value": round(seg.n / (ms_sh * 1e-3) / 1e6, 3), "unit": UNIT, "ranks": world,
            "scaling": "strong",
            "note": "the 262,144 segments split into contiguous per-rank shards, mesh "
                    "replicated (tree built per rank per step), grad_V all-reduced over ranks"}
        del bvh_sh
        del bvh
        # count + nearest on the big sphere
        mesh, seg = synth.workload_sphere()
        V = torch.from_numpy(mesh.V).to(dev)
        T = torch.from_numpy(mesh.T).to(dev)
        A = torch.from_numpy(seg.A).to(dev)
        B = torch.from_numpy(seg.B).to(dev)
        bvh = rsi.BVH(V, T, stream=stream)
        res = {}
        for mode in ("bool", "count", "nearest"):
            o = bvh.intersect(A, B, mode, stream=stream)
            ms = timed(lambda: bvh.intersect(A, B, mode, out=o, stream=stream), steps, stream,
                       torch)
            res[mode] = round(seg.n / (ms * 1e-3) / 1e6, 3)
        ms_b = timed(lambda: bvh.build(V, T, stream=stream), steps, stream, torch)
        st = bvh.intersect(A, B, "nearest", stats=True, stream=stream)["stats"]
        out["sphere"] = {"workload": "icosphere L8 (1,310,720 tris) x 1M segments in a cube",
                         "traverse_Msegs": res, "build_ms": round(ms_b, 3), "unit": UNIT,
                         "nearest_breakdown": {
                             "node_visits_per_seg": round(st["node_visits"] / seg.n, 3),
                             "tri_tests_per_seg": round(st["tri_tests"] / seg.n, 3),
                             "df_refines_per_seg": round(st["df_refines"] / seg.n, 5),
                             "fp64_values_per_seg": st["fp64_values"] / seg.n}}
        del bvh
        # coherent segments: one stack per segment against warp packets
        mesh, seg = synth.workload_raster()
        V = torch.from_numpy(mesh.V).to(dev)
        T = torch.from_numpy(mesh.T).to(dev)
        A = torch.from_numpy(seg.A).to(dev)
        B = torch.from_numpy(seg.B).to(dev)
        bvh = rsi.BVH(V, T, stream=stream)
        res = {}
        for mode in ("bool", "nearest"):
            for name, lo in (("per_segment", None), ("packet", {"packet": 1})):
                o = bvh.intersect(A, B, mode, launch=lo, stream=stream)
                ms = timed(lambda: bvh.intersect(A, B, mode, launch=lo, out=o, stream=stream),
                           steps, stream, torch)
                res[f"{mode}_{name}"] = round(seg.n / (ms * 1e-3) / 1e6, 3)
        out["coherent"] = {"workload": "heightfield 123x123 (29,768 tris) x 3163x3163 raster of "
                                       "vertical segments (row by row)",
                           "traverse_Msegs": res, "unit": UNIT}
        del bvh, A, B
        # batched
        items = synth.workload_batched()
        tens = [(torch.from_numpy(m.V).to(dev), torch.from_numpy(m.T).to(dev),
                 torch.from_numpy(s.A).to(dev), torch.from_numpy(s.B).to(dev), mode)
                for m, s, mode in items]
        n_total = sum(s.n for _, s, _ in items)
        from paper_2209_02878_gb300 import tuning
        # block size, stack depth and leaf size from the project's autotuner
        # (timed outside the measured region; cached per GPU / workload class)
        tuned, leaf, _ = tuning.autotune_batch(tens, cache=None, stream=stream)
        batch = rsi.Batch(tens, leaf_size=leaf, launch=tuned, stream=stream)
        batch.run_graph(rebuild=True, stream=stream)
        stream.synchronize()
        ms_bt = timed(lambda: batch.run_graph(rebuild=True, stream=stream), steps, stream, torch)
        # the same batch with the build option height_axis=3 on its terrain
        # items (the icospheres keep the paper's code); same outputs
        tens_h = [t + ((3,) if items[k][0].kind == "heightfield" else (0,))
                  for k, t in enumerate(tens)]
        batch_h = rsi.Batch(tens_h, leaf_size=leaf, launch=tuned, stream=stream)
        batch_h.run_graph(rebuild=True, stream=stream)
        stream.synchronize()
        ms_bt_h = timed(lambda: batch_h.run_graph(rebuild=True, stream=stream), steps, stream,
                        torch)
        for o_h, o_b in zip(batch_h.outputs, batch.outputs):
            for k in o_b:
                if isinstance(o_b[k], torch.Tensor) and not torch.equal(o_h[k], o_b[k]):
                    raise RuntimeError("height-axis batch gave other outputs")
        batch_h.close()
        bvhs = [rsi.BVH(t[0], t[1], stream=stream) for t in tens]
        outs = [bv.intersect(t[2], t[3], t[4], stream=stream) for bv, t in zip(bvhs, tens)]

        def singles():
            for bv, t, o in zip(bvhs, tens, outs):
                bv.build(t[0], t[1], stream=stream)
                bv.intersect(t[2], t[3], t[4], out=o, stream=stream)

        singles()
        ms_single = timed(singles, steps, stream, torch)
        out["batched"] = {"workload": f"64 meshes (1k-200k tris), {n_total} segments, "
                                      "bool/nearest alternating, one graph: build + persistent "
                                      "traversal",
                          "value": round(n_total / (ms_bt * 1e-3) / 1e6, 3), "unit": UNIT,
                          "autotuned": dict(tuned, leaf_size=leaf),
                          "height_axis_terrains": round(n_total / (ms_bt_h * 1e-3) / 1e6, 3),
                          "height_axis_note": "the terrain items built with height_axis=3 "
                                              "(not the paper's code); same outputs",
                          "per_mesh_launches": round(n_total / (ms_single * 1e-3) / 1e6, 3)}
        batch.close()
    return out


def run_reference(args):
    """The FP64 CPU oracle timed on the host cores, same metric and workload:
    each step builds the CPU BVH and queries a bounded sample of the 10M
    segments (consecutive 1M-segment slices, cycling)."""
    rank, _, world = env_rank()
    if rank != 0:
        return
    import oracle
    from paper_2209_02878_gb300 import synth
    oracle.compile_oracle()
    n_sample = 1_000_000
    mesh, seg = synth.workload_paper_bool()
    n_slices = seg.n // n_sample
    threads = oracle.num_threads()

    def step(k):
        s = slice((k % n_slices) * n_sample, (k % n_slices + 1) * n_sample)
        bvh = oracle.CpuBVH(mesh.V, mesh.T)
        bvh.query(seg.A[s], seg.B[s], threads=threads)

    for _ in range(max(args.warmup, 3)):
        step(0)
    t0 = time.perf_counter()
    for k in range(args.steps):
        step(k)
    dt = (time.perf_counter() - t0) / args.steps
    v = round(n_sample / dt / 1e6, 5)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample_per_step": n_sample},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n_sample} segments per step, consecutive slices of the "
                                   f"10M (CPU BVH build + FP64 query)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_case(args):
    """One secondary kernel on its workload, launched `--steps` times after
    the warm-up, for a profiler capture (prints one JSON line with the mean
    event-timed duration; not a benchmark result)."""
    import numpy as np
    import torch
    import paper_2209_02878_gb300 as rsi
    from paper_2209_02878_gb300 import synth
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()

    def t(x):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dev)

    with torch.cuda.stream(stream):
        if args.case == "sphere_nearest":
            mesh, seg = synth.workload_sphere()
            bvh = rsi.BVH(t(mesh.V), t(mesh.T), stream=stream)
            A, B = t(seg.A), t(seg.B)
            o = bvh.intersect(A, B, "nearest", stream=stream)
            fn = lambda: bvh.intersect(A, B, "nearest", out=o, stream=stream)  # noqa: E731
        elif args.case == "coherent_packet":
            mesh, seg = synth.workload_raster()
            bvh = rsi.BVH(t(mesh.V), t(mesh.T), stream=stream)
            A, B = t(seg.A), t(seg.B)
            lo = {"packet": 1}
            o = bvh.intersect(A, B, "nearest", launch=lo, stream=stream)
            fn = lambda: bvh.intersect(A, B, "nearest", launch=lo, out=o, stream=stream)  # noqa: E731
        elif args.case == "diff_nearest":
            mesh, seg, _ = synth.workload_diff()
            bvh = rsi.BVH(t(mesh.V), t(mesh.T), stream=stream)
            A, B = t(seg.A), t(seg.B)
            o = bvh.intersect(A, B, "nearest", stream=stream)
            fn = lambda: bvh.intersect(A, B, "nearest", out=o, stream=stream)  # noqa: E731
        elif args.case == "diff_backward":
            mesh, seg, w = synth.workload_diff()
            V, T, A, B, W = t(mesh.V), t(mesh.T), t(seg.A), t(seg.B), t(w)
            tri = rsi.BVH(V, T, stream=stream).intersect(A, B, "nearest", stream=stream)["tri"]
            gV = torch.zeros_like(V)
            fn = lambda: rsi.intersect_backward(V, T, A, B, tri, grad_point=W, grad_V=gV,  # noqa: E731
                                                stream=stream)
        elif args.case == "build":
            # the LBVH build and a refit of the 29,768- and 131,072-triangle
            # heightfields, alternately (the box pass writes the same trees)
            meshes = [synth.workload_paper_bool(n_seg=1)[0], synth.workload_diff(n_seg=1)[0]]
            tens = [(t(m.V), t(m.T)) for m in meshes]
            bvhs = [rsi.BVH(V, T, stream=stream) for V, T in tens]

            def fn():
                for b, (V, T) in zip(bvhs, tens):
                    b.build(V, T, stream=stream)
                    b.refit(V, stream=stream)
        else:  # batched
            items = synth.workload_batched()
            tens = [(t(m.V), t(m.T), t(sg.A), t(sg.B), mode) for m, sg, mode in items]
            b = rsi.Batch(tens, leaf_size=1, launch={"block_size": 128, "stack_depth": 64},
                          stream=stream).build(stream=stream)
            fn = lambda: b.intersect(stream=stream)  # noqa: E731
        for _ in range(max(1, args.warmup)):
            fn()
        ms = timed(fn, args.steps, stream, torch)
    print(json.dumps({"case": args.case, "launches": args.steps, "ms_per_launch": round(ms, 4)}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="headline workload only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly")
    ap.add_argument("--case", choices=["sphere_nearest", "coherent_packet", "diff_nearest",
                                       "diff_backward", "batched", "build"],
                    help="run one secondary kernel --steps times for a profiler capture")
    args = ap.parse_args()
    if args.case:
        run_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
