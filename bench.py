#!/usr/bin/env python
"""Frame benchmark of the GB300 visibility-buffer rasterizer.

Default workload: the billion-scale terrain -- 64 seeded heightfield tiles of
4096 x 4096 cells (2^31 triangles, ~43 GB of FP32 positions, uint32 indices
and RGBA8 colours resident in HBM) in an 8 x 8 layout, one 3840 x 2160
overview view whose frustum leaves out 18 tiles.  A step is one frame:
clear, stage 1, stage 2, stage 3 (curast_render).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank renders its own copy of the
frame (the rasterizer has no exchange step: replicas only); the time is
the maximum over ranks and the value counts the triangles of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--tiles", type=int, default=8, help="tiles per side of the terrain")
    p.add_argument("--cells", type=int, default=4096, help="cells per tile side")
    p.add_argument("--W", type=int, default=3840)
    p.add_argument("--H", type=int, default=2160)
    p.add_argument("--batched", choices=["full", "small", "off"], default="full",
                   help="also time the batched multi-mesh path against one launch per mesh per view")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-supersampling", dest="supersampling", action="store_false",
                   help="skip the 2x2 / 4x4 super-sampled frames")
    p.add_argument("--no-compressed", dest="compressed", action="store_false",
                   help="skip the frame with compressed geometry")
    p.add_argument("--no-ablation", dest="ablation", action="store_false",
                   help="skip the frame without the conservative cull (every triangle on the exact path)")
    p.add_argument("--no-diff", dest="diff", action="store_false",
                   help="skip the differentiable interpolation step (forward and backward)")
    p.add_argument("--no-resolve", dest="resolve", action="store_false",
                   help="skip timing the resolve and the textured resolve of the frame")
    p.add_argument("--no-unique", dest="unique", action="store_false",
                   help="skip the 100M-triangle heightfield's 8 poses at 1920x1080 and 3840x2160")
    p.add_argument("--no-raycast", dest="raycast", action="store_false",
                   help="skip the stage-3 workloads timed with the fixed-point rule and with the ray cast")
    p.add_argument("--no-thirty", dest="thirty", action="store_false",
                   help="skip the frame of the 30 tiles wholly in view (1.007 B triangles)")
    p.add_argument("--subset", type=int, default=0,
                   help="profiling aid: give geometry only to this many tiles next to the view centre "
                        "(same layout, camera and triangle density; the other tiles are empty)")
    return p.parse_args()


# ------------------------------------------------------------------ ranks ---
class Ranks:
    def __init__(self, gpus: int):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if torch.cuda.is_available():
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        return self._reduce(x, "max")

    def sum(self, x: float) -> float:
        return self._reduce(x, "sum")

    def _reduce(self, x, op):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX if op == "max" else self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------- clocks ---
class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# -------------------------------------------------------------- workloads ---
def billion_scene_gpu(tiles: int, cells: int, device, subset: int = 0):
    import torch
    import synthetic as S
    if not subset:
        return S.scene_billion(device=device, tiles=tiles, n=cells)
    # tiles nearest the point the overview camera looks at
    cx, cz = tiles / 2.0, tiles / 2.0
    order = sorted(range(tiles * tiles), key=lambda k: (k % tiles + 0.5 - cx) ** 2 + (k // tiles + 0.5 - cz) ** 2)
    sc = S.scene_billion(device=device, tiles=tiles, n=cells, only=order[:subset])
    for k, m in enumerate(sc.meshes):
        if m is None:
            sc.meshes[k] = S.Mesh(pos=torch.zeros((3, 3), device=device),
                                  idx=torch.zeros((0, 3), dtype=torch.int32, device=device),
                                  rgba8=torch.zeros((3, 4), dtype=torch.uint8, device=device))
    return sc


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def kernel_source_hash() -> str:
    """Hash of the stage kernels' source code with comments and blank space
    removed (edits to comments do not change the kernel)."""
    import re
    h = hashlib.sha256()
    for f in ("raster.cu", "stage1.cuh", "device.cuh"):
        src = open(os.path.join(ROOT, "paper_2604_21749_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(workload_key: str):
    """DRAM traffic per stage-1 launch from the committed ncu summary, if it
    was captured on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    src = kernel_source_hash()
    for line in open(p):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == "k_stage1" and f[1] == src and f[2] == workload_key:
            return float(f[3])
    return None


_CPU_SAMPLES = {}


def _cpu_sample(tiles: int, cells: int, frac: float, count: int):
    """The oracle's view of `count` adjacent central tiles of the terrain (or
    of the first `frac` of one tile's triangles), generated once and reused
    across steps."""
    key = (tiles, cells, frac, count)
    if key not in _CPU_SAMPLES:
        import synthetic as S
        from oracle import oracle as orc
        k = (tiles // 2) * tiles + tiles // 2 - count // 2      # central, visible tiles
        sc = S.scene_billion(device="cpu", tiles=tiles, n=cells, only=list(range(k, k + count)))
        counts = [2 * cells * cells] * (tiles * tiles)
        if frac < 1.0:
            m = sc.meshes[k]
            m.idx = m.idx[:max(1, int(m.T * frac))].contiguous()
            counts[k] = m.T
        T = sum(sc.meshes[j].T for j in range(k, k + count))
        _CPU_SAMPLES[key] = (orc.OracleScene(sc, tri_counts=counts), k, T)
    return _CPU_SAMPLES[key]


def _all_core_worker(k, tiles, cells, W, H, barrier, queue):
    """One process of the all-core CPU baseline: generates tile k, waits for
    every process, then renders it with the oracle (ids numbered over all
    tiles) and reports (triangles, seconds)."""
    import torch
    torch.set_num_threads(1)
    sys.path.insert(0, ROOT)
    import synthetic as S
    from oracle import oracle as orc
    cam = S.camera_billion(W, H, tiles)
    sc = S.scene_billion(tiles=tiles, n=cells, only=[k], colours=False)
    osc = orc.OracleScene(sc, tri_counts=[2 * cells * cells] * (tiles * tiles))
    import numpy as np
    out = np.full((H, W), orc.EMPTY, np.uint64)
    barrier.wait()
    t0 = time.perf_counter()
    orc.render(osc, cam, first=k, count=1, out=out)
    queue.put((2 * cells * cells, time.perf_counter() - t0))


def cpu_baseline_all_cores(args):
    """The oracle on every host core at once: one process per core (spawned,
    each single-threaded), each rendering one central tile of the frame after
    all have generated theirs; Gtris/s = all their triangles over the
    slowest process's render time (the per-tile buffers would be merged by an
    element-wise minimum, which is not timed)."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    n = min(ncores, args.tiles * args.tiles)
    cx = cz = args.tiles / 2.0
    order = sorted(range(args.tiles * args.tiles),
                   key=lambda k: (k % args.tiles + 0.5 - cx) ** 2 + (k // args.tiles + 0.5 - cz) ** 2)
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_all_core_worker, args=(k, args.tiles, args.cells, args.W, args.H, barrier, queue))
             for k in order[:n]]
    for p in procs:
        p.start()
    res = [queue.get(timeout=600) for _ in procs]
    for p in procs:
        p.join()
    tris = sum(t for t, _ in res)
    slowest = max(s for _, s in res)
    return {"value": round(tris / slowest / 1e9, 5), "unit": "Gtris/s", "cores": n, "kind": "oracle",
            "sample": f"{n} central tiles ({tris} triangles) of the same frame, one single-threaded oracle "
                      f"process per core, slowest {slowest:.1f} s"}


def cpu_baseline_sample(tiles: int, cells: int, W: int, H: int, frac: float = 1.0, count: int = 1):
    """Times the oracle (single thread) on `count` central tiles of the
    terrain, or on the first `frac` of one tile's triangles; returns
    (Gtris/s, triangles, seconds)."""
    import numpy as np
    import synthetic as S
    from oracle import oracle as orc
    osc, k, T = _cpu_sample(tiles, cells, frac, count)
    cam = S.camera_billion(W, H, tiles)
    vis = np.full((H, W), orc.EMPTY, np.uint64)
    t0 = time.perf_counter()
    orc.render(osc, cam, first=k, count=count, out=vis)
    dt = time.perf_counter() - t0
    return T / dt / 1e9, T, dt


# ------------------------------------------------------------ our arm ------
def run_ours(args, ranks: Ranks):
    import numpy as np
    import torch
    import __graft_entry__ as ge
    import synthetic as S
    from paper_2604_21749_gb300 import api

    ge.build()
    dev = torch.device("cuda", ranks.local)
    torch.cuda.set_device(dev)
    t_gen = time.perf_counter()
    sc = billion_scene_gpu(args.tiles, args.cells, dev, args.subset)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    cam = S.camera_billion(args.W, args.H, args.tiles)
    r = api.Renderer(dev.index)
    for m in sc.meshes:
        r.upload_mesh(m.pos, m.idx, m.rgba8)
    for it in sc.instances:
        r.add_instance(it.mesh, it.model)
    vis = r.new_vis(args.W, args.H)
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        r.render(cam.view, cam.proj, args.W, args.H, vis)
        r.sync()
    info = r.last_frame()

    # timed region: K frames; per-frame stage times come from the events the
    # library records around each stage on this stream
    clocks = Clocks(dev.index)
    ranks.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    stage = []
    for _ in range(args.steps):
        r.render(cam.view, cam.proj, args.W, args.H, vis)
        stage.append(r.stage_times())
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    ranks.barrier()
    clk = clocks.stop()
    ms_frame = ranks.max(ms_total / args.steps)
    r.sync()
    # one more frame, untimed, with the per-stage counters on
    r.set_config(collect_stats=1)
    r.render(cam.view, cam.proj, args.W, args.H, vis)
    stats = r.sync()
    r.set_config(collect_stats=0)

    # end to end through the public API with host buffers: every frame uploads
    # its tables from pinned host memory inside curast_render, resolves, and
    # copies the RGBA8 image back into pinned host memory
    host_img = torch.empty((args.H, args.W, 4), dtype=torch.uint8, pin_memory=True)
    rgba8 = torch.empty((args.H, args.W, 4), dtype=torch.uint8, device=dev)
    for _ in range(2):
        r.render(cam.view, cam.proj, args.W, args.H, vis)
        r.L.curast_resolve(r._h, api._mat(cam.view), api._mat(cam.proj), args.W, args.H, api._ptr(vis), None,
                           api._ptr(rgba8), api._stream())
        host_img.copy_(rgba8, non_blocking=True)
    torch.cuda.synchronize()
    ranks.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r.render(cam.view, cam.proj, args.W, args.H, vis)
        r.L.curast_resolve(r._h, api._mat(cam.view), api._mat(cam.proj), args.W, args.H, api._ptr(vis), None,
                           api._ptr(rgba8), api._stream())
        host_img.copy_(rgba8, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_ms = ranks.max((time.perf_counter() - t0) * 1e3 / args.steps)
    h2d = 256 + 40 + info["segments"] * 32 + info["pairs"] * 64 + 12 * 4 * len(sc.instances)

    tris = info["triangles"]
    total_tris = ranks.sum(tris)
    gtris = total_tris / (ms_frame * 1e-3) / 1e9
    s1 = statistics.mean(s[1] for s in stage)       # the cull kernel: reads every index and position
    s1_bytes = 12.0 * (info["unique_triangles"] + info["unique_vertices"])
    peak, peak_kind = measured_peaks()
    achieved = s1_bytes / (s1 * 1e-3) / 1e9
    workload_key = f"billion{args.tiles}x{args.cells}@{args.W}x{args.H}" + (f"-subset{args.subset}" if args.subset else "")
    result = {
        "metric": "frame ms & Gtris/s at 3840x2160 (1B tris), %HBM roofline; batched vs plain",
        "value": round(gtris, 3),
        "unit": "Gtris/s",
        "n_gpus": ranks.world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_frame, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "fp32+int64",
        "data": "synthetic",
        "config": {
            "workload": f"billion-scale terrain: {args.tiles}x{args.tiles} seeded heightfield tiles of "
                        f"{args.cells}^2 cells ({2 * args.cells ** 2 * args.tiles ** 2} triangles), "
                        f"{args.W}x{args.H}, overview camera",
            "triangles_per_frame": tris,
            "visible_tiles": info["pairs"],
            "l2": f"inputs larger than L2 ({s1_bytes / 1e9:.1f} GB of indices+positions read per frame)",
            "parallelism": "replicas" if ranks.world > 1 else "single GPU",
            "generation_s": round(t_gen, 2),
        },
        "stage_ms": {k: round(statistics.mean(s[i] for s in stage), 4)
                     for i, k in enumerate(["clear", "stage1_cull", "stage1_exact", "stage2", "stage3"])},
        "roofline": {
            "bound": "hbm",
            "kernel": "k_stage1",
            "achieved": round(achieved, 1),
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": recorded_traffic(workload_key),
            "peak_kind": peak_kind,
            "bytes_per_launch": s1_bytes,
            "bytes_rule": "12 B per index triple + 12 B per vertex, each mesh read once per launch",
        },
        "e2e": {"value": round(total_tris / (e2e_ms * 1e-3) / 1e9, 3), "unit": "Gtris/s",
                "ms_per_step": round(e2e_ms, 4), "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": args.W * args.H * 4},
        # per frame: clear, a cull and an exact kernel per round, stage 2, and
        # stage 3 as scan + scatter + tile kernels
        "gpu_launches": (5 + 2 * info["rounds"]) * args.steps,
        "clocks": clk,
        "frame_stats": {k: v for k, v in stats.items() if v},
    }
    if ranks.rank == 0 and ranks.world == 1 and args.resolve:
        result["resolve"] = resolve_timing(r, cam, args, vis, stream)
        result["resolve_textured"] = resolve_textured_timing(r, sc, cam, args, vis, stream)
    if ranks.rank == 0 and ranks.world == 1 and args.supersampling:
        result["supersampling"] = supersampling(r, cam, args, ms_frame, stream)
    if ranks.rank == 0 and ranks.world == 1 and args.ablation:
        result["conservative_cull"] = conservative_cull_ablation(r, cam, args, ms_frame, vis, stream)
    r.close()
    if ranks.rank == 0 and ranks.world == 1 and args.compressed:
        result["compressed"] = compressed_frame(args, sc, cam, dev, stream, info, ms_frame)
    if ranks.rank == 0 and ranks.world == 1 and args.thirty and args.tiles == 8 and not args.subset:
        result["thirty_tiles"] = thirty_tiles_frame(args, sc, cam, dev, stream)
    del sc, vis
    torch.cuda.empty_cache()

    if ranks.rank == 0 and ranks.world == 1 and args.unique:
        result["unique_100m"] = unique_100m(args, dev)
    if ranks.rank == 0 and ranks.world == 1 and args.raycast:
        result["raycast_stage3"] = raycast_stage3(args, dev)
    if ranks.rank == 0 and ranks.world == 1 and args.diff:
        result["differentiable"] = differentiable_step(dev)
    if ranks.rank == 0 and ranks.world == 1 and args.batched != "off":
        result["batched_vs_plain"] = batched_vs_plain(args, dev)
    if ranks.rank == 0 and ranks.world == 1 and not args.no_cpu_baseline:
        g, n, dt = cpu_baseline_sample(args.tiles, args.cells, args.W, args.H, count=3)
        result["cpu_baseline"] = {"value": round(g, 5), "unit": "Gtris/s", "cores": 1, "kind": "oracle",
                                  "sample": f"three adjacent central tiles ({n} triangles) of the same frame, "
                                            f"single-threaded oracle, {dt:.1f} s"}
        result["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args)
    result["config"]["host_cores"] = os.cpu_count()
    return result


def tiles_wholly_in_view(cam, tiles: int, count: int = 30, height: float = 0.2):
    """The `count` tiles of the tiles x tiles layout (tile k spans x in [i, i+1],
    z in [j, j+1], y in [0, height]) whose 8 box corners all project in front
    of the camera and inside the viewport, nearest the layout's centre first."""
    import numpy as np
    V = np.asarray(cam.view, np.float64)
    P = np.asarray(cam.proj, np.float64)
    inside = []
    for k in range(tiles * tiles):
        i, j = k % tiles, k // tiles
        c = np.array([[i + a, y, j + b, 1.0] for a in (0, 1) for b in (0, 1) for y in (0.0, height)])
        h = (P @ V @ c.T).T
        w = h[:, 3]
        if (w > 0).all() and (np.abs(h[:, 0] / w) <= 1).all() and (np.abs(h[:, 1] / w) <= 1).all():
            inside.append(k)
    cx = cz = tiles / 2.0
    return sorted(inside, key=lambda k: (k % tiles + 0.5 - cx) ** 2 + (k // tiles + 0.5 - cz) ** 2)[:count]


def thirty_tiles_frame(args, sc, cam, dev, stream):
    """The same layout with only the 30 tiles wholly inside the view that lie
    nearest its centre (30 x 2 x 4096^2 = 1.007 B triangles, every one of them
    in the frustum): frame ms, Gtris/s, stage ms and the cull's roofline."""
    import torch
    from paper_2604_21749_gb300 import api
    keep = tiles_wholly_in_view(cam, args.tiles)
    r = api.Renderer(dev.index)
    for n, k in enumerate(keep):
        m = sc.meshes[k]
        r.upload_mesh(m.pos, m.idx, m.rgba8)
        r.add_instance(n, sc.instances[k].model)
    vis = r.new_vis(args.W, args.H)

    def frame():
        r.render(cam.view, cam.proj, args.W, args.H, vis)

    ms = _time_calls(frame, stream, 20)
    frame()
    st = r.stage_times()
    info = r.last_frame()
    r.close()
    del vis
    torch.cuda.empty_cache()
    byts = 12.0 * (info["unique_triangles"] + info["unique_vertices"])
    peak, kind = measured_peaks()
    return {"tiles": len(keep), "tiles_in_frustum": info["pairs"], "triangles": info["triangles"],
            "frame_ms": round(ms, 4), "gtris_s": round(info["triangles"] / (ms * 1e-3) / 1e9, 2),
            "stage_ms": {n: round(v, 4) for n, v in zip(["clear", "stage1_cull", "stage1_exact", "stage2", "stage3"], st)},
            "cull_gbs": round(byts / (st[1] * 1e-3) / 1e9, 1), "cull_frac": round(byts / (st[1] * 1e-3) / 1e9 / peak, 4),
            "frame_frac": round(byts / (ms * 1e-3) / 1e9 / peak, 4), "peak_kind": kind}


def compressed_frame(args, sc, cam, dev, stream, info_plain, ms_plain):
    """The same frame with every tile uploaded compressed (Section 4.6):
    frame and stage times, and the index + position bytes the cull reads."""
    import torch
    from paper_2604_21749_gb300 import api
    r = api.Renderer(dev.index)
    for m in sc.meshes:
        r.upload_mesh(m.pos, m.idx, m.rgba8, compressed=True)
    for it in sc.instances:
        r.add_instance(it.mesh, it.model)
    vis = r.new_vis(args.W, args.H)
    for _ in range(2):
        r.render(cam.view, cam.proj, args.W, args.H, vis)
    r.sync()
    frames = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stage = []
    e0.record(stream)
    for _ in range(frames):
        r.render(cam.view, cam.proj, args.W, args.H, vis)
        stage.append(r.stage_times())
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / frames
    info = r.last_frame()
    infos = [r.mesh_info(k) for k in range(len(sc.meshes))]
    bits = [mi["index_bits"] for mi in infos]
    # the cull reads the visible tiles' packed indices and quantized positions
    # (the tiles are the same size, one instance each)
    per_mesh = sum(mi["geometry_bytes"] for mi in infos) / max(len(infos), 1)
    read_bytes = per_mesh * info["pairs"]
    plain_bytes = 12.0 * (info_plain["unique_triangles"] + info_plain["unique_vertices"])
    cull_ms = statistics.mean(s[1] for s in stage)
    r.close()
    del vis
    torch.cuda.empty_cache()
    return {"frame_ms": round(ms, 4), "vs_uncompressed": round(ms_plain / ms, 3),
            "stage_ms": {k: round(statistics.mean(s[i] for s in stage), 4)
                         for i, k in enumerate(["clear", "stage1_cull", "stage1_exact", "stage2", "stage3"])},
            "index_bits": sorted(set(bits)), "geometry_bytes_read": round(read_bytes),
            "uncompressed_bytes_read": round(plain_bytes),
            "cull_gbs": round(read_bytes / (cull_ms * 1e-3) / 1e9, 1),
            "triangles_per_frame": info["triangles"]}


def _time_calls(fn, stream, reps):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def resolve_timing(r, cam, args, vis, stream):
    """The resolve of the frame (Section 4.4) on its own: FP32 RGBA and RGBA8
    out, ms per call, and its roofline.  Algorithmic bytes: the 8-byte word
    read and 16 + 4 bytes written per pixel, plus per covered pixel the
    triangle's 12 bytes of indices, 36 of positions and 12 of vertex colours
    gathered."""
    import torch
    from paper_2604_21749_gb300 import api
    H, W = vis.shape
    f32 = torch.empty((H, W, 4), dtype=torch.float32, device=vis.device)
    u8 = torch.empty((H, W, 4), dtype=torch.uint8, device=vis.device)
    vm, pm = api._mat(cam.view), api._mat(cam.proj)

    def call():
        api._check(r.L.curast_resolve(r._h, vm, pm, W, H, api._ptr(vis), api._ptr(f32), api._ptr(u8),
                                      api._stream()), "curast_resolve")

    ms = _time_calls(call, stream, 20)
    covered = int((vis != -1).sum().item())
    nbytes = W * H * (8 + 20) + covered * (12 + 36 + 12)
    peak, kind = measured_peaks()
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"ms": round(ms, 4), "pixels": W * H, "covered": covered,
            "roofline": {"bound": "hbm", "kernel": "k_resolve", "achieved": round(gbs, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(gbs / peak, 4), "peak_kind": kind,
                         "bytes_per_launch": nbytes,
                         "bytes_rule": "8 B read + 20 B written per pixel, 60 B gathered per covered pixel"}}


def resolve_textured_timing(r, sc, cam, args, vis, stream):
    """The textured resolve of the frame (Section 4.4, mip level from four
    pixel rays): every tile textured with one shared 4096^2 RGBA8 mip chain
    over its unit square (uv = the grid coordinates), ms per call and the
    histogram of the levels chosen."""
    import torch
    import synthetic as S
    H, W = vis.shape
    n = int(round(math.sqrt(sc.meshes[0].V))) - 1
    uv = S.grid_uv(n, device=vis.device)
    tex = S.texture_mip_chain(12, seed=9, device=vis.device)
    for k, m in enumerate(sc.meshes):
        if m.T > 0 and m.V == uv.shape[0]:
            r.set_mesh_texture(k, uv, tex, 12)
    f32 = torch.empty((H, W, 4), dtype=torch.float32, device=vis.device)
    u8 = torch.empty((H, W, 4), dtype=torch.uint8, device=vis.device)
    lev = torch.empty((H, W), dtype=torch.uint8, device=vis.device)
    from paper_2604_21749_gb300 import api
    vm, pm = api._mat(cam.view), api._mat(cam.proj)

    def call():
        api._check(r.L.curast_resolve_textured(r._h, vm, pm, W, H, api._ptr(vis), api._ptr(f32), api._ptr(u8),
                                               api._ptr(lev), api._stream()), "curast_resolve_textured")

    ms = _time_calls(call, stream, 20)
    hist = torch.bincount(lev.reshape(-1).to(torch.int64), minlength=256)
    levels = {str(k): int(hist[k]) for k in range(13) if hist[k] > 0}
    for k, m in enumerate(sc.meshes):
        r.set_mesh_texture(k, None, None)
    del uv, tex, f32, u8, lev
    torch.cuda.empty_cache()
    return {"ms": round(ms, 4), "texture": "4096^2 RGBA8 with its 13-level mip chain, uv = grid coordinates",
            "levels": levels}


def unique_100m(args, dev):
    """The 100M-triangle heightfield (7072^2 cells, one mesh): its 8 seeded
    poses, whole-mesh views to close-ups, at 1920x1080 and 3840x2160; per
    pose frame ms, Gtris/s and per-stage ms."""
    import torch
    import numpy as np
    import synthetic as S
    from paper_2604_21749_gb300 import api
    t0 = time.perf_counter()
    sc = S.scene_unique(device=dev)
    torch.cuda.synchronize()
    tgen = time.perf_counter() - t0
    m = sc.meshes[0]
    r = api.Renderer(dev.index)
    r.upload_mesh(m.pos, m.idx, m.rgba8)
    r.add_instance(0, np.eye(4, dtype=np.float32))
    stream = torch.cuda.current_stream()
    poses = []
    for W, H in ((1920, 1080), (3840, 2160)):
        vis = r.new_vis(W, H)
        for k in range(8):
            cam = S.camera_unique_pose(k, W, H)
            st = []

            def frame():
                r.render(cam.view, cam.proj, W, H, vis)

            ms = _time_calls(frame, stream, 10)
            frame()
            st = r.stage_times()
            info = r.last_frame()
            poses.append({"pose": k, "W": W, "H": H, "frame_ms": round(ms, 4),
                          "gtris_s": round(info["triangles"] / (ms * 1e-3) / 1e9, 2),
                          "stage_ms": {n: round(v, 4) for n, v in
                                       zip(["clear", "stage1_cull", "stage1_exact", "stage2", "stage3"], st)}})
        del vis
    r.set_config(collect_stats=1)
    cam = S.camera_unique_pose(7, 3840, 2160)
    r.render(cam.view, cam.proj, 3840, 2160)
    stats = r.sync()
    r.close()
    del sc, m
    torch.cuda.empty_cache()
    return {"workload": f"100M unique: heightfield of 7072^2 cells ({2 * 7072 ** 2} triangles), 8 poses",
            "generation_s": round(tgen, 2), "poses": poses,
            "pose7_3840x2160_stats": {k: v for k, v in stats.items() if v}}


def conservative_cull_ablation(r, cam, args, ms_on, vis, stream):
    """The paper's Table 4 on this frame: the same frame with the conservative
    tiny-triangle cull off (stage1_exact_all), so that every (triangle, pair)
    takes the exact path, which drops tiny and off-screen triangles itself.
    The buffer is the same; frame ms and stage ms of that frame."""
    import torch
    r.set_config(stage1_exact_all=1)
    r.render(cam.view, cam.proj, args.W, args.H, vis)
    r.sync()
    frames = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(frames):
        r.render(cam.view, cam.proj, args.W, args.H, vis)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_off = e0.elapsed_time(e1) / frames
    r.render(cam.view, cam.proj, args.W, args.H, vis)
    st = r.stage_times()
    r.set_config(stage1_exact_all=0)
    return {"frame_ms_without": round(ms_off, 3), "frame_ms_with": round(ms_on, 3),
            "speedup": round(ms_off / ms_on, 2),
            "stage_ms_without": {k: round(v, 3) for k, v in
                                 zip(["clear", "stage1_cull", "stage1_exact", "stage2", "stage3"], st)}}


def supersampling(r, cam, args, ms_1x1, stream):
    """Anti-aliasing by super sampling (the paper's Table 5 on this frame):
    the same view rendered at 2x2 and 4x4 samples per pixel, then the
    box-filtered resolve to the output size; frame ms of each (render only)
    and of the resolve."""
    import torch
    out = {"1x1_ms": round(ms_1x1, 3)}
    for ss in (2, 4):
        W, H = ss * args.W, ss * args.H
        vis = r.new_vis(W, H)
        r.render(cam.view, cam.proj, W, H, vis)
        r.sync()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        frames = 3
        e0.record(stream)
        for _ in range(frames):
            r.render(cam.view, cam.proj, W, H, vis)
        e1.record(stream)
        r.resolve_ss(cam.view, cam.proj, vis, ss, want_f32=False)
        e2.record(stream)
        torch.cuda.synchronize()
        out[f"{ss}x{ss}_ms"] = round(e0.elapsed_time(e1) / frames, 3)
        out[f"{ss}x{ss}_resolve_ms"] = round(e1.elapsed_time(e2), 3)
        del vis
        torch.cuda.empty_cache()
    return out


def differentiable_step(dev):
    """The differentiable workload (1448^2-cell heightfield, 1024^2, FP32 RGB
    per-vertex colours): with the visibility buffer fixed, the interpolation
    forward (image from colours) and backward (colour and position gradients
    from an image gradient) through the public API, ms per call."""
    import torch
    import synthetic as S
    from paper_2604_21749_gb300 import api
    sc, col = S.scene_differentiable(device=dev)
    m, cam = sc.meshes[0], sc.cameras[0]
    r = api.Renderer(dev.index)
    r.upload_mesh(m.pos, m.idx, m.rgba8)
    r.add_instance(0, sc.instances[0].model)
    vis = r.render(cam.view, cam.proj, cam.W, cam.H)
    col = col.to(dev).contiguous()
    g = torch.randn((cam.H, cam.W, 3), generator=torch.Generator(device=dev).manual_seed(7), device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": f"differentiable: {m.T} triangles, {cam.W}x{cam.H}, RGB FP32 per-vertex colours"}
    for name, fn in (("forward", lambda: r.interpolate(0, cam.view, cam.proj, vis, col, pos=m.pos)),
                     ("backward", lambda: r.interpolate_backward(0, cam.view, cam.proj, vis, col, g, pos=m.pos))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[name + "_ms"] = round(ms, 4)
        out[name + "_mpix_s"] = round(cam.W * cam.H / (ms * 1e-3) / 1e6, 1)
    r.close()
    del vis, g
    torch.cuda.empty_cache()
    return out


def raycast_stage3(args, dev):
    """Stage-3 workloads rendered with the default fixed-point rule and with
    the paper's ray-cast stage 3 (stage3_raycast): the camera inside a closed
    box at the frame size (every face huge and crossing the near plane), and
    a close-up pose of a 1448^2 heightfield with stage2_max_pixels = 32 so
    that its large triangles are ray cast.  Each with every covered pixel
    written to the global buffer (the default) and with the shared-memory
    tile buffer of stage 3 (stage3_tile_buffer = 1, keys *_tile_buffer).
    Frame ms and per-stage ms of each."""
    import numpy as np
    import torch
    import synthetic as S
    from paper_2604_21749_gb300 import api
    cases = []
    room = S.scene_room(device=dev, W=args.W, H=args.H)
    cases.append((f"room: 12 triangles around the camera, {args.W}x{args.H}", room, room.cameras[0], {}))
    hf = S.heightfield_mesh(1448, seed=100, device=dev)
    close = S.Scene([hf], [S.Instance(0, np.eye(4, dtype=np.float32))], [])
    cases.append((f"close-up pose 3 of a 1448^2 heightfield, {args.W}x{args.H}, stage2_max_pixels 32", close,
                  S.camera_unique_pose(3, args.W, args.H), {"stage2_max_pixels": 32}))
    stream = torch.cuda.current_stream()
    out = []
    for name, sc, cam, cfg in cases:
        r = api.Renderer(dev.index)
        for m in sc.meshes:
            r.upload_mesh(m.pos, m.idx, m.rgba8)
        for it in sc.instances:
            r.add_instance(it.mesh, it.model)
        vis = r.new_vis(cam.W, cam.H)
        row = {"workload": name}
        for mode, tb in ((0, 0), (1, 0), (0, 1), (1, 1)):
            r.set_config(stage3_raycast=mode, stage3_tile_buffer=tb, **cfg)
            for _ in range(3):
                r.render(cam.view, cam.proj, cam.W, cam.H, vis)
            r.sync()
            frames = 20
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(frames):
                r.render(cam.view, cam.proj, cam.W, cam.H, vis)
            e1.record(stream)
            torch.cuda.synchronize()
            r.render(cam.view, cam.proj, cam.W, cam.H, vis)
            st = r.stage_times()
            key = ("ray_cast" if mode else "fixed_point") + ("_tile_buffer" if tb else "")
            row[key + "_ms"] = round(e0.elapsed_time(e1) / frames, 4)
            row[key + "_stage_ms"] = {k: round(v, 4) for k, v in
                                      zip(["clear", "stage1_cull", "stage1_exact", "stage2", "stage3"], st)}
        r.close()
        out.append(row)
        del vis
    torch.cuda.empty_cache()
    return out


def batched_vs_plain(args, dev):
    """The batched form (one persistent launch over all meshes, instances and
    views, replayed from a CUDA graph) against one launch sequence per mesh
    per view, on the many-mesh workload; the buffers must be identical."""
    import torch
    import synthetic as S
    from paper_2604_21749_gb300 import api
    if args.batched == "full":
        kw = dict(n_meshes=256, n_instances=10000, tmin=1e4, tmax=2e7)
        name = "256 meshes (T log-uniform in [1e4, 2e7]), 10000 instances, 2x 3840x2160 + 2x 1920x1080"
    else:
        kw = dict(n_meshes=32, n_instances=400, tmin=1e3, tmax=2e5)
        name = "32 meshes (T log-uniform in [1e3, 2e5]), 400 instances, 2x 3840x2160 + 2x 1920x1080"
    t0 = time.perf_counter()
    sc = S.scene_batched(device=dev, **kw)
    torch.cuda.synchronize()
    tgen = time.perf_counter() - t0
    r = api.Renderer(dev.index)
    for m in sc.meshes:
        r.upload_mesh(m.pos, m.idx, m.rgba8)
    for it in sc.instances:
        r.add_instance(it.mesh, it.model)
    views = [(c.view, c.proj, c.W, c.H, r.new_vis(c.W, c.H)) for c in sc.cameras]
    plain_out = [r.new_vis(c.W, c.H) for c in sc.cameras]
    stream = torch.cuda.current_stream()
    # the workload's configuration is autotuned (its result is kept only if
    # the buffers stay identical); both paths then run with it
    t0 = time.perf_counter()
    tuned = r.autotune(views)
    torch.cuda.synchronize()
    ttune = time.perf_counter() - t0

    def batched():
        r.render_batch(views, use_graph=True)

    def plain():
        for c, vis in zip(sc.cameras, plain_out):
            r.clear(vis)
            for m in range(len(sc.meshes)):
                r.render_mesh(m, c.view, c.proj, c.W, c.H, vis)

    def timeit(fn, reps=2):
        fn()
        r.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    tb = timeit(batched)
    info = r.last_frame()
    tp = timeit(plain)
    same = all(torch.equal(v[4], p) for v, p in zip(views, plain_out))
    r.sync()
    # one more batched frame outside the graph for per-stage times, one with counters
    r.render_batch(views, use_graph=False)
    st = r.stage_times()
    r.set_config(collect_stats=1)
    r.render_batch(views, use_graph=False)
    stats = r.sync()
    r.set_config(collect_stats=0)
    out = {"workload": name, "batched_ms": round(tb, 3), "plain_ms": round(tp, 3),
           "speedup": round(tp / tb, 3), "identical": bool(same), "pairs": info["pairs"],
           "rounds": info["rounds"], "triangle_instance_views": info["triangles"],
           "batched_gtris_s": round(info["triangles"] / (tb * 1e-3) / 1e9, 2),
           "batched_stage_ms": {k: round(v, 3) for k, v in
                                zip(["clear", "stage1_cull", "stage1_exact", "stage2", "stage3"], st)},
           "batched_stats": {k: v for k, v in stats.items() if v}, "generation_s": round(tgen, 1),
           "autotuned": {k: tuned[k] for k in ("stage1_tri_per_thread", "stage1_max_pixels", "stage2_max_pixels",
                                               "tile_log2", "pairs_per_segment", "stage1_group_min_pairs")},
           "autotune_s": round(ttune, 1)}
    r.close()
    del sc, views, plain_out
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------ reference arm ------
def run_reference(args, ranks: Ranks):
    """The oracle as it stands, on the host cores: each step renders a
    bounded sample (1/16 of one tile) of the same frame."""
    frac = 1.0 / 16.0
    for _ in range(args.warmup):
        cpu_baseline_sample(args.tiles, args.cells, args.W, args.H, frac)
    vals, secs, n = [], [], 0
    for _ in range(args.steps):
        g, n, dt = cpu_baseline_sample(args.tiles, args.cells, args.W, args.H, frac)
        vals.append(g)
        secs.append(dt)
    v = statistics.mean(vals)
    total = 2 * args.cells ** 2 * args.tiles ** 2
    return {
        "impl": "reference",
        "metric": "frame ms & Gtris/s at 3840x2160 (1B tris), %HBM roofline; batched vs plain",
        "value": round(v, 6), "unit": "Gtris/s", "n_gpus": ranks.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(secs), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "fp32+int64", "data": "synthetic",
        "config": {"workload": f"billion-scale terrain: {args.tiles}x{args.tiles} seeded heightfield tiles of "
                               f"{args.cells}^2 cells ({total} triangles), {args.W}x{args.H}, overview camera"},
        "cpu_baseline": {"value": round(v, 6), "unit": "Gtris/s", "cores": 1, "kind": "oracle",
                         "sample": f"{n} triangles (1/16 of one central tile) per step, single-threaded oracle"},
        "e2e": {"value": round(v, 6), "unit": "Gtris/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse_args()
    if args.impl == "reference":
        # the oracle runs on rank 0's host cores only; other ranks exit at once
        if int(os.environ.get("RANK", "0")) == 0:
            os.environ["WORLD_SIZE"] = "1"
            print(json.dumps(run_reference(args, Ranks(1))), flush=True)
        return
    ranks = Ranks(args.gpus)
    try:
        res = run_ours(args, ranks)
        if ranks.rank == 0:
            print(json.dumps(res), flush=True)
    finally:
        ranks.close()


if __name__ == "__main__":
    main()
