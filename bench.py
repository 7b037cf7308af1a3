"""Benchmark of the path tracer's hot path on one node.

A step is one progressive frame of the whole hot path -- camera rays, closest hit through
the compressed wide BVH, material sort, OpenPBR shading with next-event estimation and
Russian roulette, shadow rays, Kahan accumulation -- for the synthetic CAD pushbutton
(~210k triangles, analytic-sky environment + one quad light) at 1920x1080, one sample per
pixel, max depth 8.  The BVH is built once before the timed region (its build time is
reported as `bvh_build_ms`).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The metric is traced rays per second (camera + BSDF-sampled extension rays + shadow rays);
spp/s at 1080p is reported beside it.  With --impl reference the CPU oracle renders bounded
samples of the same frame on the host cores (the comparison arm of this benchmark).
Multi-GPU runs are independent replicas (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "pushbutton": "synthetic CAD pushbutton, 209,600 triangles + 2 light triangles, 1920x1080, 1 spp/step, "
                  "max depth 8, analytic sky 512x256 + 1 quad light",
    "heavy": "16 displaced level-7 icospheres, 5,242,882 triangles, 1920x1080, 1 spp/step, max depth 12, "
             "analytic sky 512x256",
    "cornell512": "Cornell-style box, 36 triangles, one quad light, 512x512, 1 spp/step, max depth 8",
    "cornell1080": "Cornell-style box, 36 triangles, one quad light, 1920x1080, 1 spp/step, max depth 8",
    "pushbutton_dof": "the pushbutton frame through a thin lens (radius 0.03, focus on the button), "
                      "1920x1080, 1 spp/step, max depth 8",
    "many_lights": "Cornell-style box lit by 248 small non-overlapping quad lights (heavy-tailed radiance, random "
                   "tints) on the ceiling and side walls, 1920x1080, 1 spp/step, max depth 4",
    "pushbutton_fuzz": "the pushbutton frame with the button's red coated plastic under a fuzz layer (velvet), "
                       "1920x1080, 1 spp/step, max depth 8",
}
NODE_BYTES = 80      # compressed 8-wide BVH node
TRI_BYTES = 48       # triangle record
RAY_BYTES = 32       # ray in (origin + direction float4 pair)
HIT_BYTES = 16       # hit record out
# algorithmic FP32 operations of the traversal: one child box test = 6 decode FMA + 6 sub +
# 6 mul + 12 min/max + 1 compare ~ 30, counted for each filled child slot of a visited node
# (the counting traversal reports those box tests); one watertight triangle test ~ 50 (9 sub,
# 12 shear, 9 edge products/differences, sign tests, det, T, divide, range)
OPS_PER_BOX = 30
OPS_PER_TRI = 50
# FP32 lane peak: SMs (read from the device) x 128 FP32 lanes x the maximum SM clock (an FMA
# counted as one operation); 2.07 GHz is the GB300's maximum SM clock, MEASURED_PEAKS.json's
# sm_max_mhz when present
FP32_LANES_PER_SM, SM_MAX_GHZ = 128, 2.07


def alu_peak_gops(sm_count: int, sm_max_ghz: float = SM_MAX_GHZ) -> float:
    return sm_count * FP32_LANES_PER_SM * sm_max_ghz


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pushbutton", choices=sorted(WORKLOADS))
    ap.add_argument("--tune", type=int, default=1,
                    help="run pt_autotune (untimed) before the timed region and render in PT_MODE_AUTO")
    ap.add_argument("--graph", type=int, default=1, help="replay each frame's wavefront launches as a CUDA graph")
    ap.add_argument("--mode", default="wavefront", choices=["auto", "wavefront", "megakernel"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--bvh-builder", default="ploc", choices=["ploc", "lbvh"],
                    help="binary tree the wide BVH is collapsed from: clustering (default) or radix tree")
    ap.add_argument("--bvh-collapse", default="optimal", choices=["optimal", "greedy"],
                    help="folding of the binary tree into wide nodes: least surface-area cost or largest child first")
    ap.add_argument("--bvh-tri-cost", type=float, default=0.0,
                    help="cost of a triangle test against a wide node visit for the optimal collapse (0: default)")
    ap.add_argument("--bvh-box-cost", type=float, default=0.0,
                    help="cost of each child slot of a visited wide node for the optimal collapse (0: default)")
    ap.add_argument("--bvh-width", type=int, default=8, choices=range(2, 9),
                    help="most children per BVH node (the node format holds 8)")
    ap.add_argument("--spp-per-step", type=int, default=4,
                    help="samples per pixel of the frame one step renders (progressive: each step adds them)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="target CPU work of the oracle sample")
    ap.add_argument("--study-frames", type=int, default=256, help="frames per curve of the NRC study")
    ap.add_argument("--batch-scenes", type=int, default=64)
    ap.add_argument("--no-bvh-tune", action="store_true",
                    help="batch study: keep the scenes' 8-wide trees (no BVH width in pt_autotune_batch)")
    ap.add_argument("--study", default=None, choices=[None, "nrc", "nrc_train", "batch", "paper", "restir", "bmfr"],
                    help="nrc: relMSE vs time, radiance cache against the plain tracer; nrc_train: the "
                         "radiance-cache training and inference kernels alone")
    ap.add_argument("--ref-spp", type=int, default=4096)
    ap.add_argument("--max-depth", type=int, default=None, help="studies: override the workload's max depth")
    ap.add_argument("--nrc-batch", type=int, default=8192, help="NRC study: training samples per Adam step")
    ap.add_argument("--nrc-frame-samples", type=int, default=32768, help="NRC study: training samples per frame")
    return ap.parse_args()


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def combine_replicas(dev_ms: float, rays: float, device=None):
    """Whole-job figures of N independent replicas (one per GPU, each rendering its own frames
    with its own seed): the slowest rank's timed milliseconds and the rays of all ranks.
    Without an initialised process group (or with one rank) the local figures are returned."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return dev_ms, rays
    t = torch.tensor([dev_ms], dtype=torch.float64, device=device)
    r = torch.tensor([rays], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(r, op=dist.ReduceOp.SUM)
    return float(t.item()), float(r.item())


def _metric_name(workload: str) -> str:
    """The headline metric is quoted on the pushbutton frame; other workloads name themselves."""
    return "Mrays/s at 1080p (pushbutton)" if workload == "pushbutton" else f"Mrays/s ({workload})"


def _source_hash():
    """Hash of the traversal kernels' and the BVH builder's code with comments and blank lines
    removed (a comment edit does not change what a recorded ncu capture measured)."""
    h = hashlib.sha256()
    for rel in ("paper_2407_19977_gb300/csrc/pt_device.cuh", "paper_2407_19977_gb300/csrc/pt_render.cu",
                "paper_2407_19977_gb300/csrc/pt_bvh.cu"):
        with open(os.path.join(ROOT, rel)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(line.rstrip() for line in src.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


def _recorded_profile(kernel: str, workload: str, spp_per_step: int):
    """The committed ncu record of `kernel` (`profiles/<kernel>_traffic.txt`) as a dict, if it
    was taken on the current kernel source (the record holds the source hash) and on this
    launch shape (the workload and the samples per step, which set the wave size); else None."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_traffic.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_hash") != _source_hash():
        return None
    if vals.get("workload") != workload or vals.get("spp_per_step") != str(spp_per_step):
        return None
    return vals


def _recorded_traffic(kernel: str, workload: str, spp_per_step: int, launches_per_step: int):
    """DRAM bytes per launch of `kernel` from its committed ncu record (see _recorded_profile):
    the bytes of all its launches in a step, over the launches this run issues per step (the
    autotuned tail bounce decides how many of the bounces' launches a step issues; the ones it
    leaves out moved no data)."""
    vals = _recorded_profile(kernel, workload, spp_per_step)
    try:
        return float(vals["dram_bytes_per_step"]) / max(launches_per_step, 1) if vals else None
    except (KeyError, ValueError):
        return None


def _recorded_issue(kernel: str, workload: str, spp_per_step: int):
    """Instruction issue of `kernel` from the full ncu capture named in its record: the share of
    issue slots used and the active lanes per warp instruction (None when the record does not
    match the current source)."""
    vals = _recorded_profile(kernel, workload, spp_per_step)
    try:
        return {"issue_slots_busy": float(vals["issue_slots_busy_pct"]) / 100.0,
                "active_lanes_per_warp_instruction": float(vals["active_threads_per_inst"]),
                "lane_fraction": float(vals["active_threads_per_inst"]) / 32.0,
                "source": vals.get("issue_source", "ncu")} if vals else None
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """SM clock and clock-event (throttle) reasons sampled while running: NVML read through
    ctypes every 2 ms (a 20-frame timed region lasts about 70 ms), else nvidia-smi every 50 ms.
    Only reads; changes no setting."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, gpu_index: int, period_s: float = 0.002):
        self.gpu = gpu_index
        self.period = period_s
        self.proc = None
        self.file = None
        self.nvml = None
        self.rows = []
        self.thread = None
        self.stop = None
        self.source = None

    def _nvml_open(self):
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = C.c_void_p()
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(self.gpu)
            bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        except Exception:
            bus = None
        ok = bus is not None and lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), C.byref(h)) == 0
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(self.gpu), C.byref(h)) != 0:
            return None
        mx = C.c_uint()
        lib.nvmlDeviceGetMaxClockInfo(h, C.c_int(1), C.byref(mx))
        self.max_mhz = float(mx.value)
        return lib, h

    def _nvml_loop(self):
        import ctypes as C
        lib, h = self.nvml
        mhz, reasons = C.c_uint(), C.c_ulonglong()
        get_reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        while not self.stop.is_set():
            if lib.nvmlDeviceGetClockInfo(h, C.c_int(1), C.byref(mhz)) == 0 and \
                    get_reasons(h, C.byref(reasons)) == 0:
                self.rows.append((float(mhz.value), int(reasons.value)))
            self.stop.wait(self.period)

    def __enter__(self):
        import threading
        try:
            self.nvml = self._nvml_open()
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self.source = f"NVML every {self.period * 1e3:.0f} ms"
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._nvml_loop, daemon=True)
            self.thread.start()
            return self
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
            self.source = "nvidia-smi every 50 ms"
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.thread is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.nvml is not None:
            if not self.rows:
                return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"], "source": self.source}
            reasons = sorted({name for _, r in self.rows for bit, name in self.REASONS.items() if r & bit})
            return {"sm_mhz": statistics.median(m for m, _ in self.rows), "sm_max_mhz": self.max_mhz,
                    "sm_mhz_min": min(m for m, _ in self.rows), "reasons": reasons, "samples": len(self.rows),
                    "source": self.source}
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mhz = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "source": self.source}


def _make_workload(name):
    from paper_2407_19977_gb300 import scenes
    if name == "pushbutton":
        return scenes.pushbutton()
    if name == "heavy":
        return scenes.heavy_scene(level=7)
    if name == "cornell512":
        return scenes.cornell_box(width=512, height=512, spp=1, max_depth=8)
    if name == "cornell1080":
        return scenes.cornell_box(width=1920, height=1080, spp=1, max_depth=8)
    if name == "many_lights":
        return scenes.many_light_box(256, width=1920, height=1080, spp=1, max_depth=4, seed=0)
    if name == "pushbutton_fuzz":
        return scenes.pushbutton_fuzz()
    if name == "pushbutton_dof":
        sc = scenes.pushbutton()
        c = sc.camera
        focus = math.dist(c.target, c.origin)
        sc.camera = type(c)(**{**c.__dict__, "lens_radius": 0.03, "focus_distance": focus})
        return sc
    raise ValueError(name)


def cpu_baseline(sc, target_s: float, seed: int = 0):
    """The oracle as it stands, on all host cores, over a bounded sample of the frame:
    every `row_step`-th row at one sample per pixel, sized to about `target_s` seconds."""
    import oracle
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    osc = oracle.OracleScene(sc)
    setup = time.perf_counter() - t0
    # calibration on every 64th row (warms the threads and caches), then on every 16th, and
    # the sample scaled from the second to the target time
    osc.render(spp=1, seed=seed, row_step=64, threads=threads)
    t0 = time.perf_counter()
    _, _, st = osc.render(spp=1, seed=seed, row_step=16, threads=threads)
    cal = max(time.perf_counter() - t0, 1e-3)
    rows_cal = len(range(0, sc.camera.height, 16))
    rows = max(1, min(sc.camera.height, int(rows_cal * target_s / cal)))
    row_step = max(1, sc.camera.height // rows)
    spp = 1
    if row_step == 1:
        spp = max(1, int(round(target_s / (cal * sc.camera.height / rows_cal))))
    t0 = time.perf_counter()
    _, _, st = osc.render(spp=spp, seed=seed, s0=1000, row_step=row_step, threads=threads)
    dt = time.perf_counter() - t0
    rays = st["ext_rays"] + st["shadow_rays"]
    px = st["paths"] / spp
    # the same oracle on one core, over a sixteenth of the rows of that sample
    t1 = time.perf_counter()
    _, _, st1 = osc.render(spp=spp, seed=seed, s0=1000, row_step=row_step * 16, threads=1)
    dt1 = time.perf_counter() - t1
    one_core = (st1["ext_rays"] + st1["shadow_rays"]) / max(dt1, 1e-9) / 1e6
    return {
        "value_1core": one_core,
        "value": rays / dt / 1e6, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
        "sample": f"every {row_step}th row of the {sc.camera.width}x{sc.camera.height} frame ({int(px)} pixels) "
                  f"at {spp} spp, "
                  f"{rays} rays in {dt:.2f} s; oracle BVH setup {setup:.2f} s",
        "spp_per_s_1080p": st["paths"] / dt / (sc.camera.width * sc.camera.height),
    }


def run_reference(args, world, rank):
    """--impl reference: the CPU oracle on this host, same workload, metric and unit."""
    if rank != 0:
        return
    sc = _make_workload(args.workload)
    import oracle
    threads = os.cpu_count() or 1
    osc = oracle.OracleScene(sc)
    # each step renders a bounded slice of the frame at 1 spp: every row_step-th row, with
    # at least 16 rows per host thread so that the oracle's round-robin rows keep every
    # thread busy (the same loading as the cpu_baseline leg)
    row_step = max(1, sc.camera.height // (16 * threads))
    for w in range(args.warmup):
        osc.render(spp=1, seed=0, s0=w, row_step=row_step, threads=threads)
    t0 = time.perf_counter()
    rays = paths = 0
    for k in range(args.steps):
        _, _, st = osc.render(spp=1, seed=0, s0=100 + k, row_step=row_step, threads=threads)
        rays += st["ext_rays"] + st["shadow_rays"]
        paths += st["paths"]
    dt = time.perf_counter() - t0
    value = rays / dt / 1e6
    out = {
        "metric": _metric_name(args.workload), "value": value, "unit": "Mrays/s", "impl": "reference",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload].replace("1 spp/step", f"{args.spp_per_step} spp/step"),
                   "spp_per_step": args.spp_per_step,
                   "sample": f"every {row_step}th row at 1 spp per step (a bounded slice of each step's rays)"},
        "spp_per_s_1080p": paths / dt / (sc.camera.width * sc.camera.height),
        "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": threads, "kind": "oracle",
                         "sample": f"every {row_step}th row of the {sc.camera.width}x{sc.camera.height} frame "
                                   f"({len(range(0, sc.camera.height, row_step))} rows) at 1 spp per step, "
                                   f"{args.steps} steps"},
        "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist

    from paper_2407_19977_gb300 import api
    from paper_2407_19977_gb300 import native as N

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    sc = _make_workload(args.workload)
    cam = sc.camera
    W, H = cam.width, cam.height
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    scene = api.Scene(sc, build=False)
    torch.cuda.synchronize()
    upload_ms = (time.perf_counter() - t0) * 1e3
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bvh = {"builder": {"ploc": N.PT_BVH_PLOC, "lbvh": N.PT_BVH_LBVH}[args.bvh_builder],
           "collapse": {"optimal": N.PT_COLLAPSE_OPTIMAL, "greedy": N.PT_COLLAPSE_GREEDY}[args.bvh_collapse],
           "tri_cost": args.bvh_tri_cost, "box_cost": args.bvh_box_cost, "max_width": args.bvh_width}
    scene.build(**bvh)                      # first build: allocations and module load
    torch.cuda.synchronize()
    ev0.record(stream)
    scene.build(**bvh)
    ev1.record(stream)
    torch.cuda.synchronize()
    bvh_ms = ev0.elapsed_time(ev1)
    mode = {"auto": N.PT_MODE_AUTO, "wavefront": N.PT_MODE_WAVEFRONT, "megakernel": N.PT_MODE_MEGAKERNEL}[args.mode]
    tuned = None
    if args.tune:
        # untimed: the schedule (wavefront/megakernel, tail limit, sort, wave size) that renders
        # this frame fastest; PT_MODE_AUTO then uses it
        tuned, tuned_ms = scene.autotune(spp=args.spp_per_step, frames=2)
        mode = N.PT_MODE_AUTO
    acc = api.Accum(W, H)
    seed = 1000 * rank
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    for _ in range(args.warmup):
        scene.render(args.spp_per_step, seed=seed, accum=acc, mode=mode, use_graph=args.graph)
    torch.cuda.synchronize()
    # untimed instrumented frame at the first timed sample index: node visits and triangle
    # tests per ray give the traversal's algorithmic bytes
    s_first = acc.spp_done
    probe = api.Accum(W, H)
    probe.c.spp_done = s_first
    before = scene.stats()
    scene.render(args.spp_per_step, seed=seed, accum=probe, mode=mode, flags=N.PT_FLAG_COUNT)
    after = scene.stats()
    cnt = {k: after[k] - before[k] for k in ("ext_rays", "shadow_rays", "trace_nodes", "trace_tris",
                                             "trace_boxes", "shadow_nodes", "shadow_tris", "tail_ext_rays")}
    # rays the per-bounce closest-hit kernel traced (the tail kernel counts its own)
    cnt["trace_rays"] = cnt["ext_rays"] - cnt["tail_ext_rays"]
    trace_bytes_step = (cnt["trace_nodes"] * NODE_BYTES + cnt["trace_tris"] * TRI_BYTES +
                        cnt["trace_rays"] * (RAY_BYTES + HIT_BYTES))
    trace_ops_step = cnt["trace_boxes"] * OPS_PER_BOX + cnt["trace_tris"] * OPS_PER_TRI
    # timed region
    kernel_ms = (N.f32 * len(N.KERNEL_KINDS))()
    kernel_launches = (N.u32 * len(N.KERNEL_KINDS))()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    st_before = scene.stats()
    launches_before = api.launch_count()
    with ClockSampler(local) as clocks:
        # NVTX range "timed": profilers can select exactly these frames (ncu --nvtx
        # --nvtx-include "timed/")
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            flush.fill_(float(k))  # L2 flush between steps, outside the timed events
            starts[k].record(stream)
            scene.render(args.spp_per_step, seed=seed, accum=acc, mode=mode, use_graph=args.graph)
            ends[k].record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    launches = api.launch_count() - launches_before
    st_after = scene.stats()
    # per-kernel split: the same frames again with a CUDA-event pair around every launch on
    # the render stream (the event bookkeeping costs a little host time, so these frames
    # are kept out of the headline timing)
    for k in range(args.steps):
        flush.fill_(float(k))
        scene.render(args.spp_per_step, seed=seed, accum=acc, mode=mode, kernel_ms=kernel_ms, kernel_launches=kernel_launches)
    torch.cuda.synchronize()
    dev_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    rays = (st_after["ext_rays"] - st_before["ext_rays"]) + (st_after["shadow_rays"] - st_before["shadow_rays"])
    t_max, rays_all = combine_replicas(dev_ms, float(rays), dev if world > 1 else None)
    value = rays_all / (t_max * 1e-3) / 1e6
    spp_s = world * args.steps * args.spp_per_step / (t_max * 1e-3)
    # end to end through the public API: the step's inputs cross host->device (the camera and
    # seed, marshalled into the launch) and every frame estimate comes back to pinned host
    # memory.  Double-buffered: the frame is snapshotted on the device, then copied to the host
    # on a copy stream while the next frame renders; the host waits for frame k's image before
    # reusing its buffer at frame k + 2, and for the last two at the end.
    host_img = [torch.empty((H, W, 3), dtype=torch.float32, pin_memory=True) for _ in range(2)]
    stage = [torch.empty_like(acc.sum) for _ in range(2)]
    copy_stream = torch.cuda.Stream()
    compute = torch.cuda.current_stream()
    done = [None, None]
    e2e_steps = max(3, args.steps // 2)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e_before = scene.stats()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        b = k % 2
        if done[b] is not None:
            done[b].synchronize()                 # frame k - 2 is on the host
            compute.wait_event(done[b])
        cam_k = type(cam)(**cam.__dict__)
        scene.render(args.spp_per_step, seed=seed, accum=acc, mode=mode, camera=cam_k, use_graph=args.graph)
        stage[b].copy_(acc.sum)
        ready = torch.cuda.Event()
        ready.record(compute)
        copy_stream.wait_event(ready)
        with torch.cuda.stream(copy_stream):
            host_img[b].copy_(stage[b], non_blocking=True)
            done[b] = torch.cuda.Event()
            done[b].record(copy_stream)
    for d in done:
        if d is not None:
            d.synchronize()
    e2e_s = time.perf_counter() - t0
    e_after = scene.stats()
    e2e_rays = (e_after["ext_rays"] - e_before["ext_rays"]) + (e_after["shadow_rays"] - e_before["shadow_rays"])
    e2e_val = e2e_rays / e2e_s / 1e6 * world
    # roofline of the dominant kernel (closest-hit traversal)
    kms = {n: float(kernel_ms[i]) / args.steps for i, n in enumerate(N.KERNEL_KINDS)}
    kl = {n: int(kernel_launches[i]) // args.steps for i, n in enumerate(N.KERNEL_KINDS)}
    peaks, peak_src = _peaks()
    trace_ms = kms["trace"]
    achieved_gbs = trace_bytes_step / (trace_ms * 1e-3) / 1e9 if trace_ms > 0 else None
    achieved_gops = trace_ops_step / (trace_ms * 1e-3) / 1e9 if trace_ms > 0 else None
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_ghz = float(_peaks()[0].get("sm_max_mhz", SM_MAX_GHZ * 1e3)) / 1e3
    alu_peak = alu_peak_gops(sm_count, sm_ghz)
    trace_launches = max(kl["trace"], 1)
    traffic = _recorded_traffic("trace", args.workload, args.spp_per_step, trace_launches)
    result = {
        "metric": _metric_name(args.workload),
        "value": value, "unit": "Mrays/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload].replace("1 spp/step", f"{args.spp_per_step} spp/step"),
                   "spp_per_step": args.spp_per_step, "bvh_builder": args.bvh_builder, "bvh_width": args.bvh_width,
                   "bvh_collapse": args.bvh_collapse + (f" (tri_cost {args.bvh_tri_cost}, box_cost {args.bvh_box_cost})"
                                                        if args.bvh_tri_cost or args.bvh_box_cost else ""),
                   "mode": "auto (autotuned)" if tuned else args.mode,
                   "l2": "flushed between steps",
                   "parallelism": f"replicas x{world}", "cuda_graph": bool(args.graph),
                   "schedule": ({"autotuned": tuned} if tuned else {"mode": args.mode})},
        "spp_per_s_1080p": spp_s,
        "rays_per_step": rays / args.steps,
        "bvh_build_ms": bvh_ms, "upload_ms": upload_ms,
        "kernel_ms_per_step": kms, "kernel_launches_per_step": kl,
        "gpu_launches": int(launches),
        "e2e": {"value": e2e_val, "unit": "Mrays/s", "h2d_bytes_per_step": 48 + 8,
                "d2h_bytes_per_step": W * H * 3 * 4,
                "copies": "each frame's image to pinned host memory, double-buffered on a copy stream"},
        "roofline": {"bound": "alu", "kernel": "k_wf_trace (closest hit)",
                     "achieved": achieved_gops, "peak": alu_peak, "unit": "GOP/s",
                     "frac": achieved_gops / alu_peak if achieved_gops else None,
                     "traffic": traffic,
                     "issue_view": _recorded_issue("trace", args.workload, args.spp_per_step),
                     "peak_source": f"{sm_count} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x "
                                    f"{sm_ghz:.2f} GHz maximum SM clock (recipe unit counts and clock)",
                     "algorithmic_ops_per_launch": trace_ops_step / trace_launches,
                     "launch_ms": trace_ms / trace_launches,
                     "per_ray": {"nodes": cnt["trace_nodes"] / max(cnt["trace_rays"], 1),
                                 "box_tests": cnt["trace_boxes"] / max(cnt["trace_rays"], 1),
                                 "tris": cnt["trace_tris"] / max(cnt["trace_rays"], 1),
                                 "rays_per_step": cnt["trace_rays"],
                                 "ops": f"{OPS_PER_BOX} per child box test, {OPS_PER_TRI} per triangle test"},
                     "hbm_view": {"algorithmic_bytes_per_step": trace_bytes_step, "achieved_gbs": achieved_gbs,
                                  "peak_gbs": peaks["hbm_gbs"], "peak_source": peak_src}},
        "clocks": clocks.summary(),
    }
    # display resolve (off the timed path): tone map of the accumulated frame, 12 B in + 4 B out
    # per pixel
    rgba = torch.empty((H, W, 4), dtype=torch.uint8, device=dev)
    for _ in range(3):
        acc.tonemap(out=rgba)
    t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_a.record(stream)
    for _ in range(20):
        acc.tonemap(out=rgba)
    t_b.record(stream)
    torch.cuda.synchronize()
    tm_ms = t_a.elapsed_time(t_b) / 20
    result["tonemap"] = {"kernel": "k_tonemap", "us": tm_ms * 1e3, "bytes": W * H * 16,
                         "gbs": W * H * 16 / (tm_ms * 1e-3) / 1e9, "note": "after the timed region"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def _relmse(img, ref, eps=1e-2):
    """Mean over pixels and channels of (x - ref)^2 / (ref^2 + eps)."""
    d = img - ref
    return float((d * d / (ref * ref + eps)).mean())


def _time_to(curve, target):
    """Device time at which a relMSE curve (points with spp, ms, relmse) first reaches
    `target`, interpolated log-log between the marks around the crossing; None if never."""
    prev = None
    for p in curve:
        if p["relmse"] <= target:
            if prev is None:
                return p["ms"]
            a, b = math.log(prev["relmse"]), math.log(p["relmse"])
            w = (math.log(target) - a) / (b - a) if b != a else 1.0
            return math.exp(math.log(prev["ms"]) + w * (math.log(p["ms"]) - math.log(prev["ms"])))
        prev = p
    return None


def run_restir_study(args, local):
    """relMSE against a high-spp plain reference as a function of device time on the
    many-light box at 1080p: the plain tracer (next-event estimation with MIS) against ReSTIR DI
    at the primary vertex, both progressive at 1 spp per frame with graph replay."""
    import torch
    from paper_2407_19977_gb300 import api
    from paper_2407_19977_gb300 import native as N
    torch.cuda.set_device(local)
    name = args.workload if args.workload != "pushbutton" else "many_lights"
    sc = _make_workload(name)
    if args.max_depth is not None:
        sc.max_depth = args.max_depth
    W, H = sc.camera.width, sc.camera.height
    scene = api.Scene(sc)
    stream = torch.cuda.current_stream()
    ref = api.Accum(W, H)
    chunk = 64
    for _ in range(args.ref_spp // chunk):
        scene.render(chunk, seed=777, accum=ref, mode=N.PT_MODE_WAVEFRONT)
    torch.cuda.synchronize()
    ref_img = ref.image()
    # pixels whose first hit always scatters (the surfaces ReSTIR lights; pixels that see a
    # light directly carry the same anti-aliasing noise either way)
    surf = scene.features(16, seed=9)[..., 3] >= 1.0
    marks = [m for m in (1, 2, 4, 8, 16, 32, 64, 128, 256) if m <= args.study_frames]
    variants = {"plain": None, "restir_M32_K5_R10": (32, 5, 10), "restir_M8_K5_R10": (8, 5, 10),
                "restir_M8_K5_R10_L8": (8, 5, 10, 8)}
    curves, split = {}, {}
    for kind, r in variants.items():
        acc = api.Accum(W, H)
        for _ in range(3):     # warm-up and graph capture, then start over
            scene.render(1, seed=0, accum=acc, mode=N.PT_MODE_WAVEFRONT, restir=r, use_graph=True)
        acc.reset()
        t_ms = 0.0
        pts = []
        for f in range(1, marks[-1] + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            scene.render(1, seed=0, accum=acc, mode=N.PT_MODE_WAVEFRONT, restir=r, use_graph=True)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ms += e0.elapsed_time(e1)
            if f in marks:
                img = acc.image()
                pts.append({"spp": f, "ms": t_ms, "relmse": _relmse(img, ref_img),
                            "relmse_surfaces": _relmse(img[surf], ref_img[surf])})
        curves[kind] = pts
        km = (N.f32 * len(N.KERNEL_KINDS))()
        probe = api.Accum(W, H)
        for _ in range(4):
            scene.render(1, seed=1, accum=probe, mode=N.PT_MODE_WAVEFRONT, restir=r, kernel_ms=km)
        split[kind] = {n: round(float(km[i]) / 4, 4) for i, n in enumerate(N.KERNEL_KINDS) if km[i] > 0}
    out = {"study": "restir_equal_time", "workload": WORKLOADS[name], "max_depth": sc.max_depth, "ref_spp": args.ref_spp,
           "relmse_eps": 1e-2, "surface_pixels": float(surf.float().mean()), "curves": curves,
           "kernel_ms_per_frame": split}
    for key in ("relmse", "relmse_surfaces"):
        for spp in (16, 64):
            if spp > marks[-1]:
                continue
            target = next(p[key] for p in curves["plain"] if p["spp"] == spp)
            tp = next(p["ms"] for p in curves["plain"] if p["spp"] == spp)
            res = {key: target, "plain_ms": tp}
            for kind in variants:
                if kind == "plain":
                    continue
                curve = [{"spp": p["spp"], "ms": p["ms"], "relmse": p[key]} for p in curves[kind]]
                tr = _time_to(curve, target)
                res[kind] = {"ms": tr, "speedup": (tp / tr) if tr else None}
            out[f"{key}_at_plain_{spp}spp"] = res
    print(json.dumps(out))


def run_bmfr_study(args, local):
    """The regression denoiser on a 1080p frame: relMSE against a high-spp plain reference of
    the noisy mean and of its BMFR output (one 32-pixel grid, and the mean over four grids
    shifted by half a block), with the device time of the feature pass and of the regression."""
    import torch
    from paper_2407_19977_gb300 import api
    from paper_2407_19977_gb300 import native as N
    torch.cuda.set_device(local)
    name = args.workload
    sc = _make_workload(name)
    W, H = sc.camera.width, sc.camera.height
    scene = api.Scene(sc)
    stream = torch.cuda.current_stream()
    ref = api.Accum(W, H)
    chunk = 64
    for _ in range(args.ref_spp // chunk):
        scene.render(chunk, seed=777, accum=ref, mode=N.PT_MODE_WAVEFRONT)
    torch.cuda.synchronize()
    ref_img = ref.image()

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return r, a.elapsed_time(b) / reps

    rows = []
    for spp in (1, 4, 16):
        acc = api.Accum(W, H)
        _, t_render = timed(lambda: (acc.reset(), scene.render(spp, seed=1, accum=acc, mode=N.PT_MODE_WAVEFRONT)))
        color = acc.image()
        feats, t_feat = timed(lambda: scene.features(spp, seed=1))
        den, t_bmfr = timed(lambda: api.bmfr(color, feats, block=32))
        grids = [(0, 0), (16, 0), (0, 16), (16, 16)]
        den4 = sum(api.bmfr(color, feats, block=32, offset=o) for o in grids) / 4.0
        rows.append({"spp": spp, "render_ms": t_render, "features_ms": t_feat, "bmfr_ms": t_bmfr,
                     "relmse_noisy": _relmse(color, ref_img), "relmse_bmfr": _relmse(den, ref_img),
                     "relmse_bmfr_4_grids": _relmse(den4, ref_img)})
    print(json.dumps({"study": "bmfr", "workload": WORKLOADS[name], "ref_spp": args.ref_spp, "block": 32,
                      "relmse_eps": 1e-2, "rows": rows}))


def run_nrc_study(args, local):
    """relMSE against a high-spp plain reference as a function of device time, for the plain
    tracer and for the radiance-cache tracer (trained online every frame), both progressive
    at 1 spp per frame with graph replay (the first frame, which captures, is timed too)."""
    import torch
    from paper_2407_19977_gb300 import api
    from paper_2407_19977_gb300 import native as N
    torch.cuda.set_device(local)
    sc = _make_workload(args.workload)
    W, H = sc.camera.width, sc.camera.height
    scene = api.Scene(sc)
    stream = torch.cuda.current_stream()
    ref = api.Accum(W, H)
    chunk = 64
    for i in range(args.ref_spp // chunk):
        scene.render(chunk, seed=777, accum=ref, mode=N.PT_MODE_WAVEFRONT)
    torch.cuda.synchronize()
    ref_img = ref.image()
    # where the light comes from: the image rendered with paths cut after their first and
    # second vertices, against the full reference (the cache can only replace what lies past
    # the second diffuse-ish vertex, so the shares bound what it can gain)
    shares = {}
    for depth in (1, 2):
        part = api.Accum(W, H)
        for i in range(256 // chunk):
            scene.render(chunk, max_depth=depth, seed=778, accum=part, mode=N.PT_MODE_WAVEFRONT)
        torch.cuda.synchronize()
        shares[f"depth_le_{depth}"] = float(part.image().mean() / ref_img.mean())
    marks = [m for m in (1, 2, 4, 8, 16, 32, 64, 128, 256) if m <= args.study_frames]
    curves = {}
    lo = sc.vertices.min(0) - 0.05
    hi = sc.vertices.max(0) + 0.05
    for kind in ("plain", "nrc"):
        net = (api.Nrc(seed=5, box=(tuple(map(float, lo)), tuple(map(float, hi))), batch=args.nrc_batch,
                       frame_samples=args.nrc_frame_samples) if kind == "nrc" else None)
        acc = api.Accum(W, H)
        t_ms = 0.0
        pts = []
        for f in range(1, marks[-1] + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            scene.render(1, seed=0, accum=acc, mode=N.PT_MODE_WAVEFRONT, nrc=net, nrc_train=net is not None,
                         use_graph=True)
            e1.record(stream)
            torch.cuda.synchronize()
            t_ms += e0.elapsed_time(e1)
            if f in marks:
                pts.append({"spp": f, "ms": t_ms, "relmse": _relmse(acc.image(), ref_img)})
        curves[kind] = pts

    time_to = _time_to
    out = {"study": "nrc_equal_time", "workload": WORKLOADS[args.workload], "ref_spp": args.ref_spp,
           "nrc_batch": args.nrc_batch, "nrc_frame_samples": args.nrc_frame_samples,
           "relmse_eps": 1e-2, "radiance_share_of_paths_cut_at_depth": shares, "curves": curves}
    for spp in (16, 64):
        if spp > marks[-1]:
            continue
        target = next(p["relmse"] for p in curves["plain"] if p["spp"] == spp)
        tp = next(p["ms"] for p in curves["plain"] if p["spp"] == spp)
        tn = time_to(curves["nrc"], target)
        out[f"at_plain_{spp}spp"] = {"relmse": target, "plain_ms": tp, "nrc_ms": tn,
                                     "speedup": (tp / tn) if tn else None}
    # the equal-time factor splits into the error removed per sample and the time each sample
    # costs: at equal spp, plain relMSE / NRC relMSE and NRC ms / plain ms
    out["per_spp"] = [{"spp": a["spp"], "relmse_plain_over_nrc": a["relmse"] / b["relmse"],
                       "ms_nrc_over_plain": b["ms"] / a["ms"]}
                      for a, b in zip(curves["plain"], curves["nrc"])]
    print(json.dumps(out))


def run_nrc_train_study(args, local):
    """Radiance-cache kernels alone at the production configuration (16 levels x 2^19 entries,
    64-wide 4-hidden MLP): one frame's online training (65,536 samples by default, Adam steps of
    8,192) with the fused tcgen05 kernel and with the multi-kernel path, and inference on one
    1080p frame of queries with each inference kernel.  Synthetic records: positions uniform in
    the unit box, directions and normals uniform on the sphere, roughness and targets uniform.
    MLP FLOPs per sample: forward 2 (4 * 64 * 64 + 3 * 64); training three times that (forward,
    input gradients, weight gradients)."""
    import numpy as np
    import torch
    from paper_2407_19977_gb300 import api
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()

    def records(rng, n):
        rec = np.zeros((n, 16), np.float32)
        rec[:, 0:3] = rng.random((n, 3))
        d = rng.normal(size=(n, 3))
        rec[:, 3:6] = d / np.linalg.norm(d, axis=1, keepdims=True)
        m = rng.normal(size=(n, 3))
        rec[:, 6:9] = m / np.linalg.norm(m, axis=1, keepdims=True)
        rec[:, 9] = rng.random(n)
        rec[:, 10:13] = rng.random((n, 3))
        return torch.from_numpy(rec).to("cuda")

    rng = np.random.default_rng(0)
    n_train = args.nrc_frame_samples
    train = records(rng, n_train)
    queries = records(rng, 1920 * 1080)
    flops_fwd = 2.0 * (4 * 64 * 64 + 3 * 64)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps

    out = {"study": "nrc_kernels", "grid": "16 levels x 2^19 entries x 2 FP16 features", "mlp": "64 wide, 4 hidden",
           "train_samples_per_frame": n_train, "batch": args.nrc_batch, "infer_queries": queries.shape[0],
           "steps": args.steps, "train": {}, "infer": {}}
    for tk, name in ((0, "fused_tcgen05"), (1, "multi_kernel")):
        net = api.Nrc(batch=args.nrc_batch, seed=3, train_kernels=tk)
        ms = timed(lambda: net.train(train))
        out["train"][name] = {"ms_per_frame": ms, "ms_per_batch": ms * args.nrc_batch / n_train,
                              "mlp_tflops": 3 * flops_fwd * n_train / (ms * 1e-3) / 1e12,
                              "final_loss": net.last_loss()}
        del net
    for tc, name in ((False, "mma_sync"), (True, "tcgen05")):
        net = api.Nrc(batch=args.nrc_batch, seed=3, tcgen05=tc)
        net.train(train)
        ms = timed(lambda: net.infer(queries))
        out["infer"][name] = {"ms_per_frame": ms, "mlp_tflops": flops_fwd * queries.shape[0] / (ms * 1e-3) / 1e12}
        del net
    print(json.dumps(out))


def run_batch_study(args, local):
    """64 seeded scenes of uneven size (pushbutton / heavy generators, 1k-500k triangles
    log-uniform, 256^2 .. 1920x1080, 1-32 spp, depth 8): aggregate samples per second of the
    batch schedules (the one pt_autotune_batch picks on 1-spp copies of the jobs; one persistent
    megakernel launch; per-job wavefronts on 4 and 8 streams; one merged wavefront for all jobs
    as a captured graph at 2^21 .. 2^24 paths per wave) against the same jobs as per-scene
    pt_render calls (PT_MODE_AUTO: wavefront from 2^16 pixels with graph replay, megakernel
    below), all on one stream."""
    import torch
    from paper_2407_19977_gb300 import api, scenes
    from paper_2407_19977_gb300 import native as N
    torch.cuda.set_device(local)
    specs = scenes.batch_specs(args.batch_scenes)
    t0 = time.perf_counter()
    scs = [scenes.scene_from_spec(s) for s in specs]
    gen_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    gs = [api.Scene(sc) for sc in scs]
    torch.cuda.synchronize()
    upload_build_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    samples = sum(s["width"] * s["height"] * s["spp"] for s in specs)
    tris = sum(len(sc.indices) for sc in scs)

    def timed(fn, reps=2):
        out = []
        for _ in range(reps):   # the first pass captures graphs
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return out[-1]

    accs = [api.Accum(s["width"], s["height"]) for s in specs]

    def per_scene():
        for sp, g, sc, acc in zip(specs, gs, scs, accs):
            g.render(sp["spp"], max_depth=sp["max_depth"], seed=sp["seed"], accum=acc, mode=N.PT_MODE_AUTO,
                     use_graph=True)
    baccs = [api.Accum(s["width"], s["height"]) for s in specs]
    tune_jobs = [(g, sc.camera, 1, sp["max_depth"], sp["seed"], acc) for sp, g, sc, acc in zip(specs, gs, scs, baccs)]
    # BVH width (every scene rebuilt at 8, 6 and 4 children per node) and schedule; every
    # variant below, per-scene launches included, then runs on the trees it leaves
    best, tune_ms = api.autotune_batch(tune_jobs, frames=1, bvh=not args.no_bvh_tune)
    bvh_width = gs[0].stats()["bvh_width"]
    t_scene = timed(per_scene)
    jobs = [(g, sc.camera, sp["spp"], sp["max_depth"], sp["seed"], acc) for sp, g, sc, acc in zip(specs, gs, scs, baccs)]
    variants = {"tuned": best,
                "megakernel_one_launch": {"mode": N.PT_MODE_MEGAKERNEL, "streams": 0, "tile_pixels": 32,
                                          "blocks_per_sm": 4, "use_graph": 1},
                "wavefront_4_streams": {"mode": N.PT_MODE_WAVEFRONT, "streams": 4, "tile_pixels": 0,
                                        "blocks_per_sm": 0, "use_graph": 0},
                "wavefront_8_streams": {"mode": N.PT_MODE_WAVEFRONT, "streams": 8, "tile_pixels": 0,
                                        "blocks_per_sm": 0, "use_graph": 0}}
    for wp in (1 << 21, 1 << 22, 1 << 23, 1 << 24):
        variants[f"merged_wavefront_{wp >> 20}M_graph"] = {"mode": N.PT_MODE_WAVEFRONT, "streams": 0, "tile_pixels": 0,
                                                          "blocks_per_sm": 0, "use_graph": 1, "merged": 1,
                                                          "wave_paths": wp}
    res = {}
    for name, o in variants.items():
        t = timed(lambda: api.render_batch(jobs, tile_pixels=o["tile_pixels"], blocks_per_sm=o["blocks_per_sm"],
                                           use_graph=bool(o["use_graph"]), mode=o["mode"], streams=o["streams"],
                                           merged=bool(o.get("merged", 0)), wave_paths=o.get("wave_paths", 0)))
        res[name] = {"ms": t, "msamples_per_s": samples / (t * 1e-3) / 1e6, "opts": o,
                     "over_per_scene": t_scene / t}
    out = {"study": "batch", "workload": f"{len(specs)} seeded scenes: pushbutton/heavy generators, "
                                          f"{tris:,} triangles in all, 256^2..1920x1080, 1-32 spp, depth 8",
           "samples": samples, "scene_gen_s": gen_s, "upload_build_s": upload_build_s,
           "per_scene": {"ms": t_scene, "msamples_per_s": samples / (t_scene * 1e-3) / 1e6},
           "batch": res, "tune_ms_per_1spp_batch": tune_ms, "bvh_width": bvh_width}
    print(json.dumps(out))


# Table 2 and Table 1 of the paper (context only: WebGPU in Chrome on an RTX 3080 / Ryzen 5 5600X)
PAPER_TABLE2_MS = {1_068_735: (1058.73, 59.47), 106_873: (790.20, 3.79), 10_687: (790.83, 4.18)}
PAPER_TABLE1_MS = {1_068_735: 383.10, 106_873: 41.77, 10_687: 8.43}


def run_paper_study(args, local):
    """The paper's own workload shape (Tables 1 and 2): the pushbutton at about 10.7k, 107k and
    1.07M triangles, 512x512, 100 spp, ray depth 5, each figure the mean and standard deviation
    of 30 runs.  Per mesh: the device BVH build (30 timed builds after 3 untimed) and the
    100-spp frame (schedule from pt_autotune at 100 spp, 3 untimed frames, then 30 timed frames,
    each into a zeroed accumulator, L2 flushed between frames outside the timed events)."""
    import torch
    from paper_2407_19977_gb300 import api, scenes
    from paper_2407_19977_gb300 import native as N
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    runs = 30
    rows = []

    def ev_ms(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    clocks = ClockSampler(local)
    with clocks:
        for n in sorted(PAPER_TABLE2_MS):
            sc = scenes.pushbutton_lod(n)
            g = api.Scene(sc, build=False)
            for _ in range(3):
                g.build()
            builds = []
            for _ in range(runs):
                flush.fill_(1.0)
                builds.append(ev_ms(lambda: g.build()))
            opts, _ = g.autotune(spp=sc.spp, max_depth=sc.max_depth, frames=1)
            acc = api.Accum(sc.camera.width, sc.camera.height)

            def frame():
                g.render(sc.spp, max_depth=sc.max_depth, seed=0, accum=acc, mode=N.PT_MODE_AUTO)
            for _ in range(3):
                acc.reset()
                frame()
            st0 = g.stats()
            frames = []
            for k in range(runs):
                acc.reset()
                flush.fill_(float(k))
                frames.append(ev_ms(frame))
            st1 = g.stats()
            rays = (st1["ext_rays"] - st0["ext_rays"]) + (st1["shadow_rays"] - st0["shadow_rays"])
            fm, fs = statistics.mean(frames), statistics.stdev(frames)
            bm, bs = statistics.mean(builds), statistics.stdev(builds)
            samples = sc.camera.width * sc.camera.height * sc.spp
            row = {"target_tris": n, "tris": g.n_tris, "bvh_build_ms": [round(bm, 3), round(bs, 3)],
                   "frame_ms": [round(fm, 3), round(fs, 3)], "spp_per_s": sc.spp / (fm * 1e-3),
                   "msamples_per_s": samples / (fm * 1e-3) / 1e6, "mrays_per_s": rays / (sum(frames) * 1e-3) / 1e6,
                   "rays_per_frame": rays / runs, "schedule": opts,
                   "paper_rtx3080_frame_ms": list(PAPER_TABLE2_MS[n]),
                   "paper_cpu_bvh_build_ms": PAPER_TABLE1_MS[n],
                   "frame_time_ratio_vs_paper": PAPER_TABLE2_MS[n][0] / fm}
            if not args.no_cpu_baseline:
                row["cpu_baseline"] = cpu_baseline(sc, args.cpu_seconds / 3)
            rows.append(row)
            del g
    print(json.dumps({"study": "paper_tables", "workload": "pushbutton at the Table 1/2 triangle counts, 512x512, "
                      "100 spp, depth 5, 30 runs each (mean, std)", "rows": rows, "clocks": clocks.summary(),
                      "note": "paper figures are WebGPU in a browser on other hardware: context, not a target"}))


def main():
    args = _args()
    world, rank, local = _dist()
    if args.study == "nrc":
        if rank == 0:
            run_nrc_study(args, local)
        return
    if args.study == "bmfr":
        if rank == 0:
            run_bmfr_study(args, local)
        return
    if args.study == "restir":
        if rank == 0:
            run_restir_study(args, local)
        return
    if args.study == "paper":
        if rank == 0:
            run_paper_study(args, local)
        return
    if args.study == "batch":
        if rank == 0:
            run_batch_study(args, local)
        return
    if args.study == "nrc_train":
        if rank == 0:
            run_nrc_train_study(args, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
