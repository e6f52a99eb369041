"""Benchmark: dense RGBD plane fitting on GB300.

One step = one pass of the whole hot path (fixed-point quantum, window
moments, per-pixel solve) over the batch
  8 x 1920x1080 + 2 x 4096x3072 float32 depth frames, 0.3-10 m,
  sigma_Z = 0.0015 Z^2, 5 % missing, 31 x 31 windows, disparity form,
with the inputs resident in HBM (167 MB of depth in, 834 MB of results out:
both larger than the 129 MB L2, so no flush is needed between steps).

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import os
import re
import shutil
import signal
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "Mpix plane-fits/s at 640x480 & 1080p, % HBM peak, vs plain fit on same GPU"
UNIT = "Mpix/s"
BYTES_PER_PIXEL = 24  # algorithmic: 4 B depth in + 12 B normal + 4 B offset + 4 B curvature out
WORKLOAD = "8x1920x1080+2x4096x3072 f32 depth, 0.3-10 m, sigma 0.0015 Z^2, 5% missing, 31x31 windows, disparity form"
K = 31


def workload_frames():
    """[(W, H, intrinsics, [frames])] of the benchmark batch (seeded, synthetic)."""
    groups = []
    for (W, H, n, seed0) in [(1920, 1080, 8, scenes.BASE_SEED + 300), (4096, 3072, 2, scenes.BASE_SEED + 400)]:
        intr = scenes.Intrinsics.scaled(W, H)
        frames = [scenes.wide_range_frame(seed0 + i, intr, W, H) for i in range(n)]
        groups.append((W, H, intr, frames))
    return groups


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# NVML clock-event (throttle) reason bits kept in the record
NVML_REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown", 0x4: "sw_power_cap"}


class _Nvml:
    """Read-only NVML queries through ctypes (the driver's libnvidia-ml; no Python package needed)."""

    SM = 1  # NVML_CLOCK_SM

    def __init__(self, uuid, pci_bus_id, index):
        import ctypes

        self.c = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        rc = 1
        if uuid:
            rc = self.lib.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h))
        if rc != 0 and pci_bus_id:
            rc = self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci_bus_id.encode(), ctypes.byref(self.h))
        if rc != 0:
            rc = self.lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.h))
        if rc != 0:
            raise OSError("no NVML handle for the device")
        try:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reasons_fn = self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        u = ctypes.c_uint()
        self.max_mhz = float(u.value) if self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, ctypes.byref(u)) == 0 \
            else None
        self.sample()

    def sample(self):
        c = self.c
        mhz, mw, r = c.c_uint(), c.c_uint(), c.c_ulonglong()
        ok = self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, c.byref(mhz)) == 0
        self.lib.nvmlDeviceGetPowerUsage(self.h, c.byref(mw))
        self.reasons_fn(self.h, c.byref(r))
        return (float(mhz.value) if ok else None, mw.value / 1000.0, int(r.value))

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """SM clock, power and throttle reasons sampled every 2 ms by NVML on a host thread (nvidia-smi every
    50 ms where NVML cannot be loaded); `stop` keeps the samples taken inside a host-time window (the
    timed region), else the two nearest ones."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_S = 0.002

    def __init__(self, gpu_index: int, device=None):
        import threading

        self.rows = []  # (host time, sm_mhz, max_mhz, [reasons])
        self.proc = None
        self.path = None
        self.nvml = None
        self.source = None
        uuid = pci = None
        if device is not None:
            import torch

            p = torch.cuda.get_device_properties(device)
            uuid = "GPU-" + str(p.uuid) if getattr(p, "uuid", None) is not None else None
            if getattr(p, "pci_bus_id", None) is not None:
                pci = "%08x:%02x:%02x.0" % (p.pci_domain_id, p.pci_bus_id, p.pci_device_id)
        try:
            self.nvml = _Nvml(uuid, pci, gpu_index)
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self.source = "nvml every %g ms" % (1000 * self.PERIOD_S)
            self.halt = threading.Event()

            def run():
                while not self.halt.is_set():
                    mhz, _, bits = self.nvml.sample()
                    self.rows.append((time.time(), mhz, self.nvml.max_mhz,
                                      [n for m, n in NVML_REASONS.items() if bits & m]))
                    time.sleep(self.PERIOD_S)

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        smi = shutil.which("nvidia-smi")
        if smi:
            self.source = "nvidia-smi every 50 ms"
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen([smi, "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            # wait (up to 3 s) for the first sample, so that sampling covers what follows
            t_end = time.time() + 3.0
            while time.time() < t_end and os.path.getsize(self.path) == 0:
                time.sleep(0.02)

    def _smi_rows(self):
        time.sleep(0.1)  # one more sample after the region
        self.proc.send_signal(signal.SIGTERM)
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 10:
                    continue
                try:
                    t = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                num = lambda v: float(v) if v.replace(".", "").isdigit() else None  # noqa: E731
                rows.append((t, num(p[2]), num(p[3]), [names[i] for i in range(4) if p[6 + i].lower() == "active"]))
        os.unlink(self.path)
        return rows

    def stop(self, window=None):
        if self.nvml is not None:
            time.sleep(2 * self.PERIOD_S)
            self.halt.set()
            self.thread.join(timeout=5)
            self.nvml.close()
            rows = list(self.rows)
        elif self.proc is not None:
            rows = self._smi_rows()
        else:
            return None
        if not rows:
            return None
        inside = rows
        if window is not None:
            inside = [r for r in rows if window[0] <= r[0] <= window[1]]
            if not inside:
                mid = 0.5 * (window[0] + window[1])
                inside = sorted(rows, key=lambda r: abs(r[0] - mid))[:2]
        sm = [r[1] for r in inside if r[1] is not None]
        mx = [r[2] for r in inside if r[2] is not None]
        reasons = sorted({n for r in inside for n in r[3]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "source": self.source,
                "samples_in_timed_region": len([r for r in rows if window and window[0] <= r[0] <= window[1]])}


def cpu_oracle_sample(time_budget_s: float = 15.0):
    """Time the FP64 oracle on the benchmark's 1080p frames (bounded sample, ~10-30 s)."""
    import oracle

    W, H = 1920, 1080
    intr = scenes.Intrinsics.scaled(W, H)
    frames = [scenes.wide_range_frame(scenes.BASE_SEED + 300 + i, intr, W, H) for i in range(8)]
    t0 = time.perf_counter()
    oracle.fit(frames[0], intr.as_tuple(), K, "disparity")
    dt0 = time.perf_counter() - t0
    n = int(max(1, min(8, time_budget_s / max(dt0, 1e-3))))
    t0 = time.perf_counter()
    for f in frames[:n]:
        oracle.fit(f, intr.as_tuple(), K, "disparity")
    dt = time.perf_counter() - t0
    px = n * W * H
    return {"value": px / dt / 1e6, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "%d of the 8 1920x1080 frames of the benchmark batch (%d px), k=31, disparity form, "
                      "FP64 direct window sums, OpenMP over rows" % (n, px), "seconds": dt}


def mixed_batch_report(dev, timed, world=1):
    """64 frames, resolutions uniform over {320x240, 640x480, 1280x720, 1920x1080}, windows over
    {5, 7, 11, 21}, intrinsics scaled with the resolution, 0-15 % blob holes: one persistent launch per
    stage replayed from a CUDA graph, tile shapes from the autotuner."""
    import torch

    from paper_2103_06644_gb300 import SurfaceFitBatch, autotune

    spec = scenes.mixed_batch_spec(64)
    frames = []
    for i, (W, H, k) in enumerate(spec):
        depth, intr = scenes.mixed_frame(scenes.BASE_SEED + 800 + i, W, H)
        frames.append(dict(W=W, H=H, window=k, intrinsics=intr.as_tuple(), depth=torch.from_numpy(depth).to(dev)))
    t0 = time.perf_counter()
    tuned = autotune.tune(frames)
    tune_s = time.perf_counter() - t0
    b = SurfaceFitBatch(tuned, use_graph=True)
    for _ in range(3):
        b.run()
    ms = timed(20, b.run)
    rep = {"workload": "64 mixed frames (320x240..1920x1080, k in {5,7,11,21}), disparity form, CUDA graph",
           "pixels": b.pixels, "value": whole_job_rate(world, b.pixels, ms), "unit": UNIT, "ms_per_step": ms,
           "launches_per_step": b.launches, "autotune_seconds": tune_s,
           "tile_shapes": len({(f["hseg"], f["vband"]) for f in tuned})}
    b.close()
    return rep


def segmentation_report(dev, timed, world=1):
    """Planar segmentation (Section III): 30 frames of 512x424, root tiles 64 px, up to 3 splits,
    every form; one step = the whole segmentation of the 30 frames (nodes stay on the device)."""
    import torch

    from paper_2103_06644_gb300 import SurfaceFitter

    frames = torch.from_numpy(np.stack([scenes.segmentation_frame(scenes.BASE_SEED + 1000 + i)
                                        for i in range(30)])).to(dev)
    intr = scenes.SEG_INTRINSICS.as_tuple()
    taus = {"disparity": 1e-2, "standard": 2e-2, "explicit_disparity": 5e-3, "explicit_standard": 2.6e-2}
    rep = {"workload": "30 x 512x424 f32, 6-10 planes, 0.5-4.5 m, sigma 1.425e-3 Z^2, 2-8 % holes; "
                       "root tile 64, max 3 splits, min 50 % valid", "tau": taus}
    for method, tau in taus.items():
        f = SurfaceFitter(intr, scenes.SEG_W, scenes.SEG_H, 5, method=method)
        bufs = f.quadtree(frames, tile=64, max_level=3, tau=tau, to_host=False)
        for _ in range(3):
            f.quadtree(frames, tile=64, max_level=3, tau=tau, out=bufs, to_host=False)
        ms = timed(20, lambda: f.quadtree(frames, tile=64, max_level=3, tau=tau, out=bufs, to_host=False))
        nodes = int(bufs[1].item())
        rep[method] = {"ms_per_30_frames": ms, "frames_per_s": world * 30 / (ms / 1000), "nodes": nodes,
                       "Mnodes_per_s": world * nodes / (ms / 1000) / 1e6,
                       "value": whole_job_rate(world, 30 * scenes.SEG_W * scenes.SEG_H, ms), "unit": UNIT}
        f.close()
    return rep


def precision_report(group, dev):
    """Worst errors against the FP64 oracle on the first 1080p frame of the batch for each precision mode
    (0: float32 solve; 1: FP64-class refinement of the windows the float32 solve cannot vouch for;
    2: every window), over the windows with relative eigenvalue gap >= 1e-3 and >= 1e-6.  Offsets are
    relative to the window centroid's distance |mu|; a plane through the camera centre to within
    1e-4 |mu| is compared up to sign."""
    import torch

    import oracle
    from paper_2103_06644_gb300 import SurfaceFitter

    W, H, intr, frames = group
    depth = frames[0]
    ref = oracle.fit(depth, intr.as_tuple(), K, "disparity", want_lambda=True, want_moments=True)
    ok = np.isfinite(ref["offsets"])
    lam = ref["lam"]
    gap = np.where(ok, (lam[..., 1] - lam[..., 0]) / np.where(ok, lam[..., 2], 1), 0)
    mu = np.linalg.norm(ref["moments"][..., 6:9] / np.where(ok[..., None], ref["moments"][..., 9:10], 1), axis=-1)
    free = np.abs(np.where(ok, ref["offsets"], 1.0)) <= 1e-4 * np.where(ok, mu, 1.0)
    d = torch.from_numpy(depth).to(dev)
    rep = {"frame": "first 1920x1080 frame of the batch, k=31, disparity form", "valid": int(ok.sum()),
           "tolerance": "normal 1e-3 rad, offset 1e-4 |mu|"}
    for mode in (0, 1, 2):
        f = SurfaceFitter(intr.as_tuple(), W, H, K)
        f.set_precision(mode)
        n, o, c = [t.cpu().numpy().astype(np.float64) for t in f.fit(d)]
        torch.cuda.synchronize()
        ent = {"queued": f.precision_stats()[0]} if mode else {}
        for name, gmin in (("gamma>=1e-3", 1e-3), ("gamma>=1e-6", 1e-6)):
            sel = ok & (gap >= gmin)
            a, b, fr = n[sel], ref["normals"][sel], free[sel]
            ang = np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, -1))
            ang = np.where(fr, np.minimum(ang, np.pi - ang), ang)
            od = np.where(fr, np.abs(np.abs(o[sel]) - np.abs(ref["offsets"][sel])),
                          np.abs(o[sel] - ref["offsets"][sel])) / mu[sel]
            ent[name] = {"windows": int(sel.sum()), "max_angle_rad": float(ang.max()),
                         "max_offset_rel": float(od.max()),
                         "max_curvature_err": float(np.abs(c[sel] - ref["curvature"][sel]).max())}
        rep["mode%d" % mode] = ent
        f.close()
    return rep


def tolerance_met_report(fitters, step, timed, world, total_px, what="disparity"):
    """The same batch in precision mode 1 (the configuration that holds the tolerance on every window with
    gamma >= 1e-6): throughput and the share of windows refined."""
    for f in fitters:
        f.set_precision(1)
    for _ in range(3):
        step()
    ms1 = timed(10, step)
    queued = sum(f.precision_stats()[0] for f in fitters)
    for f in fitters:
        f.set_precision(0)
    return {"precision_mode": 1, "tau": 1e-3, "form": what, "value": whole_job_rate(world, total_px, ms1),
            "unit": UNIT, "ms_per_step": ms1, "windows_refined_frac": queued / total_px,
            "accuracy": "normal 1e-3 rad, offset 1e-4 |mu| on every window with gamma >= 1e-6"}


PROFILE_LAUNCHES = os.path.join(ROOT, "profiles", "batch_1080p_4k_k31_launches.md")
STAGE_KERNEL = {"range": "range", "hpass": "hpass", "vpass_solve": "vpass", "fp64_resolve": "resolve"}


def kernel_source_hash() -> str:
    """Hash of the device sources (kernels + solve); host-side changes do not alter it."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2103_06644_gb300", "csrc")
    for f in ("sf_kernels.cuh", "sf_solve.cuh"):
        h.update(f.encode())
        with open(os.path.join(d, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_record(name: str, stage: str, field: str):
    """A per-launch figure of a stage's kernel from the committed ncu launch summary
    (`<name>: kernel=K sources=HASH <field>=N`), or None when that capture was taken on other kernel
    sources (or is missing)."""
    kern = STAGE_KERNEL.get(stage)
    try:
        with open(PROFILE_LAUNCHES) as fh:
            text = fh.read()
    except OSError:
        return None
    m = re.search(r"%s: kernel=%s sources=([0-9a-f]+) %s=(\d+)" % (name, kern, field), text)
    if not m or m.group(1) != kernel_source_hash():
        return None
    return int(m.group(2))


def recorded_traffic(stage: str):
    """DRAM bytes (read + write) per launch of a stage's kernel, from ncu."""
    return _profile_record("traffic_record", stage, "bytes_per_launch")


def recorded_instructions(stage: str):
    """Thread instructions executed per launch of a stage's kernel, from ncu."""
    return _profile_record("instr_record", stage, "thread_inst_per_launch")


def issue_roofline(stage: str, launch_ms: float, clocks, sms: int):
    """The stage's kernel against instruction issue: executed thread instructions (ncu count per
    launch) / CUDA-event launch time, against SMs x 4 schedulers x 32 lanes x SM clock (one warp
    instruction per scheduler per cycle).  None without a matching ncu record."""
    inst = recorded_instructions(stage)
    if inst is None or launch_ms <= 0:
        return None
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    peak = sms * 128 * mhz * 1e6 / 1e12
    achieved = inst / (launch_ms / 1000.0) / 1e12
    return {"bound": "alu", "kernel": stage, "achieved": achieved, "peak": peak, "unit": "Tinst/s",
            "frac": achieved / peak, "thread_inst_per_launch": inst, "sm_mhz": mhz, "sms": sms,
            "peak_source": "SMs x 128 lanes x sampled SM clock"}


def rank_max(x: float, world: int, device) -> float:
    """Max of a per-rank scalar over all ranks (the job's slowest rank sets the time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, px_per_rank: int, ms: float) -> float:
    """Mpix/s of the whole job: every rank fits px_per_rank pixels per step in ms (max over ranks)."""
    return world * px_per_rank / (ms / 1000.0) / 1e6


def run_single_case(args):
    """One seeded 1920x1080 frame of the benchmark batch fitted --steps times (for ncu captures)."""
    import torch

    from paper_2103_06644_gb300 import SurfaceFitter

    W, H = 1920, 1080
    intr = scenes.Intrinsics.scaled(W, H)
    d = torch.from_numpy(scenes.wide_range_frame(scenes.BASE_SEED + 300, intr, W, H)).cuda()
    f = SurfaceFitter(intr.as_tuple(), W, H, K, method=args.method)
    for _ in range(max(1, args.steps)):
        f.fit(d)
    torch.cuda.synchronize()
    f.close()
    print(json.dumps({"case": "single1080", "method": args.method, "fits": max(1, args.steps)}))


def run_vga_case(args):
    """One seeded 640x480 frame, k=7, fitted --steps times through the C ABI with fixed arguments (repeated
    calls replay the context's captured graph), for ncu captures of the small-frame case."""
    import torch

    from paper_2103_06644_gb300 import SurfaceFitter, _native

    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    d = torch.from_numpy(scenes.kinect_frame(scenes.BASE_SEED, intr, 640, 480)).cuda()
    out = (torch.empty((480, 640, 3), device="cuda"), torch.empty((480, 640), device="cuda"),
           torch.empty((480, 640), device="cuda"))
    f = SurfaceFitter(intr.as_tuple(), 640, 480, 7, method=args.method)
    cargs = (f._h, 1, d.data_ptr(), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None,
             torch.cuda.current_stream().cuda_stream)
    lib = _native.lib()
    for _ in range(max(1, args.steps)):
        _native.check(lib.sf_fit_ex(*cargs))
    torch.cuda.synchronize()
    print(json.dumps({"case": "vga", "method": args.method, "fits": max(1, args.steps),
                      "graph_replays": f.graph_replays()}))
    f.close()


def run_mixed_case(args):
    """The 64-frame mixed batch of `mixed_batch`, tuned, then run --steps times (one persistent launch per
    pass, replayed from a CUDA graph), for ncu captures of the batch kernel."""
    import torch

    from paper_2103_06644_gb300 import SurfaceFitBatch, autotune

    frames = []
    for i, (W, H, k) in enumerate(scenes.mixed_batch_spec(64)):
        depth, intr = scenes.mixed_frame(scenes.BASE_SEED + 800 + i, W, H)
        frames.append(dict(W=W, H=H, window=k, intrinsics=intr.as_tuple(), depth=torch.from_numpy(depth).cuda()))
    b = SurfaceFitBatch(autotune.tune(frames), use_graph=True)
    for _ in range(max(1, args.steps)):
        b.run()
    b.check()
    print(json.dumps({"case": "mixed", "passes": max(1, args.steps), "pixels": b.pixels, "launches": b.launches}))
    b.close()


def run_tolerance_case(args):
    """The benchmark batch (8 x 1080p + 2 x 4K, k=31) in precision mode 1, tau 1e-3 (the configuration of
    `tolerance_met_config`), fitted --steps times, for ncu captures of the refinement kernels."""
    import torch

    from paper_2103_06644_gb300 import SurfaceFitter

    fits = []
    for (W, H, intr, frames) in workload_frames():
        f = SurfaceFitter(intr.as_tuple(), W, H, K, method=args.method)
        f.set_precision(1, 1e-3)
        fits.append((f, torch.from_numpy(np.stack(frames)).cuda()))
    for _ in range(max(1, args.steps)):
        for f, t in fits:
            f.fit(t)
    torch.cuda.synchronize()
    print(json.dumps({"case": "tolerance", "method": args.method, "steps": max(1, args.steps),
                      "queued_resummed": [f.precision_stats() for f, _ in fits]}))
    for f, _ in fits:
        f.close()


def run_diff_case(args):
    """16 x 640x480 f32 frames, k=9 (or --window): forward, upstream gradient and backward, --steps times
    (for ncu captures of the backward kernels)."""
    import torch

    from paper_2103_06644_gb300 import SurfaceFitter

    intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
    nd = 16
    dd = torch.from_numpy(np.stack([scenes.kinect_frame(scenes.BASE_SEED + 600 + i, intr, 640, 480)
                                    for i in range(nd)])).cuda()
    tgt = torch.from_numpy(np.stack([scenes.target_normals(scenes.BASE_SEED + 700 + i, 480, 640)
                                     for i in range(nd)]).astype(np.float32)).cuda()
    zero = torch.zeros((nd, 480, 640), device="cuda")
    fd = SurfaceFitter(intr.as_tuple(), 640, 480, args.window, method=args.method)
    for _ in range(max(1, args.steps)):
        n_, o_, c_ = fd.fit(dd)
        valid = torch.isfinite(o_)
        gn = torch.where(valid[..., None], 2.0 * (n_ - tgt), torch.zeros_like(n_))
        gk = torch.where(valid, torch.full_like(c_, 0.1), torch.zeros_like(c_))
        fd.backward(dd, gn, zero, gk)
    torch.cuda.synchronize()
    fd.close()
    print(json.dumps({"case": "diff16", "method": args.method, "window": args.window, "steps": max(1, args.steps)}))


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on bounded samples of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    W, H = 1920, 1080
    intr = scenes.Intrinsics.scaled(W, H)
    frame = scenes.wide_range_frame(scenes.BASE_SEED + 300, intr, W, H)
    rows = 24
    band = frame[:rows + K - 1]
    for _ in range(args.warmup):
        oracle.fit(band[:K + 1], intr.as_tuple(), K, "disparity")
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.fit(band, intr.as_tuple(), K, "disparity")
        times.append(time.perf_counter() - t0)
    px = band.shape[0] * W
    ms = 1000 * statistics.mean(times)
    value = px / (ms / 1000) / 1e6
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "each step: rows 0-%d of one 1920x1080 frame" % (
                band.shape[0] - 1)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "rows 0-%d of one 1920x1080 frame, k=31" % (band.shape[0] - 1)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="few steps, no extras (for ncu)")
    ap.add_argument("--case", default=None, choices=["single1080", "diff16", "vga", "mixed", "tolerance"],
                    help="small profiling case instead of the benchmark: one 1920x1080 frame, --steps fits "
                         "(single1080), 16 x 640x480 frames fitted and differentiated --steps times (diff16), or "
                         "one 640x480 frame at k=7, --steps fits through the C ABI (vga), or the 64-frame "
                         "mixed batch run --steps times (mixed), or the benchmark batch in precision mode 1 "
                         "(tolerance)")
    ap.add_argument("--window", type=int, default=9, help="window of the diff16 case")
    ap.add_argument("--method", default="disparity", choices=["disparity", "standard"])
    args = ap.parse_args()
    if args.case == "single1080":
        run_single_case(args)
        return
    if args.case == "diff16":
        run_diff_case(args)
        return
    if args.case == "vga":
        run_vga_case(args)
        return
    if args.case == "mixed":
        run_mixed_case(args)
        return
    if args.case == "tolerance":
        run_tolerance_case(args)
        return
    args.warmup = max(args.warmup, 3) if not args.profile_only else args.warmup
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    from paper_2103_06644_gb300 import SurfaceFitter

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    groups = workload_frames()
    fitters, inputs, outputs = [], [], []
    total_px = 0
    for (W, H, intr, frames) in groups:
        f = SurfaceFitter(intr.as_tuple(), W, H, K, method="disparity")
        d = torch.from_numpy(np.stack(frames)).to(dev)
        n = len(frames)
        out = (torch.empty((n, H, W, 3), device=dev), torch.empty((n, H, W), device=dev),
               torch.empty((n, H, W), device=dev))
        fitters.append(f)
        inputs.append(d)
        outputs.append(out)
        total_px += n * W * H

    def step(fs=fitters):
        for f, d, o in zip(fs, inputs, outputs):
            f.fit(d, out=o)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(nsteps, fn):
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(nsteps):
            fn()
        e1.record()
        barrier()
        return rank_max(e0.elapsed_time(e1) / nsteps, world, dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    for f in fitters:
        f.profile(True)
    sampler = ClockSampler(local, dev)
    t_region = [time.time(), 0.0]
    ms = timed(args.steps, step)
    t_region[1] = time.time()
    clocks = sampler.stop(t_region)
    prof = {}
    for f in fitters:
        for stage, (t, n) in f.profile_read().items():
            a = prof.setdefault(stage, [0.0, 0, 0])
            a[0] += t
            a[1] += n
        f.profile(False)
    # pixels processed per launch of each stage (every launch covers a whole group)
    px_per_launch = {}
    value = whole_job_rate(world, total_px, ms)
    peak, peak_kind = load_peaks()
    dom = max(prof, key=lambda s: prof[s][0])
    dom_ms, dom_n = prof[dom][0], prof[dom][1]
    launches_per_step = sum(v[1] for v in prof.values()) / max(1, args.steps)
    dom_avg_ms = dom_ms / max(1, dom_n)
    px_per_dom_launch = total_px * args.steps / max(1, dom_n)
    achieved = BYTES_PER_PIXEL * px_per_dom_launch / (dom_avg_ms / 1000.0) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64+f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames": 10, "pixels_per_step_per_gpu": total_px, "window": K,
                   "l2": "inputs (167 MB) and outputs (834 MB) larger than L2; no flush",
                   "precision_mode": 0,
                   "accuracy": "float32 solve: normal 1e-3 rad, offset 1e-4 |mu| on windows with gamma >= 1e-3; "
                               "tolerance_met_config holds it down to gamma >= 1e-6"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": recorded_traffic(dom),
                     "algorithmic_bytes_per_pixel": BYTES_PER_PIXEL,
                     "stage_ms_per_step": {s: v[0] / args.steps for s, v in prof.items()}},
        "issue_roofline": issue_roofline(dom, dom_avg_ms, clocks,
                                         torch.cuda.get_device_properties(dev).multi_processor_count),
        "path_hbm_frac": BYTES_PER_PIXEL * total_px / (ms / 1000.0) / 1e9 / peak,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clocks,
    }
    if not args.profile_only:
        # the plain (standard) algebraic fit on the same batch and GPU
        std = []
        for (W, H, intr, frames) in groups:
            std.append(SurfaceFitter(intr.as_tuple(), W, H, K, method="standard"))
        for _ in range(3):
            step(std)
        ms_std = timed(max(3, args.steps // 2), lambda: step(std))
        line["standard_fit"] = {"value": whole_job_rate(world, total_px, ms_std), "unit": UNIT,
                                "ms_per_step": ms_std, "speedup_of_disparity_form": ms_std / ms}
        # both forms at the tolerance down to gamma >= 1e-6 (precision mode 1)
        line["tolerance_met_config"] = tolerance_met_report(fitters, step, timed, world, total_px)
        std_tol = tolerance_met_report(std, lambda: step(std), timed, world, total_px, "standard")
        line["standard_fit"]["tolerance_met"] = {"value": std_tol["value"], "ms_per_step": std_tol["ms_per_step"],
                                                 "windows_refined_frac": std_tol["windows_refined_frac"],
                                                 "speedup_of_disparity_form": std_tol["ms_per_step"] /
                                                 line["tolerance_met_config"]["ms_per_step"]}
        for f in std:
            f.close()
        # the explicit fits (Eq. 15-16, Eq. 7-9) on the same batch
        expl = {}
        for method in ("explicit_disparity", "explicit_standard"):
            ef = [SurfaceFitter(intr.as_tuple(), W, H, K, method=method) for (W, H, intr, frames) in groups]
            for _ in range(3):
                step(ef)
            ms_e = timed(max(3, args.steps // 4), lambda: step(ef))
            expl[method] = {"value": whole_job_rate(world, total_px, ms_e), "unit": UNIT, "ms_per_step": ms_e}
            for f in ef:
                f.close()
        line["explicit_fits"] = expl
        # the disparity form on the same batch under the literal |(a,b,c,d)| = 1 constraint (row N4) and
        # with a per-pixel ray table (row N3)
        nxt = {}
        for name in ("unit4", "delta_table"):
            fs2 = []
            for (W, H, intr, frames) in groups:
                f2 = SurfaceFitter(intr.as_tuple(), W, H, K)
                if name == "unit4":
                    f2.set_constraint(True)
                else:
                    f2.set_delta_table(*scenes.delta_table(scenes.BASE_SEED + 600, intr, W, H))
                fs2.append(f2)
            for _ in range(3):
                step(fs2)
            ms2 = timed(max(3, args.steps // 4), lambda: step(fs2))
            nxt[name] = {"value": whole_job_rate(world, total_px, ms2), "unit": UNIT, "ms_per_step": ms2}
            for f2 in fs2:
                f2.close()
        # raw disparity input (row N3): the batch's depth as 1/8-pixel stereo disparity of a 7.5 cm baseline
        fs3, ins3 = [], []
        for (W, H, intr, frames) in groups:
            alpha = 1.0 / (8.0 * intr.fx * 0.075)
            z = np.stack(frames).astype(np.float64)
            disp = np.zeros(z.shape)
            ok = np.isfinite(z) & (z > 0)
            disp[ok] = np.round(1.0 / z[ok] / alpha)
            disp[(disp < 1) | (disp > 65535)] = 0
            f3 = SurfaceFitter(intr.as_tuple(), W, H, K, depth_type="disparity_u16")
            f3.set_disparity_model(alpha, 0.0)
            fs3.append(f3)
            ins3.append(torch.from_numpy(disp.astype(np.uint16).view(np.int16)).to(dev).view(torch.uint16))

        def step3():
            for f3, d3, o in zip(fs3, ins3, outputs):
                f3.fit(d3, out=o)

        for _ in range(3):
            step3()
        ms3 = timed(max(3, args.steps // 4), step3)
        nxt["disparity_input"] = {"value": whole_job_rate(world, total_px, ms3), "unit": UNIT, "ms_per_step": ms3,
                                  "input": "uint16 disparity, 1/Z = D / (8 fx 0.075 m)"}
        for f3 in fs3:
            f3.close()
        del ins3
        line["next_rows"] = nxt
        # 640x480, 7x7: the small single-frame case (launch-bound)
        intr = scenes.Intrinsics(525.0, 525.0, 319.5, 239.5)
        vga = torch.from_numpy(scenes.kinect_frame(scenes.BASE_SEED, intr, 640, 480)).to(dev)
        vres = {}
        for method in ("disparity", "standard"):
            fv = SurfaceFitter(intr.as_tuple(), 640, 480, 7, method=method)
            ov = (torch.empty((480, 640, 3), device=dev), torch.empty((480, 640), device=dev),
                  torch.empty((480, 640), device=dev))
            for _ in range(5):
                fv.fit(vga, out=ov)
            t = timed(50, lambda: fv.fit(vga, out=ov))
            # the C ABI with its arguments marshalled once (as a C caller makes the call): repeated calls on
            # the same buffers replay a captured CUDA graph
            from paper_2103_06644_gb300 import _native

            lib = _native.lib()
            cargs = (fv._h, 1, vga.data_ptr(), ov[0].data_ptr(), ov[1].data_ptr(), ov[2].data_ptr(), None,
                     torch.cuda.current_stream().cuda_stream)
            for _ in range(5):
                lib.sf_fit_ex(*cargs)
            t_c = timed(200, lambda: lib.sf_fit_ex(*cargs))
            # device time of one pass: CUDA events around each stage's launch
            fv.profile(True)
            for _ in range(20):
                fv.fit(vga, out=ov)
            torch.cuda.synchronize()
            dev_ms = sum(v[0] for v in fv.profile_read().values()) / 20
            fv.profile(False)
            vres[method] = {"us_per_frame": 1000 * t, "value": whole_job_rate(world, 307200, t), "unit": UNIT,
                            "us_per_frame_c_abi": 1000 * t_c, "us_per_frame_device": 1000 * dev_ms,
                            "api": "us_per_frame: SurfaceFitter.fit (Python); _c_abi: sf_fit_ex called in a loop "
                                   "with fixed arguments; _device: sum of the stages' CUDA-event times"}
            fv.close()
        line["vga_k7"] = vres
        # differentiation: 16 x 640x480 f32, k=9, loss = sum |n - n*|^2 + 0.1 kappa over valid pixels;
        # one step = forward + upstream gradient + backward to the depth
        nd = 16
        dd = torch.from_numpy(np.stack([scenes.kinect_frame(scenes.BASE_SEED + 600 + i, intr, 640, 480)
                                        for i in range(nd)])).to(dev)
        tgt = torch.from_numpy(np.stack([scenes.target_normals(scenes.BASE_SEED + 700 + i, 480, 640)
                                         for i in range(nd)]).astype(np.float32)).to(dev)
        fd = SurfaceFitter(intr.as_tuple(), 640, 480, 9, method="disparity")
        zero = torch.zeros((nd, 480, 640), device=dev)

        def diff_step():
            n_, o_, c_ = fd.fit(dd)
            valid = torch.isfinite(o_)
            gn = torch.where(valid[..., None], 2.0 * (n_ - tgt), torch.zeros_like(n_))
            gk = torch.where(valid, torch.full_like(c_, 0.1), torch.zeros_like(c_))
            # the depth is the one just fitted: the backward may reuse that fit's row pass
            return fd.backward(dd, gn, zero, gk, after_fit=True)

        for _ in range(3):
            diff_step()
        t_fb = timed(20, diff_step)
        t_f = timed(20, lambda: fd.fit(dd))
        fd.close()
        # the same step with 31 x 31 windows (the box sums of the backward are O(1) per pixel)
        fd = SurfaceFitter(intr.as_tuple(), 640, 480, 31, method="disparity")
        for _ in range(3):
            diff_step()
        t_fb31 = timed(10, diff_step)
        t_f31 = timed(10, lambda: fd.fit(dd))
        line["mixed_batch"] = mixed_batch_report(dev, timed, world)
        line["segmentation_512x424"] = segmentation_report(dev, timed, world)
        line["differentiation_k9"] = {"workload": "16x640x480 f32, k=9, loss |n-n*|^2 + 0.1 kappa; the backward "
                                                  "reuses the fit's row pass (SF_BACKWARD_AFTER_FIT)",
                                      "value": whole_job_rate(world, nd * 307200, t_fb), "unit": UNIT,
                                      "ms_per_step_fwd_bwd": t_fb, "ms_forward": t_f,
                                      "k31": {"value": whole_job_rate(world, nd * 307200, t_fb31), "unit": UNIT,
                                              "ms_per_step_fwd_bwd": t_fb31, "ms_forward": t_f31}}
        fd.close()
    if not args.no_e2e and not args.profile_only:
        # inputs and caller-owned result arrays in pinned (page-locked) host memory, reused every step
        # (as a streaming user would); the copies run as DMA and the two directions overlap
        def pinned(shape, dtype=np.float32):
            return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()

        host = []
        for (_, _, _, frames) in groups:
            h = pinned((len(frames),) + frames[0].shape)
            h[...] = np.stack(frames)
            host.append(h)
        hout = [(pinned(h.shape + (3,)), pinned(h.shape), pinned(h.shape)) for h in host]
        for f, h, o in zip(fitters, host, hout):
            f.fit_host(h, out=o)  # device staging, and the first touch of the result pages
        # the two resolution groups are independent contexts: their calls run on two host threads
        # (the binding releases the GIL), so one group's copies overlap the other's
        from concurrent.futures import ThreadPoolExecutor

        pool = ThreadPoolExecutor(len(fitters))

        def e2e_step():
            for fut in [pool.submit(f.fit_host, h, False, o) for f, h, o in zip(fitters, host, hout)]:
                fut.result()

        def e2e_step_sequential():
            for f, h, o in zip(fitters, host, hout):
                f.fit_host(h, out=o)

        e2e_step()
        e2e_step_sequential()
        # the two ways of calling, in three alternating rounds of ne steps (the host link's rate varies
        # from moment to moment): each one's median round, and the faster of the two as the e2e figure
        ne = 10
        rounds = {"concurrent": [], "sequential": []}
        for _ in range(3):
            for name, fn in (("concurrent", e2e_step), ("sequential", e2e_step_sequential)):
                barrier()
                t0 = time.perf_counter()
                for _ in range(ne):
                    fn()
                rounds[name].append(rank_max((time.perf_counter() - t0) / ne, world, dev))
        pool.shutdown()
        res = {name: sorted(v)[len(v) // 2] for name, v in rounds.items()}
        best = min(res, key=res.get)
        dt = res[best]
        calls = {"concurrent": "the two resolution groups' calls on two host threads",
                 "sequential": "the two resolution groups' calls one after the other"}
        line["e2e"] = {"value": whole_job_rate(world, total_px, 1000 * dt), "unit": UNIT,
                       "h2d_bytes_per_step": int(sum(h.nbytes for h in host)),
                       "d2h_bytes_per_step": int(20 * total_px), "ms_per_step": 1000 * dt,
                       "ms_per_step_two_threads": 1000 * res["concurrent"],
                       "ms_per_step_one_after_the_other": 1000 * res["sequential"],
                       "api": "sf_fit_host (pinned host buffers, copies inside the call, result arrays reused; "
                              + calls[best] + "; median of 3 rounds of %d steps)" % ne}
        # the same with ordinary pageable numpy arrays
        host_p = [np.array(h) for h in host]
        hout_p = [tuple(np.empty_like(a) for a in o) for o in hout]
        for f, h, o in zip(fitters, host_p, hout_p):
            f.fit_host(h, out=o)
        pool = ThreadPoolExecutor(len(fitters))
        barrier()
        t0 = time.perf_counter()
        for _ in range(ne):
            for fut in [pool.submit(f.fit_host, h, False, o) for f, h, o in zip(fitters, host_p, hout_p)]:
                fut.result()
        dtp = rank_max((time.perf_counter() - t0) / ne, world, dev)
        pool.shutdown()
        line["e2e"]["pageable"] = {"value": whole_job_rate(world, total_px, 1000 * dtp), "ms_per_step": 1000 * dtp}
    if rank == 0 and world == 1 and not args.no_cpu and not args.profile_only:
        line["cpu_baseline"] = cpu_oracle_sample()
        try:
            line["precision_vs_oracle"] = precision_report(groups[0], dev)
        except Exception as exc:  # a report failure must not lose the benchmark line
            line["precision_vs_oracle"] = {"error": repr(exc)}
    if rank == 0:
        # the rows read most often go last, where a truncated log still shows them
        tail = ["explicit_fits", "segmentation_512x424", "vga_k7", "tolerance_met_config", "standard_fit",
                "differentiation_k9", "mixed_batch", "next_rows"]
        ordered = {k: v for k, v in line.items() if k not in tail}
        ordered.update((k, line[k]) for k in tail if k in line)
        print(json.dumps(ordered), flush=True)
    for f in fitters:
        f.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
