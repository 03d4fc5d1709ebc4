"""Benchmark: frames/s of the virtual-memory 3DGS per-frame path.

A step is one frame: page determination (visibility buffer + reduction) ->
page-table update with host->pool streaming -> render of the resident
Gaussians, for one camera of a seeded flythrough.  Two arms on the same scene
and path:
  plain     fp32 page pool, copies in line with the frame (the paper's
            synchronous transfers)
  headline  fp16 page pool, copies on a separate copy stream
`value` is the headline arm's whole-job frames/s; `plain_vm` carries the plain
arm.  Default workload: 50M Gaussians on a 2 km x 2 km city (5,000 boxes),
SH degree 3, pages of 4096 with 3 LOD levels, whole scene in page-locked host
memory, 2 GiB device pool, 1000-frame walking-speed flythrough at 1920x1080.
Synthetic, seeded inputs (scenegen); no dataset.

  python bench.py [--gpus N --steps K --warmup W] [--config city50m|blobs1m|tiny]
  python bench.py --impl reference ...   (the CPU oracle, bounded sample)
  python bench.py --table pagesize|buffer (the page-size / buffer-size tables of Sec. 5)
  python bench.py --table lod            (k-means LOD against moment matching: time and PSNR)
  python bench.py --table disk           (the scene from a memory-mapped file through a staging buffer)
  python bench.py --table quality        (page links x LOD ablation on a 500-page buffer: PSNR / SSIM, Sec. 5.2)
  python bench.py --table vq             (compressed pages: SH codebook against the fp16 pool)
  python bench.py --table fade           (LOD cross-fade: its cost along the walk)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


# ----------------------------------------------------------------------------- workloads
def workload(name):
    import scenegen
    if name == "city50m":
        ext = 2000.0
        return dict(
            name="city 50M Gaussians, 2 km x 2 km, 5000 boxes, SH3, pages 4096 x 3 LOD (fanout 8), 2 GiB pool, "
                 "1080p walking flythrough",
            gen=lambda: scenegen.city_scene(n=50_000_000, n_boxes=5000, extent=ext),
            build=dict(page_size=4096, paging="octree", lod_levels=3, lod_fanout=8, lo=(-4, -4, -4),
                       hi=(ext + 4, ext + 4, 88), voxel=2.0, kappa=0.5, link_samples=4, fp16=True),
            path=lambda n: scenegen.city_walk_path(n_frames=n),
            train_path=lambda n, seed: scenegen.city_walk_path(n_frames=n, seed=seed),
            frames=1000, pool_bytes=2 << 30, lod=True, gaussians=50_000_000,
            sample=dict(extent=150.0, n=int(50_000_000 * (150.0 / ext) ** 2), n_boxes=max(1, int(5000 * (150.0 / ext) ** 2))))
    if name == "citypatch":
        ext = 1000.0
        return dict(
            name="city patch 12.5M Gaussians, 1 km x 1 km, 1250 boxes, SH3, pages 4096 x 3 LOD, 512 MiB pool, 1080p "
                 "walking flythrough (profiling size)",
            gen=lambda: scenegen.city_scene(n=12_500_000, n_boxes=1250, extent=ext),
            build=dict(page_size=4096, paging="octree", lod_levels=3, lod_fanout=8, lo=(-4, -4, -4),
                       hi=(ext + 4, ext + 4, 88), voxel=2.0, kappa=0.5, link_samples=4, fp16=True),
            path=lambda n: scenegen.city_walk_path(n_frames=n, n_boxes=1250, extent=ext),
            train_path=lambda n, seed: scenegen.city_walk_path(n_frames=n, seed=seed, n_boxes=1250, extent=ext),
            frames=1000, pool_bytes=512 << 20, lod=True, gaussians=12_500_000, sample=None)
    if name == "blobs1m":
        return dict(
            name="1M Gaussians in 200 blobs (sigma 0.5 m) in a 50 m cube, SH3, octree pages 4096, 64 MiB pool, 1080p "
                 "orbit + flythrough",
            gen=lambda: scenegen.blob_scene(n=1_000_000),
            build=dict(page_size=4096, paging="octree", lod_levels=1, lo=(-5, -5, -5), hi=(55, 55, 55),
                       voxel=60.0 / 64, kappa=2.0, link_samples=4, fp16=True),
            path=lambda n: scenegen.orbit_fly_path(n_frames=n),
            train_path=lambda n, seed: scenegen.random_fly_path(n, seed=seed, speed=0.5),
            frames=300, pool_bytes=64 << 20, lod=False, gaussians=1_000_000, sample=None)
    if name == "tiny":
        return dict(
            name="16,384 Gaussians uniform in a 10 m cube, SH0, 64 Morton pages of 256, all resident, 256x256",
            gen=lambda: scenegen.uniform_scene(),
            build=dict(page_size=256, paging="morton", lo=(-5, -5, -5), hi=(5, 5, 5), voxel=10 / 32, kappa=0.5,
                       link_samples=8, fp16=True),
            path=lambda n: [scenegen.tiny_camera()] * n,
            frames=1, pool_bytes=None, lod=False, gaussians=16384, sample=None)
    raise SystemExit("unknown config " + name)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """SM clock and throttle reasons sampled through NVML every `period` s
    in a background thread while it runs, plus one sample at start and one
    at stop, so even a timed region of a few milliseconds has samples."""
    REASONS = (("hw_slowdown", 0x8), ("hw_thermal_slowdown", 0x40), ("sw_thermal_slowdown", 0x20),
               ("sw_power_cap", 0x4), ("hw_power_brake_slowdown", 0x80))

    def __init__(self, index, period=0.002):
        self.index, self.period, self.rows, self.h, self.t = index, period, [], None, None
        self.stop_flag = threading.Event()
        self.err = ""
        try:
            self._open_ctypes(index)
        except Exception as e:  # noqa: BLE001 (no NVML: reported in the line)
            self.err = str(e)
            self.h = None

    def _open_ctypes(self, index):
        """NVML's C library (read-only queries: clocks and their reasons)."""
        import ctypes
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        h = ctypes.c_void_p()
        if nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(h)) != 0:
            raise RuntimeError("no NVML handle for device %d" % index)
        reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        self.nv, self.h, self.reasons_fn, self.ct = nv, h, reasons, ctypes

    def _smi_sample(self):
        """One nvidia-smi query (when NVML's library cannot be opened)."""
        q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active"
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10).stdout
            sm, mx, act = [x.strip() for x in out.strip().split(",")[:3]]
            self.rows.append((int(float(sm)), int(float(mx)), int(act, 16)))
        except (OSError, ValueError, subprocess.SubprocessError):
            pass

    def _sample(self):
        if self.h is None:
            return self._smi_sample()
        ct, nv, h = self.ct, self.nv, self.h
        sm, mx, rs_ = ct.c_uint(0), ct.c_uint(0), ct.c_ulonglong(0)
        nv.nvmlDeviceGetClockInfo(h, ct.c_int(1), ct.byref(sm))      # NVML_CLOCK_SM = 1
        nv.nvmlDeviceGetMaxClockInfo(h, ct.c_int(1), ct.byref(mx))
        self.reasons_fn(h, ct.byref(rs_))
        self.rows.append((int(sm.value), int(mx.value), int(rs_.value)))

    def _loop(self):
        while not self.stop_flag.wait(self.period):
            self._sample()

    def start(self):
        self.rows = []
        self.stop_flag.clear()
        self._sample()
        if self.h is not None:
            self.t = threading.Thread(target=self._loop, daemon=True)
            self.t.start()

    def stop(self):
        if self.h is not None:
            self.stop_flag.set()
            self.t.join()
        self._sample()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no clock source: " + self.err], "samples": 0}
        sm = [r[0] for r in self.rows]
        reasons = sorted({name for r in self.rows for name, bit in self.REASONS if r[2] & bit})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in self.rows),
                "sm_mhz_min": min(sm), "reasons": reasons, "samples": len(self.rows),
                "how": ("NVML every %.0f ms during the timed frames" % (1e3 * self.period)) if self.h is not None
                else "nvidia-smi at the start and end of the timed frames (NVML library unavailable)"}


# ----------------------------------------------------------------------------- GPU arm
def build_scene(W):
    import paper_2506_19415_b300 as v
    t0 = time.time()
    raw = W["gen"]()
    t1 = time.time()
    scene = v.vm3dgs_build_pages(raw, v.BuildConfig(**W["build"], seed=77))
    del raw
    return scene, t1 - t0, time.time() - t1


def make_renderer(v, scene, W, fp16, width, height, pool_slots=None, max_pairs=0, sort_mode=0):
    cfg = v.RenderConfig(staging_bytes=40 * 2048 * 236, feedback_ds=4, links=True, lod=W["lod"], fp16_pool=fp16,
                         max_width=width, max_height=height, tau0=1.0, step0=0.1, max_pairs=max_pairs,
                         sort_mode=sort_mode)
    if pool_slots is not None:
        return v.Renderer(scene, cfg, pool_slots=pool_slots)
    if W["pool_bytes"] is None:
        return v.Renderer(scene, cfg, pool_slots=scene.info.n_pages)
    return v.Renderer(scene, cfg, pool_bytes=W["pool_bytes"])


def quality_eval(v, scene, W, cams, every=25, frames=150):
    """PSNR of the fp16 pool's images against the fp32 pool's (equal pool
    bytes) along the first frames of the walk, both renderers from a cold
    start on one stream; and the cold first frame's time."""
    import torch
    width, height = cams[0].width, cams[0].height
    rs = [make_renderer(v, scene, W, fp16, width, height) for fp16 in (False, True)]
    st = torch.cuda.current_stream()
    imgs = [torch.empty((3, height, width), dtype=torch.float32, device="cuda") for _ in rs]
    psnr, cold = [], []
    for k, r in enumerate(rs):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r.render_feedback([cams[0]], st)
        r.update_residency(st)
        r.render([cams[0]], [imgs[k]], st)
        e1.record(st)
        torch.cuda.synchronize()
        cold.append(round(e0.elapsed_time(e1), 3))
    for f in range(1, frames + 1):
        for k, r in enumerate(rs):
            r.render_feedback([cams[f]], st)
            r.update_residency(st)
            r.render([cams[f]], [imgs[k]], st)
        if f % every == 0:
            a, b = (im.clamp(0.0, 1.0).double() for im in imgs)
            mse = float(((a - b) ** 2).mean())
            psnr.append(round(10.0 * math.log10(1.0 / max(mse, 1e-30)), 2))
    st32, st16 = rs[0].stats(st), rs[1].stats(st)
    del rs
    torch.cuda.empty_cache()
    return {"psnr_fp16_vs_fp32_db": psnr, "min_psnr_db": min(psnr), "frames": [f for f in range(every, frames + 1, every)],
            "same_draw_list": st32["drawn_gaussians"] == st16["drawn_gaussians"],
            "cold_first_frame_ms": {"fp32": cold[0], "fp16": cold[1]},
            "note": "fp16 and fp32 pools of equal bytes, cold start, one stream; images clamped to [0, 1]"}


def train_prefetcher(v, scene, W, width, height, n_paths=16, frames=60, steps=600):
    """The learned prefetcher for this scene, trained on the renderer's own
    feedback over seeded walks that do not include the benchmark path."""
    from paper_2506_19415_b300 import prefetch_train as ptr
    import torch
    n_out = 4096 if scene.info.n_pages >= 4096 else max(16, (scene.info.n_pages + 15) // 16 * 16)
    r = make_renderer(v, scene, W, True, width, height)
    paths = [W["train_path"](frames, 3000 + k) for k in range(n_paths)]
    t0 = time.time()
    X, Y, M = ptr.make_dataset(v, r, paths, n_out, 12 + n_out // 16, horizon=15)
    p = v.Prefetcher(v.MlpShape(n_in=12 + n_out // 16, n_hidden=256, n_out=n_out, max_batch=256, seed=5, lr=1e-3))
    curve = ptr.train(p, X, Y, M, steps=steps, batch=256)
    del X, Y, M, r
    torch.cuda.empty_cache()
    return p, {"train_paths": n_paths, "frames_per_path": frames, "steps": steps, "window_pages": n_out,
               "label_horizon_frames": 15, "prefetch_every_frames": PREFETCH_EVERY,
               "loss_first": round(curve[0], 4), "loss_last": round(curve[-1], 4), "seconds": round(time.time() - t0, 1)}


PREFETCH_EVERY = 4   # frames between prefetch steps (the network predicts the next 15 frames' pages)


# Frames of the walk rendered untimed before an arm's warm-up frames, so that
# the timed frames see the warm pool of a running walk (the cold fill of the
# first frame is reported separately under "quality").
PREROLL = 60


def run_arm(v, r, cams, warmup, steps, copy_stream=None, e2e=False, timing=False, dist=None, pf=None, pf_thr=0.0,
            serial=False, clocks=None, preroll=0):
    import torch
    dev = torch.device("cuda")
    st = torch.cuda.current_stream()
    H, W = cams[0].height, cams[0].width
    # NB image buffers: with e2e, frame i's image goes to pinned host memory
    # on its own stream while the next frames render into the other buffers
    NB = 4
    images = [torch.empty((3, H, W), dtype=torch.float32, device=dev) for _ in range(NB)]
    hosts = [torch.empty((3, H, W), dtype=torch.float32, pin_memory=True) for _ in range(NB)] if e2e else None
    d2h = torch.cuda.Stream() if e2e else None
    # page determination (a frame ahead, on the double-buffered request
    # words) and the page-table update of frame i+1 run on their own streams
    # while frame i renders, and consecutive frames render on two streams (the
    # renderer's two render contexts): the renderer orders them with events
    # (update after the previous projection, render after the update, a
    # buffer's or context's reuse after its last reader)
    fbst, fst = torch.cuda.Stream(), torch.cuda.Stream()
    rst = [st, torch.cuda.Stream()]
    if serial:  # every call on one stream: each kernel's time is its own (roofline)
        fbst = fst = rst[0] = rst[1] = st
    copied = [torch.cuda.Event() for _ in range(NB)] if e2e else None
    rendered = [torch.cuda.Event() for _ in range(NB)] if e2e else None
    n = len(cams)

    def frame(i):
        c = [cams[i % n]]
        b = i % NB
        rs = rst[i & 1]
        r.render_feedback(c, fbst)
        r.update_residency(fst, copy_stream)
        if e2e:
            rs.wait_event(copied[b])   # the copy of frame i-NB out of this buffer is done
        r.render(c, [images[b]], rs)
        if pf is not None:
            if i % PREFETCH_EVERY == 0:
                v.vm3dgs_prefetch(r, pf, c[0], cams[(i - 1) % n], pf_thr, rs, copy_stream)
        if e2e:
            rendered[b].record(rs)
            d2h.wait_event(rendered[b])
            with torch.cuda.stream(d2h):
                hosts[b].copy_(images[b], non_blocking=True)
            copied[b].record(d2h)

    for i in range(preroll + warmup):
        frame(i)
    torch.cuda.synchronize()
    r.reset_sums(st)
    if timing:
        r.timing(True)
        r.timing_read()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks is not None:
        clocks.start()
    t_wall = time.perf_counter()
    e0.record(st)
    for i in range(preroll + warmup, preroll + warmup + steps):
        frame(i)
    issue = time.perf_counter() - t_wall  # host time to enqueue the frames
    if e2e:
        st.wait_stream(d2h)   # the last image is on the host before the clock stops
    st.wait_stream(rst[1])
    st.wait_stream(fst)
    st.wait_stream(fbst)
    e1.record(st)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop() if clocks is not None else None
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    stage = r.timing_read() if timing else None
    if timing:
        r.timing(False)
    stats = r.stats(st)
    return dict(ms=ms, wall=wall, issue=issue, stage=stage, stats=stats, clocks=clk)


# DRAM bytes per sort pass per sorted pair, from an ncu capture of the
# current sort kernel (dram__bytes_read.sum + dram__bytes_write.sum of one
# launch over the profiling workload divided by its pairs and passes); None
# until a capture of the current kernel exists.
SORT_DRAM_BYTES_PER_PAIR_PASS = None

# The blend's binding bound is instruction issue, not memory: the pipe
# utilisation of one blend launch from an ncu --set full capture (1M-Gaussian
# city at 1080p, fp16 pool, the full-size parity test's frame 1), which the
# bench cannot read live.
BLEND_ISSUE = {"issue_active_pct": 77.1, "alu_pipe_pct": 51.7, "fma_pipe_pct": 33.8, "dram_pct_of_peak": 1.6,
               "source": "ncu --set full, one launch (smsp__issue_active, sm__pipe_alu_cycles_active, "
                         "sm__pipe_fma_cycles_active, gpu__dram_throughput), of the kernel before its two-splat walk"}


def roofline(v, stage, stats, peaks, rec16, width, height, alt_sort=None):
    """Roofline of the dominant kernel (the radix sort) and of the gather
    (projection) and blend kernels, from the CUDA-event spans of the timed
    frames: algorithmic bytes per launch / mean launch time.  The sort moves
    every 8-byte packed key in and out once per pass (16 B per pair per pass);
    one cooperative launch runs all of a view's passes."""
    ms, launches = stage
    names = v.STAGES
    frames = max(stats["acc_frames"], 1)
    views = max(stats["acc_views"], 1)
    pairs = stats["acc_pairs"] / views              # per view
    gauss = stats["acc_drawn_gaussians"] / frames   # per frame
    peak = peaks.get("hbm_gbs", 6400.0)
    passes = -(-(stats["key_tile_bits"] + stats["key_depth_bits"]) // 8)

    def per_launch_s(stage_name, n):
        return ms[names.index(stage_name)] / max(n, 1) / 1e3

    sort_launches = launches[names.index("sort")]
    per_view = sort_launches / views
    kern = {
        "sort": (pairs * 16 * passes / max(per_view, 1), per_launch_s("sort", sort_launches),
                 "16 B per pair per pass (8 B key read + written) x %d passes / %g launches per view" %
                 (passes, per_view)),
        # pool record (fp16) read + 64 B of splat outputs written per drawn Gaussian
        "project": (gauss * (rec16 + 64), per_launch_s("project", frames),
                    "%d B record read + 64 B splat record written per drawn Gaussian" % rec16),
        # per pair: 8 B key + 36 B splat (s0, s1, s2) read; 12 B image written per pixel
        "blend": (pairs * 44 + width * height * 12, per_launch_s("blend", views),
                  "44 B per pair read + 12 B per pixel written"),
    }
    detail = {}
    for k, (b, t, note) in kern.items():
        a = b / t / 1e9 if t > 0 else 0.0
        detail[k] = {"achieved": round(a, 1), "frac": round(a / peak, 4), "us_per_launch": round(t * 1e6, 2),
                     "algorithmic_bytes_per_launch": int(b), "per_unit": note}
    detail["blend"]["alu"] = BLEND_ISSUE
    if alt_sort is not None:
        detail["sort_cooperative"] = alt_sort
    coop = per_view < passes
    traffic = None if SORT_DRAM_BYTES_PER_PAIR_PASS is None else \
        int(SORT_DRAM_BYTES_PER_PAIR_PASS * pairs * passes / max(per_view, 1))
    out = {"bound": "hbm",
           "kernel": ("coop_sort_kernel (all %d passes in one cooperative launch)" % passes) if coop
           else "onesweep_kernel (one sort pass)",
           "achieved": detail["sort"]["achieved"], "peak": peak, "unit": "GB/s", "frac": detail["sort"]["frac"],
           "traffic": traffic,
           "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6400 GB/s",
           "passes_per_view": passes, "sort_launches_per_view": per_view, "kernels": detail,
           "stage_ms": {names[i]: round(ms[i], 3) for i in range(len(ms))},
           "stage_launches": {names[i]: int(launches[i]) for i in range(len(ms))},
           "note": ("blend's inputs (sorted keys and splats, < 126 MB) stay in L2 and it is bound by FP32/ALU issue, "
                    "so its HBM fraction is low by construction")}
    return out


def coop_sort_reference(v, scene, W, cams, warmup, steps, copy_stream, dist, pf, width, height, peaks):
    """The same single-stream frames with the cooperative sort (all passes
    in one launch): its time per view and HBM fraction beside the onesweep
    sort's (the default)."""
    rn = make_renderer(v, scene, W, True, width, height, sort_mode=1)
    res = run_arm(v, rn, cams, warmup, steps, copy_stream, timing=True, dist=dist, pf=pf, serial=True,
                  preroll=PREROLL)
    ms, launches = res["stage"]
    st = res["stats"]
    views = max(st["acc_views"], 1)
    i = v.STAGES.index("sort")
    passes = -(-(st["key_tile_bits"] + st["key_depth_bits"]) // 8)
    t = ms[i] / max(launches[i], 1) / 1e3
    b = st["acc_pairs"] / views * 16 * passes * views / max(launches[i], 1)
    a = b / t / 1e9 if t > 0 else 0.0
    del rn
    return {"us_per_launch": round(t * 1e6, 2), "launches_per_view": launches[i] / views,
            "sort_ms_per_view": round(ms[i] / views, 4), "achieved": round(a, 1),
            "frac": round(a / peaks.get("hbm_gbs", 6400.0), 4), "ms_per_step_one_stream": round(res["ms"] / steps, 4),
            "kernel": "coop_sort_kernel (sort_mode 1)"}


def prefetch_eval(v, n_train=50, n_test=10, frames=300, turn_every=30, steps=1200):
    """The learned-prefetch configuration as stated: the 1M-Gaussian blob
    scene (SH3, octree pages of 4096), a 64 MiB fp32 pool (69 page slots
    against about 245 pages), the paper's 18.4 MiB staging budget, 1920x1080;
    the MLP 12 + 256 -> 256 -> 256 -> 4096 (one logit per page of a 4096-page
    window, BF16 weights, FP32 accumulation) trained on the renderer's own
    feedback over n_train seeded random flythroughs of `frames` frames (every
    other one with an abrupt 90 degree turn every `turn_every` frames; labels:
    the pages requested within the next 15 frames), evaluated on n_test
    held-out flythroughs with an abrupt 90 degree turn every `turn_every`
    frames: page misses per frame and the per-frame time of the page copies
    a frame waits for (stall), with and without the prefetcher."""
    import torch
    from paper_2506_19415_b300 import prefetch_train as ptr
    W2 = workload("blobs1m")
    raw = W2["gen"]()
    scene = v.vm3dgs_build_pages(raw, v.BuildConfig(**W2["build"], seed=77))
    del raw
    n_out, Wd, Hd = 4096, 1920, 1080
    cfg = v.RenderConfig(max_width=Wd, max_height=Hd, lod=False, staging_bytes=STAGING, fp16_pool=False)
    rr = v.Renderer(scene, cfg, pool_bytes=64 << 20)
    slots = rr.n_slots
    t0 = time.time()
    train = [scenegen_fly(frames, 2000 + k, turn_every if k % 2 else 0) for k in range(n_train)]
    test = [scenegen_fly(frames, 9000 + k, turn_every) for k in range(n_test)]
    X, Y, M = ptr.make_dataset(v, rr, train, n_out, 12 + n_out // 16, horizon=15)
    t_data = time.time() - t0
    p = v.Prefetcher(v.MlpShape(n_in=12 + n_out // 16, n_hidden=256, n_out=n_out, max_batch=256, seed=4, lr=1e-3))
    t0 = time.time()
    curve = ptr.train(p, X, Y, M, steps=steps, batch=256)
    t_train = time.time() - t0
    n_samples = X.shape[0]
    del X, Y, M, rr
    torch.cuda.empty_cache()
    cs = torch.cuda.Stream()
    a = ptr.evaluate(v, v.Renderer(scene, cfg, pool_bytes=64 << 20), test, None, copy_stream=cs)
    b = ptr.evaluate(v, v.Renderer(scene, cfg, pool_bytes=64 << 20), test, p, threshold=-1.0, copy_stream=cs)
    r4 = lambda d: {k: (round(x, 4) if isinstance(x, float) else x) for k, x in d.items()}
    return {"workload": "1M-Gaussian blob scene (config 2), pages of 4096 (%d pages), 64 MiB fp32 pool (%d slots), "
                        "18.4 MiB staging budget, 1920x1080; MLP 268-256-256-4096" % (scene.info.n_pages, slots),
            "train": "%d flythroughs x %d frames (%d samples; half with a 90 deg turn every %d frames), %d Adam steps "
                     "of 256, %.1f s dataset + %.1f s training" % (n_train, frames, n_samples, turn_every, steps,
                                                                  t_data, t_train),
            "test": "%d held-out flythroughs x %d frames, abrupt 90 deg turn every %d frames" % (n_test, frames,
                                                                                           turn_every),
            "loss_first_last": [round(curve[0], 4), round(curve[-1], 4)], "feedback_only": r4(a),
            "with_prefetcher": r4(b),
            "miss_reduction": round(1.0 - b["misses_per_frame"] / max(a["misses_per_frame"], 1e-9), 4),
            "stall_reduction": round(1.0 - b["stall_ms_per_frame"] / max(a["stall_ms_per_frame"], 1e-9), 4)}


def scenegen_fly(n, seed, turn_every):
    import scenegen
    return scenegen.random_fly_path(n, seed=seed, lo=0.0, hi=50.0, speed=0.25, turn_every=turn_every)


def batched_views_eval(v, reps=5):
    """64 cameras of uneven resolution (512x512 .. 1920x1080, fov 40-90 deg)
    on the 1M-Gaussian blob scene sharing one 64 MiB fp16 pool: views/s of 64
    sequential single-view renders vs the autotuned, graph-captured batch."""
    import scenegen
    import torch
    W2 = workload("blobs1m")
    raw = W2["gen"]()
    scene = v.vm3dgs_build_pages(raw, v.BuildConfig(**W2["build"], seed=77))
    del raw
    cams = scenegen.batched_views(n_views=64)
    cfg = v.RenderConfig(staging_bytes=64 << 20, lod=False, fp16_pool=True, max_width=1920, max_height=1080,
                         max_views=64, max_pairs=1 << 27)
    r = v.Renderer(scene, cfg, pool_bytes=64 << 20)
    st = torch.cuda.current_stream()
    r.render_feedback(cams, st)
    r.update_residency(st)
    images = [torch.empty((3, c.height, c.width), dtype=torch.float32, device="cuda") for c in cams]
    for _ in range(2):
        for k, c in enumerate(cams):
            r.render([c], [images[k]], st)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        for k, c in enumerate(cams):
            r.render([c], [images[k]], st)
    e1.record(st)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1) / reps
    t0 = time.time()
    tuned = r.autotune_tiles(cams, images, repeats=3)
    tune_s = time.time() - t0
    shapes = {}
    for c in tuned:
        shapes["%dx%d" % (c.tile_w, c.tile_h)] = shapes.get("%dx%d" % (c.tile_w, c.tile_h), 0) + 1
    r.render_batched(tuned, images, st)
    s = torch.cuda.Stream()
    s.wait_stream(st)
    with torch.cuda.stream(s):
        r.batch_graph_capture(tuned, images, s)
        for _ in range(2):
            r.batch_graph_launch(tuned, s)
    s.synchronize()
    e0.record(s)
    for _ in range(reps):
        r.batch_graph_launch(tuned, s)
    e1.record(s)
    s.synchronize()
    batch_ms = e0.elapsed_time(e1) / reps
    st_ = r.stats(st)
    pix = sum(c.width * c.height for c in cams)
    return {"workload": "64 views 512x512..1920x1080 (%.1f Mpx), fov 40-90 deg, 1M-Gaussian blob scene, shared 64 MiB "
                        "fp16 pool" % (pix / 1e6),
            "views_per_s_batched_graph": round(64 / (batch_ms / 1e3), 1),
            "views_per_s_sequential": round(64 / (seq_ms / 1e3), 1),
            "ms_batch": round(batch_ms, 3), "ms_sequential": round(seq_ms, 3), "tile_shapes": shapes,
            "autotune_s": round(tune_s, 2), "pairs_per_batch": st_["pairs"], "status": st_["status"]}


def aggregate_ranks(ms_list, steps, world, dist=None, device="cpu"):
    """Replicas only: every rank renders `steps` frames of its own; the job's
    time is the slowest rank's (max over ranks) and the job's frames/s counts
    the frames of all ranks.  Returns (max ms per entry, frames/s per entry)."""
    import torch
    t = torch.tensor(ms_list, dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = [float(x) for x in t.tolist()]
    return ms, [world * steps / (m / 1e3) for m in ms]


def gpu_main(args):
    import torch
    import paper_2506_19415_b300 as v
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    W = workload(args.config)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    scene, t_gen, t_build = build_scene(W)
    n_frames = W["frames"]
    cams = W["path"](n_frames)
    if rank:
        cams = cams[rank % len(cams):] + cams[:rank % len(cams)]
    width, height = cams[0].width, cams[0].height
    K = (scene.info.sh_degree + 1) ** 2
    # plain arm
    rp = make_renderer(v, scene, W, False, width, height)
    plain = run_arm(v, rp, cams, args.warmup, args.steps, None, dist=dist, preroll=PREROLL,
                    clocks=ClockSampler(torch.cuda.current_device()))
    del rp
    torch.cuda.empty_cache()
    # headline arm: fp16 pool, copies on a copy stream, learned prefetch
    pf, pf_info = (None, None)
    if W.get("train_path") is not None and not args.no_prefetch:
        pf, pf_info = train_prefetcher(v, scene, W, width, height)
    rh = make_renderer(v, scene, W, True, width, height)
    copy_stream = torch.cuda.Stream()
    head = run_arm(v, rh, cams, args.warmup, args.steps, copy_stream, dist=dist, pf=pf, preroll=PREROLL,
                   clocks=ClockSampler(torch.cuda.current_device()))
    # the same frames with every call on one stream: per-kernel CUDA-event
    # times without the other streams' kernels sharing the GPU, for the roofline
    ser = run_arm(v, rh, cams, args.warmup, min(args.steps, 100), copy_stream, timing=True, dist=dist, pf=pf,
                  serial=True, preroll=PREROLL)
    clk = head["clocks"]
    # end to end through the public API: the rendered image returns to pinned host memory every frame
    e2e = run_arm(v, rh, cams, args.warmup, args.steps, copy_stream, e2e=True, dist=dist, pf=pf, preroll=PREROLL)
    # same fp16 arm without the prefetcher, for its misses and copy stall
    nopf = None
    if pf is not None:
        rn = make_renderer(v, scene, W, True, width, height)
        nopf = run_arm(v, rn, cams, args.warmup, min(args.steps, 100), copy_stream, timing=True, dist=dist,
                       serial=True, preroll=PREROLL)
        del rn
    # fp16 pool with the fp32 arm's slot count (equal pages, half the bytes), no prefetcher
    eq = None
    if W["pool_bytes"] is not None:
        slots32 = W["pool_bytes"] // v.vm3dgs_pool_slot_bytes(scene, fp16_pool=False)
        rq = make_renderer(v, scene, W, True, width, height, pool_slots=slots32)
        eq = run_arm(v, rq, cams, args.warmup, args.steps, copy_stream, dist=dist, preroll=PREROLL)
        eq["slots"] = int(slots32)
        del rq
    torch.cuda.empty_cache()

    (ms_head, ms_plain, ms_e2e), (fps, fps_plain, fps_e2e) = aggregate_ranks(
        [head["ms"], plain["ms"], e2e["ms"]], args.steps, world, dist, "cuda")
    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    hs = head["stats"]
    frames = max(hs["acc_frames"], 1)
    # (rank 0 only: the other ranks have returned, so no barrier here)
    alt = coop_sort_reference(v, scene, W, cams, args.warmup, min(args.steps, 100), copy_stream, None, pf, width,
                              height, peaks)
    rl = roofline(v, ser["stage"], ser["stats"], peaks, scene.info.record_bytes16, width, height, alt)
    rl["timing"] = ("kernels timed by CUDA events in a single-stream pass over %d frames of the same walk "
                    "(bench.py); the timed headline loop itself records no per-stage events" % min(args.steps, 100))
    launches_per_frame = sum(ser["stage"][1]) / max(ser["stats"]["acc_frames"], 1)
    line = {
        "metric": "1080p frames/s on 50M-Gaussian scene, plain VM vs FP16+prefetch, PSNR>=45dB",
        "value": round(fps, 2),
        "unit": "frames/s",
        "plain_vm_value": round(fps_plain, 2),
        "speedup_vs_plain_vm": round(fps / fps_plain, 4),
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_head / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "storage": "f16 pool records (scale, rotation, SH); bf16 prefetcher weights",
        "data": "synthetic (seeded scenegen), no dataset",
        "config": {"workload": W["name"], "config": args.config, "gaussians": W["gaussians"],
                   "pages": scene.info.n_pages, "resolution": [width, height], "frames_in_path": n_frames,
                   "pool_bytes": W["pool_bytes"], "staging_bytes": 40 * 2048 * 236,
                   "l2": "per-frame inputs (2 GiB pool, splat and pair buffers) exceed the 126 MB L2",
                   "arm": "fp16 pool + copy stream + learned prefetch", "parallelism": "replicas, one renderer per GPU",
                   "timed_frames": [PREROLL + args.warmup, PREROLL + args.warmup + args.steps],
                   "preroll": "frames 0..%d of the walk rendered untimed before the warm-up frames (warm pool)"
                              % (PREROLL - 1),
                   "streams": "page determination and page-table update on their own streams, consecutive renders on two streams (two render contexts), event-ordered"},
        "plain_vm": {"value": round(fps_plain, 2), "unit": "frames/s", "ms_per_step": round(ms_plain / args.steps, 4),
                     "arm": "fp32 pool, in-line copies", "clocks": plain["clocks"],
                     "missing_per_frame": plain["stats"]["acc_missing"] / max(plain["stats"]["acc_frames"], 1)},
        "per_frame": {"missing": hs["acc_missing"] / frames, "requested": hs["acc_requested"] / frames,
                      "drawn_gaussians": hs["acc_drawn_gaussians"] / frames, "pairs": hs["acc_pairs"] / frames,
                      "streamed_bytes": hs["acc_streamed_bytes"] / frames, "tau": hs["tau"], "usage": hs["usage"]},
        "e2e": {"value": round(fps_e2e, 2), "unit": "frames/s", "h2d_bytes_per_step": int(76 + hs["acc_streamed_bytes"] / frames),
                "d2h_bytes_per_step": 3 * width * height * 4,
                "host_issue_ms_per_step": round(1e3 * e2e["issue"] / args.steps, 4)},
        "host_issue_ms_per_step": round(1e3 * head["issue"] / args.steps, 4),
        "gpu_launches": int(round(launches_per_frame * args.steps)),
        "prefetcher": None if pf is None else dict(pf_info, **{
            "with": {"missing_per_frame": hs["acc_missing"] / frames,
                     "stall_ms_per_frame": ser["stage"][0][v.STAGES.index("stream")] / max(ser["stats"]["acc_frames"], 1),
                     "prefetched_pages_per_frame": hs["acc_prefetched_pages"] / frames,
                     "prefetch_hits_per_frame": hs["acc_prefetch_hits"] / frames,
                     "ms_per_step": round(ms_head / args.steps, 4)},
            "without": {"missing_per_frame": nopf["stats"]["acc_missing"] / max(nopf["stats"]["acc_frames"], 1),
                        "stall_ms_per_frame": nopf["stage"][0][v.STAGES.index("stream")] / max(nopf["stats"]["acc_frames"], 1),
                        "ms_per_step_one_stream": round(nopf["ms"] / min(args.steps, 100), 4)},
            "ms_per_step_one_stream": round(ser["ms"] / min(args.steps, 100), 4)}),
        "roofline": {k: rl[k] for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")},
        "roofline_detail": rl,
        "clocks": clk,
        "scene_build_s": {"generate": round(t_gen, 1), "prepare": round(t_build, 1)},
    }
    if eq is not None:
        line["fp16_equal_slots"] = {"value": round(1000.0 * args.steps / eq["ms"], 2), "unit": "frames/s",
                                    "ms_per_step": round(eq["ms"] / args.steps, 4), "pool_slots": eq["slots"],
                                    "arm": "fp16 pool with the fp32 arm's slot count, copy stream, no prefetcher",
                                    "missing_per_frame": eq["stats"]["acc_missing"] / max(eq["stats"]["acc_frames"], 1)}
    if world == 1 and W["pool_bytes"] is not None:
        line["quality"] = quality_eval(v, scene, W, cams)
    if not args.no_batched and world == 1:
        line["batched_views"] = batched_views_eval(v)
    if not args.no_prefetch and world == 1:
        line["prefetch_c4"] = prefetch_eval(v)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"], sample = cpu_baseline(args, W, keep=True)
        line.setdefault("quality", {})["vs_fp64_oracle"] = quality_vs_oracle(v, W, sample)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- CPU oracle arm
STAGING = 40 * 2048 * 236   # the paper's staging buffer (about 18.4 MiB)


def rec_bytes16(K):
    """Bytes per Gaussian of the fp16 pool record (position and opacity in
    float, scale, rotation and SH in half, padded to an even half count)."""
    return 16 + 2 * (((7 + 3 * K) + 1) & ~1)


def cpu_sample(W, n_frames):
    """Bounded sample of the workload for the oracle: the same generator and
    density on a small patch (city) or the same scene (others), same camera
    model and resolution, and a page table kept as the headline arm keeps it
    (fp16 records, the pool scaled to the patch, the paper's staging budget).
    Returns (raw, build params, oracle scene, page table, cameras, slots)."""
    import scenegen
    from oracle import build as ob
    from oracle import residency as rs
    b = dict(W["build"])
    b.pop("fp16", None)
    if W["sample"] is not None:
        s = W["sample"]
        raw = scenegen.city_scene(n=s["n"], n_boxes=s["n_boxes"], extent=s["extent"])
        b["hi"] = (s["extent"] + 4, s["extent"] + 4, 88)
        cams = scenegen.city_walk_path(n_frames=n_frames, n_boxes=s["n_boxes"], extent=s["extent"])
        pool_bytes = int(W["pool_bytes"] * s["n"] / W["gaussians"])
    else:
        raw = W["gen"]()
        cams = W["path"](max(n_frames, 1))[:n_frames]
        pool_bytes = W["pool_bytes"]
    sc = ob.build_scene(raw, ob.BuildParams(**b, seed=77))
    rec = rec_bytes16((raw.sh_degree + 1) ** 2)
    P = sc.n_pages if pool_bytes is None else max(1, pool_bytes // (sc.params.page_size * rec))
    pt = rs.PageTable(rs.ResidencyParams(n_entries=P, page_size=sc.params.page_size, levels=len(sc.levels),
                                         fanout=sc.params.lod_fanout, record_bytes=rec, budget_bytes=STAGING,
                                         lod=W["lod"]))
    return raw, b, sc, pt, cams, P


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(args, W, n_frames=20, keep=False):
    """The oracle, as it stands, timed on all host cores (OpenMP over the
    Gaussians of the projection, the tiles of the blend and the triangles of
    the feedback raster; the page table and the rest in single-threaded
    Python) over n_frames consecutive frames of the bounded sample.  With
    keep, also returns what the GPU quality check needs."""
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)
    raw, b, sc, pt, cams, P = cpu_sample(W, n_frames)
    outs = []
    try:
        t0 = time.perf_counter()
        for c in cams[:n_frames]:
            o = oracle.frame(sc, pt, c, ds=4, links=True)
            if keep:
                outs.append({"image": o["render"]["image"], "draw": o["update"]["draw"]})
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    s = W["sample"]
    desc = ("%d consecutive oracle frames of the full per-frame path at %dx%d on %s, page table of %d fp16 slots" %
            (n_frames, cams[0].width, cams[0].height,
             ("a %.0f m x %.0f m patch of the city at the same density (%d Gaussians, %d boxes)" %
              (s["extent"], s["extent"], s["n"], s["n_boxes"])) if s else "the same scene", P))
    res = {"value": round(n_frames / dt, 5), "unit": "frames/s", "cores": threads, "kind": "oracle",
           "sample": desc, "nproc": os.cpu_count(), "cpu": cpu_model(), "seconds": round(dt, 2)}
    return (res, (raw, b, cams[:n_frames], P, outs)) if keep else res


def quality_vs_oracle(v, W, sample):
    """PSNR of the GPU fp16 pool's images against the FP64 oracle's renders
    of the fp32 scene, on the frames of the CPU-baseline sample (same scene,
    built by the library from the same raw input; same page-table size and
    budget, so the same pages are drawn, which is checked too)."""
    import torch
    raw, b, cams, P, outs = sample
    scene = v.vm3dgs_build_pages(raw, v.BuildConfig(**b, fp16=True, seed=77))
    cfg = v.RenderConfig(staging_bytes=STAGING, feedback_ds=4, links=True, lod=W["lod"], fp16_pool=True,
                         max_width=cams[0].width, max_height=cams[0].height, tau0=1.0, step0=0.1)
    r = v.Renderer(scene, cfg, pool_slots=P)
    img = torch.empty((3, cams[0].height, cams[0].width), dtype=torch.float32, device="cuda")
    psnr, same = [], 0
    for c, o in zip(cams, outs):
        r.render_feedback([c])
        r.update_residency()
        r.render([c], [img])
        g = img.clamp(0.0, 1.0).double().cpu().numpy()
        mse = float(np.mean((g - np.clip(o["image"], 0.0, 1.0)) ** 2))
        psnr.append(round(10.0 * math.log10(1.0 / max(mse, 1e-30)), 2))
        draw = r.debug(v.DBG_DRAW, np.int32).reshape(-1, 4)
        same += int(np.array_equal(draw, np.asarray(o["draw"], np.int32).reshape(-1, 4)))
    st = r.stats()
    del r, scene
    torch.cuda.empty_cache()
    return {"psnr_fp16_vs_fp64_oracle_db": psnr, "min_psnr_db": min(psnr), "frames": len(psnr),
            "draw_lists_equal": "%d of %d" % (same, len(psnr)), "status": st["status"],
            "note": "GPU fp16 pool (FP32 math) against the oracle's FP64 render of the fp32 attributes of the same "
                    "drawn pages; images clamped to [0, 1]; the frames of cpu_baseline.sample"}


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = workload(args.config)
    cb = cpu_baseline(args, W, n_frames=max(1, args.steps))
    line = {"impl": "reference", "metric": "1080p frames/s on 50M-Gaussian scene, plain VM vs FP16+prefetch, PSNR>=45dB",
            "value": cb["value"], "unit": "frames/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 (oracle)", "data": "synthetic (seeded scenegen), no dataset",
            "config": {"workload": W["name"], "config": args.config}, "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- paging tables
def frame_medians(v, r, cams, warmup, frames):
    """Frames on one stream with a CUDA-event time per stage and the counters
    of each frame; medians over the frames (the statistic of the page-size and
    buffer-size tables of Sec. 5)."""
    import torch
    st = torch.cuda.current_stream()
    img = torch.empty((3, cams[0].height, cams[0].width), dtype=torch.float32, device="cuda")
    n = len(cams)

    def frame(i):
        c = [cams[i % n]]
        r.render_feedback(c, st)
        r.update_residency(st)
        r.render(c, [img], st)

    for i in range(warmup):
        frame(i)
    torch.cuda.synchronize()
    r.timing(True)
    r.timing_read()
    per = []
    for i in range(warmup, warmup + frames):
        frame(i)
        ms, _ = r.timing_read()
        s = r.stats(st)
        if s["status"] != 0:
            raise RuntimeError("renderer status %d" % s["status"])
        d = dict(zip(v.STAGES, ms))
        per.append(dict(
            page_table_update_ms=d["residency"], stream_ms=d["stream"],
            depth_sort_ms=d["scan_emit"] + d["sort"] + d["ranges"], render_ms=d["project"] + d["blend"],
            feedback_ms=d["feedback"], frame_ms=sum(ms), missing_pages=s["missing"],
            requested_pages=s["requested"], drawn_pages=s["drawn_pages"], drawn_gaussians=s["drawn_gaussians"],
            pairs=s["pairs"], tau=s["tau"], usage=s["usage"], staged_projection=s["staged_projection"]))
    r.timing(False)
    out = {k: float(np.median([p[k] for p in per])) for k in per[0]}
    out["missing_pages_mean"] = float(np.mean([p["missing_pages"] for p in per]))
    # the LOD controller's approach: mean missing pages per block of 50 frames, and tau at the end
    out["missing_pages_per_50_frames"] = [round(float(np.mean([p["missing_pages"] for p in per[b:b + 50]])), 1)
                                          for b in range(0, frames, 50)]
    out["tau_last"] = float(per[-1]["tau"])
    out["frames"] = frames
    return {k: (round(x, 4) if isinstance(x, float) else x) for k, x in out.items()}


def paging_tables(args):
    """The page-size and buffer-size tables of Sec. 5 on a city walk (by
    default the 50M-Gaussian city): per-stage medians over the frames for page sizes 2048/4096/8192 at a
    fixed pool of bytes, and for pools of 250/500/1000 pages of 2048 Gaussians
    with and without LOD.  Column mapping: page-table update = the residency
    kernel; depth sort = key emission + radix sort + tile ranges; render =
    projection + blend."""
    import torch
    import paper_2506_19415_b300 as v
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    base = workload(args.config)
    frames = min(args.steps, 300)
    cams = base["path"](base["frames"])
    width, height = cams[0].width, cams[0].height
    rows = []

    def scene_at(ps):
        W = dict(base, build=dict(base["build"], page_size=ps))
        scene, _, t_build = build_scene(W)
        return W, scene, t_build

    if args.table == "pagesize":
        for ps in (2048, 4096, 8192):
            W, scene, t_build = scene_at(ps)
            r = make_renderer(v, scene, W, True, width, height)
            row = dict(page_size=ps, pages=scene.info.n_pages, pool_slots=r.n_slots, build_s=round(t_build, 1))
            row.update(frame_medians(v, r, cams, args.warmup, frames))
            rows.append(row)
            del r, scene
            torch.cuda.empty_cache()
        what = "page size (2 GiB fp16 pool, LOD on)"
    else:
        W, scene, t_build = scene_at(2048)
        for lod in (False, True):
            for slots in (250, 500, 1000):
                # small pools at close range put many more pairs on each resident Gaussian
                # than the default capacity (8 per pool Gaussian) allows
                r = make_renderer(v, scene, dict(W, lod=lod), True, width, height, pool_slots=slots,
                                  max_pairs=32 << 20)
                row = dict(page_size=2048, pool_slots=slots, lod=lod)
                row.update(frame_medians(v, r, cams, args.warmup, frames))
                rows.append(row)
                del r
                torch.cuda.empty_cache()
        what = "pool size in pages of 2048 Gaussians (fp16 pool), without and with LOD"
    print(json.dumps({"table": args.table, "varies": what, "workload": base["name"], "frames": frames,
                      "warmup": args.warmup, "statistic": "median over frames (missing pages also as a mean)",
                      "timing": "CUDA events per stage, every call on one stream", "rows": rows}))


def lod_table(args, every=25):
    """The paper's LOD (Sec. 3.4: k-means inside each page, the page halving
    per level, four levels) beside the moment-matching LOD (fanout 8, three
    levels), pages of 2048, on pools of 125, 250 and 500 pages where LOD has
    to cut detail.  All renderers step through the same walk in lockstep on one
    stream; per-frame medians of the stage times, drawn Gaussians and missing
    pages, and the PSNR of every `every`-th frame against the full-detail
    render (LOD off, the whole 2 GiB pool)."""
    import torch
    import paper_2506_19415_b300 as v
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    base = workload(args.config)
    frames, warm = min(args.steps, 300), args.warmup
    cams = base["path"](base["frames"])
    width, height = cams[0].width, cams[0].height
    st = torch.cuda.current_stream()
    Wm = dict(base, build=dict(base["build"], page_size=2048))
    Wk = dict(base, build=dict(base["build"], page_size=2048, lod_levels=4, lod_fanout=2, lod_method="kmeans"))
    sm, _, tbm = build_scene(Wm)
    sk, _, tbk = build_scene(Wk)
    ref = make_renderer(v, sm, dict(Wm, lod=False), True, width, height)
    arms = []
    for label, sc, W, tb in (("moment matching, fanout 8, 3 levels", sm, Wm, tbm),
                             ("k-means, halving, 4 levels", sk, Wk, tbk)):
        for slots in (125, 250, 500):
            arms.append(dict(lod=label, pool_slots=slots, build_s=round(tb, 1), host_bytes=int(sc.info.host_bytes),
                             r=make_renderer(v, sc, W, True, width, height, pool_slots=slots, max_pairs=32 << 20),
                             per=[], mse=[]))
    img_ref = torch.empty((3, height, width), dtype=torch.float32, device="cuda")
    img = torch.empty_like(img_ref)
    ref_missing = 0

    def frame(r, i, out):
        c = [cams[i % len(cams)]]
        r.render_feedback(c, st)
        r.update_residency(st)
        r.render(c, [out], st)

    for i in range(warm + frames):
        if i == warm:
            torch.cuda.synchronize()
            for a in arms:
                a["r"].timing(True)
                a["r"].timing_read()
        frame(ref, i, img_ref)
        sample = i >= warm and (i - warm) % every == 0
        if sample:
            ref_missing = max(ref_missing, ref.stats(st)["missing"])
        for a in arms:
            frame(a["r"], i, img)
            if i < warm:
                continue
            ms, _ = a["r"].timing_read()
            s = a["r"].stats(st)
            if s["status"] != 0:
                raise RuntimeError("renderer status %d" % s["status"])
            d = dict(zip(v.STAGES, ms))
            a["per"].append(dict(frame_ms=sum(ms), render_ms=d["project"] + d["blend"],
                                 depth_sort_ms=d["scan_emit"] + d["sort"] + d["ranges"],
                                 page_table_update_ms=d["residency"], drawn_gaussians=s["drawn_gaussians"],
                                 missing_pages=s["missing"], tau=s["tau"]))
            if sample:
                x, y = img.clamp(0.0, 1.0).double(), img_ref.clamp(0.0, 1.0).double()
                a["mse"].append(float(((x - y) ** 2).mean()))
    rows = []
    for a in arms:
        a["r"].timing(False)
        per = a.pop("per")
        row = {k: a[k] for k in ("lod", "pool_slots", "build_s", "host_bytes")}
        for k in per[0]:
            row[k] = round(float(np.median([p[k] for p in per])), 4)
        row["missing_pages_mean"] = round(float(np.mean([p["missing_pages"] for p in per])), 2)
        row["tau_last"] = round(float(per[-1]["tau"]), 3)
        mse = np.asarray(a["mse"])
        psnr = lambda e: round(10.0 * math.log10(1.0 / e), 2) if e > 0 else None  # None: identical images
        row["psnr_db_pooled"] = psnr(float(mse.mean()))
        row["psnr_db_worst_frame"] = psnr(float(mse.max()))
        row["frames_identical"] = "%d of %d" % (int((mse == 0).sum()), len(mse))
        rows.append(row)
    print(json.dumps({"table": "lod", "workload": base["name"] + "; pages of 2048", "frames": frames, "warmup": warm,
                      "psnr": "every %dth frame against the LOD-off render with every page resident (images clamped "
                              "to [0, 1]): over the pooled squared error of those frames and on the worst one; "
                              "the reference missed at most %d pages on them" % (every, ref_missing),
                      "statistic": "median over frames (missing pages also as a mean)",
                      "timing": "CUDA events per stage, every call on one stream", "rows": rows}))


def ssim(x, y):
    """Mean SSIM of two [3, H, W] images in [0, 1] (Wang et al. 2004: Gaussian
    window sigma 1.5 truncated at 11 px, C1 = 0.01^2, C2 = 0.03^2), averaged
    over the channels."""
    from scipy.ndimage import gaussian_filter
    f = lambda a: gaussian_filter(a, sigma=1.5, truncate=3.5, mode="reflect")
    out = []
    for c in range(x.shape[0]):
        a, b = x[c], y[c]
        ma, mb = f(a), f(b)
        va, vb, cab = f(a * a) - ma * ma, f(b * b) - mb * mb, f(a * b) - ma * mb
        c1, c2 = 0.01 ** 2, 0.03 ** 2
        out.append(float((((2 * ma * mb + c1) * (2 * cab + c2)) / ((ma * ma + mb * mb + c1) * (va + vb + c2))).mean()))
    return float(np.mean(out))


def quality_table(args, every=25, pools=(500, 250)):
    """The ablation of Sec. 5.2 (its PSNR/SSIM table): images rendered with
    virtual memory, with and without page links and with and without LOD, on
    buffers of 500 pages (the paper's; here none of the arms fills it) and of
    250 (which the links fill, so LOD has to coarsen), against the same view
    rendered without virtual
    memory (every level-0 page resident), for the paper's mesh proxy (Sec.
    3.1-3.3, paging "mesh") and for the voxel-face proxy.  A 12.5M-Gaussian
    city patch (1 km, 1250 boxes, SH3, pages of 4096, 3 LOD levels), fp16
    pools, the street-level walk; every `every`-th frame is compared."""
    import torch
    import paper_2506_19415_b300 as v
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    base = workload("citypatch")
    frames, warm = min(args.steps, 300), args.warmup
    cams = base["path"](base["frames"])
    width, height = cams[0].width, cams[0].height
    st = torch.cuda.current_stream()
    raw = base["gen"]()
    out_rows, proxies = [], []
    for proxy, extra in (("mesh (Sec. 3.1-3.3)", dict(paging="mesh", mesh_kappa=2.0, mesh_op_min=0.1, mesh_closing=1,
                                                      mesh_qem_ratio=0.25)),
                         ("voxel faces", dict(paging="octree"))):
        t0 = time.time()
        scene = v.vm3dgs_build_pages(raw, v.BuildConfig(**dict(base["build"], **extra), seed=77))
        t_build = time.time() - t0
        proxies.append(dict(proxy=proxy, build_s=round(t_build, 1), pages=int(scene.info.n_pages),
                            proxy_triangles=int(scene.info.n_tris), links=int(scene.info.n_links)))
        # (no copy budget: every page is resident from the first sampled frame on)
        ref = v.Renderer(scene, v.RenderConfig(staging_bytes=1 << 40, feedback_ds=4, links=False, lod=False,
                                               fp16_pool=True, max_width=width, max_height=height, max_pairs=64 << 20),
                         pool_slots=scene.info.n_pages)
        arms = []
        # the paper's four rows on each pool, and the first two again with a
        # full-resolution visibility buffer (what the lower feedback
        # resolution costs)
        confs = [(pool, links, lod, 4) for pool in pools for links in (True, False) for lod in (True, False)]
        confs += [(pools[0], True, True, 1), (pools[0], True, False, 1)]
        for pool_pages, links, lod, ds in confs:
            cfg = v.RenderConfig(staging_bytes=40 * 2048 * 236, feedback_ds=ds, links=links, lod=lod,
                                 fp16_pool=True, max_width=width, max_height=height, tau0=1.0, step0=0.1,
                                 max_pairs=32 << 20)
            arms.append(dict(pool=pool_pages, links=links, lod=lod, ds=ds, r=v.Renderer(scene, cfg, pool_slots=pool_pages),
                             mse=[], ssim=[], usage=[], required=[], missing=[], tau=[]))
        img_ref = torch.empty((3, height, width), dtype=torch.float32, device="cuda")
        img = torch.empty_like(img_ref)
        for i in range(warm + frames):
            c = [cams[i % len(cams)]]
            sample = i >= warm and (i - warm) % every == 0
            if sample:
                ref.request_all(st)
                ref.update_residency(st)
                ref.render(c, [img_ref], st)
                y = img_ref.clamp(0.0, 1.0).double()
                yh = y.cpu().numpy()
            for a in arms:
                r = a["r"]
                r.render_feedback(c, st)
                r.update_residency(st)
                r.render(c, [img], st)
                if not sample:
                    continue
                s = r.stats(st)
                if s["status"] != 0:
                    raise RuntimeError("renderer status %d" % s["status"])
                x = img.clamp(0.0, 1.0).double()
                a["mse"].append(float(((x - y) ** 2).mean()))
                a["ssim"].append(ssim(x.cpu().numpy(), yh))
                a["usage"].append(s["usage"])
                a["required"].append(s["requested"])
                a["missing"].append(s["missing"])
                a["tau"].append(s["tau"])
        psnr = lambda e: round(10.0 * math.log10(1.0 / e), 3) if e > 0 else None  # None: identical images
        for a in arms:
            mse = np.asarray(a["mse"])
            out_rows.append(dict(proxy=proxy, pool_pages=a["pool"], page_links=a["links"], lod=a["lod"],
                                 feedback_ds=a["ds"], mse_mean=float(mse.mean()),
                                 psnr_db_pooled=psnr(float(mse.mean())),
                                 psnr_db_worst_frame=psnr(float(mse.max())), ssim_mean=round(float(np.mean(a["ssim"])), 4),
                                 required_pages_mean=round(float(np.mean(a["required"])), 1),
                                 usage_mean=round(float(np.mean(a["usage"])), 3),
                                 missing_pages_mean=round(float(np.mean(a["missing"])), 2),
                                 tau_last=round(float(a["tau"][-1]), 3)))
        del arms, ref, scene
        torch.cuda.empty_cache()
    print(json.dumps({"table": "quality", "workload": base["name"] + "; fp16 pools of %s pages" % (pools,),
                      "frames": frames, "warmup": warm, "compared": "every %dth frame" % every,
                      "reference": "the same view rendered without virtual memory: every level-0 page resident, "
                                   "no feedback", "proxies": proxies, "rows": out_rows}))


def vq_table(args, n_codes=1024, every=25):
    """Compressed pages (the SH codebook of vm3dgs_scene_quantize_sh) on the
    50M-Gaussian city: the fp16 pool against VQ pools of the same 2 GiB and of
    the fp16 pool's slot count (equal pages, a third of the bytes).  Frames/s
    of the overlapped frame loop (as the headline arm, without the
    prefetcher), per-stage kernel times of a one-stream pass, bytes streamed,
    and the PSNR of the VQ images against the fp16 pool's on every `every`-th
    frame of a one-stream lockstep pass from a cold start."""
    import torch
    import paper_2506_19415_b300 as v
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    W = workload(args.config)
    scene, t_gen, t_build = build_scene(W)
    t0 = time.time()
    scene.quantize_sh(n_codes, 10, 65536)
    t_vq = time.time() - t0
    cams = W["path"](W["frames"])
    width, height = cams[0].width, cams[0].height
    copy_stream = torch.cuda.Stream()
    slots16 = W["pool_bytes"] // v.vm3dgs_pool_slot_bytes(scene, v.POOL_FP16)
    arms = [("fp16 pool", v.POOL_FP16, None), ("VQ pool, same bytes", v.POOL_VQ, None),
            ("VQ pool, the fp16 slot count", v.POOL_VQ, slots16)]

    def renderer(fmt, slots):
        cfg = v.RenderConfig(staging_bytes=40 * 2048 * 236, feedback_ds=4, links=True, lod=W["lod"], fp16_pool=fmt,
                             max_width=width, max_height=height, tau0=1.0, step0=0.1)
        if slots is not None:
            return v.Renderer(scene, cfg, pool_slots=slots)
        return v.Renderer(scene, cfg, pool_bytes=W["pool_bytes"])

    rows = []
    steps = min(args.steps, 300)
    for label, fmt, slots in arms:
        r = renderer(fmt, slots)
        run = run_arm(v, r, cams, args.warmup, steps, copy_stream, preroll=PREROLL)
        ser = run_arm(v, r, cams, args.warmup, min(steps, 100), copy_stream, timing=True, serial=True,
                      preroll=PREROLL)
        n = max(ser["stats"]["acc_frames"], 1)
        st = run["stats"]
        fr = max(st["acc_frames"], 1)
        rows.append(dict(arm=label, pool_slots=int(r.n_slots),
                         record_bytes=int(scene.info.record_bytes_vq if fmt == v.POOL_VQ else scene.info.record_bytes16),
                         frames_per_s=round(1000.0 * steps / run["ms"], 2), ms_per_frame=round(run["ms"] / steps, 4),
                         stage_ms_one_stream={k: round(x / n, 4) for k, x in zip(v.STAGES, ser["stage"][0])},
                         streamed_bytes_per_frame=st["acc_streamed_bytes"] / fr,
                         missing_per_frame=st["acc_missing"] / fr, drawn_gaussians_per_frame=st["acc_drawn_gaussians"] / fr,
                         tau=st["tau"], usage=st["usage"]))
        del r
        torch.cuda.empty_cache()
    # image quality: the VQ pool (same bytes) against the fp16 pool, lockstep
    rs = [renderer(v.POOL_FP16, None), renderer(v.POOL_VQ, slots16)]
    stq = torch.cuda.current_stream()
    imgs = [torch.empty((3, height, width), dtype=torch.float32, device="cuda") for _ in rs]
    psnr = []
    for f in range(0, 301):
        for k, r in enumerate(rs):
            r.render_feedback([cams[f]], stq)
            r.update_residency(stq)
            r.render([cams[f]], [imgs[k]], stq)
        if f and f % every == 0:
            a, b = (im.clamp(0.0, 1.0).double() for im in imgs)
            mse = float(((a - b) ** 2).mean())
            psnr.append(round(10.0 * math.log10(1.0 / max(mse, 1e-30)), 2))
    same = rs[0].stats(stq)["drawn_gaussians"] == rs[1].stats(stq)["drawn_gaussians"]
    print(json.dumps({"table": "vq", "workload": W["name"], "codes": n_codes, "code_dim": int(scene.codebook().shape[1]),
                      "build_s": {"generate": round(t_gen, 1), "pages": round(t_build, 1), "quantize": round(t_vq, 1)},
                      "host_bytes": int(scene.info.host_bytes), "frames": steps, "warmup": args.warmup,
                      "rows": rows,
                      "psnr_vq_vs_fp16_db": psnr, "psnr_frames": list(range(every, 301, every)),
                      "psnr_same_draw_list": bool(same),
                      "psnr_note": "VQ pool with the fp16 slot count against the fp16 pool, one stream, cold start; "
                                   "images clamped to [0, 1]; the SH of this synthetic scene are independent "
                                   "normal draws (no structure for a codebook to exploit)"}))


def fade_table(args, pools=(250, 500), fade=8):
    """LOD cross-fade (lod_fade_frames) on the 50M city with pages of 2048
    and fp16 pools small enough that LOD has to coarsen (as --table lod),
    with and without the fade, frames 400 on of the street walk: per-frame
    medians of the stage times (the fade's cost), the pages drawn at two
    levels and the Gaussians drawn."""
    import torch
    import paper_2506_19415_b300 as v
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    base = workload(args.config)
    W = dict(base, build=dict(base["build"], page_size=2048))
    scene, _, t_build = build_scene(W)
    cams = base["path"](base["frames"])
    width, height = cams[0].width, cams[0].height
    st = torch.cuda.current_stream()
    frames, warm = min(args.steps, 300), args.warmup
    arms = []
    for pool in pools:
        for F in (0, fade):
            cfg = v.RenderConfig(staging_bytes=40 * 2048 * 236, feedback_ds=4, links=True, lod=True, fp16_pool=True,
                                 max_width=width, max_height=height, tau0=1.0, step0=0.1, max_pairs=32 << 20,
                                 lod_fade_frames=F)
            arms.append(dict(pool=pool, fade=F, r=v.Renderer(scene, cfg, pool_slots=pool), per=[],
                             img=torch.zeros((3, height, width), dtype=torch.float32, device="cuda")))
    start = 400 - warm
    for i in range(start, start + warm + frames):
        c = [cams[i % len(cams)]]
        for a in arms:
            r = a["r"]
            if i == start + warm:
                torch.cuda.synchronize()
                r.timing(True)
                r.timing_read()
            r.render_feedback(c, st)
            r.update_residency(st)
            r.render(c, [a["img"]], st)
            if i < start + warm:
                continue
            ms, _ = r.timing_read()
            s = r.stats(st)
            if s["status"] != 0:
                raise RuntimeError("renderer status %d" % s["status"])
            d = dict(zip(v.STAGES, ms))
            a["per"].append(dict(frame_ms=sum(ms), render_ms=d["project"] + d["blend"], residency_ms=d["residency"],
                                 fading=s["fading"], drawn_gaussians=s["drawn_gaussians"], missing=s["missing"],
                                 tau=s["tau"]))
    rows = []
    for a in arms:
        a["r"].timing(False)
        per = a["per"]
        row = dict(pool_pages=a["pool"], fade_frames=a["fade"])
        for k in per[0]:
            row[k] = round(float(np.median([p[k] for p in per])), 4)
        row["fading_mean"] = round(float(np.mean([p["fading"] for p in per])), 2)
        row["drawn_gaussians_mean"] = round(float(np.mean([p["drawn_gaussians"] for p in per])), 1)
        rows.append(row)
    print(json.dumps({"table": "fade", "workload": base["name"] + "; pages of 2048, fp16 pools, frames 400 on",
                      "frames": frames, "warmup": warm, "fade_frames": fade,
                      "statistic": "median over frames (fading pages and drawn Gaussians also as means)",
                      "timing": "CUDA events per stage, one stream", "rows": rows}))


def disk_table(args):
    """Sec. 3.5 / Sec. 4.1 "Transfer": the scene saved to a file and opened
    as a read-only mapping, its pages gathered by host threads into a
    page-locked staging buffer each frame, against the same scene held in
    page-locked memory and pulled by the GPU.  The walk runs through the
    public calls (fp16 pool, the overlapped streams of the headline loop);
    "cold" first drops the file's pages from the OS cache, so the first
    touches read the disk."""
    import tempfile
    import torch
    import paper_2506_19415_b300 as v
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    W = workload(args.config)
    cams = W["path"](W["frames"])
    width, height = cams[0].width, cams[0].height
    scene, _, _ = build_scene(W)
    d = args.scene_dir or tempfile.gettempdir()
    path = os.path.join(d, "vm3dgs_%s_%d.scene" % (args.config, os.getpid()))
    t0 = time.time()
    scene.save(path)
    t_save = time.time() - t0
    rows, img = [], {}
    try:
        for label in ("in memory (page-locked, GPU pulls)", "file, warm OS cache", "file, cold OS cache"):
            if label.startswith("file"):
                if "cold" in label:
                    fd = os.open(path, os.O_RDONLY)
                    os.fsync(fd)
                    os.posix_fadvise(fd, 0, 0, os.POSIX_FADV_DONTNEED)
                    os.close(fd)
                sc = v.vm3dgs_scene_open(path)
            else:
                sc = scene
            r = make_renderer(v, sc, W, True, width, height)
            warm = 0 if "cold" in label else args.warmup
            res = run_arm(v, r, cams, warm, args.steps, torch.cuda.Stream())
            st = res["stats"]
            frames = max(st["acc_frames"], 1)
            out = torch.empty((3, height, width), dtype=torch.float32, device="cuda")
            r.render([cams[(warm + args.steps - 1) % len(cams)]], [out])
            img[label] = out.cpu()
            rows.append(dict(scene=label, ms_per_frame=round(res["ms"] / args.steps, 4),
                             frames_per_s=round(1e3 * args.steps / res["ms"], 1),
                             streamed_mb_per_frame=round(st["acc_streamed_bytes"] / frames / 1e6, 3),
                             missing_per_frame=round(st["acc_missing"] / frames, 2), warmup=warm))
            del r, sc
            torch.cuda.empty_cache()
    finally:
        os.remove(path)
    same = torch.equal(img[rows[0]["scene"]], img[rows[1]["scene"]])   # same frames, same last camera
    print(json.dumps({"table": "disk", "workload": W["name"], "steps": args.steps,
                      "scene_bytes": int(scene.info.host_bytes), "save_s": round(t_save, 1),
                      "last_image_file_equals_memory": same,
                      "note": "the cold row starts from an empty pool without warm-up, so its first frames also fill "
                              "the pool", "rows": rows}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--config", default="city50m")
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-prefetch", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--table", choices=("pagesize", "buffer", "lod", "disk", "quality", "vq", "fade"), default=None,
                    help="print the page-size or buffer-size table of Sec. 5, the LOD comparison or the "
                         "file-backed scene measurement instead of the benchmark line")
    ap.add_argument("--scene-dir", default=None, help="directory for the scene file of --table disk")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_main(args)
    elif args.table == "lod":
        lod_table(args)
    elif args.table == "disk":
        disk_table(args)
    elif args.table == "quality":
        quality_table(args)
    elif args.table == "vq":
        vq_table(args)
    elif args.table == "fade":
        fade_table(args)
    elif args.table is not None:
        paging_tables(args)
    else:
        gpu_main(args)


if __name__ == "__main__":
    main()
