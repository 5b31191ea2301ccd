#!/usr/bin/env python
"""Benchmark of the NIRC two-level Monte Carlo hot path on one GB300 per rank.

One step = one 1920x1080 frame of the whole path on synthetic input:
  nirc_estimate_frame  camera hits, N = 16 cache + M = 1 residual BSDF samples
                       per pixel, residual paths (depth 5, Russian roulette),
                       cache integral over 35.3 M rows
  nirc_gen_train       65,536 training paths (separate pass)
  nirc_train_step      relative-L2 loss, backward, dense Adam over 16.8 M + 17 k
                       parameters
  nirc_frame_mrse      FP64 MRSE against a 256-spp path-traced reference
The scene (256 primitives, moving emitter, GGX materials) is the dynamic
procedural Cornell family; frames W..W+K-1 are timed after W warm-up frames.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain FP64 implementation in oracle/) on a bounded sample of the same
workload instead.  Under torchrun every rank runs an independent replica
(the path shards by frame; there is no cross-GPU exchange).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2412_04634_gb300 import scenes  # noqa: E402

METRIC = "NIRC queries/s & 1080p ms/frame, FP16 TC vs FP32 at equal MRSE; p50/p99"
WORKLOAD = "1080p dynamic Cornell family (256 prims, GGX), hash-grid NIRC 16x2 T=2^19, MLP 64x4, N=16 M=1 depth 5, 65536 train samples/frame"
WORKLOAD_SH = ("1080p dynamic Cornell family (256 prims, GGX), the paper's NIRC input: hash grid 12x2 T=2^19 + "
               "spherical harmonics l<=4 (25) + albedo/one-blob normal/one-blob roughness (15), MLP 64x4, N=16 M=1 "
               "depth 5, 65536 train samples/frame")


def workload_name(args):
    name = WORKLOAD_SH if getattr(args, "input", "freq") == "sh" else WORKLOAD
    if getattr(args, "scene", "cornell") == "env":
        name = ("1080p outdoor scene (ground + 255 spheres/quads, GGX) under a procedural 6 x 64^2 cube-map sky, "
                "direct environment light (light mode 2), hash-grid cache 16x2 T=2^19, MLP 64x4, N=16 M=1, "
                f"65536 train samples/frame, {getattr(args, 'output', 'radiance')} cache output")
    if getattr(args, "estimator", "two_level") == "bth":
        name += "; biased estimator (Balanced Termination Heuristic, N cache samples at the stopping vertex, M=0)"
    elif getattr(args, "estimator", "two_level") == "mv":
        name += (f"; two levels at the first three vertices (N_c = {args.n_cache} / {args.n_cache2} / "
                 f"{args.n_cache3})")
    return name


def estimator_code(args):
    return {"two_level": 0, "bth": 1, "mv": 2}[getattr(args, "estimator", "two_level")]


def later_vertex_samples(args):
    """(N_c^2, N_c^3) of the multi-vertex estimator, else (0, 0)."""
    if estimator_code(args) != 2:
        return 0, 0
    return args.n_cache2, args.n_cache3


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp16", "bf16", "fp8"], default="fp16")
    ap.add_argument("--train-precision", choices=["fp32", "fp16"], default="fp16",
                    help="arithmetic of the training step's MLP forward and backward: FP32 SIMT kernels, or the "
                         "tensor-core training kernel (FP16 operands, per-record scaled deltas)")
    ap.add_argument("--overlap-records", type=int, default=1,
                    help="1: generate each frame's training records on a second stream, concurrently with the "
                         "frame estimate (they read only the scene); 0: one stream")
    ap.add_argument("--pipeline-trace", type=int, default=1,
                    help="1: trace frame f + 1 (NIRC_PHASE_TRACE, on a third stream) while frame f trains; the "
                         "path-tracing pass reads no cache weights.  0: each frame estimated in one call")
    ap.add_argument("--compare-fp32", type=int, default=1)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--n-cache", type=int, default=16)
    ap.add_argument("--n-resid", type=int, default=1)
    ap.add_argument("--depth", type=int, default=5)
    ap.add_argument("--train", type=int, default=65536)
    ap.add_argument("--prims", type=int, default=256)
    ap.add_argument("--ref-spp", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-budget-s", type=float, default=12.0)
    ap.add_argument("--workload", choices=["frame", "train", "serve"], default="frame",
                    help="frame: the 1080p frame step (default); train: the training step alone on "
                         "2^16 / 2^18 / 2^20 samples of the analytic radiance field; serve: the frame-request "
                         "server on a Poisson stream of mixed-resolution requests over 8 resident scenes")
    ap.add_argument("--scene", choices=["cornell", "env"], default="cornell",
                    help="env: an outdoor scene under a cube-map sky with direct environment light (light mode 2), "
                         "the Neural Visibility Cache workload")
    ap.add_argument("--output", choices=["radiance", "visibility"], default="radiance",
                    help="cache output: radiance (exp) or visibility (sigmoid, the Neural Visibility Cache)")
    ap.add_argument("--input", choices=["freq", "sh"], default="freq",
                    help="network input of the frame workload: frequency encodings of direction and normal with "
                         "the 16-level hash grid (default), or the paper's (12-level hash grid, spherical "
                         "harmonics, albedo / one-blob normal and roughness)")
    ap.add_argument("--estimator", choices=["two_level", "bth", "mv"], default="two_level",
                    help="two_level: eq. L_mlmc at the first hit (default); bth: the biased variant with the "
                         "Balanced Termination Heuristic (N cache samples at the stopping vertex, M forced to 0); "
                         "mv: the unbiased variant with the two levels also at the second and third vertex of "
                         "each residual path (--n-cache2 / --n-cache3 cache samples there)")
    ap.add_argument("--n-cache2", type=int, default=5)
    ap.add_argument("--n-cache3", type=int, default=4)
    ap.add_argument("--light-mode", type=int, choices=[0, 1, 2], default=0,
                    help="1: the cache carries L_ind, direct light by NEE + MIS (frame and serve workloads)")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--serve-low-budget-gb", type=float, default=1.0)
    ap.add_argument("--serve-deterministic", type=int, default=1)
    return ap.parse_args()


def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(rank: int) -> int:
    """Replicas only: every rank renders and trains its own independent
    replica (scene, weights and Philox seed offset by the rank); no data
    crosses ranks."""
    return 1 + rank


def max_over_ranks(x: float, dev) -> float:
    """The slowest rank's time (the only cross-rank operation: timing)."""
    import torch
    if dist_info()[0] <= 1:
        return x
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str | None):
        self.proc = None
        self.gpu_id = gpu_id

    def start(self):
        cmd = ["nvidia-smi", "--query-gpu=" + ",".join(self.FIELDS), "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd[1:1] = ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sms, maxs, reasons = [], [], set()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < len(self.FIELDS):
                continue
            try:
                sms.append(float(f[0]))
                maxs.append(float(f[1]))
            except ValueError:
                continue
            for name, val in zip(self.NAMES, f[3:]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxs), "reasons": sorted(reasons),
                "samples": len(sms)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def build_workload(args, seed_offset=0):
    import dataclasses
    W, H = args.width, args.height
    if getattr(args, "scene", "cornell") == "env":
        sc = scenes.env_scene(W, H, seed=1 + seed_offset, n_prims=args.prims, env_size=64)
        frames = [sc] * 60
    else:
        base = scenes.cornell_scene(W, H, seed=1 + seed_offset, n_prims=args.prims, glossy=True, moving_emitter=True)
        frames = [scenes.scene_at_frame(base, f) for f in range(60)]
    cfg = scenes.config_paper_1080p() if getattr(args, "input", "freq") == "sh" else scenes.config_1080p()
    if getattr(args, "output", "radiance") == "visibility":
        cfg = dataclasses.replace(cfg, output=scenes.OUT_VISIBILITY)
    params = scenes.init_params(cfg, 1 + seed_offset)
    return cfg, params, frames


def rows_per_frame(args):
    """Cache queries per frame: N + M rows per pixel, and with the
    multi-vertex estimator N_k + 1 rows per residual path at vertices 2, 3."""
    n2, n3 = later_vertex_samples(args)
    per = args.n_cache + args.n_resid + args.n_resid * ((n2 + 1 if n2 else 0) + (n3 + 1 if n3 else 0))
    return args.width * args.height * per


def flops_per_frame(cfg, args):
    """Algorithmic FLOPs of the cache integral: per row the direction part of
    layer 0, the hidden layers and the output layer; per pixel the shared
    per-surface part of layer 0."""
    per_row = 2 * (cfg.n_dir_features * 64 + (cfg.hidden_layers - 1) * 64 * 64 + 64 * 3)
    n_pix_features = cfg.n_pos_features + cfg.n_surface_features
    per_pixel = 2 * n_pix_features * 64
    n2, n3 = later_vertex_samples(args)
    units = args.width * args.height * (1 + args.n_resid * ((1 if n2 else 0) + (1 if n3 else 0)))
    return rows_per_frame(args) * per_row + units * per_pixel, per_row, per_pixel


def fp32_alu_peak_tflops(num_sms, sm_mhz):
    # 128 FP32 FMA lanes per SM, 2 FLOP per FMA
    return num_sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def measured_tensor_peak(window_s):
    """Dense 16-bit tensor peak from MEASURED_PEAKS.json (FP16 and BF16 have
    the same dense rate): the burst cuBLAS bf16 figure when the timed window
    is shorter than a second (the clocks stay at their maximum, as the
    burst measurement's did), the sustained power-capped figure for longer
    windows; else the documented fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    key = "bf16_tflops" if window_s < 1.0 else "bf16_tflops_sustained"
    try:
        with open(path) as f:
            mp = json.load(f)
        return float(mp[key]), f"MEASURED_PEAKS.json {key} (of measured; timed window {window_s:.2f} s)"
    except (OSError, KeyError, ValueError):
        if window_s < 1.0:
            return 1900.0, "fallback burst bf16 1.9 PFLOP/s (of fallback)"
        return 1700.0, "fallback sustained bf16 1.7 PFLOP/s (of fallback)"


def _precision_code(N, name):
    return {"fp32": N.NIRC_FP32_SIMT, "fp16": N.NIRC_FP16_TC, "bf16": N.NIRC_BF16_TC,
            "fp8": N.NIRC_FP8_E4M3_TC}[name]


class FrameRunner:
    """Device buffers and the per-frame step of one cache replica."""

    def __init__(self, N, args, cfg, params, frames, dev, seed):
        import torch
        self.N, self.args, self.dev, self.seed = N, args, dev, seed
        self.W, self.H = args.width, args.height
        self.P = self.W * self.H
        self.cache = N.Cache(cfg)
        self.cache.set_params(params)
        self.scene_dev = [N.scene_to_tensor(f, dev) for f in frames]
        self.n_prims = frames[0].n_prims
        T = args.train
        self.img = torch.empty((self.P, 4), device=dev)
        self.recs = torch.empty((T, 16), device=dev)
        self.dirs = torch.empty((T, 3), device=dev)
        self.tgts = torch.empty((T, 3), device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.mrse = torch.zeros(1, dtype=torch.float64, device=dev)
        self.side = torch.cuda.Stream(device=dev) if getattr(args, "overlap_records", 0) else None
        self.pt_stream = torch.cuda.Stream(device=dev) if getattr(args, "pipeline_trace", 0) else None
        self.traced = None  # (frame, event) of a frame traced ahead

    def set_precision(self, name, train="fp32"):
        self.N.nirc_set_precision(self.cache.h, _precision_code(self.N, name))
        self.N.nirc_set_train_precision(self.cache.h, _precision_code(self.N, train))

    def reference(self, frame_index, spp):
        """Plain path tracing (zero cache) of one frame, averaged over launches."""
        import torch
        N, a = self.N, self.args
        per = min(16, spp)
        n = max(1, spp // per)
        ref = torch.zeros((self.P, 4), device=self.dev)
        tmp = torch.empty((self.P, 4), device=self.dev)
        for k in range(n):
            # light mode 2 estimates direct environment light only: its reference does the same
            d = N.frame_desc(self.W, self.H, 0, per, 16, 1000 + k, self.seed, self.n_prims, cache_mode=1,
                             light_mode=2 if a.light_mode == 2 else 0)
            N.nirc_estimate_frame(self.cache.h, self.scene_dev[frame_index], d, tmp)
            ref += tmp
        ref /= n
        return ref, n * per

    def desc(self, f, phase=0):
        N, a = self.N, self.args
        n2, n3 = later_vertex_samples(a)
        return N.frame_desc(self.W, self.H, a.n_cache, a.n_resid, a.depth, f, self.seed, self.n_prims,
                            light_mode=a.light_mode, estimator=estimator_code(a), n_cache2=n2, n_cache3=n3,
                            phase=phase)

    def step(self, f, ref, scene=None, next_scene=None, ahead=False):
        """One frame: estimate, training records, training step, MRSE.  With
        --pipeline-trace, frame f's path tracing was enqueued by the step
        before (else it is traced here) and, when `ahead`, frame f + 1's is
        enqueued here on its own stream once frame f's cache pass has read
        the scratch, so it overlaps frame f's training: in steady state
        every step traces one frame, the next one."""
        import torch
        N, a = self.N, self.args
        sc = self.scene_dev[f % 60] if scene is None else scene
        h = self.cache.h
        main = torch.cuda.current_stream(self.dev)
        pipe = self.pt_stream is not None
        if pipe:
            if self.traced is not None and self.traced[0] == f:
                main.wait_event(self.traced[1])
            else:
                N.nirc_estimate_frame(h, sc, self.desc(f, N.NIRC_PHASE_TRACE), None)
            self.traced = None
        if self.side is not None:
            # the records of frame f replace those the previous training step read, so the side
            # stream first waits for everything enqueued so far; the step waits for the records
            self.side.wait_stream(main)
            N.nirc_gen_train(h, sc, self.n_prims, self.W, self.H, a.train, f, self.seed, a.depth, self.recs,
                             self.dirs, self.tgts, stream=self.side, light_mode=a.light_mode)
        N.nirc_estimate_frame(h, sc, self.desc(f, N.NIRC_PHASE_CACHE if pipe else N.NIRC_PHASE_ALL), self.img)
        if pipe and ahead:
            ev = torch.cuda.Event()
            ev.record(main)  # frame f's cache pass has read the scratch
            self.pt_stream.wait_event(ev)
            nsc = self.scene_dev[(f + 1) % 60] if next_scene is None else next_scene
            N.nirc_estimate_frame(h, nsc, self.desc(f + 1, N.NIRC_PHASE_TRACE), None, stream=self.pt_stream)
            done = torch.cuda.Event()
            done.record(self.pt_stream)
            self.traced = (f + 1, done)
        if self.side is not None:
            main.wait_stream(self.side)
        else:
            N.nirc_gen_train(h, sc, self.n_prims, self.W, self.H, a.train, f, self.seed, a.depth, self.recs,
                             self.dirs, self.tgts, light_mode=a.light_mode)
        N.nirc_train_step(h, self.recs, self.dirs, self.tgts, self.loss)
        N.nirc_frame_mrse(self.img, ref, self.mrse)

    def rays_per_frame(self, f):
        """Rays the path-tracing pass of frame f traces (camera rays, path
        segments, shadow and visibility rays), from the library's counter."""
        import torch
        N, a = self.N, self.args
        n2, n3 = later_vertex_samples(a)
        d = N.frame_desc(self.W, self.H, a.n_cache, a.n_resid, a.depth, f, self.seed, self.n_prims,
                         light_mode=a.light_mode, estimator=estimator_code(a), n_cache2=n2, n_cache3=n3)
        r = torch.zeros(1, dtype=torch.int64, device=self.dev)
        N.nirc_estimate_frame(self.cache.h, self.scene_dev[f % 60], d, self.img, rays=r)
        return int(r.item())

    def timed(self, ref, first, steps, stream, sampler=None):
        """Time `steps` frames on the device (CUDA events on `stream`)."""
        import torch
        N = self.N
        if sampler:
            sampler.start()
            time.sleep(0.3)
        N.nirc_timing_enable(self.cache.h, True)
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        world = dist_info()[0]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(self.dev)
        evs[0].record(stream)
        for k in range(steps):
            self.step(first + k, ref, ahead=True)
            evs[k + 1].record(stream)
        torch.cuda.synchronize(self.dev)
        if world > 1:
            torch.distributed.barrier()
        clocks = sampler.stop() if sampler else None
        N.nirc_sync(self.cache.h)  # raises if a tensor-core kernel reported a bounded-wait timeout
        timing = N.nirc_timing_read(self.cache.h)
        N.nirc_timing_enable(self.cache.h, False)
        step_ms = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
        total_ms = max_over_ranks(evs[0].elapsed_time(evs[-1]), self.dev)
        return dict(total_ms=total_ms, step_ms=step_ms, timing=timing, clocks=clocks, mrse=float(self.mrse.item()))

    def e2e(self, ref, first, steps, frames, stream):
        """Same steps through the public API with host buffers: the frame's
        scene blob copied in from pinned memory, image + MRSE + loss copied out."""
        import torch
        host_scenes = [torch.from_numpy(f.blob()).pin_memory() for f in frames]
        host_img = [torch.empty((self.P, 4), pin_memory=True) for _ in range(2)]
        host_small = torch.empty(2, dtype=torch.float64, pin_memory=True)
        # two device scenes: with --pipeline-trace frame f + 1 is traced during step f
        dev_scenes = [torch.empty_like(self.scene_dev[0]) for _ in range(2)]
        loaded = [None]  # the frame whose scene is already on the device
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # the image of frame f leaves on a copy stream while frame f + 1 renders into the
        # other of two device images; frame f + 2 waits for that copy before reusing it
        imgs = [self.img, torch.empty_like(self.img)]
        copy = torch.cuda.Stream(device=self.dev)
        done = [None, None]

        def one(f, ahead):
            main = torch.cuda.current_stream(self.dev)
            b = f % 2
            if done[b] is not None:
                main.wait_event(done[b])
            self.img = imgs[b]
            if loaded[0] != f:
                dev_scenes[b].copy_(host_scenes[f % 60], non_blocking=True)
            loaded[0] = f
            if self.pt_stream is not None and ahead:
                dev_scenes[1 - b].copy_(host_scenes[(f + 1) % 60], non_blocking=True)
                loaded[0] = f + 1
            self.step(f, ref, scene=dev_scenes[b], next_scene=dev_scenes[1 - b], ahead=ahead)
            host_small[0:1].copy_(self.mrse, non_blocking=True)
            host_small[1:2].copy_(self.loss.double(), non_blocking=True)
            copy.wait_stream(main)
            with torch.cuda.stream(copy):
                host_img[b].copy_(imgs[b], non_blocking=True)
            done[b] = torch.cuda.Event()
            done[b].record(copy)

        # untimed warm-up of the host-buffer path (first transfers into fresh pinned pages),
        # frames first - 3 .. first - 1, the last of which traces frame `first` ahead
        for k in range(3):
            one(max(0, first - 3 + k), True)
        torch.cuda.synchronize(self.dev)
        e0.record(stream)
        for k in range(steps):
            one(first + k, True)
        stream.wait_stream(copy)  # the last images are on the host inside the timed region
        e1.record(stream)
        torch.cuda.synchronize(self.dev)
        self.img = imgs[0]
        ms = max_over_ranks(e0.elapsed_time(e1), self.dev)
        return ms, int(frames[0].blob().nbytes), int(self.P * 16 + 8 + 4)


def recorded_traffic(args, precision):
    """DRAM bytes per launch of the cache kernel from the committed ncu
    record, or None when the record is for another workload or precision,
    or the kernel's sources have changed since the counters were taken."""
    path = os.path.join(ROOT, "profiles", f"k_cache_tc_{precision}_1080p.traffic.txt")
    if not os.path.exists(path) or (args.width, args.height, args.n_cache, args.n_resid) != (1920, 1080, 16, 1) \
            or args.input != "freq":
        return None
    rec, srcs = {}, []
    for line in open(path):
        if line.startswith("# valid while these sources hash"):
            srcs = line.split(":", 1)[1].split()
        elif ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    try:
        digest = code_sha256(srcs)
    except OSError:
        return None
    if not srcs or digest != rec.get("sources_sha256"):
        return None
    return int(rec["dram_bytes_per_launch"])


def code_sha256(paths):
    """SHA-256 of C/CUDA sources with comments and blank space removed, so a
    documentation edit keeps a counter record valid and a code edit voids it."""
    import hashlib
    import re
    h = hashlib.sha256()
    for sp in paths:
        with open(os.path.join(ROOT, sp), encoding="utf-8") as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
        h.update(b"\0")
    return h.hexdigest()


def dominant_class(timing, args):
    """The kernel class with the most device time among the library's timers
    ({class: (total ms, launches)}).  Classes whose phases run beside another
    stream's kernels time spans (they include waits for the SMs the other
    stream holds), not device time, and are left out: the training-record pass
    beside the cache pass, the training step beside the next frame's path
    tracing."""
    spans = set()
    if getattr(args, "overlap_records", 0):
        spans.add("train_records")
    if getattr(args, "pipeline_trace", 0):
        spans |= {"train_fwd", "train_bwd", "train_gradw", "adam"}
    return max((k for k, v in timing.items() if v[1] and k not in spans), key=lambda k: timing[k][0])


def _roofline(args, cfg, props, kernel_ms, dominant, sm_max, window_s):
    fl_frame, per_row, per_pixel = flops_per_frame(cfg, args)
    P = args.width * args.height
    avg_ms = kernel_ms["cache"][0]
    achieved = fl_frame / (avg_ms / 1e3) / 1e12
    algorithmic = f"{per_row} FLOP/row x {rows_per_frame(args)} rows + {per_pixel} FLOP/pixel x {P} pixels"
    if args.precision == "fp32":
        peak = fp32_alu_peak_tflops(props.multi_processor_count, sm_max)
        roof = {"kernel": "k_cache_simt", "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2),
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
                "peak_source": f"derived FP32 FMA rate: {props.multi_processor_count} SMs x 128 lanes x 2 FLOP "
                               f"x {sm_max:.0f} MHz"}
    else:
        peak, src = measured_tensor_peak(window_s)
        if args.precision == "fp8":
            # hidden layers at the E4M3 rate (nominally 2x the 16-bit rate), the rest at the 16-bit rate
            f8 = rows_per_frame(args) * 2 * (cfg.hidden_layers - 1) * 64 * 64
            f16 = fl_frame - f8
            peak = peak * fl_frame / (f8 / 2.0 + f16)
            src += " x nominal E4M3/BF16 ratio 2 on the hidden-layer share of the FLOPs"
        traffic = recorded_traffic(args, args.precision) if args.light_mode == 0 else None
        roof = {"kernel": f"k_cache_tc<{args.precision}>", "bound": "tensor", "achieved": round(achieved, 3),
                "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": src}
        if traffic is not None:
            roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch, "
                                      f"profiles/k_cache_tc_{args.precision}_1080p.traffic.txt (sources unchanged since)")
            roof["traffic_vs_algorithmic"] = round(traffic / (args.width * args.height * (64 + 32 + 32 + 16)), 3)
    roof["algorithmic"] = algorithmic
    roof["launch_ms"] = round(avg_ms, 4)
    roof["dominant_kernel"] = dominant
    return roof


def run_ours(args):
    import torch
    world, rank, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2412_04634_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2412_04634_gb300 import nirc as N

    cfg, params, frames = build_workload(args, seed_offset=replica_seed(rank) - 1)
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    gpu_id = None
    try:
        gpu_id = "GPU-" + str(props.uuid)
    except Exception:
        pass
    seed = replica_seed(rank)
    first = args.warmup
    last_frame = (first + args.steps - 1) % 60

    run = FrameRunner(N, args, cfg, params, frames, dev, seed)
    ref, ref_spp = run.reference(last_frame, args.ref_spp)
    run.set_precision(args.precision, args.train_precision)
    for f in range(args.warmup):  # the last warm-up step traces the first timed frame ahead
        run.step(f, ref, ahead=True)
    res = run.timed(ref, first, args.steps, stream, ClockSampler(gpu_id))
    # ray count of the last timed frame (an extra, untimed estimate of the same frame)
    pt_rays = run.rays_per_frame(first + args.steps - 1)
    e2e = None
    if not args.no_e2e:
        ms, bi, bo = run.e2e(ref, first, args.steps, frames, stream)
        e2e = {"value": world * rows_per_frame(args) * args.steps / (ms / 1e3), "unit": "queries/s",
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo}

    # the FP32 SIMT twin on the same frames, training data and parameter trajectory
    cmp = None
    if args.compare_fp32 and args.precision != "fp32":
        run.cache.close()
        run32 = FrameRunner(N, args, cfg, params, frames, dev, seed)
        run32.set_precision("fp32")
        for f in range(args.warmup):
            run32.step(f, ref, ahead=True)
        r32 = run32.timed(ref, first, args.steps, stream)
        cmp = {"value": world * rows_per_frame(args) * args.steps / (r32["total_ms"] / 1e3),
               "ms_per_step": r32["total_ms"] / args.steps, "p50_ms": float(np.percentile(r32["step_ms"], 50)),
               "p99_ms": float(np.percentile(r32["step_ms"], 99)), "frame_mrse": r32["mrse"],
               "cache_kernel_ms": round(r32["timing"]["cache"][0] / args.steps, 4)}
        run32.cache.close()

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    timing, clocks = res["timing"], res["clocks"]
    ms_per_step = res["total_ms"] / args.steps
    value = world * rows_per_frame(args) * args.steps / (res["total_ms"] / 1e3)
    # per frame: device ms of each kernel class and the library kernels it launched
    kernel_ms = {k: (v[0] / args.steps, v[1] / args.steps) for k, v in timing.items() if v[1]}
    dominant = dominant_class(timing, args)
    launches = sum(v[1] for v in timing.values()) + args.steps  # library kernels + one MRSE launch per step
    sm_max = (clocks or {}).get("sm_max_mhz") or 2070.0
    roofline = _roofline(args, cfg, props, kernel_ms, dominant, sm_max, res["total_ms"] / 1e3)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(args, budget_s=args.cpu_budget_s)
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16", "bf16": "bf16", "fp8": "e4m3+f16"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_name(args), "width": args.width, "height": args.height, "n_cache": args.n_cache,
                   "n_resid": args.n_resid, "max_depth": args.depth, "prims": run.n_prims,
                   "train_samples": args.train,
                   "train_precision": {"fp32": "fp32_simt", "fp16": "fp16_tc"}[args.train_precision],
                   "precision": {"fp32": "fp32_simt", "fp16": "fp16_tc", "bf16": "bf16_tc",
                                 "fp8": "fp8_e4m3_tc (hidden layers)"}[args.precision],
                   "frames": f"{first}..{first + args.steps - 1} (mod 60)",
                   "l2": "no flush: per-frame working set (~0.6 GB of records, rows, images, tables) > 129 MB L2",
                   "train_records_stream": "second stream, concurrent with the frame estimate (kernel_ms of "
                                           "train_records spans the overlap)" if args.overlap_records else "main",
                   "path_trace_stream": "third stream: frame f + 1 traced (NIRC_PHASE_TRACE) while frame f "
                                        "trains; in steady state each timed step traces exactly one frame, the "
                                        "next (the first timed frame was traced by the last warm-up step)"
                   if args.pipeline_trace else "main",
                   "light_mode": args.light_mode, "estimator": args.estimator, "input": args.input,
                   "scene": args.scene, "output": args.output,
                   "parallelism": f"replicas x{world}"},
        "p50_ms": float(np.percentile(res["step_ms"], 50)), "p99_ms": float(np.percentile(res["step_ms"], 99)),
        "frame_mrse": res["mrse"], "mrse_reference": f"{ref_spp} spp path tracing, depth 16, frame {last_frame}",
        "kernel_ms": {k: round(v[0], 4) for k, v in kernel_ms.items()},
        "kernels_per_step": {k: round(v[1], 2) for k, v in kernel_ms.items()},
        "path_trace_rays": {"rays_per_frame": pt_rays,
                            "rays_per_s": round(pt_rays / (kernel_ms["path_trace"][0] / 1e3)) if "path_trace" in
                            kernel_ms else None},
        "fp32_simt": cmp,
        "mrse_rel_diff_vs_fp32": (abs(res["mrse"] - cmp["frame_mrse"]) / cmp["frame_mrse"]) if cmp else None,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------
# CPU oracle: cpu_baseline leg and the reference arm
# ---------------------------------------------------------------------------

def oracle_step(O, cfg, params64, m, v, blob, args, frame, pix, T_s, seed):
    """One bounded sample of the frame step on the oracle: the listed pixels'
    two-level estimates, T_s training paths, loss + gradient, Adam, MRSE."""
    W, H = args.width, args.height
    n2, n3 = later_vertex_samples(args)
    fd = O.oframe(W, H, args.n_cache, args.n_resid, args.depth, frame, seed, light_mode=args.light_mode,
                  estimator=estimator_code(args), n_cache2=n2, n_cache3=n3)
    est = O.estimate(cfg, params64, blob, fd, pixels=pix)
    recs, dirs, tg, _ = O.gen_train(blob, W, H, T_s, frame, seed, args.depth, scenes.RECORD_DTYPE,
                                    light_mode=args.light_mode, visibility=int(cfg.output == scenes.OUT_VISIBILITY))
    loss, g = O.loss_grad(cfg, params64, recs, dirs, tg)
    O.adam_step(params64, m, v, g, 1, cfg.lr, cfg.beta1, cfg.beta2, cfg.adam_eps)
    O.mrse(est["pixel"], est["pixel"])
    return est


def _oracle_setup(args):
    from oracle import oracle as O
    cfg, params, frames = build_workload(args)
    p64 = params.astype(np.float64)
    return O, cfg, p64, np.zeros_like(p64), np.zeros_like(p64), frames


def _calibrate(O, cfg, p64, m, v, frames, args, budget_s):
    P = args.width * args.height
    rng = np.random.default_rng(0)
    n = 1024
    while True:
        pix = np.sort(rng.choice(P, n, replace=False)).astype(np.uint32)
        T_s = max(1, int(round(args.train * n / P)))
        t0 = time.perf_counter()
        oracle_step(O, cfg, p64, m, v, frames[10].blob(), args, 10, pix, T_s, 1)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * budget_s or n >= P:
            return n, dt
        n = min(P, int(n * max(2.0, 0.5 * budget_s / max(dt, 1e-3))))


def cpu_baseline(args, budget_s):
    O, cfg, p64, m, v, frames = _oracle_setup(args)
    S = rows_per_frame(args) // (args.width * args.height)
    n, _ = _calibrate(O, cfg, p64, m, v, frames, args, budget_s)
    P = args.width * args.height
    n = min(P, int(n * 2))
    rng = np.random.default_rng(1)
    pix = np.sort(rng.choice(P, n, replace=False)).astype(np.uint32)
    T_s = max(1, int(round(args.train * n / P)))
    t0 = time.perf_counter()
    oracle_step(O, cfg, p64, m, v, frames[11].blob(), args, 11, pix, T_s, 1)
    dt = time.perf_counter() - t0
    return {"value": n * S / dt, "unit": "queries/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n} random pixels of frame 11 ({n * S} queries) + {T_s} training paths "
                      f"(same fraction of 65536), loss/grad, dense FP64 Adam over all "
                      f"{cfg.n_params} parameters, MRSE; {dt:.1f} s"}


def run_reference(args):
    world, rank, _ = dist_info()
    if rank != 0:
        return
    O, cfg, p64, m, v, frames = _oracle_setup(args)
    S = rows_per_frame(args) // (args.width * args.height)
    per_step_budget = max(0.5, 150.0 / (args.steps + args.warmup))
    n, dt = _calibrate(O, cfg, p64, m, v, frames, args, per_step_budget * 4)
    n = max(64, int(n * per_step_budget / max(dt, 1e-3)))
    P = args.width * args.height
    n = min(P, n)
    rng = np.random.default_rng(2)
    T_s = max(1, int(round(args.train * n / P)))
    for k in range(args.warmup):
        pix = np.sort(rng.choice(P, n, replace=False)).astype(np.uint32)
        oracle_step(O, cfg, p64, m, v, frames[k % 60].blob(), args, k, pix, T_s, 1)
    times = []
    for k in range(args.steps):
        f = args.warmup + k
        pix = np.sort(rng.choice(P, n, replace=False)).astype(np.uint32)
        t0 = time.perf_counter()
        oracle_step(O, cfg, p64, m, v, frames[f % 60].blob(), args, f, pix, T_s, 1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * S * args.steps / total
    sample = (f"{n} random pixels per step ({n * S} queries) + {T_s} training paths, loss/grad, "
              f"FP64 Adam over {cfg.n_params} parameters, MRSE")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "width": args.width, "height": args.height, "n_cache": args.n_cache,
                   "n_resid": args.n_resid, "max_depth": args.depth, "train_samples": args.train,
                   "sample_pixels_per_step": n},
        "cpu_baseline": {"value": value, "unit": "queries/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# training step alone (--workload train)
# ---------------------------------------------------------------------------

def train_flops_per_sample(cfg):
    """Algorithmic FLOPs of one training sample: forward (all layers), the
    backward deltas (hidden + output layers, and the input layer's columns of
    the hash features whose gradient is scattered) and the weight gradients
    (every layer incl. biases)."""
    n_in, H = cfg.n_inputs, cfg.hidden_layers
    fwd = 2 * (n_in * 64 + (H - 1) * 64 * 64 + 64 * 3)
    dx = 2 * ((H - 1) * 64 * 64 + 64 * 3 + (cfg.n_pos_features if cfg.pos_encoding else 0) * 64)
    dw = 2 * (n_in * 64 + (H - 1) * 64 * 64 + 64 * 3)
    return fwd, dx, dw


def run_train_bench(args):
    import torch
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    from paper_2412_04634_gb300 import build
    build.build()
    from paper_2412_04634_gb300 import nirc as N
    cfg = scenes.config_1080p()
    params = scenes.init_params(cfg, 1)
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    fwd_f, dx_f, dw_f = train_flops_per_sample(cfg)
    steps, warm = max(3, args.steps), max(3, args.warmup)
    sampler = ClockSampler(None)
    sampler.start()
    time.sleep(0.3)
    out = {}
    for logb in (16, 18, 20):
        B = 1 << logb
        recs, dirs, tg = scenes.training_batch(B, seed=100 + logb)
        rt, dt, tt = N.records_to_tensor(recs, dev), torch.from_numpy(dirs).to(dev), torch.from_numpy(tg).to(dev)
        for mode in (("stored", "recompute") if logb == 20 else ("stored",)):
            cache = N.Cache(cfg)
            cache.set_params(params)
            N.nirc_set_train_mode(cache.h, mode == "stored", 1 << 15)
            N.nirc_set_train_precision(cache.h, _precision_code(N, args.train_precision))
            loss = torch.zeros(1, device=dev)
            for _ in range(warm):
                N.nirc_train_step(cache.h, rt, dt, tt, loss)
            N.nirc_timing_enable(cache.h, True)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(steps):
                N.nirc_train_step(cache.h, rt, dt, tt, loss)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            tm = N.nirc_timing_read(cache.h)
            N.nirc_timing_enable(cache.h, False)
            ph = {k: tm[k][0] / steps for k in ("train_fwd", "train_bwd", "train_gradw", "adam")}
            peak32 = fp32_alu_peak_tflops(props.multi_processor_count, 2070.0)
            fwd_n = 2 if mode == "recompute" else 1
            adam_bytes = cfg.n_params * 28 + cfg.n_hash_params * 2
            tc = args.train_precision == "fp16"
            out[f"2^{logb} {mode}"] = {
                "samples_per_s": B / (ms / 1e3), "ms_per_step": round(ms, 4),
                "phase_ms": {k: round(v, 4) for k, v in ph.items()},
                # the tensor-core kernel runs forward and backward in one launch (timed as train_fwd)
                "fwd_tflops": None if tc else round(fwd_n * fwd_f * B / (ph["train_fwd"] / 1e3) / 1e12, 2),
                "bwd_tflops": None if tc else round(dx_f * B / (ph["train_bwd"] / 1e3) / 1e12, 2),
                "fwd_bwd_tflops": round((fwd_f + dx_f) * B / (ph["train_fwd"] / 1e3) / 1e12, 2) if tc else None,
                "gradw_tflops": round(dw_f * B / (ph["train_gradw"] / 1e3) / 1e12, 2),
                "fp32_peak_tflops": round(peak32, 2),
                "adam_gbs": round(adam_bytes / (ph["adam"] / 1e3) / 1e9, 1),
                "loss": float(loss.item()),
                "activation_bytes": int(B * (cfg.n_inputs + 128 * cfg.hidden_layers) * 4) if mode == "stored"
                else int((1 << 15) * (cfg.n_inputs + 128 * cfg.hidden_layers) * 4 + B * 12),
            }
            cache.close()
    clocks = sampler.stop()
    hbm = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm = float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        hbm = 6800.0
    first = out["2^16 stored"]
    line = {
        "metric": "NIRC training step (fused encoding+MLP fwd, bwd, dense Adam) samples/s",
        "value": first["samples_per_s"], "unit": "samples/s", "n_gpus": 1, "steps": steps, "warmup": warm,
        "ms_per_step": first["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.train_precision == "fp32" else "f16",
        "data": "synthetic",
        "config": {"workload": "training step alone: x ~ U[0,1]^3, directions and normals uniform on the sphere, "
                               "targets = 8 Gaussian lobes in w modulated by 3D sinusoids in x; hash grid 16x2 "
                               "T=2^19, MLP 64x4; " + ("FP32 SIMT kernels" if args.train_precision == "fp32" else
                                                       "tensor-core forward+backward (FP16 operands), FP32 "
                                                       "weight gradients and Adam"),
                   "flops_per_sample": {"fwd": fwd_f, "bwd_dx": dx_f, "dw": dw_f},
                   "adam_bytes_per_step": int(cfg.n_params * 28 + cfg.n_hash_params * 2),
                   "hbm_peak_gbs": hbm, "recompute_chunk": 1 << 15,
                   "l2": "no flush: per-step working set (>= 570 MB of Adam state) > 129 MB L2"},
        "batches": out, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# frame-request server (--workload serve)
# ---------------------------------------------------------------------------

SERVE_RES = [(256, 256), (512, 512), (1280, 720), (1920, 1080)]
SERVE_N = [4, 8, 16, 32]


def serve_requests(n, n_scenes, seed):
    """Seeded request stream: resolution, N and scene uniform; M = 1,
    depth 5; each scene's frames numbered in arrival order."""
    rng = np.random.default_rng(seed)
    next_frame = [0] * n_scenes
    out = []
    for i in range(n):
        W, H = SERVE_RES[rng.integers(len(SERVE_RES))]
        s = int(rng.integers(n_scenes))
        out.append((i, s, W, H, SERVE_N[rng.integers(len(SERVE_N))], 1, 5, next_frame[s]))
        next_frame[s] += 1
    return out


def _serve_run(N, srv, reqs, arrivals, light_mode=0):
    """Submit reqs[i] at server time arrivals[i] (seconds after the start);
    returns per-request (latency, batch size) and the makespan."""
    import torch
    t0 = srv.clock()
    lat, bs = {}, {}
    i = 0
    n = len(reqs)
    while len(lat) < n:
        now = srv.clock() - t0
        while i < n and arrivals[i] <= now:
            srv.submit(*reqs[i], light_mode=light_mode)
            i += 1
        for c in srv.poll(wait=False):
            if c.status != 0:
                raise RuntimeError(f"request {c.id} failed with status {c.status}")
            lat[c.id] = c.t_done - c.t_submit
            bs[c.id] = c.batch_size
            srv.release(c.id)
        if i < n:
            wait = arrivals[i] - (srv.clock() - t0)
            if wait > 0:
                time.sleep(min(wait, 2e-4))
        else:
            time.sleep(5e-5)
    makespan = srv.clock() - t0
    torch.cuda.synchronize()
    return lat, bs, makespan


def _serve_summary(lat, bs, makespan, reqs):
    v = np.array([lat[r[0]] for r in reqs]) * 1e3
    px = np.array([r[2] * r[3] for r in reqs])
    big = px == 1920 * 1080
    return {"frames_per_s": len(reqs) / makespan, "p50_ms": float(np.percentile(v, 50)),
            "p99_ms": float(np.percentile(v, 99)), "mean_ms": float(v.mean()),
            "p50_ms_1080p": float(np.percentile(v[big], 50)) if big.any() else None,
            "p99_ms_1080p": float(np.percentile(v[big], 99)) if big.any() else None,
            "mean_batch": float(np.mean([bs[r[0]] for r in reqs])), "makespan_s": makespan}


def run_serve_bench(args):
    import torch
    torch.cuda.set_device(0)
    from paper_2412_04634_gb300 import build
    build.build()
    from paper_2412_04634_gb300 import nirc as N
    n_scenes = 8
    cfg = scenes.config_1080p()
    caches, frames = [], []
    for k in range(n_scenes):
        c = N.Cache(cfg)
        c.set_params(scenes.init_params(cfg, 1 + k))
        N.nirc_set_precision(c.h, N.NIRC_FP16_TC)
        N.nirc_set_deterministic(c.h, bool(args.serve_deterministic))
        caches.append(c)
        base = scenes.cornell_scene(1920, 1080, seed=1 + k, n_prims=256, glossy=True, moving_emitter=True)
        frames.append([scenes.scene_at_frame(base, f) for f in range(60)])
    T = args.train

    def make_server(budget_gb):
        srv = N.Server(int(budget_gb * (1 << 30)), slots=8, max_batches=2, train_samples=T, use_graphs=True)
        for k in range(n_scenes):
            srv.add_scene(caches[k], frames[k], seed=1 + k)
        return srv

    n = args.serve_requests
    results = {}
    sampler = ClockSampler(None)
    sampler.start()
    time.sleep(0.3)
    srv = make_server(args.serve_budget_gb)
    # warm-up: every scene, every size once (graph instantiation, first-touch)
    warm = serve_requests(32, n_scenes, seed=99)
    warm = [(10_000 + r[0],) + r[1:] for r in warm]
    lm = args.light_mode
    _serve_run(N, srv, warm, [0.0] * len(warm), lm)
    reqs = serve_requests(n, n_scenes, seed=5)
    lat, bs, mk = _serve_run(N, srv, reqs, [0.0] * n, lm)
    sat = _serve_summary(lat, bs, mk, reqs)
    results["saturated (all at t=0)"] = sat
    rng = np.random.default_rng(17)
    for frac in (0.5, 0.8, 1.0):
        rate = frac * sat["frames_per_s"]
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
        reqs = [(r[0] + int(frac * 10) * 100_000,) + r[1:] for r in serve_requests(n, n_scenes, seed=6)]
        lat, bs, mk = _serve_run(N, srv, reqs, arrivals, lm)
        results[f"poisson {frac:.1f}x"] = dict(_serve_summary(lat, bs, mk, reqs), offered_per_s=rate)
    st = srv.stats()
    srv.close()
    # low budget: admission throttles concurrency
    srv = make_server(args.serve_low_budget_gb)
    rate = 0.8 * sat["frames_per_s"]
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    reqs = [(r[0] + 900_000,) + r[1:] for r in serve_requests(n, n_scenes, seed=7)]
    lat, bs, mk = _serve_run(N, srv, reqs, arrivals, lm)
    st_low = srv.stats()
    results[f"poisson 0.8x, {args.serve_low_budget_gb:g} GB budget"] = dict(
        _serve_summary(lat, bs, mk, reqs), offered_per_s=rate, arena_peak_gb=st_low["arena_peak_bytes"] / 2**30)
    srv.close()
    clocks = sampler.stop()
    for c in caches:
        c.close()
    head = results["poisson 0.8x"]
    line = {
        "metric": "NIRC serving: frame latency p50/p99 and frames/s (Poisson arrivals, continuous batching)",
        "value": sat["frames_per_s"], "unit": "frames/s", "n_gpus": 1, "steps": n, "warmup": len(warm),
        "ms_per_step": 1e3 / sat["frames_per_s"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16", "data": "synthetic",
        "p50_ms": head["p50_ms"], "p99_ms": head["p99_ms"],
        "config": {"workload": f"{n} requests over {n_scenes} resident 1080p-family scenes (seeds 1-8, 256 prims, "
                               f"hash-grid NIRC 16x2 T=2^19, MLP 64x4, FP16 tensor cores); resolution uniform in "
                               f"256^2/512^2/1280x720/1920x1080, N uniform in 4/8/16/32, M=1, depth 5; one training "
                               f"pass ({T} paths) + Adam step per served frame",
                   "budget_gb": args.serve_budget_gb, "slots": 8, "max_batches": 2, "graphs": True,
                   "deterministic_training": bool(args.serve_deterministic), "light_mode": args.light_mode,
                   "latency": "server clock from submission to the completion of the request's batch on the device"},
        "runs": results,
        "server_stats": {k: st[k] for k in ("batches", "graph_instantiations", "graph_updates", "max_batch_seen",
                                            "arena_peak_bytes", "resident_bytes", "frame_launches")},
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.estimator == "bth":
        args.n_resid = 0  # the biased estimator has no residual level
    if args.scene == "env":
        args.light_mode = 2  # direct environment light
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "train":
        run_train_bench(args)
    elif args.workload == "serve":
        run_serve_bench(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
