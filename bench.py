"""Benchmark: contact pairs per second of the local-crop contact detector.

Workload (default): batched uneven scenes -- 8192 environments, each with
Poisson(8) objects clipped to [1, 25] drawn from a 64-shape procedural library
(unions of 2-5 boxes / ellipsoids, 300-2000 triangles, 2048 surface samples per
shape), uniform rotations, positions uniform in [-1, 1]^3.  One step is the
whole path on the device: AABB broadphase -> crop gather -> encoder -> head ->
epilogue, issued as one ``locc_step`` call (no host synchronisation inside).
Inputs are synthetic and resident in HBM before timing; L2 is flushed (a
256 MiB write) between timed steps, and each step is timed with CUDA events on
the launching stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|fp32|fp8]
    python bench.py --impl reference ...   # the CPU oracle on the same workload

After the timed steps: ``e2e`` from page-locked host arrays through the
pipelined host-buffer API (``locc_stepper``, with the synchronous
``locc_step_host`` beside it); on rank 0 the oracle on a bounded sample of the
same scene (``cpu_baseline``), a training leg (full Adam steps, both trainer
precisions) and a serving
leg (``--serve-seconds`` each: Poisson arrivals of client batches at
``--serve-rate`` requests/s through the request server, then at half of the
capacity measured there; p50/p99 latency).

Under torchrun every rank runs its own scene (weak scaling, no collective on
the data path); the timing is the max over ranks.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N_ENV = 8192
N_SHAPES = 64
LIB_SEED = 4
RADIUS = 0.25
MAX_PAIRS = 400_000
FLOP_ENC = 2 * 128 * (3 * 64 + 64 * 128 + 128 * 256)       # per pair
FLOP_HEAD = 2 * (512 * 256 + 256 * 256 + 256 * 8)          # per pair
# MMA work the BF16 head executes per pair: layer 1 in split precision (three
# products per K step), layer 2 plain, layer 3 two products into 16 columns
FLOP_HEAD_EXEC_BF16 = 2 * (3 * 512 * 256 + 256 * 256 + 2 * 256 * 16)
FLOP_POINT = 2 * (3 * 64 + 64 * 128 + 128 * 256)           # encoder, per crop point
# encoder work per object with a non-empty crop (64 point rows); an empty
# crop's pooled feature is 0 by definition and takes no arithmetic
FLOP_OBJ = 64 * FLOP_POINT
WORKLOAD = "uneven_scenes_8192env_poisson8_64shapes"
# DRAM bytes (read + write) per pair of the encoder kernel from one ncu capture
# of the bench's scene at 4096 environments (76,965 pairs; the ncu summary of
# the crop, encoder and head kernels under profiles/): scaled by the pairs of a
# launch to give the per-launch traffic (both kernels' traffic grows in
# proportion to the pairs).
ENC_DRAM_BYTES_PER_PAIR = {"bf16": (205.417216e6 + 194.258944e6) / 76965,
                           "fp8": (110.662912e6 + 25.118720e6) / 76965}
# the same for the head kernel (same capture)
HEAD_DRAM_BYTES_PER_PAIR = {"bf16": (160.763904e6 + 3.801600e6) / 76965,
                            "fp8": (42.317824e6 + 0.0) / 76965}
WEIGHTS = os.path.join(ROOT, "paper_2304_09439_b300", "weights", "locc_trained.bin")


def trained_layers():
    """The committed trained network (trained on the GPU by this library)."""
    from paper_2304_09439_b300 import weights
    with open(WEIGHTS, "rb") as f:
        return weights.unpack(f.read())


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0,
                "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region is short: start it only once samples are flowing
            t0 = time.time()
            while not self.lines and time.time() - t0 < 10.0 and self.proc.poll() is None:
                time.sleep(0.02)
            self.lines.clear()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(rank: int, n_sets: int, n_env: int = N_ENV):
    lib = synth.make_library(N_SHAPES, LIB_SEED)
    scenes = [synth.uneven_scene(n_env, N_SHAPES, seed=sd) for sd in rank_scene_seeds(rank, n_sets)]
    return lib, scenes


def run_reference(args, rank: int, world: int) -> None:
    """The oracle (plain CPU code) on the same workload, rank 0 only."""
    if rank != 0:
        return
    import oracle
    lib, scenes = make_inputs(0, 1)
    poses, osh, env = scenes[0]
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    params = oracle.flatten_params(trained_layers())
    cores = os.cpu_count() or 1
    sample = int(args.ref_sample)
    rng = np.random.default_rng(0)
    times = []
    for i in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(len(pairs), min(sample, len(pairs)), replace=False))
        t0 = time.perf_counter()
        oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs[sel], RADIUS, params,
                            n_threads=cores)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    value = sample * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": "contact pairs/sec", "value": value, "unit": "pairs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.mean(times)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_env": N_ENV, "n_shapes": N_SHAPES,
                   "pairs_per_step": int(len(pairs)), "crop_radius": RADIUS},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} random broadphase pairs of one scene per step "
                                   "(crop selection + float64 network forward)"},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _pinned_like(a):
    import torch
    t = torch.empty(a.shape, dtype=torch.from_numpy(a[:0]).dtype, pin_memory=True).numpy()
    t[...] = a
    return t


def serving_pool(n_tmpl: int, seed: int):
    """Client batches of the serving workload: environments log-uniform in
    [64, 16384], pairs log-uniform in [1e2, 1e6] (page-locked host arrays)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(np.log(1e2), np.log(1e6), n_tmpl)).astype(int)
    envs = np.exp(rng.uniform(np.log(64), np.log(16384), n_tmpl)).astype(int)
    pool = []
    for i, (e, n) in enumerate(zip(envs, sizes)):
        p, s, q = synth.client_batch(N_SHAPES, int(e), int(n), seed + 1 + i)
        pool.append((_pinned_like(p), _pinned_like(s), _pinned_like(q),
                     _pinned_like(np.zeros((int(n), 8), np.float32))))
    return pool


def serving_run(srv, pool, rate: float, seconds: float, seed: int):
    """Poisson arrivals at `rate` requests/s for `seconds`; each arrival
    submits a random batch of the pool.  Returns achieved pairs/s over the
    arrival window, latency percentiles of completed requests and counts.
    Results land in per-batch output arrays that concurrent requests of the
    same batch share (their contents are not checked here; the serving tests
    check results)."""
    import queue as _q
    from paper_2304_09439_b300 import LoccError
    rng = np.random.default_rng(seed)
    srv.stats(reset=True)
    ids = _q.Queue()
    lat, offered = [], [0, 0]
    done_pairs = [0]

    def waiter():
        while True:
            item = ids.get()
            if item is None:
                return
            rid, n = item
            info = srv.wait(rid)
            lat.append(info["done_us"])
            done_pairs[0] += n

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    rejected = 0
    t0 = time.perf_counter()
    t_next = t0
    while True:
        t_next += rng.exponential(1.0 / rate)
        if t_next - t0 > seconds:
            break
        d = t_next - time.perf_counter()
        if d > 0:
            time.sleep(d)
        p, s, q, o = pool[int(rng.integers(len(pool)))]
        offered[0] += 1
        offered[1] += len(q)
        try:
            ids.put((srv.submit(p, s, q, out=o), len(q)))
        except LoccError as e:
            if e.code != -7:
                raise
            rejected += 1
    t_end = time.perf_counter()
    st_window = srv.stats()
    ids.put(None)
    th.join()
    st = srv.stats()
    window = t_end - t0
    return {"offered_req_per_s": offered[0] / window, "offered_pairs_per_s": offered[1] / window,
            "achieved_pairs_per_s": st_window["pairs_completed"] / window,
            "completed": st["completed"], "rejected": rejected,
            "latency_p50_ms": st["latency_p50_us"] / 1e3,
            "latency_p99_ms": st["latency_p99_us"] / 1e3,
            "latency_max_ms": st["latency_max_us"] / 1e3,
            "mean_pairs_per_launch": st["mean_pairs_per_launch"],
            "max_active": st["max_active_seen"], "arena_peak_bytes": st["arena_peak"],
            "window_s": window}


def serving_leg(det, seconds: float, rate: float, max_queued: int, max_active: int = 256,
                seed: int = 6):
    """Serving workload: an overloaded run at `rate` requests/s, then a run at
    half of the capacity measured there."""
    from paper_2304_09439_b300 import Server
    pool = serving_pool(48, seed)
    mean_pairs = float(np.mean([len(x[2]) for x in pool]))
    with Server(det, arena_bytes=8 << 30, max_batch_pairs=131072, max_active=max_active,
                max_queued_pairs=max_queued) as srv:
        # warm-up: one pass over a few batches
        for p, s, q, o in pool[:4]:
            srv.wait(srv.submit(p, s, q, out=o))
        over = serving_run(srv, pool, rate, seconds, seed + 1)
        cap = over["achieved_pairs_per_s"]
        half = serving_run(srv, pool, 0.5 * cap / mean_pairs, seconds, seed + 2)
    return {"workload": "clients: envs log-U[64,16384], pairs log-U[1e2,1e6], Poisson arrivals",
            "pool_batches": len(pool), "mean_pairs_per_request": mean_pairs,
            "max_batch_pairs": 131072, "max_queued_pairs": max_queued, "max_active": max_active,
            "arena_bytes": 8 << 30, "overload": over, "half_capacity": half}


def combine_ranks(ms, pairs, e2e_s, e2e_pairs, world: int, device):
    """Whole-job figures over the ranks: the slowest rank's times (MAX) and
    everyone's pairs (SUM) -- weak scaling, each rank runs its own scenes."""
    import torch
    if world <= 1:
        return float(ms), float(pairs), float(e2e_s), float(e2e_pairs)
    import torch.distributed as dist
    stats = torch.tensor([ms, float(pairs), e2e_s, float(e2e_pairs)], dtype=torch.float64,
                         device=device)
    mx = stats.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = stats.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return mx[0].item(), sm[1].item(), mx[2].item(), sm[3].item()


def rank_scene_seeds(rank: int, n_sets: int):
    """Seeds of the scenes a rank runs: distinct per rank (no shared work)."""
    return [LIB_SEED + 1000 * rank + i for i in range(n_sets)]


def cpu_baseline_geometric(lib, scene, seconds: float = 6.0):
    """Oracle (a), the float64 geometric contact detector, on a bounded sample
    of the same scene's broadphase pairs (host cores)."""
    import oracle
    poses, osh, env = scene
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(2)
    n, dt = 64, 0.0
    while True:
        sel = np.sort(rng.choice(len(pairs), min(n, len(pairs)), replace=False))
        t0 = time.perf_counter()
        oracle.contact(lib.meshes, lib.points, poses, osh, pairs[sel], n_threads=cores)
        dt = time.perf_counter() - t0
        if dt > seconds / 4 or n >= len(pairs):
            break
        n = min(len(pairs), int(n * max(2.0, seconds / 4 / max(dt, 1e-3))))
    return {"value": len(sel) / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sel)} random broadphase pairs of one scene (float64 triangle-pair "
                      f"contact: label, point, normal, depth), {dt:.1f} s"}


def cpu_baseline(lib, scene, seconds: float = 12.0):
    """Oracle (b) on a bounded sample of the workload (host cores)."""
    import oracle
    poses, osh, env = scene
    pairs = oracle.broadphase(lib.aabb, poses, osh, env)
    params = oracle.flatten_params(trained_layers())
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1)
    n, dt = 512, 0.0
    while True:
        sel = np.sort(rng.choice(len(pairs), min(n, len(pairs)), replace=False))
        t0 = time.perf_counter()
        oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs[sel], RADIUS, params,
                            n_threads=cores)
        dt = time.perf_counter() - t0
        if dt > seconds / 4 or n >= len(pairs):
            break
        n = min(len(pairs), int(n * max(2.0, seconds / 4 / max(dt, 1e-3))))
    return {"value": len(sel) / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(sel)} random broadphase pairs of one scene (crop selection + "
                      f"float64 network forward), {dt:.1f} s"}


def oracle_configs(stream, reps: int = 20):
    """Oracle (a) and oracle (b) on the two small configurations named for
    oracle timing -- the tiny case (L-bracket vs torus, all 256 relative poses,
    seed 0) and a seeded 4,096-pair sample of the precision-sweep recipe
    (64-shape library, half uniform, half near contact) -- beside the BF16 path
    on the same pairs (one detect call per repetition, CUDA events on the
    launching stream, median).  Host cores for the oracles."""
    import torch
    import oracle
    import synth
    from paper_2304_09439_b300 import Detector
    dev = torch.device("cuda", torch.cuda.current_device())
    params = oracle.flatten_params(trained_layers())
    with open(WEIGHTS, "rb") as f:
        blob = f.read()
    cores = os.cpu_count() or 1
    lib64 = synth.make_library(N_SHAPES, LIB_SEED)
    sp, ss, sq, _ = synth.sweep_pairs(lib64, 4096, 5)
    cases = (("tiny_256", synth.tiny_library(), synth.compose_relative_tiny(256, 0)),
             ("sweep_sample_4096", lib64, (sp, ss, sq)))
    res = {}
    for name, lib, (poses, osh, pairs) in cases:
        t0 = time.perf_counter()
        oracle.crop_forward(lib.points, lib.aabb, poses, osh, pairs, RADIUS, params, n_threads=cores)
        tb = time.perf_counter() - t0
        t0 = time.perf_counter()
        oracle.contact(lib.meshes, lib.points, poses, osh, pairs, n_threads=cores)
        ta = time.perf_counter() - t0
        with Detector(lib.points, lib.aabb, blob, RADIUS, "bf16") as det:
            tp, ts, tq = (torch.from_numpy(x).to(dev) for x in (poses, osh, pairs))
            det.detect(tp, ts, tq, stream=stream)
            det.status(stream)
            ms = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                det.detect(tp, ts, tq, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            det.status(stream)
        n = len(pairs)
        res[name] = {"pairs": n, "gpu_bf16_pairs_per_s": n / (float(np.median(ms)) * 1e-3),
                     "oracle_b_pairs_per_s": n / tb, "oracle_a_pairs_per_s": n / ta,
                     "cores": cores}
    return res


FLOP_VOX = 2 * (2 * (23 * 128 + 2 * 128 * 128) + 3 * 128 * 128 + 128)  # predictor, per pair


def train_leg(lib, dsc, scene_pairs, stream, flush, steps, warmup, batches=(1024, 8192),
              precisions=("fp32", "bf16")):
    """Training throughput: full Adam steps (crop, forward, loss, backward,
    update) of the trainer on broadphase pairs of the bench scenes with
    random labels, targets and augmentation rotations (values do not change
    the work), in both trainer precisions.  L2 flushed between steps."""
    import torch
    from scipy.spatial.transform import Rotation
    from paper_2304_09439_b300 import Detector, Trainer
    rng = np.random.default_rng(11)
    out = {"what": "training step (crop + forward + loss + backward + Adam) on broadphase "
                   "pairs of the bench scenes", "weights_start": "trained", "batches": {}}
    with Detector(lib.points, lib.aabb, trained_layers(), RADIUS, "fp32") as det:
        for B in batches:
            p, s, _ = dsc[0]
            pairs = scene_pairs[0][:B].contiguous()
            tgt = np.zeros((B, 8), np.float32)
            tgt[:, 0] = rng.integers(0, 2, B)
            tgt[:, 1:4] = rng.normal(0, 1, (B, 3))
            nv = rng.normal(size=(B, 3))
            tgt[:, 4:7] = nv / np.linalg.norm(nv, axis=1, keepdims=True)
            tgt[:, 7] = rng.normal(0, 0.03, B)
            tt = torch.from_numpy(tgt).to(p.device)
            rot = torch.from_numpy(Rotation.random(B, random_state=5).as_matrix()
                                   .reshape(B, 9).astype(np.float32)).to(p.device)
            row = {}
            for prec in precisions:
                tr = Trainer(det, B, precision=prec, w_len=2.0)
                loss = torch.zeros(1, dtype=torch.float32, device=p.device)
                for _ in range(warmup):
                    flush.zero_()
                    tr.step(p, s, pairs, tt, rot, update=True, loss_out=loss, stream=stream)
                torch.cuda.synchronize()
                ms = 0.0
                n = max(3, steps // (4 if prec == "fp32" else 1))
                for _ in range(n):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    tr.step(p, s, pairs, tt, rot, update=True, loss_out=loss, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    ms += e0.elapsed_time(e1)
                det.status()
                if not np.isfinite(loss.item()):
                    raise RuntimeError(f"training loss not finite ({prec}, batch {B})")
                tr.close()
                row[prec] = {"pairs_per_s": B * n / (ms * 1e-3), "ms_per_step": ms / n,
                             "steps": n}
            if "bf16" in row and "fp32" in row:
                row["bf16_over_fp32"] = row["bf16"]["pairs_per_s"] / row["fp32"]["pairs_per_s"]
            out["batches"][str(B)] = row
    return out


def voxel_leg(lib, dsc, scene_pairs, stream, flush, steps, warmup, peaks):
    """The voxel-latent variant (the paper's own design) on the same scenes:
    latents of the 64-shape library, then per step the cell selection,
    pooling and predictor of every broadphase pair (float32, CUDA cores).
    Weights are He-uniform random (seed 7): no trained voxel network exists,
    which changes no timing."""
    import torch
    from paper_2304_09439_b300 import VoxelDetector, weights as W
    flat = synth.voxel_weights(W.VOXEL_LAYERS, 7)
    with VoxelDetector(lib.points, lib.aabb, flat) as vd:
        enc = []
        for _ in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            vd.encode(stream)
            e1.record(stream)
            e1.synchronize()
            enc.append(e0.elapsed_time(e1))
        logits = [torch.empty(len(p), dtype=torch.float32, device=p.device) for p in scene_pairs]

        def one(i):
            k = i % len(dsc)
            vd.detect(dsc[k][0], dsc[k][1], scene_pairs[k], logit=logits[k], stream=stream)

        def timed():
            for i in range(warmup):
                flush.zero_()
                one(i)
            torch.cuda.synchronize()
            ms, pairs = 0.0, 0
            for i in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one(i)
                e1.record(stream)
                e1.synchronize()
                ms += e0.elapsed_time(e1)
                pairs += len(scene_pairs[i % len(dsc)])
            vd.status(stream)
            return ms, pairs

        ms, pairs = timed()
        vd.set_precision("bf16")
        ms16, pairs16 = timed()
        vd.set_precision("fp32")
    per_launch = ms / steps
    achieved = FLOP_VOX * (pairs / steps) / (per_launch * 1e-3) / 1e12
    peak = 148 * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    per16 = ms16 / steps
    ach16 = FLOP_VOX * (pairs16 / steps) / (per16 * 1e-3) / 1e12
    peak16 = peaks["bf16_tflops_sustained"]
    return {"what": "voxel-latent variant: per-pair cell selection + average pooling + "
                    "symmetric predictor over device-resident shape latents",
            "pairs_per_s": pairs / (ms * 1e-3), "ms_per_step": per_launch, "dtype": "f32",
            "gpu_launches_per_step": 1,
            "encode_ms_64_shapes": float(np.median(enc[1:])),
            "weights": "He-uniform random (seed 7); no trained voxel network",
            "roofline": {"kernel": "vox_detect_kernel", "bound": "alu", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": None,
                         "peak_source": "derived: 148 SM x 128 FP32 lanes x 2 x sm_max_mhz",
                         "algorithmic": f"{FLOP_VOX} FLOP per pair x pairs per launch"},
            "bf16": {"pairs_per_s": pairs16 / (ms16 * 1e-3), "ms_per_step": per16,
                     "dtype": "bf16",
                     "roofline": {"kernel": "vox_tc_kernel", "bound": "tensor",
                                  "achieved": ach16, "peak": peak16, "unit": "TFLOP/s",
                                  "frac": ach16 / peak16, "traffic": None,
                                  "peak_source": "measured bf16_tflops_sustained",
                                  "algorithmic": f"{FLOP_VOX} FLOP per pair x pairs per launch"}}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--ref-sample", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time plain launches, not graph replays")
    ap.add_argument("--pipeline", default="auto",
                    help="'auto' (autotune) or 'CHUNKS,CROP_CTAS_PER_SM'")
    ap.add_argument("--sets", type=int, default=3, help="distinct scenes cycled over steps")
    ap.add_argument("--serve-seconds", type=float, default=8.0,
                    help="length of each serving run (0 = no serving leg)")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="offered requests/s")
    ap.add_argument("--serve-max-queued", type=int, default=8_000_000,
                    help="queued pairs beyond which requests are refused")
    ap.add_argument("--serve-max-active", type=int, default=256,
                    help="requests admitted at once (sharing the launches)")
    ap.add_argument("--no-voxel", action="store_true", help="skip the voxel-latent variant leg")
    ap.add_argument("--no-train", action="store_true", help="skip the training-throughput leg")
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="steps in flight in the end-to-end leg (pipelined stepper, 1-4)")
    ap.add_argument("--train-only", action="store_true",
                    help="run only the training leg and print its JSON (profiler captures)")
    ap.add_argument("--train-batches", default="1024,8192",
                    help="comma-separated training batch sizes of the training leg")
    ap.add_argument("--train-precisions", default="fp32,bf16")
    ap.add_argument("--n-env", type=int, default=N_ENV,
                    help="environments per scene (smaller scenes for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    from paper_2304_09439_b300 import Detector

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    lib, scenes = make_inputs(rank, args.sets, args.n_env)
    layers = trained_layers()
    det = Detector(lib.points, lib.aabb, layers, RADIUS, args.precision)
    det.reserve(MAX_PAIRS, args.n_env)
    dsc = []
    for poses, osh, env in scenes:
        dsc.append((torch.from_numpy(poses).to(dev), torch.from_numpy(osh).to(dev),
                    torch.from_numpy(env).to(dev)))
    pairs_buf = torch.empty((MAX_PAIRS, 2), dtype=torch.int32, device=dev)
    n_buf = torch.zeros(1, dtype=torch.int32, device=dev)
    out_buf = torch.empty((MAX_PAIRS, 8), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    # pairs per scene (counted once, outside timing)
    n_pairs, scene_pairs = [], []
    for p, s, e in dsc:
        det.step(p, s, e, MAX_PAIRS, pairs_buf, n_buf, out_buf)
        n_pairs.append(int(n_buf.item()))
        scene_pairs.append(pairs_buf[:n_pairs[-1]].clone())
    det.status()
    if max(n_pairs) > MAX_PAIRS:
        raise RuntimeError("pair buffer too small")
    # crop statistics of each scene, from the library's own crop kernel (device
    # counts): valid crop rows and objects with a non-empty crop
    valid_rows, nonempty = [], []
    for (p, s, _), pr in zip(dsc, scene_pairs):
        cnt = det.crop(p, s, pr, with_idx=False)["cnt"]
        valid_rows.append(int(cnt.sum().item()))
        nonempty.append(int((cnt > 0).sum().item()))

    if args.train_only:
        training = train_leg(lib, dsc, scene_pairs, stream, flush, args.steps, args.warmup,
                             tuple(int(b) for b in args.train_batches.split(",")),
                             tuple(args.train_precisions.split(",")))
        print(json.dumps({"training": training}), flush=True)
        det.close()
        return
    # pipelining: autotuned on the first scene, or given
    if args.pipeline == "auto":
        (chunks, cap), tune_ms = det.autotune(*dsc[0], MAX_PAIRS, reps=3, pairs_out=pairs_buf,
                                              n_pairs_out=n_buf, out=out_buf)
    else:
        chunks, cap = (int(x) for x in args.pipeline.split(","))
        det.set_pipeline(chunks, cap)
        tune_ms = None
    # broadphase (3 kernels), then per chunk: crop (which also lists the
    # objects with non-empty crops), crop fallback, encoder, head
    launches_per_step = 3 + 4 * (chunks if max(n_pairs) >= 4096 else 1)
    if chunks == 0:  # fused crop + encoder, fallback crop, deferred-object encoder, head
        launches_per_step = 3 + 4

    def step_plain(i):
        p, s, e = dsc[i % len(dsc)]
        det.step(p, s, e, MAX_PAIRS, pairs_buf, n_buf, out_buf)

    graphs = []
    if not args.no_graph:
        for i in range(len(dsc)):
            step_plain(i)  # warm-up outside capture
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream):
                step_plain(i)
            graphs.append(g)
        torch.cuda.synchronize()

    def run_timed(use_graph, profile):
        det.profile(profile)
        for i in range(args.warmup):
            flush.zero_()
            graphs[i % len(graphs)].replay() if use_graph else step_plain(i)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        stage = np.zeros(5)
        total = rows = objs = 0
        for i in range(args.steps):
            flush.zero_()
            ev0[i].record(stream)
            graphs[i % len(graphs)].replay() if use_graph else step_plain(i)
            ev1[i].record(stream)
            ev1[i].synchronize()
            if profile:
                stage += det.stage_times()
            total += n_pairs[i % len(dsc)]
            rows += valid_rows[i % len(dsc)]
            objs += nonempty[i % len(dsc)]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        det.profile(False)
        ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
        return ms, total, stage, rows, objs

    use_graph = not args.no_graph
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        ms, total_pairs, _, _, _ = run_timed(use_graph, profile=False)
        t_wall = time.perf_counter() - t_wall
        # second pass, plain launches with per-stage CUDA events (roofline)
        ms_prof, _, stage, rows_prof, objs_prof = run_timed(False, profile=True)
    det.status()

    # end to end from page-locked host buffers (what a simulator feeding the
    # detector keeps them in, allocated once): every step's inputs copied in and
    # its count, pairs and outputs copied out inside the timed region.
    # Headline: the pipelined host-buffer API (locc_stepper, two steps in
    # flight: the copies of one step overlap the next step on the device; its
    # copy-out moves the full MAX_PAIRS capacity, counted as such).  Beside
    # it: the synchronous call locc_step_host (copies, then the step, then
    # copies, one call at a time).
    from paper_2304_09439_b300 import Stepper
    host_scenes = [tuple(_pinned_like(a) for a in sc) for sc in scenes]
    h_pairs = _pinned_like(np.zeros((MAX_PAIRS, 2), np.int32))
    h_out = _pinned_like(np.zeros((MAX_PAIRS, 8), np.float32))
    det.step_host(*host_scenes[0], MAX_PAIRS, pairs_out=h_pairs, out=h_out)
    sync_t, sync_pairs = 0.0, 0
    for i in range(args.steps):
        poses, osh, env = host_scenes[i % len(host_scenes)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pr, out, n = det.step_host(poses, osh, env, MAX_PAIRS, pairs_out=h_pairs, out=h_out)
        sync_t += time.perf_counter() - t0
        sync_pairs += n
    depth = args.e2e_depth
    bufs = [(_pinned_like(np.zeros((MAX_PAIRS, 2), np.int32)),
             _pinned_like(np.zeros((MAX_PAIRS, 8), np.float32))) for _ in range(depth)]
    max_obj = max(len(sc[0]) for sc in scenes)
    e2e_t, e2e_pairs, h2d, d2h = 0.0, 0, 0, 0
    with Stepper(det, MAX_PAIRS, args.n_env, max_obj, depth) as stp:
        for rep in range(2):  # warm-up pass, then the timed one
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            flight, done_pairs = [], 0
            for i in range(args.steps):
                if len(flight) == depth:
                    done_pairs += stp.wait(flight.pop(0))[2]
                poses, osh, env = host_scenes[i % len(host_scenes)]
                flight.append(stp.submit(poses, osh, env, *bufs[i % depth]))
                if rep == 1:
                    h2d += poses.nbytes + osh.nbytes + env.nbytes
                    d2h += 4 + MAX_PAIRS * (8 + 32)
            while flight:
                done_pairs += stp.wait(flight.pop(0))[2]
            if rep == 1:
                e2e_t, e2e_pairs = time.perf_counter() - t0, done_pairs
    det.status()

    ms_max, pairs_all, e2e_max, e2e_pairs_all = combine_ranks(ms, total_pairs, e2e_t, e2e_pairs,
                                                              world, dev)

    if rank == 0:
        peaks, src = _peaks()
        per_step_pairs = total_pairs / args.steps
        enc_ms = stage[2] / args.steps
        if args.precision == "fp32":
            # CUDA-core float32: 148 SMs x 128 FMA lanes x 2 FLOP x max SM clock
            peak = 148 * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
            bound, peak_src = "alu", "derived: 148 SM x 128 FP32 lanes x 2 x sm_max_mhz"
        else:
            # burst figure: the encoder runs ~1 ms per launch inside a timed
            # region well under a second (the sustained figure is a cuBLAS loop
            # held for seconds under the power cap)
            peak = peaks["bf16_tflops"] * (2.0 if args.precision == "fp8" else 1.0)
            bound, peak_src = "tensor", f"{src} bf16_tflops (burst)" + \
                (" x 2 (fp8/bf16 nominal ratio)" if args.precision == "fp8" else "")
        # the tensor-core encoders skip objects with empty crops (their pooled
        # feature is exactly 0); the float32 encoder computes every object
        enc_flop = (FLOP_ENC * per_step_pairs if args.precision == "fp32"
                    else FLOP_OBJ * objs_prof / args.steps)
        achieved = enc_flop / (enc_ms * 1e-3) / 1e12
        achieved_padded = FLOP_ENC * per_step_pairs / (enc_ms * 1e-3) / 1e12
        # the same kernel time against the FLOPs of the valid crop rows only
        # (padded rows of partly filled or empty crops excluded)
        achieved_valid = FLOP_POINT * (rows_prof / args.steps) / (enc_ms * 1e-3) / 1e12
        head_ms = stage[3] / args.steps
        achieved_head = FLOP_HEAD * per_step_pairs / (head_ms * 1e-3) / 1e12
        cpu = cpu_geo = small = None
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(lib, scenes[0])
            cpu_geo = cpu_baseline_geometric(lib, scenes[0])
            small = oracle_configs(stream)
        voxel = None
        if not args.no_voxel:
            voxel = voxel_leg(lib, dsc, scene_pairs, stream, flush, args.steps, args.warmup, peaks)
        training = None
        if not args.no_train and world == 1:
            training = train_leg(lib, dsc, scene_pairs, stream, flush, args.steps, args.warmup,
                                 tuple(int(b) for b in args.train_batches.split(",")),
                                 tuple(args.train_precisions.split(",")))
        serving = None
        if args.serve_seconds > 0:
            serving = serving_leg(det, args.serve_seconds, args.serve_rate,
                                  args.serve_max_queued, args.serve_max_active)
        line = {
            "metric": "contact pairs/sec", "value": pairs_all / (ms_max * 1e-3),
            "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision if args.precision != "fp8" else "e4m3",
            "data": "synthetic",
            "config": {"workload": (WORKLOAD if args.n_env == N_ENV else
                                    f"uneven_scenes_{args.n_env}env_poisson8_64shapes"),
                       "n_env": args.n_env, "n_shapes": N_SHAPES,
                       "pairs_per_step": per_step_pairs, "crop_radius": RADIUS,
                       "points_per_shape": 2048, "crop_points": 64, "precision": args.precision,
                       "l2": "flushed between steps (256 MiB write)",
                       "cuda_graph": use_graph, "pipeline_chunks": chunks,
                       "crop_ctas_per_sm": cap, "autotune_ms": tune_ms,
                       "nonempty_crop_objects_per_step": float(np.mean(nonempty)),
                       "weights": "trained (paper_2304_09439_b300/weights/locc_trained.bin)",
                       "parallelism": f"replicas{world}"},
            "stage_ms": {"broadphase": stage[0] / args.steps, "crop": stage[1] / args.steps,
                         "encoder": enc_ms, "head": stage[3] / args.steps,
                         "step_profiled": stage[4] / args.steps,
                         "note": "crop / encoder / head summed over pipeline chunks; they overlap"},
            "roofline": {"kernel": "encoder", "bound": bound, "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "kernel_ms": enc_ms,
                         "frac_valid_rows": achieved_valid / peak,
                         "frac_all_pairs_padded": achieved_padded / peak,
                         "valid_rows_per_step": rows_prof / args.steps,
                         "valid_row_share": rows_prof / args.steps / (128 * per_step_pairs),
                         "stage_ms": {"broadphase": stage[0] / args.steps,
                                      "crop": stage[1] / args.steps, "encoder": enc_ms,
                                      "head": stage[3] / args.steps},
                         "traffic": (ENC_DRAM_BYTES_PER_PAIR[args.precision] * per_step_pairs
                                     if args.precision in ENC_DRAM_BYTES_PER_PAIR else None),
                         "nonempty_objects_per_step": objs_prof / args.steps,
                         "traffic_unit": "bytes per launch (ncu dram read+write per pair x pairs)",
                         "peak_source": peak_src,
                         "algorithmic": (f"{FLOP_ENC} FLOP per pair x pairs per launch"
                                         if args.precision == "fp32" else
                                         f"{FLOP_OBJ} FLOP per object with a non-empty crop "
                                         "(64 point rows) x such objects per launch")},
            # the head GEMMs on their own (the second tensor-core kernel)
            "roofline_head": {"kernel": "head", "bound": bound, "achieved": achieved_head,
                              "peak": peak, "unit": "TFLOP/s", "frac": achieved_head / peak,
                              "traffic": (HEAD_DRAM_BYTES_PER_PAIR[args.precision] * per_step_pairs
                                          if args.precision in HEAD_DRAM_BYTES_PER_PAIR else None),
                              "traffic_unit": "bytes per launch (ncu dram read+write per pair x "
                                              "pairs)",
                              "peak_source": peak_src,
                              "algorithmic": f"{FLOP_HEAD} FLOP per pair x pairs per launch",
                              "executed_mma_frac": (FLOP_HEAD_EXEC_BF16 * per_step_pairs /
                                                    (head_ms * 1e-3) / 1e12 / peak
                                                    if args.precision == "bf16" else None)},
            "e2e": {"value": e2e_pairs_all / e2e_max, "unit": "pairs/s",
                    "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
                    "api": f"locc_stepper (page-locked host arrays, {args.e2e_depth} steps in flight)",
                    "sync_call": {"api": "locc_step_host", "value": sync_pairs / sync_t,
                                  "unit": "pairs/s"}},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "cpu_baseline_geometric": cpu_geo,
            "oracle_configs": small,
            "context": "paper: 5-10x over its uniform-flow GJK at comparable accuracy (Sec. I, "
                       "IV-B); the only GPU it names is an RTX A6000 (training machine, "
                       "hyper-parameter table); quoted as context, not a target",
            "serving": serving,
            "voxel_path": voxel,
            "training": training,
            "wall_s_timed": t_wall,
        }
        print(json.dumps(line), flush=True)
    det.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
