"""Benchmark of the RIFT2 hot path on GB300: pairs/s at 1024x1024.

One step = extract(A) + extract(B) + match(A -> B) for every pair of one batch of
synthetic 1024^2 pairs (400 blobs, 200 segments, random rotation, intensity remap and
gamma speckle; at most 5000 keypoints per image).  Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--pairs B] [--impl ours|reference]
                  [--workload 1|2|3]

--workload 2 times the uneven batch (64 pairs, sides 384..2048 step 128, <= 4000
keypoints) and --workload 3 the 4096^2 scene (<= 20000 keypoints); the default line also
carries an open-loop serving sweep (Poisson arrivals at 50..400 pairs/s).  Besides the
headline (one context, one stream) the line reports the same step as one replayed CUDA
graph (graph_form), on one context with two lanes (RIFT2_FLAG_TWO_LANES: each call's second
half of images and pairs on the library's second stream; two_lane_form), and the plain
one-pair-per-call forms.

Multi-GPU: independent replicas (the pairs shard with no exchange step); launched with
torch.distributed.run, one rank per GPU, timing = max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s at 1024x1024 (extract A + extract B + NN match A->B)"


def _uneven(n, rank):
    import synth
    return synth.batch_sizes(n, seed=20232001 + rank)


WORKLOADS = {
    1: {"metric": METRIC, "max_kp": 5000, "pairs": 8,
        "sizes": lambda n, rank: [(1024, 1024)] * n,
        "desc": "1024x1024 synthetic multimodal pairs (400 blobs, 200 segments, random rotation, "
                "1-v^0.6 remap, gamma speckle), <=5000 kp"},
    2: {"metric": "pairs/s, uneven batch (sides 384..2048 step 128, aspect <= 2)", "max_kp": 4000,
        "pairs": 64, "sizes": _uneven,
        "desc": "64 pairs per step, sides uniform on 384..2048 step 128 (aspect <= 2), random "
                "rotation, <=4000 kp"},
    3: {"metric": "pairs/s, 4096x4096 large scene", "max_kp": 20000, "pairs": 1,
        "sizes": lambda n, rank: [(4096, 4096)] * n,
        "desc": "4096x4096 pair, <=20000 kp, ~20000x20000x216 matching"},
}
H = W = 1024
MAX_KP = 5000
ROTATE = 4   # input batches rotated between steps


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 8:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[4:8]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------- roofline model
# Algorithmic bytes per pixel of one image for each stage (minimal traffic of the
# two-pass schedule): the column pass reads the spectrum once (8 B) and writes 24
# complex responses (192 B); the row pass reads them (192 B) and writes Er, q, |EO_0|
# for 6 orientations (72 B) and the MIM (1 B).
STAGE_BYTES_PER_PX = {"fft_fwd": 16.0, "lg_cols": 200.0, "lg_rows": 265.0, "noise": 24.0,
                      "moment": 52.0, "detect": 4.0}


# Kernel source each stage's DRAM-traffic figure in profiles/traffic.json was captured
# from; the figure is reported only while these files are unchanged.
STAGE_SOURCES = {"lg_cols": ("k_filterbank.cu", "fft_reg.cuh", "fft.cuh", "common.cuh"),
                 "lg_rows": ("k_filterbank.cu", "fft_reg.cuh", "fft.cuh", "common.cuh")}


def stage_source_hash(stage: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in STAGE_SOURCES.get(stage, ()):
        with open(os.path.join(ROOT, "paper_2303_00319_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(stage: str, images: int):
    """DRAM bytes per launch of `stage` for `images` images, scaled from the ncu capture in
    profiles/traffic.json (bytes grow in proportion to the images a launch processes), or
    None when the kernel source changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            d = json.load(fh)[stage]
    except Exception:
        return None
    if d.get("source_hash") != stage_source_hash(stage):
        return None
    return d["dram_bytes_per_image"] * images


def load_tensor_peak():
    """Sustained dense BF16 TFLOP/s (a kernel timed inside a long step)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        return 1700.0, "fallback (sustained)"


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ oracle timing
def oracle_pair_seconds(size: int, max_kp: int, seed: int) -> float:
    import oracle
    import synth
    pr = synth.make_pair(size, size, seed, angle_deg=None)
    p = oracle.Params(max_keypoints=max_kp)
    t0 = time.perf_counter()
    fa = oracle.extract(pr.a.astype(np.float64), p)
    fb = oracle.extract(pr.b.astype(np.float64), p)
    oracle.match(fa.desc, fb.desc)
    return time.perf_counter() - t0


def reference_sample_size(steps: int, warmup: int) -> int:
    # ~25 s per 1024^2 pair on one host: keep the whole run near two minutes
    for s in (1024, 768, 512, 384, 256):
        if (steps + warmup) * 25.0 * (s / 1024.0) ** 2 <= 150.0:
            return s
    return 256


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    s = reference_sample_size(args.steps, args.warmup)
    frac = (s / 1024.0) ** 2
    kp = max(100, int(round(MAX_KP * frac)))
    for i in range(args.warmup):
        oracle_pair_seconds(s, kp, 20231001 + i)
    times = [oracle_pair_seconds(s, kp, 20232001 + i) for i in range(args.steps)]
    t = sum(times) / len(times)
    value = frac / t
    sample = (f"each step: one {s}x{s} pair (2 FP64 oracle extracts with <= {kp} keypoints + "
              f"brute-force match), credited as {frac:.4f} of a 1024^2 pair (pixel ratio)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1000.0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "1024x1024 synthetic multimodal pairs", "pairs_per_step": frac,
                       "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------- parity of the sampled pair
def _worst(got, exp, floor, extra=None):
    got = np.asarray(got, dtype=np.float64)
    exp = np.asarray(exp, dtype=np.float64)
    scale = float(np.max(np.abs(exp)))
    if scale == 0:
        return float(np.max(np.abs(got)))
    den = np.maximum(np.abs(exp), floor * scale)
    if extra is not None:
        den = np.maximum(den, extra)
    return float(np.max(np.abs(got - exp) / den))


def parity_summary(pkg, dev, pair, oa, ob, of_match):
    """Every output of the GPU path on one pair against the FP64 oracle's: worst element-wise
    relative error of each float map above its floor, integer outputs that differ and how
    many of those the oracle certifies as near ties (relative top-two margin < 1e-5)."""
    import torch
    ctx = pkg.Context(pkg.default_params(max_keypoints=MAX_KP), device=dev.index)
    fa, fb = ctx.extract([torch.from_numpy(pair.a).to(dev), torch.from_numpy(pair.b).to(dev)],
                         debug=True)
    m = ctx.match([fa], [fb])[0]
    ctx.sync()
    out = {"pair": "1024x1024 pair of the generator (seed 20231001), images A and B"}
    maps = {}
    mim_bad = mim_diff = near_px = 0
    kp_only = kp_cert = 0
    hosts = []
    for f, o in ((fa, oa), (fb, ob)):
        d = {k: v.cpu().numpy() for k, v in f.debug.items()}
        mo = o.maps
        amax = float(np.max(mo["A"]))
        with np.errstate(divide="ignore", invalid="ignore"):
            cq = np.where(mo["A"] > 0, mo["q"] * 2.5e-3 * amax / mo["A"], 0.0)
        ce = mo["A"] / (4.0 * mo["X"]) * 1e-2 * amax
        vals = {"A_o": _worst(d["amp"], mo["A"], 2.5e-3), "|EO0|": _worst(d["an0"], mo["An0"], 1e-2),
                "q": _worst(d["q"], mo["q"], 1e-3, cq), "Er": _worst(d["er"], mo["Er"], 5e-2, ce),
                "PC": _worst(d["pc"], mo["pc"], 1.0), "M": _worst(d["moment"], mo["M"], 2e-2),
                "T_o": float(np.max(np.abs(d["noise_t"] - mo["T"]) / np.abs(mo["T"]))),
                "M_normalised_abs": float(np.max(np.abs(d["moment"] - mo["M"])) /
                                          (mo["M"].max() - mo["M"].min()))}
        for k, v in vals.items():
            maps[k] = max(maps.get(k, 0.0), v)
        mis = d["mim"] != mo["mim"]
        mim_diff += int(mis.sum())
        mim_bad += int((mis & (mo["mim_margin"] >= 1e-5)).sum())
        near_px += int((mo["mim_margin"] < 1e-5).sum())
        g = f.host()
        hosts.append(g)
        gs = {tuple(map(int, q)) for q in g["xy"]}
        osx = {tuple(map(int, q)) for q in o.xy}
        for q in gs ^ osx:
            kp_only += 1
            kp_cert += int(bool(mo["kp_uncertain"][q[1], q[0]]))
    out["max_rel_err"] = maps
    out["tolerance"] = "1e-4 relative above each floor (A_o 2.5e-3, |EO0| 1e-2, q 1e-3 with A's floor, Er 5e-2 with its A/X conditioning, PC 1.0), M 2e-4 above 2e-2 (quadratic in PC); T_o 1e-4 relative; M 5e-6 in FAST's normalised units"
    out["mim"] = {"pixels_differing": mim_diff, "of_which_not_near_ties": mim_bad,
                  "oracle_near_tie_pixels": near_px}
    out["keypoints"] = {"in_one_list_only": kp_only, "of_which_certified": kp_cert,
                        "per_image": [len(h["xy"]) for h in hosts]}
    # descriptors of keypoints both lists share whose patch has no differing MIM pixel
    checked = bad = 0
    for g, f, o in ((hosts[0], fa, oa), (hosts[1], fb, ob)):
        mis = f.debug["mim"].cpu().numpy() != o.maps["mim"]
        gi = {tuple(map(int, q)): i for i, q in enumerate(g["xy"])}
        for k, (x, y) in enumerate(np.asarray(o.xy).tolist()):
            if (x, y) not in gi or mis[y - 48:y + 48, x - 48:x + 48].any():
                continue
            jo = np.flatnonzero(o.desc_kp == k)
            jg = np.flatnonzero(g["desc_kp"] == gi[(x, y)])
            checked += 1
            bad += int(not np.array_equal(g["desc"][jg].astype(np.int64), o.desc[jo]))
    out["descriptors"] = {"keypoints_compared": checked, "differing": bad}
    nn, d1, d2, near = of_match(hosts[0]["desc"].astype(np.int64), hosts[1]["desc"].astype(np.int64))
    mh = m.host()
    diff = mh["nn_desc"] != nn
    fin = np.isfinite(d1) & (d1 > 0)
    out["matches"] = {"rows": int(len(nn)), "nn_differing": int(diff.sum()),
                      "of_which_not_near_ties": int((diff & ~near).sum()),
                      "oracle_near_ties": int(near.sum()),
                      "d1_max_rel_err": float(np.max(np.abs(mh["d1"][fin] - d1[fin]) / d1[fin]))
                      if fin.any() else 0.0,
                      "reference": "the oracle's exhaustive search on the GPU's descriptors"}
    ctx.close()
    return out


# ------------------------------------------------- summaries of the other workloads
def _make_pair_job(args):
    import synth
    h, w, seed = args
    kw = dict(n_blobs=400, n_segments=200) if (h, w) == (1024, 1024) else {}
    pr = synth.make_pair(h, w, seed, angle_deg=None, **kw)
    return pr.a, pr.b


def make_pairs(jobs):
    """Synthetic pairs generated on the host cores (a spawn pool: safe after CUDA init)."""
    import multiprocessing as mp
    n = min(len(jobs), os.cpu_count() or 1)
    if n <= 1:
        return [_make_pair_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(_make_pair_job, jobs, chunksize=1)


def workload_summary(pkg, dev, wl_id, steps=4, warmup=3):
    """pairs/s of a workload other than the headline one, timed the same way (inputs
    resident, CUDA events on the launching stream), with the kernel launches per step."""
    import torch
    wl = WORKLOADS[wl_id]
    B = wl["pairs"]
    sizes = wl["sizes"](B, 0)
    pairs = make_pairs([(h, w, synth_seed(wl_id, b)) for b, (h, w) in enumerate(sizes)])
    imgs = []
    for a, b in pairs:
        imgs += [torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)]
    px = sum(2 * h * w for h, w in sizes)
    st = torch.cuda.current_stream()

    def timed(flags, stages=False):
        ctx = pkg.Context(pkg.default_params(max_keypoints=wl["max_kp"], flags=flags),
                          device=dev.index, hbm_budget=96 << 30)
        feats = [ctx.alloc_features() for _ in range(2 * B)]
        matches = [ctx.alloc_matches() for _ in range(B)]

        def step():
            ctx.extract(imgs, feats, stream=st)
            ctx.match(feats[0::2], feats[1::2], matches, stream=st)

        for _ in range(warmup):
            step()
        ctx.sync()
        torch.cuda.synchronize()
        l0 = ctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            step()
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ctx.sync()
        res = {"value": B / (ms / 1000.0), "unit": "pairs/s", "ms_per_step": ms,
               "mpix_per_s": px / 1e6 / (ms / 1000.0),
               "launches_per_step": (ctx.launch_count() - l0) // steps}
        if stages:   # one more step with per-stage events (after the timed ones)
            ctx.set_profiling(True)
            step()
            ctx.sync()
            res["stage_ms_per_step"] = {k: round(v[0], 4) for k, v in ctx.profile_read().items()}
            ctx.set_profiling(False)
        ctx.close()
        return res

    out = {"workload": wl["desc"], "metric": wl["metric"], "pairs_per_step": B}
    out.update(timed(pkg.FLAG_AUTOTUNE, stages=True))
    out.update({"steps": steps, "warmup": warmup})
    if len({tuple(x) for x in sizes}) > 1:
        # the same batch with launch groups of one image size each (RIFT2_FLAG_SIZE_GROUPS)
        sg = timed(pkg.FLAG_AUTOTUNE | pkg.FLAG_SIZE_GROUPS)
        out["size_groups_form"] = {"value": sg["value"], "unit": "pairs/s",
                                   "ms_per_step": sg["ms_per_step"],
                                   "launches_per_step": sg["launches_per_step"],
                                   "form": "launch groups of one image size each"}
    return out


def synth_seed(wl_id, b):
    import synth
    return synth.pair_seed(wl_id, b)


# ------------------------------------------------------------- multi-rank timing
def max_over_ranks(ms: float, device=None) -> float:
    """The slowest rank's time: every rank's value, MAX-reduced (no-op on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, pairs_per_step: int, steps: int, max_ms: float) -> float:
    """Pairs per second over all ranks: each rank (replica) processed pairs_per_step pairs
    in each of `steps` steps, and the job took as long as its slowest rank."""
    return world * pairs_per_step * steps / (max_ms / 1000.0)


# --------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2303_00319_gb300 as pkg
    import synth
    from paper_2303_00319_gb300 import _build

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    _build.build()
    wl = WORKLOADS[args.workload]
    B = args.pairs if args.workload == 1 else wl["pairs"]
    rot = ROTATE if args.workload == 1 else 1
    max_kp = wl["max_kp"]
    # the autotuner times the shared-memory column tiles (the uneven batch) and the
    # matcher's split once, during the warm-up steps.  One lane: the timed steps read the
    # per-stage device times, and a profiling context runs every call on the caller's stream
    ctx = pkg.Context(pkg.default_params(max_keypoints=max_kp, flags=pkg.FLAG_AUTOTUNE),
                      device=local, hbm_budget=96 << 30)

    # inputs: `rot` batches of B pairs, distinct per rank; pinned host copies for e2e
    host = []
    sizes = wl["sizes"](B, rank)
    jobs = [(sizes[b][0], sizes[b][1], synth.pair_seed(args.workload, 100000 * rank + r * B + b))
            for r in range(rot) for b in range(B)]
    made = make_pairs(jobs)   # on the host cores, in parallel
    for r in range(rot):
        batch = []
        for b in range(B):
            a, bb = made[r * B + b]
            batch += [torch.from_numpy(a).pin_memory(), torch.from_numpy(bb).pin_memory()]
        host.append(batch)
    devb = [[t.to(dev) for t in batch] for batch in host]
    feats = [ctx.alloc_features() for _ in range(2 * B)]
    matches = [ctx.alloc_matches() for _ in range(B)]
    stream = torch.cuda.current_stream()
    px_per_step = sum(2 * h * w for h, w in sizes)

    def step(imgs, st=None):
        st = stream if st is None else st
        ctx.extract([imgs[i] for i in range(2 * B)], feats, stream=st)
        ctx.match(feats[0::2], feats[1::2], matches, stream=st)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        step(devb[i % rot])
    ctx.sync()
    ctx.profile_read()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    ctx.set_profiling(True)
    launches0 = ctx.launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    barrier()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        evs[i][0].record(stream)
        step(devb[i % rot])
        evs[i][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    launches = ctx.launch_count() - launches0
    ctx.set_profiling(False)
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    prof = ctx.profile_read()
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, B, args.steps, total_ms)

    # end to end through the public API with host buffers: every step copies its pinned
    # input images in on a copy stream (overlapping the previous step's kernels through
    # two device input buffers), runs extract + match, and copies its matches out; all K
    # steps' copies lie inside the timed region
    copy_stream = torch.cuda.Stream(device=dev)
    # inputs: each batch as one pinned host tensor and two device tensors [2B][H][W] (one
    # H2D copy per step); outputs: every pair's correspondences (q_desc, nn_desc, kp_a, kp_b,
    # d1, d2, near_tie, count) and both images' keypoints (xy, score, counts) as views into
    # one device arena (one D2H copy per step), descriptors in their own buffers
    ncap = matches[0].nn_desc.shape[0]
    kcap = feats[0].kp_xy.shape[0]
    al = lambda n: (n + 15) // 16 * 16  # noqa: E731  (64-byte aligned sub-arrays)
    per_pair = 6 * al(ncap) + al((ncap + 3) // 4) + 16
    per_img = al(2 * kcap) + al(kcap) + 16
    arena = torch.zeros(B * per_pair + 2 * B * per_img, dtype=torch.int32, device=dev)
    e2e_feats, e2e_matches = [], []
    for b in range(B):
        o = b * per_pair
        m = ctx.alloc_matches()
        views = []
        for k in range(6):
            views.append(arena[o + k * al(ncap):o + k * al(ncap) + ncap])
        o6 = o + 6 * al(ncap)
        tie = arena[o6:o6 + (ncap + 3) // 4].view(torch.uint8)[:ncap]
        cnt = arena[o6 + al((ncap + 3) // 4):o6 + al((ncap + 3) // 4) + 1]
        e2e_matches.append(pkg.Matches(views[0], views[1], views[2], views[3],
                                       views[4].view(torch.float32), views[5].view(torch.float32),
                                       tie, cnt))
    for j in range(2 * B):
        o = B * per_pair + j * per_img
        f = ctx.alloc_features()
        f.kp_xy = arena[o:o + 2 * kcap].view(kcap, 2)
        f.kp_score = arena[o + al(2 * kcap):o + al(2 * kcap) + kcap].view(torch.float32)
        f.counts = arena[o + al(2 * kcap) + al(kcap):o + al(2 * kcap) + al(kcap) + 2]
        e2e_feats.append(f)
    # each batch flattened into one buffer (sizes may differ), images as views into it
    offs = [0]
    for t in host[0]:
        offs.append(offs[-1] + t.numel())
    host_flat = [torch.cat([t.reshape(-1) for t in batch]).pin_memory() for batch in host]
    dflat = [torch.empty_like(host_flat[0], device=dev) for _ in range(2)]
    shapes = [tuple(t.shape) for t in host[0]]
    views = lambda flat: [flat[offs[k]:offs[k + 1]].view(shapes[k]) for k in range(2 * B)]  # noqa: E731
    arena_h = [torch.empty(arena.shape, dtype=torch.int32).pin_memory() for _ in range(2)]
    ev_copied = [torch.cuda.Event() for _ in range(args.steps)]
    ev_done = [torch.cuda.Event() for _ in range(args.steps)]

    def e2e_step(imgs):
        ctx.extract(imgs, e2e_feats, stream=stream)
        ctx.match(e2e_feats[0::2], e2e_feats[1::2], e2e_matches, stream=stream)

    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_stream(stream)
    for i in range(args.steps):
        buf = dflat[i % 2]
        with torch.cuda.stream(copy_stream):
            if i >= 2:
                copy_stream.wait_event(ev_done[i - 2])   # this buffer's previous step is done
            buf.copy_(host_flat[i % rot], non_blocking=True)
            ev_copied[i].record(copy_stream)
        stream.wait_event(ev_copied[i])
        e2e_step(views(buf))
        arena_h[i % 2].copy_(arena, non_blocking=True)
        ev_done[i].record(stream)
    e1.record(stream)
    e1.synchronize()
    e2e_ms = [e0.elapsed_time(e1)]
    barrier()
    e2e_value = whole_job_rate(world, B, args.steps, max_over_ranks(sum(e2e_ms), dev))
    h2d = int(host_flat[0].numel() * 4)
    d2h = int(arena.numel() * 4)
    # the last step's copied-back correspondences equal those of the device-resident steps
    # on the same batch (the timed loop's last step ran batch (steps - 1) % rot as well)
    last = arena_h[(args.steps - 1) % 2]
    n0 = int(matches[0].count.item())
    e2e_same = bool(torch.equal(last[al(ncap):al(ncap) + n0], matches[0].nn_desc[:n0].cpu()))

    # graph form: the step's launches (extract + match of the whole batch, every size
    # group) captured once into a CUDA graph and replayed; the context's plans, tables and
    # workspace already exist from the steps above, so the capture makes no allocation
    graph = None
    if not args.no_graph:
        g = torch.cuda.CUDAGraph()
        gs = torch.cuda.Stream(device=dev)
        gs.wait_stream(stream)
        torch.cuda.synchronize()
        launches_g0 = ctx.launch_count()
        with torch.cuda.graph(g, stream=gs):
            step(devb[0], st=torch.cuda.current_stream())
        glaunches = ctx.launch_count() - launches_g0
        torch.cuda.synchronize()
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.replay()
        e1.record()
        e1.synchronize()
        gms = e0.elapsed_time(e1)
        graph = {"value": whole_job_rate(world, B, args.steps, max_over_ranks(gms, dev)),
                 "unit": "pairs/s", "ms_per_step": gms / args.steps,
                 "kernels_per_graph": glaunches,
                 "form": "one CUDA graph per batch (extract + match of every pair), replayed"}
        del g

    # two-lane form: one context with RIFT2_FLAG_TWO_LANES, called exactly as the headline
    # calls its context; the library forks each call's second half of images (pairs) onto
    # its second stream and joins it back, so that one lane's under-filled stages (top-K
    # sort, median selection, re-rank) overlap the other lane's full-GPU kernels
    lanes = None
    if not args.no_lanes and B >= 2:
        lctx = pkg.Context(pkg.default_params(max_keypoints=max_kp,
                                              flags=pkg.FLAG_AUTOTUNE | pkg.FLAG_TWO_LANES),
                           device=local, hbm_budget=96 << 30)

        def step_lanes(imgs):
            lctx.extract([imgs[i] for i in range(2 * B)], feats, stream=stream)
            lctx.match(feats[0::2], feats[1::2], matches, stream=stream)

        for i in range(args.warmup):
            step_lanes(devb[i % rot])
        lctx.sync()
        barrier()
        l0 = lctx.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.steps):
            step_lanes(devb[i % rot])
        e1.record(stream)
        e1.synchronize()
        lms = e0.elapsed_time(e1)
        barrier()
        lanes = {"value": whole_job_rate(world, B, args.steps, max_over_ranks(lms, dev)),
                 "unit": "pairs/s", "ms_per_step": lms / args.steps,
                 "launches_per_step": (lctx.launch_count() - l0) / args.steps,
                 "form": f"one context with two lanes, {B // 2} + {B - B // 2} pairs per call"}
        lctx.close()

    # plain forms: one pair per call, no launch grouping; with the CUDA-core matcher and
    # with the tensor-core one (the latter isolates the gain from batching)
    def plain_form(flags, label):
        pctx = pkg.Context(pkg.default_params(max_keypoints=MAX_KP, flags=flags),
                           device=local, hbm_budget=16 << 30)
        pf = [pctx.alloc_features() for _ in range(2)]
        pm = [pctx.alloc_matches()]
        lat = []
        for i in range(2 + min(args.steps, 8)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            imgs = devb[i % rot]
            e0.record(stream)
            pctx.extract([imgs[0], imgs[1]], pf, stream=stream)
            pctx.match([pf[0]], [pf[1]], pm, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if i >= 2:
                lat.append(e0.elapsed_time(e1))
        lat.sort()
        pctx.close()
        return {"value": 1000.0 / statistics.mean(lat), "unit": "pairs/s",
                "latency_ms_p50": lat[len(lat) // 2],
                "latency_ms_p99": lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)],
                "form": label}

    plain = plain_tc = None
    if not args.no_plain and args.workload == 1:
        plain = plain_form(pkg.FLAG_PLAIN_MATCH | pkg.FLAG_NO_GROUPING,
                           "one pair per call, no launch grouping, CUDA-core matcher")
        plain_tc = plain_form(pkg.FLAG_NO_GROUPING,
                              "one pair per call, no launch grouping, tensor-core matcher")

    # roofline of the dominant HBM-bound stage
    peak, peak_kind = load_peaks()
    dom = max((k for k in STAGE_BYTES_PER_PX if prof[k][1] > 0), key=lambda k: prof[k][0])
    ms_dom, n_dom = prof[dom]
    imgs_per_launch = 2 * B
    # one launch per same-size group; the bytes of one step's launches over their time
    n_dom = max(1, n_dom // args.steps) * args.steps if args.workload != 2 else args.steps
    bytes_per_launch = STAGE_BYTES_PER_PX[dom] * px_per_step / (n_dom / args.steps)
    achieved = bytes_per_launch / (ms_dom / n_dom / 1000.0) / 1e9
    stage_ms = {k: round(v[0] / args.steps, 4) for k, v in prof.items()}
    # the matching GEMM against the tensor roofline: 2 nA nB 216 flop per pair
    na = [int(f.counts[1].item()) for f in feats[0::2]]
    nb = [int(f.counts[1].item()) for f in feats[1::2]]
    gemm_flop = sum(2.0 * a * b * 216 for a, b in zip(na, nb))
    tpeak, tkind = load_tensor_peak()
    # the match stage's device time per step (all of the step's match launches) against
    # the step's flops
    match_s = prof["match"][0] / args.steps / 1000.0 if prof["match"][1] else float("nan")
    match_tensor = {"bound": "tensor", "achieved": gemm_flop / match_s / 1e12, "peak": tpeak,
                    "peak_kind": tkind, "unit": "TFLOP/s",
                    "frac": gemm_flop / match_s / 1e12 / tpeak,
                    "flop_per_step": gemm_flop, "descriptors": [na, nb],
                    "note": "whole match stage (BF16 prep, tcgen05 GEMM + top-4 screen per column "
                            "half, certified exact re-rank, exhaustive pass for uncertified queries)"}

    # RIFT's own rotation handling on the same batches (§II-C): template descriptors for A,
    # the six-member convolution ring for B, matching A against all ring members
    rift = None
    if not args.no_rift and args.workload == 1:
        rt = pkg.Context(pkg.default_params(max_keypoints=MAX_KP, flags=pkg.FLAG_RIFT_TEMPLATE),
                         device=local, hbm_budget=48 << 30)
        rr = pkg.Context(pkg.default_params(max_keypoints=MAX_KP, flags=pkg.FLAG_RIFT_RING),
                         device=local, hbm_budget=48 << 30)
        fa_t = [rt.alloc_features() for _ in range(B)]
        fb_r = [rr.alloc_features() for _ in range(B)]
        mr = [rr.alloc_matches() for _ in range(B)]

        def rift_step(imgs):
            rt.extract([imgs[2 * i] for i in range(B)], fa_t, stream=stream)
            rr.extract([imgs[2 * i + 1] for i in range(B)], fb_r, stream=stream)
            rr.match(fa_t, fb_r, mr, stream=stream)

        for i in range(2):
            rift_step(devb[i % rot])
        torch.cuda.synchronize()
        rms = []
        for i in range(min(args.steps, 10)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rift_step(devb[i % rot])
            e1.record(stream)
            e1.synchronize()
            rms.append(e0.elapsed_time(e1))
        rift_ms = statistics.mean(rms)
        rift = {"pairs_per_s": B / (rift_ms / 1000.0), "ms_per_step": rift_ms,
                "rift2_speedup": rift_ms / ms_per_step,
                "form": "RIFT baseline: template descriptors for A, six-member ring for B"}
        rt.close()
        rr.close()

    # RIFT's corner keypoints on the minimum moment beside the edge ones (up to twice the
    # keypoints, so more descriptors and a larger matching problem) on the same batches
    corners = None
    if not args.no_rift and args.workload == 1:
        cc = pkg.Context(pkg.default_params(max_keypoints=MAX_KP, flags=pkg.FLAG_CORNERS),
                         device=local, hbm_budget=96 << 30)
        fc = [cc.alloc_features() for _ in range(2 * B)]
        mc = [cc.alloc_matches() for _ in range(B)]

        def corner_step(imgs):
            cc.extract([imgs[i] for i in range(2 * B)], fc, stream=stream)
            cc.match(fc[0::2], fc[1::2], mc, stream=stream)

        for i in range(2):
            corner_step(devb[i % rot])
        torch.cuda.synchronize()
        cms = []
        for i in range(min(args.steps, 10)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            corner_step(devb[i % rot])
            e1.record(stream)
            e1.synchronize()
            cms.append(e0.elapsed_time(e1))
        nkp = [int(f.counts[0].item()) for f in fc]
        corners = {"pairs_per_s": B / (statistics.mean(cms) / 1000.0),
                   "ms_per_step": statistics.mean(cms),
                   "keypoints_per_image": statistics.mean(nkp),
                   "form": "edge keypoints (maximum moment) + corner keypoints (minimum moment)"}
        cc.close()

    serving = serving1024 = None
    if args.serve_requests > 0 and args.workload == 1:
        serving = run_serving(args, local)
    if args.serve1024_requests > 0 and args.workload == 1 and args.serve_requests > 0:
        serving1024 = run_serving_1024(args, local)

    cpu = parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == 1:
        import oracle
        pr = synth.config_pair(1)
        op = oracle.Params(max_keypoints=MAX_KP)
        t0 = time.perf_counter()
        oa = oracle.extract(pr.a.astype(np.float64), op, keep_maps=True)
        ob = oracle.extract(pr.b.astype(np.float64), op, keep_maps=True)
        oracle.match(oa.desc, ob.desc)
        tcpu = time.perf_counter() - t0
        cpu = {"value": 1.0 / tcpu, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "one 1024x1024 pair (2 FP64 oracle extracts keeping their maps + "
                         "brute-force match); numpy FFT runs on one core, the matching matmul "
                         "on the BLAS threads"}
        parity = parity_summary(pkg, dev, pr, oa, ob, oracle.match)

    others = None
    if rank == 0 and world == 1 and args.workload == 1 and not args.no_other_workloads:
        others = {"workload2": workload_summary(pkg, dev, 2), "workload3": workload_summary(pkg, dev, 3)}

    if rank == 0:
        line = {
            "metric": wl["metric"], "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl["desc"], "pairs_per_step": B,
                       "parallelism": f"replicas x{world}",
                       "l2": f"inputs rotate over {rot} batch(es) ({rot * px_per_step * 4 / 1e6:.0f} MB)"
                             " and each step streams ~0.3 KB of workspace per pixel, > L2"},
            "mpix_per_s": value * px_per_step / B / 1e6,
            "plain_form": plain,
            "plain_form_tensor_matcher": plain_tc,
            "graph_form": graph,
            "two_lane_form": lanes,
            "serving": serving,
            "serving_1024": serving1024,
            "rift_baseline": rift,
            "corners_form": corners,
            "stage_ms_per_step": stage_ms,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": measured_traffic(dom, imgs_per_launch) if args.workload == 1 else None,
                         "algorithmic_bytes_per_launch": bytes_per_launch},
            "match_tensor": match_tensor,
            "cpu_baseline": cpu,
            "parity": parity,
            "other_workloads": others,
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                    "form": "pinned host images in (one copy per step, on a copy stream: step "
                            "i+1's copy overlaps step i's kernels); every step copies out each "
                            "pair's full correspondences (q_desc, nn_desc, kp_a, kp_b, d1, d2, "
                            "near_tie, count) and both images' keypoints (xy, score, counts), "
                            "packed in one device arena (one copy per step)",
                    "d2h_bytes_per_step": d2h, "results_equal_device_resident_steps": e2e_same},
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def run_serving(args, device: int):
    """Open-loop Poisson arrivals of pairs of mixed sizes (each side log-uniform in
    [256, 4096], snapped to transform-friendly sizes) through the continuous-batching loop;
    a pool of distinct pairs is generated once and cycled."""
    import synth
    from paper_2303_00319_gb300 import serve
    sizes = synth.serving_sizes(args.serve_pool, seed=synth.pair_seed(4, 0))
    pool = make_pairs([(h, w, synth.pair_seed(4, i + 1)) for i, (h, w) in enumerate(sizes)])
    srv = serve.Server(device=device, max_keypoints=MAX_KP, max_batch_pairs=8,
                       hbm_budget=120 << 30, lanes=2, keep_resident=True)
    warm = [serve.PairRequest(-1 - i, a, b) for i, (a, b) in enumerate(pool)]
    for r in warm:
        srv.submit(r)
    srv.drain()                           # plans, tables, workspaces and pools for every size
    for r in warm:
        srv.release(r.rid)
    pools0 = srv.pool_stats()
    runs = []
    for k, rate in enumerate(float(x) for x in str(args.serve_rate).split(",")):
        reqs = [serve.PairRequest(i, *pool[i % len(pool)]) for i in range(args.serve_requests)]
        runs.append(serve.run_open_loop(srv, reqs, rate=rate, seed=7 + k))
    grown = {k: v - pools0[k] for k, v in srv.pool_stats().items()}
    srv.close()
    return {"workload": (f"{len(pool)} distinct pairs cycled, integer sides log-uniform "
                         f"256..4096 (most with a prime factor above 13: Bluestein transforms), mean "
                         f"{np.mean([a.size for a, _ in pool]) / 1e6:.2f} MPix per image, "
                         "<= 5000 keypoints, HBM admission budget 120 GB (the library's "
                         "workspace figure per batch), each request's features, matches, "
                         "spectra and MIMs device-resident until the client releases them "
                         "on completion"),
            "buffers_created_during_the_runs": grown,
            "rates": runs}


def run_serving_1024(args, device: int):
    """The served form at 1024^2 (the plain forms' size): open-loop Poisson arrivals of
    1024^2 pairs (8 distinct pairs cycled, held in pinned host memory as a client would
    hand them over) through the same continuous-batching loop, at offered rates around and
    above what the plain single-pair forms sustain."""
    import torch

    import synth
    from paper_2303_00319_gb300 import serve
    pool = make_pairs([(H, W, synth.pair_seed(6, i)) for i in range(8)])
    pool = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()) for a, b in pool]
    srv = serve.Server(device=device, max_keypoints=MAX_KP, max_batch_pairs=8,
                       hbm_budget=120 << 30, lanes=2, keep_resident=True)
    warm = [serve.PairRequest(-1 - i, a, b) for i, (a, b) in enumerate(pool * 4)]
    for r in warm:
        srv.submit(r)
    srv.drain()
    for r in warm:
        srv.release(r.rid)
    runs = []
    for k, rate in enumerate(float(x) for x in str(args.serve1024_rate).split(",")):
        reqs = [serve.PairRequest(i, *pool[i % len(pool)]) for i in range(args.serve1024_requests)]
        runs.append(serve.run_open_loop(srv, reqs, rate=rate, seed=17 + k))
    srv.close()
    return {"workload": "1024x1024 pairs (8 distinct, cycled; pinned host images), <= 5000 "
                        "keypoints, up to 8 pairs per batch, two lanes, state resident until "
                        "the client releases it on completion",
            "rates": runs}


def run_probe(spec: str):
    """Per-stage device times of extracting four H x W images of the generator with one
    context (the first call creates the plans and tables; three profiled calls follow):
    the case the ncu summaries of the shared-memory transforms are taken on."""
    import torch

    import paper_2303_00319_gb300 as pkg
    import synth
    from paper_2303_00319_gb300 import _build
    _build.build()
    h, w = (int(v) for v in spec.split(","))
    dev = torch.device("cuda:0")
    imgs = [torch.from_numpy(synth.make_pair(h, w, 100 + i, angle_deg=None).a).to(dev)
            for i in range(4)]
    ctx = pkg.Context(pkg.default_params(max_keypoints=4000), device=0)
    feats = [ctx.alloc_features() for _ in imgs]
    ctx.extract(imgs, feats)
    ctx.sync()
    ctx.set_profiling(True)
    for _ in range(3):
        ctx.extract(imgs, feats)
    ctx.sync()
    st = {k: round(v[0] / 3, 4) for k, v in ctx.profile_read().items()}
    ctx.close()
    print(json.dumps({"probe": f"{h}x{w}", "images": 4, "stage_ms_per_call": st}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--pairs", type=int, default=8, help="pairs per step (1024^2 workload)")
    ap.add_argument("--workload", type=int, default=1, choices=(1, 2, 3),
                    help="1: 1024^2 pairs (headline); 2: uneven batch; 3: 4096^2 scene")
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-rift", action="store_true", help="skip the RIFT-ring baseline")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay form")
    ap.add_argument("--no-lanes", action="store_true", help="skip the two-stream form")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests of the open-loop serving run (0: skip)")
    ap.add_argument("--serve-rate", default="50,100,200,400",
                    help="offered pairs/s, comma-separated for a sweep")
    ap.add_argument("--serve-pool", type=int, default=32, help="distinct pairs generated")
    ap.add_argument("--serve1024-requests", type=int, default=600,
                    help="requests per rate of the 1024^2 serving run (0: skip)")
    ap.add_argument("--serve1024-rate", default="500,1000,2000,4000",
                    help="offered pairs/s of the 1024^2 serving run")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip the uneven-batch and 4096^2 summaries of the default line")
    ap.add_argument("--probe", default=None, metavar="H,W",
                    help="only print the per-stage times of extracting four H x W images")
    args = ap.parse_args()
    if args.probe:
        run_probe(args.probe)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
