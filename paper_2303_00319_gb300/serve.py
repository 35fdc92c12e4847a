"""Continuous-batching request loop over the RIFT2 C ABI.

Requests are image pairs of any supported size.  They are admitted in arrival order as
device memory and batch slots free up, batched into shared launches (one extract call
per batch, in which the library runs images of any sizes in one launch per stage), and run
on one of several lanes; each lane
is a context (own workspace) with its own CUDA stream, so a batch that is admitted while
another one is on the GPU overlaps with it on the device.  Per request the loop records
arrival, admission, launch and completion times (host clock; completion is when the
request's results are back in host memory).

Device-resident state.  With keep_resident, every finished request keeps its features
(keypoints, descriptors), its matches and both images' spectrum and maximum index map on
the device until the caller releases it (release(rid)); the bytes it holds count against
the HBM budget, so new requests wait (back-pressure) while the resident budget is full.

Memory.  Admission asks the library how much workspace a batch needs
(rift2_workspace_bytes) and never admits more than a lane's share of the budget; pinned
host staging, device input buffers, feature and match buffers come from pools keyed by
image size and are reused across requests, so steady-state serving allocates nothing.

All computation runs in the library's kernels; this module only schedules, copies and
keeps time.  The per-image kernels are deterministic and independent of what else shares
a launch, so a request's results are the same alone and in a mixed batch.
"""
from __future__ import annotations

import math
import time
from collections import defaultdict, deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import FLAG_AUTOTUNE, Context, default_params


@dataclass
class PairRequest:
    rid: int
    a: np.ndarray            # float32 [H][W] in [0, 1] (or a pinned host tensor: no staging copy)
    b: np.ndarray
    arrival: float = 0.0     # seconds, host clock
    admitted: float = math.nan
    launched: float = math.nan
    done: float = math.nan
    result: dict | None = None

    @property
    def pixels(self) -> int:
        return int(np.prod(self.a.shape) + np.prod(self.b.shape))


@dataclass
class Resident:
    """Device state a finished request keeps until release: features of A and B (with
    their spectrum and MIM attached as .debug), the matches A -> B."""
    fa: object
    fb: object
    matches: object
    nbytes: int


@dataclass
class _Lane:
    ctx: Context
    stream: torch.cuda.Stream
    batch: list = field(default_factory=list)
    event: torch.cuda.Event | None = None
    outputs: list = field(default_factory=list)
    inputs: list = field(default_factory=list)
    state: list = field(default_factory=list)


class _Pool:
    """Free lists of reusable buffers keyed by a hashable shape."""

    def __init__(self, make):
        self.make = make
        self.free = defaultdict(list)
        self.created = 0

    def take(self, key):
        lst = self.free[key]
        if lst:
            return lst.pop()
        self.created += 1
        return self.make(key)

    def give(self, key, obj):
        self.free[key].append(obj)


def _state_bytes(h: int, w: int, feat_bytes: int) -> int:
    return h * w * (8 + 1) + feat_bytes   # spectrum complex64 + MIM uint8 + features


class Server:
    """Admits pairs by HBM budget and batch size, runs them on `lanes` overlapping lanes.

    hbm_budget covers the lanes' workspaces (resident_fraction of it is reserved for the
    requests' device-resident state when keep_resident is set)."""

    def __init__(self, device: int = 0, max_keypoints: int = 5000, max_batch_pairs: int = 8,
                 hbm_budget: int = 64 << 30, lanes: int = 2, keep_resident: bool = False,
                 resident_fraction: float = 0.25):
        self.device = device
        self.max_batch = max_batch_pairs
        self.budget = hbm_budget
        self.dev = torch.device(f"cuda:{device}")
        self.keep_resident = keep_resident
        self.resident_budget = int(hbm_budget * resident_fraction) if keep_resident else 0
        per_lane = (hbm_budget - self.resident_budget) // lanes
        self.lanes = [_Lane(Context(default_params(max_keypoints=max_keypoints, flags=FLAG_AUTOTUNE),
                                    device, per_lane),
                            torch.cuda.Stream(device=self.dev)) for _ in range(lanes)]
        self.per_lane_budget = per_lane
        self.queue: deque[PairRequest] = deque()
        self.finished: list[PairRequest] = []
        self.resident: dict[int, Resident] = {}
        self.resident_bytes = 0
        ctx0 = self.lanes[0].ctx
        f = ctx0.alloc_features()
        m = ctx0.alloc_matches()
        self._feat_bytes = sum(t.numel() * t.element_size() for t in
                               (f.kp_xy, f.kp_score, f.desc, f.desc_norm, f.desc_kp, f.desc_dom,
                                f.counts))
        self._match_bytes = sum(t.numel() * t.element_size() for t in
                                (m.q_desc, m.nn_desc, m.kp_a, m.kp_b, m.d1, m.d2, m.near_tie,
                                 m.count))
        del f, m
        self._pinned_in = _Pool(lambda hw: torch.empty(hw, dtype=torch.float32).pin_memory())
        self._dev_in = _Pool(lambda hw: torch.empty(hw, dtype=torch.float32, device=self.dev))
        self._feats = _Pool(lambda key: ctx0.alloc_features())
        self._matches = _Pool(lambda key: ctx0.alloc_matches())
        self._host_out = _Pool(self._make_host_out)
        self._maps = _Pool(lambda hw: {"mim": torch.empty(hw, dtype=torch.uint8, device=self.dev),
                                       "spectrum": torch.empty(hw, dtype=torch.complex64,
                                                               device=self.dev)})
        self._ws_cache: dict[tuple, int] = {}

    # ------------------------------------------------------------------ requests
    def submit(self, req: PairRequest, now: float | None = None):
        req.arrival = time.perf_counter() if now is None else now
        self.queue.append(req)

    def release(self, rid: int):
        """Frees a finished request's device-resident state (its buffers return to the
        pools)."""
        st = self.resident.pop(rid, None)
        if st is None:
            return
        self.resident_bytes -= st.nbytes
        for f in (st.fa, st.fb):
            self._maps.give(tuple(f.debug["mim"].shape), f.debug)
            f.debug = None
            self._feats.give(0, f)
        self._matches.give(0, st.matches)

    def _workspace(self, ctx: Context, sizes: tuple, npairs: int) -> int:
        key = (sizes, npairs)
        if key not in self._ws_cache:
            self._ws_cache[key] = ctx.workspace_bytes(list(sizes), npairs)
        return self._ws_cache[key]

    def _resident_need(self, r: PairRequest) -> int:
        if not self.keep_resident:
            return 0
        h, w = r.a.shape
        return 2 * _state_bytes(h, w, self._feat_bytes) + self._match_bytes

    def _take_batch(self, lane: _Lane) -> list[PairRequest]:
        """Requests in arrival order while the batch's workspace (the library's own
        figure for the grouped extract + match) fits the lane and their resident state fits
        what the resident budget has left."""
        batch, sizes, res = [], [], 0
        while self.queue and len(batch) < self.max_batch:
            r = self.queue[0]
            need_res = self._resident_need(r)
            if self.keep_resident and self.resident_bytes + res + need_res > self.resident_budget:
                break                     # back-pressure until the caller releases state
            trial = sizes + [r.a.shape, r.b.shape]
            order = tuple(sorted(trial))  # the library orders a call's images by size too
            if self._workspace(lane.ctx, order, len(batch) + 1) > self.per_lane_budget:
                if batch:
                    break
                # alone it does not fit a lane: fail it rather than the whole loop
                self.queue.popleft()
                r.admitted = r.launched = r.done = time.perf_counter()
                r.result = {"error": "workspace of this pair exceeds the lane's HBM budget"}
                self.finished.append(r)
                continue
            batch.append(self.queue.popleft())
            sizes, res = trial, res + need_res
        return batch

    # -------------------------------------------------------------------- lanes
    def _make_host_out(self, key):
        ncap, kcap = key
        return {k: torch.empty(n, dtype=dt).pin_memory() for k, n, dt in (
            ("nn_desc", ncap, torch.int32), ("d1", ncap, torch.float32),
            ("d2", ncap, torch.float32), ("count", 1, torch.int32),
            ("kp_a", 2 * kcap, torch.int32), ("kp_b", 2 * kcap, torch.int32),
            ("counts_a", 2, torch.int32), ("counts_b", 2, torch.int32),
            ("desc_kp_a", ncap, torch.int32))}

    def _launch(self, lane: _Lane, batch: list[PairRequest]):
        now = time.perf_counter()
        for r in batch:
            r.admitted = now
        ctx = lane.ctx
        with torch.cuda.stream(lane.stream):
            imgs, inputs = [None] * (2 * len(batch)), []
            for j in range(2 * len(batch)):
                r = batch[j // 2]
                x = r.a if j % 2 == 0 else r.b
                hw = tuple(x.shape)
                d = self._dev_in.take(hw)
                if isinstance(x, torch.Tensor) and x.is_pinned():
                    ph = None                 # already in pinned host memory
                    d.copy_(x, non_blocking=True)
                else:
                    ph = self._pinned_in.take(hw)
                    ph.numpy()[...] = x
                    d.copy_(ph, non_blocking=True)
                imgs[j] = d
                inputs.append((hw, ph, d))
            feats = [self._feats.take(0) for _ in imgs]
            for j, f in enumerate(feats):
                f.debug = self._maps.take(tuple(imgs[j].shape)) if self.keep_resident else None
            matches = [self._matches.take(0) for _ in batch]
            for r in batch:
                r.launched = time.perf_counter()
            ctx.extract(imgs, feats, stream=lane.stream)
            ctx.match(feats[0::2], feats[1::2], matches, stream=lane.stream)
            outs = []
            ncap, kcap = matches[0].nn_desc.shape[0], feats[0].kp_xy.shape[0]
            for i, m in enumerate(matches):
                fa, fb = feats[2 * i], feats[2 * i + 1]
                o = self._host_out.take((ncap, kcap))
                for k, v in (("nn_desc", m.nn_desc), ("d1", m.d1), ("d2", m.d2),
                             ("count", m.count), ("kp_a", fa.kp_xy.view(-1)),
                             ("kp_b", fb.kp_xy.view(-1)), ("counts_a", fa.counts),
                             ("counts_b", fb.counts), ("desc_kp_a", fa.desc_kp)):
                    o[k].copy_(v, non_blocking=True)
                outs.append(o)
            ev = torch.cuda.Event()
            ev.record(lane.stream)
        lane.batch, lane.event, lane.outputs = batch, ev, outs
        lane.inputs, lane.state = inputs, (feats, matches)

    def _drain(self, lane: _Lane, block: bool) -> bool:
        if not lane.batch:
            return False
        if not block and not lane.event.query():
            return False
        lane.event.synchronize()
        lane.ctx.sync(lane.stream)
        now = time.perf_counter()
        feats, matches = lane.state
        ncap, kcap = matches[0].nn_desc.shape[0], feats[0].kp_xy.shape[0]
        for i, (r, o) in enumerate(zip(lane.batch, lane.outputs)):
            n = int(o["count"][0])
            na, nb = int(o["counts_a"][0]), int(o["counts_b"][0])
            r.result = {"nn_desc": o["nn_desc"][:n].numpy().copy(),
                        "d1": o["d1"][:n].numpy().copy(), "d2": o["d2"][:n].numpy().copy(),
                        "kp_a": o["kp_a"][:2 * na].numpy().reshape(-1, 2).copy(),
                        "kp_b": o["kp_b"][:2 * nb].numpy().reshape(-1, 2).copy(),
                        "desc_kp_a": o["desc_kp_a"][:n].numpy().copy()}
            r.done = now
            self._host_out.give((ncap, kcap), o)
            if self.keep_resident:
                need = self._resident_need(r)
                self.resident[r.rid] = Resident(feats[2 * i], feats[2 * i + 1], matches[i], need)
                self.resident_bytes += need
            else:
                self._feats.give(0, feats[2 * i])
                self._feats.give(0, feats[2 * i + 1])
                self._matches.give(0, matches[i])
            self.finished.append(r)
        for hw, ph, d in lane.inputs:
            if ph is not None:
                self._pinned_in.give(hw, ph)
            self._dev_in.give(hw, d)
        lane.batch, lane.event, lane.outputs, lane.inputs, lane.state = [], None, [], [], []
        return True

    def step(self, block: bool = False) -> bool:
        """Completes finished lanes, then launches queued work on idle lanes."""
        progressed = False
        for lane in self.lanes:
            progressed |= self._drain(lane, block=False)
        for lane in self.lanes:
            if not lane.batch and self.queue:
                batch = self._take_batch(lane)
                if batch:
                    self._launch(lane, batch)
                    progressed = True
        if block and not progressed:
            busy = [ln for ln in self.lanes if ln.batch]
            if busy:
                self._drain(min(busy, key=lambda ln: ln.batch[0].admitted), block=True)
                progressed = True
        return progressed

    def drain(self):
        while self.queue or any(ln.batch for ln in self.lanes):
            if not self.step(block=True) and self.queue and not any(ln.batch for ln in self.lanes):
                raise RuntimeError("queued requests cannot be admitted: release resident "
                                   "state or raise the budget")

    def pool_stats(self) -> dict:
        """Buffers each pool has created (steady state: no growth)."""
        return {k: p.created for k, p in (("pinned_in", self._pinned_in), ("dev_in", self._dev_in),
                                          ("features", self._feats), ("matches", self._matches),
                                          ("host_out", self._host_out))}

    def close(self):
        for ln in self.lanes:
            ln.ctx.close()


def run_open_loop(server: Server, requests: list[PairRequest], rate: float, seed: int = 0,
                  release: bool = True):
    """Open-loop Poisson arrivals at `rate` pairs/s (exponential gaps), served continuously;
    a finished request's resident state is released as soon as it completes (the client has
    consumed it) unless release is False.  Returns latency percentiles and throughput."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=len(requests))
    t0 = time.perf_counter()
    due = t0 + np.cumsum(gaps)
    i = 0
    seen = len(server.finished)
    while i < len(requests) or server.queue or any(ln.batch for ln in server.lanes):
        now = time.perf_counter()
        while i < len(requests) and due[i] <= now:
            server.submit(requests[i], now=due[i])
            i += 1
        progressed = server.step(block=False)
        if release:
            for r in server.finished[seen:]:
                server.release(r.rid)
            seen = len(server.finished)
        if not progressed:
            time.sleep(5e-5)
    t1 = time.perf_counter()
    lat = np.array(sorted(r.done - r.arrival for r in requests)) * 1e3
    pct = lambda p: float(lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)])  # noqa: E731
    return {"requests": len(requests), "rate_offered": rate,
            "pairs_per_s": len(requests) / (t1 - t0),
            "mpix_per_s": sum(r.pixels for r in requests) / 1e6 / (t1 - t0),
            "latency_ms_p50": pct(0.50), "latency_ms_p99": pct(0.99),
            "latency_ms_p999": pct(0.999), "latency_ms_max": float(lat[-1])}
