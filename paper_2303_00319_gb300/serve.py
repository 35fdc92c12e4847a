"""Continuous-batching request loop over the RIFT2 C ABI.

Requests are image pairs of any supported size.  They are admitted in arrival order as
device memory and batch slots free up, grouped into shared launches (the library groups
equal-size images inside one extract call), and run on one of several lanes; each lane
is a context (own workspace) with its own CUDA stream, so a batch that is admitted while
another one is on the GPU overlaps with it on the device.  Per request the loop records
arrival, admission, launch and completion times (host clock; completion is when the
request's results are back in host memory).

All computation runs in the library's kernels; this module only schedules, copies and
keeps time.  The per-image kernels are deterministic and independent of what else shares
a launch, so a request's results are the same alone and in a mixed batch.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import FLAG_AUTOTUNE, Context, default_params

# Workspace bytes per pixel of one image in an extract launch (spectrum, 24 responses,
# PC terms, maps, candidates) plus a margin; used for admission against the budget.
WS_BYTES_PER_PX = 300


@dataclass
class PairRequest:
    rid: int
    a: np.ndarray            # float32 [H][W] in [0, 1]
    b: np.ndarray
    arrival: float = 0.0     # seconds, host clock
    admitted: float = math.nan
    launched: float = math.nan
    done: float = math.nan
    result: dict | None = None

    @property
    def pixels(self) -> int:
        return int(self.a.size + self.b.size)


@dataclass
class _Lane:
    ctx: Context
    stream: torch.cuda.Stream
    batch: list = field(default_factory=list)
    event: torch.cuda.Event | None = None
    outputs: list = field(default_factory=list)


class Server:
    """Admits pairs by HBM budget and batch size, runs them on `lanes` overlapping lanes."""

    def __init__(self, device: int = 0, max_keypoints: int = 5000, max_batch_pairs: int = 8,
                 hbm_budget: int = 64 << 30, lanes: int = 2):
        self.device = device
        self.max_batch = max_batch_pairs
        self.budget = hbm_budget
        self.dev = torch.device(f"cuda:{device}")
        per_lane = hbm_budget // lanes
        self.lanes = [_Lane(Context(default_params(max_keypoints=max_keypoints, flags=FLAG_AUTOTUNE),
                                    device, per_lane),
                            torch.cuda.Stream(device=self.dev)) for _ in range(lanes)]
        self.per_lane_budget = per_lane
        self.queue: deque[PairRequest] = deque()
        self.finished: list[PairRequest] = []

    # ------------------------------------------------------------------ requests
    def submit(self, req: PairRequest, now: float | None = None):
        req.arrival = time.perf_counter() if now is None else now
        self.queue.append(req)

    def _bytes(self, req: PairRequest) -> int:
        return req.pixels * WS_BYTES_PER_PX

    def _take_batch(self) -> list[PairRequest]:
        batch, used = [], 0
        while self.queue and len(batch) < self.max_batch:
            r = self.queue[0]
            need = self._bytes(r)
            if batch and used + need > self.per_lane_budget:
                break
            batch.append(self.queue.popleft())
            used += need
        return batch

    # -------------------------------------------------------------------- lanes
    def _launch(self, lane: _Lane, batch: list[PairRequest]):
        now = time.perf_counter()
        for r in batch:
            r.admitted = now
        ctx = lane.ctx
        with torch.cuda.stream(lane.stream):
            imgs = []
            for r in batch:
                for x in (r.a, r.b):
                    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).pin_memory()
                    imgs.append(t.to(self.dev, non_blocking=True))
            feats = [ctx.alloc_features() for _ in imgs]
            matches = [ctx.alloc_matches() for _ in batch]
            for r in batch:
                r.launched = time.perf_counter()
            ctx.extract(imgs, feats, stream=lane.stream)
            ctx.match(feats[0::2], feats[1::2], matches, stream=lane.stream)
            outs = []
            for i, m in enumerate(matches):
                fa, fb = feats[2 * i], feats[2 * i + 1]
                o = {}
                for k, v in (("nn_desc", m.nn_desc), ("d1", m.d1), ("d2", m.d2),
                             ("count", m.count), ("kp_a", fa.kp_xy), ("kp_b", fb.kp_xy),
                             ("counts_a", fa.counts), ("counts_b", fb.counts),
                             ("desc_kp_a", fa.desc_kp)):
                    h = torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                    h.copy_(v, non_blocking=True)
                    o[k] = h
                outs.append(o)
            ev = torch.cuda.Event()
            ev.record(lane.stream)
        lane.batch, lane.event, lane.outputs = batch, ev, outs
        lane.keep = (imgs, feats, matches)   # device buffers live until the lane is drained

    def _drain(self, lane: _Lane, block: bool) -> bool:
        if not lane.batch:
            return False
        if not block and not lane.event.query():
            return False
        lane.event.synchronize()
        lane.ctx.sync(lane.stream)
        now = time.perf_counter()
        for r, o in zip(lane.batch, lane.outputs):
            n = int(o["count"][0])
            na, nb = int(o["counts_a"][0]), int(o["counts_b"][0])
            r.result = {"nn_desc": o["nn_desc"][:n].numpy(), "d1": o["d1"][:n].numpy(),
                        "d2": o["d2"][:n].numpy(), "kp_a": o["kp_a"][:na].numpy(),
                        "kp_b": o["kp_b"][:nb].numpy(), "desc_kp_a": o["desc_kp_a"][:n].numpy()}
            r.done = now
            self.finished.append(r)
        lane.batch, lane.event, lane.outputs, lane.keep = [], None, [], None
        return True

    def step(self, block: bool = False) -> bool:
        """Completes finished lanes, then launches queued work on idle lanes."""
        progressed = False
        for lane in self.lanes:
            progressed |= self._drain(lane, block=False)
        for lane in self.lanes:
            if not lane.batch and self.queue:
                self._launch(lane, self._take_batch())
                progressed = True
        if block and not progressed:
            busy = [ln for ln in self.lanes if ln.batch]
            if busy:
                self._drain(min(busy, key=lambda ln: ln.batch[0].admitted), block=True)
                progressed = True
        return progressed

    def drain(self):
        while self.queue or any(ln.batch for ln in self.lanes):
            self.step(block=True)

    def close(self):
        for ln in self.lanes:
            ln.ctx.close()


def run_open_loop(server: Server, requests: list[PairRequest], rate: float, seed: int = 0):
    """Open-loop Poisson arrivals at `rate` pairs/s (exponential gaps), served continuously.
    Returns latency percentiles and throughput."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=len(requests))
    t0 = time.perf_counter()
    due = t0 + np.cumsum(gaps)
    i = 0
    while i < len(requests) or server.queue or any(ln.batch for ln in server.lanes):
        now = time.perf_counter()
        while i < len(requests) and due[i] <= now:
            server.submit(requests[i], now=due[i])
            i += 1
        if not server.step(block=False):
            time.sleep(5e-5)
    t1 = time.perf_counter()
    lat = np.array(sorted(r.done - r.arrival for r in requests)) * 1e3
    pct = lambda p: float(lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)])  # noqa: E731
    return {"requests": len(requests), "rate_offered": rate,
            "pairs_per_s": len(requests) / (t1 - t0),
            "mpix_per_s": sum(r.pixels for r in requests) / 1e6 / (t1 - t0),
            "latency_ms_p50": pct(0.50), "latency_ms_p99": pct(0.99),
            "latency_ms_p999": pct(0.999), "latency_ms_max": float(lat[-1])}
