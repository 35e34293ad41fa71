"""Batched, multi-map serving of integration requests, and a launch-shape autotuner.

The serving loop is the batched form of the path: depth frames from several
cameras and LiDARs of different resolutions, each addressed to one of
several device-resident maps, are integrated by `integrate_batch` launches of
up to 32 frames over up to 16 maps.  It is continuous batching:

- requests are admitted in arrival order while the batch being formed has a
  free slot (frames per launch) and the device staging ring has room for the
  request's depth image (admission by HBM footprint); the rest wait;
- the admitted frames are copied from pinned host memory on a copy stream
  (one `stage_frames` call per batch) while the previous batch is still
  integrating on the compute stream, so a batch's copies overlap the GPU
  work of the one before it;
- a batch launches as soon as its copies are enqueued; its staging bytes are
  released when its completion event has fired;
- per-request latency is completion minus arrival (host clock), reported as
  p50 / p99 beside the aggregate voxel-update throughput.

Each map sees its frames in arrival order, so the result of a request stream
is the same alone and in the mix (checked by the test suite).  Everything on
the device runs in the library's kernels; this module only schedules.
"""
from __future__ import annotations

import json
import os
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import FrameDesc, TsdfMap, frame_desc, integrate_batch, stage_frames

MAX_FRAMES = 32
MAX_MAPS = 16


@dataclass
class Request:
    rid: int
    map_id: int
    sensor: dict
    T: np.ndarray
    depth: object          # pinned host torch tensor (float32, contiguous)
    arrival: float = 0.0   # seconds from the start of the run
    done: float = -1.0     # completion time (seconds from the start)

    @property
    def nbytes(self) -> int:
        return int(self.depth.numel()) * 4


class StagingRing:
    """Device byte ring for in-flight depth images (256-byte aligned slices,
    released in allocation order)."""

    def __init__(self, torch, nbytes: int, device):
        self.buf = torch.empty(nbytes // 4, dtype=torch.float32, device=device)
        self.base = self.buf.data_ptr()
        self.cap = nbytes
        self.head = 0      # next free byte
        self.used = 0
        self.live = deque()  # (offset, size) in allocation order

    def alloc(self, nbytes: int):
        size = (nbytes + 255) // 256 * 256
        if size > self.cap:
            raise ValueError("request larger than the staging budget")
        if self.used + size > self.cap:
            return None
        off = self.head
        if off + size > self.cap:  # wrap: skip the tail
            waste = self.cap - off
            if self.used + waste + size > self.cap:
                return None
            self.live.append((off, waste))
            self.used += waste
            off = 0
        self.live.append((off, size))
        self.used += size
        self.head = (off + size) % self.cap
        return off, size

    def release(self, count: int):
        for _ in range(count):
            _, size = self.live.popleft()
            self.used -= size

    def view(self, off: int, n_floats: int):
        return self.buf[off // 4: off // 4 + n_floats]


@dataclass
class _Batch:
    reqs: list
    event: object
    ring_slices: int


class Server:
    """Continuous-batching integration server over device-resident maps."""

    def __init__(self, maps: list, staging_bytes: int = 256 << 20, max_frames: int = MAX_FRAMES,
                 max_in_flight: int = 4):
        import torch
        self.torch = torch
        self.maps = maps
        self.max_frames = min(max_frames, MAX_FRAMES)
        self.max_in_flight = max_in_flight
        dev = torch.device("cuda", torch.cuda.current_device())
        self.ring = StagingRing(torch, staging_bytes, dev)
        self.copy_stream = torch.cuda.Stream()
        self.compute_stream = torch.cuda.Stream()
        self.pending = deque()
        self.in_flight = deque()
        self.completed = []
        self.t0 = time.perf_counter()
        self.launches = 0

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, req: Request):
        self.pending.append(req)

    def _admit(self, now: float):
        """Admit arrived requests in order while slots and staging memory last."""
        batch, slices, maps = [], 0, set()
        while self.pending and len(batch) < self.max_frames:
            r = self.pending[0]
            if r.arrival > now:
                break
            if r.map_id not in maps and len(maps) == MAX_MAPS:
                break
            ring_before = len(self.ring.live)
            got = self.ring.alloc(r.nbytes)
            if got is None:
                break  # staging memory full: wait for a batch to complete
            slices += len(self.ring.live) - ring_before
            self.pending.popleft()
            r._slot = got
            batch.append(r)
            maps.add(r.map_id)
        return batch, slices

    def _launch(self, batch, slices):
        torch = self.torch
        # the batch's images into their ring slices: one library call
        for r in batch:
            r._dev = self.ring.base + r._slot[0]
        stage_frames([r.depth.data_ptr() for r in batch], [r._dev for r in batch],
                     [r.nbytes for r in batch], self.copy_stream)
        copied = torch.cuda.Event()
        copied.record(self.copy_stream)
        self.compute_stream.wait_event(copied)
        # maps of this batch in first-appearance order; frames in arrival order
        order, index = [], {}
        for r in batch:
            if r.map_id not in index:
                index[r.map_id] = len(order)
                order.append(r.map_id)
        descs = [frame_desc(index[r.map_id], r.sensor, r.T, r._dev) for r in batch]
        with torch.cuda.stream(self.compute_stream):
            integrate_batch([self.maps[m].handle for m in order], descs)
            ev = torch.cuda.Event()
            ev.record(self.compute_stream)
        self.launches += 1
        self.in_flight.append(_Batch(batch, ev, slices))

    def _retire(self, block: bool):
        while self.in_flight:
            b = self.in_flight[0]
            if block:
                b.event.synchronize()
            elif not b.event.query():
                return
            t = self.now()
            for r in b.reqs:
                r.done = t
                r._dev = None
            self.ring.release(b.ring_slices)
            self.completed.extend(b.reqs)
            self.in_flight.popleft()
            block = False

    def run(self, requests, paced: bool = True):
        """Serve `requests` (sorted by arrival).  paced: arrivals follow the
        wall clock from now on; else every request is available at once."""
        for r in requests:
            self.submit(r)
        self.t0 = time.perf_counter()
        while self.pending or self.in_flight:
            self._retire(block=False)
            now = self.now() if paced else float("inf")
            if len(self.in_flight) < self.max_in_flight:
                batch, slices = self._admit(now)
                if batch:
                    self._launch(batch, slices)
                    continue
            if self.in_flight:
                # nothing admissible right now: wait for the oldest batch,
                # unless the next arrival comes first
                if paced and self.pending and len(self.in_flight) < self.max_in_flight:
                    wait = self.pending[0].arrival - self.now()
                    if wait > 0:
                        time.sleep(min(wait, 2e-4))
                    continue
                self._retire(block=True)
            elif self.pending:
                wait = self.pending[0].arrival - self.now()
                if wait > 0:
                    time.sleep(min(wait, 1e-3))
        self.torch.cuda.synchronize()
        return self.completed

    @staticmethod
    def latency_stats(done):
        lat = np.array([r.done - r.arrival for r in done]) * 1e3
        if len(lat) == 0:
            return {"p50_ms": None, "p99_ms": None, "max_ms": None}
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max())}


# ---------------------------------------------------------------- autotuner

_TUNE_CACHE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           ".synth_cache", "autotune.json")


def autotune(name: str, run_fn, candidates, repeats: int = 3, cache: bool = True):
    """Pick the fastest launch shape for a workload.

    run_fn(cfg) runs the workload once with launch-shape config `cfg` (a dict
    of map options and frames per launch) and returns its device time in ms;
    each candidate is timed `repeats` times (after one warm-up) and the one
    with the smallest median wins.  Results are cached per workload name and
    GPU under .synth_cache/autotune.json.
    """
    import torch
    key = f"{name}|{torch.cuda.get_device_name()}"
    table = {}
    if cache and os.path.exists(_TUNE_CACHE):
        try:
            with open(_TUNE_CACHE) as fh:
                table = json.load(fh)
        except Exception:
            table = {}
    if cache and key in table:
        return table[key]["best"], table[key]["timings"]
    timings = []
    for cfg in candidates:
        run_fn(cfg)
        ts = sorted(run_fn(cfg) for _ in range(repeats))
        timings.append({"cfg": cfg, "ms": ts[len(ts) // 2]})
    best = min(timings, key=lambda x: x["ms"])["cfg"]
    if cache:
        os.makedirs(os.path.dirname(_TUNE_CACHE), exist_ok=True)
        table[key] = {"best": best, "timings": timings}
        with open(_TUNE_CACHE, "w") as fh:
            json.dump(table, fh, indent=1)
    return best, timings


def launch_shape_candidates(frames_per_launch=(8, 16, 32), tile_h=(16, 32), ctas_per_sm=(0, 6)):
    return [{"frames_per_launch": f, "alloc_tile_h": t, "integrate_ctas_per_sm": c}
            for f in frames_per_launch for t in tile_h for c in ctas_per_sm]
