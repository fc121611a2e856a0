"""Continuous-batching server for streams of lidar frames.

Requests (one frame of one scene stream) arrive over time.  Whenever one of
the server's slots is free, the queued requests that can run form that slot's
next batch and are launched at once (`rt3d_reconstruct_batch` on the slot's
own CUDA stream and context), so batches admitted while others run overlap on
the device.  Admission rules:

  * a stream has at most one frame in flight: its next frame warm-starts from
    the point cloud its previous frame left in device memory;
  * a batch holds frames of one kind (first frames of streams start cold, the
    later ones warm);
  * frames join a batch only while the slot's workspace holds them -- the
    batch's pixels within the context's pixel capacity and its worst-case
    nonzero bins within the context's sparse-entry capacity;
  * with a device-memory budget for frame data (SlotLimits.mem_budget), a
    batch is admitted only while the bytes of the frames in flight (their
    dense histograms) plus the streams' device-resident point clouds stay
    within it (admission by memory: frames wait in the queue, not on the
    device).

The device work is behind a small backend interface so that the scheduling
logic can be exercised without a GPU.  Host logic only: every step of the
method runs in the library's kernels.
"""
from __future__ import annotations

import dataclasses
import heapq
import time
from collections import deque
from typing import Callable, Dict, List, Optional, Sequence


@dataclasses.dataclass
class Request:
    stream: int
    index: int                 # frame number within its stream
    h: int
    w: int
    t: int
    arrival: float             # seconds, on the server's clock
    payload: object = None     # backend data (e.g. the device histogram)
    admitted: float = float("nan")
    done: float = float("nan")

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def pixels(self) -> int:
        return self.h * self.w


@dataclasses.dataclass
class SlotLimits:
    max_frames: int            # frames per batch (the context's max_batch)
    max_pixels: int            # pixels per batch (max_batch * max_h * max_w)
    max_entries: int           # sparse-entry capacity of the context
    max_h: int
    max_w: int
    max_t: int
    mem_budget: int = 0        # device bytes for frame data over all slots (0 = no limit)
    k_max: int = 3             # point slots per pixel (size of a stream's point cloud)


def input_bytes(req: "Request") -> int:
    """Device bytes of a frame's dense histogram while it is in flight."""
    return 2 * req.pixels * req.t


def state_bytes(req: "Request", k_max: int) -> int:
    """Device bytes of a stream's resident point cloud (t, r float32 and an
    alive byte per slot and pixel, a float32 background per pixel)."""
    return req.pixels * (9 * k_max + 4)


class Backend:
    """What the server needs from the device."""

    def limits(self) -> SlotLimits:
        raise NotImplementedError

    def n_slots(self) -> int:
        raise NotImplementedError

    def launch(self, slot: int, batch: List[Request], warm: bool) -> None:
        raise NotImplementedError

    def done(self, slot: int) -> bool:
        raise NotImplementedError


class Server:
    def __init__(self, backend: Backend, clock: Callable[[], float] = time.perf_counter):
        self.backend = backend
        self.clock = clock
        # queued frames per stream, in frame order (a stream's frames run in
        # order, one at a time, so only each stream's oldest can join a batch)
        self.queues: Dict[int, deque] = {}
        self.busy_streams: Dict[int, Request] = {}
        self.started_streams: set = set()
        self.inflight: Dict[int, List[Request]] = {}
        self.completed: List[Request] = []
        self.batches: List[List[Request]] = []
        self.inflight_bytes = 0            # dense inputs of the frames on the device
        self.resident_bytes = 0            # the streams' point clouds
        self.peak_bytes = 0
        self.t0 = clock()

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, req: Request) -> None:
        lim = self.backend.limits()
        if req.h > lim.max_h or req.w > lim.max_w or req.t > lim.max_t \
                or req.pixels > lim.max_pixels or req.pixels * req.t > lim.max_entries \
                or (lim.mem_budget and input_bytes(req) + state_bytes(req, lim.k_max) > lim.mem_budget):
            # a frame that cannot fit a slot (or the memory budget) on its own would wait forever
            raise ValueError(f"frame {req.h}x{req.w}x{req.t} exceeds the server's slot capacity")
        self.queues.setdefault(req.stream, deque()).append(req)

    def queued(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def _form_batch(self) -> Optional[List[Request]]:
        lim = self.backend.limits()
        batch: List[Request] = []
        warm = None
        pixels = entries = 0
        mem = self.inflight_bytes + self.resident_bytes
        # candidates: the oldest queued frame of every stream with none in flight,
        # in arrival order
        heads = [q[0] for st, q in self.queues.items() if q and st not in self.busy_streams]
        heads.sort(key=lambda r: (r.arrival, r.stream, r.index))
        for req in heads:
            # the first frame of a stream starts cold
            req_warm = req.stream in self.started_streams
            if warm is None:
                warm = req_warm
            if req_warm != warm:
                continue
            if pixels + req.pixels > lim.max_pixels or entries + req.pixels * req.t > lim.max_entries:
                continue
            need = input_bytes(req) + (0 if req.stream in self.started_streams else state_bytes(req, lim.k_max))
            if lim.mem_budget and mem + need > lim.mem_budget:
                continue
            batch.append(req)
            pixels += req.pixels
            entries += req.pixels * req.t
            mem += need
            if len(batch) >= lim.max_frames:
                break
        if not batch:
            return None
        for req in batch:
            self.queues[req.stream].popleft()
        self._warm = bool(warm)
        return batch

    def step(self) -> int:
        """Retire finished batches, then admit queued frames into free slots.
        Returns the number of frames completed."""
        finished = 0
        for slot in list(self.inflight):
            if self.backend.done(slot):
                t = self.now()
                for req in self.inflight.pop(slot):
                    req.done = t
                    self.busy_streams.pop(req.stream, None)
                    self.completed.append(req)
                    self.inflight_bytes -= input_bytes(req)
                    finished += 1
        for slot in range(self.backend.n_slots()):
            if slot in self.inflight:
                continue
            batch = self._form_batch()
            if batch is None:
                break
            t = self.now()
            lim = self.backend.limits()
            for req in batch:
                req.admitted = t
                self.busy_streams[req.stream] = req
                self.inflight_bytes += input_bytes(req)
                if req.stream not in self.started_streams:
                    self.resident_bytes += state_bytes(req, lim.k_max)
            self.peak_bytes = max(self.peak_bytes, self.inflight_bytes + self.resident_bytes)
            self.backend.launch(slot, batch, self._warm)
            for req in batch:
                self.started_streams.add(req.stream)
            self.inflight[slot] = batch
            self.batches.append(batch)
        return finished

    def run(self, arrivals: Sequence[Request], timeout_s: float = 600.0) -> List[Request]:
        """Serve requests that arrive at their `arrival` times (seconds from the
        start of the run); returns them completed, in completion order."""
        pending = sorted(arrivals, key=lambda r: r.arrival)
        heap = [(r.arrival, i, r) for i, r in enumerate(pending)]
        heapq.heapify(heap)
        total = len(pending)
        self.t0 = self.clock()
        deadline = self.t0 + timeout_s
        while len(self.completed) < total:
            now = self.now()
            while heap and heap[0][0] <= now:
                self.submit(heapq.heappop(heap)[2])
            self.step()
            if self.clock() > deadline:
                raise TimeoutError(f"served {len(self.completed)} of {total} frames in {timeout_s} s")
        return self.completed


def summarize(done: Sequence[Request]) -> dict:
    import numpy as np
    lat = np.array([r.latency for r in done]) * 1000.0
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"frames": len(done), "frames_per_s": len(done) / span,
            "latency_ms_p50": float(np.percentile(lat, 50)),
            "latency_ms_p99": float(np.percentile(lat, 99)),
            "latency_ms_max": float(lat.max())}


def poisson_arrivals(n_streams: int, rate_hz: float, duration_s: float, sizes, seed: int = 0):
    """Frame requests of n_streams scene streams arriving by one Poisson process
    of total rate rate_hz; stream s has frame size sizes[s] = (h, w, t)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    count = [0] * n_streams
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        s = int(rng.integers(0, n_streams))
        h, w, tt = sizes[s]
        reqs.append(Request(s, count[s], h, w, tt, t))
        count[s] += 1
    return reqs


class GpuBackend(Backend):
    """Slots = (context, CUDA stream, completion event).  Each stream's point
    cloud lives in device buffers owned by the backend and is the warm start
    of the stream's next frame."""

    def __init__(self, n_slots: int, limits: SlotLimits, irf_samples, irf_origin, params: dict,
                 k_max: int, frame_source: Callable[[Request], object], device: int = 0, depth_net=None):
        import torch
        from . import rt3d as R
        self.torch = torch
        self.R = R
        self._limits = limits
        self.params = dict(params)
        self.k_max = k_max
        self.frame_source = frame_source
        self.ctx = [R.Context(limits.max_h, limits.max_w, limits.max_t, k_max, irf_samples, irf_origin,
                              max_batch=limits.max_frames, max_entries=limits.max_entries, device=device)
                    for _ in range(n_slots)]
        # the learned depth denoiser (read-only at inference) serves every slot
        if depth_net is not None:
            for c in self.ctx:
                c.set_depth_net(depth_net)
        self.streams = [torch.cuda.Stream(device=device) for _ in range(n_slots)]
        self.events = [None] * n_slots
        self.slot_batch: Dict[int, List[Request]] = {}
        self.state: Dict[int, dict] = {}
        self.snapshots: Optional[Dict[tuple, dict]] = None    # test hook: inputs per frame
        self.results: Optional[Dict[tuple, dict]] = None      # test hook: outputs per frame

    def limits(self) -> SlotLimits:
        return self._limits

    def n_slots(self) -> int:
        return len(self.ctx)

    def stream_state(self, req: Request) -> dict:
        st = self.state.get(req.stream)
        if st is None:
            st = self.ctx[0].new_result(req.h, req.w, self.k_max)
            self.state[req.stream] = st
        return st

    def launch(self, slot: int, batch: List[Request], warm: bool) -> None:
        torch = self.torch
        s = self.streams[slot]
        frames, outs = [], []
        for req in batch:
            st = self.stream_state(req)
            dense = req.payload if req.payload is not None else self.frame_source(req)
            frames.append(dict(dense=dense))
            outs.append(st)
        prm = dict(self.params, warm_start=1 if warm else 0)
        with torch.cuda.stream(s):
            # the previous work of these streams may have run on another slot
            s.wait_stream(torch.cuda.current_stream())
            if self.snapshots is not None:
                for req, st in zip(batch, outs):
                    self.snapshots[(req.stream, req.index)] = {
                        "warm": warm, "dense": frames[batch.index(req)]["dense"],
                        "state": {k: v.clone() for k, v in st.items()}}
            self.ctx[slot].reconstruct_batch(prm, frames, outs, stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        self.events[slot] = ev
        self.slot_batch[slot] = list(batch)

    def done(self, slot: int) -> bool:
        ev = self.events[slot]
        if ev is not None and not ev.query():
            return False
        if self.results is not None and slot in self.slot_batch:
            for req in self.slot_batch.pop(slot):
                st = self.state[req.stream]
                self.results[(req.stream, req.index)] = {k: v.clone() for k, v in st.items()}
            self.torch.cuda.synchronize()
        return True
