"""Continuous-batching scheduler: admission, ordering and overlap, with a fake
device backend and a manual clock (no GPU)."""
import dataclasses

import pytest

from paper_1905_06700_b300.serve import Backend, Request, Server, SlotLimits, poisson_arrivals, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend(Backend):
    """A batch takes 1 ms plus 1 us per 100 pixels on its slot."""

    def __init__(self, clock, n_slots=2, limits=None):
        self.clock = clock
        self._slots = n_slots
        self._limits = limits or SlotLimits(max_frames=4, max_pixels=3 * 64 * 64, max_entries=10 ** 8,
                                            max_h=256, max_w=256, max_t=4096)
        self.until = {}
        self.launched = []      # (slot, start, end, batch, warm)

    def limits(self):
        return self._limits

    def n_slots(self):
        return self._slots

    def launch(self, slot, batch, warm):
        start = self.clock()
        end = start + 1e-3 + sum(r.pixels for r in batch) * 1e-8
        self.until[slot] = end
        self.launched.append((slot, start, end, list(batch), warm))

    def done(self, slot):
        return self.clock() >= self.until.get(slot, 0.0)


def drive(server, clock, arrivals, dt=1e-4, limit=100000):
    pending = sorted(arrivals, key=lambda r: r.arrival)
    i = 0
    for _ in range(limit):
        while i < len(pending) and pending[i].arrival <= clock.t:
            server.submit(pending[i])
            i += 1
        server.step()
        if len(server.completed) == len(arrivals):
            return server.completed
        clock.t += dt
    raise AssertionError("did not finish")


def _arrivals(n_streams=6, rate=2000.0, duration=0.05, seed=1):
    sizes = [(32, 32, 1024), (64, 64, 1024), (64, 64, 4096), (32, 32, 4096)] * 4
    return poisson_arrivals(n_streams, rate, duration, sizes[:n_streams], seed=seed)


def test_each_stream_has_one_frame_in_flight_and_keeps_its_order():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, clock)
    arr = _arrivals()
    done = drive(srv, clock, arr)
    assert len(done) == len(arr)
    # never two frames of a stream in one batch, never overlapping in time
    for _, start, end, batch, _ in be.launched:
        streams = [r.stream for r in batch]
        assert len(streams) == len(set(streams))
    spans = {}
    for _, start, end, batch, _ in be.launched:
        for r in batch:
            spans.setdefault(r.stream, []).append((r.index, start, end))
    for s, lst in spans.items():
        lst.sort()
        assert [i for i, _, _ in lst] == list(range(len(lst)))      # in order
        for (_, s0, e0), (_, s1, e1) in zip(lst, lst[1:]):
            assert s1 >= e0                                          # previous frame finished first


def test_first_frame_is_cold_and_batches_do_not_mix_cold_and_warm():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, clock)
    drive(srv, clock, _arrivals())
    first = {}
    for _, start, end, batch, warm in be.launched:
        for r in batch:
            if r.stream not in first:
                first[r.stream] = warm
                assert r.index == 0 and warm is False
            else:
                assert warm is True
    assert set(first) == set(range(6))


def test_admission_by_memory_bounds_every_batch():
    clock = FakeClock()
    lim = SlotLimits(max_frames=8, max_pixels=2 * 64 * 64, max_entries=64 * 64 * 4096 + 32 * 32 * 4096,
                     max_h=64, max_w=64, max_t=4096)
    be = FakeBackend(clock, limits=lim)
    srv = Server(be, clock)
    drive(srv, clock, _arrivals(rate=5000.0))
    for _, _, _, batch, _ in be.launched:
        assert sum(r.pixels for r in batch) <= lim.max_pixels
        assert sum(r.pixels * r.t for r in batch) <= lim.max_entries
        assert len(batch) <= lim.max_frames


def test_requests_arriving_during_a_batch_overlap_on_another_slot():
    clock = FakeClock()
    be = FakeBackend(clock, n_slots=2)
    srv = Server(be, clock)
    arr = [Request(0, 0, 64, 64, 1024, 0.0), Request(1, 0, 64, 64, 1024, 2e-4)]
    drive(srv, clock, arr, dt=1e-4)
    (s0, a0, e0, b0, _), (s1, a1, e1, b1, _) = be.launched[:2]
    assert s0 != s1 and a1 < e0            # the second batch started while the first ran
    assert [r.stream for r in b0] == [0] and [r.stream for r in b1] == [1]


def test_latency_accounting_and_summary():
    clock = FakeClock()
    be = FakeBackend(clock)
    srv = Server(be, clock)
    done = drive(srv, clock, _arrivals())
    for r in done:
        assert r.admitted >= r.arrival - 1e-12 and r.done > r.admitted
        assert r.latency >= 1e-3
    s = summarize(done)
    assert s["frames"] == len(done) and s["latency_ms_p99"] >= s["latency_ms_p50"] >= 1.0


def test_oversized_frames_are_rejected_at_submission():
    clock = FakeClock()
    lim = SlotLimits(max_frames=4, max_pixels=64 * 64, max_entries=64 * 64 * 1024,
                     max_h=256, max_w=256, max_t=4096)
    srv = Server(FakeBackend(clock, limits=lim), clock)
    with pytest.raises(ValueError):
        srv.submit(Request(0, 0, 512, 512, 1024, 0.0))      # beyond the frame size
    with pytest.raises(ValueError):
        srv.submit(Request(0, 0, 128, 128, 64, 0.0))        # beyond the slot's pixels
    with pytest.raises(ValueError):
        srv.submit(Request(0, 0, 64, 64, 2048, 0.0))        # beyond the sparse capacity
    srv.submit(Request(0, 0, 64, 64, 1024, 0.0))


def test_admission_by_device_memory_budget():
    """With a device-memory budget for frame data, the frames in flight (their
    dense histograms) plus the streams' resident point clouds never exceed it;
    frames wait in the queue instead, every frame completes, and a frame that
    cannot fit the budget on its own is refused at submission."""
    from paper_1905_06700_b300.serve import input_bytes, state_bytes
    clock = FakeClock()
    arrivals = _arrivals(n_streams=6, rate=4000.0, duration=0.05, seed=3)
    big = max(input_bytes(r) for r in arrivals)
    states = sum(state_bytes(r, 3) for r in {r.stream: r for r in arrivals}.values())
    budget = states + big                         # one of the largest frames in flight at a time
    lim = SlotLimits(max_frames=4, max_pixels=3 * 64 * 64, max_entries=10 ** 8, max_h=256, max_w=256,
                     max_t=4096, mem_budget=budget, k_max=3)
    be = FakeBackend(clock, n_slots=3, limits=lim)
    server = Server(be, clock=clock)
    done = drive(server, clock, arrivals)
    assert len(done) == len(arrivals)
    assert 0 < server.peak_bytes <= budget and server.inflight_bytes == 0
    # the same arrivals without the budget hold more on the device at once
    clock2 = FakeClock()
    free = Server(FakeBackend(clock2, n_slots=3, limits=dataclasses.replace(lim, mem_budget=0)), clock=clock2)
    drive(free, clock2, _arrivals(n_streams=6, rate=4000.0, duration=0.05, seed=3))
    assert free.peak_bytes > budget
    with pytest.raises(ValueError):
        Server(FakeBackend(clock, limits=SlotLimits(4, 10 ** 6, 10 ** 9, 256, 256, 4096, mem_budget=1000)),
               clock=clock).submit(Request(0, 0, 64, 64, 1024, 0.0))
