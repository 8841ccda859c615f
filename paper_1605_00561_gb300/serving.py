"""A transform server with continuous batching over dwt_batch_submit.

Requests (image, wavelet, storage type, level count, direction) arrive at
any time.  The server admits waiting requests while the device-memory
budget allows (the budget is the free HBM at start-up minus a reserve; a
request costs its output plane plus the LL scratch its batch work area
holds), and whenever fewer than ``max_inflight`` batches are on the GPU it
launches every admitted request as one persistent-kernel batch on the next
of its streams.  Requests that arrive while batches run are admitted as
memory and batch slots free up, so their work overlaps the running
batches on the device.  Completion is observed with CUDA events; a
request's latency is the time from its arrival to the host seeing its
batch done.

``per_request=True`` launches each request alone as it is admitted (one
launch per request), the comparison the batching is measured against.
Results do not depend on the grouping: the batch kernel computes each
request exactly as a batch of one does.

Plans only supply parameters to batches (they own no device memory unless
used for single-image calls), so the server keeps a bounded LRU of them by
shape.  Every transform runs in the library's CUDA kernels; this module
only orders work and memory.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
from typing import Callable, Deque, List, Optional

import torch

from . import dwt

ELEM = {"f32": 4, "f16s": 2, "i32": 4}
TDT = {"f32": torch.float32, "f16s": torch.float16, "i32": torch.int32}


def out_pitch(w: int, dtype: str) -> int:
    """Row pitch (bytes) of a served output: rows padded to 128 bytes, so
    that the kernels store whole aligned vectors and an inverse of the
    output can load its planes by TMA."""
    return (w * ELEM[dtype] + 127) // 128 * 128


@dataclass
class Request:
    """One transform.  ``src`` is a device view of the input (any row pitch);
    ``out`` is a w x h tensor the server fills (a view of its batch's output
    allocation, made when first read)."""
    w: int
    h: int
    levels: int
    wavelet: str = "cdf97"
    dtype: str = "f32"
    inverse: bool = False
    src: Optional[torch.Tensor] = None
    arrival: float = 0.0
    done: Optional[float] = None
    status: int = -1
    cost: int = 0
    tag: object = None
    _slab: Optional[torch.Tensor] = field(default=None, repr=False)
    _off: int = 0
    _out: Optional[torch.Tensor] = field(default=None, repr=False)

    @property
    def out(self) -> Optional[torch.Tensor]:
        if self._out is None and self._slab is not None:
            pitch = out_pitch(self.w, self.dtype)
            rows = self._slab[self._off:self._off + pitch * self.h].view(TDT[self.dtype])
            self._out = rows.view(self.h, pitch // ELEM[self.dtype])[:, :self.w]
        return self._out

    @out.setter
    def out(self, value: Optional[torch.Tensor]) -> None:
        self._out = value
        self._slab = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def request_bytes(r: Request) -> int:
    """Device bytes a request holds while in flight: its output plane (rows
    at a 128-byte pitch) and the LL buffers of its batch work area, one per
    level after the first (ceil(W_k/2) x ceil(H_k/2) elements, rows at a
    128-byte pitch, each buffer starting on a 256-byte boundary), plus a
    bound on its share of the work list: per level a 1 KiB descriptor, an
    8-byte item per strip and 12 bytes per row of strips, for strips of at
    least 2 quadruple rows and 120 columns."""
    es = ELEM[r.dtype]
    total = out_pitch(r.w, r.dtype) * r.h
    w, h = r.w, r.h
    for k in range(r.levels):
        cw, ch = (w + 1) // 2, (h + 1) // 2
        nrs = (ch + 1) // 2
        total += 1024 + 8 * ((cw + 119) // 120) * nrs + 12 * nrs
        if k + 1 < r.levels:
            total += ((cw * es + 127) // 128 * 128 * ch + 255) // 256 * 256
        w, h = cw, ch
    return total


@dataclass
class _Batch:
    event: torch.cuda.Event
    reqs: List[Request]
    status: torch.Tensor  # page-locked host copy, valid once the event completed
    cost: int


class Server:
    def __init__(self, budget_bytes: Optional[int] = None, reserve_bytes: int = 4 << 30,
                 max_inflight: int = 8, max_batch: int = 1024, per_request: bool = False,
                 plan_cache: int = 4096, device: Optional[int] = None,
                 on_done: Optional[Callable[[Request], None]] = None):
        if not torch.cuda.is_available():
            raise RuntimeError("the transform server needs a CUDA device")
        dwt.lib()  # fail loudly without the CUDA library
        self.device = torch.cuda.current_device() if device is None else device
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = max(0, free - reserve_bytes)
        self.budget = int(budget_bytes)
        self.in_use = 0
        self.per_request = per_request
        self.max_inflight = max_inflight if not per_request else max(max_inflight, 64)
        self.max_batch = max_batch
        nstreams = 4 if per_request else max_inflight
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(nstreams)]
        self._next_stream = 0
        self.waiting: Deque[Request] = collections.deque()
        self.inflight: List[_Batch] = []
        self.plans: "collections.OrderedDict[tuple, dwt.Plan]" = collections.OrderedDict()
        self.plan_cache = plan_cache
        self.batches = 0
        self.completed = 0
        # called with each finished request; the output is the caller's from
        # then on and no longer counts against the budget
        self.on_done = on_done

    # -- plans -------------------------------------------------------------
    def _plan(self, r: Request) -> dwt.Plan:
        key = (r.w, r.h, r.levels, r.wavelet, r.dtype)
        p = self.plans.get(key)
        if p is None:
            p = dwt.Plan(r.w, r.h, r.wavelet, r.levels, r.dtype)
            self.plans[key] = p
            while len(self.plans) > self.plan_cache:
                _, old = self.plans.popitem(last=False)
                old.close()  # host-only plan: no device synchronisation
        else:
            self.plans.move_to_end(key)
        return p

    # -- queue -------------------------------------------------------------
    def enqueue(self, r: Request) -> None:
        r.cost = request_bytes(r)
        if r.cost > self.budget:
            raise ValueError(f"request of {r.cost} bytes exceeds the server budget of {self.budget}")
        self.waiting.append(r)

    def busy(self) -> bool:
        return bool(self.waiting or self.inflight)

    def _retire(self, now: float) -> int:
        n = 0
        keep = []
        for b in self.inflight:
            if b.event.query():
                st = b.status.tolist()
                for r, s in zip(b.reqs, st):
                    r.done = now
                    r.status = s
                    if self.on_done is not None:
                        self.on_done(r)
                self.in_use -= b.cost
                self.completed += len(b.reqs)
                n += len(b.reqs)
            else:
                keep.append(b)
        self.inflight = keep
        return n

    def _launch(self, reqs: List[Request], cost: int) -> None:
        stream = self.streams[self._next_stream]
        self._next_stream = (self._next_stream + 1) % len(self.streams)
        with torch.cuda.stream(stream):
            status = torch.empty(len(reqs), dtype=torch.int32, device=self.device)
            # every output of the batch is a view of one allocation (256-byte
            # aligned offsets): one allocator call per batch, not per request
            offs, total = [], 0
            for r in reqs:
                offs.append(total)
                total += (out_pitch(r.w, r.dtype) * r.h + 255) // 256 * 256
            slab = torch.empty(max(total, 256), dtype=torch.uint8, device=self.device)
            base = slab.data_ptr()
            entries = []
            for r, off in zip(reqs, offs):
                es = ELEM[r.dtype]
                r._slab, r._off, r._out = slab, off, None
                entries.append(dwt.DwtRequest(self._plan(r).handle, r.src.data_ptr(), r.src.stride(0) * es,
                                              base + off, out_pitch(r.w, r.dtype), int(r.inverse)))
            dwt.submit(entries, status=status, stream=stream.cuda_stream)
            # read back on the batch's own stream: no synchronisation with
            # the other batches in flight
            host = torch.empty(len(reqs), dtype=torch.int32, pin_memory=True)
            host.copy_(status, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        self.inflight.append(_Batch(ev, reqs, host, cost))
        self.batches += 1

    def pump(self, now: Optional[float] = None) -> int:
        """Retire finished batches, then admit and launch what fits.
        Returns the number of requests completed by this call."""
        now = time.perf_counter() if now is None else now
        done = self._retire(now)
        while self.waiting and len(self.inflight) < self.max_inflight:
            take, cost = [], 0
            while (self.waiting and len(take) < (1 if self.per_request else self.max_batch)
                   and self.in_use + cost + self.waiting[0].cost <= self.budget):
                r = self.waiting.popleft()
                take.append(r)
                cost += r.cost
            if not take:
                break  # memory-bound: wait for a batch to retire
            self.in_use += cost
            self._launch(take, cost)
        return done

    def drain(self) -> None:
        while self.busy():
            self.pump()

    def close(self) -> None:
        torch.cuda.synchronize(self.device)
        for p in self.plans.values():
            p.close()
        self.plans.clear()


def percentile(xs: List[float], q: float) -> float:
    if not xs:
        return float("nan")
    s = sorted(xs)
    k = min(len(s) - 1, max(0, int(round(q / 100.0 * (len(s) - 1)))))
    return s[k]


@dataclass
class ReplayResult:
    requests: List[Request] = field(default_factory=list)
    wall_s: float = 0.0
    batches: int = 0

    def summary(self) -> dict:
        lat = [r.latency for r in self.requests]
        px = sum(r.w * r.h for r in self.requests)
        return {"requests": len(self.requests), "batches": self.batches,
                "p50_ms": percentile(lat, 50) * 1e3, "p99_ms": percentile(lat, 99) * 1e3,
                "mean_ms": sum(lat) / max(len(lat), 1) * 1e3, "gpixel_per_s": px / self.wall_s / 1e9,
                "wall_s": self.wall_s,
                "failed": sum(1 for r in self.requests if r.status != dwt.DWT_OK)}


def replay(server: Server, requests: List[Request], offsets: List[float]) -> ReplayResult:
    """Feed ``requests`` to ``server`` at ``offsets`` seconds after the start
    (real time), pumping continuously, and wait for all of them."""
    t0 = time.perf_counter()
    i, n = 0, len(requests)
    while i < n or server.busy():
        now = time.perf_counter()
        while i < n and offsets[i] <= now - t0:
            requests[i].arrival = t0 + offsets[i]
            server.enqueue(requests[i])
            i += 1
        server.pump(now)
    return ReplayResult(requests=requests, wall_s=time.perf_counter() - t0, batches=server.batches)
