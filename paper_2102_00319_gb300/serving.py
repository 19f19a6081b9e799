"""Continuous-batching request loop for single-ciphertext encrypted inference.

Requests are single-ciphertext CNN inferences (an image packed in one
ciphertext, a 3x3 convolution by rotations with the model owner's encrypted
filter, then x^2), each at the ring degree and level of its client.  Keys,
weights and request ciphertexts stay resident in device memory.  The loop:

* admits queued requests while the estimated device footprint of everything
  in flight stays under a budget (admission by HBM footprint),
* groups the admitted requests by ring degree and launches one batched step
  per group (hc_enc_conv2d_single_batch or its hoisted form, then x^2) without waiting
  for earlier steps, so work of successive admissions overlaps on the GPU,
* retires a step when its CUDA event has completed (with a stream per ring
  degree, the events of all the streams: `AllOf`) and records each
  request's latency from arrival to completion.

All computation runs in libhecnn; this module only schedules calls.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np

from . import hecnn as H


@dataclass
class Model:
    """Device-resident key set and encrypted filter of one ring degree."""
    ctx: object
    evk: object
    weights: list   # kh*kw slot-constant ciphertexts
    n: int
    n_special: int
    width: int = 8
    kh: int = 3
    kw: int = 3
    hoisted: bool = False   # rotations hoisted (one ModUp per image) or plain


@dataclass
class Request:
    rid: int
    log_n: int
    ct: object          # device-resident input ciphertext
    arrival: float      # seconds (loop clock)
    admitted: float = -1.0
    done: float = -1.0
    result: object = None


def footprint_bytes(model: Model, level: int) -> int:
    """Device bytes one request holds while in flight: input, kh*kw rotated
    copies, the rotations' key-switch workspaces, tensor outputs and the
    outputs.  Plain rotations: kh*kw - 1 automorphed copies, each with a
    whole key-switch workspace (one batched key switch over the steps).
    Hoisted: one coefficient copy of c1 and its raised digits, then per step
    the key product and ModDown's conversion."""
    n, nq = model.n, level + 1
    alpha = model.n_special
    nxt = nq + alpha
    dnum = -(-nq // alpha)
    limb = 8 * n
    ct = 2 * nq * limb
    taps = model.kh * model.kw
    rotated = taps * ct
    outs = 3 * nq * limb + 2 * ct
    if model.hoisted:
        raised = (nq + dnum * nxt) * limb
        per_step = (2 * nxt + 2 * nq) * limb
        return ct + rotated + raised + (taps - 1) * per_step + outs
    ks = (nq + dnum * nxt + 2 * nxt + 2 * nq + 2) * limb
    return ct + rotated + (taps - 1) * (ct + ks) + outs


@dataclass
class _Step:
    event: object
    requests: list
    outputs: list
    bytes: int


@dataclass
class Server:
    models: dict                # log_n -> Model
    budget_bytes: int
    max_batch: int = 64
    clock: object = time.perf_counter
    queue: list = field(default_factory=list)
    inflight: list = field(default_factory=list)
    used_bytes: int = 0
    peak_bytes: int = 0
    done: list = field(default_factory=list)
    budget_waits: int = 0       # ticks on which the queue head did not fit the budget

    def submit(self, req: Request):
        self.queue.append(req)

    def _launch(self, reqs, stream_event_factory):
        by_n = {}
        for r in reqs:
            by_n.setdefault(r.log_n, []).append(r)
        outputs = []
        for log_n, group in sorted(by_n.items()):
            m = self.models[log_n]
            conv = H.hc_enc_conv2d_single_hoisted_batch if m.hoisted else H.hc_enc_conv2d_single_batch
            y = conv(m.ctx, m.evk, [r.ct for r in group], m.width, m.weights, 1, m.kh, m.kw)
            # one activation call over every level of the group (the library
            # runs each level's batch as a concurrent branch)
            for r, a in zip(group, H.hc_enc_poly_act(m.ctx, m.evk, y, (0.0, 0.0, 1.0))):
                r.result = a
                outputs.append(a)
        return stream_event_factory()

    def tick(self, stream_event_factory):
        """Retire finished steps, then admit and launch what fits."""
        now = self.clock()
        still = []
        for st in self.inflight:
            if st.event.query():
                t = self.clock()
                for r in st.requests:
                    r.done = t
                    self.done.append(r)
                self.used_bytes -= st.bytes
            else:
                still.append(st)
        self.inflight = still
        admit, nbytes = [], 0
        while self.queue and len(admit) < self.max_batch:
            r = self.queue[0]
            fb = footprint_bytes(self.models[r.log_n], r.ct.level)
            if self.used_bytes + nbytes + fb > self.budget_bytes and (admit or self.inflight):
                self.budget_waits += 1
                break
            admit.append(self.queue.pop(0))
            nbytes += fb
        if admit:
            for r in admit:
                r.admitted = now
            ev = self._launch(admit, stream_event_factory)
            self.inflight.append(_Step(ev, admit, [r.result for r in admit], nbytes))
            self.used_bytes += nbytes
            self.peak_bytes = max(self.peak_bytes, self.used_bytes)
        return bool(admit)

    def busy(self):
        return bool(self.queue or self.inflight)


class AllOf:
    """Completion of several events (one per stream, when the models' contexts
    run on separate streams): query() is true once every one has completed."""

    def __init__(self, events):
        self.events = list(events)

    def query(self):
        return all(e.query() for e in self.events)


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process with the given rate."""
    gaps = np.random.Generator(np.random.PCG64(seed)).exponential(1.0 / rate, count)
    return np.cumsum(gaps)


def run(server: Server, requests: list, arrivals, stream_event_factory, poll_s: float = 2e-4):
    """Feeds requests at their arrival times (relative to now) and runs the
    loop until all are done.  Returns summary statistics."""
    t0 = server.clock()
    pending = [(float(a), i) for i, a in enumerate(arrivals)]
    heapq.heapify(pending)
    while pending or server.busy():
        now = server.clock() - t0
        while pending and pending[0][0] <= now:
            _, i = heapq.heappop(pending)
            requests[i].arrival = t0 + arrivals[i]
            server.submit(requests[i])
        launched = server.tick(stream_event_factory)
        if not launched:
            wait = (pending[0][0] - now) if pending and not server.busy() else poll_s
            time.sleep(max(0.0, min(wait, poll_s if server.busy() else wait)))
    lat = np.array([r.done - r.arrival for r in requests])
    queued = np.array([r.admitted - r.arrival for r in requests])
    span = max(r.done for r in requests) - t0
    return {
        "requests": len(requests), "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
        "queue_p50_ms": float(np.percentile(queued, 50) * 1e3), "queue_p99_ms": float(np.percentile(queued, 99) * 1e3),
        "images_per_s": len(requests) / span, "offered_per_s": len(requests) / max(float(arrivals[-1]), 1e-9),
        "peak_admitted_bytes": server.peak_bytes, "budget_bytes": server.budget_bytes,
        "budget_waits": server.budget_waits,
    }
