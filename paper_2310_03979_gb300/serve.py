"""Serving loop: continuous batching of sample requests over cached plans.

Requests name a spectrum (a Workload: lattice, cutoffs, Kaimal U and z,
target) and a number of samples with their seeds.  The server keeps plans
on the device in an LRU cache bounded by an HBM budget, builds missing
plans on a background thread, and admits waiting requests whenever one of
its stream slots is free: all admitted requests go into one batch
(srm3_batch_*), where requests for the same spectrum share a plan and
spectra of one lattice shape share the lanes of the pair sum.  Requests
are light or heavy by the pair-terms of one sample (heavy above
`heavy_terms`); each class has its own queue and stream slots, and a heavy
batch's persistent pair sum is capped at one CTA per SM so that light
batches run beside it instead of queueing behind it.  Batches admitted
while others run overlap with them on the device.  A request's latency runs
from its arrival to the completion of its batch.

Device memory of a plan (the estimate the budget counts): the FP64/FP32
plan tables, about 136 bytes per lattice point, plus the W table when
stored.  Batch buffers are stream-ordered allocations of the batch and are
released when it completes.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time

from . import srm3
from .workloads import Workload


def plan_key(wl: Workload):
    """Everything a plan depends on (the seeds do not matter)."""
    return (wl.n_kappa, wl.n_omega, wl.kappa_u, wl.omega_u, wl.U, wl.z, wl.z0, wl.k_vk,
            wl.lam, wl.n_x, wl.n_t, wl.precision, wl.target, wl.sigma_g, wl.beta, wl.storage)


def plan_bytes_estimate(wl: Workload, table_bytes: float = 0.0) -> float:
    return 136.0 * wl.n_kappa * wl.n_omega + table_bytes


@dataclasses.dataclass
class Request:
    rid: int
    wl: Workload
    seeds: tuple
    arrival: float = 0.0          # seconds from the start of the run
    admitted: float | None = None
    done: float | None = None
    out: object = None            # device tensor [n][n_x][n_t] once done

    @property
    def n(self) -> int:
        return len(self.seeds)

    @property
    def latency(self) -> float | None:
        return None if self.done is None else self.done - self.arrival


class PlanCache:
    """Plans on the device, bounded by an HBM budget: the least recently used
    plan that is not in flight is evicted first.  `builder` creates a plan
    from a Workload (srm3.Plan.create by default)."""

    def __init__(self, budget_bytes: float, builder=None):
        self.budget = float(budget_bytes)
        self.builder = builder or (lambda wl: srm3.Plan.create(wl))
        self.plans = collections.OrderedDict()   # key -> plan, least recent first
        self.size = {}
        self.pins = collections.Counter()
        self.used = 0.0
        self.builds = 0
        self.evictions = 0
        self.build_seconds = 0.0
        self.lock = threading.Lock()

    def lookup(self, wl):
        key = plan_key(wl)
        with self.lock:
            p = self.plans.get(key)
            if p is not None:
                self.plans.move_to_end(key)
            return p

    def build(self, wl):
        """Build and insert the plan of wl (evicting as needed); returns it."""
        key = plan_key(wl)
        with self.lock:
            if key in self.plans:
                self.plans.move_to_end(key)
                return self.plans[key]
        t0 = time.perf_counter()
        p = self.builder(wl)
        dt = time.perf_counter() - t0
        info_bytes = 0.0
        try:
            info_bytes = float(p.info().table_bytes)
        except Exception:  # noqa: BLE001 -- stand-in plans in tests
            info_bytes = 0.0
        need = plan_bytes_estimate(wl, info_bytes)
        with self.lock:
            self.builds += 1
            self.build_seconds += dt
            while self.used + need > self.budget:
                victim = next((k for k in self.plans if self.pins[k] == 0), None)
                if victim is None:
                    break  # everything in flight: admit over budget rather than deadlock
                old = self.plans.pop(victim)
                self.used -= self.size.pop(victim)
                self.evictions += 1
                old.destroy()
            self.plans[key] = p
            self.size[key] = need
            self.used += need
        return p

    def pin(self, wl):
        with self.lock:
            self.pins[plan_key(wl)] += 1

    def unpin(self, wl):
        with self.lock:
            self.pins[plan_key(wl)] -= 1

    def clear(self):
        with self.lock:
            for p in self.plans.values():
                p.destroy()
            self.plans.clear()
            self.size.clear()
            self.used = 0.0


class Server:
    """Continuous batching over `slots` CUDA streams (see the module text)."""

    def __init__(self, budget_bytes: float = 150e9, light_slots: int = 1, heavy_slots: int = 1,
                 max_samples: int = 4096, cache: PlanCache | None = None,
                 heavy_terms: float = 1e9):
        import torch
        self.torch = torch
        self.cache = cache or PlanCache(budget_bytes)
        self.slot_class = ["light"] * light_slots + ["heavy"] * heavy_slots
        self.streams = [torch.cuda.Stream() for _ in self.slot_class]
        self.inflight = [None] * len(self.slot_class)
        self.max_samples = max_samples
        self.heavy_terms = heavy_terms
        self.heavy_ctas = torch.cuda.get_device_properties(0).multi_processor_count
        self.queues = {"light": collections.deque(), "heavy": collections.deque()}
        self.missing = collections.deque()      # plans being built
        self.finished = []
        self.batches = 0
        self.launches = 0                       # kernels: phases + 2 FFT stages per plan, 1 pair sum
        self.busy = 0.0                         # seconds with a batch in flight
        self._busy_since = None
        self._cv = threading.Condition()
        self._stop = False
        self._builder = threading.Thread(target=self._build_loop, daemon=True)
        self._builder.start()

    # -- plan builds off the serving thread --------------------------------
    def _build_loop(self):
        while True:
            with self._cv:
                while not self.missing and not self._stop:
                    self._cv.wait()
                if self._stop:
                    return
                req = self.missing[0]
            self.cache.build(req.wl)
            with self._cv:
                # every waiting request whose plan now exists moves to its queue
                keep = collections.deque()
                for r in self.missing:
                    if self.cache.lookup(r.wl) is not None:
                        self.queues[self._class(r)].append(r)
                    else:
                        keep.append(r)
                self.missing = keep

    def _class(self, req):
        return "heavy" if 2 * req.wl.pairs() > self.heavy_terms else "light"

    def submit(self, req: Request):
        with self._cv:
            if self.cache.lookup(req.wl) is not None:
                self.queues[self._class(req)].append(req)
            else:
                self.missing.append(req)
                self._cv.notify()

    # -- batches -----------------------------------------------------------
    def _launch(self, slot, now):
        torch = self.torch
        q = self.queues[self.slot_class[slot]]
        with self._cv:
            take, total = [], 0
            while q and total + q[0].n <= self.max_samples:
                r = q.popleft()
                take.append(r)
                total += r.n
        if not take:
            return False
        groups = collections.OrderedDict()  # one batch entry per plan
        for r in take:
            groups.setdefault(plan_key(r.wl), []).append(r)
        plans, counts, outs, seeds = [], [], [], []
        s = self.streams[slot]
        with torch.cuda.stream(s):
            for key, rs in groups.items():
                wl = rs[0].wl
                p = self.cache.lookup(wl)
                self.cache.pin(wl)
                n = sum(r.n for r in rs)
                dt = torch.float32 if wl.precision == "fp32" else torch.float64
                o = torch.empty((n, wl.n_x, wl.n_t), dtype=dt, device="cuda")
                k = 0
                for r in rs:
                    r.out = o[k:k + r.n]
                    r.admitted = now
                    seeds.extend(r.seeds)
                    k += r.n
                plans.append(p)
                counts.append(n)
                outs.append(o)
        b = srm3.Batch(plans, counts, outs, stream=s.cuda_stream)
        if self.slot_class[slot] == "heavy":
            b.set_max_ctas(self.heavy_ctas)
        b.run(seeds)
        ev = torch.cuda.Event()
        ev.record(s)
        self.inflight[slot] = (b, ev, take, [rs[0].wl for rs in groups.values()], outs)
        self.batches += 1
        self.launches += 3 * len(plans) + 1
        return True

    def _poll(self, now):
        for i, f in enumerate(self.inflight):
            if f is None or not f[1].query():
                continue
            b, ev, reqs, wls, outs = f
            b.sync()
            b.destroy()
            for wl in wls:
                self.cache.unpin(wl)
            for r in reqs:
                r.done = now
                self.finished.append(r)
            self.inflight[i] = None

    def _account(self, now):
        active = any(f is not None for f in self.inflight)
        if active and self._busy_since is None:
            self._busy_since = now
        elif not active and self._busy_since is not None:
            self.busy += now - self._busy_since
            self._busy_since = None

    def run(self, requests, idle_sleep=1e-4):
        """Serve `requests` (arrival times in seconds from now) in real time;
        returns the wall time of the run."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        total = len(pending)
        t0 = time.perf_counter()
        while len(self.finished) < total:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                self.submit(pending.popleft())
            self._poll(now)
            self._account(now)
            launched = False
            for i in range(len(self.streams)):
                if self.inflight[i] is None and self.queues[self.slot_class[i]]:
                    launched |= self._launch(i, time.perf_counter() - t0)
            self._account(time.perf_counter() - t0)
            if not launched:
                time.sleep(idle_sleep)
        wall = time.perf_counter() - t0
        self._account(wall)
        return wall

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify()
        self._builder.join(timeout=60)
        for f in self.inflight:
            if f is not None:
                f[0].sync()
                f[0].destroy()
        self.inflight = [None] * len(self.inflight)


def percentile(values, q):
    v = sorted(values)
    if not v:
        return None
    k = (len(v) - 1) * q / 100.0
    lo = int(k)
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)
