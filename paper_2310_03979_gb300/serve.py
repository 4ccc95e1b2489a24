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

Memory budget.  A plan is charged what the library reports it holds
(srm3_info.device_bytes: lattice and sampling tables, recursion state, W
table, sampling workspace), measured after it is built and again after each
batch it takes part in (its workspace can grow).  A batch is charged, at
admission, an upper bound of what it will allocate (batch_bytes_estimate:
the shape-group buffers the library allocates -- y, C, H, factor pointers,
seeds, work units -- and the output fields); it is admitted only when the
cached plans, the batches in flight and it fit the budget together, else its
requests wait for memory to come back (a batch that would exceed the budget
with nothing in flight is admitted alone rather than never).  Unpinned plans
are evicted, least recently used first, to make room.  A plan build or a
batch that fails (an allocation refused by the device, for instance) fails
its own requests (Request.error) and the server goes on serving the others.
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


def plan_bytes(p) -> float:
    """Device memory plan p holds now (srm3_info.device_bytes)."""
    return float(p.info().device_bytes)


def _sspad(n: int) -> int:
    """Sheet-samples of n samples, rounded up to whole 64-wide groups."""
    return ((2 * n + 63) // 64) * 64


def _shape_key(wl: Workload):
    return (wl.n_kappa, wl.n_omega, wl.n_x, wl.n_t, wl.kappa_u, wl.omega_u, wl.sigma_g,
            wl.beta)


def batch_bytes_estimate(entries) -> float:
    """Upper bound of the device memory one batch takes: ``entries`` are
    (workload, samples, grouped) per plan of the batch, grouped when the
    plan joins a shape group (FP32, W recomputed, the plain pair set).  Per
    shape group with T samples, at most m from one plan: y + y0 = (n_kappa
    (n_omega + 128) + 1) sspad(T) 8 bytes, C = 2 T n_kappa n_omega 8, the
    transform's intermediate m n_x n_omega 8, 16 T of factor pointers (the
    formula of
    srm3_batch_device_bytes); per sample 8 bytes of seed and its output field;
    512 bytes per plan and 16 per work unit of descriptors and unit list."""
    groups = {}
    total = 0.0
    for wl, n, grouped in entries:
        es = 4 if wl.precision == "fp32" else 8
        total += n * (8 + wl.n_x * wl.n_t * es) + 512
        sw = 32  # outputs per work unit along omega
        units = wl.n_kappa * ((wl.n_omega + sw - 1) // sw) * (_sspad(n) // 64)
        total += 16 * units
        if grouped:
            g = groups.setdefault(_shape_key(wl), [wl, 0, 0])
            g[1] += n
            g[2] = max(g[2], n)
    for wl, T, m in groups.values():
        nk, nw = wl.n_kappa, wl.n_omega
        total += 8.0 * ((nk * (nw + 128) + 1) * _sspad(T) + 2 * T * nk * nw + m * wl.n_x * nw)
        total += 16.0 * T
        total += 16 * nk * ((nw + 31) // 32) * (_sspad(T) // 64)
    return total


def admit(queue, max_samples: int, fits) -> list:
    """Requests taken from the head of ``queue`` for one batch: as many as
    keep the batch within ``max_samples`` samples and ``fits(candidates)``;
    the rest stay queued, in order."""
    take, total = [], 0
    while queue and total + queue[0].n <= max_samples:
        if not fits(take + [queue[0]]):
            break
        r = queue.popleft()
        take.append(r)
        total += r.n
    return take


@dataclasses.dataclass
class Request:
    rid: int
    wl: Workload
    seeds: tuple
    arrival: float = 0.0          # seconds from the start of the run
    admitted: float | None = None
    done: float | None = None
    out: object = None            # device tensor [n][n_x][n_t] once done
    error: str | None = None      # why the request failed (it then has no out)

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

    def _evict_for(self, need, reserved=0.0, keep=()):
        """Evict unpinned plans (none whose key is in `keep`), least recently
        used first, until need more bytes fit beside the plans and `reserved`
        (lock held).  Returns whether they fit."""
        while self.used + reserved + need > self.budget:
            victim = next((k for k in self.plans if self.pins[k] == 0 and k not in keep), None)
            if victim is None:
                return False
            old = self.plans.pop(victim)
            self.used -= self.size.pop(victim)
            self.evictions += 1
            old.destroy()
        return True

    def build(self, wl, reserved=0.0):
        """Build and insert the plan of wl, charged the device memory it
        reports, evicting as needed to fit beside `reserved` bytes (batches
        in flight); returns it.  A builder that raises leaves the cache as it
        was and the exception goes to the caller."""
        key = plan_key(wl)
        with self.lock:
            if key in self.plans:
                self.plans.move_to_end(key)
                return self.plans[key]
        t0 = time.perf_counter()
        p = self.builder(wl)
        dt = time.perf_counter() - t0
        need = plan_bytes(p)
        with self.lock:
            self.builds += 1
            self.build_seconds += dt
            # everything in flight: keep the plan over budget rather than deadlock
            self._evict_for(need, reserved)
            self.plans[key] = p
            self.size[key] = need
            self.used += need
        return p

    def refresh(self, wl):
        """Charge the plan of wl what it holds now (its workspace may have
        grown in a batch)."""
        key = plan_key(wl)
        with self.lock:
            p = self.plans.get(key)
            if p is None:
                return
            need = plan_bytes(p)
            self.used += need - self.size[key]
            self.size[key] = need

    def make_room(self, need, reserved, keep=()):
        """Evict unpinned plans outside `keep` until `need` bytes fit beside
        the plans and `reserved`; returns whether they fit."""
        with self.lock:
            return self._evict_for(need, reserved, set(keep))

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
        self.failed = []
        self.inflight_bytes = [0.0] * len(self.slot_class)  # charge of each slot's batch
        self.over_budget = 0                    # batches admitted alone over the budget
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
            try:
                self.cache.build(req.wl, reserved=sum(self.inflight_bytes))
            except Exception as e:  # noqa: BLE001 -- the spectrum's requests fail, serving goes on
                with self._cv:
                    key = plan_key(req.wl)
                    keep = collections.deque()
                    for r in self.missing:
                        if plan_key(r.wl) == key:
                            self._fail(r, f"plan build failed: {e}")
                        else:
                            keep.append(r)
                    self.missing = keep
                continue
            with self._cv:
                # every waiting request whose plan now exists moves to its queue
                keep = collections.deque()
                for r in self.missing:
                    if self.cache.lookup(r.wl) is not None:
                        self.queues[self._class(r)].append(r)
                    else:
                        keep.append(r)
                self.missing = keep

    def _fail(self, req, why):
        req.error = why
        req.done = req.done if req.done is not None else 0.0
        self.failed.append(req)
        self.finished.append(req)

    def _entries(self, reqs):
        """batch_bytes_estimate entries of the plans a batch of reqs uses."""
        groups = collections.OrderedDict()
        for r in reqs:
            groups.setdefault(plan_key(r.wl), []).append(r)
        out = []
        for rs in groups.values():
            wl = rs[0].wl
            p = self.cache.lookup(wl)
            info = p.info() if p is not None else None
            grouped = (info is not None and wl.precision == "fp32" and info.storage == 2
                       and info.interactions == 0 and wl.envelope == "gauss")
            out.append((wl, sum(r.n for r in rs), grouped))
        return out

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
        reserved = sum(self.inflight_bytes)
        alone = not any(f is not None for f in self.inflight)

        # plans that queued requests still need are not evicted for room
        wanted = {plan_key(r.wl) for qq in self.queues.values() for r in qq}

        def fits(cand):
            need = batch_bytes_estimate(self._entries(cand))
            if self.cache.make_room(need, reserved, keep=wanted | {plan_key(r.wl) for r in cand}):
                return True
            return alone and len(cand) == 1  # never hold the only possible batch forever

        with self._cv:
            take = admit(q, self.max_samples, fits)
            # a plan evicted while its request waited (building another plan
            # made room) is built again before the request runs
            gone = [r for r in take if self.cache.lookup(r.wl) is None]
            if gone:
                take = [r for r in take if self.cache.lookup(r.wl) is not None]
                self.missing.extend(gone)
                self._cv.notify()
        if not take:
            return False
        charge = batch_bytes_estimate(self._entries(take))
        if self.cache.used + reserved + charge > self.cache.budget:
            self.over_budget += 1
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
        try:
            b = srm3.Batch(plans, counts, outs, stream=s.cuda_stream)
            if self.slot_class[slot] == "heavy":
                b.set_max_ctas(self.heavy_ctas)
            b.run(seeds)
        except Exception as e:  # noqa: BLE001 -- these requests fail, serving goes on
            for rs in groups.values():
                self.cache.unpin(rs[0].wl)
            del outs
            for r in take:
                r.out = None
                r.done = now
                self._fail(r, f"batch failed: {e}")
            return True
        ev = torch.cuda.Event()
        ev.record(s)
        self.inflight_bytes[slot] = charge
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
                self.cache.refresh(wl)
            self.inflight_bytes[i] = 0.0
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
