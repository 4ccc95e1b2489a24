"""Serving loop: the plan cache's HBM budget and LRU eviction (CPU, stand-in
plans), and on the GPU that every request served in a mix of spectra,
lattice shapes and arrival times gives the field it gives alone."""
import pytest

import collections

from paper_2310_03979_gb300 import serve
from paper_2310_03979_gb300 import workloads as W


class FakeInfo:
    def __init__(self, nbytes):
        self.table_bytes = 0.0
        self.device_bytes = nbytes
        self.storage = 2
        self.interactions = 0


class FakePlan:
    """Stand-in for a plan: reports device_bytes = 1000 per lattice row."""

    def __init__(self, wl):
        self.wl = wl
        self.destroyed = False
        self.nbytes = 1000.0 * wl.n_kappa

    def info(self):
        return FakeInfo(self.nbytes)

    def destroy(self):
        self.destroyed = True


def _wl(nk, U):
    return W.small_case(nk=nk, nw=32, nx=64, nt=64, U=U)


def test_plan_cache_lru_budget_and_pins():
    per = 1000.0 * 32
    c = serve.PlanCache(budget_bytes=2.5 * per, builder=FakePlan)
    a, b, d = _wl(32, 20.0), _wl(32, 30.0), _wl(32, 40.0)
    pa = c.build(a)
    pb = c.build(b)
    assert c.lookup(a) is pa  # a is now the most recently used
    c.pin(b)
    pd = c.build(d)          # over budget: the LRU plan that is not pinned goes
    key = serve.plan_key    # membership checks that do not touch the LRU order
    assert key(d) in c.plans and c.evictions == 1
    assert key(a) not in c.plans and pa.destroyed
    assert key(b) in c.plans and not pb.destroyed
    c.unpin(b)
    c.build(a)               # now b (least recent, unpinned) is evicted
    assert key(b) not in c.plans and pb.destroyed and not pd.destroyed
    assert c.used <= c.budget and c.builds == 4


def test_plan_cache_charges_what_plans_report_and_refreshes():
    c = serve.PlanCache(budget_bytes=1e9, builder=FakePlan)
    p = c.build(_wl(20, 20.0))
    assert c.used == 20000.0
    p.nbytes = 50000.0  # its workspace grew in a batch
    c.refresh(_wl(20, 20.0))
    assert c.used == 50000.0
    c.build(_wl(10, 30.0))
    assert c.used == 60000.0


def test_plan_cache_builder_failure_leaves_it_unchanged():
    def builder(wl):
        if wl.U == 99.0:
            raise RuntimeError("injected: device allocation refused")
        return FakePlan(wl)

    c = serve.PlanCache(budget_bytes=1e9, builder=builder)
    c.build(_wl(8, 20.0))
    used, n = c.used, len(c.plans)
    try:
        c.build(_wl(8, 99.0))
        raise AssertionError("the injected failure did not surface")
    except RuntimeError as e:
        assert "injected" in str(e)
    assert c.used == used and len(c.plans) == n and c.builds == 1
    assert c.lookup(_wl(8, 99.0)) is None
    c.build(_wl(8, 30.0))  # and it goes on building
    assert len(c.plans) == 2


def test_admission_holds_requests_at_the_budget():
    """Requests are admitted from the head of the queue while the plans, the
    batches in flight and the new batch fit the budget; the rest wait, in
    order, and go once memory comes back."""
    wl = W.small_case(nk=16, nw=32, nx=256, nt=1024)  # 1 MB of field per sample
    reqs = collections.deque(serve.Request(i, wl, tuple(range(2))) for i in range(10))
    one = serve.batch_bytes_estimate([(wl, 2, True)])
    budget, plans = 10 * one, 2 * one
    inflight = [5 * one]

    def fits(cand):
        need = serve.batch_bytes_estimate([(wl, sum(r.n for r in cand), True)])
        return plans + sum(inflight) + need <= budget

    first = serve.admit(reqs, max_samples=1000, fits=fits)
    assert 1 <= len(first) < 10
    assert fits(first) and not fits(first + [reqs[0]])  # held exactly at the budget
    assert [r.rid for r in reqs] == list(range(len(first), 10))  # the rest wait, in order
    inflight[0] = 0.0  # the batch in flight completes
    second = serve.admit(reqs, max_samples=1000, fits=fits)
    assert len(second) > len(first) and fits(second)
    assert [r.rid for r in first + second] == list(range(len(first) + len(second)))
    # the sample cap holds too
    third = serve.admit(collections.deque(serve.Request(i, wl, (1, 2, 3)) for i in range(5)),
                        max_samples=7, fits=lambda c: True)
    assert len(third) == 2


def test_batch_bytes_estimate_adds_up():
    wl = W.small_case(nk=24, nw=37, nx=64, nt=128)
    grouped = serve.batch_bytes_estimate([(wl, 5, True), (wl, 3, True)])
    alone = serve.batch_bytes_estimate([(wl, 5, False), (wl, 3, False)])
    fields = 8 * (64 * 128 * 4 + 8)
    assert alone >= fields
    # a shape group of 8 samples: y + y0 for 64 sheet-samples, C, and the
    # transform's intermediate (n_x n_omega) for 5
    group = 8.0 * ((24 * (37 + 128) + 1) * 64 + 2 * 8 * 24 * 37 + 5 * 64 * 37) + 16 * 8
    assert grouped - alone >= group


@pytest.mark.gpu
def test_plan_and_batch_device_bytes():
    """srm3_info.device_bytes counts the plan's memory and its workspace as it
    grows; a batch's own allocation stays within batch_bytes_estimate."""
    torch = pytest.importorskip("torch")
    from paper_2310_03979_gb300 import srm3
    wl = W.small_case(nk=24, nw=37, nx=64, nt=128)
    other = W.small_case(nk=24, nw=37, nx=64, nt=128, U=41.0, target=0.3)
    with srm3.Plan.create(wl, storage="recompute") as p, \
            srm3.Plan.create(other, storage="recompute") as q:
        b0 = p.info().device_bytes
        assert b0 > 24 * 37 * 8 * 4  # at least its FP64 tables
        p.sample(list(range(1, 101)))
        torch.cuda.synchronize()
        assert p.info().device_bytes > b0  # the workspace grew
        outs = [torch.empty((5, 64, 128), device="cuda"), torch.empty((3, 64, 128), device="cuda")]
        with srm3.Batch([p, q], [5, 3], outs) as b:
            est = serve.batch_bytes_estimate([(wl, 5, True), (other, 3, True)])
            fields = 8 * 64 * 128 * 4
            assert 0 < b.device_bytes <= est - fields
            assert b.device_bytes >= 0.9 * (est - fields - 2 * 512 - 16 * 24 * 2 * 2)


@pytest.mark.gpu
def test_server_serves_through_an_injected_failure():
    """A plan build that fails (injected on the host: the builder raises as
    srm3_plan_create does when the device refuses an allocation) fails that
    spectrum's requests only; every other request is served and equals the
    same request sampled alone."""
    torch = pytest.importorskip("torch")
    from paper_2310_03979_gb300 import srm3
    bad = W.small_case(nk=24, nw=37, nx=64, nt=128, U=33.0, target=0.4)

    def builder(wl):
        if wl.U == 33.0:
            raise srm3.SRM3Error(-5, "injected: out of device memory")
        return srm3.Plan.create(wl)

    good = [W.small_case(nk=24, nw=37, nx=64, nt=128, U=30.0),
            W.small_case(nk=40, nw=20, nx=64, nt=64, U=25.0, target=0.6)]
    reqs = [serve.Request(i, (good + [bad])[i % 3], (7 * i + 1, 7 * i + 2), arrival=0.001 * i)
            for i in range(18)]
    srv = serve.Server(budget_bytes=1e9, max_samples=8, heavy_terms=2e5,
                       cache=serve.PlanCache(1e9, builder=builder))
    try:
        srv.run(reqs)
        assert len(srv.finished) == 18
        failed = [r for r in reqs if r.error is not None]
        assert sorted(r.rid for r in failed) == [i for i in range(18) if i % 3 == 2]
        assert all("injected" in r.error and r.out is None for r in failed)
        torch.cuda.synchronize()
        for r in reqs:
            if r.error is None:
                with srm3.Plan.create(r.wl) as p:
                    alone = p.sample(list(r.seeds))
                    torch.cuda.synchronize()
                assert torch.equal(r.out, alone), r.rid
    finally:
        srv.close()
        srv.cache.clear()


@pytest.mark.gpu
def test_server_results_equal_requests_alone():
    torch = pytest.importorskip("torch")
    from paper_2310_03979_gb300 import srm3
    spectra = [W.small_case(nk=24, nw=37, nx=64, nt=128, U=U, target=t)
               for U, t in ((30.0, 0.5), (42.0, 0.3))]
    spectra.append(W.small_case(nk=40, nw=20, nx=64, nt=64, U=25.0, target=0.6))
    reqs = []
    for i in range(40):
        wl = spectra[i % 3]
        n = 1 + (i * 7) % 4
        reqs.append(serve.Request(i, wl, tuple(100 * i + j for j in range(n)),
                                  arrival=0.002 * i))
    srv = serve.Server(budget_bytes=1e9, light_slots=1, heavy_slots=1, max_samples=9,
                       heavy_terms=2e5)
    try:
        srv.run(reqs)
        assert len(srv.finished) == 40 and srv.batches >= 2
        torch.cuda.synchronize()
        for r in reqs:
            with srm3.Plan.create(r.wl) as p:
                alone = p.sample(list(r.seeds))
                torch.cuda.synchronize()
            assert torch.equal(r.out, alone), r.rid
            assert r.latency >= 0.0
    finally:
        srv.close()
        srv.cache.clear()
