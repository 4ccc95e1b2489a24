"""Serving loop: the plan cache's HBM budget and LRU eviction (CPU, stand-in
plans), and on the GPU that every request served in a mix of spectra,
lattice shapes and arrival times gives the field it gives alone."""
import pytest

from paper_2310_03979_gb300 import serve
from paper_2310_03979_gb300 import workloads as W


class FakeInfo:
    table_bytes = 0.0


class FakePlan:
    def __init__(self, wl):
        self.wl = wl
        self.destroyed = False

    def info(self):
        return FakeInfo()

    def destroy(self):
        self.destroyed = True


def _wl(nk, U):
    return W.small_case(nk=nk, nw=32, nx=64, nt=64, U=U)


def test_plan_cache_lru_budget_and_pins():
    per = serve.plan_bytes_estimate(_wl(32, 20.0))
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
