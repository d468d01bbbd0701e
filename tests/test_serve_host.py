"""Scheduling logic of the serving loop on the host, against a fake batch
(no GPU): first-come-first-served admission under the HBM budget, exact step
budgets, residual stops, retirement freeing memory for later admissions."""
import goc_inputs as gi
from paper_2607_15362_b300.serve import Request, Server


class FakeLattice:
    def __init__(self, b, slot):
        self.b, self.slot = b, slot

    def moments(self):
        return (self.b.steps[self.slot],)

    def sync(self):
        pass


class FakeBatch:
    """Stand-in for Batch: each lattice costs `nodes` bytes; the residual of a
    checked slot decays as 1/steps."""

    def __init__(self, budget):
        self.budget, self.used = budget, 0
        self.size, self.steps, self.checked = {}, {}, set()
        self.calls, self.max_resident, self.next_slot = [], 0, 0

    def try_add(self, spec, storage=None):
        need = spec["nx"] * spec["ny"]
        if self.used + need > self.budget:
            return None
        slot = self.next_slot
        self.next_slot += 1
        self.size[slot], self.steps[slot] = need, 0
        self.used += need
        self.max_resident = max(self.max_resident, len(self.size))
        return slot

    def check(self, slot, on=True):
        self.checked.add(slot)

    def step(self, k):
        self.calls.append(k)
        for s in self.steps:
            self.steps[s] += k

    def residual(self, slot):
        return 1.0 / self.steps[slot], 0.0

    def lattice(self, slot):
        return FakeLattice(self, slot)

    def remove(self, slot):
        self.used -= self.size.pop(slot)
        self.steps.pop(slot)


def _req(rid, t, n, budget, tol=None):
    p = gi.Problem("poiseuille", n, n, {"kind": "uniform"}, {"kind": "tanh2", "beta": 1.0}, {"Re": 10.0, "tau": 0.8})
    return Request(rid, t, p, budget, tol)


def test_budgets_are_exact_and_admission_respects_the_budget():
    fb = FakeBatch(budget=3 * 64 * 64)
    reqs = [_req(0, 0.0, 64, 700), _req(1, 0.0, 64, 1300), _req(2, 0.0, 64, 250), _req(3, 0.0, 64, 900),
            _req(4, 0.0, 32, 50)]
    srv = Server(0, chunk=400, batch=fb, spec_fn=lambda p: {"nx": p.nx, "ny": p.ny}, keep_fields=True)
    results, summary = srv.run(reqs)
    by = {r.rid: r for r in results}
    assert all(r.status == "done" for r in results)
    for rq in reqs:
        assert by[rq.rid].steps == rq.budget
        assert by[rq.rid].fields[0] == rq.budget        # the lattice saw exactly its budget
    assert fb.max_resident <= 3 + 1                      # three 64^2 fit; the 32^2 one squeezes in
    assert fb.used == 0 and summary["done"] == 5
    assert max(fb.calls) <= 400


def test_residual_requests_stop_below_tolerance():
    fb = FakeBatch(budget=10 ** 9)
    reqs = [_req(0, 0.0, 16, 100000, tol=1.0 / 950), _req(1, 0.0, 16, 3000)]
    srv = Server(0, chunk=300, batch=fb, spec_fn=lambda p: {"nx": p.nx, "ny": p.ny})
    results, _ = srv.run(reqs)
    by = {r.rid: r for r in results}
    assert by[0].status == "done" and 950 < by[0].steps <= 1200 and by[0].residual < 1.0 / 950
    assert by[1].steps == 3000


def test_first_come_first_served():
    fb = FakeBatch(budget=64 * 64)
    reqs = [_req(0, 0.0, 64, 100), _req(1, 0.0, 64, 100), _req(2, 0.0, 64, 100)]
    srv = Server(0, chunk=1000, batch=fb, spec_fn=lambda p: {"nx": p.nx, "ny": p.ny})
    results, _ = srv.run(reqs)
    order = [r.rid for r in sorted(results, key=lambda r: r.admitted_s)]
    assert order == [0, 1, 2]


def test_a_diverged_request_is_evicted_and_the_others_finish():
    """A lattice whose status word reports divergence when its result is
    collected is recorded as "diverged" and removed; the requests beside it
    finish with their exact budgets and the memory is released."""
    from paper_2607_15362_b300._abi import GOC_EDIVERGED, GocError

    class DivergingLattice(FakeLattice):
        def sync(self):
            if self.slot == 1:
                raise GocError(GOC_EDIVERGED, "lattice diverged")

    class DivergingBatch(FakeBatch):
        def lattice(self, slot):
            return DivergingLattice(self, slot)

    fb = DivergingBatch(budget=10 ** 9)
    reqs = [_req(0, 0.0, 16, 500), _req(1, 0.0, 16, 500), _req(2, 0.0, 16, 800)]
    srv = Server(0, chunk=300, batch=fb, spec_fn=lambda p: {"nx": p.nx, "ny": p.ny})
    results, summary = srv.run(reqs)
    by = {r.rid: r for r in results}
    assert by[1].status == "diverged" and by[0].status == by[2].status == "done"
    assert by[2].steps == 800 and summary["diverged"] == 1 and summary["done"] == 2
    assert fb.used == 0


def test_a_cancelled_request_is_withdrawn_waiting_or_running():
    """cancel(rid) drops a waiting request and evicts a running one at the
    next chunk boundary (its memory released); both are reported as
    cancelled and the other requests finish with their exact budgets."""
    fb = FakeBatch(budget=2 * 16 * 16)
    reqs = [_req(0, 0.0, 16, 3000), _req(1, 0.0, 16, 900), _req(2, 0.0, 16, 600), _req(3, 0.0, 16, 400)]
    srv = Server(0, chunk=300, batch=fb, spec_fn=lambda p: {"nx": p.nx, "ny": p.ny})

    orig_step = fb.step

    def step(k):   # after the first chunk: cancel request 0 (running) and 3 (waiting)
        orig_step(k)
        if len(fb.calls) == 1:
            srv.cancel(0)
            srv.cancel(3)
    fb.step = step
    results, summary = srv.run(reqs)
    by = {r.rid: r for r in results}
    assert by[0].status == "cancelled" and by[0].steps == 300
    assert by[3].status == "cancelled" and by[3].steps == 0
    assert by[1].status == by[2].status == "done" and by[1].steps == 900 and by[2].steps == 600
    assert summary["cancelled"] == 2 and fb.used == 0
