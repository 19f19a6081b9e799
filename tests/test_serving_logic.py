"""Host-side logic of the serving loop (no GPU): admission by device
footprint, FIFO order, overlap of steps, retirement on event completion."""
import numpy as np

from paper_2102_00319_gb300 import serving


class FakeCt:
    def __init__(self, level):
        self.level = level


class FakeEvent:
    def __init__(self, polls):
        self.polls = polls

    def query(self):
        self.polls -= 1
        return self.polls < 0


def test_admission_respects_budget_and_completes(monkeypatch):
    launched = []

    def fake_conv(ctx, evk, xs, W, ws, cout, kh, kw):
        launched.append(len(xs))
        return [FakeCt(x.level - 1) for x in xs]

    monkeypatch.setattr(serving.H, "hc_enc_conv2d_single_batch", fake_conv)
    monkeypatch.setattr(serving.H, "hc_enc_poly_act", lambda ctx, evk, xs, c: [FakeCt(x.level - 1) for x in xs])
    model = serving.Model(ctx=None, evk=None, weights=[None] * 9, n=1 << 12, n_special=1)
    one = serving.footprint_bytes(model, 2)
    srv = serving.Server(models={12: model}, budget_bytes=3 * one, max_batch=8)
    reqs = [serving.Request(i, 12, FakeCt(2), 0.0) for i in range(10)]
    for r in reqs:
        srv.submit(r)
    ticks = 0
    while srv.busy():
        srv.tick(lambda: FakeEvent(2))
        assert srv.used_bytes <= 3 * one
        ticks += 1
        assert ticks < 1000
    assert sum(launched) == 10 and max(launched) <= 3
    assert [r.rid for r in srv.done] == list(range(10))
    assert all(r.done >= r.admitted >= r.arrival for r in reqs)
    assert srv.peak_bytes <= 3 * one


def test_hoisted_model_calls_the_hoisted_conv_and_is_counted_smaller(monkeypatch):
    calls = []

    def fake(name):
        def conv(ctx, evk, xs, W, ws, cout, kh, kw):
            calls.append(name)
            return [FakeCt(x.level - 1) for x in xs]
        return conv

    monkeypatch.setattr(serving.H, "hc_enc_conv2d_single_batch", fake("plain"))
    monkeypatch.setattr(serving.H, "hc_enc_conv2d_single_hoisted_batch", fake("hoisted"))
    monkeypatch.setattr(serving.H, "hc_enc_poly_act", lambda ctx, evk, xs, c: [FakeCt(x.level - 1) for x in xs])
    plain = serving.Model(ctx=None, evk=None, weights=[None] * 9, n=1 << 13, n_special=1)
    hoisted = serving.Model(ctx=None, evk=None, weights=[None] * 9, n=1 << 13, n_special=1, hoisted=True)
    # one raised copy of c1 instead of eight whole key-switch workspaces
    for level in (3, 7, 12):
        assert serving.footprint_bytes(hoisted, level) < serving.footprint_bytes(plain, level)
    for model, name in ((plain, "plain"), (hoisted, "hoisted")):
        calls.clear()
        srv = serving.Server(models={13: model}, budget_bytes=1 << 40, max_batch=4)
        for i in range(3):
            srv.submit(serving.Request(i, 13, FakeCt(5), 0.0))
        while srv.busy():
            srv.tick(lambda: FakeEvent(0))
        assert calls == [name]


def test_oversized_request_runs_alone():
    model = serving.Model(ctx=None, evk=None, weights=[None] * 9, n=1 << 12, n_special=1)
    assert serving.footprint_bytes(model, 2) > 0
    # a budget smaller than one request still admits it when nothing else runs
    srv = serving.Server(models={12: model}, budget_bytes=1, max_batch=4)
    srv.submit(serving.Request(0, 12, FakeCt(2), 0.0))
    srv.inflight = []
    calls = []
    srv._launch = lambda reqs, f: calls.append(len(reqs)) or FakeEvent(0)
    srv.tick(lambda: FakeEvent(0))
    assert calls == [1]


def test_poisson_arrivals_rate():
    a = serving.poisson_arrivals(100.0, 20000, 1)
    assert np.all(np.diff(a) > 0)
    assert abs(len(a) / a[-1] - 100.0) < 3.0


def test_all_of_completes_when_every_event_has():
    evs = [FakeEvent(0), FakeEvent(2)]
    done = serving.AllOf(evs)
    assert not done.query()  # the second event still has polls to go
    assert not done.query()
    assert done.query()
