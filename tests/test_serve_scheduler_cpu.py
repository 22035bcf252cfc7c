"""Host-side policy of the serving loop (no GPU): FIFO admission under a
slot cap and a memory budget, one frame per active viewer per tick,
latency accounting and retirement."""
from paper_2504_20937_b300 import inputs
from paper_2504_20937_b300.serve import ContinuousBatcher


def _req(v, t, frames=3, n=1000):
    return inputs.ViewerRequest(viewer=v, arrival_s=t, W=64, H=48, frames=frames, private_n=n, start_deg=0.0,
                                init_seed=v)


class FakeEngine:
    """Admits a viewer while its bytes fit the budget; ids are reused."""

    def __init__(self, budget):
        self.budget, self.held, self.ids = budget, 0, {}

    def try_add(self, req):
        if self.held + req.private_n > self.budget:
            return None
        vid = min(set(range(len(self.ids) + 1)) - set(self.ids))
        self.ids[vid] = req.private_n
        self.held += req.private_n
        return vid

    def remove(self, vid):
        self.held -= self.ids.pop(vid)


def test_fifo_admission_slots_and_retirement():
    b = ContinuousBatcher(max_viewers=2)
    b.load([_req(0, 0.0), _req(1, 0.0), _req(2, 0.0), _req(3, 5.0)])
    eng = FakeEngine(budget=10**9)
    b.arrive(0.0)
    assert [r.viewer for _, r in b.admit(eng.try_add)] == [0, 1]     # slot cap 2
    assert [r.viewer for r in b.waiting] == [2] and len(b.pending) == 1
    for t in (1.0, 2.0, 3.0):
        first, later, done = b.tick_done(t)
        for vid in done:
            eng.remove(vid)
    assert not b.active                                                # both had 3 frames
    assert first == [] and sorted(later) == [1.0, 1.0]
    assert [r.viewer for _, r in b.admit(eng.try_add)] == [2]
    assert b.busy()


def test_budget_refusal_keeps_arrival_order():
    b = ContinuousBatcher(max_viewers=8)
    b.load([_req(0, 0.0, n=600), _req(1, 0.1, n=600), _req(2, 0.2, n=100)])
    eng = FakeEngine(budget=1000)
    b.arrive(1.0)
    assert [r.viewer for _, r in b.admit(eng.try_add)] == [0]
    # viewer 1 does not fit; viewer 2 would, but must not overtake it
    assert [r.viewer for r in b.waiting] == [1, 2] and b.refused == 1
    _, _, done = b.tick_done(1.5)
    assert done == []


def test_latency_of_first_and_later_frames():
    b = ContinuousBatcher(max_viewers=4)
    b.load([_req(0, 0.25, frames=2)])
    eng = FakeEngine(budget=10**9)
    b.arrive(0.5)
    b.admit(eng.try_add)
    assert b.frames_due() == [(0, b.active[0][0], 0)]
    first, later, _ = b.tick_done(1.0)
    assert first == [0.75] and later == []                   # from arrival to the first frame
    first, later, done = b.tick_done(1.5)
    assert first == [] and later == [0.5] and done == [0]    # from the previous frame
    assert not b.busy()


def test_latency_from_the_display_refresh():
    """With a display rate a later frame's latency runs from the refresh that
    asked for it; the first frame's still from the arrival."""
    b = ContinuousBatcher(max_viewers=4)
    b.load([_req(0, 0.25, frames=3)])
    eng = FakeEngine(budget=10**9)
    b.arrive(0.5)
    b.admit(eng.try_add)
    first, later, _ = b.tick_done(0.625, refresh=0.5)
    assert first == [0.375] and later == []
    first, later, _ = b.tick_done(1.125, refresh=1.0)       # rendered 1/8 s after its refresh
    assert first == [] and later == [0.125]
