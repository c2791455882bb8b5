"""Host logic of the densification loop (no GPU): the event window and the
warm-up of the gradient-threshold masking."""
from types import SimpleNamespace

import pytest

loop_mod = pytest.importorskip("paper_2603_08661_gb300.loop")
DensifyLoop = loop_mod.DensifyLoop


def _due(every, start, until):
    return SimpleNamespace(every=every, densify_from=start, densify_until=until)


def test_paper_window_gives_thirty_densification_steps():
    """Sec. 2.3: every 500 iterations from 500 to 15,000 is exactly 30 steps."""
    cfg = _due(500, 500, 15000)
    events = [it for it in range(1, 30001) if DensifyLoop.event_due(cfg, it)]
    assert len(events) == 30 and events[0] == 500 and events[-1] == 15000
    assert all(b - a == 500 for a, b in zip(events, events[1:]))


def test_open_window_and_offsets():
    assert [it for it in range(1, 101) if DensifyLoop.event_due(_due(20, 0, None), it)] == [20, 40, 60, 80, 100]
    assert [it for it in range(1, 101) if DensifyLoop.event_due(_due(20, 30, 70), it)] == [40, 60]


def test_warmup_of_the_gradient_threshold():
    """The first three events select by score alone (Sec. 2.3, warm-up)."""
    state = SimpleNamespace(pos_grad=(object(), object()), warmup_events=3, events=0)
    seen = []
    for _ in range(5):
        seen.append(DensifyLoop.gated(state))
        state.events += 1
    assert seen == [False, False, False, True, True]
    assert not DensifyLoop.gated(SimpleNamespace(pos_grad=None, warmup_events=3, events=9))
