"""The plane pipeline of the one-pass kernel, replayed on the CPU.

A z-block of the one-pass step loads planes k0-1 .. k1 (load index L = 0 .. nplanes-1) into
S shared-memory stages by TMA, each stage with its own mbarrier.  Load L goes to stage L % S and
is the (L // S)-th completion of that stage's barrier, so its wait uses parity (L // S) & 1.
Thread 0 issues the first min(S, nplanes) loads.  After each plane's CTA barrier it refills
the stage just consumed with the load S further on.  If a wait gives up, thread 0 waits once
more, bounded, for every load issued from the first unfinished one on.

This replays that schedule (the same index arithmetic as the kernel) with a model of the
stages and barriers.  It checks, for every block length and stage count:
- each load is issued once, into a stage whose previous contents were consumed before the
  barrier that released the refill;
- each wait names the right parity;
- the drain after an abort covers exactly the loads still in flight.
"""
import pytest


def replay(nplanes, S, fail_at=None):
    """Run the schedule; return (issued, events).  fail_at: load index whose wait gives up."""
    stage_load = [None] * S          # load index currently held by each stage
    completions = [0] * S            # phases completed per stage barrier
    consumed = set()
    events = []
    issued = 0

    def issue(L):
        s = L % S
        prev = stage_load[s]
        assert prev is None or prev in consumed, f"load {L} overwrites unconsumed load {prev}"
        stage_load[s] = L
        events.append(("issue", L))

    def wait(L):
        s = L % S
        parity = (L // S) & 1
        assert stage_load[s] == L, f"wait for load {L} but stage {s} holds {stage_load[s]}"
        # the barrier's phase for this load is its completion count before the load lands
        assert completions[s] & 1 == parity, (L, completions[s], parity)
        if L == fail_at:
            return False
        completions[s] += 1
        consumed.add(L)              # read by every thread before the next CTA barrier
        events.append(("wait", L))
        return True

    while issued < S and issued < nplanes:                          # prologue
        issue(issued)
        issued += 1
    ok, waited = True, 0
    if nplanes > 0:
        ok = wait(0)
        waited = 1
    aborted = not ok
    if not aborted and S < nplanes:                                 # plane k0-1 is in registers
        issue(S)
        issued += 1
    q_loads = range(1, nplanes)                                     # planes k0 .. k1
    for iq in q_loads:
        if aborted:
            break
        if ok:
            ok = wait(iq)
        waited = iq + 1
        if not ok:                                                  # the CTA barrier sees it
            aborted = True
            break
        nxt = iq + S                                                # plane q + S, as a load index
        if nxt <= nplanes - 1:
            issue(nxt)
            issued += 1
    drained = []
    if aborted:
        start = waited - 1 if waited > 0 else 0
        drained = list(range(start, issued))
    return issued, events, drained, consumed


@pytest.mark.parametrize("S", [2, 3, 4, 5, 8])
def test_schedule_issues_each_load_once_and_waits_in_order(S):
    for nplanes in range(1, 40):
        issued, events, drained, consumed = replay(nplanes, S)
        assert issued == nplanes
        assert [L for e, L in events if e == "issue"] == list(range(nplanes))
        assert [L for e, L in events if e == "wait"] == list(range(nplanes))
        assert consumed == set(range(nplanes)) and drained == []


@pytest.mark.parametrize("S", [2, 4])
def test_abort_drains_exactly_the_loads_in_flight(S):
    for nplanes in range(1, 30):
        for fail_at in range(nplanes):
            issued, events, drained, consumed = replay(nplanes, S, fail_at)
            in_flight = [L for L in range(issued) if L not in consumed]
            assert drained == in_flight, (nplanes, fail_at, drained, in_flight)
            assert fail_at in drained
