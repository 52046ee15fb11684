"""The controller's colouring pass, modelled on the host.

In a quiet sweep (no accepted exchange applies) sigma does not change, so the
accepted edges (all stale) are only re-evaluated: each dies or comes back as
an applicable edge at its position.  A run of quiet sweeps is then a run of
rounds, each accepting the greedy set of the edges left, and the controller
replaces up to eight such sweeps by one colouring pass: first-fit edge
colouring of the stale edges in position order by reservation rounds with
8-bit colour masks, the first round E in which an applicable edge would be
accepted, and the first birth round R of a re-evaluated edge that lives on;
the F = min(E, R, 8) rounds before both are applied at once.

This test replays the pass step by step (reservation rounds, masks, quick
closing of edges whose agents' masks are full) on random hub-heavy edge
lists and checks it against sweeps simulated one by one: the same number of
quiet sweeps, the same accepted count in each, and the same edges left."""
import random

import pytest

CAP = 8


def greedy(live):
    """Accepted positions of one sweep: the greedy set in position order."""
    claimed, acc = set(), []
    for p in sorted(live):
        u, v, _ = live[p]
        if u not in claimed and v not in claimed:
            acc.append(p)
            claimed.update((u, v))
    return acc


def sweeps_one_by_one(live, refresh, limit):
    """Quiet sweeps until an accepted edge applies (or none is left); returns
    the accepted counts of the quiet sweeps and the edges left."""
    live = dict(live)
    counts = []
    while live and len(counts) < limit:
        acc = greedy(live)
        if any(live[p][2] for p in acc):
            break  # an event: not quiet
        counts.append(len(acc))
        for p in acc:
            if refresh[p] is None:
                del live[p]
            else:
                live[p] = (refresh[p][0], refresh[p][1], True)
    return counts, live


def colour_pass(live, refresh, max_sweeps=0, span=1 << 14, rnd0=0):
    """One pass as the controller runs it; returns (F, per-round counts, live)."""
    mask = {}
    res = {}
    state = {p: 0 for p in live}  # 0 pending, c + 1 coloured, 15 closed
    e_round, r_round = CAP, CAP
    rnd = rnd0
    rounds = 0
    while True:
        rounds += 1
        assert rounds <= len(live) + 2
        if rnd % span == 0 and rnd != 0:
            res.clear()
        base = (span - 1 - rnd % span) << 18
        pend = False
        for p in sorted(live):
            if state[p]:
                continue
            u, v, appl = live[p]
            mu, mv = mask.get(u, 0), mask.get(v, 0)
            if ((mu | mv) == 0xFF) if appl else (mu == 0xFF or mv == 0xFF):
                state[p] = 15
                continue
            pend = True
            key = base | p
            for a in (u, v):
                res[a] = min(res.get(a, 1 << 40), key)
        if not pend:
            break
        for p in sorted(live):
            if state[p]:
                continue
            u, v, appl = live[p]
            key = base | p
            if res[u] != key or res[v] != key:
                continue
            free = ~(mask.get(u, 0) | mask.get(v, 0)) & 0xFF
            if appl:
                if free:
                    e_round = min(e_round, (free & -free).bit_length() - 1)
                state[p] = 15
            elif free:
                c = (free & -free).bit_length() - 1
                mask[u] = mask.get(u, 0) | (1 << c)
                mask[v] = mask.get(v, 0) | (1 << c)
                state[p] = c + 1
            else:
                state[p] = 15
        rnd += 1
    hist = [0] * CAP
    for p in live:
        if 1 <= state[p] <= CAP:
            hist[state[p] - 1] += 1
            if refresh[p] is not None:
                r_round = min(r_round, state[p])
    f = min(e_round, r_round)
    if max_sweeps:
        f = min(f, max_sweeps)
    while f > 0 and hist[f - 1] == 0:  # no edge left: the run ends
        f -= 1
    counts = hist[:f]
    out = dict(live)
    for p in live:
        if 1 <= state[p] <= f:
            if refresh[p] is None:
                del out[p]
            else:
                out[p] = (refresh[p][0], refresh[p][1], True)
    return f, counts, out


def random_case(rng):
    agents = rng.choice([6, 20, 60, 300])
    hubs = [rng.randrange(agents) for _ in range(rng.choice([1, 2, 4, 8]))]
    L = rng.choice([5, 40, 200, 600])
    live, refresh = {}, {}
    for p in range(L):
        if rng.random() < 0.15:
            continue  # a dead position
        if rng.random() < 0.8:
            u, v = rng.choice(hubs), rng.randrange(agents)
        else:
            u, v = rng.randrange(agents), rng.randrange(agents)
        if u == v:
            v = (v + 1) % agents
        live[p] = (u, v, rng.random() < rng.choice([0.0, 0.01, 0.1]))
        refresh[p] = None
        if rng.random() < rng.choice([0.0, 0.05, 0.3]):
            a, b = rng.randrange(agents), rng.randrange(agents)
            refresh[p] = (a, b if b != a else (b + 1) % agents)
    return live, refresh


@pytest.mark.parametrize("seed", range(120))
def test_colour_pass_equals_quiet_sweeps(seed):
    rng = random.Random(seed)
    live, refresh = random_case(rng)
    span = rng.choice([1 << 14, 4])
    rnd = rng.randrange(8)
    total = 0
    for _ in range(400):
        f, counts, after = colour_pass(live, refresh, span=span, rnd0=rnd)
        ref_counts, ref_live = sweeps_one_by_one(live, refresh, f)
        assert counts == ref_counts[:f] and len(ref_counts) >= f
        if f:
            assert after == ref_live
        total += f
        if f == 0 or not after:
            break
        live = after
        refresh = {p: (refresh[p] if p in live and not live[p][2] else None) for p in live}
        rnd += 3


def test_pass_stops_at_the_sweep_cap():
    rng = random.Random(7)
    live, refresh = random_case(rng)
    f, counts, after = colour_pass(live, refresh, max_sweeps=1)
    assert f <= 1
