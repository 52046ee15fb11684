"""The conflict check's parallel form, modelled on the host.

Algorithm 4 (reading R3) accepts a slot when neither agent of its exchange
was claimed by an earlier accepted slot: the greedy set in priority order.
The controller computes it in chunks of the priority order, rejecting edges
blocked by earlier chunks' claims and running deterministic reservations
among each chunk's remaining edges.  This test replays that procedure step
by step (chunk filter, reservation rounds with decreasing round keys,
claims, rejections) on random edge lists with heavy conflicts and
self-edges, and checks it against the greedy definition for several chunk
sizes, including the reservation-key wrap."""
import random

import pytest


def greedy_accepted(edges):
    claimed, acc = set(), []
    for p, (u, v) in enumerate(edges):
        if u not in claimed and v not in claimed:
            acc.append(p)
            claimed.update((u, v))
    return acc


def chunked_reservations(edges, chunk, span=1 << 14, filter_blocked=True):
    claimed, acc = set(), []
    res = {}
    rnd = 0
    for c0 in range(0, len(edges), chunk):
        cand = {p for p in range(c0, min(c0 + chunk, len(edges)))
                if not filter_blocked or (edges[p][0] not in claimed and edges[p][1] not in claimed)}
        rounds = 0
        while cand:
            rounds += 1
            assert rounds <= chunk + 1
            if rnd % span == 0 and rnd != 0:
                res.clear()  # the key period wraps
            base = (span - 1 - rnd % span) << 18  # later rounds: smaller keys
            for p in cand:
                key = base | p
                for a in edges[p]:
                    res[a] = min(res.get(a, 1 << 40), key)
            won = {p for p in cand if all(res[a] == (base | p) for a in edges[p])}
            assert won, "the first candidate always wins its round"
            for p in sorted(won):
                acc.append(p)
                claimed.update(edges[p])
            cand = {p for p in cand - won if edges[p][0] not in claimed and edges[p][1] not in claimed}
            rnd += 1
    return sorted(acc)


@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("chunk", [1, 3, 16, 1024])
def test_chunked_reservations_equal_the_greedy_set(seed, chunk):
    rng = random.Random(seed)
    agents = rng.choice([3, 8, 40, 200])
    hot = rng.randrange(agents)
    edges = []
    for _ in range(rng.randrange(1, 300)):
        u = rng.randrange(agents)
        r = rng.random()
        v = u if r < 0.1 else (hot if r < 0.5 else rng.randrange(agents))  # self-edges, a hot agent
        edges.append((u, v))
    assert chunked_reservations(edges, chunk) == greedy_accepted(edges)


def test_chunked_reservations_across_key_wraps():
    rng = random.Random(7)
    edges = [(rng.randrange(6), rng.randrange(6)) for _ in range(200)]
    for span in (2, 4, 8):
        assert chunked_reservations(edges, 16, span=span) == greedy_accepted(edges)


def test_model_catches_a_missing_chunk_filter():
    # without the filter, an edge blocked by an earlier chunk's claim competes
    # in its own chunk and can be accepted: the check must see the difference
    differ = 0
    for seed in range(40):
        rng = random.Random(seed)
        edges = [(rng.randrange(8), rng.randrange(8)) for _ in range(60)]
        differ += chunked_reservations(edges, 4, filter_blocked=False) != greedy_accepted(edges)
    assert differ > 0
