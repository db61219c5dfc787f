"""CPU model check of the resident serving kernel's tile hand-off.

The resident kernel's producers claim tile indices from a device counter and
wait until the host has published them (resident_kernels.cuh,
ResidentSource::claim): the waiter holding the first unpublished index polls
the host's tail and mirrors it into several device copies; the others read
their copy; a stop flag, read by the head waiter only every 8th poll and
always before the tail, ends the instance once every published tile is taken.

This test runs that protocol step by step under seeded random interleavings of
the host (publishing batches of tiles, then setting stop) and the producers
(each memory access of the claim loop is one step; the mirror update writes
its copies one at a time).  Invariants checked on every run:

  * every published tile is taken exactly once, and no index beyond the final
    tail is taken;
  * every producer ends (the run terminates once stop is set);
  * a producer ends only holding an index at or beyond the final tail.

A second model checks the completion side: tiles finishing in any order on
any CTA, the last one of a request resetting its slot's count and writing the
request's sequence number, the host recycling slots only after it has seen
that number.  The host must never see a request done before all its tiles
are, and every count must return to zero.

The models are of the protocol, written here from its description; they share
no code with the CUDA source.
"""
import random

import pytest

MIRRORS = 8


class Model:
    def __init__(self, n_producers, batches, seed):
        self.rng = random.Random(seed)
        self.claimed = 0                      # device claim counter
        self.m_tail = [0] * MIRRORS           # mirrored tail, per copy
        self.m_stop = [0] * MIRRORS           # mirrored stop, per copy
        self.tail = 0                         # host tail
        self.stop = 0                         # host stop flag
        self.batches = list(batches)
        self.taken = []
        self.ended = []
        self.producers = [self._producer(p) for p in range(n_producers)]
        self.host = self._host()

    # every yield is one step another actor may interleave with
    def _host(self):
        for n in self.batches:
            self.tail += n
            yield
        self.stop = 1
        yield

    def _mirror_all(self, word, value):
        for c in range(MIRRORS):
            arr = self.m_tail if word == 0 else self.m_stop
            arr[c] = max(arr[c], value)
            yield

    def _producer(self, p):
        copy = p % MIRRORS
        while True:
            k = self.claimed
            self.claimed += 1
            yield
            i = 0
            while True:
                i += 1
                seen = self.m_tail[copy]
                yield
                if k < seen:
                    self.taken.append(k)
                    break
                if k == seen:
                    st = 0
                    if i % 8 == 0:
                        st = self.stop
                        yield
                    tl = self.tail
                    yield
                    if tl > seen:
                        yield from self._mirror_all(0, tl)
                    if k < tl:
                        self.taken.append(k)
                        break
                    if st:
                        yield from self._mirror_all(1, 1)
                        self.ended.append(k)
                        return
                else:
                    stopped = self.m_stop[copy]
                    yield
                    if stopped:
                        again = self.m_tail[copy]
                        yield
                        if k < again:
                            self.taken.append(k)
                            break
                        self.ended.append(k)
                        return
            yield   # the tile is processed; claim the next

    def run(self, max_steps=2_000_000):
        actors = list(self.producers) + [self.host]
        steps = 0
        while actors:
            a = self.rng.choice(actors)
            try:
                next(a)
            except StopIteration:
                actors.remove(a)
            steps += 1
            assert steps < max_steps, "the protocol did not terminate"
        return steps


@pytest.mark.parametrize("seed", range(40))
def test_every_published_tile_taken_once_and_every_producer_ends(seed):
    rng = random.Random(1000 + seed)
    n_prod = rng.choice([1, 2, 3, 5, 9, 17])
    batches = [rng.choice([0, 1, 1, 2, 3, 7, 20]) for _ in range(rng.randint(0, 12))]
    m = Model(n_prod, batches, seed)
    m.run()
    final = sum(batches)
    assert sorted(m.taken) == list(range(final)), (n_prod, batches)
    assert len(m.ended) == n_prod
    assert all(k >= final for k in m.ended)


def test_stop_with_nothing_published_ends_every_producer():
    m = Model(6, [], 7)
    m.run()
    assert m.taken == [] and len(m.ended) == 6


def test_a_planted_mistake_is_caught():
    # reading the tail before the stop flag (the order the kernel avoids) can
    # end the instance with published tiles untaken: some seed shows it
    class TailFirst(Model):
        def _producer(self, p):
            copy = p % MIRRORS
            while True:
                k = self.claimed
                self.claimed += 1
                yield
                while True:
                    seen = self.m_tail[copy]
                    yield
                    if k < seen:
                        self.taken.append(k)
                        break
                    if k == seen:
                        tl = self.tail
                        yield
                        st = self.stop
                        yield
                        if tl > seen:
                            yield from self._mirror_all(0, tl)
                        if k < tl:
                            self.taken.append(k)
                            break
                        if st:
                            yield from self._mirror_all(1, 1)
                            self.ended.append(k)
                            return
                    else:
                        stopped = self.m_stop[copy]
                        yield
                        if stopped:
                            again = self.m_tail[copy]
                            yield
                            if k < again:
                                self.taken.append(k)
                                break
                            self.ended.append(k)
                            return
                yield

    lost = 0
    for seed in range(300):
        m = TailFirst(2, [1, 1, 1], seed)
        m.run()
        lost += sorted(m.taken) != list(range(3))
    assert lost > 0


class CompletionModel:
    """The completion side: CTAs count finished tiles per slot; the CTA that
    counts a request's last tile resets the count and writes the request's
    sequence number to the slot's completion word; the host reuses a slot only
    after it has seen that word.  Steps interleave at random."""

    def __init__(self, n_slots, requests, n_ctas, seed):
        self.rng = random.Random(seed)
        self.counts = [0] * n_slots
        self.done = [0] * n_slots
        self.seq = [0] * n_slots
        self.free = list(range(n_slots))
        self.pending = list(requests)         # tile counts of the requests to serve
        self.queue = []                       # published (slot, seq, n_tiles, tile id)
        self.finished_tiles = {}              # (slot, seq) -> tiles finished so far
        self.live = {}                        # slot -> (seq, n_tiles)
        self.seen_done = []
        self.ctas = [self._cta() for _ in range(n_ctas)]
        self.host = self._host()

    def _host(self):
        while self.pending or self.live:
            # completions
            for slot, (sq, n) in list(self.live.items()):
                if self.done[slot] == sq:
                    assert self.finished_tiles[(slot, sq)] == n, "completion seen before every tile finished"
                    self.seen_done.append((slot, sq))
                    del self.live[slot]
                    self.free.append(slot)
                yield
            # admission
            if self.pending and self.free:
                n = self.pending.pop(0)
                slot = self.free.pop()
                self.seq[slot] += 1
                sq = self.seq[slot]
                self.live[slot] = (sq, n)
                self.finished_tiles[(slot, sq)] = 0
                for t in range(n):
                    self.queue.append((slot, sq, n, t))
            yield

    def _cta(self):
        while True:
            if not self.queue:
                if not self.pending and not self.live:
                    return
                yield
                continue
            slot, sq, n, t = self.queue.pop(self.rng.randrange(len(self.queue)))
            yield                               # the tile runs
            self.finished_tiles[(slot, sq)] += 1
            yield                               # barrier, fence
            old = self.counts[slot]
            self.counts[slot] = old + 1         # the atomic add
            yield
            if old == n - 1:
                self.counts[slot] = 0
                yield                           # system fence
                self.done[slot] = sq
            yield

    def run(self):
        actors = [self.host] + self.ctas
        steps = 0
        while actors:
            a = self.rng.choice(actors)
            try:
                next(a)
            except StopIteration:
                actors.remove(a)
            steps += 1
            assert steps < 2_000_000, "did not terminate"


@pytest.mark.parametrize("seed", range(30))
def test_completion_is_seen_only_after_every_tile_and_slots_recycle(seed):
    rng = random.Random(5000 + seed)
    requests = [rng.choice([1, 1, 2, 3, 8]) for _ in range(rng.randint(1, 40))]
    m = CompletionModel(n_slots=rng.choice([1, 2, 4]), requests=requests, n_ctas=rng.choice([1, 3, 6]), seed=seed)
    m.run()
    assert len(m.seen_done) == len(requests)
    assert all(c == 0 for c in m.counts)
