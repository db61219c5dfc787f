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

The model is of the protocol, written here from its description; it shares no
code with the CUDA source.
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
