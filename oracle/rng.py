"""SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), used for the seeded cubature draws.

The paper draws cubature candidates at random (Sec. 5) without naming a generator. Both
sides implement this one published generator independently so their draws coincide.

keyed(seed, a, b) derives a stream state from a seed and two integer keys by feeding the
keys through two generator outputs; draws are `next() % n` (modulo bias accepted, it is
part of the definition).

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix(z):
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


class SplitMix64:
    def __init__(self, state):
        self.s = state & M64

    def next(self):
        self.s = (self.s + GAMMA) & M64
        return mix(self.s)


def keyed(seed, a, b):
    g = SplitMix64(seed)
    g.s = g.next() ^ (a & M64)
    g.s = g.next() ^ (b & M64)
    return g


def draw_without_replacement(gen, items, k):
    """Partial Fisher-Yates over `items` (in the given order); returns the first k picks."""
    arr = list(items)
    n = len(arr)
    k = min(k, n)
    for j in range(k):
        r = j + gen.next() % (n - j)
        arr[j], arr[r] = arr[r], arr[j]
    return arr[:k]
