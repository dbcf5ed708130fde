"""Algorithm 1's "u not in L" test against the visited sets a search may keep
instead (Alg. 1, Sec. 3.2): a permanent set, and the forgetful set the GPU
search keeps (2^b slots, two probes, a new id replacing the first slot's id
when both are taken).  A forgotten id only costs a recomputed distance: a
vertex still in L is dropped as a repeat, and one that left a full L cannot
re-enter it, because the key of L's last entry only decreases.  So the final
list and the number of expansions are the same for every variant; only the
count of distance computations differs.

Pure-Python searches on small random graphs; the keys are (dist_F, dist, id)
with a label filter, compared lexicographically."""
import numpy as np
import pytest


def _keys(x, labels, q, lab):
    d = ((x.astype(np.float64) - q) ** 2).sum(1)
    f = (labels != lab).astype(np.int64)
    return f, d


class _Exact:
    def __init__(self):
        self.s = set()

    def check_insert(self, u):
        if u in self.s:
            return False
        self.s.add(u)
        return True


class _None:
    def check_insert(self, u):
        return True


class _Forgetful:
    def __init__(self, bits):
        self.bits = bits
        self.t = [None] * (1 << bits)

    def check_insert(self, u):
        h = ((u * 0x9E3779B1) & 0xFFFFFFFF) >> (32 - self.bits)
        h1 = (h + 1) & ((1 << self.bits) - 1)
        if self.t[h] is None:
            self.t[h] = u
            return True
        if self.t[h] == u:
            return False
        if self.t[h1] is None:
            self.t[h1] = u
            return True
        if self.t[h1] == u:
            return False
        self.t[h] = u
        return True


def _search(graph, f, d, entry, ls, visited):
    """Greedy search with the lexicographic key; returns (ids of L, hops,
    distance computations)."""
    def key(u):
        return (int(f[u]), float(d[u]), int(u))

    L = [key(entry)]
    expanded = set()
    visited.check_insert(entry)
    hops, dcs = 0, 1
    while True:
        sel = next((e for e in L if e[2] not in expanded), None)
        if sel is None:
            break
        expanded.add(sel[2])
        hops += 1
        for u in graph[sel[2]]:
            if u < 0:
                continue
            full = len(L) == ls
            if full and f[u] > L[-1][0]:
                continue                              # early rejection on dist_F
            if not visited.check_insert(int(u)):
                continue
            dcs += 1
            ku = key(int(u))
            if any(e[2] == ku[2] for e in L):        # u in L: a repeat
                continue
            if full and not ku < L[-1]:
                continue
            L.append(ku)
            L.sort()
            del L[ls:]
    return [e[2] for e in L], hops, dcs


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("ls", [4, 10, 24])
def test_forgetful_sets_change_no_result(seed, ls):
    rng = np.random.default_rng(seed)
    n, dim, R = 400, 6, 8
    x = rng.standard_normal((n, dim)).astype(np.float32)
    labels = rng.integers(0, 5, n)
    graph = np.full((n, R), -1, np.int64)
    for v in range(n):
        nb = rng.choice(np.delete(np.arange(n), v), R, replace=False)
        deg = int(rng.integers(R // 2, R + 1))
        graph[v, :deg] = nb[:deg]
    entry = int(rng.integers(0, n))
    dcs_seen = []
    for qi in range(12):
        q = rng.standard_normal(dim)
        f, d = _keys(x, labels, q, int(rng.integers(0, 5)))
        ref = _search(graph, f, d, entry, ls, _Exact())
        dcs_seen.append(ref[2])
        for vis in (_None(), _Forgetful(2), _Forgetful(4), _Forgetful(6)):
            got = _search(graph, f, d, entry, ls, vis)
            assert got[0] == ref[0] and got[1] == ref[1]
            assert got[2] >= ref[2]
    assert sum(dcs_seen) > 0


def test_forgetful_set_recomputes_less_than_none():
    rng = np.random.default_rng(5)
    n, dim, R = 500, 6, 10
    x = rng.standard_normal((n, dim)).astype(np.float32)
    labels = np.zeros(n, np.int64)
    graph = np.stack([rng.choice(np.delete(np.arange(n), v), R, replace=False) for v in range(n)])
    f, d = _keys(x, labels, rng.standard_normal(dim), 0)
    exact = _search(graph, f, d, 0, 32, _Exact())
    none = _search(graph, f, d, 0, 32, _None())
    small = _search(graph, f, d, 0, 32, _Forgetful(5))
    assert exact[0] == none[0] == small[0]
    assert exact[2] <= small[2] <= none[2]
