"""Cache keys and hit / miss sets of a scripted query sequence, exactly.

Alg. 1 evaluates a window only if it is not processed, and eviction (LRU,
Sec. 3.3) makes it unprocessed again.  The library keeps the processed state
as finalized stride x stride tiles of every step keyed (step, tile row, tile
column), with least-recently-used eviction of tiles the running query does
not use.  The expectation here is a model of that tile cache whose window
sets come from the oracle's kappa (Alg. 3): the windows of step k-1 are
kappa of the missing tiles of J_k, and the tiles they read are those their
regions (oracle window_rect) cover.  After every query of the sequence the
windows evaluated per step, the hit / miss / eviction counts and the cached
key set of every step must equal the model's, integer for integer; the
sequence mixes overlapping, repeated, disjoint and negative-coordinate
queries with a cache small enough to evict, and one query too large for the
cache (IDF_ENOMEM, after which the world stays usable)."""
from collections import OrderedDict

import numpy as np
import pytest

import synth
from oracle import kappa as K_

class TileCacheModel:
    def __init__(self, n_slots, H, s, K):
        self.n, self.H, self.s, self.K = n_slots, H, s, K
        self.lru = OrderedDict()          # (step, ty, tx) -> None, least recent first
        self.hits = self.misses = self.evictions = self.windows = self.tiles = 0

    def _tiles_of(self, y0, x0, h, w):
        s = self.s
        return {(ty, tx) for ty in range(y0 // s, (y0 + h - 1) // s + 1)
                for tx in range(x0 // s, (x0 + w - 1) // s + 1)}

    def plan(self, x0, y0, w, h, mutate):
        """Missing tiles per step and windows per step; with mutate, the LRU
        walk of a real query (hits touched, counters advanced)."""
        need = self._tiles_of(y0, x0, h, w)
        missing, windows = {}, {}
        pinned = set()
        for k in range(self.K, 0, -1):
            mk = []
            for t in sorted(need):
                key = (k,) + t
                if key in self.lru:
                    if mutate:
                        self.lru.move_to_end(key)
                        pinned.add(key)
                        self.hits += 1
                else:
                    mk.append(t)
            if mutate:
                self.misses += len(mk)
            missing[k] = mk
            ws = set()
            for (ty, tx) in mk:
                ws.update(K_.kappa(ty * self.s, tx * self.s, self.s, self.s, self.H, self.s))
            windows[k - 1] = sorted(ws)
            need = set()
            for (i, j) in ws:
                need |= self._tiles_of(*K_.window_rect(i, j, self.H, self.s))
        return missing, windows, pinned

    def query(self, x0, y0, w, h):
        missing, windows, pinned = self.plan(x0, y0, w, h, True)
        inserted = []
        for k in range(1, self.K + 1):
            for t in missing[k]:
                key = (k,) + t
                if len(self.lru) >= self.n:
                    victim = next((v for v in self.lru if v not in pinned), None)
                    if victim is None:
                        for v in inserted:
                            del self.lru[v]
                        return False
                    del self.lru[victim]
                    self.evictions += 1
                self.lru[key] = None
                pinned.add(key)
                inserted.append(key)
        self.windows += sum(len(v) for v in windows.values())
        self.tiles += sum(len(v) for v in missing.values())
        return True

    def keys(self, k):
        return sorted((ty, tx) for (kk, ty, tx) in self.lru if kk == k)


QUERIES = [
    (0, 0, 48, 48),          # cold
    (16, 16, 48, 48),        # overlaps the first: hits, misses, evictions
    (10000, 10000, 32, 32),  # disjoint
    (0, 0, 48, 48),          # the first again, partly evicted
    (-40, 8, 20, 70),        # unaligned, negative coordinates
    (0, 0, 200, 200),        # working set above the cache: IDF_ENOMEM
    (16, 0, 16, 16),         # the world is still usable
    (-40, 8, 20, 70),        # repeat after the failed plan
]


@pytest.mark.gpu
def test_scripted_sequence_cache_keys_and_hits():
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config1_stack(test_denoiser=1)
    lv = st["level"][0]
    H, s, K = lv["window"], lv["stride"], lv["steps"]
    n_slots = 200
    W = idf.World(0, st, None, precision="fp32", cache_bytes=n_slots * s * s * 4)
    M = TileCacheModel(n_slots, H, s, K)
    assert W.stats()["levels"][0]["slots"] == n_slots
    prev = W.stats()["levels"][0]
    for qi, (x0, y0, w, h) in enumerate(QUERIES):
        _, windows, _ = M.plan(x0, y0, w, h, False)
        for k in range(K):
            assert W.debug_cone(x0, y0, w, h, 0, k) == windows[k], (qi, k)
        ok = M.query(x0, y0, w, h)
        if ok:
            W.query(x0, y0, w, h)
        else:
            with pytest.raises(idf.IdfError) as e:
                W.query(x0, y0, w, h)
            assert e.value.status == idf.IDF_ENOMEM
        cur = W.stats()["levels"][0]
        got = {f: cur[f] - prev[f] for f in ("cache_hits", "cache_misses", "evictions",
                                              "windows_evaluated", "tiles_computed")}
        prev = cur
        want = {"cache_hits": M.hits, "cache_misses": M.misses, "evictions": M.evictions,
                "windows_evaluated": M.windows, "tiles_computed": M.tiles}
        M.hits = M.misses = M.evictions = M.windows = M.tiles = 0
        assert got == want, (qi, got, want)
        for k in range(1, K + 1):
            assert W.debug_cache_keys(0, k) == M.keys(k), (qi, k)
        assert cur["tiles_cached"] == len(M.lru)
    W.close()


def test_model_counts_match_cone_closed_form():
    # the model's window count for an aligned cold query is Lemma 4's
    # sum_k (n + 2k + 1)^2 (n tiles per side), the oracle's cone count
    M = TileCacheModel(10 ** 9, 32, 16, 4)
    _, windows, _ = M.plan(0, 0, 48, 48, False)
    n = 3
    assert sum(len(v) for v in windows.values()) == sum((n + 2 * k + 1) ** 2 for k in range(4))
    assert [len(windows[k]) for k in range(3, -1, -1)] == K_.cone_window_counts(0, 0, 48, 48, 32, 16, 4)
