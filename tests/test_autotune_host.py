"""Autotuner host logic (no GPU): the search over a synthetic timer, the
size-class keys, the on-disk cache and the batch thread-count choice."""
import json

import pytest

from paper_1908_06909_gb300 import autotune as A


def synthetic(best, bwd_best_scatter, calls):
    """Timer whose fwd+bwd minimum is `best` (tile_u, tile_v, order) and whose
    bwd minimum for that tile is `bwd_best_scatter`."""
    def measure(c, what):
        calls.append((c, what))
        d = abs(c.tile_u - best[0]) + abs(c.tile_v - best[1]) + 3 * (c.order != best[2])
        if what == "fwd+bwd":
            assert c.scatter == A.SCATTER_ATOMIC
            return 10.0 + d
        return 4.0 + d + (0.0 if c.scatter == bwd_best_scatter else 1.5)
    return measure


@pytest.mark.parametrize("threads", [None, 32, 64, 128, 256])
def test_search_finds_minimum(threads):
    cands = A.candidates(threads)
    for k, (tu, tv, o) in enumerate(cands):
        for sc in A.SCATTERS:
            calls = []
            choice, ms = A.search(synthetic((tu, tv, o), sc, calls), threads)
            assert choice == A.Choice(tu, tv, o, sc)
            # every tile/order candidate measured once, plus each scatter
            assert len(calls) == len(cands) + len(A.SCATTERS)
            # a faster scatter than atomic drops the bwd part from 5.5 to 4.0
            assert ms == pytest.approx(10.0 if sc == A.SCATTER_ATOMIC else 8.5)


def test_candidates_respect_thread_count():
    for n, tiles in A.TILES.items():
        for tu, tv, o in A.candidates(n):
            assert tu * tv == n and o in (A.ORDER_ROW, A.ORDER_MORTON)
    assert len(A.candidates(None)) == 2 * sum(len(t) for t in A.TILES.values())
    with pytest.raises(ValueError):
        A.candidates(96)


def test_size_class_buckets():
    assert A.size_class(4096, 64 * 64, 1, 64) == "t12_p12_c1_n64"
    assert A.size_class(4097, 64 * 64, 1, 64) == "t13_p12_c1_n64"
    assert A.size_class(1, 1, 4, None) == "t0_p0_c4_nany"
    assert A.size_class(1, 1, 4, 32) == "t0_p0_c4_n32"
    assert A.size_class(5_308_416, 512 * 512, 1, 128) == "t23_p18_c1_n128"


def test_cache_roundtrip_and_hit(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    c = A.Cache(path, device="devA", version="1")
    calls = []
    key = A.size_class(1000, 4096, 1, 64)
    ch, ms = A.tune_problem(key, lambda: synthetic((16, 4, A.ORDER_ROW), A.SCATTER_ATOMIC, calls),
                            64, c)
    assert ch == A.Choice(16, 4, A.ORDER_ROW, A.SCATTER_ATOMIC) and calls
    c.save()
    data = json.load(open(path))
    assert data["devA|1"][key]["choice"] == [16, 4, A.ORDER_ROW, A.SCATTER_ATOMIC]
    # a fresh cache object on the same file answers without measuring
    c2 = A.Cache(path, device="devA", version="1")
    calls2 = []
    ch2, ms2 = A.tune_problem(key, lambda: calls2.append("built") or synthetic((8, 8, 1), 1, calls2),
                              64, c2)
    assert (ch2, ms2) == (ch, ms) and not calls2
    # another device or library version does not share entries
    c3 = A.Cache(path, device="devB", version="1")
    assert c3.get(key) is None
    # a corrupt file is ignored
    open(path, "w").write("{not json")
    assert A.Cache(path, device="devA", version="1").get(key) is None


def test_candidates_hold_whole_warps():
    cands = A.candidates(None)
    assert cands and all(tu * tv >= 32 and (tu * tv) % 32 == 0 for tu, tv, _ in cands)
    assert len(A.candidates(None, min_threads=128)) == 2 * (len(A.TILES[128]) + len(A.TILES[256]))
    assert A.size_class(10, 10, 4, None) == "t4_p4_c4_nany"
    assert A.size_class(10, 10, 4, None, 64) == "t4_p4_c4_nge64"


def test_batch_scatter_space():
    calls = []
    ch, _ = A.search(synthetic((8, 8, 1), A.SCATTER_SORT, calls), None, scatters=A.BATCH_SCATTERS)
    assert ch.scatter in A.BATCH_SCATTERS
    assert sum(1 for _, what in calls if what == "bwd") == len(A.BATCH_SCATTERS)
