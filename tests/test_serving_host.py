"""Host-side pieces of the server that need no GPU: request sizing and stats."""
import numpy as np

from paper_2006_07057_gb300 import serve


def test_request_bytes_grows_with_size_and_features():
    small = serve.request_bytes(256, 256, 128, 3)
    big = serve.request_bytes(1 << 16, 1 << 16, 128, 3)
    wide = serve.request_bytes(256, 256, 512, 3)
    assert big > small and wide > small
    # dominated by the stored features: 4 bytes per entry on both clouds
    assert big >= 4 * (2 << 16) * 128


def test_latency_stats_percentiles():
    reqs = []
    for i in range(100):
        r = serve.Request(i, np.zeros((1, 2), np.float32), np.zeros((1, 2), np.float32),
                          np.ones(1, np.float32), np.ones(1, np.float32), np.zeros((1, 2), np.float32),
                          1.0, 1, arrival_s=0.01 * i)
        r.done_s = r.arrival_s + 0.001 * (i + 1)
        reqs.append(r)
    st = serve.latency_stats(reqs)
    assert st["requests"] == 100
    assert abs(st["latency_ms_p50"] - 51.0) < 1e-6 and abs(st["latency_ms_p99"] - 100.0) < 1e-6


def test_free_list_first_fit_against_a_brute_force_model():
    # random allocations and frees; the free list must hand out disjoint,
    # 256-byte aligned ranges inside the pool, account for every byte, coalesce
    # neighbours, and fail exactly when no free gap is large enough
    rng = np.random.default_rng(0)
    size = 1 << 20
    fl = serve.FreeList(size)
    used = {}   # offset -> length
    for _ in range(3000):
        if used and rng.random() < 0.45:
            off = int(rng.choice(list(used)))
            fl.free(off, used.pop(off))
        else:
            want = int(rng.integers(1, 40000))
            got = fl.alloc(want)
            need = max(256, (want + 255) // 256 * 256)
            # brute force: the gaps between used ranges, in address order
            gaps, pos = [], 0
            for o in sorted(used):
                if o > pos:
                    gaps.append((pos, o - pos))
                pos = o + used[o]
            if pos < size:
                gaps.append((pos, size - pos))
            first = next((g for g in gaps if g[1] >= need), None)
            if first is None:
                assert got is None
                continue
            assert got == (first[0], need)
            used[got[0]] = got[1]
        assert fl.in_use == sum(used.values())
        assert sum(ln for _, ln in fl.free_list) == size - fl.in_use
        offs = [o for o, _ in fl.free_list]
        assert offs == sorted(offs)
        for (o1, l1), (o2, _) in zip(fl.free_list, fl.free_list[1:]):
            assert o1 + l1 < o2            # coalesced: no two free ranges touch
        assert all(o % 256 == 0 and ln % 256 == 0 for o, ln in fl.free_list)


def test_first_mode_takes_the_hybrid_pass_for_large_low_dimensional_requests():
    def req(n, d, r):
        z = np.zeros((n, d), np.float32)
        w = np.ones(n, np.float32) / n
        return serve.Request(0, z, z, w, w, np.zeros((r, d), np.float32), 1.0, 1)
    big = 1 << 15   # 2 n ldr = 2^25 entries at r = 512: past the one-launch solver
    assert [serve.first_mode(req(big, d, 512)) for d in (1, 2, 3, 4, 5, 16)] == \
        ["hybrid"] * 4 + ["stored"] * 2
    # within the one-launch solver's size rule ((n + m) ldr <= 2^24 per term)
    assert serve.first_mode(req(1 << 14, 3, 512)) == "stored"
    assert serve.first_mode(req(1 << 14, 3, 513)) == "hybrid"
