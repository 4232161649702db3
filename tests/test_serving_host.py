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
