"""Host-side helpers of bench.py (no GPU): the algorithmic work counts the
roofline divides by, and the ncu-traffic record it reads from profiles/."""
import importlib.util
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_work_per_query_at_the_full_scale_parameters():
    """N = 8192, L = 3, g = h = 16, one chunk: 30 key switches.  Per key
    switch: L digit INTTs, L^2 digit NTTs, 2 INTTs of the P residues, 2L
    NTTs of ModDown (each N/2 log2 N butterflies, inverses + N scalings),
    2(L+1)L N key products and 2LN P^-1 products; plus g h 2 L N MACs."""
    b = _bench()
    N, L, lg = 8192, 3, 13
    ntt = N // 2 * lg
    per_ks = L * (ntt + N) + L * L * ntt + 2 * (ntt + N) + 2 * (L + 1) * L * N + 2 * L * ntt + 2 * L * N
    w = b.work_per_kind(L, N, lg, 1, 1, 16, 16)
    path = sum(sum(w[k].values()) for k in ("ks_a", "ks_b", "ks_c", "mac"))
    assert path == 30 * per_ks + 16 * 16 * 2 * L * N
    assert abs(path / 1e6 - 53.1) < 0.1
    # the digit transforms: at the two chain starts in ks_a, the other 28 in ks_c
    assert w["ks_a"]["bfly"] == 2 * L * ntt and w["ks_c"]["bfly"] == 30 * 2 * L * ntt + 28 * L * ntt
    assert w["ks_b"]["mac"] == 30 * 2 * L * (L + 1) * N and w["mac"]["mac"] == 16 * 16 * 2 * L * N
    # butterfly equivalents weight each class by its own peak
    peaks = {"butterfly_per_s": 2.0, "modmul_per_s": 4.0, "mac128_per_s": 8.0}
    assert b.butterfly_equivalents({"bfly": 10, "mm": 8, "mac": 16}, peaks) == 10 + 4 + 4


def test_recorded_traffic_is_scaled_per_item_and_gated_by_the_source_hash():
    b = _bench()
    t = b.recorded_traffic("ks_b")
    if t is None:  # the committed capture predates the current kernel sources
        return
    t1 = b.recorded_traffic("ks_b", 1)
    assert abs(b.recorded_traffic("ks_b", 2048) - 2048 * t1) < 1e-3 * 2048 * t1
    assert b.recorded_traffic("no_such_kernel") is None


class _Ev:
    def __init__(self, t):
        self.t = t

    def elapsed_time(self, other):
        return other.t - self.t


def test_batch_latency_per_wave():
    """Queries finish with their wave: two steps of two calls each; the second
    call of a step starts 30 ms after the step; waves report their time from
    their call's start."""
    import numpy as np
    bench = _bench()
    marks = [("step", _Ev(0.0)), ("call", _Ev(0.0)), ("call", _Ev(30.0)),
             ("step", _Ev(100.0)), ("call", _Ev(100.0)), ("call", _Ev(130.0))]
    call = np.array([0, 0, 1, 2, 3], np.uint32)
    q = np.array([3, 1, 4, 2, 2], np.uint32)
    ms = np.array([10.0, 20.0, 5.0, 12.0, 7.0], np.float32)
    r = bench.batch_latency(marks, call, q, ms)
    lat = np.repeat([10.0, 20.0, 35.0, 12.0, 37.0], [3, 1, 4, 2, 2])
    assert r["waves"] == 5
    assert abs(r["p50"] - np.percentile(lat, 50)) < 1e-6 and abs(r["p99"] - np.percentile(lat, 99)) < 1e-6
    assert r["max"] == 37.0
