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
    w = b.modmuls_per_kind(L, N, lg, 30, 1, 16, 16)
    assert sum(w.values()) == 30 * per_ks + 16 * 16 * 2 * L * N
    assert abs(sum(w.values()) / 1e6 - 53.1) < 0.1


def test_recorded_traffic_is_scaled_per_item_and_gated_by_the_source_hash():
    b = _bench()
    t = b.recorded_traffic("ks_b")
    if t is None:  # the committed capture predates the current kernel sources
        return
    assert b.recorded_traffic("ks_b", 1024) == t
    assert abs(b.recorded_traffic("ks_b", 2048) - 2 * t) < 1
    assert b.recorded_traffic("no_such_kernel") is None
