"""The serving loop's request stream (host only): Poisson arrivals at the
offered rate, real queries on clusters in proportion to their sizes, fakes
uniform, and submissions of real and fake queries from disjoint parts of the
client pool."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2406_06761_gb300 import serving as S  # noqa: E402


def test_poisson_stream_statistics():
    sizes = np.array([100, 300, 600], np.int64)
    st = S.poisson_stream(20000.0, 2.0, sizes, 64, fake_fraction=0.05, seed=3)
    n = len(st.arrival)
    assert abs(n - 40000) < 5 * np.sqrt(40000)                       # Poisson count
    assert np.all(np.diff(st.arrival) >= 0) and st.arrival[0] >= 0 and st.arrival[-1] <= 2.0
    gaps = np.diff(st.arrival)
    assert abs(gaps.mean() - 1 / 20000) / (1 / 20000) < 0.05           # exponential gaps
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05
    real = st.is_real
    assert abs((~real).mean() - 0.05) < 0.01
    share = np.bincount(st.cluster[real], minlength=3) / real.sum()
    assert np.allclose(share, sizes / sizes.sum(), atol=0.01)         # proportional to size
    fshare = np.bincount(st.cluster[~real], minlength=3) / (~real).sum()
    assert np.allclose(fshare, 1 / 3, atol=0.03)                      # uniform fakes
    n_fake_entries = round(64 * 0.05)
    assert st.entry[real].max() < 64 - n_fake_entries <= st.entry[~real].min()
