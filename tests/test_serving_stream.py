"""The serving loop's request stream (host only): clients each send one real
query and negative-binomial fakes (Alg. "Client Query Generation"), every
query at its own uniform time (Alg. "Schedule"), so the arrivals form a
Poisson process; real queries pick clusters in proportion to their sizes,
fakes uniformly; real and fake submissions come from disjoint parts of the
client pool."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2406_06761_gb300 import serving as S  # noqa: E402


def test_poisson_stream_statistics():
    sizes = np.array([100, 300, 600], np.int64)
    st = S.poisson_stream(20000.0, 2.0, sizes, 64, seed=3)
    n = len(st.arrival)
    assert abs(n - 40000) < 6 * np.sqrt(40000)                       # offered rate, real + fake
    assert np.all(np.diff(st.arrival) >= 0) and st.arrival[0] >= 0 and st.arrival[-1] <= 2.0
    gaps = np.diff(st.arrival)
    assert abs(gaps.mean() - 1 / 20000) / (1 / 20000) < 0.05           # exponential gaps
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05
    real = st.is_real
    share = np.bincount(st.cluster[real], minlength=3) / real.sum()
    assert np.allclose(share, sizes / sizes.sum(), atol=0.01)         # proportional to size
    fshare = np.bincount(st.cluster[~real], minlength=3) / (~real).sum()
    assert np.allclose(fshare, 1 / 3, atol=0.05)                      # uniform fakes
    assert st.entry[real].max() < st.entry[~real].min() <= st.entry[~real].max() < 64


def test_fakes_per_client_are_negative_binomial():
    """One real query per client and NB(r = 0.5, p = 0.9) fakes (numpy's
    convention: mean r(1-p)/p = 0.0556, variance r(1-p)/p^2 = 0.0617)."""
    st = S.poisson_stream(200000.0, 2.0, np.array([5, 5]), 256, nb_r=0.5, nb_p=0.9, seed=7)
    clients = st.client.max() + 1
    real_per_client = np.bincount(st.client[st.is_real], minlength=clients)
    assert np.all(real_per_client == 1)
    fakes = np.bincount(st.client[~st.is_real], minlength=clients)
    mean, var = fakes.mean(), fakes.var()
    se = np.sqrt(0.0617 / clients)
    assert abs(mean - 0.5 * 0.1 / 0.9) < 5 * se
    assert abs(var - 0.5 * 0.1 / 0.81) < 0.1 * 0.0617
    # the count distribution: P(0) = p^r = 0.9487, P(1) = r(1-p)p^r = 0.0474
    assert abs((fakes == 0).mean() - 0.9 ** 0.5) < 0.005
    assert abs((fakes == 1).mean() - 0.5 * 0.1 * 0.9 ** 0.5) < 0.005
    # a client's fakes reach the server at independent times, not as one burst
    multi = np.flatnonzero(fakes >= 2)
    assert len(multi) > 0
    spread = [np.ptp(st.arrival[st.client == c]) for c in multi[:200]]
    assert np.median(spread) > 0.2
