"""Host-side wave planning of the library (csrc/plan.cpp), built with g++
and checked on random batches without a GPU: waves cover the cluster-sorted
positions in order, hold at most W queries and, with the compact store, at
most C encoded chunks, list exactly the chunks of the clusters their
positions touch, and end only where the next query or cluster would not fit."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2406_06761_gb300", "csrc")

WRAP = r"""
#include "plan.hpp"
#include <cstring>
extern "C" int plan(const uint32_t *chunks, uint32_t K, uint32_t C, const uint32_t *cnt, uint32_t W,
                    uint32_t *waves /* [max][4] */, uint32_t max_waves, uint32_t *z /* [2][max_z] */,
                    uint32_t max_z, uint32_t *nz_total)
{
    std::vector<wally::Wave> w;
    std::vector<uint32_t> zc, zk;
    wally::compact_waves(chunks, K, C, cnt, W, w, zc, zk);
    if (w.size() > max_waves || zc.size() > max_z) return -1;
    for (size_t i = 0; i < w.size(); i++) {
        waves[4 * i] = w[i].begin; waves[4 * i + 1] = w[i].len; waves[4 * i + 2] = w[i].z_off; waves[4 * i + 3] = w[i].nz;
    }
    for (size_t i = 0; i < zc.size(); i++) { z[i] = zc[i]; z[max_z + i] = zk[i]; }
    *nz_total = (uint32_t)zc.size();
    return (int)w.size();
}
extern "C" int plan_fixed(uint32_t n, uint32_t W, uint32_t *waves, uint32_t max_waves)
{
    std::vector<wally::Wave> w;
    wally::fixed_waves(n, W, w);
    if (w.size() > max_waves) return -1;
    for (size_t i = 0; i < w.size(); i++) { waves[2 * i] = w[i].begin; waves[2 * i + 1] = w[i].len; }
    return (int)w.size();
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("plan")
    src = d / "wrap.cpp"
    src.write_text(WRAP)
    so = d / "libplan.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, str(src),
                           os.path.join(CSRC, "plan.cpp"), "-o", str(so)])
    return ctypes.CDLL(str(so))


def _plan(lib, chunks, C, cnt, W):
    K = len(chunks)
    maxw, maxz = int(cnt.sum()) + 1, int((cnt > 0).sum() * chunks.max() * 4 + 16 + cnt.sum() * chunks.max())
    waves = np.zeros(4 * maxw, np.uint32)
    z = np.zeros(2 * maxz, np.uint32)
    tot = ctypes.c_uint32()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    nw = lib.plan(p(chunks), K, C, p(cnt), W, p(waves), maxw, p(z), maxz, ctypes.byref(tot))
    assert nw >= 0
    return waves[:4 * nw].reshape(nw, 4), z[:tot.value], z[maxz:maxz + tot.value]


@pytest.mark.parametrize("seed", range(12))
def test_compact_waves_invariants(lib, seed):
    rng = np.random.default_rng(seed)
    K = int(rng.integers(1, 40))
    chunks = rng.integers(1, 4, K).astype(np.uint32)
    cnt = (rng.integers(0, 30, K) * (rng.random(K) < 0.7)).astype(np.uint32)
    C = int(chunks.max()) + int(rng.integers(0, 6))
    W = int(rng.integers(1, 50))
    n = int(cnt.sum())
    waves, zc, zk = _plan(lib, chunks, C, cnt, W)
    start = np.concatenate([[0], np.cumsum(cnt.astype(np.int64))])
    cluster_of = np.repeat(np.arange(K), cnt)           # cluster of every sorted position
    pos = 0
    for i, (b, ln, zoff, nz) in enumerate(waves):
        assert b == pos and 1 <= ln <= W                 # contiguous cover, at most W queries
        pos += ln
        touched = list(dict.fromkeys(cluster_of[b:b + ln].tolist()))
        want_c = [k for k in touched for _ in range(chunks[k])]
        want_j = [j for k in touched for j in range(chunks[k])]
        assert list(zc[zoff:zoff + nz]) == want_c and list(zk[zoff:zoff + nz]) == want_j
        assert nz == sum(int(chunks[k]) for k in touched) <= C
        if i + 1 < len(waves):                           # ends only where the next would not fit
            nxt = int(cluster_of[b + ln])
            same = nxt == touched[-1]
            assert ln == W or (not same and nz + chunks[nxt] > C)
    assert pos == n
    assert len(zc) == sum(w[3] for w in waves)


def test_compact_waves_empty_and_fixed(lib):
    chunks = np.array([1, 2], np.uint32)
    waves, zc, _ = _plan(lib, chunks, 2, np.zeros(2, np.uint32), 8)
    assert len(waves) == 0 and len(zc) == 0
    out = np.zeros(64, np.uint32)
    nw = lib.plan_fixed(10, 4, out.ctypes.data_as(ctypes.c_void_p), 32)
    assert nw == 3 and out[:6].tolist() == [0, 4, 4, 4, 8, 2]
