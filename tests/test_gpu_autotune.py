"""Launch shapes and the autotuner: every shape gives the same bits, the
autotuner keeps the fastest candidate it timed, and a candidate whose
workspace cannot be allocated is skipped rather than failing the call."""
import numpy as np
import pytest
import torch

from paper_2406_06761_gb300 import harness as H
from paper_2406_06761_gb300 import wally as Wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wl():
    w = H.DeviceWorkload("batched", max_wave=256)
    yield w
    w.close()


def _run(wl, batch):
    out = wl.alloc_out(batch[3])
    out.zero_()
    wl.eval(batch, out)
    Wl.wally_sync(wl.ctx.ptr)
    return out


SHAPES = [
    dict(max_wave=256, lanes=2, mac_ctas_per_sm=3, ntt_ctas_per_sm=0, ks_core=0, mac_halves=0),
    dict(max_wave=100, lanes=1, mac_ctas_per_sm=1, ntt_ctas_per_sm=1, ks_core=1, mac_halves=1),
    dict(max_wave=333, lanes=2, mac_ctas_per_sm=2, ntt_ctas_per_sm=2, ks_core=0, mac_halves=1),
    dict(max_wave=2048, lanes=1, mac_ctas_per_sm=3, ntt_ctas_per_sm=3, ks_core=1, mac_halves=0),
]


def test_every_shape_gives_the_same_outputs(wl):
    batch = wl.device_batch(0, wl.n)
    Wl.wally_set_tuning(wl.ctx.ptr, **SHAPES[0])
    ref = _run(wl, batch)
    for s in SHAPES[1:]:
        Wl.wally_set_tuning(wl.ctx.ptr, **s)
        assert Wl.wally_get_tuning(wl.ctx.ptr).as_dict() == s
        assert torch.equal(_run(wl, batch), ref), s
    Wl.wally_set_tuning(wl.ctx.ptr, **SHAPES[0])


def test_autotune_keeps_the_fastest(wl):
    batch = wl.device_batch(0, 600)
    ids, idx, offs, chunks, _ = batch
    out = wl.alloc_out(chunks)
    best, table = Wl.wally_autotune(wl.ctx.ptr, ids.numel(), ids, wl.pool.cts, wl.pool.keys, idx, offs, out,
                                    candidates=SHAPES, reps=1)
    ms = [m for _, m in table]
    assert all(m > 0 for m in ms)
    assert best == int(np.argmin(ms))
    assert Wl.wally_get_tuning(wl.ctx.ptr).as_dict() == SHAPES[best]
    # the outputs of the last timed call are those of any shape
    Wl.wally_set_tuning(wl.ctx.ptr, **SHAPES[0])
    assert torch.equal(out, _run(wl, batch))


def test_autotune_skips_a_shape_that_does_not_fit(wl):
    batch = wl.device_batch(0, 64)
    ids, idx, offs, chunks, _ = batch
    out = wl.alloc_out(chunks)
    huge = dict(max_wave=1 << 22, lanes=2, mac_ctas_per_sm=3, ntt_ctas_per_sm=0, ks_core=0, mac_halves=0)  # ~100 TB
    best, table = Wl.wally_autotune(wl.ctx.ptr, ids.numel(), ids, wl.pool.cts, wl.pool.keys, idx, offs, out,
                                    candidates=[huge, SHAPES[0]], reps=1)
    assert table[0][1] == -1 and table[1][1] > 0 and best == 1
    assert Wl.wally_get_tuning(wl.ctx.ptr).as_dict() == SHAPES[0]


def test_invalid_shapes_are_rejected(wl):
    for bad in (dict(max_wave=0), dict(max_wave=8, lanes=3), dict(max_wave=8, mac_ctas_per_sm=4),
                dict(max_wave=8, ks_core=2), dict(max_wave=8, mac_halves=2)):
        with pytest.raises(Wl.WallyError) as e:
            Wl.wally_set_tuning(wl.ctx.ptr, **bad)
        assert e.value.code == Wl.WALLY_EINVAL


def test_staged_search(wl):
    """Without candidates: wave size x lanes first, then the CTA counts at the
    best of those, then the other NTT shape of the key-switch kernels at the
    best so far, then the half-tile multiply-accumulate at the best so far;
    the kept shape is the fastest timed."""
    batch = wl.device_batch(0, wl.n)
    ids, idx, offs, chunks, _ = batch
    out = wl.alloc_out(chunks)
    best, table = Wl.wally_autotune(wl.ctx.ptr, ids.numel(), ids, wl.pool.cts, wl.pool.keys, idx, offs, out, reps=1)
    assert len(table) == 11
    first = table[:6]
    assert sorted((s["max_wave"], s["lanes"]) for s, _ in first) == [(w, l) for w in (512, 1024, 2048) for l in (1, 2)]
    ok = [m for _, m in first if m > 0]
    s1 = first[[m for _, m in first].index(min(ok))][0]
    for s, _ in table[6:]:
        assert (s["max_wave"], s["lanes"]) == (s1["max_wave"], s1["lanes"])
    assert all(s["ks_core"] == 0 for s, _ in table[:9]) and table[9][0]["ks_core"] == 1
    ms9 = [m if m > 0 else float("inf") for _, m in table[:9]]
    s2 = table[int(np.argmin(ms9))][0]
    assert dict(table[9][0], ks_core=0) == s2
    assert all(s["mac_halves"] == 0 for s, _ in table[:10]) and table[10][0]["mac_halves"] == 1
    ms10 = [m if m > 0 else float("inf") for _, m in table[:10]]
    assert dict(table[10][0], mac_halves=0) == table[int(np.argmin(ms10))][0]
    ms = [m if m > 0 else float("inf") for _, m in table]
    assert best == int(np.argmin(ms))
    assert Wl.wally_get_tuning(wl.ctx.ptr).as_dict() == table[best][0]
    Wl.wally_set_tuning(wl.ctx.ptr, **SHAPES[0])
    assert torch.equal(out, _run(wl, batch))


def test_tuned_shapes_match_the_oracle(wl):
    """The other NTT shape of the key-switch kernels and the half-tile
    multiply-accumulate, on sampled queries of the batch: bit for bit the
    oracle's evaluation (the default shape is checked by the parity tests)."""
    import oracle as O
    from tests.test_gpu_workloads import _oracle_check
    prm = O.params(wl.w.log_n, wl.w.num_q, wl.w.q_bits, wl.w.t_bits, wl.w.dim)
    batch = wl.device_batch(0, wl.n)
    offs = batch[4]
    Wl.wally_set_tuning(wl.ctx.ptr, **SHAPES[1])
    out = _run(wl, batch).cpu().numpy().view(np.uint64)
    Wl.wally_set_tuning(wl.ctx.ptr, **SHAPES[0])
    for qi in (0, wl.n // 2, wl.n - 1):
        m = int(wl.chunks[wl.ids[qi]])
        _oracle_check(wl, prm, qi, out[int(offs[qi]):int(offs[qi]) + m])
