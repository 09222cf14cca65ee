"""wally_rotate_noalloc: the rotation for callers that cannot allocate device
memory at call time (a serving thread that must not trigger the device-wide
synchronisation of cudaMalloc/cudaFree, or a process whose framework allocator
owns all device memory).  Its result must equal wally_rotate's, bit for bit
(integer arithmetic, zero tolerance), on consecutive calls that share its
static scratch.  Collected last, after every other test."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import wally as Wl
from paper_2406_06761_gb300 import workload as W

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda", 0)


def _inputs(prm, n, seed, which_key):
    cr = W.client_randomness(n, prm.N, prm.q, prm.P, seed=seed)
    v = np.random.default_rng(seed).integers(0, prm.t, size=(n, prm.N), dtype=np.uint64)
    cts = np.stack([O.encrypt_slots(prm, cr.secret[i], v[i], cr.enc_a[i], cr.enc_e[i]) for i in range(n)])
    k = prm.k1 if which_key == 0 else prm.kg
    keys = np.stack([O.keygen(prm, cr.secret[i], k, cr.key_a[i, which_key], cr.key_e[i, which_key])
                     for i in range(n)])
    return k, Wl.u64_tensor(cts, DEV), Wl.u64_tensor(keys, DEV)


@pytest.mark.parametrize("name", ["tiny", "batched"])
def test_rotate_noalloc_matches_rotate_on_consecutive_calls(name):
    w = W.WORKLOADS[name]
    prm = O.params(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    n = 3
    for call, (seed, which_key) in enumerate([(21, 0), (22, 1)]):
        k, cts, keys = _inputs(prm, n, seed, which_key)
        ref = torch.empty((n, 2, prm.L, prm.N), dtype=torch.int64, device=DEV)
        got = torch.full_like(ref, -1)
        Wl.wally_rotate(ctx.ptr, n, k, cts, keys, ref)
        Wl.wally_rotate_noalloc(ctx.ptr, n, k, cts, keys, got)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"call {call}"
    ctx.close()


def test_rotate_noalloc_rejects_too_many():
    w = W.WORKLOADS["batched"]
    ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim)
    N, L = ctx.N, ctx.L
    per_item = 8 * N * (7 * L + 2 + 3 * L * (L + 1))
    n = (16 << 20) // per_item + 1
    x = torch.zeros(8, dtype=torch.int64, device=DEV)
    with pytest.raises(Wl.WallyError) as ei:
        Wl.wally_rotate_noalloc(ctx.ptr, n, 3, x, x, x)
    assert ei.value.code == Wl.WALLY_EINVAL
    ctx.close()
