"""Plaintext CRT recombination (host side, no GPU): exact for values within
half the product of the moduli, and the GPU path with two plaintext moduli
(each its own context) recovers dot products that wrap around either one."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import crt
from paper_2406_06761_gb300 import workload as W


def test_combine_recovers_centred_values():
    t0, t1 = 114689, O.prev_prime_1mod(114689, 8192)
    rng = np.random.default_rng(3)
    x = rng.integers(-(t0 * t1 // 2) + 1, t0 * t1 // 2, size=1000)
    r0 = (x + t0 // 2) % t0 - t0 // 2
    r1 = x % t1
    assert np.array_equal(crt.combine([r0, r1], [t0, t1]), x)


def test_combine_three_moduli_edges():
    ts = [7, 11, 13]
    M = 7 * 11 * 13
    x = np.array([-(M // 2), -1, 0, 1, M // 2])
    assert np.array_equal(crt.combine([x % t for t in ts], ts), x)


@pytest.mark.gpu
def test_two_plaintext_moduli_on_the_gpu():
    from paper_2406_06761_gb300 import wally as Wl
    dev = torch.device("cuda", 0)
    w = W.WORKLOADS["tiny"]
    t0 = O.prev_prime_1mod(1 << w.t_bits, 2 << w.log_n)
    t1 = O.prev_prime_1mod(t0, 2 << w.log_n)
    E = W.embeddings(1024, w.dim, 127, seed=31)          # |E q| up to 192 * 127^2, beyond t/2
    q = W.query_vectors(1, w.dim, 127, seed=31)
    exact = E.astype(np.int64) @ q[0].astype(np.int64)
    assert np.abs(exact).max() > t0 // 2
    res = []
    for t in (t0, t1):
        ctx = Wl.Context(w.log_n, w.num_q, w.q_bits, w.t_bits, w.dim, t=t)
        Wl.wally_load_clusters(ctx.ptr, np.array([1024], np.uint32), E)
        cr = W.client_randomness(1, ctx.N, ctx.q, ctx.P, seed=32)
        sec = torch.from_numpy(cr.secret).to(dev)
        keys = torch.empty((1, 2, ctx.L, 2, ctx.L + 1, ctx.N), dtype=torch.int64, device=dev)
        cts = torch.empty((1, 2, ctx.L, ctx.N), dtype=torch.int64, device=dev)
        Wl.wally_keygen(ctx.ptr, 1, sec, Wl.u64_tensor(cr.key_a, dev), torch.from_numpy(cr.key_e).to(dev), keys)
        Wl.wally_encrypt_query(ctx.ptr, 1, sec, torch.from_numpy(q).to(dev), Wl.u64_tensor(cr.enc_a, dev),
                               torch.from_numpy(cr.enc_e).to(dev), cts)
        out = torch.empty((1, 2, ctx.L, ctx.N), dtype=torch.int64, device=dev)
        Wl.wally_eval_batch(ctx.ptr, 1, torch.zeros(1, dtype=torch.int32, device=dev), cts, keys, None,
                            torch.zeros(1, dtype=torch.int64, device=dev), out)
        scores = torch.empty((1, ctx.N), dtype=torch.int64, device=dev)
        Wl.wally_decrypt_scores(ctx.ptr, 1, sec, None, out, scores)
        Wl.wally_sync(ctx.ptr)
        res.append(scores.cpu().numpy()[0, :1024])
        ctx.close()
    assert not np.array_equal(res[0], exact)             # one modulus alone wraps around
    assert np.array_equal(crt.combine(res, [t0, t1]), exact)
