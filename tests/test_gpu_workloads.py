"""GPU parity at the workloads' full sizes, in the launch configuration the
benchmark uses (device-resident client submissions, waves of max_wave
queries, device-side grouping by cluster): sampled outputs bit for bit
against the oracle, and every output checked by decryption against the
plain integer dot products (a property that holds at any size)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2406_06761_gb300 import harness as H
from paper_2406_06761_gb300 import wally as Wl

pytestmark = pytest.mark.gpu


def _oracle_check(wl, prm, qi, got):
    """Recompute query qi with the oracle from the randomness its client drew."""
    e = int(wl.input_index[qi])
    c = int(wl.ids[qi])
    cr = wl.entry_randomness(e)
    keys = O.keygen_pair(prm, cr.secret, cr.key_a, cr.key_e)
    ct = O.encrypt_query(prm, cr.secret, wl.entry_query(e), cr.enc_a, cr.enc_e)
    E = wl.embeddings[wl.row0[c]:wl.row0[c] + wl.sizes[c]]
    m, pt = O.encode_cluster(prm, E)
    ref = O.eval_query(prm, m, pt, ct, keys)
    assert np.array_equal(got, ref), qi


def _decrypt_all(wl, out, offs):
    """GPU-decrypt every output and compare with E q (fakes: zeros)."""
    N = wl.N
    m_of = wl.chunks[wl.ids]
    sec_idx = []
    ct_rows = []
    for qi in range(wl.n):
        for k in range(m_of[qi]):
            sec_idx.append(int(wl.input_index[qi]))
            ct_rows.append(int(offs[qi]) + k)
    # client secrets, regenerated per randomness chunk
    secrets = wl.secrets()
    bad = 0
    step = 512
    for a in range(0, len(ct_rows), step):
        rows = ct_rows[a:a + step]
        scores = torch.empty((len(rows), N), dtype=torch.int64, device=wl.dev)
        Wl.wally_decrypt_scores(wl.ctx.ptr, len(rows), torch.from_numpy(secrets).to(wl.dev),
                                torch.tensor(sec_idx[a:a + step], dtype=torch.int32, device=wl.dev),
                                out[torch.tensor(rows, device=wl.dev)].contiguous(), scores)
        sc = scores.cpu().numpy()
        for j, r in enumerate(rows):
            qi = int(np.searchsorted(offs, r, side="right") - 1)
            k = r - int(offs[qi])
            c = int(wl.ids[qi])
            expect = wl.expected_scores(c, wl.entry_query(int(wl.input_index[qi])))
            seg = expect[k * N:(k + 1) * N]
            if not (np.array_equal(sc[j, :len(seg)], seg) and np.all(sc[j, len(seg):] == 0)):
                bad += 1
    return bad


def test_batched_workload_full_size():
    """64 clusters (log-normal sizes), 1,000 real queries + NB(0.5, 0.9)
    fakes per client, N = 8192, three 50-bit limbs: one call."""
    wl = H.DeviceWorkload("batched", max_wave=512)
    prm = O.params(wl.w.log_n, wl.w.num_q, wl.w.q_bits, wl.w.t_bits, wl.w.dim)
    ids, idx, offs_d, chunks, offs = wl.device_batch(0, wl.n)
    out = wl.alloc_out(chunks)
    wl.eval((ids, idx, offs_d, chunks, offs), out)
    Wl.wally_sync(wl.ctx.ptr)
    assert _decrypt_all(wl, out, offs) == 0
    got = Wl.to_u64_numpy(out)
    # sampled bit-exact checks: a fake, the largest cluster, the first and last
    big = int(np.argmax(wl.sizes))
    picks = {0, wl.n - 1, int(np.flatnonzero(wl.ids == big)[0])}
    if (~wl.is_real).any():
        picks.add(int(np.flatnonzero(~wl.is_real)[0]))
    for qi in sorted(picks):
        m = int(wl.chunks[wl.ids[qi]])
        _oracle_check(wl, prm, qi, got[offs[qi]:offs[qi] + m])
    wl.close()
