"""Plaintext CRT on the client (Sec. 7 "Parameters Selection": to raise the
precision of the scores beyond what one plaintext modulus holds without
wrap-around, the query is evaluated under several plaintext moduli t_k and
the decrypted scores are recombined by the Chinese remainder theorem).

The server side needs nothing new: one context per t_k (``wally_params.t``),
the same clusters loaded in each, the client's query encrypted under each.
This module recombines the centred residues the client decrypts.
"""
from __future__ import annotations

import numpy as np


def combine(residues, moduli) -> np.ndarray:
    """Scores x with x = residues[k] (mod moduli[k]) for every k, centred in
    (-M/2, M/2] with M the product of the (pairwise coprime) moduli.
    residues: int64 arrays of one shape (any representatives)."""
    M = 1
    for t in moduli:
        M *= int(t)
    acc = np.zeros(np.shape(residues[0]), dtype=object)
    for r, t in zip(residues, moduli):
        t = int(t)
        Mt = M // t
        coef = Mt * pow(Mt % t, -1, t)  # = 1 mod t, 0 mod the others
        acc = acc + (np.asarray(r, dtype=np.int64).astype(object) % t) * coef
    acc = acc % M
    acc = np.where(acc > M // 2, acc - M, acc)
    return acc.astype(np.int64)
