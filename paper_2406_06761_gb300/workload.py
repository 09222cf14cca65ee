"""Seeded synthetic inputs shaped like Wally's workloads (arXiv 2406.06761).

This module holds no arithmetic of the method.  It only draws random numbers
(and states workload shapes) so that the CUDA library and the CPU oracle can be
fed byte-identical inputs: embeddings, query vectors, cluster sizes, cluster
ids, negative-binomial fake-query counts, and the random numbers the client
draws for key generation and encryption (ternary secrets, uniform residues,
small errors).  Every draw comes from its own stream, keyed by
(seed, purpose, index), so that any single item can be regenerated alone.

Stand-ins: the paper's MS MARCO passages embedded by TAS-B and reduced to
192 dimensions by PCA (Sec. 7 "Embedding and Clustering", "Dataset") are not
available; embeddings here are i.i.d. uniform integers in [-B, B], clusters
have log-normal sizes, and real queries pick clusters in proportion to size.
"""
from __future__ import annotations

import dataclasses
import zlib

import numpy as np

ERROR_SIGMA = 3.2  # Sec. 7 "Parameters Selection": error standard deviation 3.2
ERROR_TAIL = 19    # discrete Gaussian truncated at |e| <= 19 (about 6 sigma)


def stream(seed: int, purpose: str, index: int = 0) -> np.random.Generator:
    """Independent generator for (seed, purpose, index)."""
    key = zlib.crc32(purpose.encode())
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, key, index])))


# ------------------------------------------------------------------ configs

@dataclasses.dataclass(frozen=True)
class Workload:
    """One workload shape: ring/modulus sizes and the database/query mix."""
    name: str
    log_n: int
    num_q: int
    q_bits: int
    t_bits: int
    dim: int
    entry_bound: int
    num_clusters: int
    size_mu: float           # log-normal cluster sizes: log-mean
    size_sigma: float
    size_cap: int | None     # cap per cluster (None: none)
    total_embeddings: int | None  # rescale sizes to this total (None: keep the draws)
    real_queries: int
    nb_r: float = 0.5        # per-client fake-query count ~ NB(r, p)
    nb_p: float = 0.9
    arrival_qps: float | None = None  # serving: Poisson arrival rate
    window_ms: float | None = None    # serving: per-cluster grouping window


WORKLOADS = {
    "tiny": Workload("tiny", 12, 2, 36, 17, 192, 15, 1, float(np.log(1024)), 0.0, None, 1024, 1, nb_r=0.0),
    "batched": Workload("batched", 13, 3, 50, 20, 192, 15, 64, float(np.log(2000)), 0.6, 8192, None, 1000),
    "serving": Workload("serving", 13, 3, 50, 20, 192, 15, 1800, float(np.log(1700)), 0.5, None, 3_200_000, 0,
                        arrival_qps=50_000.0, window_ms=10.0),
    "full_scale": Workload("full_scale", 13, 3, 50, 20, 192, 15, 1800, float(np.log(1700)), 0.5, None,
                           3_200_000, 500_000),
    "wide": Workload("wide", 14, 6, 50, 22, 768, 7, 1000, float(np.log(1000)), 0.7, None, 1_000_000, 100_000),
}


def cluster_sizes(w: Workload, seed: int = 0) -> np.ndarray:
    """Log-normal cluster sizes, optionally capped, optionally rescaled to the
    stated total by largest-remainder rounding with a minimum of one."""
    rng = stream(seed, "cluster_sizes")
    raw = rng.lognormal(w.size_mu, w.size_sigma, w.num_clusters)
    if w.total_embeddings is not None:
        scaled = raw / raw.sum() * w.total_embeddings
        base = np.maximum(np.floor(scaled).astype(np.int64), 1)
        short = w.total_embeddings - int(base.sum())
        if short > 0:
            order = np.argsort(-(scaled - np.floor(scaled)), kind="stable")
            base[order[:short]] += 1
        elif short < 0:
            order = np.argsort(-base, kind="stable")
            for i in range(-short):
                base[order[i % len(order)]] -= 1
        sizes = base
    else:
        sizes = np.maximum(np.rint(raw).astype(np.int64), 1)
    if w.size_cap is not None:
        sizes = np.minimum(sizes, w.size_cap)
    return sizes


def embeddings(total: int, dim: int, bound: int, seed: int = 0, index: int = 0) -> np.ndarray:
    """int8 [total][dim], uniform in [-bound, bound] (grouped by cluster in id order)."""
    rng = stream(seed, "embeddings", index)
    return rng.integers(-bound, bound + 1, size=(total, dim), dtype=np.int8)


def query_vectors(n: int, dim: int, bound: int, seed: int = 0, index: int = 0) -> np.ndarray:
    rng = stream(seed, "queries", index)
    return rng.integers(-bound, bound + 1, size=(n, dim), dtype=np.int8)


def real_cluster_ids(n: int, sizes: np.ndarray, seed: int = 0) -> np.ndarray:
    """Cluster of each real query, drawn with probability proportional to size."""
    rng = stream(seed, "real_ids")
    p = np.asarray(sizes, dtype=np.float64)
    return rng.choice(len(p), size=n, p=p / p.sum()).astype(np.uint32)


def fake_counts(n_clients: int, r: float, p: float, seed: int = 0) -> np.ndarray:
    """Fake queries per client, NB(r, p) in numpy's convention (failures before
    r successes of probability p; mean r(1-p)/p)."""
    if r <= 0 or n_clients == 0:
        return np.zeros(n_clients, dtype=np.int64)
    rng = stream(seed, "fake_counts")
    return rng.negative_binomial(r, p, size=n_clients)


def fake_cluster_ids(n: int, num_clusters: int, seed: int = 0) -> np.ndarray:
    rng = stream(seed, "fake_ids")
    return rng.integers(0, num_clusters, size=n, dtype=np.int64).astype(np.uint32)


def query_mix(w: Workload, sizes: np.ndarray, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(cluster ids, is_real) for the real queries followed by every client's
    fakes, then shuffled (Alg. "Client Query Generation" permutes the list)."""
    real = real_cluster_ids(w.real_queries, sizes, seed)
    nf = int(fake_counts(w.real_queries, w.nb_r, w.nb_p, seed).sum())
    fake = fake_cluster_ids(nf, len(sizes), seed)
    ids = np.concatenate([real, fake])
    is_real = np.concatenate([np.ones(len(real), bool), np.zeros(nf, bool)])
    perm = stream(seed, "mix_perm").permutation(len(ids))
    return ids[perm], is_real[perm]


# ------------------------------------------------------------------ client randomness

def ternary(n: int, N: int, seed: int = 0, purpose: str = "secret") -> np.ndarray:
    """Secret keys: int8 [n][N] uniform over {-1, 0, 1}."""
    rng = stream(seed, purpose)
    return rng.integers(-1, 2, size=(n, N), dtype=np.int8)


def _gauss_table() -> tuple[np.ndarray, np.ndarray]:
    xs = np.arange(-ERROR_TAIL, ERROR_TAIL + 1)
    w = np.exp(-(xs.astype(np.float64) ** 2) / (2 * ERROR_SIGMA ** 2))
    return xs, w / w.sum()


def errors(shape, seed: int = 0, purpose: str = "error") -> np.ndarray:
    """int8 errors from the discrete Gaussian of width sigma = 3.2, |e| <= 19."""
    rng = stream(seed, purpose)
    xs, p = _gauss_table()
    return rng.choice(xs, size=shape, p=p).astype(np.int8)


def uniform_residues(prefix_shape, moduli, N: int, seed: int = 0, purpose: str = "uniform") -> np.ndarray:
    """uint64 [*prefix_shape][len(moduli)][N]: row j uniform in [0, moduli[j])."""
    rng = stream(seed, purpose)
    prefix = tuple(prefix_shape)
    out = np.empty(prefix + (len(moduli), N), dtype=np.uint64)
    for j, m in enumerate(moduli):
        out[..., j, :] = rng.integers(0, int(m), size=prefix + (N,), dtype=np.uint64)
    return out


@dataclasses.dataclass
class ClientRandomness:
    """Everything a batch of clients draws: secrets, key and encryption randomness."""
    secret: np.ndarray      # int8 [n][N]
    key_a: np.ndarray       # uint64 [n][2 keys][L digits][L+1 moduli][N]
    key_e: np.ndarray       # int8 [n][2][L][N]
    enc_a: np.ndarray       # uint64 [n][L][N]
    enc_e: np.ndarray       # int8 [n][N]


def client_randomness(n: int, N: int, q: list[int], P: int, seed: int = 0, index: int = 0) -> ClientRandomness:
    L = len(q)
    tag = f"clients{index}"
    return ClientRandomness(
        secret=ternary(n, N, seed, tag + "/s"),
        key_a=uniform_residues((n, 2, L), list(q) + [P], N, seed, tag + "/ka"),
        key_e=errors((n, 2, L, N), seed, tag + "/ke"),
        enc_a=uniform_residues((n,), list(q), N, seed, tag + "/ea"),
        enc_e=errors((n, N), seed, tag + "/ee"),
    )


@dataclasses.dataclass
class PirClientRandomness:
    """What a PIR client draws: a secret, one substitution key per expansion
    level (uniform a, small errors), and the query encryption's a and e."""
    secret: np.ndarray   # int8 [n][N]
    key_a: np.ndarray    # uint64 [n][levels][L][L+1][N]
    key_e: np.ndarray    # int8 [n][levels][L][N]
    enc_a: np.ndarray    # uint64 [n][L][N]
    enc_e: np.ndarray    # int8 [n][N]


def pir_client_randomness(n: int, levels: int, N: int, q: list[int], P: int, seed: int = 0,
                          index: int = 0) -> PirClientRandomness:
    L = len(q)
    tag = f"pir{index}"
    return PirClientRandomness(
        secret=ternary(n, N, seed, tag + "/s"),
        key_a=uniform_residues((n, levels, L), list(q) + [P], N, seed, tag + "/ka"),
        key_e=errors((n, levels, L, N), seed, tag + "/ke"),
        enc_a=uniform_residues((n,), list(q), N, seed, tag + "/ea"),
        enc_e=errors((n, N), seed, tag + "/ee"),
    )


def pir_plaintexts(rows: int, cols: int, N: int, t: int, seed: int = 0) -> np.ndarray:
    """A PIR table of uniform plaintext coefficients in [0, t): [rows][cols][N]."""
    return stream(seed, "pir_table").integers(0, t, size=(rows, cols, N), dtype=np.uint64)
