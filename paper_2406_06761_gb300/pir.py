"""Keyword PIR for metadata (Sec. 4.2 "Reducing Communication in Metadata
Fetch"): host-side tables and client logic around the library's index PIR.

- The server places every (keyword, value) entry of a cluster in one of two
  cuckoo tables ("splitting cuckoo hash tables"): entry e may sit only at
  h1(e) in table 1 or at h2(e) in table 2, so the client runs one index PIR
  on each table.
- Each table is a d1 x d2 matrix of plaintexts, d2 about 0.41 sqrt(slots)
  ("uneven dimensions": d2 = sqrt(1/(gamma + 1)) sqrt(N') with gamma = 5).
- A slot's plaintext packs the keyword, the value length and the value, two
  bytes a coefficient; empty slots are zero (keyword 0 is reserved).
- The client sends, per table, a query ciphertext for the slot's row (and
  column) and one set of expansion keys (the same Galois elements N/2^a + 1
  serve both tables); the server answers with the slot's whole row
  (wally_pir_answer, MulPIR's first dimension) or with the slot alone
  (wally_pir_answer2, both dimensions, which also needs a relinearisation
  key); the client decrypts and keeps the entry whose keyword matches.

Every homomorphic step runs in libwally; this module only builds tables and
packs bytes.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK = (1 << 64) - 1
HEADER_BYTES = 10  # keyword (8) + value length (2)


def _mix(x: int) -> int:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014)."""
    x = (x + 0x9E3779B97F4A7C15) & _MASK
    x = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    x = ((x ^ (x >> 27)) * 0x94D049BB133111EB) & _MASK
    return x ^ (x >> 31)


def slot_of(keyword: int, table: int, seed: int, size: int) -> int:
    """h_table(keyword): the only slot of `table` (0 or 1) the entry may use."""
    return _mix(keyword ^ _mix((seed << 1) | table)) % size


def dims(slots: int, gamma: float = 5.0) -> tuple[int, int]:
    """(d1, d2) with d1 d2 >= slots and d2 = ceil(sqrt(1/(gamma+1)) sqrt(slots))."""
    d2 = max(1, math.ceil(math.sqrt(1.0 / (gamma + 1.0)) * math.sqrt(slots)))
    d1 = math.ceil(slots / d2)
    return d1, d2


def pack(keyword: int, value: bytes, n: int) -> np.ndarray:
    """One slot's plaintext: [keyword (8 B) | length (2 B) | value], two bytes
    a coefficient (little-endian), zero-padded to n coefficients."""
    raw = keyword.to_bytes(8, "little") + len(value).to_bytes(2, "little") + value
    if len(raw) > 2 * n:
        raise ValueError(f"value of {len(value)} bytes does not fit a plaintext of {n} coefficients")
    raw += b"\0" * (len(raw) & 1)
    out = np.zeros(n, np.uint64)
    out[:len(raw) // 2] = np.frombuffer(raw, dtype="<u2").astype(np.uint64)
    return out


def unpack(coeffs) -> tuple[int, bytes] | None:
    """(keyword, value) from a decrypted slot, or None for an empty slot."""
    c = np.asarray(coeffs, dtype=np.int64)
    if np.any(c < 0) or np.any(c > 0xFFFF):
        return None
    raw = c.astype("<u2").tobytes()
    kw = int.from_bytes(raw[:8], "little")
    if kw == 0:
        return None
    ln = int.from_bytes(raw[8:10], "little")
    if HEADER_BYTES + ln > len(raw):
        return None
    return kw, raw[HEADER_BYTES:HEADER_BYTES + ln]


@dataclasses.dataclass
class CuckooTables:
    seed: int
    sizes: tuple[int, int]
    slots: list            # two lists of (keyword, value) or None
    dims: tuple            # ((d1, d2), (d1, d2))

    def position(self, keyword: int, table: int) -> tuple[int, int]:
        """(row, column) of the keyword's slot in `table`."""
        s = slot_of(keyword, table, self.seed, self.sizes[table])
        return divmod(s, self.dims[table][1])

    def plaintexts(self, table: int, n: int) -> np.ndarray:
        """The table as a [d1][d2][n] plaintext matrix for wally_pir_load."""
        d1, d2 = self.dims[table]
        out = np.zeros((d1, d2, n), np.uint64)
        for s, e in enumerate(self.slots[table]):
            if e is not None:
                out[s // d2, s % d2] = pack(e[0], e[1], n)
        return out


def build(entries: dict[int, bytes], load: float = 2.2, max_kicks: int = 500, seed: int = 0,
          tries: int = 32) -> CuckooTables:
    """Cuckoo insertion into two tables of ceil(load * len / 2) slots each; a
    failed insertion restarts with the next seed.  Sec. 4.2 quotes (1 + u) N'
    slots with u about 0.5, but cuckoo insertion with two hash functions
    succeeds reliably only below half occupancy, so the default is
    load = 1 + u = 2.2 (each split table 1.1 N')."""
    if any(k <= 0 or k > _MASK for k in entries):
        raise ValueError("keywords must be in 1 .. 2^64 - 1")
    n = len(entries)
    milli = int(round(load * 1000))
    size = max(1, -(-milli * n // 2000))  # ceil(load n / 2) without floating error
    for attempt in range(tries):
        sd = seed + attempt
        tabs = [[None] * size, [None] * size]
        ok = True
        for kw, val in entries.items():
            cur, t = (kw, val), 0
            for _ in range(max_kicks):
                s = slot_of(cur[0], t, sd, size)
                cur, tabs[t][s] = tabs[t][s], cur
                if cur is None:
                    break
                t ^= 1
            else:
                ok = False
                break
        if ok:
            return CuckooTables(sd, (size, size), tabs, (dims(size), dims(size)))
    raise RuntimeError("cuckoo insertion failed; raise the load factor")


def lookup_plain(tables: CuckooTables, keyword: int) -> bytes | None:
    """The value of a keyword read directly from the tables (for checking)."""
    for t in (0, 1):
        e = tables.slots[t][slot_of(keyword, t, tables.seed, tables.sizes[t])]
        if e is not None and e[0] == keyword:
            return e[1]
    return None


def levels(d1: int) -> int:
    """Expansion levels of a table with d1 rows: ceil(log2 d1)."""
    return max(0, (d1 - 1).bit_length())


def galois_elements(n: int, levels: int) -> list[int]:
    """The substitution elements of the expansion levels: N/2^a + 1."""
    return [n // (1 << a) + 1 for a in range(levels)]


def query_plaintext(n: int, t: int, levels: int, row: int, col: int | None = None, d1: int = 0) -> np.ndarray:
    """The client's query plaintext: (2^levels)^-1 mod t at X^row, and for a
    two-dimensional query also at X^(d1 + col)."""
    m = np.zeros(n, np.uint64)
    inv = pow(1 << levels, -1, t)
    m[row] = inv
    if col is not None:
        m[d1 + col] = (int(m[d1 + col]) + inv) % t
    return m
