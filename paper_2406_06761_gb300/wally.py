"""Thin ctypes binding of libwally (include/wally.h).

Argument marshalling only: every call forwards torch tensors (device memory,
or host memory for the ``_host`` variant) as raw pointers to the C ABI, where
all of the computation runs in the library's CUDA kernels.  There is no CPU
fallback: importing this module on a machine without the built library, or
calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

WALLY_OK, WALLY_EINVAL, WALLY_ENOMEM, WALLY_ECUDA, WALLY_ETIMEOUT, WALLY_ESTATE = range(6)
MAX_LIMBS = 8
STORE_AUTO, STORE_NTT, STORE_COMPACT = 0, 1, 2


class WallyError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"wally error {code}: {msg}")
        self.code = code


class wally_params(ctypes.Structure):
    _fields_ = [
        ("log_n", ctypes.c_uint32), ("num_q", ctypes.c_uint32), ("q_bits", ctypes.c_uint32),
        ("t_bits", ctypes.c_uint32), ("dim", ctypes.c_uint32), ("device", ctypes.c_int32),
        ("q", ctypes.POINTER(ctypes.c_uint64)), ("p_special", ctypes.c_uint64), ("t", ctypes.c_uint64),
        ("max_wave", ctypes.c_uint32), ("store", ctypes.c_uint32), ("cache_chunks", ctypes.c_uint32),
        ("baby_steps", ctypes.c_uint32),
    ]


class wally_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32), ("log_n", ctypes.c_uint32), ("num_q", ctypes.c_uint32), ("dim", ctypes.c_uint32),
        ("d_pad", ctypes.c_uint32), ("g", ctypes.c_uint32), ("h", ctypes.c_uint32),
        ("num_clusters", ctypes.c_uint32), ("q", ctypes.c_uint64 * MAX_LIMBS),
        ("p_special", ctypes.c_uint64), ("t", ctypes.c_uint64), ("zeta_t", ctypes.c_uint64),
        ("k1", ctypes.c_uint64), ("kg", ctypes.c_uint64), ("ct_words", ctypes.c_uint64),
        ("keys_words", ctypes.c_uint64), ("total_chunks", ctypes.c_uint64), ("cluster_bytes", ctypes.c_uint64),
        ("max_wave", ctypes.c_uint32), ("drop_c0", ctypes.c_uint32), ("drop_c1", ctypes.c_uint32),
        ("compressed_bytes", ctypes.c_uint64), ("store", ctypes.c_uint32), ("cache_chunks", ctypes.c_uint32),
    ]


class wally_tuning(ctypes.Structure):
    _fields_ = [("max_wave", ctypes.c_uint32), ("lanes", ctypes.c_uint32), ("mac_ctas_per_sm", ctypes.c_uint32),
                ("ntt_ctas_per_sm", ctypes.c_uint32), ("ks_core", ctypes.c_uint32), ("mac_halves", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


AUTOTUNE_MAX = 16


class wally_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 16), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64

# name -> (restype, argtypes): the full C ABI of include/wally.h
SIGNATURES = {
    "wally_setup_params": (ctypes.c_int, [ctypes.POINTER(wally_params), ctypes.POINTER(_vp)]),
    "wally_destroy": (None, [_vp]),
    "wally_query_info": (ctypes.c_int, [_vp, ctypes.POINTER(wally_info)]),
    "wally_load_clusters": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp]),
    "wally_cluster_chunks": (ctypes.c_int, [_vp, _u32, ctypes.POINTER(_u32)]),
    "wally_export_cluster": (ctypes.c_int, [_vp, _u32, _vp, _vp]),
    "wally_eval_batch": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "wally_eval_batch_lane": (ctypes.c_int, [_vp, _u32, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "wally_eval_batch_host": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "wally_rotate": (ctypes.c_int, [_vp, _u32, _u64, _vp, _vp, _vp, _vp]),
    "wally_rotate_noalloc": (ctypes.c_int, [_vp, _u32, _u64, _vp, _vp, _vp, _vp]),
    "wally_sync": (ctypes.c_int, [_vp, _vp]),
    "wally_keygen": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    "wally_encrypt_query": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "wally_decrypt_scores": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    "wally_compress_responses": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp]),
    "wally_decrypt_compressed": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    "wally_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "wally_profile_read": (ctypes.c_int, [_vp, _vp, _u32, ctypes.POINTER(_u32)]),
    "wally_profile_waves": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, ctypes.POINTER(_u32)]),
    "wally_measure_pipe_rates": (ctypes.c_int, [ctypes.c_int32, _vp]),
    "wally_measure_int_peaks": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "wally_pir_load": (ctypes.c_int, [_vp, _u32, _u32, _vp, _vp]),
    "wally_pir_answer": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp]),
    "wally_keygen_galois": (ctypes.c_int, [_vp, _u32, _u32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "wally_pir_answer2": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    "wally_pir_derive_keys": (ctypes.c_int, [_vp, ctypes.c_int]),
    "wally_pir_key_levels": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(_u32), ctypes.POINTER(_u32)]),
    "wally_keygen_relin": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    "wally_encrypt_poly": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "wally_decrypt_poly": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp, _vp, _vp]),
    "wally_get_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(wally_tuning)]),
    "wally_set_tuning": (ctypes.c_int, [_vp, ctypes.POINTER(wally_tuning)]),
    "wally_autotune": (ctypes.c_int, [_vp, _vp, _u32, _u32, _u32, _vp, _vp, _vp, _vp, _vp, _vp,
                                      _vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_u32),
                                      ctypes.POINTER(_u32), _vp]),
    "wally_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libwally.so (optionally building it first).  Raises if absent."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"libwally.so is not built ({path}); run __graft_entry__.build()")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int) -> None:
    if rc != WALLY_OK:
        raise WallyError(rc, load().wally_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to libwally must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("this call takes device tensors")


def _u64_view(t: torch.Tensor) -> torch.Tensor:
    """uint64 residues are carried in int64 tensors (same bits)."""
    return t


# ------------------------------------------------------------------ same names as the C ABI

def wally_setup_params(log_n: int, num_q: int, q_bits: int, t_bits: int, dim: int, device: int = 0,
                       q=None, p_special: int = 0, t: int = 0, max_wave: int = 0, store: int = STORE_AUTO,
                       cache_chunks: int = 0, baby_steps: int = 0) -> int:
    lib = load()
    prm = wally_params(log_n, num_q, q_bits, t_bits, dim, device, None, p_special, t, max_wave, store, cache_chunks,
                       baby_steps)
    qarr = None
    if q is not None:
        qarr = (ctypes.c_uint64 * len(q))(*q)
        prm.q = ctypes.cast(qarr, ctypes.POINTER(ctypes.c_uint64))
    out = _vp()
    _check(lib.wally_setup_params(ctypes.byref(prm), ctypes.byref(out)))
    return out.value


def wally_destroy(ctx: int) -> None:
    load().wally_destroy(ctx)


def wally_query_info(ctx: int) -> wally_info:
    info = wally_info()
    _check(load().wally_query_info(ctx, ctypes.byref(info)))
    return info


def wally_load_clusters(ctx: int, sizes, embeddings, stream=None) -> None:
    """sizes: uint32 numpy array [K]; embeddings: int8 numpy array [sum sizes][dim] (host)."""
    import numpy as np
    sizes = np.ascontiguousarray(sizes, dtype=np.uint32)
    emb = np.ascontiguousarray(embeddings, dtype=np.int8)
    _check(load().wally_load_clusters(ctx, len(sizes), sizes.ctypes.data, emb.ctypes.data if emb.size else None,
                                      _stream(stream)))


def wally_cluster_chunks(ctx: int, cluster_id: int) -> int:
    m = _u32()
    _check(load().wally_cluster_chunks(ctx, cluster_id, ctypes.byref(m)))
    return m.value


def wally_export_cluster(ctx: int, cluster_id: int, out: torch.Tensor, stream=None) -> None:
    _require_cuda(out)
    _check(load().wally_export_cluster(ctx, cluster_id, _ptr(out), _stream(stream)))


def wally_eval_batch(ctx: int, n: int, cluster_ids, cts, galois_keys, input_index, out_offsets, out,
                     stream=None) -> None:
    _require_cuda(cluster_ids, cts, galois_keys, input_index, out_offsets, out)
    _check(load().wally_eval_batch(ctx, n, _ptr(cluster_ids), _ptr(cts), _ptr(galois_keys), _ptr(input_index),
                                   _ptr(out_offsets), _ptr(out), _stream(stream)))


def wally_eval_batch_lane(ctx: int, lane: int, n: int, cluster_ids, cts, galois_keys, input_index, out_offsets,
                          out, stream=None) -> None:
    _require_cuda(cluster_ids, cts, galois_keys, input_index, out_offsets, out)
    _check(load().wally_eval_batch_lane(ctx, lane, n, _ptr(cluster_ids), _ptr(cts), _ptr(galois_keys),
                                        _ptr(input_index), _ptr(out_offsets), _ptr(out), _stream(stream)))


def wally_eval_batch_host(ctx: int, n: int, cluster_ids, cts, galois_keys, input_index, out_offsets, out,
                          stream=None) -> None:
    """Host tensors (pinned for asynchronous copies); returns when out is filled."""
    for t in (cluster_ids, cts, galois_keys, input_index, out_offsets, out):
        if t is not None and t.is_cuda:
            raise ValueError("wally_eval_batch_host takes host tensors")
    _check(load().wally_eval_batch_host(ctx, n, _ptr(cluster_ids), _ptr(cts), _ptr(galois_keys),
                                        _ptr(input_index), _ptr(out_offsets), _ptr(out), _stream(stream)))


def wally_rotate(ctx: int, n: int, galois_elt: int, cts, keys, out, stream=None) -> None:
    _require_cuda(cts, keys, out)
    _check(load().wally_rotate(ctx, n, galois_elt, _ptr(cts), _ptr(keys), _ptr(out), _stream(stream)))


def wally_rotate_noalloc(ctx: int, n: int, galois_elt: int, cts, keys, out, stream=None) -> None:
    """wally_rotate without device allocation (fixed static scratch; small n)."""
    _require_cuda(cts, keys, out)
    _check(load().wally_rotate_noalloc(ctx, n, galois_elt, _ptr(cts), _ptr(keys), _ptr(out), _stream(stream)))


def wally_sync(ctx: int, stream=None) -> None:
    _check(load().wally_sync(ctx, _stream(stream)))


def wally_keygen(ctx: int, n: int, secret, key_a, key_e, galois_keys, stream=None) -> None:
    _require_cuda(secret, key_a, key_e, galois_keys)
    _check(load().wally_keygen(ctx, n, _ptr(secret), _ptr(key_a), _ptr(key_e), _ptr(galois_keys), _stream(stream)))


def wally_encrypt_query(ctx: int, n: int, secret, queries, enc_a, enc_e, cts, stream=None) -> None:
    _require_cuda(secret, queries, enc_a, enc_e, cts)
    _check(load().wally_encrypt_query(ctx, n, _ptr(secret), _ptr(queries), _ptr(enc_a), _ptr(enc_e), _ptr(cts),
                                      _stream(stream)))


def wally_decrypt_scores(ctx: int, n: int, secret, secret_index, cts, scores, stream=None) -> None:
    _require_cuda(secret, secret_index, cts, scores)
    _check(load().wally_decrypt_scores(ctx, n, _ptr(secret), _ptr(secret_index), _ptr(cts), _ptr(scores),
                                       _stream(stream)))


def wally_compress_responses(ctx: int, n: int, cts, out, stream=None) -> None:
    """out: uint8 device tensor [n][compressed_bytes]."""
    _require_cuda(cts, out)
    _check(load().wally_compress_responses(ctx, n, _ptr(cts), _ptr(out), _stream(stream)))


def wally_decrypt_compressed(ctx: int, n: int, secret, secret_index, packed, scores, stream=None) -> None:
    _require_cuda(secret, secret_index, packed, scores)
    _check(load().wally_decrypt_compressed(ctx, n, _ptr(secret), _ptr(secret_index), _ptr(packed), _ptr(scores),
                                           _stream(stream)))


def wally_profile_enable(ctx: int, enable: bool = True) -> None:
    _check(load().wally_profile_enable(ctx, 1 if enable else 0))


def wally_profile_read(ctx: int) -> dict:
    """{kernel kind: (launches, total milliseconds)} since profiling was enabled."""
    arr = (wally_kernel_time * 16)()
    cnt = _u32()
    _check(load().wally_profile_read(ctx, ctypes.cast(arr, _vp), 16, ctypes.byref(cnt)))
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(cnt.value)}


def wally_profile_waves(ctx: int, cap: int = 1 << 16):
    """Wave completions since profiling was enabled: (call, queries, done_ms)
    numpy arrays, one entry per wave in submission order."""
    import numpy as np
    call = np.zeros(cap, np.uint32)
    q = np.zeros(cap, np.uint32)
    ms = np.zeros(cap, np.float32)
    cnt = _u32()
    _check(load().wally_profile_waves(ctx, cap, call.ctypes.data, q.ctypes.data, ms.ctypes.data, ctypes.byref(cnt)))
    n = min(cap, cnt.value)
    return call[:n], q[:n], ms[:n]


def wally_measure_int_peaks(device: int = 0) -> dict:
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(load().wally_measure_int_peaks(device, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"modmul_per_s": a.value, "butterfly_per_s": b.value, "mac128_per_s": c.value}


def wally_measure_pipe_rates(device: int = 0) -> dict:
    """Issue rates of the 32-bit multiply instructions, the SM clock, and
    the NTT butterfly's multiplier ceiling (operations per second, Hz)."""
    arr = (ctypes.c_double * 5)()
    _check(load().wally_measure_pipe_rates(device, ctypes.cast(arr, _vp)))
    names = ("mad_lo_per_s", "mul_hi_per_s", "mad_wide_per_s", "sm_clock_hz", "bfly_ceiling_per_s")
    return dict(zip(names, (float(x) for x in arr)))


def wally_pir_load(ctx: int, table, stream=None) -> None:
    """table: uint64 numpy array [rows][cols][N] (host), coefficients in [0, t)."""
    import numpy as np
    table = np.ascontiguousarray(table, dtype=np.uint64)
    _check(load().wally_pir_load(ctx, table.shape[0], table.shape[1], table.ctypes.data, _stream(stream)))


def wally_pir_answer(ctx: int, n: int, queries, keys, out, stream=None) -> None:
    _require_cuda(queries, keys, out)
    _check(load().wally_pir_answer(ctx, n, _ptr(queries), _ptr(keys), _ptr(out), _stream(stream)))


def wally_pir_answer2(ctx: int, n: int, queries, keys, relin_keys, out, stream=None) -> None:
    _require_cuda(queries, keys, relin_keys, out)
    _check(load().wally_pir_answer2(ctx, n, _ptr(queries), _ptr(keys), _ptr(relin_keys), _ptr(out),
                                    _stream(stream)))


def wally_pir_derive_keys(ctx: int, enable: bool) -> None:
    _check(load().wally_pir_derive_keys(ctx, 1 if enable else 0))


def wally_pir_key_levels(ctx: int, two_dims: bool = False) -> tuple[int, int]:
    """(first level, number of levels) whose keys the client sends."""
    f, c = _u32(), _u32()
    _check(load().wally_pir_key_levels(ctx, 1 if two_dims else 0, ctypes.byref(f), ctypes.byref(c)))
    return f.value, c.value


def wally_keygen_relin(ctx: int, n: int, secret, key_a, key_e, keys, stream=None) -> None:
    _require_cuda(secret, key_a, key_e, keys)
    _check(load().wally_keygen_relin(ctx, n, _ptr(secret), _ptr(key_a), _ptr(key_e), _ptr(keys), _stream(stream)))


def wally_keygen_galois(ctx: int, n: int, galois, secret, key_a, key_e, keys, stream=None) -> None:
    _require_cuda(secret, key_a, key_e, keys)
    g = (ctypes.c_uint64 * len(galois))(*[int(x) for x in galois])
    _check(load().wally_keygen_galois(ctx, n, len(galois), ctypes.cast(g, _vp), _ptr(secret), _ptr(key_a),
                                      _ptr(key_e), _ptr(keys), _stream(stream)))


def wally_encrypt_poly(ctx: int, n: int, secret, m, enc_a, enc_e, cts, stream=None) -> None:
    _require_cuda(secret, m, enc_a, enc_e, cts)
    _check(load().wally_encrypt_poly(ctx, n, _ptr(secret), _ptr(m), _ptr(enc_a), _ptr(enc_e), _ptr(cts),
                                     _stream(stream)))


def wally_decrypt_poly(ctx: int, n: int, secret, secret_index, cts, coeffs, stream=None) -> None:
    _require_cuda(secret, secret_index, cts, coeffs)
    _check(load().wally_decrypt_poly(ctx, n, _ptr(secret), _ptr(secret_index), _ptr(cts), _ptr(coeffs),
                                     _stream(stream)))


def wally_get_tuning(ctx: int) -> wally_tuning:
    t = wally_tuning()
    _check(load().wally_get_tuning(ctx, ctypes.byref(t)))
    return t


def wally_set_tuning(ctx: int, max_wave: int, lanes: int = 2, mac_ctas_per_sm: int = 3,
                     ntt_ctas_per_sm: int = 0, ks_core: int = 0, mac_halves: int = 0) -> None:
    t = wally_tuning(max_wave, lanes, mac_ctas_per_sm, ntt_ctas_per_sm, ks_core, mac_halves)
    _check(load().wally_set_tuning(ctx, ctypes.byref(t)))


def wally_autotune(ctx: int, n: int, cluster_ids, cts, galois_keys, input_index, out_offsets, out,
                   candidates=None, reps: int = 1, stream=None) -> tuple[int, list]:
    """Time the sample batch under each candidate shape (dicts or
    wally_tuning; None = the library's staged search), keep the fastest.
    Returns (index of the best, [(shape dict, ms per query or -1), ...]) in
    the order the shapes were timed."""
    _require_cuda(cluster_ids, cts, galois_keys, input_index, out_offsets, out)
    if candidates is None:
        arr, nc, cap = None, 0, AUTOTUNE_MAX
    else:
        cs = [c if isinstance(c, wally_tuning) else wally_tuning(**c) for c in candidates]
        arr = (wally_tuning * len(cs))(*cs)
        nc = cap = len(cs)
    tried = (wally_tuning * cap)()
    ms = (ctypes.c_double * cap)()
    count, best = _u32(), _u32()
    _check(load().wally_autotune(ctx, ctypes.cast(arr, _vp) if arr is not None else None, nc, reps, n,
                                 _ptr(cluster_ids), _ptr(cts), _ptr(galois_keys), _ptr(input_index),
                                 _ptr(out_offsets), _ptr(out), ctypes.cast(tried, _vp), ms, ctypes.byref(count),
                                 ctypes.byref(best), _stream(stream)))
    return best.value, [(tried[i].as_dict(), ms[i]) for i in range(min(count.value, cap))]


def wally_last_error() -> str:
    return load().wally_last_error().decode()


# ------------------------------------------------------------------ convenience

def u64_tensor(a, device) -> torch.Tensor:
    """numpy uint64 array -> int64 tensor with the same bits, on `device`."""
    import numpy as np
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def to_u64_numpy(t: torch.Tensor):
    import numpy as np
    return t.detach().cpu().numpy().view(np.uint64)


class Context:
    """Owns one wally_ctx; a convenience wrapper around the functions above."""

    def __init__(self, log_n, num_q, q_bits, t_bits, dim, device=0, max_wave=0, **kw):
        self.ptr = wally_setup_params(log_n, num_q, q_bits, t_bits, dim, device=device, max_wave=max_wave, **kw)
        self.info = wally_query_info(self.ptr)
        self.device = torch.device("cuda", device)

    @property
    def N(self):
        return self.info.n

    @property
    def L(self):
        return self.info.num_q

    @property
    def q(self):
        return [int(self.info.q[i]) for i in range(self.L)]

    @property
    def P(self):
        return int(self.info.p_special)

    def refresh(self):
        self.info = wally_query_info(self.ptr)

    def close(self):
        if self.ptr:
            wally_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
