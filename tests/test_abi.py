"""The C ABI library builds, loads, and exports every entry point that
include/wally.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

from paper_2406_06761_gb300 import build as B
from paper_2406_06761_gb300 import wally as W

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "wally.h")


def declared_entry_points():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wally_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("wally_setup_params", "wally_load_clusters", "wally_eval_batch", "wally_keygen",
                 "wally_encrypt_query", "wally_decrypt_scores", "wally_sync", "wally_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(B.build())
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    names = declared_entry_points()
    assert sorted(W.SIGNATURES) == names
    for name in names:
        assert callable(getattr(W, name))


def test_oracle_builds_and_shares_nothing_with_the_library():
    import oracle
    path = oracle.build()
    assert os.path.exists(path)
    src = open(os.path.join(os.path.dirname(oracle.__file__), "wally_oracle.c")).read()
    assert "wally.h" not in src and "common.cuh" not in src
    csrc = os.path.join(os.path.dirname(B.__file__), "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read()
