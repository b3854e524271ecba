"""CPU oracle of the VaultxGPU plotting path: Python side.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline leg and ``--impl reference``) may import this
module.  The product library never loads it; it shares no code with the CUDA
path and never imports it.

The arithmetic lives in ``vx_oracle.c`` (plain C, compiled with gcc by
:func:`build`).  This module only marshals numpy arrays in and out and adds
a few plain-numpy views (key64, bucket) used by the tests' invariants.

Paper sections followed: Sec. II-B (hash -> sort -> match stages), Sec. III-A
and III-B (Table 1 in 2^24 buckets by hash prefix, pairwise match against an
expected-distance threshold, Table 2).  Readings R1..R11 fix what the paper
leaves unstated; see the header of vx_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vx_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

REC_BYTES = 12     # {LE32 nonce, hash[0..7]}            (R4)
T2_BYTES = 16      # {LE32 a, LE32 b, hash2[0..7]}       (R10)
BUCKET_BITS = 24   # 2^24 logical buckets for every K    (R5)

_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile vx_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            L.orc_round.argtypes = [u32p, u32p]
            L.orc_iv.argtypes = [u32p]
            L.orc_compress.argtypes = [u32p, u32p, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, u32p]
            L.orc_keyed_hash.argtypes = [u8p, u8p, ctypes.c_size_t, u8p, ctypes.c_size_t]
            L.orc_table1_unsorted.argtypes = [ctypes.c_int, u8p, u8p]
            L.orc_hash_range_mt.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, u8p,
                                            ctypes.c_int]
            L.orc_sort_table1.argtypes = [u8p, ctypes.c_uint64]
            L.orc_table1.argtypes = [ctypes.c_int, u8p, u8p]
            L.orc_bucket_offsets.argtypes = [u8p, ctypes.c_uint64, u64p]
            L.orc_default_distance.argtypes = [ctypes.c_int]
            L.orc_default_distance.restype = ctypes.c_uint64
            L.orc_match.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint64, u8p,
                                    ctypes.c_uint64]
            L.orc_match.restype = ctypes.c_int64
            L.orc_match_bruteforce.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, u32p,
                                               ctypes.c_uint64]
            L.orc_match_bruteforce.restype = ctypes.c_int64
            L.orc_match_global.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint64, u8p,
                                           ctypes.c_uint64]
            L.orc_match_global.restype = ctypes.c_int64
            L.orc_match_global_bruteforce.argtypes = [u8p, ctypes.c_uint64, ctypes.c_uint64, u32p,
                                                      ctypes.c_uint64]
            L.orc_match_global_bruteforce.restype = ctypes.c_int64
            L.orc_pair_hash_mt.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_size_t, u8p,
                                           ctypes.c_int]
            L.orc_table1_mt.argtypes = [ctypes.c_int, u8p, u8p, u8p, ctypes.c_int]
            L.orc_match_mt.argtypes = [u8p, u8p, ctypes.c_uint64, ctypes.c_uint64, u8p, ctypes.c_int]
            L.orc_match_mt.restype = ctypes.c_int64
            _lib = L
    return _lib


def _p(a: np.ndarray, ctype):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _key_arr(key: bytes) -> np.ndarray:
    if len(key) != 32:
        raise ValueError("plot key must be 32 bytes")
    return np.frombuffer(bytes(key), dtype=np.uint8).copy()


# ---------------------------------------------------------------- BLAKE3 --

def round_fn(v: np.ndarray, m: np.ndarray) -> np.ndarray:
    """One G-round on a 16-word state (columns, then diagonals)."""
    v = np.ascontiguousarray(v, dtype=np.uint32).copy()
    m = np.ascontiguousarray(m, dtype=np.uint32)
    lib().orc_round(_p(v, ctypes.c_uint32), _p(m, ctypes.c_uint32))
    return v


def iv() -> np.ndarray:
    out = np.zeros(8, dtype=np.uint32)
    lib().orc_iv(_p(out, ctypes.c_uint32))
    return out


def compress(cv, block, counter: int, block_len: int, flags: int) -> np.ndarray:
    cv = np.ascontiguousarray(cv, dtype=np.uint32)
    block = np.ascontiguousarray(block, dtype=np.uint32)
    out = np.zeros(16, dtype=np.uint32)
    lib().orc_compress(_p(cv, ctypes.c_uint32), _p(block, ctypes.c_uint32), counter,
                       block_len, flags, _p(out, ctypes.c_uint32))
    return out


def keyed_hash(key: bytes, msg: bytes, out_len: int = 32) -> bytes:
    """BLAKE3 keyed_hash of a message of at most 64 bytes."""
    k = _key_arr(key)
    m = np.frombuffer(bytes(msg) + b"\0", dtype=np.uint8).copy()
    out = np.zeros(out_len, dtype=np.uint8)
    rc = lib().orc_keyed_hash(_p(k, ctypes.c_uint8), _p(m, ctypes.c_uint8), len(msg),
                              _p(out, ctypes.c_uint8), out_len)
    if rc != 0:
        raise ValueError("message longer than one block or output longer than 32 bytes")
    return out.tobytes()


# --------------------------------------------------------------- Table 1 --

def table1_unsorted(K: int, key: bytes) -> np.ndarray:
    """Records in nonce order, shape (2^K, 12) uint8."""
    n = 1 << K
    out = np.zeros((n, REC_BYTES), dtype=np.uint8)
    rc = lib().orc_table1_unsorted(K, _p(_key_arr(key), ctypes.c_uint8), _p(out, ctypes.c_uint8))
    if rc:
        raise ValueError("bad K")
    return out


def hash_range(key: bytes, lo: int, hi: int, threads: int = 1) -> np.ndarray:
    """Records of nonces lo..hi-1 (nonce order), hashed on `threads` threads."""
    out = np.zeros((hi - lo, REC_BYTES), dtype=np.uint8)
    lib().orc_hash_range_mt(_p(_key_arr(key), ctypes.c_uint8), lo, hi,
                            _p(out, ctypes.c_uint8), threads)
    return out


def sort_table1(recs: np.ndarray) -> np.ndarray:
    out = np.ascontiguousarray(recs, dtype=np.uint8).copy()
    lib().orc_sort_table1(_p(out, ctypes.c_uint8), out.shape[0])
    return out


def table1(K: int, key: bytes) -> np.ndarray:
    """The sorted Table 1, shape (2^K, 12) uint8."""
    n = 1 << K
    out = np.zeros((n, REC_BYTES), dtype=np.uint8)
    rc = lib().orc_table1(K, _p(_key_arr(key), ctypes.c_uint8), _p(out, ctypes.c_uint8))
    if rc:
        raise ValueError("bad K")
    return out


def bucket_offsets(t1: np.ndarray) -> np.ndarray:
    """offsets[b] = number of records with logical bucket < b, b = 0..2^24."""
    t1 = np.ascontiguousarray(t1, dtype=np.uint8)
    out = np.zeros((1 << BUCKET_BITS) + 1, dtype=np.uint64)
    lib().orc_bucket_offsets(_p(t1, ctypes.c_uint8), t1.shape[0], _p(out, ctypes.c_uint64))
    return out


# --------------------------------------------------------------- Table 2 --

def default_distance(K: int) -> int:
    return int(lib().orc_default_distance(K))


def match_count(key: bytes, t1: np.ndarray, D: int) -> int:
    t1 = np.ascontiguousarray(t1, dtype=np.uint8)
    return int(lib().orc_match(_p(_key_arr(key), ctypes.c_uint8), _p(t1, ctypes.c_uint8),
                               t1.shape[0], D, None, 0))


def match(key: bytes, t1: np.ndarray, D: int) -> np.ndarray:
    """Table 2, shape (pairs, 16) uint8, in bucket / i / j order."""
    t1 = np.ascontiguousarray(t1, dtype=np.uint8)
    n = match_count(key, t1, D)
    out = np.zeros((n, T2_BYTES), dtype=np.uint8)
    got = lib().orc_match(_p(_key_arr(key), ctypes.c_uint8), _p(t1, ctypes.c_uint8),
                          t1.shape[0], D, _p(out, ctypes.c_uint8), n)
    assert got == n
    return out


def pair_hash(key: bytes, recs: np.ndarray, threads: int = 1) -> np.ndarray:
    """hash2 (R10) of every row of recs (rows of 8 or more bytes: LE32 a,
    LE32 b, ...), shape (rows, 8) uint8, hashed on `threads` threads."""
    recs = np.ascontiguousarray(recs, dtype=np.uint8)
    if recs.ndim != 2 or recs.shape[1] < 8:
        raise ValueError("pair rows must hold at least 8 bytes")
    out = np.zeros((recs.shape[0], 8), dtype=np.uint8)
    lib().orc_pair_hash_mt(_p(_key_arr(key), ctypes.c_uint8), _p(recs, ctypes.c_uint8),
                           recs.shape[0], recs.shape[1], _p(out, ctypes.c_uint8), threads)
    return out


def table1_allcores(K: int, key: bytes, threads: int) -> np.ndarray:
    """The sorted Table 1 with every step on `threads` threads: hashing, a
    grouping pass by the top key byte, and qsort of each group."""
    n = 1 << K
    out = np.empty((n, REC_BYTES), dtype=np.uint8)
    scratch = np.empty((n, REC_BYTES), dtype=np.uint8)
    rc = lib().orc_table1_mt(K, _p(_key_arr(key), ctypes.c_uint8), _p(out, ctypes.c_uint8),
                             _p(scratch, ctypes.c_uint8), threads)
    if rc:
        raise ValueError("bad K")
    return out


def match_allcores(key: bytes, t1: np.ndarray, D: int, threads: int) -> np.ndarray:
    """Table 2 of :func:`match`, Table 1 cut into runs of whole buckets, one
    per thread."""
    t1 = np.ascontiguousarray(t1, dtype=np.uint8)
    L = lib()
    kp, tp = _p(_key_arr(key), ctypes.c_uint8), _p(t1, ctypes.c_uint8)
    n = int(L.orc_match_mt(kp, tp, t1.shape[0], D, None, threads))
    out = np.empty((n, T2_BYTES), dtype=np.uint8)
    got = L.orc_match_mt(kp, tp, t1.shape[0], D, _p(out, ctypes.c_uint8), threads)
    assert got == n
    return out


def plot_allcores(K: int, key: bytes, threads: int, D: int | None = None):
    """(Table 1, Table 2) of :func:`plot` with every stage on `threads`
    threads (the all-core CPU baseline)."""
    t1 = table1_allcores(K, key, threads)
    t2 = match_allcores(key, t1, default_distance(K) if D is None else D, threads)
    return t1, t2


def match_bruteforce(recs_unsorted: np.ndarray, D: int) -> np.ndarray:
    """All matching nonce pairs (a, b) by an O(n^2) scan, shape (pairs, 2) uint32."""
    recs = np.ascontiguousarray(recs_unsorted, dtype=np.uint8)
    L = lib()
    n = int(L.orc_match_bruteforce(_p(recs, ctypes.c_uint8), recs.shape[0], D, None, 0))
    out = np.zeros((n, 2), dtype=np.uint32)
    L.orc_match_bruteforce(_p(recs, ctypes.c_uint8), recs.shape[0], D,
                           _p(out, ctypes.c_uint32), n)
    return out


def match_global(key: bytes, t1: np.ndarray, D: int) -> np.ndarray:
    """Table 2 of the cross-bucket variant: every pair i < j of the whole
    Table-1 order with key64_j - key64_i < D, in i / j order."""
    t1 = np.ascontiguousarray(t1, dtype=np.uint8)
    L = lib()
    kp, tp = _p(_key_arr(key), ctypes.c_uint8), _p(t1, ctypes.c_uint8)
    n = int(L.orc_match_global(kp, tp, t1.shape[0], D, None, 0))
    out = np.zeros((n, T2_BYTES), dtype=np.uint8)
    got = L.orc_match_global(kp, tp, t1.shape[0], D, _p(out, ctypes.c_uint8), n)
    assert got == n
    return out


def match_global_bruteforce(recs_unsorted: np.ndarray, D: int) -> np.ndarray:
    """Cross-bucket pairs (a, b) by an O(n^2) scan of the unsorted records."""
    recs = np.ascontiguousarray(recs_unsorted, dtype=np.uint8)
    L = lib()
    n = int(L.orc_match_global_bruteforce(_p(recs, ctypes.c_uint8), recs.shape[0], D, None, 0))
    out = np.zeros((n, 2), dtype=np.uint32)
    L.orc_match_global_bruteforce(_p(recs, ctypes.c_uint8), recs.shape[0], D,
                                  _p(out, ctypes.c_uint32), n)
    return out


def table2_key(t2: np.ndarray) -> np.ndarray:
    """key2 of Table-2 records: big-endian u64 of the hash2 bytes (8..15)."""
    t2 = np.ascontiguousarray(t2, dtype=np.uint8)
    return t2[:, 8:16].copy().view(">u8").reshape(-1).astype(np.uint64)


def sort_table2(t2: np.ndarray) -> np.ndarray:
    """Table 2 ordered by (key2, a, b) ascending: the same 16-byte records,
    sorted by their hash for lookups (NEXT-3); numpy's stable lexsort as the
    sorting step, ties on key2 broken by the pair's nonces."""
    t2 = np.ascontiguousarray(t2, dtype=np.uint8)
    a = t2[:, 0:4].copy().view("<u4").reshape(-1)
    b = t2[:, 4:8].copy().view("<u4").reshape(-1)
    order = np.lexsort((b, a, table2_key(t2)))
    return t2[order]


def plot(K: int, key: bytes, D: int | None = None):
    """(Table 1, Table 2) of one plot."""
    t1 = table1(K, key)
    t2 = match(key, t1, default_distance(K) if D is None else D)
    return t1, t2


# --------------------------------------------------------- numpy views --

def key64(recs: np.ndarray) -> np.ndarray:
    """Big-endian u64 of the 8 hash bytes of each 12-byte record."""
    h = np.ascontiguousarray(recs[:, 4:12])
    return h.view(">u8").reshape(-1).astype(np.uint64)


def nonces(recs: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(recs[:, 0:4]).view("<u4").reshape(-1).astype(np.uint32)
