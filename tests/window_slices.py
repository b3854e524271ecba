"""Slices of the oracle's whole-plot tables by window: the expected tables of
a window plot (vx_opts.window_bits = c, window = w) are the records whose
key64 has top c bits == w and the Table-2 pairs of those records (a pair's
records share a logical bucket, hence a window)."""
import numpy as np


def window_of_t1(r1, c):
    key64 = np.ascontiguousarray(r1[:, 4:12]).view(">u8").ravel().astype(np.uint64)
    return (key64 >> np.uint64(64 - c)).astype(np.int64), key64


def oracle_windows(r1, r2, c):
    """[(Table-1 slice, Table-2 slice)] of the 2^c windows."""
    w1, key64 = window_of_t1(r1, c)
    nonce = np.ascontiguousarray(r1[:, :4]).view("<u4").ravel()
    key_of = np.empty(r1.shape[0], dtype=np.uint64)
    key_of[nonce] = key64
    a = np.ascontiguousarray(r2[:, :4]).view("<u4").ravel()
    w2 = (key_of[a] >> np.uint64(64 - c)).astype(np.int64)
    return [(r1[w1 == w], r2[w2 == w]) for w in range(1 << c)]
