"""Pins of the CPU oracle to things other than itself (no GPU).

* BLAKE3's G function, round pattern and IV are the ones BLAKE2s uses
  (BLAKE3 spec Sec. 2.2; RFC 7693 Sec. 3.1-3.2).  BLAKE2s assembled from the
  oracle's own round function and IV must reproduce hashlib.blake2s.
* The whole BLAKE3 compression (message permutation, counter / block-length
  / flag words, seven-round schedule, output fold) must reproduce the
  published BLAKE3 digests of the empty input and of "abc"
  (tests/golden/blake3_vectors.json).  The keyed mode is that compression
  with the key as chaining value and the KEYED_HASH flag.
* Table 1 order (R5, R6) must equal numpy's lexsort of the big-endian key64
  and nonce; bucket offsets must equal numpy's bincount + cumsum.
* The match (R8, R9, R11) must equal an O(n^2) numpy scan, satisfy
  hand-worked boundary cases, and hit the closed-form expected pair count.
* Paper numbers (2^24 buckets, 24.7 GB at K=31) are checked against the
  record layout of R4 from tests/golden/paper_numbers.json.
"""
import hashlib
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2606_14007_gb300.inputs import plot_key

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# RFC 7693 Sec. 2.7: BLAKE2s message schedule.
SIGMA = [
    [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15],
    [14, 10, 4, 8, 9, 15, 13, 6, 1, 12, 0, 2, 11, 7, 5, 3],
    [11, 8, 12, 0, 5, 2, 15, 13, 10, 14, 3, 6, 7, 1, 9, 4],
    [7, 9, 3, 1, 13, 12, 11, 14, 2, 6, 5, 10, 4, 0, 15, 8],
    [9, 0, 5, 7, 2, 4, 10, 15, 14, 1, 11, 12, 6, 8, 3, 13],
    [2, 12, 6, 10, 0, 11, 8, 3, 4, 13, 7, 5, 15, 14, 1, 9],
    [12, 5, 1, 15, 14, 13, 4, 10, 0, 7, 6, 3, 9, 2, 8, 11],
    [13, 11, 7, 14, 12, 1, 3, 9, 5, 0, 15, 4, 8, 6, 2, 10],
    [6, 15, 14, 9, 11, 3, 0, 8, 12, 2, 13, 7, 1, 4, 10, 5],
    [10, 2, 8, 4, 7, 6, 1, 5, 15, 11, 9, 14, 3, 12, 13, 0],
]


def _blake2s_from_oracle(msg: bytes, key: bytes = b"", outlen: int = 32) -> bytes:
    """BLAKE2s (RFC 7693 Sec. 3.2-3.3) whose rounds are the oracle's round function."""
    IV = orc.iv()
    h = IV.copy()
    h[0] ^= np.uint32(0x01010000 ^ (len(key) << 8) ^ outlen)
    data = (key.ljust(64, b"\0") if key else b"") + msg
    if not data:
        blocks = [b"\0" * 64]
    else:
        blocks = [data[i:i + 64].ljust(64, b"\0") for i in range(0, len(data), 64)]
    t = 0
    for bi, blk in enumerate(blocks):
        last = bi == len(blocks) - 1
        t = len(data) if last else t + 64
        m = np.frombuffer(blk, dtype="<u4").astype(np.uint32)
        v = np.concatenate([h, IV]).astype(np.uint32)
        v[12] ^= np.uint32(t & 0xFFFFFFFF)
        v[13] ^= np.uint32(t >> 32)
        if last:
            v[14] ^= np.uint32(0xFFFFFFFF)
        for r in range(10):
            v = orc.round_fn(v, m[SIGMA[r]])
        h = h ^ v[:8] ^ v[8:]
    return h.astype("<u4").tobytes()[:outlen]


@pytest.mark.parametrize("seed", range(6))
def test_round_and_iv_reproduce_blake2s(seed):
    rng = np.random.default_rng(seed)
    for n in [0, 1, 3, 4, 8, 63, 64, 65, 130]:
        msg = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
        assert _blake2s_from_oracle(msg) == hashlib.blake2s(msg).digest()
        key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
        assert _blake2s_from_oracle(msg, key) == hashlib.blake2s(msg, key=key).digest()


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("case", _golden("blake3_vectors.json")["hash"],
                         ids=lambda c: repr(c["input_ascii"]))
def test_compress_reproduces_published_blake3_digests(case):
    # One-chunk, one-block BLAKE3 hash (spec Sec. 2.2-2.4): chaining value =
    # IV, counter 0, block_len = message length, flags CHUNK_START | CHUNK_END
    # | ROOT; the digest is output words 0..7, little-endian.  The empty input
    # pins block_len 0, "abc" block_len 3 and a nonzero message word.
    fl = _golden("blake3_vectors.json")["flags"]
    msg = case["input_ascii"].encode()
    block = np.frombuffer(msg.ljust(64, b"\0"), dtype="<u4").astype(np.uint32)
    out = orc.compress(orc.iv(), block, 0, len(msg),
                       fl["CHUNK_START"] | fl["CHUNK_END"] | fl["ROOT"])
    assert out[:8].astype("<u4").tobytes().hex() == case["digest"]


@pytest.mark.parametrize("n", [0, 1, 4, 8, 33, 64])
def test_keyed_hash_is_compress_with_key_and_keyed_flag(n):
    # keyed_hash (spec Sec. 2.3): the key's eight LE words are the chaining
    # value and every block carries KEYED_HASH; one chunk of one block for
    # messages of at most 64 bytes.
    fl = _golden("blake3_vectors.json")["flags"]
    rng = np.random.default_rng(100 + n)
    key = rng.integers(0, 256, 32, dtype=np.uint8).tobytes()
    msg = rng.integers(0, 256, n, dtype=np.uint8).tobytes()
    cv = np.frombuffer(key, dtype="<u4").astype(np.uint32)
    block = np.frombuffer(msg.ljust(64, b"\0"), dtype="<u4").astype(np.uint32)
    out = orc.compress(cv, block, 0, n,
                       fl["CHUNK_START"] | fl["CHUNK_END"] | fl["ROOT"] | fl["KEYED_HASH"])
    assert orc.keyed_hash(key, msg, 32) == out[:8].astype("<u4").tobytes()


def test_keyed_hash_shapes():
    key = plot_key(0)
    full = orc.keyed_hash(key, b"\x01\x00\x00\x00", 32)
    assert orc.keyed_hash(key, b"\x01\x00\x00\x00", 8) == full[:8]
    # Every message byte, every key byte and the length take part in the hash.
    assert orc.keyed_hash(key, b"\x01\x00\x00\x00") != orc.keyed_hash(key, b"\x01\x00\x00")
    for i in range(32):
        k2 = bytearray(key)
        k2[i] ^= 0x80
        assert orc.keyed_hash(bytes(k2), b"\x01\x00\x00\x00") != full
    with pytest.raises(ValueError):
        orc.keyed_hash(key, b"\0" * 65)


@pytest.mark.parametrize("K,seed", [(1, 0), (5, 1), (10, 2), (14, 3)])
def test_table1_is_numpy_sort_of_hash_records(K, seed):
    key = plot_key(seed)
    raw = orc.table1_unsorted(K, key)
    t1 = orc.table1(K, key)
    n = 1 << K
    assert t1.shape == (n, 12)
    # R1: nonce i sits in record i of the unsorted table as LE32.
    assert np.array_equal(orc.nonces(raw), np.arange(n, dtype=np.uint32))
    # R3/R4: record bytes 4..11 are the first 8 bytes of the keyed hash.
    for i in [0, 1, n // 2, n - 1]:
        assert raw[i, 4:].tobytes() == orc.keyed_hash(key, int(i).to_bytes(4, "little"), 8)
    # R5/R6: sorted by big-endian key64, ties by nonce -- numpy lexsort.
    order = np.lexsort((orc.nonces(raw), orc.key64(raw)))
    assert np.array_equal(t1, raw[order])


def test_table1_tie_break_by_nonce():
    # Crafted records: equal hashes, nonces out of order (R6 tie-break).
    recs = np.zeros((6, 12), dtype=np.uint8)
    hashes = [b"\x00" * 8, b"\xff" * 8, b"\x00" * 8, b"\x01" + b"\x00" * 7, b"\x00" * 8,
              b"\x00" * 7 + b"\x01"]
    for i, (nonce, h) in enumerate(zip([9, 1, 3, 2, 7, 5], hashes)):
        recs[i, :4] = np.frombuffer(int(nonce).to_bytes(4, "little"), dtype=np.uint8)
        recs[i, 4:] = np.frombuffer(h, dtype=np.uint8)
    out = orc.sort_table1(recs)
    assert list(orc.nonces(out)) == [3, 7, 9, 5, 2, 1]


@pytest.mark.parametrize("K", [6, 13])
def test_bucket_offsets_match_numpy(K):
    t1 = orc.table1(K, plot_key(K))
    off = orc.bucket_offsets(t1)
    b = (orc.key64(t1) >> np.uint64(40)).astype(np.int64)
    ref = np.zeros((1 << 24) + 1, dtype=np.uint64)
    ref[1:] = np.cumsum(np.bincount(b, minlength=1 << 24))
    assert np.array_equal(off, ref)


def _numpy_pairs(recs: np.ndarray, D: int) -> set:
    """O(n^2) numpy scan of the match predicate (R8) over unsorted records."""
    k = orc.key64(recs)
    nz = orc.nonces(recs)
    b = k >> np.uint64(40)
    same = b[:, None] == b[None, :]
    before = (k[:, None] < k[None, :]) | ((k[:, None] == k[None, :]) & (nz[:, None] < nz[None, :]))
    with np.errstate(over="ignore"):
        close = (k[None, :] - k[:, None]) < np.uint64(D)
    xs, ys = np.nonzero(same & before & close)
    return set(zip(nz[xs].tolist(), nz[ys].tolist()))


def _records(keys64, nonces=None):
    keys64 = np.asarray(keys64, dtype=np.uint64)
    n = keys64.shape[0]
    if nonces is None:
        nonces = np.arange(n, dtype=np.uint32)
    recs = np.zeros((n, 12), dtype=np.uint8)
    recs[:, :4] = np.asarray(nonces, dtype="<u4").view(np.uint8).reshape(n, 4)
    recs[:, 4:] = keys64.astype(">u8").view(np.uint8).reshape(n, 8)
    return recs


@pytest.mark.parametrize("K,seed,shift", [(8, 0, 0), (11, 1, 0), (12, 2, 0), (12, 3, 20),
                                          (10, 4, 30)])
def test_match_equals_bruteforce(K, seed, shift):
    key = plot_key(seed)
    raw = orc.table1_unsorted(K, key)
    if shift:
        # Squeeze every key64 into a few buckets so that D < bucket width
        # matters at small K (the K >= 25 regime).
        k = orc.key64(raw) >> np.uint64(shift)
        raw = _records(k, orc.nonces(raw))
    t1 = orc.sort_table1(raw)
    D = orc.default_distance(K + shift)
    t2 = orc.match(key, t1, D)
    got = set(zip(orc.nonces(t2[:, 0:4]).tolist(), orc.nonces(t2[:, 4:8]).tolist()))
    assert len(got) == t2.shape[0]
    ref = _numpy_pairs(raw, D)
    assert got == ref
    bf = orc.match_bruteforce(raw, D)
    assert set(map(tuple, bf.tolist())) == ref
    # R10: hash2 recomputes; R11: bucket, then i, then j order.
    pos = {int(nv): i for i, nv in enumerate(orc.nonces(t1))}
    ranks = [(pos[a], pos[b]) for a, b in zip(orc.nonces(t2[:, 0:4]).tolist(),
                                               orc.nonces(t2[:, 4:8]).tolist())]
    assert ranks == sorted(ranks)
    for r in range(0, t2.shape[0], max(1, t2.shape[0] // 17)):
        assert t2[r, 8:].tobytes() == orc.keyed_hash(key, t2[r, :8].tobytes(), 8)


def test_match_hand_worked_boundaries():
    B = 1 << 40  # logical bucket width in key64 units
    D = 1000
    keys = [
        5 * B + 10,          # n0
        5 * B + 10,          # n1: delta 0 with n0 -> match
        5 * B + 1009,        # n2: delta 999 from n0/n1 -> match; from itself none
        5 * B + 1010,        # n3: delta 1000 from n0/n1 -> NO (strict <); 1 from n2 -> match
        6 * B - 1,           # n4: bucket 5, far away
        6 * B,               # n5: bucket 6, delta 1 from n4 -> NO (other bucket)
    ]
    t1 = orc.sort_table1(_records(keys))
    t2 = orc.match(plot_key(0), t1, D)
    pairs = list(zip(orc.nonces(t2[:, 0:4]).tolist(), orc.nonces(t2[:, 4:8]).tolist()))
    assert pairs == [(0, 1), (0, 2), (1, 2), (2, 3)]


def test_match_closed_form_pair_count():
    # n uniform keys in one bucket; a pair matches iff |dx| < D.  For u = D/W
    # the pair probability is 2u - u^2, so E = C(n,2)(2u - u^2) and, the
    # pair indicators being nearly uncorrelated, sd ~ sqrt(E).
    rng = np.random.default_rng(11)
    n, W = 20000, 1 << 40
    D = W // 1000
    keys = (np.uint64(7 * W) + rng.integers(0, W, n, dtype=np.uint64)).astype(np.uint64)
    t1 = orc.sort_table1(_records(keys))
    got = orc.match_count(plot_key(1), t1, D)
    u = D / W
    E = n * (n - 1) / 2 * (2 * u - u * u)
    assert abs(got - E) < 6 * math.sqrt(E) + 6 * n * u, (got, E)


def test_full_plot_pair_count_closed_form():
    # K <= 24: D spans the whole bucket, so every same-bucket pair matches:
    # E|T2| = 2^24 * lambda^2 / 2 with lambda = 2^(K-24); for Poisson bucket
    # sizes Var C(n,2) = lambda^3 + lambda^2/2 per bucket.
    for K, seed in [(16, 5), (17, 6)]:
        lam = 2.0 ** (K - 24)
        t1 = orc.table1(K, plot_key(seed))
        got = orc.match_count(plot_key(seed), t1, orc.default_distance(K))
        E = 2 ** 24 * lam * lam / 2
        sd = math.sqrt(2 ** 24 * (lam ** 3 + lam * lam / 2))
        assert abs(got - E) < 6 * sd, (K, got, E, sd)


def test_paper_numbers_fixture():
    with open(os.path.join(GOLDEN, "paper_numbers.json")) as f:
        g = json.load(f)
    assert g["bucket_count"]["value"] == 2 ** 24
    # R4: 12-byte records reproduce the printed K=31 Table-1 footprint within
    # the few percent the paper's capacity slack / rounding allow.
    t1_gb = 12 * 2 ** 31 / 1e9
    assert abs(t1_gb - g["table1_gb_k31"]["value"]) / g["table1_gb_k31"]["value"] < 0.05
    # 11- and 13-byte records would miss by more.
    assert abs(11 * 2 ** 31 / 1e9 - 24.7) > abs(t1_gb - 24.7)
    assert abs(13 * 2 ** 31 / 1e9 - 24.7) > abs(t1_gb - 24.7)
    assert orc.default_distance(31) == 2 ** 33


# ---------------------------------------------------------------------------
# Cross-bucket variant of the match (every pair of the whole Table-1 order
# under the threshold; Sec. II-B's pairwise match without the bucket edge).

def _numpy_pairs_global(recs: np.ndarray, D: int) -> set:
    """O(n^2) numpy scan of the cross-bucket predicate over unsorted records."""
    k = orc.key64(recs)
    nz = orc.nonces(recs)
    before = (k[:, None] < k[None, :]) | ((k[:, None] == k[None, :]) & (nz[:, None] < nz[None, :]))
    with np.errstate(over="ignore"):
        close = (k[None, :] - k[:, None]) < np.uint64(D)
    xs, ys = np.nonzero(before & close)
    return set(zip(nz[xs].tolist(), nz[ys].tolist()))


@pytest.mark.parametrize("K,seed,shift", [(8, 20, 0), (11, 21, 0), (12, 22, 0), (12, 23, 30),
                                          (10, 24, 36)])
def test_match_global_equals_bruteforce(K, seed, shift):
    key = plot_key(seed)
    raw = orc.table1_unsorted(K, key)
    if shift:
        # squeeze the keys so that many pairs straddle logical buckets
        k = orc.key64(raw) >> np.uint64(shift)
        raw = _records(k << np.uint64(shift - 4), orc.nonces(raw))
    t1 = orc.sort_table1(raw)
    D = orc.default_distance(K) >> np.uint64(shift // 2) if shift else orc.default_distance(K)
    D = int(D)
    t2 = orc.match_global(key, t1, D)
    got = set(zip(orc.nonces(t2[:, 0:4]).tolist(), orc.nonces(t2[:, 4:8]).tolist()))
    assert len(got) == t2.shape[0]
    ref = _numpy_pairs_global(raw, D)
    assert got == ref
    bf = orc.match_global_bruteforce(raw, D)
    assert set(map(tuple, bf.tolist())) == ref
    # i, then j order over the whole Table 1; hash2 recomputes (R10)
    pos = {int(nv): i for i, nv in enumerate(orc.nonces(t1))}
    ranks = [(pos[a], pos[b]) for a, b in zip(orc.nonces(t2[:, 0:4]).tolist(),
                                               orc.nonces(t2[:, 4:8]).tolist())]
    assert ranks == sorted(ranks)
    for r in range(0, t2.shape[0], max(1, t2.shape[0] // 13)):
        assert t2[r, 8:].tobytes() == orc.keyed_hash(key, t2[r, :8].tobytes(), 8)


def test_match_global_contains_bucket_match():
    # With D at most the bucket width the bucket-scope pairs are exactly the
    # cross-bucket variant's pairs whose two keys share a logical bucket,
    # in the same relative order.
    key = plot_key(25)
    t1 = orc.table1(16, key)
    for D in [1 << 40, 1 << 38, 1 << 35]:
        g = orc.match_global(key, t1, D)
        b = orc.match(key, t1, D)
        kg = {int(n): int(k) for n, k in zip(orc.nonces(t1), orc.key64(t1))}
        same = [r for r in g if (kg[int(r[:4].view("<u4")[0])] >> 40) ==
                (kg[int(r[4:8].view("<u4")[0])] >> 40)]
        assert np.array_equal(np.array(same, dtype=np.uint8).reshape(-1, 16), b)


def test_match_global_closed_form_pair_count():
    # N uniform key64 values: a pair is within D with probability 2u - u^2,
    # u = D / 2^64, so E|T2| = C(N,2)(2u - u^2) ~ N at the default distance
    # 2^(64-K).  Each record's partner count is ~Poisson(1): Var ~ 3N/2.
    for K, seed in [(16, 26), (18, 27)]:
        N = 1 << K
        got = orc.match_global(plot_key(seed), orc.table1(K, plot_key(seed)),
                               orc.default_distance(K)).shape[0]
        u = orc.default_distance(K) / 2.0 ** 64
        E = N * (N - 1) / 2 * (2 * u - u * u)
        assert abs(got - E) < 6 * math.sqrt(2 * N), (K, got, E)


def test_match_global_all_pairs():
    # D = 2^64 - 1 matches every pair except those exactly 2^64 - 1 apart:
    # C(N, 2) records, (i, j) in lexicographic order of Table-1 ranks.
    K, key = 7, plot_key(28)
    t1 = orc.table1(K, key)
    t2 = orc.match_global(key, t1, (1 << 64) - 1)
    n = t1.shape[0]
    assert t2.shape[0] == n * (n - 1) // 2
    nz = orc.nonces(t1).tolist()
    want = [(nz[i], nz[j]) for i in range(n) for j in range(i + 1, n)]
    assert list(zip(orc.nonces(t2[:, 0:4]).tolist(), orc.nonces(t2[:, 4:8]).tolist())) == want


# ---------------------------------------------------------------------------
# Table 2 sorted by hash2 (NEXT-3): the same records ordered by (key2, a, b).

def test_sort_table2_hand_example():
    # five records, two with equal hash2 (tie broken by a, then b)
    def rec(a, b, h):
        return (np.array([a, b], dtype="<u4").view(np.uint8).tolist() +
                list(int(h).to_bytes(8, "big")))
    rows = np.array([rec(7, 9, 0x0200), rec(1, 2, 0xFFFF000000000000), rec(3, 4, 0x0200),
                     rec(3, 1, 0x0200), rec(9, 9, 0x0001)], dtype=np.uint8)
    got = orc.sort_table2(rows)
    want = rows[[4, 3, 2, 0, 1]]
    assert np.array_equal(got, want)


def test_sort_table2_is_an_ordered_permutation():
    key = plot_key(40)
    t1 = orc.table1(15, key)
    t2 = orc.match_global(key, t1, orc.default_distance(15))
    s = orc.sort_table2(t2)
    # same multiset of records
    assert np.array_equal(np.sort(t2.view("V16").reshape(-1)), np.sort(s.view("V16").reshape(-1)))
    # ascending (key2, a, b) between neighbours
    k = orc.table2_key(s).astype(object)
    a = s[:, 0:4].copy().view("<u4").reshape(-1).astype(object)
    b = s[:, 4:8].copy().view("<u4").reshape(-1).astype(object)
    keys = list(zip(k, a, b))
    assert all(x < y for x, y in zip(keys, keys[1:]))
    # key2 is the big-endian reading of the hash bytes the record carries
    r = s[len(s) // 2]
    assert int(orc.table2_key(s[len(s) // 2: len(s) // 2 + 1])[0]) == int.from_bytes(r[8:].tobytes(), "big")


def test_window_slices_partition_the_plot():
    # The expected tables of window plots (tests/window_slices.py) partition
    # the whole plot's tables in order: concatenated over the windows they
    # are Table 1 and Table 2; every record of slice w has key64's top c bits
    # == w, and both records of every pair of slice w lie in window w.
    from window_slices import oracle_windows, window_of_t1
    K, key = 14, plot_key(321)
    r1 = orc.table1(K, key)
    r2 = orc.match(key, r1, orc.default_distance(K))
    for c in (1, 2, 3, 5):
        sl = oracle_windows(r1, r2, c)
        assert np.array_equal(np.concatenate([s1 for s1, _ in sl]), r1)
        assert np.array_equal(np.concatenate([s2 for _, s2 in sl]), r2)
        win_of_nonce = {}
        for w, (s1, _) in enumerate(sl):
            ws, _ = window_of_t1(s1, c)
            assert (ws == w).all()
            for n in np.ascontiguousarray(s1[:, :4]).view("<u4").ravel():
                win_of_nonce[int(n)] = w
        for w, (_, s2) in enumerate(sl):
            ab = np.ascontiguousarray(s2[:, :8]).view("<u4")
            assert all(win_of_nonce[int(a)] == w and win_of_nonce[int(b)] == w for a, b in ab)


def test_pair_hash_rows():
    key = plot_key(11)
    rng = np.random.default_rng(11)
    rows = rng.integers(0, 256, (257, 16), dtype=np.uint8)
    for threads in (1, 4):
        h = orc.pair_hash(key, rows, threads)
        for i in range(rows.shape[0]):
            assert h[i].tobytes() == orc.keyed_hash(key, rows[i, :8].tobytes(), 8)
    assert orc.pair_hash(key, rows[:, :8], 2).tobytes() == orc.pair_hash(key, rows, 1).tobytes()
    with pytest.raises(ValueError):
        orc.pair_hash(key, rows[:, :7])


@pytest.mark.parametrize("K,seed,D", [(1, 12, None), (10, 13, None), (16, 14, None),
                                      (16, 15, 1 << 37)])
def test_allcore_plot_equals_plain_plot(K, seed, D):
    # plot_allcores (threaded hash, grouping by the top key byte, threaded
    # qsort per group, match over runs of whole buckets) = the plain oracle.
    key = plot_key(seed)
    t1 = orc.table1(K, key)
    t2 = orc.match(key, t1, orc.default_distance(K) if D is None else D)
    for threads in (1, 2, 7, 16):
        a1, a2 = orc.plot_allcores(K, key, threads, D)
        assert np.array_equal(a1, t1) and np.array_equal(a2, t2)
