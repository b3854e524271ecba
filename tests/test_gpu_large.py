"""Full-size plots over K = 23 ... 32, compared with the oracle.

K = 23 ... 27: both tables element by element against the oracle's, run
on every host core (its all-core variant, pinned to the plain oracle).

K = 27 ... 31 (K=31 is the configuration bench.py times): properties that
hold at any size, computed on the device with torch independently of the
kernels, plus every record's hash and every pair's hash2 recomputed by the
oracle.  Together these fix both tables bit for bit:

Table 1: strictly increasing in (key64, nonce); every nonce exactly once;
every record's hash bytes equal the oracle's keyed hash of its nonce.  The
oracle's Table 1 is the unique (key64, nonce)-sorted list of those records.
Table 2: every entry (a, b) has pos(a) < pos(b) in Table 1, the same logical
bucket (bucket scope) and key64_b - key64_a < D; entries strictly increasing
in (pos(a), pos(b)); their number equals an independent count of qualifying
pairs; every hash2 equals the oracle's.  The oracle's Table 2 is the unique
(i, j)-ordered list of all qualifying pairs, so the two are equal.  The
count is also checked against the closed-form expectation 2^24 (lambda -
1/2), or C(N,2) 2D / 2^64 for the cross-bucket match.

K = 32 (beyond the paper's range) keeps the sampled recomputation.
"""
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_2606_14007_gb300.inputs import plot_key  # noqa: E402

CHUNK = 1 << 27
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def vx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_14007_gb300 import vaultx
    return vaultx


def fields(t1_rows):
    b = t1_rows.long()
    nonce = b[:, 0] | (b[:, 1] << 8) | (b[:, 2] << 16) | (b[:, 3] << 24)
    hi = (b[:, 4] << 24) | (b[:, 5] << 16) | (b[:, 6] << 8) | b[:, 7]
    lo = (b[:, 8] << 24) | (b[:, 9] << 16) | (b[:, 10] << 8) | b[:, 11]
    return nonce, hi, lo


def check_plot(vx, K, seed, scope=0, every_hash=True, **kw):
    # scope 1: the cross-bucket match (no same-bucket condition; E|T2| ~ N)
    key = plot_key(seed)
    N = 1 << K
    p = vx.Plot(K, key, vx.make_opts(match_scope=scope, **kw) if (scope or kw) else None)
    p.run()
    n2 = p.sync()
    t1 = p.t1
    check_tables(K, key, seed, t1, p.t2, n2, scope, every_hash=every_hash)
    # first and last records of Table 1 and Table 2, and the bucket offsets
    off = p.offsets()
    assert int(off[0]) == 0 and int(off[-1]) == N
    b_first = int(fields(t1[:1])[1][0] >> 8)
    assert int(off[b_first]) == 0 and int(off[b_first + 1]) > 0
    p.close()
    torch.cuda.empty_cache()


def first_diff(got, ref):
    bad = np.nonzero((got != ref).any(axis=1))[0]
    return int(bad[0]) if bad.size else -1


def check_every_hash(key, t1, t2, n2, pos):
    """Every Table-1 record's hash bytes against the oracle's keyed hash of
    its nonce (records found through pos, nonce -> Table-1 position), and
    every Table-2 record's hash2 against the oracle's pair hash of its
    (a, b); the oracle runs on every host core, chunk by chunk."""
    N = t1.shape[0]
    for s in range(0, N, CHUNK):
        e = min(N, s + CHUNK)
        ref = orc.hash_range(key, s, e, THREADS)[:, 4:]
        got = t1[pos[s:e].long(), 4:].cpu().numpy()
        d = first_diff(got, ref)
        assert d < 0, "Table-1 hash of nonce %d differs from the oracle" % (s + d)
    for s in range(0, n2, CHUNK):
        e = min(n2, s + CHUNK)
        rows = t2[s:e].cpu().numpy()
        ref = orc.pair_hash(key, rows, THREADS)
        d = first_diff(rows[:, 8:], ref)
        assert d < 0, "Table-2 hash2 of record %d differs from the oracle" % (s + d)


def check_tables(K, key, seed, t1, t2, n2, scope=0, every_hash=True):
    """The properties of a whole plot's tables t1 (2^K x 12) and t2 (n2 x 16),
    uint8 tensors on the device; with every_hash, every hash recomputed by
    the oracle, else 3000 sampled records and pairs."""
    N = 1 << K
    D = 1 << (64 - K)
    assert t1.shape[0] == N and t2.shape[0] == n2
    dev = t1.device
    counts = torch.zeros(N, dtype=torch.int32, device=dev)
    pos = torch.empty(N, dtype=torch.int32, device=dev)
    independent = 0
    prev = None
    for s in range(0, N, CHUNK):
        e = min(N, s + CHUNK)
        nonce, hi, lo = fields(t1[s:e])
        counts.index_add_(0, nonce, torch.ones_like(nonce, dtype=torch.int32))
        pos[nonce] = torch.arange(s, e, dtype=torch.int32, device=dev)
        # strictly increasing (key64, nonce), including across the chunk seam
        if prev is not None:
            nonce = torch.cat([prev[0], nonce]); hi = torch.cat([prev[1], hi]); lo = torch.cat([prev[2], lo])
        inc = (hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & ((lo[1:] > lo[:-1]) |
                                                           ((lo[1:] == lo[:-1]) & (nonce[1:] > nonce[:-1]))))
        assert bool(inc.all()), "Table 1 not sorted near record %d" % s
        prev = (nonce[-1:], hi[-1:], lo[-1:])
        # independent pair count for records of this chunk (needs a look-ahead)
        ahead = min(N, e + 4096)
        _, hi2, lo2 = fields(t1[s:ahead])
        bucket = hi2 >> 8
        k40 = ((hi2 & 0xFF) << 32) | lo2
        n_own = e - s
        idx = torch.arange(n_own, device=dev)
        alive = torch.ones(n_own, dtype=torch.bool, device=dev)
        k = 1
        while bool(alive.any()):
            j = idx + k
            ok = j < bucket.shape[0]
            jj = torch.where(ok, j, torch.zeros_like(j))
            same = (bucket[jj] == bucket[:n_own]) if not scope else torch.ones_like(alive)
            gap = (k40[jj] - k40[:n_own]) + ((bucket[jj] - bucket[:n_own]) << 40)
            m = alive & ok & same & (gap < D)
            independent += int(m.sum())
            alive = m
            k += 1
            assert k < 4096, "look-ahead too short"
    assert bool((counts == 1).all()), "a nonce is missing or repeated in Table 1"
    assert n2 == independent, (n2, independent)
    lam = N / 2 ** 24
    E = 2 ** 24 * (lam - 0.5) if not scope else N * (N - 1) / 2 * (2 * D / 2 ** 64)
    assert abs(n2 - E) < 8 * math.sqrt(8 * N), (n2, E)
    # Table 2 entries
    last = None
    for s in range(0, n2, CHUNK):
        e = min(n2, s + CHUNK)
        b = t2[s:e].long()
        a_n = b[:, 0] | (b[:, 1] << 8) | (b[:, 2] << 16) | (b[:, 3] << 24)
        b_n = b[:, 4] | (b[:, 5] << 8) | (b[:, 6] << 16) | (b[:, 7] << 24)
        i = pos[a_n].long()
        j = pos[b_n].long()
        assert bool((j > i).all())
        _, hi_i, lo_i = fields(t1[i])
        _, hi_j, lo_j = fields(t1[j])
        if not scope:
            assert bool(((hi_i >> 8) == (hi_j >> 8)).all()), "pair crosses a bucket"
        k40i = ((hi_i & 0xFF) << 32) | lo_i
        k40j = ((hi_j & 0xFF) << 32) | lo_j
        gap = (k40j - k40i) + (((hi_j >> 8) - (hi_i >> 8)) << 40)
        assert bool((gap < D).all()), "pair beyond the match distance"
        if last is not None:
            i = torch.cat([last[0], i]); j = torch.cat([last[1], j])
        order = (i[1:] > i[:-1]) | ((i[1:] == i[:-1]) & (j[1:] > j[:-1]))
        assert bool(order.all()), "Table 2 out of (i, j) order"
        last = (i[-1:], j[-1:])
    if every_hash:
        check_every_hash(key, t1, t2, n2, pos)
    else:
        rng = np.random.default_rng(seed)
        rows = torch.from_numpy(rng.integers(0, N, 3000)).to(dev)
        for r in t1[rows].cpu().numpy():
            assert r[4:].tobytes() == orc.keyed_hash(key, r[:4].tobytes(), 8)
        rows = torch.from_numpy(rng.integers(0, n2, 3000)).to(dev)
        for r in t2[rows].cpu().numpy():
            assert r[8:].tobytes() == orc.keyed_hash(key, r[:8].tobytes(), 8)
    del counts, pos


@pytest.mark.parametrize("K", [23, 24, 25, 26, 27])
def test_plot_equals_oracle_elementwise(vx, K):
    # The small-K parity test's comparison at K = 23 ... 27 (key from seed K,
    # as bench.py's plots): whole tables and the bucket offsets.
    key = plot_key(K)
    p = vx.Plot(K, key)
    p.run()
    n2 = p.sync()
    g1 = p.t1.cpu().numpy()
    g2 = p.t2.cpu().numpy()
    off = p.offsets().cpu().numpy()
    p.close()
    torch.cuda.empty_cache()
    r1, r2 = orc.plot_allcores(K, key, THREADS)
    assert g1.shape == r1.shape
    d = first_diff(g1, r1)
    assert d < 0, "Table 1 differs from the oracle at record %d" % d
    assert n2 == r2.shape[0], (n2, r2.shape[0])
    d = first_diff(g2, r2)
    assert d < 0, "Table 2 differs from the oracle at record %d" % d
    assert np.array_equal(off.astype(np.uint64), orc.bucket_offsets(r1))


@pytest.mark.parametrize("K", [24, 25])
def test_split_path_equals_oracle_elementwise(vx, K):
    # vx_table1 then vx_match (the sort's count mode, the pair-offset scan
    # and the match kernel) at sizes past the small-K parity test.
    key = plot_key(K + 300)
    p = vx.Plot(K, key)
    p.run_split()
    n2 = p.sync()
    g1 = p.t1.cpu().numpy()
    g2 = p.t2.cpu().numpy()
    p.close()
    torch.cuda.empty_cache()
    r1, r2 = orc.plot_allcores(K, key, THREADS)
    d = first_diff(g1, r1)
    assert d < 0, "Table 1 differs from the oracle at record %d" % d
    assert n2 == r2.shape[0], (n2, r2.shape[0])
    d = first_diff(g2, r2)
    assert d < 0, "Table 2 differs from the oracle at record %d" % d


@pytest.mark.parametrize("K", [24, 25])
def test_sorted_table2_equals_oracle_elementwise(vx, K):
    # vx_sort_table2 at sizes past its small-K test: the oracle's Table 2
    # in (key2, a, b) order, byte for byte.
    key = plot_key(K + 400)
    p = vx.Plot(K, key)
    p.run()
    n2 = p.sync()
    wb = vx.vx_sort_table2_work_bytes(p.handle)
    work = torch.empty(max(wb, 256), dtype=torch.uint8, device="cuda")
    vx.vx_sort_table2(p.handle, work.data_ptr(), wb)
    assert vx.vx_sync(p.handle) == vx.VX_OK
    got = p.t2.cpu().numpy()
    p.close()
    del work
    torch.cuda.empty_cache()
    _, r2 = orc.plot_allcores(K, key, THREADS)
    assert n2 == r2.shape[0], (n2, r2.shape[0])
    ref = orc.sort_table2(r2)
    d = first_diff(got, ref)
    assert d < 0, "sorted Table 2 differs from the oracle at record %d" % d


@pytest.mark.parametrize("K", [27, 28, 29, 30, 31])
def test_plot_bit_exact_by_properties(vx, K):
    check_plot(vx, K, K)


def test_plot_k27_cross_bucket_properties(vx):
    check_plot(vx, 27, 127, scope=1)


def test_plot_k27_with_2pow21_partitions(vx):
    # partitions of ~64 records: 2^21 of them, an 11-bit second scatter level
    # (the layout K=32 uses with its default ~2048-record partitions)
    check_plot(vx, 27, 227, partition_log2=6)


def test_plot_k32_properties(vx):
    # K=32 in one GB300 (about 185 GB: Table 1 51.5 GB, Table 2 68.7 GB,
    # partition slots 62 GB), no chunking.  Without a 2^32-entry position
    # map: Table 1 strictly increasing with nonce sums of a permutation of
    # 0..N-1 (sum and sum of squares mod 2^64), the pair count equal to an
    # independent count and to the closed form, and sampled Table-2 pairs
    # re-derived by the oracle (same bucket, distance, hash).
    K, seed = 32, 32
    key = plot_key(seed)
    N = 1 << K
    D = 1 << (64 - K)
    p = vx.Plot(K, key)
    p.run()
    n2 = p.sync()
    t1 = p.t1
    dev = t1.device
    s1 = torch.zeros((), dtype=torch.int64, device=dev)
    s2 = torch.zeros((), dtype=torch.int64, device=dev)
    independent = 0
    prev = None
    for s in range(0, N, CHUNK):
        e = min(N, s + CHUNK)
        nonce, hi, lo = fields(t1[s:e])
        s1 += nonce.sum()
        s2 += (nonce * nonce).sum()  # wraps mod 2^64, like the reference below
        if prev is not None:
            nonce = torch.cat([prev[0], nonce]); hi = torch.cat([prev[1], hi]); lo = torch.cat([prev[2], lo])
        inc = (hi[1:] > hi[:-1]) | ((hi[1:] == hi[:-1]) & ((lo[1:] > lo[:-1]) |
                                                           ((lo[1:] == lo[:-1]) & (nonce[1:] > nonce[:-1]))))
        assert bool(inc.all()), "Table 1 not sorted near record %d" % s
        prev = (nonce[-1:], hi[-1:], lo[-1:])
        ahead = min(N, e + 4096)
        _, hi2, lo2 = fields(t1[s:ahead])
        bucket = hi2 >> 8
        k40 = ((hi2 & 0xFF) << 32) | lo2
        n_own = e - s
        idx = torch.arange(n_own, device=dev)
        alive = torch.ones(n_own, dtype=torch.bool, device=dev)
        k = 1
        while bool(alive.any()):
            j = idx + k
            ok = j < bucket.shape[0]
            jj = torch.where(ok, j, torch.zeros_like(j))
            m = alive & ok & (bucket[jj] == bucket[:n_own]) & ((k40[jj] - k40[:n_own]) < D)
            independent += int(m.sum())
            alive = m
            k += 1
            assert k < 4096, "look-ahead too short"
    wrap = lambda x: (x + (1 << 63)) % (1 << 64) - (1 << 63)  # noqa: E731
    assert int(s1) == wrap(N * (N - 1) // 2)
    assert int(s2) == wrap((N - 1) * N * (2 * N - 1) // 6)
    assert n2 == independent, (n2, independent)
    lam = N / 2 ** 24
    E = 2 ** 24 * (lam - 0.5)
    assert abs(n2 - E) < 8 * math.sqrt(8 * N), (n2, E)
    rng = np.random.default_rng(seed)
    for r in t1[torch.from_numpy(rng.integers(0, N, 2000)).to(dev)].cpu().numpy():
        assert r[4:].tobytes() == orc.keyed_hash(key, r[:4].tobytes(), 8)
    for r in p.t2[torch.from_numpy(rng.integers(0, n2, 3000)).to(dev)].cpu().numpy():
        assert r[8:].tobytes() == orc.keyed_hash(key, r[:8].tobytes(), 8)
        ka = int.from_bytes(orc.keyed_hash(key, r[0:4].tobytes(), 8), "big")
        kb = int.from_bytes(orc.keyed_hash(key, r[4:8].tobytes(), 8), "big")
        assert ka >> 40 == kb >> 40 and 0 <= kb - ka < D
    p.close()
    torch.cuda.empty_cache()


def test_plot_k27_tiled_properties(vx):
    # The K=27 plot built in four windows of whole logical buckets
    # (vx_plot_tiled: two window buffers, ~2/4 of the plot's device
    # footprint), its tables gathered in pinned host memory, then checked on
    # the device by the whole-plot properties.
    K, seed = 27, 327
    key = plot_key(seed)
    dev_bytes, _, _ = vx.vx_plot_tiled_bytes(K, 2)
    whole = sum(vx.vx_plot_required_bytes(K))
    assert dev_bytes < 0.65 * whole, (dev_bytes, whole)
    t1, t2 = vx.plot_tiled(K, key, 2)
    check_tables(K, key, seed, t1.cuda(), t2.cuda(), t2.shape[0])
    torch.cuda.empty_cache()
