"""GPU path vs the CPU oracle, element by element (bit-exact: all integer).

Every call goes through the C ABI (ctypes binding).  Sizes run from K=1 to
K=22 (the small configuration) and cover both scatter levels, ragged tiles,
custom match distances, slot overflow, Table-2 capacity and determinism.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_2606_14007_gb300.inputs import plot_key  # noqa: E402


@pytest.fixture(scope="module")
def vx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_14007_gb300 import vaultx
    assert torch.cuda.is_available()
    return vaultx


def run_plot(vx, K, key, opts=None, split=False):
    p = vx.Plot(K, key, opts)
    if split:
        p.run_split()
    else:
        p.run()
    n2 = p.sync()
    t1 = p.t1.cpu().numpy()
    t2 = p.t2.cpu().numpy()
    off = p.offsets().cpu().numpy()
    torch.cuda.synchronize()
    p.close()
    return t1, t2, n2, off


def oracle_plot(K, key, D=None):
    t1 = orc.table1(K, key)
    t2 = orc.match(key, t1, orc.default_distance(K) if D is None else D)
    return t1, t2


def oracle_plot_global(K, key, D=None):
    t1 = orc.table1(K, key)
    t2 = orc.match_global(key, t1, orc.default_distance(K) if D is None else D)
    return t1, t2


def test_hash_row_matches_oracle(vx):
    key = plot_key(3)
    for nonce0, count in [(0, 5000), (2 ** 32 - 3000, 3000), (123456789, 777), (2 ** 31 - 5, 10)]:
        out = torch.empty(12 * count, dtype=torch.uint8, device="cuda")
        vx.vx_hash_nonces(key, nonce0, count, out.data_ptr())
        got = out.view(count, 12).cpu().numpy()
        ref = orc.hash_range(key, nonce0, nonce0 + count, threads=4)
        assert np.array_equal(got, ref), (nonce0, count)


def test_hash_peak_fold_matches_oracle(vx):
    # The hash-only ceiling kernel hashes what it is asked to: the XOR of its
    # per-thread folds is the XOR of h0 ^ h1 over every nonce, whatever the
    # grid (its 2048-nonce tiles end in a ragged one here).
    key = plot_key(4)
    nonce0, count = 7000, 300001
    ref = orc.hash_range(key, nonce0, nonce0 + count, threads=4)[:, 4:].copy().view("<u4")
    want = int(np.bitwise_xor.reduce(ref[:, 0] ^ ref[:, 1]))
    for blocks in (1, 3, 152):
        fold = torch.zeros(256 * blocks, dtype=torch.int32, device="cuda")
        vx.vx_hash_peak(key, nonce0, count, fold.data_ptr(), 256 * blocks)
        got = int(np.bitwise_xor.reduce(fold.cpu().numpy().view(np.uint32)))
        assert got == want, blocks


def test_pair_hash_row_matches_oracle(vx):
    key = plot_key(4)
    rng = np.random.default_rng(5)
    pairs = rng.integers(0, 2 ** 32, size=(3000, 2), dtype=np.uint64).astype(np.uint32)
    pairs[0] = [0, 0]
    pairs[1] = [0xFFFFFFFF, 0xFFFFFFFF]
    dp = torch.from_numpy(pairs.view(np.int32)).cuda()
    out = torch.empty(3000 * 16, dtype=torch.uint8, device="cuda")
    vx.vx_pair_hash(key, dp.data_ptr(), 3000, out.data_ptr())
    got = out.view(3000, 16).cpu().numpy()
    assert np.array_equal(got[:, :8].view("<u4"), pairs)
    for i in range(3000):
        assert got[i, 8:].tobytes() == orc.keyed_hash(key, got[i, :8].tobytes(), 8), i


STAGED = dict(scatter_mode=1)
DIRECT = dict(scatter_mode=2)
FUSED = dict(fuse_pair_hash=1)
LOOKBACK = dict(t2_placement=1)   # partitions chained by look-back, records at final offsets
SLOTS = dict(t2_placement=2)      # pairs staged in the partition slots, offsets by a scan
# (K, seed, opts) -- sizes from one record to the small configuration;
# opts exercise both bucketing strategies, both scatter levels and the sort
# digit widths.
CASES = [
    (1, 0, {}), (2, 1, {}), (3, 2, {}), (5, 3, {}), (8, 4, {}), (11, 5, {}), (12, 6, {}),
    (13, 7, {}), (14, 8, {}), (16, 9, {}), (18, 10, {}), (20, 11, {}), (22, 0, {}),
    (1, 0, STAGED), (5, 3, STAGED), (12, 6, STAGED), (17, 18, STAGED), (22, 0, STAGED),
    (1, 0, DIRECT), (5, 3, DIRECT), (12, 6, DIRECT), (17, 18, DIRECT), (22, 0, DIRECT),
    (20, 20, dict(DIRECT, partition_log2=6)),
    (1, 0, FUSED), (9, 21, FUSED), (16, 22, FUSED), (22, 0, FUSED),
    # two-stream pipeline forced at sizes the oracle covers
    (20, 24, dict(partition_log2=8, pipeline_chunks=8)),
    (22, 25, dict(pipeline_chunks=8)),
    (21, 26, dict(partition_log2=9, pipeline_chunks=2)),
    (18, 27, dict(DIRECT, partition_log2=7, pipeline_chunks=4)),
    (3, 28, dict(pipeline_chunks=8)),
    (19, 23, dict(FUSED, scatter_mode=2, partition_log2=7)),
    (16, 12, dict(STAGED, partition_log2=6, coarse_bits=4)),   # two levels, 1024 partitions
    (20, 13, dict(STAGED, partition_log2=8)),                  # two levels (auto)
    (12, 15, dict(STAGED, partition_log2=6, coarse_bits=0)),   # single first-level slot
    (17, 16, dict(STAGED, partition_log2=7, coarse_bits=10)),  # 10 + 0 bits
    (18, 14, dict(partition_log2=13)),                         # large partitions, 13-bit digits
    (19, 17, dict(partition_log2=9, slack_sigma=40)),          # roomy slots
    (20, 19, dict(partition_log2=6)),                          # 2^14 tiny partitions
    # the Table-1 hash with 4 and 16 nonces per thread (tiles of 1024 and
    # 4096 nonces; K=11 and 13 end in or fit one ragged tile)
    (11, 40, dict(nonces_per_thread=16)), (13, 41, dict(nonces_per_thread=16)),
    (22, 42, dict(nonces_per_thread=16)), (9, 43, dict(nonces_per_thread=4)),
    (21, 44, dict(nonces_per_thread=4)), (20, 45, dict(nonces_per_thread=16, pipeline_chunks=4)),
    # both Table-2 placements forced (automatic = the pair slots wherever a
    # partition's pairs fit them with a wide margin, as at every K here)
    (1, 0, LOOKBACK), (2, 1, LOOKBACK), (5, 3, LOOKBACK), (12, 6, LOOKBACK), (14, 8, LOOKBACK),
    (16, 9, LOOKBACK), (18, 10, LOOKBACK), (20, 11, LOOKBACK), (22, 0, LOOKBACK),
    (22, 0, dict(STAGED, t2_placement=1)), (20, 19, dict(partition_log2=6, t2_placement=1)),
    (17, 18, dict(DIRECT, t2_placement=1)), (19, 29, dict(partition_log2=13, t2_placement=1)),
    (1, 0, SLOTS), (5, 3, SLOTS), (14, 8, SLOTS), (22, 0, SLOTS),
    (20, 19, dict(partition_log2=6, t2_placement=2)),          # 2^14 groups of 8 partitions
    (11, 30, dict(partition_log2=6, t2_placement=2)),          # 32 partitions: a ragged last group
    (18, 14, dict(partition_log2=13, t2_placement=2)),
    (17, 31, dict(DIRECT, t2_placement=2)),
]


@pytest.mark.parametrize("split", [False, True], ids=["fused", "split"])
@pytest.mark.parametrize("K,seed,kw", CASES)
def test_plot_matches_oracle(vx, K, seed, kw, split):
    key = plot_key(seed)
    opts = vx.make_opts(**kw) if kw else None
    t1, t2, n2, off = run_plot(vx, K, key, opts, split)
    r1, r2 = oracle_plot(K, key)
    assert np.array_equal(t1, r1)
    assert n2 == r2.shape[0]
    assert np.array_equal(t2, r2)
    assert np.array_equal(off.astype(np.uint64), orc.bucket_offsets(r1))


# Cross-bucket match (every pair of the whole Table-1 order under D): the
# halo of the next partition joins each partition's pair scan.
GLOBAL_CASES = [
    (1, 0, {}), (5, 3, {}), (11, 5, {}), (12, 6, {}), (14, 8, {}), (16, 9, {}), (20, 11, {}),
    (22, 0, {}), (22, 0, DIRECT), (17, 18, STAGED), (19, 32, dict(partition_log2=7)),
    (16, 12, dict(STAGED, partition_log2=6, coarse_bits=4)),   # two levels, 1024 partitions
    (20, 24, dict(partition_log2=8, pipeline_chunks=8)),
    (16, 22, FUSED), (14, 8, SLOTS), (20, 19, dict(partition_log2=6, t2_placement=2)),
    (16, 20, dict(match_distance=1 << 44)),                    # fewer pairs than records
    (14, 31, dict(match_distance=1 << 52)),                    # ~4 halo records per partition
    (18, 33, dict(partition_log2=6, match_distance=1 << 49)),  # ~8 per partition, 4096 of them
]


@pytest.mark.parametrize("split", [False, True], ids=["fused", "split"])
@pytest.mark.parametrize("K,seed,kw", GLOBAL_CASES)
def test_cross_bucket_match_matches_oracle(vx, K, seed, kw, split):
    key = plot_key(seed)
    t1, t2, n2, _ = run_plot(vx, K, key, vx.make_opts(match_scope=1, **kw), split)
    r1, r2 = oracle_plot_global(K, key, kw.get("match_distance"))
    assert np.array_equal(t1, r1)
    assert n2 == r2.shape[0]
    assert np.array_equal(t2, r2)


def test_cross_bucket_halo_overflow_is_reported(vx):
    # 4096 partitions of ~64 records, D one partition wide: halos of ~64
    # records against 64 + 1 sd + 16 places; some overflow, and the plot must
    # say so (VX_EOVERFLOW naming the halo), never drop pairs silently.
    p = vx.Plot(18, plot_key(34), vx.make_opts(match_scope=1, partition_log2=6, slack_sigma=1,
                                               match_distance=1 << 52))
    p.run()
    assert vx.vx_sync(p.handle, check=False) == vx.VX_EOVERFLOW
    assert "halo" in vx.last_error(p.handle)
    p.close()


@pytest.mark.parametrize("split", [False, True], ids=["fused", "split"])
@pytest.mark.parametrize("K,seed,D", [(16, 20, 1 << 34), (18, 21, 1 << 37), (14, 22, 1),
                                      (15, 23, (1 << 64) - 1), (17, 24, 12345678901)])
def test_custom_match_distance(vx, K, seed, D, split):
    key = plot_key(seed)
    t1, t2, n2, _ = run_plot(vx, K, key, vx.make_opts(match_distance=D), split)
    r1, r2 = oracle_plot(K, key, D)
    assert np.array_equal(t1, r1)
    assert np.array_equal(t2, r2)


def test_dense_buckets_match(vx):
    # K=22 with D spanning all buckets is the K <= 24 all-pairs regime;
    # a D of 1/8 bucket mimics the K=27 density on a small plot.
    key = plot_key(30)
    D = 1 << 37
    t1, t2, _, _ = run_plot(vx, 22, key, vx.make_opts(match_distance=D))
    r1, r2 = oracle_plot(22, key, D)
    assert np.array_equal(t2, r2)


def test_deterministic_repeat(vx):
    key = plot_key(40)
    p = vx.Plot(20, key)
    outs = []
    for _ in range(3):
        p.run()
        p.sync()
        outs.append((p.t1.cpu().numpy().copy(), p.t2.cpu().numpy().copy()))
    p.close()
    for a in outs[1:]:
        assert np.array_equal(a[0], outs[0][0]) and np.array_equal(a[1], outs[0][1])


@pytest.mark.parametrize("placement", [1, 2], ids=["lookback", "slots"])
@pytest.mark.parametrize("K,seed,D", [(16, 20, 1 << 34), (15, 23, (1 << 64) - 1)])
def test_custom_match_distance_both_placements(vx, K, seed, D, placement):
    key = plot_key(seed)
    t1, t2, n2, _ = run_plot(vx, K, key, vx.make_opts(match_distance=D, t2_placement=placement))
    r1, r2 = oracle_plot(K, key, D)
    assert np.array_equal(t2, r2)


def test_pair_slot_overflow_is_reported(vx):
    # K=26 with every pair of a logical bucket matching: ~4096 pairs per
    # partition, more than a pair slot (1.5 x 2607) holds.  Forced slots
    # must fail with VX_EOVERFLOW; the look-back placement (automatic here:
    # the slots would not hold the expected pairs) agrees with the split
    # path, which places pairs by a plain scan.
    K, key, D = 26, plot_key(65), (1 << 64) - 1
    p = vx.Plot(K, key, vx.make_opts(match_distance=D, t2_placement=2))
    p.run()
    assert vx.vx_sync(p.handle, check=False) == vx.VX_EOVERFLOW
    assert "pair slot" in vx.last_error(p.handle)
    p.close()
    p = vx.Plot(K, key, vx.make_opts(match_distance=D))
    assert vx.vx_plot_kernel_mask(p.handle)[-2:] == ["sortmatch", "pairhash"]
    assert "scan_pairs" not in vx.vx_plot_kernel_mask(p.handle)
    p.run()
    n_auto = p.sync()
    t2_auto = p.t2.cpu().numpy()
    p.run_split()
    n_split = p.sync()
    assert n_auto == n_split > 2 ** 26
    assert np.array_equal(t2_auto, p.t2.cpu().numpy())
    p.close()


@pytest.mark.parametrize("mode", [1, 2], ids=["staged", "direct"])
def test_slot_overflow_is_reported(vx, mode):
    # Slots of mean + 1 sd (+16) overflow in many partitions: the plot must
    # report VX_EOVERFLOW, never produce silently short tables or fault.
    key = plot_key(50)
    p = vx.Plot(18, key, vx.make_opts(partition_log2=6, slack_sigma=1, scatter_mode=mode))
    p.run()
    rc = vx.vx_sync(p.handle, check=False)
    assert rc == vx.VX_EOVERFLOW
    p.close()


@pytest.mark.parametrize("split", [False, True], ids=["fused", "split"])
def test_table2_capacity_then_rebind(vx, split):
    key = plot_key(60)
    K = 16
    p = vx.Plot(K, key, vx.make_opts(t2_capacity=16))
    p.run_split() if split else p.run()
    assert vx.vx_sync(p.handle, check=False) == vx.VX_ENOMEM
    _, need, _, rc = vx.vx_table_info(p.handle, vx.VX_TABLE2, check=False)
    assert rc == vx.VX_ENOMEM
    r1, r2 = oracle_plot(K, key)
    assert need == r2.shape[0] > 16
    # A bigger Table-2 buffer, same Table 1 and scratch: only vx_match reruns.
    big = torch.empty(16 * need + 256, dtype=torch.uint8, device="cuda")
    vx.vx_plot_bind(p.handle, p._t1.data_ptr(), big.data_ptr(), p._scratch.data_ptr(), need)
    vx.vx_match(p.handle)
    vx.vx_sync(p.handle)
    got = big[: 16 * need].view(need, 16).cpu().numpy()
    assert np.array_equal(got, r2)
    p.close()


def test_sync_reads_its_own_plot_when_buffers_are_reused(vx):
    # Two plots on one stream share Table 1 and scratch, each with its own
    # Table 2: vx_sync on the first, issued after both, must report the first
    # plot's count (not the second's, whose kernels overwrote the scratch),
    # and both Table 2 buffers must hold their own plot.
    K = 16
    ka, kb = plot_key(63), plot_key(64)
    t1b, t2b, scb = vx.vx_plot_required_bytes(K)
    t1 = torch.empty(t1b, dtype=torch.uint8, device="cuda")
    sc = torch.empty(scb, dtype=torch.uint8, device="cuda")
    t2 = [torch.empty(t2b, dtype=torch.uint8, device="cuda") for _ in range(2)]
    hs = []
    for key, buf in [(ka, t2[0]), (kb, t2[1])]:
        h = vx.vx_plot_create(K, key)
        vx.vx_plot_bind(h, t1.data_ptr(), buf.data_ptr(), sc.data_ptr(), t2b // 16)
        vx.vx_plot_run(h)
        hs.append(h)
    refs = [oracle_plot(K, ka)[1], oracle_plot(K, kb)[1]]
    assert refs[0].shape[0] != refs[1].shape[0]
    for h, buf, r2 in zip(hs, t2, refs):
        vx.vx_sync(h)
        _, n2, _, _ = vx.vx_table_info(h, vx.VX_TABLE2)
        assert n2 == r2.shape[0]
        assert np.array_equal(buf[: 16 * n2].view(n2, 16).cpu().numpy(), r2)
    for h in hs:
        vx.vx_plot_destroy(h)


@pytest.mark.parametrize("K,s,placement", [(16, 8, 1), (20, 6, 2)], ids=["lookback", "slots"])
def test_lookback_wait_times_out(vx, K, s, placement):
    # Partition 0 (look-back placement) or chunk 0 of the pair-count scan
    # (slot placement: 2^14 partitions = 4 scan chunks) withholds its
    # Table-2 prefix: every later wait must run out (bounded), the plot must
    # report VX_ETIMEDOUT, and the context must stay usable for the next plot.
    p = vx.Plot(K, plot_key(61), vx.make_opts(partition_log2=s, t2_placement=placement,
                                               test_flags=vx.VX_TEST_WITHHOLD_PREFIX))
    assert ("scan_pairs" in vx.vx_plot_kernel_mask(p.handle)) == (placement == 2)
    p.run()
    assert vx.vx_sync(p.handle, check=False) == vx.VX_ETIMEDOUT
    p.close()
    t1, t2, n2, _ = run_plot(vx, 14, plot_key(62))
    r1, r2 = oracle_plot(14, plot_key(62))
    assert np.array_equal(t2, r2)


def test_alloc_failure_injection(vx):
    h = vx.vx_plot_create(16, plot_key(1))
    vx.vx_test_fail_next_allocs(1)
    with pytest.raises(vx.VxError) as ei:
        vx.vx_plot_alloc(h)
    assert ei.value.code == vx.VX_ENOMEM
    vx.vx_plot_alloc(h)      # the next one succeeds
    vx.vx_table1(h)
    vx.vx_match(h)
    vx.vx_sync(h)
    vx.vx_plot_destroy(h)


def test_library_owned_memory_and_copy(vx):
    K, key = 15, plot_key(70)
    h = vx.vx_plot_create(K, key)
    vx.vx_table1(h)
    vx.vx_match(h)
    vx.vx_sync(h)
    _, n2, rb, _ = vx.vx_table_info(h, vx.VX_TABLE2)
    host = torch.empty(n2 * 16, dtype=torch.uint8).pin_memory()
    vx.vx_table_copy(h, vx.VX_TABLE2, host.data_ptr(), n2 * 16)
    torch.cuda.synchronize()
    r1, r2 = oracle_plot(K, key)
    assert np.array_equal(host.numpy().reshape(-1, 16), r2)
    vx.vx_plot_destroy(h)


def test_plot_write_file(vx, tmp_path):
    K, key = 17, plot_key(80)
    p = vx.Plot(K, key)
    p.run()
    p.sync()
    path = str(tmp_path / "plot.bin")
    d2h, total = vx.vx_plot_write(p.handle, path)
    data = np.fromfile(path, dtype=np.uint8).reshape(-1, 16)
    # The file is Table 2 in its order, no header (R12): the oracle's table.
    _, r2 = oracle_plot(K, key)
    assert np.array_equal(data, r2)
    assert np.array_equal(data, p.t2.cpu().numpy())
    assert total >= d2h >= 0
    p.close()


def test_profile_trace(vx):
    p = vx.Plot(20, plot_key(90))
    vx.vx_plot_profile(p.handle, 3)
    p.run()
    p.run_split()
    p.run()
    p.sync()
    ms, runs = vx.vx_plot_profile_read(p.handle)
    assert runs == 3
    assert set(ms) == {"key_setup", "hash_staged", "hash_direct", "scatter2", "scan_counts",
                       "sort", "scan_pairs", "match", "sortmatch", "pairhash"}
    assert ms["hash_staged"] > 0 and ms["sortmatch"] > 0 and ms["sort"] > 0 and ms["match"] > 0
    assert ms["pairhash"] > 0
    assert vx.vx_plot_kernel_mask(p.handle) == ["key_setup", "hash_staged", "scan_counts",
                                                "scan_pairs", "sortmatch", "pairhash"]
    assert vx.vx_plot_kernel_mask(p.handle, split=True) == [
        "key_setup", "hash_staged", "scan_counts", "sort", "scan_pairs", "match"]
    p.close()


def test_split_and_fused_agree_mid_size(vx):
    # K=24 (no oracle at this size in the fast suite): both paths and both
    # bucketing strategies give identical bytes.
    key = plot_key(91)
    outs = []
    for kw, split in [({}, False), ({}, True), (DIRECT, False), (dict(partition_log2=12), False),
                      (FUSED, False), (dict(pipeline_chunks=1), False),
                      (dict(pipeline_chunks=2), False)]:
        p = vx.Plot(24, key, vx.make_opts(**kw) if kw else None)
        p.run_split() if split else p.run()
        p.sync()
        outs.append((p.t1.clone(), p.t2.clone()))
        p.close()
    for t1, t2 in outs[1:]:
        assert torch.equal(t1, outs[0][0]) and torch.equal(t2, outs[0][1])
