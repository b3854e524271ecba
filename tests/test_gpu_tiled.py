"""Windowed plots and chunked device-memory tiling vs the CPU oracle.

A window (vx_opts.window_bits = c, window = w) keeps the records whose key64
has top c bits == w: 2^(24-c) consecutive logical buckets.  A window plot of
its own hashes every nonce and filters; vx_plot_tiled stores every nonce's
window in a first pass and lets each window hash only its listed nonces
(up to 8 window bits, hash in one nonce chunk).  The bucket-scope
match never leaves a bucket, so a window's tables must equal the oracle's
whole-plot tables restricted to those buckets, and vx_plot_tiled's host
tables (all windows, in order) must equal the whole plot's, bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_2606_14007_gb300.inputs import plot_key  # noqa: E402
from window_slices import oracle_windows  # noqa: E402


@pytest.fixture(scope="module")
def vx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_14007_gb300 import vaultx
    assert torch.cuda.is_available()
    return vaultx


def oracle_tables(K, key, D=None):
    r1 = orc.table1(K, key)
    r2 = orc.match(key, r1, orc.default_distance(K) if D is None else D)
    return r1, r2


STAGED = dict(scatter_mode=1)
DIRECT = dict(scatter_mode=2)
# (K, seed, window bits, opts): one and several partitions per window, one
# and two scatter levels, both bucketing strategies, both Table-2
# placements, the fused pair hash, nonce chunks, a custom match distance.
WIN_CASES = [
    (12, 50, 1, dict(partition_log2=6)),
    (12, 51, 6, dict(partition_log2=6)),                       # one partition per window
    (16, 52, 2, {}),
    (16, 53, 3, dict(STAGED, partition_log2=6, coarse_bits=4)),  # 4 + 3 bits per window
    (22, 55, 2, dict(partition_log2=6)),                       # two levels of 7 bits
    (20, 56, 3, DIRECT),
    (18, 57, 2, dict(fuse_pair_hash=1)),
    (18, 58, 2, dict(t2_placement=2)),
    (18, 63, 2, dict(t2_placement=1)),
    (22, 64, 3, dict(partition_log2=6, t2_placement=1)),
    (20, 59, 1, dict(pipeline_chunks=4, partition_log2=8)),    # 4 nonce chunks, two levels
    (22, 60, 4, {}),
    (17, 61, 2, dict(match_distance=1 << 45)),
    (14, 62, 3, dict(partition_log2=6, t2_placement=2, scatter_mode=2)),
]


@pytest.mark.parametrize("split", [False, True], ids=["fused", "split"])
@pytest.mark.parametrize("K,seed,c,kw", WIN_CASES)
def test_windows_are_oracle_slices(vx, K, seed, c, kw, split):
    key = plot_key(seed)
    r1, r2 = oracle_tables(K, key, kw.get("match_distance"))
    off = orc.bucket_offsets(r1).astype(np.int64)
    for w, (s1, s2) in enumerate(oracle_windows(r1, r2, c)):
        p = vx.Plot(K, key, vx.make_opts(window_bits=c, window=w, **kw))
        if split:
            p.run_split()
        else:
            p.run()
        n2 = p.sync()
        assert p.n1 == s1.shape[0] and n2 == s2.shape[0], (w, p.n1, n2)
        assert np.array_equal(p.t1.cpu().numpy(), s1), w
        assert np.array_equal(p.t2.cpu().numpy(), s2), w
        # bucket offsets: relative to the window's first bucket, clipped to it
        w0 = w << (24 - c)
        want = np.clip(off - off[w0], 0, s1.shape[0])
        got = p.offsets().cpu().numpy()
        assert np.array_equal(got, want), w
        p.close()


TILED_CASES = [
    (16, 70, 0, {}),                                           # one window: the whole plot
    (16, 71, 1, {}),
    (20, 72, 2, {}),
    (22, 73, 3, {}),
    (22, 74, 2, dict(partition_log2=6)),
    (18, 75, 4, DIRECT),
    (19, 76, 2, dict(t2_placement=2)),
    (19, 77, 3, dict(fuse_pair_hash=1)),
    (13, 78, 7, dict(partition_log2=6)),                       # 128 windows of one partition
    # windows that hash every nonce and filter (no window-id pass): the hash
    # split into nonce chunks, and more than 8 window bits
    (20, 83, 2, dict(pipeline_chunks=4, partition_log2=8)),
    (16, 84, 9, dict(partition_log2=6)),
]


@pytest.mark.parametrize("K,seed,c,kw", TILED_CASES)
def test_tiled_plot_equals_oracle(vx, K, seed, c, kw):
    key = plot_key(seed)
    t1, t2 = vx.plot_tiled(K, key, c, vx.make_opts(**kw) if kw else None)
    r1, r2 = oracle_tables(K, key)
    assert np.array_equal(t1.numpy(), r1)
    assert np.array_equal(t2.numpy(), r2)


def test_tiled_plot_pageable_host_memory(vx):
    key = plot_key(79)
    t1, t2 = vx.plot_tiled(18, key, 2, pin=False)
    r1, r2 = oracle_tables(18, key)
    assert np.array_equal(t1.numpy(), r1)
    assert np.array_equal(t2.numpy(), r2)


def test_tiled_plot_table2_only(vx):
    key = plot_key(80)
    t1, t2 = vx.plot_tiled(20, key, 2, table1=False)
    assert t1 is None
    _, r2 = oracle_tables(20, key)
    assert np.array_equal(t2.numpy(), r2)


def test_tiled_plot_small_table2_buffer(vx):
    # Table 2 does not fit: VX_ENOMEM, the count needed, Table 1 complete.
    K, key = 18, plot_key(81)
    r1, r2 = oracle_tables(K, key)
    h1 = torch.empty(12 << K, dtype=torch.uint8, pin_memory=True)
    small = 16 * (r2.shape[0] // 2)
    h2 = torch.empty(small, dtype=torch.uint8, pin_memory=True)
    rc, n1, n2 = vx.vx_plot_tiled(K, key, 2, h1.data_ptr(), h1.numel(), h2.data_ptr(), small,
                                  check=False)
    assert rc == vx.VX_ENOMEM
    assert n1 == 1 << K and n2 == r2.shape[0]
    assert np.array_equal(h1.view(-1, 12).numpy(), r1)


def test_tiled_plot_rejects_bad_arguments(vx):
    key = plot_key(82)
    h1 = torch.empty(12 << 14, dtype=torch.uint8)
    h2 = torch.empty(1 << 20, dtype=torch.uint8)
    # window bits above the partition bits (K=14: 3 bits with 2^11-record partitions)
    rc, _, _ = vx.vx_plot_tiled(14, key, 4, h1.data_ptr(), h1.numel(), h2.data_ptr(), h2.numel(),
                                check=False)
    assert rc == vx.VX_EINVAL
    # opts that already name a window
    rc, _, _ = vx.vx_plot_tiled(14, key, 2, h1.data_ptr(), h1.numel(), h2.data_ptr(), h2.numel(),
                                vx.make_opts(window_bits=1), check=False)
    assert rc == vx.VX_EINVAL
    # a Table-1 buffer shorter than 12 * 2^K
    rc, _, _ = vx.vx_plot_tiled(14, key, 2, h1.data_ptr(), h1.numel() - 12, h2.data_ptr(),
                                h2.numel(), check=False)
    assert rc == vx.VX_EINVAL


def test_batch_with_windows_and_whole_plots(vx):
    # One batch launch mixing windows, whole plots and a cross-bucket plot
    # (the window filter and the halo code in one kernel instance): each
    # member equals its oracle slice.
    mix = [(16, 90, 2, 1, {}), (18, 91, 0, 0, {}), (14, 92, 0, 0, dict(match_scope=1)),
           (16, 90, 2, 3, {}), (20, 93, 3, 5, dict(partition_log2=8)), (12, 94, 6, 63, dict(partition_log2=6))]
    plots = [vx.Plot(K, plot_key(s), vx.make_opts(window_bits=c, window=w, **kw)) for K, s, c, w, kw in mix]
    for rep in range(2):  # the second launch replays the recorded graph
        vx.vx_plot_batch([p.handle for p in plots])
        for (K, s, c, w, kw), p in zip(mix, plots):
            p.sync()
            key = plot_key(s)
            if kw.get("match_scope"):
                r1 = orc.table1(K, key)
                r2 = orc.match_global(key, r1, orc.default_distance(K))
                s1, s2 = r1, r2
            else:
                r1, r2 = oracle_tables(K, key)
                s1, s2 = oracle_windows(r1, r2, c)[w] if c else (r1, r2)
            assert np.array_equal(p.t1.cpu().numpy(), s1), (rep, K, c, w)
            assert np.array_equal(p.t2.cpu().numpy(), s2), (rep, K, c, w)
    for p in plots:
        p.close()


def test_window_table1_count_needs_sync(vx):
    # A window's record count is random: the Table-1 view waits for vx_sync.
    p = vx.Plot(16, plot_key(95), vx.make_opts(window_bits=2, window=1))
    p.table1()
    _, _, _, rc = vx.vx_table_info(p.handle, vx.VX_TABLE1, check=False)
    assert rc == vx.VX_ENOTREADY
    vx.vx_sync(p.handle)
    _, n1, rb, rc = vx.vx_table_info(p.handle, vx.VX_TABLE1, check=False)
    assert rc == vx.VX_OK and rb == 12 and 0 < n1 < (1 << 16)
    p.close()


@pytest.mark.parametrize("K,seed,c", [(16, 85, 0), (18, 86, 2), (20, 87, 3), (14, 88, 5)])
def test_tiled_plot_file_equals_oracle(vx, tmp_path, K, seed, c):
    # Table 2 streamed window by window into a flat plot file; Table 1 into
    # pinned host memory.
    key = plot_key(seed)
    path = str(tmp_path / "plot.bin")
    h1 = torch.empty(12 << K, dtype=torch.uint8, pin_memory=True)
    opts = vx.make_opts(partition_log2=6) if c > K - 11 else None
    rc, n1, n2, sec = vx.vx_plot_tiled_write(K, key, c, path, h1.data_ptr(), h1.numel(), opts)
    r1, r2 = oracle_tables(K, key)
    data = np.fromfile(path, dtype=np.uint8)
    assert n1 == 1 << K and n2 == r2.shape[0] and data.size == 16 * n2 and sec > 0
    assert np.array_equal(data.reshape(-1, 16), r2)
    assert np.array_equal(h1.view(-1, 12).numpy(), r1)


def test_tiled_plot_file_equals_whole_plot_file(vx, tmp_path):
    # the bytes vx_plot_write gives for the whole plot
    K, key = 20, plot_key(89)
    a, b = str(tmp_path / "whole.bin"), str(tmp_path / "tiled.bin")
    p = vx.Plot(K, key)
    p.run()
    p.sync()
    vx.vx_plot_write(p.handle, a)
    p.close()
    vx.vx_plot_tiled_write(K, key, 3, b)
    assert open(a, "rb").read() == open(b, "rb").read()


def test_tiled_plot_file_bad_path(vx, tmp_path):
    rc, _, _, _ = vx.vx_plot_tiled_write(16, plot_key(90), 2, str(tmp_path / "no" / "such" / "dir.bin"),
                                         check=False)
    assert rc == vx.VX_EIO  # the file cannot be opened: an I/O error, before any device work


def test_tiled_plots_in_a_caller_work_buffer(vx, tmp_path):
    # Window buffers cut from one caller-owned device buffer, reused by
    # consecutive plots (host memory, then a plot file).
    K, c = 20, 2
    dev_bytes, _, _ = vx.vx_plot_tiled_bytes(K, c)
    work = torch.empty(dev_bytes, dtype=torch.uint8, device="cuda")
    for seed in (96, 97):
        key = plot_key(seed)
        t1, t2 = vx.plot_tiled(K, key, c, work=work)
        r1, r2 = oracle_tables(K, key)
        assert np.array_equal(t1.numpy(), r1) and np.array_equal(t2.numpy(), r2), seed
    path = str(tmp_path / "plot.bin")
    vx.vx_plot_tiled_write(K, plot_key(98), c, path, d_work=work.data_ptr(), work_bytes=work.numel())
    _, r2 = oracle_tables(K, plot_key(98))
    assert np.array_equal(np.fromfile(path, dtype=np.uint8).reshape(-1, 16), r2)


def test_tiled_work_buffer_checks(vx):
    K, c = 18, 2
    dev_bytes, h1b, h2b = vx.vx_plot_tiled_bytes(K, c)
    work = torch.empty(dev_bytes + 256, dtype=torch.uint8, device="cuda")
    h1 = torch.empty(h1b, dtype=torch.uint8)
    h2 = torch.empty(h2b, dtype=torch.uint8)
    key = plot_key(99)
    for ptr, nb in [(work.data_ptr(), dev_bytes - 256),        # too small
                    (work.data_ptr() + 128, dev_bytes)]:      # not 256-byte aligned
        rc, _, _ = vx.vx_plot_tiled(K, key, c, h1.data_ptr(), h1b, h2.data_ptr(), h2b, check=False,
                                    d_work=ptr, work_bytes=nb)
        assert rc == vx.VX_EINVAL
