"""C ABI checks that need no GPU: the library builds and loads, exports every
symbol include/vaultx.h declares, and its host logic (planner, argument
validation, call-order errors) behaves.  No compute call is made here."""
import ctypes
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vaultx.h")


@pytest.fixture(scope="module")
def vx():
    from paper_2606_14007_gb300 import _build
    _build.build()
    from paper_2606_14007_gb300 import vaultx
    vaultx.lib()
    return vaultx


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vx_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_boundary_calls():
    names = declared_symbols()
    for must in ["vx_plot_create", "vx_table1", "vx_match", "vx_plot_batch", "vx_serve_submit",
                 "vx_serve_poll", "vx_plot_required_bytes", "vx_plot_bind", "vx_table_info",
                 "vx_table1_offsets", "vx_table_copy", "vx_plot_write", "vx_plot_destroy",
                 "vx_sync", "vx_strerror", "vx_hash_nonces", "vx_pair_hash"]:
        assert must in names


def test_library_exports_every_declared_symbol(vx):
    out = subprocess.run(["nm", "-D", "--defined-only", vx.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vx_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    L = vx.lib()
    for n in declared_symbols():
        assert getattr(L, n) is not None


def test_library_is_sm103a_only():
    from paper_2606_14007_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_strerror_and_version(vx):
    assert vx.strerror(0) == "ok"
    assert "overflow" in vx.strerror(vx.VX_EOVERFLOW)
    assert "I/O" in vx.strerror(vx.VX_EIO)
    assert vx.lib().vx_version() >> 16 == 1


def test_required_bytes_footprints(vx):
    for K in range(1, 33):
        t1, t2, sc = vx.vx_plot_required_bytes(K)
        N = 1 << K
        assert t1 >= 12 * N and t1 % 256 == 0
        lam = N / 2 ** 24
        E = 2 ** 24 * lam * lam / 2 * (1.0 if K <= 24 else (2 / lam - 1 / lam ** 2))
        assert t2 >= 16 * E
        assert sc > 0 and sc % 256 == 0
    # K = 31: tables at their record sizes; scratch holds the partition slots
    # (12 B per record plus the slot slack) and megabytes of counters.
    t1, t2, sc = vx.vx_plot_required_bytes(31)
    assert t1 < 1.05 * 12 * 2 ** 31
    assert t2 < 1.05 * 16 * 2 ** 31
    assert 12 * 2 ** 31 < sc < 1.4 * 12 * 2 ** 31


def test_required_bytes_rejects_bad_arguments(vx):
    for K in [0, -1, 33, 64]:
        with pytest.raises(vx.VxError) as ei:
            vx.vx_plot_required_bytes(K)
        assert ei.value.code == vx.VX_EINVAL
    for kw in [dict(partition_log2=5), dict(partition_log2=14),
               dict(coarse_bits=11, scatter_mode=1), dict(scatter_mode=3),
               dict(slack_sigma=400, partition_log2=12), dict(t2_placement=3),
               dict(t2_placement=2, pipeline_chunks=2), dict(t2_placement=2, fuse_pair_hash=1),
               dict(hash_block=128), dict(nonces_per_thread=6), dict(nonces_per_thread=32),
               dict(nonces_per_thread=4, scatter_mode=2),           # direct: 8 only
               dict(nonces_per_thread=16, window_bits=2, window=1),  # windows: 8 only
               dict(match_scope=2),
               dict(match_scope=1, match_distance=1 << 60),        # wider than a partition
               dict(match_scope=1, match_distance=1 << 43)]:       # halo of ~1024 records
        with pytest.raises(vx.VxError):
            vx.vx_plot_required_bytes(31, vx.make_opts(**kw))
    vx.vx_plot_required_bytes(31, vx.make_opts(hash_block=256, nonces_per_thread=8))
    for npt in (4, 16):  # the staged Table-1 hash's other shapes
        vx.vx_plot_required_bytes(31, vx.make_opts(nonces_per_thread=npt, scatter_mode=1))
    bad = vx.make_opts()
    bad.size = 8
    with pytest.raises(vx.VxError):
        vx.vx_plot_required_bytes(20, bad)


def test_create_and_destroy_without_device(vx):
    key = bytes(range(32))
    h = vx.vx_plot_create(20, key)
    assert h
    # Call-order errors are reported, not crashed on.
    _, _, _, rc = vx.vx_table_info(h, vx.VX_TABLE1, check=False)
    assert rc == vx.VX_ENOTREADY
    assert vx.lib().vx_match(h, None) == vx.VX_ENOTREADY
    assert vx.lib().vx_sync(h) == vx.VX_ENOTREADY
    vx.vx_plot_destroy(h)
    with pytest.raises(ValueError):
        vx.vx_plot_create(20, b"short")
    assert vx.lib().vx_plot_create(40, key, None, ctypes.byref(ctypes.c_void_p())) == vx.VX_EINVAL


def test_kernel_mask_follows_plan(vx):
    slots = ["key_setup", "hash_staged", "scatter2", "scan_counts", "scan_pairs", "sortmatch",
             "pairhash"]
    lookback = ["key_setup", "hash_staged", "scatter2", "scan_counts", "sortmatch", "pairhash"]
    h = vx.vx_plot_create(31, bytes(32), vx.make_opts(t2_placement=1))
    assert vx.vx_plot_kernel_mask(h) == lookback
    vx.vx_plot_destroy(h)
    h = vx.vx_plot_create(31, bytes(32), vx.make_opts(t2_placement=2))
    assert vx.vx_plot_kernel_mask(h) == slots
    vx.vx_plot_destroy(h)
    # automatic: the pair slots while a partition's expected pairs fit them
    # with a wide margin, the look-back otherwise (dense matching, the fused
    # pair hash, partition chunks)
    for K, kw, want in [(31, {}, slots), (22, {}, slots), (27, dict(match_scope=1), slots),
                        (27, dict(match_distance=1 << 40), lookback),
                        (24, dict(pipeline_chunks=2), lookback)]:
        h = vx.vx_plot_create(K, bytes(32), vx.make_opts(**kw) if kw else None)
        assert vx.vx_plot_kernel_mask(h) == want, (K, kw)
        vx.vx_plot_destroy(h)
    h = vx.vx_plot_create(20, bytes(32), vx.make_opts(scatter_mode=2, fuse_pair_hash=1))
    assert vx.vx_plot_kernel_mask(h) == ["key_setup", "hash_direct", "scan_counts", "sortmatch"]
    vx.vx_plot_destroy(h)


def test_bind_rejects_misaligned(vx):
    h = vx.vx_plot_create(12, bytes(32))
    assert vx.lib().vx_plot_bind(h, 0x1000 + 8, 0x2000, 0x3000, 0) == vx.VX_EINVAL
    assert vx.lib().vx_plot_bind(h, None, 0x2000, 0x3000, 0) == vx.VX_EINVAL
    vx.vx_plot_destroy(h)


def test_partition_plan_shape(vx):
    # More partitions as K grows; single level while partitions fit one
    # scatter level; a slot must hold the mean plus the slack.
    prev = None
    for K in [12, 16, 22, 24, 27, 31, 32]:
        t1, t2, sc = vx.vx_plot_required_bytes(K)
        if prev:
            assert sc >= prev
        prev = sc
    o = vx.make_opts(partition_log2=12)
    t1a, _, _ = vx.vx_plot_required_bytes(31, o)
    t1b, _, _ = vx.vx_plot_required_bytes(31)
    assert t1a >= 12 * 2 ** 31 and t1b >= 12 * 2 ** 31


def test_cross_bucket_scope_plans_a_halo(vx):
    # The cross-bucket match keeps, per partition, the next partition's
    # records within D of its edge: mean 2^11 D / 2^(64-p) = 1 at the
    # default D, so the halo arrays are small beside the partition slots.
    _, _, sb = vx.vx_plot_required_bytes(31)
    _, t2g, sg = vx.vx_plot_required_bytes(31, vx.make_opts(match_scope=1))
    assert sb < sg < sb * 1.03
    assert t2g >= 16 * 2 ** 31  # E|T2| = N for the cross-bucket match
    h = vx.vx_plot_create(31, bytes(32), vx.make_opts(match_scope=1))
    assert vx.vx_plot_kernel_mask(h) == ["key_setup", "hash_staged", "scatter2", "scan_counts",
                                         "scan_pairs", "sortmatch", "pairhash"]
    vx.vx_plot_destroy(h)


def test_planner_sweep_plans_or_rejects_cleanly(vx):
    # Every K and a grid of option combinations: the planner either returns
    # footprints that hold the tables (12 B per nonce; 16 B per expected
    # pair, within the 24-sigma margin) or refuses with VX_EINVAL -- never
    # another code, never a crash.
    import itertools
    planned = rejected = 0
    for K in range(1, 33):
        N = 1 << K
        for s, mode, scope, place, pc in itertools.product(
                (0, 6, 9, 11, 13), (0, 1, 2), (0, 1), (0, 1, 2), (0, 2, 8)):
            o = vx.make_opts(partition_log2=s, scatter_mode=mode, match_scope=scope,
                             t2_placement=place, pipeline_chunks=pc)
            try:
                t1, t2, sc = vx.vx_plot_required_bytes(K, o)
            except vx.VxError as e:
                assert e.code == vx.VX_EINVAL, (K, s, mode, scope, place, pc, e.code)
                rejected += 1
                continue
            planned += 1
            assert t1 >= 12 * N and t1 % 256 == 0 and t2 % 256 == 0 and sc % 256 == 0
            if scope:
                E = N * (N - 1) / 2 * (2 * 2.0 ** (64 - K) / 2 ** 64)
            else:
                lam = N / 2 ** 24
                u = min(1.0, 2.0 ** (64 - K) / 2 ** 40)
                E = 2 ** 24 * lam * lam / 2 * (2 * u - u * u)
            assert t2 >= 16 * E, (K, s, scope, t2, E)
    assert planned > 5000 and rejected > 0


def test_window_plans_shrink_and_reject_cleanly(vx):
    # A window of c bits keeps ~2^-c of the records: its buffers shrink by
    # about that factor (Table 1 is sized for the most its partition slots
    # can hold, so a little less), and two of them (vx_plot_tiled) fit in
    # about 2^(1-c) of the whole plot's footprint.
    whole = sum(vx.vx_plot_required_bytes(31))
    E = 2 ** 24 * (2 ** 7 - 0.5)  # expected Table-2 records at K=31
    for c in (1, 2, 3, 4, 8):
        parts = vx.vx_plot_required_bytes(31, vx.make_opts(window_bits=c, window=(1 << c) - 1))
        t1, t2, sc = parts
        assert t1 >= 12 * 2 ** 31 / 2 ** c and t2 >= 16 * E / 2 ** c
        assert sum(parts) < 1.25 * whole / 2 ** c + (64 << 20), (c, sum(parts), whole)
        dev, h1, h2 = vx.vx_plot_tiled_bytes(31, c)
        assert dev == 2 * sum(parts) + 2 ** 31  # + one window-id byte per nonce
        assert h1 == 12 * 2 ** 31 and h2 >= 16 * E
    # c = 0 is the whole plot, one buffer
    assert vx.vx_plot_tiled_bytes(31, 0)[0] == whole
    # K=32 in two windows of ~1/4 of its footprint each
    assert vx.vx_plot_tiled_bytes(32, 2)[0] < 0.6 * sum(vx.vx_plot_required_bytes(32))
    bad = [dict(window_bits=21, window=0),                # more bits than the 20 partition bits of K=31
           dict(window_bits=17, window=0, partition_log2=6),  # above the 16-bit limit
           dict(window_bits=2, window=4),                 # window index out of range
           dict(window_bits=0, window=1),
           dict(window_bits=2, window=1, match_scope=1)]  # no halo across windows
    for kw in bad:
        with pytest.raises(vx.VxError) as ei:
            vx.vx_plot_required_bytes(31, vx.make_opts(**kw))
        assert ei.value.code == vx.VX_EINVAL, kw
    vx.vx_plot_required_bytes(31, vx.make_opts(window_bits=16, window=(1 << 16) - 1))
    for c in (-1, 17):
        with pytest.raises(vx.VxError):
            vx.vx_plot_tiled_bytes(31, c)
    with pytest.raises(vx.VxError):   # opts that already name a window
        vx.vx_plot_tiled_bytes(31, 2, vx.make_opts(window_bits=2))


def test_window_plan_at_the_partition_limit(vx):
    # c equal to the partition bits: each window is one partition.
    for K, s in [(12, 6), (20, 11), (27, 11)]:
        p = K - s
        t1, t2, sc = vx.vx_plot_required_bytes(K, vx.make_opts(window_bits=p, window=0, partition_log2=s))
        assert t1 >= 12 * 2 ** s
        with pytest.raises(vx.VxError):
            vx.vx_plot_required_bytes(K, vx.make_opts(window_bits=p + 1, window=0, partition_log2=s))


def test_tiled_write_rejects_bad_arguments_before_creating_the_file(vx, tmp_path):
    # argument errors come back before any file or device work
    path = tmp_path / "plot.bin"
    for K, c, o in [(31, 17, None), (31, -1, None), (14, 2, vx.make_opts(window_bits=1))]:
        rc, _, _, _ = vx.vx_plot_tiled_write(K, bytes(32), c, str(path), opts=o, stream=0, check=False)
        assert rc == vx.VX_EINVAL
        assert not path.exists()


def test_server_rejects_window_options(vx):
    # A served request is a whole plot: window options in the server's plot
    # options are refused before any device work.
    o = vx.vx_serve_opts()
    o.size = ctypes.sizeof(vx.vx_serve_opts)
    o.plot_opts = vx.make_opts(window_bits=1)
    with pytest.raises(vx.VxError) as ei:
        vx.vx_serve_create(o)
    assert ei.value.code == vx.VX_EINVAL


def test_tiled_window_bits_fit_a_budget(vx):
    # The fewest window bits whose two window buffers (and window ids) fit.
    for K, budget in [(31, 100 << 30), (31, 60 << 30), (31, 30 << 30), (32, 120 << 30), (32, 60 << 30),
                      (20, 1 << 40)]:
        c = vx.vx_plot_tiled_window_bits(K, budget)
        assert vx.vx_plot_tiled_bytes(K, c)[0] <= budget, (K, budget, c)
        for smaller in range(c):
            assert vx.vx_plot_tiled_bytes(K, smaller)[0] > budget, (K, budget, smaller)
    assert vx.vx_plot_tiled_window_bits(31, 1 << 40) == 0        # the whole plot fits
    assert vx.vx_plot_tiled_window_bits(31, 60 << 30) == 2       # two quarter-plot windows + ids
    with pytest.raises(vx.VxError) as ei:                        # no window count fits 1 MB
        vx.vx_plot_tiled_window_bits(31, 1 << 20)
    assert ei.value.code == vx.VX_ENOMEM


def test_tiled_hash_passes_and_the_capped_choice(vx):
    # Whole plot: one hash of every nonce; 1..8 window bits: the id pass and
    # each window's list, two; above 8 bits every window hashes every nonce.
    assert vx.vx_plot_tiled_hash_passes(31, 0) == 1
    for c in range(1, 9):
        assert vx.vx_plot_tiled_hash_passes(31, c) == 2, c
    assert vx.vx_plot_tiled_hash_passes(31, 9) == 512
    assert vx.vx_plot_tiled_hash_passes(31, 10) == 1024
    # nonce chunks turn the id pass off
    assert vx.vx_plot_tiled_hash_passes(31, 3, vx.make_opts(pipeline_chunks=2)) == 8
    # A budget between the 9-bit and the 8-bit footprints: the default choice
    # refuses (it would hash the plot 512 times), the capped one takes 9 bits
    # only when told that 512 passes are acceptable.
    f8 = vx.vx_plot_tiled_bytes(31, 8)[0]
    f9 = vx.vx_plot_tiled_bytes(31, 9)[0]
    assert f9 < f8
    budget = (f8 + f9) // 2
    with pytest.raises(vx.VxError) as ei:
        vx.vx_plot_tiled_window_bits(31, budget)
    assert ei.value.code == vx.VX_ENOMEM
    with pytest.raises(vx.VxError):
        vx.vx_plot_tiled_window_bits(31, budget, max_hash_passes=511)
    assert vx.vx_plot_tiled_window_bits(31, budget, max_hash_passes=512) == 9
    assert vx.vx_plot_tiled_window_bits(31, f8, max_hash_passes=512) == 8


def test_window_planner_sweep(vx):
    # Every K and every window count the planner accepts: a window's buffers
    # hold its share of the tables (Table 1 at least 12 B per expected record,
    # Table 2 at least 16 B per expected pair and, for a window, its nonce
    # list of 4 B per expected record), and from 2 window bits on each extra
    # bit shrinks the tiled footprint.  Anything else is VX_EINVAL.
    for K in range(1, 33):
        p = max(0, min(21, K - 11))
        prev = None
        for c in range(0, min(p, 16) + 2):
            try:
                t1, t2, sc = vx.vx_plot_required_bytes(K, vx.make_opts(window_bits=c, window=0))
            except vx.VxError as e:
                assert e.code == vx.VX_EINVAL and c > min(p, 16), (K, c)
                continue
            assert c <= min(p, 16)
            recs = 2 ** K / 2 ** c
            lam = 2 ** K / 2 ** 24
            u = min(1.0, 2.0 ** (64 - K) / 2 ** 40)
            pairs = 2 ** 24 * lam * lam / 2 * (2 * u - u * u) / 2 ** c
            assert t1 >= 12 * recs and t2 >= 16 * pairs, (K, c, t1, t2)
            if c:
                assert t2 >= 4 * recs, (K, c, t2)  # the window's nonce list
            dev = vx.vx_plot_tiled_bytes(K, c)[0]
            if prev is not None and c >= 3:
                assert dev < prev, (K, c, dev, prev)
            prev = dev


def test_plot_file_that_cannot_be_opened_is_an_io_error(vx, tmp_path):
    # The file is opened before any device work: a path in a missing
    # directory gives VX_EIO, not VX_EINVAL (bad arguments) or VX_ECUDA.
    path = str(tmp_path / "no_such_dir" / "plot.bin")
    rc, _, _, _ = vx.vx_plot_tiled_write(12, bytes(32), 0, path, check=False, stream=0)
    assert rc == vx.VX_EIO
    rc, _, _, _ = vx.vx_plot_tiled_write(12, bytes(32), 40, path, check=False, stream=0)
    assert rc == vx.VX_EINVAL  # bad window bits are still refused first
