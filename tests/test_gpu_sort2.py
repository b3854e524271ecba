"""Table 2 sorted by hash2 (vx_sort_table2) against the oracle's sort of the
oracle's Table 2, byte for byte, through the C ABI."""
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
    return vaultx


def sorted_plot(vx, K, key, kw, split=False):
    p = vx.Plot(K, key, vx.make_opts(**kw) if kw else None)
    p.run_split() if split else p.run()
    n2 = p.sync()
    wb = vx.vx_sort_table2_work_bytes(p.handle)
    work = torch.empty(max(wb, 256), dtype=torch.uint8, device="cuda")
    vx.vx_sort_table2(p.handle, work.data_ptr(), wb)
    assert vx.vx_sync(p.handle) == vx.VX_OK
    _, n_after, _, _ = vx.vx_table_info(p.handle, vx.VX_TABLE2)
    assert n_after == n2
    t2 = p.t2.cpu().numpy()
    return p, t2, work


CASES = [(1, 0, {}), (5, 3, {}), (11, 5, {}), (12, 6, {}), (14, 8, {}), (16, 9, {}), (18, 10, {}),
         (20, 11, {}), (22, 0, {}), (22, 1, dict(match_scope=1)), (18, 12, dict(partition_log2=8)),
         (17, 18, dict(scatter_mode=2)), (16, 22, dict(fuse_pair_hash=1)),
         (14, 8, dict(t2_placement=2)), (19, 13, dict(match_scope=1, partition_log2=7))]


@pytest.mark.parametrize("K,seed,kw", CASES)
def test_sort_table2_matches_oracle(vx, K, seed, kw):
    key = plot_key(seed)
    p, got, _ = sorted_plot(vx, K, key, kw)
    t1 = orc.table1(K, key)
    D = orc.default_distance(K)
    ref = orc.match_global(key, t1, D) if kw.get("match_scope") else orc.match(key, t1, D)
    assert np.array_equal(got, orc.sort_table2(ref))
    p.close()


def test_sort_table2_after_split_path_and_twice(vx):
    K, key = 20, plot_key(44)
    p, got, work = sorted_plot(vx, K, key, {}, split=True)
    ref = orc.sort_table2(orc.match(key, orc.table1(K, key), orc.default_distance(K)))
    assert np.array_equal(got, ref)
    # sorting the sorted table again changes nothing
    vx.vx_sort_table2(p.handle, work.data_ptr(), work.numel())
    assert vx.vx_sync(p.handle) == vx.VX_OK
    assert np.array_equal(p.t2.cpu().numpy(), ref)
    p.close()


def test_sort_table2_call_errors(vx):
    p = vx.Plot(14, plot_key(45))
    # not run / not synced yet
    with pytest.raises(vx.VxError) as ei:
        vx.vx_sort_table2_work_bytes(p.handle)
    assert ei.value.code == vx.VX_ENOTREADY
    p.run()
    p.sync()
    wb = vx.vx_sort_table2_work_bytes(p.handle)
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    assert vx.lib().vx_sort_table2(p.handle, work.data_ptr(), wb - 256, None) == vx.VX_EINVAL
    assert vx.lib().vx_sort_table2(p.handle, work.data_ptr() + 8, wb - 256, None) == vx.VX_EINVAL
    p.close()
