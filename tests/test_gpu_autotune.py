"""The autotuner picks a plan that plots correctly, and its on-disk cache
serves later calls (keyed by device and K)."""
import json

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


def test_autotune_plan_plots_correctly_and_caches(vx, tmp_path):
    path = str(tmp_path / "tune.json")
    K = 18
    o = vx.autotune(K, cache_path=path)
    assert 9 <= o.partition_log2 <= 13 and o.scatter_mode in (1, 2)
    assert o.nonces_per_thread in ((4, 8, 16) if o.scatter_mode == 1 else (8,))
    cache = json.load(open(path))
    assert len(cache) == 1
    (k, entry), = cache.items()
    assert entry["ms"] > 0 and entry["partition_log2"] == o.partition_log2
    assert entry["nonces_per_thread"] == o.nonces_per_thread
    key = plot_key(130)
    p = vx.Plot(K, key, o)
    p.run()
    p.sync()
    t1 = orc.table1(K, key)
    assert np.array_equal(p.t1.cpu().numpy(), t1)
    assert np.array_equal(p.t2.cpu().numpy(), orc.match(key, t1, orc.default_distance(K)))
    p.close()
    # a later call takes the cached choice (changed here to prove it is read)
    entry["partition_log2"] = 12 if o.partition_log2 != 12 else 10
    json.dump({k: entry}, open(path, "w"))
    again = vx.autotune(K, cache_path=path)
    assert again.partition_log2 == entry["partition_log2"]
    # another K is tuned and added beside it
    vx.autotune(12, cache_path=path)
    assert len(json.load(open(path))) == 2


def test_autotune_keeps_the_base_options(vx, tmp_path):
    o = vx.autotune(14, vx.make_opts(match_scope=1), cache_path=str(tmp_path / "t.json"))
    assert o.match_scope == 1
