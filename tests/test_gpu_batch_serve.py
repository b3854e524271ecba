"""Batched and served plotting give every plot exactly the tables it gets
alone (the oracle's), whatever the mix of K and keys."""
import time

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


_cache = {}


def oracle_tables(K, seed):
    if (K, seed) not in _cache:
        key = plot_key(seed)
        t1 = orc.table1(K, key)
        _cache[(K, seed)] = (t1, orc.match(key, t1, orc.default_distance(K)))
    return _cache[(K, seed)]


def copy_table(vx, h, which):
    _, n, rb, _ = vx.vx_table_info(h, which)
    host = torch.empty(max(1, n * rb), dtype=torch.uint8).pin_memory()
    vx.vx_table_copy(h, which, host.data_ptr(), n * rb)
    torch.cuda.synchronize()
    return host[: n * rb].numpy().reshape(n, rb)


@pytest.mark.parametrize("placement", [1, 2], ids=["lookback", "slots"])
def test_batch_mixed_k_equals_oracle(vx, placement):
    mix = [(10, 101), (14, 102), (16, 103), (18, 104), (20, 105), (12, 106), (22, 107), (17, 108),
           (1, 109), (24, 110)]
    plots = [vx.Plot(K, plot_key(s), vx.make_opts(t2_placement=placement)) for K, s in mix]
    handles = [p.handle for p in plots]
    for rep in range(2):  # the second launch replays the recorded graph
        vx.vx_plot_batch(handles)
        for (K, s), p in zip(mix, plots):
            p.sync()
            if K > 22:
                continue
            r1, r2 = oracle_tables(K, s)
            assert np.array_equal(p.t1.cpu().numpy(), r1), (rep, K)
            assert np.array_equal(p.t2.cpu().numpy(), r2), (rep, K)
    # the K=24 member equals its own single-plot run
    single = vx.Plot(24, plot_key(110))
    single.run()
    single.sync()
    assert torch.equal(single.t1, plots[-1].t1) and torch.equal(single.t2, plots[-1].t2)
    for p in plots + [single]:
        p.close()


def test_serve_mix_equals_oracle(vx):
    srv = vx.vx_serve_create()
    rng = np.random.default_rng(9)
    reqs = []
    for r in range(16):
        K = int(rng.integers(12, 21))
        seed = 500 + r
        reqs.append((vx.vx_serve_submit(srv, K, plot_key(seed)), K, seed))
        if r % 5 == 4:
            vx.vx_serve_step(srv)   # later requests arrive while earlier ones run
    done = {}
    t0 = time.time()
    while len(done) < len(reqs):
        assert time.time() - t0 < 120, "server did not finish"
        for t, K, seed in reqs:
            if t in done:
                continue
            st, h = vx.vx_serve_poll(srv, t)
            assert st != vx.VX_FAILED
            if st == vx.VX_DONE:
                done[t] = h
        time.sleep(0.002)
    for t, K, seed in reqs:
        h = done[t]
        r1, r2 = oracle_tables(K, seed)
        assert np.array_equal(copy_table(vx, h, vx.VX_TABLE1), r1)
        assert np.array_equal(copy_table(vx, h, vx.VX_TABLE2), r2)
        assert vx.vx_serve_latency(srv, t) > 0
        vx.vx_plot_destroy(h)
    assert vx.vx_serve_step(srv) == 0
    vx.vx_serve_destroy(srv)


def test_serve_rejects_oversized(vx):
    srv = vx.vx_serve_create(vx.vx_serve_opts(size=0, memory_budget=1 << 20))
    with pytest.raises(vx.VxError):
        vx.vx_serve_submit(srv, 20, plot_key(1))
    vx.vx_serve_destroy(srv)


def test_batch_mixed_scope_and_placement(vx):
    # One batch launch mixing cross-bucket and bucket-scope plots (the
    # halo-capable kernel instances run both kinds) and both Table-2
    # placements (a mixed launch places every plot by look-back): each plot
    # equals its own oracle.
    mix = [(14, 120, dict(match_scope=1)), (16, 121, dict(t2_placement=1, nonces_per_thread=16)),
           (18, 122, dict(match_scope=1, t2_placement=2)),
           (12, 123, dict(t2_placement=2)), (20, 124, dict(match_scope=1)), (1, 125, dict(match_scope=1))]
    plots = [vx.Plot(K, plot_key(s), vx.make_opts(**kw)) for K, s, kw in mix]
    for rep in range(2):
        vx.vx_plot_batch([p.handle for p in plots])
        for (K, s, kw), p in zip(mix, plots):
            p.sync()
            key = plot_key(s)
            t1 = orc.table1(K, key)
            D = orc.default_distance(K)
            r2 = orc.match_global(key, t1, D) if kw.get("match_scope") else orc.match(key, t1, D)
            assert np.array_equal(p.t1.cpu().numpy(), t1), (rep, K)
            assert np.array_equal(p.t2.cpu().numpy(), r2), (rep, K)
    for p in plots:
        p.close()
