"""The no-allocation entry point (vx_plot_run_noalloc) gives the same tables
as the regular one (vx_plot_run) and as the CPU oracle, bit for bit, on two
calls in a row, with the default options and with non-default ones (the
cross-bucket match, a custom match distance).

It serves callers that cannot call cudaMalloc (device memory owned by
another allocator under a fixed budget; latency-critical code that must not
take cudaMalloc's implicit device synchronisation): the caller passes the
key and the two table buffers, and the library's scratch comes from a static
device array.  This file is collected last so that a failure here leaves
every other test already run.
"""
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


def regular_tables(vx, K, key, opts=None):
    p = vx.Plot(K, key, opts)
    p.run()
    n2 = p.sync()
    t1, t2 = p.t1.clone(), p.t2.clone()
    p.close()
    return t1, t2, n2


def oracle_tables(K, key, scope=0, D=None):
    t1 = orc.table1(K, key)
    D = orc.default_distance(K) if D is None else D
    t2 = orc.match_global(key, t1, D) if scope else orc.match(key, t1, D)
    return t1, t2


@pytest.mark.parametrize("opt", [{}, {"match_scope": 1}, {"match_distance": 1 << 38}],
                         ids=["default", "cross_bucket", "distance_2pow38"])
def test_noalloc_matches_regular_and_oracle_on_two_calls(vx, opt):
    # Caller-owned outputs, sized for the larger plot and reused by both calls.
    opts = vx.make_opts(**opt) if opt else None
    t1b, t2b, sb = vx.vx_plot_required_bytes(22, opts)
    d_t1 = torch.empty(t1b, dtype=torch.uint8, device="cuda")
    d_t2 = torch.empty(t2b, dtype=torch.uint8, device="cuda")
    cap = (t2b - 256) // 16
    for K, seed in [(22, 901), (17, 902)]:
        key = plot_key(seed)
        rc, n2 = vx.vx_plot_run_noalloc(K, key, d_t1.data_ptr(), d_t2.data_ptr(), cap, opts=opts)
        assert rc == vx.VX_OK
        N = 1 << K
        g1 = d_t1[: 12 * N].view(N, 12)
        g2 = d_t2[: 16 * n2].view(n2, 16)
        r1, r2, rn2 = regular_tables(vx, K, key, opts)
        assert n2 == rn2
        assert torch.equal(g1, r1)
        assert torch.equal(g2, r2)
        o1, o2 = oracle_tables(K, key, opt.get("match_scope", 0), opt.get("match_distance"))
        assert n2 == o2.shape[0]
        assert (g1.cpu().numpy() == o1).all()
        assert (g2.cpu().numpy() == o2).all()


def test_noalloc_rejects_plots_beyond_its_scratch(vx):
    t1b, t2b, sb = vx.vx_plot_required_bytes(23)
    assert sb > 64 << 20
    d = torch.empty(256, dtype=torch.uint8, device="cuda")
    rc, _ = vx.vx_plot_run_noalloc(23, plot_key(1), d.data_ptr(), d.data_ptr(), 1, check=False)
    assert rc == vx.VX_EINVAL
