"""Batched form: many hypergraphs with their own s in one captured pipeline
give, member by member, exactly the oracle's L_s."""
import numpy as np
import pytest

import hypergen as hg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
slg = pytest.importorskip("paper_2010_11448_gb300")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_11448_gb300 import build_lib
    build_lib.build()
    slg.load()


def members(count, seed):
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(np.log(200), np.log(8000), size=count)).astype(int)
    ss = rng.integers(1, 12, size=count)
    gs = [hg.chung_lu(int(m), 2 * int(m), seed=seed + k, size_cap=800)
          for k, m in enumerate(ms)]
    # a member without incidences and a member with a huge s
    gs.append(hg.from_rows([[], []], 3))
    ss = np.append(ss, 2)
    gs.append(hg.uniform(300, 400, 1, 10, seed=5))
    ss = np.append(ss, 1000)
    return gs, [int(x) for x in ss]


def as_np(t):
    i, j, w = t
    if i.shape[0] == 0:
        return np.zeros((0, 3), np.int64)
    return np.stack([i.cpu().numpy(), j.cpu().numpy(), w.cpu().numpy()], 1).astype(np.int64)


@pytest.mark.parametrize("dual", [False, True])
def test_members_match_oracle(dual):
    gs, ss = members(24, 11)
    plan = slg.Plan([slg.to_device(g) for g in gs], ss, dual=dual)
    info = plan.info()
    assert info["launches"] > 0 and info["tuned_ms"] > 0
    assert info["bins"][0] <= 128 and info["bins"][1] <= 1024 and info["bins"][2] <= 4096
    for rep in range(2):                     # the captured graph replays cleanly
        plan.execute()
        res = plan.results()
        for g, s, r in zip(gs, ss, res):
            want = oracle.canonical(*oracle.line_graph_of(g, s, dual=dual, threads=4))
            assert np.array_equal(as_np(r), want)
    plan.close()


def test_unweighted_batch_pairs():
    gs, ss = members(8, 3)
    plan = slg.Plan([slg.to_device(g) for g in gs], ss, unweighted=True)
    plan.execute()
    for g, s, (i, j, w) in zip(gs, ss, plan.results()):
        assert w is None
        want = oracle.canonical(*oracle.line_graph_of(g, s))
        got = np.stack([i.cpu().numpy(), j.cpu().numpy()], 1) if i.shape[0] else np.zeros((0, 2))
        assert np.array_equal(got, want[:, :2])


def test_union_beyond_one_super_chunk():
    # two members with large rows first, then a filler of 4.2M small rows:
    # the union has more than 4M rows, so the early rows' id span covers
    # several super-chunks of the giant bin (member 0, s = 1: its large rows
    # take the giant bin) or several windows of the sparse bin (member 1,
    # s = 3) while all their far ends lie in the first one (the later ones
    # are empty for them)
    gs = [hg.chung_lu(20_000, 40_000, seed=61, size_cap=4000),
          hg.lognormal_web(20_000, 40_000, seed=62, cap=2000, core_edges=256,
                           core_vertices=512, core_density=0.3),
          hg.uniform(4_200_000, 600_000, 1, 3, seed=3)]
    ss = [1, 3, 2]
    dhs = [slg.to_device(h) for h in gs]
    plan = slg.Plan(dhs, ss)
    for _ in range(3):
        plan.execute()
    res = plan.results()
    for k in range(2):
        want = oracle.canonical(*oracle.line_graph_of(gs[k], ss[k], threads=16))
        assert np.array_equal(as_np(res[k]), want), k
        st = slg.build(dhs[k], ss[k])
        assert np.array_equal(as_np(st), want), k
    filler = slg.build(dhs[2], ss[2])
    assert all(torch.equal(a, b) for a, b in zip(res[2], filler))
