"""CUDA path vs the CPU oracle, element by element (bit-exact: every count is
an exact integer).  All calls go through the C ABI via the thin binding."""
import ctypes

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


def as_np(t):
    i, j, w = t
    cols = [i.cpu().numpy(), j.cpu().numpy()]
    cols.append(w.cpu().numpy() if w is not None else np.zeros_like(cols[0]))
    return np.stack(cols, 1).astype(np.int64) if cols[0].shape[0] else np.zeros((0, 3), np.int64)


def gpu_lg(dh, s, dual=False, **kw):
    return as_np(slg.build(dh, s, dual=dual, **kw))


def want_lg(h, s, dual=False, rows=None, threads=8):
    return oracle.canonical(*oracle.line_graph_of(h, s, dual=dual, rows=rows, threads=threads))


# ------------------------------------------------------------- small cases --

@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [1, 2, 3])
def test_uniform_2k(dual, s):
    h = hg.config("uniform_2k")
    dh = slg.to_device(h)
    assert np.array_equal(gpu_lg(dh, s, dual), want_lg(h, s, dual))


def test_random_small_edge_cases():
    # empty rows, singletons, duplicated rows, isolated vertices
    for seed in range(40):
        h = hg.random_small(seed)
        dh = slg.to_device(h)
        for dual in (False, True):
            for s in (1, 2, 3):
                got = gpu_lg(dh, s, dual)
                assert np.array_equal(got, want_lg(h, s, dual)), (seed, dual, s)


def test_fig1():
    import pins
    names, rows, facts = pins.load_fig1()
    h = hg.from_rows(rows, 12)
    dh = slg.to_device(h)
    for dual in (False, True):
        for s in (1, 2, 3):
            assert np.array_equal(gpu_lg(dh, s, dual), want_lg(h, s, dual))


def test_degenerate_inputs():
    # no incidences at all, s above every size, a single hyperedge
    for h in (hg.from_rows([[], [], []], 5), hg.from_rows([[0, 1, 2]], 3),
              hg.from_rows([[0, 1], [0, 1]], 2)):
        dh = slg.to_device(h)
        for dual in (False, True):
            for s in (1, 2, 3, 100):
                assert np.array_equal(gpu_lg(dh, s, dual), want_lg(h, s, dual))
                assert slg.count(dh, s, dual) == want_lg(h, s, dual).shape[0]


def test_graph_special_case():
    rng = np.random.default_rng(3)
    edges = sorted({tuple(sorted(rng.choice(300, 2, replace=False).tolist()))
                    for _ in range(2000)})
    h = hg.graph(300, edges)
    dh = slg.to_device(h)
    for dual in (False, True):
        for s in (1, 2):
            assert np.array_equal(gpu_lg(dh, s, dual), want_lg(h, s, dual))


# --------------------------------------- medium: every bin incl. giant rows --

@pytest.fixture(scope="module")
def medium():
    # Sizes capped at 3000 with mean 20: rows reach every bin, including the
    # giant one (work > 8192) on both sides.
    h = hg.chung_lu(30_000, 60_000, seed=21, size_cap=3000)
    return h, slg.to_device(h)


@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [1, 2, 4, 8, 16])
def test_medium_all_bins(medium, dual, s):
    h, dh = medium
    got = gpu_lg(dh, s, dual)
    assert np.array_equal(got, want_lg(h, s, dual))
    st = slg.last_stats()
    m, n, off, idx = oracle.side(h, dual)
    assert st["wedges"] == oracle.wedges(m, n, off, idx, s)
    if s <= 4:
        assert st["rows_bin"][3] > 0, "giant bin not exercised"
    if dual and s >= 2:
        assert st["rows_bin"][4] > 0, "sparse bin not exercised"


def test_medium_unweighted_same_pairs(medium):
    h, dh = medium
    for dual in (False, True):
        for s in (2, 8):
            a = gpu_lg(dh, s, dual)
            b = gpu_lg(dh, s, dual, unweighted=True)
            assert np.array_equal(a[:, :2], b[:, :2])


def test_medium_count_and_wedges(medium):
    h, dh = medium
    for dual in (False, True):
        m, n, off, idx = oracle.side(h, dual)
        for s in (1, 3, 9):
            assert slg.count(dh, s, dual) == want_lg(h, s, dual).shape[0]
            assert slg.wedges(dh, s, dual) == oracle.wedges(m, n, off, idx, s)


def test_medium_row_ranges_concatenate(medium):
    h, dh = medium
    s = 2
    full = want_lg(h, s)
    parts = []
    bounds = [0, 7, 1000, 1001, 17_000, h.m]
    for a, b in zip(bounds[:-1], bounds[1:]):
        try:
            parts.append(as_np(slg.build_rows(dh, s, a, b, capacity=0)))
        except slg.SlgError as exc:
            assert exc.status == 2
            parts.append(as_np(slg.build_rows(dh, s, a, b, capacity=max(exc.needed, 1))))
    assert np.array_equal(np.concatenate(parts), full)


def test_capacity_error_reports_count(medium):
    h, dh = medium
    n = slg.count(dh, 3)
    with pytest.raises(slg.SlgError) as ei:
        slg.build(dh, 3, capacity=max(n - 1, 1))
    assert ei.value.status == 2


def test_small_staging_falls_back_to_direct(medium):
    # A capacity equal to the count makes staging exact; the result must be
    # identical whichever emission path ran.
    h, dh = medium
    n = slg.count(dh, 2, True)
    got = as_np(slg.build(dh, 2, dual=True, capacity=n))
    assert np.array_equal(got, want_lg(h, 2, True))


def test_host_entry_point(medium):
    h, _ = medium
    want = want_lg(h, 4)
    got = slg.build_host(h, 4, capacity=want.shape[0] + 5)
    assert np.array_equal(np.stack([a for a in got], 1).astype(np.int64), want)


def test_host_entry_point_pinned(medium):
    # page-locked host buffers in and out, as the end-to-end benchmark uses
    h, _ = medium
    for dual, s in ((False, 2), (True, 3)):
        want = want_lg(h, s, dual)
        cap = want.shape[0] + 7
        out = tuple(torch.full((cap,), -1, dtype=torch.int32).pin_memory() for _ in range(3))
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()

        class HostH:
            pass
        hh = HostH()
        hh.m, hh.n = h.m, h.n
        hh.e_off, hh.e_idx, hh.v_off, hh.v_idx = (pin(h.e_off), pin(h.e_idx), pin(h.v_off),
                                                  pin(h.v_idx))
        got = slg.build_host(hh, s, dual=dual, out=out)
        assert np.array_equal(np.stack([a.numpy() for a in got], 1).astype(np.int64), want)
        assert int(out[0][want.shape[0]]) == -1  # nothing written past the pairs
        # too small: the count comes back, nothing overruns
        small = tuple(torch.zeros(3, dtype=torch.int32).pin_memory() for _ in range(3))
        with pytest.raises(slg.SlgError) as ei:
            slg.build_host(hh, s, dual=dual, out=small)
        assert ei.value.status == 2 and ei.value.needed == want.shape[0]


def test_host_entry_point_async_streams(medium):
    # SLG_ASYNC: four builds on four streams, each returning once its copies
    # back are enqueued; after the streams complete every list is the oracle's
    h, _ = medium
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()

    class HostH:
        pass
    hh = HostH()
    hh.m, hh.n = h.m, h.n
    hh.e_off, hh.e_idx, hh.v_off, hh.v_idx = (pin(h.e_off), pin(h.e_idx), pin(h.v_off),
                                              pin(h.v_idx))
    jobs = [(False, 2), (True, 2), (False, 5), (True, 3)]
    wants = [want_lg(h, s, dual) for dual, s in jobs]
    streams = [torch.cuda.Stream() for _ in jobs]
    for rep in range(2):
        outs = [tuple(torch.full((w.shape[0] + 5,), -1, dtype=torch.int32).pin_memory()
                      for _ in range(3)) for w in wants]
        got = []
        for (dual, s), o, st in zip(jobs, outs, streams):
            got.append(slg.build_host(hh, s, dual=dual, out=o, stream=st, wait=False))
        for st in streams:
            st.synchronize()
        for g, w, o in zip(got, wants, outs):
            assert np.array_equal(np.stack([a.numpy() for a in g], 1).astype(np.int64), w)
            assert int(o[0][w.shape[0]]) == -1


def test_on_side_stream(medium):
    h, dh = medium
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        got = gpu_lg(dh, 4, stream=st)
    st.synchronize()
    assert np.array_equal(got, want_lg(h, 4))


# ------------------------------------------------------------ bad inputs --

def _corrupt(h, what):
    e_off, e_idx = h.e_off.copy(), h.e_idx.copy()
    v_off, v_idx = h.v_off.copy(), h.v_idx.copy()
    if what == "unsorted_row":
        k = int(np.argmax(np.diff(e_off) >= 3))
        a = e_off[k]
        e_idx[a], e_idx[a + 1] = e_idx[a + 1], e_idx[a]
    elif what == "id_out_of_range":
        e_idx[0] = h.n + 5
    elif what == "offset_beyond_nnz":
        e_off[-1] = e_off[-1] + 10
    elif what == "csc_mismatch":
        v_idx = v_idx.copy()
        v_idx[0] = (v_idx[0] + 1) % h.m
        v_idx[: v_off[1]] = np.sort(v_idx[: v_off[1]])
    return hg.Hypergraph(h.m, h.n, e_off, e_idx, v_off, v_idx)


@pytest.mark.parametrize("what", ["unsorted_row", "id_out_of_range",
                                  "offset_beyond_nnz", "csc_mismatch"])
def test_malformed_input_is_an_error_status(what):
    h = hg.uniform(500, 800, 3, 12, seed=2)
    bad = _corrupt(h, what)
    dh = slg.to_device(bad)
    with pytest.raises(slg.SlgError) as ei:
        slg.count(dh, 2)
    assert ei.value.status == 1
    # the library stays usable afterwards
    good = slg.to_device(h)
    assert np.array_equal(gpu_lg(good, 2), want_lg(h, 2))


def test_bad_arguments():
    h = hg.uniform(50, 80, 1, 5, seed=2)
    dh = slg.to_device(h)
    for s in (0, -3):
        with pytest.raises(slg.SlgError) as ei:
            slg.count(dh, s)
        assert ei.value.status == 1


# ---------------------------------------------- full size, sampled outputs --

@pytest.fixture(scope="module")
def chung_lu_1m():
    h = hg.config("chung_lu_1m")
    return h, slg.to_device(h)


@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("s", [2, 8])
def test_chung_lu_1m_sampled_rows(chung_lu_1m, dual, s):
    """Full-size workload in the benchmark's launch configuration; every
    97th row (plus the rows of the largest hyperedges) compared with the
    oracle, and order / threshold / size-filter properties checked on all
    pairs (on the device: the output has up to ~5e8 pairs)."""
    h, dh = chung_lu_1m
    i, j, w = slg.build(dh, s, dual=dual)
    m, n, off, idx = oracle.side(h, dual)
    sizes_np = np.diff(off)
    heavy = np.argsort(sizes_np)[-64:]
    rows = np.unique(np.concatenate([np.arange(0, m, 97), heavy])).astype(np.int32)
    want = oracle.canonical(*oracle.line_graph(m, n, off, idx, s, rows=rows, threads=16))
    sel = torch.isin(i, torch.from_numpy(rows).to(i.device))
    got = np.stack([i[sel].cpu().numpy(), j[sel].cpu().numpy(), w[sel].cpu().numpy()],
                   1).astype(np.int64)
    assert np.array_equal(got, want)
    # properties of every pair, checked on the device
    assert bool(torch.all(i < j)) and bool(torch.all(w >= s))
    key = i.long() * m + j.long()
    assert bool(torch.all(key[1:] > key[:-1]))
    sizes = torch.from_numpy(sizes_np.astype(np.int32)).to(i.device)
    assert bool(torch.all(sizes[i.long()] >= s)) and bool(torch.all(sizes[j.long()] >= s))
    assert slg.last_stats()["wedges"] == oracle.wedges(m, n, off, idx, s)


def test_ids_beyond_one_super_chunk():
    # the dual of 1500 large hyperedges over 5M vertices: rows are vertices,
    # far-end ids span up to 5M.  At s >= 2 the large rows are sparse in that
    # span and cross several windows of the sparse bin.
    h = hg.uniform(1500, 5_000_000, 500, 6000, seed=9)
    dh = slg.to_device(h)
    m, n, off, idx = oracle.side(h, True)
    deg = np.diff(off)
    top = np.argsort(-deg, kind="stable")[:3000]
    rows = np.unique(np.concatenate([top, np.arange(0, m, 97)])).astype(np.int32)
    for s in (2, 3):
        got = gpu_lg(dh, s, dual=True)
        st = slg.last_stats()
        assert st["rows_bin"][4] > 0  # sparse large rows present
        sel = got[np.isin(got[:, 0], rows)]
        want = oracle.canonical(*oracle.line_graph(m, n, off, idx, s, rows=rows, threads=16))
        assert np.array_equal(sel, want), s
        assert got.shape[0] == slg.count(dh, s, dual=True)


def test_giant_rows_beyond_one_super_chunk():
    # s = 1 sends every large row to the giant bin.  The dual of one
    # hyperedge of 8000 random vertices out of 5M (plus small hyperedges):
    # its first ~1800 vertices have more than 6144 wedges (the giant bin's
    # partitioned rows), and their far-end span (v, 5M) covers more than the
    # 4M ids of one super-chunk of the giant bin, most of them empty.
    rng = np.random.default_rng(12)
    n = 5_000_000
    big = np.sort(rng.choice(n, 8000, replace=False))
    small = [np.sort(rng.choice(n, int(k), replace=False)) for k in rng.integers(2, 40, 3000)]
    h = hg.from_rows([big] + small, n)
    dh = slg.to_device(h)
    m, n_, off, idx = oracle.side(h, True)
    rows = np.unique(np.concatenate([big[:2000:3], np.arange(0, m, 4999)])).astype(np.int32)
    got = gpu_lg(dh, 1, dual=True)
    st = slg.last_stats()
    assert st["rows_bin"][3] > 0 and st["rows_bin"][4] == 0
    sel = got[np.isin(got[:, 0], rows)]
    want = oracle.canonical(*oracle.line_graph(m, n_, off, idx, 1, rows=rows, threads=16))
    assert np.array_equal(sel, want)
    assert got.shape[0] == slg.count(dh, 1, dual=True)


# ------------------------------------------------ compressed row form (CSR) --

def _csr_to_triples(ptr, j, w):
    ptr = np.asarray(ptr, np.int64)
    i = np.repeat(np.arange(ptr.shape[0] - 1, dtype=np.int64), np.diff(ptr))
    return np.stack([i, np.asarray(j, np.int64), np.asarray(w, np.int64)], 1)


@pytest.mark.parametrize("dual", [False, True])
def test_build_csr_matches_oracle(medium, dual):
    h, dh = medium
    for s in (2, 5):
        want = want_lg(h, s, dual)
        ptr, j, w = slg.build_csr(dh, s, dual=dual)
        R = h.n if dual else h.m
        assert ptr.shape[0] == R + 1 and int(ptr[-1]) == want.shape[0]
        got = _csr_to_triples(ptr.cpu().numpy(), j.cpu().numpy(), w.cpu().numpy())
        assert np.array_equal(got, want)


def test_build_host_many_both_forms(medium):
    # one upload, four builds; two in compressed row form, two as triples;
    # every result equals the oracle's; a query with too small a capacity
    # reports its count without stopping the others
    h, _ = medium
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()

    class HostH:
        pass
    hh = HostH()
    hh.m, hh.n = h.m, h.n
    hh.e_off, hh.e_idx, hh.v_off, hh.v_idx = (pin(h.e_off), pin(h.e_idx), pin(h.v_off),
                                              pin(h.v_idx))
    jobs = [(True, 2, True), (False, 2, False), (True, 6, False), (False, 3, True)]
    wants = [want_lg(h, s, dual) for dual, s, _ in jobs]
    queries = []
    for (dual, s, csr), want in zip(jobs, wants):
        cap = want.shape[0] + 3
        q = {"s": s, "dual": dual, "capacity": cap,
             "out_j": torch.full((cap,), -1, dtype=torch.int32).pin_memory(),
             "out_w": torch.full((cap,), -1, dtype=torch.int32).pin_memory()}
        if csr:
            q["row_ptr"] = torch.full(((h.n if dual else h.m) + 1,), -1,
                                      dtype=torch.int64).pin_memory()
        else:
            q["out_i"] = torch.full((cap,), -1, dtype=torch.int32).pin_memory()
        queries.append(q)
    small = {"s": 2, "dual": True, "capacity": 5, "out_i": np.zeros(5, np.int32),
             "out_j": np.zeros(5, np.int32), "out_w": np.zeros(5, np.int32)}
    res = slg.build_host_many(hh, queries[:2] + [small] + queries[2:])
    assert [r[0] for r in res] == [0, 0, 2, 0, 0]
    assert res[2][1] == wants[0].shape[0]
    for (dual, s, csr), want, q, (st, n) in zip(jobs, wants, queries, res[:2] + res[3:]):
        assert n == want.shape[0]
        if csr:
            got = _csr_to_triples(q["row_ptr"].numpy(), q["out_j"][:n].numpy(),
                                  q["out_w"][:n].numpy())
        else:
            got = np.stack([q["out_i"][:n].numpy(), q["out_j"][:n].numpy(),
                            q["out_w"][:n].numpy()], 1).astype(np.int64)
        assert np.array_equal(got, want), (dual, s, csr)
        assert int(q["out_j"][n]) == -1  # nothing past the pairs


def test_build_host_csr_entry_point(medium):
    h, _ = medium
    want = want_lg(h, 4, True)
    R = h.n
    ptr = np.full(R + 1, -1, np.int64)
    j = np.zeros(want.shape[0] + 1, np.int32)
    w = np.zeros(want.shape[0] + 1, np.int32)
    n = ctypes.c_int64(0)
    st = slg._host_struct(h)
    rc = slg.load().slg_build_host_csr(ctypes.byref(st), 4, slg.SLG_DUAL, ptr.ctypes.data,
                                       j.ctypes.data, w.ctypes.data, j.shape[0],
                                       ctypes.byref(n), None)
    assert rc == 0 and n.value == want.shape[0]
    assert np.array_equal(_csr_to_triples(ptr, j[:n.value], w[:n.value]), want)
    # relabelling and the SpGEMM path have no row form
    for flags in (slg.SLG_DUAL | slg.SLG_RELABEL_ASC, slg.SLG_DUAL | slg.SLG_ALGO_SPGEMM):
        assert slg.load().slg_build_host_csr(ctypes.byref(st), 4, flags, ptr.ctypes.data,
                                             j.ctypes.data, w.ctypes.data, j.shape[0],
                                             ctypes.byref(n), None) == 6


def _host_h(h):
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).pin_memory()

    class HostH:
        pass
    hh = HostH()
    hh.m, hh.n = h.m, h.n
    hh.e_off, hh.e_idx, hh.v_off, hh.v_idx = (pin(h.e_off), pin(h.e_idx), pin(h.v_off),
                                              pin(h.v_idx))
    return hh


def test_build_host_many_w16(medium):
    # SLG_W16: the same lists with the weights returned as uint16
    h, _ = medium
    hh = _host_h(h)
    jobs = [(True, 2, True), (False, 3, False)]
    wants = [want_lg(h, s, dual) for dual, s, _ in jobs]
    queries = []
    for (dual, s, csr), want in zip(jobs, wants):
        cap = want.shape[0] + 2
        q = {"s": s, "dual": dual, "capacity": cap, "w16": True,
             "out_j": torch.full((cap,), -1, dtype=torch.int32).pin_memory(),
             "out_w": torch.full((cap,), -1, dtype=torch.int16).pin_memory()}
        if csr:
            q["row_ptr"] = torch.zeros((h.n if dual else h.m) + 1, dtype=torch.int64).pin_memory()
        else:
            q["out_i"] = torch.zeros(cap, dtype=torch.int32).pin_memory()
        queries.append(q)
    res = slg.build_host_many(hh, queries)
    assert [r[0] for r in res] == [0, 0]
    for (dual, s, csr), want, q, (_, n) in zip(jobs, wants, queries, res):
        assert n == want.shape[0]
        w = q["out_w"][:n].numpy().view(np.uint16).astype(np.int64)
        if csr:
            got = _csr_to_triples(q["row_ptr"].numpy(), q["out_j"][:n].numpy(), w)
        else:
            got = np.stack([q["out_i"][:n].numpy(), q["out_j"][:n].numpy(), w], 1).astype(np.int64)
        assert np.array_equal(got, want), (dual, s)
        assert int(q["out_w"][n]) == -1  # nothing past the pairs


def test_build_host_many_w16_overflow():
    # two hyperedges sharing 70,000 vertices: w = 70,000 does not fit 16 bits,
    # so that query fails with SLG_ERR_UNSUPPORTED; a 32-bit query of the same
    # call and a later 16-bit one (s above every weight: no pairs) are
    # unaffected
    n = 70_010
    shared = list(range(70_000))
    h = hg.from_rows([shared + [70_000], shared + [70_001], [70_002, 70_003], [70_002, 70_003]], n)
    hh = _host_h(h)

    def q(w16, s):
        return {"s": s, "dual": False, "capacity": 4, "w16": w16,
                "out_i": np.zeros(4, np.int32), "out_j": np.zeros(4, np.int32),
                "out_w": np.zeros(4, np.int16 if w16 else np.int32)}
    qs = [q(True, 2), q(False, 2), q(True, 70_001)]
    res = slg.build_host_many(hh, qs)
    assert res[0] == (6, 2) and res[1] == (0, 2) and res[2] == (0, 0)
    assert qs[1]["out_i"][:2].tolist() == [0, 2] and qs[1]["out_j"][:2].tolist() == [1, 3]
    assert qs[1]["out_w"][:2].tolist() == [70_000, 2]


def test_graph_handle(medium):
    # slg_graph: validated and mapped once; builds and counts through it on
    # both sides equal the oracle and skip the three validation/map kernels
    h, dh = medium
    with slg.Graph(dh) as g:
        for dual in (False, True):
            for s in (2, 4):
                want = want_lg(h, s, dual)
                assert g.count(s, dual) == want.shape[0]
                got = g.build(s, dual=dual)
                launches_handle = slg.last_stats()["kernel_launches"]
                assert np.array_equal(as_np(got), want), (dual, s)
                slg.build(dh, s, dual=dual)
                assert slg.last_stats()["kernel_launches"] == launches_handle + 3
            assert np.array_equal(as_np(g.build(3, dual=dual, algo="plain")), want_lg(h, 3, dual))


def test_graph_handle_rejects_bad_input():
    # CSR and CSC of different incidences: the handle is refused, as every
    # build on that input would be
    a = hg.from_rows([[0, 1], [1, 2]], 3)
    b = hg.from_rows([[0, 1], [0, 2]], 3)
    bad = slg.DeviceHypergraph(a.m, a.n, *[torch.from_numpy(np.ascontiguousarray(x, np.int32)).cuda()
                                          for x in (a.e_off, a.e_idx, b.v_off, b.v_idx)])
    with pytest.raises(slg.SlgError) as exc:
        slg.Graph(bad)
    assert exc.value.status == 1
