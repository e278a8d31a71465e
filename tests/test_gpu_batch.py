"""Batches of independent operators (bf_batch_* through the C ABI): every
operator's output against the FP64 oracle apply of its factors, in all three
modes (one operator at a time, grouped launches, CUDA graph), forward and
adjoint; the modes agree bit for bit; the autotuner and its cache."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1502_01379_gb300 import build as pkg_build
    pkg_build.build()
    import paper_1502_01379_gb300 as mod
    mod.load()
    torch.cuda.set_device(0)
    return mod


def _rel(a, b):
    from oracle.kernel import rel_err
    return rel_err(np.asarray(a), np.asarray(b))


MIXED = [(0, 5, 3, 2), (2, 2, 3, 1), (4, 3, 5, 7), (6, 16, 12, 3), (8, 16, 16, 9), (4, 64, 32, 2),
         (6, 1, 1, 5), (8, 32, 8, 4), (2, 16, 16, 1), (10, 2, 7, 6)]


def _batch_inputs(shapes, seed):
    from bfinputs import complex_normal, synthetic_factors
    Fs, gs = [], []
    for i, (L, n0, r, nrhs) in enumerate(shapes):
        Fs.append(synthetic_factors(L, n0, r, seed=seed + i, dtype=np.complex64))
        gs.append(complex_normal((nrhs, n0 << L), seed=seed + 100 + i, dtype=np.complex64))
    return Fs, gs


@pytest.mark.parametrize("T,route", [(1, None), (2, None), (4, None), (8, None), (2, (4, 4)), (4, (2, 2))])
def test_mixed_batch_all_modes_against_oracle(bf, T, route):
    """route = (route_min_rhs, route_min_L): operators with that many vectors on
    trees that deep run their own CUDA-core multi-RHS passes on side streams
    beside the grouped launches (None: the defaults, which route none of these)."""
    from oracle import apply as A
    from paper_1502_01379_gb300 import capi
    Fs, gs = _batch_inputs(MIXED, seed=900 + T)
    ins = [torch.from_numpy(g).cuda() for g in gs]
    outs = [torch.empty_like(x) for x in ins]
    kw = {} if route is None else dict(route_min_rhs=route[0], route_min_L=route[1])
    b = capi.bf_batch_create(Fs, ins, outs, [g.shape[0] for g in gs], T=T, **kw)
    assert capi.bf_batch_items(b) > 0
    results = {}
    for adjoint in (False, True):
        for mode in (capi.BF_BATCH_EACH, capi.BF_BATCH_GROUPED, capi.BF_BATCH_GRAPH):
            for o in outs:
                o.fill_(float("nan"))
            capi.bf_batch_apply(b, adjoint, mode)
            torch.cuda.synchronize()
            capi.bf_batch_check(b)
            results[(adjoint, mode)] = [o.cpu().numpy() for o in outs]
        for o, (F, g) in enumerate(zip(Fs, gs)):
            fn = A.bf_adjoint if adjoint else A.bf_apply
            ref = fn(F.astype(np.complex128), g.T.astype(np.complex128)).T
            for mode in (capi.BF_BATCH_EACH, capi.BF_BATCH_GROUPED, capi.BF_BATCH_GRAPH):
                assert _rel(results[(adjoint, mode)][o], ref) < TOL, (o, adjoint, mode)
            # grouped and graph launches run the same thread blocks as the per-operator path
            assert np.array_equal(results[(adjoint, capi.BF_BATCH_GROUPED)][o], results[(adjoint, capi.BF_BATCH_GRAPH)][o])
    b.destroy()


def test_graph_replays_are_identical(bf):
    from paper_1502_01379_gb300 import capi
    Fs, gs = _batch_inputs(MIXED[:5], seed=950)
    ins = [torch.from_numpy(g).cuda() for g in gs]
    outs = [torch.empty_like(x) for x in ins]
    b = capi.bf_batch_create(Fs, ins, outs, [g.shape[0] for g in gs], T=2)
    capi.bf_batch_apply(b, False, capi.BF_BATCH_GRAPH)
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    for _ in range(3):
        capi.bf_batch_apply(b, False, capi.BF_BATCH_GRAPH)
    torch.cuda.synchronize()
    for a, c in zip(first, outs):
        assert torch.equal(a, c)
    b.destroy()


def test_batched_workload_256_operators(bf):
    """The batched workload: 256 operators, N log-uniform over 2^10 .. 2^16,
    r in {8, 12, 16}, 1..32 RHS each: graph-mode outputs equal the
    per-operator outputs bit for bit, and eight sampled operators (two RHS
    each) match the FP64 C loops of the oracle."""
    from bfinputs import batched_workload, complex_normal, synthetic_factors
    from oracle import capply
    from paper_1502_01379_gb300 import capi
    members = batched_workload()
    Fs = [synthetic_factors(m.L, m.n0, m.r, seed=2000 + i, dtype=np.complex64) for i, m in enumerate(members)]
    gs = [complex_normal((m.nrhs, m.N), seed=3000 + i, dtype=np.complex64) for i, m in enumerate(members)]
    ins = [torch.from_numpy(g).cuda() for g in gs]
    outs = [torch.empty_like(x) for x in ins]
    b = capi.bf_batch_create(Fs, ins, outs, [m.nrhs for m in members], T=2)
    capi.bf_batch_apply(b, False, capi.BF_BATCH_EACH)
    torch.cuda.synchronize()
    each = [o.cpu().numpy() for o in outs]
    capi.bf_batch_apply(b, False, capi.BF_BATCH_GRAPH)
    torch.cuda.synchronize()
    capi.bf_batch_check(b)
    graph = [o.cpu().numpy() for o in outs]
    for a, c in zip(each, graph):
        assert np.array_equal(a, c)
    rng = np.random.default_rng(0)
    for o in rng.choice(len(members), size=8, replace=False):
        P = capply.PreparedFactors(Fs[o])
        for j in sorted({0, members[o].nrhs - 1}):
            assert _rel(graph[o][j], capply.bf_apply_c(P, gs[o][j])) < TOL
    b.destroy()


def test_autotuner_caches_its_choice(bf, tmp_path):
    from paper_1502_01379_gb300 import batch as B
    Fs, gs = _batch_inputs(MIXED[:6], seed=970)
    ins = [torch.from_numpy(g).cuda() for g in gs]
    outs = [torch.empty_like(x) for x in ins]
    nrhs = [g.shape[0] for g in gs]
    path = str(tmp_path / "tune.json")
    cand = [(1, 16, 2), (2, 16, 2), (4, 8, 2)]
    first = B.autotune(Fs, ins, outs, nrhs, candidates=cand, cache_path=path, reps=2)
    assert not first["cached"] and (first["T"], first["slot_kb"], first["stages"]) in cand
    assert len(first["tried"]) == 3
    again = B.autotune(Fs, ins, outs, nrhs, candidates=cand, cache_path=path, reps=2)
    assert again["cached"] and again["T"] == first["T"]
    b, cfg = B.create_tuned(Fs, ins, outs, nrhs, cache_path=path)
    assert cfg["cached"]
    b.destroy()
