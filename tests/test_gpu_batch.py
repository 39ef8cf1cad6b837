"""Batches of geometries in one concatenated tile list (not in the paper).

A batch only concatenates independent tile lists, so each sample must come
out bit for bit as if it had run alone, for every kernel mapping (block size,
persistent grid), and match the FP64 oracle."""
import numpy as np
import pytest

from paper_1703_08015_gb300 import geometry as geo
from paper_1703_08015_gb300 import lbm

pytestmark = pytest.mark.gpu


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _samples():
    out = []
    for k, (side, phi) in enumerate([(16, 0.6), (24, 0.3), (8, 0.5), (32, 0.15), (12, 0.45)]):
        shape = (side, side + 4 * (k % 2), side - 2 * (k % 3 == 1))
        m, _ = geo.sphere_pack_3d(shape=shape, seed=60 + k, r_min=2, r_max=max(3, side // 5), target_fluid=phi)
        out.append(m)
    return out


ARGS = dict(periodic=(1, 0, 0), tau=0.65, force=(1e-5, 0, 0))


@pytest.mark.parametrize("storage", [lbm.LBM_STORE_F64, lbm.LBM_STORE_F32S], ids=["f64", "f32s"])
def test_batch_equals_single_runs(oracle, storage):
    _cuda()
    masks = _samples()
    steps = 60
    b = lbm.BatchSolver(masks, 19, 4, storage=storage, **ARGS)
    try:
        b.step(steps)
        got = [b.export_pdfs(k) for k in range(len(masks))]
        stats, rc = b.stats()
        assert rc == 0
    finally:
        b.close()
    for k, m in enumerate(masks):
        s = lbm.Solver(m, 19, 4, storage=storage, **ARGS)
        try:
            s.step(steps)
            ref = s.export_pdfs()
            st, _ = s.stats()
        finally:
            s.close()
        fl = m.astype(bool)
        assert np.array_equal(got[k][:, fl].view(np.uint64), ref[:, fl].view(np.uint64)), k
        assert stats[k].mass == st.mass and stats[k].n_fluid == st.n_fluid
        if storage == lbm.LBM_STORE_F64:
            o = oracle.run(19, m, ARGS["periodic"], ARGS["tau"], ARGS["force"], oracle.init(19, m), steps)
            assert np.max(np.abs(got[k][:, fl] - o[:, fl]) / o[:, fl]) <= 1e-12


@pytest.mark.parametrize("block_nodes,persistent", [(128, 0), (256, 1), (128, 1)])
def test_batch_mappings_are_bit_identical(block_nodes, persistent):
    _cuda()
    masks = _samples()
    res = []
    for bn, pe in [(0, 0), (block_nodes, persistent)]:
        b = lbm.BatchSolver(masks, 19, 4, storage=lbm.LBM_STORE_F32S, block_nodes=bn, persistent=pe, **ARGS)
        try:
            b.step(45)
            res.append([b.export_pdfs(k) for k in range(len(masks))])
        finally:
            b.close()
    for a, c, m in zip(res[0], res[1], masks):
        fl = m.astype(bool)
        assert np.array_equal(a[:, fl].view(np.uint64), c[:, fl].view(np.uint64))


def test_batch_global_stats_are_the_sum_of_samples():
    _cuda()
    masks = _samples()
    b = lbm.BatchSolver(masks, 19, 4, storage=lbm.LBM_STORE_F32S, **ARGS)
    try:
        b.step(30)
        per, _ = b.stats()
        st = lbm.lbm_stats()
        lbm.lbm_moments(b.ctx, None, None, st, 0, b._s())
        assert lbm.library().lbm_num_samples(b.ctx) == len(masks)
        with pytest.raises(lbm.LBMError):
            lbm.lbm_export_pdfs(b.ctx, np.empty(1), 0, b._s())
    finally:
        b.close()
    assert st.n_fluid == sum(p.n_fluid for p in per)
    assert st.mass == pytest.approx(sum(p.mass for p in per), rel=1e-15)


def test_autotune_picks_a_compiled_mapping_and_reuses_its_cache(tmp_path, monkeypatch):
    """The tuner times every compiled candidate for the batch, returns the
    fastest, caches it under the GPU / lattice / storage / workload key, and
    a second call reads the cache without timing anything; the chosen
    mapping computes the same bits as the default one."""
    _cuda()
    from paper_1703_08015_gb300 import autotune

    masks = _samples()
    storage = lbm.LBM_STORE_F32S
    cache = tmp_path / "autotune.json"
    cands = autotune.candidates(19, storage, masks, ARGS["periodic"])
    assert {"tile_a": 4, "block_nodes": 0, "persistent": 0, "prefetch_blocks": 0} in cands
    assert {"tile_a": 4, "block_nodes": 0, "persistent": 0, "prefetch_blocks": -1} in cands
    best, trials = autotune.tune(masks, 19, storage, steps=8, cache_path=str(cache), **ARGS)
    assert best in cands
    assert len(trials) == len(cands) and all(v > 0 for v in trials.values())
    assert trials[autotune.mapping_name(best)] == max(trials.values())
    assert cache.exists()

    def no_timing(*a, **k):
        raise AssertionError("a cached choice was timed again")

    monkeypatch.setattr(autotune, "time_mapping", no_timing)
    again, trials2 = autotune.tune(masks, 19, storage, steps=8, cache_path=str(cache), **ARGS)
    assert again == best and trials2 == trials

    res = []
    for cfg in ({"tile_a": 4, "block_nodes": 0, "persistent": 0}, best):
        b = lbm.BatchSolver(masks, 19, cfg["tile_a"], storage=storage, block_nodes=cfg["block_nodes"],
                            persistent=cfg["persistent"], prefetch_blocks=cfg.get("prefetch_blocks", 0), **ARGS)
        try:
            b.step(40)
            res.append([b.export_pdfs(k) for k in range(len(masks))])
        finally:
            b.close()
    for a, c, m in zip(res[0], res[1], masks):
        fl = m.astype(bool)
        assert np.array_equal(a[:, fl].view(np.uint64), c[:, fl].view(np.uint64))
