"""Host logic of the cell-size autotuner (density buckets, cache keys) and,
on the GPU, a tuning run: cells from the candidate set, a second run served
from the cache, and a tuned batch whose results equal the oracle."""
import json

import numpy as np
import pytest
import torch

import cloudgen
from paper_2502_11602_gb300 import autotune


def test_density_bucket_is_log2_of_xy_density():
    rng = np.random.default_rng(0)
    for dens, side in ((5.0, 40.0), (12.0, 30.0), (48.0, 20.0), (60.0, 10.0)):
        n = int(dens * side * side)
        xyz = np.concatenate([rng.uniform(0, side, (n, 2)), rng.normal(0, 1, (n, 1))], 1)
        xyz[0, :2], xyz[1, :2] = 0.0, side  # exact bounding box
        assert autotune.density_bucket(xyz) == int(np.floor(np.log2(n / side ** 2)))


def test_cache_keys_separate_every_parameter():
    keys = {autotune._key("G", d, r, kern, k, p, b)
            for d in (2, 3) for r in (0.5, 1.0) for kern in (0, 1) for k in (0, 16) for p in (0, 1) for b in (2, 3)}
    assert len(keys) == 64


@pytest.mark.gpu
def test_tuning_run_and_cache(tmp_path):
    import oracle
    import paper_2502_11602_gb300 as cg
    xyz, off = cloudgen.batched_tiles(12, 150_000, seed=7)
    path = str(tmp_path / "tune.json")
    cells, report = autotune.tune(xyz, off, radius=1.0, k=8, cache_path=path)
    assert len(cells) == 12 and set(cells.tolist()) <= set(autotune.CANDIDATES)
    assert report and all(v["best"] in autotune.CANDIDATES for v in report.values())
    cells2, report2 = autotune.tune(xyz, off, radius=1.0, k=8, cache_path=path)
    assert report2 == {} and np.array_equal(cells, cells2)
    assert len(json.load(open(path))) == len(report)
    x = torch.from_numpy(xyz).to("cuda:0")
    pipe = cg.Pipeline(x, off, cells, radius=1.0, k=8)
    pipe.run()
    out = pipe.outputs()
    g_off = out["offsets"].cpu().numpy()
    g_ind = out["indices"].cpu().numpy()
    for t in (0, 5, 11):
        a, b = off[t], off[t + 1]
        o_off, o_ind = oracle.Index(xyz[a:b], cells[t]).radius_search(xyz[a:b], 1.0, threads=8)
        assert np.array_equal(g_off[a:b + 1] - g_off[a], o_off)
        assert np.array_equal(g_ind[g_off[a]:g_off[b]], o_ind + a)
    pipe.close()


def test_tuning_record_defaults_and_checks():
    # the launch tuning is host state of the library: no GPU needed
    import paper_2502_11602_gb300 as cg
    cg.cg_set_tuning(None)
    d = cg.cg_get_tuning()
    assert d == {"radius_chunk_height": 8.0, "radius_chunk_max": 256, "count_shape": 0, "fill_shape": 0}
    cg.cg_set_tuning({"radius_chunk_height": 4.0, "count_shape": 2, "fill_shape": 1})
    assert cg.cg_get_tuning() == {"radius_chunk_height": 4.0, "radius_chunk_max": 256, "count_shape": 2,
                                  "fill_shape": 1}
    for bad in ({"count_shape": 3}, {"fill_shape": -1}, {"radius_chunk_height": 0.0},
                {"radius_chunk_max": 0}, {"radius_chunk_max": 513}):
        with pytest.raises(cg.CheeseError):
            cg.cg_set_tuning(bad)
        assert cg.cg_get_tuning()["count_shape"] == 2  # unchanged by a refused call
    cg.cg_set_tuning(None)
    assert cg.cg_get_tuning() == d


@pytest.mark.gpu
def test_tuned_launch_shapes_pipeline_matches_oracle(tmp_path):
    import oracle
    import paper_2502_11602_gb300 as cg
    xyz, off = cloudgen.batched_tiles(10, 300_000, seed=9)
    path = str(tmp_path / "tune.json")
    cells, _ = autotune.tune(xyz, off, radius=1.0, k=0, cache_path=path)
    tuning, report = autotune.tune_launch(xyz, off, cells, radius=1.0, cache_path=path)
    assert report and set(tuning) == {"radius_chunk_height", "count_shape", "fill_shape"}
    assert tuning["count_shape"] in autotune.SHAPES and tuning["fill_shape"] in autotune.SHAPES
    tuning2, report2 = autotune.tune_launch(xyz, off, cells, radius=1.0, cache_path=path)
    assert report2 == {} and tuning2 == tuning
    # launch shapes of a captured batch, timed on the batch
    x = torch.from_numpy(xyz).to("cuda:0")
    shapes, prep = autotune.tune_pipeline(x, off, cells, radius=1.0, k=0, cache_path=path)
    assert set(shapes) == {"count_shape", "fill_shape"} and len(prep) >= 5
    assert autotune.tune_pipeline(x, off, cells, radius=1.0, k=0, cache_path=path) == (shapes, {})
    tuning = dict(tuning, **shapes)
    saved = cg.cg_get_tuning()
    cg.cg_set_tuning(tuning)
    try:
        pipe = cg.Pipeline(torch.from_numpy(xyz).to("cuda:0"), off, cells, radius=1.0, k=0)
        pipe.run()
        out = pipe.outputs()
        g_off = out["offsets"].cpu().numpy()
        g_ind = out["indices"].cpu().numpy()
        pipe.close()
    finally:
        cg.cg_set_tuning(saved)
    for t in (0, 5):
        a, b = off[t], off[t + 1]
        ref = oracle.Index(xyz[a:b], cells[t])
        o_off, o_ind = ref.radius_search(xyz[a:b], 1.0, threads=8)
        assert np.array_equal(g_off[a:b + 1] - g_off[a], o_off)
        assert np.array_equal(g_ind[g_off[a]:g_off[b]], o_ind + a)
