"""Launch shapes (persistent or per-journey CTAs, rows per thread, block sizes, one-block sort limit) change
where the work runs, never a result bit; the autotuner picks valid shapes and leaves the context
ready for transform and load."""
import pytest

from parity import exact
from test_gpu_batch import make, on_device

pytestmark = pytest.mark.gpu

SHAPES = [dict(journey_ctas=0, row_unroll=4, small_sort_max=2048, row_block=256, small_journey_max=0, scatter_block=128),
          dict(journey_ctas=1, row_unroll=2, small_sort_max=0, row_block=128, small_journey_max=512, scatter_block=256),
          dict(journey_ctas=3, row_unroll=8, small_sort_max=512, row_block=512, small_journey_max=128, scatter_block=512),
          dict(journey_ctas=2, row_unroll=4, small_sort_max=1024, row_block=128, small_journey_max=0, scatter_block=128),
          dict(journey_ctas=0, row_unroll=4, small_sort_max=2048, row_block=256, small_journey_max=256, scatter_block=512),
          dict(journey_ctas=0, row_unroll=4, small_sort_max=4096, row_block=256, small_journey_max=512, scatter_block=256)]


def tables(p, insts):
    res = p.run_batch(insts)
    return res


def same(a, b):
    for x, y in zip(a, b):
        for part in ("cells", "journeys", "points"):
            for k in x[part]:
                exact(f"{part} {k}", y[part][k], x[part][k])


def test_results_do_not_depend_on_the_launch_shapes():
    import paper_2305_07454_b300 as P

    insts = on_device(make(seed=7, days=1, lo=2e4, hi=2e5, zipf_max=20000))  # journeys above 4096 points
    ref = None
    for prec in (P.FP64, P.FP32):
        ref = None
        with P.Pipeline(materialize_points=1, precision=prec) as p:
            for shape in SHAPES:
                p.tuning = shape
                assert p.tuning == shape
                got = tables(p, insts)
                if ref is None:
                    ref = got
                else:
                    same(ref, got)


def test_autotune_picks_valid_shapes_and_leaves_the_context_extracted():
    import paper_2305_07454_b300 as P

    insts = on_device(make(seed=8, days=1))
    with P.Pipeline(materialize_points=1) as p:
        ref = p.run_batch(insts)
        p.extract_batch(insts)
        t = p.autotune(reps=1)
        assert t["journey_ctas"] in (0, 1, 2, 3) and t["row_unroll"] in (2, 4, 8)
        assert t["small_sort_max"] in (0, 512, 1024, 2048, 4096) and t["row_block"] in (128, 256, 512) and t["ms"] > 0
        assert t["small_journey_max"] in (0, 128, 256, 512) and t["scatter_block"] in (128, 256, 512)
        assert {k: v for k, v in t.items() if k != "ms"} == p.tuning
        p.transform()
        p.load()
        r = p.results()
        rg = p.batch_ranges()
        for i, x in enumerate(ref):
            c0, c1 = rg["cell_begin"][i], rg["cell_begin"][i + 1]
            for k in x["cells"]:
                exact("cells " + k, r["cells"][k][c0:c1], x["cells"][k])


def test_bad_shapes_are_rejected():
    import paper_2305_07454_b300 as P

    with P.Pipeline() as p:
        before = p.tuning
        for bad in (dict(journey_ctas=4), dict(row_unroll=3), dict(small_sort_max=4097), dict(journey_ctas=-1),
                    dict(row_block=64), dict(small_journey_max=513), dict(small_journey_max=-1),
                    dict(scatter_block=1024)):
            with pytest.raises(P.CvetlError) as e:
                p.tuning = bad
            assert e.value.status == P.EINVAL
        assert p.tuning == before
        with pytest.raises(P.CvetlError) as e:
            p.autotune()
        assert e.value.status == P.ESTATE
