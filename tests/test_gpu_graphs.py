"""CUDA graphs of the UNet forwards: a forward repeated with the same batch
buffers and size is captured once and replayed with one launch call.  The
replayed kernels and their arguments are those of the eager forward, so a
world with graphs answers bit for bit as one without, and its stats show the
replays (fewer host launch calls than kernels)."""
import numpy as np
import pytest

import synth
from oracle import unet as OU

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,autotune", [("tf32", False), ("tf32", True), ("bf16x3", False),
                                                ("fp32", False)])
def test_graph_replays_equal_eager_launches(precision, autotune):
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack(steps=2)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    rects = [(-64, 32, 96, 80), (576, 32, 96, 80), (576, 2000, 96, 80)]
    out = {}
    stats = {}
    for graphs in (True, False):
        W = idf.World(0, st, wts, precision=precision, max_batch=8, autotune=autotune, cuda_graphs=graphs)
        out[graphs] = [W.query(*r, kind=idf.IDF_OUT_METRES) for r in rects]
        stats[graphs] = W.stats()
        W.close()
    g = stats[True]["graphs"]
    print(f"{precision}: {g['captured']} forwards captured, {g['replays']} replayed "
          f"({g['replayed_kernels']} kernels); host launch calls {g['host_launch_calls']} "
          f"of {stats[True]['kernel_launches']} kernels")
    assert g["captured"] > 0 and g["replays"] > g["captured"]
    assert g["host_launch_calls"] < stats[True]["kernel_launches"]
    assert stats[False]["graphs"]["replays"] == 0
    assert stats[True]["kernel_launches"] == stats[False]["kernel_launches"]
    for a, b in zip(out[True], out[False]):
        assert np.array_equal(a, b)


def test_graphs_stay_off_while_profiling():
    import paper_2512_08309_gb300 as idf
    idf.lib()
    st = synth.config2_stack(steps=2)
    wts = [synth.weights([s for _, s in OU.param_shapes(lv)], 0, i) for i, lv in enumerate(st["level"])]
    W = idf.World(0, st, wts, precision="tf32", max_batch=8, profile=True, cuda_graphs=True)
    W.query(-64, 32, 96, 80)
    W.query(576, 32, 96, 80)
    s = W.stats()
    W.close()
    assert s["graphs"]["replays"] == 0 and s["profile"]["conv_tc"]["launches"] > 0
