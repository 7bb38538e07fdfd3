"""Host-side parts of the cost model that need no GPU: the shipped weights file is a consistent
network for the library's feature and class layout, and the training-graph recipe is seeded,
covers its four families and stays inside its scale range."""
import json

import numpy as np

import graphgen as gg
from paper_1904_02241_gb300 import costmodel as cm


def test_weights_file_is_a_consistent_network():
    d = json.load(open(cm.WEIGHTS))
    W1, W2, W3 = (np.asarray(d[k]) for k in ("W1", "W2", "W3"))
    assert W1.shape == (cm.N_FEATURES, cm.HIDDEN) and W2.shape == (cm.HIDDEN, cm.HIDDEN)
    assert tuple(d["heads"]) == cm.HEADS and W3.shape == (cm.HIDDEN, sum(cm.HEADS))
    assert len(d["b1"]) == len(d["b2"]) == cm.HIDDEN and len(d["b3"]) == sum(cm.HEADS)
    assert d["block_classes"] == [str(c) for c in cm.BLOCK_CLASSES]  # stored as strings
    assert d["lb_classes"] == cm.LB_CLASSES and d["dir_classes"] == cm.DIR_CLASSES
    assert d["tau_classes"] == cm.TAU_CLASSES and d["push_classes"] == cm.PUSH_CLASSES
    assert cm.BFS_HEURISTIC[0] in cm.TAU_CLASSES and cm.BFS_HEURISTIC[1] in cm.PUSH_CLASSES
    sd = np.asarray(d["sd"])
    assert sd.shape == (cm.N_FEATURES,) and np.all(sd > 0)
    for k in ("W1", "W2", "W3", "b1", "b2", "b3", "mu"):
        assert np.all(np.isfinite(np.asarray(d[k]))), k


def test_training_recipe_is_seeded_and_covers_the_families():
    a, b = cm.graph_specs(40, seed=1000, scale_lo=14, scale_hi=24), cm.graph_specs(40, seed=1000, scale_lo=14,
                                                                                  scale_hi=24)
    assert a == b
    kinds = [s["kind"] for s in a]
    assert {k: kinds.count(k) for k in set(kinds)} == {"rmat": 10, "er": 10, "plc": 10, "grid": 10}
    for s in a:
        if s["kind"] == "rmat":
            assert 14 <= s["scale"] <= 24 and 0.45 <= s["a"] <= 0.65
        elif s["kind"] in ("er", "plc"):
            assert 1 << 14 <= s["V"] <= 1 << 24
        else:
            assert 2 ** 7 - 1 <= s["rows"] <= 2 ** 12 and 0.0 <= s["drop"] <= 0.2
        if s["kind"] == "plc":
            assert 2.1 <= s["exp"] <= 2.9
    assert cm.graph_specs(40, seed=1001) != a


def test_small_training_graphs_build_on_the_host():
    for s in cm.graph_specs(8, seed=7, scale_lo=9, scale_hi=10):
        g = cm.make_graph(s, device="cpu")
        rp, ci = g.numpy()
        assert rp[0] == 0 and rp[-1] == g.E and np.all(np.diff(rp) >= 0)
        assert g.E == 0 or (ci.min() >= 0 and ci.max() < g.V)
    assert cm.heuristic_config() == ("pull", "l2", "hybrid")
    assert isinstance(gg.rmat(6), gg.CSRGraph)
