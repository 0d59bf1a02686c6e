"""GPU tests of the runtime options: the single-precision application
replayed from captured CUDA graphs (opts.graph) gives bit for bit the
results of direct launches -- applications, solves and time steps, where
every step's new geometry re-captures the graphs -- and keeps the profiler's
events around the near sum; the tile-shape autotuner (opts.autotune) keeps
the fastest shape it timed, and the tuned operator meets the same
tolerances (2e-5 against FP64 for single-precision pairs, 1e-10 residual).
Two solutions that both meet a 1e-10 residual differ by up to the condition
number times that; the tuned and the default-shape solutions are compared at
1e-8."""
import numpy as np
import pytest

from paper_1912_04501_gb300 import workloads

pytestmark = pytest.mark.gpu

bie = pytest.importorskip("paper_1912_04501_gb300.bie")


def _cells():
    return [workloads.small_cell(n_bodies=4, nodes=128, seed=3, phi=0.25),
            workloads.two_ellipses(2e-3, 160)]


def test_graph_replay_is_bitwise():
    for cells in (_cells()[0], _cells()):
        g = bie.Context(cells, precision=bie.BIE_MIXED, graph=1)
        d = bie.Context(cells, precision=bie.BIE_MIXED, graph=0)
        sigma = np.random.default_rng(1).standard_normal(2 * g.N)
        for _ in range(2):  # the second call replays the captured graphs
            assert np.array_equal(g.apply(sigma, precision=bie.BIE_MIXED), d.apply(sigma, precision=bie.BIE_MIXED))
        sg, ig = g.solve()
        sd, idd = d.solve()
        assert np.array_equal(sg, sd) and ig == idd
        g.profile(True)
        mg, _ = g.step(1e-3, 3)
        md, _ = d.step(1e-3, 3)
        assert np.array_equal(mg, md)
        a, b = g.get_state(), d.get_state()
        assert np.array_equal(a["xc"], b["xc"]) and np.array_equal(a["sigma"], b["sigma"])
        p = g.profile_read()
        assert p["near32_launches"] > 0 and p["near32_ms"] > 0
        g.close()
        d.close()


def test_autotune_keeps_fastest_shape():
    cell = workloads.config2()
    t = bie.Context(cell, precision=bie.BIE_MIXED, autotune=1)
    shape, ms = t.near_shape()
    assert 0 <= shape < bie.BIE_NEAR32_SHAPES and all(m > 0 for m in ms)
    assert ms[shape] == min(ms), (shape, ms)
    ref = bie.Context(cell, precision=bie.BIE_MIXED)
    assert ref.near_shape() == (0, [0.0] * bie.BIE_NEAR32_SHAPES)
    sigma = np.random.default_rng(2).standard_normal(2 * t.N)
    y64 = t.apply(sigma, precision=bie.BIE_FP64)
    y32 = t.apply(sigma, precision=bie.BIE_MIXED)
    err = np.abs(y32 - y64).max() / np.abs(y64).max()
    assert err < 2e-5, err
    st, it = t.solve()
    sr, ir = ref.solve()
    assert it["rel_residual"] <= 1e-10, it
    diff = np.abs(st - sr).max() / np.abs(sr).max()
    assert diff < 1e-8, diff
    t.close()
    ref.close()
