"""CUDA-graph replay of the ensemble's steps (flood_set_graphs): runs of
steps captured once and replayed must give, bit for bit, what the same steps
launched one by one give, on every engine, with land cover (tiles outside the
domain skipped), with the running maximum, and when the launch arguments
change between windows (which captures again)."""
import numpy as np
import pytest

from paper_2302_08341_gb300 import synth
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def capi():
    return require_gpu()


def _run(capi, graphs, engine=1, land=False, track=False, reshape=None, windows=(120.0, 240.0)):
    ny, nx, M = 150, 300, 5
    terr = synth.make_terrain(ny, nx, seed=71)
    hy = synth.hyetograph_constant(90.0, 600.0)
    rm, sc = synth.ensemble_prior(71, M)
    with capi.Grid(terr.z, terr.n) as g:
        if land:
            cls = synth.land_cover(terr, seed=71, pond_side=(6, 14))
            g.set_land_cover(cls, synth.LAND_CLASSES)
        g.ensemble_init(M, rm, sc, hy)
        if land:
            n_m, d_m = synth.land_prior(71, M)
            g.set_land_params(n_m, d_m)
        g.set_engine(engine)
        if track:
            g.track_max_depth(True)
        g.set_graphs(graphs)
        launches = []
        for i, t in enumerate(windows):
            if reshape is not None and i == 1:
                g.set_launch(*reshape)
            c0 = g.launch_count
            g.advance_to(t)
            launches.append(g.launch_count - c0)
        g.sync()
        states = [np.stack(g.get_state(m)) for m in range(M)]
        hm = [g.max_depth(m) for m in range(M)] if track else []
        out = dict(states=states, members=g.members(), volumes=g.volumes(), hm=hm,
                   stats=g.graph_stats(), launches=launches)
        if land:
            out["drained"] = g.drained()
        return out


def _same(a, b):
    for x, y in zip(a["states"], b["states"]):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    for x, y in zip(a["hm"], b["hm"]):
        np.testing.assert_array_equal(x.view(np.uint32), y.view(np.uint32))
    for k in ("t", "steps", "rain_mult", "scale", "hmax"):
        np.testing.assert_array_equal(a["members"][k], b["members"][k])
    for k, v in a["volumes"].items():
        np.testing.assert_array_equal(v, b["volumes"][k])
    if "drained" in a:
        np.testing.assert_array_equal(a["drained"], b["drained"])
    # the replayed steps count their kernels as launches too
    assert a["launches"] == b["launches"]


@pytest.mark.parametrize("engine,land,track", [(1, False, False), (0, False, False),
                                               (2, False, False), (1, True, False),
                                               (0, True, False), (1, False, True)])
def test_graph_replay_matches_plain_launches(capi, engine, land, track):
    plain = _run(capi, False, engine, land, track)
    graph = _run(capi, True, engine, land, track)
    _same(plain, graph)
    assert plain["stats"] == (0, 0)
    captures, replays = graph["stats"]
    assert captures == 2          # one per window: t_end is a launch argument
    assert replays >= 8           # about 120 steps of 1 s per window, runs of 24


def test_a_changed_launch_shape_captures_again(capi):
    plain = _run(capi, False, reshape=(32, 1))
    graph = _run(capi, True, reshape=(32, 1))
    _same(plain, graph)
    assert graph["stats"][0] == 2


def test_timed_steps_launch_plainly(capi):
    ny, nx, M = 64, 140, 4
    terr = synth.make_terrain(ny, nx, seed=72)
    hy = synth.hyetograph_constant(60.0, 600.0)
    rm, sc = synth.ensemble_prior(72, M)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, hy)
        g.set_graphs(True)
        g.profile(True)
        g.advance_to(60.0)
        ms, n = g.profile(False)
        assert g.graph_stats() == (0, 0) and n >= 60 and ms > 0
        g.advance_to(120.0)
        assert g.graph_stats()[1] >= 2
