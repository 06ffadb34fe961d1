"""CUDA-graph replay of self-consistency iterations (CBDG_OPT_GRAPH): the
replayed iterations give exactly the results of direct launches, and a graph
is dropped when an option changes or a buffer is reallocated."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs
from tests.test_gpu_parity import K, gpu_lattice, rect

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def iterate(lat, p, n):
    diffs = [lat.scf_step(p.T, p.M, p.mix) for _ in range(n)]
    return diffs, lat.delta


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_replay_equals_direct_launches(precision):
    p = wl.swave_clean(16, 256)
    direct = gpu_lattice(p, precision, graph=0)
    replay = gpu_lattice(p, precision)
    d0, delta0 = iterate(direct, p, 10)
    l0 = cbdg.cbdg_launch_count(direct.handle)
    d1, delta1 = iterate(replay, p, 10)
    l1 = cbdg.cbdg_launch_count(replay.handle)
    assert d0 == d1
    assert np.array_equal(delta0, delta1)
    assert l0 == l1  # replays count the kernels of the captured iteration


def test_replay_matches_oracle_scf():
    p = wl.swave_clean(16, 64, iters=6)
    lat = gpu_lattice(p, "fp64")
    for _ in range(6):
        lat.scf_step(p.T, p.M, p.mix)
    ol = as_oracle(p)
    od, _hist, _n, _it = orc.scf(ol, p.T, p.M, K, p.mix, 0.0, 6)
    assert max_abs(lat.delta, od) < 1e-10


def test_graph_dropped_on_option_change_and_reallocation():
    p = rect(12, 10, 40, seed=21, periodic=0)
    ref = gpu_lattice(p, "fp64", graph=0)
    lat = gpu_lattice(p, "fp64")
    for _ in range(3):  # direct, capture, replay
        assert lat.scf_step(p.T, p.M, p.mix) == ref.scf_step(p.T, p.M, p.mix)
    # an option change (a different slab width) must not replay the old graph
    lat.set_option(cbdg.CBDG_OPT_SLAB_WIDTH, 2)
    ref.set_option(cbdg.CBDG_OPT_SLAB_WIDTH, 2)
    for _ in range(3):
        assert lat.scf_step(p.T, p.M, p.mix) == ref.scf_step(p.T, p.M, p.mix)
    # a larger moment count reallocates buffers; later iterations stay exact
    sites = np.arange(p.N, dtype=np.int32)
    lat.moments(np.concatenate([sites, sites]), 2 * p.M)
    ref.moments(np.concatenate([sites, sites]), 2 * p.M)
    for _ in range(3):
        assert lat.scf_step(p.T, p.M, p.mix) == ref.scf_step(p.T, p.M, p.mix)
    assert np.array_equal(lat.delta, ref.delta)
    # a different temperature is a different graph
    assert lat.scf_step(0.05, p.M, p.mix) == ref.scf_step(0.05, p.M, p.mix)
    assert np.array_equal(lat.delta, ref.delta)
