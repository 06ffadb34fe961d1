"""Batched ensembles of disordered lattices of uneven size (persistent
recursion launch per iteration, CUDA-graph-replayed self-consistency) vs
the oracle's self-consistency loop run sample by sample.  The recursion is
FP32 with FP64 folds: converged Delta within 1e-4."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

K = 1 << 14


def test_small_ensemble_converges_like_the_oracle():
    probs = wl.ensemble(n_samples=9, sides=(5, 8, 11, 13, 17), M=96)
    ens = cbdg.Ensemble(probs)
    ens.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    ok, it, mask = ens.scf(0.01, 96, 0.5, 1e-4, 200)
    assert ok and mask.all()
    oits = []
    for s, p in enumerate(probs):
        od, hist, _, oit = orc.scf(as_oracle(p), p.T, 96, K, 0.5, 1e-4, 200)
        oits.append(oit)
        assert max_abs(ens.delta(s), od) < 1e-4, (s, max_abs(ens.delta(s), od))
    assert abs(it - max(oits)) <= 1  # the slowest sample sets the iteration count


def test_ensemble_matches_single_lattice_path():
    """Each member after 3 iterations equals the single-lattice FP32 path."""
    probs = wl.ensemble(n_samples=5, sides=(7, 9, 16), M=64)
    ens = cbdg.Ensemble(probs)
    ens.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    ok, it, mask = ens.scf(0.01, 64, 0.5, 0.0, 3)
    assert it == 3 and not mask.any()
    for s, p in enumerate(probs):
        lat = cbdg.Lattice(p, precision="fp32")
        cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
        for _ in range(3):
            lat.scf_step(p.T, 64, 0.5)
        assert max_abs(ens.delta(s), lat.delta) < 1e-5


@pytest.mark.parametrize("M", [64, 66, 68])
def test_uneven_members_match_the_oracle_for_every_step_remainder(M):
    """Members of uneven shape -- tall, wide (two sites per thread), two and
    one rows, a ragged last column slab -- through three-step passes while
    three steps remain, then single steps (M = 64, 66, 68: 31, 32 and 33
    steps).  Delta_out of one iteration (2 Delta_1 - Delta_0) vs the oracle
    at every site, and vs the single-lattice FP32 path."""
    from tests.test_gpu_parity import rect
    shapes = [(96, 5), (5, 96), (70, 2), (13, 1), (33, 17), (1, 40)]
    probs = [rect(lx, ly, M, seed=lx * 31 + ly + M, periodic=0) for lx, ly in shapes]
    ens = cbdg.Ensemble(probs)
    ens.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    ok, it, mask = ens.scf(0.02, M, 0.5, 0.0, 1)
    assert it == 1
    for s, p in enumerate(probs):
        ol = as_oracle(p)
        a = orc.rescale(ol)
        od, _ = orc.order_parameter(ol, a, p.T, M, K)
        dout = 2 * ens.delta(s) - p.delta0
        assert max_abs(dout, od) < 1e-5, (p.name, max_abs(dout, od))
        lat = cbdg.Lattice(p, precision="fp32")
        cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
        lat.scf_step(p.T, M, 0.5)
        assert max_abs(ens.delta(s), lat.delta) < 1e-5
        lat.close()


def test_full_ensemble_first_iteration_sampled():
    """The full ensemble workload (256 samples, sides 32..96, M = 512) for one
    iteration: Delta_out = 2 Delta_1 - Delta_0 at sampled sites of sampled
    samples vs the oracle."""
    probs = wl.ensemble()
    ens = cbdg.Ensemble(probs)
    ens.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    ok, it, mask = ens.scf(0.01, 512, 0.5, 0.0, 1)
    assert it == 1
    rng = np.random.default_rng(4)
    for s in (0, 77, 255):
        p = probs[s]
        ol = as_oracle(p)
        a = orc.rescale(ol)
        sites = rng.choice(p.N, 3, replace=False).astype(np.int32)
        od, _ = orc.order_parameter_sites(ol, a, p.T, 512, K, sites)
        dout = 2 * ens.delta(s)[sites] - p.delta0[sites]
        assert max_abs(dout, od) < 1e-4, (s, max_abs(dout, od))
