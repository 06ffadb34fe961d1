"""Parity of the general recursion (complex Peierls hoppings, next-nearest
neighbours, nearest-neighbour bond pairing) with the FP64 oracle, through
the C ABI.  Tolerances as for the real path: FP64 1e-11 on moments and 1e-10
on Delta; FP32 (complex64 vectors, FP64 folds) 1e-5 and 1e-4."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = {"fp64": (1e-11, 1e-10), "fp32": (1e-5, 1e-4)}
K = 1 << 14

CASES = {
    "swave_field_6x6": lambda M: wl.random_swave(6, M, seed=31, periodic=1, complex_delta=True,
                                                 flux_quanta=2.0),
    "swave_nnn_field_7x7": lambda M: wl.random_swave(7, M, seed=32, periodic=1, complex_delta=True,
                                                     flux_quanta=2.0, tp=-0.3),
    "swave_nnn_real_open_9x5": lambda M: rect_nnn(9, 5, M, seed=33),
    "dwave_field_6x6": lambda M: wl.random_dwave(6, M, seed=34, flux_quanta=2.0),
    "dwave_nnn_5x5": lambda M: wl.random_dwave(5, M, seed=35, tp=-0.3),
    "dwave_nn_only_6x6": lambda M: wl.random_dwave(6, M, seed=37, tp=0.0),
    "dwave_vortex_12x12": lambda M: wl.dwave_vortex(12, M),
}


def rect_nnn(Lx, Ly, M, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    N = Lx * Ly
    return wl.Problem(name=f"nnn{Lx}x{Ly}", Lx=Lx, Ly=Ly, periodic_x=0, periodic_y=0,
                      eps=rng.uniform(-0.5, 0.5, N), mu=-0.5,
                      hop=wl.square_hops(Lx, Ly, 0, 0, t=1.0, tp=-0.3), pairing=wl.ONSITE,
                      coupling=2.0, delta0=rng.uniform(0.2, 0.8, N).astype(np.complex128),
                      T=0.02, M=M)


def gpu_lattice(p, precision, **opts):
    lat = cbdg.Lattice(p, precision=precision, complex_field=True)
    lat.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    for k, v in opts.items():
        lat.set_option(getattr(cbdg, "CBDG_OPT_" + k.upper()), v)
    return lat


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_general_moments_match_oracle(case, precision):
    M = 41
    p = CASES[case](M)
    rng = np.random.default_rng(2)
    sites = np.concatenate([rng.permutation(p.N)[: min(p.N, 29)], [0]]).astype(np.int32)
    lat = gpu_lattice(p, precision)
    ee, eh = lat.moments(sites, M)
    a = lat.rescale
    ol = as_oracle(p)
    assert a == pytest.approx(orc.rescale(ol), rel=1e-14)
    oee, oeh = orc.moments(ol, a, sites, M)
    tol = TOL[precision][0]
    assert max_abs(ee, oee) < tol, max_abs(ee, oee)
    assert max_abs(eh, oeh) < tol, max_abs(eh, oeh)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_general_order_parameter_matches_oracle(case, precision):
    M = 64
    p = CASES[case](M)
    lat = gpu_lattice(p, precision)
    d, n = lat.order_parameter(p.T, M)
    od, on = orc.order_parameter(as_oracle(p), lat.rescale, p.T, M, K)
    tol = TOL[precision][1]
    assert max_abs(d, od) < tol, max_abs(d, od)
    assert max_abs(n, on) < tol, max_abs(n, on)


@pytest.mark.parametrize("opts", [dict(slab_width=1), dict(slab_width=4, row_split=2),
                                  dict(column_chunk=6), dict(pipeline_depth=1)])
def test_general_tiling_options(opts):
    p = wl.random_dwave(6, 24, seed=36, flux_quanta=2.0)
    sites = np.arange(p.N, dtype=np.int32)
    ref = gpu_lattice(p, "fp64").moments(sites, 24)
    alt = gpu_lattice(p, "fp64", **opts).moments(sites, 24)
    assert max_abs(ref[0], alt[0]) < 1e-13 and max_abs(ref[1], alt[1]) < 1e-13
    dref = gpu_lattice(p, "fp64").order_parameter(p.T, 24)[0]
    dalt = gpu_lattice(p, "fp64", **opts).order_parameter(p.T, 24)[0]
    assert max_abs(dref, dalt) < 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dwave_scf_iterations(precision):
    p = wl.dwave_vortex(10, 48)
    lat = gpu_lattice(p, precision)
    hist = [lat.scf_step(p.T, p.M, 0.5) for _ in range(4)]
    od, ohist, _, _ = orc.scf(as_oracle(p), p.T, p.M, K, 0.5, 0.0, 4)
    tol = TOL[precision][1]
    assert max_abs(lat.delta, od) < tol
    assert np.allclose(hist, ohist, atol=tol)


def test_vortex_256_full_lattice_sampled_bonds():
    """The d-wave vortex lattice at its full size (256x256 periodic, t' = -0.3,
    2 h/2e of flux) with all 65536 sites as start vectors in FP32 (complex64)
    at M = 64: bond Delta and n at sampled sites vs the oracle."""
    M = 64
    p = wl.dwave_vortex(256, M)
    lat = gpu_lattice(p, "fp32", workspace_mb=40000)  # four column chunks
    d, n = lat.order_parameter(p.T, M)
    ol = as_oracle(p)
    a = lat.rescale
    assert a == pytest.approx(orc.rescale(ol), rel=1e-14)
    sample = np.array([0, 255, 128 * 256 + 77, 65535], dtype=np.int32)
    od, on = orc.order_parameter_bonds(ol, a, p.T, M, K, sample)
    assert max_abs(d[sample], od) < 1e-4, max_abs(d[sample], od)
    assert max_abs(n[sample], on) < 1e-4
    # d-wave symmetry of the initial bonds survives one map: x and y bonds of opposite sign
    assert np.all(d[:, 0].real > 0) and np.all(d[:, 2].real < 0)


def test_vortex_256_full_moments_sampled_fp64():
    """M = 2048 moments of two start sites on the full 256x256 vortex lattice
    (complex128), including the four bond readouts."""
    p = wl.dwave_vortex(256, 2048)
    sites = np.array([1000, 40000], dtype=np.int32)
    lat = gpu_lattice(p, "fp64")
    ee, eh = lat.moments(sites, p.M)
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < 1e-11
    assert max_abs(eh, oeh) < 1e-11
