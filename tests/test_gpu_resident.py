"""The shared-memory-resident recursion for small real lattices
(CBDG_OPT_RESIDENT, on by default): moments and order parameter against the
FP64 oracle and against the streamed kernels, up to the largest lattices
that fit on chip."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs
from tests.test_gpu_parity import K, TOL, gpu_lattice, rect

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

CASES = {
    "clean16_M256": lambda: wl.swave_clean(16, 256),
    "ragged7x5_M33": lambda: rect(7, 5, 33, seed=3, periodic=0),
    "periodic6x9_M64": lambda: rect(6, 9, 64, seed=4, periodic=1),
    "chain1x12_M20": lambda: rect(1, 12, 20, seed=5, periodic=0),
    "chain13x1_M21": lambda: rect(13, 1, 21, seed=6, periodic=0),
    "single_site_M8": lambda: rect(1, 1, 8, seed=7, periodic=0),
    "rect40x24_M48": lambda: rect(40, 24, 48, seed=8, periodic=0),
    "max48x48_M64": lambda: rect(48, 48, 64, seed=9, periodic=0),
}


def resident_used(lat):
    W, D, split = lat.last_tile()
    return D == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_moments_match_oracle_and_streamed(case, precision):
    p = CASES[case]()
    sites = np.arange(p.N, dtype=np.int32)
    lat = gpu_lattice(p, precision)
    ee, eh = lat.moments(sites, p.M)
    assert resident_used(lat), lat.last_tile()
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    tol = TOL[precision][0]
    assert max_abs(ee, oee) < tol and max_abs(eh, oeh) < tol, (max_abs(ee, oee), max_abs(eh, oeh))
    ref = gpu_lattice(p, precision, resident=0)
    ree, reh = ref.moments(sites, p.M)
    assert not resident_used(ref)
    close = 1e-13 if precision == "fp64" else 2e-6
    assert max_abs(ee, ree) < close and max_abs(eh, reh) < close


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["clean16_M256", "periodic6x9_M64", "max48x48_M64"])
def test_order_parameter_matches_oracle(case, precision):
    p = CASES[case]()
    lat = gpu_lattice(p, precision)
    d, n = lat.order_parameter(p.T, p.M)
    assert resident_used(lat)
    od, on = orc.order_parameter(as_oracle(p), lat.rescale, p.T, p.M, K)
    tol = TOL[precision][1]
    assert max_abs(d, od) < tol and max_abs(n, on) < tol, (max_abs(d, od), max_abs(n, on))


def test_sampled_sites_and_repeats():
    p = rect(20, 17, 40, seed=12, periodic=0)
    rng = np.random.default_rng(3)
    sites = np.concatenate([rng.choice(p.N, 37, replace=False), [0, 0]]).astype(np.int32)
    lat = gpu_lattice(p, "fp64")
    ee, eh = lat.moments(sites, p.M)
    assert resident_used(lat)
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < 1e-11 and max_abs(eh, oeh) < 1e-11


def test_too_large_lattice_streams():
    p = rect(64, 64, 16, seed=13, periodic=0)
    lat = gpu_lattice(p, "fp64")
    lat.moments(np.arange(p.N, dtype=np.int32), p.M)
    assert not resident_used(lat)


def test_spectrum_violation_is_reported_on_chip():
    p = rect(8, 8, 64, seed=14, periodic=0)
    lat = gpu_lattice(p, "fp64", fixed_rescale_pico=int(0.5e12))  # a far inside the band
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.moments(np.arange(p.N, dtype=np.int32), p.M)
    assert ei.value.status == cbdg.CBDG_ERR_SPECTRUM
