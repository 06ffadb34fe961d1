"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 recursion 1e-11 absolute on moments and 1e-10 on Delta_i;
FP32 recursion with FP64 folds 1e-5 on moments and 1e-4 on Delta_i.
Inputs come from the seeded generators in paper_1007_1609_gb300.workloads;
the oracle and the library receive the same arrays.
"""
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


def gpu_lattice(p, precision, **opts):
    lat = cbdg.Lattice(p, precision=precision)
    lat.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    for k, v in opts.items():
        lat.set_option(getattr(cbdg, "CBDG_OPT_" + k.upper()), v)
    return lat


SMALL = {
    "clean16_M256": lambda: wl.swave_clean(16, 256),
    "ragged7x5_M33": lambda: rect(7, 5, 33, seed=3, periodic=0),
    "periodic6x9_M64": lambda: rect(6, 9, 64, seed=4, periodic=1),
    "chain1x12_M20": lambda: rect(1, 12, 20, seed=5, periodic=0),
    "chain13x1_M21": lambda: rect(13, 1, 21, seed=6, periodic=0),
    "single_site_M8": lambda: rect(1, 1, 8, seed=7, periodic=0),
    "wide200x3_M16": lambda: rect(200, 3, 16, seed=8, periodic=0),
}


def rect(Lx, Ly, M, seed, periodic):
    """Rectangular disordered s-wave problem (real), random Delta_i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = Lx * Ly
    eps = rng.uniform(-0.5, 0.5, size=N)
    hop = wl.square_hops(Lx, Ly, periodic if Lx >= 3 else 0, periodic if Ly >= 3 else 0)
    d0 = rng.uniform(0.2, 0.8, size=N).astype(np.complex128)
    return wl.Problem(name=f"rect{Lx}x{Ly}", Lx=Lx, Ly=Ly,
                      periodic_x=periodic if Lx >= 3 else 0, periodic_y=periodic if Ly >= 3 else 0,
                      eps=eps, mu=-0.5, hop=hop, pairing=wl.ONSITE, coupling=2.0, delta0=d0,
                      T=0.02, M=M)


def site_sample(N, rng, n=None):
    """A ragged site list with a repeat (not a multiple of any slab width)."""
    if N <= 3:
        return np.array(list(range(N)) + [0], dtype=np.int32)
    n = n or min(N, 37)
    s = rng.choice(N, size=n, replace=False)
    return np.concatenate([s, s[:1]]).astype(np.int32)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(SMALL))
def test_moments_match_oracle(case, precision):
    p = SMALL[case]()
    M = p.M
    rng = np.random.default_rng(1)
    for sites in (np.arange(p.N, dtype=np.int32), site_sample(p.N, rng)):
        lat = gpu_lattice(p, precision)
        ee, eh = lat.moments(sites, M)
        a = lat.rescale
        ol = as_oracle(p)
        assert a == pytest.approx(orc.rescale(ol), rel=1e-14)
        oee, oeh = orc.moments(ol, a, sites, M)
        tol = TOL[precision][0]
        assert max_abs(ee, oee) < tol, (case, max_abs(ee, oee))
        assert max_abs(eh, oeh) < tol, (case, max_abs(eh, oeh))
        lat.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["clean16_M256", "ragged7x5_M33", "periodic6x9_M64", "wide200x3_M16"])
def test_order_parameter_matches_oracle(case, precision):
    p = SMALL[case]()
    lat = gpu_lattice(p, precision)
    d, n = lat.order_parameter(p.T, p.M)
    ol = as_oracle(p)
    od, on = orc.order_parameter(ol, lat.rescale, p.T, p.M, K)
    tol = TOL[precision][1]
    assert max_abs(d, od) < tol, max_abs(d, od)
    assert max_abs(n, on) < tol, max_abs(n, on)
    # the input Delta is untouched
    assert np.array_equal(lat.delta, p.delta0)


@pytest.mark.parametrize("kernel", ["jackson", "lorentz"])
def test_kernels_and_zero_temperature(kernel):
    p = rect(6, 6, 48, seed=11, periodic=0)
    lat = gpu_lattice(p, "fp64")
    ol = as_oracle(p)
    for T in (0.0, 0.05):
        d, n = lat.order_parameter(T, p.M, kernel=kernel, lam=4.0)
        od, on = orc.order_parameter(ol, lat.rescale, T, p.M, K, kernel=1 if kernel == "lorentz" else 0, lam=4.0)
        assert max_abs(d, od) < 1e-10 and max_abs(n, on) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_scf_ten_iterations_clean16(precision):
    """The 16x16 clean workload: 10 mixed iterations from Delta = 0.5."""
    p = wl.swave_clean(16, 256, iters=10)
    lat = gpu_lattice(p, precision)
    hist = [lat.scf_step(p.T, p.M, p.mix) for _ in range(p.max_iter)]
    od, ohist, _, it = orc.scf(as_oracle(p), p.T, p.M, K, p.mix, 0.0, p.max_iter)
    tol = TOL[precision][1]
    assert max_abs(lat.delta, od) < tol, max_abs(lat.delta, od)
    assert np.allclose(hist, ohist, atol=tol)


def test_fp32_converged_delta_within_1e4():
    """Disordered 16x16, SCF to max|dDelta| < 1e-6 in the oracle and < 1e-4
    on the FP32 path: converged Delta agrees to 1e-4."""
    p = wl.swave_disordered(16, 256, seed=1001)
    od, ohist, _, it = orc.scf(as_oracle(p), p.T, p.M, K, p.mix, 1e-6, 200)
    assert ohist[-1] < 1e-6
    lat = gpu_lattice(p, "fp32")
    for _ in range(200):
        if lat.scf_step(p.T, p.M, p.mix) < 1e-5:
            break
    assert max_abs(lat.delta, od) < 1e-4, max_abs(lat.delta, od)


@pytest.mark.parametrize("opts", [
    dict(slab_width=4), dict(slab_width=8, row_split=3), dict(slab_width=32, row_split=2),
    dict(column_chunk=40), dict(row_split=5), dict(workspace_mb=1), dict(pipeline_depth=1),
    dict(slab_width=2, pipeline_depth=2)])
def test_tiling_options_give_same_result(opts):
    p = rect(12, 10, 40, seed=13, periodic=0)
    sites = np.arange(p.N, dtype=np.int32)
    ref = gpu_lattice(p, "fp64").moments(sites, p.M)
    alt = gpu_lattice(p, "fp64", **opts).moments(sites, p.M)
    assert max_abs(ref[0], alt[0]) < 1e-13 and max_abs(ref[1], alt[1]) < 1e-13


def test_repeatable_bitwise():
    p = rect(16, 16, 64, seed=17, periodic=1)
    lat = gpu_lattice(p, "fp32")
    a = lat.order_parameter(p.T, p.M)
    b = lat.order_parameter(p.T, p.M)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_device_buffers_match_host_buffers():
    torch = pytest.importorskip("torch")
    p = rect(9, 8, 30, seed=19, periodic=0)
    lat = gpu_lattice(p, "fp64")
    sites_h = np.arange(p.N, dtype=np.int32)
    ee_h, eh_h = lat.moments(sites_h, p.M)
    sites_d = torch.arange(p.N, dtype=torch.int32, device="cuda")
    ee_d = torch.zeros((p.N, p.M), dtype=torch.float64, device="cuda")
    eh_d = torch.zeros((p.N, p.M), dtype=torch.complex128, device="cuda")
    cbdg.cbdg_moments(lat.handle, sites_d, p.N, p.M, ee_d, eh_d)
    torch.cuda.synchronize()
    assert np.array_equal(ee_d.cpu().numpy(), ee_h)
    assert np.array_equal(eh_d.cpu().numpy(), eh_h[..., 0])
    dd = torch.zeros(p.N, dtype=torch.complex128, device="cuda")
    nd = torch.zeros(p.N, dtype=torch.float64, device="cuda")
    cbdg.cbdg_order_parameter(lat.handle, p.T, 0, 0.0, p.M, dd, nd)
    dh, nh = lat.order_parameter(p.T, p.M)
    assert np.array_equal(dd.cpu().numpy(), dh) and np.array_equal(nd.cpu().numpy(), nh)


def test_spectrum_violation_is_reported():
    """An under-scaled rescale (a below the spectral radius) makes moments
    grow; the library reports CBDG_ERR_SPECTRUM instead of returning them."""
    p = rect(8, 8, 200, seed=23, periodic=0)
    lat = gpu_lattice(p, "fp64", rescale_milli=300)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.moments(np.arange(4, dtype=np.int32), p.M)
    assert ei.value.status == cbdg.CBDG_ERR_SPECTRUM
    lat.set_option(cbdg.CBDG_OPT_RESCALE_MILLI, 1100)
    lat.moments(np.arange(4, dtype=np.int32), p.M)  # usable afterwards


def test_empty_and_minimal_calls():
    p = rect(5, 5, 2, seed=29, periodic=0)
    lat = gpu_lattice(p, "fp64")
    ee, eh = lat.moments(np.zeros(0, dtype=np.int32), 2)
    assert ee.shape == (0, 2)
    ee, eh = lat.moments(np.arange(25, dtype=np.int32), 2)  # M = 2: start vectors only
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, np.arange(25), 2)
    assert max_abs(ee, oee) < 1e-14 and max_abs(eh, oeh) < 1e-14
    with pytest.raises(cbdg.CbdgError):
        lat.moments(np.array([25], dtype=np.int32), 4)
    with pytest.raises(cbdg.CbdgError):
        lat.order_parameter(-1.0, 8)


# ------------------------------------------------------------- full size


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_disordered_128_sampled(precision):
    """The 128x128 disordered workload at M = 1024 with all 16384 sites as
    start vectors, in the launch configuration the benchmark uses: Delta_out
    and n at sampled sites, and the moments of sampled columns, vs the oracle."""
    p = wl.swave_disordered(128, 1024, seed=1001)
    lat = gpu_lattice(p, precision)
    d, n = lat.order_parameter(p.T, p.M)
    a = lat.rescale
    ol = as_oracle(p)
    assert a == pytest.approx(orc.rescale(ol), rel=1e-14)
    rng = np.random.default_rng(7)
    sample = np.concatenate([[0, 127, 128 * 64 + 64, p.N - 1], rng.choice(p.N, 8, replace=False)]).astype(np.int32)
    od, on = orc.order_parameter_sites(ol, a, p.T, p.M, K, sample)
    tol = TOL[precision][1]
    assert max_abs(d[sample], od) < tol, max_abs(d[sample], od)
    assert max_abs(n[sample], on) < tol, max_abs(n[sample], on)
    ee, eh = lat.moments(sample[:6], p.M)
    oee, oeh = orc.moments(ol, a, sample[:6], p.M)
    assert max_abs(ee, oee) < TOL[precision][0], max_abs(ee, oee)
    assert max_abs(eh, oeh) < TOL[precision][0], max_abs(eh, oeh)
    # properties at every site: |Delta| bounded by U/2, 0 <= n <= 2
    assert np.all(np.abs(d) <= 0.5 * p.coupling + 1e-9)
    assert np.all((n > -1e-9) & (n < 2 + 1e-9))


def test_lost_copy_times_out_and_lattice_stays_usable():
    """Failure detection without a fault: the test hook makes every recursion
    CTA wait for 16 bytes that never arrive; the wait runs out after 20 ms,
    the call reports CBDG_ERR_CUDA, and the same lattice then computes
    correct moments."""
    p = rect(8, 8, 24, seed=41, periodic=0)
    lat = gpu_lattice(p, "fp64", wait_limit_ms=20, test_stall_copy=1)
    sites = np.arange(p.N, dtype=np.int32)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.moments(sites, p.M)
    assert ei.value.status == cbdg.CBDG_ERR_CUDA and "gave up waiting" in str(ei.value)
    lat.set_option(cbdg.CBDG_OPT_TEST_STALL_COPY, 0)
    ee, eh = lat.moments(sites, p.M)
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < 1e-11 and max_abs(eh, oeh) < 1e-11


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotuned_tile(precision):
    p = rect(40, 24, 48, seed=43, periodic=0)
    sites = np.arange(p.N, dtype=np.int32)
    ref = gpu_lattice(p, precision).moments(sites, p.M)
    lat = gpu_lattice(p, precision, autotune=1)
    got = lat.moments(sites, p.M)
    W, D, split = lat.last_tile()
    assert W in (1, 2, 4, 8, 16, 32) and 1 <= D <= 4 and split >= 1
    tol = TOL[precision][0]
    assert max_abs(got[0], ref[0]) < tol and max_abs(got[1], ref[1]) < tol
    again = lat.moments(sites, p.M)  # cached tile: bitwise repeatable
    assert lat.last_tile() == (W, D, split)
    assert np.array_equal(again[0], got[0])
    # FP32 on open edges also weighs two to four steps per pass
    k = cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL)
    assert 1 <= k <= (4 if precision == "fp32" else 1)
