"""Temporal blocking (several recursion steps of Eq. 15 per pass over the
vectors) against the FP64 oracle.

The multi-step kernel serves real on-site FP32 lattices with open edges along
y; everything else falls back to one step per pass.  Tolerances are those of
the FP32 recursion: 1e-5 on moments and 1e-4 on Delta_i.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs
from tests.test_gpu_parity import K, gpu_lattice, rect

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL_MOM, TOL_DELTA = 1e-5, 1e-4


def grouped(Lx, steps, slab, depth=0):
    """Shapes the multi-step kernel serves: one lattice site per thread (256
    threads, slab/4 threads per site) for any K, two sites per thread for K = 2,
    and two sites per thread for K = 3 in the lean pass (slab 16, depth 1)."""
    per_thread = 2 if steps == 2 else 1
    if Lx <= per_thread * 256 // (slab // 4):
        return True
    return steps == 3 and slab == 16 and depth in (0, 1) and Lx <= 128


def recursion_launches(lat, sites, M):
    lat.set_option(cbdg.CBDG_OPT_PROFILE, 1)
    cbdg.cbdg_profile_read(lat.handle, reset=True)
    out = lat.moments(sites, M)
    _, n, _ = cbdg.cbdg_profile_read(lat.handle, reset=True)
    return out, n


@pytest.mark.parametrize("slab", [8, 16])
@pytest.mark.parametrize("depth", [1, 2])
@pytest.mark.parametrize("steps", [2, 3, 4])
@pytest.mark.parametrize("case", [(7, 5, 33), (40, 24, 48), (80, 3, 17), (3, 2, 64), (64, 9, 10)])
def test_moments_match_oracle(case, steps, depth, slab):
    Lx, Ly, M = case
    p = rect(Lx, Ly, M, seed=Lx * 31 + Ly, periodic=0)
    sites = np.arange(p.N, dtype=np.int32)
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=steps, pipeline_depth=depth, slab_width=slab)
    (ee, eh), launches = recursion_launches(lat, sites, M)
    n_steps = (M + 1) // 2 - 1
    # the grouped launches ran: K steps per pass, then single steps for the rest
    if grouped(Lx, steps, slab, depth):
        assert launches == n_steps // steps + n_steps % steps
    else:
        assert launches == n_steps
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, M)
    assert max_abs(ee, oee) < TOL_MOM, max_abs(ee, oee)
    assert max_abs(eh, oeh) < TOL_MOM, max_abs(eh, oeh)
    lat.close()


@pytest.mark.parametrize("steps", [2, 4])
def test_same_as_one_step_per_pass(steps):
    """Same arithmetic in the same order per level: the multi-step result
    equals the one-step-per-pass result to FP32 rounding of the sums."""
    p = rect(33, 17, 65, seed=5, periodic=0)
    sites = np.arange(p.N, dtype=np.int32)[::-1].copy()
    one = gpu_lattice(p, "fp32", resident=0, temporal_steps=1).moments(sites, p.M)
    got = gpu_lattice(p, "fp32", resident=0, temporal_steps=steps).moments(sites, p.M)
    assert max_abs(got[0], one[0]) < 1e-6 and max_abs(got[1], one[1]) < 1e-6


def test_periodic_y_falls_back_to_one_step():
    p = rect(6, 9, 40, seed=4, periodic=1)
    sites = np.arange(p.N, dtype=np.int32)
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=4)
    (ee, eh), launches = recursion_launches(lat, sites, p.M)
    assert launches == (p.M + 1) // 2 - 1
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < TOL_MOM and max_abs(eh, oeh) < TOL_MOM


def test_option_range():
    p = rect(4, 4, 8, seed=2, periodic=0)
    lat = gpu_lattice(p, "fp32")
    for bad in (-1, 5):
        with pytest.raises(cbdg.CbdgError):
            lat.set_option(cbdg.CBDG_OPT_TEMPORAL_STEPS, bad)
    lat.set_option(cbdg.CBDG_OPT_TEMPORAL_STEPS, 3)
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_OPT_TEMPORAL_STEPS) == 3


@pytest.mark.parametrize("slab", [16, 8])
@pytest.mark.parametrize("case", [(65, 7, 40), (100, 23, 33), (128, 2, 64), (128, 31, 129), (97, 64, 24),
                                  (64, 19, 37), (33, 40, 26)])
def test_lean_three_steps_match_oracle(case, slab):
    """Three steps per pass: at slab 16 and 64 < Lx <= 128 the lean pass
    (two sites per thread, level 0 read from its shared-memory ring,
    parameters in a ring of their own, FP32 column sums flushed into FP64
    every few rows), otherwise one site per thread with every level in
    register windows.  Moments vs the oracle, and vs one step per pass."""
    Lx, Ly, M = case
    p = rect(Lx, Ly, M, seed=Lx * 7 + Ly, periodic=0)
    sites = np.arange(p.N, dtype=np.int32)[::-1].copy()
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=3, slab_width=slab)
    (ee, eh), launches = recursion_launches(lat, sites, M)
    n_steps = (M + 1) // 2 - 1
    assert launches == n_steps // 3 + n_steps % 3
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 3
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, M)
    assert max_abs(ee, oee) < TOL_MOM, max_abs(ee, oee)
    assert max_abs(eh, oeh) < TOL_MOM, max_abs(eh, oeh)
    one = gpu_lattice(p, "fp32", resident=0, temporal_steps=1).moments(sites, M)
    assert max_abs(ee, one[0]) < 5e-6 and max_abs(eh, one[1]) < 5e-6


@pytest.mark.parametrize("Lx,slab", [(100, 16), (100, 8), (40, 8)])
def test_lost_copy_times_out_in_the_lean_pass(Lx, slab):
    """The bounded waits of the three-step pass (the lean pass at slab 16,
    one site per thread at slab 8): a copy that never arrives makes the call
    report CBDG_ERR_CUDA, and the lattice then computes correct moments."""
    p = rect(Lx, 12, 40, seed=52, periodic=0)
    sites = np.arange(p.N, dtype=np.int32)
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=3, wait_limit_ms=20, test_stall_copy=1,
                      slab_width=slab)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.moments(sites, p.M)
    assert ei.value.status == cbdg.CBDG_ERR_CUDA and "gave up waiting" in str(ei.value)
    lat.set_option(cbdg.CBDG_OPT_TEST_STALL_COPY, 0)
    (ee, eh), launches = recursion_launches(lat, sites, p.M)
    assert launches == 19 // 3 + 19 % 3
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < TOL_MOM and max_abs(eh, oeh) < TOL_MOM


@pytest.mark.parametrize("steps,slab", [(2, 16), (3, 8), (4, 8), (3, 16)])
def test_full_size_disordered_128_sampled(steps, slab):
    """The 128x128 disordered workload at M = 1024, all 16384 start vectors:
    Delta_out and n at sampled sites vs the oracle."""
    p = wl.swave_disordered(128, 1024, seed=1001)
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=steps, slab_width=slab, profile=1)
    d, n = lat.order_parameter(p.T, p.M)
    _, launches, _ = cbdg.cbdg_profile_read(lat.handle, reset=True)
    assert launches == 511 // steps + 511 % steps
    ol = as_oracle(p)
    rng = np.random.default_rng(11)
    sample = np.concatenate([[0, 127, 128 * 64 + 64, p.N - 1],
                             rng.choice(p.N, 6, replace=False)]).astype(np.int32)
    od, on = orc.order_parameter_sites(ol, lat.rescale, p.T, p.M, K, sample)
    assert max_abs(d[sample], od) < TOL_DELTA, max_abs(d[sample], od)
    assert max_abs(n[sample], on) < TOL_DELTA, max_abs(n[sample], on)
    assert np.all(np.abs(d) <= 0.5 * p.coupling + 1e-9)


def tall_disordered(Lx, Ly, M, seed):
    """Open Lx x Ly s-wave lattice of the 128x128 workload's physics (eps_i ~
    U[-0.5, 0.5], t = 1, mu = -0.5, U = 2, T = 0.01, Delta = 0.5)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = Lx * Ly
    return wl.Problem(name=f"tall{Lx}x{Ly}", Lx=Lx, Ly=Ly, periodic_x=0, periodic_y=0,
                      eps=rng.uniform(-0.5, 0.5, size=N), mu=-0.5, hop=wl.square_hops(Lx, Ly, 0, 0),
                      pairing=wl.ONSITE, coupling=2.0, delta0=np.full(N, 0.5 + 0j), T=0.01, M=M)


@pytest.mark.parametrize("slab", [16, 8])
@pytest.mark.parametrize("shape", [(128, 1024, 256), (128, 512, 1024), (96, 2048, 128)])
def test_lean_pass_tall_lattices_match_oracle(shape, slab):
    """Three steps per pass on lattices much taller than wide: in the lean
    pass (slab 16) each thread's FP32 column sums are flushed into FP64 every
    few rows, at slab 8 (one site per thread) they are Kahan-compensated, so
    in neither does their error grow with Ly.  Moments of 16 sampled start sites (among
    them the first and last rows) vs the oracle at the FP32 moment tolerance;
    at M = 1024 on 128 x 512 every start vector spreads over the whole
    height."""
    Lx, Ly, M = shape
    p = tall_disordered(Lx, Ly, M, seed=Lx + Ly)
    rng = np.random.default_rng(Ly)
    sites = np.concatenate([[0, Lx - 1, p.N - Lx, p.N - 1, (Ly // 2) * Lx + Lx // 2],
                            rng.choice(p.N, 11, replace=False)]).astype(np.int32)
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=3, slab_width=slab)
    (ee, eh), launches = recursion_launches(lat, sites, M)
    n_steps = (M + 1) // 2 - 1
    assert launches == n_steps // 3 + n_steps % 3
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 3
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, M)
    assert max_abs(ee, oee) < TOL_MOM, max_abs(ee, oee)
    assert max_abs(eh, oeh) < TOL_MOM, max_abs(eh, oeh)
    lat.close()


def test_lean_pass_tall_lattice_order_parameter_sampled():
    """Delta_out and n_i of one self-consistency map on the 128 x 512 lattice
    at M = 1024 with all 65536 start vectors (the lean pass), at sampled sites
    vs the oracle."""
    p = tall_disordered(128, 512, 1024, seed=640)
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=3)
    d, n = lat.order_parameter(p.T, p.M)
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 3
    rng = np.random.default_rng(12)
    sample = np.concatenate([[0, 127, 256 * 128 + 64, p.N - 1],
                             rng.choice(p.N, 6, replace=False)]).astype(np.int32)
    od, on = orc.order_parameter_sites(as_oracle(p), lat.rescale, p.T, p.M, K, sample)
    assert max_abs(d[sample], od) < TOL_DELTA, max_abs(d[sample], od)
    assert max_abs(n[sample], on) < TOL_DELTA, max_abs(n[sample], on)
    lat.close()


def test_lost_copy_times_out_in_the_two_step_kernel():
    """Failure detection without a fault in the two-step pass: the stall hook
    makes the first staged row of every CTA expect 16 bytes that never
    arrive; the bounded wait runs out (20 ms), the call reports
    CBDG_ERR_CUDA, and the same lattice then computes correct moments."""
    p = rect(24, 16, 40, seed=51, periodic=0)
    sites = np.arange(p.N, dtype=np.int32)
    lat = gpu_lattice(p, "fp32", resident=0, temporal_steps=2, wait_limit_ms=20, test_stall_copy=1)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.moments(sites, p.M)
    assert ei.value.status == cbdg.CBDG_ERR_CUDA and "gave up waiting" in str(ei.value)
    lat.set_option(cbdg.CBDG_OPT_TEST_STALL_COPY, 0)
    (ee, eh), launches = recursion_launches(lat, sites, p.M)
    assert launches == 19 // 2 + 19 % 2  # the two-step kernel ran
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < TOL_MOM and max_abs(eh, oeh) < TOL_MOM


@pytest.mark.parametrize("case", [(150, 50, 40, 8, 16), (150, 12, 40, 4, 37), (300, 33, 33, 4, 20),
                                  (500, 19, 24, 4, 12), (200, 3, 17, 8, 24), (140, 64, 21, 4, 300)])
def test_row_blocks_match_oracle_and_one_step(case):
    """Lattices too wide for the whole-column pass run two steps per pass over
    row blocks on request (CBDG_OPT_TEMPORAL_STEPS = 2): each CTA recomputes
    K - t halo rows of level t on either side of its rows, writes the two new
    vectors out of place and sums its own rows only.  Few start sites, so the rows split into several blocks (ragged last
    block, blocks shorter than the halo at Ly = 3).  Moments vs the oracle
    and vs one step per pass."""
    Lx, Ly, M, slab, n_sites = case
    p = rect(Lx, Ly, M, seed=Lx + Ly, periodic=0)
    rng = np.random.default_rng(Lx)
    sites = np.sort(rng.choice(p.N, min(n_sites, p.N), replace=False)).astype(np.int32)
    lat = gpu_lattice(p, "fp32", resident=0, slab_width=slab, temporal_steps=2)
    (ee, eh), launches = recursion_launches(lat, sites, M)
    n_steps = (M + 1) // 2 - 1
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 2
    assert launches == n_steps // 2 + n_steps % 2
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, M)
    assert max_abs(ee, oee) < TOL_MOM, max_abs(ee, oee)
    assert max_abs(eh, oeh) < TOL_MOM, max_abs(eh, oeh)
    one = gpu_lattice(p, "fp32", resident=0, slab_width=slab, temporal_steps=1).moments(sites, M)
    assert max_abs(ee, one[0]) < 5e-6 and max_abs(eh, one[1]) < 5e-6


def test_row_blocks_order_parameter():
    """Delta_out and n of every site through row-block passes (all sites as
    start vectors on a 160 x 24 lattice at slab width 8) vs the oracle."""
    p = rect(160, 24, 48, seed=77, periodic=0)
    lat = gpu_lattice(p, "fp32", resident=0, slab_width=8, temporal_steps=2)
    d, n = lat.order_parameter(p.T, p.M)
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 2
    od, on = orc.order_parameter(as_oracle(p), lat.rescale, p.T, p.M, K)
    assert max_abs(d, od) < TOL_DELTA and max_abs(n, on) < TOL_DELTA


def test_lost_copy_times_out_in_row_blocks():
    """The bounded waits of the row-block pass: a copy that never arrives
    makes the call report CBDG_ERR_CUDA; the lattice then computes correct
    moments."""
    p = rect(150, 20, 30, seed=53, periodic=0)
    sites = np.arange(0, p.N, 97, dtype=np.int32)
    lat = gpu_lattice(p, "fp32", resident=0, slab_width=4, temporal_steps=2, wait_limit_ms=20, test_stall_copy=1)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.moments(sites, p.M)
    assert ei.value.status == cbdg.CBDG_ERR_CUDA and "gave up waiting" in str(ei.value)
    lat.set_option(cbdg.CBDG_OPT_TEST_STALL_COPY, 0)
    ee, eh = lat.moments(sites, p.M)
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 2
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < TOL_MOM and max_abs(eh, oeh) < TOL_MOM

