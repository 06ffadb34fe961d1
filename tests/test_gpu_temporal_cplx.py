"""Two recursion steps (Eq. 15) per pass over the vectors for general
lattices: complex hoppings with Peierls phases, next-nearest neighbours,
on-site or bond (d-wave) pairing, periodic or open edges, FP32 complex
vectors (step_cplx_multi.cu, selected with CBDG_OPT_TEMPORAL_STEPS = 2; the
default for these lattices is one step per pass).

Both vectors of a pass land in HBM, so the moment readouts are those of the
one-step path: with bond pairing the moments come straight from the vectors,
which are bit for bit the one-step path's (the same site update on the same
inputs); with on-site pairing the column sums are formed in another order,
within FP32 rounding.  Against the oracle at the FP32 moment tolerance 1e-5.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL_MOM = 1e-5
K = 1 << 14


def lattice(p, temporal_steps=2, **opts):
    lat = cbdg.Lattice(p, precision="fp32", complex_field=True)
    lat.set_option(cbdg.CBDG_OPT_TEMPORAL_STEPS, temporal_steps)
    lat.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    for k, v in opts.items():
        lat.set_option(getattr(cbdg, "CBDG_OPT_" + k.upper()), v)
    return lat


def rect_general(Lx, Ly, M, seed, periodic, flux, tp, bond):
    """Rectangular general lattice: disorder, optional field and t', random
    complex on-site Delta or random symmetric complex bond amplitudes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = Lx * Ly
    hop = wl.square_hops(Lx, Ly, periodic, periodic, t=1.0, tp=tp, flux_quanta=flux)
    eps = rng.uniform(-0.5, 0.5, N)
    if not bond:
        d = (rng.uniform(0.2, 0.8, N) * np.exp(1j * rng.uniform(-np.pi, np.pi, N))).astype(np.complex128)
        return wl.Problem(name=f"gen{Lx}x{Ly}", Lx=Lx, Ly=Ly, periodic_x=periodic, periodic_y=periodic, eps=eps,
                          mu=-0.5, hop=hop, pairing=wl.ONSITE, coupling=2.0, delta0=d, T=0.02, M=M)
    d = np.zeros((N, 4), dtype=np.complex128)
    for s in range(N):
        x, y = s % Lx, s // Lx
        for dd, (dx, dy) in ((0, (1, 0)), (2, (0, 1))):
            xj, yj = x + dx, y + dy
            if not periodic and (xj >= Lx or yj >= Ly):
                continue
            j = (xj % Lx) + Lx * (yj % Ly)
            val = rng.uniform(0.2, 0.6) * np.exp(1j * rng.uniform(-0.5, 0.5)) * (1 if dd == 0 else -1)
            d[s, dd] = val
            d[j, dd ^ 1] = val
    return wl.Problem(name=f"genb{Lx}x{Ly}", Lx=Lx, Ly=Ly, periodic_x=periodic, periodic_y=periodic, eps=eps,
                      mu=-0.8, hop=hop, pairing=wl.BOND, coupling=1.5, delta0=d, T=0.02, M=M)


CASES = {
    # (Lx, Ly, M, seed, periodic, flux, tp, bond)
    "onsite_field_nnn_periodic": (7, 6, 33, 1, 1, 1.0, -0.3, False),
    "onsite_open_field": (9, 5, 40, 2, 0, 0.0, 0.0, False),
    "onsite_ly3_periodic": (5, 3, 21, 3, 1, 1.0, -0.3, False),
    "bond_field_nnn_periodic": (6, 7, 29, 4, 1, 1.0, -0.3, True),
    "bond_open": (8, 5, 30, 5, 0, 0.0, -0.3, True),
    "bond_nn_periodic_wide": (40, 4, 17, 6, 1, 2.0, 0.0, True),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_two_step_moments_match_oracle_and_one_step(case):
    Lx, Ly, M, seed, periodic, flux, tp, bond = CASES[case]
    p = rect_general(Lx, Ly, M, seed, periodic, flux, tp, bond)
    sites = np.arange(p.N, dtype=np.int32)[::-1].copy()
    two = lattice(p, profile=1)
    ee, eh = two.moments(sites, M)
    _, launches, _ = cbdg.cbdg_profile_read(two.handle, reset=True)
    assert cbdg.cbdg_get_option(two.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 2
    steps = M - 2 if bond else (M + 1) // 2 - 1
    assert launches == steps // 2 + steps % 2
    oee, oeh = orc.moments(as_oracle(p), two.rescale, sites, M)
    assert max_abs(ee, oee) < TOL_MOM, max_abs(ee, oee)
    assert max_abs(eh, oeh) < TOL_MOM, max_abs(eh, oeh)
    one = lattice(p, temporal_steps=0)  # the default: one step per pass
    ee1, eh1 = one.moments(sites, M)
    assert cbdg.cbdg_get_option(one.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 1
    if bond:
        # moments read from the vectors: the same values bit for bit
        assert np.array_equal(ee, ee1) and np.array_equal(eh, eh1)
    else:
        assert max_abs(ee, ee1) < 2e-6 and max_abs(eh, eh1) < 2e-6
    two.close()
    one.close()


def test_two_step_order_parameter_and_currents_on_the_vortex_lattice():
    """The currents workload's physics on a 24x24 periodic lattice (field,
    t', imprinted vortices): bond Delta_out and the bond currents (Eq. 20,
    through the target readout) vs the oracle and equal to the one-step path."""
    p = wl.currents_dwave(24, 48)
    two = lattice(p)
    d2, n2 = two.order_parameter(p.T, p.M)
    assert cbdg.cbdg_get_option(two.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 2
    J2 = two.bond_currents(p.T, p.M)
    one = lattice(p, temporal_steps=1)
    d1, n1 = one.order_parameter(p.T, p.M)
    J1 = one.bond_currents(p.T, p.M)
    assert np.array_equal(d2, d1) and np.array_equal(n2, n1) and np.array_equal(J2, J1)
    ol = as_oracle(p)
    a = orc.rescale(ol)
    od, on = orc.order_parameter(ol, a, p.T, p.M, K)
    assert max_abs(d2, od) < 1e-4 and max_abs(n2, on) < 1e-4
    oJ = 2.0 * orc.bond_currents(ol, a, p.T, p.M, K)
    assert max_abs(J2, oJ) < 1e-4
    two.close()
    one.close()


def test_two_step_vortex_chunk_full_size_sampled():
    """The 256x256 d-wave vortex lattice (field, t', bond pairing) in the
    benchmark's launch shape, 4096 start sites, M = 34: moments equal to the
    one-step path bit for bit, and sampled columns vs the oracle."""
    pv = wl.dwave_vortex(256, 34)
    sites = (np.arange(4096, dtype=np.int64) * (pv.N // 4096)).astype(np.int32)
    two = lattice(pv)
    ee, eh = two.moments(sites, pv.M)
    assert cbdg.cbdg_get_option(two.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 2
    one = lattice(pv, temporal_steps=1)
    ee1, eh1 = one.moments(sites, pv.M)
    assert np.array_equal(ee, ee1) and np.array_equal(eh, eh1)
    pick = np.array([0, 1, 2047, 4095])
    oee, oeh = orc.moments(as_oracle(pv), two.rescale, sites[pick], pv.M)
    assert max_abs(ee[pick], oee) < TOL_MOM and max_abs(eh[pick], oeh) < TOL_MOM
    two.close()
    one.close()


def test_lost_copy_times_out_in_the_two_step_complex_pass():
    """Failure detection without a fault: the stall hook makes the first load
    of every CTA expect 16 bytes that never arrive; the bounded wait runs out
    (20 ms), the call reports CBDG_ERR_CUDA, and the lattice then computes
    correct moments."""
    p = rect_general(6, 5, 20, 7, 1, 1.0, -0.3, True)
    sites = np.arange(p.N, dtype=np.int32)
    lat = lattice(p, wait_limit_ms=20, test_stall_copy=1)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.moments(sites, p.M)
    assert ei.value.status == cbdg.CBDG_ERR_CUDA and "gave up waiting" in str(ei.value)
    assert cbdg.cbdg_get_option(lat.handle, cbdg.CBDG_INFO_LAST_TEMPORAL) == 2
    lat.set_option(cbdg.CBDG_OPT_TEST_STALL_COPY, 0)
    ee, eh = lat.moments(sites, p.M)
    oee, oeh = orc.moments(as_oracle(p), lat.rescale, sites, p.M)
    assert max_abs(ee, oee) < TOL_MOM and max_abs(eh, oeh) < TOL_MOM
    lat.close()
