"""Nonlocal Green's functions and bond currents on the GPU against the oracle.

cbdg_green_moments reads the direct recursion (Eq. 15) at chosen target
sites, cbdg_green_function contracts those moments into the retarded G(E) of
gf1, and cbdg_bond_currents folds the nearest-bond moments into the currents
of Eq. 20.  Each is compared element by element with the FP64 oracle on the
same seeded lattices (real, complex field, next-nearest hopping, bond
pairing; ragged site and target lists, several column chunks), and at the
full size of the current benchmark (128 x 128, M = 512) on sampled start
sites plus the properties that hold at any size.

Tolerances: moments as in the other parity tests (1e-11 FP64, 1e-5 FP32);
currents sum about M terms C_n <e_j|T_n|e_i> with sum |C_n| of a few, so the
order-parameter tolerances apply (1e-10 FP64, 1e-4 FP32); G(E) is a sum of M
moments times weights up to 2/(a sin theta), taken relative to max |G|
(1e-10 FP64, 2e-4 FP32)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

K = 1 << 14
TOL_MOM = {"fp64": 1e-11, "fp32": 1e-5}
TOL_J = {"fp64": 1e-10, "fp32": 1e-4}
TOL_G = {"fp64": 1e-10, "fp32": 2e-4}


def rect_real(Lx, Ly, M, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    N = Lx * Ly
    return wl.Problem(name=f"rect{Lx}x{Ly}", Lx=Lx, Ly=Ly, periodic_x=0, periodic_y=0,
                      eps=rng.uniform(-0.5, 0.5, N), mu=-0.5, hop=wl.square_hops(Lx, Ly, 0, 0),
                      pairing=wl.ONSITE, coupling=2.0,
                      delta0=rng.uniform(0.2, 0.8, N).astype(np.complex128), T=0.02, M=M)


CASES = {
    "real_open_12": lambda M: wl.random_swave(12, M, seed=301, T=0.05),
    "field_12": lambda M: wl.random_swave(12, M, seed=302, periodic=1, complex_delta=True,
                                          flux_quanta=2.0, T=0.05),
    "nnn_field_10": lambda M: wl.random_swave(10, M, seed=303, periodic=1, complex_delta=True,
                                              flux_quanta=2.0, tp=-0.3, T=0.05),
    "dwave_field_10": lambda M: wl.random_dwave(10, M, seed=304, flux_quanta=2.0, T=0.05),
    "ragged_7x5": lambda M: rect_real(7, 5, M, seed=305),
}


def gpu_lattice(p, precision, **opts):
    lat = cbdg.Lattice(p, precision=precision)
    lat.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    for k, v in opts.items():
        lat.set_option(getattr(cbdg, "CBDG_OPT_" + k.upper()), v)
    return lat


def currents_oracle(p, M, sites=None):
    lat = as_oracle(p)
    a = orc.rescale(lat)
    return 2.0 * orc.bond_currents(lat, a, p.T, M, K, sites=sites)   # both spins (J_up = J_down)


def ragged(N, rng, n):
    s = rng.choice(N, size=min(n, N), replace=False)
    return np.concatenate([s, s[:1]]).astype(np.int32)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_green_moments_match_oracle(case, precision):
    M = 48
    p = CASES[case](M)
    rng = np.random.default_rng(7)
    sites, targets = ragged(p.N, rng, 37), ragged(p.N, rng, 29)
    lat = gpu_lattice(p, precision)
    a11, a12 = lat.green_moments(sites, targets, M)
    ol = as_oracle(p)
    oe, oh = orc.green_moments(ol, orc.rescale(ol), sites, targets, M)
    assert lat.rescale == pytest.approx(orc.rescale(ol), rel=1e-14)
    tol = TOL_MOM[precision]
    assert max_abs(a11, oe) < tol, max_abs(a11, oe)
    assert max_abs(a12, oh) < tol, max_abs(a12, oh)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_bond_currents_match_oracle(case, precision):
    M = 96
    p = CASES[case](M)
    lat = gpu_lattice(p, precision)
    J = lat.bond_currents(p.T, M)
    ref = currents_oracle(p, M)
    assert max_abs(J, ref) < TOL_J[precision], max_abs(J, ref)
    if case.startswith("real") or case.startswith("ragged"):
        assert np.abs(J).max() < (1e-12 if precision == "fp64" else 1e-6)
    else:
        assert np.abs(ref).max() > 1e-3


@pytest.mark.parametrize("opts", [{"column_chunk": 40}, {"column_chunk": 24, "slab_width": 2}, {"pipeline_depth": 1}])
def test_currents_with_column_chunks_and_tiles(opts):
    """Several column chunks (ragged last chunk) and other tiles give the same
    currents (the accumulators are indexed by start site)."""
    M = 64
    p = CASES["dwave_field_10"](M)
    J0 = gpu_lattice(p, "fp64").bond_currents(p.T, M)
    J1 = gpu_lattice(p, "fp64", **opts).bond_currents(p.T, M)
    assert max_abs(J0, J1) < 1e-13


@pytest.mark.parametrize("kernel,lam", [("jackson", 0.0), ("lorentz", 4.0)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_green_function_matches_oracle(precision, kernel, lam):
    M = 128
    p = CASES["field_12"](M)
    rng = np.random.default_rng(11)
    sites, targets = ragged(p.N, rng, 9), ragged(p.N, rng, 21)
    lat = gpu_lattice(p, precision)
    a = orc.rescale(as_oracle(p))
    E = np.linspace(-0.9 * a, 0.9 * a, 67)
    G11, G12 = lat.green_function(sites, targets, M, E, kernel=kernel, lam=lam)
    ol = as_oracle(p)
    oe, oh = orc.green_moments(ol, a, sites, targets, M)
    kid = 0 if kernel == "jackson" else 1
    R11 = orc.green_function(oe, a, E, kernel=kid, lam=lam)
    R12 = orc.green_function(oh, a, E, kernel=kid, lam=lam)
    scale = max(np.abs(R11).max(), np.abs(R12).max())
    assert max_abs(G11, R11) < TOL_G[precision] * scale, max_abs(G11, R11) / scale
    assert max_abs(G12, R12) < TOL_G[precision] * scale, max_abs(G12, R12) / scale


def test_green_function_diagonal_is_minus_pi_ldos():
    """Im G11_ii(E) = -pi LDOS(E, i) (Eq. 17), the LDOS from its own
    tensor-core path (3xTF32, so the FP32-level tolerance)."""
    M = 128
    p = CASES["field_12"](M)
    lat = gpu_lattice(p, "fp64")
    a = orc.rescale(as_oracle(p))
    sites = np.array([3, 50, 97], dtype=np.int32)
    E = np.linspace(-0.8 * a, 0.8 * a, 40)
    G11, _ = lat.green_function(sites, sites, M, E)
    rho = lat.ldos(sites, M, E)
    for c in range(sites.size):
        assert max_abs(-G11[c, c].imag / np.pi, rho[c]) < 1e-5 * max(1.0, np.abs(rho[c]).max())


def test_green_edge_cases():
    M = 16
    p = CASES["field_12"](M)
    lat = gpu_lattice(p, "fp64")
    a = orc.rescale(as_oracle(p))
    # empty lists: nothing computed, no error
    e11, e12 = lat.green_moments(np.zeros(0, np.int32), np.array([1], np.int32), M)
    assert e11.size == 0 and e12.size == 0
    g11, _ = lat.green_function(np.array([1], np.int32), np.zeros(0, np.int32), M, [0.1])
    assert g11.size == 0
    # M = 2: only j_0 and j_1
    a11, a12 = lat.green_moments(np.array([5], np.int32), np.arange(p.N, dtype=np.int32), 2)
    ol = as_oracle(p)
    oe, oh = orc.green_moments(ol, a, [5], np.arange(p.N), 2)
    assert max_abs(a11, oe) < 1e-15 and max_abs(a12, oh) < 1e-15
    with pytest.raises(cbdg.CbdgError):
        lat.green_moments(np.array([0], np.int32), np.array([p.N], np.int32), M)
    with pytest.raises(cbdg.CbdgError):
        lat.green_moments(np.array([-1], np.int32), np.array([0], np.int32), M)
    with pytest.raises(cbdg.CbdgError):
        lat.green_function(np.array([0], np.int32), np.array([1], np.int32), M, [1.01 * a])
    with pytest.raises(cbdg.CbdgError):
        lat.green_function(np.array([0], np.int32), np.array([1], np.int32), M, [0.0], kernel="lorentz", lam=0.0)
    with pytest.raises(cbdg.CbdgError):
        lat.bond_currents(p.T, 1)
    with pytest.raises(cbdg.CbdgError):
        lat.bond_currents(-1.0, M)
    # the lattice stays usable after the refusals
    J = lat.bond_currents(p.T, M)
    assert max_abs(J, currents_oracle(p, M)) < 1e-10


def test_single_site_and_chain_currents():
    """No bonds on a 1x1 lattice; a periodic-free 13x1 chain with a complex
    Delta gradient carries current only along x."""
    for Lx, Ly in ((1, 1), (13, 1)):
        N = Lx * Ly
        x = np.arange(N) % Lx
        p = wl.Problem(name="chain", Lx=Lx, Ly=Ly, periodic_x=0, periodic_y=0,
                       eps=np.zeros(N), mu=-0.3, hop=wl.square_hops(Lx, Ly, 0, 0), pairing=wl.ONSITE,
                       coupling=2.0, delta0=0.4 * np.exp(0.3j * x), T=0.05, M=32)
        lat = gpu_lattice(p, "fp64")
        J = lat.bond_currents(p.T, 32)
        ref = currents_oracle(p, 32)
        assert max_abs(J, ref) < 1e-10
        assert np.abs(J[:, 2:]).max() == 0.0


def test_normal_state_currents_conserved_64():
    """Delta = 0 on a 64 x 64 periodic lattice with a field: the currents out
    of every site sum to zero and J_{i->j} = -J_{j->i} (two different start
    vectors), at a size the oracle does not run in full."""
    M = 128
    p = wl.random_swave(64, M, seed=306, periodic=1, flux_quanta=4.0, tp=-0.3, T=0.05)
    p.delta0 = np.zeros(p.N, dtype=np.complex128)
    lat = gpu_lattice(p, "fp64")
    J = lat.bond_currents(p.T, M)
    assert np.abs(J).max() > 1e-5          # a weak field: 4 h/2e through 4096 plaquettes
    assert np.abs(J.sum(1)).max() < 1e-11
    Lx = p.Lx
    x, y = np.arange(p.N) % Lx, np.arange(p.N) // Lx
    for d in range(8):
        j = (x + wl.DX[d]) % Lx + Lx * ((y + wl.DY[d]) % p.Ly)
        assert np.abs(J[:, d] + J[j, d ^ 1]).max() < 1e-12
    sample = np.array([0, 777, 2080, 4095], dtype=np.int32)
    ref = currents_oracle(p, M, sites=sample)
    assert max_abs(J[sample], ref) < 1e-10


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_dwave_vortex_128_sampled(precision):
    """The bond-current benchmark workload (d-wave, 128 x 128, two flux
    quanta, M = 512), all 16384 start sites on the GPU; sampled sites against
    the oracle and antisymmetry over every bond."""
    p = wl.currents_dwave(128, 512)
    M = p.M
    lat = gpu_lattice(p, precision)
    J = lat.bond_currents(p.T, M)
    rng = np.random.default_rng(13)
    sample = rng.choice(p.N, size=6, replace=False).astype(np.int32)
    ref = currents_oracle(p, M, sites=sample)
    assert max_abs(J[sample], ref) < TOL_J[precision], max_abs(J[sample], ref)
    Lx = p.Lx
    x, y = np.arange(p.N) % Lx, np.arange(p.N) // Lx
    for d in range(p.n_dirs):
        j = (x + wl.DX[d]) % Lx + Lx * ((y + wl.DY[d]) % p.Ly)
        assert np.abs(J[:, d] + J[j, d ^ 1]).max() < TOL_J[precision]


def test_device_buffers_match_host_buffers():
    """Device (torch) outputs and inputs give the same bits as host arrays for
    the nonlocal moments, the Green's function and the currents."""
    import torch
    M = 40
    p = CASES["nnn_field_10"](M)
    lat = gpu_lattice(p, "fp64")
    sites = np.array([3, 3, 57, 99], dtype=np.int32)
    targets = np.array([3, 4, 13, 3, 98], dtype=np.int32)   # repeats, and the start sites themselves
    h11, h12 = lat.green_moments(sites, targets, M)
    d11 = torch.empty((sites.size, M, targets.size), dtype=torch.complex128, device="cuda")
    d12 = torch.empty_like(d11)
    cbdg.cbdg_green_moments(lat.handle, torch.from_numpy(sites).cuda(), sites.size,
                            torch.from_numpy(targets).cuda(), targets.size, M, d11, d12)
    assert np.array_equal(d11.cpu().numpy(), h11) and np.array_equal(d12.cpu().numpy(), h12)
    a = orc.rescale(as_oracle(p))
    E = np.linspace(-0.7 * a, 0.7 * a, 19)
    g11, g12 = lat.green_function(sites, targets, M, E, kernel="lorentz", lam=2.0)
    G11 = torch.empty((sites.size, targets.size, E.size), dtype=torch.complex128, device="cuda")
    G12 = torch.empty_like(G11)
    cbdg.cbdg_green_function(lat.handle, sites, sites.size, targets, targets.size, M, 1, 2.0,
                             torch.from_numpy(E).cuda(), E.size, G11, G12)
    assert np.array_equal(G11.cpu().numpy(), g11) and np.array_equal(G12.cpu().numpy(), g12)
    J = lat.bond_currents(p.T, M)
    Jd = torch.empty((p.N, 8), dtype=torch.float64, device="cuda")
    cbdg.cbdg_bond_currents(lat.handle, p.T, M, 0, 0.0, Jd)
    assert np.array_equal(Jd.cpu().numpy(), J)
    # only one of the two outputs
    o11 = np.zeros_like(h11)
    cbdg.cbdg_green_moments(lat.handle, sites, sites.size, targets, targets.size, M, o11, None)
    assert np.array_equal(o11, h11)
