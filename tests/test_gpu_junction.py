"""Site-dependent coupling (cbdg_set_coupling) and the junction workloads.

Per-site U_i (zero on normal-metal sites) and per-bond V_{i,d} enter Eq. 19
through the fold; the order parameter, the self-consistency loop and the
map gradient are compared with the oracle (same coupling array), on small
lattices in both precisions and on the S/N slab at full size (the printed
500-site plane x 320 layers, M = 2048, one start site per layer through the
plane's translation symmetry) on sampled sites, with its surface LDOS under
the Lorentz kernel of Eq. 16.  Tolerances as in the other parity tests: Delta 1e-10 (FP64) and
1e-4 (FP32); gradients 1e-9 relative (FP64); LDOS 1e-5 of the absolute
series (3xTF32 contraction)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import gpu_available, max_abs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

K = 1 << 14
TOL = {"fp64": 1e-10, "fp32": 1e-4}


def oracle_lattice(p, cpl, delta=None):
    return orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu, p.hop, p.pairing, p.coupling,
                       p.delta0 if delta is None else delta, coupling_site=cpl)


def gpu_lattice(p, precision, cpl, **opts):
    lat = cbdg.Lattice(p, precision=precision)
    lat.set_option(cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    for k, v in opts.items():
        lat.set_option(getattr(cbdg, "CBDG_OPT_" + k.upper()), v)
    lat.set_coupling(cpl)
    return lat


def strip_coupling(p, U=2.0, width=3):
    """U on the first `width` columns' complement, 0 on a normal strip."""
    x = np.arange(p.N) % p.Lx
    return np.where(x < p.Lx - width, U, 0.0)


def bond_coupling(p, seed):
    lat0 = oracle_lattice(p, None)
    rng = np.random.default_rng(seed)
    V = np.zeros((p.N, 4))
    for i in range(p.N):
        for d in (0, 2):
            j = orc.neighbour(lat0, i, d)
            if j >= 0:
                V[i, d] = V[j, d ^ 1] = rng.uniform(0.0, 2.0)
    return V


CASES = {
    "real_open_9": lambda M: (lambda p: (p, strip_coupling(p)))(wl.random_swave(9, M, seed=401, T=0.05)),
    "field_8": lambda M: (lambda p: (p, strip_coupling(p)))(
        wl.random_swave(8, M, seed=402, periodic=1, complex_delta=True, flux_quanta=2.0, T=0.05)),
    "nnn_field_7": lambda M: (lambda p: (p, strip_coupling(p, width=2)))(
        wl.random_swave(7, M, seed=403, periodic=1, complex_delta=True, flux_quanta=2.0, tp=-0.3, T=0.05)),
    "dwave_bonds_6": lambda M: (lambda p: (p, bond_coupling(p, 5)))(wl.random_dwave(6, M, seed=404, T=0.05)),
}


@pytest.mark.parametrize("resident", [1, 0])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_site_coupling_order_parameter(case, precision, resident):
    M = 64
    p, cpl = CASES[case](M)
    lat = gpu_lattice(p, precision, cpl, resident=resident)
    d, n = lat.order_parameter(p.T, M)
    ol = oracle_lattice(p, cpl)
    od, on = orc.order_parameter(ol, orc.rescale(ol), p.T, M, K)
    assert max_abs(d, od) < TOL[precision], max_abs(d, od)
    assert max_abs(n, on) < TOL[precision]
    if p.pairing == wl.ONSITE:
        assert np.all(d[cpl == 0.0] == 0.0)
    lat.set_coupling(None)  # back to the scalar
    d0, _ = lat.order_parameter(p.T, M)
    od0, _ = orc.order_parameter(oracle_lattice(p, None), orc.rescale(ol), p.T, M, K)
    assert max_abs(d0, od0) < TOL[precision]


@pytest.mark.parametrize("symmetric", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sn_slab_small_scf(precision, symmetric):
    """Five mixed self-consistency iterations of a small S/N slab (graph
    replay from the third call) against the oracle's loop, with every site a
    start vector or one per layer (cbdg_set_symmetry with the plane's
    translations)."""
    p = wl.sn_slab(Lx=8, L_S=12, L_N=4, M=128, T=0.02)
    cpl = p.extra["coupling_site"]
    lat = gpu_lattice(p, precision, cpl)
    if symmetric:
        lat.set_symmetry(p.extra["symmetry"])
    for _ in range(5):
        lat.scf_step(p.T, p.M, p.mix)
    ref, _, _, _ = orc.scf(oracle_lattice(p, cpl), p.T, p.M, K, p.mix, 0.0, 5)
    assert max_abs(lat.delta, ref) < TOL[precision], max_abs(lat.delta, ref)
    y = np.arange(p.N) // p.Lx
    assert np.all(lat.delta[y >= 12] == 0.0)


def test_symmetry_reduction_equals_every_site():
    """One recursion per representative gives the same Delta_out and n as one
    per site (FP64, to round-off of the column reductions), also after
    switching back; invalid maps and bond pairing are rejected."""
    p = wl.sn_slab(Lx=10, L_S=9, L_N=5, M=96, T=0.02)
    cpl = p.extra["coupling_site"]
    full = gpu_lattice(p, "fp64", cpl)
    d_all, n_all = full.order_parameter(p.T, p.M)
    sym = gpu_lattice(p, "fp64", cpl)
    sym.set_symmetry(p.extra["symmetry"])
    cbdg.cbdg_launch_count(sym.handle, reset=True)
    d_sym, n_sym = sym.order_parameter(p.T, p.M)
    assert max_abs(d_sym, d_all) < 1e-13 and max_abs(n_sym, n_all) < 1e-13
    sym.set_symmetry(None)
    d_back, _ = sym.order_parameter(p.T, p.M)
    assert max_abs(d_back, d_all) < 1e-13
    bad = p.extra["symmetry"].copy()
    bad[3] = 5  # 5 is not its own representative
    with pytest.raises(cbdg.CbdgError) as ei:
        sym.set_symmetry(bad)
    assert ei.value.status == cbdg.CBDG_ERR_INVALID_ARG
    q = wl.random_dwave(4, 16, seed=2)
    lq = cbdg.Lattice(q, precision="fp64")
    with pytest.raises(cbdg.CbdgError) as ei:
        lq.set_symmetry(np.zeros(q.N, dtype=np.int32))
    assert ei.value.status == cbdg.CBDG_ERR_UNSUPPORTED


def test_site_coupling_gradient_matches_oracle():
    p = wl.random_swave(8, 64, seed=405, T=0.05)
    cpl = strip_coupling(p, U=2.5)
    lat = gpu_lattice(p, "fp64", cpl)
    lat.order_parameter(p.T, p.M)
    a = lat.rescale
    w = np.random.default_rng(8).normal(size=p.N)
    ge, gh, gd = lat.backward(p.T, p.M, w.astype(np.complex128))
    C = orc.fold_coefficients(p.M, K, a, p.T)
    oe, oh, od = orc.scf_map_gradient(oracle_lattice(p, cpl), a, C, w)
    for g, o in ((ge, oe), (gh, oh), (gd, od)):
        assert max_abs(g, o) < 1e-9 * np.abs(o).max()


def test_set_coupling_validation():
    p, V = CASES["dwave_bonds_6"](16)
    lat = gpu_lattice(p, "fp64", None)
    bad = V.copy()
    bad[0, 0] += 0.5                      # no longer symmetric
    with pytest.raises(cbdg.CbdgError):
        lat.set_coupling(bad)
    bad = V.copy()
    bad[3, 2] = np.nan
    with pytest.raises(cbdg.CbdgError):
        lat.set_coupling(bad)
    lat.set_coupling(V)
    d, _ = lat.order_parameter(p.T, 16)
    od, _ = orc.order_parameter(oracle_lattice(p, V), orc.rescale(oracle_lattice(p, V)), p.T, 16, K)
    assert max_abs(d, od) < 1e-10


def test_sns_junction_small_currents():
    """A small S/N/S junction with a phase difference across the normal layer
    and a Gaussian impurity: bond currents against the oracle."""
    p = wl.sns_junction(L_S=5, L_N=4, W=7, M=96, r0=(3, 7), phase=np.pi / 2, T=0.05)
    cpl = p.extra["coupling_site"]
    lat = gpu_lattice(p, "fp64", cpl)
    J = lat.bond_currents(p.T, p.M)
    ol = oracle_lattice(p, cpl)
    ref = 2.0 * orc.bond_currents(ol, orc.rescale(ol), p.T, p.M, K)
    assert max_abs(J, ref) < 1e-10
    assert np.abs(J).max() > 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_sn_slab_full_size_sampled(precision):
    """The S/N slab workload (the printed 500-site plane, 320 layers, U = 0
    on the top 20 rows, M = 2048): Delta_out of one self-consistency map on
    the GPU with one start site per layer (the plane's translations), at
    sampled sites (bulk S, interface, N) against the oracle, and the surface
    LDOS with the Lorentz kernel (broadening 0.001 t) against the oracle's."""
    p = wl.sn_slab()
    cpl = p.extra["coupling_site"]
    lat = gpu_lattice(p, precision, cpl)
    lat.set_symmetry(p.extra["symmetry"])
    d, _ = lat.order_parameter(p.T, p.M)
    ol = oracle_lattice(p, cpl)
    a = orc.rescale(ol)
    assert lat.rescale == pytest.approx(a, rel=1e-14)
    L = p.Lx
    sample = np.array([5, L * 150 + 7, L * 299 + 3, L * 300 + 3, L * 319 + L - 1], dtype=np.int32)
    od, _ = orc.order_parameter_sites(ol, a, p.T, p.M, K, sample)
    assert max_abs(d[sample], od) < TOL[precision], max_abs(d[sample], od)
    assert np.all(d[L * 300:] == 0.0)
    if precision == "fp64":
        return
    lam = lat.lorentz_lambda(p.extra["broadening"], p.M)
    # the ABI's lambda = broadening * M / a (Eq. 16 and the paragraph after it) for the current Delta
    assert lam == pytest.approx(p.extra["broadening"] * p.M / a, rel=1e-14)
    E = p.extra["energy_frac"] * 0.5 * a        # within +-0.025 a of the band centre
    surf = p.extra["surface_sites"][:3]
    rho = lat.ldos(surf, p.M, E, kernel="lorentz", lam=lam)
    mu_ee, _ = orc.moments(ol, a, surf, p.M)
    orho = orc.ldos_from_moments(mu_ee, a, E, kernel=1, lam=lam)
    # bound: 1e-5 of the absolute series of Eq. 17 at each (site, E)
    g = orc.lorentz(p.M, lam) * np.where(np.arange(p.M) == 0, 1.0, 2.0)
    x = E / a
    T = np.cos(np.arange(p.M)[:, None] * np.arccos(x)[None, :])
    scale = (np.abs(mu_ee * g) @ np.abs(T)) / (np.pi * a * np.sqrt(1 - x * x))
    assert np.all(np.abs(rho - orho) <= 1e-5 * scale), (np.abs(rho - orho) / scale).max()
