"""Adjoint of one self-consistency map on general lattices
(cbdg_order_parameter_backward with complex vectors): Peierls hoppings of a
uniform field, next-nearest neighbours, complex on-site Delta_i, and
nearest-neighbour bond (d-wave) pairing, against the oracle's general
reverse mode (orc.map_gradient_general, pinned by central differences).
Complex gradients dL/dRe + i dL/dIm per hopping, on-site Delta and bond
Delta; FP64 within 1e-9 of the oracle relative to the largest component,
the FP32 (complex64) recursion within 1e-3."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

K = 1 << 14


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


CASES = {
    "field_nnn_onsite_6": lambda M: wl.random_swave(6, M, seed=31, periodic=1, complex_delta=True, flux_quanta=1.0,
                                                    tp=-0.3, T=0.05),
    "field_onsite_open_7": lambda M: wl.random_swave(7, M, seed=32, periodic=0, complex_delta=True,
                                                     flux_quanta=0.0, T=0.05),
    "dwave_field_6": lambda M: wl.random_dwave(6, M, seed=33, flux_quanta=1.0, T=0.05),
    "dwave_5": lambda M: wl.random_dwave(5, M, seed=34, T=0.05),
}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("M", [2, 40])
@pytest.mark.parametrize("case", sorted(CASES))
def test_general_backward_matches_oracle(case, M, precision, tol):
    p = CASES[case](M)
    lat = cbdg.Lattice(p, precision=precision, complex_field=True)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    ol = as_oracle(p)
    a = orc.rescale(ol)
    rng = np.random.default_rng(M + len(case))
    shape = (p.N, 4) if p.pairing == wl.BOND else (p.N,)
    g = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    if p.pairing == wl.BOND:
        g = g * (np.abs(p.delta0) > 0)
    ge, gh, gd = lat.backward(p.T, M, g)
    assert lat.rescale == pytest.approx(a, rel=1e-14)
    C = orc.fold_coefficients(M, K, a, p.T)
    oe, oh, od = orc.map_gradient_general(ol, a, C, g)
    if M == 2:
        # two moments: only C_0, C_1; the gradients are those of the first step
        assert np.abs(oe).max() + np.abs(oh).max() + np.abs(od).max() > 0
    assert rel(ge, oe) < tol and rel(gh, oh) < tol and rel(gd, od) < tol, (rel(ge, oe), rel(gh, oh), rel(gd, od))
    lat.close()


def test_general_backward_with_bond_couplings():
    """Per-bond V_{i,d} (cbdg_set_coupling) enters the source of each bond."""
    p = wl.random_dwave(6, 32, seed=35, flux_quanta=1.0, T=0.05)
    rng = np.random.default_rng(9)
    lat0 = as_oracle(p)
    V = np.zeros((p.N, 4))
    for i in range(p.N):
        for d in (0, 2):
            j = orc.neighbour(lat0, i, d)
            V[i, d] = V[j, d ^ 1] = rng.uniform(0.5, 2.0)
    lat = cbdg.Lattice(p, precision="fp64", complex_field=True)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    lat.set_coupling(V)
    g = rng.normal(size=(p.N, 4)) + 1j * rng.normal(size=(p.N, 4))
    ge, gh, gd = lat.backward(p.T, p.M, g)
    ol = orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu, p.hop, p.pairing, p.coupling, p.delta0,
                     coupling_site=V.reshape(-1))
    a = orc.rescale(ol)
    oe, oh, od = orc.map_gradient_general(ol, a, orc.fold_coefficients(p.M, K, a, p.T), g)
    assert rel(ge, oe) < 1e-9 and rel(gh, oh) < 1e-9 and rel(gd, od) < 1e-9


def test_real_lattice_gradients_are_complex_with_zero_imaginary_parts():
    p = wl.random_swave(6, 24, seed=36, T=0.05)
    lat = cbdg.Lattice(p, precision="fp64")
    w = np.random.default_rng(1).normal(size=p.N)
    ge, gh, gd = lat.backward(p.T, p.M, w.astype(np.complex128))
    assert gh.dtype == np.complex128 and gd.dtype == np.complex128
    assert np.abs(gh.imag).max() == 0.0 and np.abs(gd.imag).max() == 0.0
    ol = as_oracle(p)
    a = orc.rescale(ol)
    oe, oh, od = orc.scf_map_gradient(ol, a, orc.fold_coefficients(p.M, K, a, p.T), w)
    assert rel(ge, oe) < 1e-9 and rel(gh.real, oh) < 1e-9 and rel(gd.real, od) < 1e-9


@pytest.mark.parametrize("shape", [(70, 5, 24, 1, True), (130, 3, 20, 1, False), (66, 4, 18, 0, True)])
def test_fp32_general_backward_wide_rows(shape):
    """The FP32 gradient sums of general lattices run one CTA per block of
    64 sites of a lattice row (whole rows staged); rows wider than 64 sites
    take several blocks, with the periodic x wrap between the first and the
    last.  Against the oracle's reverse mode (1e-3) and the FP64 path (1e-3)."""
    from tests.test_gpu_temporal_cplx import rect_general
    Lx, Ly, M, periodic, bond = shape
    p = rect_general(Lx, Ly, M, seed=Lx + Ly, periodic=periodic, flux=1.0 if periodic else 0.0, tp=-0.3, bond=bond)
    rng = np.random.default_rng(Lx)
    shp = (p.N, 4) if bond else (p.N,)
    g = rng.normal(size=shp) + 1j * rng.normal(size=shp)
    if bond:
        g = g * (np.abs(p.delta0) > 0)
    out = {}
    for prec in ("fp32", "fp64"):
        lat = cbdg.Lattice(p, precision=prec, complex_field=True)
        cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
        out[prec] = lat.backward(p.T, M, g)
        a = lat.rescale
        lat.close()
    ol = as_oracle(p)
    oe, oh, od = orc.map_gradient_general(ol, a, orc.fold_coefficients(M, K, a, p.T), g)
    for got, ref in zip(out["fp32"], (oe, oh, od)):
        assert rel(got, ref) < 1e-3, rel(got, ref)
    for got, ref in zip(out["fp64"], (oe, oh, od)):
        assert rel(got, ref) < 1e-9, rel(got, ref)

