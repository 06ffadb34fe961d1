"""Adjoint of a loss on the LDOS (cbdg_ldos_backward): the gradient of
L = sum_{c,e} G[c,e] LDOS(E_e, i_c) (Eq. 17 with Eq. 10, a frozen) with
respect to eps_i, the bond hoppings and Delta_i, against the oracle's
reverse mode (orc.ldos_gradient, itself pinned by central differences and
quadrature closed forms) and against central differences of the GPU's own
FP64 moments.  Tolerances as for the self-consistency map's adjoint: FP64
within 1e-9 of the oracle relative to the largest component and 1e-6 of
finite differences; the FP32 recursion within 1e-3 of the FP64 gradient."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("kernel,lam", [("jackson", 0.0), ("lorentz", 2.5)])
@pytest.mark.parametrize("L,M,periodic", [(8, 64, 0), (7, 33, 1), (10, 5, 0), (1, 12, 0)])
def test_ldos_backward_matches_oracle_gradient(precision, tol, kernel, lam, L, M, periodic):
    p = wl.random_swave(L, M, seed=70 + L, periodic=periodic, T=0.05)
    lat = cbdg.Lattice(p, precision=precision)
    rng = np.random.default_rng(L + M)
    sites = rng.choice(p.N, size=min(p.N, 9), replace=False).astype(np.int32)
    sites = np.concatenate([sites, sites[:2]])  # a repeated site counts twice
    ol = as_oracle(p)
    a = orc.rescale(ol)
    E = np.linspace(-0.9, 0.85, 13) * a
    G = rng.normal(size=(sites.size, E.size))
    ge, gh, gd = lat.ldos_backward(sites, M, E, G, kernel=kernel, lam=lam)
    assert lat.rescale == pytest.approx(a, rel=1e-14)
    oe, oh, od = orc.ldos_gradient(ol, a, sites, M, E, G, 0 if kernel == "jackson" else 1, lam)
    assert rel(ge, oe) < tol and rel(gh, oh) < tol and rel(gd, od) < tol, (rel(ge, oe), rel(gh, oh), rel(gd, od))
    lat.close()


def gpu_weights(M, E, a):
    """Eq. 17's weights w_m(E) = (2 - delta_m0) g_m T_m(E/a) / (pi a sqrt(1 - (E/a)^2)),
    Jackson g_m, restated here for the finite-difference loss."""
    n = np.arange(M)
    q = np.pi / (M + 1)
    g = ((M - n + 1) * np.cos(n * q) + np.sin(n * q) / np.tan(q)) / (M + 1)
    x = E / a
    w = (np.where(n == 0, 1.0, 2.0) * g)[:, None] * np.cos(n[:, None] * np.arccos(x)[None, :])
    return w / (np.pi * a * np.sqrt(1 - x * x))[None, :]


def test_ldos_backward_full_size_vs_finite_differences_and_oracle():
    """The differentiation workload's lattice (64x64 open, eps ~ U[-0.5, 0.5],
    M = 512) with a loss on the LDOS at 48 sampled sites x 24 energies: FP64
    adjoint vs the oracle's gradient, vs central differences (h = 1e-6) of
    L = sum G . (W^T mu) built from the GPU's FP64 moments, with a frozen; the
    FP32 recursion's gradient vs the FP64 one."""
    p = wl.gradient_case()
    ol = as_oracle(p)
    a = orc.rescale(ol)
    rng = np.random.default_rng(21)
    sites = rng.choice(p.N, size=48, replace=False).astype(np.int32)
    sites[:3] = [0, 2080, 4095]
    E = np.linspace(-0.8, 0.8, 24) * a
    G = rng.normal(size=(sites.size, E.size))
    lat = cbdg.Lattice(p, precision="fp64")
    ge, gh, gd = lat.ldos_backward(sites, p.M, E, G)
    oe, oh, od = orc.ldos_gradient(ol, a, sites, p.M, E, G)
    assert rel(ge, oe) < 1e-9 and rel(gh, oh) < 1e-9 and rel(gd, od) < 1e-9
    S = G @ gpu_weights(p.M, E, a).T  # dL/dmu [n_sites, M]

    def loss(eps=None, hop=None, delta=None):
        q = wl.Problem(name="fd", Lx=p.Lx, Ly=p.Ly, periodic_x=0, periodic_y=0,
                       eps=p.eps if eps is None else eps, mu=p.mu, hop=p.hop if hop is None else hop,
                       pairing=0, coupling=p.coupling, delta0=p.delta0 if delta is None else delta, T=p.T, M=p.M)
        lt = cbdg.Lattice(q, precision="fp64")
        lt.freeze_rescale(a)
        mu, _ = lt.moments(sites, p.M)
        lt.close()
        return float((S * mu).sum())

    h = 1e-6
    for i in (0, 2080, 4095, int(sites[5])):
        e1, e2 = p.eps.copy(), p.eps.copy()
        e1[i] += h
        e2[i] -= h
        assert ge[i] == pytest.approx((loss(eps=e1) - loss(eps=e2)) / (2 * h), rel=1e-6, abs=1e-9 * np.abs(ge).max())
        d1, d2 = p.delta0.copy(), p.delta0.copy()
        d1[i] += h
        d2[i] -= h
        assert gd[i] == pytest.approx((loss(delta=d1) - loss(delta=d2)) / (2 * h), rel=1e-6,
                                      abs=1e-9 * np.abs(gd).max())
    for (i, dd) in ((0, 0), (2080, 2), (2079, 0)):
        j = i + 1 if dd == 0 else i + 64
        h1, h2 = p.hop.copy(), p.hop.copy()
        h1[i, dd] += h
        h1[j, dd ^ 1] += h
        h2[i, dd] -= h
        h2[j, dd ^ 1] -= h
        assert gh[i, dd] == pytest.approx((loss(hop=h1) - loss(hop=h2)) / (2 * h), rel=1e-6,
                                          abs=1e-9 * np.abs(gh).max())
    lat32 = cbdg.Lattice(p, precision="fp32")
    g32 = lat32.ldos_backward(sites, p.M, E, G)
    assert rel(g32[0], ge) < 1e-3 and rel(g32[1], gh) < 1e-3 and rel(g32[2], gd) < 1e-3
    lat.close()
    lat32.close()


def test_ldos_backward_device_arrays_and_errors():
    """Device inputs give the host result bit for bit; an energy outside the
    band and a complex lattice are rejected."""
    import torch
    p = wl.random_swave(9, 40, seed=3, T=0.05)
    lat = cbdg.Lattice(p, precision="fp64")
    a = orc.rescale(as_oracle(p))
    sites = np.array([4, 40, 80], dtype=np.int32)
    E = np.linspace(-0.5, 0.5, 7) * a
    G = np.random.default_rng(5).normal(size=(3, 7))
    host = lat.ldos_backward(sites, 40, E, G)
    ds, dE, dG = (torch.from_numpy(x).cuda() for x in (sites, E, G))
    out = [torch.zeros(p.N, dtype=torch.float64, device="cuda"),
           torch.zeros(p.N * 4, dtype=torch.float64, device="cuda"),
           torch.zeros(p.N, dtype=torch.float64, device="cuda")]
    cbdg.cbdg_ldos_backward(lat.handle, ds, 3, 40, cbdg.CBDG_JACKSON, 0.0, dE, 7, dG, out[0], out[1], out[2])
    torch.cuda.synchronize()
    assert np.array_equal(out[0].cpu().numpy(), host[0])
    assert np.array_equal(out[1].cpu().numpy().reshape(p.N, 4), host[1])
    assert np.array_equal(out[2].cpu().numpy(), host[2])
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.ldos_backward(sites, 40, np.array([1.01 * a]), np.ones((3, 1)))
    assert ei.value.status == cbdg.CBDG_ERR_INVALID_ARG
    lat.close()
    q = wl.random_dwave(4, 16, seed=1, flux_quanta=1.0)
    lq = cbdg.Lattice(q, precision="fp64", complex_field=True)
    with pytest.raises(cbdg.CbdgError) as ei:
        lq.ldos_backward(np.array([0], dtype=np.int32), 16, np.array([0.0]), np.ones((1, 1)))
    assert ei.value.status == cbdg.CBDG_ERR_UNSUPPORTED
    lq.close()
