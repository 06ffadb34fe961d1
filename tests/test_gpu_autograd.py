"""The torch.autograd.Functions of paper_1007_1609_gb300.autograd with CUDA
tensors: outputs and gradients stay on the inputs' device and dtype, one
cached lattice serves repeated calls of a geometry, torch.autograd.gradcheck
passes in FP64 (a frozen) on a 6x6 lattice for one self-consistency map, and
the LDOS function's gradients equal cbdg_ldos_backward's and the oracle's."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def setup_6x6(seed=5, M=48):
    import torch
    from paper_1007_1609_gb300.autograd import bond_list
    p = wl.random_swave(6, M, seed=seed, T=0.05)
    bonds = bond_list(6, 6)
    geom = dict(Lx=6, Ly=6, periodic_x=0, periodic_y=0, mu=p.mu, U=p.coupling)
    t = p.hop.reshape(p.N, -1)[bonds[0], bonds[1]].real.copy()
    return p, bonds, geom, t, torch


def test_order_parameter_map_on_cuda_tensors_matches_the_library():
    from paper_1007_1609_gb300.autograd import OrderParameterMap, clear_cache
    p, bonds, geom, t0, torch = setup_6x6()
    dev = torch.device("cuda")
    eps = torch.tensor(p.eps, device=dev, requires_grad=True)
    t = torch.tensor(t0, device=dev, requires_grad=True)
    dl = torch.tensor(p.delta0.real, device=dev, requires_grad=True)
    out = OrderParameterMap.apply(eps, t, dl, geom, p.T, 48, "fp64", None)
    assert out.is_cuda and out.dtype == torch.float64
    ((out - 0.3) ** 2).sum().backward()
    for x in (eps, t, dl):
        assert x.grad.is_cuda and x.grad.dtype == torch.float64
    lat = cbdg.Lattice(p, precision="fp64")
    d, _ = lat.order_parameter(p.T, 48)
    ge, gh, gd = lat.backward(p.T, 48, (2 * (d.real - 0.3)).astype(np.complex128))
    assert np.allclose(out.detach().cpu().numpy(), d.real, rtol=0, atol=1e-14)
    assert np.allclose(eps.grad.cpu().numpy(), ge, rtol=1e-12, atol=1e-14)
    assert np.allclose(dl.grad.cpu().numpy(), gd, rtol=1e-12, atol=1e-14)
    assert np.allclose(t.grad.cpu().numpy(), gh[bonds[0], bonds[1]], rtol=1e-12, atol=1e-14)
    # float32 inputs get float32 gradients; a second geometry gets its own lattice
    eps32 = torch.tensor(p.eps, device=dev, dtype=torch.float32, requires_grad=True)
    out32 = OrderParameterMap.apply(eps32, t.detach(), dl.detach(), geom, p.T, 48, "fp64", None)
    out32.sum().backward()
    assert eps32.grad.dtype == torch.float32 and eps32.grad.is_cuda
    clear_cache()


def test_order_parameter_map_gradcheck_fp64():
    """torch.autograd.gradcheck (central differences against the adjoint) on
    the 6x6 map with the rescale frozen at one value for every evaluation."""
    from paper_1007_1609_gb300.autograd import OrderParameterMap, clear_cache
    p, bonds, geom, t0, torch = setup_6x6(seed=7, M=32)
    a = orc.rescale(as_oracle(p))
    dev = torch.device("cuda")
    eps = torch.tensor(p.eps, device=dev, requires_grad=True)
    t = torch.tensor(t0, device=dev, requires_grad=True)
    dl = torch.tensor(p.delta0.real, device=dev, requires_grad=True)
    f = lambda e_, t_, d_: OrderParameterMap.apply(e_, t_, d_, geom, p.T, 32, "fp64", a)  # noqa: E731
    assert torch.autograd.gradcheck(f, (eps, t, dl), eps=1e-6, atol=1e-7, rtol=1e-5)
    clear_cache()


def test_local_dos_gradients_match_library_and_oracle():
    from paper_1007_1609_gb300.autograd import LocalDOS, clear_cache
    p, bonds, geom, t0, torch = setup_6x6(seed=9, M=40)
    ol = as_oracle(p)
    a = orc.rescale(ol)
    dev = torch.device("cuda")
    sites = np.array([0, 14, 21, 35], dtype=np.int32)
    E = np.linspace(-0.7, 0.7, 11) * a
    eps = torch.tensor(p.eps, device=dev, requires_grad=True)
    t = torch.tensor(t0, device=dev, requires_grad=True)
    dl = torch.tensor(p.delta0.real, device=dev, requires_grad=True)
    rho = LocalDOS.apply(eps, t, dl, geom, sites, E, 40, "jackson", 0.0, "fp64", None)
    assert rho.is_cuda and rho.shape == (4, 11)
    orho = orc.ldos(ol, a, sites, 40, E)
    assert np.abs(rho.detach().cpu().numpy() - orho).max() < 1e-5 * np.abs(orho).max()
    w = torch.tensor(np.random.default_rng(2).normal(size=(4, 11)), device=dev, dtype=torch.float32)
    (rho * w).sum().backward()
    oe, oh, od = orc.ldos_gradient(ol, a, sites, 40, E, w.double().cpu().numpy())
    scale = max(np.abs(oe).max(), np.abs(oh).max(), np.abs(od).max())
    assert np.abs(eps.grad.cpu().numpy() - oe).max() < 1e-9 * scale
    assert np.abs(dl.grad.cpu().numpy() - od).max() < 1e-9 * scale
    assert np.abs(t.grad.cpu().numpy() - oh[bonds[0], bonds[1]]).max() < 1e-9 * scale
    clear_cache()
