"""Gradient through the self-consistent fixed point (cbdg_fixed_point_backward)
against central finite differences of the oracle's converged self-consistency
loop (a frozen), on a small disordered lattice: FP64 within 1e-6 relative, FP32
within 1e-3 of FP64."""
import dataclasses

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from tests._common import as_oracle, gpu_available
from tests.test_gpu_parity import K, gpu_lattice, rect

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

T, M, MIX = 0.05, 48, 0.5


def problem():
    # U = 3: a superconducting fixed point (|Delta*| ~ 0.85; at U = 2 this small
    # disordered lattice relaxes to the normal state Delta* = 0)
    return dataclasses.replace(rect(6, 6, M, seed=71, periodic=0), coupling=3.0)


def oracle_fixed_point(p, a, eps=None, hop=None):
    ol = as_oracle(p)
    if eps is not None:
        ol.eps = np.ascontiguousarray(eps, dtype=np.float64)
    if hop is not None:
        ol.hop = np.ascontiguousarray(hop, dtype=np.complex128).reshape(-1)
    d = ol.delta.copy()
    for _ in range(2000):
        ol.delta = d
        out, _ = orc.order_parameter(ol, a, T, M, K)
        nd = d + MIX * (out - d)
        if np.max(np.abs(nd - d)) < 1e-15:
            return nd.real
        d = nd
    raise AssertionError("oracle self-consistency did not converge")


def gpu_fixed_point(p, precision, pico):
    lat = gpu_lattice(p, precision, fixed_rescale_pico=pico)
    for _ in range(2000):
        if lat.scf_step(T, M, MIX) < (1e-14 if precision == "fp64" else 1e-7):
            return lat
    raise AssertionError("GPU self-consistency did not converge")


def test_fixed_point_gradient_matches_finite_differences():
    p = problem()
    a = orc.rescale(as_oracle(p))
    pico = int(round(a * 1e12))
    a = pico * 1e-12
    target = 0.3 + 0.1 * np.cos(np.arange(p.N))
    lat = gpu_fixed_point(p, "fp64", pico)
    dstar = lat.delta.real
    ref = oracle_fixed_point(p, a)
    assert np.max(np.abs(dstar - ref)) < 1e-10
    assert np.min(np.abs(dstar)) > 0.1  # a superconducting fixed point
    g = 2.0 * (dstar - target)
    ge, gh, it = lat.fixed_point_backward(T, M, MIX, g, tol=1e-13, max_iter=2000)
    assert it >= 2

    def loss(d):
        return float(np.sum((d - target) ** 2))

    h = 1e-5
    for i in (0, 14, 35):
        e1, e2 = p.eps.copy(), p.eps.copy()
        e1[i] += h
        e2[i] -= h
        fd = (loss(oracle_fixed_point(p, a, eps=e1)) - loss(oracle_fixed_point(p, a, eps=e2))) / (2 * h)
        assert abs(fd) > 1e-3 and abs(ge[i] - fd) <= 1e-6 * abs(fd), (i, ge[i], fd)
    # one bond (7 -> 8 along +x): both directed entries move together
    i, j = 7, 8
    hop = p.hop.reshape(p.N, -1)
    h1, h2 = hop.copy(), hop.copy()
    h1[i, 0] += h
    h1[j, 1] += h
    h2[i, 0] -= h
    h2[j, 1] -= h
    fd = (loss(oracle_fixed_point(p, a, hop=h1)) - loss(oracle_fixed_point(p, a, hop=h2))) / (2 * h)
    assert abs(fd) > 1e-3 and abs(gh[i, 0] - fd) <= 1e-6 * abs(fd), (gh[i, 0], fd)
    assert gh[j, 1] == gh[i, 0]
    # the fixed-point gradient differs from the one-map gradient (the loop matters)
    ge1, _, _ = lat.backward(T, M, g)
    assert np.max(np.abs(ge1 - ge)) > 1e-3 * np.max(np.abs(ge))


def test_fp32_fixed_point_gradient_close_to_fp64():
    p = problem()
    pico = int(round(orc.rescale(as_oracle(p)) * 1e12))
    target = 0.3 + 0.1 * np.cos(np.arange(p.N))
    out = {}
    for prec in ("fp64", "fp32"):
        lat = gpu_fixed_point(p, prec, pico)
        g = 2.0 * (lat.delta.real - target)
        tol = 1e-13 if prec == "fp64" else 1e-6
        out[prec] = lat.fixed_point_backward(T, M, MIX, g, tol=tol, max_iter=2000)[0]
    scale = np.max(np.abs(out["fp64"]))
    assert np.max(np.abs(out["fp32"] - out["fp64"])) < 1e-3 * scale


def test_not_converged_is_reported():
    p = problem()
    lat = gpu_fixed_point(p, "fp64", int(round(orc.rescale(as_oracle(p)) * 1e12)))
    g = np.ones(p.N)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.fixed_point_backward(T, M, MIX, g, tol=1e-13, max_iter=2)
    assert ei.value.status == cbdg.CBDG_ERR_NOT_CONVERGED


def test_autograd_through_the_fixed_point():
    torch = pytest.importorskip("torch")
    from paper_1007_1609_gb300.autograd import SelfConsistentDelta, bond_list
    p = problem()
    a = int(round(orc.rescale(as_oracle(p)) * 1e12)) * 1e-12
    bonds = bond_list(6, 6)
    hop = p.hop.reshape(p.N, -1)
    t = torch.tensor(hop[bonds[0], bonds[1]].real.copy(), requires_grad=True)
    eps = torch.tensor(p.eps, requires_grad=True)
    geom = dict(Lx=6, Ly=6, periodic_x=0, periodic_y=0, mu=p.mu, U=p.coupling)
    out = SelfConsistentDelta.apply(eps, t, torch.tensor(p.delta0.real), geom, T, M, MIX, 1e-14, "fp64", a)
    target = torch.tensor(0.3 + 0.1 * np.cos(np.arange(p.N)))
    ((out - target) ** 2).sum().backward()
    lat = gpu_fixed_point(p, "fp64", int(round(a * 1e12)))
    assert np.max(np.abs(lat.delta.real - out.detach().numpy())) < 1e-12
    ge, gh, _ = lat.fixed_point_backward(T, M, MIX, 2.0 * (lat.delta.real - target.numpy()), tol=1e-13,
                                         max_iter=2000)
    assert np.allclose(eps.grad.numpy(), ge, rtol=1e-8, atol=1e-12)
    assert np.allclose(t.grad.numpy(), gh[bonds[0], bonds[1]], rtol=1e-8, atol=1e-12)
