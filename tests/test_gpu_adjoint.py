"""Adjoint of one self-consistency map (cbdg_order_parameter_backward and
the torch.autograd.Function over it) vs the oracle's reverse-mode gradient
and vs central finite differences (h = 1e-6, a frozen): FP64 within 1e-6
relative; FP32 recursion within 1e-3 of the FP64 gradient's scale."""
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-3)])
@pytest.mark.parametrize("L,M,periodic", [(8, 64, 0), (7, 33, 1), (10, 5, 0)])
def test_backward_matches_oracle_gradient(precision, tol, L, M, periodic):
    p = wl.random_swave(L, M, seed=90 + L, periodic=periodic, T=0.05)
    lat = cbdg.Lattice(p, precision=precision)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    d, _ = lat.order_parameter(p.T, M)
    a = lat.rescale
    w = np.random.default_rng(L).normal(size=p.N)
    ge, gh, gd = lat.backward(p.T, M, w.astype(np.complex128))
    ol = as_oracle(p)
    C = orc.fold_coefficients(M, K, a, p.T)
    oe, oh, od = orc.scf_map_gradient(ol, a, C, w)
    assert rel(ge, oe) < tol and rel(gh, oh) < tol and rel(gd, od) < tol, (rel(ge, oe), rel(gh, oh), rel(gd, od))


def rect_swave(Lx, Ly, M, seed):
    """Open Lx x Ly disordered s-wave lattice with a random real Delta_i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = Lx * Ly
    return wl.Problem(name=f"adj{Lx}x{Ly}", Lx=Lx, Ly=Ly, periodic_x=0, periodic_y=0,
                      eps=rng.uniform(-0.5, 0.5, N), mu=-0.5, hop=wl.square_hops(Lx, Ly, 0, 0),
                      pairing=wl.ONSITE, coupling=2.0,
                      delta0=rng.uniform(0.2, 0.8, N).astype(np.complex128), T=0.05, M=M)


@pytest.mark.parametrize("Lx,Ly,M", [(20, 13, 40), (70, 9, 64), (33, 17, 101), (16, 40, 50), (128, 3, 23)])
def test_fp32_backward_with_multi_step_passes(Lx, Ly, M):
    """The FP32 adjoint runs its forward and recomputed recursions three (or
    two) steps per pass, each level written to its own vector, the reverse
    recursion one step per launch.  Segment lengths of 7, 8, 11, 8 and 5
    steps exercise every remainder; Lx = 70 and 128 the lean pass.  Against
    the oracle's reverse mode (1e-3 of the gradient's scale) and against the
    same adjoint with one step per pass (FP32 rounding only)."""
    p = rect_swave(Lx, Ly, M, seed=Lx + Ly + M)
    w = np.random.default_rng(M).normal(size=p.N)
    out = {}
    for steps in (0, 1):
        lat = cbdg.Lattice(p, precision="fp32")
        cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
        cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_TEMPORAL_STEPS, steps)
        out[steps] = lat.backward(p.T, M, w.astype(np.complex128))
        a = lat.rescale
        lat.close()
    ol = as_oracle(p)
    oe, oh, od = orc.scf_map_gradient(ol, a, orc.fold_coefficients(M, K, a, p.T), w)
    ge, gh, gd = out[0]
    assert rel(ge, oe) < 1e-3 and rel(gh.real, oh) < 1e-3 and rel(gd.real, od) < 1e-3
    for x, y in zip(out[0], out[1]):
        assert rel(x, y) < 2e-5, rel(x, y)


def test_lost_copy_times_out_in_the_adjoint():
    """Failure detection without a fault in the FP32 adjoint's multi-step
    passes: with the stall hook the first staged row of every CTA expects
    bytes that never arrive, the bounded waits run out (20 ms) and the call
    reports CBDG_ERR_CUDA; the same lattice then gives the oracle's gradient."""
    p = rect_swave(20, 13, 40, seed=7)
    w = np.random.default_rng(3).normal(size=p.N).astype(np.complex128)
    lat = cbdg.Lattice(p, precision="fp32")
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_QUADRATURE_NODES, K)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_WAIT_LIMIT_MS, 20)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_TEST_STALL_COPY, 1)
    with pytest.raises(cbdg.CbdgError) as ei:
        lat.backward(p.T, p.M, w)
    assert ei.value.status == cbdg.CBDG_ERR_CUDA and "gave up waiting" in str(ei.value)
    cbdg.cbdg_set_option(lat.handle, cbdg.CBDG_OPT_TEST_STALL_COPY, 0)
    ge, gh, gd = lat.backward(p.T, p.M, w)
    a = lat.rescale
    lat.close()
    oe, oh, od = orc.scf_map_gradient(as_oracle(p), a, orc.fold_coefficients(p.M, K, a, p.T), w.real)
    assert rel(ge, oe) < 1e-3 and rel(gh.real, oh) < 1e-3 and rel(gd.real, od) < 1e-3


def test_gradient_loss_full_size_vs_finite_differences():
    """The differentiation workload: 64x64 open, M = 512, L = sum (Delta_out -
    target)^2 with a Gaussian bump target.  Adjoint (FP64) vs central
    differences of the GPU forward with a frozen, on sampled eps_i and bonds;
    the FP32 recursion's gradient vs the FP64 one."""
    p = wl.gradient_case()
    target = p.extra["target"]
    lat = cbdg.Lattice(p, precision="fp64")
    d, _ = lat.order_parameter(p.T, p.M)
    a = lat.rescale
    w = 2.0 * (d.real - target)
    ge, gh, gd = lat.backward(p.T, p.M, w.astype(np.complex128))

    def loss(eps=None, hop=None):
        q = wl.Problem(name="fd", Lx=p.Lx, Ly=p.Ly, periodic_x=0, periodic_y=0,
                       eps=p.eps if eps is None else eps, mu=p.mu, hop=p.hop if hop is None else hop,
                       pairing=0, coupling=p.coupling, delta0=p.delta0, T=p.T, M=p.M)
        lt = cbdg.Lattice(q, precision="fp64")
        lt.freeze_rescale(a)
        dd, _ = lt.order_parameter(p.T, p.M)
        lt.close()
        return float(((dd.real - target) ** 2).sum())

    h = 1e-6
    for i in (0, 2080, 4095):
        e1, e2 = p.eps.copy(), p.eps.copy()
        e1[i] += h
        e2[i] -= h
        fd = (loss(eps=e1) - loss(eps=e2)) / (2 * h)
        assert ge[i] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(ge).max())
    for (i, dd) in ((0, 0), (2080, 2), (33, 2)):
        j = i + 1 if dd == 0 else i + 64
        h1, h2 = p.hop.copy(), p.hop.copy()
        h1[i, dd] += h
        h1[j, dd ^ 1] += h
        h2[i, dd] -= h
        h2[j, dd ^ 1] -= h
        fd = (loss(hop=h1) - loss(hop=h2)) / (2 * h)
        assert gh[i, dd] == pytest.approx(fd, rel=1e-6, abs=1e-9 * np.abs(gh).max())
    lat32 = cbdg.Lattice(p, precision="fp32")
    lat32.freeze_rescale(a)
    d32, _ = lat32.order_parameter(p.T, p.M)
    g32 = lat32.backward(p.T, p.M, (2.0 * (d32.real - target)).astype(np.complex128))
    assert rel(g32[0], ge) < 1e-3 and rel(g32[1], gh) < 1e-3


def test_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_1007_1609_gb300.autograd import OrderParameterMap, bond_list
    p = wl.random_swave(6, 48, seed=5, T=0.05)
    bonds = bond_list(6, 6)
    t = torch.ones(len(bonds[0]), dtype=torch.float64, requires_grad=True)
    eps = torch.tensor(p.eps, requires_grad=True)
    dl = torch.tensor(p.delta0.real, requires_grad=True)
    geom = dict(Lx=6, Ly=6, periodic_x=0, periodic_y=0, mu=p.mu, U=p.coupling)
    out = OrderParameterMap.apply(eps, t, dl, geom, p.T, 48, "fp64", None)
    target = torch.full_like(out, 0.3)
    loss = ((out - target) ** 2).sum()
    loss.backward()
    lat = cbdg.Lattice(p, precision="fp64")
    d, _ = lat.order_parameter(p.T, 48)
    ge, gh, gd = lat.backward(p.T, 48, (2 * (d.real - 0.3)).astype(np.complex128))
    assert np.allclose(eps.grad.numpy(), ge, rtol=1e-12, atol=1e-14)
    assert np.allclose(dl.grad.numpy(), gd, rtol=1e-12, atol=1e-14)
    assert np.allclose(t.grad.numpy(), gh[bonds[0], bonds[1]], rtol=1e-12, atol=1e-14)
