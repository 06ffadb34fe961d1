"""The seeded synthetic inputs (CPU): each generator in workloads.py against
the recipe it states -- lattice shape and edges, the physics parameters, the
seeded disorder's range and moments, the symmetries every Hamiltonian of
Eq. 2 must have (H Hermitian: t(j -> i) = conj t(i -> j); singlet bonds:
Delta_ij = Delta_ji), and determinism under the stated seeds."""
import numpy as np
import pytest

from paper_1007_1609_gb300 import workloads as wl


def neighbour(p, s, d):
    x, y = s % p.Lx, s // p.Lx
    nx, ny = x + wl.DX[d], y + wl.DY[d]
    if not (0 <= nx < p.Lx) and not p.periodic_x:
        return -1
    if not (0 <= ny < p.Ly) and not p.periodic_y:
        return -1
    return (nx % p.Lx) + p.Lx * (ny % p.Ly)


def check_hermitian_hops(p):
    for s in range(p.N):
        for d in range(p.n_dirs):
            j = neighbour(p, s, d)
            if j < 0:
                assert p.hop[s, d] == 0
            else:
                assert p.hop[s, d] == np.conj(p.hop[j, d ^ 1])


def test_swave_disordered_recipe():
    p = wl.swave_disordered(128, 1024)
    assert (p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.M) == (128, 128, 0, 0, 1024)
    assert (p.mu, p.coupling, p.T, p.pairing) == (-0.5, 2.0, 0.01, wl.ONSITE)
    assert np.all(p.delta0 == 0.5)
    # eps ~ U[-0.5, 0.5]: range, mean and variance 1/12 of 16384 draws
    assert p.eps.min() >= -0.5 and p.eps.max() <= 0.5
    assert abs(p.eps.mean()) < 0.01 and abs(p.eps.var() - 1.0 / 12.0) < 0.003
    # the same seed gives the same lattice, another seed another one
    assert np.array_equal(p.eps, wl.swave_disordered(128, 1024).eps)
    assert not np.array_equal(p.eps, wl.swave_disordered(128, 1024, seed=1002).eps)
    # nearest-neighbour t = 1 inside, nothing across the open edges
    assert p.n_dirs == 4 and p.is_real
    assert np.count_nonzero(p.hop) == 2 * 2 * 128 * 127
    assert np.all(np.abs(p.hop[p.hop != 0]) == 1.0)


@pytest.mark.parametrize("L", [8, 17])
def test_hops_are_hermitian(L):
    check_hermitian_hops(wl.swave_disordered(L, 16))
    check_hermitian_hops(wl.dwave_vortex(L, 16))
    check_hermitian_hops(wl.sns_junction(L_S=3, L_N=2, W=L, M=16))


def test_dwave_vortex_recipe():
    p = wl.dwave_vortex(24, 64)
    assert (p.periodic_x, p.periodic_y, p.n_dirs, p.pairing) == (1, 1, 8, wl.BOND)
    assert (p.mu, p.coupling, p.T) == (-1.0, 1.5, 0.005)
    mags = np.abs(p.hop)
    assert np.allclose(mags[:, :4], 1.0) and np.allclose(mags[:, 4:], 0.3)
    # d-wave initial bonds: +0.5 along x, -0.5 along y
    assert np.all(p.delta0[:, :2] == 0.5) and np.all(p.delta0[:, 2:] == -0.5)
    e = p.extra["energy_frac"]
    assert e.size == 512 and e[0] == -0.9 and e[-1] == 0.9


def test_field_threads_the_stated_flux():
    """The phases of the hoppings around every plaquette add up to the same
    flux, and the cell holds flux_quanta h/2e: a total phase of pi per h/2e."""
    L, f = 12, 2.0
    p = wl.dwave_vortex(L, 16, flux_quanta=f)
    total = 0.0
    for y in range(L):
        for x in range(L):
            s = x + L * y
            sx = neighbour(p, s, 0)
            sxy = neighbour(p, sx, 2)
            sy = neighbour(p, s, 2)
            loop = p.hop[s, 0] * p.hop[sx, 2] * p.hop[sxy, 1] * p.hop[sy, 3]
            phase = np.angle(loop)
            assert abs(phase - np.pi * f / (L * L)) < 1e-12
            total += phase
    assert abs(total - np.pi * f) < 1e-9


def test_currents_dwave_bonds():
    L = 32
    p = wl.currents_dwave(L, 64)
    assert (p.periodic_x, p.periodic_y, p.pairing, p.n_dirs) == (1, 1, wl.BOND, 8)
    for s in range(p.N):
        for d in range(4):
            j = neighbour(p, s, d)
            assert p.delta0[s, d] == p.delta0[j, d ^ 1]  # singlet: Delta_ij = Delta_ji
    mag = np.abs(p.delta0)
    # tanh(r / 3) envelopes around the two cores: close to 0.5 far away, small near a core
    assert mag.max() <= 0.5 and mag.max() > 0.45 and mag.min() < 0.15
    # the x bonds keep the +0.5 sign and the y bonds the -0.5 sign away from the cores:
    # the product of the two core phase factors rotates both the same way
    far = mag > 0.45
    ratio = p.delta0[:, 2][far[:, 2]] / p.delta0[:, 0][far[:, 2]]
    assert np.all(np.abs(ratio + 1.0) < 0.6)


def test_ensemble_recipe():
    ps = wl.ensemble()
    assert len(ps) == 256
    sides = np.array([p.Lx for p in ps])
    assert set(sides.tolist()) == {32, 48, 64, 80, 96}
    assert all(p.Lx == p.Ly and p.periodic_x == 0 and p.periodic_y == 0 and p.M == 512 for p in ps)
    for p in ps:
        W = p.extra["W"]
        assert 0.5 <= W <= 2.0
        assert np.abs(p.eps).max() <= 0.5 * W
    # sizes and W come from one seed, the disorder from the other
    again = wl.ensemble(seed_eps=2004)
    assert [p.Lx for p in again] == sides.tolist()
    assert [p.extra["W"] for p in again] == [p.extra["W"] for p in ps]
    assert not np.array_equal(again[0].eps, ps[0].eps)


def test_gradient_case_target():
    p = wl.gradient_case(64, 512)
    t = p.extra["target"]
    assert t.shape == (p.N,) and t.min() > 0.4 and t.max() < 0.7
    # the Gaussian bump of width 8 is centred at ((L-1)/2, (L-1)/2): the four
    # central sites share the maximum, the corners sit at its 0.4 floor
    c = [31 + 64 * 31, 32 + 64 * 31, 31 + 64 * 32, 32 + 64 * 32]
    assert np.allclose(t[c], t.max())
    assert abs(t[0] - 0.4) < 1e-6
    assert abs(t.max() - (0.4 + 0.3 * np.exp(-0.5 / 128.0))) < 1e-12
