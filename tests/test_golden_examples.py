"""The paper's two worked examples, as printed (tests/golden/paper_examples.json),
against the synthetic workloads that stand in for them, and the bulk gap of
the S/N slab's superconductor against the printed 0.1 t (the uniform BCS gap
equation on a fine k-grid, independent of the oracle and of the CUDA path)."""
import json
import os

import numpy as np
from scipy.optimize import brentq

from paper_1007_1609_gb300 import workloads as wl

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "paper_examples.json")))


def test_sn_slab_matches_the_printed_example():
    g = GOLD["sn_slab"]
    p = wl.sn_slab()
    y = np.arange(p.N) // p.Lx
    U = p.extra["coupling_site"]
    assert (U[y < g["layer_S"]] > 0).all() and (U[y >= g["layer_S"]] == 0).all()
    assert p.Ly == g["layer_S"] + g["layer_N"]
    assert p.extra["broadening"] == g["broadening"]
    assert p.M >= g["moments_at_least"] - 48   # 2048: the next power of two above 2000
    assert p.periodic_x == 1 and p.periodic_y == 0
    assert p.Lx == g["plane_width"]           # the plane (periodic) is the printed L_y
    rep = p.extra["symmetry"]
    assert np.array_equal(rep, (np.arange(p.N) // p.Lx) * p.Lx)
    # the translations are a symmetry of the workload: every array is constant along a row
    for arr in (p.eps, p.extra["coupling_site"], p.delta0):
        assert np.array_equal(arr, arr[rep])


def test_sn_slab_bulk_gap_is_the_printed_one():
    """Uniform gap equation Delta = (U/N) sum_k Delta tanh(E_k/2T) / (2 E_k),
    E_k = sqrt(xi_k^2 + Delta^2), xi_k = -2(cos kx + cos ky) - mu, on a 512 x 512
    k-grid: the workload's U gives the printed bulk gap, and the BCS coherence
    length hbar v_F / (pi Delta) averaged over the Fermi surface is about 7 a."""
    g = GOLD["sn_slab"]
    p = wl.sn_slab()
    L = 512
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    xi = -2 * (np.cos(kx) + np.cos(ky)) - p.mu

    def residual(D):
        E = np.sqrt(xi ** 2 + D ** 2)
        return p.coupling * np.mean(np.tanh(E / (2 * p.T)) / (2 * E)) - 1.0

    D = brentq(residual, 1e-3, 1.0)
    assert abs(D - g["bulk_gap"]) < 0.05 * g["bulk_gap"]     # within 5% of the printed gap
    # Fermi velocity |grad xi| on the Fermi surface, weighted by the density of states
    vx, vy = 2 * np.sin(kx), 2 * np.sin(ky)
    near = np.abs(xi) < 0.05
    vF = np.sqrt(vx[near] ** 2 + vy[near] ** 2).mean()
    xi_bcs = vF / (np.pi * D)
    assert abs(xi_bcs - g["coherence_length"]) < 1.5


def test_sns_junction_matches_the_printed_example():
    g = GOLD["sns_junction"]
    p = wl.sns_junction()
    y = np.arange(p.N) // p.Lx
    x = np.arange(p.N) % p.Lx
    S1, Nl, S2 = g["layers"]
    assert p.Ly == S1 + Nl + S2 and p.Lx == g["width"]
    U = p.extra["coupling_site"]
    assert (U[(y >= S1) & (y < S1 + Nl)] == 0).all() and (U[(y < S1) | (y >= S1 + Nl)] > 0).all()
    # the impurity: peak 2 t at r0 (junction axis along y here), Gaussian of width a
    i0 = int(np.argmax(p.eps))
    assert p.eps[i0] == g["impurity_amplitude"]
    assert y[i0] == g["impurity_position_along_junction"] and x[i0] == g["impurity_position_across"]
    r2 = (x - x[i0]) ** 2 + (y - y[i0]) ** 2
    assert np.allclose(p.eps, g["impurity_amplitude"] * np.exp(-r2 / g["impurity_width"]))
    assert S1 <= y[i0] < S1 + Nl   # inside the normal layer
