"""Seeded synthetic inputs for the lattice BdG problems.

This module only generates problem inputs (lattice geometry, hopping
amplitudes with Peierls phases, disorder, initial order parameters, targets).
It holds none of the Chebyshev-BdG arithmetic, so both the CUDA path and the
FP64 oracle consume exactly the same arrays.  Random numbers come from numpy's
PCG64 with fixed seeds.

Conventions (shared by every consumer):

* site index s = x + Lx * y;
* directions d: 0:+x 1:-x 2:+y 3:-y 4:+x+y 5:-x-y 6:+x-y 7:-x+y
  (d and d^1 are opposite);
* hop[s, d] is the amplitude t_ij of the bond from s to its neighbour along d,
  entering H_{e_i e_j} = -t_ij and H_{h_i h_j} = conj(t_ij) (Eq. 2); it is zero
  where an open edge cuts the bond, and hop[j, d^1] = conj(hop[i, d]);
* Peierls phases t_ij = |t| exp(i theta_ij) for a uniform field in the Landau
  gauge A = (0, B x): a total of ``flux_quanta`` superconducting flux quanta
  h/2e through the periodic cell, i.e. a phase of pi * flux_quanta / (Lx Ly)
  per plaquette.  Bonds that cross the x seam pick up the gauge twist
  -2 pi (flux per cell in units of h/e) * y_end / Ly that keeps the flux uniform.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

DX = (1, -1, 0, 0, 1, -1, 1, -1)
DY = (0, 0, 1, -1, 1, -1, -1, 1)

ONSITE = 0
BOND = 1


@dataclass
class Problem:
    """One lattice BdG problem (Eq. 2) plus the run parameters of a workload."""

    name: str
    Lx: int
    Ly: int
    periodic_x: int
    periodic_y: int
    eps: np.ndarray          # [N] float64
    mu: float
    hop: np.ndarray          # [N, n_dirs] complex128
    pairing: int             # ONSITE or BOND
    coupling: float          # U or V
    delta0: np.ndarray       # [N] or [N, 4] complex128
    T: float
    M: int
    mix: float = 0.5
    tol: float = 1e-6
    max_iter: int = 10
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.Lx * self.Ly

    @property
    def n_dirs(self) -> int:
        return int(self.hop.shape[1])

    @property
    def is_real(self) -> bool:
        return (not np.iscomplexobj(self.hop) or not np.any(self.hop.imag)) and \
            not np.any(np.asarray(self.delta0).imag)


def square_hops(Lx, Ly, periodic_x, periodic_y, t=1.0, tp=0.0, flux_quanta=0.0):
    """Hopping amplitudes on an Lx x Ly square lattice (NN t, optional NNN t').

    Returns hop [N, 4] (tp == 0) or [N, 8], complex128.  With a nonzero flux
    both directions must be periodic (the field is defined on the torus)."""
    n_dirs = 8 if tp != 0.0 else 4
    N = Lx * Ly
    hop = np.zeros((N, n_dirs), dtype=np.complex128)
    if flux_quanta != 0.0 and not (periodic_x and periodic_y):
        raise ValueError("a uniform field needs a periodic cell")
    # phase per plaquette: pi/phi0 * flux with phi0 = h/2e -> 2 pi * (flux/(h/e))
    phi = np.pi * flux_quanta / (Lx * Ly)       # phase per plaquette
    twist = np.pi * flux_quanta / Ly            # x-seam twist per unit of y
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            for d in (0, 2, 4, 6):              # forward directions; reverse is conj
                if d >= n_dirs:
                    continue
                dx, dy = DX[d], DY[d]
                nx, ny = x + dx, y + dy
                cross_x = not (0 <= nx < Lx)
                cross_y = not (0 <= ny < Ly)
                if (cross_x and not periodic_x) or (cross_y and not periodic_y):
                    continue
                amp = t if d < 4 else tp
                # straight-line integral of A = (0, B x): B * (x + dx/2) * dy
                theta = phi * (x + 0.5 * dx) * dy
                if cross_x:
                    theta -= twist * (ny % Ly)
                j = (nx % Lx) + Lx * (ny % Ly)
                val = amp * np.exp(1j * theta)
                hop[s, d] = val
                hop[j, d ^ 1] = np.conj(val)
    return hop


def _problem(name, L, periodic, eps, mu, hop, pairing, coupling, delta0, T, M, **kw):
    return Problem(name=name, Lx=L, Ly=L, periodic_x=periodic, periodic_y=periodic,
                   eps=np.ascontiguousarray(eps, dtype=np.float64), mu=mu,
                   hop=np.ascontiguousarray(hop, dtype=np.complex128), pairing=pairing,
                   coupling=coupling, delta0=np.ascontiguousarray(delta0, dtype=np.complex128),
                   T=T, M=M, **kw)


def swave_clean(L=16, M=256, iters=10):
    """Clean s-wave square lattice, open edges: t=1, mu=-0.5, U=2, T=0.01,
    uniform initial Delta = 0.5, linear mixing 0.5 (16x16 with M=256 by default)."""
    N = L * L
    return _problem(f"swave_clean_{L}x{L}_M{M}", L, 0, np.zeros(N), -0.5,
                    square_hops(L, L, 0, 0), ONSITE, 2.0, np.full(N, 0.5 + 0j), 0.01, M,
                    mix=0.5, tol=0.0, max_iter=iters)


def swave_disordered(L=128, M=1024, W=1.0, seed=1001, tol=1e-6):
    """Disordered s-wave lattice, open edges: eps_i ~ U[-W/2, W/2] (PCG64 seed),
    t=1, mu=-0.5, U=2, T=0.01, initial Delta = 0.5 (128x128, M=1024 by default)."""
    N = L * L
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = rng.uniform(-0.5 * W, 0.5 * W, size=N)
    return _problem(f"swave_disordered_{L}x{L}_M{M}_W{W:g}", L, 0, eps, -0.5,
                    square_hops(L, L, 0, 0), ONSITE, 2.0, np.full(N, 0.5 + 0j), 0.01, M,
                    mix=0.5, tol=tol, max_iter=200)


def dwave_vortex(L=256, M=2048, flux_quanta=2.0, n_energies=512):
    """d-wave vortex lattice: periodic L x L, t=1, t'=-0.3, mu=-1, bond pairing
    V=1.5, T=0.005, uniform field of ``flux_quanta`` h/2e through the cell,
    initial bonds Delta_{+-x} = +0.5, Delta_{+-y} = -0.5, LDOS energies uniform
    in [-0.9 a, 0.9 a] (expressed as fractions of a in extra['energy_frac'])."""
    N = L * L
    hop = square_hops(L, L, 1, 1, t=1.0, tp=-0.3, flux_quanta=flux_quanta)
    d0 = np.zeros((N, 4), dtype=np.complex128)
    d0[:, 0] = d0[:, 1] = 0.5
    d0[:, 2] = d0[:, 3] = -0.5
    return _problem(f"dwave_vortex_{L}x{L}_M{M}", L, 1, np.zeros(N), -1.0, hop, BOND, 1.5,
                    d0, 0.005, M, mix=0.5, tol=1e-6, max_iter=100,
                    extra={"energy_frac": np.linspace(-0.9, 0.9, n_energies)})


def currents_dwave(L=128, M=512, flux_quanta=2.0, xi=3.0):
    """Bond-current workload: the d-wave vortex lattice (periodic L x L, t=1,
    t'=-0.3, mu=-1, V=1.5, T=0.005, uniform field of ``flux_quanta`` h/2e)
    with ``flux_quanta`` vortices imprinted on the initial bonds: vortex k at
    r_k on a diagonal, each bond Delta_{ij} = +-0.5 (x / y bonds) times
    prod_k tanh(|r_m - r_k| / xi) exp(i arg(r_m - r_k)) at the bond midpoint
    r_m (the neighbour taken unwrapped across the seam)."""
    N = L * L
    hop = square_hops(L, L, 1, 1, t=1.0, tp=-0.3, flux_quanta=flux_quanta)
    nv = max(1, int(round(flux_quanta)))
    cores = [((k + 0.5) * L / nv + 0.25, (k + 0.5) * L / nv + 0.25) for k in range(nv)]
    d0 = np.zeros((N, 4), dtype=np.complex128)
    for s in range(N):
        x, y = s % L, s // L
        for d in (0, 2):
            mx, my = x + 0.5 * DX[d], y + 0.5 * DY[d]
            z = 0.5 if d == 0 else -0.5
            for cx, cy in cores:
                r = np.hypot(mx - cx, my - cy)
                z *= np.tanh(r / xi) * np.exp(1j * np.arctan2(my - cy, mx - cx))
            j = ((x + DX[d]) % L) + L * ((y + DY[d]) % L)
            d0[s, d] = z
            d0[j, d ^ 1] = z
    return _problem(f"currents_dwave_{L}x{L}_M{M}", L, 1, np.zeros(N), -1.0, hop, BOND, 1.5, d0,
                    0.005, M, mix=0.5, tol=1e-6, max_iter=100)


def sn_slab(Lx=500, L_S=300, L_N=20, M=2048, U=1.41, mu=-0.5, T=0.005, broadening=0.001):
    """Planar S/N system after the paper's first example: superconductor (U)
    for rows y < L_S, normal metal (U = 0) for the L_N rows above it, open
    along y (the slab normal) and periodic along x (the plane, Lx = 500
    sites: the printed L_y = 500 a).  t = 1, no disorder; U = 1.41 at
    mu = -0.5 gives a bulk gap of about 0.1 t (coherence length about 7
    sites).  Initial Delta 0.1 in S, 0 in N.  LDOS at the N surface (row
    y = L_S + L_N - 1) with the Lorentz kernel, energy broadening
    ``broadening`` (in units of t).  Per-site couplings in
    extra['coupling_site']; the plane's translations map every site to the
    site of its row at x = 0 (extra['symmetry'], for cbdg_set_symmetry)."""
    Ly = L_S + L_N
    N = Lx * Ly
    y = np.arange(N) // Lx
    U_site = np.where(y < L_S, U, 0.0)
    d0 = np.where(y < L_S, 0.1, 0.0).astype(np.complex128)
    surface = np.arange((Ly - 1) * Lx, Ly * Lx, dtype=np.int32)
    p = Problem(name=f"sn_slab_{Lx}x{Ly}_M{M}", Lx=Lx, Ly=Ly, periodic_x=1, periodic_y=0, eps=np.zeros(N),
                mu=mu, hop=np.ascontiguousarray(square_hops(Lx, Ly, 1, 0), dtype=np.complex128),
                pairing=ONSITE, coupling=U, delta0=d0, T=T, M=M, mix=0.5, tol=1e-6, max_iter=200,
                extra={"coupling_site": U_site, "surface_sites": surface, "broadening": broadening,
                       "energy_frac": np.linspace(-0.05, 0.05, 201),
                       "symmetry": (Lx * y).astype(np.int32)})
    return p


def sns_junction(L_S=50, L_N=50, W=100, M=2048, U=1.41, mu=-0.5, T=0.005, impurity=2.0, r0=(50, 60),
                 phase=0.0, broadening=0.001):
    """S/N/S junction with a Gaussian impurity after the paper's second
    example: along y, L_S superconducting rows, L_N normal rows (U = 0) and
    L_S superconducting rows; W sites across (x); open edges.  On-site
    potential eps_i = impurity * exp(-|r_i - r0|^2) (lattice constant 1) at
    r0 = (x, y) in the normal layer.  Initial Delta 0.1 in the lower S layer
    and 0.1 exp(i phase) in the upper one (phase != 0 drives a Josephson
    current; the lattice is then complex).  Per-site couplings in
    extra['coupling_site']; LDOS sites around the impurity in
    extra['ldos_sites']."""
    Ly = 2 * L_S + L_N
    N = W * Ly
    x, y = np.arange(N) % W, np.arange(N) // W
    in_s = (y < L_S) | (y >= L_S + L_N)
    U_site = np.where(in_s, U, 0.0)
    eps = impurity * np.exp(-((x - r0[0]) ** 2 + (y - r0[1]) ** 2))
    d0 = np.where(y < L_S, 0.1, 0.0) + np.where(y >= L_S + L_N, 0.1 * np.exp(1j * phase), 0.0)
    near = np.array([(r0[0] + dx) + W * r0[1] for dx in range(-5, 6)], dtype=np.int32)
    return Problem(name=f"sns_junction_{W}x{Ly}_M{M}", Lx=W, Ly=Ly, periodic_x=0, periodic_y=0, eps=eps,
                   mu=mu, hop=np.ascontiguousarray(square_hops(W, Ly, 0, 0), dtype=np.complex128),
                   pairing=ONSITE, coupling=U, delta0=np.ascontiguousarray(d0, dtype=np.complex128), T=T, M=M,
                   mix=0.5, tol=1e-6, max_iter=200,
                   extra={"coupling_site": U_site, "ldos_sites": near, "broadening": broadening,
                          "energy_frac": np.linspace(-0.05, 0.05, 201)})


def ensemble(n_samples=256, sides=(32, 48, 64, 80, 96), M=512, seed_sizes=1003, seed_eps=1004):
    """Ensemble of independent disordered s-wave lattices: sides drawn
    uniformly from ``sides`` and W ~ U[0.5, 2] per sample (seed_sizes),
    eps ~ U[-W/2, W/2] (seed_eps); open edges, t=1, mu=-0.5, U=2, T=0.01."""
    rs = np.random.Generator(np.random.PCG64(seed_sizes))
    Ls = rs.choice(np.asarray(sides), size=n_samples)
    Ws = rs.uniform(0.5, 2.0, size=n_samples)
    re = np.random.Generator(np.random.PCG64(seed_eps))
    out = []
    for k in range(n_samples):
        L = int(Ls[k])
        N = L * L
        eps = re.uniform(-0.5 * Ws[k], 0.5 * Ws[k], size=N)
        out.append(_problem(f"ensemble_{k}_{L}x{L}", L, 0, eps, -0.5, square_hops(L, L, 0, 0),
                            ONSITE, 2.0, np.full(N, 0.5 + 0j), 0.01, M, mix=0.5, tol=1e-4,
                            max_iter=100, extra={"W": float(Ws[k])}))
    return out


def gradient_case(L=64, M=512, seed=1005):
    """Differentiation workload: open L x L s-wave lattice, eps ~ U[-0.5, 0.5],
    t=1, mu=-0.5, U=2, T=0.01, Delta_in = 0.5, target Delta = 0.4 + 0.3 *
    exp(-|r - r_c|^2 / (2 * 8^2)) with r_c the lattice centre."""
    N = L * L
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = rng.uniform(-0.5, 0.5, size=N)
    y, x = np.divmod(np.arange(N), L)
    c = 0.5 * (L - 1)
    target = 0.4 + 0.3 * np.exp(-((x - c) ** 2 + (y - c) ** 2) / (2.0 * 8.0 ** 2))
    return _problem(f"gradient_{L}x{L}_M{M}", L, 0, eps, -0.5, square_hops(L, L, 0, 0), ONSITE,
                    2.0, np.full(N, 0.5 + 0j), 0.01, M, extra={"target": target})


def random_swave(L, M, seed, periodic=0, W=1.0, complex_delta=False, flux_quanta=0.0, tp=0.0,
                 mu=-0.5, U=2.0, T=0.01, delta_scale=0.5):
    """Small random on-site problems for parity and edge-case tests: random
    disorder, random (optionally complex) Delta_i, optional field and t'."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = L * L
    eps = rng.uniform(-0.5 * W, 0.5 * W, size=N)
    hop = square_hops(L, L, periodic, periodic, t=1.0, tp=tp, flux_quanta=flux_quanta)
    d = delta_scale * rng.uniform(0.5, 1.5, size=N).astype(np.complex128)
    if complex_delta:
        d = d * np.exp(1j * rng.uniform(-np.pi, np.pi, size=N))
    return _problem(f"random_swave_{L}x{L}_s{seed}", L, periodic, eps, mu, hop, ONSITE, U, d, T, M)


def random_dwave(L, M, seed, flux_quanta=0.0, tp=-0.3, mu=-1.0, V=1.5, T=0.005):
    """Small random bond-pairing problems on a periodic lattice: random
    symmetric bond amplitudes Delta_ij = Delta_ji (complex), optional field."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = L * L
    hop = square_hops(L, L, 1, 1, t=1.0, tp=tp, flux_quanta=flux_quanta)
    d = np.zeros((N, 4), dtype=np.complex128)
    for s in range(N):
        x, y = s % L, s // L
        for dd in (0, 2):
            j = ((x + DX[dd]) % L) + L * ((y + DY[dd]) % L)
            val = (0.5 if dd == 0 else -0.5) * rng.uniform(0.5, 1.5) * np.exp(1j * rng.uniform(-0.5, 0.5))
            d[s, dd] = val
            d[j, dd ^ 1] = val
    eps = rng.uniform(-0.25, 0.25, size=N)
    return _problem(f"random_dwave_{L}x{L}_s{seed}", L, 1, eps, mu, hop, BOND, V, d, T, M)
