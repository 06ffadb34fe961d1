"""torch.autograd.Function around one self-consistency map of the
Chebyshev-BdG method: Delta_out = F(eps, t, Delta_in) for a real on-site
(s-wave) square lattice, with the rescale a frozen.  The forward pass calls
cbdg_order_parameter, the backward pass cbdg_order_parameter_backward (the
reverse Chebyshev recursion with sqrt(M) checkpointing); both run in the
CUDA library.  Hoppings are one real parameter per undirected bond."""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np
import torch

from . import cbdg


def bond_list(Lx, Ly, periodic_x=0, periodic_y=0):
    """Undirected nearest-neighbour bonds as (site, direction) with direction
    0 (+x) or 2 (+y), in site order."""
    sites, dirs = [], []
    for s in range(Lx * Ly):
        x, y = s % Lx, s // Lx
        if x + 1 < Lx or periodic_x:
            sites.append(s)
            dirs.append(0)
        if y + 1 < Ly or periodic_y:
            sites.append(s)
            dirs.append(2)
    return np.array(sites, dtype=np.int64), np.array(dirs, dtype=np.int64)


def hop_from_bonds(Lx, Ly, periodic_x, periodic_y, t_bonds, bonds):
    """[N, 4] directed hoppings from one value per undirected bond."""
    N = Lx * Ly
    hop = np.zeros((N, 4), dtype=np.complex128)
    for (s, d), t in zip(zip(*bonds), t_bonds):
        x, y = s % Lx, s // Lx
        j = ((x + 1) % Lx + Lx * y) if d == 0 else (x + Lx * ((y + 1) % Ly))
        hop[s, d] = t
        hop[j, d ^ 1] = t
    return hop


class OrderParameterMap(torch.autograd.Function):
    """Delta_out = OrderParameterMap.apply(eps, t_bonds, delta_in, geom, T, M, precision, a).

    geom: dict(Lx, Ly, periodic_x, periodic_y, mu, U); a: frozen rescale
    (None: the Gershgorin value of the input, then frozen for the backward)."""

    @staticmethod
    def forward(ctx, eps, t_bonds, delta_in, geom, T, M, precision="fp64", a=None):
        bonds = bond_list(geom["Lx"], geom["Ly"], geom.get("periodic_x", 0), geom.get("periodic_y", 0))
        hop = hop_from_bonds(geom["Lx"], geom["Ly"], geom.get("periodic_x", 0), geom.get("periodic_y", 0),
                             t_bonds.detach().cpu().numpy(), bonds)
        p = SimpleNamespace(Lx=geom["Lx"], Ly=geom["Ly"], periodic_x=geom.get("periodic_x", 0),
                            periodic_y=geom.get("periodic_y", 0),
                            eps=eps.detach().cpu().numpy().astype(np.float64), mu=geom["mu"], hop=hop,
                            pairing=0, coupling=geom["U"],
                            delta0=delta_in.detach().cpu().numpy().astype(np.complex128))
        lat = cbdg.Lattice(p, precision=precision, complex_field=False)
        if a is not None:
            lat.freeze_rescale(a)
        d, _ = lat.order_parameter(T, M)
        if a is None:
            lat.freeze_rescale(lat.rescale)
        ctx.lat, ctx.T, ctx.M, ctx.bonds = lat, T, M, bonds
        return torch.from_numpy(np.ascontiguousarray(d.real))

    @staticmethod
    def backward(ctx, grad_out):
        w = grad_out.detach().cpu().numpy().astype(np.complex128)
        g_eps, g_hop, g_delta = ctx.lat.backward(ctx.T, ctx.M, w)
        g_t = g_hop[ctx.bonds[0], ctx.bonds[1]]
        ctx.lat.close()
        return (torch.from_numpy(g_eps), torch.from_numpy(np.ascontiguousarray(g_t)),
                torch.from_numpy(g_delta), None, None, None, None, None)
