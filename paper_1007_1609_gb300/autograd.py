"""torch.autograd.Functions around the self-consistency of the
Chebyshev-BdG method for a real on-site (s-wave) square lattice, with the
rescale a frozen: OrderParameterMap is one map Delta_out = F(eps, t,
Delta_in) (forward cbdg_order_parameter, backward
cbdg_order_parameter_backward, the reverse Chebyshev recursion with sqrt(M)
checkpointing); SelfConsistentDelta is the converged Delta* (forward
cbdg_scf_step to convergence, backward cbdg_fixed_point_backward through the
fixed point).  All arithmetic runs in the CUDA library.  Hoppings are one
real parameter per undirected bond."""
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


class SelfConsistentDelta(torch.autograd.Function):
    """Delta* = SelfConsistentDelta.apply(eps, t_bonds, delta0, geom, T, M, mix, tol, precision, a).

    The forward pass iterates cbdg_scf_step from delta0 until max|Delta_out -
    Delta_in| < tol (the rescale a frozen: the Gershgorin value of the input
    when a is None); the backward pass differentiates through the fixed point
    with cbdg_fixed_point_backward (implicit function theorem; no gradient
    flows to delta0, which only selects the fixed point)."""

    @staticmethod
    def forward(ctx, eps, t_bonds, delta0, geom, T, M, mix=0.5, tol=1e-12, precision="fp64", a=None,
                max_iter=5000):
        bonds = bond_list(geom["Lx"], geom["Ly"], geom.get("periodic_x", 0), geom.get("periodic_y", 0))
        hop = hop_from_bonds(geom["Lx"], geom["Ly"], geom.get("periodic_x", 0), geom.get("periodic_y", 0),
                             t_bonds.detach().cpu().numpy(), bonds)
        p = SimpleNamespace(Lx=geom["Lx"], Ly=geom["Ly"], periodic_x=geom.get("periodic_x", 0),
                            periodic_y=geom.get("periodic_y", 0),
                            eps=eps.detach().cpu().numpy().astype(np.float64), mu=geom["mu"], hop=hop,
                            pairing=0, coupling=geom["U"],
                            delta0=delta0.detach().cpu().numpy().astype(np.complex128))
        lat = cbdg.Lattice(p, precision=precision, complex_field=False)
        if a is None:
            lat.order_parameter(T, 2)  # the Gershgorin rescale of the input
            a = lat.rescale
        lat.freeze_rescale(a)
        for _ in range(max_iter):
            if lat.scf_step(T, M, mix) < tol:
                break
        else:
            lat.close()
            raise RuntimeError(f"self-consistency did not reach {tol} in {max_iter} iterations")
        ctx.lat, ctx.T, ctx.M, ctx.mix, ctx.bonds = lat, T, M, mix, bonds
        ctx.bw_tol = 1e-13 if precision == "fp64" else 1e-6
        ctx.max_iter = max_iter
        return torch.from_numpy(np.ascontiguousarray(lat.delta.real))

    @staticmethod
    def backward(ctx, grad_out):
        g = grad_out.detach().cpu().numpy().astype(np.complex128)
        g_eps, g_hop, _ = ctx.lat.fixed_point_backward(ctx.T, ctx.M, ctx.mix, g, tol=ctx.bw_tol,
                                                       max_iter=ctx.max_iter)
        g_t = g_hop[ctx.bonds[0], ctx.bonds[1]]
        ctx.lat.close()
        return (torch.from_numpy(g_eps), torch.from_numpy(np.ascontiguousarray(g_t)),
                None, None, None, None, None, None, None, None, None)
