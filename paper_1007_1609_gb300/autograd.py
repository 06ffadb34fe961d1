"""torch.autograd.Functions around the Chebyshev-BdG method for a real
on-site (s-wave) square lattice, with the rescale a frozen:

* OrderParameterMap: one self-consistency map Delta_out = F(eps, t,
  Delta_in) (forward cbdg_order_parameter, backward
  cbdg_order_parameter_backward: the reverse Chebyshev recursion with sqrt(M)
  checkpointing);
* SelfConsistentDelta: the converged Delta* (forward cbdg_scf_step to
  convergence, backward cbdg_fixed_point_backward through the fixed point);
* LocalDOS: the up-spin LDOS of Eq. 17 at chosen sites and energies
  (forward cbdg_ldos on the tensor cores, backward cbdg_ldos_backward).

Every array crosses the C ABI as a device pointer: eps, the hoppings and
Delta go into one lattice per (geometry, precision, device), kept in a small
cache and refilled with cbdg_set_hamiltonian / cbdg_set_delta at every call,
and the outputs and gradients are written by the library straight into
device tensors.  Gradients come back on each input's own device and dtype.
All arithmetic runs in the CUDA library; this module only lays out
arguments (one real hopping per undirected bond, scattered into the
descriptor's [N, 4] directed layout with index tensors).
"""
from __future__ import annotations

from collections import OrderedDict

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
    """[N, 4] directed hoppings from one value per undirected bond (numpy)."""
    N = Lx * Ly
    hop = np.zeros((N, 4), dtype=np.complex128)
    for (s, d), t in zip(zip(*bonds), t_bonds):
        x, y = s % Lx, s // Lx
        j = ((x + 1) % Lx + Lx * y) if d == 0 else (x + Lx * ((y + 1) % Ly))
        hop[s, d] = t
        hop[j, d ^ 1] = t
    return hop


def _geometry(geom):
    return (int(geom["Lx"]), int(geom["Ly"]), int(geom.get("periodic_x", 0)), int(geom.get("periodic_y", 0)))


class _Geometry:
    """Index tensors of one lattice shape on one device: bond i joins site s[i]
    (direction d[i]) and site j[i] (direction d[i] ^ 1)."""

    def __init__(self, Lx, Ly, px, py, device):
        s, d = bond_list(Lx, Ly, px, py)
        x, y = s % Lx, s // Lx
        j = np.where(d == 0, (x + 1) % Lx + Lx * y, x + Lx * ((y + 1) % Ly))
        self.N = Lx * Ly
        self.s = torch.from_numpy(s).to(device)
        self.d = torch.from_numpy(d).to(device)
        self.j = torch.from_numpy(j).to(device)
        self.db = torch.from_numpy(d ^ 1).to(device)

    def hop(self, t):
        """Directed hoppings [N * 4] (complex128, on t's device) from t [bonds]."""
        h = torch.zeros((self.N, 4), dtype=torch.complex128, device=t.device)
        tc = t.to(torch.complex128)
        h.index_put_((self.s, self.d), tc)
        h.index_put_((self.j, self.db), tc)
        return h.reshape(-1)

    def bond_grad(self, g_hop):
        """One value per undirected bond from the library's [N * 4] gradient."""
        return g_hop.reshape(self.N, 4)[self.s, self.d]


class _Entry:
    def __init__(self, key, device):
        Lx, Ly, px, py, mu, U, precision = key[:7]
        self.geo = _Geometry(Lx, Ly, px, py, device)
        N = Lx * Ly
        eps0 = torch.zeros(N, dtype=torch.float64, device=device)
        hop0 = torch.zeros(N * 4, dtype=torch.complex128, device=device)
        d0 = torch.zeros(N, dtype=torch.complex128, device=device)
        desc = cbdg.cbdg_lattice_desc()
        desc.Lx, desc.Ly, desc.periodic_x, desc.periodic_y = Lx, Ly, px, py
        desc.eps, desc.hop, desc.delta0 = eps0.data_ptr(), hop0.data_ptr(), d0.data_ptr()
        desc.mu, desc.n_dirs, desc.pairing, desc.coupling = mu, 4, cbdg.CBDG_ONSITE_U, U
        desc.precision, desc.complex_field = cbdg.PRECISIONS[precision], 0
        with torch.cuda.device(device):
            self.stream = torch.cuda.current_stream(device)
            self.handle = cbdg.cbdg_build_lattice(desc, self.stream)

    def close(self):
        if self.handle:
            cbdg.cbdg_destroy(self.handle)
            self.handle = None


_CACHE: "OrderedDict[tuple, _Entry]" = OrderedDict()
_CACHE_SIZE = 4


def clear_cache():
    """Frees every cached lattice (their device buffers)."""
    while _CACHE:
        _CACHE.popitem(last=False)[1].close()


def _device_of(*tensors):
    for t in tensors:
        if isinstance(t, torch.Tensor) and t.is_cuda:
            return t.device
    if not torch.cuda.is_available():
        raise RuntimeError("the Chebyshev-BdG autograd functions need a CUDA device")
    return torch.device("cuda", torch.cuda.current_device())


def _entry(geom, precision, device):
    key = _geometry(geom) + (float(geom["mu"]), float(geom["U"]), precision, device.index)
    e = _CACHE.get(key)
    if e is None:
        e = _Entry(key, device)
        _CACHE[key] = e
        while len(_CACHE) > _CACHE_SIZE:
            _CACHE.popitem(last=False)[1].close()
    _CACHE.move_to_end(key)
    return e


def _load(e, eps_d, hop_d, delta_d, a):
    """Puts this call's parameters into the cached lattice; a (None: the
    Gershgorin rescale of the input) is frozen."""
    cbdg.cbdg_set_hamiltonian(e.handle, eps_d, hop_d)
    cbdg.cbdg_set_delta(e.handle, delta_d)
    cbdg.cbdg_set_option(e.handle, cbdg.CBDG_OPT_FIXED_RESCALE_PICO, 0 if a is None else int(round(a * 1e12)))


def _inputs(eps, t_bonds, delta, geom, precision):
    dev = _device_of(eps, t_bonds, delta)
    e = _entry(geom, precision, dev)
    eps_d = eps.detach().to(device=dev, dtype=torch.float64).contiguous()
    hop_d = e.geo.hop(t_bonds.detach().to(device=dev, dtype=torch.float64))
    delta_d = delta.detach().to(device=dev, dtype=torch.complex128).contiguous()
    # the library works on the lattice's stream: let it see this stream's work first
    e.stream.wait_stream(torch.cuda.current_stream(dev))
    return dev, e, eps_d, hop_d, delta_d


def _meta(*tensors):
    """(device, dtype) of each input tensor, for returning its gradient alike."""
    return tuple((t.device, t.dtype) if isinstance(t, torch.Tensor) else None for t in tensors)


def _like(g, meta):
    return None if meta is None else g.to(device=meta[0], dtype=meta[1])


def _freeze(e, a):
    """The rescale actually used (the one just computed when a is None)."""
    return cbdg.cbdg_get_rescale(e.handle) if a is None else a


class OrderParameterMap(torch.autograd.Function):
    """Delta_out = OrderParameterMap.apply(eps, t_bonds, delta_in, geom, T, M, precision, a).

    geom: dict(Lx, Ly, periodic_x, periodic_y, mu, U); a: frozen rescale
    (None: the Gershgorin value of the input, then frozen for the backward)."""

    @staticmethod
    def forward(ctx, eps, t_bonds, delta_in, geom, T, M, precision="fp64", a=None):
        dev, e, eps_d, hop_d, delta_d = _inputs(eps, t_bonds, delta_in, geom, precision)
        _load(e, eps_d, hop_d, delta_d, a)
        dout = torch.empty(e.geo.N, dtype=torch.complex128, device=dev)
        cbdg.cbdg_order_parameter(e.handle, T, cbdg.CBDG_JACKSON, 0.0, M, dout, None)
        ctx.a = _freeze(e, a)
        ctx.geom, ctx.precision, ctx.T, ctx.M, ctx.dev = geom, precision, T, M, dev
        ctx.save_for_backward(eps_d, hop_d, delta_d)
        ctx.meta = _meta(eps, t_bonds, delta_in)
        return _like(dout.real.contiguous(), ctx.meta[2])

    @staticmethod
    def backward(ctx, grad_out):
        eps_d, hop_d, delta_d = ctx.saved_tensors
        e = _entry(ctx.geom, ctx.precision, ctx.dev)
        N = e.geo.N
        w = torch.complex(grad_out.detach().to(device=ctx.dev, dtype=torch.float64),
                          torch.zeros(N, dtype=torch.float64, device=ctx.dev)).contiguous()
        e.stream.wait_stream(torch.cuda.current_stream(ctx.dev))
        _load(e, eps_d, hop_d, delta_d, ctx.a)
        g_eps = torch.empty(N, dtype=torch.float64, device=ctx.dev)
        g_delta = torch.empty(N, dtype=torch.complex128, device=ctx.dev)
        g_hop = torch.empty(N * 4, dtype=torch.complex128, device=ctx.dev)
        cbdg.cbdg_order_parameter_backward(e.handle, ctx.T, ctx.M, w, g_eps, g_hop, g_delta)
        m = ctx.meta
        # real lattice: the gradients are real (imaginary parts 0)
        return (_like(g_eps, m[0]), _like(e.geo.bond_grad(g_hop.real), m[1]), _like(g_delta.real, m[2]),
                None, None, None, None, None)


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
        dev, e, eps_d, hop_d, delta_d = _inputs(eps, t_bonds, delta0, geom, precision)
        _load(e, eps_d, hop_d, delta_d, a)
        if a is None:
            cbdg.cbdg_order_parameter(e.handle, T, cbdg.CBDG_JACKSON, 0.0, 2, None, None)  # Gershgorin of the input
            a = cbdg.cbdg_get_rescale(e.handle)
            cbdg.cbdg_set_option(e.handle, cbdg.CBDG_OPT_FIXED_RESCALE_PICO, int(round(a * 1e12)))
        for _ in range(max_iter):
            if cbdg.cbdg_scf_step(e.handle, T, M, mix) < tol:
                break
        else:
            raise RuntimeError(f"self-consistency did not reach {tol} in {max_iter} iterations")
        dstar = torch.empty(e.geo.N, dtype=torch.complex128, device=dev)
        cbdg.cbdg_get_delta(e.handle, dstar)
        ctx.a, ctx.geom, ctx.precision, ctx.T, ctx.M, ctx.mix, ctx.dev = a, geom, precision, T, M, mix, dev
        ctx.bw_tol = 1e-13 if precision == "fp64" else 1e-6
        ctx.max_iter = max_iter
        ctx.save_for_backward(eps_d, hop_d, dstar)
        ctx.meta = _meta(eps, t_bonds, delta0)
        return _like(dstar.real.contiguous(), ctx.meta[2])

    @staticmethod
    def backward(ctx, grad_out):
        eps_d, hop_d, dstar = ctx.saved_tensors
        e = _entry(ctx.geom, ctx.precision, ctx.dev)
        N = e.geo.N
        g = torch.complex(grad_out.detach().to(device=ctx.dev, dtype=torch.float64),
                          torch.zeros(N, dtype=torch.float64, device=ctx.dev)).contiguous()
        e.stream.wait_stream(torch.cuda.current_stream(ctx.dev))
        _load(e, eps_d, hop_d, dstar, ctx.a)
        g_eps = torch.empty(N, dtype=torch.float64, device=ctx.dev)
        g_hop = torch.empty(N * 4, dtype=torch.float64, device=ctx.dev)
        cbdg.cbdg_fixed_point_backward(e.handle, ctx.T, ctx.M, ctx.mix, g, ctx.bw_tol, ctx.max_iter, g_eps, g_hop)
        m = ctx.meta
        return (_like(g_eps, m[0]), _like(e.geo.bond_grad(g_hop), m[1]),
                None, None, None, None, None, None, None, None, None)


class LocalDOS(torch.autograd.Function):
    """LDOS [n_sites, n_E] = LocalDOS.apply(eps, t_bonds, delta, geom, sites, energies, M, kernel, lam,
    precision, a).

    The up-spin LDOS of Eq. 17 at the listed sites and energies (|E| < a),
    FP32 from the tensor-core contraction; its backward is the reverse
    recursion of cbdg_ldos_backward (a frozen: the Gershgorin value of the
    input when a is None), giving gradients for eps, the bond hoppings and
    Delta.  kernel: "jackson" or "lorentz" (with lam)."""

    @staticmethod
    def forward(ctx, eps, t_bonds, delta, geom, sites, energies, M, kernel="jackson", lam=0.0, precision="fp64",
                a=None):
        dev, e, eps_d, hop_d, delta_d = _inputs(eps, t_bonds, delta, geom, precision)
        _load(e, eps_d, hop_d, delta_d, a)
        s_d = torch.as_tensor(sites, dtype=torch.int32).to(dev).contiguous()
        E_d = torch.as_tensor(energies, dtype=torch.float64).to(dev).contiguous()
        e.stream.wait_stream(torch.cuda.current_stream(dev))
        out = torch.empty((s_d.numel(), E_d.numel()), dtype=torch.float32, device=dev)
        kid = cbdg.KERNELS[kernel]
        cbdg.cbdg_ldos(e.handle, s_d, s_d.numel(), M, kid, lam, E_d, E_d.numel(), out)
        ctx.a = _freeze(e, a)
        ctx.geom, ctx.precision, ctx.M, ctx.kid, ctx.lam, ctx.dev = geom, precision, M, kid, lam, dev
        ctx.save_for_backward(eps_d, hop_d, delta_d, s_d, E_d)
        ctx.meta = _meta(eps, t_bonds, delta)
        return out if ctx.meta[0] is None or ctx.meta[0][0].type == "cuda" else out.cpu()

    @staticmethod
    def backward(ctx, grad_out):
        eps_d, hop_d, delta_d, s_d, E_d = ctx.saved_tensors
        e = _entry(ctx.geom, ctx.precision, ctx.dev)
        N = e.geo.N
        G = grad_out.detach().to(device=ctx.dev, dtype=torch.float64).contiguous()
        e.stream.wait_stream(torch.cuda.current_stream(ctx.dev))
        _load(e, eps_d, hop_d, delta_d, ctx.a)
        g_eps, g_delta = (torch.empty(N, dtype=torch.float64, device=ctx.dev) for _ in range(2))
        g_hop = torch.empty(N * 4, dtype=torch.float64, device=ctx.dev)
        cbdg.cbdg_ldos_backward(e.handle, s_d, s_d.numel(), ctx.M, ctx.kid, ctx.lam, E_d, E_d.numel(), G,
                                g_eps, g_hop, g_delta)
        m = ctx.meta
        return (_like(g_eps, m[0]), _like(e.geo.bond_grad(g_hop), m[1]), _like(g_delta, m[2]),
                None, None, None, None, None, None, None, None)
