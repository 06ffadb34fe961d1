"""ctypes front end of the FP64 oracle in ``oracle.c``.

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this module, and this module
imports nothing from the product package: inputs arrive as plain numpy arrays.

The C source is compiled on first use with the host C compiler into
``oracle/_build/`` (rebuilt when the source is newer than the library).

Functions and the passages of arXiv:1007.1609 they follow:

* ``dense_hamiltonian``, ``gershgorin`` -- Eq. 2 (hamil2); rescale below Eq. 8.
* ``jackson``, ``lorentz`` -- kernel damping, Eq. 16 (Lorentz) and the Jackson
  kernel of the KPM review the paper cites.
* ``tanh_coefficients``, ``fold_coefficients`` -- Chebyshev expansion
  normalisation below the KPM introduction (Eqs. 6-7).
* ``moments`` -- direct recursion, Eq. 15 (ref2), with Eqs. 11 and 14.
* ``order_parameter`` -- Eqs. 18-19 read as expectation values of tanh(H/2T).
* ``ldos`` -- Eq. 17 with Eq. 10.
* ``scf`` -- the self-consistency loop described after Eq. 20.
* ``jacobi_eigh`` -- exact diagonalisation (cyclic Jacobi), an independent check.
* ``scf_map_gradient`` -- reverse mode of one self-consistency map.
* ``green_moments`` -- Eq. 15 read at arbitrary target sites (a^{11}, a^{12}
  of Eqs. 11 and coeff2 for every target from one recursion).
* ``green_function`` -- the full retarded G(E) of gf1 (imag2 + real1).
* ``bond_currents`` -- Eq. 20 read as the continuity equation of the hopping
  term, from the damped series of the Fermi function.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def _stamp(cmd) -> str:
    """SHA-256 of the source, the compile command and the machine type."""
    import hashlib
    import platform
    h = hashlib.sha256()
    with open(_SRC, "rb") as fh:
        h.update(fh.read())
    h.update(repr(cmd).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, FP64, OpenMP); rebuilt
    whenever the stamp of source, command and machine changes."""
    os.makedirs(_BUILD, exist_ok=True)
    flags = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-D_GNU_SOURCE"]
    want = _stamp(flags)
    stamp_path = _LIB + ".stamp"
    fresh = (os.path.exists(_LIB) and os.path.exists(stamp_path)
             and open(stamp_path).read().strip() == want)
    if force or not fresh:
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.run(flags + ["-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        with open(stamp_path + ".tmp", "w") as fh:
            fh.write(want + "\n")
        os.replace(stamp_path + ".tmp", stamp_path)
    return _LIB


class _Lat(ctypes.Structure):
    _fields_ = [
        ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("n_dirs", ctypes.c_int32),
        ("eps", ctypes.c_void_p),
        ("mu", ctypes.c_double),
        ("hop", ctypes.c_void_p),
        ("pairing", ctypes.c_int32),
        ("coupling", ctypes.c_double),
        ("delta", ctypes.c_void_p),
        ("coupling_site", ctypes.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_gershgorin.restype = D
            lib.orc_gershgorin.argtypes = [P]
            lib.orc_dense_hamiltonian.argtypes = [P, P]
            lib.orc_jackson.argtypes = [I, P]
            lib.orc_lorentz.argtypes = [I, D, P]
            lib.orc_tanh_coefficients.argtypes = [I, I, D, D, P]
            lib.orc_fold_coefficients.argtypes = [I, I, D, D, I, D, P]
            lib.orc_moments.argtypes = [P, D, P, I, I, P, P]
            lib.orc_order_parameter.argtypes = [P, D, D, I, I, I, D, P, P]
            lib.orc_ldos.argtypes = [P, D, P, I, I, I, D, P, I, P]
            lib.orc_ldos_from_moments.argtypes = [P, I, I, D, I, D, P, I, P]
            lib.orc_order_parameter_sites.argtypes = [P, D, D, I, I, I, D, P, I, P, P]
            lib.orc_order_parameter_bonds.argtypes = [P, D, D, I, I, I, D, P, I, P, P]
            lib.orc_scf.argtypes = [P, D, I, I, D, D, I, P, P, P]
            lib.orc_jacobi_eigh.argtypes = [I, P, P, P, D, I]
            lib.orc_scf_map_gradient.argtypes = [P, D, P, I, P, P, P, P]
            lib.orc_ldos_gradient.argtypes = [P, D, P, I, I, I, D, P, I, P, P, P, P]
            lib.orc_map_gradient_general.argtypes = [P, D, P, I, P, P, P, P]
            lib.orc_neighbour.argtypes = [P, I, I]
            lib.orc_green_moments.argtypes = [P, D, I, P, I, P, I, I, P, P]
            lib.orc_green_function.argtypes = [P, I, I, I, D, I, D, P, I, P]
            lib.orc_bond_currents.argtypes = [P, D, D, I, I, I, D, I, P, I, P]
            lib.orc_num_threads.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Lattice:
    """Square-lattice BdG problem of Eq. 2 in plain numpy arrays.

    hop is [N, n_dirs] complex (t_ij of the bond from site i along direction d;
    directions 0:+x 1:-x 2:+y 3:-y 4:+x+y 5:-x-y 6:+x-y 7:-x+y).  delta is [N]
    (on-site pairing) or [N, 4] (bond pairing, directions 0..3).  coupling_site,
    when given, holds one coupling per Delta entry (U_i, or V_{i,d}) in place of
    the scalar coupling.
    """

    def __init__(self, Lx, Ly, periodic_x, periodic_y, eps, mu, hop, pairing, coupling, delta,
                 coupling_site=None):
        self.Lx, self.Ly = int(Lx), int(Ly)
        self.periodic_x, self.periodic_y = int(periodic_x), int(periodic_y)
        self.eps = np.ascontiguousarray(eps, dtype=np.float64).reshape(-1)
        self.mu = float(mu)
        hop = np.ascontiguousarray(hop, dtype=np.complex128)
        self.n_dirs = int(hop.shape[-1]) if hop.ndim == 2 else int(hop.size // self.eps.size)
        self.hop = hop.reshape(-1)
        self.pairing = int(pairing)
        self.coupling = float(coupling)
        self.delta = np.ascontiguousarray(delta, dtype=np.complex128).reshape(-1).copy()
        self.coupling_site = None if coupling_site is None else \
            np.ascontiguousarray(coupling_site, dtype=np.float64).reshape(-1).copy()

    @property
    def N(self):
        return self.Lx * self.Ly

    def _c(self):
        s = _Lat()
        s.Lx, s.Ly = self.Lx, self.Ly
        s.periodic_x, s.periodic_y = self.periodic_x, self.periodic_y
        s.n_dirs = self.n_dirs
        s.eps = _ptr(self.eps)
        s.mu = self.mu
        s.hop = _ptr(self.hop)
        s.pairing = self.pairing
        s.coupling = self.coupling
        s.delta = _ptr(self.delta)
        s.coupling_site = None if self.coupling_site is None else _ptr(self.coupling_site)
        return s

    def with_delta(self, delta):
        return Lattice(self.Lx, self.Ly, self.periodic_x, self.periodic_y, self.eps, self.mu,
                       self.hop.reshape(self.N, self.n_dirs), self.pairing, self.coupling, delta,
                       self.coupling_site)


def neighbour(lat: Lattice, s: int, d: int) -> int:
    c = lat._c()
    return _load().orc_neighbour(ctypes.byref(c), int(s), int(d))


def dense_hamiltonian(lat: Lattice) -> np.ndarray:
    n = 2 * lat.N
    out = np.zeros((n, n), dtype=np.complex128)
    c = lat._c()
    _load().orc_dense_hamiltonian(ctypes.byref(c), _ptr(out))
    return out


def gershgorin(lat: Lattice) -> float:
    c = lat._c()
    return _load().orc_gershgorin(ctypes.byref(c))


def rescale(lat: Lattice) -> float:
    """a = 1.1 * Gershgorin bound (b = 0)."""
    return 1.1 * gershgorin(lat)


def jackson(M: int) -> np.ndarray:
    g = np.zeros(M)
    _load().orc_jackson(M, _ptr(g))
    return g


def lorentz(M: int, lam: float) -> np.ndarray:
    g = np.zeros(M)
    _load().orc_lorentz(M, float(lam), _ptr(g))
    return g


def tanh_coefficients(M: int, K: int, a: float, T: float) -> np.ndarray:
    c = np.zeros(M)
    _load().orc_tanh_coefficients(M, K, float(a), float(T), _ptr(c))
    return c


def fold_coefficients(M: int, K: int, a: float, T: float, kernel: int = 0, lam: float = 0.0):
    C = np.zeros(M)
    _load().orc_fold_coefficients(M, K, float(a), float(T), int(kernel), float(lam), _ptr(C))
    return C


def moments(lat: Lattice, a: float, sites, M: int):
    """Returns (mu_ee [n_sites, M] float64, mu_eh [n_sites, M, n_eh] complex128)."""
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    n_eh = 5 if lat.pairing == 1 else 1
    mu_ee = np.zeros((sites.size, M))
    mu_eh = np.zeros((sites.size, M, n_eh), dtype=np.complex128)
    c = lat._c()
    _load().orc_moments(ctypes.byref(c), float(a), _ptr(sites), sites.size, M, _ptr(mu_ee), _ptr(mu_eh))
    return mu_ee, mu_eh


def order_parameter(lat: Lattice, a: float, T: float, M: int, K: int, kernel: int = 0, lam: float = 0.0):
    """Returns (delta_out [N] or [N,4] complex128, n [N])."""
    nd = 4 * lat.N if lat.pairing == 1 else lat.N
    d = np.zeros(nd, dtype=np.complex128)
    n = np.zeros(lat.N)
    c = lat._c()
    _load().orc_order_parameter(ctypes.byref(c), float(a), float(T), M, K, int(kernel), float(lam),
                                _ptr(d), _ptr(n))
    if lat.pairing == 1:
        d = d.reshape(lat.N, 4)
    return d, n


def order_parameter_sites(lat: Lattice, a: float, T: float, M: int, K: int, sites, kernel: int = 0,
                          lam: float = 0.0):
    """On-site Delta and n at the listed start sites only (sampled parity)."""
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    d = np.zeros(sites.size, dtype=np.complex128)
    n = np.zeros(sites.size)
    c = lat._c()
    rc = _load().orc_order_parameter_sites(ctypes.byref(c), float(a), float(T), M, K, int(kernel),
                                           float(lam), _ptr(sites), sites.size, _ptr(d), _ptr(n))
    if rc != 0:
        raise ValueError("on-site pairing only")
    return d, n


def order_parameter_bonds(lat: Lattice, a: float, T: float, M: int, K: int, sites, kernel: int = 0,
                          lam: float = 0.0):
    """Bond Delta [n, 4] and n at the listed sites only (sampled parity)."""
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    d = np.zeros(sites.size * 4, dtype=np.complex128)
    n = np.zeros(sites.size)
    c = lat._c()
    rc = _load().orc_order_parameter_bonds(ctypes.byref(c), float(a), float(T), M, K, int(kernel),
                                           float(lam), _ptr(sites), sites.size, _ptr(d), _ptr(n))
    if rc != 0:
        raise ValueError("bond pairing only")
    return d.reshape(sites.size, 4), n


def ldos(lat: Lattice, a: float, sites, M: int, energies, kernel: int = 0, lam: float = 0.0):
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    energies = np.ascontiguousarray(energies, dtype=np.float64)
    out = np.zeros((sites.size, energies.size))
    c = lat._c()
    _load().orc_ldos(ctypes.byref(c), float(a), _ptr(sites), sites.size, M, int(kernel), float(lam),
                     _ptr(energies), energies.size, _ptr(out))
    return out


def ldos_from_moments(mu_ee, a: float, energies, kernel: int = 0, lam: float = 0.0):
    """LDOS (Eq. 17) at the given energies from oracle moments mu_ee [n_sites, M]."""
    mu_ee = np.ascontiguousarray(mu_ee, dtype=np.float64)
    energies = np.ascontiguousarray(energies, dtype=np.float64)
    out = np.zeros((mu_ee.shape[0], energies.size))
    _load().orc_ldos_from_moments(_ptr(mu_ee), mu_ee.shape[0], mu_ee.shape[1], float(a), int(kernel),
                                  float(lam), _ptr(energies), energies.size, _ptr(out))
    return out


def scf(lat: Lattice, T: float, M: int, K: int, mix: float, tol: float, max_iter: int):
    """Returns (delta, history, n, iterations); lat is not modified."""
    delta = lat.delta.copy()
    hist = np.zeros(max_iter)
    n = np.zeros(lat.N)
    c = lat._c()
    it = _load().orc_scf(ctypes.byref(c), float(T), M, K, float(mix), float(tol), max_iter,
                         _ptr(delta), _ptr(hist), _ptr(n))
    if lat.pairing == 1:
        delta = delta.reshape(lat.N, 4)
    return delta, hist[:it], n, it


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """Own cyclic Jacobi: returns (w ascending, V columns) for Hermitian A."""
    n = A.shape[0]
    work = np.ascontiguousarray(A, dtype=np.complex128).copy()
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128)
    _load().orc_jacobi_eigh(n, _ptr(work), _ptr(w), _ptr(V), float(tol), int(max_sweeps))
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def scf_map_gradient(lat: Lattice, a: float, C, w):
    """Reverse-mode gradient of sum_i w_i * Dout_i (real s-wave lattices only).

    Returns (g_eps [N], g_hop [N, n_dirs], g_delta [N])."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    g_eps = np.zeros(lat.N)
    g_hop = np.zeros(lat.N * lat.n_dirs)
    g_delta = np.zeros(lat.N)
    c = lat._c()
    _load().orc_scf_map_gradient(ctypes.byref(c), float(a), _ptr(C), C.size, _ptr(w),
                                 _ptr(g_eps), _ptr(g_hop), _ptr(g_delta))
    return g_eps, g_hop.reshape(lat.N, lat.n_dirs), g_delta


def map_gradient_general(lat: Lattice, a: float, C, g):
    """Reverse-mode gradient of the self-consistency map for any lattice
    (complex hoppings, next-nearest neighbours, on-site or bond pairing), a
    and C frozen.  g: dL/dRe Delta_out + i dL/dIm Delta_out ([N] or [N, 4]).

    Returns (g_eps [N], g_hop [N, n_dirs] complex, g_delta [N] or [N, 4]
    complex), each complex entry dL/dRe + i dL/dIm of that parameter."""
    C = np.ascontiguousarray(C, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.complex128).reshape(-1)
    nd = lat.N * 4 if lat.pairing == 1 else lat.N
    assert g.size == nd
    g_eps = np.zeros(lat.N)
    g_hop = np.zeros(lat.N * lat.n_dirs, dtype=np.complex128)
    g_delta = np.zeros(nd, dtype=np.complex128)
    c = lat._c()
    _load().orc_map_gradient_general(ctypes.byref(c), float(a), _ptr(C), C.size, _ptr(g), _ptr(g_eps),
                                     _ptr(g_hop), _ptr(g_delta))
    return (g_eps, g_hop.reshape(lat.N, lat.n_dirs),
            g_delta.reshape(lat.N, 4) if lat.pairing == 1 else g_delta)


def ldos_gradient(lat: Lattice, a: float, sites, M: int, energies, dL_dldos, kernel: int = 0,
                  lam: float = 0.0):
    """Reverse-mode gradient of a loss on the LDOS of Eq. 17 at the listed
    sites, given dL/dLDOS [n_sites, n_E], a frozen (real s-wave lattices only).

    Returns (g_eps [N], g_hop [N, n_dirs], g_delta [N])."""
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    energies = np.ascontiguousarray(energies, dtype=np.float64)
    G = np.ascontiguousarray(dL_dldos, dtype=np.float64).reshape(sites.size, energies.size)
    g_eps = np.zeros(lat.N)
    g_hop = np.zeros(lat.N * lat.n_dirs)
    g_delta = np.zeros(lat.N)
    c = lat._c()
    _load().orc_ldos_gradient(ctypes.byref(c), float(a), _ptr(sites), sites.size, M, int(kernel), float(lam),
                              _ptr(energies), energies.size, _ptr(G), _ptr(g_eps), _ptr(g_hop), _ptr(g_delta))
    return g_eps, g_hop.reshape(lat.N, lat.n_dirs), g_delta


def green_moments(lat: Lattice, a: float, sites, targets, M: int, start_part: int = 0):
    """Returns (a_e, a_h), each [n_sites, M, n_targets] complex128:
    a_e[c, n, t] = <e_t|T_n(H/a)|j_0>, a_h[c, n, t] = <h_t|T_n(H/a)|j_0>, with
    j_0 = e_i (start_part 0) or h_i (start_part 1), i = sites[c]."""
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    targets = np.ascontiguousarray(targets, dtype=np.int32)
    a_e = np.zeros((sites.size, M, targets.size), dtype=np.complex128)
    a_h = np.zeros_like(a_e)
    c = lat._c()
    _load().orc_green_moments(ctypes.byref(c), float(a), int(start_part), _ptr(sites), sites.size,
                              _ptr(targets), targets.size, M, _ptr(a_e), _ptr(a_h))
    return a_e, a_h


def green_function(mom, a: float, energies, kernel: int = 0, lam: float = 0.0):
    """G(E) of gf1 from moments [n_sites, M, n_t]; returns [n_sites, n_t, n_E] complex."""
    mom = np.ascontiguousarray(mom, dtype=np.complex128)
    energies = np.ascontiguousarray(energies, dtype=np.float64)
    ns, M, nt = mom.shape
    G = np.zeros((ns, nt, energies.size), dtype=np.complex128)
    _load().orc_green_function(_ptr(mom), ns, nt, M, float(a), int(kernel), float(lam),
                               _ptr(energies), energies.size, _ptr(G))
    return G


def bond_currents(lat: Lattice, a: float, T: float, M: int, K: int, kernel: int = 0, lam: float = 0.0,
                  spin: int = 0, sites=None):
    """Per-spin particle current J[c, d] from site i = sites[c] (all sites in
    order by default) to i + d (Eq. 20); spin 0 from the electron start
    vectors, 1 from the hole start vectors."""
    c = lat._c()
    if sites is None:
        J = np.zeros(lat.N * lat.n_dirs)
        _load().orc_bond_currents(ctypes.byref(c), float(a), float(T), M, K, int(kernel), float(lam),
                                  int(spin), None, 0, _ptr(J))
        return J.reshape(lat.N, lat.n_dirs)
    sites = np.ascontiguousarray(sites, dtype=np.int32)
    J = np.zeros(sites.size * lat.n_dirs)
    _load().orc_bond_currents(ctypes.byref(c), float(a), float(T), M, K, int(kernel), float(lam),
                              int(spin), _ptr(sites), sites.size, _ptr(J))
    return J.reshape(sites.size, lat.n_dirs)


def num_threads() -> int:
    return int(_load().orc_num_threads())
