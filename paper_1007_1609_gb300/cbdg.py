"""Thin ctypes binding of libcbdg (include/cbdg.h), same names as the C ABI.

Only argument marshalling happens here: every step of the Chebyshev-BdG path
runs in the CUDA library.  Arrays may be numpy arrays (host memory) or torch
CUDA tensors (device memory, passed by pointer); the library detects which.
If libcbdg.so has not been built, every call raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

CBDG_OK = 0
CBDG_ERR_INVALID_ARG = 1
CBDG_ERR_CUDA = 2
CBDG_ERR_OOM = 3
CBDG_ERR_SPECTRUM = 4
CBDG_ERR_NOT_CONVERGED = 5
CBDG_ERR_UNSUPPORTED = 6
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "SPECTRUM",
                5: "NOT_CONVERGED", 6: "UNSUPPORTED"}

CBDG_ONSITE_U, CBDG_BOND_V = 0, 1
CBDG_FP64, CBDG_FP32_MIXED = 0, 1
CBDG_JACKSON, CBDG_LORENTZ = 0, 1
CBDG_OPT_QUADRATURE_NODES = 0
CBDG_OPT_COLUMN_CHUNK = 1
CBDG_OPT_PROFILE = 2
CBDG_OPT_SLAB_WIDTH = 3
CBDG_OPT_ROW_SPLIT = 4
CBDG_OPT_WORKSPACE_MB = 5
CBDG_OPT_RESCALE_MILLI = 6
CBDG_OPT_PIPELINE_DEPTH = 7
CBDG_OPT_FIXED_RESCALE_PICO = 8
CBDG_OPT_WAIT_LIMIT_MS = 9
CBDG_OPT_TEST_STALL_COPY = 10
CBDG_OPT_AUTOTUNE = 11
CBDG_OPT_TEMPORAL_STEPS = 12
CBDG_OPT_GRAPH = 13
CBDG_OPT_RESIDENT = 14
CBDG_INFO_LAST_TILE = 100
CBDG_INFO_LAST_TEMPORAL = 101


class CbdgError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"cbdg status {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class cbdg_lattice_desc(ctypes.Structure):
    _fields_ = [
        ("Lx", ctypes.c_int32), ("Ly", ctypes.c_int32),
        ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
        ("eps", ctypes.c_void_p),
        ("mu", ctypes.c_double),
        ("n_dirs", ctypes.c_int32),
        ("hop", ctypes.c_void_p),
        ("pairing", ctypes.c_int32),
        ("coupling", ctypes.c_double),
        ("delta0", ctypes.c_void_p),
        ("precision", ctypes.c_int32),
        ("complex_field", ctypes.c_int32),
    ]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Loads the in-tree libcbdg.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libcbdg.so is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "cbdg_build_lattice": [P, P, P],
            "cbdg_destroy": [P],
            "cbdg_moments": [P, P, I32, I32, P, P],
            "cbdg_order_parameter": [P, D, I32, D, I32, P, P],
            "cbdg_ldos": [P, P, I32, I32, I32, D, P, I32, P],
            "cbdg_green_moments": [P, P, I32, P, I32, I32, P, P],
            "cbdg_green_function": [P, P, I32, P, I32, I32, I32, D, P, I32, P, P],
            "cbdg_bond_currents": [P, D, I32, I32, D, P],
            "cbdg_set_coupling": [P, P],
            "cbdg_scf_step": [P, D, I32, D, P],
            "cbdg_get_delta": [P, P],
            "cbdg_set_delta": [P, P],
            "cbdg_set_hamiltonian": [P, P, P],
            "cbdg_set_symmetry": [P, P],
            "cbdg_get_rescale": [P, P],
            "cbdg_lorentz_lambda": [P, D, I32, P],
            "cbdg_set_option": [P, I32, I64],
            "cbdg_get_option": [P, I32, P],
            "cbdg_profile_read": [P, P, P, P, I32],
            "cbdg_launch_count": [P, P, I32],
            "cbdg_moments_noalloc": [P, P, I32, I32, P, P, P],
            "cbdg_measure_peak": [I32, I64, P, P],
            "cbdg_peak_status": [P],
            "cbdg_contract_tf32x3": [P, I32, P, I32, P, I32, I32, I32, I32, P],
            "cbdg_contract_kp": [I32],
            "cbdg_split_tf32": [P, I32, I32, I32, P, P, P],
            "cbdg_contract_tf32x3_planes": [P, P, P, P, I32, P, I32, I32, I32, P],
            "cbdg_order_parameter_backward": [P, D, I32, P, P, P, P],
            "cbdg_ldos_backward": [P, P, I32, I32, I32, D, P, I32, P, P, P, P],
            "cbdg_fixed_point_backward": [P, D, I32, D, P, D, I32, P, P, P],
            "cbdg_build_ensemble": [P, I32, P, P],
            "cbdg_ensemble_destroy": [P],
            "cbdg_ensemble_scf": [P, D, I32, D, D, I32, P, P],
            "cbdg_ensemble_get_delta": [P, I32, P],
            "cbdg_ensemble_set_option": [P, I32, I64],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int32
        lib.cbdg_last_error.restype = ctypes.c_char_p
        lib.cbdg_last_error.argtypes = []
        lib.cbdg_version.restype = ctypes.c_char_p
        lib.cbdg_version.argtypes = []
        _lib = lib
        return lib


def header_functions(header=None):
    """Names of the functions include/cbdg.h declares."""
    header = header or os.path.join(_build.ROOT, "include", "cbdg.h")
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cbdg_[a-z_]+)\s*\(", text)))


def _check(status):
    if status != CBDG_OK:
        msg = load().cbdg_last_error().decode()
        raise CbdgError(status, msg)


def _ptr(x):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


# ---------------------------------------------------------------- C ABI names


def cbdg_build_lattice(desc: cbdg_lattice_desc, stream=None):
    out = ctypes.c_void_p()
    _check(load().cbdg_build_lattice(ctypes.byref(desc), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def cbdg_destroy(lat):
    _check(load().cbdg_destroy(lat))


def cbdg_moments(lat, sites, n_sites, M, mu_ee, mu_eh):
    _check(load().cbdg_moments(lat, _ptr(sites), int(n_sites), int(M), _ptr(mu_ee), _ptr(mu_eh)))


def cbdg_order_parameter(lat, T, kernel, lam, M, delta_out, n_out):
    _check(load().cbdg_order_parameter(lat, float(T), int(kernel), float(lam), int(M),
                                       _ptr(delta_out), _ptr(n_out)))


def cbdg_ldos(lat, sites, n_sites, M, kernel, lam, energies, n_E, ldos):
    _check(load().cbdg_ldos(lat, _ptr(sites), int(n_sites), int(M), int(kernel), float(lam),
                            _ptr(energies), int(n_E), _ptr(ldos)))


def cbdg_green_moments(lat, sites, n_sites, targets, n_targets, M, a11, a12):
    _check(load().cbdg_green_moments(lat, _ptr(sites), int(n_sites), _ptr(targets), int(n_targets), int(M),
                                     _ptr(a11), _ptr(a12)))


def cbdg_green_function(lat, sites, n_sites, targets, n_targets, M, kernel, lam, energies, n_E, G11, G12):
    _check(load().cbdg_green_function(lat, _ptr(sites), int(n_sites), _ptr(targets), int(n_targets), int(M),
                                      int(kernel), float(lam), _ptr(energies), int(n_E), _ptr(G11), _ptr(G12)))


def cbdg_bond_currents(lat, T, M, kernel, lam, J):
    _check(load().cbdg_bond_currents(lat, float(T), int(M), int(kernel), float(lam), _ptr(J)))


def cbdg_set_coupling(lat, coupling):
    _check(load().cbdg_set_coupling(lat, _ptr(coupling)))


def cbdg_scf_step(lat, T, M, mix):
    out = ctypes.c_double(0.0)
    _check(load().cbdg_scf_step(lat, float(T), int(M), float(mix), ctypes.byref(out)))
    return out.value


def cbdg_get_delta(lat, delta):
    _check(load().cbdg_get_delta(lat, _ptr(delta)))


def cbdg_set_delta(lat, delta):
    _check(load().cbdg_set_delta(lat, _ptr(delta)))


def cbdg_set_hamiltonian(lat, eps, hop):
    _check(load().cbdg_set_hamiltonian(lat, _ptr(eps), _ptr(hop)))


def cbdg_set_symmetry(lat, rep):
    _check(load().cbdg_set_symmetry(lat, _ptr(rep)))


def cbdg_get_rescale(lat):
    out = ctypes.c_double(0.0)
    _check(load().cbdg_get_rescale(lat, ctypes.byref(out)))
    return out.value


def cbdg_lorentz_lambda(lat, broadening, M):
    out = ctypes.c_double()
    _check(load().cbdg_lorentz_lambda(lat, float(broadening), int(M), ctypes.byref(out)))
    return out.value


def cbdg_set_option(lat, option, value):
    _check(load().cbdg_set_option(lat, int(option), int(value)))


def cbdg_get_option(lat, option):
    out = ctypes.c_int64(0)
    _check(load().cbdg_get_option(lat, int(option), ctypes.byref(out)))
    return out.value


def cbdg_profile_read(lat, reset=False):
    ms, n, b = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(load().cbdg_profile_read(lat, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(b),
                                    1 if reset else 0))
    return ms.value, n.value, b.value


def cbdg_launch_count(lat, reset=False):
    out = ctypes.c_int64(0)
    _check(load().cbdg_launch_count(lat, ctypes.byref(out), 1 if reset else 0))
    return out.value


def cbdg_moments_noalloc(desc, sites, n_sites, M, mu_ee, mu_eh, stream=None):
    """Moments without device allocation: every array must be in device memory."""
    _check(load().cbdg_moments_noalloc(ctypes.byref(desc), _ptr(sites), int(n_sites), int(M),
                                       _ptr(mu_ee), _ptr(mu_eh), _stream_handle(stream)))


CBDG_PEAK_FP64_FMA, CBDG_PEAK_FP32_FMA, CBDG_PEAK_TF32_MMA = 0, 1, 2


def cbdg_measure_peak(kind, work, stream=None):
    """Queues one peak-probe launch on `stream`; returns its flops."""
    out = ctypes.c_double()
    _check(load().cbdg_measure_peak(int(kind), int(work), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def cbdg_peak_status(stream=None):
    _check(load().cbdg_peak_status(_stream_handle(stream)))


def cbdg_contract_tf32x3(A, lda, B, ldb, D, ldd, m, n, k, stream=None):
    _check(load().cbdg_contract_tf32x3(_ptr(A), int(lda), _ptr(B), int(ldb), _ptr(D), int(ldd),
                                       int(m), int(n), int(k), _stream_handle(stream)))


def cbdg_contract_kp(k):
    return int(load().cbdg_contract_kp(int(k)))


def cbdg_split_tf32(src, ld, rows, k, hi, lo, stream=None):
    _check(load().cbdg_split_tf32(_ptr(src), int(ld), int(rows), int(k), _ptr(hi), _ptr(lo),
                                  _stream_handle(stream)))


def cbdg_contract_tf32x3_planes(a_hi, a_lo, b_hi, b_lo, kp, D, ldd, m, n, stream=None):
    _check(load().cbdg_contract_tf32x3_planes(_ptr(a_hi), _ptr(a_lo), _ptr(b_hi), _ptr(b_lo), int(kp),
                                              _ptr(D), int(ldd), int(m), int(n), _stream_handle(stream)))


def cbdg_fixed_point_backward(lat, T, M, mix, dL_ddelta, tol, max_iter, dL_deps, dL_dhop):
    """Gradient through the self-consistent fixed point; returns the iteration count."""
    it = ctypes.c_int32(0)
    _check(load().cbdg_fixed_point_backward(lat, float(T), int(M), float(mix), _ptr(dL_ddelta), float(tol),
                                            int(max_iter), _ptr(dL_deps), _ptr(dL_dhop), ctypes.byref(it)))
    return it.value


def cbdg_order_parameter_backward(lat, T, M, dL_ddelta_out, dL_deps, dL_dhop, dL_ddelta_in):
    _check(load().cbdg_order_parameter_backward(lat, float(T), int(M), _ptr(dL_ddelta_out),
                                                _ptr(dL_deps), _ptr(dL_dhop), _ptr(dL_ddelta_in)))


def cbdg_ldos_backward(lat, sites, n_sites, M, kernel, lam, energies, n_E, dL_dldos, dL_deps, dL_dhop,
                       dL_ddelta):
    _check(load().cbdg_ldos_backward(lat, _ptr(sites), int(n_sites), int(M), int(kernel), float(lam),
                                     _ptr(energies), int(n_E), _ptr(dL_dldos), _ptr(dL_deps), _ptr(dL_dhop),
                                     _ptr(dL_ddelta)))


def cbdg_build_ensemble(descs, stream=None):
    arr = (cbdg_lattice_desc * len(descs))(*descs)
    out = ctypes.c_void_p()
    _check(load().cbdg_build_ensemble(arr, len(descs), _stream_handle(stream), ctypes.byref(out)))
    return out.value


def cbdg_ensemble_destroy(ens):
    _check(load().cbdg_ensemble_destroy(ens))


def cbdg_ensemble_scf(ens, T, M, mix, tol, max_iter, converged_mask):
    """Returns (status, iterations); NOT_CONVERGED is returned, not raised."""
    it = ctypes.c_int32(0)
    st = load().cbdg_ensemble_scf(ens, float(T), int(M), float(mix), float(tol), int(max_iter),
                                  ctypes.byref(it), _ptr(converged_mask))
    if st not in (CBDG_OK, CBDG_ERR_NOT_CONVERGED):
        _check(st)
    return st, it.value


def cbdg_ensemble_get_delta(ens, sample, delta):
    _check(load().cbdg_ensemble_get_delta(ens, int(sample), _ptr(delta)))


def cbdg_ensemble_set_option(ens, option, value):
    _check(load().cbdg_ensemble_set_option(ens, int(option), int(value)))


def cbdg_last_error():
    return load().cbdg_last_error().decode()


def cbdg_version():
    return load().cbdg_version().decode()


# ---------------------------------------------------------------- convenience


def make_desc(problem, precision="fp64", complex_field=None):
    """A cbdg_lattice_desc for a workloads.Problem-like object; returns
    (desc, arrays) -- keep `arrays` alive while the descriptor is used."""
    p = problem
    eps = np.ascontiguousarray(p.eps, dtype=np.float64)
    hop = np.ascontiguousarray(p.hop, dtype=np.complex128)
    delta = np.ascontiguousarray(p.delta0, dtype=np.complex128)
    if complex_field is None:
        complex_field = bool(np.any(hop.imag) or np.any(delta.imag))
    d = cbdg_lattice_desc()
    d.Lx, d.Ly = int(p.Lx), int(p.Ly)
    d.periodic_x, d.periodic_y = int(p.periodic_x), int(p.periodic_y)
    d.eps, d.hop, d.delta0 = _ptr(eps), _ptr(hop), _ptr(delta)
    d.mu = float(p.mu)
    d.n_dirs = int(hop.shape[-1]) if hop.ndim == 2 else int(hop.size // eps.size)
    d.pairing = int(p.pairing)
    d.coupling = float(p.coupling)
    d.precision = PRECISIONS[precision]
    d.complex_field = 1 if complex_field else 0
    return d, (eps, hop, delta)


class Ensemble:
    """Independent lattices iterated to self-consistency together (FP32)."""

    def __init__(self, problems, stream=None):
        self._keep = []
        descs = []
        for p in problems:
            d, arrays = make_desc(p, precision="fp32", complex_field=False)
            descs.append(d)
            self._keep.append(arrays)
        self.sizes = [int(p.Lx * p.Ly) for p in problems]
        self.handle = cbdg_build_ensemble(descs, stream)

    def set_option(self, option, value):
        cbdg_ensemble_set_option(self.handle, option, value)

    def scf(self, T, M, mix, tol, max_iter):
        mask = np.zeros(len(self.sizes), dtype=np.int32)
        st, it = cbdg_ensemble_scf(self.handle, T, M, mix, tol, max_iter, mask)
        return st == CBDG_OK, it, mask

    def delta(self, sample):
        d = np.zeros(self.sizes[sample], dtype=np.complex128)
        cbdg_ensemble_get_delta(self.handle, sample, d)
        return d

    def close(self):
        if getattr(self, "handle", None):
            cbdg_ensemble_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PRECISIONS = {"fp64": CBDG_FP64, "fp32": CBDG_FP32_MIXED}
KERNELS = {"jackson": CBDG_JACKSON, "lorentz": CBDG_LORENTZ}


class Lattice:
    """Owns a cbdg_lattice built from a workloads.Problem-like object
    (attributes Lx, Ly, periodic_x, periodic_y, eps, mu, hop, pairing,
    coupling, delta0)."""

    def __init__(self, problem, precision="fp64", stream=None, complex_field=None):
        p = problem
        self.N = int(p.Lx * p.Ly)
        self.pairing = int(p.pairing)
        self._eps = np.ascontiguousarray(p.eps, dtype=np.float64)
        self._hop = np.ascontiguousarray(p.hop, dtype=np.complex128)
        self._delta = np.ascontiguousarray(p.delta0, dtype=np.complex128)
        if complex_field is None:
            complex_field = bool(np.any(self._hop.imag) or np.any(self._delta.imag))
        d = cbdg_lattice_desc()
        d.Lx, d.Ly = int(p.Lx), int(p.Ly)
        d.periodic_x, d.periodic_y = int(p.periodic_x), int(p.periodic_y)
        d.eps = _ptr(self._eps)
        d.mu = float(p.mu)
        d.n_dirs = int(self._hop.shape[-1]) if self._hop.ndim == 2 else int(self._hop.size // self.N)
        self.n_dirs = int(d.n_dirs)
        d.hop = _ptr(self._hop)
        d.pairing = self.pairing
        d.coupling = float(p.coupling)
        d.delta0 = _ptr(self._delta)
        d.precision = PRECISIONS[precision]
        d.complex_field = 1 if complex_field else 0
        self.desc = d
        self.handle = cbdg_build_lattice(d, stream)
        self.nd = 4 * self.N if self.pairing == CBDG_BOND_V else self.N

    def close(self):
        if getattr(self, "handle", None):
            cbdg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value):
        cbdg_set_option(self.handle, option, value)

    def last_tile(self):
        """(slab width, pipeline depth, row split) of the last recursion pass."""
        v = cbdg_get_option(self.handle, CBDG_INFO_LAST_TILE)
        return v & 0xFFFF, (v >> 16) & 0xFFFF, v >> 32

    def moments(self, sites, M):
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        n_eh = 5 if self.pairing == CBDG_BOND_V else 1
        mu_ee = np.zeros((sites.size, M))
        mu_eh = np.zeros((sites.size, M, n_eh), dtype=np.complex128)
        cbdg_moments(self.handle, sites, sites.size, M, mu_ee, mu_eh)
        return mu_ee, mu_eh

    def order_parameter(self, T, M, kernel="jackson", lam=0.0):
        d = np.zeros(self.nd, dtype=np.complex128)
        n = np.zeros(self.N)
        cbdg_order_parameter(self.handle, T, KERNELS[kernel], lam, M, d, n)
        return (d.reshape(self.N, 4) if self.pairing == CBDG_BOND_V else d), n

    def ldos(self, sites, M, energies, kernel="jackson", lam=0.0):
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        energies = np.ascontiguousarray(energies, dtype=np.float64)
        out = np.zeros((sites.size, energies.size), dtype=np.float32)
        cbdg_ldos(self.handle, sites, sites.size, M, KERNELS[kernel], lam, energies, energies.size, out)
        return out

    def green_moments(self, sites, targets, M):
        """(a11, a12), each [n_sites, M, n_targets] complex128: <e_t|T_n|e_i>, <h_t|T_n|e_i>."""
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        targets = np.ascontiguousarray(targets, dtype=np.int32)
        a11 = np.zeros((sites.size, M, targets.size), dtype=np.complex128)
        a12 = np.zeros_like(a11)
        cbdg_green_moments(self.handle, sites, sites.size, targets, targets.size, M, a11, a12)
        return a11, a12

    def green_function(self, sites, targets, M, energies, kernel="jackson", lam=0.0):
        """(G11, G12), each [n_sites, n_targets, n_E] complex128 (Eq. gf1)."""
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        targets = np.ascontiguousarray(targets, dtype=np.int32)
        energies = np.ascontiguousarray(energies, dtype=np.float64)
        G11 = np.zeros((sites.size, targets.size, energies.size), dtype=np.complex128)
        G12 = np.zeros_like(G11)
        cbdg_green_function(self.handle, sites, sites.size, targets, targets.size, M, KERNELS[kernel], lam,
                            energies, energies.size, G11, G12)
        return G11, G12

    def set_coupling(self, coupling):
        """One coupling per Delta entry (U_i [N] or V_{i,d} [N, 4]); None restores the scalar."""
        if coupling is None:
            cbdg_set_coupling(self.handle, None)
            return
        self._cpl = np.ascontiguousarray(coupling, dtype=np.float64).reshape(-1)
        cbdg_set_coupling(self.handle, self._cpl)

    def set_symmetry(self, rep):
        """Representative site of every site's orbit ([N]; None: no reduction)."""
        if rep is None:
            cbdg_set_symmetry(self.handle, None)
            return
        self._rep = np.ascontiguousarray(rep, dtype=np.int32)
        cbdg_set_symmetry(self.handle, self._rep)

    def lorentz_lambda(self, broadening, M):
        """lambda of the Lorentz kernel (Eq. 16) for an energy broadening at the
        band centre, with the rescale of the current Delta (cbdg_lorentz_lambda)."""
        return cbdg_lorentz_lambda(self.handle, broadening, M)

    def bond_currents(self, T, M, kernel="jackson", lam=0.0):
        """J [N, n_dirs]: current from site i to its neighbour along d, both spins (Eq. 20)."""
        J = np.zeros((self.N, self.n_dirs))
        cbdg_bond_currents(self.handle, T, M, KERNELS[kernel], lam, J)
        return J

    def scf_step(self, T, M, mix):
        return cbdg_scf_step(self.handle, T, M, mix)

    @property
    def delta(self):
        d = np.zeros(self.nd, dtype=np.complex128)
        cbdg_get_delta(self.handle, d)
        return d.reshape(self.N, 4) if self.pairing == CBDG_BOND_V else d

    @delta.setter
    def delta(self, value):
        cbdg_set_delta(self.handle, np.ascontiguousarray(value, dtype=np.complex128).reshape(-1))

    @property
    def rescale(self):
        return cbdg_get_rescale(self.handle)

    def freeze_rescale(self, a):
        """Use a fixed a (None: back to the Gershgorin rescale)."""
        cbdg_set_option(self.handle, CBDG_OPT_FIXED_RESCALE_PICO, 0 if a is None else int(round(a * 1e12)))

    def fixed_point_backward(self, T, M, mix, dL_ddelta, tol=1e-12, max_iter=500):
        """(dL/deps [N], dL/dhop [N, 4], iterations) through the converged Delta."""
        g = np.ascontiguousarray(dL_ddelta, dtype=np.complex128).reshape(-1)
        ge = np.zeros(self.N)
        gh = np.zeros(self.N * 4)
        it = cbdg_fixed_point_backward(self.handle, T, M, mix, g, tol, max_iter, ge, gh)
        return ge, gh.reshape(self.N, 4), it

    def ldos_backward(self, sites, M, energies, dL_dldos, kernel="jackson", lam=0.0):
        """(dL/deps [N], dL/dhop [N, 4], dL/dDelta [N]) of a loss on the LDOS at
        (sites, energies), given dL/dLDOS [n_sites, n_E] (a frozen)."""
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        energies = np.ascontiguousarray(energies, dtype=np.float64)
        g = np.ascontiguousarray(dL_dldos, dtype=np.float64).reshape(sites.size, energies.size)
        ge, gd = np.zeros(self.N), np.zeros(self.N)
        gh = np.zeros(self.N * 4)
        cbdg_ldos_backward(self.handle, sites, sites.size, M, KERNELS[kernel], lam, energies, energies.size, g,
                           ge, gh, gd)
        return ge, gh.reshape(self.N, 4), gd

    def backward(self, T, M, dL_ddelta_out):
        """Gradients of one map (see the C ABI): (eps [N] real, hop [N, n_dirs]
        complex, delta_in [N] or [N, 4] complex), each complex entry
        dL/dRe + i dL/dIm; dL_ddelta_out is [N] or [N, 4] (complex)."""
        w = np.ascontiguousarray(dL_ddelta_out, dtype=np.complex128).reshape(-1)
        g_eps = np.zeros(self.N)
        g_hop = np.zeros(self.N * self.n_dirs, dtype=np.complex128)
        g_delta = np.zeros(self.nd, dtype=np.complex128)
        cbdg_order_parameter_backward(self.handle, T, M, w, g_eps, g_hop, g_delta)
        return (g_eps, g_hop.reshape(self.N, self.n_dirs),
                g_delta.reshape(self.N, 4) if self.pairing == CBDG_BOND_V else g_delta)
