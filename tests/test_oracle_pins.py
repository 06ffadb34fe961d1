"""Pins of the FP64 oracle against facts fixed by the mathematics (no GPU).

Each test checks an oracle function against something other than itself:
exact diagonalisation (own Jacobi cross-checked with LAPACK), k-space closed
forms on uniform periodic lattices, invariants of the Chebyshev moments,
independent quadrature, and central finite differences.  The comments say
which plausible mistake each one would catch.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as orc
from paper_1007_1609_gb300 import workloads as wl


def as_oracle(p, delta=None):
    return orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu, p.hop, p.pairing,
                       p.coupling, p.delta0 if delta is None else delta)


def ed(lat):
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    return w, V


def cheb_T(n, x):
    return np.cos(n * np.arccos(np.clip(x, -1.0, 1.0)))


# ---------------------------------------------------------------- Hamiltonian


def test_hamiltonian_entries_and_hermiticity():
    """Eq. 2 entry by entry on a 3x3 periodic lattice with complex t and Delta:
    catches swapped e/h rows, a missing conjugate or a sign slip."""
    p = wl.random_swave(3, 8, seed=7, periodic=1, complex_delta=True, flux_quanta=2.0)
    lat = as_oracle(p)
    H = orc.dense_hamiltonian(lat)
    assert np.allclose(H, H.conj().T, atol=0, rtol=0)
    for i in range(lat.N):
        xi = p.eps[i] - p.mu
        assert H[2 * i, 2 * i] == pytest.approx(xi)
        assert H[2 * i + 1, 2 * i + 1] == pytest.approx(-xi)
        assert H[2 * i, 2 * i + 1] == pytest.approx(p.delta0[i])
        for d in range(4):
            j = orc.neighbour(lat, i, d)
            t = p.hop[i, d]
            assert H[2 * i, 2 * j] == pytest.approx(-t)
            assert H[2 * i + 1, 2 * j + 1] == pytest.approx(np.conj(t))
    # each row has 2 on-site + 4 hopping entries on a periodic 3x3 lattice
    assert np.count_nonzero(np.abs(H) > 0, axis=1).max() == 6


def test_open_edges_cut_bonds():
    p = wl.random_swave(4, 8, seed=3, periodic=0)
    lat = as_oracle(p)
    assert orc.neighbour(lat, 3, 0) == -1 and orc.neighbour(lat, 0, 1) == -1
    assert orc.neighbour(lat, 0, 3) == -1 and orc.neighbour(lat, 15, 2) == -1
    H = orc.dense_hamiltonian(lat)
    # corner site 0 couples to two neighbours only
    assert np.count_nonzero(H[0]) == 2 + 2


def test_jacobi_matches_lapack():
    """Own cyclic Jacobi vs LAPACK on a random Hermitian matrix and on a BdG
    matrix with field: a wrong rotation or phase would break A V = V w."""
    rng = np.random.default_rng(11)
    A = rng.normal(size=(40, 40)) + 1j * rng.normal(size=(40, 40))
    A = A + A.conj().T
    w, V = orc.jacobi_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-11)
    assert np.allclose(A @ V, V * w, atol=1e-10)
    assert np.allclose(V.conj().T @ V, np.eye(40), atol=1e-12)
    p = wl.random_swave(4, 8, seed=5, periodic=1, complex_delta=True, flux_quanta=2.0)
    H = orc.dense_hamiltonian(as_oracle(p))
    w2, V2 = orc.jacobi_eigh(H)
    assert np.allclose(w2, np.linalg.eigvalsh(H), atol=1e-12)
    assert np.allclose(H @ V2, V2 * w2, atol=1e-11)


@pytest.mark.parametrize("case", ["swave_open", "swave_field", "dwave_field"])
def test_particle_hole_symmetric_spectrum(case):
    """The BdG spectrum is symmetric under E -> -E for symmetric pairing."""
    if case == "swave_open":
        p = wl.random_swave(5, 8, seed=1)
    elif case == "swave_field":
        p = wl.random_swave(4, 8, seed=2, periodic=1, complex_delta=True, flux_quanta=2.0, tp=-0.3)
    else:
        p = wl.random_dwave(4, 8, seed=3, flux_quanta=2.0)
    w = np.linalg.eigvalsh(orc.dense_hamiltonian(as_oracle(p)))
    assert np.allclose(np.sort(w), np.sort(-w), atol=1e-12)


def test_gershgorin_bounds_spectrum():
    for seed in range(3):
        p = wl.random_swave(5, 8, seed=seed, periodic=seed % 2, complex_delta=True)
        lat = as_oracle(p)
        H = orc.dense_hamiltonian(lat)
        bound = orc.gershgorin(lat)
        assert bound == pytest.approx(np.abs(H).sum(axis=1).max(), rel=1e-14)
        assert np.abs(np.linalg.eigvalsh(H)).max() <= bound


def test_normal_state_reduces_to_hopping_matrix():
    """At Delta = 0 the BdG spectrum is {xi_m} U {-xi_m} with xi_m the
    eigenvalues of the N x N hopping matrix (Hofstadter problem with field)."""
    p = wl.random_swave(6, 8, seed=4, periodic=1, flux_quanta=2.0, tp=-0.3)
    lat = as_oracle(p, delta=np.zeros(36, dtype=complex))
    h = np.zeros((36, 36), dtype=complex)
    for i in range(36):
        h[i, i] = p.eps[i] - p.mu
        for d in range(p.n_dirs):
            j = orc.neighbour(lat, i, d)
            h[i, j] += -p.hop[i, d]
    xi = np.linalg.eigvalsh(h)
    w = np.linalg.eigvalsh(orc.dense_hamiltonian(lat))
    assert np.allclose(np.sort(w), np.sort(np.concatenate([xi, -xi])), atol=1e-12)


def test_peierls_phases_uniform_flux():
    """Every plaquette of the generated field encloses phase pi*f/(Lx*Ly)."""
    L, f = 8, 2.0
    hop = wl.square_hops(L, L, 1, 1, flux_quanta=f)
    for y in range(L):
        for x in range(L):
            s = x + L * y
            s1 = (x + 1) % L + L * y
            s2 = (x + 1) % L + L * ((y + 1) % L)
            s3 = x + L * ((y + 1) % L)
            loop = hop[s, 0] * hop[s1, 2] * hop[s2, 1] * hop[s3, 3]
            assert np.angle(loop) == pytest.approx(np.pi * f / L ** 2, abs=1e-12)
    # conjugate pairs
    for s in range(L * L):
        for d in range(4):
            x, y = s % L, s // L
            j = (x + wl.DX[d]) % L + L * ((y + wl.DY[d]) % L)
            assert hop[j, d ^ 1] == pytest.approx(np.conj(hop[s, d]))


# ---------------------------------------------------------------- moments


@pytest.mark.parametrize("case", ["open_real", "periodic_field", "nnn_field", "dwave_bonds"])
def test_moments_match_exact_diagonalisation(case):
    """Direct recursion (Eq. 15) vs ED: mu_n = sum_k u_k(i) conj(u_k(i)) T_n(E_k/a)
    and <h_j|T_n|e_i> = sum_k v_k(j) conj(u_k(i)) T_n(E_k/a).  Exact to
    round-off for every n: catches a wrong recursion start, index or scale."""
    M = 96
    if case == "open_real":
        p = wl.random_swave(4, M, seed=21)
    elif case == "periodic_field":
        p = wl.random_swave(4, M, seed=22, periodic=1, complex_delta=True, flux_quanta=2.0)
    elif case == "nnn_field":
        p = wl.random_swave(5, M, seed=23, periodic=1, complex_delta=True, flux_quanta=2.0, tp=-0.3)
    else:
        p = wl.random_dwave(4, M, seed=24, flux_quanta=2.0)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    H = orc.dense_hamiltonian(lat)
    w, V = orc.jacobi_eigh(H)
    sites = np.arange(lat.N)
    mu_ee, mu_eh = orc.moments(lat, a, sites, M)
    n = np.arange(M)
    Tn = cheb_T(n[:, None], (w / a)[None, :])           # [M, 2N]
    for i in sites:
        u = V[2 * i]                                      # u_k(i) = <e_i|k>
        v = V[2 * i + 1]
        ref_ee = Tn @ (np.abs(u) ** 2)
        ref_eh = Tn @ (v * np.conj(u))
        assert np.allclose(mu_ee[i], ref_ee, atol=1e-12, rtol=0)
        assert np.allclose(mu_eh[i, :, 0], ref_eh, atol=1e-12, rtol=0)
        if p.pairing == wl.BOND:
            for d in range(4):
                j = orc.neighbour(lat, i, d)
                ref = Tn @ (V[2 * j + 1] * np.conj(u))
                assert np.allclose(mu_eh[i, :, 1 + d], ref, atol=1e-12, rtol=0)


def test_moment_invariants():
    """mu_0 = 1, |mu_n| <= 1, <h_i|T_2n|e_i> = 0 (particle-hole symmetry),
    and 2 sum_i mu_2m(i) = Tr T_2m(H/a) from the eigenvalues alone."""
    M = 64
    p = wl.random_swave(5, M, seed=31, periodic=1, complex_delta=True, flux_quanta=2.0)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    mu_ee, mu_eh = orc.moments(lat, a, np.arange(lat.N), M)
    assert np.allclose(mu_ee[:, 0], 1.0, atol=0)
    assert np.abs(mu_ee).max() <= 1.0 + 1e-13
    assert np.abs(mu_eh[:, 0::2, 0]).max() < 1e-13
    w = np.linalg.eigvalsh(orc.dense_hamiltonian(lat))
    for m in range(0, M, 2):
        assert 2 * mu_ee[:, m].sum() == pytest.approx(cheb_T(m, w / a).sum(), abs=1e-11)


def test_normal_state_moments_closed_form():
    """Delta = 0, periodic, uniform: mu_n(i) = (1/N) sum_k T_n(xi_k / a) with
    xi_k = -2t(cos kx + cos ky) - 4t' cos kx cos ky - mu."""
    L, M, t, tp, mu = 8, 80, 1.0, -0.3, -1.0
    N = L * L
    hop = wl.square_hops(L, L, 1, 1, t=t, tp=tp)
    lat = orc.Lattice(L, L, 1, 1, np.zeros(N), mu, hop, 0, 2.0, np.zeros(N, dtype=complex))
    a = 7.3
    mu_ee, _ = orc.moments(lat, a, np.array([0, 9, 37]), M)
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    xi = (-2 * t * (np.cos(kx) + np.cos(ky)) - 4 * tp * np.cos(kx) * np.cos(ky) - mu).ravel()
    ref = np.array([cheb_T(n, xi / a).mean() for n in range(M)])
    for r in mu_ee:
        assert np.allclose(r, ref, atol=1e-13)


# ---------------------------------------------------------------- coefficients


def test_jackson_kernel_properties():
    """g_0 = 1, g_1 = cos(pi/(M+1)), and the Jackson-damped delta function is
    non-negative everywhere (the kernel's defining property)."""
    for M in (8, 64, 257):
        g = orc.jackson(M)
        assert g[0] == pytest.approx(1.0, abs=1e-15)
        assert g[1] == pytest.approx(np.cos(np.pi / (M + 1)), abs=1e-15)
        x = np.cos(np.pi * (np.arange(400) + 0.5) / 400)
        for y in (-0.7, 0.0, 0.31, 0.95):
            n = np.arange(1, M)
            delta = g[0] + 2 * (g[1:, None] * cheb_T(n[:, None], x[None, :]) * cheb_T(n, y)[:, None]).sum(0)
            assert delta.min() > -1e-12


def test_lorentz_kernel_values():
    g = orc.lorentz(100, 4.0)
    assert g[0] == pytest.approx(1.0)
    assert g[50] == pytest.approx(np.sinh(2.0) / np.sinh(4.0))


@pytest.mark.parametrize("a,T", [(5.0, 0.25), (5.5, 0.01), (8.8, 0.005)])
def test_tanh_coefficients_vs_adaptive_quadrature(a, T):
    """Gauss-Chebyshev sum vs scipy's adaptive quadrature of
    (1/pi) int_0^pi tanh(a cos th / 2T) cos(n th) d th."""
    M, K = 40, 1 << 16
    c = orc.tanh_coefficients(M, K, a, T)
    for n in (0, 1, 2, 3, 7, 21, 39):
        f = lambda th: np.tanh(a * np.cos(th) / (2 * T)) * np.cos(n * th) / np.pi
        ref, err = integrate.quad(f, 0, np.pi, points=[np.pi / 2], limit=500, epsabs=1e-14, epsrel=1e-13)
        assert c[n] == pytest.approx(ref, abs=1e-12)


def test_tanh_series_reconstructs_function():
    """sum_n (2 - delta_n0) c_n T_n(x) reproduces tanh(a x / 2T) (undamped)."""
    a, T, M = 5.0, 0.2, 400
    c = orc.tanh_coefficients(M, 1 << 14, a, T)
    x = np.linspace(-0.99, 0.99, 37)
    s = c[0] + 2 * sum(c[n] * cheb_T(n, x) for n in range(1, M))
    assert np.allclose(s, np.tanh(a * x / (2 * T)), atol=1e-10)


def test_zero_temperature_coefficients():
    """At T = 0 the function is sign(x) with c_n = (2/(pi n)) sin(n pi/2):
    the quadrature converges like 1/K."""
    c = orc.tanh_coefficients(16, 1 << 16, 1.0, 0.0)
    n = np.arange(1, 16)
    assert np.allclose(c[1:], 2 / (np.pi * n) * np.sin(n * np.pi / 2), atol=1e-3)
    assert abs(c[0]) < 1e-14


# ---------------------------------------------------------------- observables


@pytest.mark.parametrize("case", ["open_real", "periodic_field"])
def test_order_parameter_and_density_match_ed(case):
    """Delta_i = (U/2) sum_k u_k(i) conj(v_k(i)) F_M(E_k/a) and
    n_i = 1 - sum_k |u_k(i)|^2 F_M(E_k/a), F_M = sum_n C_n T_n, to round-off."""
    M, K = 128, 1 << 14
    if case == "open_real":
        p = wl.random_swave(5, M, seed=41, T=0.05)
    else:
        p = wl.random_swave(4, M, seed=42, periodic=1, complex_delta=True, flux_quanta=2.0, T=0.05)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    d, nn = orc.order_parameter(lat, a, p.T, M, K)
    C = orc.fold_coefficients(M, K, a, p.T)
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    F = sum(C[n] * cheb_T(n, w / a) for n in range(M))
    u, v = V[0::2], V[1::2]
    ref_d = 0.5 * p.coupling * (u * np.conj(v) * F).sum(1)
    ref_n = 1 - (np.abs(u) ** 2 * F).sum(1)
    assert np.allclose(d, ref_d, atol=1e-12)
    assert np.allclose(nn, ref_n, atol=1e-12)


def test_bond_order_parameter_matches_ed():
    """Non-uniform complex bonds with field: Delta_{i,d} = (V/8) sum_k
    [u_k(i) conj(v_k(j)) + u_k(j) conj(v_k(i))] F_M(E_k/a), j = i + d.
    Catches a wrong direction for the reverse-bond moment."""
    M, K = 96, 1 << 13
    p = wl.random_dwave(4, M, seed=44, flux_quanta=2.0)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    d, _ = orc.order_parameter(lat, a, p.T, M, K)
    C = orc.fold_coefficients(M, K, a, p.T)
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    F = sum(C[n] * cheb_T(n, w / a) for n in range(M))
    for i in range(lat.N):
        for dd in range(4):
            j = orc.neighbour(lat, i, dd)
            ref = p.coupling / 8 * ((V[2 * i] * np.conj(V[2 * j + 1]) +
                                     V[2 * j] * np.conj(V[2 * i + 1])) * F).sum()
            assert d[i, dd] == pytest.approx(ref, abs=1e-12)


def test_sampled_sites_match_full_order_parameter():
    M, K = 64, 1 << 12
    p = wl.random_swave(5, M, seed=45, T=0.05)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    d, n = orc.order_parameter(lat, a, p.T, M, K)
    sites = np.array([3, 0, 24, 3, 11])
    ds, ns = orc.order_parameter_sites(lat, a, p.T, M, K, sites)
    assert np.array_equal(ds, d[sites]) and np.array_equal(ns, n[sites])


def test_sampled_bonds_match_full_order_parameter():
    M, K = 48, 1 << 12
    p = wl.random_dwave(5, M, seed=46, flux_quanta=2.0)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    d, n = orc.order_parameter(lat, a, p.T, M, K)
    sites = np.array([7, 0, 24, 13])
    ds, ns = orc.order_parameter_bonds(lat, a, p.T, M, K, sites)
    assert np.allclose(ds, d[sites], atol=1e-15) and np.allclose(ns, n[sites], atol=1e-15)


def test_order_parameter_converges_to_exact_tanh():
    """As M grows the damped series converges to the exact ED order parameter
    (U/2) sum_k u conj(v) tanh(E_k/2T); the error falls monotonically."""
    p = wl.random_swave(4, 0, seed=43, T=0.1)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    ref = 0.5 * p.coupling * (V[0::2] * np.conj(V[1::2]) * np.tanh(w / (2 * p.T))).sum(1)
    errs = []
    for M in (64, 256, 1024):
        d, _ = orc.order_parameter(lat, a, p.T, M, 1 << 13)
        errs.append(np.abs(d - ref).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-4


def test_uniform_swave_kspace_closed_form():
    """Uniform periodic s-wave: Delta^KPM = (U/2N) sum_k F_M(E_k/a) Delta/E_k,
    E_k = sqrt(xi_k^2 + Delta^2): pins the sign and the factor U/2."""
    L, M, K, T, U, mu, D = 8, 200, 1 << 14, 0.02, 2.0, -0.5, 0.4
    N = L * L
    lat = orc.Lattice(L, L, 1, 1, np.zeros(N), mu, wl.square_hops(L, L, 1, 1), 0, U,
                      np.full(N, D, dtype=complex))
    a = orc.rescale(lat)
    d, nn = orc.order_parameter(lat, a, T, M, K)
    C = orc.fold_coefficients(M, K, a, T)
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    xi = (-2 * (np.cos(kx) + np.cos(ky)) - mu).ravel()
    E = np.sqrt(xi ** 2 + D ** 2)
    F = sum(C[n] * cheb_T(n, E / a) for n in range(M))
    assert np.allclose(d, U / (2 * N) * (F * D / E).sum(), atol=1e-12)
    assert np.allclose(nn, 1 - (F * xi / E).sum() / N, atol=1e-12)
    assert d.real.min() > 0


def test_bcs_gap_equation_limit():
    """Large M: the uniform solution satisfies the BCS gap equation
    Delta = (U/N) sum_k Delta/(2E_k) tanh(E_k/2T)."""
    L, T, U, mu, D = 8, 0.05, 2.0, -0.5, 0.3
    N = L * L
    lat = orc.Lattice(L, L, 1, 1, np.zeros(N), mu, wl.square_hops(L, L, 1, 1), 0, U,
                      np.full(N, D, dtype=complex))
    a = orc.rescale(lat)
    d, _ = orc.order_parameter(lat, a, T, 4096, 1 << 15)
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    xi = (-2 * (np.cos(kx) + np.cos(ky)) - mu).ravel()
    E = np.sqrt(xi ** 2 + D ** 2)
    gap = U / N * (D / (2 * E) * np.tanh(E / (2 * T))).sum()
    assert np.allclose(d.real, gap, atol=2e-4)


def test_uniform_dwave_kspace_closed_form():
    """Uniform periodic d-wave bonds Delta_{+-x} = D, Delta_{+-y} = -D:
    Delta_x = (V/4N) sum_k cos(kx) F(E_k/a) Delta_k/E_k with
    Delta_k = 2D (cos kx - cos ky): pins the bond readout and the V/8 form."""
    L, M, K, T, V, mu, tp, D = 8, 160, 1 << 14, 0.02, 1.5, -1.0, -0.3, 0.3
    N = L * L
    d0 = np.zeros((N, 4), dtype=complex)
    d0[:, 0] = d0[:, 1] = D
    d0[:, 2] = d0[:, 3] = -D
    lat = orc.Lattice(L, L, 1, 1, np.zeros(N), mu, wl.square_hops(L, L, 1, 1, tp=tp), 1, V, d0)
    a = orc.rescale(lat)
    d, nn = orc.order_parameter(lat, a, T, M, K)
    C = orc.fold_coefficients(M, K, a, T)
    k = 2 * np.pi * np.arange(L) / L
    kx, ky = np.meshgrid(k, k)
    xi = (-2 * (np.cos(kx) + np.cos(ky)) - 4 * tp * np.cos(kx) * np.cos(ky) - mu).ravel()
    Dk = (2 * D * (np.cos(kx) - np.cos(ky))).ravel()
    E = np.sqrt(xi ** 2 + Dk ** 2)
    F = sum(C[n] * cheb_T(n, E / a) for n in range(M))
    ratio = np.where(E > 0, F / np.where(E > 0, E, 1), 0)
    ref_x = V / (4 * N) * (np.cos(kx).ravel() * ratio * Dk).sum()
    ref_y = V / (4 * N) * (np.cos(ky).ravel() * ratio * Dk).sum()
    assert np.allclose(d[:, 0], ref_x, atol=1e-12) and np.allclose(d[:, 1], ref_x, atol=1e-12)
    assert np.allclose(d[:, 2], ref_y, atol=1e-12) and np.allclose(d[:, 3], ref_y, atol=1e-12)
    assert ref_x > 0 > ref_y


def test_ldos_matches_ed_and_is_normalised():
    """LDOS (Eq. 17) vs the Jackson-broadened ED sum; positive; integrates to 1."""
    M = 128
    p = wl.random_swave(4, M, seed=51, periodic=1, complex_delta=True, flux_quanta=2.0)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    Kq = 2000
    xq = np.cos(np.pi * (np.arange(Kq) + 0.5) / Kq)
    E = a * xq
    sites = np.array([0, 5, 11])
    rho = orc.ldos(lat, a, sites, M, E)
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    g = orc.jackson(M)
    n = np.arange(1, M)
    for r, i in zip(rho, sites):
        wt = np.abs(V[2 * i]) ** 2
        ref = np.zeros_like(E)
        for e_k, wk in zip(w / a, wt):
            ref += wk * (g[0] + 2 * (g[1:, None] * cheb_T(n[:, None], xq[None, :]) *
                                     cheb_T(n, e_k)[:, None]).sum(0))
        ref /= np.pi * a * np.sqrt(1 - xq ** 2)
        assert np.allclose(r, ref, atol=1e-11)
        assert r.min() > -1e-12
        # int N(E) dE with E = a cos th: Gauss-Chebyshev weights pi/Kq * a sqrt(1-x^2)
        total = (r * np.pi / Kq * a * np.sqrt(1 - xq ** 2)).sum()
        assert total == pytest.approx(1.0, abs=1e-10)
    mu_ee, _ = orc.moments(lat, a, sites, M)
    assert np.array_equal(orc.ldos_from_moments(mu_ee, a, E), rho)


def test_gauge_covariance():
    """t_ij -> t_ij e^{i(chi_j - chi_i)}, Delta_i -> Delta_i e^{-2i chi_i}
    leaves mu_ee and n unchanged and rotates Delta_out by e^{-2i chi_i}."""
    M, K = 64, 1 << 13
    p = wl.random_swave(4, M, seed=61, periodic=1, complex_delta=True, flux_quanta=2.0, tp=-0.3)
    lat = as_oracle(p)
    chi = np.random.default_rng(5).uniform(-np.pi, np.pi, lat.N)
    hop2 = p.hop.copy()
    for i in range(lat.N):
        for d in range(p.n_dirs):
            j = orc.neighbour(lat, i, d)
            hop2[i, d] = p.hop[i, d] * np.exp(1j * (chi[j] - chi[i]))
    lat2 = orc.Lattice(p.Lx, p.Ly, 1, 1, p.eps, p.mu, hop2, 0, p.coupling, p.delta0 * np.exp(-2j * chi))
    a = orc.rescale(lat)
    assert orc.rescale(lat2) == pytest.approx(a, rel=1e-14)
    d1, n1 = orc.order_parameter(lat, a, p.T, M, K)
    d2, n2 = orc.order_parameter(lat2, a, p.T, M, K)
    assert np.allclose(n1, n2, atol=1e-12)
    assert np.allclose(d2, d1 * np.exp(-2j * chi), atol=1e-12)


# ---------------------------------------------------------------- SCF


def test_scf_matches_ed_route():
    """Ten mixed iterations of the oracle loop vs the same loop driven by
    dense eigendecomposition (a from the Gershgorin bound each iteration)."""
    M, K, iters = 96, 1 << 13, 10
    p = wl.random_swave(5, M, seed=71, T=0.03)
    lat = as_oracle(p, delta=np.full(25, 0.5, dtype=complex))
    d_orc, hist, _, it = orc.scf(lat, p.T, M, K, 0.5, 0.0, iters)
    assert it == iters
    delta = np.full(25, 0.5, dtype=complex)
    for _ in range(iters):
        l2 = lat.with_delta(delta)
        a = orc.rescale(l2)
        C = orc.fold_coefficients(M, K, a, p.T)
        w, V = np.linalg.eigh(orc.dense_hamiltonian(l2))
        F = sum(C[n] * cheb_T(n, w / a) for n in range(M))
        dout = 0.5 * p.coupling * (V[0::2] * np.conj(V[1::2]) * F).sum(1)
        delta = delta + 0.5 * (dout - delta)
    assert np.allclose(d_orc, delta, atol=1e-12)
    assert hist[-1] < hist[0]


# ---------------------------------------------------------------- gradient


def test_scf_map_gradient_vs_finite_differences():
    """Reverse-mode gradient of L = sum_i w_i Dout_i vs central differences
    (h = 1e-6) of the forward map with a frozen."""
    M, K = 48, 1 << 12
    p = wl.random_swave(4, M, seed=81, T=0.05)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    C = orc.fold_coefficients(M, K, a, p.T)
    w = np.random.default_rng(3).normal(size=lat.N)
    g_eps, g_hop, g_delta = orc.scf_map_gradient(lat, a, C, w)

    def loss(eps=None, hop=None, delta=None):
        l2 = orc.Lattice(p.Lx, p.Ly, 0, 0, p.eps if eps is None else eps, p.mu,
                         p.hop if hop is None else hop, 0, p.coupling,
                         p.delta0 if delta is None else delta)
        d, _ = orc.order_parameter(l2, a, p.T, M, K)
        return float((w * d.real).sum())

    h = 1e-6
    for i in (0, 5, 10, 15):
        e1, e2 = p.eps.copy(), p.eps.copy()
        e1[i] += h
        e2[i] -= h
        fd = (loss(eps=e1) - loss(eps=e2)) / (2 * h)
        assert g_eps[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        d1, d2 = p.delta0.copy(), p.delta0.copy()
        d1[i] += h
        d2[i] -= h
        fd = (loss(delta=d1) - loss(delta=d2)) / (2 * h)
        assert g_delta[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    for (i, d) in ((0, 0), (5, 2), (6, 1), (14, 3)):
        j = orc.neighbour(lat, i, d)
        h1, h2 = p.hop.copy(), p.hop.copy()
        h1[i, d] += h
        h1[j, d ^ 1] += h
        h2[i, d] -= h
        h2[j, d ^ 1] -= h
        fd = (loss(hop=h1) - loss(hop=h2)) / (2 * h)
        assert g_hop[i, d] == pytest.approx(fd, rel=1e-6, abs=1e-9)
        assert g_hop[j, d ^ 1] == pytest.approx(g_hop[i, d], rel=1e-12)


def _general_loss(p, a, M, K, g):
    """L = Re sum_k conj(g_k) Delta_out,k and a closure over perturbed arrays."""
    def loss(eps=None, hop=None, delta=None):
        l2 = orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps if eps is None else eps, p.mu,
                         p.hop if hop is None else hop, p.pairing, p.coupling,
                         p.delta0 if delta is None else delta)
        d, _ = orc.order_parameter(l2, a, p.T, M, K)
        return float(np.real(np.conj(g) * d.reshape(g.shape)).sum())
    return loss


def _fd_check_general(p, M, g_seed, sites, bonds, pair_bonds):
    K = 1 << 12
    lat = as_oracle(p)
    a = orc.rescale(lat)
    C = orc.fold_coefficients(M, K, a, p.T)
    rng = np.random.default_rng(g_seed)
    shape = (p.N, 4) if p.pairing == wl.BOND else (p.N,)
    g = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    if p.pairing == wl.BOND:
        g = g * (np.abs(p.delta0) > 0)  # no output across a missing bond
    g_eps, g_hop, g_delta = orc.map_gradient_general(lat, a, C, g)
    loss = _general_loss(p, a, M, K, g)
    h = 1e-6

    def fd(**kw):
        plus = {k: v[0] for k, v in kw.items()}
        minus = {k: v[1] for k, v in kw.items()}
        return (loss(**plus) - loss(**minus)) / (2 * h)

    scale = max(np.abs(g_eps).max(), np.abs(g_hop).max(), np.abs(g_delta).max())
    tol = dict(rel=1e-6, abs=1e-8 * scale)
    for i in sites:
        e1, e2 = p.eps.copy(), p.eps.copy()
        e1[i] += h
        e2[i] -= h
        assert g_eps[i] == pytest.approx(fd(eps=(e1, e2)), **tol)
        if p.pairing != wl.BOND:
            for unit, part in ((1.0, np.real), (1j, np.imag)):
                d1, d2 = p.delta0.copy(), p.delta0.copy()
                d1[i] += unit * h
                d2[i] -= unit * h
                assert part(g_delta[i]) == pytest.approx(fd(delta=(d1, d2)), **tol)
    hop = p.hop.reshape(p.N, -1)
    for (i, d) in bonds:
        j = orc.neighbour(lat, i, d)
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            h1, h2 = hop.copy(), hop.copy()
            h1[i, d] += unit * h          # t_{i,d} and its Hermitian mirror t_{j,d^1} = conj(t_{i,d})
            h1[j, d ^ 1] += np.conj(unit) * h
            h2[i, d] -= unit * h
            h2[j, d ^ 1] -= np.conj(unit) * h
            assert part(g_hop[i, d]) == pytest.approx(fd(hop=(h1, h2)), **tol)
        assert g_hop[j, d ^ 1] == pytest.approx(np.conj(g_hop[i, d]), rel=1e-12, abs=1e-14)
    for (i, d) in pair_bonds:
        j = orc.neighbour(lat, i, d)
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            d1, d2 = p.delta0.copy(), p.delta0.copy()
            d1[i, d] += unit * h          # symmetric pairing: Delta_{j,d^1} moves with Delta_{i,d}
            d1[j, d ^ 1] += unit * h
            d2[i, d] -= unit * h
            d2[j, d ^ 1] -= unit * h
            assert part(g_delta[i, d]) == pytest.approx(fd(delta=(d1, d2)), **tol)
        assert g_delta[j, d ^ 1] == pytest.approx(g_delta[i, d], rel=1e-12, abs=1e-14)
    assert scale > 1e-3


def test_general_map_gradient_field_nnn_onsite_vs_finite_differences():
    """Complex hoppings (uniform field, Peierls phases), t' and complex Delta_i:
    the general reverse mode vs central differences of the oracle's
    order parameter (Re and Im of eps, every hopping kind, Delta)."""
    p = wl.random_swave(4, 32, seed=84, periodic=1, complex_delta=True, flux_quanta=1.0, tp=-0.3, T=0.05)
    _fd_check_general(p, 32, 5, sites=(0, 6, 15), bonds=((0, 0), (5, 2), (6, 4), (9, 7), (3, 1)),
                      pair_bonds=())


def test_general_map_gradient_dwave_bonds_vs_finite_differences():
    """Bond pairing (d-wave, complex symmetric Delta_ij) with a field: gradients
    for eps, the hoppings and each bond amplitude vs central differences."""
    p = wl.random_dwave(4, 24, seed=85, flux_quanta=1.0)
    p.T = 0.05
    _fd_check_general(p, 24, 6, sites=(0, 7, 13), bonds=((0, 0), (5, 2), (6, 4), (10, 6)),
                      pair_bonds=((0, 0), (5, 2), (7, 1), (12, 3)))


def test_general_map_gradient_reduces_to_the_real_one():
    """On a real lattice with a real g the general reverse mode gives the real
    routine's gradients (independently pinned above), with zero imaginary
    parts."""
    M, K = 40, 1 << 12
    p = wl.random_swave(5, M, seed=86, T=0.05)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    C = orc.fold_coefficients(M, K, a, p.T)
    w = np.random.default_rng(8).normal(size=p.N)
    ge, gh, gd = orc.scf_map_gradient(lat, a, C, w)
    he, hh, hd = orc.map_gradient_general(lat, a, C, w.astype(np.complex128))
    assert np.allclose(he, ge, rtol=1e-12, atol=1e-15)
    assert np.allclose(hh.real, gh, rtol=1e-12, atol=1e-15) and np.abs(hh.imag).max() < 1e-15
    assert np.allclose(hd.real, gd, rtol=1e-12, atol=1e-15) and np.abs(hd.imag).max() < 1e-15


def _ldos_loss_lattice(seed):
    M = 40
    p = wl.random_swave(4, M, seed=seed, T=0.05)
    return p, as_oracle(p), M


@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 3.0)])
def test_ldos_gradient_vs_finite_differences(kernel, lam):
    """Reverse-mode gradient of L = sum_{c,e} G[c,e] LDOS(E_e, i_c) (Eq. 17
    with Eq. 10, Jackson or Lorentz damping) vs central differences (h = 1e-6)
    of the oracle's LDOS, a frozen; a repeated start site counts twice."""
    p, lat, M = _ldos_loss_lattice(82)
    a = orc.rescale(lat)
    sites = np.array([0, 5, 10, 15, 6, 5], dtype=np.int32)
    E = np.linspace(-0.85, 0.8, 9) * a
    G = np.random.default_rng(4).normal(size=(sites.size, E.size))
    g_eps, g_hop, g_delta = orc.ldos_gradient(lat, a, sites, M, E, G, kernel, lam)

    def loss(eps=None, hop=None, delta=None):
        l2 = orc.Lattice(p.Lx, p.Ly, 0, 0, p.eps if eps is None else eps, p.mu,
                         p.hop if hop is None else hop, 0, p.coupling,
                         p.delta0 if delta is None else delta)
        return float((G * orc.ldos(l2, a, sites, M, E, kernel, lam)).sum())

    h = 1e-6
    for i in (0, 5, 9, 15):
        e1, e2 = p.eps.copy(), p.eps.copy()
        e1[i] += h
        e2[i] -= h
        assert g_eps[i] == pytest.approx((loss(eps=e1) - loss(eps=e2)) / (2 * h), rel=1e-6, abs=1e-9)
        d1, d2 = p.delta0.copy(), p.delta0.copy()
        d1[i] += h
        d2[i] -= h
        assert g_delta[i] == pytest.approx((loss(delta=d1) - loss(delta=d2)) / (2 * h), rel=1e-6, abs=1e-9)
    for (i, d) in ((0, 0), (5, 2), (6, 1), (14, 3)):
        j = orc.neighbour(lat, i, d)
        h1, h2 = p.hop.copy(), p.hop.copy()
        h1[i, d] += h
        h1[j, d ^ 1] += h
        h2[i, d] -= h
        h2[j, d ^ 1] -= h
        assert g_hop[i, d] == pytest.approx((loss(hop=h1) - loss(hop=h2)) / (2 * h), rel=1e-6, abs=1e-9)
        assert g_hop[j, d ^ 1] == pytest.approx(g_hop[i, d], rel=1e-12)
    assert np.abs(g_eps).max() > 1e-3 and np.abs(g_hop).max() > 1e-3 and np.abs(g_delta).max() > 1e-3


@pytest.mark.parametrize("kernel,lam", [(0, 0.0), (1, 2.0)])
def test_ldos_gradient_of_quadrature_moments(kernel, lam):
    """Closed forms: with K-node Gauss-Chebyshev weights, sum_k w_k LDOS(E_k)
    is the exact integral of the truncated series, i.e. g_0 mu_0 = 1 for every
    lattice, so its gradient vanishes; and sum_k w_k E_k LDOS(E_k) = a g_1 mu_1
    = g_1 (eps_i - mu) (mu_1 = <e_i|H~|e_i>), so its gradient is g_1 on eps_i
    of each listed site and zero for every hopping and Delta."""
    p, lat, M = _ldos_loss_lattice(83)
    a = orc.rescale(lat)
    K = 64  # 2K > M + 1: both identities are exact
    th = np.pi * (np.arange(K) + 0.5) / K
    x = np.cos(th)
    E = a * x
    w = np.pi * a / K * np.sqrt(1.0 - x * x)
    sites = np.array([1, 7, 12, 7], dtype=np.int32)
    G0 = np.tile(w, (sites.size, 1))
    g_eps, g_hop, g_delta = orc.ldos_gradient(lat, a, sites, M, E, G0, kernel, lam)
    assert np.abs(g_eps).max() < 1e-12 and np.abs(g_hop).max() < 1e-12 and np.abs(g_delta).max() < 1e-12
    # the integral itself is 1 at every listed site
    rho = orc.ldos(lat, a, sites, M, E, kernel, lam)
    assert np.allclose((rho * w).sum(1), 1.0, atol=1e-12)
    g1 = (orc.jackson(M) if kernel == 0 else orc.lorentz(M, lam))[1]
    g_eps, g_hop, g_delta = orc.ldos_gradient(lat, a, sites, M, E, G0 * E, kernel, lam)
    want = np.zeros(p.N)
    for i in sites:
        want[i] += g1
    assert np.allclose(g_eps, want, atol=1e-12)
    assert np.abs(g_hop).max() < 1e-12 and np.abs(g_delta).max() < 1e-12


# ---------------------------------------------------------------- site-dependent coupling


def _site_lattice(p, cpl):
    return orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu, p.hop, p.pairing,
                       p.coupling, p.delta0, coupling_site=cpl)


def test_site_coupling_onsite_matches_ed():
    """U_i per site (zero on a normal strip, as in an S/N junction):
    Delta_i = (U_i/2) sum_k u_k(i) conj(v_k(i)) F_M(E_k/a), exactly zero where
    U_i = 0, and n_i unaffected; the sampled-site routine agrees."""
    M, K = 96, 1 << 13
    p = wl.random_swave(5, M, seed=91, periodic=1, complex_delta=True, flux_quanta=2.0, T=0.05)
    U = np.random.default_rng(4).uniform(1.0, 3.0, p.N)
    U[(np.arange(p.N) % p.Lx) >= 3] = 0.0
    lat = _site_lattice(p, U)
    a = orc.rescale(lat)
    d, nn = orc.order_parameter(lat, a, p.T, M, K)
    C = orc.fold_coefficients(M, K, a, p.T)
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    F = sum(C[n] * cheb_T(n, w / a) for n in range(M))
    u, v = V[0::2], V[1::2]
    assert np.allclose(d, 0.5 * U * (u * np.conj(v) * F).sum(1), atol=1e-12)
    assert np.all(d[U == 0.0] == 0.0)
    _, n_scalar = orc.order_parameter(as_oracle(p), a, p.T, M, K)
    assert np.array_equal(nn, n_scalar)
    sites = np.array([0, 7, 4, 0])
    ds, _ = orc.order_parameter_sites(lat, a, p.T, M, K, sites)
    assert np.array_equal(ds, d[sites])


def test_site_coupling_bond_matches_ed():
    """V_{i,d} per bond (symmetric): each bond's Delta scales by its own V."""
    M, K = 64, 1 << 13
    p = wl.random_dwave(4, M, seed=92, flux_quanta=2.0)
    lat0 = as_oracle(p)
    rng = np.random.default_rng(5)
    Vb = np.zeros((p.N, 4))
    for i in range(p.N):
        for dd in (0, 2):
            j = orc.neighbour(lat0, i, dd)
            Vb[i, dd] = Vb[j, dd ^ 1] = rng.uniform(0.5, 2.0)
    lat = _site_lattice(p, Vb)
    a = orc.rescale(lat)
    d, _ = orc.order_parameter(lat, a, p.T, M, K)
    d0, _ = orc.order_parameter(lat0, a, p.T, M, K)
    assert np.allclose(d, d0 * Vb / p.coupling, atol=1e-13)
    C = orc.fold_coefficients(M, K, a, p.T)
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    F = sum(C[n] * cheb_T(n, w / a) for n in range(M))
    i, dd = 5, 2
    j = orc.neighbour(lat, i, dd)
    ref = Vb[i, dd] / 8 * ((V[2 * i] * np.conj(V[2 * j + 1]) + V[2 * j] * np.conj(V[2 * i + 1])) * F).sum()
    assert d[i, dd] == pytest.approx(ref, abs=1e-12)
    ds, _ = orc.order_parameter_bonds(lat, a, p.T, M, K, np.array([i, 0]))
    assert np.allclose(ds, d[[i, 0]], atol=1e-15)


def test_site_coupling_uniform_equals_scalar_and_gradient():
    """A uniform coupling array reproduces the scalar bit for bit; the
    reverse-mode gradient with U_i matches central differences."""
    M, K = 48, 1 << 12
    p = wl.random_swave(4, M, seed=93, T=0.05)
    a = orc.rescale(as_oracle(p))
    d_s, n_s = orc.order_parameter(as_oracle(p), a, p.T, M, K)
    d_u, n_u = orc.order_parameter(_site_lattice(p, np.full(p.N, p.coupling)), a, p.T, M, K)
    assert np.array_equal(d_s, d_u) and np.array_equal(n_s, n_u)
    U = np.where(np.arange(p.N) % 2 == 0, 2.5, 0.0)
    lat = _site_lattice(p, U)
    C = orc.fold_coefficients(M, K, a, p.T)
    w = np.random.default_rng(6).normal(size=p.N)
    g_eps, _, g_delta = orc.scf_map_gradient(lat, a, C, w)

    def loss(eps=None, delta=None):
        l2 = orc.Lattice(p.Lx, p.Ly, 0, 0, p.eps if eps is None else eps, p.mu, p.hop, 0, p.coupling,
                         p.delta0 if delta is None else delta, coupling_site=U)
        d, _ = orc.order_parameter(l2, a, p.T, M, K)
        return float((w * d.real).sum())

    h = 1e-6
    for i in (0, 3, 6, 9):
        e1, e2 = p.eps.copy(), p.eps.copy()
        e1[i] += h
        e2[i] -= h
        assert g_eps[i] == pytest.approx((loss(eps=e1) - loss(eps=e2)) / (2 * h), rel=1e-6, abs=1e-9)
        d1, d2 = p.delta0.copy(), p.delta0.copy()
        d1[i] += h
        d2[i] -= h
        assert g_delta[i] == pytest.approx((loss(delta=d1) - loss(delta=d2)) / (2 * h), rel=1e-6, abs=1e-9)


def test_tanh_coefficients_odd_and_half_node_identity():
    """tanh is odd and the Gauss-Chebyshev nodes are symmetric: the even c_n
    vanish (to round-off) and the odd c_n equal twice the sum over the first
    K/2 nodes, the identity the coefficient kernels use; also at T = 0."""
    M, K, a = 200, 4096, 6.3
    for T in (0.02, 0.0):
        c = orc.tanh_coefficients(M, K, a, T)
        assert np.abs(c[0::2]).max() < 1e-15
        k = np.arange(K // 2)
        x = np.cos(np.pi * (k + 0.5) / K)
        f = np.tanh(a * x / (2 * T)) if T > 0 else np.sign(x)
        n = np.arange(1, M, 2)
        half = 2.0 / K * (f[None, :] * np.cos(n[:, None] * np.pi * (k[None, :] + 0.5) / K)).sum(1)
        assert np.allclose(c[1::2], half, atol=1e-15, rtol=0)
