"""Pins of the oracle's nonlocal Green's functions and bond currents (no GPU).

The oracle reads the direct recursion of Eq. 15 at arbitrary target sites
(``green_moments``), builds the full retarded G(E) of gf1 from them
(``green_function``), and takes bond currents from the one-body density
matrix f(H) (``bond_currents``, Eq. 20 read as the continuity equation of the
hopping term of Eq. 2).  Each test checks one of them against something other
than the oracle itself: dense diagonalisation, Bloch-state closed forms,
exact conservation laws and symmetries, and the U-polynomial form of Eq. real1.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import workloads as wl

K_QUAD = 1 << 13


def as_oracle(p, delta=None, hop=None):
    return orc.Lattice(p.Lx, p.Ly, p.periodic_x, p.periodic_y, p.eps, p.mu,
                       p.hop if hop is None else hop, p.pairing, p.coupling,
                       p.delta0 if delta is None else delta)


def cheb_T(n, x):
    return np.cos(n * np.arccos(np.clip(x, -1.0, 1.0)))


def case_lattice(case, M=96):
    if case == "open_real":
        return wl.random_swave(4, M, seed=121)
    if case == "periodic_field":
        return wl.random_swave(4, M, seed=122, periodic=1, complex_delta=True, flux_quanta=2.0, T=0.05)
    if case == "nnn_field":
        return wl.random_swave(4, M, seed=123, periodic=1, complex_delta=True, flux_quanta=2.0, tp=-0.3,
                               T=0.05)
    return wl.random_dwave(4, M, seed=124, flux_quanta=2.0, T=0.05)


def ed_currents(lat, p, a, C, exact_T=None):
    """J[i, d] (both spins) from the dense density matrix.  With exact_T the
    Fermi function itself, else the damped series F_M = sum_n C_n T_n."""
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    if exact_T is None:
        F = sum(C[n] * cheb_T(n, w / a) for n in range(C.size))     # ~ tanh(E/2T)
    else:
        F = np.tanh(w / (2 * exact_T))
    f = 0.5 * (1.0 - F)
    rho = (V * f[None, :]) @ V.conj().T                              # <row|f(H)|col>
    J = np.zeros((lat.N, lat.n_dirs))
    for i in range(lat.N):
        for d in range(lat.n_dirs):
            j = orc.neighbour(lat, i, d)
            if j < 0:
                continue
            up = rho[2 * j, 2 * i]                       # <c+_{i up} c_{j up}> = <e_j|f|e_i>
            dn = -rho[2 * i + 1, 2 * j + 1]              # <c+_{i dn} c_{j dn}> = -<h_i|f|h_j>
            t = lat.hop[i * lat.n_dirs + d]
            J[i, d] = 2 * np.imag(t * up) + 2 * np.imag(t * dn)
    return J


def total_current(lat, a, T, M, **kw):
    return orc.bond_currents(lat, a, T, M, K_QUAD, spin=0, **kw) + \
        orc.bond_currents(lat, a, T, M, K_QUAD, spin=1, **kw)


# ------------------------------------------------------------ nonlocal moments


@pytest.mark.parametrize("case", ["open_real", "periodic_field", "nnn_field", "dwave_bonds"])
@pytest.mark.parametrize("start_part", [0, 1])
def test_green_moments_match_ed(case, start_part):
    """<alpha_t|T_n(H/a)|j_0> = sum_k V[t,k] conj(V[i,k]) T_n(E_k/a) for every
    target, both target parts and both start parts, to round-off: catches a
    transposed read, a wrong start row or a missing conjugate."""
    M = 64
    p = case_lattice(case, M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    w, V = orc.jacobi_eigh(orc.dense_hamiltonian(lat))
    sites = np.array([0, 5, lat.N - 1], dtype=np.int32)
    targets = np.arange(lat.N, dtype=np.int32)
    a_e, a_h = orc.green_moments(lat, a, sites, targets, M, start_part=start_part)
    Tn = cheb_T(np.arange(M)[:, None], (w / a)[None, :])            # [M, 2N]
    for c, i in enumerate(sites):
        start = V[2 * i + start_part].conj()                        # conj(<start|k>)
        ref_e = Tn @ (V[0::2] * start[None, :]).T                    # [M, N]
        ref_h = Tn @ (V[1::2] * start[None, :]).T
        assert np.allclose(a_e[c], ref_e, atol=1e-12, rtol=0)
        assert np.allclose(a_h[c], ref_h, atol=1e-12, rtol=0)


def test_green_moments_agree_with_onsite_moments():
    """The on-site targets reproduce the moments of the separate on-site and
    bond readout (mu_ee, <h_i|T_n|e_i>, <h_{i+d}|T_n|e_i>)."""
    M = 48
    p = case_lattice("dwave_bonds", M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    sites = np.arange(lat.N, dtype=np.int32)
    mu_ee, mu_eh = orc.moments(lat, a, sites, M)
    a_e, a_h = orc.green_moments(lat, a, sites, sites, M)
    for i in sites:
        assert np.allclose(a_e[i, :, i].real, mu_ee[i], atol=1e-14)
        assert np.abs(a_e[i, :, i].imag).max() < 1e-14
        assert np.allclose(a_h[i, :, i], mu_eh[i, :, 0], atol=1e-14)
        for d in range(4):
            j = orc.neighbour(lat, i, d)
            assert np.allclose(a_h[i, :, j], mu_eh[i, :, 1 + d], atol=1e-14)


def test_green_moments_hermitian_pairs():
    """T_n(H) is Hermitian: <e_j|T_n|e_i> = conj(<e_i|T_n|e_j>) from two
    different recursions."""
    M = 64
    p = case_lattice("nnn_field", M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    sites = np.arange(lat.N, dtype=np.int32)
    a_e, _ = orc.green_moments(lat, a, sites, sites, M)
    assert np.allclose(a_e, np.conj(np.transpose(a_e, (2, 1, 0))), atol=1e-13)


# ------------------------------------------------------------ Green's function


def test_green_function_imag_part_is_ldos():
    """-Im G_ii(E) / pi is the LDOS of Eq. 17 (computed by the separate
    LDOS routine) for both kernels."""
    M = 128
    p = case_lattice("periodic_field", M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    sites = np.array([0, 7], dtype=np.int32)
    a_e, _ = orc.green_moments(lat, a, sites, sites, M)
    diag = np.stack([a_e[0, :, 0], a_e[1, :, 1]])
    E = np.linspace(-0.9 * a, 0.9 * a, 41)
    for kernel, lam in ((0, 0.0), (1, 4.0)):
        G = orc.green_function(a_e, a, E, kernel=kernel, lam=lam)
        rho = orc.ldos_from_moments(diag.real, a, E, kernel=kernel, lam=lam)
        assert np.allclose(-G[0, 0].imag / np.pi, rho[0], atol=1e-12)
        assert np.allclose(-G[1, 1].imag / np.pi, rho[1], atol=1e-12)


def test_green_function_real_part_u_polynomials():
    """Re G of a real moment sequence equals Eq. real1,
    -(2/a) sum_{n>=1} g_n mu_n U_{n-1}(x), with U from its own recurrence."""
    M = 96
    p = case_lattice("open_real", M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    s = np.array([3], dtype=np.int32)
    a_e, _ = orc.green_moments(lat, a, s, s, M)
    mu = a_e[0, :, 0].real
    g = orc.jackson(M)
    E = np.linspace(-0.95 * a, 0.95 * a, 37)
    x = E / a
    U = np.zeros((M, x.size))                      # U[k] = U_{k-1}(x), U_{-1} = 0
    U[1] = 1.0
    if M > 2:
        U[2] = 2 * x
    for k in range(3, M):
        U[k] = 2 * x * U[k - 1] - U[k - 2]
    ref = -(2.0 / a) * ((g * mu)[1:, None] * U[1:]).sum(0)
    G = orc.green_function(a_e, a, E)
    assert np.allclose(G[0, 0].real, ref, atol=1e-11)


def test_green_function_single_level_lorentz():
    """Moments T_n(x0) of one level with the Lorentz kernel approximate the
    resolvent 1/(E - E0 + i eta): the kernel of Eq. 16 broadens by
    eps = lambda/M in theta = arccos(x), eta = a eps sin(theta0).  Away from the
    pole the two agree to 0.5%; at the pole the truncated kernel is a few
    percent low (its sum reaches 1 - e^{-lambda} of the Poisson kernel)."""
    M, lam, a, E0 = 4096, 4.0, 2.0, 0.3
    x0 = E0 / a
    mom = cheb_T(np.arange(M), x0).astype(np.complex128)[None, :, None]
    E = np.linspace(-1.0, 1.0, 81)
    G = orc.green_function(mom, a, E, kernel=1, lam=lam)[0, 0]
    eta = a * lam / M * np.sqrt(1 - x0 ** 2)
    ref = 1.0 / (E - E0 + 1j * eta)
    far = np.abs(E - E0) > 20 * eta
    assert (np.abs(G - ref) / np.abs(ref))[far].max() < 5e-3
    assert np.abs(G - ref).max() < 0.05 * np.abs(ref).max()


def test_green_function_matches_resolvent():
    """Nonlocal G^{11}_ij(E) and G^{12}_ij(E) with the Lorentz kernel vs the
    spectral sum sum_k <alpha_i|k><k|e_j> / (E - E_k + i eta_k) over the dense
    eigenpairs, eta_k = a (lambda/M) sin(arccos(E_k/a)): a transposed pair,
    a conjugate or the sign of the real part would miss by order one."""
    M, lam = 4096, 3.0
    p = case_lattice("periodic_field", M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    i, j = 2, 13
    a_e, a_h = orc.green_moments(lat, a, np.array([j], np.int32), np.array([i], np.int32), M)
    E = np.linspace(-0.6 * a, 0.6 * a, 25)
    G11 = orc.green_function(a_e, a, E, kernel=1, lam=lam)[0, 0]
    G12 = orc.green_function(a_h, a, E, kernel=1, lam=lam)[0, 0]
    w, V = np.linalg.eigh(orc.dense_hamiltonian(lat))
    eta = a * lam / M * np.sqrt(1 - (w / a) ** 2)
    res = 1.0 / (E[:, None] - w[None, :] + 1j * eta[None, :])       # [n_E, 2N]
    ref11 = res @ (V[2 * i] * V[2 * j].conj())
    ref12 = res @ (V[2 * i + 1] * V[2 * j].conj())
    scale = max(np.abs(ref11).max(), np.abs(ref12).max())
    far = np.abs(E[:, None] - w[None, :]).min(1) > 20 * eta.max()
    assert far.sum() >= 10
    for G, ref in ((G11, ref11), (G12, ref12)):
        assert np.abs(G - ref)[far].max() < 5e-3 * scale      # away from the poles
        assert np.abs(G - ref).max() < 0.05 * scale           # truncated kernel at a pole


# ------------------------------------------------------------ bond currents


@pytest.mark.parametrize("case", ["open_real", "periodic_field", "nnn_field", "dwave_bonds"])
def test_bond_currents_match_ed(case):
    """J (both spins) vs 2 Im[t <c+_i c_j>] with the density matrix
    V f_M(E) V^dagger from dense diagonalisation, f_M = (1 - F_M)/2 with the
    same damped series: exact to round-off.  Catches a wrong direction of the
    read, a sign of the current or a dropped spin."""
    M = 128
    p = case_lattice(case, M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    C = orc.fold_coefficients(M, K_QUAD, a, p.T)
    J = total_current(lat, a, p.T, M)
    ref = ed_currents(lat, p, a, C)
    assert np.allclose(J, ref, atol=1e-12, rtol=0)
    if case == "open_real":
        assert np.abs(J).max() < 1e-13              # a real H carries no current
    else:
        assert np.abs(J).max() > 1e-3


def test_bond_currents_spin_and_bond_symmetry():
    """J_up (electron starts) = J_down (hole starts) by particle-hole symmetry,
    and J_{i->j} = -J_{j->i} from two different start vectors."""
    M = 96
    p = case_lattice("nnn_field", M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    up = orc.bond_currents(lat, a, p.T, M, K_QUAD, spin=0)
    dn = orc.bond_currents(lat, a, p.T, M, K_QUAD, spin=1)
    assert np.allclose(up, dn, atol=1e-14)
    for i in range(lat.N):
        for d in range(lat.n_dirs):
            j = orc.neighbour(lat, i, d)
            assert up[i, d] == pytest.approx(-up[j, d ^ 1], abs=1e-14)


@pytest.mark.parametrize("periodic", [0, 1])
def test_normal_state_currents_conserved(periodic):
    """Delta = 0: f_M(H) commutes with H, so the hopping currents out of every
    site sum to zero exactly (no pairing source), whatever M."""
    M = 40
    p = wl.random_swave(5, M, seed=131, periodic=periodic, flux_quanta=2.0 if periodic else 0.0, tp=-0.3)
    hop = p.hop
    if not periodic:   # a field on an open lattice: random phases on every bond
        rng = np.random.default_rng(3)
        hop = hop.copy()
        lat0 = as_oracle(p)
        for i in range(p.N):
            for d in (0, 2, 4, 7):
                j = orc.neighbour(lat0, i, d)
                if j >= 0:
                    hop[i, d] *= np.exp(1j * rng.uniform(-1, 1))
                    hop[j, d ^ 1] = np.conj(hop[i, d])
    lat = as_oracle(p, delta=np.zeros(p.N, dtype=complex), hop=hop)
    a = orc.rescale(lat)
    J = total_current(lat, a, 0.1, M)
    assert np.abs(J).max() > 1e-3
    assert np.abs(J.sum(1)).max() < 1e-13


def test_uniform_ring_closed_form():
    """Clean periodic normal metal with phase phi on every +x bond: Bloch
    states give, per spin, J_x = (2/N) sum_k sin(kx + phi) f_M(xi_k) and
    J_y = 0, xi_k = -2 cos(kx + phi) - 2 cos ky - mu."""
    Lx, Ly, M, T, mu, phi = 7, 5, 80, 0.2, -0.4, 0.37
    N = Lx * Ly
    hop = wl.square_hops(Lx, Ly, 1, 1).astype(np.complex128)
    for s in range(N):
        x, y = s % Lx, s // Lx
        j = (x + 1) % Lx + Lx * y
        hop[s, 0] = np.exp(1j * phi)
        hop[j, 1] = np.exp(-1j * phi)
    lat = orc.Lattice(Lx, Ly, 1, 1, np.zeros(N), mu, hop, 0, 2.0, np.zeros(N, dtype=complex))
    a = orc.rescale(lat)
    J = orc.bond_currents(lat, a, T, M, K_QUAD, spin=0)
    C = orc.fold_coefficients(M, K_QUAD, a, T)
    kx = 2 * np.pi * np.arange(Lx) / Lx
    ky = 2 * np.pi * np.arange(Ly) / Ly
    KX, KY = np.meshgrid(kx, ky)
    xi = (-2 * np.cos(KX + phi) - 2 * np.cos(KY) - mu).ravel()
    f = 0.5 * (1 - sum(C[n] * cheb_T(n, xi / a) for n in range(M)))
    jx = 2.0 / N * (np.sin(KX.ravel() + phi) * f).sum()
    assert np.allclose(J[:, 0], jx, atol=1e-13)
    assert np.allclose(J[:, 1], -jx, atol=1e-13)
    assert np.abs(J[:, 2:]).max() < 1e-13


def test_time_reversal_and_gauge():
    """Conjugating H (t -> t*, Delta -> Delta*) reverses every current; a
    gauge transformation t_ij -> t_ij e^{i(chi_j - chi_i)},
    Delta_i -> Delta_i e^{-2 i chi_i} leaves them unchanged."""
    M = 96
    p = case_lattice("periodic_field", M)
    lat = as_oracle(p)
    a = orc.rescale(lat)
    J = total_current(lat, a, p.T, M)
    lat_c = as_oracle(p, delta=np.conj(p.delta0), hop=np.conj(p.hop))
    assert np.allclose(total_current(lat_c, a, p.T, M), -J, atol=1e-13)
    chi = np.random.default_rng(9).uniform(-np.pi, np.pi, lat.N)
    hop2 = p.hop.copy()
    for i in range(lat.N):
        for d in range(p.n_dirs):
            j = orc.neighbour(lat, i, d)
            hop2[i, d] = p.hop[i, d] * np.exp(1j * (chi[j] - chi[i]))
    lat_g = as_oracle(p, delta=p.delta0 * np.exp(-2j * chi), hop=hop2)
    assert np.allclose(total_current(lat_g, a, p.T, M), J, atol=1e-12)


def test_josephson_phase_gradient():
    """Real hopping, Delta with a phase winding along x on a periodic strip:
    a supercurrent flows along x, odd in the winding, none along y."""
    L, M = 6, 128
    N = L * L
    hop = wl.square_hops(L, L, 1, 1)
    x = np.arange(N) % L
    eps = np.zeros(N)
    runs = []
    for q in (1, -1):
        delta = 0.4 * np.exp(2j * np.pi * q * x / L)
        lat = orc.Lattice(L, L, 1, 1, eps, -0.5, hop, 0, 2.0, delta)
        a = orc.rescale(lat)
        runs.append(total_current(lat, a, 0.05, M))
    assert np.abs(runs[0][:, 0]).min() > 1e-4
    assert np.allclose(runs[0], -runs[1], atol=1e-13)
    assert np.abs(runs[0][:, 2:]).max() < 1e-12


def test_currents_converge_to_fermi_function():
    """With more moments the damped series approaches tanh(E/2T): the
    currents approach those of the exact Fermi function (about M^-2 with the
    Jackson kernel once the kernel resolves T)."""
    errs = []
    for M in (512, 2048):
        p = case_lattice("periodic_field", M)
        lat = as_oracle(p)
        a = orc.rescale(lat)
        J = total_current(lat, a, p.T, M)
        ref = ed_currents(lat, p, a, None, exact_T=p.T)
        errs.append(np.abs(J - ref).max() / np.abs(ref).max())
    assert errs[1] < errs[0] / 8
    assert errs[1] < 6e-3
