"""The LDOS of Eq. 17 and the tensor-core contraction behind it.

cbdg_contract_tf32x3 (tcgen05, 3xTF32) is checked against an FP64 matrix
product; cbdg_ldos against the oracle's LDOS, built from the oracle's own
moments.  Tolerance, from the arithmetic: each product keeps about 21 bits
(3xTF32) and the tensor cores accumulate in FP32 over M terms, so the error
of LDOS(E) is bounded by 1e-5 times the absolute series
sum_n |g_n (2 - delta_n0) mu_n T_n(E/a)| / (pi a sqrt(1 - (E/a)^2)); for the
small cases that is also within 1e-5 of max|LDOS|."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def contract(A, B):
    import torch
    m, k = A.shape
    n = B.shape[0]
    ld = (k + 3) // 4 * 4
    At = torch.zeros((m, ld), dtype=torch.float32, device="cuda")
    Bt = torch.zeros((n, ld), dtype=torch.float32, device="cuda")
    At[:, :k] = torch.from_numpy(A.astype(np.float32))
    Bt[:, :k] = torch.from_numpy(B.astype(np.float32))
    D = torch.full((m, n), float("nan"), dtype=torch.float32, device="cuda")
    cbdg.cbdg_contract_tf32x3(At, ld, Bt, ld, D, n, m, n, k)
    return D.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("m,n,k", [(128, 256, 32), (1, 1, 1), (300, 300, 100), (129, 257, 33),
                                   (640, 512, 2048), (200, 520, 600),
                                   # more tiles than SMs: each persistent CTA walks several tiles
                                   (25600, 520, 40), (20000, 300, 700)])
def test_contraction_matches_fp64_product(m, n, k):
    rng = np.random.default_rng(m * 7 + n + k)
    A = rng.standard_normal((m, k)).astype(np.float32).astype(np.float64)
    B = rng.standard_normal((n, k)).astype(np.float32).astype(np.float64)
    D = contract(A, B)
    ref = A @ B.T
    scale = np.abs(A) @ np.abs(B).T
    err = np.abs(D - ref) / scale
    # 3xTF32 products (~2^-21) plus FP32 accumulation over k terms (~sqrt(k) 2^-24)
    assert err.max() < 1e-5, (err.max(), np.unravel_index(err.argmax(), err.shape))


def test_contraction_unaligned_rows_and_presplit_planes():
    """Odd row strides and an offset base (no alignment), then the same
    product through split-once planes: identical bits."""
    import torch
    rng = np.random.default_rng(5)
    m, n, k, ld = 150, 70, 77, 79
    Ah = rng.standard_normal((m, ld)).astype(np.float32)
    Bh = rng.standard_normal((n, ld)).astype(np.float32)
    A_buf = torch.zeros(m * ld + 1, dtype=torch.float32, device="cuda")
    A_buf[1:] = torch.from_numpy(Ah.ravel())
    A = A_buf[1:]  # 4-byte aligned only
    B = torch.from_numpy(Bh).cuda()
    D = torch.empty((m, n), dtype=torch.float32, device="cuda")
    cbdg.cbdg_contract_tf32x3(A, ld, B, ld, D, n, m, n, k)
    ref = Ah[:, :k].astype(np.float64) @ Bh[:, :k].astype(np.float64).T
    scale = np.abs(Ah[:, :k]).astype(np.float64) @ np.abs(Bh[:, :k]).astype(np.float64).T
    assert (np.abs(D.cpu().numpy() - ref) / scale).max() < 1e-5
    kp = cbdg.cbdg_contract_kp(k)
    assert kp == 96 and cbdg.cbdg_contract_kp(0) == 0 and cbdg.cbdg_contract_kp(32) == 32
    ahi, alo = (torch.empty((m, kp), dtype=torch.float32, device="cuda") for _ in range(2))
    bhi, blo = (torch.empty((n, kp), dtype=torch.float32, device="cuda") for _ in range(2))
    cbdg.cbdg_split_tf32(A, ld, m, k, ahi, alo)
    cbdg.cbdg_split_tf32(B, ld, n, k, bhi, blo)
    # the planes hold TF32 values (low 13 mantissa bits clear), hi + lo ~ x, zero padding
    for p in (ahi, alo):
        assert int((p.view(torch.int32) & 0x1FFF).abs().sum()) == 0
    assert torch.all(ahi[:, k:] == 0) and torch.all(alo[:, k:] == 0)
    x = torch.from_numpy(Ah[:, :k]).cuda()
    assert float(((ahi[:, :k] + alo[:, :k]) - x).abs().max()) <= float(x.abs().max()) * 2.0 ** -21
    D2 = torch.empty_like(D)
    cbdg.cbdg_contract_tf32x3_planes(ahi, alo, bhi, blo, kp, D2, n, m, n)
    assert torch.equal(D, D2)
    with pytest.raises(cbdg.CbdgError):
        cbdg.cbdg_contract_tf32x3_planes(ahi, alo, bhi, blo, 48, D2, n, m, n)


def test_contraction_structured_layout():
    """Each A row and B row a distinct one-hot pattern: any swizzle or
    transposition mistake shows up as a misplaced entry."""
    m, n, k = 128, 256, 64
    A = np.zeros((m, k))
    B = np.zeros((n, k))
    for i in range(m):
        A[i, i % k] = 1.0 + i
    for j in range(n):
        B[j, (3 * j) % k] = 1.0 + 0.5 * j
    D = contract(A, B)
    assert np.array_equal(D, A @ B.T)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["swave_open", "dwave_field"])
def test_ldos_matches_oracle(case, precision):
    M = 160
    if case == "swave_open":
        p = wl.random_swave(9, M, seed=51)
    else:
        p = wl.random_dwave(8, M, seed=52, flux_quanta=2.0)
    lat = cbdg.Lattice(p, precision=precision, complex_field=(case != "swave_open"))
    sites = np.array([0, 5, 17, 40, 63, 5], dtype=np.int32)
    lat.moments(sites[:1], 4)  # sets the rescale
    a = lat.rescale
    E = a * np.linspace(-0.9, 0.9, 77)
    rho = lat.ldos(sites, M, E)
    mu_ee, _ = orc.moments(as_oracle(p), a, sites, M)
    ref = orc.ldos_from_moments(mu_ee, a, E)
    assert max_abs(rho, ref) < 1e-5 * np.abs(ref).max(), max_abs(rho, ref) / np.abs(ref).max()


def test_ldos_vortex_256_full_lattice_sampled():
    """The full d-wave vortex lattice (256x256, complex Peierls hoppings,
    t' = -0.3) at M = 2048 and 512 energies in [-0.9a, 0.9a], LDOS of sampled
    sites vs the oracle (FP64 moments, same sites)."""
    p = wl.dwave_vortex(256, 2048)
    sites = np.array([1000, 40000], dtype=np.int32)
    lat = cbdg.Lattice(p, precision="fp64", complex_field=True)
    lat.moments(sites[:1], 4)
    a = lat.rescale
    E = a * p.extra["energy_frac"]
    rho = lat.ldos(sites, p.M, E)
    mu_ee, _ = orc.moments(as_oracle(p), a, sites, p.M)
    ref = orc.ldos_from_moments(mu_ee, a, E)
    # bound scale: the absolute series of Eq. 17 at each (site, E)
    g = orc.jackson(p.M) * np.where(np.arange(p.M) == 0, 1.0, 2.0)
    x = E / a
    T = np.cos(np.arange(p.M)[:, None] * np.arccos(x)[None, :])
    scale = (np.abs(mu_ee * g) @ np.abs(T)) / (np.pi * a * np.sqrt(1 - x * x))
    assert np.all(np.abs(rho - ref) <= 1e-5 * scale), (np.abs(rho - ref) / scale).max()
    assert max_abs(rho, ref) < 5e-5 * np.abs(ref).max()
    assert rho.min() > -1e-4 * rho.max()  # Jackson damping keeps the LDOS non-negative
