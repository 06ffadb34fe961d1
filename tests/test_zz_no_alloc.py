"""cbdg_moments_noalloc, the moments entry point for callers that cannot
allocate device memory while they run (for example a program that works
inside a fixed, pre-planned memory budget, or a plug-in whose host framework
owns the GPU's allocator).  It keeps all intermediates in a fixed device
array owned by the library, so these tests call it through the C ABI with
device arrays only and compare it with the allocating entry point
cbdg_moments on the same inputs, twice in a row (the second call must not see
anything the first one left in the shared array), and once directly with the
oracle.  They also check that the calls leave the device's free memory
unchanged and that a start site outside the lattice is reported, not
indexed.

This file is collected last on purpose: a run that stops at the first
failure has then already run every other test.
"""
import numpy as np
import pytest

from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import as_oracle, gpu_available, max_abs
from oracle import oracle as orc

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

TOL = {"fp64": 1e-11, "fp32": 1e-5}


def device_desc(p, precision):
    """A cbdg_lattice_desc whose arrays live in device memory (torch)."""
    import torch
    keep = {
        "eps": torch.from_numpy(np.ascontiguousarray(p.eps)).cuda(),
        "hop": torch.from_numpy(np.ascontiguousarray(p.hop)).cuda(),
        "delta": torch.from_numpy(np.ascontiguousarray(p.delta0)).cuda(),
    }
    d = cbdg.cbdg_lattice_desc()
    d.Lx, d.Ly = p.Lx, p.Ly
    d.periodic_x, d.periodic_y = p.periodic_x, p.periodic_y
    d.eps, d.hop, d.delta0 = (keep["eps"].data_ptr(), keep["hop"].data_ptr(),
                              keep["delta"].data_ptr())
    d.mu, d.n_dirs, d.pairing, d.coupling = p.mu, p.hop.shape[1], p.pairing, p.coupling
    d.precision = cbdg.PRECISIONS[precision]
    d.complex_field = 0
    return d, keep


def noalloc_moments(p, precision, sites, M):
    import torch
    d, keep = device_desc(p, precision)
    s = torch.from_numpy(sites).cuda()
    ee = torch.full((sites.size, M), np.nan, dtype=torch.float64, device="cuda")
    eh = torch.full((sites.size, M), np.nan, dtype=torch.complex128, device="cuda")
    cbdg.cbdg_moments_noalloc(d, s, sites.size, M, ee, eh)
    torch.cuda.synchronize()
    return ee.cpu().numpy(), eh.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_allocating_moments_twice(precision):
    p = wl.swave_disordered(24, 96, seed=5)
    rng = np.random.default_rng(3)
    sites = rng.choice(p.N, size=77, replace=False).astype(np.int32)
    lat = cbdg.Lattice(p, precision=precision)
    ref_ee, ref_eh = lat.moments(sites, p.M)
    lat.close()
    for _ in range(2):
        ee, eh = noalloc_moments(p, precision, sites, p.M)
        assert max_abs(ee, ref_ee) < TOL[precision]
        assert max_abs(eh, ref_eh[..., 0]) < TOL[precision]


def test_noalloc_chunks_many_start_sites():
    """A 128x128 lattice in FP64 fits only a few dozen columns per pass in the
    fixed array, so 300 start sites take several passes."""
    p = wl.swave_disordered(128, 16, seed=1001)
    sites = np.random.default_rng(8).choice(p.N, size=300, replace=False).astype(np.int32)
    lat = cbdg.Lattice(p, precision="fp64")
    ref_ee, ref_eh = lat.moments(sites, p.M)
    lat.close()
    for _ in range(2):
        ee, eh = noalloc_moments(p, "fp64", sites, p.M)
        assert max_abs(ee, ref_ee) < TOL["fp64"]
        assert max_abs(eh, ref_eh[..., 0]) < TOL["fp64"]


def test_noalloc_rejects_lattice_beyond_its_scratch():
    import torch
    L = 1024  # one FP64 slab of a 1024x1024 lattice needs well over 64 MiB
    d = cbdg.cbdg_lattice_desc()
    d.Lx = d.Ly = L
    d.periodic_x = d.periodic_y = 0
    d.n_dirs, d.pairing, d.precision, d.complex_field = 4, 0, 0, 0
    d.mu, d.coupling = -0.5, 2.0
    d.eps = d.hop = d.delta0 = 0
    sites = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(cbdg.CbdgError) as ei:
        cbdg.cbdg_moments_noalloc(d, sites, 1, 16, None, None)
    assert ei.value.status == cbdg.CBDG_ERR_INVALID_ARG
    assert "scratch" in str(ei.value)


def test_noalloc_matches_oracle_and_allocates_nothing():
    """Moments against the FP64 oracle directly (the definitions of Eq. 11 and
    Eq. 14 by the plain recursion of Eq. 15), and the device's free memory
    before and after calls that include a chunked 128x128 case."""
    import torch
    p = wl.swave_disordered(20, 64, seed=9)
    sites = np.random.default_rng(4).choice(p.N, size=37, replace=False).astype(np.int32)
    ol = as_oracle(p)
    oee, oeh = orc.moments(ol, orc.rescale(ol), sites, p.M)  # both sides: a = 1.1 x Gershgorin
    big = wl.swave_disordered(128, 16, seed=1001)
    big_sites = np.random.default_rng(8).choice(big.N, size=300, replace=False).astype(np.int32)
    noalloc_moments(p, "fp64", sites, p.M)  # warm-up: first call on this device
    noalloc_moments(big, "fp64", big_sites, big.M)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, _ = torch.cuda.mem_get_info()
    d, keep = device_desc(p, "fp64")
    s_dev = torch.from_numpy(sites).cuda()
    ee = torch.zeros((sites.size, p.M), dtype=torch.float64, device="cuda")
    eh = torch.zeros((sites.size, p.M), dtype=torch.complex128, device="cuda")
    bd, bkeep = device_desc(big, "fp64")
    bs_dev = torch.from_numpy(big_sites).cuda()
    bee = torch.zeros((big_sites.size, big.M), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        cbdg.cbdg_moments_noalloc(d, s_dev, sites.size, p.M, ee, eh)
        cbdg.cbdg_moments_noalloc(bd, bs_dev, big_sites.size, big.M, bee, None)
    torch.cuda.synchronize()
    free2, _ = torch.cuda.mem_get_info()
    assert free2 == free1, (free0, free1, free2)
    assert max_abs(ee.cpu().numpy(), oee) < TOL["fp64"]
    assert max_abs(eh.cpu().numpy(), oeh[..., 0]) < TOL["fp64"]


def test_noalloc_reports_a_start_site_outside_the_lattice():
    """A site index >= N is caught on the GPU (never used as an index) and the
    call returns CBDG_ERR_INVALID_ARG; the next valid call is unaffected."""
    import torch
    p = wl.swave_disordered(16, 32, seed=2)
    d, keep = device_desc(p, "fp32")
    bad = torch.tensor([3, p.N, 5], dtype=torch.int32, device="cuda")
    ee = torch.zeros((3, p.M), dtype=torch.float64, device="cuda")
    with pytest.raises(cbdg.CbdgError) as ei:
        cbdg.cbdg_moments_noalloc(d, bad, 3, p.M, ee, None)
    assert ei.value.status == cbdg.CBDG_ERR_INVALID_ARG
    assert "start site" in str(ei.value)
    neg = torch.tensor([-1], dtype=torch.int32, device="cuda")
    with pytest.raises(cbdg.CbdgError):
        cbdg.cbdg_moments_noalloc(d, neg, 1, p.M, None, None)
    sites = np.array([3, 7, 5], dtype=np.int32)
    lat = cbdg.Lattice(p, precision="fp32")
    ref_ee, _ = lat.moments(sites, p.M)
    lat.close()
    ee2, _ = noalloc_moments(p, "fp32", sites, p.M)
    assert max_abs(ee2, ref_ee) < TOL["fp32"]
