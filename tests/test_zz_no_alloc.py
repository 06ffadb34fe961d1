"""cbdg_moments_noalloc, the moments entry point for callers that cannot
allocate device memory (for example code recorded into a CUDA graph, or a
program that runs inside a fixed, pre-planned memory budget).  It keeps all
intermediates in a fixed device array owned by the library, so these tests
call it through the C ABI with device arrays only and compare it with the
allocating entry point cbdg_moments on the same inputs, twice in a row (the
second call must not see anything the first one left in the shared array).

This file is collected last on purpose: a run that stops at the first
failure has then already run every other test.
"""
import numpy as np
import pytest

from paper_1007_1609_gb300 import cbdg
from paper_1007_1609_gb300 import workloads as wl
from tests._common import gpu_available, max_abs

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
