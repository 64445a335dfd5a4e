"""The allocation-free sign-function entry point against the allocating one.

Callers that cannot allocate device memory at apply time use
sign_apply_multishift_noalloc, whose workspace is a fixed static device array.
This checks, through the C ABI, that two calls in a row give the same result
as sign_apply_multishift (FP64 tolerance 1e-12), and that a problem larger
than the array is refused with a clear error.  Kept in a file that pytest
collects last.
"""
import numpy as np
import pytest
import torch

import synthetic_fields as sf
from paper_1701_00726_gb300 import BriError, Lattice

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point():
    dims = (4, 4, 4, 4)
    u = sf.gauge_field(dims, 0)
    x = torch.from_numpy(sf.gaussian_source(dims, 2, 1000)).cuda()
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(u).cuda(), 1.0)
    ref, st_ref = lat.sign_apply(x, n=8, rho=1.0, tol=1e-12)
    assert st_ref["converged"]
    refn = ref.cpu().numpy()
    out = torch.empty_like(x)
    allocs0 = Lattice.device_allocations()
    for _ in range(2):  # the static scratch keeps the previous call's contents
        y, st = lat.sign_apply_noalloc(x, n=8, rho=1.0, tol=1e-12, out=out)
        assert st["converged"]
        got = y.cpu().numpy()
        assert np.abs(got - refn).max() <= 1e-12 * np.abs(refn).max()
    # the defining property: no device allocation by the library in those calls
    assert Lattice.device_allocations() == allocs0
    big = torch.zeros((64,) + tuple(x.shape[1:]), dtype=torch.complex128, device="cuda")
    with pytest.raises(BriError, match="static scratch"):
        lat.sign_apply_noalloc(big, n=8)
    lat.close()


def test_noalloc_documented_size_limit():
    """8^4 with one right-hand side fits up to KL order 19; order 20 is refused."""
    dims = (8, 8, 8, 8)
    lat = Lattice(dims)
    lat.build_links(torch.from_numpy(sf.gauge_field(dims, 2)).cuda(), 0.0)
    x = torch.from_numpy(sf.gaussian_source(dims, 1, 1002)).cuda()
    out = torch.empty_like(x)
    allocs0 = Lattice.device_allocations()
    _, st = lat.sign_apply_noalloc(x, n=19, rho=1.0, tol=1e-10, out=out)
    assert st["converged"]
    assert Lattice.device_allocations() == allocs0
    with pytest.raises(BriError, match="static scratch"):
        lat.sign_apply_noalloc(x, n=20, out=out)
    lat.close()
