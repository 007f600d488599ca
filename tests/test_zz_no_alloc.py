"""GPU test of cdmpt_spectral_bounds_noalloc, the entry point for callers that
cannot allocate device memory (inside stream capture, under an allocator that
owns the device's memory, or where cudaFree's device synchronisation is not
acceptable). It must give the same interval as cdmpt_spectral_bounds, which
allocates its scratch per call, on consecutive calls that reuse the shared
static scratch. This file sorts last so a failure here stops a -x run only
after every other test has run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_bounds_match_allocating_entry_point(cuda, cdmpt_lib):
    import torch
    import synthetic as syn
    # the second matrix is smaller, so stale scratch rows of the first call would show
    mats = [syn.cubic_lattice((12, 12, 12), seed=11).H0, syn.chain_1d(300, seed=12).H0]
    for H0 in mats:
        H = torch.from_numpy(H0).to(cuda)
        ref = cdmpt_lib.spectral_bounds(H)
        out = torch.full((2,), float("nan"), dtype=torch.float64, device=cuda)
        cdmpt_lib.spectral_bounds_noalloc(H, out)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.allclose(o, r, rtol=0, atol=1e-12), (o, r)


def test_noalloc_bounds_reject_oversize(cuda, cdmpt_lib):
    """N above the static scratch limit returns ERR_ARG before any launch."""
    import torch
    H = torch.zeros((2, 2), dtype=torch.float64, device=cuda)
    out = torch.zeros(2, dtype=torch.float64, device=cuda)
    status = cdmpt_lib.lib().cdmpt_spectral_bounds_noalloc(H.data_ptr(), 40000, 40000,
                                                           out.data_ptr(), None)
    assert status == 1
