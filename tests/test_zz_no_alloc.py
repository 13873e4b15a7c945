"""The allocation-free sketch entry point against the allocating one.

rks_sketch_apply_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory pool, loops that cannot pay cudaFree's
device-wide synchronisation).  It must give the same z = Omega x as
rks_sketch_apply, call after call, although both calls share its fixed
scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2508_05400_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05400_gb300 import build as B
    B.build()
    return torch


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    from paper_2508_05400_gb300 import rks
    cases = [(262144, 320, 8, 0, 21), (100003, 80, 4, 3, 22)]   # the second call has a smaller d
    for n, d, zeta, seed, xseed in cases:
        x = torch.from_numpy(I.normal(xseed, n)).cuda()
        z_ref = rks.sketch_apply(x, d, zeta, seed)
        z = torch.full((d,), float("nan"), dtype=torch.float64, device="cuda")
        rc = rks.sketch_apply_noalloc(x, z, d, zeta, seed)
        assert rc == rks.RKS_OK
        torch.cuda.synchronize()
        a, b = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)


def test_noalloc_rejects_sizes_beyond_its_array(torch_cuda):
    torch = torch_cuda
    from paper_2508_05400_gb300 import rks
    x = torch.zeros(1000, dtype=torch.float64, device="cuda")
    z = torch.zeros(9000, dtype=torch.float64, device="cuda")
    assert rks.sketch_apply_noalloc(x, z, 8193, 8, 0) == rks.RKS_EINVAL
