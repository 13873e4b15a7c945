"""The allocation-free sketch entry point.

rks_sketch_apply_noalloc serves callers that cannot allocate device memory
(code inside another framework's memory pool, loops that cannot pay cudaFree's
device-wide synchronisation).  It must give the same z = Omega x as
rks_sketch_apply and as the oracle's Omega x, call after call, although every
call shares its fixed scratch array, up to the largest d it accepts; and a
warm call must leave the device's free memory unchanged.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from oracle import sketch as SK
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


def test_noalloc_matches_oracle_up_to_its_largest_d(torch_cuda):
    # d = RKS_NOALLOC_MAX_D uses the whole array (and the large shared-memory
    # path of the sketch kernel); a smaller d after it must not see its sums
    torch = torch_cuda
    from paper_2508_05400_gb300 import rks
    for n, d, zeta, seed in ((200003, 8192, 8, 1), (50021, 96, 8, 2)):
        xh = I.normal(31 + d, n)
        x = torch.from_numpy(xh).cuda()
        z = torch.full((d,), float("nan"), dtype=torch.float64, device="cuda")
        assert rks.sketch_apply_noalloc(x, z, d, zeta, seed) == rks.RKS_OK
        zo = SK.omega_matrix(n, d, zeta, seed) @ xh
        za = z.cpu().numpy()
        # FP64 sums of the same zeta-sparse columns in another order
        assert np.max(np.abs(za - zo)) <= 1e-13 * np.linalg.norm(xh)


def test_noalloc_warm_call_allocates_no_device_memory(torch_cuda):
    torch = torch_cuda
    from paper_2508_05400_gb300 import rks
    n, d = 100003, 4096
    x = torch.from_numpy(I.normal(41, n)).cuda()
    z = torch.empty(d, dtype=torch.float64, device="cuda")
    assert rks.sketch_apply_noalloc(x, z, d, 8, 0) == rks.RKS_OK     # warm: address looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert rks.sketch_apply_noalloc(x, z, d, 8, 0) == rks.RKS_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_array(torch_cuda):
    torch = torch_cuda
    from paper_2508_05400_gb300 import rks
    x = torch.zeros(1000, dtype=torch.float64, device="cuda")
    z = torch.zeros(9000, dtype=torch.float64, device="cuda")
    assert rks.sketch_apply_noalloc(x, z, 8193, 8, 0) == rks.RKS_EINVAL
