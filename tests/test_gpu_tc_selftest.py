"""tcgen05 operand path: one MMA chain through the product kernels' shared-memory layout and
descriptors against a host GEMM (exact on small integers, FP32-accurate on random data)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

import __graft_entry__  # noqa: E402

__graft_entry__.build()
from paper_2103_06393_gb300 import zbc  # noqa: E402


@pytest.mark.parametrize("fmt", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("N", [16, 32, 64])
def test_integer_exact(fmt, N):
    rng = np.random.default_rng(fmt * 100 + N)
    K = 32
    A = rng.integers(-3, 4, size=(128, K)).astype(np.float32)
    B = rng.integers(-3, 4, size=(N, K)).astype(np.float32)
    D = zbc.zbc_tc_selftest(A, B, fmt)
    assert np.array_equal(D, A @ B.T)


@pytest.mark.parametrize("fmt,K", [(0, 16), (1, 64), (2, 8), (2, 64), (3, 16), (3, 64), (4, 32)])
def test_random_against_rounded_host(fmt, K):
    rng = np.random.default_rng(K + fmt)
    A = rng.normal(size=(128, K)).astype(np.float32)
    B = rng.normal(size=(48, K)).astype(np.float32)
    if fmt in (0, 3):
        Ar, Br = A.astype(np.float16).astype(np.float64), B.astype(np.float16).astype(np.float64)
    elif fmt in (1, 4):
        Ar = torch.from_numpy(A).to(torch.bfloat16).double().numpy()
        Br = torch.from_numpy(B).to(torch.bfloat16).double().numpy()
    else:
        def tf32(x):
            i = x.view(np.uint32).astype(np.uint64)
            i = ((i + 0x1000) & ~np.uint64(0x1FFF)).astype(np.uint32)
            return i.view(np.float32).astype(np.float64)
        Ar, Br = tf32(A), tf32(B)
    D = zbc.zbc_tc_selftest(A, B, fmt)
    ref = Ar @ Br.T
    assert np.max(np.abs(D - ref)) <= 1e-5 * np.max(np.abs(ref))
