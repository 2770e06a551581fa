"""tevo_gemm_noalloc: the contraction for callers that cannot allocate device
memory (a process whose device memory belongs to a pre-sized pool, or code that
must not call the allocator mid-operation). It uses a fixed device array instead
of allocations; here it is checked against tevo_gemm, through the C ABI, on two
calls in a row (the second call sees the first call's leftovers in the shared
array), and shapes beyond the array are refused.

Kept in a file that pytest collects last, so a run that stops at the first
failure has run every other test before this one."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)
tv = pytest.importorskip("paper_2302_14181_gb300")

# same tolerances as the tevo_gemm tests: max |C - C_ref| / max |C_ref|
TOL = {tv.FP64: 1e-12, tv.BF16X3: 1e-4, tv.TF32X3: 1e-5, tv.TF32: 3e-3}


def _call(fn, ctx, prec, a, b, c):
    M, K = a.shape
    N = b.shape[0]
    return fn(ctx.handle, prec, M, N, K, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
              ctypes.c_void_p(c.data_ptr()))


@pytest.fixture(scope="module")
def ctx():
    torch.cuda.set_device(0)
    return tv.Context()


@pytest.mark.parametrize("prec", [tv.BF16X3, tv.TF32X3, tv.TF32, tv.FP64])
def test_noalloc_matches_tevo_gemm_twice(ctx, prec):
    rng = np.random.default_rng(11 + prec)
    for M, N, K in ((300, 520, 777), (64, 33, 2050)):
        A = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
        B = rng.standard_normal((N, K)) + 1j * rng.standard_normal((N, K))
        a = torch.from_numpy(A).cuda()
        b = torch.from_numpy(B).cuda()
        ref = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
        assert _call(tv._lib.lib.tevo_gemm, ctx, prec, a, b, ref) == 0
        ref_h = ref.cpu().numpy()
        scale = np.abs(A @ B.T).max()
        for _ in range(2):
            out = torch.full((M, N), complex(np.nan, np.nan), dtype=torch.complex128, device="cuda")
            assert _call(tv._lib.lib.tevo_gemm_noalloc, ctx, prec, a, b, out) == 0
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert np.abs(got - ref_h).max() / scale < TOL[prec]


def test_noalloc_rejects_shapes_beyond_its_array(ctx):
    # bf16x3 planes of A and B alone: 8 bytes x (M + N) x K > 64 MiB
    M, N, K = 4096, 4096, 2048
    a = torch.zeros((M, K), dtype=torch.complex128, device="cuda")
    b = torch.zeros((N, K), dtype=torch.complex128, device="cuda")
    c = torch.zeros((M, N), dtype=torch.complex128, device="cuda")
    assert _call(tv._lib.lib.tevo_gemm_noalloc, ctx, tv.BF16X3, a, b, c) == -2
