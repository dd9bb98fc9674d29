"""Unit test of the tcgen05 / TMA building blocks used by the tensor-core contraction:
one 128 x 128 x K BF16 GEMM with the shared-memory layouts of the joint kernels,
compared with a plain FP32 matrix product of the same BF16 values."""
import ctypes
import os

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def st():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build
    build.build()
    L = ctypes.CDLL(build.SELFTEST_LIB)
    f = L.jtfs_selftest_umma
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 3 + [ctypes.c_void_p] * 2
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("K,a_swz,b_mn", [(64, 128, 1), (32, 64, 1), (64, 64, 1), (128, 128, 1),
                                          (32, 32, 1), (64, 128, 0), (128, 64, 0)])
def test_umma_bf16_gemm(st, K, a_swz, b_mn):
    g = torch.Generator(device="cuda").manual_seed(K + a_swz + b_mn)
    A = torch.randn(128, K, device="cuda", generator=g).to(torch.bfloat16).contiguous()
    Bkn = torch.randn(K, 128, device="cuda", generator=g).to(torch.bfloat16)
    B = Bkn.contiguous() if b_mn else Bkn.t().contiguous()
    D = torch.full((128, 128), float("nan"), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = st(A.data_ptr(), B.data_ptr(), D.data_ptr(), K, a_swz, b_mn, status.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.float() @ Bkn.float()
    err = (D - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


@pytest.mark.parametrize("K,b_mn", [(32, 0), (64, 0)])
def test_umma_tf32_gemm(K, b_mn):
    """kind::tf32 with A and B K-major, against FP64 products of the FP32 operands (TF32
    keeps 10 mantissa bits).  An MN-major B operand gives zeros for kind::tf32 on this
    hardware (measured with this kernel), so the TF32 contraction reads Y transposed."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build
    build.build()
    L = ctypes.CDLL(build.SELFTEST_LIB)
    f = L.jtfs_selftest_umma_tf32
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 2
    f.restype = ctypes.c_int
    g = torch.Generator(device="cuda").manual_seed(7 * K + b_mn)
    A = torch.randn(128, K, device="cuda", generator=g).contiguous()
    Bkn = torch.randn(K, 128, device="cuda", generator=g)
    B = Bkn.contiguous() if b_mn else Bkn.t().contiguous()
    D = torch.full((128, 128), float("nan"), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert f(A.data_ptr(), B.data_ptr(), D.data_ptr(), K, b_mn, status.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.double() @ Bkn.double()
    err = (D.double() - ref).abs().max().item() / ref.abs().max().item()
    assert err < 2e-3, err


@pytest.mark.parametrize("K", [16, 32, 64])
def test_umma_bf16_gemm_a_in_tmem(K):
    """A stored into tensor memory with tcgen05.st (row r in lane r, two BF16 per column),
    B MN-major in shared memory: D = A B."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build
    build.build()
    L = ctypes.CDLL(build.SELFTEST_LIB)
    f = L.jtfs_selftest_umma_ta
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] + [ctypes.c_void_p] * 2
    f.restype = ctypes.c_int
    g = torch.Generator(device="cuda").manual_seed(100 + K)
    A = torch.randn(128, K, device="cuda", generator=g).to(torch.bfloat16).contiguous()
    Bkn = torch.randn(K, 128, device="cuda", generator=g).to(torch.bfloat16).contiguous()
    D = torch.full((128, 128), float("nan"), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = f(A.data_ptr(), Bkn.data_ptr(), D.data_ptr(), K, status.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    ref = A.float() @ Bkn.float()
    err = (D - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, err


@pytest.mark.parametrize("K,b_mn", [(64, 1), (128, 1), (64, 0), (128, 0)])
def test_umma_cta_pair_gemm(K, b_mn):
    """cta_group::2 on a cluster of two CTAs: D[256 x 128] = A B with A's rows and B's columns
    split between the two CTAs' shared memories and D's rows between their TMEMs; both CTAs
    must receive the same TMEM base from the collective allocation."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_08269_gb300 import build
    build.build()
    L = ctypes.CDLL(build.SELFTEST_LIB)
    f = L.jtfs_selftest_umma2
    f.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 3
    f.restype = ctypes.c_int
    g = torch.Generator(device="cuda").manual_seed(11 * K + b_mn)
    A = torch.randn(256, K, device="cuda", generator=g).to(torch.bfloat16).contiguous()
    Bkn = torch.randn(K, 128, device="cuda", generator=g).to(torch.bfloat16)
    B = Bkn.contiguous() if b_mn else Bkn.t().contiguous()
    D = torch.full((256, 128), float("nan"), device="cuda")
    status = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    info = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = f(A.data_ptr(), B.data_ptr(), D.data_ptr(), K, b_mn, status.data_ptr(), info.data_ptr(),
           None)
    assert rc == 0
    torch.cuda.synchronize()
    inf = info.cpu().tolist()
    assert status.cpu().tolist() == [0, 0], (status.cpu().tolist(), inf)
    assert inf[1] == 0 and inf[5] == 1 and inf[0] == inf[4], inf
    ref = A.float() @ Bkn.float()
    err = (D - ref).abs().max().item() / ref.abs().max().item()
    assert err < 1e-5, (err, inf)
