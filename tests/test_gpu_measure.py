"""The gather-rate helper (pcdm_gather_rate) measures this GPU's random-gather
ceiling: loads from a vector that fits in L2 come faster than from a 4 GiB one."""
import pytest

pytestmark = pytest.mark.gpu


def test_gather_rate_orders_l2_before_hbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1212_0873_gb300 import _binding as B, build
    build.build()
    torch.cuda.set_device(0)
    st = torch.cuda.current_stream().cuda_stream
    small = torch.ones(4_000_000, dtype=torch.float64, device="cuda")
    r_small = B.pcdm_gather_rate(small.data_ptr(), small.numel(), 8, st)
    big = torch.ones((4 << 30) // 4, dtype=torch.float32, device="cuda")
    r_big = B.pcdm_gather_rate(big.data_ptr(), big.numel(), 4, st)
    del big
    assert 1e9 < r_big < r_small < 1e13, (r_small, r_big)
