"""The gather-rate probe (a diagnostic entry point) computes what it claims: per-thread sums of src[idx]."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2110_02901_b300 as rmb  # noqa: E402
from paper_2110_02901_b300 import build as rbuild  # noqa: E402


def test_gather_probe_checksum():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    g = torch.Generator(device="cuda").manual_seed(1)
    src = torch.rand(100000, device="cuda", generator=g)
    idx = torch.randint(0, 100000, (1 << 20,), dtype=torch.int32, device="cuda", generator=g)
    out = rmb.rmb_diag_gather_probe(src, idx, reps=3)
    want = 3 * src.double()[idx.long()].sum().item()
    assert abs(out.double().sum().item() - want) <= 1e-5 * abs(want)


def test_gather4_probe_checksum():
    """The tensor-memory-access form: same sums, through gather4 copies of 16-byte rows (src length
    a multiple of 4, including indices in the last row)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rbuild.build()
    g = torch.Generator(device="cuda").manual_seed(2)
    src = torch.rand(100000, device="cuda", generator=g)
    idx = torch.randint(0, 100000, (1 << 20,), dtype=torch.int32, device="cuda", generator=g)
    idx[:8] = torch.tensor([0, 1, 2, 3, 99996, 99997, 99998, 99999], dtype=torch.int32, device="cuda")
    out = rmb.rmb_diag_gather_probe_tma(src, idx, reps=3)
    assert torch.isfinite(out).all()
    want = 3 * src.double()[idx.long()].sum().item()
    assert abs(out.double().sum().item() - want) <= 1e-5 * abs(want)
