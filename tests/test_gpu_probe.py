"""The FP64 issue-cost probe (grbk_fp64_issue_probe) through the C ABI: finite,
positive cycle counts; a division costs more than an add; 16 warps sharing one
SM's FP64 unit see at least the one-warp cost; argument checks."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2408_05444_gb300 as g  # noqa: E402


def test_issue_probe_orders_costs():
    add1 = g.grbk_fp64_issue_probe("add", 1, 32, 1024)
    div1 = g.grbk_fp64_issue_probe("div", 1, 32, 256)
    add16 = g.grbk_fp64_issue_probe("add", 16, 32, 1024)
    add16_one_lane = g.grbk_fp64_issue_probe("add", 16, 1, 1024)
    assert 0 < add1 < div1
    assert add16 >= 0.9 * add1
    assert add16_one_lane > 0


def test_issue_probe_rejects_bad_arguments():
    L = g.lib()
    import ctypes
    c = ctypes.c_double(0.0)
    assert L.grbk_fp64_issue_probe(5, 1, 32, 16, ctypes.byref(c), None) == g.GRBK_EINVAL
    assert L.grbk_fp64_issue_probe(0, 0, 32, 16, ctypes.byref(c), None) == g.GRBK_EINVAL
    assert L.grbk_fp64_issue_probe(0, 1, 33, 16, ctypes.byref(c), None) == g.GRBK_EINVAL
    assert L.grbk_fp64_issue_probe(0, 1, 32, 0, ctypes.byref(c), None) == g.GRBK_EINVAL
    assert L.grbk_fp64_issue_probe(0, 1, 32, 16, None, None) == g.GRBK_EINVAL
