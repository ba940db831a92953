"""Failure detection on the GPU without a fault: every device-side wait of the
library (the scan's look-back spin on a flag, the TMA ring's mbarrier waits)
is bounded and reports ECC_E_TIMEOUT instead of hanging.  The self-test makes
both kinds of wait run out (a flag nothing sets, an mbarrier nothing arrives
on) and the test checks that the status comes back and that the context still
computes correct results afterwards."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_bounded_waits_report_timeout_and_context_survives():
    import paper_2203_09087_gb300 as E

    st, gave = E.ecc_selftest_wait_timeout(20_000)
    assert st == E.ECC_E_TIMEOUT
    assert gave == [1, 1]
    assert "gave up" in E.ecc_last_error()

    rng = np.random.default_rng(12)
    img = rng.integers(0, 256, size=(40, 48, 72), dtype=np.uint8)
    plan = E.ecc_plan("u8", 0, 255, max_voxels=img.size)
    out = torch.zeros(256, dtype=torch.int64, device="cuda")
    E.ecc_compute(plan, torch.from_numpy(img).cuda(), out)
    E.ecc_status_get(plan)
    assert np.array_equal(out.cpu().numpy(), oracle.ecc(img, 0, 255))


def test_selftest_rejects_bad_limit():
    import paper_2203_09087_gb300 as E

    with pytest.raises(E.EccError):
        E.ecc_selftest_wait_timeout(0)
