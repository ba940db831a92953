"""A new plan is ready for any stream the moment ecc_plan returns.

The plan's workspace holds the histogram accumulator, the status word, the
3D kernel's work counter and the scan's look-back state, all of which must
start at zero.  A clear issued on the legacy default stream is not ordered
before work on a non-blocking stream (the serving loop's streams, torch side
streams), so a computation launched there right after ecc_plan could read
stale memory and have its histogram cleared under it.  Here the legacy
stream is held busy by a bounded spin kernel while a plan is created over
freed memory filled with ones, and the first computations run at once on a
non-blocking stream; their results must be exact.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _dirty_free_memory(nbytes):
    junk = torch.full((nbytes,), 0xFF, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    del junk
    torch.cuda.empty_cache()


@pytest.mark.parametrize("kind", ["2d", "3d", "batch"])
def test_first_use_on_a_non_blocking_stream(kind):
    import paper_2203_09087_gb300 as ecc
    rng = np.random.default_rng(91)
    imgs = [rng.integers(0, 256, size=(300, 301)).astype(np.uint8),
            rng.integers(0, 256, size=(40, 64, 96)).astype(np.uint8)]
    want = [oracle.ecc(a, 0, 255, "vertex") for a in imgs]
    dev = [torch.from_numpy(a).cuda() for a in imgs]
    side = torch.cuda.Stream()
    for _ in range(3):
        _dirty_free_memory(256 << 20)
        torch.cuda._sleep(400_000_000)          # ~0.2 s on the legacy default stream
        plan = ecc.ecc_plan("u8", 0, 255, max_voxels=1 << 24, max_images=4)
        with torch.cuda.stream(side):
            if kind == "batch":
                got = ecc.ecc_compute_batch(plan, dev)
            else:
                got = ecc.ecc_compute(plan, dev[0] if kind == "2d" else dev[1])
        side.synchronize()
        got = got.cpu().numpy()
        torch.cuda.synchronize()
        if kind == "batch":
            for i in range(2):
                assert np.array_equal(got[i], want[i])
        else:
            assert np.array_equal(got, want[0] if kind == "2d" else want[1])
        ecc.ecc_status_get(plan)
        plan.close()
