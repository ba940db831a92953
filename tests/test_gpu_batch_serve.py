"""Batched path (ecc_compute_batch) and serving loop (ecc_submit) against the
oracle: every image's ECC must be identical alone, in a batch, and in the
served mix (tolerance 0)."""
import threading

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def ecc_mod():
    import paper_2203_09087_gb300 as ecc
    return ecc


def _mixed_images(n, seed, dtype=np.uint8, max2d=300, max3d=48):
    rng = np.random.default_rng(seed)
    imgs = []
    hi = 255 if dtype == np.uint8 else 65535
    for i in range(n):
        if rng.uniform() < 0.7:
            shape = tuple(rng.integers(1, max2d + 1, size=2))
        else:
            shape = tuple(rng.integers(1, max3d + 1, size=3))
        levels = int(rng.choice([2, 5, hi + 1]))
        imgs.append(rng.integers(0, levels, size=shape).astype(dtype))
    return imgs


@pytest.mark.parametrize("flags", [0, 0x40])
@pytest.mark.parametrize("mode", [0, 1])
def test_batch_uneven_u8(flags, mode):
    ecc = ecc_mod()
    imgs = _mixed_images(150, seed=1 + mode)
    plan = ecc.ecc_plan("u8", 0, 255, complex_mode=mode, max_images=len(imgs),
                        max_voxels=sum(i.size for i in imgs), flags=flags)
    got = ecc.ecc_compute_batch(plan, [torch.from_numpy(i).cuda() for i in imgs])
    ecc.ecc_status_get(plan)
    got = got.cpu().numpy()
    om = oracle.VERTEX if mode == 0 else oracle.TOPCELL
    for k, img in enumerate(imgs):
        assert np.array_equal(got[k], oracle.ecc(img, 0, 255, om)), (k, img.shape)


def test_batch_u16_and_subrange():
    ecc = ecc_mod()
    rng = np.random.default_rng(5)
    imgs = [rng.integers(1000, 1400, size=tuple(rng.integers(1, 60, size=int(rng.integers(2, 4)))),
                         dtype=np.uint16) for _ in range(40)]
    plan = ecc.ecc_plan("u16", 990, 1410, max_images=64, max_voxels=1 << 24)
    got = ecc.ecc_compute_batch(plan, [torch.from_numpy(i).cuda() for i in imgs]).cpu().numpy()
    ecc.ecc_status_get(plan)
    for k, img in enumerate(imgs):
        assert np.array_equal(got[k], oracle.ecc(img, 990, 1410))


def test_batch_repeated_and_resized():
    """The same plan serves batches of different sizes back to back."""
    ecc = ecc_mod()
    plan = ecc.ecc_plan("u8", 0, 255, max_images=80, max_voxels=1 << 24)
    for seed, n in [(11, 80), (12, 3), (13, 80), (14, 1)]:
        imgs = _mixed_images(n, seed)
        got = ecc.ecc_compute_batch(plan, [torch.from_numpy(i).cuda() for i in imgs]).cpu().numpy()
        for k, img in enumerate(imgs):
            assert np.array_equal(got[k], oracle.ecc(img, 0, 255))


def _oracle_many(arrays, his, mode=oracle.VERTEX):
    """The single-threaded oracle on every host array, several arrays at a
    time on the host's cores (the C library releases the GIL); arrays above
    32 M voxels run slab-parallel on all cores instead."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 4
    out = [None] * len(arrays)
    small = [k for k, a in enumerate(arrays) if a.size <= 32 << 20]
    with ThreadPoolExecutor(max_workers=cores) as ex:
        for k, r in zip(small, ex.map(lambda k: oracle.ecc(arrays[k], 0, his[k], mode), small)):
            out[k] = r
    for k, a in enumerate(arrays):
        if out[k] is None:
            out[k] = oracle.ecc_from_vcec(oracle.vcec_parallel(a, 0, his[k], mode, threads=cores))
    return out


def test_uneven_batch_4352_images_every_row():
    """The uneven 4096 + 256 batch at full size: every row equals the
    oracle, and the one-launch-per-image path gives the same rows."""
    import synth
    ecc = ecc_mod()
    specs = synth.batch_specs()
    imgs = synth.batch_images(specs, device="cuda")
    total = sum(i.numel() for i in imgs)
    plan_b = ecc.ecc_plan("u8", 0, 255, max_images=len(imgs), max_voxels=total)
    plan_p = ecc.ecc_plan("u8", 0, 255, max_images=len(imgs), max_voxels=total, flags=ecc.ECC_FLAG_BATCH_PER_IMAGE)
    got_b = ecc.ecc_compute_batch(plan_b, imgs).cpu().numpy()
    got_p = ecc.ecc_compute_batch(plan_p, imgs).cpu().numpy()
    ecc.ecc_status_get(plan_b)
    ecc.ecc_status_get(plan_p)
    assert np.array_equal(got_b, got_p)
    want = _oracle_many([t.cpu().numpy() for t in imgs], [255] * len(imgs))
    bad = [k for k in range(len(imgs)) if not np.array_equal(got_b[k], want[k])]
    assert not bad, (len(bad), bad[:5])


def test_serving_poisson_sample_against_oracle():
    """A seeded sample of 100 requests drawn from the serving workload (the
    60 s Poisson list, 2D uint8 128^2-4096^2 and 3D uint8/uint16 64^3-768^3,
    crops of the resident seeded fields) served together under the 120 GB
    budget: every result equals the oracle."""
    import synth
    ecc = ecc_mod()
    reqs = synth.poisson_requests(2000.0, 60.0)
    views = synth.serving_crops(reqs, synth.serving_bases(device="cuda"))
    rng = np.random.default_rng(5)
    pick = sorted(rng.choice(len(views), size=100, replace=False).tolist())
    # the largest shapes of the distribution are in the sample too
    big2 = max((k for k in range(len(reqs)) if len(reqs[k]["shape"]) == 2), key=lambda k: reqs[k]["shape"][0])
    big3 = max((k for k in range(len(reqs)) if len(reqs[k]["shape"]) == 3), key=lambda k: reqs[k]["shape"][0])
    pick = sorted(set(pick) | {big2, big3})
    sample = [views[k] for k in pick]
    assert {str(v.dtype) for v, _ in sample} == {"torch.uint8", "torch.uint16"}
    srv = ecc.ecc_server_create(120 << 30, n_streams=4, max_batch=64)
    outs = [np.zeros(hi + 1, np.int64) for _, hi in sample]
    tickets = [ecc.ecc_submit(srv, v, 0, hi, out=outs[i]) for i, (v, hi) in enumerate(sample)]
    for t in tickets:
        assert ecc.ecc_wait(srv, t, 600_000_000) == ecc.ECC_OK
    ecc.ecc_server_destroy(srv)
    want = _oracle_many([v.contiguous().cpu().numpy() for v, _ in sample], [hi for _, hi in sample])
    bad = [pick[i] for i in range(len(sample)) if not np.array_equal(outs[i], want[i])]
    assert not bad, bad[:5]


# ------------------------------------------------------------------ serving

def _server(ecc, budget=1 << 30, streams=4, max_batch=16):
    return ecc.ecc_server_create(budget, n_streams=streams, max_batch=max_batch)


def test_served_results_equal_alone_and_oracle():
    ecc = ecc_mod()
    rng = np.random.default_rng(21)
    jobs = []
    for i in range(120):
        dt = np.uint8 if rng.uniform() < 0.7 else np.uint16
        hi = 255 if dt == np.uint8 else 65535
        shape = tuple(rng.integers(1, 200, size=2)) if rng.uniform() < 0.6 else tuple(rng.integers(1, 40, size=3))
        img = rng.integers(0, hi + 1, size=shape).astype(dt)
        mode = int(rng.integers(0, 2))
        jobs.append((img, hi, mode))
    srv = _server(ecc)
    outs = [np.zeros(hi + 1, np.int64) for _, hi, _ in jobs]
    dev = [torch.from_numpy(img).cuda() if k % 2 else None for k, (img, _, _) in enumerate(jobs)]
    tickets = [None] * len(jobs)

    def submit(lo_k, hi_k):
        for k in range(lo_k, hi_k):
            img, hi, mode = jobs[k]
            src = dev[k] if dev[k] is not None else img
            tickets[k] = ecc.ecc_submit(srv, src, 0, hi, mode, out=outs[k])

    ts = [threading.Thread(target=submit, args=(a, a + 30)) for a in range(0, 120, 30)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for k in range(len(jobs)):
        assert ecc.ecc_wait(srv, tickets[k], 60_000_000) == ecc.ECC_OK
    stats = ecc.ecc_server_stats(srv)
    assert stats["jobs"] == len(jobs) and stats["p99_us"] >= stats["p50_us"] > 0
    ecc.ecc_server_destroy(srv)
    for k, (img, hi, mode) in enumerate(jobs):
        om = oracle.VERTEX if mode == 0 else oracle.TOPCELL
        assert np.array_equal(outs[k], oracle.ecc(img, 0, hi, om)), k
    # the same job alone gives the same bits
    srv1 = _server(ecc, streams=1, max_batch=1)
    img, hi, mode = jobs[7]
    alone = np.zeros(hi + 1, np.int64)
    t = ecc.ecc_submit(srv1, img, 0, hi, mode, out=alone)
    assert ecc.ecc_wait(srv1, t) == ecc.ECC_OK
    ecc.ecc_server_destroy(srv1)
    assert np.array_equal(alone, outs[7])


def test_budget_admission_and_errors():
    ecc = ecc_mod()
    img = np.random.default_rng(1).integers(0, 256, size=(64, 64, 64), dtype=np.uint8)  # 256 KiB per job
    srv = _server(ecc, budget=600_000, streams=2, max_batch=4)   # room for two jobs at a time
    outs = [np.zeros(256, np.int64) for _ in range(10)]
    tickets = [ecc.ecc_submit(srv, img, 0, 255, out=o) for o in outs]
    for t in tickets:
        assert ecc.ecc_wait(srv, t, 60_000_000) == ecc.ECC_OK
    want = oracle.ecc(img, 0, 255)
    for o in outs:
        assert np.array_equal(o, want)
    assert ecc.ecc_server_stats(srv)["peak_bytes"] <= 600_000
    big = np.zeros((100, 100, 100), np.uint8)   # 1 MB alone exceeds the budget
    with pytest.raises(ecc.EccError) as ei:
        ecc.ecc_submit(srv, big, 0, 255)
    assert ei.value.status == ecc.ECC_E_NOMEM
    with pytest.raises(ecc.EccError):
        ecc.ecc_submit(srv, img, 10, 5)
    ecc.ecc_server_destroy(srv)


def test_destroy_with_cancel_drains_or_cancels():
    ecc = ecc_mod()
    img = np.random.default_rng(2).integers(0, 256, size=(128, 256, 256), dtype=np.uint8)
    srv = _server(ecc, budget=20_000_000, streams=1, max_batch=1)
    tickets = [ecc.ecc_submit(srv, img, 0, 255) for _ in range(20)]
    srv.close(cancel=True)
    # nothing hangs; the handle is gone
    assert not srv.handle.value


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_degenerate_and_boundary_shapes(mode):
    """Shapes at the edges of the 2D lane packing (one window of 30 columns,
    one row, row counts around the row-chunk length) and of the 3D tiles."""
    ecc = ecc_mod()
    rng = np.random.default_rng(17 + mode)
    shapes = [(1, 1), (1, 70), (70, 1), (3, 31), (31, 3), (29, 30), (30, 31), (33, 61), (64, 64),
              (5, 960), (2, 961), (15, 17), (16, 900), (31, 29), (32, 33), (63, 30), (65, 91), (97, 2),
              (1, 1, 1), (1, 31, 1), (2, 2, 33), (31, 33, 1), (17, 30, 31), (9, 61, 29)]
    imgs = [rng.integers(0, int(rng.choice([2, 7, 256])), size=s).astype(np.uint8) for s in shapes]
    plan = ecc.ecc_plan("u8", 0, 255, complex_mode=mode, max_images=len(imgs),
                        max_voxels=sum(i.size for i in imgs))
    got = ecc.ecc_compute_batch(plan, [torch.from_numpy(i).cuda() for i in imgs])
    ecc.ecc_status_get(plan)
    got = got.cpu().numpy()
    om = oracle.VERTEX if mode == 0 else oracle.TOPCELL
    for k, img in enumerate(imgs):
        assert np.array_equal(got[k], oracle.ecc(img, 0, 255, om)), (k, img.shape)


def test_prepared_keys_serve_exactly():
    """ecc_server_prepare makes every slot's plan for a key ahead of its
    jobs; prepared and unprepared keys then serve alike, exactly."""
    ecc = ecc_mod()
    srv = ecc.ecc_server_create(1 << 30, n_streams=3, max_batch=8)
    try:
        ecc.ecc_server_prepare(srv, "u8", 0, 255)
        ecc.ecc_server_prepare(srv, "u16", 1000, 1410, ecc.ECC_TOPCELL_MIN)
        with pytest.raises(ecc.EccError) as ei:
            ecc.ecc_server_prepare(srv, "u8", 10, 300)
        assert ei.value.status == ecc.ECC_E_INVALID
        rng = np.random.default_rng(77)
        jobs = []
        for i in range(24):
            if i % 3 == 2:
                img = rng.integers(1000, 1411, size=(9, 20, 31)).astype(np.uint16)
                lo, hi, mode = 1000, 1410, ecc.ECC_TOPCELL_MIN
            else:
                img = rng.integers(0, 256, size=(int(rng.integers(5, 90)), int(rng.integers(5, 90))), dtype=np.uint8)
                lo, hi, mode = 0, 255, ecc.ECC_VERTEX_MAX
            out = np.zeros(hi - lo + 1, np.int64)
            t = ecc.ecc_submit(srv, torch.from_numpy(img).cuda(), lo, hi, mode, out=out)
            jobs.append((t, img, lo, hi, mode, out))
        for t, img, lo, hi, mode, out in jobs:
            assert ecc.ecc_wait(srv, t, 60_000_000) == ecc.ECC_OK
            om = oracle.VERTEX if mode == ecc.ECC_VERTEX_MAX else oracle.TOPCELL
            assert np.array_equal(out, oracle.ecc(img, lo, hi, om))
    finally:
        ecc.ecc_server_destroy(srv)
