"""Benchmark: exact ECC of a 512^3 uint8 Gaussian-smoothed volume on GB300.

One step = the whole per-image hot path through the C ABI (``ecc_compute``):
one launch of the stencil + histogram kernel, whose last CTA also scans the
256 bins.  The input is resident in HBM; L2 is flushed (a 2x-L2 write)
before every timed step and each step is timed with CUDA events on the
launching stream.

Also reported on the same JSON line:
  roofline      the stencil kernel's algorithmic bytes per launch
                (voxels x bytes/voxel + nbins x 8) over its event-timed
                duration (the steps' own events when a step is that one
                launch), against the measured HBM copy bandwidth;
  e2e           the same metric through ``ecc_compute_host`` from pinned host
                memory (chunked H2D overlapped with the kernels, ECC copied
                back), copies inside the timed region;
  cpu_baseline  the CPU oracle (as it stands) on a bounded slab of the same
                volume, on all host cores;
  latency_256x256, single_u16, batched, serving
                the other configurations (256^2 uint8 latency, 1024^3 uint16,
                the uneven 4352-image batch against one launch per image,
                Poisson serving with p50/p99 and a saturating replay), each with its own
                timing; --main-only leaves them out, --extras adds the
                NEXT-row workloads (float thresholds, smoothing pipeline,
                top-cell and 4D, one-core CPU baselines).

``--impl reference`` times the CPU oracle on the same workload (bounded slab
samples per step) and prints the same line with "impl": "reference".

Multi-GPU (torchrun, N ranks): replicas only -- every rank runs the same
independent workload on its own GPU; no data-path collective; value is the
voxels of all ranks over the max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "ECC Gvoxel/s"
UNIT = "Gvoxel/s"
WORKLOAD = "plain 3D ECC, 512x512x512 uint8 Gaussian-smoothed (sigma=4) field, seed 1, 256 bins, vertex complex"


def _peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _counters_for(kernel_digest: str):
    """The 512^3 stencil launch's committed ncu counters, if the kernel is unchanged."""
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return {}
    d = json.loads(p.read_text())
    ent = d.get("stencil_512cube_u8")
    if not ent or ent.get("kernel_digest") != kernel_digest:
        return {}
    return ent


def _traffic_for(kernel_digest: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    return _counters_for(kernel_digest).get("dram_bytes_per_launch")


# integer (ALU) pipe issue rate of a GB300 SM: 4 sub-partitions, each issuing
# one ALU warp instruction every other cycle (16 lanes a sub-partition)
ALU_WARP_INSTR_PER_SM_CYCLE = 2


def alu_roofline(kernel_digest: str, kernel_s: float, sms: int, sm_mhz):
    """The stencil's second roofline: ALU-pipe warp instructions per launch
    (committed ncu count, null once the kernel changed) over the launch's
    measured duration, against SMs x 2 per cycle x the SM clock sampled under
    load."""
    ent = _counters_for(kernel_digest)
    n = ent.get("alu_warp_instr_per_launch")
    peak = sms * ALU_WARP_INSTR_PER_SM_CYCLE * sm_mhz * 1e6 / 1e12 if sm_mhz else None
    achieved = n / kernel_s / 1e12 if n else None
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T warp-instr/s",
            "frac": achieved / peak if achieved and peak else None,
            "alu_warp_instr_per_launch": n, "warp_instr_per_launch": ent.get("warp_instr_per_launch"),
            "peak_source": f"{sms} SMs x {ALU_WARP_INSTR_PER_SM_CYCLE} ALU warp-instr/cycle x median SM clock "
                           f"under load ({sm_mhz} MHz)",
            "count_source": ent.get("source") if n else "no ncu count for the current kernel sources"}


STENCIL_SOURCES = ("ecc_bs3d.cu", "ecc_walk3.cuh", "ecc_bitlogic.cuh", "ecc_bitslice.cuh", "ecc_walk.cuh",
                   "ecc_sync.cuh", "ecc_internal.h", "ecc_scan_block.cuh")


def _kernel_digest():
    """Digest of the sources the 3D stencil kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for name in STENCIL_SOURCES:
        h.update((ROOT / "paper_2203_09087_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            dev = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0] or str(os.environ.get("LOCAL_RANK", 0))
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={dev}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    """One process per GPU under torchrun: (dist, rank, world_size); (None, 0, 1) alone.
    NCCL when CUDA is present, else gloo (the multi-rank host logic on CPU)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _barrier(dist, torch):
    if dist:
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def _max_over_ranks(dist, torch, x: float) -> float:
    if not dist:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gvox_s(voxels_per_step: int, steps: int, world_size: int, slowest_seconds: float) -> float:
    """Replicas: every rank processes its own copy of the workload, so the job
    processed voxels_per_step * steps * world_size voxels in the slowest rank's time."""
    return voxels_per_step * steps * world_size / slowest_seconds / 1e9


def cpu_oracle_sample(vol_host, budget_s: float = 12.0, threads: int | None = None):
    """Time the oracle (all host cores) on a slab of planes sized for ~budget_s of CPU time."""
    import numpy as np

    import oracle
    threads = threads or os.cpu_count() or 1
    # calibrate on one plane with one thread
    t0 = time.perf_counter()
    oracle.vcec_rows(vol_host, 0, 1, 0, 255, oracle.VERTEX)
    per_plane = max(time.perf_counter() - t0, 1e-4)
    planes = int(max(threads, min(vol_host.shape[0], budget_s / per_plane)))
    planes = min(planes, vol_host.shape[0])
    t0 = time.perf_counter()
    oracle.vcec_parallel(vol_host, 0, 255, oracle.VERTEX, threads=threads, rows=(0, planes))
    dt = time.perf_counter() - t0
    vox = planes * vol_host.shape[1] * vol_host.shape[2]
    return {"value": vox / dt / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"cells based on planes 0..{planes - 1} of the same volume ({vox} voxels), "
                      f"slab-parallel over {threads} threads, {dt:.2f} s wall"}


def run_reference(args):
    """The CPU oracle as the reference arm (rank 0 only)."""
    import torch
    dist, rank, ws = None, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    import synth
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    vol = synth.smooth_3d_512(device=dev).cpu().numpy()
    import oracle
    threads = os.cpu_count() or 1
    # each step: the oracle on a bounded slab (about 10 s of CPU work)
    t0 = time.perf_counter()
    oracle.vcec_rows(vol, 0, 1, 0, 255, oracle.VERTEX)
    per_plane = max(time.perf_counter() - t0, 1e-4)
    planes = int(max(threads, min(vol.shape[0], 10.0 / per_plane)))
    rows = (0, min(planes, vol.shape[0]))
    for _ in range(args.warmup):
        oracle.vcec_parallel(vol[: rows[1] + 1], 0, 255, oracle.VERTEX, threads=threads, rows=rows)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.vcec_parallel(vol[: rows[1] + 1], 0, 255, oracle.VERTEX, threads=threads, rows=rows)
    dt = time.perf_counter() - t0
    vox = (rows[1] - rows[0]) * vol.shape[1] * vol.shape[2]
    value = vox * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_planes": rows[1] - rows[0]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"cells based on planes {rows[0]}..{rows[1] - 1} per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_batched(args):
    """Uneven batch (4096 2D + 256 3D uint8 smoothed fields): one graph launch
    of the persistent batch kernel vs one stencil launch per image."""
    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    specs = synth.batch_specs()
    imgs = synth.batch_images(specs, device="cuda")
    total = sum(int(i.numel()) for i in imgs)
    out = torch.empty((len(imgs), 256), dtype=torch.int64, device="cuda")
    res = {"workload": "4096 2D (H,W ~ U{64..1024}) + 256 3D (sides ~ U{32..256}) uint8, sigma ~ U[1,6], seed 3",
           "voxels": total}
    ref = None
    # the descriptor array is built once (host marshalling, timed separately)
    t0 = time.perf_counter()
    descs = ecc.image_descs(imgs)
    res["descriptor_build_ms"] = (time.perf_counter() - t0) * 1e3
    modes = (("batched", 0), ("per_image", ecc.ECC_FLAG_BATCH_PER_IMAGE))
    plans = {}
    for name, flags in modes:
        plan = ecc.ecc_plan("u8", 0, 255, max_images=len(imgs), max_voxels=total, flags=flags)
        for _ in range(3):
            ecc.ecc_compute_batch(plan, descs, out)
        ecc.ecc_status_get(plan)
        got = out.cpu().numpy()
        if ref is None:
            ref = got
        assert np.array_equal(ref, got)
        plans[name] = plan
    # trials alternate the two modes; each trial is the mean of `reps` calls,
    # and the figures reported are the medians over the trials
    trials, reps = 5, 5
    ms = {name: [] for name, _ in modes}
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(trials):
        for name, _ in modes:
            torch.cuda.synchronize()
            s.record()
            for _ in range(reps):
                ecc.ecc_compute_batch(plans[name], descs, out)
            e.record()
            torch.cuda.synchronize()
            ms[name].append(s.elapsed_time(e) / reps)
    for name, _ in modes:
        med = statistics.median(ms[name])
        res[name] = {"ms": med, "gvox_s": total / med / 1e6, "launches": ecc.ecc_plan_last_launches(plans[name]),
                     "trial_ms": ms[name]}
    ratios = [p / b for p, b in zip(ms["per_image"], ms["batched"])]
    res["speedup"] = statistics.median(ratios)
    res["speedup_trials"] = ratios
    res["timing"] = f"{trials} alternating trials of {reps} calls each; medians over trials"
    return res


def time_c1(reps: int):
    """The 256^2 uint8 image: one checked call, then `reps` calls each queued
    behind a spin kernel and timed with CUDA events (the device work alone)."""
    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    t = torch.from_numpy(synth.uniform_2d_256()).cuda()
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=t.numel())
    out = ecc.ecc_compute(plan, t)
    ecc.ecc_status_get(plan)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(200_000)
        a.record()
        ecc.ecc_compute(plan, t, out)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e3)
    return {"workload": "256x256 uint8 uniform [0,255], seed 0, 256 bins", "device_us_p50": float(np.median(ts))}


def time_present(reps: int):
    """ecc_levels_present on the 512^3 float32 field (sigma 4, seed 1) rounded
    to its 1024 quantile levels: one call checked against torch.unique, then
    `reps` calls (CUDA events, mean)."""
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    f = synth.smooth(torch.randn((512, 512, 512), generator=g, device="cuda"), 4.0).contiguous()
    levels = torch.quantile(f.flatten()[::97].float(), torch.linspace(0, 1, 1024, device="cuda")).float()
    fq = levels[torch.bucketize(f, levels).clamp_(max=1023)].contiguous()
    del f
    plan = ecc.ecc_plan("u16", 0, 65535, max_voxels=fq.numel())
    lv, cnt = ecc.ecc_levels_present(plan, fq, max_levels=4096)
    want = torch.unique(fq)
    n = int(cnt.item())
    assert n == want.numel() and torch.equal(lv[:n], want)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ecc.ecc_levels_present(plan, fq, max_levels=4096, levels_out=lv, count_out=cnt)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    return {"workload": "512^3 float32 field rounded to 1024 quantile levels", "distinct_values": n, "ms": ms,
            "gvox_s": fq.numel() / ms / 1e6}


def time_pipe(side: int, rounds: int):
    """The smoothing pipeline on a side^2 float32 field (sigma 3, seed 5) at
    255 levels (the fused round): four warm-up rounds, then `rounds` timed
    rounds in one call (CUDA events)."""
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    base = synth.smooth(torch.randn((side, side), generator=g, device="cuda"), 3.0).contiguous()
    levels = torch.linspace(float(base.min()), float(base.max()), 255, device="cuda").float().contiguous()
    plan = ecc.ecc_plan("u16", 0, 255, max_voxels=base.numel())
    taps = ecc.gaussian_taps(2.0)
    img = base.clone()
    ecc.ecc_pipeline_gaussian(plan, img, taps, 4, levels)
    ecc.ecc_status_get(plan)
    img.copy_(base)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    res = ecc.ecc_pipeline_gaussian(plan, img, taps, rounds, levels)
    b.record()
    torch.cuda.synchronize()
    ecc.ecc_status_get(plan)
    assert int(res[0, -1].item()) == 1
    return {"workload": f"{side}^2 float32 field, 13 taps, 255 levels", "us_per_round": a.elapsed_time(b) * 1e3 / rounds}


def time_c4_part(part: str, reps: int):
    """The uneven batch (or only its 2D or 3D images) through one batched call:
    one untimed call, then `reps` timed calls (CUDA events on the stream,
    mean), then the per-image path on the same images, whose results must
    equal the batched ones (last, so the batched launches come first)."""
    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    imgs = synth.batch_images(synth.batch_specs(), device="cuda")
    if part != "all":
        imgs = [i for i in imgs if i.dim() == (2 if part == "2d" else 3)]
    total = sum(int(i.numel()) for i in imgs)
    descs = ecc.image_descs(imgs)
    out = torch.empty((len(imgs), 256), dtype=torch.int64, device="cuda")
    ref = torch.empty_like(out)
    plan = ecc.ecc_plan("u8", 0, 255, max_images=len(imgs), max_voxels=total)
    pplan = ecc.ecc_plan("u8", 0, 255, max_images=len(imgs), max_voxels=total, flags=ecc.ECC_FLAG_BATCH_PER_IMAGE)
    ecc.ecc_compute_batch(plan, descs, out)
    ecc.ecc_status_get(plan)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        ecc.ecc_compute_batch(plan, descs, out)
    e.record()
    torch.cuda.synchronize()
    ms = s.elapsed_time(e) / reps
    ecc.ecc_status_get(plan)
    ecc.ecc_compute_batch(pplan, descs, ref)
    ecc.ecc_status_get(pplan)
    assert torch.equal(out, ref)
    return {"workload": f"uneven batch ({part}): {len(imgs)} images", "voxels": total, "ms": ms,
            "gvox_s": total / ms / 1e6}


def run_single_u16(args):
    """The 16-bit single-volume workload: 1024^3 uint16 smoothed field (sigma
    8) plus 2000 bright blobs, 65536 bins (global int64 bins: the histogram
    does not fit in shared memory).  Stencil kernel time from CUDA events on
    the launching stream, L2 flushed before every step; roofline bytes =
    2 bytes per voxel + 65536 x 8."""
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    vol = synth.smooth_blobs_u16_1024(device="cuda")
    nvox = vol.numel()
    plan = ecc.ecc_plan("u16", 0, 65535, max_voxels=nvox, flags=ecc.ECC_FLAG_TIME_KERNELS)
    out = torch.empty(65536, dtype=torch.int64, device="cuda")
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    flush = torch.empty(2 * l2 + (1 << 20), dtype=torch.uint8, device="cuda")
    ecc.ecc_compute(plan, vol, out)
    ecc.ecc_status_get(plan)
    assert int(out[-1].item()) == 1
    for _ in range(3):
        flush.fill_(1)
        ecc.ecc_compute(plan, vol, out)
    ecc.ecc_plan_kernel_time(plan)
    steps = 10
    st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        st[i].record()
        ecc.ecc_compute(plan, vol, out)
        en[i].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(st, en)) / steps
    kern_ms, kern_n = ecc.ecc_plan_kernel_time(plan)
    kern_s = kern_ms / max(kern_n, 1) * 1e-3
    peak, src = _peaks()
    alg = nvox * 2 + 65536 * 8
    res = {"workload": "1024^3 uint16, sigma 8 smoothed field + 2000 blobs (seed 2), 65536 bins",
           "gvox_s": nvox / (ms * 1e-3) / 1e9, "ms_per_step": ms, "kernel_us": kern_s * 1e6,
           "roofline": {"bound": "hbm", "achieved": alg / kern_s / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": alg / kern_s / 1e9 / peak, "peak_source": src}}

    # out of core: the same 2 GB volume from pinned host memory through 256 MiB
    # of device chunk buffers (ecc_compute_stream), against the resident result
    import numpy as np
    want = out.cpu().numpy()
    host = vol.cpu().pin_memory().numpy()
    del vol
    torch.cuda.empty_cache()
    budget = 256 << 20
    got = ecc.ecc_compute_stream(plan, host, budget)
    assert np.array_equal(got, want)
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        ecc.ecc_compute_stream(plan, host, budget, out=got)
    sec = (time.perf_counter() - t0) / reps
    ecc.ecc_plan_kernel_time(plan)
    res["out_of_core"] = {"path": "ecc_compute_stream, pinned host volume, 256 MiB of device chunk buffers",
                          "device_budget_bytes": budget, "gvox_s": nvox / sec / 1e9, "ms": sec * 1e3,
                          "h2d_bytes": nvox * 2, "identical_to_resident": True}
    return res


def time_c3(reps=3):
    """The 1024^3 uint16 volume alone: one checked call, then `reps` calls
    timed with CUDA events (for profiler captures of the 16-bit kernel)."""
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    vol = synth.smooth_blobs_u16_1024(device="cuda")
    plan = ecc.ecc_plan("u16", 0, 65535, max_voxels=vol.numel())
    out = torch.empty(65536, dtype=torch.int64, device="cuda")
    ecc.ecc_compute(plan, vol, out)
    ecc.ecc_status_get(plan)
    assert int(out[-1].item()) == 1
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ecc.ecc_compute(plan, vol, out)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": "1024^3 uint16 smoothed field + 2000 blobs, 65536 bins", "ms_per_call": ms,
            "gvox_s": vol.numel() / ms / 1e6}


def run_float_levels(args):
    """Float32 input at given thresholds (the paper's Gaussian random fields
    are float32 with 1024 values): a 512^3 float32 field smoothed with sigma
    4 (seed 1, before any quantization), 1024 thresholds at the field's
    quantiles, through ecc_compute_levels (quantize to uint16 level indices,
    stencil, scan).  Whole-call time from CUDA events, L2 flushed before
    every step; HBM bytes = 4 read + 2 written + 2 read per voxel."""
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    g = torch.Generator(device="cuda")
    g.manual_seed(1)
    f = synth.smooth(torch.randn((512, 512, 512), generator=g, device="cuda"), 4.0).contiguous()
    m = 1024
    sample = f.flatten()[:: 97].float()
    levels = torch.quantile(sample, torch.linspace(0, 1, m, device="cuda")).float().contiguous()
    levels[-1] = f.max()
    nvox = f.numel()
    plan = ecc.ecc_plan("u16", 0, m, max_voxels=nvox, flags=ecc.ECC_FLAG_TIME_KERNELS)
    out = ecc.ecc_compute_levels(plan, f, levels)
    ecc.ecc_status_get(plan)
    assert int(out[-1].item()) == 1    # the last threshold is the max: the full box
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    flush = torch.empty(2 * l2 + (1 << 20), dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ecc.ecc_compute_levels(plan, f, levels, out=out)
    torch.cuda.synchronize()
    ecc.ecc_plan_kernel_time(plan)
    steps = 10
    st = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    en = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(i & 0xFF)
        st[i].record()
        ecc.ecc_compute_levels(plan, f, levels, out=out)
        en[i].record()
    torch.cuda.synchronize()
    ecc.ecc_status_get(plan)
    ms = sorted(a.elapsed_time(b) for a, b in zip(st, en))[steps // 2]
    kern_ms, kern_n = ecc.ecc_plan_kernel_time(plan)
    peak, src = _peaks()
    alg = nvox * (4 + 2 + 2)
    return {"workload": "512^3 float32 Gaussian-smoothed (sigma=4) field, seed 1, 1024 quantile thresholds",
            "gvox_s": nvox / (ms * 1e-3) / 1e9, "ms_per_step": ms,
            "stencil_us": kern_ms / max(kern_n, 1) * 1e3,
            "hbm": {"bytes_per_step": alg, "achieved_gbs": alg / (ms * 1e-3) / 1e9, "peak": peak,
                    "frac": alg / (ms * 1e-3) / 1e9 / peak, "peak_source": src},
            "present_levels": run_present_levels(f, levels, flush)}


def run_present_levels(f, levels, flush):
    """The paper's own thresholds (Eq. 1: the values present): the same field
    rounded to its 1024 quantile levels, so it holds 1024 distinct float32
    values as the paper's Gaussian random fields do (those levels that some
    voxel takes).  Times ecc_levels_present (three launches) and
    ecc_compute_present (levels, one host read of their number, then the ECC
    at them), CUDA events, L2 flushed before each call; the levels found must
    be the field's distinct values (torch.unique as the check)."""
    import torch

    import paper_2203_09087_gb300 as ecc
    idx = torch.bucketize(f, levels).clamp_(max=levels.numel() - 1)
    fq = levels[idx].contiguous()
    del idx
    nvox = fq.numel()
    plan = ecc.ecc_plan("u16", 0, 65535, max_voxels=nvox)
    lv, cnt = ecc.ecc_levels_present(plan, fq, max_levels=4096)
    n = int(cnt.item())
    want = torch.unique(fq)
    assert n == int(want.numel()) and torch.equal(lv[:n], want)
    times = {"levels_present": [], "compute_present": []}
    for i in range(8):
        for name in times:
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            if name == "levels_present":
                ecc.ecc_levels_present(plan, fq, max_levels=4096, levels_out=lv, count_out=cnt)
            else:
                ecc.ecc_compute_present(plan, fq, max_levels=4096)
            b.record()
            torch.cuda.synchronize()
            times[name].append(a.elapsed_time(b))
    ecc.ecc_status_get(plan)
    med = {k: sorted(v)[len(v) // 2] for k, v in times.items()}
    return {"workload": "the 512^3 field rounded to its 1024 quantile levels (1024 distinct float32 values)",
            "distinct_values": n, "levels_present_ms": med["levels_present"],
            "compute_present_ms": med["compute_present"],
            "levels_present_gvox_s": nvox / (med["levels_present"] * 1e-3) / 1e9,
            "compute_present_gvox_s": nvox / (med["compute_present"] * 1e-3) / 1e9}


def run_gaussian_pipeline(args):
    """The paper's GPU-only pipeline (Table 2): a float32 Gaussian random
    field resident on the device, (ECC at the levels, then 13-tap separable
    Gaussian smoothing) repeated n times through ecc_pipeline_gaussian.
    1024^2 (the paper's size) at 255 levels -- one fused kernel per round --
    for n = 1, 10, 100, 1000, and per-round times at 1024^2 and 8192^2 (a
    size that fills the GPU) for 255 levels (fused) and 256 levels (the
    round as level search, stencil and one filter kernel per axis).
    Whole-call time from CUDA events."""
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    taps = ecc.gaussian_taps(2.0)

    def field(side):
        g = torch.Generator(device="cuda")
        g.manual_seed(5)
        return synth.smooth(torch.randn((side, side), generator=g, device="cuda"), 3.0).contiguous()

    def rounds(base, m, n, out=None):
        levels = torch.linspace(float(base.min()), float(base.max()), m, device="cuda").float().contiguous()
        plan = ecc.ecc_plan("u16", 0, m, max_voxels=base.numel())
        img = base.clone()
        ecc.ecc_pipeline_gaussian(plan, img, taps, 4, levels)   # warm-up (captured graph)
        ecc.ecc_status_get(plan)
        img.copy_(base)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        res = ecc.ecc_pipeline_gaussian(plan, img, taps, n, levels, out=out)
        b.record()
        torch.cuda.synchronize()
        ecc.ecc_status_get(plan)
        assert int(res[0, -1].item()) == 1
        return a.elapsed_time(b)

    base = field(1024)
    rows = {}
    for n in (1, 10, 100, 1000):
        ms = rounds(base, 255, n)
        rows[f"x{n}"] = {"overall_ms": ms, "per_iteration_ms": ms / n}
    per_round = {}
    for side, n in ((1024, 200), (8192, 20)):
        b = base if side == 1024 else field(side)
        for m, kind in ((255, "fused"), (256, "unfused")):
            us = rounds(b, m, n) * 1e3 / n
            px = side * side
            per_round[f"{side}^2_{kind}"] = {"levels": m, "us_per_round": us, "gpx_s": px / us / 1e3,
                                             "hbm_bytes_per_round": (8 if kind == "fused" else 24) * px,
                                             "gb_s_at_those_bytes": (8 if kind == "fused" else 24) * px / us / 1e3}
    return {"workload": "float32 Gaussian random field (sigma 3, seed 5), 13-tap Gaussian (sigma 2), "
                        "(ECC + smoothing) x n on the device; 1024^2 at 255 levels for the paper's x1..x1000",
            "rounds": rows, "per_round": per_round,
            "bytes_note": "fused: the image read and written once per round (8 B/px, halo re-reads "
                          "excluded); unfused: two filter passes (16 B/px), the level search (6 B/px) "
                          "and the stencil (2 B/px)"}


def run_latency_256sq(args):
    """The 256x256 uint8 uniform image: too small to fill the GPU, so the
    figure is the latency of one ecc_compute call (stencil and scan) measured
    with CUDA events on the stream, median of 200 calls -- on an idle stream
    (launch latency included) and queued behind a spin kernel (the device
    work alone) -- and the same for a call through ecc_compute_host (host
    image in, host ECC out, host clock)."""
    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    img = synth.uniform_2d_256()
    t = torch.from_numpy(img).cuda()
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=t.numel())
    out = ecc.ecc_compute(plan, t)
    ecc.ecc_status_get(plan)
    ts = []
    for _ in range(200):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ecc.ecc_compute(plan, t, out)
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b) * 1e3)
    # the same with the stream kept busy ahead of the call (a spin kernel),
    # so the events bracket the device work alone and not the host's launch
    # latency on an idle stream
    ks = []
    for _ in range(200):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda._sleep(200_000)
        a.record()
        ecc.ecc_compute(plan, t, out)
        b.record()
        b.synchronize()
        ks.append(a.elapsed_time(b) * 1e3)
    host = np.ascontiguousarray(img)
    hout = np.empty(256, np.int64)
    hs = []
    for _ in range(50):
        t0 = time.perf_counter()
        ecc.ecc_compute_host(plan, host, hout)
        hs.append((time.perf_counter() - t0) * 1e6)
    assert np.array_equal(hout, out.cpu().numpy())
    return {"workload": "256x256 uint8 uniform [0,255], seed 0, 256 bins", "device_call_us_p50": float(np.median(ts)),
            "device_call_us_p99": float(np.percentile(ts, 99)),
            "device_call_timing": "events on an idle stream around one call: includes the launch latency",
            "device_busy_stream_us_p50": float(np.median(ks)), "device_busy_stream_us_p99": float(np.percentile(ks, 99)),
            "device_busy_stream_timing": "events around one call queued behind a spin kernel: the device work alone",
            "host_call_us_p50": float(np.median(hs))}


def run_cpu_baselines(args):
    """The CPU oracle (as it stands, one host thread) on the other
    configurations, each a bounded sample: the 256^2 image in full, a slab of
    planes of the 1024^3 uint16 volume (65536 bins), and the first 2D images
    and first 3D patches of the uneven batch.  Reported baselines, not
    targets."""
    import numpy as np

    import oracle
    import synth
    res = {}
    img = synth.uniform_2d_256()
    t0 = time.perf_counter()
    oracle.ecc(img, 0, 255, oracle.VERTEX)
    dt = time.perf_counter() - t0
    res["uniform_256x256"] = {"value": img.size / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                      "sample": "the whole 256x256 image"}
    vol = synth.smooth_blobs_u16_1024(device="cuda").cpu().numpy()
    t0 = time.perf_counter()
    planes = 6
    oracle.vcec_rows(vol, 0, planes, 0, 65535, oracle.VERTEX)
    dt = time.perf_counter() - t0
    res["u16_1024cube_slab"] = {"value": planes * vol.shape[1] * vol.shape[2] / dt / 1e9, "unit": UNIT, "cores": 1,
                      "kind": "oracle", "sample": f"cells based on planes 0..{planes - 1} of the 1024^3 uint16 volume"}
    del vol
    specs = synth.batch_specs()
    pick = [i for i, (shape, _) in enumerate(specs) if len(shape) == 2][:16] + \
           [i for i, (shape, _) in enumerate(specs) if len(shape) == 3][:2]
    imgs = [synth.smoothed_field(specs[i][0], specs[i][1], np.uint8, seed=3 * 100003 + i, device="cuda").cpu().numpy()
            for i in pick]
    t0 = time.perf_counter()
    for im in imgs:
        oracle.ecc(im, 0, 255, oracle.VERTEX)
    dt = time.perf_counter() - t0
    vox = sum(im.size for im in imgs)
    res["uneven_batch_first_images"] = {"value": vox / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                      "sample": f"the first 16 2D images and first 2 3D patches of the batch ({vox} voxels)"}
    return res


def run_topcell_and_4d(args):
    """NEXT-4 of the scope: (1) the top-cell complex (the paper's own
    Sec. 2.1 reading) on the 512^3 benchmark volume, stencil time beside the
    vertex complex, same flush and timing; (2) 4D images through
    ecc_compute_nd: smoothed fields (sigma 2), 64^4 and 128^4 uint8 and 64^4
    at 10-bit levels."""
    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    vol = synth.smooth_3d_512(device="cuda")
    l2 = torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size
    flush = torch.empty(2 * l2 + (1 << 20), dtype=torch.uint8, device="cuda")
    res = {}
    for name, mode in (("vertex", ecc.ECC_VERTEX_MAX), ("topcell", ecc.ECC_TOPCELL_MIN)):
        plan = ecc.ecc_plan("u8", 0, 255, complex_mode=mode, max_voxels=vol.numel(), flags=ecc.ECC_FLAG_TIME_KERNELS)
        out = ecc.ecc_compute(plan, vol)
        ecc.ecc_status_get(plan)
        for _ in range(3):
            flush.fill_(1)
            ecc.ecc_compute(plan, vol, out)
        torch.cuda.synchronize()
        ecc.ecc_plan_kernel_time(plan)
        for i in range(10):
            flush.fill_(i & 0xFF)
            ecc.ecc_compute(plan, vol, out)
        kern_ms, kern_n = ecc.ecc_plan_kernel_time(plan)
        res[f"{name}_512cube_stencil_us"] = kern_ms / max(kern_n, 1) * 1e3
    res["4d"] = [time_4d(side, dt, hi) for side, dt, hi in ((64, np.uint8, 255), (128, np.uint8, 255),
                                                             (64, np.uint16, 1023))]
    return res


def time_4d(side, dt, hi, reps=5):
    """One 4D case through ecc_compute_nd: a side^4 smoothed field (sigma 2,
    seed 6) quantized to dt (uint16: 10-bit levels), vertex complex; mean
    of `reps` calls timed with CUDA events after one checked call."""
    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    g = torch.Generator(device="cuda")
    g.manual_seed(6)
    f = synth.smooth(torch.randn((side,) * 4, generator=g, device="cuda"), 2.0)
    img4 = synth.quantize(f, dt).contiguous()
    del f
    if dt == np.uint16:   # 10-bit levels
        img4 = (img4.to(torch.int32) // 64).to(torch.uint16)
    plan = ecc.ecc_plan("u8" if dt == np.uint8 else "u16", 0, hi, max_voxels=img4.numel())
    out = ecc.ecc_compute_nd(plan, img4)
    ecc.ecc_status_get(plan)
    assert int(out[-1].item()) == 1   # the whole box is contractible
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ecc.ecc_compute_nd(plan, img4, out)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    return {"workload": f"{side}^4 {np.dtype(dt).name} smoothed field (sigma 2), {hi + 1} bins, vertex complex",
            "ms": ms, "gvox_s": img4.numel() / (ms * 1e-3) / 1e9}


def run_serving(args):
    """Poisson stream of mixed 2D/3D uint8/uint16 requests (crops of resident
    seeded fields): p50/p99 latency at the nominal rate, and throughput of a
    saturating replay of the same list against the sequential plain path."""
    import threading

    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth
    reqs = synth.poisson_requests(2000.0, args.serve_seconds)
    views = synth.serving_crops(reqs, synth.serving_bases(device="cuda"))
    vox = sum(int(v.numel()) for v, _ in views)

    def serve(replay_rate: bool):
        srv = ecc.ecc_server_create(120 << 30, n_streams=4, max_batch=64)
        # start-up: the plans of the two job keys on every slot (workspace,
        # autotuning, batch graph), before the first request arrives
        ecc.ecc_server_prepare(srv, "u8", 0, 255)
        ecc.ecc_server_prepare(srv, "u16", 0, 65535)
        outs = [np.zeros(hi + 1, np.int64) for _, hi in views]
        tickets = [0] * len(views)
        t0 = time.perf_counter()
        for i, ((v, hi), r) in enumerate(zip(views, reqs)):
            if replay_rate:
                delay = r["t"] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            tickets[i] = ecc.ecc_submit(srv, v, 0, hi, out=outs[i])
        for t in tickets:
            assert ecc.ecc_wait(srv, t, 600_000_000) == ecc.ECC_OK
        wall = time.perf_counter() - t0
        st = ecc.ecc_server_stats(srv)
        ecc.ecc_server_destroy(srv)
        return wall, st, outs

    wall_rt, st_rt, outs_rt = serve(True)
    wall_sat, st_sat, outs_sat = serve(False)
    # sequential plain path: one ecc_compute per request, synchronized
    plans = {255: ecc.ecc_plan("u8", 0, 255, max_voxels=1 << 31), 65535: ecc.ecc_plan("u16", 0, 65535, max_voxels=1 << 31)}
    outs_seq = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for v, hi in views:
        o = ecc.ecc_compute(plans[hi], v)
        outs_seq.append(o.cpu().numpy())
    wall_seq = time.perf_counter() - t0
    mism_rt = [i for i, (a, b) in enumerate(zip(outs_seq, outs_rt)) if not np.array_equal(a, b)]
    mism_sat = [i for i, (a, b) in enumerate(zip(outs_seq, outs_sat)) if not np.array_equal(a, b)]
    same = not mism_rt and not mism_sat
    if not same:
        raise AssertionError(f"served results differ from the sequential plain path: nominal {mism_rt[:4]}, "
                             f"saturating {mism_sat[:4]}")
    return {"workload": f"Poisson 2000 req/s x {args.serve_seconds:g} s (seed 4), 70% 2D u8 128^2-4096^2, "
                        "30% 3D u8/u16 64^3-768^3, crops of resident seeded fields",
            "requests": len(views), "voxels": vox,
            "nominal": {"p50_ms": st_rt["p50_us"] / 1e3, "p99_ms": st_rt["p99_us"] / 1e3,
                        "max_ms": st_rt["max_us"] / 1e3, "launches": st_rt["launches"],
                        "gvox_s": vox / wall_rt / 1e9},
            "saturating": {"gvox_s": vox / wall_sat / 1e9, "p50_ms": st_sat["p50_us"] / 1e3,
                           "p99_ms": st_sat["p99_us"] / 1e3, "launches": st_sat["launches"]},
            "sequential_plain": {"gvox_s": vox / wall_seq / 1e9},
            "served_vs_sequential": wall_seq / wall_sat,
            "identical_results": bool(same),
            "mismatches": {"nominal": len(mism_rt), "saturating": len(mism_sat),
                           "first": [(i, list(views[i][0].shape), str(views[i][0].dtype)) for i in (mism_rt + mism_sat)[:4]]}}


def arg_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=None,
                    help="GPUs (one rank each); default: WORLD_SIZE under a launcher, else 1")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="default", choices=["default", "direct"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--extras", action="store_true", help="also run the batched and serving workloads")
    ap.add_argument("--shape", default="512,512,512")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="duration of the serving workload's Poisson request stream (the configuration's 60 s)")
    ap.add_argument("--main-only", action="store_true",
                    help="only the headline 512^3 workload (no keys for the other configurations)")
    ap.add_argument("--quick", action="store_true",
                    help="profiler runs: no one-second warm-up floor, no e2e and CPU legs")
    ap.add_argument("--only-4d", type=int, default=0, metavar="SIDE",
                    help="profiler runs: only the 4D case SIDE^4 uint8 (three calls after the checked one)")
    ap.add_argument("--only-c3", action="store_true",
                    help="profiler runs: only the 1024^3 uint16 volume (three calls after the checked one)")
    ap.add_argument("--only-c1", action="store_true",
                    help="profiler runs: only the 256^2 uint8 image (ten calls after the checked one)")
    ap.add_argument("--only-pipe", type=int, default=0, metavar="SIDE",
                    help="profiler runs: only the smoothing pipeline on a SIDE^2 field at 255 levels (four "
                         "warm-up rounds, then four timed rounds)")
    ap.add_argument("--only-present", action="store_true",
                    help="profiler runs: only ecc_levels_present on the 512^3 field rounded to 1024 levels (one "
                         "checked call, then three)")
    ap.add_argument("--only-c4", default=None, choices=["all", "2d", "3d"],
                    help="profiler runs: only the uneven batch, or its 2D or 3D images (three calls after "
                         "the checked one)")
    return ap


def main():
    args = arg_parser().parse_args()
    args.warmup = max(args.warmup, 3)
    ws_env = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus is None:
        args.gpus = ws_env
    if "WORLD_SIZE" in os.environ and ws_env != args.gpus:
        print(f"bench.py: --gpus {args.gpus} but WORLD_SIZE={ws_env}: launch one rank per GPU, "
              f"--nproc-per-node equal to --gpus", file=sys.stderr)
        return 2
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # one process per GPU: relaunch under torch.distributed.run
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr", "127.0.0.1", "--master-port", os.environ.get("MASTER_PORT", "29531"),
               str(ROOT / "bench.py"), *sys.argv[1:]]
        return subprocess.call(cmd)
    if args.impl == "reference":
        return run_reference(args)
    if args.only_4d:
        import numpy as np
        print(json.dumps(time_4d(args.only_4d, np.uint8, 255, reps=3)))
        return
    if args.only_c3:
        print(json.dumps(time_c3(reps=3)))
        return
    if args.only_c1:
        print(json.dumps(time_c1(reps=10)))
        return
    if args.only_c4:
        print(json.dumps(time_c4_part(args.only_c4, reps=3)))
        return
    if args.only_present:
        print(json.dumps(time_present(reps=3)))
        return
    if args.only_pipe:
        print(json.dumps(time_pipe(args.only_pipe, rounds=4)))
        return

    import numpy as np
    import torch

    import paper_2203_09087_gb300 as ecc
    import synth

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    shape = tuple(int(x) for x in args.shape.split(","))
    vol = synth.smooth_3d_512(device="cuda", shape=shape)
    nvox = vol.numel()
    # no ECC_FLAG_TIME_KERNELS in the timed plan: its events inside every call
    # cost ~5 us a step; a step of one launch is timed by the step's own events
    flags = ecc.ECC_FLAG_KERNEL_DIRECT if args.kernel == "direct" else 0
    plan = ecc.ecc_plan("u8", 0, 255, max_voxels=nvox, flags=flags)
    out = torch.empty(256, dtype=torch.int64, device="cuda")
    l2 = torch.cuda.get_device_properties(local).L2_cache_size
    flush = torch.empty(2 * l2 + (1 << 20), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    # correctness guard on the benchmarked volume: last ECC value of a full box is 1
    ecc.ecc_compute(plan, vol, out)
    ecc.ecc_status_get(plan)
    assert int(out[-1].item()) == 1

    clock_fd, clock_path = tempfile.mkstemp(prefix=f"ecc_clocks_rank{rank}_", suffix=".csv")
    os.close(clock_fd)
    sampler = ClockSampler(clock_path)
    with sampler:
        # warm-up (at least W steps and about a second, so clocks are sampled under load)
        t_end = time.perf_counter() + (0.0 if args.quick else 1.0)
        w = 0
        while w < args.warmup or time.perf_counter() < t_end:
            flush.fill_(w & 0xFF)
            ecc.ecc_compute(plan, vol, out)
            w += 1
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        _barrier(dist, torch)
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            starts[i].record(stream)
            ecc.ecc_compute(plan, vol, out)
            ends[i].record(stream)
        _barrier(dist, torch)
        launches_per_step = ecc.ecc_plan_last_launches(plan)
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        if launches_per_step == 1:
            # the step's events on the launching stream bracket the one
            # stencil launch (the scan is fused into it): its duration
            kern_ms, kern_n = sum(step_ms), len(step_ms)
            kern_src = "the timed steps' own CUDA events, each around the single stencil launch"
        else:
            # several launches a step: the stencil alone, timed by the
            # library's events in a pass of its own, same flush per step
            tplan = ecc.ecc_plan("u8", 0, 255, max_voxels=nvox, flags=flags | ecc.ECC_FLAG_TIME_KERNELS)
            for i in range(args.warmup):
                flush.fill_(i & 0xFF)
                ecc.ecc_compute(tplan, vol, out)
            torch.cuda.synchronize()
            ecc.ecc_plan_kernel_time(tplan)
            for i in range(args.steps):
                flush.fill_(i & 0xFF)
                ecc.ecc_compute(tplan, vol, out)
            torch.cuda.synchronize()
            kern_ms, kern_n = ecc.ecc_plan_kernel_time(tplan)
            tplan.close()
            kern_src = "ECC_FLAG_TIME_KERNELS events around the stencil launch, a pass after the timed steps"

        # warm-L2 steps (no flush; the 134 MB input is about the size of L2)
        warm_steps = min(args.steps, 20)
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        for _ in range(warm_steps):
            ecc.ecc_compute(plan, vol, out)
        w1.record(stream)
        torch.cuda.synchronize()
        warm_ms = w0.elapsed_time(w1) / warm_steps

        # end to end from pinned host memory through ecc_compute_host
        e2e_steps, e2e_s = 0, float("nan")
        if not args.quick:
            host = vol.cpu().pin_memory().numpy()
            e2e_out = np.empty(256, np.int64)
            for _ in range(3):
                ecc.ecc_compute_host(plan, host, e2e_out)
            e2e_steps = max(3, min(args.steps, 20))
            _barrier(dist, torch)
            t0 = time.perf_counter()
            for _ in range(e2e_steps):
                ecc.ecc_compute_host(plan, host, e2e_out)
            _barrier(dist, torch)
            e2e_s = time.perf_counter() - t0
            assert np.array_equal(e2e_out, out.cpu().numpy())

    total_ms = _max_over_ranks(dist, torch, sum(step_ms))
    e2e_s = _max_over_ranks(dist, torch, e2e_s)
    value = whole_job_gvox_s(nvox, args.steps, ws, total_ms * 1e-3)
    e2e_value = whole_job_gvox_s(nvox, e2e_steps, ws, e2e_s) if e2e_steps else None

    peak, peak_src = _peaks()
    alg_bytes = nvox * 1 + 256 * 8
    kern_avg_s = kern_ms / max(kern_n, 1) * 1e-3
    achieved = alg_bytes / kern_avg_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                # the committed counters are the bit-sliced kernel's
                "traffic": _traffic_for(_kernel_digest()) if args.kernel == "default" else None,
                "peak_source": peak_src,
                "kernel_us": kern_avg_s * 1e6, "algorithmic_bytes_per_launch": alg_bytes,
                "duration_source": kern_src}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "shape": list(shape), "nbins": 256, "complex": "vertex",
                       "parallelism": f"replicas{ws}", "l2": "flushed (2x L2 write) before every step",
                       "kernel": args.kernel},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nvox, "d2h_bytes_per_step": 256 * 8,
                    "path": "ecc_compute_host, pinned host input, chunked H2D overlapped with kernels"},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": sampler.summary()}
    if args.kernel == "default":
        clk = line["clocks"]
        line["roofline_alu"] = alu_roofline(_kernel_digest(), kern_avg_s,
                                            torch.cuda.get_device_properties(local).multi_processor_count,
                                            clk.get("sm_mhz") or clk.get("sm_max_mhz"))
    os.unlink(clock_path)
    # voxels with a nonzero signed count (the histogram insertions), from one
    # extra counting call outside the timed region
    cplan = ecc.ecc_plan("u8", 0, 255, max_voxels=nvox, flags=ecc.ECC_FLAG_COUNT_EMITTED)
    ecc.ecc_compute(cplan, vol, out)
    nonzero = ecc.ecc_plan_emitted(cplan)
    cplan.close()
    srt = sorted(step_ms)
    line["timing"] = {"cold_l2_ms_mean": total_ms / args.steps, "cold_l2_ms_median": srt[len(srt) // 2],
                      "cold_l2_ms_min": srt[0], "warm_l2_ms_mean": warm_ms, "warm_steps": warm_steps}
    line["kernel_stats"] = {"nonzero_kappa_voxels": nonzero, "nonzero_kappa_fraction": nonzero / nvox}
    if rank == 0 and not args.no_cpu and not args.quick:
        host_vol = vol.cpu().numpy()
        line["cpu_baseline"] = cpu_oracle_sample(host_vol)
        line["cpu_baseline_1core"] = cpu_oracle_sample(host_vol, budget_s=4.0, threads=1)
    if rank == 0 and not args.main_only and not args.quick:
        # the other configurations, each with its own timing
        line["latency_256x256"] = run_latency_256sq(args)  # 256^2 uint8 latency
        line["single_u16"] = run_single_u16(args)        # 1024^3 uint16
        line["batched"] = run_batched(args)              # uneven batch vs one launch per image
        line["serving"] = run_serving(args)              # Poisson stream, p50/p99, saturating replay
    if args.extras and rank == 0:
        line["float_levels"] = run_float_levels(args)
        line["gaussian_pipeline"] = run_gaussian_pipeline(args)
        line["topcell_and_4d"] = run_topcell_and_4d(args)
        if not args.no_cpu:
            line["cpu_baselines_1core"] = run_cpu_baselines(args)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
