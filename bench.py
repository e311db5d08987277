#!/usr/bin/env python
"""Guided samples/s of the wavefront path-guiding hot path on GB300.

Workload (default): the 1080p frame -- Cornell-style box with the front open
plus 200 seeded spheres, SVO depth 9 (512^3), 1920x1080 pinhole primary hits
(about 1.6M alive rays), one radiance record per hit from one Lambertian
bounce, 2048 bins cut as Zipf(1.2) runs of spatially sorted rays, 32 x 32
fields with jitter and blur.  Inputs are synthetic and seeded
(paper_2405_06997_gb300.inputs).

One step = one frame of the per-frame hot path, all through libwfpg.so:
  svo_accumulate (scatter the frame's records + bottom-up average),
  bin_rays, guide_build_pdf, guide_sample (one guided sample per ray),
  guide_eval_pdf (MIS density of one BSDF direction per ray).
The SVO itself is built once per scene (reported as svo_build_ms).

value = alive rays (= guided samples) per second, device time of the step
measured with CUDA events on the launching stream, L2 flushed between steps.
e2e = the same step through the C ABI with host buffers: pinned-host -> device
copies of the frame's inputs and device -> host copies of its results inside
the timed region.

--impl reference times the CPU oracle (the plain C++ restatement of the
method) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "guided samples/s at 1080p on 1 GB300"
UNIT = "guided samples/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="wfpg", choices=["wfpg", "reference"])
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-bins", type=int, default=64, help="bins in the oracle's timed sample")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal section")
    ap.add_argument("--learned-steps", type=int, default=2000, help="online training steps (65,536 bins each)")
    ap.add_argument("--learned-frames", type=int, default=16, help="frames of the equal-spp comparison")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-frame section")
    ap.add_argument("--batched-frames", type=int, default=20, help="timed frames of the batched section")
    ap.add_argument("--no-city", action="store_true", help="skip the large city section")
    ap.add_argument("--city-only", action="store_true", help="run only the city section and print it")
    ap.add_argument("--city-frames", type=int, default=8, help="frames per proposal in the city section")
    ap.add_argument("--city-train-steps", type=int, default=200, help="online training steps on the city")
    ap.add_argument("--no-mesh", action="store_true", help="skip the triangle-mesh section")
    ap.add_argument("--mesh-only", action="store_true", help="run only the triangle-mesh section and print it")
    ap.add_argument("--l2-peak-only", action="store_true",
                    help="print the L2 read bandwidth measured by wfpg_stream_read over a sweep of buffer sizes")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the batched section with a fixed N = 32 tile (for profiling) and print it")
    return ap.parse_args()


def dist_init(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units, seconds, world):
    """Whole-job throughput of replicas: units summed over ranks / the slowest
    rank's time (weak scaling: every rank runs its own frame)."""
    return sum_over_ranks(float(units), world) / max_over_ranks(float(seconds), world)


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if r[5 + k].lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks(key="hbm_gbs"):
    """The measured GB300 peak from MEASURED_PEAKS.json (HBM copy GB/s, or
    cuBLAS bf16 TFLOP/s burst / sustained), else an earlier GB300 measurement."""
    fallback = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        if key in p:
            return float(p[key]), "measured"
    return fallback[key], "fallback"


def make_workload(seed):
    from paper_2405_06997_gb300 import inputs
    w = inputs.frame_spheres(seed)
    rng = np.random.default_rng(seed * 1000 + 7)
    mis = inputs.cosine_dirs(w.ray_nrm, rng).astype(np.float32)   # one BSDF direction per ray
    return w, mis


# ------------------------------------------------------------------ oracle timing
def oracle_frame_time(w, mis, bins_sample, frame=0, svo=None):
    """Time the CPU oracle on one frame with the field/sampling stages run for a
    bounded sample of bins; returns (extrapolated frame seconds, detail).  The
    SVO is built once per scene (not part of the frame)."""
    import oracle
    t0 = time.perf_counter()
    s = svo if svo is not None else oracle.SVO(w.scene, w.depth)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    s.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    t_acc = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = s.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=w.bin_sizes, seed=w.seed, frame=frame)
    t_bin = time.perf_counter() - t0
    nb = b["n_bins"]
    sel = np.linspace(0, nb - 1, min(bins_sample, nb)).astype(np.int64)
    t0 = time.perf_counter()
    g = s.guide_build(w.ray_pos[b["origin_ray"][sel]], sel, w.grid_n, jitter=True, blur=True,
                      seed=w.seed, frame=frame)
    t_guide = time.perf_counter() - t0
    rays = np.flatnonzero(np.isin(b["bin_of_ray"], sel))
    remap = np.zeros(nb, np.uint32)
    remap[sel] = np.arange(len(sel), dtype=np.uint32)
    local = remap[b["bin_of_ray"][rays]]
    t0 = time.perf_counter()
    d, p, c = oracle.guide_sample(g["pdf"], g["cdf_row"], g["cdf_marg"], w.grid_n, local, w.u[rays])
    oracle.guide_eval_pdf(g["pdf"], w.grid_n, local, mis[rays])
    t_samp = time.perf_counter() - t0
    frac_bins = len(sel) / nb
    frac_rays = max(len(rays), 1) / len(w.ray_pos)
    t_frame = t_acc + t_bin + t_guide / frac_bins + t_samp / frac_rays
    detail = dict(svo_build_s=t_build, accumulate_s=t_acc, bin_s=t_bin, guide_s=t_guide,
                  sample_s=t_samp, bins=len(sel), rays=int(len(rays)))
    return t_frame, detail


# The field stage (per bin: cone rays, blur, CDFs, then the bin's samples) is
# independent across bins, so the oracle runs it on every host core: a pool of
# spawned processes (the CUDA context of this process is never forked), each
# holding its own copy of the oracle's SVO with the frame's records accumulated
# and the frame's binning (built once, before any timed region), each timing
# its share of the bins.  Accumulation and binning stay single-threaded, as the
# oracle is.
_OW = None


def _oracle_worker_init(seed):
    global _OW
    import oracle
    w, mis = make_workload(seed)
    s = oracle.SVO(w.scene, w.depth)
    s.accumulate(w.rec_pos, w.rec_wout, w.rec_L)
    b = s.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=w.bin_sizes, seed=w.seed, frame=0)
    _OW = (w, mis, s, b)


def _oracle_worker_fields(task):
    """Fields + sampling + PDF evaluation for the given bins; returns (seconds, rays)."""
    import oracle
    sel, frame = task
    w, mis, s, b = _OW
    sel = np.asarray(sel, np.int64)
    nb = b["n_bins"]
    t0 = time.perf_counter()
    g = s.guide_build(w.ray_pos[b["origin_ray"][sel]], sel, w.grid_n, jitter=True, blur=True, seed=w.seed,
                      frame=frame)
    rays = np.flatnonzero(np.isin(b["bin_of_ray"], sel))
    remap = np.zeros(nb, np.uint32)
    remap[sel] = np.arange(len(sel), dtype=np.uint32)
    local = remap[b["bin_of_ray"][rays]]
    oracle.guide_sample(g["pdf"], g["cdf_row"], g["cdf_marg"], w.grid_n, local, w.u[rays])
    oracle.guide_eval_pdf(g["pdf"], w.grid_n, local, mis[rays])
    return time.perf_counter() - t0, int(len(rays))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_cpu():
    """The host CPU's name: /proc/cpuinfo's model name (x86), else its
    implementer and part codes (Arm), with the machine type."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, sep, v = line.partition(":")
                if sep and k.strip() not in fields:
                    fields[k.strip()] = v.strip()
    except OSError:
        pass
    if "model name" in fields:
        name = fields["model name"]
    elif "CPU part" in fields:
        name = f"implementer {fields.get('CPU implementer', '?')} part {fields['CPU part']}"
    else:
        name = platform.processor() or "unknown"
    return f"{platform.machine()} {name}"


def oracle_pool(seed, cores):
    import multiprocessing as mp
    pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init, initargs=(seed,))
    pool.map(_oracle_worker_fields, [([0], 0)] * cores)  # every worker has finished its set-up
    return pool


def oracle_fields_parallel(pool, cores, nb, per_worker, frame, offset=0):
    """Field stage for cores x per_worker bins spread over the frame, one share
    per process; returns (wall seconds of the parallel region scaled to all nb
    bins, bins timed, rays)."""
    total = min(nb, cores * per_worker)
    sel = (np.arange(total, dtype=np.int64) * (nb // total) + offset) % nb
    shares = [(list(c), frame) for c in np.array_split(sel, cores) if len(c)]
    t0 = time.perf_counter()
    out = pool.map(_oracle_worker_fields, shares, chunksize=1)
    wall = time.perf_counter() - t0
    return wall * nb / total, total, sum(r for _, r in out)


def oracle_step(w, mis, s, full_bins, nsel, k, pool, cores):
    """One measured step of the CPU oracle over a fraction f = nsel / bins of
    the frame: accumulate f of its records and bin f of its rays on one core
    (rotating slices), then build the fields of nsel of its bins (rotating,
    spread over the frame, from one full binning done beforehand) and sample
    and evaluate their rays over the process pool.  Returns the wall seconds
    of the step, the guided samples it made (the sampled rays) and each
    stage's time scaled to the whole frame."""
    nr, R, nb = len(w.rec_L), len(w.ray_pos), full_bins["n_bins"]
    f = nsel / nb
    na = max(1, int(round(f * nr)))
    o = (k * na) % nr
    sl = slice(o, min(nr, o + na))
    t_start = time.perf_counter()
    s.accumulate(w.rec_pos[sl], w.rec_wout[sl], w.rec_L[sl])
    t_acc = time.perf_counter() - t_start
    nrb = max(1, int(round(f * R)))
    o = (k * nrb) % R
    sr = slice(o, min(R, o + nrb))
    n_sub = sr.stop - sr.start
    t0 = time.perf_counter()
    s.bin_rays(w.ray_pos[sr], w.ray_nrm[sr], mode=1, sizes=np.array([n_sub], np.uint32), seed=w.seed, frame=k)
    t_bin = time.perf_counter() - t0
    per = max(1, -(-nsel // cores))
    t0 = time.perf_counter()
    t_fs_scaled, nsel_done, nrays = oracle_fields_parallel(pool, cores, nb, per, k, offset=k)
    t_fields = time.perf_counter() - t0
    wall = time.perf_counter() - t_start
    frame_s = t_acc * nr / (sl.stop - sl.start) + t_bin * R / n_sub + t_fs_scaled
    return wall, nrays, frame_s, dict(records=sl.stop - sl.start, binned_rays=n_sub, bins=nsel_done,
                                      sampled_rays=nrays, accumulate_s=t_acc, bin_s=t_bin, fields_s=t_fields)


def arm_config(w, svo_nodes, world):
    """The workload description both arms print."""
    return {"workload": w.desc, "rays": len(w.ray_pos), "records": len(w.rec_L), "bins": len(w.bin_sizes),
            "grid": w.grid_n, "svo_depth": w.depth, "svo_nodes": int(svo_nodes),
            "l2": "flushed (256 MiB write) between steps", "parallelism": f"replicas x{world}",
            "streams": "bin_rays on a second stream beside svo_accumulate; the field waits for both"}


def run_reference(args, world, rank):
    """The CPU oracle on the GPU arm's workload, metric and unit.  Each step
    does a fraction of the frame's work in every stage (records, rays, bins
    alike), sized so that warm-up + timed steps take about two minutes; the
    line's value and ms_per_step are the measured guided samples per second
    and wall time of those steps, and the full-frame rate their stages
    project is reported beside them."""
    if rank != 0:
        return
    import oracle
    w, mis = make_workload(args.seed)
    R = len(w.ray_pos)
    svo = oracle.SVO(w.scene, w.depth)
    full_bins = svo.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=w.bin_sizes, seed=w.seed, frame=0)
    nb = full_bins["n_bins"]
    cores = host_cores()
    pool = oracle_pool(args.seed, cores)
    try:
        # probe one small step, then size the per-step fraction to the budget
        n0 = min(nb, 4 * cores)
        wall0, *_ = oracle_step(w, mis, svo, full_bins, n0, 0, pool, cores)
        budget = 100.0 / max(1, args.warmup + args.steps)
        nsel = int(min(nb, max(n0, round(n0 * budget / max(wall0, 1e-3)))))
        walls, units, frames, detail = [], [], [], None
        for k in range(args.warmup + args.steps):
            wall, nrays, frame_s, detail = oracle_step(w, mis, svo, full_bins, nsel, k + 1, pool, cores)
            if k >= args.warmup:
                walls.append(wall)
                units.append(nrays)
                frames.append(frame_s)
    finally:
        pool.close()
        pool.join()
    ms = statistics.mean(walls) * 1e3
    value = sum(units) / sum(walls)
    frame_rate = R / statistics.mean(frames)
    sample = (f"per step {nsel} of {nb} bins (fraction f = {nsel / nb:.3f} of the frame): accumulate f of the "
              f"{len(w.rec_L)} records and bin f of the {R} rays on one core, fields/CDFs of the {nsel} bins and "
              f"sampling + PDF evaluation of their rays over {cores} processes; value = guided samples made / "
              f"wall time of the timed steps")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "impl": "reference",
            "config": arm_config(w, svo.n_nodes, world),
            "guided_samples_per_step": statistics.mean(units),
            "frame_rate_projected": {"value": frame_rate, "unit": UNIT,
                                     "how": "each stage's measured time scaled by its fraction of the frame "
                                            "(records, rays, bins), summed: one full frame's time"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, world, rank, local):
    import torch
    from paper_2405_06997_gb300 import wfpg as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w, mis = make_workload(args.seed)
    R = len(w.ray_pos)
    n_rec = len(w.rec_L)
    B = len(w.bin_sizes)
    N = w.grid_n
    stream = torch.cuda.current_stream()
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    # SVO generation, once per scene
    q = T(w.scene.quads)
    sp = T(w.scene.spheres)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    svo = W.svo_build(q, sp, w.scene.lo, w.scene.size, w.depth)
    e1.record()
    torch.cuda.synchronize()
    svo_build_ms = e0.elapsed_time(e1)

    inp = dict(rec_pos=T(w.rec_pos), rec_wout=T(w.rec_wout), rec_L=T(w.rec_L), ray_pos=T(w.ray_pos),
               ray_nrm=T(w.ray_nrm), u=T(w.u), mis=T(mis), sizes=T(w.bin_sizes.view(np.int32)))
    binout = dict(bin_of_ray=torch.empty(R, dtype=torch.int32, device=dev),
                  ray_order=torch.empty(R, dtype=torch.int32, device=dev),
                  bin_offset=torch.empty(B + 1, dtype=torch.int32, device=dev),
                  origin_ray=torch.empty(B, dtype=torch.int32, device=dev),
                  n_bins=torch.zeros(1, dtype=torch.int32, device=dev))
    ws = torch.empty(W.bin_rays_workspace_size(svo, R, W.BIN_RUNS, B), dtype=torch.uint8, device=dev)
    guide = (torch.empty((B, N * N), dtype=torch.float32, device=dev),
             torch.empty((B, N * N), dtype=torch.float32, device=dev),
             torch.empty((B, N), dtype=torch.float32, device=dev))
    samp = (torch.empty((R, 3), dtype=torch.float32, device=dev),
            torch.empty(R, dtype=torch.float32, device=dev),
            torch.empty(R, dtype=torch.int32, device=dev))
    evalout = torch.empty(R, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    stage_names = ("accumulate", "bin_rays", "guide_build_pdf", "guide_sample", "guide_eval_pdf")
    sev = [torch.cuda.Event(enable_timing=True) for _ in range(len(stage_names) + 1)]
    stage_ms = {k: [] for k in stage_names}

    # UpdateExitance and the binning are independent (the binning reads only the
    # tree's structure and the rays): by default the binning runs on a second
    # stream beside the accumulation, and the field waits for both
    side = torch.cuda.Stream()

    def step(frame, x, time_guide=False, outs=None, overlap=True):
        so, eo = outs if outs is not None else (samp, evalout)
        mark = (lambda i: sev[i].record()) if time_guide else (lambda i: None)
        if overlap:
            main = torch.cuda.current_stream()
            side.wait_stream(main)
            with torch.cuda.stream(side):
                W.bin_rays(svo, x["ray_pos"], x["ray_nrm"], mode=W.BIN_RUNS, sizes=x["sizes"], seed=w.seed,
                           frame=frame, bin_cap=B, out=binout, workspace=ws)
            W.svo_accumulate(svo, x["rec_pos"], x["rec_wout"], x["rec_L"])
            main.wait_stream(side)
        else:
            mark(0)
            W.svo_accumulate(svo, x["rec_pos"], x["rec_wout"], x["rec_L"])
            mark(1)
            W.bin_rays(svo, x["ray_pos"], x["ray_nrm"], mode=W.BIN_RUNS, sizes=x["sizes"], seed=w.seed,
                       frame=frame, bin_cap=B, out=binout, workspace=ws)
        mark(2)
        W.guide_build_pdf(svo, x["ray_pos"], binout["origin_ray"], binout["n_bins"], B, N=N,
                          jitter=True, blur=True, seed=w.seed, frame=frame, out=guide)
        mark(3)
        W.guide_sample(*guide, N, binout["bin_of_ray"], x["u"], out=so)
        mark(4)
        W.guide_eval_pdf(guide[0], N, binout["bin_of_ray"], x["mis"], out=eo)
        mark(5)

    for k in range(args.warmup):
        step(k, inp)
    torch.cuda.synchronize()
    status = svo.status()

    clocks = ClockSampler(local) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.5)  # the sampler is up before the timed region starts
    launches0 = W.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    step_ms, guide_ms = [], []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()            # evict L2 between timed steps (outside the timed events)
        ev[k][0].record()
        step(args.warmup + k, inp, time_guide=True)
        ev[k][1].record()
        sev[-1].synchronize()
        for j in range(2, len(stage_names)):
            stage_ms[stage_names[j]].append(sev[j].elapsed_time(sev[j + 1]))
        guide_ms.append(stage_ms["guide_build_pdf"][-1])
    torch.cuda.synchronize()
    barrier(world)
    launches = W.kernel_launches() - launches0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = statistics.mean(step_ms)
    # the accumulation and the binning timed one after the other (outside the timed region)
    seq_ms = []
    for k in range(min(args.steps, 50)):
        flush.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        step(args.warmup + args.steps + k, inp, time_guide=True, overlap=False)
        a1.record()
        sev[-1].synchronize()
        for j in range(2):
            stage_ms[stage_names[j]].append(sev[j].elapsed_time(sev[j + 1]))
        seq_ms.append(a0.elapsed_time(a1))
    seq_v = job_rate(R, statistics.mean(seq_ms) / 1e3, world)
    ms_max = max_over_ranks(ms, world)
    rays_all = sum_over_ranks(float(R), world)
    value = job_rate(R, ms / 1e3, world)

    # the same five calls captured once into a CUDA graph (every call of the ABI is
    # stream-ordered and capturable) and replayed: the work per step is unchanged,
    # only the host launches and the gaps between kernels go (the frame index that
    # keys the random streams is the one captured)
    gstream = torch.cuda.Stream()
    gstream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(gstream):
        step(7000, inp)
    torch.cuda.current_stream().wait_stream(gstream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(7001, inp)
    torch.cuda.synchronize()
    for _ in range(3):
        graph.replay()
    graph_ms = []
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        b.synchronize()
        graph_ms.append(a.elapsed_time(b))
    graph_v = rays_all / (max_over_ranks(statistics.mean(graph_ms), world) / 1e3)
    del graph

    # end to end through the C ABI with host buffers: every step copies its inputs
    # from pinned host memory and reads its results back.  An upload stream fills
    # one half of a double buffer while the compute stream works on the other, and
    # a download stream returns the previous step's results; each step's copies are
    # inside the timed region, they only overlap another step's compute.
    pinned = {k: v.cpu().pin_memory() for k, v in inp.items()}
    dev_in = [{k: torch.empty_like(v) for k, v in inp.items()} for _ in range(2)]
    outs = [(samp, evalout), (tuple(torch.empty_like(t) for t in samp), torch.empty_like(evalout))]
    host_out = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (*o[0], o[1])] for o in outs]
    h2d = sum(v.numel() * v.element_size() for v in pinned.values())
    d2h = sum(t.numel() * t.element_size() for t in host_out[0])
    up, down = torch.cuda.Stream(), torch.cuda.Stream()  # host -> device, device -> host
    ev = {k: [torch.cuda.Event(), torch.cuda.Event()] for k in ("copied", "done", "read")}

    def e2e_run(n, frame0):
        comp = torch.cuda.current_stream()
        for k in range(n):
            i = k % 2
            with torch.cuda.stream(up):
                up.wait_event(ev["done"][i])  # the step that read dev_in[i] two steps ago
                for key, v in pinned.items():
                    dev_in[i][key].copy_(v, non_blocking=True)
                ev["copied"][i].record(up)
            comp.wait_event(ev["copied"][i])
            comp.wait_event(ev["read"][i])  # results of two steps ago are on the host
            flush.zero_()
            step(frame0 + k, dev_in[i], outs=outs[i])
            ev["done"][i].record(comp)
            with torch.cuda.stream(down):
                down.wait_event(ev["done"][i])
                for h, d in zip(host_out[i], (*outs[i][0], outs[i][1])):
                    h.copy_(d, non_blocking=True)
                ev["read"][i].record(down)
        comp.wait_stream(up)
        comp.wait_stream(down)

    for e in (*ev["done"], *ev["read"]):
        e.record()
    e2e_run(4, 1000)
    torch.cuda.synchronize()
    n_e2e = max(3, args.steps // 2)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    e2e_run(n_e2e, 2000)
    b.record()
    b.synchronize()
    e2e_ms = [a.elapsed_time(b) / n_e2e]
    e2e_v = rays_all / (max_over_ranks(statistics.mean(e2e_ms), world) / 1e3)

    # the same frame with GuideRays fused as Alg. 3 states it (field, PDF and
    # CDFs in shared memory; each ray draws from alpha * guided + (1 - alpha) *
    # cosine with its exact density): accumulate + bin_rays + guide_build_sample
    u3 = torch.cat([inp["u"], T(inputs_uniforms(w.seed + 5, (R, 1)))], dim=1).contiguous()
    fused_out = (torch.empty((R, 3), dtype=torch.float32, device=dev), torch.empty(R, dtype=torch.float32, device=dev))

    def fused_step(frame):
        main = torch.cuda.current_stream()
        side.wait_stream(main)
        with torch.cuda.stream(side):
            W.bin_rays(svo, inp["ray_pos"], inp["ray_nrm"], mode=W.BIN_RUNS, sizes=inp["sizes"], seed=w.seed,
                       frame=frame, bin_cap=B, out=binout, workspace=ws)
        W.svo_accumulate(svo, inp["rec_pos"], inp["rec_wout"], inp["rec_L"])
        main.wait_stream(side)
        W.guide_build_sample(svo, inp["ray_pos"], inp["ray_nrm"], binout, u3, alpha=0.5, N=N, jitter=True,
                             blur=True, seed=w.seed, frame=frame, out=fused_out)

    for k in range(3):
        fused_step(3000 + k)
    fused_ms = []
    for k in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fused_step(4000 + k)
        b.record()
        b.synchronize()
        fused_ms.append(a.elapsed_time(b))
    fused_v = rays_all / (max_over_ranks(statistics.mean(fused_ms), world) / 1e3)

    # product guiding (Sec. 3.6) on the same frame's fields: block sums + the
    # two-stage product sample mixed 50/50 with cosine sampling (density included)
    step(5000, inp)
    psums = torch.empty((B, 64), dtype=torch.float32, device=dev)
    pout = (torch.empty((R, 3), dtype=torch.float32, device=dev), torch.empty(R, dtype=torch.float32, device=dev),
            torch.empty(R, dtype=torch.int32, device=dev))
    prod_ms = []
    for k in range(3 + args.steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        W.guide_product_sums(guide[0], N, n_bins=binout["n_bins"], out=psums)
        W.guide_product_sample(guide[0], psums, N, binout["bin_of_ray"], inp["ray_nrm"], u3, alpha=0.5,
                               n_bins=binout["n_bins"], out=pout)
        b.record()
        b.synchronize()
        if k >= 3:
            prod_ms.append(a.elapsed_time(b))
    clk = clocks.stop() if clocks else None

    if rank != 0:
        return
    # roofline of the dominant kernel (guide_build_pdf's field kernel)
    peak, peak_kind = measured_peaks()
    l2_peak, l2_how = l2_read_peak(dev)
    gms = statistics.mean(guide_ms)
    alg = trace_algorithmic_bytes(w, B, N)
    achieved = alg["bytes"] / (gms / 1e3) / 1e9
    traffic, issue = read_profile_traffic()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": arm_config(w, svo.n_nodes, world),
        "sequential_step": {"value": seq_v, "unit": UNIT,
                            "ms_per_step": statistics.mean(seq_ms),
                            "calls": "the same five calls one after the other on one stream (the stage times)"},
        "svo_build_ms": svo_build_ms,
        "guide_build_ms": gms,
        "status": status,
        "gpu_launches": launches,
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms[0], "copies": "pinned host <-> device on upload / download streams, double-buffered",
                "l2": "flushed (256 MiB write) before every step"},
        "product_sampling": {"ms": statistics.mean(prod_ms), "samples_per_s": R / (statistics.mean(prod_ms) / 1e3),
                             "calls": "guide_product_sums + guide_product_sample (alpha 0.5) on the step's fields"},
        "fused_step": {"value": fused_v, "unit": UNIT, "ms_per_step": statistics.mean(fused_ms),
                       "calls": "svo_accumulate + bin_rays + guide_build_sample (alpha 0.5)"},
        "graph_step": {"value": graph_v, "unit": UNIT, "ms_per_step": statistics.mean(graph_ms),
                       "calls": "the timed step's five calls captured once into a CUDA graph and replayed "
                                "(same work; the captured frame index keys the random streams)"},
        "stages": stage_rooflines(stage_ms, alg["bytes"], R, n_rec, svo.n_nodes, peak),
        "roofline": {"kernel": "k_guide_stream + k_field_pdf (guide_build_pdf)", "bound": "hbm", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "algorithmic_bytes": alg["bytes"],
                     "algorithmic_model": alg["model"], "ncu": issue,
                     "note": "algorithmic bytes over the measured HBM copy bandwidth, as the contract defines it; "
                             "most of these bytes are L1/L2 hits (traffic = DRAM bytes per launch), so "
                             "l2_roofline, dram_roofline and issue_roofline say what bounds the kernel"},
        "issue_roofline": issue_roofline(issue, gms, clk.get("sm_mhz") if clk else None,
                                         torch.cuda.get_device_properties(dev).multi_processor_count),
        "l2_roofline": {"kernel": "k_guide_stream + k_field_pdf (guide_build_pdf)", "bound": "l2", "achieved": achieved, "peak": l2_peak,
                        "unit": "GB/s", "frac": achieved / l2_peak, "peak_kind": l2_how,
                        "note": "the same algorithmic bytes against the L2 read bandwidth measured here: the "
                                "walk's node records are served from L1/L2"},
        "dram_roofline": ({"kernel": "k_guide_stream", "bound": "hbm", "achieved": traffic / (gms / 1e3) / 1e9,
                           "peak": peak, "unit": "GB/s", "frac": traffic / (gms / 1e3) / 1e9 / peak,
                           "note": "DRAM bytes per launch (ncu, committed capture of this source) over the "
                                   "live kernel time"} if traffic else None),
        "clocks": clk,
    }
    line["large_fields"] = large_field_records(w, svo, inp, binout, B, peak, l2_peak, flush)
    if not args.no_learned:
        line["learned"] = learned_section(args, w, svo)
    if not args.no_batched:
        line["batched"] = batched_section(args)
    if not args.no_city:
        line["city"] = city_section(args)
    if not args.no_mesh:
        line["mesh"] = mesh_section(args)
    if not args.no_cpu_baseline:
        t_frame, detail = oracle_frame_time(w, mis, args.cpu_bins)
        single = {"value": R / t_frame, "unit": UNIT, "cores": 1, "kind": "oracle",
                  "sample": f"one frame: full accumulate + binning, fields for {detail['bins']} of {B} "
                            f"bins and sampling/eval of their {detail['rays']} rays, scaled to the frame"}
        cores = host_cores()
        pool = oracle_pool(args.seed, cores)
        try:
            t_fields, nbins, nrays = oracle_fields_parallel(pool, cores, B, args.cpu_bins, 0)
        finally:
            pool.close()
            pool.join()
        t_all = detail["accumulate_s"] + detail["bin_s"] + t_fields
        line["cpu_baseline"] = {
            "value": R / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one frame: full accumulate + binning on one core, then fields + sampling/eval for "
                      f"{nbins} of {B} bins ({nrays} rays) split over {cores} processes, the parallel "
                      f"region's wall time scaled to the frame",
            "single_core": single, "cpu": host_cpu()}
    print(json.dumps(line))


def learned_section(args, w, svo):
    """Learned proposal vs the SVO-traced field on the same frame: online
    training (65,536 traced bins per step), held-out KL, and the per-pixel
    variance and guided samples/s of the batched frame (one guided bounce per
    path from the 1080p camera, cache fixed) at equal samples per pixel."""
    import torch
    from paper_2405_06997_gb300 import learned as LG, wfpg as W
    # online training on the frame's own guided points (the primary hits), targets traced on the fly
    tr = LG.OnlineTrainer(svo, w.scene, batch=65536, lr=1e-3, seed=w.seed, points=(w.ray_pos, w.ray_nrm))
    kl0 = tr.heldout_kl()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tr.train(args.learned_steps)
    train_s = time.perf_counter() - t0
    kl1 = tr.heldout_kl()
    floor = LG.traced_frame_kl(tr)
    # the MLP's own training step (forward + backward + Adam, tcgen05 GEMMs) on one traced batch
    tr._targets(tr.pos[:65536], tr.tgt, 0)
    for _ in range(3):
        W.guide_learned_train_step(tr.mlp, tr.pos[:65536], tr.nrm[:65536], tr.tgt[0], lo=tr.lo, size=tr.size,
                                   lr=0.0, loss=tr.loss)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        W.guide_learned_train_step(tr.mlp, tr.pos[:65536], tr.nrm[:65536], tr.tgt[0], lo=tr.lo, size=tr.size,
                                   lr=0.0, loss=tr.loss)
    e1.record()
    e1.synchronize()
    step_ms = e0.elapsed_time(e1) / 20
    flop = 3 * 157440 * 65536  # forward + both backward GEMMs per layer
    peak, _ = measured_peaks("bf16_tflops_sustained")
    tau = 1.5 * floor
    cam = dict(eye=(0.5, 0.5, -1.0), forward=(0.0, 0.0, 1.0), up=(0.0, 1.0, 0.0), vfov=40.0, width=1920,
               height=1080, max_depth=1, rr_depth=2)
    cmp = LG.compare_proposals(svo, w.scene, tr.mlp, cam, batches=8, frames=args.learned_frames, alpha=0.5,
                               seed=w.seed)
    return {"train_steps": args.learned_steps, "train_batch_bins": 65536, "train_seconds": train_s,
            "train_points": "the frame's primary hits (4096 held out)",
            "train_step_mlp_ms": step_ms,
            "tensor": {"bound": "tensor", "achieved": flop / (step_ms / 1e3) / 1e12, "peak": peak,
                       "unit": "TFLOP/s", "frac": flop / (step_ms / 1e3) / 1e12 / peak,
                       "flop_per_step": flop, "note": "65,536 bins; 3 x 157,440 FLOP per bin"},
            "heldout_kl_untrained": kl0, "heldout_kl_trained": kl1, "traced_frame_to_frame_kl": floor,
            "fallback_threshold": tau, "uses_learned": LG.use_learned(kl1, tau),
            "equal_spp": cmp, "mlp_status": tr.mlp.status()}


def inputs_uniforms(seed, shape):
    from paper_2405_06997_gb300 import inputs
    return inputs.uniforms24(seed, shape)


def batched_section(args, autotune=True):
    """The batched wavefront frame: the closed box of the small workload
    (SVO depth 6, seeded with its 100k records) seen from inside at 1920x1080,
    4 guided bounces with Russian roulette from the second hit, Eq. 5 records
    of every vertex accumulated after each frame, Partition-S bins (l_min 2,
    c_ray 512), everything in one CUDA graph per frame; N and the field
    kernel's tile picked by the native autotuner."""
    import torch
    from paper_2405_06997_gb300 import inputs, wfpg as W
    w = inputs.tiny_box(args.seed)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    svo = W.svo_from_scene(w.scene, w.depth)
    W.svo_accumulate(svo, T(w.rec_pos), T(w.rec_wout), T(w.rec_L))
    f = W.Frame(svo, w.scene, eye=(0.5, 0.5, 0.05), forward=(0.0, 0.0, 1.0), up=(0.0, 1.0, 0.0), vfov=70.0,
                width=1920, height=1080, max_depth=4, rr_depth=2, alpha=0.5, l_min=2, c_ray=512, N=32,
                seed=args.seed)
    t0 = time.perf_counter()
    choice, tune_ms = f.autotune((16, 32, 64), frames=4) if autotune else ({"N": 32, "block": 0, "stage": 0}, None)
    tune_s = time.perf_counter() - t0
    f.run(3)
    f.reset_image()
    torch.cuda.synchronize()
    launches0 = W.kernel_launches()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    f.run(args.batched_frames)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / args.batched_frames
    st = f.stats()
    m, v = f.image()
    # the same frames with next-event estimation (power-heuristic MIS against the mixture)
    f.set_params(nee=1)
    f.run(3)
    f.reset_image()
    torch.cuda.synchronize()
    a.record()
    f.run(args.batched_frames)
    b.record()
    b.synchronize()
    ms_nee = a.elapsed_time(b) / args.batched_frames
    m2, v2 = f.image()
    var0, var1 = float(v.double().mean()), float(v2.double().mean())
    nee = {"ms_per_frame": ms_nee, "mean_pixel_variance": var1, "mean_radiance": float(m2.double().mean()),
           "variance_ratio": var1 / var0, "efficiency_gain": (var0 * ms) / (var1 * ms_nee),
           "note": "one light sample per guided vertex (light by power, uniform point, shadow ray); "
                   "efficiency = 1 / (variance x time), against the same frames without it"}
    field = field_validation(f, svo, w, args)
    return {"workload": "closed box (D 6, 100k seed records), camera inside at (0.5, 0.5, 0.05) looking +z, "
                        "vfov 70, 1920x1080, 4 guided bounces, RR from vertex 2 (survival min(0.95, albedo)), "
                        "alpha 0.5 guided / 0.5 cosine, Partition-S l_min 2 c_ray 512, jitter + blur",
            "autotune": {"choice": choice, "ms_per_frame": tune_ms, "seconds": tune_s,
                         "candidates": {"N": [16, 32, 64], "block": [64, 128, 256], "staged": [True, False]}},
            "frames": args.batched_frames, "ms_per_frame": ms,
            "guided_samples_per_s": st["guided_samples"] / (ms * args.batched_frames / 1e3),
            "paths_per_s": f.pixels / (ms / 1e3),
            "paths_per_depth": st["paths"], "bins_per_depth": st["bins"], "records_per_frame": st["records"],
            "graph_kernels_per_frame": st["kernels_per_frame"],
            "gpu_launches": W.kernel_launches() - launches0,
            "mean_pixel_variance": float(v.double().mean()), "mean_radiance": float(m.double().mean()),
            "status": st["status"], "l2": "working set (path state ~0.6 GB) larger than L2", "nee": nee,
            "field_validation": field}


def mesh_section(args, frames=10):
    """Triangle meshes (the paper voxelises triangle scenes): the mesh room at
    subdivision 5 (about 42k triangles: a closed box, a ceiling light of two
    triangles, an icosphere, a rock and a torus), SVO depth 9 (SAT
    voxelisation + k-means winding normals), then batched 1080p frames from
    inside the room (4 guided bounces, RR, NEE with the triangle light, closest
    hits by the SVO walk over the leaves' triangle lists), constant N = 32 and
    the decaying resolution (64, 32, 16, 8 over the depths)."""
    import torch
    from paper_2405_06997_gb300 import inputs, wfpg as W
    sc = inputs.mesh_room(args.seed, 9, subdiv=5)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    q, sp, tr = T(sc.quads), T(sc.spheres), T(sc.tris)
    W.svo_build(q, sp, sc.lo, sc.size, 9, tris=tr)  # first build: module load and allocator warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    svo = W.svo_build(q, sp, sc.lo, sc.size, 9, tris=tr)
    b.record()
    b.synchronize()
    build_ms = a.elapsed_time(b)
    out = {"workload": f"mesh room ({sc.n_tris} triangles), SVO depth 9, camera at (0.5, 0.5, 0.05) looking +z, "
                       "vfov 70, 1920x1080, 4 guided bounces, RR from vertex 2, alpha 0.5, NEE, Partition-S "
                       "l_min 2 c_ray 512, closest hits by the SVO walk",
           "triangles": sc.n_tris, "svo_build_ms": build_ms, "svo_nodes": svo.n_nodes}
    for name, kw in (("constant_32", dict(N=32)), ("decay_64", dict(N=64, decay=True))):
        f = W.Frame(svo, sc, eye=(0.5, 0.5, 0.05), vfov=70.0, width=1920, height=1080, max_depth=4, rr_depth=2,
                    alpha=0.5, l_min=2, c_ray=512, seed=args.seed, nee=True, caster=2, **kw)
        f.run(3)
        f.reset_image()
        torch.cuda.synchronize()
        a.record()
        f.run(frames)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / frames
        st = f.stats()
        m, v = f.image()
        out[name] = {"ms_per_frame": ms, "guided_samples_per_s": st["guided_samples"] / (ms * frames / 1e3),
                     "paths_per_depth": st["paths"], "bins_per_depth": st["bins"],
                     "mean_pixel_variance": float(v.double().mean()), "mean_radiance": float(m.double().mean()),
                     "status": st["status"]}
        del f
    return out


def field_validation(f, svo, w, args, n_probes=16, N=32, ref_frames=64):
    """Radiance-field validation (Fig. 3): at free-space points of the box, the
    frame's probe mode path-traces the cell-averaged incident radiance (alpha 0,
    light sampling, ref_frames frames); the SVO-traced PDF at the same points
    (the cache as the timed frames left it; jitter off, blur on, eps 1e-2) is
    scored by KL(reference || traced), next to the uniform distribution's."""
    import torch
    from paper_2405_06997_gb300 import wfpg as W
    rng = np.random.default_rng(args.seed + 100)
    pts = rng.uniform(0.25, 0.75, (n_probes, 3)).astype(np.float32)
    pr = W.Frame(svo, w.scene, eye=(0.5, 0.5, 0.05), max_depth=4, rr_depth=2, alpha=0.0, l_min=2, c_ray=512, N=16,
                 seed=args.seed + 7, update=False, nee=True, probes=pts, probe_n=N)
    pr.run(ref_frames)
    ref = pr.image()[0].double().cpu().numpy().reshape(n_probes, N * N)
    pos = torch.from_numpy(pts).cuda()
    pdf, _, _ = W.guide_build_pdf(svo, pos, None, None, n_probes, N=N, jitter=False, blur=True, eps=1e-2)
    p = pdf.double().cpu().numpy()

    def kl(q, p):
        q = q / q.sum(axis=1, keepdims=True)
        p = p / p.sum(axis=1, keepdims=True)
        m = q > 0
        return float(np.sum(np.where(m, q * np.log(np.where(m, q, 1.0) / p), 0.0)) / q.shape[0])

    return {"probes": n_probes, "N": N, "reference_frames": ref_frames,
            "kl_reference_to_traced": kl(ref, p), "kl_reference_to_uniform": kl(ref, np.ones_like(ref)),
            "note": "incident radiance per octahedral cell path-traced at free-space points (probe camera) "
                    "against the SVO-traced field of the cache after the timed frames"}


def city_section(args):
    """The large configuration: procedural city (5000 boxes, 50 area lights,
    S = 500), SVO depth 11 (2048^3), 3840x2160, 4 guided bounces, closest hits
    by the SVO walk, 64 x 64 traced fields; the learned proposal trained online
    on the city's traced fields, used or replaced by the traced field by the
    fallback rule; both proposals mixed 50/50 with cosine (BSDF) sampling."""
    import torch
    from paper_2405_06997_gb300 import inputs, learned as LG, wfpg as W
    sc = inputs.city(args.seed)
    q = torch.from_numpy(np.ascontiguousarray(sc.quads)).cuda()
    sp = torch.from_numpy(np.ascontiguousarray(sc.spheres)).cuda()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    svo = W.svo_build(q, sp, sc.lo, sc.size, 11)
    b.record()
    b.synchronize()
    build_ms = a.elapsed_time(b)
    cam = dict(eye=(250.0, 100.0, -50.0), forward=(0.0, -0.31622777, 0.9486833), up=(0.0, 0.9486833, 0.31622777),
               vfov=60.0, width=3840, height=2160, max_depth=4, rr_depth=2, alpha=0.5, l_min=2, c_ray=512,
               seed=args.seed, caster=2)
    out = {"workload": "city (5000 boxes log-U[0.5, 20], 50 area lights, S 500), SVO depth 11, camera at "
                       "(250, 100, -50) looking down 18.4 deg, vfov 60, 3840x2160, 4 guided bounces, RR from "
                       "vertex 2, alpha 0.5, Partition-S l_min 2 c_ray 512, closest hits by the SVO walk",
           "svo_build_ms": build_ms, "svo_nodes": svo.n_nodes, "svo_leaves": int(svo.level_off[12] - svo.level_off[11])}
    # the traced proposal (64 x 64) warms the cache, then is timed
    f = W.Frame(svo, sc, N=64, **cam)
    f.run(4)
    f.reset_image()
    torch.cuda.synchronize()

    def timed(frame, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        frame.reset_image()
        e0.record()
        frame.run(n)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / n
        st = frame.stats()
        m, v = frame.image()
        return {"ms_per_frame": ms, "guided_samples_per_s": st["guided_samples"] / (ms * n / 1e3),
                "paths_per_depth": st["paths"], "bins_per_depth": st["bins"], "records_per_frame": st["records"],
                "mean_pixel_variance": float(v.double().mean()), "mean_radiance": float(m.double().mean()),
                "status": st["status"], "graph_kernels_per_frame": st["kernels_per_frame"]}

    out["svo_traced_64"] = timed(f, args.city_frames)
    # the learned proposal: trained online against traced 32 x 32 fields at the frame's own
    # guided points (its first-depth queue: the camera hits that continue)
    f1 = W.Frame(svo, sc, N=64, max_depth=1, update=False, **{k: v for k, v in cam.items() if k != "max_depth"})
    f1.run(1, use_graph=False)
    n1 = f1.stats()["paths"][0]
    pts = (f1.export("q_pos")[:n1].clone(), f1.export("q_nrm")[:n1].clone())
    del f1
    tr = LG.OnlineTrainer(svo, sc, batch=65536, lr=1e-3, seed=args.seed, points=pts)
    t0 = time.perf_counter()
    tr.train(args.city_train_steps)
    train_s = time.perf_counter() - t0
    kl = tr.heldout_kl()
    tau = 1.5 * LG.traced_frame_kl(tr)
    fl = W.Frame(svo, sc, N=32, proposal=1, **cam)
    fl.set_mlp(tr.mlp, sc.lo, sc.size)
    fl.run(2)
    out["learned_32"] = timed(fl, args.city_frames)
    del fl
    # the MLP costs a few hundred kFLOP per bin: finer bins (c_ray 128) at little cost
    ff = W.Frame(svo, sc, N=32, proposal=1, **dict(cam, c_ray=128))
    ff.set_mlp(tr.mlp, sc.lo, sc.size)
    ff.run(2)
    out["learned_32_fine"] = dict(timed(ff, args.city_frames), c_ray=128)
    del ff
    use = LG.use_learned(kl, tau)
    out["learned_training"] = {"steps": args.city_train_steps, "batch_bins": 65536, "seconds": train_s,
                               "heldout_kl": kl, "fallback_threshold": tau, "uses_learned": use}
    out["chosen"] = "learned" if use else "svo_traced (fallback)"
    return out


def large_field_records(w, svo, inp, binout, B, peak, l2_peak, flush, reps=10):
    """guide_build_pdf on the 1080p workload's bins at N = 64 and 128 (the paper's
    first-depth resolutions): mean CUDA-event time of `reps` launches (L2
    flushed before each), cone rays/s, and the roofline of its algorithmic bytes
    (the oracle's block counts at that N) against HBM and the measured L2."""
    import torch
    from paper_2405_06997_gb300 import wfpg as W
    out = {}
    dev = inp["ray_pos"].device
    for N in (64, 128):
        guide = (torch.empty((B, N * N), dtype=torch.float32, device=dev),
                 torch.empty((B, N * N), dtype=torch.float32, device=dev),
                 torch.empty((B, N), dtype=torch.float32, device=dev))
        for k in range(3):
            W.guide_build_pdf(svo, inp["ray_pos"], binout["origin_ray"], binout["n_bins"], B, N=N, jitter=True,
                              blur=True, seed=w.seed, frame=9000 + k, out=guide)
        ms = []
        for k in range(reps):
            flush.zero_()
            a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            W.guide_build_pdf(svo, inp["ray_pos"], binout["origin_ray"], binout["n_bins"], B, N=N, jitter=True,
                              blur=True, seed=w.seed, frame=9100 + k, out=guide)
            b2.record()
            b2.synchronize()
            ms.append(a.elapsed_time(b2))
        m = statistics.mean(ms)
        alg = trace_algorithmic_bytes(w, B, N)
        ach = alg["bytes"] / (m / 1e3) / 1e9
        out[f"N{N}"] = {"ms": m, "cone_rays_per_s": B * N * N / (m / 1e3),
                        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                     "l2_peak": l2_peak, "l2_frac": ach / l2_peak, "algorithmic_bytes": alg["bytes"],
                                     "algorithmic_model": alg["model"]},
                        "kernels": "k_guide_stream (cone rays of every bin as 32-cell batches) + k_field_pdf (blur, CDFs, PDF)"}
    return out


def stage_rooflines(stage_ms, trace_bytes, R, n_rec, n_nodes, peak):
    """Mean CUDA-event time of each call of the step, its algorithmic bytes and
    the achieved fraction of the measured HBM bandwidth (bytes per unit:
    accumulate 40 B per record (28 B read + 12 B atomics) + 48 B per node for the
    bottom-up average; run-mode binning 92 B per ray (pos + normal 24, keys 8,
    3 radix passes x 16, order + bin id 12); the field kernel as modelled in the
    roofline object; sampling 32 B and evaluation 20 B per ray)."""
    model = {"accumulate": 40.0 * n_rec + 48.0 * n_nodes, "bin_rays": 92.0 * R, "guide_build_pdf": trace_bytes,
             "guide_sample": 32.0 * R, "guide_eval_pdf": 20.0 * R}
    out = {}
    for name, ts in stage_ms.items():
        ms = statistics.mean(ts)
        gbs = model[name] / (ms / 1e3) / 1e9
        out[name] = {"ms": ms, "algorithmic_bytes": model[name], "GB_s": gbs, "frac": gbs / peak}
    return out


def trace_algorithmic_bytes(w, B, N, sample_bins=8):
    """Bytes the field kernel must move for one launch: its outputs (pdf,
    cdf_row, cdf_marg: B (2 N^2 + N) 4 B) plus, per cone ray, one 8-byte node
    record per block the walk passes (the oracle counts the maximal empty
    blocks and leaves on a sample of bins) and the hit node's normal and values
    (16 + 8 B)."""
    import oracle
    s = oracle.SVO(w.scene, w.depth)
    b = s.bin_rays(w.ray_pos, w.ray_nrm, mode=1, sizes=w.bin_sizes, seed=w.seed, frame=0)
    sel = np.linspace(0, b["n_bins"] - 1, sample_bins).astype(np.int64)
    g = s.guide_build(w.ray_pos[b["origin_ray"][sel]], sel, N, jitter=True, blur=True, seed=w.seed,
                      count_blocks=True)
    blocks_per_ray = g["blocks"] / (len(sel) * N * N)
    per_ray = 8.0 * blocks_per_ray + 24.0
    total = B * (2 * N * N + N) * 4 + B * N * N * per_ray
    return {"bytes": total, "model": f"outputs B(2N^2+N)*4 + cone rays x (8 B x {blocks_per_ray:.2f} "
                                     f"blocks + 24 B); blocks counted by the oracle on {len(sel)} bins"}


def issue_roofline(counters, kernel_ms, sm_mhz, n_sm, schedulers=4):
    """Instruction-issue roofline of the field kernel, beside its HBM one:
    the warp instructions of one launch (the committed ncu capture of the same
    source and workload) over the launch's mean CUDA-event duration in the
    timed steps, against one warp instruction per scheduler per cycle (SMs x 4
    schedulers x the SM clock sampled during the timed steps).  lane_frac
    weighs each issued instruction by its active lanes out of 32.  None when
    a figure is missing."""
    if not counters or not kernel_ms or not sm_mhz or not n_sm:
        return None
    inst = counters.get("warp_instructions_per_launch")
    lanes = counters.get("active_lanes_per_warp_instruction")
    if inst is None or lanes is None:
        return None
    achieved = inst / (kernel_ms * 1e-3) / 1e9
    peak = n_sm * schedulers * sm_mhz * 1e6 / 1e9
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "G warp instructions/s",
            "frac": achieved / peak, "lane_frac": achieved * lanes / (peak * 32.0),
            "peak_model": f"{n_sm} SMs x {schedulers} schedulers x 1 warp instruction per cycle x {sm_mhz:.0f} MHz"}


def read_profile_traffic():
    """DRAM bytes per launch of the field kernel (k_guide_stream) and its issue
    counters from the committed ncu summary -- only while the kernel source is
    the one captured."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_guide_stream_frame1080p.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as f:
        d = json.load(f)
    with open(os.path.join(ROOT, d["source"]), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest() != d["source_sha256"]:
            return None, None
    return d["dram_bytes_per_launch"], {"issue_active_pct": d["issue_active_pct"],
                                        "active_lanes_per_warp_instruction": d["active_lanes_per_warp_instruction"],
                                        "warp_instructions_per_launch": d["warp_instructions_per_launch"],
                                        "limiter": "instruction issue and latency with divergence (DRAM well below peak)"}


def l2_read_peak(dev, mib=32, reps=40, trials=5):
    """L2 read bandwidth of this GPU, measured here: wfpg_stream_read over an
    L2-resident buffer (reads through L2 only), best of `trials` launches,
    bytes read / CUDA-event time."""
    import torch
    from paper_2405_06997_gb300 import wfpg as W
    buf = torch.ones(mib << 18, dtype=torch.float32, device=dev)
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    blocks = 4 * torch.cuda.get_device_properties(dev).multi_processor_count
    W.stream_read(buf, 2, sink, blocks)
    best = None
    for _ in range(trials):
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        W.stream_read(buf, reps, sink, blocks)
        b2.record()
        b2.synchronize()
        ms = a.elapsed_time(b2)
        best = ms if best is None else min(best, ms)
    return (mib << 20) * reps / (best / 1e3) / 1e9, f"wfpg_stream_read: {mib} MiB buffer x {reps} passes through L2, " \
        f"{blocks} blocks of 512 threads, best of {trials}"


def main():
    args = parse()
    world, rank, local = dist_init(args.gpus)
    if args.city_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(city_section(args)))
    elif args.mesh_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(mesh_section(args)))
    elif args.batched_only:
        import torch
        torch.cuda.set_device(local)
        print(json.dumps(batched_section(args, autotune=False)))
    elif args.l2_peak_only:
        import torch
        torch.cuda.set_device(local)
        sweep = {}
        for mib, reps in ((8, 160), (16, 80), (32, 40), (64, 20), (2048, 2)):
            gbs, how = l2_read_peak(local, mib=mib, reps=reps)
            sweep[f"{mib}MiB"] = {"GB_s": gbs, "how": how}
        print(json.dumps({"l2_read_peak": sweep, "note": "buffers up to 64 MiB stay in the 126 MB L2; "
                          "the 2 GiB buffer streams from HBM"}))
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
