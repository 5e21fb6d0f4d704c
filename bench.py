#!/usr/bin/env python
"""Benchmark of the multislice forward model + adjoint (one loss-gradient
evaluation) on synthetic CSSI volumes.

Workload (one step): 512 x 512 (y, z) grid at 2 nm, 1024 slices of 20 nm,
9 incidence angles 0.10-0.50 deg through one volume, Si substrate with 50 Au
pillars/lines, amplitude loss against Poisson targets (1e6 counts per angle),
gradient on delta/beta with checkpoints every 32 slices.

Metric: voxel-slice-steps/s, one unit = one grid point of one wavefield taken
through one slice forward AND back (ny*nz*ns*nw units per step).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Under torchrun each rank runs its own volume (seed = rank): weak scaling, no
data-path collective; the JSON line (rank 0) reports the whole-job rate.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

NY = NZ = 512
NS = 1024
NW = 9
DZ = DY = 2.0
SLICE = 20.0
LAM = 0.155
COUNTS = 1e6
CKPT = 32
METRIC = "multislice voxel-steps/s fwd+adjoint"
UNIT = "voxel-slice-steps/s"
HBM_BYTES_PER_UNIT = 48      # minimum HBM bytes per voxel-slice-step of loss + gradient


def config(nw=NW, ns=NS, ckpt=CKPT):
    return {
        "workload": "512x512 grid (2 nm), %d slices of 20 nm, %d incidence angles 0.10-0.50 deg, "
                    "Si + 50 Au pillars/lines, loss + gradient (checkpoint every %d slices%s)"
                    % (ns, nw, ckpt, ": every a_j kept, no recompute" if ckpt >= ns else ""),
        "grid": [NY, NZ], "slices": ns, "angles": nw, "wavelength_nm": LAM,
        "l2": "inputs larger than L2: the 2 GiB volume and 2 GiB transmission stream from HBM every pass",
    }


def checkpoint_interval(args, ny, nz, ns, nw, dev):
    """Adjoint checkpoint interval: --checkpoint if given, else every a_j kept
    (one segment, no recompute) when that workspace fits in half of the
    device's memory, else every 32 slices."""
    import torch

    from paper_2212_01253_gb300 import binding as B
    if args.checkpoint > 0:
        return args.checkpoint
    total = torch.cuda.get_device_properties(dev).total_memory
    need = B.mslice_workspace_size(B.make_params(ny, nz, ns, angles(nw), checkpoint_every=ns),
                                   B.MSLICE_OP_LOSS_GRAD)
    return ns if need + 4 * ny * nz * ns * 8 <= total // 2 else CKPT


def angles(nw=NW):
    return np.linspace(0.1, 0.5, nw)


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# algorithmic work per unit (FFT flops counted as 5 N log2 N per length-N
# complex transform, complex multiply 6, per grid point per slice)
# ---------------------------------------------------------------------------
def flops_per_unit(kernel, ny=NY, nz=NZ):
    fft_pair = 2 * 5 * (np.log2(ny) + np.log2(nz))  # forward + inverse along y and z
    if kernel == "k_fwd":
        return 6 + fft_pair + 12                   # transmission, FFTs, P_y and P_z
    if kernel == "k_adj":
        return 6 + fft_pair + 12 + 8               # + gradient a conj(g) scaled
    if kernel == "k_last":
        return 6 + 5 * (np.log2(ny) + np.log2(nz)) * 2 + 20
    return 0.0


def fp32_peak_tflops(sms, mhz):
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


SWEEP_SOURCES = ("mslice_device.cuh", "mslice_slice.cuh", "mslice_inst.cu", "mslice_kernels.h", "mslice_generic.cu")


def source_hash():
    """Hash of the sources of the slice-loop kernels (the ncu traffic record is
    void once they change)."""
    h = hashlib.sha256()
    for f in SWEEP_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2212_01253_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record(kernel):
    """DRAM bytes per unit from a committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
        h = source_hash()
        if rec.get("source_sha256_16") != h:
            return None
        return rec["kernels"].get(kernel, {}).get("dram_bytes_per_unit")
    except (OSError, ValueError, KeyError):
        return None


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def oracle_rate(ns_sample, nangles=1, reps=1):
    """Oracle loss+gradient on 512^2 x ns_sample slices x nangles angles; units per run."""
    import cssi_inputs as ci
    import oracle

    geo = oracle.Geometry(NY, NZ, ns_sample, LAM, SLICE, DY, DZ,
                          alpha_i_deg=np.linspace(0.1, 0.5, nangles) if nangles > 1 else (0.3,))
    vol = ci.pillars_large(0, ns=ns_sample)
    meas = np.ones((nangles, NZ, NY), np.float64)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.loss_grad(geo, vol, meas, 1.0)
        times.append(time.perf_counter() - t0)
    units = NY * NZ * ns_sample * nangles
    return units, times, oracle.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    ns_sample = 256
    units, times, cores = oracle_rate(ns_sample, reps=args.warmup + args.steps)
    timed = times[args.warmup:]
    per_step = sum(timed) / len(timed)
    value = units / per_step
    sample = "512x512 grid, %d of 1024 slices, 1 of 9 angles per step (FP64 oracle loss+gradient)" % ns_sample
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(ckpt=NS),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300 import build as cuda_build
    from paper_2212_01253_gb300.shard import whole_job_rate

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    nw, ns = args.angles, args.slices
    ckpt = checkpoint_interval(args, NY, NZ, ns, nw, dev)
    p = B.make_params(NY, NZ, ns, angles(nw), LAM, SLICE, DY, DZ, ckpt,
                      flags=B.MSLICE_ANGULAR if args.angular else 0)
    if not args.no_tune:
        # launch shape (blocks, column-group width, schedule) from the autotuner,
        # tuned once per device and shape outside the timed region, cached on disk
        from paper_2212_01253_gb300 import autotune
        autotune.apply(p, dev)

    # inputs: volume (seed = rank) and Poisson targets of a ground-truth volume
    vol_h = ci.pillars_large(rank, ns=ns)
    truth_h = ci.pillars_large(1000 + rank, ns=ns)
    vol = torch.from_numpy(vol_h).to(dev)
    ws = torch.empty(B.mslice_workspace_size(p, B.MSLICE_OP_LOSS_GRAD), dtype=torch.uint8, device=dev)
    inten = torch.empty((nw, NZ, NY), dtype=torch.float32, device=dev)
    B.mslice_forward(p, torch.from_numpy(truth_h).to(dev), None, inten, None, ws)
    I_gt = inten.cpu().numpy()
    meas_h = np.empty_like(I_gt, dtype=np.float32)
    scales = []
    for w in range(nw):
        m, s = ci.poisson_target(I_gt[w], COUNTS, seed=rank * 100 + w)
        meas_h[w] = m
        scales.append(s)
    # one scale for all angles: the flux is the same, so use their mean
    s = float(np.mean(scales))
    meas = torch.from_numpy(meas_h).to(dev)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grad = torch.empty_like(vol)
    stream = torch.cuda.current_stream()

    def step():
        B.mslice_loss_grad(p, vol, None, meas, s, loss, grad, None, ws)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if B.mslice_status(ws) != 0:
        raise RuntimeError("device-side wait timed out during warm-up")
    if world > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.1)
    B.mslice_profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof = B.mslice_profile_read()
    B.mslice_profile_enable(False)
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if B.mslice_status(ws) != 0:
        raise RuntimeError("device-side wait timed out in the timed region")
    units_step = NY * NZ * ns * nw
    value, ms_max = whole_job_rate(units_step, ms, dev)

    # the same step with a checkpoint every 32 slices and segment recompute
    # (the schedule that keeps deep stacks small: ns/32 + 32 fields instead of
    # every a_j), timed the same way
    ck32 = None
    if not args.no_ckpt32 and ckpt != 32 and world == 1:
        p32 = B.make_params(NY, NZ, ns, angles(nw), LAM, SLICE, DY, DZ, 32,
                            flags=B.MSLICE_ANGULAR if args.angular else 0)
        p32.grid_blocks, p32.col_width, p32.schedule = p.grid_blocks, p.col_width, p.schedule
        ws32 = torch.empty(B.mslice_workspace_size(p32, B.MSLICE_OP_LOSS_GRAD), dtype=torch.uint8, device=dev)
        loss32 = torch.zeros(1, dtype=torch.float64, device=dev)

        def step32():
            B.mslice_loss_grad(p32, vol, None, meas, s, loss32, grad, None, ws32)

        for _ in range(3):
            step32()
        n32 = max(3, min(args.steps, 5))
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n32):
            step32()
        e1.record(stream)
        torch.cuda.synchronize()
        if B.mslice_status(ws32) != 0:
            raise RuntimeError("device-side wait timed out in the checkpoint-32 leg")
        ms32 = e0.elapsed_time(e1) / n32
        ck32 = {"checkpoint_every": 32, "ms_per_step": ms32, "value": units_step / (ms32 / 1e3), "unit": UNIT,
                "steps": n32, "warmup": 3, "ratio_to_headline": ms32 / ms,
                "workspace_gb": ws32.numel() / 1e9, "headline_workspace_gb": ws.numel() / 1e9,
                "loss_matches_headline": bool(abs(float(loss32.item()) - float(loss.item()))
                                              <= 1e-12 * abs(float(loss.item())))}
        del ws32

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # end to end from pinned host memory through the public API: every step
        # copies its volume and targets in and its gradient and loss out; the
        # copies of one step overlap the slice loop of its neighbours
        # (HostPipeline: copy-in, compute and copy-out streams, two device
        # slots; three, which let a step's copy-in and the previous step's
        # copy-out run at once, measured no faster)
        from paper_2212_01253_gb300.pipeline import HostPipeline
        pipe = HostPipeline(p, s, dev, slots=2)
        vol_pin = torch.from_numpy(vol_h).pin_memory()
        meas_pin = torch.from_numpy(meas_h).pin_memory()
        grad_pin = [torch.empty(grad.shape, dtype=grad.dtype).pin_memory() for _ in range(2)]
        loss_pin = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
        for k in range(len(pipe.slots)):
            pipe.submit(vol_pin, meas_pin, grad_pin[k % 2], loss_pin[k % 2])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(pipe.s_in)
        for k in range(args.steps):
            pipe.submit(vol_pin, meas_pin, grad_pin[k % 2], loss_pin[k % 2])
        f1.record(pipe.s_out)
        torch.cuda.synchronize()
        if pipe.status() != 0:
            raise RuntimeError("device-side wait timed out in the end-to-end leg")
        e_value, e_ms = whole_job_rate(units_step, f0.elapsed_time(f1) / args.steps, dev)
        e2e = {"value": e_value, "unit": UNIT,
               "h2d_bytes_per_step": vol_pin.numel() * 8 + meas_pin.numel() * 4,
               "d2h_bytes_per_step": grad_pin[0].numel() * 8 + 8,
               "ms_per_step": e_ms,
               "api": "HostPipeline.submit (mslice_loss_grad with copies on their own streams, 2 device slots)",
               "loss_matches_device_leg": bool(abs(float(loss_pin[(args.steps - 1) % 2].item()) - float(loss.item()))
                                               <= 1e-9 * abs(float(loss.item())))}
        del pipe

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    # roofline of the dominant kernel
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    name, (launches, total_ms, units) = dom
    flops = flops_per_unit(name) * units / launches
    launch_s = total_ms / launches / 1e3
    achieved = flops / launch_s / 1e12
    peak = fp32_peak_tflops(sms, mhz)
    tb = traffic_record(name)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None if tb is None else tb * units / launches,
                "kernel": name, "launches": launches, "avg_launch_ms": total_ms / launches,
                "peak_basis": "FP32 FMA rate: %d SMs x 128 lanes x 2 flop x %.0f MHz (of measured "
                              "sm_max_mhz)" % (sms, mhz),
                "flops_per_unit": flops_per_unit(name)}
    kernels = {k: {"launches": v[0], "total_ms": v[1], "units": v[2]} for k, v in prof.items()}
    gpu_launches = sum(v[0] for v in prof.values())
    # effective bandwidth of the whole step: the rate times the HBM bytes per
    # unit that one wavefield's loss + gradient needs when the field stays on
    # chip and the adjoint recomputes a_j from checkpoints (forward: volume 8;
    # recompute: volume 8, a_j stored 8; adjoint: a_j reloaded 8, volume 8,
    # gradient written 8), against the HBM copy rate.  The DRAM bytes that ncu
    # counted for the step's two slice-loop kernels are lower: the angles share
    # the volume and every a_j is kept, so nothing is recomputed.
    hbm_gbs = float(peaks.get("hbm_gbs", 6800.0))
    tf, ta = traffic_record("k_fwd"), traffic_record("k_adj")
    eff = value * HBM_BYTES_PER_UNIT / 1e9
    hbm = {"bytes_per_unit": HBM_BYTES_PER_UNIT, "effective": eff, "peak": hbm_gbs, "unit": "GB/s",
           "frac": eff / hbm_gbs, "peak_basis": "measured" if "hbm_gbs" in peaks else "fallback",
           "dram_bytes_per_unit_counted": None if tf is None or ta is None else tf + ta,
           "dram_gbs_counted": None if tf is None or ta is None else value * (tf + ta) / 1e9}

    cpu = None
    if not args.no_cpu_baseline:
        ns_sample, na = args.cpu_slices, args.cpu_angles
        u, times, cores = oracle_rate(ns_sample, nangles=na, reps=1)
        cpu = {"value": u / times[0], "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "512x512 grid, %d of 1024 slices, %d of 9 angles (FP64 oracle loss+gradient, "
                         "%.1f s)" % (ns_sample, na, times[0])}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config(nw, ns, ckpt), launch_shape={"grid_blocks": p.grid_blocks, "col_width": p.col_width,
                                                         "schedule": p.schedule},
                           propagator="angular spectrum" if args.angular else "paraxial (Eq. 1)"),
            "roofline": roofline, "effective_hbm": hbm, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": gpu_launches, "kernels": kernels, "loss": float(loss.item()),
            "checkpoint32": ck32,
            "recon": None if (args.no_recon or world > 1) else recon_leg(args, dev)}
    if not args.no_batch and world == 1:
        bl = batch_measure(args, dev)
        bl["of_headline"] = bl["value"] / value
        line["batch"] = bl
    else:
        line["batch"] = None
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# extra workloads (not the headline line): batched uneven jobs, reconstruction
# ---------------------------------------------------------------------------
def batch_measure(args, dev, world=1, rank=0):
    """Loss + gradient of the 64 uneven structures (this rank's share of
    them) as one CUDA-graph replay of mslice_loss_grad_batched; returns the
    whole-job rate and the details of the run."""
    import torch
    import torch.distributed as dist

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300.batch import BatchedLossGrad
    from paper_2212_01253_gb300.shard import shard, whole_job_rate

    all_specs = ci.batched_jobs(0, args.jobs)
    specs = [all_specs[i] for i in shard(len(all_specs), rank, world)]
    jobs = []
    t0 = time.perf_counter()
    for k, sp in enumerate(specs):
        ny, nz, ns = sp["ny"], sp["nz"], sp["ns"]
        vol = torch.from_numpy(ci.pillars_large(sp["seed"] % (1 << 20), ny=ny, nz=nz, ns=ns,
                                                count=max(4, ny * ns // 10000))).to(dev)
        p = B.make_params(ny, nz, ns, (sp["alpha_deg"],))
        ws = B.workspace(p, B.MSLICE_OP_FORWARD)
        inten = torch.empty((1, nz, ny), dtype=torch.float32, device=dev)
        B.mslice_forward(p, vol, None, inten, None, ws)
        del ws
        jobs.append(dict(vol=vol, meas=torch.sqrt(inten[0] * 1.05).contiguous(), scale=1.0,
                         alpha_deg=sp["alpha_deg"]))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    # checkpoint interval as for the headline: --checkpoint if given, else
    # every a_j kept (one segment per group, no recompute) when the batch's
    # workspace fits in half of the device's memory, else every 32 slices
    ckpt = args.checkpoint if args.checkpoint > 0 else 1 << 30
    if args.checkpoint <= 0:
        probe_jobs = B.make_jobs([dict(vol=jb["vol"], alpha_deg=jb["alpha_deg"], meas=jb["meas"], scale=1.0,
                                       grad=jb["vol"]) for jb in jobs])
        need = B.mslice_batched_workspace_size(B.make_params(64, 64, 1, checkpoint_every=ckpt), probe_jobs,
                                               B.MSLICE_OP_LOSS_GRAD, args.lanes)
        free, _ = torch.cuda.mem_get_info(dev)
        if need + sum(jb["vol"].numel() * 8 for jb in jobs) > free // 2:
            ckpt = CKPT
    bat = BatchedLossGrad(jobs, tune=not args.no_tune, lanes=args.lanes, checkpoint_every=ckpt, device=dev)
    bat.capture()
    for _ in range(args.warmup):
        bat.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        bat.replay()
    e1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    bat.check()
    value, ms = whole_job_rate(bat.units, e0.elapsed_time(e1) / args.steps, dev)
    # the same batch as eager calls (no graph) for comparison
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    for _ in range(args.steps):
        bat.run()
    f1.record()
    torch.cuda.synchronize()
    out = {"value": value, "unit": UNIT, "ms_per_step": ms, "eager_ms_per_step": f0.elapsed_time(f1) / args.steps,
           "workload": "%d structures, grids 128-512 per axis, 128-1024 slices, 0.1-0.5 deg, one CUDA graph "
                       "per rank" % len(all_specs),
           "checkpoint": "every a_j kept" if ckpt > 1024 else "every %d slices" % ckpt,
           "structures_rank0": len(jobs), "groups_rank0": bat.ngroups, "lanes": bat.lanes,
           "hw_queues": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8 (default)"),
           "api": "mslice_loss_grad_batched (one C call: grouping, lanes and launch sequences in the library)",
           "units_per_step_rank0": bat.units, "setup_s": setup_s, "steps": args.steps}
    del bat, jobs
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """64 independent structures of uneven shape (grids 128..512 per axis,
    128..1024 slices, 0.1-0.5 deg), loss + gradient of all of them as one
    CUDA-graph launch; voxel-slice-steps/s over the whole batch.  Under
    torchrun the structures are split between the ranks by index (strong
    scaling: the batch is fixed)."""
    import torch
    import torch.distributed as dist

    from paper_2212_01253_gb300 import build as cuda_build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0 or not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    if world > 1:
        dist.barrier()
    r = batch_measure(args, dev, world, rank)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    cfg = {k: r[k] for k in ("workload", "checkpoint", "structures_rank0", "groups_rank0", "lanes", "hw_queues",
                             "api", "units_per_step_rank0", "setup_s")}
    line = {"metric": "batched multislice voxel-steps/s fwd+adjoint", "value": r["value"],
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"], "eager_ms_per_step": r["eager_ms_per_step"],
            "higher_is_better": True, "scaling": "strong", "dtype": "f32", "data": "synthetic", "config": cfg}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def recon_leg(args, dev):
    """Reconstruction at 256x256x512 with a checkpoint every 32 slices: wall
    time to chi2_red <= 1.1 chi2_red(truth) of one held-out pillar layout from
    the learned start (network trained here on fresh forward-model samples,
    inference included) and from the zero start (bare substrate), each capped
    at args.recon_cap iterations."""
    import torch

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300.learned import ARCH_256, EncoderDecoder, PillarSampler, train
    from paper_2212_01253_gb300.recon import Reconstructor

    ny = nz = 256
    ns = 512
    shape, block, off = (64, 64, 64), (8, 2, 4), (0, 128, 0)
    p = B.make_params(ny, nz, ns, (0.3,), checkpoint_every=32)
    c = B.make_coarse(shape, block, off)
    base = torch.from_numpy(ci.substrate(ny, nz, ns)).to(dev)
    batch = 64
    sampler = PillarSampler(p, c, base, n_pillars=(4, 16), foot=(2, 9), height=(1, 9), chunk=args.chunk,
                            tune=not args.no_tune)
    net = EncoderDecoder(ARCH_256, batch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    train(net, sampler, args.recon_train_samples, batch, lr=1e-3, seed=1000)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    seed = 200000
    meas, sc, chi2_gt, _ = _pillar_case(B, ci, torch, p, c, base, sampler, seed)
    measd = torch.from_numpy(meas).to(dev)
    out = {}
    for name in ("learned", "zero"):
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        th0 = None if name == "zero" else net.predict(sampler.features_of(measd)).reshape(-1).contiguous()
        torch.cuda.synchronize()
        t_init = time.perf_counter() - t1
        R = Reconstructor(p, c, base, measd, sc, theta0=th0, lr=args.lr)
        it, sec, hist = R.run(chi2_target=1.1 * chi2_gt, max_iters=args.recon_cap, check_every=5)
        out[name] = {"seconds": t_init + sec, "iterations": it,
                     "reached": bool(hist and hist[-1][1] <= 1.1 * chi2_gt),
                     "chi2_start": hist[0][1] if hist else None, "chi2_end": hist[-1][1] if hist else None,
                     "ms_per_iteration": 1e3 * sec / it, "init_seconds": t_init}
    ratio = out["zero"]["seconds"] / out["learned"]["seconds"]
    return {"metric": "recon wall time to chi2_red <= 1.1 chi2_red(truth)", "unit": "s",
            "chi2_truth": chi2_gt, "target": 1.1 * chi2_gt, "cap_iterations": args.recon_cap,
            "learned": out["learned"], "zero": out["zero"],
            "zero_over_learned": ratio,
            "ratio_kind": ("measured (both reached the target)" if out["zero"]["reached"] and out["learned"]["reached"]
                           else "lower bound (the zero start did not reach the target within the cap)"
                           if out["learned"]["reached"] else "learned start did not reach the target"),
            "training": {"samples": args.recon_train_samples, "seconds": t_train, "batch": batch},
            "config": {"workload": "256x256 grid (2 nm), 512 slices of 20 nm, 0.3 deg, checkpoint every 32 "
                                   "slices; 64^3 coarse delta (8x2x4 fine voxels, top half); held-out layout of "
                                   "4-16 Au pillars (seed %d), Poisson target 1e6 counts; ADAM lr %g"
                                   % (seed, args.lr)}}


def run_recon(args):
    """Reconstruction of a coarse 64^3 Au occupancy on a 256x256x512 grid from a
    Poisson target (1e6 counts): iterations and wall time until the reduced
    chi^2 reaches 1.1x that of the ground truth (or the iteration cap)."""
    import torch

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300 import build as cuda_build
    from paper_2212_01253_gb300.recon import Reconstructor

    cuda_build.build()
    torch.cuda.set_device(0)
    ny = nz = 256
    ns = 512
    shape, block, off = (64, 64, 64), (8, 2, 4), (0, 128, 0)
    # one angle (0.3 deg), or a joint reconstruction over several incidence angles
    # sharing the volume (loss and gradient summed over the views)
    ang = (0.3,) if args.recon_angles <= 1 else tuple(np.linspace(0.1, 0.5, args.recon_angles))
    nw = len(ang)
    # in-plane angle of each view: 0, or swept over [-recon_psi, recon_psi] deg
    psi = np.deg2rad(np.linspace(-args.recon_psi, args.recon_psi, nw)) if nw > 1 else np.zeros(1)
    p = B.make_params(ny, nz, ns, ang, checkpoint_every=ns, psi_rad=psi)   # every a_j kept
    c = B.make_coarse(shape, block, off)
    rng = np.random.default_rng(0)
    truth = np.zeros(shape, np.float32)
    for _ in range(16):   # 16 Au pillars in coarse space, 1-8 coarse voxels tall
        a0, c0 = rng.integers(0, 56), rng.integers(0, 56)
        la, lc, h = rng.integers(2, 9), rng.integers(2, 9), rng.integers(1, 9)
        truth[a0:a0 + la, :h, c0:c0 + lc] = 4.7e-5
    base = torch.from_numpy(ci.substrate(ny, nz, ns)).cuda()
    vol_gt = base.clone()
    B.mslice_coarse_to_fine(p, c, torch.from_numpy(truth.ravel()).cuda(), vol_gt)
    ws = B.workspace(p, B.MSLICE_OP_FORWARD)
    inten = torch.empty((nw, nz, ny), dtype=torch.float32, device="cuda")
    B.mslice_forward(p, vol_gt, None, inten, None, ws)
    I_gt = inten.cpu().numpy().astype(np.float64)
    meas = np.empty(I_gt.shape, np.float32)
    scales = []
    for w in range(nw):                      # 1e6 counts per view
        meas[w], sw = ci.poisson_target(I_gt[w], COUNTS, seed=w)
        scales.append(sw)
    s = float(np.mean(scales))               # views differ in total intensity by < 1e-3 (absorption)
    chi2_gt = 4 * ((np.sqrt(s * I_gt) - meas) ** 2).sum() / meas.size
    R = Reconstructor(p, c, base, torch.from_numpy(meas).cuda(), s, lr=args.lr)
    it, sec, hist = R.run(chi2_target=1.1 * chi2_gt, max_iters=args.max_iters, check_every=5)
    occ = R.theta.cpu().numpy().reshape(shape) / 4.7e-5
    line = {"metric": "reconstruction wall time to chi2_red <= 1.1 chi2_red(truth)", "value": sec, "unit": "s",
            "higher_is_better": False, "reached": bool(hist and hist[-1][1] <= 1.1 * chi2_gt), "iterations": it,
            "ms_per_iteration": 1e3 * sec / it, "chi2_truth": chi2_gt, "chi2_start": hist[0][1] if hist else None,
            "chi2_end": hist[-1][1] if hist else None,
            "occupancy_error": float(np.abs(occ - truth / 4.7e-5).mean()),
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256x256 grid, 512 slices, %s, 64^3 coarse delta (8x2x4 fine voxels each, "
                                   "top half), Poisson targets 1e6 counts per view, zero (bare substrate) start, "
                                   "ADAM lr %g" % ("%d views %.2f-%.2f deg, in-plane %+.2f..%+.2f deg"
                                                   % (nw, ang[0], ang[-1], -args.recon_psi, args.recon_psi)
                                                   if nw > 1 else "0.3 deg", args.lr)}}
    print(json.dumps(line), flush=True)
    return 0


def run_buried(args):
    """Sec. 4.1's reconstruction on synthetic data: 6x6x6 coarse voxels, each Si
    or Au, buried 10 nm under the Si surface, 0.5 deg incidence; ADAM from pure
    silicon with material snapping every 20 epochs, until chi2_red <= 1.1
    chi2_red(truth) or the epoch cap."""
    import torch

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300 import build as cuda_build
    from paper_2212_01253_gb300.recon import Reconstructor

    cuda_build.build()
    torch.cuda.set_device(0)
    ny = nz = 256
    ns = 512
    surf = nz // 2
    shape, block = (6, 6, 6), (80, 8, 40)                   # 1.6 um x 16 nm x 80 nm per coarse voxel
    off = (16, surf - 5 - 6 * 8, 8)                         # top of the pattern 5 rows (10 nm) below the surface
    d_au = ci.AU.real - ci.SI.real
    ratio = (ci.AU.imag - ci.SI.imag) / d_au
    p = B.make_params(ny, nz, ns, (0.5,), checkpoint_every=ns)
    c = B.make_coarse(shape, block, off, beta_ratio=ratio, base=ci.SI)
    base = torch.from_numpy(ci.substrate(ny, nz, ns)).cuda()
    rows = []
    for seed in range(args.heldout if args.heldout < 10 else 3):
        rng = np.random.default_rng(seed)
        truth = (rng.random(shape) < 0.35).astype(np.float32) * d_au
        if args.buried_extrude:               # the same (z, y) pattern in every cell along the beam
            truth[:] = truth[0]
        vol_gt = base.clone()
        B.mslice_coarse_to_fine(p, c, torch.from_numpy(truth.ravel()).cuda(), vol_gt)
        ws = B.workspace(p, B.MSLICE_OP_FORWARD)
        inten = torch.empty((1, nz, ny), dtype=torch.float32, device="cuda")
        B.mslice_forward(p, vol_gt, None, inten, None, ws)
        I_gt = inten.cpu().numpy().astype(np.float64)
        meas, sc = ci.poisson_target(I_gt, COUNTS, seed=seed)
        chi2_gt = 4 * ((np.sqrt(sc * I_gt) - meas) ** 2).sum() / meas.size
        R = Reconstructor(p, c, base, torch.from_numpy(meas).cuda(), sc, lr=args.lr, lo=0.0, hi=d_au,
                          snap_every=args.snap_every, snap_levels=(0.0, d_au), snap_start=args.snap_start,
                          shrinkwrap_every=args.shrinkwrap_every, shrinkwrap_sigma=args.shrinkwrap_sigma,
                          shrinkwrap_threshold=args.shrinkwrap_threshold)
        it, sec, hist = R.run(chi2_target=1.1 * chi2_gt, max_iters=args.max_iters, check_every=20)
        th = R.theta.cpu().numpy().reshape(shape)
        rows.append({"seed": seed, "reached": bool(hist and hist[-1][1] <= 1.1 * chi2_gt), "epochs": it,
                     "seconds": sec, "chi2_truth": chi2_gt, "chi2_start": hist[0][1] if hist else None,
                     "chi2_end": hist[-1][1] if hist else None,
                     "voxels_correct": int(((th > d_au / 2) == (truth > d_au / 2)).sum()),
                     "au_voxels": int((truth > 0).sum())})
    line = {"metric": "buried-pattern reconstruction: epochs and wall time to chi2_red <= 1.1 chi2_red(truth)",
            "value": statistics.median(r["seconds"] for r in rows), "unit": "s", "higher_is_better": False,
            "reached": "%d/%d" % (sum(r["reached"] for r in rows), len(rows)), "per_seed": rows,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256x256 grid (2 nm), 512 slices of 20 nm, 0.5 deg; 6x6x6 coarse voxels "
                                   "(1.6 um x 16 nm x 80 nm) of Si or Au buried 10 nm under the Si surface, "
                                   "35 %% Au%s; Poisson target 1e6 counts; start pure Si; ADAM lr %g, snapping "
                                   "to {Si, Au} every %d epochs from epoch %d; shrink-wrap every %d epochs "
                                   "(sigma %g, threshold %g); cap %d epochs"
                                   % (", uniform along the beam" if args.buried_extrude else "", args.lr,
                                      args.snap_every, args.snap_start, args.shrinkwrap_every,
                                      args.shrinkwrap_sigma, args.shrinkwrap_threshold, args.max_iters)}}
    print(json.dumps(line), flush=True)
    return 0


def _pillar_case(B, ci, torch, p, c, base, sampler, seed):
    """Held-out ground truth: one sampler layout of ``seed``, its intensity and
    a Poisson target (1e6 counts); returns (meas, s, chi2_truth, occupancy)."""
    _, occ, theta = sampler.sample(np.random.default_rng(seed), 1, noise=False)
    vol = base.clone()
    B.mslice_coarse_to_fine(p, c, theta.reshape(-1).contiguous(), vol)
    ws = B.workspace(p, B.MSLICE_OP_FORWARD)
    inten = torch.empty(p.nz * p.ny, dtype=torch.float32, device=base.device)
    B.mslice_forward(p, vol, None, inten, None, ws)
    I_gt = inten.cpu().numpy().astype(np.float64).reshape(p.nz, p.ny)
    meas, s = ci.poisson_target(I_gt, COUNTS, seed=seed)
    chi2_gt = 4 * ((np.sqrt(s * I_gt) - meas) ** 2).sum() / meas.size
    return meas, s, chi2_gt, occ


def network_step_flops(net, nb):
    """FLOPs of one training step of the network (forward, dW, db, dX GEMMs)."""
    f = 0
    for i, L in enumerate(net.layers):
        rows = net._rows(L, nb)
        f += 2 * rows * L["N"] * L["K"] * (3 if i else 2) + 2 * rows * L["N"]
    return f


def run_learned(args):
    """Learned initialiser vs zero and constant starts: train the encoder-decoder
    on forward-model samples (256x256 detector -> 64^3 coarse delta, 4.47M
    parameters), then reconstruct held-out pillar layouts from each start until
    chi2_red <= 1.1 chi2_red(truth) or the iteration cap."""
    import torch

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300 import build as cuda_build
    from paper_2212_01253_gb300.learned import ARCH_256, AU_DELTA, EncoderDecoder, PillarSampler, train
    from paper_2212_01253_gb300.recon import Reconstructor

    cuda_build.build()
    torch.cuda.set_device(0)
    ny = nz = 256
    ns = 512
    shape, block, off = (64, 64, 64), (8, 2, 4), (0, 128, 0)
    p = B.make_params(ny, nz, ns, (0.3,), checkpoint_every=ns)   # every a_j kept (268 MB)
    c = B.make_coarse(shape, block, off)
    base = torch.from_numpy(ci.substrate(ny, nz, ns)).cuda()
    batch = 64
    sampler = PillarSampler(p, c, base, n_pillars=(4, 16), foot=(2, 9), height=(1, 9), chunk=args.chunk,
                            tune=not args.no_tune)
    net = EncoderDecoder(ARCH_256, batch)

    # mean occupancy of the training distribution (the constant start)
    _, occ0, _ = sampler.sample(np.random.default_rng(999), 256, noise=False)
    occ_mean = float(occ0.cpu().numpy().mean())

    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = train(net, sampler, args.train_samples, batch, lr=1e-3, seed=1000)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0

    # network step alone (fixed batch), CUDA events on the launching stream
    x, occ, _ = sampler.sample(np.random.default_rng(5), batch)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        net.loss_grad(x, occ, batch)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    nrep = 20
    for _ in range(nrep):
        net.loss_grad(x, occ, batch)
    e1.record(stream)
    torch.cuda.synchronize()
    step_ms = e0.elapsed_time(e1) / nrep
    # forward-model sample generation alone
    e0.record(stream)
    sampler.sample(np.random.default_rng(6), batch)
    e1.record(stream)
    torch.cuda.synchronize()
    gen_ms = e0.elapsed_time(e1)

    per_seed, res = [], {"zero": [], "constant": [], "learned": []}
    cap = args.max_iters
    for k in range(args.heldout):
        seed = 200000 + k
        meas, s, chi2_gt, occ_t = _pillar_case(B, ci, torch, p, c, base, sampler, seed)
        measd = torch.from_numpy(meas).cuda()
        row = {"seed": seed, "chi2_truth": chi2_gt}
        for name in ("zero", "constant", "learned"):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            if name == "zero":
                th0 = None
            elif name == "constant":
                th0 = torch.full((int(np.prod(shape)),), occ_mean * AU_DELTA, dtype=torch.float32, device="cuda")
            else:
                th0 = net.predict(sampler.features_of(measd)).reshape(-1).contiguous()
            torch.cuda.synchronize()
            t_init = time.perf_counter() - t1
            R = Reconstructor(p, c, base, measd, s, theta0=th0, lr=args.lr)
            it, sec, hist = R.run(chi2_target=1.1 * chi2_gt, max_iters=cap, check_every=5)
            reached = bool(hist and hist[-1][1] <= 1.1 * chi2_gt)
            row[name] = {"seconds": t_init + sec, "iterations": it, "reached": reached,
                         "chi2_end": hist[-1][1] if hist else None}
            res[name].append(row[name])
        per_seed.append(row)
    clk = clocks.stop()

    def summary(rows):
        return {"median_s": statistics.median(r["seconds"] for r in rows),
                "reached": "%d/%d" % (sum(r["reached"] for r in rows), len(rows)),
                "median_iterations": statistics.median(r["iterations"] for r in rows)}

    peaks = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = network_step_flops(net, batch) / (step_ms / 1e3) / 1e12
    k = max(1, len(losses) // 10)
    line = {"metric": "recon wall time to chi2_red <= 1.1 chi2_red(truth), learned init (median over held-out "
                      "layouts; unreached runs count at the iteration cap)",
            "value": summary(res["learned"])["median_s"], "unit": "s", "higher_is_better": False,
            "learned_init": summary(res["learned"]), "zero_init": summary(res["zero"]),
            "constant_init": dict(summary(res["constant"]), occupancy=occ_mean),
            "training": {"samples": args.train_samples, "batch": batch, "seconds": t_train,
                         "samples_per_s": args.train_samples / t_train, "loss_first": float(np.mean(losses[:k])),
                         "loss_last": float(np.mean(losses[-k:])), "network_step_ms": step_ms,
                         "sample_generation_ms_per_batch": gen_ms, "structures_per_forward_launch": args.chunk,
                         "params": net.n_params},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": "network training step (k_gemm BF16 mma.sync + permutations), batch %d" % batch,
                         "peak_basis": "bf16_tflops of measured (burst)"},
            "per_seed": per_seed, "clocks": clk, "dtype": "bf16/f32", "data": "synthetic",
            "config": {"workload": "256x256 grid, 512 slices, 0.3 deg, 64^3 coarse delta (8x2x4 fine voxels, top "
                                   "half), 4-16 Au pillars per layout, Poisson targets 1e6 counts, ADAM lr %g, cap %d "
                                   "iterations; network trained on %d fresh forward-model samples"
                                   % (args.lr, cap, args.train_samples)}}
    print(json.dumps(line), flush=True)
    return 0


def run_convergence(args):
    """Slice-thickness convergence: one structure 10 um long along the beam
    (Si substrate + 20 Au boxes sized in nm, each slice holding its thickness
    average), cut into slices of 200 down to 5 nm.  Far-field intensities at
    three incidence angles, with the transmission-first and the symmetric
    splitting, against the symmetric splitting at 2.5 nm; forward time per
    thickness."""
    import torch

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300 import build as cuda_build

    cuda_build.build()
    torch.cuda.set_device(0)
    ny = nz = 256
    length = 10000.0
    ang = (0.15, 0.3, 0.5)
    boxes = ci.boxes_nm(0, ny, nz, length)

    def forward(delta, flags):
        vol = torch.from_numpy(ci.slice_boxes(boxes, ny, nz, length, delta)).cuda()
        p = B.make_params(ny, nz, vol.shape[0], ang, slice_nm=delta, flags=flags)
        ws = B.workspace(p, B.MSLICE_OP_FORWARD)
        inten = torch.empty((len(ang), nz, ny), dtype=torch.float32, device="cuda")
        for _ in range(args.warmup):
            B.mslice_forward(p, vol, None, inten, None, ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            B.mslice_forward(p, vol, None, inten, None, ws)
        e1.record()
        torch.cuda.synchronize()
        if B.mslice_status(ws) != 0:
            raise RuntimeError("device-side wait timed out")
        return inten.double().cpu().numpy(), e0.elapsed_time(e1) / args.steps, vol.shape[0]

    I_ref, ms_ref, ns_ref = forward(2.5, B.MSLICE_STRANG)
    rows = []
    for delta in (200.0, 100.0, 50.0, 20.0, 10.0, 5.0):
        for name, flags in (("transmission-first", 0), ("symmetric", B.MSLICE_STRANG)):
            I, ms, ns = forward(delta, flags)
            err = [float(np.linalg.norm(I[w] - I_ref[w]) / np.linalg.norm(I_ref[w])) for w in range(len(ang))]
            rows.append({"slice_nm": delta, "slices": ns, "splitting": name, "rel_l2_per_angle": err,
                         "ms_forward": ms})
    line = {"metric": "far-field intensity error vs slice thickness", "unit": "relative L2", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "256x256 grid (2 nm), 10 um along the beam, Si + 20 Au boxes, "
                                   "angles 0.15/0.3/0.5 deg; reference: symmetric splitting at 2.5 nm "
                                   "(%d slices, %.2f ms per forward)" % (ns_ref, ms_ref)},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_gemm(args):
    """Dense layer of the learned initialiser on the tcgen05 tensor cores
    (mslice_nn_gemm_bf16): C = A B^T with BF16 operands packed K-major and
    FP32 accumulation, at 8192^3 (operands 134 MB each and C 268 MB, larger
    than L2) and at the network's largest layer shape; TFLOP/s against the
    measured cuBLAS BF16 rate."""
    import torch

    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300 import build as cuda_build

    cuda_build.build()
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    res = {}
    for (M, N, K) in ((8192, 8192, 8192), (16384, 4096, 4096)):
        gen = torch.Generator(device="cuda").manual_seed(0)
        A = torch.randn(M, K, generator=gen, device="cuda").to(torch.bfloat16)
        Bm = torch.randn(N, K, generator=gen, device="cuda").to(torch.bfloat16)
        C = torch.empty(M, N, device="cuda")
        for _ in range(args.warmup):
            B.mslice_nn_gemm_bf16(M, N, K, A, K, Bm, K, C, N)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            B.mslice_nn_gemm_bf16(M, N, K, A, K, Bm, K, C, N)
        e1.record()
        torch.cuda.synchronize()
        if B.mslice_nn_gemm_bf16_status() != 0:
            raise RuntimeError("a bounded wait of the tensor-core GEMM ran out")
        ms = e0.elapsed_time(e1) / args.steps
        tf = 2.0 * M * N * K / (ms / 1e3) / 1e12
        res["%dx%dx%d" % (M, N, K)] = {"ms": ms, "tflops": tf, "frac_of_measured_bf16": tf / peak}
        del A, Bm, C
    head = res["8192x8192x8192"]
    line = {"metric": "BF16 GEMM TFLOP/s (tcgen05, FP32 accumulate)", "value": head["tflops"], "unit": "TFLOP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "bf16",
            "data": "synthetic",
            "config": {"workload": "C = A B^T, M = N = K = 8192, A and B BF16 K-major, C FP32; operands larger "
                                   "than L2"},
            "roofline": {"bound": "tensor", "achieved": head["tflops"], "peak": peak, "unit": "TFLOP/s",
                         "frac": head["frac_of_measured_bf16"], "traffic": None,
                         "peak_basis": "measured cuBLAS BF16 burst" if "bf16_tflops" in peaks else "fallback"},
            "shapes": res}
    print(json.dumps(line), flush=True)
    return 0


def run_rotate(args):
    """Frame rotation of Eq. 2-3 on the headline volume (512x512x1024, Si + 50
    Au pillars/lines): lab-frame resampling at 0.3 deg pitch without and with a
    0.5 deg yaw, and the transpose; HBM bandwidth against the measured copy
    rate (8 B read and 8 B written per voxel)."""
    import torch

    import cssi_inputs as ci
    from paper_2212_01253_gb300 import binding as B
    from paper_2212_01253_gb300 import build as cuda_build

    cuda_build.build()
    torch.cuda.set_device(0)
    ns, nz, ny = NS, NZ, NY
    p = B.make_params(ny, nz, ns, (0.3,), LAM, SLICE, DY, DZ)
    vol = torch.from_numpy(ci.pillars_large(0)).cuda()
    out = torch.empty_like(vol)
    c = (0.0, (nz / 2 - 0.5) * DZ, (ny - 1) / 2 * DY)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    res = {}
    cases = (("rotate_pitch", B.mslice_rotate, 0.0), ("rotate_pitch_yaw", B.mslice_rotate, 0.5),
             ("adjoint_pitch", B.mslice_rotate_adjoint, 0.0), ("adjoint_pitch_yaw", B.mslice_rotate_adjoint, 0.5))
    for name, fn, psi_deg in cases:
        a, ps = np.deg2rad(0.3), np.deg2rad(psi_deg)
        src, dst = (vol, out) if fn is B.mslice_rotate else (out, vol)
        for _ in range(args.warmup):
            fn(p, a, ps, c, src, dst)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn(p, a, ps, c, src, dst)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        gbs = vol.numel() * 16 / (ms / 1e3) / 1e9
        res[name] = {"ms": ms, "voxels_per_s": vol.numel() / (ms / 1e3), "gbs_algorithmic": gbs,
                     "frac_of_measured_hbm": gbs / peak}
    head = res["rotate_pitch_yaw"]
    line = {"metric": "frame rotation voxels/s", "value": head["voxels_per_s"], "unit": "voxels/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "512x512x1024 volume (Si + 50 Au pillars/lines), pitch 0.3 deg, yaw 0.5 deg, "
                                   "trilinear; inputs 2 GiB in and out (larger than L2)"},
            "roofline": {"bound": "hbm", "achieved": head["gbs_algorithmic"], "peak": peak, "unit": "GB/s",
                         "frac": head["frac_of_measured_hbm"], "traffic": None},
            "kernels": res}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--angles", type=int, default=NW)
    ap.add_argument("--slices", type=int, default=NS)
    ap.add_argument("--cpu-slices", type=int, default=1024)
    ap.add_argument("--cpu-angles", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "batch", "recon", "learned", "buried", "convergence", "rotate", "gemm"],
                    help="sweep: the headline 512x512x1024 9-angle step; batch: 64 uneven "
                         "structures in one graph; recon: time to a fixed chi^2; learned: "
                         "learned vs zero vs constant start; buried: coarse Si/Au voxels under the "
                         "surface; convergence: intensity error vs slice thickness; rotate: frame "
                         "rotation of the headline volume")
    ap.add_argument("--train-samples", type=int, default=100000)
    ap.add_argument("--heldout", type=int, default=10)
    ap.add_argument("--chunk", type=int, default=64, help="learned: structures per forward launch")
    ap.add_argument("--snap-every", type=int, default=20, help="buried: material snapping period (epochs)")
    ap.add_argument("--snap-start", type=int, default=0, help="buried: first epoch that snaps")
    ap.add_argument("--buried-extrude", action="store_true", help="buried: pattern uniform along the beam")
    ap.add_argument("--shrinkwrap-every", type=int, default=0, help="buried: shrink-wrap support period (0: off)")
    ap.add_argument("--shrinkwrap-sigma", type=float, default=1.0, help="buried: shrink-wrap blur (coarse voxels)")
    ap.add_argument("--shrinkwrap-threshold", type=float, default=0.2, help="buried: shrink-wrap threshold")
    ap.add_argument("--recon-angles", type=int, default=1, help="recon: incidence angles (views) sharing the volume")
    ap.add_argument("--recon-psi", type=float, default=0.0,
                    help="recon: in-plane angles of the views swept over [-psi, psi] deg")
    ap.add_argument("--checkpoint", type=int, default=0,
                    help="adjoint checkpoint interval (0: keep every a_j when it fits in half the HBM, else 32)")
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--lanes", type=int, default=16,
                    help="batch: concurrent lanes (each group's kernels on the blocks its tasks need)")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-ckpt32", action="store_true", help="sweep: skip the checkpoint-every-32 leg")
    ap.add_argument("--no-recon", action="store_true", help="sweep: skip the reconstruction leg")
    ap.add_argument("--no-batch", action="store_true", help="sweep: skip the batched uneven-structures leg")
    ap.add_argument("--recon-train-samples", type=int, default=65536,
                    help="sweep: forward-model samples the reconstruction leg's network trains on")
    ap.add_argument("--recon-cap", type=int, default=3000, help="sweep: iteration cap of the reconstruction leg")
    ap.add_argument("--angular", action="store_true", help="sweep: angular-spectrum propagator instead of Eq. 1's")
    ap.add_argument("--lr", type=float, default=2e-6)
    ap.add_argument("--max-iters", type=int, default=300)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("at least 3 warm-up steps")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "recon":
        return run_recon(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "buried":
        return run_buried(args)
    if args.workload == "convergence":
        return run_convergence(args)
    if args.workload == "rotate":
        return run_rotate(args)
    if args.workload == "gemm":
        return run_gemm(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
