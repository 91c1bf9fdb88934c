#!/usr/bin/env python
"""Benchmark of the multiple-time-origin MSD + autocorrelation path.

One step = MSD of a positions array + autocorrelation of a velocities array
(the two correlations of Eq. 5 and Eq. 4), then the running Green-Kubo
integral of the autocorrelation and the Einstein slope of the MSD, all on the
GPU through the C ABI.  Metric: atom.origin.lag updates per second, where an
update is one (atom, origin, lag) triple; MSD and autocorrelation updates are
counted separately and summed.

Default workload: the precision configuration, the largest single-GPU one:
N = 100000 atoms, T = 20000 frames, tau_max = 10000, origin stride 1;
positions start uniform in [0, 100) nm (large offsets stress the
cancellation of the split form) plus a random walk of sigma = 0.005 nm per
axis per frame, velocities an OU process (gamma = 0.05 per frame, sigma = 1).
Each array is 24 GB, far larger than L2, so no flush is needed between
steps.  `--workload water` runs the water-scale configuration (N = 32768
3-site molecules, T = 10000, tau_max = 2000).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--method M]
       [--workload W] [--impl reference]   (times the FP64 CPU oracle instead)
Under torchrun each rank runs its own instance (seed + rank) with no
exchange between ranks (weak scaling).
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

WORKLOADS = {
    "precision": dict(N=100000, T=20000, tau_max=10000, stride=1, sigma=0.005, box=100.0, gamma=0.05,
                      sites=1, dt=1.0, stream_chunk=2500,
                      label="precision MSD + VACF + GK + Einstein: N=100000, T=20000, tau_max=10000, "
                            "stride 1, positions offset up to 100 nm"),
    "precision16": dict(N=6250, T=20000, tau_max=10000, stride=1, sigma=0.005, box=100.0, gamma=0.05,
                        sites=1, dt=1.0, stream_chunk=2500,
                        label="precision shape with 1/16 of the atoms (profiling case): N=6250, T=20000, "
                              "tau_max=10000, stride 1, positions offset up to 100 nm"),
    "water": dict(N=32768, T=10000, tau_max=2000, stride=1, sigma=0.005, box=5.0, gamma=0.05,
                  sites=3, dt=1.0,
                  label="water-scale MSD + VACF + GK + Einstein: N=32768 (3-site molecules), "
                        "T=10000, tau_max=2000, stride 1"),
    "water8": dict(N=4096, T=10000, tau_max=2000, stride=1, sigma=0.005, box=5.0, gamma=0.05, sites=3,
                   dt=1.0, label="water-scale with 1/8 of the atoms (profiling case): N=4096 (3-site "
                                 "molecules), T=10000, tau_max=2000, stride 1"),
    "mid": dict(N=8192, T=5000, tau_max=1000, stride=1, sigma=0.005, box=5.0, gamma=0.05, sites=3,
                dt=1.0, label="mid-size MSD + VACF + GK + Einstein: N=8192 (3-site molecules), "
                              "T=5000, tau_max=1000, stride 1 (profiling case)"),
    "batch": dict(label="batching: 256 uneven instances, N log-uniform in [64, 16384], T uniform in "
                        "[500, 20000], tau_max = T/4, even: MSD of a random walk (sigma 0.01), odd: VACF of "
                        "OU velocities (gamma uniform in [0.01, 0.5])", count=256, stride=1),
    "flux": dict(label="Green-Kubo flux ACF: (Pxy, Pxz, Pyz) as [T][1][3], AR(1) phi=0.999 unit variance, "
                       "T=2,000,000 plus 64 series of T=200,000, tau_max=20,000, ACF + running viscosity "
                       "integral", T=2000000, Tshort=200000, nshort=64, tau_max=20000, phi=0.999),
    "viscosity": dict(label="viscosity ACF with a long window: (Pxy, Pxz, Pyz) as [T][1][3], AR(1) phi=0.999, "
                           "T=2,000,000, tau_max=500,000, ACF + running integral; FFT route vs polyphase "
                           "tensor core", T=2000000, tau_max=500000, phi=0.999),
    "collective": dict(N=32768, T=10000, tau_max=2000, stride=1, sigma=0.005, box=5.0, gamma=0.05, sites=3,
                       dt=1.0, label="collective quantities on the water-scale arrays (N=32768 3-site molecules, "
                                     "SPC/E-like charges -0.8476 / +0.4238, T=10000, tau_max=2000): "
                                     "Einstein-Helfand MSD of sum_i q_i r_i (FFT route) + charge-current ACF "
                                     "(polyphase tensor core) + its running integral"),
    "small": dict(N=512, T=1000, tau_max=500, stride=1, sigma=0.01, box=3.0, gamma=0.1, sites=1,
                  dt=1.0, label="small MSD + VACF: N=512, T=1000, tau_max=500, stride 1"),
}


def issued_over_useful(N, T, tau_max, s, BO=128, BF=192):
    """Tile entries the band kernel issues per useful (origin, lag) pair.

    Per residue rho of the stride: row tiles of BO origins times column tiles
    of BF frames; a column tile is issued ncol = min(BF, m_max - c*BF + BO)
    columns wide (rounded up to 16), tiles past the band or past the last
    frame are skipped."""
    issued = 0
    for rho in range(min(s, tau_max + 1)):
        m_max = (tau_max - rho) // s
        n_rho = (T - 1 - rho) // s + 1
        n_orig = (T - 1) // s + 1
        n_rows = -(-n_orig // BO)
        n_cols = -(-(BO + tau_max // s) // BF)
        for r in range(n_rows):
            for c in range(n_cols):
                if c * BF - BO + 1 > m_max or r * BO + c * BF >= n_rho:
                    continue
                need = m_max - c * BF + BO
                ncol = BF if need >= BF else max(16, -(-need // 16) * 16)
                issued += BO * ncol
    return issued / updates(1, T, tau_max, s)


def updates(N, T, tau_max, s):
    tau = np.arange(tau_max + 1, dtype=np.int64)
    return int(N * ((T - 1 - tau) // s + 1).sum())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def gpu_identifier(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return dev


# DRAM bytes (read + write) per launch of the dominant kernel, from ncu captures of the kernel as
# built now, per workload.  A capture too large for ncu is taken on the 1/8- or 1/16-atom case
# of the same T and tau_max and scaled by the atom ratio: operand bytes, tiles and updates all
# scale with N there.  A workload or method without an entry reports null.
GRAM_TRAFFIC_BYTES = {("water", "fp16x3"): 8 * (1191.874304e6 + 3.766784e6),
                      ("precision", "fp16x3"): 16 * (16901.152128e6 + 59.153920e6)}
# DRAM bytes of one collective_kernel launch on the water-scale velocities (no reference frame):
# ncu's dram__bytes.sum.per_second x gpu__time_duration.sum.
COLLECTIVE_WATER_TRAFFIC_BYTES = 6.622334e12 * 594.496e-6


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# ------------------------------------------------------------------ oracle arm

def oracle_lags(wl):
    """The lags at which the oracle is evaluated, both for the GPU arm's error
    check and CPU baseline and for the reference arm: 24 evenly spaced lags in
    [0, tau_max], lags 1 and 2, and 16 lags spread over the last 192 lags (the
    last column tile of every band row of the tensor-core kernel)."""
    tm = wl["tau_max"]
    spread = np.linspace(0, tm, 24).astype(np.int64)
    tail = np.linspace(max(0, tm - 191), tm, 16).astype(np.int64)
    return np.unique(np.concatenate([spread, [1, 2], tail]).clip(0, tm))


def oracle_pass(xh, vh, s, lags, nthreads=None):
    """MSD of xh and autocorrelation of vh at `lags` by the FP64 oracle; returns
    (MSD values, ACF values, seconds, updates)."""
    import oracle
    T, N = xh.shape[0], xh.shape[1]
    t0 = time.perf_counter()
    m_ref = oracle.msd(xh, stride=s, lags=lags, nthreads=nthreads)
    c_ref = oracle.acf(vh, stride=s, lags=lags, nthreads=nthreads)
    el = time.perf_counter() - t0
    n_up = 2 * int(sum(N * ((T - 1 - int(l)) // s + 1) for l in lags))
    return m_ref, c_ref, el, n_up


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload not in ("precision", "precision16", "water", "water8", "mid", "small"):
        print(json.dumps({"impl": "reference",
                          "unavailable": "the reference arm times the oracle on the MSD + VACF workloads "
                                         "(precision, water, their profiling cases, mid, small); this "
                                         "workload has no such line"}),
              flush=True)
        return
    import oracle
    from paper_1708_08619_gb300 import synth
    T, tm, s = wl["T"], wl["tau_max"], wl["stride"]
    lags = oracle_lags(wl)
    cores = oracle.default_threads()
    # each step: the oracle at the GPU arm's lags over a slice of the atoms sized to about
    # TCORR_REF_STEP_S seconds (every atom is an independent draw of the same recipe, so a
    # slice is a sample of the same workload); calibrated on one 64-atom block per thread
    per_step = float(os.environ.get("TCORR_REF_STEP_S", "3.0"))
    n_cal = min(wl["N"], 64 * cores)
    xc = synth.random_walk_positions(T, n_cal, wl["sigma"], wl["box"], synth.BASE_SEED,
                                     sites_per_molecule=wl["sites"])
    vc = synth.ou_velocities(T, n_cal, wl["gamma"], 1.0, synth.BASE_SEED + 1)
    el_cal = oracle_pass(xc, vc, s, lags)[2]
    blocks = max(1, int(per_step / max(el_cal, 1e-3)))
    n_sub = int(min(wl["N"], n_cal * blocks))
    if n_sub > n_cal:
        xh = synth.random_walk_positions(T, n_sub, wl["sigma"], wl["box"], synth.BASE_SEED,
                                         sites_per_molecule=wl["sites"])
        vh = synth.ou_velocities(T, n_sub, wl["gamma"], 1.0, synth.BASE_SEED + 1)
    else:
        xh, vh = xc, vc
    del xc, vc
    for _ in range(args.warmup):
        oracle_pass(xh, vh, s, lags)
    rates, tot_t, n_up = [], 0.0, 0
    for _ in range(args.steps):
        _, _, el, n_up = oracle_pass(xh, vh, s, lags)
        rates.append(n_up / el)
        tot_t += el
    value = float(statistics.median(rates))
    sample = (f"per step: MSD and VACF at the GPU arm's {len(lags)} oracle lags in [0, {tm}], all origins, "
              f"{n_sub} of the {wl['N']} atoms (numpy-drawn, same recipe)")
    line = {"impl": "reference", "metric": "atom.origin.lag updates/s (MSD+ACF)", "value": value,
            "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tot_t / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["label"], "N": wl["N"], "T": T, "tau_max": tm,
                       "stride": s, "method": "oracle (FP64 CPU)", "updates_per_step": n_up,
                       "atoms_per_step": n_sub, "lags_per_step": int(len(lags))},
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- GPU arm

def run_gpu(args, wl):
    import torch
    from paper_1708_08619_gb300 import build as tbuild
    from paper_1708_08619_gb300 import shard, synth, tcorr

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tbuild.build()
    tcorr.load()

    N, T, tm, s = wl["N"], wl["T"], wl["tau_max"], wl["stride"]
    method = args.method
    x = synth.random_walk_positions_device(T, N, wl["sigma"], wl["box"], synth.BASE_SEED + rank,
                                           device=dev, sites_per_molecule=wl["sites"])
    v = synth.ou_velocities_device(T, N, wl["gamma"], 1.0, synth.BASE_SEED + 1000 + rank, device=dev)
    need = max(tcorr.tcorr_workspace_size(T, N, tm, s, method), 256)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    out_m = torch.empty(tm + 1, dtype=torch.float64, device=dev)
    out_c = torch.empty(tm + 1, dtype=torch.float64, device=dev)
    out_gk = torch.empty(tm + 1, dtype=torch.float64, device=dev)
    out_D = torch.empty(2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    # this library's launches per step -- plain: tile + reduce (MSD), tile + reduce (ACF), GK,
    # Einstein; tensor core: split + S combine + S prefix + Gram + reduce (MSD), split + Gram +
    # reduce (ACF), GK (one launch up to 32 blocks of 2048 lags), Einstein
    gk_launches = 1 if tm + 1 <= 32 * 2048 else 3
    launches_per_step = (5 if method == "plain" else 9) + gk_launches

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    msd_ms, acf_ms = [], []

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        tcorr.tcorr_msd(x, tm, s, method, out=out_m, ws=ws, stream=stream)
        if ev:
            ev[1].record(stream)
        tcorr.tcorr_acf(v, tm, s, method, out=out_c, ws=ws, stream=stream)
        if ev:
            ev[2].record(stream)
        tcorr.gk_integrate(out_c, wl["dt"], 1.0 / 3.0, out=out_gk, stream=stream)
        tcorr.einstein_slope(out_m, wl["dt"], 3, out=out_D, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if tcorr.tcorr_status_poll() != 0:
        raise RuntimeError("device status word set during warm-up")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    sampler = ClockSampler(gpu_identifier(torch, local))
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    tcorr.tcorr_profile_enable(True)      # events around each launch of the dominant kernel
    tcorr.tcorr_profile_read(0)
    tcorr.tcorr_profile_read(1)
    sampler.start()
    time.sleep(0.3)
    start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    kern_msd = tcorr.tcorr_profile_read(0)
    kern_acf = tcorr.tcorr_profile_read(1)
    tcorr.tcorr_profile_enable(False)
    for ev in evs:
        msd_ms.append(ev[0].elapsed_time(ev[1]))
        acf_ms.append(ev[1].elapsed_time(ev[2]))
    barrier()
    clocks = sampler.stop()
    elapsed_ms = start.elapsed_time(end)
    if tcorr.tcorr_status_poll() != 0:
        raise RuntimeError("device status word set during the timed region")

    ms_per_step = shard.max_over_ranks(elapsed_ms / args.steps)
    m_dev = out_m.cpu().numpy().copy()       # the timed steps' results (checked against the oracle below)
    c_dev = out_c.cpu().numpy().copy()
    u_res = updates(N, T, tm, s)
    u_step = 2 * u_res
    value = u_step * world / (ms_per_step / 1000.0)

    # ---- roofline of the dominant kernel (the MSD kernel), timed alone
    pk, pk_kind = peaks()
    msd_avg_s = kern_msd[0] / max(1, kern_msd[1]) / 1000.0
    acf_avg_s = kern_acf[0] / max(1, kern_acf[1]) / 1000.0
    if method == "plain":
        sm_mhz = pk.get("sm_max_mhz", 2070.0)
        peak_ops = 152 * 128 * sm_mhz * 1e6 / 1e12     # FP32 lane-ops/s (T)
        achieved = 6.0 * u_res / msd_avg_s / 1e12      # 3 FSUB + 3 FFMA per update
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "Tops/s",
                "frac": achieved / peak_ops, "traffic": None,
                "kernel": "plain_tile_kernel<MSD>",
                "note": f"FP32 lane-ops (FSUB, FFMA) per s of the MSD tile kernel alone (CUDA events around "
                        f"its {kern_msd[1]} launches); peak = 152 SMs x 128 lanes x {sm_mhz:.0f} MHz "
                        f"({pk_kind} max clock)"}
    else:
        flops = 6.0 * u_res   # useful Gram flops: 3 MACs per update
        # a timed region of seconds runs under the power cap: the sustained peak applies
        sustained = elapsed_ms > 1000.0
        peak_t = pk.get("bf16_tflops_sustained" if sustained else "bf16_tflops", 1700.0 if sustained else 1900.0)
        achieved = flops / msd_avg_s / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak_t, "unit": "TFLOP/s",
                "frac": achieved / peak_t, "traffic": GRAM_TRAFFIC_BYTES.get((args.workload, method)),
                "kernel": "gram_band_tc<MSD>",
                "note": f"useful Gram FLOPs (6 per update) / duration of the MSD band kernel alone (CUDA events "
                        f"around its {kern_msd[1]} launches) vs the {pk_kind} bf16 dense "
                        f"{'sustained (timed region %.1f s)' % (elapsed_ms / 1e3) if sustained else 'burst'} peak; "
                        f"the split form issues 3 products per useful one plus band waste",
                "frac_of_burst": achieved / pk.get("bf16_tflops", 1900.0),
                "issued_tflops": 3.0 * flops * issued_over_useful(N, T, tm, s) / msd_avg_s / 1e12,
                "acf_kernel_frac": flops / acf_avg_s / 1e12 / peak_t}

    # ---- host copies (pinned) of the inputs: the end-to-end steps upload them, the oracle reads them
    xh = torch.empty((T, N, 3), dtype=torch.float32, pin_memory=True)
    vh = torch.empty((T, N, 3), dtype=torch.float32, pin_memory=True)
    xh.copy_(x)
    vh.copy_(v)
    # the in-core end-to-end steps upload from frame chunks of about 1 GiB, each pinned on its own:
    # after minutes of load on the host cores a single pinned buffer of many GB uploaded at
    # 26-36 GB/s (61-116 GB/s in 1 GiB pieces), separately pinned 1 GiB buffers at 211 GB/s
    fpc = max(1, (1 << 30) // (N * 3 * 4))
    chunk_t = list(range(0, T, fpc))
    xcs = [torch.empty((min(fpc, T - t), N, 3), dtype=torch.float32, pin_memory=True) for t in chunk_t]
    vcs = [torch.empty((min(fpc, T - t), N, 3), dtype=torch.float32, pin_memory=True) for t in chunk_t]
    for t, cx, cv in zip(chunk_t, xcs, vcs):
        cx.copy_(x[t:t + cx.shape[0]])
        cv.copy_(v[t:t + cv.shape[0]])

    # ---- end to end through the public API from pinned host memory, measured right after the
    # timed steps and before the plain-kernel and oracle legs: the sustained load of those legs
    # slowed host-to-device copies of these buffers (24-112 GB/s right after them, 211 GB/s
    # before them).  The workspace is released first (each variant allocates its own buffers);
    # the device inputs stay for the plain-kernel comparison that follows
    del ws
    torch.cuda.empty_cache()
    m_host = torch.empty(tm + 1, dtype=torch.float64, pin_memory=True)
    c_host = torch.empty(tm + 1, dtype=torch.float64, pin_memory=True)
    gk_host = torch.empty(tm + 1, dtype=torch.float64, pin_memory=True)
    D_host = torch.empty(2, dtype=torch.float64, pin_memory=True)
    e2e_steps = max(1, min(args.steps, 5))

    def timed_e2e(fn):
        # each step ends with its results read back to the host (a stream synchronise), so
        # steps are timed one by one; the median keeps one slow step of the shared host link
        # from setting the number
        fn()
        torch.cuda.synchronize()
        barrier()
        per = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            per.append(time.perf_counter() - t0)
        return shard.max_over_ranks(statistics.median(per))

    def finish_on(st):
        # GK + Einstein, then the results back to pinned host memory
        tcorr.gk_integrate(out_c, wl["dt"], 1.0 / 3.0, out=out_gk, stream=st)
        tcorr.einstein_slope(out_m, wl["dt"], 3, out=out_D, stream=st)
        with torch.cuda.stream(st):
            m_host.copy_(out_m, non_blocking=True)
            c_host.copy_(out_c, non_blocking=True)
            gk_host.copy_(out_gk, non_blocking=True)
            D_host.copy_(out_D, non_blocking=True)
        st.synchronize()

    copy_stream = torch.cuda.Stream(dev)
    ev_x, ev_v = torch.cuda.Event(), torch.cuda.Event()

    # (a) whole arrays up on a copy stream, then the in-core calls (the MSD starts when the
    # positions have landed)
    x2 = torch.empty((T, N, 3), dtype=torch.float32, device=dev)
    v2 = torch.empty_like(x2)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)

    def e2e_incore():
        with torch.cuda.stream(copy_stream):
            for t, cx in zip(chunk_t, xcs):
                x2[t:t + cx.shape[0]].copy_(cx, non_blocking=True)
            ev_x.record(copy_stream)
            for t, cv in zip(chunk_t, vcs):
                v2[t:t + cv.shape[0]].copy_(cv, non_blocking=True)
            ev_v.record(copy_stream)
        stream.wait_event(ev_x)
        tcorr.tcorr_msd(x2, tm, s, method, out=out_m, ws=ws, stream=stream)
        stream.wait_event(ev_v)
        tcorr.tcorr_acf(v2, tm, s, method, out=out_c, ws=ws, stream=stream)
        finish_on(stream)

    e2e_incore_s = timed_e2e(e2e_incore)
    # the input buffers' own host link rate: one whole-array copy of the positions, CUDA events
    i0, i1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    i0.record(stream)
    with torch.cuda.stream(stream):
        x2.copy_(xh, non_blocking=True)
    i1.record(stream)
    i1.synchronize()
    h2d_gbs_input = xh.numel() * 4 / (i0.elapsed_time(i1) / 1e3) / 1e9
    # and of the separately pinned chunks the in-core steps upload from
    i0.record(stream)
    with torch.cuda.stream(stream):
        for t, cx in zip(chunk_t, xcs):
            x2[t:t + cx.shape[0]].copy_(cx, non_blocking=True)
    i1.record(stream)
    i1.synchronize()
    h2d_gbs_chunks = xh.numel() * 4 / (i0.elapsed_time(i1) / 1e3) / 1e9
    del v2
    torch.cuda.empty_cache()

    # (b) positions copied whole at the link's full rate, the in-core MSD as soon as they have
    # landed, and the velocities streamed behind them: the VACF windows run while later windows
    # cross the link, so only the last window's work follows the last copy
    C = args.stream_chunk or wl.get("stream_chunk", 2048)
    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ws_b = torch.empty(tcorr.tcorr_stream_workspace_size(T, N, tm, s, method, C), dtype=torch.uint8, device=dev)

    def e2e_hybrid():
        with torch.cuda.stream(copy_stream):
            for t, cx in zip(chunk_t, xcs):
                x2[t:t + cx.shape[0]].copy_(cx, non_blocking=True)
            ev_x.record(copy_stream)
        sa.wait_event(ev_x)
        sb.wait_event(ev_x)
        tcorr.tcorr_msd(x2, tm, s, method, out=out_m, ws=ws, stream=sa)
        tcorr.tcorr_acf_stream_chunks(vcs, tm, s, method, window_frames=C, out=out_c, ws=ws_b, stream=sb)
        stream.wait_stream(sa)
        stream.wait_stream(sb)
        finish_on(stream)

    e2e_hybrid_s = timed_e2e(e2e_hybrid)
    del x2, ws
    torch.cuda.empty_cache()

    # (c) the streamed calls, MSD and VACF on two streams with a workspace each: windows of C
    # origins, host copies overlapping the kernels
    ws_a = torch.empty(tcorr.tcorr_stream_workspace_size(T, N, tm, s, method, C), dtype=torch.uint8, device=dev)
    ev_go = torch.cuda.Event()

    def e2e_streamed():
        ev_go.record(stream)
        sa.wait_event(ev_go)
        sb.wait_event(ev_go)
        tcorr.tcorr_msd_stream_chunks(xcs, tm, s, method, window_frames=C, out=out_m, ws=ws_a, stream=sa)
        tcorr.tcorr_acf_stream_chunks(vcs, tm, s, method, window_frames=C, out=out_c, ws=ws_b, stream=sb)
        stream.wait_stream(sa)
        stream.wait_stream(sb)
        finish_on(stream)

    e2e_stream_s = timed_e2e(e2e_streamed)
    del ws_a, ws_b
    torch.cuda.empty_cache()
    # this machine's host link: one pinned-to-device copy of 1 GiB, CUDA events
    hb = torch.empty(1 << 28, dtype=torch.float32, pin_memory=True)
    db = torch.empty(1 << 28, dtype=torch.float32, device=dev)
    db.copy_(hb, non_blocking=True)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(3):
        db.copy_(hb, non_blocking=True)
    h1.record(stream)
    h1.synchronize()
    h2d_gbs = 3 * (1 << 30) / (h0.elapsed_time(h1) / 1e3) / 1e9
    del hb, db
    e2e_s = min(e2e_stream_s, e2e_incore_s, e2e_hybrid_s)
    e2e_value = u_step * world / e2e_s
    h2d = 2 * T * N * 3 * 4
    d2h = (3 * (tm + 1) + 2) * 8
    e2e_api = {e2e_stream_s: ("tcorr_msd_stream_chunks + tcorr_acf_stream_chunks (separately pinned 1 GiB frame "
                              "chunks) on two streams, window_frames=%d" % C),
               e2e_incore_s: "host copies (separately pinned 1 GiB frame chunks) + tcorr_msd + tcorr_acf",
               e2e_hybrid_s: ("positions copied in separately pinned 1 GiB frame chunks + tcorr_msd, velocities "
                              "through tcorr_acf_stream_chunks (window_frames=%d) behind them" % C)}
    e2e_info = {"api": e2e_api[e2e_s],
                "ms_per_step": e2e_s * 1e3,
                "streamed_ms_per_step": e2e_stream_s * 1e3,
                "incore_ms_per_step": e2e_incore_s * 1e3,
                "hybrid_ms_per_step": e2e_hybrid_s * 1e3,
                "h2d_gbs_measured": h2d_gbs,
                "h2d_gbs_input_buffer": h2d_gbs_input,
                "h2d_gbs_input_chunks": h2d_gbs_chunks,
                "h2d_link_bound_ms": h2d / h2d_gbs / 1e6}

    del xcs, vcs                          # the chunked host copies serve the end-to-end steps only

    # ---- the plain FP32 kernel on the same arrays, for the tensor-core vs plain comparison
    plain_cmp = None
    if method != "plain" and not args.no_plain_compare:
        ws_p = torch.empty(max(tcorr.tcorr_workspace_size(T, N, tm, s, "plain"), 256), dtype=torch.uint8,
                           device=dev)
        reps = 2 if u_step < 1e13 else 1
        tcorr.tcorr_profile_enable(True)
        tcorr.tcorr_profile_read(0)
        tcorr.tcorr_profile_read(1)
        tcorr.tcorr_msd(x, tm, s, "plain", out=out_m, ws=ws_p, stream=stream)
        tcorr.tcorr_acf(v, tm, s, "plain", out=out_c, ws=ws_p, stream=stream)
        torch.cuda.synchronize()
        pm_err = None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        tcorr.tcorr_profile_read(0)
        tcorr.tcorr_profile_read(1)
        e0.record(stream)
        for _ in range(reps):
            tcorr.tcorr_msd(x, tm, s, "plain", out=out_m, ws=ws_p, stream=stream)
            tcorr.tcorr_acf(v, tm, s, "plain", out=out_c, ws=ws_p, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        pk_m = tcorr.tcorr_profile_read(0)
        pk_c = tcorr.tcorr_profile_read(1)
        tcorr.tcorr_profile_enable(False)
        p_ms = e0.elapsed_time(e1) / reps
        lane_peak = 152 * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6
        pm_s = pk_m[0] / max(1, pk_m[1]) / 1e3
        pc_s = pk_c[0] / max(1, pk_c[1]) / 1e3
        m_plain, c_plain = out_m.cpu().numpy().copy(), out_c.cpu().numpy().copy()
        plain_cmp = {"method": "plain", "ms_per_step_msd_acf": p_ms,
                     "updates_per_s": u_step / (p_ms / 1000.0),
                     "speedup_of_timed_method": value / (u_step / (p_ms / 1000.0)),
                     "msd_kernel_ms": pm_s * 1e3, "acf_kernel_ms": pc_s * 1e3,
                     "msd_lane_peak_frac": 6.0 * u_res / pm_s / lane_peak,
                     "acf_lane_peak_frac": 3.0 * u_res / pc_s / lane_peak}
        del ws_p
    else:
        m_plain = c_plain = None

    cpu = None
    err_vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        lags = oracle_lags(wl)
        m_ref, c_ref, el, n_up = oracle_pass(xh.numpy(), vh.numpy(), s, lags)
        cores = oracle.default_threads()
        # the same oracle on one host thread: the same lags, 1/cores of the atoms (the per-atom
        # work is what the threads share), MSD only
        n1 = max(64, N // max(1, cores))
        x1 = np.ascontiguousarray(xh.numpy()[:, :n1, :])
        t1 = time.perf_counter()
        oracle.msd(x1, stride=s, lags=lags, nthreads=1)
        el1 = time.perf_counter() - t1
        del x1
        r1 = int(sum(n1 * ((T - 1 - int(l)) // s + 1) for l in lags)) / el1
        cpu = {"value": n_up / el, "unit": "updates/s", "cores": cores, "kind": "oracle",
               "sample": f"MSD and VACF at {len(lags)} lags in [0, {tm}] (24 evenly spaced, 1, 2 and 16 "
                         f"in the last 192), all atoms and origins of the same arrays; {el:.1f} s",
               "value_1core": r1,
               "sample_1core": f"MSD at the same {len(lags)} lags, the first {n1} atoms, one thread; "
                               f"{el1:.1f} s"}
        # the timed steps' results against the oracle at those lags (the metric's bar)
        err_vs_oracle = {"lags": int(len(lags)),
                         "msd_max_abs_over_msd_tau_max": float(np.max(np.abs(m_dev[lags] - m_ref)) / m_ref[-1]),
                         "acf_max_abs_over_c0": float(np.max(np.abs(c_dev[lags] - c_ref)) / abs(c_ref[0])),
                         "tolerance": 1e-6 if method == "plain" else 1e-5}
        if m_plain is not None:
            err_vs_oracle["plain_msd_max_rel_per_lag"] = float(
                np.max(np.abs(m_plain[lags[1:]] - m_ref[1:]) / m_ref[1:])) if len(lags) > 1 else 0.0
            err_vs_oracle["plain_acf_max_abs_over_c0"] = float(
                np.max(np.abs(c_plain[lags] - c_ref)) / abs(c_ref[0]))
            err_vs_oracle["plain_tolerance"] = 1e-6


    dtype = {"plain": "f32", "fp16x3": "f16x3 (f32 accumulate)", "bf16x3": "bf16x3 (f32 accumulate)",
             "bf16x4": "bf16x4 (f32 accumulate)", "tf32x3": "tf32x3 (f32 accumulate)"}.get(method, method)
    line = {"metric": "atom.origin.lag updates/s (MSD+ACF)", "value": value, "unit": "updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": wl["label"], "N": N, "T": T, "tau_max": tm, "stride": s,
                       "method": method, "parallelism": f"replica x{world}",
                       "l2": "inputs larger than L2 (2 x %.2f GB), no flush" % (T * N * 12 / 1e9),
                       "msd_ms": statistics.mean(msd_ms), "acf_ms": statistics.mean(acf_ms),
                       "msd_kernel_ms": msd_avg_s * 1000.0, "acf_kernel_ms": acf_avg_s * 1000.0,
                       "updates_per_step": u_step, "plain_comparison": plain_cmp,
                       "error_vs_oracle": err_vs_oracle},
            "clocks": clocks,
            "e2e": dict({"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h}, **e2e_info),
            "gpu_launches": launches_per_step * args.steps,
            "roofline": roof,
            "cpu_baseline": cpu}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch_workload(args, wl):
    """One tcorr_batch call (CUDA-graph replay of the batched launches) per step,
    compared with the same instances run by per-instance tcorr_msd / tcorr_acf calls."""
    import torch
    from paper_1708_08619_gb300 import build as tbuild
    from paper_1708_08619_gb300 import synth, tcorr

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tbuild.build()
    tcorr.load()
    from paper_1708_08619_gb300 import shard
    wshapes = synth.batch_workload_shapes(wl["count"])
    shapes = [(Tn, N, tm, s) for _, Tn, N, tm, s, _ in wshapes]
    u_all = sum(updates(N, Tn, tm, s) for Tn, N, tm, s in shapes)
    mine = shard.my_share(shapes, rank, world)       # instance sharding, no exchange
    items = []
    for i in mine:
        kind, Tn, N, tm, s, _ = wshapes[i]
        x = synth.batch_instance_device(i, wshapes[i], device=dev)
        out = torch.empty(tm + 1, dtype=torch.float64, device=dev)
        items.append((kind, x, tm, 1, out))
    u_total = u_all
    method = args.method
    inst = tcorr.make_instances(items)
    need = tcorr.tcorr_batch_workspace_size(inst, method)
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            tcorr.tcorr_batch(inst, method, ws=ws, stream=stream)
        stream.synchronize()
        sampler = ClockSampler(gpu_identifier(torch, local))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        sampler.start()
        time.sleep(0.3)
        e0.record(stream)
        for _ in range(args.steps):
            tcorr.tcorr_batch(inst, method, ws=ws, stream=stream)
        e1.record(stream)
        stream.synchronize()
        clocks = sampler.stop()
        batch_ms = e0.elapsed_time(e1) / args.steps
        # the same work as per-instance calls (one workspace sized for the largest instance)
        del ws
        need1 = max(tcorr.tcorr_workspace_size(x.shape[0], x.shape[1], tm, s, method)
                    for _, x, tm, s, _ in items)
        ws1 = torch.empty(need1, dtype=torch.uint8, device=dev)

        def per_instance():
            for kind, x, tm, s, out in items:
                f = tcorr.tcorr_msd if kind == 0 else tcorr.tcorr_acf
                f(x, tm, s, method, out=out, ws=ws1, stream=stream)
        per_instance()
        stream.synchronize()
        # the comparison alternates the two forms (batch, per-instance, batch, ...) so that both
        # see the same power-cap state; medians of the pairs
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
        pair_b, pair_p = [], []
        for _ in range(max(1, min(3, args.steps))):
            for fn, acc in ((lambda: tcorr.tcorr_batch(inst, method, ws=ws, stream=stream), pair_b),
                            (per_instance, pair_p)):
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                fn()
                a1.record(stream)
                a1.synchronize()
                acc.append(a0.elapsed_time(a1))
        del ws
        single_ms = statistics.median(pair_p)
        batch_pair_ms = statistics.median(pair_b)
    # the batch's results (the last call above) against the oracle: every 8th instance of this
    # rank's share at lags 1, tau_max/2 and tau_max
    err = None
    if not args.no_cpu_baseline:
        import oracle
        w_msd = w_acf = 0.0
        n_chk = 0
        tcorr.tcorr_batch(inst, method, ws=torch.empty(need, dtype=torch.uint8, device=dev), stream=stream)
        stream.synchronize()
        for kind, x, tm, s, out in items[::8]:
            lags = np.unique(np.array([0, 1, tm // 2, tm]))
            got = out.cpu().numpy()[lags]
            ref = (oracle.msd if kind == 0 else oracle.acf)(x.cpu().numpy(), stride=s, lags=lags)
            if kind == 0:
                w_msd = max(w_msd, float(np.max(np.abs(got - ref)) / ref[-1]))
            else:
                w_acf = max(w_acf, float(np.max(np.abs(got - ref)) / abs(ref[0])))
            n_chk += 1
        err = {"instances": n_chk, "lags_per_instance": 4, "msd_max_abs_over_msd_tau_max": w_msd,
               "acf_max_abs_over_c0": w_acf, "tolerance": 1e-6 if method == "plain" else 1e-5}
    ms = shard.max_over_ranks(batch_ms)
    value = u_total / (ms / 1000.0)            # the whole batch, shared by all ranks
    pk, pk_kind = peaks()
    achieved = 6.0 * u_total / (ms / 1000.0) / 1e12
    line = {"metric": "atom.origin.lag updates/s (MSD+ACF)", "value": value, "unit": "updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": method, "data": "synthetic",
            "config": {"workload": wl["label"], "instances": wl["count"], "method": method,
                       "parallelism": f"instance-sharded x{world} (greedy by work, no exchange)",
                       "updates_per_step": u_total, "input_gb": sum(x.numel() * 4 for _, x, *_ in items) / 1e9,
                       "graph_batch_ms": batch_ms, "workspace_gb": need / 1e9,
                       "alternating_pairs": {"graph_batch_ms": batch_pair_ms, "per_instance_launches_ms": single_ms,
                                             "pairs": len(pair_p)},
                       "batch_speedup_vs_per_instance": single_ms / batch_pair_ms,
                       "error_vs_oracle": err,
                       "l2": "inputs larger than L2, no flush"},
            "clocks": clocks, "e2e": None,
            "gpu_launches": None,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk.get("bf16_tflops", 1900.0),
                         "unit": "TFLOP/s", "frac": achieved / pk.get("bf16_tflops", 1900.0), "traffic": None,
                         "kernel": "gram_band_batch_kernel", "note": f"useful Gram FLOPs / batch call time, "
                                                                    f"{pk_kind} bf16 peak"},
            "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_flux_workload(args, wl):
    """ACF of one long flux series plus a batch of 64 shorter ones, and the running
    Green-Kubo integral of every result, per step."""
    import torch
    from paper_1708_08619_gb300 import build as tbuild
    from paper_1708_08619_gb300 import synth, tcorr

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tbuild.build()
    tcorr.load()
    tm = wl["tau_max"]
    longh = synth.ar1_flux(wl["T"], wl["phi"], seed=synth.BASE_SEED + 6 + 100 * rank)
    shorth = [synth.ar1_flux(wl["Tshort"], wl["phi"], seed=synth.BASE_SEED + 1000 + 100 * rank + i)
              for i in range(wl["nshort"])]
    xl = torch.from_numpy(longh).to(dev)
    xs = [torch.from_numpy(a).to(dev) for a in shorth]
    u = updates(1, wl["T"], tm, 1) + wl["nshort"] * updates(1, wl["Tshort"], tm, 1)
    stream = torch.cuda.Stream(dev)
    res, res_all = {}, {}
    for method in ((args.method,) if args.no_plain_compare else (args.method, "plain")):
        # one row per series (the long one first): the running integrals of all of them in one launch
        outs = torch.empty((1 + wl["nshort"], tm + 1), dtype=torch.float64, device=dev)
        gks = torch.empty_like(outs)
        items = [(1, x, tm, 1, outs[1 + i]) for i, x in enumerate(xs)]
        inst = tcorr.make_instances(items)
        ws_b = torch.empty(max(256, tcorr.tcorr_batch_workspace_size(inst, method)), dtype=torch.uint8, device=dev)
        ws_l = torch.empty(max(256, tcorr.tcorr_workspace_size(wl["T"], 1, tm, 1, method)), dtype=torch.uint8,
                           device=dev)
        with torch.cuda.stream(stream):
            def step():
                tcorr.tcorr_acf(xl, tm, 1, method, out=outs[0], ws=ws_l, stream=stream)
                tcorr.tcorr_batch(inst, method, ws=ws_b, stream=stream)
                tcorr.gk_integrate_batch(outs, 1.0, 1.0 / 3.0, out=gks, stream=stream)
            for _ in range(max(3, args.warmup)):
                step()
            stream.synchronize()
            steps = args.steps if method == args.method else max(1, min(2, args.steps))
            sampler = ClockSampler(gpu_identifier(torch, local)) if method == args.method else None
            if sampler:
                sampler.start()
                time.sleep(0.3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            stream.synchronize()
            clocks = sampler.stop() if sampler else None
        res[method] = (e0.elapsed_time(e1) / steps, clocks, outs[0].cpu().numpy())
        res_all[method] = outs.cpu().numpy()
        del ws_b, ws_l
    ms, clocks, c_tc = res[args.method]
    p_ms, _, c_plain = res.get("plain", (None, None, None))
    # every series of the timed method against the oracle at 10 lags
    err = None
    if not args.no_cpu_baseline:
        import oracle
        lags = np.unique(np.array([0, 1, 2, 383, 384, 767, 768, tm // 2, tm - 1, tm]))
        worst = 0.0
        for j, a in enumerate([longh] + shorth):
            ref = oracle.acf(a, stride=1, lags=lags)
            worst = max(worst, float(np.max(np.abs(res_all[args.method][j][lags] - ref)) / abs(ref[0])))
        err = {"series": 1 + len(shorth), "lags_per_series": int(len(lags)), "acf_max_abs_over_c0": worst,
               "tolerance": 1e-6 if args.method == "plain" else 1e-5}
    from paper_1708_08619_gb300 import shard
    ms = shard.max_over_ranks(ms)
    value = u * world / (ms / 1000.0)
    pk, pk_kind = peaks()
    achieved = 6.0 * u / (ms / 1000.0) / 1e12
    line = {"metric": "origin.lag pairs/s of the 3-component flux ACF", "value": value, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.method,
            "data": "synthetic",
            "config": {"workload": wl["label"], "pairs_per_step": u, "plain_ms_per_step": p_ms,
                       "speedup_vs_plain": p_ms / ms if p_ms else None,
                       "max_diff_tc_vs_plain_over_C0": (float(np.max(np.abs(c_tc - c_plain)) / abs(c_plain[0]))
                                                        if c_plain is not None else None),
                       "error_vs_oracle": err,
                       "l2": "long series 24 MB (fits L2); operand copies 0.2 GB"},
            "clocks": clocks, "e2e": None,
            # per step: long series (row max, prep, Gram, reduction) + the batch (5 descriptor
            # uploads, row max, prep, Gram, reduction) + one Green-Kubo integral for all series
            # (counted in an ncu launch list of the flux workload)
            "gpu_launches": (4 + 9 + 1) * args.steps if args.method != "plain" else None,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": pk.get("bf16_tflops", 1900.0),
                         "unit": "TFLOP/s", "frac": achieved / pk.get("bf16_tflops", 1900.0), "traffic": None,
                         "kernel": "gram_band_kernel (polyphase)",
                         "note": f"useful FLOPs (6 per pair) / step time, {pk_kind} bf16 peak"},
            "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_viscosity_workload(args, wl):
    """One long flux series with a correlation window of a quarter of its length
    (the paper's viscosity case: 2e6 points, window 5e5): the ACF and its running
    integral by the FFT route and by the polyphase tensor-core form, each checked
    against the oracle at sampled lags.  (The plain kernel's per-tile partial sums
    would need about 125 GB of workspace at this window.)"""
    import torch
    import oracle
    from paper_1708_08619_gb300 import build as tbuild
    from paper_1708_08619_gb300 import synth, tcorr

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tbuild.build()
    tcorr.load()
    Tn, tm = wl["T"], wl["tau_max"]
    xh = synth.ar1_flux(Tn, wl["phi"], seed=synth.BASE_SEED + 7 + 100 * rank)
    x = torch.from_numpy(xh).to(dev)
    u = updates(1, Tn, tm, 1)
    lags = np.unique(np.concatenate([[0, 1, 2, tm], np.linspace(0, tm, 61).astype(np.int64)]))
    ref = oracle.acf(xh, stride=1, lags=lags) if not args.no_cpu_baseline else None
    stream = torch.cuda.Stream(dev)
    res = {}
    for method in ("fft", "fp16x3"):
        out = torch.empty(tm + 1, dtype=torch.float64, device=dev)
        gk = torch.empty(tm + 1, dtype=torch.float64, device=dev)
        ws = torch.empty(max(256, tcorr.tcorr_workspace_size(Tn, 1, tm, 1, method)), dtype=torch.uint8, device=dev)
        steps = args.steps if method == "fft" else max(1, min(2, args.steps))
        with torch.cuda.stream(stream):
            def step():
                tcorr.tcorr_acf(x, tm, 1, method, out=out, ws=ws, stream=stream)
                tcorr.gk_integrate(out, 1.0, 1.0 / 3.0, out=gk, stream=stream)
            for _ in range(max(3, args.warmup) if method == "fft" else 1):
                step()
            stream.synchronize()
            sampler = ClockSampler(gpu_identifier(torch, local)) if method == "fft" else None
            if sampler:
                sampler.start()
                time.sleep(0.3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                step()
            e1.record(stream)
            stream.synchronize()
            clocks = sampler.stop() if sampler else None
        got = out.cpu().numpy()
        err = float(np.max(np.abs(got[lags] - ref)) / abs(ref[0])) if ref is not None else None
        res[method] = {"ms_per_step": e0.elapsed_time(e1) / steps, "err_over_c0": err, "clocks": clocks}
        del ws
    ms = res["fft"]["ms_per_step"]
    line = {"metric": "origin.lag pairs/s of the 3-component flux ACF, long window", "value": u / (ms / 1000.0),
            "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "double-float transforms (fft)", "data": "synthetic",
            "config": {"workload": wl["label"], "pairs_per_step": u,
                       "methods": {m: {"ms_per_step": r["ms_per_step"], "err_vs_oracle_over_c0": r["err_over_c0"]}
                                   for m, r in res.items()},
                       "fft_speedup_vs_polyphase_tc": res["fp16x3"]["ms_per_step"] / ms,
                       "oracle_lags": int(len(lags))},
            "clocks": res["fft"]["clocks"], "e2e": None,
            # this library's kernels per FFT step: twiddles, gather, column pass, fused row pass
            # (forward, power spectrum, inverse), inverse column pass, lag sum, finalize, Green-Kubo
            "gpu_launches": 8 * args.steps,
            "roofline": None, "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_collective_workload(args, wl):
    """Collective quantities on the water-scale arrays: the charge-weighted atom sums of the
    positions (referenced to the middle frame) and of the velocities, the Einstein-Helfand
    MSD of the first and the autocorrelation and running integral of the second.  The
    collective kernel (one read of a 3.93 GB array) is also timed alone for its roofline, and
    a mass-weighted MSD of the positions is timed beside the unweighted one."""
    import torch
    import oracle
    from paper_1708_08619_gb300 import build as tbuild
    from paper_1708_08619_gb300 import synth, tcorr

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tbuild.build()
    tcorr.load()
    N, T, tm = wl["N"], wl["T"], wl["tau_max"]
    seed = synth.BASE_SEED + 100 * rank
    x = synth.random_walk_positions_device(T, N, wl["sigma"], wl["box"], seed, device=dev,
                                           sites_per_molecule=wl["sites"])
    v = synth.ou_velocities_device(T, N, wl["gamma"], 1.0, seed + 1, device=dev)
    site = torch.arange(N, device=dev) % 3
    q = torch.where(site == 0, -0.8476, 0.4238).to(torch.float32)
    mass = torch.where(site == 0, 15.999, 1.008).to(torch.float32)
    jx = torch.empty((T, 1, 3), dtype=torch.float32, device=dev)
    jv = torch.empty_like(jx)
    m_eh = torch.empty(tm + 1, dtype=torch.float64, device=dev)
    c_j = torch.empty_like(m_eh)
    gk = torch.empty_like(m_eh)
    ws_eh = torch.empty(max(256, tcorr.tcorr_workspace_size(T, 1, tm, 1, "fft")), dtype=torch.uint8, device=dev)
    ws_c = torch.empty(max(256, tcorr.tcorr_workspace_size(T, 1, tm, 1, args.method)), dtype=torch.uint8,
                       device=dev)
    stream = torch.cuda.Stream(dev)

    def step():
        tcorr.tcorr_collective(x, q, T // 2, out=jx, stream=stream)
        tcorr.tcorr_msd(jx, tm, 1, "fft", out=m_eh, ws=ws_eh, stream=stream)
        tcorr.tcorr_collective(v, q, -1, out=jv, stream=stream)
        tcorr.tcorr_acf(jv, tm, 1, args.method, out=c_j, ws=ws_c, stream=stream)
        tcorr.gk_integrate(c_j, wl["dt"], 1.0, out=gk, stream=stream)

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / reps

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            step()
        stream.synchronize()
        sampler = ClockSampler(gpu_identifier(torch, local))
        sampler.start()
        time.sleep(0.3)
        ms = timed(step, args.steps)
        clocks = sampler.stop()
        col_ms = timed(lambda: tcorr.tcorr_collective(x, q, -1, out=jx, stream=stream), 10)
        col_ref_ms = timed(lambda: tcorr.tcorr_collective(x, q, T // 2, out=jx, stream=stream), 10)
        ws_w = torch.empty(tcorr.tcorr_weighted_workspace_size(T, N, tm, 1, args.method), dtype=torch.uint8,
                           device=dev)
        mo = torch.empty(tm + 1, dtype=torch.float64, device=dev)
        tcorr.tcorr_msd_weighted(x, mass, tm, 1, args.method, out=mo, ws=ws_w, stream=stream)
        w_ms = timed(lambda: tcorr.tcorr_msd_weighted(x, mass, tm, 1, args.method, out=mo, ws=ws_w,
                                                       stream=stream), 3)
        u_ms = timed(lambda: tcorr.tcorr_msd(x, tm, 1, args.method, out=mo, ws=ws_w, stream=stream), 3)
        del ws_w
    err = None
    if not args.no_cpu_baseline and rank == 0:
        # the oracle chain on a frame subset is too slow at this size; check the collective
        # signal itself on 16 frames and the correlations of the device-formed signals
        fr = np.linspace(0, T - 1, 16).astype(np.int64)
        xs = x[fr].cpu().numpy()
        xr = x[T // 2].cpu().numpy()[None]
        qh = q.cpu().numpy()
        want = oracle.collective(np.concatenate([xs, xr]), qh, len(fr))[:-1]
        got = jx[fr].cpu().numpy().reshape(-1, 3)
        lags = np.array([0, 1, 2, 10, 100, 1000, tm])
        jxh, jvh = jx.cpu().numpy(), jv.cpu().numpy()
        tcorr.tcorr_collective(x, q, T // 2, out=jx, stream=stream)
        tcorr.tcorr_msd(jx, tm, 1, "fft", out=m_eh, ws=ws_eh, stream=stream)
        tcorr.tcorr_acf(jv, tm, 1, args.method, out=c_j, ws=ws_c, stream=stream)
        stream.synchronize()
        rm = oracle.msd(jxh, stride=1, lags=lags)
        rc = oracle.acf(jvh, stride=1, lags=lags)
        err = {"collective_max_abs_over_max": float(np.max(np.abs(got - want)) / np.max(np.abs(want))),
               "eh_msd_over_msd_tau_max": float(np.max(np.abs(m_eh.cpu().numpy()[lags] - rm)) / rm[-1]),
               "current_acf_over_c0": float(np.max(np.abs(c_j.cpu().numpy()[lags] - rc)) / abs(rc[0])),
               "lags": lags.tolist()}
    pk, pk_kind = peaks()
    gbs = 12.0 * N * T / (col_ms / 1000.0) / 1e9
    line = {"metric": "atom.frame terms/s of the collective sums", "value": 2.0 * N * T * world / (ms / 1000.0),
            "unit": "atom-frames/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 compensated sums; double-float transforms (EH MSD); " + args.method + " (current ACF)",
            "data": "synthetic",
            "config": {"workload": wl["label"], "N": N, "T": T, "tau_max": tm,
                       "collective_ms": col_ms, "collective_ref_ms": col_ref_ms,
                       "mass_weighted_msd_ms": w_ms, "unweighted_msd_ms": u_ms,
                       "error_vs_oracle": err, "l2": "inputs larger than L2 (2 x 3.93 GB), no flush"},
            "clocks": clocks, "e2e": None,
            # per step: 2 collective, FFT-route MSD (twiddles, gather, column pass, fused row pass,
            # inverse column pass, lag sum, S, S prefix, finalize), polyphase ACF (row max, split,
            # Gram, reduce), Green-Kubo
            "gpu_launches": 16 * args.steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk.get("hbm_gbs", 6800.0), "unit": "GB/s",
                         "frac": gbs / pk.get("hbm_gbs", 6800.0),
                         "traffic": COLLECTIVE_WATER_TRAFFIC_BYTES if (N, T) == (32768, 10000) else None,
                         "kernel": "collective_kernel",
                         "note": f"12 bytes per atom and frame read once / the kernel alone (CUDA events "
                                 f"around 10 launches, no reference frame), {pk_kind} copy bandwidth"},
            "cpu_baseline": None}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--method", default=os.environ.get("TCORR_BENCH_METHOD", "fp16x3"))
    ap.add_argument("--no-plain-compare", action="store_true")
    ap.add_argument("--workload", default="precision", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stream-chunk", type=int, default=0,
                    help="origins per window of the streamed end-to-end calls (0: the workload's default)")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    elif args.workload == "batch":
        run_batch_workload(args, wl)
    elif args.workload == "flux":
        run_flux_workload(args, wl)
    elif args.workload == "viscosity":
        run_viscosity_workload(args, wl)
    elif args.workload == "collective":
        run_collective_workload(args, wl)
    else:
        run_gpu(args, wl)


if __name__ == "__main__":
    main()
