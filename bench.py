#!/usr/bin/env python
"""Throughput of the propagation of a 4D cross-spectral density on GB300.

Metric: 4D CSD points propagated per second (N^4 / time of one full propagation step) and the
HBM-roofline fraction of the dominant kernel.  One step = reset to the source plane, the source
(GSM x mask), Fresnel propagation (pass A: source build + input propagators + point-2 2D DFT;
pass B: point-1 2D DFT + output propagators + S), then S and mu(P1, .) of the output plane.

Default workload (the headline line): N = 256 (4.3 G points, complex64 CSDA of 34 GB), GSM x a
seeded unit-modulus phase screen (3 px correlation), dxi = 20 um, lambda = 633 nm, sigma_S =
0.1 mm, sigma_mu = 0.05 mm, z = 0.5 m.  Inside the same line, under "n128": N = 128 (2.1 GB),
GSM x 0.8 mm aperture x f = 0.3 m thin lens, z = 0.3 m.  Each is timed in blocks of --steps
steps (CUDA events), repeated until the blocks span at least 0.5 s; the median block is reported.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]

N > 1 runs under torch.distributed.run: each rank propagates its own copy of the workload
(independent replicas, no collective on the data path), so the job processes N x N^4 points
per step ("scaling": "weak"); time is the maximum over ranks.

--impl reference times the FP64 CPU oracle (the reference arm of this build) on the host
cores, each step one oracle propagation of the same configuration on an N = 64 grid.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as WL  # noqa: E402

WORKLOADS = {WL.GSM_APERTURE_LENS_N128["name"]: WL.GSM_APERTURE_LENS_N128,
             WL.PHASE_SCREEN_N256["name"]: WL.PHASE_SCREEN_N256,
             WL.POLYCHROMATIC_BATCH["name"]: WL.POLYCHROMATIC_BATCH,
             WL.INVERSE_N96["name"]: WL.INVERSE_N96,
             WL.PADDED_PHASE_SCREEN_N200["name"]: WL.PADDED_PHASE_SCREEN_N200,
             WL.PADDED_PHASE_SCREEN_N80["name"]: WL.PADDED_PHASE_SCREEN_N80}
# The headline: the largest single-GPU configuration (N = 256, 34 GB per CSDA); the N = 128
# configuration is measured in the same run and reported inside the same line.
DEFAULT_WORKLOAD = WL.PHASE_SCREEN_N256["name"]
CFG = WORKLOADS[DEFAULT_WORKLOAD]
METRIC = "4D CSD points propagated/s (Fresnel, N^4) and % HBM roofline vs plain FP32 path"
UNIT = "points/s"
SAMPLE_N = 64  # grid of the bounded CPU sample of the same configuration


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD,
                   help="default: the N = 256 phase-screen workload (with the N = 128 one inside its line)")
    p.add_argument("--headline-only", action="store_true",
                   help="with the default workload: skip the N = 128 measurement reported inside the line")
    p.add_argument("--skip-cpu", action="store_true",
                   help="leave out the two CPU baselines (for profiler runs of the GPU kernels)")
    p.add_argument("--dft", choices=["auto", "fp32", "tc_bf16x3"], default="auto",
                   help="arithmetic of the DFT work with a tensor-core form (the N = 256 first stage, the dense "
                        "contractions of padded workloads): auto (the library's per-path default), FP32 on the "
                        "CUDA cores, or split-BF16x3 on the tensor cores")
    a = p.parse_args()
    global CFG
    CFG = WORKLOADS[a.workload]
    return a


def source_mask_host(N, cfg=None):
    """Host-side (complex64) mask input of the workload: the aperture as a user mask for the N = 128
    workload, the seeded phase screen for the N = 256 one."""
    import numpy as np
    cfg = cfg or CFG
    if "corr_px" in cfg:
        return WL.to_c64(WL.phase_screen(N, seed=WL.SEED, corr_px=cfg["corr_px"]))
    n = np.arange(N)
    r2 = (n[:, None] - N // 2) ** 2 + (N // 2 - n[None, :]) ** 2
    rp = cfg["aperture"] / cfg["dxi"]
    return (r2 <= rp * rp).astype(np.complex64)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------------- CPU oracle
def sample_n():
    """Grid (and padded size) of the bounded CPU sample of the workload."""
    return CFG.get("sample_N", SAMPLE_N), CFG.get("sample_Nz")


def oracle_sample_step():
    """One FP64 oracle propagation of the workload's configuration on the sample grid (zero-padded
    to the sample's Nz for a padded workload), including the source build, S and mu.  Returns the
    number of points propagated."""
    import oracle as O
    N, Nz = sample_n()
    if "corr_px" in CFG:
        m = WL.phase_screen(N, seed=WL.SEED, corr_px=CFG["corr_px"])
    else:
        m = O.circle_aperture(N, CFG["dxi"], CFG["aperture"]) * O.thin_lens(N, CFG["dxi"], CFG["lam"], CFG["lens_f"])
    W0 = O.apply_mask(O.gsm_source(N, CFG["dxi"], CFG["sigma_S"], CFG["sigma_mu"], CFG["A"]), m)
    if Nz:
        W, _ = O.propagate_padded(W0, CFG["dxi"], CFG["lam"], CFG["z"], Nz)
    else:
        W, _ = O.propagate_fft(W0, CFG["dxi"], CFG["lam"], CFG["z"])
    O.spectral_density(W)
    O.degree_of_coherence(W, N // 2, N // 2)
    return N ** 4


def cpu_baseline(min_s=10.0, max_s=30.0):
    t0 = time.perf_counter()
    pts = 0
    runs = 0
    while True:
        pts += oracle_sample_step()
        runs += 1
        el = time.perf_counter() - t0
        if el >= min_s or el + el / runs > max_s:
            break
    return {"value": pts / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "FP64 NumPy oracle (single-threaded) on the same configuration at N=%s, %d full "
                      "propagation(s) incl. source build, S and mu, %.1f s" % (sample_desc(), runs, el)}


PLAIN_N_MAX = 128  # largest grid the plain FP32 CPU path runs at (N = 128: 2.1 GB per CSDA copy)


def sample_desc():
    N, Nz = sample_n()
    return "%d (zero-padded to Nz=%d)" % (N, Nz) if Nz else "%d" % N


def cpu_plain_fp32(max_s=30.0):
    """The plain FP32 CPU path (complex64, scipy.fft on every host core) on the workload's
    configuration, at the workload's N up to PLAIN_N_MAX (the same configuration at that grid
    above it).  One untimed propagation at N = 32 first (imports, FFT plans)."""
    import numpy as np
    import oracle as O
    from oracle import plain_fp32 as P
    N = min(CFG["N"], PLAIN_N_MAX)
    Nz = None
    if "Nz" in CFG:  # padded: the sample grid, FFTs at the sample's padded size, output cropped
        N, Nz = sample_n()

    def mask(n):
        if "corr_px" in CFG:
            return WL.phase_screen(n, seed=WL.SEED, corr_px=CFG["corr_px"])
        return O.circle_aperture(n, CFG["dxi"], CFG["aperture"]) * O.thin_lens(n, CFG["dxi"], CFG["lam"],
                                                                               CFG["lens_f"])

    def step(n):
        if Nz and n == N:
            o = (Nz - N) // 2
            mp = np.zeros((Nz, Nz), dtype=np.complex128)
            mp[o:o + N, o:o + N] = mask(N)  # the source on the padded grid, zeros around it
            W, S, mu, _ = P.propagate_gsm_fp32(Nz, CFG["dxi"], CFG["lam"], CFG["z"], CFG["sigma_S"],
                                               CFG["sigma_mu"], CFG["A"], mask=mp)
            return W[o:o + N, o:o + N, o:o + N, o:o + N]
        P.propagate_gsm_fp32(n, CFG["dxi"], CFG["lam"], CFG["z"], CFG["sigma_S"], CFG["sigma_mu"], CFG["A"],
                             mask=mask(n))

    step(32)
    runs, t0 = 0, time.perf_counter()
    while True:
        step(N)
        runs += 1
        el = time.perf_counter() - t0
        if el + el / runs > max_s or (el >= 6.0 and runs >= 3):
            break
    return {"value": runs * N ** 4 / el, "unit": UNIT, "cores": P.host_cores(), "kind": "plain FP32 path",
            "sample": "complex64 array operations + scipy.fft (Algorithm 2 order) on the host cores, the same "
                      "configuration at N=%s, %d full propagation(s) incl. source build, S and mu, %.1f s"
                      % ("%d (zero-padded to Nz=%d)" % (N, Nz) if Nz else "%d" % N, runs, el)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample_step()
    t0 = time.perf_counter()
    pts = 0
    for _ in range(args.steps):
        pts += oracle_sample_step()
    el = time.perf_counter() - t0
    v = pts / el
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": CFG["name"], "N": sample_n()[0], "Nz": sample_n()[1], "sample_of_N": CFG["N"]},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: one FP64 oracle propagation of the configuration at "
                                       "N=%s on the host cores (NumPy, single-threaded)" % sample_desc()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU helpers
# Per grid size: the committed ncu summary of its pass kernels and the device-code headers they
# are built from (a recorded traffic figure is used only while those headers are unchanged).
PROFILED = {128: ("pass_kernels_n128.md", ("cluster.cuh", "fft.cuh", "propagate.cuh", "r128.cuh")),
            256: ("pass_kernels_n256.md", ("fft.cuh", "propagate.cuh", "r128.cuh", "t256.cuh", "tc16.cuh"))}


def kernel_source_sha(N=128):
    """Hash of the device-code headers the pass kernels at grid size N are built from."""
    h = hashlib.sha256()
    for name in PROFILED[N][1]:
        h.update(open(os.path.join(ROOT, "paper_2203_02734_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def measured_peak_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(kernel, N):
    """DRAM bytes per launch of `kernel` at grid size N from the committed ncu summary, or None
    when there is none or the kernel sources changed since it was taken."""
    if N not in PROFILED:
        return None
    try:
        txt = open(os.path.join(ROOT, "profiles", PROFILED[N][0])).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch %s (\d+) sha=(\w+)" % kernel, txt)
    if not m or m.group(2) != kernel_source_sha(N):
        return None
    return int(m.group(1))


def roofline_dense(N, pts, avg_a, avg_b, clocks, tc):
    """Padded workloads: four dense axis contractions, N complex multiply-adds (8 flop) per output
    point each; the second pass's events span two contractions.
    CUDA cores (tc False): FP32 FMA work against SMs x 128 FP32 lanes x 2 flop x the maximum SM clock.
    Tensor cores (tc True): the BF16 MMA flops one launch issues, ceil(N^3 / 128) tiles x
    Np / 16 chunks x 24 MMAs of 2 x 128 x Np x 16 flop (Np = N rounded up to 16; six split products),
    against the measured BF16 peak."""
    import torch
    avg = avg_b / 2
    fp32_flops = 8.0 * N * pts
    if tc:
        Np = (N + 15) // 16 * 16
        tiles = (N ** 3 + 127) // 128
        flops = tiles * (Np // 16) * 24 * 2.0 * 128 * Np * 16
        try:
            peak, src = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]), "measured"
        except Exception:
            peak, src = 1900.0, "fallback"
        achieved = flops / (avg / 1e3) / 1e12
        return {"bound": "tensor", "kernel": "dense_tc::axis_tc_kernel", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": src + " (bf16, burst)", "traffic": None,
                "algorithmic_flops_per_launch": flops,
                "fp32_equivalent_tflops": fp32_flops / (avg / 1e3) / 1e12,
                # the method's own work (8 N flop per output point) against the split-BF16x3 ceiling:
                # each FP32 product costs six BF16 products, so at most peak / 6 of FP32 work
                "method_work": {"achieved": fp32_flops / (avg / 1e3) / 1e12, "ceiling": peak / 6.0,
                                "frac": fp32_flops / (avg / 1e3) / 1e12 / (peak / 6.0), "unit": "TFLOP/s"},
                "pass_ms": {"pass_a": avg_a, "pass_b": avg_b}}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    peak = sms * 128 * 2 * mhz * 1e6 / 1e12
    achieved = fp32_flops / (avg / 1e3) / 1e12
    return {"bound": "alu", "kernel": "dense::axis_kernel", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 flop x %.0f MHz" % (sms, mhz),
            "traffic": None, "algorithmic_flops_per_launch": fp32_flops,
            "pass_ms": {"pass_a": avg_a, "pass_b": avg_b}}


def max_over_ranks(x, dist, device):
    """Maximum of a float over all ranks (identity without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, pts_per_step, steps, seconds):
    """Whole-job points/s: every rank propagates its own workload (weak scaling)."""
    return world * pts_per_step * steps / seconds


class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "20", "-i", str(index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self, t0, t1):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = []
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[5:]))
            except (ValueError, IndexError):
                continue
        os.unlink(self.f.name)
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05]
        note = None
        if not inside and rows:
            inside = sorted(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))[:3]
            note = "timed region shorter than the sampling period: nearest samples"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3][1:5]) if v.lower() == "active"})
        out = {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
               "reasons": reasons, "samples": len(inside)}
        if note:
            out["note"] = note
        return out


def timed_blocks(run_block, stream, min_s=0.5, min_blocks=3, max_blocks=400):
    """Run blocks of steps, each bracketed by CUDA events on `stream` (synchronised after each block),
    until the blocks together span >= min_s seconds of device time and at least min_blocks ran.
    Returns the device milliseconds of every block."""
    import torch
    ms = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    while len(ms) < max_blocks and (len(ms) < min_blocks or sum(ms) < 1e3 * min_s):
        torch.cuda.synchronize()
        e0.record(stream)
        run_block()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def measure(cfg, args, rank, world, dist):
    """One workload of single propagations through the library: device-timed blocks of
    `args.steps` steps, the per-pass times, the end-to-end blocks with host buffers, and the
    roofline of the dominant pass.  Returns the fields of a bench line (rank 0) or None."""
    import torch
    import paper_2203_02734_gb300 as pw

    N = cfg["N"]
    stream = torch.cuda.current_stream()
    W = torch.empty((N,) * 4, dtype=torch.complex64, device="cuda")
    work = torch.empty((N,) * 4, dtype=torch.complex64, device="cuda")
    S = torch.empty((N, N), dtype=torch.float32, device="cuda")
    mu = torch.empty((N, N), dtype=torch.complex64, device="cuda")
    c = pw.CSD(N, cfg["dxi"], cfg["lam"], W=W, work=work, stream=stream)
    h = c.h
    P1 = cfg["P1"]
    pw.pw_csd_set_dft_mode(h, {"auto": pw.PW_DFT_AUTO, "fp32": pw.PW_DFT_FP32,
                               "tc_bf16x3": pw.PW_DFT_TC_BF16X3}[args.dft])
    if cfg.get("Nz"):
        pw.pw_csd_set_padding(h, cfg["Nz"])

    screen = "corr_px" in cfg
    mask_dev0 = torch.from_numpy(source_mask_host(N, cfg)).cuda() if screen else None

    def step():
        pw.pw_csd_reset(h, cfg["dxi"])
        pw.pw_source_gsm(h, cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
        if screen:
            pw.pw_source_mask(h, mask_dev0.data_ptr())
        else:
            pw.pw_source_aperture(h, cfg["aperture"])
            pw.pw_source_lens(h, cfg["lens_f"])
        pw.pw_propagate_fresnel(h, cfg["z"])
        pw.pw_spectral_density(h, S.data_ptr())
        pw.pw_degree_of_coherence(h, P1[0], P1[1], mu.data_ptr())

    def block():
        for _ in range(args.steps):
            step()

    # tables, pass A, pass B, S kernel, mu kernel (N = 256: three passes); padded: tables, dense
    # tables, source, four axis contractions (+ two matrix splits on the tensor cores), S, mu
    launches_per_step = ((11 if args.dft != "fp32" and N <= 256 else 9) if cfg.get("Nz")
                         else (6 if N == 256 and args.dft != "tc_bf16x3" else 5))
    max_blocks = 400
    pw.pw_csd_enable_timing(h, max(args.steps * max_blocks, args.warmup, 1))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pw.pw_csd_pass_times(h)  # discard warm-up records
    clock = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if dist:
        dist.barrier()
    t0 = time.time()
    blocks = timed_blocks(block, stream, max_blocks=max_blocks)
    t1 = time.time()
    if dist:
        dist.barrier()
    ms = statistics.median(blocks)
    ms_a, ms_b, ms_c, nrec = pw.pw_csd_pass_times3(h)
    clocks = clock.stop(t0, t1) if clock else None
    ms = max_over_ranks(ms, dist, "cuda")

    # End to end through the public API with host buffers: each step copies the source mask (the
    # aperture as a user mask for the N = 128 workload, the phase screen for N = 256) from pinned
    # host memory to the device and reads S and mu back into pinned host memory; the same
    # configuration as above, so the result is identical.
    mask_h = torch.from_numpy(source_mask_host(N, cfg)).pin_memory()
    mask_d = torch.empty_like(mask_h, device="cuda")
    S_h = torch.empty((N, N), dtype=torch.float32).pin_memory()
    mu_h = torch.empty((N, N), dtype=torch.complex64).pin_memory()

    def step_e2e():
        mask_d.copy_(mask_h, non_blocking=True)
        pw.pw_csd_reset(h, cfg["dxi"])
        pw.pw_source_gsm(h, cfg["sigma_S"], cfg["sigma_mu"], cfg["A"])
        pw.pw_source_mask(h, mask_d.data_ptr())
        if not screen:
            pw.pw_source_lens(h, cfg["lens_f"])
        pw.pw_propagate_fresnel(h, cfg["z"])
        pw.pw_spectral_density(h, S.data_ptr())
        pw.pw_degree_of_coherence(h, P1[0], P1[1], mu.data_ptr())
        S_h.copy_(S, non_blocking=True)
        mu_h.copy_(mu, non_blocking=True)

    S_ref = S.clone()
    for _ in range(args.warmup):
        step_e2e()
    torch.cuda.synchronize()
    same = bool(torch.equal(S_h, S_ref.cpu()))
    if dist:
        dist.barrier()
    e2e_blocks = []
    while len(e2e_blocks) < 3 or sum(e2e_blocks) < 0.5:
        torch.cuda.synchronize()
        te0 = time.perf_counter()
        for _ in range(args.steps):
            step_e2e()
        torch.cuda.synchronize()
        e2e_blocks.append(time.perf_counter() - te0)
    te = max_over_ranks(statistics.median(e2e_blocks), dist, "cuda")
    pw.pw_csd_pass_times(h)
    c.close()
    del W, work
    torch.cuda.empty_cache()
    if rank != 0:
        return None

    pts = N ** 4
    value = job_throughput(world, pts, args.steps, ms / 1e3)
    peak, peak_kind = measured_peak_hbm()
    avg_a, avg_b, avg_c = (x / max(nrec, 1) for x in (ms_a, ms_b, ms_c))
    if avg_c > 0:  # N = 256: three streaming passes, 8 + 16 + 16 bytes per point
        passes = {"pass1": (avg_a, 8 * pts), "pass2": (avg_b, 16 * pts), "pass3": (avg_c, 16 * pts)}
        engine_bytes = 40
    else:  # two passes, 8 + 16 bytes per point
        passes = {"pass_a": (avg_a, 8 * pts), "pass_b": (avg_b, 16 * pts)}
        engine_bytes = 24
    kern = max(passes, key=lambda k: passes[k][0])
    avg, bytes_launch = passes[kern]
    achieved = bytes_launch / (avg / 1e3) / 1e9
    return {
        "value": value, "ms_per_step": ms / args.steps,
        "config": {"workload": cfg["name"], "N": N, "dft_first_stage": args.dft, "points_per_step": pts,
                   "dxi_m": cfg["dxi"],
                   "lambda_m": cfg["lam"], "z_m": cfg["z"], "aperture_m": cfg.get("aperture"),
                   "lens_f_m": cfg.get("lens_f"), "phase_screen_corr_px": cfg.get("corr_px"), "P1": list(P1),
                   "parallelism": "replicas x%d" % world,
                   "l2": "inputs larger than L2: 2 x %.1f GB CSDA buffers stream through HBM every step"
                         % (8 * pts / 1e9),
                   "timing": "median of %d blocks of %d steps (%.2f s of device time in all)"
                             % (len(blocks), args.steps, sum(blocks) / 1e3)},
        "roofline": roofline_dense(N, pts, avg_a, avg_b, clocks, args.dft != "fp32" and N <= 256) if cfg.get("Nz") else
                    {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_kind, "traffic": recorded_traffic(kern, N),
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "pass_ms": {k: v[0] for k, v in passes.items()},
                     "pass_hbm_frac": {k: v[1] / (v[0] / 1e3) / 1e9 / peak for k, v in passes.items()},
                     "engine_bytes_per_point": engine_bytes,
                     "step_hbm_frac": (24 * pts / (ms / args.steps / 1e3) / 1e9) / peak,
                     "step_hbm_frac_note": "24 bytes per point, the two-pass minimum of the method, over "
                                           "the measured peak"},
        "e2e": {"value": job_throughput(world, pts, args.steps, te), "unit": UNIT,
                "h2d_bytes_per_step": mask_h.numel() * 8, "d2h_bytes_per_step": S_h.numel() * 4 + mu_h.numel() * 8,
                "result_matches_device_path": same},
        "gpu_launches": launches_per_step * args.steps,
        "gpu_launches_per_step": launches_per_step,
        "clocks": clocks,
    }


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # The headline workload (by default N = 256, the largest single-GPU configuration); with it, the
    # N = 128 workload is measured the same way and reported inside the same line.
    second = None
    if CFG is WL.PHASE_SCREEN_N256 and not args.headline_only:
        second = measure(WL.GSM_APERTURE_LENS_N128, args, rank, world, dist)
    r = measure(CFG, args, rank, world, dist)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    line = {"metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    for k in ("config", "roofline", "e2e", "gpu_launches", "gpu_launches_per_step", "clocks"):
        line[k] = r[k]
    if second is not None:
        line["n128"] = {k: second[k] for k in ("value", "ms_per_step", "config", "roofline", "e2e", "clocks")}
        line["n128"]["unit"] = UNIT
    if world == 1 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline()
        line["cpu_plain_fp32"] = cpu_plain_fp32()
    print(json.dumps(line), flush=True)


def batch_instances():
    """The polychromatic workload: 16 frequencies of a Gaussian spectrum (weights as GSM
    amplitudes) x N in {64, 96, 128} x z in {0.1, 0.5, 1, 5} m = 192 instances."""
    lams, wts = WL.polychromatic_samples(CFG["lam0"], CFG["fwhm_lam"], CFG["n_freq"])
    out = []
    for lam, wt in zip(lams, wts):
        for N in CFG["Ns"]:
            for z in CFG["zs"]:
                out.append(dict(N=N, lam=float(lam), A=float(wt), z=z))
    return out


def run_batch(args):
    """Batched polychromatic run: all instances in one persistent launch, captured once in a CUDA
    graph and replayed; S and mu of every instance.  Reported next to the plain path (the
    single-instance calls, one instance after the other) on the same GPU."""
    import torch
    import paper_2203_02734_gb300 as pw

    torch.cuda.set_device(0)
    specs = batch_instances()
    s = torch.cuda.Stream()
    bufs, insts = [], []
    for sp in specs:
        N = sp["N"]
        S = torch.empty((N, N), dtype=torch.float32, device="cuda")
        mu = torch.empty((N, N), dtype=torch.complex64, device="cuda")
        bufs.append((S, mu))
        insts.append(pw.pw_instance(N, CFG["dxi"], sp["lam"], sp["z"], 0, CFG["sigma_S"], CFG["sigma_mu"], sp["A"],
                                    0.0, 0.0, None, N // 2, N // 2, None, S.data_ptr(), mu.data_ptr()))
    pool = 4
    nb = pw.pw_batch_workspace_bytes(insts, pool)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    b = pw.pw_batch_create(insts, pool, ws.data_ptr(), nb, s.cuda_stream)
    chunk = pw.pw_batch_autotune(b)
    mode = "persistent launch" if pw.pw_batch_get_mode(b) == pw.PW_BATCH_PERSISTENT else "sequenced launches"
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        pw.pw_batch_run(b)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clock = ClockSampler(torch.cuda.current_device())
    t0 = time.time()
    e0.record()
    for _ in range(args.steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    t1 = time.time()
    clocks = clock.stop(t0, t1)
    pw.pw_batch_check(b)
    ms = e0.elapsed_time(e1) / args.steps
    pts = sum(sp["N"] ** 4 for sp in specs)
    # plain path: the same instances through the single-instance calls, one after the other
    maxN = max(sp["N"] for sp in specs)
    W = torch.empty(maxN ** 4, dtype=torch.complex64, device="cuda")
    work = torch.empty(maxN ** 4, dtype=torch.complex64, device="cuda")
    # one handle per (N, wavelength): create them up front (not timed)
    hl = {}
    for sp in specs:
        key = (sp["N"], sp["lam"])
        if key not in hl:
            hl[key] = pw.pw_csd_create(sp["N"], CFG["dxi"], sp["lam"], W.data_ptr(), W.numel() * 8, work.data_ptr(),
                                       work.numel() * 8, torch.cuda.current_stream().cuda_stream)

    def plain_exact():
        for sp, (S, mu) in zip(specs, bufs):
            h = hl[(sp["N"], sp["lam"])]
            pw.pw_csd_reset(h, CFG["dxi"])
            pw.pw_source_gsm(h, CFG["sigma_S"], CFG["sigma_mu"], sp["A"])
            pw.pw_propagate_fresnel(h, sp["z"])
            pw.pw_spectral_density(h, S.data_ptr())
            pw.pw_degree_of_coherence(h, sp["N"] // 2, sp["N"] // 2, mu.data_ptr())

    plain_exact()
    torch.cuda.synchronize()
    e0.record()
    reps = max(1, min(args.steps, 5))
    for _ in range(reps):
        plain_exact()
    e1.record()
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1) / reps
    peak, peak_src = measured_peak_hbm()
    for h in hl.values():
        pw.pw_csd_destroy(h)
    pw.pw_batch_destroy(b)
    line = {"metric": METRIC, "value": pts / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CFG["name"], "instances": len(specs), "points_per_step": pts,
                       "Ns": list(CFG["Ns"]), "zs": list(CFG["zs"]), "n_freq": CFG["n_freq"],
                       "outputs": "S and mu per instance", "pool": pool, "chunk": chunk,
                       "launch": "autotuned mode: %s, replayed from a CUDA graph" % mode},
            "roofline": {"bound": "hbm", "kernel": "whole batch (V written by pass A, read by the S/mu pass)",
                         "achieved": 16.0 * pts / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": 16.0 * pts / (ms * 1e-3) / 1e9 / peak, "peak_source": peak_src, "traffic": None,
                         "algorithmic_bytes_per_point": 16},
            "plain_path": {"value": pts / (ms_plain / 1e3), "unit": UNIT, "ms_per_step": ms_plain,
                           "what": "the same instances through the single-instance calls, one after another"},
            "gpu_launches": (4 if mode.startswith("persistent") else 2 + 2 * len(specs)) * args.steps,
            "clocks": clocks}
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Differentiable workload (N = 96, z = 1 m, amplitude-masked GSM): one step = forward S and the
    backward pass of a least-squares S loss through the hand-written adjoint (gradients for sigma_S,
    sigma_mu, A and the N x N mask); reported next to the forward alone (the plain path)."""
    import torch
    from paper_2203_02734_gb300.autograd import GSMIntensity

    torch.cuda.set_device(0)
    N = CFG["N"]
    model = GSMIntensity(N, CFG["dxi"], CFG["lam"], CFG["z"])
    am = torch.tensor(WL.amplitude_mask(N).real, dtype=torch.float32, device="cuda", requires_grad=True)
    sS = torch.tensor(CFG["sigma_S"], dtype=torch.float64, requires_grad=True)
    sM = torch.tensor(CFG["sigma_mu"], dtype=torch.float64, requires_grad=True)
    A = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    with torch.no_grad():
        target = model(sS * 1.2, sM * 0.8, A, am * 0.9).double()

    def fwd_bwd():
        S = model(sS, sM, A, am)
        L = torch.sum((S.double() - target) ** 2)
        L.backward()

    def fwd():
        with torch.no_grad():
            model(sS, sM, A, am)

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / steps

    clock = ClockSampler(torch.cuda.current_device())
    t0 = time.time()
    t_fb = timed(fwd_bwd, args.steps)
    t1 = time.time()
    clocks = clock.stop(t0, t1)
    t_f = timed(fwd, args.steps)
    # device time of the forward (S, mu) and of the adjoint call alone: CUDA events around the library
    # calls, no host synchronisation inside (the autograd step above copies the three parameter
    # gradients back to host tensors, which synchronises every step)
    from paper_2203_02734_gb300 import abi
    m = model.m
    model.mask_c.real.copy_(am.detach())
    gS_dev = torch.randn(N, N, device="cuda", dtype=torch.float32)

    def dev_fwd():
        abi.pw_csd_reset(m.csd.h, m.dxi)
        abi.pw_source_gsm(m.csd.h, CFG["sigma_S"], CFG["sigma_mu"], 1.0)
        abi.pw_source_mask(m.csd.h, model.mask_c.data_ptr())
        m.propagate_and_read()

    def dev_bwd():
        m.adjoint(gS_dev, None, m.S, m.mu, sigma_S_m=CFG["sigma_S"], sigma_mu_m=CFG["sigma_mu"], amplitude=1.0,
                  dev_amask=am.data_ptr(), dev_grad3=m.g3.data_ptr(), dev_grad_amask=m.gmask.data_ptr())

    def dev_timed(fn, n):
        for _ in range(args.warmup):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(n):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    nd = max(args.steps, 50)
    d_f = dev_timed(dev_fwd, nd)
    d_b = dev_timed(dev_bwd, nd)
    model.close()
    pts = N ** 4
    line = {"metric": METRIC, "value": pts / t_fb, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_fb, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": CFG["name"], "N": N, "z_m": CFG["z"], "points_per_step": pts,
                       "step": "forward S + backward of a least-squares S loss (hand-written adjoint)"},
            "plain_path": {"value": pts / t_f, "unit": UNIT, "ms_per_step": 1e3 * t_f,
                           "what": "the forward propagation + S alone"},
            "device": {"forward_ms": d_f, "backward_ms": d_b, "backward_over_forward": d_b / d_f,
                       "what": "CUDA-event time of the forward (S, mu) and of one adjoint call, %d calls each" % nd},
            "gpu_launches": 7 * args.steps, "clocks": clocks}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
    elif CFG is WL.POLYCHROMATIC_BATCH:
        run_batch(a)
    elif CFG is WL.INVERSE_N96:
        run_adjoint(a)
    else:
        run_ours(a)
