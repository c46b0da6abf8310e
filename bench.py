#!/usr/bin/env python
"""Benchmark of the visibility MABS / 3D bispectrum hot path on GB300.

Metric: MABS bin-triple x channel evaluations per second (one evaluation = one
ring triple with at least one closed triangle x one ordered channel triple,
i.e. one value of Eq. estimator_t of arXiv:2506.10526).

Workload (default ``mwa``): the MWA-like configuration -- 256^2 uv grid,
768 channels, 20 log-spaced rings in |U| from 4.41 to 128 grid units,
image side M = 384, seeded quadratic non-Gaussian sky (f_NG = 0.5,
P(k) ~ k^-2), no flagging.  The full job is every ring triple x every channel
triple (768^3), far more than a minute of work, so one step is one pass of the
whole hot path over one channel block of the job: the grid load of all 768
channels (shell masks + inverse FFTs of all 15,360 fields), the triple
contraction of every closable ring triple over one B x B x B3 channel block
(128 x 128 x 256 for ``mwa``: the tensor-core tiles take 256 third-ring
fields at a time, so nu3 runs of 256 channels fill them), the collapse into
the (dnu1, dnu2) plane and the delay transform of Eq. (dft).
Consecutive steps (and ranks) take consecutive blocks of the job.

Timing: W untimed warm-up steps, then K steps between CUDA events on the
launching stream with a device synchronise and a barrier on both sides;
inputs (403 MB of visibilities, 9 GB of fields) exceed the 129 MB L2.
``e2e`` repeats the steps through the same C ABI starting from host memory:
each step copies the visibilities host->device and reads the 3D bispectrum
back.  ``--impl reference`` times the FP64 CPU oracle (the only reference
implementation: the paper ships no code) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "mwa": dict(nt=256, nc=768, nb=20, edges=("log", 4.41, 128.0), block=128, block3=256, cube=256,
                desc="MWA-like: 256^2 uv grid, 768 channels (30.72 MHz at 40 kHz), 20 log rings "
                     "|U| in [4.41, 128), no flagging"),
    "mwa64": dict(nt=256, nc=64, nb=20, edges=("log", 4.41, 128.0), block=64,
                  desc="profiling case: the MWA-like grid and rings with 64 channels"),
    "small": dict(nt=128, nc=128, nb=12, edges=("log", 2.2, 64.0), block=32, block3=128,
                  desc="profiling case: 128^2 uv grid, 128 channels, 12 log rings |U| in "
                       "[2.2, 64), no flagging"),
    "delay768": dict(nt=64, nc=768, nb=6, edges=("log", 2.0, 32.0), block=128, block3=256,
                     desc="profiling case: the MWA-like 768-channel delay axis on a 64^2 grid "
                          "with 6 log rings |U| in [2, 32)"),
    "tiny": dict(nt=64, nc=16, nb=8, edges=("linear", 0.0, 32.0), block=16,
                 desc="tiny: 64^2 uv grid, 16 channels, 8 linear rings |U| < 32, no flagging"),
}
SMS = 152
FP32_LANES_PER_SM = 128
PROFILES = {"fp32": (os.path.join(ROOT, "profiles", "contract_simt_mwa.txt"),
                     os.path.join(ROOT, "paper_2506_10526_gb300", "csrc", "contract_simt.cu")),
            "split_bf16": (os.path.join(ROOT, "profiles", "contract_tc_mwa.txt"),
                           os.path.join(ROOT, "paper_2506_10526_gb300", "csrc", "contract_tc.cu")),
            "split_fp16": (os.path.join(ROOT, "profiles", "contract_tc_fp16_mwa.txt"),
                           os.path.join(ROOT, "paper_2506_10526_gb300", "csrc", "contract_tc.cu"))}
# tensor-core products per algorithmic product, and the operand dtype label
SPLIT_PRODUCTS = {"split_bf16": 3, "split_fp16": 3}
DTYPE = {"fp32": "f32", "split_bf16": "bf16x3", "split_fp16": "fp16x3"}
# error targets against the FP64 oracle (kappa-normalised, and relative on
# well-conditioned bins) and the unit u of each arithmetic for the
# well-conditioned test kappa u <= tol / 10
TOL = {"fp32": 1e-5, "split_bf16": 1e-3, "split_fp16": 1e-4}
UNIT = {"fp32": 2.0 ** -24, "split_bf16": 2.0 ** -17, "split_fp16": 2.0 ** -22}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mwa", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="split_bf16",
                    choices=["fp32", "split_bf16", "split_fp16"])
    ap.add_argument("--no-multires", action="store_true",
                    help="one image side for every ring triple (split-BF16 path)")
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip timing the plain FP32 contraction beside the split-BF16 one")
    ap.add_argument("--block", type=int, default=0, help="channel block side (0 = workload default)")
    ap.add_argument("--block3", type=int, default=0,
                    help="channel block side along nu3 (0 = workload default)")
    ap.add_argument("--ordinary", action="store_true",
                    help="time ordinary channel blocks (block x block x block3) instead of "
                         "channel-symmetric sub-band cubes")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU baseline budget")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-mc", action="store_true",
                    help="skip the batched Monte Carlo and surrogate measurements")
    ap.add_argument("--only-surrogate", action="store_true",
                    help="run only the surrogate network measurement (profiling)")
    ap.add_argument("--only-mc-cfg4", type=int, default=None, metavar="SHAPE",
                    help="run only the batched Monte Carlo configuration, on one of its "
                         "shapes (index into the drawn shapes; profiling)")
    ap.add_argument("--cfg4-total", type=int, default=256,
                    help="realisations of the batched Monte Carlo configuration")
    ap.add_argument("--only-mc", action="store_true",
                    help="run only the batched Monte Carlo measurement (profiling)")
    return ap.parse_args()


def edges_of(w):
    import synth
    kind, lo, hi = w["edges"]
    return synth.edges_log(w["nb"], lo, hi) if kind == "log" else synth.edges_linear(w["nb"], hi)


def make_vis(w, seed):
    import numpy as np
    import synth
    return synth.sky_visibilities(w["nt"], w["nc"], seed, f_ng=0.5, sigma=0.5).astype(np.complex64)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # a run that fails before stop() must not leave the sampler running
            atexit.register(self._end)
        except OSError:
            self.proc = None

    def _end(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self._end()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) < 8:
                continue
            for k, n in enumerate(names):
                if r[4 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def profile_traffic(precision):
    """DRAM bytes per evaluation of the contraction from the committed ncu
    summary, valid only while the kernel source still has the hash recorded there."""
    prof, src = PROFILES[precision]
    if not os.path.exists(prof):
        return None
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    vals = {}
    for line in open(prof):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != h:
        return None
    try:
        return {"bytes_per_unit": float(vals["dram_bytes_per_eval"])}
    except (KeyError, ValueError):
        return None


def cpu_baseline(w, seconds, vis=None):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    uniformly sampled closable ring triples x the channel triples of the first
    4 channels, enumerated with all host cores until the time budget is used."""
    import numpy as np
    import oracle
    edges = edges_of(w)
    nsub = min(4, w["nc"])
    if vis is None:
        vis = make_vis(w, seed=2000)
    v = np.ascontiguousarray(vis[:nsub]).astype(np.complex128)
    T = oracle.counts(w["nt"], edges)
    trips = [t for t in oracle.ring_triples(w["nb"]) if T[t] > 0]
    rng = np.random.default_rng(12345)
    order = rng.permutation(len(trips))
    cores = os.cpu_count() or 1
    done = 0
    t0 = time.perf_counter()
    k = 0
    while k < len(order) and time.perf_counter() - t0 < seconds:
        chunk = [trips[i] for i in order[k:k + cores]]
        oracle.mabs_full(v, edges, triples=chunk, nthreads=cores)
        done += len(chunk)
        k += cores
    dt = time.perf_counter() - t0
    evals = done * nsub ** 3
    return {"value": evals / dt, "unit": "evals/s", "cores": cores, "kind": "oracle",
            "sample": f"FP64 closed-triangle enumeration of {done} uniformly sampled closable ring "
                      f"triples x {nsub}^3 channel triples (channels 0-{nsub - 1}) of the "
                      f"{w['nt']}^2 grid, {dt:.1f} s"}


def measure_error(plan, vis, edges, blk, out_delta, tri, precision, closable=True):
    """Error of a step's folded plane against the FP64 oracle, measured in this
    run: the oracle evaluates the collapsed mean over the block's channel
    triples at sampled points (the cheapest closable ring triples, and one of
    medium size; separations from channel triples inside the block), on V and
    on |V| (B_abs).  Reported: the kappa-normalised error |B - B64| / B_abs,
    the relative error, and the relative error of the well-conditioned points
    (kappa u <= tol / 10); and whether the library's own error bound
    (bs_mabs_error_bound) covers the measured error at every point."""
    import numpy as np
    import oracle
    import torch
    bound, _ = plan.error_bound()
    torch.cuda.synchronize()
    nc = vis.shape[0]
    trips = oracle.ring_triples(len(edges) - 1)
    clos = np.flatnonzero(tri > 0)
    pos = {int(t): k for k, t in enumerate(clos)}
    chosen = [int(t) for t in clos[:4]] + [int(clos[len(clos) // 5])]
    # and the first closable (i, j, j), i < j: its channel orderings nu2 > nu3 are
    # filled in from nu2 < nu3 under channel-symmetric accumulation
    chosen += [int(t) for t in clos if trips[t][0] < trips[t][1] == trips[t][2]][:1]
    b = blk
    mid3 = (b[4] + b[5]) // 2
    picks = [(b[0], b[2]), (b[1] - 1, b[3] - 1), ((b[0] + b[1]) // 2, b[2] + 1),
             (b[0] + 1, (b[2] + b[3]) // 2)]
    pts = []
    for n, t in enumerate(chosen):
        for n1, n2 in (picks[n % len(picks)], picks[(n + 1) % len(picks)]):
            pts.append((*trips[t], n1 - mid3, n2 - mid3))
    nmax = max(b[1], b[3], b[5])
    sub = np.ascontiguousarray(vis[:nmax]).astype(np.complex128)
    t0 = time.perf_counter()
    want, cnt = oracle.delta_points(sub, edges, pts, block=b)
    babs, _ = oracle.delta_points(np.abs(sub), edges, pts, block=b)
    dt = time.perf_counter() - t0
    got = np.array([out_delta[0, pos[trips.index(tuple(p[:3]))] if closable else
                              trips.index(tuple(p[:3])), p[3] + nc - 1, p[4] + nc - 1].item()
                    for p in pts])
    beta = np.array([bound[0, trips.index(tuple(p[:3]))].item() for p in pts])
    want, babs = want.real, babs.real
    err = np.abs(got - want)
    kappa = babs / np.abs(want)
    good = kappa * UNIT[precision] <= TOL[precision] / 10
    erel = err / np.abs(want)
    return {"points": len(pts), "kappa_err_max": float((err / babs).max()),
            "rel_err_max": float(erel.max()),
            "kappa_min_max": [float(kappa.min()), float(kappa.max())],
            "well_conditioned": {"points": int(good.sum()), "u": UNIT[precision],
                                 "tol": TOL[precision],
                                 "rel_err_max": float(erel[good].max()) if good.any() else None},
            "bound_covers_every_point": bool(np.all(err <= beta)),
            "bound_over_error_min": float(np.min(beta / np.maximum(err, 1e-300))),
            "rel_bound_median": float(np.median(beta / np.abs(want))),
            "min_triples_per_point": int(cnt.min()),
            "sample": (f"FP64 oracle collapsed means at {len(pts)} points (ring triples "
                       f"{sorted(set(tuple(trips[t]) for t in chosen))}) over the channel block "
                       f"{list(b)}, {dt:.1f} s of CPU")}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per = max(2.0, min(20.0, 90.0 / max(1, args.steps + args.warmup)))
    vis = make_vis(w, seed=2000)
    for _ in range(args.warmup):
        cpu_baseline(w, per / 4, vis)
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, per, vis))
    value = statistics.mean(v["value"] for v in vals)
    line = {"impl": "reference", "metric": "mabs_bin_triple_x_channel_evals_per_s", "value": value,
            "unit": "evals/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w["desc"], "sample": vals[-1]["sample"]},
            "cpu_baseline": {"kind": "oracle", "cores": vals[-1]["cores"], "value": value,
                             "unit": "evals/s", "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_monopole(plan, b3, stream, nc, reps=5):
    """The binned 3D-bispectrum monopole (bs_bs_monopole) of the step's own
    closable-plane output: 12 log k1 bins x 5 mu x 5 t, CUDA events on the
    launching stream; the algorithmic bytes are one read of the planes."""
    import numpy as np
    import torch
    kperp = 2 * np.pi * plan.ring_umean()  # r = 1 in the bench plans
    kpar = (np.arange(nc) - nc // 2) * (2 * np.pi / nc)
    kmax = float(np.sqrt(kperp.max() ** 2 + 4 * np.abs(kpar).max() ** 2))
    edges = np.geomspace(0.9 * kperp.min(), 1.01 * kmax, 13)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)  # the first call with this geometry also builds the bin table
    sums, cnt = plan.bs_monopole(b3, kperp, kpar, edges, 5, 5)
    ev[1].record(stream)
    torch.cuda.synchronize()
    first_ms = ev[0].elapsed_time(ev[1])
    for _ in range(2):
        sums, cnt = plan.bs_monopole(b3, kperp, kpar, edges, 5, 5)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        sums, cnt = plan.bs_monopole(b3, kperp, kpar, edges, 5, 5)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.bs_monopole(None, kperp, kpar, edges, 5, 5, model=(1.0, 1.0, -2.0))
    e1.record(stream)
    torch.cuda.synchronize()
    samples = b3.numel()
    gbs = samples * 8 / (ms / 1e3) / 1e9
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    # the (k_par1, k_par2) grid of Section 5: 20 x 20 bins over 90% of the k_par range
    ke = np.linspace(-0.9 * np.abs(kpar).max(), 0.9 * np.abs(kpar).max(), 21)
    for _ in range(3):
        plan.bs_cylindrical(b3, kpar, ke)
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        plan.bs_cylindrical(b3, kpar, ke)
    ev[1].record(stream)
    torch.cuda.synchronize()
    cms = ev[0].elapsed_time(ev[1]) / reps
    cgbs = samples * 8 / (cms / 1e3) / 1e9
    return {"bins": "12 log k1 x 5 mu x 5 t", "samples": samples, "ms": ms,
            "first_call_ms": first_ms,
            "samples_per_s": samples / (ms / 1e3), "binned": int(cnt.sum().item()),
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "bytes": samples * 8},
            "model_ms": e0.elapsed_time(e1),
            "cylindrical": {"bins": "20 x 20 (k_par1, k_par2)", "ms": cms,
                            "roofline": {"bound": "hbm", "achieved": cgbs, "peak": peak,
                                         "unit": "GB/s", "frac": cgbs / peak,
                                         "bytes": samples * 8}},
            "note": "kernels k_mono_sum<1> (bins from the plan's cached int16 table: 8 B of "
                    "values + 2 B of bins per sample, one FP64 add per binned sample), "
                    "k_bs_cylindrical; first_call_ms includes k_mono_bins (the bin decision "
                    "of every sample, once per geometry); model_ms bins Eq. (bsana) (FP64 pow "
                    "per sample)"}


def run_gridding(plan, nt, nc, stream, reps=5):
    """Eq. (vg) gridding (bs_grid_visibilities) of 8128 baselines (a 128-antenna
    array) x nc channels onto the plan's grid, 15% of the data flagged, CUDA
    events on the launching stream.  Algorithmic bytes: the visibilities,
    flags and coordinates read once, the output grid written once."""
    import numpy as np
    import torch
    nbl = 8128
    r = np.random.default_rng(5)
    uv = torch.from_numpy(r.uniform(-0.5 * nt + 1, 0.5 * nt - 1, size=(nbl, 2))).cuda()
    g = torch.Generator(device="cuda").manual_seed(6)
    vis = torch.complex(torch.randn((nbl, nc), device="cuda", generator=g),
                        torch.randn((nbl, nc), device="cuda", generator=g))
    flags = (torch.rand((nbl, nc), device="cuda", generator=g) < 0.15).to(torch.uint8)
    for _ in range(3):
        out = plan.grid_visibilities(uv, vis, flags)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        out = plan.grid_visibilities(uv, vis, flags)
    ev[1].record(stream)
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / reps
    nv = nbl * nc
    nbytes = nv * (8 + 1) + nbl * 16 + nc * nt * nt * (8 + 4)
    gbs = nbytes / (ms / 1e3) / 1e9
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    del out
    return {"baselines": nbl, "channels": nc, "visibilities_per_s": nv / (ms / 1e3), "ms": ms,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "bytes": nbytes},
            "note": "memsets of the output grid + k_grid_vis (6 FP32 atomics per visibility)"}


def run_e2e(args, step_e2e, vis_h, vis_d, out3d, stream, world, dev, barrier):
    """End-to-end throughput through the C ABI from host memory.  Every step
    copies its visibilities host->device (pinned) and reads its 3D bispectrum
    back device->host (pinned), all inside the timed region.  Copies run on a
    second stream with double buffers, so step i's read-back and step i+1's
    upload overlap the compute of the neighbouring step; the host waits for
    each step's read-back to complete."""
    import torch
    import torch.distributed as dist
    copy = torch.cuda.Stream(device=dev)
    vis_d2 = [vis_d, torch.empty_like(vis_d)]
    out2 = [out3d, torch.empty_like(out3d)]
    res_h2 = [torch.empty(out3d.shape, dtype=out3d.dtype).pin_memory() for _ in range(2)]
    ev = lambda: torch.cuda.Event()
    ev_in, ev_used, ev_out, ev_back = ([ev(), ev()] for _ in range(4))

    def upload(k):
        copy.wait_event(ev_used[k])  # the grid load that read this buffer last has run
        with torch.cuda.stream(copy):
            vis_d2[k].copy_(vis_h, non_blocking=True)
        ev_in[k].record(copy)

    def run(first, n):
        for k in range(2):
            ev_used[k].record(stream)
            ev_back[k].record(copy)
        upload(0)
        evals = 0
        for i in range(n):
            k = i % 2
            stream.wait_event(ev_in[k])
            stream.wait_event(ev_back[k])  # read-back of step i - 2 done before out2[k] is rewritten
            evals += step_e2e(first + i, vis_d2[k], out2[k])
            ev_out[k].record(stream)
            if i + 1 < n:
                ev_used[k].record(stream)
                upload(1 - k)
            copy.wait_event(ev_out[k])
            with torch.cuda.stream(copy):
                res_h2[k].copy_(out2[k], non_blocking=True)
            ev_back[k].record(copy)
            if i > 0:
                ev_back[1 - k].synchronize()  # the host has step i - 1's result
        ev_back[(n - 1) % 2].synchronize()
        return evals

    run(args.warmup + args.steps, 1)
    torch.cuda.synchronize()
    barrier()
    e0 = time.perf_counter()
    ev2 = run(args.warmup + args.steps, args.steps)
    torch.cuda.synchronize()
    barrier()
    edt = time.perf_counter() - e0
    if world > 1:
        tt = torch.tensor([edt, float(ev2)], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        edt = float(tt[0].item())
        ev2 = ev2 * world
    return {"value": ev2 / edt, "unit": "evals/s", "h2d_bytes_per_step": vis_h.numel() * 8,
            "d2h_bytes_per_step": out3d.numel() * 8,
            "overlap": "double-buffered copies on a second stream"}


# Batched Monte Carlo measurement: uneven shape groups in one persistent,
# graph-replayed launch, skies drawn on the GPU each iteration.  A scaled-down
# form of the 256-realisation ensemble of 128^2..512^2 grids with 384-768
# channels: the channel counts are kept in that range, the grids are smaller.
MC_GROUPS = [dict(nt=128, nchan=384, nb=12, edges=("log", 2.2, 64.0), batch=1),
             dict(nt=96, nchan=256, nb=10, edges=("log", 2.0, 48.0), batch=1),
             dict(nt=64, nchan=192, nb=8, edges=("linear", 0.0, 32.0), batch=2)]


def contracted_flops(tri, sides, nb, dims, symmetric):
    """Algorithmic FLOPs of contracting a channel block of dims = (n1, n2, n3)
    channels: 2 M^2 per channel triple of every closable ring triple; with the
    channel symmetry of a cube block (n channels), n^2 (n + 1) / 2 channel triples
    (one ordering) for the ring triples with a repeated ring.  Ring triples in the
    plan's order (i <= j <= l, lexicographic)."""
    import numpy as np
    per = 2.0 * np.asarray(sides, dtype=np.float64) ** 2
    ok = np.asarray(tri) > 0
    n3 = float(dims[0]) * dims[1] * dims[2]
    if not symmetric:
        return float(per[ok].sum()) * n3
    rep = np.array([i == j or j == l for i in range(nb) for j in range(i, nb)
                    for l in range(j, nb)])
    n = float(dims[0])
    return float(per[ok & ~rep].sum()) * n3 + float(per[ok & rep].sum()) * n * n * (n + 1) / 2


def run_mc(dev, precision, iters=3):
    import numpy as np
    import torch
    import paper_2506_10526_gb300 as bs
    specs = [dict(nt=g["nt"], nchan=g["nchan"], edges=list(edges_of(g)), batch=g["batch"],
                  multires=True, precision=precision) for g in MC_GROUPS]
    ens = bs.Ensemble(specs)
    gens, bufs = [], []
    for k, sp in enumerate(specs):
        gens.append(bs.SkyGenerator(sp["nt"], sp["nchan"], max_batch=sp["batch"]))
        bufs.append(torch.empty((sp["batch"], sp["nchan"], sp["nt"], sp["nt"]),
                                dtype=torch.complex64, device=dev))
        ens.set_input(k, bufs[k])
    # algorithmic FLOPs of the contraction: sum over closable ring triples of 2 M^2 per
    # channel triple, from a plan of the same shape; the full cubes of 64 channels or
    # more run with the channel symmetry of repeated rings
    flops, evals = 0.0, 0
    for sp in specs:
        pl = bs.Plan(sp["nt"], sp["nchan"], sp["edges"], precision=precision, multires=True)
        pl.grid_load(torch.zeros((1, sp["nchan"], sp["nt"], sp["nt"]), dtype=torch.complex64,
                                 device=dev))
        tri, _ = pl.counts()
        sides = pl.trip_sides()
        ok = tri > 0
        nc = sp["nchan"]
        flops += sp["batch"] * contracted_flops(tri, sides, len(sp["edges"]) - 1, (nc, nc, nc),
                                                nc >= 64)
        evals += sp["batch"] * int(ok.sum()) * nc ** 3
        pl.close()
    tiles = ens.autotune()

    def one(i):
        for k, sp in enumerate(specs):
            gens[k].generate(77, i * sp["batch"], out=bufs[k])
        ens.run(use_graph=True)

    for i in range(2):
        one(i)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(iters):
        one(2 + i)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    _, _, nreal = ens.stats(0, 1)
    ens.close()
    # the same realisations one at a time: a plan per shape with batch 1, each
    # realisation through grid load, full-cube contraction, collapse and Eq. (dft)
    # as separate calls (sky generation included, as in the batched run)
    loop = []
    for k, sp in enumerate(specs):
        pl = bs.Plan(sp["nt"], sp["nchan"], sp["edges"], precision=precision, multires=True)
        one_buf = torch.empty((1, sp["nchan"], sp["nt"], sp["nt"]), dtype=torch.complex64,
                              device=dev)
        gen1 = bs.SkyGenerator(sp["nt"], sp["nchan"], max_batch=1)
        gen1.generate(77, 0, out=one_buf)
        pl.grid_load(one_buf)  # the first load counts the closed triangles
        ncl = pl.n_closable
        n2 = 2 * sp["nchan"] - 1
        dd = torch.empty((1, ncl, n2, n2), dtype=torch.float64, device=dev)
        b3 = torch.empty((1, ncl, sp["nchan"], sp["nchan"]), dtype=torch.float64, device=dev)
        loop.append((sp, pl, one_buf, gen1, dd, b3))

    def one_at_a_time(i):
        for sp, pl, one_buf, gen1, dd, b3 in loop:
            for r in range(sp["batch"]):
                gen1.generate(77, i * sp["batch"] + r, out=one_buf)
                pl.grid_load(one_buf)
                pl.mabs(accumulate=True, symmetric=sp["nchan"] >= 64)  # as the ensemble
                pl.mabs_delta_closable(dd)
                pl.bs3d_closable(b3)

    one_at_a_time(0)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(iters):
        one_at_a_time(2 + i)
    e1.record(stream)
    torch.cuda.synchronize()
    loop_ms = e0.elapsed_time(e1) / iters
    for sp, pl, one_buf, gen1, dd, b3 in loop:
        pl.close()
        gen1.close()
    for gg in gens:
        gg.close()
    npr = 3  # tensor products per algorithmic one (split BF16 and split FP16 alike)
    peak = float(measured_peaks().get("bf16_tflops", 1900.0)) / npr
    nr = sum(sp["batch"] for sp in specs)
    return {"groups": [f'{g["nt"]}^2 x {g["nchan"]} ch x {g["nb"]} rings x {g["batch"]}'
                       for g in MC_GROUPS],
            "realisations_per_run": nr, "ms_per_run": ms,
            "realisations_per_s": nr / (ms / 1e3), "evals_per_s": evals / (ms / 1e3),
            "tiles_per_sm": tiles, "realisations_accumulated": int(nreal),
            "contraction_flops_frac_of_run": (flops / (ms / 1e3) / 1e12) / peak,
            "one_at_a_time_ms_per_run": loop_ms, "batched_speedup": loop_ms / ms,
            "note": "one graph replay per run: GPU sky generation, fields, one persistent "
                    "tensor-core launch over all groups, collapse, delay transform, Welford "
                    "statistics; frac = algorithmic contraction FLOP/s over the whole run "
                    f"against the measured BF16 burst peak / {npr} ({npr} split products)"}


def run_mc_small(dev, precision, batch=256, loop_real=32, iters=3):
    """The flagged tiny configuration (64^2 grid, 16 channels, 8 linear rings,
    coarse-band flags) as a Monte Carlo ensemble: `batch` realisations per run in
    one graph-replayed persistent launch, against the same realisations one at a
    time through a batch-1 plan (grid load, contraction, collapse, Eq. (dft) as
    separate calls; `loop_real` of them timed).  Sky generation is inside both."""
    import numpy as np
    import torch
    import paper_2506_10526_gb300 as bs
    import synth
    nt, nc = 64, 16
    edges = list(synth.edges_linear(8, 32))
    flags = synth.flag_mask_coarse_band(nc)
    ens = bs.Ensemble([dict(nt=nt, nchan=nc, edges=edges, batch=batch, multires=True,
                            precision=precision)])
    ens.set_flags(0, flags)
    gen = bs.SkyGenerator(nt, nc, max_batch=batch)
    buf = torch.empty((batch, nc, nt, nt), dtype=torch.complex64, device=dev)
    ens.set_input(0, buf)
    stream = torch.cuda.current_stream()

    def run(i):
        gen.generate(91, i * batch, out=buf)
        ens.run(use_graph=True)

    for i in range(2):
        run(i)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(iters):
        run(2 + i)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / iters
    ens.close()
    gen.close()
    pl = bs.Plan(nt, nc, edges, precision=precision, multires=True)
    g1 = bs.SkyGenerator(nt, nc, max_batch=1)
    one = torch.empty((1, nc, nt, nt), dtype=torch.complex64, device=dev)
    g1.generate(91, 0, out=one)
    pl.grid_load(one, chan_flags=flags)
    n2 = 2 * nc - 1
    dd = torch.empty((1, pl.n_closable, n2, n2), dtype=torch.float64, device=dev)
    b3 = torch.empty((1, pl.n_closable, nc, nc), dtype=torch.float64, device=dev)

    def loop(r0, n):
        for r in range(r0, r0 + n):
            g1.generate(91, r, out=one)
            pl.grid_load(one, chan_flags=flags)
            pl.mabs(accumulate=True)
            pl.mabs_delta_closable(dd)
            pl.bs3d_closable(b3)

    loop(0, 4)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    loop(4, loop_real)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3
    loop_ms = max(e0.elapsed_time(e1), wall) / loop_real
    pl.close()
    g1.close()
    return {"shape": "64^2 x 16 ch x 8 linear rings, coarse-band flags", "batch": batch,
            "ms_per_run": ms, "realisations_per_s": batch / (ms / 1e3),
            "one_at_a_time_ms_per_realisation": loop_ms,
            "batched_speedup": loop_ms / (ms / batch),
            "note": "batched: one graph replay (sky generation, fields, one persistent "
                    "tensor-core launch, collapse, Eq. (dft), Welford statistics) per run of "
                    f"{batch} realisations; one at a time: {loop_real} realisations through a "
                    "batch-1 plan, per-realisation time from the larger of CUDA-event and "
                    "host wall time (the loop is launch-bound)"}


# Smooth channel counts (2^a 3^b 5^c, as the sky generator's FFTs need) in [384, 768]
CFG4_NC = [384, 400, 432, 450, 480, 500, 512, 540, 576, 600, 640, 648, 675, 720, 729, 750, 768]


def cfg4_shapes(seed=4000, n=8):
    """Realisation shapes of the batched Monte Carlo configuration, drawn by
    seed: grid side in {128, 256, 512}, channels in [384, 768], log rings
    12..24 from |U| = 4.41 nt / 256 to nt / 2."""
    import numpy as np
    r = np.random.default_rng(seed)
    return [(int(r.choice([128, 256, 512])), int(r.choice(CFG4_NC)), int(r.integers(12, 25)))
            for _ in range(n)]


def cfg4_block_shapes(b=32):
    """Candidate channel blocks of the batched Monte Carlo configuration: all
    hold b^3 channel triples (the same evaluations per ring triple), shaped
    for the contraction's tiles -- 32 x 16 channel pairs per tile, 256 field
    rows of (third ring, nu3) per tile.  (b/2, b/2, 4b) would fill the rows
    further but needs a 4b-channel plan per shape: 74 GB for the largest
    shape, beyond the device with the others resident."""
    return [(b, b, b), (b, b // 2, 2 * b)]


def _mc_cfg4_setup(dev, precision, shapes, dims, per_shape):
    import torch
    import paper_2506_10526_gb300 as bs
    import synth
    import numpy as np
    nch = max(dims)
    blk = (0, dims[0], 0, dims[1], 0, dims[2])
    specs, gens, skies, bufs = [], [], [], []
    for nt, nc, nb in shapes:
        e = list(synth.edges_log(nb, 4.41 * nt / 256, nt / 2))
        specs.append(dict(nt=nt, nchan=nch, edges=e, batch=per_shape, multires=True,
                          precision=precision))
        gens.append(bs.SkyGenerator(nt, nc, max_batch=per_shape))
        skies.append(torch.empty((per_shape, nc, nt, nt), dtype=torch.complex64, device=dev))
        bufs.append(torch.empty((per_shape, nch, nt, nt), dtype=torch.complex64, device=dev))
    ens = bs.Ensemble(specs)
    for k in range(len(specs)):
        ens.set_input(k, bufs[k])
        ens.set_block(k, blk)
    flops = 0.0
    evals = 0
    ntrip3 = dims[0] * dims[1] * dims[2]
    for sp in specs:
        pl = bs.Plan(sp["nt"], nch, sp["edges"], precision=precision, multires=True)
        pl.grid_load(torch.zeros((1, nch, sp["nt"], sp["nt"]), dtype=torch.complex64,
                                 device=dev))
        tri, _ = pl.counts()
        sides = pl.trip_sides()
        ok = tri > 0
        flops += per_shape * float(np.sum(2.0 * sides[ok].astype(np.float64) ** 2)) * ntrip3
        evals += per_shape * int(ok.sum()) * ntrip3
        pl.close()

    def draw(i):
        for k in range(len(specs)):
            gens[k].generate(44, i * per_shape, out=skies[k])
            bufs[k].copy_(skies[k][:, :nch])

    def close():
        ens.close()
        for g in gens:
            g.close()
    return ens, draw, close, flops, evals


def run_mc_cfg4(dev, precision, block=32, per_shape=4, total=256, only_shape=None):
    """The batched Monte Carlo configuration: `total` realisations of uneven
    shapes (cfg4_shapes) through graph-replayed persistent launches, with a
    declared subset of the tiles of every realisation: one channel block of
    block^3 channel triples, [0, a) x [0, b) x [0, c) with a b c = block^3.
    Each realisation's sky is drawn on the GPU at its full depth (nt^2 x nc
    cells, Eq. mb1), and the group plans hold the block's channels only (the
    full channel cube of the largest shape would need 249 GB of plan
    workspace).  One run covers `per_shape` realisations of every shape.  The
    autotuner picks the block shape (cfg4_block_shapes, by the time of one
    run each) and then the tiles' K extent and order (bs_mc_autotune)."""
    import torch
    shapes = cfg4_shapes()
    if only_shape is not None:  # profiling: one of the shapes
        shapes = [shapes[only_shape]]
    stream = torch.cuda.current_stream()
    trial = {}
    for dims in cfg4_block_shapes(block):
        ens, draw, close, _, _ = _mc_cfg4_setup(dev, precision, shapes, dims, per_shape)
        draw(0)
        ens.autotune()
        ens.run(use_graph=True)  # capture
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ens.run(use_graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        trial[dims] = e0.elapsed_time(e1)
        close()
    dims = min(trial, key=trial.get)
    ens, draw, close, flops, evals = _mc_cfg4_setup(dev, precision, shapes, dims, per_shape)
    draw(0)
    ens.autotune()
    tps, order = ens.tuning()
    nper = per_shape * len(shapes)
    runs = max(1, total // nper)
    draw(1)
    ens.run(use_graph=True)  # capture
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(runs)]
    torch.cuda.synchronize()
    for i in range(runs):
        ev[i][0].record(stream)
        draw(2 + i)
        ev[i][1].record(stream)
        ens.run(use_graph=True)
        ev[i][2].record(stream)
    torch.cuda.synchronize()
    ms = ev[0][0].elapsed_time(ev[-1][2])
    sky_ms = sum(a.elapsed_time(b) for a, b, _ in ev)
    _, _, nreal = ens.stats(0, 1)
    close()
    peak = float(measured_peaks().get("bf16_tflops", 1900.0)) / 3
    return {"shapes": [f"{nt}^2 x {nc} ch x {nb} rings" for nt, nc, nb in shapes],
            "declared_subset": f"channel block [0, {dims[0]}) x [0, {dims[1]}) x [0, {dims[2]}) "
                               f"({block}^3 channel triples) of every realisation",
            "block_trials_ms": {f"{a}x{b}x{c}": t for (a, b, c), t in trial.items()},
            "realisations": runs * nper, "ms": ms, "sky_generation_ms": sky_ms,
            "realisations_per_s": runs * nper / (ms / 1e3),
            "evals_per_s": runs * evals / (ms / 1e3),
            "tuning": {"tiles_per_sm": tps, "tile_order": order, "block": list(dims)},
            "contraction_flops_frac_of_run": (runs * flops / (ms / 1e3) / 1e12) / peak,
            "realisations_accumulated_group0": int(nreal),
            "note": "per run: GPU sky generation of every realisation at full depth, the "
                    "block's channels copied into the group inputs, one graph replay (fields, "
                    "one persistent tensor-core launch over all groups, collapse, Eq. (dft), "
                    "Welford statistics); the block shape is picked among equal-size shapes by "
                    "the time of one run; frac against the measured BF16 burst peak / 3"}


def run_surrogate(dev, steps=200, rows=1 << 17):
    """Training and inference rates of the surrogate network on synthetic rows,
    on the tensor-core kernels (the default) and on the FP32 SIMT checker."""
    import torch
    import paper_2506_10526_gb300 as bs
    g = torch.Generator(device=dev).manual_seed(3)
    x = torch.randn((rows, bs.MLP_FEATURES), device=dev, generator=g)
    t = torch.randn((rows,), device=dev, generator=g)
    d, w = bs.MLP_FEATURES, 128
    fwd = 2.0 * (d * w + w * w + w)  # FLOP per row, forward
    trn = 2.0 * (2 * d * w + 3 * w * w + 2 * w)  # forward + dz1 + dW1 + dW2 + dw3 per row
    out = {}
    for kind in ("tensor", "simt"):
        net = bs.Surrogate(d, w, seed=1)
        net.set_kernels(kind)
        net.fit_norm(x, t)
        net.train(x, t, steps=10, batch=8192, lr=1e-3)
        stream = torch.cuda.current_stream()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        nst = steps if kind == "tensor" else steps // 4
        torch.cuda.synchronize()
        e[0].record(stream)
        net.train(x, t, steps=nst, batch=8192, lr=1e-3)
        e[1].record(stream)
        e[2].record(stream)
        for _ in range(10):
            net.forward(x)
        e[3].record(stream)
        torch.cuda.synchronize()
        tr_ms, inf_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3]) / 10
        net.close()
        pre = "" if kind == "tensor" else "simt_"
        out[pre + "train_rows_per_s"] = nst * 8192 / (tr_ms / 1e3)
        out[pre + "train_tflops"] = nst * 8192 * trn / (tr_ms / 1e3) / 1e12
        out[pre + "inference_bins_per_s"] = rows / (inf_ms / 1e3)
        out[pre + "inference_tflops"] = rows * fwd / (inf_ms / 1e3) / 1e12
    out["speedup_inference"] = out["inference_tflops"] / out["simt_inference_tflops"]
    out["speedup_train"] = out["train_tflops"] / out["simt_train_tflops"]
    out["note"] = ("3-layer tanh MLP, width 128, BF16 weights; default kernels: BF16 mma.sync "
                   "(m16n8k16) with activations and gradients split hi + lo, FP32 accumulation; "
                   "simt_*: the FP32 SIMT checker; training = Adam steps on minibatches of 8192 "
                   "rows, FLOP counted once per algorithmic product")
    return out


def main():
    args = parse()
    w = dict(WORKLOADS[args.workload])
    if args.block:
        w["block"] = args.block
    if args.block3:
        w["block3"] = args.block3
    if args.impl == "reference":
        run_reference(args, w)
        return
    if args.only_surrogate:
        import torch
        print(json.dumps({"surrogate": run_surrogate(torch.device("cuda", 0))}), flush=True)
        return
    if args.only_mc_cfg4 is not None:
        import torch
        import paper_2506_10526_gb300 as bs
        prec = bs.PREC_SPLIT_FP16 if args.precision == "split_fp16" else bs.PREC_SPLIT_BF16
        print(json.dumps({"mc_cfg4": run_mc_cfg4(torch.device("cuda", 0), prec,
                                                 total=args.cfg4_total,
                                                 only_shape=args.only_mc_cfg4)}), flush=True)
        return
    if args.only_mc:
        import torch
        import paper_2506_10526_gb300 as bs
        prec = bs.PREC_SPLIT_FP16 if args.precision == "split_fp16" else bs.PREC_SPLIT_BF16
        dev = torch.device("cuda", 0)
        print(json.dumps({"mc": run_mc(dev, prec), "mc_small": run_mc_small(dev, prec),
                          "mc_cfg4": run_mc_cfg4(dev, prec)}), flush=True)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2506_10526_gb300 as bs
    from paper_2506_10526_gb300.sharding import blocks_of, cubes_of, rank_block, reduce_step_stats

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    edges = edges_of(w)
    nt, nc = w["nt"], w["nc"]
    prec = {"fp32": bs.PREC_FP32, "split_bf16": bs.PREC_SPLIT_BF16,
            "split_fp16": bs.PREC_SPLIT_FP16}[args.precision]
    vis = make_vis(w, seed=1000 * 2 + rank)
    multires = args.precision != "fp32" and not args.no_multires
    plan = bs.Plan(nt, nc, edges, precision=prec, multires=multires)
    stream = torch.cuda.current_stream()
    vis_h = torch.from_numpy(vis[None]).pin_memory()
    vis_d = vis_h.to(dev)
    plan.grid_load(vis_d)
    tri, _ = plan.counts()
    nclos = int((tri > 0).sum())
    # results of the closable ring triples only: the other planes are undefined (NaN) or
    # zero by construction and carry no information
    out_delta = torch.empty((1, nclos, 2 * nc - 1, 2 * nc - 1), dtype=torch.float64, device=dev)
    out3d = torch.empty((1, nclos, nc, nc), dtype=torch.float64, device=dev)
    nlev = plan.info()[6]  # image sides the plan keeps fields at
    # kernels per step: column + row pass per image side (+ the FP16 split), the
    # accumulator reset, the contraction, the folded-sampling reciprocals and the
    # normalisation, the delay sampling table, two delay-transform passes
    # channel-symmetric sub-band cubes (accumulate = 2): one more kernel per step fills
    # in the channel orderings of repeated rings that the contraction leaves out
    sym = bool(w.get("cube")) and not args.ordinary and args.precision != "fp32"
    # a symmetric cube wider than 128 channels contracts in one launch per 128 x 128
    # sub-block of its pair plane
    ncontract = ((w["cube"] + 127) // 128) ** 2 if sym else 1
    launches_per_step = ((3 if args.precision == "split_fp16" else 2) * nlev + 7 + (1 if sym else 0)
                         + ncontract - 1)
    sides = plan.trip_sides()
    nb = w["nb"]
    jobs = cubes_of(nc, w["cube"]) if sym else blocks_of(nc, w["block"], w.get("block3"))

    def block_evals(b):
        return nclos * (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])

    def block_flops(b, symmetric):
        return contracted_flops(tri, sides, nb, (b[1] - b[0], b[3] - b[2], b[5] - b[4]),
                                symmetric)

    def step(i, ev=None, vis_in=None, out=None):
        b = rank_block(jobs, i, world, rank)
        plan.grid_load(vis_d if vis_in is None else vis_in)
        if ev is not None:
            ev[0].record(stream)
        plan.mabs(block=b, accumulate=True, symmetric=sym)
        if ev is not None:
            ev[1].record(stream)
        plan.mabs_delta_closable(out_delta)
        plan.bs3d_closable(out3d if out is None else out)
        return block_evals(b)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    barrier()
    t0.record(stream)
    evals = 0
    for i in range(args.steps):
        evals += step(args.warmup + i, ev=kev[i])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    kms = [a.elapsed_time(b) for a, b in kev]
    ms, evals = reduce_step_stats(ms, evals, world, dev)
    value = evals / (ms / 1e3)

    e2e = None
    if not args.no_e2e:
        eclk = ClockSampler(local)
        eclk.start()
        e2e = run_e2e(args, step_e2e=lambda i, v, o: step(i, vis_in=v, out=o), vis_h=vis_h,
                      vis_d=vis_d, out3d=out3d, stream=stream, world=world, dev=dev,
                      barrier=barrier)
        e2e["clocks"] = eclk.stop()  # runs after the timed region, GPU already warm
    mono = run_monopole(plan, out3d, stream, nc) if world == 1 else None
    # error of the timed path against the FP64 oracle, measured in this run on the
    # first block of the job (after the timed region)
    err_info = None
    if rank == 0 and world == 1 and not args.no_cpu:
        step(0)
        err_info = measure_error(plan, vis, edges, jobs[0], out_delta, tri, args.precision)
    # measured arithmetic ceilings (FP32 / FP64 FMA) for the FP32 path's roofline
    peak_fp32 = bs.measure_peak("fp32", 1 << 22)
    peak_fp64 = bs.measure_peak("fp64", 1 << 16)

    # roofline of the contraction (dominant kernel): algorithmic FLOPs = 2 M^2 per evaluation
    M = plan.M
    per_launch_evals = block_evals(jobs[0])
    avg_ms = statistics.mean(kms)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    if args.precision == "fp32":
        peak = peak_fp32 / 1e12
        roof = {"bound": "alu", "peak_source": "measured FP32 FMA rate (bs_measure_peak), "
                f"nominal {SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12:.1f} TFLOP/s at "
                f"{sm_max:.0f} MHz"}
    else:
        # FP16 and BF16 share the dense tensor rate (kind::f16, nominal ratio 1)
        npr = SPLIT_PRODUCTS[args.precision]
        peak = float(peaks.get("bf16_tflops", 1900.0)) / npr
        roof = {"bound": "tensor",
                "peak_source": (f"measured bf16 burst / {npr} ({npr} split products"
                                + ("; FP16 has the BF16 dense rate)"
                                   if args.precision == "split_fp16" else ")"))}
    b0 = jobs[0]
    flops_launch = block_flops(b0, sym)
    achieved = flops_launch / (avg_ms / 1e3) / 1e12
    tr = profile_traffic(args.precision)
    roof.update({"achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                 "kernel": "k_contract_simt" if args.precision == "fp32" else "k_contract_tc",
                 "avg_launch_ms": avg_ms, "launches_per_call": ncontract,
                 "traffic": None if tr is None else tr["bytes_per_unit"] * per_launch_evals})
    if args.precision != "fp32" and "bf16_tflops_sustained" in peaks:
        # the contraction runs back to back for the whole timed region: the measured
        # sustained (power-capped) GEMM rate is the other fair denominator
        sus = float(peaks["bf16_tflops_sustained"]) / SPLIT_PRODUCTS[args.precision]
        roof.update({"peak_sustained": sus, "frac_sustained": achieved / sus})

    line = {
        "metric": "mabs_bin_triple_x_channel_evals_per_s",
        "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision],
        "data": "synthetic",
        "config": {"workload": w["desc"], "M": M, "multires": multires,
                   "image_sides": sorted(set(int(x) for x in sides[tri > 0])),
                   "channel_block": ([w["cube"]] * 3 if sym else
                                     [w["block"], w["block"], w.get("block3") or w["block"]]),
                   "channel_symmetry": (
                       "each step is one sub-band's whole channel cube (bs_mabs accumulate = 2): "
                       "for ring triples with a repeated ring only one ordering of that ring's "
                       "channels is contracted and the other is filled in; evaluations count "
                       "every channel triple of the cube" if sym else None),
                   "contracted_fraction_of_cube_flops": (
                       block_flops(jobs[0], True) / block_flops(jobs[0], False) if sym else 1.0),
                   "closable_ring_triples": nclos, "ring_triples": plan.ntrip,
                   "outputs": (f"folded MABS and 3D bispectrum planes of the {nclos} closable "
                               f"ring triples (bs_mabs_delta_closable, bs_bs3d_closable)"),
                   "evals_per_step_per_gpu": per_launch_evals, "precision": args.precision,
                   "l2": (f"inputs larger than L2 ({vis_h.numel() * 8 / 1e6:.0f} MB visibilities, "
                          f"{plan.info()[3] / 1e9:.1f} GB plan workspace holding the fields)"),
                   "parallelism": f"blocks of the channel cube sharded over {world} GPU(s)"},
        "roofline": roof, "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
        "e2e": e2e,
    }
    if mono is not None:
        line["monopole"] = mono
        line["gridding"] = run_gridding(plan, nt, nc, stream)
    line["error"] = err_info
    line["peaks_measured"] = {"fp32_fma_tflops": peak_fp32 / 1e12,
                              "fp64_fma_tflops": peak_fp64 / 1e12,
                              "source": "bs_measure_peak: 8 independent FMA chains per thread, "
                                        "4 x 256 threads per SM, CUDA events"}
    contraction_rate = per_launch_evals / (avg_ms / 1e3)
    line["contraction_evals_per_s"] = contraction_rate
    ordinary_rate = contraction_rate
    if sym and world == 1:
        # the ordinary accumulation (every channel triple contracted) of the
        # 128 x 128 x 256 block, timed the same way: the like-for-like rate
        ob = blocks_of(nc, w["block"], w.get("block3"))[0]
        oev = []
        for i in range(4):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            plan.grid_load(vis_d)
            e0.record(stream)
            plan.mabs(block=ob, accumulate=True)
            e1.record(stream)
            oev.append((e0, e1))
        torch.cuda.synchronize()
        oms = statistics.mean(a.elapsed_time(b) for a, b in oev[1:])
        ordinary_rate = block_evals(ob) / (oms / 1e3)
        oach = block_flops(ob, False) / (oms / 1e3) / 1e12
        line["ordinary_block"] = {
            "channel_block": [ob[1] - ob[0], ob[3] - ob[2], ob[5] - ob[4]],
            "contraction_evals_per_s": ordinary_rate, "avg_launch_ms": oms,
            "achieved_tflops": oach, "frac": oach / peak}
    plan.close()
    del out3d
    torch.cuda.empty_cache()
    if not args.no_mc and world == 1 and args.precision != "fp32":
        line["mc"] = run_mc(dev, prec)
        line["mc_small"] = run_mc_small(dev, prec)
        line["mc_cfg4"] = run_mc_cfg4(dev, prec)
        line["surrogate"] = run_surrogate(dev)
    if args.precision != "fp32" and not args.no_fp32_compare and world == 1:
        # the plain FP32 GPU path (FP32 FFTs, FP32 SIMT contraction) on the same input,
        # timed the same way on 64^3 blocks: with the same per-triple image sides as the
        # split path (equal work), and with one image side for every triple
        fb = min(64, w["block"])
        fjobs = blocks_of(nc, fb)
        fb_evals = nclos * fb ** 3

        def fp32_rate(mr):
            fp = bs.Plan(nt, nc, edges, precision=bs.PREC_FP32, multires=mr)
            fp.grid_load(vis_d)
            fev = []
            for i in range(3):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fp.mabs(block=fjobs[i % len(fjobs)], accumulate=True)
                e1.record(stream)
                fev.append((e0, e1))
            torch.cuda.synchronize()
            fms = statistics.mean(a.elapsed_time(b) for a, b in fev[1:])
            ferr = None
            if mr and not args.no_cpu:
                fp.grid_load(vis_d)
                fp.mabs(block=fjobs[0], accumulate=True)
                fp.mabs_delta_closable(out_delta)
                ferr = measure_error(fp, vis, edges, fjobs[0], out_delta, tri, "fp32")
            fs = fp.trip_sides()
            fflops = float(np.sum(2.0 * fs[tri > 0].astype(np.float64) ** 2)) * fb ** 3
            fp.close()
            return fb_evals / (fms / 1e3), fms, fflops / (fms / 1e3) / 1e12, ferr

        r_eq, ms_eq, tf_eq, err_eq = fp32_rate(True)
        r_one, ms_one, tf_one, _ = fp32_rate(False)
        p32 = peak_fp32 / 1e12
        line["fp32_plain"] = {
            "channel_block": fb, "contraction_evals_per_s": r_eq, "avg_launch_ms": ms_eq,
            "image_sides": "per ring triple, as the split path",
            "roofline": {"bound": "alu", "achieved": tf_eq, "peak": p32, "unit": "TFLOP/s",
                         "frac": tf_eq / p32, "peak_source": "measured FP32 FMA rate"},
            "error": err_eq,
            "single_side": {"contraction_evals_per_s": r_one, "avg_launch_ms": ms_one,
                            "achieved_tflops": tf_one, "frac": tf_one / p32}}
        # precision gain at equal work (both contract every channel triple); the
        # single-side ratio adds the work saved by per-triple image sides, the
        # symmetric one the work saved by the channel symmetry of repeated rings
        line["speedup_vs_fp32"] = ordinary_rate / r_eq
        line["speedup_vs_fp32_single_side"] = ordinary_rate / r_one
        if sym:
            line["speedup_vs_fp32_with_channel_symmetry"] = contraction_rate / r_eq
    del out_delta
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(w, args.cpu_seconds, vis)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
