#!/usr/bin/env python
"""Benchmark of the DASH 4D-hash deformation hot path (arXiv 2507.19141,
Sec. 4.2-4.3) on GB300.

One step = one training pass of the path over one batch of seeded synthetic
input resident in HBM: compaction of the static/dynamic mask (2M Gaussians,
1M dynamic), the fused forward (Eqs. 8-10: encode, tensor-core decoder,
Eq. 10 update, per-Gaussian state for the backward) and the fused backward (decoder gradients,
table-gradient scatter into FP32 buffers).  Metric: dynamic Gaussians per
second.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank processes its own shard of the same size (weak
scaling; the path needs no data exchange), timed between barriers, max over
ranks.  --impl reference times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "dynamic Gaussians/s, 4D hash enc+MLP fwd+bwd, N=1M L=16; % gather roofline"
UNIT = "Gaussians/s"
N_ALL = 2_000_000
N_DYN = 1_000_000
# algorithmic bytes per dynamic Gaussian (L=16, F=2, FP16 tables, 16 corners):
#   forward : xyzt 16 + idx 4 + gather 16*16*4 = 1024 + delta 40 + state 80 (f_h BF16 + masks) + Eq. 10 in/out 80
#   backward: xyzt 16 + idx 4 + state 80 + ddelta 40 + scatter 16*16*8 = 2048 (FP32 read-modify-write units)
#   compaction: 2 mask bytes (2M Gaussians for 1M dynamic) + 4 index bytes
FWD_BYTES = 16 + 4 + 1024 + 40 + 80 + 80
BWD_BYTES = 16 + 4 + 80 + 40 + 2048
STEP_BYTES = 2 + 4 + FWD_BYTES + BWD_BYTES

# DRAM bytes read + written per launch at 1M Gaussians from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of the profile case), valid
# while the kernel's device sources hash to the captured value; otherwise the
# benchmark reports no traffic.  A changed kernel is re-captured before its
# record changes: the record and the summary of its capture change together.
NCU_TRAFFIC = {
    "bwd": {"bytes": (214.4 + 7.0) * 1e6, "n": 1_000_000, "sha256_16": "751b2ae1b27781ca",
            "sources": ("deform_bwd.cu", "deform_bwd_common.cuh", "deform_common.cuh", "dash_internal.cuh",
                        "tc_ptx.cuh", "replicas.cu")},
    "fwd": {"bytes": (46.6 + 70.9) * 1e6, "n": 1_000_000, "sha256_16": "6045a322b2a9b744",
            "sources": ("deform_fwd.cu", "deform_common.cuh", "dash_internal.cuh", "tc_ptx.cuh")},
}


def captured_traffic(kernel, n):
    """Per-launch DRAM traffic of `kernel` at n Gaussians, or None when the
    capture was taken at another size or the kernel has changed since."""
    import hashlib
    rec = NCU_TRAFFIC[kernel]
    if n != rec["n"]:
        return None
    m = hashlib.sha256()
    for f in rec["sources"]:
        with open(os.path.join(ROOT, "paper_2507_19141_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return rec["bytes"] if m.hexdigest()[:16] == rec["sha256_16"] else None
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)  # ~1.6 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n-dyn", type=int, default=N_DYN)
    ap.add_argument("--n-all", type=int, default=N_ALL)
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--cpu-sample", type=int, default=0, help="oracle sample size (0 = calibrate to ~10 s)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run the small profiling case (1M points, two launches of each kernel) and exit")
    return ap.parse_args(argv)


# ------------------------------------------------------------ distributed --
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def dist_init(backend):
    import torch.distributed as dist
    ws, rank, _ = dist_env()
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, rank=rank, world_size=ws)
    return ws, rank


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.5)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (ts, l) in self.lines if t0 <= ts <= t1 + 0.25]
        if not rows:
            rows = [l for (_, l) in self.lines]
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [v.strip() for v in r.split(",")]
            if len(f) < 10:
                continue
            try:
                mhz.append(float(f[2]))
                mx = float(f[3])
            except ValueError:
                continue
            for name, v in zip(names, f[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not mhz:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(mhz), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(mhz)}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            v = float(json.load(fh)["hbm_gbs"])
            return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ----------------------------------------------------------------- workload --
class Workload:
    """Seeded synthetic inputs of the precision/differentiation form: 2M
    Gaussians, exactly 1M dynamic, scene-like coordinates, FP16 tables, BF16
    decoder weights, N(0,1) upstream gradients; resident on the device."""

    def __init__(self, seed, n_all, n_dyn, device, morton=False):
        import numpy as np
        import torch
        from paper_2507_19141_gb300 import dash, synth
        self.np_rng = np.random.default_rng(seed)
        rng = self.np_rng
        self.grid, self.mlpc = synth.PAPER_GRID, synth.PAPER_MLP
        self.n_all, self.n_dyn = n_all, n_dyn
        self.layout = dash.layout_from(self.grid)
        self.mask_h = synth.exact_count_mask(rng, n_all, n_dyn)
        self.coords_h = synth.scene_coords(rng, n_all)
        self.table_h = synth.table_values(rng, self.layout.total, self.grid.F, np.float16)
        self.params_h = synth.mlp_params(rng, self.mlpc)
        self.attrs_h = synth.gaussian_attrs(rng, n_all)
        if morton:  # the same Gaussians stored in the Z order of their positions
            order = np.argsort(morton3(*self.coords_h[:3]), kind="stable")
            self.mask_h = self.mask_h[order]
            self.coords_h = tuple(c[order] for c in self.coords_h)
            self.attrs_h = np.ascontiguousarray(self.attrs_h[:, order])
        dd = synth.upstream_grad(rng, self.mlpc.d_out, n_dyn)
        self.ddelta_h = dd
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        self.mask = dev(self.mask_h)
        self.x, self.y, self.z, self.t = (dev(c) for c in self.coords_h)
        self.table = dev(self.table_h)
        self.params = dev(self.params_h)
        self.attrs_in = dev(self.attrs_h)
        self.attrs_out = self.attrs_in.clone()
        O = self.mlpc.d_out
        # SoA buffers are sized by the capacity n_all; the device count selects the live prefix
        self.ddelta = torch.zeros((O, n_all), dtype=torch.float32, device=device)
        self.ddelta[:, :n_dyn] = dev(dd)
        self.delta = torch.empty((O, n_all), dtype=torch.float32, device=device)
        self.idx = torch.empty(n_all, dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.ws = torch.empty(dash.dash_compact_workspace_size(n_all), dtype=torch.uint8, device=device)
        self.table_grad = torch.zeros((self.layout.total, self.grid.F), dtype=torch.float32, device=device)
        self.mlp_grad = torch.zeros(self.mlpc.n_params, dtype=torch.float32, device=device)
        self.mlp = dash.Mlp(self.params, self.mlpc.d_in, self.mlpc.d_hidden, self.mlpc.d_out)
        self.fsave = dash.deform_state(self.mlp, n_all, device)
        self.pts = dash.Points(self.x, self.y, self.z, self.t, idx=self.idx, n=n_all, n_dev=self.count)
        # the backward's workspace: replicas of the dense levels' gradients
        self.bws = torch.empty(dash.dash_deform_bwd_workspace_size(self.layout, n_all), dtype=torch.uint8,
                               device=device)
        self.dash = dash

    def compact(self):
        self.dash.dash_compact_dynamic(self.mask, idx_out=self.idx, count_out=self.count, ws=self.ws)

    def forward(self):
        self.dash.dash_deform_mlp_fwd(self.layout, self.pts, self.table, self.mlp, delta_out=self.delta,
                                      fwd_state=self.fsave, apply=(self.attrs_in, self.attrs_out))

    def backward(self, smooth=None, ws=None):
        self.dash.dash_deform_mlp_bwd(self.layout, self.pts, self.table, self.mlp, self.ddelta, self.table_grad,
                                      self.mlp_grad, fwd_state=self.fsave, smooth=smooth,
                                      ws=self.bws if ws is None else ws)

    def step(self):
        self.compact()
        self.forward()
        self.backward()


LAUNCHES_PER_STEP = 6  # compaction count/scan/write, fused forward, fused backward, replica sum


def morton3(x, y, z, bits=10):
    """Z-order (Morton) keys of points in [0,1]^3: each coordinate quantised
    to `bits` bits and the bits interleaved (x lowest)."""
    import numpy as np

    def spread(v):  # bit i of v moves to bit 3 i
        v = v.astype(np.uint64)
        out = np.zeros_like(v)
        for i in range(bits):
            out |= ((v >> np.uint64(i)) & np.uint64(1)) << np.uint64(3 * i)
        return out

    q = lambda c: np.minimum((np.clip(c, 0.0, 1.0) * (1 << bits)).astype(np.int64), (1 << bits) - 1)
    return spread(q(x)) | (spread(q(y)) << np.uint64(1)) | (spread(q(z)) << np.uint64(2))


def time_region(torch, fn, steps, stream):
    """The contract's timed region: `steps` calls of fn between one pair of
    CUDA events on `stream`; returns ms per step (the mean over the region)."""
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(steps):
        fn()
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / steps


MIN_REPS, WARMUP_REPS = 20, 5


def time_steps(torch, fn, reps, stream):
    """A secondary row: WARMUP_REPS untimed calls of fn, then at least
    MIN_REPS calls each bracketed by its own pair of CUDA events on `stream`;
    returns the median in ms."""
    for _ in range(WARMUP_REPS):
        fn()
    E = lambda: torch.cuda.Event(enable_timing=True)
    evs = [(E(), E()) for _ in range(max(reps, MIN_REPS))]
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    evs[-1][1].synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in evs)


# L2/L1 operations per dynamic Gaussian of the fused kernels' table accesses
# (L = 16 levels, 16 corners, F = 2).  The lane pairs put an x-neighbour
# pair's two accesses in one warp instruction; the hardware serves them as
# one sector operation when both entries share a 32-byte sector.  With
# pi_1 = 1 (and on dense levels) the pair's entries are c and
# c ^ (2^(k+1) - 1), k the trailing one bits of the lower x coordinate:
#   backward, 8-byte FP32 gradient entries (4 per sector): shared unless
#   k >= 2, probability 1/4 -> 8 pairs x 1.25 = 10 sector reductions a level;
#   forward, 4-byte FP16 entries (8 per sector): shared unless k >= 3,
#   probability 1/8 -> 8 x 1.125 = 9 sector loads a level.
LEVELS, CORNERS = 16, 16
BWD_RED_SECTORS = LEVELS * 8 * 1.25   # 160 per Gaussian
FWD_GATHER_SECTORS = LEVELS * 8 * 1.125  # 144 per Gaussian


def measure_ceilings(torch, stream, entries):
    """Measured rates (median of 20 launches after 5 warm-ups) of the access
    patterns that bound the fused kernels, on buffers sized like the
    gradient buffer (entries x 8 B) and the FP16 table (entries x 4 B), both
    L2-resident: random 8- and 16-byte FP32 reductions (sector operations/s),
    lane-paired 8-byte reductions (lane reductions/s), random and lane-paired
    4-byte gathers (lane loads/s)."""
    from paper_2507_19141_gb300 import dash
    grad = torch.zeros(entries * 2, dtype=torch.float32, device="cuda")
    tab = torch.rand(entries, dtype=torch.float32, device="cuda")
    sink = torch.empty(dash.dash_probe_threads(dash.PROBE_GATHER4), dtype=torch.float32, device="cuda")
    iters = 256
    out = {}
    for key, kind, buf in (("red8", dash.PROBE_RED8, grad), ("red16", dash.PROBE_RED16, grad),
                           ("red8_paired", dash.PROBE_RED8_PAIRED, grad), ("gather4", dash.PROBE_GATHER4, tab),
                           ("gather4_paired", dash.PROBE_GATHER4_PAIRED, tab)):
        ops = [0]

        def once():
            ops[0] = dash.dash_probe_rate(kind, buf, iters, sink)

        ms = time_steps(torch, once, MIN_REPS, stream)
        out[f"{key}_per_s"] = ops[0] / (ms / 1e3)
    del grad, tab, sink
    torch.cuda.empty_cache()
    # a sector operation serves two paired lanes; the best measured rate of each unit
    out["l2_red_sector_peak_per_s"] = max(out["red8_per_s"], out["red16_per_s"], out["red8_paired_per_s"] / 2)
    out["l1_gather_sector_peak_per_s"] = max(out["gather4_per_s"], out["gather4_paired_per_s"] / 2)
    out["buffers"] = f"{entries} entries: {entries * 8 / 1e6:.1f} MB FP32 pairs (reductions), " \
                     f"{entries * 4 / 1e6:.1f} MB (gathers); {dash.dash_probe_threads(1)} threads x {iters} ops"
    return out


def step_config(args, ws):
    """The workload both arms report (the reference arm times a bounded
    sample of it on the host)."""
    return {"workload": "DASH 4D-hash deformation step: compaction of 2M Gaussians (1M dynamic) + fused "
                        "encoder/decoder forward (Eq. 10 applied, f_h saved) + fused backward; L=16 F=2 "
                        "T=2^19 res 16->2048 / 8->150, decoder 32-64-64-10",
            "n_dynamic_per_gpu": args.n_dyn, "n_gaussians_per_gpu": args.n_all,
            "l2": "working set ~0.4 GB/step > 129 MB L2 (no flush); tables stay L2-warm as across frames",
            "parallelism": f"{ws} independent shard(s)"}


def run_ours(args):
    import torch
    ws, rank = dist_init("nccl")
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    wl = Workload(seed=2 + rank, n_all=args.n_all, n_dyn=args.n_dyn, device=device)
    stream = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 3)):
        wl.step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, per-kernel events, clocks sampled meanwhile
    ev = {k: [] for k in ("compact", "fwd", "bwd", "step")}
    E = lambda: torch.cuda.Event(enable_timing=True)

    def step_events():
        marks = [E() for _ in range(4)]
        marks[0].record(stream)
        wl.compact()
        marks[1].record(stream)
        wl.forward()
        marks[2].record(stream)
        wl.backward()
        marks[3].record(stream)
        ev["compact"].append((marks[0], marks[1]))
        ev["fwd"].append((marks[1], marks[2]))
        ev["bwd"].append((marks[2], marks[3]))
        ev["step"].append((marks[0], marks[3]))

    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        t0 = time.time()
        ms = time_region(torch, step_events, args.steps, stream)
        torch.cuda.synchronize()
        barrier()
        t1 = time.time()
    ms = max_over_ranks(ms, device)
    clocks = clk.summary(t0, t1)
    # per-kernel and per-step medians over the K timed steps (each bracketed by its own events)
    per_kernel = {k: statistics.median(a.elapsed_time(b) for a, b in v) for k, v in ev.items()}
    per_kernel_mean = {k: statistics.mean(a.elapsed_time(b) for a, b in v) for k, v in ev.items()}
    step_median = per_kernel.pop("step")
    per_kernel_mean.pop("step")

    n_units = args.n_dyn * ws
    value = n_units / (ms / 1e3)
    peak, peak_kind = measured_hbm_peak()
    dom = max(("fwd", "bwd"), key=lambda k: per_kernel_mean[k])
    dom_bytes = (FWD_BYTES if dom == "fwd" else BWD_BYTES) * args.n_dyn
    achieved = dom_bytes / (per_kernel_mean[dom] / 1e3) / 1e9  # the average launch over the timed region
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp16 tables / bf16 MLP / fp32 acc+grads",
        "data": "synthetic (seeded; stands in for Neural 3D Video / Technicolor scenes)",
        "config": step_config(args, ws),
        "gpu_launches": LAUNCHES_PER_STEP * args.steps,
        "ms_per_step_median": step_median,
        "per_kernel_ms": per_kernel, "per_kernel_stat": f"median of the {args.steps} timed steps",
        "per_kernel_mean_ms": per_kernel_mean,
        "roofline": {"bound": "hbm", "kernel": f"fused {dom}", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs",
                     "algorithmic_bytes_per_gaussian": FWD_BYTES if dom == "fwd" else BWD_BYTES,
                     "traffic": captured_traffic(dom, args.n_dyn),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch at 1M "
                                       "Gaussians without an index list (profile case)"},
        "clocks": clocks,
        "step_roofline": {"bytes_per_gaussian": STEP_BYTES, "achieved_gbs": STEP_BYTES * value / 1e9,
                          "frac": STEP_BYTES * value / 1e9 / peak,
                          "gaussians_per_s_at_peak": peak * 1e9 / STEP_BYTES},
    }
    # the binding units: the L2's reduction rate (backward) and the L1's
    # gather rate (forward), measured in this process after the timed region
    ceil = measure_ceilings(torch, stream, wl.layout.total)
    n_b, t_b = args.n_dyn, per_kernel_mean["bwd"] / 1e3
    n_f, t_f = args.n_dyn, per_kernel_mean["fwd"] / 1e3
    out["roofline_l2"] = {"bound": "l2_reductions", "kernel": "fused bwd", "unit": "sector reductions/s",
                          "ops_per_gaussian": BWD_RED_SECTORS, "achieved": BWD_RED_SECTORS * n_b / t_b,
                          "peak": ceil["l2_red_sector_peak_per_s"],
                          "frac": BWD_RED_SECTORS * n_b / t_b / ceil["l2_red_sector_peak_per_s"],
                          "lane_reductions_per_gaussian": LEVELS * CORNERS,
                          "peak_source": "measured in this process (dash_probe_rate, best of RED8/RED16/RED8_PAIRED)"}
    out["roofline_l1"] = {"bound": "l1_gather_sectors", "kernel": "fused fwd", "unit": "sector loads/s",
                          "ops_per_gaussian": FWD_GATHER_SECTORS, "achieved": FWD_GATHER_SECTORS * n_f / t_f,
                          "peak": ceil["l1_gather_sector_peak_per_s"],
                          "frac": FWD_GATHER_SECTORS * n_f / t_f / ceil["l1_gather_sector_peak_per_s"],
                          "lane_loads_per_gaussian": LEVELS * CORNERS,
                          "peak_source": "measured in this process (dash_probe_rate, GATHER4 / GATHER4_PAIRED)"}
    out["ceilings"] = ceil
    if rank == 0:
        out["e2e"] = run_e2e(torch, wl, args, stream)
    if rank == 0 and not args.no_extras:
        out["extras"] = run_extras(torch, wl, args, stream)
        out["cpu_baseline"] = cpu_baseline(args, wl)
        out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(out["cpu_baseline"]["value"])
        out["cpu_baseline_configs"] = oracle_plain_configs()
    if rank == 0:
        print(json.dumps(out), flush=True)
    barrier()


class Slot:
    """One in-flight step's device buffers (mask, coordinates, upstream
    gradient, index list, state, offsets); the model (tables, decoder) and
    its gradients are shared with the workload."""

    def __init__(self, torch, wl):
        from paper_2507_19141_gb300 import dash
        self.wl, self.dash = wl, dash
        self.mask = torch.empty_like(wl.mask)
        self.x, self.y, self.z, self.t = (torch.empty_like(v) for v in (wl.x, wl.y, wl.z, wl.t))
        self.ddelta = torch.zeros_like(wl.ddelta)
        self.delta = torch.empty_like(wl.delta)
        self.idx = torch.empty_like(wl.idx)
        self.count = torch.zeros_like(wl.count)
        self.ws = torch.empty_like(wl.ws)
        self.state = torch.empty_like(wl.fsave)
        self.bws = torch.empty_like(wl.bws)
        self.pts = dash.Points(self.x, self.y, self.z, self.t, idx=self.idx, n=wl.n_all, n_dev=self.count)

    def step(self):
        wl, d = self.wl, self.dash
        d.dash_compact_dynamic(self.mask, idx_out=self.idx, count_out=self.count, ws=self.ws)
        d.dash_deform_mlp_fwd(wl.layout, self.pts, wl.table, wl.mlp, delta_out=self.delta, fwd_state=self.state,
                              apply=(wl.attrs_in, wl.attrs_out))
        d.dash_deform_mlp_bwd(wl.layout, self.pts, wl.table, wl.mlp, self.ddelta, wl.table_grad, wl.mlp_grad,
                              fwd_state=self.state, ws=self.bws)


def run_e2e(torch, wl, args, stream):
    """Same step through the public API from pinned HOST buffers: every step
    uploads its mask, coordinates and upstream gradient and downloads its
    offsets and the decoder gradient, all inside the timed region.  Two
    buffer slots and two copy streams let step k+1's upload and step k-1's
    download overlap step k's kernels."""
    n = args.n_dyn
    pin = lambda a: torch.from_numpy(a).pin_memory()
    mask_h = pin(wl.mask_h)
    xyzt_h = [pin(c) for c in wl.coords_h]
    dd_h = pin(wl.ddelta_h)
    delta_h = [torch.empty((wl.mlpc.d_out, n), dtype=torch.float32).pin_memory() for _ in range(2)]
    grad_h = [torch.empty(wl.mlpc.n_params, dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = mask_h.numel() + sum(c.numel() * 4 for c in xyzt_h) + dd_h.numel() * 4
    d2h = delta_h[0].numel() * 4 + grad_h[0].numel() * 4
    slots = [Slot(torch, wl), Slot(torch, wl)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    done = [None, None]

    def e2e_step(k):
        s = slots[k % 2]
        with torch.cuda.stream(up):
            if done[k % 2] is not None:
                up.wait_event(done[k % 2])  # slot free: step k-2 has finished computing
            s.mask.copy_(mask_h, non_blocking=True)
            for dv, hv in zip((s.x, s.y, s.z, s.t), xyzt_h):
                dv.copy_(hv, non_blocking=True)
            for j in range(dd_h.shape[0]):  # contiguous rows of the SoA layout: plain async copies
                s.ddelta[j, :n].copy_(dd_h[j], non_blocking=True)
            uploaded = torch.cuda.Event()
            uploaded.record(up)
        stream.wait_event(uploaded)
        s.step()
        computed = torch.cuda.Event()
        computed.record(stream)
        done[k % 2] = computed
        with torch.cuda.stream(down):
            down.wait_event(computed)
            for j in range(delta_h[k % 2].shape[0]):
                delta_h[k % 2][j].copy_(s.delta[j, :n], non_blocking=True)
            grad_h[k % 2].copy_(wl.mlp_grad, non_blocking=True)

    steps = max(10, min(args.steps, 100))
    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    up.wait_event(start)
    for k in range(steps):
        e2e_step(k)
    stream.wait_stream(up)
    stream.wait_stream(down)
    end.record(stream)
    end.synchronize()
    wall = (time.perf_counter() - t0) * 1e3 / steps
    ms = max(start.elapsed_time(end) / steps, wall)
    torch.cuda.synchronize()
    return {"value": n / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "overlap": "two buffer slots; uploads and downloads on their own streams overlap the kernels"}


def run_extras(torch, wl, args, stream):
    """Secondary rows: forward only, backward with the Eq. 11 term, the plain
    FP32 GPU form at the same N, and a cold-L2 step."""
    from paper_2507_19141_gb300 import dash
    n = args.n_dyn
    reps = 30
    res = {}
    for _ in range(3):
        wl.forward()
    res["fwd_ms"] = time_steps(torch, wl.forward, reps, stream)
    loss = torch.zeros(1, dtype=torch.float32, device=wl.table.device)
    smooth = (1.0, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300, loss)
    # dL/df_h handed to the Eq. 11 kernel through the workspace, gradient replicas (the default) ...
    sws = torch.empty(dash.dash_deform_bwd_workspace_size(wl.layout, wl.pts.n, smooth), dtype=torch.uint8,
                      device=wl.table.device)
    wl.backward(smooth, sws)
    res["bwd_smooth_ms"] = time_steps(torch, lambda: wl.backward(smooth, sws), reps, stream)
    res["fwd_bwd_smooth_gaussians_per_s"] = n / ((res["fwd_ms"] + res["bwd_smooth_ms"]) / 1e3)
    # ... and without a workspace: the fused backward scatters dL/df_h, the Eq. 11 kernel its own term
    wl.backward(smooth, False)
    res["bwd_smooth_separate_ms"] = time_steps(torch, lambda: wl.backward(smooth, False), reps, stream)
    # the plain backward without the gradient replicas
    wl.backward(None, False)
    res["bwd_no_replicas_ms"] = time_steps(torch, lambda: wl.backward(None, False), reps, stream)
    # backward that also returns d loss / d(x, y, z, t) (gathers the corner entries as well)
    cgrad = torch.empty((4, wl.n_all), dtype=torch.float32, device=wl.table.device)

    def bwd_coord():
        wl.dash.dash_deform_mlp_bwd(wl.layout, wl.pts, wl.table, wl.mlp, wl.ddelta, wl.table_grad, wl.mlp_grad,
                                    fwd_state=wl.fsave, coord_grad=cgrad)

    bwd_coord()
    res["bwd_coord_grad_ms"] = time_steps(torch, bwd_coord, reps, stream)
    del cgrad
    res["fwd_gaussians_per_s"] = n / (res["fwd_ms"] / 1e3)
    # plain FP32 GPU form (baseline to beat): FP32 tables, f_h in HBM, CUDA-core decoder, scalar atomics
    tab32 = wl.table.float()
    grad32 = torch.zeros_like(wl.table_grad)
    feat = torch.empty((n, wl.mlpc.d_in), dtype=torch.float32, device=wl.table.device)
    dfeat = torch.empty_like(feat)
    delta = torch.empty((wl.mlpc.d_out, n), dtype=torch.float32, device=wl.table.device)
    dd = wl.ddelta[:, :n].contiguous()
    mg = torch.zeros_like(wl.mlp_grad)
    wsz = torch.empty(4 * wl.mlpc.d_hidden * n * 4, dtype=torch.uint8, device=wl.table.device)
    torch.cuda.synchronize()
    pts = dash.Points(wl.x, wl.y, wl.z, wl.t, idx=wl.idx[:n].contiguous(), n=n)

    def plain():
        dash.dash_compact_dynamic(wl.mask, idx_out=wl.idx, count_out=wl.count, ws=wl.ws)
        dash.dash_plain_hash4d_fwd(wl.layout, pts, tab32, out=feat)
        dash.dash_plain_mlp_fwd(wl.mlp, feat, out=delta)
        dash.dash_plain_mlp_bwd(wl.mlp, feat, dd, mg, dfeat=dfeat, ws=wsz)
        dash.dash_plain_hash4d_bwd(wl.layout, pts, dfeat, grad32)

    for _ in range(3):
        plain()
    res["plain_fp32_step_ms"] = time_steps(torch, plain, 10, stream)
    res["plain_fp32_gaussians_per_s"] = n / (res["plain_fp32_step_ms"] / 1e3)
    # cold L2: write 512 MB before every step, time only the step
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=wl.table.device)
    cold = []
    for _ in range(WARMUP_REPS):
        wl.step()
    for _ in range(MIN_REPS):
        flush.fill_(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        wl.step()
        b.record(stream)
        b.synchronize()
        cold.append(a.elapsed_time(b))
    res["cold_l2_step_ms"] = statistics.median(cold)
    res["cold_l2_gaussians_per_s"] = n / (res["cold_l2_step_ms"] / 1e3)
    del flush
    # the table-gradient scatter alone: FP32 buffers (the form the backward uses) and the
    # reduced-precision FP16 variant (half2 vector atomics), with the FP16 error against FP32
    dfeat = torch.randn((n, wl.mlpc.d_in), dtype=torch.float32, device=wl.table.device) * 0.05
    pts_c = dash.Points(wl.x, wl.y, wl.z, wl.t, idx=wl.idx[:n].contiguous(), n=n)
    g32 = torch.zeros_like(wl.table_grad)
    g16 = torch.zeros(wl.table_grad.shape, dtype=torch.float16, device=wl.table.device)
    res["scatter_fp32_ms"] = time_steps(torch, lambda: dash.dash_hash4d_bwd(wl.layout, pts_c, dfeat, g32), 10, stream)
    res["scatter_fp16_ms"] = time_steps(torch, lambda: dash.dash_hash4d_bwd_half(wl.layout, pts_c, dfeat, g16), 10,
                                        stream)
    g32.zero_()
    g16.zero_()
    dash.dash_hash4d_bwd(wl.layout, pts_c, dfeat, g32)
    dash.dash_hash4d_bwd_half(wl.layout, pts_c, dfeat, g16)
    torch.cuda.synchronize()
    res["scatter_fp16_rel_err_vs_fp32"] = float((g16.float() - g32).norm() / g32.norm())
    del g32, g16, dfeat
    res.update(run_morton(torch, args, stream))
    res.update(run_one_frame(torch, args, stream))
    res.update(run_decomp(torch, wl, stream))
    res.update(run_wo_dec(torch, stream))
    res.update(run_render(torch, stream))
    res.update(run_plain_configs(torch, stream))
    res.update(run_batched(torch, stream))
    return res


def run_morton(torch, args, stream):
    """The benchmark step on the same kind of scene with the Gaussians stored
    in the Z order of their positions (so consecutive dynamic Gaussians are
    spatial neighbours)."""
    wl = Workload(seed=2, n_all=args.n_all, n_dyn=args.n_dyn, device=torch.device("cuda"), morton=True)
    for _ in range(3):
        wl.step()
    res = {"morton_step_ms": time_steps(torch, wl.step, 50, stream)}
    for _ in range(3):
        wl.forward()
    res["morton_fwd_ms"] = time_steps(torch, wl.forward, 50, stream)
    res["morton_bwd_ms"] = time_steps(torch, wl.backward, 50, stream)
    res["morton_gaussians_per_s"] = args.n_dyn / (res["morton_step_ms"] / 1e3)
    del wl
    torch.cuda.empty_cache()
    return res


def run_one_frame(torch, args, stream):
    """The benchmark step with one timestamp for all Gaussians (t = 0.37
    broadcast, as when a training step renders one frame), in input order
    and in Z order."""
    from paper_2507_19141_gb300 import dash
    res = {}
    for key, morton in (("one_frame", False), ("one_frame_morton", True)):
        wl = Workload(seed=2, n_all=args.n_all, n_dyn=args.n_dyn, device=torch.device("cuda"), morton=morton)
        wl.t1 = torch.full((1,), 0.37, dtype=torch.float32, device="cuda")
        wl.pts = dash.Points(wl.x, wl.y, wl.z, wl.t1, idx=wl.idx, n=wl.n_all, n_dev=wl.count)
        for _ in range(3):
            wl.step()
        res[f"{key}_step_ms"] = time_steps(torch, wl.step, 50, stream)
        res[f"{key}_bwd_ms"] = time_steps(torch, wl.backward, 50, stream)
        res[f"{key}_bwd_no_replicas_ms"] = time_steps(torch, lambda: wl.backward(None, False), 50, stream)
        res[f"{key}_gaussians_per_s"] = args.n_dyn / (res[f"{key}_step_ms"] / 1e3)
        del wl
        torch.cuda.empty_cache()
    return res


def render_frame_setup(torch, n=106_600, width=1352, height=1014, seed=13, scale=(0.001, 0.01)):
    """Inference frame at the paper's FPS shape (1352 x 1014, ~106.6k Gaussians,
    half of them dynamic): canonical attributes SoA [10][n] (position,
    quaternion, scale), normalised canonical coordinates for the encoder, FP16
    tables and a BF16 decoder whose last layer is scaled by 1e-2 (small
    offsets), opacities and degree-3 SH colours."""
    import numpy as np
    from paper_2507_19141_gb300 import dash, synth
    rng = np.random.default_rng(seed)
    cam, g = synth.raster_scene(rng, n, width, height, scale=scale)
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    lo = g["mean"].min(axis=1, keepdims=True)
    hi = g["mean"].max(axis=1, keepdims=True)
    ncoord = ((g["mean"] - lo) / (hi - lo)).astype(np.float32)
    lay = dash.layout_from(grid)
    params = synth.mlp_params(rng, mlpc)
    D, H, O = mlpc.d_in, mlpc.d_hidden, mlpc.d_out
    params[H * D + H + H * H + H:] *= 1e-2
    f = {"cam": dash.camera(cam["view"], cam["fx"], cam["fy"], cam["cx"], cam["cy"], width, height, cam["near"],
                            cam["dilation"], cam["campos"], cam["bg"]),
         "n": n, "lay": lay, "mask": dev(synth.bernoulli_mask(rng, n)),
         "x": dev(ncoord[0]), "y": dev(ncoord[1]), "z": dev(ncoord[2]), "t": dev(np.array([0.37], np.float32)),
         "table": dev(synth.table_values(rng, lay.total, grid.F, np.float16)),
         "mlp": dash.Mlp(dev(params), D, H, O),
         "attrs_in": dev(np.concatenate([g["mean"], g["rot"], g["scale"]], 0)),
         "opacity": dev(g["opacity"]), "sh": dev(g["sh"])}
    f["attrs_out"] = f["attrs_in"].clone()
    f["idx"] = torch.empty(n, dtype=torch.int32, device="cuda")
    f["cnt"] = torch.empty(1, dtype=torch.int64, device="cuda")
    f["cws"] = torch.empty(dash.dash_compact_workspace_size(n), dtype=torch.uint8, device="cuda")
    f["delta"] = torch.empty((O, n), dtype=torch.float32, device="cuda")
    f["pts"] = dash.Points(f["x"], f["y"], f["z"], f["t"], idx=f["idx"], n=n, n_dev=f["cnt"])
    ao = f["attrs_out"]
    # the renderer reads the Eq. 10 output rows in place: x (0-2), r (3-6), s (7-9)
    f["G"] = dash.Gaussians(ao[0:3], ao[7:10], ao[3:7], f["opacity"], f["sh"], 3)
    f["image"] = torch.empty((3, height, width), dtype=torch.float32, device="cuda")
    return f


def render_frame(f, ws, cap, pairs):
    from paper_2507_19141_gb300 import dash
    dash.dash_compact_dynamic(f["mask"], idx_out=f["idx"], count_out=f["cnt"], ws=f["cws"])
    dash.dash_deform_mlp_fwd(f["lay"], f["pts"], f["table"], f["mlp"], delta_out=f["delta"],
                             apply=(f["attrs_in"], f["attrs_out"]))
    dash.dash_raster_fwd(f["cam"], f["G"], image=f["image"], ws=ws, max_pairs=cap, pairs_needed=pairs)


def run_render(torch, stream):
    """Inference frames at the paper's FPS shape: compaction + deformation
    forward (Eq. 10 applied) + splatting of all Gaussians; and the renderer's
    forward and backward alone."""
    from paper_2507_19141_gb300 import dash
    f = render_frame_setup(torch)
    dash.dash_compact_dynamic(f["mask"], idx_out=f["idx"], count_out=f["cnt"], ws=f["cws"])
    dash.dash_deform_mlp_fwd(f["lay"], f["pts"], f["table"], f["mlp"], delta_out=f["delta"],
                             apply=(f["attrs_in"], f["attrs_out"]))
    _, ws, cap, pairs = dash.dash_raster_fwd(f["cam"], f["G"], image=f["image"])   # sizes the pair buffer
    for _ in range(3):
        render_frame(f, ws, cap, pairs)
    r = {"render_n": f["n"], "render_size": [f["cam"].width, f["cam"].height], "render_pairs": int(pairs.item()),
         "render_pairs_per_gaussian": int(pairs.item()) / f["n"]}
    r["render_frame_ms"] = time_steps(torch, lambda: render_frame(f, ws, cap, pairs), 50, stream)
    r["render_fps"] = 1e3 / r["render_frame_ms"]
    r["render_raster_fwd_ms"] = time_steps(torch, lambda: dash.dash_raster_fwd(
        f["cam"], f["G"], image=f["image"], ws=ws, max_pairs=cap, pairs_needed=pairs), 50, stream)
    grads = {k: torch.zeros_like(getattr(f["G"], k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dimg = torch.randn_like(f["image"])
    dash.dash_raster_bwd(f["cam"], f["G"], dimg, ws, cap, grads)
    r["render_raster_bwd_ms"] = time_steps(torch, lambda: dash.dash_raster_bwd(f["cam"], f["G"], dimg, ws, cap, grads),
                                           20, stream)
    r["render_nan_free"] = bool(torch.isfinite(f["image"]).all().item())
    # a training frame: the frame above + splatting backward + Eq. 10 backward
    # + fused deformation backward with the Eq. 11 term (loss gradient stands
    # in as N(0,1) per pixel; no optimiser step)
    n = f["n"]
    st = dash.deform_state(f["mlp"], n, "cuda")
    d10 = torch.zeros((10, n), dtype=torch.float32, device="cuda")
    tg = {"mean": d10[0:3], "rot": d10[3:7], "scale": d10[7:10], "opacity": grads["opacity"], "sh": grads["sh"]}
    ddelta = torch.zeros((10, n), dtype=torch.float32, device="cuda")
    table_grad = torch.zeros((f["lay"].total, 2), dtype=torch.float32, device="cuda")
    mlp_grad = torch.zeros(f["mlp"].params.numel(), dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    smooth = (1.0, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300, loss)

    def train_frame():
        dash.dash_compact_dynamic(f["mask"], idx_out=f["idx"], count_out=f["cnt"], ws=f["cws"])
        dash.dash_deform_mlp_fwd(f["lay"], f["pts"], f["table"], f["mlp"], delta_out=f["delta"], fwd_state=st,
                                 apply=(f["attrs_in"], f["attrs_out"]))
        dash.dash_raster_fwd(f["cam"], f["G"], image=f["image"], ws=ws, max_pairs=cap, pairs_needed=pairs)
        dash.dash_raster_bwd(f["cam"], f["G"], dimg, ws, cap, tg)
        dash.dash_deform_apply_bwd(f["pts"], d10, ddelta=ddelta)
        dash.dash_deform_mlp_bwd(f["lay"], f["pts"], f["table"], f["mlp"], ddelta, table_grad, mlp_grad,
                                 fwd_state=st, smooth=smooth)

    for _ in range(3):
        train_frame()
    r["train_frame_ms"] = time_steps(torch, train_frame, 30, stream)
    r["train_frames_per_s"] = 1e3 / r["train_frame_ms"]
    # the same frame captured once into a CUDA graph and replayed
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):          # captured on a side stream, replayed on this one
        train_frame()
    graph.replay()
    r["train_frame_graph_ms"] = time_steps(torch, graph.replay, 30, stream)
    return r


def run_wo_dec(torch, stream):
    """The "w/o dec" comparison on the 600k-Gaussian scene shape (Bernoulli(0.5)
    dynamic mask, scene coordinates, per-Gaussian t): fused forward + backward
    over all Gaussians against compaction + the same over the dynamic ones,
    and the tables' occupancy (touched vertices, occupied entries, colliding
    vertices over the hashed levels) for both point sets."""
    import numpy as np
    from paper_2507_19141_gb300 import dash, synth
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(12)
    n_all = 600_000
    mask_h = synth.bernoulli_mask(rng, n_all)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, z, t = (dev(c) for c in synth.scene_coords(rng, n_all))
    lay = dash.layout_from(grid)
    table = dev(synth.table_values(rng, lay.total, grid.F, np.float16))
    mlp = dash.Mlp(dev(synth.mlp_params(rng, mlpc)), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    mask = dev(mask_h)
    idx = torch.empty(n_all, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    cws = torch.empty(dash.dash_compact_workspace_size(n_all), dtype=torch.uint8, device="cuda")
    dd = dev(synth.upstream_grad(rng, mlpc.d_out, n_all))
    delta = torch.empty((mlpc.d_out, n_all), dtype=torch.float32, device="cuda")
    st = dash.deform_state(mlp, n_all, "cuda")
    tg = torch.zeros((lay.total, grid.F), dtype=torch.float32, device="cuda")
    pg = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    pts_all = dash.Points(x, y, z, t)
    pts_dyn = dash.Points(x, y, z, t, idx=idx, n=n_all, n_dev=cnt)

    def step(pts, compact):
        if compact:
            dash.dash_compact_dynamic(mask, idx_out=idx, count_out=cnt, ws=cws)
        dash.dash_deform_mlp_fwd(lay, pts, table, mlp, delta_out=delta, fwd_state=st)
        dash.dash_deform_mlp_bwd(lay, pts, table, mlp, dd, tg, pg, fwd_state=st)

    r = {"wo_dec_n_all": n_all}
    for name, pts, compact in (("all", pts_all, False), ("dynamic", pts_dyn, True)):
        for _ in range(3):
            step(pts, compact)
        r[f"wo_dec_{name}_step_ms"] = time_steps(torch, lambda: step(pts, compact), 20, stream)
    r["wo_dec_dynamic_count"] = int(cnt.item())
    hashed = [l for l in range(grid.L) if not lay.dense[l]]
    cws2 = torch.empty(dash.dash_collision_workspace_size(lay, n_all), dtype=torch.uint8, device="cuda")
    for name, pts in (("all", pts_all), ("dynamic", pts_dyn)):
        stats = dash.dash_hash4d_collision_stats(lay, pts, ws=cws2)
        r[f"wo_dec_{name}_occupancy_ms"] = time_steps(torch, lambda: dash.dash_hash4d_collision_stats(
            lay, pts, out=stats, ws=cws2), 3, stream)
        s = stats.cpu().numpy()[hashed]
        V, E, C = (int(v) for v in s.sum(axis=0))
        r[f"wo_dec_{name}_hashed_vertices"] = V
        r[f"wo_dec_{name}_hashed_entries"] = E
        r[f"wo_dec_{name}_colliding_vertices"] = C
        r[f"wo_dec_{name}_collision_rate"] = C / V if V else 0.0
        r[f"wo_dec_{name}_vertices_per_entry"] = V / E if E else 0.0
        r[f"wo_dec_{name}_collision_rate_per_level"] = [round(float(c) / float(v), 4) if v else 0.0
                                                       for v, _, c in s]
    r["wo_dec_hashed_levels"] = hashed
    return r


# decomposition, algorithmic bytes per Gaussian: x, y, z, t (16) + 16 levels x 8
# corners x one FP16 F=2 entry (512) + dp (12) + norm (4) + p(t) (12);
# top-k: norm (4) + mask (1)
DECOMP_BYTES = 16 + 16 * 8 * 4 + 12 + 4 + 12
TOPK_BYTES = 4 + 1


def run_decomp(torch, wl, stream):
    """Decomposition producing the mask, over all Gaussians of the workload:
    G_3D (16 levels 16..2048, T = 2^19, FP16) + phi_p/phi_l norms, the top-50 %
    threshold, mask and Eq. 5 static loss, and the chain decomposition (with
    Eq. 4's p(t) at each Gaussian's timestamp) -> mask -> compaction."""
    import numpy as np
    from paper_2507_19141_gb300 import dash, synth
    rng = np.random.default_rng(11)
    lay3 = dash.dash_hash3d_layout(16, 2, 19, 16, 2048)
    D, H = 32, 64
    k = 1 / np.sqrt(D)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    table3 = dev(synth.table_values(rng, lay3.total, 2, np.float16))
    dec = dash.Mlp(dev(rng.uniform(-k, k, H * D + H + 3 * H + 3).astype(np.float32)), D, H, 3)
    n = wl.n_all
    dp = torch.empty((3, n), dtype=torch.float32, device="cuda")
    norm = torch.empty(n, dtype=torch.float32, device="cuda")
    mask = torch.empty(n, dtype=torch.uint8, device="cuda")
    tau = torch.empty(1, dtype=torch.float32, device="cuda")
    ls = torch.empty(1, dtype=torch.float32, device="cuda")
    pt = torch.empty((3, n), dtype=torch.float32, device="cuda")
    ws = torch.empty(dash.dash_topk_workspace_size(), dtype=torch.uint8, device="cuda")
    idx = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int64, device="cuda")
    cws = torch.empty(dash.dash_compact_workspace_size(n), dtype=torch.uint8, device="cuda")

    def dec_fwd():
        dash.dash_decomp_fwd(lay3, wl.x, wl.y, wl.z, table3, dec, dp_out=dp, norm_out=norm, t=wl.t, pt_out=pt)

    def topk():
        dash.dash_topk_mask(norm, 50.0, mask_out=mask, tau_out=tau, ws=ws, static_loss_out=ls)

    def chain():
        dec_fwd()
        topk()
        dash.dash_compact_dynamic(mask, idx_out=idx, count_out=cnt, ws=cws)

    for _ in range(3):
        chain()
    r = {"decomp_n": n, "decomp_ms": time_steps(torch, dec_fwd, 20, stream),
         "topk_ms": time_steps(torch, topk, 20, stream), "decomp_chain_ms": time_steps(torch, chain, 20, stream)}
    r["decomp_gbs"] = DECOMP_BYTES * n / (r["decomp_ms"] / 1e3) / 1e9
    r["topk_gbs"] = TOPK_BYTES * n / (r["topk_ms"] / 1e3) / 1e9
    r["decomp_chain_gaussians_per_s"] = n / (r["decomp_chain_ms"] / 1e3)
    r["decomp_dynamic_count"] = int(cnt.item())
    # training the decomposition: backward of an upstream dp gradient plus lambda_s L_s
    tg3 = torch.zeros((lay3.total, 2), dtype=torch.float32, device="cuda")
    pg3 = torch.zeros(dec.params.numel(), dtype=torch.float32, device="cuda")
    d_dp = torch.randn((3, n), dtype=torch.float32, device="cuda")
    bws = torch.empty(dash.dash_decomp_bwd_workspace_size(), dtype=torch.uint8, device="cuda")

    def dec_bwd():
        dash.dash_decomp_bwd(lay3, wl.x, wl.y, wl.z, table3, dec, tg3, pg3, d_dp=d_dp, mask=mask, lambda_s=1.0, ws=bws)

    dec_bwd()
    r["decomp_bwd_ms"] = time_steps(torch, dec_bwd, 20, stream)
    return r


def run_batched(torch, stream):
    """Batched form: 8 scenes with dynamic counts log-uniform in 50k..2M, 64
    timestamps each, FP16 tables and BF16 decoders per scene, one persistent
    graph-captured launch with the autotuned kernel form; then the same
    work list forward + backward in one graph."""
    import numpy as np
    from paper_2507_19141_gb300 import dash, synth
    counts, tss, rng = synth.batched()
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    lay = dash.layout_from(grid)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    scenes = []
    for n, ts in zip(counts, tss):
        x, y, z, _ = synth.scene_coords(rng, n)
        scenes.append({"table": dev(synth.table_values(rng, lay.total, grid.F, np.float16)),
                       "params": dev(synth.mlp_params(rng, mlpc)), "x": dev(x), "y": dev(y), "z": dev(z),
                       "timestamps": dev(ts),
                       "delta_out": torch.empty((len(ts), mlpc.d_out, n), dtype=torch.float32, device="cuda")})
    plan = dash.BatchPlan(lay, scenes)
    cache = os.path.join(ROOT, "paper_2507_19141_gb300", "_build", "autotune.json")
    form = plan.autotune(cache)
    plan.run()
    torch.cuda.synchronize()
    ms = time_steps(torch, plan.run, 3, stream)
    evals = sum(counts) * len(tss[0])
    plan.close()
    # forward + backward in one graph: upstream gradients N(0, 1) drawn on the
    # device (14 GB), FP32 table and decoder gradients per scene
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    for sc in scenes:
        sc["ddelta"] = torch.randn(sc["delta_out"].shape, generator=gen, device="cuda")
        sc["table_grad"] = torch.zeros((lay.total, grid.F), dtype=torch.float32, device="cuda")
        sc["mlp_grad"] = torch.zeros(mlpc.n_params, dtype=torch.float32, device="cuda")
    plan = dash.BatchPlan(lay, scenes, backward=True)
    form_b = plan.autotune(cache)  # forward form + 16 * backward form
    plan.run()
    torch.cuda.synchronize()
    ms_b = time_steps(torch, plan.run, 3, stream)
    plan.close()
    return {"batched_scenes": len(counts), "batched_counts": counts, "batched_timestamps": len(tss[0]),
            "batched_evaluations": evals, "batched_launch_ms": ms, "batched_form": form,
            "batched_evaluations_per_s": evals / (ms / 1e3),
            "batched_fwd_bwd_launch_ms": ms_b, "batched_fwd_bwd_form": form_b,
            "batched_fwd_bwd_evaluations_per_s": evals / (ms_b / 1e3)}


# --------------------------------------- the two plain FP32 configurations --
PLAIN_CONFIGS = {
    "tiny": "N=10k, xyzt ~ U[0,1], L=4 F=2 T=2^14, res 16->128 / 8->32, decoder 8-64-64-10, FP32 tables and "
            "weights, seed 0",
    "paper_plain": "600k Gaussians, Bernoulli(0.5) mask (~300k dynamic), scene coordinates, L=16 F=2 T=2^19, "
                   "res 16->2048 / 8->150, decoder 32-64-64-10, FP32 tables and weights, seed 1",
}


def plain_config(name, total):
    """Seeded inputs of one plain FP32 configuration: the synth workload, an
    FP32 table of `total` entries, FP32 decoder weights and the upstream
    gradient of its dynamic Gaussians (the GPU and oracle legs draw the same)."""
    import numpy as np
    from paper_2507_19141_gb300 import synth
    wl = synth.tiny() if name == "tiny" else synth.paper_plain()
    rng = np.random.default_rng(1000 + wl.seed)
    table = synth.table_values(rng, total, wl.grid.F, np.float32)
    params = synth.mlp_params(rng, wl.mlp, bf16=False)
    n_dyn = len(wl.coords[0]) if wl.mask is None else int(np.count_nonzero(wl.mask))
    dd = synth.upstream_grad(rng, wl.mlp.d_out, n_dyn)
    return wl, table, params, dd


def run_plain_configs(torch, stream):
    """The plain FP32 GPU form and the fused form on the two plain FP32
    configurations, one step each (compaction where the configuration has a
    mask, encoder + decoder forward, decoder + encoder backward)."""
    import numpy as np
    from paper_2507_19141_gb300 import dash
    res = {}
    for name in PLAIN_CONFIGS:
        from paper_2507_19141_gb300 import synth
        grid = (synth.tiny() if name == "tiny" else synth.paper_plain()).grid
        lay = dash.layout_from(grid)
        wl, table, params, dd_h = plain_config(name, lay.total)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        n_all, n = len(wl.coords[0]), dd_h.shape[1]
        D, H, O = wl.mlp.d_in, wl.mlp.d_hidden, wl.mlp.d_out
        x, y, z, t = (dev(c) for c in wl.coords)
        tab, dd = dev(table), dev(dd_h)
        mlp = dash.Mlp(dev(params), D, H, O)
        idx = torch.arange(n_all, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), n, dtype=torch.int64, device="cuda")
        mask = None if wl.mask is None else dev(wl.mask)
        cws = torch.empty(dash.dash_compact_workspace_size(n_all), dtype=torch.uint8, device="cuda")
        pts = dash.Points(x, y, z, t, idx=idx, n=n, n_dev=cnt)
        feat = torch.empty((n, D), dtype=torch.float32, device="cuda")
        dfeat = torch.empty_like(feat)
        delta = torch.empty((O, n), dtype=torch.float32, device="cuda")
        tg = torch.zeros((lay.total, grid.F), dtype=torch.float32, device="cuda")
        pg = torch.zeros(wl.mlp.n_params, dtype=torch.float32, device="cuda")
        wsz = torch.empty(4 * H * n * 4, dtype=torch.uint8, device="cuda")
        state = dash.deform_state(mlp, n, "cuda")

        def compact():
            if mask is not None:
                dash.dash_compact_dynamic(mask, idx_out=idx, count_out=cnt, ws=cws)

        def plain():
            compact()
            dash.dash_plain_hash4d_fwd(lay, pts, tab, out=feat)
            dash.dash_plain_mlp_fwd(mlp, feat, out=delta)
            dash.dash_plain_mlp_bwd(mlp, feat, dd, pg, dfeat=dfeat, ws=wsz)
            dash.dash_plain_hash4d_bwd(lay, pts, dfeat, tg)

        def fused():
            compact()
            dash.dash_deform_mlp_fwd(lay, pts, tab, mlp, delta_out=delta, fwd_state=state)
            dash.dash_deform_mlp_bwd(lay, pts, tab, mlp, dd, tg, pg, fwd_state=state)

        for key, fn in (("plain_fp32", plain), ("fused", fused)):
            ms = time_steps(torch, fn, MIN_REPS, stream)
            res[f"{name}_{key}_step_ms"] = ms
            res[f"{name}_{key}_gaussians_per_s"] = n / (ms / 1e3)
        res[f"{name}_n_dynamic"] = n
        del tab, tg, state, wsz
        torch.cuda.empty_cache()
    res["plain_configs"] = PLAIN_CONFIGS
    return res


# ------------------------------------------------------------ CPU oracle --
class OracleTimer:
    """The FP64 oracle's forward + backward (one host thread) on samples of
    the benchmark's distribution.  The tables, decoder weights and the
    gradient buffer are made once (the buffer written through, so no timed
    call pays first-touch page faults); each sample draws new coordinates
    and upstream gradients."""

    def __init__(self, seed=7):
        import numpy as np
        import oracle
        from paper_2507_19141_gb300 import synth
        self.np, self.oracle, self.synth = np, oracle, synth
        grid, self.mlpc = synth.PAPER_GRID, synth.PAPER_MLP
        rng = np.random.default_rng(seed)
        self.g = oracle.layout(grid.L, grid.F, grid.log2_T, grid.nmin_s, grid.nmax_s, grid.nmin_t, grid.nmax_t)
        self.table = synth.table_values(rng, self.g.total, grid.F, np.float16).astype(np.float64)
        self.params = synth.mlp_params(rng, self.mlpc).astype(np.float64)
        self.tg = np.zeros((self.g.total, grid.F))
        self.tg[:] = 1.0
        self.tg[:] = 0.0

    def run(self, sample_n, seed):
        """Returns (Gaussians/s, seconds) for one sample of sample_n Gaussians."""
        np, oracle, synth, mlpc = self.np, self.oracle, self.synth, self.mlpc
        rng = np.random.default_rng(seed)
        pts = oracle.Points(*synth.scene_coords(rng, sample_n))
        dd = synth.upstream_grad(rng, mlpc.d_out, sample_n).astype(np.float64)
        t0 = time.perf_counter()
        oracle.deform_fwd(self.g, pts, self.table, mlpc.d_hidden, mlpc.d_out, self.params)
        oracle.deform_bwd(self.g, pts, self.table, mlpc.d_hidden, mlpc.d_out, self.params, dd, table_grad=self.tg)
        dt = time.perf_counter() - t0
        return sample_n / dt, dt


def cpu_baseline(args, wl=None):
    timer = OracleTimer()
    n = args.cpu_sample
    if n <= 0:
        rate, _ = timer.run(5000, seed=6)
        n = int(min(max(rate * 10.0, 5000), 1_000_000))
    rate, dt = timer.run(n, seed=7)
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n} dynamic Gaussians of the same distribution, forward + backward, {dt:.1f} s, "
                      f"1 host thread of {os.cpu_count()} cores"}


def _oracle_process(n, seed, barrier, queue):
    """One host process of the all-cores oracle timing (spawned)."""
    timer = OracleTimer()
    timer.run(200, seed=seed + 10_000)
    barrier.wait(timeout=300)
    _, dt = timer.run(n, seed)
    queue.put((n, dt))


def cpu_baseline_all_cores(per_core_rate, seconds=5.0):
    """The same oracle in one single-threaded process per host core, all
    started together (spawned processes: the parent holds a CUDA context),
    each on its own sample of about `seconds` of work; the rate is the
    Gaussians of all samples over the slowest process's time."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    n = int(min(max(per_core_rate * seconds, 1000), 500_000))
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_process, args=(n, 500 + i, barrier, queue), daemon=True)
             for i in range(cores)]
    for pr in procs:
        pr.start()
    try:
        res = [queue.get(timeout=600) for _ in procs]
    except Exception as e:  # a process that died: report, do not hang the benchmark
        for pr in procs:
            pr.terminate()
        return {"unavailable": f"all-cores oracle timing failed: {type(e).__name__}"}
    for pr in procs:
        pr.join(timeout=60)
    wall = max(dt for _, dt in res)
    total = sum(k for k, _ in res)
    return {"value": total / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} processes x {n} dynamic Gaussians of the same distribution, forward + backward, "
                      f"{wall:.1f} s (one single-threaded oracle per host core)"}


class PlainOracle:
    """The FP64 oracle on one plain FP32 configuration: compaction of its
    mask (where it has one), forward and backward of its dynamic Gaussians
    (or of the slice [lo, hi) of them) into an FP64 table gradient."""

    def __init__(self, name):
        import numpy as np
        import oracle
        from paper_2507_19141_gb300 import synth
        grid = (synth.tiny() if name == "tiny" else synth.paper_plain()).grid
        self.np, self.oracle = np, oracle
        self.g = oracle.layout(grid.L, grid.F, grid.log2_T, grid.nmin_s, grid.nmax_s, grid.nmin_t, grid.nmax_t)
        self.wl, table, params, self.dd = plain_config(name, self.g.total)
        self.table, self.params = table.astype(np.float64), params.astype(np.float64)
        self.dd = self.dd.astype(np.float64)
        self.tg = np.zeros((self.g.total, grid.F))

    def run(self, lo=0, hi=None):
        """Returns (Gaussians evaluated, seconds)."""
        np, oracle, wl = self.np, self.oracle, self.wl
        t0 = time.perf_counter()
        if wl.mask is None:
            idx = np.arange(len(wl.coords[0]), dtype=np.int32)
        else:
            idx, _ = oracle.compact(wl.mask)
        hi = len(idx) if hi is None else hi
        pts = oracle.Points(*wl.coords, idx=idx[lo:hi])
        oracle.deform_fwd(self.g, pts, self.table, wl.mlp.d_hidden, wl.mlp.d_out, self.params)
        oracle.deform_bwd(self.g, pts, self.table, wl.mlp.d_hidden, wl.mlp.d_out, self.params,
                          np.ascontiguousarray(self.dd[:, lo:hi]), table_grad=self.tg)
        return hi - lo, time.perf_counter() - t0


def _plain_oracle_process(name, lo, hi, barrier, queue):
    """One host process of the all-cores timing of a plain configuration (spawned)."""
    po = PlainOracle(name)
    barrier.wait(timeout=300)
    queue.put(po.run(lo, hi))


def oracle_plain_configs():
    """The FP64 oracle on the two plain FP32 configurations in full: one host
    thread, and one single-threaded process per host core, each on its own
    contiguous slice of the dynamic Gaussians (the rate is all Gaussians over
    the slowest process's time)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    out = {}
    for name in PLAIN_CONFIGS:
        po = PlainOracle(name)
        n, dt = po.run()
        out[f"{name}_oracle_1_thread"] = {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                          "sample": f"all {n} dynamic Gaussians (compaction + forward + "
                                                    f"backward), {dt:.2f} s"}
        ctx = mp.get_context("spawn")
        barrier, queue = ctx.Barrier(cores), ctx.Queue()
        cuts = [n * i // cores for i in range(cores + 1)]
        procs = [ctx.Process(target=_plain_oracle_process, args=(name, cuts[i], cuts[i + 1], barrier, queue),
                             daemon=True) for i in range(cores)]
        for pr in procs:
            pr.start()
        try:
            res = [queue.get(timeout=600) for _ in procs]
        except Exception as e:  # a process that died: report, do not hang the benchmark
            for pr in procs:
                pr.terminate()
            out[f"{name}_oracle_all_cores"] = {"unavailable": f"all-cores oracle timing failed: {type(e).__name__}"}
            continue
        for pr in procs:
            pr.join(timeout=60)
        wall = max(d for _, d in res)
        out[f"{name}_oracle_all_cores"] = {"value": n / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
                                           "sample": f"all {n} dynamic Gaussians in {cores} slices, one "
                                                     f"single-threaded process per core, {wall:.2f} s"}
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist_init("gloo")
        if rank != 0:
            barrier()
            return
    timer = OracleTimer()
    rate, _ = timer.run(2000, seed=99)
    budget = 120.0  # seconds of oracle work for the whole warmup + steps run
    per_step = budget / max(1, args.steps + args.warmup)
    sample = int(min(max(rate * per_step, 500), 100_000))
    for i in range(args.warmup):
        timer.run(sample, seed=100 + i)
    total_t, total_n = 0.0, 0
    for i in range(args.steps):
        r, dt = timer.run(sample, seed=200 + i)
        total_t += dt
        total_n += sample
    value = total_n / total_t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_t / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded)",
           "config": step_config(args, ws),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": f"FP64 oracle forward + backward (no compaction) of {sample} dynamic "
                                      f"Gaussians of the same distribution per step x {args.steps} steps, "
                                      f"1 host thread"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    if ws > 1:
        barrier()


def profile_case(n):
    """Small case for ncu captures: n dynamic Gaussians (no compaction), about
    1 GB on the device, two launches each of the encoder forward/backward, the
    fused forward/backward (the backward once more with the coordinate
    gradient and once with the Eq. 11 term), the decomposition with its top-k mask and its backward, one
    occupancy count, two runs of a batched forward + backward plan (2 scenes
    of 600k and 400k, 2 timestamps each), and
    two render frames (1352 x 1014, 106.6k Gaussians) with the renderer's
    backward."""
    import numpy as np
    import torch
    from paper_2507_19141_gb300 import dash, synth
    grid, mlpc = synth.PAPER_GRID, synth.PAPER_MLP
    rng = np.random.default_rng(2)
    x, y, z, t = synth.scene_coords(rng, n)
    lay = dash.layout_from(grid)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    table = dev(synth.table_values(rng, lay.total, grid.F, np.float16))
    mlp = dash.Mlp(dev(synth.mlp_params(rng, mlpc)), mlpc.d_in, mlpc.d_hidden, mlpc.d_out)
    pts = dash.Points(dev(x), dev(y), dev(z), dev(t))
    delta = torch.empty((mlpc.d_out, n), device="cuda")
    state = dash.deform_state(mlp, n, "cuda")
    feat = torch.empty((n, mlpc.d_in), dtype=torch.bfloat16, device="cuda")
    tg = torch.zeros((lay.total, grid.F), device="cuda")
    pg = torch.zeros(mlpc.n_params, device="cuda")
    dd = dev(synth.upstream_grad(rng, mlpc.d_out, n))
    dfeat = dev(rng.standard_normal((n, mlpc.d_in)).astype(np.float32))
    lay3 = dash.dash_hash3d_layout(16, 2, 19, 16, 2048)
    table3 = dev(synth.table_values(rng, lay3.total, 2, np.float16))
    k = 1 / np.sqrt(32)
    dec = dash.Mlp(dev(rng.uniform(-k, k, 64 * 32 + 64 + 3 * 64 + 3).astype(np.float32)), 32, 64, 3)
    cg = torch.empty((4, n), device="cuda")
    tg3 = torch.zeros((lay3.total, 2), dtype=torch.float32, device="cuda")
    pg3 = torch.zeros(dec.params.numel(), dtype=torch.float32, device="cuda")
    d_dp = torch.randn((3, n), dtype=torch.float32, device="cuda")
    for _ in range(2):
        dash.dash_hash4d_fwd(lay, pts, table, torch.bfloat16, out=feat)
        dash.dash_hash4d_bwd(lay, pts, dfeat, tg)
        dash.dash_deform_mlp_fwd(lay, pts, table, mlp, delta_out=delta, fwd_state=state)
        dash.dash_deform_mlp_bwd(lay, pts, table, mlp, dd, tg, pg, fwd_state=state)
        dash.dash_deform_mlp_bwd(lay, pts, table, mlp, dd, tg, pg, fwd_state=state, coord_grad=cg)
        dash.dash_deform_mlp_bwd(lay, pts, table, mlp, dd, tg, pg, fwd_state=state,
                                 smooth=(1.0, (1 / 2048, 1 / 2048, 1 / 2048), 1 / 300, None))
        _, norm, _ = dash.dash_decomp_fwd(lay3, pts.x, pts.y, pts.z, table3, dec, t=pts.t)
        mask, _ = dash.dash_topk_mask(norm, 50.0)
        dash.dash_decomp_bwd(lay3, pts.x, pts.y, pts.z, table3, dec, tg3, pg3, d_dp=d_dp, mask=mask, lambda_s=1.0)
    dash.dash_hash4d_collision_stats(lay, pts)
    # the batched forward + backward: 2 scenes (600k, 400k) x 2 timestamps
    scenes = []
    for m in (600_000, 400_000):
        bx, by, bz, _ = synth.scene_coords(rng, m)
        scenes.append({"table": dev(synth.table_values(rng, lay.total, grid.F, np.float16)),
                       "params": dev(synth.mlp_params(rng, mlpc)), "x": dev(bx), "y": dev(by), "z": dev(bz),
                       "timestamps": dev(np.array([0.25, 0.75], dtype=np.float32)),
                       "delta_out": torch.empty((2, mlpc.d_out, m), device="cuda"),
                       "ddelta": torch.randn((2, mlpc.d_out, m), device="cuda"),
                       "table_grad": torch.zeros((lay.total, grid.F), device="cuda"),
                       "mlp_grad": torch.zeros(mlpc.n_params, device="cuda")})
    plan = dash.BatchPlan(lay, scenes, backward=True)
    for _ in range(2):
        plan.run()
    torch.cuda.synchronize()
    plan.close()
    # render frames at 1352 x 1014 with 106.6k Gaussians, and the renderer's backward
    f = render_frame_setup(torch)
    _, rws, cap, pairs = dash.dash_raster_fwd(f["cam"], f["G"], image=f["image"])
    grads = {k: torch.zeros_like(getattr(f["G"], k)) for k in ("mean", "scale", "rot", "opacity", "sh")}
    dimg = torch.randn_like(f["image"])
    for _ in range(2):
        render_frame(f, rws, cap, pairs)
        dash.dash_raster_bwd(f["cam"], f["G"], dimg, rws, cap, grads)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": n, "delta_abs_mean": float(delta.abs().mean()),
                      "grad_abs_sum": float(tg.abs().sum())}))


def main(argv=None):
    args = parse_args(argv)
    if args.profile_case:
        profile_case(args.n_dyn)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
