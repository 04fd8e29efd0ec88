#!/usr/bin/env python
"""Benchmark of the VG-rtTDDFTB propagation step on GB300.

Workload: 512-atom silicon-like supercell (4x4x4 diamond cells, Gaussian
displacements sigma = 0.3 bohr, sp3 basis, N = 2048 orbitals), Gamma point,
delta kick A_x = 0.001 a.u., dt = 0.2 a.u., SCC on (synthetic inputs from
paper_2308_09782_gb300.inputs, config "si512_kick").  One step = one leapfrog
step of the whole hot path: Mulliken/current/energy reductions, SCC shift,
Bloch-sum phase build, both commutator products, leapfrog update.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  value = steps/s of the split-precision
(tcgen05 BF16x3, delta form) path summed over ranks (independent replicas);
the plain FP64 path and the J(t) error of the split path against it are
reported beside it.  --impl reference times the CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "steps/s at 512-atom Si: FP64 vs split-precision @ J err≤1e-4; % of peak"
CONFIG = "si512_kick"
WORKLOAD = ("512-atom Si supercell (diamond 4x4x4, sigma=0.3 bohr), sp3, N=2048 orbitals, Gamma, "
            "kick A_x=0.001 au, dt=0.2 au, SCC on")
AU_FS = 0.0241888432658
P1 = {"auto": 0, "dense": 1, "blocks": 2}     # vgtb_options.product1
CHAIN = {"auto": 0, "off": 1, "on": 2}       # vgtb_options.chain


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["native", "reference"], default="native")
    p.add_argument("--fp64-steps", type=int, default=20)
    p.add_argument("--cpu-steps", type=int, default=6)
    p.add_argument("--tiles", default="auto",
                   help="tcgen05 tile variants of product 1,2 (e.g. 1,0) instead of the autotuner's choice")
    p.add_argument("--laser-steps", type=int, default=0,
                   help="laser workload: steps to run (0 = the whole 20 fs pulse)")
    p.add_argument("--cn-steps", type=int, default=4,
                   help="timed steps of the FP64 Crank-Nicolson integrator (0 = skip)")
    p.add_argument("--steady-steps", type=int, default=1000,
                   help="steps per window of the three steady-state windows timed after the headline (0 = skip)")
    p.add_argument("--batched-steps", type=int, default=100,
                   help="timed steps of the batched form inside the headline run (0 = skip)")
    p.add_argument("--product1", choices=["auto", "dense", "blocks"], default="auto",
                   help="form of the split path's first product (vgtb_options.product1)")
    p.add_argument("--chain", choices=["auto", "off", "on"], default="auto",
                   help="both tcgen05 products in one launch (vgtb_options.chain): auto = kept when faster at create")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-1thread-steps", type=int, default=1,
                   help="oracle steps timed again with one BLAS thread (0 = skip)")
    p.add_argument("--oracle-probe", type=int, default=0, help=argparse.SUPPRESS)
    p.add_argument("--workload", choices=["si512", "batched", "laser"], default="si512",
                   help="si512: the headline; batched: 64/216/512-atom supercells x 8 k x 6 fields in one context; "
                        "laser: the 2.3/3.9/6.0 eV pulse sweep on the 512-atom cell with charge transfer between "
                        "coordination classes")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; independent replicas)
# ---------------------------------------------------------------------------
def dist_setup(use_cuda: bool):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if use_cuda:
        torch.cuda.set_device(local)
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return rank, world, local


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        lines = open(self.path).read().splitlines()
        os.unlink(self.path)
        return parse_clock_csv(lines)


def parse_clock_csv(lines):
    """Median SM clock, max clock and the throttle reasons seen in nvidia-smi CSV rows
    (fields as in ClockSampler.FIELDS, no header, no units)."""
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
            power.append(float(f[3]))
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    return {"sm_mhz": float(np.median(sm)) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------
def fp64_peak_tflops(torch, n=2048, reps=5):
    """cuBLAS ZGEMM yardstick for the FP64 kernels: best of `reps` complex128
    n^3 products (8 n^3 flops each) on the current device."""
    a = torch.randn(n, n, dtype=torch.complex128, device="cuda")
    b = torch.randn(n, n, dtype=torch.complex128, device="cuda")
    torch.matmul(a, b)
    best = 1e30
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 8.0 * n ** 3 / (best * 1e-3) / 1e12


def nonzeros(sysd):
    """Complex nonzeros of H_k: the n_I x n_J elements of every distinct atom pair (I, J)."""
    blk = np.asarray(sysd["blk_ijl"])
    norb = np.diff(np.asarray(sysd["orb_offset"]))
    pairs = np.unique(blk[:, :2], axis=0)
    return int(np.sum(norb[pairs[:, 0]] * norb[pairs[:, 1]]))


def fp32_alu_peak(peaks):
    """FP32 FMA peak of the GPU from its unit counts and maximum SM clock: SMs x 128
    FP32 lanes x 2 flops x clock (the block-sparse product runs on these lanes)."""
    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz") or 2070.0)
    return nsm * 128 * 2 * mhz * 1e6 / 1e12, (f"FP32 FMA: {nsm} SMs x 128 lanes x 2 flops x {mhz:.0f} MHz "
                                             "(derived from unit counts and the maximum SM clock)")


def split_product_rooflines(systems, n_items, stats, tiles, peaks):
    """Roofline of both commutator products of the split form, in algorithmic flops.

    Product 1, block-sparse (product1 = BLOCKS): W = dD H + D0 dH over the nonzero
    atom blocks, 2 x 8 nnz(H) N FP32 flops per item (the minimum of Eq. 6 is one
    such product, 8 nnz N), against the FP32 ALU peak.  Product 1, dense tcgen05
    (the split form's default): 3 split terms x 8 N^3 = 24 N^3 per item.  Product 2 (tcgen05
    BF16x3): 24 N^3 per item (unpadded N; the kernel executes 24 Np^3).  Both
    tensor figures are against the measured sustained BF16 peak."""
    sust = peaks.get("bf16_tflops_sustained")
    sust_kind = "measured sustained bf16 (MEASURED_PEAKS.json)"
    if sust is None:
        sust, sust_kind = 1700.0, "fallback sustained bf16"
    burst = peaks.get("bf16_tflops", 1900.0)
    g1 = stats["gemm1"][1] / max(stats["gemm1"][0], 1)
    g2 = stats["gemm2"][1] / max(stats["gemm2"][0], 1)
    n3 = sum(n_it * float(int(s["orb_offset"][-1])) ** 3 for s, n_it in zip(systems, n_items))
    np3 = sum(n_it * float((int(s["orb_offset"][-1]) + 127) // 128 * 128) ** 3 for s, n_it in zip(systems, n_items))
    if "one launch" in tiles["product1"].get("schedule", ""):
        # both products run in one persistent launch (the library times it as
        # product 1): one roofline over the launch, 2 x 24 N^3 algorithmic flops
        f = 48.0 * n3
        a = f / (g1 * 1e-3) / 1e12
        kept = tiles["product1"]["schedule"]
        pc = {"kernel": "k_tc_chain (products 1 and 2 in one persistent tcgen05 launch: W = [dD|D0][H|dH]^dagger, "
                        "then X = S^-1 W^dagger, BF16x3)",
              "bound": "tensor", "achieved": round(a, 1), "peak": sust, "unit": "TFLOP/s",
              "frac": round(a / sust, 4), "peak_kind": sust_kind, "frac_of_burst": round(a / burst, 4),
              "flops_per_launch": f,
              "flops_note": "2 products x 3 split terms x 8 N^3 (algorithmic, unpadded N); the launch executes "
                            f"at most {72 * np3:.3e} BF16 flops (product 1 with K' = 4 Np before its zero k-panels "
                            "are skipped, product 2 with K' = 2 Np)",
              "executed_tflops_upper": round(72 * np3 / (g1 * 1e-3) / 1e12, 1), "avg_launch_ms": round(g1, 4),
              "schedule": kept, "traffic": kernel_traffic("tc_chain", float(sum(n_items)), tiles["product1"])}
        return pc, None
    if tiles["product1"].get("schedule") == "block-sparse":
        f1 = sum(n_it * 2 * 8.0 * nonzeros(s) * int(s["orb_offset"][-1]) for s, n_it in zip(systems, n_items))
        alu, alu_kind = fp32_alu_peak(peaks)
        a1 = f1 / (g1 * 1e-3) / 1e12
        p1 = {"kernel": "k_bsr<float,8> (product 1: W = dD H + D0 dH over the nonzero atom blocks, FP32)",
              "bound": "alu", "achieved": round(a1, 2), "peak": round(alu, 2), "unit": "TFLOP/s",
              "frac": round(a1 / alu, 4), "peak_kind": alu_kind, "flops_per_launch": f1,
              "flops_note": "2 x 8 nnz(H) N (delta form: dD H and D0 dH); Eq. 6 minimum is 8 nnz(H) N",
              "avg_launch_ms": round(g1, 4), "traffic": kernel_traffic("bsr_f32", float(sum(n_items)))}
    else:
        f1 = 24.0 * n3
        a1 = f1 / (g1 * 1e-3) / 1e12
        p1 = {"kernel": "k_tc_gemm (product 1: W = [dD|D0][H|dH]^dagger, tcgen05 BF16x3, dense)",
              "bound": "tensor", "achieved": round(a1, 1), "peak": sust, "unit": "TFLOP/s",
              "frac": round(a1 / sust, 4), "peak_kind": sust_kind, "frac_of_burst": round(a1 / burst, 4),
              "flops_per_launch": f1, "flops_note": "3 split terms x 8 N^3 (algorithmic); the kernel executes "
                                                    f"{48 * np3:.3e} BF16 flops (K' = 4 Np, padded)",
              "executed_tflops": round(48 * np3 / (g1 * 1e-3) / 1e12, 1), "avg_launch_ms": round(g1, 4),
              "traffic": kernel_traffic("tc_gemm1", float(sum(n_items)), tiles["product1"])}
    f2 = 24.0 * n3
    a2 = f2 / (g2 * 1e-3) / 1e12
    p2 = {"kernel": "k_tc_gemm2<3,1> (product 2: X = S^-1 W^dagger, tcgen05 BF16x3)", "bound": "tensor",
          "achieved": round(a2, 1), "peak": sust, "unit": "TFLOP/s", "frac": round(a2 / sust, 4),
          "peak_kind": sust_kind, "frac_of_burst": round(a2 / burst, 4), "flops_per_launch": f2,
          "flops_note": "3 split terms x 8 N^3 (algorithmic, unpadded N)",
          "executed_tflops": round(24 * np3 / (g2 * 1e-3) / 1e12, 1), "avg_launch_ms": round(g2, 4),
          "traffic": kernel_traffic("tc_gemm2", float(sum(n_items)), tiles["product2"])}
    return p1, p2



def launches_per_step(tiles):
    """Kernels of one split-form step: the observable and SCC kernels, the phase build,
    the products (one launch when chained, else two) and the leapfrog."""
    return 5 if "one launch" in tiles["product1"].get("schedule", "") else 6


def hbm_rates(sysd, Np, kern_ms, peak_gbs, sparse=True):
    """Achieved GB/s of the HBM-side kernels from their algorithmic bytes per step and
    their live CUDA-event times (the small kernels are latency-bound)."""
    blk = np.asarray(sysd["blk_ijl"])
    off = np.asarray(sysd["orb_offset"])
    norb = np.diff(off)
    el_img = int(np.sum(norb[blk[:, 0]] * norb[blk[:, 1]]))          # values of all image blocks
    pairs = np.unique(blk[:, :2], axis=0)
    n_el = int(np.sum(norb[pairs[:, 0]] * norb[pairs[:, 1]]))        # nonzeros of H_k
    nat = len(norb)
    nk = len(sysd["wk"])
    byts = {
        "leap": 56 * Np * Np,                                        # X, R0 f32; dD r/w f64; f32 copy or pieces
        # S, H0, dS f32 per image; out: H and dH at the nonzeros (2 x float2) or embedded BF16 pieces (16 x 2 B)
        "phase": nk * (20 * el_img + 8 * len(blk) + (16 if sparse else 32) * n_el),
        "obs": nk * 96 * n_el + 40 * nat,                            # dD f64 + S, P, H0 blocks f64
        "scc": 8 * nat * nat + 64 * nat,                             # gamma + per-atom vectors
    }
    out = {}
    for k, b in byts.items():
        ms = kern_ms.get(k)
        if not ms:
            continue
        gbs = b / (ms * 1e-3) / 1e9
        out[k] = {"bytes": int(b), "GB/s": round(gbs, 1),
                  "frac": round(gbs / peak_gbs, 4) if peak_gbs else None}
    out["peak_gbs"] = peak_gbs
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def kernel_traffic(kernel: str, per_launch_units: float, tile=None):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source
    is unchanged since the capture and (for the products) the capture ran the
    same tile variant; None otherwise."""
    try:
        recs = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    for rec in (recs if isinstance(recs, list) else [recs]):
        src = os.path.join(ROOT, rec["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()
        if h == rec["sha256"] and (tile is None or rec.get("tile") == tile):
            return rec["bytes_per_unit"] * per_launch_units
    return None


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def cpu_baseline(nsteps: int, sysd=None, A=None, warm_up=True):
    import oracle as O
    from paper_2308_09782_gb300 import inputs
    if sysd is None:
        sysd, A, _ = inputs.config(CONFIG)
    t0 = time.perf_counter()
    ctx = O.setup(sysd)
    # a Hermitian start density with Tr(D S) = N_el; a step costs the same for any values
    n_orb = int(sysd["orb_offset"][-1])
    D0 = [(float(sysd["n_electrons"]) / n_orb) * Si for Si in ctx["Sinv"]]
    t_setup = time.perf_counter() - t0
    if warm_up:
        O.propagate(sysd, A, 1, D0, ctx=ctx)        # warm-up (one step)
    t1 = time.perf_counter()
    O.propagate(sysd, A, nsteps, D0, ctx=ctx)
    dt = time.perf_counter() - t1
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": nsteps / dt, "unit": "steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{nsteps} oracle steps{' (plus 1 warm-up)' if warm_up else ''} of {CONFIG} (N=2048, "
                      f"Gamma) from D0 = (N_el/N) S^-1; numpy complex128, OpenBLAS threads = {cores} cores; "
                      f"setup {t_setup:.1f} s not timed"}


def cpu_baseline_1thread(nsteps: int):
    """The same oracle timing in a child process limited to one BLAS/OpenMP thread."""
    if nsteps <= 0:
        return None
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-probe", str(nsteps)],
                             env=env, capture_output=True, text=True, timeout=900)
    except subprocess.TimeoutExpired:
        return None
    if out.returncode != 0 or not out.stdout.strip():
        return None
    return json.loads(out.stdout.strip().splitlines()[-1])


def with_1thread(cpu: dict, nsteps: int) -> dict:
    one = cpu_baseline_1thread(nsteps)
    if one is not None:
        cpu["value_1thread"] = one["value"]
        cpu["sample_1thread"] = one["sample"].replace(f"{one['cores']} cores", "1 thread")
    return cpu


def steady_windows(ctx, stream, nsteps, local, windows=3):
    """Three more windows of nsteps steps after the headline region, each timed with
    CUDA events on the context stream, with the SM clocks sampled meanwhile: the
    median and spread of steps/s, and ms/step x median SM MHz (clock-normalised)."""
    import torch
    clk = ClockSampler(local)
    torch.cuda.synchronize()
    clk.start()
    vals = []
    for _ in range(windows):
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        ctx.propagate(nsteps)
        a1.record(stream)
        torch.cuda.synchronize()
        vals.append(nsteps / (a0.elapsed_time(a1) / 1e3))
    clocks = clk.stop()
    med = float(np.median(vals))
    out = {"steps_per_window": nsteps, "windows": windows, "steps_per_s": [round(v, 2) for v in sorted(vals)],
           "median": round(med, 2), "spread": round((max(vals) - min(vals)) / med, 4), "clocks": clocks}
    if clocks.get("sm_mhz"):
        out["ms_per_step_x_sm_mhz"] = round(1e3 / med * clocks["sm_mhz"], 2)
    return out


# ---------------------------------------------------------------------------
# native (GPU) arm
# ---------------------------------------------------------------------------
def native(args):
    import torch
    from paper_2308_09782_gb300 import inputs, vgtb
    rank, world, local = dist_setup(True)
    vgtb.load()
    sysd, A, _ = inputs.config(CONFIG)
    K, W = args.steps, max(args.warmup, 3)
    Kp = min(K, 500)                             # separate profiled pass for the per-kernel times
    Ks = max(args.steady_steps, 0)
    n_need = W + K + 3 * Ks + Kp + 1
    if A.shape[0] < n_need:                      # the kick is constant after t = 0
        A = np.tile(A[:1], (n_need, 1))
    stream = torch.cuda.current_stream()
    tile_opts = {"autotune": 1}
    if args.tiles != "auto":
        tile_opts = {"autotune": 0, "tile_variant": [int(x) for x in args.tiles.split(",")]}
    ctx = vgtb.Context(sysd, precision=vgtb.SPLIT_BF16X3, init=vgtb.INIT_GROUND,
                       cuda_stream=stream.cuda_stream, graph_steps=50, product1=P1[args.product1],
                       chain=CHAIN[args.chain], **tile_opts)
    ctx.set_field(0, A[:n_need])
    tiles = {f"product{p}": ctx.tile_config(p) for p in (1, 2)}
    tiles["choice"] = ("autotuned at create: fastest of the tcgen05 tile variants (median of 9 launches)"
                       if args.tiles == "auto" else f"forced: variants {args.tiles}")
    ctx.propagate(W)
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    torch.cuda.nvtx.range_push("split_timed")
    ctx.propagate(K)
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    steady = steady_windows(ctx, stream, Ks, local) if Ks > 0 else None
    # per-kernel device times from a separate pass with CUDA events around every
    # kernel (the event nodes in the graph would slow the timed region above)
    ctx.profile(True)
    ctx.propagate(Kp)
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.profile(False)
    J_split, E_split, q_split = ctx.observables(0)
    D0 = ctx.get_initial_density(0, 0)

    # plain FP64 path on the same ground state
    Kf = args.fp64_steps
    cf = vgtb.Context(sysd, precision=vgtb.FP64, init=vgtb.INIT_USER, cuda_stream=stream.cuda_stream,
                      graph_steps=1)
    cf.set_density(0, 0, D0)
    fp64_sparse = cf._opt.product1 != vgtb.P1_DENSE and all(d == 4 for d in np.diff(np.asarray(sysd["orb_offset"])))
    cf.set_field(0, A[:Kf + 3])
    cf.propagate(2)
    cf.profile(True)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    torch.cuda.nvtx.range_push("fp64_timed")
    cf.propagate(Kf)
    torch.cuda.nvtx.range_pop()
    f1.record(stream)
    torch.cuda.synchronize()
    ms_f = max_over_ranks(f0.elapsed_time(f1))
    stats_f = cf.kernel_stats()
    J_f, E_f, q_f = cf.observables(0)
    cf.close()
    p64 = fp64_peak_tflops(torch)

    # FP64 Crank-Nicolson integrator (Eq. 5) from the library's ground state
    cn = None
    Kc = args.cn_steps
    if Kc > 0:
        cc = vgtb.Context(sysd, precision=vgtb.FP64, init=vgtb.INIT_GROUND, integrator=vgtb.CRANK_NICOLSON,
                          cuda_stream=stream.cuda_stream, graph_steps=1)
        cc.set_field(0, A[:Kc + 3])
        cc.propagate(2)
        cc.profile(True)
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        torch.cuda.nvtx.range_push("cn_timed")
        cc.propagate(Kc)
        torch.cuda.nvtx.range_pop()
        c1.record(stream)
        torch.cuda.synchronize()
        ms_c = max_over_ranks(c0.elapsed_time(c1))
        st_c = cc.kernel_stats()
        sweeps = cc._opt.cn_iter
        cc.close()
        nocc = int(round(float(sysd["n_electrons"]) / 2))
        Nc = int(sysd["orb_offset"][-1])
        Npc = (Nc + 127) // 128 * 128
        f_sweep = 8.0 * nocc * Npc * Npc                 # one fixed-point sweep, complex FP64
        t_sweep = st_c["gemm2"][1] / max(st_c["gemm2"][0], 1) / sweeps
        a_sweep = f_sweep / (t_sweep * 1e-3) / 1e12
        cn = {"value": round(world * Kc / (ms_c / 1e3), 4), "unit": "steps/s", "steps": Kc,
              "ms_per_step": round(ms_c / Kc, 2), "sweeps_per_step": sweeps, "dtype": "f64",
              "kernel_ms_per_step": {k: round(v[1] / max(v[0], 1), 3) for k, v in st_c.items()},
              "roofline": {"bound": "fp64", "kernel": "k_gemm_f64 (fixed-point sweep C^dagger + i dt/2 Y^dagger M^dagger)",
                           "achieved": round(a_sweep, 3), "peak": round(p64, 3), "unit": "TFLOP/s",
                           "frac": round(a_sweep / p64, 4),
                           "peak_kind": "cuBLAS ZGEMM 2048^3 measured in this run (torch.matmul complex128)",
                           "flops_per_launch": f_sweep}}
    nj = min(len(J_f), len(J_split))
    j_err = float(np.linalg.norm(J_split[:nj] - J_f[:nj]) / np.linalg.norm(J_f[:nj]))
    q_err = float(np.abs(q_split[:nj] - q_f[:nj]).max())
    e_err = float(np.abs(E_split[:nj] - E_f[:nj]).max() / np.abs(E_f[:nj]).max())

    # end to end through the C-ABI: pinned host A table in, J/E/q series out
    e2e = None
    if not args.no_e2e:
        Ah = torch.from_numpy(np.ascontiguousarray(A[:K + 1])).pin_memory().numpy()
        nat = len(sysd["z_ref"])
        outJ = torch.empty((K + 1, 3), dtype=torch.float64).pin_memory().numpy()
        outE = torch.empty((K + 1,), dtype=torch.float64).pin_memory().numpy()
        outQ = torch.empty((K + 1, nat), dtype=torch.float64).pin_memory().numpy()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_field(0, Ah)
        ctx.propagate(K)
        ctx.observables_into(0, outJ, outE, outQ)
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        e2e = {"value": world * K / t_e2e, "unit": "steps/s",
               "h2d_bytes_per_step": int(Ah.nbytes / K),
               "d2h_bytes_per_step": int((outJ.nbytes + outE.nbytes + outQ.nbytes) / K)}
    ctx.close()

    N = int(sysd["orb_offset"][-1])
    Np = (N + 127) // 128 * 128
    peaks = measured_peaks()
    p1, p2 = split_product_rooflines([sysd], [1], stats, tiles, peaks)
    dominant = p1 if p2 is None or p1["avg_launch_ms"] >= p2["avg_launch_ms"] else p2
    roof = dict(dominant)
    if p2 is not None:
        roof["other_product"] = p2 if dominant is p1 else p1
    # FP64 path: product 1 block-sparse (8 nnz(H) N) or dense (8 N^3), product 2 dense (8 N^3)
    nnz = nonzeros(sysd)
    f64_1 = stats_f["gemm1"][1] / max(stats_f["gemm1"][0], 1)
    f64_2 = stats_f["gemm2"][1] / max(stats_f["gemm2"][0], 1)
    fl64_1 = 8.0 * nnz * N if fp64_sparse else 8.0 * N ** 3
    fl64_2 = 8.0 * N ** 3
    a64_1 = fl64_1 / (f64_1 * 1e-3) / 1e12
    a64_2 = fl64_2 / (f64_2 * 1e-3) / 1e12
    step_ms = ms / K
    value = world * K / (ms / 1e3)
    kern_ms = {k: (v[1] / max(v[0], 1)) for k, v in stats.items()}
    bat = run_batched(args, args.batched_steps, 3, timing_start=True) if args.batched_steps > 0 else None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = with_1thread(cpu_baseline(args.cpu_steps), args.cpu_1thread_steps)
    if rank != 0:
        return
    clocks_source = "sampled during the timed region"
    if not clocks.get("samples") and steady and steady["clocks"].get("samples"):
        # a short timed region can end before nvidia-smi's first 200 ms sample: take the
        # record of the steady windows that follow it directly in the same process
        clocks = dict(steady["clocks"])
        clocks_source = (f"timed region ({ms:.1f} ms) shorter than the 200 ms sampling interval: sampled during "
                         f"the {steady['windows']} steady windows of {steady['steps_per_window']} steps that follow it")
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3 (f32 accumulate) + f64 master", "data": "synthetic",
        "config": {"workload": WORKLOAD, "name": CONFIG, "precision": "split_bf16x3 delta form",
                   "product1": args.product1, "tiles": tiles,
                   "parallelism": f"{world} independent replica(s)",
                   "l2": "working set ~0.6 GB per step, larger than the 129 MB L2 (no flush)",
                   "fs_per_hour": round(value / world * 0.2 * AU_FS * 3600, 2)},
        "fp64": {"value": round(world * Kf / (ms_f / 1e3), 3), "unit": "steps/s", "steps": Kf,
                 "ms_per_step": round(ms_f / Kf, 3),
                 "fs_per_hour": round(Kf / (ms_f / 1e3) * 0.2 * AU_FS * 3600, 3),
                 "kernel_ms_per_step": {k: round(v[1] / max(v[0], 1), 3) for k, v in stats_f.items()},
                 "roofline": {"bound": "fp64", "kernel": "k_gemm_f64 (product 2: X = S^-1 W^dagger, dense)",
                              "achieved": round(a64_2, 3), "peak": round(p64, 3), "unit": "TFLOP/s",
                              "frac": round(a64_2 / p64, 4), "flops_per_launch": fl64_2,
                              "peak_kind": "cuBLAS ZGEMM 2048^3 measured in this run (torch.matmul complex128)"},
                 "product1": {"kernel": ("k_bsr<double,4> (W = D H over the nonzero atom blocks)" if fp64_sparse
                                         else "k_gemm_f64 (W = D H, dense)"),
                              "achieved": round(a64_1, 3), "peak": round(p64, 3), "unit": "TFLOP/s",
                              "frac": round(a64_1 / p64, 4), "flops_per_launch": fl64_1,
                              "avg_launch_ms": round(f64_1, 3)}},
        "crank_nicolson": cn,
        "j_rel_err_split_vs_fp64": j_err, "j_err_steps": nj - 1,
        "split_vs_fp64": {"J_rel_fro": j_err, "q_max_abs": q_err, "E_max_rel": e_err, "levels": nj,
                          "note": "same ground state and field; the 5000-step run against the stored oracle "
                                  "is tests/test_gpu_long.py"},
        "hbm": hbm_rates(sysd, Np, kern_ms, peaks.get("hbm_gbs"), tiles["product1"].get("schedule") == "block-sparse"),
        "roofline": roof,
        "kernel_ms_per_step": {k: round(v, 4) for k, v in kern_ms.items()},
        "kernel_ms_note": f"CUDA events around each kernel in a separate pass of {Kp} steps after the timed region",
        "steady": steady,
        "batched": bat,
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches_per_step(tiles) * K + 2,
        "clocks": clocks, "clocks_source": clocks_source,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# batched form: every trajectory and k-point of three supercells in one context
# ---------------------------------------------------------------------------
BATCH_WORKLOAD = ("batched: Si supercells of 64 / 216 / 512 atoms (N = 256 / 864 / 2048), MP 2x2x2 k-grid, "
                  "fields x,y,z x w in {0.05, 0.1} Ha, sin^2 pulse E0 = 0.01 au over 3000 steps: 18 trajectories, "
                  "144 k-propagations per step")


LASER_WORKLOAD = ("laser sweep: 512-atom Si supercell (sigma=0.3 bohr), Gamma, 20 fs sin^2 pulses along x at "
                  "2.3 / 3.9 / 6.0 eV, E0 = 0.00534 au (10^12 W/cm^2), 3 trajectories in one context, full pulse; "
                  "Mulliken charge transfer between 3- and 4-coordinated atoms (2.85 A bond cut-off)")


def laser(args):
    """The laser experiment of Sec. 3.3 on the synthetic 512-atom cell: one context, three
    trajectories (one per photon energy), the whole 20 fs pulse, then dQ(t) per
    coordination class averaged over 2 fs windows (vgtb_group_charges on the device)."""
    import torch
    from paper_2308_09782_gb300 import inputs, vgtb
    rank, world, local = dist_setup(True)
    vgtb.load()
    sysd, _, _ = inputs.config(CONFIG)
    fields, n = inputs.laser_sweep(sysd["dt"])
    K = n if args.laser_steps <= 0 else min(args.laser_steps, n)
    cn = inputs.coordination_numbers(sysd)
    classes = sorted(set(cn.tolist()))
    group = np.array([classes.index(c) for c in cn], np.int32)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    ctx = vgtb.Context([sysd], traj_sys=[0, 0, 0], precision=vgtb.SPLIT_BF16X3, init=vgtb.INIT_GROUND,
                       cuda_stream=stream.cuda_stream, graph_steps=50, autotune=1)
    t_setup = time.perf_counter() - t0
    tiles = {f"product{p}": ctx.tile_config(p) for p in (1, 2)}
    Kp = 200                                   # profiled pass after the pulse (A constant there)
    for tr, f in enumerate(fields):
        ctx.set_field(tr, np.vstack([f[:K + 1], np.tile(f[K:K + 1], (Kp, 1))]))
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.propagate(K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    win = int(round(2.0 / inputs.AU_TIME_FS / sysd["dt"]))    # 2 fs of steps
    dq = {}
    for tr, ev in enumerate((2.3, 3.9, 6.0)):
        g = ctx.group_charges(tr, group, len(classes))[:K + 1]  # [K+1, n_classes]
        nw = (K + 1) // win
        avg = g[:nw * win].reshape(nw, win, len(classes)).mean(axis=1)
        dq[f"{ev} eV"] = {f"{classes[c]}-coordinated": [round(float(x), 8) for x in avg[:, c]]
                          for c in range(len(classes))}
    ctx.profile(True)
    ctx.propagate(Kp)
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.close()
    if rank != 0:
        return
    steps_s = world * K / (ms / 1e3)
    line = {"metric": "laser sweep steps/s (3 trajectories per step)", "value": round(steps_s, 3), "unit": "steps/s",
            "n_gpus": world, "steps": K, "warmup": 0, "ms_per_step": round(ms / K, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 (f32 accumulate) + f64 master",
            "data": "synthetic",
            "config": {"workload": LASER_WORKLOAD, "setup_s": round(t_setup, 1),
                       "atoms_per_class": {f"{c}-coordinated": int(np.sum(cn == c)) for c in classes},
                       "simulated_fs": round(K * sysd["dt"] * inputs.AU_TIME_FS, 2)},
            "trajectory_steps_per_s": round(3 * steps_s, 1),
            "dQ_2fs_averages": dq,
            "kernel_ms_per_step": {k: round(v[1] / max(v[0], 1), 4) for k, v in stats.items()},
            "gpu_launches": launches_per_step(tiles) * K + 2, "clocks": clocks}
    print(json.dumps(line), flush=True)


BATCH_FIELD_STEPS = 3000


def batched_inputs():
    systems = [inputs_mod().diamond_si(2, 0.05, seed=64, kgrid="mp2"),
               inputs_mod().diamond_si(3, 0.2, seed=216, kgrid="mp2"),
               inputs_mod().diamond_si(4, 0.3, seed=512, kgrid="mp2")]
    traj_sys, fields = [], []
    for s in range(3):
        for pol in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            for w in (0.05, 0.1):
                traj_sys.append(s)
                fields.append(inputs_mod().pulse_field(BATCH_FIELD_STEPS, 0.2, 0.01, w, pol=pol))
    return systems, traj_sys, fields


def inputs_mod():
    from paper_2308_09782_gb300 import inputs
    return inputs


def run_batched(args, K, W, timing_start=False):
    """The batched form (config 5): 64/216/512-atom supercells x 8 k-points x 6 fields in
    one context, one graph-captured sequence of batched launches per step.  With
    timing_start the trajectories start from D0 = (N_el/N) I (Hermitian, Tr(D0 S) =
    N_el since S has a unit diagonal) instead of the SCC ground states, which saves the
    ground-state set-up: a step does the same work for any density.  Returns the
    result dict (rank 0) or None."""
    import torch
    from paper_2308_09782_gb300 import vgtb
    rank, world, local = dist_setup(True)
    vgtb.load()
    systems, traj_sys, fields = batched_inputs()
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tile_opts = {"autotune": 1}
    if args.tiles != "auto":
        tile_opts = {"autotune": 0, "tile_variant": [int(x) for x in args.tiles.split(",")]}
    ctx = vgtb.Context(systems, traj_sys=traj_sys, precision=vgtb.SPLIT_BF16X3,
                       init=vgtb.INIT_USER if timing_start else vgtb.INIT_GROUND,
                       cuda_stream=stream.cuda_stream, graph_steps=20, obs_stride=10, product1=P1[args.product1],
                       chain=CHAIN[args.chain],
                       **tile_opts)
    if timing_start:
        for si, sd in enumerate(systems):
            n = int(sd["orb_offset"][-1])
            d0 = (float(sd["n_electrons"]) / n) * np.eye(n, dtype=np.complex128)
            for k in range(len(sd["wk"])):
                ctx.set_density(si, k, d0)
    t_setup = time.perf_counter() - t0
    tiles = {f"product{p}": ctx.tile_config(p) for p in (1, 2)}
    tiles["choice"] = "autotuned at create" if args.tiles == "auto" else f"forced: variants {args.tiles}"
    Kp = min(K, 200)
    n_need = W + K + Kp + 1
    for t, f in enumerate(fields):
        ctx.set_field(t, f if len(f) >= n_need else np.vstack([f, np.tile(f[-1:], (n_need - len(f), 1))]))
    ctx.propagate(W)
    clk = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    torch.cuda.nvtx.range_push("batched_timed")
    ctx.propagate(K)
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(e0.elapsed_time(e1))
    ctx.profile(True)                          # per-kernel times: a separate pass with events
    ctx.propagate(Kp)
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.close()
    n_items = [sum(1 for t in traj_sys if t == s) * len(systems[s]["wk"]) for s in range(len(systems))]
    p1, p2 = split_product_rooflines(systems, n_items, stats, tiles, measured_peaks())
    steps_s = world * K / (ms / 1e3)
    if rank != 0:
        return None
    return {"value": round(steps_s, 3), "unit": "steps/s", "steps": K, "warmup": W, "ms_per_step": round(ms / K, 4),
            "timed_window": f"steps {W}..{W + K} of the {BATCH_FIELD_STEPS}-step pulses",
            "start": ("D0 = (N_el/N) I (timing start; a step does the same work for any density)" if timing_start
                      else "SCC ground state of each system"),
            "setup_s": round(t_setup, 1), "tiles": tiles,
            "trajectory_steps_per_s": round(len(traj_sys) * steps_s, 1),
            "k_propagation_steps_per_s": round(sum(n_items) * steps_s, 1),
            "product1": p1, "product2": p2,
            "kernel_ms_per_step": {k: round(v[1] / max(v[0], 1), 4) for k, v in stats.items()},
            "gpu_launches": launches_per_step(tiles) * K + 2, "clocks": clocks}


def batched(args):
    K, W = args.steps, max(args.warmup, 3)
    r = run_batched(args, K, W)
    if r is None:
        return
    p1, p2 = r["product1"], r["product2"]
    dominant = p1 if p2 is None or p1["avg_launch_ms"] >= p2["avg_launch_ms"] else p2
    line = {"metric": "batched steps/s (18 trajectories x 8 k per step)", "value": r["value"],
            "unit": "steps/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": K, "warmup": W,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3 (f32 accumulate) + f64 master", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "setup_s": r["setup_s"], "tiles": r["tiles"],
                       "timed_window": r["timed_window"], "start": r["start"]},
            "trajectory_steps_per_s": r["trajectory_steps_per_s"],
            "k_propagation_steps_per_s": r["k_propagation_steps_per_s"],
            "roofline": dominant, "product1": r["product1"], "product2": r["product2"],
            "kernel_ms_per_step": r["kernel_ms_per_step"], "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle on the host cores
# ---------------------------------------------------------------------------
def reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, min(args.steps, 40))
    cpu = with_1thread(cpu_baseline(steps), args.cpu_1thread_steps)
    v = cpu["value"]
    line = {"metric": METRIC, "value": round(v, 5), "unit": "steps/s", "n_gpus": 0, "steps": steps,
            "warmup": 1, "ms_per_step": round(1e3 / v, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "name": CONFIG},
            "cpu_baseline": cpu,
            "e2e": {"value": round(v, 5), "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.oracle_probe > 0:
        print(json.dumps(cpu_baseline(a.oracle_probe, warm_up=False)), flush=True)
    elif a.impl == "reference":
        reference(a)
    elif a.workload == "batched":
        batched(a)
    elif a.workload == "laser":
        laser(a)
    else:
        native(a)
