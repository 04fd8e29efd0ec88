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


def hbm_rates(sysd, Np, kern_ms, peak_gbs):
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
        "leap": 56 * Np * Np,                                        # X, R0 f32; dD r/w f64; pieces
        "phase": nk * (20 * el_img + 8 * len(blk) + 32 * n_el),      # S, H0, dS f32 per image; 16 bf16 out
        "obs": nk * 64 * n_el + 40 * nat,                            # dD f64 + packed f32 blocks
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
    n_need = W + K + Kp + 1
    if A.shape[0] < n_need:                      # the kick is constant after t = 0
        A = np.tile(A[:1], (n_need, 1))
    stream = torch.cuda.current_stream()
    tile_opts = {"autotune": 1}
    if args.tiles != "auto":
        tile_opts = {"autotune": 0, "tile_variant": [int(x) for x in args.tiles.split(",")]}
    ctx = vgtb.Context(sysd, precision=vgtb.SPLIT_BF16X3, init=vgtb.INIT_GROUND,
                       cuda_stream=stream.cuda_stream, graph_steps=50, **tile_opts)
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
    flops1 = 3 * 2 * Np * (2 * Np) * (4 * Np)      # executed BF16 flops, product 1 (K' = 2 x 2Np)
    flops2 = 3 * 2 * Np * (2 * Np) * (2 * Np)      # product 2
    g1_n, g1_ms = stats["gemm1"]
    g2_n, g2_ms = stats["gemm2"]
    peaks = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained")
    peak_kind = "measured sustained bf16 (MEASURED_PEAKS.json)"
    if peak is None:
        peak, peak_kind = 1700.0, "fallback sustained bf16"
    avg1 = g1_ms / max(g1_n, 1)
    ach1 = flops1 / (avg1 * 1e-3) / 1e12
    ach2 = flops2 / (g2_ms / max(g2_n, 1) * 1e-3) / 1e12
    step_ms = ms / K
    value = world * K / (ms / 1e3)
    kern_ms = {k: (v[1] / max(v[0], 1)) for k, v in stats.items()}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = with_1thread(cpu_baseline(args.cpu_steps), args.cpu_1thread_steps)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "steps/s", "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3 (f32 accumulate) + f64 master", "data": "synthetic",
        "config": {"workload": WORKLOAD, "name": CONFIG, "precision": "split_bf16x3 delta form",
                   "tiles": tiles,
                   "parallelism": f"{world} independent replica(s)",
                   "l2": "working set ~0.6 GB per step, larger than the 129 MB L2 (no flush)",
                   "fs_per_hour": round(value / world * 0.2 * AU_FS * 3600, 2)},
        "fp64": {"value": round(world * Kf / (ms_f / 1e3), 3), "unit": "steps/s", "steps": Kf,
                 "ms_per_step": round(ms_f / Kf, 3),
                 "fs_per_hour": round(Kf / (ms_f / 1e3) * 0.2 * AU_FS * 3600, 3),
                 "kernel_ms_per_step": {k: round(v[1] / max(v[0], 1), 3) for k, v in stats_f.items()},
                 "roofline": {"bound": "fp64", "kernel": "k_gemm_f64 (product 1: W = D H)",
                              "achieved": round(8.0 * Np ** 3 / (stats_f["gemm1"][1] / max(stats_f["gemm1"][0], 1)
                                                                  * 1e-3) / 1e12, 3),
                              "peak": round(p64, 3), "unit": "TFLOP/s",
                              "frac": round(8.0 * Np ** 3 / (stats_f["gemm1"][1] / max(stats_f["gemm1"][0], 1)
                                                             * 1e-3) / 1e12 / p64, 4),
                              "peak_kind": "cuBLAS ZGEMM 2048^3 measured in this run (torch.matmul complex128)"}},
        "crank_nicolson": cn,
        "j_rel_err_split_vs_fp64": j_err, "j_err_steps": nj - 1,
        "split_vs_fp64": {"J_rel_fro": j_err, "q_max_abs": q_err, "E_max_rel": e_err, "levels": nj,
                          "note": "same ground state and field; the 5000-step run against the stored oracle "
                                  "is tests/test_gpu_long.py"},
        "hbm": hbm_rates(sysd, Np, kern_ms, peaks.get("hbm_gbs")),
        "roofline": {"bound": "tensor", "kernel": "k_tc_gemm (product 1: W = [dD|D0][H|dH]^dagger)",
                     "achieved": round(ach1, 1), "peak": peak, "unit": "TFLOP/s",
                     "frac": round(ach1 / peak, 4), "peak_kind": peak_kind,
                     "frac_of_burst": round(ach1 / peaks.get("bf16_tflops", 1900.0), 4),
                     "traffic": kernel_traffic("tc_gemm1", 1.0, tiles["product1"]),
                     "flops_per_launch": flops1, "avg_launch_ms": round(avg1, 4),
                     "product2_achieved": round(ach2, 1), "product2_frac": round(ach2 / peak, 4)},
        "kernel_ms_per_step": {k: round(v, 4) for k, v in kern_ms.items()},
        "kernel_ms_note": f"CUDA events around each kernel in a separate pass of {Kp} steps after the timed region",
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": 6 * K + 2,
        "clocks": clocks,
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
            "gpu_launches": 6 * K + 2, "clocks": clocks}
    print(json.dumps(line), flush=True)


def batched(args):
    import torch
    from paper_2308_09782_gb300 import inputs, vgtb
    rank, world, local = dist_setup(True)
    vgtb.load()
    systems = [inputs.diamond_si(2, 0.05, seed=64, kgrid="mp2"),
               inputs.diamond_si(3, 0.2, seed=216, kgrid="mp2"),
               inputs.diamond_si(4, 0.3, seed=512, kgrid="mp2")]
    K, W = args.steps, max(args.warmup, 3)
    nsteps = 3000
    traj_sys, fields = [], []
    for s in range(3):
        for pol in ((1, 0, 0), (0, 1, 0), (0, 0, 1)):
            for w in (0.05, 0.1):
                traj_sys.append(s)
                fields.append(inputs.pulse_field(nsteps, 0.2, 0.01, w, pol=pol))
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    tile_opts = {"autotune": 1}
    if args.tiles != "auto":
        tile_opts = {"autotune": 0, "tile_variant": [int(x) for x in args.tiles.split(",")]}
    ctx = vgtb.Context(systems, traj_sys=traj_sys, precision=vgtb.SPLIT_BF16X3, init=vgtb.INIT_GROUND,
                       cuda_stream=stream.cuda_stream, graph_steps=20, obs_stride=10, **tile_opts)
    t_setup = time.perf_counter() - t0
    tiles = {f"product{p}": ctx.tile_config(p) for p in (1, 2)}
    tiles["choice"] = "autotuned at create" if args.tiles == "auto" else f"forced: variants {args.tiles}"
    for t, f in enumerate(fields):
        ctx.set_field(t, f)
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
    ctx.profile(True)                          # per-kernel times: a separate pass with events
    ctx.propagate(min(K, 200))
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.close()
    nps = [(int(s["orb_offset"][-1]) + 127) // 128 * 128 for s in systems]
    items = [(np_, 8 * 6) for np_ in nps]
    flops1 = sum(n_it * 48 * np_ ** 3 for np_, n_it in items)
    flops2 = sum(n_it * 24 * np_ ** 3 for np_, n_it in items)
    g1 = stats["gemm1"][1] / max(stats["gemm1"][0], 1)
    g2 = stats["gemm2"][1] / max(stats["gemm2"][0], 1)
    peak = measured_peaks().get("bf16_tflops_sustained", 1700.0)
    burst = measured_peaks().get("bf16_tflops", 1900.0)
    steps_s = world * K / (ms / 1e3)
    if rank != 0:
        return
    line = {"metric": "batched steps/s (18 trajectories x 8 k per step)", "value": round(steps_s, 3),
            "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": round(ms / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16x3 (f32 accumulate) + f64 master", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "setup_s": round(t_setup, 1), "tiles": tiles},
            "trajectory_steps_per_s": round(18 * steps_s, 1), "k_propagation_steps_per_s": round(144 * steps_s, 1),
            "roofline": {"bound": "tensor", "achieved": round(flops1 / (g1 * 1e-3) / 1e12, 1), "peak": peak,
                         "unit": "TFLOP/s", "frac": round(flops1 / (g1 * 1e-3) / 1e12 / peak, 4),
                         "peak_kind": "measured sustained bf16 (MEASURED_PEAKS.json; its clocks under load "
                                      "had a 1470 MHz median, this run's are in clocks)",
                         "frac_of_burst": round(flops1 / (g1 * 1e-3) / 1e12 / burst, 4),
                         "product2_frac": round(flops2 / (g2 * 1e-3) / 1e12 / peak, 4)},
            "kernel_ms_per_step": {k: round(v[1] / max(v[0], 1), 4) for k, v in stats.items()},
            "gpu_launches": 6 * K + 2, "clocks": clocks}
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
