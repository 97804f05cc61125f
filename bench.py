#!/usr/bin/env python
"""Two-qubit gates/s at chi = 256 on one GB300 (contract + SVD + truncate + absorb).

Workload: a 100-qubit Haar SU(4) brickwork, chi_max = 256, complex64 (FP32
arithmetic), batched schedule.  The state is first evolved (untimed) until the
interior bonds saturate at chi = 256; then W warm-up layers, then K timed layers.
A step is one brickwork layer (49 or 50 gates).  The inputs (gates) sit in HBM
before the timed region starts; the state (88 MB) and per-layer workspace
(2 x 2 MiB per gate) together exceed the 126 MB L2.

Also reported on the same line: the end-to-end rate through the synchronous C-ABI
call with host gate buffers (e2e), the Jacobi kernel's fraction of the FP32 ALU
roofline (per-kernel CUDA events recorded on the library's stream during the
timed region), the plain per-pair complex128 GPU path on sampled gates of the same
state, and the FP64 oracle timed on the host cores (cpu_baseline).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun, one rank per GPU) every rank runs its own replica circuit
(seed 1000 + rank): replicas only, weak scaling, no data-path collective.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2-qubit gates/s at χ=256 (contract+SVD+truncate), % roofline, vs plain path"
UNIT = "2q gates/s"
N_QUBITS, CHI, PRESAT = 100, 256, 10
JACOBI_SRC = os.path.join(ROOT, "paper_2601_04422_gb300", "csrc", "k_jacobi.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_jacobi_chi256.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-gates", type=int, default=4, help="gates timed on the plain c128 path")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="budget of the oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shots", type=int, default=1024, help="perfect-sampling shots on the saturated state")
    ap.add_argument("--grad-reps", type=int, default=3, help="timed energy-gradient evaluations (50-qubit HEA)")
    ap.add_argument("--nonlocal-ops", type=int, default=60,
                    help="gates at distance <= 6 applied to the saturated state by the SWAP method")
    ap.add_argument("--gemm", default="tf32x3", choices=["fp32", "fp32_3m", "tf32x3", "bf16x3"],
                    help="arithmetic of the merge + gate contraction")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(rank: int) -> int:
    """Every rank simulates its own replica circuit."""
    return 1000 + int(rank)


def replica_reduce(elapsed, units, dist=None, device="cpu"):
    """Whole-job figures over the replicas: the slowest rank's elapsed time (MAX) and
    the units all ranks processed (SUM).  dist: torch.distributed or None (one rank);
    device: where the reduction tensors live (the rank's GPU under NCCL, the CPU under
    gloo)."""
    if dist is None:
        return elapsed, units
    import torch
    t = torch.tensor([float(elapsed)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def peaks():
    p = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
         "src": "fallback"}
    f = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(f):
        d = json.load(open(f))
        p.update({k: d[k] for k in ("hbm_gbs", "sm_max_mhz", "bf16_tflops", "bf16_tflops_sustained") if k in d})
        p["src"] = "measured"
    return p


def fp32_alu_peak_tflops(sm_mhz: float) -> float:
    """152 SMs x 128 FP32 lanes x 2 flops per FMA x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def jacobi_traffic():
    """DRAM bytes per Jacobi launch from the committed ncu summary, if it was taken on the
    current kernel source (matched by its sha256), else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    txt = open(TRAFFIC_FILE).read()
    m1 = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m2 = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    if not (m1 and m2):
        return None
    sha = hashlib.sha256(open(JACOBI_SRC, "rb").read()).hexdigest()
    return float(m1.group(1)) if sha == m2.group(1) else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_gate_rate(seconds: float, seed: int = 5):
    """FP64 oracle: chi = 256 two-qubit updates on random sites, for about `seconds`."""
    import workloads as W
    from oracle import mps as om
    a, b = W.random_sites(CHI, CHI, CHI, seed)
    rng = np.random.default_rng(seed)
    gates, t0 = 0, time.perf_counter()
    while True:
        m = om.MPS([a.copy(), b.copy()])
        om.apply_2q(m, 0, W.haar_su4(rng), CHI)
        gates += 1
        dt = time.perf_counter() - t0
        if dt >= seconds:
            break
    return gates / dt, gates, dt


def host_cores():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            try:
                return int(os.environ[k])
            except ValueError:
                pass
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args, world, rank):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_gate_rate(0.0)
    per_step = max(1.0, min(10.0, 120.0 / max(args.steps, 1)))
    rates, gates, secs = [], 0, 0.0
    for _ in range(args.steps):
        r, g, s = oracle_gate_rate(per_step)
        rates.append(r)
        gates += g
        secs += s
    value = gates / secs
    sample = (f"{gates} two-qubit updates at chi_L = chi_M = chi_R = 256 on random complex "
              f"Gaussian sites (512x512 complex128 SVD each), {args.steps} steps of ~{per_step:.0f} s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config():
    return {"workload": "Haar SU(4) brickwork, 100 qubits, chi_max 256, saturated bonds, "
                        "complex64, batched layer (49-50 gates per step)",
            "n_qubits": N_QUBITS, "chi_max": CHI, "state_dtype": "complex64",
            "l2": "inputs larger than L2: state 88 MB + theta/W workspace 196 MB per layer"}


def run_ours(args, world, rank, local):
    import torch
    import __graft_entry__ as g
    g.build()
    import paper_2601_04422_gb300 as T
    import workloads as W

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    depth = PRESAT + args.warmup + 2 * args.steps + 2
    circ = W.brickwork_su4(N_QUBITS, depth, seed=replica_seed(rank))
    stream = torch.cuda.Stream(device=dev)
    gemm = getattr(T, "TNSIM_GEMM_" + args.gemm.upper())
    m = T.MPS(N_QUBITS, dtype=T.TNSIM_C64, chi_max=CHI, gemm=gemm, stream=stream.cuda_stream)
    gdev = [torch.from_numpy(np.ascontiguousarray(l.g4).view(np.float64).copy()).to(dev)
            for l in circ.layers]
    eps_dev = torch.zeros(N_QUBITS, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    def layer_dev(i):
        T.tnsim_apply_layer_device(m.h, circ.layers[i].pairs, gdev[i].data_ptr(), 0, eps_dev.data_ptr())

    for i in range(PRESAT):
        layer_dev(i)
    m.sync()
    for i in range(PRESAT, PRESAT + args.warmup):
        layer_dev(i)
    m.sync()
    dims = m.bond_dims()
    # autotuner: time the Jacobi launch configurations on the first timed layer's gates
    tune_choice, tune_ms = T.tnsim_autotune(m.h, circ.layers[PRESAT + args.warmup].pairs,
                                            circ.layers[PRESAT + args.warmup].g4, reps=2)
    T.tnsim_last_stats(m.h)
    T.tnsim_profile_read(m.h)

    # ---- timed region: device-resident inputs
    t_lo = PRESAT + args.warmup
    timed = list(range(t_lo, t_lo + args.steps))
    gates_rank = sum(circ.layers[i].n2 for i in timed)
    clk = ClockSampler(local)
    clk.start()
    T.tnsim_profile_enable(m.h, True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in timed:
        layer_dev(i)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    m.sync()
    prof = T.tnsim_profile_read(m.h)
    T.tnsim_profile_enable(m.h, False)
    stats = T.tnsim_last_stats(m.h)

    # ---- end to end: the synchronous C-ABI call on host buffers (copies inside)
    e2e = None
    if not args.no_e2e:
        host_layers = circ.layers[t_lo + args.steps: t_lo + 2 * args.steps]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        g_e2e = 0
        for l in host_layers:
            T.tnsim_apply_layer(m.h, l.pairs, l.g4, None)
            g_e2e += l.n2
        t_e2e = time.perf_counter() - t0
        if dist:
            dist.barrier()
        e2e = (g_e2e, t_e2e, host_layers)
    clocks = clk.stop()

    # ---- aggregate over ranks
    ms_max, gates_all = replica_reduce(ms, gates_rank, dist, dev)
    value = gates_all / (ms_max / 1000.0)
    e2e_obj = None
    if e2e is not None:
        g_e2e, t_e2e, host_layers = e2e
        t_max, g_all = replica_reduce(t_e2e, g_e2e, dist, dev)
        h2d = sum(l.n2 * 32 * 8 for l in host_layers) / len(host_layers)
        d2h = sum(l.n2 * 8 for l in host_layers) / len(host_layers)
        e2e_obj = {"value": g_all / t_max, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h),
                   "note": "tnsim_apply_layer on host gate arrays: gate upload, all kernels, "
                           "discarded-weight and bond-dimension read-back per step"}

    # ---- roofline of the dominant kernel (the Jacobi SVD), FP32 ALU bound
    pk = peaks()
    jac_ms, jac_n = prof["jacobi"]
    # per examined pair-row: g = x_i^H x_j (4 FMA); per rotated pair-row: both columns updated (20 flops);
    # the column norms are tracked, not recomputed per pair
    flops = 8.0 * stats["visit_rows"] + 20.0 * stats["rotation_rows"]
    achieved = flops / (jac_ms / 1000.0) / 1e12 if jac_ms > 0 else 0.0
    sm_mhz = pk["sm_max_mhz"]
    peak = fp32_alu_peak_tflops(sm_mhz)
    traffic = jacobi_traffic()
    roofline = {"bound": "alu", "kernel": "k_jacobi", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak if peak else None,
                "traffic": (traffic if traffic is not None else None),
                "peak_src": f"derived: 152 SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz ({pk['src']} max clock)",
                "algorithmic_flops_per_launch": flops / max(jac_n, 1),
                "avg_launch_ms": jac_ms / max(jac_n, 1)}
    # ---- whole-gate roofline time T* (contraction on the tensor pipe at the TF32 rate;
    # QR preconditioning, Jacobi and site product on the FP32 ALUs; site reads and writes
    # at HBM rate)
    ng = max(stats["gates"], 1)
    tf32_peak = pk["bf16_tflops_sustained"] * (1.1 / 2.25)          # nominal TF32 : BF16 dense ratio
    t_contract = 8.0 * stats["theta_cmacs"] / ng / (tf32_peak * 1e12)
    t_svd = flops / ng / (peak * 1e12)
    t_right = 8.0 * stats["right_cmacs"] / ng / (peak * 1e12)
    t_qr = 8.0 * stats["qr_cmacs"] / ng / (peak * 1e12)
    site_bytes = 4.0 * 2 * CHI * CHI * 8                             # read A, B; write A', B' (complex64)
    t_mem = site_bytes / (pk["hbm_gbs"] * 1e9)
    t_star = t_contract + t_qr + t_svd + t_right + t_mem
    path_roofline = {"t_star_us_per_gate": t_star * 1e6, "gates_per_s_at_roofline": 1.0 / t_star,
                     "frac": value / (1.0 / t_star),
                     "parts_us": {"contraction_tf32": t_contract * 1e6, "qr_fp32": t_qr * 1e6,
                                  "jacobi_fp32": t_svd * 1e6, "site_product_fp32": t_right * 1e6,
                                  "site_bytes_hbm": t_mem * 1e6},
                     "peaks": f"TF32 {tf32_peak:.0f} TFLOP/s (measured sustained BF16 x 1.1/2.25), FP32 ALU "
                              f"{peak:.1f} TFLOP/s, HBM {pk['hbm_gbs']:.0f} GB/s"}
    total_k_ms = sum(v[0] for v in prof.values())
    kernels = {k: {"ms": v[0], "launches": v[1], "share": (v[0] / total_k_ms if total_k_ms else 0.0)}
               for k, v in prof.items() if v[1]}
    launches = sum(v[1] for v in prof.values())

    # ---- plain per-pair complex128 path on sampled gates of the same saturated state
    plain = None
    if args.plain_gates > 0 and rank == 0:
        sites = m.export_sites()
        mp = T.MPS(N_QUBITS, dtype=T.TNSIM_C128, chi_max=CHI, schedule=T.TNSIM_SCHED_PLAIN,
                   stream=stream.cuda_stream)
        mp.import_sites(sites)
        lay = circ.layers[t_lo + 2 * args.steps]
        mid = len(lay.pairs) // 2
        sel = list(range(mid - args.plain_gates // 2, mid - args.plain_gates // 2 + args.plain_gates))
        q = lay.pairs[sel]
        gg = lay.g4[sel]
        chis = [int(dims[int(x)]) for x in q] + [int(dims[int(x) + 2]) for x in q]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        T.tnsim_apply_layer(mp.h, q, gg, None)
        tp = time.perf_counter() - t0
        st_p = T.tnsim_last_stats(mp.h)
        plain = {"value": len(sel) / tp, "unit": UNIT, "dtype": "f64", "schedule": "one pair per launch",
                 "sample": f"{len(sel)} gates of one layer at chi_L, chi_R in {sorted(set(chis))}",
                 "jacobi_sweeps_per_gate": st_p["sweeps"] / max(st_p["gates"], 1)}
        mp.close()

    # ---- non-local gates (SWAP method, tnsim_apply_circuit) on the same saturated state
    nonlocal_obj = None
    if args.nonlocal_ops > 0 and rank == 0:
        mn = T.MPS(N_QUBITS, dtype=T.TNSIM_C64, chi_max=CHI, gemm=gemm, stream=stream.cuda_stream)
        mn.import_sites(m.export_sites())
        ops = W.nonlocal_ops(N_QUBITS, args.nonlocal_ops, seed=7, p1=0.0, max_dist=6)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n_layers, n_local, _ = mn.apply_circuit(ops)
        tn = time.perf_counter() - t0
        nonlocal_obj = {"value": n_local / tn, "unit": "local 2q updates/s (SWAPs included)",
                        "ops_per_s": len(ops) / tn, "ops": len(ops), "local_updates": n_local,
                        "layers": n_layers, "seconds": tn,
                        "sample": f"{len(ops)} Haar U(4) gates at distance 1-6 in either qubit order on the "
                                  f"saturated chi {CHI} state, one synchronous tnsim_apply_circuit call "
                                  "(gate upload and read-back included)"}
        mn.close()

    # ---- perfect sampling (tnsim_sample) of the same saturated state
    sampling_obj = None
    if args.shots > 0 and rank == 0:
        u = np.random.default_rng(17).random((args.shots, N_QUBITS))
        T.tnsim_sample(m.h, u[:8])          # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, nodes = T.tnsim_sample(m.h, u)
        ts = time.perf_counter() - t0
        sampling_obj = {"value": args.shots / ts, "unit": "shots/s", "shots": args.shots, "seconds": ts,
                        "prefixes_evaluated": nodes, "prefixes_without_memoisation": args.shots * N_QUBITS,
                        "sample": f"{args.shots} bitstrings of the saturated {N_QUBITS}-qubit chi {CHI} state, "
                                  "one synchronous tnsim_sample call (right environments, uniforms upload "
                                  "and bit read-back included)"}

    # ---- reverse-mode energy gradient (tnsim_grad) of the 50-qubit, 10-layer HEA at chi 64
    grad_obj = None
    if args.grad_reps > 0 and rank == 0:
        nq = 50
        hcirc, hang = W.hea_circuit(nq, 10, seed=1, sigma=0.3)
        hl = [(l.pairs, l.g4) for l in hcirc.layers]
        hax = ["YZ" if i % 2 == 0 else "" for i in range(len(hl))]
        hth = [hang[i // 2] if i % 2 == 0 else np.zeros((nq, 0)) for i in range(len(hl))]
        hp = ["".join("Z" if k in (i, i + 1) else "I" for k in range(nq)) for i in range(nq - 1)] + \
             ["".join("X" if k == i else "I" for k in range(nq)) for i in range(nq)]
        hc = [1.0] * (nq - 1) + [0.5] * nq
        gp = T.tnsim_params_default(T.TNSIM_C64)
        gp.chi_max = 64
        T.tnsim_grad(nq, hl, hax, hth, hp, hc, T.TNSIM_C64, gp, stream.cuda_stream)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.grad_reps):
            ge, _ = T.tnsim_grad(nq, hl, hax, hth, hp, hc, T.TNSIM_C64, gp, stream.cuda_stream)
        tg = (time.perf_counter() - t0) / args.grad_reps
        grad_obj = {"value": 1.0 / tg, "unit": "energy gradients/s (1000 angles each)", "seconds": tg,
                    "energy": ge,
                    "sample": "50-qubit hardware-efficient ansatz, 10 layers of RY RZ on every qubit and a CZ "
                              "ladder, angles N(0, 0.3^2), chi_max 64, complex64, H = sum Z_i Z_i+1 + 0.5 sum X_i; "
                              "one synchronous tnsim_grad call: forward with checkpoints, final adjoint, "
                              "recompute and backward of every layer"}

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        r, gcount, secs = oracle_gate_rate(args.cpu_seconds)
        cpu = {"value": r, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{gcount} two-qubit updates at chi_L = chi_M = chi_R = 256 on random "
                         f"sites (numpy/LAPACK complex128 SVD), {secs:.1f} s"}

    if rank == 0:
        cfg = workload_config()
        cfg["gates_per_step"] = gates_all / args.steps
        cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
        cfg["jacobi_sweeps_per_gate"] = stats["sweeps"] / max(stats["gates"], 1)
        cfg["jacobi_config"] = {"chosen": int(tune_choice), "autotune_ms": [float(x) for x in tune_ms],
                                "configs": ["16-column blocks, 1 CTA/SM", "8-column blocks, 2 CTAs/SM",
                                            "16-column blocks, 1 CTA/SM, QR-preconditioned",
                                            "8-column blocks, 2 CTAs/SM, QR-preconditioned"]}
        cfg["interior_chi"] = int(np.max(dims))
        cfg["contraction"] = {"fp32": "FP32 FMA (4M)", "fp32_3m": "FP32 FMA (3M)",
                              "tf32x3": "tcgen05 3xTF32, FP32 accumulate",
                              "bf16x3": "tcgen05 BF16x3, FP32 accumulate"}[args.gemm]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e_obj,
                "gpu_launches": launches, "clocks": clocks, "plain_path": plain,
                "vs_plain": (value / plain["value"]) if plain else None, "kernels": kernels,
                "nonlocal": nonlocal_obj, "sampling": sampling_obj, "grad": grad_obj,
                "path_roofline": path_roofline}
        print(json.dumps(line), flush=True)
    m.close()
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
