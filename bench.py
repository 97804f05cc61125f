#!/usr/bin/env python
"""Two-qubit gates/s at chi = 256 on one GB300 (contract + SVD + truncate + absorb).

Workload: a 100-qubit Haar SU(4) brickwork, chi_max = 256, complex64 (FP32
arithmetic), batched schedule.  The state is first evolved (untimed) until the
interior bonds saturate at chi = 256; then W warm-up layers, then K timed layers.
A step is one brickwork layer (49 or 50 gates).  The inputs (gates) sit in HBM
before the timed region starts; the state (88 MB) and per-layer workspace
(2 x 2 MiB per gate) together exceed the 126 MB L2.  Nothing but the layers runs
in the timed region (no per-kernel events).

Also reported on the same line:
  e2e          the synchronous C-ABI call with host gate buffers (copies included);
  roofline     the Jacobi kernel against the FP32 ALU peak, from per-kernel CUDA
               events recorded in a separate pass over the next layers;
  fidelity     1 - F of the complex64 states against the complex128 GPU path run
               from the same start state (after one layer and after all K layers);
  batched_c128 the complex128 path with the headline's schedule on the same layers;
  plain_path   the plain per-pair complex128 path on one layer of the same state;
  c4           256 independent circuits of uneven width, depth and chi_max as one
               CUDA graph of frozen plans;
  cpu_baseline the FP64 oracle on the host cores (all cores, and one thread).

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
HEA_CUTOFF = 1e-10          # discarded-weight cutoff of the gradient workload
# the column kernel and the scheduling header it includes (hashed together)
JACOBI_SRC = [os.path.join(ROOT, "paper_2601_04422_gb300", "csrc", f) for f in ("k_jacobi.cu", "jacobi_sched.cuh")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_jacobi_chi256.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-gates", type=int, default=64,
                    help="gates timed on the plain c128 path (at most one layer)")
    ap.add_argument("--profile-layers", type=int, default=3,
                    help="layers of the separate pass with per-kernel CUDA events")
    ap.add_argument("--no-fidelity", dest="fidelity", action="store_false",
                    help="skip the complex128 run from the timed region's start state")
    ap.add_argument("--c4-circuits", type=int, default=256, help="circuits of the batched graph leg (0 = skip)")
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
    sha = hashlib.sha256(b"".join(open(f, "rb").read() for f in JACOBI_SRC)).hexdigest()
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


def host_cores() -> int:
    """The host cores this process may run on (nproc)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


_ONE_THREAD = {k: "1" for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")}


def oracle_gate_rate_one_thread(seconds: float):
    """The same oracle sample in a child process whose BLAS/LAPACK runs on one thread
    (the thread count of a BLAS library is fixed when it loads)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "r, g, s = bench.oracle_gate_rate(%r); print(json.dumps([r, g, s]))" % (ROOT, float(seconds)))
    env = dict(os.environ, **_ONE_THREAD)
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=max(120.0, 10 * seconds))
    if out.returncode != 0:
        return None
    r, g, s = json.loads(out.stdout.strip().splitlines()[-1])
    return r, g, s


def mps_overlap(sa, sb) -> complex:
    """<a|b> of two MPS given as site lists (chi_l, 2, chi_r), by left-to-right transfer
    matrices with BLAS matrix products (measurement only: compares two outputs of the
    library, e.g. a complex64 and a complex128 run from the same start state)."""
    e = np.ones((1, 1), dtype=np.complex128)
    for a, b in zip(sa, sb):
        nxt = np.zeros((a.shape[2], b.shape[2]), dtype=np.complex128)
        for p in range(2):
            nxt += a[:, p, :].conj().T @ (e @ b[:, p, :])
        e = nxt
    return complex(e[0, 0])


def infidelity(sa, sb) -> float:
    ab = mps_overlap(sa, sb)
    return float(1.0 - abs(ab) ** 2 / (mps_overlap(sa, sa).real * mps_overlap(sb, sb).real))


def kernels_per_layer(gemm: str, cfg: int) -> int:
    """Kernels one batched layer launches: contraction (split + tcgen05 GEMM on the tensor
    path), QR (configurations 2, 3), Jacobi, truncation (column norms + selection), left
    site, right site, and the two site kernels of the QR route."""
    theta = 2 if gemm in ("tf32x3", "bf16x3") else 1
    return theta + 1 + 2 + 1 + 1 + (3 if cfg & 2 else 0)


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


def make_gates_dev(torch, dev, layers):
    return [torch.from_numpy(np.ascontiguousarray(l.g4).view(np.float64).copy()).to(dev) for l in layers]


def c4_leg(T, W, torch, dev, n_circ, gemm):
    """The batching workload: n_circ independent Haar SU(4) brickwork circuits of uneven
    width, depth and chi_max, every step a frozen plan of all states' gates, the whole run
    captured into one CUDA graph.  The graph is replayed once untimed (warm-up, from
    |0...0>), the states are reset to |0...0>, and one replay is timed by CUDA events."""
    batch = W.batch_circuits(n_circ, base_seed=1000)
    circs = [c for c, _ in batch]
    depth = max(len(c.layers) for c in circs)
    stream = torch.cuda.Stream(device=dev)
    ms = [T.MPS(c.n_qubits, dtype=T.TNSIM_C64, chi_max=chi, gemm=gemm, stream=stream.cuda_stream)
          for c, chi in batch]
    gdev = {}
    for i, c in enumerate(circs):
        for t, lay in enumerate(c.layers):
            gdev[(i, t)] = torch.from_numpy(np.ascontiguousarray(lay.g4).view(np.float64).copy()).to(dev)
    torch.cuda.synchronize()
    # autotune on the widest state with the largest chi_max, from its state after half its depth
    big = max(range(n_circ), key=lambda i: (batch[i][1], circs[i].n_qubits))
    half = len(circs[big].layers) // 2
    for lay in circs[big].layers[:half]:
        ms[big].apply_layer(lay)
    lay = circs[big].layers[half]
    choice, tune_ms = T.tnsim_autotune(ms[big].h, lay.pairs, lay.g4, reps=1)
    for m in ms:
        T.tnsim_set_jacobi_config(m.h, choice)
    zero = {}

    def reset():
        for i, m in enumerate(ms):
            n = circs[i].n_qubits
            if n not in zero:
                z = np.zeros((1, 2, 1), np.complex128)
                z[0, 0, 0] = 1.0
                zero[n] = [z] * n
            m.import_sites(zero[n])

    reset()
    plans = []
    for t in range(depth):
        idx = [i for i, c in enumerate(circs) if t < len(c.layers)]
        plans.append(T.tnsim_plan_create([ms[i].h for i in idx],
                                         [(circs[i].layers[t].pairs, gdev[(i, t)].data_ptr(), 0) for i in idx]))
    graph = T.tnsim_graph_create(plans)
    t0 = time.perf_counter()
    T.tnsim_graph_launch(graph)
    ms[0].sync()
    warm_s = time.perf_counter() - t0
    reset()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    T.tnsim_graph_launch(graph)
    e1.record(stream)
    ms[0].sync()
    ms_graph = e0.elapsed_time(e1)
    gates = sum(l.n2 for c in circs for l in c.layers)
    T.tnsim_graph_destroy(graph)
    for pl in plans:
        T.tnsim_plan_destroy(pl)
    for m in ms:
        m.close()
    return {"value": gates / (ms_graph / 1000.0), "unit": UNIT, "gates": gates, "ms": ms_graph,
            "circuits": n_circ, "steps": depth, "jacobi_config": int(choice),
            "autotune_ms": [float(x) for x in tune_ms], "warmup_replay_s": warm_s,
            "sample": f"{n_circ} Haar SU(4) brickwork circuits (width U{{16..128}}, depth U{{8..32}}, chi_max in "
                      "{16, 32, 64, 128, 256}, seeds 1000+i), complex64, every step one frozen plan of all "
                      "states' gates (one persistent Jacobi launch per step), all steps one CUDA graph; the "
                      "timed replay starts from |0...0> (CUDA events around the graph launch)"}


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

    K = args.steps
    n_prof = max(1, min(K, args.profile_layers))
    depth = PRESAT + args.warmup + 2 * K + n_prof + 2
    circ = W.brickwork_su4(N_QUBITS, depth, seed=replica_seed(rank))
    stream = torch.cuda.Stream(device=dev)
    gemm = getattr(T, "TNSIM_GEMM_" + args.gemm.upper())
    m = T.MPS(N_QUBITS, dtype=T.TNSIM_C64, chi_max=CHI, gemm=gemm, stream=stream.cuda_stream)
    gdev = make_gates_dev(torch, dev, circ.layers)
    eps_dev = torch.zeros(N_QUBITS, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()

    def layer_dev(mm, i):
        T.tnsim_apply_layer_device(mm.h, circ.layers[i].pairs, gdev[i].data_ptr(), 0, eps_dev.data_ptr())

    for i in range(PRESAT):
        layer_dev(m, i)
    m.sync()
    for i in range(PRESAT, PRESAT + args.warmup):
        layer_dev(m, i)
    m.sync()
    dims = m.bond_dims()
    t_lo = PRESAT + args.warmup
    # autotuner: time the Jacobi launch configurations on the first timed layer's gates
    tune_choice, tune_ms = T.tnsim_autotune(m.h, circ.layers[t_lo].pairs, circ.layers[t_lo].g4, reps=2)
    T.tnsim_last_stats(m.h)
    start_sites = m.export_sites() if (args.fidelity and rank == 0) else None

    # ---- timed region: device-resident inputs, no profiling
    timed = list(range(t_lo, t_lo + K))
    gates_rank = sum(circ.layers[i].n2 for i in timed)
    clk = ClockSampler(local)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in timed:
        layer_dev(m, i)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    m.sync()
    stats_timed = T.tnsim_last_stats(m.h)
    end_sites = m.export_sites() if start_sites is not None else None

    # ---- end to end: the synchronous C-ABI call on host buffers (copies inside)
    e2e = None
    disc_mean = None
    if not args.no_e2e:
        host_layers = circ.layers[t_lo + K: t_lo + 2 * K]
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        g_e2e = 0
        eps_all = []
        for l in host_layers:
            eps_all.append(T.tnsim_apply_layer(m.h, l.pairs, l.g4, None))
            g_e2e += l.n2
        t_e2e = time.perf_counter() - t0
        if dist:
            dist.barrier()
        e2e = (g_e2e, t_e2e, host_layers)
        disc_mean = float(np.mean(np.concatenate(eps_all)))

    # ---- per-kernel CUDA events, in a separate profiled pass over the next layers
    T.tnsim_last_stats(m.h)
    T.tnsim_profile_read(m.h)
    T.tnsim_profile_enable(m.h, True)
    for i in range(t_lo + 2 * K, t_lo + 2 * K + n_prof):
        layer_dev(m, i)
    m.sync()
    prof = T.tnsim_profile_read(m.h)
    T.tnsim_profile_enable(m.h, False)
    stats = T.tnsim_last_stats(m.h)

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

    # ---- roofline of the dominant kernel (the Jacobi SVD), FP32 ALU bound, from the profiled pass
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
                "avg_launch_ms": jac_ms / max(jac_n, 1),
                "profiled_layers": n_prof}
    # ---- whole-gate roofline time T* (contraction on the tensor pipe at the TF32 rate;
    # QR preconditioning and Jacobi on the FP32 ALUs; the site product on the tensor pipe
    # when the QR configurations run it there (tensor-core contraction modes), else on the
    # FP32 ALUs; site reads and writes at HBM rate)
    ng = max(stats["gates"], 1)
    tf32_peak = pk["bf16_tflops_sustained"] * (1.1 / 2.25)          # nominal TF32 : BF16 dense ratio
    site_tc = bool(int(tune_choice) & 2) and args.gemm in ("tf32x3", "bf16x3")
    t_contract = 8.0 * stats["theta_cmacs"] / ng / (tf32_peak * 1e12)
    t_svd = flops / ng / (peak * 1e12)
    t_right = 8.0 * stats["right_cmacs"] / ng / ((tf32_peak if site_tc else peak) * 1e12)
    t_qr = 8.0 * stats["qr_cmacs"] / ng / (peak * 1e12)
    site_bytes = 4.0 * 2 * CHI * CHI * 8                             # read A, B; write A', B' (complex64)
    t_mem = site_bytes / (pk["hbm_gbs"] * 1e9)
    t_star = t_contract + t_qr + t_svd + t_right + t_mem
    path_roofline = {"t_star_us_per_gate": t_star * 1e6, "gates_per_s_at_roofline": 1.0 / t_star,
                     "frac": value / (1.0 / t_star),
                     "parts_us": {"contraction_tf32": t_contract * 1e6, "qr_fp32": t_qr * 1e6,
                                  "jacobi_fp32": t_svd * 1e6,
                                  ("site_product_tf32" if site_tc else "site_product_fp32"): t_right * 1e6,
                                  "site_bytes_hbm": t_mem * 1e6},
                     "peaks": f"TF32 {tf32_peak:.0f} TFLOP/s (measured sustained BF16 x 1.1/2.25), FP32 ALU "
                              f"{peak:.1f} TFLOP/s, HBM {pk['hbm_gbs']:.0f} GB/s"}
    total_k_ms = sum(v[0] for v in prof.values())
    kernels = {k: {"ms": v[0], "launches": v[1], "share": (v[0] / total_k_ms if total_k_ms else 0.0)}
               for k, v in prof.items() if v[1]}
    launches = kernels_per_layer(args.gemm, int(tune_choice)) * K

    # ---- complex128 on the same saturated state: the batched schedule (same layers as the
    # timed region, from the same start state: also the fidelity reference) and the plain
    # per-pair schedule
    batched128 = fidelity = None
    if start_sites is not None:
        mb = T.MPS(N_QUBITS, dtype=T.TNSIM_C128, chi_max=CHI, stream=stream.cuda_stream)
        T.tnsim_set_jacobi_config(mb.h, int(tune_choice))
        mb.import_sites(start_sites)
        layer_dev(mb, timed[0])
        mb.sync()
        one128 = mb.export_sites()
        mb.stats()
        nb = len(timed) - 1
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for i in timed[1:]:
            layer_dev(mb, i)
        b1.record(stream)
        mb.sync()
        st_b = mb.stats()
        ms_b = b0.elapsed_time(b1)
        end128 = mb.export_sites()
        mb.close()
        g_b = sum(circ.layers[i].n2 for i in timed[1:])
        if nb > 0:
            batched128 = {"value": g_b / (ms_b / 1000.0), "unit": UNIT, "dtype": "f64",
                          "schedule": "batched, same launches as the headline", "layers": nb,
                          "ms_per_layer": ms_b / nb,
                          "jacobi_sweeps_per_gate": st_b["sweeps"] / max(st_b["gates"], 1),
                          "sample": f"timed layers 2..{K} of the headline from the same start state, complex128 "
                                    "(FP64 contraction and Jacobi), CUDA events"}
        # per layer: the complex64 replay of the timed layers from the same start state; at the
        # first, middle and last timed layer the complex128 path applies the same layer to the
        # complex64 input state
        m1 = T.MPS(N_QUBITS, dtype=T.TNSIM_C64, chi_max=CHI, gemm=gemm, stream=stream.cuda_stream)
        T.tnsim_set_jacobi_config(m1.h, int(tune_choice))
        m1.import_sites(start_sites)
        mc = T.MPS(N_QUBITS, dtype=T.TNSIM_C128, chi_max=CHI, stream=stream.cuda_stream)
        T.tnsim_set_jacobi_config(mc.h, int(tune_choice))
        probe = sorted({0, K // 2, K - 1})
        per_layer = []
        for j, i in enumerate(timed):
            pre = m1.export_sites() if j in probe else None
            layer_dev(m1, i)
            if pre is not None:
                post = m1.export_sites()
                if j == 0:
                    ref = one128
                else:
                    mc.import_sites(pre)
                    layer_dev(mc, i)
                    ref = mc.export_sites()
                per_layer.append({"timed_layer": j + 1, "1-F": infidelity(post, ref)})
        m1.close()
        mc.close()
        fidelity = {"per_layer": per_layer, "max_per_layer": max(x["1-F"] for x in per_layer),
                    "all_timed_layers": infidelity(end_sites, end128), "layers": K, "unit": "1 - F",
                    "note": "1 - |<a|b>|^2 / (<a|a><b|b>) against the complex128 GPU path.  per_layer: one layer "
                            "applied by both precisions to the same complex64 input state.  all_timed_layers: both "
                            "precisions run through all K timed layers from the same start state; the truncated "
                            "dynamics at chi 256 amplify any difference ~3.5x per layer, so the two runs drift apart "
                            "(the same holds between any two precisions)"}
    plain = None
    if args.plain_gates > 0 and rank == 0:
        sites = m.export_sites()
        mp = T.MPS(N_QUBITS, dtype=T.TNSIM_C128, chi_max=CHI, schedule=T.TNSIM_SCHED_PLAIN,
                   stream=stream.cuda_stream)
        T.tnsim_set_jacobi_config(mp.h, int(tune_choice))
        mp.import_sites(sites)
        lay_w = circ.layers[t_lo + 2 * K + n_prof]
        lay = circ.layers[t_lo + 2 * K + n_prof + 1]
        # warm-up: four gates of another layer on their own (module loads, first launches)
        mid = len(lay_w.pairs) // 2
        wsel = list(range(mid - 2, mid + 2))
        T.tnsim_apply_layer(mp.h, lay_w.pairs[wsel], lay_w.g4[wsel], None)
        mp.import_sites(sites)
        sel = list(range(min(args.plain_gates, lay.n2)))
        gp = torch.from_numpy(np.ascontiguousarray(lay.g4[sel]).view(np.float64).copy()).to(dev)
        mp.stats()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        T.tnsim_apply_layer_device(mp.h, lay.pairs[sel], gp.data_ptr(), 0, 0)
        p1.record(stream)
        mp.sync()
        tp = p0.elapsed_time(p1) / 1000.0
        st_p = mp.stats()
        chis = sorted({int(dims[int(x)]) for x in lay.pairs[sel]} | {int(dims[int(x) + 2]) for x in lay.pairs[sel]})
        plain = {"value": len(sel) / tp, "unit": UNIT, "dtype": "f64", "schedule": "one pair per launch sequence",
                 "sample": f"{len(sel)} gates of one layer of the saturated state (chi_L, chi_R in {chis}), after "
                           "a 4-gate warm-up, CUDA events on the library's stream",
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
    m.close()

    # ---- reverse-mode energy gradient (tnsim_grad) of the 50-qubit, 10-layer HEA at chi 64
    grad_obj = None
    if args.grad_reps > 0 and rank == 0:
        nq = 50
        hcirc, hang = W.hea_circuit(nq, 10, seed=7, sigma=0.3)
        hl = [(l.pairs, l.g4) for l in hcirc.layers]
        hax = ["YZ" if i % 2 == 0 else "" for i in range(len(hl))]
        hth = [hang[i // 2] if i % 2 == 0 else np.zeros((nq, 0)) for i in range(len(hl))]
        hp = ["".join("Z" if k in (i, i + 1) else "I" for k in range(nq)) for i in range(nq - 1)] + \
             ["".join("X" if k == i else "I" for k in range(nq)) for i in range(nq)]
        hc = [1.0] * (nq - 1) + [0.5] * nq
        gp = T.tnsim_params_default(T.TNSIM_C64)
        gp.chi_max = 64
        gp.cutoff = HEA_CUTOFF
        T.tnsim_grad(nq, hl, hax, hth, hp, hc, T.TNSIM_C64, gp, stream.cuda_stream)   # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.grad_reps):
            ge, _ = T.tnsim_grad(nq, hl, hax, hth, hp, hc, T.TNSIM_C64, gp, stream.cuda_stream)
        tg = (time.perf_counter() - t0) / args.grad_reps
        grad_obj = {"value": 1.0 / tg, "unit": "energy gradients/s (1000 angles each)", "seconds": tg,
                    "energy": ge,
                    "sample": "50-qubit hardware-efficient ansatz, 10 layers of RY RZ on every qubit and a CZ "
                              f"ladder, angles N(0, 0.3^2), chi_max 64, cutoff {HEA_CUTOFF:g}, complex64, "
                              "H = sum Z_i Z_i+1 + 0.5 sum X_i; one synchronous tnsim_grad call: forward with "
                              "checkpoints, final adjoint, recompute and backward of every layer"}

    # ---- the batching workload as one CUDA graph
    c4 = None
    if args.c4_circuits > 0 and rank == 0:
        c4 = c4_leg(T, W, torch, dev, args.c4_circuits, gemm)

    cpu = None
    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        r, gcount, secs = oracle_gate_rate(args.cpu_seconds)
        cpu = {"value": r, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": f"{gcount} two-qubit updates at chi_L = chi_M = chi_R = 256 on random "
                         f"sites (numpy/LAPACK complex128 SVD, BLAS threads on every core), {secs:.1f} s"}
        one = oracle_gate_rate_one_thread(args.cpu_seconds)
        if one is not None:
            cpu["single_thread"] = {"value": one[0], "unit": UNIT, "cores": 1,
                                    "sample": f"{one[1]} updates, same sample, BLAS/LAPACK on one thread, "
                                              f"{one[2]:.1f} s"}

    if rank == 0:
        cfg = workload_config()
        cfg["gates_per_step"] = gates_all / K
        cfg["parallelism"] = f"replicas x{world}" if world > 1 else "single GPU"
        cfg["jacobi_sweeps_per_gate"] = stats_timed["sweeps"] / max(stats_timed["gates"], 1)
        cfg["jacobi_config"] = {"chosen": int(tune_choice), "autotune_ms": [float(x) for x in tune_ms],
                                "configs": ["16-column blocks, 1 CTA/SM", "8-column blocks, 2 CTAs/SM",
                                            "16-column blocks, 1 CTA/SM, QR-preconditioned",
                                            "8-column blocks, 2 CTAs/SM, QR-preconditioned",
                                            "Gram-matrix visits, tcgen05 block products",
                                            "same as 4 (bit 0 has no effect)",
                                            "Gram-matrix visits, tcgen05 block products, QR-preconditioned",
                                            "same as 6 (bit 0 has no effect)"]}
        cfg["interior_chi"] = int(np.max(dims))
        cfg["discarded_weight_per_gate"] = disc_mean
        cfg["contraction"] = {"fp32": "FP32 FMA (4M)", "fp32_3m": "FP32 FMA (3M)",
                              "tf32x3": "tcgen05 3xTF32, FP32 accumulate",
                              "bf16x3": "tcgen05 BF16x3, FP32 accumulate"}[args.gemm]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
                "warmup": args.warmup, "ms_per_step": ms_max / K, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e_obj,
                "gpu_launches": launches, "clocks": clocks, "fidelity": fidelity,
                "batched_c128": batched128, "plain_path": plain,
                "vs_plain": (value / plain["value"]) if plain else None,
                "vs_batched_c128": (value / batched128["value"]) if batched128 else None,
                "kernels": kernels, "c4": c4, "nonlocal": nonlocal_obj, "sampling": sampling_obj,
                "grad": grad_obj, "path_roofline": path_roofline}
        print(json.dumps(line), flush=True)
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
