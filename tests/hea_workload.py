"""The differentiation workload (50-qubit hardware-efficient ansatz) and one oracle
energy evaluation of it at shifted angles, importable by spawned worker processes for
the finite differences of tests/test_gpu_grad.py.

Workload: 50 qubits, 10 layers of RY(t) RZ(t) on every qubit then a CZ ladder,
t ~ N(0, 0.3^2) (1000 angles), chi_max 64, H = sum Z_i Z_i+1 + 0.5 sum X_i.
Readings stated here (the workload names neither):
  seed 2 of the angle generator;
  a discarded-weight cutoff of 1e-10.  Without a cutoff the truncation keeps
  numerically zero singular directions (s ~ 1e-14 s_max) whenever the bond has room;
  which ones is decided by rounding, and because the paper's form truncates later
  bonds in a gauge that these directions enter with full weight, the truncated energy
  then jumps by ~1e-5 under angle changes of 1e-6 and has no derivative.  With the
  cutoff those directions are dropped and the energy is smooth at the scale of the
  finite differences.
"""
import numpy as np

import workloads as W
from oracle import grad as OG

N, N_LAYERS, SIGMA, CHI = 50, 10, 0.3, 64
SEED, CUTOFF = 7, 1e-10


def hea(n=N, n_layers=N_LAYERS, seed=SEED, sigma=SIGMA):
    circ, angles = W.hea_circuit(n, n_layers, seed=seed, sigma=sigma)
    layers = [(l.pairs, l.g4) for l in circ.layers]
    axes = ["YZ" if i % 2 == 0 else "" for i in range(len(layers))]
    theta = [angles[i // 2].copy() if i % 2 == 0 else np.zeros((n, 0)) for i in range(len(layers))]
    paulis = ["".join("Z" if k in (i, i + 1) else "I" for k in range(n)) for i in range(n - 1)] + \
             ["".join("X" if k == i else "I" for k in range(n)) for i in range(n)]
    coeffs = [1.0] * (n - 1) + [0.5] * n
    return layers, axes, theta, paulis, coeffs


def energy_shifted(arg):
    """Oracle energy with angle theta[L][q, j] shifted by h (FP64); arg = (L, q, j, h) or
    (L, q, j, h, seed, cutoff)."""
    L, q, j, h = arg[:4]
    seed, cutoff = (arg[4], arg[5]) if len(arg) > 4 else (SEED, CUTOFF)
    layers, axes, theta, paulis, coeffs = hea(seed=seed)
    theta[L][q, j] += h
    m, _ = OG.run(N, layers, axes, theta, CHI, cutoff)
    return OG.energy_local(m, paulis, coeffs)
