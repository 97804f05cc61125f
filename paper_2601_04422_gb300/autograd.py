"""torch.autograd.Function around tnsim_grad: the energy of a layered circuit as a
differentiable function of its angles.

The forward runs the library's reverse-mode gradient once (tnsim_grad returns the
energy and every angle derivative together) and keeps the gradient; the backward
scales it by the incoming gradient.  Argument marshalling only: the simulation and
its adjoint run in libtnsim.so.
"""
from __future__ import annotations

import numpy as np

from . import _abi


def _energy_function():
    import torch

    class CircuitEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, n_qubits, layers, axes, paulis, coeffs, dtype, params):
            sizes = [n_qubits * len(a) for a in axes]
            flat = theta.detach().to("cpu", torch.float64).numpy()
            th, off = [], 0
            for a, k in zip(axes, sizes):
                th.append(flat[off:off + k].reshape(n_qubits, len(a)))
                off += k
            e, grads = _abi.tnsim_grad(n_qubits, layers, axes, th, paulis, coeffs, dtype, params)
            g = np.concatenate([x.reshape(-1) for x in grads] + [np.zeros(0)])
            ctx.save_for_backward(torch.from_numpy(g).to(theta.device, theta.dtype))
            return theta.new_tensor(e)

        @staticmethod
        def backward(ctx, grad_e):
            (g,) = ctx.saved_tensors
            return (grad_e * g, None, None, None, None, None, None, None)

    return CircuitEnergy


def circuit_energy(theta, n_qubits, layers, axes, paulis, coeffs, dtype=_abi.TNSIM_C128, params=None):
    """E(theta) for a flat tensor of angles (layer after layer, [n_qubits][len(axes[L])]),
    differentiable with torch.autograd."""
    return _energy_function().apply(theta, n_qubits, layers, axes, paulis, coeffs, dtype, params)
