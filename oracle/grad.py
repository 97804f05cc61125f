"""Reverse-mode gradient of an energy through the MPS simulation -- oracle (FP64).

Test infrastructure only (see the package docstring).  The paper does not
differentiate its simulator; this module is the plain reference for the library's
adjoint (tnsim_grad), written from the chain rule of the paper's own steps
(Sec. III.A "One Qubit Gate", "Two Qubit Gate"; Eq. 1, Eq. 3):

  forward, layer by layer: every qubit gets the product of its rotations
  R_a(t) = exp(-i t P_a / 2) (the first listed acts first), then the layer's
  two-qubit gates run the merge / gate / truncated SVD / absorb update of apply_2q;
  the energy is E = <psi|H|psi> / <psi|psi> for H = sum_t c_t P_t (Pauli strings).

Conventions: for a complex intermediate X, Xb = dE/d(conj X) (conjugate Wirtinger
derivative), so that dE = 2 Re <Xb, dX>; for the real singular values, g = dE/ds.

The truncated update is differentiated through its kept subspace
(truncation_backward): the new sites are U (the top-k left singular vectors of the
gated block T) and c Y with Y = U^H T, and the loss depends on U only through
span(U).  Perturbing that subspace couples kept and discarded directions only, with
the broadened denominators 1 / (s_j^2 - s_l^2) across the cut; the result is the
exact derivative of the truncated map (degenerate kept singular values included),
and the renormalisation factor c = |T|_F / |Y|_F is differentiated exactly.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np

from . import mps as M

PAULI = M.PAULI


def rotation(axis: str, t: float) -> np.ndarray:
    """R_a(t) = exp(-i t P_a / 2) = cos(t/2) I - i sin(t/2) P_a."""
    return np.cos(t / 2) * np.eye(2, dtype=np.complex128) - 1j * np.sin(t / 2) * PAULI[axis]


def rotation_product(axes: str, ts: Sequence[float]) -> np.ndarray:
    """u = R_{a_last}(t_last) ... R_{a_0}(t_0): the first rotation acts first."""
    u = np.eye(2, dtype=np.complex128)
    for a, t in zip(axes, ts):
        u = rotation(a, t) @ u
    return u


def rotation_product_grad(axes: str, ts: Sequence[float], ub: np.ndarray) -> np.ndarray:
    """dE/dt_j = 2 Re <ub, du/dt_j> with dR_a/dt = (-i/2) P_a R_a."""
    out = np.zeros(len(axes))
    for j in range(len(axes)):
        u = np.eye(2, dtype=np.complex128)
        for i, (a, t) in enumerate(zip(axes, ts)):
            r = rotation(a, t)
            if i == j:
                r = -0.5j * PAULI[a] @ r
            u = r @ u
        out[j] = 2.0 * np.real(np.vdot(ub, u))
    return out


# --------------------------------------------------------------------------
# forward


def layer_u1(n: int, axes: str, th: np.ndarray):
    """One-qubit gates of a layer from its angles th[n, len(axes)] (None if no rotations)."""
    if len(axes) == 0:
        return None
    return np.stack([rotation_product(axes, th[q]) for q in range(n)])


def energy(mps: M.MPS, paulis: Sequence[str], coeffs: Sequence[float]) -> float:
    """E = sum_t c_t <P_t> / <psi|psi>."""
    num = sum(c * M.expect_pauli(mps, p).real for p, c in zip(paulis, coeffs))
    return float(num / M.norm2(mps))


def energy_local(mps: M.MPS, paulis: Sequence[str], coeffs: Sequence[float]) -> float:
    """The same E as ``energy``, with each Pauli string contracted only over its support:
    <P> = L_lo . (sites lo..hi with their operators) . R_{hi+1}, where L and R are the
    left / right environments of the identity (every site outside the support carries
    the identity, so the rest of the chain is L and R)."""
    n = mps.n
    eye = [PAULI["I"]] * n
    L0, R0 = _env_left(mps.sites, eye), _env_right(mps.sites, eye)
    nrm = float(L0[n][0, 0].real)
    num = 0.0
    for p, c in zip(paulis, coeffs):
        sup = [q for q, ch in enumerate(p) if ch != "I"]
        if not sup:
            num += c * nrm
            continue
        e = L0[sup[0]]
        for q in range(sup[0], sup[-1] + 1):
            a = mps.sites[q]
            op = PAULI[p[q]]
            # e'[a', b'] = sum conj(A[x, p, a']) op[p, p'] e[x, y] A[y, p', b']
            e = np.einsum("xpa,pq,xy,yqb->ab", a.conj(), op, e, a, optimize=True)
        num += c * float(np.einsum("ab,ab->", e, R0[sup[-1] + 1]).real)
    return float(num / nrm)


def run(n: int, layers, axes: List[str], theta: List[np.ndarray], chi_max: int, cutoff: float = 0.0,
        renormalize: bool = True):
    """Forward pass; layers[L] = (pairs, g4[n2,4,4]); returns (final mps, checkpoints before each layer)."""
    m = M.zero_state(n)
    ckpt = []
    for L, (pairs, g4) in enumerate(layers):
        ckpt.append(m.copy())
        u1 = layer_u1(n, axes[L], theta[L])
        if u1 is not None:
            for q in range(n):
                M.apply_1q(m, q, u1[q])
        for q, g in zip(pairs, g4):
            M.apply_2q(m, int(q), g, chi_max, cutoff, renormalize)
    return m, ckpt


# --------------------------------------------------------------------------
# adjoint of the final state


def _env_left(sites, ops):
    """E_q[a, b] = sum conj(A..)[.., a] O A..[.., b] over sites < q, q = 0..n."""
    envs = [np.ones((1, 1), dtype=np.complex128)]
    for a, o in zip(sites, ops):
        e = envs[-1]
        envs.append(np.einsum("xy,xpa,pq,yqb->ab", e, a.conj(), o, a, optimize=True))
    return envs


def _env_right(sites, ops):
    """R_q[a, b] = sum conj(A..)[a, ..] O A..[b, ..] over sites >= q, q = 0..n."""
    n = len(sites)
    envs = [None] * (n + 1)
    envs[n] = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        a = sites[q]
        envs[q] = np.einsum("xpa,pq,yqb,ab->xy", a.conj(), ops[q], a, envs[q + 1], optimize=True)
    return envs


def final_adjoint(mps: M.MPS, paulis: Sequence[str], coeffs: Sequence[float]):
    """(E, [Ab_q]) with Ab_q = dE/d(conj A_q) for E = <psi|H|psi> / <psi|psi>.

    For one Pauli string P, d<psi|P|psi>/d(conj A_q)[l, p, r]
      = sum E_q[l, l'] P_q[p, p'] A_q[l', p', r'] R_{q+1}[r, r']
    with the left / right environments of P.  This is the plain per-term version."""
    n = mps.n
    eye = [PAULI["I"]] * n
    L0, R0 = _env_left(mps.sites, eye), _env_right(mps.sites, eye)
    nrm = float(L0[n][0, 0].real)
    hsum = 0.0
    abar_h = [np.zeros_like(a) for a in mps.sites]
    for p, c in zip(paulis, coeffs):
        ops = [PAULI[ch] for ch in p]
        Lp, Rp = _env_left(mps.sites, ops), _env_right(mps.sites, ops)
        hsum += c * Lp[n][0, 0].real
        for q in range(n):
            abar_h[q] += c * np.einsum("xy,pq,yqb,ab->xpa", Lp[q], ops[q], mps.sites[q], Rp[q + 1], optimize=True)
    e = hsum / nrm
    abar = []
    for q in range(n):
        an = np.einsum("xy,yqb,ab->xqa", L0[q], mps.sites[q], R0[q + 1], optimize=True)
        abar.append((abar_h[q] - e * an) / nrm)
    return e, abar


# --------------------------------------------------------------------------
# backward through the steps


def truncation_backward(T, uk, y, s, nz, u_all, ub, yb, tau: float = 0.0, broaden: float = 1e-32):
    """Tb for the truncated update T -> (U, Y): U (m x k) the kept left singular vectors
    of T as the forward produced them, Y = U^H T, given Ub and the total Yb.

    The loss is unchanged by U -> U R, Y -> R^H Y for any unitary R (a gauge change of
    the new bond), so it depends on U only through the kept subspace span(U), the
    dominant k-dimensional eigenspace of H = T T^H.  First-order perturbation of that
    subspace only couples kept directions j to discarded ones l, with denominators
    s_j^2 - s_l^2 across the cut:
      Tb = U Yb + (I - P) Ut S_k^-2 Y + (Z + Z^H) T,
      Ut = Ub + T Yb^H,  Z = U_D (G o (U_D^H Ut)) U^H,  G_lj = 1 / (s_j^2 - s_l^2) (broadened),
    with P the projector on every nonzero singular direction and U_D the discarded
    nonzero ones.  S_k^-1 V_k^H is written as S_k^-2 Y, which holds in any gauge of
    U (the gauge freedom of an SVD commutes with S).  U and Y must be the forward's
    own factors: for degenerate singular values a recomputed SVD may pick another
    basis, and the incoming adjoints refer to the forward's.  s, u_all: a full SVD of
    T (descending; only gauge-invariant parts of it are used); nz: how many s are
    nonzero.  This is the exact derivative of the truncated map.

    (I - P) Ut equals (I - P) Ub exactly, since (I - P) T = 0; the latter is used, which
    avoids dividing the rounding of (I - P) T Yb^H by s_j.  tau > 0: kept directions with
    s_j <= tau s_max get no inverse factors (a pseudo-inverse cutoff): their rows of
    S_k^-2 Y and their columns of G are zero.  tau = 0 is the exact derivative.
    broaden: G_lj = d / (d^2 + broaden s_max^2 (s_j + s_l)^2) with d = s_j^2 - s_l^2, a
    Lorentzian broadening of the cut's denominators on the scale of the rounding error
    of d: singular values computed with absolute errors ~ eps s_max give |delta d| ~
    eps s_max (s_j + s_l), so broaden = eps^2 regularises exactly the pairs whose
    denominator is not resolved, and leaves small but separated singular values
    alone.  At a degenerate cut the truncated map is not differentiable and this
    keeps the result finite."""
    k = uk.shape[1]
    sk = s[:k]
    ud, sd = u_all[:, k:nz], s[k:nz]
    ut = ub + T @ yb.conj().T
    tb = uk @ yb
    p_all = u_all[:, :nz] @ u_all[:, :nz].conj().T
    live = sk > tau * s[0]
    inv2 = np.where(live, 1.0 / np.where(live, sk * sk, 1.0), 0.0)
    tb += (ub - p_all @ ub) @ (y * inv2[:, None])
    if nz > k:
        d = sk[None, :] ** 2 - sd[:, None] ** 2                 # [l, j] = s_j^2 - s_l^2
        eps_b = broaden * sk[0] ** 2 * (sk[None, :] + sd[:, None]) ** 2
        G = (d / (d * d + eps_b)) * live[None, :]
        Z = ud @ (G * (ud.conj().T @ ut)) @ uk.conj().T
        tb += (Z + Z.conj().T) @ T
    return tb


def gate_backward(a, b, g4, ul, ur, a_new, b_new, ab_new, bb_new, renormalize, tau: float = 0.0,
                  broaden: float = 1e-32):
    """Backward of one two-qubit update on pre-gate sites a, b (before the one-qubit gates
    ul, ur of the layer, None = identity) that produced a_new (U) and b_new (c Y, c the
    renormalisation factor |T|_F / |Y|_F).  ab_new, bb_new: adjoints of the new sites.
    Returns (ab, bb, ubar_l, ubar_r)."""
    chi_l, chi_m, chi_r = a.shape[0], a.shape[2], b.shape[2]
    k = a_new.shape[2]
    ul = np.eye(2, dtype=np.complex128) if ul is None else ul
    ur = np.eye(2, dtype=np.complex128) if ur is None else ur
    K = np.kron(ul, ur)
    Gt = g4 @ K
    merged = M.merge_sites(a, b)                                   # [l, c, d, r]
    theta = M.contract_gate(merged, Gt)
    T = theta.reshape(2 * chi_l, 2 * chi_r)
    u_all, s, _ = np.linalg.svd(T, full_matrices=False)
    nz = max(k, int(np.count_nonzero(s > M.EPS64 * max(T.shape) * s[0])))
    uk = a_new.reshape(2 * chi_l, k)
    F2 = float(np.sum(s * s))
    K2 = float(np.sum(s[:k] ** 2))
    c = np.sqrt(F2 / K2) if renormalize and K2 > 0 else 1.0
    Y = b_new.reshape(k, 2 * chi_r) / c
    ub_ = ab_new.reshape(2 * chi_l, k)
    Bb = bb_new.reshape(k, 2 * chi_r)
    yb = c * Bb
    Tb = np.zeros_like(T)
    if renormalize and K2 > 0:
        dldc = 2.0 * float(np.real(np.vdot(Bb, Y)))
        Tb += (dldc * c / (2.0 * F2)) * T
        yb = yb - (dldc * c / (2.0 * K2)) * Y
    Tb += truncation_backward(T, uk, Y, s, nz, u_all, ub_, yb, tau, broaden)
    thb = Tb.reshape(chi_l, 2, 2, chi_r)
    Gt4 = Gt.reshape(2, 2, 2, 2)
    mb = np.einsum("abcd,labr->lcdr", Gt4.conj(), thb)
    gtb = np.einsum("labr,lcdr->abcd", thb, merged.conj()).reshape(4, 4)
    ab = np.einsum("lcdr,mdr->lcm", mb, b.conj())
    bb = np.einsum("lcm,lcdr->mdr", a.conj(), mb)
    Kb = (g4.conj().T @ gtb).reshape(2, 2, 2, 2)                   # [a, b, c, d]
    ubl = np.einsum("abcd,bd->ac", Kb, ur.conj())
    ubr = np.einsum("abcd,ac->bd", Kb, ul.conj())
    return ab, bb, ubl, ubr


def grad(n: int, layers, axes: List[str], theta: List[np.ndarray], paulis, coeffs, chi_max: int,
         cutoff: float = 0.0, renormalize: bool = True, tau: float = 0.0, broaden: float = 1e-32):
    """(E, [dE/dtheta_L]) for the layered circuit; theta[L] has shape [n, len(axes[L])]."""
    final, ckpt = run(n, layers, axes, theta, chi_max, cutoff, renormalize)
    e, abar = final_adjoint(final, paulis, coeffs)
    post_states = ckpt[1:] + [final]
    grads = [np.zeros_like(np.asarray(t, dtype=np.float64)) for t in theta]
    for L in range(len(layers) - 1, -1, -1):
        pairs, g4 = layers[L]
        pre = ckpt[L]
        u1 = layer_u1(n, axes[L], theta[L])
        ubar = [np.zeros((2, 2), dtype=np.complex128) for _ in range(n)]
        paired = set()
        new_abar = list(abar)
        for q, g in zip(pairs, g4):
            q = int(q)
            paired.update((q, q + 1))
            ul = None if u1 is None else u1[q]
            ur = None if u1 is None else u1[q + 1]
            post = post_states[L]
            ab, bb, ubl, ubr = gate_backward(pre.sites[q], pre.sites[q + 1], g, ul, ur, post.sites[q],
                                             post.sites[q + 1], abar[q], abar[q + 1], renormalize, tau,
                                             broaden)
            new_abar[q], new_abar[q + 1] = ab, bb
            ubar[q] += ubl
            ubar[q + 1] += ubr
        if u1 is not None:
            for q in range(n):
                if q in paired:
                    continue
                a_pre = pre.sites[q]
                ubar[q] += np.einsum("lpr,lsr->ps", abar[q], a_pre.conj())
                new_abar[q] = np.einsum("ps,lpr->lsr", u1[q].conj(), abar[q])
            for q in range(n):
                grads[L][q] = rotation_product_grad(axes[L], theta[L][q], ubar[q])
        abar = new_abar
    return e, grads
