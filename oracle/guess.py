"""Oracle for the learned density guess. TEST INFRASTRUCTURE ONLY.

Plain numpy (FP64) statements of what the GPU guess computes:

* the local frame of an atom pair (A, B): e_z along A -> B (for A == B towards
  A's nearest neighbour), e_x from the atom nearest to the pair midpoint
  (for A == B the second-nearest neighbour of A), made orthogonal to e_z,
  e_y = e_z x e_x;
* rotation-invariant features: element one-hots of A and B, a same-atom flag,
  R_AB, a Gaussian expansion of R_AB, and the K nearest neighbours of the
  midpoint (element one-hot, local coordinates, 1/r);
* the representation of a rotation on the basis functions of one atom
  (s: 1; p: the 3x3 rotation; d: the 5x5 matrix of the real solid harmonics,
  c_mn = <Q_m, U Q_n U^T> / 1.5 with Q_n the traceless symmetric matrix of
  harmonic n), and the block transform D_local = M_A^T D_lab M_B;
* a multilayer perceptron with SiLU activations, mean-squared error and its
  gradient by the chain rule written out layer by layer.
"""
from __future__ import annotations

import math

import numpy as np

ELEMENTS = (1, 6, 8)          # H, C, O
NNEIGH = 8                    # neighbours of the pair midpoint in the features
NRBF = 16                     # Gaussian radial functions of R_AB
RCUT = 4.0 / 0.529177210903   # pair cutoff, 4 Angstrom in bohr
NFEAT = 3 + 3 + 1 + 1 + NRBF + 7 * NNEIGH   # 80
NFEAT_PAD = 96


def _onehot(z):
    return np.array([1.0 if z == e else 0.0 for e in ELEMENTS])


def _unit(v):
    return v / np.linalg.norm(v)


def pair_frame(xyz, A, B):
    """3x3 matrix whose rows are the local axes (e_x, e_y, e_z) in the lab."""
    n = len(xyz)
    if A != B:
        ez = _unit(xyz[B] - xyz[A])
        M = 0.5 * (xyz[A] + xyz[B])
        cand = [i for i in range(n) if i not in (A, B)]
        ref = min(cand, key=lambda i: (np.linalg.norm(xyz[i] - M), i)) if cand else None
        origin = M
    else:
        cand = sorted((i for i in range(n) if i != A), key=lambda i: (np.linalg.norm(xyz[i] - xyz[A]), i))
        ez = _unit(xyz[cand[0]] - xyz[A]) if cand else np.array([0.0, 0.0, 1.0])
        ref = cand[1] if len(cand) > 1 else None
        origin = xyz[A]
    v = (xyz[ref] - origin) if ref is not None else np.array([1.0, 0.0, 0.0])
    v = v - (v @ ez) * ez
    if np.linalg.norm(v) < 1e-8:
        # reference collinear with the pair axis: any vector normal to e_z
        v = np.array([1.0, 0.0, 0.0]) if abs(ez[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        v = v - (v @ ez) * ez
    ex = _unit(v)
    ey = np.cross(ez, ex)
    return np.stack([ex, ey, ez])


def pair_features(Z, xyz, A, B):
    """Invariant feature vector (length NFEAT_PAD, zero-padded)."""
    U = pair_frame(xyz, A, B)
    M = 0.5 * (xyz[A] + xyz[B])
    R = float(np.linalg.norm(xyz[B] - xyz[A]))
    f = [*_onehot(Z[A]), *_onehot(Z[B]), 1.0 if A == B else 0.0, R]
    mu = np.linspace(0.0, RCUT, NRBF)
    w = RCUT / (NRBF - 1)
    f += list(np.exp(-((R - mu) / w) ** 2))
    others = sorted((i for i in range(len(Z)) if i not in (A, B)), key=lambda i: (np.linalg.norm(xyz[i] - M), i))
    for k in range(NNEIGH):
        if k < len(others):
            i = others[k]
            d = xyz[i] - M
            r = float(np.linalg.norm(d))
            f += [*_onehot(Z[i]), *(U @ d), 1.0 / max(r, 1e-6)]
        else:
            f += [0.0] * 7
    out = np.zeros(NFEAT_PAD)
    out[:len(f)] = f
    return out


_S3 = math.sqrt(3.0)
# real solid harmonics of the d shell (order m = -2..2) as quadratic forms r^T Q r
_QD = [
    np.array([[0, _S3 / 2, 0], [_S3 / 2, 0, 0], [0, 0, 0]]),        # sqrt3 xy
    np.array([[0, 0, 0], [0, 0, _S3 / 2], [0, _S3 / 2, 0]]),        # sqrt3 yz
    np.array([[-0.5, 0, 0], [0, -0.5, 0], [0, 0, 1.0]]),            # zz - (xx+yy)/2
    np.array([[0, 0, _S3 / 2], [0, 0, 0], [_S3 / 2, 0, 0]]),        # sqrt3 xz
    np.array([[_S3 / 2, 0, 0], [0, -_S3 / 2, 0], [0, 0, 0]]),       # sqrt3/2 (xx-yy)
]


def shell_rotation(l, U):
    """M with phi_lab = M phi_local for the functions of one shell, U the
    frame (rows = local axes): a lab function evaluated at r = U^T r'."""
    if l == 0:
        return np.ones((1, 1))
    if l == 1:
        return U.T.copy()
    C = np.zeros((5, 5))
    for n in range(5):
        Qr = U @ _QD[n] @ U.T
        for m in range(5):
            C[n, m] = float(np.sum(_QD[m] * Qr)) / 1.5
    return C


def atom_rotation(shell_ls, U):
    mats = [shell_rotation(l, U) for l in shell_ls]
    n = sum(m.shape[0] for m in mats)
    M = np.zeros((n, n))
    o = 0
    for m in mats:
        k = m.shape[0]
        M[o:o + k, o:o + k] = m
        o += k
    return M


def to_local(D_lab_block, MA, MB):
    return MA.T @ D_lab_block @ MB


def to_lab(D_loc_block, MA, MB):
    return MA @ D_loc_block @ MB.T


# ------------------------------------------------------------------ MLP
def silu(x):
    return x / (1.0 + np.exp(-x))


def dsilu(x):
    s = 1.0 / (1.0 + np.exp(-x))
    return s * (1.0 + x * (1.0 - s))


def mlp_forward(params, X):
    """params: list of (W, b) for the hidden layers, then (Wo, bo).
    Returns (output, cache)."""
    acts = [X]
    pres = []
    h = X
    for W, b in params[:-1]:
        z = h @ W + b
        pres.append(z)
        h = silu(z)
        acts.append(h)
    Wo, bo = params[-1]
    return h @ Wo + bo, (acts, pres)


def mse_loss_and_grads(params, X, Y):
    """L = mean over all entries of (out - Y)^2 and dL/dparams by backprop."""
    out, (acts, pres) = mlp_forward(params, X)
    n = out.size
    L = float(np.sum((out - Y) ** 2)) / n
    d = 2.0 * (out - Y) / n
    grads = [None] * len(params)
    Wo, bo = params[-1]
    grads[-1] = (acts[-1].T @ d, d.sum(axis=0))
    dh = d @ Wo.T
    for k in range(len(params) - 2, -1, -1):
        dz = dh * dsilu(pres[k])
        W, b = params[k]
        grads[k] = (acts[k].T @ dz, dz.sum(axis=0))
        dh = dz @ W.T
    return L, grads
