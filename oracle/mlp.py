"""Learned block smoother (oracle): features, two-layer MLP, loss and gradients.

Test infrastructure (an extension; the paper has no learned component): the
plain FP64 reference of what the library's learned smoother computes, used to
check the GPU features, forward pass and gradients.

* Features of face F (level 0): the residual blocks of F's neighbourhood in
  the operator's slot order -- F itself, then the other faces of its first
  element, then of its second (zeros for missing slots) -- followed by the
  pressure blocks of its first and second element (zeros on the boundary),
  zero-padded to d_in.  The feature vector is divided by its Euclidean norm
  s_F (the map is then homogeneous of degree one: N(a r) = a N(r)).
* Network: h = relu(W1^T x + b1) (hidden width n_h), y = W2^T h + b2; the
  correction to the block-Jacobi output on face F's rows is s_F y[:b].
* Training target for a pair (r, e): t_F = (e_F - (M_J^{-1} r)_F) / s_F, the
  part of the error the block-Jacobi step misses; loss = mean over samples of
  ||y - t||^2 (sum over the b outputs).
* Gradients by the chain rule: dY = 2 (Y - T) / B; dW2 = H^T dY,
  db2 = sum dY; dH = (dY W2^T) * [H > 0]; dW1 = X^T dH, db1 = sum dH.
  Pinned against central finite differences of the loss.
"""
from __future__ import annotations

import numpy as np


def face_features(S, nf, b, nP, slots, ptri, r):
    """(nf, S_max*b + 2*nP) raw features and their norms.

    slots: (S_max, nf) column face of each slot (-1 missing); ptri: (2, nf)
    element of each side (-1 missing); r: level-0 vector (faces then elements)."""
    S_max = slots.shape[0]
    X = np.zeros((nf, S_max * b + 2 * nP))
    for s in range(S_max):
        G = slots[s]
        ok = G >= 0
        idx = G[ok][:, None] * b + np.arange(b)[None, :]
        X[np.where(ok)[0], s * b:(s + 1) * b] = r[idx]
    for p in range(2):
        T = ptri[p]
        ok = T >= 0
        idx = nf * b + T[ok][:, None] * nP + np.arange(nP)[None, :]
        X[np.where(ok)[0], S_max * b + p * nP:S_max * b + (p + 1) * nP] = r[idx]
    s = np.linalg.norm(X, axis=1)
    return X, s


def forward(X, W1, b1, W2, b2):
    """H (B, n_h) after relu and Y (B, n_out)."""
    H = np.maximum(X @ W1 + b1, 0.0)
    return H, H @ W2 + b2


def loss_and_grads(X, T, W1, b1, W2, b2):
    H, Y = forward(X, W1, b1, W2, b2)
    B = X.shape[0]
    D = Y - T
    loss = float(np.sum(D * D) / B)
    dY = 2.0 * D / B
    dW2 = H.T @ dY
    db2 = dY.sum(axis=0)
    dH = (dY @ W2.T) * (H > 0.0)
    dW1 = X.T @ dH
    db1 = dH.sum(axis=0)
    return loss, dict(W1=dW1, b1=db1, W2=dW2, b2=db2)


def bf16_round(a):
    """Round to bfloat16 (round to nearest even on the upper 16 bits of the float32)."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
