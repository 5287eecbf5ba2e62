"""Pins of the learned-smoother oracle (oracle/mlp.py) against what mathematics fixes.

* gradients equal central finite differences of the loss (chain rule check
  independent of the backward formulas);
* the loss is zero at the targets the network reproduces exactly;
* bfloat16 rounding is exact on representable values, round-to-nearest-even
  on ties, and within half a unit in the 8th significant bit otherwise;
* features place each neighbour block where the slot rule (the face, the other
  faces of its first element, of its second; then the two elements' pressure
  blocks) puts it, and the map is homogeneous: scaling r scales s_F only.
"""
import numpy as np

from oracle.mlp import bf16_round, face_features, forward, loss_and_grads
from synthetic import tri_mesh


def _params(rng, din=12, hid=16, dout=8):
    return (rng.standard_normal((din, hid)) * 0.5, rng.standard_normal(hid) * 0.1,
            rng.standard_normal((hid, dout)) * 0.5, rng.standard_normal(dout) * 0.1)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    W1, b1, W2, b2 = _params(rng)
    X = rng.standard_normal((9, 12))
    T = rng.standard_normal((9, 8))
    loss, g = loss_and_grads(X, T, W1, b1, W2, b2)
    params = dict(W1=W1, b1=b1, W2=W2, b2=b2)
    h = 1e-6
    for name, P in params.items():
        flat = P.reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = loss_and_grads(X, T, W1, b1, W2, b2)
            flat[idx] = old - h
            lm, _ = loss_and_grads(X, T, W1, b1, W2, b2)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx)


def test_loss_zero_on_own_outputs():
    rng = np.random.default_rng(1)
    W1, b1, W2, b2 = _params(rng)
    X = rng.standard_normal((5, 12))
    _, Y = forward(X, W1, b1, W2, b2)
    loss, g = loss_and_grads(X, Y, W1, b1, W2, b2)
    assert loss == 0.0
    assert all(np.abs(v).max() == 0.0 for v in g.values())


def test_bf16_rounding():
    exact = np.array([1.0, -2.5, 0.15625, 3.0 * 2.0**-20, 0.0])
    assert np.array_equal(bf16_round(exact), exact)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1)
    assert bf16_round(np.array([1.0 + 2.0**-8]))[0] == 1.0
    assert bf16_round(np.array([1.0 + 3 * 2.0**-8]))[0] == 1.0 + 2.0**-6
    x = np.random.default_rng(2).standard_normal(1000)
    r = bf16_round(x)
    assert np.all(np.abs(r - x) <= 2.0**-8 * np.abs(x) * (1 + 1e-6))


def _slots(mesh):
    nf = mesh.n_face
    rows = []
    for F in range(nf):
        sl = [F]
        for T in mesh.face_elem[F]:
            if T < 0:
                continue
            sl += [int(G) for G in mesh.faces_of(T) if G != F]
        rows.append(sl)
    S_max = max(len(r) for r in rows)
    slots = -np.ones((S_max, nf), dtype=np.int64)
    for F, sl in enumerate(rows):
        slots[:len(sl), F] = sl
    return slots, mesh.face_elem.T.copy()


def test_features_follow_the_slot_rule_and_scale():
    mesh = tri_mesh(3, 2, jitter=0.1, seed=4, neumann_sides=(1,))
    b, nP = 4, 3
    nf, ne = mesh.n_face, mesh.n_elem
    slots, ptri = _slots(mesh)
    r = np.random.default_rng(3).standard_normal(nf * b + ne * nP)
    X, s = face_features(None, nf, b, nP, slots, ptri, r)
    S_max = slots.shape[0]
    for F in range(nf):
        for sidx in range(S_max):
            G = slots[sidx, F]
            want = r[G * b:(G + 1) * b] if G >= 0 else np.zeros(b)
            assert np.array_equal(X[F, sidx * b:(sidx + 1) * b], want)
        for p in range(2):
            T = ptri[p, F]
            want = r[nf * b + T * nP:nf * b + (T + 1) * nP] if T >= 0 else np.zeros(nP)
            assert np.array_equal(X[F, S_max * b + p * nP:S_max * b + (p + 1) * nP], want)
    assert np.allclose(s, np.linalg.norm(X, axis=1))
    X2, s2 = face_features(None, nf, b, nP, slots, ptri, -3.0 * r)
    assert np.allclose(X2, -3.0 * X) and np.allclose(s2, 3.0 * s)
