"""FP64 oracle of the learned rotation proposal and the sparse Maximize.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU legs); the GPU
library never uses it. Plain numpy in float64, written from the definitions.

The paper has no learned proposal; this follows the workload's statement of it:
per frame, 32 radial x 16 angular bins of log(1 + mean count) feed an MLP with
three hidden layers of 512 GELU units and one logit per sampled rotation; the
top-M logits give candidate rotations, and the Maximize step runs over those
candidates only (Eq. 2.4 and Eq. 2.11 restricted to the candidate set C_k):
  S_jk for j in C_k,  P_jk = exp(S_jk - log sum_{j' in C_k} exp(S_j'k)),
  Num_j = sum_{k: j in C_k} P_jk K_k,  den_j = sum_{k: j in C_k} P_jk.
Training: soft targets T_k from dense EMC responsibilities (top R per frame,
renormalised); loss = -mean_k sum_j T_jk log softmax(z_k)_j; Adam.
"""
from __future__ import annotations

import math

import numpy as np

N_RAD, N_ANG = 32, 16
N_FEAT = N_RAD * N_ANG


# ----------------------------------------------------------------------------
# features
# ----------------------------------------------------------------------------

def feature_bins(q: np.ndarray) -> np.ndarray:
    """Bin index (radial * 16 + angular) of every pixel.

    radial bin: floor(32 |q_i| / max_i |q_i|), capped at 31;
    angular bin: floor(16 (atan2(q_y, q_x) + pi) / (2 pi)), capped at 15.
    """
    q = np.asarray(q, dtype=np.float64)
    r = np.sqrt(q[:, 0] * q[:, 0] + q[:, 1] * q[:, 1] + q[:, 2] * q[:, 2])
    rmax = r.max()
    rb = np.minimum(np.floor(N_RAD * r / rmax).astype(np.int64), N_RAD - 1)
    th = np.arctan2(q[:, 1], q[:, 0])
    ab = np.minimum(np.floor(N_ANG * (th + math.pi) / (2 * math.pi)).astype(np.int64), N_ANG - 1)
    return rb * N_ANG + ab


def features(q: np.ndarray, K: np.ndarray) -> np.ndarray:
    """feat[k, b] = log(1 + mean of K_k over the pixels of bin b) (0 for empty bins)."""
    bins = feature_bins(q)
    K = np.asarray(K, dtype=np.float64)
    out = np.zeros((K.shape[0], N_FEAT))
    for b in range(N_FEAT):
        sel = bins == b
        n = int(sel.sum())
        if n:
            out[:, b] = np.log1p(K[:, sel].sum(axis=1) / n)
    return out


# ----------------------------------------------------------------------------
# MLP: x -> GELU(x W1 + b1) -> GELU(. W2 + b2) -> GELU(. W3 + b3) -> . W4 + b4
# params: list [W1, b1, W2, b2, W3, b3, W4, b4]; W_l has shape [in, out]
# ----------------------------------------------------------------------------

def gelu(x):
    from scipy.special import erf
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def bf16_round(x):
    """Nearest BF16 value of every element (ties to even), taken from its FP32
    value: the rounding the library documents for the operands of the MLP's
    matrix products (its activations are FP32). BF16 keeps the sign, the 8
    exponent bits and the top 7 fraction bits of an FP32 number."""
    x32 = np.ascontiguousarray(x, dtype=np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    keep = (u + 0x7FFF + ((u >> 16) & 1)) >> 16  # round half to even on the dropped 16 bits
    return ((keep << 16) & 0xFFFFFFFF).astype(np.uint32).view(np.float32).astype(np.float64)


def _same(x):
    return x


def mlp_forward(params, X, operand=_same):
    """Returns (logits, cache) with cache = pre-activations and layer inputs.
    operand: applied to both operands of every matrix product (bf16_round for
    the library's documented BF16 products; the identity by default)."""
    h = np.asarray(X, dtype=np.float64)
    ins, pres = [], []
    n_layers = len(params) // 2
    for l in range(n_layers):
        W, b = params[2 * l], params[2 * l + 1]
        ins.append(h)
        a = operand(h) @ operand(W) + b
        pres.append(a)
        h = gelu(a) if l < n_layers - 1 else a
    return h, (ins, pres)


def log_softmax(z):
    m = z.max(axis=1, keepdims=True)
    return z - (m + np.log(np.exp(z - m).sum(axis=1, keepdims=True)))


def soft_ce_loss(z, T):
    """-mean_k sum_j T_kj log softmax(z_k)_j with dense targets T [B, n_out]."""
    return float(-(T * log_softmax(z)).sum() / z.shape[0])


def mlp_loss_grads(params, X, T, operand=_same):
    """Loss and gradients (same order as params) by backpropagation; operand
    as in mlp_forward, applied to the operands of the backward products too."""
    z, (ins, pres) = mlp_forward(params, X, operand)
    B = z.shape[0]
    loss = soft_ce_loss(z, T)
    p = np.exp(log_softmax(z))
    g = (p * T.sum(axis=1, keepdims=True) - T) / B  # d loss / d z
    grads = [None] * len(params)
    n_layers = len(params) // 2
    for l in range(n_layers - 1, -1, -1):
        W = params[2 * l]
        grads[2 * l] = operand(ins[l]).T @ operand(g)
        grads[2 * l + 1] = g.sum(axis=0)
        if l > 0:
            g = (operand(g) @ operand(W).T) * gelu_grad(pres[l - 1])
    return loss, grads


def adam_step(params, grads, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (bias-corrected), in place; t counts from 1."""
    for i in range(len(params)):
        m[i] = b1 * m[i] + (1 - b1) * grads[i]
        v[i] = b2 * v[i] + (1 - b2) * grads[i] * grads[i]
        mh = m[i] / (1 - b1 ** t)
        vh = v[i] / (1 - b2 ** t)
        params[i] -= lr * mh / (np.sqrt(vh) + eps)


def soft_targets(P_dense: np.ndarray, R: int):
    """Top-R responsibilities of each frame (columns of P [n_rot, n_data]),
    renormalised: (idx [n_data, R], prob [n_data, R])."""
    idx = np.argsort(-P_dense, axis=0, kind="stable")[:R].T
    prob = np.take_along_axis(P_dense.T, idx, axis=1)
    prob = prob / prob.sum(axis=1, keepdims=True)
    return idx, prob


def dense_targets(idx, prob, n_out):
    T = np.zeros((idx.shape[0], n_out))
    np.put_along_axis(T, idx, prob, axis=1)
    return T


# ----------------------------------------------------------------------------
# top-M and the sparse Maximize
# ----------------------------------------------------------------------------

def topm(logits: np.ndarray, M: int) -> np.ndarray:
    """The M largest logits of each row, as a sorted index set [B, M]
    (ties broken towards the lower index)."""
    order = np.argsort(-logits, axis=1, kind="stable")[:, :M]
    return np.sort(order, axis=1)


def merge_candidates(first: np.ndarray, rest: np.ndarray, M: int) -> np.ndarray:
    """Candidate sets from two ranked lists per frame: every entry of `first`
    (the dense E-step's top R, distinct), then the entries of `rest` (the
    network's top list) not already taken, in order, until M: [B, M]."""
    out = np.empty((first.shape[0], M), dtype=np.int64)
    for k in range(first.shape[0]):
        row = list(first[k][:M])
        seen = set(row)
        for c in rest[k]:
            if len(row) == M:
                break
            if c not in seen:
                row.append(c)
                seen.add(c)
        assert len(row) == M, "rest too short"
        out[k] = row
    return out


def sparse_estep(S: np.ndarray, cand: np.ndarray):
    """Eq. 2.4 over candidate sets. S: dense scores [n_rot, n_data];
    cand [n_data, M]. Returns (P_c [n_data, M], lse_c [n_data])."""
    Sc = np.take_along_axis(S.T, cand, axis=1)
    m = Sc.max(axis=1, keepdims=True)
    lse = m[:, 0] + np.log(np.exp(Sc - m).sum(axis=1))
    return np.exp(Sc - lse[:, None]), lse


def sparse_mstep(P_c: np.ndarray, cand: np.ndarray, K: np.ndarray, n_rot: int):
    """Eq. 2.11 over candidate sets: Num [n_rot, n_pix], den [n_rot]."""
    K = np.asarray(K, dtype=np.float64)
    Num = np.zeros((n_rot, K.shape[1]))
    den = np.zeros(n_rot)
    for k in range(cand.shape[0]):
        for m in range(cand.shape[1]):
            j = cand[k, m]
            Num[j] += P_c[k, m] * K[k]
            den[j] += P_c[k, m]
    return Num, den


def missed_mass(P_dense: np.ndarray, cand: np.ndarray) -> np.ndarray:
    """1 - sum_{j in C_k} P_jk of the dense responsibilities, per frame."""
    return 1.0 - np.take_along_axis(P_dense.T, cand, axis=1).sum(axis=1)
