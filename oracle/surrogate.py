"""Learned surrogate of the IC activation frequencies -- fp64 CPU oracle, TEST INFRASTRUCTURE ONLY.

The paper has no learned component; this network exists to screen candidate
seeds in greedy influence maximisation (Sec. 2 "Influence Maximization"), while
the exact Monte Carlo simulator makes every decision.  It maps a seed set S to a
prediction of every node's activation frequency under IC (the per-node counts
of the paper's activation heatmap, Sec. 4 "Visualizations", divided by the
trial count).

Definition (both the oracle and the GPU follow it; hidden width H = 64, input
width D0 = 16, three layers):

  q_e      = fp32(thr_e) * 2^-32 for the IC threshold thr_e of edge e
             (thr_e = floor(p_e * 2^32), p_e = 1 -> 1.0): the live probability
  x_v      = bf16([s_v, ln(1 + indeg v), ln(1 + outdeg v), 0 * 13])
  a^l_v    = bf16( sum over in-edges e = (u -> v) of q_e * h^{l-1}_u )
  z^l_v    = W_s^l h^{l-1}_v + W_n^l a^l_v + b^l                      l = 1, 2, 3
  h^l_v    = bf16(relu(z^l_v)),   h^0 = x
  o_v      = w_o . h^3_v + b_o
  yhat_v   = s_v + (1 - s_v) * sigmoid(o_v)
  loss     = mean over v of (yhat_v - y_v)^2

Weights are held as fp32 masters; the matrices W_s, W_n are used as their
bf16 roundings (tensor-core operands: bf16 weights, fp32 accumulation), the
biases b^l, w_o and b_o as fp32.  Backward, with the same rounding points as the
tensor-core kernels (their operands are bf16):

  g_v      = d loss / d o_v = (2/n) (yhat_v - y_v) (1 - s_v) sig(o_v)(1 - sig(o_v))
  dh^3_v   = g_v w_o
  dz^l     = dh^l * [h^l > 0];  e^l = bf16(dz^l)
  dW_s^l   = sum_v e^l_v (h^{l-1}_v)^T,  dW_n^l = sum_v e^l_v (a^l_v)^T,  db^l = sum_v dz^l_v
  dh^{l-1}_v = W_s^{lT} e^l_v + sum over out-edges e = (v -> w) of q_e W_n^{lT} e^l_w     (l > 1)

Screening score of candidate c for seed set S (first-order gain of the
predicted spread P = sum_v yhat_v when c joins S): the same backward with
g_v = (1 - s_v) sig'(o_v), carried down to the seed-indicator input:
  score_c = (1 - s_c)(1 - sig(o_c)) + [W_s^{1T} e^1_c]_0 + sum over out-edges (c -> w) of q [W_n^{1T} e^1_w]_0

One-hop screening score (needs only the forward): with yhat = yhat(S),
  onehop_c = (1 - yhat_c) (1 + sum over out-edges (c -> w) of q (1 - yhat_w))

Parameters travel as one fp32 vector in the order
  [W_s^1 (64x16), W_n^1 (64x16), b^1, W_s^2 (64x64), W_n^2, b^2, W_s^3, W_n^3, b^3, w_o (64), b_o]
(matrices row-major, out x in): 18,689 values.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

H = 64
D0 = 16
LAYERS = 3
DIMS = [D0, H, H]


def param_shapes():
    shapes = []
    for l in range(LAYERS):
        shapes += [(f"Ws{l + 1}", (H, DIMS[l])), (f"Wn{l + 1}", (H, DIMS[l])), (f"b{l + 1}", (H,))]
    shapes += [("wo", (H,)), ("bo", (1,))]
    return shapes


N_PARAMS = sum(int(np.prod(s)) for _, s in param_shapes())


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64).ravel()
    assert flat.size == N_PARAMS
    out, o = {}, 0
    for name, shape in param_shapes():
        k = int(np.prod(shape))
        out[name] = flat[o:o + k].reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in param_shapes()])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), via fp32; values returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def edge_q(ic_prob):
    """Live probability of every edge as the fp32 value fp32(thr) * 2^-32 (thr as defined for IC)."""
    p = np.asarray(ic_prob, dtype=np.float32).astype(np.float64)
    thr = np.floor(p * 4294967296.0)
    q = thr.astype(np.float32).astype(np.float64) * 2.0 ** -32
    return np.where(p == 1.0, 1.0, q)


class Graph:
    """The in- and out-aggregation operators of a CSR graph with edge weights q."""

    def __init__(self, g, ic_prob):
        self.n = int(g.n)
        src = np.repeat(np.arange(self.n), np.diff(g.row_ptr))
        dst = np.asarray(g.col, dtype=np.int64)
        q = edge_q(ic_prob)
        # A_in[v, u] = sum of q over edges u -> v ;  A_out = A_in^T
        self.A_in = sp.csr_matrix((q, (dst, src)), shape=(self.n, self.n))
        self.A_out = self.A_in.T.tocsr()
        indeg = np.bincount(dst, minlength=self.n)
        outdeg = np.diff(g.row_ptr)
        self.x_rest = np.zeros((self.n, D0))
        self.x_rest[:, 1] = np.log1p(indeg)
        self.x_rest[:, 2] = np.log1p(outdeg)


def seed_indicator(n, seeds):
    """0/1 vector of the seed set; a float array of length n is taken as the indicator itself
    (the continuous extension the finite-difference pins differentiate)."""
    arr = np.asarray(seeds)
    if arr.dtype.kind == "f" and arr.shape == (n,):
        return arr.astype(np.float64)
    s = np.zeros(n)
    s[arr.astype(np.int64)] = 1.0
    return s


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def forward(flat, G: Graph, seeds):
    P = {k: (bf16(v) if k.startswith(("Ws", "Wn")) else v) for k, v in unpack(flat).items()}
    s = seed_indicator(G.n, seeds)
    x = G.x_rest.copy()
    x[:, 0] = s
    h = [bf16(x)]
    a = [None]
    for l in range(1, LAYERS + 1):
        al = bf16(G.A_in @ h[l - 1])
        z = h[l - 1] @ P[f"Ws{l}"].T + al @ P[f"Wn{l}"].T + P[f"b{l}"]
        a.append(al)
        h.append(bf16(np.maximum(z, 0.0)))
    o = h[LAYERS] @ P["wo"] + P["bo"][0]
    sig = sigmoid(o)
    yhat = s + (1.0 - s) * sig
    return {"P": P, "s": s, "h": h, "a": a, "o": o, "sig": sig, "yhat": yhat}


def backward(cache, G: Graph, g, want_input_grad=False):
    """Parameter gradients (flat, fp64) for head gradient g = d objective / d o; optionally d/ds."""
    P, h, a = cache["P"], cache["h"], cache["a"]
    grads = {"wo": h[LAYERS].T @ g, "bo": np.array([g.sum()])}
    dh = np.outer(g, P["wo"])
    dx0 = None
    for l in range(LAYERS, 0, -1):
        dz = dh * (h[l] > 0)
        e = bf16(dz)
        grads[f"Ws{l}"] = e.T @ h[l - 1]
        grads[f"Wn{l}"] = e.T @ a[l]
        grads[f"b{l}"] = dz.sum(axis=0)
        if l > 1 or want_input_grad:
            da = e @ P[f"Wn{l}"]
            dprev = e @ P[f"Ws{l}"] + G.A_out @ da
            if l > 1:
                dh = dprev
            else:
                dx0 = dprev
    return pack(grads), dx0


def loss_and_grad(flat, G: Graph, seeds, y):
    c = forward(flat, G, seeds)
    n = G.n
    s, sig, yhat = c["s"], c["sig"], c["yhat"]
    y = np.asarray(y, dtype=np.float64)
    loss = float(np.mean((yhat - y) ** 2))
    g = (2.0 / n) * (yhat - y) * (1.0 - s) * sig * (1.0 - sig)
    grad, _ = backward(c, G, g)
    return loss, grad, c


def screen_scores(flat, G: Graph, seeds):
    c = forward(flat, G, seeds)
    s, sig = c["s"], c["sig"]
    g = (1.0 - s) * sig * (1.0 - sig)
    _, dx0 = backward(c, G, g, want_input_grad=True)
    return (1.0 - s) * (1.0 - sig) + dx0[:, 0], c


def onehop_scores(flat, G: Graph, seeds):
    """Expected one-hop gain under yhat = yhat(S): (1 - yhat_c)(1 + sum over out-edges (c -> w) of q (1 - yhat_w))."""
    c = forward(flat, G, seeds)
    y = c["yhat"]
    return (1.0 - y) * (1.0 + G.A_out @ (1.0 - y)), c


def adam(flat, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba 2015) on the fp32 master weights; t counts from 1."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
