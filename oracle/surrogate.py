"""Plain CPU oracle of the learned mesh surrogate (test infrastructure only).

Only the tests and ``bench.py``'s CPU-baseline leg may import this module;
the product library never does.  It shares no code with the CUDA path.

The surrogate is a small message-passing network on the node graph of the
linear-tet mesh.  It maps the nodal state of the explicit enthalpy scheme at
step n (the temperature T(E) of Eqs. 5 and 11, the latent state, the
material) to the enthalpy content after ``MACRO`` = 16 explicit steps
(Eq. 14), so that one evaluation replaces 16 steps bounded by the explicit
stability limit (Eq. 13).  The paper has no surrogate: what follows is this
build's definition, written out once here and once in the CUDA kernels.

Graph.  Nodes are the mesh nodes; an edge joins two nodes of one tet.  Its
weight is the assembled conductance W_ij = -sum_e K^e_ab over the tets that
hold the edge (Eq. 9; the K^e of the oracle), so that for a field T
    sum_j W_ij (T_j - T_i) = -(K T)_i
is the conduction part of the explicit residual (zero row sums of K^e).
Per node: s_i = dt / C_i (C_i the row-sum lumped capacity), the Robin
boundary of Eq. 4 lumped to its row sums, hA_i = sum_f h_f A_f / 3 and
g_i = sum_f A_f (h_f T_inf,f - q_f) / 3.

Features x_i (NF = 16 channels, T_C = 600 K, T_S = 300 K):
    0  (T_i - T_C) / T_S                      temperature, T = T(E) (Eqs. 5, 11)
    1  f_i = (E_i - C_i T_i) / Lc_i            liquid fraction (0 without latent heat)
    2  Lc_i / (C_i T_S)                        latent capacity
    3  16 s_i hA_i                             Robin strength over 16 steps
    4  16 s_i (g_i - hA_i T_i) / T_S           Robin drive over 16 steps
    5  16 s_i sum_j W_ij (T_j - T_i) / T_S     16 x the conduction change of one step
    6  16 s_i sum_j W_ij (f_j - f_i)           the same for the liquid fraction
    7  1
    8  (T_i - Ts_i) / T_S   (phase-change nodes, else 0)
    9  (T_i - Tl_i) / T_S   (phase-change nodes, else 0)
    10 16 s_i sum_j W_ij                        coupling strength
    11-15 0

Network (HID = 64 hidden, MSG = 32 message channels, LAYERS = 3), weights
in the PyTorch Linear convention y = W x + b:
    h0  = relu(W_in x + b_in)                                   16 -> 64
    for l = 1..3:
        phi_l = relu(P_l h_{l-1} + p_l)                         64 -> 32
        m_l,i = s_i sum_j W_ij (phi_l,j - phi_l,i)              graph message
        r_l   = relu(U_l [h_{l-1}; m_l] + u_l)                  96 -> 64
        h_l   = h_{l-1} + r_l
    z   = relu(D1 h3 + d1)                                      64 -> 64
    y   = d2 . z + d2b                                          64 -> 1
    E_out,i = E_i + C_i Y_S y_i        (Y_S = 10 K)

Precision (``emulate=True``, the CUDA path's arithmetic): weights, x, h,
phi, m, dz-type GEMM operands are rounded to bfloat16 where the kernels
round them; every product is formed from those bf16 values and accumulated
in FP32 or better; W_ij, s_i, the message sums, z, y and E are FP32.
``emulate=False`` runs the same steps in FP64 with no rounding (for the
finite-difference pins).

Training: loss = mean_i (y_i - y*_i)^2 with y*_i = (E*_i - E_i) / (C_i Y_S),
E* the state after 16 explicit steps; gradients by the chain rule (below);
Adam (Kingma and Ba, 2015) on FP32 master weights.
"""
from __future__ import annotations

import numpy as np

from .oracle import OracleProblem, T_from_E

NF, HID, MSG, LAYERS, MACRO = 16, 64, 32, 3, 16
T_C, T_S, Y_S = 600.0, 300.0, 10.0

# flat parameter vector: (name, shape) in order
PARAM_SHAPES = [("W_in", (HID, NF)), ("b_in", (HID,))]
for _l in range(1, LAYERS + 1):
    PARAM_SHAPES += [(f"P{_l}", (MSG, HID)), (f"p{_l}", (MSG,)),
                     (f"U{_l}", (HID, HID + MSG)), (f"u{_l}", (HID,))]
PARAM_SHAPES += [("D1", (HID, HID)), ("d1", (HID,)), ("d2", (HID,)), ("d2b", (1,))]
N_PARAMS = int(sum(int(np.prod(s)) for _, s in PARAM_SHAPES))


def unpack(theta):
    """Flat vector -> dict of named views."""
    out, k = {}, 0
    for name, shape in PARAM_SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    r = ((x + np.uint32(0x7FFF) + ((x >> np.uint32(16)) & np.uint32(1)))
         & np.uint32(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32)


class SurrogateGraph:
    """The surrogate's graph and node data for one problem and time step,
    in the problem's own node order."""

    def __init__(self, prob, dt):
        o = OracleProblem(prob, dirichlet=False)
        n = prob.n_nodes
        self.n = n
        self.dt = float(dt)
        C, _, Lc = o.lumped()
        self.C, self.Lc = C, Lc
        # assembled conductances W_ij = -sum_e K^e_ab over the tets holding (i, j)
        rows, cols, vals = [], [], []
        for e in range(prob.n_tets):
            nodes, K, _ = o.element(e)
            for a in range(4):
                for b in range(4):
                    if a != b:
                        rows.append(nodes[a])
                        cols.append(nodes[b])
                        vals.append(-K[a, b])
        rows, cols, vals = np.array(rows, np.int64), np.array(cols, np.int64), np.array(vals)
        key = rows * n + cols
        uk, inv = np.unique(key, return_inverse=True)
        W = np.zeros(uk.shape[0])
        np.add.at(W, inv, vals)
        self.ei, self.ej, self.W = uk // n, uk % n, W      # directed edges, sorted by (i, j)
        self.s = self.dt / C
        self.wsum = np.zeros(n)
        np.add.at(self.wsum, self.ei, self.W)
        # phase-change range of each node (one per node, Section 3 data)
        self.Ts = np.zeros(n)
        self.Tl = np.zeros(n)
        for mt, m in enumerate(prob.materials):
            if m[3] > 0:
                nd = prob.tets[prob.mat == mt].ravel()
                self.Ts[nd], self.Tl[nd] = m[4], m[5]
        # Robin faces of Eq. 4 lumped to their row sums
        self.hA = np.zeros(n)
        self.g = np.zeros(n)
        x = prob.xyz
        for f in range(prob.faces.shape[0]):
            a, b, c = prob.faces[f]
            A = 0.5 * np.linalg.norm(np.cross(x[b] - x[a], x[c] - x[a]))
            for v in (a, b, c):
                self.hA[v] += prob.h[f] * A / 3.0
                self.g[v] += A * (prob.h[f] * prob.t_inf[f] - prob.q[f]) / 3.0


def temperature(g, E):
    """T(E) of every node: the oracle's exact inverse of E(T) = C T + Lc f_l(T)
    (Eqs. 5, 11)."""
    E = np.asarray(E, np.float64)
    return np.array([T_from_E(E[i], g.C[i], g.Lc[i], g.Ts[i], g.Tl[i]) for i in range(g.n)])


def _edge_sum(g, w, v, n):
    """sum_j w_ij v_j over the directed edges (i, j), per node i."""
    out = np.zeros((n,) + v.shape[1:], dtype=np.float64)
    np.add.at(out, g.ei, (w.reshape((-1,) + (1,) * (v.ndim - 1)) * v[g.ej]))
    return out


def features(g, E, emulate=True):
    """x [n, NF] from the enthalpy contents E [n] (FP32 when emulating)."""
    Ed = np.asarray(E, np.float64)
    if emulate:
        Ed = np.asarray(E, np.float32).astype(np.float64)
    T = temperature(g, Ed)
    f = np.where(g.Lc > 0, (Ed - g.C * T) / np.where(g.Lc > 0, g.Lc, 1.0), 0.0)
    W = g.W.astype(np.float32).astype(np.float64) if emulate else g.W
    pc = g.Lc > 0
    x = np.zeros((g.n, NF))
    x[:, 0] = (T - T_C) / T_S
    x[:, 1] = f
    x[:, 2] = g.Lc / (g.C * T_S)
    x[:, 3] = MACRO * g.s * g.hA
    x[:, 4] = MACRO * g.s * (g.g - g.hA * T) / T_S
    x[:, 5] = MACRO * g.s * (_edge_sum(g, W, T, g.n) - _edge_sum(g, W, np.ones(g.n), g.n) * T) / T_S
    x[:, 6] = MACRO * g.s * (_edge_sum(g, W, f, g.n) - _edge_sum(g, W, np.ones(g.n), g.n) * f)
    x[:, 7] = 1.0
    x[:, 8] = np.where(pc, (T - g.Ts) / T_S, 0.0)
    x[:, 9] = np.where(pc, (T - g.Tl) / T_S, 0.0)
    x[:, 10] = MACRO * g.s * _edge_sum(g, W, np.ones(g.n), g.n)
    return x.astype(np.float32) if emulate else x


def _message(g, W, phi):
    """m_i = s_i sum_j W_ij (phi_j - phi_i)."""
    acc = _edge_sum(g, W, phi, g.n) - _edge_sum(g, W, np.ones(g.n), g.n)[:, None] * phi
    return g.s[:, None] * acc


def forward(theta, g, E, emulate=True):
    """Returns (E_out, saved) with y and every intermediate the backward
    pass needs."""
    R = bf16 if emulate else (lambda a: np.asarray(a, np.float64))
    F = (lambda a: np.asarray(a, np.float32)) if emulate else (lambda a: np.asarray(a, np.float64))
    p = unpack(np.asarray(theta, np.float32 if emulate else np.float64))
    W = g.W.astype(np.float32).astype(np.float64) if emulate else g.W
    x = R(features(g, E, emulate))
    sv = {"x": x}

    def lin(inp, Wm, b):     # products of the (rounded) operands, accumulated in FP64
        return inp.astype(np.float64) @ R(Wm).astype(np.float64).T + np.asarray(b, np.float64)

    h = R(np.maximum(lin(x, p["W_in"], p["b_in"]), 0.0))
    sv["h0"] = h
    for l in range(1, LAYERS + 1):
        phi = R(np.maximum(lin(h, p[f"P{l}"], p[f"p{l}"]), 0.0))
        m = R(F(_message(g, W, phi.astype(np.float64))))
        r = F(np.maximum(lin(np.concatenate([h, m], axis=1), p[f"U{l}"], p[f"u{l}"]), 0.0))
        sv[f"phi{l}"], sv[f"m{l}"], sv[f"r{l}"] = phi, m, R(r)
        h = R(F(h.astype(np.float64) + r))
        sv[f"h{l}"] = h
    z = F(np.maximum(lin(h, p["D1"], p["d1"]), 0.0))
    y = F(z.astype(np.float64) @ R(p["d2"]).astype(np.float64) + float(p["d2b"][0]))
    sv["z"], sv["y"] = z, y
    E_out = F(np.asarray(E, np.float64) + g.C * Y_S * y.astype(np.float64))
    return E_out, sv


def target(g, E, E_star, emulate=True):
    """y* = (E* - E) / (C Y_S)."""
    F = np.float32 if emulate else np.float64
    return ((np.asarray(E_star, np.float64) - np.asarray(E, np.float64)) / (g.C * Y_S)).astype(F)


def backward(theta, g, sv, y_star, emulate=True):
    """Loss and its gradient with respect to the flat parameter vector, for
    the forward pass saved in sv.  Bias gradients are sums of the rounded
    output gradients (the kernels form them in the same products as the
    weight gradients)."""
    R = bf16 if emulate else (lambda a: np.asarray(a, np.float64))
    F = (lambda a: np.asarray(a, np.float32)) if emulate else (lambda a: np.asarray(a, np.float64))
    p = unpack(np.asarray(theta, np.float32 if emulate else np.float64))
    W = g.W.astype(np.float32).astype(np.float64) if emulate else g.W
    n = g.n
    grad = {name: np.zeros(shape) for name, shape in PARAM_SHAPES}
    y = sv["y"].astype(np.float64)
    diff = y - np.asarray(y_star, np.float64)
    loss = float(np.mean(diff * diff))
    dy = F(2.0 * diff / n).astype(np.float64)
    z = sv["z"].astype(np.float64)

    def wgrad(dout, inp):        # sum over nodes of dout^T inp, operands rounded
        return R(dout).astype(np.float64).T @ inp.astype(np.float64)

    def bgrad(dout):
        return R(dout).astype(np.float64).sum(axis=0)

    def back(dout, Wm):          # dout @ W, operands rounded
        return R(dout).astype(np.float64) @ R(Wm).astype(np.float64)

    grad["d2"] = F(z.T @ dy)
    grad["d2b"] = F(np.array([dy.sum()]))
    dz = F(dy[:, None] * R(p["d2"]).astype(np.float64)[None, :] * (z > 0))
    h3 = sv[f"h{LAYERS}"]
    grad["D1"], grad["d1"] = wgrad(dz, h3), bgrad(dz)
    dh = F(back(dz, p["D1"]))
    for l in range(LAYERS, 0, -1):
        hin = sv[f"h{l - 1}"]
        xin = np.concatenate([hin, sv[f"m{l}"]], axis=1)
        du = F(dh.astype(np.float64) * (sv[f"r{l}"] > 0))
        grad[f"U{l}"], grad[f"u{l}"] = wgrad(du, xin), bgrad(du)
        dX = F(back(du, p[f"U{l}"]))
        dh_dir = F(dh.astype(np.float64) + dX[:, :HID])
        gm = F(g.s[:, None] * dX[:, HID:].astype(np.float64))
        # adjoint of m_i = s_i sum_j W_ij (phi_j - phi_i) for symmetric W:
        # dphi_j = sum_i W_ji (gm_i - gm_j), gm = s dm
        dphi = F(_edge_sum(g, W, gm.astype(np.float64), n)
                 - _edge_sum(g, W, np.ones(n), n)[:, None] * gm)
        dpre = F(dphi.astype(np.float64) * (sv[f"phi{l}"] > 0))
        grad[f"P{l}"], grad[f"p{l}"] = wgrad(dpre, hin), bgrad(dpre)
        dh = F(dh_dir.astype(np.float64) + back(dpre, p[f"P{l}"]))
    d0 = F(dh.astype(np.float64) * (sv["h0"] > 0))
    grad["W_in"], grad["b_in"] = wgrad(d0, sv["x"]), bgrad(d0)
    flat = np.concatenate([np.asarray(grad[name], np.float64).ravel() for name, _ in PARAM_SHAPES])
    return loss, (flat.astype(np.float32) if emulate else flat)


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015, Algorithm 1), FP32; t counts from
    1.  Returns the new (theta, m, v)."""
    th, gr = np.asarray(theta, np.float32), np.asarray(grad, np.float32)
    m = np.float32(b1) * np.asarray(m, np.float32) + np.float32(1 - b1) * gr
    v = np.float32(b2) * np.asarray(v, np.float32) + np.float32(1 - b2) * gr * gr
    mh = m / np.float32(1 - b1 ** t)
    vh = v / np.float32(1 - b2 ** t)
    th = th - np.float32(lr) * mh / (np.sqrt(vh) + np.float32(eps))
    return th.astype(np.float32), m.astype(np.float32), v.astype(np.float32)
