"""Pins of the surrogate oracle (oracle/surrogate.py) against things other
than itself.

* bf16 rounding equals torch's float32 -> bfloat16 conversion (library).
* The graph's conduction message equals the FE oracle's explicit residual
  (Eq. 14 with the K^e of Eq. 9, faces off): s_i sum_j W_ij (T_j - T_i)
  = dt R_i / C_i for a random field; it vanishes at interior nodes for a
  linear field (patch test).
* The lumped Robin terms equal the FE oracle's face residual for a uniform
  field (the consistent face matrix of Eq. 4 has row sums h A / 3).
* The liquid-fraction feature equals the FE oracle's f_l(T) at mushy nodes.
* With hand-set weights that route feature 5 through the network, the
  output is exactly 16 times the FE oracle's one-step conduction change.
* The vectorised forward pass equals a brute-force per-node loop.
* Gradients equal central finite differences of the FP64 loss.
* Adam equals torch.optim.Adam (library) over several steps.
"""
import numpy as np
import pytest

import oracle
from oracle import surrogate as sg
from paper_1005_3158_gb300 import meshgen as mg


def _small(seed=5):
    return mg.random_small(seed, nx=3, ny=3, nz=2)


def test_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-20, 100),
                        rng.normal(0, 1e20, 100),
                        1.0 + np.arange(-8, 9) * 2.0 ** -9]).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(sg.bf16(a), ref)


def test_conduction_message_is_the_explicit_residual():
    p = _small()
    dt = 0.37
    g = sg.SurrogateGraph(p, dt)
    o = oracle.OracleProblem(p, faces=False, dirichlet=False)
    T = mg.rng_of(3).uniform(300, 1000, size=p.n_nodes)
    R, _ = o.residual(T)
    ones = np.ones(p.n_nodes)
    msg = g.s * (sg._edge_sum(g, g.W, T, g.n) - sg._edge_sum(g, g.W, ones, g.n) * T)
    assert np.allclose(msg, dt * R / g.C, rtol=1e-11, atol=1e-11 * np.abs(dt * R / g.C).max())
    # symmetric weights
    key = dict(zip(zip(g.ei.tolist(), g.ej.tolist()), g.W.tolist()))
    assert all(abs(w - key[(j, i)]) <= 1e-12 * abs(w) for (i, j), w in key.items())


def test_patch_test_linear_field():
    p = mg.unit_cube(4, jitter=0.2)
    g = sg.SurrogateGraph(p, 1.0)
    T = 500.0 + 30.0 * p.xyz[:, 0] - 20.0 * p.xyz[:, 1] + 7.0 * p.xyz[:, 2]
    lap = sg._edge_sum(g, g.W, T, g.n) - sg._edge_sum(g, g.W, np.ones(g.n), g.n) * T
    inner = np.all((p.xyz > 1e-9) & (p.xyz < 1 - 1e-9), axis=1)
    assert inner.sum() > 10
    assert np.abs(lap[inner]).max() <= 1e-9 * 150 * 30


def test_robin_lumping_is_the_face_residual_row_sum():
    p = _small(7)
    g = sg.SurrogateGraph(p, 1.0)
    o = oracle.OracleProblem(p, dirichlet=False)
    Tu = 612.5
    R, _ = o.residual(np.full(p.n_nodes, Tu))
    assert np.allclose(g.g - g.hA * Tu, R, rtol=1e-10, atol=1e-10 * np.abs(R).max())


def test_liquid_fraction_feature():
    p = mg.unit_cube(3)
    g = sg.SurrogateGraph(p, 1.0)
    rng = mg.rng_of(9)
    T = rng.uniform(830.0, 900.0, size=p.n_nodes)      # mushy (821-913 K)
    E = np.array([oracle.E_from_T(T[i], g.C[i], g.Lc[i], 821.0, 913.0) for i in range(g.n)])
    x = sg.features(g, E, emulate=False)
    fl = np.array([oracle.liquid_fraction(t, 821.0, 913.0) for t in T])
    assert np.allclose(x[:, 1], fl, atol=1e-12)
    assert np.allclose(x[:, 0], (T - sg.T_C) / sg.T_S, atol=1e-12)
    assert np.allclose(x[:, 8], (T - 821.0) / sg.T_S, atol=1e-12)


def _routing_params():
    """Weights that carry feature 5 (16 x the one-step conduction change)
    through the network unchanged: h0 = (relu(x5), relu(-x5), 0...), every
    layer adds relu(u) = 0, z = h3, y = 30 (z0 - z1) = 30 x5."""
    th = np.zeros(sg.N_PARAMS)
    p = sg.unpack(th)
    p["W_in"][0, 5], p["W_in"][1, 5] = 1.0, -1.0
    p["D1"][0, 0], p["D1"][1, 1] = 1.0, 1.0
    p["d2"][0], p["d2"][1] = sg.T_S / sg.Y_S, -sg.T_S / sg.Y_S
    return th


def test_routed_output_is_sixteen_explicit_conduction_steps():
    p = _small(11)
    o = oracle.OracleProblem(p, faces=False, dirichlet=False)
    o.set_temperature(p.T0)
    dt = 0.5 * o.stable_dt()
    E0 = o.enthalpy()
    o.step(1, dt)
    dE1 = o.enthalpy() - E0
    g = sg.SurrogateGraph(p, dt)
    E_out, _ = sg.forward(_routing_params(), g, E0, emulate=False)
    assert np.allclose(E_out - E0, 16.0 * dE1, rtol=1e-9, atol=1e-9 * np.abs(dE1).max())


def _brute_forward(theta, g, x):
    """Per-node loops, FP64, written without the oracle's vectorisation."""
    p = sg.unpack(np.asarray(theta, np.float64))
    n = g.n
    nbr = [[] for _ in range(n)]
    for i, j, w in zip(g.ei, g.ej, g.W):
        nbr[i].append((j, w))
    relu = lambda v: v if v > 0 else 0.0   # noqa: E731
    h = [[relu(sum(p["W_in"][c, k] * x[i, k] for k in range(sg.NF)) + p["b_in"][c])
          for c in range(sg.HID)] for i in range(n)]
    for l in range(1, sg.LAYERS + 1):
        P, pb, U, ub = p[f"P{l}"], p[f"p{l}"], p[f"U{l}"], p[f"u{l}"]
        phi = [[relu(sum(P[c, k] * h[i][k] for k in range(sg.HID)) + pb[c])
                for c in range(sg.MSG)] for i in range(n)]
        m = [[g.s[i] * sum(w * (phi[j][c] - phi[i][c]) for j, w in nbr[i])
              for c in range(sg.MSG)] for i in range(n)]
        new = []
        for i in range(n):
            inp = h[i] + m[i]
            new.append([h[i][c] + relu(sum(U[c, k] * inp[k] for k in range(sg.HID + sg.MSG))
                                       + ub[c]) for c in range(sg.HID)])
        h = new
    y = []
    for i in range(n):
        z = [relu(sum(p["D1"][c, k] * h[i][k] for k in range(sg.HID)) + p["d1"][c])
             for c in range(sg.HID)]
        y.append(sum(p["d2"][c] * z[c] for c in range(sg.HID)) + p["d2b"][0])
    return np.array(y)


def test_forward_equals_brute_force():
    p = mg.random_small(4, nx=2, ny=2, nz=1)
    g = sg.SurrogateGraph(p, 0.2)
    th = mg.surrogate_init(sg.PARAM_SHAPES, seed=1).astype(np.float64)
    th += mg.rng_of(2).normal(0, 0.05, size=th.shape)      # non-zero biases too
    E = mg.rng_of(3).uniform(2e5, 9e5, size=g.n) * g.C / 900.0
    _, sv = sg.forward(th, g, E, emulate=False)
    x = sg.features(g, E, emulate=False)
    assert np.allclose(sv["y"], _brute_forward(th, g, x), rtol=1e-10, atol=1e-12)


def test_gradient_equals_finite_differences():
    p = mg.random_small(8, nx=2, ny=1, nz=1)
    g = sg.SurrogateGraph(p, 0.3)
    rng = mg.rng_of(4)
    th = mg.surrogate_init(sg.PARAM_SHAPES, seed=3).astype(np.float64)
    th += rng.normal(0, 0.1, size=th.shape)
    E = rng.uniform(500, 950, size=g.n) * g.C
    y_star = rng.normal(0, 1, size=g.n)
    _, sv = sg.forward(th, g, E, emulate=False)
    loss, grad = sg.backward(th, g, sv, y_star, emulate=False)

    def L(t):
        _, s = sg.forward(t, g, E, emulate=False)
        return float(np.mean((s["y"] - y_star) ** 2))

    assert loss == pytest.approx(L(th), rel=1e-14)
    idx = np.concatenate([rng.choice(sg.N_PARAMS, 300, replace=False),
                          np.arange(sg.N_PARAMS - 130, sg.N_PARAMS)])
    eps = 1e-6
    fd = np.array([(L(th + eps * np.eye(1, sg.N_PARAMS, k)[0])
                    - L(th - eps * np.eye(1, sg.N_PARAMS, k)[0])) / (2 * eps) for k in idx])
    scale = np.abs(grad).max()
    assert np.abs(fd - grad[idx]).max() <= 1e-6 * scale
    assert np.count_nonzero(np.abs(grad[idx]) > 1e-6 * scale) > 100


def test_adam_equals_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    th = rng.normal(size=200).astype(np.float32)
    m = np.zeros(200, np.float32)
    v = np.zeros(200, np.float32)
    pt = torch.nn.Parameter(torch.from_numpy(th.copy()))
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for t in range(1, 6):
        gr = rng.normal(size=200).astype(np.float32)
        th, m, v = sg.adam(th, gr, m, v, t, 1e-3)
        pt.grad = torch.from_numpy(gr.copy())
        opt.step()
    assert np.allclose(th, pt.detach().numpy(), rtol=0, atol=2e-7)
