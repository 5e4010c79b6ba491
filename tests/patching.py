"""Patches for checking sampled outputs of a large mesh with the oracle.

patch(p, S) is the sub-problem of every tet and Robin face that touches the
nodes S.  A node of S has all of its elements, faces and lumped capacity in
it, so one explicit step of the patch from the same temperatures gives that
node exactly the value one step of the whole mesh gives it.  The other patch
nodes only supply temperatures.  Input handling only: no arithmetic of the
method lives here.
"""
import numpy as np

from paper_1005_3158_gb300 import meshgen as mg


def patch(p, S):
    """The sub-problem of every tet and Robin face touching the nodes S
    (node ids renumbered; returns the problem and the local ids of S)."""
    mark = np.zeros(p.n_nodes, bool)
    mark[S] = True
    tsel = mark[p.tets].any(axis=1)
    fsel = mark[p.faces].any(axis=1)
    tets, faces = p.tets[tsel], p.faces[fsel]
    used = np.unique(np.concatenate([tets.ravel(), faces.ravel()]))
    new = np.full(p.n_nodes, -1, np.int64)
    new[used] = np.arange(used.size)
    sub = mg.Problem(xyz=p.xyz[used], tets=new[tets].astype(np.int32), mat=p.mat[tsel],
                     materials=p.materials, faces=new[faces].astype(np.int32).reshape(-1, 3),
                     h=p.h[fsel], t_inf=p.t_inf[fsel], q=p.q[fsel], T0=p.T0[used])
    return sub, used, new[S]


def sample_nodes(p, T, rng, n_random=3000, n_each=300):
    """Random nodes, plus boundary, material-interface and mushy nodes."""
    S = [rng.choice(p.n_nodes, n_random, replace=False)]
    bnd = np.unique(p.faces)
    S.append(rng.choice(bnd, min(n_each, bnd.size), replace=False))
    mats = np.zeros((p.n_nodes, 2), bool)
    for m in (0, 1):
        mats[np.unique(p.tets[p.mat == m]), m] = True
    iface = np.flatnonzero(mats.all(axis=1))
    if iface.size:
        S.append(rng.choice(iface, min(n_each, iface.size), replace=False))
    lat = p.materials[:, 3] > 0
    Ts, Tl = p.materials[lat][0, 4], p.materials[lat][0, 5]
    mushy = np.flatnonzero((T > Ts) & (T < Tl))
    if mushy.size:
        S.append(rng.choice(mushy, min(n_each, mushy.size), replace=False))
    return np.unique(np.concatenate(S)), mushy.size
