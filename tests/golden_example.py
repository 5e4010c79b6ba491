"""Reads the hand-worked example of tests/golden/unit_tet_worked_example.txt
into problems (input handling only)."""
import os

import numpy as np

from paper_1005_3158_gb300 import meshgen as mg

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "unit_tet_worked_example.txt")


def load():
    kv = {}
    with open(PATH) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if "=" in line:
                k, v = line.split("=", 1)
                kv[k.strip()] = v.strip()
    return kv


def vec(s):
    return np.array([float(x) for x in s.split()])


def problem(kv, case):
    xyz = np.array([vec(r) for r in kv["nodes"].split(";")])
    h, t_inf, q = vec(kv["face_h_tinf_q"])
    return mg.Problem(xyz=xyz, tets=vec(kv["tet"]).astype(np.int32).reshape(1, 4),
                      mat=np.zeros(1, np.int32),
                      materials=vec(kv[f"material_{case}"]).reshape(1, 6),
                      faces=vec(kv["face"]).astype(np.int32).reshape(1, 3),
                      h=np.array([h]), t_inf=np.array([t_inf]), q=np.array([q]),
                      T0=vec(kv["T0"]), name=f"unit_tet_{case}")
