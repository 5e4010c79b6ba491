"""Default element-block partition (host side, no GPU): with constant k
and the enthalpy formulation the automatic FP32 block size starts at 1,792
tets and shrinks until the largest block's shared memory leaves room for
four CTAs per SM; with staged conductances (512 threads) it stays 2,048."""
import numpy as np
import pytest

from paper_1005_3158_gb300 import meshgen as mg

fem = pytest.importorskip("paper_1005_3158_gb300.fem")

FOUR_CTA_SMEM = 57216   # bytes of dynamic shared memory per CTA for four per SM


def _smem_l2(m, real_size=4):
    """Dynamic shared memory of the L2-conductance block kernel for the
    largest block of m's plan: barriers and header, schedule chunk, slots,
    local node data (every part 16-byte aligned)."""
    b = m.plan("blocks").reshape(-1, 16)
    ngrp, nrounds, nint, nsh = b[:, 9], b[:, 14], b[:, 5], b[:, 7]
    ne_pad, nf_pad = b[:, 10], b[:, 11]
    a16 = lambda x: (int(x) + 15) // 16 * 16
    cw = int((((ngrp + 4) & ~3) + 16 * nrounds).max())
    slots = int((4 * ne_pad + 3 * nf_pad + 1).max())
    ls = (int((nint + nsh).max()) + 31) // 32 * 32
    slots = (max(slots, 2 * ls) + 3) & ~3
    return 96 + a16(cw * 4) + a16(slots * real_size) + a16(ls * (real_size + 5))


@pytest.mark.parametrize("make", [lambda: mg.flanged_casting(40, 40, 38),
                                  lambda: mg.block_with_cores(40)])
def test_auto_block_size_fits_four_ctas(make):
    p = make()
    with fem.Mesh(p, "fp32") as m:
        ne = m.plan("blocks").reshape(-1, 16)[:, 1]
        assert 1024 <= ne.max() <= 1792
        assert _smem_l2(m) <= FOUR_CTA_SMEM


def test_staged_conductances_keep_2048():
    p = mg.block_with_cores(30)
    with fem.Mesh(p, "fp32", threads=512) as m:
        ne = m.plan("blocks").reshape(-1, 16)[:, 1]
        assert ne.max() > 1792 and ne.max() <= 2048


def test_explicit_block_size_is_kept():
    p = mg.block_with_cores(30)
    with fem.Mesh(p, "fp32", block_elems=2560) as m:   # no automatic shrink
        ne = m.plan("blocks").reshape(-1, 16)[:, 1]
        assert ne.max() > 1792


def test_conductivity_tables_keep_the_l2_kernel_size():
    """k(T) reads the conductances from L2 like constant k, so it gets the
    same automatic block size (four CTAs per SM); the apparent capacity
    keeps them in shared memory (its element capacities go over them) and
    stays at 2,048."""
    p = mg.block_with_cores(40)
    p.k_tables = ((0, [300.0, 900.0], [150.0, 120.0]), (1, [300.0, 900.0], [30.0, 26.0]))
    with fem.Mesh(p, "fp32") as m:
        ne = m.plan("blocks").reshape(-1, 16)[:, 1]
        assert 1024 <= ne.max() <= 1792
        assert _smem_l2(m) <= FOUR_CTA_SMEM
    with fem.Mesh(mg.block_with_cores(40), "fp32", formulation="apparent") as m:
        ne = m.plan("blocks").reshape(-1, 16)[:, 1]
        assert ne.max() > 1792 and ne.max() <= 2048
