"""Host: the row plan of the split-precision contraction (lrtddft_row_plan), no GPU.

The Hermitian split needs one row pair per (G <= G'): N_G (N_G + 1) / 2 of them, 128 per
256-row super-tile.  The plan must cover every pair exactly once, with the least number of
super-tiles any covering has, each reading at most 6 blocks of 8 G from the pair densities.
"""
import math

import numpy as np
import pytest

from paper_2510_01875_gb300 import binding, build


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return binding.load()


@pytest.mark.parametrize("nG", list(range(1, 121)) + [130, 137, 169, 200, 257, 512])
def test_plan_covers_every_pair_once_with_fewest_super_tiles(nG):
    n_st, n_list, max_blocks, rp = binding.row_plan(nG)
    assert n_st == math.ceil(nG * (nG + 1) / 256)
    assert 1 <= max_blocks <= 6
    assert (rp == rp.T).all()
    upper = rp[np.triu_indices(nG)]
    assert len(np.unique(upper)) == nG * (nG + 1) // 2   # no two pairs share a row pair
    assert upper.min() >= 0 and upper.max() < 128 * n_st
    assert 0 <= n_list <= n_st * 8


def test_plan_keeps_quad_blocks_where_they_lose_nothing():
    # N_G a multiple of 4 whose quad covering is already the shortest: no lists
    n_st, n_list, _, _ = binding.row_plan(60)
    assert (n_st, n_list) == (15, 0)
    # N_G = 59: 15 quads would take 15 super-tiles; the plan takes 14
    n_st, n_list, _, rp = binding.row_plan(59)
    assert n_st == 14 and n_list > 0
    # off-diagonal pairs of two full quads stay in quad blocks: slot 4 i + j of one sub-block
    s = rp[0:4, 4:8] // 16
    assert (s == s[0, 0]).all()
    assert ((rp[0:4, 4:8] % 16) == 4 * np.arange(4)[:, None] + np.arange(4)[None, :]).all()


def test_plan_arguments():
    lib = binding.load()
    import ctypes as C
    a, b, d = C.c_int(), C.c_int(), C.c_int()
    for nG in (0, -1, 4097):
        assert lib.lrtddft_row_plan(nG, C.byref(a), C.byref(b), C.byref(d), None) == binding.LRT_EINVAL
    assert lib.lrtddft_row_plan(10, None, C.byref(b), C.byref(d), None) == binding.LRT_EINVAL
    assert lib.lrtddft_row_plan(10, C.byref(a), C.byref(b), C.byref(d), None) == 0
    assert a.value == 1
