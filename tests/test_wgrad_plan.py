"""Bounds of the tensor-core weight-gradient kernel's tile plans, checked on the CPU
against the library's own planner (cnn_wgrad_plan, host code): the TEM columns, the
TMA boxes and their landing places inside a stage, the transaction bytes, and every
shared-memory read of an MMA operand (under both readings of the descriptor's two
byte offsets for an MN-major operand, so that the reads stay inside the allocation
whichever the hardware takes) stay within the hardware limits and the CTA's
dynamic shared memory.  No GPU is needed."""
import itertools

import pytest


@pytest.fixture(scope="module")
def n():
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native
    return native


KEYS = ("ktiles", "tw", "rows", "P", "tiles_x", "tiles_y", "phases", "cx", "cx0", "gchunks", "tpg", "ngroups",
        "max_chunks", "plane", "stage", "ns", "slack", "tmem_cols", "splits", "smem")


def _plan(n, mode, c0, c1, npad, hin, win, nb, sms=148):
    return n.cnn_wgrad_plan(mode, c0, c1, npad, hin, win, nb, sms)


def _check(g, mode, c0, c1, npad, hin, win, nb):
    hout, wout = (hin // 2, win // 2) if mode == 1 else ((2 * hin, 2 * win) if mode == 2 else (hin, win))
    Ht, Wt = (hin, win) if mode == 2 else (hout, wout)
    assert g["cx"] == (c0 + c1) // 8 and g["cx0"] == c0 // 8 and g["gchunks"] == npad // 8
    assert g["P"] == g["tw"] * g["rows"] and g["P"] % 16 == 0 and g["tw"] % 16 == 0 and g["tw"] <= 128
    assert g["plane"] == 16 * g["P"]
    assert g["tiles_x"] == -(-Wt // g["tw"]) and g["tiles_y"] == -(-Ht // g["rows"])
    assert g["ktiles"] == nb * g["tiles_x"] * g["tiles_y"] * g["phases"]
    assert g["phases"] == (4 if mode == 2 else 1)
    assert 1 <= g["splits"] <= g["ktiles"]
    # TMA boxes: at most 256 per dimension (8-byte elements along a row)
    es_x, es_g = (2 if mode == 1 else 1), (2 if mode == 2 else 1)
    for es, ch in ((es_x, g["cx0"]), (es_x, g["cx"] - g["cx0"]), (es_g, g["gchunks"])):
        assert 2 * g["tw"] <= 256 and es * g["rows"] <= 256 and ch <= 256
    # TMEM: M blocks x npad columns of every group
    tpg = g["tpg"]
    assert g["ngroups"] == -(-9 // tpg) and g["max_chunks"] == tpg * g["cx"]
    cols = g["tmem_cols"]
    assert 32 <= cols <= 512 and cols & (cols - 1) == 0
    assert -(-g["max_chunks"] // 16) * npad <= cols
    # shared memory: ring + slack inside the CTA's allocation (<= 227 KB)
    assert 2 <= g["ns"] <= 4
    assert g["stage"] == (g["max_chunks"] + g["gchunks"]) * g["plane"]
    total = g["ns"] * g["stage"] + g["slack"]
    assert total <= 200 * 1024 and g["smem"] >= total and g["smem"] <= 227 * 1024
    covered = []
    for grp in range(g["ngroups"]):
        t0 = grp * tpg
        ntap = min(9, t0 + tpg) - t0
        chunks = ntap * g["cx"]
        covered += [(t0 + i, c) for i in range(ntap) for c in range(g["cx"])]
        # TMA landing places within a stage: x0, x1 per tap, then g
        boxes = []
        for i in range(ntap):
            boxes.append((i * g["cx"] * g["plane"], g["cx0"] * g["plane"]))
            if c1:
                boxes.append(((i * g["cx"] + g["cx0"]) * g["plane"], (g["cx"] - g["cx0"]) * g["plane"]))
        gofs = g["max_chunks"] * g["plane"]
        boxes.append((gofs, g["gchunks"] * g["plane"]))
        for lo, size in boxes:
            assert lo % 16 == 0 and 0 <= lo and lo + size <= g["stage"]
        assert sum(sz for _, sz in boxes) == (chunks + g["gchunks"]) * g["plane"]   # transaction bytes
        # MMA operand reads from the last stage (the highest addresses)
        base = (g["ns"] - 1) * g["stage"]
        for mb in range(-(-chunks // 16)):
            for kk in range(g["P"] // 16):
                a = base + 16 * mb * g["plane"] + 256 * kk
                b = base + gofs + 256 * kk
                # reading 1: 8-channel chunks SBO = plane apart, K groups LBO = 128 B apart
                assert a + 15 * g["plane"] + 128 + 128 <= total
                assert b + (g["gchunks"] - 1) * g["plane"] + 256 <= base + g["stage"]
                # reading 2: the two offsets the other way round
                assert a + 15 * 128 + g["plane"] + 128 <= total
                assert b + (g["gchunks"] - 1) * 128 + g["plane"] + 128 <= total
                assert (a >> 4) < (1 << 14) and (b >> 4) < (1 << 14)    # descriptor start field
    assert sorted(covered) == [(t, c) for t in range(9) for c in range(g["cx"])]   # each (tap, chunk) once


# the layers of the 16/32/64/128 network (mode, c0, c1, npad) and some others
LAYERS = [(0, 16, 0, 16), (0, 16, 16, 16), (0, 32, 0, 32), (0, 32, 32, 32), (0, 64, 0, 64), (0, 64, 64, 64),
          (0, 128, 0, 128), (0, 128, 128, 128), (1, 16, 0, 32), (1, 32, 0, 64), (1, 64, 0, 128), (2, 32, 0, 16),
          (2, 64, 0, 32), (2, 128, 0, 64), (0, 16, 0, 32), (1, 16, 0, 16), (2, 16, 0, 16), (0, 8, 0, 16),
          (0, 64, 0, 128), (1, 128, 0, 128), (2, 128, 0, 128)]
GRIDS = [(512, 1024), (256, 512), (128, 256), (64, 128), (32, 32), (16, 16), (8, 8), (2, 2), (37, 40), (6, 200),
         (4, 300), (64, 20)]


@pytest.mark.parametrize("layer", LAYERS)
def test_weight_gradient_plans_stay_in_bounds(n, layer):
    mode, c0, c1, npad = layer
    checked = 0
    for (h, w), nb in itertools.product(GRIDS, (1, 3, 16)):
        if mode == 1 and (h % 2 or w % 2):
            continue
        g = _plan(n, mode, c0, c1, npad, h, w, nb)
        assert g is not None, (layer, h, w, nb)
        _check(g, mode, c0, c1, npad, h, w, nb)
        checked += 1
    assert checked >= 20


def test_plans_of_the_benchmark_network(n):
    """16-channel layers at 1024 x 512: one group of all nine taps, 128-pixel K tiles;
    the 256-channel concatenation of the coarsest level splits its taps over groups."""
    g = _plan(n, 0, 16, 0, 16, 512, 1024, 16)
    assert (g["ngroups"], g["P"], g["tmem_cols"]) == (1, 128, 32)
    g = _plan(n, 0, 128, 128, 128, 64, 128, 16)
    assert g["ngroups"] == 5 and g["tmem_cols"] == 512
