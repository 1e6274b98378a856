"""Bounds of the TMA convolution's tile plans, checked on the CPU against the
library's own planner (cnn_conv_plan): every shared-memory read of an MMA operand
stays inside its stage, every output node of a tile is written exactly once, and
TMEM columns, TMA box extents and the stage ring stay within the hardware limits.
No GPU is needed: the planner is host code."""
import itertools

import pytest


@pytest.fixture(scope="module")
def n():
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native
    return native


SHAPES = [(20, 12), (16, 16), (16, 24), (8, 16), (12, 20), (8, 8), (6, 200), (5, 130), (5, 127), (3, 127),
          (37, 40), (64, 1024), (512, 1024), (256, 512), (128, 256), (64, 128), (16, 32), (4, 8), (2, 4), (1, 2),
          (1, 1), (7, 300), (33, 129), (6, 254), (3, 256), (10, 126)]
BUDGETS = [(0, 0, 0), (36, 110, 0), (56, 112, 0), (100, 200, 0), (47, 200, 0), (0, 0, 4)]


def _taps(mode, py, px, pw):
    """(parity sub-plane, offset in pixels) of each contributing tap (the kernel's tap_source)."""
    out = []
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        if mode == 0:
            out.append((0, (dy + 1) * pw + dx + 1))
        elif mode == 1:
            out.append(((2 if dy == 0 else 0) + (1 if dx == 0 else 0), (pw if dy == 1 else 0) + (1 if dx == 1 else 0)))
        elif mode == 2:
            out.append((0, (((py + dy) >> 1) + 1) * pw + ((px + dx) >> 1) + 1))
        else:
            uy, ux = py - 1 - dy, px - 1 - dx
            if uy % 2 == 0 and ux % 2 == 0:
                out.append((0, ((uy >> 1) + 1) * pw + (ux >> 1) + 1))
    return out


def _check(g, mode, npad, hin, win, nb):
    H, W = (hin, win) if mode >= 2 else ((hin // 2, win // 2) if mode == 1 else (hin, win))
    used = g["mode"]
    halo = 1 if mode == 1 else 2
    assert g["tiles"] == -(-W // g["tw"]) * -(-H // g["rows"]) * nb
    # TMA boxes (8-byte elements along a row, rows): at most 256 per dimension
    if mode == 1:
        assert 2 * g["pw"] <= 256 and 2 * (g["rows"] + 1) <= 256 and g["pw"] == g["tw"] + 1
    else:
        assert 2 * g["pw"] <= 256 and g["rows"] + 2 <= 256 and g["pw"] == g["tw"] + 2
    # stage layout: [parity][half][staged pixels x 16 B], then the weights
    assert g["plane"] == (g["rows"] + halo) * g["pw"] * 16
    assert g["pstride"] >= 2 * g["plane"] and g["pstride"] % 128 == 0
    assert g["stage"] == g["nplanes"] * g["pstride"] + g["wbytes"] and g["stage"] % 128 == 0
    assert g["wbytes"] == 9 * 2 * npad * 16
    assert 2 <= g["ns"] <= 6 and g["ns"] * g["stage"] <= 200 * 1024
    assert g["tmem_cols"] <= 512 and g["tmem_cols"] >= 32 and g["tmem_cols"] & (g["tmem_cols"] - 1) == 0
    stage_end = g["stage"]
    cover = set()
    if used == 4:
        assert npad == 16 and 3 * npad <= g["slot_cols"] and g["nslot"] * g["slot_cols"] <= g["tmem_cols"]
        assert g["nslot"] % 2 == 0          # two warpgroups drain alternate slots
        for m in range(g["mb"]):
            for dy in range(3):
                for h in (0, 1):
                    lo = h * g["plane"] + (m * 96 + dy * g["pw"]) * 16
                    assert lo >= 0 and lo + (15 * 6 + 8) * 16 <= stage_end
            for grp in range(16):
                for i in range(6):
                    yy, xx = divmod(m * 96 + 6 * grp + i, g["pw"])
                    if xx < g["tw"] and yy < g["rows"]:
                        assert (yy, xx) not in cover
                        cover.add((yy, xx))
        assert len(cover) == g["rows"] * g["tw"]
        return
    nph = g["nph"]
    assert 2 * nph * g["mb"] * npad <= g["tmem_cols"]
    for ph in range(nph):
        py, px = ph >> 1, ph & 1
        taps = _taps(mode, py, px, g["pw"])
        for m in range(g["mb"]):
            for pl, off in taps:
                for h in (0, 1):
                    lo = pl * g["pstride"] + h * g["plane"] + (m * 128 + off) * 16
                    assert lo >= 0 and lo + 128 * 16 <= stage_end, (mode, hin, win, g, m, pl, off)
            for r in range(128):
                yy, xx = divmod(m * 128 + r, g["pw"])
                if xx < g["tw"] and yy < g["rows"]:
                    assert (ph, yy, xx) not in cover
                    cover.add((ph, yy, xx))
    assert len(cover) == nph * g["rows"] * g["tw"]


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_tile_plans_stay_in_bounds(n, mode):
    checked = 0
    for (H, W), c0, npad, (skb, rkb, cap) in itertools.product(SHAPES, (16, 64), (16, 32, 64, 128), BUDGETS):
        if mode == 1:
            hin, win = 2 * H, 2 * W
        else:
            hin, win = H, W
        g = n.cnn_conv_plan(mode, c0, 0, npad, hin, win, 2, skb, rkb, cap)
        if g is None:
            continue                 # the launcher rejects it too (gather kernel): one shared decision
        _check(g, mode, npad, hin, win, 2)
        checked += 1
    assert checked > 100


def test_column_taps_in_n_plans_stay_in_bounds(n):
    checked = 0
    for (H, W), c1 in itertools.product(SHAPES, (0, 16, 32)):
        g = n.cnn_conv_plan(0, 16, c1, 16, H, W, 3, narrow=True)
        if g is None or g["mode"] != 4:
            continue
        assert g["ns"] >= (16 + c1) // 16 + 1      # every group of a tile resident, and one more
        _check(g, 0, 16, H, W, 3)
        checked += 1
    assert checked > 20


def test_default_plans_of_the_benchmark_network(n):
    """The 1024x512 network's first layers: 8-row tiles at two CTAs per SM; stride-2
    layers take 100 KB stages (one CTA per SM)."""
    g0 = n.cnn_conv_plan(0, 16, 0, 16, 512, 1024)
    assert (g0["rows"], g0["tw"], g0["ns"], g0["tmem_cols"]) == (8, 114, 2, 256)
    g1 = n.cnn_conv_plan(1, 16, 0, 32, 512, 1024)
    assert g1["rows"] == 4 and g1["stage"] > 47 * 1024 and g1["ns"] * g1["stage"] <= 200 * 1024
