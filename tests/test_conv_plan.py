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
            # the parity's four merged taps (ey, ex): coarse node (Y + py - 1 + ey, X + px - 1 + ex)
            if t < 4:
                out.append((0, (py + (t >> 1)) * pw + px + (t & 1)))
        else:
            uy, ux = py - 1 - dy, px - 1 - dx
            if uy % 2 == 0 and ux % 2 == 0:
                out.append((0, ((uy >> 1) + 1) * pw + (ux >> 1) + 1))
    return out


def test_merged_up_taps_read_the_nodes_of_the_nine_taps():
    """Nearest x2 upsampling then a 3x3 convolution: per output parity the nine taps read
    the 2 x 2 coarse nodes that the four merged taps of the kernel read, each tap the node
    of its merged tap (fine node 2Y + p, tap d -> coarse node floor((2Y + p + d) / 2))."""
    pw = 13
    for py in (0, 1):
        for px in (0, 1):
            merged = [off for _, off in _taps(2, py, px, pw)]
            assert len(merged) == 4 and len(set(merged)) == 4
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    for Y in range(3):
                        cy = (2 * Y + py + dy) // 2 - Y           # coarse row offset of the tap
                        cx = (2 * Y + px + dx) // 2 - Y
                        ey, ex = (py + dy + 2) // 2 - 1 - py + 1, (px + dx + 2) // 2 - 1 - px + 1
                        assert ey in (0, 1) and ex in (0, 1)
                        assert cy == py - 1 + ey and cx == px - 1 + ex
                        # staged with a one-node halo: offset of node (cy, cx) from the tile's pixel
                        assert merged[2 * ey + ex] == (cy + 1) * pw + cx + 1


def _check(g, mode, npad, hin, win, nb, split=False):
    H, W = (hin, win) if mode >= 2 else ((hin // 2, win // 2) if mode == 1 else (hin, win))
    used = g["mode"]
    halo = 1 if mode == 1 else 2
    split = split and mode == 2      # up layers: a tile per output row parity
    assert g["nph"] == (1 if mode < 2 else (2 if split else 4))
    assert g["tiles"] == -(-W // g["tw"]) * -(-H // g["rows"]) * nb * (2 if split else 1)
    # TMA boxes (8-byte elements along a row, rows): at most 256 per dimension
    if mode == 1:
        assert 2 * g["pw"] <= 256 and 2 * (g["rows"] + 1) <= 256 and g["pw"] == g["tw"] + 1
    else:
        assert 2 * g["pw"] <= 256 and g["rows"] + 2 <= 256 and g["pw"] == g["tw"] + 2
    # stage layout: [parity][half][staged pixels x 16 B], then the weights
    assert g["plane"] == (g["rows"] + halo) * g["pw"] * 16
    assert g["pstride"] >= 2 * g["plane"] and g["pstride"] % 128 == 0
    assert g["stage"] == g["nplanes"] * g["pstride"] + g["wbytes"] and g["stage"] % 128 == 0
    # up: 4 (split: 2) column/row parities x 4 merged taps
    assert g["wbytes"] == ((8 if split else 16) if mode == 2 else 9) * 2 * npad * 16
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
    assert g["nbuf"] in (1, 2) and g["nbuf"] * nph * g["mb"] * npad <= g["tmem_cols"]
    for ph, py in itertools.product(range(nph), (0, 1) if split else (None,)):
        py, px = (py, ph) if split else (ph >> 1, ph & 1)
        taps = _taps(mode, py, px, g["pw"])
        for m in range(g["mb"]):
            for pl, off in taps:
                for h in (0, 1):
                    lo = pl * g["pstride"] + h * g["plane"] + (m * 128 + off) * 16
                    assert lo >= 0 and lo + 128 * 16 <= stage_end, (mode, hin, win, g, m, pl, off)
            for r in range(128):
                yy, xx = divmod(m * 128 + r, g["pw"])
                if xx < g["tw"] and yy < g["rows"]:
                    assert (py, px, yy, xx) not in cover
                    cover.add((py, px, yy, xx))
    assert len(cover) == (4 if split else nph) * g["rows"] * g["tw"]


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_tile_plans_stay_in_bounds(n, mode):
    checked = 0
    for (H, W), c0, npad, (skb, rkb, cap), single, split in itertools.product(
            SHAPES, (16, 64), (16, 32, 64, 128), BUDGETS, (0, 1), (0, 1) if mode == 2 else (0,)):
        if mode == 1:
            hin, win = 2 * H, 2 * W
        else:
            hin, win = H, W
        narrow = (5 if single else 4) if split else (3 if single else 0)
        g = n.cnn_conv_plan(mode, c0, 0, npad, hin, win, 2, skb, rkb, cap, narrow=narrow)
        if g is None:
            continue                 # the launcher rejects it too (gather kernel): one shared decision
        _check(g, mode, npad, hin, win, 2, split=bool(split))
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


def _rowtaps_schedule(rows, ntiles, nslot, nwg=4, chunk=4, nbar=10):
    """The row-taps-in-N kernel's slot protocol, run as a simulation: the MMA side fills staged
    row jb (all tiles in order, rows + 2 per tile) into slot jb % nslot once the slot's
    previous fill took its 3 arrivals (x 128 threads), and commits after every `chunk` rows
    of a tile and after its last row (commit id c on barrier c % nbar); warpgroup w computes
    the output rows m = w, w + nwg, ... of every tile in order, each once the commit that
    covers staged row m + 2 is done, and arrives once on each of its three rows (the tile's
    first output row twice more on staged row 0 and once on row 1, its last once more on
    row R and twice on row R + 1).  The sides advance round-robin.  Returns True when
    everything finishes; asserts that no slot takes more than 3 arrivals per fill, that
    outputs read committed, unreleased rows, and that every parity wait is unambiguous: the
    barrier's previous commit is known complete to the waiting warpgroup, and its next
    commit cannot be done before the warpgroup arrives."""
    per = rows + 2
    cpt = -(-per // chunk)
    total = per * ntiles
    committed = [False] * total
    arrivals = [0] * total
    commits_done = 0
    jb = 0
    queues = [[(k, m) for k in range(ntiles) for m in range(w, rows, nwg)] for w in range(nwg)]
    heads = [0] * nwg
    known = [-1] * nwg          # commit ids this warpgroup's earlier waits proved complete
    progress = True
    while progress:
        progress = False
        while jb < total and (jb < nslot or arrivals[jb - nslot] == 3):
            jb += 1
            b = (jb - 1) % per
            if (b + 1) % chunk == 0 or b == per - 1:
                k = (jb - 1) // per
                for r in range(k * per + (b // chunk) * chunk, jb):
                    committed[r] = True
                commits_done += 1
            progress = True
        for w in range(nwg):
            if heads[w] >= len(queues[w]):
                continue
            k, m = queues[w][heads[w]]
            base = k * per
            cid = k * cpt + (m + 2) // chunk
            if cid >= commits_done:
                continue
            assert cid < nbar or cid - nbar <= known[w], (rows, nslot, nwg, k, m)
            assert commits_done <= cid + nbar, (rows, nslot, nwg, k, m)
            known[w] = cid
            for d in range(3):
                assert committed[base + m + d] and arrivals[base + m + d] < 3
            add = [base + m, base + m + 1, base + m + 2]
            if m == 0:
                add += [base, base, base + 1]
            if m == rows - 1:
                add += [base + rows, base + rows + 1, base + rows + 1]
            for b in add:
                arrivals[b] += 1
                assert arrivals[b] <= 3
            heads[w] += 1
            progress = True
    return jb == total and all(h == len(q) for h, q in zip(heads, queues)) and all(a == 3 for a in arrivals)


def test_rowtaps_plans_stay_in_bounds(n):
    """Mode 6 (tap rows in N): the A operand of staged row b at column shift dx (128 rows of
    16 bytes per 8-channel half) and the B operand of each shift stay inside the stage;
    every output node is lane x < tw of its row's three slots, read once; the slot ring
    (3 npad columns a slot) fits TMEM; every group of a tile and one more stage fit the
    ring; the slot protocol finishes for the planned ring."""
    checked = 0
    for (H, W), c0, c1, npad in itertools.product(SHAPES, (16, 32), (0, 16), (16, 32)):
        g = n.cnn_conv_plan(0, c0, c1, npad, H, W, 2, narrow=2)
        if g is None or g["mode"] != 6:
            continue
        rows, tw, pw = g["rows"], g["tw"], g["pw"]
        groups = (c0 + c1) // 16
        assert pw == tw + 2 and 2 * pw <= 256 and rows + 2 <= 256 and rows <= 32
        assert g["tiles"] == -(-W // tw) * -(-H // rows) * 2
        assert g["mb"] == rows + 2 and g["nph"] == 1 and g["nplanes"] == 1
        assert g["plane"] == (rows + 2) * pw * 16
        assert g["pstride"] >= 2 * g["plane"] and g["pstride"] % 128 == 0
        assert g["stage"] == g["pstride"] + g["wbytes"] and g["stage"] % 128 == 0
        assert g["wbytes"] == 9 * 2 * npad * 16
        assert groups + 1 <= g["ns"] <= 6 and g["ns"] * g["stage"] <= 200 * 1024
        assert g["tmem_cols"] == (256 if npad == 16 else 512)
        assert g["slot_cols"] == 3 * npad and g["nslot"] == min(10, g["tmem_cols"] // (3 * npad)) and g["nslot"] >= 3
        assert g["nslot"] * g["slot_cols"] <= g["tmem_cols"]
        assert g["ns"] * g["stage"] <= (100 if npad == 16 else 200) * 1024
        for b in range(rows + 2):
            for dx in range(3):
                for h in (0, 1):
                    lo = h * g["plane"] + (b * pw + dx) * 16
                    assert lo + 128 * 16 <= g["stage"]
        for dx in range(3):
            assert g["pstride"] + (dx + 1) * 6 * npad * 16 <= g["stage"]
        cover = set()
        for m in range(rows):
            for x in range(128):
                if x < tw:
                    assert 0 <= x + 2 < pw        # the three column shifts stay in the staged row
                    assert (m, x) not in cover
                    cover.add((m, x))
        assert len(cover) == rows * tw
        assert g["nwg"] in (1, 2) and g["nwg"] <= rows
        assert 1 <= g["chunk"] <= min(4, g["nslot"] - 2)
        assert _rowtaps_schedule(rows, 3, g["nslot"], g["nwg"], chunk=g["chunk"])
        checked += 1
    assert checked > 20


def test_rowtaps_slot_protocol_for_every_ring():
    """The slot protocol finishes with exactly three arrivals per fill and unambiguous parity
    waits for every tile height down to one row, every ring of at least three slots, and
    the warpgroup count and commit chunk the planner's rule gives (the largest of 4, 2, 1
    not above the tile height; at most 4 rows and nslot - 2); commit barriers reused too
    soon would not be, and a larger chunk deadlocks."""
    for nslot in range(3, 11):
        for rows in range(1, 40):
            nwg = 4
            while nwg > 1 and nwg > rows:
                nwg //= 2
            assert _rowtaps_schedule(rows, 4, nslot, nwg, chunk=min(4, nslot - 2))
    assert not _rowtaps_schedule(16, 3, 5, 4, chunk=4)
    with pytest.raises(AssertionError):
        _rowtaps_schedule(16, 4, 10, 4, chunk=1, nbar=3)
