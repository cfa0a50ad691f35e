"""Which kernel writes which node on the one-pass path, replayed on the CPU.

A Python copy of the index arithmetic of the one-pass tiles (fused_interior: tile origin,
column / row ownership, z-blocks), of the band geometry set up on the host, and of the band
warps' node decoding (band_lane, with the per-component `have` masks).  Over grids near every
tiling boundary, every node of every component must be written exactly once in each phase.
The one exception is the first interior H layer (index 3 or n-2 on some axis, inside
[3, n-2]^3), which the one-pass step and band H both write with the same bits.  A change to
either side's indexing that loses or doubles a node fails here before any GPU run.
"""
import itertools

import numpy as np
import pytest

FTX, FTY = 64, 8                        # H footprint of a one-pass CTA: columns x rows
ON_PLUS = ((0, 1, 1), (1, 0, 1), (1, 1, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1))


def extents(n, c):
    """Nodes per axis of component c: n+1 on the plus grid, n+2 on the minus grid."""
    return tuple(n[a] + (1 if ON_PLUS[c][a] else 2) for a in range(3))


def fused_nodes(n, depth, rows=FTY, width=FTX):
    """(H nodes, E nodes) the one-pass kernel stores, as lists of (i, j, k) (one entry per store).
    A tile is `width` columns by `rows` rows; with 128 columns two warps share a row, warp
    group g taking columns 64 g .. 64 g + 63 of it."""
    nx, ny, nz = n
    FTX = width
    tx = (nx - 5 + FTX - 2) // (FTX - 1)
    ty = (ny - 5 + rows - 2) // (rows - 1)
    tz = (nz - 5 + depth - 1) // depth
    hs, es = [], []
    for bx, by, bz in itertools.product(range(tx), range(ty), range(tz)):
        x0, y0, k0 = 3 + bx * (FTX - 1), 3 + by * (rows - 1), 3 + bz * depth
        k1 = min(k0 + depth, nz - 2)
        for w in range(rows):
            j = y0 + w
            row_e = w < rows - 1 and j <= ny - 3
            row_h = j <= ny - 2 and (w < rows - 1 or j == ny - 2)
            for g, lane, h in itertools.product(range(FTX // 64), range(32), range(2)):
                c = 64 * g + lane + 32 * h
                i = x0 + c
                col_h = row_h and i <= nx - 2 and (c < FTX - 1 or i == nx - 2)
                col_e = row_e and c < FTX - 1 and i <= nx - 3
                for q in range(k0, k1 + 1):
                    if col_h and (q < k1 or q == nz - 2):
                        hs.append((i, j, q))
                    if q > k0 and col_e:
                        es.append((i, j, q - 1))
    return hs, es


def band_geometry(n, lo):
    hi = [n[a] - 3 for a in range(3)]
    segs = hi[0] // 32 + 1
    ey, ez = n[1] + 2, n[2] + 2
    zplanes = lo + (n[2] + 1 - hi[2])
    yrows = lo + (n[1] + 1 - hi[1])
    jin = hi[1] - lo + 1
    xgroups = (ey + 7) // 8
    wz, wy, wx = zplanes * jin * segs, ez * yrows * segs, ez * xgroups * 2
    return dict(lo=lo, hi=hi, segs=segs, jin=jin, yrows=yrows, xgroups=xgroups, wz=wz, wy=wy, wx=wx)


def band_lane(b, n, w, lane):
    """(i, j, k) of the lane's node in band warp w, or None."""
    lo, hi = b["lo"], b["hi"]
    if w < b["wz"] + b["wy"]:
        zs = w < b["wz"]
        if not zs:
            w -= b["wz"]
        r, seg = divmod(w, b["segs"])
        if zs:
            pl, jr = divmod(r, b["jin"])
            j = lo + jr
            k = pl if pl < lo else hi[2] + 1 + (pl - lo)
        else:
            k, jr = divmod(r, b["yrows"])
            j = jr if jr < lo else hi[1] + 1 + (jr - lo)
        i = seg * 32 + lane
        return (i, j, k) if lo <= i <= hi[0] else None
    w -= b["wz"] + b["wy"]
    side, r = w & 1, w >> 1
    k, g = divmod(r, b["xgroups"])
    jl = 8 * g
    jh = min(jl + 7, n[1] + 1)
    j = jl + (lane >> 2)
    c = lane & 3
    i = (hi[0] + 1 if side else 0) + c
    ok = j <= jh and (i <= n[0] + 1 if side else c < lo)
    return (i, j, k) if ok else None


def band_nodes(n, lo):
    b = band_geometry(n, lo)
    out = []
    for w in range(b["wz"] + b["wy"] + b["wx"]):
        for lane in range(32):
            node = band_lane(b, n, w, lane)
            if node is not None:
                out.append(node)
    return out


def _counts(n, comps, written):
    """Per component, how many times each node of its extent is written."""
    res = {}
    for c in comps:
        ext = extents(n, c)
        cnt = np.zeros(ext, dtype=np.int32)
        for nodes in written:
            for (i, j, k) in nodes:
                if i < ext[0] and j < ext[1] and k < ext[2]:
                    cnt[i, j, k] += 1
        res[c] = cnt
    return res


GRIDS = [((66, 9, 9), 8), ((67, 9, 10), 8), ((128, 9, 9), 16), ((129, 10, 9), 8), ((8, 8, 8), 8), ((9, 12, 13), 8), ((10, 13, 21), 13), ((68, 12, 17), 8), ((69, 20, 9), 8),
         ((70, 19, 33), 13), ((40, 11, 40), 64), ((132, 9, 9), 8), ((133, 15, 9), 8), ((259, 9, 10), 16)]


@pytest.mark.parametrize("width, rows", [(64, 8), (64, 16), (128, 8), (128, 12)])
@pytest.mark.parametrize("n, depth", GRIDS)
def test_every_node_written_once(n, depth, width, rows):
    """A one-pass tile of width x rows H nodes (the four tiles the host accepts)."""
    fh, fe = fused_nodes(n, depth, rows, width)
    bh, be = band_nodes(n, 4), band_nodes(n, 3)
    for nodes in (fh, fe, bh, be):                                  # no kernel writes a node twice
        assert len(nodes) == len(set(nodes))
    # H: once, except the first interior layer, written by both (same bits)
    for c, cnt in _counts(n, range(3, 6), [fh, bh]).items():
        idx = np.indices(cnt.shape)
        inner = np.all([(idx[a] >= 3) & (idx[a] <= n[a] - 2) for a in range(3)], axis=0)
        deep = np.all([(idx[a] >= 4) & (idx[a] <= n[a] - 3) for a in range(3)], axis=0)
        layer = inner & ~deep
        assert np.all(cnt[~layer] == 1), (c, np.argwhere(cnt[~layer] != 1)[:5])
        assert np.all(cnt[layer] == 2), c
    for c, cnt in _counts(n, range(3), [fe, be]).items():
        assert np.all(cnt == 1), (c, np.argwhere(cnt != 1)[:5])
    # the one-pass kernel stays inside its boxes
    assert all(3 <= v[a] <= n[a] - 2 for v in fh for a in range(3))
    assert all(3 <= v[a] <= n[a] - 3 for v in fe for a in range(3))


def test_band_geometry_is_what_the_host_accepts():
    """x-end slabs at most 4 nodes wide, and x segments from 0 reach past the interior."""
    for n in (8, 13, 64, 255, 512):
        for lo in (3, 4):
            b = band_geometry((n, n, n), lo)
            assert lo <= 4 and n + 1 - b["hi"][0] <= 4
            assert b["segs"] * 32 > b["hi"][0]


def _find_slot(pre, n, b):
    """The batched kernels' lookup: the largest g < n with pre[g] <= b (binary search)."""
    lo, hi = 0, n - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if pre[mid] <= b:
            lo = mid
        else:
            hi = mid - 1
    return lo


def test_batched_ctas_map_to_every_tile_of_every_grid_once():
    """A batched launch of sum(count_g) CTAs: CTA b serves grid find_slot(pre, b), local index
    b - pre[g], decoded as tile (local % tx, (local / tx) % ty, local / (tx ty)).  Grids with
    no CTAs of a kind (e.g. no band nodes) are skipped; every tile of every grid is served once."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        n = int(rng.integers(1, 12))
        tiles = [tuple(int(v) for v in rng.integers(1, 6, size=3)) for _ in range(n)]
        counts = [tx * ty * tz if rng.random() > 0.15 else 0 for tx, ty, tz in tiles]
        pre = np.concatenate([[0], np.cumsum(counts)]).astype(int)
        seen = set()
        for b in range(int(pre[-1])):
            g = _find_slot(pre, n, b)
            assert pre[g] <= b < pre[g + 1]
            local = b - pre[g]
            tx, ty, _ = tiles[g]
            seen.add((g, local % tx, (local // tx) % ty, local // (tx * ty)))
        want = {(g, x, y, z) for g, (tx, ty, tz) in enumerate(tiles) if counts[g]
                for x in range(tx) for y in range(ty) for z in range(tz)}
        assert seen == want


def test_persistent_tickets_cover_every_item_and_wait_only_backwards():
    """The persistent batched kernel's ticket decoding, replayed: ticket t is item t mod T of
    step t div T; the T items go grid by grid (prefix of the grids' item counts, binary
    search), and within a grid its band-H items, its tiles, its band-E items, a band item
    being up to 8 band CTAs.  Every (step, kind, grid, item) is served exactly once, every
    band CTA of every grid lies in exactly one band item, and each item's dependencies (all
    items of its grid at the previous step; band H of its grid at its step for band E) have
    smaller tickets, so a CTA never waits for work that no running CTA holds."""
    group = 8
    rng = np.random.default_rng(11)
    for _ in range(100):
        n = int(rng.integers(1, 7))
        K = int(rng.integers(1, 5))
        hct, nf, ect = (rng.integers(0, 30, size=n) for _ in range(3))
        nh = [(c + group - 1) // group for c in hct]
        ne = [(c + group - 1) // group for c in ect]
        pi = np.concatenate([[0], np.cumsum([nh[g] + nf[g] + ne[g] for g in range(n)])]).astype(int)
        T = int(pi[-1])
        seen, ticket_of = set(), {}
        for t in range(K * T):
            o, r = divmod(t, T)
            g = _find_slot(pi, n, r)
            assert pi[g] <= r < pi[g + 1]
            r -= pi[g]
            kind = 0 if r < nh[g] else 1 if r < nh[g] + nf[g] else 2
            r -= 0 if kind == 0 else nh[g] if kind == 1 else nh[g] + nf[g]
            key = (o, kind, g, r)
            assert key not in seen
            seen.add(key)
            ticket_of[key] = t
        want = {(o, k, g, i) for o in range(K) for g in range(n)
                for k, cnt in enumerate((nh[g], nf[g], ne[g])) for i in range(cnt)}
        assert seen == want
        for g in range(n):        # band CTAs (8 warps each) of an item: [item * group, (item + 1) * group)
            for cnt, items in ((hct[g], nh[g]), (ect[g], ne[g])):
                covered = [c for it in range(items) for c in range(it * group, min((it + 1) * group, cnt))]
                assert covered == list(range(cnt))
        for (o, kind, g, i), t in ticket_of.items():
            deps = [key for key in ticket_of if key[2] == g and key[0] == o - 1]
            if kind == 2:
                deps += [key for key in ticket_of if key[2] == g and key[0] == o and key[1] == 0]
            assert all(ticket_of[d] < t for d in deps)
