"""The tiled split-CSR layout rule, restated in plain Python from its description, for tests.

A side with row pointers row_ptr is cut into tiles of 32 consecutive rows.  A row with more than
128 entries is long; then, while a tile's short rows hold more than 1024 entries, its longest
short row (the first of equal ones) becomes long.  Each tile's short segment starts at a multiple
of 4 in the short array; long rows go to a separate array, each starting at a multiple of 4, cut
into chunks of 256 entries.  M short tiles are walked per work item: the largest of 4 and 2 with
at least 2M tiles, a mean group segment of at most 256 entries (aligned short length times M
over the tile count) and a longest group segment of at most 1024 entries; else 1.  The staging
stride is the longest segment of a work item's group, rounded up to 4, plus 4.

FP64 walks sum a tile's longest short rows warp-wide when that saves work over the whole side:
per tile, lane-per-row sums cost the longest short row rounded up to 4 (FP64 adds per warp);
with a threshold c of 8, 16 or 32 (below the longest row, tried only when the longest exceeds
16) they cost c plus, for every short row longer than c, ceil(len / 32) + 5.  The side takes
warp-wide sums when the tiles' best costs add up to at most 85% of the lane-per-row costs.
"""
import numpy as np


def _align4(v: int) -> int:
    return (v + 3) & ~3


def plan(row_ptr) -> dict:
    return _plan(row_ptr)[0]


def group_fits(row_ptr, m: int) -> bool:
    """Whether walking m consecutive short tiles per work item fits the staging area: the longest
    group segment has at most 1024 entries (always true for m = 1)."""
    return m == 1 or _plan(row_ptr)[1](m) <= 1024


def _plan(row_ptr):
    lens = np.diff(np.asarray(row_ptr, dtype=np.int64))
    n = len(lens)
    nt = (n + 31) // 32
    cur = cl = 0
    n_long = chunks = 0
    seg_b, seg_e = [], []
    cost_plain = cost_best = 0
    for t in range(nt):
        L = lens[32 * t:32 * (t + 1)]
        short = L <= 128
        s = int(L[short].sum())
        while s > 1024:
            i = max((i for i in range(len(L)) if short[i]), key=lambda i: (L[i], -i))
            short[i] = False
            s -= int(L[i])
        cur = _align4(cur)
        seg_b.append(cur)
        for r in range(len(L)):
            if short[r]:
                cur += int(L[r])
            else:
                cl = _align4(cl) + int(L[r])
                n_long += 1
                chunks += -(-int(L[r]) // 256)
        seg_e.append(cur)
        sl = [int(L[r]) if short[r] else 0 for r in range(len(L))]
        mx = max(sl, default=0)
        plain = _align4(mx)
        best = plain
        if mx > 16:
            for c in (8, 16, 32):
                if c < mx:
                    best = min(best, c + sum(-(-x // 32) + 5 for x in sl if x > c))
        cost_plain += plain
        cost_best += best
    maxseg = max((e - b for b, e in zip(seg_b, seg_e)), default=0)

    def longest_group(m):
        if nt == 0:
            return 1 << 30
        return max(seg_e[min(nt, t + m) - 1] - seg_b[t] for t in range(0, nt, m))

    mult = 1
    for m in (4, 2):
        if nt < 2 * m or _align4(cur) * m > nt * 256:
            continue
        mx = longest_group(m)
        if mx <= 1024:
            mult, maxseg = m, mx
            break
    return dict(tiles=nt, tile_mult=mult, long_rows=n_long, chunks=chunks,
                seg=_align4(maxseg) + 4, nnz_short=_align4(cur) + 4, nnz_long=_align4(cl) + 256,
                wide_rows=int(cost_plain > 0 and cost_best <= 0.85 * cost_plain)), longest_group


def expected_tile_mult(row_ptr) -> int:
    return plan(row_ptr)["tile_mult"]
