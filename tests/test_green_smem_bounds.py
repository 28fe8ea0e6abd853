"""Index arithmetic of the FP32 LU Green kernel's trailing update, checked on
the host for every basis size the mixed path accepts (no GPU).

The update reads the panel (rows NB + r, stride PSTR) and the U12 rows
(Us[k M + c]) without bounds guards: a thread's TX x TY micro-tile takes rows
rg + x tr and columns cg + y tc, which for a ragged trailing block reach up
to TX - 1 rows and TY - 1 columns past its edge; those products are never
stored.  The reads must still stay inside the block's dynamic shared memory:
the panel region (M PSTR complex values) followed by the U12 region
(us_len(M) values), and a U12 read must stay inside its own row k.  The
constants are read from the kernel source, so a change of panel width or
micro-tile is checked again here.
"""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2012_12228_gb300", "csrc", "green_blocked.cu")


def _constants():
    s = open(SRC).read()
    nb = int(re.search(r"constexpr int NB = (\d+);", s).group(1))
    tx, ty = map(int, re.search(r"constexpr int TX = (\d+), TY = (\d+);", s).groups())
    m = re.search(r"constexpr int PSTR = NB \+ (\d+);", s)
    pstr = nb + int(m.group(1))
    a, b = map(int, re.search(r"constexpr int TILE = (\d+) \* (\d+);", s).groups())
    assert "int us_len(int M) { return NB * M > TILE ? NB * M : TILE; }" in s
    return nb, tx, ty, pstr, a * b


def test_trailing_update_reads_stay_in_shared_memory():
    NB, TX, TY, PSTR, TILE = _constants()
    checked = 0
    for M in range(1, 1022):                     # the mixed path accepts M <= 1021
        us_len = max(NB * M, TILE)
        for jb in range(0, M, NB):
            nb = min(NB, M - jb)
            c0 = jb + nb
            nrr = ncr = M - c0
            if nrr <= 0:
                continue
            assert nb == NB                      # only a full panel has a trailing block
            tr, tc = -(-nrr // TX), -(-ncr // TY)
            row_max = NB + (tr - 1) + (TX - 1) * tr          # largest panel row read
            col_max = (tc - 1) + (TY - 1) * tc               # largest U12 column read
            assert row_max * PSTR + (NB - 1) < M * PSTR + us_len, (M, jb)
            assert col_max < M, (M, jb)                      # inside row k of U12
            assert (NB - 1) * M + col_max < us_len, (M, jb)
            # the stored entries are exactly the trailing block, each once
            rows = {rg + x * tr for rg in range(tr) for x in range(TX) if rg + x * tr < nrr}
            cols = {cg + y * tc for cg in range(tc) for y in range(TY) if cg + y * tc < ncr}
            assert rows == set(range(nrr)) and cols == set(range(ncr)), (M, jb)
            checked += 1
    assert checked > 30000
