"""Stencil library: which compiled six-group stencil serves a given m/T_R.

Second-order quadratures with positive weights exist only on intervals of
mbar = m/T_R for a given group set (Sec. III D; none as mbar -> 0).  The four
group sets with compiled kernels cover, with all six weights positive at the
centre of the widest v0 window (found by the library's window search):

    E5  {1,14,49,51,60,70}   mbar in [0.36, 0.58]
    M1  {5,12,14,17,21,26}   mbar in [0.65, 1.40]
    S2  {3,9,10,14,17,21}    mbar in [1.10, 8.40]
    G16 {1,2,3,4,5,6}        mbar in [4.50, 10.0] (and above)

``choose(m)`` returns the set and the mbar actually used: below 0.36 it clamps
to 0.36 (the paper's second-order coverage limit), inside the gap
(0.58, 0.65) it snaps to the nearer edge, above 10 it keeps G16.
"""
E5 = (1, 14, 49, 51, 60, 70)
M1 = (5, 12, 14, 17, 21, 26)
S2 = (3, 9, 10, 14, 17, 21)
G16 = (1, 2, 3, 4, 5, 6)

RANGES = [(E5, 0.36, 0.58), (M1, 0.65, 1.2), (S2, 1.2, 6.0), (G16, 6.0, float("inf"))]


def choose(m):
    """(groups, mbar_used) for a requested mbar."""
    m = float(m)
    if m < 0.36:
        m = 0.36
    if 0.58 < m < 0.65:
        m = 0.58 if m - 0.58 < 0.65 - m else 0.65
    for groups, lo, hi in RANGES:
        if lo <= m < hi or (groups is E5 and m == hi):
            return list(groups), m
    return list(G16), m
