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

Third order (eleven groups; Sec. III D finds working stencils for mbar >= 1.5):
an LP scan over the Table I groups with components up to 5 (weights
nonnegative, minimal folded population count, v0 on a grid), refined by the
library's window search, gives five sets whose positive windows, checked on a
1/16 grid of mbar, tile [1.875, 14]:

    O3_A  {8,15,20,24,26,27,28,30,36,37,42}   mbar in [1.875, 2.125)  Q = 149, halo 5
    O3_B  {4,10,15,20,24,26,27,28,30,36,37}   mbar in [2.125, 3.375)  Q = 133, halo 5
    O3_C  {4,8,14,15,16,17,18,21,22,23,26}    mbar in [3.375, 4.75)   Q = 133, halo 4
    O3_D  {2,3,5,6,7,8,9,10,11,13,15}         mbar in [4.75, 6.5)     Q = 103, halo 3
    O3_E  {1,2,3,6,7,8,9,10,11,13,15}         mbar in [6.5, 14]       Q = 99,  halo 3

and the set with a compiled FP32 kernel, O3_M5 {1,2,5,6,7,9,10,11,12,13,15}
(Q = 100), is taken for mbar in [4.875, 5.125].  Below 1.875 the scan found
only a six-component set at mbar = 1.5 whose window is narrower than 1e-5;
``choose(m, order=3)`` clamps to 1.875 and keeps O3_E above 14.
"""
E5 = (1, 14, 49, 51, 60, 70)
M1 = (5, 12, 14, 17, 21, 26)
S2 = (3, 9, 10, 14, 17, 21)
G16 = (1, 2, 3, 4, 5, 6)

RANGES = [(E5, 0.36, 0.58), (M1, 0.65, 1.2), (S2, 1.2, 6.0), (G16, 6.0, float("inf"))]


O3_A = (8, 15, 20, 24, 26, 27, 28, 30, 36, 37, 42)
O3_B = (4, 10, 15, 20, 24, 26, 27, 28, 30, 36, 37)
O3_C = (4, 8, 14, 15, 16, 17, 18, 21, 22, 23, 26)
O3_D = (2, 3, 5, 6, 7, 8, 9, 10, 11, 13, 15)
O3_E = (1, 2, 3, 6, 7, 8, 9, 10, 11, 13, 15)
O3_M5 = (1, 2, 5, 6, 7, 9, 10, 11, 12, 13, 15)

RANGES_O3 = [(O3_M5, 4.875, 5.125), (O3_A, 1.875, 2.125), (O3_B, 2.125, 3.375), (O3_C, 3.375, 4.75),
             (O3_D, 4.75, 6.5), (O3_E, 6.5, float("inf"))]


def choose(m, order=2):
    """(groups, mbar_used) for a requested mbar; order 2 (six groups) or 3
    (eleven groups)."""
    if order == 3:
        m = max(float(m), 1.875)
        for groups, lo, hi in RANGES_O3:
            if lo <= m <= hi if groups is O3_M5 else lo <= m < hi:
                return list(groups), m
        return list(O3_E), m
    if order != 2:
        raise ValueError("order must be 2 or 3")
    m = float(m)
    if m < 0.36:
        m = 0.36
    if 0.58 < m < 0.65:
        m = 0.58 if m - 0.58 < 0.65 - m else 0.65
    for groups, lo, hi in RANGES:
        if lo <= m < hi or (groups is E5 and m == hi):
            return list(groups), m
    return list(G16), m
