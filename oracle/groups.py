"""Velocity groups of Table I (App. C, "Stencils for three-dimensional lattices").

Each group is the full-symmetric (FS) orbit of one integer vector: every
permutation of its components with every choice of signs.  The table prints
the generating vector, the orbit size ("# Vectors") and the common length.
Those three columns are restated here as printed; tests check that the
generated orbits reproduce the printed sizes and lengths.

Misprint: the printed lengths of rows 17 and 18 are exchanged.  Row 17,
(3,2,2), has length sqrt(17), and row 18, (3,3,1), has length sqrt(19); the
table prints sqrt(19) and sqrt(17).  Every computation therefore takes the
length from the vector (``length2``), never from the printed column.

TEST INFRASTRUCTURE ONLY (see the package docstring)."""
import itertools
import math

# group id -> (generating vector, printed cardinality, printed length squared)
TABLE_I = {
    1: ((0, 0, 0), 1, 0), 2: ((1, 0, 0), 6, 1), 3: ((1, 1, 0), 12, 2),
    4: ((1, 1, 1), 8, 3), 5: ((2, 0, 0), 6, 4), 6: ((2, 1, 0), 24, 5),
    7: ((2, 2, 0), 12, 8), 8: ((2, 1, 1), 24, 6), 9: ((2, 2, 1), 24, 9),
    10: ((2, 2, 2), 8, 12), 11: ((3, 0, 0), 6, 9), 12: ((3, 1, 0), 24, 10),
    13: ((3, 2, 0), 24, 13), 14: ((3, 3, 0), 12, 18), 15: ((3, 1, 1), 24, 11),
    16: ((3, 2, 1), 48, 14), 17: ((3, 2, 2), 24, 19), 18: ((3, 3, 1), 24, 17),
    19: ((3, 3, 2), 24, 22), 20: ((3, 3, 3), 8, 27), 21: ((4, 0, 0), 6, 16),
    22: ((4, 1, 0), 24, 17), 23: ((4, 2, 0), 24, 20), 24: ((4, 3, 0), 24, 25),
    25: ((4, 4, 0), 12, 32), 26: ((4, 1, 1), 24, 18), 27: ((4, 2, 1), 48, 21),
    28: ((4, 3, 1), 48, 26), 29: ((4, 4, 1), 24, 33), 30: ((4, 2, 2), 24, 24),
    31: ((4, 3, 2), 48, 29), 32: ((4, 4, 2), 24, 36), 33: ((4, 3, 3), 24, 34),
    34: ((4, 4, 3), 24, 41), 35: ((4, 4, 4), 8, 48), 36: ((5, 0, 0), 6, 25),
    37: ((5, 1, 0), 24, 26), 38: ((5, 2, 0), 24, 29), 39: ((5, 3, 0), 24, 34),
    40: ((5, 4, 0), 24, 41), 41: ((5, 5, 0), 12, 50), 42: ((5, 1, 1), 24, 27),
    43: ((5, 2, 1), 48, 30), 44: ((5, 3, 1), 48, 35), 45: ((5, 4, 1), 48, 42),
    46: ((5, 5, 1), 24, 51), 47: ((5, 2, 2), 24, 33), 48: ((5, 3, 2), 48, 38),
    49: ((5, 4, 2), 48, 45), 50: ((5, 5, 2), 24, 54), 51: ((5, 3, 3), 24, 43),
    52: ((5, 4, 3), 48, 50), 53: ((5, 5, 3), 24, 59), 54: ((5, 4, 4), 24, 57),
    55: ((5, 5, 4), 24, 66), 56: ((5, 5, 5), 8, 75), 57: ((6, 0, 0), 6, 36),
    58: ((6, 1, 0), 24, 37), 59: ((6, 2, 0), 24, 40), 60: ((6, 3, 0), 24, 45),
    61: ((6, 4, 0), 24, 52), 62: ((6, 5, 0), 24, 61), 63: ((6, 6, 0), 12, 72),
    64: ((6, 1, 1), 24, 38), 65: ((6, 2, 1), 48, 41), 66: ((6, 3, 1), 48, 46),
    67: ((6, 4, 1), 48, 53), 68: ((6, 5, 1), 48, 62), 69: ((6, 6, 1), 24, 73),
    70: ((6, 2, 2), 24, 44), 71: ((6, 3, 2), 48, 49), 72: ((6, 4, 2), 48, 56),
    73: ((6, 5, 2), 48, 65), 74: ((6, 6, 2), 24, 76), 75: ((6, 3, 3), 24, 54),
    76: ((6, 4, 3), 48, 61), 77: ((6, 5, 3), 48, 70), 78: ((6, 6, 3), 24, 81),
    79: ((6, 4, 4), 24, 68), 80: ((6, 5, 4), 48, 77), 81: ((6, 6, 4), 24, 88),
    82: ((6, 5, 5), 24, 86), 83: ((6, 6, 5), 24, 97), 84: ((6, 6, 6), 8, 108),
}


def orbit(group_id):
    """All distinct vectors of group ``group_id``: permutations x signs (Table I, "FS")."""
    base = TABLE_I[group_id][0]
    out = set()
    for perm in itertools.permutations(base):
        for signs in itertools.product((1, -1), repeat=3):
            out.add(tuple(s * c for s, c in zip(signs, perm)))
    return sorted(out)


def length2(group_id):
    """Squared common length ||n_k||^2 of the vectors of a group, from the vector."""
    return sum(c * c for c in TABLE_I[group_id][0])


def length(group_id):
    """Common Euclidean length ||n_k|| of the vectors of a group (Sec. III C)."""
    return math.sqrt(length2(group_id))
