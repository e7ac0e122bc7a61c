// Table I (App. C) and the folded second-order stencils known at compile
// time.  Usable from host and device code (constexpr).
#pragma once

#include <utility>

namespace rlbm {

// Generating vector (a >= b >= c >= 0) of the 84 full-symmetric groups of
// Table I, in table order (row k-1 is group k).
struct TableI {
  int v[84][3];
};
constexpr TableI kTableI = {{
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {1, 1, 1}, {2, 0, 0}, {2, 1, 0}, {2, 2, 0}, {2, 1, 1},
    {2, 2, 1}, {2, 2, 2}, {3, 0, 0}, {3, 1, 0}, {3, 2, 0}, {3, 3, 0}, {3, 1, 1}, {3, 2, 1},
    {3, 2, 2}, {3, 3, 1}, {3, 3, 2}, {3, 3, 3}, {4, 0, 0}, {4, 1, 0}, {4, 2, 0}, {4, 3, 0},
    {4, 4, 0}, {4, 1, 1}, {4, 2, 1}, {4, 3, 1}, {4, 4, 1}, {4, 2, 2}, {4, 3, 2}, {4, 4, 2},
    {4, 3, 3}, {4, 4, 3}, {4, 4, 4}, {5, 0, 0}, {5, 1, 0}, {5, 2, 0}, {5, 3, 0}, {5, 4, 0},
    {5, 5, 0}, {5, 1, 1}, {5, 2, 1}, {5, 3, 1}, {5, 4, 1}, {5, 5, 1}, {5, 2, 2}, {5, 3, 2},
    {5, 4, 2}, {5, 5, 2}, {5, 3, 3}, {5, 4, 3}, {5, 5, 3}, {5, 4, 4}, {5, 5, 4}, {5, 5, 5},
    {6, 0, 0}, {6, 1, 0}, {6, 2, 0}, {6, 3, 0}, {6, 4, 0}, {6, 5, 0}, {6, 6, 0}, {6, 1, 1},
    {6, 2, 1}, {6, 3, 1}, {6, 4, 1}, {6, 5, 1}, {6, 6, 1}, {6, 2, 2}, {6, 3, 2}, {6, 4, 2},
    {6, 5, 2}, {6, 6, 2}, {6, 3, 3}, {6, 4, 3}, {6, 5, 3}, {6, 6, 3}, {6, 4, 4}, {6, 5, 4},
    {6, 6, 4}, {6, 5, 5}, {6, 6, 5}, {6, 6, 6}}};

constexpr int kMaxFolded = 160;

// Folded populations of a six-group stencil: the full-symmetric orbit of each
// group with (nx, ny, +nz) and (nx, ny, -nz) merged.  Order: group by group,
// inside a group by (nx, ny, |nz|) lexicographically -- the host builder uses
// the same order.
struct Folded {
  int Q;
  int halo;
  int grp[kMaxFolded];
  int nx[kMaxFolded], ny[kMaxFolded], nz2[kMaxFolded], mult[kMaxFolded];
};

template <int NG>
constexpr Folded fold_groups(const int (&gs)[NG]) {
  Folded F{};
  int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  F.Q = 0;
  F.halo = 0;
  for (int g = 0; g < NG; ++g) {
    const int* b = kTableI.v[gs[g] - 1];
    // collect distinct (nx, ny, |nz|) with multiplicity = number of distinct
    // 3D vectors mapping to it
    int key[48][3] = {};
    int vec[48][3] = {};
    int nvec = 0;
    for (int p = 0; p < 6; ++p)
      for (int s = 0; s < 8; ++s) {
        int v[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) v[a] = ((s >> a) & 1 ? -1 : 1) * b[perms[p][a]];
        bool seen = false;
        for (int q = 0; q < nvec; ++q)
          if (vec[q][0] == v[0] && vec[q][1] == v[1] && vec[q][2] == v[2]) seen = true;
        if (!seen) {
          vec[nvec][0] = v[0];
          vec[nvec][1] = v[1];
          vec[nvec][2] = v[2];
          ++nvec;
        }
      }
    int nkey = 0;
    int mult[48] = {};
    for (int q = 0; q < nvec; ++q) {
      const int az = vec[q][2] < 0 ? -vec[q][2] : vec[q][2];
      int found = -1;
      for (int k = 0; k < nkey; ++k)
        if (key[k][0] == vec[q][0] && key[k][1] == vec[q][1] && key[k][2] == az) found = k;
      if (found < 0) {
        key[nkey][0] = vec[q][0];
        key[nkey][1] = vec[q][1];
        key[nkey][2] = az;
        mult[nkey] = 1;
        ++nkey;
      } else {
        mult[found] += 1;
      }
    }
    // lexicographic order of the keys
    for (int i = 0; i < nkey; ++i)
      for (int j = i + 1; j < nkey; ++j) {
        bool less = key[j][0] < key[i][0] || (key[j][0] == key[i][0] && key[j][1] < key[i][1]) ||
                    (key[j][0] == key[i][0] && key[j][1] == key[i][1] && key[j][2] < key[i][2]);
        if (less) {
          for (int a = 0; a < 3; ++a) {
            const int t = key[i][a];
            key[i][a] = key[j][a];
            key[j][a] = t;
          }
          const int t = mult[i];
          mult[i] = mult[j];
          mult[j] = t;
        }
      }
    for (int k = 0; k < nkey; ++k) {
      F.grp[F.Q] = g;
      F.nx[F.Q] = key[k][0];
      F.ny[F.Q] = key[k][1];
      F.nz2[F.Q] = key[k][2] * key[k][2];
      F.mult[F.Q] = mult[k];
      const int ax = key[k][0] < 0 ? -key[k][0] : key[k][0];
      const int ay = key[k][1] < 0 ? -key[k][1] : key[k][1];
      if (ax > F.halo) F.halo = ax;
      if (ay > F.halo) F.halo = ay;
      ++F.Q;
    }
  }
  return F;
}

constexpr Folded fold_stencil(int g0, int g1, int g2, int g3, int g4, int g5) {
  const int gs[6] = {g0, g1, g2, g3, g4, g5};
  return fold_groups<6>(gs);
}

// Unfolded six-group stencil for 3D lattices: every vector of the groups'
// orbits, group by group, inside a group by (n_x, n_y, n_z) lexicographically
// (the host's 3D builder uses the same order).
constexpr int kMaxUnfolded = 160;
struct Unfolded {
  int Q;
  int halo;
  int grp[kMaxUnfolded], nx[kMaxUnfolded], ny[kMaxUnfolded], nz[kMaxUnfolded];
};

constexpr Unfolded unfold_stencil(int g0, int g1, int g2, int g3, int g4, int g5) {
  Unfolded U{};
  const int gs[6] = {g0, g1, g2, g3, g4, g5};
  int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  U.Q = 0;
  U.halo = 0;
  for (int g = 0; g < 6; ++g) {
    const int* b = kTableI.v[gs[g] - 1];
    int vec[48][3] = {};
    int nvec = 0;
    for (int p = 0; p < 6; ++p)
      for (int s = 0; s < 8; ++s) {
        int v[3] = {0, 0, 0};
        for (int a = 0; a < 3; ++a) v[a] = ((s >> a) & 1 ? -1 : 1) * b[perms[p][a]];
        bool seen = false;
        for (int q = 0; q < nvec; ++q)
          if (vec[q][0] == v[0] && vec[q][1] == v[1] && vec[q][2] == v[2]) seen = true;
        if (!seen) {
          for (int a = 0; a < 3; ++a) vec[nvec][a] = v[a];
          ++nvec;
        }
      }
    for (int i = 0; i < nvec; ++i)
      for (int j = i + 1; j < nvec; ++j) {
        const bool less = vec[j][0] < vec[i][0] || (vec[j][0] == vec[i][0] && vec[j][1] < vec[i][1]) ||
                          (vec[j][0] == vec[i][0] && vec[j][1] == vec[i][1] && vec[j][2] < vec[i][2]);
        if (less)
          for (int a = 0; a < 3; ++a) {
            const int t = vec[i][a];
            vec[i][a] = vec[j][a];
            vec[j][a] = t;
          }
      }
    for (int q = 0; q < nvec; ++q) {
      U.grp[U.Q] = g;
      U.nx[U.Q] = vec[q][0];
      U.ny[U.Q] = vec[q][1];
      U.nz[U.Q] = vec[q][2];
      for (int a = 0; a < 3; ++a) {
        const int c = vec[q][a] < 0 ? -vec[q][a] : vec[q][a];
        if (c > U.halo) U.halo = c;
      }
      ++U.Q;
    }
  }
  return U;
}

// Compiled 3D stencils (group ids ascending).
template <int G0, int G1, int G2, int G3, int G4, int G5>
struct Stencil3Def {
  static constexpr int groups[6] = {G0, G1, G2, G3, G4, G5};
  static constexpr Unfolded U = unfold_stencil(G0, G1, G2, G3, G4, G5);
  static constexpr int Q = U.Q;
};

using Stencil3M1 = Stencil3Def<5, 12, 14, 17, 21, 26>;
using Stencil3G16 = Stencil3Def<1, 2, 3, 4, 5, 6>;
using Stencil3E5 = Stencil3Def<1, 14, 49, 51, 60, 70>;
using Stencil3S2 = Stencil3Def<3, 9, 10, 14, 17, 21>;

// Reflection orbits of a folded stencil: the populations of one group with
// the same |n_x|, |n_y| and n_z^2 under n_x -> -n_x and n_y -> -n_y.  kind 4:
// quartet, members (+,+), (-,+), (+,-), (-,-); kind 2: (+a_x, 0), (-a_x, 0);
// kind 3: (0, +a_y), (0, -a_y); kind 1: the single population (0, 0).
struct Orbits {
  int K;
  int kind[kMaxFolded], grp[kMaxFolded], ax[kMaxFolded], ay[kMaxFolded], mult[kMaxFolded];
  int idx[kMaxFolded][4];
};

constexpr int find_pop(const Folded& F, int g, int nx, int ny, int nz2) {
  for (int i = 0; i < F.Q; ++i)
    if (F.grp[i] == g && F.nx[i] == nx && F.ny[i] == ny && F.nz2[i] == nz2) return i;
  return -1;
}

constexpr Orbits make_orbits(const Folded& F) {
  Orbits O{};
  O.K = 0;
  for (int i = 0; i < F.Q; ++i) {
    const int nx = F.nx[i], ny = F.ny[i];
    if (nx < 0 || ny < 0) continue;   // the (+,+) member represents the orbit
    const int k = O.K++;
    O.grp[k] = F.grp[i];
    O.ax[k] = nx;
    O.ay[k] = ny;
    O.mult[k] = F.mult[i];
    O.kind[k] = (nx > 0 && ny > 0) ? 4 : (nx > 0) ? 2 : (ny > 0) ? 3 : 1;
    O.idx[k][0] = i;
    O.idx[k][1] = find_pop(F, F.grp[i], -nx, ny, F.nz2[i]);
    O.idx[k][2] = find_pop(F, F.grp[i], nx, -ny, F.nz2[i]);
    O.idx[k][3] = find_pop(F, F.grp[i], -nx, -ny, F.nz2[i]);
  }
  return O;
}

// Every population in exactly one orbit, with the multiplicity of its
// representative (the orbits are closed under the reflections).
constexpr bool orbits_cover(const Folded& F, const Orbits& O) {
  int seen[kMaxFolded] = {};
  for (int k = 0; k < O.K; ++k) {
    const int n = O.kind[k] == 4 ? 4 : (O.kind[k] == 1 ? 1 : 2);
    for (int j = 0; j < n; ++j) {
      const int i = (O.kind[k] == 3 && j == 1) ? O.idx[k][2] : O.idx[k][j];
      if (i < 0 || F.mult[i] != O.mult[k]) return false;
      seen[i] += 1;
    }
  }
  for (int i = 0; i < F.Q; ++i)
    if (seen[i] != 1) return false;
  return true;
}

// Word layout of the BF16-deviation storage: the bfloat16 values of two
// populations share one 32-bit word, so that the writer converts and stores
// them together.  Partners are the members of a reflection orbit that the
// collision relaxes side by side ((+,+) with (-,-), (-,+) with (+,-); the two
// members of a pair orbit); single populations (n = 0) share words among
// themselves, an odd last one a word of its own.  Population i sits in word
// plane word[i], half half[i] (0: low, 1: high).
struct BfWords {
  int words;
  int word[kMaxFolded], half[kMaxFolded];
};

constexpr BfWords make_bf_words(const Folded& F, const Orbits& O) {
  BfWords W{};
  W.words = 0;
  int single = -1;
  for (int k = 0; k < O.K; ++k) {
    const int i0 = O.idx[k][0], i1 = O.idx[k][1], i2 = O.idx[k][2], i3 = O.idx[k][3];
    if (O.kind[k] == 4) {
      W.word[i0] = W.word[i3] = W.words++;
      W.half[i0] = 0, W.half[i3] = 1;
      W.word[i1] = W.word[i2] = W.words++;
      W.half[i1] = 0, W.half[i2] = 1;
    } else if (O.kind[k] == 2) {
      W.word[i0] = W.word[i1] = W.words++;
      W.half[i0] = 0, W.half[i1] = 1;
    } else if (O.kind[k] == 3) {
      W.word[i0] = W.word[i2] = W.words++;
      W.half[i0] = 0, W.half[i2] = 1;
    } else if (single < 0) {
      single = i0;
      W.word[i0] = W.words++;
      W.half[i0] = 0;
    } else {
      W.word[i0] = W.word[single];
      W.half[i0] = 1;
      single = -1;
    }
  }
  (void)F;
  return W;
}

// Every (word, half) slot used by exactly one population.
constexpr bool bf_words_ok(const Folded& F, const BfWords& W) {
  int used[kMaxFolded][2] = {};
  for (int i = 0; i < F.Q; ++i) {
    if (W.word[i] < 0 || W.word[i] >= W.words || W.half[i] < 0 || W.half[i] > 1) return false;
    used[W.word[i]][W.half[i]] += 1;
  }
  for (int w = 0; w < W.words; ++w)
    if (used[w][0] != 1 || used[w][1] > 1) return false;
  return true;
}

// Stencils with compiled fused kernels (group ids ascending).
template <int G0, int G1, int G2, int G3, int G4, int G5>
struct StencilDef {
  static constexpr int groups[6] = {G0, G1, G2, G3, G4, G5};
  static constexpr Folded F = fold_stencil(G0, G1, G2, G3, G4, G5);
  static constexpr int Q = F.Q;
  static constexpr int halo = F.halo;
  static constexpr Orbits O = make_orbits(F);
  static_assert(orbits_cover(F, O), "reflection orbits must partition the folded stencil");
  static constexpr BfWords B = make_bf_words(F, O);
  static_assert(bf_words_ok(F, B), "every population needs its own half of a BF16 word");
  static_assert(B.words == (F.Q + 1) / 2, "BF16 buffers hold Q rounded up to even slots");
};

using StencilM1 = StencilDef<5, 12, 14, 17, 21, 26>;    // m/T_R ~ 1
using StencilG16 = StencilDef<1, 2, 3, 4, 5, 6>;        // m/T_R >~ 5 (Sec. III D example)
using StencilE5 = StencilDef<1, 14, 49, 51, 60, 70>;    // m/T_R in [0.36, 0.58] (Sec. IV, Fig. 5)
using StencilS2 = StencilDef<3, 9, 10, 14, 17, 21>;     // m/T_R in [1.1, 8.4]

// Third-order stencils (eleven groups, ascending) with a compiled FP32 kernel.
template <int... G>
struct StencilO3Def {
  static_assert(sizeof...(G) == 11, "a third-order stencil has eleven groups");
  static constexpr int groups[11] = {G...};
  static constexpr Folded F = fold_groups<11>({G...});
  static constexpr int Q = F.Q;
  static constexpr int halo = F.halo;
  static constexpr Orbits O = make_orbits(F);
  static_assert(orbits_cover(F, O), "reflection orbits must partition the folded stencil");
  static constexpr BfWords B = make_bf_words(F, O);
  static_assert(bf_words_ok(F, B), "every population needs its own half of a BF16 word");
  static_assert(B.words == (F.Q + 1) / 2, "BF16 buffers hold Q rounded up to even slots");
};

using StencilO3M5 = StencilO3Def<1, 2, 5, 6, 7, 9, 10, 11, 12, 13, 15>;   // m/T_R in [4.75, 5.19]
using StencilO3D = StencilO3Def<2, 3, 5, 6, 7, 8, 9, 10, 11, 13, 15>;    // m/T_R in [4.75, 8]
using StencilO3E = StencilO3Def<1, 2, 3, 6, 7, 8, 9, 10, 11, 13, 15>;    // m/T_R in [6.25, 14]
using StencilO3A = StencilO3Def<8, 15, 20, 24, 26, 27, 28, 30, 36, 37, 42>;  // m/T_R in [1.875, 2.25]
using StencilO3B = StencilO3Def<4, 10, 15, 20, 24, 26, 27, 28, 30, 36, 37>;  // m/T_R in [2.0, 3.5]
using StencilO3C = StencilO3Def<4, 8, 14, 15, 16, 17, 18, 21, 22, 23, 26>;   // m/T_R in [3.25, 5.0]

}  // namespace rlbm
