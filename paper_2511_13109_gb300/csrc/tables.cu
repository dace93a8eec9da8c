// Refinement tables of the Kuhn grid hierarchy (Sec. 2, Fig. 2; Eq. 2.4).
//
// Refining a Kuhn tetrahedron (halving the cube size) yields eight children.
// Child membership follows from the ordering rule that defines the
// tetrahedra: a point s of the parent cube (unit coordinates) lies in the
// type-t parent iff s[p0] >= s[p1] >= s[p2]; at a child's centroid the
// inequalities are strict, so evaluating them there in exact integer
// arithmetic (units of 1/8) assigns every child to exactly one parent.
// The local interpolation of Eq. 2.4 is the parent's barycentric coordinate
// vector at the child's vertices; along the Kuhn path these are
// lambda = (1 - s[p0], s[p0] - s[p1], s[p1] - s[p2], s[p2]) and take values in
// {0, 1/2, 1} at child vertices (stored doubled as integers).
#include <cstdio>
#include <cstring>

#include "agca_internal.cuh"

namespace agca {

void build_refine_tables(RefineTables* out) {
  std::memset(out, 0, sizeof(*out));
  for (int t = 0; t < 6; ++t) {
    int k = 0;
    for (int oz = 0; oz < 2; ++oz)
      for (int oy = 0; oy < 2; ++oy)
        for (int ox = 0; ox < 2; ++ox)
          for (int tc = 0; tc < 6; ++tc) {
            const int o[3] = {ox, oy, oz};
            int c8[3];  // 8 * centroid in parent-cube units: 4 o + 3 e_q0 + 2 e_q1 + e_q2
            for (int m = 0; m < 3; ++m) c8[m] = 4 * o[m];
            c8[perm(tc, 0)] += 3;
            c8[perm(tc, 1)] += 2;
            c8[perm(tc, 2)] += 1;
            if (!(c8[perm(t, 0)] > c8[perm(t, 1)] && c8[perm(t, 1)] > c8[perm(t, 2)])) continue;
            out->child[t][k][0] = (int8_t)ox;
            out->child[t][k][1] = (int8_t)oy;
            out->child[t][k][2] = (int8_t)oz;
            out->child[t][k][3] = (int8_t)tc;
            for (int i = 0; i < 4; ++i) {
              const int q = tet_corner(tc, i);
              const int s2[3] = {o[0] + (q & 1), o[1] + ((q >> 1) & 1), o[2] + ((q >> 2) & 1)};
              out->pk2[t][k][i][0] = (int8_t)(2 - s2[perm(t, 0)]);
              out->pk2[t][k][i][1] = (int8_t)(s2[perm(t, 0)] - s2[perm(t, 1)]);
              out->pk2[t][k][i][2] = (int8_t)(s2[perm(t, 1)] - s2[perm(t, 2)]);
              out->pk2[t][k][i][3] = (int8_t)(s2[perm(t, 2)]);
            }
            ++k;
          }
    if (k != 8) std::fprintf(stderr, "agca: refinement table broken (type %d has %d children)\n", t, k);
  }
}

const RefineTables& refine_tables() {
  static const RefineTables tab = [] {
    RefineTables t;
    build_refine_tables(&t);
    return t;
  }();
  return tab;
}

}  // namespace agca
