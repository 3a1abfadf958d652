// Delaunay triangulation of the sparse support points (Sec. III-C "Disparity
// Prior": the prior is built on a Delaunay triangulation of sparse matches, as
// in ELAS).  Host code, double precision, compiled without FP contraction so
// that every machine rounds the predicates identically.
//
// Algorithm: Bowyer-Watson incremental insertion.  The unbounded outside of
// the current hull is covered by "ghost" triangles that share a symbolic
// vertex at infinity, so no finite super-triangle (and none of its precision
// trouble near the hull) is needed:
//   * a finite triangle (a, b, c), counter-clockwise, conflicts with p when p
//     lies strictly inside its circumcircle;
//   * a ghost triangle (a, b, inf) -- hull edge a->b with the outside on its
//     left -- conflicts with p when p is strictly left of a->b, or on the
//     line a-b strictly between a and b.
// Inserting p deletes every conflicting triangle and fans the boundary of the
// deleted cavity to p.  Points are inserted in input order; repeated (x, y)
// are skipped.  With points in general position the result is the unique
// Delaunay triangulation.
#include <cmath>
#include <vector>

#include "lf_internal.h"

namespace lf {
namespace {

constexpr int kInf = -1;

struct Tri {
  int v[3];
};

inline double orient(const double* P, int a, int b, int c) {
  const double ax = P[2 * a], ay = P[2 * a + 1];
  const double bx = P[2 * b], by = P[2 * b + 1];
  const double cx = P[2 * c], cy = P[2 * c + 1];
  return (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
}

// > 0 when d is strictly inside the circumcircle of the ccw triangle (a, b, c).
inline double incircle(const double* P, int a, int b, int c, int d) {
  const double dx = P[2 * d], dy = P[2 * d + 1];
  const double adx = P[2 * a] - dx, ady = P[2 * a + 1] - dy;
  const double bdx = P[2 * b] - dx, bdy = P[2 * b + 1] - dy;
  const double cdx = P[2 * c] - dx, cdy = P[2 * c + 1] - dy;
  const double ab = adx * bdy - bdx * ady;
  const double bc = bdx * cdy - cdx * bdy;
  const double ca = cdx * ady - adx * cdy;
  const double al = adx * adx + ady * ady;
  const double bl = bdx * bdx + bdy * bdy;
  const double cl = cdx * cdx + cdy * cdy;
  return al * bc + bl * ca + cl * ab;
}

bool conflicts(const double* P, const Tri& t, int p) {
  if (t.v[2] != kInf) return incircle(P, t.v[0], t.v[1], t.v[2], p) > 0.0;
  const int a = t.v[0], b = t.v[1];
  const double o = orient(P, a, b, p);
  if (o > 0.0) return true;
  if (o < 0.0) return false;
  // collinear with the hull edge: conflict when strictly inside the segment
  const double ax = P[2 * a], ay = P[2 * a + 1], bx = P[2 * b], by = P[2 * b + 1];
  const double px = P[2 * p], py = P[2 * p + 1];
  const double t0 = (px - ax) * (bx - ax) + (py - ay) * (by - ay);
  const double len = (bx - ax) * (bx - ax) + (by - ay) * (by - ay);
  return t0 > 0.0 && t0 < len;
}

// Rotate so that a symbolic vertex, if any, sits in slot 2 (cyclic order kept).
Tri make_tri(int a, int b, int c) {
  if (a == kInf) return Tri{{b, c, a}};
  if (b == kInf) return Tri{{c, a, b}};
  return Tri{{a, b, c}};
}

}  // namespace

int delaunay(const double* P, int n, int* out, int max_tris) {
  if (n < 3) return 0;
  // seed: first point, first point distinct from it, first point off their line
  int i0 = 0, i1 = -1, i2 = -1;
  for (int i = 1; i < n; ++i)
    if (P[2 * i] != P[0] || P[2 * i + 1] != P[1]) { i1 = i; break; }
  if (i1 < 0) return 0;
  for (int i = i1 + 1; i < n; ++i)
    if (orient(P, i0, i1, i) != 0.0) { i2 = i; break; }
  if (i2 < 0) return 0;  // all points collinear: no triangle
  if (orient(P, i0, i1, i2) < 0.0) { int t = i1; i1 = i2; i2 = t; }

  std::vector<Tri> tris;
  tris.reserve(static_cast<size_t>(2 * n + 8));
  tris.push_back(Tri{{i0, i1, i2}});
  tris.push_back(Tri{{i1, i0, kInf}});
  tris.push_back(Tri{{i2, i1, kInf}});
  tris.push_back(Tri{{i0, i2, kInf}});

  std::vector<char> inserted(static_cast<size_t>(n), 0);
  inserted[i0] = inserted[i1] = inserted[i2] = 1;
  std::vector<char> bad;
  std::vector<int> badlist;
  std::vector<int> edges;  // boundary edges of the cavity, as (from, to) pairs
  for (int p = 0; p < n; ++p) {
    if (inserted[p]) continue;
    inserted[p] = 1;
    bool dup = false;
    for (int q = 0; q < p && !dup; ++q)
      if (q != p && P[2 * q] == P[2 * p] && P[2 * q + 1] == P[2 * p + 1] && inserted[q]) dup = true;
    if (dup) continue;
    bad.assign(tris.size(), 0);
    badlist.clear();
    for (size_t t = 0; t < tris.size(); ++t)
      if (conflicts(P, tris[t], p)) { bad[t] = 1; badlist.push_back(static_cast<int>(t)); }
    if (badlist.empty()) continue;  // cannot happen for a new distinct point; be safe
    // cavity boundary: directed edges of bad triangles whose reverse edge is
    // not also in a bad triangle
    edges.clear();
    for (int t : badlist) {
      for (int e = 0; e < 3; ++e) {
        const int a = tris[t].v[e], b = tris[t].v[(e + 1) % 3];
        bool shared = false;
        for (int s2 : badlist) {
          if (s2 == t) continue;
          for (int f = 0; f < 3; ++f)
            if (tris[s2].v[f] == b && tris[s2].v[(f + 1) % 3] == a) { shared = true; break; }
          if (shared) break;
        }
        if (!shared) { edges.push_back(a); edges.push_back(b); }
      }
    }
    std::vector<Tri> keep;
    keep.reserve(tris.size() + edges.size() / 2);
    for (size_t t = 0; t < tris.size(); ++t)
      if (!bad[t]) keep.push_back(tris[t]);
    for (size_t e = 0; e < edges.size(); e += 2) {
      const int a = edges[e], b = edges[e + 1];
      if (a == kInf && b == kInf) continue;
      keep.push_back(make_tri(a, b, p));
    }
    tris.swap(keep);
  }
  int m = 0;
  for (const Tri& t : tris) {
    if (t.v[2] == kInf) continue;
    if (m < max_tris && out) {
      out[3 * m] = t.v[0];
      out[3 * m + 1] = t.v[1];
      out[3 * m + 2] = t.v[2];
    }
    ++m;
  }
  return m;
}

}  // namespace lf
