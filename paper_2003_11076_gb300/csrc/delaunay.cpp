// Delaunay triangulation of the sparse support points (Sec. III-C "Disparity
// Prior": the prior is built on a Delaunay triangulation of sparse matches, as
// in ELAS).  Host code, double precision, compiled without FP contraction so
// that every machine rounds the predicates identically.
//
// Algorithm: Bowyer-Watson incremental insertion over a triangle mesh with
// neighbour links.  The unbounded outside of the current hull is covered by
// "ghost" triangles sharing a symbolic vertex at infinity, so no finite
// super-triangle (and none of its precision trouble near the hull) is needed:
//   * a finite triangle (a, b, c), counter-clockwise, conflicts with p when p
//     lies strictly inside its circumcircle;
//   * a ghost triangle (a, b, inf) -- hull edge a->b with the outside on its
//     left -- conflicts with p when p is strictly left of a->b, or on the
//     line a-b strictly between a and b.
// Each point is located by a visibility walk from the last inserted
// triangle.  Points are inserted in a biased randomised order: rounds of
// doubling size drawn by a fixed hash of the point index (the same order on
// every machine), each round in Morton order of the coordinates, so the
// walks are short and most points land inside the current hull, where the
// cavities are small.  The conflict cavity is grown from the located triangle
// by breadth-first search over neighbours (it is connected), deleted, and its
// boundary fanned to the new point.  Repeated (x, y) keep their first
// occurrence.  With points in general position the result is the unique
// Delaunay triangulation, independent of the insertion order.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "lf_internal.h"

namespace lf {
namespace {

constexpr int kInf = -1;

struct Tri {
  int v[3];   // counter-clockwise; a ghost has kInf in slot 2
  int nb[3];  // nb[i]: the triangle across the edge opposite v[i]
  bool dead;
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
  const double ax = P[2 * a], ay = P[2 * a + 1], bx = P[2 * b], by = P[2 * b + 1];
  const double px = P[2 * p], py = P[2 * p + 1];
  const double t0 = (px - ax) * (bx - ax) + (py - ay) * (by - ay);
  const double len = (bx - ax) * (bx - ax) + (by - ay) * (by - ay);
  return t0 > 0.0 && t0 < len;
}

uint32_t spread16(uint32_t x) {
  x &= 0xffffu;
  x = (x | (x << 8)) & 0x00ff00ffu;
  x = (x | (x << 4)) & 0x0f0f0f0fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}

class Mesh {
 public:
  // n: number of input points (vertex ids are 0 .. n-1)
  Mesh(const double* P, int n) : P_(P), fan_at_(static_cast<size_t>(n) + 1, 0), fan_stamp_(static_cast<size_t>(n) + 1, 0u) {}

  void seed(int a, int b, int c) {
    // finite (a, b, c) ccw plus three ghosts on its outside
    tris_.clear();
    tris_.push_back(Tri{{a, b, c}, {-1, -1, -1}, false});      // 0
    tris_.push_back(Tri{{b, a, kInf}, {-1, -1, -1}, false});   // 1: across edge a-b
    tris_.push_back(Tri{{c, b, kInf}, {-1, -1, -1}, false});   // 2: across edge b-c
    tris_.push_back(Tri{{a, c, kInf}, {-1, -1, -1}, false});   // 3: across edge c-a
    link_all();
    last_ = 0;
  }

  // Insert point p; returns false when p could not be placed (not expected).
  bool insert(int p) {
    const int t = locate(p);
    if (t < 0) return false;
    // grow the conflict cavity by breadth-first search from t
    cavity_.clear();
    next_stamp();
    mark(t);
    cavity_.push_back(t);
    for (size_t q = 0; q < cavity_.size(); ++q) {
      const int u = cavity_[q];
      for (int i = 0; i < 3; ++i) {
        const int n = tris_[u].nb[i];
        if (n < 0 || marked(n)) continue;
        mark(n);
        if (conflicts(P_, tris_[n], p)) cavity_.push_back(n);
      }
    }
    for (int u : cavity_) tris_[u].dead = true;
    // boundary of the cavity: edge (a -> b) of a dead triangle whose
    // neighbour across it survives (and the slot of that neighbour which
    // points back into the cavity)
    bedges_.clear();
    for (int u : cavity_)
      for (int i = 0; i < 3; ++i) {
        const int n = tris_[u].nb[i];
        if (n >= 0 && tris_[n].dead) continue;
        int back = -1;
        if (n >= 0)
          for (int j = 0; j < 3; ++j)
            if (tris_[n].nb[j] == u) back = j;
        bedges_.push_back(Edge{tris_[u].v[(i + 1) % 3], tris_[u].v[(i + 2) % 3], n, back});
      }
    // fan the boundary to p: triangle (a, b, p), rotated so that a symbolic
    // vertex sits in slot 2; dead slots are reused.  Slot of the edge
    // (a, b): 2 for (a, b, p), 1 for (b, p, inf), 0 for (p, a, inf).
    made_.clear();
    size_t reuse = 0;
    for (const Edge& e : bedges_) {
      int slot;
      if (reuse < cavity_.size()) {
        slot = cavity_[reuse++];
      } else {
        slot = static_cast<int>(tris_.size());
        tris_.push_back(Tri{});
      }
      Tri& T = tris_[slot];
      int s_ab;
      if (e.a == kInf) { T.v[0] = e.b; T.v[1] = p; T.v[2] = kInf; s_ab = 1; }
      else if (e.b == kInf) { T.v[0] = p; T.v[1] = e.a; T.v[2] = kInf; s_ab = 0; }
      else { T.v[0] = e.a; T.v[1] = e.b; T.v[2] = p; s_ab = 2; }
      T.nb[0] = T.nb[1] = T.nb[2] = -1;
      T.dead = false;
      T.nb[s_ab] = e.out;
      if (e.out >= 0) tris_[e.out].nb[e.back] = slot;
      made_.push_back(slot);
    }
    link_fan();
    last_ = made_.empty() ? last_ : made_.back();
    return true;
  }

  int write(int* out, int max_tris) const {
    int m = 0;
    for (const Tri& t : tris_) {
      if (t.dead || t.v[2] == kInf) continue;
      if (out && m < max_tris) {
        out[3 * m] = t.v[0];
        out[3 * m + 1] = t.v[1];
        out[3 * m + 2] = t.v[2];
      }
      ++m;
    }
    return m;
  }

 private:
  struct Edge {
    int a, b, out, back;  // back: the slot of `out` across this edge
  };

  const double* P_;
  std::vector<Tri> tris_;
  std::vector<int> cavity_, made_;
  std::vector<Edge> bedges_;
  std::vector<uint32_t> mark_;
  uint32_t stamp_ = 0;
  int last_ = 0;
  // per vertex (slot 0: the vertex at infinity): index of the boundary edge
  // that starts there in the current fan, valid when its stamp is current
  std::vector<int> fan_at_;
  std::vector<uint32_t> fan_stamp_;
  uint32_t fan_now_ = 0;

  void next_stamp() {
    if (mark_.size() < tris_.size()) mark_.resize(2 * tris_.size() + 64, 0u);  // geometric growth
    if (++stamp_ == 0) {
      std::fill(mark_.begin(), mark_.end(), 0u);
      stamp_ = 1;
    }
  }
  void mark(int t) {
    if (static_cast<size_t>(t) >= mark_.size()) mark_.resize(2 * tris_.size() + 64, 0u);
    mark_[t] = stamp_;
  }
  bool marked(int t) const { return static_cast<size_t>(t) < mark_.size() && mark_[t] == stamp_; }

  // edge (a -> b) of triangle t: slot i with v[i+1] == a, v[i+2] == b
  static int edge_slot(const Tri& T, int a, int b) {
    for (int i = 0; i < 3; ++i)
      if (T.v[(i + 1) % 3] == a && T.v[(i + 2) % 3] == b) return i;
    return -1;
  }

  void link_all() {
    for (size_t t = 0; t < tris_.size(); ++t)
      for (int i = 0; i < 3; ++i) {
        const int a = tris_[t].v[(i + 1) % 3], b = tris_[t].v[(i + 2) % 3];
        for (size_t s = 0; s < tris_.size(); ++s) {
          if (s == t) continue;
          if (edge_slot(tris_[s], b, a) >= 0) { tris_[t].nb[i] = static_cast<int>(s); break; }
        }
      }
  }

  // The new triangle made from boundary edge (a_i -> b_i) meets, across its
  // edge (b_i, p), the new triangle whose boundary edge starts at b_i, across
  // that one's edge (p, a_j).  Slots of (b, p): 0 for (a, b, p), 2 for
  // (b, p, inf), 1 for (p, a, inf); of (p, a): 1, 0 and 2.
  // The cavity boundary is a closed cycle, so every vertex starts exactly
  // one boundary edge: index them by start vertex, then link in one pass.
  void link_fan() {
    const size_t m = made_.size();
    auto slot_bp = [&](const Edge& e) { return e.a == kInf ? 2 : (e.b == kInf ? 1 : 0); };
    auto slot_pa = [&](const Edge& e) { return e.a == kInf ? 0 : (e.b == kInf ? 2 : 1); };
    if (++fan_now_ == 0) {
      std::fill(fan_stamp_.begin(), fan_stamp_.end(), 0u);
      fan_now_ = 1;
    }
    for (size_t j = 0; j < m; ++j) {
      const size_t va = static_cast<size_t>(bedges_[j].a + 1);
      fan_at_[va] = static_cast<int>(j);
      fan_stamp_[va] = fan_now_;
    }
    for (size_t i = 0; i < m; ++i) {
      const size_t vb = static_cast<size_t>(bedges_[i].b + 1);
      if (fan_stamp_[vb] != fan_now_) continue;
      const size_t j = static_cast<size_t>(fan_at_[vb]);
      if (j == i) continue;
      tris_[made_[i]].nb[slot_bp(bedges_[i])] = made_[j];
      tris_[made_[j]].nb[slot_pa(bedges_[j])] = made_[i];
    }
  }

  int find_alive_from(size_t hint) const {
    for (size_t t = std::min(hint, tris_.size() - 1) + 1; t-- > 0;)
      if (!tris_[t].dead) return static_cast<int>(t);
    return 0;
  }

  // Visibility walk to a triangle in conflict with p (a finite triangle
  // containing p, or a ghost whose hull edge sees p); linear scan fallback.
  int locate(int p) {
    int t = (last_ >= 0 && static_cast<size_t>(last_) < tris_.size() && !tris_[last_].dead) ? last_
                                                                                            : find_alive_from(tris_.size());
    const int limit = 4 * static_cast<int>(tris_.size()) + 16;
    for (int step = 0; step < limit; ++step) {
      const Tri& T = tris_[t];
      if (T.v[2] == kInf) {
        if (conflicts(P_, T, p)) return t;
        // step into the finite triangle across the hull edge
        t = T.nb[2];
        if (t < 0) break;
        continue;
      }
      int next = -1;
      const int start = step % 3;
      for (int r = 0; r < 3; ++r) {
        const int i = (start + r) % 3;
        const int a = T.v[(i + 1) % 3], b = T.v[(i + 2) % 3];
        if (orient(P_, a, b, p) < 0.0) { next = T.nb[i]; break; }
      }
      if (next < 0) return conflicts(P_, T, p) ? t : scan(p);
      t = next;
    }
    return scan(p);
  }

  int scan(int p) const {
    for (size_t t = 0; t < tris_.size(); ++t)
      if (!tris_[t].dead && conflicts(P_, tris_[t], p)) return static_cast<int>(t);
    return -1;
  }
};

}  // namespace

int delaunay(const double* P, int n, int* out, int max_tris) {
  if (n < 3) return 0;
  // Morton order (for short walks) in one sort that also brings repeated
  // (x, y) together: key, then x, then y, then index; the first of a run of
  // repeats is the first occurrence
  double x0 = P[0], x1 = x0, y0 = P[1], y1 = y0;
  for (int i = 1; i < n; ++i) {
    x0 = std::min(x0, P[2 * i]); x1 = std::max(x1, P[2 * i]);
    y0 = std::min(y0, P[2 * i + 1]); y1 = std::max(y1, P[2 * i + 1]);
  }
  const double sx = x1 > x0 ? 65535.0 / (x1 - x0) : 0.0, sy = y1 > y0 ? 65535.0 / (y1 - y0) : 0.0;
  std::vector<std::pair<uint32_t, int>> order;
  order.reserve(static_cast<size_t>(n));
  for (int i = 0; i < n; ++i) {
    const uint32_t qx = static_cast<uint32_t>((P[2 * i] - x0) * sx);
    const uint32_t qy = static_cast<uint32_t>((P[2 * i + 1] - y0) * sy);
    order.emplace_back(spread16(qx) | (spread16(qy) << 1), i);
  }
  std::sort(order.begin(), order.end(), [&](const std::pair<uint32_t, int>& u, const std::pair<uint32_t, int>& w) {
    if (u.first != w.first) return u.first < w.first;
    const int a = u.second, b = w.second;
    if (P[2 * a] != P[2 * b]) return P[2 * a] < P[2 * b];
    if (P[2 * a + 1] != P[2 * b + 1]) return P[2 * a + 1] < P[2 * b + 1];
    return a < b;
  });
  std::vector<int> pts;
  pts.reserve(order.size());
  for (size_t i = 0; i < order.size(); ++i) {
    const int q = order[i].second;
    if (i > 0) {
      const int r = order[i - 1].second;
      if (P[2 * q] == P[2 * r] && P[2 * q + 1] == P[2 * r + 1]) continue;
    }
    pts.push_back(q);
  }
  if (pts.size() < 3) return 0;
  {
    auto mix = [](uint64_t z) {  // SplitMix64 finaliser
      z += 0x9e3779b97f4a7c15ull;
      z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
      z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
      return z ^ (z >> 31);
    };
    std::vector<std::pair<uint64_t, int>> byh;  // (hash, Morton position)
    byh.reserve(pts.size());
    for (size_t i = 0; i < pts.size(); ++i) byh.emplace_back(mix(static_cast<uint64_t>(pts[i])), static_cast<int>(i));
    std::sort(byh.begin(), byh.end());
    // hash rank r -> round floor(log2(r + 1)); inside a round, Morton order
    std::vector<std::pair<int, int>> rk;
    rk.reserve(pts.size());
    for (size_t r = 0; r < byh.size(); ++r) {
      int lv = 0;
      while ((2ull << lv) <= r + 1) ++lv;
      rk.emplace_back(lv, byh[r].second);
    }
    std::sort(rk.begin(), rk.end());
    std::vector<int> brio;
    brio.reserve(pts.size());
    for (const auto& q : rk) brio.push_back(pts[q.second]);
    pts.swap(brio);
  }
  // seed: first point, next point, first point off their line
  const int a = pts[0], b = pts[1];
  int c = -1;
  size_t ci = 0;
  for (size_t i = 2; i < pts.size(); ++i)
    if (orient(P, a, b, pts[i]) != 0.0) { c = pts[i]; ci = i; break; }
  if (c < 0) return 0;  // all points collinear
  Mesh mesh(P, n);
  if (orient(P, a, b, c) > 0.0) mesh.seed(a, b, c);
  else mesh.seed(a, c, b);
  for (size_t i = 2; i < pts.size(); ++i) {
    if (i == ci) continue;
    mesh.insert(pts[i]);
  }
  return mesh.write(out, max_tris);
}

}  // namespace lf
