// Ray tracing through the triangle mesh by half-edge walk (Sec. 3.1: ray-mesh intersection by
// HEDS traversal), written once for the host (g++) and the device (nvcc): both compilations use
// IEEE double arithmetic with no contraction of multiply-adds, so the two walks take identical
// decisions and produce bit-identical segments.
#pragma once
#include <cstdint>
#include <cmath>

#ifdef __CUDACC__
#define MOC_HD __host__ __device__ __forceinline__
#else
#define MOC_HD inline
#endif

namespace moc {
namespace walkdef {

constexpr double kSliver = 1e-12;     // pieces shorter than this (cm) are dropped
constexpr double kVertexEps = 1e-12;  // an exit this close (cm) to a vertex crosses the vertex
constexpr double kEventEps = 1e-9;    // entry events closer than this along a ray coincide
constexpr int kMaxFan = 64;           // vertex-fan candidates examined at a boundary vertex

// The mesh as plain arrays: half-edge e = 3 t + k runs tri[t][k] -> tri[t][(k+1)%3].
struct MeshView {
  const double *xy;        // [V][2]
  const int32_t *tri;      // [R][3] counter-clockwise
  const int32_t *twin;     // [3R] opposite half-edge, -1 on the boundary
  const int32_t *vt_off;   // [V+1] vertex -> incident triangles
  const int32_t *vt_list;
  int n_tri;
};

// A boundary half-edge crossed by a ray: ray parameter s, position t in [0, 1] along the edge.
struct Event {
  double s;
  int32_t he;
  int32_t pad;
  double t;
};

// the selection rules of std::min / std::max (first argument on ties)
MOC_HD double dmin(double a, double b) { return (b < a) ? b : a; }
MOC_HD double dmax(double a, double b) { return (a < b) ? b : a; }

// Side test of the line p0 + s u against edge k of triangle t: f0 = n . (p0 - a) and fu = n . u
// with n the inward normal of the counter-clockwise edge a -> b. Both are evaluated from the
// edge's lower-id endpoint and negated for the other orientation, so the two triangles sharing
// an edge get exactly opposite values: a line along the edge is claimed by exactly one of them
// and an exit parameter equals the neighbour's entry parameter bit for bit.
MOC_HD void edge_side(const MeshView &m, int t, int k, const double *p0, const double *u, double &f0, double &fu,
                      double &nx, double &ny) {
  const int ia = m.tri[3 * (size_t)t + k], ib = m.tri[3 * (size_t)t + (k + 1) % 3];
  const bool fwd = ia < ib;
  const double *p = &m.xy[2 * (size_t)(fwd ? ia : ib)];
  const double *q = &m.xy[2 * (size_t)(fwd ? ib : ia)];
  const double cx = -(q[1] - p[1]), cy = q[0] - p[0];  // inward normal of p -> q
  const double g0 = cx * (p0[0] - p[0]) + cy * (p0[1] - p[1]);
  const double gu = cx * u[0] + cy * u[1];
  f0 = fwd ? g0 : -g0;
  fu = fwd ? gu : -gu;
  nx = fwd ? cx : -cx;
  ny = fwd ? cy : -cy;
}

// Interval of the line p0 + s u inside triangle t (Cyrus-Beck half-planes). A line running
// exactly along an edge belongs to the triangle on its left. Returns false if empty.
MOC_HD bool clip(const MeshView &m, int t, const double *p0, const double *u, double &lo, double &hi) {
  lo = -INFINITY;
  hi = INFINITY;
  for (int k = 0; k < 3; ++k) {
    double f0, fu, nx, ny;
    edge_side(m, t, k, p0, u, f0, fu, nx, ny);
    if (fu == 0.0) {
      if (f0 < 0.0) return false;
      if (f0 == 0.0 && (nx * (-u[1]) + ny * u[0]) <= 0.0) return false;
      continue;
    }
    const double s = -f0 / fu;
    if (fu > 0.0) lo = dmax(lo, s);
    else hi = dmin(hi, s);
  }
  return hi > lo;
}

// Walk from triangle t0 (entered at s_start) along the ray until it leaves the mesh, emitting
// (triangle, length) pieces through em.piece(). Returns the exit parameter, or NaN if the walk
// got lost. *npieces counts the pieces emitted.
template <class Emit>
MOC_HD double walk(const MeshView &m, int t0, double s_start, const double *p0, const double *u, double L,
                   Emit &em, int64_t *npieces) {
  int T = t0, prev = -1;
  double s_cur = s_start;
  int64_t np = 0;
  const int64_t limit = 4 * (int64_t)m.n_tri + 64;
  for (int64_t step = 0; step < limit; ++step) {
    double lo, hi;
    if (!clip(m, T, p0, u, lo, hi)) hi = s_cur;
    hi = dmin(hi, L);
    const double l = hi - s_cur;
    if (l > kSliver) {
      em.piece(T, l);
      ++np;
    }
    *npieces = np;
    if (hi >= L) return L;
    // leaving edge: smallest leaving parameter
    int ex = -1;
    double best = INFINITY;
    for (int k = 0; k < 3; ++k) {
      double f0, fu, nx, ny;
      edge_side(m, T, k, p0, u, f0, fu, nx, ny);
      if (fu >= 0.0) continue;
      const double s = -f0 / fu;
      if (s < best) {
        best = s;
        ex = k;
      }
    }
    if (ex < 0) return NAN;
    const double P[2] = {p0[0] + hi * u[0], p0[1] + hi * u[1]};
    const int va = m.tri[3 * (size_t)T + ex], vb = m.tri[3 * (size_t)T + (ex + 1) % 3];
    const double ax = P[0] - m.xy[2 * (size_t)va], ay = P[1] - m.xy[2 * (size_t)va + 1];
    const double bx = P[0] - m.xy[2 * (size_t)vb], by = P[1] - m.xy[2 * (size_t)vb + 1];
    const double da = sqrt(ax * ax + ay * ay), db = sqrt(bx * bx + by * by);
    const int he = 3 * T + ex;
    const int nxt = (m.twin[he] >= 0) ? m.twin[he] / 3 : -1;
    int v = -1;
    if (da <= kVertexEps || db <= kVertexEps) v = (da <= db) ? va : vb;
    else if (nxt == prev && nxt >= 0) v = (da <= db) ? va : vb;  // no progress: resolve at the vertex
    if (v < 0) {
      if (nxt < 0) return hi;  // boundary edge: the ray leaves the mesh
      prev = T;
      T = nxt;
      s_cur = hi;
      continue;
    }
    // vertex crossing: the triangle of the vertex fan the ray continues into
    int pick = -1;
    double pick_hi = hi + kSliver;
    for (int q = m.vt_off[v]; q < m.vt_off[v + 1]; ++q) {
      const int c = m.vt_list[q];
      if (c == T) continue;
      double lo2, hi2;
      if (!clip(m, c, p0, u, lo2, hi2)) continue;
      if (lo2 <= hi + kEventEps && hi2 > pick_hi) {
        pick = c;
        pick_hi = hi2;
      }
    }
    if (pick < 0) return hi;  // leaves the mesh through a boundary vertex
    prev = T;
    T = pick;
    s_cur = hi;
  }
  return NAN;
}

// One ray: its boundary-entry events (sorted by s) each start a walk unless an earlier walk
// already passed them; every walk with pieces becomes a track, reported by
// em.track(s0, s1, n_pieces) after its pieces. Returns 0, or -1 if a walk got lost.
template <class Emit>
MOC_HD int trace_ray(const MeshView &m, const double *p0, const double *u, double L, const Event *ev, int64_t nev,
                     Emit &em) {
  double s_done = -INFINITY;
  for (int64_t q = 0; q < nev; ++q) {
    const Event E = ev[q];
    if (E.s <= s_done + kEventEps) continue;
    // candidate start triangles: owners of the boundary edges hit here, and the vertex fans of
    // edge endpoints hit
    int best = -1;
    double best_lo = 0, best_hi = E.s + kSliver;
    for (int64_t q2 = q; q2 < nev && ev[q2].s <= E.s + kEventEps; ++q2) {
      const Event F = ev[q2];
      const int t = F.he / 3, k = F.he % 3;
      int cands[1 + kMaxFan];
      int nc = 0;
      cands[nc++] = t;
      int vs[2] = {-1, -1};
      if (F.t < 1e-9) vs[0] = m.tri[3 * (size_t)t + k];
      if (F.t > 1.0 - 1e-9) vs[1] = m.tri[3 * (size_t)t + (k + 1) % 3];
      for (int iv = 0; iv < 2; ++iv) {
        const int vv = vs[iv];
        if (vv < 0) continue;
        for (int w = m.vt_off[vv]; w < m.vt_off[vv + 1] && nc < 1 + kMaxFan; ++w) cands[nc++] = m.vt_list[w];
      }
      for (int c = 0; c < nc; ++c) {
        double lo, hi;
        if (!clip(m, cands[c], p0, u, lo, hi)) continue;
        hi = dmin(hi, L);
        if (lo <= E.s + kEventEps && hi > best_hi) {
          best = cands[c];
          best_hi = hi;
          best_lo = lo;
        }
      }
    }
    if (best < 0) continue;
    const double s0 = dmax(0.0, best_lo);
    int64_t n = 0;
    const double s1 = walk(m, best, s0, p0, u, L, em, &n);
    if (s1 != s1) return -1;
    s_done = s1;
    if (n > 0) em.track(s0, s1, n);
  }
  return 0;
}

}  // namespace walkdef
}  // namespace moc
