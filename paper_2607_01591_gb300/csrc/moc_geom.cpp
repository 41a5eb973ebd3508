// Host-side geometry: half-edge mesh, cyclic modular rays over the bounding box, ray-mesh
// intersection by half-edge walk (moc_walk.h, run here or on the device), reflective links and
// tracked areas (Sec. 3.1 of the paper: half-edge traversal of the mesh, modular rays over the
// bounding box of the whole domain, segments computed once before any sweep).
#include "moc_geom.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "moc_gb300.h"

namespace moc {

namespace {

constexpr double kPi = 3.14159265358979323846;

inline double cross(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

}  // namespace

int set_mesh(Geometry &g, int n_vert, const double *xy, int n_tri, const int32_t *tri,
             const int32_t *mat, const double *bbox, const int32_t *bc, std::string &err) {
  if (n_vert < 3 || n_tri < 1 || !xy || !tri || !mat || !bbox || !bc) {
    err = "set_mesh: bad sizes or NULL arrays";
    return MOC_ERR_ARG;
  }
  if (!(bbox[1] > bbox[0]) || !(bbox[3] > bbox[2]) || !std::isfinite(bbox[0]) || !std::isfinite(bbox[1]) ||
      !std::isfinite(bbox[2]) || !std::isfinite(bbox[3])) {
    err = "set_mesh: bad bounding box";
    return MOC_ERR_ARG;
  }
  for (int i = 0; i < 4; ++i)
    if (bc[i] != MOC_BC_VACUUM && bc[i] != MOC_BC_REFLECTIVE) {
      err = "set_mesh: boundary condition must be 0 (vacuum) or 1 (reflective)";
      return MOC_ERR_ARG;
    }
  double tolb = 1e-9 * std::max(bbox[1] - bbox[0], bbox[3] - bbox[2]);
  for (int v = 0; v < n_vert; ++v) {
    double x = xy[2 * v], y = xy[2 * v + 1];
    if (!std::isfinite(x) || !std::isfinite(y) || x < bbox[0] - tolb || x > bbox[1] + tolb || y < bbox[2] - tolb ||
        y > bbox[3] + tolb) {
      err = "set_mesh: vertex " + std::to_string(v) + " is not finite or lies outside the bounding box";
      return MOC_ERR_ARG;
    }
  }
  for (int t = 0; t < n_tri; ++t) {
    for (int k = 0; k < 3; ++k)
      if (tri[3 * t + k] < 0 || tri[3 * t + k] >= n_vert) {
        err = "set_mesh: triangle " + std::to_string(t) + " has a vertex id out of range";
        return MOC_ERR_ARG;
      }
    const double *a = xy + 2 * tri[3 * t], *b = xy + 2 * tri[3 * t + 1], *c = xy + 2 * tri[3 * t + 2];
    if (!(cross(b[0] - a[0], b[1] - a[1], c[0] - a[0], c[1] - a[1]) > 0.0)) {
      err = "set_mesh: triangle " + std::to_string(t) + " is degenerate or not counter-clockwise";
      return MOC_ERR_ARG;
    }
    if (mat[t] < 0) {
      err = "set_mesh: negative material id";
      return MOC_ERR_ARG;
    }
  }
  Geometry ng;
  ng.n_vert = n_vert;
  ng.n_tri = n_tri;
  ng.xy.assign(xy, xy + 2 * (size_t)n_vert);
  ng.tri.assign(tri, tri + 3 * (size_t)n_tri);
  ng.mat.assign(mat, mat + n_tri);
  for (int i = 0; i < 4; ++i) {
    ng.bbox[i] = bbox[i];
    ng.bc[i] = bc[i];
  }
  // half-edge twins by sorting undirected edge keys
  size_t ne = 3 * (size_t)n_tri;
  std::vector<std::pair<uint64_t, int32_t>> keys(ne);
  for (size_t e = 0; e < ne; ++e) {
    uint32_t a = (uint32_t)ng.tri[e], b = (uint32_t)ng.tri[(e / 3) * 3 + (e % 3 + 1) % 3];
    uint64_t lo = std::min(a, b), hi = std::max(a, b);
    keys[e] = {(lo << 32) | hi, (int32_t)e};
  }
  std::sort(keys.begin(), keys.end());
  ng.twin.assign(ne, -1);
  for (size_t i = 0; i < ne;) {
    size_t j = i;
    while (j < ne && keys[j].first == keys[i].first) ++j;
    if (j - i > 2) {
      err = "set_mesh: an edge is shared by more than two triangles";
      return MOC_ERR_ARG;
    }
    if (j - i == 2) {
      int32_t e0 = keys[i].second, e1 = keys[i + 1].second;
      if (ng.tri[e0] == ng.tri[e1]) {
        err = "set_mesh: neighbouring triangles have inconsistent orientation";
        return MOC_ERR_ARG;
      }
      ng.twin[e0] = e1;
      ng.twin[e1] = e0;
    }
    i = j;
  }
  // vertex -> incident triangles
  ng.vt_off.assign(n_vert + 1, 0);
  for (size_t e = 0; e < ne; ++e) ng.vt_off[ng.tri[e] + 1]++;
  for (int v = 0; v < n_vert; ++v) ng.vt_off[v + 1] += ng.vt_off[v];
  ng.vt_list.resize(ne);
  std::vector<int32_t> fill(ng.vt_off.begin(), ng.vt_off.end() - 1);
  for (size_t e = 0; e < ne; ++e) ng.vt_list[fill[ng.tri[e]]++] = (int32_t)(e / 3);
  ng.has_mesh = true;
  // keep a quadrature already set
  ng.n_azim = g.n_azim;
  ng.n_dir = g.n_dir;
  ng.n_polar = g.n_polar;
  ng.spacing = g.spacing;
  ng.sin_theta = g.sin_theta;
  ng.polar_w = g.polar_w;
  ng.has_quad = g.has_quad;
  ng.layout = g.layout;
  g = std::move(ng);
  return MOC_OK;
}

int set_quadrature(Geometry &g, int n_azim, double spacing, int n_polar, const double *sin_theta,
                   const double *polar_w, std::string &err) {
  if (n_azim < 4 || n_azim % 4 != 0 || !(spacing > 0.0) || !std::isfinite(spacing) || n_polar < 1 ||
      n_polar > 6 || !sin_theta || !polar_w) {
    err = "set_quadrature: n_azim must be a positive multiple of 4, spacing > 0, 1 <= n_polar <= 6";
    return MOC_ERR_ARG;
  }
  double wsum = 0.0;
  for (int p = 0; p < n_polar; ++p) {
    if (!(sin_theta[p] > 0.0 && sin_theta[p] <= 1.0) || !(polar_w[p] > 0.0)) {
      err = "set_quadrature: need 0 < sin_theta <= 1 and positive polar weights";
      return MOC_ERR_ARG;
    }
    wsum += polar_w[p];
  }
  if (std::fabs(wsum - 1.0) > 1e-5) {
    err = "set_quadrature: polar weights must sum to 1 over one hemisphere";
    return MOC_ERR_ARG;
  }
  g.n_azim = n_azim;
  g.n_dir = n_azim / 2;
  g.spacing = spacing;
  g.n_polar = n_polar;
  g.sin_theta.assign(sin_theta, sin_theta + n_polar);
  g.polar_w.assign(polar_w, polar_w + n_polar);
  g.has_quad = true;
  g.has_tracks = false;
  return MOC_OK;
}

namespace {

// extent [lo, hi] of the mesh vertices projected on the unit vector (vx, vy)
void projected_extent(const Geometry &g, double vx, double vy, double &lo, double &hi) {
  lo = INFINITY;
  hi = -INFINITY;
  for (int v = 0; v < g.n_vert; ++v) {
    const double c = vx * g.xy[2 * (size_t)v] + vy * g.xy[2 * (size_t)v + 1];
    lo = std::min(lo, c);
    hi = std::max(hi, c);
  }
}

// Direction set over [0, pi) and azimuthal weights over [0, 2 pi). Modular layout: the cyclic
// correction of the angles and spacings over the bounding box. Back projection: the nominal
// angles 2 pi (j + 1/2)/n_azim, and per direction n = ceil(extent/spacing) rays evenly spread
// over the projection of the mesh on the direction's normal (spacing extent/n).
int build_directions(Geometry &g, std::string &err) {
  double W = g.bbox[1] - g.bbox[0], H = g.bbox[3] - g.bbox[2];
  int nd = g.n_dir, nq = g.n_azim / 4;
  g.phi.assign(nd, 0.0);
  g.delta.assign(nd, 0.0);
  g.omega.assign(nd, 0.0);
  g.nx.assign(nd, 0);
  g.ny.assign(nd, 0);
  if (g.layout == MOC_RAYS_BACK_PROJECTION) {
    for (int j = 0; j < nd; ++j) {
      const double ph = 2.0 * kPi * (j + 0.5) / g.n_azim;
      double lo, hi;
      projected_extent(g, -std::sin(ph), std::cos(ph), lo, hi);
      const double ext = hi - lo;
      const int n = std::max(1, (int)std::ceil(ext / g.spacing));
      g.phi[j] = ph;
      g.delta[j] = (ext > 0.0) ? ext / n : g.spacing;
      g.nx[j] = n;
    }
    nq = 0;  // no modular directions below
  }
  for (int a = 0; a < nq; ++a) {
    double nominal = 2.0 * kPi * (a + 0.5) / g.n_azim;
    int nx = (int)std::floor(W * std::sin(nominal) / g.spacing) + 1;
    int ny = (int)std::floor(H * std::cos(nominal) / g.spacing) + 1;
    double ph = std::atan((H * nx) / (W * ny));
    double d = (W / nx) * std::sin(ph);
    int b = nd - 1 - a;  // mirror image pi - phi in the second quadrant
    g.phi[a] = ph;
    g.phi[b] = kPi - ph;
    g.delta[a] = g.delta[b] = d;
    g.nx[a] = g.nx[b] = nx;
    g.ny[a] = g.ny[b] = ny;
  }
  for (int j = 1; j < nd; ++j)
    if (!(g.phi[j] > g.phi[j - 1])) {
      err = "generate_tracks: corrected azimuthal angles are not increasing (ray spacing too coarse)";
      return MOC_ERR_ARG;
    }
  // neighbours over the 2 pi set: angle j + pi has the same weight by point symmetry
  for (int j = 0; j < nd; ++j) {
    double prev = (j == 0) ? g.phi[nd - 1] - kPi : g.phi[j - 1];
    double next = (j == nd - 1) ? g.phi[0] + kPi : g.phi[j + 1];
    g.omega[j] = (next - prev) / (4.0 * kPi);
  }
  return MOC_OK;
}

double box_exit(const Geometry &g, const double *p, const double *u) {
  double s = INFINITY;
  if (u[0] > 0) s = std::min(s, (g.bbox[1] - p[0]) / u[0]);
  if (u[0] < 0) s = std::min(s, (g.bbox[0] - p[0]) / u[0]);
  if (u[1] > 0) s = std::min(s, (g.bbox[3] - p[1]) / u[1]);
  if (u[1] < 0) s = std::min(s, (g.bbox[2] - p[1]) / u[1]);
  return s;
}

walkdef::MeshView mesh_view(const Geometry &g) {
  return walkdef::MeshView{g.xy.data(), g.tri.data(), g.twin.data(), g.vt_off.data(), g.vt_list.data(), g.n_tri};
}

// Host emitter of the walk: pieces and tracks appended to one direction's output (a walk that
// emits no piece is not a track and adds nothing).
struct HostEmit {
  WalkResult *out;
  const double *p0, *u;
  int dir;
  void piece(int t, double l) {
    out->seg_reg.push_back(t);
    out->seg_len.push_back(l);
  }
  void track(double s0, double s1, int64_t n) {
    out->track_dir.push_back(dir);
    out->track_xy.push_back(p0[0] + s0 * u[0]);
    out->track_xy.push_back(p0[1] + s0 * u[1]);
    out->track_xy.push_back(p0[0] + s1 * u[0]);
    out->track_xy.push_back(p0[1] + s1 * u[1]);
    out->seg_count.push_back(n);
  }
};

}  // namespace

int generate_tracks(Geometry &g, std::string &err, const Walker *walker) {
  if (!g.has_mesh || !g.has_quad) {
    err = "generate_tracks: set the mesh and the quadrature first";
    return MOC_ERR_STATE;
  }
  if (g.layout == MOC_RAYS_BACK_PROJECTION)
    for (int i = 0; i < 4; ++i)
      if (g.bc[i] != MOC_BC_VACUUM) {
        err = "generate_tracks: back-projected rays are not cyclic; every boundary must be vacuum";
        return MOC_ERR_ARG;
      }
  int rc = build_directions(g, err);
  if (rc) return rc;
  const double W = g.bbox[1] - g.bbox[0], H = g.bbox[3] - g.bbox[2];
  const double tolw = 1e-9 * std::max(W, H);
  std::vector<int32_t> bnd;
  for (size_t e = 0; e < g.twin.size(); ++e)
    if (g.twin[e] < 0) bnd.push_back((int32_t)e);

  // Rays of every direction (cyclic laydown over the bounding box) and, per ray, the boundary
  // edges it crosses, found by projecting each boundary edge onto the direction's normal.
  // Directions are processed independently (in parallel when OpenMP is on) and concatenated in
  // direction order, so the result does not depend on the thread count.
  struct DirRays {
    std::vector<double> ray;  // x0 y0 L
    std::vector<std::vector<walkdef::Event>> ev;
  };
  std::vector<DirRays> dr(g.n_dir);
  RayBatch rb;
  rb.u.resize(2 * (size_t)g.n_dir);
  for (int j = 0; j < g.n_dir; ++j) {
    rb.u[2 * j] = std::cos(g.phi[j]);
    rb.u[2 * j + 1] = std::sin(g.phi[j]);
  }
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < g.n_dir; ++j) {
    DirRays &D = dr[j];
    const double u[2] = {rb.u[2 * j], rb.u[2 * j + 1]};
    const double nrm[2] = {-u[1], u[0]};
    const int nr = g.nx[j] + g.ny[j];
    std::vector<double> &ray = D.ray;
    ray.resize(3 * (size_t)nr);
    if (g.layout == MOC_RAYS_BACK_PROJECTION) {
      // ray i on the line n . x = lo + (i + 1/2) delta, from where the line enters the
      // bounding box's extent along u to where it leaves it
      double lo, hi, ulo = INFINITY, uhi = -INFINITY;
      projected_extent(g, nrm[0], nrm[1], lo, hi);
      for (int cx = 0; cx < 2; ++cx)
        for (int cy = 0; cy < 2; ++cy) {
          const double t = u[0] * g.bbox[cx] + u[1] * g.bbox[2 + cy];
          ulo = std::min(ulo, t);
          uhi = std::max(uhi, t);
        }
      for (int i = 0; i < nr; ++i) {
        const double c = lo + (i + 0.5) * g.delta[j];
        ray[3 * i] = c * nrm[0] + ulo * u[0];
        ray[3 * i + 1] = c * nrm[1] + ulo * u[1];
        ray[3 * i + 2] = uhi - ulo;
      }
    } else {
      for (int i = 0; i < g.nx[j]; ++i) {
        ray[3 * i] = g.bbox[0] + (i + 0.5) * W / g.nx[j];
        ray[3 * i + 1] = g.bbox[2];
      }
      for (int i = 0; i < g.ny[j]; ++i) {
        int r = g.nx[j] + i;
        ray[3 * r] = (u[0] > 0) ? g.bbox[0] : g.bbox[1];
        ray[3 * r + 1] = g.bbox[2] + (i + 0.5) * H / g.ny[j];
      }
      for (int r = 0; r < nr; ++r) ray[3 * r + 2] = box_exit(g, &ray[3 * r], u);
    }
    // rays sorted by their offset along the normal, to find the rays a boundary edge spans
    std::vector<std::pair<double, int>> off(nr);
    for (int r = 0; r < nr; ++r) off[r] = {nrm[0] * ray[3 * r] + nrm[1] * ray[3 * r + 1], r};
    std::sort(off.begin(), off.end());
    std::vector<std::vector<walkdef::Event>> &ev = D.ev;
    ev.resize(nr);
    for (int32_t he : bnd) {
      int t = he / 3, k = he % 3;
      const double *a = &g.xy[2 * (size_t)g.tri[3 * (size_t)t + k]];
      const double *b = &g.xy[2 * (size_t)g.tri[3 * (size_t)t + (k + 1) % 3]];
      double ca = nrm[0] * a[0] + nrm[1] * a[1], cb = nrm[0] * b[0] + nrm[1] * b[1];
      double clo = std::min(ca, cb) - tolw, chi = std::max(ca, cb) + tolw;
      auto it = std::lower_bound(off.begin(), off.end(), std::make_pair(clo, -1));
      double dx = b[0] - a[0], dy = b[1] - a[1];
      double den = cross(u[0], u[1], dx, dy);
      if (den == 0.0) continue;  // parallel to the ray
      for (; it != off.end() && it->first <= chi; ++it) {
        int r = it->second;
        const double *p0 = &ray[3 * r];
        double ax = a[0] - p0[0], ay = a[1] - p0[1];
        double sp = cross(ax, ay, dx, dy) / den;
        double tt = cross(ax, ay, u[0], u[1]) / den;
        if (tt < -1e-12 || tt > 1.0 + 1e-12) continue;
        if (sp < -walkdef::kEventEps || sp > ray[3 * r + 2] - walkdef::kEventEps) continue;
        ev[r].push_back(walkdef::Event{sp, he, 0, tt});
      }
    }
    for (int r = 0; r < nr; ++r)
      std::sort(ev[r].begin(), ev[r].end(), [](const walkdef::Event &x, const walkdef::Event &y) { return x.s < y.s; });
  }
  // flatten, direction-major
  int64_t n_rays = 0, n_ev = 0;
  for (int j = 0; j < g.n_dir; ++j) {
    n_rays += (int64_t)dr[j].ev.size();
    for (auto &e : dr[j].ev) n_ev += (int64_t)e.size();
  }
  rb.p0.reserve(2 * n_rays);
  rb.len.reserve(n_rays);
  rb.dir.reserve(n_rays);
  rb.ev_off.assign(1, 0);
  rb.ev_off.reserve(n_rays + 1);
  rb.ev.reserve(n_ev);
  for (int j = 0; j < g.n_dir; ++j) {
    DirRays &D = dr[j];
    for (size_t r = 0; r < D.ev.size(); ++r) {
      rb.p0.push_back(D.ray[3 * r]);
      rb.p0.push_back(D.ray[3 * r + 1]);
      rb.len.push_back(D.ray[3 * r + 2]);
      rb.dir.push_back(j);
      rb.ev.insert(rb.ev.end(), D.ev[r].begin(), D.ev[r].end());
      rb.ev_off.push_back((int64_t)rb.ev.size());
    }
    DirRays().ray.swap(D.ray);
    std::vector<std::vector<walkdef::Event>>().swap(D.ev);
  }
  // the walk
  WalkResult wr;
  if (walker) {
    rc = walker->run(walker->ctx, g, rb, wr, err);
    if (rc) return rc;
  } else {
    std::vector<int64_t> dir_ray(g.n_dir + 1, 0);
    for (int64_t r = 0; r < n_rays; ++r) dir_ray[rb.dir[r] + 1]++;
    for (int j = 0; j < g.n_dir; ++j) dir_ray[j + 1] += dir_ray[j];
    std::vector<WalkResult> outs(g.n_dir);
    std::vector<int64_t> lost(g.n_dir, -1);
    const walkdef::MeshView mv = mesh_view(g);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < g.n_dir; ++j) {
      for (int64_t r = dir_ray[j]; r < dir_ray[j + 1]; ++r) {
        HostEmit em{&outs[j], &rb.p0[2 * r], &rb.u[2 * j], j};
        if (walkdef::trace_ray(mv, &rb.p0[2 * r], &rb.u[2 * j], rb.len[r], rb.ev.data() + rb.ev_off[r],
                               rb.ev_off[r + 1] - rb.ev_off[r], em)) {
          lost[j] = r;
          break;
        }
      }
    }
    for (int j = 0; j < g.n_dir; ++j)
      if (lost[j] >= 0) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "generate_tracks: half-edge walk lost on direction %d ray %lld", j,
                      (long long)(lost[j] - dir_ray[j]));
        err = buf;
        return MOC_ERR_GEOMETRY;
      }
    size_t nt = 0, ns = 0;
    for (const WalkResult &o : outs) {
      nt += o.track_dir.size();
      ns += o.seg_reg.size();
    }
    wr.track_dir.reserve(nt);
    wr.track_xy.reserve(4 * nt);
    wr.seg_count.reserve(nt);
    wr.seg_reg.reserve(ns);
    wr.seg_len.reserve(ns);
    for (int j = 0; j < g.n_dir; ++j) {
      WalkResult &o = outs[j];
      wr.track_dir.insert(wr.track_dir.end(), o.track_dir.begin(), o.track_dir.end());
      wr.track_xy.insert(wr.track_xy.end(), o.track_xy.begin(), o.track_xy.end());
      wr.seg_count.insert(wr.seg_count.end(), o.seg_count.begin(), o.seg_count.end());
      wr.seg_reg.insert(wr.seg_reg.end(), o.seg_reg.begin(), o.seg_reg.end());
      wr.seg_len.insert(wr.seg_len.end(), o.seg_len.begin(), o.seg_len.end());
      WalkResult().seg_reg.swap(o.seg_reg);
      std::vector<double>().swap(o.seg_len);
    }
  }
  g.seg_off.assign(1, 0);
  g.seg_off.reserve(wr.seg_count.size() + 1);
  for (int64_t c : wr.seg_count) g.seg_off.push_back(g.seg_off.back() + c);
  g.track_dir.swap(wr.track_dir);
  g.track_xy.swap(wr.track_xy);
  g.seg_reg.swap(wr.seg_reg);
  g.seg_len.swap(wr.seg_len);
  const int64_t T = g.n_tracks();
  if (T == 0) {
    err = "generate_tracks: no ray crosses the mesh";
    return MOC_ERR_GEOMETRY;
  }
  // Reflective links, matched combinatorially: a wall point is identified by its wall and its
  // slot index (i + 1/2) along the wall; reflection maps travel direction j (+ n_dir if
  // reversed) to n_dir - 1 - j, keeping the sense on x walls and flipping it on y walls.
  auto wall_slot = [&](double x, double y, int j, int &w, int64_t &slot) {
    w = -1;
    if (std::fabs(x - g.bbox[0]) <= tolw) w = 0;
    else if (std::fabs(x - g.bbox[1]) <= tolw) w = 1;
    else if (std::fabs(y - g.bbox[2]) <= tolw) w = 2;
    else if (std::fabs(y - g.bbox[3]) <= tolw) w = 3;
    if (w < 0) return false;
    double pos = (w <= 1) ? (y - g.bbox[2]) * g.ny[j] / H : (x - g.bbox[0]) * g.nx[j] / W;
    slot = (int64_t)std::llround(pos - 0.5);
    double back = (w <= 1) ? g.bbox[2] + (slot + 0.5) * H / g.ny[j] : g.bbox[0] + (slot + 0.5) * W / g.nx[j];
    return std::fabs(back - ((w <= 1) ? y : x)) <= tolw;
  };
  std::vector<std::pair<int64_t, int64_t>> incoming;  // key -> end code
  incoming.reserve(2 * T);
  for (int64_t t = 0; t < T; ++t) {
    for (int d = 0; d < 2; ++d) {
      double x = g.track_xy[4 * t + (d ? 2 : 0)], y = g.track_xy[4 * t + (d ? 3 : 1)];
      int w;
      int64_t slot;
      if (!wall_slot(x, y, g.track_dir[t], w, slot)) continue;
      int64_t a2 = g.track_dir[t] + d * g.n_dir;
      incoming.push_back({((a2 * 4 + w) << 32) | slot, 2 * t + d});
    }
  }
  std::sort(incoming.begin(), incoming.end());
  g.link.assign(2 * T, -1);
  for (int64_t t = 0; t < T; ++t) {
    for (int d = 0; d < 2; ++d) {
      double x = g.track_xy[4 * t + (d ? 0 : 2)], y = g.track_xy[4 * t + (d ? 1 : 3)];
      int w;
      int64_t slot;
      if (!wall_slot(x, y, g.track_dir[t], w, slot)) continue;   // leaves through the mesh edge
      if (g.bc[w] != MOC_BC_REFLECTIVE) continue;
      int64_t j2 = g.n_dir - 1 - g.track_dir[t];
      int64_t d2 = (w <= 1) ? d : 1 - d;
      int64_t key = (((j2 + d2 * g.n_dir) * 4 + w) << 32) | slot;
      auto it = std::lower_bound(incoming.begin(), incoming.end(), std::make_pair(key, (int64_t)-1));
      if (it == incoming.end() || it->first != key) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "generate_tracks: no reflective partner for track %lld end %d",
                      (long long)t, d);
        err = buf;
        return MOC_ERR_GEOMETRY;
      }
      g.link[2 * t + d] = it->second;
    }
  }
  // tracked areas: both senses of each track count, with weight omega_j delta_j. One partial sum
  // per direction (tracks are direction-major), added in direction order: the result does not
  // depend on the thread count.
  std::vector<int64_t> dir_trk(g.n_dir + 1, 0);
  for (int64_t t = 0; t < T; ++t) dir_trk[g.track_dir[t] + 1]++;
  for (int j = 0; j < g.n_dir; ++j) dir_trk[j + 1] += dir_trk[j];
  std::vector<std::vector<double>> part(g.n_dir);
#pragma omp parallel for schedule(dynamic, 1)
  for (int j = 0; j < g.n_dir; ++j) {
    std::vector<double> &a = part[j];
    a.assign(g.n_tri, 0.0);
    const double w = 2.0 * g.omega[j] * g.delta[j];
    for (int64_t t = dir_trk[j]; t < dir_trk[j + 1]; ++t)
      for (int64_t s = g.seg_off[t]; s < g.seg_off[t + 1]; ++s) a[g.seg_reg[s]] += w * g.seg_len[s];
  }
  g.area.assign(g.n_tri, 0.0);
  for (int j = 0; j < g.n_dir; ++j) {
    for (int r = 0; r < g.n_tri; ++r) g.area[r] += part[j][r];
    std::vector<double>().swap(part[j]);
  }
  g.has_tracks = true;
  return MOC_OK;
}

}  // namespace moc
