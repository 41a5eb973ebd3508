// Host-side geometry of the GB300 MOC library: mesh with half-edge adjacency, cyclic ray
// laydown, half-edge-walk segmentation, reflective links and tracked areas (Sec. 3.1).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "moc_walk.h"

namespace moc {

struct Geometry {
  // mesh
  int n_vert = 0, n_tri = 0;
  std::vector<double> xy;        // [V][2]
  std::vector<int32_t> tri;      // [R][3] CCW
  std::vector<int32_t> mat;      // [R]
  double bbox[4] = {0, 0, 0, 0}; // xmin xmax ymin ymax
  int bc[4] = {0, 0, 0, 0};
  // half-edge structure: half-edge e = 3 t + k runs tri[t][k] -> tri[t][(k+1)%3]
  std::vector<int32_t> twin;     // [3R] opposite half-edge or -1 on the boundary
  std::vector<int32_t> vt_off;   // [V+1] vertex -> incident triangles (CSR)
  std::vector<int32_t> vt_list;
  bool has_mesh = false;
  // quadrature
  int n_azim = 0, n_dir = 0, n_polar = 0;
  double spacing = 0;
  std::vector<double> sin_theta, polar_w;
  std::vector<double> phi, delta, omega;   // [n_dir]
  std::vector<int> nx, ny;                 // [n_dir] rays from the bottom / side walls (back projection: nx rays, ny = 0)
  int layout = 0;                          // MOC_RAYS_MODULAR or MOC_RAYS_BACK_PROJECTION
  bool has_quad = false;
  // tracks, in the external order
  std::vector<int64_t> seg_off;    // [T+1]
  std::vector<int32_t> seg_reg;    // [S]
  std::vector<double> seg_len;     // [S]
  std::vector<int32_t> track_dir;  // [T]
  std::vector<double> track_xy;    // [T][4]
  std::vector<int64_t> link;       // [T][2]
  std::vector<double> area;        // [R]
  bool has_tracks = false;

  int64_t n_tracks() const { return (int64_t)track_dir.size(); }
  int64_t n_segments() const { return (int64_t)seg_reg.size(); }
};

// All rays of all directions (direction-major) with their boundary-entry events, the input of the
// half-edge walk (moc_walk.h).
struct RayBatch {
  std::vector<double> p0;       // [n_rays][2] start point (on the bounding box)
  std::vector<double> len;      // [n_rays] parameter where the ray leaves the bounding box
  std::vector<int32_t> dir;     // [n_rays] direction index
  std::vector<double> u;        // [n_dir][2] unit direction
  std::vector<int64_t> ev_off;  // [n_rays+1] events of each ray, sorted by s
  std::vector<walkdef::Event> ev;
  int64_t n_rays() const { return (int64_t)dir.size(); }
};

// What the walk produced, in ray order (tracks of one ray in walk order).
struct WalkResult {
  std::vector<int32_t> track_dir;  // [T]
  std::vector<double> track_xy;    // [T][4]
  std::vector<int64_t> seg_count;  // [T]
  std::vector<int32_t> seg_reg;    // [S]
  std::vector<double> seg_len;     // [S]
};

// A walk run elsewhere (the device): fills `out` from `rays` for the mesh of `g`; returns 0 or a
// negative moc_status with a message in err.
struct Walker {
  int (*run)(void *ctx, const Geometry &g, const RayBatch &rays, WalkResult &out, std::string &err);
  void *ctx;
};

// Each returns 0 on success or a negative moc_status with a message in err.
int set_mesh(Geometry &g, int n_vert, const double *xy, int n_tri, const int32_t *tri,
             const int32_t *mat, const double *bbox, const int32_t *bc, std::string &err);
int set_quadrature(Geometry &g, int n_azim, double spacing, int n_polar, const double *sin_theta,
                   const double *polar_w, std::string &err);
// Ray laydown, segmentation, links, tracked areas. The walk runs on the host (OpenMP over
// directions) unless `walker` is given.
int generate_tracks(Geometry &g, std::string &err, const Walker *walker = nullptr);

}  // namespace moc
