// Segmentation on the GPU: the half-edge walk of moc_walk.h, one thread per ray, in two passes
// (count, then fill at offsets from a host prefix sum). This translation unit is compiled with
// --fmad=false so every double multiply-add rounds twice, as in the host build: the device walk
// takes the same decisions as the host walk and its segments are bit-identical.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "moc_gb300.h"
#include "moc_geom.h"
#include "moc_track.h"

namespace moc {
namespace {

using walkdef::Event;
using walkdef::MeshView;

struct CountEmit {
  int64_t segs = 0;
  int32_t tracks = 0;
  __device__ void piece(int, double) { ++segs; }
  __device__ void track(double, double, int64_t) { ++tracks; }
};

struct FillEmit {
  int32_t *reg;
  double *len;
  int64_t seg;
  int32_t *tdir;
  double *txy;
  int64_t *tcnt;
  int64_t trk;
  const double *p0, *u;
  int dir;
  __device__ void piece(int t, double l) {
    reg[seg] = t;
    len[seg] = l;
    ++seg;
  }
  __device__ void track(double s0, double s1, int64_t n) {
    tdir[trk] = dir;
    txy[4 * trk] = p0[0] + s0 * u[0];
    txy[4 * trk + 1] = p0[1] + s0 * u[1];
    txy[4 * trk + 2] = p0[0] + s1 * u[0];
    txy[4 * trk + 3] = p0[1] + s1 * u[1];
    tcnt[trk] = n;
    ++trk;
  }
};

struct RaysDev {
  const double *p0, *len, *u;
  const int32_t *dir;
  const int64_t *ev_off;
  const Event *ev;
  int64_t n;
};

// pass 1: tracks and segments of each ray; a lost walk records the smallest such ray
__global__ void walk_count_kernel(MeshView m, RaysDev rd, int32_t *__restrict__ n_trk, int64_t *__restrict__ n_seg,
                                  unsigned long long *__restrict__ lost) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rd.n) return;
  const double p0[2] = {rd.p0[2 * r], rd.p0[2 * r + 1]};
  const int j = rd.dir[r];
  const double u[2] = {rd.u[2 * j], rd.u[2 * j + 1]};
  CountEmit em;
  const int rc = walkdef::trace_ray(m, p0, u, rd.len[r], rd.ev + rd.ev_off[r], rd.ev_off[r + 1] - rd.ev_off[r], em);
  if (rc) atomicMin(lost, (unsigned long long)r);
  n_trk[r] = em.tracks;
  n_seg[r] = em.segs;
}

// pass 2: the same walk writing at the ray's offsets
__global__ void walk_fill_kernel(MeshView m, RaysDev rd, const int64_t *__restrict__ trk_base,
                                 const int64_t *__restrict__ seg_base, int32_t *__restrict__ reg,
                                 double *__restrict__ len, int32_t *__restrict__ tdir, double *__restrict__ txy,
                                 int64_t *__restrict__ tcnt) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rd.n) return;
  const double p0[2] = {rd.p0[2 * r], rd.p0[2 * r + 1]};
  const int j = rd.dir[r];
  const double u[2] = {rd.u[2 * j], rd.u[2 * j + 1]};
  FillEmit em{reg, len, seg_base[r], tdir, txy, tcnt, trk_base[r], p0, u, j};
  walkdef::trace_ray(m, p0, u, rd.len[r], rd.ev + rd.ev_off[r], rd.ev_off[r + 1] - rd.ev_off[r], em);
}

// device buffers freed on every return path
struct Bufs {
  std::vector<void *> p;
  ~Bufs() {
    for (void *q : p) cudaFree(q);
  }
  template <typename T> cudaError_t alloc(T *&out, size_t n) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) p.push_back(q);
    out = (T *)q;
    return e;
  }
  template <typename T> cudaError_t put(T *&out, const T *src, size_t n, cudaStream_t st) {
    cudaError_t e = alloc(out, n);
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(out, src, n * sizeof(T), cudaMemcpyHostToDevice, st);
    return e;
  }
};

}  // namespace

int device_walk(void *vctx, const Geometry &g, const RayBatch &rb, WalkResult &out, std::string &err) {
  DeviceWalkCtx &c = *static_cast<DeviceWalkCtx *>(vctx);
  cudaStream_t st = c.stream;
  Bufs b;
  cudaError_t e = cudaSuccess;
#define TRY(call)                                                                   \
  do {                                                                              \
    e = (call);                                                                     \
    if (e != cudaSuccess) {                                                         \
      err = std::string("generate_tracks (device walk): ") + cudaGetErrorString(e); \
      return e == cudaErrorMemoryAllocation ? MOC_ERR_OOM : MOC_ERR_CUDA;           \
    }                                                                               \
  } while (0)
  double *xy;
  int32_t *tri, *twin, *vt_off, *vt_list;
  TRY(b.put(xy, g.xy.data(), g.xy.size(), st));
  TRY(b.put(tri, g.tri.data(), g.tri.size(), st));
  TRY(b.put(twin, g.twin.data(), g.twin.size(), st));
  TRY(b.put(vt_off, g.vt_off.data(), g.vt_off.size(), st));
  TRY(b.put(vt_list, g.vt_list.data(), g.vt_list.size(), st));
  const MeshView m{xy, tri, twin, vt_off, vt_list, g.n_tri};
  const int64_t n = rb.n_rays();
  double *p0, *len, *u;
  int32_t *dir;
  int64_t *ev_off;
  Event *ev;
  TRY(b.put(p0, rb.p0.data(), rb.p0.size(), st));
  TRY(b.put(len, rb.len.data(), rb.len.size(), st));
  TRY(b.put(u, rb.u.data(), rb.u.size(), st));
  TRY(b.put(dir, rb.dir.data(), rb.dir.size(), st));
  TRY(b.put(ev_off, rb.ev_off.data(), rb.ev_off.size(), st));
  TRY(b.put(ev, rb.ev.data(), rb.ev.size(), st));
  const RaysDev rd{p0, len, u, dir, ev_off, ev, n};
  int32_t *n_trk;
  int64_t *n_seg;
  unsigned long long *lost;
  TRY(b.alloc(n_trk, n));
  TRY(b.alloc(n_seg, n));
  TRY(b.alloc(lost, 1));
  TRY(cudaMemsetAsync(lost, 0xff, sizeof(unsigned long long), st));
  cudaEvent_t e0, e1, e2, e3;
  TRY(cudaEventCreate(&e0));
  TRY(cudaEventCreate(&e1));
  TRY(cudaEventCreate(&e2));
  TRY(cudaEventCreate(&e3));
  struct EvFree {
    cudaEvent_t *a;
    ~EvFree() {
      for (int i = 0; i < 4; ++i) cudaEventDestroy(a[i]);
    }
  };
  cudaEvent_t evs[4] = {e0, e1, e2, e3};
  EvFree evfree{evs};
  const int bs = 128;
  const unsigned nb = (unsigned)((n + bs - 1) / bs);
  TRY(cudaEventRecord(e0, st));
  if (n) walk_count_kernel<<<nb, bs, 0, st>>>(m, rd, n_trk, n_seg, lost);
  TRY(cudaGetLastError());
  TRY(cudaEventRecord(e1, st));
  std::vector<int32_t> h_trk(n);
  std::vector<int64_t> h_seg(n);
  unsigned long long h_lost = 0;
  TRY(cudaMemcpyAsync(h_trk.data(), n_trk, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(h_seg.data(), n_seg, n * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(&h_lost, lost, sizeof h_lost, cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  if (h_lost != ~0ull) {
    const int64_t r = (int64_t)h_lost;
    int64_t first = 0;
    while (first < r && rb.dir[first] != rb.dir[r]) ++first;
    char buf[160];
    std::snprintf(buf, sizeof buf, "generate_tracks: half-edge walk lost on direction %d ray %lld", rb.dir[r],
                  (long long)(r - first));
    err = buf;
    return MOC_ERR_GEOMETRY;
  }
  std::vector<int64_t> trk_base(n), seg_base(n);
  int64_t T = 0, S = 0;
  for (int64_t r = 0; r < n; ++r) {
    trk_base[r] = T;
    seg_base[r] = S;
    T += h_trk[r];
    S += h_seg[r];
  }
  int64_t *d_tb, *d_sb, *tcnt;
  int32_t *reg, *tdir;
  double *slen, *txy;
  TRY(b.put(d_tb, trk_base.data(), trk_base.size(), st));
  TRY(b.put(d_sb, seg_base.data(), seg_base.size(), st));
  TRY(b.alloc(reg, S));
  TRY(b.alloc(slen, S));
  TRY(b.alloc(tdir, T));
  TRY(b.alloc(txy, 4 * T));
  TRY(b.alloc(tcnt, T));
  TRY(cudaEventRecord(e2, st));
  if (n) walk_fill_kernel<<<nb, bs, 0, st>>>(m, rd, d_tb, d_sb, reg, slen, tdir, txy, tcnt);
  TRY(cudaGetLastError());
  TRY(cudaEventRecord(e3, st));
  out.seg_reg.resize(S);
  out.seg_len.resize(S);
  out.track_dir.resize(T);
  out.track_xy.resize(4 * T);
  out.seg_count.resize(T);
  TRY(cudaMemcpyAsync(out.seg_reg.data(), reg, S * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(out.seg_len.data(), slen, S * sizeof(double), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(out.track_dir.data(), tdir, T * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(out.track_xy.data(), txy, 4 * T * sizeof(double), cudaMemcpyDeviceToHost, st));
  TRY(cudaMemcpyAsync(out.seg_count.data(), tcnt, T * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  TRY(cudaStreamSynchronize(st));
  float ms_count = 0.f, ms_fill = 0.f;
  TRY(cudaEventElapsedTime(&ms_count, e0, e1));
  TRY(cudaEventElapsedTime(&ms_fill, e2, e3));
  c.walk_ms = (double)ms_count + (double)ms_fill;
#undef TRY
  return MOC_OK;
}

}  // namespace moc
