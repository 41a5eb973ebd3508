// C ABI of the GB300 MOC library: context, uploads, the outer-iteration driver and CUDA graphs.
// See include/moc_gb300.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <vector>

#include "moc_gb300.h"
#include "moc_geom.h"
#include "moc_aniso.cuh"
#include "moc_cmfd.cuh"
#include "moc_dg.cuh"
#include "moc_track.h"
#include "moc_kernels.cuh"

using namespace moc;

struct moc_ctx {
  int device = -1;
  int precision = MOC_FP64;
  cudaStream_t stream = nullptr;      // all work is enqueued here
  bool own_stream = false;
  cudaStream_t cap_stream = nullptr;  // graphs are captured here (never the legacy stream)
  std::string err;
  Geometry geo;
  // problem sizes
  int G = 0, Gp = 0, P = 0, M = 0;
  int64_t T = 0, S = 0;
  int order_mode = 0;         // internal track order: 0 longest first, 1 length classes (see upload_tracks)
  std::vector<int64_t> perm;  // internal track -> external track
  std::vector<int64_t> inv;   // external -> internal
  // device data
  void *d_seg = nullptr;
  TrackRec *d_trk = nullptr;
  int32_t *d_link = nullptr;
  uint8_t *d_fed = nullptr;  // per internal track end: 1 if some outgoing end feeds it
  long long *d_inv = nullptr;  // external track -> internal track
  double *h_scal = nullptr;   // pinned, device-mapped copy of the scalars written by state_out_kernel
  bool pageable_ok = false;   // the GPU reads and writes pageable host memory coherently
  void *d_wgt = nullptr, *d_inv_sin = nullptr;
  int32_t *d_mat = nullptr;
  double *d_area = nullptr;
  void *d_sig_t = nullptr, *d_nsf = nullptr, *d_chi = nullptr, *d_sig_s = nullptr;
  void *d_xsq = nullptr, *d_phi = nullptr, *d_tsum = nullptr, *d_tcomp = nullptr;
  void *d_psi[2] = {nullptr, nullptr};
  double *d_fold = nullptr, *d_ext = nullptr, *d_part = nullptr, *d_scal = nullptr;
  void *d_inv_ta = nullptr;    // [R][Gp] 1/(Sigma_t A) in the sweep's type, 0 where the tracked area is 0
  unsigned *d_ticket = nullptr;  // finalize's last-block counter (back to 0 after each launch)
  int2 *d_srange = nullptr;      // [M][G] first and last source group of each scattering column
  void *d_sig_sT = nullptr;      // FP32: [M][G][Gp4] the scattering matrix's columns as rows (many groups)
  int Gp4 = 0;                   // G rounded up to a multiple of 4
  int n_sm = 0;                  // the device's multiprocessor count
  int cur = 0;          // psi buffer holding the incoming flux of the next sweep
  bool eigen = true;
  bool tracks_on_device = false, xs_set = false;
  std::vector<double> h_nsf;  // host copy of nu*Sigma_f [M][G] (normalising a caller's state)
  // anisotropic scattering (off unless moc_set_scattering was called)
  int aniso_L = 0, aniso_NK = 0;
  void *d_ssl = nullptr, *d_harm = nullptr, *d_gm = nullptr, *d_mom = nullptr, *d_srck = nullptr, *d_tmom = nullptr;
  // CMFD acceleration (off unless moc_set_cmfd was called)
  bool cmfd = false;
  int n_cells = 0, n_if = 0, cm_outer = 0, cm_inner = 0, cm_colors = 0;
  double cm_omega = 1.0;
  double cm_tol = 0.0;  // coarse power iteration stops early when k and the source settle to this (0: fixed count)
  int32_t *d_xoff = nullptr, *d_cell = nullptr;
  int2 *d_xent = nullptr;
  int32_t *d_cif_off = nullptr, *d_cif = nullptr, *d_if_cells = nullptr, *d_nbr = nullptr, *d_coff = nullptr;
  size_t cm_smem = 0;  // dynamic shared memory of the coarse solve (0: its working set stays in global memory)
  bool cm_idx16 = false;  // neighbour ids staged as 16-bit
  int cm_cluster = 0;     // CTAs of the cluster coarse solve (0: one-block solve)
  size_t cm_cl_smem = 0;  // its dynamic shared memory per CTA
  int32_t *d_cl = nullptr;  // the cluster solve's ownership arrays (one allocation)
  CmfdCluster cl{};
  void *d_cur = nullptr, *d_leak = nullptr, *d_cphi = nullptr, *d_TV = nullptr, *d_SV = nullptr, *d_FV = nullptr;
  void *d_CHI = nullptr, *d_din = nullptr, *d_diag = nullptr, *d_phic = nullptr, *d_phin = nullptr, *d_fis = nullptr;
  void *d_ratio = nullptr, *d_phio = nullptr, *d_src = nullptr;
  double *d_psum = nullptr, *d_vol = nullptr;  // [N][M][G] flux sums, [N] cell areas
  double *d_cpart = nullptr;
  unsigned *d_cticket = nullptr;
  void *h_stage = nullptr;    // pinned staging buffer for state transfers (grown on demand)
  size_t h_stage_bytes = 0;
  double *d_ostage = nullptr;  // device staging of get_state into pinned host arrays (grown on demand)
  size_t d_ostage_n = 0;
  // DGMOC (off unless moc_set_axial was called): nz planes, bottom/top condition
  int dg_nz = 0;
  int dg_bc[2] = {0, 0};
  size_t dg_res_smem = 0;  // shared memory of the plane-inner sweep per block (0: plane-by-plane sweep)
  // axial coarse-mesh acceleration of DGMOC (planes as coarse cells; off unless moc_set_dg_cmfd)
  int dgcm_outer = 0, dgcm_inner = 0;
  double dgcm_omega = 1.0;
  size_t dgcm_smem = 0;
  void *d_mu = nullptr, *d_dzr = nullptr;
  double *d_dgcur = nullptr, *d_dgleak = nullptr, *d_dgvol = nullptr, *d_dgpsum = nullptr;
  double *d_dgdiag = nullptr, *d_dgphic = nullptr, *d_dgfis = nullptr, *d_dgpart = nullptr;
  void *d_dgcphi = nullptr, *d_dgTV = nullptr, *d_dgSV = nullptr, *d_dgFV = nullptr, *d_dgCHI = nullptr,
       *d_dgratio = nullptr;
  unsigned *d_dgticket = nullptr;
  std::vector<double> h_dz;
  std::vector<int32_t> h_mat3;
  int32_t *d_mat3 = nullptr;
  double *d_dz = nullptr, *d_fold3 = nullptr, *d_part3 = nullptr;
  void *d_cz = nullptr, *d_wdg = nullptr, *d_sin = nullptr, *d_xs3 = nullptr, *d_phi3 = nullptr, *d_tal3 = nullptr;
  void *d_psi3[2] = {nullptr, nullptr};
  void *d_face = nullptr;
  // graphs: [parity of cur at launch]
  cudaGraphExec_t graph2[2] = {nullptr, nullptr};
  // iteration history: (outer count, k, k before, residual) at every host read of the scalars,
  // the last kHistory reads kept (a ring)
  std::vector<double> hist;
  int64_t hist_n = 0;
  // timing
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  double timed_ms = 0.0;
  int64_t timed_n = 0;
};

namespace {

size_t rsize(const moc_ctx *c) { return c->precision == MOC_FP64 ? sizeof(double) : sizeof(float); }
int tally_mode(const moc_ctx *c) { return c->precision == MOC_FP32 ? 1 : 0; }

int fail(moc_ctx *c, int code, const std::string &m) {
  if (c) c->err = m;
  return code;
}

#define CUDA_TRY(c, call)                                                                   \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((c), e_ == cudaErrorMemoryAllocation ? MOC_ERR_OOM : MOC_ERR_CUDA,        \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

void dfree(void *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}
template <typename T> void dfree(T *&p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void drop_graphs(moc_ctx *c) {
  for (auto &g : c->graph2)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

void free_cmfd(moc_ctx *c) {
  drop_graphs(c);
  dfree(c->d_xoff);
  dfree(c->d_xent);
  dfree(c->d_cell);
  dfree(c->d_cif_off);
  dfree(c->d_cif);
  dfree(c->d_if_cells);
  dfree(c->d_nbr);
  dfree(c->d_coff);
  dfree(c->d_cl);
  c->cm_cluster = 0;
  dfree(c->d_cur);
  dfree(c->d_leak);
  dfree(c->d_cphi);
  dfree(c->d_TV);
  dfree(c->d_SV);
  dfree(c->d_FV);
  dfree(c->d_CHI);
  dfree(c->d_din);
  dfree(c->d_diag);
  dfree(c->d_phic);
  dfree(c->d_phin);
  dfree(c->d_fis);
  dfree(c->d_ratio);
  dfree(c->d_phio);
  dfree(c->d_src);
  dfree(c->d_psum);
  dfree(c->d_vol);
  dfree(c->d_cpart);
  dfree(c->d_cticket);
  c->cmfd = false;
}

void free_aniso(moc_ctx *c) {
  drop_graphs(c);
  dfree(c->d_ssl);
  dfree(c->d_harm);
  dfree(c->d_gm);
  dfree(c->d_mom);
  dfree(c->d_srck);
  dfree(c->d_tmom);
  c->aniso_L = c->aniso_NK = 0;
}

void free_dgcm(moc_ctx *c) {
  drop_graphs(c);
  dfree(c->d_mu);
  dfree(c->d_dzr);
  dfree(c->d_dgcur);
  dfree(c->d_dgleak);
  dfree(c->d_dgvol);
  dfree(c->d_dgpsum);
  dfree(c->d_dgdiag);
  dfree(c->d_dgphic);
  dfree(c->d_dgfis);
  dfree(c->d_dgpart);
  dfree(c->d_dgcphi);
  dfree(c->d_dgTV);
  dfree(c->d_dgSV);
  dfree(c->d_dgFV);
  dfree(c->d_dgCHI);
  dfree(c->d_dgratio);
  dfree(c->d_dgticket);
  c->dgcm_outer = 0;
  c->dgcm_smem = 0;
}

void free_dg(moc_ctx *c) {
  free_dgcm(c);
  dfree(c->d_mat3);
  dfree(c->d_dz);
  dfree(c->d_fold3);
  dfree(c->d_part3);
  dfree(c->d_cz);
  dfree(c->d_wdg);
  dfree(c->d_sin);
  dfree(c->d_xs3);
  dfree(c->d_phi3);
  dfree(c->d_tal3);
  dfree(c->d_psi3[0]);
  dfree(c->d_psi3[1]);
  dfree(c->d_face);
  c->dg_nz = 0;
  c->dg_res_smem = 0;
  c->h_dz.clear();
  c->h_mat3.clear();
}

void free_problem(moc_ctx *c) {
  free_cmfd(c);
  free_aniso(c);
  free_dg(c);
  drop_graphs(c);
  dfree(c->d_xsq);
  dfree(c->d_phi);
  dfree(c->d_tsum);
  dfree(c->d_tcomp);
  dfree(c->d_psi[0]);
  dfree(c->d_psi[1]);
  dfree(c->d_fold);
  dfree(c->d_ext);
  dfree(c->d_part);
  dfree(c->d_inv_ta);
  dfree(c->d_ticket);
  dfree(c->d_sig_t);
  dfree(c->d_nsf);
  dfree(c->d_chi);
  dfree(c->d_sig_s);
  dfree(c->d_srange);
  dfree(c->d_sig_sT);
  c->xs_set = false;
}

void free_tracks(moc_ctx *c) {
  free_problem(c);
  dfree(c->d_seg);
  dfree(c->d_trk);
  dfree(c->d_link);
  dfree(c->d_fed);
  dfree(c->d_inv);
  dfree(c->d_wgt);
  dfree(c->d_inv_sin);
  dfree(c->d_mat);
  dfree(c->d_area);
  c->tracks_on_device = false;
}

int need_gpu(moc_ctx *c) {
  if (!c) return MOC_ERR_ARG;
  if (c->device < 0) return fail(c, MOC_ERR_STATE, "host-only context: no GPU work possible");
  return MOC_OK;
}

int need_ready(moc_ctx *c) {
  int rc = need_gpu(c);
  if (rc) return rc;
  if (!c->tracks_on_device) return fail(c, MOC_ERR_STATE, "generate tracks first");
  if (!c->xs_set) return fail(c, MOC_ERR_STATE, "set cross sections first");
  return MOC_OK;
}

template <typename Real> std::vector<Real> to_real(const double *p, size_t n) {
  std::vector<Real> v(n);
  for (size_t i = 0; i < n; ++i) v[i] = (Real)p[i];
  return v;
}

template <typename T> int upload(moc_ctx *c, T *&dst, const T *src, size_t n) {
  CUDA_TRY(c, cudaMalloc((void **)&dst, std::max<size_t>(n, 1) * sizeof(T)));
  if (n) CUDA_TRY(c, cudaMemcpyAsync(dst, src, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MOC_OK;
}

// Pinned host staging of at least `bytes` (reused across calls; freed in moc_destroy).
int stage(moc_ctx *c, size_t bytes, unsigned char *&out) {
  if (bytes > c->h_stage_bytes) {
    if (c->h_stage) cudaFreeHost(c->h_stage);
    c->h_stage = nullptr;
    c->h_stage_bytes = 0;
    CUDA_TRY(c, cudaHostAlloc(&c->h_stage, bytes, cudaHostAllocDefault));
    c->h_stage_bytes = bytes;
  }
  out = (unsigned char *)c->h_stage;
  return MOC_OK;
}

// Upload tracks in the internal order, longest first so that the longest characteristic chains
// start first and neighbouring threads do similar work. order_mode 0: sorted by segment count.
// order_mode 1 (the four-group chunked sweep): sorted by length class, 16 classes per octave of
// segment count, and within a class in laydown order (direction, then position across it), so the
// threads of a warp sweep neighbouring parallel tracks that read and tally the same region rows at
// about the same time (measured 5% faster on the 33-group hex core, 3% slower on the 7-group
// assembly's group-per-thread sweep; on the hex core 16 classes per octave beat 2, 4, 8, 32 and 64).
template <typename Real> int upload_tracks(moc_ctx *c) {
  const Geometry &g = c->geo;
  const int64_t T = g.n_tracks(), S = g.n_segments();
  c->T = T;
  c->S = S;
  c->P = g.n_polar;
  c->perm.resize(T);
  std::iota(c->perm.begin(), c->perm.end(), 0);
  auto len = [&](int64_t t) { return g.seg_off[t + 1] - g.seg_off[t]; };
  if (c->order_mode == 1) {
    auto cls = [&](int64_t t) { return len(t) > 0 ? (int)std::floor(std::log2((double)len(t)) * 16.0) : -1; };
    std::stable_sort(c->perm.begin(), c->perm.end(), [&](int64_t a, int64_t b) { return cls(a) > cls(b); });
  } else {
    std::stable_sort(c->perm.begin(), c->perm.end(), [&](int64_t a, int64_t b) { return len(a) > len(b); });
  }
  c->inv.resize(T);
  for (int64_t i = 0; i < T; ++i) c->inv[c->perm[i]] = i;
  if (2 * T >= (int64_t)1 << 31) return fail(c, MOC_ERR_ARG, "too many tracks for 32-bit links");
  std::vector<TrackRec> trk(T);
  std::vector<int32_t> link(2 * T);
  int64_t o = kSegPad;
  for (int64_t i = 0; i < T; ++i) {
    const int64_t t = c->perm[i];
    const int64_t n = g.seg_off[t + 1] - g.seg_off[t];
    trk[i].off = o;
    trk[i].n = (int)n;
    trk[i].dir = g.track_dir[t];
    o += n;
    for (int d = 0; d < 2; ++d) {
      int64_t e = g.link[2 * t + d];
      link[2 * i + d] = (e < 0) ? -1 : (int32_t)(2 * c->inv[e >> 1] + (e & 1));
    }
  }
  // kSegPad padding records at each end: the sweep's prefetch reads them unconditionally. Every
  // record is written below (tracks in parallel), so the array is not zero-filled first.
  std::unique_ptr<SegRec<Real>[]> seg(new SegRec<Real>[S + 2 * kSegPad]);
  for (int k = 0; k < kSegPad; ++k) {
    std::memset(&seg[k], 0, sizeof(SegRec<Real>));
    std::memset(&seg[kSegPad + S + k], 0, sizeof(SegRec<Real>));
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < T; ++i) {
    const int64_t t = c->perm[i], b = g.seg_off[t];
    for (int64_t k = 0; k < trk[i].n; ++k) {
      SegRec<Real> r;
      std::memset(&r, 0, sizeof r);
      r.r = g.seg_reg[b + k];
      r.l = (Real)g.seg_len[b + k];
      seg[trk[i].off + k] = r;
    }
  }
  std::vector<Real> wgt((size_t)g.n_dir * c->P), inv_sin(c->P);
  for (int j = 0; j < g.n_dir; ++j)
    for (int p = 0; p < c->P; ++p)
      wgt[(size_t)j * c->P + p] = (Real)(kFourPi * g.omega[j] * g.polar_w[p] * g.delta[j] * g.sin_theta[p]);
  for (int p = 0; p < c->P; ++p) inv_sin[p] = (Real)(1.0 / g.sin_theta[p]);
  int rc;
  SegRec<Real> *ds = nullptr;
  if ((rc = upload(c, ds, seg.get(), (size_t)(S + 2 * kSegPad)))) return rc;
  c->d_seg = ds;
  if ((rc = upload(c, c->d_trk, trk.data(), trk.size()))) return rc;
  if ((rc = upload(c, c->d_link, link.data(), link.size()))) return rc;
  std::vector<uint8_t> fed(2 * T, 0);
  for (int32_t e : link)
    if (e >= 0) fed[e] = 1;
  if ((rc = upload(c, c->d_fed, fed.data(), fed.size()))) return rc;
  {
    std::vector<long long> il(c->inv.begin(), c->inv.end());
    if ((rc = upload(c, c->d_inv, il.data(), il.size()))) return rc;
  }
  Real *dw = nullptr, *di = nullptr;
  if ((rc = upload(c, dw, wgt.data(), wgt.size()))) return rc;
  c->d_wgt = dw;
  if ((rc = upload(c, di, inv_sin.data(), inv_sin.size()))) return rc;
  c->d_inv_sin = di;
  if ((rc = upload(c, c->d_mat, g.mat.data(), g.mat.size()))) return rc;
  if ((rc = upload(c, c->d_area, g.area.data(), g.area.size()))) return rc;
  c->tracks_on_device = true;
  return MOC_OK;
}

template <typename Real> int upload_xs(moc_ctx *c, int n_mat, int G, const double *st, const double *nsf,
                                       const double *chi, const double *ss) {
  const Geometry &g = c->geo;
  const int R = g.n_tri;
  c->G = G;
  // padded group count of the region rows: 8 up to 8 groups (one 64/32-byte row per region for the
  // group-per-thread sweep), a multiple of 4 beyond (the chunked sweep's 16-byte loads and atomics)
  c->Gp = G <= 8 ? 8 : (G + 3) & ~3;
  c->M = n_mat;
  const int Gp = c->Gp;
  int rc;
  auto vst = to_real<Real>(st, (size_t)n_mat * G), vnsf = to_real<Real>(nsf, (size_t)n_mat * G),
       vchi = to_real<Real>(chi, (size_t)n_mat * G), vss = to_real<Real>(ss, (size_t)n_mat * G * G);
  Real *p1 = nullptr, *p2 = nullptr, *p3 = nullptr, *p4 = nullptr;
  if ((rc = upload(c, p1, vst.data(), vst.size()))) return rc;
  c->d_sig_t = p1;
  if ((rc = upload(c, p2, vnsf.data(), vnsf.size()))) return rc;
  c->d_nsf = p2;
  if ((rc = upload(c, p3, vchi.data(), vchi.size()))) return rc;
  c->d_chi = p3;
  if ((rc = upload(c, p4, vss.data(), vss.size()))) return rc;
  c->d_sig_s = p4;
  {
    // nonzero band of every scattering column (g' -> g over g'), for the many-group source
    std::vector<int2> band((size_t)n_mat * G);
    for (int m = 0; m < n_mat; ++m)
      for (int g = 0; g < G; ++g) {
        int lo = G, hi = -1;
        for (int gp = 0; gp < G; ++gp)
          if (vss[((size_t)m * G + gp) * G + g] != (Real)0) {
            lo = std::min(lo, gp);
            hi = gp;
          }
        band[(size_t)m * G + g] = (hi < 0) ? make_int2(1, 0) : make_int2(lo, hi);
      }
    if ((rc = upload(c, c->d_srange, band.data(), band.size()))) return rc;
    // FP32 many-group source: each column g (sources g' -> g) stored as a contiguous, 16-byte
    // aligned row, zero-padded to a multiple of 4 groups
    c->Gp4 = (G + 3) & ~3;
    if (sizeof(Real) == 4 && G > 8) {
      std::vector<Real> sT((size_t)n_mat * G * c->Gp4, (Real)0);
      for (int m = 0; m < n_mat; ++m)
        for (int g = 0; g < G; ++g)
          for (int gp = 0; gp < G; ++gp) sT[((size_t)m * G + g) * c->Gp4 + gp] = vss[((size_t)m * G + gp) * G + g];
      Real *dT = nullptr;
      if ((rc = upload(c, dT, sT.data(), sT.size()))) return rc;
      c->d_sig_sT = dT;
    }
  }
  // region pairs {Sigma_t, q/Sigma_t}; padding groups get Sigma_t = 1, q = 0
  std::vector<typename Pair<Real>::T> xsq((size_t)R * Gp);
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < Gp; ++k) {
      typename Pair<Real>::T v;
      v.x = (k < G) ? (Real)st[(size_t)g.mat[r] * G + k] : (Real)1;
      v.y = 0;
      xsq[(size_t)r * Gp + k] = v;
    }
  typename Pair<Real>::T *dx = nullptr;
  if ((rc = upload(c, dx, xsq.data(), xsq.size()))) return rc;
  c->d_xsq = dx;
  // 1/(Sigma_t A) in FP64 from the Sigma_t the sweep uses (rounded to Real)
  std::vector<double> inv_ta((size_t)R * Gp, 0.0);
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < G; ++k) {
      const double A = g.area[r];
      const double sig = (double)(Real)st[(size_t)g.mat[r] * G + k];
      inv_ta[(size_t)r * Gp + k] = (A > 0.0) ? 1.0 / (sig * A) : 0.0;
    }
  {
    std::vector<Real> inv_r(inv_ta.begin(), inv_ta.end());
    Real *di = nullptr;
    if ((rc = upload(c, di, inv_r.data(), inv_r.size()))) return rc;
    c->d_inv_ta = di;
    const unsigned zero = 0;
    if ((rc = upload(c, c->d_ticket, &zero, 1))) return rc;
  }
  const size_t RG = (size_t)R * Gp, PB = (size_t)c->T * 2 * c->P * G;
  CUDA_TRY(c, cudaMalloc(&c->d_phi, RG * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_tsum, RG * sizeof(Real)));
  CUDA_TRY(c, cudaMemsetAsync(c->d_tsum, 0, RG * sizeof(Real), c->stream));
  if (tally_mode(c) == 1) {
    CUDA_TRY(c, cudaMalloc(&c->d_tcomp, RG * sizeof(Real)));
    CUDA_TRY(c, cudaMemsetAsync(c->d_tcomp, 0, RG * sizeof(Real), c->stream));
  }
  for (int b = 0; b < 2; ++b) {
    CUDA_TRY(c, cudaMalloc(&c->d_psi[b], std::max<size_t>(PB, 1) * sizeof(Real)));
    CUDA_TRY(c, cudaMemsetAsync(c->d_psi[b], 0, std::max<size_t>(PB, 1) * sizeof(Real), c->stream));
  }
  CUDA_TRY(c, cudaMalloc(&c->d_fold, (size_t)R * sizeof(double)));
  CUDA_TRY(c, cudaMemsetAsync(c->d_fold, 0, (size_t)R * sizeof(double), c->stream));
  // enough block partials for either finalize variant (4 per block of 32 regions) and for the state
  // kernel's normalisation
  const size_t nb = std::max<size_t>((size_t)(R + 31) / 32 * 4, (RG + 255) / 256);
  CUDA_TRY(c, cudaMalloc(&c->d_part, nb * sizeof(double)));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->xs_set = true;
  return MOC_OK;
}

// state upload: phi [R][G] (NULL: ones) and psi [T][2][P][G] in external track order (NULL: 0)
template <typename Real> int upload_state(moc_ctx *c, const double *phi, const double *psi) {
  const int R = c->geo.n_tri, G = c->G, Gp = c->Gp, P = c->P;
  const size_t per = (size_t)2 * P * G;
  const size_t nphi = (size_t)R * Gp, npsi = (size_t)c->T * per;
  unsigned char *buf;
  int rc = stage(c, (nphi + npsi) * sizeof(Real), buf);
  if (rc) return rc;
  Real *hp = (Real *)buf, *hpsi = hp + nphi;
#pragma omp parallel for schedule(static)
  for (int r = 0; r < R; ++r)
    for (int g = 0; g < Gp; ++g) hp[(size_t)r * Gp + g] = (g < G) ? (Real)(phi ? phi[(size_t)r * G + g] : 1.0) : (Real)0;
  // vacuum boundary: incoming ends that no outgoing end feeds keep zero inflow
  std::vector<char> fed(2 * (size_t)c->T, 0);
  if (psi)
    for (int64_t e : c->geo.link)
      if (e >= 0) fed[e] = 1;
  const size_t half = per / 2;
#pragma omp parallel for schedule(static)
  for (int64_t t = 0; t < c->T; ++t)
    for (int d = 0; d < 2; ++d) {
      Real *dst = hpsi + (size_t)c->inv[t] * per + d * half;
      if (!psi || !fed[2 * t + d]) {
        for (size_t q = 0; q < half; ++q) dst[q] = (Real)0;
      } else {
        const double *src = psi + (size_t)t * per + d * half;
        for (size_t q = 0; q < half; ++q) dst[q] = (Real)src[q];
      }
    }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_phi, hp, nphi * sizeof(Real), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_psi[c->cur], hpsi, npsi * sizeof(Real), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MOC_OK;
}

template <typename Real> int download_state(moc_ctx *c, double scale, double *phi, double *psi) {
  const int R = c->geo.n_tri, G = c->G, Gp = c->Gp, P = c->P;
  const size_t per = (size_t)2 * P * G;
  const size_t nphi = phi ? (size_t)R * Gp : 0, npsi = psi ? (size_t)c->T * per : 0;
  unsigned char *buf;
  int rc = stage(c, (nphi + npsi) * sizeof(Real) + 16, buf);
  if (rc) return rc;
  Real *hp = (Real *)buf, *hpsi = hp + nphi;
  if (phi) CUDA_TRY(c, cudaMemcpyAsync(hp, c->d_phi, nphi * sizeof(Real), cudaMemcpyDeviceToHost, c->stream));
  if (psi) CUDA_TRY(c, cudaMemcpyAsync(hpsi, c->d_psi[c->cur], npsi * sizeof(Real), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (phi) {
#pragma omp parallel for schedule(static)
    for (int r = 0; r < R; ++r)
      for (int g = 0; g < G; ++g) phi[(size_t)r * G + g] = (double)hp[(size_t)r * Gp + g] * scale;
  }
  if (psi) {
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < c->T; ++t) {
      const Real *src = hpsi + (size_t)c->inv[t] * per;
      double *dst = psi + (size_t)t * per;
      for (size_t q = 0; q < per; ++q) dst[q] = (double)src[q] * scale;
    }
  }
  return MOC_OK;
}

// ---------------------------------------------------------------------------------- launches
// the many-group source and finalize kernels (eight threads per region) apply for 8 < G <= 256
bool lane_rows(const moc_ctx *c) { return c->G > 8 && c->Gp <= 256; }

template <typename Real> int launch_source(moc_ctx *c, cudaStream_t st) {
  const int R = c->geo.n_tri;
  if (lane_rows(c)) {
    const unsigned nb = (unsigned)((R + 31) / 32);
    const int gpl = (c->Gp + 7) / 8;
    const size_t sm = (size_t)32 * 8 * gpl * sizeof(Real);  // 32 staged rows of 8 gpl groups
    auto src = gpl == 5 ? source_lanes_kernel<Real, 5> : gpl == 2 ? source_lanes_kernel<Real, 2>
             : gpl == 3 ? source_lanes_kernel<Real, 3> : gpl == 4 ? source_lanes_kernel<Real, 4>
                        : source_lanes_kernel<Real, 0>;
    src<<<nb, 256, sm, st>>>(R, c->G, c->Gp, c->d_mat, (const Real *)c->d_sig_s, (const Real *)c->d_sig_sT, c->Gp4,
                            (const Real *)c->d_nsf, (const Real *)c->d_chi, c->d_srange, c->d_ext,
                            (const Real *)c->d_sig_t, (Real *)c->d_phi, (typename Pair<Real>::T *)c->d_xsq,
                            c->d_fold, c->d_scal, c->eigen ? 1 : 0);
    CUDA_TRY(c, cudaGetLastError());
    return MOC_OK;
  }
  size_t sm = (size_t)c->M * c->G * c->G * sizeof(Real);
  if (sm > 48 * 1024) return fail(c, MOC_ERR_ARG, "scattering tables too large for shared memory (n_mat*G*G)");
  source_kernel<Real><<<(R + 127) / 128, 128, sm, st>>>(
      R, c->G, c->Gp, c->M, c->d_mat, (const Real *)c->d_sig_t, (const Real *)c->d_nsf, (const Real *)c->d_chi,
      (const Real *)c->d_sig_s, c->d_ext, (Real *)c->d_phi, (typename Pair<Real>::T *)c->d_xsq, c->d_fold, c->d_scal,
      c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <typename Real, int P, int TM, bool CM> void sweep_launch(moc_ctx *c, cudaStream_t st) {
  const long long n = (long long)c->T * 2 * c->G;
  const int bs = 128;  // matches the kernel's launch bounds (128 threads, 9 blocks per SM)
  const long long nb = (n + bs - 1) / bs;
  CmfdDev<Real> cm{c->d_xoff, c->d_xent, c->d_cell, (double *)c->d_cur, (double *)c->d_leak};
  sweep_kernel<Real, P, TM, CM><<<(unsigned)nb, bs, 0, st>>>(
      c->d_trk, (const SegRec<Real> *)c->d_seg, c->d_link, (const Real *)c->d_wgt, (const Real *)c->d_inv_sin,
      (const typename Pair<Real>::T *)c->d_xsq, (Real *)c->d_tsum, (Real *)c->d_tcomp,
      (const Real *)c->d_psi[c->cur], (Real *)c->d_psi[c->cur ^ 1], c->d_scal, n, c->G, c->Gp, cm);
}

template <typename Real, int TM, bool CM> int launch_sweep_p(moc_ctx *c, cudaStream_t st) {
  switch (c->P) {
    case 1: sweep_launch<Real, 1, TM, CM>(c, st); break;
    case 2: sweep_launch<Real, 2, TM, CM>(c, st); break;
    case 3: sweep_launch<Real, 3, TM, CM>(c, st); break;
    case 4: sweep_launch<Real, 4, TM, CM>(c, st); break;
    case 5: sweep_launch<Real, 5, TM, CM>(c, st); break;
    case 6: sweep_launch<Real, 6, TM, CM>(c, st); break;
    default: return fail(c, MOC_ERR_ARG, "unsupported polar count");
  }
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

// FP32 with 3 polar angles: ceil(G / (2 NP)) lanes of NP group pairs per track end
template <int TM, int NP = 2> int launch_chunk(moc_ctx *c, cudaStream_t st) {
  const int lanes = (c->G + 2 * NP - 1) / (2 * NP);
  const long long n = (long long)c->T * 2 * lanes;
  PolarInv<3> is;
  for (int p = 0; p < 3; ++p) is.v[p] = (float)(1.0 / c->geo.sin_theta[p]);
  sweep_chunk_kernel<3, TM, NP><<<(unsigned)((n + 63) / 64), 64, 0, st>>>(
      c->d_trk, (const SegRec<float> *)c->d_seg, c->d_link, (const float *)c->d_wgt, is, (const float2 *)c->d_xsq,
      (float *)c->d_tsum, (float *)c->d_tcomp, (const float *)c->d_psi[c->cur], (float *)c->d_psi[c->cur ^ 1],
      c->d_scal, n, c->G, c->Gp, lanes);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <typename Real, int P, int TM, int NK> void aniso_sweep_launch(moc_ctx *c, cudaStream_t st) {
  const long long n = (long long)c->T * 2 * c->G;
  sweep_aniso_kernel<Real, P, TM, NK><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
      c->d_trk, (const SegRec<Real> *)c->d_seg, c->d_link, (const Real *)c->d_wgt, (const Real *)c->d_inv_sin,
      (const Real *)c->d_harm, (const typename Pair<Real>::T *)c->d_xsq, (const Real *)c->d_srck, (Real *)c->d_tsum,
      (Real *)c->d_tcomp, (Real *)c->d_tmom, (const Real *)c->d_psi[c->cur], (Real *)c->d_psi[c->cur ^ 1], c->d_scal,
      n, c->G, c->Gp);
}

template <typename Real, int TM, int NK> int launch_aniso_p(moc_ctx *c, cudaStream_t st) {
  switch (c->P) {
    case 1: aniso_sweep_launch<Real, 1, TM, NK>(c, st); break;
    case 2: aniso_sweep_launch<Real, 2, TM, NK>(c, st); break;
    case 3: aniso_sweep_launch<Real, 3, TM, NK>(c, st); break;
    default: return fail(c, MOC_ERR_ARG, "anisotropic scattering supports up to 3 polar angles");
  }
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <typename Real, int TM> int launch_aniso(moc_ctx *c, cudaStream_t st) {
  switch (c->aniso_NK) {
    case 2: return launch_aniso_p<Real, TM, 2>(c, st);
    case 5: return launch_aniso_p<Real, TM, 5>(c, st);
    default: return launch_aniso_p<Real, TM, 9>(c, st);
  }
}

int launch_sweep(moc_ctx *c, cudaStream_t st) {
  if (c->aniso_L) {
    if (c->precision == MOC_FP64) return launch_aniso<double, 0>(c, st);
    if (c->precision == MOC_FP32) return launch_aniso<float, 1>(c, st);
    return launch_aniso<float, 0>(c, st);
  }
  if (c->cmfd) {
    if (c->precision == MOC_FP64) return launch_sweep_p<double, 0, true>(c, st);
    if (c->precision == MOC_FP32) return launch_sweep_p<float, 1, true>(c, st);
    return launch_sweep_p<float, 0, true>(c, st);
  }
  if (c->precision == MOC_FP64) return launch_sweep_p<double, 0, false>(c, st);
  // many groups: one thread per chunk of 4 groups shares the per-segment cost; few groups: one
  // thread per group keeps each lane's serial chain along a long track short
  if (c->P == 3 && c->G > 8) return c->precision == MOC_FP32 ? launch_chunk<1>(c, st) : launch_chunk<0>(c, st);
  if (c->precision == MOC_FP32) return launch_sweep_p<float, 1, false>(c, st);
  return launch_sweep_p<float, 0, false>(c, st);
}

template <int TM, int GPL> int launch_finalize_bulk_t(moc_ctx *c, cudaStream_t st) {
  const int R = c->geo.n_tri;
  const size_t sm = 2 * (size_t)finalize_bulk_stage_floats(c->Gp, TM, c->eigen ? 1 : 0) * sizeof(float);
  auto fn = finalize_bulk_kernel<TM, GPL>;
  // the opt-in covers dynamic memory beyond what the default leaves next to the static reduction buffers
  CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int per_sm = 0;
  CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, sm));
  per_sm = std::max(1, std::min(per_sm, 8));
  const unsigned nb = (unsigned)std::max(1, std::min((R + 31) / 32, per_sm * std::max(c->n_sm, 1)));
  fn<<<nb, 256, sm, st>>>(R, c->G, c->Gp, c->d_mat, (const float *)c->d_nsf, (const float *)c->d_inv_ta,
                          (const float2 *)c->d_xsq, (float *)c->d_tsum, (float *)c->d_tcomp, (float *)c->d_phi,
                          c->d_fold, c->d_area, c->d_part, c->d_ticket, c->d_scal, c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <int TM> int launch_finalize_bulk_tm(moc_ctx *c, cudaStream_t st) {
  switch ((c->Gp + 7) / 8) {
    case 1: return launch_finalize_bulk_t<TM, 1>(c, st);
    case 2: return launch_finalize_bulk_t<TM, 2>(c, st);
    case 3: return launch_finalize_bulk_t<TM, 3>(c, st);
    case 4: return launch_finalize_bulk_t<TM, 4>(c, st);
    case 5: return launch_finalize_bulk_t<TM, 5>(c, st);
    case 6: return launch_finalize_bulk_t<TM, 6>(c, st);
    case 7: return launch_finalize_bulk_t<TM, 7>(c, st);
    default: return launch_finalize_bulk_t<TM, 8>(c, st);
  }
}

int launch_finalize_bulk(moc_ctx *c, cudaStream_t st) {
  return tally_mode(c) == 1 ? launch_finalize_bulk_tm<1>(c, st) : launch_finalize_bulk_tm<0>(c, st);
}

template <typename Real> int launch_finalize_reduce(moc_ctx *c, cudaStream_t st) {
  const int R = c->geo.n_tri;
  if (c->Gp == 8 && sizeof(Real) == 4) {
    // FP32, one group per lane: the bulk-staged finalize
    if constexpr (sizeof(Real) == 4) return launch_finalize_bulk(c, st);
  }
  if (c->Gp == 8) {
    // 8 lanes per region, 32 regions per block of 256 threads; the last block also reduces
    const int nb8 = (R + 31) / 32;
    if (tally_mode(c) == 1)
      finalize8_kernel<Real, 1><<<nb8, 256, 0, st>>>(
          R, c->G, c->d_mat, (const Real *)c->d_nsf, (const Real *)c->d_inv_ta, (const typename Pair<Real>::T *)c->d_xsq,
          (Real *)c->d_tsum, (Real *)c->d_tcomp, (Real *)c->d_phi, c->d_fold, c->d_area, c->d_part, c->d_ticket,
          c->d_scal, c->eigen ? 1 : 0);
    else
      finalize8_kernel<Real, 0><<<nb8, 256, 0, st>>>(
          R, c->G, c->d_mat, (const Real *)c->d_nsf, (const Real *)c->d_inv_ta, (const typename Pair<Real>::T *)c->d_xsq,
          (Real *)c->d_tsum, (Real *)c->d_tcomp, (Real *)c->d_phi, c->d_fold, c->d_area, c->d_part, c->d_ticket,
          c->d_scal, c->eigen ? 1 : 0);
    CUDA_TRY(c, cudaGetLastError());
    return MOC_OK;
  }
  if (lane_rows(c) && sizeof(Real) == 4 && c->Gp <= 64) {
    // FP32, rows of 12 to 64 groups: tiles of 32 regions staged by bulk copies, double-buffered,
    // as many blocks as fit on the device (at most 8 per multiprocessor)
    if constexpr (sizeof(Real) == 4) return launch_finalize_bulk(c, st);
  }
  if (lane_rows(c)) {
    // tiles of 32 regions, blocks striding over them: at most 8 blocks per multiprocessor
    const unsigned nb = (unsigned)std::max(1, std::min((R + 31) / 32, 8 * std::max(c->n_sm, 1)));
    const bool tm = tally_mode(c) == 1;
    const int gpl = (c->Gp + 7) / 8;
    auto fin = gpl == 5 ? (tm ? finalize_lanes_kernel<Real, 1, 5> : finalize_lanes_kernel<Real, 0, 5>)
             : gpl == 2 ? (tm ? finalize_lanes_kernel<Real, 1, 2> : finalize_lanes_kernel<Real, 0, 2>)
             : gpl == 3 ? (tm ? finalize_lanes_kernel<Real, 1, 3> : finalize_lanes_kernel<Real, 0, 3>)
             : gpl == 4 ? (tm ? finalize_lanes_kernel<Real, 1, 4> : finalize_lanes_kernel<Real, 0, 4>)
                        : (tm ? finalize_lanes_kernel<Real, 1, 0> : finalize_lanes_kernel<Real, 0, 0>);
    fin<<<nb, 256, 0, st>>>(R, c->G, c->Gp, c->d_mat, (const Real *)c->d_nsf, (const Real *)c->d_inv_ta,
                            (const typename Pair<Real>::T *)c->d_xsq, (Real *)c->d_tsum, (Real *)c->d_tcomp,
                            (Real *)c->d_phi, c->d_fold, c->d_area, c->d_part, c->d_ticket, c->d_scal,
                            c->eigen ? 1 : 0);
    CUDA_TRY(c, cudaGetLastError());
    return MOC_OK;
  }
  const int nb = (R + 255) / 256;
  if (tally_mode(c) == 1)
    finalize_kernel<Real, 1><<<nb, 256, 0, st>>>(R, c->G, c->Gp, c->d_mat, (const Real *)c->d_nsf, c->d_area,
                                                 (const Real *)c->d_inv_ta,
                                                 (const typename Pair<Real>::T *)c->d_xsq, (Real *)c->d_tsum,
                                                 (Real *)c->d_tcomp, (Real *)c->d_phi, c->d_fold, c->d_part,
                                                 c->eigen ? 1 : 0);
  else
    finalize_kernel<Real, 0><<<nb, 256, 0, st>>>(R, c->G, c->Gp, c->d_mat, (const Real *)c->d_nsf, c->d_area,
                                                 (const Real *)c->d_inv_ta,
                                                 (const typename Pair<Real>::T *)c->d_xsq, (Real *)c->d_tsum,
                                                 (Real *)c->d_tcomp, (Real *)c->d_phi, c->d_fold, c->d_part,
                                                 c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  reduce_kernel<<<1, 256, 0, st>>>(nb, c->d_part, c->d_scal, c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <typename Real> int launch_aniso_source(moc_ctx *c, cudaStream_t st) {
  const int R = c->geo.n_tri;
  const size_t sm = (size_t)c->aniso_L * c->M * c->G * c->G * sizeof(Real);
  aniso_source_kernel<Real><<<(R + 127) / 128, 128, sm, st>>>(
      R, c->G, c->Gp, c->M, c->aniso_NK, c->d_mat, (const Real *)c->d_ssl, (const typename Pair<Real>::T *)c->d_xsq,
      (Real *)c->d_mom, (Real *)c->d_srck, c->d_scal, c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <typename Real> int launch_aniso_moments(moc_ctx *c, cudaStream_t st) {
  const long long n = (long long)c->geo.n_tri * c->G;
  aniso_moments_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      c->geo.n_tri, c->G, c->Gp, c->aniso_NK, (const Real *)c->d_gm, (const Real *)c->d_inv_ta,
      (typename Pair<Real>::T *)c->d_xsq, (const Real *)c->d_srck, (Real *)c->d_tmom, (Real *)c->d_mom);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <typename Real> int launch_aniso_init(moc_ctx *c, cudaStream_t st) {
  const long long n = (long long)c->geo.n_tri * c->aniso_NK * c->Gp;
  aniso_init_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      c->geo.n_tri, c->G, c->Gp, c->aniso_NK, (const Real *)c->d_gm, (const Real *)c->d_phi, (Real *)c->d_mom);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

// ----------------------------------------------------------------------------- DGMOC launches
template <typename Real> int launch_dg_source(moc_ctx *c, cudaStream_t st) {
  const int R = c->geo.n_tri, E = c->dg_nz * R;
  const size_t sm = (size_t)c->M * c->G * c->G * sizeof(Real);
  dg_source_kernel<Real><<<(E + 127) / 128, 128, sm, st>>>(
      E, R, c->G, c->Gp, c->M, c->d_mat3, (const Real *)c->d_sig_t, (const Real *)c->d_nsf, (const Real *)c->d_chi,
      (const Real *)c->d_sig_s, c->d_ext, (Real *)c->d_phi3, (DgXs<Real> *)c->d_xs3, c->d_fold3, c->d_scal,
      c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

constexpr size_t kDgResSmemMax = 100 * 1024;

template <typename Real, int P> size_t dg_res_smem(int nz) {
  return (size_t)kDgResBlock * nz * (4 * P + 3) * sizeof(Real);
}

template <typename Real, int P> void dg_sweep_launch(moc_ctx *c, cudaStream_t st) {
  const long long n = (long long)c->T * 2 * c->G;
  if (c->dg_res_smem) {
    const unsigned nb = (unsigned)((n + kDgResBlock - 1) / kDgResBlock);
    const DgCm<Real> cm{(const Real *)c->d_mu, (const Real *)c->d_dzr, c->d_dgcur, c->d_dgleak};
    if (c->dgcm_outer && c->eigen)
      dg_sweep_res_kernel<Real, P, true><<<nb, kDgResBlock, c->dgcm_smem, st>>>(
          c->d_trk, (const SegRec<Real> *)c->d_seg, c->d_link, (const Real *)c->d_wdg, (const Real *)c->d_sin,
          (const Real *)c->d_inv_sin, (const Real *)c->d_cz, (const DgXs<Real> *)c->d_xs3, (Real *)c->d_tal3,
          (const Real *)c->d_psi3[c->cur], (Real *)c->d_psi3[c->cur ^ 1], (Real *)c->d_face, c->d_scal, n, c->G,
          c->Gp, c->geo.n_tri, c->dg_nz, c->dg_bc[0], c->dg_bc[1], cm);
    else
      dg_sweep_res_kernel<Real, P, false><<<nb, kDgResBlock, c->dg_res_smem, st>>>(
          c->d_trk, (const SegRec<Real> *)c->d_seg, c->d_link, (const Real *)c->d_wdg, (const Real *)c->d_sin,
          (const Real *)c->d_inv_sin, (const Real *)c->d_cz, (const DgXs<Real> *)c->d_xs3, (Real *)c->d_tal3,
          (const Real *)c->d_psi3[c->cur], (Real *)c->d_psi3[c->cur ^ 1], (Real *)c->d_face, c->d_scal, n, c->G,
          c->Gp, c->geo.n_tri, c->dg_nz, c->dg_bc[0], c->dg_bc[1], cm);
    return;
  }
  dg_sweep_kernel<Real, P><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(
      c->d_trk, (const SegRec<Real> *)c->d_seg, c->d_link, (const Real *)c->d_wdg, (const Real *)c->d_sin,
      (const Real *)c->d_inv_sin, (const Real *)c->d_cz, (const DgXs<Real> *)c->d_xs3, (Real *)c->d_tal3,
      (const Real *)c->d_psi3[c->cur], (Real *)c->d_psi3[c->cur ^ 1], (Real *)c->d_face, c->d_scal, n, c->G, c->Gp,
      c->geo.n_tri, c->dg_nz, c->dg_bc[0], c->dg_bc[1]);
}

template <typename Real> int launch_dg_sweep(moc_ctx *c, cudaStream_t st) {
  if (c->T > 0) {
    switch (c->P) {
      case 1: dg_sweep_launch<Real, 1>(c, st); break;
      case 2: dg_sweep_launch<Real, 2>(c, st); break;
      case 3: dg_sweep_launch<Real, 3>(c, st); break;
      case 4: dg_sweep_launch<Real, 4>(c, st); break;
      default: return fail(c, MOC_ERR_ARG, "DGMOC: up to 4 polar angles");
    }
  }
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

// axial CMFD after finalize and the buffer flip: homogenise per plane, coarse solve, prolong the
// moments, the next sweep's radial boundary flux and the stored top traces
template <typename Real> int launch_dg_cmfd(moc_ctx *c, cudaStream_t st) {
  const int R = c->geo.n_tri, G = c->G, nz = c->dg_nz, E = nz * R;
  CUDA_TRY(c, cudaMemsetAsync(c->d_dgpsum, 0, (size_t)nz * c->M * G * sizeof(double), st));
  const long long neg = (long long)E * G;
  dg_cm_sums_kernel<Real><<<(unsigned)((neg + 255) / 256), 256, 0, st>>>(E, R, G, c->Gp, c->M, c->d_mat3, c->d_area,
                                                                       (const Real *)c->d_dzr, (const Real *)c->d_phi3,
                                                                       c->d_dgpsum);
  cmfd_coeff_kernel<Real><<<(nz * G + 127) / 128, 128, 0, st>>>(
      nz, G, c->M, c->d_dgpsum, c->d_dgvol, (const Real *)c->d_sig_t, (const Real *)c->d_nsf, (const Real *)c->d_chi,
      (const Real *)c->d_sig_s, (Real *)c->d_dgcphi, (Real *)c->d_dgTV, (Real *)c->d_dgSV, (Real *)c->d_dgFV,
      (Real *)c->d_dgCHI);
  dg_cm_solve_kernel<Real><<<1, 256, 0, st>>>(nz, G, c->Gp, c->d_dgcur, c->d_dgleak, (const Real *)c->d_dgcphi,
                                              (const Real *)c->d_dgTV, (const Real *)c->d_dgSV,
                                              (const Real *)c->d_dgFV, (const Real *)c->d_dgCHI, c->d_dgdiag,
                                              c->d_dgphic, c->d_dgfis, (Real *)c->d_dgratio, c->d_scal,
                                              c->dgcm_outer, c->dgcm_inner, c->dgcm_omega);
  dg_cm_prolong_kernel<Real><<<(E + 255) / 256, 256, 0, st>>>(E, R, G, c->Gp, nz, c->d_mat3, (const Real *)c->d_nsf,
                                                              c->d_area, (const Real *)c->d_dzr,
                                                              (const Real *)c->d_dgratio, (Real *)c->d_phi3,
                                                              c->d_dgpart, c->d_dgticket, c->d_scal);
  const long long n_psi = (long long)c->T * 2 * 2 * nz * c->P * 2 * G;
  const long long n_face = (c->dg_bc[1] && c->d_face) ? (long long)(c->S + 2 * kSegPad) * 2 * c->P * G : 0;
  dg_cm_psi_kernel<Real><<<(unsigned)((n_psi + n_face + 255) / 256), 256, 0, st>>>(
      n_psi, n_face, c->P, G, nz, (const Real *)c->d_dgratio, (Real *)c->d_psi3[c->cur], (Real *)c->d_face);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

template <typename Real> int launch_dg_finalize(moc_ctx *c, cudaStream_t st) {
  const int R = c->geo.n_tri, E = c->dg_nz * R;
  const int nb = (E + 255) / 256;
  dg_finalize_kernel<Real><<<nb, 256, 0, st>>>(E, R, c->G, c->Gp, c->d_mat3, (const Real *)c->d_nsf, c->d_area,
                                               c->d_dz, (const DgXs<Real> *)c->d_xs3, (Real *)c->d_tal3,
                                               (Real *)c->d_phi3, c->d_fold3, c->d_part3, c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  reduce_kernel<<<1, 256, 0, st>>>(nb, c->d_part3, c->d_scal, c->eigen ? 1 : 0);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

int enqueue_source(moc_ctx *c, cudaStream_t st) {
  if (c->dg_nz) return c->precision == MOC_FP64 ? launch_dg_source<double>(c, st) : launch_dg_source<float>(c, st);
  int rc = c->precision == MOC_FP64 ? launch_source<double>(c, st) : launch_source<float>(c, st);
  if (rc || !c->aniso_L) return rc;
  return c->precision == MOC_FP64 ? launch_aniso_source<double>(c, st) : launch_aniso_source<float>(c, st);
}

// CMFD after finalize: homogenise, coarse solve, prolong phi and the incoming boundary flux
template <typename Real> int launch_cmfd(moc_ctx *c, cudaStream_t st) {
  const int N = c->n_cells, G = c->G, R = c->geo.n_tri;
  CUDA_TRY(c, cudaMemsetAsync(c->d_psum, 0, (size_t)N * c->M * G * sizeof(double), st));
  const long long nrg = (long long)R * G;
  cmfd_flux_sums_kernel<Real><<<(unsigned)((nrg + 255) / 256), 256, 0, st>>>(R, G, c->Gp, c->M, c->d_cell, c->d_mat,
                                                                          c->d_area, (const Real *)c->d_phi,
                                                                          c->d_psum);
  cmfd_coeff_kernel<Real><<<(N * G + 127) / 128, 128, 0, st>>>(
      N, G, c->M, c->d_psum, c->d_vol, (const Real *)c->d_sig_t, (const Real *)c->d_nsf, (const Real *)c->d_chi,
      (const Real *)c->d_sig_s, (Real *)c->d_cphi, (Real *)c->d_TV, (Real *)c->d_SV, (Real *)c->d_FV,
      (Real *)c->d_CHI);
  CUDA_TRY(c, cudaGetLastError());
  CmfdTopo t{N, G, c->Gp, 2 * c->n_if, c->cm_colors, c->d_nbr, c->d_cif_off, c->d_cif, c->d_if_cells, c->d_coff};
  if (c->cm_cluster) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c->cm_cluster);
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = c->cm_cl_smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = c->cm_cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CUDA_TRY(c, cudaLaunchKernelEx(&cfg, cmfd_solve_cluster_kernel<Real>, t, c->cl, (double *)c->d_cur,
                                   (double *)c->d_leak, (const Real *)c->d_cphi, (const Real *)c->d_TV,
                                   (const Real *)c->d_SV, (const Real *)c->d_FV, (const Real *)c->d_CHI,
                                   (Real *)c->d_din, (Real *)c->d_diag, (Real *)c->d_phic, (Real *)c->d_fis,
                                   (Real *)c->d_ratio, c->d_scal, c->cm_outer, c->cm_inner, (Real)c->cm_omega,
                                   c->cm_tol));
  } else {
  auto solve = !c->cm_smem ? cmfd_solve_kernel<Real, false, int32_t>
               : c->cm_idx16 ? cmfd_solve_kernel<Real, true, uint16_t> : cmfd_solve_kernel<Real, true, int32_t>;
  solve<<<1, 1024, c->cm_smem, st>>>(t, (double *)c->d_cur, (double *)c->d_leak, (const Real *)c->d_cphi,
                                     (const Real *)c->d_TV, (const Real *)c->d_SV, (const Real *)c->d_FV,
                                     (const Real *)c->d_CHI, (Real *)c->d_din, (Real *)c->d_diag,
                                     (Real *)c->d_phic, (Real *)c->d_phin, (Real *)c->d_phio,
                                     (Real *)c->d_src, (Real *)c->d_fis, (Real *)c->d_ratio, c->d_scal,
                                     c->cm_outer, c->cm_inner, (Real)c->cm_omega, c->cm_tol);
  }
  CUDA_TRY(c, cudaGetLastError());
  cmfd_prolong_kernel<Real><<<(R + 255) / 256, 256, 0, st>>>(R, G, c->Gp, N, c->d_cell, c->d_mat, (const Real *)c->d_nsf,
                                                             c->d_area, (const Real *)c->d_ratio, (Real *)c->d_phi,
                                                             c->d_cpart, c->d_cticket, c->d_scal);
  CUDA_TRY(c, cudaGetLastError());
  const long long n = (long long)c->T * 2 * G;
  cmfd_psi_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      n, c->P, G, N, c->d_trk, (const SegRec<Real> *)c->d_seg, c->d_fed, c->d_cell, (const Real *)c->d_ratio,
      (Real *)c->d_psi[c->cur]);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

// sweep + finalize + reduce; flips the boundary-flux buffer
int enqueue_sweep(moc_ctx *c, cudaStream_t st, bool timed) {
  int rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (timed) {
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    CUDA_TRY(c, cudaEventRecord(e0, st));
  }
  if (c->dg_nz) rc = c->precision == MOC_FP64 ? launch_dg_sweep<double>(c, st) : launch_dg_sweep<float>(c, st);
  else rc = launch_sweep(c, st);
  if (rc) return rc;
  if (timed) {
    CUDA_TRY(c, cudaEventRecord(e1, st));
    c->ev.push_back({e0, e1});
  }
  if (c->dg_nz) {
    rc = c->precision == MOC_FP64 ? launch_dg_finalize<double>(c, st) : launch_dg_finalize<float>(c, st);
    c->cur ^= 1;
    if (!rc && c->dgcm_outer && c->eigen)
      rc = c->precision == MOC_FP64 ? launch_dg_cmfd<double>(c, st) : launch_dg_cmfd<float>(c, st);
    return rc;
  }
  if (c->aniso_L) {
    rc = c->precision == MOC_FP64 ? launch_aniso_moments<double>(c, st) : launch_aniso_moments<float>(c, st);
    if (rc) return rc;
  }
  rc = c->precision == MOC_FP64 ? launch_finalize_reduce<double>(c, st) : launch_finalize_reduce<float>(c, st);
  if (rc) return rc;
  c->cur ^= 1;
  if (c->cmfd) rc = c->precision == MOC_FP64 ? launch_cmfd<double>(c, st) : launch_cmfd<float>(c, st);
  return rc;
}

int enqueue_outer(moc_ctx *c, cudaStream_t st, bool timed) {
  int rc = enqueue_source(c, st);
  if (rc) return rc;
  return enqueue_sweep(c, st, timed);
}

// Graph of two outers (the boundary-flux buffers swap twice, so the graph for a given starting
// buffer can be relaunched any number of times).
int get_graph(moc_ctx *c, cudaGraphExec_t &out) {
  cudaGraphExec_t &ge = c->graph2[c->cur];
  if (!ge) {
    const int cur0 = c->cur;
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_outer(c, c->cap_stream, false);
    if (!rc) rc = enqueue_outer(c, c->cap_stream, false);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &gr);
    c->cur = cur0;
    if (rc) {
      if (gr) cudaGraphDestroy(gr);
      return rc;
    }
    if (e != cudaSuccess) return fail(c, MOC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&ge, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      ge = nullptr;
      return fail(c, MOC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
  }
  out = ge;
  return MOC_OK;
}

int run_outers(moc_ctx *c, int n) {
  int rc;
  if (c->timing) {
    for (int i = 0; i < n; ++i)
      if ((rc = enqueue_outer(c, c->stream, true))) return rc;
    return MOC_OK;
  }
  int pairs = n / 2;
  for (int i = 0; i < pairs; ++i) {
    cudaGraphExec_t ge;
    if ((rc = get_graph(c, ge))) return rc;
    CUDA_TRY(c, cudaGraphLaunch(ge, c->stream));
    // two outers: the buffer parity is unchanged
  }
  if (n % 2)
    if ((rc = enqueue_outer(c, c->stream, false))) return rc;
  return MOC_OK;
}

constexpr int kHistory = 4096;

void record_history(moc_ctx *c, const double *s) {
  if (c->hist.size() != 4 * (size_t)kHistory) c->hist.assign(4 * (size_t)kHistory, 0.0);
  double *h = &c->hist[4 * (size_t)(c->hist_n % kHistory)];
  h[0] = s[S_NOUTER];
  h[1] = s[S_K];
  h[2] = s[S_KPREV];
  h[3] = s[S_RESID];
  ++c->hist_n;
}

int read_scalars(moc_ctx *c, double *s) {
  CUDA_TRY(c, cudaMemcpyAsync(s, c->d_scal, S_COUNT * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MOC_OK;
}

int reset_scalars(moc_ctx *c, double k, double scale) {
  double s[S_COUNT] = {0};
  s[S_K] = k;
  s[S_KPREV] = k;
  s[S_SCALE] = scale;
  s[S_RESID] = INFINITY;
  s[S_FISS] = 1.0 / scale;
  CUDA_TRY(c, cudaMemcpyAsync(c->d_scal, s, sizeof s, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MOC_OK;
}

// F = sum_i A_i sum_g nuSigma_f phi on the host (used to normalise a state set by the caller):
// 64 fixed chunks of regions summed in parallel, then in chunk order, so F does not depend on the
// thread count.
double host_fission(const moc_ctx *c, const double *phi, const std::vector<double> &nsf) {
  const Geometry &g = c->geo;
  const int R = g.n_tri, G = c->G, NC = 64;
  double part[NC];
#pragma omp parallel for schedule(static)
  for (int q = 0; q < NC; ++q) {
    const int r0 = (int)((int64_t)R * q / NC), r1 = (int)((int64_t)R * (q + 1) / NC);
    double F = 0.0;
    for (int r = r0; r < r1; ++r) {
      double f = 0.0;
      for (int k = 0; k < G; ++k) f += nsf[(size_t)g.mat[r] * G + k] * (phi ? phi[(size_t)r * G + k] : 1.0);
      F += g.area[r] * f;
    }
    part[q] = F;
  }
  double F = 0.0;
  for (int q = 0; q < NC; ++q) F += part[q];
  return F;
}

// Device-addressable view of a caller's host array (pinned or registered memory; pageable memory
// where this GPU accesses it coherently), or nullptr: the state then goes through the staged copy.
const void *host_view(const moc_ctx *c, const void *p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type == cudaMemoryTypeHost) return a.devicePointer;
  if (a.type == cudaMemoryTypeUnregistered && c->pageable_ok) return p;
  return nullptr;
}

// The caller's state read in place by one kernel; in eigenvalue mode the kernel also sums the
// fission source F of the state and sets the normalisation 1/F itself (no host pass over phi).
// Pinned arrays are read by the kernel over the host link directly: staging them on the device
// through the copy engine first was measured slower for the 0.55 GB state of the 199-assembly core.
template <typename Real> int state_in(moc_ctx *c, const double *dphi, const double *dpsi, double k) {
  const int R = c->geo.n_tri;
  const long long n = std::max<long long>(1, (long long)R * c->Gp + c->T * 2 * c->P * c->G);
  double *hs = nullptr;
  CUDA_TRY(c, cudaHostGetDevicePointer((void **)&hs, c->h_scal, 0));
  c->h_scal[S_FISS] = 0.0;
  state_in_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
      R, c->G, c->Gp, (long long)c->T, c->P, dphi, dpsi, c->d_inv, c->d_fed, (Real *)c->d_phi,
      (Real *)c->d_psi[c->cur], c->d_scal, k, 1.0, c->eigen ? 1 : 0, c->d_mat, (const Real *)c->d_nsf, c->d_area,
      c->d_part, c->d_ticket, hs);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->eigen && !std::isfinite(c->h_scal[S_FISS]))
    return fail(c, MOC_ERR_ARG, "set_state: the fission source of the state is not finite");
  return MOC_OK;
}

// The state written into the caller's host arrays (dphi, dpsi: their device views) by one kernel,
// which also copies the scalars. Pinned arrays (pinned = 1) are written through a device staging
// buffer and one copy each by the copy engine, which moves large states over the host link far
// faster than the kernel's own stores to host memory; other device-addressable arrays are written
// by the kernel directly.
template <typename Real>
int state_out(moc_ctx *c, double *dphi, double *dpsi, double *s, double *hphi, double *hpsi, bool pinned) {
  const int R = c->geo.n_tri;
  const long long nphi = dphi ? (long long)R * c->G : 0, npsi = dpsi ? c->T * 2 * c->P * c->G : 0;
  const long long n = std::max<long long>(1, nphi + npsi);
  double *hs = nullptr;
  CUDA_TRY(c, cudaHostGetDevicePointer((void **)&hs, c->h_scal, 0));
  double *wphi = dphi, *wpsi = dpsi;
  if (pinned) {
    if ((size_t)n > c->d_ostage_n) {
      dfree(c->d_ostage);
      c->d_ostage_n = 0;
      CUDA_TRY(c, cudaMalloc(&c->d_ostage, (size_t)n * sizeof(double)));
      c->d_ostage_n = (size_t)n;
    }
    wphi = dphi ? c->d_ostage : nullptr;
    wpsi = dpsi ? c->d_ostage + nphi : nullptr;
  }
  state_out_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
      R, c->G, c->Gp, (long long)c->T, c->P, (const Real *)c->d_phi, (const Real *)c->d_psi[c->cur], c->d_inv,
      c->d_scal, c->eigen ? 1 : 0, wphi, wpsi, hs);
  CUDA_TRY(c, cudaGetLastError());
  if (pinned && hphi)
    CUDA_TRY(c, cudaMemcpyAsync(hphi, wphi, (size_t)nphi * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (pinned && hpsi)
    CUDA_TRY(c, cudaMemcpyAsync(hpsi, wpsi, (size_t)npsi * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < S_COUNT; ++i) s[i] = c->h_scal[i];
  return MOC_OK;
}

bool is_pinned(const void *p) {
  if (!p) return true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

}  // namespace

namespace {

// DGMOC state: flux moments phi [nz][R][2][G] (NULL: phi_0 = 1, phi_1 = 0), zero radial and axial
// boundary flux, scalars reset with k and the normalisation 1/F
template <typename Real> int dg_set_state(moc_ctx *c, const double *phi, double k, const double *psi) {
  if (psi) return fail(c, MOC_ERR_ARG, "set_state: with DGMOC the boundary flux restarts at zero (psi must be NULL)");
  const int R = c->geo.n_tri, G = c->G, nz = c->dg_nz;
  const long long E = (long long)nz * R;
  double scale = 1.0;
  if (c->eigen) {
    double F = 0.0;
    for (long long e = 0; e < E; ++e) {
      const int m = c->h_mat3[e];
      double f = 0.0;
      for (int g = 0; g < G; ++g) f += c->h_nsf[(size_t)m * G + g] * (phi ? phi[(size_t)e * 2 * G + g] : 1.0);
      F += c->h_dz[e / R] * c->geo.area[e % R] * f;
    }
    if (!std::isfinite(F)) return fail(c, MOC_ERR_ARG, "set_state: the fission source of the state is not finite");
    if (F > 0.0) scale = 1.0 / F;
  }
  double *dphi = nullptr;
  if (phi) {
    CUDA_TRY(c, cudaMalloc(&dphi, (size_t)E * 2 * G * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(dphi, phi, (size_t)E * 2 * G * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) {
      cudaFree(dphi);
      return fail(c, MOC_ERR_CUDA, std::string("set_state: ") + cudaGetErrorString(e));
    }
  }
  const long long n = E * c->Gp * 2;
  dg_phi_in_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(n, G, c->Gp, dphi, (Real *)c->d_phi3);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (dphi) cudaFree(dphi);
  if (e != cudaSuccess) return fail(c, MOC_ERR_CUDA, std::string("set_state: ") + cudaGetErrorString(e));
  const size_t nb = (size_t)c->T * 2 * 2 * nz * c->P * 2 * G * sizeof(Real);
  CUDA_TRY(c, cudaMemsetAsync(c->d_psi3[0], 0, nb, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_psi3[1], 0, nb, c->stream));
  if (c->d_face)
    CUDA_TRY(c, cudaMemsetAsync(c->d_face, 0, (size_t)(c->S + 2 * kSegPad) * 2 * c->P * G * sizeof(Real), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->d_tal3, 0, (size_t)E * c->Gp * 2 * sizeof(Real), c->stream));
  return reset_scalars(c, k, scale);
}

template <typename Real> int dg_get_state(moc_ctx *c, double *phi, double *k, double *psi) {
  if (psi) return fail(c, MOC_ERR_ARG, "get_state: with DGMOC only the flux moments are returned (psi must be NULL)");
  double s[S_COUNT];
  int rc = read_scalars(c, s);
  if (rc) return rc;
  if (k) *k = s[S_K];
  if (!phi) return MOC_OK;
  const long long E = (long long)c->dg_nz * c->geo.n_tri, n = E * 2 * c->G;
  double *dphi = nullptr;
  CUDA_TRY(c, cudaMalloc(&dphi, (size_t)n * sizeof(double)));
  dg_phi_out_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
      n, c->G, c->Gp, (const Real *)c->d_phi3, c->eigen ? s[S_SCALE] : 1.0, dphi);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(phi, dphi, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(dphi);
  if (e != cudaSuccess) return fail(c, MOC_ERR_CUDA, std::string("get_state: ") + cudaGetErrorString(e));
  return MOC_OK;
}

template <typename Real> int dg_alloc(moc_ctx *c) {
  const int R = c->geo.n_tri, G = c->G, Gp = c->Gp, P = c->P, nz = c->dg_nz, nd = c->geo.n_dir;
  const size_t E = (size_t)nz * R;
  std::vector<Real> cz((size_t)nz * P), wdg((size_t)nd * P), sn(P);
  for (int p = 0; p < P; ++p) {
    const double st = c->geo.sin_theta[p];
    sn[p] = (Real)st;
    for (int z = 0; z < nz; ++z) cz[(size_t)z * P + p] = (Real)(std::sqrt(std::max(0.0, 1.0 - st * st)) / c->h_dz[z]);
    for (int j = 0; j < nd; ++j)
      wdg[(size_t)j * P + p] = (Real)(0.5 * kFourPi * c->geo.omega[j] * c->geo.polar_w[p] * c->geo.delta[j]);
  }
  int rc;
  Real *p_cz = nullptr, *p_w = nullptr, *p_s = nullptr;
  if ((rc = upload(c, p_cz, cz.data(), cz.size()))) return rc;
  c->d_cz = p_cz;
  if ((rc = upload(c, p_w, wdg.data(), wdg.size()))) return rc;
  c->d_wdg = p_w;
  if ((rc = upload(c, p_s, sn.data(), sn.size()))) return rc;
  c->d_sin = p_s;
  if ((rc = upload(c, c->d_mat3, c->h_mat3.data(), c->h_mat3.size()))) return rc;
  if ((rc = upload(c, c->d_dz, c->h_dz.data(), c->h_dz.size()))) return rc;
  CUDA_TRY(c, cudaMalloc(&c->d_xs3, E * Gp * sizeof(DgXs<Real>)));
  CUDA_TRY(c, cudaMemset(c->d_xs3, 0, E * Gp * sizeof(DgXs<Real>)));
  CUDA_TRY(c, cudaMalloc(&c->d_phi3, E * Gp * 2 * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_tal3, E * Gp * 2 * sizeof(Real)));
  const size_t nb = (size_t)c->T * 2 * 2 * nz * P * 2 * G;
  CUDA_TRY(c, cudaMalloc(&c->d_psi3[0], std::max<size_t>(nb, 1) * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_psi3[1], std::max<size_t>(nb, 1) * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_fold3, E * sizeof(double)));
  CUDA_TRY(c, cudaMemset(c->d_fold3, 0, E * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_part3, ((E + 255) / 256) * 4 * sizeof(double)));
  // the plane-inner sweep when its per-block shared memory stays moderate, else plane by plane
  size_t sm = 0;
  cudaError_t e = cudaSuccess;
  switch (P) {
    case 1: sm = dg_res_smem<Real, 1>(nz); if (sm <= kDgResSmemMax) e = cudaFuncSetAttribute(dg_sweep_res_kernel<Real, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
    case 2: sm = dg_res_smem<Real, 2>(nz); if (sm <= kDgResSmemMax) e = cudaFuncSetAttribute(dg_sweep_res_kernel<Real, 2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
    case 3: sm = dg_res_smem<Real, 3>(nz); if (sm <= kDgResSmemMax) e = cudaFuncSetAttribute(dg_sweep_res_kernel<Real, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
    default: sm = dg_res_smem<Real, 4>(nz); if (sm <= kDgResSmemMax) e = cudaFuncSetAttribute(dg_sweep_res_kernel<Real, 4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); break;
  }
  if (e != cudaSuccess) return fail(c, MOC_ERR_CUDA, std::string("set_axial: ") + cudaGetErrorString(e));
  c->dg_res_smem = sm <= kDgResSmemMax ? sm : 0;
  // the interface buffer: every plane's traces for the plane-by-plane sweep; for the plane-inner
  // sweep only the top traces a reflective top needs (none at all with a vacuum top)
  if (!c->dg_res_smem || c->dg_bc[1])
    CUDA_TRY(c, cudaMalloc(&c->d_face, (size_t)(c->S + 2 * kSegPad) * 2 * P * G * sizeof(Real)));
  return MOC_OK;
}

}  // namespace

// ====================================================================================== C ABI
extern "C" {

int moc_set_axial(moc_ctx *c, int nz, const double *dz, const int32_t *mat3, int bc_bottom, int bc_top) {
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  free_dg(c);
  if (nz == 0) return moc_set_state(c, nullptr, 1.0, nullptr);
  if (nz < 0 || !dz) return fail(c, MOC_ERR_ARG, "set_axial: nz > 0 plane heights required");
  if (c->cmfd || c->aniso_L) return fail(c, MOC_ERR_STATE, "set_axial: not combined with CMFD or anisotropic scattering");
  if (c->P > 4) return fail(c, MOC_ERR_ARG, "set_axial: up to 4 polar angles");
  const int R = c->geo.n_tri;
  if ((long long)nz * R >= (1LL << 31)) return fail(c, MOC_ERR_ARG, "set_axial: nz * n_regions too large");
  for (int z = 0; z < nz; ++z)
    if (!(dz[z] >= kDgMinPlane) || !std::isfinite(dz[z]))
      return fail(c, MOC_ERR_ARG, "set_axial: plane heights must be finite and at least 1e-9 cm");
  std::vector<int32_t> m3((size_t)nz * R);
  for (int z = 0; z < nz; ++z)
    for (int r = 0; r < R; ++r) {
      const int32_t m = mat3 ? mat3[(size_t)z * R + r] : c->geo.mat[r];
      if (m < 0 || m >= c->M) return fail(c, MOC_ERR_ARG, "set_axial: a material id is out of range");
      m3[(size_t)z * R + r] = m;
    }
  for (double ph : c->geo.omega)
    if (!std::isfinite(ph)) return fail(c, MOC_ERR_STATE, "set_axial: direction weights unknown");
  c->h_mat3 = std::move(m3);
  c->h_dz.assign(dz, dz + nz);
  c->dg_nz = nz;
  c->dg_bc[0] = bc_bottom ? 1 : 0;
  c->dg_bc[1] = bc_top ? 1 : 0;
  rc = c->precision == MOC_FP64 ? dg_alloc<double>(c) : dg_alloc<float>(c);
  if (rc) {
    free_dg(c);
    return rc;
  }
  return moc_set_state(c, nullptr, 1.0, nullptr);
}

}  // extern "C"

namespace {

template <typename Real, int P> int dg_cm_attr(moc_ctx *c, size_t sm) {
  CUDA_TRY(c, cudaFuncSetAttribute(dg_sweep_res_kernel<Real, P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sm));
  return MOC_OK;
}

template <typename Real> int dg_cm_alloc(moc_ctx *c) {
  const int nz = c->dg_nz, G = c->G, Gp = c->Gp, P = c->P, R = c->geo.n_tri;
  const size_t sm = c->dg_res_smem + (size_t)kDgResBlock * 3 * nz * sizeof(Real);
  if (!c->dg_res_smem || sm > kDgResSmemMax)
    return fail(c, MOC_ERR_ARG, "set_dg_cmfd: too many planes for the plane-inner sweep's shared memory");
  int rc = P == 1 ? dg_cm_attr<Real, 1>(c, sm) : P == 2 ? dg_cm_attr<Real, 2>(c, sm)
         : P == 3 ? dg_cm_attr<Real, 3>(c, sm) : dg_cm_attr<Real, 4>(c, sm);
  if (rc) return rc;
  std::vector<Real> mu(P), dzr(nz);
  for (int p = 0; p < P; ++p) mu[p] = (Real)std::sqrt(std::max(0.0, 1.0 - c->geo.sin_theta[p] * c->geo.sin_theta[p]));
  for (int z = 0; z < nz; ++z) dzr[z] = (Real)c->h_dz[z];
  std::vector<double> vol(nz, 0.0);
  for (int z = 0; z < nz; ++z)
    for (int r = 0; r < R; ++r) vol[z] += c->geo.area[r] * (double)(Real)c->h_dz[z];
  Real *pm = nullptr, *pz = nullptr;
  if ((rc = upload(c, pm, mu.data(), mu.size()))) return rc;
  c->d_mu = pm;
  if ((rc = upload(c, pz, dzr.data(), dzr.size()))) return rc;
  c->d_dzr = pz;
  if ((rc = upload(c, c->d_dgvol, vol.data(), vol.size()))) return rc;
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgcur, (size_t)2 * nz * Gp * sizeof(double)));
  CUDA_TRY(c, cudaMemset(c->d_dgcur, 0, (size_t)2 * nz * Gp * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgleak, (size_t)nz * Gp * sizeof(double)));
  CUDA_TRY(c, cudaMemset(c->d_dgleak, 0, (size_t)nz * Gp * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgpsum, (size_t)nz * c->M * G * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgdiag, (size_t)nz * G * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgphic, (size_t)nz * G * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgfis, (size_t)nz * sizeof(double)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgpart, (size_t)((nz * R + 255) / 256) * sizeof(double)));
  CUDA_TRY(c, cudaMalloc(&c->d_dgcphi, (size_t)nz * G * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_dgTV, (size_t)nz * G * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_dgSV, (size_t)nz * G * G * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_dgFV, (size_t)nz * G * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_dgCHI, (size_t)nz * G * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc(&c->d_dgratio, (size_t)nz * G * sizeof(Real)));
  CUDA_TRY(c, cudaMalloc((void **)&c->d_dgticket, sizeof(unsigned)));
  CUDA_TRY(c, cudaMemset(c->d_dgticket, 0, sizeof(unsigned)));
  c->dgcm_smem = sm;
  return MOC_OK;
}

}  // namespace

extern "C" {

int moc_set_dg_cmfd(moc_ctx *c, int n_outer, int n_inner, double omega) {
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  free_dgcm(c);
  if (n_outer == 0) return MOC_OK;
  if (!c->dg_nz) return fail(c, MOC_ERR_STATE, "set_dg_cmfd: call moc_set_axial first");
  if (n_outer < 0 || n_inner < 1) return fail(c, MOC_ERR_ARG, "set_dg_cmfd: bad iteration counts");
  if (!(omega > 0.0 && omega < 2.0)) return fail(c, MOC_ERR_ARG, "set_dg_cmfd: omega must lie in (0, 2)");
  rc = c->precision == MOC_FP64 ? dg_cm_alloc<double>(c) : dg_cm_alloc<float>(c);
  if (rc) {
    free_dgcm(c);
    return rc;
  }
  c->dgcm_outer = n_outer;
  c->dgcm_inner = n_inner;
  c->dgcm_omega = omega;
  return MOC_OK;
}

int moc_create(moc_ctx **out, int device, int precision, void *stream) {
  if (!out) return MOC_ERR_ARG;
  *out = nullptr;
  if (precision != MOC_FP64 && precision != MOC_FP32 && precision != MOC_FP32_PLAIN) return MOC_ERR_ARG;
  moc_ctx *c = new (std::nothrow) moc_ctx;
  if (!c) return MOC_ERR_OOM;
  c->device = device;
  c->precision = precision;
  if (device >= 0) {
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) {
      if (stream) {
        c->stream = (cudaStream_t)stream;
      } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = (e == cudaSuccess);
      }
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_scal, S_COUNT * sizeof(double));
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&c->h_scal, S_COUNT * sizeof(double), cudaHostAllocMapped);
    if (e == cudaSuccess) {
      int pm = 0;
      if (cudaDeviceGetAttribute(&pm, cudaDevAttrPageableMemoryAccess, device) == cudaSuccess) c->pageable_ok = pm != 0;
      e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    }
    if (e != cudaSuccess) {
      moc_destroy(c);
      return MOC_ERR_CUDA;
    }
  }
  *out = c;
  return MOC_OK;
}

void moc_destroy(moc_ctx *c) {
  if (!c) return;
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto &p : c->ev) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    free_tracks(c);
    dfree(c->d_scal);
    dfree(c->d_ostage);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->h_scal) cudaFreeHost(c->h_scal);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  }
  delete c;
}

const char *moc_last_error(const moc_ctx *c) { return c ? c->err.c_str() : "null context"; }

int moc_set_mesh(moc_ctx *c, int n_vert, const double *xy, int n_tri, const int32_t *tri, const int32_t *mat,
                 const double *bbox, const int32_t *bc) {
  if (!c) return MOC_ERR_ARG;
  int rc = set_mesh(c->geo, n_vert, xy, n_tri, tri, mat, bbox, bc, c->err);
  if (rc) return rc;
  if (c->device >= 0) free_tracks(c);
  return MOC_OK;
}

int moc_set_quadrature(moc_ctx *c, int n_azim, double spacing, int n_polar, const double *sin_theta,
                       const double *polar_w) {
  if (!c) return MOC_ERR_ARG;
  int rc = set_quadrature(c->geo, n_azim, spacing, n_polar, sin_theta, polar_w, c->err);
  if (rc) return rc;
  if (c->device >= 0) free_tracks(c);
  return MOC_OK;
}

int moc_set_ray_layout(moc_ctx *c, int layout) {
  if (!c) return MOC_ERR_ARG;
  if (layout != MOC_RAYS_MODULAR && layout != MOC_RAYS_BACK_PROJECTION)
    return fail(c, MOC_ERR_ARG, "set_ray_layout: layout must be MOC_RAYS_MODULAR or MOC_RAYS_BACK_PROJECTION");
  c->geo.layout = layout;
  c->geo.has_tracks = false;
  if (c->device >= 0) free_tracks(c);
  return MOC_OK;
}

int moc_generate_tracks(moc_ctx *c) {
  if (!c) return MOC_ERR_ARG;
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    free_tracks(c);
  }
  int rc = generate_tracks(c->geo, c->err);
  if (rc) return rc;
  if (c->device < 0) return MOC_OK;
  return c->precision == MOC_FP64 ? upload_tracks<double>(c) : upload_tracks<float>(c);
}

int moc_generate_tracks_device(moc_ctx *c, double *walk_ms) {
  if (!c) return MOC_ERR_ARG;
  if (c->device < 0) return fail(c, MOC_ERR_STATE, "generate_tracks_device: the context has no device");
  cudaSetDevice(c->device);
  free_tracks(c);
  DeviceWalkCtx wc{c->device, c->stream, 0.0};
  const Walker w{device_walk, &wc};
  int rc = generate_tracks(c->geo, c->err, &w);
  if (rc) return rc;
  if (walk_ms) *walk_ms = wc.walk_ms;
  return c->precision == MOC_FP64 ? upload_tracks<double>(c) : upload_tracks<float>(c);
}

int moc_set_tracks(moc_ctx *c, int64_t n_tracks, const int64_t *seg_off, const int32_t *seg_region,
                   const double *seg_len, const int32_t *track_azim, const double *azim_weight,
                   const double *azim_spacing, const int32_t *link) {
  if (!c) return MOC_ERR_ARG;
  Geometry &g = c->geo;
  if (!g.has_mesh || !g.has_quad) return fail(c, MOC_ERR_STATE, "set_tracks: set the mesh and the quadrature first");
  if (n_tracks < 1 || !seg_off || !seg_region || !seg_len || !track_azim || !azim_weight || !azim_spacing || !link)
    return fail(c, MOC_ERR_ARG, "set_tracks: bad sizes or NULL arrays");
  const int nd = g.n_dir;
  if (seg_off[0] != 0) return fail(c, MOC_ERR_ARG, "set_tracks: seg_off[0] must be 0");
  for (int64_t t = 0; t < n_tracks; ++t)
    if (!(seg_off[t + 1] > seg_off[t])) return fail(c, MOC_ERR_ARG, "set_tracks: every track needs at least one segment");
  const int64_t S = seg_off[n_tracks];
  if (S >= ((int64_t)1 << 31) * 16) return fail(c, MOC_ERR_ARG, "set_tracks: too many segments");
  for (int64_t s = 0; s < S; ++s) {
    if (seg_region[s] < 0 || seg_region[s] >= g.n_tri) return fail(c, MOC_ERR_ARG, "set_tracks: region id out of range");
    if (!(seg_len[s] > 0.0) || !std::isfinite(seg_len[s])) return fail(c, MOC_ERR_ARG, "set_tracks: lengths must be finite and > 0");
  }
  for (int j = 0; j < nd; ++j)
    if (!(azim_weight[j] > 0.0) || !std::isfinite(azim_weight[j]) || !(azim_spacing[j] > 0.0) || !std::isfinite(azim_spacing[j]))
      return fail(c, MOC_ERR_ARG, "set_tracks: azimuthal weights and spacings must be finite and > 0");
  std::vector<char> fed(2 * n_tracks, 0);
  for (int64_t t = 0; t < n_tracks; ++t) {
    if (track_azim[t] < 0 || track_azim[t] >= nd) return fail(c, MOC_ERR_ARG, "set_tracks: track direction out of range");
    for (int d = 0; d < 2; ++d) {
      const int64_t e = link[2 * t + d];
      if (e < 0) continue;
      if (e >= 2 * n_tracks) return fail(c, MOC_ERR_ARG, "set_tracks: link target out of range");
      if (fed[e]) return fail(c, MOC_ERR_ARG, "set_tracks: an incoming end is linked twice (links must be a bijection)");
      fed[e] = 1;
    }
  }
  if (c->device >= 0) {
    cudaSetDevice(c->device);
    free_tracks(c);
  }
  // the caller's tracks replace any laid down here: directions are known only by their weights
  g.phi.assign(nd, NAN);
  g.omega.assign(azim_weight, azim_weight + nd);
  g.delta.assign(azim_spacing, azim_spacing + nd);
  g.nx.assign(nd, 0);
  g.ny.assign(nd, 0);
  g.seg_off.assign(seg_off, seg_off + n_tracks + 1);
  g.seg_reg.assign(seg_region, seg_region + S);
  g.seg_len.assign(seg_len, seg_len + S);
  g.track_dir.assign(track_azim, track_azim + n_tracks);
  g.track_xy.assign(4 * (size_t)n_tracks, NAN);
  g.link.assign(link, link + 2 * n_tracks);
  g.area.assign(g.n_tri, 0.0);
  for (int64_t t = 0; t < n_tracks; ++t) {
    const double w = 2.0 * g.omega[g.track_dir[t]] * g.delta[g.track_dir[t]];
    for (int64_t s = g.seg_off[t]; s < g.seg_off[t + 1]; ++s) g.area[g.seg_reg[s]] += w * g.seg_len[s];
  }
  g.has_tracks = true;
  if (c->device < 0) return MOC_OK;
  return c->precision == MOC_FP64 ? upload_tracks<double>(c) : upload_tracks<float>(c);
}

int moc_get_track_counts(const moc_ctx *c, int64_t *n_tracks, int64_t *n_segments) {
  if (!c || !c->geo.has_tracks) return c ? MOC_ERR_STATE : MOC_ERR_ARG;
  if (n_tracks) *n_tracks = c->geo.n_tracks();
  if (n_segments) *n_segments = c->geo.n_segments();
  return MOC_OK;
}

int moc_get_tracks(const moc_ctx *c, int64_t *seg_off, int32_t *seg_region, double *seg_len, int32_t *track_dir,
                   double *track_xy, int64_t *link) {
  if (!c || !c->geo.has_tracks) return c ? MOC_ERR_STATE : MOC_ERR_ARG;
  const Geometry &g = c->geo;
  if (seg_off) std::copy(g.seg_off.begin(), g.seg_off.end(), seg_off);
  if (seg_region) std::copy(g.seg_reg.begin(), g.seg_reg.end(), seg_region);
  if (seg_len) std::copy(g.seg_len.begin(), g.seg_len.end(), seg_len);
  if (track_dir) std::copy(g.track_dir.begin(), g.track_dir.end(), track_dir);
  if (track_xy) std::copy(g.track_xy.begin(), g.track_xy.end(), track_xy);
  if (link) std::copy(g.link.begin(), g.link.end(), link);
  return MOC_OK;
}

int moc_get_quadrature(const moc_ctx *c, double *phi, double *delta, double *omega) {
  if (!c || !c->geo.has_tracks) return c ? MOC_ERR_STATE : MOC_ERR_ARG;
  const Geometry &g = c->geo;
  if (phi) std::copy(g.phi.begin(), g.phi.end(), phi);
  if (delta) std::copy(g.delta.begin(), g.delta.end(), delta);
  if (omega) std::copy(g.omega.begin(), g.omega.end(), omega);
  return MOC_OK;
}

int moc_get_region_areas(const moc_ctx *c, double *area) {
  if (!c || !c->geo.has_tracks || !area) return (!c || !area) ? MOC_ERR_ARG : MOC_ERR_STATE;
  std::copy(c->geo.area.begin(), c->geo.area.end(), area);
  return MOC_OK;
}

int moc_set_xs(moc_ctx *c, int n_mat, int G, const double *st, const double *nsf, const double *chi,
               const double *ss) {
  int rc = need_gpu(c);
  if (rc) return rc;
  if (!c->tracks_on_device) return fail(c, MOC_ERR_STATE, "set_xs: generate tracks first");
  if (n_mat < 1 || G < 1 || G > 1024 || !st || !nsf || !chi || !ss) return fail(c, MOC_ERR_ARG, "set_xs: bad sizes");
  for (int m : c->geo.mat)
    if (m >= n_mat) return fail(c, MOC_ERR_ARG, "set_xs: a mesh material id is >= n_mat");
  for (size_t i = 0; i < (size_t)n_mat * G; ++i) {
    if (!(st[i] > 0.0) || !std::isfinite(st[i])) return fail(c, MOC_ERR_ARG, "set_xs: sigma_t must be finite and > 0");
    if (!(nsf[i] >= 0.0) || !std::isfinite(nsf[i]) || !(chi[i] >= 0.0) || !std::isfinite(chi[i]))
      return fail(c, MOC_ERR_ARG, "set_xs: nu_sigma_f and chi must be finite and >= 0");
  }
  for (size_t i = 0; i < (size_t)n_mat * G * G; ++i)
    if (!(ss[i] >= 0.0) || !std::isfinite(ss[i])) return fail(c, MOC_ERR_ARG, "set_xs: sigma_s must be finite and >= 0");
  // no material may scatter out of a group more than it removes from it (absorption >= 0)
  for (int m = 0; m < n_mat; ++m)
    for (int g = 0; g < G; ++g) {
      double out = 0.0;
      for (int h = 0; h < G; ++h) out += ss[((size_t)m * G + g) * G + h];
      if (out > st[(size_t)m * G + g] * (1.0 + 1e-12))
        return fail(c, MOC_ERR_ARG, "set_xs: sigma_t must be >= the total scattering out of each group");
    }
  cudaSetDevice(c->device);
  free_problem(c);
  // the sweep that will run decides the internal track order (re-uploaded when it changes)
  const int order = (G > 8 && c->P == 3 && c->precision != MOC_FP64) ? 1 : 0;
  if (order != c->order_mode) {
    free_tracks(c);
    c->order_mode = order;
    rc = c->precision == MOC_FP64 ? upload_tracks<double>(c) : upload_tracks<float>(c);
    if (rc) return rc;
  }
  c->eigen = true;
  // the device tables hold the values rounded to the sweep's type; normalise with the same
  c->h_nsf.resize((size_t)n_mat * G);
  for (size_t i = 0; i < c->h_nsf.size(); ++i)
    c->h_nsf[i] = c->precision == MOC_FP64 ? nsf[i] : (double)(float)nsf[i];
  c->cur = 0;
  rc = c->precision == MOC_FP64 ? upload_xs<double>(c, n_mat, G, st, nsf, chi, ss)
                                : upload_xs<float>(c, n_mat, G, st, nsf, chi, ss);
  if (rc) return rc;
  return moc_set_state(c, nullptr, 1.0, nullptr);
}

int moc_set_scattering(moc_ctx *c, int L, const double *sigma_sl) {
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  free_aniso(c);
  if (L == 0 || !sigma_sl) return MOC_OK;
  if (L < 0 || L > kMaxAnisoL) return fail(c, MOC_ERR_ARG, "set_scattering: 0 <= L <= 3");
  if (c->cmfd) return fail(c, MOC_ERR_STATE, "set_scattering: not combined with CMFD acceleration");
  if (c->dg_nz) return fail(c, MOC_ERR_STATE, "set_scattering: not combined with DGMOC");
  if (c->P > 3) return fail(c, MOC_ERR_ARG, "set_scattering: up to 3 polar angles");
  for (double ph : c->geo.phi)
    if (!std::isfinite(ph)) return fail(c, MOC_ERR_STATE, "set_scattering: the track directions' angles are unknown (tracks set by the caller)");
  const int M = c->M, G = c->G, P = c->P, nd = c->geo.n_dir, NK = L * (L + 3) / 2;
  if ((size_t)L * M * G * G * rsize(c) > 48 * 1024) return fail(c, MOC_ERR_ARG, "set_scattering: tables too large");
  for (size_t i = 0; i < (size_t)L * M * G * G; ++i)
    if (!std::isfinite(sigma_sl[i])) return fail(c, MOC_ERR_ARG, "set_scattering: sigma_sl must be finite");
  // real harmonics with l + m even, l = 1..L (Schmidt semi-normalised, no Condon-Shortley phase),
  // for every stored direction j in [0, pi) and polar angle p
  auto harm = [](int l, int m, double ph, double st) {
    const double ct2 = 1.0 - st * st;
    switch (l) {
      case 1: return m < 0 ? st * std::sin(ph) : st * std::cos(ph);
      case 2:
        if (m == 0) return 0.5 * (3.0 * ct2 - 1.0);
        return 0.5 * std::sqrt(3.0) * st * st * (m < 0 ? std::sin(2 * ph) : std::cos(2 * ph));
      default:
        if (m == -1 || m == 1) return 0.25 * std::sqrt(6.0) * (5.0 * ct2 - 1.0) * st * (m < 0 ? std::sin(ph) : std::cos(ph));
        return 0.25 * std::sqrt(10.0) * st * st * st * (m < 0 ? std::sin(3 * ph) : std::cos(3 * ph));
    }
  };
  std::vector<int> kl, km;
  for (int l = 1; l <= L; ++l)
    for (int m = -l; m <= l; m += 2) {
      kl.push_back(l);
      km.push_back(m);
    }
  std::vector<double> H((size_t)nd * P * NK);
  for (int j = 0; j < nd; ++j)
    for (int p = 0; p < P; ++p)
      for (int k = 0; k < NK; ++k) H[((size_t)j * P + p) * NK + k] = harm(kl[k], km[k], c->geo.phi[j], c->geo.sin_theta[p]);
  // Gram matrix over the discrete directions (both senses; R_0 = 1): 4 pi sum omega w R_k R_k'
  const int n = NK + 1;
  std::vector<double> Gm((size_t)n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const int la = a ? kl[a - 1] : 0, lb = b ? kl[b - 1] : 0;
      if ((la + lb) & 1) continue;  // the two senses cancel exactly
      double sum = 0.0;
      for (int j = 0; j < nd; ++j)
        for (int p = 0; p < P; ++p) {
          const double ra = a ? H[((size_t)j * P + p) * NK + a - 1] : 1.0;
          const double rb = b ? H[((size_t)j * P + p) * NK + b - 1] : 1.0;
          sum += 2.0 * c->geo.omega[j] * c->geo.polar_w[p] * ra * rb;
        }
      Gm[(size_t)a * n + b] = kFourPi * sum;
    }
  const size_t rs = rsize(c);
  auto put = [&](void *&dst, const std::vector<double> &v) -> int {
    CUDA_TRY(c, cudaMalloc(&dst, std::max<size_t>(v.size(), 1) * rs));
    if (c->precision == MOC_FP64) {
      CUDA_TRY(c, cudaMemcpy(dst, v.data(), v.size() * rs, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> f(v.begin(), v.end());
      CUDA_TRY(c, cudaMemcpy(dst, f.data(), f.size() * rs, cudaMemcpyHostToDevice));
    }
    return MOC_OK;
  };
  std::vector<double> ssl(sigma_sl, sigma_sl + (size_t)L * M * G * G);
  if ((rc = put(c->d_ssl, ssl))) return rc;
  if ((rc = put(c->d_harm, H))) return rc;
  if ((rc = put(c->d_gm, Gm))) return rc;
  const size_t nm = (size_t)c->geo.n_tri * NK * c->Gp * rs;
  for (void **pp : {&c->d_mom, &c->d_srck, &c->d_tmom}) {
    CUDA_TRY(c, cudaMalloc(pp, nm));
    CUDA_TRY(c, cudaMemsetAsync(*pp, 0, nm, c->stream));
  }
  c->aniso_L = L;
  c->aniso_NK = NK;
  drop_graphs(c);
  // moments of the current state's isotropic angular flux
  rc = c->precision == MOC_FP64 ? launch_aniso_init<double>(c, c->stream) : launch_aniso_init<float>(c, c->stream);
  if (rc) return rc;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MOC_OK;
}

int moc_set_cmfd(moc_ctx *c, const int32_t *cell_in, int n_cells, int n_outer, int n_inner, double omega) {
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  free_cmfd(c);
  if (!cell_in) return MOC_OK;
  if (c->aniso_L) return fail(c, MOC_ERR_STATE, "set_cmfd: not combined with anisotropic scattering");
  if (c->dg_nz) return fail(c, MOC_ERR_STATE, "set_cmfd: not combined with DGMOC");
  const Geometry &g = c->geo;
  const int R = g.n_tri, G = c->G;
  if (n_cells < 1 || n_outer < 1 || n_inner < 1) return fail(c, MOC_ERR_ARG, "set_cmfd: bad sizes or iteration counts");
  if (!(omega > 0.0 && omega < 2.0)) return fail(c, MOC_ERR_ARG, "set_cmfd: omega must lie in (0, 2)");
  for (int r = 0; r < R; ++r)
    if (cell_in[r] < 0 || cell_in[r] >= n_cells) return fail(c, MOC_ERR_ARG, "set_cmfd: cell id out of range");
  const int64_t T = g.n_tracks();
  // interfaces: pairs of cells that consecutive segments of some track cross between
  auto find_pairs = [&](const int32_t *cell) {
    std::vector<uint64_t> pr;
    for (int64_t t = 0; t < T; ++t)
      for (int64_t q = g.seg_off[t]; q + 1 < g.seg_off[t + 1]; ++q) {
        const uint32_t a = (uint32_t)cell[g.seg_reg[q]], b = (uint32_t)cell[g.seg_reg[q + 1]];
        if (a != b) pr.push_back(((uint64_t)std::min(a, b) << 32) | std::max(a, b));
      }
    std::sort(pr.begin(), pr.end());
    pr.erase(std::unique(pr.begin(), pr.end()), pr.end());
    return pr;
  };
  std::vector<uint64_t> pairs = find_pairs(cell_in);
  // greedy colouring in ascending cell id (smallest colour none of the lower-id neighbours has),
  // then cells renumbered colour by colour (ascending id within a colour), so the over-relaxed
  // sweeps update one contiguous range of independent cells per colour
  std::vector<int32_t> adj_off(n_cells + 1, 0), adj((size_t)2 * pairs.size());
  for (uint64_t p : pairs) {
    adj_off[(p >> 32) + 1]++;
    adj_off[(p & 0xffffffffu) + 1]++;
  }
  for (int i = 0; i < n_cells; ++i) adj_off[i + 1] += adj_off[i];
  {
    std::vector<int32_t> fill(adj_off.begin(), adj_off.end() - 1);
    for (uint64_t p : pairs) {
      const int a = (int)(p >> 32), b = (int)(p & 0xffffffffu);
      adj[fill[a]++] = b;
      adj[fill[b]++] = a;
    }
  }
  std::vector<int32_t> color(n_cells, 0), used(n_cells + 1, -1);
  int n_colors = 0;
  for (int i = 0; i < n_cells; ++i) {
    for (int q = adj_off[i]; q < adj_off[i + 1]; ++q)
      if (adj[q] < i) used[color[adj[q]]] = i;
    int col = 0;
    while (used[col] == i) ++col;
    color[i] = col;
    n_colors = std::max(n_colors, col + 1);
  }
  std::vector<int32_t> coff(n_colors + 1, 0), newid(n_cells);
  for (int i = 0; i < n_cells; ++i) coff[color[i] + 1]++;
  for (int k = 0; k < n_colors; ++k) coff[k + 1] += coff[k];
  {
    std::vector<int32_t> fill(coff.begin(), coff.end() - 1);
    for (int i = 0; i < n_cells; ++i) newid[i] = fill[color[i]]++;
  }
  std::vector<int32_t> cellv(R);
  for (int r = 0; r < R; ++r) cellv[r] = newid[cell_in[r]];
  const int32_t *cell = cellv.data();
  for (uint64_t &p : pairs) {
    const uint32_t a = (uint32_t)newid[p >> 32], b = (uint32_t)newid[p & 0xffffffffu];
    p = ((uint64_t)std::min(a, b) << 32) | std::max(a, b);
  }
  std::sort(pairs.begin(), pairs.end());
  const int n_if = (int)pairs.size();
  auto iface = [&](uint32_t a, uint32_t b) {
    const uint64_t key = ((uint64_t)std::min(a, b) << 32) | std::max(a, b);
    return (int)(std::lower_bound(pairs.begin(), pairs.end(), key) - pairs.begin());
  };
  // coarse boundaries crossed by each track, in internal track order and along the track:
  // {segment p after which the boundary lies (forward numbering), 2 * interface + (a > b)}
  std::vector<int32_t> xoff(T + 1, 0);
  std::vector<int2> xent;
  for (int64_t i = 0; i < T; ++i) {
    const int64_t t = c->perm[i];
    for (int64_t q = g.seg_off[t]; q + 1 < g.seg_off[t + 1]; ++q) {
      const uint32_t a = (uint32_t)cell[g.seg_reg[q]], b = (uint32_t)cell[g.seg_reg[q + 1]];
      if (a != b) xent.push_back(make_int2((int)(q - g.seg_off[t]), 2 * iface(a, b) + (a > b ? 1 : 0)));
    }
    if (xent.size() > (size_t)INT32_MAX) return fail(c, MOC_ERR_ARG, "set_cmfd: too many coarse-boundary crossings");
    xoff[i + 1] = (int32_t)xent.size();
  }
  // incidences: each interface appears in the lists of both its cells, in interface order
  std::vector<int32_t> cif_off(n_cells + 1, 0), cif(2 * (size_t)n_if), if_cells(2 * (size_t)n_if);
  for (int e = 0; e < n_if; ++e) {
    const int a = (int)(pairs[e] >> 32), b = (int)(pairs[e] & 0xffffffffu);
    if_cells[2 * e] = a;
    if_cells[2 * e + 1] = b;
    cif_off[a + 1]++;
    cif_off[b + 1]++;
  }
  for (int i = 0; i < n_cells; ++i) cif_off[i + 1] += cif_off[i];
  {
    std::vector<int32_t> fill(cif_off.begin(), cif_off.end() - 1);
    for (int e = 0; e < n_if; ++e) {
      cif[fill[if_cells[2 * e]]++] = (e << 1) | 0;
      cif[fill[if_cells[2 * e + 1]]++] = (e << 1) | 1;
    }
  }
  std::vector<int32_t> nbr(2 * (size_t)n_if);
  for (size_t q = 0; q < nbr.size(); ++q) nbr[q] = if_cells[2 * (cif[q] >> 1) + ((cif[q] & 1) ^ 1)];
  if ((rc = upload(c, c->d_xoff, xoff.data(), xoff.size()))) return rc;
  if ((rc = upload(c, c->d_xent, xent.data(), xent.size()))) return rc;
  if ((rc = upload(c, c->d_cell, cellv.data(), cellv.size()))) return rc;
  if ((rc = upload(c, c->d_cif_off, cif_off.data(), cif_off.size()))) return rc;
  if ((rc = upload(c, c->d_cif, cif.data(), cif.size()))) return rc;
  if ((rc = upload(c, c->d_if_cells, if_cells.data(), if_cells.size()))) return rc;
  if ((rc = upload(c, c->d_nbr, nbr.data(), nbr.size()))) return rc;
  if ((rc = upload(c, c->d_coff, coff.data(), coff.size()))) return rc;
  const size_t rs = rsize(c), Gp = c->Gp, N = n_cells;
  auto alloc0 = [&](void *&ptr, size_t bytes) -> int {
    CUDA_TRY(c, cudaMalloc(&ptr, std::max<size_t>(bytes, 8)));
    CUDA_TRY(c, cudaMemsetAsync(ptr, 0, std::max<size_t>(bytes, 8), c->stream));
    return MOC_OK;
  };
  if ((rc = alloc0(c->d_cur, 2 * (size_t)n_if * Gp * sizeof(double)))) return rc;
  if ((rc = alloc0(c->d_leak, N * Gp * sizeof(double)))) return rc;
  if ((rc = alloc0(c->d_cphi, N * G * rs))) return rc;
  if ((rc = alloc0(c->d_TV, N * G * rs))) return rc;
  if ((rc = alloc0(c->d_SV, N * G * G * rs))) return rc;
  if ((rc = alloc0(c->d_FV, N * G * rs))) return rc;
  if ((rc = alloc0(c->d_CHI, N * G * rs))) return rc;
  // one more group's worth of din: the per-group coefficients of the coarse solve when its working
  // set does not fit in shared memory (phin, phio and src hold the iterate, 1/diagonal, source)
  if ((rc = alloc0(c->d_din, 2 * (size_t)n_if * (G + 1) * rs))) return rc;
  if ((rc = alloc0(c->d_diag, N * G * rs))) return rc;
  if ((rc = alloc0(c->d_phic, N * G * rs))) return rc;
  if ((rc = alloc0(c->d_phin, N * rs))) return rc;
  if ((rc = alloc0(c->d_phio, N * rs))) return rc;
  if ((rc = alloc0(c->d_src, N * rs))) return rc;
  {
    void *ps = nullptr, *pv = nullptr;
    if ((rc = alloc0(ps, N * (size_t)c->M * G * sizeof(double)))) return rc;
    c->d_psum = (double *)ps;
    std::vector<double> vol(N, 0.0);
    for (int r = 0; r < R; ++r) vol[cell[r]] += g.area[r];
    if ((rc = alloc0(pv, N * sizeof(double)))) return rc;
    c->d_vol = (double *)pv;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_vol, vol.data(), N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  }
  if ((rc = alloc0(c->d_fis, N * rs))) return rc;
  if ((rc = alloc0(c->d_ratio, N * G * rs))) return rc;
  void *cp = nullptr, *ct = nullptr;
  if ((rc = alloc0(cp, ((size_t)R + 255) / 256 * sizeof(double)))) return rc;
  c->d_cpart = (double *)cp;
  if ((rc = alloc0(ct, sizeof(unsigned)))) return rc;
  c->d_cticket = (unsigned *)ct;
  // the coarse solve's per-group working set in shared memory when it fits (next to the kernel's
  // 8 KB reduction buffer): source, 1/diagonal and iterate per cell, one coefficient per entry,
  // the entry offsets, and the neighbour ids (16-bit when the cell count allows)
  {
    const size_t ne = 2 * (size_t)n_if;
    const bool idx16 = n_cells <= 65535;
    const size_t need = (3 * N + ne) * rs + (N + 1) * sizeof(int32_t) + ne * (idx16 ? 2 : 4);
    int dev_max = 0;
    CUDA_TRY(c, cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    c->cm_smem = 0;
    c->cm_idx16 = idx16;
    if (need + 8192 + 1024 <= (size_t)dev_max) {
      const void *fn;
      if (c->precision == MOC_FP64)
        fn = idx16 ? (const void *)cmfd_solve_kernel<double, true, uint16_t> : (const void *)cmfd_solve_kernel<double, true, int32_t>;
      else
        fn = idx16 ? (const void *)cmfd_solve_kernel<float, true, uint16_t> : (const void *)cmfd_solve_kernel<float, true, int32_t>;
      CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need));
      c->cm_smem = need;
    }
  }
  // coarse problems of 1,024 cells and more: the cluster solve (8 CTAs, each owning a slice of
  // every colour), if such a cluster fits on the device
  c->cm_cluster = 0;
  if (n_cells >= 1024) {
    const int C = 8, ncol = n_colors;
    std::vector<std::vector<int32_t>> own(C);
    std::vector<int32_t> owner(n_cells), local(n_cells), ccoff((size_t)C * (ncol + 1), 0);
    for (int col = 0; col < ncol; ++col) {
      const int lo = coff[col], len = coff[col + 1] - coff[col];
      for (int b = 0; b < C; ++b) {
        const int a0 = lo + (int)((int64_t)len * b / C), a1 = lo + (int)((int64_t)len * (b + 1) / C);
        ccoff[(size_t)b * (ncol + 1) + col] = (int32_t)own[b].size();
        for (int i = a0; i < a1; ++i) {
          owner[i] = b;
          local[i] = (int32_t)own[b].size();
          own[b].push_back(i);
        }
      }
    }
    for (int b = 0; b < C; ++b) ccoff[(size_t)b * (ncol + 1) + ncol] = (int32_t)own[b].size();
    std::vector<int32_t> cbase(C + 1, 0), ebase(C + 1, 0), own_cell, eoff, loc;
    size_t need_max = 0;
    bool fits = true;
    for (int b = 0; b < C; ++b) {
      cbase[b + 1] = cbase[b] + (int32_t)own[b].size();
      int32_t ne = 0;
      eoff.push_back(0);
      for (int i : own[b]) {
        own_cell.push_back(i);
        for (int q = cif_off[i]; q < cif_off[i + 1]; ++q) {
          const int j = nbr[q];
          loc.push_back((owner[j] << 16) | local[j]);
          ++ne;
        }
        eoff.push_back(ne);
      }
      ebase[b + 1] = ebase[b] + ne;
      if (own[b].size() >= 65536) fits = false;
    }
    {
      size_t ncmax = 0;
      for (int b = 0; b < C; ++b) ncmax = std::max(ncmax, own[b].size());
      for (int b = 0; b < C; ++b) {
        const size_t ne = (size_t)(ebase[b + 1] - ebase[b]);
        need_max = std::max(need_max, (4 * ncmax + ne) * rs + (ncmax + 1) * 4 + 8 + ne * sizeof(void *));
      }
    }
    int dev_max = 0;
    CUDA_TRY(c, cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    if (fits && need_max + 1024 <= (size_t)dev_max) {
      const void *fn = c->precision == MOC_FP64 ? (const void *)cmfd_solve_cluster_kernel<double>
                                                : (const void *)cmfd_solve_cluster_kernel<float>;
      CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need_max));
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C);
      cfg.blockDim = dim3(1024);
      cfg.dynamicSmemBytes = need_max;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n_cl = 0;
      if (cudaOccupancyMaxActiveClusters(&n_cl, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        n_cl = 0;
      }
      if (n_cl >= 1) {
        // one allocation: cbase | own_cell | ccoff | ebase | eoff | loc
        std::vector<int32_t> all;
        std::vector<size_t> at_off;
        for (const std::vector<int32_t> *v : {&cbase, &own_cell, &ccoff, &ebase, &eoff, &loc}) {
          at_off.push_back(all.size());
          all.insert(all.end(), v->begin(), v->end());
        }
        if ((rc = upload(c, c->d_cl, all.data(), all.size()))) return rc;
        c->cl = CmfdCluster{c->d_cl + at_off[0], c->d_cl + at_off[1], c->d_cl + at_off[2], c->d_cl + at_off[3],
                            c->d_cl + at_off[4], c->d_cl + at_off[5]};
        c->cm_cluster = C;
        c->cm_cl_smem = need_max;
      }
    }
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->n_cells = n_cells;
  c->n_if = n_if;
  c->cm_outer = n_outer;
  c->cm_inner = n_inner;
  c->cm_omega = omega;
  c->cm_colors = n_colors;
  c->cmfd = true;
  drop_graphs(c);
  return MOC_OK;
}

int moc_set_cmfd_tolerance(moc_ctx *c, double tol) {
  if (!c) return MOC_ERR_ARG;
  if (!(tol >= 0.0) || !std::isfinite(tol)) return fail(c, MOC_ERR_ARG, "set_cmfd_tolerance: tol must be finite and >= 0");
  c->cm_tol = tol;
  return MOC_OK;
}

int moc_get_cmfd_iterations(moc_ctx *c, int64_t *total) {
  int rc = need_gpu(c);
  if (rc) return rc;
  if (!total) return fail(c, MOC_ERR_ARG, "get_cmfd_iterations: null output");
  double s[S_COUNT];
  if ((rc = read_scalars(c, s))) return rc;
  *total = (int64_t)s[S_CMFD_IT];
  return MOC_OK;
}

int moc_set_fixed_source(moc_ctx *c, const double *S) {
  int rc = need_ready(c);
  if (rc) return rc;
  dfree(c->d_ext);
  drop_graphs(c);
  const size_t RG = (size_t)c->geo.n_tri * c->G;
  if (!S) {
    c->eigen = true;
    return moc_set_state(c, nullptr, 1.0, nullptr);
  }
  if (c->cmfd) return fail(c, MOC_ERR_STATE, "set_fixed_source: CMFD acceleration is for eigenvalue mode only");
  for (size_t i = 0; i < RG; ++i)
    if (!(S[i] >= 0.0) || !std::isfinite(S[i])) return fail(c, MOC_ERR_ARG, "set_fixed_source: S must be finite and >= 0");
  if ((rc = upload(c, c->d_ext, S, RG))) return rc;
  c->eigen = false;
  return moc_set_state(c, nullptr, 1.0, nullptr);
}

int moc_set_state(moc_ctx *c, const double *phi, double k, const double *psi) {
  int rc = need_ready(c);
  if (rc) return rc;
  if (!(k > 0.0) || !std::isfinite(k)) return fail(c, MOC_ERR_ARG, "set_state: k must be finite and > 0");
  c->hist_n = 0;
  cudaSetDevice(c->device);
  if (c->dg_nz) return c->precision == MOC_FP64 ? dg_set_state<double>(c, phi, k, psi) : dg_set_state<float>(c, phi, k, psi);
  // arrays the device can address are read in place by one kernel, which also normalises; others
  // are staged and normalised from a host pass
  const void *vphi = host_view(c, phi), *vpsi = host_view(c, psi);
  if ((!phi || vphi) && (!psi || vpsi)) {
    rc = c->precision == MOC_FP64 ? state_in<double>(c, (const double *)vphi, (const double *)vpsi, k)
                                  : state_in<float>(c, (const double *)vphi, (const double *)vpsi, k);
  } else {
    double scale = 1.0;
    if (c->eigen) {
      double F = host_fission(c, phi, c->h_nsf);
      if (!std::isfinite(F)) return fail(c, MOC_ERR_ARG, "set_state: the fission source of the state is not finite");
      if (F > 0.0) scale = 1.0 / F;   // no fission at all: power iteration will report MOC_ERR_NONFINITE
    }
    rc = c->precision == MOC_FP64 ? upload_state<double>(c, phi, psi) : upload_state<float>(c, phi, psi);
    if (!rc) rc = reset_scalars(c, k, scale);
  }
  if (rc || !c->aniso_L) return rc;
  // anisotropic moments restart from an isotropic angular flux
  rc = c->precision == MOC_FP64 ? launch_aniso_init<double>(c, c->stream) : launch_aniso_init<float>(c, c->stream);
  if (rc) return rc;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MOC_OK;
}

int moc_get_state(moc_ctx *c, double *phi, double *k, double *psi) {
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  if (c->dg_nz) return c->precision == MOC_FP64 ? dg_get_state<double>(c, phi, k, psi) : dg_get_state<float>(c, phi, k, psi);
  double s[S_COUNT];
  void *vphi = (void *)host_view(c, phi), *vpsi = (void *)host_view(c, psi);
  if ((phi || psi) && (!phi || vphi) && (!psi || vpsi)) {
    // written in place by one kernel, which also copies the scalars (pinned arrays through the
    // copy engine)
    const bool pinned = is_pinned(phi) && is_pinned(psi);
    rc = c->precision == MOC_FP64 ? state_out<double>(c, (double *)vphi, (double *)vpsi, s, phi, psi, pinned)
                                  : state_out<float>(c, (double *)vphi, (double *)vpsi, s, phi, psi, pinned);
    if (rc) return rc;
    if (k) *k = s[S_K];
    return MOC_OK;
  }
  if ((rc = read_scalars(c, s))) return rc;
  const double scale = c->eigen ? s[S_SCALE] : 1.0;
  if (k) *k = s[S_K];
  if (phi || psi) {
    rc = c->precision == MOC_FP64 ? download_state<double>(c, scale, phi, psi)
                                  : download_state<float>(c, scale, phi, psi);
    if (rc) return rc;
  }
  return MOC_OK;
}

int moc_update_source(moc_ctx *c) {
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  return enqueue_source(c, c->stream);
}

int moc_sweep(moc_ctx *c) {
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  return enqueue_sweep(c, c->stream, c->timing);
}

int moc_outer(moc_ctx *c, int n, double *k_out, double *resid_out) {
  int rc = need_ready(c);
  if (rc) return rc;
  if (n < 0) return fail(c, MOC_ERR_ARG, "outer: n < 0");
  cudaSetDevice(c->device);
  if ((rc = run_outers(c, n))) return rc;
  if (k_out || resid_out) {
    double s[S_COUNT];
    if ((rc = read_scalars(c, s))) return rc;
    if (n > 0) record_history(c, s);
    if (k_out) *k_out = s[S_K];
    if (resid_out) *resid_out = s[S_RESID];
    if (s[S_STATUS] == 2.0) return fail(c, MOC_ERR_CUDA, "outer: a bulk copy of the finalize did not complete");
    if (s[S_STATUS] != 0.0) return fail(c, MOC_ERR_NONFINITE, "outer: k or the residual is not finite");
  }
  return MOC_OK;
}

}  // extern "C"

namespace {

template <typename Real> int sweep_dev(moc_ctx *c, cudaStream_t st, const void *in, void *out) {
  const int R = c->geo.n_tri;
  const long long n_in = (long long)R * c->Gp, n_out = (long long)R * c->G;
  if (in) {
    // the caller's flux is taken as normalised: the boundary flux settles the pending factor
    if (c->eigen) {
      const long long np = c->T * 2 * c->P * c->G;
      settle_scale_kernel<Real><<<(unsigned)((np + 255) / 256), 256, 0, st>>>(np, (Real *)c->d_psi[c->cur], c->d_scal);
      reset_scale_kernel<<<1, 32, 0, st>>>(c->d_scal);
    }
    flux_in_kernel<Real><<<(unsigned)((n_in + 255) / 256), 256, 0, st>>>(R, c->G, c->Gp, (const Real *)in, (Real *)c->d_phi);
    CUDA_TRY(c, cudaGetLastError());
  }
  int rc = enqueue_outer(c, st, false);
  if (rc) return rc;
  if (out) {
    flux_out_kernel<Real><<<(unsigned)((n_out + 255) / 256), 256, 0, st>>>(R, c->G, c->Gp, (const Real *)c->d_phi,
                                                                          c->d_scal, c->eigen ? 1 : 0, (Real *)out);
    CUDA_TRY(c, cudaGetLastError());
  }
  return MOC_OK;
}

}  // namespace

extern "C" {

int moc_sweep_dev(moc_ctx *c, void *stream, const void *phi_in_dev, void *phi_out_dev) {
  int rc = need_ready(c);
  if (rc) return rc;
  if (c->dg_nz) return fail(c, MOC_ERR_STATE, "sweep_dev: planar method only (DGMOC is on)");
  cudaSetDevice(c->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  if (st != c->stream) {
    // order the caller's stream after the context's pending work and the context's after this
    cudaEvent_t ev;
    CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CUDA_TRY(c, cudaEventRecord(ev, c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(st, ev, 0));
    rc = c->precision == MOC_FP64 ? sweep_dev<double>(c, st, phi_in_dev, phi_out_dev)
                                  : sweep_dev<float>(c, st, phi_in_dev, phi_out_dev);
    if (!rc) {
      CUDA_TRY(c, cudaEventRecord(ev, st));
      CUDA_TRY(c, cudaStreamWaitEvent(c->stream, ev, 0));
    }
    cudaEventDestroy(ev);
    return rc;
  }
  return c->precision == MOC_FP64 ? sweep_dev<double>(c, st, phi_in_dev, phi_out_dev)
                                  : sweep_dev<float>(c, st, phi_in_dev, phi_out_dev);
}

int moc_get_history(const moc_ctx *c, double *entries, int max_entries, int *n_out) {
  if (!c || max_entries < 0 || (max_entries > 0 && !entries)) return MOC_ERR_ARG;
  const int64_t avail = std::min<int64_t>(c->hist_n, kHistory);
  const int n = (int)std::min<int64_t>(avail, max_entries);
  for (int i = 0; i < n; ++i) {
    const int64_t idx = c->hist_n - n + i;  // oldest of the returned first
    const double *h = &c->hist[4 * (size_t)(idx % kHistory)];
    for (int q = 0; q < 4; ++q) entries[4 * i + q] = h[q];
  }
  if (n_out) *n_out = n;
  return MOC_OK;
}

int moc_get_stats(moc_ctx *c, double *sweep_ms, double *updates_per_s) {
  double ms = 0.0;
  int64_t n = 0;
  int rc = moc_get_timing(c, &ms, &n);
  if (rc) return rc;
  const double avg = n ? ms / (double)n : 0.0;
  if (sweep_ms) *sweep_ms = avg;
  if (updates_per_s) {
    const double ups = 2.0 * (double)c->geo.n_segments() * c->geo.n_polar * c->G;
    *updates_per_s = avg > 0.0 ? ups / (avg * 1e-3) : 0.0;
  }
  return MOC_OK;
}

int moc_power_iterate(moc_ctx *c, double tol_k, double tol_flux, int max_outer, int check_every, double *k_out,
                      int *n_outer_out, double *resid_out) {
  if (!c) return MOC_ERR_ARG;
  // arguments first: a NaN or negative tolerance could never be met
  if (max_outer < 1 || check_every < 1 || !(tol_flux >= 0.0) || !(tol_k >= 0.0))
    return fail(c, MOC_ERR_ARG, "power_iterate: bad arguments");
  int rc = need_ready(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  int n = 0;
  double s[S_COUNT] = {0};
  bool conv = false;
  while (n < max_outer) {
    int m = std::min(check_every, max_outer - n);
    // each reduce kernel keeps the k before its outer, so after m outers S_KPREV is the k
    // before the last one
    if ((rc = run_outers(c, m))) return rc;
    n += m;
    if ((rc = read_scalars(c, s))) return rc;
    record_history(c, s);
    if (s[S_STATUS] == 2.0)
      return fail(c, MOC_ERR_CUDA, "power_iterate: a bulk copy of the finalize did not complete");
    if (s[S_STATUS] != 0.0) return fail(c, MOC_ERR_NONFINITE, "power_iterate: k or the residual is not finite");
    bool ok_k = !c->eigen || std::fabs(s[S_K] - s[S_KPREV]) <= tol_k;
    if (ok_k && s[S_RESID] <= tol_flux) {
      conv = true;
      break;
    }
  }
  if (k_out) *k_out = s[S_K];
  if (n_outer_out) *n_outer_out = n;
  if (resid_out) *resid_out = s[S_RESID];
  return conv ? MOC_OK : fail(c, MOC_ERR_NOT_CONVERGED, "power_iterate: max_outer reached");
}

int moc_enable_timing(moc_ctx *c, int enable) {
  int rc = need_gpu(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  for (auto &p : c->ev) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  c->ev.clear();
  c->timed_ms = 0.0;
  c->timed_n = 0;
  c->timing = enable != 0;
  return MOC_OK;
}

int moc_get_timing(moc_ctx *c, double *ms, int64_t *n) {
  int rc = need_gpu(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (auto &p : c->ev) {
    float t = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&t, p.first, p.second));
    c->timed_ms += t;
    c->timed_n += 1;
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  c->ev.clear();
  if (ms) *ms = c->timed_ms;
  if (n) *n = c->timed_n;
  return MOC_OK;
}

int moc_get_work(const moc_ctx *c, int64_t *n_segments, int64_t *updates, int *kernels) {
  if (!c || !c->geo.has_tracks) return c ? MOC_ERR_STATE : MOC_ERR_ARG;
  if (n_segments) *n_segments = c->geo.n_segments();
  // DGMOC: every segment in every plane, both marches
  const int64_t planes = c->dg_nz ? 2 * (int64_t)c->dg_nz : 1;
  if (updates) *updates = 2 * c->geo.n_segments() * (int64_t)c->geo.n_polar * (int64_t)std::max(c->G, 0) * planes;
  if (kernels)
    *kernels = c->dg_nz ? 4 + (c->dgcm_outer && c->eigen ? 5 : 0)
                        : ((c->Gp == 8 || lane_rows(c)) ? 3 : 4) + (c->cmfd ? 5 : 0) + (c->aniso_L ? 2 : 0);
  return MOC_OK;
}

}  // extern "C"

namespace {
template <typename Real> int ws_features_t(moc_ctx *c, const float *geo, int n_geo, const float *glob_dev, int n_glob,
                                          float *feat) {
  const int R = c->geo.n_tri;
  ws_features_kernel<Real><<<(R + 255) / 256, 256, 0, c->stream>>>(R, c->G, n_geo, n_glob, c->d_mat,
                                                                   (const Real *)c->d_sig_t, (const Real *)c->d_nsf,
                                                                   (const Real *)c->d_sig_s, geo, glob_dev, feat);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

}  // namespace

extern "C" {

int moc_ws_features(moc_ctx *c, const float *geo, int n_geo, const float *glob, int n_glob, float *feat) {
  int rc = need_ready(c);
  if (rc) return rc;
  if (c->dg_nz) return fail(c, MOC_ERR_STATE, "ws_features: planar method only (DGMOC is on)");
  if (n_geo < 0 || n_glob < 0 || (n_geo > 0 && !geo) || (n_glob > 0 && !glob) || !feat)
    return fail(c, MOC_ERR_ARG, "ws_features: bad arguments");
  cudaSetDevice(c->device);
  float *dglob = nullptr;
  CUDA_TRY(c, cudaMalloc(&dglob, std::max(n_glob, 1) * sizeof(float)));
  if (n_glob) CUDA_TRY(c, cudaMemcpyAsync(dglob, glob, n_glob * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  rc = c->precision == MOC_FP64 ? ws_features_t<double>(c, geo, n_geo, dglob, n_glob, feat)
                                : ws_features_t<float>(c, geo, n_geo, dglob, n_glob, feat);
  cudaStreamSynchronize(c->stream);
  cudaFree(dglob);
  return rc;
}

}  // extern "C"

namespace {
template <typename Real> int ws_apply_t(moc_ctx *c, const float *pred) {
  const int R = c->geo.n_tri;
  const int nb = (R + 255) / 256;
  ws_apply_kernel<Real><<<nb, 256, 0, c->stream>>>(R, c->G, c->Gp, c->d_mat, (const Real *)c->d_nsf, c->d_area,
                                                   pred, (Real *)c->d_phi, c->d_part);
  CUDA_TRY(c, cudaGetLastError());
  ws_reduce_kernel<<<1, 256, 0, c->stream>>>(nb, c->d_part, c->d_scal);
  CUDA_TRY(c, cudaGetLastError());
  const long long n = (long long)c->T * 2 * c->G;
  ws_psi_kernel<Real><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
      n, c->P, c->G, c->Gp, c->d_trk, (const SegRec<Real> *)c->d_seg, c->d_fed, (const Real *)c->d_phi,
      (Real *)c->d_psi[c->cur]);
  CUDA_TRY(c, cudaGetLastError());
  return MOC_OK;
}

}  // namespace

extern "C" {

int moc_ws_apply(moc_ctx *c, const float *pred, double *k_out) {
  int rc = need_ready(c);
  if (rc) return rc;
  if (c->dg_nz) return fail(c, MOC_ERR_STATE, "ws_apply: planar method only (DGMOC is on)");
  if (!pred) return fail(c, MOC_ERR_ARG, "ws_apply: NULL prediction");
  if (!c->eigen) return fail(c, MOC_ERR_STATE, "ws_apply: eigenvalue mode only");
  cudaSetDevice(c->device);
  rc = c->precision == MOC_FP64 ? ws_apply_t<double>(c, pred) : ws_apply_t<float>(c, pred);
  if (rc) return rc;
  if (k_out) {
    double s[S_COUNT];
    if ((rc = read_scalars(c, s))) return rc;
    *k_out = s[S_K];
    if (s[S_STATUS] != 0.0) return fail(c, MOC_ERR_NONFINITE, "ws_apply: predicted k or flux not finite/positive");
  }
  return MOC_OK;
}

int moc_eval_one_minus_exp_f32(int device, const float *tau, float *out, int64_t n) {
  if (device < 0 || n < 0 || (n > 0 && (!tau || !out))) return MOC_ERR_ARG;
  if (n == 0) return MOC_OK;
  if (cudaSetDevice(device) != cudaSuccess) return MOC_ERR_CUDA;
  float *d = nullptr;
  if (cudaMalloc(&d, 2 * (size_t)n * sizeof(float)) != cudaSuccess) return MOC_ERR_OOM;
  cudaError_t e = cudaMemcpy(d, tau, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    eval_exp_kernel<<<(unsigned)((n + 255) / 256), 256>>>(d, d + n, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? MOC_OK : MOC_ERR_CUDA;
}

int moc_eval_one_minus_exp_f32x2(int device, const float *tau, float *out, int64_t n) {
  if (device < 0 || n < 0 || (n > 0 && (!tau || !out))) return MOC_ERR_ARG;
  if (n == 0) return MOC_OK;
  if (cudaSetDevice(device) != cudaSuccess) return MOC_ERR_CUDA;
  float *d = nullptr;
  if (cudaMalloc(&d, 2 * (size_t)n * sizeof(float)) != cudaSuccess) return MOC_ERR_OOM;
  cudaError_t e = cudaMemcpy(d, tau, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const long long pairs = (n + 1) / 2;
    eval_exp2_kernel<<<(unsigned)((pairs + 255) / 256), 256>>>(d, d + n, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? MOC_OK : MOC_ERR_CUDA;
}

int moc_synchronize(moc_ctx *c) {
  int rc = need_gpu(c);
  if (rc) return rc;
  cudaSetDevice(c->device);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return MOC_OK;
}

}  // extern "C"
