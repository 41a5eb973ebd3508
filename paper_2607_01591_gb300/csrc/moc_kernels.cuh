// Device kernels of the GB300 MOC library (sm_103a).
//
// Per outer iteration the library launches four kernels on one stream:
//   source_kernel   Eq. (MGNTE_element) source, isotropic: q = [S phi + chi/k nuSigma_f phi]/(4 pi),
//                   stored as q / Sigma_t next to Sigma_t (one 8/16-byte pair per region and group)
//   sweep_kernel    Eq. (MOC_sol) along every track, both senses, all polar angles and groups,
//                   tallying W (psi_in - psi_out) per segment into its region (Sec. 2.1, 3.1)
//   finalize_kernel scalar flux phi = 4 pi q/Sigma_t + tally/(Sigma_t A) and FP64 block partials
//                   of the fission source and of the residual
//   reduce_kernel   one block: FP64 fission source, k update, normalisation, residual
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "exp_f32_coef.h"

namespace moc {

constexpr double kFourPi = 12.566370614359172953850;

// scalar slots in device memory (double)
enum Scal { S_K = 0, S_SCALE = 1, S_RESID = 2, S_FISS = 3, S_KPREV = 4, S_STATUS = 5, S_NOUTER = 6, S_COUNT = 8 };

struct TrackRec {
  long long off;  // first segment
  int n;          // number of segments
  int dir;        // direction index (weights row)
};

template <typename Real> struct SegRec;
template <> struct SegRec<float> {
  int r;
  float l;
};
template <> struct SegRec<double> {
  int r;
  int pad;
  double l;
};

template <typename Real> struct Pair;
template <> struct Pair<float> { using T = float2; };
template <> struct Pair<double> { using T = double2; };

// 1 - exp(-tau), tau >= 0, in FP32: tau = n ln2 + r with n = nearest integer (|r| <= ln2/2),
// 1 - exp(-r) = r + r^2 H(r) with H a degree-4 polynomial (coefficients from gen_exp_coef.py),
// and 1 - exp(-tau) = (1 - 2^-n) + 2^-n (1 - exp(-r)) -- exact reformulation, no cancellation
// for small tau (n = 0 gives r + r^2 H(r) directly). tau is clamped at 80 (exp(-80) < 2^-115).
__device__ __forceinline__ float one_minus_exp(float tau) {
  tau = fminf(tau, 80.0f);
  const float t = fmaf(tau, 1.44269504088896341f, 12582912.0f);  // 1.5*2^23: rounds to integer
  const float n = t - 12582912.0f;
  float r = fmaf(n, -0.693145751953125f, tau);         // ln2 split: high part exact in n * hi
  r = fmaf(n, -1.42860682030941723212e-6f, r);
  const float h = fmaf(fmaf(fmaf(fmaf(MOC_EXP_H4, r, MOC_EXP_H3), r, MOC_EXP_H2), r, MOC_EXP_H1), r, MOC_EXP_H0);
  const float p = fmaf(r * r, h, r);                   // 1 - exp(-r)
  const float sc = __int_as_float(0x3F800000 - (__float_as_int(t) << 23));  // 2^-n
  return fmaf(sc, p, 1.0f - sc);
}

__device__ __forceinline__ double one_minus_exp(double tau) { return -expm1(-tau); }

__global__ void eval_exp_kernel(const float *__restrict__ tau, float *__restrict__ out, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = one_minus_exp(tau[i]);
}

// ----------------------------------------------------------------------------- source update
// One thread per region: normalise phi (eigen mode: multiply by the pending 1/F), record the
// normalised fission rate, and write q/Sigma_t for every group.
template <typename Real>
__global__ void source_kernel(int R, int G, int Gp, int M, const int32_t *__restrict__ mat,
                              const Real *__restrict__ sig_t, const Real *__restrict__ nsf,
                              const Real *__restrict__ chi, const Real *__restrict__ sig_s,
                              const double *__restrict__ ext, Real *__restrict__ phi,
                              typename Pair<Real>::T *__restrict__ xsq, double *__restrict__ fold,
                              const double *__restrict__ scal, int eigen) {
  extern __shared__ unsigned char smem_raw[];
  Real *s_ss = reinterpret_cast<Real *>(smem_raw);  // [M][G][G]
  for (int i = threadIdx.x; i < M * G * G; i += blockDim.x) s_ss[i] = sig_s[i];
  __syncthreads();
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int m = mat[r];
  const Real scale = eigen ? (Real)scal[S_SCALE] : (Real)1;
  const Real inv_k = eigen ? (Real)(1.0 / scal[S_K]) : (Real)0;
  Real *ph = phi + (size_t)r * Gp;
  Real fis = 0;
  double fis_d = 0.0;
  for (int g = 0; g < G; ++g) {
    Real v = ph[g] * scale;
    ph[g] = v;
    fis += nsf[m * G + g] * v;
    fis_d += (double)nsf[m * G + g] * (double)v;
  }
  if (eigen) fold[r] = fis_d;
  const Real *ss = s_ss + (size_t)m * G * G;
  const Real inv4pi = (Real)(1.0 / kFourPi);
  for (int g = 0; g < G; ++g) {
    Real sc = 0;
    for (int gp = 0; gp < G; ++gp) sc += ss[gp * G + g] * ph[gp];
    Real src = sc + chi[m * G + g] * inv_k * fis;
    if (ext) src += (Real)ext[(size_t)r * G + g];
    typename Pair<Real>::T v = xsq[(size_t)r * Gp + g];
    v.y = src * inv4pi / v.x;
    xsq[(size_t)r * Gp + g] = v;
  }
}

// ----------------------------------------------------------------------------- sweep
// Tally modes: 0 plain atomic add, 1 compensated (TwoSum error of each FP32 atomic add is
// accumulated in a second array).
template <int TM, typename Real> struct Tally;
template <typename Real> struct Tally<0, Real> {
  __device__ __forceinline__ void add(Real *sum, Real *, size_t a, Real x) { atomicAdd(sum + a, x); }
  __device__ __forceinline__ void flush(Real *) {}
};
template <> struct Tally<1, float> {
  float old = 0.f, x = 0.f;
  size_t addr = 0;
  bool pending = false;
  // The returned old value of this add is used one segment later, so the atomic's latency is
  // hidden behind the next segment's arithmetic.
  __device__ __forceinline__ void add(float *sum, float *comp, size_t a, float v) {
    float o = atomicAdd(sum + a, v);
    flush(comp);
    old = o;
    x = v;
    addr = a;
    pending = true;
  }
  __device__ __forceinline__ void flush(float *comp) {
    if (pending) {
      // TwoSum (Knuth): s = old + x exactly as the atomic unit rounded it; err = (old + x) - s
      float s = old + x;
      float bb = s - old;
      float err = (old - (s - bb)) + (x - bb);
      atomicAdd(comp + addr, err);
      pending = false;
    }
  }
};

// One thread per (track, sense, group); polar angles held in registers; g fastest so the G
// threads of one track end read one contiguous row of region data and hit one tally row.
template <typename Real, int P, int TM>
__global__ void __launch_bounds__(256) sweep_kernel(
    const TrackRec *__restrict__ trk, const SegRec<Real> *__restrict__ seg, const int32_t *__restrict__ link,
    const Real *__restrict__ wgt, const Real *__restrict__ inv_sin,
    const typename Pair<Real>::T *__restrict__ xsq, Real *__restrict__ tsum, Real *__restrict__ tcomp,
    const Real *__restrict__ psi_in, Real *__restrict__ psi_out, const double *__restrict__ scal,
    long long n_threads, int G, int Gp) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_threads) return;
  const long long td = idx / G;
  const int g = (int)(idx - td * G);
  const TrackRec tr = trk[td >> 1];
  const int d = (int)(td & 1);
  const Real scale = (Real)scal[S_SCALE];
  Real psi[P], w[P], is[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    psi[p] = psi_in[(td * P + p) * G + g] * scale;
    w[p] = wgt[tr.dir * P + p];
    is[p] = inv_sin[p];
  }
  const long long step = d ? -1 : 1;
  long long s = d ? tr.off + tr.n - 1 : tr.off;
  Tally<TM, Real> tally;
  const int N = tr.n;
  SegRec<Real> sg0 = seg[s];
  SegRec<Real> sg1 = (N > 1) ? seg[s + step] : sg0;
  typename Pair<Real>::T xq0 = xsq[(size_t)sg0.r * Gp + g];
  for (int n = 0; n < N; ++n, s += step) {
    SegRec<Real> sg2 = (n + 2 < N) ? seg[s + 2 * step] : sg1;
    typename Pair<Real>::T xq1 = (n + 1 < N) ? xsq[(size_t)sg1.r * Gp + g] : xq0;
    const Real tau0 = xq0.x * sg0.l;
    Real acc = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const Real F = one_minus_exp(tau0 * is[p]);
      const Real dl = (psi[p] - xq0.y) * F;
      psi[p] -= dl;
      acc = fma(w[p], dl, acc);
    }
    tally.add(tsum, tcomp, (size_t)sg0.r * Gp + g, acc);
    sg0 = sg1;
    sg1 = sg2;
    xq0 = xq1;
  }
  tally.flush(tcomp);
  const int e = link[td];
  if (e >= 0) {
#pragma unroll
    for (int p = 0; p < P; ++p) psi_out[((long long)e * P + p) * G + g] = psi[p];
  }
}

// ----------------------------------------------------------------------------- finalize
// One thread per region. Writes phi' (unnormalised), zeroes the tallies, and per block:
// [0] sum_i A_i f'_i, [1] min and [2] max of fold_i / f'_i over f'_i > 0 (eigen mode),
// [3] max relative flux change (fixed-source mode).
template <typename Real, int TM>
__global__ void __launch_bounds__(256) finalize_kernel(
    int R, int G, int Gp, const int32_t *__restrict__ mat, const Real *__restrict__ nsf,
    const double *__restrict__ area, const typename Pair<Real>::T *__restrict__ xsq, Real *__restrict__ tsum,
    Real *__restrict__ tcomp, Real *__restrict__ phi, const double *__restrict__ fold,
    double *__restrict__ part, int eigen) {
  __shared__ double s_sum[256], s_min[256], s_max[256], s_res[256];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double fsum = 0.0, rmin = INFINITY, rmax = -INFINITY, res = 0.0;
  if (r < R) {
    const int m = mat[r];
    const double A = area[r];
    double f = 0.0;
    for (int g = 0; g < G; ++g) {
      const size_t a = (size_t)r * Gp + g;
      const typename Pair<Real>::T v = xsq[a];
      double t = (double)tsum[a];
      tsum[a] = (Real)0;
      if (TM == 1) {
        t += (double)tcomp[a];
        tcomp[a] = (Real)0;
      }
      double ph = kFourPi * (double)v.y;
      if (A > 0.0) ph += t / ((double)v.x * A);
      if (!eigen) {
        const double old = (double)phi[a];
        if (ph > 0.0) res = fmax(res, fabs(ph - old) / ph);
      }
      phi[a] = (Real)ph;
      f += (double)nsf[m * G + g] * (double)(Real)ph;
    }
    fsum = A * f;
    if (eigen && f > 0.0) {
      const double rho = fold[r] / f;
      rmin = rho;
      rmax = rho;
    }
  }
  s_sum[threadIdx.x] = fsum;
  s_min[threadIdx.x] = rmin;
  s_max[threadIdx.x] = rmax;
  s_res[threadIdx.x] = res;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + k];
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + k]);
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + k]);
      s_res[threadIdx.x] = fmax(s_res[threadIdx.x], s_res[threadIdx.x + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[4 * blockIdx.x + 0] = s_sum[0];
    part[4 * blockIdx.x + 1] = s_min[0];
    part[4 * blockIdx.x + 2] = s_max[0];
    part[4 * blockIdx.x + 3] = s_res[0];
  }
}

// ----------------------------------------------------------------------------- reduce
// One block of 256 threads, fixed reduction order (deterministic). k' = k F' (the flux the
// source was built from is normalised to F = 1); scale = 1/F'; residual
// max_i |f'_i/F' - fold_i| / (f'_i/F') = max(|1 - F' rho_min|, |1 - F' rho_max|).
__global__ void __launch_bounds__(256) reduce_kernel(int nb, const double *__restrict__ part,
                                                     double *__restrict__ scal, int eigen) {
  __shared__ double s_sum[256], s_min[256], s_max[256], s_res[256];
  double a = 0.0, mn = INFINITY, mx = -INFINITY, rs = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    a += part[4 * b];
    mn = fmin(mn, part[4 * b + 1]);
    mx = fmax(mx, part[4 * b + 2]);
    rs = fmax(rs, part[4 * b + 3]);
  }
  s_sum[threadIdx.x] = a;
  s_min[threadIdx.x] = mn;
  s_max[threadIdx.x] = mx;
  s_res[threadIdx.x] = rs;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      s_sum[threadIdx.x] += s_sum[threadIdx.x + k];
      s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + k]);
      s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + k]);
      s_res[threadIdx.x] = fmax(s_res[threadIdx.x], s_res[threadIdx.x + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (eigen) {
      const double F = s_sum[0];
      const double k_old = scal[S_K];
      const double k_new = k_old * F;
      double res = 0.0;
      if (s_min[0] <= s_max[0]) res = fmax(fabs(1.0 - F * s_min[0]), fabs(1.0 - F * s_max[0]));
      scal[S_KPREV] = k_old;
      scal[S_K] = k_new;
      scal[S_SCALE] = 1.0 / F;
      scal[S_FISS] = F;
      scal[S_RESID] = res;
      if (!isfinite(k_new) || !isfinite(res) || !(F > 0.0)) scal[S_STATUS] = 1.0;
    } else {
      scal[S_KPREV] = scal[S_K];
      scal[S_SCALE] = 1.0;
      scal[S_RESID] = s_res[0];
      if (!isfinite(s_res[0])) scal[S_STATUS] = 1.0;
    }
    scal[S_NOUTER] += 1.0;
  }
}

}  // namespace moc
