// Anisotropic (P_L) scattering: the Legendre expansion of the scattering kernel (Sec. 2) carried
// as angular moments. By the addition theorem, P_l(Om . Om') = sum_m R_lm(Om) R_lm(Om') with real
// harmonics R_lm; in a plane problem (psi even in the polar direction) only the l + m even
// harmonics survive, NK = L(L+3)/2 of them beyond the scalar flux. Per region and group:
//   flux moments      phi_k = sum over directions 4 pi omega w R_k(Om) psi_bar(Om)
//   source moments    src_k = (2 l_k + 1) sum_g' Sigma_s,l g'->g phi_k,g' / (4 pi Sigma_t)
//   direction source  q(Om)/Sigma_t = src_0 + sum_k src_k R_k(Om)
// The sweep tallies W R_k(Om) (psi_in - psi_out) per moment; the moments after a sweep are
// phi_k = sum_k' Gm[k][k'] src_k' + tally_k / (Sigma_t A), with Gm[k][k'] = 4 pi sum over
// directions of omega w R_k R_k' (the discrete Gram matrix; R_0 = 1).
#pragma once
#include "moc_kernels.cuh"

namespace moc {

constexpr int kMaxAnisoL = 3;

// Legendre order of harmonic k (k = 0 .. NK-1 for l = 1..L, l + 1 harmonics each)
__host__ __device__ __forceinline__ int harmonic_l(int k) { return k < 2 ? 1 : (k < 5 ? 2 : 3); }

// Moment arrays are [R][NK][Gp] for NK > 2: for one moment, the groups of a region are
// contiguous, so the group lanes of one track end read one row and their tally atomics hit one L2
// sector. For P1 (NK = 2) they are [R][Gp][2]: a lane's two moments are one 8-byte pair, read with
// one load and, in FP32, added with one float2 atomic (the warp's pairs still fill whole sectors);
// wider vector atomics over more moments were measured slower.
__host__ __device__ __forceinline__ size_t mom_at(int r, int k, int g, int NK, int Gp) {
  return NK == 2 ? ((size_t)r * Gp + g) * 2 + k : ((size_t)r * NK + k) * Gp + g;
}

template <typename Real, int NK> __device__ __forceinline__ void mom_load(const Real *a, int r, int g, int Gp, Real *v) {
  if (NK == 2 && sizeof(Real) == 4) {
    const float2 x = *reinterpret_cast<const float2 *>(a + mom_at(r, 0, g, NK, Gp));
    v[0] = x.x;
    v[NK - 1] = x.y;
  } else {
#pragma unroll
    for (int k = 0; k < NK; ++k) v[k] = a[mom_at(r, k, g, NK, Gp)];
  }
}

template <typename Real, int NK> __device__ __forceinline__ void mom_add(Real *a, int r, int g, int Gp, const Real *v) {
  if (NK == 2 && sizeof(Real) == 4) {
    atomicAdd(reinterpret_cast<float2 *>(a + mom_at(r, 0, g, NK, Gp)), make_float2(v[0], v[NK - 1]));
  } else {
#pragma unroll
    for (int k = 0; k < NK; ++k) atomicAdd(a + mom_at(r, k, g, NK, Gp), v[k]);
  }
}
// source moments, one thread per region: the pending normalisation is applied to the moments
// first (as source_kernel does to phi), then src_k = (2l+1) sum_g' Sigma_s,l phi_k / (4 pi Sigma_t)
template <typename Real>
__global__ void aniso_source_kernel(int R, int G, int Gp, int M, int NK, const int32_t *__restrict__ mat,
                                    const Real *__restrict__ ssl, const typename Pair<Real>::T *__restrict__ xsq,
                                    Real *__restrict__ mom, Real *__restrict__ srck, const double *__restrict__ scal,
                                    int eigen) {
  extern __shared__ unsigned char smem_raw[];
  const int L = NK == 2 ? 1 : (NK == 5 ? 2 : 3);
  Real *s_ssl = reinterpret_cast<Real *>(smem_raw);  // [L][M][G][G]
  for (int i = threadIdx.x; i < L * M * G * G; i += blockDim.x) s_ssl[i] = ssl[i];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int m = mat[r];
  const Real scale = eigen ? (Real)scal[S_SCALE] : (Real)1;
  const Real inv4pi = (Real)(1.0 / kFourPi);
  for (int k = 0; k < NK; ++k) {
    const int l = harmonic_l(k);
    for (int g = 0; g < G; ++g) mom[mom_at(r, k, g, NK, Gp)] *= scale;
    const Real *ss = s_ssl + ((size_t)(l - 1) * M + m) * G * G;
    for (int g = 0; g < G; ++g) {
      Real a = 0;
      for (int gp = 0; gp < G; ++gp) a += ss[gp * G + g] * mom[mom_at(r, k, gp, NK, Gp)];
      srck[mom_at(r, k, g, NK, Gp)] = (Real)(2 * l + 1) * a * inv4pi / xsq[(size_t)r * Gp + g].x;
    }
  }
}

// Sweep with a direction-dependent flat source (one thread per track, sense and group, as
// sweep_kernel): per segment the NK source moments of the region, per polar angle the source of
// this direction, and NK moment tallies besides the scalar-flux tally.
template <typename Real, int P, int TM, int NK>
__global__ void __launch_bounds__(128) sweep_aniso_kernel(
    const TrackRec *__restrict__ trk, const SegRec<Real> *__restrict__ seg, const int32_t *__restrict__ link,
    const Real *__restrict__ wgt, const Real *__restrict__ inv_sin, const Real *__restrict__ harm,
    const typename Pair<Real>::T *__restrict__ xsq, const Real *__restrict__ srck, Real *__restrict__ tsum,
    Real *__restrict__ tcomp, Real *__restrict__ tmom, const Real *__restrict__ psi_in, Real *__restrict__ psi_out,
    const double *__restrict__ scal, long long n_threads, int G, int Gp) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_threads) return;
  const long long td = idx / G;
  const int g = (int)(idx - td * G);
  const TrackRec tr = trk[td >> 1];
  const int d = (int)(td & 1);
  const Real scale = (Real)scal[S_SCALE];
  Real psi[P], w[P], is[P], hr[P][NK];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    psi[p] = psi_in[(td * P + p) * G + g] * scale;
    w[p] = wgt[tr.dir * P + p];
    is[p] = inv_sin[p];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      // the reverse sense turns Om_xy around: R_lm -> (-1)^l R_lm for the harmonics kept
      const Real h = harm[((size_t)tr.dir * P + p) * NK + k];
      hr[p][k] = (d && (harmonic_l(k) & 1)) ? -h : h;
    }
  }
  // P1: segments two ahead, region rows and moments one ahead (the segment array's padding
  // records make the look-ahead safe without a bounds test). More moments: the rows are read at
  // use, since the look-ahead registers cost more occupancy than they save.
  constexpr bool PF = NK <= 2;
  const int step = d ? -1 : 1;
  const SegRec<Real> *sp = seg + (d ? tr.off + tr.n - 1 : tr.off);
  Tally<TM, Real> tally;
  SegRec<Real> s0 = sp[0], s1 = s0;
  typename Pair<Real>::T xq0 = xsq[(size_t)s0.r * Gp + g];
  Real sk0[NK];
  if (PF) {
    s1 = sp[step];
    mom_load<Real, NK>(srck, s0.r, g, Gp, sk0);
  }
  tally.init((unsigned)(s0.r * Gp + g));
  for (int n = 0; n < tr.n; ++n) {
    typename Pair<Real>::T xq;
    Real sk[NK];
    SegRec<Real> s2;
    typename Pair<Real>::T xq1;
    Real sk1[NK];
    if (PF) {
      s2 = sp[2 * step];
      xq1 = xsq[(size_t)s1.r * Gp + g];
      mom_load<Real, NK>(srck, s1.r, g, Gp, sk1);
      xq = xq0;
#pragma unroll
      for (int k = 0; k < NK; ++k) sk[k] = sk0[k];
    } else {
      s0 = *sp;
      xq = xsq[(size_t)s0.r * Gp + g];
      mom_load<Real, NK>(srck, s0.r, g, Gp, sk);
    }
    const Real tau0 = xq.x * s0.l;
    Real acc = 0, ak[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) ak[k] = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      Real qr = xq.y;
#pragma unroll
      for (int k = 0; k < NK; ++k) qr = fma(sk[k], hr[p][k], qr);
      const Real F = one_minus_exp(tau0 * is[p]);
      const Real dl = (psi[p] - qr) * F;
      psi[p] -= dl;
      acc = fma(w[p], dl, acc);
      const Real wd = w[p] * dl;
#pragma unroll
      for (int k = 0; k < NK; ++k) ak[k] = fma(hr[p][k], wd, ak[k]);
    }
    tally.add(tsum, tcomp, (unsigned)(s0.r * Gp + g), acc);
    mom_add<Real, NK>(tmom, s0.r, g, Gp, ak);
    if (PF) {
      s0 = s1;
      s1 = s2;
      xq0 = xq1;
#pragma unroll
      for (int k = 0; k < NK; ++k) sk0[k] = sk1[k];
    }
    sp += step;
  }
  tally.flush(tcomp);
  const int e = link[td];
  if (e >= 0) {
#pragma unroll
    for (int p = 0; p < P; ++p) psi_out[((long long)e * P + p) * G + g] = psi[p];
  }
}

// After the sweep, before finalize: the flux moments from the moment tallies (which are cleared),
// and the directional part of the scalar flux's flat-source term folded into q/Sigma_t, so that
// finalize's 4 pi q/Sigma_t becomes sum_k' Gm[0][k'] src_k'. One thread per region and group.
template <typename Real>
__global__ void aniso_moments_kernel(int R, int G, int Gp, int NK, const Real *__restrict__ gm,
                                     const Real *__restrict__ inv_ta, typename Pair<Real>::T *__restrict__ xsq,
                                     const Real *__restrict__ srck, Real *__restrict__ tmom, Real *__restrict__ mom) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)R * G) return;
  const int r = (int)(x / G), g = (int)(x - (long long)r * G);
  const size_t a = (size_t)r * Gp + g;
  const int n = NK + 1;
  typename Pair<Real>::T v = xsq[a];
  Real s[1 + 9];
  s[0] = v.y;
  for (int k = 0; k < NK; ++k) s[1 + k] = srck[mom_at(r, k, g, NK, Gp)];
  const Real ita = inv_ta[a];
  for (int k = 1; k < n; ++k) {
    Real ph = 0;
    for (int k2 = 0; k2 < n; ++k2) ph = fma(gm[k * n + k2], s[k2], ph);
    const size_t b = mom_at(r, k - 1, g, NK, Gp);
    ph = fma(tmom[b], ita, ph);
    tmom[b] = (Real)0;
    mom[b] = ph;
  }
  Real c0 = (gm[0] - (Real)kFourPi) * s[0];
  for (int k2 = 1; k2 < n; ++k2) c0 = fma(gm[k2], s[k2], c0);
  v.y += c0 * (Real)(1.0 / kFourPi);
  xsq[a] = v;
}

// Isotropic start of the moments for a state set by the caller: psi_bar = phi / (4 pi) in every
// direction, i.e. phi_k = Gm[k][0] phi / (4 pi).
template <typename Real>
__global__ void aniso_init_kernel(int R, int G, int Gp, int NK, const Real *__restrict__ gm,
                                  const Real *__restrict__ phi, Real *__restrict__ mom) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)R * NK * Gp) return;
  const int r = (int)(x / ((long long)NK * Gp));
  const int rest = (int)(x - (long long)r * NK * Gp), k = rest / Gp, g = rest - k * Gp;
  mom[mom_at(r, k, g, NK, Gp)] = (g < G) ? gm[(k + 1) * (NK + 1)] * phi[(size_t)r * Gp + g] * (Real)(1.0 / kFourPi) : (Real)0;
}

}  // namespace moc
