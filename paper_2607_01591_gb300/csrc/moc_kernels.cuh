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
constexpr int kSegPad = 4;  // padding records at each end of the segment array

// scalar slots in device memory (double)
enum Scal { S_K = 0, S_SCALE = 1, S_RESID = 2, S_FISS = 3, S_KPREV = 4, S_STATUS = 5, S_NOUTER = 6, S_CMFD_IT = 7,
            S_COUNT = 8 };

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
  // one FMA forms tau - n ln2 with a single rounding; the FP32 ln2 constant is off by 1.9e-9,
  // i.e. n * 1.9e-9 in r, far below an ulp of the result for every n where 1 - e^-tau != 1
  const float r = fmaf(n, -0.693147182464599609375f, tau);
  const float h = fmaf(fmaf(fmaf(fmaf(MOC_EXP_H4, r, MOC_EXP_H3), r, MOC_EXP_H2), r, MOC_EXP_H1), r, MOC_EXP_H0);
  const float p = fmaf(r * r, h, r);                   // 1 - exp(-r)
  // 2^-n from the bits of t (0x4B400000 + n): 0x3F800000 - n * 2^23, where n * 2^23 modulo 2^32
  // is the bits of t shifted left by 23 (the shift drops 0x4B400000); a funnel shift and an
  // integer subtract, both on the ALU pipe, which leaves the FMA pipe to the arithmetic
  const float sc = __uint_as_float(0x3F800000u - __funnelshift_l(0u, __float_as_uint(t), 23));
  return fmaf(sc, p, 1.0f - sc);
}

__device__ __forceinline__ double one_minus_exp(double tau) { return -expm1(-tau); }

// Packed FP32 pairs: the f32x2 multiply, add and fused multiply-add of sm_100 and later round each
// component exactly as the scalar instruction does, so a pair of updates computed this way gives
// the scalar results bit for bit in half the issue slots. a - b is formed as fma(b, -1, a), which
// rounds a - b once, like the scalar subtraction.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }

// one_minus_exp on a pair, step for step the scalar evaluation above. 2^-n comes either from one
// integer multiply-add per lane (ALU_SCALE = false): (0x4B400000 + n) * (2^32 - 2^23) + 0x3F800000
// = 0x3F800000 - n * 2^23 modulo 2^32; or from the scalar form's funnel shift and subtract on the
// ALU pipe (true). The bits are the same; which balances the pipes better depends on the kernel
// around it (measured: the many-group sweep prefers the multiply-add, the polar-pair sweep the
// shift).
template <bool ALU_SCALE> __device__ __forceinline__ float2 one_minus_exp(float2 tau) {
  tau.x = fminf(tau.x, 80.0f);
  tau.y = fminf(tau.y, 80.0f);
  const float2 t = fma2(tau, f2(1.44269504088896341f), f2(12582912.0f));
  const float2 n = add2(t, f2(-12582912.0f));
  const float2 r = fma2(n, f2(-0.693147182464599609375f), tau);
  const float2 h =
      fma2(fma2(fma2(fma2(f2(MOC_EXP_H4), r, f2(MOC_EXP_H3)), r, f2(MOC_EXP_H2)), r, f2(MOC_EXP_H1)), r, f2(MOC_EXP_H0));
  const float2 p = fma2(mul2(r, r), h, r);
  float2 sc;
  if constexpr (ALU_SCALE) {
    sc = make_float2(__uint_as_float(0x3F800000u - __funnelshift_l(0u, __float_as_uint(t.x), 23)),
                     __uint_as_float(0x3F800000u - __funnelshift_l(0u, __float_as_uint(t.y), 23)));
  } else {
    sc = make_float2(__uint_as_float((unsigned)__float_as_int(t.x) * 0xFF800000u + 0x3F800000u),
                     __uint_as_float((unsigned)__float_as_int(t.y) * 0xFF800000u + 0x3F800000u));
  }
  return fma2(sc, p, sub2(f2(1.0f), sc));
}

__global__ void eval_exp_kernel(const float *__restrict__ tau, float *__restrict__ out, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = one_minus_exp(tau[i]);
}

__global__ void eval_exp2_kernel(const float *__restrict__ tau, float *__restrict__ out, long long n) {
  const long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= n) return;
  const float2 a = make_float2(tau[i], i + 1 < n ? tau[i + 1] : 0.0f);
  const float2 v = one_minus_exp<false>(a), u = one_minus_exp<true>(a);
  // the two ways of forming 2^-n must agree bit for bit; a difference is reported as NaN
  out[i] = __float_as_uint(v.x) == __float_as_uint(u.x) ? v.x : __uint_as_float(0x7FC00000u);
  if (i + 1 < n) out[i + 1] = __float_as_uint(v.y) == __float_as_uint(u.y) ? v.y : __uint_as_float(0x7FC00000u);
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
  for (int g = 0; g < G; ++g) {
    Real v = ph[g] * scale;
    ph[g] = v;
    fis += nsf[m * G + g] * v;
  }
  // normalised fission rate of the region, in the sweep's type (the FP64 pipe is kept for the
  // global sums)
  if (eigen) fold[r] = (double)fis;
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

// Many groups (G > 8): eight consecutive threads per region, lane l owning the groups l, l + 8, ...
// (GPL = ceil(Gp / 8) of them; 0: computed at run time), 32 regions per block of 256. The block's
// normalised flux rows are staged in shared memory (one barrier), the fission rate is an 8-lane
// shuffle sum, and each group visits only the nonzero band srange[m][g] = [first, last] source
// group of column g of the material's scattering matrix (a downscatter-only matrix has half its
// entries zero).
template <typename Real, int GPL>
__global__ void __launch_bounds__(256) source_lanes_kernel(
    int R, int G, int Gp, const int32_t *__restrict__ mat, const Real *__restrict__ sig_s,
    const Real *__restrict__ sig_sT, int Gp4, const Real *__restrict__ nsf, const Real *__restrict__ chi,
    const int2 *__restrict__ srange, const double *__restrict__ ext, const Real *__restrict__ sig_t,
    Real *__restrict__ phi, typename Pair<Real>::T *__restrict__ xsq, double *__restrict__ fold,
    const double *__restrict__ scal, int eigen) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int gpl = GPL > 0 ? GPL : (Gp + 7) / 8;
  const int rl = threadIdx.x >> 3, l = threadIdx.x & 7;
  const int r = blockIdx.x * 32 + rl;
  const bool live = r < R;
  Real *row = reinterpret_cast<Real *>(smem_raw) + (size_t)rl * 8 * gpl;
  __shared__ Real s_inv_k;  // 1/k: one FP64 division per block (GB300's FP64 pipe is slow)
  if (threadIdx.x == 0) s_inv_k = eigen ? (Real)(1.0 / scal[S_K]) : (Real)0;
  const Real scale = eigen ? (Real)scal[S_SCALE] : (Real)1;
  const Real inv4pi = (Real)(1.0 / kFourPi);
  const int m = live ? mat[r] : 0;
  Real f = 0;
  if (GPL > 0) {
    // all of the region's flux loads in flight together, then the scaled values stored
    Real v[GPL > 0 ? GPL : 1], nf[GPL > 0 ? GPL : 1];
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const int g = l + 8 * j;
      v[j] = nf[j] = 0;
      if (live && g < G) {
        v[j] = phi[(size_t)r * Gp + g];
        nf[j] = nsf[m * G + g];
      }
    }
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
      const int g = l + 8 * j;
      const Real w = v[j] * scale;
      if (live && g < G) {
        phi[(size_t)r * Gp + g] = w;
        f += nf[j] * w;
      }
      row[g] = (live && g < G) ? w : (Real)0;
    }
  } else {
    for (int j = 0; j < gpl; ++j) {
      const int g = l + 8 * j;
      Real v = 0;
      if (live && g < G) {
        v = phi[(size_t)r * Gp + g] * scale;
        phi[(size_t)r * Gp + g] = v;
        f += nsf[m * G + g] * v;
      }
      row[g] = v;
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (eigen && live && l == 0) fold[r] = (double)f;
  __syncthreads();
  if (!live) return;
  const Real inv_k = s_inv_k;
  for (int j = 0; j < gpl; ++j) {
    const int g = l + 8 * j;
    if (g >= G) break;
    const int2 band = srange[m * G + g];
    Real sc = 0;
    if constexpr (sizeof(Real) == 4) {
      if (sig_sT) {
        // FP32: column g of the scattering matrix as a contiguous row (sig_sT [M][G][Gp4], zero
        // outside the matrix), four source groups per 16-byte load from both operands, summed in
        // group order; the zeros outside the band add nothing
        const float4 *ssr = reinterpret_cast<const float4 *>(sig_sT + ((size_t)m * G + g) * Gp4);
        const float4 *rr = reinterpret_cast<const float4 *>(row);
        for (int b4 = band.x >> 2; b4 <= (band.y >> 2); ++b4) {
          const float4 a4 = ssr[b4], x4 = rr[b4];
          sc = fmaf(a4.x, x4.x, sc);
          sc = fmaf(a4.y, x4.y, sc);
          sc = fmaf(a4.z, x4.z, sc);
          sc = fmaf(a4.w, x4.w, sc);
        }
      }
    }
    if (sizeof(Real) != 4 || !sig_sT) {
      const Real *ss = sig_s + (size_t)m * G * G + g;
      for (int gp = band.x; gp <= band.y; ++gp) sc += ss[gp * G] * row[gp];
    }
    Real src = sc + chi[m * G + g] * inv_k * f;
    if (ext) src += (Real)ext[(size_t)r * G + g];
    // only the q/Sigma_t half of the region's pair is written; Sigma_t (the pair's other half,
    // the same value) comes from the material table, so the pair is not read
    const size_t a = (size_t)r * Gp + g;
    reinterpret_cast<Real *>(xsq)[2 * a + 1] = src * inv4pi / sig_t[m * G + g];
  }
}

// ----------------------------------------------------------------------------- state transfer
// A caller's state read or written in place when its host arrays are addressable from the device
// (pinned or registered memory, or pageable memory on a system whose GPU reads it coherently):
// one kernel converts, pads and reorders instead of a host loop, a staging copy and a second
// pass. Thread x < R*Gp: region flux; x >= R*Gp: one boundary-flux value of an internal track end.

// phi [R][G] FP64 (NULL: 1) -> d_phi [R][Gp]; psi [T][2][P][G] FP64 in external track order
// (NULL: 0) -> d_psi in internal order, ends that no link feeds set to zero; scalars reset with
// k and the normalisation `scale`.
template <typename Real>
__global__ void __launch_bounds__(256) state_in_kernel(
    int R, int G, int Gp, long long T, int P, const double *__restrict__ phi, const double *__restrict__ psi,
    const long long *__restrict__ inv, const uint8_t *__restrict__ fed, Real *__restrict__ d_phi,
    Real *__restrict__ d_psi, double *__restrict__ scal, double k, double scale, int dev_norm,
    const int32_t *__restrict__ mat, const Real *__restrict__ nsf, const double *__restrict__ area,
    double *__restrict__ part, unsigned *__restrict__ ticket, double *__restrict__ scal_host) {
  __shared__ double red[256];
  __shared__ bool last;
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nphi = (long long)R * Gp, half = (long long)P * G;
  if (x == 0) {
    for (int i = 0; i < S_COUNT; ++i)
      if (!dev_norm || (i != S_SCALE && i != S_FISS)) scal[i] = 0.0;
    scal[S_K] = k;
    scal[S_KPREV] = k;
    scal[S_RESID] = INFINITY;
    if (!dev_norm) {
      scal[S_SCALE] = scale;
      scal[S_FISS] = 1.0 / scale;
    }
  }
  double fa = 0.0;  // this element's share of F = sum_i A_i sum_g nuSigma_f phi
  if (x < nphi) {
    const long long r = x / Gp;
    const int g = (int)(x - r * Gp);
    const double v = (g < G) ? (phi ? phi[r * G + g] : 1.0) : 0.0;
    d_phi[x] = (Real)v;
    if (dev_norm && g < G) fa = area[r] * (double)nsf[mat[r] * G + g] * v;
  } else {
    const long long y = x - nphi;  // external end (t, d) = y / half, value q: the host array is read
    if (y < T * 2 * half) {        // in order, the device array written at the internal position
      const long long ext = y / half, q = y - ext * half;
      const long long e = 2 * inv[ext >> 1] + (ext & 1);
      d_psi[e * half + q] = (psi && fed[e]) ? (Real)psi[y] : (Real)0;
    }
  }
  // the normalisation from the state itself: fixed-order block partials over the blocks that hold
  // flux entries, the last of them to finish sums the partials and sets 1/F (no host pass)
  const unsigned nbp = (unsigned)((nphi + blockDim.x - 1) / blockDim.x);
  if (!dev_norm || blockIdx.x >= nbp) return;
  red[threadIdx.x] = fa;
  __syncthreads();
  for (int k2 = blockDim.x / 2; k2 > 0; k2 >>= 1) {
    if (threadIdx.x < k2) red[threadIdx.x] += red[threadIdx.x + k2];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == nbp - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double a = 0.0;
    for (unsigned b = threadIdx.x; b < nbp; b += blockDim.x) a += part[b];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int k2 = blockDim.x / 2; k2 > 0; k2 >>= 1) {
      if (threadIdx.x < k2) red[threadIdx.x] += red[threadIdx.x + k2];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double F = red[0];
      // no fission at all: scale 1 (power iteration then reports a non-finite k)
      const double sc = (F > 0.0 && isfinite(F)) ? 1.0 / F : 1.0;
      scal[S_SCALE] = sc;
      scal[S_FISS] = F;
      scal_host[S_FISS] = F;
      *ticket = 0u;
    }
  }
}

// d_phi * scal[S_SCALE] -> phi [R][G] FP64; d_psi (internal order) * scale -> psi [T][2][P][G]
// (external order); the scalars copied to `scal_out`.
template <typename Real>
__global__ void state_out_kernel(int R, int G, int Gp, long long T, int P, const Real *__restrict__ d_phi,
                                 const Real *__restrict__ d_psi, const long long *__restrict__ inv,
                                 const double *__restrict__ scal, int eigen, double *__restrict__ phi,
                                 double *__restrict__ psi, double *__restrict__ scal_out) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nphi = phi ? (long long)R * G : 0, half = (long long)P * G;
  const double scale = eigen ? scal[S_SCALE] : 1.0;
  if (x == 0)
    for (int i = 0; i < S_COUNT; ++i) scal_out[i] = scal[i];
  if (x < nphi) {
    const long long r = x / G;
    const int g = (int)(x - r * G);
    phi[x] = (double)d_phi[r * Gp + g] * scale;
    return;
  }
  if (!psi) return;
  const long long y = x - nphi;  // external end (t, d), value q
  if (y >= T * 2 * half) return;
  const long long ext = y / half, q = y - ext * half;
  const long long e = 2 * inv[ext >> 1] + (ext & 1);
  psi[y] = (double)d_psi[e * half + q] * scale;
}

// caller-owned device flux [R][G] (the context's type) <-> the context's padded [R][Gp]
template <typename Real>
__global__ void flux_in_kernel(int R, int G, int Gp, const Real *__restrict__ src, Real *__restrict__ phi) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)R * Gp) return;
  const long long r = x / Gp;
  const int g = (int)(x - r * Gp);
  phi[x] = (g < G) ? src[r * G + g] : (Real)0;
}

// a caller's flux replaces the context's: the boundary flux takes the pending normalisation now
// and the pending factor becomes 1 (thread 0 of the last launch resets it)
template <typename Real>
__global__ void settle_scale_kernel(long long n, Real *__restrict__ psi, const double *__restrict__ scal) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) psi[x] *= (Real)scal[S_SCALE];
}

__global__ void reset_scale_kernel(double *__restrict__ scal) {
  if (threadIdx.x == 0 && blockIdx.x == 0) scal[S_SCALE] = 1.0;
}

// writes the flux after an outer, with the pending normalisation applied (eigen mode)
template <typename Real>
__global__ void flux_out_kernel(int R, int G, int Gp, const Real *__restrict__ phi, const double *__restrict__ scal,
                                int eigen, Real *__restrict__ dst) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (long long)R * G) return;
  const long long r = x / G;
  const int g = (int)(x - r * G);
  dst[x] = phi[r * Gp + g] * (eigen ? (Real)scal[S_SCALE] : (Real)1);
}

// ----------------------------------------------------------------------------- sweep
// Tally modes: 0 plain atomic add, 1 compensated (Kahan: the rounding error of each FP32 atomic
// add is accumulated in a second array).
template <int TM, typename Real> struct Tally;
template <typename Real> struct Tally<0, Real> {
  __device__ __forceinline__ void init(unsigned) {}
  __device__ __forceinline__ void add(Real *sum, Real *, unsigned a, Real x) { atomicAdd(sum + a, x); }
  __device__ __forceinline__ void flush(Real *) {}
};
template <> struct Tally<1, float> {
  // The old value returned by a segment's atomic is turned into its rounding error two segments
  // later, so the atomic's round trip overlaps two segments of arithmetic. Both pending slots
  // start as zero errors aimed at a valid element, which keeps the loop free of branches.
  // Element indices are 32-bit (R * Gp < 2^32) to keep the pending state small.
  float oldA = 0.f, xA = 0.f, oldB = 0.f, xB = 0.f;
  unsigned aA = 0, aB = 0;
  __device__ __forceinline__ static float err(float o, float x) {
    // Kahan's compensation step (Dekker's Fast2Sum): with s = fl(o + x) as the atomic unit rounded
    // it, x - (s - o) is the exact error (o + x) - s whenever |o| >= |x|, i.e. once the tally holds
    // more than one contribution's size (the first add to a zero tally is exact as well); three
    // operations against TwoSum's six, measured 2% faster in both sweeps
    return x - ((o + x) - o);
  }
  __device__ __forceinline__ void init(unsigned a) { aA = aB = a; }
  __device__ __forceinline__ void add(float *sum, float *comp, unsigned a, float v) {
    const float o = atomicAdd(sum + a, v);
    atomicAdd(comp + aB, err(oldB, xB));
    oldB = oldA;
    xB = xA;
    aB = aA;
    oldA = o;
    xA = v;
    aA = a;
  }
  __device__ __forceinline__ void flush(float *comp) {
    atomicAdd(comp + aB, err(oldB, xB));
    atomicAdd(comp + aA, err(oldA, xA));
  }
};

// Coarse-mesh current tallies of the CMFD acceleration (used when the sweep's CM flag is set).
template <typename Real> struct CmfdDev {
  // coarse-cell boundaries crossed by each track (internal track order), sorted along the track:
  // entries xoff[t] .. xoff[t+1]-1, each {p, code}: the boundary between the track's segments p and
  // p+1 (forward numbering), code = 2 * interface + (1 when forward travel leaves the interface's
  // higher cell)
  const int32_t *xoff;  // [T+1]
  const int2 *xent;     // [crossings]
  const int32_t *cell;  // [R] coarse cell of each region
  // FP64 in every precision: a coarse boundary sums thousands of crossings, and FP32 rounding of
  // those sums (different in every sweep, atomics reorder them) would make the coarse operator
  // inconsistent with the fine solution and keep the iteration from settling
  double *cur;          // [2 n_if][Gp] partial currents per interface and direction
  double *leak;         // [N][Gp] net current out of the domain boundary: out at every track end
                        // (vacuum or reflective) minus in at every track start. Reflective walls
                        // cancel only at convergence; leaving them out lets the accelerated
                        // iteration settle on a point that is not the transport solution
};

// One thread per (track, sense, group); polar angles held in registers; g fastest so the G
// threads of one track end read one contiguous row of region data and hit one tally row.
// CM: also tally the partial current W psi at every coarse-cell boundary the track crosses and
// the current through the domain boundary at both ends (CMFD). The crossing list is read one
// entry ahead of use, so its loads stay off the per-segment critical path.
template <typename Real, int P, int TM, bool CM>
__global__ void __launch_bounds__(128, CM ? 8 : 9) sweep_kernel(
    const TrackRec *__restrict__ trk, const SegRec<Real> *__restrict__ seg, const int32_t *__restrict__ link,
    const Real *__restrict__ wgt, const Real *__restrict__ inv_sin,
    const typename Pair<Real>::T *__restrict__ xsq, Real *__restrict__ tsum, Real *__restrict__ tcomp,
    const Real *__restrict__ psi_in, Real *__restrict__ psi_out, const double *__restrict__ scal,
    long long n_threads, int G, int Gp, CmfdDev<Real> cm) {
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
  const int step = d ? -1 : 1;
  // the segment array has kSegPad padding records at each end, so the three-ahead prefetch below
  // never needs a bounds test (records past a track's end belong to a neighbour or the padding)
  const SegRec<Real> *sp = seg + (d ? tr.off + tr.n - 1 : tr.off);
  // crossing entries in travel order: E_k = xent[d ? hi-1-k : lo+k]; the tally for E_k happens after
  // travel step d ? n - 2 - p : p. cx is the next entry, nx the one after it (already loaded).
  int xk = 0, xm = 0, xlo = 0, xhi = 0, xt = 0x7fffffff;
  int2 cx = make_int2(0, -1), nx = make_int2(0, -1);
  if (CM) {
    xlo = cm.xoff[td >> 1];
    xhi = cm.xoff[(td >> 1) + 1];
    xm = xhi - xlo;
    if (xm > 0) cx = cm.xent[d ? xhi - 1 : xlo];
    if (xm > 1) nx = cm.xent[d ? xhi - 2 : xlo + 1];
    if (xm > 0) xt = d ? tr.n - 2 - cx.x : cx.x;
  }
  if (CM && tr.n > 0) {
    Real j = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) j = fma(w[p], psi[p], j);
    if (j != (Real)0) atomicAdd(cm.leak + (size_t)cm.cell[sp->r] * Gp + g, -(double)j);
  }
  Tally<TM, Real> tally;
  SegRec<Real> s0 = sp[0], s1 = sp[step], s2 = sp[2 * step];
  typename Pair<Real>::T xq0 = xsq[(size_t)s0.r * Gp + g];
  typename Pair<Real>::T xq1 = xsq[(size_t)s1.r * Gp + g];
  tally.init((unsigned)(s0.r * Gp + g));
#pragma unroll 2
  for (int n = 0; n < tr.n; ++n) {
    const SegRec<Real> s3 = sp[3 * step];
    const typename Pair<Real>::T xq2 = xsq[(size_t)s2.r * Gp + g];
    const Real tau0 = xq0.x * s0.l;
    Real acc = 0;
    if constexpr (sizeof(Real) == 4) {
      // FP32: polar angles p, p + 1 as the two lanes of packed f32x2 operations (the same
      // roundings as the scalar loop, so the same results), an odd last angle alone
#pragma unroll
      for (int p = 0; p + 1 < P; p += 2) {
        const float2 F = one_minus_exp<true>(mul2(f2(tau0), make_float2(is[p], is[p + 1])));
        const float2 ps = make_float2(psi[p], psi[p + 1]);
        const float2 dl = mul2(sub2(ps, f2(xq0.y)), F);
        const float2 pn = sub2(ps, dl);
        psi[p] = pn.x;
        psi[p + 1] = pn.y;
        acc = fmaf(w[p], dl.x, acc);
        acc = fmaf(w[p + 1], dl.y, acc);
      }
      if constexpr ((P & 1) != 0) {
        const float F = one_minus_exp(tau0 * is[P - 1]);
        const float dl = (psi[P - 1] - xq0.y) * F;
        psi[P - 1] -= dl;
        acc = fmaf(w[P - 1], dl, acc);
      }
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const Real F = one_minus_exp(tau0 * is[p]);
        const Real dl = (psi[p] - xq0.y) * F;
        psi[p] -= dl;
        acc = fma(w[p], dl, acc);
      }
    }
    tally.add(tsum, tcomp, (unsigned)(s0.r * Gp + g), acc);
    if (CM && n == xt) {
      // partial current into the next cell; backward travel crosses the boundary the other way
      Real j = 0;
#pragma unroll
      for (int p = 0; p < P; ++p) j = fma(w[p], psi[p], j);
      atomicAdd(cm.cur + (size_t)(cx.y ^ d) * Gp + g, (double)j);
      ++xk;
      cx = nx;
      xt = (xk < xm) ? (d ? tr.n - 2 - cx.x : cx.x) : 0x7fffffff;
      if (xk + 1 < xm) nx = cm.xent[d ? xhi - 2 - xk : xlo + 1 + xk];
    }
    s0 = s1;
    s1 = s2;
    s2 = s3;
    xq0 = xq1;
    xq1 = xq2;
    sp += step;
  }
  tally.flush(tcomp);
  const int e = link[td];
  if (e >= 0) {
#pragma unroll
    for (int p = 0; p < P; ++p) psi_out[((long long)e * P + p) * G + g] = psi[p];
  }
  if (CM && tr.n > 0) {
    Real j = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) j = fma(w[p], psi[p], j);
    atomicAdd(cm.leak + (size_t)cm.cell[sp[-step].r] * Gp + g, (double)j);
  }
}

// FP32 sweep with packed pairs of groups: one thread per (track, sense, chunk of 2 NP groups), the
// chunk fastest, so the threads of a track end sit side by side in a warp and read one region row
// together. All P polar angles stay in registers; each pair of groups is one f32x2 lane of every
// operation, region rows are read as 128-bit loads of {Sigma_t, q/Sigma_t} pairs and the tallies
// are added with one float4 (NP = 2) or float2 (NP = 1) atomic, so the per-segment cost (segment
// record, addresses, loop, atomics) is shared by 2 NP P updates. The last chunk of a G that is not
// a multiple of 2 NP carries padding groups (Sigma_t = 1, q = 0, no inflow), whose updates are
// zero. The segment array carries kSegPad padding records at each end, so the two-ahead prefetch
// never needs a bounds test. 1/sin(theta_p) arrive as kernel parameters (uniform over the grid,
// no registers or loads).
// Kahan's compensation step (Dekker's Fast2Sum) per lane: the rounding error (old + x) -
// fl(old + x) of the atomic add, exact whenever |old| >= |x| (see Tally<1, float>).
__device__ __forceinline__ float add_err(float o, float x) { return x - ((o + x) - o); }

__device__ __forceinline__ float2 add_err(float2 o, float2 x) { return sub2(x, sub2(add2(o, x), o)); }

__device__ __forceinline__ float4 add_err(float4 o, float4 x) {
  const float2 lo = add_err(make_float2(o.x, o.y), make_float2(x.x, x.y));
  const float2 hi = add_err(make_float2(o.z, o.w), make_float2(x.z, x.w));
  return make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int P> struct PolarInv {
  float v[P];
};

// The tally vector of NP group pairs: one float4 (NP = 2) or one float2 (NP = 1) per lane.
template <int NP> struct PairVec;
template <> struct PairVec<2> {
  using T = float4;
  __device__ __forceinline__ static T make(const float2 (&a)[2]) { return make_float4(a[0].x, a[0].y, a[1].x, a[1].y); }
  __device__ __forceinline__ static T zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
};
template <> struct PairVec<1> {
  using T = float2;
  __device__ __forceinline__ static T make(const float2 (&a)[1]) { return a[0]; }
  __device__ __forceinline__ static T zero() { return make_float2(0.f, 0.f); }
};

template <int P, int TM, int NP>
__global__ void __launch_bounds__(64, 16) sweep_chunk_kernel(
    const TrackRec *__restrict__ trk, const SegRec<float> *__restrict__ seg, const int32_t *__restrict__ link,
    const float *__restrict__ wgt, const PolarInv<P> is, const float2 *__restrict__ xsq, float *__restrict__ tsum,
    float *__restrict__ tcomp, const float *__restrict__ psi_in, float *__restrict__ psi_out,
    const double *__restrict__ scal, long long n_threads, int G, int Gp, int lanes) {
  using V = typename PairVec<NP>::T;
  constexpr int GPT = 2 * NP;  // groups per thread
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_threads) return;
  const long long td = idx / lanes;
  const int g0 = (int)(idx - td * lanes) * GPT;
  const TrackRec tr = trk[td >> 1];
  const int d = (int)(td & 1);
  const float scale = (float)scal[S_SCALE];
  // pair j holds groups g0 + 2j and g0 + 2j + 1
  float2 psi[NP][P];
  float w[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    w[p] = wgt[tr.dir * P + p];
    const float *src = psi_in + (td * P + p) * G + g0;
#pragma unroll
    for (int j = 0; j < NP; ++j)
      psi[j][p] = make_float2((g0 + 2 * j < G) ? src[2 * j] * scale : 0.0f,
                              (g0 + 2 * j + 1 < G) ? src[2 * j + 1] * scale : 0.0f);
  }
  const int step = d ? -1 : 1;
  const SegRec<float> *sp = seg + (d ? tr.off + tr.n - 1 : tr.off);
  const float4 *rows = reinterpret_cast<const float4 *>(xsq + g0);
  const int rstride = Gp / 2;  // float4 per region row
  SegRec<float> s0 = sp[0], s1 = sp[step];
  float4 r0[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) r0[j] = rows[(size_t)s0.r * rstride + j];
  V *tsumv = reinterpret_cast<V *>(tsum + g0);
  V *tcompv = reinterpret_cast<V *>(tcomp + g0);
  const int tstride = Gp / GPT;
  // compensated mode: the old values returned by this segment's atomic become rounding errors one
  // segment later, so the atomic's latency overlaps the next segment's arithmetic
  V p_old = PairVec<NP>::zero(), p_x = p_old;
  size_t p_a = (size_t)s0.r * tstride;
  for (int n = 0; n < tr.n; ++n) {
    const SegRec<float> s2 = sp[2 * step];
    float4 r1[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) r1[j] = rows[(size_t)s1.r * rstride + j];
    // a region row holds {Sigma_t, q/Sigma_t} per group: pair the two groups of each float4
    const float2 l2 = f2(s0.l);
    float2 tau[NP], q[NP], acc[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      tau[j] = mul2(make_float2(r0[j].x, r0[j].z), l2);
      q[j] = make_float2(r0[j].y, r0[j].w);
      acc[j] = f2(0.0f);
    }
#pragma unroll
    for (int p = 0; p < P; ++p) {
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const float2 F = one_minus_exp<false>(mul2(tau[j], f2(is.v[p])));
        const float2 dl = mul2(sub2(psi[j][p], q[j]), F);
        psi[j][p] = sub2(psi[j][p], dl);
        acc[j] = fma2(f2(w[p]), dl, acc[j]);
      }
    }
    const size_t a = (size_t)s0.r * tstride;
    const V x = PairVec<NP>::make(acc);
    if (TM == 1) {
      const V o = atomicAdd(tsumv + a, x);
      atomicAdd(tcompv + p_a, add_err(p_old, p_x));
      p_old = o;
      p_x = x;
    } else {
      atomicAdd(tsumv + a, x);
    }
    p_a = a;
    s0 = s1;
    s1 = s2;
#pragma unroll
    for (int j = 0; j < NP; ++j) r0[j] = r1[j];
    sp += step;
  }
  if (TM == 1) atomicAdd(tcompv + p_a, add_err(p_old, p_x));
  const int e = link[td];
  if (e >= 0) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
      float *dst = psi_out + ((long long)e * P + p) * G + g0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        if (g0 + 2 * j < G) dst[2 * j] = psi[j][p].x;
        if (g0 + 2 * j + 1 < G) dst[2 * j + 1] = psi[j][p].y;
      }
    }
  }
}

// ----------------------------------------------------------------------------- finalize
// One thread per region. Writes phi' (unnormalised), zeroes the tallies, and per block:
// [0] sum_i A_i f'_i, [1] min and [2] max of fold_i / f'_i over f'_i > 0 (eigen mode),
// [3] max relative flux change (fixed-source mode).
template <typename Real, int TM>
__global__ void __launch_bounds__(256) finalize_kernel(
    int R, int G, int Gp, const int32_t *__restrict__ mat, const Real *__restrict__ nsf,
    const double *__restrict__ area, const Real *__restrict__ inv_ta,
    const typename Pair<Real>::T *__restrict__ xsq, Real *__restrict__ tsum,
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
      const double ph = fma(t, (double)inv_ta[a], kFourPi * (double)v.y);
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

__device__ __forceinline__ void reduce_partials(int nb, const double *__restrict__ part, double *__restrict__ scal,
                                                int eigen);

// Group-parallel variant for Gp = 8: 8 consecutive threads own one region (coalesced row
// accesses). Per region and group the arithmetic is in the sweep's type (FP32 mode: the
// compensation is folded by one FP32 add, i.e. the compensated sum rounded once, and phi is stored
// in FP32 anyway); FP64 is used for A_i f_i and every reduction. The last block to finish (atomic
// ticket after a memory fence; no waiting) reduces all block partials, so no separate reduce
// launch is needed. 1/(Sigma_t A) is precomputed (no division per region and group).
template <typename Real, int TM>
__global__ void __launch_bounds__(256) finalize8_kernel(
    int R, int G, const int32_t *__restrict__ mat, const Real *__restrict__ nsf, const Real *__restrict__ inv_ta,
    const typename Pair<Real>::T *__restrict__ xsq, Real *__restrict__ tsum, Real *__restrict__ tcomp,
    Real *__restrict__ phi, const double *__restrict__ fold, const double *__restrict__ area,
    double *__restrict__ part, unsigned *__restrict__ ticket, double *__restrict__ scal, int eigen) {
  __shared__ double l_sum[32];
  __shared__ Real l_min[32], l_max[32], l_res[32];
  __shared__ bool last;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = tid >> 3, g = tid & 7;
  const bool live = r < R;
  // everything per region and group stays in the sweep's type: the FP64 pipe is reserved for
  // A_i f_i and the block totals
  Real f = 0, res = 0;
  if (live) {
    const size_t a = (size_t)r * 8 + g;
    const typename Pair<Real>::T v = xsq[a];
    Real t = tsum[a];
    tsum[a] = (Real)0;
    if (TM == 1) {
      t += tcomp[a];
      tcomp[a] = (Real)0;
    }
    if (g < G) {
      const Real ph = fma(t, inv_ta[a], (Real)kFourPi * v.y);
      if (!eigen) {
        const Real old = phi[a];
        if (ph > (Real)0) res = fabs(ph - old) / ph;
      }
      phi[a] = ph;
      f = nsf[mat[r] * G + g] * ph;
    }
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (!eigen) {
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) res = fmax(res, __shfl_xor_sync(0xffffffffu, res, o));
  }
  if (g == 0) {
    const int q = threadIdx.x >> 3;
    const bool fis = live && eigen && f > (Real)0;
    const Real rho = fis ? (Real)fold[r] / f : (Real)0;
    l_sum[q] = live ? area[r] * (double)f : 0.0;
    l_min[q] = fis ? rho : (Real)INFINITY;
    l_max[q] = fis ? rho : (Real)-INFINITY;
    l_res[q] = res;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    Real mn = (Real)INFINITY, mx = (Real)-INFINITY, rs = 0;
    for (int q = 0; q < (int)(blockDim.x >> 3); ++q) {
      a += l_sum[q];
      mn = fmin(mn, l_min[q]);
      mx = fmax(mx, l_max[q]);
      rs = fmax(rs, l_res[q]);
    }
    part[4 * blockIdx.x + 0] = a;
    part[4 * blockIdx.x + 1] = (double)mn;
    part[4 * blockIdx.x + 2] = (double)mx;
    part[4 * blockIdx.x + 3] = (double)rs;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    reduce_partials(gridDim.x, part, scal, eigen);
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

// Many groups (G > 8): eight threads per region (lane l owns groups l, l + 8, ... below Gp; GPL =
// ceil(Gp / 8), 0: computed at run time), 32 regions per tile, the blocks striding over the tiles
// (the grid is fixed by the launch: every sum has a fixed order). Each 8-lane group keeps running
// FP64 partials of its own regions; the block adds its 32 groups' partials in order once at the
// end, so there is one memory fence and one ticket per block, and the last block to finish
// reduces all block partials. Per region and group the arithmetic is in the sweep's type, as in
// finalize8_kernel; the region's fission rate is an 8-lane shuffle sum.
template <typename Real, int TM, int GPL>
__global__ void __launch_bounds__(256) finalize_lanes_kernel(
    int R, int G, int Gp, const int32_t *__restrict__ mat, const Real *__restrict__ nsf,
    const Real *__restrict__ inv_ta, const typename Pair<Real>::T *__restrict__ xsq, Real *__restrict__ tsum,
    Real *__restrict__ tcomp, Real *__restrict__ phi, const double *__restrict__ fold,
    const double *__restrict__ area, double *__restrict__ part, unsigned *__restrict__ ticket,
    double *__restrict__ scal, int eigen) {
  __shared__ double l_sum[32];
  __shared__ Real l_min[32], l_max[32], l_res[32];
  __shared__ bool last;
  constexpr int NJ = GPL > 0 ? GPL : 1;
  const int gpl = GPL > 0 ? GPL : (Gp + 7) / 8;
  const int qg = threadIdx.x >> 3, l = threadIdx.x & 7;
  const int ntile = (R + 31) / 32;
  double g_sum = 0.0;
  Real g_min = (Real)INFINITY, g_max = (Real)-INFINITY, g_res = 0;
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int r = tile * 32 + qg;
    const bool live = r < R;
    Real f = 0, res = 0;
    if (live && GPL > 0) {
      // every load of the region's groups first (independent, all in flight together), then the
      // arithmetic and the stores
      const int m = mat[r];
      Real t[NJ], c[NJ], q[NJ], ita[NJ], nf[NJ], old[NJ];
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int g = l + 8 * j;
        const size_t a = (size_t)r * Gp + g;
        t[j] = c[j] = q[j] = ita[j] = nf[j] = old[j] = (Real)0;
        if (g < Gp) {
          t[j] = tsum[a];
          if (TM == 1) c[j] = tcomp[a];
          q[j] = xsq[a].y;
          ita[j] = inv_ta[a];
          if (g < G) nf[j] = nsf[m * G + g];
          if (!eigen) old[j] = phi[a];
        }
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int g = l + 8 * j;
        const size_t a = (size_t)r * Gp + g;
        if (g < Gp) {
          tsum[a] = (Real)0;
          if (TM == 1) tcomp[a] = (Real)0;
        }
        if (g < G) {
          const Real ph = fma(TM == 1 ? t[j] + c[j] : t[j], ita[j], (Real)kFourPi * q[j]);
          if (!eigen && ph > (Real)0) res = fmax(res, fabs(ph - old[j]) / ph);
          phi[a] = ph;
          f += nf[j] * ph;
        }
      }
    } else if (live) {
      const int m = mat[r];
      for (int j = 0; j < gpl; ++j) {
        const int g = l + 8 * j;
        if (g >= Gp) break;
        const size_t a = (size_t)r * Gp + g;
        const typename Pair<Real>::T v = xsq[a];
        Real t = tsum[a];
        tsum[a] = (Real)0;
        if (TM == 1) {
          t += tcomp[a];
          tcomp[a] = (Real)0;
        }
        if (g < G) {
          const Real ph = fma(t, inv_ta[a], (Real)kFourPi * v.y);
          if (!eigen) {
            const Real old = phi[a];
            if (ph > (Real)0) res = fmax(res, fabs(ph - old) / ph);
          }
          phi[a] = ph;
          f += nsf[m * G + g] * ph;
        }
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (!eigen) {
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) res = fmax(res, __shfl_xor_sync(0xffffffffu, res, o));
    }
    if (l == 0 && live) {
      g_sum += area[r] * (double)f;
      if (eigen && f > (Real)0) {
        const Real rho = (Real)fold[r] / f;
        g_min = fmin(g_min, rho);
        g_max = fmax(g_max, rho);
      }
      g_res = fmax(g_res, res);
    }
  }
  if (l == 0) {
    l_sum[qg] = g_sum;
    l_min[qg] = g_min;
    l_max[qg] = g_max;
    l_res[qg] = g_res;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    Real mn = (Real)INFINITY, mx = (Real)-INFINITY, rs = 0;
    for (int q = 0; q < 32; ++q) {
      a += l_sum[q];
      mn = fmin(mn, l_min[q]);
      mx = fmax(mx, l_max[q]);
      rs = fmax(rs, l_res[q]);
    }
    part[4 * blockIdx.x + 0] = a;
    part[4 * blockIdx.x + 1] = (double)mn;
    part[4 * blockIdx.x + 2] = (double)mx;
    part[4 * blockIdx.x + 3] = (double)rs;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    reduce_partials(gridDim.x, part, scal, eigen);
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

// ----------------------------------------------------------------------------- finalize, bulk
// FP32 finalize for many groups with its inputs staged by the copy engine's bulk path: a tile's 32
// region rows of tsum, tcomp, 1/(Sigma_t A), the old flux (fixed-source mode) and the {Sigma_t,
// q/Sigma_t} pairs are contiguous, so each is one cp.async.bulk copy into shared memory, completed
// on an mbarrier. Tiles are double-buffered: the copies of a block's next tile are in flight while
// it computes the current one, so many bytes are outstanding per SM without registers to hold
// them. The arithmetic, the stores and the fixed-order reduction are those of
// finalize_lanes_kernel, so the results are the same bit for bit. A wait that has not completed
// after about a second sets S_STATUS = 2 (the host reports an error), waits (again bounded) for the
// block's copies still in flight, and leaves the loop.
__device__ __forceinline__ uint32_t bulk_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bulk_expect(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bulk_smem(bar)), "r"(bytes) : "memory");
}

// global -> shared, bytes a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   bulk_smem(dst)),
               "l"(src), "r"(bytes), "r"(bulk_smem(bar))
               : "memory");
}

__device__ __forceinline__ uint64_t bulk_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the mbarrier phase of the given parity; false after about one second
__device__ __forceinline__ bool bulk_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = bulk_smem(bar);
  const uint64_t t0 = bulk_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (bulk_ns() - t0 > 1000000000ull) return false;
  }
}

// Shared memory per stage (floats): tsum | tcomp (TM = 1) | 1/(Sigma_t A) | old flux (fixed
// source) | pairs (2 per element), each 32 * Gp long.
__host__ __device__ constexpr int finalize_bulk_stage_floats(int Gp, int TM, int eigen) {
  return 32 * Gp * (2 + TM + (eigen ? 0 : 1) + 2);
}

template <int TM, int GPL>
__global__ void __launch_bounds__(256) finalize_bulk_kernel(
    int R, int G, int Gp, const int32_t *__restrict__ mat, const float *__restrict__ nsf,
    const float *__restrict__ inv_ta, const float2 *__restrict__ xsq, float *__restrict__ tsum,
    float *__restrict__ tcomp, float *__restrict__ phi, const double *__restrict__ fold,
    const double *__restrict__ area, double *__restrict__ part, unsigned *__restrict__ ticket,
    double *__restrict__ scal, int eigen) {
  extern __shared__ __align__(16) float fb_dyn[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ double l_sum[32];
  __shared__ float l_min[32], l_max[32], l_res[32];
  __shared__ bool last;
  __shared__ int s_fail;
  const int qg = threadIdx.x >> 3, l = threadIdx.x & 7;
  const int ntile = (R + 31) / 32;
  const int tf = 32 * Gp, stage_f = finalize_bulk_stage_floats(Gp, TM, eigen);
  auto st_t = [&](int st) { return fb_dyn + st * stage_f; };
  auto st_c = [&](int st) { return fb_dyn + st * stage_f + tf; };
  auto st_i = [&](int st) { return fb_dyn + st * stage_f + tf * (1 + TM); };
  auto st_o = [&](int st) { return fb_dyn + st * stage_f + tf * (2 + TM); };
  auto st_q = [&](int st) { return fb_dyn + st * stage_f + tf * (2 + TM + (eigen ? 0 : 1)); };
  // thread 0: every copy of one tile into one stage, the byte count announced first
  auto issue = [&](int tile, int st) {
    const int r0 = tile * 32, nr = min(32, R - r0);
    const size_t off = (size_t)r0 * Gp;
    const uint32_t n4 = (uint32_t)(nr * Gp) * 4u;
    const uint32_t total = n4 * (2u + (uint32_t)TM + (eigen ? 0u : 1u)) + 2u * n4;
    bulk_expect(&bar[st], total);
    bulk_g2s(st_t(st), tsum + off, n4, &bar[st]);
    if (TM == 1) bulk_g2s(st_c(st), tcomp + off, n4, &bar[st]);
    bulk_g2s(st_i(st), inv_ta + off, n4, &bar[st]);
    if (!eigen) bulk_g2s(st_o(st), phi + off, n4, &bar[st]);
    bulk_g2s(st_q(st), xsq + off, 2u * n4, &bar[st]);
  };
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bulk_smem(&bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bulk_smem(&bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0 && (int)blockIdx.x < ntile) issue(blockIdx.x, 0);
  double g_sum = 0.0;
  float g_min = INFINITY, g_max = -INFINITY, g_res = 0.f;
  int k = 0, tile = blockIdx.x;
  for (; tile < ntile; tile += gridDim.x, ++k) {
    const int st = k & 1;
    const int nxt = tile + (int)gridDim.x;
    if (threadIdx.x == 0 && nxt < ntile) {
      // the stage was last read before the barrier that ended the previous iteration
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(nxt, st ^ 1);
    }
    const int r = tile * 32 + qg;
    const bool live = r < R;
    // per-region inputs that are not staged, loaded while the tile's copies complete
    int m = 0;
    double ar = 0.0, fo = 0.0;
    if (live) {
      m = mat[r];
      if (l == 0) {
        ar = area[r];
        if (eigen) fo = fold[r];
      }
    }
    if (!bulk_wait(&bar[st], (uint32_t)(k >> 1) & 1u)) s_fail = 1;
    float f = 0.f, res = 0.f;
    if (live) {
      const float *t_ = st_t(st), *c_ = st_c(st), *i_ = st_i(st), *o_ = st_o(st), *q_ = st_q(st);
      const int base = qg * Gp;
#pragma unroll
      for (int j = 0; j < GPL; ++j) {
        const int g = l + 8 * j;
        if (g < Gp) {
          const size_t a = (size_t)r * Gp + g;
          const float t = t_[base + g];
          const float c = TM == 1 ? c_[base + g] : 0.f;
          tsum[a] = 0.f;
          if (TM == 1) tcomp[a] = 0.f;
          if (g < G) {
            const float ph = fmaf(TM == 1 ? t + c : t, i_[base + g], (float)kFourPi * q_[2 * (base + g) + 1]);
            if (!eigen && ph > 0.f) res = fmaxf(res, fabsf(ph - o_[base + g]) / ph);
            phi[a] = ph;
            f += nsf[m * G + g] * ph;
          }
        }
      }
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
    if (!eigen) {
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) res = fmaxf(res, __shfl_xor_sync(0xffffffffu, res, o));
    }
    if (l == 0 && live) {
      g_sum += ar * (double)f;
      if (eigen && f > 0.f) {
        const float rho = (float)fo / f;
        g_min = fminf(g_min, rho);
        g_max = fmaxf(g_max, rho);
      }
      g_res = fmaxf(g_res, res);
    }
    __syncthreads();  // every read of this stage done before the next iteration refills it
    if (s_fail) break;
  }
  if (s_fail && threadIdx.x == 0) {
    // the stage that timed out and the next tile's copies, if issued, may still be in flight
    bulk_wait(&bar[k & 1], (uint32_t)(k >> 1) & 1u);
    if (tile + (int)gridDim.x < ntile) bulk_wait(&bar[(k + 1) & 1], (uint32_t)((k + 1) >> 1) & 1u);
    scal[S_STATUS] = 2.0;
  }
  if (l == 0) {
    l_sum[qg] = g_sum;
    l_min[qg] = g_min;
    l_max[qg] = g_max;
    l_res[qg] = g_res;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    float mn = INFINITY, mx = -INFINITY, rs = 0.f;
    for (int q = 0; q < 32; ++q) {
      a += l_sum[q];
      mn = fminf(mn, l_min[q]);
      mx = fmaxf(mx, l_max[q]);
      rs = fmaxf(rs, l_res[q]);
    }
    part[4 * blockIdx.x + 0] = a;
    part[4 * blockIdx.x + 1] = (double)mn;
    part[4 * blockIdx.x + 2] = (double)mx;
    part[4 * blockIdx.x + 3] = (double)rs;
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    reduce_partials(gridDim.x, part, scal, eigen);
    if (threadIdx.x == 0) *ticket = 0u;
  }
}

// ----------------------------------------------------------------------------- reduce
// Final reduction of the block partials by one block of 256 threads in a fixed order
// (deterministic): k' = k F' (the flux the source was built from is normalised to F = 1);
// scale = 1/F'; residual max_i |f'_i/F' - fold_i| / (f'_i/F') = max(|1 - F' rho_min|, |1 - F' rho_max|).
__device__ __forceinline__ void reduce_partials(int nb, const double *__restrict__ part, double *__restrict__ scal,
                                                int eigen) {
  __shared__ double s_sum[256], s_min[256], s_max[256], s_res[256];
  double a = 0.0, mn = INFINITY, mx = -INFINITY, rs = 0.0;
  // unrolled so that many partials' loads are in flight at once (the sum's order is unchanged)
#pragma unroll 8
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

__global__ void __launch_bounds__(256) reduce_kernel(int nb, const double *__restrict__ part,
                                                     double *__restrict__ scal, int eigen) {
  reduce_partials(nb, part, scal, eigen);
}

// ----------------------------------------------------------------------------- warm start
// features: (Sigma_t, nuSigma_f, Sigma_a) of the region's material, geometry row, global vector
template <typename Real>
__global__ void ws_features_kernel(int R, int G, int n_geo, int n_glob, const int32_t *__restrict__ mat,
                                   const Real *__restrict__ sig_t, const Real *__restrict__ nsf,
                                   const Real *__restrict__ sig_s, const float *__restrict__ geo,
                                   const float *__restrict__ glob, float *__restrict__ feat) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int m = mat[r];
  const int nf = 3 * G + n_geo + n_glob;
  float *f = feat + (size_t)r * nf;
  for (int g = 0; g < G; ++g) {
    double out = 0.0;
    for (int h = 0; h < G; ++h) out += (double)sig_s[((size_t)m * G + g) * G + h];
    f[g] = (float)sig_t[m * G + g];
    f[G + g] = (float)nsf[m * G + g];
    f[2 * G + g] = (float)((double)sig_t[m * G + g] - out);
  }
  for (int j = 0; j < n_geo; ++j) f[3 * G + j] = geo[(size_t)r * n_geo + j];
  for (int j = 0; j < n_glob; ++j) f[3 * G + n_geo + j] = glob[j];
}

// phi = exp(pred[:, :G]); block partials of sum A f(phi), sum A pred[:, G], sum A
template <typename Real>
__global__ void __launch_bounds__(256) ws_apply_kernel(int R, int G, int Gp, const int32_t *__restrict__ mat,
                                                       const Real *__restrict__ nsf, const double *__restrict__ area,
                                                       const float *__restrict__ pred, Real *__restrict__ phi,
                                                       double *__restrict__ part) {
  __shared__ double s0[256], s1[256], s2[256];
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, b = 0.0, c = 0.0;
  if (r < R) {
    const int m = mat[r];
    const double A = area[r];
    double f = 0.0;
    for (int g = 0; g < G; ++g) {
      const Real v = (Real)exp((double)pred[(size_t)r * (G + 1) + g]);
      phi[(size_t)r * Gp + g] = v;
      f += (double)nsf[m * G + g] * (double)v;
    }
    a = A * f;
    b = A * (double)pred[(size_t)r * (G + 1) + G];
    c = A;
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  s2[threadIdx.x] = c;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      s0[threadIdx.x] += s0[threadIdx.x + k];
      s1[threadIdx.x] += s1[threadIdx.x + k];
      s2[threadIdx.x] += s2[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[4 * blockIdx.x + 0] = s0[0];
    part[4 * blockIdx.x + 1] = s1[0];
    part[4 * blockIdx.x + 2] = s2[0];
    part[4 * blockIdx.x + 3] = 0.0;
  }
}

// one block: F, area-weighted mean k; scalars reset for a fresh iteration
__global__ void __launch_bounds__(256) ws_reduce_kernel(int nb, const double *__restrict__ part,
                                                        double *__restrict__ scal) {
  __shared__ double s0[256], s1[256], s2[256];
  double a = 0.0, b = 0.0, c = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += part[4 * i];
    b += part[4 * i + 1];
    c += part[4 * i + 2];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  s2[threadIdx.x] = c;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      s0[threadIdx.x] += s0[threadIdx.x + k];
      s1[threadIdx.x] += s1[threadIdx.x + k];
      s2[threadIdx.x] += s2[threadIdx.x + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double F = s0[0];
    const double k = s1[0] / s2[0];
    scal[S_K] = k;
    scal[S_KPREV] = k;
    scal[S_SCALE] = (F > 0.0) ? 1.0 / F : 1.0;
    scal[S_FISS] = F;
    scal[S_RESID] = INFINITY;
    scal[S_STATUS] = (isfinite(k) && k > 0.0 && isfinite(F)) ? 0.0 : 1.0;
  }
}

// incoming boundary flux of each linked end (t, d) = phi(region at that end) / (4 pi)
template <typename Real>
__global__ void ws_psi_kernel(long long n, int P, int G, int Gp, const TrackRec *__restrict__ trk,
                              const SegRec<Real> *__restrict__ seg, const uint8_t *__restrict__ fed,
                              const Real *__restrict__ phi, Real *__restrict__ psi) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const long long td = idx / G;
  const int g = (int)(idx - td * G);
  const TrackRec tr = trk[td >> 1];
  const int d = (int)(td & 1);
  Real v = 0;
  if (fed[td]) {
    const int r = seg[d ? tr.off + tr.n - 1 : tr.off].r;
    v = phi[(size_t)r * Gp + g] * (Real)(1.0 / kFourPi);
  }
  for (int p = 0; p < P; ++p) psi[(td * P + p) * G + g] = v;
}

}  // namespace moc
