// DGMOC kernels (Sec. 2.2 "DGMOC formulation", Eq. DGMOC_expansion to DGMOC_weak_up; the
// plane-by-plane upward/downward march of Alg. 2): the planar tracks extruded through nz axial
// planes, the angular flux on each characteristic expanded in every plane as a + b xi (xi from -1
// at the plane's bottom to +1 at its top), axial faces upwinded.
//
// Along a track, for a march in the direction of increasing xi (upward; a downward march is the
// same system for (a, -b) with the linear source negated), c = mu / dz:
//     y' = r - K y,   y = (a, b),   K = [(Sigma_t + 2c) I + c N] / sin(theta),   N = [[-1, 1], [-3, 1]],
//     r = (q0 + c psi_in, q1 - 3 c psi_in) / sin(theta),
// with psi_in the axial inflow (segment average of the upwind plane's outflow trace a + b).
// N^2 = -2 I, so every function of K is a combination of I and N: with
//     gamma = (Sigma_t + 2c) l / sin(theta),  beta = sqrt(2) c l / sin(theta),
//     exp(-K l) = e^-gamma [cos(beta) I - sin(beta)/sqrt(2) N],
//     K^-1 = sin(theta) [(Sigma_t + 2c) I - c N] / D,   D = (Sigma_t + 2c)^2 + 2 c^2,
// and one segment is
//     y_inf = [(Sigma_t + 2c) rr - c N rr] / D          (rr = sin(theta) r: sin(theta) cancels),
//     (I - E)(y0 - y_inf) = A0 d + A1 N d,  d = y0 - y_inf,
//         A0 = (1 - e^-gamma) + e^-gamma 2 sin^2(beta/2),  A1 = e^-gamma sin(beta)/sqrt(2),
//     y(l) = y0 - (I - E) d,
//     integral of y over the segment = l y_inf + K^-1 (y0 - y(l)).
// The closed forms avoid a general matrix exponential and any cancellation in 1 - e^-gamma.
//
// Per outer: dg_source_kernel (source moments), the sweep (dg_sweep_res_kernel, or
// dg_sweep_kernel when its shared memory would not fit: both marches of every track, sense, polar
// angle and group), dg_finalize_kernel (flux moments, FP64 block partials) and the planar
// reduce_kernel (k, normalisation, residual); with the axial acceleration also dg_cm_sums_kernel,
// the planar cmfd_coeff_kernel, dg_cm_solve_kernel, dg_cm_prolong_kernel and dg_cm_psi_kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "moc_kernels.cuh"

namespace moc {

template <typename Real> struct alignas(4 * sizeof(Real)) DgXs {
  Real t;    // Sigma_t
  Real q0;   // plane-average source per steradian
  Real q1;   // linear (xi) source coefficient per steradian
  Real pad;
};

// thinnest plane moc_set_axial accepts (cm); it bounds c = mu/dz for the approximate reciprocal
constexpr double kDgMinPlane = 1e-9;

template <typename Real> struct DgMath;
template <> struct DgMath<double> {
  __device__ static double rcp(double x) { return 1.0 / x; }
  __device__ static double rcp_fast(double x) { return 1.0 / x; }
  __device__ static double one_minus_exp(double x) { return -expm1(-x); }
  __device__ static void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
};
template <> struct DgMath<float> {
  __device__ static float rcp(float x) { return __frcp_rn(x); }  // correctly rounded 1/x
  // the per-update 1/D (D = (Sigma_t + 2c)^2 + 2c^2, c = mu/dz): CUDA's approximate division,
  // within 2 ulp for D up to 2^126, in place of the correctly rounded reciprocal, whose longer
  // path cost 13% of the sweep. moc_set_axial rejects planes thinner than kDgMinPlane, so
  // c <= 1e9/cm and D stays far below 2^126 for any Sigma_t under 1e18/cm (above 2^126 the
  // approximate quotient would flush to 0)
  __device__ static float rcp_fast(float x) { return __fdividef(1.0f, x); }
  __device__ static float one_minus_exp(float x) { return moc::one_minus_exp(x); }
  // x >= 0. Below 0.5 (thick planes: the usual case) the Taylor polynomials of sin to x^7 and cos
  // to x^8, whose remainders (x^9/9!, x^10/10!) stay below 1.1e-8 relative, i.e. within FP32
  // rounding; above it CUDA's sincosf.
  __device__ static void sincos_(float x, float *s, float *c) {
    if (x <= 0.5f) {
      const float x2 = x * x;
      *s = x * fmaf(x2, fmaf(x2, fmaf(x2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), 1.0f);
      *c = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 1.0f);
    } else {
      sincosf(x, s, c);
    }
  }
};

// Source moments of every element (plane z, region r): one thread per element.
// phi3 [E][Gp][2] (m fastest), E = nz * R, is scaled by the pending normalisation first; fold[e]
// receives the element's normalised fission rate.
template <typename Real>
__global__ void dg_source_kernel(int E, int R, int G, int Gp, int M, const int32_t *__restrict__ mat3,
                                 const Real *__restrict__ sig_t, const Real *__restrict__ nsf,
                                 const Real *__restrict__ chi, const Real *__restrict__ sig_s,
                                 const double *__restrict__ ext, Real *__restrict__ phi3, DgXs<Real> *__restrict__ xs3,
                                 double *__restrict__ fold, const double *__restrict__ scal, int eigen) {
  extern __shared__ unsigned char smem_raw[];
  Real *s_ss = reinterpret_cast<Real *>(smem_raw);  // [M][G][G]
  for (int i = threadIdx.x; i < M * G * G; i += blockDim.x) s_ss[i] = sig_s[i];
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int r = e % R;
  const int m = mat3[e];
  const Real scale = eigen ? (Real)scal[S_SCALE] : (Real)1;
  const Real inv_k = eigen ? (Real)(1.0 / scal[S_K]) : (Real)0;
  Real *ph = phi3 + (size_t)e * Gp * 2;
  Real fis0 = 0, fis1 = 0;
  for (int g = 0; g < G; ++g) {
    const Real v0 = ph[2 * g] * scale, v1 = ph[2 * g + 1] * scale;
    ph[2 * g] = v0;
    ph[2 * g + 1] = v1;
    fis0 += nsf[m * G + g] * v0;
    fis1 += nsf[m * G + g] * v1;
  }
  if (eigen) fold[e] = (double)fis0;
  const Real *ss = s_ss + (size_t)m * G * G;
  const Real inv4pi = (Real)(1.0 / kFourPi);
  for (int g = 0; g < G; ++g) {
    Real s0 = 0, s1 = 0;
    for (int gp = 0; gp < G; ++gp) {
      s0 += ss[gp * G + g] * ph[2 * gp];
      s1 += ss[gp * G + g] * ph[2 * gp + 1];
    }
    s0 += chi[m * G + g] * inv_k * fis0;
    s1 += chi[m * G + g] * inv_k * fis1;
    if (ext) s0 += (Real)ext[(size_t)r * G + g];
    DgXs<Real> x;
    x.t = sig_t[m * G + g];
    x.q0 = s0 * inv4pi;
    x.q1 = s1 * inv4pi;
    x.pad = 0;
    xs3[(size_t)e * Gp + g] = x;
  }
}

// One segment of one plane for one polar angle: (y0, y1) = (a, +-b) entering, pin the axial
// inflow, cc = mu/dz, lis = l/sin(theta), st = sin(theta). Updates (y0, y1) to the segment's end
// and returns the segment integrals (i0, i1) of the two moments.
template <typename Real>
__device__ __forceinline__ void dg_update(Real t, Real q0, Real q1s, Real cc, Real l, Real lis, Real st, Real pin,
                                          Real &y0, Real &y1, Real &i0, Real &i1) {
  const Real rs2 = (Real)0.70710678118654752440;  // 1/sqrt(2)
  const Real al = t + 2 * cc;
  const Real iD = DgMath<Real>::rcp_fast(al * al + 2 * cc * cc);
  // y_inf = (al rr - c N rr) / D
  const Real r0 = q0 + cc * pin, r1 = q1s - 3 * cc * pin;
  const Real n0 = r1 - r0, n1 = r1 - 3 * r0;  // N rr
  const Real yi0 = (al * r0 - cc * n0) * iD, yi1 = (al * r1 - cc * n1) * iD;
  const Real omg = DgMath<Real>::one_minus_exp(al * lis);
  const Real eg = (Real)1 - omg;
  Real sh, ch;
  DgMath<Real>::sincos_(cc * lis * rs2, &sh, &ch);  // beta / 2
  const Real A0 = omg + eg * 2 * sh * sh;
  const Real A1 = eg * (2 * sh * ch) * rs2;
  const Real d0 = y0 - yi0, d1 = y1 - yi1;
  const Real dy0 = A0 * d0 + A1 * (d1 - d0);  // (I - E) d
  const Real dy1 = A0 * d1 + A1 * (d1 - 3 * d0);
  y0 -= dy0;
  y1 -= dy1;
  // segment integral: l y_inf + sin(theta) (al dy - c N dy) / D
  const Real sD = st * iD;
  i0 = l * yi0 + sD * (al * dy0 - cc * (dy1 - dy0));
  i1 = l * yi1 + sD * (al * dy1 - cc * (dy1 - 3 * dy0));
}

template <typename Real> __device__ __forceinline__ void dg_tally(Real *t, Real a0, Real a1) {
  atomicAdd(t, a0);
  atomicAdd(t + 1, a1);
}
template <> __device__ __forceinline__ void dg_tally<float>(float *t, float a0, float a1) {
  atomicAdd(reinterpret_cast<float2 *>(t), make_float2(a0, a1));
}

// One thread per (track, sense, group); polar angles in registers. The thread marches its track
// down through the planes (top first), then up, each plane a pass over the track's segments. The
// axial inflow of a segment comes from `face`, where the same thread stored the segment's outflow
// trace in the previous plane of the march, so no other thread is involved:
//   face [S + pad][2 sense][P][G]: before the downward march it holds the previous sweep's upward
//   top traces (used if the top is reflective), after it the bottom traces (used by the upward
//   march if the bottom is reflective), after the upward march the top traces again.
// Radial boundary moments psi3 [2T][2 march][nz][P][2][G] are routed through the planar links
// (Jacobi, double-buffered). Tally [E][Gp][2]: sum of W * segment integral of (a, b) per element.
template <typename Real, int P>
__global__ void __launch_bounds__(128) dg_sweep_kernel(
    const TrackRec *__restrict__ trk, const SegRec<Real> *__restrict__ seg, const int32_t *__restrict__ link,
    const Real *__restrict__ wdg, const Real *__restrict__ sin_t, const Real *__restrict__ inv_sin,
    const Real *__restrict__ cz, const DgXs<Real> *__restrict__ xs3, Real *__restrict__ tally,
    const Real *__restrict__ psi_in, Real *__restrict__ psi_out, Real *__restrict__ face,
    const double *__restrict__ scal, long long n_threads, int G, int Gp, int R, int nz, int bc_bottom, int bc_top) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_threads) return;
  const long long td = idx / G;
  const int g = (int)(idx - td * G);
  const TrackRec tr = trk[td >> 1];
  const int d = (int)(td & 1);
  const Real scale = (Real)scal[S_SCALE];
  Real w[P], st[P], is[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    w[p] = wdg[tr.dir * P + p];
    st[p] = sin_t[p];
    is[p] = inv_sin[p];
  }
  const int step = d ? -1 : 1;
  const long long s_first = d ? tr.off + tr.n - 1 : tr.off;
  const int e_out = link[td];
  for (int ud = 0; ud < 2; ++ud) {
    const Real sg = ud ? (Real)1 : (Real)-1;
    // inflow of the march's first plane: reflective top (downward) reads the previous sweep's
    // top traces in the previous normalisation; reflective bottom (upward) this sweep's bottom
    // traces; vacuum: none
    const bool refl = ud ? (bc_bottom != 0) : (bc_top != 0);
    const Real f0scale = ud ? (Real)1 : scale;
    for (int zi = 0; zi < nz; ++zi) {
      const int z = ud ? zi : nz - 1 - zi;
      const bool first = (zi == 0);
      const Real fmul = first ? (refl ? f0scale : (Real)0) : (Real)1;
      Real y0[P], y1[P], c[P];
      const long long bb = (((td * 2 + ud) * nz + z) * P) * 2;
#pragma unroll
      for (int p = 0; p < P; ++p) {
        y0[p] = psi_in[(bb + 2 * p) * G + g] * scale;
        y1[p] = psi_in[(bb + 2 * p + 1) * G + g] * scale;
        c[p] = cz[z * P + p];
      }
      const DgXs<Real> *xz = xs3 + (size_t)z * R * Gp + g;
      Real *tz = tally + ((size_t)z * R * Gp + g) * 2;
      const SegRec<Real> *sp = seg + s_first;
      Real *fp = face + ((s_first * 2 + d) * P) * G + g;
      const long long fstep = (long long)step * 2 * P * G;
      for (int n = 0; n < tr.n; ++n) {
        const SegRec<Real> s = *sp;
        const DgXs<Real> x = xz[(size_t)s.r * Gp];
        const Real q1s = sg * x.q1;
        const Real il = DgMath<Real>::rcp(s.l);
        Real a0 = 0, a1 = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          // a vacuum or reflective first inflow is zero or the stored trace, without branching
          const Real fin = fp[p * G];
          const Real pin = fmul == (Real)0 ? (Real)0 : fin * fmul;
          Real i0, i1;
          dg_update<Real>(x.t, x.q0, q1s, c[p], s.l, s.l * is[p], st[p], pin, y0[p], y1[p], i0, i1);
          a0 = fma(w[p], i0, a0);
          a1 = fma(w[p], i1, a1);
          fp[p * G] = (i0 + i1) * il;  // outflow trace, segment average
        }
        dg_tally<Real>(tz + (size_t)s.r * Gp * 2, a0, sg * a1);
        sp += step;
        fp += fstep;
      }
      if (e_out >= 0) {
        const long long ob = ((((long long)e_out * 2 + ud) * nz + z) * P) * 2;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          psi_out[(ob + 2 * p) * G + g] = y0[p];
          psi_out[(ob + 2 * p + 1) * G + g] = y1[p];
        }
      }
    }
  }
}

// The same sweep with the loops interchanged: for each segment of the track, the downward march
// through all planes and then the upward march, so the axial inflow of a plane is the outflow the
// thread computed for the same segment one plane upwind, kept in a register (no interface buffer
// in memory; only a reflective top stores its top traces for the next sweep). The radial state of
// every (march, plane, polar angle) lives in shared memory, one column per thread
// ([slot][blockDim], conflict-free), and the nz cross-section rows of the segment's region are
// loaded once per segment into a shared-memory row cache (3 values per plane, no padding: 7
// blocks of 64 threads fit an SM at 8 planes and 3 polar angles in FP32). Every value computed
// equals the plane-by-plane order's (the same inflows, the same radial states); only the order of
// the tally atomics differs.
constexpr int kDgResBlock = 64;  // threads per block of the plane-inner sweep

// Axial coarse-mesh acceleration (coarse cells = planes), tallied by the plane-inner sweep:
// partial currents between planes and the net current out of each plane through the domain
// boundary (radial track ends, bottom and top faces: out minus in), FP64 as in the planar CMFD.
template <typename Real> struct DgCm {
  const Real *mu;   // [P] polar cosines
  const Real *dz;   // [nz] plane heights
  double *cur;      // [2][nz][Gp]: [0][z] plane z -> z+1, [1][z] plane z+1 -> z
  double *leak;     // [nz][Gp]
};

template <typename Real, int P, bool CM>
__global__ void __launch_bounds__(kDgResBlock) dg_sweep_res_kernel(
    const TrackRec *__restrict__ trk, const SegRec<Real> *__restrict__ seg, const int32_t *__restrict__ link,
    const Real *__restrict__ wdg, const Real *__restrict__ sin_t, const Real *__restrict__ inv_sin,
    const Real *__restrict__ cz, const DgXs<Real> *__restrict__ xs3, Real *__restrict__ tally,
    const Real *__restrict__ psi_in, Real *__restrict__ psi_out, Real *__restrict__ face,
    const double *__restrict__ scal, long long n_threads, int G, int Gp, int R, int nz, int bc_bottom, int bc_top,
    DgCm<Real> cm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int B = kDgResBlock;  // launched with exactly this many threads
  const int tid = threadIdx.x;
  Real *ys = reinterpret_cast<Real *>(smem_raw);  // [2][nz][P][2][B]
  Real *rc = ys + (size_t)4 * nz * P * B;         // [3][nz][B]: Sigma_t, q0, q1 of the segment's region
  Real *ca = rc + (size_t)3 * nz * B;             // CM: [3][nz][B] current up, current down, boundary
  const long long idx = (long long)blockIdx.x * B + tid;
  if (idx >= n_threads) return;
  const long long td = idx / G;
  const int g = (int)(idx - td * G);
  const TrackRec tr = trk[td >> 1];
  const int d = (int)(td & 1);
  const Real scale = (Real)scal[S_SCALE];
  Real w[P], st[P], is[P];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    w[p] = wdg[tr.dir * P + p];
    st[p] = sin_t[p];
    is[p] = inv_sin[p];
  }
  const int nslot = 4 * nz * P;
  {
    const Real *pi = psi_in + td * nslot * G + g;  // [2T][2][nz][P][2][G]: slots of one end in order
    for (int k = 0; k < nslot; ++k) ys[(size_t)k * B + tid] = pi[(size_t)k * G] * scale;
  }
  Real mu[P];
  if (CM) {
#pragma unroll
    for (int p = 0; p < P; ++p) mu[p] = cm.mu[p];
    for (int k = 0; k < 3 * nz; ++k) ca[(size_t)k * B + tid] = 0;
    // radial current in at the track's start, every plane and march
    for (int ud = 0; ud < 2; ++ud)
      for (int z = 0; z < nz; ++z) {
        Real j = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) j = fma(w[p] * st[p], ys[((size_t)((ud * nz + z) * P + p) * 2) * B + tid], j);
        ca[(size_t)(2 * nz + z) * B + tid] -= j * cm.dz[z];
      }
  }
  const int step = d ? -1 : 1;
  const SegRec<Real> *sp = seg + (d ? tr.off + tr.n - 1 : tr.off);
  // the top traces (reflective top only; the buffer is not allocated otherwise)
  Real *fp = bc_top ? face + (((d ? tr.off + tr.n - 1 : tr.off) * 2 + d) * P) * G + g : nullptr;
  const long long fstep = (long long)step * 2 * P * G;
  SegRec<Real> s = sp[0];
  for (int n = 0; n < tr.n; ++n) {
    const SegRec<Real> s_next = sp[step];  // padding records at both ends of the array
    for (int z = 0; z < nz; ++z) {
      const DgXs<Real> x = xs3[((size_t)z * R + s.r) * Gp + g];
      rc[(size_t)z * B + tid] = x.t;
      rc[(size_t)(nz + z) * B + tid] = x.q0;
      rc[(size_t)(2 * nz + z) * B + tid] = x.q1;
    }
    const Real il = DgMath<Real>::rcp(s.l);
    Real fin[P];
    if (bc_top) {
#pragma unroll
      for (int p = 0; p < P; ++p) fin[p] = fp[p * G] * scale;
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) fin[p] = 0;
    }
    for (int ud = 0; ud < 2; ++ud) {
      const Real sg = ud ? (Real)1 : (Real)-1;
      if (ud == 1 && !bc_bottom) {
#pragma unroll
        for (int p = 0; p < P; ++p) fin[p] = 0;
      }
      if (CM) {
        // current entering the march's first plane through the top or bottom face
        Real j = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) j = fma(w[p] * mu[p], fin[p], j);
        ca[(size_t)(2 * nz + (ud ? 0 : nz - 1)) * B + tid] -= j * s.l;
      }
      for (int zi = 0; zi < nz; ++zi) {
        const int z = ud ? zi : nz - 1 - zi;
        const Real xt = rc[(size_t)z * B + tid], xq0 = rc[(size_t)(nz + z) * B + tid];
        const Real q1s = sg * rc[(size_t)(2 * nz + z) * B + tid];
        Real *yz = ys + ((size_t)((ud * nz + z) * P) * 2) * B + tid;
        Real a0 = 0, a1 = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
          Real y0 = yz[(2 * p) * B], y1 = yz[(2 * p + 1) * B];
          Real i0, i1;
          dg_update<Real>(xt, xq0, q1s, cz[z * P + p], s.l, s.l * is[p], st[p], fin[p], y0, y1, i0, i1);
          yz[(2 * p) * B] = y0;
          yz[(2 * p + 1) * B] = y1;
          a0 = fma(w[p], i0, a0);
          a1 = fma(w[p], i1, a1);
          fin[p] = (i0 + i1) * il;
        }
        dg_tally<Real>(tally + (((size_t)z * R + s.r) * Gp + g) * 2, a0, sg * a1);
        if (CM) {
          // the plane's outflow through its downwind face: into the next plane or out of the domain
          Real j = 0;
#pragma unroll
          for (int p = 0; p < P; ++p) j = fma(w[p] * mu[p], fin[p], j);
          const int slot = ud ? (z < nz - 1 ? z : 2 * nz + z) : (z > 0 ? nz + z - 1 : 2 * nz);
          ca[(size_t)slot * B + tid] += j * s.l;
        }
      }
    }
    if (bc_top) {
#pragma unroll
      for (int p = 0; p < P; ++p) fp[p * G] = fin[p];
    }
    s = s_next;
    sp += step;
    if (bc_top) fp += fstep;
  }
  const int e_out = link[td];
  if (e_out >= 0) {
    Real *po = psi_out + (long long)e_out * nslot * G + g;
    for (int k = 0; k < nslot; ++k) po[(size_t)k * G] = ys[(size_t)k * B + tid];
  }
  if (CM) {
    // radial current out at the track's end, then this thread's sums into the FP64 totals
    for (int ud = 0; ud < 2; ++ud)
      for (int z = 0; z < nz; ++z) {
        Real j = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) j = fma(w[p] * st[p], ys[((size_t)((ud * nz + z) * P + p) * 2) * B + tid], j);
        ca[(size_t)(2 * nz + z) * B + tid] += j * cm.dz[z];
      }
    for (int z = 0; z < nz; ++z) {
      if (z < nz - 1) {
        atomicAdd(cm.cur + (size_t)z * Gp + g, (double)ca[(size_t)z * B + tid]);
        atomicAdd(cm.cur + (size_t)(nz + z) * Gp + g, (double)ca[(size_t)(nz + z) * B + tid]);
      }
      atomicAdd(cm.leak + (size_t)z * Gp + g, (double)ca[(size_t)(2 * nz + z) * B + tid]);
    }
  }
}

// ----------------------------------------------------------------------------- axial CMFD
// flux sums per (plane, material, group): psum[(z M + m) G + g] += A dz phi_0 (the planar CMFD's
// homogenisation input with the planes as cells)
template <typename Real>
__global__ void dg_cm_sums_kernel(int E, int R, int G, int Gp, int M, const int32_t *__restrict__ mat3,
                                  const double *__restrict__ area, const Real *__restrict__ dz,
                                  const Real *__restrict__ phi3, double *__restrict__ psum) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)E * G) return;
  const int e = (int)(idx / G), g = (int)(idx - (long long)e * G);
  const int z = e / R, r = e - z * R;
  atomicAdd(psum + ((size_t)z * M + mat3[e]) * G + g,
            area[r] * (double)dz[z] * (double)phi3[((size_t)e * Gp + g) * 2]);
}

// One block: the coarse eigenproblem on the planes (the arrays from cmfd_coeff_kernel, group-major
// [g][z]; SV [g_to][h_from][z]), a fixed number of power iterations, each Gauss-Seidel in energy
// with n_inner over-relaxed sweeps over the even planes then the odd ones; then the coarse/fine
// ratio per (group, plane), the coarse k, and the current tallies cleared for the next sweep.
template <typename Real>
__global__ void __launch_bounds__(256) dg_cm_solve_kernel(int nz, int G, int Gp, double *__restrict__ cur,
                                                          double *__restrict__ leak, const Real *__restrict__ cphi,
                                                          const Real *__restrict__ TV, const Real *__restrict__ SV,
                                                          const Real *__restrict__ FV, const Real *__restrict__ CHI,
                                                          double *__restrict__ diag, double *__restrict__ phic,
                                                          double *__restrict__ fis, Real *__restrict__ ratio,
                                                          double *__restrict__ scal, int n_outer, int n_inner,
                                                          double omega) {
  __shared__ double s_k, s_fold;
  const int N = nz;
  for (int x = threadIdx.x; x < N * G; x += blockDim.x) {
    const int g = x / N, z = x - g * N;
    const double pz = (double)cphi[x];
    double dg = (double)TV[x] - (double)SV[((size_t)g * G + g) * N + z];
    if (pz > 0.0) {
      dg += leak[(size_t)z * Gp + g] / pz;
      if (z < nz - 1) dg += cur[(size_t)z * Gp + g] / pz;
      if (z > 0) dg += cur[(size_t)(nz + z - 1) * Gp + g] / pz;
    }
    diag[x] = dg;
    phic[x] = pz;
  }
  if (threadIdx.x == 0) s_k = scal[S_K];
  __syncthreads();
  for (int it = 0; it < n_outer; ++it) {
    for (int z = threadIdx.x; z < N; z += blockDim.x) {
      double f = 0.0;
      for (int g = 0; g < G; ++g) f += (double)FV[(size_t)g * N + z] * phic[(size_t)g * N + z];
      fis[z] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double F = 0.0;
      for (int z = 0; z < N; ++z) F += fis[z];
      s_fold = F;
    }
    __syncthreads();
    const double kc = s_k;
    for (int g = 0; g < G; ++g)
      for (int j = 0; j < n_inner; ++j)
        for (int c = 0; c < 2; ++c) {
          for (int z = c + 2 * threadIdx.x; z < N; z += 2 * blockDim.x) {
            const size_t x = (size_t)g * N + z;
            double rhs = (double)CHI[x] * fis[z] / kc;
            for (int h = 0; h < G; ++h)
              if (h != g) rhs += (double)SV[((size_t)g * G + h) * N + z] * phic[(size_t)h * N + z];
            if (z > 0 && cphi[x - 1] > (Real)0) rhs += cur[(size_t)(z - 1) * Gp + g] / (double)cphi[x - 1] * phic[x - 1];
            if (z < nz - 1 && cphi[x + 1] > (Real)0)
              rhs += cur[(size_t)(nz + z) * Gp + g] / (double)cphi[x + 1] * phic[x + 1];
            if (diag[x] > 0.0) phic[x] += omega * (rhs / diag[x] - phic[x]);
          }
          __syncthreads();
        }
    if (threadIdx.x == 0) {
      double F = 0.0;
      for (int z = 0; z < N; ++z)
        for (int g = 0; g < G; ++g) F += (double)FV[(size_t)g * N + z] * phic[(size_t)g * N + z];
      if (F > 0.0 && s_fold > 0.0) s_k = s_k * F / s_fold;
    }
    __syncthreads();
  }
  for (int x = threadIdx.x; x < N * G; x += blockDim.x) {
    const double pz = (double)cphi[x];
    ratio[x] = (Real)((pz > 0.0 && phic[x] > 0.0) ? phic[x] / pz : 1.0);
  }
  for (int x = threadIdx.x; x < 2 * nz * Gp; x += blockDim.x) cur[x] = 0.0;
  for (int x = threadIdx.x; x < nz * Gp; x += blockDim.x) leak[x] = 0.0;
  if (threadIdx.x == 0) scal[S_K] = s_k;
}

// both moments of every element *= the ratio of its plane; FP64 fission partials; the last block
// sets the pending normalisation 1/F (as the planar prolongation does)
template <typename Real>
__global__ void __launch_bounds__(256) dg_cm_prolong_kernel(int E, int R, int G, int Gp, int nz,
                                                            const int32_t *__restrict__ mat3,
                                                            const Real *__restrict__ nsf,
                                                            const double *__restrict__ area,
                                                            const Real *__restrict__ dz, const Real *__restrict__ ratio,
                                                            Real *__restrict__ phi3, double *__restrict__ part,
                                                            unsigned *__restrict__ ticket, double *__restrict__ scal) {
  __shared__ double red[256];
  __shared__ bool last;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double fa = 0.0;
  if (e < E) {
    const int z = e / R, r = e - z * R, m = mat3[e];
    Real f = 0;
    for (int g = 0; g < G; ++g) {
      const Real q = ratio[(size_t)g * nz + z];
      Real *ph = phi3 + ((size_t)e * Gp + g) * 2;
      const Real v = ph[0] * q;
      ph[0] = v;
      ph[1] *= q;
      f += nsf[m * G + g] * v;
    }
    fa = area[r] * (double)dz[z] * (double)f;
  }
  red[threadIdx.x] = fa;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = red[0];
    __threadfence();
    last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    double a = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) a += part[b];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double F = red[0];
      if (F > 0.0 && isfinite(F)) {
        scal[S_SCALE] = 1.0 / F;
        scal[S_FISS] = F;
      } else {
        scal[S_STATUS] = 1.0;
      }
      *ticket = 0u;
    }
  }
}

// the radial boundary moments of the next sweep ([2T][2][nz][P][2][G]) and the stored top traces
// ([S + pad][2][P][G], top plane) *= the ratio of their plane
template <typename Real>
__global__ void dg_cm_psi_kernel(long long n_psi, long long n_face, int P, int G, int nz,
                                 const Real *__restrict__ ratio, Real *__restrict__ psi, Real *__restrict__ face) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n_psi) {
    const int g = (int)(x % G);
    const int z = (int)((x / ((long long)G * 2 * P)) % nz);
    psi[x] *= ratio[(size_t)g * nz + z];
  } else if (x < n_psi + n_face) {
    const long long y = x - n_psi;
    face[y] *= ratio[(size_t)(y % G) * nz + nz - 1];
  }
}

// Flux moments of every element from the tallies (phi_m = tally_m / A; the source's
// infinite-medium value 4 pi q_m / Sigma_t where the tracked area is 0), tallies cleared, FP64
// block partials for the planar reduce: sum of dz A f, min and max of fold / f, and the
// fixed-source residual over the plane-average moments.
template <typename Real>
__global__ void __launch_bounds__(256) dg_finalize_kernel(
    int E, int R, int G, int Gp, const int32_t *__restrict__ mat3, const Real *__restrict__ nsf,
    const double *__restrict__ area, const double *__restrict__ dz, const DgXs<Real> *__restrict__ xs3,
    Real *__restrict__ tally, Real *__restrict__ phi3, const double *__restrict__ fold, double *__restrict__ part,
    int eigen) {
  __shared__ double s_sum[256], s_min[256], s_max[256], s_res[256];
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double fsum = 0.0, rmin = INFINITY, rmax = -INFINITY, res = 0.0;
  if (e < E) {
    const int r = e % R, z = e / R;
    const int m = mat3[e];
    const double A = area[r];
    double f = 0.0;
    for (int g = 0; g < G; ++g) {
      const size_t a = ((size_t)e * Gp + g) * 2;
      double v0, v1;
      if (A > 0.0) {
        v0 = (double)tally[a] / A;
        v1 = (double)tally[a + 1] / A;
      } else {
        const DgXs<Real> x = xs3[(size_t)e * Gp + g];
        v0 = kFourPi * (double)x.q0 / (double)x.t;
        v1 = kFourPi * (double)x.q1 / (double)x.t;
      }
      tally[a] = (Real)0;
      tally[a + 1] = (Real)0;
      if (!eigen) {
        const double old = (double)phi3[a];
        if (v0 > 0.0) res = fmax(res, fabs(v0 - old) / v0);
      }
      phi3[a] = (Real)v0;
      phi3[a + 1] = (Real)v1;
      f += (double)nsf[m * G + g] * (double)(Real)v0;
    }
    fsum = dz[z] * A * f;
    if (eigen && f > 0.0) {
      const double rho = fold[e] / f;
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

// state in/out of the flux moments: phi [E][2][G] FP64 (NULL: phi_0 = 1, phi_1 = 0) <-> phi3
// [E][Gp][2] in the sweep's type, scaled by `scale` on the way out
template <typename Real>
__global__ void dg_phi_in_kernel(long long n, int G, int Gp, const double *__restrict__ phi, Real *__restrict__ phi3) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;  // n = E * Gp * 2
  const int m = (int)(x & 1);
  const long long eg = x >> 1;
  const long long e = eg / Gp;
  const int g = (int)(eg - e * Gp);
  Real v = 0;
  if (g < G) v = phi ? (Real)phi[(e * 2 + m) * G + g] : (Real)(m == 0 ? 1 : 0);
  phi3[x] = v;
}

template <typename Real>
__global__ void dg_phi_out_kernel(long long n, int G, int Gp, const Real *__restrict__ phi3, double scale,
                                  double *__restrict__ phi) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;  // n = E * 2 * G
  const long long e = x / (2 * G);
  const int rem = (int)(x - e * 2 * G);
  const int m = rem / G, g = rem - m * G;
  phi[x] = (double)phi3[(e * Gp + g) * 2 + m] * scale;
}

}  // namespace moc
