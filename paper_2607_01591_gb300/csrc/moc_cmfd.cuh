// Coarse-mesh finite difference (CMFD) acceleration of the power iteration: the paper's Alg. 1
// solves CMFD on a coarse mesh with the MOC surface currents and updates the fine MOC solution with
// the accelerated result. Here, in partial-current form:
//   - coarse cells are any partition of the triangles (given per region);
//   - the sweep tallies, per coarse interface and direction, the partial current W * psi of every
//     track crossing between cells, and at vacuum ends the outgoing current (reflective walls carry
//     no net current at convergence and are not tallied);
//   - coarse balance per cell i and group g, with flux-volume homogenised cross sections:
//       (Sigma_t V - Sigma_s,gg V + sum_out D_out + D_vac) phi_i - sum_in D_in phi_j
//         = sum_{g' != g} Sigma_s,g'g V phi_i,g' + chi_i,g / k sum_g' nuSigma_f V phi_i,g'
//     where D(a->b) = J(a->b) / phi_a reproduces the MOC currents at the current iterate, so the
//     converged MOC solution is a fixed point of the acceleration;
//   - the coarse eigenproblem is iterated a fixed number of times (power iteration, Gauss-Seidel
//     in energy, Jacobi in space), and the fine flux and boundary flux are scaled by the coarse
//     flux ratio of their cell.
#pragma once
#include "moc_kernels.cuh"

namespace moc {

template <typename Real> struct CmfdDev {
  const int32_t *xing;  // [S + pads] code of the boundary after each segment (forward order), -1 none
  const int32_t *cell;  // [R] coarse cell of each region
  Real *cur;            // [2 n_if][Gp] partial currents per interface and direction
  Real *leak;           // [N][Gp] outgoing current at vacuum ends
};

// Sweep with the CMFD current tallies (one thread per track end and group, as sweep_kernel).
template <typename Real, int P, int TM>
__global__ void __launch_bounds__(128) sweep_cmfd_kernel(
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
  const long long first = d ? tr.off + tr.n - 1 : tr.off;
  Tally<TM, Real> tally;
  tally.init((unsigned)(seg[first].r * Gp + g));
  int r_last = seg[first].r;
  for (int n = 0; n < tr.n; ++n) {
    const long long s = first + (long long)n * step;
    const SegRec<Real> sg = seg[s];
    const typename Pair<Real>::T xq = xsq[(size_t)sg.r * Gp + g];
    const Real tau0 = xq.x * sg.l;
    Real acc = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const Real F = one_minus_exp(tau0 * is[p]);
      const Real dl = (psi[p] - xq.y) * F;
      psi[p] -= dl;
      acc = fma(w[p], dl, acc);
    }
    tally.add(tsum, tcomp, (unsigned)(sg.r * Gp + g), acc);
    r_last = sg.r;
    if (n + 1 < tr.n) {
      // boundary between this segment and the next in travel order: forward uses the code stored
      // at this segment, backward the one stored at the previous segment, with the direction bit
      // flipped
      const int code = cm.xing[d ? s - 1 : s];
      if (code >= 0) {
        Real j = 0;
#pragma unroll
        for (int p = 0; p < P; ++p) j = fma(w[p], psi[p], j);
        atomicAdd(cm.cur + (size_t)(code ^ d) * Gp + g, j);
      }
    }
  }
  tally.flush(tcomp);
  const int e = link[td];
  if (e >= 0) {
#pragma unroll
    for (int p = 0; p < P; ++p) psi_out[((long long)e * P + p) * G + g] = psi[p];
  } else {
    Real j = 0;
#pragma unroll
    for (int p = 0; p < P; ++p) j = fma(w[p], psi[p], j);
    atomicAdd(cm.leak + (size_t)cm.cell[r_last] * Gp + g, j);
  }
}

// Flux-volume homogenisation in two steps. (1) One thread per region and group adds A phi into
// the (cell, material, group) flux sum. (2) One thread per cell and group builds the cell's
// coefficients from those sums and the material tables -- exact because the cross sections are
// constant per material:
//   cphi = sum A phi / V; TV = sum_m Sigma_t,m PHI_m / cphi; SV[g'][g] = sum_m Sigma_s,m,g'g
//   PHI_m,g' / cphi_g'; FV = sum_m nuSigma_f,m PHI_m / cphi; CHI = fission-weighted chi.
template <typename Real>
__global__ void cmfd_flux_sums_kernel(int R, int G, int Gp, int M, const int32_t *__restrict__ cell,
                                      const int32_t *__restrict__ mat, const double *__restrict__ area,
                                      const Real *__restrict__ phi, double *__restrict__ psum) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)R * G) return;
  const int r = (int)(idx / G), g = (int)(idx - (long long)r * G);
  atomicAdd(psum + ((size_t)cell[r] * M + mat[r]) * G + g, area[r] * (double)phi[(size_t)r * Gp + g]);
}

template <typename Real>
__global__ void cmfd_coeff_kernel(int N, int G, int M, const double *__restrict__ psum, const double *__restrict__ vol,
                                  const Real *__restrict__ sig_t, const Real *__restrict__ nsf,
                                  const Real *__restrict__ chi, const Real *__restrict__ sig_s,
                                  Real *__restrict__ cphi, Real *__restrict__ TV, Real *__restrict__ SV,
                                  Real *__restrict__ FV, Real *__restrict__ CHI) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N * G) return;
  const int i = x / G, g = x - i * G;
  const double *P = psum + (size_t)i * M * G;
  double raw = 0.0, tv = 0.0, fv = 0.0, ch = 0.0, chs = 0.0;
  for (int m = 0; m < M; ++m) {
    const double pm = P[(size_t)m * G + g];
    raw += pm;
    tv += (double)sig_t[m * G + g] * pm;
    fv += (double)nsf[m * G + g] * pm;
    double fm = 0.0;  // fission production of material m in the cell
    for (int h = 0; h < G; ++h) fm += (double)nsf[m * G + h] * P[(size_t)m * G + h];
    ch += (double)chi[m * G + g] * fm;
    double cs = 0.0;
    for (int h = 0; h < G; ++h) cs += (double)chi[m * G + h];
    chs += cs * fm;
  }
  const double V = vol[i];
  Real *sv = SV + ((size_t)i * G + g) * G;
  if (raw > 0.0) {
    TV[x] = (Real)(tv * V / raw);
    FV[x] = (Real)(fv * V / raw);
    for (int h = 0; h < G; ++h) {
      double s = 0.0;
      for (int m = 0; m < M; ++m) s += (double)sig_s[((size_t)m * G + g) * G + h] * P[(size_t)m * G + g];
      sv[h] = (Real)(s * V / raw);
    }
  } else {
    TV[x] = FV[x] = (Real)0;
    for (int h = 0; h < G; ++h) sv[h] = (Real)0;
  }
  cphi[x] = (V > 0.0) ? (Real)(raw / V) : (Real)0;
  CHI[x] = (chs > 0.0) ? (Real)(ch / chs) : (Real)0;
}

struct CmfdTopo {
  int N, G, Gp, n_entries;
  const int32_t *nbr;       // [n_entries] the neighbouring cell of each entry
  const int32_t *cif_off;   // [N+1] entries of each cell
  const int32_t *cif;       // [n_entries] (interface << 1) | side (side 0: the cell is the interface's lower id)
  const int32_t *if_cells;  // [2 n_if] the two cells of each interface
};

// The whole coarse solve in one block (fixed iteration counts, deterministic order); writes the
// flux ratio per cell and group and the accelerated k. Scratch arrays are owned by the context.
template <typename Real, bool SMEM>
__global__ void __launch_bounds__(1024) cmfd_solve_kernel(CmfdTopo t, Real *__restrict__ cur, Real *__restrict__ leak,
                                                          const Real *__restrict__ cphi, const Real *__restrict__ TV,
                                                          const Real *__restrict__ SV, const Real *__restrict__ FV,
                                                          const Real *__restrict__ CHI, Real *__restrict__ din,
                                                          Real *__restrict__ diag, Real *__restrict__ phic,
                                                          Real *__restrict__ phin, Real *__restrict__ phio,
                                                          Real *__restrict__ src, Real *__restrict__ fis,
                                                          Real *__restrict__ ratio, double *__restrict__ scal,
                                                          int n_outer, int n_inner) {
  __shared__ double red[1024];
  const int N = t.N, G = t.G, Gp = t.Gp;
  // per-group working set: in shared memory (SMEM) or in the context's global scratch
  extern __shared__ unsigned char dyn[];
  Real *s_src, *s_diag, *s_a, *s_b, *s_din;
  const int32_t *s_off, *s_nbr;
  if (SMEM) {
    Real *base = reinterpret_cast<Real *>(dyn);
    s_src = base;
    s_diag = s_src + N;
    s_a = s_diag + N;
    s_b = s_a + N;
    s_din = s_b + N;
    int32_t *ib = reinterpret_cast<int32_t *>(s_din + t.n_entries);
    int32_t *w_off = ib, *w_nbr = ib + (N + 1);
    for (int i = threadIdx.x; i <= N; i += blockDim.x) w_off[i] = t.cif_off[i];
    for (int q = threadIdx.x; q < t.n_entries; q += blockDim.x) w_nbr[q] = t.nbr[q];
    s_off = w_off;
    s_nbr = w_nbr;
  } else {
    s_src = src;
    s_diag = phio + N;  // the global scratch holds N values each (see the host allocation)
    s_a = phin;
    s_b = phio;
    s_din = din + (size_t)t.n_entries * G;
    s_off = t.cif_off;
    s_nbr = t.nbr;
  }
  __syncthreads();
  // 1. coefficients from the tallied currents, then clear the tallies for the next sweep
  for (int x = threadIdx.x; x < N * G; x += blockDim.x) {
    const int i = x / G, g = x - i * G;
    const Real pi = cphi[(size_t)i * G + g];
    Real dg = TV[(size_t)i * G + g] - SV[((size_t)i * G + g) * G + g];
    if (pi > (Real)0) dg += leak[(size_t)i * Gp + g] / pi;
    for (int q = t.cif_off[i]; q < t.cif_off[i + 1]; ++q) {
      const int e = t.cif[q] >> 1, side = t.cif[q] & 1;
      const int j = t.if_cells[2 * e + (side ^ 1)];
      const Real pj = cphi[(size_t)j * G + g];
      if (pi > (Real)0) dg += cur[(size_t)(2 * e + side) * Gp + g] / pi;
      din[(size_t)q * G + g] = (pj > (Real)0) ? cur[(size_t)(2 * e + (side ^ 1)) * Gp + g] / pj : (Real)0;
    }
    diag[(size_t)i * G + g] = dg;
    phic[(size_t)i * G + g] = pi;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < t.n_entries * Gp; x += blockDim.x) cur[x] = (Real)0;
  for (int x = threadIdx.x; x < N * Gp; x += blockDim.x) leak[x] = (Real)0;
  double kc = scal[S_K];
  // 2. coarse power iteration
  for (int it = 0; it < n_outer; ++it) {
    double fsum = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      Real f = 0;
      for (int g = 0; g < G; ++g) f += FV[(size_t)i * G + g] * phic[(size_t)i * G + g];
      fis[i] = f;
      fsum += (double)f;
    }
    red[threadIdx.x] = fsum;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
      __syncthreads();
    }
    const double F_old = red[0];
    __syncthreads();
    const Real inv_k = (Real)(1.0 / kc);
    for (int g = 0; g < G; ++g) {
      // the group's fixed source (other groups' scattering and fission) and its coefficients,
      // staged in shared memory when they fit, so the sweeps run on-chip
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        Real rhs = CHI[(size_t)i * G + g] * fis[i] * inv_k;
        for (int h = 0; h < G; ++h)
          if (h != g) rhs += SV[((size_t)i * G + h) * G + g] * phic[(size_t)i * G + h];
        s_src[i] = rhs;
        s_diag[i] = diag[(size_t)i * G + g];
        s_a[i] = phic[(size_t)i * G + g];
      }
      for (int q = threadIdx.x; q < t.n_entries; q += blockDim.x) s_din[q] = din[(size_t)q * G + g];
      __syncthreads();
      // Jacobi sweeps alternating between two vectors (one barrier per sweep)
      for (int j = 0; j < n_inner; ++j) {
        const Real *from = (j & 1) ? s_b : s_a;
        Real *to = (j & 1) ? s_a : s_b;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
          Real rhs = s_src[i];
          for (int q = s_off[i]; q < s_off[i + 1]; ++q) rhs += s_din[q] * from[s_nbr[q]];
          const Real dg = s_diag[i];
          to[i] = (dg > (Real)0) ? rhs / dg : (Real)0;
        }
        __syncthreads();
      }
      const Real *res = (n_inner & 1) ? s_b : s_a;
      for (int i = threadIdx.x; i < N; i += blockDim.x) phic[(size_t)i * G + g] = res[i];
      __syncthreads();
    }
    fsum = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      Real f = 0;
      for (int g = 0; g < G; ++g) f += FV[(size_t)i * G + g] * phic[(size_t)i * G + g];
      fsum += (double)f;
    }
    red[threadIdx.x] = fsum;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
      __syncthreads();
    }
    if (red[0] > 0.0 && F_old > 0.0) kc = kc * red[0] / F_old;
    __syncthreads();
  }
  // 3. prolongation ratios and the accelerated k
  for (int x = threadIdx.x; x < N * G; x += blockDim.x) {
    const Real a = cphi[x], b = phic[x];
    ratio[x] = (a > (Real)0 && b > (Real)0) ? b / a : (Real)1;
  }
  if (threadIdx.x == 0) {
    if (isfinite(kc) && kc > 0.0) scal[S_K] = kc;
    else scal[S_STATUS] = 1.0;
  }
}

// phi *= ratio(cell); block partials of sum A f(phi); the last block sets the normalisation.
template <typename Real>
__global__ void __launch_bounds__(256) cmfd_prolong_kernel(int R, int G, int Gp, const int32_t *__restrict__ cell,
                                                           const int32_t *__restrict__ mat,
                                                           const Real *__restrict__ nsf,
                                                           const double *__restrict__ area,
                                                           const Real *__restrict__ ratio, Real *__restrict__ phi,
                                                           double *__restrict__ part, unsigned *__restrict__ ticket,
                                                           double *__restrict__ scal) {
  __shared__ double red[256];
  __shared__ bool last;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  double fa = 0.0;
  if (r < R) {
    const int c = cell[r], m = mat[r];
    Real f = 0;
    for (int g = 0; g < G; ++g) {
      const Real v = phi[(size_t)r * Gp + g] * ratio[(size_t)c * G + g];
      phi[(size_t)r * Gp + g] = v;
      f += nsf[m * G + g] * v;
    }
    fa = area[r] * (double)f;
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

// boundary flux of each linked incoming end *= ratio of the cell of the region at that end
template <typename Real>
__global__ void cmfd_psi_kernel(long long n, int P, int G, const TrackRec *__restrict__ trk,
                                const SegRec<Real> *__restrict__ seg, const uint8_t *__restrict__ fed,
                                const int32_t *__restrict__ cell, const Real *__restrict__ ratio,
                                Real *__restrict__ psi) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const long long td = idx / G;
  const int g = (int)(idx - td * G);
  if (!fed[td]) return;
  const TrackRec tr = trk[td >> 1];
  const int d = (int)(td & 1);
  const int r = seg[d ? tr.off + tr.n - 1 : tr.off].r;
  const Real f = ratio[(size_t)cell[r] * G + g];
  for (int p = 0; p < P; ++p) psi[(td * P + p) * G + g] *= f;
}

}  // namespace moc
