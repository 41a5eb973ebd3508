// Coarse-mesh finite difference (CMFD) acceleration of the power iteration: the paper's Alg. 1
// solves CMFD on a coarse mesh with the MOC surface currents and updates the fine MOC solution with
// the accelerated result. Here, in partial-current form:
//   - coarse cells are any partition of the triangles (given per region);
//   - the sweep tallies, per coarse interface and direction, the partial current W * psi of every
//     track crossing between cells, and per cell the net current through the domain boundary
//     (out at every track end, vacuum or reflective, minus in at every track start): reflective
//     walls carry no net current only at convergence, so the coarse balance matches the sweep's
//     own balance at every iterate;
//   - coarse balance per cell i and group g, with flux-volume homogenised cross sections:
//       (Sigma_t V - Sigma_s,gg V + sum_out D_out + D_bnd) phi_i - sum_in D_in phi_j
//         = sum_{g' != g} Sigma_s,g'g V phi_i,g' + chi_i,g / k sum_g' nuSigma_f V phi_i,g'
//     where D(a->b) = J(a->b) / phi_a reproduces the MOC currents at the current iterate, so the
//     converged MOC solution is a fixed point of the acceleration;
//   - the coarse eigenproblem is iterated a fixed number of times (power iteration, Gauss-Seidel
//     in energy, over-relaxed Gauss-Seidel sweeps in space over a colouring of the cells), and the
//     fine flux and boundary flux are scaled by the coarse flux ratio of their cell.
#pragma once
#include <cooperative_groups.h>

#include "moc_kernels.cuh"

namespace moc {

// Coarse arrays are group-major ([g][i] over the N cells) so that every per-group pass of the
// coarse solve reads them with coalesced loads; SV is [g_to][h_from][i].

// Flux-volume homogenisation in two steps. (1) One thread per region and group adds A phi into
// the (cell, material, group) flux sum. (2) One thread per cell and group builds the cell's
// coefficients from those sums and the material tables -- exact because the cross sections are
// constant per material:
//   cphi = sum A phi / V; TV = sum_m Sigma_t,m PHI_m / cphi; SV[h->g] = sum_m Sigma_s,m,hg
//   PHI_m,h / cphi_h; FV = sum_m nuSigma_f,m PHI_m / cphi; CHI = fission-weighted chi.
template <typename Real>
__global__ void cmfd_flux_sums_kernel(int R, int G, int Gp, int M, const int32_t *__restrict__ cell,
                                      const int32_t *__restrict__ mat, const double *__restrict__ area,
                                      const Real *__restrict__ phi, double *__restrict__ psum) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)R * G) return;
  const int r = (int)(idx / G), g = (int)(idx - (long long)r * G);
  atomicAdd(psum + ((size_t)cell[r] * M + mat[r]) * G + g, area[r] * (double)phi[(size_t)r * Gp + g]);
}

// thread x = g * N + i: cell i, source group g (the row of SV leaving g)
template <typename Real>
__global__ void cmfd_coeff_kernel(int N, int G, int M, const double *__restrict__ psum, const double *__restrict__ vol,
                                  const Real *__restrict__ sig_t, const Real *__restrict__ nsf,
                                  const Real *__restrict__ chi, const Real *__restrict__ sig_s,
                                  Real *__restrict__ cphi, Real *__restrict__ TV, Real *__restrict__ SV,
                                  Real *__restrict__ FV, Real *__restrict__ CHI) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N * G) return;
  const int g = x / N, i = x - g * N;
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
  if (raw > 0.0) {
    TV[x] = (Real)(tv * V / raw);
    FV[x] = (Real)(fv * V / raw);
    for (int h = 0; h < G; ++h) {
      double s = 0.0;
      for (int m = 0; m < M; ++m) s += (double)sig_s[((size_t)m * G + g) * G + h] * P[(size_t)m * G + g];
      SV[((size_t)h * G + g) * N + i] = (Real)(s * V / raw);
    }
  } else {
    TV[x] = FV[x] = (Real)0;
    for (int h = 0; h < G; ++h) SV[((size_t)h * G + g) * N + i] = (Real)0;
  }
  cphi[x] = (V > 0.0) ? (Real)(raw / V) : (Real)0;
  CHI[x] = (chs > 0.0) ? (Real)(ch / chs) : (Real)0;
}

struct CmfdTopo {
  int N, G, Gp, n_entries, n_colors;
  const int32_t *nbr;       // [n_entries] the neighbouring cell of each entry
  const int32_t *cif_off;   // [N+1] entries of each cell
  const int32_t *cif;       // [n_entries] (interface << 1) | side (side 0: the cell is the interface's lower id)
  const int32_t *if_cells;  // [2 n_if] the two cells of each interface
  const int32_t *coff;      // [n_colors+1] cells are numbered colour by colour: colour c is
                            // [coff[c], coff[c+1]); no interface joins two cells of one colour
};

// Sum of v over the block (1024 threads): warp shuffles, one partial per warp, two barriers.
__device__ __forceinline__ double block_sum_1024(double v, double *red32) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red32[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < 32; ++w) s += red32[w];  // every thread, same order: same result everywhere
  __syncthreads();
  return s;
}

// Maximum of v over the block (1024 threads), the same in every thread.
__device__ __forceinline__ double block_max_1024(double v, double *red32) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red32[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < 32; ++w) s = fmax(s, red32[w]);
  __syncthreads();
  return s;
}

// The whole coarse solve in one block of 1024 threads (fixed iteration counts, deterministic
// order); writes the flux ratio per cell and group and the accelerated k. Scratch arrays are owned
// by the context. SMEM: the per-group working set (source, 1/diagonal, iterate, coefficients,
// offsets and neighbour ids of type Idx) lives in dynamic shared memory; otherwise in the global
// scratch.
// Per-cell sums over the groups, in group order (the same additions as a plain loop), read in
// batches of 8 predicated loads so that a thread waits for one round trip per batch instead of
// one per group.
template <typename Real>
__device__ __forceinline__ Real cell_fission(const Real *__restrict__ FV, const Real *__restrict__ phic, int G, int N,
                                             int i) {
  Real f = 0;
  for (int g0 = 0; g0 < G; g0 += 8) {
    Real a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = g0 + u < G;
      a[u] = in ? FV[(size_t)(g0 + u) * N + i] : (Real)0;
      b[u] = in ? phic[(size_t)(g0 + u) * N + i] : (Real)0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (g0 + u < G) f += a[u] * b[u];
  }
  return f;
}

// rhs + sum over h != g of Sigma_s(h -> g) V phi_h, in h order, batched as above
template <typename Real>
__device__ __forceinline__ Real cell_inscatter(const Real *__restrict__ SV, const Real *__restrict__ phic, int g,
                                               int G, int N, int i, Real rhs) {
  for (int h0 = 0; h0 < G; h0 += 8) {
    Real a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = h0 + u < G && h0 + u != g;
      a[u] = in ? SV[((size_t)g * G + h0 + u) * N + i] : (Real)0;
      b[u] = in ? phic[(size_t)(h0 + u) * N + i] : (Real)0;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (h0 + u < G && h0 + u != g) rhs += a[u] * b[u];
  }
  return rhs;
}

template <typename Real, bool SMEM, typename Idx>
__global__ void __launch_bounds__(1024, 1) cmfd_solve_kernel(CmfdTopo t, double *__restrict__ cur, double *__restrict__ leak,
                                                             const Real *__restrict__ cphi, const Real *__restrict__ TV,
                                                             const Real *__restrict__ SV, const Real *__restrict__ FV,
                                                             const Real *__restrict__ CHI, Real *__restrict__ din,
                                                             Real *__restrict__ diag, Real *__restrict__ phic,
                                                             Real *__restrict__ gx, Real *__restrict__ grd,
                                                             Real *__restrict__ gsrc, Real *__restrict__ fis,
                                                             Real *__restrict__ ratio, double *__restrict__ scal,
                                                             int n_outer, int n_inner, Real omega, double tol) {
  __shared__ double red32[32];
  const int N = t.N, G = t.G, Gp = t.Gp, NE = t.n_entries;
  extern __shared__ unsigned char dyn[];
  Real *s_src, *s_rd, *s_x, *s_din;
  const int32_t *s_off;
  const Idx *s_nbr;
  if (SMEM) {
    Real *base = reinterpret_cast<Real *>(dyn);
    s_src = base;
    s_rd = s_src + N;
    s_x = s_rd + N;
    s_din = s_x + N;
    int32_t *w_off = reinterpret_cast<int32_t *>(s_din + NE);
    Idx *w_nbr = reinterpret_cast<Idx *>(w_off + (N + 1));
    for (int i = threadIdx.x; i <= N; i += blockDim.x) w_off[i] = t.cif_off[i];
    for (int q = threadIdx.x; q < NE; q += blockDim.x) w_nbr[q] = (Idx)t.nbr[q];
    s_off = w_off;
    s_nbr = w_nbr;
  } else {
    s_src = gsrc;
    s_rd = grd;
    s_x = gx;
    s_din = din + (size_t)NE * G;  // one group's worth past the [G][NE] coefficients
    s_off = t.cif_off;
    s_nbr = reinterpret_cast<const Idx *>(t.nbr);
  }
  // 1. coefficients from the tallied currents (leakage terms formed in FP64); thread x = g N + i
  for (int x = threadIdx.x; x < N * G; x += blockDim.x) {
    const int g = x / N, i = x - g * N;
    const Real pi = cphi[x];
    const double inv_pi = (pi > (Real)0) ? 1.0 / (double)pi : 0.0;
    double out = leak[(size_t)i * Gp + g];
    for (int q = t.cif_off[i]; q < t.cif_off[i + 1]; ++q) {
      const int e = t.cif[q] >> 1, side = t.cif[q] & 1;
      const int j = t.if_cells[2 * e + (side ^ 1)];
      const Real pj = cphi[(size_t)g * N + j];
      out += cur[(size_t)(2 * e + side) * Gp + g];
      din[(size_t)g * NE + q] = (pj > (Real)0) ? (Real)(cur[(size_t)(2 * e + (side ^ 1)) * Gp + g] / (double)pj) : (Real)0;
    }
    diag[x] = TV[x] - SV[((size_t)g * G + g) * N + i] + (Real)(out * inv_pi);
    phic[x] = pi;
  }
  __syncthreads();
  // clear the tallies for the next sweep
  for (int x = threadIdx.x; x < NE * Gp; x += blockDim.x) cur[x] = 0.0;
  for (int x = threadIdx.x; x < N * Gp; x += blockDim.x) leak[x] = 0.0;
  double kc = scal[S_K];
  // 2. coarse power iteration
  for (int it = 0; it < n_outer; ++it) {
    double fsum = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const Real f = cell_fission(FV, phic, G, N, i);
      fis[i] = f;
      fsum += (double)f;
    }
    const double F_old = block_sum_1024(fsum, red32);
    const Real inv_k = (Real)(1.0 / kc);
    for (int g = 0; g < G; ++g) {
      // the group's fixed source (fission and other groups' scattering), 1/diagonal and
      // coefficients, staged once per group
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        Real rhs = CHI[(size_t)g * N + i] * fis[i] * inv_k;
        rhs = cell_inscatter(SV, phic, g, G, N, i, rhs);
        s_src[i] = rhs;
        const Real dg = diag[(size_t)g * N + i];
        s_rd[i] = (dg > (Real)0) ? (Real)1 / dg : (Real)0;
        s_x[i] = phic[(size_t)g * N + i];
      }
      for (int q = threadIdx.x; q < NE; q += blockDim.x) s_din[q] = din[(size_t)g * NE + q];
      __syncthreads();
      // over-relaxed Gauss-Seidel, colour by colour, in place (one barrier per colour)
      for (int j = 0; j < n_inner; ++j) {
        for (int c = 0; c < t.n_colors; ++c) {
          const int c1 = t.coff[c + 1];
          for (int i = t.coff[c] + threadIdx.x; i < c1; i += blockDim.x) {
            Real rhs = s_src[i];
            for (int q = s_off[i]; q < s_off[i + 1]; ++q) rhs += s_din[q] * s_x[s_nbr[q]];
            const Real rd = s_rd[i];
            if (rd > (Real)0) s_x[i] = fma(omega, rhs * rd - s_x[i], s_x[i]);
          }
          __syncthreads();
        }
      }
      for (int i = threadIdx.x; i < N; i += blockDim.x) phic[(size_t)g * N + i] = s_x[i];
      __syncthreads();
    }
    fsum = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const Real f = cell_fission(FV, phic, G, N, i);
      fsum += (double)f;
    }
    const double F_new = block_sum_1024(fsum, red32);
    const double k_prev = kc;
    if (F_new > 0.0 && F_old > 0.0) kc = kc * F_new / F_old;
    if (tol > 0.0 && F_new > 0.0 && F_old > 0.0) {
      // stop once k and the normalised coarse fission source have settled to tol
      double dmax = 0.0;
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const Real f = cell_fission(FV, phic, G, N, i);
        if (f > (Real)0) dmax = fmax(dmax, fabs(1.0 - ((double)fis[i] / F_old) * (F_new / (double)f)));
      }
      const double dm = block_max_1024(dmax, red32);
      if (threadIdx.x == 0) scal[S_CMFD_IT] += 1.0;
      if (fabs(kc - k_prev) <= tol * kc && dm <= tol) break;
    } else if (threadIdx.x == 0) {
      scal[S_CMFD_IT] += 1.0;
    }
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

// The same coarse solve on a thread-block cluster: CTA b of the cluster owns, in every colour, a
// contiguous slice of that colour's cells, and keeps the per-group working set of its cells
// (source, 1/diagonal, iterate, coefficients, neighbour locators) in its own shared memory.
// A neighbour owned by another CTA is read from that CTA's shared memory (distributed shared
// memory); one cluster barrier ends each colour sweep. Fission sums are reduced per CTA, then
// summed over the CTAs in rank order by every CTA, so all of them take identical k updates.
struct CmfdCluster {
  const int32_t *cbase;    // [C+1] owned cells of CTA b: own_cell[cbase[b] .. cbase[b+1])
  const int32_t *own_cell; // global cell id of each owned cell, colour by colour
  const int32_t *ccoff;    // [C][n_colors+1] local offsets of each colour within a CTA's cells
  const int32_t *ebase;    // [C+1] owned entries of CTA b
  const int32_t *eoff;     // [sum of cells + C] local entry offsets per owned cell (per CTA)
  const int32_t *loc;      // [entries] neighbour's owner CTA << 16 | its local index there
};

template <typename Real>
__global__ void __launch_bounds__(1024, 1) cmfd_solve_cluster_kernel(CmfdTopo t, CmfdCluster cl, double *__restrict__ cur,
                                                                      double *__restrict__ leak, const Real *__restrict__ cphi,
                                                                      const Real *__restrict__ TV, const Real *__restrict__ SV,
                                                                      const Real *__restrict__ FV, const Real *__restrict__ CHI,
                                                                      Real *__restrict__ din, Real *__restrict__ diag,
                                                                      Real *__restrict__ phic, Real *__restrict__ fis,
                                                                      Real *__restrict__ ratio, double *__restrict__ scal,
                                                                      int n_outer, int n_inner, Real omega, double tol) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks(), b = (int)cluster.block_rank();
  __shared__ double red32[32];
  __shared__ double s_part[2];
  const int N = t.N, G = t.G, Gp = t.Gp, NE = t.n_entries;
  const int c0 = cl.cbase[b], nc = cl.cbase[b + 1] - c0;
  const int e0 = cl.ebase[b], ne = cl.ebase[b + 1] - e0;
  const int32_t *own = cl.own_cell + c0;
  const int32_t *eoff = cl.eoff + c0 + b;  // nc + 1 local offsets
  const int32_t *coff = cl.ccoff + (size_t)b * (t.n_colors + 1);
  // the iterate sits at the same shared-memory offset in every CTA (sized by the largest slice),
  // so a neighbour's value is read at its owner's copy of that offset; two copies (s_x and
  // s_x + ncmax) alternate from group to group, so the next group is staged while other CTAs may
  // still read the current one
  int ncmax = 0;
  for (int r = 0; r < C; ++r) ncmax = max(ncmax, cl.cbase[r + 1] - cl.cbase[r]);
  extern __shared__ unsigned char dyn[];
  Real *s_x = reinterpret_cast<Real *>(dyn);
  Real *s_src = s_x + 2 * ncmax;
  Real *s_rd = s_src + ncmax;
  Real *s_din = s_rd + ncmax;
  int32_t *s_eoff = reinterpret_cast<int32_t *>(s_din + ne);
  // each entry's neighbour iterate as one generic address (this CTA's shared memory or another's
  // through distributed shared memory), resolved once, so a colour sweep loads it without a branch
  uintptr_t np_at = reinterpret_cast<uintptr_t>(s_eoff + nc + 1);
  np_at = (np_at + 7) & ~(uintptr_t)7;
  const Real **s_np = reinterpret_cast<const Real **>(np_at);
  for (int q = threadIdx.x; q < ne; q += blockDim.x) {
    const int l = cl.loc[e0 + q], r = l >> 16, k = l & 0xffff;
    s_np[q] = (r == b) ? s_x + k : cluster.map_shared_rank(s_x + k, r);
  }
  for (int i = threadIdx.x; i <= nc; i += blockDim.x) s_eoff[i] = eoff[i];
  // 1. coefficients of the owned cells from the tallied currents (FP64 leakage terms)
  for (int x = threadIdx.x; x < nc * G; x += blockDim.x) {
    const int li = x / G, g = x - li * G, i = own[li];
    const size_t xi = (size_t)g * N + i;
    const Real pi = cphi[xi];
    const double inv_pi = (pi > (Real)0) ? 1.0 / (double)pi : 0.0;
    double out = leak[(size_t)i * Gp + g];
    // coefficients stored in this CTA's entry order (its slice e0 .. e0 + ne of each group's
    // row), so the per-group staging below reads them contiguously
    const int q_base = t.cif_off[i];
    Real *drow = din + (size_t)g * NE + e0 + eoff[li];
    for (int q = q_base; q < t.cif_off[i + 1]; ++q) {
      const int e = t.cif[q] >> 1, side = t.cif[q] & 1;
      const int j = t.if_cells[2 * e + (side ^ 1)];
      const Real pj = cphi[(size_t)g * N + j];
      out += cur[(size_t)(2 * e + side) * Gp + g];
      drow[q - q_base] = (pj > (Real)0) ? (Real)(cur[(size_t)(2 * e + (side ^ 1)) * Gp + g] / (double)pj) : (Real)0;
    }
    diag[xi] = TV[xi] - SV[((size_t)g * G + g) * N + i] + (Real)(out * inv_pi);
    phic[xi] = pi;
  }
  cluster.sync();  // every CTA's currents read before any are cleared
  for (int x = b * blockDim.x + threadIdx.x; x < NE * Gp; x += C * blockDim.x) cur[x] = 0.0;
  for (int x = b * blockDim.x + threadIdx.x; x < N * Gp; x += C * blockDim.x) leak[x] = 0.0;
  // cluster-wide reductions publish each CTA's partial in one of two slots, alternately: a slot is
  // written again only after the next reduction's barrier, which no CTA passes before every CTA
  // has finished reading the slot, so one barrier per reduction suffices
  int sp = 0;
  auto cluster_sum = [&](double v) {
    const double p = block_sum_1024(v, red32);
    if (threadIdx.x == 0) s_part[sp] = p;
    cluster.sync();
    double tot = 0.0;
    for (int r = 0; r < C; ++r) tot += *cluster.map_shared_rank(&s_part[sp], r);
    sp ^= 1;
    return tot;
  };
  auto cluster_max = [&](double v) {
    const double p = block_max_1024(v, red32);
    if (threadIdx.x == 0) s_part[sp] = p;
    cluster.sync();
    double m = 0.0;
    for (int r = 0; r < C; ++r) m = fmax(m, *cluster.map_shared_rank(&s_part[sp], r));
    sp ^= 1;
    return m;
  };
  // the group's fixed source, 1/diagonal, coefficients and iterate (into copy `to` of s_x)
  auto stage = [&](int g, Real inv_k, int to) {
    Real *sx = s_x + to * ncmax;
    for (int li = threadIdx.x; li < nc; li += blockDim.x) {
      const int i = own[li];
      Real rhs = CHI[(size_t)g * N + i] * fis[i] * inv_k;
      rhs = cell_inscatter(SV, phic, g, G, N, i, rhs);
      s_src[li] = rhs;
      const Real dg = diag[(size_t)g * N + i];
      s_rd[li] = (dg > (Real)0) ? (Real)1 / dg : (Real)0;
      sx[li] = phic[(size_t)g * N + i];
    }
    for (int q = threadIdx.x; q < ne; q += blockDim.x) s_din[q] = din[(size_t)g * NE + e0 + q];
  };
  int xb = 0;  // the copy of s_x that holds the current group
  double kc = scal[S_K];
  // 2. coarse power iteration. The fission sum that ends an iteration is, operation for operation,
  // the one that starts the next (same cells, same threads, same order), so it is carried over
  // instead of reduced again.
  double F_carry = 0.0;
  for (int it = 0; it < n_outer; ++it) {
    double fsum = 0.0;
    for (int li = threadIdx.x; li < nc; li += blockDim.x) {
      const int i = own[li];
      const Real f = cell_fission(FV, phic, G, N, i);
      fis[i] = f;
      fsum += (double)f;
    }
    const double F_old = it == 0 ? cluster_sum(fsum) : F_carry;
    const Real inv_k = (Real)(1.0 / kc);
    // the first group is staged after the fission sum's barrier, which every CTA passes only once
    // its last colour sweep of the previous iteration is done
    xb ^= 1;
    stage(0, inv_k, xb);
    cluster.sync();  // every CTA's iterate staged before any is read remotely
    for (int g = 0; g < G; ++g) {
      Real *sx = s_x + xb * ncmax;
      const int xo = xb * ncmax;
      for (int j = 0; j < n_inner; ++j) {
        for (int c = 0; c < t.n_colors; ++c) {
          for (int li = coff[c] + threadIdx.x; li < coff[c + 1]; li += blockDim.x) {
            Real rhs = s_src[li];
            const int q0 = s_eoff[li], q1 = s_eoff[li + 1];
            // neighbours in batches of 8: the (local or remote) loads first, then the additions
            // in entry order
            for (int qb = q0; qb < q1; qb += 8) {
              Real xv[8], dv[8];
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const bool in = qb + u < q1;
                xv[u] = in ? s_np[qb + u][xo] : (Real)0;
                dv[u] = in ? s_din[qb + u] : (Real)0;
              }
#pragma unroll
              for (int u = 0; u < 8; ++u)
                if (qb + u < q1) rhs += dv[u] * xv[u];
            }
            const Real rd = s_rd[li];
            if (rd > (Real)0) sx[li] = fma(omega, rhs * rd - sx[li], sx[li]);
          }
          // the group's last colour sweep ends with the next group's staging barrier instead
          if (j + 1 < n_inner || c + 1 < t.n_colors) cluster.sync();
        }
      }
      // this CTA's sweeps are done (its own reads of the staged source, diagonal and
      // coefficients; its own iterate final); other CTAs may still read this copy of the iterate
      __syncthreads();
      for (int li = threadIdx.x; li < nc; li += blockDim.x) phic[(size_t)g * N + own[li]] = sx[li];
      if (g + 1 < G) {
        // each thread stages only owned cells whose other-group values it wrote itself
        xb ^= 1;
        stage(g + 1, inv_k, xb);
        cluster.sync();  // every CTA's last colour sweep of g done and group g + 1 staged
      }
    }
    fsum = 0.0;
    for (int li = threadIdx.x; li < nc; li += blockDim.x) {
      const int i = own[li];
      const Real f = cell_fission(FV, phic, G, N, i);
      fsum += (double)f;
    }
    const double F_new = cluster_sum(fsum);
    F_carry = F_new;
    const double k_prev = kc;
    if (F_new > 0.0 && F_old > 0.0) kc = kc * F_new / F_old;
    if (tol > 0.0 && F_new > 0.0 && F_old > 0.0) {
      // stop once k and the normalised coarse fission source have settled to tol (every CTA takes
      // the same decision from the same cluster-wide values)
      double dmax = 0.0;
      for (int li = threadIdx.x; li < nc; li += blockDim.x) {
        const int i = own[li];
        const Real f = cell_fission(FV, phic, G, N, i);
        if (f > (Real)0) dmax = fmax(dmax, fabs(1.0 - ((double)fis[i] / F_old) * (F_new / (double)f)));
      }
      const double dm = cluster_max(dmax);
      if (b == 0 && threadIdx.x == 0) scal[S_CMFD_IT] += 1.0;
      if (fabs(kc - k_prev) <= tol * kc && dm <= tol) break;
    } else if (b == 0 && threadIdx.x == 0) {
      scal[S_CMFD_IT] += 1.0;
    }
  }
  // 3. prolongation ratios of the owned cells and the accelerated k
  for (int x = threadIdx.x; x < nc * G; x += blockDim.x) {
    const int li = x / G, g = x - li * G;
    const size_t xi = (size_t)g * N + own[li];
    const Real a = cphi[xi], bb = phic[xi];
    ratio[xi] = (a > (Real)0 && bb > (Real)0) ? bb / a : (Real)1;
  }
  if (b == 0 && threadIdx.x == 0) {
    if (isfinite(kc) && kc > 0.0) scal[S_K] = kc;
    else scal[S_STATUS] = 1.0;
  }
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

// phi *= ratio(cell); block partials of sum A f(phi); the last block sets the normalisation.
template <typename Real>
__global__ void __launch_bounds__(256) cmfd_prolong_kernel(int R, int G, int Gp, int N, const int32_t *__restrict__ cell,
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
      const Real v = phi[(size_t)r * Gp + g] * ratio[(size_t)g * N + c];
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
__global__ void cmfd_psi_kernel(long long n, int P, int G, int N, const TrackRec *__restrict__ trk,
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
  const Real f = ratio[(size_t)g * N + cell[r]];
  for (int p = 0; p < P; ++p) psi[(td * P + p) * G + g] *= f;
}

}  // namespace moc
