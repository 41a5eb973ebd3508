// Tensor-core GEMM of the warm-start network on sm_103a: tcgen05.mma with the accumulator in
// tensor memory (TMEM), operands staged by the CTA's threads into shared memory in the canonical
// K-major layout (no swizzle), one elected thread issuing the MMAs, completion signalled on an
// mbarrier by tcgen05.commit, and the epilogue read back with tcgen05.ld.
//
// D[m][n] = sum_k A(m, k) B(n, k) over a 128-row tile of A and up to 256 columns. Operands in FP32
// are split into bf16 pairs x = hi + lo (hi = bf16(x), lo = bf16(x - hi)), so the products keep
// about 16 significant bits of every FP32 operand; bf16 operands (the network's weights) are used
// as they are. Accumulation is FP32 in TMEM:
//   A FP32, B bf16:  D = A_hi B + A_lo B                 (2 MMAs per k step)
//   A FP32, B FP32:  D = A_hi B_hi + A_lo B_hi + A_hi B_lo (3 MMAs per k step)
//
// Every wait is bounded (about one second of the global timer); a wait that runs out sets *err,
// skips the epilogue, and the CTA still frees its TMEM before it returns.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mlp_tc {

constexpr int kTileM = 128;   // rows of D per CTA: one TMEM lane per row
constexpr int kMaxN = 256;    // columns of D (FP32 TMEM columns)
constexpr int kKC = 64;       // k elements staged per round
constexpr int kThreads = 256;

// operand sources
enum { SRC_F32 = 0,      // FP32, element (r, k) at p[r * ld + k]   (k contiguous)
       SRC_F32_T = 1,    // FP32, element (r, k) at p[k * ld + r]   (r contiguous)
       SRC_BF16 = 2,     // bf16, element (r, k) at p[r * ld + k]
       SRC_BF16_T = 3 }; // bf16, element (r, k) at p[k * ld + r]

// epilogues
enum { EPI_ACT = 0,      // Z = D + bias; A_next = SiLU(Z)
       EPI_LAST = 1,     // Z = D + bias; y = Z * out_sd + out_mean (when y != null)
       EPI_DACT = 2,     // dZ = D * SiLU'(Zprev)
       EPI_ATOMIC = 3 }; // C += D (atomically: split-k partial)

struct TcArgs {
  int M, N, K;            // D is M x N, reduction over K
  const void *a;          // A source
  int lda;
  const void *b;          // B source
  int ldb;
  int k_per_cta;          // k range of one CTA (blockIdx.y splits K; EPI_ATOMIC only)
  float *out;             // Z, dZ or C  [M][ldo]
  int ldo;
  float *out2;            // A_next (EPI_ACT) or y (EPI_LAST)
  const float *bias;      // [N]
  const float *aux;       // Zprev [M][ldo] (EPI_DACT)
  const float *out_mean, *out_sd;  // EPI_LAST de-standardisation
  int *err;               // set to 1 when a wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a tile with kc columns in the canonical K-major layout without
// swizzle: 8 x 8 core matrices of 128 contiguous bytes (8 rows of 16 bytes), core matrices
// adjacent in k 128 bytes apart (the leading byte offset), 8-row groups kc * 16 bytes apart (the
// stride byte offset)
__device__ __forceinline__ uint32_t kmaj_off(int r, int k, int kc) {
  return (uint32_t)(((r >> 3) * (kc >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start address, leading and stride byte offsets (16-byte
// units), descriptor version 1 (bits 46-47), no swizzle (layout 0 in bits 61-63)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B bf16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the mbarrier phase with the given parity; false after about one second
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}

__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }

__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.0f / (1.0f + __expf(-z));
  return s * (1.0f + z * (1.0f - s));
}

template <int SRC> __device__ __forceinline__ float fetch(const void *p, int ld, int r, int k) {
  if (SRC == SRC_F32) return static_cast<const float *>(p)[(size_t)r * ld + k];
  if (SRC == SRC_F32_T) return static_cast<const float *>(p)[(size_t)k * ld + r];
  if (SRC == SRC_BF16) return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[(size_t)r * ld + k]);
  return __bfloat162float(static_cast<const __nv_bfloat16 *>(p)[(size_t)k * ld + r]);
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 a, __nv_bfloat16 b) {
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// stage rows [r0, r0 + R) x k [k0, k0 + kKC) of a source into hi (and lo for FP32 sources) tiles;
// out-of-range elements are zero. The loop order follows the source's contiguous index. Sources
// with k contiguous and 16-byte aligned rows move 4 FP32 (or 8 bf16) values per thread step:
// one 16-byte load, and 8 (16) contiguous bytes of one core-matrix row in shared memory.
template <int SRC>
__device__ __forceinline__ void stage(unsigned char *hi, unsigned char *lo, const void *p, int ld, int r0, int R,
                                      int rmax, int k0, int kmax) {
  constexpr bool T = (SRC == SRC_F32_T || SRC == SRC_BF16_T);
  constexpr bool F32 = (SRC == SRC_F32 || SRC == SRC_F32_T);
  if (SRC == SRC_F32 && (ld & 3) == 0 && ((uintptr_t)p & 15) == 0) {
    const float *q = static_cast<const float *>(p);
    for (int e = threadIdx.x; e < R * (kKC / 4); e += kThreads) {
      const int r = e / (kKC / 4), k = (e % (kKC / 4)) * 4;
      const int gr = r0 + r, gk = k0 + k;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < rmax) {
        if (gk + 3 < kmax) {
          v = *reinterpret_cast<const float4 *>(q + (size_t)gr * ld + gk);
        } else {
          if (gk < kmax) v.x = q[(size_t)gr * ld + gk];
          if (gk + 1 < kmax) v.y = q[(size_t)gr * ld + gk + 1];
          if (gk + 2 < kmax) v.z = q[(size_t)gr * ld + gk + 2];
        }
      }
      const __nv_bfloat16 hx = __float2bfloat16_rn(v.x), hy = __float2bfloat16_rn(v.y), hz = __float2bfloat16_rn(v.z),
                          hw = __float2bfloat16_rn(v.w);
      const uint32_t o = kmaj_off(r, k, kKC);
      *reinterpret_cast<uint2 *>(hi + o) = make_uint2(pack_bf16(hx, hy), pack_bf16(hz, hw));
      *reinterpret_cast<uint2 *>(lo + o) = make_uint2(
          pack_bf16(__float2bfloat16_rn(v.x - __bfloat162float(hx)), __float2bfloat16_rn(v.y - __bfloat162float(hy))),
          pack_bf16(__float2bfloat16_rn(v.z - __bfloat162float(hz)), __float2bfloat16_rn(v.w - __bfloat162float(hw))));
    }
    return;
  }
  if (SRC == SRC_BF16 && (ld & 7) == 0 && ((uintptr_t)p & 15) == 0) {
    const __nv_bfloat16 *q = static_cast<const __nv_bfloat16 *>(p);
    for (int e = threadIdx.x; e < R * (kKC / 8); e += kThreads) {
      const int r = e / (kKC / 8), k = (e % (kKC / 8)) * 8;
      const int gr = r0 + r, gk = k0 + k;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gr < rmax) {
        if (gk + 7 < kmax) {
          v = *reinterpret_cast<const uint4 *>(q + (size_t)gr * ld + gk);
        } else {
          __nv_bfloat16 t[8];
          for (int j = 0; j < 8; ++j) t[j] = (gk + j < kmax) ? q[(size_t)gr * ld + gk + j] : __float2bfloat16_rn(0.f);
          v = make_uint4(pack_bf16(t[0], t[1]), pack_bf16(t[2], t[3]), pack_bf16(t[4], t[5]), pack_bf16(t[6], t[7]));
        }
      }
      *reinterpret_cast<uint4 *>(hi + kmaj_off(r, k, kKC)) = v;
    }
    return;
  }
  for (int e = threadIdx.x; e < R * kKC; e += kThreads) {
    const int r = T ? (e % R) : (e / kKC);
    const int k = T ? (e / R) : (e % kKC);
    const int gr = r0 + r, gk = k0 + k;
    const float v = (gr < rmax && gk < kmax) ? fetch<SRC>(p, ld, gr, gk) : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const uint32_t o = kmaj_off(r, k, kKC);
    *reinterpret_cast<__nv_bfloat16 *>(hi + o) = h;
    if (F32) *reinterpret_cast<__nv_bfloat16 *>(lo + o) = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t addr, uint32_t *v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// the epilogue of NC columns c0 .. c0 + NC - 1 of the tile (local), for one row: groups of 4
// columns that lie inside the tile and start 16-byte aligned in the output go out as float4
template <int EPI, int NC>
__device__ __forceinline__ void epilogue_cols(const TcArgs &g, const float *s_bias, const uint32_t *v, int row, int n0,
                                              int c0, int Nt) {
  if (row >= g.M) return;
  // float4 accesses need 16-byte aligned rows: the row pitch a multiple of 4 and every array's base
  // aligned (a caller's workspace carved at arbitrary float offsets need not be)
  const bool vec = (g.ldo & 3) == 0 && ((uintptr_t)g.out & 15) == 0 && ((uintptr_t)g.out2 & 15) == 0 &&
                   ((uintptr_t)g.aux & 15) == 0;
#pragma unroll
  for (int j0 = 0; j0 < NC; j0 += 4) {
    const int cl = c0 + j0;
    if (cl >= Nt) break;
    const size_t o = (size_t)row * g.ldo + n0 + cl;
    float d[4], z[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) d[j] = __uint_as_float(v[j0 + j]);
    const bool full = vec && cl + 3 < Nt;
    if (EPI == EPI_ATOMIC) {
      for (int j = 0; j < 4 && cl + j < Nt; ++j) atomicAdd(g.out + o + j, d[j]);
      continue;
    }
    if (EPI == EPI_DACT) {
      float a[4];
      if (full) {
        const float4 t = *reinterpret_cast<const float4 *>(g.aux + o);
        a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
      } else {
        for (int j = 0; j < 4; ++j) a[j] = (cl + j < Nt) ? g.aux[o + j] : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) z[j] = d[j] * silu_grad(a[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) z[j] = d[j] + s_bias[cl + j];
    }
    if (full) {
      *reinterpret_cast<float4 *>(g.out + o) = make_float4(z[0], z[1], z[2], z[3]);
    } else {
      for (int j = 0; j < 4 && cl + j < Nt; ++j) g.out[o + j] = z[j];
    }
    if (EPI == EPI_ACT || (EPI == EPI_LAST && g.out2)) {
      float y[4];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        y[j] = (EPI == EPI_ACT) ? silu(z[j])
                                : z[j] * g.out_sd[n0 + min(cl + j, Nt - 1)] + g.out_mean[n0 + min(cl + j, Nt - 1)];
      if (full) {
        *reinterpret_cast<float4 *>(g.out2 + o) = make_float4(y[0], y[1], y[2], y[3]);
      } else {
        for (int j = 0; j < 4 && cl + j < Nt; ++j) g.out2[o + j] = y[j];
      }
    }
  }
}

// One CTA: D tile rows [m0, m0 + 128) (blockIdx.x), columns [n0, n0 + 256) (blockIdx.z), k range
// [kb, ke) (blockIdx.y).
// Shared memory: A hi/lo (2 x 16 KB), B hi/lo (2 x 32 KB), mbarrier, TMEM address.
template <int ASRC, int BSRC, int EPI>
__global__ void __launch_bounds__(kThreads, 2) tc_gemm_kernel(TcArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *a_hi = sm, *a_lo = sm + kTileM * kKC * 2;
  unsigned char *b_hi = a_lo + kTileM * kKC * 2, *b_lo = b_hi + kMaxN * kKC * 2;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int failed;
  __shared__ float s_bias[kMaxN];
  constexpr bool A32 = (ASRC == SRC_F32 || ASRC == SRC_F32_T);
  constexpr bool B32 = (BSRC == SRC_F32 || BSRC == SRC_F32_T);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTileM, n0 = blockIdx.z * kMaxN;
  const int kb = blockIdx.y * g.k_per_cta, ke = min(g.K, kb + g.k_per_cta);
  const int Nt = min(kMaxN, g.N - n0);                // columns of this tile
  const int Np = (Nt + 15) & ~15;                     // MMA N: a multiple of 16 (M = 128)
  const uint32_t ncols = Np <= 32 ? 32 : Np <= 64 ? 64 : Np <= 128 ? 128 : 256;
  if (threadIdx.x == 0) {
    failed = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(kTileM, Np);
  // the tile's bias values (read by the epilogue; made visible by the first round's barrier)
  if (EPI == EPI_ACT || EPI == EPI_LAST)
    for (int n = threadIdx.x; n < Nt; n += kThreads) s_bias[n] = g.bias[n0 + n];
  uint32_t parity = 0;
  int first = 1;
  for (int k0 = kb; k0 < ke; k0 += kKC) {
    stage<ASRC>(a_hi, a_lo, g.a, g.lda, m0, kTileM, g.M, k0, ke);
    stage<BSRC>(b_hi, b_lo, g.b, g.ldb, n0, Np, g.N, k0, ke);
    // make the threads' shared-memory writes visible to the tensor core's (async) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t sa = smem_u32(a_hi), sal = smem_u32(a_lo), sb = smem_u32(b_hi), sbl = smem_u32(b_lo);
      const uint32_t lbo = 128, sbo = kKC * 16;
#pragma unroll
      for (int kk = 0; kk < kKC / 16; ++kk) {
        const uint32_t step = kk * 2 * 128;  // 16 k = two core matrices
        const uint64_t dah = smem_desc(sa + step, lbo, sbo), dbh = smem_desc(sb + step, lbo, sbo);
        mma_bf16(tmem, dah, dbh, idesc, first ? 0u : 1u);
        first = 0;
        if (A32) mma_bf16(tmem, smem_desc(sal + step, lbo, sbo), dbh, idesc, 1u);
        if (B32) mma_bf16(tmem, dah, smem_desc(sbl + step, lbo, sbo), idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar))
                   : "memory");
    }
    first = 0;
    // the MMAs read the staged tiles: wait for them before the next round overwrites them
    if (!mbar_wait(smem_u32(&bar), parity)) failed = 1;
    parity ^= 1u;
    __syncthreads();
    if (failed) break;
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (!failed && kb < ke) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of D), column half w / 4, 32
    // columns per tcgen05.ld where the half allows (8 otherwise); results leave as float4 stores
    const int q = warp & 3, half = warp >> 2;
    const int row = m0 + 32 * q + lane;
    const int c_beg = half * (Np / 2), c_end = c_beg + Np / 2;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    int c0 = c_beg;
    for (; c0 + 32 <= c_end; c0 += 32) {
      uint32_t v[32];
      tmem_ld32(lane_base + (uint32_t)c0, v);
      epilogue_cols<EPI, 32>(g, s_bias, v, row, n0, c0, Nt);
    }
    for (; c0 < c_end; c0 += 8) {
      uint32_t v[8];
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                   : "r"(lane_base + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      epilogue_cols<EPI, 8>(g, s_bias, v, row, n0, c0, Nt);
    }
  }
  if (failed && threadIdx.x == 0) atomicExch(g.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

// dynamic shared memory of tc_gemm_kernel
constexpr size_t kSmemBytes = (size_t)2 * kTileM * kKC * 2 + (size_t)2 * kMaxN * kKC * 2;

}  // namespace mlp_tc
