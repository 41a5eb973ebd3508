// Learned warm start: a 4-layer MLP (bf16 weights, FP32 accumulation, FP32 master weights, Adam)
// in hand-written CUDA kernels. See include/moc_mlp.h for the contract.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "moc_gb300.h"
#include "moc_mlp.h"

namespace {

constexpr int kLayers = 4;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// C[M][N] (=, or += atomically) sum over k of A(m,k) B(k,n); A(m,k) = TA ? A[k lda + m] :
// A[m lda + k]; B(k,n) = TB ? B[n ldb + k] : B[k ldb + n]. 64x64 tiles, 16-deep k slices, 256
// threads each owning a 4x4 block of C; blockIdx.z splits K into chunks of k_per_block.
template <bool TA, bool TB, typename BT>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda,
                                                   const BT *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                                   int k_per_block, int atomic_out) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kbeg = blockIdx.z * k_per_block;
  const int kend = min(K, kbeg + k_per_block);
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int mm, kk;
      if (TA) { mm = e & 63; kk = e >> 6; } else { kk = e & 15; mm = e >> 4; }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < kend) v = TA ? A[(size_t)gk * lda + gm] : A[(size_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < 1024; e += 256) {
      int nn, kk;
      if (TB) { kk = e & 15; nn = e >> 4; } else { nn = e & 63; kk = e >> 6; }
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < kend) v = to_f(TB ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn]);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
      if (gm < M && gn < N) {
        if (atomic_out) atomicAdd(&C[(size_t)gm * ldc + gn], acc[i][j]);
        else C[(size_t)gm * ldc + gn] = acc[i][j];
      }
    }
}

__device__ __forceinline__ float sigmoid(float x) { return 1.0f / (1.0f + expf(-x)); }

__global__ void normalize_kernel(int64_t n, int d, const float *__restrict__ x, const float *__restrict__ mean,
                                 const float *__restrict__ sd, float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  const int j = (int)(i % d);
  out[i] = (x[i] - mean[j]) / sd[j];
}

// Z += b (per column); if act, A = SiLU(Z)
__global__ void bias_act_kernel(int64_t n, int d, float *__restrict__ Z, const float *__restrict__ b,
                                float *__restrict__ Aout, int act) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  const float z = Z[i] + b[i % d];
  Z[i] = z;
  if (act) Aout[i] = z * sigmoid(z);
}

__global__ void denorm_kernel(int64_t n, int d, const float *__restrict__ z, const float *__restrict__ mean,
                              const float *__restrict__ sd, float *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  const int j = (int)(i % d);
  y[i] = z[i] * sd[j] + mean[j];
}

// dZ = 2 (z - (y - mean)/sd) / (n d); loss += sum (z - y_norm)^2 / (n d)
__global__ void mse_grad_kernel(int64_t n, int d, const float *__restrict__ z, const float *__restrict__ y,
                                const float *__restrict__ mean, const float *__restrict__ sd, float *__restrict__ dz,
                                float *__restrict__ loss) {
  __shared__ float red[256];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (i < n * d) {
    const int j = (int)(i % d);
    const float diff = z[i] - (y[i] - mean[j]) / sd[j];
    const float inv = 1.0f / (float)(n * d);
    dz[i] = 2.0f * diff * inv;
    l = diff * diff * inv;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// dZ = dA * SiLU'(Z)
__global__ void silu_back_kernel(int64_t n, const float *__restrict__ dA, const float *__restrict__ Z,
                                 float *__restrict__ dZ) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = sigmoid(Z[i]);
  dZ[i] = dA[i] * s * (1.0f + Z[i] * (1.0f - s));
}

// gb[j] += sum over a chunk of rows of dZ[row][j]
__global__ void colsum_kernel(int64_t n, int d, const float *__restrict__ dZ, float *__restrict__ gb, int rows) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows;
  const int64_t r1 = min(n, r0 + rows);
  float s = 0.f;
  for (int64_t r = r0; r < r1; ++r) s += dZ[r * d + j];
  atomicAdd(&gb[j], s);
}

__global__ void adam_kernel(int64_t n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float c1, float c2, __nv_bfloat16 *__restrict__ wh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
  w[i] = wi;
  if (wh) wh[i] = __float2bfloat16(wi);
}

__global__ void to_bf16_kernel(int64_t n, const float *__restrict__ w, __nv_bfloat16 *__restrict__ wh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wh[i] = __float2bfloat16(w[i]);
}

inline unsigned grid1(int64_t n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

struct moc_mlp {
  int device = 0;
  int dims[kLayers + 1] = {0};
  std::string err;
  float *W[kLayers] = {}, *b[kLayers] = {};
  __nv_bfloat16 *Wh[kLayers] = {};
  float *mW[kLayers] = {}, *vW[kLayers] = {}, *mb[kLayers] = {}, *vb[kLayers] = {};
  float *gW[kLayers] = {}, *gb[kLayers] = {};
  float *in_mean = nullptr, *in_std = nullptr, *out_mean = nullptr, *out_std = nullptr;
  int64_t cap = 0;
  float *Z[kLayers] = {}, *A[kLayers] = {};
  float *dA = nullptr, *dZ = nullptr, *dZ2 = nullptr, *loss = nullptr;
  int64_t step = 0;
};

namespace {

int mfail(moc_mlp *n, int code, const std::string &m) {
  if (n) n->err = m;
  return code;
}

#define MLP_TRY(n, call)                                                                       \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return mfail((n), e_ == cudaErrorMemoryAllocation ? MOC_ERR_OOM : MOC_ERR_CUDA,          \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

int64_t wsize(const moc_mlp *n, int l) { return (int64_t)n->dims[l + 1] * n->dims[l]; }

template <bool TA, bool TB, typename BT>
void gemm(int M, int N, int K, const float *A, int lda, const BT *B, int ldb, float *C, int ldc, cudaStream_t st,
          int k_per_block = 0, bool atomic_out = false) {
  if (k_per_block <= 0) k_per_block = K;
  dim3 grid((N + 63) / 64, (M + 63) / 64, (K + k_per_block - 1) / k_per_block);
  gemm_kernel<TA, TB, BT><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, k_per_block, atomic_out ? 1 : 0);
}

int ensure_workspace(moc_mlp *n, int64_t rows) {
  if (rows <= n->cap) return MOC_OK;
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(n->Z[l]);
    cudaFree(n->A[l]);
    n->Z[l] = n->A[l] = nullptr;
  }
  cudaFree(n->dA);
  cudaFree(n->dZ);
  cudaFree(n->dZ2);
  n->dA = n->dZ = n->dZ2 = nullptr;
  int wmax = 0;
  for (int l = 0; l <= kLayers; ++l) wmax = std::max(wmax, n->dims[l]);
  for (int l = 0; l < kLayers; ++l) {
    MLP_TRY(n, cudaMalloc(&n->Z[l], (size_t)rows * n->dims[l + 1] * sizeof(float)));
    MLP_TRY(n, cudaMalloc(&n->A[l], (size_t)rows * n->dims[l] * sizeof(float)));
  }
  MLP_TRY(n, cudaMalloc(&n->dA, (size_t)rows * wmax * sizeof(float)));
  MLP_TRY(n, cudaMalloc(&n->dZ, (size_t)rows * wmax * sizeof(float)));
  MLP_TRY(n, cudaMalloc(&n->dZ2, (size_t)rows * wmax * sizeof(float)));
  n->cap = rows;
  return MOC_OK;
}

// forward pass into Z[3] (standardised outputs); keeps Z/A for the backward pass
int forward(moc_mlp *n, const float *x, int64_t rows, cudaStream_t st) {
  int rc = ensure_workspace(n, rows);
  if (rc) return rc;
  normalize_kernel<<<grid1(rows * n->dims[0]), 256, 0, st>>>(rows, n->dims[0], x, n->in_mean, n->in_std, n->A[0]);
  for (int l = 0; l < kLayers; ++l) {
    const int din = n->dims[l], dout = n->dims[l + 1];
    gemm<false, true, __nv_bfloat16>((int)rows, dout, din, n->A[l], din, n->Wh[l], din, n->Z[l], dout, st);
    const bool act = l < kLayers - 1;
    bias_act_kernel<<<grid1(rows * dout), 256, 0, st>>>(rows, dout, n->Z[l], n->b[l], act ? n->A[l + 1] : nullptr,
                                                        act ? 1 : 0);
  }
  MLP_TRY(n, cudaGetLastError());
  return MOC_OK;
}

// backward pass of the MSE loss; fills gW, gb and the loss scalar
int backward(moc_mlp *n, const float *y, int64_t rows, cudaStream_t st) {
  const int dlast = n->dims[kLayers];
  MLP_TRY(n, cudaMemsetAsync(n->loss, 0, sizeof(float), st));
  mse_grad_kernel<<<grid1(rows * dlast), 256, 0, st>>>(rows, dlast, n->Z[kLayers - 1], y, n->out_mean, n->out_std,
                                                       n->dZ, n->loss);
  float *dZ = n->dZ, *dZn = n->dZ2;
  for (int l = kLayers - 1; l >= 0; --l) {
    const int din = n->dims[l], dout = n->dims[l + 1];
    MLP_TRY(n, cudaMemsetAsync(n->gW[l], 0, wsize(n, l) * sizeof(float), st));
    MLP_TRY(n, cudaMemsetAsync(n->gb[l], 0, dout * sizeof(float), st));
    // gW[out][in] = sum_rows dZ[row][out] A[row][in], split over chunks of 2048 rows
    gemm<true, false, float>(dout, din, (int)rows, dZ, dout, n->A[l], din, n->gW[l], din, st, 2048, true);
    dim3 g2((dout + 255) / 256, (unsigned)((rows + 2047) / 2048));
    colsum_kernel<<<g2, 256, 0, st>>>(rows, dout, dZ, n->gb[l], 2048);
    if (l > 0) {
      // dA[row][in] = sum_out dZ[row][out] W[out][in]; dZ_prev = dA * SiLU'(Z_prev)
      gemm<false, false, __nv_bfloat16>((int)rows, din, dout, dZ, dout, n->Wh[l], din, n->dA, din, st);
      silu_back_kernel<<<grid1(rows * din), 256, 0, st>>>(rows * din, n->dA, n->Z[l - 1], dZn);
      std::swap(dZ, dZn);
    }
  }
  MLP_TRY(n, cudaGetLastError());
  return MOC_OK;
}

uint64_t splitmix(uint64_t &s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

extern "C" {

int moc_mlp_create(moc_mlp **out, int device, int n_in, int width, int n_out, uint64_t seed) {
  if (!out) return MOC_ERR_ARG;
  *out = nullptr;
  if (n_in < 1 || n_in > 1024 || n_out < 1 || n_out > 1024 ||
      !(width == 32 || width == 64 || width == 128 || width == 256 || width == 512) || device < 0)
    return MOC_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MOC_ERR_CUDA;
  moc_mlp *n = new (std::nothrow) moc_mlp;
  if (!n) return MOC_ERR_OOM;
  n->device = device;
  n->dims[0] = n_in;
  n->dims[1] = n->dims[2] = n->dims[3] = width;
  n->dims[4] = n_out;
  bool ok = true;
  for (int l = 0; l < kLayers && ok; ++l) {
    const size_t w = (size_t)wsize(n, l), bsz = n->dims[l + 1];
    ok = cudaMalloc(&n->W[l], w * 4) == cudaSuccess && cudaMalloc(&n->b[l], bsz * 4) == cudaSuccess &&
         cudaMalloc(&n->Wh[l], w * 2) == cudaSuccess && cudaMalloc(&n->mW[l], w * 4) == cudaSuccess &&
         cudaMalloc(&n->vW[l], w * 4) == cudaSuccess && cudaMalloc(&n->mb[l], bsz * 4) == cudaSuccess &&
         cudaMalloc(&n->vb[l], bsz * 4) == cudaSuccess && cudaMalloc(&n->gW[l], w * 4) == cudaSuccess &&
         cudaMalloc(&n->gb[l], bsz * 4) == cudaSuccess;
  }
  ok = ok && cudaMalloc(&n->in_mean, n_in * 4) == cudaSuccess && cudaMalloc(&n->in_std, n_in * 4) == cudaSuccess &&
       cudaMalloc(&n->out_mean, n_out * 4) == cudaSuccess && cudaMalloc(&n->out_std, n_out * 4) == cudaSuccess &&
       cudaMalloc(&n->loss, 4) == cudaSuccess;
  if (!ok) {
    moc_mlp_destroy(n);
    return MOC_ERR_OOM;
  }
  // Glorot-uniform weights from a seeded splitmix64 stream, zero biases
  int64_t np = 0;
  moc_mlp_dims(n, nullptr, &np);
  std::vector<float> p((size_t)np, 0.f);
  uint64_t s = seed;
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    const double lim = std::sqrt(6.0 / (n->dims[l] + n->dims[l + 1]));
    for (int64_t i = 0; i < wsize(n, l); ++i) {
      const double u = (double)(splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
      p[o++] = (float)((2.0 * u - 1.0) * lim);
    }
    o += n->dims[l + 1];
  }
  std::vector<float> ones(std::max(n_in, n_out), 1.f), zeros(std::max(n_in, n_out), 0.f);
  int rc = moc_mlp_set_params(n, p.data());
  if (!rc) rc = moc_mlp_set_normalization(n, zeros.data(), ones.data(), zeros.data(), ones.data());
  if (rc) {
    moc_mlp_destroy(n);
    return rc;
  }
  *out = n;
  return MOC_OK;
}

void moc_mlp_destroy(moc_mlp *n) {
  if (!n) return;
  cudaSetDevice(n->device);
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(n->W[l]);
    cudaFree(n->b[l]);
    cudaFree(n->Wh[l]);
    cudaFree(n->mW[l]);
    cudaFree(n->vW[l]);
    cudaFree(n->mb[l]);
    cudaFree(n->vb[l]);
    cudaFree(n->gW[l]);
    cudaFree(n->gb[l]);
    cudaFree(n->Z[l]);
    cudaFree(n->A[l]);
  }
  cudaFree(n->in_mean);
  cudaFree(n->in_std);
  cudaFree(n->out_mean);
  cudaFree(n->out_std);
  cudaFree(n->dA);
  cudaFree(n->dZ);
  cudaFree(n->dZ2);
  cudaFree(n->loss);
  delete n;
}

const char *moc_mlp_last_error(const moc_mlp *n) { return n ? n->err.c_str() : "null network"; }

int moc_mlp_dims(const moc_mlp *n, int *dims, int64_t *n_params) {
  if (!n) return MOC_ERR_ARG;
  int64_t np = 0;
  for (int l = 0; l < kLayers; ++l) np += wsize(n, l) + n->dims[l + 1];
  if (dims)
    for (int l = 0; l <= kLayers; ++l) dims[l] = n->dims[l];
  if (n_params) *n_params = np;
  return MOC_OK;
}

int moc_mlp_get_params(moc_mlp *n, float *p) {
  if (!n || !p) return MOC_ERR_ARG;
  cudaSetDevice(n->device);
  MLP_TRY(n, cudaDeviceSynchronize());
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    MLP_TRY(n, cudaMemcpy(p + o, n->W[l], wsize(n, l) * 4, cudaMemcpyDeviceToHost));
    o += wsize(n, l);
    MLP_TRY(n, cudaMemcpy(p + o, n->b[l], n->dims[l + 1] * 4, cudaMemcpyDeviceToHost));
    o += n->dims[l + 1];
  }
  return MOC_OK;
}

int moc_mlp_set_params(moc_mlp *n, const float *p) {
  if (!n || !p) return MOC_ERR_ARG;
  cudaSetDevice(n->device);
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    const int64_t w = wsize(n, l);
    for (int64_t i = 0; i < w + n->dims[l + 1]; ++i)
      if (!std::isfinite(p[o + i])) return mfail(n, MOC_ERR_ARG, "set_params: non-finite parameter");
    MLP_TRY(n, cudaMemcpy(n->W[l], p + o, w * 4, cudaMemcpyHostToDevice));
    o += w;
    MLP_TRY(n, cudaMemcpy(n->b[l], p + o, n->dims[l + 1] * 4, cudaMemcpyHostToDevice));
    o += n->dims[l + 1];
    to_bf16_kernel<<<grid1(w), 256>>>(w, n->W[l], n->Wh[l]);
    MLP_TRY(n, cudaMemset(n->mW[l], 0, w * 4));
    MLP_TRY(n, cudaMemset(n->vW[l], 0, w * 4));
    MLP_TRY(n, cudaMemset(n->mb[l], 0, n->dims[l + 1] * 4));
    MLP_TRY(n, cudaMemset(n->vb[l], 0, n->dims[l + 1] * 4));
  }
  MLP_TRY(n, cudaGetLastError());
  MLP_TRY(n, cudaDeviceSynchronize());
  n->step = 0;
  return MOC_OK;
}

int moc_mlp_set_normalization(moc_mlp *n, const float *in_mean, const float *in_std, const float *out_mean,
                              const float *out_std) {
  if (!n || !in_mean || !in_std || !out_mean || !out_std) return MOC_ERR_ARG;
  for (int j = 0; j < n->dims[0]; ++j)
    if (!(in_std[j] > 0.f) || !std::isfinite(in_mean[j])) return mfail(n, MOC_ERR_ARG, "normalization: bad input stats");
  for (int j = 0; j < n->dims[kLayers]; ++j)
    if (!(out_std[j] > 0.f) || !std::isfinite(out_mean[j]))
      return mfail(n, MOC_ERR_ARG, "normalization: bad output stats");
  cudaSetDevice(n->device);
  MLP_TRY(n, cudaMemcpy(n->in_mean, in_mean, n->dims[0] * 4, cudaMemcpyHostToDevice));
  MLP_TRY(n, cudaMemcpy(n->in_std, in_std, n->dims[0] * 4, cudaMemcpyHostToDevice));
  MLP_TRY(n, cudaMemcpy(n->out_mean, out_mean, n->dims[kLayers] * 4, cudaMemcpyHostToDevice));
  MLP_TRY(n, cudaMemcpy(n->out_std, out_std, n->dims[kLayers] * 4, cudaMemcpyHostToDevice));
  return MOC_OK;
}

int moc_mlp_forward(moc_mlp *n, const float *x, float *y, int64_t rows, void *stream) {
  if (!n || rows < 0 || (rows > 0 && (!x || !y))) return MOC_ERR_ARG;
  if (rows == 0) return MOC_OK;
  cudaSetDevice(n->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = forward(n, x, rows, st);
  if (rc) return rc;
  const int dlast = n->dims[kLayers];
  denorm_kernel<<<grid1(rows * dlast), 256, 0, st>>>(rows, dlast, n->Z[kLayers - 1], n->out_mean, n->out_std, y);
  MLP_TRY(n, cudaGetLastError());
  return MOC_OK;
}

int moc_mlp_train_step(moc_mlp *n, const float *x, const float *y, int64_t rows, float lr, float *loss_out,
                       void *stream) {
  if (!n || rows < 1 || !x || !y || !(lr > 0.f)) return MOC_ERR_ARG;
  cudaSetDevice(n->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = forward(n, x, rows, st);
  if (!rc) rc = backward(n, y, rows, st);
  if (rc) return rc;
  n->step += 1;
  const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)n->step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)n->step)));
  for (int l = 0; l < kLayers; ++l) {
    adam_kernel<<<grid1(wsize(n, l)), 256, 0, st>>>(wsize(n, l), n->W[l], n->gW[l], n->mW[l], n->vW[l], lr, c1, c2,
                                                    n->Wh[l]);
    adam_kernel<<<grid1(n->dims[l + 1]), 256, 0, st>>>(n->dims[l + 1], n->b[l], n->gb[l], n->mb[l], n->vb[l], lr, c1,
                                                       c2, nullptr);
  }
  MLP_TRY(n, cudaGetLastError());
  if (loss_out) {
    MLP_TRY(n, cudaMemcpyAsync(loss_out, n->loss, 4, cudaMemcpyDeviceToHost, st));
    MLP_TRY(n, cudaStreamSynchronize(st));
  }
  return MOC_OK;
}

int moc_mlp_gradients(moc_mlp *n, const float *x, const float *y, int64_t rows, float *grad, float *loss_out,
                      void *stream) {
  if (!n || rows < 1 || !x || !y || !grad) return MOC_ERR_ARG;
  cudaSetDevice(n->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = forward(n, x, rows, st);
  if (!rc) rc = backward(n, y, rows, st);
  if (rc) return rc;
  MLP_TRY(n, cudaStreamSynchronize(st));
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    MLP_TRY(n, cudaMemcpy(grad + o, n->gW[l], wsize(n, l) * 4, cudaMemcpyDeviceToHost));
    o += wsize(n, l);
    MLP_TRY(n, cudaMemcpy(grad + o, n->gb[l], n->dims[l + 1] * 4, cudaMemcpyDeviceToHost));
    o += n->dims[l + 1];
  }
  if (loss_out) MLP_TRY(n, cudaMemcpy(loss_out, n->loss, 4, cudaMemcpyDeviceToHost));
  return MOC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------ no-allocation
// Workspace of moc_mlp_forward_noalloc: one fixed array per device, never allocated at run time.
static __device__ __align__(256) float g_noalloc_ws[MOC_MLP_NOALLOC_FLOATS];

namespace {
constexpr int kMaxDevices = 64;
float *g_noalloc_addr[kMaxDevices] = {};  // device address of g_noalloc_ws, looked up once per device
}  // namespace

extern "C" int moc_mlp_forward_noalloc(moc_mlp *n, const float *x, float *y, int64_t rows, void *stream) {
  if (!n || rows < 0 || (rows > 0 && (!x || !y))) return MOC_ERR_ARG;
  if (rows == 0) return MOC_OK;
  if (n->device >= kMaxDevices) return mfail(n, MOC_ERR_ARG, "forward_noalloc: device index beyond the supported 64");
  const int64_t per_row = (int64_t)n->dims[0] + 2 * n->dims[1] + 2 * n->dims[2] + 2 * n->dims[3] + n->dims[4];
  if (rows > (int64_t)MOC_MLP_NOALLOC_FLOATS / per_row)
    return mfail(n, MOC_ERR_ARG,
                 "forward_noalloc: batch of " + std::to_string(rows) + " rows exceeds the fixed workspace (" +
                     std::to_string((int64_t)MOC_MLP_NOALLOC_FLOATS / per_row) + " rows for this network)");
  MLP_TRY(n, cudaSetDevice(n->device));
  if (!g_noalloc_addr[n->device]) {
    // host code cannot use the array's name as a device address: ask the runtime for it
    float *p = nullptr;
    MLP_TRY(n, cudaGetSymbolAddress((void **)&p, g_noalloc_ws));
    g_noalloc_addr[n->device] = p;
  }
  // carve A0 | Z0 | A1 | Z1 | A2 | Z2 | A3 | Z3 out of the workspace
  float *ws = g_noalloc_addr[n->device];
  float *Aw[kLayers], *Zw[kLayers];
  size_t o = 0;
  for (int l = 0; l < kLayers; ++l) {
    Aw[l] = ws + o;
    o += (size_t)rows * n->dims[l];
    Zw[l] = ws + o;
    o += (size_t)rows * n->dims[l + 1];
  }
  cudaStream_t st = (cudaStream_t)stream;
  normalize_kernel<<<grid1(rows * n->dims[0]), 256, 0, st>>>(rows, n->dims[0], x, n->in_mean, n->in_std, Aw[0]);
  for (int l = 0; l < kLayers; ++l) {
    const int din = n->dims[l], dout = n->dims[l + 1];
    gemm<false, true, __nv_bfloat16>((int)rows, dout, din, Aw[l], din, n->Wh[l], din, Zw[l], dout, st);
    const bool act = l < kLayers - 1;
    bias_act_kernel<<<grid1(rows * dout), 256, 0, st>>>(rows, dout, Zw[l], n->b[l], act ? Aw[l + 1] : nullptr,
                                                        act ? 1 : 0);
  }
  const int dlast = n->dims[kLayers];
  denorm_kernel<<<grid1(rows * dlast), 256, 0, st>>>(rows, dlast, Zw[kLayers - 1], n->out_mean, n->out_std, y);
  MLP_TRY(n, cudaGetLastError());
  return MOC_OK;
}
