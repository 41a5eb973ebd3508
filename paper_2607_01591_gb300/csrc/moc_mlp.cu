// Learned warm start: a 4-layer MLP (bf16 weights, FP32 accumulation, FP32 master weights, Adam)
// in hand-written CUDA kernels. The GEMMs of the forward and backward passes run on the tensor
// cores (tcgen05, moc_tc.cuh) with bias, SiLU and its derivative fused into their epilogues. See
// include/moc_mlp.h for the contract.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "moc_gb300.h"
#include "moc_mlp.h"
#include "moc_tc.cuh"

namespace {

constexpr int kLayers = 4;

__global__ void normalize_kernel(int64_t n, int d, const float *__restrict__ x, const float *__restrict__ mean,
                                 const float *__restrict__ sd, float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  const int j = (int)(i % d);
  out[i] = (x[i] - mean[j]) / sd[j];
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
  float *dZ = nullptr, *dZ2 = nullptr, *loss = nullptr;
  int *d_err = nullptr;  // set by a tensor-core GEMM whose wait ran out
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

// D = A B^T on the tensor cores (mlp_tc::tc_gemm_kernel): rows of D in tiles of 128, columns in
// tiles of 256, k split over blockIdx.y in chunks of k_per_cta (the atomic epilogue only)
template <int ASRC, int BSRC, int EPI> int tc_gemm(moc_mlp *n, mlp_tc::TcArgs g, cudaStream_t st) {
  auto kern = mlp_tc::tc_gemm_kernel<ASRC, BSRC, EPI>;
  // the kernel's shared-memory limit (a per-device function attribute; setting it allocates nothing)
  MLP_TRY(n, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mlp_tc::kSmemBytes));
  if (g.k_per_cta <= 0) g.k_per_cta = g.K;
  g.err = n->d_err;
  const dim3 grid((unsigned)((g.M + mlp_tc::kTileM - 1) / mlp_tc::kTileM),
                  (unsigned)((g.K + g.k_per_cta - 1) / g.k_per_cta),
                  (unsigned)((g.N + mlp_tc::kMaxN - 1) / mlp_tc::kMaxN));
  kern<<<grid, mlp_tc::kThreads, mlp_tc::kSmemBytes, st>>>(g);
  MLP_TRY(n, cudaGetLastError());
  return MOC_OK;
}

mlp_tc::TcArgs targs(int M, int N, int K, const void *a, int lda, const void *b, int ldb, float *out, int ldo) {
  mlp_tc::TcArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.a = a;
  g.lda = lda;
  g.b = b;
  g.ldb = ldb;
  g.out = out;
  g.ldo = ldo;
  return g;
}

// the four layers' GEMMs with fused epilogues: A_in [rows][dims[0]] (standardised) -> Z[l], A[l+1]
// (SiLU) -> ... -> Z[3]; y (may be null) gets the de-standardised output
int forward_layers(moc_mlp *n, float *const *Aw, float *const *Zw, int64_t rows, float *y, cudaStream_t st) {
  int rc = MOC_OK;
  for (int l = 0; l < kLayers && !rc; ++l) {
    const int din = n->dims[l], dout = n->dims[l + 1];
    mlp_tc::TcArgs g = targs((int)rows, dout, din, Aw[l], din, n->Wh[l], din, Zw[l], dout);
    g.bias = n->b[l];
    if (l < kLayers - 1) {
      g.out2 = Aw[l + 1];
      rc = tc_gemm<mlp_tc::SRC_F32, mlp_tc::SRC_BF16, mlp_tc::EPI_ACT>(n, g, st);
    } else {
      g.out2 = y;
      g.out_mean = n->out_mean;
      g.out_sd = n->out_std;
      rc = tc_gemm<mlp_tc::SRC_F32, mlp_tc::SRC_BF16, mlp_tc::EPI_LAST>(n, g, st);
    }
  }
  return rc;
}

int ensure_workspace(moc_mlp *n, int64_t rows) {
  if (rows <= n->cap) return MOC_OK;
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(n->Z[l]);
    cudaFree(n->A[l]);
    n->Z[l] = n->A[l] = nullptr;
  }
  cudaFree(n->dZ);
  cudaFree(n->dZ2);
  n->dZ = n->dZ2 = nullptr;
  int wmax = 0;
  for (int l = 0; l <= kLayers; ++l) wmax = std::max(wmax, n->dims[l]);
  for (int l = 0; l < kLayers; ++l) {
    MLP_TRY(n, cudaMalloc(&n->Z[l], (size_t)rows * n->dims[l + 1] * sizeof(float)));
    MLP_TRY(n, cudaMalloc(&n->A[l], (size_t)rows * n->dims[l] * sizeof(float)));
  }
  MLP_TRY(n, cudaMalloc(&n->dZ, (size_t)rows * wmax * sizeof(float)));
  MLP_TRY(n, cudaMalloc(&n->dZ2, (size_t)rows * wmax * sizeof(float)));
  n->cap = rows;
  return MOC_OK;
}

// forward pass into Z[3] (standardised outputs); keeps Z/A for the backward pass; y (may be null)
// gets the de-standardised outputs
int forward(moc_mlp *n, const float *x, int64_t rows, float *y, cudaStream_t st) {
  int rc = ensure_workspace(n, rows);
  if (rc) return rc;
  normalize_kernel<<<grid1(rows * n->dims[0]), 256, 0, st>>>(rows, n->dims[0], x, n->in_mean, n->in_std, n->A[0]);
  MLP_TRY(n, cudaGetLastError());
  return forward_layers(n, n->A, n->Z, rows, y, st);
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
    // gW[out][in] = sum_rows dZ[row][out] A[row][in], the rows split over CTAs in chunks of 2048
    mlp_tc::TcArgs g = targs(dout, din, (int)rows, dZ, dout, n->A[l], din, n->gW[l], din);
    g.k_per_cta = 2048;
    int rc = tc_gemm<mlp_tc::SRC_F32_T, mlp_tc::SRC_F32_T, mlp_tc::EPI_ATOMIC>(n, g, st);
    if (rc) return rc;
    dim3 g2((dout + 255) / 256, (unsigned)((rows + 2047) / 2048));
    colsum_kernel<<<g2, 256, 0, st>>>(rows, dout, dZ, n->gb[l], 2048);
    if (l > 0) {
      // dZ_prev[row][in] = (sum_out dZ[row][out] W[out][in]) SiLU'(Z_prev[row][in])
      mlp_tc::TcArgs h = targs((int)rows, din, dout, dZ, dout, n->Wh[l], din, dZn, din);
      h.aux = n->Z[l - 1];
      rc = tc_gemm<mlp_tc::SRC_F32, mlp_tc::SRC_BF16_T, mlp_tc::EPI_DACT>(n, h, st);
      if (rc) return rc;
      std::swap(dZ, dZn);
    }
  }
  MLP_TRY(n, cudaGetLastError());
  return MOC_OK;
}

// a tensor-core GEMM whose wait ran out (read at the calls that synchronise anyway)
int check_err(moc_mlp *n) {
  int e = 0;
  MLP_TRY(n, cudaMemcpy(&e, n->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) return mfail(n, MOC_ERR_CUDA, "tensor-core GEMM: a wait for the MMA ran out");
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
       cudaMalloc(&n->loss, 4) == cudaSuccess && cudaMalloc(&n->d_err, sizeof(int)) == cudaSuccess &&
       cudaMemset(n->d_err, 0, sizeof(int)) == cudaSuccess;
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
  cudaFree(n->dZ);
  cudaFree(n->dZ2);
  cudaFree(n->loss);
  cudaFree(n->d_err);
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
  return forward(n, x, rows, y, st);
}

int moc_mlp_train_step(moc_mlp *n, const float *x, const float *y, int64_t rows, float lr, float *loss_out,
                       void *stream) {
  if (!n || rows < 1 || !x || !y || !(lr > 0.f)) return MOC_ERR_ARG;
  cudaSetDevice(n->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = forward(n, x, rows, nullptr, st);
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
    return check_err(n);
  }
  return MOC_OK;
}

int moc_mlp_gradients(moc_mlp *n, const float *x, const float *y, int64_t rows, float *grad, float *loss_out,
                      void *stream) {
  if (!n || rows < 1 || !x || !y || !grad) return MOC_ERR_ARG;
  cudaSetDevice(n->device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = forward(n, x, rows, nullptr, st);
  if (!rc) rc = backward(n, y, rows, st);
  if (rc) return rc;
  MLP_TRY(n, cudaStreamSynchronize(st));
  if ((rc = check_err(n))) return rc;
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
  MLP_TRY(n, cudaGetLastError());
  return forward_layers(n, Aw, Zw, rows, y, st);
}
