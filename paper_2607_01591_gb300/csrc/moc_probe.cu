// Hardware rate probes (include/moc_probe.h): FP32/FP64 FMA issue rates and L2 atomic rates for
// the access shapes the sweep kernels use. Fixed, bounded work per launch; no waits.
#include <cuda_runtime.h>

#include <cstdint>

#include "moc_gb300.h"
#include "moc_probe.h"

namespace {

constexpr int kThreads = 256;
constexpr int kFmaChains = 8;
constexpr int kFmaIters = 2048;   // FP32: 8 x 2048 FMAs per thread
constexpr int kDfmaIters = 48;    // FP64: 8 x 48 per thread (GB300's FP64 rate is far lower)
constexpr int kAtomIters = 512;   // atomics per thread
constexpr uint32_t kL2Sectors = (64u << 20) / 32;    // 64 MiB buffer
constexpr uint32_t kHbmSectors = 1u << 27;              // 4 GiB buffer (2^27 sectors of 32 bytes)

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_probe(T b, T c, T *out, int iters) {
  T a[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) a[k] = (T)(threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += a[k];
  // never true for the probe's arguments; keeps the chains live
  if (s == (T)-1.2345) out[0] = s;
}

// a pseudo-random sector for (unit, iteration): an integer mix of the two, masked to the buffer
__device__ __forceinline__ uint32_t sector_of(uint32_t unit, uint32_t it, uint32_t mask) {
  uint32_t x = unit * 0x9E3779B1u ^ (it * 0x85EBCA77u + 0x165667B1u);
  x ^= x >> 15;
  x *= 0x2C1B3C6Du;
  x ^= x >> 12;
  x *= 0x297A2D39u;
  x ^= x >> 15;
  return x & mask;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) atom_probe(float *buf, uint32_t mask, float v, float *out) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  for (int it = 0; it < kAtomIters; ++it) {
    if (KIND == MOC_PROBE_RED_F32) {
      atomicAdd(buf + (size_t)sector_of(tid, it, mask) * 8, v);
    } else if (KIND == MOC_PROBE_RED_F32X2) {
      atomicAdd(reinterpret_cast<float2 *>(buf) + (size_t)sector_of(tid, it, mask) * 4, make_float2(v, v));
    } else if (KIND == MOC_PROBE_RED_F32X4 || KIND == MOC_PROBE_RED_F32X4_HBM) {
      atomicAdd(reinterpret_cast<float4 *>(buf) + (size_t)sector_of(tid, it, mask) * 2, make_float4(v, v, v, v));
    } else if (KIND == MOC_PROBE_RED_F32X4_PAIR) {
      atomicAdd(reinterpret_cast<float4 *>(buf) + (size_t)sector_of(tid >> 1, it, mask) * 2 + (tid & 1),
                make_float4(v, v, v, v));
    } else if (KIND == MOC_PROBE_RED_F32_ROW8) {
      atomicAdd(buf + (size_t)sector_of(tid >> 3, it, mask) * 8 + (tid & 7), v);
    } else if (KIND == MOC_PROBE_ATOM_F32) {
      acc += atomicAdd(buf + (size_t)sector_of(tid, it, mask) * 8, v);
    } else if (KIND == MOC_PROBE_RED_F64) {
      atomicAdd(reinterpret_cast<double *>(buf) + (size_t)sector_of(tid, it, mask) * 4, (double)v);
    }
  }
  if (KIND == MOC_PROBE_ATOM_F32 && acc == -1.2345f) out[0] = acc;
}

struct Ev {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Ev() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

template <typename F> int time_best(cudaStream_t st, F launch, float *best_ms) {
  Ev ev;
  if (cudaEventCreate(&ev.a) != cudaSuccess || cudaEventCreate(&ev.b) != cudaSuccess) return MOC_ERR_CUDA;
  launch();  // warm-up
  if (cudaGetLastError() != cudaSuccess) return MOC_ERR_CUDA;
  float best = 1e30f;
  for (int r = 0; r < 3; ++r) {
    cudaEventRecord(ev.a, st);
    launch();
    cudaEventRecord(ev.b, st);
    if (cudaEventSynchronize(ev.b) != cudaSuccess) return MOC_ERR_CUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev.a, ev.b);
    if (ms < best) best = ms;
  }
  *best_ms = best;
  return cudaGetLastError() == cudaSuccess ? MOC_OK : MOC_ERR_CUDA;
}

template <int KIND> void launch_atom(cudaStream_t st, int blocks, float *buf, uint32_t mask, float *out) {
  atom_probe<KIND><<<blocks, kThreads, 0, st>>>(buf, mask, 1e-7f, out);
}

}  // namespace

extern "C" int moc_probe_rate(int device, int kind, double *lane_ops_per_s, double *sectors_per_s, int *sm_count) {
  if (kind < 0 || kind >= MOC_PROBE_COUNT) return MOC_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MOC_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return MOC_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return MOC_ERR_CUDA;
  if (sm_count) *sm_count = sms;
  cudaStream_t st = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return MOC_ERR_CUDA;
  const bool hbm = kind == MOC_PROBE_RED_F32X4_HBM;
  const bool fmak = kind == MOC_PROBE_FFMA || kind == MOC_PROBE_DFMA;
  const size_t bytes = fmak ? 64 : (size_t)(hbm ? kHbmSectors : kL2Sectors) * 32;
  void *buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, bytes);
  if (e != cudaSuccess) {
    cudaStreamDestroy(st);
    return e == cudaErrorMemoryAllocation ? MOC_ERR_OOM : MOC_ERR_CUDA;
  }
  int rc = MOC_OK;
  float ms = 0.f;
  double lane_ops = 0.0, sectors = 0.0;
  if (cudaMemsetAsync(buf, 0, bytes, st) != cudaSuccess) rc = MOC_ERR_CUDA;
  float *out = (float *)buf;
  if (!rc && kind == MOC_PROBE_FFMA) {
    const int blocks = sms * 8;
    rc = time_best(st, [&] { fma_probe<float><<<blocks, kThreads, 0, st>>>(0.999f, 1e-3f, out, kFmaIters); }, &ms);
    lane_ops = (double)blocks * kThreads * kFmaChains * kFmaIters;
  } else if (!rc && kind == MOC_PROBE_DFMA) {
    const int blocks = sms * 8;
    rc = time_best(st, [&] { fma_probe<double><<<blocks, kThreads, 0, st>>>(0.999, 1e-3, (double *)buf, kDfmaIters); },
                   &ms);
    lane_ops = (double)blocks * kThreads * kFmaChains * kDfmaIters;
  } else if (!rc) {
    const int blocks = sms * 16;
    const uint32_t mask = (hbm ? kHbmSectors : kL2Sectors) - 1;
    float *fb = (float *)buf;
    auto go = [&] {
      switch (kind) {
        case MOC_PROBE_RED_F32: launch_atom<MOC_PROBE_RED_F32>(st, blocks, fb, mask, out); break;
        case MOC_PROBE_RED_F32X2: launch_atom<MOC_PROBE_RED_F32X2>(st, blocks, fb, mask, out); break;
        case MOC_PROBE_RED_F32X4: launch_atom<MOC_PROBE_RED_F32X4>(st, blocks, fb, mask, out); break;
        case MOC_PROBE_RED_F32X4_PAIR: launch_atom<MOC_PROBE_RED_F32X4_PAIR>(st, blocks, fb, mask, out); break;
        case MOC_PROBE_RED_F32_ROW8: launch_atom<MOC_PROBE_RED_F32_ROW8>(st, blocks, fb, mask, out); break;
        case MOC_PROBE_ATOM_F32: launch_atom<MOC_PROBE_ATOM_F32>(st, blocks, fb, mask, out); break;
        case MOC_PROBE_RED_F64: launch_atom<MOC_PROBE_RED_F64>(st, blocks, fb, mask, out); break;
        default: launch_atom<MOC_PROBE_RED_F32X4_HBM>(st, blocks, fb, mask, out); break;
      }
    };
    rc = time_best(st, go, &ms);
    lane_ops = (double)blocks * kThreads * kAtomIters;
    const double per = kind == MOC_PROBE_RED_F32X4_PAIR ? 0.5 : kind == MOC_PROBE_RED_F32_ROW8 ? 0.125 : 1.0;
    sectors = lane_ops * per;
  }
  cudaStreamSynchronize(st);
  cudaFree(buf);
  cudaStreamDestroy(st);
  if (rc) return rc;
  const double s = ms * 1e-3;
  if (lane_ops_per_s) *lane_ops_per_s = s > 0 ? lane_ops / s : 0.0;
  if (sectors_per_s) *sectors_per_s = s > 0 ? sectors / s : 0.0;
  return MOC_OK;
}
