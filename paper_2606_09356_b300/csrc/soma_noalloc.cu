// soma_noalloc.cu -- S(q) of caller-owned device positions without any
// device allocation.
//
// Who needs it: code that may not allocate GPU memory at the point where it
// wants a structure factor, for instance a caller whose device memory is
// handed out by a fixed arena or pool it must not bypass, a caller that runs
// where a cudaMalloc would synchronise the device (cudaMalloc/cudaFree can
// serialise with work in flight), or a caller that measures S(q) from inside a
// tight loop and cannot afford an allocation per call.  It does not need a
// soma handle either: it reads positions the caller already holds on the
// device.
//
// How: the per-q accumulators and the q list live in file-scope
// `static __device__` arrays of fixed size (kNoAllocMaxQ vectors), so every
// GPU that loads this library holds them until the process exits (about
// 112 KiB).  Host code cannot use the array names as device addresses; the
// device address of each array is looked up once per device with
// cudaGetSymbolAddress, on the first call made while that device is current.
// That first call therefore does host-side set-up and should be made before
// any stream capture begins.  All calls share the arrays: each call clears
// the accumulators before use, and two calls whose work overlaps on the GPU
// (different streams, no ordering between them) race on the same arrays.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/soma.h"
#include "soma_device.cuh"

namespace {

constexpr int kNoAllocMaxQ = 4096;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_sq_acc[kNoAllocMaxQ][2];   // sum of s_j cos, s_j sin
static __device__ __align__(256) int32_t g_sq_m[kNoAllocMaxQ][3];    // the q list, copied per call

struct NoAllocScratch {
  double* acc = nullptr;
  int32_t* m = nullptr;
  bool ready = false;
};

NoAllocScratch g_scratch[kNoAllocMaxDevices];
std::mutex g_scratch_mutex;

// Device addresses of the static arrays on the current device (set-up once).
int scratch_for_current_device(NoAllocScratch** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return SOMA_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  NoAllocScratch& s = g_scratch[dev];
  if (!s.ready) {
    void* acc = nullptr;
    void* m = nullptr;
    if (cudaGetSymbolAddress(&acc, g_sq_acc) != cudaSuccess || cudaGetSymbolAddress(&m, g_sq_m) != cudaSuccess) {
      cudaGetLastError();
      return SOMA_ECUDA;
    }
    s.acc = static_cast<double*>(acc);
    s.m = static_cast<int32_t*>(m);
    s.ready = true;
  }
  *out = &s;
  return SOMA_OK;
}

__global__ void k_sq_clear(double* __restrict__ acc, int nq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 2 * nq; i += gridDim.x * blockDim.x) acc[i] = 0.0;
}

// The handle's S(q) arithmetic (sq_accumulate in soma_device.cuh) on an
// array [n][3] of wrapped positions in logical bead order; every chain is the
// base diblock, beads 0 .. n_A-1 A and the rest B.
__global__ void k_sq_accumulate(const float* __restrict__ pos, int64_t n, int N, int n_A, float ilx, float ily,
                                float ilz, const int32_t* __restrict__ m, int nq, double* __restrict__ acc) {
  soma::sq_accumulate(
      n,
      [=](int64_t b, float& fx, float& fy, float& fz) {
        fx = pos[3 * b] * ilx;
        fy = pos[3 * b + 1] * ily;
        fz = pos[3 * b + 2] * ilz;
      },
      [=](int64_t b) { return ((int)(b % N) < n_A) ? 1.0 : -1.0; }, m, nq, acc);
}

__global__ void k_sq_finish(const double* __restrict__ acc, int nq, double inv_n, double* __restrict__ S) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x)
    S[q] = (acc[2 * q] * acc[2 * q] + acc[2 * q + 1] * acc[2 * q + 1]) * inv_n;
}

}  // namespace

extern "C" int soma_structure_factor_noalloc(const float* pos, int64_t n_beads, int32_t N, int32_t n_A,
                                             const double* box, int nq, const int32_t* m_xyz, double* S,
                                             void* stream) {
  if (nq == 0) return SOMA_OK;
  if (!pos || !box || !m_xyz || !S || n_beads < 1 || N < 1 || n_A < 0 || n_A > N || n_beads % N != 0)
    return SOMA_EINVAL;
  if (nq < 0 || nq > kNoAllocMaxQ) return SOMA_EINVAL;
  for (int a = 0; a < 3; ++a)
    if (!(box[a] > 0.0)) return SOMA_EINVAL;
  NoAllocScratch* sc = nullptr;
  int rc = scratch_for_current_device(&sc);
  if (rc) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SOMA_ECUDA;
  }
  if (cudaMemcpyAsync(sc->m, m_xyz, sizeof(int32_t) * 3 * (size_t)nq, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return SOMA_ECUDA;
  }
  k_sq_clear<<<(2 * nq + 255) / 256, 256, 0, s>>>(sc->acc, nq);
  k_sq_accumulate<<<sms * 4, 256, 0, s>>>(pos, n_beads, N, n_A, (float)(1.0 / box[0]), (float)(1.0 / box[1]),
                                          (float)(1.0 / box[2]), sc->m, nq, sc->acc);
  k_sq_finish<<<(nq + 255) / 256, 256, 0, s>>>(sc->acc, nq, 1.0 / (double)n_beads, S);
  if (cudaGetLastError() != cudaSuccess) return SOMA_ECUDA;
  return SOMA_OK;
}
