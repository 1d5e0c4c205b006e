// soma_sort.cu -- periodic chain reorder.
//
// Chains are sorted by the Morton (Z-order) key of their first bead's
// position, quantised to 1024 steps per box edge, so that chains stored
// next to each other sit next to each other in space: the field gathers of
// the move kernel and the count atomics of the histogram then touch compact,
// cache-resident cell ranges.  The random numbers follow the logical chain id
// carried along in chain_id, so a reorder never changes the trajectory.
// The sort is the library's own stable radix sort (soma_scan.cu); keys,
// permutation and copy-back are kernels of this file.
#include <cuda_runtime.h>

#include "soma_launch.h"

namespace soma {

__device__ __forceinline__ unsigned long long spread3(uint32_t v) {
  unsigned long long x = v & 0x3FFu;
  x = (x | (x << 16)) & 0x030000FFull;
  x = (x | (x << 8)) & 0x0300F00Full;
  x = (x | (x << 4)) & 0x030C30C3ull;
  x = (x | (x << 2)) & 0x09249249ull;
  return x;
}

__device__ __forceinline__ uint32_t quant1024(float x, float invL) {
  int q = (int)(x * invL * 1024.f);
  return (uint32_t)(q < 0 ? 0 : (q > 1023 ? 1023 : q));
}

__global__ void k_sort_keys(const SysDev* __restrict__ systems, const int32_t* __restrict__ chain_sys,
                            int64_t n_chains, unsigned long long* __restrict__ keys, uint32_t* __restrict__ vals) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n_chains; g += (int64_t)gridDim.x * blockDim.x) {
    const int s = chain_sys[g];
    const SysDev& S = systems[s];
    const int64_t b = (g - S.chain_base) * S.N;
    const uint32_t qx = quant1024(S.x[b], S.invL[0]);
    const uint32_t qy = quant1024(S.y[b], S.invL[1]);
    const uint32_t qz = quant1024(S.z[b], S.invL[2]);
    // 30 bits of Morton key, the system above them: a sort over 30 + log2(systems) bits
    keys[g] = ((unsigned long long)s << 30) | (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
    vals[g] = (uint32_t)g;
  }
}

// One warp per chain in the new order: copy its beads from the old slot.
__global__ void k_permute(const SysDev* __restrict__ systems, const int32_t* __restrict__ chain_sys,
                          int64_t n_chains, const uint32_t* __restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_chains; j += warps) {
    const int s = chain_sys[j];
    const SysDev& S = systems[s];
    const int64_t old_slot = (int64_t)perm[j] - S.chain_base, new_slot = j - S.chain_base;
    const int N = S.N;
    for (int i = lane; i < N; i += 32) {
      const int64_t src = old_slot * N + i, dst = new_slot * N + i;
      S.x_alt[dst] = S.x[src];
      S.y_alt[dst] = S.y[src];
      S.z_alt[dst] = S.z[src];
      reinterpret_cast<short4*>(S.img_alt)[dst] = reinterpret_cast<const short4*>(S.img)[src];
    }
    if (lane == 0) S.chain_id_alt[new_slot] = S.chain_id[old_slot];
  }
}

// Copy the permuted chains back from the alternate buffers.
__global__ void k_copy_back(const SysDev* __restrict__ systems, const int32_t* __restrict__ chain_sys,
                            int64_t n_chains) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t j = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < n_chains; j += warps) {
    const SysDev& S = systems[chain_sys[j]];
    const int64_t slot = j - S.chain_base;
    const int N = S.N;
    for (int i = lane; i < N; i += 32) {
      const int64_t b = slot * N + i;
      S.x[b] = S.x_alt[b];
      S.y[b] = S.y_alt[b];
      S.z[b] = S.z_alt[b];
      reinterpret_cast<short4*>(S.img)[b] = reinterpret_cast<const short4*>(S.img_alt)[b];
    }
    if (lane == 0) S.chain_id[slot] = S.chain_id_alt[slot];
  }
}

size_t sort_temp_bytes(int64_t n_chains, int end_bit) {
  (void)end_bit;
  return radix_sort_temp_bytes(n_chains);
}

cudaError_t launch_reorder(SysDev* systems, int n_sys, const SortWork& w, int sm_count, cudaStream_t s) {
  const int blocks = sm_count * 8;
  k_sort_keys<<<blocks, 256, 0, s>>>(systems, w.chain_sys, w.n_chains, w.keys_in, w.vals_in);
  bool in_b = false;
  cudaError_t e = launch_radix_sort_pairs(w.keys_in, w.keys_out, w.vals_in, w.vals_out, w.n_chains, w.end_bit, w.temp,
                                          &in_b, s);
  if (e != cudaSuccess) return e;
  k_permute<<<blocks, 256, 0, s>>>(systems, w.chain_sys, w.n_chains, in_b ? w.vals_out : w.vals_in);
  k_copy_back<<<blocks, 256, 0, s>>>(systems, w.chain_sys, w.n_chains);
  return cudaGetLastError();
}

}  // namespace soma
