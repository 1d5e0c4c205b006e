// soma_launch.h -- host-side launchers of the kernels (internal to libsoma).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "soma_internal.cuh"

namespace soma {

// Kernel (a) with fused (b), soma_move.cu.
// warps: consumer warps per CTA of the single-system kernel, 8, 12 or 24.
cudaError_t launch_move(const MoveArgs& a, int grid, bool from_counts, StepRef r, cudaStream_t s, int warps);
cudaError_t launch_move_batch(const BatchArgs& p, int grid, StepRef r, cudaStream_t s);
int move_batch_max_ctas_per_sm(bool smart, bool wall);
// Block shapes of the one-system move kernel (consumer warps per CTA).
constexpr int kMoveShapes = 3;
constexpr int kMoveWarps[kMoveShapes] = {8, 12, 24};
// Index of a shape in kMoveWarps, -1 for no shape.
inline int move_shape(int warps) {
  for (int i = 0; i < kMoveShapes; ++i)
    if (kMoveWarps[i] == warps) return i;
  return -1;
}
// Resident CTAs per SM of a shape on the current device (0: it cannot run).
int move_kernel_max_ctas_per_sm(int warps);
int move_kernel_chains_per_tile(int P, int warps);
// The smart move's standard normal deviates of n words (verification aid).
cudaError_t launch_normal_words(const uint32_t* w, float* out, int64_t n, cudaStream_t s);
// One mbarrier wait that nothing satisfies, bounded by `cycles` (sets kErrTimeout in *err).
cudaError_t launch_wait_selfcheck(int* err, long long cycles, cudaStream_t s);
cudaError_t launch_move_generic(const SysDev* systems, int sys, int64_t n_poly, int N, StepRef r, int sm_count,
                                cudaStream_t s);
cudaError_t launch_bin(const SysDev* systems, int sys, int64_t n_b, StepRef r, int sm_count, cudaStream_t s);
cudaError_t launch_field(const FieldArgs& f, StepRef r, int zero_next, cudaStream_t s);
cudaError_t launch_deinterleave(const uint32_t* counts, int64_t n_c, uint32_t* out, int sm_count, cudaStream_t s);
cudaError_t launch_field_from_phi(const SysDev* systems, int sys, const float* phi, int sm_count, cudaStream_t s);
cudaError_t launch_advance(unsigned long long* counters, int n_sys, long long n, cudaStream_t s);
// Per-layer sums (nA, nB) of an interleaved count buffer along one axis:
// out [layers][2] (layers = the grid size along `axis`).
cudaError_t launch_profile(const uint32_t* counts, int nx, int ny, int nz, int axis, unsigned long long* out,
                           cudaStream_t s);
// Placement from target volume fractions phi [2][n_c] (device); q and prefix
// hold n_c 64-bit words each; *total receives the weight sum (0: nothing
// placed).  Synchronises the stream once.
cudaError_t launch_place(const SysDev* systems, int sys, const SysDev& host, const float* phi,
                         unsigned long long* q, unsigned long long* prefix, void* temp, size_t temp_bytes,
                         unsigned long long* total, int sm_count, cudaStream_t s);
size_t place_temp_bytes(int64_t n_c);
// Vertical pair sums of an interleaved count buffer (type `type`): out
// [nz + 1][4] = (sum a b, sum a, sum b, pairs) per dz, then (sum n^2,
// sum n, -, cells).
cudaError_t launch_vcorr(const uint32_t* counts, int64_t n_c, int nz, int type, int wall, unsigned long long* out,
                         cudaStream_t s);
cudaError_t launch_set_step(unsigned long long* counters, int n_sys, unsigned long long value, cudaStream_t s);
cudaError_t launch_init(const SysDev* systems, int sys, int64_t n_poly, cudaStream_t s);
cudaError_t launch_gather_state(const SysDev* systems, int sys, float* pos, int16_t* img, int sm_count,
                                cudaStream_t s);
cudaError_t launch_scatter_state(const SysDev* systems, int sys, const float* pos, const int16_t* img,
                                 int sm_count, cudaStream_t s);
cudaError_t launch_validate(const SysDev* systems, int sys, int* err, int sm_count, cudaStream_t s);
cudaError_t launch_validate_pos(const float* pos, int64_t n, const float* L, int* err, int sm_count,
                                cudaStream_t s);
cudaError_t launch_sum_acc(const SysDev* systems, int sys, unsigned long long* out, cudaStream_t s);
cudaError_t launch_zero_acc(const SysDev* systems, int sys, cudaStream_t s);
cudaError_t launch_observables(const SysDev* systems, int sys, long long t_done, double* out,
                               unsigned long long* acc_out, int sm_count, cudaStream_t s);
cudaError_t launch_structure_factor(const SysDev* systems, int sys, int nq, const int32_t* m, double* out,
                                    int sm_count, cudaStream_t s);

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, cudaStream_t s);

// FP64-position form (soma_f64.cu).
cudaError_t launch_move64(const SysDev* systems, int sys, StepRef r, int sm_count, cudaStream_t s);
cudaError_t launch_init64(const SysDev* systems, int sys, int64_t n_poly, cudaStream_t s);
cudaError_t launch_get_types(const SysDev* systems, int sys, uint8_t* out, int sm_count, cudaStream_t s);
cudaError_t launch_set_types(const SysDev* systems, int sys, const uint8_t* types, int sm_count, cudaStream_t s);
cudaError_t launch_bin64(const SysDev* systems, int sys, long long t, int sm_count, cudaStream_t s);
cudaError_t launch_gather_state64(const SysDev* systems, int sys, double* pos, int16_t* img, int sm_count,
                                  cudaStream_t s);
cudaError_t launch_scatter_state64(const SysDev* systems, int sys, const double* pos, const int16_t* img,
                                   int sm_count, cudaStream_t s);
cudaError_t launch_validate_pos64(const double* pos, int64_t n, const double* L, int* err, int sm_count,
                                  cudaStream_t s);
cudaError_t launch_obs_chains64(const SysDev* systems, int sys, double* out, int sm_count, cudaStream_t s);
cudaError_t launch_structure_factor64(const SysDev* systems, int sys, int nq, const int32_t* m, double* out,
                                      int sm_count, cudaStream_t s);

// Chain reorder (soma_sort.cu): sort the chains of every system by the
// Morton key of their first bead's position, permute positions, images and
// chain ids into the alternate buffers and copy them back, so the arrays
// keep their addresses.
struct SortWork {
  unsigned long long* keys_in;
  unsigned long long* keys_out;
  uint32_t* vals_in;
  uint32_t* vals_out;
  void* temp;
  size_t temp_bytes;
  int32_t* chain_sys;  // global chain -> system
  int64_t n_chains;
  int end_bit;
};
size_t sort_temp_bytes(int64_t n_chains, int end_bit);

// Prefix sums and the stable radix sort (soma_scan.cu).  The scans take
// scratch of scan_temp_bytes_u64(n) bytes; out may be in.
size_t scan_temp_bytes_u64(int64_t n);
cudaError_t launch_scan_u64(const unsigned long long* in, unsigned long long* out, int64_t n, bool inclusive,
                            void* temp, cudaStream_t s);
// Sort n (key, value) pairs by the key's bits [0, end_bit), stably; a and b
// are ping-pong buffers (the input in a), *in_b says where the result is.
size_t radix_sort_temp_bytes(int64_t n);
cudaError_t launch_radix_sort_pairs(unsigned long long* keys_a, unsigned long long* keys_b, uint32_t* vals_a,
                                    uint32_t* vals_b, int64_t n, int end_bit, void* temp, bool* in_b,
                                    cudaStream_t s);
cudaError_t launch_reorder(SysDev* systems, int n_sys, const SortWork& w, int sm_count, cudaStream_t s);

}  // namespace soma
