// soma_internal.cuh -- device-side layout shared by the kernels and the host
// code of libsoma.  Nothing here is part of the C ABI (include/soma.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace soma {

constexpr uint32_t kInitStep = 0xFFFFFFFFu;  // Philox step word reserved for init

// Molecule types (boundary-zone conversion): the top bit of a chain-id word
// is the chain's molecule type (1: converted), the rest its logical id.
constexpr uint32_t kTypeBit = 0x80000000u;
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr uint32_t kConvWord = 0xFFFFFFFFu;  // Philox bead word of the conversion draw (no bead has it)

// Per-system constants and array pointers, one entry per system in a device
// array.  Kernels copy their system's entry into shared memory.
struct alignas(16) SysDev {
  int32_t n_poly, N, n_A, P;  // P: lanes per chain in the register kernel (0 = generic)
  int32_t nx, ny, nz, sys_index;
  int64_t n_b, n_c;
  float L[3], invL[3], cps[3];  // box edge, 1/L, cells per unit length n/L
  float A, kb;                  // proposal half-width, bond constant 3(N-1)/2
  float chiN_N, kappaN_N, inv_rho;
  int32_t frozen;               // 1: fields are held (not rebuilt from counts)
  uint32_t rk[10][2];           // Philox round keys (seed lo/hi bumped per round)
  float* x;                     // wrapped positions, SoA, [n_b]
  float* y;
  float* z;
  int16_t* img;                 // images [n_b][4] (x, y, z, unused)
  uint32_t* chain_id;           // storage slot -> logical chain id [n_poly]
  float* x_alt;                 // second position set (reorder target, staging)
  float* y_alt;
  float* z_alt;
  int16_t* img_alt;
  uint32_t* chain_id_alt;
  uint32_t* counts;             // [3 buffers][n_c][2 types], see count_buffer()
  float* w;                     // [2 types][n_c]
  unsigned long long* acc;      // accepted moves, one counter per move tile
  int32_t acc_first, acc_count; // this system's range of accepted-move slots
  int64_t chain_base;           // first chain of this system in the global chain order
  uint32_t id_base;             // logical id of this handle's first chain (a chain partition; else 0)
  int32_t pad_id;
  double rho_bar;               // beads per cell of the whole system (a partition holds only its share)
  // FP64-position form (precision reference): wrapped FP64 positions
  double* x64;
  double* y64;
  double* z64;
  double L64[3];
  double invL64[3], cps64[3];  // 1/L and n/L in FP64
  double chiN64, kappaN64;
  // umbrella restraint toward target volume fractions (coupling start-up):
  // w_t += umbN_N (phi_t - phi*_t) with umbN_N = lambdaN / N
  float* phi_target;            // [2 types][n_c], allocated on first use
  float umbN_N;
  int32_t umbrella;             // 1: the restraint is on
  int32_t wall_z;               // 1: hard walls at z = 0 and z = L_z (z not periodic)
  // molecule types and boundary-zone conversion (the types ride in chain_id's top bit)
  int32_t conv;                 // 1: types honoured, conversion draws open every step
  int32_t n_A_alt;              // A beads of a converted (type-1) molecule
  float zone_lo, zone_hi;       // bottom zone: z < zone_lo; top zone: z >= zone_hi (FP32)
  unsigned long long thr[4];    // convert iff word < thr: {bottom 0->1, bottom 1->0, top 0->1, top 1->0}
  unsigned long long* conv_count;  // [4] conversions since the rates were last set
};

// Everything the move kernel needs for one system, passed by value as a
// __grid_constant__ kernel parameter (constant bank: no loads in the loop).
struct MoveArgs {
  float L[3], invL[3], cps[3];
  float Lm[3];               // largest float below L
  int32_t smart;             // 1: bond-force-biased proposals (host-side flag; kernels are templated)
  int32_t n[3];
  float A, kb;
  uint32_t rk[10][2];        // Philox round keys
  int32_t N, n_A, P, sys_index;
  int32_t n_poly, chains_per_tile, n_tiles, bin;
  int64_t n_c;
  float* x;
  float* y;
  float* z;
  int16_t* img;
  uint32_t* chain_id;        // read by the bulk copies; a converted chain's word is rewritten
  uint32_t* counts;          // [3 buffers][n_c][2 types]
  const float* w;            // [2 types][n_c], read only when fields are held
  float inv_rho, chiN_N, kappaN_N;
  int32_t from_counts;       // batched launches: 1 = fields from counts, 0 = field array
  unsigned long long* acc;   // accepted-move slots of this system, one per CTA of a launch
  int* err;
  // bond-force-biased proposal d = -drift s + sig xi, s the sum of the bead's
  // bond vectors, xi standard normal; s2 = A^2/3, drift = s2 k_b, sig = sqrt(s2)
  float sig, drift, inv2s2;  // inv2s2 = 1 / (2 s2)
  int32_t wall_z;            // 1: hard walls at z = 0 and z = L_z (host-side flag; kernels are templated)
  int32_t conv;              // 1: molecule types in chain_id's top bit (single launches: templated)
  int32_t n_A_alt;           // A beads of a converted molecule
  float zone_lo, zone_hi;    // conversion zones: bottom z < zone_lo, top z >= zone_hi
  unsigned long long thr[4]; // convert iff word < thr: {bottom 0->1, bottom 1->0, top 0->1, top 1->0}
  unsigned long long* conv_count;  // [4] conversions since the rates were last set
};

// Up to kMaxBatch systems stepped by one persistent launch: their constants
// and the first global tile of each (tile_start[n_sys] = total tiles).
constexpr int kMaxBatch = 64;
struct BatchArgs {
  int32_t n_sys;
  int32_t tile_start[kMaxBatch + 1];
  int32_t pad[2];
  MoveArgs sys[kMaxBatch];
};

// Which step a launch performs: a number the host fixes (plain launches) or
// a device counter plus an offset (CUDA-graph replays, where the same nodes
// run again and again; the graph's last node advances the counter).
struct StepRef {
  const unsigned long long* counter;
  long long fixed;
  int32_t use_counter;
  int32_t offset;
#ifdef __CUDACC__
  __device__ __forceinline__ long long get() const {
    return use_counter ? (long long)*counter + offset : fixed;
  }
#endif
};

// The field kernel's view of one system (also by value).
struct FieldArgs {
  uint32_t* counts;          // [3 buffers][n_c][2 types]
  float* w;                  // [2 types][n_c]
  int64_t n_c;
  float inv_rho, chiN_N, kappaN_N;
  int32_t frozen;
  const float* target;       // [2 types][n_c] umbrella target (read when umbrella = 1)
  float umbN_N;
  int32_t umbrella;
};

// Count buffers: three per system, each [n_c][2] (the two types of a cell
// side by side, so one 8-byte load serves a cell).  Step t accumulates buffer
// t mod 3, takes the previous step's counts (its fields) from (t - 1) mod 3
// and clears (t + 1) mod 3 for the next step, so the three roles never
// overlap within a step.  t may be -1 (the configuration before step 0).
__host__ __device__ inline int count_buffer_index(long long t) { return (int)(((t % 3) + 3) % 3); }
__host__ __device__ inline uint32_t* count_buffer(uint32_t* base, int64_t n_c, long long t) {
  return base + (size_t)count_buffer_index(t) * 2 * (size_t)n_c;
}

// Device error word bits.
constexpr int kErrBounds = 1;
constexpr int kErrTimeout = 2;

}  // namespace soma
