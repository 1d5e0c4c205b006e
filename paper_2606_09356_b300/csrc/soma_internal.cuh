// soma_internal.cuh -- device-side layout shared by the kernels and the host
// code of libsoma.  Nothing here is part of the C ABI (include/soma.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace soma {

constexpr uint32_t kInitStep = 0xFFFFFFFFu;  // Philox step word reserved for init

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
  uint32_t* counts;             // [2 buffers][2 types][n_c]
  float* w;                     // [2 types][n_c]
  unsigned long long* acc;      // accepted moves, one counter per move tile
  int32_t acc_first, acc_count; // this system's range of move tiles
  int64_t chain_base;           // first chain of this system in the global chain order
};

// Everything the move kernel needs for one system, passed by value as a
// __grid_constant__ kernel parameter (constant bank: no loads in the loop).
struct MoveArgs {
  float L[3], invL[3], cps[3];
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
  const uint32_t* chain_id;
  uint32_t* counts;          // [2 buffers][2 types][n_c]
  const float* w;            // [2 types][n_c]
  unsigned long long* acc;   // one accepted-move slot per CTA of this system
  const unsigned long long* step_base;
  int* err;
};

// The field kernel's view of one system (also by value).
struct FieldArgs {
  uint32_t* counts;          // [2 buffers][2 types][n_c]
  float* w;                  // [2 types][n_c]
  int64_t n_c;
  float inv_rho, chiN_N, kappaN_N;
  int32_t frozen;
  const unsigned long long* step_base;
};

// Device error word bits.
constexpr int kErrBounds = 1;
constexpr int kErrTimeout = 2;

}  // namespace soma
