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

// A CTA's share of the move kernel: consecutive storage slots of one system.
struct MoveTile {
  int32_t sys;
  int32_t first_chain;
  int32_t n_chains;
  int32_t acc_index;
};

// A CTA's share of a per-cell kernel: cells [begin, end) of one system.
struct CellTile {
  int32_t sys;
  int32_t pad;
  int64_t begin, end;
};

// Device error word bits.
constexpr int kErrBounds = 1;
constexpr int kErrTimeout = 2;

}  // namespace soma
