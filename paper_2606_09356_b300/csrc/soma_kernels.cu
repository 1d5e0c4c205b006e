// soma_kernels.cu -- sm_103a kernels of the SCMF Monte Carlo step.
//
// (a) the register/TMA move kernel lives in soma_move.cu; this file holds
//     the generic move path for chains longer than 64 beads.
// (b) k_bin: stand-alone density histogram (the density-field update of
//     Sec. 2.2), used at start-up, after a restore and with the generic path.
// (c) k_field: per-cell field array from the counts (the register move kernel
//     evaluates the same fields from the counts on the fly; this kernel
//     serves the generic path and requests for the field array).
// plus initialisation, placement from target fields and the umbrella
// restraint's field array (Sec. 3.2), molecule types of the boundary-zone
// conversion (read and set; the conversion itself runs in the move kernel),
// state gather/scatter, validation, layer profiles, vertical correlations,
// observables and S(q).
//
// Layout (per system, see soma_internal.cuh): positions as three FP32 arrays
// x, y, z [n_b] wrapped into [0, L), bead = slot * N + i; images int16
// [n_b][4]; counts uint32 [3 buffers][n_c][2 types]; fields FP32 [2][n_c].
#include <cuda_runtime.h>
#include <cstdint>

#include <algorithm>

#include "soma_device.cuh"
#include "soma_internal.cuh"
#include "soma_launch.h"

namespace soma {

// ---------------------------------------------------------------------------
// Generic move of one set for chains longer than 64 beads: one thread per
// bead of the set, neighbours read from global memory (they belong to the
// other set, so they do not change during this launch).  The histogram runs
// as the separate kernel k_bin afterwards.
// ---------------------------------------------------------------------------
__global__ void k_move_set_generic(const SysDev* __restrict__ systems, int sys, StepRef r, int set) {
  __shared__ SysDev S;
  __shared__ unsigned int s_acc;
  if (threadIdx.x == 0) s_acc = 0;
  load_sys(&S, systems + sys);
  const uint32_t t = (uint32_t)r.get();
  const int N = S.N;
  const int per_chain = (N - set + 1) / 2;
  const int64_t total = (int64_t)S.n_poly * per_chain;
  int nacc = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < total;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int slot = (int)(j / per_chain);
    const int i = set + 2 * (int)(j % per_chain);
    const int64_t b = (int64_t)slot * N + i;
    float x = S.x[b], y = S.y[b], z = S.z[b];
    const bool ha = i > 0, hb = i + 1 < N;
    const float ax = ha ? S.x[b - 1] : 0.f, ay = ha ? S.y[b - 1] : 0.f, az = ha ? S.z[b - 1] : 0.f;
    const float bx = hb ? S.x[b + 1] : 0.f, by = hb ? S.y[b + 1] : 0.f, bz = hb ? S.z[b + 1] : 0.f;
    int cell = cell_of(S, x, y, z), wrap = 21;
    const float* wt = S.w + (i < S.n_A ? 0 : S.n_c);
    const int ok = try_move(S, wt, (uint32_t)i, S.chain_id[slot] & kIdMask, t, x, y, z, cell, wrap, ax, ay, az,
                            ha ? 1.f : 0.f, bx, by, bz, hb ? 1.f : 0.f);
    if (ok) {
      S.x[b] = x; S.y[b] = y; S.z[b] = z;
      apply_wrap(S.img, b, wrap);
    }
    nacc += ok;
  }
  nacc = __reduce_add_sync(0xffffffffu, nacc);
  if ((threadIdx.x & 31) == 0 && nacc) atomicAdd(&s_acc, (unsigned)nacc);
  __syncthreads();
  if (threadIdx.x == 0 && s_acc) atomicAdd(S.acc + S.acc_first, (unsigned long long)s_acc);
}

// ---------------------------------------------------------------------------
// (b) Stand-alone histogram of the current positions into count buffer t mod 3
// (used at start-up, after a state restore and for chains the register move
// kernel does not cover).  One thread per bead, one global atomic each.
// ---------------------------------------------------------------------------
__global__ void k_bin(const SysDev* __restrict__ systems, int sys, StepRef r) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  uint32_t* cnt = count_buffer(S.counts, S.n_c, r.get());
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(b % S.N);
    atomicAdd(cnt + 2 * cell_of(S, S.x[b], S.y[b], S.z[b]) + (i < chain_n_A(S, b / S.N) ? 0 : 1), 1u);
  }
}

// ---------------------------------------------------------------------------
// (c) Field array from count buffer t mod 3:  phi_t = n_t / rho_bar,
//   w_A = chiN/N phi_B + kappaN/N (phi_A + phi_B - 1), w_B = chiN/N phi_A + ...
// optionally clearing buffer t+1 mod 3 for the next step.  Held (frozen)
// fields are not overwritten.  One system per launch, two cells per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void field_pair(const FieldArgs& f, uint32_t nA, uint32_t nB, float& wA, float& wB) {
  const float pA = (float)nA * f.inv_rho, pB = (float)nB * f.inv_rho;
  const float ex = f.kappaN_N * (pA + pB - 1.f);
  wA = fmaf(f.chiN_N, pB, ex);
  wB = fmaf(f.chiN_N, pA, ex);
}

// The umbrella restraint's share, umbN_N (phi_t - phi*_t), of a cell's fields.
__device__ __forceinline__ void umbrella_pair(const FieldArgs& f, uint32_t nA, uint32_t nB, float tA, float tB,
                                              float& wA, float& wB) {
  wA = fmaf(f.umbN_N, fmaf((float)nA, f.inv_rho, -tA), wA);
  wB = fmaf(f.umbN_N, fmaf((float)nB, f.inv_rho, -tB), wB);
}

__global__ void __launch_bounds__(256) k_field(const __grid_constant__ FieldArgs f, StepRef r, int zero_next) {
  const long long t = r.get();
  const int64_t nc = f.n_c;
  const uint32_t* __restrict__ cur = count_buffer(f.counts, nc, t);
  uint32_t* __restrict__ nxt = count_buffer(f.counts, nc, t + 1);
  float* __restrict__ w = f.w;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  if ((nc & 1) == 0) {
    const int64_t n2 = nc >> 1;  // pairs of cells
    const uint4* cur4 = reinterpret_cast<const uint4*>(cur);
    uint4* nxt4 = reinterpret_cast<uint4*>(nxt);
    float2* wa2 = reinterpret_cast<float2*>(w);
    float2* wb2 = reinterpret_cast<float2*>(w + nc);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
      const uint4 c = __ldg(cur4 + i);  // (nA, nB) of cells 2i and 2i+1
      if (!f.frozen) {
        float2 wa, wb;
        field_pair(f, c.x, c.y, wa.x, wb.x);
        field_pair(f, c.z, c.w, wa.y, wb.y);
        if (f.umbrella) {
          const float2 ta = __ldg(reinterpret_cast<const float2*>(f.target) + i);
          const float2 tb = __ldg(reinterpret_cast<const float2*>(f.target + nc) + i);
          umbrella_pair(f, c.x, c.y, ta.x, tb.x, wa.x, wb.x);
          umbrella_pair(f, c.z, c.w, ta.y, tb.y, wa.y, wb.y);
        }
        wa2[i] = wa;
        wb2[i] = wb;
      }
      if (zero_next) nxt4[i] = make_uint4(0, 0, 0, 0);
    }
  } else {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += stride) {
      if (!f.frozen) {
        float wa, wb;
        field_pair(f, cur[2 * c], cur[2 * c + 1], wa, wb);
        if (f.umbrella) umbrella_pair(f, cur[2 * c], cur[2 * c + 1], f.target[c], f.target[nc + c], wa, wb);
        w[c] = wa;
        w[nc + c] = wb;
      }
      if (zero_next) {
        nxt[2 * c] = 0u;
        nxt[2 * c + 1] = 0u;
      }
    }
  }
}

// Interleaved counts [n_c][2] -> the ABI's [2][n_c].
__global__ void k_deinterleave(const uint32_t* __restrict__ counts, int64_t nc, uint32_t* __restrict__ out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const uint2 v = reinterpret_cast<const uint2*>(counts)[c];
    out[c] = v.x;
    out[nc + c] = v.y;
  }
}

// Fields from given volume fractions phi [2][n_c] (coupling write).
__global__ void k_field_from_phi(const SysDev* __restrict__ systems, int sys, const float* __restrict__ phi) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const int64_t nc = S.n_c;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += (int64_t)gridDim.x * blockDim.x) {
    const float pA = phi[c], pB = phi[nc + c];
    const float ex = S.kappaN_N * (pA + pB - 1.f);
    float wA = fmaf(S.chiN_N, pB, ex), wB = fmaf(S.chiN_N, pA, ex);
    if (S.umbrella) {
      wA = fmaf(S.umbN_N, pA - S.phi_target[c], wA);
      wB = fmaf(S.umbN_N, pB - S.phi_target[nc + c], wB);
    }
    S.w[c] = wA;
    S.w[nc + c] = wB;
  }
}

// Layer sums of the counts along one axis: block k adds the (nA, nB) of the
// m cells of layer k (interleaved count buffer) into out[2k], out[2k+1].
__global__ void k_profile(const uint32_t* __restrict__ counts, int nx, int ny, int nz, int axis,
                          unsigned long long* __restrict__ out) {
  const int k = blockIdx.x;
  const int64_t m = (int64_t)nx * ny * nz / (axis == 0 ? nx : axis == 1 ? ny : nz);
  unsigned long long a = 0, b = 0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    int64_t c;
    if (axis == 0)
      c = (int64_t)k * ny * nz + i;
    else if (axis == 1)
      c = ((i / nz) * ny + k) * nz + i % nz;
    else
      c = i * nz + k;
    a += counts[2 * c];
    b += counts[2 * c + 1];
  }
  __shared__ unsigned long long sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sa[threadIdx.x >> 5] = a;
    sb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long ta = 0, tb = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ta += sa[w];
      tb += sb[w];
    }
    out[2 * k] = ta;
    out[2 * k + 1] = tb;
  }
}

// Vertical pair sums of the type-t counts: block dz adds, over the cells c
// whose partner c + dz e_z exists (periodic, or inside the slab between
// walls), a b, a and b with a = n_t(c), b = n_t(c + dz e_z); block nz adds
// n and n^2 over all cells.  Integer sums, exact.  out [nz + 1][4].
__global__ void k_vcorr(const uint32_t* __restrict__ counts, int64_t n_c, int nz, int type, int wall,
                        unsigned long long* __restrict__ out) {
  const int dz = blockIdx.x;
  unsigned long long s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  for (int64_t c = threadIdx.x; c < n_c; c += blockDim.x) {
    const unsigned long long a = counts[2 * c + type];
    if (dz == nz) {
      s0 += a * a;
      s1 += a;
      s3 += 1;
      continue;
    }
    const int iz = (int)(c % nz);
    int jz = iz + dz;
    if (jz >= nz) {
      if (wall) continue;
      jz -= nz;
    }
    const unsigned long long b = counts[2 * (c - iz + jz) + type];
    s0 += a * b;
    s1 += a;
    s2 += b;
    s3 += 1;
  }
  __shared__ unsigned long long sh[4][32];
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_down_sync(0xffffffffu, s0, o);
    s1 += __shfl_down_sync(0xffffffffu, s1, o);
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
    s3 += __shfl_down_sync(0xffffffffu, s3, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = s0;
    sh[1][threadIdx.x >> 5] = s1;
    sh[2][threadIdx.x >> 5] = s2;
    sh[3][threadIdx.x >> 5] = s3;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
    out[4 * dz + threadIdx.x] = t;
  }
}

// Step counters of graph replays: advance n_sys counters by n, or set them.
__global__ void k_advance_step(unsigned long long* counters, int n_sys, long long n) {
  for (int i = threadIdx.x; i < n_sys; i += blockDim.x) counters[i] += (unsigned long long)n;
}

__global__ void k_set_step(unsigned long long* counters, int n_sys, unsigned long long value) {
  for (int i = threadIdx.x; i < n_sys; i += blockDim.x) counters[i] = value;
}

// ---------------------------------------------------------------------------
// Initial configuration: one thread per chain; bead 0 uniform in the box,
// bond i a Gaussian with per-axis variance 1/(3(N-1)) by Box-Muller on the
// word pairs (0,1) and (2,3).  Accumulated in FP64, then wrapped.
// ---------------------------------------------------------------------------
// Chain c (logical = storage slot) from bead 0 at (X, Y, Z): the bonds of
// the initial configuration, accumulated in FP64, wrapped (z folded between
// walls), written.
__device__ void grow_chain(const SysDev& S, int64_t c, double X, double Y, double Z) {
  const int N = S.N;
  const double sigma = N > 1 ? sqrt(1.0 / (3.0 * (N - 1))) : 0.0;
  const uint32_t id = (uint32_t)c + S.id_base;  // logical chain id
  S.chain_id[c] = id;
  for (int i = 0; i < N; ++i) {
    if (i > 0) {
      const uint4 r = philox10(make_uint4((uint32_t)i, id, kInitStep, (uint32_t)S.sys_index), S.rk);
      const double m1 = sqrt(-2.0 * log(((double)(r.x >> 8) + 0.5) * 0x1p-24));
      const double m2 = sqrt(-2.0 * log(((double)(r.z >> 8) + 0.5) * 0x1p-24));
      double s1, c1, s2, c2;
      sincospi(2.0 * ((double)(r.y >> 8) * 0x1p-24), &s1, &c1);
      sincospi(2.0 * ((double)(r.w >> 8) * 0x1p-24), &s2, &c2);
      X += sigma * m1 * c1;
      Y += sigma * m1 * s1;
      Z += sigma * m2 * c2;
    }
    const int64_t b = (int64_t)c * N + i;
    const double P[3] = {X, Y, Z};
    float* dst[3] = {S.x, S.y, S.z};
    short im[3];
    for (int a = 0; a < 3; ++a) {
      const double L = (double)S.L[a];
      if (a == 2 && S.wall_z) {
        // between walls: folded into [0, L) by mirror reflection, no image
        const double t = P[a] - 2.0 * L * floor(P[a] / (2.0 * L));
        float zw = (float)(t < L ? t : 2.0 * L - t);
        if (zw >= S.L[a]) zw = nextafterf(S.L[a], 0.f);
        if (zw < 0.f) zw = 0.f;
        dst[a][b] = zw;
        im[a] = 0;
        continue;
      }
      double n = floor(P[a] / L);
      float xw = (float)(P[a] - n * L);
      if (xw >= S.L[a]) { xw = 0.f; n += 1.0; }
      if (xw < 0.f) xw = 0.f;
      dst[a][b] = xw;
      im[a] = (short)n;
    }
    reinterpret_cast<short4*>(S.img)[b] = make_short4(im[0], im[1], im[2], 0);
  }
}

__global__ void k_init(const SysDev* __restrict__ systems, int sys) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_poly; c += (int64_t)gridDim.x * blockDim.x) {
    const uint4 r = philox10(make_uint4(0u, (uint32_t)c + S.id_base, kInitStep, (uint32_t)S.sys_index), S.rk);
    grow_chain(S, c, (double)S.L[0] * ((double)(r.x >> 8) * 0x1p-24),
               (double)S.L[1] * ((double)(r.y >> 8) * 0x1p-24), (double)S.L[2] * ((double)(r.z >> 8) * 0x1p-24));
  }
}

// ---------------------------------------------------------------------------
// Placement from target volume fractions (coupling start-up, Sec. 3.2):
// integer weights q(c) = floor(phi*(c) 2^16) of bead 0's type, their running
// sums P (64-bit), then per chain: cell = first c with P(c) > floor(r Q/2^64),
// r = (w1 << 32 | w0) of counter (0, c, kPlaceStep, s); bead 0 at a uniform
// point of that cell (counter (1, c, ...)) plus an offset uniform in
// [-h, h)^3, h = 1/(2 sqrt 3) (counter (2, c, ...)); the chain's bonds are
// those of the initial configuration.
// ---------------------------------------------------------------------------
constexpr uint32_t kPlaceStep = 0xFFFFFFFEu;

__global__ void k_place_weights(const float* __restrict__ phi, int64_t n, unsigned long long* __restrict__ q) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    const float v = phi[c];
    q[c] = v > 0.f ? (unsigned long long)(uint32_t)fminf(v * 65536.0f, 4294967040.0f) : 0ull;
  }
}

__global__ void k_place(const SysDev* __restrict__ systems, int sys, const unsigned long long* __restrict__ prefix,
                        unsigned long long Q) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const double h = 0.5 / sqrt(3.0);  // correctly rounded, as on the host
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_poly; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t id = (uint32_t)c + S.id_base;  // logical chain id
    const uint4 r0 = philox10(make_uint4(0u, id, kPlaceStep, (uint32_t)S.sys_index), S.rk);
    const uint4 r1 = philox10(make_uint4(1u, id, kPlaceStep, (uint32_t)S.sys_index), S.rk);
    const uint4 r2 = philox10(make_uint4(2u, id, kPlaceStep, (uint32_t)S.sys_index), S.rk);
    const unsigned long long r = ((unsigned long long)r0.y << 32) | r0.x;
    const unsigned long long k = __umul64hi(r, Q);
    int64_t lo = 0, hi = S.n_c - 1;  // first cell whose running sum exceeds k
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (prefix[mid] > k)
        hi = mid;
      else
        lo = mid + 1;
    }
    const int64_t ix = lo / ((int64_t)S.ny * S.nz), iy = (lo / S.nz) % S.ny, iz = lo % S.nz;
    const double X = ((double)ix + (double)(r1.x >> 8) * 0x1p-24) * (double)S.L[0] / S.nx +
                     h * fma((double)(r2.x >> 8), 0x1p-23, -1.0);
    const double Y = ((double)iy + (double)(r1.y >> 8) * 0x1p-24) * (double)S.L[1] / S.ny +
                     h * fma((double)(r2.y >> 8), 0x1p-23, -1.0);
    const double Z = ((double)iz + (double)(r1.z >> 8) * 0x1p-24) * (double)S.L[2] / S.nz +
                     h * fma((double)(r2.z >> 8), 0x1p-23, -1.0);
    grow_chain(S, c, X, Y, Z);
  }
}

// Positions and images in logical chain order <-> storage order.
__global__ void k_gather_state(const SysDev* __restrict__ systems, int sys, float* __restrict__ pos,
                               int16_t* __restrict__ img) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = b / S.N, i = b % S.N;
    const int64_t lb = (int64_t)((S.chain_id[slot] & kIdMask) - S.id_base) * S.N + i;
    pos[3 * lb + 0] = S.x[b];
    pos[3 * lb + 1] = S.y[b];
    pos[3 * lb + 2] = S.z[b];
    const short4 v = reinterpret_cast<const short4*>(S.img)[b];
    img[3 * lb + 0] = v.x;
    img[3 * lb + 1] = v.y;
    img[3 * lb + 2] = v.z;
  }
}

__global__ void k_scatter_state(const SysDev* __restrict__ systems, int sys, const float* __restrict__ pos,
                                const int16_t* __restrict__ img) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = b / S.N, i = b % S.N;
    const int64_t lb = (int64_t)((S.chain_id[slot] & kIdMask) - S.id_base) * S.N + i;
    S.x[b] = pos[3 * lb + 0];
    S.y[b] = pos[3 * lb + 1];
    S.z[b] = pos[3 * lb + 2];
    reinterpret_cast<short4*>(S.img)[b] = make_short4(img[3 * lb + 0], img[3 * lb + 1], img[3 * lb + 2], 0);
  }
}

// Molecule types in logical chain order <-> the chain-id words' top bit.
__global__ void k_get_types(const SysDev* __restrict__ systems, int sys, uint8_t* __restrict__ out) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_poly; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t word = S.chain_id[c];
    out[(word & kIdMask) - S.id_base] = (word & kTypeBit) ? 1 : 0;
  }
}

// types == nullptr: every chain back to type 0.
__global__ void k_set_types(const SysDev* __restrict__ systems, int sys, const uint8_t* __restrict__ types) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_poly; c += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t id = S.chain_id[c] & kIdMask;
    S.chain_id[c] = id | ((types && types[id - S.id_base]) ? kTypeBit : 0u);
  }
}

// Start-up consistency checks (Sec. 2.2 moves SOMA's validation to the GPU):
// every coordinate finite and inside [0, L).  Sets kErrBounds on failure.
__global__ void k_validate(const SysDev* __restrict__ systems, int sys, int* __restrict__ err) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
    const float v[3] = {S.x[b], S.y[b], S.z[b]};
    for (int a = 0; a < 3; ++a)
      if (!(v[a] >= 0.f && v[a] < S.L[a])) atomicOr(err, kErrBounds);
  }
}

// Check staged positions [n][3] before they replace the state.
__global__ void k_validate_pos(const float* __restrict__ pos, int64_t n, float Lx, float Ly, float Lz,
                               int* __restrict__ err) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const float x = pos[3 * b], y = pos[3 * b + 1], z = pos[3 * b + 2];
    if (!(x >= 0.f && x < Lx && y >= 0.f && y < Ly && z >= 0.f && z < Lz)) atomicOr(err, kErrBounds);
  }
}

// Sum of a system's accepted-move counters into *out.
__global__ void k_sum_acc(const SysDev* __restrict__ systems, int sys, unsigned long long* __restrict__ out) {
  const SysDev* S = systems + sys;
  unsigned long long a = 0;
  for (int i = threadIdx.x; i < S->acc_count; i += blockDim.x) a += S->acc[S->acc_first + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  __shared__ unsigned long long part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    *out = t;
  }
}

__global__ void k_zero_acc(const SysDev* __restrict__ systems, int sys) {
  const SysDev* S = systems + sys;
  for (int i = threadIdx.x; i < S->acc_count; i += blockDim.x) S->acc[S->acc_first + i] = 0ull;
}

// ---------------------------------------------------------------------------
// Observables in FP64: per chain R_e^2, R_g^2 and the bond energy from the
// unwrapped positions x + image * L; per cell the non-bonded energy from the
// counts of the current configuration.  out[0..4] = sum Re2, sum Rg2,
// sum |b|^2, sum_c f(phi), accepted.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_obs_chains(const SysDev* __restrict__ systems, int sys, double* __restrict__ out) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const int N = S.N;
  double re2 = 0, rg2 = 0, bb = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_poly; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b0 = (int64_t)c * N;
    // unwrapped positions relative to bead 0 (keeps the sums well conditioned)
    double first[3] = {0, 0, 0}, prev[3] = {0, 0, 0}, sum[3] = {0, 0, 0}, sq = 0;
    for (int i = 0; i < N; ++i) {
      const short4 im = reinterpret_cast<const short4*>(S.img)[b0 + i];
      const double p[3] = {(double)S.x[b0 + i] + (double)im.x * S.L[0],
                           (double)S.y[b0 + i] + (double)im.y * S.L[1],
                           (double)S.z[b0 + i] + (double)im.z * S.L[2]};
      for (int a = 0; a < 3; ++a) {
        if (i == 0) first[a] = p[a];
        const double r = p[a] - first[a];
        if (i > 0) bb += (p[a] - prev[a]) * (p[a] - prev[a]);
        sum[a] += r;
        sq += r * r;
        prev[a] = p[a];
      }
    }
    for (int a = 0; a < 3; ++a) re2 += (prev[a] - first[a]) * (prev[a] - first[a]);
    rg2 += sq / N - (sum[0] * sum[0] + sum[1] * sum[1] + sum[2] * sum[2]) / ((double)N * N);
  }
  re2 = warp_sum(re2);
  rg2 = warp_sum(rg2);
  bb = warp_sum(bb);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out + 0, re2);
    atomicAdd(out + 1, rg2);
    atomicAdd(out + 2, bb);
  }
}

__global__ void k_obs_cells(const SysDev* __restrict__ systems, int sys, long long t_done,
                            double* __restrict__ out, unsigned long long* __restrict__ acc_out) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  // counts of the current configuration sit in buffer (steps_done - 1) mod 3
  const uint32_t* cur = count_buffer(S.counts, S.n_c, t_done - 1);
  const double rho = S.rho_bar;
  const double chiN = (double)S.chiN_N * S.N, kappaN = (double)S.kappaN_N * S.N;
  double f = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_c; c += (int64_t)gridDim.x * blockDim.x) {
    const double pA = cur[2 * c] / rho, pB = cur[2 * c + 1] / rho, ex = pA + pB - 1.0;
    f += chiN * pA * pB + 0.5 * kappaN * ex * ex;
  }
  f = warp_sum(f);
  if ((threadIdx.x & 31) == 0) atomicAdd(out + 3, f);
  if (blockIdx.x == 0) {
    unsigned long long a = 0;
    for (int i = threadIdx.x; i < S.acc_count; i += blockDim.x) a += S.acc[S.acc_first + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc_out, a);
  }
}

// ---------------------------------------------------------------------------
// S(q) of one system of the handle (sq_accumulate in soma_device.cuh): the
// stored wrapped coordinates, the bead's type from its chain's A block.
// ---------------------------------------------------------------------------
__global__ void k_structure_factor(const SysDev* __restrict__ systems, int sys, int nq,
                                   const int32_t* __restrict__ m, double* __restrict__ out) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  sq_accumulate(
      S.n_b,
      [&](int64_t b, float& fx, float& fy, float& fz) {
        fx = S.x[b] * S.invL[0];
        fy = S.y[b] * S.invL[1];
        fz = S.z[b] * S.invL[2];
      },
      [&](int64_t b) { return ((int)(b % S.N) < chain_n_A(S, b / S.N)) ? 1.0 : -1.0; }, m, nq, out);
}

// The device Philox on explicit counters and keys (verification entry point).
__global__ void k_philox(const uint32_t* __restrict__ ctr, const uint32_t* __restrict__ key,
                         uint32_t* __restrict__ out, int64_t n) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rk[10][2];
    uint32_t k0 = key[2 * j], k1 = key[2 * j + 1];
    for (int r = 0; r < 10; ++r) {
      rk[r][0] = k0;
      rk[r][1] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint4 v = philox10(make_uint4(ctr[4 * j], ctr[4 * j + 1], ctr[4 * j + 2], ctr[4 * j + 3]), rk);
    out[4 * j] = v.x;
    out[4 * j + 1] = v.y;
    out[4 * j + 2] = v.z;
    out[4 * j + 3] = v.w;
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers.
// ---------------------------------------------------------------------------
cudaError_t launch_move_generic(const SysDev* systems, int sys, int64_t n_poly, int N, StepRef r, int sm_count,
                                cudaStream_t s) {
  for (int set = 0; set < 2; ++set) {
    const int64_t work = n_poly * ((N - set + 1) / 2);
    int blocks = (int)((work + 255) / 256);
    if (blocks > sm_count * 8) blocks = sm_count * 8;
    if (blocks < 1) blocks = 1;
    k_move_set_generic<<<blocks, 256, 0, s>>>(systems, sys, r, set);
  }
  return cudaGetLastError();
}

cudaError_t launch_bin(const SysDev* systems, int sys, int64_t n_b, StepRef r, int sm_count, cudaStream_t s) {
  const int threads = 512;
  int64_t blocks = (n_b + threads - 1) / threads;
  if (blocks > (int64_t)sm_count * 16) blocks = (int64_t)sm_count * 16;
  if (blocks < 1) blocks = 1;
  k_bin<<<(unsigned)blocks, threads, 0, s>>>(systems, sys, r);
  return cudaGetLastError();
}

cudaError_t launch_field(const FieldArgs& f, StepRef r, int zero_next, cudaStream_t s) {
  const int64_t groups = (f.n_c & 1) == 0 ? (f.n_c >> 1) : f.n_c;
  int64_t blocks = (groups + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  if (blocks < 1) blocks = 1;
  k_field<<<(unsigned)blocks, 256, 0, s>>>(f, r, zero_next);
  return cudaGetLastError();
}

cudaError_t launch_deinterleave(const uint32_t* counts, int64_t n_c, uint32_t* out, int sm_count, cudaStream_t s) {
  k_deinterleave<<<sm_count * 8, 256, 0, s>>>(counts, n_c, out);
  return cudaGetLastError();
}

cudaError_t launch_field_from_phi(const SysDev* systems, int sys, const float* phi, int sm_count, cudaStream_t s) {
  k_field_from_phi<<<sm_count * 4, 256, 0, s>>>(systems, sys, phi);
  return cudaGetLastError();
}

cudaError_t launch_place(const SysDev* systems, int sys, const SysDev& host, const float* phi,
                         unsigned long long* q, unsigned long long* prefix, void* temp, size_t temp_bytes,
                         unsigned long long* total, int sm_count, cudaStream_t s) {
  const int64_t nc = host.n_c;
  const float* w = phi + (host.n_A > 0 ? 0 : nc);  // weights of bead 0's type
  k_place_weights<<<sm_count * 4, 256, 0, s>>>(w, nc, q);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  (void)temp_bytes;
  e = launch_scan_u64(q, prefix, nc, true, temp, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(total, prefix + nc - 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (*total == 0) return cudaSuccess;
  const int grid = (int)std::min<int64_t>(((int64_t)host.n_poly + 127) / 128, (int64_t)sm_count * 8);
  k_place<<<grid, 128, 0, s>>>(systems, sys, prefix, *total);
  return cudaGetLastError();
}

size_t place_temp_bytes(int64_t n_c) { return scan_temp_bytes_u64(n_c); }

cudaError_t launch_profile(const uint32_t* counts, int nx, int ny, int nz, int axis, unsigned long long* out,
                           cudaStream_t s) {
  const int layers = axis == 0 ? nx : axis == 1 ? ny : nz;
  k_profile<<<layers, 256, 0, s>>>(counts, nx, ny, nz, axis, out);
  return cudaGetLastError();
}

cudaError_t launch_vcorr(const uint32_t* counts, int64_t n_c, int nz, int type, int wall, unsigned long long* out,
                         cudaStream_t s) {
  k_vcorr<<<nz + 1, 256, 0, s>>>(counts, n_c, nz, type, wall, out);
  return cudaGetLastError();
}

cudaError_t launch_advance(unsigned long long* counters, int n_sys, long long n, cudaStream_t s) {
  k_advance_step<<<1, 256, 0, s>>>(counters, n_sys, n);
  return cudaGetLastError();
}

cudaError_t launch_set_step(unsigned long long* counters, int n_sys, unsigned long long value, cudaStream_t s) {
  k_set_step<<<1, 256, 0, s>>>(counters, n_sys, value);
  return cudaGetLastError();
}

cudaError_t launch_init(const SysDev* systems, int sys, int64_t n_poly, cudaStream_t s) {
  const int threads = 128;
  const int64_t blocks = (n_poly + threads - 1) / threads;
  k_init<<<(unsigned)blocks, threads, 0, s>>>(systems, sys);
  return cudaGetLastError();
}

cudaError_t launch_get_types(const SysDev* systems, int sys, uint8_t* out, int sm_count, cudaStream_t s) {
  k_get_types<<<sm_count * 4, 256, 0, s>>>(systems, sys, out);
  return cudaGetLastError();
}

cudaError_t launch_set_types(const SysDev* systems, int sys, const uint8_t* types, int sm_count, cudaStream_t s) {
  k_set_types<<<sm_count * 4, 256, 0, s>>>(systems, sys, types);
  return cudaGetLastError();
}

cudaError_t launch_gather_state(const SysDev* systems, int sys, float* pos, int16_t* img, int sm_count, cudaStream_t s) {
  k_gather_state<<<sm_count * 8, 256, 0, s>>>(systems, sys, pos, img);
  return cudaGetLastError();
}

cudaError_t launch_scatter_state(const SysDev* systems, int sys, const float* pos, const int16_t* img, int sm_count,
                                 cudaStream_t s) {
  k_scatter_state<<<sm_count * 8, 256, 0, s>>>(systems, sys, pos, img);
  return cudaGetLastError();
}

cudaError_t launch_validate(const SysDev* systems, int sys, int* err, int sm_count, cudaStream_t s) {
  k_validate<<<sm_count * 4, 256, 0, s>>>(systems, sys, err);
  return cudaGetLastError();
}

cudaError_t launch_validate_pos(const float* pos, int64_t n, const float* L, int* err, int sm_count,
                                cudaStream_t s) {
  k_validate_pos<<<sm_count * 4, 256, 0, s>>>(pos, n, L[0], L[1], L[2], err);
  return cudaGetLastError();
}

cudaError_t launch_sum_acc(const SysDev* systems, int sys, unsigned long long* out, cudaStream_t s) {
  k_sum_acc<<<1, 1024, 0, s>>>(systems, sys, out);
  return cudaGetLastError();
}

cudaError_t launch_zero_acc(const SysDev* systems, int sys, cudaStream_t s) {
  k_zero_acc<<<1, 256, 0, s>>>(systems, sys);
  return cudaGetLastError();
}

cudaError_t launch_observables(const SysDev* systems, int sys, long long t_done, double* out,
                               unsigned long long* acc_out, int sm_count, cudaStream_t s) {
  k_obs_chains<<<sm_count * 4, 256, 0, s>>>(systems, sys, out);
  k_obs_cells<<<sm_count * 4, 256, 0, s>>>(systems, sys, t_done, out, acc_out);
  return cudaGetLastError();
}

cudaError_t launch_structure_factor(const SysDev* systems, int sys, int nq, const int32_t* m, double* out,
                                    int sm_count, cudaStream_t s) {
  k_structure_factor<<<sm_count * 4, 256, 0, s>>>(systems, sys, nq, m, out);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n, cudaStream_t s) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  k_philox<<<(unsigned)blocks, 256, 0, s>>>(ctr, key, out, n);
  return cudaGetLastError();
}

}  // namespace soma
