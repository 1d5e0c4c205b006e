// soma_device.cuh -- device helpers shared by the kernels of libsoma:
// Philox4x32-10, cell indexing, periodic wrap and minimum image, the
// Metropolis trial of one bead, image bookkeeping, the S(q) accumulation.
#pragma once

#include <cstdint>

#include "soma_internal.cuh"

namespace soma {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  The round keys are
// precomputed per system on the host (seed lo/hi plus r times the published
// Weyl increments), so a round is two wide multiplies and two 3-input XORs.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, const uint32_t (*rk)[2]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned long long p0 = (unsigned long long)0xD2511F53u * c.x;
    const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[r][0], (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ rk[r][1], (uint32_t)p0);
  }
  return c;
}

// Copy one system's constants into shared memory (all threads call).
__device__ __forceinline__ void load_sys(SysDev* dst, const SysDev* src) {
  const int words = sizeof(SysDev) / 4;
  const uint32_t* s = reinterpret_cast<const uint32_t*>(src);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = __ldg(s + i);
  __syncthreads();
}

// A-block length of the chain in storage slot `slot`: n_A, or n_A_alt for a
// converted molecule (conversion on and the chain-id word's top bit set).
__device__ __forceinline__ int chain_n_A(const SysDev& S, int64_t slot) {
  return (S.conv && (S.chain_id[slot] & kTypeBit)) ? S.n_A_alt : S.n_A;
}

__device__ __forceinline__ int cell_axis(float x, float cps, int n) {
  const int i = (int)(x * cps);  // x >= 0 (and a NaN converts to 0), so truncation is floor
  return min(i, n - 1);
}

__device__ __forceinline__ int cell_of(const SysDev& S, float x, float y, float z) {
  return (cell_axis(x, S.cps[0], S.nx) * S.ny + cell_axis(y, S.cps[1], S.ny)) * S.nz +
         cell_axis(z, S.cps[2], S.nz);
}

// Wrap a proposed coordinate back into [0, L); delta receives the image step.
__device__ __forceinline__ float wrap_coord(float p, float L, int& delta) {
  delta = 0;
  if (p >= L) {
    p -= L;  // exact: L <= p < 2L
    delta = 1;
  } else if (p < 0.f) {
    p += L;
    delta = -1;
    if (p >= L) {  // |p| below half an ulp of L: the wrapped value is 0 in this image
      p = 0.f;
      delta = 0;
    }
  }
  return p;
}

__device__ __forceinline__ float min_image(float d, float L, float invL) {
  return d - L * rintf(d * invL);
}

// One Metropolis trial of bead `bead` of logical chain `cid` at step t.
// (x, y, z, cell) is updated in place on acceptance; wrap receives the image
// steps packed as (dx+1) | (dy+1) << 2 | (dz+1) << 4 (21 = no wrap).
// Neighbours a and b enter with weights wa, wb in {0, 1}.
//   dE_bond = k_b sum_j (|r + d - r_j|^2 - |r - r_j|^2)
//           = k_b (2 d . sum_j (r - r_j) + n_j |d|^2)
__device__ __forceinline__ int try_move(const SysDev& S, const float* __restrict__ wt, uint32_t bead,
                                        uint32_t cid, uint32_t t, float& x, float& y, float& z,
                                        int& cell, int& wrap, float ax, float ay, float az, float wa,
                                        float bx, float by, float bz, float wb) {
  const uint4 r = philox10(make_uint4(bead, cid, t, (uint32_t)S.sys_index), S.rk);
  // d_k = A (2 U_k - 1), U_k = (r_k >> 8) 2^-24; (r_k >> 8) 2^-23 - 1 is exact in FP32.
  const float dx = S.A * fmaf((float)(r.x >> 8), 0x1p-23f, -1.0f);
  const float dy = S.A * fmaf((float)(r.y >> 8), 0x1p-23f, -1.0f);
  const float dz = S.A * fmaf((float)(r.z >> 8), 0x1p-23f, -1.0f);
  const float sx = wa * min_image(x - ax, S.L[0], S.invL[0]) + wb * min_image(x - bx, S.L[0], S.invL[0]);
  const float sy = wa * min_image(y - ay, S.L[1], S.invL[1]) + wb * min_image(y - by, S.L[1], S.invL[1]);
  // z between hard walls (S.wall_z): plain differences, no wrap
  const float sz = S.wall_z ? wa * (z - az) + wb * (z - bz)
                            : wa * min_image(z - az, S.L[2], S.invL[2]) + wb * min_image(z - bz, S.L[2], S.invL[2]);
  const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float dEb = fmaf(2.f, fmaf(dx, sx, fmaf(dy, sy, dz * sz)), (wa + wb) * d2);
  int ex, ey, ez;
  const float px = wrap_coord(x + dx, S.L[0], ex);
  const float py = wrap_coord(y + dy, S.L[1], ey);
  float pz;
  if (S.wall_z) {
    pz = z + dz;
    ez = 0;
    if (!(pz >= 0.f && pz < S.L[2])) return 0;  // through a wall: rejected
  } else {
    pz = wrap_coord(z + dz, S.L[2], ez);
  }
  const int cnew = cell_of(S, px, py, pz);
  const float dE = fmaf(S.kb, dEb, __ldg(wt + cnew) - __ldg(wt + cell));
  // Metropolis: accept iff dE + ln u < 0 with u = ((r_3 >> 9) + 1/2) 2^-23 in
  // (0, 1); dE <= 0 always accepts because ln u < 0.
  bool ok = dE <= 0.f;
  if (!ok) {
    const float u = fmaf((float)(r.w >> 9), 0x1p-23f, 0x1p-24f);
    ok = dE + __logf(u) < 0.f;
  }
  if (ok) {
    x = px;
    y = py;
    z = pz;
    cell = cnew;
    wrap = (ex + 1) | ((ey + 1) << 2) | ((ez + 1) << 4);
  }
  return ok ? 1 : 0;
}

__device__ __forceinline__ void apply_wrap(int16_t* img, int64_t bead, int wrap) {
  if (wrap != 21) {
    short4* p = reinterpret_cast<short4*>(img) + bead;
    short4 v = *p;
    v.x += (short)((wrap & 3) - 1);
    v.y += (short)(((wrap >> 2) & 3) - 1);
    v.z += (short)(((wrap >> 4) & 3) - 1);
    *p = v;
  }
}


// ---------------------------------------------------------------------------
// S(q) accumulation, shared by the handle's structure-factor kernel and the
// allocation-free entry point.  Per bead the phase 2 pi m.r/L is taken from
// the wrapped position (q is a lattice vector, so images drop out) as the
// fractional part of m.(r/L) in FP32, and s_j cos, s_j sin are accumulated in
// FP64.  Each thread sums a chunk of up to kSqChunk q vectors over its beads
// (grid-stride), warps reduce, and lane 0 adds to out[2 q + {0, 1}].
// frac(b, fx, fy, fz) gives bead b's coordinates over the box edges, sign(b)
// its composition sign (+1 for A, -1 for B).
// ---------------------------------------------------------------------------
constexpr int kSqChunk = 8;

__device__ __forceinline__ double sq_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

template <class Frac, class Sign>
__device__ __forceinline__ void sq_accumulate(int64_t n, const Frac& frac, const Sign& sign,
                                              const int32_t* __restrict__ m, int nq, double* __restrict__ out) {
  for (int q0 = 0; q0 < nq; q0 += kSqChunk) {
    double re[kSqChunk], im[kSqChunk];
    float mx[kSqChunk], my[kSqChunk], mz[kSqChunk];
#pragma unroll
    for (int j = 0; j < kSqChunk; ++j) {
      re[j] = im[j] = 0.0;
      const int q = q0 + j < nq ? q0 + j : nq - 1;
      mx[j] = (float)m[3 * q + 0];
      my[j] = (float)m[3 * q + 1];
      mz[j] = (float)m[3 * q + 2];
    }
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
      float fx, fy, fz;
      frac(b, fx, fy, fz);
      const double s = sign(b);
#pragma unroll
      for (int j = 0; j < kSqChunk; ++j) {
        float f = fmaf(mx[j], fx, fmaf(my[j], fy, mz[j] * fz));
        f -= floorf(f);
        float sn, cs;
        sincospif(2.f * f, &sn, &cs);
        re[j] += s * (double)cs;
        im[j] += s * (double)sn;
      }
    }
#pragma unroll
    for (int j = 0; j < kSqChunk; ++j) {
      const double r = sq_warp_sum(re[j]), i = sq_warp_sum(im[j]);
      if ((threadIdx.x & 31) == 0 && q0 + j < nq) {
        atomicAdd(out + 2 * (q0 + j) + 0, r);
        atomicAdd(out + 2 * (q0 + j) + 1, i);
      }
    }
  }
}


}  // namespace soma
