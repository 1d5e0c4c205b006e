// soma_f64.cu -- the FP64-position form of the SCMF step (a precision
// reference for the FP32 + image form the throughput path uses).
//
// Positions are FP64, wrapped into [0, L) with the same int16 image counts;
// a step runs the same algorithm as k_move with the same Philox counters:
// d = A (2U - 1) is exact in FP64, the bond term is
// k_b (2 d . sum_j (r - r_j) + n_j |d|^2), the field term is evaluated from
// the previous step's integer counts, acceptance is dE + ln u < 0 with FP64
// logarithm.  Kernels here favour plainness over speed: one warp holds 32/P
// chains (lane k: beads 2k and 2k+1), grid-stride over such groups, plain
// loads.  One system per handle, no chain reorder.
#include <cuda_runtime.h>

#include <cstdint>

#include "soma_device.cuh"
#include "soma_internal.cuh"
#include "soma_launch.h"

namespace soma {

__device__ __forceinline__ int cell_axis64(double x, double cps, int n) {
  const int i = (int)(x * cps);  // x >= 0
  return i < n - 1 ? i : n - 1;
}

__device__ __forceinline__ int cell_of64(const SysDev& S, double x, double y, double z) {
  return (cell_axis64(x, S.cps64[0], S.nx) * S.ny + cell_axis64(y, S.cps64[1], S.ny)) * S.nz +
         cell_axis64(z, S.cps64[2], S.nz);
}

// Wrap into [0, L): image step in {-1, 0, 1}; a tiny negative coordinate
// whose shift rounds to L is kept at the largest double below L.
__device__ __forceinline__ double wrap64(double p, double L, int& step) {
  step = p >= L ? 1 : (p < 0.0 ? -1 : 0);
  double q = p - step * L;
  if (q >= L) q = nextafter(L, 0.0);
  return q;
}

__device__ __forceinline__ double min_image64(double d, double L, double invL) { return d - L * rint(d * invL); }

__device__ __forceinline__ double field_diff64(const SysDev& S, const uint2* prev, int type, int c0, int c1) {
  const uint2 n0 = prev[c0], n1 = prev[c1];
  const double d_other = type ? (double)((int)n1.x - (int)n0.x) : (double)((int)n1.y - (int)n0.y);
  const double d_tot = (double)(((int)n1.x + (int)n1.y) - ((int)n0.x + (int)n0.y));
  // (chiN/N dn_other + kappaN/N dn_total) / rho_bar, constants folded on the host
  return S.chiN64 * d_other + S.kappaN64 * d_tot;
}

__global__ void k_move64(const SysDev* __restrict__ systems, int sys, StepRef rs) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const long long tl = rs.get();
  const uint32_t t = (uint32_t)tl;
  const int lane = threadIdx.x & 31;
  const int P = S.P, N = S.N, cpw = 32 / P;
  const int k = lane & (P - 1);
  const int e = 2 * k, o = 2 * k + 1;
  const int te = e < S.n_A ? 0 : 1, to = o < S.n_A ? 0 : 1;
  const uint2* prev = reinterpret_cast<const uint2*>(count_buffer(S.counts, S.n_c, tl - 1));
  uint32_t* cnt = count_buffer(S.counts, S.n_c, tl);
  const double kb = (double)S.kb;
  const int64_t groups = ((int64_t)S.n_poly + cpw - 1) / cpw;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  unsigned nacc = 0;
  for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < groups; g += warps) {
    const int64_t chain = g * cpw + lane / P;
    const bool chain_ok = chain < S.n_poly;
    const bool he = chain_ok && e < N, ho = chain_ok && o < N;
    const int64_t be = (chain_ok ? chain : 0) * N + e;
    double xe = 0, ye = 0, ze = 0, xo = 0, yo = 0, zo = 0;
    if (he) { xe = S.x64[be]; ye = S.y64[be]; ze = S.z64[be]; }
    if (ho) { xo = S.x64[be + 1]; yo = S.y64[be + 1]; zo = S.z64[be + 1]; }
    const uint32_t cid = chain_ok ? S.chain_id[chain] : 0u;
    const double L0 = S.L64[0], L1 = S.L64[1], L2 = S.L64[2];

    // set 0: even bead, neighbours 2k-1 (lane k-1) and 2k+1 (own)
    const double lx = __shfl_up_sync(0xffffffffu, xo, 1, P);
    const double ly = __shfl_up_sync(0xffffffffu, yo, 1, P);
    const double lz = __shfl_up_sync(0xffffffffu, zo, 1, P);
    const double wL = k > 0 ? 1.0 : 0.0, wR = o < N ? 1.0 : 0.0;
    const double I0 = S.invL64[0], I1 = S.invL64[1], I2 = S.invL64[2];
    const double sx = wL * min_image64(xe - lx, L0, I0) + wR * min_image64(xe - xo, L0, I0);
    const double sy = wL * min_image64(ye - ly, L1, I1) + wR * min_image64(ye - yo, L1, I1);
    const double sz = wL * min_image64(ze - lz, L2, I2) + wR * min_image64(ze - zo, L2, I2);
    const uint4 re = philox10(make_uint4((uint32_t)e, cid, t, (uint32_t)S.sys_index), S.rk);
    const double A = (double)S.A;
    const double dx = A * ((double)(re.x >> 8) * 0x1p-23 - 1.0);
    const double dy = A * ((double)(re.y >> 8) * 0x1p-23 - 1.0);
    const double dz = A * ((double)(re.z >> 8) * 0x1p-23 - 1.0);
    int sxw, syw, szw;
    const double pex = wrap64(xe + dx, L0, sxw), pey = wrap64(ye + dy, L1, syw), pez = wrap64(ze + dz, L2, szw);
    const int ce0 = cell_of64(S, xe, ye, ze), ce1 = cell_of64(S, pex, pey, pez);
    const double dEb = 2.0 * (dx * sx + dy * sy + dz * sz) + (wL + wR) * (dx * dx + dy * dy + dz * dz);
    const double dE = kb * dEb + field_diff64(S, prev, te, ce0, ce1);
    const double u = ((double)(re.w >> 9) + 0.5) * 0x1p-23;
    const bool acc = he && (dE + log(u) < 0.0);
    if (acc) {
      xe = pex; ye = pey; ze = pez;
      if (sxw | syw | szw) {
        short4* ip = reinterpret_cast<short4*>(S.img) + be;
        short4 v = *ip;
        v.x += (short)sxw; v.y += (short)syw; v.z += (short)szw;
        *ip = v;
      }
    }

    // set 1: odd bead, neighbours 2k (own, updated) and 2k+2 (lane k+1)
    const double rx = __shfl_down_sync(0xffffffffu, xe, 1, P);
    const double ry = __shfl_down_sync(0xffffffffu, ye, 1, P);
    const double rz = __shfl_down_sync(0xffffffffu, ze, 1, P);
    const double w2 = o + 1 < N ? 1.0 : 0.0;
    const double ox = min_image64(xo - xe, L0, I0) + w2 * min_image64(xo - rx, L0, I0);
    const double oy = min_image64(yo - ye, L1, I1) + w2 * min_image64(yo - ry, L1, I1);
    const double oz = min_image64(zo - ze, L2, I2) + w2 * min_image64(zo - rz, L2, I2);
    const uint4 ro = philox10(make_uint4((uint32_t)o, cid, t, (uint32_t)S.sys_index), S.rk);
    const double ex = A * ((double)(ro.x >> 8) * 0x1p-23 - 1.0);
    const double ey = A * ((double)(ro.y >> 8) * 0x1p-23 - 1.0);
    const double ez = A * ((double)(ro.z >> 8) * 0x1p-23 - 1.0);
    const double pox = wrap64(xo + ex, L0, sxw), poy = wrap64(yo + ey, L1, syw), poz = wrap64(zo + ez, L2, szw);
    const int co0 = cell_of64(S, xo, yo, zo), co1 = cell_of64(S, pox, poy, poz);
    const double dEbo = 2.0 * (ex * ox + ey * oy + ez * oz) + (1.0 + w2) * (ex * ex + ey * ey + ez * ez);
    const double dEo = kb * dEbo + field_diff64(S, prev, to, co0, co1);
    const double uo = ((double)(ro.w >> 9) + 0.5) * 0x1p-23;
    const bool acco = ho && (dEo + log(uo) < 0.0);
    if (acco) {
      xo = pox; yo = poy; zo = poz;
      if (sxw | syw | szw) {
        short4* ip = reinterpret_cast<short4*>(S.img) + be + 1;
        short4 v = *ip;
        v.x += (short)sxw; v.y += (short)syw; v.z += (short)szw;
        *ip = v;
      }
    }
    if (acc) { S.x64[be] = xe; S.y64[be] = ye; S.z64[be] = ze; }
    if (acco) { S.x64[be + 1] = xo; S.y64[be + 1] = yo; S.z64[be + 1] = zo; }
    if (he) atomicAdd(cnt + 2 * (acc ? ce1 : ce0) + te, 1u);
    if (ho) atomicAdd(cnt + 2 * (acco ? co1 : co0) + to, 1u);
    nacc += (acc ? 1u : 0u) + (acco ? 1u : 0u);
  }
  nacc = __reduce_add_sync(0xffffffffu, nacc);
  if (lane == 0 && nacc) atomicAdd(S.acc + S.acc_first + (blockIdx.x % S.acc_count), (unsigned long long)nacc);
  // clear count buffer t+1 mod 3 for the next step
  uint2* next2 = reinterpret_cast<uint2*>(count_buffer(S.counts, S.n_c, tl + 1));
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_c; c += (int64_t)gridDim.x * blockDim.x)
    next2[c] = make_uint2(0u, 0u);
}

// Start-up configuration as k_init, kept in FP64.
__global__ void k_init64(const SysDev* __restrict__ systems, int sys) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const int N = S.N;
  const double sigma = N > 1 ? sqrt(1.0 / (3.0 * (N - 1))) : 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_poly; c += (int64_t)gridDim.x * blockDim.x) {
    double X = 0, Y = 0, Z = 0;
    S.chain_id[c] = (uint32_t)c;
    for (int i = 0; i < N; ++i) {
      const uint4 r = philox10(make_uint4((uint32_t)i, (uint32_t)c, kInitStep, (uint32_t)S.sys_index), S.rk);
      if (i == 0) {
        X = S.L64[0] * ((double)(r.x >> 8) * 0x1p-24);
        Y = S.L64[1] * ((double)(r.y >> 8) * 0x1p-24);
        Z = S.L64[2] * ((double)(r.z >> 8) * 0x1p-24);
      } else {
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
      double* dst[3] = {S.x64, S.y64, S.z64};
      short im[3];
      for (int a = 0; a < 3; ++a) {
        const double L = S.L64[a];
        double n = floor(P[a] / L);
        double xw = P[a] - n * L;
        if (xw >= L) { xw = 0.0; n += 1.0; }
        if (xw < 0.0) xw = 0.0;
        dst[a][b] = xw;
        im[a] = (short)n;
      }
      reinterpret_cast<short4*>(S.img)[b] = make_short4(im[0], im[1], im[2], 0);
    }
  }
}

__global__ void k_bin64(const SysDev* __restrict__ systems, int sys, long long t) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  uint32_t* cnt = count_buffer(S.counts, S.n_c, t);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(b % S.N);
    atomicAdd(cnt + 2 * cell_of64(S, S.x64[b], S.y64[b], S.z64[b]) + (i < S.n_A ? 0 : 1), 1u);
  }
}

__global__ void k_gather_state64(const SysDev* __restrict__ systems, int sys, double* __restrict__ pos,
                                 int16_t* __restrict__ img) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lb = (int64_t)(S.chain_id[b / S.N] & kIdMask) * S.N + b % S.N;
    pos[3 * lb + 0] = S.x64[b];
    pos[3 * lb + 1] = S.y64[b];
    pos[3 * lb + 2] = S.z64[b];
    const short4 v = reinterpret_cast<const short4*>(S.img)[b];
    img[3 * lb + 0] = v.x;
    img[3 * lb + 1] = v.y;
    img[3 * lb + 2] = v.z;
  }
}

__global__ void k_scatter_state64(const SysDev* __restrict__ systems, int sys, const double* __restrict__ pos,
                                  const int16_t* __restrict__ img) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lb = (int64_t)(S.chain_id[b / S.N] & kIdMask) * S.N + b % S.N;
    S.x64[b] = pos[3 * lb + 0];
    S.y64[b] = pos[3 * lb + 1];
    S.z64[b] = pos[3 * lb + 2];
    reinterpret_cast<short4*>(S.img)[b] = make_short4(img[3 * lb + 0], img[3 * lb + 1], img[3 * lb + 2], 0);
  }
}

__global__ void k_validate_pos64(const double* __restrict__ pos, int64_t n, double Lx, double Ly, double Lz,
                                 int* __restrict__ err) {
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const double x = pos[3 * b], y = pos[3 * b + 1], z = pos[3 * b + 2];
    if (!(x >= 0.0 && x < Lx && y >= 0.0 && y < Ly && z >= 0.0 && z < Lz)) atomicOr(err, kErrBounds);
  }
}

__device__ __forceinline__ double warp_sum64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_obs_chains64(const SysDev* __restrict__ systems, int sys, double* __restrict__ out) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  const int N = S.N;
  double re2 = 0, rg2 = 0, bb = 0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < S.n_poly; c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b0 = (int64_t)c * N;
    double first[3] = {0, 0, 0}, prev[3] = {0, 0, 0}, sum[3] = {0, 0, 0}, sq = 0;
    for (int i = 0; i < N; ++i) {
      const short4 im = reinterpret_cast<const short4*>(S.img)[b0 + i];
      const double p[3] = {S.x64[b0 + i] + (double)im.x * S.L64[0], S.y64[b0 + i] + (double)im.y * S.L64[1],
                           S.z64[b0 + i] + (double)im.z * S.L64[2]};
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
  re2 = warp_sum64(re2);
  rg2 = warp_sum64(rg2);
  bb = warp_sum64(bb);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out + 0, re2);
    atomicAdd(out + 1, rg2);
    atomicAdd(out + 2, bb);
  }
}

// S(q) with FP64 phases of the wrapped FP64 positions.
__global__ void k_structure_factor64(const SysDev* __restrict__ systems, int sys, int nq,
                                     const int32_t* __restrict__ m, double* __restrict__ out) {
  __shared__ SysDev S;
  load_sys(&S, systems + sys);
  for (int q = 0; q < nq; ++q) {
    const double mx = m[3 * q], my = m[3 * q + 1], mz = m[3 * q + 2];
    double re = 0, im = 0;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < S.n_b; b += (int64_t)gridDim.x * blockDim.x) {
      double f = mx * S.x64[b] * S.invL64[0] + my * S.y64[b] * S.invL64[1] + mz * S.z64[b] * S.invL64[2];
      f -= floor(f);
      double sn, cs;
      sincospi(2.0 * f, &sn, &cs);
      const double s = ((int)(b % S.N) < S.n_A) ? 1.0 : -1.0;
      re += s * cs;
      im += s * sn;
    }
    re = warp_sum64(re);
    im = warp_sum64(im);
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(out + 2 * q, re);
      atomicAdd(out + 2 * q + 1, im);
    }
  }
}

cudaError_t launch_move64(const SysDev* systems, int sys, StepRef r, int sm_count, cudaStream_t s) {
  k_move64<<<sm_count * 8, 256, 0, s>>>(systems, sys, r);
  return cudaGetLastError();
}
cudaError_t launch_init64(const SysDev* systems, int sys, int64_t n_poly, cudaStream_t s) {
  k_init64<<<(unsigned)((n_poly + 127) / 128), 128, 0, s>>>(systems, sys);
  return cudaGetLastError();
}
cudaError_t launch_bin64(const SysDev* systems, int sys, long long t, int sm_count, cudaStream_t s) {
  k_bin64<<<sm_count * 16, 512, 0, s>>>(systems, sys, t);
  return cudaGetLastError();
}
cudaError_t launch_gather_state64(const SysDev* systems, int sys, double* pos, int16_t* img, int sm_count,
                                  cudaStream_t s) {
  k_gather_state64<<<sm_count * 8, 256, 0, s>>>(systems, sys, pos, img);
  return cudaGetLastError();
}
cudaError_t launch_scatter_state64(const SysDev* systems, int sys, const double* pos, const int16_t* img,
                                   int sm_count, cudaStream_t s) {
  k_scatter_state64<<<sm_count * 8, 256, 0, s>>>(systems, sys, pos, img);
  return cudaGetLastError();
}
cudaError_t launch_validate_pos64(const double* pos, int64_t n, const double* L, int* err, int sm_count,
                                  cudaStream_t s) {
  k_validate_pos64<<<sm_count * 4, 256, 0, s>>>(pos, n, L[0], L[1], L[2], err);
  return cudaGetLastError();
}
cudaError_t launch_obs_chains64(const SysDev* systems, int sys, double* out, int sm_count, cudaStream_t s) {
  k_obs_chains64<<<sm_count * 4, 256, 0, s>>>(systems, sys, out);
  return cudaGetLastError();
}
cudaError_t launch_structure_factor64(const SysDev* systems, int sys, int nq, const int32_t* m, double* out,
                                      int sm_count, cudaStream_t s) {
  k_structure_factor64<<<sm_count * 4, 256, 0, s>>>(systems, sys, nq, m, out);
  return cudaGetLastError();
}

}  // namespace soma
