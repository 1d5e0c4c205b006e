// soma_move.cu -- kernel (a) of the SCMF step with the histogram (b) fused as
// its epilogue: the biased trial moves and energy evaluations of the move
// kernel profiled in Sec. 2.2, for chains of up to 64 beads.
//
// Design (one system per launch, constants in the parameter bank):
//  * persistent CTAs, warp-specialised: one producer warp streams each
//    tile's positions (x, y, z) and logical chain ids from HBM into a ring of
//    kStages shared-memory stages with cp.async.bulk, completion tracked by
//    mbarriers; kConsumerWarps consumer warps compute;
//  * a consumer lane k of a chain holds beads 2k (even set) and 2k+1 (odd
//    set); neighbours come from the adjacent lane by width-P shuffles;
//  * both beads' proposals are formed first, so the four field gathers of
//    the lane (old and proposed cell of each bead) go out together;
//  * set 0 (even beads) is decided first; set 1 reuses set 0's bond vectors
//    plus the accepted displacement, so no second minimum image is needed;
//  * new positions go straight back to global memory; the final cells are
//    added to count buffer t & 1 by fire-and-forget atomics (kernel (b)).
// Every mbarrier wait is bounded: on expiry the kernel sets kErrTimeout in the
// device error word, drains its own copies (again bounded) and returns.
#include <cuda_runtime.h>

#include <cstdint>

#include "soma_device.cuh"
#include "soma_internal.cuh"
#include "soma_launch.h"

namespace soma {

constexpr int kConsumerWarps = 8;
constexpr int kStages = 4;
constexpr int kTileBeads = kConsumerWarps * 64;   // a warp holds at most 64 beads
constexpr int kTileChains = kConsumerWarps * 32;  // at most 32 chains per warp (P = 1)
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz: a wait that long is an error

struct __align__(128) MoveStage {
  float x[kTileBeads];
  float y[kTileBeads];
  float z[kTileBeads];
  uint32_t cid[kTileChains];
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Wait for the phase of the given parity to complete, at most kWaitCycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicOr(err, kErrTimeout);
      return false;
    }
  }
  return true;
}

// One-dimensional bulk copy global -> shared (16-byte aligned, multiple of
// 16 bytes), completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t round16(uint32_t b) { return (b + 15u) & ~15u; }

__device__ __forceinline__ int cell_idx(const MoveArgs& a, float x, float y, float z) {
  return (cell_axis(x, a.cps[0], a.n[0]) * a.n[1] + cell_axis(y, a.cps[1], a.n[1])) * a.n[2] +
         cell_axis(z, a.cps[2], a.n[2]);
}

__global__ void __launch_bounds__((kConsumerWarps + 1) * 32)
    k_move(const __grid_constant__ MoveArgs a, int step_offset) {
  __shared__ MoveStage stage[kStages];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == kConsumerWarps) {
    // ---------------- producer warp: lane 0 streams the tiles ----------------
    if (lane == 0) {
      int it = 0;
      for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
        const int s = it % kStages;
        if (it >= kStages && !mbar_wait(&empty[s], (uint32_t)((it / kStages) - 1) & 1u, a.err)) break;
        const int c0 = tile * a.chains_per_tile;
        const int nch = min(a.chains_per_tile, a.n_poly - c0);
        const int64_t b0 = (int64_t)c0 * a.N;
        const uint32_t pbytes = round16((uint32_t)(nch * a.N) * 4u);
        const uint32_t cbytes = round16((uint32_t)nch * 4u);
        mbar_expect_tx(&full[s], 3u * pbytes + cbytes);
        bulk_g2s(stage[s].x, a.x + b0, pbytes, &full[s]);
        bulk_g2s(stage[s].y, a.y + b0, pbytes, &full[s]);
        bulk_g2s(stage[s].z, a.z + b0, pbytes, &full[s]);
        bulk_g2s(stage[s].cid, a.chain_id + c0, cbytes, &full[s]);
      }
      // no copy may still be in flight when the CTA exits
      const int issued = it;
      for (int j = issued - kStages < 0 ? 0 : issued - kStages; j < issued; ++j)
        if (!mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u, a.err)) break;
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const uint32_t t = (uint32_t)(*a.step_base + (long long)step_offset);
  const int P = a.P, N = a.N;
  const int k = lane & (P - 1);
  const int chain_in_tile = warp * (32 / P) + lane / P;
  const int e = 2 * k, o = 2 * k + 1;
  const int te = e < a.n_A ? 0 : 1, to = o < a.n_A ? 0 : 1;
  const float* __restrict__ wte = a.w + (te ? a.n_c : 0);
  const float* __restrict__ wto = a.w + (to ? a.n_c : 0);
  uint32_t* __restrict__ cnt = a.counts + (size_t)(t & 1u) * 2 * a.n_c;
  const float wR0 = (o < N) ? 1.f : 0.f;          // even bead has a right neighbour
  const float wL0 = (k > 0) ? 1.f : 0.f;          // even bead has a left neighbour
  const float wR1 = (o + 1 < N) ? 1.f : 0.f;      // odd bead has a right neighbour
  unsigned nacc = 0;

  int it = 0;
  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
    const int s = it % kStages;
    if (!mbar_wait(&full[s], (uint32_t)(it / kStages) & 1u, a.err)) break;
    const int c0 = tile * a.chains_per_tile;
    const int nch = min(a.chains_per_tile, a.n_poly - c0);
    const bool chain_ok = chain_in_tile < nch;
    const bool he = chain_ok && e < N, ho = chain_ok && o < N;
    const int lb = chain_in_tile * N + e;  // bead e within the tile
    float xe = 0.f, ye = 0.f, ze = 0.f, xo = 0.f, yo = 0.f, zo = 0.f;
    const MoveStage& st = stage[s];
    if ((N & 1) == 0) {
      if (he) {
        const float2 vx = *reinterpret_cast<const float2*>(st.x + lb);
        const float2 vy = *reinterpret_cast<const float2*>(st.y + lb);
        const float2 vz = *reinterpret_cast<const float2*>(st.z + lb);
        xe = vx.x; xo = vx.y; ye = vy.x; yo = vy.y; ze = vz.x; zo = vz.y;
      }
    } else {
      if (he) { xe = st.x[lb]; ye = st.y[lb]; ze = st.z[lb]; }
      if (ho) { xo = st.x[lb + 1]; yo = st.y[lb + 1]; zo = st.z[lb + 1]; }
    }
    const uint32_t cid = chain_ok ? st.cid[chain_in_tile] : 0u;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with the stage

    // ---- proposals of both beads, then all four field gathers ----
    const uint4 re = philox10(make_uint4((uint32_t)e, cid, t, (uint32_t)a.sys_index), a.rk);
    const uint4 ro = philox10(make_uint4((uint32_t)o, cid, t, (uint32_t)a.sys_index), a.rk);
    const float dex = a.A * fmaf((float)(re.x >> 8), 0x1p-23f, -1.0f);
    const float dey = a.A * fmaf((float)(re.y >> 8), 0x1p-23f, -1.0f);
    const float dez = a.A * fmaf((float)(re.z >> 8), 0x1p-23f, -1.0f);
    const float dox = a.A * fmaf((float)(ro.x >> 8), 0x1p-23f, -1.0f);
    const float doy = a.A * fmaf((float)(ro.y >> 8), 0x1p-23f, -1.0f);
    const float doz = a.A * fmaf((float)(ro.z >> 8), 0x1p-23f, -1.0f);
    int wx, wy, wz;
    const float pex = wrap_coord(xe + dex, a.L[0], wx);
    const float pey = wrap_coord(ye + dey, a.L[1], wy);
    const float pez = wrap_coord(ze + dez, a.L[2], wz);
    const int wrap_e = (wx + 1) | ((wy + 1) << 2) | ((wz + 1) << 4);
    const float pox = wrap_coord(xo + dox, a.L[0], wx);
    const float poy = wrap_coord(yo + doy, a.L[1], wy);
    const float poz = wrap_coord(zo + doz, a.L[2], wz);
    const int wrap_o = (wx + 1) | ((wy + 1) << 2) | ((wz + 1) << 4);
    const int ce0 = cell_idx(a, xe, ye, ze), ce1 = cell_idx(a, pex, pey, pez);
    const int co0 = cell_idx(a, xo, yo, zo), co1 = cell_idx(a, pox, poy, poz);
    const float fe = __ldg(wte + ce1) - __ldg(wte + ce0);
    const float fo = __ldg(wto + co1) - __ldg(wto + co0);

    // ---- set 0: even bead, bonds to 2k-1 (lane k-1) and 2k+1 (own) ----
    const float lx = __shfl_up_sync(0xffffffffu, xo, 1, P);
    const float ly = __shfl_up_sync(0xffffffffu, yo, 1, P);
    const float lz = __shfl_up_sync(0xffffffffu, zo, 1, P);
    const float bLx = min_image(xe - lx, a.L[0], a.invL[0]);
    const float bLy = min_image(ye - ly, a.L[1], a.invL[1]);
    const float bLz = min_image(ze - lz, a.L[2], a.invL[2]);
    const float bRx = min_image(xe - xo, a.L[0], a.invL[0]);
    const float bRy = min_image(ye - yo, a.L[1], a.invL[1]);
    const float bRz = min_image(ze - zo, a.L[2], a.invL[2]);
    {
      const float sx = fmaf(wL0, bLx, wR0 * bRx), sy = fmaf(wL0, bLy, wR0 * bRy), sz = fmaf(wL0, bLz, wR0 * bRz);
      const float d2 = fmaf(dex, dex, fmaf(dey, dey, dez * dez));
      const float dEb = fmaf(2.f, fmaf(dex, sx, fmaf(dey, sy, dez * sz)), (wL0 + wR0) * d2);
      const float dE = fmaf(a.kb, dEb, fe);
      // accept iff dE + ln u < 0, u = ((r3 >> 9) + 1/2) 2^-23 in (0, 1)
      const float u = fmaf((float)(re.w >> 9), 0x1p-23f, 0x1p-24f);
      const bool acc = he && (dE + __logf(u) < 0.f);
      // displacement actually applied to bead e (0 if rejected)
      const float ax = acc ? dex : 0.f, ay = acc ? dey : 0.f, az = acc ? dez : 0.f;
      if (acc) {
        xe = pex; ye = pey; ze = pez;
      }
      nacc += acc;
      // ---- set 1: odd bead, bonds to 2k (own, moved by a) and 2k+2 (lane k+1) ----
      // o - e_k' = -(bR + a_k);  o - e_{k+1}' = -(bL_{k+1} + a_{k+1})
      const float qx = __shfl_down_sync(0xffffffffu, bLx + ax, 1, P);
      const float qy = __shfl_down_sync(0xffffffffu, bLy + ay, 1, P);
      const float qz = __shfl_down_sync(0xffffffffu, bLz + az, 1, P);
      const float ox = -fmaf(wR1, qx, bRx + ax), oy = -fmaf(wR1, qy, bRy + ay), oz = -fmaf(wR1, qz, bRz + az);
      const float o2 = fmaf(dox, dox, fmaf(doy, doy, doz * doz));
      const float dEbo = fmaf(2.f, fmaf(dox, ox, fmaf(doy, oy, doz * oz)), (1.f + wR1) * o2);
      const float dEo = fmaf(a.kb, dEbo, fo);
      const float uo = fmaf((float)(ro.w >> 9), 0x1p-23f, 0x1p-24f);
      const bool acco = ho && (dEo + __logf(uo) < 0.f);
      if (acco) {
        xo = pox; yo = poy; zo = poz;
      }
      nacc += acco;

      // ---- write back, images on wrap, fused histogram ----
      const int64_t gb = (int64_t)c0 * N + lb;
      if ((N & 1) == 0) {
        if (he && (acc || acco)) {
          *reinterpret_cast<float2*>(a.x + gb) = make_float2(xe, xo);
          *reinterpret_cast<float2*>(a.y + gb) = make_float2(ye, yo);
          *reinterpret_cast<float2*>(a.z + gb) = make_float2(ze, zo);
        }
      } else {
        if (acc) { a.x[gb] = xe; a.y[gb] = ye; a.z[gb] = ze; }
        if (acco) { a.x[gb + 1] = xo; a.y[gb + 1] = yo; a.z[gb + 1] = zo; }
      }
      if (acc && wrap_e != 21) apply_wrap(a.img, gb, wrap_e);
      if (acco && wrap_o != 21) apply_wrap(a.img, gb + 1, wrap_o);
      if (a.bin) {
        if (he) atomicAdd(cnt + (te ? a.n_c : 0) + (acc ? ce1 : ce0), 1u);
        if (ho) atomicAdd(cnt + (to ? a.n_c : 0) + (acco ? co1 : co0), 1u);
      }
    }
  }

  nacc = __reduce_add_sync(0xffffffffu, nacc);
  if (lane == 0 && nacc) atomicAdd(a.acc + blockIdx.x, (unsigned long long)nacc);
}

int move_kernel_max_ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move, (kConsumerWarps + 1) * 32, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

int move_kernel_chains_per_tile(int P) { return kConsumerWarps * (32 / P); }

cudaError_t launch_move(const MoveArgs& a, int grid, int step_offset, cudaStream_t s) {
  k_move<<<grid, (kConsumerWarps + 1) * 32, 0, s>>>(a, step_offset);
  return cudaGetLastError();
}

}  // namespace soma
