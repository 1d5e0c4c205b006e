// soma_move.cu -- kernel (a) of the SCMF step with the histogram (b) and the
// field evaluation (c) folded in: the biased trial moves and energy
// evaluations of the move kernel profiled in Sec. 2.2, for chains of up to 64
// beads.
//
// Design (constants in the parameter bank):
//  * persistent CTAs, warp-specialised: one producer warp streams each
//    tile's positions (x, y, z) and logical chain ids from HBM into a ring of
//    kStages shared-memory stages with cp.async.bulk, completion tracked by
//    mbarriers; W consumer warps compute (W = 8, 12 or 24: the single-system
//    kernel is built for all three and the autotuner picks one per workload,
//    the batch kernel uses 8);
//  * a consumer lane k of a chain holds beads 2k (even set) and 2k+1 (odd
//    set); neighbours come from the adjacent lane by width-P shuffles;
//  * both beads' proposals are formed first, so the four gathers of the lane
//    (old and proposed cell of each bead) go out together; their arithmetic
//    runs as packed FP32x2 pairs (each lane rounded as the scalar operation);
//  * set 0 (even beads) is decided first; set 1 reuses set 0's bond vectors
//    plus the accepted displacement, so no second minimum image is needed;
//  * the field term of a move comes straight from the integer counts of the
//    previous step: for a bead of type t the field difference between cells
//    c1 and c0 is
//      (1/rho) [chiN/N (n_other(c1) - n_other(c0)) + kappaN/N (n(c1) - n(c0))]
//    with exact integer differences, one 8-byte gather per cell; held or
//    coupling-supplied fields are read from the field array instead;
//  * new positions go straight back to global memory; the final cells are
//    added to count buffer t mod 3 by fire-and-forget atomics (kernel (b)),
//    and the CTAs clear count buffer t+1 mod 3 for the next step.
// k_move steps one system; k_move_batch steps up to kMaxBatch systems in one
// persistent launch (tiles of all systems in one sequence).  Both are
// specialised on the proposal (uniform, or bond-force-biased: smart_pair)
// and on the z boundary (periodic, or hard walls: a proposal leaving the
// slab is rejected, z bonds are plain differences); k_move also on molecule
// types (boundary-zone conversion: each step opens with the conversions of
// the chains whose bead 0 lies in a zone, decided by the chain's bead-0
// lane; a bead's type follows the A block of its chain's type, carried in
// the chain-id word's top bit).
// Every mbarrier wait is bounded: on expiry the kernel sets kErrTimeout in the
// device error word, drains its own copies (again bounded) and returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "soma_device.cuh"
#include "soma_internal.cuh"
#include "soma_launch.h"

namespace soma {

constexpr int kStages = 4;
constexpr int kBatchWarps = 8;  // consumer warps of the batch kernel
// Resident CTAs per SM the register budget (72) is for: 3 of 8 + 1 warps,
// 2 of 12 + 1, 1 of 24 + 1.
template <int W>
constexpr int move_min_blocks() { return W <= 8 ? 3 : (W <= 12 ? 2 : 1); }
// A tile's bulk copies start at chain c0 = tile * W * 32/P and bead c0 * N;
// both addresses are 16-byte aligned for every P and N only when the chains
// per tile are a multiple of 4 (P = 32: W itself).
template <int W>
constexpr bool tile_copies_aligned() { return W % 4 == 0; }
constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz: a wait that long is an error
constexpr float kLog2e = 1.4426950408889634f;

// A batch rides in the kernel's parameter space (at most 32,764 bytes).
static_assert(sizeof(BatchArgs) <= 32000, "BatchArgs exceeds the kernel parameter limit");

// A tile of W warps: at most 64 beads per warp, at most 32 chains (P = 1).
template <int W>
struct __align__(128) MoveStage {
  static_assert(tile_copies_aligned<W>(), "tile copies would start off a 16-byte boundary");
  float x[W * 64];
  float y[W * 64];
  float z[W * 64];
  uint32_t cid[W * 32];
  uint32_t sys;  // batched launches: the tile's system, written by the producer
  uint32_t pad[3];
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

// Wait for the phase of the given parity to complete, at most `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err,
                                          long long limit = kWaitCycles) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(bar, parity)) {
    if (clock64() - t0 > limit) {
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

// The stage ring of a W-warp CTA: static shared memory up to the 48 KiB a
// static allocation may take (8 and 12 warps), dynamic shared memory above
// it (24 warps: 86,592 bytes, opted in per kernel by set_move_smem_limit).
constexpr size_t kStaticSmemLimit = 48 * 1024;
template <int W>
__host__ __device__ constexpr size_t move_ring_bytes() { return kStages * sizeof(MoveStage<W>); }
template <int W>
__host__ __device__ constexpr size_t move_dynamic_smem() {
  return move_ring_bytes<W>() <= kStaticSmemLimit ? 0 : move_ring_bytes<W>();
}

template <int W>
__device__ __forceinline__ MoveStage<W>* move_ring() {
  if constexpr (move_dynamic_smem<W>() == 0) {
    __shared__ MoveStage<W> ring[kStages];
    return ring;
  } else {
    extern __shared__ __align__(128) unsigned char move_dyn_smem[];
    return reinterpret_cast<MoveStage<W>*>(move_dyn_smem);
  }
}

// Stage reads as volatile shared loads: each is performed exactly once, in
// program order before the warp releases the stage to the producer.  (A
// plain load may legally be re-executed later by the compiler to save a
// register, and after the release the stage may already hold the next tile,
// written by the copy engine outside the compiler's view.)  Keep them
// volatile: an earlier build with plain stage loads under a tighter register
// cap gave trajectories that changed with the number of resident CTAs per SM
// -- a stage value re-read after the early release, once the producer had
// refilled the stage, fits that symptom exactly.
__device__ __forceinline__ float2 lds2(const float* p) {
  float2 v;
  asm volatile("ld.volatile.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ float lds1(const float* p) {
  float v;
  asm volatile("ld.volatile.shared.f32 %0, [%1];" : "=f"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lds1(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}

// Periodic wrap of a proposed coordinate p in (-L, 2L) into [0, L): the
// image step fl in {-1, 0, 1}, then p - fl L, kept strictly below L (p just
// below 0 would round to L; the largest float below L, Lm, is the same
// point to within rounding and lies in the last cell, as the exact wrap
// does).  For fl = 1 the subtraction is exact.
__device__ __forceinline__ float wrap_step(float p, float L, float Lm, float& fl) {
  fl = p >= L ? 1.f : (p < 0.f ? -1.f : 0.f);
  return fminf(fmaf(-L, fl, p), Lm);
}

// Image steps of the three axes packed as fx + 3 fy + 9 fz (balanced
// ternary: zero only when nothing wrapped), applied in the rare case.
__device__ __forceinline__ void apply_image_steps(int16_t* img, int64_t bead, float code, int* err) {
  if (code != 0.f) {
    const int c = __float2int_rn(code) + 13;  // 0 .. 26, digits fx+1, fy+1, fz+1
    short4* p = reinterpret_cast<short4*>(img) + bead;
    short4 v = *p;
#ifdef SOMA_DEBUG
    // checked build: an image counter about to leave the int16 range
    if (v.x <= -32767 || v.x >= 32767 || v.y <= -32767 || v.y >= 32767 || v.z <= -32767 || v.z >= 32767)
      atomicOr(err, kErrBounds);
#endif
    v.x += (short)(c % 3 - 1);
    v.y += (short)((c / 3) % 3 - 1);
    v.z += (short)(c / 9 - 1);
    *p = v;
  }
}

// wrap_step of two coordinates of the same axis, the FMA packed.
__device__ __forceinline__ float2 wrap_step2(float2 p, float L, float Lm, float2& fl) {
  fl.x = p.x >= L ? 1.f : (p.x < 0.f ? -1.f : 0.f);
  fl.y = p.y >= L ? 1.f : (p.y < 0.f ? -1.f : 0.f);
  const float2 q = __ffma2_rn(make_float2(-L, -L), fl, p);
  return make_float2(fminf(q.x, Lm), fminf(q.y, Lm));
}

// Cells of two positions, the scalings packed.
__device__ __forceinline__ int2 cell_idx2(const MoveArgs& a, float2 x, float2 y, float2 z) {
  const float2 sx = __fmul2_rn(x, make_float2(a.cps[0], a.cps[0]));
  const float2 sy = __fmul2_rn(y, make_float2(a.cps[1], a.cps[1]));
  const float2 sz = __fmul2_rn(z, make_float2(a.cps[2], a.cps[2]));
  const int n0 = a.n[0] - 1, n1 = a.n[1] - 1, n2 = a.n[2] - 1;
  return make_int2((min((int)sx.x, n0) * a.n[1] + min((int)sy.x, n1)) * a.n[2] + min((int)sz.x, n2),
                   (min((int)sx.y, n0) * a.n[1] + min((int)sy.y, n1)) * a.n[2] + min((int)sz.y, n2));
}

__device__ __forceinline__ int cell_idx(const MoveArgs& a, float x, float y, float z) {
  return (cell_axis(x, a.cps[0], a.n[0]) * a.n[1] + cell_axis(y, a.cps[1], a.n[1])) * a.n[2] +
         cell_axis(z, a.cps[2], a.n[2]);
}

// Producer: issue the copies of tile `tile` (local to system a) into stage st.
template <int W>
__device__ __forceinline__ void produce_tile(const MoveArgs& a, int tile, MoveStage<W>& st, uint64_t* full) {
  const int c0 = tile * a.chains_per_tile;
  const int nch = min(a.chains_per_tile, a.n_poly - c0);
  const int64_t b0 = (int64_t)c0 * a.N;
  const uint32_t pbytes = round16((uint32_t)(nch * a.N) * 4u);
  const uint32_t cbytes = round16((uint32_t)nch * 4u);
  mbar_expect_tx(full, 3u * pbytes + cbytes);
  bulk_g2s(st.x, a.x + b0, pbytes, full);
  bulk_g2s(st.y, a.y + b0, pbytes, full);
  bulk_g2s(st.z, a.z + b0, pbytes, full);
  bulk_g2s(st.cid, a.chain_id + c0, cbytes, full);
}

// Field difference w_t(c1) - w_t(c0) for a bead of type t from the integer
// counts n0 = (nA, nB) of c0 and n1 of c1 (the chi term couples to the other
// type's count, the kappa term to the total).
__device__ __forceinline__ float field_from_counts(const MoveArgs& a, int type, uint2 n0, uint2 n1) {
  const int d_other = type ? (int)(n1.x - n0.x) : (int)(n1.y - n0.y);
  const int d_tot = (int)(n1.x + n1.y) - (int)(n0.x + n0.y);
  return a.inv_rho * fmaf(a.chiN_N, (float)d_other, a.kappaN_N * (float)d_tot);
}

// field_from_counts of the lane's two beads, the arithmetic packed.
__device__ __forceinline__ float2 fields_from_counts2(const MoveArgs& a, int te, int to, uint2 ne0, uint2 ne1,
                                                      uint2 no0, uint2 no1) {
  const int de_other = te ? (int)(ne1.x - ne0.x) : (int)(ne1.y - ne0.y);
  const int do_other = to ? (int)(no1.x - no0.x) : (int)(no1.y - no0.y);
  const int de_tot = (int)(ne1.x + ne1.y) - (int)(ne0.x + ne0.y);
  const int do_tot = (int)(no1.x + no1.y) - (int)(no0.x + no0.y);
  const float2 k = __fmul2_rn(make_float2(a.kappaN_N, a.kappaN_N), make_float2((float)de_tot, (float)do_tot));
  const float2 f = __ffma2_rn(make_float2(a.chiN_N, a.chiN_N), make_float2((float)de_other, (float)do_other), k);
  return __fmul2_rn(make_float2(a.inv_rho, a.inv_rho), f);
}

// Standard normal deviate of a Philox word: Phi^-1(((w >> 8) + 1/2) 2^-24).
// The argument is formed exactly in FP32 by evaluating the lower tail of
// whichever half of (0, 1) it falls in (Phi^-1(1 - v) = -Phi^-1(v)).  (A
// degree-(4, 4) rational in sqrt(-2 ln v) fitted for this purpose was no
// faster than the library's normcdfinvf on the melt of 131,072 chains of 32
// beads, 71.5 against 70.7 us.)
__device__ __forceinline__ float normal_of_word(uint32_t w) {
  const uint32_t m = w >> 8;
  const bool upper = m >= (1u << 23);
  const uint32_t odd = upper ? (0x2000000u - 2u * m - 1u) : (2u * m + 1u);  // odd < 2^24: exact
  const float v = normcdfinvf((float)odd * 0x1p-25f);
  return upper ? -v : v;
}

// Verification aid: the deviates of n words (the function above, as the
// smart-move kernel evaluates it).
__global__ void k_normal_words(const uint32_t* __restrict__ w, float* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = normal_of_word(w[i]);
}

cudaError_t launch_normal_words(const uint32_t* w, float* out, int64_t n, cudaStream_t s) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 16);
  k_normal_words<<<(int)std::max<int64_t>(blocks, 1), 256, 0, s>>>(w, out, n);
  return cudaGetLastError();
}

// z component of a bond vector: minimum image, or the plain difference
// between hard walls (kWall: z is not periodic).
template <bool kWall>
__device__ __forceinline__ float bond_z(float d, const MoveArgs& a) {
  return kWall ? d : min_image(d, a.L[2], a.invL[2]);
}

// Proposed z of the two beads: wrapped into [0, L) (periodic), or, between
// walls, kept where it is when it would leave [0, L) (in_e / in_o false: the
// move is rejected; the old z keeps the cell lookup inside the grid).
template <bool kWall>
__device__ __forceinline__ float2 propose_z(const MoveArgs& a, float ze, float zo, float2 dZ, float2& fZ, bool& in_e,
                                            bool& in_o) {
  const float2 q = __fadd2_rn(make_float2(ze, zo), dZ);
  if (kWall) {
    in_e = q.x >= 0.f && q.x < a.L[2];
    in_o = q.y >= 0.f && q.y < a.L[2];
    fZ = make_float2(0.f, 0.f);
    return make_float2(in_e ? q.x : ze, in_o ? q.y : zo);
  }
  in_e = in_o = true;
  return wrap_step2(q, a.L[2], a.Lm[2], fZ);
}

// The bead pair of one lane: positions in, decisions, final cells and image
// codes out.  Uniform proposals (Sec. 2, the SOMA paragraph: the MC propagation of beads).
template <bool kFromCounts, bool kWall>
__device__ __forceinline__ void uniform_pair(const MoveArgs& a, long long tl, const uint2* __restrict__ prev,
                                             uint32_t cid, int k, int e, int o,
                                             int te, int to, bool he, bool ho, float& xe, float& ye, float& ze,
                                             float& xo, float& yo, float& zo, bool& acc, bool& acco, int& ce,
                                             int& co, float& wrap_e, float& wrap_o) {
  const uint32_t t = (uint32_t)tl;
  const int P = a.P, N = a.N;
  // ---- proposals of both beads, then all four gathers ----
  const uint4 re = philox10(make_uint4((uint32_t)e, cid, t, (uint32_t)a.sys_index), a.rk);
  const uint4 ro = philox10(make_uint4((uint32_t)o, cid, t, (uint32_t)a.sys_index), a.rk);
  // d = A (2 U - 1) = A ((w >> 8) 2^-23 - 1): the bracket is exact in FP32,
  // so one FMA with A 2^-23 and -A rounds the same exact value once
  const float A23 = a.A * 0x1p-23f;
  // the two beads' arithmetic runs as packed pairs (Blackwell FP32x2 ops,
  // each lane rounded exactly as the scalar operation)
  const float2 A23v = make_float2(A23, A23), mA = make_float2(-a.A, -a.A);
  const float2 dX = __ffma2_rn(make_float2((float)(re.x >> 8), (float)(ro.x >> 8)), A23v, mA);
  const float2 dY = __ffma2_rn(make_float2((float)(re.y >> 8), (float)(ro.y >> 8)), A23v, mA);
  const float2 dZ = __ffma2_rn(make_float2((float)(re.z >> 8), (float)(ro.z >> 8)), A23v, mA);
  const float dex = dX.x, dey = dY.x, dez = dZ.x, dox = dX.y, doy = dY.y, doz = dZ.y;
  float2 fX, fY, fZ;
  const float2 pX = wrap_step2(__fadd2_rn(make_float2(xe, xo), dX), a.L[0], a.Lm[0], fX);
  const float2 pY = wrap_step2(__fadd2_rn(make_float2(ye, yo), dY), a.L[1], a.Lm[1], fY);
  bool in_e, in_o;
  const float2 pZ = propose_z<kWall>(a, ze, zo, dZ, fZ, in_e, in_o);
  const float2 wr = __ffma2_rn(make_float2(9.f, 9.f), fZ, __ffma2_rn(make_float2(3.f, 3.f), fY, fX));
  wrap_e = wr.x;
  wrap_o = wr.y;
  const float pex = pX.x, pey = pY.x, pez = pZ.x, pox = pX.y, poy = pY.y, poz = pZ.y;
  const int2 c_old = cell_idx2(a, make_float2(xe, xo), make_float2(ye, yo), make_float2(ze, zo));
  const int2 c_new = cell_idx2(a, pX, pY, pZ);
  const int ce0 = c_old.x, co0 = c_old.y, ce1 = c_new.x, co1 = c_new.y;
  float fe, fo;
  if (kFromCounts) {
    const uint2 ne0 = __ldg(prev + ce0), ne1 = __ldg(prev + ce1);
    const uint2 no0 = __ldg(prev + co0), no1 = __ldg(prev + co1);
    const float2 f = fields_from_counts2(a, te, to, ne0, ne1, no0, no1);
    fe = f.x;
    fo = f.y;
  } else {
    const float* __restrict__ wte = a.w + (te ? a.n_c : 0);
    const float* __restrict__ wto = a.w + (to ? a.n_c : 0);
    fe = __ldg(wte + ce1) - __ldg(wte + ce0);
    fo = __ldg(wto + co1) - __ldg(wto + co0);
  }

  // ---- set 0: even bead, bonds to 2k-1 (lane k-1) and 2k+1 (own) ----
  const float wR0 = (o < N) ? 1.f : 0.f;      // even bead has a right neighbour
  const float wL0 = (k > 0) ? 1.f : 0.f;      // even bead has a left neighbour
  const float wR1 = (o + 1 < N) ? 1.f : 0.f;  // odd bead has a right neighbour
  const float lx = __shfl_up_sync(0xffffffffu, xo, 1, P);
  const float ly = __shfl_up_sync(0xffffffffu, yo, 1, P);
  const float lz = __shfl_up_sync(0xffffffffu, zo, 1, P);
  const float bLx = min_image(xe - lx, a.L[0], a.invL[0]);
  const float bLy = min_image(ye - ly, a.L[1], a.invL[1]);
  const float bLz = bond_z<kWall>(ze - lz, a);
  const float bRx = min_image(xe - xo, a.L[0], a.invL[0]);
  const float bRy = min_image(ye - yo, a.L[1], a.invL[1]);
  const float bRz = bond_z<kWall>(ze - zo, a);
  const float sx = fmaf(wL0, bLx, wR0 * bRx), sy = fmaf(wL0, bLy, wR0 * bRy), sz = fmaf(wL0, bLz, wR0 * bRz);
  const float d2 = fmaf(dex, dex, fmaf(dey, dey, dez * dez));
  const float dEb = fmaf(2.f, fmaf(dex, sx, fmaf(dey, sy, dez * sz)), (wL0 + wR0) * d2);
  const float dE = fmaf(a.kb, dEb, fe);
  // accept iff dE + ln u < 0, u = ((r3 >> 9) + 1/2) 2^-23 in (0, 1),
  // evaluated as dE log2(e) + log2(u) < 0
  const float u = fmaf((float)(re.w >> 9), 0x1p-23f, 0x1p-24f);
  acc = he && in_e && (fmaf(dE, kLog2e, __log2f(u)) < 0.f);
  // displacement actually applied to bead e (0 if rejected)
  const float ax = acc ? dex : 0.f, ay = acc ? dey : 0.f, az = acc ? dez : 0.f;
  if (acc) {
    xe = pex; ye = pey; ze = pez;
  }
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
  acco = ho && in_o && (fmaf(dEo, kLog2e, __log2f(uo)) < 0.f);
  if (acco) {
    xo = pox; yo = poy; zo = poz;
  }
  ce = acc ? ce1 : ce0;
  co = acco ? co1 : co0;
}

// Bond-force-biased proposals (the smart moves named in Sec. 2): bead i is
// displaced by d = -drift s + sig xi, with s the sum of its bond vectors
// (the bond force is F = -2 k_b s, so -drift s = (s2/2) F), xi standard
// normal from Philox words x, y, z, and the Metropolis margin gains
//   ln q(r -> r') - ln q(r' -> r) = (|b|^2 - |f|^2) / (2 s2),
// f = sig xi the forward residual, b = -d + drift (s + n d) the reverse one
// (n bonds).  The odd bead's force depends on set 0's outcome, so its
// proposal and its new-cell gather follow the even bead's decision.  Every
// bond vector is minimum-imaged, so |s| <= L per axis and, with the bounds
// the host enforces (drift <= k_b A^2/3 <= 1/2, 6 sig < L/2), a proposal
// stays within one image of the box.
template <bool kFromCounts, bool kWall>
__device__ __forceinline__ void smart_pair(const MoveArgs& a, long long tl, const uint2* __restrict__ prev,
                                           uint32_t cid, int k, int e, int o,
                                           int te, int to, bool he, bool ho, float& xe, float& ye, float& ze,
                                           float& xo, float& yo, float& zo, bool& acc, bool& acco, int& ce,
                                           int& co, float& wrap_e, float& wrap_o) {
  const uint32_t t = (uint32_t)tl;
  const int P = a.P, N = a.N;
  const uint4 re = philox10(make_uint4((uint32_t)e, cid, t, (uint32_t)a.sys_index), a.rk);
  const uint4 ro = philox10(make_uint4((uint32_t)o, cid, t, (uint32_t)a.sys_index), a.rk);
  const float wR0 = (o < N) ? 1.f : 0.f;
  const float wL0 = (k > 0) ? 1.f : 0.f;
  const float wR1 = (o + 1 < N) ? 1.f : 0.f;
  // ---- set 0: even bead ----
  const float lx = __shfl_up_sync(0xffffffffu, xo, 1, P);
  const float ly = __shfl_up_sync(0xffffffffu, yo, 1, P);
  const float lz = __shfl_up_sync(0xffffffffu, zo, 1, P);
  const float bLx = min_image(xe - lx, a.L[0], a.invL[0]);
  const float bLy = min_image(ye - ly, a.L[1], a.invL[1]);
  const float bLz = bond_z<kWall>(ze - lz, a);
  const float bRx = min_image(xe - xo, a.L[0], a.invL[0]);
  const float bRy = min_image(ye - yo, a.L[1], a.invL[1]);
  const float bRz = bond_z<kWall>(ze - zo, a);
  const float sx = fmaf(wL0, bLx, wR0 * bRx), sy = fmaf(wL0, bLy, wR0 * bRy), sz = fmaf(wL0, bLz, wR0 * bRz);
  const float n0 = wL0 + wR0;
  const float fex = a.sig * normal_of_word(re.x);
  const float fey = a.sig * normal_of_word(re.y);
  const float fez = a.sig * normal_of_word(re.z);
  const float dex = fmaf(-a.drift, sx, fex);
  const float dey = fmaf(-a.drift, sy, fey);
  const float dez = fmaf(-a.drift, sz, fez);
  float fx, fy, fz;
  const float pex = wrap_step(xe + dex, a.L[0], a.Lm[0], fx);
  const float pey = wrap_step(ye + dey, a.L[1], a.Lm[1], fy);
  bool in_e = true, in_o = true;
  float pez;
  if (kWall) {
    const float q = ze + dez;
    in_e = q >= 0.f && q < a.L[2];
    pez = in_e ? q : ze;
    fz = 0.f;
  } else {
    pez = wrap_step(ze + dez, a.L[2], a.Lm[2], fz);
  }
  wrap_e = fmaf(9.f, fz, fmaf(3.f, fy, fx));
  const int ce0 = cell_idx(a, xe, ye, ze), ce1 = cell_idx(a, pex, pey, pez);
  const int co0 = cell_idx(a, xo, yo, zo);
  const float* __restrict__ wte = a.w + (te ? a.n_c : 0);
  const float* __restrict__ wto = a.w + (to ? a.n_c : 0);
  float fe;
  uint2 no0 = make_uint2(0u, 0u);
  float wo0 = 0.f;
  if (kFromCounts) {
    const uint2 ne0 = __ldg(prev + ce0), ne1 = __ldg(prev + ce1);
    no0 = __ldg(prev + co0);
    fe = field_from_counts(a, te, ne0, ne1);
  } else {
    fe = __ldg(wte + ce1) - __ldg(wte + ce0);
    wo0 = __ldg(wto + co0);
  }
  {
    const float d2 = fmaf(dex, dex, fmaf(dey, dey, dez * dez));
    const float dEb = fmaf(2.f, fmaf(dex, sx, fmaf(dey, sy, dez * sz)), n0 * d2);
    const float brx = fmaf(a.drift, fmaf(n0, dex, sx), -dex);
    const float bry = fmaf(a.drift, fmaf(n0, dey, sy), -dey);
    const float brz = fmaf(a.drift, fmaf(n0, dez, sz), -dez);
    const float rev = fmaf(brx, brx, fmaf(bry, bry, brz * brz));
    const float fwd = fmaf(fex, fex, fmaf(fey, fey, fez * fez));
    const float dE = fmaf(a.kb, dEb, fe) + (rev - fwd) * a.inv2s2;
    const float u = fmaf((float)(re.w >> 9), 0x1p-23f, 0x1p-24f);
    acc = he && in_e && (fmaf(dE, kLog2e, __log2f(u)) < 0.f);
  }
  const float ax = acc ? dex : 0.f, ay = acc ? dey : 0.f, az = acc ? dez : 0.f;
  if (acc) {
    xe = pex; ye = pey; ze = pez;
  }
  // ---- set 1: odd bead, force from the bonds after set 0 ----
  const float qx = __shfl_down_sync(0xffffffffu, bLx + ax, 1, P);
  const float qy = __shfl_down_sync(0xffffffffu, bLy + ay, 1, P);
  const float qz = __shfl_down_sync(0xffffffffu, bLz + az, 1, P);
  const float ox = fmaf(wR1, min_image(-qx, a.L[0], a.invL[0]), min_image(-(bRx + ax), a.L[0], a.invL[0]));
  const float oy = fmaf(wR1, min_image(-qy, a.L[1], a.invL[1]), min_image(-(bRy + ay), a.L[1], a.invL[1]));
  const float oz = fmaf(wR1, bond_z<kWall>(-qz, a), bond_z<kWall>(-(bRz + az), a));
  const float n1 = 1.f + wR1;
  const float fox = a.sig * normal_of_word(ro.x);
  const float foy = a.sig * normal_of_word(ro.y);
  const float foz = a.sig * normal_of_word(ro.z);
  const float dox = fmaf(-a.drift, ox, fox);
  const float doy = fmaf(-a.drift, oy, foy);
  const float doz = fmaf(-a.drift, oz, foz);
  const float pox = wrap_step(xo + dox, a.L[0], a.Lm[0], fx);
  const float poy = wrap_step(yo + doy, a.L[1], a.Lm[1], fy);
  float poz;
  if (kWall) {
    const float q = zo + doz;
    in_o = q >= 0.f && q < a.L[2];
    poz = in_o ? q : zo;
    fz = 0.f;
  } else {
    poz = wrap_step(zo + doz, a.L[2], a.Lm[2], fz);
  }
  wrap_o = fmaf(9.f, fz, fmaf(3.f, fy, fx));
  const int co1 = cell_idx(a, pox, poy, poz);
  float fo;
  if (kFromCounts)
    fo = field_from_counts(a, to, no0, __ldg(prev + co1));
  else
    fo = __ldg(wto + co1) - wo0;
  {
    const float d2 = fmaf(dox, dox, fmaf(doy, doy, doz * doz));
    const float dEb = fmaf(2.f, fmaf(dox, ox, fmaf(doy, oy, doz * oz)), n1 * d2);
    const float brx = fmaf(a.drift, fmaf(n1, dox, ox), -dox);
    const float bry = fmaf(a.drift, fmaf(n1, doy, oy), -doy);
    const float brz = fmaf(a.drift, fmaf(n1, doz, oz), -doz);
    const float rev = fmaf(brx, brx, fmaf(bry, bry, brz * brz));
    const float fwd = fmaf(fox, fox, fmaf(foy, foy, foz * foz));
    const float dE = fmaf(a.kb, dEb, fo) + (rev - fwd) * a.inv2s2;
    const float u = fmaf((float)(ro.w >> 9), 0x1p-23f, 0x1p-24f);
    acco = ho && in_o && (fmaf(dE, kLog2e, __log2f(u)) < 0.f);
  }
  if (acco) {
    xo = pox; yo = poy; zo = poz;
  }
  ce = acc ? ce1 : ce0;
  co = acco ? co1 : co0;
}

// Consumer warp: one tile of system a at step t.  Reads the stage, releases
// it, moves the even then the odd beads of its chains, writes back, bins.
// Returns the number of accepted moves of this lane.
// prev: count buffer of step t-1 (fields), cur: count buffer of step t (histogram).
template <bool kFromCounts, bool kSmart, bool kWall, bool kConv, int W>
__device__ __forceinline__ unsigned consume_tile(const MoveArgs& a, int tile, const MoveStage<W>& st, uint64_t* empty,
                                                 long long tl, const uint2* __restrict__ prev,
                                                 uint32_t* __restrict__ cur, int warp, int lane) {
  const int P = a.P, N = a.N;
  const int k = lane & (P - 1);
  const int chain_in_tile = warp * (32 / P) + lane / P;
  const int e = 2 * k, o = 2 * k + 1;
  const int c0 = tile * a.chains_per_tile;
  const int nch = min(a.chains_per_tile, a.n_poly - c0);
  const bool chain_ok = chain_in_tile < nch;
  const bool he = chain_ok && e < N, ho = chain_ok && o < N;
  const int lb = chain_in_tile * N + e;  // bead e within the tile
  float xe = 0.f, ye = 0.f, ze = 0.f, xo = 0.f, yo = 0.f, zo = 0.f;
  if ((N & 1) == 0) {
    if (he) {
      const float2 vx = lds2(st.x + lb);
      const float2 vy = lds2(st.y + lb);
      const float2 vz = lds2(st.z + lb);
      xe = vx.x; xo = vx.y; ye = vy.x; yo = vy.y; ze = vz.x; zo = vz.y;
    }
  } else {
    if (he) { xe = lds1(st.x + lb); ye = lds1(st.y + lb); ze = lds1(st.z + lb); }
    if (ho) { xo = lds1(st.x + lb + 1); yo = lds1(st.y + lb + 1); zo = lds1(st.z + lb + 1); }
  }
  const uint32_t cid_word = chain_ok ? lds1(st.cid + chain_in_tile) : 0u;
  __syncwarp();
  if (lane == 0) mbar_arrive(empty);  // this warp is done with the stage
  // bead types: the A block of the chain's molecule type (with conversion
  // on, the chain-id word's top bit; the random numbers follow the id alone)
  uint32_t cid = cid_word;
  int n_A = a.n_A;
  if (kConv) {
    // boundary zones (Sec. 3.2): the step opens with the conversions.  The
    // chain's bead-0 lane (k = 0) holds bead 0's stored z: in a zone, it
    // draws word 0 of counter (kConvWord, id, t, system) and flips the type
    // if the word is below the zone's threshold for the current type; the
    // chain's other lanes take the new word by a width-P shuffle.
    uint32_t word = cid_word;
    const bool in_lo = ze < a.zone_lo, in_hi = ze >= a.zone_hi;
    const bool cand = he && k == 0 && (in_lo || in_hi);
    if (__any_sync(0xffffffffu, cand)) {
      int slot_conv = -1;  // 0..3 when this lane's chain converts
      if (cand) {
        const int zone = in_lo ? 0 : 1, m = (word & kTypeBit) ? 1 : 0;
        const uint4 w = philox10(make_uint4(kConvWord, word & kIdMask, (uint32_t)tl, (uint32_t)a.sys_index), a.rk);
        if ((unsigned long long)w.x < a.thr[2 * zone + m]) {
          word ^= kTypeBit;
          a.chain_id[c0 + chain_in_tile] = word;
          slot_conv = 2 * zone + m;
        }
      }
      word = __shfl_sync(0xffffffffu, word, 0, P);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int n_q = __popc(__ballot_sync(0xffffffffu, slot_conv == q));
        if (lane == 0 && n_q) atomicAdd(a.conv_count + q, (unsigned long long)n_q);
      }
    }
    cid = word & kIdMask;
    if (word & kTypeBit) n_A = a.n_A_alt;
  }
  const int te = e < n_A ? 0 : 1, to = o < n_A ? 0 : 1;

  bool acc, acco;
  int ce, co;
  float wrap_e, wrap_o;
  if (kSmart)
    smart_pair<kFromCounts, kWall>(a, tl, prev, cid, k, e, o, te, to, he, ho, xe, ye, ze, xo, yo, zo, acc, acco, ce,
                                   co, wrap_e, wrap_o);
  else
    uniform_pair<kFromCounts, kWall>(a, tl, prev, cid, k, e, o, te, to, he, ho, xe, ye, ze, xo, yo, zo, acc, acco,
                                     ce, co, wrap_e, wrap_o);

#ifdef SOMA_DEBUG
  // checked build: final cells inside the grid, positions finite in [0, L)
  if ((he && (ce < 0 || ce >= a.n_c || !(xe >= 0.f && xe < a.L[0] && ye >= 0.f && ye < a.L[1] && ze >= 0.f &&
                                          ze < a.L[2]))) ||
      (ho && (co < 0 || co >= a.n_c || !(xo >= 0.f && xo < a.L[0] && yo >= 0.f && yo < a.L[1] && zo >= 0.f &&
                                          zo < a.L[2]))))
    atomicOr(a.err, kErrBounds);
#endif
  // ---- write back, images on wrap, fused histogram ----
  const int64_t gb = (int64_t)c0 * N + lb;
  if ((N & 1) == 0) {
    if (he) {  // unconditional: a rejected pair rewrites its own values, no branch on the outcome
      *reinterpret_cast<float2*>(a.x + gb) = make_float2(xe, xo);
      *reinterpret_cast<float2*>(a.y + gb) = make_float2(ye, yo);
      *reinterpret_cast<float2*>(a.z + gb) = make_float2(ze, zo);
    }
  } else {
    if (acc) { a.x[gb] = xe; a.y[gb] = ye; a.z[gb] = ze; }
    if (acco) { a.x[gb + 1] = xo; a.y[gb + 1] = yo; a.z[gb + 1] = zo; }
  }
  // image counters change only when an accepted move crossed the box: one
  // warp vote skips the update in the common case
  if (__any_sync(0xffffffffu, (acc && wrap_e != 0.f) || (acco && wrap_o != 0.f))) {
    if (acc) apply_image_steps(a.img, gb, wrap_e, a.err);
    if (acco) apply_image_steps(a.img, gb + 1, wrap_o, a.err);
  }
  if (a.bin) {
    if (he) atomicAdd(cur + 2 * ce + te, 1u);
    if (ho) atomicAdd(cur + 2 * co + to, 1u);
  }
  return (acc ? 1u : 0u) + (acco ? 1u : 0u);
}

// This CTA's share of count buffer t+1 mod 3 of system a (not touched in step t).
__device__ __forceinline__ void clear_next(const MoveArgs& a, long long tl, int tid, int nthreads) {
  uint2* next2 = reinterpret_cast<uint2*>(count_buffer(a.counts, a.n_c, tl + 1));
  const int64_t cells = a.n_c;  // one uint2 per cell
  const int64_t per = (cells + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = min(lo + per, cells);
  for (int64_t i = lo + tid; i < hi; i += nthreads) next2[i] = make_uint2(0u, 0u);
}

__device__ __forceinline__ void init_barriers(uint64_t* full, uint64_t* empty, int consumer_warps) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], consumer_warps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
}

// The producer's drain: no copy may still be in flight when the CTA exits.
__device__ __forceinline__ void drain(uint64_t* full, int issued, int* err) {
  for (int j = issued - kStages < 0 ? 0 : issued - kStages; j < issued; ++j)
    if (!mbar_wait(&full[j % kStages], (uint32_t)(j / kStages) & 1u, err)) break;
}

// W consumer warps and one producer warp; register budget 72 (no spill).
template <int W, bool kFromCounts, bool kSmart, bool kWall, bool kConv>
__global__ void __launch_bounds__((W + 1) * 32, move_min_blocks<W>())
    k_move(const __grid_constant__ MoveArgs a, StepRef r) {
  MoveStage<W>* stage = move_ring<W>();
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  init_barriers(full, empty, W);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == W) {  // producer warp: lane 0 streams the tiles
    if (lane == 0) {
      int it = 0;
      for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
        const int s = it % kStages;
        if (it >= kStages && !mbar_wait(&empty[s], (uint32_t)((it / kStages) - 1) & 1u, a.err)) break;
        produce_tile(a, tile, stage[s], &full[s]);
      }
      drain(full, it, a.err);
    }
    return;
  }

  const long long tl = r.get();
  const uint2* prev = reinterpret_cast<const uint2*>(count_buffer(a.counts, a.n_c, tl - 1));
  uint32_t* cur = count_buffer(a.counts, a.n_c, tl);
  unsigned nacc = 0;
  int it = 0;
  for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++it) {
    const int s = it % kStages;
    if (!mbar_wait(&full[s], (uint32_t)(it / kStages) & 1u, a.err)) break;
    nacc += consume_tile<kFromCounts, kSmart, kWall, kConv, W>(a, tile, stage[s], &empty[s], tl, prev, cur, warp,
                                                               lane);
  }
  nacc = __reduce_add_sync(0xffffffffu, nacc);
  if (lane == 0 && nacc) atomicAdd(a.acc + blockIdx.x, (unsigned long long)nacc);
  clear_next(a, tl, threadIdx.x, W * 32);
}

// System of a global tile index (uniform across the CTA): binary search.
__device__ __forceinline__ int batch_system(const BatchArgs& p, int tile) {
  int lo = 0, hi = p.n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.tile_start[mid] <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// One move kind and one z boundary per launch (the host groups systems so).
// Register budget for 3 resident CTAs per SM as the 8-warp k_move (with the
// warp-uniform system index below, only the walled bond-force-biased
// specialisation still spills, 12 bytes; it beats 2 CTAs per SM).
template <bool kSmart, bool kWall>
__global__ void __launch_bounds__((kBatchWarps + 1) * 32, move_min_blocks<kBatchWarps>())
    k_move_batch(const __grid_constant__ BatchArgs p, StepRef r) {
  __shared__ MoveStage<kBatchWarps> stage[kStages];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ __align__(8) uint64_t empty[kStages];
  init_barriers(full, empty, kBatchWarps);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = p.tile_start[p.n_sys];
  int* err = p.sys[0].err;

  if (warp == kBatchWarps) {
    if (lane == 0) {
      int it = 0;
      for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int s = it % kStages;
        if (it >= kStages && !mbar_wait(&empty[s], (uint32_t)((it / kStages) - 1) & 1u, err)) break;
        const int sys = batch_system(p, tile);
        stage[s].sys = (uint32_t)sys;  // ordered before the stage's arrive (release semantics)
        produce_tile(p.sys[sys], tile - p.tile_start[sys], stage[s], &full[s]);
      }
      drain(full, it, err);
    }
    return;
  }

  const long long tl = r.get();
  // the step's count buffers, as indices (each system's buffers sit at the
  // same positions within its own block of three)
  const int prev_buf = count_buffer_index(tl - 1), cur_buf = count_buffer_index(tl);
  int it = 0;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
    const int s = it % kStages;
    if (!mbar_wait(&full[s], (uint32_t)(it / kStages) & 1u, err)) break;
    // the producer's search, not one per thread.  The bond-force-biased
    // kernels pass the index through a warp reduction, whose result the
    // compiler keeps in a uniform register: the system's constants are then
    // loaded once per warp instead of into every thread's registers, which
    // removes the spill at 72 registers (64-system batch: 761 against
    // 834 us per step).  The uniform move is 2 % slower so (613 against
    // 601 us) and keeps the plain load.
    const int sys = kSmart ? (int)__reduce_max_sync(0xffffffffu, lds1(&stage[s].sys)) : (int)lds1(&stage[s].sys);
    const MoveArgs& a = p.sys[sys];
    const uint2* prev = reinterpret_cast<const uint2*>(a.counts) + (int64_t)prev_buf * a.n_c;
    uint32_t* cur = a.counts + (int64_t)cur_buf * 2 * a.n_c;
    const int lt = tile - p.tile_start[sys];
    unsigned n;
    if (a.conv)
      n = a.from_counts
              ? consume_tile<true, kSmart, kWall, true, kBatchWarps>(a, lt, stage[s], &empty[s], tl, prev, cur, warp, lane)
              : consume_tile<false, kSmart, kWall, true, kBatchWarps>(a, lt, stage[s], &empty[s], tl, prev, cur, warp, lane);
    else
      n = a.from_counts
              ? consume_tile<true, kSmart, kWall, false, kBatchWarps>(a, lt, stage[s], &empty[s], tl, prev, cur, warp, lane)
              : consume_tile<false, kSmart, kWall, false, kBatchWarps>(a, lt, stage[s], &empty[s], tl, prev, cur, warp, lane);
    n = __reduce_add_sync(0xffffffffu, n);
    if (lane == 0 && n) atomicAdd(a.acc + blockIdx.x, (unsigned long long)n);
  }
  for (int sys = 0; sys < p.n_sys; ++sys) clear_next(p.sys[sys], tl, threadIdx.x, kBatchWarps * 32);
}

// Self-check of the bounded-wait failure path: one thread waits on an
// mbarrier that nothing arrives on, for at most `cycles`; the wait gives up,
// sets kErrTimeout and the kernel returns, as every wait of the move kernels
// does when its copies or its consumers never come.
__global__ void k_wait_selfcheck(int* err, long long cycles) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(&bar, 0u, err, cycles);
  }
}

cudaError_t launch_wait_selfcheck(int* err, long long cycles, cudaStream_t s) {
  k_wait_selfcheck<<<1, 32, 0, s>>>(err, cycles);
  return cudaGetLastError();
}

int move_kernel_chains_per_tile(int P, int warps) { return warps * (32 / P); }

using MoveKernel = void (*)(MoveArgs, StepRef);

// [conv][smart][wall][from_counts] of the W-warp kernel
template <int W>
static MoveKernel move_kernel_of(bool conv, bool smart, bool wall, bool from_counts) {
  static const MoveKernel table[2][2][2][2] = {
      {{{k_move<W, false, false, false, false>, k_move<W, true, false, false, false>},
        {k_move<W, false, false, true, false>, k_move<W, true, false, true, false>}},
       {{k_move<W, false, true, false, false>, k_move<W, true, true, false, false>},
        {k_move<W, false, true, true, false>, k_move<W, true, true, true, false>}}},
      {{{k_move<W, false, false, false, true>, k_move<W, true, false, false, true>},
        {k_move<W, false, false, true, true>, k_move<W, true, false, true, true>}},
       {{k_move<W, false, true, false, true>, k_move<W, true, true, false, true>},
        {k_move<W, false, true, true, true>, k_move<W, true, true, true, true>}}}};
  return table[conv ? 1 : 0][smart ? 1 : 0][wall ? 1 : 0][from_counts ? 1 : 0];
}

// Every specialisation of the W-warp kernel may take the ring's dynamic
// shared memory (a per-kernel attribute of the current device; nothing to
// do where the ring is static).
template <int W>
static cudaError_t set_move_smem_limit() {
  if constexpr (move_dynamic_smem<W>() != 0) {
    for (int i = 0; i < 16; ++i) {
      const MoveKernel k = move_kernel_of<W>(i & 8, i & 4, i & 2, i & 1);
      const cudaError_t e =
          cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)move_dynamic_smem<W>());
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Resident CTAs per SM of the W-warp variant that runs every ordinary step
// (fields from counts), 0 where the shape cannot run on this device.  Sets
// the W-warp kernels' shared-memory limit on the current device, so it is
// called before any launch of the shape.  The held-field variant uses more
// registers; launched with the same grid its extra CTAs simply wait for a
// slot (CTAs never wait on one another).
template <int W>
static int max_ctas_of() {
  int n = 0;
  if (set_move_smem_limit<W>() != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_move<W, true, false, false, false>, (W + 1) * 32,
                                                    move_dynamic_smem<W>()) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

int move_kernel_max_ctas_per_sm(int warps) {
  switch (warps) {
    case 8: return max_ctas_of<8>();
    case 12: return max_ctas_of<12>();
    case 24: return max_ctas_of<24>();
    default: return 0;
  }
}

template <int W>
static void launch_move_w(const MoveArgs& a, int grid, bool from_counts, StepRef r, cudaStream_t s) {
  move_kernel_of<W>(a.conv != 0, a.smart != 0, a.wall_z != 0, from_counts)<<<grid, (W + 1) * 32,
                                                                             move_dynamic_smem<W>(), s>>>(a, r);
}

cudaError_t launch_move(const MoveArgs& a, int grid, bool from_counts, StepRef r, cudaStream_t s, int warps) {
  switch (warps) {
    case 12: launch_move_w<12>(a, grid, from_counts, r, s); break;
    case 24: launch_move_w<24>(a, grid, from_counts, r, s); break;
    default: launch_move_w<8>(a, grid, from_counts, r, s); break;
  }
  return cudaGetLastError();
}

static_assert(sizeof(BatchArgs) + sizeof(StepRef) <= 32764, "batch parameters exceed the kernel parameter space");

cudaError_t launch_move_batch(const BatchArgs& p, int grid, StepRef r, cudaStream_t s) {
  const bool smart = p.n_sys > 0 && p.sys[0].smart, wall = p.n_sys > 0 && p.sys[0].wall_z;
  const int threads = (kBatchWarps + 1) * 32;
  if (smart)
    wall ? k_move_batch<true, true><<<grid, threads, 0, s>>>(p, r) : k_move_batch<true, false><<<grid, threads, 0, s>>>(p, r);
  else
    wall ? k_move_batch<false, true><<<grid, threads, 0, s>>>(p, r) : k_move_batch<false, false><<<grid, threads, 0, s>>>(p, r);
  return cudaGetLastError();
}

// Resident CTAs per SM of one specialisation of the batch kernel (they
// differ in registers: the persistent grid must fit in one wave).
int move_batch_max_ctas_per_sm(bool smart, bool wall) {
  using Kernel = void (*)(BatchArgs, StepRef);
  const Kernel k = smart ? (wall ? k_move_batch<true, true> : k_move_batch<true, false>)
                         : (wall ? k_move_batch<false, true> : k_move_batch<false, false>);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, (kBatchWarps + 1) * 32, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n > 0 ? n : 1;
}

}  // namespace soma
