// soma_api.cu -- the C ABI of include/soma.h: handle life cycle, step
// scheduling (plain launches or CUDA-graph replay; a batch of independent
// systems steps in one persistent launch), state I/O, the coupling calls
// (fields given, held or restrained; placement; boundary-zone conversion),
// observables, reorder scheduling, per-kernel timing and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/soma.h"
#include "soma_internal.cuh"
#include "soma_launch.h"

#include <nvtx3/nvToolsExt.h>

using namespace soma;

namespace {

// NVTX range around an API call (visible in Nsight timelines; a no-op
// without a tool attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Makes `device` (>= 0) the calling thread's current device for the scope
// and gives the caller's current device back at its end.
class DeviceScope {
 public:
  explicit DeviceScope(int device) {
    if (device < 0) return;
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      ok_ = false;
      return;
    }
    if (cur == device) return;
    if (cudaSetDevice(device) != cudaSuccess) {
      ok_ = false;
      return;
    }
    prev_ = cur;
  }
  ~DeviceScope() {
    if (prev_ >= 0) cudaSetDevice(prev_);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
  bool ok() const { return ok_; }

 private:
  int prev_ = -1;
  bool ok_ = true;
};

// Opening of every call on a handle: the handle must be usable, and the call
// runs with the handle's device current (the caller's is restored on return).
#define SOMA_ENTER(h)                            \
  int rc = check_live(h);                        \
  if (rc) return rc;                             \
  const DeviceScope device_scope((h)->device);   \
  if (!device_scope.ok()) return SOMA_ECUDA

constexpr int kDefaultSortInterval = 200;
constexpr int kDefaultGraphSteps = 16;
enum { T_MOVE = 0, T_BIN = 1, T_FIELD = 2, T_SORT = 3 };

struct TimedEvent {
  cudaEvent_t a, b;
  int kind;
  bool timed;  // a and b were created and recorded
};

int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

struct soma_handle {
  int device = -1, sm_count = 0;  // the handle's CUDA device (set at creation)
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // dedicated stream for graph capture
  cudaEvent_t order_ev = nullptr;  // recorded after every soma_mc_steps, on its stream
  soma_options opt{};
  int n_sys = 0;
  bool partition = false;  // the handle holds a range of one system's chains (soma_create_partition)
  std::vector<soma_system_desc> desc;
  std::vector<SysDev> host_sys;  // device pointers and constants (fixed for the handle's life)
  SysDev* d_sys = nullptr;
  std::vector<MoveArgs> margs;
  std::vector<FieldArgs> fargs;
  std::vector<BatchArgs> batches;          // groups of up to kMaxBatch register-path systems
  std::vector<std::vector<int>> batch_members;
  std::vector<int> n_tiles;
  std::vector<char> phi_pending;  // next step moves against coupling-supplied fields
  std::vector<void*> owned;
  // launch geometry
  int max_ctas_per_sm = 1;             // of the single-system move kernel in its current shape
  int move_warps = 8;                  // its consumer warps per CTA (8, 12 or 24; the autotuner picks)
  int max_ctas_warps[kMoveShapes] = {};  // resident CTAs per SM of each shape (0: cannot run here)
  int max_ctas_batch = 1;              // the largest over the batch kernel's specialisations
  int max_ctas_batch_kind[2][2] = {};  // [smart][wall]
  int ctas_per_sm = 1;
  int hist_mode = SOMA_HIST_FUSED;
  int sort_interval = kDefaultSortInterval;
  int acc_per_sys = 1;
  unsigned long long* d_acc = nullptr;
  // Step counters, one per system (all equal), read by CUDA-graph replays;
  // plain launches carry the step number itself.  h->step mirrors the steps
  // enqueued; dev_synced says whether the counters hold it.
  unsigned long long* d_step = nullptr;
  bool dev_synced = true;
  uint64_t step = 0;
  uint64_t acc_since = 0;  // step at which the acceptance counters were last cleared
  uint64_t steps_since_sort = 0;
  int* d_err = nullptr;
  double* d_obs = nullptr;
  unsigned long long* d_acc_sum = nullptr;
  int32_t* d_m = nullptr;
  int m_cap = 0;
  double* d_sq = nullptr;
  float* d_stage_pos = nullptr;
  int16_t* d_stage_img = nullptr;
  float* d_stage_phi = nullptr;
  unsigned long long* d_profile = nullptr;  // layer sums of soma_density_profile (first use)
  unsigned long long* d_vcorr = nullptr;    // pair sums of soma_vertical_correlation (first use)
  size_t vcorr_words = 0;
  void* place_temp = nullptr;  // CUB scan scratch of soma_place (allocated on first use)
  size_t place_temp_bytes = 0;
  int64_t max_nb = 0, max_nc = 0;
  SortWork sort{};
  // graph
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  // timing
  std::vector<TimedEvent> pending;
  double ms[4] = {0, 0, 0, 0};
  int64_t launches[4] = {0, 0, 0, 0};
  bool tuned = false;
  bool f64 = false;  // SOMA_PREC_FP64 handle
  double* d_stage_pos64 = nullptr;
  int sticky = SOMA_OK;
};

namespace {

int fail(soma_handle* h, int code) {
  if (h && h->sticky == SOMA_OK) h->sticky = code;
  return code;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      if (getenv("SOMA_VERBOSE"))                                                       \
        fprintf(stderr, "soma: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), \
                __FILE__, __LINE__);                                                    \
      return fail(h, e_ == cudaErrorMemoryAllocation ? SOMA_ENOMEM : SOMA_ECUDA);       \
    }                                                                                   \
  } while (0)

void* dev_alloc(soma_handle* h, size_t bytes) {
  bytes = ((bytes + 255) / 256) * 256;
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (h->opt.alloc) {
    p = h->opt.alloc(bytes, h->opt.alloc_ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->owned.push_back(p);
  return p;
}

void dev_free_all(soma_handle* h) {
  for (void* p : h->owned) {
    if (h->opt.free)
      h->opt.free(p, h->opt.alloc_ctx);
    else
      cudaFree(p);
  }
  h->owned.clear();
}

cudaStream_t pick(soma_handle* h, void* stream) { return stream ? (cudaStream_t)stream : h->stream; }

int check_live(const soma_handle* h) {
  if (!h) return SOMA_EINVAL;
  if (h->sticky != SOMA_OK) return SOMA_ESTATE;
  return SOMA_OK;
}

int validate_desc(const soma_system_desc& d) {
  if (d.n_poly < 1 || d.N < 1 || d.N > 4096 || d.n_A < 0 || d.n_A > d.N) return SOMA_EINVAL;
  if ((int64_t)d.n_poly * d.N > (int64_t)INT32_MAX - 64) return SOMA_EINVAL;
  int64_t nc = 1;
  for (int a = 0; a < 3; ++a) {
    if (d.grid[a] < 1 || !(d.box[a] > 0.0) || !std::isfinite(d.box[a])) return SOMA_EINVAL;
    nc *= d.grid[a];
  }
  if (nc >= (int64_t)INT32_MAX / 4) return SOMA_EINVAL;
  if (!std::isfinite(d.chiN) || !std::isfinite(d.kappaN) || !std::isfinite(d.A)) return SOMA_EINVAL;
  if (d.N == 1 && !(d.A > 0.0)) return SOMA_EINVAL;  // no default half-width without bonds
  if (d.N > 1) {
    const double min_box = 16.0 / std::sqrt(3.0 * (d.N - 1));  // 2 x 8 bond standard deviations
    for (int a = 0; a < 3; ++a)
      if (d.box[a] < min_box) return SOMA_EINVAL;
  }
  const double A = d.A > 0 ? d.A : 0.5 / std::sqrt((double)(d.N - 1));
  for (int a = 0; a < 3; ++a)
    if (A >= d.box[a]) return SOMA_EINVAL;  // a proposal must wrap at most once
  if (d.move != SOMA_MOVE_UNIFORM && d.move != SOMA_MOVE_SMART) return SOMA_EINVAL;
  if (d.wall_z != 0 && d.wall_z != 1) return SOMA_EINVAL;
  if (d.move == SOMA_MOVE_SMART) {
    // |drift s| <= (A^2 (N-1)/2) L and |sig xi| < 6 A/sqrt(3) with |xi| < 6:
    // both below L/2 keeps a proposal within one image of the box
    if (0.5 * A * A * (d.N - 1) > 0.5) return SOMA_EINVAL;
    for (int a = 0; a < 3; ++a)
      if (12.0 / std::sqrt(3.0) * A >= d.box[a]) return SOMA_EINVAL;
  }
  return SOMA_OK;
}

// Persistent grid of a move launch: every resident slot, at most one CTA per tile.
int move_grid(const soma_handle* h, int64_t tiles, int max_ctas) {
  const int64_t capacity = (int64_t)h->sm_count * std::min(h->ctas_per_sm, max_ctas);
  return (int)std::max<int64_t>(1, std::min<int64_t>(capacity, tiles));
}

StepRef fixed_step(long long t) {
  StepRef r;
  r.counter = nullptr;
  r.fixed = t;
  r.use_counter = 0;
  r.offset = 0;
  return r;
}

StepRef counter_step(const unsigned long long* counter, int offset) {
  StepRef r;
  r.counter = counter;
  r.fixed = 0;
  r.use_counter = 1;
  r.offset = offset;
  return r;
}

void build_args(soma_handle* h) {
  h->margs.resize(h->n_sys);
  h->fargs.resize(h->n_sys);
  h->n_tiles.resize(h->n_sys);
  for (int s = 0; s < h->n_sys; ++s) {
    const SysDev& S = h->host_sys[s];
    MoveArgs& a = h->margs[s];
    std::memset(&a, 0, sizeof(a));
    for (int i = 0; i < 3; ++i) {
      a.L[i] = S.L[i];
      a.invL[i] = S.invL[i];
      a.cps[i] = S.cps[i];
      a.Lm[i] = std::nextafter(S.L[i], 0.0f);
    }
    a.n[0] = S.nx;
    a.n[1] = S.ny;
    a.n[2] = S.nz;
    a.A = S.A;
    a.kb = S.kb;
    std::memcpy(a.rk, S.rk, sizeof(a.rk));
    a.N = S.N;
    a.n_A = S.n_A;
    a.P = S.P;
    a.sys_index = S.sys_index;
    a.n_poly = S.n_poly;
    // several systems step in the batch kernel, whose tiles are 8 warps
    a.chains_per_tile = S.P ? move_kernel_chains_per_tile(S.P, h->n_sys > 1 ? 8 : h->move_warps) : 0;
    a.n_tiles = S.P ? (int)(((int64_t)S.n_poly + a.chains_per_tile - 1) / a.chains_per_tile) : 0;
    a.bin = h->hist_mode == SOMA_HIST_FUSED ? 1 : 0;
    a.n_c = S.n_c;
    a.x = S.x;
    a.y = S.y;
    a.z = S.z;
    a.img = S.img;
    a.chain_id = S.chain_id;
    a.counts = S.counts;
    a.w = S.w;
    a.inv_rho = S.inv_rho;
    a.chiN_N = S.chiN_N;
    a.kappaN_N = S.kappaN_N;
    a.from_counts = (S.frozen || S.umbrella) ? 0 : 1;
    a.acc = h->d_acc + S.acc_first;
    a.err = h->d_err;
    a.smart = h->desc[s].move == SOMA_MOVE_SMART ? 1 : 0;
    a.wall_z = S.wall_z;
    a.conv = S.conv;
    a.n_A_alt = S.n_A_alt;
    a.zone_lo = S.zone_lo;
    a.zone_hi = S.zone_hi;
    std::memcpy(a.thr, S.thr, sizeof(a.thr));
    a.conv_count = S.conv_count;
    {
      const double s2 = (double)S.A * (double)S.A / 3.0;
      a.sig = (float)std::sqrt(s2);
      a.drift = (float)(s2 * (double)S.kb);
      a.inv2s2 = (float)(0.5 / s2);
    }
    h->n_tiles[s] = a.n_tiles;

    FieldArgs& f = h->fargs[s];
    std::memset(&f, 0, sizeof(f));
    f.counts = S.counts;
    f.w = S.w;
    f.n_c = S.n_c;
    f.inv_rho = S.inv_rho;
    f.chiN_N = S.chiN_N;
    f.kappaN_N = S.kappaN_N;
    f.frozen = S.frozen;
    f.target = S.phi_target;
    f.umbN_N = S.umbN_N;
    f.umbrella = S.umbrella;
  }
  // batched launches: register-path systems in groups of at most kMaxBatch
  h->batches.clear();
  h->batch_members.clear();
  if (h->n_sys > 1) {
    // a group holds one move kind and one z boundary (the batch kernel is
    // specialised on both)
    for (int kind = 0; kind < 4; ++kind) {
      std::vector<int> reg;
      for (int s = 0; s < h->n_sys; ++s)
        if (h->host_sys[s].P && h->desc[s].move == (kind & 1) && h->desc[s].wall_z == (kind >> 1)) reg.push_back(s);
      for (size_t g0 = 0; g0 < reg.size(); g0 += kMaxBatch) {
        BatchArgs b;
        std::memset(&b, 0, sizeof(b));
        std::vector<int> members(reg.begin() + g0, reg.begin() + std::min(reg.size(), g0 + kMaxBatch));
        b.n_sys = (int)members.size();
        int tiles = 0;
        for (int i = 0; i < b.n_sys; ++i) {
          b.tile_start[i] = tiles;
          b.sys[i] = h->margs[members[i]];
          tiles += h->n_tiles[members[i]];
        }
        b.tile_start[b.n_sys] = tiles;
        h->batches.push_back(b);
        h->batch_members.push_back(members);
      }
    }
  }
}

void drop_graph(soma_handle* h) {
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
}

// Around every launch of the library's kernels: CUDA events when the handle
// times its kernels (kernel_timing), and the launch count of its kind unless
// the launch is being captured into a graph (a captured launch runs once per
// replay, which the host does not see).
void begin_timed(soma_handle* h, cudaStream_t s, TimedEvent& te, int kind, bool timing) {
  te.kind = kind;
  te.timed = timing;
  if (!timing) return;
  cudaEventCreate(&te.a);
  cudaEventCreate(&te.b);
  cudaEventRecord(te.a, s);
}
void end_timed(soma_handle* h, cudaStream_t s, TimedEvent& te, bool count) {
  if (te.timed) {
    cudaEventRecord(te.b, s);
    h->pending.push_back(te);
  }
  if (count) h->launches[te.kind] += 1;
}

// Step i of a sequence: the fixed number t0 + i (plain launches) or the
// device counter + i (graph capture).
StepRef step_ref(const soma_handle* h, int sys, bool graph, long long t0, int i) {
  return graph ? counter_step(h->d_step + sys, i) : fixed_step(t0 + i);
}

// Histogram, field array and the generic move: the parts of a step that are
// not the register move kernel.
int enqueue_aux(soma_handle* h, cudaStream_t s, int sys, StepRef r, bool timing, bool moved) {
  const SysDev& S = h->host_sys[sys];
  TimedEvent te;
  if (S.P == 0 && !moved) {
    begin_timed(h, s, te, T_MOVE, timing);
    CK(launch_move_generic(h->d_sys, sys, S.n_poly, S.N, r, h->sm_count, s));
    end_timed(h, s, te, !r.use_counter);
  }
  if (S.P == 0 || h->hist_mode == SOMA_HIST_SEPARATE) {
    begin_timed(h, s, te, T_BIN, timing);
    CK(launch_bin(h->d_sys, sys, S.n_b, r, h->sm_count, s));
    end_timed(h, s, te, !r.use_counter);
  }
  if (S.P == 0) {
    begin_timed(h, s, te, T_FIELD, timing);
    CK(launch_field(h->fargs[sys], r, 1, s));
    end_timed(h, s, te, !r.use_counter);
  }
  return SOMA_OK;
}

// With the umbrella restraint on, the register move reads the field array,
// filled before each step from the previous step's counts (the restraint's
// target term is not folded into the move kernel).  Not for held fields or
// a step whose fields came from soma_set_density.
int enqueue_umbrella_fields(soma_handle* h, cudaStream_t s, int sys, bool graph, long long t0, int i) {
  const SysDev& S = h->host_sys[sys];
  if (!S.P || !S.umbrella || S.frozen || (i == 0 && h->phi_pending[sys])) return SOMA_OK;
  TimedEvent te;
  const bool timing = h->opt.kernel_timing != 0;
  begin_timed(h, s, te, T_FIELD, timing);
  CK(launch_field(h->fargs[sys], step_ref(h, sys, graph, t0, i - 1), 0, s));
  end_timed(h, s, te, !graph);
  return SOMA_OK;
}

// n steps of every system on stream `s`.  One system: one move kernel per
// step (fields from the previous counts, fused histogram, clearing of the
// next count buffer).  Several systems: one k_move_batch launch per step and
// group of up to kMaxBatch systems.  Chains longer than 64 beads: generic
// move, histogram and field array per system.
int enqueue_steps(soma_handle* h, cudaStream_t s, int n, bool graph, long long t0) {
  const bool timing = h->opt.kernel_timing != 0;
  const bool batched = h->n_sys > 1;
  int rc;
  for (int i = 0; i < n; ++i) {
    if (batched) {
      for (size_t g = 0; g < h->batches.size(); ++g) {
        const BatchArgs* b = &h->batches[g];
        BatchArgs pending_copy;
        if (i == 0) {  // coupling-supplied fields move the first step of their system
          bool any = false;
          for (int m = 0; m < b->n_sys; ++m) any |= h->phi_pending[h->batch_members[g][m]] != 0;
          if (any) {
            pending_copy = *b;
            for (int m = 0; m < b->n_sys; ++m)
              if (h->phi_pending[h->batch_members[g][m]]) pending_copy.sys[m].from_counts = 0;
            b = &pending_copy;
          }
        }
        TimedEvent te;
        for (int m = 0; m < b->n_sys; ++m)
          if ((rc = enqueue_umbrella_fields(h, s, h->batch_members[g][m], graph, t0, i))) return rc;
        begin_timed(h, s, te, T_MOVE, timing);
        // one wave: at most as many CTAs as this specialisation keeps resident
        const int fit = h->max_ctas_batch_kind[b->sys[0].smart ? 1 : 0][b->sys[0].wall_z ? 1 : 0];
        CK(launch_move_batch(*b, move_grid(h, b->tile_start[b->n_sys], fit),
                             step_ref(h, 0, graph, t0, i), s));
        end_timed(h, s, te, !graph);
      }
      for (int sys = 0; sys < h->n_sys; ++sys)
        if ((rc = enqueue_aux(h, s, sys, step_ref(h, sys, graph, t0, i), timing, false))) return rc;
    } else if (h->f64) {
      TimedEvent te;
      begin_timed(h, s, te, T_MOVE, timing);
      CK(launch_move64(h->d_sys, 0, step_ref(h, 0, graph, t0, i), h->sm_count, s));
      end_timed(h, s, te, !graph);
    } else {
      const SysDev& S = h->host_sys[0];
      const StepRef r = step_ref(h, 0, graph, t0, i);
      if (S.P) {
        const bool from_counts = !S.frozen && !S.umbrella && !(i == 0 && h->phi_pending[0]);
        if ((rc = enqueue_umbrella_fields(h, s, 0, graph, t0, i))) return rc;
        TimedEvent te;
        begin_timed(h, s, te, T_MOVE, timing);
        CK(launch_move(h->margs[0], move_grid(h, h->n_tiles[0], h->max_ctas_per_sm), from_counts, r, s,
                       h->move_warps));
        end_timed(h, s, te, !graph);
      }
      if ((rc = enqueue_aux(h, s, 0, r, timing, false))) return rc;
    }
  }
  return SOMA_OK;
}

// Key, value and CUB buffers of the chain reorder (about 40 bytes per chain),
// allocated once, on first need.
int ensure_sort_work(soma_handle* h) {
  SortWork& w = h->sort;
  if (w.temp) return SOMA_OK;
  const size_t n = (size_t)w.n_chains;
  w.keys_in = (unsigned long long*)dev_alloc(h, 8 * n);
  w.keys_out = (unsigned long long*)dev_alloc(h, 8 * n);
  w.vals_in = (uint32_t*)dev_alloc(h, 4 * n);
  w.vals_out = (uint32_t*)dev_alloc(h, 4 * n);
  w.chain_sys = (int32_t*)dev_alloc(h, 4 * n);
  w.temp_bytes = sort_temp_bytes(w.n_chains, w.end_bit);
  void* temp = dev_alloc(h, w.temp_bytes);
  if (!w.keys_in || !w.keys_out || !w.vals_in || !w.vals_out || !w.chain_sys || !temp) return SOMA_ENOMEM;
  std::vector<int32_t> cs(n);
  for (int s = 0; s < h->n_sys; ++s)
    std::fill(cs.begin() + h->host_sys[s].chain_base, cs.begin() + h->host_sys[s].chain_base + h->host_sys[s].n_poly,
              s);
  CK(cudaMemcpy(w.chain_sys, cs.data(), 4 * n, cudaMemcpyHostToDevice));
  w.temp = temp;  // set last: a failed attempt is retried in full
  return SOMA_OK;
}

int enqueue_reorder(soma_handle* h, cudaStream_t s) {
  int rc = ensure_sort_work(h);
  if (rc) return rc;
  TimedEvent te;
  begin_timed(h, s, te, T_SORT, h->opt.kernel_timing != 0);
  CK(launch_reorder(h->d_sys, h->n_sys, h->sort, h->sm_count, s));
  end_timed(h, s, te, true);
  h->steps_since_sort = 0;
  return SOMA_OK;
}

int capture_graph(soma_handle* h, int steps) {
  drop_graph(h);
  cudaStream_t cs = h->cap_stream;
  CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  int rc = enqueue_steps(h, cs, steps, true, 0);
  if (rc == SOMA_OK && launch_advance(h->d_step, h->n_sys, steps, cs) != cudaSuccess) rc = SOMA_ECUDA;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &g);
  if (rc != SOMA_OK) {
    if (g) cudaGraphDestroy(g);
    return fail(h, rc);
  }
  CK(e);
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  h->graph_steps = steps;
  return SOMA_OK;
}

// Clear the three count buffers, bin the current positions into buffer
// (step - 1) mod 3 and fill the field array from them (unless held).
int rebin_one(soma_handle* h, int g, cudaStream_t s) {
  SysDev& S = h->host_sys[g];
  CK(cudaMemsetAsync(S.counts, 0, sizeof(uint32_t) * 6 * S.n_c, s));
  if (h->f64)
    CK(launch_bin64(h->d_sys, g, (long long)h->step - 1, h->sm_count, s));
  else
    CK(launch_bin(h->d_sys, g, S.n_b, fixed_step((long long)h->step - 1), h->sm_count, s));
  CK(launch_field(h->fargs[g], fixed_step((long long)h->step - 1), 0, s));
  return SOMA_OK;
}

int rebin_all(soma_handle* h, cudaStream_t s) {
  int rc;
  for (int g = 0; g < h->n_sys; ++g)
    if ((rc = rebin_one(h, g, s))) return rc;
  return SOMA_OK;
}

int check_device_error(soma_handle* h) {
  int err = 0;
  CK(cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (err & kErrTimeout) return fail(h, SOMA_ETIMEOUT);
  if (err & kErrBounds) return fail(h, SOMA_EDEVICE_CHECK);
  return SOMA_OK;
}

int sync_all(soma_handle* h) {
  CK(cudaDeviceSynchronize());
  return check_device_error(h);
}

int set_frozen(soma_handle* h, int sys, int frozen) {
  h->host_sys[sys].frozen = frozen;
  h->fargs[sys].frozen = frozen;
  drop_graph(h);
  CK(cudaMemcpy(reinterpret_cast<char*>(h->d_sys + sys) + offsetof(SysDev, frozen), &frozen, sizeof(int),
                cudaMemcpyHostToDevice));
  return SOMA_OK;
}

// Resident CTAs per SM of the shape with `warps` consumer warps (a shape
// the options were validated against).
int shape_ctas(const soma_handle* h, int warps) { return h->max_ctas_warps[std::max(0, move_shape(warps))]; }

void apply_geometry(soma_handle* h, int ctas_per_sm, int hist_mode, int move_warps) {
  h->move_warps = move_warps;
  h->max_ctas_per_sm = shape_ctas(h, move_warps);
  h->ctas_per_sm = std::max(1, std::min(ctas_per_sm, std::max(h->max_ctas_per_sm, h->max_ctas_batch)));
  h->hist_mode = hist_mode;
  build_args(h);
  drop_graph(h);
}

}  // namespace

extern "C" {

int soma_options_default(soma_options* o) {
  if (!o) return SOMA_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->device = -1;
  o->sort_interval = -1;
  o->ctas_per_sm = 0;
  o->hist_mode = SOMA_HIST_AUTO;
  o->graph_steps = kDefaultGraphSteps;
  o->kernel_timing = 0;
  o->autotune = 0;
  return SOMA_OK;
}

const char* soma_strerror(int code) {
  switch (code) {
    case SOMA_OK: return "ok";
    case SOMA_EINVAL: return "invalid argument";
    case SOMA_ENOMEM: return "out of memory";
    case SOMA_ECUDA: return "CUDA runtime error";
    case SOMA_ETIMEOUT: return "device-side wait timed out";
    case SOMA_EDEVICE_CHECK: return "device-side consistency check failed";
    case SOMA_ESTATE: return "handle is in a failed state";
    case SOMA_ENOTSUP: return "not supported";
    default: return "unknown error";
  }
}

int soma_last_error(const soma_handle* h) { return h ? h->sticky : SOMA_EINVAL; }

void soma_destroy(soma_handle* h) {
  if (!h) return;
  const DeviceScope device_scope(h->device);
  if (h->order_ev) cudaEventSynchronize(h->order_ev);  // steps enqueued on a caller's stream
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& te : h->pending) {
    cudaEventDestroy(te.a);
    cudaEventDestroy(te.b);
  }
  drop_graph(h);
  dev_free_all(h);
  if (h->stream) cudaStreamDestroy(h->stream);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->order_ev) cudaEventDestroy(h->order_ev);
  delete h;
}

// Create a handle for n_sys systems, or (part_end >= 0, n_sys = 1) for the
// logical chains [part_begin, part_end) of one system.
static int create_handle(const soma_system_desc* sys, int n_sys, const soma_options* opt, int64_t part_begin,
                         int64_t part_end, soma_handle** out) {
  if (!out) return SOMA_EINVAL;
  *out = nullptr;
  if (!sys || n_sys < 1 || n_sys > (1 << 16)) return SOMA_EINVAL;
  const bool partition = part_end >= 0;
  if (partition && (n_sys != 1 || part_begin < 0 || part_end <= part_begin || part_end > sys[0].n_poly))
    return SOMA_EINVAL;
  int64_t total_chains = 0;
  for (int s = 0; s < n_sys; ++s) {
    if (validate_desc(sys[s]) != SOMA_OK) return SOMA_EINVAL;
    total_chains += sys[s].n_poly;
  }
  if (total_chains > (int64_t)UINT32_MAX) return SOMA_EINVAL;  // the reorder numbers chains in 32 bits
  soma_options o;
  if (opt)
    o = *opt;
  else
    soma_options_default(&o);
  if (o.ctas_per_sm < 0 || o.ctas_per_sm > 64) return SOMA_EINVAL;
  if (o.precision != SOMA_PREC_FP32 && o.precision != SOMA_PREC_FP64) return SOMA_EINVAL;
  if (o.precision == SOMA_PREC_FP64) {
    if (n_sys != 1) return SOMA_EINVAL;  // the FP64 form steps one system per handle
    for (int s = 0; s < n_sys; ++s)
      if (sys[s].N > 64 || sys[s].move != SOMA_MOVE_UNIFORM || sys[s].wall_z) return SOMA_ENOTSUP;
  }
  for (int s = 0; s < n_sys; ++s)
    if (sys[s].move == SOMA_MOVE_SMART && sys[s].N > 64) return SOMA_ENOTSUP;
  if (partition) {
    // the exchange follows every step: one step per call, no autotuner (its
    // trial steps would run between exchanges), fields from the counts of the
    // register move kernel (chains of at most 64 beads), FP32 positions
    if (o.autotune) return SOMA_EINVAL;
    if (sys[0].N > 64 || o.precision != SOMA_PREC_FP32) return SOMA_ENOTSUP;
  }
  if (o.hist_mode < SOMA_HIST_AUTO || o.hist_mode > SOMA_HIST_SEPARATE) return SOMA_EINVAL;
  if (o.graph_steps < 0 || o.graph_steps > 4096) return SOMA_EINVAL;
  if ((o.alloc == nullptr) != (o.free == nullptr)) return SOMA_EINVAL;
  if (o.move_warps != 0 && move_shape(o.move_warps) < 0) return SOMA_EINVAL;

  // creation runs on opt.device and leaves the caller's current device as it was
  const DeviceScope device_scope(o.device);
  if (!device_scope.ok()) return SOMA_ECUDA;
  soma_handle* h = new (std::nothrow) soma_handle();
  if (!h) return SOMA_ENOMEM;
  h->opt = o;
  h->n_sys = n_sys;
  h->partition = partition;
  h->desc.assign(sys, sys + n_sys);
  int rc = SOMA_OK;
  auto bail = [&](int code) {
    soma_destroy(h);
    return code;
  };

  if (cudaGetDevice(&h->device) != cudaSuccess) return bail(SOMA_ECUDA);  // opt.device, or the current one
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) return bail(SOMA_ECUDA);
  h->sm_count = prop.multiProcessorCount;
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->order_ev, cudaEventDisableTiming) != cudaSuccess)
    return bail(SOMA_ECUDA);
  for (int i = 0; i < kMoveShapes; ++i) h->max_ctas_warps[i] = move_kernel_max_ctas_per_sm(kMoveWarps[i]);
  h->max_ctas_warps[0] = std::max(1, h->max_ctas_warps[0]);  // the default shape always launches
  h->move_warps = (o.move_warps > 8 && n_sys == 1) ? o.move_warps : 8;
  if (shape_ctas(h, h->move_warps) == 0) return bail(SOMA_ENOTSUP);
  h->max_ctas_per_sm = shape_ctas(h, h->move_warps);
  for (int sm = 0; sm < 2; ++sm)
    for (int wz = 0; wz < 2; ++wz) {
      h->max_ctas_batch_kind[sm][wz] = move_batch_max_ctas_per_sm(sm != 0, wz != 0);
      h->max_ctas_batch = std::max(h->max_ctas_batch, h->max_ctas_batch_kind[sm][wz]);
    }
  h->ctas_per_sm = o.ctas_per_sm ? std::min<int>(o.ctas_per_sm, h->max_ctas_per_sm) : h->max_ctas_per_sm;
  h->hist_mode = o.hist_mode == SOMA_HIST_AUTO ? SOMA_HIST_FUSED : o.hist_mode;
  h->sort_interval = o.sort_interval < 0 ? kDefaultSortInterval : o.sort_interval;
  h->f64 = o.precision == SOMA_PREC_FP64;
  if (h->f64) h->sort_interval = 0;  // the precision reference keeps its storage order
  h->acc_per_sys = h->sm_count * std::max(*std::max_element(h->max_ctas_warps, h->max_ctas_warps + kMoveShapes),
                                          h->max_ctas_batch);

  // --- per-system constants and arrays ---------------------------------
  h->host_sys.resize(n_sys);
  int64_t chain_base = 0;
  for (int s = 0; s < n_sys; ++s) {
    const soma_system_desc& d = sys[s];
    SysDev& S = h->host_sys[s];
    std::memset(&S, 0, sizeof(S));
    S.n_poly = partition ? (int32_t)(part_end - part_begin) : d.n_poly;
    S.id_base = partition ? (uint32_t)part_begin : 0u;
    S.N = d.N;
    S.n_A = d.n_A;
    S.P = d.N <= 64 ? next_pow2((d.N + 1) / 2) : 0;
    S.nx = d.grid[0];
    S.ny = d.grid[1];
    S.nz = d.grid[2];
    S.sys_index = d.system_id;
    S.wall_z = d.wall_z;
    S.n_b = (int64_t)S.n_poly * d.N;
    S.n_c = (int64_t)d.grid[0] * d.grid[1] * d.grid[2];
    S.rho_bar = (double)d.n_poly * d.N / (double)S.n_c;  // the whole system's density
    for (int a = 0; a < 3; ++a) {
      S.L[a] = (float)d.box[a];
      S.invL[a] = (float)(1.0 / d.box[a]);
      S.cps[a] = (float)(d.grid[a] / d.box[a]);
    }
    S.A = (float)(d.A > 0 ? d.A : 0.5 / std::sqrt((double)(d.N - 1)));
    S.kb = (float)(1.5 * (d.N - 1));
    S.chiN_N = (float)(d.chiN / d.N);
    S.kappaN_N = (float)(d.kappaN / d.N);
    S.inv_rho = (float)(1.0 / S.rho_bar);
    uint32_t k0 = (uint32_t)(d.seed & 0xFFFFFFFFu), k1 = (uint32_t)(d.seed >> 32);
    for (int r = 0; r < 10; ++r) {
      S.rk[r][0] = k0;
      S.rk[r][1] = k1;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    for (int a = 0; a < 3; ++a) {
      S.L64[a] = d.box[a];
      S.invL64[a] = 1.0 / d.box[a];
      S.cps64[a] = (double)d.grid[a] / d.box[a];
    }
    // field differences of the FP64 form: (chiN dn_other + kappaN dn_total) / (N rho_bar)
    {
      const double rho = S.rho_bar;
      S.chiN64 = d.chiN / d.N / rho;
      S.kappaN64 = d.kappaN / d.N / rho;
    }
    S.chain_base = chain_base;
    chain_base += S.n_poly;
    S.acc_first = s * h->acc_per_sys;
    S.acc_count = h->acc_per_sys;
    h->max_nb = std::max<int64_t>(h->max_nb, S.n_b);
    h->max_nc = std::max<int64_t>(h->max_nc, S.n_c);

    // bulk copies read whole 16-byte granules: pad position and id arrays
    const size_t nb = (size_t)S.n_b + 8, nc = (size_t)S.n_c, np = (size_t)S.n_poly + 8;
    S.x = (float*)dev_alloc(h, nb * 4);
    S.y = (float*)dev_alloc(h, nb * 4);
    S.z = (float*)dev_alloc(h, nb * 4);
    S.img = (int16_t*)dev_alloc(h, nb * 8);
    S.chain_id = (uint32_t*)dev_alloc(h, np * 4);
    S.x_alt = (float*)dev_alloc(h, nb * 4);
    S.y_alt = (float*)dev_alloc(h, nb * 4);
    S.z_alt = (float*)dev_alloc(h, nb * 4);
    S.img_alt = (int16_t*)dev_alloc(h, nb * 8);
    S.chain_id_alt = (uint32_t*)dev_alloc(h, np * 4);
    S.counts = (uint32_t*)dev_alloc(h, nc * 24);
    S.w = (float*)dev_alloc(h, nc * 8);
    if (!S.x || !S.y || !S.z || !S.img || !S.chain_id || !S.x_alt || !S.y_alt || !S.z_alt || !S.img_alt ||
        !S.chain_id_alt || !S.counts || !S.w)
      return bail(SOMA_ENOMEM);
    if (h->f64) {
      S.x64 = (double*)dev_alloc(h, nb * 8);
      S.y64 = (double*)dev_alloc(h, nb * 8);
      S.z64 = (double*)dev_alloc(h, nb * 8);
      if (!S.x64 || !S.y64 || !S.z64) return bail(SOMA_ENOMEM);
    }
    if (cudaMemset(S.x, 0, nb * 4) != cudaSuccess || cudaMemset(S.y, 0, nb * 4) != cudaSuccess ||
        cudaMemset(S.z, 0, nb * 4) != cudaSuccess || cudaMemset(S.chain_id, 0, np * 4) != cudaSuccess)
      return bail(SOMA_ECUDA);
  }
  h->d_acc = (unsigned long long*)dev_alloc(h, sizeof(unsigned long long) * (size_t)h->acc_per_sys * n_sys);
  for (int s = 0; s < n_sys; ++s) h->host_sys[s].acc = h->d_acc;
  h->d_sys = (SysDev*)dev_alloc(h, sizeof(SysDev) * n_sys);
  h->d_step = (unsigned long long*)dev_alloc(h, 8 * (size_t)n_sys);
  h->d_err = (int*)dev_alloc(h, 4);
  h->d_obs = (double*)dev_alloc(h, 8 * sizeof(double));
  h->d_acc_sum = (unsigned long long*)dev_alloc(h, 8);
  h->d_stage_pos = (float*)dev_alloc(h, (size_t)h->max_nb * 12);
  h->d_stage_img = (int16_t*)dev_alloc(h, (size_t)h->max_nb * 6);
  h->d_stage_phi = (float*)dev_alloc(h, (size_t)h->max_nc * 8);
  if (h->f64) {
    h->d_stage_pos64 = (double*)dev_alloc(h, (size_t)h->max_nb * 24);
    if (!h->d_stage_pos64) return bail(SOMA_ENOMEM);
  }
  if (!h->d_acc || !h->d_sys || !h->d_step || !h->d_err || !h->d_obs || !h->d_acc_sum || !h->d_stage_pos ||
      !h->d_stage_img || !h->d_stage_phi)
    return bail(SOMA_ENOMEM);
  // sort work: allocated here when chains may be reordered (a sort interval
  // or the autotuner), else on the first soma_reorder
  {
    int bits = 0;
    while ((1 << bits) < n_sys) ++bits;
    h->sort.n_chains = chain_base;
    h->sort.end_bit = 30 + bits;  // the sort keys: 30 bits of Morton key, then the system
    if ((h->sort_interval != 0 || o.autotune) && (rc = ensure_sort_work(h)) != SOMA_OK) return bail(rc);
  }
  if (cudaMemcpy(h->d_sys, h->host_sys.data(), sizeof(SysDev) * n_sys, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(h->d_step, 0, 8 * (size_t)n_sys) != cudaSuccess || cudaMemset(h->d_err, 0, 4) != cudaSuccess ||
      cudaMemset(h->d_acc, 0, sizeof(unsigned long long) * (size_t)h->acc_per_sys * n_sys) != cudaSuccess)
    return bail(SOMA_ECUDA);
  h->phi_pending.assign(n_sys, 0);
  build_args(h);

  // --- initial configuration, start-up checks, counts, fields, sort -----
  for (int s = 0; s < n_sys && rc == SOMA_OK; ++s) {
    if (h->f64) {
      if (launch_init64(h->d_sys, s, h->host_sys[s].n_poly, h->stream) != cudaSuccess) rc = SOMA_ECUDA;
    } else if (launch_init(h->d_sys, s, h->host_sys[s].n_poly, h->stream) != cudaSuccess) {
      rc = SOMA_ECUDA;
    } else if (launch_validate(h->d_sys, s, h->d_err, h->sm_count, h->stream) != cudaSuccess) {
      rc = SOMA_ECUDA;
    }
  }
  if (rc == SOMA_OK) rc = rebin_all(h, h->stream);
  if (rc == SOMA_OK && h->sort_interval != 0) rc = enqueue_reorder(h, h->stream);
  if (rc == SOMA_OK && cudaStreamSynchronize(h->stream) != cudaSuccess) rc = SOMA_ECUDA;
  if (rc == SOMA_OK) rc = check_device_error(h);
  if (rc != SOMA_OK) return bail(rc);
  h->tuned = !o.autotune || h->f64;
  *out = h;
  return SOMA_OK;
}

int soma_create(const soma_system_desc* sys, int n_sys, const soma_options* opt, soma_handle** out) {
  NvtxRange nvtx_range("soma_create");
  return create_handle(sys, n_sys, opt, 0, -1, out);
}

int soma_create_partition(const soma_system_desc* sys, const soma_options* opt, int32_t chain_begin,
                          int32_t chain_end, soma_handle** out) {
  NvtxRange nvtx_range("soma_create_partition");
  return create_handle(sys, 1, opt, chain_begin, chain_end, out);
}

int soma_exchange_counts(soma_handle* h, uint32_t** counts, size_t* n_words) {
  SOMA_ENTER(h);
  if (!counts || !n_words || h->f64 || h->n_sys != 1) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[0];
  *counts = count_buffer(S.counts, S.n_c, (long long)h->step - 1);
  *n_words = 2 * (size_t)S.n_c;
  return SOMA_OK;
}

int soma_mc_steps(soma_handle* h, int64_t n_steps, void* stream) {
  NvtxRange nvtx_range("soma_mc_steps");
  SOMA_ENTER(h);
  if (n_steps < 0) return SOMA_EINVAL;
  if (h->step + (uint64_t)n_steps >= (uint64_t)kInitStep) return SOMA_EINVAL;
  if (n_steps == 0) return SOMA_OK;
  if (h->partition && n_steps != 1) return SOMA_EINVAL;  // the counts are exchanged after every step
  if (!h->tuned) {
    rc = soma_autotune(h);
    if (rc) return rc;
  }
  cudaStream_t s = pick(h, stream);
  const bool use_graph = h->opt.graph_steps > 0 && !h->opt.kernel_timing;
  int64_t left = n_steps;
  bool pending = false;
  for (char p : h->phi_pending) pending |= p != 0;
  if (pending) {  // one plain step against the coupling-supplied fields
    if (h->sort_interval > 0 && h->steps_since_sort >= (uint64_t)h->sort_interval) {
      if ((rc = enqueue_reorder(h, s))) return rc;
    }
    if ((rc = enqueue_steps(h, s, 1, false, (long long)h->step))) return rc;
    h->dev_synced = false;
    std::fill(h->phi_pending.begin(), h->phi_pending.end(), 0);
    h->step += 1;
    h->steps_since_sort += 1;
    left -= 1;
  }
  while (left > 0) {
    if (h->sort_interval > 0 && h->steps_since_sort >= (uint64_t)h->sort_interval) {
      rc = enqueue_reorder(h, s);
      if (rc) return rc;
    }
    int64_t chunk = left;
    if (h->sort_interval > 0) chunk = std::min<int64_t>(chunk, h->sort_interval - (int64_t)h->steps_since_sort);
    if (use_graph && chunk >= h->opt.graph_steps) {
      if (!h->graph || h->graph_steps != h->opt.graph_steps) {
        rc = capture_graph(h, h->opt.graph_steps);
        if (rc) return rc;
      }
      if (!h->dev_synced) {
        CK(launch_set_step(h->d_step, h->n_sys, h->step, s));
        h->dev_synced = true;
      }
      const int64_t reps = chunk / h->graph_steps;
      for (int64_t r = 0; r < reps; ++r) CK(cudaGraphLaunch(h->graph, s));
      chunk = reps * h->graph_steps;
    } else {
      chunk = std::min<int64_t>(chunk, 1 << 16);
      if ((rc = enqueue_steps(h, s, (int)chunk, false, (long long)h->step))) return rc;
      h->dev_synced = false;
    }
    left -= chunk;
    h->step += (uint64_t)chunk;
    h->steps_since_sort += (uint64_t)chunk;
  }
  CK(cudaEventRecord(h->order_ev, s));
  return SOMA_OK;
}

int soma_sync(soma_handle* h, void* stream) {
  NvtxRange nvtx_range("soma_sync");
  SOMA_ENTER(h);
  CK(cudaStreamSynchronize(pick(h, stream)));
  CK(cudaStreamSynchronize(h->stream));
  return check_device_error(h);
}

int soma_get_density(soma_handle* h, int sys, uint32_t* out, size_t n, int where) {
  NvtxRange nvtx_range("soma_get_density");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !out) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if (n != (size_t)(2 * S.n_c)) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  const uint32_t* src = count_buffer(S.counts, S.n_c, (long long)h->step - 1);
  uint32_t* dst = where == SOMA_DEVICE ? out : reinterpret_cast<uint32_t*>(h->d_stage_phi);
  CK(launch_deinterleave(src, S.n_c, dst, h->sm_count, h->stream));
  if (where != SOMA_DEVICE) CK(cudaMemcpyAsync(out, dst, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SOMA_OK;
}

int soma_density_profile(soma_handle* h, int sys, int axis, double* out, size_t n) {
  NvtxRange nvtx_range("soma_density_profile");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !out || axis < 0 || axis > 2) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  const int dims[3] = {S.nx, S.ny, S.nz};
  const int layers = dims[axis];
  if (n != (size_t)(2 * layers)) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  if (!h->d_profile) {  // per-layer sums of the largest grid dimension, allocated on first use
    int most = 1;
    for (const SysDev& T : h->host_sys) most = std::max(most, std::max(T.nx, std::max(T.ny, T.nz)));
    h->d_profile = (unsigned long long*)dev_alloc(h, 16 * (size_t)most);
    if (!h->d_profile) return SOMA_ENOMEM;
  }
  unsigned long long* d_sum = h->d_profile;
  const uint32_t* src = count_buffer(S.counts, S.n_c, (long long)h->step - 1);
  CK(launch_profile(src, S.nx, S.ny, S.nz, axis, d_sum, h->stream));
  std::vector<unsigned long long> sums(2 * (size_t)layers);
  CK(cudaMemcpyAsync(sums.data(), d_sum, sizeof(unsigned long long) * sums.size(), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const double rho_bar = S.rho_bar;
  const double per_layer = (double)(S.n_c / layers);
  for (int k = 0; k < layers; ++k)
    for (int t = 0; t < 2; ++t) out[(size_t)t * layers + k] = (double)sums[2 * (size_t)k + t] / rho_bar / per_layer;
  return SOMA_OK;
}

int soma_vertical_correlation(soma_handle* h, int sys, int type, double* out, size_t n) {
  NvtxRange nvtx_range("soma_vertical_correlation");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !out || type < 0 || type > 1) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if (n != (size_t)S.nz) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  const size_t words = 4 * ((size_t)S.nz + 1);
  if (h->vcorr_words < words) {  // sums buffer, grown on demand (kept for the handle's life)
    int most = 1;
    for (const SysDev& T : h->host_sys) most = std::max(most, T.nz);
    h->vcorr_words = 4 * ((size_t)most + 1);
    h->d_vcorr = (unsigned long long*)dev_alloc(h, 8 * h->vcorr_words);
    if (!h->d_vcorr) return SOMA_ENOMEM;
  }
  const uint32_t* src = count_buffer(S.counts, S.n_c, (long long)h->step - 1);
  CK(launch_vcorr(src, S.n_c, S.nz, type, S.wall_z, h->d_vcorr, h->stream));
  std::vector<unsigned long long> v(words);
  CK(cudaMemcpyAsync(v.data(), h->d_vcorr, 8 * words, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const size_t all = 4 * (size_t)S.nz;
  const double cells = (double)v[all + 3];
  const double mean = (double)v[all + 1] / cells;
  const double var = (double)v[all + 0] / cells - mean * mean;
  for (int dz = 0; dz < S.nz; ++dz) {
    const double p = (double)v[4 * dz + 3];
    const double cov = (double)v[4 * dz] / p - ((double)v[4 * dz + 1] / p) * ((double)v[4 * dz + 2] / p);
    out[dz] = var > 0.0 ? cov / var : 0.0;
  }
  return SOMA_OK;
}

int soma_get_fields(soma_handle* h, int sys, float* out, size_t n, int where) {
  NvtxRange nvtx_range("soma_get_fields");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !out) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if (n != (size_t)(2 * S.n_c)) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  // the move kernel evaluates unheld fields from the counts on the fly: fill
  // the array from the counts of the current configuration first
  if (!S.frozen && !h->phi_pending[sys]) {
    CK(launch_field(h->fargs[sys], fixed_step((long long)h->step - 1), 0, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  CK(cudaMemcpy(out, S.w, sizeof(float) * n, where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  return SOMA_OK;
}

int soma_set_density(soma_handle* h, int sys, const float* phi, size_t n, int where) {
  NvtxRange nvtx_range("soma_set_density");
  SOMA_ENTER(h);
  if (h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys || !phi) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if (n != (size_t)(2 * S.n_c)) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  CK(cudaMemcpy(h->d_stage_phi, phi, sizeof(float) * n, where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  CK(launch_field_from_phi(h->d_sys, sys, h->d_stage_phi, h->sm_count, h->stream));
  h->phi_pending[sys] = 1;
  drop_graph(h);
  return sync_all(h);
}

int soma_freeze_fields(soma_handle* h, int sys, const float* w, size_t n, int where) {
  NvtxRange nvtx_range("soma_freeze_fields");
  SOMA_ENTER(h);
  if (h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if ((rc = sync_all(h))) return rc;
  if (w) {
    if (n != (size_t)(2 * S.n_c)) return SOMA_EINVAL;
    if ((rc = set_frozen(h, sys, 1))) return rc;
    h->phi_pending[sys] = 0;
    CK(cudaMemcpy(S.w, w, sizeof(float) * n, where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  } else {
    if ((rc = set_frozen(h, sys, 0))) return rc;
    h->phi_pending[sys] = 0;
    // the field array again follows the counts of the current configuration
    CK(launch_field(h->fargs[sys], fixed_step((long long)h->step - 1), 0, h->stream));
  }
  return sync_all(h);
}

int soma_get_state(soma_handle* h, int sys, float* pos, int16_t* img, uint64_t* step, int where) {
  NvtxRange nvtx_range("soma_get_state");
  SOMA_ENTER(h);
  if (h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if ((rc = sync_all(h))) return rc;
  if (pos || img) {
    CK(launch_gather_state(h->d_sys, sys, h->d_stage_pos, h->d_stage_img, h->sm_count, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const cudaMemcpyKind k = where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (pos) CK(cudaMemcpy(pos, h->d_stage_pos, (size_t)S.n_b * 12, k));
    if (img) CK(cudaMemcpy(img, h->d_stage_img, (size_t)S.n_b * 6, k));
  }
  if (step) *step = h->step;
  return SOMA_OK;
}

int soma_set_state(soma_handle* h, int sys, const float* pos, const int16_t* img, uint64_t step, int where) {
  NvtxRange nvtx_range("soma_set_state");
  SOMA_ENTER(h);
  if (h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys || !pos || !img) return SOMA_EINVAL;
  if (step >= (uint64_t)kInitStep) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if ((rc = sync_all(h))) return rc;
  // both copies, the validation and the read of its outcome are queued on
  // the handle's stream and waited for once (from pinned host memory the
  // copies run as DMA while the host queues the rest)
  const cudaMemcpyKind k = where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemsetAsync(h->d_err, 0, 4, h->stream));
  CK(cudaMemcpyAsync(h->d_stage_pos, pos, (size_t)S.n_b * 12, k, h->stream));
  CK(launch_validate_pos(h->d_stage_pos, S.n_b, S.L, h->d_err, h->sm_count, h->stream));
  CK(cudaMemcpyAsync(h->d_stage_img, img, (size_t)S.n_b * 6, k, h->stream));
  int err = 0;
  CK(cudaMemcpyAsync(&err, h->d_err, 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err) {
    CK(cudaMemset(h->d_err, 0, 4));
    return SOMA_EINVAL;  // a position outside [0, L): rejected, the state is untouched
  }
  CK(launch_scatter_state(h->d_sys, sys, h->d_stage_pos, h->d_stage_img, h->sm_count, h->stream));
  h->step = step;
  h->acc_since = step;
  CK(launch_set_step(h->d_step, h->n_sys, step, h->stream));
  h->dev_synced = true;
  CK(cudaMemsetAsync(h->d_acc, 0, sizeof(unsigned long long) * (size_t)h->acc_per_sys * h->n_sys, h->stream));
  std::fill(h->phi_pending.begin(), h->phi_pending.end(), 0);
  if ((rc = rebin_all(h, h->stream))) return rc;
  return sync_all(h);
}

int soma_get_state64(soma_handle* h, int sys, double* pos, int16_t* img, uint64_t* step, int where) {
  NvtxRange nvtx_range("soma_get_state64");
  SOMA_ENTER(h);
  if (!h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if ((rc = sync_all(h))) return rc;
  if (pos || img) {
    CK(launch_gather_state64(h->d_sys, sys, h->d_stage_pos64, h->d_stage_img, h->sm_count, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const cudaMemcpyKind k = where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (pos) CK(cudaMemcpy(pos, h->d_stage_pos64, (size_t)S.n_b * 24, k));
    if (img) CK(cudaMemcpy(img, h->d_stage_img, (size_t)S.n_b * 6, k));
  }
  if (step) *step = h->step;
  return SOMA_OK;
}

int soma_set_state64(soma_handle* h, int sys, const double* pos, const int16_t* img, uint64_t step, int where) {
  NvtxRange nvtx_range("soma_set_state64");
  SOMA_ENTER(h);
  if (!h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys || !pos || !img) return SOMA_EINVAL;
  if (step >= (uint64_t)kInitStep) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if ((rc = sync_all(h))) return rc;
  const cudaMemcpyKind k = where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemsetAsync(h->d_err, 0, 4, h->stream));
  CK(cudaMemcpyAsync(h->d_stage_pos64, pos, (size_t)S.n_b * 24, k, h->stream));
  CK(launch_validate_pos64(h->d_stage_pos64, S.n_b, S.L64, h->d_err, h->sm_count, h->stream));
  CK(cudaMemcpyAsync(h->d_stage_img, img, (size_t)S.n_b * 6, k, h->stream));
  int err = 0;
  CK(cudaMemcpyAsync(&err, h->d_err, 4, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (err) {
    CK(cudaMemset(h->d_err, 0, 4));
    return SOMA_EINVAL;
  }
  CK(launch_scatter_state64(h->d_sys, sys, h->d_stage_pos64, h->d_stage_img, h->sm_count, h->stream));
  h->step = step;
  h->acc_since = step;
  CK(launch_set_step(h->d_step, h->n_sys, step, h->stream));
  h->dev_synced = true;
  CK(cudaMemsetAsync(h->d_acc, 0, sizeof(unsigned long long) * (size_t)h->acc_per_sys * h->n_sys, h->stream));
  std::fill(h->phi_pending.begin(), h->phi_pending.end(), 0);
  if ((rc = rebin_all(h, h->stream))) return rc;
  return sync_all(h);
}

int soma_get_accepted(soma_handle* h, int sys, uint64_t* accepted) {
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !accepted) return SOMA_EINVAL;
  // the steps may have gone to a caller's stream: read after them
  CK(cudaStreamWaitEvent(h->stream, h->order_ev, 0));
  CK(launch_sum_acc(h->d_sys, sys, h->d_acc_sum, h->stream));
  unsigned long long a = 0;
  CK(cudaMemcpyAsync(&a, h->d_acc_sum, 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *accepted = a;
  return SOMA_OK;
}

int soma_copy_accepted(soma_handle* h, int sys, uint64_t* dst, void* stream) {
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !dst) return SOMA_EINVAL;
  cudaStream_t s = pick(h, stream);
  CK(cudaStreamWaitEvent(s, h->order_ev, 0));  // after the latest steps, on any stream
  // Pinned host memory that this device can address (8-byte aligned): the
  // reduction stores the count there itself, with no copy-engine round trip
  // behind the step.  Any other host memory: reduce, then copy.
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, dst) == cudaSuccess && at.type == cudaMemoryTypeHost &&
      at.devicePointer != nullptr && at.device == h->device &&
      (reinterpret_cast<uintptr_t>(at.devicePointer) & 7u) == 0) {
    CK(launch_sum_acc(h->d_sys, sys, static_cast<unsigned long long*>(at.devicePointer), s));
    return SOMA_OK;
  }
  (void)cudaGetLastError();  // an unregistered pointer is not an error here
  CK(launch_sum_acc(h->d_sys, sys, h->d_acc_sum, s));
  CK(cudaMemcpyAsync(dst, h->d_acc_sum, 8, cudaMemcpyDeviceToHost, s));
  return SOMA_OK;
}

int soma_observables(soma_handle* h, int sys, soma_obs* out) {
  NvtxRange nvtx_range("soma_observables");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !out) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if ((rc = sync_all(h))) return rc;
  CK(cudaMemsetAsync(h->d_obs, 0, 8 * sizeof(double), h->stream));
  CK(cudaMemsetAsync(h->d_acc_sum, 0, 8, h->stream));
  CK(launch_observables(h->d_sys, sys, (long long)h->step, h->d_obs, h->d_acc_sum, h->sm_count, h->stream));
  if (h->f64) {  // the chain sums again, from the FP64 positions
    CK(cudaMemsetAsync(h->d_obs, 0, 3 * sizeof(double), h->stream));
    CK(launch_obs_chains64(h->d_sys, sys, h->d_obs, h->sm_count, h->stream));
  }
  double r[8];
  unsigned long long acc = 0;
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(r, h->d_obs, sizeof(r), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&acc, h->d_acc_sum, 8, cudaMemcpyDeviceToHost));
  const soma_system_desc& d = h->desc[sys];
  out->step = h->step;
  out->accepted = acc;
  out->attempted = (uint64_t)S.n_b * (h->step - h->acc_since);
  out->acc = out->attempted ? (double)acc / (double)out->attempted : 0.0;
  out->Re2 = r[0] / S.n_poly;  // over the handle's chains (a partition: its own)
  out->Rg2 = r[1] / S.n_poly;
  out->Ebond = 1.5 * (d.N - 1) * r[2];
  out->Enb = (double)d.n_poly / (double)S.n_c * r[3];  // rho_bar / N of the whole system
  return SOMA_OK;
}

int soma_structure_factor(soma_handle* h, int sys, int nq, const int32_t* m_xyz, double* S_out) {
  NvtxRange nvtx_range("soma_structure_factor");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || nq < 0 || (nq > 0 && (!m_xyz || !S_out))) return SOMA_EINVAL;
  if (nq == 0) return SOMA_OK;
  if ((rc = sync_all(h))) return rc;
  if (nq > h->m_cap) {
    h->d_m = (int32_t*)dev_alloc(h, sizeof(int32_t) * 3 * nq);
    h->d_sq = (double*)dev_alloc(h, sizeof(double) * 2 * nq);
    if (!h->d_m || !h->d_sq) return fail(h, SOMA_ENOMEM);
    h->m_cap = nq;
  }
  CK(cudaMemcpy(h->d_m, m_xyz, sizeof(int32_t) * 3 * nq, cudaMemcpyHostToDevice));
  CK(cudaMemsetAsync(h->d_sq, 0, sizeof(double) * 2 * nq, h->stream));
  if (h->f64)
    CK(launch_structure_factor64(h->d_sys, sys, nq, h->d_m, h->d_sq, h->sm_count, h->stream));
  else
    CK(launch_structure_factor(h->d_sys, sys, nq, h->d_m, h->d_sq, h->sm_count, h->stream));
  std::vector<double> acc(2 * (size_t)nq);
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(acc.data(), h->d_sq, sizeof(double) * 2 * nq, cudaMemcpyDeviceToHost));
  const double nb = (double)h->host_sys[sys].n_b;
  for (int q = 0; q < nq; ++q) S_out[q] = (acc[2 * q] * acc[2 * q] + acc[2 * q + 1] * acc[2 * q + 1]) / nb;
  return SOMA_OK;
}

int soma_set_umbrella(soma_handle* h, int sys, const float* phi_target, size_t n, double lambdaN, int where) {
  NvtxRange nvtx_range("soma_set_umbrella");
  SOMA_ENTER(h);
  if (h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys) return SOMA_EINVAL;
  if (!std::isfinite(lambdaN) || lambdaN < 0.0) return SOMA_EINVAL;
  SysDev& S = h->host_sys[sys];
  const bool on = phi_target != nullptr && lambdaN > 0.0;
  if (on && n != (size_t)(2 * S.n_c)) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  if (on) {
    if (!S.phi_target) {
      S.phi_target = (float*)dev_alloc(h, sizeof(float) * 2 * (size_t)S.n_c);
      if (!S.phi_target) return SOMA_ENOMEM;
    }
    CK(cudaMemcpy(S.phi_target, phi_target, sizeof(float) * n,
                  where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    S.umbN_N = (float)(lambdaN / S.N);
    S.umbrella = 1;
  } else {
    S.umbN_N = 0.f;
    S.umbrella = 0;
  }
  CK(cudaMemcpy(h->d_sys + sys, &S, sizeof(SysDev), cudaMemcpyHostToDevice));
  build_args(h);
  drop_graph(h);
  // the field array (read by the generic move and by the next step when the
  // restraint is on) follows the new functional at once; fields the caller
  // supplied for the next step (soma_set_density) or holds stay as given
  if (!h->phi_pending[sys] && !S.frozen)
    CK(launch_field(h->fargs[sys], fixed_step((long long)h->step - 1), 0, h->stream));
  return sync_all(h);
}

int soma_set_conversion(soma_handle* h, int sys, int32_t n_A_alt, double zone_lo, double zone_hi, const double* p) {
  NvtxRange nvtx_range("soma_set_conversion");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys) return SOMA_EINVAL;
  SysDev& S = h->host_sys[sys];
  const bool on = n_A_alt >= 0;
  if (on) {
    if (h->f64 || S.P == 0) return SOMA_ENOTSUP;  // register-path FP32 systems only
    if (n_A_alt > S.N || !p) return SOMA_EINVAL;
    const double Lz = h->desc[sys].box[2];
    if (!std::isfinite(zone_lo) || !std::isfinite(zone_hi) || zone_lo < 0.0 || zone_hi < 0.0 ||
        zone_lo + zone_hi > Lz)
      return SOMA_EINVAL;
    for (int k = 0; k < 4; ++k)
      if (!(p[k] >= 0.0 && p[k] <= 1.0)) return SOMA_EINVAL;
  }
  if ((rc = sync_all(h))) return rc;
  if (on) {
    if (!S.conv_count) {
      S.conv_count = (unsigned long long*)dev_alloc(h, 32);
      if (!S.conv_count) return SOMA_ENOMEM;
    }
    CK(cudaMemset(S.conv_count, 0, 32));
    S.conv = 1;
    S.n_A_alt = n_A_alt;
    S.zone_lo = (float)zone_lo;
    S.zone_hi = (float)(h->desc[sys].box[2] - zone_hi);
    for (int k = 0; k < 4; ++k)  // convert iff word < floor(p 2^32 + 1/2)
      S.thr[k] = p[k] <= 0.0 ? 0ull
                 : p[k] >= 1.0 ? 4294967296ull
                               : (unsigned long long)std::floor(p[k] * 4294967296.0 + 0.5);
  } else if (S.conv) {  // off: every chain back to the system's own molecule
    CK(launch_set_types(h->d_sys, sys, nullptr, h->sm_count, h->stream));
    S.conv = 0;
  }
  CK(cudaMemcpy(h->d_sys + sys, &S, sizeof(SysDev), cudaMemcpyHostToDevice));
  build_args(h);
  drop_graph(h);
  if (!on) {  // the counts and fields follow the types
    h->phi_pending[sys] = 0;
    if ((rc = rebin_one(h, sys, h->stream))) return rc;
  }
  return sync_all(h);
}

int soma_get_conversions(soma_handle* h, int sys, uint64_t* out) {
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !out) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if ((rc = sync_all(h))) return rc;
  if (!S.conv_count) {
    for (int k = 0; k < 4; ++k) out[k] = 0;
    return SOMA_OK;
  }
  CK(cudaMemcpy(out, S.conv_count, 32, cudaMemcpyDeviceToHost));
  return SOMA_OK;
}

int soma_get_chain_types(soma_handle* h, int sys, uint8_t* out, size_t n) {
  NvtxRange nvtx_range("soma_get_chain_types");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !out) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if (n != (size_t)S.n_poly) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  uint8_t* stage = reinterpret_cast<uint8_t*>(h->d_stage_img);  // max_nb * 6 >= n_poly bytes
  CK(launch_get_types(h->d_sys, sys, stage, h->sm_count, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  CK(cudaMemcpy(out, stage, n, cudaMemcpyDeviceToHost));
  return SOMA_OK;
}

int soma_set_chain_types(soma_handle* h, int sys, const uint8_t* types, size_t n) {
  NvtxRange nvtx_range("soma_set_chain_types");
  SOMA_ENTER(h);
  if (sys < 0 || sys >= h->n_sys || !types) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if (n != (size_t)S.n_poly || !S.conv) return SOMA_EINVAL;
  for (size_t c = 0; c < n; ++c)
    if (types[c] > 1) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  uint8_t* stage = reinterpret_cast<uint8_t*>(h->d_stage_img);
  CK(cudaMemcpy(stage, types, n, cudaMemcpyHostToDevice));
  CK(launch_set_types(h->d_sys, sys, stage, h->sm_count, h->stream));
  // the counts of the current positions with the new types, and their fields
  h->phi_pending[sys] = 0;
  if ((rc = rebin_one(h, sys, h->stream))) return rc;
  return sync_all(h);
}

int soma_place(soma_handle* h, int sys, const float* phi_target, size_t n, int where) {
  NvtxRange nvtx_range("soma_place");
  SOMA_ENTER(h);
  if (h->f64) return SOMA_ENOTSUP;
  if (sys < 0 || sys >= h->n_sys || !phi_target) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  if (n != (size_t)(2 * S.n_c)) return SOMA_EINVAL;
  if ((rc = sync_all(h))) return rc;
  if (!h->place_temp) {
    h->place_temp_bytes = place_temp_bytes(h->max_nc);
    h->place_temp = dev_alloc(h, h->place_temp_bytes);
    if (!h->place_temp) return SOMA_ENOMEM;
  }
  CK(cudaMemcpy(h->d_stage_phi, phi_target, sizeof(float) * n,
                where == SOMA_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
  // the count buffers (24 bytes per cell) serve as the weights' scratch; the
  // counts are rebuilt below either way
  unsigned long long* q = reinterpret_cast<unsigned long long*>(S.counts);
  unsigned long long total = 0;
  CK(launch_place(h->d_sys, sys, S, h->d_stage_phi, q, q + S.n_c, h->place_temp, h->place_temp_bytes, &total,
                  h->sm_count, h->stream));
  if (total == 0) {
    if ((rc = rebin_all(h, h->stream))) return rc;
    if ((rc = sync_all(h))) return rc;
    return SOMA_EINVAL;  // no weight for bead 0's type: nothing placed
  }
  h->acc_since = h->step;
  CK(cudaMemsetAsync(h->d_acc, 0, sizeof(unsigned long long) * (size_t)h->acc_per_sys * h->n_sys, h->stream));
  std::fill(h->phi_pending.begin(), h->phi_pending.end(), 0);
  if ((rc = rebin_all(h, h->stream))) return rc;
  // placement leaves the chains in logical order: restore the cell order
  if (h->sort_interval > 0 && (rc = enqueue_reorder(h, h->stream))) return rc;
  return sync_all(h);
}

int soma_normal_deviates(const uint32_t* words, float* out, size_t n) {
  if (n == 0) return SOMA_OK;
  if (!words || !out) return SOMA_EINVAL;
  uint32_t* dw = nullptr;
  float* dout = nullptr;
  int rc = SOMA_ECUDA;
  if (cudaMalloc(&dw, n * 4) != cudaSuccess || cudaMalloc(&dout, n * 4) != cudaSuccess) {
    cudaGetLastError();
    rc = SOMA_ENOMEM;
  } else if (cudaMemcpy(dw, words, n * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
             launch_normal_words(dw, dout, (int64_t)n, nullptr) == cudaSuccess &&
             cudaMemcpy(out, dout, n * 4, cudaMemcpyDeviceToHost) == cudaSuccess) {
    rc = SOMA_OK;
  }
  cudaFree(dw);
  cudaFree(dout);
  return rc;
}

int soma_selfcheck_timeout(int device, uint64_t cycles) {
  if (cycles < 1000 || cycles > 20000000000ull) return SOMA_EINVAL;
  const DeviceScope device_scope(device);
  if (!device_scope.ok()) return SOMA_ECUDA;
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return SOMA_ENOMEM;
  }
  int rc = SOMA_ECUDA, value = 0;
  if (cudaMemset(err, 0, sizeof(int)) == cudaSuccess &&
      launch_wait_selfcheck(err, (long long)cycles, nullptr) == cudaSuccess &&
      cudaDeviceSynchronize() == cudaSuccess &&
      cudaMemcpy(&value, err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess)
    rc = (value & kErrTimeout) ? SOMA_ETIMEOUT : SOMA_OK;
  cudaFree(err);
  return rc;
}

int soma_reorder(soma_handle* h, void* stream) {
  NvtxRange nvtx_range("soma_reorder");
  SOMA_ENTER(h);
  if (h->f64) return SOMA_ENOTSUP;
  return enqueue_reorder(h, pick(h, stream));
}

int soma_get_info(soma_handle* h, int sys, soma_info* out) {
  if (!h || !out || sys < 0 || sys >= h->n_sys) return SOMA_EINVAL;
  const SysDev& S = h->host_sys[sys];
  out->n_beads = S.n_b;
  out->n_cells = S.n_c;
  out->k_b = S.kb;
  out->A = S.A;
  out->rho_bar = S.rho_bar;
  out->lanes_per_chain = S.P;
  out->ctas_per_sm = h->ctas_per_sm;
  out->sort_interval = h->sort_interval;
  out->hist_mode = h->hist_mode;
  out->move_warps = h->n_sys > 1 ? 8 : h->move_warps;
  return SOMA_OK;
}

int soma_kernel_times(soma_handle* h, double* ms, int64_t* launches, int reset) {
  if (!h) return SOMA_EINVAL;
  if (!h->pending.empty()) {
    CK(cudaDeviceSynchronize());
    for (auto& te : h->pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, te.a, te.b) == cudaSuccess) h->ms[te.kind] += t;
      cudaEventDestroy(te.a);
      cudaEventDestroy(te.b);
    }
    h->pending.clear();
  }
  for (int i = 0; i < 4; ++i) {
    if (ms) ms[i] = h->ms[i];
    if (launches) launches[i] = h->launches[i];
    if (reset) {
      h->ms[i] = 0;
      h->launches[i] = 0;
    }
  }
  return SOMA_OK;
}

// Autotuner: time a few steps per candidate (resident CTAs per SM of the
// move kernel, fused or separate histogram) from a saved copy of the state,
// restore the state between candidates and keep the fastest.  Random numbers
// are counter-based, so the restored trajectory is the one that would have
// run; the acceptance counters are restored as well.
int soma_autotune(soma_handle* h) {
  NvtxRange nvtx_range("soma_autotune");
  SOMA_ENTER(h);
  if (h->partition) return SOMA_ENOTSUP;  // its trial steps would run between count exchanges
  h->tuned = true;
  if ((rc = sync_all(h))) return rc;
  const uint64_t step0 = h->step;
  std::vector<std::vector<char>> save(h->n_sys);
  for (int s = 0; s < h->n_sys; ++s) {
    const SysDev& S = h->host_sys[s];
    save[s].resize((size_t)S.n_b * 20 + (size_t)S.n_poly * 4 + (size_t)S.n_c * 32);
    char* p = save[s].data();
    CK(cudaMemcpy(p, S.x, S.n_b * 4, cudaMemcpyDeviceToHost)); p += S.n_b * 4;
    CK(cudaMemcpy(p, S.y, S.n_b * 4, cudaMemcpyDeviceToHost)); p += S.n_b * 4;
    CK(cudaMemcpy(p, S.z, S.n_b * 4, cudaMemcpyDeviceToHost)); p += S.n_b * 4;
    CK(cudaMemcpy(p, S.img, S.n_b * 8, cudaMemcpyDeviceToHost)); p += S.n_b * 8;
    CK(cudaMemcpy(p, S.chain_id, (size_t)S.n_poly * 4, cudaMemcpyDeviceToHost)); p += (size_t)S.n_poly * 4;
    CK(cudaMemcpy(p, S.counts, S.n_c * 24, cudaMemcpyDeviceToHost)); p += S.n_c * 24;
    CK(cudaMemcpy(p, S.w, S.n_c * 8, cudaMemcpyDeviceToHost));
  }
  const size_t acc_n = (size_t)h->acc_per_sys * h->n_sys;
  std::vector<unsigned long long> acc_save(acc_n), conv_save(4 * (size_t)h->n_sys, 0ull);
  CK(cudaMemcpy(acc_save.data(), h->d_acc, 8 * acc_n, cudaMemcpyDeviceToHost));
  for (int s = 0; s < h->n_sys; ++s)
    if (h->host_sys[s].conv_count)
      CK(cudaMemcpy(&conv_save[4 * (size_t)s], h->host_sys[s].conv_count, 32, cudaMemcpyDeviceToHost));
  auto restore = [&]() -> int {
    for (int s = 0; s < h->n_sys; ++s) {
      const SysDev& S = h->host_sys[s];
      const char* p = save[s].data();
      CK(cudaMemcpy(S.x, p, S.n_b * 4, cudaMemcpyHostToDevice)); p += S.n_b * 4;
      CK(cudaMemcpy(S.y, p, S.n_b * 4, cudaMemcpyHostToDevice)); p += S.n_b * 4;
      CK(cudaMemcpy(S.z, p, S.n_b * 4, cudaMemcpyHostToDevice)); p += S.n_b * 4;
      CK(cudaMemcpy(S.img, p, S.n_b * 8, cudaMemcpyHostToDevice)); p += S.n_b * 8;
      CK(cudaMemcpy(S.chain_id, p, (size_t)S.n_poly * 4, cudaMemcpyHostToDevice)); p += (size_t)S.n_poly * 4;
      CK(cudaMemcpy(S.counts, p, S.n_c * 24, cudaMemcpyHostToDevice)); p += S.n_c * 24;
      CK(cudaMemcpy(S.w, p, S.n_c * 8, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(h->d_acc, acc_save.data(), 8 * acc_n, cudaMemcpyHostToDevice));
    for (int s = 0; s < h->n_sys; ++s)
      if (h->host_sys[s].conv_count)
        CK(cudaMemcpy(h->host_sys[s].conv_count, &conv_save[4 * (size_t)s], 32, cudaMemcpyHostToDevice));
    h->step = step0;
    return SOMA_OK;
  };
  const int steps = 6;
  float best = 1e30f;
  int best_c = h->ctas_per_sm, best_h = h->hist_mode, best_w = h->move_warps;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  const int timing = h->opt.kernel_timing;
  h->opt.kernel_timing = 0;
  // block shapes: one system tries 8, 12 and 24 consumer warps per CTA (the
  // batch kernel and the FP64 form have one shape)
  const bool shapes = h->n_sys == 1 && !h->f64 && h->host_sys[0].P > 0;
  for (int w : kMoveWarps) {
    if (w != 8 && !shapes) continue;
    if (h->opt.move_warps && w != h->opt.move_warps) continue;
    const int max_c = h->n_sys > 1 ? h->max_ctas_batch : shape_ctas(h, w);
    for (int c = 1; c <= max_c; ++c) {
      if (h->opt.ctas_per_sm && c != h->opt.ctas_per_sm) continue;
      for (int hm = SOMA_HIST_FUSED; hm <= SOMA_HIST_SEPARATE; ++hm) {
        if (h->opt.hist_mode != SOMA_HIST_AUTO && hm != h->opt.hist_mode) continue;
        apply_geometry(h, c, hm, w);
        if ((rc = enqueue_steps(h, h->stream, 2, false, (long long)step0))) return rc;  // warm-up
        CK(cudaEventRecord(a, h->stream));
        if ((rc = enqueue_steps(h, h->stream, steps, false, (long long)step0 + 2))) return rc;
        CK(cudaEventRecord(b, h->stream));
        CK(cudaEventSynchronize(b));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) {
          best = ms;
          best_c = c;
          best_h = hm;
          best_w = w;
        }
        if ((rc = restore())) return rc;
      }
    }
  }
  apply_geometry(h, best_c, best_h, best_w);

  // Sort interval (opt.sort_interval < 0): time one chain reorder, then the
  // step time at growing distances j from it (chains drift out of cell
  // order as they move); the interval K of least average cost per step,
  // (t_sort + sum_{i<K} t(i)) / K with t linear between the marks, wins.
  if (h->opt.sort_interval < 0 && !h->f64) {
    float t_sort = 0.f;
    CK(cudaEventRecord(a, h->stream));
    if ((rc = enqueue_reorder(h, h->stream))) return rc;
    CK(cudaEventRecord(b, h->stream));
    CK(cudaEventSynchronize(b));
    CK(cudaEventElapsedTime(&t_sort, a, b));
    const int marks[] = {0, 32, 64, 128, 256, 512, 1024};
    const int n_marks = (int)(sizeof(marks) / sizeof(marks[0]));
    float t_at[n_marks];
    long long done = 0;
    for (int m = 0; m < n_marks; ++m) {
      if (marks[m] > done) {
        if ((rc = enqueue_steps(h, h->stream, (int)(marks[m] - done), false, (long long)step0 + done))) return rc;
        done = marks[m];
      }
      CK(cudaEventRecord(a, h->stream));
      if ((rc = enqueue_steps(h, h->stream, 8, false, (long long)step0 + done))) return rc;
      CK(cudaEventRecord(b, h->stream));
      CK(cudaEventSynchronize(b));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, a, b));
      t_at[m] = ms / 8.f;
      done += 8;
    }
    if ((rc = restore())) return rc;
    double best_cost = 1e300;
    int best_k = h->sort_interval;
    for (int m = 1; m < n_marks; ++m) {
      const int K = marks[m];
      double sum = 0.0;  // trapezoids between the marks up to K
      for (int j = 1; j <= m; ++j) sum += 0.5 * (t_at[j - 1] + t_at[j]) * (marks[j] - marks[j - 1]);
      const double cost = (t_sort + sum) / K;
      if (cost < best_cost) {
        best_cost = cost;
        best_k = K;
      }
    }
    h->sort_interval = best_k;
    if ((rc = enqueue_reorder(h, h->stream))) return rc;  // start the tuned interval sorted
  }
  h->opt.kernel_timing = timing;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return sync_all(h);
}

int soma_philox4x32(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n) {
  if (n == 0) return SOMA_OK;
  if (!ctr || !key || !out) return SOMA_EINVAL;
  uint32_t* d = nullptr;
  if (cudaMalloc(&d, n * 40) != cudaSuccess) {
    cudaGetLastError();
    return SOMA_ENOMEM;
  }
  int rc = SOMA_OK;
  if (cudaMemcpy(d, ctr, n * 16, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d + 4 * n, key, n * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      launch_philox(d, d + 4 * n, d + 6 * n, (int64_t)n, 0) != cudaSuccess ||
      cudaMemcpy(out, d + 6 * n, n * 16, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = SOMA_ECUDA;
  cudaFree(d);
  return rc;
}

int soma_sort_pairs(const uint64_t* keys, const uint32_t* vals, size_t n, int end_bit, uint64_t* keys_out,
                    uint32_t* vals_out) {
  if (n == 0) return SOMA_OK;
  if (!keys || !vals || !keys_out || !vals_out || end_bit < 1 || end_bit > 64 || n > (size_t)UINT32_MAX)
    return SOMA_EINVAL;
  const size_t temp = radix_sort_temp_bytes((int64_t)n);
  char* d = nullptr;
  if (cudaMalloc(&d, n * 24 + temp) != cudaSuccess) {
    cudaGetLastError();
    return SOMA_ENOMEM;
  }
  auto* ka = reinterpret_cast<unsigned long long*>(d);
  auto* kb = ka + n;
  auto* va = reinterpret_cast<uint32_t*>(kb + n);
  auto* vb = va + n;
  bool in_b = false;
  int rc = SOMA_OK;
  if (cudaMemcpy(ka, keys, n * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(va, vals, n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      launch_radix_sort_pairs(ka, kb, va, vb, (int64_t)n, end_bit, vb + n, &in_b, 0) != cudaSuccess ||
      cudaMemcpy(keys_out, in_b ? kb : ka, n * 8, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(vals_out, in_b ? vb : va, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = SOMA_ECUDA;
  cudaGetLastError();
  cudaFree(d);
  return rc;
}

}  // extern "C"
