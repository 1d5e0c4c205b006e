/* soma.h -- C ABI of the B300 single-chain-in-mean-field Monte Carlo library.
 *
 * The library runs the SCMF Monte Carlo step of a soft coarse-grained AB
 * polymer melt on one GPU (the particle model of Sec. 2 of the paper, the
 * SOMA paragraph; its two dominant kernels, the bead-move kernel and the
 * density-field update, are the ones Sec. 2.2 profiles).  One step is:
 *
 *   (a) every bead proposes a uniform displacement d in [-A, A]^3 and is
 *       Metropolis-accepted against its two harmonic bonds, k_b = 3(N-1)/2,
 *       and the frozen per-cell field w_type; even beads of every chain move
 *       first, then odd beads (the two sets share no bond);
 *   (b) the final positions are re-binned into integer counts n_A(c), n_B(c);
 *   (c) the fields are rebuilt per cell from phi_t = n_t / rho_bar:
 *       w_A = [chiN phi_B + kappaN (phi_A + phi_B - 1)] / N, w_B likewise
 *       with phi_A in the chi term.
 *
 * Per system, instead of (a): bond-force-biased proposals (desc.move =
 * SOMA_MOVE_SMART); hard walls in z (desc.wall_z); molecule types with
 * conversion in boundary zones (soma_set_conversion); a restraint toward
 * target fields (soma_set_umbrella); fields given or held by the caller
 * (soma_set_density, soma_freeze_fields).
 *
 * Units: R_e = 1, kT = 1.  Random numbers: Philox4x32-10 (Salmon et al.,
 * SC'11) with counter (bead, logical chain, step, system_id) and key = seed,
 * so a trajectory does not depend on chain storage order or launch shape.
 *
 * Conventions for every call below:
 *   - The return value is SOMA_OK (0) or a negative SOMA_E* code; nothing
 *     else signals an error and no C++ exception crosses this boundary.  A
 *     handle keeps the first error it met (soma_last_error); once a CUDA
 *     error has occurred every later call on that handle returns SOMA_ESTATE.
 *   - The library owns all device memory it allocates (through the optional
 *     allocator in soma_options, else cudaMalloc).  Buffers passed in are
 *     owned by the caller; `where` says whether a pointer is host memory
 *     (SOMA_HOST) or device memory on the handle's GPU (SOMA_DEVICE).
 *   - Work is enqueued on the caller's CUDA stream (NULL = the handle's own
 *     stream).  Calls that return data to the host wait for all work on the
 *     device (soma_get_accepted and soma_copy_accepted order themselves
 *     after the latest soma_mc_steps only).  A handle is not thread-safe:
 *     the caller serialises the calls on one handle; distinct handles are
 *     independent.
 *   - Layouts: positions [bead][xyz] with bead = chain * N + i in LOGICAL
 *     chain order; counts and fields [type][cell], type 0 = A, 1 = B;
 *     cell = (ix * ny + iy) * nz + iz.
 *   - Positions are stored as FP32 wrapped into [0, L) plus an int16 image
 *     count per axis (unwrapped = x + image * L).  Bond vectors are taken by
 *     the minimum-image rule, so the box must exceed twice any bond length:
 *     soma_create rejects boxes with L < 16 / sqrt(3 (N - 1)) (eight bond
 *     standard deviations either way).
 */
#ifndef SOMA_H
#define SOMA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SOMA_OK 0
#define SOMA_EINVAL (-1)        /* bad argument or descriptor */
#define SOMA_ENOMEM (-2)        /* device or host allocation failed */
#define SOMA_ECUDA (-3)         /* a CUDA runtime call failed */
#define SOMA_ETIMEOUT (-4)      /* a bounded device-side wait ran out */
#define SOMA_EDEVICE_CHECK (-5) /* a device-side consistency check failed */
#define SOMA_ESTATE (-6)        /* handle already in a failed state */
#define SOMA_ENOTSUP (-7)       /* valid request the library does not support */

#define SOMA_HOST 0
#define SOMA_DEVICE 1

/* Position precision of a handle (soma_options.precision). */
#define SOMA_PREC_FP32 0  /* FP32 wrapped positions + int16 images: the throughput path */
#define SOMA_PREC_FP64 1  /* FP64 wrapped positions + int16 images: a precision reference
                             (one system per handle, no chain reorder, no autotuning) */

/* Histogram strategies of kernel (b) (soma_options.hist_mode). */
#define SOMA_HIST_AUTO 0
#define SOMA_HIST_FUSED 1     /* binned in the epilogue of the move kernel */
#define SOMA_HIST_SEPARATE 2  /* separate histogram kernel after the moves */

/* Trial-move kinds (soma_system_desc.move). */
#define SOMA_MOVE_UNIFORM 0 /* displacement uniform in [-A, A)^3 (step (a) above; Sec. 2, the SOMA paragraph) */
#define SOMA_MOVE_SMART 1   /* bond-force-biased ("smart") move named in Sec. 2: a
                               Gaussian displacement of per-axis variance s2 = A^2/3
                               centred on (s2/2) F, F the bond force on the bead, with
                               the proposal asymmetry in the acceptance.  N <= 64,
                               SOMA_PREC_FP32 only (else SOMA_ENOTSUP); needs
                               A^2 (N-1)/2 <= 1/2 and 6.93 A < every box edge
                               (else SOMA_EINVAL), so a proposal wraps at most once. */

/* One system: an AB diblock melt A_{n_A} B_{N - n_A} in a periodic box. */
typedef struct soma_system_desc {
  int32_t n_poly;  /* chains, >= 1 */
  int32_t N;       /* beads per chain, 1 <= N <= 4096 */
  int32_t n_A;     /* beads 0 .. n_A-1 of a chain are type A, 0 <= n_A <= N */
  int32_t system_id; /* fourth Philox counter word; systems that share a seed
                        need distinct ids.  A system's trajectory depends on
                        (seed, system_id) only, not on its place in a batch. */
  int32_t grid[3]; /* cells per axis, >= 1 each; total cells < 2^31 */
  int32_t move;    /* SOMA_MOVE_UNIFORM or SOMA_MOVE_SMART */
  double box[3];   /* box edges in R_e */
  double chiN;     /* Flory-Huggins chi times N */
  double kappaN;   /* Helfand compressibility kappa times N */
  double A;        /* proposal half-width; <= 0 selects 0.5 / sqrt(N - 1) */
  uint64_t seed;   /* Philox key */
  int32_t wall_z;  /* 0: periodic in z; 1: hard walls at z = 0 and z = L_z (the
                      particle subdomain as a slab between walls, Sec. 3.2):
                      a move leaving [0, L_z) is rejected, initial and placed
                      chains are folded into the slab by mirror reflection.
                      SOMA_ENOTSUP with SOMA_PREC_FP64. */
  int32_t reserved2; /* 0 */
} soma_system_desc;

typedef void* (*soma_alloc_fn)(size_t bytes, void* ctx);
typedef void (*soma_free_fn)(void* ptr, void* ctx);

typedef struct soma_options {
  int32_t device;        /* CUDA device ordinal; -1 = the device current at creation.  Every
                            call on the handle (creation and soma_destroy included) makes
                            this device current for its duration and restores the caller's
                            current device on return; streams passed to a call must belong
                            to it. */
  int32_t sort_interval; /* steps between chain reorders; 0 = never; -1 = tuned by the
                            autotuner (reorder cost against the step-time drift
                            after a reorder), 200 until it runs */
  int32_t ctas_per_sm;   /* resident CTAs per SM of the persistent move kernel; 0 = as many as fit */
  int32_t hist_mode;     /* SOMA_HIST_* */
  int32_t graph_steps;   /* steps per captured CUDA graph; 0 = plain launches */
  int32_t kernel_timing; /* 1 = record CUDA events around each kernel (plain launches) */
  int32_t autotune;      /* 1 = time candidate shapes on the first soma_mc_steps */
  int32_t precision;     /* SOMA_PREC_FP32 or SOMA_PREC_FP64 */
  soma_alloc_fn alloc;   /* optional device allocator, with free and ctx */
  soma_free_fn free;
  void* alloc_ctx;
  int32_t move_warps;    /* consumer warps per CTA of the one-system move kernel: 0 = 8, or the
                            autotuner's choice of 8, 12 and 24; 8, 12 or 24 fixes it (other
                            values: SOMA_EINVAL; a shape the device cannot launch:
                            SOMA_ENOTSUP).  A handle of several systems always uses 8 (the
                            batch kernel). */
  int32_t reserved;      /* 0 */
} soma_options;

typedef struct soma_obs {
  uint64_t step;      /* MC steps done */
  uint64_t accepted;  /* accepted moves since creation or the last set_state */
  uint64_t attempted; /* attempted moves over the same span */
  double acc;         /* accepted / attempted (0 if none) */
  double Re2;         /* mean over chains of |r_{N-1} - r_0|^2, unwrapped, FP64 sum */
  double Rg2;         /* mean over chains of (1/N) sum |r_i - r_cm|^2 */
  double Ebond;       /* k_b sum over bonds |b|^2 */
  double Enb;         /* (n_poly / n_c) sum_c [chiN phiA phiB + (kappaN/2)(phiA + phiB - 1)^2] */
} soma_obs;

typedef struct soma_info {
  int64_t n_beads, n_cells;
  double k_b;       /* 3 (N - 1) / 2 */
  double A;         /* proposal half-width actually used (FP32 value) */
  double rho_bar;   /* n_beads / n_cells */
  int32_t lanes_per_chain; /* move-kernel lanes per chain (0 = generic path) */
  int32_t ctas_per_sm;     /* move-kernel CTAs per SM in use */
  int32_t sort_interval;   /* reorder interval in use */
  int32_t hist_mode;       /* histogram strategy in use */
  int32_t move_warps;      /* consumer warps per CTA of the move kernel in use (8, 12 or 24) */
  int32_t reserved2;
} soma_info;

typedef struct soma_handle soma_handle;

/* Fill *opt with defaults (device -1, default sort interval, full occupancy,
 * SOMA_HIST_AUTO, graphs of 16 steps, no timing, no autotune).
 * Paper: no counterpart (configuration of this library). */
int soma_options_default(soma_options* opt);

/* Create a handle for n_sys independent systems that always step together
 * (each with its own descriptor, seed and system_id s).
 * Validates every descriptor, allocates device memory, builds the initial
 * configuration on the GPU (bead 0 uniform in the box, bonds Gaussian with
 * per-axis variance 1/(3(N-1)), Philox counter (bead, chain, 0xFFFFFFFF,
 * system_id)),
 * bins it, builds the fields and sorts the chains.  opt may be NULL.
 * Paper: Sec. 2, the SOMA paragraph (an SCMF system of soft coarse-grained
 * polymers: chain architecture, box, grid, chiN, kappaN) and Sec. 2.2 (SOMA
 * generates its bead coordinates and validates them on the GPU at start-up).
 * The initial Gaussian-chain configuration is a reading; the paper gives no
 * recipe. */
int soma_create(const soma_system_desc* sys, int n_sys, const soma_options* opt,
                soma_handle** out);
/* Chain partition of one system: a handle that holds the logical chains
 * [chain_begin, chain_end) of the system *sys describes (sys->n_poly is the
 * whole system's chain count).  Chains interact only through the fields,
 * which come from the whole system's counts, so the system splits into
 * partitions, one per GPU, that exchange exactly one thing per step: their
 * partial counts, summed over all partitions (soma_exchange_counts).
 * Random numbers follow logical chain ids, so the partitions of a system,
 * stepped with the exchange, reproduce the whole system's trajectory bit for
 * bit.  The partition's own chains are what soma_get_state/soma_set_state
 * (logical order, chain_begin first), soma_get_chain_types, the acceptance
 * counters, soma_observables' R_e^2, R_g^2 and E_bond and
 * soma_structure_factor cover; soma_observables' E_nb, soma_get_density,
 * soma_get_fields, soma_density_profile and soma_vertical_correlation read
 * the counts, which are the whole system's once exchanged.  rho_bar and every
 * field constant are the whole system's.
 * Constraints: N <= 64, SOMA_PREC_FP32 (else SOMA_ENOTSUP); opt->autotune = 0
 * and 0 <= chain_begin < chain_end <= sys->n_poly (else SOMA_EINVAL);
 * soma_mc_steps takes one step per call (else SOMA_EINVAL), so that the
 * exchange can follow it; soma_autotune returns SOMA_ENOTSUP.
 * Paper: Sec. 2.2, the SOMA scaling figure and its discussion (standalone
 * SOMA on 4 to 16 GPUs loses efficiency to the communication of the density
 * fields between GPUs); the chain split is the reading of that
 * decomposition. */
int soma_create_partition(const soma_system_desc* sys, const soma_options* opt, int32_t chain_begin,
                          int32_t chain_end, soma_handle** out);

/* The counts the next step of handle h reads: *counts receives a device
 * pointer (the handle's GPU, owned by the handle) to uint32 [n_cells][2] --
 * cell-major, the A and B counts of a cell side by side, cell = (ix * ny +
 * iy) * nz + iz -- and *n_words = 2 n_cells.  For a chain partition these
 * are its own chains' counts until the caller replaces them, in place, by
 * their sum over all partitions of the system (for example
 * ncclAllReduce(p, p, n_words, ncclUint32, ncclSum, comm, stream)), ordered
 * after the call that wrote them and before the next step: after
 * soma_create_partition, after every soma_mc_steps, and after soma_set_state,
 * soma_place and soma_set_chain_types.  For any other one-system handle the
 * same buffer holds the whole counts.  The pointer stays valid until the
 * handle's next call that steps or re-bins.  Does not synchronise.
 * SOMA_EINVAL for NULL arguments, a handle of several systems or
 * SOMA_PREC_FP64.
 * Paper: Sec. 2.2 (the density fields communicated between GPUs). */
int soma_exchange_counts(soma_handle* h, uint32_t** counts, size_t* n_words);

/* Paper: no counterpart (resource release and error reporting of this
 * library). */
void soma_destroy(soma_handle* h);
const char* soma_strerror(int code);
int soma_last_error(const soma_handle* h);

/* Enqueue n_steps MC steps of every system on `stream` (cudaStream_t, NULL =
 * the handle's stream).  Asynchronous.  Steps are numbered from the current
 * step counter; the step counter must stay below 2^32 - 1.
 * Paper: Sec. 2, the SOMA paragraph (MC propagation of the beads, non-bonded
 * interactions through quasi-instantaneous fields) and Sec. 2.2 (the two
 * kernels one step runs: mc_polymer_iteration, the trial moves and their
 * energies, and update_density_fields, the density fields). */
int soma_mc_steps(soma_handle* h, int64_t n_steps, void* stream);

/* Wait for the handle's work and check the device error word.
 * Paper: no counterpart. */
int soma_sync(soma_handle* h, void* stream);

/* Density counts of the current configuration, [2][n_cells] uint32, to host
 * or device memory per `where`.  SOMA_EINVAL for a bad sys index, a NULL out
 * or n != 2 n_cells.  Synchronises.
 * Paper: Sec. 2.2 (the particle density fields update_density_fields
 * builds) and Sec. 3.2 (the continuum model takes over the subdomain
 * concentrations the particle run returns). */
int soma_get_density(soma_handle* h, int sys, uint32_t* out, size_t n, int where);

/* Laterally averaged volume fractions of the current configuration along
 * one axis (0 = x, 1 = y, 2 = z): out[t * n_layers + k] = the mean over the
 * cells of layer k of n_t(c) / rho_bar, in FP64 from exact integer layer
 * sums (the profiles phi_t(z) Sec. 4 compares); n must be 2 * grid[axis]
 * (host buffer).  Synchronises.  Paper: Sec. 4 (the particle, continuum
 * and coupled runs are compared by such profiles). */
int soma_density_profile(soma_handle* h, int sys, int axis, double* out, size_t n);

/* Vertical correlation of the type-`type` counts of the current
 * configuration (the vertical correlation Sec. 4 compares):
 *   C(dz) = [<a b> - <a><b>] / [<n^2> - <n>^2],  a = n(c), b = n(c + dz e_z),
 * over all cell pairs at vertical distance dz (periodic in z, or only those
 * inside the slab with wall_z), the variance over all cells; from exact
 * integer sums, in FP64.  out has n = grid[2] entries, dz = 0 .. nz-1 (host
 * buffer); 0 where the field has no variance.  Synchronises.
 * Paper: Sec. 4 (a vertical correlation compares the runs; its formula is a
 * reading). */
int soma_vertical_correlation(soma_handle* h, int sys, int type, double* out, size_t n);

/* Fields used by the next step, [2][n_cells] FP32 (built from the current
 * counts unless held or supplied).  SOMA_EINVAL as for soma_get_density.
 * Synchronises.
 * Paper: Sec. 2, the SOMA paragraph (the quasi-instantaneous fields of the
 * non-bonded interactions); their functional form is a reading. */
int soma_get_fields(soma_handle* h, int sys, float* out, size_t n, int where);

/* Coupling write: replace the fields of the next step by those of the given
 * volume fractions phi [2][n_cells] (FP32, host or device per `where`;
 * copied); later steps rebuild from counts.
 * Paper: Sec. 3.2 (the particle run is handed the continuum's concentration
 * fields at each synchronisation).  SOMA_EINVAL for a bad sys, NULL
 * phi or n != 2 n_cells; SOMA_ENOTSUP on SOMA_PREC_FP64 handles.
 * Synchronises. */
int soma_set_density(soma_handle* h, int sys, const float* phi, size_t n, int where);

/* Coupling start-up (Sec. 3.2: molecules placed from the supplied
 * concentration fields are equilibrated under an umbrella potential).
 * Turn on a harmonic restraint toward target volume fractions
 * phi_target [2][n_cells] (FP32, host or device per `where`; copied):
 *   H_umb = (rho_bar/N) (lambdaN/2) sum_c sum_t (phi_t(c) - phi_target_t(c))^2,
 * which adds lambdaN (phi_t(c) - phi_target_t(c)) / N to the field of a
 * type-t bead in cell c from the next step on.  phi_target == NULL or
 * lambdaN == 0 turns it off.  lambdaN must be finite and >= 0
 * (SOMA_EINVAL); n must be 2 n_cells when on (SOMA_EINVAL); target values
 * are not checked.  The restraint enters every field build after the call;
 * fields already supplied for the next step by soma_set_density, or held by
 * soma_freeze_fields, stay as given.  While on, each step fills the field
 * array from the previous counts before the move kernel (one more launch per
 * step).
 * soma_observables' Enb excludes the restraint.  SOMA_ENOTSUP on
 * SOMA_PREC_FP64 handles.  Synchronises.
 * Paper: Sec. 3.2 (equilibration under an umbrella potential for about half
 * a synchronisation period); the harmonic form is a reading. */
int soma_set_umbrella(soma_handle* h, int sys, const float* phi_target, size_t n, double lambdaN, int where);

/* Coupling start-up: replace system `sys`'s configuration by molecules
 * placed from target volume fractions phi_target [2][n_cells] (FP32, host
 * or device; not retained).  Chain c's bead 0 goes to a point drawn from
 * the target of bead 0's type (cell weights floor(phi 2^16), 0 where
 * phi <= 0 or NaN) plus an offset uniform in [-h, h)^3, h = 1/(2 sqrt 3),
 * so within R_e/2 of it (Sec. 3.2); the chain keeps the Gaussian
 * conformation of the initial configuration.  Random numbers: Philox
 * counters (j, c, 0xFFFFFFFE, system_id), j = 0, 1, 2.  The step counter is
 * kept; counts and fields are rebuilt from the new state, and the
 * acceptance counters of every system of the handle restart (as after
 * soma_set_state).
 * SOMA_EINVAL (state kept) when the weights of bead 0's type sum to zero or
 * n != 2 n_cells; SOMA_ENOTSUP on SOMA_PREC_FP64 handles.  Synchronises.
 * Paper: Sec. 3.2 (molecules placed within half a mean end-to-end distance
 * of target positions that reproduce the supplied fields). */
int soma_place(soma_handle* h, int sys, const float* phi_target, size_t n, int where);

/* Boundary zones (Sec. 3.2): layers at the bottom and top of the box in z
 * where molecules are converted to and from the continuum model's units, at
 * rates the continuum model supplies and updates.  With conversion on,
 * every chain carries a molecule type: 0, the system's own architecture
 * (n_A A-beads), or 1, a converted molecule with n_A_alt A-beads (the rest
 * B).  Each step then opens with the conversions: a chain whose bead 0 lies
 * in the bottom zone (z < zone_lo) or the top zone (z >= L_z - zone_hi), both
 * compared in FP32 with the stored z, changes its type iff word 0 of the
 * Philox counter (0xFFFFFFFF, logical chain, step, system_id) is below
 * floor(p 2^32 + 1/2), p the zone's per-step probability for the chain's
 * current type: p[4] = {bottom 0->1, bottom 1->0, top 0->1, top 1->0} (host,
 * not retained).  The step's moves and counts use the new types; the fields
 * entering it come from the previous counts.  Calling again updates the
 * zones and rates (types kept) and restarts the conversion counts.
 * n_A_alt < 0 switches conversion off: every chain returns to type 0 and the
 * counts and fields are rebuilt.  soma_place and the initial configuration
 * build every chain as type 0.
 * SOMA_EINVAL for a bad sys, n_A_alt > N, p NULL or outside [0, 1], or zone
 * widths negative, not finite or together wider than L_z; SOMA_ENOTSUP on
 * SOMA_PREC_FP64 handles and for chains longer than 64 beads.  Synchronises.
 * Paper: Sec. 3.2 (boundary zones as transition layers converting particles
 * to and from continuum units at rates the continuum model updates); the
 * mechanism is a reading. */
int soma_set_conversion(soma_handle* h, int sys, int32_t n_A_alt, double zone_lo, double zone_hi, const double* p);
/* Conversions since the rates were last set, out[4] (host) in the order of
 * p above (zeros if conversion was never on).  SOMA_EINVAL for a bad sys or
 * NULL out.  Synchronises.  Paper: Sec. 3.2 (the boundary fluxes the
 * continuum model keeps track of). */
int soma_get_conversions(soma_handle* h, int sys, uint64_t* out);
/* Molecule type (0 or 1) of every chain in logical order, out[n_poly]
 * (host).  SOMA_EINVAL for a bad sys, NULL out or n != n_poly.
 * Synchronises.  Paper: Sec. 3.2 (molecule-type conversion). */
int soma_get_chain_types(soma_handle* h, int sys, uint8_t* out, size_t n);
/* Set the molecule types (conversion must be on; each 0 or 1), in logical
 * order, types[n_poly] (host); the counts of the current positions and
 * their fields are rebuilt with the new types (fields supplied for the next
 * step by soma_set_density are replaced).  With soma_get_state/soma_set_state
 * this completes a checkpoint.  SOMA_EINVAL (state kept) for a bad sys,
 * NULL types, n != n_poly, a value above 1, or conversion off.
 * Synchronises.  Paper: Sec. 3.2 (molecule-type conversion); the checkpoint
 * role has no counterpart. */
int soma_set_chain_types(soma_handle* h, int sys, const uint8_t* types, size_t n);

/* Test mode: hold the fields at w [2][n_cells] (FP32, copied) for every
 * later step (w == NULL releases them and rebuilds from the current counts).
 * SOMA_EINVAL for a bad sys or n != 2 n_cells; SOMA_ENOTSUP on
 * SOMA_PREC_FP64 handles.  Synchronises.
 * Paper: no counterpart.  It serves the reading of Sec. 2's
 * quasi-instantaneous fields as fixed within a step: with the fields held,
 * one bead or an AB dimer has an exact Boltzmann law that the tests check. */
int soma_freeze_fields(soma_handle* h, int sys, const float* w, size_t n, int where);

/* Checkpoint: positions [n_beads][3] FP32 wrapped into [0, L), images
 * [n_beads][3] int16, and the step counter, in logical chain order (host or
 * device buffers per `where`; any of pos, img, step may be NULL).  Molecule
 * types, when conversion is on, are saved separately (soma_get_chain_types).
 * SOMA_ENOTSUP on SOMA_PREC_FP64 handles.  Synchronises.
 * Paper: no counterpart (the paper restarts a subdomain by spawning a new
 * run, Sec. 3.2).  State out and in serve checkpoint/resume and the
 * step-by-step parity reading: the oracle and the GPU start each compared
 * step from the same FP32 state. */
int soma_get_state(soma_handle* h, int sys, float* pos, int16_t* img, uint64_t* step, int where);
/* Restore: positions must lie in [0, L) per axis (else SOMA_EINVAL and the
 * state is kept); resets the acceptance counters of every system of the
 * handle and re-bins; the step counter is shared by all systems and must be
 * below 2^32 - 1.  Synchronises.  Paper: as soma_get_state. */
int soma_set_state(soma_handle* h, int sys, const float* pos, const int16_t* img, uint64_t step,
                   int where);

/* The same for handles created with SOMA_PREC_FP64: positions FP64 [n][3].
 * Paper: no counterpart (the FP64 form measures what FP32 positions cost).
 * (soma_get_state / soma_set_state return SOMA_ENOTSUP on such handles.) */
int soma_get_state64(soma_handle* h, int sys, double* pos, int16_t* img, uint64_t* step, int where);
int soma_set_state64(soma_handle* h, int sys, const double* pos, const int16_t* img, uint64_t step,
                     int where);

/* FP64 observables of the current configuration (R_e^2, R_g^2 from
 * unwrapped positions, E_bond, E_nb from the counts, acceptance since the
 * last restore).  SOMA_EINVAL for a bad sys or NULL out.  Synchronises.
 * Paper: no counterpart; the paper defines none of these measures.  They
 * are the standard chain and melt observables the benchmark's statistical
 * parity and precision study use (E_nb is the H_nb of the field reading). */
int soma_observables(soma_handle* h, int sys, soma_obs* out);
/* Paper (this and soma_copy_accepted): no counterpart; the acceptance of the
 * trial moves of Sec. 2.2's move kernel.
 * Accepted-move counter only (one small device-to-host read, ordered after
 * the latest soma_mc_steps on whichever stream it was given; waits for it). */
int soma_get_accepted(soma_handle* h, int sys, uint64_t* accepted);
/* The same count, enqueued: on `stream` (NULL = the handle's stream), after
 * the latest soma_mc_steps, the count is reduced on the device and lands in
 * *dst (host memory).  Pinned host memory that the handle's device can
 * address, 8-byte aligned, is written by the reduction kernel itself (no
 * copy); other host memory gets an asynchronous copy (asynchronous only if
 * pinned).  Returns without waiting; *dst is valid once the stream has
 * synchronised.  Calls on one stream complete in order, so a caller may
 * enqueue one per step and read them all after a single synchronisation.
 * SOMA_EINVAL for a bad sys or NULL dst. */
int soma_copy_accepted(soma_handle* h, int sys, uint64_t* dst, void* stream);

/* S(q) = (1/n_beads) |sum_j s_j exp(i q.r_j)|^2, s_j = +1 (A) / -1 (B), for
 * q = 2 pi m / L at the nq integer triples m_xyz [nq][3] (host); S is FP64
 * [nq] (host).  SOMA_EINVAL for a bad sys, nq < 0 or NULL buffers (nq = 0
 * does nothing).
 * Synchronises.
 * Paper: no counterpart; the composition structure factor is the standard
 * measure of the microphase separation the model describes (Sec. 2). */
int soma_structure_factor(soma_handle* h, int sys, int nq, const int32_t* m_xyz, double* S);

/* Reorder the chains of every system now (storage order only; the
 * trajectory is unchanged because random numbers follow logical ids).
 * Paper: no counterpart; Sec. 2.2 names memory coalescing and data reuse as
 * what its kernel work improved, which the cell-sorted chain order serves. */
int soma_reorder(soma_handle* h, void* stream);

/* Shape and tuning facts of one system.  Paper: no counterpart. */
int soma_get_info(soma_handle* h, int sys, soma_info* out);

/* Launch counts of the move kernel, the separate histogram kernel, the field
 * kernel and the reorder since the last reset (launches[4]; plain launches --
 * launches replayed from a CUDA graph are not counted), and, with
 * kernel_timing = 1, their accumulated milliseconds (ms[4]; 0 otherwise).
 * Synchronises when timings are pending.
 * Paper: Sec. 2.2 profiles SOMA's time per kernel the same way. */
int soma_kernel_times(soma_handle* h, double* ms, int64_t* launches, int reset);

/* Run the autotuner now (also run by the first soma_mc_steps when
 * opt.autotune = 1).  The state is saved and restored, so the trajectory is
 * unchanged.  Synchronises.
 * Paper: Sec. 2.2 tunes launch configurations by hand; no counterpart. */
int soma_autotune(soma_handle* h);

/* The library's device Philox4x32-10 on n counters: ctr [n][4], key [n][2],
 * out [n][4], all uint32 host buffers (a verification aid; it runs the same
 * device function the move kernel uses).  Synchronous.
 * Paper: no counterpart (the generator is a reading). */
int soma_philox4x32(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n);

/* The library's stable radix sort on n (key, value) pairs: keys [n] uint64
 * and vals [n] uint32 (host, read), sorted by the key bits [0, end_bit)
 * into keys_out and vals_out (host, n entries each); pairs with equal key
 * bits keep their input order.  It is the sort of the chain reorder, which
 * orders chains by the Morton key of their first bead (a verification aid;
 * allocates and frees device memory).  SOMA_EINVAL for NULL buffers,
 * end_bit outside [1, 64] or n >= 2^32.  Synchronous.
 * Paper: no counterpart (Sec. 2.2 names data reuse among the optimisations;
 * the spatial chain order serves it). */
int soma_sort_pairs(const uint64_t* keys, const uint32_t* vals, size_t n, int end_bit, uint64_t* keys_out,
                    uint32_t* vals_out);

/* The standard normal deviates the smart move draws from n Philox words,
 * xi = Phi^-1(((w >> 8) + 1/2) 2^-24) as the kernel evaluates it (FP32,
 * the lower tail of either half through normcdfinvf); words and out are
 * host buffers of n entries (a verification aid).  Synchronous.
 * Paper: Sec. 2 (the bond-force-biased moves these deviates drive). */
int soma_normal_deviates(const uint32_t* words, float* out, size_t n);

/* Failure-path self-check (no counterpart in the paper, which names no
 * fault mechanism): on `device` (-1 = current) one thread waits, with the
 * move kernels' bounded mbarrier wait, on a barrier that nothing arrives
 * on, for at most `cycles` SM clock cycles (1e3 .. 2e10, else SOMA_EINVAL);
 * the caller's current device is restored on return.
 * Returns SOMA_ETIMEOUT when the wait gave up, set the device error bit and
 * returned as designed (the context stays usable); SOMA_OK would mean the
 * wait completed, SOMA_ECUDA / SOMA_ENOMEM a CUDA failure.  Allocates and
 * frees 4 bytes of device memory; synchronises the device. */
int soma_selfcheck_timeout(int device, uint64_t cycles);

/* S(q) of positions the caller already holds on the device, with no device
 * allocation: the paper has no counterpart; this entry point serves callers
 * that must not allocate GPU memory at the point of the call -- code whose
 * device memory comes from a fixed arena or pool it may not bypass, code on a
 * path where a cudaMalloc/cudaFree would synchronise the device with work in
 * flight, or a loop that samples S(q) often and cannot pay an allocation per
 * sample.  It needs no soma handle.
 *   pos    device FP32 [n_beads][3], wrapped into [0, L), bead = chain*N + i
 *   N, n_A chain length and A-block length: every chain is taken as the base
 *          diblock A_{n_A} B_{N-n_A} (no per-chain molecule types, so after
 *          boundary-zone conversion this differs from the handle's S(q))
 *   box    host double[3], the box edges
 *   m_xyz  host int32 [nq][3] integer q vectors, q = 2 pi m / L; each call
 *          copies them to the device with cudaMemcpyAsync on `stream`
 *   S      device double [nq] output, (1/n_beads)|sum_j s_j exp(i q.r_j)|^2
 *   stream cudaStream_t (NULL = default stream); asynchronous.
 * pos and S must be device memory of the current device with room for
 * 3 n_beads floats and nq doubles; they are not checked (SOMA_EINVAL only
 * for NULL pointers, n_beads < 1, N < 1, n_A outside [0, N], n_beads not a
 * multiple of N, a box edge <= 0, or nq outside [0, 4096]).
 * Scratch (the q list and the FP64 accumulators) is a fixed static device
 * array sized for at most 4096 q vectors (about 112 KiB on every GPU that
 * loads the library, held until exit); nq > 4096 returns SOMA_EINVAL.  The
 * first call on each device (that device current) looks up the array's
 * device address.  Calls are not for stream capture: each copies m_xyz from
 * the caller's host memory, which a capture refuses when it is pageable and,
 * when it is pinned, would re-read at every replay.  All calls share the
 * array and each clears it first: calls that overlap on the GPU race.
 * Never calls cudaMalloc, cudaFree or an allocating library routine. */
int soma_structure_factor_noalloc(const float* pos, int64_t n_beads, int32_t N, int32_t n_A,
                                  const double* box, int nq, const int32_t* m_xyz, double* S,
                                  void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SOMA_H */
