// soma_oracle.cpp -- TEST INFRASTRUCTURE, not part of the product path.
//
// A plain, slow, FP64 CPU restatement of the single-chain-in-mean-field (SCMF)
// Monte Carlo step that the paper's particle model (SOMA) runs (Sec. 2, the
// SOMA paragraph: soft coarse-grained polymer model, quasi-instantaneous
// fields for the non-bonded interactions, MC propagation of beads; Sec. 2.2:
// the two kernels that dominate, the move kernel and the density-field
// update).  Only tests, the package's smoke check and the benchmark's CPU
// baseline may load this library.  It shares no code, header, table or
// generator with the CUDA path.
//
// The paper names the model but prints none of its equations.  Every formula
// below is the standard SCMF bead-spring model written out in the order the
// step runs; each reading of an unstated detail is marked "Reading:".
//
// Conventions (all lengths in units of R_e = 1, energies in kT):
//   beads of chain c are i = 0..N-1; bead i is type A if i < n_A, else B;
//   positions are unwrapped FP64, stored pos[((c*N)+i)*3 + axis];
//   cells are c = (ix*ny + iy)*nz + iz; counts and fields are [type][cell].
//
// Parity status of each exported function (what pins it in tests/):
//   orc_philox4x32, orc_philox4x32_many
//                         pinned: an independent third-party Philox4x32-10
//                         (Triton's, run by its CPU interpreter) bit for bit;
//                         chi-square uniformity of its words.
//   orc_params            pinned: k_b, the proposal half-width (an FP32
//                         number) and rho_bar of the melt workloads as their
//                         definitions print them.
//   orc_cell_index        pinned with orc_density (brute-force binning).
//   orc_normal_quantile   pinned: scipy's ndtri and the mirror symmetry.
//   orc_init              pinned: bond statistics of a Gaussian chain
//                         (<b^2> = 1/(N-1), <R_e^2> = 1, <R_g^2> = (N+1)/6N).
//   orc_density           pinned: count invariants and brute-force binning.
//   orc_fields            pinned: central difference of the energy functional
//                         and the incompressible exchange-field special case.
//   orc_energy_nb         pinned absolutely on counts built by hand (a uniform
//                         phi_A = phi_B = 1/2 melt gives n_poly chiN/4, a
//                         one-cell excess, two hand-worked cells at two
//                         prefactors); its central differences are the fields.
//   orc_fields_from_phi   pinned: the incompressible exchange-field case.
//   orc_mc_step_chains    pinned: a sample of chains moves exactly as inside
//                         the whole step of orc_mc_step.
//   orc_mc_step/orc_run   pinned: <R_e^2> = 1 and the acceptance quadrature at
//                         chiN = kappaN = 0; Boltzmann occupancy of one bead in
//                         a frozen field; exact 64-state cell-pair law of an AB
//                         dimer on a 2^3 grid.
//   orc_observables       pinned: rigid straight and right-angle chains whose
//                         R_e^2, R_g^2 and bond energy are known by hand, and
//                         equipartition on Gaussian chains read through this
//                         function (<E_bond> per chain 3(N-1)/2, <R_e^2> = 1,
//                         <R_g^2> = (N+1)/6N); E_nb as orc_energy_nb.
//   orc_structure_factor  pinned: ideal-chain closed form at chiN = kappaN = 0.
//   force-biased moves    pinned: the same Gaussian-chain statistics, the
//                         one-bead Boltzmann law and the dimer cell-pair law
//                         (detailed balance makes them stationary).
//   orc_fields_umbrella   pinned: central difference of H_nb + H_umb.
//   orc_energy_umbrella   pinned absolutely on counts and targets by hand.
//   orc_vertical_correlation pinned: a cosine layer pattern (periodic), a
//                         linear ramp between walls (closed forms), C(0) = 1.
//   orc_density_profile   pinned: closed form on constructed counts and the
//                         mean over layers = the global composition.
//   wall confinement      pinned: the exact cell-pair law of an AB dimer
//                         between walls (no periodic images in z).
//   orc_place             pinned: the exact law of the bead-0 cell (target
//                         weights convolved with the uniform offset) and the
//                         Gaussian bond statistics of the placed chains.
//   orc_conversion_threshold, orc_convert
//                         pinned: the two-state Markov law of a molecule's
//                         type inside a zone (binomial counts after t steps),
//                         the zone occupancy law of bead 0 (uniform, so the
//                         fraction converted by certain flips is the zone's
//                         share of the box), and the one-bead Boltzmann law
//                         of a converted molecule's bead type.
//   The chiN, kappaN > 0 statistics of a dense melt have no closed form:
//   parity unpinned there except against this oracle itself.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

// One system: chain architecture, box, grid, interaction strengths, seed.
typedef struct {
  int32_t n_poly;     // number of chains
  int32_t N;          // beads per chain
  int32_t n_A;        // beads 0..n_A-1 are type A, the rest type B
  int32_t sys_index;  // system number s, the fourth Philox counter word
  int32_t grid[3];    // cells per axis
  int32_t move;       // 0: uniform proposal; 1: bond-force-biased (smart) proposal
  double box[3];      // box edge per axis, R_e units
  double chiN, kappaN;
  double A;           // proposal half-width; A <= 0 means 0.5/sqrt(N-1)
  uint64_t seed;      // Philox key (lo, hi)
  int32_t wall_z;     // 1: hard walls at z = 0 and z = L_z instead of periodic z
  int32_t pos64;      // 1: positions are held in FP64 (cell lookup in FP64), 0: in FP32
  // molecule types and boundary-zone conversion (Sec. 3.2), conv = 1:
  int32_t conv;       // 1: chains carry a molecule type and convert in the zones
  int32_t n_A_alt;    // beads 0..n_A_alt-1 of a converted (type-1) molecule are A
  double zone_lo;     // width of the bottom conversion zone, z in [0, zone_lo)
  double zone_hi;     // width of the top conversion zone, z in [L_z - zone_hi, L_z)
  uint64_t thr[4];    // thresholds {bottom 0->1, bottom 1->0, top 0->1, top 1->0}
  uint8_t* mol;       // molecule type per logical chain (0 own, 1 converted)
} orc_desc;

typedef struct {
  double Re2;    // mean over chains of |r_{N-1} - r_0|^2
  double Rg2;    // mean over chains of (1/N) sum_i |r_i - r_cm|^2
  double Ebond;  // k_b * sum over bonds |b|^2
  double Enb;    // (n_poly/n_c) sum_c [chiN phiA phiB + kappaN/2 (phiA+phiB-1)^2]
} orc_obs;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): a 4-word counter and a
// 2-word key; ten rounds, each multiplying counter words 0 and 2 by the two
// published round multipliers, crossing high halves into the other pair with
// the key, then bumping the key by the two published Weyl constants.
// ---------------------------------------------------------------------------
void orc_philox4x32(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    x0 = hi1 ^ x1 ^ k0;
    x1 = lo1;
    x2 = hi0 ^ x3 ^ k1;
    x3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox4x32_many(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  for (int64_t j = 0; j < n; ++j) orc_philox4x32(ctr + 4 * j, key + 2 * j, out + 4 * j);
}

// Reading: the counter of a bead move is (bead i, logical chain c, step t,
// system s) and the key is the 64-bit seed split (lo, hi).  Step value
// 0xFFFFFFFF is reserved for initialisation.
static void draw(const orc_desc* d, uint32_t bead, uint32_t chain, uint32_t step, uint32_t r[4]) {
  uint32_t ctr[4] = {bead, chain, step, (uint32_t)d->sys_index};
  uint32_t key[2] = {(uint32_t)(d->seed & 0xFFFFFFFFu), (uint32_t)(d->seed >> 32)};
  orc_philox4x32(ctr, key, r);
}

// Reading: a word w maps to a uniform on [0,1) as (w >> 8) * 2^-24 and to a
// uniform on the open interval (0,1) as ((w >> 9) + 1/2) * 2^-23.
static double unit_closed_open(uint32_t w) { return (double)(w >> 8) * 0x1p-24; }
static double unit_open(uint32_t w) { return ((double)(w >> 9) + 0.5) * 0x1p-23; }
static double unit_open24(uint32_t w) { return ((double)(w >> 8) + 0.5) * 0x1p-24; }

// The standard normal quantile x = Phi^-1(p), p in (0, 1): bisection to a
// bracket, then Newton steps on Phi(x) - p with Phi(x) = erfc(-x/sqrt 2)/2.
static double normal_quantile(double p) {
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 60; ++it) {
    double mid = 0.5 * (lo + hi);
    if (0.5 * std::erfc(-mid / std::sqrt(2.0)) < p) lo = mid; else hi = mid;
    if (hi - lo < 1e-6) break;
  }
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 4; ++it) {
    double f = 0.5 * std::erfc(-x / std::sqrt(2.0)) - p;
    double dens = std::exp(-0.5 * x * x) / std::sqrt(2.0 * M_PI);
    x -= f / dens;
  }
  return x;
}

double orc_normal_quantile(double p) { return normal_quantile(p); }

// ---------------------------------------------------------------------------
// Model constants.
// ---------------------------------------------------------------------------
// Harmonic bond energy (3(N-1)/2) |b|^2 in units of kT and R_e^2.
static double bond_k(const orc_desc* d) { return 1.5 * (double)(d->N - 1); }

// Proposal half-width: 0.5 R_e / sqrt(N-1) unless given; rounded through FP32
// so that both implementations use the identical constant.
static double proposal_A(const orc_desc* d) {
  double a = d->A > 0.0 ? d->A : 0.5 / std::sqrt((double)(d->N - 1));
  return (double)(float)a;
}

static int64_t n_beads(const orc_desc* d) { return (int64_t)d->n_poly * d->N; }
static int64_t n_cells(const orc_desc* d) {
  return (int64_t)d->grid[0] * d->grid[1] * d->grid[2];
}
// Bead i of logical chain c is type A (0) if i is below the A-block length
// of the chain's molecule type, else B (1).
static int type_of(const orc_desc* d, int64_t c, int i) {
  const int nA = (d->conv && d->mol && d->mol[c]) ? d->n_A_alt : d->n_A;
  return i < nA ? 0 : 1;
}

void orc_params(const orc_desc* d, double* k_b, double* A_eff, double* rho_bar) {
  *k_b = bond_k(d);
  *A_eff = proposal_A(d);
  *rho_bar = (double)n_beads(d) / (double)n_cells(d);
}

// Cell of a position: wrap into [0, L) per axis, scale by n/L, floor, clamp.
// Reading (precision of the lookup): the product is formed in the precision
// the positions are stored in -- in FP32 from the FP32-rounded coordinate and
// scale for the FP32 form, in FP64 for the FP64-position form.  For a
// coordinate that is an FP32 value and a power-of-two spacing L/n (every
// workload here) the two agree and equal the exact floor.
static int64_t cell_of(const orc_desc* d, const double r[3]) {
  int64_t idx[3];
  for (int a = 0; a < 3; ++a) {
    double L = d->box[a];
    double xw = r[a] - L * std::floor(r[a] / L);
    const double scaled = d->pos64 ? xw * ((double)d->grid[a] / L)
                                   : (double)((float)xw * (float)((double)d->grid[a] / L));
    int64_t i = (int64_t)std::floor(scaled);
    if (i > d->grid[a] - 1) i = d->grid[a] - 1;
    if (i < 0) i = 0;
    idx[a] = i;
  }
  return (idx[0] * d->grid[1] + idx[1]) * d->grid[2] + idx[2];
}

// Smallest distance from a position to a cell face (used by tests to set
// aside moves whose cell is decided by the last bits of a coordinate).
static double face_distance(const orc_desc* d, const double r[3]) {
  double best = 1e300;
  for (int a = 0; a < 3; ++a) {
    double L = d->box[a];
    double h = L / (double)d->grid[a];
    double xw = r[a] - L * std::floor(r[a] / L);
    double f = xw / h - std::floor(xw / h);
    double dist = std::fmin(f, 1.0 - f) * h;
    if (dist < best) best = dist;
  }
  return best;
}

int64_t orc_cell_index(const orc_desc* d, const double* r) { return cell_of(d, r); }

// ---------------------------------------------------------------------------
// Initial configuration: bead 0 uniform in the box, every bond vector an
// independent Gaussian with per-axis variance R_e^2 / (3(N-1)).
// Reading: bead 0 uses x_a = L_a * U(word a); bond i uses Box-Muller on word
// pairs (0,1) and (2,3), keeping three of the four normals.
// ---------------------------------------------------------------------------
// Reading of the wall confinement of Sec. 3.2 (the particle subdomain is a
// slab in z between walls): with wall_z the z axis is not periodic; a move
// whose proposal leaves [0, L_z) is rejected, and chains built by the
// initial configuration or the placement are folded into the slab by mirror
// reflection at the walls, z -> t if t < L_z else 2 L_z - t, t = z mod 2 L_z.
static double fold_z(double z, double L) {
  const double t = z - 2.0 * L * std::floor(z / (2.0 * L));
  double v = t < L ? t : 2.0 * L - t;
  if (v >= L) v = std::nextafter(L, 0.0);
  return v;
}

static void fold_chains(const orc_desc* d, double* pos) {
  if (!d->wall_z) return;
  for (int64_t b = 0; b < n_beads(d); ++b) pos[3 * b + 2] = fold_z(pos[3 * b + 2], d->box[2]);
}

static void init_chains(const orc_desc* d, double* pos);

void orc_init(const orc_desc* d, double* pos) {
  init_chains(d, pos);
  fold_chains(d, pos);
}

static void init_chains(const orc_desc* d, double* pos) {
  const double sigma = d->N > 1 ? std::sqrt(1.0 / (3.0 * (double)(d->N - 1))) : 0.0;
  const double two_pi = 2.0 * M_PI;
  for (int c = 0; c < d->n_poly; ++c) {
    double* p = pos + (int64_t)c * d->N * 3;
    for (int i = 0; i < d->N; ++i) {
      uint32_t r[4];
      draw(d, (uint32_t)i, (uint32_t)c, 0xFFFFFFFFu, r);
      if (i == 0) {
        for (int a = 0; a < 3; ++a) p[a] = d->box[a] * unit_closed_open(r[a]);
      } else {
        double rho1 = std::sqrt(-2.0 * std::log(unit_open24(r[0])));
        double rho2 = std::sqrt(-2.0 * std::log(unit_open24(r[2])));
        double z0 = rho1 * std::cos(two_pi * unit_closed_open(r[1]));
        double z1 = rho1 * std::sin(two_pi * unit_closed_open(r[1]));
        double z2 = rho2 * std::cos(two_pi * unit_closed_open(r[3]));
        p[3 * i + 0] = p[3 * (i - 1) + 0] + sigma * z0;
        p[3 * i + 1] = p[3 * (i - 1) + 1] + sigma * z1;
        p[3 * i + 2] = p[3 * (i - 1) + 2] + sigma * z2;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Density counts n_t(c): the number of beads of type t whose position lies in
// cell c (the density-field update of Sec. 2.2), recomputed from scratch.
// ---------------------------------------------------------------------------
void orc_density(const orc_desc* d, const double* pos, uint32_t* counts) {
  const int64_t nc = n_cells(d);
  std::memset(counts, 0, sizeof(uint32_t) * 2 * nc);
  for (int c = 0; c < d->n_poly; ++c)
    for (int i = 0; i < d->N; ++i) {
      const double* r = pos + ((int64_t)c * d->N + i) * 3;
      counts[type_of(d, c, i) * nc + cell_of(d, r)] += 1;
    }
}

// Quasi-instantaneous fields from the counts.  With phi_t = n_t / rho_bar the
// non-bonded energy is the Flory-Huggins term plus Helfand compressibility,
//   H_nb = (rho_bar/N) sum_c [chiN phiA phiB + (kappaN/2)(phiA + phiB - 1)^2],
// and the field a bead of type t feels in cell c is dH_nb / dn_t(c):
//   w_A = [chiN phiB + kappaN (phiA + phiB - 1)] / N,
//   w_B = [chiN phiA + kappaN (phiA + phiB - 1)] / N.
// Reading: the Flory-Huggins form of the chi term.
static void cell_fields(const orc_desc* d, double phiA, double phiB, double* wA, double* wB) {
  const double N = (double)d->N;
  double excess = phiA + phiB - 1.0;
  *wA = (d->chiN * phiB + d->kappaN * excess) / N;
  *wB = (d->chiN * phiA + d->kappaN * excess) / N;
}

void orc_fields(const orc_desc* d, const uint32_t* counts, double* w) {
  const int64_t nc = n_cells(d);
  const double rho_bar = (double)n_beads(d) / (double)nc;
  for (int64_t c = 0; c < nc; ++c)
    cell_fields(d, counts[c] / rho_bar, counts[nc + c] / rho_bar, &w[c], &w[nc + c]);
}

// Laterally averaged volume fractions along one axis (the layer profiles
// phi_t(z) that Sec. 4 compares between the particle, continuum and coupled
// runs): phi_t(k) = (1/m) sum over the m cells of layer k of n_t(c)/rho_bar,
// layer k = the cells whose index along `axis` is k.  out is [type][layer].
void orc_density_profile(const orc_desc* d, const uint32_t* counts, int axis, double* out) {
  const int64_t nc = n_cells(d);
  const double rho_bar = (double)n_beads(d) / (double)nc;
  const int n = d->grid[axis];
  const int64_t m = nc / n;
  for (int i = 0; i < 2 * n; ++i) out[i] = 0.0;
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t idx[3] = {c / ((int64_t)d->grid[1] * d->grid[2]), (c / d->grid[2]) % d->grid[1], c % d->grid[2]};
    for (int t = 0; t < 2; ++t) out[t * n + idx[axis]] += counts[t * nc + c] / rho_bar;
  }
  for (int i = 0; i < 2 * n; ++i) out[i] /= (double)m;
}

// Vertical correlation of the type-t counts (Sec. 4 compares a vertical
// correlation C(dz) of the concentration between runs; it gives no formula).
// Reading: the correlation coefficient of n_t(c) and n_t(c + dz e_z) over all
// cell pairs at vertical distance dz -- periodic in z, or, with walls, only
// the pairs inside the slab --, each pair set with its own means,
//   C(dz) = [<a b> - <a><b>] / [<n^2> - <n>^2],  a = n_t(c), b = n_t(c + dz e_z),
// the variance taken over all cells.  out[dz], dz = 0 .. nz-1.
void orc_vertical_correlation(const orc_desc* d, const uint32_t* counts, int type, double* out) {
  const int64_t nc = n_cells(d);
  const int nz = d->grid[2];
  const uint32_t* n = counts + (int64_t)type * nc;
  double s1 = 0.0, s2 = 0.0;
  for (int64_t c = 0; c < nc; ++c) {
    s1 += n[c];
    s2 += (double)n[c] * n[c];
  }
  const double var = s2 / nc - (s1 / nc) * (s1 / nc);
  for (int dz = 0; dz < nz; ++dz) {
    double sab = 0.0, sa = 0.0, sb = 0.0, pairs = 0.0;
    for (int64_t c = 0; c < nc; ++c) {
      const int iz = (int)(c % nz);
      int jz = iz + dz;
      if (jz >= nz) {
        if (d->wall_z) continue;
        jz -= nz;
      }
      const double a = n[c], b = n[c - iz + jz];
      sab += a * b;
      sa += a;
      sb += b;
      pairs += 1.0;
    }
    out[dz] = var > 0.0 ? (sab / pairs - (sa / pairs) * (sb / pairs)) / var : 0.0;
  }
}

// The non-bonded energy functional itself, H_nb from the counts.
double orc_energy_nb(const orc_desc* d, const uint32_t* counts) {
  const int64_t nc = n_cells(d);
  const double rho_bar = (double)n_beads(d) / (double)nc;
  double sum = 0.0;
  for (int64_t c = 0; c < nc; ++c) {
    double phiA = counts[c] / rho_bar, phiB = counts[nc + c] / rho_bar;
    double excess = phiA + phiB - 1.0;
    sum += d->chiN * phiA * phiB + 0.5 * d->kappaN * excess * excess;
  }
  return (double)d->n_poly / (double)nc * sum;
}

// Fields from given volume fractions (the coupling write of Sec. 3.2: the
// particle run is handed concentration fields).
void orc_fields_from_phi(const orc_desc* d, const double* phi, double* w) {
  const int64_t nc = n_cells(d);
  for (int64_t c = 0; c < nc; ++c) cell_fields(d, phi[c], phi[nc + c], &w[c], &w[nc + c]);
}

// ---------------------------------------------------------------------------
// Umbrella potential toward target volume fractions phi*_t(c) (the coupling
// of Sec. 3.2 equilibrates freshly placed molecules under an umbrella
// potential toward the supplied concentration fields).
// Reading: a harmonic restraint on every cell and type in the units of the
// compressibility term, with strength lambdaN >= 0,
//   H_umb = (rho_bar/N) (lambdaN/2) sum_c sum_t (phi_t(c) - phi*_t(c))^2,
// so the field it adds for a bead of type t in cell c is dH_umb/dn_t(c):
//   w_t^umb(c) = lambdaN (phi_t(c) - phi*_t(c)) / N.
// target is [type][cell].
// ---------------------------------------------------------------------------
double orc_energy_umbrella(const orc_desc* d, const uint32_t* counts, const double* target, double lambdaN) {
  const int64_t nc = n_cells(d);
  const double rho_bar = (double)n_beads(d) / (double)nc;
  double sum = 0.0;
  for (int64_t c = 0; c < 2 * nc; ++c) {
    const double dev = counts[c] / rho_bar - target[c];
    sum += dev * dev;
  }
  return rho_bar / (double)d->N * 0.5 * lambdaN * sum;
}

// The full fields with the umbrella term: w = w_nb + w^umb.
void orc_fields_umbrella(const orc_desc* d, const uint32_t* counts, const double* target, double lambdaN,
                         double* w) {
  const int64_t nc = n_cells(d);
  const double rho_bar = (double)n_beads(d) / (double)nc;
  orc_fields(d, counts, w);
  if (target)
    for (int64_t c = 0; c < 2 * nc; ++c) w[c] += lambdaN * (counts[c] / rho_bar - target[c]) / (double)d->N;
}

// ---------------------------------------------------------------------------
// Placement of molecules from target concentration fields (Sec. 3.2: a
// particle run starts from positions that reproduce the supplied fields,
// each molecule within half a mean end-to-end distance of its target).
// Reading: the target position of chain c is a point drawn from the target
// volume fraction of its bead-0 type, and bead 0 is put there plus a
// displacement uniform in [-h, h)^3 with h = 1/(2 sqrt 3), so |offset| <= 1/2;
// the chain keeps the Gaussian conformation of the initial configuration
// (the same bond draws), translated.  The target cell is chosen exactly:
// weights q(c) = floor(phi*(c) 2^16) (0 where phi* <= 0 or NaN; at most
// 2^32 - 256), running sums P(c) in 64-bit integers, k = floor(r Q / 2^64)
// with r = (w1 << 32 | w0) from counter (0, c, 0xFFFFFFFE, s) and Q the
// total; the cell is the first with P(c) > k.  Within the cell the point is
// (i_a + U(word a)) L_a/n_a from counter (1, c, 0xFFFFFFFE, s), and the
// offset is h (2 U(word a) - 1) from counter (2, c, 0xFFFFFFFE, s).
// target is the float32 [type][cell] array.  Returns 0, or -1 when the
// weights of bead 0's type sum to zero.
// ---------------------------------------------------------------------------
static uint32_t place_weight(float phi) {
  if (!(phi > 0.0f)) return 0u;
  const float v = std::fmin(phi * 65536.0f, 4294967040.0f);
  return (uint32_t)v;
}

int orc_place(const orc_desc* d, const float* target, double* pos) {
  const int64_t nc = n_cells(d);
  // every chain is built as the system's own molecule (type 0): its bead 0
  // has type A if n_A > 0
  if (d->conv && d->mol) std::memset(d->mol, 0, (size_t)d->n_poly);
  const float* phi = target + (int64_t)(d->n_A > 0 ? 0 : 1) * nc;
  std::vector<uint64_t> P(nc);
  uint64_t Q = 0;
  for (int64_t c = 0; c < nc; ++c) {
    Q += place_weight(phi[c]);
    P[c] = Q;
  }
  if (Q == 0) return -1;
  init_chains(d, pos);  // conformations (bead 0 is replaced below; folded at the end)
  const double h = 0.5 / std::sqrt(3.0);
  for (int c = 0; c < d->n_poly; ++c) {
    uint32_t r0[4], r1[4], r2[4];
    draw(d, 0u, (uint32_t)c, 0xFFFFFFFEu, r0);
    draw(d, 1u, (uint32_t)c, 0xFFFFFFFEu, r1);
    draw(d, 2u, (uint32_t)c, 0xFFFFFFFEu, r2);
    const uint64_t r = ((uint64_t)r0[1] << 32) | r0[0];
    const uint64_t k = (uint64_t)(((unsigned __int128)r * Q) >> 64);
    int64_t lo = 0, hi = nc - 1;  // first cell with P > k
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (P[mid] > k) hi = mid; else lo = mid + 1;
    }
    const int64_t cell = lo;
    const int64_t idx[3] = {cell / ((int64_t)d->grid[1] * d->grid[2]), (cell / d->grid[2]) % d->grid[1],
                            cell % d->grid[2]};
    double* p = pos + (int64_t)c * d->N * 3;
    double shift[3];
    for (int a = 0; a < 3; ++a) {
      const double x0 = ((double)idx[a] + unit_closed_open(r1[a])) * d->box[a] / d->grid[a] +
                        h * (2.0 * unit_closed_open(r2[a]) - 1.0);
      shift[a] = x0 - p[a];
    }
    for (int i = 0; i < d->N; ++i)
      for (int a = 0; a < 3; ++a) p[3 * i + a] += shift[a];
  }
  fold_chains(d, pos);
  return 0;
}

// ---------------------------------------------------------------------------
// One Monte Carlo step t with frozen fields w.
// Reading: the beads of a linear chain split into two sets, even i and odd
// i, that share no bond; set 0 (even) moves first for every chain, then set
// 1 (odd) sees the accepted set-0 positions.  The fields stay fixed for the
// whole step (quasi-instantaneous field approximation, Sec. 2).
// For every bead of the current set:
//   d_a   = A (2 U(word a) - 1), a = 0, 1, 2;  r' = r + d
//   dE    = k_b sum_{j = i +- 1, 0 <= j < N} (|r' - r_j|^2 - |r - r_j|^2)
//           + w_type(cell r') - w_type(cell r)
//   u     = open uniform from word 3
//   accept iff dE + ln u < 0   (Metropolis, strict)
// Optional per-bead records: accepted flag, the margin dE + ln u, and the
// smaller distance of r and r' to a cell face.  Returns the accepted count.
// ---------------------------------------------------------------------------
static int64_t move_set(const orc_desc* d, double* pos, const double* w, uint32_t t, int set,
                        const uint32_t* ids, int64_t n_chains, uint8_t* acc_out, double* margin_out,
                        double* face_out, int n_threads) {
  const int64_t nc = n_cells(d);
  const double k_b = bond_k(d);
  const double A = proposal_A(d);
  const int N = d->N;
  int64_t accepted = 0;
#pragma omp parallel for schedule(static) reduction(+ : accepted) num_threads(n_threads)
  for (int64_t c = 0; c < n_chains; ++c) {
    double* p = pos + c * N * 3;
    const uint32_t chain = ids ? ids[c] : (uint32_t)c;
    for (int i = set; i < N; i += 2) {
      uint32_t r[4];
      draw(d, (uint32_t)i, chain, t, r);
      double* ri = p + 3 * i;
      double rn[3];
      double dEb = 0.0, bias = 0.0;
      if (d->move == 0) {
        for (int a = 0; a < 3; ++a) rn[a] = ri[a] + A * (2.0 * unit_closed_open(r[a]) - 1.0);
        for (int j = i - 1; j <= i + 1; j += 2) {
          if (j < 0 || j >= N) continue;
          const double* rj = p + 3 * j;
          double new2 = 0.0, old2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            new2 += (rn[a] - rj[a]) * (rn[a] - rj[a]);
            old2 += (ri[a] - rj[a]) * (ri[a] - rj[a]);
          }
          dEb += new2 - old2;
        }
      } else {
        // Bond-force-biased move (Sec. 2 names the method; reading: the
        // force-biased Metropolis scheme with a Gaussian proposal of variance
        // s2 = A^2/3 per axis, the uniform proposal's variance, centred on the
        // drift (s2/2) F with F = -dE_bond/dr; the log-ratio of reverse and
        // forward proposal densities enters the acceptance, so detailed
        // balance holds).  Normals from words 0-2 by the inverse CDF of
        // ((w >> 8) + 1/2) 2^-24.
        const double s2 = A * A / 3.0;
        double F[3] = {0, 0, 0}, Fn[3] = {0, 0, 0};
        for (int j = i - 1; j <= i + 1; j += 2) {
          if (j < 0 || j >= N) continue;
          for (int a = 0; a < 3; ++a) F[a] -= 2.0 * k_b * (ri[a] - p[3 * j + a]);
        }
        double fwd = 0.0, rev = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double xi = normal_quantile(unit_open24(r[a]));
          rn[a] = ri[a] + 0.5 * s2 * F[a] + std::sqrt(s2) * xi;
        }
        for (int j = i - 1; j <= i + 1; j += 2) {
          if (j < 0 || j >= N) continue;
          const double* rj = p + 3 * j;
          double new2 = 0.0, old2 = 0.0;
          for (int a = 0; a < 3; ++a) {
            new2 += (rn[a] - rj[a]) * (rn[a] - rj[a]);
            old2 += (ri[a] - rj[a]) * (ri[a] - rj[a]);
            Fn[a] -= 2.0 * k_b * (rn[a] - rj[a]);
          }
          dEb += new2 - old2;
        }
        for (int a = 0; a < 3; ++a) {
          const double f = rn[a] - ri[a] - 0.5 * s2 * F[a];   // forward: r -> r'
          const double b = ri[a] - rn[a] - 0.5 * s2 * Fn[a];  // reverse: r' -> r
          fwd += f * f;
          rev += b * b;
        }
        bias = (rev - fwd) / (2.0 * s2);  // -ln[q(r'->r) / q(r->r')]
      }
      const double* wt = w + (int64_t)type_of(d, chain, i) * nc;
      double margin;
      if (d->wall_z && !(rn[2] >= 0.0 && rn[2] < d->box[2])) {
        margin = HUGE_VAL;  // through a wall: rejected
      } else {
        double dE = k_b * dEb + wt[cell_of(d, rn)] - wt[cell_of(d, ri)];
        margin = dE + bias + std::log(unit_open(r[3]));
      }
      bool ok = margin < 0.0;
      int64_t b = c * N + i;
      if (acc_out) acc_out[b] = ok ? 1 : 0;
      if (margin_out) margin_out[b] = margin;
      if (face_out) face_out[b] = std::fmin(face_distance(d, ri), face_distance(d, rn));
      if (ok) {
        for (int a = 0; a < 3; ++a) ri[a] = rn[a];
        accepted += 1;
      }
    }
  }
  return accepted;
}

int64_t orc_mc_step(const orc_desc* d, double* pos, const double* w, uint32_t t, uint8_t* acc_out,
                    double* margin_out, double* face_out, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  int64_t a0 = move_set(d, pos, w, t, 0, nullptr, d->n_poly, acc_out, margin_out, face_out, n_threads);
  int64_t a1 = move_set(d, pos, w, t, 1, nullptr, d->n_poly, acc_out, margin_out, face_out, n_threads);
  return a0 + a1;
}

// The same step for a sample of chains only: pos holds n_chains chains whose
// logical ids (the Philox chain word) are ids[]; w is the full system's field.
// Chains interact only through the frozen fields, so a sample moves exactly
// as it would inside the whole system.
int64_t orc_mc_step_chains(const orc_desc* d, double* pos, const uint32_t* ids, int64_t n_chains,
                           const double* w, uint32_t t, uint8_t* acc_out, double* margin_out,
                           double* face_out, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  int64_t a0 = move_set(d, pos, w, t, 0, ids, n_chains, acc_out, margin_out, face_out, n_threads);
  int64_t a1 = move_set(d, pos, w, t, 1, ids, n_chains, acc_out, margin_out, face_out, n_threads);
  return a0 + a1;
}

// ---------------------------------------------------------------------------
// Observables (FP64).  Reading: the paper defines none; these are the
// standard chain and melt measures.
// ---------------------------------------------------------------------------
void orc_observables(const orc_desc* d, const double* pos, orc_obs* out) {
  const int N = d->N;
  double re2 = 0.0, rg2 = 0.0, eb = 0.0;
  for (int c = 0; c < d->n_poly; ++c) {
    const double* p = pos + (int64_t)c * N * 3;
    double e2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      double v = p[3 * (N - 1) + a] - p[a];
      e2 += v * v;
    }
    re2 += e2;
    double cm[3] = {0, 0, 0};
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < 3; ++a) cm[a] += p[3 * i + a] / N;
    double g2 = 0.0;
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < 3; ++a) g2 += (p[3 * i + a] - cm[a]) * (p[3 * i + a] - cm[a]);
    rg2 += g2 / N;
    for (int i = 1; i < N; ++i)
      for (int a = 0; a < 3; ++a) {
        double b = p[3 * i + a] - p[3 * (i - 1) + a];
        eb += b * b;
      }
  }
  out->Re2 = re2 / d->n_poly;
  out->Rg2 = rg2 / d->n_poly;
  out->Ebond = bond_k(d) * eb;

  std::vector<uint32_t> counts(2 * n_cells(d));
  orc_density(d, pos, counts.data());
  out->Enb = orc_energy_nb(d, counts.data());
}

// Collective structure factor of the composition, S(q) = (1/n_b) |sum_j s_j
// exp(i q.r_j)|^2 with s_j = +1 for A and -1 for B, at the lattice vectors
// q = 2 pi m / L for the nq integer triples m.
void orc_structure_factor(const orc_desc* d, const double* pos, int nq, const int32_t* m,
                          double* S) {
  const int64_t nb = n_beads(d);
  for (int k = 0; k < nq; ++k) {
    double q[3];
    for (int a = 0; a < 3; ++a) q[a] = 2.0 * M_PI * (double)m[3 * k + a] / d->box[a];
    double re = 0.0, im = 0.0;
    for (int c = 0; c < d->n_poly; ++c)
      for (int i = 0; i < d->N; ++i) {
        const double* r = pos + ((int64_t)c * d->N + i) * 3;
        double ph = q[0] * r[0] + q[1] * r[1] + q[2] * r[2];
        double s = type_of(d, c, i) == 0 ? 1.0 : -1.0;
        re += s * std::cos(ph);
        im += s * std::sin(ph);
      }
    S[k] = (re * re + im * im) / (double)nb;
  }
}

// ---------------------------------------------------------------------------
// Boundary zones (Sec. 3.2): transition layers at the bottom and top of the
// box in z where molecules are converted to and from the continuum model's
// units, at conversion rates the continuum model supplies.
// Reading: each chain carries a molecule type m (0: the system's own
// architecture, n_A A-beads; 1: a converted molecule, n_A_alt A-beads).  At
// the start of step t, before set 0, a chain whose bead 0 lies in a zone --
// its wrapped z, as the FP32 number the positions are stored in, below
// (float)zone_lo (bottom), else at or above (float)(L_z - zone_hi) (top) --
// draws word 0 of the Philox counter (0xFFFFFFFF, c, t, s) (a bead word no
// bead has) and changes its type iff that word is below the threshold of
// its zone and current type, thr = floor(p 2^32 + 1/2) for the per-step
// probability p.  Positions are untouched; the step's moves and counts see
// the new types, the fields entering the step come from the previous counts.
// Returns the conversions, per zone and direction, in counts4 (if given).
// ---------------------------------------------------------------------------
uint64_t orc_conversion_threshold(double p) {
  if (!(p > 0.0)) return 0;
  if (p >= 1.0) return 4294967296ull;
  return (uint64_t)std::floor(p * 4294967296.0 + 0.5);
}

void orc_convert(const orc_desc* d, const double* pos, uint32_t t, int64_t* counts4) {
  if (!d->conv || !d->mol) return;
  const double L = d->box[2];
  const float zlo = (float)d->zone_lo;
  const float zhi = (float)(L - d->zone_hi);
  for (int c = 0; c < d->n_poly; ++c) {
    const double z = pos[(int64_t)c * d->N * 3 + 2];
    const float zw = d->wall_z ? (float)z : (float)(z - L * std::floor(z / L));
    int zone;
    if (zw < zlo)
      zone = 0;
    else if (zw >= zhi)
      zone = 1;
    else
      continue;
    uint32_t r[4];
    draw(d, 0xFFFFFFFFu, (uint32_t)c, t, r);
    const int m = d->mol[c];
    if ((uint64_t)r[0] < d->thr[2 * zone + m]) {
      d->mol[c] = (uint8_t)(1 - m);
      if (counts4) counts4[2 * zone + m] += 1;
    }
  }
}

// ---------------------------------------------------------------------------
// A run of n_steps steps starting at step t0.  Unless w_frozen is given, the
// fields entering step t come from the counts after step t-1 (or after the
// initial configuration), with the umbrella term when target is given; with
// conversion on, each step starts with the boundary-zone conversions.
// Optional accumulators per step: occupancy counts
// summed over steps, the joint cell histogram of two-bead chains, R_e^2 and
// the accepted count.  Returns the total accepted count.
// ---------------------------------------------------------------------------
int64_t orc_run(const orc_desc* d, double* pos, uint32_t t0, int64_t n_steps,
                const double* w_frozen, const double* target, double lambdaN, int n_threads, uint64_t* occ,
                uint64_t* pair_hist, double* re2_trace, int64_t* acc_trace) {
  const int64_t nc = n_cells(d);
  std::vector<uint32_t> counts(2 * nc);
  std::vector<double> w(2 * nc);
  if (w_frozen) {
    std::memcpy(w.data(), w_frozen, sizeof(double) * 2 * nc);
  } else {
    orc_density(d, pos, counts.data());
    orc_fields_umbrella(d, counts.data(), target, lambdaN, w.data());
  }
  int64_t total = 0;
  for (int64_t s = 0; s < n_steps; ++s) {
    orc_convert(d, pos, (uint32_t)(t0 + s), nullptr);
    int64_t a = orc_mc_step(d, pos, w.data(), (uint32_t)(t0 + s), nullptr, nullptr, nullptr,
                            n_threads);
    total += a;
    if (acc_trace) acc_trace[s] = a;
    if (!w_frozen || occ) orc_density(d, pos, counts.data());
    if (!w_frozen) orc_fields_umbrella(d, counts.data(), target, lambdaN, w.data());
    if (occ)
      for (int64_t c = 0; c < 2 * nc; ++c) occ[c] += counts[c];
    if (pair_hist && d->N == 2)
      for (int c = 0; c < d->n_poly; ++c) {
        const double* p = pos + (int64_t)c * 6;
        pair_hist[cell_of(d, p) * nc + cell_of(d, p + 3)] += 1;
      }
    if (re2_trace) {
      double re2 = 0.0;
      for (int c = 0; c < d->n_poly; ++c) {
        const double* p = pos + (int64_t)c * d->N * 3;
        for (int a = 0; a < 3; ++a) {
          double v = p[3 * (d->N - 1) + a] - p[a];
          re2 += v * v;
        }
      }
      re2_trace[s] = re2 / d->n_poly;
    }
  }
  return total;
}

}  // extern "C"
