/*
 * md.h -- C ABI of the GB300 engine for united-atom polyethylene molecular
 * dynamics (Xu, Ren, Ge, Yu, Yang, Li: "Molecular Dynamics Simulation of
 * Macromolecules Using Graphics Processing Unit").
 *
 * What a system is (Sec. 2, Table I, Table II): molecules of one type, linear
 * chains of `sites_per_chain` united atoms (CH3 ends = type C_33, CH2 interior
 * = type C_32), in a periodic cube.  Energy E = E_nb + E_b + E_a + E_d
 * (Eqs. 1, 3): truncated Lennard-Jones between all pairs except 1-2 and 1-3
 * bonded neighbours (Eq. 2, Sec. 3.1), harmonic bonds (Eq. 4), harmonic angles
 * in theta (Eq. 5) and cosine dihedrals (Eq. 6).  Each call below runs the
 * per-timestep path of Secs. 3.1-3.4 entirely on one GPU: binning into cells,
 * neighbour list every `rebin_every` steps, LJ and bonded forces, integration.
 *
 * Units: nm, ps, amu, kJ/mol, kelvin.  Forces kJ/mol/nm.
 * Atom order: "original order" = replicas concatenated, chain-major inside a
 * replica (atom = chain * sites_per_chain + MAIDX - 1, 0-based: GAIDX - 1).
 *
 * Ownership: every pointer argument is a HOST pointer unless stated.  Input
 * arrays are copied during the call; output arrays are written by the call.
 * No pointer is retained after a call returns, except `workspace` (below).
 *
 * Errors: every int-returning function returns MD_OK (0) or a negative
 * MD_E* code; md_last_error() then holds a one-line message.  Device-side
 * conditions (neighbour-list overflow, fixed-point overflow, non-finite
 * state) are raised on the GPU as flags and reported by the next
 * synchronising call (md_step, md_sync).  A displacement beyond skin/2 is
 * not an error unless md_desc.displacement = MD_DISP_ERROR: it triggers an
 * extra rebuild (md_early_rebins).  The library
 * never traps or spins on the GPU.
 *
 * Threads: a system must not be used from two host threads at once.
 */
#ifndef MD_GB300_H
#define MD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  MD_OK = 0,
  MD_EINVAL = -1,      /* malformed descriptor or argument */
  MD_ENOMEM = -2,      /* device allocation failed or workspace too small */
  MD_ECUDA = -3,       /* a CUDA call failed */
  MD_EOVERFLOW = -4,   /* neighbour-list capacity or fixed-point range exceeded */
  MD_EUNSTABLE = -5,   /* non-finite state, or (MD_DISP_ERROR) an atom moved more than skin/2 */
  MD_ETIMEOUT = -6     /* a bounded device wait gave up */
};

enum { MD_PLAIN_FP32 = 0, MD_MIXED = 1 };   /* precision forms */
enum { MD_NVE = 0, MD_VRESCALE = 1, MD_NOSE_HOOVER = 2 };   /* thermostat */
/* LJ work schedule: one thread block per region of cells, or a fixed grid
 * (resident blocks x SMs) whose blocks take regions from a device counter.
 * Both give the same forces bit for bit.  The list build always runs one
 * block per region. */
enum { MD_SCHED_GRID = 0, MD_SCHED_PERSISTENT = 1 };
/* What a step does when an atom has moved more than skin/2 since the last
 * list build: rebuild the bins and list before its forces (a conditional
 * node in the step graph), or report MD_EUNSTABLE at the next synchronising
 * call (graphs without conditional nodes, which profilers can take apart). */
enum { MD_DISP_REBUILD = 0, MD_DISP_ERROR = 1 };

typedef struct md_system md_system;         /* opaque, owned by the library */

/* Force-field parameters (Table I; index 0 = C_32, 1 = C_33).  Unlike pairs
 * use geometric means of eps and sigma. */
typedef struct {
  double eps[2];      /* LJ well depth, kJ/mol (Eq. 2) */
  double sigma[2];    /* LJ sigma, nm (Eq. 2) */
  double mass[2];     /* amu */
  double kb, b0;      /* Eq. 4: kJ/mol/nm^2, nm */
  double ka, theta0;  /* Eq. 5: kJ/mol/rad^2, rad */
  double kphi, phis;  /* Eq. 6: kJ/mol, rad */
  int32_t n_mult;     /* Eq. 6 periodicity n */
  int32_t pad;
} md_params;

/* Molecule topology (Sec. 3.3): the one molecule type of a system, naom
 * atoms with a bond graph and a type per atom.  From it the library builds
 * the per-type lists the paper describes: t_exclusions (every atom's 1-2
 * and 1-3 neighbours, left out of the LJ sum, Sec. 3.1), t_bonds, t_angles
 * (every path a-b-c, vertex b) and the dihedral analogue (every path
 * a-b-c-d around each bond b-c), and evaluates every term once per molecule.
 * Copied during md_create.  md_desc.topology = NULL means linear chains of
 * sites_per_chain atoms with C_33 ends (the paper's polyethylene), which
 * take the faster chain kernels; a topology needs the mixed precision form,
 * and md_observables, md_acf_sample and md_rdf (defined for linear chains)
 * then return MD_EINVAL. */
typedef struct {
  int32_t naom;                /* atoms per molecule (NAOM, Table II), 4 .. 1023 */
  int32_t n_bonds;             /* bonds per molecule, 1 .. 4 naom */
  const int32_t *bonds;        /* [2 * n_bonds] atom pairs, 0-based index in the molecule (MAIDX - 1) */
  const int32_t *types;        /* [naom] 0 = C_32, 1 = C_33 (LJ parameters and mass) */
} md_topology;

typedef struct {
  int32_t n_replicas;          /* independent systems stepped together (>= 1) */
  int32_t sites_per_chain;     /* NAOM (Table II), 4 .. 1022 (.. 1023 with a topology); < 2^20 chains in all */
  const int32_t *n_chains;     /* [n_replicas] */
  const double *box;           /* [n_replicas] cube side L, nm; L >= 3 (rc + skin) */
  const double *pos;           /* [3 * N] x,y,z per atom, original order (any image) */
  const double *vel;           /* [3 * N] nm/ps, original order */
  const double *T_target;      /* [n_replicas] thermostat targets (K); may be NULL for MD_NVE */
  md_params params;
  double dt;                   /* time step, ps */
  double rc;                   /* LJ cutoff, nm (pairs with r >= rc are left out, Sec. 3.2) */
  double skin;                 /* neighbour-list skin, nm; list radius rc + skin */
  double tau_t;                /* thermostat coupling time, ps */
  int32_t rebin_every;         /* steps between rebin + list builds (paper: 10) */
  int32_t precision;           /* MD_PLAIN_FP32 or MD_MIXED */
  int32_t thermostat;          /* MD_NVE; MD_VRESCALE (weak coupling, lambda =
                                  sqrt(1 + dt/tau (T0/T - 1)) from the previous step's T);
                                  or MD_NOSE_HOOVER, the paper's NVT ensemble (Leap-Frog with
                                  Nose-Hoover coupling, Sec. 2 and 3.4): per replica
                                  v_{k+1/2} = [v_{k-1/2}(1 - dt xi_k/2) + dt F/m]/(1 + dt xi_k/2),
                                  xi_{k+1} = xi_k + dt (T_{k+1/2} - T0)/Q, Q = tau^2 T0/(4 pi^2),
                                  T_{k+1/2} from v_{k+1/2} (3N - 3 dof), and the centre-of-mass
                                  velocity of v_{k+1/2} removed before the next step.  xi starts
                                  at 0 and persists across md_step and md_set_state calls. */
  int32_t nbr_capacity;        /* neighbour slots per atom; 0 = chosen from density */
  int32_t lj_block;            /* threads per block of the LJ kernel: 128, 256 or 384 (0 = 384 with
                                  3 x 3 regions, 256 with 2 x 2) */
  int32_t schedule;            /* MD_SCHED_GRID or MD_SCHED_PERSISTENT (see below) */
  int32_t lj_lanes;            /* lanes of the LJ kernel that share one 4-atom cluster's list:
                                  8, 16 or 32 (0 = 8) */
  int32_t lj_region;           /* cells per side (x and y) of the work unit of the list build and
                                  LJ kernels, 1 cell deep: 2 or 3 (0 = 3) */
  int32_t lj_pair_exact;       /* 1: every LJ pair force (Eq. 2) is converted once to fixed point
                                  and added to i and subtracted from j as the same integer, so the
                                  LJ forces obey Newton's third law bit for bit (their sum over
                                  all atoms is exactly zero); the pair loop does more work (about
                                  1.2x the LJ time of the default on a 1.5M-atom melt).  A pair
                                  force component of 2^17 kJ/mol/nm or more, or a non-finite one,
                                  is reported as MD_EOVERFLOW.
                                  0 (default): per-cluster FP32 sums converted once. */
  const md_topology *topology; /* NULL: linear chains; else the molecule type (sites_per_chain must
                                  equal topology->naom) */
  int32_t displacement;        /* MD_DISP_REBUILD (default) or MD_DISP_ERROR */
  void *cuda_stream;           /* cudaStream_t to run on; NULL = a stream the library creates */
  void *workspace;             /* optional DEVICE memory for all buffers (see md_workspace_size);
                                  NULL = the library allocates.  Must outlive the system. */
  size_t workspace_bytes;
} md_desc;

/* Per-replica energies of the current state (Eqs. 1-6). */
typedef struct {
  double lj;            /* truncated LJ, Eq. 2 */
  double lj_shifted;    /* same with each pair shifted by -E(rc) (continuous) */
  double bond, angle, dihedral;   /* Eqs. 4, 5, 6 */
  double kinetic;       /* 1/2 sum m v^2 */
  double temperature;   /* 2 KE / ((3N - 3) k_B) */
  double total;         /* lj_shifted + bond + angle + dihedral + kinetic */
  double virial[6];     /* sum r (x) f: xx, yy, zz, xy, xz, yz (kJ/mol) */
  double pressure;      /* (2 KE + tr virial) / (3 V), kJ/mol/nm^3 */
} md_energy_t;

/* Settings chosen by md_autotune. */
typedef struct {
  double skin;                 /* nm; sets the cell side (>= rc + skin) */
  int32_t rebin_every;
  int32_t lj_block;
  int32_t schedule;
  int32_t lj_lanes;
  int32_t lj_region;
  int32_t from_cache;          /* 1 if read from the cache file, 0 if measured now */
  double us_per_step;          /* measured time per MD step of the winner */
} md_tuning;

/* Autotuner: times short runs of candidate settings on the system the
 * descriptor describes -- region side and LJ block shape ((2, 128), (2, 256),
 * (3, 256), (3, 384) cells / threads) with schedule (grid, persistent),
 * lanes per cluster (8, 16, 32), then cell size via (skin, rebin_every) in
 * {(0.08, 6), (0.10, 10), (0.12, 12), (0.15, 16)} nm / steps -- and writes the
 * fastest into desc->skin, rebin_every, lj_block, schedule, lj_lanes and
 * lj_region.  Candidates that
 * raise a device flag (e.g. an atom moving more than skin/2 between rebins)
 * are rejected.  With cache_path != NULL the result is looked up in / appended
 * to that text file, keyed by GPU, precision, replica count and atom-count and
 * box-size buckets.  trial_cycles: rebin cycles timed per candidate (>= 1).
 * Allocates and frees its own trial systems; the caller's state is only
 * read.  out may be NULL. */
int md_autotune(md_desc *desc, int32_t trial_cycles, const char *cache_path, md_tuning *out);

/* Bytes of device memory md_create needs for this descriptor. */
int md_workspace_size(const md_desc *desc, size_t *bytes);

/* Validate, copy the initial state to the GPU, bin, build the neighbour list,
 * evaluate F(t0) and capture the per-cycle CUDA graph.  Sets *out.  This is
 * the "input initial conditions" step of the paper's MD procedure (Sec. 3,
 * Fig. 1): the topology and parameters go to the GPU once (Sec. 3.3, last
 * paragraph), after which the step loop needs no host copy; the first
 * binning and list build follow Sec. 3.1. */
int md_create(const md_desc *desc, md_system **out);

/* Advance n_steps time steps (velocity Verlet; Leap-Frog positions, Sec. 3.4).
 * The neighbour list is rebuilt at the start of every block of rebin_every
 * steps and of every call (the paper rebuilds it every 10 steps, Sec. 5),
 * and also before the force evaluation of any step in which an atom has
 * moved more than skin/2 since the last rebuild (a device-side check that
 * opens a conditional rebuild in the step graph; md_early_rebins counts
 * them), so every force comes from a list that holds all pairs within rc;
 * with MD_DISP_ERROR such a step is reported as MD_EUNSTABLE instead.
 * Synchronises and reports device flags. */
int md_step(md_system *sys, int64_t n_steps);

/* Same, without synchronising; flags are reported by the next md_sync. */
int md_step_async(md_system *sys, int64_t n_steps);

/* Wait for queued work and report device flags (then clear them). */
int md_sync(md_system *sys);

/* Total force on every atom at the current positions, F = -grad E with E of
 * Eq. 1 (LJ of Eq. 2 over the Sec. 3.1 pair set, bonded terms of Eqs. 4-6,
 * Sec. 3.2-3.3): the force the integrator of Sec. 3.4 uses.  [3 * N] doubles
 * (host or device pointer), original order, kJ/mol/nm.  Converted on the GPU
 * and copied in one DMA.  Synchronous. */
int md_forces(md_system *sys, double *f_out);

/* Energies of every replica at the current state, out[n_replicas]. */
int md_energy(md_system *sys, md_energy_t *out);

/* Re-bin the current positions and rebuild the neighbour list (Sec. 3.1). */
int md_rebin(md_system *sys);

/* Current state: the positions and velocities that the update of Sec. 3.4
 * advances, with positions wrapped into the periodic cube [0, L) that the
 * cells of Sec. 3.1 tile ([3 * N]), velocities ([3 * N]) and periodic image
 * counters ([3 * N], may be NULL); any output may be NULL; host or device
 * pointers (one DMA each, after an in-GPU transpose).  Unwrapped position =
 * pos + images * L.  Synchronous. */
int md_get_state(md_system *sys, double *pos, double *vel, int32_t *images);

/* Replace positions and velocities ([3 * N] each, original order, host or
 * device pointers, read before the call returns), reset the image counters,
 * re-bin and recompute the forces.  The arrays are copied to the GPU as they
 * are (one DMA each) and checked, wrapped and transposed there: a position
 * x is stored as x - L floor(x / L), and a result that rounds to L (a tiny
 * negative x) is stored as 0.  A non-finite value gives MD_EINVAL; the
 * system's state is then undefined until the next successful md_set_state. */
int md_set_state(md_system *sys, const double *pos, const double *vel);

/* Replace the force-field parameters and recompute the forces. */
int md_set_params(md_system *sys, const md_params *params);

/* Thermostat targets per replica ([n_replicas] kelvin). */
int md_set_temperature(md_system *sys, const double *T_target);

/* Structural observables of the current state (the quantities of Sec. 5,
 * Fig. 8), computed on the GPU with each chain made continuous by
 * minimum-image bond vectors: r_ee[3c..3c+2] = x_last - x_first of chain c
 * (nm), rg2[c] = mass-weighted squared radius of gyration (nm^2), and
 * trans_fraction[r] = fraction of backbone dihedrals of replica r with
 * |phi| > 120 deg (IUPAC, trans = 180).  Chains are numbered over all
 * replicas; host or device pointers, any may be NULL.  Synchronous. */
int md_observables(md_system *sys, double *r_ee, double *rg2, double *trans_fraction);

/* Radial distribution function of non-bonded site pairs (Sec. 5, the RDF
 * the paper compares with GROMACS): for every replica r, counts[r * n_bins +
 * k] = the number of pairs i < j, other than 1-2 and 1-3 neighbours of a
 * chain (Sec. 3.1), whose minimum-image distance lies in [edges[k],
 * edges[k + 1]) (the last bin closed).  edges: [n_bins + 1] increasing, host
 * pointer, edges[0] >= 0, edges[n_bins] = r_max at most the cell side (r_c +
 * skin or more) of every replica; 1 <= n_bins <= 16384.  The distances are
 * the FP64 definition (d = x_j - x_i, d -= L rint(d / L), r = sqrt(dx^2 +
 * dy^2 + dz^2), each operation rounded once, left to right) on the state's
 * positions, so the counts equal that definition's.  Re-bins the current
 * positions first.  counts: host or device pointer, int64.  Allocates and
 * frees two small device buffers.  Synchronous.  g(r) = counts / (n_pairs *
 * shell volume / L^3) with n_pairs = N (N - 1) / 2 - n_chains (2 S - 3). */
int md_rdf(md_system *sys, int32_t n_bins, const double *edges, int64_t *counts);

/* End-to-end vector autocorrelation (Sec. 5, Fig. 8), accumulated on the GPU
 * over samples: C_r(tau) = <R_c(t + tau) . R_c(t)> / <R_c(t) . R_c(t)>, the
 * means over the chains c of replica r and every time origin t of the
 * samples taken so far.  md_acf_reset(max_lag) starts over (0 <= max_lag <=
 * 100000; allocates a ring of max_lag + 1 samples of 3 * n_chains doubles
 * the first time, or when max_lag changes).  md_acf_sample adds the current
 * state's end-to-end vectors (chains made continuous by minimum-image
 * bonds, as md_observables) as the next sample (asynchronous); md_acf_push
 * adds a given sample r_ee[3 * n_chains] (host or device pointer) instead
 * (synchronous).  md_acf_read writes C[n_replicas * (max_lag + 1)] (NaN for
 * lags with no pair of samples yet) and the number of samples. */
int md_acf_reset(md_system *sys, int32_t max_lag);
int md_acf_sample(md_system *sys);
int md_acf_push(md_system *sys, const double *r_ee);
int md_acf_read(md_system *sys, double *C, int64_t *n_samples);

/* Binning study (Sec. 3.1, Tables IV and V): the paper's CBIN arm (positions
 * copied to the host, binned there, the binned data copied back) against
 * this library's on-GPU counting sort, on the system's current positions.
 * Each of `reps` rounds (1 .. 1000) runs the GPU arm (cell ids, histogram,
 * scans, scatter, per-cell order and sorted arrays; then the cluster list
 * build) and the host arm (position copy to pinned host memory, binning on
 * one host thread with the same FP64 cell formula and stable counting sort,
 * copy of cell_of, packed cell coordinates, cell_start, cluster starts and
 * the order back to the GPU, and the per-cell sorted arrays built from it).
 * ms[6] = mean per round of: GPU binning, GPU list build, host arm position
 * copy, host binning, binned-data copy with the sorted arrays, host arm
 * total (CUDA events; host binning by the host clock).  The host arm runs
 * last, so md_get_bins then returns its bins, which equal the GPU arm's
 * (tested against the FP64 oracle).  Allocates pinned host memory for the
 * call.  Synchronous. */
int md_bin_study(md_system *sys, int32_t reps, double *ms);

/* Number of rebuilds so far that the displacement check added (an atom
 * moved more than skin/2 between scheduled rebuilds); synchronous. */
int md_early_rebins(md_system *sys, int64_t *count);

/* Nose-Hoover friction xi (1/ps) of each replica, [n_replicas]; zeros for
 * the other thermostats.  Synchronous. */
int md_get_thermostat(md_system *sys, double *xi);

/* The cudaStream_t the system runs on (for events and ordering). */
void *md_stream(md_system *sys);

/* Sizes: n_atoms, n_cells, neighbour capacity, cells per side of replica 0. */
int md_info(md_system *sys, int64_t *n_atoms, int64_t *n_cells, int32_t *nbr_capacity, int32_t *cells_per_side);

/* Binning result of the last rebin (Sec. 3.1): cell_of[N] (original order),
 * cell_start[n_cells + 1] and perm[N] (sorted slot -> original atom), where
 * the cells of replica r follow those of replicas 0..r-1 and a replica's
 * cell index is (cz * M + cy) * M + cx.  Any output may be NULL. */
int md_get_bins(md_system *sys, int32_t *cell_of, int32_t *cell_start, int32_t *perm);

/* Neighbour list of the last rebin: count[N] and entries[cap * N], both by
 * ORIGINAL atom index; entries hold original neighbour indices (only the
 * first count[i] of row i are meaningful).  cap = md_info's nbr_capacity. */
int md_get_neighbors(md_system *sys, int32_t *count, int32_t *entries);

/* FP32 cell-unit coordinates the force kernels read, [3 * N] in original
 * order: u = x / h - (c + 1/2) for the atom's cell c at the last rebin
 * (Sec. 3.1 cells of side h = L / M), moved by whole boxes for atoms that
 * crossed a face since then.  For checking the position pipeline. */
int md_get_cell_units(md_system *sys, float *u);

/* Per-kernel GPU time recording.  When enabled, CUDA events bracket every
 * kernel group of each step (rebin, neighbour build, integrate, LJ, bonded)
 * and md_step / md_sync accumulate their durations.  ms_total[5] and
 * launches[5] are in that order; md_profile_reset clears them. */
int md_profile_enable(md_system *sys, int32_t on);
int md_profile_read(md_system *sys, double *ms_total, int64_t *launches);
int md_profile_reset(md_system *sys);

/* Kernel launches per call of md_step(n_steps) (all library kernels and
 * memsets; an early rebuild adds six more). */
int64_t md_launches_per_call(md_system *sys, int64_t n_steps);

/* Cell binning of one periodic box into caller-provided DEVICE arrays, with
 * no device allocation.  (The paper has no counterpart: this exists for
 * callers that may not allocate GPU memory themselves -- code running while
 * another component owns all device memory, such as a framework's caching
 * allocator or a fixed-budget real-time loop, where an extra cudaMalloc
 * would fragment memory, stall on a device-wide synchronisation or exceed
 * the budget.)
 *   pos        [3 * n_atoms] FP64 positions, SoA (all x, then all y, then z)
 *   box        cube side L; cells_per_side = M; cell side L / M
 *   cell_of    [n_atoms] out: cell index (cz * M + cy) * M + cx of each atom
 *   cell_start [M^3 + 1] out: first sorted slot of each cell, last = n_atoms
 *   perm       [n_atoms] out: sorted slot -> atom index, atoms of a cell in
 *              ascending index order
 *   cuda_stream the stream to run on (NULL = legacy default stream)
 * The same formulas as md_rebin, so the outputs equal md_get_bins for the
 * same positions and M.  Limits: n_atoms <= 1,048,576 and M^3 <= 131,072;
 * larger sizes return MD_EINVAL and run nothing.  Cost: the order inside a
 * cell of m atoms takes O(m log m) work (runs of 256 ordered in shared
 * memory, then merge passes), whatever the positions; the worst legal call
 * (all 2^20 atoms in one cell) runs 4,096 runs on one block and 12 merge
 * passes over the atoms, a few milliseconds.  Scratch memory is one fixed
 * array of 13.1 MB per device inside this library, present on every device
 * that loads it until the process exits; every call shares it and it keeps
 * the last call's contents (the counters are cleared by each call), so calls
 * whose work overlaps on the GPU (other streams, other host threads) race.
 * Every call looks up the array's device address on the current device (so
 * a reset context is followed); the first call on a device also loads it,
 * so make that first call before any stream capture.  Asynchronous: results are
 * ready when the stream reaches them; errors are returned as MD_E* codes
 * with md_last_error(NULL). */
int md_bin_static(const double *pos, int32_t n_atoms, double box, int32_t cells_per_side, int32_t *cell_of,
                  int32_t *cell_start, int32_t *perm, void *cuda_stream);

/* Self-test of the bounded device wait, the pattern any device wait of this
 * library follows (no hot-path kernel waits on another block or launch
 * today): one block waits on an mbarrier that nothing arrives on, gives up
 * after `spins` try_wait rounds (1 .. 100000), raises its timeout flag and
 * returns.  Returns MD_ETIMEOUT when the wait gave up
 * (the expected result), MD_OK if it did not, another MD_E* code on a
 * failure.  Allocates and frees a 4-byte device flag; synchronous. */
int md_wait_selftest(int32_t spins);

void md_destroy(md_system *sys);

/* ------------------------------------------------------------------------
 * Adjoint: gradients of trajectory means with respect to the force-field
 * parameters theta = (eps_C32, eps_C33, sigma_C32, sigma_C33, k_phi)
 * (Table I, Eqs. 2 and 6).
 *
 * One melt of n_chains linear chains (atom = chain * sites + site, both ends
 * C_33), run in FP64 on the GPU with NVE velocity Verlet (Sec. 3.4) for
 * n_steps.  The pair set at every step is all non-excluded pairs (1-2 and 1-3
 * neighbours left out, Sec. 3.1) with minimum-image r < rc, from cells of
 * side >= rc rebuilt every step.  The observables are
 *   J_U = 1/(K+1) sum_{k=0..K} U(x_k),  U = shifted LJ + bond + angle + dihedral
 *   J_R = 1/(K+1) sum_{k=0..K} mean over chains |x_last - x_first|^2
 * (the end-to-end vector of Sec. 4, Fig. 8) with x unwrapped.  The gradient
 * is that of the discrete trajectory: the reverse pass steps the adjoint of
 * velocity Verlet newest step first, with Hessian-vector products of the LJ,
 * bond, angle and dihedral terms and the parameter derivatives of the forces,
 * recomputing positions from (x, v) checkpoints taken every checkpoint_every
 * steps.  Pairs crossing rc are invisible to it (the truncated force jumps
 * there by F(rc)).
 * Device memory: about 8 * 3N * (2 * ceil(K / C) + C + 8) bytes, allocated
 * by md_adj_create.  Errors: MD_E* codes with md_last_error(NULL).
 * ------------------------------------------------------------------------ */
typedef struct md_adj md_adj;          /* opaque, owned by the library */

typedef struct {
  int32_t n_chains;            /* >= 1 */
  int32_t sites_per_chain;     /* 2 .. 4096 */
  double box;                  /* cube side L, nm */
  md_params params;            /* theta is read from eps, sigma and kphi */
  double rc;                   /* LJ cutoff, nm */
  double dt;                   /* ps */
  int32_t n_steps;             /* K, 0 .. 1e7 */
  int32_t checkpoint_every;    /* C >= 1 */
  int32_t lj_form;             /* 0: Eq. 2 truncated at rc (the paper's potential);
                                  1: force-shifted E(r) - E(rc) - (r - rc) E'(rc), a
                                     variant outside the paper whose force is continuous
                                     at rc (for gradient checks) */
  int32_t hvp_precision;       /* 0: Hessian-vector products and parameter terms of the reverse
                                  pass in FP64 dual numbers; 1: in FP32 dual numbers (pair set,
                                  separations, records, reductions and the forward run stay
                                  FP64).  Affects md_adj_backward and md_adj_tangent. */
  void *cuda_stream;           /* NULL = a stream the library creates */
} md_adj_desc;

int md_adj_create(const md_adj_desc *desc, md_adj **out);

/* Replace theta (eps and sigma positive); invalidates the last forward run. */
int md_adj_set_theta(md_adj *adj, const double theta[5]);

/* Forward run from pos, vel ([3N] x,y,z per atom, host or device pointers,
 * copied): stores the checkpoints and writes obs = (J_U, J_R).  Positions may
 * be wrapped into the box or already continuous: the library first makes
 * every chain continuous on the GPU (site k moved by whole box lengths so
 * that each bond is its minimum image; a site that needs no move keeps its
 * bits), since J_R needs unwrapped chains.  Synchronous. */
int md_adj_forward(md_adj *adj, const double *pos, const double *vel, double obs[2]);

/* d(w0 J_U + w1 J_R)/dtheta of the last forward run at the current theta.
 * Synchronous. */
int md_adj_backward(md_adj *adj, const double weight[2], double grad[5]);

/* One evaluation at pos along direction dir ([3N] each): grad_u = dU/dx,
 * hvp = H dir (H the Hessian of U), dtheta[0..4] = dU/dtheta and
 * dtheta[5..9] = d(dU/dx . dir)/dtheta.  grad_u, hvp or dtheta may be NULL.
 * Synchronous; does not disturb the checkpoints of the last forward run. */
int md_adj_tangent(md_adj *adj, const double *pos, const double *dir, double *grad_u, double *hvp,
                   double dtheta[10]);

/* Totals of the last evaluation: out = (shifted LJ, bond, angle, dihedral,
 * sum over chains of R_ee^2, U).  Synchronous. */
int md_adj_energy(md_adj *adj, double out[6]);

void md_adj_destroy(md_adj *adj);

/* Message of the last failure on this system (or of the last failed
 * md_create when sys is NULL).  Valid until the next call. */
const char *md_last_error(const md_system *sys);

#ifdef __cplusplus
}
#endif

#endif /* MD_GB300_H */
