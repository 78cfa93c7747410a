// md_kernels.cuh -- device-side data layout and kernel launchers of the GB300
// MD engine (united-atom polyethylene, Xu et al., Secs. 2-3).
//
// Layout in HBM (N atoms over all replicas, C cells over all replicas):
//   original (chain-major) order, index i:
//     mixed form : x, v  double SoA [3][N];   plain form : float SoA [3][N]
//     img        int32 SoA [3][N]  periodic image counters
//     F          force, AoS 32 B/atom: int64x3 fixed point (mixed) or float x3
//     site       uint16 [N] position of the atom in its chain (MAIDX - 1)
//     cellc      int32 [N] packed cell coordinates at the last rebin
//     ref        float4 [N] cell-unit position at the last rebin
//     inv_perm   int32 [N] sorted slot of atom i
//   sorted (cell-major) order, index s:
//     pos        float4 [N] position in cell units relative to the centre of the
//                atom's cell at the last rebin, u = (x - (c + 1/2) h) / h; w unused
//     tag        int32 [N]  chain*1024 + site | type << 30 (sites < 1024, so the
//                site fields of two chains never come within 2 of each other)
//     perm       int32 [N]  original index of slot s
//     Flj        int64 SoA [3][Npad]  LJ force on slot s (2^-32 kJ/mol/nm):
//                cleared, added to by the force kernel, read by the bonded
//                kernel
//   clusters (4 consecutive slots of a cell; cluster k of cell c is
//   cl_start[c] + k):
//     list       uint32 [clusters][cap]: tile index (bits 0..15) and the mask
//                of the cluster's atoms that pair with it (bits 16..19)
//     ncl        int32 [clusters] entries per cluster
//   cells: count int32 [C], cell_start int32 [C+1], cl_start int32 [C+1]
//   regions: up to 2 x 2 x 1 cells each, the force and list-build work units
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mdg {

constexpr int kMaxReplicas = 4096;
constexpr int kTagTypeBit = 30;
constexpr int kTagSiteBits = 10;                      // site in bits 0..9, chain in bits 10..29
constexpr uint32_t kTagMask = (1u << 30) - 1;
constexpr int kNbrIndexBits = 26;                     // j in entry bits 0..25
constexpr uint32_t kNbrIndexMask = (1u << kNbrIndexBits) - 1;
constexpr double kFixScale = 4294967296.0;            // 2^32 per kJ/mol/nm
constexpr double kFixInv = 1.0 / 4294967296.0;

// Error flags (bitmask in device memory)
enum : uint32_t {
  kFlagNbrOverflow = 1u,      // neighbour list capacity exceeded
  kFlagFixOverflow = 2u,      // a force part beyond 2^18 kJ/mol/nm (the fixed-point range)
  kFlagNaN = 4u,              // non-finite position or velocity
  kFlagDisplacement = 8u,     // an atom moved more than skin/2 since the rebin
  kFlagTimeout = 16u,         // a bounded device wait gave up
  kFlagBadInput = 32u,        // a non-finite input position or velocity (md_create / md_set_state)
};

struct RepDev {
  double L, h, inv_h, half_L;   // box, cell side, M/L, L/2
  float Lf, hf, half_Lf, Mf;    // FP32 copies; Mf = M (the box side in cell units)
  float ih_hi, ih_lo;           // 1/h split into two floats (ih_hi + ih_lo = 1/h to ~2^-48)
  float rc2u, rlist2u;          // (r_c / h)^2, ((r_c + skin) / h)^2
  float hs2u, pad1;             // (skin / 2 / h)^2
  // LJ constants in cell units, by type pair t_i + t_j (0: C_32-C_32,
  // 1: C_32-C_33, 2: C_33-C_33): C6u = c6 / h^6, C12u = c12 / h^12
  float C6u[3], C12u[3];
  float pad2[2];
  int M, cell_base, atom_off, n_atoms;
  int n_chains, chain_off, tile_off, n_tiles;
  double T0, dof;
};

struct Tile { int start, len, rep, pad; };

// Regions of up to 2 x 2 x 1 cells (the work unit of the list build and LJ
// kernels) and their tiles: the region's home cells, then the cells their
// 13 forward neighbours add, as offsets from the region's origin cell.
constexpr int kMaxTileCells = 64;   // 44 cells for a 3 x 3 x 1 region
constexpr int kMaxHome = 9;
struct RegionShape {
  int n_home, n_tile;
  signed char off[kMaxTileCells][3];      // tile cell offsets (x, y, z) from the origin cell
  unsigned char nb[kMaxHome][14];         // home cell h: its own tile cell, then its 13 forward cells
  float cx, cy, cz;                       // region centre relative to the origin cell's centre
};
struct Region { int rep, ox, oy, oz, shape, pad[3]; };

// Position of atom x (one axis) in cell units relative to the centre of cell
// c, shifted by w box lengths (w = +1/-1 for an atom that crossed a face
// since the rebin): u = x/h - (c + 1/2) + w M.
// FP64 master: one FMA in FP64, then one rounding to FP32.
__device__ __forceinline__ float cell_unit(double x, int c, int w, const RepDev& R) {
  const double k = (double)c + 0.5 - (double)w * (double)R.M;
  return __double2float_rn(fma(x, R.inv_h, -k));
}
// FP64 -> FP32 with round-to-nearest-even done on the integer pipe (FP64 <->
// FP32 conversions share the slow FP64 pipe on this GPU).  From the IEEE 754
// binary64/binary32 layouts, on the two 32-bit words of the double: for a
// normal result, keep the sign, the 11-bit exponent and the top 23 mantissa
// bits (the kept word, taken modulo 2^32), drop the low 29 mantissa bits with
// round-half-even (add 2^28 - 1 + the lowest kept bit; a carry moves into the
// exponent) and rebias the exponent by 1023 - 127 = 896.  Zero and magnitudes
// below 2^-126 give a signed zero (no subnormal results), magnitudes from
// 2^128 up give infinity, NaN stays NaN.  32-bit words rather than 64-bit
// integer arithmetic: fewer instructions on this GPU.
__device__ __forceinline__ float d2f_rn_int(double d) {
  const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
  const unsigned ha = hi & 0x7fffffffu, sign = hi & 0x80000000u;
  const unsigned kept = (ha << 3) | (lo >> 29);
  const unsigned inc = ((lo & 0x1fffffffu) + 0x0fffffffu + (kept & 1u)) >> 29;
  unsigned f = kept + inc - (896u << 23);
  f = ha < 0x38100000u ? 0u : f;                                          // below the normal range
  f = (ha > 0x47efffffu || (ha == 0x47efffffu && lo >= 0xf0000000u)) ? 0x7f800000u : f;   // overflow, inf
  f = (ha > 0x7ff00000u || (ha == 0x7ff00000u && lo != 0u)) ? 0x7fc00000u : f;            // NaN
  return __uint_as_float(f | sign);
}

// c + 1/2 as an FP64 number built from its bits (no int -> FP64 conversion):
// n = 2c + 1 is odd and below 2^12, c + 1/2 = n / 2 = 1.m * 2^(e-1), e = msb(n).
__device__ __forceinline__ double half_plus(int c) {
  const unsigned n = 2u * (unsigned)c + 1u;
  const int e = 31 - __clz(n);
  const unsigned long long m = ((unsigned long long)n << (52 - e)) & 0x000fffffffffffffull;
  return __longlong_as_double(((unsigned long long)(e + 1022) << 52) | m);
}

// k + 1/2 for any int k with |2k + 1| < 2^21 (cell indices shifted by a box,
// k = c - w M), from its bits like half_plus, with the sign bit.
__device__ __forceinline__ double half_plus_s(int k) {
  const int m = 2 * k + 1;
  const unsigned a = (unsigned)(m < 0 ? -m : m);
  const unsigned sgn = m < 0 ? 0x80000000u : 0u;
  const int e = 31 - __clz(a);
  const unsigned mh = (a << (20 - e)) & 0x000fffffu;
  return __hiloint2double((int)(sgn | ((unsigned)(e + 1022) << 20) | mh), 0);
}

// cell_unit(x, c, w, R) on the integer pipe: the centre offset c + 1/2 - w M
// built from bits and the FP32 rounding done with integer operations (same
// value).  Evaluating the conversions of cell_unit for every atom, as a
// compiler may do for a branch taken by few, would load the FP64 pipe.
__device__ __forceinline__ float cell_unit_tw(double x, int c, int w, const RepDev& R) {
  return d2f_rn_int(fma(x, R.inv_h, -half_plus_s(c - w * R.M)));
}

// Same as cell_unit with the centre offset built on the integer pipe and the
// final rounding on the integer pipe.
__device__ __forceinline__ float cell_unit_t(double x, int c, const RepDev& R) {
  return d2f_rn_int(fma(x, R.inv_h, -half_plus(c)));
}

// int64 -> FP64 on the integer pipe, exact for |n| < 2^53: the binary64
// fields are built directly (exponent from the leading-zero count, the
// mantissa by a left shift, no rounding needed).
__device__ __forceinline__ double fix_to_double_i(long long n) {
  const unsigned long long sgn = (unsigned long long)n & 0x8000000000000000ull;
  const unsigned long long a = n < 0 ? 0ull - (unsigned long long)n : (unsigned long long)n;
  const int e = 63 - __clzll((long long)a);                 // msb of a (a != 0)
  const unsigned long long m = (a << (52 - e)) & 0x000fffffffffffffull;
  const unsigned long long bits = sgn | ((unsigned long long)(e + 1023) << 52) | m;
  return a == 0ull ? 0.0 : __longlong_as_double((long long)bits);
}

// FP32 master: x/h as p + e (exact product error by FMA, plus the low part of
// 1/h), minus the exact integer-plus-half k; one final rounding.
__device__ __forceinline__ float cell_unit(float x, int c, int w, const RepDev& R) {
  const float k = (float)c + 0.5f - (float)w * R.Mf;
  const float p = x * R.ih_hi;
  const float e = fmaf(x, R.ih_hi, -p);
  return __fadd_rn(__fsub_rn(p, k), fmaf(x, R.ih_lo, e));
}

// round-half-even(f * 2^32) as int64 (the 2^-32 fixed point of the forces)
// on the integer pipe, from the binary32 fields: f * 2^32 = m * 2^s with m
// the 24-bit significand and s = e - 118; a left shift for s >= 0 (s <= 26
// for |f| < 2^18, the range the callers check), else a right shift by -s
// with round-half-even (nothing is left for -s >= 25).  Gives the bits of
// __float2ll_rn(f * 2^32) without the conversion instruction, which runs on
// the narrow FP64 pipe of this GPU.
__device__ __forceinline__ long long fix_round_int(float f) {
  const unsigned u = __float_as_uint(f);
  const int e = (int)((u >> 23) & 0xffu);
  const unsigned m = (u & 0x007fffffu) | (e ? 0x00800000u : 0u);
  const int s = e - 118;
  unsigned hi = 0u, lo;
  if (s >= 0) {
    hi = s ? m >> (32 - s) : 0u;
    lo = m << s;
  } else {
    const int r = -s;
    const unsigned q = r >= 25 ? 0u : m >> r;
    const unsigned rem = r >= 25 ? 0u : m & ((1u << r) - 1u), half = r >= 25 ? 1u : 1u << (r - 1);
    lo = q + ((rem > half || (rem == half && (q & 1u))) ? 1u : 0u);
  }
  const long long v = (long long)(((unsigned long long)hi << 32) | lo);
  return (u >> 31) ? -v : v;
}

// Per-system constants passed by value to kernels.
struct ForceParams {
  float c6[2][2], c12[2][2];      // 4 eps sigma^6, 4 eps sigma^12 (geometric mixing)
  float erc[2][2];                // pair energy at r_c (for the shifted energy)
  float rc2, rlist2;              // cutoff^2, list radius^2 (float)
  float kb, b0, ka, theta0;       // Eqs. (4), (5)
  float kphi, phis;               // Eq. (6)
  int n_mult;
  int sites;                      // atoms per chain (NAOM)
  float half_skin2;               // (skin/2)^2
  float b0sq_hi, b0sq_lo;         // b0^2 as a two-float sum
  double b0sq;                    // b0^2
  double mass[2], inv_mass[2];
  double dt;
  float hdt_m_f[2], dt_f;         // FP32 copies for the plain form
  float pad_f;
  double hdt_m[2];                // dt / (2 m) per type
  double hdt_m_fix[2];            // dt / (2 m) * 2^-32 (applied to int64 fixed-point forces)
  double mol_mass;                // mass of one molecule
  const unsigned char* mtype;     // type of each atom of the molecule (device), or null: linear
                                  // chains, whose ends (sites 0 and sites - 1) are C_33
};

// LJ / mass type of the atom at position st of its molecule
__device__ __forceinline__ int atom_type(int st, const ForceParams& fp) {
  return fp.mtype ? (int)fp.mtype[st] : ((st == 0 || st == fp.sites - 1) ? 1 : 0);
}

// The terms of a general molecule type (Sec. 3.3), in device memory, each
// term listed under its first atom (0-based index in the molecule):
// bonds (a, b), angles (a, b, c) with vertex b, dihedrals (a, b, c, d).
// Exclusions: each atom's 1-2 and 1-3 neighbours, ascending.
struct TopoDev {
  const int *b_off, *b_at;        // b_at[q] = b of bond q owned by a, q in [b_off[a], b_off[a+1])
  const int *a_off, *a_at;        // a_at[2q..2q+1] = (b, c)
  const int *d_off, *d_at;        // d_at[3q..3q+2] = (b, c, d)
  const int *x_off, *x_at;        // exclusions of a: x_at[x_off[a] .. x_off[a+1])
  int naom, pad;
};

struct F4i { long long x, y, z, w; };   // fixed-point force, 32 B

// ---------------------------------------------------------------- binning
void launch_bin_count(bool mixed, const void* x, int N, const Tile* tiles, int n_tiles,
                      const RepDev* reps, int* cell_of, int* cellc, int* count, int* slot,
                      cudaStream_t st);
void launch_scan(const int* count, int* cell_start, int C, cudaStream_t st);
// cell_start from count, and cl_start from ceil(count / 4) (clusters per cell)
void launch_scan2(const int* count, int* cell_start, int* cl_start, int C, cudaStream_t st);
// stable order by atom index inside each of C cells (n atoms in all):
// perm[cell_start[c] + rank] = atom, from the unsorted bucket contents in
// `runs` (overwritten), in O(m log m) work for a cell of m atoms.  Scratch:
// buf[n], pcell[n] and one int *maxm that the caller clears before the call.
void launch_static_order(const int* cell_start, int C, int n, int* runs, int* buf, int* pcell, int* perm, int* maxm,
                         cudaStream_t st);
void launch_bin_scatter(const int* cell_of, const int* slot, const int* cell_start, int* tmp, int N,
                        cudaStream_t st);
void launch_cell_sort(bool mixed, const void* x, int N, const int* cell_start, const int* tmp, const unsigned char* mtype,
                      const int* cellc, const uint16_t* site, const RepDev* reps, int n_reps, int C,
                      int sites, int* perm, int* inv_perm, float4* pos, int* tag, float4* ref, unsigned* flags,
                      cudaStream_t st);
// ---------------------------------------------------------------- forces
// cluster lists and LJ forces by regions (k_lj.cu).  The build writes each
// cluster's list (up to cap entries, ncl[cl] of them); the force kernel adds
// the LJ force of every atom into flj (int64 SoA [3][Npad], cleared by the
// caller before) and, with energy, the per-region energy and virial sums into
// epart (8 per cell).  persistent_grid > 0 runs that many blocks that take
// regions from work[0..1] (two ints, zero before the first launch).
// topo != null: exclusions of a general molecule type from its lists; else
// linear chains (1-2 and 1-3 neighbours by site index)
void launch_cl_build(const float4* pos, const int* tag, const int* cell_start, const int* cl_start,
                     const Region* regions, int n_regions, const RegionShape* shapes, const RepDev* reps,
                     unsigned* list, int* ncl, int cap, int tile_cap, unsigned* flags, int persistent_grid, int* work,
                     const TopoDev* topo, cudaStream_t st);
void launch_cl_force(bool energy, const float4* pos, const int* cell_start, const int* cl_start,
                     const Region* regions, int n_regions, const RegionShape* shapes, const RepDev* reps,
                     const unsigned* list, const int* ncl, int cap, int tile_cap, const ForceParams& fp,
                     long long* flj, int Npad, double* epart, unsigned* flags, int block, int lanes,
                     int persistent_grid, int* work, bool exact, cudaStream_t st);
int lj_blocks_per_sm(int block, int lanes, int tile_cap);
cudaError_t tile_kernels_init();
int tile_capacity_max();
// one block waits on an mbarrier nothing arrives on, `spins` rounds, then raises kFlagTimeout
void launch_wait_selftest(unsigned spins, unsigned* flags, cudaStream_t st);
// bonded forces plus the LJ force (read from flj[3][Npad] in sorted order)
// into F (original order); launch_bonded_generic does the same for a general
// molecule type (mixed form only): F = LJ, then every term adds its forces
// with integer atomics, energies per integrator tile
void launch_bonded_generic(bool energy, const double* x, const int* inv_perm, const long long* flj, int Npad, int N,
                           const Tile* tiles, int n_tiles, const RepDev* reps, const ForceParams& fp,
                           const TopoDev& topo, void* F, double* epart, unsigned* flags, cudaStream_t st);
void launch_bonded(bool mixed, bool energy, const void* x, const uint16_t* site, const int* inv_perm,
                   const long long* flj, int Npad, int N, const Tile* tiles, int n_tiles, const RepDev* reps,
                   const ForceParams& fp, void* F, double* epart, unsigned* flags, cudaStream_t st);

// ---------------------------------------------------------------- integration
enum IntegMode { kKickDrift = 0, kKickKickDrift = 1, kKickOnly = 2, kKineticOnly = 3 };
// Input state from a staging copy of the caller's arrays (x,y,z per atom:
// positions, then velocities): check, wrap into [0, L), write the SoA state
// and clear the image counters, on the integrator's tiles.
void launch_ingest(bool mixed, const double* stage, int N, const Tile* tiles, int n_tiles, const RepDev* reps,
                   void* x, void* v, int* img, unsigned* flags, cudaStream_t st);
// AoS FP64 copies of the state / total force in device memory (for one DMA to the caller)
void launch_egress_state(bool mixed, const void* x, const void* v, const int* img, int N, double* pos, double* vel,
                         int* im, cudaStream_t st);
void launch_egress_forces(bool mixed, const void* F, int N, double scale, double* out, cudaStream_t st);
// per chain: end-to-end vector ree[3c..3c+2], R_g^2 rg2[c]; per replica the
// number of trans dihedrals added into trans[r] (zeroed by the caller)
void launch_chain_observables(bool mixed, const void* x, int N, const RepDev* reps, int n_reps,
                              const ForceParams& fp, int n_chains_total, double* ree, double* rg2,
                              unsigned long long* trans, cudaStream_t st);
// thermostat: 0 none, 1 weak coupling, 2 Nose-Hoover
void launch_integrate(bool mixed, IntegMode mode, bool ke, int thermostat, void* x, void* v, int* img,
                      const void* F, const uint16_t* site, const int* cellc, const int* inv_perm,
                      const float4* ref, float4* pos, int N, const Tile* tiles, int n_tiles,
                      const RepDev* reps, int n_reps, const ForceParams& fp, double* kepart,
                      unsigned* done, double* ke_out, double* lam, double tau, unsigned* flags,
                      cudaStream_t st);
// RDF of non-bonded pairs (k_observe.cu): counts[r * n_bins + k] += pairs of
// replica r with edges[k] <= r < edges[k + 1] (last bin closed); norm =
// n_bins / (edges[n_bins] - edges[0]) gives the first guess of k
void launch_rdf(bool mixed, const void* x, int N, const int* cell_start, const int* perm, const RepDev* reps,
                int n_reps, int C, int sites, const double* edges, int n_bins, double norm,
                unsigned long long* counts, cudaStream_t st);
// ACF: add sample s (ring slot s % (max_lag + 1)) to acc[r][tau], tau <= min(s, max_lag)
void launch_acf_add(const double* ring, int n_chains_total, const RepDev* reps, int n_reps, long long s, int max_lag,
                    double* acc, cudaStream_t st);
// opens the conditional rebin of a step graph when kFlagDisplacement is set
// (then cleared and counted in *events)
void launch_disp_check(cudaGraphConditionalHandle h, unsigned* flags, unsigned long long* events, cudaStream_t st);
// cells per slice of the first energy-reduction pass
constexpr int kEnergySliceCells = 1024;
int energy_slice_count(int n_cells);
// slices: n_reps * max_slices * 11 doubles of scratch
void launch_energy_reduce(const double* lj_part, const double* b_part, const RepDev* reps, int n_reps, int max_slices,
                          double* slices, double* out, cudaStream_t st);

}  // namespace mdg
