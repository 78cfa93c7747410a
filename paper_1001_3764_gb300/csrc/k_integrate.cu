// k_integrate.cu -- velocity-Verlet update (Sec. 3.4), kinetic energy and
// weak-coupling thermostat, energy reductions.
//
// Velocity Verlet gives the positions of the paper's Leap-Frog scheme.  A
// step is split as: [complete the previous step's second half-kick, kinetic
// energy, thermostat scale] + [first half-kick, drift] in one kernel (mode
// KKD); a call's first step skips the completion (KD) and its last step is
// closed by a kick-only pass (K), so the state at every API boundary is
// (x(t), v(t), F(t)).
//
// The paper's Nose-Hoover coupling needs the whole-system kinetic energy,
// which it sums through a per-atom array and a tree reduction (Sec. 3.4).
// Here each block writes one FP64 partial; the last block to finish (ticket
// counter, no waiting) sums the partials of each replica in a fixed order
// (one warp per replica and summed value, see below) and computes that
// replica's rescaling factor.
// The factor computed at step k is applied at step k+1 (one-step lag).
//
// Nose-Hoover (TH = 2; the paper's NVT ensemble with Leap-Frog, Sec. 2 and
// 3.4): per replica, lam[6r..6r+5] = (xi_k, 1 - c_k, 1/(1 + c_k), V_com),
// c_k = dt xi_k / 2.  A step closes v_k = (v_{k-1/2} - V_com + dt F/(2m)) /
// (1 + c_k), opens v_{k+1/2} = (1 - c_k) v_k + dt F/(2m) and drifts; the
// last block takes T_{k+1/2} and the momentum of v_{k+1/2} and leaves
// xi_{k+1} = xi_k + dt (T_{k+1/2} - T0)/Q, Q = tau^2 T0/(4 pi^2), and the
// centre-of-mass velocity that the next step subtracts.  This is the
// leap-frog update v_{k+1/2} = [v_{k-1/2}(1 - c_k) + dt F/m]/(1 + c_k).
//
// The drift also refreshes the FP32 cell-unit positions in sorted order for
// the force kernels, wraps positions into [0, L) with image counters, and
// flags atoms that moved more than skin/2 since the last rebin.
#include <type_traits>

#include "md_kernels.cuh"

namespace mdg {

__device__ __forceinline__ double warp_sum_i(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kIntBlock = 256;

__device__ __forceinline__ bool past_box(double x, double L) { return __double_as_longlong(x) >= __double_as_longlong(L); }
__device__ __forceinline__ bool past_box(float x, float L) { return __float_as_int(x) >= __float_as_int(L); }
__device__ __forceinline__ bool negative(double x) { return __double_as_longlong(x) < 0; }
__device__ __forceinline__ bool negative(float x) { return __float_as_int(x) < 0; }

template <bool MIXED, int MODE, bool KE, int TH>
__global__ void __launch_bounds__(kIntBlock) k_integrate(void* __restrict__ xv, void* __restrict__ vv,
                                                         int* __restrict__ img, const void* __restrict__ Fv,
                                                         const uint16_t* __restrict__ site,
                                                         const int* __restrict__ cellc,
                                                         const int* __restrict__ inv_perm,
                                                         const float4* __restrict__ ref, float4* __restrict__ pos,
                                                         int N, const Tile* __restrict__ tiles,
                                                         const RepDev* __restrict__ reps, int n_reps,
                                                         const ForceParams fp, double* __restrict__ kepart,
                                                         unsigned* __restrict__ done, double* __restrict__ ke_out,
                                                         double* __restrict__ lam, double tau,
                                                         unsigned* __restrict__ flags) {
  using T = typename std::conditional<MIXED, double, float>::type;
  T* x = reinterpret_cast<T*>(xv);
  T* v = reinterpret_cast<T*>(vv);
  const Tile t = tiles[blockIdx.x];
  const RepDev& R = reps[t.rep];
  const int i = t.start + threadIdx.x;
  double ke = 0.0;
  double mom[3] = {0.0, 0.0, 0.0};   // Nose-Hoover: momentum of v_{k+1/2}
  if ((int)threadIdx.x < t.len) {
    const int sm = site[i];
    const int type = atom_type(sm, fp);
    // mixed form: F stays in fixed-point units (int64 -> FP64 is a fast
    // conversion) and 2^-32 is folded into dt / 2m
    T hdt_m;
    if constexpr (MIXED) hdt_m = fp.hdt_m_fix[type]; else hdt_m = fp.hdt_m_f[type];
    T F[3] = {(T)0, (T)0, (T)0};
    if (MODE == kKineticOnly) {
    } else if (MIXED) {
      const F4i f = reinterpret_cast<const F4i*>(Fv)[i];
      F[0] = fix_to_double_i(f.x); F[1] = fix_to_double_i(f.y); F[2] = fix_to_double_i(f.z);   // integer pipe
    } else {
      const float4 f = reinterpret_cast<const float4*>(Fv)[i];
      F[0] = f.x; F[1] = f.y; F[2] = f.z;
    }
    T vi[3] = {v[i], v[N + i], v[2 * N + i]};
    // Without a kinetic-energy read-out the two half kicks of KKD are one
    // kick of dt F/m (the full-step velocity is never needed in between).
    constexpr bool kMerged = MODE == kKickKickDrift && !KE;
    if ((MODE == kKickKickDrift && KE) || MODE == kKickOnly) {
      if constexpr (TH == 2) {
        const double* nh = lam + 6 * t.rep;
        const T fc = (T)nh[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) vi[a] = (vi[a] - (T)nh[3 + a] + hdt_m * F[a]) * fc;   // v_k
      } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) vi[a] += hdt_m * F[a];   // v(t): close the previous step
      }
    }
    if (KE && TH != 2) {
      const double m = fp.mass[type];
      ke = 0.5 * m * ((double)vi[0] * vi[0] + (double)vi[1] * vi[1] + (double)vi[2] * vi[2]);
    }
    if (MODE == kKickOnly) {
      v[i] = vi[0]; v[N + i] = vi[1]; v[2 * N + i] = vi[2];
    } else if (MODE == kKickDrift || MODE == kKickKickDrift) {
      if (TH == 1) {
        const T l = (T)lam[t.rep];
#pragma unroll
        for (int a = 0; a < 3; ++a) vi[a] *= l;
      }
      T dt, L;
      if constexpr (MIXED) { dt = fp.dt; L = R.L; } else { dt = fp.dt_f; L = R.Lf; }
      const int cc = cellc[i];
      const float4 r0 = ref[i];
      const float r0a[3] = {r0.x, r0.y, r0.z};
      const float halfM = 0.5f * R.Mf;
      float loc[3], d2 = 0.f;
      bool bad = false;
      T fo = (T)1;
      if constexpr (TH == 2) fo = (T)lam[6 * t.rep + 1];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if constexpr (TH == 2) vi[a] = vi[a] * fo + hdt_m * F[a];   // v_{k+1/2}
        else vi[a] = kMerged ? vi[a] + (hdt_m + hdt_m) * F[a] : vi[a] + hdt_m * F[a];
        T xa = x[a * N + i] + dt * vi[a];
        // wrap into [0, L): for non-negative IEEE numbers the bit patterns
        // order like the values, so the tests run on the integer pipe
        if (past_box(xa, L)) { xa -= L; img[a * N + i] += 1; }
        else if (negative(xa)) { xa += L; img[a * N + i] -= 1; if (past_box(xa, L)) xa = (T)0; }
        x[a * N + i] = xa;
        v[a * N + i] = vi[a];
        // cell units in the frame of the rebin cell; an atom that crossed a
        // face since the rebin is moved back by one box (M cell units)
        const int c = (cc >> (10 * a)) & 1023;
        float ua;
        if constexpr (MIXED) ua = cell_unit_t(xa, c, R); else ua = cell_unit(xa, c, 0, R);
        const float du = ua - r0a[a];
        if (du > halfM || du < -halfM) {
          if constexpr (MIXED) ua = cell_unit_tw(xa, c, du > halfM ? -1 : 1, R);
          else ua = cell_unit(xa, c, du > halfM ? -1 : 1, R);
        }
        loc[a] = ua;
        const float d = ua - r0a[a];
        d2 += d * d;
        bad |= !isfinite(ua);          // a non-finite x or v reaches u
      }
      if (d2 > R.hs2u) atomicOr(flags, kFlagDisplacement);
      if (bad) atomicOr(flags, kFlagNaN);
      if constexpr (TH == 2) {
        const double m = fp.mass[type];
        ke = 0.5 * m * ((double)vi[0] * vi[0] + (double)vi[1] * vi[1] + (double)vi[2] * vi[2]);
#pragma unroll
        for (int a = 0; a < 3; ++a) mom[a] = m * (double)vi[a];
      }
      pos[inv_perm[i]] = make_float4(loc[0], loc[1], loc[2], (float)type);   // w: LJ type, as the sort writes it
    }
  }
  if (KE) {
    // block sums in FP64 through shared memory: thread q < 8 NV adds the 32
    // values of warp q % 8 in order, thread 0 the 8 warp sums in order (a
    // fixed order; 255 FP64 adds per value and block, where a shuffle tree
    // per warp would issue five on every lane: this GPU's FP64 pipe is narrow)
    constexpr int NV = TH == 2 ? 4 : 1;
    constexpr int NW = kIntBlock / 32;
    __shared__ double vals[NV][kIntBlock];
    __shared__ double wsum[NV][NW];
    __shared__ bool last;
    vals[0][threadIdx.x] = ke;
    if constexpr (TH == 2) {
#pragma unroll
      for (int a = 0; a < 3; ++a) vals[1 + a][threadIdx.x] = mom[a];
    }
    __syncthreads();
    if (threadIdx.x < NV * NW) {
      const int a = threadIdx.x / NW, w = threadIdx.x % NW;
      double b = 0.0;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) b += vals[a][32 * w + k];
      wsum[a][w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = 0.0;
      for (int q = 0; q < NW; ++q) b += wsum[0][q];
      kepart[blockIdx.x] = b;
      if constexpr (TH == 2) {
        for (int a = 0; a < 3; ++a) {
          double bm = 0.0;
          for (int q = 0; q < NW; ++q) bm += wsum[1 + a][q];
          kepart[gridDim.x + 3 * blockIdx.x + a] = bm;   // momentum partials follow the energy partials
        }
      }
      __threadfence();
      last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    if (last) {
      __threadfence();
      // a warp per (replica, value): lane l keeps eight chains P_m (m = 0..7), P_m
      // adding the replica's partials l + 32 m, l + 32 m + 256, ... in order
      // (eight loads in flight); then each P_m is summed over the lanes by a
      // fixed tree and the eight results in m order.  The order depends only
      // on the replica's own tile count.
      auto replica_sum = [&](const double* base, int stride, int n) {
        double P[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int k0 = 0; k0 < n; k0 += 256) {
#pragma unroll
          for (int m = 0; m < 8; ++m) {
            const int q = k0 + lane + 32 * m;
            if (q < n) P[m] += __ldcg(base + (size_t)q * stride);
          }
        }
        double sum = 0.0;
#pragma unroll
        for (int m = 0; m < 8; ++m) sum += warp_sum_i(P[m]);
        return sum;
      };
      // (replica, value) jobs over the warps: 8 replicas per round for the
      // kinetic energy alone, 2 for energy and momentum; then one thread per
      // replica forms its thermostat factors
      constexpr int RPR = NW / NV;
      __shared__ double res[RPR][NV];
      const int w = threadIdx.x >> 5;
      for (int r0 = 0; r0 < n_reps; r0 += RPR) {
        const int r = r0 + w / NV, a = w % NV;
        if (r < n_reps) {
          const RepDev& Q = reps[r];
          const double sum = a == 0 ? replica_sum(kepart + Q.tile_off, 1, Q.n_tiles)
                                    : replica_sum(kepart + gridDim.x + 3 * Q.tile_off + (a - 1), 3, Q.n_tiles);
          if (lane == 0) res[w / NV][a] = sum;
        }
        __syncthreads();
        if ((int)threadIdx.x < RPR && r0 + (int)threadIdx.x < n_reps) {
          const int rr = r0 + threadIdx.x;
          const RepDev& Q = reps[rr];
          const double sum = res[threadIdx.x][0];
          ke_out[rr] = sum;
          if (TH == 1) {
            const double T_inst = 2.0 * sum / (Q.dof * 0.0083144626);
            lam[rr] = sqrt(1.0 + fp.dt / tau * (Q.T0 / T_inst - 1.0));
          }
          if constexpr (TH == 2) {
            const double T_half = 2.0 * sum / (Q.dof * 0.0083144626);
            const double Qm = tau * tau * Q.T0 / (4.0 * 3.14159265358979323846 * 3.14159265358979323846);
            double* nh = lam + 6 * rr;
            const double xi = nh[0] + fp.dt * (T_half - Q.T0) / Qm;
            const double c = 0.5 * fp.dt * xi;
            const double M = (double)Q.n_chains * fp.mol_mass;
            nh[0] = xi; nh[1] = 1.0 - c; nh[2] = 1.0 / (1.0 + c);
            nh[3] = res[threadIdx.x][1] / M; nh[4] = res[threadIdx.x][2] / M; nh[5] = res[threadIdx.x][3] / M;
          }
        }
        __syncthreads();
      }
      if (threadIdx.x == 0) *done = 0u;
    }
  }
}

template <bool MIXED>
static void launch_int_t(IntegMode mode, bool ke, int th, void* x, void* v, int* img, const void* F,
                         const uint16_t* site, const int* cellc, const int* inv_perm, const float4* ref, float4* pos,
                         int N, const Tile* tiles, int n_tiles, const RepDev* reps, int n_reps,
                         const ForceParams& fp, double* kepart, unsigned* done, double* ke_out, double* lam,
                         double tau, unsigned* flags, cudaStream_t st) {
#define MDG_INT(MODE, KE, TH)                                                                                   \
  k_integrate<MIXED, MODE, KE, TH><<<n_tiles, kIntBlock, 0, st>>>(x, v, img, F, site, cellc, inv_perm, ref,     \
                                                                  pos, N, tiles, reps, n_reps, fp, kepart, done, \
                                                                  ke_out, lam, tau, flags)
  // With the weak-coupling thermostat (th = 1), every step that starts (KD,
  // KKD) takes the temperature of the unscaled v(t_k), scales v(t_k) by the
  // factor of the previous step and leaves the factor of step k for the next
  // one.  With Nose-Hoover (th = 2) every KD and KKD sums the kinetic energy
  // and momentum of v_{k+1/2} for xi_{k+1} and the centre-of-mass velocity.
  // The closing kick (K) only completes v; the next call's KD picks up from
  // there.
  if (mode == kKickDrift) {
    if (th == 2) MDG_INT(kKickDrift, true, 2);
    else if (th == 1) MDG_INT(kKickDrift, true, 1);
    else MDG_INT(kKickDrift, false, 0);
  } else if (mode == kKickKickDrift) {
    if (th == 2) MDG_INT(kKickKickDrift, true, 2);
    else if (th == 1) MDG_INT(kKickKickDrift, true, 1);
    else if (ke) MDG_INT(kKickKickDrift, true, 0);
    else MDG_INT(kKickKickDrift, false, 0);
  } else if (mode == kKickOnly) {
    if (th == 2) MDG_INT(kKickOnly, false, 2);
    else if (ke) MDG_INT(kKickOnly, true, 0);
    else MDG_INT(kKickOnly, false, 0);
  } else {
    MDG_INT(kKineticOnly, true, 0);
  }
#undef MDG_INT
}

void launch_integrate(bool mixed, IntegMode mode, bool ke, int thermostat, void* x, void* v, int* img,
                      const void* F, const uint16_t* site, const int* cellc, const int* inv_perm, const float4* ref,
                      float4* pos, int N, const Tile* tiles, int n_tiles, const RepDev* reps, int n_reps,
                      const ForceParams& fp, double* kepart, unsigned* done, double* ke_out, double* lam,
                      double tau, unsigned* flags, cudaStream_t st) {
  if (mixed)
    launch_int_t<true>(mode, ke, thermostat, x, v, img, F, site, cellc, inv_perm, ref, pos, N, tiles, n_tiles, reps,
                       n_reps, fp, kepart, done, ke_out, lam, tau, flags, st);
  else
    launch_int_t<false>(mode, ke, thermostat, x, v, img, F, site, cellc, inv_perm, ref, pos, N, tiles, n_tiles, reps,
                        n_reps, fp, kepart, done, ke_out, lam, tau, flags, st);
}

// ---------------------------------------------------------------- early rebin
// After a drift: if an atom has moved more than skin/2 since the rebin (the
// integrator raised kFlagDisplacement), open the conditional rebin that
// follows in the step graph, clear the flag (the new bins reset the
// reference) and count the event; else keep it closed.  One thread, so the
// condition is set once.
__global__ void __launch_bounds__(32) k_disp_check(cudaGraphConditionalHandle h, unsigned* __restrict__ flags,
                                                   unsigned long long* __restrict__ events) {
  if (threadIdx.x != 0) return;
  const unsigned f = *(volatile unsigned*)flags;
  const bool moved = (f & kFlagDisplacement) != 0u;
  if (moved) {
    atomicAnd(flags, ~kFlagDisplacement);
    *events += 1ull;
  }
  cudaGraphSetConditional(h, moved ? 1u : 0u);
}

void launch_disp_check(cudaGraphConditionalHandle h, unsigned* flags, unsigned long long* events, cudaStream_t st) {
  k_disp_check<<<1, 32, 0, st>>>(h, flags, events);
}

// ---------------------------------------------------------------- energy reduction
// LJ partials are per cell (replica r owns cells [cell_base, cell_base + M^3)),
// bonded partials per integrator tile.  Fixed summation order.
// out[r*16 + k]: k = 0 lj, 1 lj_shifted, 2 bond, 3 angle, 4 dihedral, 5..10 virial
// Two passes, spread over the GPU (FP64 adds are slow on one SM):
//  1. slice j of replica r covers its cells [j*1024, (j+1)*1024) and the same
//     share of its bonded tiles; thread t adds every 256th entry in order,
//     then a fixed tree over the block (warp shuffles, then the warps in
//     order) gives the slice's 11 sums;
//  2. one warp per replica adds its slices in slice order.
// The slices of a replica depend only on its own size, so a replica gets the
// same bits alone or batched with others.
constexpr int kRedThreads = 256;

__host__ __device__ inline int energy_slices(int n_cells) { return (n_cells + kEnergySliceCells - 1) / kEnergySliceCells; }

__global__ void __launch_bounds__(kRedThreads) k_energy_slices(const double* __restrict__ lj_part,
                                                               const double* __restrict__ b_part,
                                                               const RepDev* __restrict__ reps, int max_slices,
                                                               double* __restrict__ slices) {
  __shared__ double sh[11][kRedThreads / 32];
  const int r = blockIdx.x / max_slices, j = blockIdx.x % max_slices;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const RepDev& R = reps[r];
  const int nc = R.M * R.M * R.M, ns = energy_slices(nc);
  if (j >= ns) return;
  const int lt = (R.n_tiles + ns - 1) / ns;
  double acc[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  const int c0 = R.cell_base + j * kEnergySliceCells, c1 = R.cell_base + min(nc, (j + 1) * kEnergySliceCells);
  for (int c = c0 + tid; c < c1; c += kRedThreads) {
    const double* p = lj_part + (size_t)c * 8;
    acc[0] += p[0]; acc[1] += p[1];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[5 + k] += p[2 + k];
  }
  const int q0 = R.tile_off + j * lt, q1 = R.tile_off + min(R.n_tiles, (j + 1) * lt);
  for (int q = q0 + tid; q < q1; q += kRedThreads) {
    const double* p = b_part + (size_t)q * 9;
    acc[2] += p[0]; acc[3] += p[1]; acc[4] += p[2];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[5 + k] += p[3 + k];
  }
#pragma unroll
  for (int k = 0; k < 11; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) sh[k][w] = v;
  }
  __syncthreads();
  if (tid < 11) {
    double v = 0.0;
    for (int q = 0; q < kRedThreads / 32; ++q) v += sh[tid][q];
    slices[(size_t)blockIdx.x * 11 + tid] = v;
  }
}

__global__ void __launch_bounds__(32) k_energy_reduce(const double* __restrict__ slices, const RepDev* __restrict__ reps,
                                                      int max_slices, double* __restrict__ out) {
  const int r = blockIdx.x, k = threadIdx.x;
  if (k >= 11) return;
  const int ns = energy_slices(reps[r].M * reps[r].M * reps[r].M);
  double v = 0.0;
  for (int j = 0; j < ns; ++j) v += slices[((size_t)r * max_slices + j) * 11 + k];
  out[r * 16 + k] = v;
}

int energy_slice_count(int n_cells) { return energy_slices(n_cells); }

void launch_energy_reduce(const double* lj_part, const double* b_part, const RepDev* reps, int n_reps, int max_slices,
                          double* slices, double* out, cudaStream_t st) {
  if (n_reps <= 0) return;
  k_energy_slices<<<n_reps * max_slices, kRedThreads, 0, st>>>(lj_part, b_part, reps, max_slices, slices);
  k_energy_reduce<<<n_reps, 32, 0, st>>>(slices, reps, max_slices, out);
}

// ------------------------------------------------------------ chain observables
// One thread per chain (the structural observables of the paper's Sec. 5):
// the chain is made continuous by adding minimum-image bond vectors from site
// 0; R_ee = x_last - x_first (Fig. 8), R_g^2 = sum m |x - x_cm|^2 / sum m
// (mass-weighted, from sums relative to site 0), and the number of backbone
// dihedrals in the trans state, |phi| > 120 deg, i.e. cos(phi) =
// n1.n2 / (|n1||n2|) < -1/2 with n1 = b1 x b2, n2 = b2 x b3 (IUPAC, trans at
// 180 deg).  The trans counts of a replica are added as integers.
template <class T>
__global__ void __launch_bounds__(128) k_chain_observables(const T* __restrict__ x, int N,
                                                           const RepDev* __restrict__ reps, int n_reps,
                                                           const ForceParams fp, int n_chains_total,
                                                           double* __restrict__ ree, double* __restrict__ rg2,
                                                           unsigned long long* __restrict__ trans) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chains_total) return;
  int r = 0;
  while (r + 1 < n_reps && reps[r + 1].chain_off <= c) ++r;
  const RepDev& R = reps[r];
  const int S = fp.sites;
  const int o = R.atom_off + (c - R.chain_off) * S;
  const double L = R.L;
  double p[3] = {0.0, 0.0, 0.0};                       // site position relative to site 0
  double m_sum = 0.0, s1[3] = {0.0, 0.0, 0.0}, s2 = 0.0;
  double b[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};   // the last three bond vectors
  unsigned long long nt = 0;
  for (int k = 0; k < S; ++k) {
    if (k > 0) {
      double d[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double e = (double)x[a * N + o + k] - (double)x[a * N + o + k - 1];
        e -= L * rint(e / L);
        d[a] = e;
        p[a] += e;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) { b[0][a] = b[1][a]; b[1][a] = b[2][a]; b[2][a] = d[a]; }
      if (k >= 3) {
        const double n1[3] = {b[0][1] * b[1][2] - b[0][2] * b[1][1], b[0][2] * b[1][0] - b[0][0] * b[1][2],
                              b[0][0] * b[1][1] - b[0][1] * b[1][0]};
        const double n2[3] = {b[1][1] * b[2][2] - b[1][2] * b[2][1], b[1][2] * b[2][0] - b[1][0] * b[2][2],
                              b[1][0] * b[2][1] - b[1][1] * b[2][0]};
        const double dn = n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2];
        const double l1 = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
        const double l2 = n2[0] * n2[0] + n2[1] * n2[1] + n2[2] * n2[2];
        // cos(phi) < -1/2  <=>  n1.n2 < 0 and (n1.n2)^2 > |n1|^2 |n2|^2 / 4
        nt += (dn < 0.0 && 4.0 * dn * dn > l1 * l2) ? 1ull : 0ull;
      }
    }
    const double m = fp.mass[(k == 0 || k == S - 1) ? 1 : 0];
    m_sum += m;
#pragma unroll
    for (int a = 0; a < 3; ++a) s1[a] += m * p[a];
    s2 += m * (p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) ree[3 * c + a] = p[a];
  const double cx = s1[0] / m_sum, cy = s1[1] / m_sum, cz = s1[2] / m_sum;
  rg2[c] = s2 / m_sum - (cx * cx + cy * cy + cz * cz);
  atomicAdd(trans + r, nt);
}

void launch_chain_observables(bool mixed, const void* x, int N, const RepDev* reps, int n_reps,
                              const ForceParams& fp, int n_chains_total, double* ree, double* rg2,
                              unsigned long long* trans, cudaStream_t st) {
  const int blocks = (n_chains_total + 127) / 128;
  if (blocks == 0) return;
  if (mixed)
    k_chain_observables<double><<<blocks, 128, 0, st>>>((const double*)x, N, reps, n_reps, fp, n_chains_total,
                                                        ree, rg2, trans);
  else
    k_chain_observables<float><<<blocks, 128, 0, st>>>((const float*)x, N, reps, n_reps, fp, n_chains_total,
                                                       ree, rg2, trans);
}

// ------------------------------------------------------------------ output state
// SoA state -> AoS FP64 positions, velocities and image counters in the
// staging buffer (one DMA each to the caller afterwards).
template <bool MIXED>
__global__ void __launch_bounds__(256) k_egress_state(const void* __restrict__ xv, const void* __restrict__ vv,
                                                      const int* __restrict__ img, int N, double* __restrict__ pos,
                                                      double* __restrict__ vel, int* __restrict__ im) {
  using T = typename std::conditional<MIXED, double, float>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const T* x = reinterpret_cast<const T*>(xv);
  const T* v = reinterpret_cast<const T*>(vv);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    pos[3 * (size_t)i + a] = (double)x[a * N + i];
    vel[3 * (size_t)i + a] = (double)v[a * N + i];
    im[3 * (size_t)i + a] = img[a * N + i];
  }
}

// total force (int64 fixed point or FP32) -> AoS FP64 kJ/mol/nm
template <bool MIXED>
__global__ void __launch_bounds__(256) k_egress_forces(const void* __restrict__ Fv, int N, double scale,
                                                       double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  if constexpr (MIXED) {
    const F4i f = reinterpret_cast<const F4i*>(Fv)[i];
    out[3 * (size_t)i] = fix_to_double_i(f.x) * scale;
    out[3 * (size_t)i + 1] = fix_to_double_i(f.y) * scale;
    out[3 * (size_t)i + 2] = fix_to_double_i(f.z) * scale;
  } else {
    const float4 f = reinterpret_cast<const float4*>(Fv)[i];
    out[3 * (size_t)i] = f.x; out[3 * (size_t)i + 1] = f.y; out[3 * (size_t)i + 2] = f.z;
  }
}

void launch_egress_state(bool mixed, const void* x, const void* v, const int* img, int N, double* pos, double* vel,
                         int* im, cudaStream_t st) {
  if (N <= 0) return;
  if (mixed) k_egress_state<true><<<(N + 255) / 256, 256, 0, st>>>(x, v, img, N, pos, vel, im);
  else k_egress_state<false><<<(N + 255) / 256, 256, 0, st>>>(x, v, img, N, pos, vel, im);
}

void launch_egress_forces(bool mixed, const void* F, int N, double scale, double* out, cudaStream_t st) {
  if (N <= 0) return;
  if (mixed) k_egress_forces<true><<<(N + 255) / 256, 256, 0, st>>>(F, N, scale, out);
  else k_egress_forces<false><<<(N + 255) / 256, 256, 0, st>>>(F, N, scale, out);
}

// ------------------------------------------------------------------ input state
template <bool MIXED>
__global__ void __launch_bounds__(kIntBlock) k_ingest(const double* __restrict__ stage, int N,
                                                      const Tile* __restrict__ tiles, const RepDev* __restrict__ reps,
                                                      void* __restrict__ xv, void* __restrict__ vv,
                                                      int* __restrict__ img, unsigned* __restrict__ flags) {
  using T = typename std::conditional<MIXED, double, float>::type;
  const Tile t = tiles[blockIdx.x];
  if ((int)threadIdx.x >= t.len) return;
  const RepDev& R = reps[t.rep];
  const int i = t.start + threadIdx.x;
  T* x = reinterpret_cast<T*>(xv);
  T* v = reinterpret_cast<T*>(vv);
  bool bad = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double xa = stage[3 * (size_t)i + a];
    const double va = stage[3 * (size_t)N + 3 * (size_t)i + a];
    bad |= !isfinite(xa) || !isfinite(va);
    xa -= R.L * floor(xa / R.L);
    if (!(xa < R.L) || xa < 0.0) xa = 0.0;
    if (!MIXED && (float)xa >= R.Lf) xa = 0.0;
    x[a * N + i] = (T)xa;
    v[a * N + i] = (T)va;
    img[a * N + i] = 0;
  }
  if (bad) atomicOr(flags, kFlagBadInput);
}

void launch_ingest(bool mixed, const double* stage, int N, const Tile* tiles, int n_tiles, const RepDev* reps,
                   void* x, void* v, int* img, unsigned* flags, cudaStream_t st) {
  if (n_tiles <= 0) return;
  if (mixed) k_ingest<true><<<n_tiles, kIntBlock, 0, st>>>(stage, N, tiles, reps, x, v, img, flags);
  else k_ingest<false><<<n_tiles, kIntBlock, 0, st>>>(stage, N, tiles, reps, x, v, img, flags);
}

}  // namespace mdg
