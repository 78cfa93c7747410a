// k_observe.cu -- structural observables of Sec. 5 on the GPU: the radial
// distribution function of non-bonded site pairs and the end-to-end vector
// autocorrelation function (Fig. 8).
//
// RDF: one block per cell; its atoms pair with the later atoms of the cell and
// with every atom of the 13 forward cells of a half shell, so each pair within
// one cell side is met once.  The distance is the plain definition in FP64
// with every operation explicitly rounded (d = x_j - x_i, d -= L rint(d / L),
// r = sqrt(dx^2 + dy^2 + dz^2), summed left to right), and the bin is the k
// with edges[k] <= r < edges[k + 1] (the last bin closed), so the integer
// counts equal those of the FP64 definition on the same positions.  Counts
// are summed in shared memory and added to the per-replica histogram with
// integer atomics (order-free).
//
// ACF: samples of the chains' end-to-end vectors go to a ring of max_lag + 1
// slots; each new sample s adds, for every lag tau <= min(s, max_lag) and
// every replica, sum_c R_c(s) . R_c(s - tau) to acc[r][tau], one block per
// (replica, tau) with a fixed-order reduction over the replica's chains.
// After n samples acc[r][tau] = sum_{t < n - tau} sum_c R_c(t + tau) . R_c(t).
#include <type_traits>

#include "md_kernels.cuh"

namespace mdg {

constexpr int kRdfThreads = 128;

__device__ __forceinline__ int rdf_find_rep(const RepDev* reps, int n_reps, int c) {
  int lo = 0, hi = n_reps - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (reps[mid].cell_base <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class T>
__global__ void __launch_bounds__(kRdfThreads) k_rdf(const T* __restrict__ x, int N, const int* __restrict__ cell_start,
                                                     const int* __restrict__ perm, const RepDev* __restrict__ reps,
                                                     int n_reps, int sites, const double* __restrict__ edges,
                                                     int n_bins, double norm, unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned int hist[];
  const int c = blockIdx.x;
  for (int k = threadIdx.x; k < n_bins; k += blockDim.x) hist[k] = 0u;
  __syncthreads();
  const int r = rdf_find_rep(reps, n_reps, c);
  const RepDev& R = reps[r];
  const int M = R.M, lc = c - R.cell_base;
  const int cx = lc % M, cy = (lc / M) % M, cz = lc / (M * M);
  const int b = cell_start[c], n = cell_start[c + 1] - b;
  const double L = R.L, r_max = edges[n_bins];
  // the cell itself, then its 13 forward neighbours
  for (int o = 0; o < 14; ++o) {
    int ox = 0, oy = 0, oz = 0;
    if (o > 0) {
      const int q = o - 1;                  // 9 cells of the z + 1 layer, 3 of y + 1, then x + 1
      if (q < 9) { oz = 1; oy = q / 3 - 1; ox = q % 3 - 1; }
      else if (q < 12) { oy = 1; ox = q - 10; }
      else { ox = 1; }
    }
    const int nc = R.cell_base + (((cz + oz + M) % M) * M + ((cy + oy + M) % M)) * M + ((cx + ox + M) % M);
    const int jb = cell_start[nc], jn = cell_start[nc + 1] - jb;
    const long long pairs = (long long)n * jn;
    for (long long p = threadIdx.x; p < pairs; p += blockDim.x) {
      const int a = (int)(p / jn), q = (int)(p % jn);
      if (o == 0 && q <= a) continue;       // the cell itself: each pair once
      const int i = perm[b + a], j = perm[jb + q];
      const int ci = (i - R.atom_off) / sites, cj = (j - R.atom_off) / sites;
      const int si = (i - R.atom_off) - ci * sites, sj = (j - R.atom_off) - cj * sites;
      if (ci == cj && abs(si - sj) <= 2) continue;   // 1-2 and 1-3 neighbours (Sec. 3.1)
      double d2 = 0.0;
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        double d = __dsub_rn((double)x[ax * N + j], (double)x[ax * N + i]);
        d = __dsub_rn(d, __dmul_rn(L, rint(__ddiv_rn(d, L))));
        d2 = ax == 0 ? __dmul_rn(d, d) : __dadd_rn(d2, __dmul_rn(d, d));
      }
      const double rr = __dsqrt_rn(d2);
      if (!(rr <= r_max) || rr < edges[0]) continue;
      int k = (int)((rr - edges[0]) * norm);
      k = k < 0 ? 0 : (k > n_bins - 1 ? n_bins - 1 : k);
      if (rr < edges[k]) --k;
      else if (k < n_bins - 1 && rr >= edges[k + 1]) ++k;
      if (k >= 0) atomicAdd(hist + k, 1u);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < n_bins; k += blockDim.x)
    if (hist[k]) atomicAdd(counts + (size_t)r * n_bins + k, (unsigned long long)hist[k]);
}

void launch_rdf(bool mixed, const void* x, int N, const int* cell_start, const int* perm, const RepDev* reps,
                int n_reps, int C, int sites, const double* edges, int n_bins, double norm,
                unsigned long long* counts, cudaStream_t st) {
  if (C <= 0) return;
  const size_t sm = (size_t)n_bins * sizeof(unsigned int);
  if (mixed)
    k_rdf<double><<<C, kRdfThreads, sm, st>>>((const double*)x, N, cell_start, perm, reps, n_reps, sites, edges,
                                                n_bins, norm, counts);
  else
    k_rdf<float><<<C, kRdfThreads, sm, st>>>((const float*)x, N, cell_start, perm, reps, n_reps, sites, edges,
                                               n_bins, norm, counts);
}

// ------------------------------------------------------------------ ACF
constexpr int kAcfThreads = 256;

// acc[r * (max_lag + 1) + tau] += sum over replica r's chains of
// R(s) . R(s - tau); ring slot of sample t is t % (max_lag + 1).  Block
// (tau, r); thread k adds chains k, k + 256, ... in order, then a fixed tree.
__global__ void __launch_bounds__(kAcfThreads) k_acf_add(const double* __restrict__ ring, int n_chains_total,
                                                         const RepDev* __restrict__ reps, long long s, int max_lag,
                                                         double* __restrict__ acc) {
  const int tau = blockIdx.x, r = blockIdx.y;
  if (tau > s) return;
  const RepDev& R = reps[r];
  const int slots = max_lag + 1;
  const double* a = ring + (size_t)(s % slots) * 3 * n_chains_total;
  const double* b = ring + (size_t)((s - tau) % slots) * 3 * n_chains_total;
  double v = 0.0;
  for (int c = R.chain_off + threadIdx.x; c < R.chain_off + R.n_chains; c += kAcfThreads)
    v += a[3 * c] * b[3 * c] + a[3 * c + 1] * b[3 * c + 1] + a[3 * c + 2] * b[3 * c + 2];
  __shared__ double red[kAcfThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kAcfThreads / 32; ++w) t += red[w];
    acc[(size_t)r * slots + tau] += t;
  }
}

void launch_acf_add(const double* ring, int n_chains_total, const RepDev* reps, int n_reps, long long s, int max_lag,
                    double* acc, cudaStream_t st) {
  const int lags = (int)(s < max_lag ? s : max_lag) + 1;
  k_acf_add<<<dim3(lags, n_reps), kAcfThreads, 0, st>>>(ring, n_chains_total, reps, s, max_lag, acc);
}

}  // namespace mdg
