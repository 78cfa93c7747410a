// md_static.cu -- cell binning that allocates no device memory.
//
// md_bin_static runs the same counting sort as md_rebin (cell id per atom,
// histogram, exclusive scan, scatter, stable order by atom index inside each
// cell) for one periodic box whose positions the caller already holds on the
// GPU.  Its scratch (per-cell counters, per-atom slots and the unsorted
// permutation, a merge buffer) lives in g_bin_scratch below, a fixed-size
// array in the library's device image; the caller passes only inputs and
// outputs.  The order inside a cell costs O(m log m) for a cell of m atoms
// (sorted runs of 256 in shared memory, then merge passes), so a call's work
// stays bounded whatever the positions: at the limits (2^20 atoms, all in
// one cell) it is 4,096 runs on one block plus 12 merge passes.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/md.h"
#include "md_kernels.cuh"

namespace mdg {

constexpr int kStaticMaxAtoms = 1 << 20;   // 1,048,576 atoms
constexpr int kStaticMaxCells = 1 << 17;   // 131,072 cells (M <= 50)
constexpr int kRun = 256;                  // atoms ordered in shared memory at once
constexpr int kMergePasses = 12;           // kRun << 12 = 2^20 = kStaticMaxAtoms (enough for any n)

// One copy per device that loads the library, kept until the process exits:
// per-cell counters, then four per-atom arrays (slots / position-to-cell map,
// the unsorted permutation, a merge buffer), then one int holding the largest
// cell of the last call: 4 * (2^17 + 3 * 2^20 + 64) bytes = 13.1 MB.
constexpr size_t kScratchInts = (size_t)kStaticMaxCells + 3 * (size_t)kStaticMaxAtoms + 64;
static __device__ __align__(256) int g_bin_scratch[kScratchInts];

// same cell formula as the system path: s = x - L floor(x/L), k = floor(s M/L)
__device__ __forceinline__ int static_coord(double x, double L, double inv_h, int M) {
  double s = x;
  if (__double_as_longlong(x) < 0 || __double_as_longlong(x) >= __double_as_longlong(L))
    s = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
  int k = __double2int_rd(__dmul_rn(s, inv_h));
  return k < 0 ? 0 : (k > M - 1 ? M - 1 : k);
}

__global__ void __launch_bounds__(256) k_static_count(const double* __restrict__ x, int n, double L, double inv_h, int M,
                                                      int* __restrict__ cell_of, int* __restrict__ count,
                                                      int* __restrict__ slot) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cx = static_coord(x[i], L, inv_h, M);
  const int cy = static_coord(x[n + i], L, inv_h, M);
  const int cz = static_coord(x[2 * n + i], L, inv_h, M);
  const int c = (cz * M + cy) * M + cx;
  cell_of[i] = c;
  slot[i] = atomicAdd(count + c, 1);
}

// Stable order inside each cell, by atom index, in bounded work.  Each run of
// kRun consecutive slots of a cell is ordered in shared memory (rank = the
// number of smaller ids in the run: kRun compares per atom).  A cell of at
// most kRun atoms is then final and goes straight to perm; a larger cell
// leaves its ordered runs in `runs` (in place) and records, per slot, its
// cell in pcell (-1 for slots of small cells) for the merge passes below.
__global__ void __launch_bounds__(kRun) k_static_runs(const int* __restrict__ cell_start, int* __restrict__ runs,
                                                      int* __restrict__ pcell, int* __restrict__ perm,
                                                      int* __restrict__ maxm) {
  __shared__ int ids[kRun];
  const int c = blockIdx.x;
  const int b = cell_start[c], m = cell_start[c + 1] - b;
  const bool small = m <= kRun;
  if (!small && threadIdx.x == 0) atomicMax(maxm, m);
  for (int r0 = 0; r0 < m; r0 += kRun) {
    const int len = min(kRun, m - r0);
    const int k = threadIdx.x;
    int id = 0;
    if (k < len) ids[k] = id = runs[b + r0 + k];
    __syncthreads();
    if (k < len) {
      int rank = 0;
      for (int q = 0; q < len; ++q) rank += ids[q] < id;
      if (small) {
        perm[b + rank] = id;
        pcell[b + k] = -1;
      } else {
        runs[b + r0 + rank] = id;
        pcell[b + r0 + k] = c;
      }
    }
    __syncthreads();
  }
}

// One merge pass: runs of R sorted ids are merged pairwise.  An id at offset q
// of its run r moves to min(r, r ^ 1) R + (q - r R) + (the number of ids of
// the partner run below it, by binary search; ids are distinct).  A cell of
// at most 2 R atoms is complete after this pass and is written to perm.
__global__ void __launch_bounds__(256) k_static_merge(const int* __restrict__ cell_start, const int* __restrict__ pcell,
                                                      const int* __restrict__ in, int* __restrict__ out,
                                                      int* __restrict__ perm, const int* __restrict__ maxm, int n,
                                                      int R) {
  if (*maxm <= R) return;   // no cell still has more than one run of R
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int c = pcell[p];
  if (c < 0) return;
  const int b = cell_start[c], m = cell_start[c + 1] - b;
  if (m <= R) return;       // completed by an earlier pass
  const int q = p - b, r = q / R, r0 = r * R, o0 = (r ^ 1) * R;
  const int olen = min(R, m - o0);
  const int id = in[p];
  int lb = 0;
  if (olen > 0) {
    int lo = 0, hi = olen;
    const int* o = in + b + o0;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (o[mid] < id) lo = mid + 1; else hi = mid;
    }
    lb = lo;
  }
  const int dst = b + min(r0, o0) + (q - r0) + lb;
  if (m <= 2 * R) perm[dst] = id; else out[dst] = id;
}

void launch_static_order(const int* cell_start, int C, int n, int* runs, int* buf, int* pcell, int* perm, int* maxm,
                         cudaStream_t st) {
  if (C <= 0 || n <= 0) return;
  k_static_runs<<<C, kRun, 0, st>>>(cell_start, runs, pcell, perm, maxm);
  int* a = runs;
  int* b = buf;
  // a cell holds at most n atoms: passes until one run covers n
  int passes = 0;
  while (passes < kMergePasses && ((long long)kRun << passes) < n) ++passes;
  for (int k = 0; k < passes; ++k) {
    k_static_merge<<<(n + 255) / 256, 256, 0, st>>>(cell_start, pcell, a, b, perm, maxm, n, kRun << k);
    int* t = a; a = b; b = t;
  }
}

}  // namespace mdg

using namespace mdg;

void md_set_global_error(const char* msg);   // md_api.cu: message for md_last_error(NULL)

extern "C" int md_bin_static(const double* pos, int32_t n_atoms, double box, int32_t cells_per_side, int32_t* cell_of,
                             int32_t* cell_start, int32_t* perm, void* cuda_stream) {
  auto fail = [](int code, const char* msg) {
    md_set_global_error(msg);
    return code;
  };
  if (!pos || !cell_of || !cell_start || !perm) return fail(MD_EINVAL, "null pointer argument");
  if (n_atoms < 1 || n_atoms > kStaticMaxAtoms) return fail(MD_EINVAL, "n_atoms must be 1 .. 1,048,576");
  if (cells_per_side < 1) return fail(MD_EINVAL, "cells_per_side must be >= 1");
  const long long C = (long long)cells_per_side * cells_per_side * cells_per_side;
  if (C > kStaticMaxCells) return fail(MD_EINVAL, "more than 131,072 cells (cells_per_side > 50)");
  if (!(box > 0) || !std::isfinite(box)) return fail(MD_EINVAL, "box must be positive");
  // The array's device address on the current device (host code may not use
  // the symbol itself).  Looked up on every call: it is cheap, and a cached
  // address would go stale if the device's context were reset and the module
  // loaded again elsewhere.
  void* sp = nullptr;
  const cudaError_t se = cudaGetSymbolAddress(&sp, g_bin_scratch);
  if (se != cudaSuccess || !sp) {
    cudaGetLastError();
    return fail(MD_ECUDA, "cudaGetSymbolAddress of the binning scratch failed");
  }
  int* scratch = (int*)sp;
  int* count = scratch;
  int* slot = count + kStaticMaxCells;       // slots, then the position-to-cell map
  int* tmp = slot + kStaticMaxAtoms;         // the unsorted permutation, then ordered runs
  int* buf = tmp + kStaticMaxAtoms;          // the other merge buffer
  int* maxm = buf + kStaticMaxAtoms;         // largest cell above one run
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double inv_h = (double)cells_per_side / box;
  if (cudaMemsetAsync(count, 0, sizeof(int) * C, st) != cudaSuccess ||
      cudaMemsetAsync(maxm, 0, sizeof(int), st) != cudaSuccess)
    return fail(MD_ECUDA, "clearing the cell counters failed");
  k_static_count<<<(n_atoms + 255) / 256, 256, 0, st>>>(pos, n_atoms, box, inv_h, cells_per_side, cell_of, count, slot);
  launch_scan(count, cell_start, (int)C, st);
  launch_bin_scatter(cell_of, slot, cell_start, tmp, n_atoms, st);
  launch_static_order(cell_start, (int)C, n_atoms, tmp, buf, slot, perm, maxm, st);
  if (cudaGetLastError() != cudaSuccess) return fail(MD_ECUDA, "a binning kernel failed to launch");
  return MD_OK;
}

extern "C" int md_wait_selftest(int32_t spins) {
  if (spins < 1 || spins > 100000) {
    md_set_global_error("spins must be 1 .. 100000");
    return MD_EINVAL;
  }
  unsigned* flag = nullptr;
  if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    md_set_global_error("device allocation failed");
    return MD_ENOMEM;
  }
  unsigned f = 0;
  const bool ok = cudaMemset(flag, 0, sizeof(unsigned)) == cudaSuccess &&
                  (launch_wait_selftest((unsigned)spins, flag, 0), cudaGetLastError() == cudaSuccess) &&
                  cudaMemcpy(&f, flag, sizeof f, cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaFree(flag);
  if (!ok) {
    md_set_global_error("the wait self-test failed to run");
    return MD_ECUDA;
  }
  if (f & kFlagTimeout) {
    md_set_global_error("a bounded device wait gave up (expected in this self-test)");
    return MD_ETIMEOUT;
  }
  return MD_OK;
}
