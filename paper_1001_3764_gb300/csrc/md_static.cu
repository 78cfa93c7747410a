// md_static.cu -- cell binning that allocates no device memory.
//
// md_bin_static runs the same counting sort as md_rebin (cell id per atom,
// histogram, exclusive scan, scatter, stable order by atom index inside each
// cell) for one periodic box whose positions the caller already holds on the
// GPU.  Its scratch (per-cell counters, per-atom slots and the unsorted
// permutation) lives in g_bin_scratch below, a fixed-size array in the
// library's device image; the caller passes only inputs and outputs.
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/md.h"
#include "md_kernels.cuh"

namespace mdg {

constexpr int kStaticMaxAtoms = 1 << 20;   // 1,048,576 atoms
constexpr int kStaticMaxCells = 1 << 17;   // 131,072 cells (M <= 50)

// One copy per device that loads the library, kept until the process exits:
// 4 * (2^17 + 2 * 2^20) bytes = 8.9 MB.
static __device__ __align__(256) int g_bin_scratch[kStaticMaxCells + 2 * kStaticMaxAtoms];

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

// stable order inside each cell: rank of each atom index among its cell's
__global__ void __launch_bounds__(128) k_static_rank(const int* __restrict__ cell_start, const int* __restrict__ tmp,
                                                     int* __restrict__ perm) {
  const int c = blockIdx.x;
  const int b = cell_start[c], m = cell_start[c + 1] - b;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const int id = tmp[b + k];
    int rank = 0;
    for (int q = 0; q < m; ++q) rank += tmp[b + q] < id;
    perm[b + rank] = id;
  }
}

void launch_cell_rank(const int* cell_start, const int* tmp, int* perm, int C, cudaStream_t st) {
  if (C > 0) k_static_rank<<<C, 128, 0, st>>>(cell_start, tmp, perm);
}

}  // namespace mdg

using namespace mdg;

void md_set_global_error(const char* msg);   // md_api.cu: message for md_last_error(NULL)

namespace {
constexpr int kMaxDevices = 64;
int* g_scratch_addr[kMaxDevices] = {nullptr};
}

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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return fail(MD_ECUDA, "no current device");
  if (!g_scratch_addr[dev]) {
    // first call on this device: the array's device address (host code may not
    // use the symbol itself)
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_scratch);
    if (e != cudaSuccess || !p) return fail(MD_ECUDA, "cudaGetSymbolAddress of the binning scratch failed");
    g_scratch_addr[dev] = (int*)p;
  }
  int* count = g_scratch_addr[dev];
  int* slot = count + kStaticMaxCells;
  int* tmp = slot + kStaticMaxAtoms;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double inv_h = (double)cells_per_side / box;
  if (cudaMemsetAsync(count, 0, sizeof(int) * C, st) != cudaSuccess) return fail(MD_ECUDA, "clearing the cell counters failed");
  k_static_count<<<(n_atoms + 255) / 256, 256, 0, st>>>(pos, n_atoms, box, inv_h, cells_per_side, cell_of, count, slot);
  launch_scan(count, cell_start, (int)C, st);
  launch_bin_scatter(cell_of, slot, cell_start, tmp, n_atoms, st);
  launch_cell_rank(cell_start, tmp, perm, (int)C, st);
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
