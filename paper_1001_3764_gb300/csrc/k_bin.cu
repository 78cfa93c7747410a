// k_bin.cu -- on-GPU cell binning and neighbour-list build (Sec. 3.1).
//
// The paper's GBIN_NEW claims a slot per atom with atomicAdd into a
// fixed-capacity bin (Sec. 3.1, GBIN_NEW listing).  Here the same histogram
// feeds a counting sort: histogram -> exclusive scan -> scatter -> per-cell
// rank by atom index.  The result is a stable order (cell, atom index) that
// does not depend on the order in which atomics were served, and no bin has
// a capacity limit.  Cell indices are computed in FP64 from the master
// positions with explicitly rounded operations, so they equal the oracle's.
//
// Sorted positions are stored in units of the cell side relative to the
// centre of the atom's cell (|u| <= 1/2 at the rebin), so neighbour cells are
// offset by exact integers and an FP32 coordinate carries about 2^-25 h.
// The cluster lists are built in k_lj.cu.
#include "md_kernels.cuh"

namespace mdg {

// --------------------------------------------------------------- helpers
__device__ __forceinline__ int find_rep_by_cell(const RepDev* reps, int n_reps, int c) {
  int lo = 0, hi = n_reps - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (reps[mid].cell_base <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// cell coordinate along one axis: s = x - L floor(x/L); k = floor(s * M/L).
// The integrator keeps x in [0, L), where the wrap leaves x unchanged, so the
// FP64 division is only taken for positions outside the box.
__device__ __forceinline__ int cell_coord(double x, double L, double inv_h, int M) {
  double s = x;
  if (__double_as_longlong(x) < 0 || __double_as_longlong(x) >= __double_as_longlong(L))
    s = __dsub_rn(x, __dmul_rn(L, floor(__ddiv_rn(x, L))));
  int k = __double2int_rd(__dmul_rn(s, inv_h));
  return k < 0 ? 0 : (k > M - 1 ? M - 1 : k);
}

// --------------------------------------------------------------- histogram
template <typename T>
__global__ void __launch_bounds__(256) k_bin_count(const T* __restrict__ x, int N, const Tile* __restrict__ tiles,
                                                   const RepDev* __restrict__ reps, int* __restrict__ cell_of,
                                                   int* __restrict__ cellc, int* __restrict__ count,
                                                   int* __restrict__ slot) {
  const Tile t = tiles[blockIdx.x];
  if ((int)threadIdx.x >= t.len) return;
  const int i = t.start + threadIdx.x;
  const RepDev& R = reps[t.rep];
  const double L = R.L, ih = R.inv_h;
  const int M = R.M;
  int cx = cell_coord((double)x[i], L, ih, M);
  int cy = cell_coord((double)x[N + i], L, ih, M);
  int cz = cell_coord((double)x[2 * N + i], L, ih, M);
  int c = R.cell_base + (cz * M + cy) * M + cx;
  cell_of[i] = c;
  cellc[i] = cx | (cy << 10) | (cz << 20);
  slot[i] = atomicAdd(count + c, 1);
}

void launch_bin_count(bool mixed, const void* x, int N, const Tile* tiles, int n_tiles, const RepDev* reps,
                      int* cell_of, int* cellc, int* count, int* slot, cudaStream_t st) {
  if (mixed)
    k_bin_count<double><<<n_tiles, 256, 0, st>>>((const double*)x, N, tiles, reps, cell_of, cellc, count, slot);
  else
    k_bin_count<float><<<n_tiles, 256, 0, st>>>((const float*)x, N, tiles, reps, cell_of, cellc, count, slot);
}

// --------------------------------------------------------------- exclusive scan (one block)
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ count, int* __restrict__ start, int C) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int per = (C + 1023) / 1024;
  const int b = tid * per, e = min(b + per, C);
  int s = 0;
  for (int k = b; k < e; ++k) s += count[k];
  part[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {     // Hillis-Steele inclusive scan
    int v = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int run = part[tid] - s;
  for (int k = b; k < e; ++k) { start[k] = run; run += count[k]; }
  if (tid == 1023) start[C] = part[1023];
}

void launch_scan(const int* count, int* cell_start, int C, cudaStream_t st) {
  k_scan<<<1, 1024, 0, st>>>(count, cell_start, C);
}

// the same scan for cell_start and, over ceil(count / 4), for cl_start
__global__ void __launch_bounds__(1024) k_scan2(const int* __restrict__ count, int* __restrict__ start,
                                                int* __restrict__ cl_start, int C) {
  __shared__ int part[2][1024];
  const int tid = threadIdx.x;
  const int per = (C + 1023) / 1024;
  const int b = tid * per, e = min(b + per, C);
  int s = 0, sc = 0;
  for (int k = b; k < e; ++k) { const int n = count[k]; s += n; sc += (n + 3) >> 2; }
  part[0][tid] = s;
  part[1][tid] = sc;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {     // Hillis-Steele inclusive scans
    const int v = tid >= off ? part[0][tid - off] : 0;
    const int vc = tid >= off ? part[1][tid - off] : 0;
    __syncthreads();
    part[0][tid] += v;
    part[1][tid] += vc;
    __syncthreads();
  }
  int run = part[0][tid] - s, runc = part[1][tid] - sc;
  for (int k = b; k < e; ++k) {
    const int n = count[k];
    start[k] = run; run += n;
    cl_start[k] = runc; runc += (n + 3) >> 2;
  }
  if (tid == 1023) { start[C] = part[0][1023]; cl_start[C] = part[1][1023]; }
}

void launch_scan2(const int* count, int* cell_start, int* cl_start, int C, cudaStream_t st) {
  k_scan2<<<1, 1024, 0, st>>>(count, cell_start, cl_start, C);
}

// --------------------------------------------------------------- scatter
__global__ void __launch_bounds__(256) k_bin_scatter(const int* __restrict__ cell_of, const int* __restrict__ slot,
                                                     const int* __restrict__ cell_start, int* __restrict__ tmp, int N) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) tmp[cell_start[cell_of[i]] + slot[i]] = i;
}

void launch_bin_scatter(const int* cell_of, const int* slot, const int* cell_start, int* tmp, int N,
                        cudaStream_t st) {
  if (N > 0) k_bin_scatter<<<(N + 255) / 256, 256, 0, st>>>(cell_of, slot, cell_start, tmp, N);
}

// --------------------------------------------------------------- per-cell stable order + sorted arrays
constexpr int kSortCap = 2048;

template <typename T>
__global__ void __launch_bounds__(128) k_cell_sort(const T* __restrict__ x, int N, const int* __restrict__ cell_start,
                                                   const int* __restrict__ tmp, const unsigned char* __restrict__ mtype,
                                                   const int* __restrict__ cellc,
                                                   const uint16_t* __restrict__ site, const RepDev* __restrict__ reps,
                                                   int n_reps, int sites, int* __restrict__ perm,
                                                   int* __restrict__ inv_perm, float4* __restrict__ pos,
                                                   int* __restrict__ tag, float4* __restrict__ ref,
                                                   unsigned* __restrict__ flags) {
  __shared__ int ids[kSortCap];
  const int c = blockIdx.x;
  const int b = cell_start[c], n = cell_start[c + 1] - b;
  if (n == 0) return;
  const RepDev& R = reps[find_rep_by_cell(reps, n_reps, c)];
  // A cell of more than kSortCap atoms (over 40 times a melt's ~46) cannot
  // be staged by the force kernels either: it is reported as a capacity
  // overflow, and its atoms keep their bucket order (bounded work).
  const bool in_smem = n <= kSortCap;
  if (!in_smem && threadIdx.x == 0) atomicOr(flags, kFlagNbrOverflow);
  if (in_smem)
    for (int k = threadIdx.x; k < n; k += blockDim.x) ids[k] = tmp[b + k];
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int id = in_smem ? ids[k] : tmp[b + k];
    int rank = k;
    if (in_smem) {
      rank = 0;
      for (int q = 0; q < n; ++q) rank += ids[q] < id;
    }
    const int s = b + rank;
    perm[s] = id;
    inv_perm[id] = s;
    const int cc = cellc[id];
    float4 p;
    if constexpr (sizeof(T) == 8) {      // FP64 master: integer-pipe offset and rounding, same value
      p.x = cell_unit_t(x[id], cc & 1023, R);
      p.y = cell_unit_t(x[N + id], (cc >> 10) & 1023, R);
      p.z = cell_unit_t(x[2 * N + id], (cc >> 20) & 1023, R);
    } else {
      p.x = cell_unit(x[id], cc & 1023, 0, R);
      p.y = cell_unit(x[N + id], (cc >> 10) & 1023, 0, R);
      p.z = cell_unit(x[2 * N + id], (cc >> 20) & 1023, 0, R);
    }
    const int st = site[id];
    const int chain = R.chain_off + (id - R.atom_off) / sites;
    const int type = mtype ? (int)mtype[st] : ((st == 0 || st == sites - 1) ? 1 : 0);
    p.w = (float)type;   // LJ type: the tile kernels copy positions as they are
    pos[s] = p;
    ref[id] = p;
    tag[s] = (chain << kTagSiteBits) | st | (type << kTagTypeBit);
  }
}

void launch_cell_sort(bool mixed, const void* x, int N, const int* cell_start, const int* tmp,
                      const unsigned char* mtype, const int* cellc,
                      const uint16_t* site, const RepDev* reps, int n_reps, int C, int sites, int* perm,
                      int* inv_perm, float4* pos, int* tag, float4* ref, unsigned* flags, cudaStream_t st) {
  if (mixed)
    k_cell_sort<double><<<C, 128, 0, st>>>((const double*)x, N, cell_start, tmp, mtype, cellc, site, reps, n_reps, sites,
                                           perm, inv_perm, pos, tag, ref, flags);
  else
    k_cell_sort<float><<<C, 128, 0, st>>>((const float*)x, N, cell_start, tmp, mtype, cellc, site, reps, n_reps, sites,
                                          perm, inv_perm, pos, tag, ref, flags);
}

}  // namespace mdg
