// k_lj.cu -- neighbour list (Sec. 3.1) and Lennard-Jones force (Eq. 2,
// Sec. 3.2) over shared-memory tiles of the 27 cells around a home cell.
//
// One thread block per home cell.  The block stages the atoms of the 27
// neighbour cells (k = (oz+1)*9 + (oy+1)*3 + ox+1, each cell in sorted order)
// in shared memory, moved into the home cell's frame: w_j = u_j + o_k in cell
// units (|w| < 1.6, so FP32 keeps ~6e-8 of a cell side).  A pair separation is
// then u_i - w_j.  The paper's neighbour-search kernel also assigns a block to
// a grid cell and stages the 27 cells (Sec. 3.1, last paragraph); here the
// same staging serves the force kernel, and the list stores 16-bit indices
// into the staged tile instead of global atom ids.
//
// List build: every thread scans the whole tile for its home atom (cutoff
// r_c + skin, 1-2 and 1-3 neighbours excluded, Sec. 3.1), keeps its entries
// in shared memory and the block writes them out row by row (coalesced).
//
// Force: up to four threads share one home atom (entries q = p, p+T, ...),
// and their partial sums are added in a fixed order, so the result does not
// depend on scheduling.  Each pair follows the Sec. 3.2 listing: r2inv = 0
// when r^2 >= r_c^2.
#include "md_kernels.cuh"

namespace mdg {

constexpr int kStageCapMax = 6144;  // largest 27-cell tile (96 KB of float4); the staged index has 15 bits

__device__ __forceinline__ int find_rep_cell(const RepDev* reps, int n_reps, int c) {
  int lo = 0, hi = n_reps - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (reps[mid].cell_base <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Neighbour-cell table of home cell c: start[k] of each cell's atoms in sorted
// order and off[k] = position of cell k's first atom in the tile; off[27] =
// tile size.  Threads 0..31 fill it (one warp scan).
struct CellTile {
  int start[27];
  int off[28];
  float ox[27], oy[27], oz[27];
};

__device__ __forceinline__ void tile_setup(CellTile& T, int c, const RepDev& R, const int* __restrict__ cell_start) {
  if (threadIdx.x < 32) {
    const int k = threadIdx.x;
    int n = 0;
    if (k < 27) {
      const int M = R.M, lc = c - R.cell_base;
      const int cx = lc % M, cy = (lc / M) % M, cz = lc / (M * M);
      const int ox = k % 3 - 1, oy = (k / 3) % 3 - 1, oz = k / 9 - 1;
      const int nc = R.cell_base + (((cz + oz + M) % M) * M + ((cy + oy + M) % M)) * M + ((cx + ox + M) % M);
      T.start[k] = cell_start[nc];
      n = cell_start[nc + 1] - T.start[k];
      T.ox[k] = (float)ox; T.oy[k] = (float)oy; T.oz[k] = (float)oz;
    }
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (k >= o) incl += v;
    }
    if (k < 27) T.off[k] = incl - n;
    if (k == 26) T.off[27] = incl;
  }
  __syncthreads();
}

// Copy the tile into shared memory, shifted into the home cell's frame: warp
// w copies cells k = w, w + nwarps, ... (each cell is one contiguous run of
// sorted atoms).
// WITH_TAG: w = the atom's chain and site bits (tag without the type bit;
// list build); otherwise w keeps the LJ type (0.0 / 1.0) that binning and
// integration store in the sorted positions (force kernel).
template <bool WITH_TAG>
__device__ __forceinline__ void tile_load(const CellTile& T, const float4* __restrict__ pos, const int* __restrict__ tag,
                                          float4* __restrict__ sp) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = threadIdx.x >> 5; k < 27; k += nw) {
    const int n = T.off[k + 1] - T.off[k], j0 = T.start[k], t0 = T.off[k];
    const float ox = T.ox[k], oy = T.oy[k], oz = T.oz[k];
    for (int q = lane; q < n; q += 32) {
      float4 p = __ldg(pos + j0 + q);
      p.x += ox; p.y += oy; p.z += oz;
      if (WITH_TAG) p.w = __int_as_float(__ldg(tag + j0 + q) & (int)kTagMask);
      sp[t0 + q] = p;
    }
  }
}

// ===================================================================== build
// List layout: blocks of 8 entries, block q of sorted atom s is nbr[q * Npad
// + s], so one 16-byte load gives a thread 8 entries and a warp reads 512
// contiguous bytes.  ncount[s] is the number of blocks.  Unused slots hold the
// tile's sentinel index (= tile size): a staged atom placed far outside the
// cutoff, so a padded slot adds exactly zero force and energy.
//
// TP adjacent threads share a home atom; in every 32-atom word of the tile
// thread p takes atoms p, p + TP, ... (the lanes of a warp read neighbouring
// 16-byte slots: one shared-memory wavefront) and keeps those within r_c +
// skin that are not itself or a 1-2/1-3 neighbour (tag test, Sec. 3.1).  The
// test and the keep are branch-free: a kept index goes to the thread's
// 16-slot ring in shared memory (a predicated store) and the ring is written
// out as a block of 8 whenever it holds 8, so no lane waits on another's set
// bits.  Thread p writes its blocks at p, p + TP, ..., entries in increasing
// tile order; the TP threads then pad to a common number of blocks.
constexpr int kBuildThreads = 256;
constexpr int kRingRow = 2 * kBuildThreads;   // bytes of one ring slot row (slot k of every thread)

__device__ __forceinline__ uint4 pack_block(unsigned long long lo, unsigned long long hi) {
  return make_uint4((unsigned)lo, (unsigned)(lo >> 32), (unsigned)hi, (unsigned)(hi >> 32));
}

// entries r0 .. r0+7 of this thread's ring (byte offset `base` of slot r0),
// slots k >= nk replaced by the sentinel
__device__ __forceinline__ uint4 ring_block(const unsigned char* ring, unsigned base, int nk, unsigned sent) {
  unsigned e[8];
#pragma unroll
  for (int k = 0; k < 8; ++k)
    e[k] = k < nk ? *reinterpret_cast<const unsigned short*>(ring + base + k * kRingRow) : sent;
  return make_uint4(e[0] | (e[1] << 16), e[2] | (e[3] << 16), e[4] | (e[5] << 16), e[6] | (e[7] << 16));
}

template <int TP>
__device__ __forceinline__ void build_atom(const float4* __restrict__ sp, int nwords, int total, float rl2, int s, int p,
                                           const float4& pi, int ti, unsigned char* ring, uint4* __restrict__ nbr,
                                           int Npad, int capb, int& nb_out) {
  constexpr int per = 32 / TP;                 // candidates of each word taken by this lane (8, 16 or 32)
  const unsigned me = 2u * threadIdx.x;        // this thread's column in the ring
  const unsigned tip2 = (unsigned)ti + 2u;
  unsigned kept = 0u, done = 0u;               // entries kept / written out, x kRingRow
  int nb = 0;
  for (int wd = 0; wd < nwords; ++wd) {
    const float4* w32 = sp + wd * 32 + p;
    const unsigned t0 = (unsigned)(wd * 32 + p);
#pragma unroll
    for (int c0 = 0; c0 < per; c0 += 8) {
#pragma unroll
      for (int u = c0; u < c0 + 8; ++u) {
        const float4 w = w32[u * TP];
        const float dx = pi.x - w.x, dy = pi.y - w.y, dz = pi.z - w.z;
        // |i - j| <= 2 within one chain: itself, 1-2 and 1-3 neighbours
        const bool keep = (dx * dx + dy * dy + dz * dz < rl2) & (tip2 - (unsigned)__float_as_int(w.w) > 4u);
        if (keep) *reinterpret_cast<unsigned short*>(ring + ((kept & (15u * kRingRow)) | me)) =
            (unsigned short)(t0 + u * TP);
        kept += keep ? (unsigned)kRingRow : 0u;
      }
      // at most 8 + 7 entries pending here, so one block of 8 drains it below 8
      if (kept - done >= 8u * kRingRow) {
        const int q = p + TP * nb;
        if (q < capb) nbr[(size_t)q * Npad + s] = ring_block(ring, (done & (8u * kRingRow)) | me, 8, 0u);
        ++nb;
        done += 8u * kRingRow;
      }
    }
  }
  const int rem = (int)((kept - done) / kRingRow);
  if (rem) {                                          // pad the open block with the sentinel
    const int q = p + TP * nb;
    if (q < capb) nbr[(size_t)q * Npad + s] = ring_block(ring, (done & (8u * kRingRow)) | me, rem, (unsigned)total);
    ++nb;
  }
  nb_out = nb;
}

__global__ void __launch_bounds__(kBuildThreads) k_nbr_tile(const float4* __restrict__ pos, const int* __restrict__ tag,
                                                            const int* __restrict__ cell_start,
                                                            const RepDev* __restrict__ reps, int n_reps,
                                                            uint4* __restrict__ nbr, int* __restrict__ ncount, int cap,
                                                            int Npad, int tile_cap, unsigned* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sp = reinterpret_cast<float4*>(smem);
  __shared__ CellTile T;
  __shared__ __align__(16) unsigned char ring[16 * kRingRow];
  const int c = blockIdx.x;
  const int b = cell_start[c], n = cell_start[c + 1] - b;
  if (n == 0) return;
  const RepDev& R = reps[find_rep_cell(reps, n_reps, c)];
  tile_setup(T, c, R, cell_start);
  const int total = T.off[27];
  const int nwords = (total + 32) >> 5;            // room for the sentinel at index total
  if (nwords * 32 > tile_cap) {
    if (threadIdx.x == 0) atomicOr(flags, kFlagNbrOverflow);
    for (int i = threadIdx.x; i < n; i += blockDim.x) ncount[b + i] = 0;
    return;
  }
  tile_load<true>(T, pos, tag, sp);
  for (int t = total + threadIdx.x; t < nwords * 32; t += blockDim.x) sp[t] = make_float4(1e9f, 1e9f, 1e9f, 0.f);
  __syncthreads();
  const float rl2 = R.rlist2u;
  const unsigned long long sent = (unsigned long long)total;
  const unsigned long long sent4 = sent | (sent << 16) | (sent << 32) | (sent << 48);
  const int TP = n > kBuildThreads / 2 ? 1 : (n > kBuildThreads / 4 ? 2 : 4);
  const int per_pass = kBuildThreads / TP;
  const int capb = cap >> 3;
  for (int a0 = 0; a0 < n; a0 += per_pass) {
    const int a = a0 + (int)threadIdx.x / TP, p = (int)threadIdx.x % TP;
    const bool active = a < n;
    const int s = b + a;
    int nb = 0;
    if (active) {
      const float4 pi = pos[s];
      const int ti = tag[s] & (int)kTagMask;
      if (TP == 1) build_atom<1>(sp, nwords, total, rl2, s, p, pi, ti, ring, nbr, Npad, capb, nb);
      else if (TP == 2) build_atom<2>(sp, nwords, total, rl2, s, p, pi, ti, ring, nbr, Npad, capb, nb);
      else build_atom<4>(sp, nwords, total, rl2, s, p, pi, ti, ring, nbr, Npad, capb, nb);
    }
    // common block count of the TP threads of an atom (adjacent lanes)
    int mb = nb;
    if (TP >= 2) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 1));
    if (TP >= 4) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, 2));
    if (active) {
      for (int k = nb; k < mb; ++k) {
        const int q = p + TP * k;
        if (q < capb) nbr[(size_t)q * Npad + s] = pack_block(sent4, sent4);
      }
      const int nblk = TP * mb;
      if (p == 0) {
        ncount[s] = min(nblk, capb);
        if (nblk > capb) atomicOr(flags, kFlagNbrOverflow);
      }
    }
  }
}

size_t nbr_tile_smem(int tile_cap) { return (size_t)tile_cap * sizeof(float4); }

void launch_nbr_tile(const float4* pos, const int* tag, const int* cell_start, const RepDev* reps, int n_reps, int C,
                     uint4* nbr, int* ncount, int cap, int Npad, int tile_cap, unsigned* flags, cudaStream_t st) {
  k_nbr_tile<<<C, kBuildThreads, nbr_tile_smem(tile_cap), st>>>(pos, tag, cell_start, reps, n_reps, nbr, ncount, cap,
                                                                Npad, tile_cap, flags);
}

// ===================================================================== force
constexpr int kEnergyVals = 8;   // lj, lj_shifted, vxx, vyy, vzz, vxy, vxz, vyz

// FP32 force -> int64 fixed point (2^-32 kJ/mol/nm).  Each part (LJ, bonded)
// is kept below 2^18 kJ/mol/nm so that their sum converts exactly to FP64.
__device__ __forceinline__ long long fix_of(float f, unsigned* flags) {
  if (!(fabsf(f) < 262144.0f)) { atomicOr(flags, kFlagFixOverflow); return 0; }
  return __float2ll_rn(f * 4294967296.0f);
}

// Energy and virial sums of one warp: the 32 lanes' FP32 partials are added
// in FP32 by a fixed shuffle tree, and lane 0 stores the warp sum as FP64
// (halved: a full list counts every pair twice).  The block then adds its
// warps in FP64, and all later sums are FP64.  A per-lane FP64 tree would
// cost 8 conversions and 40 FP64 adds per thread on this GPU's narrow FP64
// pipe, more than the pair loop of the energy kernel.
template <int NW>
__device__ __forceinline__ void warp_energy_sums(const float (&ev)[8], int lane, double (&red)[8][NW], int w) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    float sv = ev[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sv += __shfl_down_sync(0xffffffffu, sv, o);
    if (lane == 0) red[k][w] = 0.5 * (double)sv;
  }
}

// one pair of Eq. (2) in cell units (Sec. 3.2 listing: r2inv = 0 beyond r_c);
// w.w is j's type (0/1), so the pair constants are a0 + t_j (a1 - a0)
template <bool ENERGY>
__device__ __forceinline__ void lj_pair(unsigned t, const float4* __restrict__ sp, const float4& pi, float rc2, float a0c,
                                        float da, float b0c, float db, const float (&ec)[6],
                                        float& fx, float& fy, float& fz, float (&ev)[8]) {
  const float4 w = sp[t];
  const float dx = pi.x - w.x, dy = pi.y - w.y, dz = pi.z - w.z;
  const float r2 = dx * dx + dy * dy + dz * dz;
  const float A = fmaf(w.w, da, a0c), B = fmaf(w.w, db, b0c);
  const float ir2 = r2 < rc2 ? rcp_approx(r2) : 0.f;
  const float ir6 = ir2 * ir2 * ir2;
  const float ff = ir2 * ir6 * (A * ir6 - B);
  fx += ff * dx;
  fy += ff * dy;
  fz += ff * dz;
  if (ENERGY) {
    // the partner's type blends the home atom's two coefficient pairs (ec);
    // beyond r_c ir6 is 0, so only the shift needs the cutoff test
    const float c12 = fmaf(w.w, ec[1], ec[0]), c6 = fmaf(w.w, ec[3], ec[2]);
    const float eij = ir6 * (c12 * ir6 - c6);
    ev[0] += eij;
    ev[1] += eij - (r2 < rc2 ? fmaf(w.w, ec[5], ec[4]) : 0.f);
    ev[2] += dx * dx * ff; ev[3] += dy * dy * ff; ev[4] += dz * dz * ff;
    ev[5] += dx * dy * ff; ev[6] += dx * dz * ff; ev[7] += dy * dz * ff;
  }
}

// Force on the home atoms of one cell (block-wide; all threads call it).
template <bool MIXED, bool ENERGY, int NT>
__device__ __forceinline__ void lj_cell(int c, const float4* __restrict__ pos, const int* __restrict__ tag,
                                        const int* __restrict__ cell_start, const uint4* __restrict__ nbr,
                                        const int* __restrict__ ncount, int Npad, int tile_cap,
                                        const RepDev* __restrict__ reps, int n_reps, const ForceParams& fp,
                                        void* __restrict__ flj, double* __restrict__ epart, unsigned* __restrict__ flags,
                                        float4* sp, CellTile& T, double (&red)[kEnergyVals][NT / 32]) {
  const int b = cell_start[c], n = cell_start[c + 1] - b;
  float ev[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const RepDev& R = reps[find_rep_cell(reps, n_reps, c)];
  int total = 0;
  if (n > 0) {
    tile_setup(T, c, R, cell_start);
    total = T.off[27];
  }
  if (n > 0 && ((total + 32) & ~31) <= tile_cap) {
    tile_load<false>(T, pos, tag, sp);
    if (threadIdx.x == 0) sp[total] = make_float4(1e9f, 1e9f, 1e9f, 0.f);   // sentinel slot
    __syncthreads();
    // TP adjacent lanes share one home atom: entry blocks p, p + TP, ...
    const int TP = n > NT / 2 ? 1 : (n > NT / 4 ? 2 : 4);
    const float rc2 = R.rc2u;
    const float ih = R.ih_hi;
    for (int a0 = 0; a0 < n; a0 += NT / TP) {
      const int na = min(NT / TP, n - a0);
      const int a = a0 + (int)threadIdx.x / TP, p = (int)threadIdx.x % TP;
      const bool active = a < a0 + na;
      float fx = 0.f, fy = 0.f, fz = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
      if (active) {
        const int s = b + a;
        const float4 pi = pos[s];
        const int ti = (int)pi.w;                   // LJ type, kept in w by binning and integration
        const float a0c = 12.f * R.C12u[ti], b0c = 6.f * R.C6u[ti];
        const float da = 12.f * R.C12u[ti + 1] - a0c, db = 6.f * R.C6u[ti + 1] - b0c;
        float ec[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};     // energy coefficients (ENERGY only)
        if (ENERGY) {
          ec[0] = R.C12u[ti]; ec[1] = R.C12u[ti + 1] - ec[0];
          ec[2] = R.C6u[ti]; ec[3] = R.C6u[ti + 1] - ec[2];
          ec[4] = fp.erc[ti][0]; ec[5] = fp.erc[ti][1] - ec[4];
        }
        const int nblk = ncount[s];
        const uint4* np = nbr + s;
        const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
        int blk = p;
        // two blocks in flight ahead of the one being processed
        uint4 E = blk < nblk ? __ldg(np + (size_t)blk * Npad) : z4;
        uint4 E1 = blk + TP < nblk ? __ldg(np + (size_t)(blk + TP) * Npad) : z4;
        while (blk < nblk) {
          const int n2 = blk + 2 * TP;
          const uint4 E2 = n2 < nblk ? __ldg(np + (size_t)n2 * Npad) : z4;
          const unsigned ew[4] = {E.x, E.y, E.z, E.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            lj_pair<ENERGY>(ew[u] & 0xffffu, sp, pi, rc2, a0c, da, b0c, db, ec, fx, fy, fz, ev);
            lj_pair<ENERGY>(ew[u] >> 16, sp, pi, rc2, a0c, da, b0c, db, ec, gx, gy, gz, ev);
          }
          E = E1;
          E1 = E2;
          blk += TP;
        }
      }
      fx += gx; fy += gy; fz += gz;
      // sum the TP partial forces of an atom (adjacent lanes, fixed order)
      if (TP >= 2) {
        fx += __shfl_down_sync(0xffffffffu, fx, 1); fy += __shfl_down_sync(0xffffffffu, fy, 1); fz += __shfl_down_sync(0xffffffffu, fz, 1);
      }
      if (TP >= 4) {
        fx += __shfl_down_sync(0xffffffffu, fx, 2); fy += __shfl_down_sync(0xffffffffu, fy, 2); fz += __shfl_down_sync(0xffffffffu, fz, 2);
      }
      if (active && p == 0) {
        fx *= ih; fy *= ih; fz *= ih;             // back from cell units
        const int s = b + a;
        if (MIXED) {
          F4i o;
          o.x = fix_of(fx, flags); o.y = fix_of(fy, flags); o.z = fix_of(fz, flags); o.w = 0;
          reinterpret_cast<F4i*>(flj)[s] = o;
        } else {
          reinterpret_cast<float4*>(flj)[s] = make_float4(fx, fy, fz, 0.f);
        }
      }
    }
  } else if (n > 0 && threadIdx.x == 0) {
    atomicOr(flags, kFlagNbrOverflow);
  }
  if (ENERGY) {
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    warp_energy_sums(ev, lane, red, wi);
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int k = 0; k < kEnergyVals; ++k) {
        double sv = 0.0;
        for (int q = 0; q < NT / 32; ++q) sv += red[k][q];
        epart[(size_t)c * kEnergyVals + k] = sv;
      }
    }
  }
  __syncthreads();   // the tile and tables are reused by the next cell of this block
}

// One block per cell.  TPS > 0 asks the compiler for TPS / NT resident
// blocks per SM (TPS = 1536: 40 registers; 1024: 64).  The force-only form
// is launched with the largest TPS whose block count the tile's shared
// memory also allows: 2 of a block's 8 warps often have no home atom, so
// more resident blocks keep more warps at work.  Tiles too large for 1024
// threads per SM use the unconstrained allocation.  The energy form (eight
// more accumulators) is compiled for 1024 threads per SM (64 registers, no
// spills) instead of the 2 blocks its unconstrained allocation would allow.
template <bool MIXED, bool ENERGY, int NT, int TPS>
__global__ void __launch_bounds__(NT, TPS > 0 ? TPS / NT : (ENERGY ? 1024 / NT : 1)) k_lj_tile(const float4* __restrict__ pos, const int* __restrict__ tag,
                                                const int* __restrict__ cell_start,
                                                const uint4* __restrict__ nbr, const int* __restrict__ ncount,
                                                int Npad, int tile_cap, const RepDev* __restrict__ reps, int n_reps,
                                                const ForceParams fp, void* __restrict__ flj,
                                                double* __restrict__ epart, unsigned* __restrict__ flags) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sp = reinterpret_cast<float4*>(smem);      // the tile, tile_cap entries
  __shared__ CellTile T;
  __shared__ double red[kEnergyVals][NT / 32];
  lj_cell<MIXED, ENERGY, NT>(blockIdx.x, pos, tag, cell_start, nbr, ncount, Npad, tile_cap, reps, n_reps, fp, flj,
                             epart, flags, sp, T, red);
}

// ===================================================================== force, pipelined
// Persistent blocks of NT/32 consumer warps and one producer warp.  The
// producer takes the next cell from a counter, builds its 27-cell table, and
// stages the cell's tile (27 runs of sorted positions, LJ type in w) and the
// list rows of its home atoms in shared memory with bulk asynchronous copies
// (cp.async.bulk, completion counted in bytes on an mbarrier), two stages
// deep.  The consumers shift the staged tile into the home frame and evaluate
// the pairs of one cell while the next is in flight; they hand a stage back
// through a second mbarrier.  Pair arithmetic, thread split and summation
// order are those of k_lj_tile, so both give the same bits.  Every wait is
// bounded: a wait that gives up raises kFlagTimeout and the block returns.
constexpr int kPipeStages = 2;
constexpr int kPipeHomeCap = 256;           // home atoms whose list counts are staged
constexpr unsigned kPipeSpin = 1u << 22;    // try_wait rounds before a wait gives up

struct PipeMeta {
  int c, b, n, total, qmax, tile_ok, staged, ri;
  int off[28];
  int nc[kPipeHomeCap];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// wait for the completion of the phase with this parity; false if it gave up
// after `spins` try_wait rounds
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned spins = kPipeSpin) {
  const unsigned a = smem_u32(bar);
  for (unsigned k = 0; k < spins; ++k) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

template <bool MIXED, bool ENERGY, int NT>
__global__ void __launch_bounds__(NT + 32) k_lj_pipe(const float4* __restrict__ pos, const int* __restrict__ cell_start,
                                                     const uint4* __restrict__ nbr, const int* __restrict__ ncount,
                                                     int Npad, int tile_cap, int list_cap,
                                                     const RepDev* __restrict__ reps, int n_reps, int C,
                                                     const ForceParams fp, void* __restrict__ flj,
                                                     double* __restrict__ epart, unsigned* __restrict__ flags,
                                                     int* __restrict__ work) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* tiles = reinterpret_cast<float4*>(smem);
  uint4* lists = reinterpret_cast<uint4*>(smem + (size_t)kPipeStages * tile_cap * sizeof(float4));
  __shared__ __align__(8) unsigned long long full[kPipeStages], empty[kPipeStages];
  __shared__ PipeMeta meta[kPipeStages];
  __shared__ double red[kEnergyVals][NT / 32];
  __shared__ int abort_all;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    abort_all = 0;
    for (int k = 0; k < kPipeStages; ++k) {
      mbar_init(&full[k], 32);
      mbar_init(&empty[k], NT / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == NT / 32) {
    // ------------------------------------------------------------ producer
    for (int i = 0;; ++i) {
      const int s = i % kPipeStages;
      if (i >= kPipeStages && !mbar_wait(&empty[s], ((i / kPipeStages) - 1) & 1)) {
        if (lane == 0) atomicOr(flags, kFlagTimeout);
        break;
      }
      int c = 0;
      if (lane == 0) c = atomicAdd(work, 1);
      c = __shfl_sync(0xffffffffu, c, 0);
      PipeMeta& M = meta[s];
      if (c >= C) {
        if (lane == 0) M.c = -1;
        mbar_arrive(&full[s]);
        break;
      }
      const int ri = find_rep_cell(reps, n_reps, c);
      const RepDev& R = reps[ri];
      int len = 0, st = 0;
      if (lane < 27) {
        const int M3 = R.M, lc = c - R.cell_base;
        const int cx = lc % M3, cy = (lc / M3) % M3, cz = lc / (M3 * M3);
        const int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
        const int nc = R.cell_base + (((cz + oz + M3) % M3) * M3 + ((cy + oy + M3) % M3)) * M3 + ((cx + ox + M3) % M3);
        st = cell_start[nc];
        len = cell_start[nc + 1] - st;
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane < 27) M.off[lane] = incl - len;
      const int total = __shfl_sync(0xffffffffu, incl, 26);
      if (lane == 0) M.off[27] = total;
      const int b = __shfl_sync(0xffffffffu, st, 13), n = __shfl_sync(0xffffffffu, len, 13);
      int qmax = 0;
      for (int a = lane; a < n && a < kPipeHomeCap; a += 32) {
        const int v = ncount[b + a];
        M.nc[a] = v;
        qmax = max(qmax, v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) qmax = max(qmax, __shfl_xor_sync(0xffffffffu, qmax, o));
      const bool tile_ok = ((total + 32) & ~31) <= tile_cap;
      const bool staged = tile_ok && n <= kPipeHomeCap && n * qmax <= list_cap;
      const unsigned bytes = (tile_ok ? (unsigned)total * 16u : 0u) + (staged ? (unsigned)(n * qmax) * 16u : 0u);
      if (lane == 0) {
        M.c = c; M.b = b; M.n = n; M.total = total; M.qmax = qmax;
        M.tile_ok = tile_ok; M.staged = staged; M.ri = ri;
        if (bytes) mbar_expect_tx(&full[s], bytes);
      }
      __syncwarp();
      if (tile_ok && lane < 27 && len > 0)
        bulk_g2s(tiles + (size_t)s * tile_cap + (incl - len), pos + st, (unsigned)len * 16u, &full[s]);
      if (staged && n > 0)
        for (int q = lane; q < qmax; q += 32)
          bulk_g2s(lists + (size_t)s * list_cap + (size_t)q * n, nbr + (size_t)q * Npad + b, (unsigned)n * 16u,
                   &full[s]);
      mbar_arrive(&full[s]);
    }
    if (lane == 0) {
      __threadfence();
      if (atomicAdd(work + 1, 1) == (int)gridDim.x - 1) {   // last block: reset for the next launch
        work[0] = 0;
        work[1] = 0;
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  // Every consumer warp passes the same named barriers in every round, and a
  // warp whose wait gave up (twice) raises abort_all before the first one, so
  // all consumer warps leave together.
  const int tid = threadIdx.x;
  for (int i = 0;; ++i) {
    const int s = i % kPipeStages;
    const unsigned par = (i / kPipeStages) & 1;
    if (!mbar_wait(&full[s], par)) {
      if (lane == 0) atomicOr(flags, kFlagTimeout);
      if (!mbar_wait(&full[s], par) && lane == 0) atomicExch(&abort_all, 1);
    }
    consumer_sync(NT);
    if (*(volatile int*)&abort_all) break;
    const PipeMeta& M = meta[s];
    const int c = M.c;
    if (c < 0) break;
    const int n = M.n, b = M.b, total = M.total;
    const RepDev& R = reps[M.ri];
    float4* sp = tiles + (size_t)s * tile_cap;
    const uint4* lst = lists + (size_t)s * list_cap;
    float ev[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (n > 0 && M.tile_ok) {
      // move the staged runs into the home cell's frame
      for (int k = warp; k < 27; k += NT / 32) {
        if (k == 13) continue;
        const float ox = (float)(k % 3 - 1), oy = (float)((k / 3) % 3 - 1), oz = (float)(k / 9 - 1);
        for (int t = M.off[k] + lane; t < M.off[k + 1]; t += 32) {
          float4 q = sp[t];
          q.x += ox; q.y += oy; q.z += oz;
          sp[t] = q;
        }
      }
      if (tid == 0) sp[total] = make_float4(1e9f, 1e9f, 1e9f, 0.f);   // sentinel slot
    }
    consumer_sync(NT);
    if (n > 0 && M.tile_ok) {
      const float4* home = sp + M.off[13];
      const bool staged = M.staged;
      const int TP = n > NT / 2 ? 1 : (n > NT / 4 ? 2 : 4);
      const float rc2 = R.rc2u;
      const float ih = R.ih_hi;
      for (int a0 = 0; a0 < n; a0 += NT / TP) {
        const int na = min(NT / TP, n - a0);
        const int a = a0 + tid / TP, p = tid % TP;
        const bool active = a < a0 + na;
        float fx = 0.f, fy = 0.f, fz = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        if (active) {
          const float4 pi = home[a];
          const int ti = pi.w != 0.f ? 1 : 0;
          const float a0c = 12.f * R.C12u[ti], b0c = 6.f * R.C6u[ti];
          const float da = 12.f * R.C12u[ti + 1] - a0c, db = 6.f * R.C6u[ti + 1] - b0c;
          float ec[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // energy coefficients (ENERGY only)
          if (ENERGY) {
            ec[0] = R.C12u[ti]; ec[1] = R.C12u[ti + 1] - ec[0];
            ec[2] = R.C6u[ti]; ec[3] = R.C6u[ti + 1] - ec[2];
            ec[4] = fp.erc[ti][0]; ec[5] = fp.erc[ti][1] - ec[4];
          }
          const int nblk = a < kPipeHomeCap ? M.nc[a] : ncount[b + a];
          const uint4* np = nbr + b + a;
          for (int blk = p; blk < nblk; blk += TP) {
            const uint4 E = staged ? lst[(size_t)blk * n + a] : __ldg(np + (size_t)blk * Npad);
            const unsigned ew[4] = {E.x, E.y, E.z, E.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              lj_pair<ENERGY>(ew[u] & 0xffffu, sp, pi, rc2, a0c, da, b0c, db, ec, fx, fy, fz, ev);
              lj_pair<ENERGY>(ew[u] >> 16, sp, pi, rc2, a0c, da, b0c, db, ec, gx, gy, gz, ev);
            }
          }
        }
        fx += gx; fy += gy; fz += gz;
        // sum the TP partial forces of an atom (adjacent lanes, fixed order)
        if (TP >= 2) {
          fx += __shfl_down_sync(0xffffffffu, fx, 1); fy += __shfl_down_sync(0xffffffffu, fy, 1); fz += __shfl_down_sync(0xffffffffu, fz, 1);
        }
        if (TP >= 4) {
          fx += __shfl_down_sync(0xffffffffu, fx, 2); fy += __shfl_down_sync(0xffffffffu, fy, 2); fz += __shfl_down_sync(0xffffffffu, fz, 2);
        }
        if (active && p == 0) {
          fx *= ih; fy *= ih; fz *= ih;             // back from cell units
          const int sa = b + a;
          if (MIXED) {
            F4i o;
            o.x = fix_of(fx, flags); o.y = fix_of(fy, flags); o.z = fix_of(fz, flags); o.w = 0;
            reinterpret_cast<F4i*>(flj)[sa] = o;
          } else {
            reinterpret_cast<float4*>(flj)[sa] = make_float4(fx, fy, fz, 0.f);
          }
        }
      }
    } else if (n > 0 && tid == 0) {
      atomicOr(flags, kFlagNbrOverflow);
    }
    if (ENERGY) {
      warp_energy_sums(ev, lane, red, warp);
      consumer_sync(NT);
      if (tid == 0) {
        for (int k = 0; k < kEnergyVals; ++k) {
          double sv = 0.0;
          for (int q = 0; q < NT / 32; ++q) sv += red[k][q];
          epart[(size_t)c * kEnergyVals + k] = sv;
        }
      }
    }
    // hand the stage back: order this thread's shared-memory writes before
    // the producer's next bulk copy into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    consumer_sync(NT);
    if (lane == 0) mbar_arrive(&empty[s]);
  }
}

// Self-test of the bounded wait: one thread waits on an mbarrier that nothing
// arrives on, gives up after `spins` rounds and raises kFlagTimeout.
__global__ void __launch_bounds__(32) k_wait_selftest(unsigned spins, unsigned* __restrict__ flags) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0, spins)) atomicOr(flags, kFlagTimeout);
}

void launch_wait_selftest(unsigned spins, unsigned* flags, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(spins, flags);
}

// list rows staged per stage: two blocks per SM when the tile leaves room for
// 1,024 rows, else one block per SM
int lj_pipe_list_cap(int tile_cap) {
  const int two = 3400 - tile_cap;
  return two >= 1024 ? two : 7000 - tile_cap;
}

size_t lj_pipe_smem(int tile_cap) {
  return (size_t)kPipeStages * (tile_cap + lj_pipe_list_cap(tile_cap)) * sizeof(float4);
}

// true if the force kernel compiled for TPS threads per SM keeps TPS / NT
// blocks resident with this tile (shared memory is the other limit)
template <bool MIXED, int NT, int TPS>
static bool lj_tile_fits(int tile_cap) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lj_tile<MIXED, false, NT, TPS>, NT,
                                                    (size_t)tile_cap * sizeof(float4)) != cudaSuccess)
    return false;
  return nb >= TPS / NT;
}

template <bool MIXED, bool ENERGY, int NT>
static void lj_launch(bool pipe, int grid, int tile_cap, cudaStream_t st, const float4* pos, const int* tag,
                      const int* cell_start, const uint4* nbr, const int* ncount, int Npad, const RepDev* reps,
                      int n_reps, int C, const ForceParams& fp, void* flj, double* epart, unsigned* flags, int* work) {
  if (pipe)
    k_lj_pipe<MIXED, ENERGY, NT><<<grid, NT + 32, lj_pipe_smem(tile_cap), st>>>(
        pos, cell_start, nbr, ncount, Npad, tile_cap, lj_pipe_list_cap(tile_cap), reps, n_reps, C, fp, flj, epart,
        flags, work);
  else {
    const size_t sm = (size_t)tile_cap * sizeof(float4);
    if constexpr (!ENERGY) {
      if (lj_tile_fits<MIXED, NT, 1536>(tile_cap)) {
        k_lj_tile<MIXED, false, NT, 1536><<<C, NT, sm, st>>>(pos, tag, cell_start, nbr, ncount, Npad, tile_cap, reps,
                                                             n_reps, fp, flj, epart, flags);
        return;
      }
      if (lj_tile_fits<MIXED, NT, 1024>(tile_cap)) {
        k_lj_tile<MIXED, false, NT, 1024><<<C, NT, sm, st>>>(pos, tag, cell_start, nbr, ncount, Npad, tile_cap, reps,
                                                             n_reps, fp, flj, epart, flags);
        return;
      }
    }
    k_lj_tile<MIXED, ENERGY, NT, 0><<<C, NT, (size_t)tile_cap * sizeof(float4), st>>>(
        pos, tag, cell_start, nbr, ncount, Npad, tile_cap, reps, n_reps, fp, flj, epart, flags);
  }
}

// persistent_grid > 0: the pipelined kernel on that many blocks; else one
// block per cell
void launch_lj_tile(bool mixed, bool energy, const float4* pos, const int* tag, const int* cell_start,
                    const uint4* nbr, const int* ncount, int Npad, int tile_cap, const RepDev* reps, int n_reps, int C,
                    const ForceParams& fp, void* flj, double* epart, unsigned* flags, int block, int persistent_grid,
                    int* work, cudaStream_t st) {
  const bool pipe = persistent_grid > 0;
#define MDG_LJ(M, E, NT) lj_launch<M, E, NT>(pipe, persistent_grid, tile_cap, st, pos, tag, cell_start, nbr, ncount, Npad, reps, n_reps, C, fp, flj, epart, flags, work)
#define MDG_LJ2(NT) \
  if (mixed) { if (energy) MDG_LJ(true, true, NT); else MDG_LJ(true, false, NT); } \
  else { if (energy) MDG_LJ(false, true, NT); else MDG_LJ(false, false, NT); }
  if (block == 128) { MDG_LJ2(128) } else { MDG_LJ2(256) }
#undef MDG_LJ2
#undef MDG_LJ
}

// resident blocks per SM of the pipelined LJ kernel for a block size and tile
int lj_blocks_per_sm(int block, int tile_cap) {
  int nb = 0;
  const size_t sm = lj_pipe_smem(tile_cap);
  if (block == 128)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lj_pipe<true, false, 128>, 128 + 32, sm);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lj_pipe<true, false, 256>, 256 + 32, sm);
  return nb;
}

// Opt in to more than 48 KB of dynamic shared memory (once per device); the
// attribute is an upper bound, set for the largest tile accepted.
cudaError_t tile_kernels_init() {
  const int mx = kStageCapMax * sizeof(float4);
  const int mp = (int)lj_pipe_smem(kStageCapMax);
  cudaError_t e = cudaFuncSetAttribute(k_nbr_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
#define MDG_ATTR(M, E, NT) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lj_tile<M, E, NT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess && !E) e = cudaFuncSetAttribute(k_lj_tile<M, false, NT, 1536>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess && !E) e = cudaFuncSetAttribute(k_lj_tile<M, false, NT, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_lj_pipe<M, E, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, mp);
#define MDG_ATTR4(NT) MDG_ATTR(true, true, NT) MDG_ATTR(true, false, NT) MDG_ATTR(false, true, NT) MDG_ATTR(false, false, NT)
  MDG_ATTR4(128) MDG_ATTR4(256)
#undef MDG_ATTR4
#undef MDG_ATTR
  return e;
}

int tile_capacity_max() { return kStageCapMax; }

}  // namespace mdg
