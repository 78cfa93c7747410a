// k_lj.cu -- neighbour list (Sec. 3.1) and Lennard-Jones force (Eq. 2,
// Sec. 3.2) with every pair evaluated once (Newton's third law).
//
// Work unit: a region of up to G x G x 1 cells (G = 2 or 3; cells of side
// >= r_c + skin, Sec. 3.1), one thread block per region.  The block stages in
// shared memory the "tile": the region's cells and every cell that one of
// them reaches by one of the 13 forward offsets of a half shell (27 cells
// for G = 2, 44 for G = 3), each cell a contiguous run of sorted atoms, moved
// into the region's frame: w = u + (cell offset - region centre) in cell
// units, |w| < 3.  The paper's
// neighbour-search kernel also assigns a block to grid cells and stages the
// neighbour cells (Sec. 3.1, last paragraph); here the same staging serves
// the force kernel, and the list holds indices into the staged tile.
//
// Clusters: the atoms of a cell, in their sorted order (by atom index, so
// consecutive sites of a chain), are grouped four at a time; cluster k of
// cell c holds sorted slots cell_start[c] + 4k .. + 3.  Each cluster owns the
// pairs it forms with later clusters of its cell and with the 13 forward
// cells, so every pair of the periodic system belongs to exactly one
// cluster (cells per side >= 3).  The list of a cluster holds the tile atoms
// j that lie within r_c + skin of at least one of its atoms, each with a
// 4-bit mask of the atoms i that pair with j: within r_c + skin, not a 1-2 or
// 1-3 neighbour (Sec. 3.1) and, inside the cluster, i before j.
//
// Force: a warp takes 32/LP clusters at a time (LP lanes each); each lane
// evaluates list entries against its cluster's four atoms i (r2inv = 0
// beyond r_c, as in the Sec. 3.2 listing).  The force on i is
// summed in FP32 registers in list order and reduced over the lanes by a
// fixed xor tree; the force on j of one entry (at most four pairs, summed in
// FP32) is converted once to 2^-13 kJ/mol/nm fixed point and added to the
// tile's int32 accumulators in shared memory; at the end each tile atom's
// accumulator is added to the int64 force (2^-32 kJ/mol/nm) with one
// integer atomic per component.  Integer sums do not depend on the order in
// which they are made, so the forces are deterministic.
#include <type_traits>

#include "md_kernels.cuh"

namespace mdg {

constexpr int kStageCapMax = 6144;      // largest tile (atoms); list entries keep the tile index in 16 bits
constexpr int kLjAccShift = 19;         // 2^-13 accumulators -> 2^-32 fixed point
constexpr float kLjAccScale = 8192.0f;  // 2^13

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The staged tile of one region: for each tile cell k its first sorted slot,
// its first position in the tile (off[n_tile] = tile size) and its frame shift.
struct RegTile {
  int start[kMaxTileCells];
  int off[kMaxTileCells + 1];
  float sx[kMaxTileCells], sy[kMaxTileCells], sz[kMaxTileCells];
  int ncl[kMaxHome + 1];          // clusters of home cells before h (ncl[n_home] = all)
  int cl0[kMaxHome];              // global id of home cell h's first cluster
  int home_cell[kMaxHome];        // global id of home cell h
  int cnt[kMaxTileCells];         // atoms of tile cell k (set-up scratch)
  int n_tile, n_home;
};

// Threads 0..63 read the tile cells' bounds, then one warp scans the counts
// (two cells per lane: up to 64 tile cells); needs NT >= 64.
__device__ __forceinline__ void region_setup(RegTile& T, const Region& g, const RegionShape& S, const RepDev& R,
                                             const int* __restrict__ cell_start, const int* __restrict__ cl_start) {
  const int k = threadIdx.x;
  if (k < kMaxTileCells) {
    int n = 0;
    if (k < S.n_tile) {
      const int M = R.M;
      const int cx = (g.ox + S.off[k][0] + M) % M, cy = (g.oy + S.off[k][1] + M) % M, cz = (g.oz + S.off[k][2] + M) % M;
      const int c = R.cell_base + (cz * M + cy) * M + cx;
      T.start[k] = cell_start[c];
      n = cell_start[c + 1] - T.start[k];
      T.sx[k] = (float)S.off[k][0] - S.cx;
      T.sy[k] = (float)S.off[k][1] - S.cy;
      T.sz[k] = (float)S.off[k][2] - S.cz;
      if (k < S.n_home) {
        T.home_cell[k] = c;
        T.cl0[k] = cl_start[c];
      }
    }
    T.cnt[k] = n;
  }
  __syncthreads();
  if (k < 32) {
    const int a = T.cnt[2 * k], b = T.cnt[2 * k + 1];
    int incl = a + b;
    // clusters of the home cells (ceil(n / 4) each); home cells come first
    const int ca = 2 * k < S.n_home ? (a + 3) >> 2 : 0, cb = 2 * k + 1 < S.n_home ? (b + 3) >> 2 : 0;
    int ci = ca + cb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o), w = __shfl_up_sync(0xffffffffu, ci, o);
      if (k >= o) { incl += v; ci += w; }
    }
    const int ex = incl - a - b, cx = ci - ca - cb;
    if (2 * k < S.n_tile) T.off[2 * k] = ex;
    if (2 * k + 1 < S.n_tile) T.off[2 * k + 1] = ex + a;
    if (2 * k < S.n_home) T.ncl[2 * k] = cx;
    if (2 * k + 1 < S.n_home) T.ncl[2 * k + 1] = cx + ca;
    if (k == 31) {
      T.off[S.n_tile] = incl;
      T.ncl[S.n_home] = ci;
      T.n_tile = S.n_tile;
      T.n_home = S.n_home;
    }
  }
  __syncthreads();
}

// Copy the tile into shared memory in the region frame.  Warps take tile
// cells in turn and their lanes start asynchronous copies (cp.async, global
// to shared without registers) of the cell's atoms, so the whole tile is in
// flight at once; after the wait and a barrier, a warp per tile cell adds
// the cell's frame shift.  The w component keeps the LJ type
// (0.0 / 1.0) that binning and integration store; WITH_TAG (list build)
// replaces it by the bits of the atom's chain/site tag, which the build
// needs instead.  tile_issue starts the copies, tile_finish waits for them,
// shifts, and ends with a barrier.
template <int NT>
__device__ __forceinline__ void tile_issue(const RegTile& T, const float4* __restrict__ pos, float4* __restrict__ sp) {
  const int nt = T.n_tile, lane = threadIdx.x & 31;
  for (int k = threadIdx.x >> 5; k < nt; k += NT / 32) {
    const int t0 = T.off[k], n = T.off[k + 1] - t0;
    const float4* src = pos + T.start[k];
    const unsigned dst = (unsigned)__cvta_generic_to_shared(sp + t0);
    for (int q = lane; q < n; q += 32)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16u * (unsigned)q), "l"(src + q)
                   : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <bool WITH_TAG, int NT>
__device__ __forceinline__ void tile_finish(const RegTile& T, float4* __restrict__ sp, const int* __restrict__ tag) {
  const int nt = T.n_tile;
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x >> 5; k < nt; k += NT / 32) {
    const int t0 = T.off[k], n = T.off[k + 1] - t0, j0 = T.start[k];
    const float ox = T.sx[k], oy = T.sy[k], oz = T.sz[k];
    for (int q = lane; q < n; q += 32) {
      float4 p = sp[t0 + q];
      p.x += ox; p.y += oy; p.z += oz;
      if (WITH_TAG) p.w = __int_as_float(__ldg(tag + j0 + q) & (int)kTagMask);
      sp[t0 + q] = p;
    }
  }
  __syncthreads();
}

// home cluster q of the region -> (home cell h, cluster k within the cell)
__device__ __forceinline__ void cluster_of(const RegTile& T, int q, int& h, int& k) {
  h = 0;
  while (h + 1 < T.n_home && T.ncl[h + 1] <= q) ++h;
  k = q - T.ncl[h];
}

// next region of this block: blockIdx.x once (grid schedule), or from the
// work counter (persistent schedule); shared broadcast
__device__ __forceinline__ int next_region(bool persistent, int it, int* work, int* sh) {
  if (!persistent) return it == 0 ? (int)blockIdx.x : -1;
  __syncthreads();
  if (threadIdx.x == 0) *sh = atomicAdd(work, 1);
  __syncthreads();
  return *sh;
}

// the last block of a persistent launch resets the counters for the next one
__device__ __forceinline__ void persistent_done(int* work) {
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(work + 1, 1) == (int)gridDim.x - 1) {
      work[0] = 0;
      work[1] = 0;
    }
  }
}

// ===================================================================== build
// One warp per home cluster.  Candidates j are the later atoms of the
// cluster's own cell and the atoms of its 13 forward cells.  Each j is tested
// against the cluster's four atoms i (within r_c + skin, not a 1-2 or 1-3
// neighbour, and for the own cell i before j); a j with a non-empty mask is
// appended to the cluster's list in candidate order (ballot + prefix count,
// so the list is the same on every run).  The forward cells' candidates
// first pass a cheap test against a sphere around the cluster (centre c,
// radius rad: |j - c| < r_list + rad holds for every j that can pair); those
// that pass are queued per warp in shared memory and tested 32 at a time,
// so the lanes of a warp run the four-atom test on candidates that may pair
// rather than on every 32nd atom of the tile.
constexpr int kBuildQueue = 64;

// is atom b of a molecule a 1-2 or 1-3 neighbour of atom a (general type)?
__device__ __forceinline__ bool topo_excluded(int a, int b, const TopoDev& tp) {
  for (int q = tp.x_off[a]; q < tp.x_off[a + 1]; ++q)
    if (tp.x_at[q] == b) return true;
  return a == b;
}

// the four-atom test of candidate t: bit u set if atom u of the cluster pairs with t
template <bool GEN>
__device__ __forceinline__ unsigned pair_mask(const float4 (&pi)[4], const int (&ti)[4], const float4& w, float rl2,
                                              const TopoDev& tp) {
  const int tg = __float_as_int(w.w);   // the candidate's tag (list-build tile)
  unsigned m = 0u;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const float dx = pi[u].x - w.x, dy = pi[u].y - w.y, dz = pi[u].z - w.z;
    bool keep = dx * dx + dy * dy + dz * dz < rl2;
    if (GEN) {
      // same molecule: its exclusion list (Sec. 3.1, t_exclusions)
      if (keep && ((ti[u] ^ tg) >> kTagSiteBits) == 0)
        keep = !topo_excluded(ti[u] & ((1 << kTagSiteBits) - 1), tg & ((1 << kTagSiteBits) - 1), tp);
    } else {
      // |i - j| <= 2 within one chain: 1-2 and 1-3 neighbours (and i itself)
      keep &= (unsigned)(ti[u] - tg + 2) > 4u;
    }
    m |= keep ? (1u << u) : 0u;
  }
  return m;
}

template <int NT, bool GEN>
__global__ void __launch_bounds__(NT, 1024 / NT) k_cl_build(const float4* __restrict__ pos, const int* __restrict__ tag,
                                                 const int* __restrict__ cell_start, const int* __restrict__ cl_start,
                                                 const Region* __restrict__ regions, int n_regions,
                                                 const RegionShape* __restrict__ shapes, const RepDev* __restrict__ reps,
                                                 unsigned* __restrict__ list, int* __restrict__ ncl, int cap,
                                                 int tile_cap, unsigned* __restrict__ flags, int persistent,
                                                 int* __restrict__ work, const TopoDev tp) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sp = reinterpret_cast<float4*>(smem);   // w: the atom's chain/site tag bits
  __shared__ RegTile T;
  __shared__ int sh_r;
  __shared__ int queue[NT / 32][kBuildQueue];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* qw = queue[warp];
  for (int it = 0;; ++it) {
    const int r = next_region(persistent != 0, it, work, &sh_r);
    if (r < 0 || r >= n_regions) break;
    const Region g = regions[r];
    const RegionShape& S = shapes[g.shape];
    const RepDev& R = reps[g.rep];
    __syncthreads();   // the previous region's tile is no longer read
    region_setup(T, g, S, R, cell_start, cl_start);
    const int total = T.off[T.n_tile];
    if (total > tile_cap) {
      if (threadIdx.x == 0) atomicOr(flags, kFlagNbrOverflow);
      for (int q = threadIdx.x; q < T.ncl[T.n_home]; q += NT) {
        int h, k;
        cluster_of(T, q, h, k);
        ncl[T.cl0[h] + k] = 0;
      }
      continue;
    }
    tile_issue<NT>(T, pos, sp);
    tile_finish<true, NT>(T, sp, tag);
    const float rl2 = R.rlist2u;
    const float rl = sqrtf(rl2);
    const unsigned lt = (1u << lane) - 1u;
    for (int q = warp; q < T.ncl[T.n_home]; q += NT / 32) {
      int h, k;
      cluster_of(T, q, h, k);
      const int i0 = T.off[h] + 4 * k;
      const int ni = min(4, T.off[h + 1] - i0);
      float4 pi[4];
      int ti[4];
      float cx = 0.f, cy = 0.f, cz = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int t = i0 + min(u, ni - 1);
        pi[u] = sp[t];
        ti[u] = __float_as_int(pi[u].w);
        cx += pi[u].x; cy += pi[u].y; cz += pi[u].z;
      }
      cx *= 0.25f; cy *= 0.25f; cz *= 0.25f;
      float rad2 = 0.f;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float dx = pi[u].x - cx, dy = pi[u].y - cy, dz = pi[u].z - cz;
        rad2 = fmaxf(rad2, dx * dx + dy * dy + dz * dz);
        // a slot past the cell's last atom gets a far position: it pairs with nothing
        if (u >= ni) pi[u] = make_float4(1e9f, 1e9f, 1e9f, 0.f);
      }
      // the sphere test is taken with a margin of 1e-5 cell units over the
      // FP32 roundings of c and rad, so it never rejects a pair the exact
      // test keeps
      const float reach = rl + sqrtf(rad2) + 1e-5f;
      const float reach2 = reach * reach;
      const int cl = T.cl0[h] + k;
      unsigned* out = list + (size_t)cl * cap;
      int cnt = 0;
      // own cell, from the cluster on: each pair once, i before j
      {
        const int t_end = T.off[h + 1];
        for (int t0 = i0; t0 < t_end; t0 += 32) {
          const int t = t0 + lane;
          unsigned m = 0u;
          if (t < t_end) {
            m = pair_mask<GEN>(pi, ti, sp[t], rl2, tp);
            m &= ((t > i0) ? 1u : 0u) | ((t > i0 + 1) ? 2u : 0u) | ((t > i0 + 2) ? 4u : 0u) | ((t > i0 + 3) ? 8u : 0u);
          }
          const unsigned b = __ballot_sync(0xffffffffu, m != 0u);
          const int p = cnt + __popc(b & lt);
          if (m != 0u && p < cap) out[p] = (unsigned)t | (m << 16);
          cnt += __popc(b);
        }
      }
      // the 13 forward cells: sphere test, queue, four-atom test 32 at a time
      int qn = 0;
      for (int c14 = 1; c14 < 14; ++c14) {
        const int tc = S.nb[h][c14];
        const int t_end = T.off[tc + 1];
        for (int t0 = T.off[tc]; t0 < t_end; t0 += 32) {
          const int t = t0 + lane;
          bool pass = false;
          if (t < t_end) {
            const float4 w = sp[t];
            const float dx = w.x - cx, dy = w.y - cy, dz = w.z - cz;
            pass = dx * dx + dy * dy + dz * dz < reach2;
          }
          const unsigned b = __ballot_sync(0xffffffffu, pass);
          if (pass) qw[qn + __popc(b & lt)] = t;
          qn += __popc(b);
          __syncwarp();
          if (qn >= 32) {
            const int tq = qw[lane];
            const unsigned m = pair_mask<GEN>(pi, ti, sp[tq], rl2, tp);
            const unsigned bm = __ballot_sync(0xffffffffu, m != 0u);
            const int p = cnt + __popc(bm & lt);
            if (m != 0u && p < cap) out[p] = (unsigned)tq | (m << 16);
            cnt += __popc(bm);
            const int rest = qn - 32;
            const int moved = lane < rest ? qw[32 + lane] : 0;
            __syncwarp();
            if (lane < rest) qw[lane] = moved;
            __syncwarp();
            qn = rest;
          }
        }
      }
      if (qn > 0) {
        unsigned m = 0u;
        int tq = 0;
        if (lane < qn) {
          tq = qw[lane];
          m = pair_mask<GEN>(pi, ti, sp[tq], rl2, tp);
        }
        const unsigned bm = __ballot_sync(0xffffffffu, m != 0u);
        const int p = cnt + __popc(bm & lt);
        if (m != 0u && p < cap) out[p] = (unsigned)tq | (m << 16);
        cnt += __popc(bm);
      }
      __syncwarp();
      if (lane == 0) {
        ncl[cl] = min(cnt, cap);
        if (cnt > cap) atomicOr(flags, kFlagNbrOverflow);
      }
    }
  }
  if (persistent) persistent_done(work);
}

// ===================================================================== force
constexpr int kEnergyVals = 8;           // lj, lj_shifted, vxx, vyy, vzz, vxy, vxz, vyz
constexpr int kRegionClusterCap = 512;   // clusters of one region (2,048 home atoms); more is reported

// FP32 force (cell units) -> fixed point 2^-13 kJ/mol/nm; F2I saturates
// beyond +-2^31 (2^18 kJ/mol/nm)
__device__ __forceinline__ int acc_fix(float f) { return __float2int_rn(f); }

// a converted component at or beyond 2^30 (2^17 kJ/mol/nm, half the int32
// range of the tile accumulators) or not finite is reported
__device__ __forceinline__ void range_check(float sx, float sy, float sz, unsigned* flags) {
  const float a = fmaxf(fabsf(sx), fmaxf(fabsf(sy), fabsf(sz)));
  const bool finite = (sx - sx) == 0.f && (sy - sy) == 0.f && (sz - sz) == 0.f;
  if (!finite) atomicOr(flags, kFlagNaN);
  else if (!(a < 1073741824.0f)) atomicOr(flags, kFlagFixOverflow);
}

constexpr float kMagic = 12582912.0f;   // 1.5 2^23: FP32 spacing 1 in [2^23, 2^24)
constexpr unsigned kMagicBits = 0x4B400000u;

// Add the force g (cell units) on tile atom t to the 2^-13 accumulators.
// While |g| scale < 2^22 (|g| < 512 kJ/mol/nm, the usual case) the
// conversion is one FFMA: g scale + 1.5 2^23 lies in [2^23, 2^24), where
// the FP32 spacing is 1, so the sum rounds g scale to the nearest integer
// (ties to even) and its low mantissa bits are that integer plus 2^22; the
// integer subtraction removes the offset.  Larger (or non-finite) values
// take the FMUL + F2I path with the range check.  lim = 2^22 / scale.
__device__ __forceinline__ void acc_add(int* __restrict__ ax, int* __restrict__ ay, int* __restrict__ az, int t,
                                        float gx, float gy, float gz, float scale, float lim,
                                        unsigned* __restrict__ flags) {
  if (fabsf(gx) + fabsf(gy) + fabsf(gz) < lim) {
    atomicAdd(ax + 3 * t, __float_as_int(fmaf(gx, scale, kMagic)) - (int)kMagicBits);
    atomicAdd(ay + 3 * t, __float_as_int(fmaf(gy, scale, kMagic)) - (int)kMagicBits);
    atomicAdd(az + 3 * t, __float_as_int(fmaf(gz, scale, kMagic)) - (int)kMagicBits);
  } else {
    gx *= scale; gy *= scale; gz *= scale;
    range_check(gx, gy, gz, flags);
    atomicAdd(ax + 3 * t, acc_fix(gx));
    atomicAdd(ay + 3 * t, acc_fix(gy));
    atomicAdd(az + 3 * t, acc_fix(gz));
  }
}

// One list entry against the cluster's four atoms with packed FP32 pairs
// (two atoms per float2 lane: 0,1 and 2,3; one FFMA2 does both): the force
// on the four atoms is added to f*[2] and minus the force on j, summed over
// the four atoms, is returned in g* (rcp of r^2; r2inv = 0 beyond r_c or
// outside the mask).  A[p], nB[p]:
// the pair coefficients 12 C12 and -6 C6 of atoms 2p, 2p+1 with j.
__device__ __forceinline__ void entry_packed(const float2 (&px)[2], const float2 (&py)[2], const float2 (&pz)[2],
                                             const float2 (&A)[2], const float2 (&nB)[2], float rc2, const float4& w,
                                             unsigned m, float2 (&fx)[2], float2 (&fy)[2], float2 (&fz)[2], float& gx,
                                             float& gy, float& gz) {
  const float2 wx = make_float2(-w.x, -w.x), wy = make_float2(-w.y, -w.y), wz = make_float2(-w.z, -w.z);
  float2 sx = make_float2(0.f, 0.f), sy = make_float2(0.f, 0.f), sz = make_float2(0.f, 0.f);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 dx = __fadd2_rn(px[p], wx), dy = __fadd2_rn(py[p], wy), dz = __fadd2_rn(pz[p], wz);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float q0 = rcp_approx(r2.x), q1 = rcp_approx(r2.y);
    const bool k0 = ((m >> (2 * p)) & 1u) && r2.x < rc2, k1 = ((m >> (2 * p + 1)) & 1u) && r2.y < rc2;
    const float2 ir2 = make_float2(k0 ? q0 : 0.f, k1 ? q1 : 0.f);
    const float2 ir4 = __fmul2_rn(ir2, ir2), ir6 = __fmul2_rn(ir4, ir2), ir8 = __fmul2_rn(ir4, ir4);
    const float2 ff = __fmul2_rn(ir8, __ffma2_rn(A[p], ir6, nB[p]));
    fx[p] = __ffma2_rn(ff, dx, fx[p]);
    fy[p] = __ffma2_rn(ff, dy, fy[p]);
    fz[p] = __ffma2_rn(ff, dz, fz[p]);
    sx = __ffma2_rn(ff, dx, sx);
    sy = __ffma2_rn(ff, dy, sy);
    sz = __ffma2_rn(ff, dz, sz);
  }
  gx = -(sx.x + sx.y);
  gy = -(sy.x + sy.y);
  gz = -(sz.x + sz.y);
}

// Pairwise fixed-point form of entry_packed: each pair's force component v
// (the coefficients A, nB carry the 2^13 accumulator scale, so v is in
// 2^-13 kJ/mol/nm) is rounded once to the nearest integer and that integer
// is added to atom i's sum qi and subtracted from j's (returned in j*), so
// the two atoms receive exactly opposite integers.  The rounding is exact
// in FP32 for |v| < 2^30: hi = rint(v / 2^8) by one FFMA with the 1.5 2^23
// offset (t = hi + offset, in [2^23, 2^24) where the spacing is 1); the
// remainder v - 2^8 hi (|.| <= 2^7, a multiple of v's spacing) is exact in
// one FFMA and rounded by the same offset; rint(v) = 2^8 hi + rint(rem)
// (2^8 hi is an even integer, so ties go the same way).  The integer is
// taken as (bits(t) << 8) + bits(rem + offset), which is rint(v) plus the
// constant kExactOff; qi and the j sums carry one kExactOff per addition,
// which the caller removes by counting.  |v| >= 2^30 (2^17 kJ/mol/nm, the
// range checked by the default path) or a non-finite v leaves t outside
// [2^23, 2^24) and sets bit 23 or above of `chk`.
constexpr unsigned kExactOff = (kMagicBits << 8) + kMagicBits;
__device__ __forceinline__ void exact_round(float2 v, unsigned& b0, unsigned& b1, unsigned& chk) {
  const float2 mg = make_float2(kMagic, kMagic), nmg = make_float2(-kMagic, -kMagic);
  const float2 t = __ffma2_rn(v, make_float2(0.00390625f, 0.00390625f), mg);   // hi + offset
  const float2 hi = __fadd2_rn(t, nmg);
  const float2 lo = __fadd2_rn(__ffma2_rn(hi, make_float2(-256.f, -256.f), v), mg);
  const unsigned t0 = __float_as_uint(t.x), t1 = __float_as_uint(t.y);
  chk |= (t0 ^ kMagicBits) | (t1 ^ kMagicBits);
  b0 = (t0 << 8) + __float_as_uint(lo.x);
  b1 = (t1 << 8) + __float_as_uint(lo.y);
}
__device__ __forceinline__ void entry_packed_exact(const float2 (&px)[2], const float2 (&py)[2],
                                                   const float2 (&pz)[2], const float2 (&A)[2], const float2 (&nB)[2],
                                                   float rc2, const float4& w, unsigned m, unsigned (&qi)[4][3],
                                                   unsigned& jx, unsigned& jy, unsigned& jz, unsigned& chk) {
  const float2 wx = make_float2(-w.x, -w.x), wy = make_float2(-w.y, -w.y), wz = make_float2(-w.z, -w.z);
  unsigned sx = 0u, sy = 0u, sz = 0u;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 dx = __fadd2_rn(px[p], wx), dy = __fadd2_rn(py[p], wy), dz = __fadd2_rn(pz[p], wz);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float q0 = rcp_approx(r2.x), q1 = rcp_approx(r2.y);
    const bool k0 = ((m >> (2 * p)) & 1u) && r2.x < rc2, k1 = ((m >> (2 * p + 1)) & 1u) && r2.y < rc2;
    const float2 ir2 = make_float2(k0 ? q0 : 0.f, k1 ? q1 : 0.f);
    const float2 ir4 = __fmul2_rn(ir2, ir2), ir6 = __fmul2_rn(ir4, ir2), ir8 = __fmul2_rn(ir4, ir4);
    const float2 ff = __fmul2_rn(ir8, __ffma2_rn(A[p], ir6, nB[p]));
    unsigned bx0, bx1, by0, by1, bz0, bz1;
    exact_round(__fmul2_rn(ff, dx), bx0, bx1, chk);
    exact_round(__fmul2_rn(ff, dy), by0, by1, chk);
    exact_round(__fmul2_rn(ff, dz), bz0, bz1, chk);
    qi[2 * p][0] += bx0; qi[2 * p + 1][0] += bx1;
    qi[2 * p][1] += by0; qi[2 * p + 1][1] += by1;
    qi[2 * p][2] += bz0; qi[2 * p + 1][2] += bz1;
    sx += bx0 + bx1; sy += by0 + by1; sz += bz0 + bz1;
  }
  // j: minus the four pairs' integers (four offsets removed)
  jx = 4u * kExactOff - sx;
  jy = 4u * kExactOff - sy;
  jz = 4u * kExactOff - sz;
}

// Energy form: one list entry against the cluster's four atoms, packed as
// in entry_packed, adding the pair energies, the cutoff shifts of the kept
// pairs and the virial terms r (x) f to ev2[8] (two FP32 halves each); no
// force is accumulated (the energy read-out needs none).  cA[p] etc.: the
// pair coefficients C12, C6 and E(r_c) of atoms 2p, 2p+1 with j.
__device__ __forceinline__ void entry_packed_energy(const float2 (&px)[2], const float2 (&py)[2],
                                                    const float2 (&pz)[2], const float2 (&c12)[2],
                                                    const float2 (&c6)[2], const float2 (&sh)[2], float rc2,
                                                    const float4& w, unsigned m, float2 (&ev2)[kEnergyVals]) {
  const float2 wx = make_float2(-w.x, -w.x), wy = make_float2(-w.y, -w.y), wz = make_float2(-w.z, -w.z);
  const float2 k12 = make_float2(12.f, 12.f), km6 = make_float2(-6.f, -6.f);
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    const float2 dx = __fadd2_rn(px[p], wx), dy = __fadd2_rn(py[p], wy), dz = __fadd2_rn(pz[p], wz);
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const float q0 = rcp_approx(r2.x), q1 = rcp_approx(r2.y);
    const bool k0 = ((m >> (2 * p)) & 1u) && r2.x < rc2, k1 = ((m >> (2 * p + 1)) & 1u) && r2.y < rc2;
    const float2 ir2 = make_float2(k0 ? q0 : 0.f, k1 ? q1 : 0.f);
    const float2 ir4 = __fmul2_rn(ir2, ir2), ir6 = __fmul2_rn(ir4, ir2), ir8 = __fmul2_rn(ir4, ir4);
    // F/r = r^-8 (12 C12 r^-6 - 6 C6), E = r^-6 (C12 r^-6 - C6)
    const float2 ff = __fmul2_rn(ir8, __ffma2_rn(__fmul2_rn(k12, c12[p]), ir6, __fmul2_rn(km6, c6[p])));
    const float2 e = __fmul2_rn(ir6, __ffma2_rn(c12[p], ir6, make_float2(-c6[p].x, -c6[p].y)));
    ev2[0] = __fadd2_rn(ev2[0], e);
    ev2[1] = __fadd2_rn(ev2[1], make_float2(k0 ? sh[p].x : 0.f, k1 ? sh[p].y : 0.f));
    const float2 fx = __fmul2_rn(ff, dx), fy = __fmul2_rn(ff, dy);
    ev2[2] = __ffma2_rn(fx, dx, ev2[2]);
    ev2[3] = __ffma2_rn(fy, dy, ev2[3]);
    ev2[4] = __ffma2_rn(__fmul2_rn(ff, dz), dz, ev2[4]);
    ev2[5] = __ffma2_rn(fx, dy, ev2[5]);
    ev2[6] = __ffma2_rn(fx, dz, ev2[6]);
    ev2[7] = __ffma2_rn(fy, dz, ev2[7]);
  }
}

// Per-replica constants of the force evaluation (cell units).
struct LjConst {
  float rc2, scale, lim;
  float A0, A1, A2, B0, B1, B2;   // 12 C12 and 6 C6 by type sum (C32-C32, C32-C33, C33-C33)
};
__device__ __forceinline__ LjConst lj_const(const RepDev& R) {
  LjConst c;
  c.rc2 = R.rc2u;
  c.scale = R.ih_hi * kLjAccScale;     // cell-unit force -> 2^-13 kJ/mol/nm
  c.lim = 4194304.0f / c.scale;        // 2^22 accumulator units
  c.A0 = 12.f * R.C12u[0]; c.A1 = 12.f * R.C12u[1]; c.A2 = 12.f * R.C12u[2];
  c.B0 = 6.f * R.C6u[0]; c.B1 = 6.f * R.C6u[1]; c.B2 = 6.f * R.C6u[2];
  return c;
}

// One warp task: clusters s_ord[q0 .. q0 + 32/LP) of the region, LP lanes
// each; lane l of a cluster's group takes entries l, l + LP, ...  The warp's
// trip count is that of its longest cluster; a lane past its own list idles.
template <bool ENERGY, int LP, bool EXACT = false>
__device__ __forceinline__ void cluster_task(int q0, int nq, const RegTile& T, const float4* __restrict__ sp,
                                             int* __restrict__ ax, int* __restrict__ ay, int* __restrict__ az,
                                             const int* __restrict__ s_key, const short* __restrict__ s_ord,
                                             const int* __restrict__ s_cl, const int* __restrict__ s_in,
                                             float (*__restrict__ ecl)[kEnergyVals], const unsigned* __restrict__ list,
                                             int cap, const RepDev& R, const ForceParams& fp, const LjConst& c,
                                             unsigned* __restrict__ flags) {
  static_assert(LP == 8 || LP == 16 || LP == 32, "lanes per cluster: 8, 16 or 32");
  const int lane = threadIdx.x & 31, sub = lane / LP, sl = lane % LP;
  const float rc2 = c.rc2, scale = c.scale, lim = c.lim;
  // EXACT: the coefficients carry the accumulator scale (pair forces in
  // accumulator units, rounded per pair)
  const float cs = EXACT ? scale : 1.f;
  const float A0 = c.A0 * cs, A1 = c.A1 * cs, A2 = c.A2 * cs, B0 = c.B0 * cs, B1 = c.B1 * cs, B2 = c.B2 * cs;
  const bool valid = q0 + sub < nq;
  const int q = valid ? (int)s_ord[q0 + sub] : nq;
  const int in = s_in[valid ? q : nq - 1];   // first tile atom << 7 | chain-end bits << 3 | atoms
  const int i0 = in >> 7;
  const int ni = valid ? (in & 7) : 0;
  const int n = valid ? s_key[q] >> 9 : 0;
  // the task's clusters are consecutive in longest-first order: the first is the longest
  const int nmax = s_key[s_ord[q0]] >> 9;
  float4 pi[4];   // w: LJ type (1.0 for a C_33 chain end)
#pragma unroll
  for (int u = 0; u < 4; ++u) pi[u] = sp[i0 + max(0, min(u, ni - 1))];
  float fi[4][3];
#pragma unroll
  for (int u = 0; u < 4; ++u) fi[u][0] = fi[u][1] = fi[u][2] = 0.f;
  float ev[kEnergyVals] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  // packed copies for the force-only form (atoms 0,1 and 2,3)
  float2 px[2], py[2], pz[2];
  float2 qx[2], qy[2], qz[2];
  unsigned qi[4][3];   // EXACT: the cluster atoms' integer sums, with one offset per addition
  unsigned chk = 0u;
#pragma unroll
  for (int u = 0; u < 4; ++u) qi[u][0] = qi[u][1] = qi[u][2] = 0u;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    px[p] = make_float2(pi[2 * p].x, pi[2 * p + 1].x);
    py[p] = make_float2(pi[2 * p].y, pi[2 * p + 1].y);
    pz[p] = make_float2(pi[2 * p].z, pi[2 * p + 1].z);
    qx[p] = qy[p] = qz[p] = make_float2(0.f, 0.f);
  }
  // energy form: C12, C6 and E(r_c) coefficients (base, difference for a
  // C_33 j) of atoms 2p, 2p+1, and the eight sums in two FP32 halves
  float ecd[2][6];   // ec of a C_32 (0) and a C_33 (1) atom i
  float2 ev2[kEnergyVals];
  if (ENERGY) {
#pragma unroll
    for (int ty = 0; ty < 2; ++ty) {
      ecd[ty][0] = R.C12u[ty]; ecd[ty][1] = R.C12u[ty + 1] - ecd[ty][0];
      ecd[ty][2] = R.C6u[ty]; ecd[ty][3] = R.C6u[ty + 1] - ecd[ty][2];
      ecd[ty][4] = fp.erc[ty][0]; ecd[ty][5] = fp.erc[ty][1] - ecd[ty][4];
    }
#pragma unroll
    for (int a = 0; a < kEnergyVals; ++a) ev2[a] = make_float2(0.f, 0.f);
  }
  const unsigned* L = list + (size_t)(valid ? s_cl[q] : 0) * cap;
  // clusters without a chain end (the common case) share one pair
  // coefficient per j type: two scalar FMAs per entry instead of four
  // FFMA2 (same values: each coefficient is the same single-rounded FMA)
  const unsigned tb = ((unsigned)in >> 3) & 15u;   // bit u: atom u is a C_33 chain end
  const bool uni = __all_sync(0xffffffffu, tb == 0u);
  // two entries per lane per iteration (independent work for the
  // scheduler), the next two in flight; an entry past the list is 0:
  // tile atom 0 with an empty mask, which adds nothing
  auto run = [&](auto uni_tag) {
    constexpr bool UNI = decltype(uni_tag)::value;
    unsigned E0 = sl < n ? __ldg(L + sl) : 0u;
    unsigned E1 = sl + LP < n ? __ldg(L + sl + LP) : 0u;
    for (int e = sl; e - sl < nmax; e += 2 * LP) {
      const unsigned E2 = e + 2 * LP < n ? __ldg(L + e + 2 * LP) : 0u;
      const unsigned E3 = e + 3 * LP < n ? __ldg(L + e + 3 * LP) : 0u;
      const int t0 = (int)(E0 & 0xffffu), t1 = (int)(E1 & 0xffffu);
      const float4 w0 = sp[t0], w1 = sp[t1];
      float g0x = 0.f, g0y = 0.f, g0z = 0.f, g1x = 0.f, g1y = 0.f, g1z = 0.f;
      if (!ENERGY) {
        float2 cA0[2], cB0[2], cA1[2], cB1[2];
        if (UNI) {
          const float a_0 = fmaf(w0.w, A1 - A0, A0), b_0 = fmaf(w0.w, -(B1 - B0), -B0);
          const float a_1 = fmaf(w1.w, A1 - A0, A0), b_1 = fmaf(w1.w, -(B1 - B0), -B0);
          cA0[0] = cA0[1] = make_float2(a_0, a_0); cB0[0] = cB0[1] = make_float2(b_0, b_0);
          cA1[0] = cA1[1] = make_float2(a_1, a_1); cB1[0] = cB1[1] = make_float2(b_1, b_1);
        } else {
          // the coefficients of j with a C_32 and with a C_33 atom, then
          // per atom of the cluster the one of its type (bit u of tb)
          const float a2_0 = fmaf(w0.w, A1 - A0, A0), a3_0 = fmaf(w0.w, A2 - A1, A1);
          const float b2_0 = fmaf(w0.w, -(B1 - B0), -B0), b3_0 = fmaf(w0.w, -(B2 - B1), -B1);
          const float a2_1 = fmaf(w1.w, A1 - A0, A0), a3_1 = fmaf(w1.w, A2 - A1, A1);
          const float b2_1 = fmaf(w1.w, -(B1 - B0), -B0), b3_1 = fmaf(w1.w, -(B2 - B1), -B1);
#pragma unroll
          for (int p = 0; p < 2; ++p) {
            const bool ta = (tb >> (2 * p)) & 1u, tc = (tb >> (2 * p + 1)) & 1u;
            cA0[p] = make_float2(ta ? a3_0 : a2_0, tc ? a3_0 : a2_0);
            cB0[p] = make_float2(ta ? b3_0 : b2_0, tc ? b3_0 : b2_0);
            cA1[p] = make_float2(ta ? a3_1 : a2_1, tc ? a3_1 : a2_1);
            cB1[p] = make_float2(ta ? b3_1 : b2_1, tc ? b3_1 : b2_1);
          }
        }
        if constexpr (EXACT) {
          unsigned j0x, j0y, j0z, j1x, j1y, j1z;
          entry_packed_exact(px, py, pz, cA0, cB0, rc2, w0, E0 >> 16, qi, j0x, j0y, j0z, chk);
          entry_packed_exact(px, py, pz, cA1, cB1, rc2, w1, E1 >> 16, qi, j1x, j1y, j1z, chk);
          if (e < n) {
            atomicAdd(ax + 3 * t0, (int)j0x); atomicAdd(ay + 3 * t0, (int)j0y); atomicAdd(az + 3 * t0, (int)j0z);
          }
          if (e + LP < n) {
            atomicAdd(ax + 3 * t1, (int)j1x); atomicAdd(ay + 3 * t1, (int)j1y); atomicAdd(az + 3 * t1, (int)j1z);
          }
        } else {
          entry_packed(px, py, pz, cA0, cB0, rc2, w0, E0 >> 16, qx, qy, qz, g0x, g0y, g0z);
          entry_packed(px, py, pz, cA1, cB1, rc2, w1, E1 >> 16, qx, qy, qz, g1x, g1y, g1z);
        }
      } else {
        // C12, C6 and E(r_c) of j with a C_32 and with a C_33 atom, then per
        // atom of the cluster the one of its type (bit u of tb)
        float k0[2][3], k1[2][3];
#pragma unroll
        for (int ty = 0; ty < 2; ++ty)
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            k0[ty][a] = fmaf(w0.w, ecd[ty][2 * a + 1], ecd[ty][2 * a]);
            k1[ty][a] = fmaf(w1.w, ecd[ty][2 * a + 1], ecd[ty][2 * a]);
          }
        float2 c12a[2], c6a[2], sha[2], c12b[2], c6b[2], shb[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
          const bool ta = (tb >> (2 * p)) & 1u, tc = (tb >> (2 * p + 1)) & 1u;
          c12a[p] = make_float2(ta ? k0[1][0] : k0[0][0], tc ? k0[1][0] : k0[0][0]);
          c12b[p] = make_float2(ta ? k1[1][0] : k1[0][0], tc ? k1[1][0] : k1[0][0]);
          c6a[p] = make_float2(ta ? k0[1][1] : k0[0][1], tc ? k0[1][1] : k0[0][1]);
          c6b[p] = make_float2(ta ? k1[1][1] : k1[0][1], tc ? k1[1][1] : k1[0][1]);
          sha[p] = make_float2(ta ? k0[1][2] : k0[0][2], tc ? k0[1][2] : k0[0][2]);
          shb[p] = make_float2(ta ? k1[1][2] : k1[0][2], tc ? k1[1][2] : k1[0][2]);
        }
        entry_packed_energy(px, py, pz, c12a, c6a, sha, rc2, w0, E0 >> 16, ev2);
        entry_packed_energy(px, py, pz, c12b, c6b, shb, rc2, w1, E1 >> 16, ev2);
      }
      if (!ENERGY && !EXACT) {
        if (e < n) acc_add(ax, ay, az, t0, g0x, g0y, g0z, scale, lim, flags);
        if (e + LP < n) acc_add(ax, ay, az, t1, g1x, g1y, g1z, scale, lim, flags);
      }
      E0 = E2;
      E1 = E3;
    }
  };
  if (!ENERGY && uni) run(std::true_type{});
  else run(std::false_type{});
  if (ENERGY) {
#pragma unroll
    for (int a = 0; a < kEnergyVals; ++a) ev[a] = ev2[a].x + ev2[a].y;
    ev[1] = ev[0] - ev[1];   // lj_shifted: the pair energies less the kept pairs' E(r_c)
  }
  if (!ENERGY) {
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      fi[2 * p][0] = qx[p].x; fi[2 * p + 1][0] = qx[p].y;
      fi[2 * p][1] = qy[p].x; fi[2 * p + 1][1] = qy[p].y;
      fi[2 * p][2] = qz[p].x; fi[2 * p + 1][2] = qz[p].y;
    }
  }
  // forces on the cluster's atoms: a fixed xor tree over the LP lanes
  // (offsets LP/2, ..., 2, 1).  The offsets above 4 add all twelve sums;
  // at 4 and 2 each lane keeps half of the atoms it still holds and receives
  // the partner's part of them, so that after offset 1 lanes 2u and 2u + 1
  // hold atom u.  Every sum is formed by the same tree of additions as a
  // full butterfly (the same bits), with half the shuffles.
  if (!ENERGY && !EXACT) {
#pragma unroll
    for (int o = LP / 2; o > 4; o >>= 1)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int a = 0; a < 3; ++a) fi[u][a] += __shfl_xor_sync(0xffffffffu, fi[u][a], o);
    const bool hi = (sl & 4) != 0, mid = (sl & 2) != 0;
    float r1[2][3];   // atoms 2 hi + j
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float keep = hi ? fi[2 + j][a] : fi[j][a], send = hi ? fi[j][a] : fi[2 + j][a];
        r1[j][a] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
    float g[3];       // atom 2 hi + mid
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float keep = mid ? r1[1][a] : r1[0][a], send = mid ? r1[0][a] : r1[1][a];
      g[a] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
      g[a] += __shfl_xor_sync(0xffffffffu, g[a], 1);
    }
    const int u = sl >> 1;
    if ((sl & 1) == 0 && u < ni) {
      const float sx = g[0] * scale, sy = g[1] * scale, sz = g[2] * scale;
      range_check(sx, sy, sz, flags);
      atomicAdd(ax + 3 * (i0 + u), acc_fix(sx));
      atomicAdd(ay + 3 * (i0 + u), acc_fix(sy));
      atomicAdd(az + 3 * (i0 + u), acc_fix(sz));
    }
  }
  if constexpr (EXACT && !ENERGY) {
    // each lane added one offset per entry slot it processed (two per
    // iteration, the same count on every lane); the integer sums over the
    // lanes are exact in any order
    const unsigned n_add = 2u * (unsigned)((nmax + 2 * LP - 1) / (2 * LP));
    if (chk >= 0x800000u) atomicOr(flags, kFlagFixOverflow);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        unsigned v = qi[u][a] - n_add * kExactOff;
#pragma unroll
        for (int o = LP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        qi[u][a] = v;
      }
    unsigned vx = qi[0][0], vy = qi[0][1], vz = qi[0][2];
#pragma unroll
    for (int u = 1; u < 4; ++u)
      if (sl == u) { vx = qi[u][0]; vy = qi[u][1]; vz = qi[u][2]; }
    if (sl < ni) {
      atomicAdd(ax + 3 * (i0 + sl), (int)vx);
      atomicAdd(ay + 3 * (i0 + sl), (int)vy);
      atomicAdd(az + 3 * (i0 + sl), (int)vz);
    }
  }
  if (ENERGY) {
#pragma unroll
    for (int a = 0; a < kEnergyVals; ++a) {
      float v = ev[a];
#pragma unroll
      for (int o = LP / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (sl == 0 && valid) ecl[q][a] = v;
    }
  }
}

// Add the tile's accumulators to the int64 forces (2^-32 kJ/mol/nm): warps
// w0, w0 + nw, ... take tile cells; one integer atomic per component and
// tile atom with a non-zero sum (consecutive atoms: coalesced).
__device__ __forceinline__ void flush_tile(const RegTile& T, const int* __restrict__ ax, const int* __restrict__ ay,
                                           const int* __restrict__ az, long long* __restrict__ flj, int Npad, int w0,
                                           int nw) {
  const int lane = threadIdx.x & 31;
  for (int kc = w0; kc < T.n_tile; kc += nw) {
    const int t0 = T.off[kc], nk = T.off[kc + 1] - t0, s0 = T.start[kc];
    for (int q = lane; q < nk; q += 32) {
      const int t = t0 + q, sidx = s0 + q;
      const int qx = ax[3 * t], qy = ay[3 * t], qz = az[3 * t];
      if ((qx | qy | qz) == 0) continue;
      atomicAdd(reinterpret_cast<unsigned long long*>(flj + sidx), (unsigned long long)((long long)qx << kLjAccShift));
      atomicAdd(reinterpret_cast<unsigned long long*>(flj + Npad + sidx),
                (unsigned long long)((long long)qy << kLjAccShift));
      atomicAdd(reinterpret_cast<unsigned long long*>(flj + 2 * (size_t)Npad + sidx),
                (unsigned long long)((long long)qz << kLjAccShift));
    }
  }
}

// Per region: the clusters' FP32 sums added in FP64 in cluster order; the
// region's sums go to the slot of its first home cell, zeros to the others
// (the reduction sums a replica's cell slots).  Lanes 0..7 of the caller.
__device__ __forceinline__ void region_energy(const RegTile& T, int nq, bool fits,
                                              const float (*__restrict__ ecl)[kEnergyVals], double* __restrict__ epart,
                                              int a) {
  double v = 0.0;
  if (fits)
    for (int q = 0; q < nq; ++q) v += (double)ecl[q][a];
  epart[(size_t)T.home_cell[0] * kEnergyVals + a] = v;
  for (int hh = 1; hh < T.n_home; ++hh) epart[(size_t)T.home_cell[hh] * kEnergyVals + a] = 0.0;
}

// longest list first: warps that take the last clusters finish soon, and
// the clusters that share a warp have similar lengths.  Cluster q's key is
// (list length << 9) | (511 - q), unique (q < 512) so that ties go to the
// lower index; its rank is the number of larger keys (threads t0, t0 + nt,
// ...; four keys per shared load, the slots past nq hold -1).  The same
// thread records in s_in which of the cluster's four slots hold a C_33
// chain end (bit u; a slot past the cell's last atom repeats that atom).
__device__ __forceinline__ void rank_clusters(const int* __restrict__ s_key, short* __restrict__ s_ord,
                                              int* __restrict__ s_in, const float4* __restrict__ sp, int nq, int t0,
                                              int nt) {
  const int4* k4 = reinterpret_cast<const int4*>(s_key);
  const int n4 = (nq + 3) >> 2;
  for (int q = t0; q < nq; q += nt) {
    const int kq = s_key[q];
    int rank = 0;
    for (int o = 0; o < n4; ++o) {
      const int4 k = k4[o];
      rank += (k.x > kq) + (k.y > kq) + (k.z > kq) + (k.w > kq);
    }
    s_ord[rank] = (short)q;
    const int in = s_in[q], i0 = in >> 7, ni = in & 7;
    unsigned tb = 0u;
#pragma unroll
    for (int u = 0; u < 4; ++u) tb |= sp[i0 + min(u, ni - 1)].w != 0.f ? (1u << u) : 0u;
    s_in[q] = in | (int)(tb << 3);
  }
}

// One block per region (grid schedule), or a fixed grid whose blocks take
// regions from a device counter (persistent schedule).  The block stages
// the tile, its warps take tasks of 32/LP clusters from a shared counter
// (longest lists first), and after a barrier the block flushes the tile's
// accumulators.
template <bool ENERGY, int NT, int LP, bool EXACT = false>
__global__ void __launch_bounds__(NT, 768 / NT) k_cl_force(
    const float4* __restrict__ pos, const int* __restrict__ cell_start, const int* __restrict__ cl_start,
    const Region* __restrict__ regions, int n_regions, const RegionShape* __restrict__ shapes,
    const RepDev* __restrict__ reps, const unsigned* __restrict__ list, const int* __restrict__ ncl, int cap,
    int tile_cap, const ForceParams fp, long long* __restrict__ flj, int Npad, double* __restrict__ epart,
    unsigned* __restrict__ flags, int persistent, int* __restrict__ work) {
  constexpr int CPW = 32 / LP;
  extern __shared__ __align__(16) unsigned char smem[];
  float4* sp = reinterpret_cast<float4*>(smem);
  // accumulators of tile atom t at ax[3t], ay[3t] = ax[3t + 1], az[3t] = ax[3t + 2]
  // (one base register in the pair loop; lanes on consecutive t hit distinct banks)
  int* ax = reinterpret_cast<int*>(smem + (size_t)tile_cap * sizeof(float4));
  int* ay = ax + 1;
  int* az = ax + 2;
  __shared__ RegTile T;
  __shared__ int sh_r, sh_q;
  __shared__ __align__(16) int s_key[kRegionClusterCap];   // (list length << 9) | (511 - q) of cluster q
  __shared__ short s_ord[kRegionClusterCap];   // the clusters, longest list first (ties: lower index)
  __shared__ int s_cl[kRegionClusterCap];      // global id of each of the region's clusters
  __shared__ int s_in[kRegionClusterCap];      // first tile atom << 7 | chain-end bits << 3 | atoms (1..4)
  // energy form: each cluster's 8 sums (FP32 lane tree), added over the
  // region's clusters in cluster order, so the result does not depend on
  // which warp took which cluster
  __shared__ float ecl[ENERGY ? kRegionClusterCap : 1][kEnergyVals];
  const int lane = threadIdx.x & 31;
  for (int it = 0;; ++it) {
    const int r = next_region(persistent != 0, it, work, &sh_r);
    if (r < 0 || r >= n_regions) break;
    const Region g = regions[r];
    const RegionShape& S = shapes[g.shape];
    const RepDev& R = reps[g.rep];
    __syncthreads();   // the previous region's tables are no longer read
    region_setup(T, g, S, R, cell_start, cl_start);
    const int total = T.off[T.n_tile];
    const int nq = T.ncl[T.n_home];
    const bool fits = total <= tile_cap && nq <= kRegionClusterCap;
    if (!fits) {
      if (threadIdx.x == 0) atomicOr(flags, kFlagNbrOverflow);
    } else {
      // list lengths and zeroed accumulators while the tile copies fly
      tile_issue<NT>(T, pos, sp);
      if (!ENERGY)   // 3 tile_cap is a multiple of 4: the rounded-up span stays in the buffer
        for (int t = threadIdx.x; t < (3 * total + 3) / 4; t += NT) reinterpret_cast<int4*>(ax)[t] = make_int4(0, 0, 0, 0);
      for (int q = threadIdx.x; q < ((nq + 3) & ~3); q += NT) {
        if (q >= nq) { s_key[q] = -1; continue; }
        int h, k;
        cluster_of(T, q, h, k);
        const int cl = T.cl0[h] + k, i0 = T.off[h] + 4 * k;
        s_key[q] = (__ldg(ncl + cl) << 9) | (511 - q);
        s_cl[q] = cl;
        s_in[q] = (i0 << 7) | min(4, T.off[h + 1] - i0);
      }
      if (threadIdx.x == 0) sh_q = 0;
      tile_finish<false, NT>(T, sp, nullptr);   // ends with a barrier
      rank_clusters(s_key, s_ord, s_in, sp, nq, threadIdx.x, NT);
      __syncthreads();
      const LjConst c = lj_const(R);
      for (;;) {
        int q0 = 0;
        if (lane == 0) q0 = atomicAdd(&sh_q, CPW);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if (q0 >= nq) break;
        cluster_task<ENERGY, LP, EXACT>(q0, nq, T, sp, ax, ay, az, s_key, s_ord, s_cl, s_in, ecl, list, cap, R, fp, c,
                                        flags);
      }
      __syncthreads();
      if (!ENERGY) flush_tile(T, ax, ay, az, flj, Npad, threadIdx.x >> 5, NT / 32);
    }
    if (ENERGY) {
      __syncthreads();
      if (threadIdx.x < kEnergyVals) region_energy(T, nq, fits, ecl, epart, threadIdx.x);
    }
  }
  if (persistent) persistent_done(work);
}

// ===================================================================== launch
size_t cl_build_smem(int tile_cap) { return (size_t)tile_cap * sizeof(float4); }
size_t cl_force_smem(int tile_cap) { return (size_t)tile_cap * (sizeof(float4) + 3 * sizeof(int)); }

void launch_cl_build(const float4* pos, const int* tag, const int* cell_start, const int* cl_start,
                     const Region* regions, int n_regions, const RegionShape* shapes, const RepDev* reps,
                     unsigned* list, int* ncl, int cap, int tile_cap, unsigned* flags, int persistent_grid, int* work,
                     const TopoDev* topo, cudaStream_t st) {
  if (n_regions <= 0) return;
  const int grid = persistent_grid > 0 ? persistent_grid : n_regions;
  const size_t sm = cl_build_smem(tile_cap);
  if (topo)
    k_cl_build<256, true><<<grid, 256, sm, st>>>(pos, tag, cell_start, cl_start, regions, n_regions, shapes, reps, list,
                                                 ncl, cap, tile_cap, flags, persistent_grid > 0, work, *topo);
  else
    k_cl_build<256, false><<<grid, 256, sm, st>>>(pos, tag, cell_start, cl_start, regions, n_regions, shapes, reps,
                                                  list, ncl, cap, tile_cap, flags, persistent_grid > 0, work, TopoDev{});
}

void launch_cl_force(bool energy, const float4* pos, const int* cell_start, const int* cl_start,
                     const Region* regions, int n_regions, const RegionShape* shapes, const RepDev* reps,
                     const unsigned* list, const int* ncl, int cap, int tile_cap, const ForceParams& fp,
                     long long* flj, int Npad, double* epart, unsigned* flags, int block, int lanes,
                     int persistent_grid, int* work, bool exact, cudaStream_t st) {
  if (n_regions <= 0) return;
  const int grid = persistent_grid > 0 ? persistent_grid : n_regions;
  const int pers = persistent_grid > 0;
  const size_t sm = cl_force_smem(tile_cap);
#define MDG_CLF(E, NT, LP, X)                                                                                    \
  k_cl_force<E, NT, LP, X><<<grid, NT, sm, st>>>(pos, cell_start, cl_start, regions, n_regions, shapes, reps, list, \
                                                 ncl, cap, tile_cap, fp, flj, Npad, epart, flags, pers, work)
#define MDG_CLF2(NT, LP)                  \
  if (energy) MDG_CLF(true, NT, LP, false); \
  else if (exact) MDG_CLF(false, NT, LP, true); \
  else MDG_CLF(false, NT, LP, false);
  if (block == 128) {
    if (lanes == 8) { MDG_CLF2(128, 8) } else if (lanes == 32) { MDG_CLF2(128, 32) } else { MDG_CLF2(128, 16) }
  } else if (block == 384) {
    if (lanes == 8) { MDG_CLF2(384, 8) } else if (lanes == 32) { MDG_CLF2(384, 32) } else { MDG_CLF2(384, 16) }
  } else {
    if (lanes == 8) { MDG_CLF2(256, 8) } else if (lanes == 32) { MDG_CLF2(256, 32) } else { MDG_CLF2(256, 16) }
  }
#undef MDG_CLF2
#undef MDG_CLF
}

// resident blocks per SM of the force kernel for a block size, lanes per cluster and tile
int lj_blocks_per_sm(int block, int lanes, int tile_cap) {
  int nb = 0;
  const size_t sm = cl_force_smem(tile_cap);
#define MDG_OCC(NT, LP) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_cl_force<false, NT, LP>, NT, sm)
  if (block == 128) {
    if (lanes == 8) MDG_OCC(128, 8); else if (lanes == 32) MDG_OCC(128, 32); else MDG_OCC(128, 16);
  } else if (block == 384) {
    if (lanes == 8) MDG_OCC(384, 8); else if (lanes == 32) MDG_OCC(384, 32); else MDG_OCC(384, 16);
  } else {
    if (lanes == 8) MDG_OCC(256, 8); else if (lanes == 32) MDG_OCC(256, 32); else MDG_OCC(256, 16);
  }
#undef MDG_OCC
  return nb;
}

// Opt in to more than 48 KB of dynamic shared memory (once per device); the
// attribute is an upper bound, set for the largest tile accepted.
cudaError_t tile_kernels_init() {
  const int mb = (int)cl_build_smem(kStageCapMax), mf = (int)cl_force_smem(kStageCapMax);
  cudaError_t e = cudaFuncSetAttribute(k_cl_build<256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mb);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cl_build<256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mb);
#define MDG_ATTR(E, NT, LP)                                                                                   \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cl_force<E, NT, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, mf); \
  if (e == cudaSuccess && !E)                                                                                 \
    e = cudaFuncSetAttribute(k_cl_force<false, NT, LP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mf);
#define MDG_ATTR3(E, NT) MDG_ATTR(E, NT, 8) MDG_ATTR(E, NT, 16) MDG_ATTR(E, NT, 32)
  MDG_ATTR3(false, 128) MDG_ATTR3(true, 128) MDG_ATTR3(false, 256) MDG_ATTR3(true, 256)
  MDG_ATTR3(false, 384) MDG_ATTR3(true, 384)
#undef MDG_ATTR3
#undef MDG_ATTR
  return e;
}

int tile_capacity_max() { return kStageCapMax; }

// ===================================================================== bounded wait self-test
// One thread waits on an mbarrier that nothing arrives on, gives up after
// `spins` try_wait rounds and raises kFlagTimeout: the bounded-wait pattern
// that any device wait of this library must follow.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__global__ void __launch_bounds__(32) k_wait_selftest(unsigned spins, unsigned* __restrict__ flags) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool done = false;
    for (unsigned k = 0; k < spins && !done; ++k) {
      unsigned d;
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(d)
          : "r"(smem_u32(&bar)), "r"(0u)
          : "memory");
      done = d != 0u;
    }
    if (!done) atomicOr(flags, kFlagTimeout);
  }
}

void launch_wait_selftest(unsigned spins, unsigned* flags, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(spins, flags);
}

}  // namespace mdg
