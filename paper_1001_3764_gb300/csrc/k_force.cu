// k_force.cu -- Dreiding II bonded forces (Eqs. 4-6, Sec. 3.3) on sm_103a.
// The Lennard-Jones force (Eq. 2) is in k_lj.cu.
//
// Each thread block owns a contiguous range of atoms (whole or partial
// chains) plus a 3-atom halo.  Bond vectors are formed once per bond (FP64
// differences of the master positions in the mixed form, exact FP32
// differences in the plain form), every bond/angle/dihedral term is evaluated
// once by the thread of its first atom, and each home atom then sums the
// contributions of the (at most 2+3+4) terms that contain it in a fixed
// order.  This removes the paper's 2x/3x/4x redundant per-home-atom flops
// (Sec. 3.3) without atomics.  The kernel also adds the LJ force of the atom
// (read from cell-sorted order through inv_perm) so the integrator reads one
// force per atom.  Energies and the virial are block sums: FP32 warp trees,
// then FP64 across warps, in a fixed order.
#include <type_traits>

#include "md_kernels.cuh"

namespace mdg {

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Block reduction of NV FP32 per-thread values into out[NV] (FP64; thread 0
// holds the result): each warp adds its 32 lanes in FP32 by a fixed shuffle
// tree (an FP64 tree per lane would load this GPU's narrow FP64 pipe), lane 0
// converts the warp sum to FP64 and the warps are added in FP64 in order.
// Fixed shape, so the summation order is the same on every run.
template <int NV, int NT>
__device__ __forceinline__ void block_sum(const float (&v)[NV], double* out) {
  __shared__ double red[NV][NT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) red[k][w] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = 0.0;
      for (int q = 0; q < NT / 32; ++q) s += red[k][q];
      out[k] = s;
    }
  }
}

// FP32 force -> int64 fixed point (2^-32 kJ/mol/nm); each part below 2^18
__device__ __forceinline__ long long to_fix(float f, unsigned* flags) {
  if (!(fabsf(f) < 262144.0f)) { atomicOr(flags, kFlagFixOverflow); return 0; }
  return fix_round_int(f);   // = __float2ll_rn(f * 2^32), on the integer pipe
}

// ======================================================================= bonded
constexpr int kBondedBlock = 256;
constexpr int kHalo = 3;
constexpr int kBondedVals = 9;   // bond, angle, dihedral, vxx, vyy, vzz, vxy, vxz, vyz

struct f3 { float x, y, z; };
__device__ __forceinline__ f3 mk(float x, float y, float z) { return {x, y, z}; }
__device__ __forceinline__ f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ f3 operator-(f3 a) { return {-a.x, -a.y, -a.z}; }
__device__ __forceinline__ f3 operator*(float s, f3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ f3 cross(f3 a, f3 b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// bond vector x_{m+1} - x_m under the minimum image (FP64 master); |d| > L/2
// is tested on the bit patterns (integer pipe), which order like the values
__device__ __forceinline__ double bond_diff(double a, double b, double L, double hL) {
  double d = b - a;
  const long long bd = __double_as_longlong(d);
  if ((bd & 0x7fffffffffffffffll) > __double_as_longlong(hL)) d = bd < 0 ? d + L : d - L;
  return d;
}

// |b|^2 - b0^2 for an exact FP32 vector b: each square is split into its
// rounded value and exact error (FMA), the rounded parts are summed with
// error-free two-sums, and b0^2 = c_hi + c_lo is subtracted from the
// leading part, where the two nearly cancel without rounding.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ float sq_minus(f3 b, float c_hi, float c_lo) {
  const float px = b.x * b.x, py = b.y * b.y, pz = b.z * b.z;
  const float ex = fmaf(b.x, b.x, -px), ey = fmaf(b.y, b.y, -py), ez = fmaf(b.z, b.z, -pz);
  float s1, e1, s2, e2;
  two_sum(px, py, s1, e1);
  two_sum(s1, pz, s2, e2);
  return (s2 - c_hi) + ((e1 + e2) + (ex + ey + ez) - c_lo);
}
// FP32 master: the difference of two nearby floats is exact; across a face the
// partner is first moved by L (exact when it lies near the face, L being an
// FP32 number), so the result is again the exact difference.
__device__ __forceinline__ float bond_comp(float a, float b, float L, float hL) {
  float d = b - a;
  if (d > hL) d = (b - L) - a; else if (d < -hL) d = b - (a - L);
  return d;
}

__device__ __forceinline__ void add_vir(float (&W)[6], f3 r, f3 f) {
  W[0] += r.x * f.x; W[1] += r.y * f.y; W[2] += r.z * f.z;
  W[3] += r.x * f.y; W[4] += r.x * f.z; W[5] += r.y * f.z;
}

// int64 fixed point (2^-32 kJ/mol/nm) -> FP32 on the 32-bit pipes: the high
// word (|hi| < 2^24, exact) plus the low word scaled by 2^-32
__device__ __forceinline__ float fix_to_float(long long q) {
  const int hi = (int)(q >> 32);
  const unsigned lo = (unsigned)q;
  return fmaf((float)lo, 2.3283064365386963e-10f, (float)hi);
}

template <bool MIXED, bool ENERGY>
__global__ void __launch_bounds__(kBondedBlock) k_bonded(const void* __restrict__ xv, const uint16_t* __restrict__ site,
                                                         const int* __restrict__ inv_perm, const long long* __restrict__ flj,
                                                         int Npad, int N, const Tile* __restrict__ tiles,
                                                         const RepDev* __restrict__ reps, const ForceParams fp,
                                                         void* __restrict__ Fout, double* __restrict__ epart,
                                                         unsigned* __restrict__ flags) {
  using T = typename std::conditional<MIXED, double, float>::type;
  const T* x = reinterpret_cast<const T*>(xv);
  __shared__ f3 bv[kBondedBlock + 2 * kHalo];
  __shared__ float bD[kBondedBlock + 2 * kHalo];   // r^2 - b0^2 of each bond, free of cancellation
  __shared__ f3 fbd[kBondedBlock], fan_a[kBondedBlock], fan_c[kBondedBlock];
  __shared__ f3 fdi1[kBondedBlock], fdi2[kBondedBlock], fdi3[kBondedBlock];
  const Tile t = tiles[blockIdx.x];
  const RepDev& R = reps[t.rep];
  const int lo = R.atom_off, hi = R.atom_off + R.n_atoms;
  const int S = fp.sites;
  const int base = t.start - kHalo;
  // 1. bond vectors b_m = x_{m+1} - x_m for m in [start-3, start+len+3)
  for (int q = threadIdx.x; q < t.len + 2 * kHalo; q += blockDim.x) {
    const int m = base + q;
    f3 b = mk(0.f, 0.f, 0.f);
    float D = 0.f;
    if (m >= lo && m + 1 < hi && site[m] < S - 1) {
      if (MIXED) {
        const double dx = bond_diff((double)x[m], (double)x[m + 1], R.L, R.half_L);
        const double dy = bond_diff((double)x[N + m], (double)x[N + m + 1], R.L, R.half_L);
        const double dz = bond_diff((double)x[2 * N + m], (double)x[2 * N + m + 1], R.L, R.half_L);
        b = mk(d2f_rn_int(dx), d2f_rn_int(dy), d2f_rn_int(dz));
        D = d2f_rn_int(fma(dx, dx, fma(dy, dy, fma(dz, dz, -fp.b0sq))));
      } else {
        b.x = bond_comp((float)x[m], (float)x[m + 1], R.Lf, R.half_Lf);
        b.y = bond_comp((float)x[N + m], (float)x[N + m + 1], R.Lf, R.half_Lf);
        b.z = bond_comp((float)x[2 * N + m], (float)x[2 * N + m + 1], R.Lf, R.half_Lf);
        D = sq_minus(b, fp.b0sq_hi, fp.b0sq_lo);
      }
    }
    bv[q] = b;
    bD[q] = D;
  }
  __syncthreads();
  // 2. terms starting at atom m = base + q
  float Eb = 0.f, Ea = 0.f, Ed = 0.f;
  float W[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  {
    const int q = threadIdx.x;
    const int m = base + q;
    f3 z = mk(0.f, 0.f, 0.f);
    f3 fb = z, fa = z, fc = z, f1 = z, f2 = z, f3v = z;
    if (q < t.len + kHalo && m >= lo && m < hi) {
      const int sm = site[m];
      const bool own = m >= t.start;   // energy/virial counted once, by the owning tile
      if (sm <= S - 2) {               // bond (m, m+1), Eq. (4)
        const f3 b = bv[q];
        const float r = sqrtf(dot(b, b));
        const float dr = bD[q] / (r + fp.b0);   // r - b0 without cancellation
        const float g = fp.kb * dr / r;
        fb = g * b;                    // force on atom m
        if (ENERGY && own) { Eb += 0.5f * fp.kb * dr * dr; add_vir(W, b, -fb); }
      }
      if (sm <= S - 3) {               // angle (m, m+1, m+2), vertex m+1, Eq. (5)
        const f3 u = -bv[q], w = bv[q + 1];
        const float lu = sqrtf(dot(u, u)), lw = sqrtf(dot(w, w));
        const f3 cr = cross(u, w);
        const float sn = sqrtf(dot(cr, cr)), cs = dot(u, w);
        const float th = atan2f(sn, cs);
        const float dth = th - fp.theta0;
        const float inv = 1.0f / (lu * lw);
        const float sin_t = sn * inv, cos_t = cs * inv;
        if (sin_t > 1e-6f) {
          const float g = fp.ka * dth / sin_t;
          const f3 uh = (1.0f / lu) * u, wh = (1.0f / lw) * w;
          fa = (g / lu) * (wh - cos_t * uh);
          fc = (g / lw) * (uh - cos_t * wh);
        }
        if (ENERGY && own) { Ea += 0.5f * fp.ka * dth * dth; add_vir(W, u, fa); add_vir(W, w, fc); }
      }
      if (sm <= S - 4) {               // dihedral (m .. m+3), Eq. (6), IUPAC phi
        const f3 b1 = bv[q], b2 = bv[q + 1], b3 = bv[q + 2];
        const f3 mm = cross(b1, b2), nn = cross(b2, b3);
        const float lb2 = sqrtf(dot(b2, b2)), m2 = dot(mm, mm), n2 = dot(nn, nn);
        const float phi = atan2f(lb2 * dot(b1, nn), dot(mm, nn));
        const float arg = (float)fp.n_mult * phi - fp.phis;
        float sa, ca;
        sincosf(arg, &sa, &ca);
        if (m2 > 1e-24f && n2 > 1e-24f) {
          const float dEdphi = -fp.kphi * (float)fp.n_mult * sa;
          const float cam = -lb2 / m2, cdn = lb2 / n2;
          const float cbm = lb2 / m2 + dot(b1, b2) / (lb2 * m2), cbn = dot(b2, b3) / (lb2 * n2);
          const f3 ga = cam * mm, gd = cdn * nn, gb = cbm * mm + cbn * nn;
          const f3 gc = -(ga + gb + gd);
          f1 = -dEdphi * ga; f2 = -dEdphi * gb; f3v = -dEdphi * gc;
          if (ENERGY && own) {
            const f3 f4 = -(f1 + f2 + f3v);
            add_vir(W, b1, f2); add_vir(W, b1 + b2, f3v); add_vir(W, b1 + b2 + b3, f4);
          }
        }
        if (ENERGY && own) Ed += fp.kphi * (1.0f + ca);
      }
    }
    if (q < kBondedBlock) {
      fbd[q] = fb; fan_a[q] = fa; fan_c[q] = fc; fdi1[q] = f1; fdi2[q] = f2; fdi3[q] = f3v;
    }
  }
  __syncthreads();
  // 3. sum the contributions on each home atom in a fixed order
  if ((int)threadIdx.x < t.len) {
    const int q = threadIdx.x + kHalo;
    const int i = t.start + threadIdx.x;
    f3 F = fbd[q] - fbd[q - 1];
    F = F + fan_a[q] - (fan_a[q - 1] + fan_c[q - 1]) + fan_c[q - 2];
    F = F + fdi1[q] + fdi2[q - 1] + fdi3[q - 2] - (fdi1[q - 3] + fdi2[q - 3] + fdi3[q - 3]);
    // the LJ force of the atom (sorted slot s)
    const int s = inv_perm[i];
    const long long lx = __ldg(flj + s), ly = __ldg(flj + Npad + s), lz = __ldg(flj + 2 * (size_t)Npad + s);
    if (MIXED) {
      F4i o;
      o.x = lx + to_fix(F.x, flags);
      o.y = ly + to_fix(F.y, flags);
      o.z = lz + to_fix(F.z, flags);
      o.w = 0;
      reinterpret_cast<F4i*>(Fout)[i] = o;
    } else {
      reinterpret_cast<float4*>(Fout)[i] =
          make_float4(fix_to_float(lx) + F.x, fix_to_float(ly) + F.y, fix_to_float(lz) + F.z, 0.f);
    }
  }
  if (ENERGY) {
    const float v[kBondedVals] = {Eb, Ea, Ed, W[0], W[1], W[2], W[3], W[4], W[5]};
    block_sum<kBondedVals, kBondedBlock>(v, epart + (size_t)blockIdx.x * kBondedVals);
  }
}

// ======================================================================= bonded, general molecules
// A general molecule type (Sec. 3.3, t_bonds / t_angles / dihedral lists):
// one thread per atom of an integrator tile evaluates the terms listed under
// that atom (each term once, under its first atom) and adds their forces to
// every atom of the term with int64 atomics (integer sums: order-free, so
// deterministic).  The separations are FP64 minimum-image differences of the
// master positions rounded to FP32, as in the chain kernel, and the term
// formulas are those of the chain kernel.  k_bonded_init first writes the
// LJ force of every atom into F.

// FP32 separation x_b - x_a and, for a bond, |x_b - x_a|^2 - b0^2 in FP64
__device__ __forceinline__ f3 sep_ab(const double* x, int N, int a, int b, const RepDev& R) {
  const double dx = bond_diff(x[a], x[b], R.L, R.half_L);
  const double dy = bond_diff(x[N + a], x[N + b], R.L, R.half_L);
  const double dz = bond_diff(x[2 * N + a], x[2 * N + b], R.L, R.half_L);
  return mk(d2f_rn_int(dx), d2f_rn_int(dy), d2f_rn_int(dz));
}

__device__ __forceinline__ void fix_add(F4i* F, int i, f3 f, unsigned* flags) {
  atomicAdd(reinterpret_cast<unsigned long long*>(&F[i].x), (unsigned long long)to_fix(f.x, flags));
  atomicAdd(reinterpret_cast<unsigned long long*>(&F[i].y), (unsigned long long)to_fix(f.y, flags));
  atomicAdd(reinterpret_cast<unsigned long long*>(&F[i].z), (unsigned long long)to_fix(f.z, flags));
}

__global__ void __launch_bounds__(256) k_bonded_init(const int* __restrict__ inv_perm, const long long* __restrict__ flj,
                                                     int Npad, int N, F4i* __restrict__ F) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int s = inv_perm[i];
  F4i o;
  o.x = __ldg(flj + s); o.y = __ldg(flj + Npad + s); o.z = __ldg(flj + 2 * (size_t)Npad + s); o.w = 0;
  F[i] = o;
}

template <bool ENERGY>
__global__ void __launch_bounds__(kBondedBlock) k_bonded_generic(const double* __restrict__ x, int N,
                                                                 const Tile* __restrict__ tiles,
                                                                 const RepDev* __restrict__ reps, const ForceParams fp,
                                                                 const TopoDev tp, F4i* __restrict__ F,
                                                                 double* __restrict__ epart,
                                                                 unsigned* __restrict__ flags) {
  const Tile t = tiles[blockIdx.x];
  const RepDev& R = reps[t.rep];
  float Eb = 0.f, Ea = 0.f, Ed = 0.f;
  float W[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if ((int)threadIdx.x < t.len) {
    const int i = t.start + threadIdx.x;
    const int a = (i - R.atom_off) % tp.naom, m0 = i - a;
    // bonds (a, b), Eq. (4)
    for (int q = tp.b_off[a]; q < tp.b_off[a + 1]; ++q) {
      const int j = m0 + tp.b_at[q];
      const f3 b = sep_ab(x, N, i, j, R);
      const double dx = bond_diff(x[i], x[j], R.L, R.half_L), dy = bond_diff(x[N + i], x[N + j], R.L, R.half_L);
      const double dz = bond_diff(x[2 * N + i], x[2 * N + j], R.L, R.half_L);
      const float D = d2f_rn_int(fma(dx, dx, fma(dy, dy, fma(dz, dz, -fp.b0sq))));
      const float r = sqrtf(dot(b, b));
      const float dr = D / (r + fp.b0);   // r - b0 without cancellation
      const f3 fb = (fp.kb * dr / r) * b; // force on a
      fix_add(F, i, fb, flags);
      fix_add(F, j, -fb, flags);
      if (ENERGY) { Eb += 0.5f * fp.kb * dr * dr; add_vir(W, b, -fb); }
    }
    // angles (a, b, c), vertex b, Eq. (5)
    for (int q = tp.a_off[a]; q < tp.a_off[a + 1]; ++q) {
      const int jb = m0 + tp.a_at[2 * q], jc = m0 + tp.a_at[2 * q + 1];
      const f3 u = sep_ab(x, N, jb, i, R), w = sep_ab(x, N, jb, jc, R);
      const float lu = sqrtf(dot(u, u)), lw = sqrtf(dot(w, w));
      const f3 cr = cross(u, w);
      const float sn = sqrtf(dot(cr, cr)), cs = dot(u, w);
      const float th = atan2f(sn, cs);
      const float dth = th - fp.theta0;
      const float inv = 1.0f / (lu * lw);
      const float sin_t = sn * inv, cos_t = cs * inv;
      f3 fa = mk(0.f, 0.f, 0.f), fc = fa;
      if (sin_t > 1e-6f) {
        const float g = fp.ka * dth / sin_t;
        const f3 uh = (1.0f / lu) * u, wh = (1.0f / lw) * w;
        fa = (g / lu) * (wh - cos_t * uh);
        fc = (g / lw) * (uh - cos_t * wh);
      }
      fix_add(F, i, fa, flags);
      fix_add(F, jc, fc, flags);
      fix_add(F, jb, -(fa + fc), flags);
      if (ENERGY) { Ea += 0.5f * fp.ka * dth * dth; add_vir(W, u, fa); add_vir(W, w, fc); }
    }
    // dihedrals (a, b, c, d), Eq. (6), IUPAC phi
    for (int q = tp.d_off[a]; q < tp.d_off[a + 1]; ++q) {
      const int jb = m0 + tp.d_at[3 * q], jc = m0 + tp.d_at[3 * q + 1], jd = m0 + tp.d_at[3 * q + 2];
      const f3 b1 = sep_ab(x, N, i, jb, R), b2 = sep_ab(x, N, jb, jc, R), b3 = sep_ab(x, N, jc, jd, R);
      const f3 mm = cross(b1, b2), nn = cross(b2, b3);
      const float lb2 = sqrtf(dot(b2, b2)), m2 = dot(mm, mm), n2 = dot(nn, nn);
      const float phi = atan2f(lb2 * dot(b1, nn), dot(mm, nn));
      const float arg = (float)fp.n_mult * phi - fp.phis;
      float sa, ca;
      sincosf(arg, &sa, &ca);
      if (m2 > 1e-24f && n2 > 1e-24f) {
        const float dEdphi = -fp.kphi * (float)fp.n_mult * sa;
        const float cam = -lb2 / m2, cdn = lb2 / n2;
        const float cbm = lb2 / m2 + dot(b1, b2) / (lb2 * m2), cbn = dot(b2, b3) / (lb2 * n2);
        const f3 ga = cam * mm, gd = cdn * nn, gb = cbm * mm + cbn * nn;
        const f3 gc = -(ga + gb + gd);
        const f3 f1 = -dEdphi * ga, f2 = -dEdphi * gb, f3v = -dEdphi * gc;
        const f3 f4 = -(f1 + f2 + f3v);
        fix_add(F, i, f1, flags);
        fix_add(F, jb, f2, flags);
        fix_add(F, jc, f3v, flags);
        fix_add(F, jd, f4, flags);
        if (ENERGY) { add_vir(W, b1, f2); add_vir(W, b1 + b2, f3v); add_vir(W, b1 + b2 + b3, f4); }
      }
      if (ENERGY) Ed += fp.kphi * (1.0f + ca);
    }
  }
  if (ENERGY) {
    const float v[kBondedVals] = {Eb, Ea, Ed, W[0], W[1], W[2], W[3], W[4], W[5]};
    block_sum<kBondedVals, kBondedBlock>(v, epart + (size_t)blockIdx.x * kBondedVals);
  }
}

void launch_bonded_generic(bool energy, const double* x, const int* inv_perm, const long long* flj, int Npad, int N,
                           const Tile* tiles, int n_tiles, const RepDev* reps, const ForceParams& fp,
                           const TopoDev& topo, void* F, double* epart, unsigned* flags, cudaStream_t st) {
  if (N <= 0) return;
  k_bonded_init<<<(N + 255) / 256, 256, 0, st>>>(inv_perm, flj, Npad, N, reinterpret_cast<F4i*>(F));
  if (energy)
    k_bonded_generic<true><<<n_tiles, kBondedBlock, 0, st>>>(x, N, tiles, reps, fp, topo, reinterpret_cast<F4i*>(F),
                                                             epart, flags);
  else
    k_bonded_generic<false><<<n_tiles, kBondedBlock, 0, st>>>(x, N, tiles, reps, fp, topo, reinterpret_cast<F4i*>(F),
                                                              epart, flags);
}

void launch_bonded(bool mixed, bool energy, const void* x, const uint16_t* site, const int* inv_perm,
                   const long long* flj, int Npad, int N, const Tile* tiles, int n_tiles, const RepDev* reps,
                   const ForceParams& fp, void* F, double* epart, unsigned* flags, cudaStream_t st) {
#define MDG_BONDED(M, E) \
  k_bonded<M, E><<<n_tiles, kBondedBlock, 0, st>>>(x, site, inv_perm, flj, Npad, N, tiles, reps, fp, F, epart, flags)
  if (mixed) {
    if (energy) MDG_BONDED(true, true); else MDG_BONDED(true, false);
  } else {
    if (energy) MDG_BONDED(false, true); else MDG_BONDED(false, false);
  }
#undef MDG_BONDED
}

}  // namespace mdg
