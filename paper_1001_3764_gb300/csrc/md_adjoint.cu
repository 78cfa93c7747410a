// md_adjoint.cu -- gradients of trajectory means with respect to the
// force-field parameters, by a hand-written adjoint of the FP64
// velocity-Verlet run.
//
// The run is the NVE integrator of the hot path (Sec. 3 / 3.4) in FP64 on the
// GPU: x_{k+1} = x_k + dt v_{k+1/2}, v_{k+1/2} = v_{k-1/2} + dt a(x_k), with
// half kicks at both ends.  Observables J = 1/(K+1) sum_k O(x_k) with
// O = w0 U + w1 R_ee^2; U = shifted LJ (Eq. 2) + bond (Eq. 4) + angle (Eq. 5)
// + dihedral (Eq. 6), R_ee^2 the mean over chains of the squared end-to-end
// distance (the end-to-end vector of Sec. 4, Fig. 8) from unwrapped positions.
//
// Reverse pass (adjoint of the leapfrog form, newest step first), with
// alpha = dJ/dx_k and beta = dJ/dv_{k+1/2}, c_k = dt (dt/2 at k = 0, 0 at K):
//   u      = c_k M^-1 beta
//   alpha  = w_k grad O(x_k) + alpha - H(x_k) u
//   g     += w_k w0 dU/dtheta(x_k) - d/dtheta [grad U(x_k) . u]
//   beta  += dt alpha                                  (k >= 1)
// H u and d/dtheta[grad U . u] come from one forward-mode (dual-number)
// evaluation of the gradient formulas along u.  U is linear in the pair
// coefficients c12_t = 4 eps_t sigma_t^12, c6_t = 4 eps_t sigma_t^6 of the
// three pair types t and in k_phi, so the parameter derivatives are sums of
// per-pair (per-term) scalars, mapped to (eps, sigma) of the two site types
// through the geometric-mean mixing rule on the host.
//
// Positions are recomputed from (x, v) checkpoints every C steps; a segment
// store holds the C + 1 positions of the segment being reversed.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <type_traits>

#include "../../include/md.h"
#include "md_kernels.cuh"

void md_set_global_error(const char* msg);   // md_api.cu: message for md_last_error(NULL)

namespace mdg {
namespace adj {

// ------------------------------------------------------------------ dual numbers
// value and derivative along one direction of configuration space
struct Dual {
  double v, t;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.t - b.t}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.t}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.t + a.t * b.v}; }
__device__ __forceinline__ Dual operator*(double s, Dual a) { return {s * a.v, s * a.t}; }
__device__ __forceinline__ Dual operator*(Dual a, double s) { return {s * a.v, s * a.t}; }
__device__ __forceinline__ Dual operator+(Dual a, double s) { return {a.v + s, a.t}; }
__device__ __forceinline__ Dual operator+(double s, Dual a) { return {a.v + s, a.t}; }
__device__ __forceinline__ Dual operator-(Dual a, double s) { return {a.v - s, a.t}; }
__device__ __forceinline__ Dual operator-(double s, Dual a) { return {s - a.v, -a.t}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double q = a.v / b.v;
  return {q, (a.t - q * b.t) / b.v};
}
__device__ __forceinline__ Dual operator/(double s, Dual b) {
  const double q = s / b.v;
  return {q, -q * b.t / b.v};
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }

__device__ __forceinline__ double gsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ Dual gsqrt(Dual a) {
  const double r = sqrt(a.v);
  return {r, 0.5 * a.t / r};
}
__device__ __forceinline__ double gatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ Dual gatan2(Dual y, Dual x) {
  return {atan2(y.v, x.v), (x.v * y.t - y.v * x.t) / (x.v * x.v + y.v * y.v)};
}
__device__ __forceinline__ double gcos(double a) { return cos(a); }
__device__ __forceinline__ double gsin(double a) { return sin(a); }
__device__ __forceinline__ Dual gcos(Dual a) {
  double s, c;
  sincos(a.v, &s, &c);
  return {c, -s * a.t};
}
__device__ __forceinline__ Dual gsin(Dual a) {
  double s, c;
  sincos(a.v, &s, &c);
  return {s, c * a.t};
}
__device__ __forceinline__ double value(double a) { return a; }
__device__ __forceinline__ double value(Dual a) { return a.v; }
__device__ __forceinline__ double tangent(double) { return 0.0; }
__device__ __forceinline__ double tangent(Dual a) { return a.t; }

// FP32 dual numbers for the reverse pass's Hessian-vector products (the
// optional FP32 HVP): separations still come from FP64 positions and the pair
// set from an FP64 cutoff test; only the term arithmetic runs in FP32, and its
// per-atom results are added into the FP64 records.  FP64 constants are
// rounded to FP32 where they meet an FP32 dual.
struct DualF {
  float v, t;
};
__device__ __forceinline__ DualF operator+(DualF a, DualF b) { return {a.v + b.v, a.t + b.t}; }
__device__ __forceinline__ DualF operator-(DualF a, DualF b) { return {a.v - b.v, a.t - b.t}; }
__device__ __forceinline__ DualF operator-(DualF a) { return {-a.v, -a.t}; }
__device__ __forceinline__ DualF operator*(DualF a, DualF b) { return {a.v * b.v, a.v * b.t + a.t * b.v}; }
__device__ __forceinline__ DualF operator*(double s, DualF a) { const float f = (float)s; return {f * a.v, f * a.t}; }
__device__ __forceinline__ DualF operator*(DualF a, double s) { const float f = (float)s; return {f * a.v, f * a.t}; }
__device__ __forceinline__ DualF operator+(DualF a, double s) { return {a.v + (float)s, a.t}; }
__device__ __forceinline__ DualF operator+(double s, DualF a) { return {a.v + (float)s, a.t}; }
__device__ __forceinline__ DualF operator-(DualF a, double s) { return {a.v - (float)s, a.t}; }
__device__ __forceinline__ DualF operator-(double s, DualF a) { return {(float)s - a.v, -a.t}; }
__device__ __forceinline__ DualF operator/(DualF a, DualF b) {
  const float q = a.v / b.v;
  return {q, (a.t - q * b.t) / b.v};
}
__device__ __forceinline__ DualF operator/(double s, DualF b) {
  const float q = (float)s / b.v;
  return {q, -q * b.t / b.v};
}
__device__ __forceinline__ DualF& operator+=(DualF& a, DualF b) { a = a + b; return a; }
__device__ __forceinline__ DualF gsqrt(DualF a) {
  const float r = sqrtf(a.v);
  return {r, 0.5f * a.t / r};
}
__device__ __forceinline__ DualF gatan2(DualF y, DualF x) {
  return {atan2f(y.v, x.v), (x.v * y.t - y.v * x.t) / (x.v * x.v + y.v * y.v)};
}
__device__ __forceinline__ DualF gcos(DualF a) {
  float s, c;
  sincosf(a.v, &s, &c);
  return {c, -s * a.t};
}
__device__ __forceinline__ DualF gsin(DualF a) {
  float s, c;
  sincosf(a.v, &s, &c);
  return {s, c * a.t};
}
__device__ __forceinline__ double value(DualF a) { return (double)a.v; }
__device__ __forceinline__ double tangent(DualF a) { return (double)a.t; }

template <class T>
struct V3 {
  T x, y, z;
};
template <class T>
__device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T>
__device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T, class S>
__device__ __forceinline__ V3<T> scale(S s, V3<T> a) { return {s * a.x, s * a.y, s * a.z}; }
template <class T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ------------------------------------------------------------------ parameters
struct AdjDev {
  double L, inv_L, inv_h;     // box, 1/L, cells per nm
  int M, n_off;               // cells per side (1 when L < 3 r_c), neighbour cells visited (27 or 1)
  int sites, n_chains, N;
  double rc, rc2, irc6, irc12;   // cutoff and the shift terms (1/r_c)^6, (1/r_c)^12
  double irc7, irc13;            // force-shifted variant: (1/r_c)^7, (1/r_c)^13
  int sf;                        // 1 = force-shifted variant (not the paper's potential)
  float pre2;                    // FP32 prefilter: (r_c + 1e-4 nm)^2; a candidate beyond it is out in FP64 too
  double c6[3], c12[3];       // pair types 0 = C32-C32, 1 = C32-C33, 2 = C33-C33
  double kb, b0, ka, theta0, kphi, phis;
  int n_mult;
  double inv_mass[2];
};

__device__ __forceinline__ int site_type(int site, int sites) { return (site == 0 || site == sites - 1) ? 1 : 0; }

__device__ __forceinline__ double min_image(double d, const AdjDev& P) { return d - P.L * rint(d * P.inv_L); }

// separation x_b - x_a (minimum image, FP64 value) with the tangent
// u_b - u_a, u_k = cu * beta_k / m_k the direction of atom k, in the scalar
// type T of the evaluation
template <class T>
__device__ __forceinline__ V3<T> make_sep(double dx, double dy, double dz, const double* beta, double cu, int a,
                                          int b, const AdjDev& P);
template <>
__device__ __forceinline__ V3<double> make_sep<double>(double dx, double dy, double dz, const double*, double, int,
                                                       int, const AdjDev&) {
  return {dx, dy, dz};
}
template <>
__device__ __forceinline__ V3<Dual> make_sep<Dual>(double dx, double dy, double dz, const double* beta, double cu,
                                                   int a, int b, const AdjDev& P) {
  const double sa = cu * P.inv_mass[site_type(a % P.sites, P.sites)];
  const double sb = cu * P.inv_mass[site_type(b % P.sites, P.sites)];
  return {{dx, sb * beta[3 * b] - sa * beta[3 * a]}, {dy, sb * beta[3 * b + 1] - sa * beta[3 * a + 1]},
          {dz, sb * beta[3 * b + 2] - sa * beta[3 * a + 2]}};
}
template <>
__device__ __forceinline__ V3<DualF> make_sep<DualF>(double dx, double dy, double dz, const double* beta, double cu,
                                                     int a, int b, const AdjDev& P) {
  const double sa = cu * P.inv_mass[site_type(a % P.sites, P.sites)];
  const double sb = cu * P.inv_mass[site_type(b % P.sites, P.sites)];
  return {{(float)dx, (float)(sb * beta[3 * b] - sa * beta[3 * a])},
          {(float)dy, (float)(sb * beta[3 * b + 1] - sa * beta[3 * a + 1])},
          {(float)dz, (float)(sb * beta[3 * b + 2] - sa * beta[3 * a + 2])}};
}
template <class T>
__device__ __forceinline__ V3<T> sep(const double* x, const double* beta, double cu, int a, int b, const AdjDev& P) {
  return make_sep<T>(min_image(x[3 * b] - x[3 * a], P), min_image(x[3 * b + 1] - x[3 * a + 1], P),
                     min_image(x[3 * b + 2] - x[3 * a + 2], P), beta, cu, a, b, P);
}

__device__ __forceinline__ int cell_coord(double xv, const AdjDev& P) {
  const double s = xv - P.L * floor(xv * P.inv_L);
  int c = (int)floor(s * P.inv_h);
  return c < 0 ? 0 : (c > P.M - 1 ? P.M - 1 : c);
}

// ------------------------------------------------------------------ per-atom record
// fields of rec[kRec * i + f]
constexpr int kRec = 20;
constexpr int kA = 0;        // 4 per pair type t: A.v, A.t, B.v, B.t with A = sum (1/r^12 - 1/rc^12), B = sum (1/r^6 - 1/rc^6)
constexpr int kD = 12;       // D.v, D.t with D = sum (1 + cos(n phi - phi_s))
constexpr int kElj = 14;     // shifted LJ energy (half per pair)
constexpr int kEb = 15, kEa = 16, kEd = 17;
constexpr int kR2 = 18;      // |x_last - x_first|^2 on each chain's first atom
constexpr int kFields = 19;

// ------------------------------------------------------------------ binning (stable counting sort)
// wrapped coordinate in [0, L) (FP64), as the cell test takes it
__device__ __forceinline__ double wrapped(double xv, const AdjDev& P) { return xv - P.L * floor(xv * P.inv_L); }

// cell of every atom, its slot in the cell, and an FP32 copy of its wrapped
// position for the pair prefilter
__global__ void __launch_bounds__(256) k_adj_count(const double* __restrict__ x, AdjDev P, int* __restrict__ cell_of,
                                                   int* __restrict__ count, int* __restrict__ slot,
                                                   float4* __restrict__ x32) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const int c = (cell_coord(x[3 * i + 2], P) * P.M + cell_coord(x[3 * i + 1], P)) * P.M + cell_coord(x[3 * i], P);
  cell_of[i] = c;
  slot[i] = atomicAdd(count + c, 1);
  x32[i] = make_float4((float)wrapped(x[3 * i], P), (float)wrapped(x[3 * i + 1], P), (float)wrapped(x[3 * i + 2], P),
                       0.f);
}

// ------------------------------------------------------------------ LJ, Eq. (2): one warp per atom
constexpr int kLjWarps = 8;

template <class T>
__global__ void __launch_bounds__(32 * kLjWarps) k_adj_lj(const double* __restrict__ x, const double* __restrict__ beta,
                                                          double cu, const int* __restrict__ cell_start,
                                                          const int* __restrict__ perm, AdjDev P,
                                                          const float4* __restrict__ x32,
                                                          double* __restrict__ gv, double* __restrict__ gt,
                                                          double* __restrict__ rec) {
  __shared__ int s_beg[kLjWarps][27];
  __shared__ int s_pre[kLjWarps][28];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kLjWarps + w;
  if (i >= P.N) return;   // the whole warp leaves together
  const int si = i % P.sites, ci = i / P.sites, ti = site_type(si, P.sites);
  const float4 xf = x32[i];
  const float Lf = (float)P.L, iLf = (float)P.inv_L;
  // candidate cells and the prefix of their sizes
  if (lane < P.n_off) {
    int cell = 0;
    if (P.n_off == 27) {
      const int ox = lane % 3 - 1, oy = (lane / 3) % 3 - 1, oz = lane / 9 - 1;
      const int cx = (cell_coord(x[3 * i], P) + ox + P.M) % P.M;
      const int cy = (cell_coord(x[3 * i + 1], P) + oy + P.M) % P.M;
      const int cz = (cell_coord(x[3 * i + 2], P) + oz + P.M) % P.M;
      cell = (cz * P.M + cy) * P.M + cx;
    }
    s_beg[w][lane] = cell_start[cell];
    s_pre[w][lane + 1] = cell_start[cell + 1] - cell_start[cell];
  }
  __syncwarp();
  if (lane == 0) {
    s_pre[w][0] = 0;
    for (int o = 0; o < P.n_off; ++o) s_pre[w][o + 1] += s_pre[w][o];
  }
  __syncwarp();
  const int total = s_pre[w][P.n_off];
  T gx = T{}, gy = T{}, gz = T{};
  T A0 = T{}, B0 = T{}, A1 = T{}, B1 = T{};   // partners of type 0 / type 1
  double e = 0.0;
  float ef = 0.f;                               // the same in the FP32 evaluation
  int o = 0;
  for (int q = lane; q < total; q += 32) {
    while (q >= s_pre[w][o + 1]) ++o;
    const int j = perm[s_beg[w][o] + (q - s_pre[w][o])];
    if (j == i) continue;
    const int sj = j % P.sites;
    if (j / P.sites == ci && abs(sj - si) <= 2) continue;   // 1-2 and 1-3 neighbours (Sec. 3.1)
    {
      // FP32 prefilter on the wrapped copies (error ~1e-6 nm against a 1e-4 nm margin)
      const float4 w = x32[j];
      float ex = xf.x - w.x, ey = xf.y - w.y, ez = xf.z - w.z;
      ex -= Lf * rintf(ex * iLf); ey -= Lf * rintf(ey * iLf); ez -= Lf * rintf(ez * iLf);
      if (ex * ex + ey * ey + ez * ez > P.pre2) continue;
    }
    // the cutoff test on values only, as the definition reads
    const double dx = min_image(x[3 * i] - x[3 * j], P), dy = min_image(x[3 * i + 1] - x[3 * j + 1], P),
                 dz = min_image(x[3 * i + 2] - x[3 * j + 2], P);
    const double r2v = dx * dx + dy * dy + dz * dz;
    if (r2v >= P.rc2) continue;
    const int tj = site_type(sj, P.sites), t = ti + tj;
    const V3<T> d = make_sep<T>(dx, dy, dz, beta, cu, j, i, P);   // x_i - x_j
    const T r2 = dot(d, d);
    const T ir2 = 1.0 / r2;
    const T ir6 = ir2 * ir2 * ir2;
    T A = ir6 * ir6 - P.irc12, B = ir6 - P.irc6;
    T s = (6.0 * P.c6[t] - 12.0 * P.c12[t] * ir6) * ir6 * ir2;   // (1/r) dphi/dr
    if (P.sf) {
      // E_sf = E - E(r_c) - (r - r_c) E'(r_c): the same linear form in c12, c6
      const T r = gsqrt(r2);
      A = A + 12.0 * P.irc13 * (r - P.rc);
      B = B + 6.0 * P.irc7 * (r - P.rc);
      s = s - (6.0 * P.c6[t] * P.irc7 - 12.0 * P.c12[t] * P.irc13) / r;
    }
    gx += s * d.x; gy += s * d.y; gz += s * d.z;
    if (tj) { A1 += 0.5 * A; B1 += 0.5 * B; } else { A0 += 0.5 * A; B0 += 0.5 * B; }
    if constexpr (std::is_same<T, DualF>::value) ef += 0.5f * ((float)P.c12[t] * A.v - (float)P.c6[t] * B.v);
    else e += 0.5 * (P.c12[t] * value(A) - P.c6[t] * value(B));
  }
  // fixed-order butterfly: every lane ends with the same sums (the tangent
  // fields only where there is a tangent; FP32 sums for the FP32 evaluation)
  double r[15];
  if constexpr (std::is_same<T, DualF>::value) {
    float f[15] = {gx.v, gy.v, gz.v, gx.t, gy.t, gz.t, A0.v, A0.t, B0.v, B0.t, A1.v, A1.t, B1.v, B1.t, ef};
#pragma unroll
    for (int k = 0; k < 15; ++k) {
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) f[k] += __shfl_xor_sync(0xffffffffu, f[k], m);
      r[k] = (double)f[k];
    }
  } else {
    r[0] = value(gx); r[1] = value(gy); r[2] = value(gz); r[3] = tangent(gx); r[4] = tangent(gy); r[5] = tangent(gz);
    r[6] = value(A0); r[7] = tangent(A0); r[8] = value(B0); r[9] = tangent(B0);
    r[10] = value(A1); r[11] = tangent(A1); r[12] = value(B1); r[13] = tangent(B1); r[14] = e;
    constexpr bool kTan = std::is_same<T, Dual>::value;
#pragma unroll
    for (int k = 0; k < 15; ++k) {
      if (!kTan && (k == 3 || k == 4 || k == 5 || k == 7 || k == 9 || k == 11 || k == 13)) continue;   // zero
#pragma unroll
      for (int m = 16; m >= 1; m >>= 1) r[k] += __shfl_xor_sync(0xffffffffu, r[k], m);
    }
  }
  if (lane == 0) {
    gv[3 * i] = r[0]; gv[3 * i + 1] = r[1]; gv[3 * i + 2] = r[2];
    if (gt) { gt[3 * i] = r[3]; gt[3 * i + 1] = r[4]; gt[3 * i + 2] = r[5]; }
    double* R = rec + (size_t)kRec * i;
    for (int f = 0; f < 12; ++f) R[kA + f] = 0.0;
    // partner type 0 -> pair type ti, partner type 1 -> pair type ti + 1
    R[kA + 4 * ti + 0] = r[6]; R[kA + 4 * ti + 1] = r[7]; R[kA + 4 * ti + 2] = r[8]; R[kA + 4 * ti + 3] = r[9];
    R[kA + 4 * (ti + 1) + 0] = r[10]; R[kA + 4 * (ti + 1) + 1] = r[11];
    R[kA + 4 * (ti + 1) + 2] = r[12]; R[kA + 4 * (ti + 1) + 3] = r[13];
    R[kElj] = r[14];
  }
}

// ------------------------------------------------------------------ bonded, Eqs. (4)-(6)
// gradient of each term's energy with respect to its atoms (not the force)
// d = x_b - x_a (minimum image)
template <class T>
__device__ __forceinline__ T bond_grad(V3<T> d, const AdjDev& P, V3<T>* g) {
  const T r = gsqrt(dot(d, d));
  const T dr = r - P.b0;
  const T s = P.kb * dr / r;
  g[0] = scale(-s, d);
  g[1] = scale(s, d);
  return 0.5 * P.kb * dr * dr;
}

// theta = angle(u, w), u = x_a - x_b, w = x_c - x_b:
// dtheta/du = ((u.w / u.u) u - w) / |u x w|, likewise for w
template <class T>
__device__ __forceinline__ T angle_grad(V3<T> u, V3<T> w, const AdjDev& P, V3<T>* g) {
  const T c = dot(u, w);
  const T s = gsqrt(dot(cross(u, w), cross(u, w)));
  const T th = gatan2(s, c);
  const T k = P.ka * (th - P.theta0) / s;
  g[0] = scale(k, scale(c / dot(u, u), u) - w);
  g[2] = scale(k, scale(c / dot(w, w), w) - u);
  g[1] = V3<T>{-(g[0].x + g[2].x), -(g[0].y + g[2].y), -(g[0].z + g[2].z)};
  return 0.5 * P.ka * (th - P.theta0) * (th - P.theta0);
}

// IUPAC dihedral of b1 = x_b - x_a, b2 = x_c - x_b, b3 = x_d - x_c with
// m = b1 x b2, n = b2 x b3, phi = atan2(|b2| b1.n, m.n).  Gradient of phi:
// G_a = -|b2|/|m|^2 m, G_d = |b2|/|n|^2 n, G_b = -(1+p) G_a + q G_d,
// G_c = p G_a - (1+q) G_d, p = b1.b2/|b2|^2, q = b3.b2/|b2|^2.
// Returns D = 1 + cos(n phi - phi_s); the energy is k_phi D (Eq. 6).
template <class T>
__device__ __forceinline__ T dihedral_grad(V3<T> b1, V3<T> b2, V3<T> b3, const AdjDev& P, V3<T>* g) {
  const V3<T> m = cross(b1, b2), n = cross(b2, b3);
  const T bb = dot(b2, b2);
  const T lb2 = gsqrt(bb);
  const T phi = gatan2(lb2 * dot(b1, n), dot(m, n));
  const T arg = (double)P.n_mult * phi - P.phis;
  const T dEdphi = (-P.kphi * (double)P.n_mult) * gsin(arg);
  const V3<T> Ga = scale(-(lb2 / dot(m, m)), m);
  const V3<T> Gd = scale(lb2 / dot(n, n), n);
  const T p = dot(b1, b2) / bb, q = dot(b3, b2) / bb;
  const V3<T> Gb = scale(q, Gd) - scale(1.0 + p, Ga);
  const V3<T> Gc = scale(p, Ga) - scale(1.0 + q, Gd);
  g[0] = scale(dEdphi, Ga);
  g[1] = scale(dEdphi, Gb);
  g[2] = scale(dEdphi, Gc);
  g[3] = scale(dEdphi, Gd);
  return 1.0 + gcos(arg);
}

// one thread per atom: every term the atom belongs to, in a fixed order; the
// term's energy is counted on its first atom.  Adds to the LJ gradient.
template <class T>
__global__ void __launch_bounds__(128) k_adj_bonded(const double* __restrict__ x, const double* __restrict__ beta,
                                                    double cu, AdjDev P, double* __restrict__ gv,
                                                    double* __restrict__ gt, double* __restrict__ rec) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const int si = i % P.sites, o = i - si;
  V3<T> g = {T{}, T{}, T{}};
  double eb = 0.0, ea = 0.0;
  T D = T{};
  V3<T> gt4[4];
  for (int q = si - 1; q <= si; ++q) {
    if (q < 0 || q + 1 >= P.sites) continue;
    const T en = bond_grad<T>(sep<T>(x, beta, cu, o + q, o + q + 1, P), P, gt4);
    g = g + gt4[si - q];
    if (q == si) eb = value(en);
  }
  for (int q = si - 2; q <= si; ++q) {
    if (q < 0 || q + 2 >= P.sites) continue;
    const T en = angle_grad<T>(sep<T>(x, beta, cu, o + q + 1, o + q, P), sep<T>(x, beta, cu, o + q + 1, o + q + 2, P),
                               P, gt4);
    g = g + gt4[si - q];
    if (q == si) ea = value(en);
  }
  for (int q = si - 3; q <= si; ++q) {
    if (q < 0 || q + 3 >= P.sites) continue;
    const T dd = dihedral_grad<T>(sep<T>(x, beta, cu, o + q, o + q + 1, P), sep<T>(x, beta, cu, o + q + 1, o + q + 2, P),
                                  sep<T>(x, beta, cu, o + q + 2, o + q + 3, P), P, gt4);
    g = g + gt4[si - q];
    if (q == si) D = dd;
  }
  gv[3 * i] += value(g.x); gv[3 * i + 1] += value(g.y); gv[3 * i + 2] += value(g.z);
  if (gt) { gt[3 * i] += tangent(g.x); gt[3 * i + 1] += tangent(g.y); gt[3 * i + 2] += tangent(g.z); }
  double* R = rec + (size_t)kRec * i;
  R[kD] = value(D);
  R[kD + 1] = tangent(D);
  R[kEb] = eb;
  R[kEa] = ea;
  R[kEd] = P.kphi * value(D);
  double r2 = 0.0;
  if (si == 0) {
    const int l = o + P.sites - 1;
    const double ex = x[3 * l] - x[3 * o], ey = x[3 * l + 1] - x[3 * o + 1], ez = x[3 * l + 2] - x[3 * o + 2];
    r2 = ex * ex + ey * ey + ez * ez;
  }
  R[kR2] = r2;
}

// ------------------------------------------------------------------ reductions (fixed order)
constexpr int kRedBlocks = 64, kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
  return s;   // valid on thread 0
}

// stage 1: block b sums a contiguous range of atoms, field by field
__global__ void __launch_bounds__(kRedThreads) k_adj_reduce1(const double* __restrict__ rec, int N,
                                                             double* __restrict__ part) {
  __shared__ double sh[kRedThreads / 32];
  const int per = (N + gridDim.x - 1) / gridDim.x;
  const int b = blockIdx.x * per, e = min(b + per, N);
  for (int f = 0; f < kFields; ++f) {
    double s = 0.0;
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) s += rec[(size_t)kRec * i + f];
    const double t = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x * kRec + f] = t;
  }
}

// accumulator layout
constexpr int kAccU = 0, kAccR2 = 1;      // forward sums of U_k and R_ee^2_k
constexpr int kAccC12 = 2, kAccC6 = 5;    // dJ/dc12_t, dJ/dc6_t (t = 0, 1, 2)
constexpr int kAccKphi = 8;               // dJ/dk_phi
constexpr int kAccN = 16;

// stage 2: totals of each field; mode 0 = forward sums, 1 = reverse step
// (wu = w_k w0, the weight of U at this step), 2 = totals only
__global__ void __launch_bounds__(32) k_adj_reduce2(const double* __restrict__ part, int nb, int n_chains, int mode,
                                                    double wu, double* __restrict__ totals,
                                                    double* __restrict__ acc) {
  const int f = threadIdx.x;
  if (f < kFields) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b * kRec + f];
    totals[f] = s;
  }
  __syncwarp();
  if (threadIdx.x != 0) return;
  if (mode == 0) {
    acc[kAccU] += totals[kElj] + totals[kEb] + totals[kEa] + totals[kEd];
    acc[kAccR2] += totals[kR2] / (double)n_chains;
  } else if (mode == 1) {
    for (int t = 0; t < 3; ++t) {
      // U = sum_t (c12_t A_t - c6_t B_t) + bonded; the mixed term is the
      // tangent of the same sums along u
      acc[kAccC12 + t] += wu * totals[kA + 4 * t + 0] - totals[kA + 4 * t + 1];
      acc[kAccC6 + t] += -wu * totals[kA + 4 * t + 2] + totals[kA + 4 * t + 3];
    }
    acc[kAccKphi] += wu * totals[kD] - totals[kD + 1];
  }
}

// ------------------------------------------------------------------ integrator and adjoint updates
// Make every chain continuous (one thread per chain, x,y,z per atom): site k
// is moved by whole box lengths, L s_k, where s_k accumulates -rint(d / L)
// over the bonds d = x_k - x_{k-1} of the positions as given, so each bond
// becomes its minimum image.  A site with s_k = 0 keeps its bits.
__global__ void __launch_bounds__(128) k_adj_unwrap(double* __restrict__ x, AdjDev P) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.n_chains) return;
  double* xc = x + 3 * (size_t)c * P.sites;
  double prev[3] = {xc[0], xc[1], xc[2]};
  double s[3] = {0.0, 0.0, 0.0};
  for (int k = 1; k < P.sites; ++k) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double cur = xc[3 * k + a];
      s[a] -= rint((cur - prev[a]) * P.inv_L);
      prev[a] = cur;
      if (s[a] != 0.0) xc[3 * k + a] = cur + P.L * s[a];
    }
  }
}

__global__ void __launch_bounds__(256) k_adj_kick_drift(double* __restrict__ x, double* __restrict__ v,
                                                        const double* __restrict__ gv, AdjDev P, double dt,
                                                        double* __restrict__ x_store) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const double hm = 0.5 * dt * P.inv_mass[site_type(i % P.sites, P.sites)];
  for (int q = 0; q < 3; ++q) {
    const double vh = v[3 * i + q] - hm * gv[3 * i + q];
    v[3 * i + q] = vh;
    x[3 * i + q] += dt * vh;
    if (x_store) x_store[3 * i + q] = x[3 * i + q];
  }
}

__global__ void __launch_bounds__(256) k_adj_kick(double* __restrict__ v, const double* __restrict__ gv, AdjDev P,
                                                  double dt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const double hm = 0.5 * dt * P.inv_mass[site_type(i % P.sites, P.sites)];
  for (int q = 0; q < 3; ++q) v[3 * i + q] -= hm * gv[3 * i + q];
}

// alpha = wu grad U + wr grad R_ee^2 + alpha - H u;  beta += dt alpha (if update_beta)
__global__ void __launch_bounds__(256) k_adj_update(const double* __restrict__ x, const double* __restrict__ gv,
                                                    const double* __restrict__ gt, AdjDev P, double wu, double wr,
                                                    double dt, int update_beta, double* __restrict__ alpha,
                                                    double* __restrict__ beta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const int si = i % P.sites, o = i - si, l = o + P.sites - 1;
  double gr[3] = {0.0, 0.0, 0.0};
  if (si == 0 || si == P.sites - 1) {
    const double sgn = (si == 0 ? -2.0 : 2.0) / (double)P.n_chains;
    for (int q = 0; q < 3; ++q) gr[q] = sgn * (x[3 * l + q] - x[3 * o + q]);
  }
  for (int q = 0; q < 3; ++q) {
    const double a = wu * gv[3 * i + q] + wr * gr[q] + alpha[3 * i + q] - gt[3 * i + q];
    alpha[3 * i + q] = a;
    if (update_beta) beta[3 * i + q] += dt * a;
  }
}

}  // namespace adj
}  // namespace mdg

using namespace mdg;
using namespace mdg::adj;

// ------------------------------------------------------------------ handle
struct md_adj {
  AdjDev P;
  double theta[5];
  double dt;
  int K, C, S;                 // steps, checkpoint interval, segments
  cudaStream_t st;
  bool own_stream;
  int C_cells;
  bool hvp32;                  // Hessian-vector products in FP32 (md_adj_desc.hvp_precision = 1)
  // device buffers (one allocation)
  void* mem;
  double *x, *v, *gv, *gt, *alpha, *beta, *rec, *part, *acc, *totals, *ckx, *ckv, *seg, *xk;
  float4* x32;
  int *count, *cell_start, *cell_of, *slot, *tmp, *perm, *rbuf, *maxm;
  bool have_forward;
  double obs[2];
};

namespace {

int adj_fail(int code, const char* msg) {
  md_set_global_error(msg);
  return code;
}

void set_pair_coefficients(md_adj* a) {
  const double eps[2] = {a->theta[0], a->theta[1]}, sig[2] = {a->theta[2], a->theta[3]};
  const int ta[3] = {0, 0, 1}, tb[3] = {0, 1, 1};
  for (int t = 0; t < 3; ++t) {
    const double e = std::sqrt(eps[ta[t]] * eps[tb[t]]), s = std::sqrt(sig[ta[t]] * sig[tb[t]]);
    const double s6 = s * s * s * s * s * s;
    a->P.c6[t] = 4.0 * e * s6;
    a->P.c12[t] = 4.0 * e * s6 * s6;
  }
  a->P.kphi = a->theta[4];
}

// one evaluation at positions xp: gradient (and, with beta, its tangent
// along cu M^-1 beta) plus the per-atom record, then the reductions
int evaluate(md_adj* a, const double* xp, const double* beta, double cu, int mode, double wu) {
  const AdjDev& P = a->P;
  cudaStream_t st = a->st;
  const int N = P.N;
  if (cudaMemsetAsync(a->count, 0, sizeof(int) * a->C_cells, st) != cudaSuccess) return MD_ECUDA;
  k_adj_count<<<(N + 255) / 256, 256, 0, st>>>(xp, P, a->cell_of, a->count, a->slot, a->x32);
  launch_scan(a->count, a->cell_start, a->C_cells, st);
  launch_bin_scatter(a->cell_of, a->slot, a->cell_start, a->tmp, N, st);
  if (cudaMemsetAsync(a->maxm, 0, sizeof(int), st) != cudaSuccess) return MD_ECUDA;
  launch_static_order(a->cell_start, a->C_cells, N, a->tmp, a->rbuf, a->slot, a->perm, a->maxm, st);
  const int lj_blocks = (N + kLjWarps - 1) / kLjWarps;
  if (beta && a->hvp32) {
    k_adj_lj<DualF><<<lj_blocks, 32 * kLjWarps, 0, st>>>(xp, beta, cu, a->cell_start, a->perm, P, a->x32, a->gv,
                                                           a->gt, a->rec);
    k_adj_bonded<DualF><<<(N + 127) / 128, 128, 0, st>>>(xp, beta, cu, P, a->gv, a->gt, a->rec);
  } else if (beta) {
    k_adj_lj<Dual><<<lj_blocks, 32 * kLjWarps, 0, st>>>(xp, beta, cu, a->cell_start, a->perm, P, a->x32, a->gv,
                                                          a->gt, a->rec);
    k_adj_bonded<Dual><<<(N + 127) / 128, 128, 0, st>>>(xp, beta, cu, P, a->gv, a->gt, a->rec);
  } else {
    k_adj_lj<double><<<lj_blocks, 32 * kLjWarps, 0, st>>>(xp, nullptr, 0.0, a->cell_start, a->perm, P, a->x32,
                                                            a->gv, nullptr, a->rec);
    k_adj_bonded<double><<<(N + 127) / 128, 128, 0, st>>>(xp, nullptr, 0.0, P, a->gv, nullptr, a->rec);
  }
  const int nb = N < kRedBlocks ? 1 : kRedBlocks;
  k_adj_reduce1<<<nb, kRedThreads, 0, st>>>(a->rec, N, a->part);
  k_adj_reduce2<<<1, 32, 0, st>>>(a->part, nb, P.n_chains, mode, wu, a->totals, a->acc);
  return cudaPeekAtLastError() == cudaSuccess ? MD_OK : MD_ECUDA;
}

// (dJ/dc12_t, dJ/dc6_t, dJ/dk_phi) -> (eps_C32, eps_C33, sigma_C32, sigma_C33, k_phi)
void chain_rule(const md_adj* a, const double* acc, double* grad) {
  const double eps[2] = {a->theta[0], a->theta[1]}, sig[2] = {a->theta[2], a->theta[3]};
  const int ta[3] = {0, 0, 1}, tb[3] = {0, 1, 1};
  for (int k = 0; k < 4; ++k) grad[k] = 0.0;
  for (int t = 0; t < 3; ++t) {
    const double e = std::sqrt(eps[ta[t]] * eps[tb[t]]), s = std::sqrt(sig[ta[t]] * sig[tb[t]]);
    const double c6 = a->P.c6[t], c12 = a->P.c12[t];
    const double dJ_de = (acc[kAccC12 + t] * c12 + acc[kAccC6 + t] * c6) / e;
    const double dJ_ds = (12.0 * acc[kAccC12 + t] * c12 + 6.0 * acc[kAccC6 + t] * c6) / s;
    // d eps_t / d eps_a = eps_t / (2 eps_a) per appearance of a in the pair
    for (int side = 0; side < 2; ++side) {
      const int ty = side == 0 ? ta[t] : tb[t];
      grad[ty] += dJ_de * e / (2.0 * eps[ty]);
      grad[2 + ty] += dJ_ds * s / (2.0 * sig[ty]);
    }
  }
  grad[4] = acc[kAccKphi];
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Record the launches `body` enqueues on the adjoint's stream as one CUDA
// graph (the per-step launch sequence is replayed instead of re-launched).
template <class F>
bool capture(md_adj* a, cudaGraphExec_t* exec, F&& body) {
  *exec = nullptr;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(a->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return false;
  const int rc = body();
  const cudaError_t e = cudaStreamEndCapture(a->st, &g);
  if (rc != MD_OK || e != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return false;
  }
  const cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *exec = nullptr;
    cudaGetLastError();
    return false;
  }
  return true;
}

}  // namespace

extern "C" int md_adj_create(const md_adj_desc* d, md_adj** out) {
  if (!d || !out) return adj_fail(MD_EINVAL, "null argument");
  *out = nullptr;
  if (d->n_chains < 1 || d->sites_per_chain < 2 || d->sites_per_chain > 4096)
    return adj_fail(MD_EINVAL, "n_chains must be >= 1 and sites_per_chain 2 .. 4096");
  const long long N = (long long)d->n_chains * d->sites_per_chain;
  if (N > (1 << 22)) return adj_fail(MD_EINVAL, "more than 4,194,304 atoms");
  if (!(d->box > 0) || !std::isfinite(d->box) || !(d->rc > 0) || !(d->dt > 0))
    return adj_fail(MD_EINVAL, "box, rc and dt must be positive");
  if (d->n_steps < 0 || d->n_steps > 10000000 || d->checkpoint_every < 1)
    return adj_fail(MD_EINVAL, "n_steps must be 0 .. 1e7 and checkpoint_every >= 1");
  const md_params& p = d->params;
  if (!(p.mass[0] > 0) || !(p.mass[1] > 0) || !(p.eps[0] > 0) || !(p.eps[1] > 0) || !(p.sigma[0] > 0) ||
      !(p.sigma[1] > 0))
    return adj_fail(MD_EINVAL, "masses, eps and sigma must be positive");
  md_adj* a = new (std::nothrow) md_adj();
  if (!a) return adj_fail(MD_ENOMEM, "host allocation failed");
  AdjDev& P = a->P;
  P.L = d->box;
  P.inv_L = 1.0 / d->box;
  int M = (int)std::floor(d->box / d->rc);
  if (M > 256) M = 256;
  if (M < 3) M = 1;
  P.M = M;
  P.n_off = M >= 3 ? 27 : 1;
  P.inv_h = (double)M / d->box;
  P.sites = d->sites_per_chain;
  P.n_chains = d->n_chains;
  P.N = (int)N;
  P.rc2 = d->rc * d->rc;
  const double irc2 = 1.0 / P.rc2;
  P.irc6 = irc2 * irc2 * irc2;
  P.irc12 = P.irc6 * P.irc6;
  P.rc = d->rc;
  P.irc7 = P.irc6 / d->rc;
  P.irc13 = P.irc12 / d->rc;
  if (d->lj_form != 0 && d->lj_form != 1) {
    delete a;
    return adj_fail(MD_EINVAL, "lj_form must be 0 or 1");
  }
  P.sf = d->lj_form;
  if (d->hvp_precision != 0 && d->hvp_precision != 1) {
    delete a;
    return adj_fail(MD_EINVAL, "hvp_precision must be 0 (FP64) or 1 (FP32)");
  }
  a->hvp32 = d->hvp_precision == 1;
  P.pre2 = (float)((d->rc + 1e-4) * (d->rc + 1e-4));
  P.kb = p.kb; P.b0 = p.b0; P.ka = p.ka; P.theta0 = p.theta0; P.phis = p.phis; P.n_mult = p.n_mult;
  P.inv_mass[0] = 1.0 / p.mass[0];
  P.inv_mass[1] = 1.0 / p.mass[1];
  a->theta[0] = p.eps[0]; a->theta[1] = p.eps[1]; a->theta[2] = p.sigma[0]; a->theta[3] = p.sigma[1];
  a->theta[4] = p.kphi;
  set_pair_coefficients(a);
  a->dt = d->dt;
  a->K = d->n_steps;
  a->C = d->checkpoint_every < d->n_steps ? d->checkpoint_every : (d->n_steps > 0 ? d->n_steps : 1);
  a->S = d->n_steps == 0 ? 1 : (d->n_steps + a->C - 1) / a->C;
  a->C_cells = M * M * M;
  a->st = (cudaStream_t)d->cuda_stream;
  a->own_stream = false;
  if (!a->st) {
    if (cudaStreamCreateWithFlags(&a->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete a;
      return adj_fail(MD_ECUDA, "stream creation failed");
    }
    a->own_stream = true;
  }
  const size_t n3 = sizeof(double) * 3 * (size_t)N;
  const size_t sizes[] = {n3, n3, n3, n3, n3, n3, sizeof(double) * kRec * (size_t)N,
                          sizeof(double) * kRec * kRedBlocks, sizeof(double) * kAccN, sizeof(double) * kRec,
                          n3 * a->S, n3 * a->S, n3 * (size_t)(a->C + 1), sizeof(int) * a->C_cells,
                          sizeof(int) * (a->C_cells + 1), sizeof(int) * (size_t)N, sizeof(int) * (size_t)N,
                          sizeof(int) * (size_t)N, sizeof(int) * (size_t)N, n3, sizeof(float4) * (size_t)N,
                          sizeof(int) * (size_t)N, sizeof(int)};
  const int nbuf = sizeof(sizes) / sizeof(sizes[0]);
  size_t total = 0;
  for (int k = 0; k < nbuf; ++k) total += align256(sizes[k]);
  if (cudaMalloc(&a->mem, total) != cudaSuccess) {
    cudaGetLastError();
    if (a->own_stream) cudaStreamDestroy(a->st);
    delete a;
    return adj_fail(MD_ENOMEM, "device allocation for the adjoint failed");
  }
  char* m = (char*)a->mem;
  void* ptrs[nbuf];
  for (int k = 0; k < nbuf; ++k) { ptrs[k] = m; m += align256(sizes[k]); }
  a->x = (double*)ptrs[0]; a->v = (double*)ptrs[1]; a->gv = (double*)ptrs[2]; a->gt = (double*)ptrs[3];
  a->alpha = (double*)ptrs[4]; a->beta = (double*)ptrs[5]; a->rec = (double*)ptrs[6]; a->part = (double*)ptrs[7];
  a->acc = (double*)ptrs[8]; a->totals = (double*)ptrs[9]; a->ckx = (double*)ptrs[10]; a->ckv = (double*)ptrs[11];
  a->seg = (double*)ptrs[12]; a->count = (int*)ptrs[13]; a->cell_start = (int*)ptrs[14];
  a->cell_of = (int*)ptrs[15]; a->slot = (int*)ptrs[16]; a->tmp = (int*)ptrs[17]; a->perm = (int*)ptrs[18];
  a->xk = (double*)ptrs[19];
  a->x32 = (float4*)ptrs[20];
  a->rbuf = (int*)ptrs[21]; a->maxm = (int*)ptrs[22];
  a->have_forward = false;
  *out = a;
  return MD_OK;
}

extern "C" int md_adj_set_theta(md_adj* a, const double theta[5]) {
  if (!a || !theta) return adj_fail(MD_EINVAL, "null argument");
  for (int k = 0; k < 5; ++k)
    if (!std::isfinite(theta[k]) || (k < 4 && !(theta[k] > 0))) return adj_fail(MD_EINVAL, "eps and sigma must be positive");
  std::memcpy(a->theta, theta, sizeof(a->theta));
  set_pair_coefficients(a);
  a->have_forward = false;
  return MD_OK;
}

extern "C" int md_adj_forward(md_adj* a, const double* pos, const double* vel, double obs[2]) {
  if (!a || !pos || !vel) return adj_fail(MD_EINVAL, "null argument");
  const size_t n3 = sizeof(double) * 3 * (size_t)a->P.N;
  cudaStream_t st = a->st;
  if (cudaMemcpyAsync(a->x, pos, n3, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaMemcpyAsync(a->v, vel, n3, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaMemsetAsync(a->acc, 0, sizeof(double) * kAccN, st) != cudaSuccess)
    return adj_fail(MD_ECUDA, "upload of the initial state failed");
  k_adj_unwrap<<<(a->P.n_chains + 127) / 128, 128, 0, st>>>(a->x, a->P);
  const int nb = (a->P.N + 255) / 256;
  if (evaluate(a, a->x, nullptr, 0.0, 0, 0.0) != MD_OK) return adj_fail(MD_ECUDA, "force evaluation failed");
  // one velocity-Verlet step (kick-drift, forces and sums, kick) as a graph
  cudaGraphExec_t step = nullptr;
  if (a->K > 0 && !capture(a, &step, [&]() {
        k_adj_kick_drift<<<nb, 256, 0, st>>>(a->x, a->v, a->gv, a->P, a->dt, nullptr);
        const int rc = evaluate(a, a->x, nullptr, 0.0, 0, 0.0);
        k_adj_kick<<<nb, 256, 0, st>>>(a->v, a->gv, a->P, a->dt);
        return rc;
      }))
    return adj_fail(MD_ECUDA, "capturing the forward step failed");
  int grc = MD_OK;
  for (int k = 0; k < a->K && grc == MD_OK; ++k) {
    if (k % a->C == 0) {
      const size_t s = (size_t)(k / a->C);
      cudaMemcpyAsync(a->ckx + s * 3 * a->P.N, a->x, n3, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(a->ckv + s * 3 * a->P.N, a->v, n3, cudaMemcpyDeviceToDevice, st);
    }
    if (cudaGraphLaunch(step, st) != cudaSuccess) grc = MD_ECUDA;
  }
  if (step) cudaGraphExecDestroy(step);
  if (grc != MD_OK) return adj_fail(MD_ECUDA, "forward step launch failed");
  if (a->K == 0) {
    cudaMemcpyAsync(a->ckx, a->x, n3, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a->ckv, a->v, n3, cudaMemcpyDeviceToDevice, st);
  }
  double acc[2];
  if (cudaMemcpyAsync(acc, a->acc, sizeof(acc), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return adj_fail(MD_ECUDA, "forward run failed");
  a->obs[0] = acc[0] / (double)(a->K + 1);
  a->obs[1] = acc[1] / (double)(a->K + 1);
  if (!std::isfinite(a->obs[0]) || !std::isfinite(a->obs[1])) return adj_fail(MD_EUNSTABLE, "non-finite observable");
  a->have_forward = true;
  if (obs) { obs[0] = a->obs[0]; obs[1] = a->obs[1]; }
  return MD_OK;
}

extern "C" int md_adj_backward(md_adj* a, const double weight[2], double grad[5]) {
  if (!a || !weight || !grad) return adj_fail(MD_EINVAL, "null argument");
  if (!a->have_forward) return adj_fail(MD_EINVAL, "md_adj_backward needs md_adj_forward at the current parameters");
  const AdjDev& P = a->P;
  const size_t n3 = sizeof(double) * 3 * (size_t)P.N;
  const size_t stride = 3 * (size_t)P.N;
  cudaStream_t st = a->st;
  const int nb = (P.N + 255) / 256;
  const double w = 1.0 / (double)(a->K + 1);
  const double wu = w * weight[0], wr = w * weight[1];
  if (cudaMemsetAsync(a->alpha, 0, n3, st) != cudaSuccess || cudaMemsetAsync(a->beta, 0, n3, st) != cudaSuccess ||
      cudaMemsetAsync(a->acc, 0, sizeof(double) * kAccN, st) != cudaSuccess)
    return adj_fail(MD_ECUDA, "clearing the adjoint state failed");
  // graphs: a recomputed forward step, and a reverse step with c_k = dt at
  // positions copied to xk (the steps k = K and k = 0 are launched directly)
  cudaGraphExec_t rec_step = nullptr, rev_step = nullptr;
  const bool have_graphs =
      capture(a, &rec_step, [&]() {
        k_adj_kick_drift<<<nb, 256, 0, st>>>(a->x, a->v, a->gv, P, a->dt, nullptr);
        const int rc = evaluate(a, a->x, nullptr, 0.0, 2, 0.0);
        k_adj_kick<<<nb, 256, 0, st>>>(a->v, a->gv, P, a->dt);
        return rc;
      }) &&
      capture(a, &rev_step, [&]() {
        const int rc = evaluate(a, a->xk, a->beta, a->dt, 1, wu);
        k_adj_update<<<nb, 256, 0, st>>>(a->xk, a->gv, a->gt, P, wu, wr, a->dt, 1, a->alpha, a->beta);
        return rc;
      });
  if (!have_graphs) {
    if (rec_step) cudaGraphExecDestroy(rec_step);
    if (rev_step) cudaGraphExecDestroy(rev_step);
    return adj_fail(MD_ECUDA, "capturing the adjoint steps failed");
  }
  struct GraphGuard {
    cudaGraphExec_t a, b;
    ~GraphGuard() { cudaGraphExecDestroy(a); cudaGraphExecDestroy(b); }
  } guard{rec_step, rev_step};
  for (int s = a->S - 1; s >= 0; --s) {
    const int k0 = s * a->C, k1 = (k0 + a->C < a->K) ? k0 + a->C : a->K;
    // recompute the segment's positions from its checkpoint
    cudaMemcpyAsync(a->x, a->ckx + s * stride, n3, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a->v, a->ckv + s * stride, n3, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(a->seg, a->x, n3, cudaMemcpyDeviceToDevice, st);
    if (k1 > k0 && evaluate(a, a->x, nullptr, 0.0, 2, 0.0) != MD_OK)
      return adj_fail(MD_ECUDA, "force evaluation failed");
    for (int k = k0; k < k1; ++k) {
      if (k + 1 < k1) {
        if (cudaGraphLaunch(rec_step, st) != cudaSuccess) return adj_fail(MD_ECUDA, "recompute step launch failed");
        cudaMemcpyAsync(a->seg + (size_t)(k - k0 + 1) * stride, a->x, n3, cudaMemcpyDeviceToDevice, st);
      } else {
        k_adj_kick_drift<<<nb, 256, 0, st>>>(a->x, a->v, a->gv, P, a->dt, a->seg + (size_t)(k - k0 + 1) * stride);
      }
    }
    // reverse steps k1 .. k0 + 1 (and 0 in the first segment)
    const int k_lo = s == 0 ? 0 : k0 + 1;
    for (int k = k1; k >= k_lo; --k) {
      const double* xk = a->seg + (size_t)(k - k0) * stride;
      if (k != a->K && k != 0) {
        cudaMemcpyAsync(a->xk, xk, n3, cudaMemcpyDeviceToDevice, st);
        if (cudaGraphLaunch(rev_step, st) != cudaSuccess) return adj_fail(MD_ECUDA, "reverse step launch failed");
        continue;
      }
      const double ck = k == a->K ? 0.0 : 0.5 * a->dt;
      if (evaluate(a, xk, a->beta, ck, 1, wu) != MD_OK) return adj_fail(MD_ECUDA, "tangent evaluation failed");
      k_adj_update<<<nb, 256, 0, st>>>(xk, a->gv, a->gt, P, wu, wr, a->dt, k >= 1 ? 1 : 0, a->alpha, a->beta);
    }
  }
  double acc[kAccN];
  if (cudaMemcpyAsync(acc, a->acc, sizeof(acc), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return adj_fail(MD_ECUDA, "reverse run failed");
  chain_rule(a, acc, grad);
  for (int k = 0; k < 5; ++k)
    if (!std::isfinite(grad[k])) return adj_fail(MD_EUNSTABLE, "non-finite gradient");
  return MD_OK;
}

extern "C" int md_adj_tangent(md_adj* a, const double* pos, const double* dir, double* grad_u, double* hvp,
                              double dtheta[10]) {
  if (!a || !pos || !dir) return adj_fail(MD_EINVAL, "null argument");
  const AdjDev& P = a->P;
  const size_t n3 = sizeof(double) * 3 * (size_t)P.N;
  cudaStream_t st = a->st;
  // the direction enters as cu M^-1 beta; store beta = M dir so that u = dir
  double* hb = (double*)std::malloc(n3);
  if (!hb) return adj_fail(MD_ENOMEM, "host allocation failed");
  for (int i = 0; i < P.N; ++i) {
    const int si = i % P.sites;
    const double m = 1.0 / P.inv_mass[(si == 0 || si == P.sites - 1) ? 1 : 0];
    for (int q = 0; q < 3; ++q) hb[3 * i + q] = m * dir[3 * i + q];
  }
  int rc = MD_OK;
  if (cudaMemcpyAsync(a->x, pos, n3, cudaMemcpyDefault, st) != cudaSuccess ||
      cudaMemcpyAsync(a->beta, hb, n3, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(a->acc, 0, sizeof(double) * kAccN, st) != cudaSuccess)
    rc = MD_ECUDA;
  // mode 1 with weight 1 gives dU/dtheta - d(grad U . u)/dtheta; mode 2 the totals alone
  if (rc == MD_OK) rc = evaluate(a, a->x, a->beta, 1.0, 2, 0.0);
  double tot[kRec];
  if (rc == MD_OK) {
    if ((grad_u && cudaMemcpyAsync(grad_u, a->gv, n3, cudaMemcpyDefault, st) != cudaSuccess) ||
        (hvp && cudaMemcpyAsync(hvp, a->gt, n3, cudaMemcpyDefault, st) != cudaSuccess) ||
        cudaMemcpyAsync(tot, a->totals, sizeof(tot), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      rc = MD_ECUDA;
  }
  std::free(hb);
  if (rc != MD_OK) return adj_fail(rc, "tangent evaluation failed");
  if (dtheta) {
    double acc[kAccN] = {0};
    // value part: dU/dtheta
    for (int t = 0; t < 3; ++t) { acc[kAccC12 + t] = tot[kA + 4 * t]; acc[kAccC6 + t] = -tot[kA + 4 * t + 2]; }
    acc[kAccKphi] = tot[kD];
    chain_rule(a, acc, dtheta);
    // tangent part: d(grad U . u)/dtheta
    for (int t = 0; t < 3; ++t) { acc[kAccC12 + t] = tot[kA + 4 * t + 1]; acc[kAccC6 + t] = -tot[kA + 4 * t + 3]; }
    acc[kAccKphi] = tot[kD + 1];
    chain_rule(a, acc, dtheta + 5);
  }
  return MD_OK;
}

extern "C" int md_adj_energy(md_adj* a, double out[6]) {
  // totals of the last evaluation: shifted LJ, bond, angle, dihedral, sum over chains of R_ee^2, U
  if (!a || !out) return adj_fail(MD_EINVAL, "null argument");
  double tot[kRec];
  if (cudaMemcpyAsync(tot, a->totals, sizeof(tot), cudaMemcpyDeviceToHost, a->st) != cudaSuccess ||
      cudaStreamSynchronize(a->st) != cudaSuccess)
    return adj_fail(MD_ECUDA, "copy of the totals failed");
  out[0] = tot[kElj]; out[1] = tot[kEb]; out[2] = tot[kEa]; out[3] = tot[kEd]; out[4] = tot[kR2];
  out[5] = tot[kElj] + tot[kEb] + tot[kEa] + tot[kEd];
  return MD_OK;
}

extern "C" void md_adj_destroy(md_adj* a) {
  if (!a) return;
  cudaStreamSynchronize(a->st);
  cudaFree(a->mem);
  if (a->own_stream) cudaStreamDestroy(a->st);
  delete a;
}
