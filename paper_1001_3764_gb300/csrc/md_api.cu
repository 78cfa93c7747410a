// md_api.cu -- host runtime and C ABI of the GB300 MD engine (include/md.h).
//
// One md_system owns: a replica table, tile tables, every device buffer (one
// allocation, or a caller workspace), a stream, and a CUDA graph holding one
// rebin cycle (rebin + neighbour list + rebin_every steps).  Kernels are in
// k_bin.cu (binning), k_lj.cu (neighbour list and Lennard-Jones), k_force.cu
// (bonded terms), k_integrate.cu (integration, kinetic energy, thermostats,
// energy reductions, observables, state transfer) and md_adjoint.cu (the
// adjoint); md_static.cu holds the allocation-free binning entry point.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <tuple>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/md.h"
#include "md_kernels.cuh"

using namespace mdg;

namespace {

constexpr int kIntTile = 224;    // atoms per integrator / bonded block (original order)
constexpr int kNumProf = 5;      // rebin, neighbour build, integrate, lj, bonded
constexpr double kKB = 0.0083144626;

thread_local std::string g_create_error;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

struct md_system {
  // configuration
  int n_reps = 0, S = 0, R = 10;
  int64_t N = 0;
  int C = 0, Npad = 0, cap = 0;
  bool mixed = false;
  int thermo = 0;                 // MD_NVE, MD_VRESCALE or MD_NOSE_HOOVER
  double dt = 0, rc = 0, skin = 0, tau = 0.1;
  md_params params{};
  ForceParams fp{};
  std::vector<RepDev> reps_h;
  std::vector<Tile> t_int;
  std::vector<double> T0;
  // memory
  char* base = nullptr;
  size_t bytes = 0;
  bool own_mem = false;
  RepDev* reps = nullptr;
  Tile* tiles_int = nullptr;
  void *x = nullptr, *v = nullptr, *F = nullptr;
  long long* flj = nullptr;                  // LJ force, int64 SoA [3][Npad], sorted order
  long long* flj_e = nullptr;                // the same for energy read-outs (kept apart from the dynamics)
  int* img = nullptr;
  uint16_t* site = nullptr;
  int *cellc = nullptr, *inv_perm = nullptr, *tag = nullptr, *perm = nullptr;
  float4 *ref = nullptr, *pos = nullptr;
  unsigned* list = nullptr;                  // cluster lists [n_cl_max][cap]
  int* ncl = nullptr;                        // entries per cluster
  int* cl_start = nullptr;                   // first cluster of each cell [C + 1]
  int64_t n_cl_max = 0;
  std::vector<Region> regions_h;
  std::vector<RegionShape> shapes_h;
  Region* regions = nullptr;
  RegionShape* shapes = nullptr;
  int tile_cap = 0;
  int lj_block = 256, persistent_grid = 0;   // persistent_grid > 0: fixed grid for the LJ kernel
  int lj_lanes = 8;                          // lanes per 4-atom cluster in the LJ kernel
  int lj_region = 3;                         // cells per side (x, y) of an LJ / list region
  bool lj_pair_exact = false;                // each LJ pair force converted once, +q to i and -q to j
  int* work = nullptr;                       // LJ work counters (persistent schedule)
  int *count = nullptr, *cell_start = nullptr, *cell_of = nullptr;
  int *slot = nullptr, *tmp = nullptr;
  double *lj_part = nullptr, *b_part = nullptr, *kepart = nullptr, *ke_out = nullptr, *lam = nullptr;
  double* e_out = nullptr;
  double* e_slices = nullptr;   // first-pass energy sums, n_reps * max_slices * 11
  int max_slices = 1;
  double* stage = nullptr;                   // input staging (6N doubles)
  unsigned *done = nullptr, *flags = nullptr;
  // end-to-end vector ACF (allocated by md_acf_reset)
  double *acf_ring = nullptr, *acf_acc = nullptr;
  int acf_lag = -1;
  int64_t acf_n = 0;
  // execution
  cudaStream_t st = nullptr;
  bool own_stream = false;
  cudaGraphExec_t cycle = nullptr;
  cudaGraphExec_t cycle_fresh = nullptr;     // the same cycle without its leading rebin + list
  std::vector<cudaGraphExec_t> rem_graphs;   // blocks of k < R steps (remainders), captured on first use
  cudaStream_t side = nullptr;               // captures the bodies of the conditional rebins
  unsigned long long* early = nullptr;       // early rebins (displacement beyond skin/2) so far
  // a general molecule type (md_desc.topology), or linear chains
  bool generic = false;
  int disp = MD_DISP_REBUILD;                // what a displacement beyond skin/2 does
  std::vector<unsigned char> mtype_h;        // type of each atom of the molecule
  std::vector<int> t_boff, t_bat, t_aoff, t_aat, t_doff, t_dat, t_xoff, t_xat;   // term and exclusion lists
  unsigned char* mtype = nullptr;            // device copies
  TopoDev topo{};
  bool fresh = false;                        // bins, list and forces are those of the current positions
  bool profile = false;
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;
  double prof_ms[kNumProf] = {0, 0, 0, 0, 0};
  int64_t prof_n[kNumProf] = {0, 0, 0, 0, 0};
  std::string err;
};

void md_set_global_error(const char* msg) { g_create_error = msg; }

// ------------------------------------------------------------------ helpers
static int fail(md_system* s, int code, const std::string& msg) {
  if (s) s->err = msg; else g_create_error = msg;
  return code;
}
#define CU(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) return fail(s, MD_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

static void fill_force_params(md_system* s) {
  const md_params& p = s->params;
  ForceParams& f = s->fp;
  for (RepDev& q : s->reps_h)
    for (int t = 0; t < 3; ++t) {
      const int a = t >= 1 ? 1 : 0, b = t >= 2 ? 1 : 0;
      const int ta = (t == 1) ? 0 : a;   // pair (0,1) for t = 1
      const int tb = (t == 1) ? 1 : b;
      double eps = std::sqrt(p.eps[ta] * p.eps[tb]);
      double sig = std::sqrt(p.sigma[ta] * p.sigma[tb]) * q.inv_h;   // sigma in cell units
      double s6 = sig * sig * sig * sig * sig * sig;
      q.C6u[t] = (float)(4.0 * eps * s6);
      q.C12u[t] = (float)(4.0 * eps * s6 * s6);
    }
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double eps = std::sqrt(p.eps[a] * p.eps[b]);
      double sig = std::sqrt(p.sigma[a] * p.sigma[b]);
      double s6 = sig * sig * sig * sig * sig * sig;
      double c6 = 4.0 * eps * s6, c12 = 4.0 * eps * s6 * s6;
      double ir6 = 1.0 / (s->rc * s->rc * s->rc * s->rc * s->rc * s->rc);
      f.c6[a][b] = (float)c6;
      f.c12[a][b] = (float)c12;
      f.erc[a][b] = (float)(c12 * ir6 * ir6 - c6 * ir6);
    }
  f.rc2 = (float)(s->rc * s->rc);
  f.rlist2 = (float)((s->rc + s->skin) * (s->rc + s->skin));
  f.kb = (float)p.kb; f.b0 = (float)p.b0; f.ka = (float)p.ka; f.theta0 = (float)p.theta0;
  f.kphi = (float)p.kphi; f.phis = (float)p.phis; f.n_mult = p.n_mult;
  f.sites = s->S;
  f.half_skin2 = (float)(0.25 * s->skin * s->skin);
  f.b0sq = p.b0 * p.b0;
  f.b0sq_hi = (float)f.b0sq;
  f.b0sq_lo = (float)(f.b0sq - (double)f.b0sq_hi);
  for (int a = 0; a < 2; ++a) {
    f.mass[a] = p.mass[a];
    f.inv_mass[a] = 1.0 / p.mass[a];
    f.hdt_m[a] = 0.5 * s->dt / p.mass[a];
    f.hdt_m_fix[a] = f.hdt_m[a] * kFixInv;
    f.hdt_m_f[a] = (float)f.hdt_m[a];
  }
  f.dt_f = (float)s->dt;
  f.dt = s->dt;
  if (s->generic) {
    double mm = 0.0;
    for (unsigned char t : s->mtype_h) mm += p.mass[t];
    f.mol_mass = mm;
  } else {
    f.mol_mass = (double)(s->S - 2) * p.mass[0] + 2.0 * p.mass[1];
  }
  f.mtype = s->generic ? s->mtype : nullptr;
}

// Region shapes: sx x sy x 1 home cells (sx, sy in {1, 2}; shape id
// (sx - 1) + 2 (sy - 1)).  The tile lists the home cells first, then every
// cell that a home cell's 13 forward offsets reach, in the order first met;
// nb[h] gives home cell h's own tile cell and its 13 forward tile cells, in
// the offset order (dz = +1 layer, then dz = 0, dy = +1, then (+1, 0, 0)).
static RegionShape make_shape(int sx, int sy) {
  RegionShape S{};
  std::vector<std::array<int, 3>> tile;
  for (int y = 0; y < sy; ++y)
    for (int x = 0; x < sx; ++x) tile.push_back({x, y, 0});
  S.n_home = sx * sy;
  std::vector<std::array<int, 3>> fw;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx)
        if (dz > 0 || (dz == 0 && dy > 0) || (dz == 0 && dy == 0 && dx > 0)) fw.push_back({dx, dy, dz});
  std::sort(fw.begin(), fw.end(), [](const std::array<int, 3>& a, const std::array<int, 3>& b) {
    return std::make_tuple(-a[2], -a[1], a[0]) < std::make_tuple(-b[2], -b[1], b[0]);
  });
  for (int h = 0; h < S.n_home; ++h) {
    S.nb[h][0] = (unsigned char)h;
    for (int q = 0; q < 13; ++q) {
      const std::array<int, 3> c = {tile[h][0] + fw[q][0], tile[h][1] + fw[q][1], tile[h][2] + fw[q][2]};
      int k = 0;
      while (k < (int)tile.size() && tile[k] != c) ++k;
      if (k == (int)tile.size()) tile.push_back(c);
      S.nb[h][q + 1] = (unsigned char)k;
    }
  }
  S.n_tile = (int)tile.size();
  for (int k = 0; k < S.n_tile; ++k)
    for (int a = 0; a < 3; ++a) S.off[k][a] = (signed char)tile[k][a];
  S.cx = 0.5f * (float)(sx - 1);
  S.cy = 0.5f * (float)(sy - 1);
  S.cz = 0.f;
  return S;
}

// The per-type lists of Sec. 3.3 from a molecule's bond graph: each atom's
// neighbours (ascending); exclusions = 1-2 and 1-3 neighbours; angles = every
// path a-b-c (vertex b, a < c), listed under a; dihedrals = every path
// a-b-c-d around each bond b-c (in bond order, b < c), listed under a; bonds
// listed under their first atom as given.
static int build_topology(md_system* s, const md_topology* t) {
  const int n = t->naom;
  if (n < 4 || n > 1023) return fail(s, MD_EINVAL, "topology: naom must be 4 .. 1023");
  if (t->n_bonds < 1 || t->n_bonds > 4 * n || !t->bonds || !t->types)
    return fail(s, MD_EINVAL, "topology: 1 .. 4 naom bonds, bonds and types required");
  std::vector<std::vector<int>> nb(n);
  std::vector<std::pair<int, int>> bl;
  for (int k = 0; k < t->n_bonds; ++k) {
    const int a = t->bonds[2 * k], b = t->bonds[2 * k + 1];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) return fail(s, MD_EINVAL, "topology: bond atom out of range");
    for (int c : nb[a])
      if (c == b) return fail(s, MD_EINVAL, "topology: repeated bond");
    nb[a].push_back(b);
    nb[b].push_back(a);
    bl.push_back({a, b});
  }
  for (auto& v : nb) std::sort(v.begin(), v.end());
  s->mtype_h.assign(n, 0);
  for (int a = 0; a < n; ++a) {
    if (t->types[a] != 0 && t->types[a] != 1) return fail(s, MD_EINVAL, "topology: types must be 0 or 1");
    s->mtype_h[a] = (unsigned char)t->types[a];
  }
  std::vector<std::vector<int>> ob(n), oa(n), od(n), ex(n);
  for (auto& e : bl) ob[e.first].push_back(e.second);
  for (int b = 0; b < n; ++b)
    for (size_t p = 0; p < nb[b].size(); ++p)
      for (size_t q = p + 1; q < nb[b].size(); ++q) {
        oa[nb[b][p]].push_back(b);
        oa[nb[b][p]].push_back(nb[b][q]);
      }
  for (auto& e : bl) {
    const int b = std::min(e.first, e.second), c = std::max(e.first, e.second);
    for (int a : nb[b]) {
      if (a == c) continue;
      for (int d : nb[c]) {
        if (d == b || d == a) continue;
        od[a].push_back(b); od[a].push_back(c); od[a].push_back(d);
      }
    }
  }
  for (int a = 0; a < n; ++a) {
    for (int b : nb[a]) {
      ex[a].push_back(b);
      for (int c : nb[b])
        if (c != a) ex[a].push_back(c);
    }
    std::sort(ex[a].begin(), ex[a].end());
    ex[a].erase(std::unique(ex[a].begin(), ex[a].end()), ex[a].end());
  }
  auto csr = [n](const std::vector<std::vector<int>>& v, std::vector<int>& off, std::vector<int>& at) {
    off.assign(n + 1, 0);
    at.clear();
    for (int a = 0; a < n; ++a) { at.insert(at.end(), v[a].begin(), v[a].end()); off[a + 1] = (int)at.size(); }
    if (at.empty()) at.push_back(0);
  };
  csr(ob, s->t_boff, s->t_bat);
  csr(oa, s->t_aoff, s->t_aat);
  csr(od, s->t_doff, s->t_dat);
  csr(ex, s->t_xoff, s->t_xat);
  // the CSR offsets of angles and dihedrals count ints; the kernels index terms
  for (int& o : s->t_aoff) o /= 2;
  for (int& o : s->t_doff) o /= 3;
  return MD_OK;
}

// Validate the descriptor and fill geometry, tiles and sizes (no device work).
static int configure(md_system* s, const md_desc* d) {
  if (!d) return fail(s, MD_EINVAL, "null descriptor");
  if (d->n_replicas < 1 || d->n_replicas > kMaxReplicas) return fail(s, MD_EINVAL, "n_replicas out of range");
  // chains: the packed tags keep the site in 10 bits, and the last site of one
  // chain must stay more than 2 away from the next chain's first (1024 - S + 1 > 2)
  if (d->sites_per_chain < 4 || d->sites_per_chain > (d->topology ? 1023 : 1022))
    return fail(s, MD_EINVAL, "sites_per_chain must be 4..1022 (4..1023 with a topology)");
  s->generic = d->topology != nullptr;
  if (s->generic) {
    if (d->topology->naom != d->sites_per_chain) return fail(s, MD_EINVAL, "sites_per_chain must equal topology->naom");
    if (d->precision != MD_MIXED) return fail(s, MD_EINVAL, "a molecule topology needs the mixed precision form");
    const int rc = build_topology(s, d->topology);
    if (rc) return rc;
  } else {
    s->mtype_h.assign(d->sites_per_chain, 0);
    s->mtype_h[0] = s->mtype_h[d->sites_per_chain - 1] = 1;
  }
  if (!d->n_chains || !d->box) return fail(s, MD_EINVAL, "n_chains and box are required");
  if (!(d->dt > 0) || !(d->rc > 0) || !(d->skin >= 0) || d->rebin_every < 1)
    return fail(s, MD_EINVAL, "dt, rc must be > 0, skin >= 0, rebin_every >= 1");
  if (d->precision != MD_PLAIN_FP32 && d->precision != MD_MIXED) return fail(s, MD_EINVAL, "unknown precision");
  if (d->thermostat != MD_NVE && d->thermostat != MD_VRESCALE && d->thermostat != MD_NOSE_HOOVER)
    return fail(s, MD_EINVAL, "unknown thermostat");
  if (d->thermostat != MD_NVE && (!d->T_target || !(d->tau_t > 0)))
    return fail(s, MD_EINVAL, "thermostat needs T_target and tau_t > 0");
  for (int a = 0; a < 2; ++a)
    if (!(d->params.mass[a] > 0) || !(d->params.sigma[a] > 0) || !(d->params.eps[a] >= 0))
      return fail(s, MD_EINVAL, "masses and sigmas must be > 0, eps >= 0");
  if (d->params.n_mult < 0 || d->params.n_mult > 12) return fail(s, MD_EINVAL, "n_mult out of range");
  s->n_reps = d->n_replicas;
  s->S = d->sites_per_chain;
  s->R = d->rebin_every;
  s->mixed = d->precision == MD_MIXED;
  s->thermo = d->thermostat;
  s->dt = d->dt; s->rc = d->rc; s->skin = d->skin; s->tau = d->thermostat ? d->tau_t : 0.1;
  if (d->lj_block != 0 && d->lj_block != 128 && d->lj_block != 256 && d->lj_block != 384)
    return fail(s, MD_EINVAL, "lj_block must be 0, 128, 256 or 384");
  if (d->schedule != MD_SCHED_GRID && d->schedule != MD_SCHED_PERSISTENT) return fail(s, MD_EINVAL, "unknown schedule");
  if (d->lj_lanes != 0 && d->lj_lanes != 8 && d->lj_lanes != 16 && d->lj_lanes != 32)
    return fail(s, MD_EINVAL, "lj_lanes must be 0, 8, 16 or 32");
  s->lj_lanes = d->lj_lanes ? d->lj_lanes : 8;
  if (d->lj_region != 0 && d->lj_region != 2 && d->lj_region != 3)
    return fail(s, MD_EINVAL, "lj_region must be 0, 2 or 3");
  s->lj_region = d->lj_region ? d->lj_region : 3;
  if (d->lj_pair_exact != 0 && d->lj_pair_exact != 1) return fail(s, MD_EINVAL, "lj_pair_exact must be 0 or 1");
  s->lj_pair_exact = d->lj_pair_exact == 1;
  // default block: two resident blocks of 12 warps for the 3 x 3 regions'
  // larger tiles, three of 8 warps for 2 x 2
  s->lj_block = d->lj_block ? d->lj_block : (s->lj_region == 3 ? 384 : 256);
  if (d->displacement != MD_DISP_REBUILD && d->displacement != MD_DISP_ERROR)
    return fail(s, MD_EINVAL, "displacement must be MD_DISP_REBUILD or MD_DISP_ERROR");
  s->disp = d->displacement;
  s->params = d->params;
  const double rl = d->rc + d->skin;
  s->reps_h.assign(s->n_reps, RepDev{});
  s->T0.assign(s->n_reps, 0.0);
  int64_t atoms = 0, cells = 0, chains = 0;
  double max_expected = 0.0, max_tile = 0.0;
  // regions of G x G x 1 cells (narrower at the high faces when G does not divide M)
  const int G = s->lj_region;
  s->shapes_h.clear();
  for (int sy = 1; sy <= G; ++sy)
    for (int sx = 1; sx <= G; ++sx) s->shapes_h.push_back(make_shape(sx, sy));
  const double tile_cells = (double)s->shapes_h.back().n_tile;
  s->t_int.clear();
  for (int r = 0; r < s->n_reps; ++r) {
    const int nc = d->n_chains[r];
    const double L = d->box[r];
    if (nc < 1) return fail(s, MD_EINVAL, "every replica needs at least one chain");
    if (!(L > 0) || !std::isfinite(L)) return fail(s, MD_EINVAL, "box sides must be positive");
    const int M = (int)std::floor(L / rl);
    if (M < 3) return fail(s, MD_EINVAL, "box side must be at least 3 (rc + skin)");
    if (M > 1023) return fail(s, MD_EINVAL, "more than 1023 cells per side");
    RepDev& q = s->reps_h[r];
    q.L = L; q.M = M; q.h = L / M; q.inv_h = (double)M / L; q.half_L = 0.5 * L;
    q.Lf = (float)L; q.hf = (float)q.h; q.half_Lf = (float)(0.5 * L); q.Mf = (float)M;
    q.ih_hi = (float)q.inv_h; q.ih_lo = (float)(q.inv_h - (double)q.ih_hi);
    q.rc2u = (float)(d->rc * d->rc * q.inv_h * q.inv_h);
    q.rlist2u = (float)(rl * rl * q.inv_h * q.inv_h);
    q.hs2u = (float)(0.25 * d->skin * d->skin * q.inv_h * q.inv_h);
    q.cell_base = (int)cells; q.atom_off = (int)atoms;
    q.n_atoms = nc * s->S; q.n_chains = nc; q.chain_off = (int)chains;
    q.T0 = d->T_target ? d->T_target[r] : 0.0;
    q.dof = 3.0 * q.n_atoms - 3.0;
    s->T0[r] = q.T0;
    q.tile_off = (int)s->t_int.size();
    for (int o = 0; o < q.n_atoms; o += kIntTile) s->t_int.push_back(Tile{q.atom_off + o, std::min(kIntTile, q.n_atoms - o), r, 0});
    q.n_tiles = (int)s->t_int.size() - q.tile_off;
    // chains are locally as dense as a melt even in a sparse box, so the
    // density used for the capacity is at least that of a dense melt
    const double rho = std::max(q.n_atoms / (L * L * L), 40.0);
    max_expected = std::max(max_expected, 4.0 / 3.0 * M_PI * rl * rl * rl * rho);
    max_tile = std::max(max_tile, tile_cells * std::max(q.n_atoms / (L * L * L), 33.0) * q.h * q.h * q.h);
    atoms += q.n_atoms; cells += (int64_t)M * M * M; chains += nc;
    s->max_slices = std::max(s->max_slices, energy_slice_count(M * M * M));
    if (atoms >= (int64_t)kNbrIndexMask) return fail(s, MD_EINVAL, "too many atoms (limit 2^26)");
    if (chains >= (1 << 20)) return fail(s, MD_EINVAL, "too many chains (limit 2^20)");
    if (cells >= (1 << 26)) return fail(s, MD_EINVAL, "too many cells");
  }
  s->N = atoms; s->C = (int)cells;
  s->regions_h.clear();
  for (int r = 0; r < s->n_reps; ++r) {
    const int M = s->reps_h[r].M;
    for (int z = 0; z < M; ++z)
      for (int y = 0; y < M; y += G)
        for (int x = 0; x < M; x += G) {
          Region g{};
          g.rep = r; g.ox = x; g.oy = y; g.oz = z;
          g.shape = (std::min(G, M - x) - 1) + G * (std::min(G, M - y) - 1);
          s->regions_h.push_back(g);
        }
  }
  s->n_cl_max = (atoms + 3 * cells) / 4 + 1;   // sum of ceil(n_c / 4) over the cells
  s->Npad = (int)((atoms + 31) / 32 * 32);
  // default list capacity (entries per 4-atom cluster): a cluster's list holds
  // about 0.75 x the atoms within rc + skin of one atom at melt density
  // (~135 in the benchmark melt, at most ~350); 2.5 x that plus 64
  s->cap = d->nbr_capacity > 0 ? d->nbr_capacity : (int)std::ceil(2.5 * 0.75 * max_expected + 64.0);
  s->cap = (s->cap + 31) / 32 * 32;
  if (s->cap > 4096) return fail(s, MD_EINVAL, "neighbour capacity above 4096");
  // tile capacity (shared memory per block): 1.4x the mean tile of
  // the densest replica (at least melt density, 33 sites/nm^3) plus 64, in
  // multiples of 128 atoms; a larger tile is reported as MD_EOVERFLOW
  s->tile_cap = std::min(tile_capacity_max(), ((int)std::ceil(1.4 * max_tile + 64.0) + 127) / 128 * 128);
  fill_force_params(s);
  return MD_OK;
}

// Lay out every buffer; with base == nullptr only the size is computed.
static size_t plan(md_system* s, char* base) {
  size_t off = 0;
  auto take = [&](size_t b) -> char* { char* p = base ? base + off : nullptr; off += align256(b); return p; };
  const size_t N = (size_t)s->N, C = (size_t)s->C;
  const size_t fsz = s->mixed ? sizeof(double) : sizeof(float);
  s->reps = (RepDev*)take(sizeof(RepDev) * s->n_reps);
  s->tiles_int = (Tile*)take(sizeof(Tile) * s->t_int.size());
  s->x = take(3 * N * fsz);
  s->v = take(3 * N * fsz);
  s->img = (int*)take(3 * N * sizeof(int));
  s->F = take(N * (s->mixed ? sizeof(F4i) : sizeof(float4)));
  s->flj = (long long*)take(3 * (size_t)s->Npad * sizeof(long long));
  s->flj_e = (long long*)take(3 * (size_t)s->Npad * sizeof(long long));
  s->site = (uint16_t*)take(N * sizeof(uint16_t));
  s->cellc = (int*)take(N * sizeof(int));
  s->ref = (float4*)take(N * sizeof(float4));
  s->inv_perm = (int*)take(N * sizeof(int));
  s->pos = (float4*)take(N * sizeof(float4));
  s->tag = (int*)take(N * sizeof(int));
  s->perm = (int*)take(N * sizeof(int));
  s->regions = (Region*)take(sizeof(Region) * s->regions_h.size());
  s->shapes = (RegionShape*)take(sizeof(RegionShape) * s->shapes_h.size());
  s->list = (unsigned*)take((size_t)s->n_cl_max * s->cap * sizeof(unsigned));
  s->ncl = (int*)take((size_t)s->n_cl_max * sizeof(int));
  s->cl_start = (int*)take((C + 1) * sizeof(int));
  s->count = (int*)take(C * sizeof(int));
  s->cell_start = (int*)take((C + 1) * sizeof(int));
  s->cell_of = (int*)take(N * sizeof(int));
  s->slot = (int*)take(N * sizeof(int));
  s->tmp = (int*)take(N * sizeof(int));
  s->lj_part = (double*)take(C * 8 * sizeof(double));
  s->b_part = (double*)take(s->t_int.size() * 9 * sizeof(double));
  s->kepart = (double*)take(4 * s->t_int.size() * sizeof(double));   // kinetic energy, then momentum (x, y, z) per tile
  s->ke_out = (double*)take(s->n_reps * sizeof(double));
  s->lam = (double*)take(6 * s->n_reps * sizeof(double));   // rescale factor, or the Nose-Hoover state (6 per replica)
  s->e_out = (double*)take((size_t)s->n_reps * 16 * sizeof(double));
  s->e_slices = (double*)take((size_t)s->n_reps * s->max_slices * 11 * sizeof(double));
  s->done = (unsigned*)take(sizeof(unsigned));
  s->work = (int*)take(2 * sizeof(int));
  s->flags = (unsigned*)take(sizeof(unsigned));
  s->early = (unsigned long long*)take(sizeof(unsigned long long));
  s->stage = (double*)take(6 * N * sizeof(double) + 3 * N * sizeof(int));   // staging: x, v (FP64), images
  if (s->generic) {
    s->mtype = (unsigned char*)take(s->mtype_h.size());
    auto ti = [&](const std::vector<int>& v) { return (const int*)take(v.size() * sizeof(int)); };
    s->topo.b_off = ti(s->t_boff); s->topo.b_at = ti(s->t_bat);
    s->topo.a_off = ti(s->t_aoff); s->topo.a_at = ti(s->t_aat);
    s->topo.d_off = ti(s->t_doff); s->topo.d_at = ti(s->t_dat);
    s->topo.x_off = ti(s->t_xoff); s->topo.x_at = ti(s->t_xat);
    s->topo.naom = s->S;
  }
  return off;
}

// ------------------------------------------------------------------ enqueue helpers
static void prof_mark(md_system* s) {
  if (!s->profile || s->ev_used >= (int)s->ev.size()) return;
  // inside a stream capture an external record becomes an event-record node;
  // outside one (a remainder block launched directly) a plain record
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s->st, &cs);
  if (cs == cudaStreamCaptureStatusActive)
    cudaEventRecordWithFlags(s->ev[s->ev_used++], s->st, cudaEventRecordExternal);
  else
    cudaEventRecord(s->ev[s->ev_used++], s->st);
}

static void enqueue_rebin(md_system* s) {
  cudaMemsetAsync(s->count, 0, sizeof(int) * s->C, s->st);
  launch_bin_count(s->mixed, s->x, (int)s->N, s->tiles_int, (int)s->t_int.size(), s->reps, s->cell_of, s->cellc,
                   s->count, s->slot, s->st);
  launch_scan2(s->count, s->cell_start, s->cl_start, s->C, s->st);
  launch_bin_scatter(s->cell_of, s->slot, s->cell_start, s->tmp, (int)s->N, s->st);
  launch_cell_sort(s->mixed, s->x, (int)s->N, s->cell_start, s->tmp, s->fp.mtype, s->cellc, s->site, s->reps, s->n_reps, s->C,
                   s->S, s->perm, s->inv_perm, s->pos, s->tag, s->ref, s->flags, s->st);
  prof_mark(s);
  launch_cl_build(s->pos, s->tag, s->cell_start, s->cl_start, s->regions, (int)s->regions_h.size(), s->shapes,
                  s->reps, s->list, s->ncl, s->cap, s->tile_cap, s->flags, 0, s->work,
                  s->generic ? &s->topo : nullptr, s->st);
  prof_mark(s);
}
static const int kRebinLaunches = 6;   // memset counted as a launch

// F_out: where the total force goes (the dynamics' s->F, or scratch for an
// energy read-out, whose kernels need not reproduce the force bits of the
// force-only kernels: the compiler may fuse their arithmetic differently)
static void enqueue_forces(md_system* s, bool energy, void* F_out = nullptr) {
  // an energy read-out accumulates its LJ forces apart from the dynamics'
  long long* flj = F_out ? s->flj_e : s->flj;
  cudaMemsetAsync(flj, 0, 3 * (size_t)s->Npad * sizeof(long long), s->st);
  prof_mark(s);   // closes the integrate group (integrator, displacement check, clear)
  launch_cl_force(energy, s->pos, s->cell_start, s->cl_start, s->regions, (int)s->regions_h.size(), s->shapes,
                  s->reps, s->list, s->ncl, s->cap, s->tile_cap, s->fp, flj, s->Npad, s->lj_part, s->flags,
                  s->lj_block, s->lj_lanes, s->persistent_grid, s->work, s->lj_pair_exact, s->st);
  prof_mark(s);
  if (s->generic)
    launch_bonded_generic(energy, (const double*)s->x, s->inv_perm, flj, s->Npad, (int)s->N, s->tiles_int,
                          (int)s->t_int.size(), s->reps, s->fp, s->topo, F_out ? F_out : s->F, s->b_part, s->flags,
                          s->st);
  else
    launch_bonded(s->mixed, energy, s->x, s->site, s->inv_perm, flj, s->Npad, (int)s->N, s->tiles_int,
                  (int)s->t_int.size(), s->reps, s->fp, F_out ? F_out : s->F, s->b_part, s->flags, s->st);
  prof_mark(s);
}

// Inside a step-graph capture, after a drift: a one-thread check of the
// displacement flag sets the condition of an IF node whose body re-bins and
// rebuilds the list, so a step whose atoms moved more than skin/2 since the
// last rebin computes its forces from fresh bins (and is counted), instead of
// the run stopping.  No-op outside a capture.
static void enqueue_cond_rebin(md_system* s) {
  if (s->disp != MD_DISP_REBUILD) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* ed = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s->st, &cs, nullptr, &g, &deps, &ed, &nd) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive)
    return;
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) return;
  launch_disp_check(h, s->flags, s->early, s->st);
  if (cudaStreamGetCaptureInfo(s->st, &cs, nullptr, &g, &deps, &ed, &nd) != cudaSuccess) return;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, ed, nd, &p) != cudaSuccess) return;
  cudaGraph_t body = p.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(s->st, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return;
  // the body: the rebin sequence, captured on the side stream
  if (cudaStreamBeginCaptureToGraph(s->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return;
  cudaStream_t main = s->st;
  const bool prof = s->profile;
  s->st = s->side;
  s->profile = false;
  enqueue_rebin(s);
  s->st = main;
  s->profile = prof;
  cudaGraph_t out = nullptr;
  cudaStreamEndCapture(s->side, &out);
}

static void enqueue_integrate(md_system* s, IntegMode mode, bool ke, bool mark) {
  launch_integrate(s->mixed, mode, ke, s->thermo, s->x, s->v, s->img, s->F, s->site, s->cellc,
                   s->inv_perm, s->ref, s->pos, (int)s->N, s->tiles_int, (int)s->t_int.size(), s->reps, s->n_reps,
                   s->fp, s->kepart, s->done, s->ke_out, s->lam, s->tau, s->flags, s->st);
  if (mark) prof_mark(s);
}

// one block of k steps: rebin + list (unless the bins and list are already
// those of the current positions), k velocity-Verlet steps
static void enqueue_block(md_system* s, int k, bool rebin = true) {
  s->ev_used = 0;
  prof_mark(s);
  if (rebin) enqueue_rebin(s);
  enqueue_integrate(s, kKickDrift, false, false);
  enqueue_cond_rebin(s);
  enqueue_forces(s, false);
  for (int j = 1; j < k; ++j) {
    enqueue_integrate(s, kKickKickDrift, false, false);
    enqueue_cond_rebin(s);
    enqueue_forces(s, false);
  }
  enqueue_integrate(s, kKickOnly, false, true);
}
// per step: integrate, displacement check, memset, LJ, bonded (a memset
// counted as a launch; an early rebin adds kRebinLaunches)
static int64_t block_launches(int k, bool check) { return kRebinLaunches + (check ? 5LL : 4LL) * k + 1; }

// accumulate the event timings of the last block (requires a finished stream)
static void prof_collect(md_system* s, int k) {
  if (!s->profile || s->ev_used < 3 + 3 * k + 1) return;
  float ms;
  cudaEventElapsedTime(&ms, s->ev[0], s->ev[1]); s->prof_ms[0] += ms; s->prof_n[0] += 5;
  cudaEventElapsedTime(&ms, s->ev[1], s->ev[2]); s->prof_ms[1] += ms; s->prof_n[1] += 1;
  int e = 2;
  for (int j = 0; j < k; ++j) {
    cudaEventElapsedTime(&ms, s->ev[e], s->ev[e + 1]); s->prof_ms[2] += ms; s->prof_n[2] += 1;
    cudaEventElapsedTime(&ms, s->ev[e + 1], s->ev[e + 2]); s->prof_ms[3] += ms; s->prof_n[3] += 1;
    cudaEventElapsedTime(&ms, s->ev[e + 2], s->ev[e + 3]); s->prof_ms[4] += ms; s->prof_n[4] += 1;
    e += 3;
  }
  cudaEventElapsedTime(&ms, s->ev[e], s->ev[e + 1]); s->prof_ms[2] += ms; s->prof_n[2] += 1;
}

// the rebin cycle as a graph, and the same without its leading rebin + list
// (used for the first cycle after md_set_state / md_rebin, which just did
// them; never while profiling, so that the event layout stays fixed)
static void drop_rem_graphs(md_system* s) {
  for (cudaGraphExec_t& e : s->rem_graphs)
    if (e) { cudaGraphExecDestroy(e); e = nullptr; }
}

// a block of k steps (leading rebin included) as a graph
static int capture_block(md_system* s, int k, cudaGraphExec_t* out) {
  cudaGraph_t g;
  CU(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
  enqueue_block(s, k, true);
  cudaError_t e = cudaStreamEndCapture(s->st, &g);
  if (e != cudaSuccess) return fail(s, MD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(s, MD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return MD_OK;
}

static int capture_cycle(md_system* s) {
  if (s->cycle) { cudaGraphExecDestroy(s->cycle); s->cycle = nullptr; }
  if (s->cycle_fresh) { cudaGraphExecDestroy(s->cycle_fresh); s->cycle_fresh = nullptr; }
  drop_rem_graphs(s);
  s->rem_graphs.assign(s->R, nullptr);
  for (int pass = 0; pass < 2; ++pass) {
    const bool prof = s->profile;
    if (pass == 1) s->profile = false;
    cudaGraph_t g;
    CU(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    enqueue_block(s, s->R, pass == 0);
    cudaError_t e = cudaStreamEndCapture(s->st, &g);
    s->profile = prof;
    if (e != cudaSuccess) return fail(s, MD_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(pass == 0 ? &s->cycle : &s->cycle_fresh, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(s, MD_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  return MD_OK;
}

static int check_flags(md_system* s) {
  unsigned f = 0;
  CU(cudaStreamSynchronize(s->st));
  CU(cudaMemcpy(&f, s->flags, sizeof f, cudaMemcpyDeviceToHost));
  if (!f) return MD_OK;
  CU(cudaMemset(s->flags, 0, sizeof(unsigned)));
  // a non-finite value is the first thing to report: it usually comes with
  // huge finite forces nearby
  if (f & kFlagNaN) return fail(s, MD_EUNSTABLE, "non-finite position, velocity or force");
  if (f & kFlagNbrOverflow) return fail(s, MD_EOVERFLOW, "neighbour list capacity exceeded (raise nbr_capacity)");
  if (f & kFlagFixOverflow) return fail(s, MD_EOVERFLOW, "force beyond the fixed-point range (a part >= 2^17 kJ/mol/nm)");
  if (f & kFlagDisplacement) return fail(s, MD_EUNSTABLE, "an atom moved more than skin/2 between rebins (raise skin or lower rebin_every)");
  if (f & kFlagBadInput) return fail(s, MD_EINVAL, "non-finite input position or velocity");
  if (f & kFlagTimeout) return fail(s, MD_ETIMEOUT, "a bounded device wait gave up");
  return fail(s, MD_ECUDA, "unknown device flag");
}

// upload positions (wrapped) and velocities, reset images
// Caller's arrays (host or device, x,y,z per atom) -> one DMA each into the
// staging buffer -> k_ingest checks, wraps and transposes them on the GPU.  A
// non-finite value raises kFlagBadInput, reported by the next check_flags
// (refresh() runs one before md_create / md_set_state return).
static int upload_state(md_system* s, const double* pos, const double* vel) {
  const size_t N = (size_t)s->N;
  CU(cudaMemcpyAsync(s->stage, pos, 3 * N * sizeof(double), cudaMemcpyDefault, s->st));
  CU(cudaMemcpyAsync(s->stage + 3 * N, vel, 3 * N * sizeof(double), cudaMemcpyDefault, s->st));
  launch_ingest(s->mixed, s->stage, (int)N, s->tiles_int, (int)s->t_int.size(), s->reps, s->x, s->v, s->img,
                s->flags, s->st);
  CU(cudaGetLastError());
  return MD_OK;
}

static int refresh(md_system* s) {
  const bool p = s->profile;
  s->profile = false;
  enqueue_rebin(s);
  enqueue_forces(s, false);
  s->profile = p;
  const int rc = check_flags(s);
  s->fresh = rc == MD_OK;
  return rc;
}

// The paper's CBIN binning (Sec. 3.1) done here as a comparison arm: the
// cell of every atom, histogram, exclusive scans and the stable order by atom
// index, on the host from a copy of the positions, with the device's
// formulas (host code is compiled without contraction, so the FP64 cell
// coordinates agree bit for bit).
template <class T>
static void host_bins(const T* x, const md_system* s, std::vector<int>& cell_of, std::vector<int>& cellc,
                      std::vector<int>& cell_start, std::vector<int>& cl_start, std::vector<int>& perm) {
  const int64_t N = s->N;
  std::vector<int> count(s->C, 0);
  for (const RepDev& q : s->reps_h) {
    for (int i = q.atom_off; i < q.atom_off + q.n_atoms; ++i) {
      int k[3];
      for (int a = 0; a < 3; ++a) {
        const double xv = (double)x[a * N + i];
        double sv = xv;
        if (!(xv >= 0.0 && xv < q.L)) sv = xv - q.L * std::floor(xv / q.L);
        int c = (int)std::floor(sv * q.inv_h);
        k[a] = c < 0 ? 0 : (c > q.M - 1 ? q.M - 1 : c);
      }
      const int c = q.cell_base + (k[2] * q.M + k[1]) * q.M + k[0];
      cell_of[i] = c;
      cellc[i] = k[0] | (k[1] << 10) | (k[2] << 20);
      ++count[c];
    }
  }
  cell_start[0] = 0;
  cl_start[0] = 0;
  for (int c = 0; c < s->C; ++c) {
    cell_start[c + 1] = cell_start[c] + count[c];
    cl_start[c + 1] = cl_start[c] + (count[c] + 3) / 4;
  }
  std::vector<int> fill(cell_start.begin(), cell_start.end() - 1);
  for (int64_t i = 0; i < N; ++i) perm[fill[cell_of[i]]++] = (int)i;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int md_workspace_size(const md_desc* desc, size_t* bytes) {
  md_system tmp;
  md_system* s = &tmp;
  int rc = configure(s, desc);
  if (rc) { g_create_error = s->err; return rc; }
  if (!bytes) return fail(nullptr, MD_EINVAL, "null output");
  *bytes = plan(s, nullptr);
  return MD_OK;
}

int md_create(const md_desc* d, md_system** out) {
  if (!out) return fail(nullptr, MD_EINVAL, "null output pointer");
  *out = nullptr;
  md_system* s = new md_system();
  int rc = configure(s, d);
  if (rc) { g_create_error = s->err; delete s; return rc; }
  if (!d->pos || !d->vel) { delete s; return fail(nullptr, MD_EINVAL, "pos and vel are required"); }
  auto bail = [&](int code) { g_create_error = s->err; md_destroy(s); return code; };
  s->bytes = plan(s, nullptr);
  if (d->workspace) {
    if (d->workspace_bytes < s->bytes) {
      fail(s, MD_ENOMEM, "workspace too small: need " + std::to_string(s->bytes) + " bytes");
      return bail(MD_ENOMEM);
    }
    if (((uintptr_t)d->workspace & 255) != 0) { fail(s, MD_EINVAL, "workspace must be 256-byte aligned"); return bail(MD_EINVAL); }
    s->base = (char*)d->workspace;
  } else {
    if (cudaMalloc(&s->base, s->bytes) != cudaSuccess) {
      cudaGetLastError();
      s->base = nullptr;
      fail(s, MD_ENOMEM, "cudaMalloc of " + std::to_string(s->bytes) + " bytes failed");
      return bail(MD_ENOMEM);
    }
    s->own_mem = true;
  }
  plan(s, s->base);
  s->fp.mtype = s->generic ? s->mtype : nullptr;
  if (d->cuda_stream) {
    s->st = (cudaStream_t)d->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
      fail(s, MD_ECUDA, "stream creation failed");
      return bail(MD_ECUDA);
    }
    s->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess) {
    fail(s, MD_ECUDA, "stream creation failed");
    return bail(MD_ECUDA);
  }
  if (tile_kernels_init() != cudaSuccess) {
    cudaGetLastError();
    fail(s, MD_ECUDA, "cannot reserve shared memory for the neighbour-tile kernels");
    return bail(MD_ECUDA);
  }
  if (d->schedule == MD_SCHED_PERSISTENT) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = lj_blocks_per_sm(s->lj_block, s->lj_lanes, s->tile_cap);
    s->persistent_grid = std::max(1, std::min((int)s->regions_h.size(), sms * std::max(per_sm, 1)));
  }
  // static tables
  std::vector<uint16_t> site(s->N);
  for (int64_t i = 0; i < s->N; ++i) site[i] = 0;
  for (int r = 0; r < s->n_reps; ++r) {
    const RepDev& q = s->reps_h[r];
    for (int i = 0; i < q.n_atoms; ++i) site[q.atom_off + i] = (uint16_t)(i % s->S);
  }
  // thermostat state: the weak-coupling factor lam[r] = 1, or per replica the
  // Nose-Hoover (xi, 1 - c, 1/(1 + c), V_com) = (0, 1, 1, 0, 0, 0)
  std::vector<double> ones(6 * s->n_reps, 1.0);
  if (s->thermo == MD_NOSE_HOOVER)
    for (int r = 0; r < s->n_reps; ++r)
      for (int k = 0; k < 6; ++k) ones[6 * r + k] = (k == 1 || k == 2) ? 1.0 : 0.0;
  auto up = [&](void* dst, const void* src, size_t b) {
    return cudaMemcpyAsync(dst, src, b, cudaMemcpyHostToDevice, s->st) == cudaSuccess;
  };
  bool ok = up(s->reps, s->reps_h.data(), sizeof(RepDev) * s->n_reps) &&
            up(s->tiles_int, s->t_int.data(), sizeof(Tile) * s->t_int.size()) &&
            up(s->site, site.data(), sizeof(uint16_t) * s->N) &&
            up(s->lam, ones.data(), sizeof(double) * 6 * s->n_reps) &&
            up(s->regions, s->regions_h.data(), sizeof(Region) * s->regions_h.size()) &&
            (!s->generic || (up(s->mtype, s->mtype_h.data(), s->mtype_h.size()) &&
                             up((void*)s->topo.b_off, s->t_boff.data(), s->t_boff.size() * sizeof(int)) &&
                             up((void*)s->topo.b_at, s->t_bat.data(), s->t_bat.size() * sizeof(int)) &&
                             up((void*)s->topo.a_off, s->t_aoff.data(), s->t_aoff.size() * sizeof(int)) &&
                             up((void*)s->topo.a_at, s->t_aat.data(), s->t_aat.size() * sizeof(int)) &&
                             up((void*)s->topo.d_off, s->t_doff.data(), s->t_doff.size() * sizeof(int)) &&
                             up((void*)s->topo.d_at, s->t_dat.data(), s->t_dat.size() * sizeof(int)) &&
                             up((void*)s->topo.x_off, s->t_xoff.data(), s->t_xoff.size() * sizeof(int)) &&
                             up((void*)s->topo.x_at, s->t_xat.data(), s->t_xat.size() * sizeof(int)))) &&
            up(s->shapes, s->shapes_h.data(), sizeof(RegionShape) * s->shapes_h.size()) &&
            cudaMemsetAsync(s->flj, 0, 3 * (size_t)s->Npad * sizeof(long long), s->st) == cudaSuccess &&
            cudaMemsetAsync(s->flj_e, 0, 3 * (size_t)s->Npad * sizeof(long long), s->st) == cudaSuccess &&
            cudaMemsetAsync(s->done, 0, sizeof(unsigned), s->st) == cudaSuccess &&
            cudaMemsetAsync(s->work, 0, 2 * sizeof(int), s->st) == cudaSuccess &&
            cudaMemsetAsync(s->flags, 0, sizeof(unsigned), s->st) == cudaSuccess &&
            cudaMemsetAsync(s->early, 0, sizeof(unsigned long long), s->st) == cudaSuccess &&
            cudaStreamSynchronize(s->st) == cudaSuccess;
  if (!ok) { fail(s, MD_ECUDA, "initial upload failed"); return bail(MD_ECUDA); }
  rc = upload_state(s, d->pos, d->vel);
  if (rc) return bail(rc);
  rc = refresh(s);
  if (rc) return bail(rc);
  rc = capture_cycle(s);
  if (rc) return bail(rc);
  *out = s;
  return MD_OK;
}

int md_step_async(md_system* s, int64_t n) {
  if (!s || n < 0) return fail(s, MD_EINVAL, "bad arguments");
  const int64_t full = n / s->R, rem = n % s->R;
  for (int64_t c = 0; c < full; ++c) {
    const bool skip_rebin = c == 0 && s->fresh && !s->profile;
    s->fresh = false;
    CU(cudaGraphLaunch(skip_rebin ? s->cycle_fresh : s->cycle, s->st));
    if (s->profile) {
      s->ev_used = (int)std::min<int64_t>(s->ev.size(), 3 + 3 * s->R + 1);
      CU(cudaStreamSynchronize(s->st));
      prof_collect(s, s->R);
    }
  }
  if (rem) {
    s->fresh = false;
    cudaGraphExec_t& gr = s->rem_graphs[rem];
    if (!gr) {
      const int rc = capture_block(s, (int)rem, &gr);
      if (rc) return rc;
    }
    if (s->profile) s->ev_used = (int)std::min<int64_t>(s->ev.size(), 3 + 3 * rem + 1);
    CU(cudaGraphLaunch(gr, s->st));
    if (s->profile) { CU(cudaStreamSynchronize(s->st)); prof_collect(s, (int)rem); }
  }
  return MD_OK;
}

int md_step(md_system* s, int64_t n) {
  int rc = md_step_async(s, n);
  if (rc) return rc;
  return check_flags(s);
}

int md_sync(md_system* s) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  return check_flags(s);
}

int md_forces(md_system* s, double* f_out) {
  if (!s || !f_out) return fail(s, MD_EINVAL, "bad arguments");
  const size_t N = (size_t)s->N;
  launch_egress_forces(s->mixed, s->F, (int)N, kFixInv, s->stage, s->st);
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(f_out, s->stage, 3 * N * sizeof(double), cudaMemcpyDefault, s->st));
  CU(cudaStreamSynchronize(s->st));
  return MD_OK;
}

int md_energy(md_system* s, md_energy_t* out) {
  if (!s || !out) return fail(s, MD_EINVAL, "bad arguments");
  const bool p = s->profile;
  s->profile = false;
  // energies and virial of the current state; the forces of this pass go to
  // the staging buffer (6N doubles + 3N ints, room for either force layout),
  // so reading energies never changes the forces the dynamics use
  enqueue_forces(s, true, s->stage);
  launch_energy_reduce(s->lj_part, s->b_part, s->reps, s->n_reps, s->max_slices, s->e_slices, s->e_out, s->st);
  // kinetic energy of the current velocities (a pass that only reads v)
  launch_integrate(s->mixed, kKineticOnly, true, false, s->x, s->v, s->img, s->F, s->site, s->cellc, s->inv_perm,
                   s->ref, s->pos, (int)s->N, s->tiles_int, (int)s->t_int.size(), s->reps, s->n_reps, s->fp,
                   s->kepart, s->done, s->ke_out, s->lam, s->tau, s->flags, s->st);
  s->profile = p;
  CU(cudaGetLastError());
  std::vector<double> e((size_t)s->n_reps * 16), ke(s->n_reps);
  CU(cudaMemcpyAsync(e.data(), s->e_out, e.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  CU(cudaMemcpyAsync(ke.data(), s->ke_out, ke.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  int rc = check_flags(s);
  if (rc) return rc;
  for (int r = 0; r < s->n_reps; ++r) {
    md_energy_t& o = out[r];
    const double* q = e.data() + 16 * r;
    o.lj = q[0]; o.lj_shifted = q[1]; o.bond = q[2]; o.angle = q[3]; o.dihedral = q[4];
    for (int k = 0; k < 6; ++k) o.virial[k] = q[5 + k];
    o.kinetic = ke[r];
    o.temperature = 2.0 * ke[r] / (s->reps_h[r].dof * kKB);
    o.total = o.lj_shifted + o.bond + o.angle + o.dihedral + o.kinetic;
    const double V = s->reps_h[r].L * s->reps_h[r].L * s->reps_h[r].L;
    o.pressure = (2.0 * o.kinetic + o.virial[0] + o.virial[1] + o.virial[2]) / (3.0 * V);
  }
  return MD_OK;
}

int md_rebin(md_system* s) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  const bool p = s->profile;
  s->profile = false;
  enqueue_rebin(s);
  s->profile = p;
  const int rc = check_flags(s);
  s->fresh = rc == MD_OK;   // the forces already belong to these positions
  return rc;
}

int md_get_state(md_system* s, double* pos, double* vel, int32_t* images) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  const size_t N = (size_t)s->N;
  double* sp = s->stage;
  double* sv = s->stage + 3 * N;
  int* si = reinterpret_cast<int*>(s->stage + 6 * N);
  launch_egress_state(s->mixed, s->x, s->v, s->img, (int)N, sp, sv, si, s->st);
  CU(cudaGetLastError());
  if (pos) CU(cudaMemcpyAsync(pos, sp, 3 * N * sizeof(double), cudaMemcpyDefault, s->st));
  if (vel) CU(cudaMemcpyAsync(vel, sv, 3 * N * sizeof(double), cudaMemcpyDefault, s->st));
  if (images) CU(cudaMemcpyAsync(images, si, 3 * N * sizeof(int), cudaMemcpyDefault, s->st));
  CU(cudaStreamSynchronize(s->st));
  return MD_OK;
}

int md_set_state(md_system* s, const double* pos, const double* vel) {
  if (!s || !pos || !vel) return fail(s, MD_EINVAL, "bad arguments");
  CU(cudaStreamSynchronize(s->st));
  int rc = upload_state(s, pos, vel);
  if (rc) return rc;
  return refresh(s);
}

int md_set_params(md_system* s, const md_params* p) {
  if (!s || !p) return fail(s, MD_EINVAL, "bad arguments");
  for (int a = 0; a < 2; ++a)
    if (!(p->mass[a] > 0) || !(p->sigma[a] > 0) || !(p->eps[a] >= 0))
      return fail(s, MD_EINVAL, "masses and sigmas must be > 0, eps >= 0");
  CU(cudaStreamSynchronize(s->st));
  s->params = *p;
  fill_force_params(s);
  CU(cudaMemcpy(s->reps, s->reps_h.data(), sizeof(RepDev) * s->n_reps, cudaMemcpyHostToDevice));
  int rc = capture_cycle(s);
  if (rc) return rc;
  const bool pf = s->profile;
  s->profile = false;
  enqueue_forces(s, false);
  s->profile = pf;
  return check_flags(s);
}

int md_set_temperature(md_system* s, const double* T) {
  if (!s || !T) return fail(s, MD_EINVAL, "bad arguments");
  CU(cudaStreamSynchronize(s->st));
  for (int r = 0; r < s->n_reps; ++r) { s->reps_h[r].T0 = T[r]; s->T0[r] = T[r]; }
  CU(cudaMemcpy(s->reps, s->reps_h.data(), sizeof(RepDev) * s->n_reps, cudaMemcpyHostToDevice));
  return MD_OK;
}

int md_observables(md_system* s, double* r_ee, double* rg2, double* trans_fraction) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  if (s->generic) return fail(s, MD_EINVAL, "chain observables need linear chains");
  int chains = 0;
  for (int r = 0; r < s->n_reps; ++r) chains += s->reps_h[r].n_chains;
  // scratch in the staging buffer (6N doubles + 3N ints >= 4 doubles per chain + counts)
  double* ree_d = s->stage;
  double* rg_d = s->stage + 3 * (size_t)chains;
  unsigned long long* tr_d = reinterpret_cast<unsigned long long*>(s->stage + 4 * (size_t)chains);
  CU(cudaMemsetAsync(tr_d, 0, sizeof(unsigned long long) * s->n_reps, s->st));
  launch_chain_observables(s->mixed, s->x, (int)s->N, s->reps, s->n_reps, s->fp, chains, ree_d, rg_d, tr_d, s->st);
  CU(cudaGetLastError());
  std::vector<unsigned long long> tr(s->n_reps);
  if (r_ee) CU(cudaMemcpyAsync(r_ee, ree_d, 3 * (size_t)chains * sizeof(double), cudaMemcpyDefault, s->st));
  if (rg2) CU(cudaMemcpyAsync(rg2, rg_d, (size_t)chains * sizeof(double), cudaMemcpyDefault, s->st));
  CU(cudaMemcpyAsync(tr.data(), tr_d, sizeof(unsigned long long) * s->n_reps, cudaMemcpyDeviceToHost, s->st));
  CU(cudaStreamSynchronize(s->st));
  if (trans_fraction)
    for (int r = 0; r < s->n_reps; ++r) {
      const double nd = (double)s->reps_h[r].n_chains * (double)(s->S > 3 ? s->S - 3 : 0);
      trans_fraction[r] = nd > 0 ? (double)tr[r] / nd : 0.0;
    }
  return MD_OK;
}

int md_rdf(md_system* s, int32_t n_bins, const double* edges, int64_t* counts) {
  if (!s || !edges || !counts || n_bins < 1 || n_bins > 16384) return fail(s, MD_EINVAL, "bad arguments (1 <= n_bins <= 16384)");
  if (s->generic) return fail(s, MD_EINVAL, "the RDF's exclusions are those of linear chains");
  if (!(edges[0] >= 0.0)) return fail(s, MD_EINVAL, "edges[0] must be >= 0");
  for (int k = 0; k < n_bins; ++k)
    if (!(edges[k + 1] > edges[k])) return fail(s, MD_EINVAL, "edges must increase");
  for (const RepDev& q : s->reps_h)
    if (edges[n_bins] > q.h) return fail(s, MD_EINVAL, "r_max beyond the cell side of a replica");
  double* ed = nullptr;
  unsigned long long* cnt = nullptr;
  const size_t nc = (size_t)s->n_reps * n_bins;
  if (cudaMalloc(&ed, sizeof(double) * (n_bins + 1)) != cudaSuccess ||
      cudaMalloc(&cnt, sizeof(unsigned long long) * nc) != cudaSuccess) {
    cudaGetLastError();
    if (ed) cudaFree(ed);
    return fail(s, MD_ENOMEM, "device memory for the histogram");
  }
  int rc = MD_OK;
  // bins of the current positions (the last rebin's may be up to skin/2 old)
  const bool p = s->profile;
  s->profile = false;
  enqueue_rebin(s);
  s->profile = p;
  if (cudaMemcpyAsync(ed, edges, sizeof(double) * (n_bins + 1), cudaMemcpyHostToDevice, s->st) != cudaSuccess ||
      cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * nc, s->st) != cudaSuccess) {
    rc = fail(s, MD_ECUDA, "histogram set-up failed");
  } else {
    const double norm = (double)n_bins / (edges[n_bins] - edges[0]);
    launch_rdf(s->mixed, s->x, (int)s->N, s->cell_start, s->perm, s->reps, s->n_reps, s->C, s->S, ed, n_bins, norm,
               cnt, s->st);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(counts, cnt, sizeof(unsigned long long) * nc, cudaMemcpyDefault, s->st) != cudaSuccess)
      rc = fail(s, MD_ECUDA, "histogram kernel failed");
  }
  if (rc == MD_OK) {
    rc = check_flags(s);
    s->fresh = rc == MD_OK;
  } else {
    cudaStreamSynchronize(s->st);
  }
  cudaFree(ed);
  cudaFree(cnt);
  return rc;
}

int md_acf_reset(md_system* s, int32_t max_lag) {
  if (!s || max_lag < 0 || max_lag > 100000) return fail(s, MD_EINVAL, "max_lag must be 0 .. 100000");
  CU(cudaStreamSynchronize(s->st));
  int chains = 0;
  for (const RepDev& q : s->reps_h) chains += q.n_chains;
  if (max_lag != s->acf_lag) {
    if (s->acf_ring) cudaFree(s->acf_ring);
    if (s->acf_acc) cudaFree(s->acf_acc);
    s->acf_ring = s->acf_acc = nullptr;
    s->acf_lag = -1;
    if (cudaMalloc(&s->acf_ring, sizeof(double) * 3 * (size_t)chains * (max_lag + 1)) != cudaSuccess ||
        cudaMalloc(&s->acf_acc, sizeof(double) * (size_t)s->n_reps * (max_lag + 1)) != cudaSuccess) {
      cudaGetLastError();
      return fail(s, MD_ENOMEM, "device memory for the ACF ring");
    }
    s->acf_lag = max_lag;
  }
  CU(cudaMemset(s->acf_acc, 0, sizeof(double) * (size_t)s->n_reps * (max_lag + 1)));
  s->acf_n = 0;
  return MD_OK;
}

static int acf_add(md_system* s, int chains) {
  launch_acf_add(s->acf_ring, chains, s->reps, s->n_reps, s->acf_n, s->acf_lag, s->acf_acc, s->st);
  CU(cudaGetLastError());
  ++s->acf_n;
  return MD_OK;
}

int md_acf_push(md_system* s, const double* r_ee) {
  if (!s || !r_ee) return fail(s, MD_EINVAL, "bad arguments");
  if (s->acf_lag < 0) return fail(s, MD_EINVAL, "md_acf_reset first");
  int chains = 0;
  for (const RepDev& q : s->reps_h) chains += q.n_chains;
  double* slot = s->acf_ring + (size_t)(s->acf_n % (s->acf_lag + 1)) * 3 * chains;
  CU(cudaMemcpyAsync(slot, r_ee, sizeof(double) * 3 * chains, cudaMemcpyDefault, s->st));
  int rc = acf_add(s, chains);
  if (rc) return rc;
  CU(cudaStreamSynchronize(s->st));
  return MD_OK;
}

int md_acf_sample(md_system* s) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  if (s->generic) return fail(s, MD_EINVAL, "end-to-end vectors need linear chains");
  if (s->acf_lag < 0) return fail(s, MD_EINVAL, "md_acf_reset first");
  int chains = 0;
  for (const RepDev& q : s->reps_h) chains += q.n_chains;
  double* slot = s->acf_ring + (size_t)(s->acf_n % (s->acf_lag + 1)) * 3 * chains;
  // end-to-end vectors straight into the ring; R_g^2 and trans counts to scratch
  double* rg_d = s->stage;
  unsigned long long* tr_d = reinterpret_cast<unsigned long long*>(s->stage + chains);
  CU(cudaMemsetAsync(tr_d, 0, sizeof(unsigned long long) * s->n_reps, s->st));
  launch_chain_observables(s->mixed, s->x, (int)s->N, s->reps, s->n_reps, s->fp, chains, slot, rg_d, tr_d, s->st);
  CU(cudaGetLastError());
  return acf_add(s, chains);
}

int md_acf_read(md_system* s, double* C, int64_t* n_samples) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  if (s->acf_lag < 0) return fail(s, MD_EINVAL, "md_acf_reset first");
  const int slots = s->acf_lag + 1;
  std::vector<double> acc((size_t)s->n_reps * slots);
  CU(cudaMemcpyAsync(acc.data(), s->acf_acc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  CU(cudaStreamSynchronize(s->st));
  const int64_t n = s->acf_n;
  if (n_samples) *n_samples = n;
  if (C)
    for (int r = 0; r < s->n_reps; ++r) {
      const double nc = (double)s->reps_h[r].n_chains;
      const double norm = n > 0 ? acc[(size_t)r * slots] / ((double)n * nc) : 0.0;
      for (int t = 0; t < slots; ++t)
        C[(size_t)r * slots + t] = t < n ? (acc[(size_t)r * slots + t] / ((double)(n - t) * nc)) / norm : NAN;
    }
  return MD_OK;
}

int md_bin_study(md_system* s, int32_t reps, double* ms) {
  if (!s || !ms || reps < 1 || reps > 1000) return fail(s, MD_EINVAL, "bad arguments (1 <= reps <= 1000)");
  CU(cudaStreamSynchronize(s->st));
  const size_t N = (size_t)s->N, C = (size_t)s->C;
  const size_t xb = 3 * N * (s->mixed ? sizeof(double) : sizeof(float));
  void* hx = nullptr;
  CU(cudaMallocHost(&hx, xb));
  std::vector<int> cell_of(N), cellc(N), cell_start(C + 1), cl_start(C + 1), perm(N);
  cudaEvent_t ev[6];
  for (cudaEvent_t& e : ev) cudaEventCreate(&e);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const bool prof = s->profile;
  s->profile = false;
  int rc = MD_OK;
  for (int k = 0; k < reps && rc == MD_OK; ++k) {
    // GPU arm: on-GPU counting sort and sorted arrays, then the list build
    cudaEventRecord(ev[0], s->st);
    cudaMemsetAsync(s->count, 0, sizeof(int) * C, s->st);
    launch_bin_count(s->mixed, s->x, (int)N, s->tiles_int, (int)s->t_int.size(), s->reps, s->cell_of, s->cellc,
                     s->count, s->slot, s->st);
    launch_scan2(s->count, s->cell_start, s->cl_start, s->C, s->st);
    launch_bin_scatter(s->cell_of, s->slot, s->cell_start, s->tmp, (int)N, s->st);
    launch_cell_sort(s->mixed, s->x, (int)N, s->cell_start, s->tmp, s->fp.mtype, s->cellc, s->site, s->reps, s->n_reps, s->C,
                     s->S, s->perm, s->inv_perm, s->pos, s->tag, s->ref, s->flags, s->st);
    cudaEventRecord(ev[1], s->st);
    launch_cl_build(s->pos, s->tag, s->cell_start, s->cl_start, s->regions, (int)s->regions_h.size(), s->shapes,
                    s->reps, s->list, s->ncl, s->cap, s->tile_cap, s->flags, 0, s->work,
                  s->generic ? &s->topo : nullptr, s->st);
    cudaEventRecord(ev[2], s->st);
    // host arm: positions to the host, bins there, binned data back, sorted arrays
    if (cudaMemcpyAsync(hx, s->x, xb, cudaMemcpyDeviceToHost, s->st) != cudaSuccess) { rc = fail(s, MD_ECUDA, "copy"); break; }
    cudaEventRecord(ev[3], s->st);
    if (cudaStreamSynchronize(s->st) != cudaSuccess) { rc = fail(s, MD_ECUDA, "sync"); break; }
    const auto t0 = std::chrono::steady_clock::now();
    if (s->mixed) host_bins((const double*)hx, s, cell_of, cellc, cell_start, cl_start, perm);
    else host_bins((const float*)hx, s, cell_of, cellc, cell_start, cl_start, perm);
    const auto t1 = std::chrono::steady_clock::now();
    cudaEventRecord(ev[4], s->st);
    bool ok = cudaMemcpyAsync(s->cell_of, cell_of.data(), N * sizeof(int), cudaMemcpyHostToDevice, s->st) == cudaSuccess &&
              cudaMemcpyAsync(s->cellc, cellc.data(), N * sizeof(int), cudaMemcpyHostToDevice, s->st) == cudaSuccess &&
              cudaMemcpyAsync(s->cell_start, cell_start.data(), (C + 1) * sizeof(int), cudaMemcpyHostToDevice, s->st) == cudaSuccess &&
              cudaMemcpyAsync(s->cl_start, cl_start.data(), (C + 1) * sizeof(int), cudaMemcpyHostToDevice, s->st) == cudaSuccess &&
              cudaMemcpyAsync(s->tmp, perm.data(), N * sizeof(int), cudaMemcpyHostToDevice, s->st) == cudaSuccess;
    if (!ok) { rc = fail(s, MD_ECUDA, "copy"); break; }
    launch_cell_sort(s->mixed, s->x, (int)N, s->cell_start, s->tmp, s->fp.mtype, s->cellc, s->site, s->reps, s->n_reps, s->C,
                     s->S, s->perm, s->inv_perm, s->pos, s->tag, s->ref, s->flags, s->st);
    cudaEventRecord(ev[5], s->st);
    if (cudaStreamSynchronize(s->st) != cudaSuccess) { rc = fail(s, MD_ECUDA, "sync"); break; }
    float a, b, c, d;
    cudaEventElapsedTime(&a, ev[0], ev[1]);
    cudaEventElapsedTime(&b, ev[1], ev[2]);
    cudaEventElapsedTime(&c, ev[2], ev[3]);
    cudaEventElapsedTime(&d, ev[4], ev[5]);
    const double hb = std::chrono::duration<double, std::milli>(t1 - t0).count();
    acc[0] += a; acc[1] += b; acc[2] += c; acc[3] += hb; acc[4] += d; acc[5] += c + hb + d;
  }
  s->profile = prof;
  for (cudaEvent_t& e : ev) cudaEventDestroy(e);
  cudaFreeHost(hx);
  if (rc) return rc;
  // the list of the bins now in place
  launch_cl_build(s->pos, s->tag, s->cell_start, s->cl_start, s->regions, (int)s->regions_h.size(), s->shapes,
                  s->reps, s->list, s->ncl, s->cap, s->tile_cap, s->flags, 0, s->work,
                  s->generic ? &s->topo : nullptr, s->st);
  for (int k = 0; k < 6; ++k) ms[k] = acc[k] / reps;
  rc = check_flags(s);
  s->fresh = rc == MD_OK;
  return rc;
}

int md_early_rebins(md_system* s, int64_t* count) {
  if (!s || !count) return fail(s, MD_EINVAL, "bad arguments");
  unsigned long long v = 0;
  CU(cudaStreamSynchronize(s->st));
  CU(cudaMemcpy(&v, s->early, sizeof v, cudaMemcpyDeviceToHost));
  *count = (int64_t)v;
  return MD_OK;
}

int md_get_thermostat(md_system* s, double* xi) {
  if (!s || !xi) return fail(s, MD_EINVAL, "bad arguments");
  CU(cudaStreamSynchronize(s->st));
  std::vector<double> h(6 * (size_t)s->n_reps);
  CU(cudaMemcpy(h.data(), s->lam, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
  for (int r = 0; r < s->n_reps; ++r) xi[r] = s->thermo == MD_NOSE_HOOVER ? h[6 * r] : 0.0;
  return MD_OK;
}

void* md_stream(md_system* s) { return s ? (void*)s->st : nullptr; }

int md_info(md_system* s, int64_t* n_atoms, int64_t* n_cells, int32_t* cap, int32_t* M) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  if (n_atoms) *n_atoms = s->N;
  if (n_cells) *n_cells = s->C;
  if (cap) *cap = s->cap;
  if (M) *M = s->reps_h[0].M;
  return MD_OK;
}

int md_get_bins(md_system* s, int32_t* cell_of, int32_t* cell_start, int32_t* perm) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  CU(cudaStreamSynchronize(s->st));
  if (cell_of) CU(cudaMemcpy(cell_of, s->cell_of, s->N * sizeof(int), cudaMemcpyDeviceToHost));
  if (cell_start) CU(cudaMemcpy(cell_start, s->cell_start, (s->C + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  if (perm) CU(cudaMemcpy(perm, s->perm, s->N * sizeof(int), cudaMemcpyDeviceToHost));
  return MD_OK;
}

int md_get_neighbors(md_system* s, int32_t* count, int32_t* entries) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  CU(cudaStreamSynchronize(s->st));
  const size_t N = (size_t)s->N;
  std::vector<int> pm(N), cs(s->C + 1), cls(s->C + 1);
  CU(cudaMemcpy(pm.data(), s->perm, N * sizeof(int), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(cs.data(), s->cell_start, (s->C + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(cls.data(), s->cl_start, (s->C + 1) * sizeof(int), cudaMemcpyDeviceToHost));
  const size_t ncl_used = (size_t)cls[s->C];
  std::vector<int> nc(ncl_used);
  std::vector<unsigned> lst(ncl_used * s->cap);
  if (ncl_used) {
    CU(cudaMemcpy(nc.data(), s->ncl, ncl_used * sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(lst.data(), s->list, lst.size() * sizeof(unsigned), cudaMemcpyDeviceToHost));
  }
  // every listed pair, both ways, by original atom index: the region tiles
  // rebuilt here exactly as the kernels stage them
  std::vector<std::vector<int>> nb(N);
  for (const Region& g : s->regions_h) {
    const RegionShape& S = s->shapes_h[g.shape];
    const RepDev& q = s->reps_h[g.rep];
    const int M = q.M;
    int start[kMaxTileCells], off[kMaxTileCells + 1], cell[kMaxTileCells];
    off[0] = 0;
    for (int k = 0; k < S.n_tile; ++k) {
      const int cx = (g.ox + S.off[k][0] + M) % M, cy = (g.oy + S.off[k][1] + M) % M, cz = (g.oz + S.off[k][2] + M) % M;
      cell[k] = q.cell_base + (cz * M + cy) * M + cx;
      start[k] = cs[cell[k]];
      off[k + 1] = off[k] + cs[cell[k] + 1] - cs[cell[k]];
    }
    for (int h = 0; h < S.n_home; ++h) {
      const int n_h = off[h + 1] - off[h];
      for (int kq = 0; kq < (n_h + 3) / 4; ++kq) {
        const int cl = cls[cell[h]] + kq;
        for (int e = 0; e < nc[cl]; ++e) {
          const unsigned E = lst[(size_t)cl * s->cap + e];
          const int t = (int)(E & 0xffffu);
          int kc = 0;
          while (kc + 1 < S.n_tile && off[kc + 1] <= t) ++kc;
          const int j = pm[start[kc] + (t - off[kc])];
          for (int u = 0; u < 4; ++u)
            if ((E >> (16 + u)) & 1u) {
              const int i = pm[start[h] + 4 * kq + u];
              nb[i].push_back(j);
              nb[j].push_back(i);
            }
        }
      }
    }
  }
  for (size_t i = 0; i < N; ++i) {
    if ((int)nb[i].size() > s->cap) return fail(s, MD_EOVERFLOW, "an atom has more listed neighbours than the capacity");
    if (count) count[i] = (int)nb[i].size();
    if (entries)
      for (size_t m = 0; m < nb[i].size(); ++m) entries[i * s->cap + m] = nb[i][m];
  }
  return MD_OK;
}

int md_get_cell_units(md_system* s, float* u) {
  if (!s || !u) return fail(s, MD_EINVAL, "bad arguments");
  CU(cudaStreamSynchronize(s->st));
  const size_t N = (size_t)s->N;
  std::vector<float4> p(N);
  std::vector<int> ip(N);
  CU(cudaMemcpy(p.data(), s->pos, N * sizeof(float4), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(ip.data(), s->inv_perm, N * sizeof(int), cudaMemcpyDeviceToHost));
  for (size_t i = 0; i < N; ++i) {
    const float4 q = p[ip[i]];
    u[3 * i] = q.x; u[3 * i + 1] = q.y; u[3 * i + 2] = q.z;
  }
  return MD_OK;
}

int md_profile_enable(md_system* s, int32_t on) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  CU(cudaStreamSynchronize(s->st));
  const int need = 3 + 3 * s->R + 1;
  while ((int)s->ev.size() < need) {
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    s->ev.push_back(e);
  }
  s->profile = on != 0;
  return capture_cycle(s);   // the graph carries the event records when on
}

int md_profile_read(md_system* s, double* ms, int64_t* n) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  for (int k = 0; k < kNumProf; ++k) {
    if (ms) ms[k] = s->prof_ms[k];
    if (n) n[k] = s->prof_n[k];
  }
  return MD_OK;
}

int md_profile_reset(md_system* s) {
  if (!s) return fail(s, MD_EINVAL, "null system");
  for (int k = 0; k < kNumProf; ++k) { s->prof_ms[k] = 0; s->prof_n[k] = 0; }
  return MD_OK;
}

int64_t md_launches_per_call(md_system* s, int64_t n) {
  if (!s || n <= 0) return 0;
  const int64_t full = n / s->R, rem = n % s->R;
  const bool check = s->disp == MD_DISP_REBUILD;
  return full * block_launches(s->R, check) + (rem ? block_launches((int)rem, check) : 0);
}

// ------------------------------------------------------------------ autotuner
static std::string tune_key(const md_desc* d) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  std::string name = "gpu";
  int sms = 0;
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) { name = prop.name; sms = prop.multiProcessorCount; }
  for (char& ch : name) if (ch == ' ') ch = '_';
  long long N = 0;
  double lmin = 1e300, lmax = 0.0;
  for (int r = 0; r < d->n_replicas; ++r) {
    N += (long long)d->n_chains[r] * d->sites_per_chain;
    lmin = std::min(lmin, d->box[r]);
    lmax = std::max(lmax, d->box[r]);
  }
  char buf[256];
  snprintf(buf, sizeof buf, "%s:%d:p%d:t%d:r%d:n%d:L%.1f-%.1f", name.c_str(), sms, d->precision, d->thermostat,
           d->n_replicas, (int)std::floor(2.0 * std::log2((double)std::max(N, 1LL))), std::round(2.0 * lmin) / 2.0,
           std::round(2.0 * lmax) / 2.0);
  return buf;
}

// time one candidate: create, one warm-up cycle, trial_cycles timed cycles
static int tune_trial(md_desc cand, int cycles, double* us) {
  cand.workspace = nullptr;
  cand.workspace_bytes = 0;
  cand.cuda_stream = nullptr;
  md_system* s = nullptr;
  int rc = md_create(&cand, &s);
  if (rc) return rc;
  rc = md_step(s, cand.rebin_every);
  if (!rc) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s->st);
    rc = md_step_async(s, (int64_t)cand.rebin_every * cycles);
    cudaEventRecord(b, s->st);
    if (!rc) rc = md_sync(s);
    float ms = 0.f;
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    *us = 1000.0 * ms / ((double)cand.rebin_every * cycles);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  md_destroy(s);
  return rc;
}

extern "C" int md_autotune(md_desc* d, int32_t trial_cycles, const char* cache_path, md_tuning* out) {
  if (!d || trial_cycles < 1) return fail(nullptr, MD_EINVAL, "autotune needs a descriptor and trial_cycles >= 1");
  const std::string key = tune_key(d);
  const int region0 = d->lj_region ? d->lj_region : 3;
  md_tuning best{d->skin, d->rebin_every, d->lj_block ? d->lj_block : (region0 == 3 ? 384 : 256), d->schedule,
                 d->lj_lanes ? d->lj_lanes : 8, region0, 0, 1e300};
  auto apply = [&](const md_tuning& t) {
    d->skin = t.skin; d->rebin_every = t.rebin_every; d->lj_block = t.lj_block; d->schedule = t.schedule;
    d->lj_lanes = t.lj_lanes; d->lj_region = t.lj_region;
  };
  if (cache_path) {
    if (FILE* f = fopen(cache_path, "r")) {
      char line[512], k[256];
      double skin, us;
      int R, blk, sch, lanes, reg;
      bool found = false;
      // one setting per line; lines of another layout are skipped
      while (fgets(line, sizeof line, f))
        if (sscanf(line, "%255s %lf %d %d %d %d %d %lf", k, &skin, &R, &blk, &sch, &lanes, &reg, &us) == 8 && key == k) {
          best = md_tuning{skin, R, blk, sch, lanes, reg, 1, us};
          found = true;
        }
      fclose(f);
      if (found) {
        apply(best);
        if (out) *out = best;
        return MD_OK;
      }
    }
  }
  bool any = false;
  // region side x block shape x schedule at the descriptor's cell size
  const int shapes[4][2] = {{2, 128}, {2, 256}, {3, 256}, {3, 384}};
  for (const auto& rb : shapes)
    for (int sch : {(int)MD_SCHED_GRID, (int)MD_SCHED_PERSISTENT}) {
      md_desc c = *d;
      c.lj_region = rb[0];
      c.lj_block = rb[1];
      c.schedule = sch;
      c.lj_lanes = best.lj_lanes;
      double us = 0.0;
      if (tune_trial(c, trial_cycles, &us) == MD_OK && us < best.us_per_step) {
        best = md_tuning{c.skin, c.rebin_every, rb[1], sch, best.lj_lanes, rb[0], 0, us};
        any = true;
      }
    }
  // lanes per cluster with that region, block shape and schedule
  for (int lanes : {8, 16, 32}) {
    if (lanes == best.lj_lanes) continue;
    md_desc c = *d;
    c.lj_region = best.lj_region;
    c.lj_block = best.lj_block;
    c.schedule = best.schedule;
    c.lj_lanes = lanes;
    double us = 0.0;
    if (tune_trial(c, trial_cycles, &us) == MD_OK && us < best.us_per_step) {
      best = md_tuning{c.skin, c.rebin_every, best.lj_block, best.schedule, lanes, best.lj_region, 0, us};
      any = true;
    }
  }
  // cell size through (skin, rebin interval)
  const double skins[4] = {0.08, 0.10, 0.12, 0.15};
  const int reb[4] = {6, 10, 12, 16};
  for (int k = 0; k < 4; ++k) {
    if (skins[k] == best.skin && reb[k] == best.rebin_every) continue;
    md_desc c = *d;
    c.lj_region = best.lj_region;
    c.lj_block = best.lj_block;
    c.schedule = best.schedule;
    c.lj_lanes = best.lj_lanes;
    c.skin = skins[k];
    c.rebin_every = reb[k];
    double us = 0.0;
    if (tune_trial(c, trial_cycles, &us) == MD_OK && us < best.us_per_step) {
      best = md_tuning{skins[k], reb[k], best.lj_block, best.schedule, best.lj_lanes, best.lj_region, 0, us};
      any = true;
    }
  }
  if (!any) return fail(nullptr, MD_EUNSTABLE, "autotune: no candidate ran cleanly");
  apply(best);
  if (cache_path)
    if (FILE* f = fopen(cache_path, "a")) {
      fprintf(f, "%s %.4f %d %d %d %d %d %.3f\n", key.c_str(), best.skin, best.rebin_every, best.lj_block, best.schedule,
              best.lj_lanes, best.lj_region, best.us_per_step);
      fclose(f);
    }
  if (out) *out = best;
  return MD_OK;
}

void md_destroy(md_system* s) {
  if (!s) return;
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->cycle) cudaGraphExecDestroy(s->cycle);
  if (s->cycle_fresh) cudaGraphExecDestroy(s->cycle_fresh);
  drop_rem_graphs(s);
  if (s->side) cudaStreamDestroy(s->side);
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  if (s->own_mem && s->base) cudaFree(s->base);
  if (s->acf_ring) cudaFree(s->acf_ring);
  if (s->acf_acc) cudaFree(s->acf_acc);
  if (s->own_stream && s->st) cudaStreamDestroy(s->st);
  delete s;
}

const char* md_last_error(const md_system* s) { return s ? s->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
