// C ABI of the IUGKP CUDA library (declared in include/iugkp.h): context set-up
// (geometry, band split, per-(band, cell) coefficients, diffusion stencil), and the
// host loops of the steady and adjoint iterations (arXiv 2506.09465 Sec. 3-4).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"

using namespace iugkp;

struct iugkp_ctx {
  Ctx c;
};

namespace iugkp {

static thread_local std::string g_create_error;

iugkp_status fail(Ctx* c, iugkp_status s, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_error = msg;
  return s;
}

iugkp_status cuda_fail(Ctx* c, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return fail(c, IUGKP_ECUDA, m);
}

}  // namespace iugkp

#define CK(call, what)                                         \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what);      \
  } while (0)

namespace {

iugkp_status ensure_k32(Ctx* c);

// Multiplier of the device's exact division by d (>= 1): M = floor((2^32 - 1) / d).
unsigned div_magic(int d) { return (unsigned)(0xFFFFFFFFull / (unsigned long long)std::max(1, d)); }

// Largest acceptance ratio (FP32) over each cell and its neighbours across faces, edges and
// corners, per instance and band: a candidate whose acceptance draw exceeds it is rejected
// whichever of those cells it lies in.
std::vector<float> neighbour_max_ratio(const Ctx* c, const std::vector<float>& r32) {
  std::vector<float> out(r32.size());
  for (const InstDesc& in : c->h_inst) {
    const int nx = in.n[0], ny = in.n[1], nz = in.n[2];
    for (int b = 0; b < c->nb; ++b) {
      const float* r = r32.data() + in.bc_off + (size_t)b * in.ncells;
      float* o = out.data() + in.bc_off + (size_t)b * in.ncells;
      for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
          for (int x = 0; x < nx; ++x) {
            float m = 0.f;
            for (int k = std::max(z - 1, 0); k <= std::min(z + 1, nz - 1); ++k)
              for (int j = std::max(y - 1, 0); j <= std::min(y + 1, ny - 1); ++j)
                for (int i = std::max(x - 1, 0); i <= std::min(x + 1, nx - 1); ++i)
                  m = std::max(m, r[i + (size_t)nx * (j + (size_t)ny * k)]);
            o[x + (size_t)nx * (y + (size_t)ny * z)] = m;
          }
    }
  }
  return out;
}

// Largest-remainder split of N over weights r (r > 0, N >= nb): one particle per band
// first, the remaining N - nb in proportion to r, leftovers to the largest fractional
// parts (lower band first on ties).
bool split_counts(long long N, const std::vector<double>& r, std::vector<long long>& out) {
  const int nb = (int)r.size();
  if (nb < 1 || N < nb) return false;
  double rs = 0.0;
  for (double x : r) {
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    rs += x;
  }
  const long long rest = N - nb;
  out.assign(nb, 1);
  std::vector<double> frac(nb);
  long long given = 0;
  for (int b = 0; b < nb; ++b) {
    double share = (double)rest * r[b] / rs;
    long long whole = (long long)std::floor(share);
    out[b] += whole;
    frac[b] = share - (double)whole;
    given += whole;
  }
  std::vector<int> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return frac[x] > frac[y]; });
  for (long long k = 0; k < rest - given; ++k) out[order[(size_t)(k % nb)]] += 1;
  return true;
}

template <typename T>
iugkp_status dalloc(Ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? IUGKP_ENOMEM : IUGKP_ECUDA,
                std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
  }
  return IUGKP_OK;
}

template <typename T>
iugkp_status upload(Ctx* c, T** p, const std::vector<T>& h) {
  iugkp_status s = dalloc(c, p, h.size());
  if (s != IUGKP_OK) return s;
  CK(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice), "upload");
  return IUGKP_OK;
}

void free_all(Ctx* c) {
  void* ptrs[] = {c->d_vtm32, c->d_perm, c->d_wmax_bpre, c->d_inst, c->d_groups_all, c->d_groups_fwd, c->d_coef, c->d_ratio64, c->d_ratio32, c->d_ratio_nb32, c->d_taumaj,
                  c->d_v, c->d_wcoef, c->d_wallT, c->d_srcshift, c->d_source, c->d_m, c->d_Vm, c->d_invVm, c->d_VC,
                  c->d_theta, c->d_theta_m, c->d_diag, c->d_cx, c->d_cy, c->d_cz, c->d_pcg, c->d_work, c->d_T2,
                  c->d_R, c->d_W, c->d_F, c->d_wall, c->d_red, c->d_counters, c->d_work_counter, c->d_err,
                  c->d_pcg_iters, c->d_scalar, c->d_adj, c->d_mg, c->d_mg_diag, c->d_mg_dinv, c->d_mg_cx,
                  c->d_mg_cy, c->d_mg_cz, c->d_mg_cinv, c->d_mg_b, c->d_mg_x, c->d_mg_t, c->d_mg_r, c->d_fd_q, c->d_fd_lam,
                  c->d_inst_beg, c->d_inst_end, c->d_inst_next, c->d_cost_prefix, c->d_window, c->d_wmax,
                  c->d_group_mag, c->d_mag, c->d_wall_unit, c->d_all_beg, c->d_all_end, c->d_all_cost_prefix,
                  c->d_all_group_mag, c->d_R32, c->d_W32, c->d_F32, c->d_m2, c->d_wallTf,
                  c->d_pslot_off, c->d_phome_off, c->d_pnband, c->d_pnwall, c->d_px, c->d_pband, c->d_phome,
                  c->d_pcount, c->d_pfcount, c->d_phome_w, c->d_wemit, c->d_DY, c->d_EY, c->d_GX, c->d_Fd,
                  c->d_all_real, c->d_defer, c->d_defer_n};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->d_res_block) cudaFree(c->d_res_block);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->graph_stream) cudaStreamDestroy(c->graph_stream);
}

bool grid_ok(const iugkp_grid& g, int dim) {
  if (g.dim != dim || dim < 1 || dim > 3) return false;
  const int n[3] = {g.nx, g.ny, g.nz};
  const double l[3] = {g.lx, g.ly, g.lz};
  long long cells = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 1 || !(l[a] > 0.0) || !std::isfinite(l[a])) return false;
    cells *= n[a];
  }
  return cells < (1ll << 30);
}

// Emission temperature shift Q / m for every cell of every instance (or clears it).
iugkp_status set_source(Ctx* c, const std::vector<double>& Q, const std::vector<double>& m) {
  bool any = false;
  for (double q : Q) any |= (q != 0.0);
  if (!any) {
    if (c->d_srcshift) cudaFree(c->d_srcshift);
    c->d_srcshift = nullptr;
    return IUGKP_OK;
  }
  std::vector<double> shift(Q.size());
  for (size_t i = 0; i < Q.size(); ++i) shift[i] = Q[i] / m[i];
  if (!c->d_srcshift) {
    iugkp_status s = dalloc(c, &c->d_srcshift, shift.size());
    if (s != IUGKP_OK) return s;
  }
  CK(cudaMemcpy(c->d_srcshift, shift.data(), shift.size() * sizeof(double), cudaMemcpyHostToDevice), "source");
  return IUGKP_OK;
}

// Per-instance particle ranges of a group list (groups are ordered by instance), the
// prefix sums of the estimated cost (particles x expected events per particle) and the
// reciprocal of each group's emitter count.
void staged_tables(const Ctx* c, const std::vector<Group>& groups, std::vector<long long>& beg,
                   std::vector<long long>& end, std::vector<double>& prefix, double& total,
                   std::vector<unsigned>& gmag) {
  beg.assign(c->n_inst, 0);
  end.assign(c->n_inst, 0);
  std::vector<double> cost(c->n_inst, 0.0);
  std::vector<int> seen(c->n_inst, 0);
  gmag.clear();
  for (const Group& g : groups) {
    gmag.push_back(div_magic(g.n_emitters));
    const long long np = (long long)g.n_emitters * g.per_emitter;
    if (!seen[g.inst]) {
      beg[g.inst] = g.first_particle;
      end[g.inst] = g.first_particle;
      seen[g.inst] = 1;
    }
    end[g.inst] = g.first_particle + np;
    const InstDesc& in = c->h_inst[g.inst];
    double hmin = in.h[0];
    for (int a = 1; a < in.dim; ++a) hmin = std::min(hmin, in.h[a]);
    const double lam = c->h_v[g.band] * c->h_taumean[(size_t)g.inst * c->nb + g.band];
    const double nmax = (double)std::max(in.n[0], std::max(in.n[1], in.n[2]));
    cost[g.inst] += (double)np * (1.0 + std::min(lam / hmin, nmax));
  }
  prefix.assign(c->n_inst, 0.0);
  total = 0.0;
  for (int k = 0; k < c->n_inst; ++k) {
    prefix[k] = total;
    total += cost[k];
  }
}

// Visiting order of each group's emitters in the staged sweep: stable-sorted by the class
// floor(2 log2(tau / tau_maj)) of the emitter's cell (a wall face: the cell behind it), from
// the expected number of candidates per real collision, so that a warp's lanes (consecutive
// emitters) walk chains of similar length. Groups whose emitters share one class keep the
// emitter order (perm_off = -1). Draws are keyed by (emitter, particle): the order changes
// which lane traces a particle, not the particle. Sets perm_off of h_groups_all; returns the
// concatenated orders (one entry at least).
std::vector<int> emitter_orders(Ctx* c, const std::vector<float>& r32) {
  std::vector<int> perm;
  for (Group& g : c->h_groups_all) {
    g.perm_off = -1;
    const InstDesc& in = c->h_inst[g.inst];
    const float* r = r32.data() + in.bc_off + (long long)g.band * in.ncells;
    std::vector<int> cls(g.n_emitters);
    for (int e = 0; e < g.n_emitters; ++e) {
      long long cell = e;
      if (g.kind > 0) {
        const int wl = g.kind - 1, a = wl >> 1, side = wl & 1;
        const int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
        int idx[3];
        idx[a] = side ? in.n[a] - 1 : 0;
        idx[o1] = e % in.n[o1];
        idx[o2] = e / in.n[o1];
        cell = idx[0] + (long long)in.n[0] * (idx[1] + (long long)in.n[1] * idx[2]);
      }
      // r = tau_maj / tau <= 1 is the acceptance probability: 1 / r candidates per real one
      cls[e] = (int)std::floor(-2.0 * std::log2(std::min(1.0, std::max(1e-30, (double)r[cell]))));
    }
    if (std::all_of(cls.begin(), cls.end(), [&](int x) { return x == cls[0]; })) continue;
    if ((long long)perm.size() + g.n_emitters > 0x7fffffffll) continue;
    std::vector<int> order(g.n_emitters);
    for (int e = 0; e < g.n_emitters; ++e) order[e] = e;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cls[x] < cls[y]; });
    g.perm_off = (int)perm.size();
    perm.insert(perm.end(), order.begin(), order.end());
  }
  if (perm.empty()) perm.push_back(0);
  return perm;
}

// Per-face wall temperatures from the per-wall values (every face of a wall alike).
void broadcast_wall_T(Ctx* c) {
  c->h_wallTf.assign((size_t)c->total_bfaces, 0.0);
  for (const InstDesc& in : c->h_inst)
    for (int w = 0; w < 2 * in.dim; ++w) {
      const int a = w >> 1;
      const int nf = in.n[(a + 1) % 3] * in.n[(a + 2) % 3];
      for (int j = 0; j < nf; ++j) c->h_wallTf[in.bface_off + in.wface_off[w] + j] = c->h_wallT[in.wall_off + w];
    }
}

// Forward groups leave out walls whose faces are all at zero temperature (their
// particles weigh zero).
iugkp_status rebuild_forward_groups(Ctx* c) {
  c->h_groups_fwd.clear();
  long long off = 0;
  for (const Group& g0 : c->h_groups_all) {
    if (g0.kind > 0) {
      const InstDesc& in = c->h_inst[g0.inst];
      const int wl = g0.kind - 1;
      const long long f0 = in.bface_off + in.wface_off[wl];
      bool hot = false;
      for (long long j = 0; j < g0.n_emitters && !hot; ++j) hot = c->h_wallTf[f0 + j] != 0.0;
      if (!hot) continue;
    }
    Group g = g0;
    g.first_particle = off;
    off += (long long)g.n_emitters * g.per_emitter;
    c->h_groups_fwd.push_back(g);
  }
  if (c->h_groups_fwd.empty()) {  // keep one (all-zero) group so kernels see a valid table
    Group g = c->h_groups_all[0];
    g.first_particle = 0;
    c->h_groups_fwd.push_back(g);
    off = 0;
  }
  c->fwd_particles = off;
  if (c->d_groups_fwd) cudaFree(c->d_groups_fwd);
  c->d_groups_fwd = nullptr;
  iugkp_status s = upload(c, &c->d_groups_fwd, c->h_groups_fwd);
  if (s != IUGKP_OK) return s;
  {
    // w_max pre-pass: each group's blocks in proportion to its emitters, about two blocks per
    // SM in all, at least WMAX_MIN_CHUNK emitters per block
    long long total = 0;
    for (const Group& g : c->h_groups_fwd) total += g.n_emitters;
    const long long nblk = 2 * (long long)std::max(1, c->sm_count);
    const long long chunk = std::max<long long>(WMAX_MIN_CHUNK, (total + nblk - 1) / nblk);
    std::vector<int> bpre(1, 0);
    for (const Group& g : c->h_groups_fwd) bpre.push_back(bpre.back() + (int)((g.n_emitters + chunk - 1) / chunk));
    c->wmax_blocks = bpre.back();
    if (c->d_wmax_bpre) cudaFree(c->d_wmax_bpre);
    c->d_wmax_bpre = nullptr;
    if ((s = upload(c, &c->d_wmax_bpre, bpre)) != IUGKP_OK) return s;
  }
  // Staged sweep: each instance's forward particles are contiguous (groups are ordered
  // by instance); blocks start on instances in proportion to the estimated cost.
  std::vector<long long> beg, end;
  std::vector<double> prefix;
  std::vector<unsigned> gmag;
  double tot = 0.0;
  staged_tables(c, c->h_groups_fwd, beg, end, prefix, tot, gmag);
  c->cost_total = tot;
  // Shared-memory face window. 2D instances whose faces all fit take every face (two-group
  // tallies); otherwise the window holds all x-faces when they fit, else a centred run of
  // them (the rest take global atomics).
  std::vector<int2> window(c->n_inst);
  c->any_two_group = false;
  c->all_two_group = c->dim == 2;
  c->sync_ok = c->dim == 2;
  c->sync_partial = false;
  for (int k = 0; k < c->n_inst; ++k) {
    const InstDesc& in = c->h_inst[k];
    const long long X = (long long)(in.n[0] + 1) * in.n[1] * in.n[2];
    if (c->dim == 2 && in.nfaces <= c->staged_cap) {
      window[k] = make_int2(0, (int)in.nfaces);
      c->any_two_group = true;
      continue;
    }
    c->all_two_group = false;
    // 3D: no face window (the dynamic shared memory holds the warps' item tables)
    const long long len = c->dim == 3 ? 0 : std::min<long long>(X, c->staged_cap);
    window[k] = make_int2((int)((X - len) / 2), (int)len);
    if (len < X) c->sync_partial = true;
  }
  void* olds[] = {c->d_inst_beg, c->d_inst_end, c->d_cost_prefix, c->d_window, c->d_group_mag};
  for (void* p : olds)
    if (p) cudaFree(p);
  c->d_inst_beg = c->d_inst_end = nullptr;
  c->d_cost_prefix = nullptr;
  c->d_window = nullptr;
  c->d_group_mag = nullptr;
  if ((s = upload(c, &c->d_group_mag, gmag)) != IUGKP_OK) return s;
  if ((s = upload(c, &c->d_inst_beg, beg)) != IUGKP_OK) return s;
  if ((s = upload(c, &c->d_inst_end, end)) != IUGKP_OK) return s;
  if ((s = upload(c, &c->d_cost_prefix, prefix)) != IUGKP_OK) return s;
  return upload(c, &c->d_window, window);
}

}  // namespace

extern "C" {

void iugkp_default_options(iugkp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = IUGKP_TRACK_FP32;
  o->tally = IUGKP_TALLY_STAGED;
  o->draws = IUGKP_DRAWS_FROZEN;
  o->newton = 1;
  o->schedule = IUGKP_SCHED_PERSISTENT;
  o->particles_per_cell = 1024;
  o->particles_per_wall_face = 1024;
  o->seed = 0;
  o->epoch0 = 0;
  o->instance_base = 0;
  o->cg_rtol = 1e-3;
  o->cg_maxit = 5000;
  o->step_budget = 1ll << 24;
  o->block_threads = 0;
  o->blocks_per_sm = 0;
  o->refill_lanes = 0;
  o->use_graphs = 1;
  o->warp_grab = 0;
  o->walk_k = 0;
}

const char* iugkp_last_error(const iugkp_ctx* ctx) {
  return ctx ? ctx->c.err.c_str() : g_create_error.c_str();
}

iugkp_status iugkp_create_batch(int n, const iugkp_grid* g, const double* const* tau, const iugkp_bands* b,
                                const double* const* wall_T, const double* const* source, const iugkp_options* o,
                                iugkp_ctx** out) {
  Ctx* c = nullptr;
  if (!out) return fail(nullptr, IUGKP_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !g || !tau || !b || !wall_T || !o) return fail(nullptr, IUGKP_EINVAL, "NULL argument or n < 1");
  if (b->nb < 1 || b->nb > 255 || !b->C || !b->v) return fail(nullptr, IUGKP_EINVAL, "bands: need 1 <= nb <= 255");
  for (int k = 0; k < b->nb; ++k)
    if (!(b->C[k] > 0.0) || !(b->v[k] > 0.0) || !std::isfinite(b->C[k]) || !std::isfinite(b->v[k]))
      return fail(nullptr, IUGKP_EINVAL, "bands: C and v must be finite and > 0");
  const int dim = g[0].dim;
  for (int k = 0; k < n; ++k)
    if (!grid_ok(g[k], dim) || !tau[k] || !wall_T[k])
      return fail(nullptr, IUGKP_EINVAL, "grid " + std::to_string(k) + " invalid (dim, sizes, lengths) or NULL field");
  if (o->precision != IUGKP_TRACK_FP32 && o->precision != IUGKP_TRACK_FP64)
    return fail(nullptr, IUGKP_EINVAL, "options.precision");
  if (o->tally != IUGKP_TALLY_FP64 && o->tally != IUGKP_TALLY_STAGED && o->tally != IUGKP_TALLY_STAGED_K32)
    return fail(nullptr, IUGKP_EINVAL, "options.tally");
  if (o->tally == IUGKP_TALLY_STAGED_K32 && o->precision != IUGKP_TRACK_FP32)
    return fail(nullptr, IUGKP_EINVAL, "options.tally: compensated FP32 tallies need FP32 tracking");
  if (o->particles_per_cell < b->nb || o->particles_per_wall_face < b->nb || o->particles_per_cell > (1ll << 31) ||
      o->particles_per_wall_face > (1ll << 31))
    return fail(nullptr, IUGKP_EINVAL, "particles per cell / wall face must be in [nb, 2^31]");
  if (!(o->cg_rtol > 0.0) || o->cg_maxit < 1 || o->step_budget < 1) return fail(nullptr, IUGKP_EINVAL, "cg / budget options");
  if (o->draws != IUGKP_DRAWS_FRESH && o->draws != IUGKP_DRAWS_FROZEN) return fail(nullptr, IUGKP_EINVAL, "options.draws");
  // Field values, checked before any CUDA call.
  for (int k = 0; k < n; ++k) {
    long long nc = (long long)g[k].nx * (dim >= 2 ? g[k].ny : 1) * (dim >= 3 ? g[k].nz : 1);
    for (long long i = 0; i < (long long)b->nb * nc; ++i)
      if (!(tau[k][i] > 0.0) || !std::isfinite(tau[k][i]))
        return fail(nullptr, IUGKP_EINVAL, "tau must be finite and > 0 (instance " + std::to_string(k) + ")");
    for (int w = 0; w < 2 * dim; ++w)
      if (!std::isfinite(wall_T[k][w])) return fail(nullptr, IUGKP_EINVAL, "wall temperature not finite");
    if (source && source[k])
      for (long long i = 0; i < nc; ++i)
        if (!std::isfinite(source[k][i])) return fail(nullptr, IUGKP_EINVAL, "source not finite");
  }
  if (o->refill_lanes < 0 || o->refill_lanes > 32) return fail(nullptr, IUGKP_EINVAL, "refill_lanes must be in 0..32");
  if (o->warp_grab < 0 || o->warp_grab > (1 << 20) || o->walk_k < 0 || o->walk_k > 4096)
    return fail(nullptr, IUGKP_EINVAL, "warp_grab must be in 0..2^20 and walk_k in 0..4096");

  iugkp_ctx* ctx = new (std::nothrow) iugkp_ctx();
  if (!ctx) return fail(nullptr, IUGKP_ENOMEM, "host allocation failed");
  c = &ctx->c;
  c->opt = *o;
  c->n_inst = n;
  c->dim = dim;
  c->h_grids.assign(g, g + n);
  c->nb = b->nb;
  c->h_C.assign(b->C, b->C + b->nb);
  c->h_v.assign(b->v, b->v + b->nb);
  const int nb = b->nb;
  auto bail = [&](iugkp_status s) {
    g_create_error = c->err;
    free_all(c);
    delete ctx;
    return s;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    fail(c, IUGKP_ECUDA, "no CUDA device");
    return bail(IUGKP_ECUDA);
  }
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  c->smem_optin = (size_t)optin;

  // Geometry and offsets.
  long long cell_off = 0, face_off = 0;
  for (int k = 0; k < n; ++k) {
    InstDesc in;
    std::memset(&in, 0, sizeof(in));
    in.dim = dim;
    const int nn[3] = {g[k].nx, g[k].ny, g[k].nz};
    const double ll[3] = {g[k].lx, g[k].ly, g[k].lz};
    for (int a = 0; a < 3; ++a) {
      in.n[a] = a < dim ? nn[a] : 1;
      in.h[a] = a < dim ? ll[a] / nn[a] : 1.0;
    }
    in.ncells = in.n[0] * in.n[1] * in.n[2];
    in.V = in.h[0] * in.h[1] * in.h[2];
    for (int a = 0; a < 3; ++a) in.hf[a] = (float)in.h[a];
    in.refill = 8;
    in.cell_off = cell_off;
    in.bc_off = (long long)nb * cell_off;
    in.face_off = face_off;
    long long fo = 0;
    for (int a = 0; a < 3; ++a) {
      in.fax_off[a] = fo;
      if (a < dim) {
        long long m = 1;
        for (int d = 0; d < 3; ++d) m *= (d == a) ? in.n[d] + 1 : in.n[d];
        fo += m;
      }
    }
    in.nfaces = fo;
    in.wall_off = 2 * dim * k;
    in.bface_off = c->total_bfaces;
    {
      int wf = 0;
      for (int w = 0; w < 6; ++w) {
        in.wface_off[w] = wf;
        if (w < 2 * dim) wf += in.n[((w >> 1) + 1) % 3] * in.n[((w >> 1) + 2) % 3];
      }
      c->total_bfaces += wf;
    }
    in.inst_id = o->instance_base + (unsigned)k;
    c->h_inst.push_back(in);
    cell_off += in.ncells;
    face_off += fo;
    c->max_inst_cells = std::max(c->max_inst_cells, in.ncells);
    c->max_inst_faces = (int)std::max<long long>(c->max_inst_faces, fo);
  }
  c->total_cells = cell_off;
  c->total_faces = face_off;
  c->total_walls = 2LL * dim * n;

  // Per (instance, band, cell) and per-cell coefficients.
  std::vector<double> coef((size_t)nb * cell_off), r64((size_t)nb * cell_off), taumaj((size_t)n * nb);
  std::vector<float> r32((size_t)nb * cell_off);
  std::vector<double> m(cell_off, 0.0), Vm(cell_off), invVm(cell_off), VC(cell_off), kap(cell_off, 0.0);
  std::vector<double> wcoef((size_t)n * nb * 6, 0.0), wallTv(c->total_walls), Qv(cell_off, 0.0);
  std::vector<double> diag(cell_off, 0.0), cx(cell_off, 0.0), cy(cell_off, 0.0), cz(cell_off, 0.0), theta_m(cell_off);
  double csum = 0.0, cvsum = 0.0;
  for (int bb = 0; bb < nb; ++bb) {
    csum += c->h_C[bb];
    cvsum += c->h_C[bb] * c->h_v[bb];
  }
  std::vector<double> rwall(nb);
  for (int bb = 0; bb < nb; ++bb) rwall[bb] = c->h_C[bb] * c->h_v[bb];
  std::vector<long long> nwall;
  if (!split_counts(o->particles_per_wall_face, rwall, nwall)) {
    fail(c, IUGKP_EINVAL, "wall particle split");
    return bail(IUGKP_EINVAL);
  }
  long long total_particles = 0;
  for (int k = 0; k < n; ++k) {
    const InstDesc& in = c->h_inst[k];
    const long long nc = in.ncells;
    std::vector<double> rb(nb, 0.0);
    for (int bb = 0; bb < nb; ++bb) {
      double tmin = INFINITY, inv_sum = 0.0;
      for (long long i = 0; i < nc; ++i) {
        const double t = tau[k][(size_t)bb * nc + i];
        if (!(t > 0.0) || !std::isfinite(t)) {
          fail(c, IUGKP_EINVAL, "tau must be finite and > 0 (instance " + std::to_string(k) + ")");
          return bail(IUGKP_EINVAL);
        }
        tmin = std::min(tmin, t);
        inv_sum += 1.0 / t;
      }
      taumaj[(size_t)k * nb + bb] = tmin;
      rb[bb] = c->h_C[bb] * (inv_sum / (double)nc);
      c->h_taumean.push_back((double)nc / inv_sum);
    }
    std::vector<long long> nband;
    if (!split_counts(o->particles_per_cell, rb, nband)) {
      fail(c, IUGKP_EINVAL, "band particle split");
      return bail(IUGKP_EINVAL);
    }
    for (int bb = 0; bb < nb; ++bb) {
      for (long long i = 0; i < nc; ++i) {
        const size_t j = (size_t)in.bc_off + (size_t)bb * nc + i;
        const double t = tau[k][(size_t)bb * nc + i];
        coef[j] = c->h_C[bb] * in.V / (t * (double)nband[bb]);
        r64[j] = taumaj[(size_t)k * nb + bb] / t;
        r32[j] = (float)r64[j];
        m[in.cell_off + i] += c->h_C[bb] / t;
        kap[in.cell_off + i] += c->h_C[bb] * c->h_v[bb] * c->h_v[bb] * t / 3.0;
      }
      for (int w = 0; w < 2 * dim; ++w) {
        const int a = w >> 1;
        const double A = (a == 0 ? in.h[1] * in.h[2] : (a == 1 ? in.h[0] * in.h[2] : in.h[0] * in.h[1]));
        wcoef[((size_t)k * nb + bb) * 6 + w] = c->h_C[bb] * c->h_v[bb] * A / (4.0 * (double)nwall[bb]);
      }
    }
    for (int w = 0; w < 2 * dim; ++w) {
      const double tw = wall_T[k][w];
      if (!std::isfinite(tw)) {
        fail(c, IUGKP_EINVAL, "wall temperature not finite");
        return bail(IUGKP_EINVAL);
      }
      wallTv[in.wall_off + w] = tw;
    }
    if (source && source[k]) {
      for (long long i = 0; i < nc; ++i) {
        if (!std::isfinite(source[k][i])) {
          fail(c, IUGKP_EINVAL, "source not finite");
          return bail(IUGKP_EINVAL);
        }
        Qv[in.cell_off + i] = source[k][i];
      }
    }
    // Cell sums and the diffusion stencil (Sec. 3.3): face kappa harmonic; walls take
    // the half-cell conduction in series with the vacuum condition (flux = cv/2 dT).
    double hmin = in.h[0];
    for (int a = 1; a < dim; ++a) hmin = std::min(hmin, in.h[a]);
    double tmax = 0.0;
    const long long sx = 1, sy = in.n[0], sz = (long long)in.n[0] * in.n[1];
    const long long strides[3] = {sx, sy, sz};
    for (long long i = 0; i < nc; ++i) {
      const long long gi = in.cell_off + i;
      Vm[gi] = in.V * m[gi];
      invVm[gi] = 1.0 / Vm[gi];
      VC[gi] = in.V * csum;
      tmax = std::max(tmax, hmin / std::sqrt(3.0 * kap[gi] / m[gi]));
      const int idx[3] = {(int)(i % in.n[0]), (int)((i / in.n[0]) % in.n[1]), (int)(i / sz)};
      double d = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double hh = in.h[a] * in.h[a];
        for (int side = -1; side <= 1; side += 2) {
          const int j = idx[a] + side;
          if (j < 0 || j >= in.n[a]) {
            const double G = 1.0 / (in.h[a] / (2.0 * kap[gi]) + 2.0 / cvsum);
            d += G / in.h[a];
          } else {
            const long long gn = gi + side * strides[a];
            const double kf = 2.0 * kap[gi] * kap[gn] / (kap[gi] + kap[gn]);
            d += kf / hh;
            if (side > 0) (a == 0 ? cx : (a == 1 ? cy : cz))[gi] = kf / hh;
          }
        }
      }
      diag[gi] = d;
    }
    const double theta = std::min(1.0, 1.5 / tmax);
    c->h_theta.push_back(theta);
    for (long long i = 0; i < nc; ++i) theta_m[in.cell_off + i] = theta * m[in.cell_off + i];
    // Emitter groups: thermal per band, then each wall per band.
    for (int bb = 0; bb < nb; ++bb) {
      Group gr;
      std::memset(&gr, 0, sizeof(gr));
      gr.first_particle = total_particles;
      gr.inst = k;
      gr.band = bb;
      gr.kind = 0;
      gr.n_emitters = in.ncells;
      gr.per_emitter = (int)nband[bb];
      total_particles += (long long)gr.n_emitters * gr.per_emitter;
      c->h_groups_all.push_back(gr);
    }
    for (int bb = 0; bb < nb; ++bb) {
      for (int w = 0; w < 2 * dim; ++w) {
        const int a = w >> 1;
        Group gr;
        std::memset(&gr, 0, sizeof(gr));
        gr.first_particle = total_particles;
        gr.inst = k;
        gr.band = bb;
        gr.kind = 1 + w;
        gr.n_emitters = in.n[(a + 1) % 3] * in.n[(a + 2) % 3];
        gr.per_emitter = (int)nwall[bb];
        total_particles += (long long)gr.n_emitters * gr.per_emitter;
        c->h_groups_all.push_back(gr);
      }
    }
    c->h_nband.insert(c->h_nband.end(), nband.begin(), nband.end());
    {
      // Refill threshold of the staged sweep: long flights keep lanes busy (refill early,
      // few lanes at a time); short flights are dominated by emission (refill in bulk).
      double ev = 0.0, wsum = 0.0;
      for (int bb = 0; bb < nb; ++bb) {
        const double lam = c->h_v[bb] * c->h_taumean[(size_t)k * nb + bb];
        const double nmax = (double)std::max(in.n[0], std::max(in.n[1], in.n[2]));
        ev += (double)nband[bb] * (1.0 + std::min(lam / hmin, nmax));
        wsum += (double)nband[bb];
      }
      ev /= wsum;
      c->h_inst[k].refill = ev > 24.0 ? 4 : (ev > 6.0 ? 8 : 16);
    }
  }
  c->h_nwall = nwall;
  {
    // Power entering through one face of each wall per unit wall temperature: the sum
    // over bands of the particles' weights (N_w particles of C_b v_b A / (4 N_w) each).
    std::vector<double> wu((size_t)n * 6, 0.0);
    for (int k = 0; k < n; ++k)
      for (int w = 0; w < 2 * dim; ++w)
        for (int bb = 0; bb < nb; ++bb) wu[(size_t)k * 6 + w] += wcoef[((size_t)k * nb + bb) * 6 + w] * (double)nwall[bb];
    iugkp_status s2 = upload(c, &c->d_wall_unit, wu);
    if (s2 != IUGKP_OK) return bail(s2);
  }
  c->total_particles = total_particles;
  c->h_wallT = wallTv;
  broadcast_wall_T(c);

  iugkp_status s;
#define UP(ptr, vec)                                 \
  if ((s = upload(c, &(ptr), (vec))) != IUGKP_OK) return bail(s);
  {
    std::vector<int> perm = emitter_orders(c, r32);
    UP(c->d_perm, perm);
  }
  UP(c->d_inst, c->h_inst);
  UP(c->d_groups_all, c->h_groups_all);
  UP(c->d_coef, coef);
  UP(c->d_ratio64, r64);
  UP(c->d_ratio32, r32);
  {
    std::vector<float> rnb = neighbour_max_ratio(c, r32);
    UP(c->d_ratio_nb32, rnb);
  }
  {
    // bands whose every cell has tau = tau_maj: every candidate is real (the uniform, below
    // 1, always passes the test against a ratio of exactly 1)
    std::vector<int> all_real((size_t)n * nb, 1);
    for (int k = 0; k < n; ++k)
      for (int bb = 0; bb < nb; ++bb) {
        const InstDesc& in = c->h_inst[k];
        for (long long i = 0; i < in.ncells; ++i)
          if (r32[(size_t)in.bc_off + (size_t)bb * in.ncells + i] != 1.0f) {
            all_real[(size_t)k * nb + bb] = 0;
            break;
          }
      }
    UP(c->d_all_real, all_real);
    c->all_real_all = std::all_of(all_real.begin(), all_real.end(), [](int x) { return x != 0; });
  }
  UP(c->d_taumaj, taumaj);
  {
    std::vector<float> vtm((size_t)n * nb);
    for (int k = 0; k < n; ++k)
      for (int bb = 0; bb < nb; ++bb) vtm[(size_t)k * nb + bb] = (float)(c->h_v[bb] * taumaj[(size_t)k * nb + bb]);
    UP(c->d_vtm32, vtm);
  }
  UP(c->d_v, c->h_v);
  UP(c->d_wcoef, wcoef);
  UP(c->d_wallT, wallTv);
  UP(c->d_wallTf, c->h_wallTf);
  UP(c->d_m, m);
  UP(c->d_Vm, Vm);
  UP(c->d_invVm, invVm);
  UP(c->d_VC, VC);
  UP(c->d_theta, c->h_theta);
  UP(c->d_theta_m, theta_m);
  UP(c->d_diag, diag);
  UP(c->d_cx, cx);
  UP(c->d_cy, cy);
  UP(c->d_cz, cz);
  if ((s = dalloc(c, &c->d_source, cell_off)) != IUGKP_OK) return bail(s);
  if (cudaMemcpy(c->d_source, Qv.data(), Qv.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    fail(c, IUGKP_ECUDA, "source upload");
    return bail(IUGKP_ECUDA);
  }
  if ((s = set_source(c, Qv, m)) != IUGKP_OK) return bail(s);
  {
    long long maxX = 0;
    for (const InstDesc& in : c->h_inst)
      maxX = std::max(maxX, c->dim == 2 ? in.nfaces : (long long)(in.n[0] + 1) * in.n[1] * in.n[2]);
    // static shared memory of the staged kernel (the cooperative tallies' parameter table and
    // list starts, 36.2 KB, and a few words) stays below 37 KB
    const long long budget = ((long long)c->smem_optin - 37 * 1024) / (long long)sizeof(unsigned);
    c->staged_cap = c->dim == 3 ? COOP3_BYTES / (int)sizeof(unsigned)
                                : (int)std::max<long long>(1, std::min(maxX, budget));
  }
  if ((s = rebuild_forward_groups(c)) != IUGKP_OK) return bail(s);
  {
    std::vector<long long> beg, end;
    std::vector<double> prefix;
    std::vector<unsigned> gmag;
    staged_tables(c, c->h_groups_all, beg, end, prefix, c->all_cost_total, gmag);
    UP(c->d_all_beg, beg);
    UP(c->d_all_end, end);
    UP(c->d_all_cost_prefix, prefix);
    UP(c->d_all_group_mag, gmag);
  }
  {
    std::vector<unsigned> mag((size_t)5 * n);
    for (int k = 0; k < n; ++k) {
      const InstDesc& in = c->h_inst[k];
      mag[k] = div_magic(in.n[0]);
      mag[n + k] = div_magic(in.n[1]);
      for (int a = 0; a < 3; ++a) mag[2 * n + 3 * k + a] = div_magic(in.n[(a + 1) % 3]);
    }
    UP(c->d_mag, mag);
  }
  if ((s = dalloc(c, &c->d_inst_next, n)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_wmax, n)) != IUGKP_OK) return bail(s);
#undef UP
  if (configure_staged(c) != cudaSuccess) {
    cudaGetLastError();
    fail(c, IUGKP_ECUDA, "staged sweep configuration");
    return bail(IUGKP_ECUDA);
  }
  if ((s = dalloc(c, &c->d_pcg, 5 * (size_t)cell_off)) != IUGKP_OK) return bail(s);
  if ((s = build_multigrid(c, diag, cx, cy, cz, kap, cvsum)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_work, cell_off)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_T2, cell_off)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_R, (size_t)nb * cell_off)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_W, (size_t)nb * cell_off)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_F, face_off)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_wemit, (size_t)nb * cell_off)) != IUGKP_OK) return bail(s);
  {
    // queue of the particles the FP32 walk leaves to the FP64 replay: about 1e-4 of them on
    // the workloads measured; room for 1/32 of every emitter's particles
    const long long cap = std::min<long long>(c->total_particles / 32 + 65536, 1ll << 31);
    c->defer_cap = (unsigned)cap;
    if ((s = dalloc(c, &c->d_defer, (size_t)cap)) != IUGKP_OK) return bail(s);
    if ((s = dalloc(c, &c->d_defer_n, 1)) != IUGKP_OK) return bail(s);
    if (cudaMemset(c->d_defer_n, 0, sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      fail(c, IUGKP_ECUDA, "clear of the replay queue");
      return bail(IUGKP_ECUDA);
    }
  }
  if (c->dim == 2) {
    if ((s = dalloc(c, &c->d_DY, cell_off)) != IUGKP_OK) return bail(s);
    if ((s = dalloc(c, &c->d_EY, (size_t)c->total_bfaces)) != IUGKP_OK) return bail(s);
    if ((s = dalloc(c, &c->d_GX, (size_t)GX_COPIES * c->total_bfaces)) != IUGKP_OK) return bail(s);
    if ((s = dalloc(c, &c->d_Fd, face_off)) != IUGKP_OK) return bail(s);
  }
  if ((s = dalloc(c, &c->d_wall, c->total_walls)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_red, 1024)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_counters, CNT_N)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_work_counter, 4)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_err, 1)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_pcg_iters, n)) != IUGKP_OK) return bail(s);
  if ((s = dalloc(c, &c->d_scalar, 16)) != IUGKP_OK) return bail(s);
  if (cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&c->h_pinned, sizeof(double) * (16 + (size_t)n)) != cudaSuccess) {
    cudaGetLastError();
    fail(c, IUGKP_ECUDA, "set-up of error word / pinned buffer");
    return bail(IUGKP_ECUDA);
  }
  if (c->opt.tally == IUGKP_TALLY_STAGED_K32) {
    iugkp_status ks = ensure_k32(c);
    if (ks != IUGKP_OK) return bail(ks);
  }
  *out = ctx;
  return IUGKP_OK;
}

iugkp_status iugkp_create(const iugkp_grid* g, const double* tau, const iugkp_bands* b, const double* wall_T,
                          const double* source, const iugkp_options* o, iugkp_ctx** out) {
  const double* taus[1] = {tau};
  const double* walls[1] = {wall_T};
  const double* srcs[1] = {source};
  return iugkp_create_batch(1, g, taus, b, walls, srcs, o, out);
}

void iugkp_destroy(iugkp_ctx* ctx) {
  if (!ctx) return;
  free_all(&ctx->c);
  delete ctx;
}

iugkp_status iugkp_get_layout(const iugkp_ctx* ctx, iugkp_layout* lay, long long* cell_off, long long* face_off) {
  if (!ctx) return IUGKP_EINVAL;
  const Ctx* c = &ctx->c;
  if (lay) {
    lay->n_inst = c->n_inst;
    lay->dim = c->dim;
    lay->nb = c->nb;
    lay->total_cells = c->total_cells;
    lay->total_faces = c->total_faces;
    lay->total_walls = c->total_walls;
    lay->total_particles = c->total_particles;
    lay->total_wall_faces = c->total_bfaces;
  }
  for (int k = 0; k <= c->n_inst; ++k) {
    if (cell_off) cell_off[k] = k < c->n_inst ? c->h_inst[k].cell_off : c->total_cells;
    if (face_off) face_off[k] = k < c->n_inst ? c->h_inst[k].face_off : c->total_faces;
  }
  return IUGKP_OK;
}

}  // extern "C"

namespace {

SweepArgs base_args(Ctx* c) {
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.inst = c->d_inst;
  a.nb = c->nb;
  a.srcshift = c->d_srcshift;
  a.coef = c->d_coef;
  a.ratio64 = c->d_ratio64;
  a.ratio32 = c->d_ratio32;
  a.ratio_nb32 = c->d_ratio_nb32;
  a.all_real = c->d_all_real;
  a.perm = c->d_perm;
  a.taumaj = c->d_taumaj;
  a.vtm32 = c->d_vtm32;
  a.v = c->d_v;
  a.wcoef = c->d_wcoef;
  a.wallT = c->d_wallT;
  a.wemit = c->d_wemit;
  a.wallTf = c->d_wallTf;
  a.seed = c->opt.seed;
  a.budget = c->opt.step_budget;
  a.err = c->d_err;
  a.work_counter = c->d_work_counter;
  a.dim = c->dim;
  a.invVm = c->d_invVm;
  return a;
}

// Reads and clears the device error word (synchronises the stream).
iugkp_status check_device(Ctx* c, cudaStream_t s) {
  int* h = reinterpret_cast<int*>(c->h_pinned + 15);
  CK(cudaMemcpyAsync(h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, s), "error readback");
  CK(cudaStreamSynchronize(s), "stream synchronise");
  int e = *h;
  if (e) {
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), s), "error reset");
    if (e & ERR_BUDGET) return fail(c, IUGKP_EBUDGET, "a particle exceeded the step budget and was dropped");
    if (e & ERR_PCG) return fail(c, IUGKP_ENOCONV, "PCG reached cg_maxit before cg_rtol");
    if (e & ERR_DEFER)
      return fail(c, IUGKP_EDEVICE, "more particles than the replay queue holds needed the FP64 walk (queue overflow)");
    return fail(c, IUGKP_EDEVICE, "device-side check failed (code " + std::to_string(e) + ")");
  }
  return IUGKP_OK;
}

bool staged_path(const Ctx* c) {
  return c->opt.tally != IUGKP_TALLY_FP64 && c->opt.precision == IUGKP_TRACK_FP32 && c->fwd_particles < (1ll << 31);
}

// Buffers of the compensated FP32 tallies; allocated outside any stream capture.
iugkp_status ensure_k32(Ctx* c) {
  if (c->d_R32) return IUGKP_OK;
  const size_t bc = (size_t)c->nb * c->total_cells;
  iugkp_status st;
  if ((st = dalloc(c, &c->d_R32, bc)) != IUGKP_OK) return st;
  if ((st = dalloc(c, &c->d_W32, bc)) != IUGKP_OK) return st;
  return dalloc(c, &c->d_F32, (size_t)c->total_faces);
}

iugkp_status sweep_async(Ctx* c, const double* T, unsigned epoch, double* R, double* W, double* F, double* wall,
                         unsigned long long* counters, cudaStream_t s) {
  const size_t bc = (size_t)c->nb * c->total_cells;
  const bool staged = staged_path(c);
  const bool k32 = staged && c->opt.tally == IUGKP_TALLY_STAGED_K32;
  if (k32 && !c->d_R32) return fail(c, IUGKP_EINVAL, "compensated tally buffers missing");
  if (!k32) {  // the compensated mode writes R and W whole after the sweep
    CK(cudaMemsetAsync(R, 0, bc * sizeof(double), s), "clear R");
    if (W) CK(cudaMemsetAsync(W, 0, bc * sizeof(double), s), "clear W");
  }
  if (F) CK(cudaMemsetAsync(F, 0, c->total_faces * sizeof(double), s), "clear F");
  if (wall) CK(cudaMemsetAsync(wall, 0, c->total_walls * sizeof(double), s), "clear wall");
  unsigned long long* cnt = counters ? counters : c->d_counters;
  CK(cudaMemsetAsync(cnt, 0, CNT_N * sizeof(unsigned long long), s), "clear counters");
  CK(cudaMemsetAsync(c->d_work_counter, 0, sizeof(unsigned long long), s), "clear work counter");
  if (staged && wall && !F) {  // the staged sweep derives wall tallies from the face tallies
    F = c->d_F;
    CK(cudaMemsetAsync(F, 0, c->total_faces * sizeof(double), s), "clear F");
  }
  SweepArgs a = base_args(c);
  a.groups = c->d_groups_fwd;
  a.n_groups = (int)c->h_groups_fwd.size();
  a.total_particles = c->fwd_particles;
  a.T = T;
  a.R = R;
  a.W = W;
  a.F = F;
  a.wall = wall;
  a.counters = cnt;
  a.epoch = epoch;
  if (staged)
    CK(launch_sweep_staged(c, a, s), "staged sweep launch");
  else
    CK(launch_sweep(c, a, s), "sweep launch");
  return IUGKP_OK;
}

double dT_ref_of(const Ctx* c) {
  double lo = INFINITY, hi = -INFINITY, amax = 0.0;
  for (double t : c->h_wallTf) {
    lo = std::min(lo, t);
    hi = std::max(hi, t);
    amax = std::max(amax, std::fabs(t));
  }
  if (hi - lo > 0.0) return hi - lo;
  return amax;
}

// Residual between two iterates (synchronises): ||T1 - T0|| / max(||T1||, ref sqrt(N)).
iugkp_status residual(Ctx* c, const double* T0, const double* T1, double ref, cudaStream_t s, double* res) {
  CK(launch_residual(c, T0, T1, ref, c->d_scalar, s), "residual");
  CK(cudaMemcpyAsync(c->h_pinned, c->d_scalar, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "residual readback");
  CK(cudaStreamSynchronize(s), "residual sync");
  const double num = std::sqrt(c->h_pinned[0]);
  const double den = std::max(std::sqrt(c->h_pinned[1]), ref * std::sqrt((double)c->total_cells));
  *res = den > 0.0 ? num / den : (num > 0.0 ? INFINITY : 0.0);
  return IUGKP_OK;
}

iugkp_status pcg_status(Ctx* c, cudaStream_t s, int* iters) {
  int* h = reinterpret_cast<int*>(c->h_pinned + 16);
  CK(cudaMemcpyAsync(h, c->d_pcg_iters, c->n_inst * sizeof(int), cudaMemcpyDeviceToHost, s), "pcg readback");
  CK(cudaStreamSynchronize(s), "pcg sync");
  int worst = 0;
  bool fail_ = false;
  for (int k = 0; k < c->n_inst; ++k) {
    if (h[k] < 0) fail_ = true;
    worst = std::max(worst, h[k] < 0 ? c->opt.cg_maxit : h[k]);
  }
  if (iters) *iters = worst;
  if (fail_) return fail(c, IUGKP_ENOCONV, "PCG reached cg_maxit before cg_rtol");
  return IUGKP_OK;
}

// New relaxation times: every tau-dependent part of the context (band split of the particles,
// emitter groups, weights, majorants and acceptance ratios, m, the diffusion operator and its
// multigrid hierarchy, the Newton damping, the source shift Q/m) is rebuilt by creating the
// context afresh from its grids, bands, options, wall temperatures (per face) and source, and
// the fresh state replaces the old one (whose buffers are freed).
iugkp_status set_tau(iugkp_ctx* ctx, const std::vector<double>& tau) {
  Ctx* c = &ctx->c;
  for (double x : tau)
    if (!(x > 0.0)) return fail(c, IUGKP_EINVAL, "tau must be finite and > 0");
  std::vector<double> Q((size_t)c->total_cells);
  CK(cudaMemcpy(Q.data(), c->d_source, Q.size() * sizeof(double), cudaMemcpyDeviceToHost), "source readback");
  const int n = c->n_inst;
  std::vector<const double*> taus(n), walls(n), srcs(n);
  for (int k = 0; k < n; ++k) {
    const InstDesc& in = c->h_inst[k];
    taus[k] = tau.data() + in.bc_off;
    walls[k] = c->h_wallT.data() + in.wall_off;
    srcs[k] = Q.data() + in.cell_off;
  }
  const iugkp_bands bands{c->nb, c->h_C.data(), c->h_v.data()};
  iugkp_ctx* fresh = nullptr;
  const iugkp_status st =
      iugkp_create_batch(n, c->h_grids.data(), taus.data(), &bands, walls.data(), srcs.data(), &c->opt, &fresh);
  if (st != IUGKP_OK) return fail(c, st, std::string("tau: rebuilding the context: ") + iugkp_last_error(nullptr));
  Ctx* f = &fresh->c;
  if (f->h_wallTf != c->h_wallTf) {  // per-face wall temperatures set since creation
    f->h_wallTf = c->h_wallTf;
    iugkp_status ws = IUGKP_OK;
    if (cudaMemcpy(f->d_wallTf, f->h_wallTf.data(), f->h_wallTf.size() * sizeof(double), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
      cudaGetLastError();
      ws = fail(c, IUGKP_ECUDA, "tau: wall face upload");
    } else {
      ws = rebuild_forward_groups(f);
      if (ws != IUGKP_OK) fail(c, ws, f->err);
    }
    if (ws != IUGKP_OK) {
      iugkp_destroy(fresh);
      return ws;
    }
  }
  std::swap(ctx->c, fresh->c);
  iugkp_destroy(fresh);  // frees the old state
  return IUGKP_OK;
}

}  // namespace

extern "C" {

iugkp_status iugkp_set_field(iugkp_ctx* ctx, int which, const double* data, int on_device, void* cuda_stream) {
  if (!ctx || !data) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  size_t count = which == IUGKP_FIELD_SOURCE ? (size_t)c->total_cells
                 : which == IUGKP_FIELD_WALL_T ? (size_t)c->total_walls
                 : which == IUGKP_FIELD_WALL_FACE_T ? (size_t)c->total_bfaces
                 : which == IUGKP_FIELD_TAU ? (size_t)c->nb * c->total_cells : 0;
  if (!count) return fail(c, IUGKP_EINVAL, "unknown field");
  std::vector<double> h(count);
  if (on_device) {
    CK(cudaMemcpyAsync(h.data(), data, count * sizeof(double), cudaMemcpyDeviceToHost, s), "field readback");
    CK(cudaStreamSynchronize(s), "field sync");
  } else {
    std::copy(data, data + count, h.begin());
  }
  for (double x : h)
    if (!std::isfinite(x)) return fail(c, IUGKP_EINVAL, "field values must be finite");
  CK(cudaStreamSynchronize(s), "field sync");
  if (which == IUGKP_FIELD_TAU) return set_tau(ctx, h);
  if (which == IUGKP_FIELD_SOURCE) {
    CK(cudaMemcpy(c->d_source, h.data(), count * sizeof(double), cudaMemcpyHostToDevice), "source upload");
    std::vector<double> m(count);
    CK(cudaMemcpy(m.data(), c->d_m, count * sizeof(double), cudaMemcpyDeviceToHost), "m readback");
    return set_source(c, h, m);
  }
  if (which == IUGKP_FIELD_WALL_T) {  // every face of a wall takes the wall's value
    c->h_wallT = h;
    CK(cudaMemcpy(c->d_wallT, h.data(), count * sizeof(double), cudaMemcpyHostToDevice), "wall upload");
    broadcast_wall_T(c);
  } else {
    c->h_wallTf = h;
  }
  CK(cudaMemcpy(c->d_wallTf, c->h_wallTf.data(), c->h_wallTf.size() * sizeof(double), cudaMemcpyHostToDevice),
     "wall face upload");
  return rebuild_forward_groups(c);
}

iugkp_status iugkp_sweep(iugkp_ctx* ctx, const double* T_in_dev, unsigned epoch, double* R_dev, double* W_dev,
                         double* F_dev, double* wall_dev, unsigned long long* counters_dev, void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!T_in_dev || !R_dev) return fail(c, IUGKP_EINVAL, "T_in_dev and R_dev are required");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  iugkp_status st = sweep_async(c, T_in_dev, epoch, R_dev, W_dev, F_dev, wall_dev, counters_dev, s);
  if (st != IUGKP_OK) return st;
  return check_device(c, s);
}

iugkp_status iugkp_macro(iugkp_ctx* ctx, const double* R_dev, const double* W_dev, double* T_half_dev,
                         double* T_E_dev, void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!R_dev || !T_half_dev) return fail(c, IUGKP_EINVAL, "R_dev and T_half_dev are required");
  CK(launch_macro(c, R_dev, W_dev, T_half_dev, T_E_dev, (cudaStream_t)cuda_stream), "macro");
  return IUGKP_OK;
}

iugkp_status iugkp_newton_step(iugkp_ctx* ctx, const double* T_n_dev, double* T_half_inout_dev, const double* R_dev,
                               void* cuda_stream, int* cg_iters_out) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!T_n_dev || !T_half_inout_dev || !R_dev) return fail(c, IUGKP_EINVAL, "NULL device pointer");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CK(launch_newton(c, T_n_dev, T_half_inout_dev, R_dev, s), "newton");
  return pcg_status(c, s, cg_iters_out);
}

iugkp_status iugkp_autotune(iugkp_ctx* ctx, const double* T_dev, unsigned epoch, int allow_k32, iugkp_tuning* out,
                            void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!T_dev) return fail(c, IUGKP_EINVAL, "T_dev is required");
  if (!staged_path(c)) return fail(c, IUGKP_EINVAL, "autotune applies to the staged FP32 sweep");
  if (allow_k32) {
    iugkp_status ks = ensure_k32(c);
    if (ks != IUGKP_OK) return ks;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  struct Events {  // destroyed on every return path
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
    }
  } ev;
  CK(cudaEventCreate(&ev.a), "event");
  CK(cudaEventCreate(&ev.b), "event");
  // best of two sweeps (the first also warms the caches)
  auto time_sweep = [&](double* ms) -> iugkp_status {
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaEventRecord(ev.a, s), "event record");
      iugkp_status st = sweep_async(c, T_dev, epoch, c->d_R, c->d_W, c->d_F, c->d_wall, c->d_counters, s);
      if (st != IUGKP_OK) return st;
      CK(cudaEventRecord(ev.b, s), "event record");
      CK(cudaEventSynchronize(ev.b), "event sync");
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, ev.a, ev.b), "elapsed");
      best = std::min(best, t);
    }
    *ms = best;
    return IUGKP_OK;
  };
  iugkp_status st;
  double base = 0.0;
  if ((st = time_sweep(&base)) != IUGKP_OK) return st;
  double best = base;
  // coordinate descent, one tunable at a time, each keeping the best value found so far
  const int refills[] = {0, 4, 8, 16, 24};
  const int grabs[] = {128, 256, 512};
  const int walks[] = {8, 16, 32};
  const int tallies[] = {IUGKP_TALLY_STAGED, IUGKP_TALLY_STAGED_K32};
  int* knobs[4] = {&c->opt.refill_lanes, &c->opt.warp_grab, &c->opt.walk_k, &c->opt.tally};
  const int* values[4] = {refills, grabs, walks, tallies};
  const int counts[4] = {5, 3, 3, 2};
  for (int kdx = 0; kdx < (allow_k32 ? 4 : 3); ++kdx) {
    int keep = *knobs[kdx];
    for (int j = 0; j < counts[kdx]; ++j) {
      *knobs[kdx] = values[kdx][j];
      double t = 0.0;
      if ((st = time_sweep(&t)) != IUGKP_OK) {
        *knobs[kdx] = keep;
        return st;
      }
      if (t < best) {
        best = t;
        keep = values[kdx][j];
      }
    }
    *knobs[kdx] = keep;
  }
  if ((st = check_device(c, s)) != IUGKP_OK) return st;
  if (out) {
    out->refill_lanes = c->opt.refill_lanes;
    out->warp_grab = c->opt.warp_grab > 0 ? c->opt.warp_grab : 256;
    out->walk_k = c->opt.walk_k > 0 ? c->opt.walk_k : 16;
    out->tally = c->opt.tally;
    out->sweep_ms = best;
    out->baseline_ms = base;
  }
  return IUGKP_OK;
}

iugkp_status iugkp_residual(iugkp_ctx* ctx, const double* T0_dev, const double* T1_dev, double* out_dev,
                            void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!T0_dev || !T1_dev || !out_dev) return fail(c, IUGKP_EINVAL, "NULL device pointer");
  CK(launch_residual(c, T0_dev, T1_dev, 0.0, out_dev, (cudaStream_t)cuda_stream), "residual");
  return IUGKP_OK;
}

iugkp_status iugkp_replayed(iugkp_ctx* ctx, long long* n_out, void* cuda_stream) {
  if (!ctx || !n_out) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned* h = reinterpret_cast<unsigned*>(c->h_pinned + 14);
  CK(cudaMemcpyAsync(h, c->d_defer_n, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "replay count readback");
  CK(cudaStreamSynchronize(s), "stream synchronise");
  *n_out = (long long)*h;
  return IUGKP_OK;
}

iugkp_status iugkp_measure_atomics(double* ops_per_s) {
  Ctx* c = nullptr;
  if (!ops_per_s) return fail(c, IUGKP_EINVAL, "NULL output");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev), "device");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  CK(measure_atomic_rate(sms, ops_per_s), "atomic rate");
  return IUGKP_OK;
}

iugkp_status iugkp_check_fp32_walk(double* out6) {
  Ctx* c = nullptr;
  if (!out6) return fail(c, IUGKP_EINVAL, "NULL output");
  unsigned long long* d = nullptr;
  CK(cudaMalloc((void**)&d, 5 * sizeof(unsigned long long)), "check buffer");
  unsigned long long h[5];
  cudaError_t e = launch_walk_bounds(d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(c, e, "FP32 walk bound check");
  for (int k = 0; k < 5; ++k) {
    double x;
    std::memcpy(&x, &h[k], sizeof(x));
    out6[k] = x;
  }
  out6[5] = walk_bound_fraction(out6);
  return IUGKP_OK;
}

}  // extern "C"

namespace {

// One IUGKP iteration cur -> nxt without host round trips: sweep, macro update, Newton
// correction (CG status checked on the device), residual sums into res_dev[0..1].
iugkp_status iteration_async(Ctx* c, const double* cur, double* nxt, unsigned epoch, double* res_dev,
                             cudaStream_t s) {
  iugkp_status st = sweep_async(c, cur, epoch, c->d_R, c->d_W, c->d_F, c->d_wall, c->d_counters, s);
  if (st != IUGKP_OK) return st;
  CK(launch_macro(c, c->d_R, nullptr, nxt, nullptr, s), "macro");
  if (c->opt.newton) {
    CK(launch_newton(c, cur, nxt, c->d_R, s), "newton");
    CK(launch_pcg_check(c, s), "pcg check");
  }
  CK(launch_residual(c, cur, nxt, 0.0, res_dev, s), "residual");
  return IUGKP_OK;
}

double residual_from_sums(const Ctx* c, const double* sums, double ref) {
  const double num = std::sqrt(sums[0]);
  const double den = std::max(std::sqrt(sums[1]), ref * std::sqrt((double)c->total_cells));
  return den > 0.0 ? num / den : (num > 0.0 ? INFINITY : 0.0);
}

// Frozen draws: captures two iterations (T -> T2 -> T) once and replays the graph; one
// readback of the two residuals per replay.
iugkp_status solve_graph(Ctx* c, double* T, double tol, int max_iter, cudaStream_t user, int* iters_out,
                         double* res_out) {
  if (!c->graph_stream) {
    CK(cudaStreamCreateWithFlags(&c->graph_stream, cudaStreamNonBlocking), "graph stream");
    CK(cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming), "event");
    CK(cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming), "event");
    iugkp_status st = dalloc(c, &c->d_res_block, 4);
    if (st != IUGKP_OK) return st;
  }
  cudaStream_t gs = c->graph_stream;
  CK(cudaEventRecord(c->ev_in, user), "event record");
  CK(cudaStreamWaitEvent(gs, c->ev_in, 0), "stream wait");
  const double ref = dT_ref_of(c);
  const unsigned epoch = c->opt.epoch0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal), "begin capture");
  iugkp_status st = iteration_async(c, T, c->d_T2, epoch, c->d_res_block, gs);
  if (st == IUGKP_OK) st = iteration_async(c, c->d_T2, T, epoch, c->d_res_block + 2, gs);
  cudaError_t ce = cudaStreamEndCapture(gs, &graph);
  if (st != IUGKP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) return cuda_fail(c, ce, "end capture");
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return cuda_fail(c, ce, "graph instantiate");
  int it = 0;
  double res = INFINITY;
  while (it < max_iter) {
    ce = cudaGraphLaunch(exec, gs);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(c->h_pinned, c->d_res_block, 4 * sizeof(double), cudaMemcpyDeviceToHost, gs);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(gs);
    if (ce != cudaSuccess) {
      cudaGraphExecDestroy(exec);
      return cuda_fail(c, ce, "graph replay");
    }
    it += 2;
    res = residual_from_sums(c, c->h_pinned + 2, ref);
    if (res <= tol) break;
  }
  cudaGraphExecDestroy(exec);
  CK(cudaEventRecord(c->ev_out, gs), "event record");
  CK(cudaStreamWaitEvent(user, c->ev_out, 0), "stream wait");
  if ((st = check_device(c, user)) != IUGKP_OK) return st;
  if (iters_out) *iters_out = it;
  if (res_out) *res_out = res;
  if (!(res <= tol)) return fail(c, IUGKP_ENOCONV, "max_iter reached before tol");
  return IUGKP_OK;
}

}  // namespace

extern "C" {

iugkp_status iugkp_solve_steady(iugkp_ctx* ctx, double* T_inout_dev, double tol, int max_iter, int* iters_out,
                                double* res_out, void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!T_inout_dev || max_iter < 1 || !(tol >= 0.0)) return fail(c, IUGKP_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (c->opt.use_graphs && c->opt.draws == IUGKP_DRAWS_FROZEN)
    return solve_graph(c, T_inout_dev, tol, max_iter, s, iters_out, res_out);
  const double ref = dT_ref_of(c);
  double* cur = T_inout_dev;
  double* nxt = c->d_T2;
  double res = INFINITY;
  int it = 0;
  iugkp_status st;
  while (it < max_iter) {
    const unsigned epoch = c->opt.draws == IUGKP_DRAWS_FROZEN ? c->opt.epoch0 : c->opt.epoch0 + (unsigned)it;
    if ((st = sweep_async(c, cur, epoch, c->d_R, c->d_W, c->d_F, c->d_wall, c->d_counters, s)) != IUGKP_OK) return st;
    CK(launch_macro(c, c->d_R, nullptr, nxt, nullptr, s), "macro");
    if (c->opt.newton) {
      CK(launch_newton(c, cur, nxt, c->d_R, s), "newton");
      if ((st = pcg_status(c, s, nullptr)) != IUGKP_OK) return st;
    }
    if ((st = residual(c, cur, nxt, ref, s, &res)) != IUGKP_OK) return st;
    std::swap(cur, nxt);
    ++it;
    if (res <= tol) break;
  }
  if (cur != T_inout_dev) CK(cudaMemcpyAsync(T_inout_dev, cur, c->total_cells * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy result");
  if ((st = check_device(c, s)) != IUGKP_OK) return st;
  if (iters_out) *iters_out = it;
  if (res_out) *res_out = res;
  if (!(res <= tol)) return fail(c, IUGKP_ENOCONV, "max_iter reached before tol");
  return IUGKP_OK;
}

// Boundary-face homes of the persistent population over all instances and bands.
static long long pers_face_homes(const Ctx* c) { return c->pers_homes - (long long)c->nb * c->total_cells; }

iugkp_status iugkp_persistent_reset(iugkp_ctx* ctx, void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::vector<long long> slot_off(c->n_inst + 1, 0), home_off(c->n_inst + 1, 0);
  for (int k = 0; k < c->n_inst; ++k) {
    const InstDesc& in = c->h_inst[k];
    long long nbf = 0;
    for (int w = 0; w < 2 * in.dim; ++w) nbf += (long long)in.n[((w >> 1) + 1) % 3] * in.n[((w >> 1) + 2) % 3];
    long long slots = 0;
    for (int b = 0; b < c->nb; ++b) slots += c->h_nband[(size_t)k * c->nb + b] * in.ncells + c->h_nwall[b] * nbf;
    slot_off[k + 1] = slot_off[k] + slots;
    home_off[k + 1] = home_off[k] + (long long)c->nb * (in.ncells + nbf);
  }
  if (slot_off[c->n_inst] >= (1ll << 31)) return fail(c, IUGKP_EINVAL, "persistent population above 2^31 slots");
  if (c->pers_n != slot_off[c->n_inst] || !c->d_px) {
    void* olds[] = {c->d_pslot_off, c->d_phome_off, c->d_pnband, c->d_pnwall, c->d_px, c->d_pband, c->d_phome,
                    c->d_pcount, c->d_pfcount, c->d_phome_w};
    for (void* p : olds)
      if (p) cudaFree(p);
    c->d_pslot_off = c->d_phome_off = c->d_pnband = c->d_pnwall = nullptr;
    c->d_px = nullptr;
    c->d_pband = c->d_phome = nullptr;
    c->d_pcount = c->d_pfcount = nullptr;
    c->d_phome_w = nullptr;
    c->pers_n = slot_off[c->n_inst];
    c->pers_homes = home_off[c->n_inst];
    iugkp_status st;
    if ((st = upload(c, &c->d_pslot_off, slot_off)) != IUGKP_OK) return st;
    if ((st = upload(c, &c->d_phome_off, home_off)) != IUGKP_OK) return st;
    if ((st = upload(c, &c->d_pnband, c->h_nband)) != IUGKP_OK) return st;
    if ((st = upload(c, &c->d_pnwall, c->h_nwall)) != IUGKP_OK) return st;
    if ((st = dalloc(c, &c->d_px, (size_t)7 * c->pers_n)) != IUGKP_OK) return st;
    if ((st = dalloc(c, &c->d_pband, (size_t)c->pers_n)) != IUGKP_OK) return st;
    if ((st = dalloc(c, &c->d_phome, (size_t)c->pers_n)) != IUGKP_OK) return st;
    if ((st = dalloc(c, &c->d_pcount, (size_t)2 * c->pers_homes)) != IUGKP_OK) return st;
    if ((st = dalloc(c, &c->d_pfcount, (size_t)2 * PERS_FACE_REPLICAS * pers_face_homes(c))) != IUGKP_OK) return st;
    if ((st = dalloc(c, &c->d_phome_w, (size_t)c->pers_homes)) != IUGKP_OK) return st;
  }
  c->pers_parity = 0;
  CK(cudaMemsetAsync(c->d_pfcount, 0, (size_t)2 * PERS_FACE_REPLICAS * pers_face_homes(c) * sizeof(unsigned), s),
     "clear face counts");
  CK(launch_persistent_init(c, s), "persistent init");
  return check_device(c, s);
}

iugkp_status iugkp_persistent_step(iugkp_ctx* ctx, const double* T_dev, unsigned iteration, double* R_dev,
                                   double* W_dev, double* wall_dev, unsigned long long* counters_dev,
                                   long long* slots_out, void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!T_dev || !R_dev) return fail(c, IUGKP_EINVAL, "T_dev and R_dev are required");
  if (!c->d_px) return fail(c, IUGKP_EINVAL, "call iugkp_persistent_reset first");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bc = (size_t)c->nb * c->total_cells;
  double* W = W_dev ? W_dev : c->d_W;
  double* wall = wall_dev ? wall_dev : c->d_wall;
  unsigned long long* cnt = counters_dev ? counters_dev : c->d_counters;
  CK(cudaMemsetAsync(R_dev, 0, bc * sizeof(double), s), "clear R");
  CK(cudaMemsetAsync(W, 0, bc * sizeof(double), s), "clear W");
  CK(cudaMemsetAsync(wall, 0, (size_t)c->total_walls * sizeof(double), s), "clear wall");
  CK(cudaMemsetAsync(cnt, 0, CNT_N * sizeof(unsigned long long), s), "clear counters");
  {
    const size_t fr = (size_t)PERS_FACE_REPLICAS * pers_face_homes(c);
    CK(cudaMemsetAsync(c->d_pfcount + (c->pers_parity ? 0 : fr), 0, fr * sizeof(unsigned), s), "clear face counts");
  }
  CK(cudaMemsetAsync(c->d_pcount + (c->pers_parity ? 0 : c->pers_homes), 0, (size_t)c->pers_homes * sizeof(unsigned), s),
     "clear counts");
  CK(launch_persistent_step(c, T_dev, iteration, R_dev, W, wall, cnt, s), "persistent step");
  c->pers_parity ^= 1;
  if (slots_out) *slots_out = c->pers_n;
  return IUGKP_OK;
}

iugkp_status iugkp_average(iugkp_ctx* ctx, double* T_inout_dev, int n_steps, unsigned epoch_first,
                           double* T_mean_dev, double* T_var_dev, double* F_mean_dev, void* cuda_stream) {
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!T_inout_dev || !T_mean_dev || n_steps < 1) return fail(c, IUGKP_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* m2 = T_var_dev;
  if (!m2) {
    if (!c->d_m2) {
      iugkp_status st = dalloc(c, &c->d_m2, (size_t)c->total_cells);
      if (st != IUGKP_OK) return st;
    }
    m2 = c->d_m2;
  }
  const size_t cb = (size_t)c->total_cells * sizeof(double);
  CK(cudaMemsetAsync(T_mean_dev, 0, cb, s), "clear mean");
  CK(cudaMemsetAsync(m2, 0, cb, s), "clear m2");
  if (F_mean_dev) CK(cudaMemsetAsync(F_mean_dev, 0, (size_t)c->total_faces * sizeof(double), s), "clear F mean");
  double* cur = T_inout_dev;
  double* nxt = c->d_T2;
  for (int k = 0; k < n_steps; ++k) {
    // the solve's update with fresh draws: epoch_first + k
    iugkp_status st = iteration_async(c, cur, nxt, epoch_first + (unsigned)k, c->d_scalar + 4, s);
    if (st != IUGKP_OK) return st;
    CK(launch_welford(c, nxt, T_mean_dev, m2, c->total_cells, k + 1, s), "welford");
    if (F_mean_dev) CK(launch_welford(c, c->d_F, F_mean_dev, nullptr, c->total_faces, k + 1, s), "flux mean");
    std::swap(cur, nxt);
  }
  if (T_var_dev) CK(launch_scale(c, T_var_dev, c->total_cells, n_steps > 1 ? 1.0 / (n_steps - 1) : 0.0, s), "variance");
  if (cur != T_inout_dev) CK(cudaMemcpyAsync(T_inout_dev, cur, cb, cudaMemcpyDeviceToDevice, s), "copy result");
  return check_device(c, s);
}

}  // extern "C"

namespace {

// The adjoint re-trace: the staged kernel for the FP32 walk with staged tallies (the
// fast path), else the plain one-thread-per-particle kernel.
cudaError_t adjoint_sweep(Ctx* c, const SweepArgs& a, cudaStream_t s) {
  if (c->opt.tally != IUGKP_TALLY_FP64 && c->opt.precision == IUGKP_TRACK_FP32 && c->total_particles < (1ll << 31))
    return launch_adjoint_staged(c, a, s);
  return launch_adjoint(c, a, s);
}

}  // namespace

extern "C" {

iugkp_status iugkp_adjoint(iugkp_ctx* ctx, const double* T_star_dev, const double* g_dev, double tol, int max_iter,
                           double* grad_source_dev, double* grad_wall_dev, double* lambda_dev, void* cuda_stream) {
  (void)T_star_dev;
  if (!ctx) return IUGKP_EINVAL;
  Ctx* c = &ctx->c;
  if (!g_dev || !grad_source_dev || !grad_wall_dev || max_iter < 1) return fail(c, IUGKP_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  iugkp_status st;
  if (!c->d_adj) {
    if ((st = dalloc(c, &c->d_adj, 4 * (size_t)c->total_cells)) != IUGKP_OK) return st;
  }
  const size_t nc = (size_t)c->total_cells;
  double* at = c->d_adj;
  double* half = at + nc;
  double* lam = lambda_dev ? lambda_dev : half + nc;
  double* nxt = half + 2 * nc;
  CK(cudaMemsetAsync(lam, 0, nc * sizeof(double), s), "clear lambda");
  // |g| max as the residual floor.
  std::vector<double> hg(nc);
  CK(cudaMemcpyAsync(hg.data(), g_dev, nc * sizeof(double), cudaMemcpyDeviceToHost, s), "g readback");
  CK(cudaStreamSynchronize(s), "g sync");
  double gmax = 0.0;
  for (double x : hg) gmax = std::max(gmax, std::fabs(x));
  SweepArgs a = base_args(c);
  a.groups = c->d_groups_all;
  a.n_groups = (int)c->h_groups_all.size();
  a.total_particles = c->total_particles;
  a.epoch = c->opt.epoch0;
  a.adj_out = at;
  a.adj_wall = grad_wall_dev;
  a.counters = c->d_counters;  // event counts of the re-trace (diagnostic)
  double res = INFINITY;
  int it = 0;
  while (it < max_iter) {
    a.lambda = lam;
    CK(cudaMemsetAsync(at, 0, nc * sizeof(double), s), "clear");
    CK(cudaMemsetAsync(grad_wall_dev, 0, c->total_walls * sizeof(double), s), "clear");
    CK(adjoint_sweep(c, a, s), "adjoint sweep");
    CK(launch_axpy_grad(c, at, g_dev, half, s), "adjoint axpy");
    if (c->opt.newton) {
      CK(launch_adjoint_correction(c, lam, half, nxt, s), "adjoint correction");
      if ((st = pcg_status(c, s, nullptr)) != IUGKP_OK) return st;
    } else {
      CK(cudaMemcpyAsync(nxt, half, nc * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    }
    if ((st = residual(c, lam, nxt, gmax, s, &res)) != IUGKP_OK) return st;
    CK(cudaMemcpyAsync(lam, nxt, nc * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy lambda");
    ++it;
    if (res <= tol) break;
  }
  // Gradients at the converged lambda: dJ/dQ = (A^T lambda) / m, dJ/dT_w = B_w^T lambda.
  a.lambda = lam;
  CK(cudaMemsetAsync(at, 0, nc * sizeof(double), s), "clear");
  CK(cudaMemsetAsync(grad_wall_dev, 0, c->total_walls * sizeof(double), s), "clear");
  CK(adjoint_sweep(c, a, s), "adjoint sweep");
  CK(launch_grad_source(c, at, grad_source_dev, s), "grad source");
  if ((st = check_device(c, s)) != IUGKP_OK) return st;
  if (!(res <= tol)) return fail(c, IUGKP_ENOCONV, "adjoint: max_iter reached before tol");
  return IUGKP_OK;
}

}  // extern "C"
