// Host set-up of the aggregation-multigrid hierarchy used to precondition the Newton
// correction's CG (see mgpcg.cu): 2x coarsening per axis, Galerkin coarse operators
// P^T A P for piecewise-constant P, dense inverse of the coarsest level.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "mg.h"

namespace iugkp {

namespace {

struct Level {
  int n[3];
  long long nc;
  std::vector<double> diag, c[3];
};

// Gauss-Jordan inverse with partial pivoting (the coarsest matrix is SPD and tiny).
bool invert(std::vector<double>& a, int n, std::vector<double>& inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + col]) > std::fabs(a[(size_t)piv * n + col])) piv = r;
    if (!(std::fabs(a[(size_t)piv * n + col]) > 0.0)) return false;
    if (piv != col)
      for (int k = 0; k < n; ++k) {
        std::swap(a[(size_t)piv * n + k], a[(size_t)col * n + k]);
        std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
      }
    const double d = a[(size_t)col * n + col];
    for (int k = 0; k < n; ++k) {
      a[(size_t)col * n + k] /= d;
      inv[(size_t)col * n + k] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = a[(size_t)r * n + col];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        a[(size_t)r * n + k] -= f * a[(size_t)col * n + k];
        inv[(size_t)r * n + k] -= f * inv[(size_t)col * n + k];
      }
    }
  }
  return true;
}

}  // namespace

iugkp_status build_multigrid(Ctx* c, const std::vector<double>& diag, const std::vector<double>& cx,
                             const std::vector<double>& cy, const std::vector<double>& cz) {
  std::vector<InstMG> mgs;
  std::vector<float> ldiag, ldinv, lcx, lcy, lcz, cinv;
  long long level_off = 0;
  for (int k = 0; k < c->n_inst; ++k) {
    const InstDesc& in = c->h_inst[k];
    InstMG m;
    std::memset(&m, 0, sizeof(m));
    m.dim = in.dim;
    m.cell_off = in.cell_off;
    std::vector<Level> lv(1);
    for (int a = 0; a < 3; ++a) lv[0].n[a] = in.n[a];
    lv[0].nc = in.ncells;
    lv[0].diag.assign(diag.begin() + in.cell_off, diag.begin() + in.cell_off + in.ncells);
    const std::vector<double>* src[3] = {&cx, &cy, &cz};
    for (int a = 0; a < 3; ++a) lv[0].c[a].assign(src[a]->begin() + in.cell_off, src[a]->begin() + in.cell_off + in.ncells);
    while (lv.back().nc > MG_COARSE_MAX && (int)lv.size() < MG_MAXL) {
      const Level& f = lv.back();
      Level g;
      for (int a = 0; a < 3; ++a) g.n[a] = (f.n[a] + 1) / 2;
      g.nc = (long long)g.n[0] * g.n[1] * g.n[2];
      g.diag.assign(g.nc, 0.0);
      for (int a = 0; a < 3; ++a) g.c[a].assign(g.nc, 0.0);
      const long long fs[3] = {1, f.n[0], (long long)f.n[0] * f.n[1]};
      for (long long i = 0; i < f.nc; ++i) {
        const int ix = (int)(i % f.n[0]), iy = (int)((i / f.n[0]) % f.n[1]), iz = (int)(i / fs[2]);
        const long long I = (ix / 2) + (long long)g.n[0] * ((iy / 2) + (long long)g.n[1] * (iz / 2));
        g.diag[I] += f.diag[i];
        const int idx[3] = {ix, iy, iz};
        for (int a = 0; a < 3; ++a) {
          const double cc = f.c[a][i];
          if (cc == 0.0 || idx[a] + 1 >= f.n[a]) continue;
          int j3[3] = {ix, iy, iz};
          j3[a] += 1;
          const long long J = (j3[0] / 2) + (long long)g.n[0] * ((j3[1] / 2) + (long long)g.n[1] * (j3[2] / 2));
          if (J == I) g.diag[I] -= 2.0 * cc;
          else g.c[a][I] += cc;
        }
      }
      lv.push_back(std::move(g));
    }
    m.levels = (int)lv.size();
    for (int l = 0; l < m.levels; ++l) {
      for (int a = 0; a < 3; ++a) m.n[l][a] = lv[l].n[a];
      m.nc[l] = lv[l].nc;
      m.off[l] = level_off;
      level_off += lv[l].nc;
      for (long long i = 0; i < lv[l].nc; ++i) {
        ldiag.push_back((float)lv[l].diag[i]);
        ldinv.push_back((float)(1.0 / lv[l].diag[i]));
        lcx.push_back((float)lv[l].c[0][i]);
        lcy.push_back((float)lv[l].c[1][i]);
        lcz.push_back((float)lv[l].c[2][i]);
      }
    }
    // Dense coarsest matrix and its inverse.
    const Level& cl = lv.back();
    const int n = (int)cl.nc;
    std::vector<double> A((size_t)n * n, 0.0), inv;
    const long long cs[3] = {1, cl.n[0], (long long)cl.n[0] * cl.n[1]};
    for (long long i = 0; i < n; ++i) {
      A[(size_t)i * n + i] = cl.diag[i];
      for (int a = 0; a < 3; ++a) {
        const double cc = cl.c[a][i];
        if (cc == 0.0) continue;
        const long long j = i + cs[a];
        A[(size_t)i * n + j] -= cc;
        A[(size_t)j * n + i] -= cc;
      }
    }
    if (!invert(A, n, inv)) return fail(c, IUGKP_EINVAL, "multigrid: singular coarsest operator");
    m.cinv_off = (long long)cinv.size();
    for (double x : inv) cinv.push_back((float)x);
    mgs.push_back(m);
  }
  c->mg_level_cells = level_off;
  iugkp_status s;
  auto up = [&](auto** p, const auto& v) -> iugkp_status {
    using T = typename std::remove_reference<decltype(v)>::type::value_type;
    T* d = nullptr;
    if (cudaMalloc((void**)&d, (v.size() ? v.size() : 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, IUGKP_ENOMEM, "multigrid allocation");
    }
    *p = d;
    if (v.size() && cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(c, IUGKP_ECUDA, "multigrid upload");
    return IUGKP_OK;
  };
  if ((s = up(&c->d_mg, mgs)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_diag, ldiag)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_dinv, ldinv)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_cx, lcx)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_cy, lcy)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_cz, lcz)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_cinv, cinv)) != IUGKP_OK) return s;
  std::vector<float> zeros((size_t)level_off, 0.0f);
  if ((s = up(&c->d_mg_b, zeros)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_x, zeros)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_t, zeros)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_r, zeros)) != IUGKP_OK) return s;
  const cudaError_t e = configure_mgpcg(c, mg_solo_smem_bytes(mgs));
  if (e != cudaSuccess) return fail(c, IUGKP_ECUDA, std::string("multigrid kernel set-up: ") + cudaGetErrorString(e));
  return IUGKP_OK;
}

}  // namespace iugkp
