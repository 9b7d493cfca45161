// Host set-up of the aggregation-multigrid hierarchy used to precondition the Newton
// correction's CG (see mgpcg.cu): 2x coarsening per axis, Galerkin coarse operators
// P^T A P for piecewise-constant P, dense inverse of the coarsest level.
#include <cuda_runtime.h>

#include <algorithm>
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

// Number of eigenvalues below x of the symmetric tridiagonal matrix (d, e): the negative
// terms of its Sturm sequence (LDL^T pivots of T - x I).
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  const int n = (int)d.size();
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < n; ++i) {
    const double off = i > 0 ? e[i - 1] * e[i - 1] / q : 0.0;
    q = (d[i] - x) - off;
    if (q == 0.0) q = -1e-300;  // treat an exact zero pivot as a tiny negative one
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Solves (T - x I) v = r in place (r -> v) by Gaussian elimination with partial pivoting on
// the tridiagonal band (the interchanges fill a second superdiagonal). A zero pivot is
// replaced by a tiny one: x is an eigenvalue here, and the near-singular solve is what
// inverse iteration wants.
void shifted_solve(const std::vector<double>& d, const std::vector<double>& e, double x, double tiny,
                   std::vector<double>& r) {
  const int n = (int)d.size();
  std::vector<double> lo(n, 0.0), dg(n), up(n, 0.0), up2(n, 0.0), mult(n, 0.0);
  std::vector<char> swp(n, 0);
  for (int i = 0; i < n; ++i) {
    dg[i] = d[i] - x;
    if (i + 1 < n) {
      lo[i] = e[i];
      up[i] = e[i];
    }
  }
  for (int i = 0; i + 1 < n; ++i) {
    if (std::fabs(lo[i]) > std::fabs(dg[i])) {  // swap rows i and i + 1
      swp[i] = 1;
      std::swap(dg[i], lo[i]);
      std::swap(up[i], dg[i + 1]);
      if (i + 2 < n) std::swap(up2[i], up[i + 1]);
    }
    if (dg[i] == 0.0) dg[i] = tiny;
    const double m = lo[i] / dg[i];
    mult[i] = m;
    dg[i + 1] -= m * up[i];
    if (i + 2 < n) up[i + 1] -= m * up2[i];
  }
  if (dg[n - 1] == 0.0) dg[n - 1] = tiny;
  for (int i = 0; i + 1 < n; ++i) {
    if (swp[i]) std::swap(r[i], r[i + 1]);
    r[i + 1] -= mult[i] * r[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = r[i];
    if (i + 1 < n) v -= up[i] * r[i + 1];
    if (i + 2 < n) v -= up2[i] * r[i + 2];
    r[i] = v / dg[i];
  }
}

// Eigenvalues (ascending) and orthonormal eigenvectors of the symmetric tridiagonal matrix
// with diagonal d and off-diagonal e: each eigenvalue by bisection on Sturm counts inside the
// Gershgorin interval, its eigenvector by two steps of inverse iteration. Q is row-major with
// eigenvector k in column k.
void tridiag_eigen(const std::vector<double>& d, const std::vector<double>& e, std::vector<double>& lam,
                   std::vector<double>& Q) {
  const int n = (int)d.size();
  lam.assign(n, 0.0);
  Q.assign((size_t)n * n, 0.0);
  if (n == 1) {
    lam[0] = d[0];
    Q[0] = 1.0;
    return;
  }
  double glo = INFINITY, ghi = -INFINITY;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
    glo = std::min(glo, d[i] - r);
    ghi = std::max(ghi, d[i] + r);
  }
  const double scale = std::max(std::fabs(glo), std::fabs(ghi));
  for (int k = 0; k < n; ++k) {
    double lo = glo, hi = ghi;
    for (int it = 0; it < 200 && hi - lo > 4e-16 * scale; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (sturm_count(d, e, mid) > k) hi = mid;
      else lo = mid;
    }
    lam[k] = 0.5 * (lo + hi);
    std::vector<double> v(n);
    for (int i = 0; i < n; ++i) v[i] = 1.0 + 0.37 * std::sin(1.7 * i + 0.3 * k);
    for (int rep = 0; rep < 2; ++rep) {
      shifted_solve(d, e, lam[k], 1e-14 * scale, v);
      double nv = 0.0;
      for (double x : v) nv += x * x;
      nv = 1.0 / std::sqrt(nv);
      for (double& x : v) x *= nv;
    }
    for (int i = 0; i < n; ++i) Q[(size_t)i * n + k] = v[i];
  }
}

// The diffusion operator of a 1D or 2D instance with the same kappa in every cell is
// separable: A = Tx (x) I + I (x) Ty, where Tx holds the faces normal to x (kappa / hx^2
// between cells, the wall conductance over hx at each end) and Ty those normal to y (Ty = [0]
// in 1D). Its condition number is then moderate (no kappa contrast), so FP32 eigenvector
// matrices give a good approximate inverse. Returns false otherwise, or if the assembled
// operator does not split that way to 1e-12.
bool separable_parts(const InstDesc& in, const double* kap, double cvsum, const double* diag, const double* cx,
                     const double* cy, std::vector<double> part[2][2]) {
  if (in.dim > 2) return false;
  const double k0 = kap[0];
  for (long long i = 1; i < in.ncells; ++i)
    if (kap[i] != k0) return false;
  const int nn[2] = {in.n[0], in.dim == 2 ? in.n[1] : 1};
  for (int a = 0; a < 2; ++a) {
    std::vector<double>& dd = part[a][0];
    std::vector<double>& ee = part[a][1];
    dd.assign(nn[a], 0.0);
    ee.assign(nn[a] > 1 ? nn[a] - 1 : 0, 0.0);
    if (a >= in.dim) continue;  // 1D: Ty = [0]
    const double h = in.h[a], cin = k0 / (h * h);
    const double wall = 1.0 / (h / (2.0 * k0) + 2.0 / cvsum) / h;
    for (int i = 0; i < nn[a]; ++i) {
      dd[i] = (i > 0 ? cin : wall) + (i + 1 < nn[a] ? cin : wall);
      if (i + 1 < nn[a]) ee[i] = -cin;
    }
  }
  // the assembled operator must be exactly this sum (to rounding)
  for (long long c = 0; c < in.ncells; ++c) {
    const int ix = (int)(c % nn[0]), iy = (int)(c / nn[0]);
    const double want = part[0][0][ix] + part[1][0][iy];
    if (std::fabs(diag[c] - want) > 1e-12 * std::fabs(want)) return false;
    if (ix + 1 < nn[0] && std::fabs(cx[c] + part[0][1][ix]) > 1e-12 * std::fabs(part[0][1][ix])) return false;
    if (in.dim == 2 && iy + 1 < nn[1] && std::fabs(cy[c] + part[1][1][iy]) > 1e-12 * std::fabs(part[1][1][iy]))
      return false;
  }
  return true;
}

}  // namespace

iugkp_status build_multigrid(Ctx* c, const std::vector<double>& diag, const std::vector<double>& cx,
                             const std::vector<double>& cy, const std::vector<double>& cz,
                             const std::vector<double>& kap, double cvsum) {
  std::vector<InstMG> mgs;
  std::vector<float> ldiag, ldinv, lcx, lcy, lcz, cinv, fq, flam;
  long long level_off = 0;
  for (int k = 0; k < c->n_inst; ++k) {
    const InstDesc& in = c->h_inst[k];
    InstMG m;
    std::memset(&m, 0, sizeof(m));
    m.dim = in.dim;
    m.cell_off = in.cell_off;
    {
      // fast diagonalization for separable operators of moderate size
      std::vector<double> part[2][2];
      const int nx = in.n[0], ny = in.dim == 2 ? in.n[1] : 1;
      if (nx <= FD_MAX_N && ny <= FD_MAX_N &&
          separable_parts(in, kap.data() + in.cell_off, cvsum, diag.data() + in.cell_off, cx.data() + in.cell_off,
                          cy.data() + in.cell_off, part)) {
        // 2: every operand in shared memory (small axes), 1: tiles through L2
        m.direct = (nx <= fd_small_max_n() && ny <= fd_small_max_n()) ? 2 : 1;
        m.fnx = nx;
        m.fny = ny;
        std::vector<double> lam, Q;
        tridiag_eigen(part[0][0], part[0][1], lam, Q);
        m.qx_off = (long long)fq.size();
        m.lx_off = (long long)flam.size();
        for (double x : Q) fq.push_back((float)x);
        for (double x : lam) flam.push_back((float)x);
        tridiag_eigen(part[1][0], part[1][1], lam, Q);
        m.qy_off = (long long)fq.size();
        m.ly_off = (long long)flam.size();
        for (double x : Q) fq.push_back((float)x);
        for (double x : lam) flam.push_back((float)x);
      }
    }
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
  if ((s = up(&c->d_fd_q, fq)) != IUGKP_OK) return s;
  if ((s = up(&c->d_fd_lam, flam)) != IUGKP_OK) return s;
  std::vector<float> zeros((size_t)level_off, 0.0f);
  if ((s = up(&c->d_mg_b, zeros)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_x, zeros)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_t, zeros)) != IUGKP_OK) return s;
  if ((s = up(&c->d_mg_r, zeros)) != IUGKP_OK) return s;
  size_t smem = mg_solo_smem_bytes(mgs);
  for (const InstMG& m : mgs)
    if (m.direct == 2) smem = std::max(smem, fd_small_smem_bytes());
  const cudaError_t e = configure_mgpcg(c, smem);
  if (e != cudaSuccess) return fail(c, IUGKP_ECUDA, std::string("multigrid kernel set-up: ") + cudaGetErrorString(e));
  return IUGKP_OK;
}

}  // namespace iugkp
