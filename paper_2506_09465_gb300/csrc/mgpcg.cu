// Inexact-Newton correction solver (arXiv 2506.09465 Sec. 3.3, Eq. "linear-q"): CG on the
// finite-volume diffusion operator, FP64 iterates and residual, preconditioned by one
// aggregation-multigrid V-cycle in FP32.
//
// One thread-block cluster per instance: the cluster's CTAs split each level's cells in
// contiguous ranges, exchange neighbour values through global memory (L2) between
// hardware cluster barriers, and reduce dot products through distributed shared memory
// in a fixed rank order (every CTA gets the same value, so all take the same branch).
// The V-cycle: damped Jacobi smoothing (nu pre, nu post), restriction by summing the
// children (P^T), Galerkin coarse operators P^T A P built on the host, prolongation by
// injection scaled by alpha (the usual over-correction of piecewise-constant
// aggregation), dense inverse on the coarsest level. It is symmetric, so CG stays CG.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "internal.h"
#include "mg.h"

namespace cg = cooperative_groups;

namespace iugkp {

struct MGArgs {
  const InstMG* mg;         // [n_inst]
  const double* diag;       // fine FP64 operator
  const double* cx;
  const double* cy;
  const double* cz;
  const float* ldiag;       // all levels, FP32
  const float* ldiag_inv;
  const float* lcx;
  const float* lcy;
  const float* lcz;
  const float* cinv;        // coarsest dense inverses
  float* lb;                // level right-hand sides
  float* lx;                // level iterates
  float* lt;                // level scratch (ping-pong)
  float* lr;                // level residuals
  const double* rhs;        // [cells]
  double* X;                // [cells] solution
  double* Rr;               // residual
  double* P;
  double* Q;
  double* Z;
  double rtol;
  int maxit;
  int* iters_out;           // [n_inst]
  float alpha, omega;
  int nu;
};

template <int NT, int CS>
struct ClusterRed {
  double* slot;  // shared [2][4]
  int buf;
  // Sums up to 4 values over the whole cluster in a fixed order.
  __device__ __forceinline__ void sum(cg::cluster_group& cl, double* v, int nv, double* sh) {
    // block reduce each value (fixed order)
    for (int k = 0; k < nv; ++k) {
      double x = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if ((threadIdx.x & 31) == 0) sh[k * 32 + (threadIdx.x >> 5)] = x;
    }
    __syncthreads();
    if (threadIdx.x < nv) {
      double s = 0.0;
      for (int w = 0; w < NT / 32; ++w) s += sh[threadIdx.x * 32 + w];
      slot[buf * 4 + threadIdx.x] = s;
    }
    cl.sync();
    for (int k = 0; k < nv; ++k) {
      double s = 0.0;
      for (int r = 0; r < CS; ++r) {
        const double* remote = cl.map_shared_rank(slot, r);
        s += remote[buf * 4 + k];
      }
      v[k] = s;
    }
    buf ^= 1;
    __syncthreads();  // sh reused by the next reduction
  }
};

__device__ __forceinline__ void level_coords(const int* n, long long i, int& x, int& y, int& z) {
  x = (int)(i % n[0]);
  long long t = i / n[0];
  y = (int)(t % n[1]);
  z = (int)(t / n[1]);
}

// y = A_l x on level l (FP32 stencil), for one cell.
__device__ __forceinline__ float level_apply(const float* dg, const float* cx, const float* cy, const float* cz,
                                             const float* x, const int* n, int dim, long long i, long long nc) {
  const long long sy = n[0], sz = (long long)n[0] * n[1];
  float q = dg[i] * __ldcg(&x[i]);
  if (i + 1 < nc) q -= cx[i] * __ldcg(&x[i + 1]);
  if (i >= 1) q -= cx[i - 1] * __ldcg(&x[i - 1]);
  if (dim >= 2) {
    if (i + sy < nc) q -= cy[i] * __ldcg(&x[i + sy]);
    if (i >= sy) q -= cy[i - sy] * __ldcg(&x[i - sy]);
  }
  if (dim >= 3) {
    if (i + sz < nc) q -= cz[i] * __ldcg(&x[i + sz]);
    if (i >= sz) q -= cz[i - sz] * __ldcg(&x[i - sz]);
  }
  return q;
}

// Damped Jacobi sweeps on level l from the iterate in x: ping-pong between x and t;
// returns the buffer that holds the result. Every sweep ends with a cluster barrier.
template <int NT, int CS>
__device__ __forceinline__ float* jacobi(const MGArgs& A, const InstMG& m, int l, cg::cluster_group& cl, int rank,
                                         int sweeps, float* x, float* t) {
  const long long nc = m.nc[l];
  const long long chunk = (nc + CS - 1) / CS, lo = rank * chunk, hi = min(nc, lo + chunk);
  const long long o = m.off[l];
  const float* dg = A.ldiag + o;
  const float* dinv = A.ldiag_inv + o;
  const float* cx = A.lcx + o;
  const float* cy = A.lcy + o;
  const float* cz = A.lcz + o;
  const float* b = A.lb + o;
  float* src = x;
  float* dst = t;
  for (int s = 0; s < sweeps; ++s) {
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      const float ax = level_apply(dg, cx, cy, cz, src, m.n[l], m.dim, i, nc);
      dst[i] = src[i] + A.omega * (b[i] - ax) * dinv[i];
    }
    cl.sync();
    float* tmp = src;
    src = dst;
    dst = tmp;
  }
  return src;
}

// One V-cycle: Z = M^{-1} Rr over this instance (all CTAs of the cluster take part).
template <int NT, int CS>
__device__ void vcycle(const MGArgs& A, const InstMG& m, cg::cluster_group& cl, int rank, long long cell_off) {
  const int L = m.levels;
  {
    const long long nc = m.nc[0];
    const long long chunk = (nc + CS - 1) / CS, lo = rank * chunk, hi = min(nc, lo + chunk);
    float* b = A.lb + m.off[0];
    for (long long i = lo + threadIdx.x; i < hi; i += NT) b[i] = (float)A.Rr[cell_off + i];
  }
  cl.sync();
  for (int l = 0; l < L - 1; ++l) {
    const long long nc = m.nc[l];
    const long long chunk = (nc + CS - 1) / CS, lo = rank * chunk, hi = min(nc, lo + chunk);
    const long long o = m.off[l];
    const float* dg = A.ldiag + o;
    const float* dinv = A.ldiag_inv + o;
    const float* cx = A.lcx + o;
    const float* cy = A.lcy + o;
    const float* cz = A.lcz + o;
    const float* b = A.lb + o;
    float* x = A.lx + o;
    float* t = A.lt + o;
    float* r = A.lr + o;
    // first sweep from x = 0: x = omega D^{-1} b (no neighbour reads)
    for (long long i = lo + threadIdx.x; i < hi; i += NT) x[i] = A.omega * b[i] * dinv[i];
    cl.sync();
    float* src = jacobi<NT, CS>(A, m, l, cl, rank, A.nu - 1, x, t);
    // residual of the smoothed iterate; the iterate is moved into x if it ended in t
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      const float ax = level_apply(dg, cx, cy, cz, src, m.n[l], m.dim, i, nc);
      r[i] = b[i] - ax;
      if (src != x) x[i] = src[i];
    }
    cl.sync();
    // restrict: b_{l+1}[I] = sum of the children's residuals (P^T r)
    const long long ncc = m.nc[l + 1];
    const long long cchunk = (ncc + CS - 1) / CS, clo = rank * cchunk, chi = min(ncc, clo + cchunk);
    float* bc = A.lb + m.off[l + 1];
    for (long long I = clo + threadIdx.x; I < chi; I += NT) {
      int X0, Y0, Z0;
      level_coords(m.n[l + 1], I, X0, Y0, Z0);
      float s = 0.f;
      for (int dz = 0; dz < (m.dim >= 3 ? 2 : 1); ++dz)
        for (int dy = 0; dy < (m.dim >= 2 ? 2 : 1); ++dy)
          for (int dx = 0; dx < 2; ++dx) {
            const int fx = 2 * X0 + dx, fy = 2 * Y0 + dy, fz = 2 * Z0 + dz;
            if (fx < m.n[l][0] && fy < m.n[l][1] && fz < m.n[l][2])
              s += __ldcg(&r[fx + (long long)m.n[l][0] * (fy + (long long)m.n[l][1] * fz)]);
          }
      bc[I] = s;
    }
    cl.sync();
  }
  {  // coarsest level: x = Ainv b (dense)
    const int l = L - 1;
    const long long nc = m.nc[l];
    const long long chunk = (nc + CS - 1) / CS, lo = rank * chunk, hi = min(nc, lo + chunk);
    const float* inv = A.cinv + m.cinv_off;
    const float* b = A.lb + m.off[l];
    float* x = A.lx + m.off[l];
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      float s = 0.f;
      for (long long j = 0; j < nc; ++j) s += inv[i * nc + j] * __ldcg(&b[j]);
      x[i] = s;
    }
    cl.sync();
  }
  for (int l = L - 2; l >= 0; --l) {
    const long long nc = m.nc[l];
    const long long chunk = (nc + CS - 1) / CS, lo = rank * chunk, hi = min(nc, lo + chunk);
    const long long o = m.off[l];
    float* x = A.lx + o;
    float* t = A.lt + o;
    const float* xc = A.lx + m.off[l + 1];
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      int X0, Y0, Z0;
      level_coords(m.n[l], i, X0, Y0, Z0);
      const long long I = (X0 >> 1) + (long long)m.n[l + 1][0] * ((Y0 >> 1) + (long long)m.n[l + 1][1] * (Z0 >> 1));
      x[i] += A.alpha * __ldcg(&xc[I]);
    }
    cl.sync();
    float* src = jacobi<NT, CS>(A, m, l, cl, rank, A.nu, x, t);
    if (src != x) {
      for (long long i = lo + threadIdx.x; i < hi; i += NT) x[i] = src[i];
      cl.sync();
    }
  }
  {
    const long long nc = m.nc[0];
    const long long chunk = (nc + CS - 1) / CS, lo = rank * chunk, hi = min(nc, lo + chunk);
    const float* x = A.lx + m.off[0];
    for (long long i = lo + threadIdx.x; i < hi; i += NT) A.Z[cell_off + i] = (double)x[i];
  }
}

template <int NT, int CS>
__global__ void __launch_bounds__(NT) mgpcg_kernel(MGArgs A) {
  __shared__ double sh[4 * 32];
  __shared__ double slot[8];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int k = blockIdx.x / CS;
  const InstMG& m = A.mg[k];
  const long long off = m.cell_off, n = m.nc[0];
  const long long chunk = (n + CS - 1) / CS, lo = rank * chunk, hi = min(n, lo + chunk);
  const long long sy = m.n[0][0], sz = (long long)m.n[0][0] * m.n[0][1];
  ClusterRed<NT, CS> red{slot, 0};
  double v[4];
  // x = 0, r = b
  v[0] = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NT) {
    const double bi = A.rhs[off + i];
    A.X[off + i] = 0.0;
    A.Rr[off + i] = bi;
    v[0] += bi * bi;
  }
  red.sum(cl, v, 1, sh);
  const double bb = v[0];
  if (bb == 0.0) {
    if (rank == 0 && threadIdx.x == 0) A.iters_out[k] = 0;
    return;
  }
  const double tol2 = A.rtol * A.rtol * bb;
  vcycle<NT, CS>(A, m, cl, rank, off);
  v[0] = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NT) {
    const double zi = A.Z[off + i];
    A.P[off + i] = zi;
    v[0] += A.Rr[off + i] * zi;
  }
  red.sum(cl, v, 1, sh);  // also orders the P writes before the first product
  double rz = v[0];
  int it = 0;
  bool done = false;
  while (it < A.maxit) {
    ++it;
    v[0] = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      const long long g = off + i;
      double q = A.diag[g] * __ldcg(&A.P[g]);
      if (i + 1 < n) q -= A.cx[g] * __ldcg(&A.P[g + 1]);
      if (i >= 1) q -= A.cx[g - 1] * __ldcg(&A.P[g - 1]);
      if (m.dim >= 2) {
        if (i + sy < n) q -= A.cy[g] * __ldcg(&A.P[g + sy]);
        if (i >= sy) q -= A.cy[g - sy] * __ldcg(&A.P[g - sy]);
      }
      if (m.dim >= 3) {
        if (i + sz < n) q -= A.cz[g] * __ldcg(&A.P[g + sz]);
        if (i >= sz) q -= A.cz[g - sz] * __ldcg(&A.P[g - sz]);
      }
      A.Q[g] = q;
      v[0] += __ldcg(&A.P[g]) * q;
    }
    red.sum(cl, v, 1, sh);
    const double alpha = rz / v[0];
    v[0] = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      const long long g = off + i;
      A.X[g] += alpha * A.P[g];
      const double ri = A.Rr[g] - alpha * A.Q[g];
      A.Rr[g] = ri;
      v[0] += ri * ri;
    }
    red.sum(cl, v, 1, sh);
    if (v[0] <= tol2) {
      done = true;
      break;
    }
    vcycle<NT, CS>(A, m, cl, rank, off);
    // Flexible (Polak-Ribiere) beta = z_new . (r_new - r_old) / (z_old . r_old), with
    // r_new - r_old = -alpha q: robust to the FP32 preconditioner's rounding.
    v[0] = 0.0;
    v[1] = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      const double zi = A.Z[off + i];
      v[0] += A.Rr[off + i] * zi;
      v[1] += A.Q[off + i] * zi;
    }
    red.sum(cl, v, 2, sh);
    const double beta = -alpha * v[1] / rz;
    rz = v[0];
    for (long long i = lo + threadIdx.x; i < hi; i += NT) A.P[off + i] = A.Z[off + i] + beta * A.P[off + i];
    cl.sync();
  }
  if (rank == 0 && threadIdx.x == 0) A.iters_out[k] = done ? it : -1;
}

constexpr int MG_NT = 512;
constexpr int MG_CS = 8;

cudaError_t launch_mgpcg(const Ctx* c, const double* rhs, cudaStream_t s) {
  MGArgs a;
  a.mg = c->d_mg;
  a.diag = c->d_diag;
  a.cx = c->d_cx;
  a.cy = c->d_cy;
  a.cz = c->d_cz;
  a.ldiag = c->d_mg_diag;
  a.ldiag_inv = c->d_mg_dinv;
  a.lcx = c->d_mg_cx;
  a.lcy = c->d_mg_cy;
  a.lcz = c->d_mg_cz;
  a.cinv = c->d_mg_cinv;
  a.lb = c->d_mg_b;
  a.lx = c->d_mg_x;
  a.lt = c->d_mg_t;
  a.lr = c->d_mg_r;
  a.rhs = rhs;
  a.X = c->d_pcg;
  a.Rr = c->d_pcg + c->total_cells;
  a.P = c->d_pcg + 2 * c->total_cells;
  a.Q = c->d_pcg + 3 * c->total_cells;
  a.Z = c->d_pcg + 4 * c->total_cells;
  a.rtol = c->opt.cg_rtol;
  a.maxit = c->opt.cg_maxit;
  a.iters_out = c->d_pcg_iters;
  a.alpha = 1.8f;
  a.omega = 0.8f;
  a.nu = 2;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c->n_inst * MG_CS, 1, 1);
  cfg.blockDim = dim3(MG_NT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = MG_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mgpcg_kernel<MG_NT, MG_CS>, a);
}

}  // namespace iugkp
