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

constexpr int MG32_PASSES_FD = 6;  // refinement passes of the fast diagonalization solve at most

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
  const float* fq;          // fast diagonalization: eigenvector matrices
  const float* flam;        // ... and eigenvalues
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

// y = A_l x on level l (FP32 stencil), for one cell; LD loads x (through L2 when other
// CTAs of the cluster wrote it, plainly when it is in this CTA's shared memory).
template <class LD>
__device__ __forceinline__ float level_apply(const float* dg, const float* cx, const float* cy, const float* cz,
                                             const float* x, const int* n, int dim, long long i, long long nc) {
  const long long sy = n[0], sz = (long long)n[0] * n[1];
  float q = dg[i] * LD::ld(&x[i]);
  if (i + 1 < nc) q -= cx[i] * LD::ld(&x[i + 1]);
  if (i >= 1) q -= cx[i - 1] * LD::ld(&x[i - 1]);
  if (dim >= 2) {
    if (i + sy < nc) q -= cy[i] * LD::ld(&x[i + sy]);
    if (i >= sy) q -= cy[i - sy] * LD::ld(&x[i - sy]);
  }
  if (dim >= 3) {
    if (i + sz < nc) q -= cz[i] * LD::ld(&x[i + sz]);
    if (i >= sz) q -= cz[i - sz] * LD::ld(&x[i - sz]);
  }
  return q;
}

// y = A_l u for u = x + alpha P xc (x prolonged from the coarser level's correction xc, P
// injection), for one cell at coordinates (X, Y, Z), without storing u. Neighbours across a
// boundary are skipped by coordinates (their coefficient is zero).
template <class LD>
__device__ __forceinline__ float level_apply_prolonged(const float* dg, const float* cx, const float* cy,
                                                       const float* cz, const float* x, const float* xc, float alpha,
                                                       const int* n, const int* nC, int dim, long long i, int X, int Y,
                                                       int Z) {
  auto u = [&](long long j, int x0, int y0, int z0) {
    const long long J = (x0 >> 1) + (long long)nC[0] * ((y0 >> 1) + (long long)nC[1] * (z0 >> 1));
    return fmaf(alpha, LD::ld(&xc[J]), LD::ld(&x[j]));
  };
  const long long sy = n[0], sz = (long long)n[0] * n[1];
  float q = dg[i] * u(i, X, Y, Z);
  if (X + 1 < n[0]) q -= cx[i] * u(i + 1, X + 1, Y, Z);
  if (X >= 1) q -= cx[i - 1] * u(i - 1, X - 1, Y, Z);
  if (dim >= 2) {
    if (Y + 1 < n[1]) q -= cy[i] * u(i + sy, X, Y + 1, Z);
    if (Y >= 1) q -= cy[i - sy] * u(i - sy, X, Y - 1, Z);
  }
  if (dim >= 3) {
    if (Z + 1 < n[2]) q -= cz[i] * u(i + sz, X, Y, Z + 1);
    if (Z >= 1) q -= cz[i - sz] * u(i - sz, X, Y, Z - 1);
  }
  return q;
}

// Who works on a level: the whole cluster (cells split in contiguous ranges over the CTAs,
// level vectors in global memory read through L2, cluster barriers) or CTA 0 alone (level
// vectors in its shared memory, block barriers). Levels of at most MG_SOLO_CELLS cells go
// to CTA 0: their work is small, and every phase of a level waits for the previous one, so
// the latency of a barrier and of an L2 round trip is what they would cost on the cluster.
struct ClusterTeam {
  int part;
  static constexpr bool solo = false;
  __device__ static float ld(const float* p) { return __ldcg(p); }
};
struct SoloTeam {
  static constexpr bool solo = true;
  __device__ static float ld(const float* p) { return *p; }
};

// The vectors of one level (b, x, t, r) and its operator coefficients.
struct LevelView {
  const float *dg, *dinv, *cx, *cy, *cz;
  float *b, *x, *t, *r;
};

__device__ __forceinline__ LevelView global_view(const MGArgs& A, const InstMG& m, int l) {
  const long long o = m.off[l];
  return {A.ldiag + o, A.ldiag_inv + o, A.lcx + o, A.lcy + o, A.lcz + o, A.lb + o, A.lx + o, A.lt + o, A.lr + o};
}

// Shared-memory layout of CTA 0's levels ls .. L-1: per level b, x, t, r of nc floats.
__device__ __forceinline__ LevelView solo_view(const MGArgs& A, const InstMG& m, int l, int ls, float* smem) {
  const long long o = m.off[l];
  long long so = 0;
  for (int j = ls; j < l; ++j) so += 4 * m.nc[j];
  float* base = smem + so;
  const long long nc = m.nc[l];
  return {A.ldiag + o, A.ldiag_inv + o, A.lcx + o, A.lcy + o, A.lcz + o, base, base + nc, base + 2 * nc, base + 3 * nc};
}

template <class TM, int NT, int CS>
__device__ __forceinline__ void team_range(const TM& tm, long long nc, long long& lo, long long& hi) {
  if constexpr (TM::solo) {
    lo = 0;
    hi = nc;
  } else {
    const long long chunk = (nc + CS - 1) / CS;
    lo = (long long)tm.part * chunk;
    hi = min(nc, lo + chunk);
  }
}

template <class TM>
__device__ __forceinline__ void team_sync(cg::cluster_group& cl) {
  if constexpr (TM::solo) __syncthreads();
  else cl.sync();
}

constexpr long long MG_SOLO_CELLS = 1024;

// Damped Jacobi sweeps on a level from the iterate in v.x: ping-pong between v.x and v.t;
// returns the buffer that holds the result. Every sweep ends with a team barrier.
template <class TM, int NT, int CS>
__device__ __forceinline__ float* jacobi(const MGArgs& A, const InstMG& m, int l, const LevelView& v, const TM& tm,
                                         cg::cluster_group& cl, int sweeps) {
  const long long nc = m.nc[l];
  long long lo, hi;
  team_range<TM, NT, CS>(tm, nc, lo, hi);
  float* src = v.x;
  float* dst = v.t;
  for (int sw = 0; sw < sweeps; ++sw) {
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      const float ax = level_apply<TM>(v.dg, v.cx, v.cy, v.cz, src, m.n[l], m.dim, i, nc);
      dst[i] = src[i] + A.omega * (v.b[i] - ax) * v.dinv[i];
    }
    team_sync<TM>(cl);
    float* tmp = src;
    src = dst;
    dst = tmp;
  }
  return src;
}

// Downward half of the V-cycle on level l: pre-smoothing from x = 0, residual, and its
// restriction into vc.b, the right-hand side of level l + 1 (sum over the children, P^T r).
template <class TM, int NT, int CS>
__device__ void vdown(const MGArgs& A, const InstMG& m, int l, const LevelView& v, const LevelView& vc, const TM& tm,
                      cg::cluster_group& cl) {
  const long long nc = m.nc[l];
  long long lo, hi;
  team_range<TM, NT, CS>(tm, nc, lo, hi);
  // first sweep from x = 0: x = omega D^{-1} b (no neighbour reads)
  for (long long i = lo + threadIdx.x; i < hi; i += NT) v.x[i] = A.omega * v.b[i] * v.dinv[i];
  team_sync<TM>(cl);
  float* src = jacobi<TM, NT, CS>(A, m, l, v, tm, cl, A.nu - 1);
  // restriction of the smoothed iterate's residual (sum over the children, P^T r), each
  // child's residual formed where it is summed; the iterate is moved into x if it ended in t
  const long long ncc = m.nc[l + 1];
  long long clo, chi;
  team_range<TM, NT, CS>(tm, ncc, clo, chi);
  for (long long I = clo + threadIdx.x; I < chi; I += NT) {
    int X0, Y0, Z0;
    level_coords(m.n[l + 1], I, X0, Y0, Z0);
    float sum = 0.f;
    for (int dz = 0; dz < (m.dim >= 3 ? 2 : 1); ++dz)
      for (int dy = 0; dy < (m.dim >= 2 ? 2 : 1); ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int fx = 2 * X0 + dx, fy = 2 * Y0 + dy, fz = 2 * Z0 + dz;
          if (fx < m.n[l][0] && fy < m.n[l][1] && fz < m.n[l][2]) {
            const long long c = fx + (long long)m.n[l][0] * (fy + (long long)m.n[l][1] * fz);
            sum += TM::ld(&v.b[c]) - level_apply<TM>(v.dg, v.cx, v.cy, v.cz, src, m.n[l], m.dim, c, nc);
          }
        }
    vc.b[I] = sum;
  }
  if (src != v.x)
    for (long long i = lo + threadIdx.x; i < hi; i += NT) v.x[i] = src[i];
  team_sync<TM>(cl);
}

// Coarsest level: x = Ainv b (dense).
template <class TM, int NT, int CS>
__device__ void vcoarsest(const MGArgs& A, const InstMG& m, const LevelView& v, const TM& tm, cg::cluster_group& cl) {
  const int l = m.levels - 1;
  const long long nc = m.nc[l];
  long long lo, hi;
  team_range<TM, NT, CS>(tm, nc, lo, hi);
  const float* inv = A.cinv + m.cinv_off;
  for (long long i = lo + threadIdx.x; i < hi; i += NT) {
    float sum = 0.f;
    for (long long j = 0; j < nc; ++j) sum += inv[i * nc + j] * TM::ld(&v.b[j]);
    v.x[i] = sum;
  }
  team_sync<TM>(cl);
}

// Upward half on level l: prolongation of the level l + 1 correction vc.x (injection
// scaled by alpha), then post-smoothing.
template <class TM, int NT, int CS>
__device__ void vup(const MGArgs& A, const InstMG& m, int l, const LevelView& v, const LevelView& vc, const TM& tm,
                    cg::cluster_group& cl) {
  const long long nc = m.nc[l];
  long long lo, hi;
  team_range<TM, NT, CS>(tm, nc, lo, hi);
  // first sweep from u = x + alpha P xc (the prolonged iterate, formed where it is read)
  // into t; the remaining sweeps ping-pong t and x
  for (long long i = lo + threadIdx.x; i < hi; i += NT) {
    int X0, Y0, Z0;
    level_coords(m.n[l], i, X0, Y0, Z0);
    const long long I = (X0 >> 1) + (long long)m.n[l + 1][0] * ((Y0 >> 1) + (long long)m.n[l + 1][1] * (Z0 >> 1));
    const float ui = fmaf(A.alpha, TM::ld(&vc.x[I]), v.x[i]);
    const float au = level_apply_prolonged<TM>(v.dg, v.cx, v.cy, v.cz, v.x, vc.x, A.alpha, m.n[l], m.n[l + 1], m.dim, i,
                                              X0, Y0, Z0);
    v.t[i] = ui + A.omega * (v.b[i] - au) * v.dinv[i];
  }
  team_sync<TM>(cl);
  const LevelView vt{v.dg, v.dinv, v.cx, v.cy, v.cz, v.b, v.t, v.x, v.r};  // iterate in t, scratch x
  float* src = jacobi<TM, NT, CS>(A, m, l, vt, tm, cl, A.nu - 1);
  if (src != v.x) {
    for (long long i = lo + threadIdx.x; i < hi; i += NT) v.x[i] = src[i];
    team_sync<TM>(cl);
  }
}

// First level of an instance that CTA 0 handles alone (the coarsest at the latest).
__host__ __device__ __forceinline__ int solo_level(const InstMG& m) {
  int ls = 0;
  while (ls < m.levels - 1 && m.nc[ls] > MG_SOLO_CELLS) ++ls;
  return ls;
}

// One V-cycle: Z = M^{-1} Rr over this instance. The cluster shares the levels above
// solo_level; CTA 0 copies that level's right-hand side into its shared memory, runs the
// rest of the cycle there, and writes the level's correction back for the cluster.
template <int NT, int CS>
__device__ void vcycle(const MGArgs& A, const InstMG& m, cg::cluster_group& cl, int rank, long long cell_off,
                       float* smem) {
  const ClusterTeam all{rank};
  const SoloTeam solo;
  const int L = m.levels;
  const int ls = solo_level(m);
  {
    long long lo, hi;
    team_range<ClusterTeam, NT, CS>(all, m.nc[0], lo, hi);
    float* b = A.lb + m.off[0];
    for (long long i = lo + threadIdx.x; i < hi; i += NT) b[i] = (float)A.Rr[cell_off + i];
  }
  cl.sync();
  for (int l = 0; l < ls; ++l) vdown<ClusterTeam, NT, CS>(A, m, l, global_view(A, m, l), global_view(A, m, l + 1), all, cl);
  if (rank == 0) {
    const LevelView top = solo_view(A, m, ls, ls, smem);
    const float* gb = A.lb + m.off[ls];
    for (long long i = threadIdx.x; i < m.nc[ls]; i += NT) top.b[i] = __ldcg(&gb[i]);
    __syncthreads();
    for (int l = ls; l < L - 1; ++l)
      vdown<SoloTeam, NT, CS>(A, m, l, solo_view(A, m, l, ls, smem), solo_view(A, m, l + 1, ls, smem), solo, cl);
    vcoarsest<SoloTeam, NT, CS>(A, m, solo_view(A, m, L - 1, ls, smem), solo, cl);
    for (int l = L - 2; l >= ls; --l)
      vup<SoloTeam, NT, CS>(A, m, l, solo_view(A, m, l, ls, smem), solo_view(A, m, l + 1, ls, smem), solo, cl);
    float* gx = A.lx + m.off[ls];
    for (long long i = threadIdx.x; i < m.nc[ls]; i += NT) gx[i] = top.x[i];
  }
  cl.sync();
  for (int l = ls - 1; l >= 0; --l) vup<ClusterTeam, NT, CS>(A, m, l, global_view(A, m, l), global_view(A, m, l + 1), all, cl);
  {
    long long lo, hi;
    team_range<ClusterTeam, NT, CS>(all, m.nc[0], lo, hi);
    const float* x = A.lx + m.off[0];
    for (long long i = lo + threadIdx.x; i < hi; i += NT) A.Z[cell_off + i] = (double)__ldcg(&x[i]);
  }
}

// ---- Fast diagonalization (Lynch, Rice and Thomas 1964) for separable operators ----
// With A = Tx (x) I + I (x) Ty, Tx = Qx Lx Qx^T and Ty = Qy Ly Qy^T, and the right-hand side
// as an ny x nx matrix S (row j = the cells of y-row j), A X = S is solved by
//   X = Qy [(Qy^T S Qx) ./ (ly_j + lx_i)] Qx^T,
// four dense products of FP32 matrices (nx, ny <= FD_MAX_N). The rows j are split over the
// cluster's CTAs; each product reads what the other CTAs wrote through L2 after a cluster
// barrier. The solve runs inside FP64 iterative refinement: the solution is accumulated in
// FP64 and its residual S - A X is formed with the FP64 operator, until it meets rtol.

// Tiles of the dense products: FDT_BM rows x FDT_BN columns of the output per tile (each of
// the 512 threads 4 rows x 4 columns, from one float4 of each operand per term), FDT_BK terms
// per stage; the next stage's operands are loaded into registers while the current stage is
// multiplied from shared memory. Shared rows are padded by 4 words (16-byte aligned float4
// reads, at most 2-way conflicts on the transposing stores).
constexpr int FDT_BM = 64, FDT_BN = 128, FDT_BK = 16;
constexpr int FDT_AS = FDT_BM + 4, FDT_BS = FDT_BN + 4;

// out(j, i) for rows j in [j0, j1) and columns i < N of sum over k < K of L(j, k) R(k, i).
// L_KC: L is contiguous along k (else along j); R_IC: R is contiguous along i (else along
// k); the tile loads run along the contiguous index.
template <int NT, bool L_KC, bool R_IC, class FL, class FR, class FE>
__device__ __forceinline__ void tile_product(int j0, int j1, int N, int K, FL L, FR R, FE out, float* As,
                                             float* Bs) {
  static_assert(NT == 512, "4 x 4 outputs per thread: 512 threads = 16 x 32 groups");
  constexpr int NA = FDT_BK * FDT_BM / NT, NB = FDT_BK * FDT_BN / NT;  // loads per thread and stage
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int jt = j0; jt < j1; jt += FDT_BM) {
    for (int it = 0; it < N; it += FDT_BN) {
      float acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
      float ra[NA], rb[NB];
      auto load = [&](int kt) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
          const int e = threadIdx.x + q * NT;
          const int kk = L_KC ? e % FDT_BK : e / FDT_BM, jj = L_KC ? e / FDT_BK : e % FDT_BM;
          ra[q] = (jt + jj < j1 && kt + kk < K) ? L(jt + jj, kt + kk) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const int e = threadIdx.x + q * NT;
          const int kk = R_IC ? e / FDT_BN : e % FDT_BK, ii = R_IC ? e % FDT_BN : e / FDT_BK;
          rb[q] = (kt + kk < K && it + ii < N) ? R(kt + kk, it + ii) : 0.f;
        }
      };
      auto store = [&](int buf) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
          const int e = threadIdx.x + q * NT;
          const int kk = L_KC ? e % FDT_BK : e / FDT_BM, jj = L_KC ? e / FDT_BK : e % FDT_BM;
          As[(buf * FDT_BK + kk) * FDT_AS + jj] = ra[q];
        }
#pragma unroll
        for (int q = 0; q < NB; ++q) {
          const int e = threadIdx.x + q * NT;
          const int kk = R_IC ? e / FDT_BN : e % FDT_BK, ii = R_IC ? e % FDT_BN : e / FDT_BK;
          Bs[(buf * FDT_BK + kk) * FDT_BS + ii] = rb[q];
        }
      };
      load(0);
      store(0);
      __syncthreads();
      int buf = 0;
      for (int kt = 0; kt < K; kt += FDT_BK) {
        const bool more = kt + FDT_BK < K;
        if (more) load(kt + FDT_BK);
#pragma unroll
        for (int k = 0; k < FDT_BK; ++k) {
          const float4 a = *reinterpret_cast<const float4*>(&As[(buf * FDT_BK + k) * FDT_AS + 4 * ty]);
          const float4 b = *reinterpret_cast<const float4*>(&Bs[(buf * FDT_BK + k) * FDT_BS + 4 * tx]);
          const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int j = jt + 4 * ty + r;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int i = it + 4 * tx + c;
          if (j < j1 && i < N) out(j, i, acc[r][c]);
        }
      }
    }
  }
}

// Solves the instance's correction by fast diagonalization with FP64 refinement (at most
// MG32_PASSES_FD passes); returns the passes taken, or -1 if rtol was not met.
template <int NT, int CS>
__device__ int fd_solve(const MGArgs& A, const InstMG& m, cg::cluster_group& cl, int rank, ClusterRed<NT, CS>& red,
                        double* sh) {
  const int nx = m.fnx, ny = m.fny;
  const long long off = m.cell_off, n = m.nc[0];
  const long long sy = m.n[0][0];
  const int rows = (ny + CS - 1) / CS, j0 = min(ny, rank * rows), j1 = min(ny, j0 + rows);
  const long long lo = (long long)j0 * nx, hi = (long long)j1 * nx;  // this CTA's cells
  const float* Qx = A.fq + m.qx_off;
  const float* Qy = A.fq + m.qy_off;
  const float* lx = A.flam + m.lx_off;
  const float* ly = A.flam + m.ly_off;
  float* Sf = A.lt + m.off[0];  // scaled residual (FP32)
  float* T1 = A.lb + m.off[0];  // Qy^T S, then Qy T2
  float* T2 = A.lx + m.off[0];  // (Qy^T S Qx) ./ (ly + lx)
  __shared__ __align__(16) float As[2 * FDT_BK * FDT_AS];
  __shared__ __align__(16) float Bs[2 * FDT_BK * FDT_BS];
  double v[4];
  v[0] = 0.0;
  for (long long c = lo + threadIdx.x; c < hi; c += NT) {
    const double b = A.rhs[off + c];
    A.X[off + c] = 0.0;
    A.Z[off + c] = b;  // FP64 residual
    v[0] += b * b;
  }
  red.sum(cl, v, 1, sh);
  const double bb = v[0];
  if (bb == 0.0) return 0;
  const double tol2 = A.rtol * A.rtol * bb;
  double rr = bb;
  for (int pass = 1; pass <= MG32_PASSES_FD && pass <= A.maxit; ++pass) {
    const double rn = sqrt(rr), sc = 1.0 / rn;
    for (long long c = lo + threadIdx.x; c < hi; c += NT) Sf[c] = (float)(__ldcg(&A.Z[off + c]) * sc);
    cl.sync();
    // T1 = Qy^T S (rows j of this CTA), then T2 = T1 Qx ./ (ly_j + lx_i) (same rows)
    tile_product<NT, false, true>(
        j0, j1, nx, ny, [&](int j, int k) { return __ldg(&Qy[(long long)k * ny + j]); },
        [&](int k, int i) { return __ldcg(&Sf[(long long)k * nx + i]); },
        [&](int j, int i, float x) { T1[(long long)j * nx + i] = x; }, As, Bs);
    __syncthreads();
    tile_product<NT, true, true>(
        j0, j1, nx, nx, [&](int j, int k) { return __ldcg(&T1[(long long)j * nx + k]); },
        [&](int k, int i) { return __ldg(&Qx[(long long)k * nx + i]); },
        [&](int j, int i, float x) { T2[(long long)j * nx + i] = x / (ly[j] + lx[i]); }, As, Bs);
    cl.sync();
    // T1 = Qy T2, then the correction T1 Qx^T added to the FP64 solution (scaled back)
    tile_product<NT, true, true>(
        j0, j1, nx, ny, [&](int j, int k) { return __ldg(&Qy[(long long)j * ny + k]); },
        [&](int k, int i) { return __ldcg(&T2[(long long)k * nx + i]); },
        [&](int j, int i, float x) { T1[(long long)j * nx + i] = x; }, As, Bs);
    __syncthreads();
    tile_product<NT, true, false>(
        j0, j1, nx, nx, [&](int j, int k) { return __ldcg(&T1[(long long)j * nx + k]); },
        [&](int k, int i) { return __ldg(&Qx[(long long)i * nx + k]); },
        [&](int j, int i, float x) { A.X[off + (long long)j * nx + i] += (double)x * rn; }, As, Bs);
    cl.sync();
    // FP64 residual of the FP64 solution
    v[0] = 0.0;
    for (long long c = lo + threadIdx.x; c < hi; c += NT) {
      const long long g = off + c;
      double q = A.diag[g] * __ldcg(&A.X[g]);
      if (c + 1 < n) q -= A.cx[g] * __ldcg(&A.X[g + 1]);
      if (c >= 1) q -= A.cx[g - 1] * __ldcg(&A.X[g - 1]);
      if (m.dim >= 2) {
        if (c + sy < n) q -= A.cy[g] * __ldcg(&A.X[g + sy]);
        if (c >= sy) q -= A.cy[g - sy] * __ldcg(&A.X[g - sy]);
      }
      const double r = A.rhs[g] - q;
      A.Z[g] = r;
      v[0] += r * r;
    }
    red.sum(cl, v, 1, sh);  // also orders the residual's writes before the next pass
    rr = v[0];
    if (rr <= tol2) return pass;
  }
  return -1;
}

// The same solve for nx, ny <= FD_SMALL_N with every operand in shared memory: Qx (rows
// padded to FD_SMALL_N + 1 words, so that both Qx and its transpose are read without bank
// conflicts), this CTA's rows and columns of Qy, and the full ny x nx right operand of the
// products that need every row (S, then T2), gathered from the cluster's CTAs through
// distributed shared memory. Each CTA keeps its rows of S, T1 and T2 in its own memory.
constexpr int FD_SMALL_N = 128;
constexpr int FD_SMALL_R = 16;  // rows per CTA (ny <= FD_SMALL_R * cluster size)
constexpr int FDS_QX = 0;                                                   // [N][N + 1]
constexpr int FDS_QYC = FDS_QX + FD_SMALL_N * (FD_SMALL_N + 1);             // [R][N]: Qy(k, j0 + r)
constexpr int FDS_QYR = FDS_QYC + FD_SMALL_R * FD_SMALL_N;                  // [R][N]: Qy(j0 + r, k)
constexpr int FDS_FULL = FDS_QYR + FD_SMALL_R * FD_SMALL_N;                 // [N][N]
constexpr int FDS_S = FDS_FULL + FD_SMALL_N * FD_SMALL_N;                   // [R][N] rows of S
constexpr int FDS_T2 = FDS_S + FD_SMALL_R * FD_SMALL_N;                     // [R][N] rows of T2
constexpr int FDS_T1 = FDS_T2 + FD_SMALL_R * FD_SMALL_N;                    // [R][N] rows of T1
constexpr int FDS_LX = FDS_T1 + FD_SMALL_R * FD_SMALL_N;                    // [N]
constexpr int FDS_LY = FDS_LX + FD_SMALL_N;                                 // [R]
constexpr int FDS_FLOATS = FDS_LY + FD_SMALL_R;
constexpr size_t FD_SMALL_SMEM = (size_t)FDS_FLOATS * sizeof(float);

// acc[q] = sum over k < K4 of L[(tg + 4 q) * N + k] R(k), for the four rows of this thread
// (L rows N words apart, 16-byte aligned, zero beyond the true K).
template <class FR>
__device__ __forceinline__ void fds_rows4(const float* L, int tg, int K4, FR R, float (&acc)[4]) {
  acc[0] = acc[1] = acc[2] = acc[3] = 0.f;
  for (int k = 0; k < K4; k += 4) {
    const float r0 = R(k), r1 = R(k + 1), r2 = R(k + 2), r3 = R(k + 3);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 l = *reinterpret_cast<const float4*>(L + (tg + 4 * q) * FD_SMALL_N + k);
      acc[q] = fmaf(l.x, r0, fmaf(l.y, r1, fmaf(l.z, r2, fmaf(l.w, r3, acc[q]))));
    }
  }
}

// full (rows < ny) <- every CTA's rows of strip, through distributed shared memory.
template <int NT, int CS>
__device__ __forceinline__ void fds_gather(cg::cluster_group& cl, float* full, float* strip, int ny, int rows) {
  const int n4 = ny * (FD_SMALL_N / 4);
  for (int e = threadIdx.x; e < n4; e += NT) {
    const int k = e / (FD_SMALL_N / 4), c4 = e - k * (FD_SMALL_N / 4);
    const int q = k / rows;
    const float4* src = reinterpret_cast<const float4*>(cl.map_shared_rank(strip, q) + (k - q * rows) * FD_SMALL_N);
    reinterpret_cast<float4*>(full + k * FD_SMALL_N)[c4] = src[c4];
  }
}

template <int NT, int CS>
__device__ int fd_solve_small(const MGArgs& A, const InstMG& m, cg::cluster_group& cl, int rank,
                              ClusterRed<NT, CS>& red, double* sh, float* smem) {
  static_assert(NT == 4 * FD_SMALL_N, "one column and four rows per thread");
  static_assert(FD_SMALL_R * CS >= FD_SMALL_N, "rows per CTA");
  const int nx = m.fnx, ny = m.fny;
  const long long off = m.cell_off, n = m.nc[0];
  const long long sy = m.n[0][0];
  const int rows = (ny + CS - 1) / CS, j0 = min(ny, rank * rows), j1 = min(ny, j0 + rows);
  const long long lo = (long long)j0 * nx, hi = (long long)j1 * nx;  // this CTA's cells
  const int tc = threadIdx.x % FD_SMALL_N, tg = threadIdx.x / FD_SMALL_N;
  const int kx4 = (nx + 3) & ~3, ky4 = (ny + 3) & ~3;
  float* qx = smem + FDS_QX;
  float* qyc = smem + FDS_QYC;
  float* qyr = smem + FDS_QYR;
  float* full = smem + FDS_FULL;
  float* sS = smem + FDS_S;
  float* sT2 = smem + FDS_T2;
  float* sT1 = smem + FDS_T1;
  float* slx = smem + FDS_LX;
  float* sly = smem + FDS_LY;
  {
    // operands, zero outside the true sizes (the products run over multiples of 4 terms)
    const float* Qx = A.fq + m.qx_off;
    const float* Qy = A.fq + m.qy_off;
    for (int e = threadIdx.x; e < FD_SMALL_N * (FD_SMALL_N + 1); e += NT) {
      const int k = e / (FD_SMALL_N + 1), i = e - k * (FD_SMALL_N + 1);
      qx[e] = (k < nx && i < nx) ? __ldg(&Qx[(long long)k * nx + i]) : 0.f;
    }
    for (int e = threadIdx.x; e < FD_SMALL_R * FD_SMALL_N; e += NT) {
      const int r = e / FD_SMALL_N, k = e - r * FD_SMALL_N, j = j0 + r;
      const bool in = j < j1 && k < ny;
      qyc[e] = in ? __ldg(&Qy[(long long)k * ny + j]) : 0.f;
      qyr[e] = in ? __ldg(&Qy[(long long)j * ny + k]) : 0.f;
      sS[e] = 0.f;
      sT2[e] = 0.f;
      sT1[e] = 0.f;
    }
    for (int e = threadIdx.x; e < FD_SMALL_N * FD_SMALL_N; e += NT) full[e] = 0.f;
    for (int i = threadIdx.x; i < FD_SMALL_N; i += NT) slx[i] = i < nx ? A.flam[m.lx_off + i] : 1.f;
    for (int r = threadIdx.x; r < FD_SMALL_R; r += NT) sly[r] = j0 + r < j1 ? A.flam[m.ly_off + j0 + r] : 1.f;
  }
  double v[4];
  v[0] = 0.0;
  for (long long c = lo + threadIdx.x; c < hi; c += NT) {
    const double b = A.rhs[off + c];
    A.X[off + c] = 0.0;
    A.Z[off + c] = b;  // FP64 residual
    v[0] += b * b;
  }
  red.sum(cl, v, 1, sh);  // also orders the operand set-up before first use
  const double bb = v[0];
  if (bb == 0.0) return 0;
  const double tol2 = A.rtol * A.rtol * bb;
  double rr = bb;
  float acc[4];
  for (int pass = 1; pass <= MG32_PASSES_FD && pass <= A.maxit; ++pass) {
    const double rn = sqrt(rr), sc = 1.0 / rn;
    for (long long c = lo + threadIdx.x; c < hi; c += NT) {
      const int r = (int)(c / nx), i = (int)(c - (long long)r * nx);
      sS[(r - j0) * FD_SMALL_N + i] = (float)(__ldcg(&A.Z[off + c]) * sc);
    }
    cl.sync();
    fds_gather<NT, CS>(cl, full, sS, ny, rows);
    __syncthreads();
    // T1 = Qy^T S (this CTA's rows), then T2 = T1 Qx ./ (ly_j + lx_i)
    fds_rows4(qyc, tg, ky4, [&](int k) { return full[k * FD_SMALL_N + tc]; }, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (tc < nx) sT1[(tg + 4 * q) * FD_SMALL_N + tc] = acc[q];
    __syncthreads();
    fds_rows4(sT1, tg, kx4, [&](int k) { return qx[k * (FD_SMALL_N + 1) + tc]; }, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = tg + 4 * q;
      if (tc < nx && j0 + r < j1) sT2[r * FD_SMALL_N + tc] = acc[q] / (sly[r] + slx[tc]);
    }
    cl.sync();
    fds_gather<NT, CS>(cl, full, sT2, ny, rows);
    __syncthreads();
    // T1 = Qy T2, then the correction T1 Qx^T added to the FP64 solution (scaled back)
    fds_rows4(qyr, tg, ky4, [&](int k) { return full[k * FD_SMALL_N + tc]; }, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (tc < nx) sT1[(tg + 4 * q) * FD_SMALL_N + tc] = acc[q];
    __syncthreads();
    fds_rows4(sT1, tg, kx4, [&](int k) { return qx[tc * (FD_SMALL_N + 1) + k]; }, acc);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + tg + 4 * q;
      if (tc < nx && j < j1) A.X[off + (long long)j * nx + tc] += (double)acc[q] * rn;
    }
    cl.sync();
    // FP64 residual of the FP64 solution
    v[0] = 0.0;
    for (long long c = lo + threadIdx.x; c < hi; c += NT) {
      const long long g = off + c;
      double q = A.diag[g] * __ldcg(&A.X[g]);
      if (c + 1 < n) q -= A.cx[g] * __ldcg(&A.X[g + 1]);
      if (c >= 1) q -= A.cx[g - 1] * __ldcg(&A.X[g - 1]);
      if (m.dim >= 2) {
        if (c + sy < n) q -= A.cy[g] * __ldcg(&A.X[g + sy]);
        if (c >= sy) q -= A.cy[g - sy] * __ldcg(&A.X[g - sy]);
      }
      const double r = A.rhs[g] - q;
      A.Z[g] = r;
      v[0] += r * r;
    }
    red.sum(cl, v, 1, sh);  // also orders the residual's writes before the next pass
    rr = v[0];
    if (rr <= tol2) return pass;
  }
  return -1;
}

template <int NT, int CS>
__global__ void __launch_bounds__(NT) mgpcg_kernel(MGArgs A) {
  __shared__ double sh[4 * 32];
  __shared__ double slot[8];
  extern __shared__ float mg_smem[];  // CTA 0: the levels it handles alone
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int k = blockIdx.x / CS;
  const InstMG& m = A.mg[k];
  const long long off = m.cell_off, n = m.nc[0];
  const long long chunk = (n + CS - 1) / CS, lo = rank * chunk, hi = min(n, lo + chunk);
  const long long sy = m.n[0][0], sz = (long long)m.n[0][0] * m.n[0][1];
  ClusterRed<NT, CS> red{slot, 0};
  if (m.direct) {
    const int passes = m.direct == 2 ? fd_solve_small<NT, CS>(A, m, cl, rank, red, sh, mg_smem)
                                     : fd_solve<NT, CS>(A, m, cl, rank, red, sh);
    if (rank == 0 && threadIdx.x == 0) A.iters_out[k] = passes;
    cl.sync();  // no CTA leaves while another may still read its shared memory
    return;
  }
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
    cl.sync();
    return;
  }
  const double tol2 = A.rtol * A.rtol * bb;
  vcycle<NT, CS>(A, m, cl, rank, off, mg_smem);
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
    vcycle<NT, CS>(A, m, cl, rank, off, mg_smem);
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
  cl.sync();
}

// The same V-cycle for the FP32 iterates of mgpcg32_kernel: the finest level's right-hand
// side and iterate are the CG's residual and preconditioned residual themselves (no copies;
// the caller's last cluster barrier ordered the residual's writes).
template <int NT, int CS>
__device__ void vcycle_f32(const MGArgs& A, const InstMG& m, cg::cluster_group& cl, int rank, float* smem) {
  const ClusterTeam all{rank};
  const SoloTeam solo;
  const int L = m.levels;
  const int ls = solo_level(m);
  for (int l = 0; l < ls; ++l) vdown<ClusterTeam, NT, CS>(A, m, l, global_view(A, m, l), global_view(A, m, l + 1), all, cl);
  if (rank == 0) {
    const LevelView top = solo_view(A, m, ls, ls, smem);
    const float* gb = A.lb + m.off[ls];
    for (long long i = threadIdx.x; i < m.nc[ls]; i += NT) top.b[i] = __ldcg(&gb[i]);
    __syncthreads();
    for (int l = ls; l < L - 1; ++l)
      vdown<SoloTeam, NT, CS>(A, m, l, solo_view(A, m, l, ls, smem), solo_view(A, m, l + 1, ls, smem), solo, cl);
    vcoarsest<SoloTeam, NT, CS>(A, m, solo_view(A, m, L - 1, ls, smem), solo, cl);
    for (int l = L - 2; l >= ls; --l)
      vup<SoloTeam, NT, CS>(A, m, l, solo_view(A, m, l, ls, smem), solo_view(A, m, l + 1, ls, smem), solo, cl);
    float* gx = A.lx + m.off[ls];
    for (long long i = threadIdx.x; i < m.nc[ls]; i += NT) gx[i] = top.x[i];
  }
  cl.sync();
  for (int l = ls - 1; l >= 0; --l) vup<ClusterTeam, NT, CS>(A, m, l, global_view(A, m, l), global_view(A, m, l + 1), all, cl);
}

// The FP64 residual b - A x of the FP64 iterate over this CTA's cells, into Rt (FP64 fine
// operator); returns this thread's share of its squared norm.
__device__ __forceinline__ double true_residual(const MGArgs& A, const InstMG& m, double* Rt, long long off,
                                                long long lo, long long hi, long long n, int NT) {
  const long long sy = m.n[0][0], sz = (long long)m.n[0][0] * m.n[0][1];
  double rr = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NT) {
    const long long g = off + i;
    double q = A.diag[g] * __ldcg(&A.X[g]);
    if (i + 1 < n) q -= A.cx[g] * __ldcg(&A.X[g + 1]);
    if (i >= 1) q -= A.cx[g - 1] * __ldcg(&A.X[g - 1]);
    if (m.dim >= 2) {
      if (i + sy < n) q -= A.cy[g] * __ldcg(&A.X[g + sy]);
      if (i >= sy) q -= A.cy[g - sy] * __ldcg(&A.X[g - sy]);
    }
    if (m.dim >= 3) {
      if (i + sz < n) q -= A.cz[g] * __ldcg(&A.X[g + sz]);
      if (i >= sz) q -= A.cz[g - sz] * __ldcg(&A.X[g - sz]);
    }
    const double r = A.rhs[g] - q;
    Rt[g] = r;
    rr += r * r;
  }
  return rr;
}

// PCG with FP32 iterates for tolerances far above FP32's rounding (the correction is an
// inexact Newton step: its tolerance sets the cost, not the fixed point), inside FP64
// iterative refinement: the solution is accumulated in FP64 and its residual b - A x is
// formed and measured in FP64 with the FP64 operator; while that residual exceeds the
// tolerance (at most MG32_PASSES times) the FP32 PCG solves for the correction of that
// residual. Each pass scales its right-hand side to unit norm (so the FP32 sums neither
// underflow nor overflow); the stencil product uses the FP32 copy of the fine operator (the
// hierarchy's finest level); dot products are FP32 per thread and FP64 across the cluster.
// On GB300 FP64 arithmetic issues on a narrow pipe, so FP64 iterates would lengthen every
// phase of the iteration; here FP64 enters once per pass.
constexpr int MG32_PASSES = 4;

template <int NT, int CS>
__global__ void __launch_bounds__(NT, 1) mgpcg32_kernel(MGArgs A, float* V32) {
  __shared__ double sh[4 * 32];
  __shared__ double slot[8];
  extern __shared__ float mg_smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int k = blockIdx.x / CS;
  const InstMG& m = A.mg[k];
  const long long off = m.cell_off, n = m.nc[0];
  const long long chunk = (n + CS - 1) / CS, lo = rank * chunk, hi = min(n, lo + chunk);
  float* R = A.lb + m.off[0];  // residual = the V-cycle's finest right-hand side
  float* Z = A.lx + m.off[0];  // preconditioned residual = its finest iterate
  float* X = V32 + 3 * off;
  float* P = X + n;
  float* Q = P + n;
  const float *dg = A.ldiag + m.off[0], *cx = A.lcx + m.off[0], *cy = A.lcy + m.off[0], *cz = A.lcz + m.off[0];
  ClusterRed<NT, CS> red{slot, 0};
  if (m.direct) {
    const int passes = m.direct == 2 ? fd_solve_small<NT, CS>(A, m, cl, rank, red, sh, mg_smem)
                                     : fd_solve<NT, CS>(A, m, cl, rank, red, sh);
    if (rank == 0 && threadIdx.x == 0) A.iters_out[k] = passes;
    cl.sync();  // no CTA leaves while another may still read its shared memory
    return;
  }
  double v[4];
  // x = 0, FP64 residual r = b
  v[0] = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += NT) {
    const double bi = A.rhs[off + i];
    A.X[off + i] = 0.0;
    A.Z[off + i] = bi;
    v[0] += bi * bi;
  }
  red.sum(cl, v, 1, sh);
  const double bb = v[0];
  if (bb == 0.0) {
    if (rank == 0 && threadIdx.x == 0) A.iters_out[k] = 0;
    cl.sync();
    return;
  }
  const double tol2 = A.rtol * A.rtol * bb;
  double rr = bb;  // FP64 squared norm of the FP64 residual
  int it = 0;
  bool done = false;
  for (int pass = 0; pass < MG32_PASSES && it < A.maxit; ++pass) {
    // FP32 PCG for A e = r (scaled to unit norm) to the relative tolerance the FP64 residual
    // still needs, at least the requested one and at most 1/2
    const double rn = sqrt(rr), sc = 1.0 / rn;
    const double rin = fmin(0.5, fmax(A.rtol, A.rtol * sqrt(bb) / rn));
    const double in2 = rin * rin;
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      R[i] = (float)(A.Z[off + i] * sc);
      X[i] = 0.f;
    }
    cl.sync();
    vcycle_f32<NT, CS>(A, m, cl, rank, mg_smem);
    float f0 = 0.f;
    for (long long i = lo + threadIdx.x; i < hi; i += NT) {
      const float zi = Z[i];
      P[i] = zi;
      f0 += R[i] * zi;
    }
    v[0] = f0;
    red.sum(cl, v, 1, sh);  // also orders the P writes before the first product
    double rz = v[0];
    while (it < A.maxit) {
      ++it;
      f0 = 0.f;
      for (long long i = lo + threadIdx.x; i < hi; i += NT) {
        const float q = level_apply<ClusterTeam>(dg, cx, cy, cz, P, m.n[0], m.dim, i, n);
        Q[i] = q;
        f0 += __ldcg(&P[i]) * q;
      }
      v[0] = f0;
      red.sum(cl, v, 1, sh);
      const double alpha = rz / v[0];
      const float af = (float)alpha;
      f0 = 0.f;
      for (long long i = lo + threadIdx.x; i < hi; i += NT) {
        X[i] += af * P[i];
        const float ri = R[i] - af * Q[i];
        R[i] = ri;
        f0 += ri * ri;
      }
      v[0] = f0;
      red.sum(cl, v, 1, sh);  // also orders the residual's writes before the V-cycle
      if (v[0] <= in2) break;
      vcycle_f32<NT, CS>(A, m, cl, rank, mg_smem);
      // flexible (Polak-Ribiere) beta, as in the FP64 kernel
      float f1 = 0.f;
      f0 = 0.f;
      for (long long i = lo + threadIdx.x; i < hi; i += NT) {
        const float zi = Z[i];
        f0 += R[i] * zi;
        f1 += Q[i] * zi;
      }
      v[0] = f0;
      v[1] = f1;
      red.sum(cl, v, 2, sh);
      const double beta = -alpha * v[1] / rz;
      rz = v[0];
      const float bf = (float)beta;
      for (long long i = lo + threadIdx.x; i < hi; i += NT) P[i] = Z[i] + bf * P[i];
      cl.sync();
    }
    // x += rn e in FP64, then the FP64 residual of x
    for (long long i = lo + threadIdx.x; i < hi; i += NT) A.X[off + i] += (double)X[i] * rn;
    cl.sync();
    v[0] = true_residual(A, m, A.Z, off, lo, hi, n, NT);
    red.sum(cl, v, 1, sh);  // also orders the residual's writes before the next pass
    rr = v[0];
    if (rr <= tol2) {
      done = true;
      break;
    }
  }
  if (rank == 0 && threadIdx.x == 0) A.iters_out[k] = done ? it : -1;
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

// Tolerances from here up run the FP32 iterates.
constexpr double MG32_MIN_RTOL = 1e-5;

constexpr int MG_NT = 512;
constexpr int MG_CS = 8;

// Shared memory of CTA 0: b, x, t, r of every level from solo_level down (host side).
size_t mg_solo_smem_bytes(const std::vector<InstMG>& h_mg) {
  size_t best = 0;
  for (const InstMG& m : h_mg) {
    size_t cells = 0;
    for (int l = solo_level(m); l < m.levels; ++l) cells += (size_t)m.nc[l];
    best = std::max(best, 4 * cells * sizeof(float));
  }
  return best;
}

size_t fd_small_smem_bytes() { return FD_SMALL_SMEM; }
int fd_small_max_n() { return FD_SMALL_N; }

cudaError_t configure_mgpcg(Ctx* c, size_t smem) {
  c->mg_smem_bytes = smem;
  const cudaError_t e =
      cudaFuncSetAttribute(mgpcg_kernel<MG_NT, MG_CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(mgpcg32_kernel<MG_NT, MG_CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

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
  a.fq = c->d_fd_q;
  a.flam = c->d_fd_lam;
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
  cfg.dynamicSmemBytes = c->mg_smem_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = MG_CS;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (c->opt.cg_rtol >= MG32_MIN_RTOL) {
    // FP32 x, p, q in the space of the FP64 r and p (2 n doubles = 4 n floats >= 3 n floats);
    // the FP64 residual of the refinement in that of z
    float* v32 = reinterpret_cast<float*>(c->d_pcg + c->total_cells);
    return cudaLaunchKernelEx(&cfg, mgpcg32_kernel<MG_NT, MG_CS>, a, v32);
  }
  return cudaLaunchKernelEx(&cfg, mgpcg_kernel<MG_NT, MG_CS>, a);
}

}  // namespace iugkp
