// Diffusion-correction solve that allocates no device memory.
//
// The paper has no counterpart: this entry point exists for callers that cannot call
// cudaMalloc -- for example code whose device memory is owned entirely by another
// allocator (a framework's caching pool that has already reserved the GPU), or a
// latency-critical loop that cannot afford the implicit device synchronisation an
// allocation may cause. All scratch (the stencil, the CG vectors and the iteration
// count) lives in one file-scope static device array of fixed size, which every GPU that
// loads this library keeps until the process exits.
//
// Usage rules (also stated in include/iugkp.h):
//  * at most IUGKP_NOALLOC_MAX_CELLS cells per call; larger grids are rejected;
//  * every call reuses the same array, so calls whose kernels overlap on the GPU (for
//    example on two streams, or from two host threads) race with each other;
//  * the first call on a device looks the array's device address up once
//    (cudaGetSymbolAddress) with that device current; make that first call before any
//    stream capture.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/iugkp.h"
#include "internal.h"

namespace {

constexpr long long kMaxCells = IUGKP_NOALLOC_MAX_CELLS;
// Layout: diag, cx, cy, cz, r, p, q (7 x kMaxCells doubles), then the iteration count and a
// flag set when some kappa is not positive and finite.
constexpr long long kScratchDoubles = 7 * kMaxCells + 32;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_mutex;
double* g_ptr[256] = {nullptr};

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t scratch_ptr(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

struct NGrid {
  int dim, n0, n1, n2;
  double h0, h1, h2;
  long long nc;
};

// Stencil of -div(kappa grad x) per cell: harmonic face kappa over h^2 between cells; at
// a wall the half-cell conduction in series with the vacuum condition (flux = cv/2 x).
// A kappa that is not positive and finite sets *bad (the solve then stops before iterating).
__global__ void noalloc_stencil_kernel(NGrid g, const double* kappa, double cv, double* diag, double* cx, double* cy,
                                       double* cz, double* bad) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < g.nc; i += (long long)gridDim.x * blockDim.x) {
    if (!(kappa[i] > 0.0) || !isfinite(kappa[i])) *bad = 1.0;
    const int ix = (int)(i % g.n0), iy = (int)((i / g.n0) % g.n1), iz = (int)(i / ((long long)g.n0 * g.n1));
    const int idx[3] = {ix, iy, iz};
    const int n[3] = {g.n0, g.n1, g.n2};
    const double h[3] = {g.h0, g.h1, g.h2};
    const long long st[3] = {1, g.n0, (long long)g.n0 * g.n1};
    double d = 0.0, c[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < g.dim; ++a) {
      for (int side = -1; side <= 1; side += 2) {
        const int j = idx[a] + side;
        if (j < 0 || j >= n[a]) {
          d += 1.0 / (h[a] / (2.0 * kappa[i]) + 2.0 / cv) / h[a];
        } else {
          const double kn = kappa[i + side * st[a]];
          const double kf = 2.0 * kappa[i] * kn / (kappa[i] + kn);
          d += kf / (h[a] * h[a]);
          if (side > 0) c[a] = kf / (h[a] * h[a]);
        }
      }
    }
    diag[i] = d;
    cx[i] = c[0];
    cy[i] = c[1];
    cz[i] = c[2];
  }
}

__device__ __forceinline__ double nblock_sum(double x, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    double y = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
    if (lane == 0) sh[32] = y;
  }
  __syncthreads();
  return sh[32];
}

// Jacobi-preconditioned CG, one block, x0 = 0 (x is cleared here). Writes into *iters the
// iteration count, -1 when maxit is reached, -2 when a kappa was not positive and finite
// (nothing solved), -3 when a product or residual turned out not finite (NaN or Inf in rhs).
__global__ void __launch_bounds__(1024) noalloc_pcg_kernel(NGrid g, const double* diag, const double* cx,
                                                           const double* cy, const double* cz, const double* b,
                                                           double* x, double* r, double* p, double* q, double rtol,
                                                           int maxit, double* iters) {
  __shared__ double sh[33];
  const long long n = g.nc, sy = g.n0, sz = (long long)g.n0 * g.n1;
  if (iters[1] != 0.0) {
    if (threadIdx.x == 0) iters[0] = -2.0;
    return;
  }
  double bb = 0.0, rz = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    p[i] = bi / diag[i];
    bb += bi * bi;
    rz += bi * bi / diag[i];
  }
  bb = nblock_sum(bb, sh);
  rz = nblock_sum(rz, sh);
  if (bb == 0.0 || !isfinite(bb)) {
    for (long long i = threadIdx.x; i < n; i += blockDim.x) x[i] = 0.0;
    if (threadIdx.x == 0) iters[0] = bb == 0.0 ? 0.0 : -3.0;
    return;
  }
  const double tol2 = rtol * rtol * bb;
  int it = 0;
  bool done = false, bad = false;
  while (it < maxit) {
    ++it;
    double pq = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      double qi = diag[i] * p[i];
      if (i + 1 < n) qi -= cx[i] * p[i + 1];
      if (i >= 1) qi -= cx[i - 1] * p[i - 1];
      if (g.dim >= 2) {
        if (i + sy < n) qi -= cy[i] * p[i + sy];
        if (i >= sy) qi -= cy[i - sy] * p[i - sy];
      }
      if (g.dim >= 3) {
        if (i + sz < n) qi -= cz[i] * p[i + sz];
        if (i >= sz) qi -= cz[i - sz] * p[i - sz];
      }
      q[i] = qi;
      pq += p[i] * qi;
    }
    pq = nblock_sum(pq, sh);
    if (!isfinite(pq) || !(pq > 0.0)) {  // the operator is positive definite: anything else is bad data
      bad = true;
      break;
    }
    const double alpha = rz / pq;
    double rr = 0.0, rzn = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      x[i] += alpha * p[i];
      const double ri = r[i] - alpha * q[i];
      r[i] = ri;
      rr += ri * ri;
      rzn += ri * ri / diag[i];
    }
    rr = nblock_sum(rr, sh);
    rzn = nblock_sum(rzn, sh);
    if (!isfinite(rr)) {
      bad = true;
      break;
    }
    if (rr <= tol2) {
      done = true;
      break;
    }
    const double beta = rzn / rz;
    rz = rzn;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) p[i] = r[i] / diag[i] + beta * p[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) iters[0] = bad ? -3.0 : (done ? (double)it : -1.0);
}

}  // namespace

extern "C" iugkp_status iugkp_diffusion_solve_noalloc(const iugkp_grid* grid, const double* kappa_dev, double wall_cv,
                                                      const double* rhs_dev, double* x_dev, double rtol, int maxit,
                                                      int* iters_out, void* cuda_stream) {
  using iugkp::fail;
  if (!grid || !kappa_dev || !rhs_dev || !x_dev) return fail(nullptr, IUGKP_EINVAL, "noalloc solve: NULL argument");
  if (grid->dim < 1 || grid->dim > 3) return fail(nullptr, IUGKP_EINVAL, "noalloc solve: dim must be 1, 2 or 3");
  if (!(wall_cv > 0.0) || !(rtol > 0.0) || maxit < 1) return fail(nullptr, IUGKP_EINVAL, "noalloc solve: wall_cv, rtol > 0 and maxit >= 1");
  NGrid g;
  g.dim = grid->dim;
  g.n0 = grid->nx;
  g.n1 = grid->dim >= 2 ? grid->ny : 1;
  g.n2 = grid->dim >= 3 ? grid->nz : 1;
  const double l0 = grid->lx, l1 = grid->dim >= 2 ? grid->ly : 1.0, l2 = grid->dim >= 3 ? grid->lz : 1.0;
  if (g.n0 < 1 || g.n1 < 1 || g.n2 < 1 || !(l0 > 0.0) || !(l1 > 0.0) || !(l2 > 0.0))
    return fail(nullptr, IUGKP_EINVAL, "noalloc solve: cells and lengths must be positive");
  g.nc = (long long)g.n0 * g.n1 * g.n2;
  if (g.nc > kMaxCells)
    return fail(nullptr, IUGKP_EINVAL,
                "noalloc solve: grid has more than IUGKP_NOALLOC_MAX_CELLS (65536) cells; use iugkp_newton_step");
  g.h0 = l0 / g.n0;
  g.h1 = g.dim >= 2 ? l1 / g.n1 : 1.0;
  g.h2 = g.dim >= 3 ? l2 / g.n2 : 1.0;
  double* base = nullptr;
  cudaError_t e = scratch_ptr(&base);
  if (e != cudaSuccess) return fail(nullptr, IUGKP_ECUDA, std::string("noalloc solve: scratch lookup: ") + cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* diag = base;
  double* cx = base + kMaxCells;
  double* cy = base + 2 * kMaxCells;
  double* cz = base + 3 * kMaxCells;
  double* r = base + 4 * kMaxCells;
  double* p = base + 5 * kMaxCells;
  double* q = base + 6 * kMaxCells;
  double* it = base + 7 * kMaxCells;
  unsigned blocks = (unsigned)((g.nc + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  if ((e = cudaMemsetAsync(it + 1, 0, sizeof(double), s)) != cudaSuccess)
    return fail(nullptr, IUGKP_ECUDA, std::string("noalloc solve: ") + cudaGetErrorString(e));
  noalloc_stencil_kernel<<<blocks, 256, 0, s>>>(g, kappa_dev, wall_cv, diag, cx, cy, cz, it + 1);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(nullptr, IUGKP_ECUDA, std::string("noalloc solve: ") + cudaGetErrorString(e));
  noalloc_pcg_kernel<<<1, 1024, 0, s>>>(g, diag, cx, cy, cz, rhs_dev, x_dev, r, p, q, rtol, maxit, it);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(nullptr, IUGKP_ECUDA, std::string("noalloc solve: ") + cudaGetErrorString(e));
  double h_it = 0.0;
  if ((e = cudaMemcpyAsync(&h_it, it, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(nullptr, IUGKP_ECUDA, std::string("noalloc solve: ") + cudaGetErrorString(e));
  if (iters_out) *iters_out = (int)h_it;
  if (h_it == -2.0) return fail(nullptr, IUGKP_EINVAL, "noalloc solve: kappa must be positive and finite in every cell");
  if (h_it == -3.0) return fail(nullptr, IUGKP_EINVAL, "noalloc solve: a non-finite value arose (rhs not finite)");
  if (h_it < 0.0) return fail(nullptr, IUGKP_ENOCONV, "noalloc solve: maxit reached before rtol");
  return IUGKP_OK;
}
