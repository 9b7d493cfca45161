// Macroscopic kernels that close one IUGKP iteration: the macro update (arXiv
// 2506.09465 Sec. 3.1 step (3), Sec. 3.2 step (2)), the inexact-Newton correction
// (Sec. 3.3, Eqs. "macro-q-eqn", "macro-q-res", "linear-q") by matrix-free
// Jacobi-preconditioned CG on the finite-volume diffusion stencil, the residual,
// and the element-wise steps of the adjoint iteration. All FP64.
#include <cuda_runtime.h>

#include "internal.h"

namespace iugkp {

__device__ __forceinline__ int find_inst(const InstDesc* inst, int n_inst, long long g) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (inst[mid].cell_off <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// T_half = sum_b R_b / (V m); T_E = sum_b W_b / (V sum_b C_b).
__global__ void macro_kernel(const InstDesc* inst, int n_inst, int nb, long long total, const double* R,
                             const double* W, const double* Vm, const double* VC, double* T_half, double* T_E) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const int k = find_inst(inst, n_inst, g);
    const InstDesc& in = inst[k];
    const long long i = g - in.cell_off;
    const long long base = in.bc_off + i;
    double r = 0.0, w = 0.0;
    for (int b = 0; b < nb; ++b) r += R[base + (long long)b * in.ncells];
    if (T_half) T_half[g] = r / Vm[g];
    if (T_E && W) {
      for (int b = 0; b < nb; ++b) w += W[base + (long long)b * in.ncells];
      T_E[g] = w / VC[g];
    }
  }
}

// Newton source s = (sum_b R_b - T_n V m) / V (absorbed minus emitted power density).
__global__ void newton_rhs_kernel(const InstDesc* inst, int n_inst, int nb, long long total, const double* R,
                                  const double* T_n, const double* Vm, double* rhs) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    const int k = find_inst(inst, n_inst, g);
    const InstDesc& in = inst[k];
    const long long base = in.bc_off + (g - in.cell_off);
    double r = 0.0;
    for (int b = 0; b < nb; ++b) r += R[base + (long long)b * in.ncells];
    rhs[g] = (r - T_n[g] * Vm[g]) / in.V;
  }
}

// out = a + theta_k * x (theta per instance, or per cell when theta_cell is given).
__global__ void add_scaled_kernel(const InstDesc* inst, int n_inst, long long total, const double* a,
                                  const double* x, const double* theta_inst, const double* theta_cell, double* out) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    double th = theta_cell ? theta_cell[g] : theta_inst[find_inst(inst, n_inst, g)];
    out[g] = a[g] + th * x[g];
  }
}

__global__ void sub_kernel(long long total, const double* a, const double* b, double* out) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x)
    out[g] = a[g] - b[g];
}

__global__ void add_kernel(long long total, const double* a, const double* b, double* out) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x)
    out[g] = a[g] + b[g];
}

__global__ void div_kernel(long long total, const double* a, const double* b, double* out) {
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x)
    out[g] = a[g] / b[g];
}

// Block-wide sum in a fixed order (deterministic). All threads get the result.
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    double y = lane < NT / 32 ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xffffffffu, y, o);
    if (lane == 0) sh[32] = y;
  }
  __syncthreads();
  return sh[32];
}

// q = D p on instance `in` (cells [0, n) of the instance, arrays offset by cell_off).
__device__ __forceinline__ double stencil_row(const InstDesc& in, long long i, const double* diag, const double* cx,
                                              const double* cy, const double* cz, const double* p) {
  const long long n = in.ncells;
  const long long sy = in.n[0], sz = (long long)in.n[0] * in.n[1];
  double q = diag[i] * p[i];
  if (i + 1 < n) q -= cx[i] * p[i + 1];
  if (i >= 1) q -= cx[i - 1] * p[i - 1];
  if (in.dim >= 2) {
    if (i + sy < n) q -= cy[i] * p[i + sy];
    if (i >= sy) q -= cy[i - sy] * p[i - sy];
  }
  if (in.dim >= 3) {
    if (i + sz < n) q -= cz[i] * p[i + sz];
    if (i >= sz) q -= cz[i - sz] * p[i - sz];
  }
  return q;
}

// Jacobi-preconditioned CG for D x = b on one instance per block (x0 = 0).
// Stops when ||r|| <= rtol ||b|| or after maxit iterations (iters_out = -1 then).
template <int NT>
__global__ void __launch_bounds__(NT) pcg_block_kernel(const InstDesc* inst, const double* diag_g, const double* cx_g,
                                                       const double* cy_g, const double* cz_g, const double* b_g,
                                                       double* x_g, double* r_g, double* p_g, double* q_g, double rtol,
                                                       int maxit, int* iters_out) {
  __shared__ double sh[33];
  const InstDesc in = inst[blockIdx.x];
  const long long off = in.cell_off, n = in.ncells;
  const double* diag = diag_g + off;
  const double* cx = cx_g + off;
  const double* cy = cy_g + off;
  const double* cz = cz_g + off;
  const double* b = b_g + off;
  double* x = x_g + off;
  double* r = r_g + off;
  double* p = p_g + off;
  double* q = q_g + off;
  double bb = 0.0, rz = 0.0;
  for (long long i = threadIdx.x; i < n; i += NT) {
    const double bi = b[i];
    x[i] = 0.0;
    r[i] = bi;
    const double zi = bi / diag[i];
    p[i] = zi;
    bb += bi * bi;
    rz += bi * zi;
  }
  bb = block_sum<NT>(bb, sh);
  rz = block_sum<NT>(rz, sh);
  if (bb == 0.0) {
    if (threadIdx.x == 0) iters_out[blockIdx.x] = 0;
    return;
  }
  const double tol2 = rtol * rtol * bb;
  int it = 0;
  bool done = false;
  while (it < maxit) {
    ++it;
    double pq = 0.0;
    for (long long i = threadIdx.x; i < n; i += NT) {
      const double qi = stencil_row(in, i, diag, cx, cy, cz, p);
      q[i] = qi;
      pq += p[i] * qi;
    }
    pq = block_sum<NT>(pq, sh);
    const double alpha = rz / pq;
    double rr = 0.0, rzn = 0.0;
    for (long long i = threadIdx.x; i < n; i += NT) {
      x[i] += alpha * p[i];
      const double ri = r[i] - alpha * q[i];
      r[i] = ri;
      rr += ri * ri;
      rzn += ri * ri / diag[i];
    }
    rr = block_sum<NT>(rr, sh);
    rzn = block_sum<NT>(rzn, sh);
    if (rr <= tol2) {
      done = true;
      break;
    }
    const double beta = rzn / rz;
    rz = rzn;
    for (long long i = threadIdx.x; i < n; i += NT) p[i] = r[i] / diag[i] + beta * p[i];
    __syncthreads();
  }
  if (threadIdx.x == 0) iters_out[blockIdx.x] = done ? it : -1;
}

// Deterministic two-stage sums of (T1 - T0)^2 and T1^2 over all cells.
constexpr int RES_BLOCKS = 256;
__global__ void __launch_bounds__(256) residual_stage1(long long total, const double* T0, const double* T1,
                                                       double* partial) {
  __shared__ double sh[33];
  double a = 0.0, c = 0.0;
  for (long long g = (long long)blockIdx.x * 256 + threadIdx.x; g < total; g += (long long)RES_BLOCKS * 256) {
    const double d = T1[g] - T0[g];
    a += d * d;
    c += T1[g] * T1[g];
  }
  a = block_sum<256>(a, sh);
  c = block_sum<256>(c, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = c;
  }
}
__global__ void __launch_bounds__(256) residual_stage2(const double* partial, double* out) {
  __shared__ double sh[33];
  double a = partial[2 * threadIdx.x], c = partial[2 * threadIdx.x + 1];
  a = block_sum<256>(a, sh);
  c = block_sum<256>(c, sh);
  if (threadIdx.x == 0) {
    out[0] = a;
    out[1] = c;
  }
}

static unsigned grid_for(const Ctx* c, long long n) {
  long long b = (n + 255) / 256;
  long long cap = (long long)c->sm_count * 8;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_macro(const Ctx* c, const double* R, const double* W, double* T_half, double* T_E, cudaStream_t s) {
  macro_kernel<<<grid_for(c, c->total_cells), 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->total_cells, R, W, c->d_Vm,
                                                          c->d_VC, T_half, T_E);
  return cudaGetLastError();
}

static cudaError_t pcg(const Ctx* c, const double* rhs, cudaStream_t s) { return launch_mgpcg(c, rhs, s); }

// T_half += theta dT with dT solving the diffusion problem for the Newton source.
cudaError_t launch_newton(const Ctx* c, const double* T_n, double* T_half, const double* R, cudaStream_t s) {
  const unsigned gb = grid_for(c, c->total_cells);
  newton_rhs_kernel<<<gb, 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->total_cells, R, T_n, c->d_Vm, c->d_work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = pcg(c, c->d_work, s)) != cudaSuccess) return e;
  add_scaled_kernel<<<gb, 256, 0, s>>>(c->d_inst, c->n_inst, c->total_cells, T_half, c->d_pcg, c->d_theta,
                                       nullptr, T_half);
  return cudaGetLastError();
}

// Adjoint correction: out = half + theta m D^{-1}(half - lam) (transpose of the forward
// step T += theta D^{-1} m (T_half - T); D symmetric).
cudaError_t launch_adjoint_correction(const Ctx* c, const double* lam, const double* half, double* out,
                                      cudaStream_t s) {
  const unsigned gb = grid_for(c, c->total_cells);
  sub_kernel<<<gb, 256, 0, s>>>(c->total_cells, half, lam, c->d_work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if ((e = pcg(c, c->d_work, s)) != cudaSuccess) return e;
  add_scaled_kernel<<<gb, 256, 0, s>>>(c->d_inst, c->n_inst, c->total_cells, half, c->d_pcg, nullptr, c->d_theta_m, out);
  return cudaGetLastError();
}

cudaError_t launch_residual(const Ctx* c, const double* T0, const double* T1, double, double* out_dev, cudaStream_t s) {
  residual_stage1<<<RES_BLOCKS, 256, 0, s>>>(c->total_cells, T0, T1, c->d_red);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  residual_stage2<<<1, 256, 0, s>>>(c->d_red, out_dev);
  return cudaGetLastError();
}

// Sets ERR_PCG in the device error word when any instance's CG hit its iteration cap
// (lets an iteration run without a host round trip for the CG status).
__global__ void pcg_check_kernel(const int* iters, int n_inst, int* err) {
  for (int k = threadIdx.x; k < n_inst; k += blockDim.x)
    if (iters[k] < 0) atomicOr(err, ERR_PCG);
}

cudaError_t launch_pcg_check(const Ctx* c, cudaStream_t s) {
  pcg_check_kernel<<<1, 128, 0, s>>>(c->d_pcg_iters, c->n_inst, c->d_err);
  return cudaGetLastError();
}

// Statistical averaging (Sec. 4.4-4.5): the k-th sample x updates the running mean and the
// sum of squared deviations M2 (Welford's one-pass update; FP64).
__global__ void welford_kernel(long long total, const double* x, double* mean, double* m2, double inv_k) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const double d = x[i] - mean[i];
    const double mu = mean[i] + d * inv_k;
    mean[i] = mu;
    if (m2) m2[i] += d * (x[i] - mu);
  }
}

__global__ void scale_kernel(long long total, double* x, double a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    x[i] *= a;
}

cudaError_t launch_welford(const Ctx* c, const double* x, double* mean, double* m2, long long n, int k,
                           cudaStream_t s) {
  welford_kernel<<<grid_for(c, n), 256, 0, s>>>(n, x, mean, m2, 1.0 / (double)k);
  return cudaGetLastError();
}

cudaError_t launch_scale(const Ctx* c, double* x, long long n, double a, cudaStream_t s) {
  scale_kernel<<<grid_for(c, n), 256, 0, s>>>(n, x, a);
  return cudaGetLastError();
}

cudaError_t launch_axpy_grad(const Ctx* c, const double* at, const double* g, double* lam_half, cudaStream_t s) {
  add_kernel<<<grid_for(c, c->total_cells), 256, 0, s>>>(c->total_cells, at, g, lam_half);
  return cudaGetLastError();
}

cudaError_t launch_grad_source(const Ctx* c, const double* at, double* grad, cudaStream_t s) {
  div_kernel<<<grid_for(c, c->total_cells), 256, 0, s>>>(c->total_cells, at, c->d_m, grad);
  return cudaGetLastError();
}

}  // namespace iugkp
