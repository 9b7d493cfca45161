// Adjoint sweep: the transpose of the frozen-draw sweep map, applied by re-tracing
// every particle with the same draws and gathering at its real collision.
// With draws fixed the sweep is linear in the emission temperatures (arXiv 2506.09465,
// Sec. 2, Eq. "sum-g": a convex combination of neighbouring equilibria), so
//   T_half[i]    = sum over real collisions in cell i of w / (V m_i),
//   (A^T lam)[j] = sum over particles p of cell j of c_p lam[stop] / (V m_stop),
// c_p the particle's weight per unit emission temperature. No stored paths.
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"
#include "replay.cuh"

namespace iugkp {

template <typename Real>
__device__ __forceinline__ Real adj_path(uint32_t word, double v, double tm, float vtm_f);
template <>
__device__ __forceinline__ double adj_path<double>(uint32_t word, double v, double tm, float) {
  return (-log(word_uniform<double>(word)) * v) * tm;
}
template <>
__device__ __forceinline__ float adj_path<float>(uint32_t word, double, double, float vtm_f) {
  return -__logf(word_uniform<float>(word)) * vtm_f;
}

template <typename Real>
__device__ __forceinline__ Real adj_ratio(const SweepArgs& A, long long i);
template <>
__device__ __forceinline__ double adj_ratio<double>(const SweepArgs& A, long long i) { return A.ratio64[i]; }
template <>
__device__ __forceinline__ float adj_ratio<float>(const SweepArgs& A, long long i) { return A.ratio32[i]; }

// Emission of adjoint particle pid (every emitter, emitter-major numbering within its group):
// the walk, the stream, and the particle's weight per unit emission temperature.
template <typename Real, int DIM>
__device__ __forceinline__ void adjoint_emit(const SweepArgs& A, long long pid, const Group& G, Walk<Real, DIM>& wk,
                                             Stream& st, double& coefp, int& e) {
  const long long local = pid - G.first_particle;
  e = (int)(local / G.per_emitter);
  const int q = (int)(local - (long long)e * G.per_emitter);
  const InstDesc& in = A.inst[G.inst];
  const int b = G.band;
  if (G.kind == 0) {
    coefp = A.coef[in.bc_off + (long long)b * in.ncells + e];
    st.init(A.seed, in.inst_id, (uint32_t)b, A.epoch, (uint32_t)e, (uint32_t)q);
    emit_thermal<Real, DIM>(wk, st, in, e);
  } else {
    const int wl = G.kind - 1;
    coefp = A.wcoef[((long long)G.inst * A.nb + b) * 6 + wl];
    const int a = wl >> 1, side = wl & 1;
    const int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
    const int j1 = e % in.n[o1], j2 = e / in.n[o1];
    int f[3];
    f[a] = side ? in.n[a] : 0;
    f[o1] = j1;
    f[o2] = j2;
    const long long m0 = in.n[0] + (a == 0), m1 = in.n[1] + (a == 1);
    const long long face = in.fax_off[a] + f[0] + m0 * (f[1] + m1 * f[2]);
    st.init(A.seed, in.inst_id, (uint32_t)b, A.epoch, (uint32_t)(in.ncells + face), (uint32_t)q);
    emit_wall<Real, DIM>(wk, st, in, wl, j1, j2);
  }
}

// Re-traces particle pid and adds its contribution c_p lam[stop] / (V m_stop) to its emitter
// cell or wall.
template <typename Real, int DIM>
__device__ __forceinline__ void adjoint_particle(const SweepArgs& A, long long pid, int* err) {
  const int gi = find_group(A.groups, A.n_groups, pid);
  const Group G = A.groups[gi];
  const InstDesc& in = A.inst[G.inst];
  const int b = G.band;
  Walk<Real, DIM> wk;
  Stream st;
  double coefp;
  int e;
  adjoint_emit<Real, DIM>(A, pid, G, wk, st, coefp, e);
  const double tm = A.taumaj[(long long)G.inst * A.nb + b];
  const double vb = A.v[b];
  const float vtm_f = (float)(vb * tm);
  const long long bcbase = in.bc_off + (long long)b * in.ncells;
  const int stride[3] = {1, in.n[0], in.n[0] * in.n[1]};
  uint32_t ua, ub;
  st.first_pair(ua, ub);
  wk.D = adj_path<Real>(ua, vb, tm, vtm_f);
  long long steps = 0;
  double val = 0.0;
  for (;;) {
    if (++steps > A.budget) {
      atomicOr(err, ERR_BUDGET);
      return;
    }
    int a = 0;
    Real tmin = wk.tmax[0];
    if (DIM >= 2 && wk.tmax[1] < tmin) {
      a = 1;
      tmin = wk.tmax[1];
    }
    if (DIM >= 3 && wk.tmax[2] < tmin) {
      a = 2;
      tmin = wk.tmax[2];
    }
    if (wk.D <= tmin) {
      const long long ci = bcbase + wk.cell;
      if (word_uniform<Real>(ub) < adj_ratio<Real>(A, ci)) {
        const long long g = in.cell_off + wk.cell;
        val = coefp * A.lambda[g] * A.invVm[g];
        break;
      }
      st.next_pair(ua, ub);
      wk.D += adj_path<Real>(ua, vb, tm, vtm_f);
      continue;
    }
    const int stp = wk.step[a];
    wk.idx[a] += stp;
    if (wk.idx[a] < 0 || wk.idx[a] >= in.n[a]) return;  // absorbed by a wall: no gather
    wk.cell += stp * stride[a];
    wk.tmax[a] += wk.tdelta[a];
  }
  if (G.kind == 0) atomicAdd(&A.adj_out[in.cell_off + e], val);
  else atomicAdd(&A.adj_wall[in.wall_off + G.kind - 1], val);
}

template <typename Real, int DIM>
__global__ void __launch_bounds__(256) adjoint_kernel(SweepArgs A) {
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  for (long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x; pid < A.total_particles; pid += nthreads)
    adjoint_particle<Real, DIM>(A, pid, A.err);
}

// The gather of a replayed adjoint particle: c_p lam / (V m) at its real collision.
struct AdjointGather {
  const SweepArgs& A;
  const InstDesc& in;
  double coefp, val;
  __device__ void candidate(int, long long, int) {}
  __device__ void real(long long, int cell) {
    const long long g = in.cell_off + cell;
    val = coefp * A.lambda[g] * A.invVm[g];
  }
};

// FP64 re-trace (analytic along the straight segment, replay.cuh) of the particles the staged
// adjoint re-trace deferred; the forward sweep defers the same particles. One thread per
// entry; entry x: the staged index, particle q of emitter e taken q-major within its group.
template <int DIM>
__global__ void __launch_bounds__(128) adjoint_replay_kernel(SweepArgs A, const uint2* defer, const unsigned* defer_n,
                                                             unsigned defer_cap) {
  const unsigned n = min(*defer_n, defer_cap);
  // warp j of every block numbered before warp j + 1 of any, 32 entries each (as in
  // replay_kernel): the short queue's work is spread over the SMs
  const unsigned wid = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  for (unsigned i = 32u * wid + (threadIdx.x & 31); i < n; i += gridDim.x * blockDim.x) {
    const unsigned pid = defer[i].x;
    const Group G = A.groups[find_group(A.groups, A.n_groups, (long long)pid)];
    const InstDesc& in = A.inst[G.inst];
    const unsigned local = pid - (unsigned)G.first_particle;
    const int q = (int)(local / (unsigned)G.n_emitters);
    int e0 = (int)(local - (unsigned)q * (unsigned)G.n_emitters);
    if (G.perm_off >= 0) e0 = A.perm[G.perm_off + e0];  // the staged visiting order
    Walk<double, DIM> wk;
    Stream st;
    double coefp;
    int e;
    adjoint_emit<double, DIM>(A, G.first_particle + (long long)e0 * G.per_emitter + q, G, wk, st, coefp, e);
    Seg64<DIM> sg;
    sg.init(wk, in);
    AdjointGather pol{A, in, coefp, 0.0};
    int fb[DIM];
    const int res = replay_candidates<DIM>(A, in, G.inst, G.band, wk, sg, st, fb, pol);
    if (res < 0) {
      atomicOr(A.err, ERR_BUDGET);
      continue;
    }
    if (res == 0) continue;  // absorbed by a wall: no gather
    if (G.kind == 0) atomicAdd(&A.adj_out[in.cell_off + e], pol.val);
    else atomicAdd(&A.adj_wall[in.wall_off + G.kind - 1], pol.val);
  }
}

cudaError_t launch_adjoint_replay(const Ctx* c, const SweepArgs& a, cudaStream_t s) {
  const int blocks = c->sm_count * 4;
  switch (c->dim) {
    case 1: adjoint_replay_kernel<1><<<blocks, 128, 0, s>>>(a, c->d_defer, c->d_defer_n, c->defer_cap); break;
    case 2: adjoint_replay_kernel<2><<<blocks, 128, 0, s>>>(a, c->d_defer, c->d_defer_n, c->defer_cap); break;
    default: adjoint_replay_kernel<3><<<blocks, 128, 0, s>>>(a, c->d_defer, c->d_defer_n, c->defer_cap); break;
  }
  return cudaGetLastError();
}

template <typename Real, int DIM>
static cudaError_t launch_adj(const Ctx* c, const SweepArgs& a, cudaStream_t s) {
  long long blocks = (a.total_particles + 255) / 256;
  long long cap = (long long)c->sm_count * 32;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  adjoint_kernel<Real, DIM><<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adjoint(const Ctx* c, const SweepArgs& a, cudaStream_t s) {
  const bool fp32 = c->opt.precision == IUGKP_TRACK_FP32;
  switch (c->dim) {
    case 1: return fp32 ? launch_adj<float, 1>(c, a, s) : launch_adj<double, 1>(c, a, s);
    case 2: return fp32 ? launch_adj<float, 2>(c, a, s) : launch_adj<double, 2>(c, a, s);
    default: return fp32 ? launch_adj<float, 3>(c, a, s) : launch_adj<double, 3>(c, a, s);
  }
}

}  // namespace iugkp
