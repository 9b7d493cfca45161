// Forward sweep kernels: emission, cell-by-cell walk, null collisions and tallies.
// arXiv 2506.09465 Sec. 3.1 (steps (1)-(3)) and Sec. 3.2 (steps (1)-(6), with the
// candidate chain of a particle completed inside one sweep).
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace iugkp {

// Per-thread event counts, reduced once per warp at the end of a kernel.
struct Counts {
  unsigned long long v[CNT_N];
};

__device__ __forceinline__ void flush_counts(Counts& c, unsigned long long* out) {
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) {
    unsigned long long x = c.v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&out[k], x);
  }
}

// Path length to the next candidate: -ln(u) v tau_maj (Sec. 3.1 inverse sampling with
// the majorant time scale of Eq. "truncated-tf").
template <typename Real>
__device__ __forceinline__ Real candidate_path(uint32_t word, double v, double tm, float vtm_f);
template <>
__device__ __forceinline__ double candidate_path<double>(uint32_t word, double v, double tm, float) {
  return (-log(word_uniform<double>(word)) * v) * tm;
}
template <>
__device__ __forceinline__ float candidate_path<float>(uint32_t word, double, double, float vtm_f) {
  return -__logf(word_uniform<float>(word)) * vtm_f;
}

template <typename Real>
__device__ __forceinline__ Real accept_ratio(const SweepArgs& A, long long i);
template <>
__device__ __forceinline__ double accept_ratio<double>(const SweepArgs& A, long long i) { return A.ratio64[i]; }
template <>
__device__ __forceinline__ float accept_ratio<float>(const SweepArgs& A, long long i) { return A.ratio32[i]; }

// Emits particle `pid` of the sweep. Returns false when its weight is zero (nothing to
// trace: its tallies would all be zero). On true, w, the walk and the stream are set.
// EMIT_F: a wall particle's power enters the net power of its boundary face here.
template <typename Real, int DIM, bool EMIT_F = true>
__device__ __forceinline__ bool emit_particle(const SweepArgs& A, long long pid, int& gi, double& w,
                                              Walk<Real, DIM>& wk, Stream& st) {
  gi = find_group(A.groups, A.n_groups, pid);
  const Group G = A.groups[gi];
  const long long local = pid - G.first_particle;
  const int e = (int)(local / G.per_emitter);
  const int q = (int)(local - (long long)e * G.per_emitter);
  const InstDesc& in = A.inst[G.inst];
  const int b = G.band;
  if (G.kind == 0) {
    double Te = A.T[in.cell_off + e];
    if (A.srcshift) Te += A.srcshift[in.cell_off + e];
    w = A.coef[in.bc_off + (long long)b * in.ncells + e] * Te;
    if (w == 0.0) return false;
    st.init(A.seed, in.inst_id, (uint32_t)b, A.epoch, (uint32_t)e, (uint32_t)q);
    emit_thermal<Real, DIM>(wk, st, in, e);
  } else {
    const int wl = G.kind - 1;
    w = A.wcoef[((long long)G.inst * A.nb + b) * 6 + wl] * A.wallTf[in.bface_off + in.wface_off[wl] + e];
    if (w == 0.0) return false;
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
    // Power entering through the boundary face, +axis sign convention.
    if (EMIT_F && A.F) atomicAdd(&A.F[in.face_off + face], side ? -w : w);
  }
  return true;
}

// The walk of one emitted particle: cell by cell through null candidates to a real collision
// or a wall (Sec. 3.1 step (2), Sec. 3.2). The tallies are the policy's:
//   P::candidate(k, ci)     candidate k (0, 1, ...) in (band, cell) index ci
//   P::real(ci, cell)       real collision in that cell
//   P::cross(a, step, face) crossing of the face (instance index) normal to axis a
//   P::exit(a, step, face)  the crossed face was a wall's: the particle is absorbed there
template <typename Real, int DIM, class P>
__device__ __forceinline__ void walk_particle(const SweepArgs& A, const InstDesc& in, int inst, int b, Walk<Real, DIM>& wk,
                                              Stream& st, Counts& cnt, P& pol) {
  const double tm = A.taumaj[(long long)inst * A.nb + b];
  const double vb = A.v[b];
  const float vtm_f = (float)(vb * tm);
  const long long bcbase = in.bc_off + (long long)b * in.ncells;
  const int stride[3] = {1, in.n[0], in.n[0] * in.n[1]};
  uint32_t ua, ub;
  st.next_pair(ua, ub);
  wk.D = candidate_path<Real>(ua, vb, tm, vtm_f);
  long long steps = 0;
  int k = 0;
  for (;;) {
    if (++steps > A.budget) {
      cnt.v[CNT_DROPPED] += 1;
      atomicOr(A.err, ERR_BUDGET);
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
      // Candidate collision in the current cell (Sec. 3.2): W tally, then accept with
      // probability tau_maj / tau(x).
      const long long ci = bcbase + wk.cell;
      if (pol.candidate(k++, ci)) cnt.v[CNT_CANDIDATES] += 1;
      if (word_uniform<Real>(ub) < accept_ratio<Real>(A, ci)) {
        cnt.v[CNT_REAL] += 1;
        pol.real(ci, wk.cell);
        return;
      }
      st.next_pair(ua, ub);
      wk.D += candidate_path<Real>(ua, vb, tm, vtm_f);
      continue;
    }
    const int stp = wk.step[a];
    const long long face = face_index<DIM>(in, wk.idx, wk.cell, a, stp);
    pol.cross(a, stp, face);
    wk.idx[a] += stp;
    if (wk.idx[a] < 0 || wk.idx[a] >= in.n[a]) {
      cnt.v[CNT_WALL_EXITS] += 1;
      pol.exit(a, stp, face);
      return;
    }
    wk.cell += stp * stride[a];
    wk.tmax[a] += wk.tdelta[a];
    cnt.v[CNT_CROSSINGS] += 1;
  }
}

// Tallies of the plain sweep: every candidate, real collision, face and wall, each a global
// FP64 atomic.
struct PlainTally {
  const SweepArgs& A;
  const InstDesc& in;
  double w, wt;  // weight; weight x tau_maj (the candidate estimator W)
  __device__ bool candidate(int, long long ci) {
    if (A.W) atomicAdd(&A.W[ci], wt);
    return true;
  }
  __device__ void real(long long ci, int) { atomicAdd(&A.R[ci], w); }
  __device__ void cross(int, int stp, long long face) {
    if (A.F) atomicAdd(&A.F[in.face_off + face], stp > 0 ? w : -w);
  }
  __device__ void exit(int a, int stp, long long) {
    if (A.wall) atomicAdd(&A.wall[in.wall_off + 2 * a + (stp > 0 ? 1 : 0)], w);
  }
};

// One particle from emission to absorption (one thread, global FP64 atomics).
template <typename Real, int DIM>
__device__ __forceinline__ void run_particle(const SweepArgs& A, long long pid, Counts& cnt) {
  int gi;
  double w;
  Walk<Real, DIM> wk;
  Stream st;
  if (!emit_particle<Real, DIM>(A, pid, gi, w, wk, st)) return;
  const Group G = A.groups[gi];
  const InstDesc& in = A.inst[G.inst];
  cnt.v[CNT_FLIGHTS] += 1;
  PlainTally pol{A, in, w, w * A.taumaj[(long long)G.inst * A.nb + G.band]};
  walk_particle<Real, DIM>(A, in, G.inst, G.band, wk, st, cnt, pol);
}

// Tallies of a particle the staged sweep left to this FP64 replay: exactly those the staged
// sweep would have made for it. W is summed as w (the staged sweep scales it by tau_maj
// afterwards), and only from candidate k_done on (the earlier ones are tallied already).
// Faces: those normal to the axes the staged sweep tallies (x in 1D; x and y in 3D; x in 2D,
// or y for a y-group particle of a two-group instance), the wall faces among them included;
// an exit through the low wall of an untallied axis goes to that wall's face (one-group
// instances) or to the group's exit tally GX (two-group); a y-group particle's real
// collision also enters its group balance DY. Emission needs nothing: the staged sweep and
// its post-passes account for it.
struct ReplayTally {
  const SweepArgs& A;
  const StagedArgs& S;
  const InstDesc& in;
  double w;
  int k_done, dim;
  bool two, yg;
  __device__ bool tallied(int a) const { return dim == 1 || (two ? a == (yg ? 1 : 0) : a < dim - 1); }
  __device__ bool candidate(int k, long long ci) {
    if (k < k_done) return false;
    if (A.W) atomicAdd(&A.W[ci], w);
    return true;
  }
  __device__ void real(long long ci, int cell) {
    atomicAdd(&A.R[ci], w);
    if (two && yg) atomicAdd(&S.DY[in.cell_off + cell], w);
  }
  __device__ void cross(int a, int stp, long long face) {
    if (A.F && tallied(a)) atomicAdd(&A.F[in.face_off + face], stp > 0 ? w : -w);
  }
  __device__ void exit(int a, int stp, long long face) {
    if (!A.F || tallied(a) || stp > 0) return;
    if (two) {
      // the low wall's face index within its wall: the column (x-group, low y-wall) or the
      // row (y-group, low x-wall)
      const long long j = yg ? (face - in.fax_off[0]) / (in.n[0] + 1) : face - in.fax_off[1];
      atomicAdd(&S.GX[in.bface_off + in.wface_off[yg ? 0 : 2] + j], -w);
    } else {
      atomicAdd(&A.F[in.face_off + face], -w);
    }
  }
};

// FP64 replay of the particles the staged sweep deferred (one thread per queue entry). The
// entry holds the staged sweep's forward index (particle q of emitter e, q-major within its
// group) and the candidates it tallied before the decision it could not take in FP32.
template <int DIM>
__global__ void __launch_bounds__(128) replay_kernel(SweepArgs A, StagedArgs S) {
  Counts cnt;
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) cnt.v[k] = 0;
  const unsigned n = min(*S.defer_n, S.defer_cap);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const uint2 ent = S.defer[i];
    const int gi = find_group(A.groups, A.n_groups, (long long)ent.x);
    const Group G = A.groups[gi];
    const InstDesc& in = A.inst[G.inst];
    const unsigned local = ent.x - (unsigned)G.first_particle;
    const int q = (int)(local / (unsigned)G.n_emitters);
    const int e = (int)(local - (unsigned)q * (unsigned)G.n_emitters);
    const long long plain = G.first_particle + (long long)e * G.per_emitter + q;
    int gj;
    double w;
    Walk<double, DIM> wk;
    Stream st;
    if (!emit_particle<double, DIM, false>(A, plain, gj, w, wk, st)) continue;
    const bool two = DIM == 2 && A.F && S.window[G.inst].x == 0 && (long long)S.window[G.inst].y == in.nfaces;
    ReplayTally pol{A, S, in, w, (int)(ent.y >> 1), DIM, two, (ent.y & 1u) != 0};
    walk_particle<double, DIM>(A, in, G.inst, G.band, wk, st, cnt, pol);
  }
  flush_counts(cnt, A.counters);
}

cudaError_t launch_replay(const Ctx* c, const SweepArgs& a, const StagedArgs& S, cudaStream_t s) {
  const int blocks = c->sm_count * 4;
  switch (c->dim) {
    case 1: replay_kernel<1><<<blocks, 128, 0, s>>>(a, S); break;
    case 2: replay_kernel<2><<<blocks, 128, 0, s>>>(a, S); break;
    default: replay_kernel<3><<<blocks, 128, 0, s>>>(a, S); break;
  }
  return cudaGetLastError();
}

template <typename Real, int DIM>
__global__ void __launch_bounds__(256) sweep_plain_kernel(SweepArgs A) {
  Counts cnt;
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) cnt.v[k] = 0;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  for (long long pid = (long long)blockIdx.x * blockDim.x + threadIdx.x; pid < A.total_particles; pid += nthreads)
    run_particle<Real, DIM>(A, pid, cnt);
  flush_counts(cnt, A.counters);
}

template <typename Real, int DIM>
static cudaError_t launch_plain(const Ctx* c, const SweepArgs& a, cudaStream_t s) {
  long long blocks = (a.total_particles + 255) / 256;
  long long cap = (long long)c->sm_count * 32;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  sweep_plain_kernel<Real, DIM><<<(unsigned)blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const Ctx* c, const SweepArgs& a, cudaStream_t s) {
  const bool fp32 = c->opt.precision == IUGKP_TRACK_FP32;
  switch (c->dim) {
    case 1: return fp32 ? launch_plain<float, 1>(c, a, s) : launch_plain<double, 1>(c, a, s);
    case 2: return fp32 ? launch_plain<float, 2>(c, a, s) : launch_plain<double, 2>(c, a, s);
    default: return fp32 ? launch_plain<float, 3>(c, a, s) : launch_plain<double, 3>(c, a, s);
  }
}

}  // namespace iugkp
