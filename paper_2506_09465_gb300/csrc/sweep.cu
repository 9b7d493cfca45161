// Forward sweep kernels: emission, cell-by-cell walk, null collisions and tallies.
// arXiv 2506.09465 Sec. 3.1 (steps (1)-(3)) and Sec. 3.2 (steps (1)-(6), with the
// candidate chain of a particle completed inside one sweep).
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"
#include "replay.cuh"

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
  st.first_pair(ua, ub);
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

// Deposit tallies of a replayed particle: W as w (the staged sweep scales it by tau_maj
// afterwards, or sets it to tau_maj R in bands whose every candidate is real: all_real), from
// candidate k_done on (the earlier ones were tallied by the staged sweep); R, and the y-group
// balance DY for a y-group particle of a two-group instance.
struct ReplayDeposits {
  const SweepArgs& A;
  const StagedArgs& S;
  const InstDesc& in;
  double w;
  int k_done;
  bool ydy;
  bool all_real;
  Counts& cnt;
  __device__ void candidate(int k, long long ci, int) {
    if (k < k_done) return;
    cnt.v[CNT_CANDIDATES] += 1;
    if (A.W && !all_real) atomicAdd(&A.W[ci], w);
  }
  __device__ void real(long long ci, int cell) {
    cnt.v[CNT_REAL] += 1;
    atomicAdd(&A.R[ci], w);
    if (ydy) atomicAdd(&S.DY[in.cell_off + cell], w);
  }
};

// Face index within the instance of face coordinate f along axis a, cell coordinates c[] on
// the other axes.
__device__ __forceinline__ long long face_at(const InstDesc& in, int a, int f, const int* c) {
  if (a == 0) return in.fax_off[0] + f + (long long)(in.n[0] + 1) * (c[1] + (long long)in.n[1] * c[2]);
  if (a == 1) return in.fax_off[1] + c[0] + (long long)in.n[0] * (f + (long long)(in.n[1] + 1) * c[2]);
  return in.fax_off[2] + c[0] + (long long)in.n[0] * (c[1] + (long long)in.n[1] * f);
}

__device__ __forceinline__ double shfl_d(double x, int src) {
  return __hiloint2double(__shfl_sync(0xffffffffu, __double2hiint(x), src),
                          __shfl_sync(0xffffffffu, __double2loint(x), src));
}

// One thread per queue entry follows the particle's candidates in FP64 and makes its deposit
// tallies; then the warp tallies the face items of its particles together, one particle at a
// time (its segment broadcast from its lane), the lanes taking successive items. Faces
// tallied: those the staged sweep tallies for this particle (x in 1D; x and y in 3D; x in 2D,
// or y for a y-group particle of a two-group instance), the wall faces among them included;
// an exit through the low wall of an untallied axis goes to that wall's face (one-group
// instances) or to the group's exit tally GX (two-group). Emission needs nothing: the staged
// sweep and its post-passes account for it.
constexpr unsigned REPLAY_PER_WARP = 32;  // queue entries per warp and round

template <int DIM>
__global__ void __launch_bounds__(256) replay_kernel(SweepArgs A, StagedArgs S) {
  Counts cnt;
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) cnt.v[k] = 0;
  const int lane = threadIdx.x & 31;
  const unsigned n = min(*S.defer_n, S.defer_cap);
  // Warp j of block b is warp a = j G + b (G blocks: warp j of every block comes before warp
  // j + 1 of any), and warp a takes entries E a .. E a + E - 1 (E = REPLAY_PER_WARP; then E (a
  // + W) .., W warps in the grid). The queue is short: numbered b 8 + j, the warps that got
  // work were all in the first few blocks, on a few SMs (measured: the busiest SM active 3.6
  // times as long as the average); this way the first warps to get work are the first warp of
  // every block.
  const unsigned W = gridDim.x * blockDim.x >> 5;
  const unsigned wid = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  // all lanes of a warp run the same rounds (the face items are tallied by the whole warp)
  for (unsigned i0 = REPLAY_PER_WARP * wid; i0 < n; i0 += REPLAY_PER_WARP * W) {
    const unsigned i = lane < (int)REPLAY_PER_WARP ? i0 + lane : n;
    // the lane's particle, kept for the face items
    int kinst = 0, ex = 0, tall = 0;  // instance, exit axis (-1: real collision), tallied axes (bits)
    double w = 0.0;
    double t[3] = {0, 0, 0}, d[3] = {0, 0, 0}, id[3] = {0, 0, 0};
    int idx[3] = {0, 0, 0}, step[3] = {1, 1, 1}, m[3] = {1, 1, 1}, items[3] = {0, 0, 0};
    if (i < n) {
      const uint2 ent = S.defer[i];
      const Group G = A.groups[find_group(A.groups, A.n_groups, (long long)ent.x)];
      const InstDesc& in = A.inst[G.inst];
      const unsigned local = ent.x - (unsigned)G.first_particle;
      const int q = (int)(local / (unsigned)G.n_emitters);
      int e = (int)(local - (unsigned)q * (unsigned)G.n_emitters);
      if (G.perm_off >= 0) e = A.perm[G.perm_off + e];  // the staged visiting order
      int gj;
      Walk<double, DIM> wk;
      Stream st;
      if (emit_particle<double, DIM, false>(A, G.first_particle + (long long)e * G.per_emitter + q, gj, w, wk, st)) {
        Seg64<DIM> sg;
        sg.init(wk, in);
        const bool two = DIM == 2 && A.F && S.window[G.inst].x == 0 && (long long)S.window[G.inst].y == in.nfaces;
        const bool yg = two && (ent.y & 1u);
        ReplayDeposits pol{A, S, in, w, (int)(ent.y >> 1), yg,
                           A.all_real[(long long)G.inst * A.nb + G.band] != 0, cnt};
        int fb[DIM];
        const int res = replay_candidates<DIM>(A, in, G.inst, G.band, wk, sg, st, fb, pol);
        if (res < 0) {
          cnt.v[CNT_DROPPED] += 1;
          atomicOr(A.err, ERR_BUDGET);
        } else {
          // interior faces crossed per axis; at a wall the exit axis's are all of them
          const bool exit = res == 0;
          int c[3] = {0, 0, 0};
#pragma unroll
          for (int a = 0; a < DIM; ++a) {
            c[a] = exit ? (a == sg.ex ? sg.m[a] - 1 : min(count_before64(sg.tex, sg.t[a], sg.id[a]), sg.m[a] - 1))
                        : fb[a];
            cnt.v[CNT_CROSSINGS] += c[a];
            t[a] = sg.t[a];
            d[a] = sg.d[a];
            id[a] = sg.id[a];
            idx[a] = wk.idx[a];
            step[a] = wk.step[a];
            m[a] = sg.m[a];
          }
          if (exit) cnt.v[CNT_WALL_EXITS] += 1;
          kinst = G.inst;
          ex = exit ? sg.ex : -1;
          if (A.F) {
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
              const bool ta = DIM == 1 || (two ? a == (yg ? 1 : 0) : a < DIM - 1);
              if (ta) {
                tall |= 1 << a;
                items[a] = c[a] + (exit && sg.ex == a ? 1 : 0);
              }
            }
            if (exit && !((tall >> sg.ex) & 1) && wk.step[sg.ex] < 0) {
              // exit through the low wall of an untallied axis
              int cc[3] = {0, 0, 0};
#pragma unroll
              for (int a = 0; a < DIM; ++a) cc[a] = wk.idx[a] + wk.step[a] * c[a];
              if (two) {
                const int j = sg.ex == 1 ? cc[0] : cc[1];  // the low y-wall's column or the low x-wall's row
                atomicAdd(&S.gx()[in.bface_off + in.wface_off[sg.ex == 1 ? 2 : 0] + j], -w);
              } else {
                atomicAdd(&A.F[in.face_off + face_at(in, sg.ex, 0, cc)], -w);
              }
            }
          }
        }
      }
    }
    // face items, particle by particle: item j along the tallied axis p is its j-th face, at
    // path length t_p + j d_p; the cell there on each other axis follows from its face count
    unsigned pend = __ballot_sync(0xffffffffu, tall != 0);
    while (pend) {
      const int src = __ffs(pend) - 1;
      pend &= pend - 1;
      const int k = __shfl_sync(0xffffffffu, kinst, src);
      const InstDesc& in = A.inst[k];
      const double ws = shfl_d(w, src);
      const int tl = __shfl_sync(0xffffffffu, tall, src);
      double ts[3], ds[3], is[3];
      int xs[3], ss[3], ms[3], ns[3];
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        ts[a] = shfl_d(t[a], src);
        ds[a] = shfl_d(d[a], src);
        is[a] = shfl_d(id[a], src);
        xs[a] = __shfl_sync(0xffffffffu, idx[a], src);
        ss[a] = __shfl_sync(0xffffffffu, step[a], src);
        ms[a] = __shfl_sync(0xffffffffu, m[a], src);
        ns[a] = __shfl_sync(0xffffffffu, items[a], src);
      }
#pragma unroll
      for (int p = 0; p < DIM; ++p) {
        if (!((tl >> p) & 1)) continue;
        const double sgn = ss[p] > 0 ? ws : -ws;
        for (int j = lane; j < ns[p]; j += 32) {
          const double T = ts[p] + (double)j * ds[p];
          int cc[3] = {0, 0, 0};
#pragma unroll
          for (int a = 0; a < DIM; ++a)
            if (a != p) cc[a] = xs[a] + ss[a] * min(count_before64(T, ts[a], is[a]), ms[a] - 1);
          const int f = ss[p] > 0 ? xs[p] + 1 + j : xs[p] - j;
          atomicAdd(&A.F[in.face_off + face_at(in, p, f, cc)], sgn);
        }
      }
    }
    (void)ex;
  }
  flush_counts(cnt, A.counters);
}

cudaError_t launch_replay(const Ctx* c, const SweepArgs& a, const StagedArgs& S, cudaStream_t s) {
  const int blocks = c->sm_count * 8;
  switch (c->dim) {
    case 1: replay_kernel<1><<<blocks, 256, 0, s>>>(a, S); break;
    case 2: replay_kernel<2><<<blocks, 256, 0, s>>>(a, S); break;
    default: replay_kernel<3><<<blocks, 256, 0, s>>>(a, S); break;
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
