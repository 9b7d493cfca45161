// FP64 replay of particles the staged FP32 sweep (or adjoint re-trace) deferred: a decision
// of the FP32 walk lay within rounding of the FP64 walk's (sweep_staged.cu). Method: arXiv
// 2506.09465 Sec. 3.1 (the straight flight between collisions) and Sec. 3.2 (candidates at
// the majorant rate, accepted with probability tau_maj / tau = sigma / sigma_max).
#pragma once

#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace iugkp {

// Path length to the next candidate in FP64: -ln(u) v tau_maj, the FP64 walk's expression.
__device__ __forceinline__ double path64(uint32_t word, double v, double tm) {
  return (-log(word_uniform<double>(word)) * v) * tm;
}

// The replay follows the particle's straight segment (its direction never changes) in FP64,
// analytically like the staged sweep: the faces of axis a reached before path length L are
// #{k >= 0 : t_a + k d_a < L}, the candidate's cell follows from those counts, and the
// segment leaves the domain at the first wall face. This takes the cell-by-cell FP64 walk's
// decisions except where a candidate lies within FP64 rounding of a face (relative 1e-16).

// #{k >= 0 : t + k d < L} with id = 1 / d (0 when d = inf).
__device__ __forceinline__ int count_before64(double L, double t, double id) {
  return L > t ? (int)ceil((L - t) * id) : 0;
}

// The FP64 segment of an emitted particle: per axis the first-face distance t, the distance
// per cell d and its inverse, the faces up to and including the wall m, and the first wall.
template <int DIM>
struct Seg64 {
  double t[DIM], d[DIM], id[DIM];
  int m[DIM];
  double tex;  // path length of the first wall face reached
  int ex;      // its axis (lower axis on ties)
  __device__ void init(const Walk<double, DIM>& wk, const InstDesc& in) {
    const double inf = __longlong_as_double(0x7ff0000000000000ll);
    tex = inf;
    ex = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      t[a] = wk.tmax[a];
      d[a] = wk.tdelta[a];
      id[a] = d[a] < inf ? 1.0 / d[a] : 0.0;
      m[a] = wk.step[a] > 0 ? in.n[a] - wk.idx[a] : wk.idx[a] + 1;
      const double tw = m[a] > 1 ? t[a] + (double)(m[a] - 1) * d[a] : t[a];
      if (tw < tex) {
        tex = tw;
        ex = a;
      }
    }
  }
};

// Follows the candidates of the segment in FP64 from the emission draws (Sec. 3.2): returns
// true at a real collision (counts fb[] before it) and false at the first wall. P::candidate
// (k, ci, cell) is told of every candidate, P::real(ci, cell) of the real one. *steps_out:
// candidates followed (the step budget applies).
template <int DIM, class P>
__device__ __forceinline__ int replay_candidates(const SweepArgs& A, const InstDesc& in, int inst, int b,
                                                 const Walk<double, DIM>& wk, const Seg64<DIM>& sg, Stream& st,
                                                 int* fb, P& pol) {
  const double tm = A.taumaj[(long long)inst * A.nb + b];
  const double vb = A.v[b];
  const long long bcbase = in.bc_off + (long long)b * in.ncells;
  uint32_t ua, ub;
  st.first_pair(ua, ub);
  double D = path64(ua, vb, tm);
  for (long long k = 0;; ++k) {
    if (k >= A.budget) return -1;
    if (D > sg.tex) return 0;  // the wall face comes first
    int cell = 0, stride = 1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      fb[a] = count_before64(D, sg.t[a], sg.id[a]);
      cell += (wk.idx[a] + wk.step[a] * fb[a]) * stride;
      stride *= in.n[a];
    }
    const long long ci = bcbase + cell;
    pol.candidate((int)k, ci, cell);
    if (word_uniform<double>(ub) < A.ratio64[ci]) {
      pol.real(ci, cell);
      return 1;
    }
    st.next_pair(ua, ub);
    D += path64(ua, vb, tm);
  }
}

}  // namespace iugkp
