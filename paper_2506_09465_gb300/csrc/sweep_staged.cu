// Fast forward sweep and adjoint re-trace: FP32 walk, persistent blocks (a pass-synchronous
// kernel for 2D, a per-lane-refill kernel for every dimension), face tallies staged in
// shared memory in fixed point. Same method and draws as the plain sweep
// (arXiv 2506.09465 Sec. 3.1 steps (1)-(3), Sec. 3.2 null collisions); only the
// arithmetic precision of the walk and the way tallies are accumulated differ.
//
// Face tallies:
//  * faces normal to x are accumulated in a shared-memory copy of the instance's x-faces
//    (all of them when they fit, else a centred run), as integers in units of
//    q = w_max 2^-26 (exact and independent of the order of the additions): 32-bit words
//    (native shared-memory atomics, about five times the rate of 64-bit ones) whose rare
//    wrap-arounds add +-2^32 q to the FP64 face at once, flushed to the FP64 array when the
//    block leaves the instance; x-faces outside the window take global atomics;
//  * faces normal to the last axis (y in 2D, z in 3D) are not tallied, except on the low
//    boundary: every particle conserves power, so in every cell the net inflow equals the
//    absorbed minus emitted power, and the last-axis faces follow exactly by a prefix sum
//    along each column (derive_last_axis_kernel);
//  * in 3D the y-faces are tallied with global FP64 atomics;
//  * 2D instances whose faces all fit the window use two-group tallies instead: a particle
//    tallies only the faces normal to the axis it crosses less often, and each group's
//    other faces follow from that group's own per-cell balance (derive_two_group_kernel,
//    assemble_two_group_kernel);
//  * a warp tallies the face items of the particles that ended together: in the
//    pass-synchronous kernel each lane takes segments of 8 items of one list, dealt
//    round-robin; in the per-lane-refill kernel each lane takes one contiguous chunk of the
//    concatenated item lists;
//  * nothing is tallied per particle for the walls: the power a wall emits enters through
//    its faces deterministically (N particles of known weight per face), and the power it
//    absorbs is its emission plus the outward net flux through its faces
//    (boundary_emission_kernel, wall_absorbed_kernel).
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "internal.h"
#include "staged.h"

namespace iugkp {

namespace {

struct LCounts {
  unsigned v[CNT_N];  // per thread and launch: far below 2^32
};

__device__ __forceinline__ void flush_lcounts(LCounts& c, unsigned long long* out) {
  if (!out) return;
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) {
    unsigned long long x = c.v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&out[k], x);
  }
}

// Register-resident path state. The direction does not change at null collisions, so the
// path from emission to the end (real collision or wall) is one straight segment: i_a is
// the emission cell, t_a the path length at which the first face normal to axis a is
// reached, d_a the path length per cell along a (+inf when s_a = 0), so the k-th face along
// a is reached at t_a + k d_a. D: path length of the current candidate collision;
// tex: path length at which the segment leaves the domain.
struct PW {
  int i0, i1, i2;
  int s0, s1, s2;
  float t0, t1, t2;
  float d0, d1, d2;
  float D, tex;
};

__device__ __forceinline__ void axis_init(float s, float xi, float h, float& t, float& d, int& st) {
  const float as = fabsf(s);
  st = s > 0.f ? 1 : -1;
  d = __fdividef(h, as);  // +inf when s = 0
  t = (s > 0.f ? 1.f - xi : xi) * d;
}

// ceil(max(u, 0)) for u < 2^23 without a float-to-integer conversion: adding 2^23 with
// rounding upwards lands on 2^23 + ceil(u), whose bits minus those of 2^23 are the count.
__device__ __forceinline__ int ceil_count(float u) {
  return __float_as_int(__fadd_ru(fmaxf(u, 0.f), 8388608.f)) - 0x4B000000;
}

// i as a float for 0 <= i < 2^23, placed in the mantissa of 2^23 (no conversion instruction).
__device__ __forceinline__ float small_int_float(int i) { return __int_as_float(0x4B000000 | i) - 8388608.f; }

// Faces normal to one axis reached before path length L: #{k >= 0 : t + k d < L}.
__device__ __forceinline__ int faces_before(float L, float t, float d) {
  return L > t ? ceil_count(__fdividef(L - t, d)) : 0;
}

// Faces up to and including the wall along one axis, and the path length of the wall face.
__device__ __forceinline__ int faces_to_wall(int i, int s, int n) { return s > 0 ? n - i : i + 1; }
__device__ __forceinline__ float axis_exit(int i, int s, int n, float t, float d) {
  const int m = faces_to_wall(i, s, n);
  return m > 1 ? fmaf(small_int_float(m - 1), d, t) : t;
}

__device__ __forceinline__ int clampi(int v, int n) { return min(max(v, 0), n - 1); }

// ---- FP32 decisions checked against the FP64 walk ----
// The FP32 walk and the FP64 walk follow each particle with the same draws, so their path
// lengths differ by rounding only, and a decision taken in FP32 is the FP64 walk's unless the
// FP32 value lies within a bound of the decision's boundary: a face (the count of faces before
// a candidate along an axis, hence its cell), the first wall (a candidate or an absorption),
// the acceptance ratio. A particle with such a decision is not tallied further: it goes to a
// queue that the FP64 walk replays after the sweep (replay_kernel, adjoint_replay_kernel).
// Path-length bounds, FP32 against FP64:
//  * a face count's quotient u = (D - t) / d, times d: TIE_REL (D + d) + eD, TIE_REL covering
//    the rounding of the direction (sqrtf, sincospif, products), cell size, first-face
//    distance, quotient (__fdividef) and difference, about 2^-19.4 in all, taken as 2^-18;
//    the wall distance tex likewise within TIE_REL tex;
//  * eD bounds |D32 - D64|: per flight TIE_LOG_ABS v tau_maj + TIE_LOG_REL l for the fast
//    logarithm, the FP32 v tau_maj and the product's rounding, plus TIE_SUM D for each
//    addition to D. The logarithm's error over all 2^23 uniforms the walk draws is measured
//    (walk_bounds_kernel) at about a third of its share of this allowance.
// The acceptance ratio in FP32 is within 2^-24 of the FP64 ratio (both below 1).
constexpr float TIE_REL = 0x1p-18f;
constexpr float TIE_LOG_ABS = 0x1p-22f;
constexpr float TIE_LOG_REL = 0x1p-20f;
constexpr float TIE_SUM = 0x1p-23f;
constexpr float TIE_ACC = 0x1p-24f;

// Tie bits of one axis for the count n = faces_before(D, t, d): bit sh when D lies within the
// bound (base = TIE_REL D + eD, plus TIE_REL d) below a face, so that the FP64 walk may count
// one face more; bit sh + 1 when within it above one (one fewer). None when d = inf (NaN).
__device__ __forceinline__ unsigned tie_bits(float D, float t, float d, float base, int n, int sh) {
  const float u = __fdividef(D - t, d);
  const float fr = small_int_float(n) - u;  // up to the next face, in cells: [0, 1]
  const float tol = fmaf(TIE_REL, d, base);
  if (fr * d <= tol) return 1u << sh;
  if ((1.f - fr) * d <= tol && n > 0) return 2u << sh;
  return 0u;
}

// faces_before, and in `near` whether D lies within the bound of a face of this axis (either
// side; the direction is not needed when every candidate is real).
__device__ __forceinline__ int count_near(float D, float t, float d, float base, bool& near) {
  const float u = __fdividef(D - t, d);
  const float c = __fadd_ru(fmaxf(u, 0.f), 8388608.f);  // 2^23 + ceil(max(u, 0))
  const float fr = (c - 8388608.f) - u;
  near |= fminf(fr, 1.f - fr) * d <= fmaf(TIE_REL, d, base);
  return __float_as_int(c) - 0x4B000000;
}

// Axis a's bit of `hit` when the count one more than n reaches the wall (m faces to it).
__device__ __forceinline__ unsigned tie_hits_wall(unsigned tie, int a, int n, int m) {
  return ((tie >> (2 * a)) & 1u) && n + 1 >= m ? 1u << (2 * a) : 0u;
}

// A candidate flagged near faces (tie, two bits per axis) may lie, in the FP64 walk, in a cell
// across the flagged faces. True when every such cell rejects it by more than the ratio's
// rounding: the FP64 walk then goes on identically, and only the cell of this candidate's W
// may differ. False when an alternative lies beyond a wall (hit) or any cell may accept.
// st_a: the cell index step of one more face along axis a (s_a times the axis stride).
__device__ __forceinline__ bool all_reject(const float* ratio, int ncells, int cell, unsigned tie, unsigned hit, int st0,
                                           int st1, int st2, float u) {
  if (tie & hit) return false;
#pragma unroll 1
  for (unsigned k = 0; k < 8u; ++k) {
    int c = cell;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (!((k >> a) & 1u)) continue;
      const unsigned t = (tie >> (2 * a)) & 3u;
      const int st = a == 0 ? st0 : (a == 1 ? st1 : st2);
      ok = ok && t != 0u;
      c += t == 1u ? st : -st;
    }
    if (!ok) continue;
    if (c < 0 || c >= ncells || !(u - ratio[c] >= TIE_ACC)) return false;
  }
  return true;
}

// Queues a particle for the FP64 replay: forward index and (candidates tallied << 1) | group.
__device__ __forceinline__ void defer_particle(const StagedArgs& S, unsigned pid, unsigned meta) {
  const unsigned i = atomicAdd(S.defer_n, 1u);
  if (i < S.defer_cap) S.defer[i] = make_uint2(pid, meta);
  else atomicOr(S.err, ERR_DEFER);
}

enum { CAND_NULL = 0, CAND_REAL = 1, CAND_DEFER = 2 };

// Outcome of the candidate at path length f.D, whose face counts fb and cell the caller took
// in FP32 (the first wall lies beyond it by more than the bound, so it is a candidate for the
// FP64 walk too): CAND_NULL or CAND_REAL when the FP64 walk decides the same, CAND_DEFER
// otherwise. A candidate whose acceptance draw exceeds the largest ratio of its cell's
// neighbourhood (by more than the ratio's rounding) is rejected wherever it lies, and needs no
// face test; its W may sit in the neighbouring cell. ub: the acceptance word; sy, sz: cell
// index steps along y and z.
// all_real: every candidate of the band is real, and near tells whether a count lies within
// the bound of a face (count_near); otherwise the tie bits are found here when needed.
template <int DIM>
__device__ __forceinline__ int candidate_outcome(const SweepArgs& A, long long bcbase, int ncells, const PW& f,
                                                 float base, int fb0, int fb1, int fb2, int cell, bool all_real,
                                                 bool near, uint32_t ub, int n0, int n1, int n2, int sy, int sz) {
  if (all_real) return near ? CAND_DEFER : CAND_REAL;
  const float ua = word_uniform<float>(ub);
  if (ua - A.ratio_nb32[bcbase + cell] >= TIE_ACC) return CAND_NULL;
  unsigned tie = tie_bits(f.D, f.t0, f.d0, base, fb0, 0);
  if (DIM >= 2) tie |= tie_bits(f.D, f.t1, f.d1, base, fb1, 2);
  if (DIM == 3) tie |= tie_bits(f.D, f.t2, f.d2, base, fb2, 4);
  const float ra = A.ratio32[bcbase + cell];
  if (tie) {
    unsigned hit = tie_hits_wall(tie, 0, fb0, faces_to_wall(f.i0, f.s0, n0));
    if (DIM >= 2) hit |= tie_hits_wall(tie, 1, fb1, faces_to_wall(f.i1, f.s1, n1));
    if (DIM == 3) hit |= tie_hits_wall(tie, 2, fb2, faces_to_wall(f.i2, f.s2, n2));
    if (!all_reject(A.ratio32 + bcbase, ncells, cell, tie, hit, f.s0, f.s1 * sy, f.s2 * sz, ua)) return CAND_DEFER;
  }
  if (fabsf(ua - ra) < TIE_ACC) return CAND_DEFER;
  return ua < ra ? CAND_REAL : CAND_NULL;
}

}  // namespace

// The largest |weight| of each forward group's emitters, max-reduced into its instance's slot
// (non-negative doubles order like their bit patterns). Group g has blocks [bpre[g],
// bpre[g + 1]) of the grid, in proportion to its emitters (about two blocks per SM in all), so
// the FP64 weight arithmetic is spread over the SMs in proportion to the work.
__global__ void group_wmax_kernel(SweepArgs A, const int* bpre, unsigned long long* wmax_bits) {
  __shared__ double sh[32];
  int gi = 0;
  {
    int hi = A.n_groups - 1;  // the last group whose first block is at or before this one
    while (gi < hi) {
      const int mid = (gi + hi + 1) >> 1;
      if (bpre[mid] <= (int)blockIdx.x) gi = mid;
      else hi = mid - 1;
    }
  }
  const Group G = A.groups[gi];
  const int by = (int)blockIdx.x - bpre[gi], ny = bpre[gi + 1] - bpre[gi];
  const InstDesc& in = A.inst[G.inst];
  double m = 0.0;
  if (G.kind == 0) {
    const long long base = in.bc_off + (long long)G.band * in.ncells;
    for (int e = by * blockDim.x + threadIdx.x; e < in.ncells; e += ny * blockDim.x) {
      double Te = A.T[in.cell_off + e];
      if (A.srcshift) Te += A.srcshift[in.cell_off + e];
      const double w = A.coef[base + e] * Te;
      A.wemit[base + e] = w;  // the weight of every particle of this emitter
      m = fmax(m, fabs(w));
    }
  } else {
    const int wl = G.kind - 1;
    const double wc = A.wcoef[((long long)G.inst * A.nb + G.band) * 6 + wl];
    const double* tf = A.wallTf + in.bface_off + in.wface_off[wl];
    for (int j = by * blockDim.x + threadIdx.x; j < G.n_emitters; j += ny * blockDim.x)
      m = fmax(m, fabs(wc * tf[j]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
    atomicMax(&wmax_bits[G.inst], (unsigned long long)__double_as_longlong(r));
  }
}

// Emits particle pid (global forward index) into lane state. Returns false for a
// zero-weight particle (nothing to trace).
// Per-lane cache of the group of the lane's previous particle (and of the weight of a
// wall group, which is the same for all its particles).
struct EmitCache {
  unsigned g_first, g_end;  // forward particle range of the cached group
  int g_idx, g_ne, g_kind, g_band;
  int g_perm;               // perm_off of the group
  unsigned g_mag;           // division magic of n_emitters
  int e;
  double w;
};

// Emits forward particle pid into the lane state. Returns false for a zero-weight
// particle (nothing to trace).
// ADJ: the adjoint re-trace; w is then the particle's weight per unit emission
// temperature (every emitter is traced) and `emitter` receives the cell (>= 0) or the
// wall slot (-1 - wall) the particle's gather belongs to.
template <int DIM, bool ADJ>
__device__ __forceinline__ bool staged_emit(const SweepArgs& A, const StagedArgs& S, unsigned pid, bool useF,
                                            double& w, int& band, PW& f, Stream& st, uint32_t& ub, EmitCache& ec,
                                            const InstDesc& in, int k, int& emitter, bool two) {
  if (pid < ec.g_first || pid >= ec.g_end) {
    const int gi = find_group(A.groups, A.n_groups, (long long)pid);
    const Group G = A.groups[gi];
    ec.g_idx = gi;
    ec.g_first = (unsigned)G.first_particle;
    ec.g_end = (unsigned)(G.first_particle + (long long)G.n_emitters * G.per_emitter);
    ec.g_ne = G.n_emitters;
    ec.g_kind = G.kind;
    ec.g_band = G.band;
    ec.g_mag = S.group_mag[gi];
    ec.g_perm = G.perm_off;
    ec.e = -1;
  }
  band = ec.g_band;
  const int b = ec.g_band;
  // The staged sweep visits a group's particles q-major (particle q of every emitter,
  // then q + 1), so the lanes of a warp start in different cells: their face and deposit
  // tallies rarely hit the same address at the same time; within a q the emitters come in
  // the group's visiting order. Draws are keyed by (emitter, particle), so the order changes
  // nothing else.
  const unsigned local = pid - ec.g_first;
  const int q = (int)udiv(local, (unsigned)ec.g_ne, ec.g_mag);
  int e = (int)(local - (unsigned)q * (unsigned)ec.g_ne);
  if (ec.g_perm >= 0) e = A.perm[ec.g_perm + e];
  const int n0 = in.n[0], n1 = in.n[1], n2 = in.n[2];
  const int kind = ec.g_kind;
  float xi0 = 0.5f, xi1 = 0.5f, xi2 = 0.5f, sx = 0.f, sy = 0.f, sz = 0.f;
  if (kind == 0) {
    if (ADJ) {
      w = A.coef[in.bc_off + (long long)b * in.ncells + e];
    } else {
      w = A.wemit[in.bc_off + (long long)b * in.ncells + e];  // from the w_max pre-pass
      if ((__double_as_longlong(w) << 1) == 0) return false;   // +-0: nothing to trace
    }
    emitter = e;
    st.init(A.seed, in.inst_id, (uint32_t)b, A.epoch, (uint32_t)e, (uint32_t)q);
    if (DIM == 1) {
      f.i0 = e;
      f.i1 = 0;
      f.i2 = 0;
    } else {
      const int r = (int)udiv((unsigned)e, (unsigned)n0, S.mag_n0[k]);
      f.i0 = e - r * n0;
      if (DIM == 2) {
        f.i1 = r;
        f.i2 = 0;
      } else {
        f.i2 = (int)udiv((unsigned)r, (unsigned)n1, S.mag_n1[k]);
        f.i1 = r - f.i2 * n1;
      }
    }
    float u_mu, u_phi = 0.5f;
    if (DIM == 1) {
      xi0 = word_uniform<float>(st.buf.x);
      u_mu = word_uniform<float>(st.buf.y);
    } else if (DIM == 2) {
      xi0 = word_uniform<float>(st.buf.x);
      xi1 = word_uniform<float>(st.buf.y);
      u_mu = word_uniform<float>(st.buf.z);
      u_phi = word_uniform<float>(st.buf.w);
    } else {
      xi0 = word_uniform<float>(st.buf.x);
      xi1 = word_uniform<float>(st.buf.y);
      xi2 = word_uniform<float>(st.buf.z);
      u_mu = word_uniform<float>(st.buf.w);
      st.load_block(1);
      u_phi = word_uniform<float>(st.buf.x);
    }
    const float mu = 2.f * u_mu - 1.f;
    sx = mu;
    if (DIM >= 2) {
      const float sn = sqrtf(fmaf(-mu, mu, 1.f));  // 1 - mu^2 with one rounding
      float sp, cp;
      sincospif(2.f * u_phi, &sp, &cp);
      sy = sn * cp;
      sz = sn * sp;
    }
    st.j = thermal_uniforms(DIM);
  } else {
    const int wl = kind - 1;
    if (ec.e != -2) {
      ec.w = A.wcoef[((long long)k * A.nb + b) * 6 + wl];  // per unit face temperature
      ec.e = -2;
    }
    w = ADJ ? ec.w : ec.w * A.wallTf[in.bface_off + in.wface_off[wl] + e];
    if (w == 0.0) return false;
    emitter = -1 - wl;
    const int a = wl >> 1, side = wl & 1;
    // faces of wall a are enumerated over (o1, o2) = ((a+1)%3, (a+2)%3), o1 fastest
    const int no1 = a == 0 ? n1 : (a == 1 ? n2 : n0);
    const int j2 = (int)udiv((unsigned)e, (unsigned)no1, S.mag_wall[k * 3 + a]);
    const int j1 = e - j2 * no1;
    long long face;
    if (a == 0) {
      f.i0 = side ? n0 - 1 : 0;
      f.i1 = j1;
      f.i2 = j2;
      face = in.fax_off[0] + (side ? n0 : 0) + (long long)(n0 + 1) * (j1 + (long long)n1 * j2);
    } else if (a == 1) {
      f.i0 = j2;
      f.i1 = side ? n1 - 1 : 0;
      f.i2 = j1;
      face = in.fax_off[1] + j2 + (long long)n0 * ((side ? n1 : 0) + (long long)(n1 + 1) * j1);
    } else {
      f.i0 = j1;
      f.i1 = j2;
      f.i2 = side ? n2 - 1 : 0;
      face = in.fax_off[2] + j1 + (long long)n0 * (j2 + (long long)n1 * (side ? n2 : 0));
    }
    st.init(A.seed, in.inst_id, (uint32_t)b, A.epoch, (uint32_t)(in.ncells + face), (uint32_t)q);
    float u_n, u_phi = 0.5f;
    float t0 = 0.5f, t1 = 0.5f;  // tangential fractions, in axis order
    if (DIM == 1) {
      u_n = word_uniform<float>(st.buf.x);
    } else if (DIM == 2) {
      t0 = word_uniform<float>(st.buf.x);
      u_n = word_uniform<float>(st.buf.y);
      u_phi = word_uniform<float>(st.buf.z);
    } else {
      t0 = word_uniform<float>(st.buf.x);
      t1 = word_uniform<float>(st.buf.y);
      u_n = word_uniform<float>(st.buf.z);
      u_phi = word_uniform<float>(st.buf.w);
    }
    const float mn = sqrtf(u_n);
    const float sn = DIM >= 2 ? sqrtf(1.f - u_n) : 0.f;
    float sp = 0.f, cp = 0.f;
    if (DIM >= 2) sincospif(2.f * u_phi, &sp, &cp);
    const float nrm = side ? -mn : mn, ta = sn * cp, tb = sn * sp;  // tangential (o1, o2)
    if (a == 0) {
      sx = nrm; sy = ta; sz = tb;
      xi0 = side ? 1.f : 0.f; xi1 = t0; xi2 = t1;
    } else if (a == 1) {
      sy = nrm; sz = ta; sx = tb;
      xi1 = side ? 1.f : 0.f; xi0 = t0; xi2 = t1;
    } else {
      sz = nrm; sx = ta; sy = tb;
      xi2 = side ? 1.f : 0.f; xi0 = t0; xi1 = t1;
    }
    st.j = wall_uniforms(DIM);
    (void)face;  // the power entering through wall faces is added by boundary_kernel
  }
  axis_init(sx, xi0, in.hf[0], f.t0, f.d0, f.s0);
  f.tex = axis_exit(f.i0, f.s0, n0, f.t0, f.d0);
  if (DIM >= 2) {
    axis_init(sy, xi1, in.hf[1], f.t1, f.d1, f.s1);
    const float e1 = axis_exit(f.i1, f.s1, n1, f.t1, f.d1);
    // 2D: the axis of the wall the segment reaches (x on ties), kept in the unused i2
    if (DIM == 2) f.i2 = e1 < f.tex ? 1 : 0;
    f.tex = fminf(f.tex, e1);
  }
  if (DIM >= 3) {
    axis_init(sz, xi2, in.hf[2], f.t2, f.d2, f.s2);
    f.tex = fminf(f.tex, axis_exit(f.i2, f.s2, n2, f.t2, f.d2));
  }
  if (!ADJ && DIM == 2 && two && f.d0 < f.d1) {
    // y-group: its emission enters its own power balance (cell) or boundary flux (face)
    if (kind == 0) {
      atomicAdd(&S.DY[in.cell_off + e], -w);
    } else {
      const int wl = kind - 1;
      atomicAdd(&S.EY[in.bface_off + in.wface_off[wl] + e], (wl & 1) ? -w : w);
    }
  }
  // the first candidate: its path word from block 0's unused bits; its acceptance word only
  // where some cell of the band may reject (else every candidate is real and the particle ends
  // at its first candidate, so no later draw is taken)
  ub = A.all_real[(long long)k * A.nb + b] ? 0u : st.even_word();
  st.j += 2;
  f.D = __fmul_rn(-__logf(word_uniform<float>(st.first)), A.vtm32[(long long)k * A.nb + b]);
  return true;
}

// Persistent blocks. Each block works on one instance at a time (first the instance its
// index falls on by estimated cost, then any instance with work left); its warps take
// private ranges of the instance's particles and refill idle lanes together. Faces normal
// to x go to a shared-memory copy of the instance's x-faces (when it fits), in units of
// the instance's q; the block flushes it when it leaves the instance.
// ADJ = true: the adjoint re-trace (see adjoint.cu for the map it transposes): no tallies;
// a real collision gathers c_p lambda[stop] / (V m_stop) into the particle's emitter cell,
// or into its wall, accumulated per lane while the lane stays on one wall group.
// Compensated FP32 tally. The atomic returns the value it added to, so the exact rounding
// error of the stored sum is known locally (Knuth's TwoSum, six FP32 operations); that error
// and the low part of the FP64 addend go to the companion word. After n additions the pair
// holds the sum to about n 2^-48 relative. (atom.add.f32 flushes subnormal results to zero:
// an absolute error below 2^-126 per addition, far under the tally scale.)
__device__ __forceinline__ void tally_k32(float2* p, double x) {
  const float xh = __double2float_rn(x);
  const float xl = __double2float_rn(x - (double)xh);
  const float old = atomicAdd(&p->x, xh);
  const float sum = __fadd_rn(old, xh);
  const float bv = __fsub_rn(sum, old);
  const float err = __fadd_rn(__fsub_rn(old, __fsub_rn(sum, bv)), __fsub_rn(xh, bv));
  const float lo = __fadd_rn(err, xl);
  if (lo != 0.f) atomicAdd(&p->y, lo);
}

// Instance holding entry j of a [band][cell] array: the last one whose bc_off is at or before j.
__device__ __forceinline__ int bc_instance(const InstDesc* inst, int n_inst, long long j) {
  int lo = 0, hi = n_inst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].bc_off <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The candidate estimator W = sum of w tau_maj over candidates (Sec. 3.2): the staged sweep
// sums w per (band, cell) and multiplies by the instance's tau_maj of the band here; in a band
// with tau = tau_maj in every cell every candidate is real, so there W = tau_maj R (the sweep
// leaves W alone).
__global__ void scale_by_taumaj_kernel(const InstDesc* inst, int n_inst, int nb, const double* taumaj,
                                       const int* all_real, const double* R, double* W, long long total) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
    const int k = bc_instance(inst, n_inst, j);
    const long long kb = (long long)k * nb + (j - inst[k].bc_off) / inst[k].ncells;
    W[j] = (all_real[kb] ? R[j] : W[j]) * taumaj[kb];
  }
}

// FP64 value of compensated tallies: dst = hi + lo (add = 0) or dst += hi + lo (add = 1).
__global__ void k32_finalize_kernel(const float2* src, double* dst, long long n, int add) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 v = src[i];
    const double x = (double)v.x + (double)v.y;
    dst[i] = add ? dst[i] + x : x;
  }
}

template <int DIM, bool ADJ, bool K32>
__global__ void __launch_bounds__(STAGED_NT, 1) sweep_staged_kernel(SweepArgs A, StagedArgs S) {
  extern __shared__ unsigned win[];
  // cooperative tallies: per warp, each lane's particle parameters and the item list starts
  __shared__ int4 s_par[STAGED_NT / 32][64];
  __shared__ int s_lst[STAGED_NT / 32][33];
  __shared__ int s_inst;
  LCounts cnt;
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) cnt.v[k] = 0;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const bool useF = !ADJ && A.F != nullptr;
  const int n_inst = S.n_inst;
  int start = 0;
  {
    const double pos = (blockIdx.x + 0.5) / gridDim.x * S.cost_total;
    while (start + 1 < n_inst && S.cost_prefix[start + 1] <= pos) ++start;
  }
  for (int visit = 0; visit < n_inst; ++visit) {
    const int k = (start + visit) % n_inst;
    if (threadIdx.x == 0) s_inst = (*(volatile unsigned long long*)&S.inst_next[k] < (unsigned long long)S.inst_end[k]) ? k : -1;
    __syncthreads();
    if (s_inst < 0) {
      __syncthreads();
      continue;
    }
    const InstDesc& in = A.inst[k];
    // descriptor fields used inside the walk, held in registers (the atomics below would
    // otherwise force reloads)
    const int n0 = in.n[0], n1 = in.n[1], n2 = in.n[2];
    const long long face_off = in.face_off, fax1 = in.fax_off[1], fax2 = in.fax_off[2];
    const long long bc_off = in.bc_off;
    const int ncells = in.ncells, refill = S.refill > 0 ? S.refill : in.refill;
    const int sy_cell = n0, sz_cell = n0 * n1;           // cell index steps along y, z
    const int sy_xf = n0 + 1, sz_xf = (n0 + 1) * n1;     // x-face index steps along y, z
    // x-faces [wbase, wbase + wlen) of this instance are tallied in the shared window
    const int2 wd = useF ? S.window[k] : make_int2(0, 0);
    const int wbase = wd.x;
    const unsigned wlen = (unsigned)wd.y;
    const bool wfull = wbase == 0 && (long long)wlen == (long long)(n0 + 1) * n1 * n2;
    // 2D instance whose faces all fit the window: two-group tallies (see StagedArgs)
    const bool two = DIM == 2 && useF && wbase == 0 && (long long)wlen == in.nfaces;
    for (unsigned i = threadIdx.x; i < wlen; i += STAGED_NT) win[i] = WIN_BIAS;
    __syncthreads();
    const double wmax = S.wmax[k];
    const double qinv = wmax > 0.0 ? WIN_SCALE / wmax : 0.0;
    const unsigned pend = (unsigned)S.inst_end[k];
    unsigned rbeg = 0, rend = 0;  // this warp's private particle range
    double w = 0.0;
    unsigned qwx = 0;             // signed x-face contribution in units of q (two's complement)
    int band = 0;
    long long bcbase = 0;
    float vtm = 0.f;
    PW f;
    Stream st;
    uint32_t ub = 0;
    bool alive = false, exhausted = false;
    bool tally = false;     // the lane's particle has ended and tallies its faces
    int kcur = 0, kend = 0; // face items of the tally phase (x-faces, then y-faces in 3D)
    EmitCache ec;
    ec.g_first = 1;
    ec.g_end = 0;  // empty: forces a lookup on the first emission
    ec.e = -1;
    int emitter = 0;        // adjoint: gather target of the lane's particle
    int acc_slot = 0;       // adjoint: wall slot of the pending per-lane wall sum
    double acc = 0.0;
    float eD = 0.f;         // bound of |D - D_fp64| of the lane's particle
    int kc = 0;             // its candidates tallied so far
    unsigned pid = 0;       // its forward (or adjoint) index
    for (;;) {
      // ---- refill idle lanes together ----
      const unsigned dead = __ballot_sync(0xffffffffu, !alive);
      if (!exhausted && __popc(dead) >= refill) {
        if (rbeg == rend) {  // private range used up: take the next one of the instance
          unsigned long long got = 0;
          if (lane == 0) got = atomicAdd(&S.inst_next[k], (unsigned long long)S.warp_grab);
          got = __shfl_sync(0xffffffffu, got, 0);
          if (got < pend) {
            rbeg = (unsigned)got;
            rend = (unsigned)min(got + (unsigned long long)S.warp_grab, (unsigned long long)pend);
          } else {
            exhausted = true;
          }
        }
        const unsigned rank = __popc(dead & lt_mask);
        const unsigned take = min((unsigned)__popc(dead), rend - rbeg);
        if (!alive && rank < take) {
          alive = staged_emit<DIM, ADJ>(A, S, rbeg + rank, useF, w, band, f, st, ub, ec, in, k, emitter, two);
          if (ADJ && alive && emitter < 0 && emitter != acc_slot) {
            if (acc != 0.0) atomicAdd(&A.adj_wall[in.wall_off + (-1 - acc_slot)], acc);
            acc = 0.0;
            acc_slot = emitter;
          }
          if (alive) {
            cnt.v[CNT_FLIGHTS] += 1;
            // round(w / q) as the low word of w qinv + 1.5 2^52 (one FMA, |w qinv| <= 2^26)
            const int qw = __double2loint(fma(w, qinv, 0x1.8p52));
            // signed along the axis whose faces the particle tallies
            qwx = (unsigned)(((two && f.d0 < f.d1) ? f.s1 : f.s0) > 0 ? qw : -qw);
            vtm = A.vtm32[(long long)k * A.nb + band];
            bcbase = bc_off + (long long)band * ncells;
            eD = fmaf(f.D, TIE_LOG_REL, vtm * TIE_LOG_ABS);
            kc = 0;
            pid = rbeg + rank;
          }
        }
        rbeg += take;
      }
      if (!__any_sync(0xffffffffu, alive)) {
        if (exhausted) break;
        continue;
      }
      // ---- candidates (Sec. 3.2): up to walk_k per lane. The candidate lies at path length D
      // of the straight segment; its cell follows from the faces before D on each axis.
      // W tally, then acceptance with probability tau_maj / tau(x); a rejected candidate
      // draws the next flight length and the particle goes on in the same direction. In 3D
      // the walk stops early once fewer than WALK_MIN_LANES lanes are still walking: the lanes
      // whose particles ended get their items tallied and are refilled sooner, and the others go
      // on in the next pass (16-box batch at refill 4, walk_k 8: 75.9 -> 74.6 ms) ----
      int nitem = 0;  // cooperative tallies: face items of the lane's particle ended in this pass
      int nx3 = 0, ny3 = 0;  // 3D: x- and y-face items of the lane's particle ended in this pass
      bool ended = false, wall_exit = false, deferred = false;
      const bool walking = alive && !tally;
      const bool all_real = A.all_real[(long long)k * A.nb + band] != 0;
      if (walking) {
#pragma unroll 1
        for (int it = 0; it < S.walk_k; ++it) {
          if (DIM == 3 && it > 0 && __popc(__activemask()) < WALK_MIN_LANES) break;
          // a decision within rounding of the FP64 walk's defers the particle to the FP64 replay
          const float base = fmaf(TIE_REL, f.D, eD);
          if (f.D - f.tex > base) {  // the segment reaches a wall first: absorbed there
            ended = wall_exit = true;
            break;
          }
          if (f.tex - f.D <= fmaf(TIE_REL, f.tex, eD)) {  // at the first wall within rounding
            ended = deferred = true;
            break;
          }
          bool near = false;  // a count within the bound of a face, found with it for all-real bands
          int fb0, fb1 = 0, fb2 = 0;
          if (all_real) {
            fb0 = count_near(f.D, f.t0, f.d0, base, near);
            if (DIM >= 2) fb1 = count_near(f.D, f.t1, f.d1, base, near);
            if (DIM == 3) fb2 = count_near(f.D, f.t2, f.d2, base, near);
          } else {
            fb0 = faces_before(f.D, f.t0, f.d0);
            if (DIM >= 2) fb1 = faces_before(f.D, f.t1, f.d1);
            if (DIM == 3) fb2 = faces_before(f.D, f.t2, f.d2);
          }
          int cell = clampi(f.i0 + f.s0 * fb0, n0);
          if (DIM >= 2) cell += sy_cell * clampi(f.i1 + f.s1 * fb1, n1);
          if (DIM == 3) cell += sz_cell * clampi(f.i2 + f.s2 * fb2, n2);
          const long long ci = bcbase + cell;
          const int oc = candidate_outcome<DIM>(A, bcbase, ncells, f, base, fb0, fb1, fb2, cell, all_real, near, ub,
                                                n0, n1, n2, sy_cell, sz_cell);
          if (oc == CAND_DEFER) {
            ended = deferred = true;
            break;
          }
          cnt.v[CNT_CANDIDATES] += 1;
          ++kc;
          // W collects w here; the sweep scales it by tau_maj afterwards (scale_by_taumaj), and
          // a band whose every candidate is real takes W = tau_maj R there instead
          if (!ADJ && K32 && S.W32 && !all_real) tally_k32(&S.W32[ci], w);
          else if (!ADJ && !K32 && A.W && !all_real) atomicAdd(&A.W[ci], w);
          if (oc == CAND_REAL) {
            cnt.v[CNT_REAL] += 1;
            if (ADJ) {
              const long long gc = in.cell_off + cell;
              const double val = w * A.lambda[gc] * A.invVm[gc];
              if (emitter >= 0) atomicAdd(&A.adj_out[in.cell_off + emitter], val);
              else acc += val;
            } else if (K32) {
              tally_k32(&S.R32[ci], w);
            } else {
              atomicAdd(&A.R[ci], w);
            }
            if (!ADJ && two && f.d0 < f.d1) atomicAdd(&S.DY[in.cell_off + cell], w);
            ended = true;
            break;
          }
          uint32_t uw;
          st.next_pair(uw, ub);
          const float ell = __fmul_rn(-__logf(word_uniform<float>(uw)), vtm);
          f.D = __fadd_rn(f.D, ell);
          eD = fmaf(f.D, TIE_SUM, fmaf(ell, TIE_LOG_REL, eD + vtm * TIE_LOG_ABS));
        }
      }
      if (walking) {
        if (deferred) {
          defer_particle(S, pid, ADJ ? 0u : (((unsigned)kc << 1) | ((two && f.d0 < f.d1) ? 1u : 0u)));
          ended = false;
          alive = false;
        }
        if (ended) {
          // interior faces crossed before the end, per axis; on the exit axis the wall face
          // lies exactly at tex, so its count is known without rounding
          const float L = wall_exit ? f.tex : f.D;
          int ex = -1;
          if (wall_exit) {
            const float e0 = axis_exit(f.i0, f.s0, n0, f.t0, f.d0);
            const float e1 = DIM >= 2 ? axis_exit(f.i1, f.s1, n1, f.t1, f.d1) : INFINITY;
            const float e2 = DIM == 3 ? axis_exit(f.i2, f.s2, n2, f.t2, f.d2) : INFINITY;
            ex = (e0 <= e1 && e0 <= e2) ? 0 : (e1 <= e2 ? 1 : 2);
          }
          // at a wall, the faces of the other axes crossed before it: a count within rounding
          // of the FP64 walk's (the segment leaves near a cell corner) defers the particle
          bool tie = false;
          const float bx = TIE_REL * f.tex;
          const int m0 = faces_to_wall(f.i0, f.s0, n0);
          int c0 = m0 - 1, c1 = 0, c2 = 0, m1 = 1;
          if (ex != 0) {
            const int q = count_near(L, f.t0, f.d0, bx, tie);
            c0 = min(q, m0 - 1);
          }
          if (DIM >= 2) {
            m1 = faces_to_wall(f.i1, f.s1, n1);
            c1 = m1 - 1;
            if (ex != 1) {
              const int q = count_near(L, f.t1, f.d1, bx, tie);
              c1 = min(q, m1 - 1);
            }
          }
          if (DIM == 3) {
            const int m2 = faces_to_wall(f.i2, f.s2, n2);
            c2 = m2 - 1;
            if (ex != 2) {
              const int q = count_near(L, f.t2, f.d2, bx, tie);
              c2 = min(q, m2 - 1);
            }
          }
          if (!ADJ && wall_exit && tie) {
            defer_particle(S, pid, ((unsigned)kc << 1) | ((two && f.d0 < f.d1) ? 1u : 0u));
            alive = false;
          } else {
            if (wall_exit) cnt.v[CNT_WALL_EXITS] += 1;
            cnt.v[CNT_CROSSINGS] += c0 + c1 + c2;
            if (DIM == 2 && (two || wfull)) {
              // Face items k = 0 .. kend-1 along the tallied axis p (the other axis: q). Item k
              // is the face index a0 + k sp + sq min(ceil(u0 + k r), lim): the k-th face normal
              // to p, in the row (or column) given by the faces normal to q crossed before it,
              // ceil(u0 + k r) with u0 = (t_p - t_q) / d_q and r = d_p / d_q, at most lim.
              const bool yg = two && f.d0 < f.d1;
              int a0, sp, sq, lim;
              float u0, r;
              if (!yg) {
                // exit through the low y-wall: the one face normal to y this group tallies
                if (ex == 1 && f.s1 < 0) {
                  const int col = f.i0 + f.s0 * c0;
                  if (two) atomicAdd(&S.gx()[in.bface_off + in.wface_off[2] + col], -w);
                  else if (K32) tally_k32(&S.F32[face_off + fax1 + col], -w);
                  else atomicAdd(&A.F[face_off + fax1 + col], -w);
                }
                kend = c0 + (ex == 0 ? 1 : 0);
                const bool flat = !(f.d1 < INFINITY);
                u0 = flat ? -1.f : __fdividef(f.t0 - f.t1, f.d1);
                r = flat ? 0.f : __fdividef(f.d0, f.d1);
                lim = m1 - 1;
                a0 = (f.s0 > 0 ? f.i0 + 1 : f.i0) + sy_xf * f.i1;
                sp = f.s0;
                sq = f.s1 * sy_xf;
              } else {
                // exit through the low x-wall: the one face normal to x this group tallies
                if (ex == 0 && f.s0 < 0) atomicAdd(&S.gx()[in.bface_off + in.wface_off[0] + (f.i1 + f.s1 * c1)], -w);
                kend = c1 + (ex == 1 ? 1 : 0);
                u0 = __fdividef(f.t1 - f.t0, f.d0);
                r = __fdividef(f.d1, f.d0);
                lim = m0 - 1;
                a0 = (int)fax1 + f.i0 + n0 * (f.s1 > 0 ? f.i1 + 1 : f.i1);
                sp = f.s1 * n0;
                sq = f.s0;
              }
              f.i0 = a0;
              f.s0 = sp;
              f.s1 = sq;
              f.i2 = lim;
              f.D = u0;
              f.tex = r;
              nitem = kend;  // tallied below by the whole warp
              alive = false;
            } else if (useF) {
              // faces normal to the last axis: only the low boundary is tallied (the rest
              // follow from conservation)
              if (DIM == 2 && ex == 1 && f.s1 < 0) {
                const long long fi = face_off + fax1 + (f.i0 + f.s0 * c0);
                if (K32) tally_k32(&S.F32[fi], -w);
                else atomicAdd(&A.F[fi], -w);
              } else if (DIM == 3 && ex == 2 && f.s2 < 0) {
                const long long fi = face_off + fax2 + (f.i0 + f.s0 * c0) + (long long)n0 * (f.i1 + f.s1 * c1);
                if (K32) tally_k32(&S.F32[fi], -w);
                else atomicAdd(&A.F[fi], -w);
              }
              if (DIM == 3) {
                // Two item lists, tallied below by the whole warp: the x-faces crossed (the wall
                // face too when the particle leaves through x) and the y-faces. Item k of the list
                // along axis p is the face a0 + k sp + sq1 min(ceil(u1 + k r1), lim1) + sq2
                // min(ceil(u2 + k r2), lim2): the k-th face normal to p, in the cell row and
                // layer given by the faces of the other two axes crossed before it (ceil((t_p +
                // k d_p - t_q) / d_q) = ceil(u + k r), u = (t_p - t_q) / d_q, r = d_p / d_q).
                int4* tab = reinterpret_cast<int4*>(win) + (threadIdx.x >> 5) * COOP3_INT4_PER_WARP + 6 * lane;
                auto ur = [](float tp, float dp, float tq, float dq, float& u, float& r) {
                  const bool flat = !(dq < INFINITY);
                  u = flat ? -1.f : __fdividef(tp - tq, dq);
                  r = flat ? 0.f : __fdividef(dp, dq);
                };
                float u1, r1, u2, r2;
                nx3 = c0 + (ex == 0 ? 1 : 0);
                ny3 = c1 + (ex == 1 ? 1 : 0);
                ur(f.t0, f.d0, f.t1, f.d1, u1, r1);
                ur(f.t0, f.d0, f.t2, f.d2, u2, r2);
                double ws = f.s0 > 0 ? w : -w;
                tab[0] = make_int4((f.s0 > 0 ? f.i0 + 1 : f.i0) + sy_xf * f.i1 + sz_xf * f.i2, f.s0, f.s1 * sy_xf,
                                   faces_to_wall(f.i1, f.s1, n1) - 1);
                tab[1] = make_int4(f.s2 * sz_xf, faces_to_wall(f.i2, f.s2, n2) - 1, __float_as_int(u1),
                                   __float_as_int(r1));
                tab[2] = make_int4(__float_as_int(u2), __float_as_int(r2), __double2loint(ws), __double2hiint(ws));
                ur(f.t1, f.d1, f.t0, f.d0, u1, r1);
                ur(f.t1, f.d1, f.t2, f.d2, u2, r2);
                ws = f.s1 > 0 ? w : -w;
                const int sz_yf = n0 * (n1 + 1);  // y-face index step along z
                tab[3] = make_int4((int)fax1 + f.i0 + n0 * (f.s1 > 0 ? f.i1 + 1 : f.i1) + sz_yf * f.i2, f.s1 * n0, f.s0,
                                   m0 - 1);
                tab[4] = make_int4(f.s2 * sz_yf, faces_to_wall(f.i2, f.s2, n2) - 1, __float_as_int(u1),
                                   __float_as_int(r1));
                tab[5] = make_int4(__float_as_int(u2), __float_as_int(r2), __double2loint(ws), __double2hiint(ws));
                alive = false;
              } else {
              // x-faces crossed (the wall face too when the particle leaves through x),
              // then in 3D the y-faces
              kcur = 0;
              kend = c0 + (ex == 0 ? 1 : 0);
              if (DIM == 3) {
                f.tex = small_int_float(kend);  // first y-face item
                kend += c1 + (ex == 1 ? 1 : 0);
              } else if (DIM == 2) {
                // rows of the x-face crossings, incrementally: faces normal to y before the
                // k-th x-face = ceil(u0 + k r), u0 = (t0 - t1) / d1, r = d0 / d1
                const bool flat = !(f.d1 < INFINITY);
                f.D = flat ? -1.f : __fdividef(f.t0 - f.t1, f.d1);
                f.tex = flat ? 0.f : __fdividef(f.d0, f.d1);
                f.i2 = m1 - 1;  // largest count of y-faces a row index may take
              }
              tally = kend > 0;
              alive = tally;
              }
            } else {
              alive = false;
            }
          }
        }
      }
      // ---- 2D, every tallied face in the window: the warp tallies the face items of the
      // particles that ended in this pass together. The items are concatenated in lane
      // order and cut into 32 equal contiguous chunks, one per lane; a lane finds the
      // particle holding its first item by binary search over the list starts and reads
      // each particle's parameters from shared memory when its chunk enters that list ----
      if (DIM == 2 && (two || wfull)) {
        int incl = nitem;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total > 0) {
          const int first = incl - nitem;
          int4* par = s_par[threadIdx.x >> 5];
          int* lst = s_lst[threadIdx.x >> 5];
          lst[lane] = first;
          if (lane == 31) lst[32] = total;
          if (nitem > 0) {
            par[2 * lane] = make_int4(f.i0, f.s0, f.s1, f.i2);
            par[2 * lane + 1] = make_int4(__float_as_int(f.D), __float_as_int(f.tex), (int)qwx, first);
          }
          __syncwarp();
          const int c0 = (lane * total) >> 5, c1 = ((lane + 1) * total) >> 5;
          if (c0 < c1) {
            // the last list starting at or before c0 (it holds c0: empty lists start where
            // the next one does)
            int l = 0;
#pragma unroll
            for (int st = 16; st > 0; st >>= 1)
              if (lst[l + st] <= c0) l += st;
            int lend = lst[l + 1];
            int4 pa = par[2 * l], pb = par[2 * l + 1];
#pragma unroll 1
            for (int kk = c0; kk < c1; ++kk) {
              if (kk >= lend) {
                do {
                  ++l;
                  lend = lst[l + 1];
                } while (lend <= kk);
                pa = par[2 * l];
                pb = par[2 * l + 1];
              }
              // item kl of the particle: a0 + kl sp + sq min(ceil(u0 + kl r), lim)
              const int kl = kk - pb.w;
              const int face =
                  pa.x + kl * pa.y +
                  pa.z * min(ceil_count(fmaf(small_int_float(kl), __int_as_float(pb.y), __int_as_float(pb.x))), pa.w);
              const unsigned q = (unsigned)pb.z;
              const unsigned old = atomicAdd(&win[face], q);
              // |q| <= 2^26, so the word can wrap only from within 2^26 of 0 / 2^32
              if (old + 0x04000000u < 0x08000000u) {
                const int carry = ((int)q >> 31) + (old + q < old ? 1 : 0);
                if (carry) atomicAdd(&A.F[face_off + face], (double)carry * S.wmax[k] * WIN_CARRY);
              }
            }
          }
          __syncwarp();
        }
      }
      // ---- 3D: the warp tallies the x- and y-face items of the particles that ended in this
      // pass together (lists 2 lane and 2 lane + 1, concatenated in order and cut into 32
      // equal contiguous chunks, one per lane), with global atomics ----
      if (DIM == 3 && !ADJ && useF) {
        int incl = nx3 + ny3;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        if (total > 0) {
          const int4* tab = reinterpret_cast<const int4*>(win) + (threadIdx.x >> 5) * COOP3_INT4_PER_WARP;
          int* lst = reinterpret_cast<int*>(reinterpret_cast<int4*>(win) + (threadIdx.x >> 5) * COOP3_INT4_PER_WARP +
                                            3 * COOP3_LISTS);
          const int excl = incl - nx3 - ny3;
          lst[2 * lane] = excl;
          lst[2 * lane + 1] = excl + nx3;
          if (lane == 31) lst[COOP3_LISTS] = total;
          __syncwarp();
          const int k0 = (lane * total) >> 5, k1 = ((lane + 1) * total) >> 5;
          if (k0 < k1) {
            int l = 0;  // the last list starting at or before k0
#pragma unroll
            for (int st = 32; st > 0; st >>= 1)
              if (lst[l + st] <= k0) l += st;
            int lend = lst[l + 1];
            int4 pa = tab[3 * l], pb = tab[3 * l + 1], pc = tab[3 * l + 2];
#pragma unroll 1
            for (int kk = k0; kk < k1; ++kk) {
              if (kk >= lend) {  // the next non-empty list
                do {
                  ++l;
                  lend = lst[l + 1];
                } while (lend <= kk);
                pa = tab[3 * l];
                pb = tab[3 * l + 1];
                pc = tab[3 * l + 2];
              }
              const float fk = small_int_float(kk - lst[l]);
              const int face = pa.x + (kk - lst[l]) * pa.y +
                               pa.z * min(ceil_count(fmaf(fk, __int_as_float(pb.w), __int_as_float(pb.z))), pa.w) +
                               pb.x * min(ceil_count(fmaf(fk, __int_as_float(pc.y), __int_as_float(pc.x))), pb.y);
              const double val = __hiloint2double(pc.w, pc.z);
              if (K32) tally_k32(&S.F32[face_off + face], val);
              else atomicAdd(&A.F[face_off + face], val);
            }
          }
          __syncwarp();
        }
      }
      // ---- face tallies of ended particles: up to walk_k per lane ----
      if (tally) {
        const int kstop = min(kend, kcur + S.walk_k);
        float fk = small_int_float(kcur);  // the item index in FP32, advanced without conversions
        // 64-bit sums kept as 32-bit low words in the window plus carries added to the FP64
        // face: the old word tells whether an addition wrapped (rare: words start at 2^31
        // and one contribution is at most 2^26)
        auto window_add = [&](int xface, unsigned rel) {
          const unsigned old = atomicAdd(&win[rel], qwx);
          if (old + 0x04000000u < 0x08000000u) {  // a wrap starts within 2^26 of 0 / 2^32
            const int carry = ((int)qwx >> 31) + (old + qwx < old ? 1 : 0);
            if (carry) atomicAdd(&A.F[face_off + xface], (double)carry * S.wmax[k] * WIN_CARRY);
          }
        };
        if (DIM == 2 && (two || wfull)) {
          // every face of the tallied axis is in the window at its instance index; the count
          // along the other axis needs only the upper bound (the lower one holds by
          // construction)
#pragma unroll 1
          for (; kcur < kstop; ++kcur, fk += 1.f) {
            const int face = f.i0 + kcur * f.s0 + f.s1 * min(ceil_count(fmaf(fk, f.tex, f.D)), f.i2);
            window_add(face, (unsigned)face);
          }
        } else {
#pragma unroll 1
          for (; kcur < kstop; ++kcur, fk += 1.f) {
            if (DIM == 3 && fk >= f.tex) {
              // y-face item: the (kcur - kx)-th face normal to y along the segment
              const float fm = fk - f.tex;  // exact: both are small integers
              const int mm = ceil_count(fm);
              const float tm = fmaf(fm, f.d1, f.t1);
              const int col = clampi(f.i0 + f.s0 * faces_before(tm, f.t0, f.d0), n0);
              const int lay = clampi(f.i2 + f.s2 * faces_before(tm, f.t2, f.d2), n2);
              const int jf = f.s1 > 0 ? f.i1 + 1 + mm : f.i1 - mm;
              const long long fi = face_off + fax1 + col + (long long)n0 * (jf + (long long)(n1 + 1) * lay);
              if (K32) tally_k32(&S.F32[fi], f.s1 > 0 ? w : -w);
              else atomicAdd(&A.F[fi], f.s1 > 0 ? w : -w);
              continue;
            }
            int xface = f.s0 > 0 ? f.i0 + 1 + kcur : f.i0 - kcur;
            if (DIM == 2) {
              xface += sy_xf * (f.i1 + f.s1 * min(ceil_count(fmaf(fk, f.tex, f.D)), f.i2));
            } else if (DIM == 3) {
              const float tk = fmaf(fk, f.d0, f.t0);
              xface += sy_xf * clampi(f.i1 + f.s1 * faces_before(tk, f.t1, f.d1), n1) +
                       sz_xf * clampi(f.i2 + f.s2 * faces_before(tk, f.t2, f.d2), n2);
            }
            const unsigned rel = (unsigned)(xface - wbase);
            if (rel < wlen) window_add(xface, rel);
            else if (K32) tally_k32(&S.F32[face_off + xface], f.s0 > 0 ? w : -w);
            else atomicAdd(&A.F[face_off + xface], f.s0 > 0 ? w : -w);
          }
        }
        if (kcur >= kend) {
          tally = false;
          alive = false;
        }
      }
    }
    if (ADJ && acc != 0.0) atomicAdd(&A.adj_wall[in.wall_off + (-1 - acc_slot)], acc);
    __syncthreads();
    if (wlen) {
      const double qs = wmax / WIN_SCALE;
      double* Fx = A.F + face_off + wbase;  // x-faces come first
      for (unsigned i = threadIdx.x; i < wlen; i += STAGED_NT) {
        const int v = (int)(win[i] - WIN_BIAS);
        if (v) atomicAdd(&Fx[i], (double)v * qs);
      }
    }
    __syncthreads();
  }
  flush_lcounts(cnt, A.counters);
}

// 2D instances whose tallied faces all sit in the window, pass by pass: every pass of a warp
// emits up to 32 particles (one per lane), follows each to its end (real collision or
// wall), and tallies the face items of all of them together (the cooperative tallies of
// sweep_staged_kernel). A particle's state lives only inside its pass, so the tally loop
// runs with the per-particle registers free. Same particles, draws and tallies as
// sweep_staged_kernel; chosen when the candidates per flight are few (each lane waits for
// the longest flight of its pass). REAL: tau = tau_maj in every cell of every instance and
// band, so every candidate is real and the acceptance test is left out. PARTIAL: some
// instance's x-faces exceed the window (a centred run of them sits there); the faces outside
// take global atomics of the same fixed-point contribution.
template <bool K32, bool REAL, bool PARTIAL>
__global__ void __launch_bounds__(STAGED_NT, 1) sweep_sync_kernel(SweepArgs A, StagedArgs S) {
  extern __shared__ unsigned win[];
  __shared__ int4 s_par[STAGED_NT / 32][64];
  __shared__ int s_lst[STAGED_NT / 32][33];
  __shared__ int s_inst;
  LCounts cnt;
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) cnt.v[k] = 0;
  const int lane = threadIdx.x & 31;
  const int n_inst = S.n_inst;
  int start = 0;
  {
    const double pos = (blockIdx.x + 0.5) / gridDim.x * S.cost_total;
    while (start + 1 < n_inst && S.cost_prefix[start + 1] <= pos) ++start;
  }
  int4* par = s_par[threadIdx.x >> 5];
  int* lst = s_lst[threadIdx.x >> 5];
  for (int visit = 0; visit < n_inst; ++visit) {
    const int k = (start + visit) % n_inst;
    if (threadIdx.x == 0) s_inst = (*(volatile unsigned long long*)&S.inst_next[k] < (unsigned long long)S.inst_end[k]) ? k : -1;
    __syncthreads();
    if (s_inst < 0) {
      __syncthreads();
      continue;
    }
    const InstDesc& in = A.inst[k];
    const int n0 = in.n[0], n1 = in.n[1];
    const long long face_off = in.face_off, fax1 = in.fax_off[1];
    const int sy_xf = n0 + 1;
    const int wbase = PARTIAL ? S.window[k].x : 0;
    const unsigned wlen = (unsigned)S.window[k].y;
    // every face in the window (two-group tallies); else x-faces [wbase, wbase + wlen)
    const bool two = wbase == 0 && (long long)wlen == in.nfaces;
    for (unsigned i = threadIdx.x; i < wlen; i += STAGED_NT) win[i] = WIN_BIAS;
    __syncthreads();
    const double qinv = S.wmax[k] > 0.0 ? WIN_SCALE / S.wmax[k] : 0.0;
    const unsigned pend = (unsigned)S.inst_end[k];
    unsigned rbeg = 0, rend = 0;  // this warp's private particle range
    EmitCache ec;
    ec.g_first = 1;
    ec.g_end = 0;  // empty: forces a lookup on the first emission
    ec.e = -1;
    for (;;) {
      if (rbeg == rend) {  // private range used up: take the next one of the instance
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(&S.inst_next[k], (unsigned long long)S.warp_grab);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got >= pend) break;
        rbeg = (unsigned)got;
        rend = (unsigned)min(got + (unsigned long long)S.warp_grab, (unsigned long long)pend);
      }
      const unsigned take = min(32u, rend - rbeg);
      int nitem = 0;
      int4 pa_own, pb_own;  // this lane's item parameters, stored once its list slot is known
      if ((unsigned)lane < take) {
        double w;
        int band, emitter;
        PW f;
        Stream st;
        uint32_t ub;
        if (staged_emit<2, false>(A, S, rbeg + lane, true, w, band, f, st, ub, ec, in, k, emitter, two)) {
          cnt.v[CNT_FLIGHTS] += 1;
          const int qw = __double2loint(fma(w, qinv, 0x1.8p52));
          const bool yg = two && f.d0 < f.d1;
          const unsigned qwx = (unsigned)((yg ? f.s1 : f.s0) > 0 ? qw : -qw);
          const float vtm = A.vtm32[(long long)k * A.nb + band];
          const bool all_real = REAL || A.all_real[(long long)k * A.nb + band] != 0;
          const long long bcbase = in.bc_off + (long long)band * in.ncells;
          // candidates (Sec. 3.2) until the particle collides for real or reaches a wall; a
          // decision within rounding of the FP64 walk's defers the particle to the FP64 replay
          const int m0 = faces_to_wall(f.i0, f.s0, n0), m1 = faces_to_wall(f.i1, f.s1, n1);
          const float ea = vtm * TIE_LOG_ABS;
          float eD = fmaf(f.D, TIE_LOG_REL, ea);  // bound of |D - D_fp64|
          bool wall_exit = false, deferred = false;
          int fb0 = 0, fb1 = 0;  // faces before the latest candidate, per axis
          int kc = 0;            // candidates tallied
#pragma unroll 1
          for (;;) {
            const float base = fmaf(TIE_REL, f.D, eD);
            if (f.D - f.tex > base) {
              wall_exit = true;
              break;
            }
            if (f.tex - f.D <= fmaf(TIE_REL, f.tex, eD)) {  // at the first wall within rounding
              deferred = true;
              break;
            }
            bool near = false;  // a count within the bound of a face, found with it for all-real bands
            if (all_real) {
              fb0 = count_near(f.D, f.t0, f.d0, base, near);
              fb1 = count_near(f.D, f.t1, f.d1, base, near);
            } else {
              fb0 = faces_before(f.D, f.t0, f.d0);
              fb1 = faces_before(f.D, f.t1, f.d1);
            }
            const int cell = clampi(f.i0 + f.s0 * fb0, n0) + n0 * clampi(f.i1 + f.s1 * fb1, n1);
            const long long ci = bcbase + cell;
            const int oc = candidate_outcome<2>(A, bcbase, in.ncells, f, base, fb0, fb1, 0, cell, all_real, near, ub,
                                                n0, n1, 1, n0, 0);
            if (oc == CAND_DEFER) {
              deferred = true;
              break;
            }
            cnt.v[CNT_CANDIDATES] += 1;
            ++kc;
            if (!all_real) {  // else W = tau_maj R after the sweep
              if (K32 && S.W32) tally_k32(&S.W32[ci], w);
              else if (!K32 && A.W) atomicAdd(&A.W[ci], w);
            }
            if (oc == CAND_REAL) {
              cnt.v[CNT_REAL] += 1;
              if (K32) tally_k32(&S.R32[ci], w);
              else atomicAdd(&A.R[ci], w);
              if (yg) atomicAdd(&S.DY[in.cell_off + cell], w);
              break;
            }
            uint32_t uw;
            st.next_pair(uw, ub);
            const float ell = __fmul_rn(-__logf(word_uniform<float>(uw)), vtm);
            f.D = __fadd_rn(f.D, ell);
            eD = fmaf(f.D, TIE_SUM, fmaf(ell, TIE_LOG_REL, eD + ea));
          }
          // faces crossed before the end per axis: at a real collision those before its
          // candidate; at a wall the exit axis's count is known and the other axis's follows
          // from the exit distance (within rounding of one of its faces, near a cell corner,
          // the particle is deferred too)
          int ex = -1, c0, c1;
          if (wall_exit) {
            // the face count of the axis not exited, near a cell corner within rounding of
            // the FP64 walk's: deferred too
            const float bx = TIE_REL * f.tex;
            ex = f.i2;
            const int q = count_near(f.tex, ex == 0 ? f.t1 : f.t0, ex == 0 ? f.d1 : f.d0, bx, deferred);
            c0 = ex == 0 ? m0 - 1 : min(q, m0 - 1);
            c1 = ex == 1 ? m1 - 1 : min(q, m1 - 1);
          } else {
            c0 = min(fb0, m0 - 1);
            c1 = min(fb1, m1 - 1);
          }
          if (deferred) {
            defer_particle(S, rbeg + lane, ((unsigned)kc << 1) | (yg ? 1u : 0u));
          } else {
            if (wall_exit) cnt.v[CNT_WALL_EXITS] += 1;
            cnt.v[CNT_CROSSINGS] += c0 + c1;
            // face items along the tallied axis p: a0 + k sp + sq min(ceil(u0 + k r), lim)
            // p: the tallied axis (x for the x-group), q: the other one; selects, no branch
            const float tp = yg ? f.t1 : f.t0, tq = yg ? f.t0 : f.t1;
            const float dp = yg ? f.d1 : f.d0, dq = yg ? f.d0 : f.d1;
            const int cp = yg ? c1 : c0, mq = yg ? m0 : m1, axp = yg ? 1 : 0;
            if (ex == 1 - axp && (yg ? f.s0 : f.s1) < 0) {  // exit through the low q-wall
              if (two) {
                const int j = yg ? in.wface_off[0] + f.i1 + f.s1 * c1 : in.wface_off[2] + f.i0 + f.s0 * c0;
                atomicAdd(&S.gx()[in.bface_off + j], -w);
              } else {
                const int col = f.i0 + f.s0 * c0;
                if (K32) tally_k32(&S.F32[face_off + fax1 + col], -w);
                else atomicAdd(&A.F[face_off + fax1 + col], -w);
              }
            }
            nitem = cp + (ex == axp ? 1 : 0);
            const bool flat = !(dq < INFINITY);
            const float u0 = flat ? -1.f : __fdividef(tp - tq, dq);
            const float r = flat ? 0.f : __fdividef(dp, dq);
            const int lim = mq - 1;
            const int a0 = yg ? (int)fax1 + f.i0 + n0 * (f.i1 + (f.s1 > 0 ? 1 : 0))
                              : f.i0 + (f.s0 > 0 ? 1 : 0) + sy_xf * f.i1;
            const int sp = yg ? f.s1 * n0 : f.s0;
            const int sq = yg ? f.s0 : f.s1 * sy_xf;
            pa_own = make_int4(a0, sp, sq, lim);
            pb_own = make_int4(__float_as_int(u0), __float_as_int(r), (int)qwx, 0);
          }
        }
      }
      rbeg += take;
      // ---- the pass's face items: each lane's list is cut into segments of SEG items, the
      // segments are numbered in lane order and dealt to the lanes round-robin, 32 to a
      // round; a lane runs SEG steps of its segment with its list's parameters (no per-item
      // list check). Against contiguous chunks of the pass's items (a list change inside a
      // chunk at a different step on every lane): 2.46 -> 2.40 ms per bench-batch sweep (Kn
      // 10: -6 %, Kn 0.01, short lists: +3 %). The non-empty lists are stored in lane order
      // without gaps; segment g belongs to list (number of lists starting at or before g) - 1,
      // counted from a ballot of the lists starting before the round and an OR-reduction of
      // the start bits within it (no search through the starts in shared memory). ----
      constexpr int SEG = 8;
      const int nseg = (nitem + SEG - 1) / SEG;
      int incl = nseg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (total > 0) {
        const int first = incl - nseg;  // this lane's first segment
        const unsigned nonempty = __ballot_sync(0xffffffffu, nseg > 0);
        if (nseg > 0) {
          const int pos = __popc(nonempty & ((1u << lane) - 1u));
          lst[pos] = first;
          par[2 * pos] = pa_own;
          par[2 * pos + 1] = make_int4(pb_own.x, pb_own.y, pb_own.z, nitem);
        }
        __syncwarp();
        for (int r0 = 0; r0 < total; r0 += 32) {
          const bool starts_here = nseg > 0 && first >= r0 && first < r0 + 32;
          const unsigned bits = __reduce_or_sync(0xffffffffu, starts_here ? 1u << (first - r0) : 0u);
          const int before = __popc(__ballot_sync(0xffffffffu, nseg > 0 && first < r0));
          const int g = r0 + lane;
          if (g >= total) continue;
          const int l = before + __popc(bits & (0xffffffffu >> (31 - lane))) - 1;
          const int4 pa = par[2 * l], pb = par[2 * l + 1];
          const int kl0 = (g - lst[l]) * SEG;
          const int kn = min(SEG, pb.w - kl0);
#pragma unroll
          for (int t = 0; t < SEG; ++t) {
            if (t >= kn) break;
            const int kl = kl0 + t;
            const int face =
                pa.x + kl * pa.y +
                pa.z * min(ceil_count(fmaf(small_int_float(kl), __int_as_float(pb.y), __int_as_float(pb.x))), pa.w);
            const unsigned q = (unsigned)pb.z;
            const unsigned rel = (unsigned)(face - wbase);
            if (PARTIAL && rel >= wlen) {  // outside the window: the same contribution, globally
              const double val = (double)(int)q * (S.wmax[k] / WIN_SCALE);
              if (K32) tally_k32(&S.F32[face_off + face], val);
              else atomicAdd(&A.F[face_off + face], val);
              continue;
            }
            const unsigned old = atomicAdd(&win[rel], q);
            // |q| <= 2^26, so the word can wrap only from within 2^26 of 0 / 2^32
            if (old + 0x04000000u < 0x08000000u) {
              const int carry = ((int)q >> 31) + (old + q < old ? 1 : 0);
              if (carry) atomicAdd(&A.F[face_off + face], (double)carry * S.wmax[k] * WIN_CARRY);
            }
          }
        }
        __syncwarp();
      }
    }
    __syncthreads();
    {
      const double qs = S.wmax[k] / WIN_SCALE;
      double* Fx = A.F + face_off + wbase;
      for (unsigned i = threadIdx.x; i < wlen; i += STAGED_NT) {
        const int v = (int)(win[i] - WIN_BIAS);
        if (v) atomicAdd(&Fx[i], (double)v * qs);
      }
    }
    __syncthreads();
  }
  flush_lcounts(cnt, A.counters);
}

// The adjoint re-trace of 2D contexts, pass by pass: every pass of a warp emits up to 32
// particles (every emitter's, per unit emission temperature), follows each to its real
// collision or wall, and gathers c_p lambda[stop] / (V m_stop) into the particle's emitter
// cell (or its wall, summed per lane while the lane stays on one wall group). Same
// particles and draws as the per-lane-refill re-trace of sweep_staged_kernel<DIM, true>.
template <bool REAL>
__global__ void __launch_bounds__(STAGED_NT, 1) adjoint_sync_kernel(SweepArgs A, StagedArgs S) {
  __shared__ int s_inst;
  LCounts cnt;
#pragma unroll
  for (int k = 0; k < CNT_N; ++k) cnt.v[k] = 0;
  const int lane = threadIdx.x & 31;
  const int n_inst = S.n_inst;
  int start = 0;
  {
    const double pos = (blockIdx.x + 0.5) / gridDim.x * S.cost_total;
    while (start + 1 < n_inst && S.cost_prefix[start + 1] <= pos) ++start;
  }
  for (int visit = 0; visit < n_inst; ++visit) {
    const int k = (start + visit) % n_inst;
    if (threadIdx.x == 0) s_inst = (*(volatile unsigned long long*)&S.inst_next[k] < (unsigned long long)S.inst_end[k]) ? k : -1;
    __syncthreads();
    if (s_inst < 0) {
      __syncthreads();
      continue;
    }
    const InstDesc& in = A.inst[k];
    const int n0 = in.n[0], n1 = in.n[1];
    const unsigned pend = (unsigned)S.inst_end[k];
    unsigned rbeg = 0, rend = 0;  // this warp's private particle range
    EmitCache ec;
    ec.g_first = 1;
    ec.g_end = 0;  // empty: forces a lookup on the first emission
    ec.e = -1;
    int acc_slot = 0;  // wall slot of the pending per-lane wall sum
    double acc = 0.0;
    for (;;) {
      if (rbeg == rend) {  // private range used up: take the next one of the instance
        unsigned long long got = 0;
        if (lane == 0) got = atomicAdd(&S.inst_next[k], (unsigned long long)S.warp_grab);
        got = __shfl_sync(0xffffffffu, got, 0);
        if (got >= pend) break;
        rbeg = (unsigned)got;
        rend = (unsigned)min(got + (unsigned long long)S.warp_grab, (unsigned long long)pend);
      }
      const unsigned take = min(32u, rend - rbeg);
      if ((unsigned)lane < take) {
        double w;
        int band, emitter;
        PW f;
        Stream st;
        uint32_t ub;
        if (staged_emit<2, true>(A, S, rbeg + lane, false, w, band, f, st, ub, ec, in, k, emitter, false)) {
          if (emitter < 0 && emitter != acc_slot) {
            if (acc != 0.0) atomicAdd(&A.adj_wall[in.wall_off + (-1 - acc_slot)], acc);
            acc = 0.0;
            acc_slot = emitter;
          }
          cnt.v[CNT_FLIGHTS] += 1;
          const float vtm = A.vtm32[(long long)k * A.nb + band];
          const bool all_real = REAL || A.all_real[(long long)k * A.nb + band] != 0;
          const long long bcbase = in.bc_off + (long long)band * in.ncells;
          // the forward sweep's decisions, with the same deferrals to the FP64 replay
          const int m0 = faces_to_wall(f.i0, f.s0, n0), m1 = faces_to_wall(f.i1, f.s1, n1);
          const float ea = vtm * TIE_LOG_ABS;
          float eD = fmaf(f.D, TIE_LOG_REL, ea);
          bool wall_exit = false, deferred = false;
          int fb0 = 0, fb1 = 0;  // faces before the latest candidate, per axis
#pragma unroll 1
          for (;;) {
            const float base = fmaf(TIE_REL, f.D, eD);
            if (f.D - f.tex > base) {
              cnt.v[CNT_WALL_EXITS] += 1;
              wall_exit = true;
              break;
            }
            if (f.tex - f.D <= fmaf(TIE_REL, f.tex, eD)) {
              deferred = true;
              break;
            }
            bool near = false;  // a count within the bound of a face, found with it for all-real bands
            if (all_real) {
              fb0 = count_near(f.D, f.t0, f.d0, base, near);
              fb1 = count_near(f.D, f.t1, f.d1, base, near);
            } else {
              fb0 = faces_before(f.D, f.t0, f.d0);
              fb1 = faces_before(f.D, f.t1, f.d1);
            }
            const int cell = clampi(f.i0 + f.s0 * fb0, n0) + n0 * clampi(f.i1 + f.s1 * fb1, n1);
            const int oc = candidate_outcome<2>(A, bcbase, in.ncells, f, base, fb0, fb1, 0, cell, all_real, near, ub,
                                                n0, n1, 1, n0, 0);
            if (oc == CAND_DEFER) {
              deferred = true;
              break;
            }
            cnt.v[CNT_CANDIDATES] += 1;
            if (oc == CAND_REAL) {
              cnt.v[CNT_REAL] += 1;
              const long long gc = in.cell_off + cell;
              const double val = w * A.lambda[gc] * A.invVm[gc];
              if (emitter >= 0) atomicAdd(&A.adj_out[in.cell_off + emitter], val);
              else acc += val;
              break;
            }
            uint32_t uw;
            st.next_pair(uw, ub);
            const float ell = __fmul_rn(-__logf(word_uniform<float>(uw)), vtm);
            f.D = __fadd_rn(f.D, ell);
            eD = fmaf(f.D, TIE_SUM, fmaf(ell, TIE_LOG_REL, eD + ea));
          }
          if (deferred) {
            defer_particle(S, rbeg + lane, 0u);
          } else {
            // faces crossed, for the event counters (as in the forward sweep)
            int c0, c1;
            if (wall_exit) {
              c0 = f.i2 == 0 ? m0 - 1 : min(faces_before(f.tex, f.t0, f.d0), m0 - 1);
              c1 = f.i2 == 1 ? m1 - 1 : min(faces_before(f.tex, f.t1, f.d1), m1 - 1);
            } else {
              c0 = min(fb0, m0 - 1);
              c1 = min(fb1, m1 - 1);
            }
            cnt.v[CNT_CROSSINGS] += c0 + c1;
          }
        }
      }
      rbeg += take;
    }
    if (acc != 0.0) atomicAdd(&A.adj_wall[in.wall_off + (-1 - acc_slot)], acc);
    __syncthreads();
  }
  flush_lcounts(cnt, A.counters);
}

// Absorbed minus emitted power of every cell, sum_b R_b - V m T_emit (T_emit = T + Q/m), in
// one pass over the [band][cell] tallies (coalesced; the column walk below then reads one
// value per cell instead of one per band).
__global__ void cell_balance_kernel(const InstDesc* inst, int n_inst, int nb, long long total, const double* T,
                                    const double* srcshift, const double* Vm, const double* R, double* out) {
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total; g += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < n_inst && inst[k + 1].cell_off <= g) ++k;
    const InstDesc& in = inst[k];
    const long long c = g - in.cell_off;
    double r = 0.0;
    for (int b = 0; b < nb; ++b) r += R[in.bc_off + (long long)b * in.ncells + c];
    double te = T[g];
    if (srcshift) te += srcshift[g];
    out[g] = r - Vm[g] * te;
  }
}

// Faces normal to the last axis from per-cell conservation, one thread per column:
// F[k+1] = F[k] + (net inflow through the other axes' faces of cell k) - (R_k - S_k),
// S_k = V m T_emit (emitted thermal and source power; bal = R - S from cell_balance_kernel),
// starting from the tallied low boundary face.
template <int DIM>
__device__ __forceinline__ double column_step(const InstDesc& in, const double* bal, const double* Fi, long long c) {
  const int n0 = in.n[0], n1 = in.n[1];
  const long long row = c / n0;  // x-face index of the cell's low face = c + row
  double inflow = Fi[in.fax_off[0] + c + row] - Fi[in.fax_off[0] + c + row + 1];
  if (DIM == 3) {
    const int cz = (int)(c / ((long long)n0 * n1));
    const long long fy = in.fax_off[1] + c + (long long)n0 * cz;
    inflow += Fi[fy] - Fi[fy + n0];
  }
  return inflow - bal[in.cell_off + c];
}

// Block: 32 adjacent columns x DERIVE_SEG segments (one warp per segment, so loads are
// coalesced across columns). Each thread sums its segment's increments, the segments'
// offsets follow from a prefix over the block's shared sums, then each thread writes its
// segment's running values.
constexpr int DERIVE_SEG = 8;

// A 2D instance whose faces all sit in the staged window uses the two-group tallies.
__device__ __forceinline__ bool two_group(const InstDesc& in, const int2* window, int k) {
  return in.dim == 2 && window[k].x == 0 && (long long)window[k].y == in.nfaces;
}

template <int DIM>
__global__ void __launch_bounds__(32 * DERIVE_SEG) derive_last_axis_kernel(const InstDesc* inst, int n_inst,
                                                                         const int2* window, const double* bal,
                                                                         double* F) {
  __shared__ double segsum[DERIVE_SEG][32];
  const int k = blockIdx.y;
  if (k >= n_inst) return;
  const InstDesc& in = inst[k];
  if (two_group(in, window, k)) return;
  const int n0 = in.n[0], n1 = in.n[1], n2 = in.n[2];
  const int nlast = DIM == 2 ? n1 : n2;
  const int ncol = in.ncells / nlast;
  double* Fi = F + in.face_off;
  const int lane = threadIdx.x & 31, seg = threadIdx.x >> 5;
  const int seglen = (nlast + DERIVE_SEG - 1) / DERIVE_SEG;
  const int k0 = seg * seglen, k1 = min(nlast, k0 + seglen);
  for (int cbase = blockIdx.x * 32; cbase < ncol; cbase += gridDim.x * 32) {
    const int col = cbase + lane;
    const bool ok = col < ncol;
    const int ix = ok ? col % n0 : 0, iy = (ok && DIM == 3) ? col / n0 : 0;
    const long long stride = DIM == 2 ? n0 : (long long)n0 * n1;
    const long long base_cell = DIM == 2 ? ix : ix + (long long)n0 * iy;
    double part = 0.0;
    if (ok)
      for (int kk = k0; kk < k1; ++kk) part += column_step<DIM>(in, bal, Fi, base_cell + kk * stride);
    segsum[seg][lane] = part;
    __syncthreads();
    if (ok) {
      // low boundary face of this column, then the segments below this one
      const long long f0 = DIM == 2 ? in.fax_off[1] + ix : in.fax_off[2] + ix + (long long)n0 * iy;
      double acc = Fi[f0];
      for (int sg = 0; sg < seg; ++sg) acc += segsum[sg][lane];
      for (int kk = k0; kk < k1; ++kk) {
        const long long c = base_cell + kk * stride;
        acc += column_step<DIM>(in, bal, Fi, c);
        const long long fn = DIM == 2 ? in.fax_off[1] + c + n0 : in.fax_off[2] + c + (long long)n0 * n1;
        Fi[fn] = acc;
      }
    }
    __syncthreads();
  }
  (void)n2;
}

// Faces of wall w = 2a + side of an instance, enumerated as j1 + n(o1) j2 (o1 = (a+1)%3,
// o2 = (a+2)%3); returns the face index within the instance.
__device__ __forceinline__ long long wall_face(const InstDesc& in, int a, int side, int j) {
  const int n0 = in.n[0], n1 = in.n[1], n2 = in.n[2];
  if (a == 0) {
    const int j1 = j % n1, j2 = j / n1;
    return in.fax_off[0] + (side ? n0 : 0) + (long long)(n0 + 1) * (j1 + (long long)n1 * j2);
  }
  if (a == 1) {
    const int j1 = j % n2, j2 = j / n2;
    return in.fax_off[1] + j2 + (long long)n0 * ((side ? n1 : 0) + (long long)(n1 + 1) * j1);
  }
  const int j1 = j % n0, j2 = j / n0;
  return in.fax_off[2] + j1 + (long long)n0 * (j2 + (long long)n1 * (side ? n2 : 0));
}

__device__ __forceinline__ int wall_faces(const InstDesc& in, int a) {
  return in.n[(a + 1) % 3] * in.n[(a + 2) % 3];
}

// Power entering through every boundary face from its wall's emission (N_w particles of
// weight C_b v_b A T_w / (4 N_w) per face and band), except on the high side of the
// derived axis (that axis is rebuilt from conservation). Grid: (faces, walls, instances).
__global__ void boundary_emission_kernel(const InstDesc* inst, int dim, const int2* window, const double* wall_unit,
                                         const double* wallTf, double* F) {
  const int k = blockIdx.z, wl = blockIdx.y;
  const int a = wl >> 1, side = wl & 1;
  if (dim >= 2 && a == dim - 1 && side == 1) return;
  const InstDesc& in = inst[k];
  if (two_group(in, window, k)) return;  // added with the group balances
  const double u = wall_unit[k * 6 + wl];
  const double* tf = wallTf + in.bface_off + in.wface_off[wl];
  const int nf = wall_faces(in, a);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nf; j += gridDim.x * blockDim.x) {
    const double e = u * tf[j];
    if (e != 0.0) F[in.face_off + wall_face(in, a, side, j)] += side ? -e : e;
  }
}

// Two-group instances (2D): the faces each group did not tally follow from that group's
// power balance in every cell. x-group, column i, faces normal to y from the bottom up:
//   G[j+1] = G[j] + (X[i,j] - X[i+1,j]) - ((R - S)_c - D_y,c),
// starting from the x-group's net flux through the bottom face (its exits there plus its
// share of the wall's emission, the whole emission minus the y-group's); X are the x-group's
// tallied faces plus its share of the emission on the x-walls. y-group, row j, faces
// normal to x from the left:
//   H[i+1] = H[i] + (Y[i,j] - Y[i,j+1]) - D_y,c,
// starting from its exits through the left wall and its emission there; Y are its tallied
// faces plus its emission on the y-walls. One warp per line, prefix sums over chunks of 32
// cells in a fixed order; results go to Fd (F is only read).
__global__ void __launch_bounds__(256) derive_two_group_kernel(const InstDesc* inst, int nb, const int2* window,
                                                               const double* T, const double* srcshift,
                                                               const double* Vm, const double* R,
                                                               const double* wall_unit, const double* wallTf,
                                                               const double* DY, const double* EY, const double* GX,
                                                               long long gx_stride, const double* F, double* Fd) {
  const int k = blockIdx.y;
  const InstDesc& in = inst[k];
  if (!two_group(in, window, k)) return;
  const int n0 = in.n[0], n1 = in.n[1];
  const int line = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (line >= n0 + n1) return;
  const double* Fi = F + in.face_off;
  double* Fo = Fd + in.face_off;
  const long long fax1 = in.fax_off[1];
  const double* ey = EY + in.bface_off;
  // the exit tally of boundary face j, summed over the copies of GX
  auto gx = [&](long long j) {
    double t = 0.0;
    for (int r = 0; r < GX_COPIES; ++r) t += GX[r * gx_stride + in.bface_off + j];
    return t;
  };
  const double* tf = wallTf + in.bface_off;
  const double* dy = DY + in.cell_off;
  // signed flux of the whole emission of wall wl through its face j
  auto etot = [&](int wl, int j) {
    const double e = wall_unit[k * 6 + wl] * tf[in.wface_off[wl] + j];
    return (wl & 1) ? -e : e;
  };
  if (line < n0) {
    const int i = line;
    double acc = gx(in.wface_off[2] + i) + etot(2, i) - ey[in.wface_off[2] + i];
    if (lane == 0) Fo[fax1 + i] = acc;
    for (int j0 = 0; j0 < n1; j0 += 32) {
      const int j = j0 + lane;
      double v = 0.0;
      if (j < n1) {
        const long long c = i + (long long)n0 * j;
        const long long fl = c + j;  // x-face (i, j)
        double left = Fi[fl], right = Fi[fl + 1];
        if (i == 0) left += etot(0, j) - ey[in.wface_off[0] + j];
        if (i == n0 - 1) right += etot(1, j) - ey[in.wface_off[1] + j];
        double rr = 0.0;
        for (int b = 0; b < nb; ++b) rr += R[in.bc_off + (long long)b * in.ncells + c];
        double te = T[in.cell_off + c];
        if (srcshift) te += srcshift[in.cell_off + c];
        v = (left - right) - (rr - Vm[in.cell_off + c] * te - dy[c]);
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (j < n1) Fo[fax1 + i + (long long)n0 * (j + 1)] = acc + v;
      acc += __shfl_sync(0xffffffffu, v, 31);
    }
  } else {
    const int j = line - n0;
    double acc = gx(in.wface_off[0] + j) + ey[in.wface_off[0] + j];
    if (lane == 0) Fo[(long long)(n0 + 1) * j] = acc;
    for (int ib = 0; ib < n0; ib += 32) {
      const int i = ib + lane;
      double v = 0.0;
      if (i < n0) {
        const long long c = i + (long long)n0 * j;
        double bot = Fi[fax1 + c], top = Fi[fax1 + c + n0];
        if (j == 0) bot += ey[in.wface_off[2] + i];
        if (j == n1 - 1) top += ey[in.wface_off[3] + i];
        v = (bot - top) - dy[c];
      }
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
      }
      if (i < n0) Fo[(long long)(n0 + 1) * j + i + 1] = acc + v;
      acc += __shfl_sync(0xffffffffu, v, 31);
    }
  }
}

// Two-group instances: every face = its tallied group's sum + the other group's derived
// flux + the tallied group's share of the wall emission on boundary faces.
__global__ void assemble_two_group_kernel(const InstDesc* inst, const int2* window, const double* wall_unit,
                                          const double* wallTf, const double* EY, const double* Fd, double* F) {
  const int k = blockIdx.y;
  const InstDesc& in = inst[k];
  if (!two_group(in, window, k)) return;
  const int n0 = in.n[0], n1 = in.n[1];
  const long long X = in.fax_off[1];
  const double* ey = EY + in.bface_off;
  const double* tf = wallTf + in.bface_off;
  for (long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x; f < in.nfaces;
       f += (long long)gridDim.x * blockDim.x) {
    double add = Fd[in.face_off + f];
    if (f < X) {
      const int i = (int)(f % (n0 + 1)), j = (int)(f / (n0 + 1));
      if (i == 0) add += wall_unit[k * 6 + 0] * tf[in.wface_off[0] + j] - ey[in.wface_off[0] + j];
      if (i == n0) add += -wall_unit[k * 6 + 1] * tf[in.wface_off[1] + j] - ey[in.wface_off[1] + j];
    } else {
      const long long g = f - X;
      const int i = (int)(g % n0), jf = (int)(g / n0);
      if (jf == 0) add += ey[in.wface_off[2] + i];
      if (jf == n1) add += ey[in.wface_off[3] + i];
    }
    F[in.face_off + f] += add;
  }
}

// Absorbed power of each wall = its emission + the outward net flux through its faces.
// One block per (wall, instance); fixed-order reduction.
__global__ void __launch_bounds__(256) wall_absorbed_kernel(const InstDesc* inst, const double* wall_unit,
                                                            const double* wallTf, const double* F, double* wall) {
  __shared__ double sh[8], shT[8];
  const int k = blockIdx.y, wl = blockIdx.x;
  const int a = wl >> 1, side = wl & 1;
  const InstDesc& in = inst[k];
  const int nf = wall_faces(in, a);
  const double* tf = wallTf + in.bface_off + in.wface_off[wl];
  double sum = 0.0, tsum = 0.0;
  for (int j = threadIdx.x; j < nf; j += 256) {
    sum += F[in.face_off + wall_face(in, a, side, j)];
    tsum += tf[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sum += __shfl_down_sync(0xffffffffu, sum, o);
    tsum += __shfl_down_sync(0xffffffffu, tsum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    sh[threadIdx.x >> 5] = sum;
    shT[threadIdx.x >> 5] = tsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0, ts = 0.0;
    for (int w = 0; w < 8; ++w) {
      t += sh[w];
      ts += shT[w];
    }
    const double emitted = wall_unit[k * 6 + wl] * ts;  // sum over faces of their emission
    wall[in.wall_off + wl] = emitted + (side ? t : -t);
  }
}

template <bool K32>
void launch_sync(const Ctx* c, const SweepArgs& a, const StagedArgs& S, int blocks, size_t smem, cudaStream_t s) {
  if (c->all_real_all) {
    if (c->sync_partial) sweep_sync_kernel<K32, true, true><<<blocks, STAGED_NT, smem, s>>>(a, S);
    else sweep_sync_kernel<K32, true, false><<<blocks, STAGED_NT, smem, s>>>(a, S);
  } else {
    if (c->sync_partial) sweep_sync_kernel<K32, false, true><<<blocks, STAGED_NT, smem, s>>>(a, S);
    else sweep_sync_kernel<K32, false, false><<<blocks, STAGED_NT, smem, s>>>(a, S);
  }
}

cudaError_t launch_sweep_staged(const Ctx* c, const SweepArgs& a, cudaStream_t s) {
  StagedArgs S;
  S.n_inst = c->n_inst;
  S.inst_next = c->d_inst_next;
  S.inst_end = c->d_inst_end;
  S.cost_prefix = c->d_cost_prefix;
  S.cost_total = c->cost_total;
  S.window = c->d_window;
  S.wmax = reinterpret_cast<const double*>(c->d_wmax);
  S.warp_grab = c->opt.warp_grab > 0 ? c->opt.warp_grab : 256;
  S.walk_k = c->opt.walk_k > 0 ? c->opt.walk_k : 16;
  S.refill = c->opt.refill_lanes;
  S.group_mag = c->d_group_mag;
  S.mag_n0 = c->d_mag;
  S.mag_n1 = c->d_mag + c->n_inst;
  S.mag_wall = c->d_mag + 2 * c->n_inst;
  S.defer = c->d_defer;
  S.defer_n = c->d_defer_n;
  S.defer_cap = c->defer_cap;
  S.err = c->d_err;
  cudaError_t e = cudaMemcpyAsync(c->d_inst_next, c->d_inst_beg, c->n_inst * sizeof(long long),
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_wmax, 0, c->n_inst * sizeof(double), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_defer_n, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  group_wmax_kernel<<<c->wmax_blocks, 256, 0, s>>>(a, c->d_wmax_bpre, c->d_wmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smem = (size_t)c->staged_cap * sizeof(unsigned);
  const int blocks = c->sm_count * c->staged_blocks_per_sm;
  const bool two = a.F && c->dim == 2 && c->any_two_group;
  S.DY = c->d_DY;
  S.EY = c->d_EY;
  S.GX = c->d_GX;
  S.gx_stride = c->total_bfaces;
  if (two) {
    if ((e = cudaMemsetAsync(c->d_DY, 0, (size_t)c->total_cells * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_EY, 0, (size_t)c->total_bfaces * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->d_GX, 0, (size_t)GX_COPIES * c->total_bfaces * sizeof(double), s)) != cudaSuccess) return e;
  }
  const bool k32 = c->opt.tally == IUGKP_TALLY_STAGED_K32;
  // pass-synchronous schedule: refill only when all 32 lanes are idle (the default where it
  // applies)
  const bool sync = c->sync_ok && a.F && (c->opt.refill_lanes == 0 || c->opt.refill_lanes == 32);
  S.R32 = k32 ? c->d_R32 : nullptr;
  S.W32 = k32 && a.W ? c->d_W32 : nullptr;
  S.F32 = k32 && a.F ? c->d_F32 : nullptr;
  if (k32) {
    const size_t bc = (size_t)c->nb * c->total_cells;
    if ((e = cudaMemsetAsync(c->d_R32, 0, bc * sizeof(float2), s)) != cudaSuccess) return e;
    if (a.W && (e = cudaMemsetAsync(c->d_W32, 0, bc * sizeof(float2), s)) != cudaSuccess) return e;
    if (a.F && (e = cudaMemsetAsync(c->d_F32, 0, (size_t)c->total_faces * sizeof(float2), s)) != cudaSuccess)
      return e;
    switch (c->dim) {
      case 1: sweep_staged_kernel<1, false, true><<<blocks, STAGED_NT, smem, s>>>(a, S); break;
      case 2:
        if (sync) launch_sync<true>(c, a, S, blocks, smem, s);
        else sweep_staged_kernel<2, false, true><<<blocks, STAGED_NT, smem, s>>>(a, S);
        break;
      default: sweep_staged_kernel<3, false, true><<<blocks, STAGED_NT, smem, s>>>(a, S); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int fb = c->sm_count * 4;
    k32_finalize_kernel<<<fb, 256, 0, s>>>(c->d_R32, a.R, (long long)bc, 0);
    if (a.W) k32_finalize_kernel<<<fb, 256, 0, s>>>(c->d_W32, a.W, (long long)bc, 0);
    if (a.F) k32_finalize_kernel<<<fb, 256, 0, s>>>(c->d_F32, a.F, c->total_faces, 1);
    // the deferred particles add to the FP64 outputs (after the finalize, which overwrites R and W)
    if ((e = launch_replay(c, a, S, s)) != cudaSuccess) return e;
  } else {
    switch (c->dim) {
      case 1: sweep_staged_kernel<1, false, false><<<blocks, STAGED_NT, smem, s>>>(a, S); break;
      case 2:
        if (sync) launch_sync<false>(c, a, S, blocks, smem, s);
        else sweep_staged_kernel<2, false, false><<<blocks, STAGED_NT, smem, s>>>(a, S);
        break;
      default: sweep_staged_kernel<3, false, false><<<blocks, STAGED_NT, smem, s>>>(a, S); break;
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_replay(c, a, S, s)) != cudaSuccess) return e;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.W) {
    scale_by_taumaj_kernel<<<c->sm_count * 4, 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->d_taumaj, c->d_all_real,
                                                          a.R, a.W, (long long)c->nb * c->total_cells);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (a.F) {
    boundary_emission_kernel<<<dim3(8, 2 * c->dim, c->n_inst), 256, 0, s>>>(c->d_inst, c->dim, c->d_window,
                                                                           c->d_wall_unit, c->d_wallTf, a.F);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (a.F && c->dim >= 2 && !c->all_two_group) {
    // one block per 32 columns of the largest instance (columns of the last axis)
    long long maxcol = 0;
    for (const InstDesc& in : c->h_inst) maxcol = std::max<long long>(maxcol, in.ncells / (c->dim == 2 ? in.n[1] : in.n[2]));
    dim3 grid((unsigned)std::min<long long>((maxcol + 31) / 32, 4096), (unsigned)c->n_inst);
    // absorbed minus emitted power per cell, into the correction solve's scratch (free until
    // the Newton step, which runs after the sweep on the same stream)
    cell_balance_kernel<<<c->sm_count * 4, 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->total_cells, a.T, a.srcshift,
                                                        c->d_Vm, a.R, c->d_work);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (c->dim == 2)
      derive_last_axis_kernel<2><<<grid, 32 * DERIVE_SEG, 0, s>>>(c->d_inst, c->n_inst, c->d_window, c->d_work, a.F);
    else
      derive_last_axis_kernel<3><<<grid, 32 * DERIVE_SEG, 0, s>>>(c->d_inst, c->n_inst, c->d_window, c->d_work, a.F);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (two) {
    long long lines = 0, faces = 0;
    for (const InstDesc& in : c->h_inst) {
      lines = std::max<long long>(lines, in.n[0] + in.n[1]);
      faces = std::max<long long>(faces, in.nfaces);
    }
    derive_two_group_kernel<<<dim3((unsigned)((lines + 7) / 8), (unsigned)c->n_inst), 256, 0, s>>>(
        c->d_inst, c->nb, c->d_window, a.T, a.srcshift, c->d_Vm, a.R, c->d_wall_unit, c->d_wallTf, c->d_DY, c->d_EY,
        c->d_GX, c->total_bfaces, a.F, c->d_Fd);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    assemble_two_group_kernel<<<dim3((unsigned)std::min<long long>((faces + 255) / 256, 1024), (unsigned)c->n_inst), 256,
                                0, s>>>(c->d_inst, c->d_window, c->d_wall_unit, c->d_wallTf, c->d_EY, c->d_Fd, a.F);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (a.F && a.wall) {
    wall_absorbed_kernel<<<dim3(2 * c->dim, c->n_inst), 256, 0, s>>>(c->d_inst, c->d_wall_unit, c->d_wallTf, a.F,
                                                                    a.wall);
    e = cudaGetLastError();
  }
  return e;
}

// Adjoint re-trace with the staged kernel over every emitter (all groups).
cudaError_t launch_adjoint_staged(const Ctx* c, const SweepArgs& a, cudaStream_t s) {
  StagedArgs S;
  S.n_inst = c->n_inst;
  S.inst_next = c->d_inst_next;
  S.inst_end = c->d_all_end;
  S.cost_prefix = c->d_all_cost_prefix;
  S.cost_total = c->all_cost_total;
  S.window = c->d_window;
  S.wmax = reinterpret_cast<const double*>(c->d_wmax);
  S.warp_grab = c->opt.warp_grab > 0 ? c->opt.warp_grab : 256;
  S.walk_k = c->opt.walk_k > 0 ? c->opt.walk_k : 16;
  S.refill = c->opt.refill_lanes;
  S.group_mag = c->d_all_group_mag;
  S.mag_n0 = c->d_mag;
  S.mag_n1 = c->d_mag + c->n_inst;
  S.mag_wall = c->d_mag + 2 * c->n_inst;
  S.defer = c->d_defer;
  S.defer_n = c->d_defer_n;
  S.defer_cap = c->defer_cap;
  S.err = c->d_err;
  cudaError_t e = cudaMemcpyAsync(c->d_inst_next, c->d_all_beg, c->n_inst * sizeof(long long),
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c->d_defer_n, 0, sizeof(unsigned), s)) != cudaSuccess) return e;
  S.R32 = S.W32 = S.F32 = nullptr;
  S.DY = S.EY = S.GX = nullptr;
  S.gx_stride = 0;
  const int blocks = c->sm_count * c->adj_blocks_per_sm;
  if (c->dim == 2 && (c->opt.refill_lanes == 0 || c->opt.refill_lanes == 32)) {
    // pass-synchronous re-trace (refill only when all 32 lanes are idle)
    if (c->all_real_all) adjoint_sync_kernel<true><<<blocks, STAGED_NT, 0, s>>>(a, S);
    else adjoint_sync_kernel<false><<<blocks, STAGED_NT, 0, s>>>(a, S);
  } else {
    switch (c->dim) {
      case 1: sweep_staged_kernel<1, true, false><<<blocks, STAGED_NT, 0, s>>>(a, S); break;
      case 2: sweep_staged_kernel<2, true, false><<<blocks, STAGED_NT, 0, s>>>(a, S); break;
      default: sweep_staged_kernel<3, true, false><<<blocks, STAGED_NT, 0, s>>>(a, S); break;
    }
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_adjoint_replay(c, a, s);  // the deferred particles, in FP64
}

// Measured accuracy of the FP32 operations the tie bounds rely on, over every uniform the
// walk can draw ((2m + 1) 2^-24, m < 2^23), against FP64:
//  out[0] max |__logf(u) - ln u| / (TIE_LOG_ABS + (TIE_LOG_REL - 2^-23) |ln u|) (the log's
//         share of the bound on a flight length; <= 1 required);
//  out[1] max relative error of sincospif(2u), both outputs, in units of 2^-23;
//  out[2] max relative error of sqrtf(fmaf(-mu, mu, 1)), mu = 2u - 1, units of 2^-23;
//  out[3] max relative error of sqrtf(u) and sqrtf(1 - u), units of 2^-23;
//  out[4] max relative error of __fdividef(x, y) over pairs of uniforms, units of 2^-23.
// Results are max-reduced as the bit patterns of non-negative doubles.
__global__ void walk_bounds_kernel(unsigned long long* out) {
  double e[5] = {0, 0, 0, 0, 0};
  for (unsigned m = blockIdx.x * blockDim.x + threadIdx.x; m < (1u << 23); m += gridDim.x * blockDim.x) {
    const float u = word_uniform<float>(m << 9);
    const double ud = (double)u;
    const double lg = log(ud);
    e[0] = fmax(e[0], fabs((double)__logf(u) - lg) / ((double)TIE_LOG_ABS + ((double)TIE_LOG_REL - 0x1p-23) * fabs(lg)));
    float sp, cp;
    sincospif(2.f * u, &sp, &cp);
    double sd, cd;
    sincospi(2.0 * ud, &sd, &cd);
    e[1] = fmax(e[1], fmax(fabs(sp - sd) / fabs(sd), fabs(cp - cd) / fabs(cd)) * 0x1p23);
    const float mu = 2.f * u - 1.f;
    const double sn = sqrt(1.0 - (double)mu * (double)mu);
    e[2] = fmax(e[2], fabs((double)sqrtf(fmaf(-mu, mu, 1.f)) - sn) / sn * 0x1p23);
    e[3] = fmax(e[3], fmax(fabs((double)sqrtf(u) - sqrt(ud)) / sqrt(ud),
                           fabs((double)sqrtf(1.f - u) - sqrt(1.0 - ud)) / sqrt(1.0 - ud)) * 0x1p23);
    // pairs (u, u') with u' another uniform, the divisor scaled over several binades
    const float v = word_uniform<float>((m * 2654435761u) << 9) * __int_as_float((127 - (int)(m & 15u)) << 23);
    const double q = ud / (double)v;
    e[4] = fmax(e[4], fabs((double)__fdividef(u, v) - q) / q * 0x1p23);
  }
  for (int k = 0; k < 5; ++k) {
    double x = e[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&out[k], (unsigned long long)__double_as_longlong(x));
  }
}

cudaError_t launch_walk_bounds(unsigned long long* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, 5 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  walk_bounds_kernel<<<1024, 256, 0, s>>>(out);
  return cudaGetLastError();
}

// FP64 atomic additions to scattered addresses of an L2-resident array (the deposit tallies'
// access pattern): every thread adds to `per_thread` addresses spread by a multiplicative hash.
__global__ void atomic_rate_kernel(double* buf, unsigned mask, int per_thread) {
  const unsigned t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int k = 0; k < per_thread; ++k) {
    const unsigned a = ((t * 32u + (unsigned)k) * 2654435761u) & mask;
    atomicAdd(&buf[a], 1.0);
  }
}

cudaError_t measure_atomic_rate(int sm_count, double* out_rate) {
  const unsigned n = 1u << 20;  // 8 MB: L2-resident
  double* buf = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&buf, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(buf, 0, n * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sm_count * 8, threads = 256, per = 256;
  float ms = 0.f;
  if (e == cudaSuccess) {
    atomic_rate_kernel<<<blocks, threads>>>(buf, n - 1, per);  // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) atomic_rate_kernel<<<blocks, threads>>>(buf, n - 1, per);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e == cudaSuccess) *out_rate = 5.0 * blocks * threads * (double)per / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  return e;
}

// The relative bound the face-count decision needs, from the measured errors above (units of
// 2^-23): direction s = product of a square root and a sine/cosine (one more rounding), cell
// size h in FP32 (half an ulp), d = h / |s| (__fdividef), t = (1 - xi) d (one rounding), the
// quotient (D - t) / d (__fdividef) and the difference D - t (half an ulp each), and half an
// ulp for the distance to the face. Returned as a fraction of TIE_REL (<= 1 required).
double walk_bound_fraction(const double* m) {
  const double ulp = 0x1p-23;
  const double Es = (std::max(m[2], m[3]) + m[1] + 0.5) * ulp;
  const double Ed = 0.5 * ulp + Es + m[4] * ulp;
  const double Et = Ed + 0.5 * ulp;
  return (Et + Ed + m[4] * ulp + ulp) / (double)TIE_REL;
}

cudaError_t configure_staged(Ctx* c) {
  cudaError_t e = cudaSuccess;
  const size_t smem = (size_t)c->staged_cap * sizeof(unsigned);
  const void* fwd[6] = {(const void*)sweep_staged_kernel<1, false, false>, (const void*)sweep_staged_kernel<2, false, false>,
                        (const void*)sweep_staged_kernel<3, false, false>, (const void*)sweep_staged_kernel<1, false, true>,
                        (const void*)sweep_staged_kernel<2, false, true>, (const void*)sweep_staged_kernel<3, false, true>};
  for (const void* f : fwd)
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  const void* syn[8] = {(const void*)sweep_sync_kernel<false, false, false>, (const void*)sweep_sync_kernel<true, false, false>,
                        (const void*)sweep_sync_kernel<false, true, false>, (const void*)sweep_sync_kernel<true, true, false>,
                        (const void*)sweep_sync_kernel<false, false, true>, (const void*)sweep_sync_kernel<true, false, true>,
                        (const void*)sweep_sync_kernel<false, true, true>, (const void*)sweep_sync_kernel<true, true, true>};
  for (const void* f : syn)
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  int nb = 0, nk = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fwd[c->dim - 1], STAGED_NT, smem)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nk, fwd[c->dim + 2], STAGED_NT, smem)) != cudaSuccess) return e;
  nb = std::min(nb, nk);  // one grid size for both tally modes
  c->staged_blocks_per_sm = nb > 0 ? nb : 1;
  void* fa = c->dim == 1 ? (void*)sweep_staged_kernel<1, true, false>
                         : (c->dim == 2 ? (void*)sweep_staged_kernel<2, true, false> : (void*)sweep_staged_kernel<3, true, false>);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fa, STAGED_NT, 0)) != cudaSuccess) return e;
  c->adj_blocks_per_sm = nb > 0 ? nb : 1;
  return cudaSuccess;
}

}  // namespace iugkp
