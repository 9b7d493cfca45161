// Persistent null-collision population (arXiv 2506.09465 Sec. 3.2 steps (1)-(6)). Positions,
// directions and flight lengths in FP64 or FP32 (the context's tracking precision), weights
// and tallies in FP64.
//
// A fixed population of particles (the paper's count stays fixed, so one array holds it)
// makes one candidate flight per iteration. Every particle has a home: the cell of its last
// real collision, or the boundary face through which a wall last absorbed it. A particle
// whose last flight ended at its home is re-emitted from there with the home's equilibrium
// power shared by the particles that ended there in the previous iteration:
// w = S_{b,c} / N(b, c) in a cell (S = C_b T_emit V / tau_b, T_emit = T + Q/m), and
// w = (C_b v_b T_face A / 4) / N(b, face) on a face. A null candidate keeps its position,
// direction and weight and flies again. One thread per particle; state in structure-of-
// arrays form, read and written once per iteration (coalesced, streaming: the state does not
// displace the descriptors and the home powers from the caches). A slot's home word carries
// its due flag in the top bit. The face-home index of face bf of instance k, band b is
// home_off[k] - nb cell_off[k] + b nbf_k + bf (the homes less the cell homes before it).
//
// Slots of an instance: per band, N_b per cell in q-major order (slot q * ncells + cell, so
// neighbouring slots start in different cells and their tallies rarely meet at one
// address), then per band N_w,b per boundary face (slot q * faces + face), faces in wall
// order (-x, +x, -y, +y, -z, +z; on the wall normal to axis a the faces run over axes
// (a+1)%3 and (a+2)%3, the first fastest). Draws of slot
// k of instance i in iteration it: Philox counter (block, k, 0x80000000, band << 24 | it),
// key (seed low word, seed high word ^ instance id): the emission uniforms when the particle
// is re-emitted, then the (path, accept) pair of its flight.
#include <cuda_runtime.h>

#include "device.cuh"
#include "internal.h"

namespace iugkp {

namespace {

struct PArgs {
  const InstDesc* inst;
  int n_inst, nb;
  const long long* slot_off;   // [n_inst + 1]
  const long long* home_off;   // [n_inst + 1] offsets of the per-(band, home) counts
  const long long* nband;      // [n_inst * nb] thermal particles per cell and band
  const long long* nwall;      // [nb] particles per boundary face and band
  const double* T;
  const double* srcshift;
  const double* coef;          // [bc] C_b V / (tau N_b)
  const double* ratio64;       // [bc] tau_maj / tau
  const float* ratio32;        // [bc] tau_maj / tau in FP32
  const float* vtm32;          // [inst * nb] v_b tau_maj in FP32
  const int* all_real;         // [inst * nb] 1 where tau = tau_maj in every cell
  const unsigned* mag;         // [5 n_inst] division magics of n_x, n_y, and n((a+1)%3) per wall axis a
  const double* taumaj;        // [inst * nb]
  const double* v;             // [nb]
  const double* wcoef;         // [inst * nb * 6] C_b v_b A / (4 N_w)
  const double* wallTf;        // [boundary faces]
  void* state;                 // positions and directions: 6 arrays of n_slots Real
  double* pw;                  // [n_slots] weights
  const double* home_w;        // [homes] power per particle re-emitted from each home
  const int* band;
  unsigned* home;              // home index | DUE_BIT when due for re-emission
  const unsigned* n_prev;
  unsigned* n_new;             // [homes] counts of cell homes
  unsigned* f_new;             // [PERS_FACE_REPLICAS][face homes] counts of boundary-face homes
  long long n_fhomes;          // face homes of all instances and bands
  double* R;
  double* W;
  double* wall;
  unsigned long long* counters;
  unsigned long long seed;
  unsigned it;
  long long n_slots;
};

// Element i of a 3-vector with a runtime index, by selects on constant indices (the vectors
// stay in registers instead of local memory).
template <typename V>
__device__ __forceinline__ V pick(const V (&v)[3], int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}
template <typename V>
__device__ __forceinline__ void put(V (&v)[3], int i, V x) {
  v[0] = i == 0 ? x : v[0];
  v[1] = i == 1 ? x : v[1];
  v[2] = i == 2 ? x : v[2];
}

// Tracking-precision values without FP64-pipe conversions in the FP32 variant: the FP32
// cell sizes of the descriptor, integers below 2^23 turned into floats by placing them in
// the mantissa of 2^23, floor of a float in (-2^23, 2^23) by a round-down add of 2^23 (the
// FP32 variant's conversions otherwise issue on the slow FP64 pipe).
template <typename Real>
__device__ __forceinline__ Real cell_h(const InstDesc& in, int a);
template <>
__device__ __forceinline__ double cell_h<double>(const InstDesc& in, int a) { return in.h[a]; }
template <>
__device__ __forceinline__ float cell_h<float>(const InstDesc& in, int a) { return in.hf[a]; }

template <typename Real>
__device__ __forceinline__ Real int_to_real(int i) { return (Real)i; }
template <>
__device__ __forceinline__ float int_to_real<float>(int i) {
  return __int_as_float(0x4B000000 | i) - 8388608.0f;  // exact for 0 <= i < 2^23
}

// max(floor(y), 0)
template <typename Real>
__device__ __forceinline__ int floor_nonneg(Real y) { return max((int)floor(y), 0); }
template <>
__device__ __forceinline__ int floor_nonneg<float>(float y) {
  return max(__float_as_int(__fadd_rd(y, 8388608.0f)) - 0x4B000000, 0);
}

template <typename Real>
__device__ __forceinline__ Real mean_path(const PArgs& A, int k, int b, double tm);
template <>
__device__ __forceinline__ double mean_path<double>(const PArgs& A, int, int b, double tm) { return A.v[b] * tm; }
template <>
__device__ __forceinline__ float mean_path<float>(const PArgs& A, int k, int b, double) {
  return A.vtm32[(long long)k * A.nb + b];
}

template <typename Real>
__device__ __forceinline__ Real accept_ratio(const PArgs& A, long long jb);
template <>
__device__ __forceinline__ double accept_ratio<double>(const PArgs& A, long long jb) { return A.ratio64[jb]; }
template <>
__device__ __forceinline__ float accept_ratio<float>(const PArgs& A, long long jb) { return A.ratio32[jb]; }

// Quotients of the flight geometry (distance to a wall, position over cell size): IEEE
// division in FP64 tracking; in FP32 tracking the reciprocal approximation (2 ulp), well inside
// the FP32 rounding the positions carry anyway.
template <typename Real>
__device__ __forceinline__ Real quot(Real a, Real b) { return a / b; }
template <>
__device__ __forceinline__ float quot<float>(float a, float b) { return __fdividef(a, b); }

// Wall power: each thread sums its absorptions per wall of the instance it is in (one FP64
// add per absorption); a warp adds its sums, grouped by wall, to the block's shared copy when
// the instance of one of its lanes changes and at the end, and the block adds its copy to
// global memory once (every absorption adding to one of 2 dim addresses per instance in global
// memory would serialise at the L2).
constexpr int PERS_SHARED_WALLS = 384;

constexpr int PERS_NT = 256;            // threads per block of the step kernel
constexpr int PERS_SHARED_INST = 32;    // instance descriptors copied to shared memory
constexpr unsigned DUE_BIT = 0x80000000u;

// acc: the block's per-thread sums, [wall of the instance][thread] in shared memory.
template <int NW>
__device__ __forceinline__ void flush_wall_sums(double* acc, int k_acc, bool to_shared, double* swall, double* wall,
                                                int lane) {
#pragma unroll
  for (int q = 0; q < NW; ++q) {
    const double v = acc[q * PERS_NT + threadIdx.x];
    const int key = NW * k_acc + q;  // wall index: 2 dim per instance, in instance order
    unsigned pending = __ballot_sync(0xffffffffu, v != 0.0);
    while (pending) {
      const int lead = __shfl_sync(0xffffffffu, key, __ffs(pending) - 1);
      const bool mine = key == lead && v != 0.0;
      double x = mine ? v : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) {
        if (to_shared) atomicAdd(&swall[lead], x);
        else atomicAdd(&wall[lead], x);
      }
      pending &= ~__ballot_sync(0xffffffffu, mine);
    }
    acc[q * PERS_NT + threadIdx.x] = 0.0;
  }
}

template <int DIM, typename Real>
__global__ void __launch_bounds__(PERS_NT, 4) persistent_step_kernel(PArgs A) {
  constexpr int NW = 2 * DIM;
  __shared__ double swall[PERS_SHARED_WALLS];
  __shared__ double wacc[NW * PERS_NT];  // this thread's absorbed power per wall of instance k_acc
  __shared__ InstDesc sinst[PERS_SHARED_INST];
  const int n_walls = 2 * DIM * A.n_inst;
  const bool wall_shared = n_walls <= PERS_SHARED_WALLS;
  const bool inst_shared = A.n_inst <= PERS_SHARED_INST;
  for (int j = threadIdx.x; j < PERS_SHARED_WALLS; j += blockDim.x) swall[j] = 0.0;
  if (inst_shared) {
    const int words = A.n_inst * (int)(sizeof(InstDesc) / sizeof(int));
    for (int j = threadIdx.x; j < words; j += blockDim.x)
      reinterpret_cast<int*>(sinst)[j] = reinterpret_cast<const int*>(A.inst)[j];
  }
#pragma unroll
  for (int q = 0; q < NW; ++q) wacc[q * PERS_NT + threadIdx.x] = 0.0;
  __syncthreads();
  const InstDesc* INS = inst_shared ? sinst : A.inst;
  Real* px = reinterpret_cast<Real*>(A.state);
  const long long ns = A.n_slots;
  unsigned c_flights = 0, c_cand = 0, c_real = 0, c_exit = 0;
  const int lane = threadIdx.x & 31;
  int k = 0, k_acc = 0;
  long long k_beg = 0, k_end = A.slot_off[1];  // slots of instance k (slots only grow below)
  // per (instance, band): reloaded when either changes (bands change rarely along a thread's
  // slots, instances more rarely still)
  int kb = -1;
  double tm = 0.0;
  Real vtm = (Real)0;
  bool all_real = false;
  long long hbase = 0;  // offset of the (instance, band)'s homes
  long long fbase = 0;  // offset of its face homes among all face homes
  // every thread of a block runs the same number of passes, so warps are converged at the
  // start and end of each pass (for the warp sums of the wall tallies)
  for (long long base = (long long)blockIdx.x * blockDim.x; base < ns; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    if (i < ns)
      while (k + 1 < A.n_inst && k_end <= i) {
        k_beg = k_end;
        k_end = A.slot_off[++k + 1];
      }
    if (__any_sync(0xffffffffu, k != k_acc)) {
      flush_wall_sums<NW>(wacc, k_acc, wall_shared, swall, A.wall, lane);
      k_acc = k;
    }
    if (i >= ns) continue;
    const InstDesc& in = INS[k];
    const int b = __ldcs(A.band + i);
    const unsigned hw = __ldcs(A.home + i);
    Real x[3], s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x[a] = a < DIM ? __ldcs(px + a * ns + i) : (Real)0;
      s[a] = a < DIM ? __ldcs(px + (3 + a) * ns + i) : (Real)0;
    }
    double w = __ldcs(A.pw + i);
    int h = (int)(hw & ~DUE_BIT);
    const int n0 = in.n[0], n1 = in.n[1];
    if (k * A.nb + b != kb) {
      kb = k * A.nb + b;
      tm = A.taumaj[kb];
      vtm = mean_path<Real>(A, k, b, tm);
      all_real = A.all_real[kb] != 0;
      const int nbf = in.wface_off[2 * DIM - 1] + in.n[((2 * DIM - 1) / 2 + 1) % 3] * in.n[((2 * DIM - 1) / 2 + 2) % 3];
      hbase = A.home_off[k] + (long long)b * ((long long)in.ncells + nbf);
      fbase = A.home_off[k] - (long long)A.nb * in.cell_off + (long long)b * nbf;
    }
    Stream st;  // block 0 is computed by the emission, or else by the flight's draw
    st.init_lazy(A.seed, in.inst_id, (uint32_t)b, A.it, 0x80000000u, (uint32_t)(i - k_beg));
    if (hw & DUE_BIT) {
      w = A.home_w[hbase + h];
      st.load_block(0);
      if (h < in.ncells) {
        // re-emission in the cell of the real collision (Sec. 3.2 step (2))
        const unsigned r0 = udiv((unsigned)h, (unsigned)n0, A.mag[k]);
        const unsigned r1 = DIM == 3 ? udiv(r0, (unsigned)n1, A.mag[A.n_inst + k]) : 0u;
        const int ci[3] = {h - (int)r0 * n0, (int)(r0 - r1 * (unsigned)n1), (int)r1};
        const Real hx = cell_h<Real>(in, 0), hy = cell_h<Real>(in, 1), hz = cell_h<Real>(in, 2);
        Real u_mu, u_phi = (Real)0.5;
        if (DIM == 1) {
          x[0] = (int_to_real<Real>(ci[0]) + word_uniform<Real>(st.buf.x)) * hx;
          u_mu = word_uniform<Real>(st.buf.y);
        } else if (DIM == 2) {
          x[0] = (int_to_real<Real>(ci[0]) + word_uniform<Real>(st.buf.x)) * hx;
          x[1] = (int_to_real<Real>(ci[1]) + word_uniform<Real>(st.buf.y)) * hy;
          u_mu = word_uniform<Real>(st.buf.z);
          u_phi = word_uniform<Real>(st.buf.w);
        } else {
          x[0] = (int_to_real<Real>(ci[0]) + word_uniform<Real>(st.buf.x)) * hx;
          x[1] = (int_to_real<Real>(ci[1]) + word_uniform<Real>(st.buf.y)) * hy;
          x[2] = (int_to_real<Real>(ci[2]) + word_uniform<Real>(st.buf.z)) * hz;
          u_mu = word_uniform<Real>(st.buf.w);
          st.load_block(1);
          u_phi = word_uniform<Real>(st.buf.x);
        }
        const Real mu = (Real)2 * u_mu - (Real)1;
        s[0] = mu;
        if (DIM >= 2) {
          const Real sn = sqrt((Real)1 - mu * mu);
          Real sp, cp;
          RealTraits<Real>::sincos2pi(u_phi, &sp, &cp);
          s[1] = sn * cp;
          s[2] = sn * sp;
        }
        st.j = thermal_uniforms(DIM);
      } else {
        // re-emission from the boundary face that absorbed it (black wall)
        const int bf = h - in.ncells;
        int wl = 0;
        while (wl + 1 < 2 * DIM && bf >= in.wface_off[wl + 1]) ++wl;
        const int a = wl >> 1, side = wl & 1, o1 = (a + 1) % 3, o2 = (a + 2) % 3;
        const int j = bf - in.wface_off[wl];
        const int no1 = in.n[o1];
        const int jq = (int)udiv((unsigned)j, (unsigned)no1, A.mag[2 * A.n_inst + 3 * k + a]);
        int f[3] = {0, 0, 0};
        put(f, a, side ? in.n[a] : 0);
        put(f, o1, j - jq * no1);
        put(f, o2, jq);
        Real u_n, u_phi = (Real)0.5;
        if (DIM == 1) {
          u_n = word_uniform<Real>(st.buf.x);
        } else if (DIM == 2) {
          const int t = (o1 < 2) ? o1 : o2;
          put(x, t, (int_to_real<Real>(pick(f, t)) + word_uniform<Real>(st.buf.x)) * cell_h<Real>(in, t));
          u_n = word_uniform<Real>(st.buf.y);
          u_phi = word_uniform<Real>(st.buf.z);
        } else {
          const int t0 = o1 < o2 ? o1 : o2, t1 = o1 < o2 ? o2 : o1;
          put(x, t0, (int_to_real<Real>(pick(f, t0)) + word_uniform<Real>(st.buf.x)) * cell_h<Real>(in, t0));
          put(x, t1, (int_to_real<Real>(pick(f, t1)) + word_uniform<Real>(st.buf.y)) * cell_h<Real>(in, t1));
          u_n = word_uniform<Real>(st.buf.z);
          u_phi = word_uniform<Real>(st.buf.w);
        }
        put(x, a, int_to_real<Real>(pick(f, a)) * cell_h<Real>(in, a));
        const Real mn = sqrt(u_n);
        put(s, a, side ? -mn : mn);
        if (DIM >= 2) {
          const Real stn = sqrt((Real)1 - u_n);
          Real sp, cp;
          RealTraits<Real>::sincos2pi(u_phi, &sp, &cp);
          put(s, o1, stn * cp);
          put(s, o2, stn * sp);
        } else {
          put(s, o1, (Real)0);
          put(s, o2, (Real)0);
        }
        st.j = wall_uniforms(DIM);
      }
    }
    // one flight (Sec. 3.2 step (3)): path -ln(u) v tau_maj
    c_flights += 1;
    uint32_t ua, ub;
    st.next_pair(ua, ub);
    const Real ell = -RealTraits<Real>::log_(word_uniform<Real>(ua)) * vtm;
    Real tw = RealTraits<Real>::inf();
    int wl = -1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (s[a] == (Real)0) continue;
      const Real L = cell_h<Real>(in, a) * int_to_real<Real>(in.n[a]);
      const Real t = quot<Real>(s[a] > (Real)0 ? L - x[a] : -x[a], s[a]);
      if (t < tw) {
        tw = t;
        wl = 2 * a + (s[a] > (Real)0 ? 1 : 0);
      }
    }
    unsigned due = DUE_BIT;
    if (wl >= 0 && tw < ell) {
      // absorbed by the wall it reaches first; its home is the face it crossed
      c_exit += 1;
      wacc[wl * PERS_NT + threadIdx.x] += w;
      const int a = wl >> 1, o1 = (a + 1) % 3, o2 = (a + 2) % 3;
      int j1 = 0, j2 = 0;
      if (o1 < DIM) j1 = min(floor_nonneg<Real>(quot<Real>(pick(x, o1) + tw * pick(s, o1), cell_h<Real>(in, o1))), in.n[o1] - 1);
      if (o2 < DIM) j2 = min(floor_nonneg<Real>(quot<Real>(pick(x, o2) + tw * pick(s, o2), cell_h<Real>(in, o2))), in.n[o2] - 1);
      const int bf = in.wface_off[wl] + j2 * in.n[o1] + j1;
      h = in.ncells + bf;
      atomicAdd(&A.f_new[(long long)lane * A.n_fhomes + fbase + bf], 1u);
    } else {
      int ci[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        x[a] += ell * s[a];
        ci[a] = min(floor_nonneg<Real>(quot<Real>(x[a], cell_h<Real>(in, a))), in.n[a] - 1);
      }
      const int c = ci[0] + n0 * (ci[1] + n1 * ci[2]);
      // candidate (steps (4)-(5)): W from every candidate, R and the count from real ones;
      // W collects w here and is scaled by tau_maj afterwards, and a band with tau = tau_maj
      // in every cell accepts every candidate (the uniform is below 1), so its W is tau_maj R
      c_cand += 1;
      const long long jb = in.bc_off + (long long)b * in.ncells + c;
      if (all_real || word_uniform<Real>(ub) < accept_ratio<Real>(A, jb)) {
        c_real += 1;
        if (!all_real) atomicAdd(&A.W[jb], w);
        atomicAdd(&A.R[jb], w);
        h = c;
        atomicAdd(&A.n_new[hbase + h], 1u);
      } else {
        atomicAdd(&A.W[jb], w);
        due = 0u;  // step (6): same direction and weight, a new path next iteration
      }
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      __stcs(px + a * ns + i, x[a]);
      __stcs(px + (3 + a) * ns + i, s[a]);
    }
    __stcs(A.pw + i, w);
    __stcs(A.home + i, (unsigned)h | due);
  }
  flush_wall_sums<NW>(wacc, k_acc, wall_shared, swall, A.wall, lane);
  __syncthreads();
  if (wall_shared)
    for (int j = threadIdx.x; j < n_walls; j += blockDim.x)
      if (swall[j] != 0.0) atomicAdd(&A.wall[j], swall[j]);
  unsigned long long vals[4] = {c_flights, c_cand, c_real, c_exit};
  const int slots[4] = {CNT_FLIGHTS, CNT_CANDIDATES, CNT_REAL, CNT_WALL_EXITS};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    unsigned long long v = vals[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&A.counters[slots[q]], v);
  }
}

// W of the step: the kernel summed w per candidate, or nothing for bands whose every
// candidate is real (there W = tau_maj R); both are scaled by the instance's tau_maj here.
__global__ void persistent_finish_W_kernel(const InstDesc* inst, int n_inst, int nb, const double* taumaj,
                                           const int* all_real, const double* R, double* W, long long total) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < total; j += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < n_inst && inst[k + 1].bc_off <= j) ++k;
    const int kb = k * nb + (int)((j - inst[k].bc_off) / inst[k].ncells);
    W[j] = (all_real[kb] ? R[j] : W[j]) * taumaj[kb];
  }
}

// Power per particle re-emitted from each (band, home) this iteration: the home's power
// (C_b T_emit V / tau_b for a cell, C_b v_b T_face A / 4 for a boundary face) over the
// particles that ended there in the previous iteration (0 where none did).
__global__ void persistent_home_power_kernel(const InstDesc* inst, int n_inst, int nb, const long long* home_off,
                                             const long long* nband, const long long* nwall, const double* T,
                                             const double* srcshift, const double* coef, const double* wcoef,
                                             const double* wallTf, const unsigned* n_prev, const unsigned* f_prev,
                                             long long n_fhomes, double* home_w, long long n_homes) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n_homes;
       j += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < n_inst && home_off[k + 1] <= j) ++k;
    const InstDesc& in = inst[k];
    const long long nh = (home_off[k + 1] - home_off[k]) / nb;
    const long long r = j - home_off[k];
    const int b = (int)(r / nh);
    const long long h = r - (long long)b * nh;
    unsigned n = 0;
    if (h < in.ncells) {
      n = n_prev[j];
    } else {
      const long long f = home_off[k] - (long long)nb * in.cell_off + (long long)b * (nh - in.ncells) + (h - in.ncells);
#pragma unroll 8
      for (int q = 0; q < PERS_FACE_REPLICAS; ++q) n += f_prev[(long long)q * n_fhomes + f];
    }
    double pw = 0.0;
    if (n > 0) {
      if (h < in.ncells) {
        double te = T[in.cell_off + h];
        if (srcshift) te += srcshift[in.cell_off + h];
        // C_b V / tau_{b,c} = coef * N_b
        pw = coef[in.bc_off + (long long)b * in.ncells + h] * (double)nband[(long long)k * nb + b] * te / (double)n;
      } else {
        const int bf = (int)(h - in.ncells);
        int wl = 0;
        while (wl + 1 < 2 * in.dim && bf >= in.wface_off[wl + 1]) ++wl;
        pw = wcoef[((long long)k * nb + b) * 6 + wl] * (double)nwall[b] * wallTf[in.bface_off + bf] / (double)n;
      }
    }
    home_w[j] = pw;
  }
}

}  // namespace

cudaError_t launch_persistent_step(const Ctx* c, const double* T, unsigned it, double* R, double* W, double* wall,
                                   unsigned long long* counters, cudaStream_t s) {
  PArgs a;
  a.inst = c->d_inst;
  a.n_inst = c->n_inst;
  a.nb = c->nb;
  a.slot_off = c->d_pslot_off;
  a.home_off = c->d_phome_off;
  a.nband = c->d_pnband;
  a.nwall = c->d_pnwall;
  a.T = T;
  a.srcshift = c->d_srcshift;
  a.coef = c->d_coef;
  a.ratio64 = c->d_ratio64;
  a.ratio32 = c->d_ratio32;
  a.vtm32 = c->d_vtm32;
  a.all_real = c->d_all_real;
  a.mag = c->d_mag;
  a.taumaj = c->d_taumaj;
  a.v = c->d_v;
  a.wcoef = c->d_wcoef;
  a.wallTf = c->d_wallTf;
  a.state = c->d_px;
  a.pw = reinterpret_cast<double*>(c->d_px) + 6 * c->pers_n;  // after 6 arrays of FP64 or FP32
  a.home_w = c->d_phome_w;
  a.band = c->d_pband;
  a.home = reinterpret_cast<unsigned*>(c->d_phome);
  a.n_prev = c->d_pcount + (c->pers_parity ? c->pers_homes : 0);
  a.n_new = c->d_pcount + (c->pers_parity ? 0 : c->pers_homes);
  a.n_fhomes = c->pers_homes - (long long)c->nb * c->total_cells;
  const long long fr = (long long)PERS_FACE_REPLICAS * a.n_fhomes;
  const unsigned* f_prev = c->d_pfcount + (c->pers_parity ? fr : 0);
  a.f_new = c->d_pfcount + (c->pers_parity ? 0 : fr);
  a.R = R;
  a.W = W;
  a.wall = wall;
  a.counters = counters;
  a.seed = c->opt.seed;
  a.it = it;
  a.n_slots = c->pers_n;
  {
    const unsigned hb = (unsigned)std::min<long long>((c->pers_homes + 255) / 256 + 1, (long long)c->sm_count * 16);
    persistent_home_power_kernel<<<hb, 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->d_phome_off, c->d_pnband,
                                                    c->d_pnwall, T, c->d_srcshift, c->d_coef, c->d_wcoef, c->d_wallTf,
                                                    a.n_prev, f_prev, a.n_fhomes, c->d_phome_w, c->pers_homes);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long long want = (c->pers_n + PERS_NT - 1) / PERS_NT;
  const unsigned blocks = (unsigned)std::min<long long>(std::max<long long>(want, 1), (long long)c->sm_count * 16);
  const bool f32 = c->opt.precision == IUGKP_TRACK_FP32;
  switch (c->dim * 2 + (f32 ? 1 : 0)) {
    case 2: persistent_step_kernel<1, double><<<blocks, PERS_NT, 0, s>>>(a); break;
    case 3: persistent_step_kernel<1, float><<<blocks, PERS_NT, 0, s>>>(a); break;
    case 4: persistent_step_kernel<2, double><<<blocks, PERS_NT, 0, s>>>(a); break;
    case 5: persistent_step_kernel<2, float><<<blocks, PERS_NT, 0, s>>>(a); break;
    case 6: persistent_step_kernel<3, double><<<blocks, PERS_NT, 0, s>>>(a); break;
    default: persistent_step_kernel<3, float><<<blocks, PERS_NT, 0, s>>>(a); break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !W) return e;
  persistent_finish_W_kernel<<<c->sm_count * 4, 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->d_taumaj, c->d_all_real,
                                                             R, W, (long long)c->nb * c->total_cells);
  return cudaGetLastError();
}

}  // namespace iugkp

namespace iugkp {

namespace {

// Initial population (Sec. 3.2 step (1)): every slot due for emission from its home, and
// every home counted with its own number of slots.
__global__ void persistent_init_kernel(const InstDesc* inst, int n_inst, int nb, const long long* slot_off,
                                       const long long* home_off, const long long* nband, const long long* nwall,
                                       long long n_slots, long long n_homes, double* state, int* band, unsigned* home,
                                       unsigned* count_prev, unsigned* fcount_prev) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_slots; i += stride) {
    int k = 0;
    while (k + 1 < n_inst && slot_off[k + 1] <= i) ++k;
    const InstDesc& in = inst[k];
    long long r = i - slot_off[k];
    int b = 0, h = 0;
    long long thermal = 0;
    for (int bb = 0; bb < nb; ++bb) thermal += nband[(long long)k * nb + bb] * in.ncells;
    if (r < thermal) {
      while (r >= nband[(long long)k * nb + b] * in.ncells) r -= nband[(long long)k * nb + b] * in.ncells, ++b;
      h = (int)(r % in.ncells);
    } else {
      r -= thermal;
      const long long nbf = (home_off[k + 1] - home_off[k]) / nb - in.ncells;
      while (r >= nwall[b] * nbf) r -= nwall[b] * nbf, ++b;
      h = in.ncells + (int)(r % nbf);
    }
    band[i] = b;
    home[i] = (unsigned)h | DUE_BIT;
    for (int q = 0; q < 7; ++q) state[q * n_slots + i] = 0.0;
  }
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n_homes; j += stride) {
    int k = 0;
    while (k + 1 < n_inst && home_off[k + 1] <= j) ++k;
    const InstDesc& in = inst[k];
    const long long nh = (home_off[k + 1] - home_off[k]) / nb;
    const long long r = j - home_off[k];
    const int b = (int)(r / nh);
    const long long h = r - (long long)b * nh;
    if (h < in.ncells) count_prev[j] = (unsigned)nband[(long long)k * nb + b];
    else fcount_prev[home_off[k] - (long long)nb * in.cell_off + (long long)b * (nh - in.ncells) + (h - in.ncells)] =
        (unsigned)nwall[b];  // copy 0 of the face's counts (the others are cleared)
  }
}

}  // namespace

cudaError_t launch_persistent_init(Ctx* c, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<long long>((c->pers_n + 255) / 256 + 1, (long long)c->sm_count * 16);
  persistent_init_kernel<<<blocks, 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->d_pslot_off, c->d_phome_off, c->d_pnband,
                                                c->d_pnwall, c->pers_n, c->pers_homes, c->d_px, c->d_pband,
                                                reinterpret_cast<unsigned*>(c->d_phome), c->d_pcount, c->d_pfcount);
  return cudaGetLastError();
}

}  // namespace iugkp
