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
// arrays form, read and written once per iteration (coalesced).
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
  const double* taumaj;        // [inst * nb]
  const double* v;             // [nb]
  const double* wcoef;         // [inst * nb * 6] C_b v_b A / (4 N_w)
  const double* wallTf;        // [boundary faces]
  void* state;                 // positions and directions: 6 arrays of n_slots Real
  double* pw;                  // [n_slots] weights
  const double* home_w;        // [homes] power per particle re-emitted from each home
  const int* band;
  int* home;
  int* due;
  const unsigned* n_prev;
  unsigned* n_new;
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

// Wall power is accumulated per block in shared memory and flushed once: every absorption
// adding to one of 2 dim addresses per instance in global memory would serialise at the L2.
constexpr int PERS_SHARED_WALLS = 384;

template <int DIM, typename Real>
__global__ void __launch_bounds__(256, 4) persistent_step_kernel(PArgs A) {
  __shared__ double swall[PERS_SHARED_WALLS];
  const int n_walls = 2 * DIM * A.n_inst;
  const bool wall_shared = n_walls <= PERS_SHARED_WALLS;
  for (int j = threadIdx.x; j < PERS_SHARED_WALLS; j += blockDim.x) swall[j] = 0.0;
  __syncthreads();
  Real* px = reinterpret_cast<Real*>(A.state);
  Real* py = px + A.n_slots;
  Real* pz = px + 2 * A.n_slots;
  Real* sx = px + 3 * A.n_slots;
  Real* sy = px + 4 * A.n_slots;
  Real* sz = px + 5 * A.n_slots;
  unsigned c_flights = 0, c_cand = 0, c_real = 0, c_exit = 0;
  const int lane = threadIdx.x & 31;
  // every thread of a block runs the same number of passes, so warps are converged at the
  // end of each pass (for the warp reduction of the wall tallies)
  for (long long base = (long long)blockIdx.x * blockDim.x; base < A.n_slots;
       base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    int exit_key = -1;  // global wall index of this pass's absorption, if any
    double exit_w = 0.0;
    if (i < A.n_slots) {
    int k = 0;
    while (k + 1 < A.n_inst && A.slot_off[k + 1] <= i) ++k;
    const InstDesc& in = A.inst[k];
    const long long local = i - A.slot_off[k];
    const int b = A.band[i];
    const int n0 = in.n[0], n1 = in.n[1], n2 = in.n[2];
    const int nbf = in.wface_off[2 * DIM - 1] + in.n[((2 * DIM - 1) / 2 + 1) % 3] * in.n[((2 * DIM - 1) / 2 + 2) % 3];
    const long long nh = (long long)in.ncells + nbf;  // homes per band
    Stream st;
    st.init(A.seed, in.inst_id, (uint32_t)b, A.it, 0x80000000u, (uint32_t)local);
    Real x[3] = {px[i], DIM >= 2 ? py[i] : (Real)0, DIM >= 3 ? pz[i] : (Real)0};
    Real s[3] = {sx[i], DIM >= 2 ? sy[i] : (Real)0, DIM >= 3 ? sz[i] : (Real)0};
    double w = A.pw[i];
    int h = A.home[i];
    st.j = 0;
    if (A.due[i]) {
      w = A.home_w[A.home_off[k] + (long long)b * nh + h];
      if (h < in.ncells) {
        // re-emission in the cell of the real collision (Sec. 3.2 step (2))
        const int ci[3] = {h % n0, (h / n0) % n1, h / (n0 * n1)};
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
        int f[3] = {0, 0, 0};
        put(f, a, side ? in.n[a] : 0);
        put(f, o1, j % no1);
        put(f, o2, j / no1);
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
    const double tm = A.taumaj[(long long)k * A.nb + b];
    const Real ell = -RealTraits<Real>::log_(word_uniform<Real>(ua)) * mean_path<Real>(A, k, b, tm);
    Real tw = RealTraits<Real>::inf();
    int wl = -1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (s[a] == (Real)0) continue;
      const Real L = cell_h<Real>(in, a) * int_to_real<Real>(in.n[a]);
      const Real t = s[a] > (Real)0 ? (L - x[a]) / s[a] : -x[a] / s[a];
      if (t < tw) {
        tw = t;
        wl = 2 * a + (s[a] > (Real)0 ? 1 : 0);
      }
    }
    int due = 1;
    if (wl >= 0 && tw < ell) {
      // absorbed by the wall it reaches first; its home is the face it crossed
      c_exit += 1;
      exit_key = in.wall_off + wl;
      exit_w = w;
      const int a = wl >> 1, o1 = (a + 1) % 3, o2 = (a + 2) % 3;
      int j1 = 0, j2 = 0;
      if (o1 < DIM) j1 = min(floor_nonneg<Real>((pick(x, o1) + tw * pick(s, o1)) / cell_h<Real>(in, o1)), in.n[o1] - 1);
      if (o2 < DIM) j2 = min(floor_nonneg<Real>((pick(x, o2) + tw * pick(s, o2)) / cell_h<Real>(in, o2)), in.n[o2] - 1);
      h = in.ncells + in.wface_off[wl] + j2 * in.n[o1] + j1;
      atomicAdd(&A.n_new[A.home_off[k] + (long long)b * nh + h], 1u);
    } else {
      int ci[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        x[a] += ell * s[a];
        ci[a] = min(floor_nonneg<Real>(x[a] / cell_h<Real>(in, a)), in.n[a] - 1);
      }
      const int c = ci[0] + n0 * (ci[1] + n1 * ci[2]);
      // candidate (steps (4)-(5)): W from every candidate, R and the count from real ones
      c_cand += 1;
      const long long jb = in.bc_off + (long long)b * in.ncells + c;
      atomicAdd(&A.W[jb], w * tm);
      // (a band with tau = tau_maj everywhere accepts every candidate: the uniform is below 1)
      if (A.all_real[(long long)k * A.nb + b] || word_uniform<Real>(ub) < accept_ratio<Real>(A, jb)) {
        c_real += 1;
        atomicAdd(&A.R[jb], w);
        h = c;
        atomicAdd(&A.n_new[A.home_off[k] + (long long)b * nh + h], 1u);
      } else {
        due = 0;  // step (6): same direction and weight, a new path next iteration
      }
    }
    px[i] = x[0];
    if (DIM >= 2) py[i] = x[1];
    if (DIM >= 3) pz[i] = x[2];
    sx[i] = s[0];
    if (DIM >= 2) sy[i] = s[1];
    if (DIM >= 3) sz[i] = s[2];
    A.pw[i] = w;
    A.home[i] = h;
    A.due[i] = due;
    (void)n2;
    }
    // wall tallies: the lanes that hit one wall are summed first, one atomic per wall
    unsigned pending = __ballot_sync(0xffffffffu, exit_key >= 0);
    while (pending) {
      const int key = __shfl_sync(0xffffffffu, exit_key, __ffs(pending) - 1);
      double v = exit_key == key ? exit_w : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) {
        if (wall_shared) atomicAdd(&swall[key], v);
        else atomicAdd(&A.wall[key], v);
      }
      pending &= ~__ballot_sync(0xffffffffu, exit_key == key);
    }
  }
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

// Power per particle re-emitted from each (band, home) this iteration: the home's power
// (C_b T_emit V / tau_b for a cell, C_b v_b T_face A / 4 for a boundary face) over the
// particles that ended there in the previous iteration (0 where none did).
__global__ void persistent_home_power_kernel(const InstDesc* inst, int n_inst, int nb, const long long* home_off,
                                             const long long* nband, const long long* nwall, const double* T,
                                             const double* srcshift, const double* coef, const double* wcoef,
                                             const double* wallTf, const unsigned* n_prev, double* home_w,
                                             long long n_homes) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n_homes;
       j += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < n_inst && home_off[k + 1] <= j) ++k;
    const InstDesc& in = inst[k];
    const long long nh = (home_off[k + 1] - home_off[k]) / nb;
    const long long r = j - home_off[k];
    const int b = (int)(r / nh);
    const long long h = r - (long long)b * nh;
    const unsigned n = n_prev[j];
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
  a.taumaj = c->d_taumaj;
  a.v = c->d_v;
  a.wcoef = c->d_wcoef;
  a.wallTf = c->d_wallTf;
  a.state = c->d_px;
  a.pw = reinterpret_cast<double*>(c->d_px) + 6 * c->pers_n;  // after 6 arrays of FP64 or FP32
  a.home_w = c->d_phome_w;
  a.band = c->d_pband;
  a.home = c->d_phome;
  a.due = c->d_pdue;
  a.n_prev = c->d_pcount + (c->pers_parity ? c->pers_homes : 0);
  a.n_new = c->d_pcount + (c->pers_parity ? 0 : c->pers_homes);
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
                                                    a.n_prev, c->d_phome_w, c->pers_homes);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const long long want = (c->pers_n + 255) / 256;
  const unsigned blocks = (unsigned)std::min<long long>(std::max<long long>(want, 1), (long long)c->sm_count * 16);
  const bool f32 = c->opt.precision == IUGKP_TRACK_FP32;
  switch (c->dim * 2 + (f32 ? 1 : 0)) {
    case 2: persistent_step_kernel<1, double><<<blocks, 256, 0, s>>>(a); break;
    case 3: persistent_step_kernel<1, float><<<blocks, 256, 0, s>>>(a); break;
    case 4: persistent_step_kernel<2, double><<<blocks, 256, 0, s>>>(a); break;
    case 5: persistent_step_kernel<2, float><<<blocks, 256, 0, s>>>(a); break;
    case 6: persistent_step_kernel<3, double><<<blocks, 256, 0, s>>>(a); break;
    default: persistent_step_kernel<3, float><<<blocks, 256, 0, s>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace iugkp

namespace iugkp {

namespace {

// Initial population (Sec. 3.2 step (1)): every slot due for emission from its home, and
// every home counted with its own number of slots.
__global__ void persistent_init_kernel(const InstDesc* inst, int n_inst, int nb, const long long* slot_off,
                                       const long long* home_off, const long long* nband, const long long* nwall,
                                       long long n_slots, long long n_homes, double* state, int* band, int* home,
                                       int* due, unsigned* count_prev) {
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
    home[i] = h;
    due[i] = 1;
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
    count_prev[j] = (unsigned)(h < in.ncells ? nband[(long long)k * nb + b] : nwall[b]);
  }
}

}  // namespace

cudaError_t launch_persistent_init(Ctx* c, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<long long>((c->pers_n + 255) / 256 + 1, (long long)c->sm_count * 16);
  persistent_init_kernel<<<blocks, 256, 0, s>>>(c->d_inst, c->n_inst, c->nb, c->d_pslot_off, c->d_phome_off, c->d_pnband,
                                                c->d_pnwall, c->pers_n, c->pers_homes, c->d_px, c->d_pband, c->d_phome,
                                                c->d_pdue, c->d_pcount);
  return cudaGetLastError();
}

}  // namespace iugkp
