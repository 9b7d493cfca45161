// Persistent null-collision population (arXiv 2506.09465 Sec. 3.2 steps (1)-(6)), FP64.
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
// Slots of an instance: N_b per (band, cell), band-major then cell order, then N_w,b per
// (band, boundary face) with faces in wall order (-x, +x, -y, +y, -z, +z; on the wall normal
// to axis a the faces run over axes (a+1)%3 and (a+2)%3, the first fastest). Draws of slot
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
  const double* taumaj;        // [inst * nb]
  const double* v;             // [nb]
  const double* wcoef;         // [inst * nb * 6] C_b v_b A / (4 N_w)
  const double* wallTf;        // [boundary faces]
  double *px, *py, *pz, *sx, *sy, *sz, *pw;
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

template <int DIM>
__global__ void __launch_bounds__(256) persistent_step_kernel(PArgs A) {
  unsigned c_flights = 0, c_cand = 0, c_real = 0, c_exit = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < A.n_slots;
       i += (long long)gridDim.x * blockDim.x) {
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
    double x[3] = {A.px[i], DIM >= 2 ? A.py[i] : 0.0, DIM >= 3 ? A.pz[i] : 0.0};
    double s[3] = {A.sx[i], DIM >= 2 ? A.sy[i] : 0.0, DIM >= 3 ? A.sz[i] : 0.0};
    double w = A.pw[i];
    int h = A.home[i];
    st.j = 0;
    if (A.due[i]) {
      const double nprev = (double)A.n_prev[A.home_off[k] + (long long)b * nh + h];
      if (h < in.ncells) {
        // re-emission in the cell of the real collision (Sec. 3.2 step (2))
        const int ci[3] = {h % n0, (h / n0) % n1, h / (n0 * n1)};
        double u_mu, u_phi = 0.5;
        if (DIM == 1) {
          x[0] = (ci[0] + word_uniform<double>(st.buf.x)) * in.h[0];
          u_mu = word_uniform<double>(st.buf.y);
        } else if (DIM == 2) {
          x[0] = (ci[0] + word_uniform<double>(st.buf.x)) * in.h[0];
          x[1] = (ci[1] + word_uniform<double>(st.buf.y)) * in.h[1];
          u_mu = word_uniform<double>(st.buf.z);
          u_phi = word_uniform<double>(st.buf.w);
        } else {
          x[0] = (ci[0] + word_uniform<double>(st.buf.x)) * in.h[0];
          x[1] = (ci[1] + word_uniform<double>(st.buf.y)) * in.h[1];
          x[2] = (ci[2] + word_uniform<double>(st.buf.z)) * in.h[2];
          u_mu = word_uniform<double>(st.buf.w);
          st.load_block(1);
          u_phi = word_uniform<double>(st.buf.x);
        }
        const double mu = 2.0 * u_mu - 1.0;
        s[0] = mu;
        if (DIM >= 2) {
          const double sn = sqrt(1.0 - mu * mu);
          double sp, cp;
          RealTraits<double>::sincos2pi(u_phi, &sp, &cp);
          s[1] = sn * cp;
          s[2] = sn * sp;
        }
        st.j = thermal_uniforms(DIM);
        double te = A.T[in.cell_off + h];
        if (A.srcshift) te += A.srcshift[in.cell_off + h];
        // C_b V / tau_{b,c} = coef * N_b
        w = A.coef[in.bc_off + (long long)b * in.ncells + h] * (double)A.nband[(long long)k * A.nb + b] * te / nprev;
      } else {
        // re-emission from the boundary face that absorbed it (black wall)
        const int bf = h - in.ncells;
        int wl = 0;
        while (wl + 1 < 2 * DIM && bf >= in.wface_off[wl + 1]) ++wl;
        const int a = wl >> 1, side = wl & 1, o1 = (a + 1) % 3, o2 = (a + 2) % 3;
        const int j = bf - in.wface_off[wl];
        const int no1 = in.n[o1];
        int f[3];
        f[a] = side ? in.n[a] : 0;
        f[o1] = j % no1;
        f[o2] = j / no1;
        double u_n, u_phi = 0.5;
        if (DIM == 1) {
          u_n = word_uniform<double>(st.buf.x);
        } else if (DIM == 2) {
          const int t = (o1 < 2) ? o1 : o2;
          x[t] = (f[t] + word_uniform<double>(st.buf.x)) * in.h[t];
          u_n = word_uniform<double>(st.buf.y);
          u_phi = word_uniform<double>(st.buf.z);
        } else {
          const int t0 = o1 < o2 ? o1 : o2, t1 = o1 < o2 ? o2 : o1;
          x[t0] = (f[t0] + word_uniform<double>(st.buf.x)) * in.h[t0];
          x[t1] = (f[t1] + word_uniform<double>(st.buf.y)) * in.h[t1];
          u_n = word_uniform<double>(st.buf.z);
          u_phi = word_uniform<double>(st.buf.w);
        }
        x[a] = f[a] * in.h[a];
        const double mn = sqrt(u_n);
        s[a] = side ? -mn : mn;
        if (DIM >= 2) {
          const double stn = sqrt(1.0 - u_n);
          double sp, cp;
          RealTraits<double>::sincos2pi(u_phi, &sp, &cp);
          s[o1] = stn * cp;
          s[o2] = stn * sp;
        } else {
          s[o1] = 0.0;
          s[o2] = 0.0;
        }
        st.j = wall_uniforms(DIM);
        w = A.wcoef[((long long)k * A.nb + b) * 6 + wl] * (double)A.nwall[b] * A.wallTf[in.bface_off + bf] / nprev;
      }
    }
    // one flight (Sec. 3.2 step (3)): path -ln(u) v tau_maj
    c_flights += 1;
    uint32_t ua, ub;
    st.next_pair(ua, ub);
    const double tm = A.taumaj[(long long)k * A.nb + b];
    const double ell = -log(word_uniform<double>(ua)) * A.v[b] * tm;
    double tw = INFINITY;
    int wl = -1;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      if (s[a] == 0.0) continue;
      const double L = in.h[a] * in.n[a];
      const double t = s[a] > 0.0 ? (L - x[a]) / s[a] : -x[a] / s[a];
      if (t < tw) {
        tw = t;
        wl = 2 * a + (s[a] > 0.0 ? 1 : 0);
      }
    }
    int due = 1;
    if (wl >= 0 && tw < ell) {
      // absorbed by the wall it reaches first; its home is the face it crossed
      c_exit += 1;
      atomicAdd(&A.wall[in.wall_off + wl], w);
      const int a = wl >> 1, o1 = (a + 1) % 3, o2 = (a + 2) % 3;
      int j1 = 0, j2 = 0;
      if (o1 < DIM) j1 = min(max((int)floor((x[o1] + tw * s[o1]) / in.h[o1]), 0), in.n[o1] - 1);
      if (o2 < DIM) j2 = min(max((int)floor((x[o2] + tw * s[o2]) / in.h[o2]), 0), in.n[o2] - 1);
      h = in.ncells + in.wface_off[wl] + j2 * in.n[o1] + j1;
      atomicAdd(&A.n_new[A.home_off[k] + (long long)b * nh + h], 1u);
    } else {
      int ci[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        x[a] += ell * s[a];
        ci[a] = min(max((int)floor(x[a] / in.h[a]), 0), in.n[a] - 1);
      }
      const int c = ci[0] + n0 * (ci[1] + n1 * ci[2]);
      // candidate (steps (4)-(5)): W from every candidate, R and the count from real ones
      c_cand += 1;
      const long long jb = in.bc_off + (long long)b * in.ncells + c;
      atomicAdd(&A.W[jb], w * tm);
      if (word_uniform<double>(ub) < A.ratio64[jb]) {
        c_real += 1;
        atomicAdd(&A.R[jb], w);
        h = c;
        atomicAdd(&A.n_new[A.home_off[k] + (long long)b * nh + h], 1u);
      } else {
        due = 0;  // step (6): same direction and weight, a new path next iteration
      }
    }
    A.px[i] = x[0];
    if (DIM >= 2) A.py[i] = x[1];
    if (DIM >= 3) A.pz[i] = x[2];
    A.sx[i] = s[0];
    if (DIM >= 2) A.sy[i] = s[1];
    if (DIM >= 3) A.sz[i] = s[2];
    A.pw[i] = w;
    A.home[i] = h;
    A.due[i] = due;
    (void)n2;
  }
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
  a.taumaj = c->d_taumaj;
  a.v = c->d_v;
  a.wcoef = c->d_wcoef;
  a.wallTf = c->d_wallTf;
  a.px = c->d_px;
  a.py = c->d_px + c->pers_n;
  a.pz = c->d_px + 2 * c->pers_n;
  a.sx = c->d_px + 3 * c->pers_n;
  a.sy = c->d_px + 4 * c->pers_n;
  a.sz = c->d_px + 5 * c->pers_n;
  a.pw = c->d_px + 6 * c->pers_n;
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
  const long long want = (c->pers_n + 255) / 256;
  const unsigned blocks = (unsigned)std::min<long long>(std::max<long long>(want, 1), (long long)c->sm_count * 16);
  switch (c->dim) {
    case 1: persistent_step_kernel<1><<<blocks, 256, 0, s>>>(a); break;
    case 2: persistent_step_kernel<2><<<blocks, 256, 0, s>>>(a); break;
    default: persistent_step_kernel<3><<<blocks, 256, 0, s>>>(a); break;
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
      h = (int)(r / nband[(long long)k * nb + b]);
    } else {
      r -= thermal;
      const long long nbf = (home_off[k + 1] - home_off[k]) / nb - in.ncells;
      while (r >= nwall[b] * nbf) r -= nwall[b] * nbf, ++b;
      h = in.ncells + (int)(r / nwall[b]);
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
