// IUGKP steady-state phonon BTE: plain FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference legs may load this library. The product path (the CUDA
// library and its Python binding) never calls, links or imports anything here, and
// this file shares no code, header, table or helper with it.
//
// What it computes, step by step, in the order of the paper (Liu, Yang, Zhang, Ji, Xu,
// "Implicit unified gas kinetic particle method for steady-state solution of
// multiscale phonon transport", arXiv 2506.09465):
//   * linearised equilibrium e_eq = C (T - T_ref) / 4pi with T_ref = 0 (Sec. 2, Eq.
//     "derivation final equilibrium"); moments E, T, q (Sec. 2, moment equations);
//   * one sweep of the constant-tau iteration (Sec. 3.1, steps (1)-(3)): every cell
//     emits particles sampled from its own equilibrium (uniform position, isotropic
//     direction), each flies an exponential path -u tau ln(eta) (Sec. 3.1, inverse
//     sampling) and deposits where it stops (Sec. 3.1, Eq. "sum-g-particle");
//   * variable tau through null collisions (Sec. 3.2): candidate flights at the
//     per-band majorant rate 1/(u tau_min) (Eq. "truncated-tf"), accepted as real with
//     probability tau_min / tau(x) (Sec. 3.2, P_real = sigma / sigma_max); real and
//     candidate tallies W^h and W (Sec. 3.2, W = sum w_nc + sum w_rc, W^h = sum w_rc);
//   * macro update and the inexact-Newton correction from the diffusion equation
//     (Sec. 3.3, Eqs. "macro-q-eqn", "macro-q-res", "linear-q"), solved here by a
//     direct banded elimination (no iteration);
//   * the adjoint of one sweep (with draws fixed a sweep is a linear map, Sec. 2,
//     Eq. "sum-g"), by re-tracing each particle and gathering at its real collision.
//
// Readings of the paper that this file fixes:
//   * emission weights are powers (thermal C_b T V / tau_b, wall C_b v_b T_w A / 4),
//     so that with constant tau, multiplying by tau gives the paper's w = W / N;
//   * a particle keeps flying through its null collisions inside the same sweep, with
//     its direction unchanged, until a real collision or a wall absorbs it;
//   * walls are black and isothermal; wall particles enter with a cosine-weighted
//     direction;
//   * 1D and 2D use the first one or two components of a 3D isotropic direction;
//   * a heat source Q is emitted by the cell's thermal particles: the emission
//     temperature is T + Q / m with m = sum_b C_b / tau_b;
//   * the Newton step: dT solves -div(kappa grad dT) = (R - S(T^n)) / V with
//     kappa = sum_b C_b v_b^2 tau_b / 3 and harmonic face kappa; at a wall the error
//     sees a black wall at zero temperature, so the correction takes the vacuum
//     (Marshak) condition: outward flux = (sum_b C_b v_b / 2) dT_wall, in series with
//     the half-cell conduction; T^{n+1} = T^{n+1/2} + theta dT, where
//     theta = min(1, 1.5 / t) damps the correction when cells are optically thick
//     (t = max over cells of h_min / lambda_eff, lambda_eff = sqrt(3 kappa / m)).
//
// Precision: FP64 throughout. Build with -ffp-contract=off so that no multiply-add is
// fused (the expressions below are evaluated exactly as written).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies, with the key bumped by
// the Weyl constants between rounds.
// ---------------------------------------------------------------------------
const uint32_t PHILOX_M0 = 0xD2511F53u;
const uint32_t PHILOX_M1 = 0xCD9E8D57u;
const uint32_t PHILOX_W0 = 0x9E3779B9u;
const uint32_t PHILOX_W1 = 0xBB67AE85u;

void philox4x32_10(const uint32_t in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {in[0], in[1], in[2], in[3]};
  uint32_t k[2] = {key_in[0], key_in[1]};
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k[0] += PHILOX_W0;
      k[1] += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

// A 32-bit Philox word to a uniform in the open interval (0, 1): the top 23 bits m
// give u = (2m + 1) / 2^24, exactly representable in float and in double.
double word_to_uniform(uint32_t a) {
  uint32_t m = a >> 9;
  return (double)(2u * m + 1u) * (1.0 / 16777216.0);
}

// The uniform stream of one particle. Uniform j of the stream is word (j mod 4) of
// Philox block (j / 4), block k having counter (k, particle, emitter, band<<24|epoch)
// and key (lo32(seed), hi32(seed) ^ instance). A flight's draws: the emission takes
// uniforms 0 .. j0 - 1 (j0 even); the first candidate's path uniform is made of bits the
// emission leaves unused (first_path_uniform), its acceptance uniform is uniform j0;
// uniform j0 + 1 is not used; candidate k >= 2 takes uniforms j0 + 2k - 2 (path) and
// j0 + 2k - 1 (acceptance).
struct Stream {
  uint32_t ctr[4];
  uint32_t key[2];
  uint32_t words[4];
  long long next;  // index of the next uniform
  long long loaded_block;

  Stream(uint64_t seed, uint32_t instance, uint32_t band, uint32_t epoch,
         uint32_t emitter, uint32_t particle) {
    key[0] = (uint32_t)(seed & 0xFFFFFFFFull);
    key[1] = (uint32_t)(seed >> 32) ^ instance;
    ctr[0] = 0;
    ctr[1] = particle;
    ctr[2] = emitter;
    ctr[3] = (band << 24) | (epoch & 0xFFFFFFu);
    next = 0;
    loaded_block = -1;
  }
  double uniform() {
    long long block = next / 4;
    int word = (int)(next % 4);
    if (block != loaded_block) {
      ctr[0] = (uint32_t)block;
      philox4x32_10(ctr, key, words);
      loaded_block = block;
    }
    ++next;
    return word_to_uniform(words[word]);
  }
  void skip_to(long long j) { next = j; }
  // The first candidate's path uniform: 23 bits that the emission leaves unused in block 0,
  // the low 9 bits of words 0 and 1 and bits 4..8 of word 2 (uniforms take the top 23 bits),
  // m = (w0 mod 2^9) 2^14 + (w1 mod 2^9) 2^5 + floor((w2 mod 2^9) / 2^4), u = (2m + 1) / 2^24.
  double first_path_uniform() const {
    uint32_t c[4] = {0u, ctr[1], ctr[2], ctr[3]};
    uint32_t w[4];
    philox4x32_10(c, key, w);
    const uint32_t m = ((w[0] & 511u) << 14) | ((w[1] & 511u) << 5) | ((w[2] & 511u) >> 4);
    return (double)(2u * m + 1u) * (1.0 / 16777216.0);
  }
};

// ---------------------------------------------------------------------------
// Problem description (one instance).
// ---------------------------------------------------------------------------
}  // namespace

extern "C" {

struct OrcProblem {
  int dim;                 // 1, 2 or 3
  int nx, ny, nz;          // cells per axis (unused axes = 1)
  double lx, ly, lz;       // domain lengths (unused axes: 1, so per unit area/depth)
  int nb;                  // band-branches
  const double* C;         // [nb] volumetric specific heat per band
  const double* v;         // [nb] group speed per band
  const double* tau;       // [nb][ncells] relaxation time, > 0
  const double* wall_T;    // [2*dim] deviational wall temperatures: -x,+x,-y,+y,-z,+z
  const double* source;    // [ncells] heat source power density, or NULL
  const long long* n_band;       // [nb] thermal particles per cell per band
  const long long* n_wall_band;  // [nb] particles per boundary face per band
  unsigned long long seed;
  unsigned int instance;
  long long budget;        // max steps (crossings + candidates) per particle
  const double* wall_face_T;  // [boundary faces] temperature of every boundary face, or
                              // NULL (each wall uniform at wall_T). Walls in the order of
                              // wall_T; on wall (a, side) the faces run over the two other
                              // axes o1 = (a+1)%3, o2 = (a+2)%3, o1 fastest.
};

}  // extern "C"

namespace {

struct Geo {
  int dim, n[3];
  double L[3], h[3];
  long long ncells, nfaces[3], face_off[3], nfaces_total;
  double V;        // cell volume (per unit area / depth for 1D / 2D)
  double A[3];     // face area normal to each axis
  explicit Geo(const OrcProblem& p) {
    dim = p.dim;
    n[0] = p.nx; n[1] = dim >= 2 ? p.ny : 1; n[2] = dim >= 3 ? p.nz : 1;
    L[0] = p.lx; L[1] = dim >= 2 ? p.ly : 1.0; L[2] = dim >= 3 ? p.lz : 1.0;
    for (int a = 0; a < 3; ++a) h[a] = a < dim ? L[a] / n[a] : 1.0;
    ncells = (long long)n[0] * n[1] * n[2];
    V = h[0] * h[1] * h[2];
    A[0] = h[1] * h[2]; A[1] = h[0] * h[2]; A[2] = h[0] * h[1];
    long long off = 0;
    for (int a = 0; a < 3; ++a) {
      if (a < dim) {
        long long m = 1;
        for (int b = 0; b < 3; ++b) m *= (b == a) ? (n[b] + 1) : n[b];
        nfaces[a] = m;
      } else {
        nfaces[a] = 0;
      }
      face_off[a] = off;
      off += nfaces[a];
    }
    nfaces_total = off;
  }
  long long cell(const int i[3]) const { return i[0] + (long long)n[0] * (i[1] + (long long)n[1] * i[2]); }
  // Face of axis a with lower-corner index f[a] in [0, n[a]] along a.
  long long face(int a, const int f[3]) const {
    long long m0 = n[0] + (a == 0 ? 1 : 0);
    long long m1 = n[1] + (a == 1 ? 1 : 0);
    return face_off[a] + f[0] + m0 * (f[1] + m1 * f[2]);
  }
};

struct Tallies {
  double* R;
  double* W;
  double* F;
  double* wall;
  unsigned long long counters[6];  // flights, candidates, real, crossings, wall exits, dropped
};

// One particle from emission to absorption, following the candidate-collision chain
// of Sec. 3.2 with the DDA cell walk; tallies as described at the top of the file.
// x, idx: start position and cell; s: direction; w: power weight; band b.
// Adjoint mode (lambda != nullptr): no tallies; returns lambda at the real collision
// cell divided by (V m) there, or 0 if the particle reached a wall.
double trace_particle(const OrcProblem& p, const Geo& g, int b, double tau_maj,
                      const double* m_cell, Stream& st, double x[3], int idx[3],
                      const double s[3], double w, Tallies* t, const double* lambda) {
  const long long nc = g.ncells;
  double speed = p.v[b];
  long long steps = 0;
  double d = -std::log(st.first_path_uniform()) * speed * tau_maj;  // path to the first candidate
  bool first = true;
  for (;;) {
    // Distance along s to the next face on each axis.
    double tmin = INFINITY;
    int amin = -1;
    for (int a = 0; a < g.dim; ++a) {
      double ta = INFINITY;
      if (s[a] > 0.0) ta = ((idx[a] + 1) * g.h[a] - x[a]) / s[a];
      else if (s[a] < 0.0) ta = (idx[a] * g.h[a] - x[a]) / s[a];
      if (ta < tmin) { tmin = ta; amin = a; }
    }
    if (++steps > p.budget) {
      if (t) t->counters[5] += 1;
      return 0.0;
    }
    long long c = g.cell(idx);
    if (d <= tmin) {
      // Candidate collision inside the current cell.
      for (int a = 0; a < g.dim; ++a) x[a] = x[a] + d * s[a];
      double tau_here = p.tau[(long long)b * nc + c];
      if (t) {
        t->counters[1] += 1;
        t->W[(long long)b * nc + c] += w * tau_maj;
      }
      double u_acc = st.uniform();
      if (first) {  // the first candidate's acceptance is uniform j0; j0 + 1 is not used
        st.skip_to(st.next + 1);
        first = false;
      }
      if (u_acc < tau_maj / tau_here) {
        if (t) {
          t->counters[2] += 1;
          t->R[(long long)b * nc + c] += w;
        }
        if (lambda) return lambda[c] / (g.V * m_cell[c]);
        return 0.0;
      }
      d = -std::log(st.uniform()) * speed * tau_maj;  // null: same direction, new path
      continue;
    }
    // Cross the face of axis amin.
    for (int a = 0; a < g.dim; ++a) x[a] = x[a] + tmin * s[a];
    d = d - tmin;
    int step = s[amin] > 0.0 ? 1 : -1;
    int f[3] = {idx[0], idx[1], idx[2]};
    if (step > 0) f[amin] += 1;
    x[amin] = f[amin] * g.h[amin];
    if (t) t->F[g.face(amin, f)] += w * step;
    idx[amin] += step;
    if (idx[amin] < 0 || idx[amin] >= g.n[amin]) {
      if (t) {
        t->counters[4] += 1;
        t->wall[2 * amin + (step > 0 ? 1 : 0)] += w;
      }
      return 0.0;
    }
    if (t) t->counters[3] += 1;
  }
}

// Direction of a cell (thermal) particle: mu = cos(theta) ~ U(-1, 1), phi ~ U(0, 2pi),
// s = (cos theta, sin theta cos phi, sin theta sin phi) (Sec. 2, below Eq. "eq:BGKBTE").
void thermal_direction(int dim, double u_mu, double u_phi, double s[3]) {
  double mu = 2.0 * u_mu - 1.0;
  double sn = std::sqrt(1.0 - mu * mu);
  double phi = 2.0 * M_PI * u_phi;
  s[0] = mu;
  s[1] = dim >= 2 ? sn * std::cos(phi) : 0.0;
  s[2] = dim >= 2 ? sn * std::sin(phi) : 0.0;
}

int emission_uniforms_thermal(int dim) { return dim == 1 ? 2 : (dim == 2 ? 4 : 6); }
int emission_uniforms_wall(int dim) { return dim == 1 ? 2 : 4; }

void majorants(const OrcProblem& p, const Geo& g, std::vector<double>& tmaj) {
  tmaj.assign(p.nb, INFINITY);
  for (int b = 0; b < p.nb; ++b)
    for (long long c = 0; c < g.ncells; ++c) tmaj[b] = std::min(tmaj[b], p.tau[(long long)b * g.ncells + c]);
}

void cell_m(const OrcProblem& p, const Geo& g, std::vector<double>& m) {
  m.assign(g.ncells, 0.0);
  for (long long c = 0; c < g.ncells; ++c)
    for (int b = 0; b < p.nb; ++b) m[c] += p.C[b] / p.tau[(long long)b * g.ncells + c];
}

bool valid(const OrcProblem* p) {
  if (!p || p->dim < 1 || p->dim > 3 || p->nx < 1) return false;
  if (p->dim >= 2 && p->ny < 1) return false;
  if (p->dim >= 3 && p->nz < 1) return false;
  if (p->nb < 1 || !p->C || !p->v || !p->tau || !p->n_band || !p->n_wall_band) return false;
  return true;
}

// Start state of a wall particle on the boundary face with lower corner f of wall (a, side)
// (Sec. 4 black walls): position uniform along the in-domain tangential axes (taken in
// axis order), direction cosine-weighted about the inward normal, mu_n = sqrt(u_n), the
// tangential part sqrt(1 - u_n) (cos 2 pi u_phi, sin 2 pi u_phi) on the axes (a+1)%3, (a+2)%3.
// Consumes emission_uniforms_wall(dim) uniforms.
void wall_start(const Geo& g, int a, int side, const int f[3], Stream& st, double x[3], double s[3], int idx[3]) {
  const int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
  x[0] = x[1] = x[2] = 0.0;
  int tang[2] = {std::min(o1, o2), std::max(o1, o2)};
  for (int k = 0; k < 2; ++k) {
    int ax = tang[k];
    if (ax < g.dim) x[ax] = (f[ax] + st.uniform()) * g.h[ax];
  }
  x[a] = f[a] * g.h[a];
  double u_n = st.uniform();
  double u_phi = g.dim >= 2 ? st.uniform() : 0.5;
  double mu_n = std::sqrt(u_n);
  double st_ = std::sqrt(1.0 - u_n);
  double phi = 2.0 * M_PI * u_phi;
  s[a] = side == 0 ? mu_n : -mu_n;
  s[o1] = g.dim >= 2 ? st_ * std::cos(phi) : 0.0;
  s[o2] = g.dim >= 2 ? st_ * std::sin(phi) : 0.0;
  for (int ax = g.dim; ax < 3; ++ax) s[ax] = 0.0;
  st.skip_to(emission_uniforms_wall(g.dim));
  idx[0] = f[0]; idx[1] = f[1]; idx[2] = f[2];
  if (side == 1) idx[a] = g.n[a] - 1;
  for (int ax = g.dim; ax < 3; ++ax) idx[ax] = 0;
}

// Visit every particle of one sweep. For each: emitter kind (0 cell, 1 wall), band,
// emitter id, particle index, unit-temperature weight coefficient, start state.
template <typename F>
void for_each_particle(const OrcProblem& p, const Geo& g, uint32_t epoch, bool skip_zero,
                       const double* T_emit, const double* wall_T, const double* wall_face_T, F&& fn) {
  // Thermal emission (Sec. 3.1 step (1)): N_b particles per cell and band, power
  // C_b T V / tau_b shared equally.
  for (int b = 0; b < p.nb; ++b) {
    long long nbp = p.n_band[b];
    if (nbp <= 0) continue;
    for (long long c = 0; c < g.ncells; ++c) {
      double tau_c = p.tau[(long long)b * g.ncells + c];
      double coef = p.C[b] * g.V / (tau_c * (double)nbp);
      double w = coef * (T_emit ? T_emit[c] : 0.0);
      if (skip_zero && w == 0.0) continue;
      int idx[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((long long)g.n[0] * g.n[1]))};
      for (long long q = 0; q < nbp; ++q) {
        Stream st(p.seed, p.instance, (uint32_t)b, epoch, (uint32_t)c, (uint32_t)q);
        double x[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < g.dim; ++a) x[a] = (idx[a] + st.uniform()) * g.h[a];
        double u_mu = st.uniform();
        double u_phi = g.dim >= 2 ? st.uniform() : 0.5;
        double s[3];
        thermal_direction(g.dim, u_mu, u_phi, s);
        st.skip_to(emission_uniforms_thermal(g.dim));
        int ii[3] = {idx[0], idx[1], idx[2]};
        fn(0, b, c, c, coef, w, st, x, ii, s);
      }
    }
  }
  // Wall emission: every boundary face emits the hemispherical power C_b v_b T_w A / 4,
  // T_w the temperature of its wall, or of the face itself when wall_face_T is given.
  long long wall_face_off[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int wl = 0; wl < 2 * g.dim; ++wl) {
    int a = wl / 2;
    wall_face_off[wl + 1] = wall_face_off[wl] + (long long)g.n[(a + 1) % 3] * g.n[(a + 2) % 3];
  }
  for (int b = 0; b < p.nb; ++b) {
    long long nwp = p.n_wall_band[b];
    if (nwp <= 0) continue;
    for (int a = 0; a < g.dim; ++a) {
      for (int side = 0; side < 2; ++side) {
        int wall = 2 * a + side;
        double Tw = wall_T ? wall_T[wall] : 0.0;
        double coef = p.C[b] * p.v[b] * g.A[a] / (4.0 * (double)nwp);
        if (skip_zero && !wall_face_T && coef * Tw == 0.0) continue;
        int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
        // Faces on this wall: all (i_o1, i_o2) with the a-index at 0 or n[a].
        for (int j2 = 0; j2 < g.n[o2]; ++j2) {
          for (int j1 = 0; j1 < g.n[o1]; ++j1) {
            double Tf = wall_face_T ? wall_face_T[wall_face_off[wall] + (long long)j2 * g.n[o1] + j1] : Tw;
            double w = coef * Tf;
            if (skip_zero && w == 0.0) continue;
            int f[3];
            f[a] = side == 0 ? 0 : g.n[a];
            f[o1] = j1; f[o2] = j2;
            long long face = g.face(a, f);
            uint32_t emitter = (uint32_t)(g.ncells + face);
            for (long long q = 0; q < nwp; ++q) {
              Stream st(p.seed, p.instance, (uint32_t)b, epoch, emitter, (uint32_t)q);
              double x[3], s[3];
              int idx[3];
              wall_start(g, a, side, f, st, x, s, idx);
              fn(1, b, wall, face, coef, w, st, x, idx, s);
            }
          }
        }
      }
    }
  }
}

}  // namespace

extern "C" {

// Raw Philox4x32-10 block, for tests.
void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

double orc_word_to_uniform(uint32_t a) { return word_to_uniform(a); }

// First n uniforms of the stream of one particle (for sampler tests).
void orc_stream(unsigned long long seed, uint32_t instance, uint32_t band, uint32_t epoch,
                uint32_t emitter, uint32_t particle, long long n, double* out) {
  Stream st(seed, instance, band, epoch, emitter, particle);
  for (long long j = 0; j < n; ++j) out[j] = st.uniform();
}

long long orc_ncells(const OrcProblem* p) { Geo g(*p); return g.ncells; }
long long orc_nfaces(const OrcProblem* p) { Geo g(*p); return g.nfaces_total; }

// One sweep (Sec. 3.1 steps (1)-(3), generalised by Sec. 3.2): emission from T (plus
// the source as an emission-temperature shift), transport, null/real collisions,
// tallies R (real-collision power, W^h), W (candidate estimator of energy, W), F (net
// power across each face, +axis direction), wall (absorbed power per wall).
// Outputs are overwritten. counters: flights, candidates, real, crossings, wall exits,
// dropped (step budget exceeded). Returns 0, or -1 on invalid input.
int orc_sweep(const OrcProblem* p, const double* T, uint32_t epoch, double* R, double* W,
              double* F, double* wall, unsigned long long* counters) {
  if (!valid(p)) return -1;
  Geo g(*p);
  std::vector<double> tmaj, m;
  majorants(*p, g, tmaj);
  cell_m(*p, g, m);
  std::vector<double> T_emit(g.ncells);
  for (long long c = 0; c < g.ncells; ++c) T_emit[c] = T[c] + (p->source ? p->source[c] / m[c] : 0.0);
  std::fill(R, R + (long long)p->nb * g.ncells, 0.0);
  std::fill(W, W + (long long)p->nb * g.ncells, 0.0);
  std::fill(F, F + g.nfaces_total, 0.0);
  std::fill(wall, wall + 2 * p->dim, 0.0);
  Tallies t{R, W, F, wall, {0, 0, 0, 0, 0, 0}};
  for_each_particle(*p, g, epoch, true, T_emit.data(), p->wall_T, p->wall_face_T,
                    [&](int kind, int b, long long emitter, long long face_or_cell, double, double w, Stream& st,
                        double* x, int* idx, const double* s) {
                      t.counters[0] += 1;
                      if (kind == 1) {
                        // Entering power through the boundary face (+axis sign convention);
                        // for a wall particle the emitter id is the wall 2*axis + side.
                        int a = (int)(emitter / 2);
                        t.F[face_or_cell] += s[a] > 0.0 ? w : -w;
                      }
                      trace_particle(*p, g, b, tmaj[b], m.data(), st, x, idx, s, w, &t, nullptr);
                    });
  for (int k = 0; k < 6; ++k) counters[k] = t.counters[k];
  return 0;
}

// Macro update (Sec. 3.1 step (3); Sec. 3.2 step (2) resamples from W^h):
// T_half = sum_b R_b / (V sum_b C_b / tau_b); T_E = sum_b W_b / (V sum_b C_b).
int orc_macro(const OrcProblem* p, const double* R, const double* W, double* T_half, double* T_E) {
  if (!valid(p)) return -1;
  Geo g(*p);
  double csum = 0.0;
  for (int b = 0; b < p->nb; ++b) csum += p->C[b];
  for (long long c = 0; c < g.ncells; ++c) {
    double r = 0.0, w = 0.0, m = 0.0;
    for (int b = 0; b < p->nb; ++b) {
      r += R[(long long)b * g.ncells + c];
      w += W[(long long)b * g.ncells + c];
      m += p->C[b] / p->tau[(long long)b * g.ncells + c];
    }
    if (T_half) T_half[c] = r / (g.V * m);
    if (T_E) T_E[c] = w / (g.V * csum);
  }
  return 0;
}

}  // extern "C"

namespace {

// Cell conductivity kappa = sum_b C_b v_b^2 tau_b / 3 (Sec. 3.3, Eq. "linear-q").
void cell_kappa(const OrcProblem& p, const Geo& g, std::vector<double>& k) {
  k.assign(g.ncells, 0.0);
  for (long long c = 0; c < g.ncells; ++c)
    for (int b = 0; b < p.nb; ++b)
      k[c] += p.C[b] * p.v[b] * p.v[b] * p.tau[(long long)b * g.ncells + c] / 3.0;
}

// The finite-volume diffusion operator A dT = -div(kappa grad dT), written out as a
// row per cell: diag and the coefficient to each neighbour (negative).
struct DiffRow { double diag; long long nb[6]; double coef[6]; int count; };

// sum_b C_b v_b: twice the wall conductance of the vacuum condition.
double wall_cv(const OrcProblem& p) {
  double s = 0.0;
  for (int b = 0; b < p.nb; ++b) s += p.C[b] * p.v[b];
  return s;
}

void diffusion_row(const Geo& g, const std::vector<double>& kap, double cv, long long c, DiffRow& row) {
  int idx[3] = {(int)(c % g.n[0]), (int)((c / g.n[0]) % g.n[1]), (int)(c / ((long long)g.n[0] * g.n[1]))};
  row.diag = 0.0;
  row.count = 0;
  for (int a = 0; a < g.dim; ++a) {
    for (int side = -1; side <= 1; side += 2) {
      int j[3] = {idx[0], idx[1], idx[2]};
      j[a] += side;
      double hh = g.h[a] * g.h[a];
      if (j[a] < 0 || j[a] >= g.n[a]) {
        // Wall face: half-cell conduction in series with the vacuum condition
        // (flux = cv / 2 times the face value). Conductance per unit area G; the row
        // divides by the cell width along a.
        double G = 1.0 / (g.h[a] / (2.0 * kap[c]) + 2.0 / cv);
        row.diag += G / g.h[a];
      } else {
        long long n = g.cell(j);
        double kf = 2.0 * kap[c] * kap[n] / (kap[c] + kap[n]);
        row.diag += kf / hh;
        row.nb[row.count] = n;
        row.coef[row.count] = -kf / hh;
        row.count += 1;
      }
    }
  }
}

// Solve A x = rhs by Gaussian elimination on the band of half-width bw = the largest
// neighbour index distance (A is symmetric positive definite, no pivoting needed).
bool banded_solve(const Geo& g, const std::vector<double>& kap, double cv, const double* rhs, double* x) {
  long long n = g.ncells;
  long long bw = g.dim == 1 ? 1 : (g.dim == 2 ? g.n[0] : (long long)g.n[0] * g.n[1]);
  long long width = 2 * bw + 1;
  std::vector<double> band((size_t)(n * width), 0.0);  // band[i*width + (j - i + bw)]
  auto at = [&](long long i, long long j) -> double& { return band[(size_t)(i * width + (j - i + bw))]; };
  std::vector<double> b(rhs, rhs + n);
  for (long long i = 0; i < n; ++i) {
    DiffRow row;
    diffusion_row(g, kap, cv, i, row);
    at(i, i) += row.diag;
    for (int k = 0; k < row.count; ++k) at(i, row.nb[k]) += row.coef[k];
  }
  for (long long k = 0; k < n; ++k) {
    double piv = at(k, k);
    if (!(piv > 0.0)) return false;
    long long iend = std::min(n - 1, k + bw);
    for (long long i = k + 1; i <= iend; ++i) {
      double f = at(i, k) / piv;
      if (f == 0.0) continue;
      long long jend = std::min(n - 1, k + bw);
      for (long long j = k; j <= jend; ++j) at(i, j) -= f * at(k, j);
      b[i] -= f * b[k];
    }
  }
  for (long long i = n - 1; i >= 0; --i) {
    double s = b[i];
    long long jend = std::min(n - 1, i + bw);
    for (long long j = i + 1; j <= jend; ++j) s -= at(i, j) * x[j];
    x[i] = s / at(i, i);
  }
  return true;
}

}  // namespace

extern "C" {

// y = A x with A the diffusion operator above (for tests of the stencil).
int orc_diffusion_apply(const OrcProblem* p, const double* x, double* y) {
  if (!valid(p)) return -1;
  Geo g(*p);
  std::vector<double> kap;
  cell_kappa(*p, g, kap);
  for (long long c = 0; c < g.ncells; ++c) {
    DiffRow row;
    diffusion_row(g, kap, wall_cv(*p), c, row);
    double s = row.diag * x[c];
    for (int k = 0; k < row.count; ++k) s += row.coef[k] * x[row.nb[k]];
    y[c] = s;
  }
  return 0;
}

// x = A^{-1} rhs (direct banded elimination).
int orc_diffusion_solve(const OrcProblem* p, const double* rhs, double* x) {
  if (!valid(p)) return -1;
  Geo g(*p);
  std::vector<double> kap;
  cell_kappa(*p, g, kap);
  return banded_solve(g, kap, wall_cv(*p), rhs, x) ? 0 : -2;
}

// Damping of the correction: theta = min(1, 1.5 / t), t = max over cells of
// h_min / sqrt(3 kappa / m) (the cell's optical thickness for the gray case).
double orc_newton_theta(const OrcProblem* p) {
  if (!valid(p)) return -1.0;
  Geo g(*p);
  std::vector<double> kap, m;
  cell_kappa(*p, g, kap);
  cell_m(*p, g, m);
  double hmin = g.h[0];
  for (int a = 1; a < g.dim; ++a) hmin = std::min(hmin, g.h[a]);
  double tmax = 0.0;
  for (long long c = 0; c < g.ncells; ++c) tmax = std::max(tmax, hmin / std::sqrt(3.0 * kap[c] / m[c]));
  return std::min(1.0, 1.5 / tmax);
}

// Inexact-Newton correction (Sec. 3.3): s = (sum_b R_b - sum_b C_b T_n V / tau_b) / V,
// solve -div(kappa grad dT) = s, T_half += theta dT. dT_out (may be NULL) receives
// theta dT.
int orc_newton(const OrcProblem* p, const double* T_n, double* T_half, const double* R, double* dT_out) {
  if (!valid(p)) return -1;
  Geo g(*p);
  std::vector<double> kap, rhs(g.ncells), dT(g.ncells);
  cell_kappa(*p, g, kap);
  double theta = orc_newton_theta(p);
  for (long long c = 0; c < g.ncells; ++c) {
    double r = 0.0, s = 0.0;
    for (int b = 0; b < p->nb; ++b) {
      r += R[(long long)b * g.ncells + c];
      s += p->C[b] * T_n[c] * g.V / p->tau[(long long)b * g.ncells + c];
    }
    rhs[c] = (r - s) / g.V;
  }
  if (!banded_solve(g, kap, wall_cv(*p), rhs.data(), dT.data())) return -2;
  for (long long c = 0; c < g.ncells; ++c) {
    T_half[c] += theta * dT[c];
    if (dT_out) dT_out[c] = theta * dT[c];
  }
  return 0;
}

// Relative change between iterates: ||T1 - T0||_2 / max(||T1||_2, dT_ref sqrt(ncells)).
double orc_residual(long long n, const double* T0, const double* T1, double dT_ref) {
  double num = 0.0, den = 0.0;
  for (long long c = 0; c < n; ++c) {
    num += (T1[c] - T0[c]) * (T1[c] - T0[c]);
    den += T1[c] * T1[c];
  }
  double floor_ = dT_ref * std::sqrt((double)n);
  return std::sqrt(num) / std::max(std::sqrt(den), floor_);
}

// Steady driver (Sec. 4 usage of the iteration): repeat sweep -> macro update ->
// [Newton] until the residual is <= tol. frozen: epoch stays epoch0; else epoch0 + n.
// T is the initial guess on entry and the final iterate on exit.
int orc_solve_steady(const OrcProblem* p, double* T, double tol, int max_iter, int frozen,
                     uint32_t epoch0, int newton, double dT_ref, int* iters_out, double* res_out,
                     double* res_history) {
  if (!valid(p)) return -1;
  Geo g(*p);
  long long nbc = (long long)p->nb * g.ncells;
  std::vector<double> R(nbc), W(nbc), F(g.nfaces_total), wall(2 * p->dim), Th(g.ncells);
  unsigned long long counters[6];
  double res = INFINITY;
  int it = 0;
  while (it < max_iter) {
    uint32_t epoch = frozen ? epoch0 : epoch0 + (uint32_t)it;
    orc_sweep(p, T, epoch, R.data(), W.data(), F.data(), wall.data(), counters);
    orc_macro(p, R.data(), W.data(), Th.data(), nullptr);
    if (newton) {
      int rc = orc_newton(p, T, Th.data(), R.data(), nullptr);
      if (rc != 0) return rc;
    }
    res = orc_residual(g.ncells, T, Th.data(), dT_ref);
    std::copy(Th.begin(), Th.end(), T);
    if (res_history) res_history[it] = res;
    ++it;
    if (res <= tol) break;
  }
  if (iters_out) *iters_out = it;
  if (res_out) *res_out = res;
  return 0;
}

// Adjoint of one sweep with its draws fixed. The forward map is
//   T_half[i] = sum over real collisions in i of w / (V m_i),  w = coef_p (T_emit[j] or T_w).
// Its transpose applied to lambda, by re-tracing each particle and gathering:
//   out[j]      = sum over particles p of cell j   of coef_p lambda[stop] / (V m_stop)
//   grad_wall[w] = sum over particles p of wall w  of coef_p lambda[stop] / (V m_stop)
// Every emitter is traced (no zero-weight skip). Outputs are overwritten.
int orc_adjoint_apply(const OrcProblem* p, const double* lambda, uint32_t epoch, double* out, double* grad_wall) {
  if (!valid(p)) return -1;
  Geo g(*p);
  std::vector<double> tmaj, m;
  majorants(*p, g, tmaj);
  cell_m(*p, g, m);
  std::fill(out, out + g.ncells, 0.0);
  std::fill(grad_wall, grad_wall + 2 * p->dim, 0.0);
  for_each_particle(*p, g, epoch, false, nullptr, nullptr, nullptr,
                    [&](int kind, int b, long long emitter, long long, double coef, double, Stream& st,
                        double* x, int* idx, const double* s) {
                      double gv = trace_particle(*p, g, b, tmaj[b], m.data(), st, x, idx, s, 0.0, nullptr, lambda);
                      if (kind == 0) out[emitter] += coef * gv;
                      else grad_wall[emitter] += coef * gv;
                    });
  return 0;
}

// Emission state of every particle of one emitter kind, for sampler tests: kind 0 =
// cell particles of cell `emitter`, kind 1 = particles of boundary face `emitter` (an
// index into the face numbering). Writes n_particles rows of x[3], s[3], and the
// first path length d (drawn exactly as trace_particle draws it).
int orc_emit(const OrcProblem* p, int kind, int band, long long emitter, uint32_t epoch,
             double* x_out, double* s_out, double* d_out) {
  if (!valid(p)) return -1;
  Geo g(*p);
  std::vector<double> tmaj;
  majorants(*p, g, tmaj);
  std::vector<double> ones(g.ncells, 1.0), wones(2 * p->dim, 1.0);
  long long k = 0;
  for_each_particle(*p, g, epoch, false, ones.data(), wones.data(), nullptr,
                    [&](int knd, int b, long long, long long face_or_cell, double, double, Stream& st,
                        double* x, int*, const double* s) {
                      if (knd != kind || b != band || face_or_cell != emitter) return;
                      for (int a = 0; a < 3; ++a) {
                        x_out[3 * k + a] = x[a];
                        s_out[3 * k + a] = s[a];
                      }
                      d_out[k] = -std::log(st.first_path_uniform()) * p->v[b] * tmaj[b];
                      ++k;
                    });
  return (int)k;
}

// Default split of N particles over bands by largest remainder of N r_b / sum r,
// with at least one particle per band (requires N >= nb). r_b > 0.
int orc_band_split(int nb, long long N, const double* r, long long* out) {
  if (nb < 1 || N < nb) return -1;
  double rs = 0.0;
  for (int b = 0; b < nb; ++b) {
    if (!(r[b] > 0.0)) return -1;
    rs += r[b];
  }
  // One particle to each band first, the remaining N - nb by largest remainder.
  long long rest = N - nb;
  std::vector<double> frac(nb);
  long long given = 0;
  for (int b = 0; b < nb; ++b) {
    double q = (double)rest * r[b] / rs;
    long long fl = (long long)std::floor(q);
    out[b] = 1 + fl;
    frac[b] = q - (double)fl;
    given += fl;
  }
  long long left = rest - given;
  std::vector<int> order(nb);
  for (int b = 0; b < nb; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return frac[a] > frac[c]; });
  for (long long k = 0; k < left; ++k) out[order[(size_t)(k % nb)]] += 1;
  return 0;
}

// ---------------------------------------------------------------------------
// Persistent null-collision population (Sec. 3.2 steps (1)-(6)). A fixed population of
// particles (Sec. 4.1: the count stays fixed, so a plain array holds it) makes one candidate
// flight per iteration. Each particle has a home: the cell of its last real collision or
// the boundary face through which a wall last absorbed it. A particle whose last flight
// ended at home is re-emitted from there (step (2)) with the home's equilibrium power shared
// by the particles that ended there: w = S_{b,c} / N_rc(b, c) in a cell
// (S = C_b T_emit V / tau_b, T_emit = T + Q/m from the current macro state), and
// w = (C_b v_b T_face A / 4) / N_abs(b, face) on a face (a black wall absorbs what reaches
// it and emits at its temperature). A null candidate keeps position, direction and weight
// and flies again (step (6)).
// Slots: per band N_b per cell in q-major order (slot q * ncells + cell), then per band
// N_w,b per boundary face (slot q * faces + face).
// Draws of slot k in iteration it: Stream(seed, instance, band, it, 0x80000000, k):
// emission uniforms if re-emitted, then the (path, accept) pair.
// Per slot: x[3], s[3], w, home (cell index, or ncells + boundary-face index in wall
// order), due (1: re-emit this iteration). n_home_prev / n_home_new: [nb * (ncells +
// boundary faces)] particles that ended at each home in the previous / this iteration.
// Outputs R, W, wall (overwritten), counters {flights, candidates, real, 0, wall exits, 0}.
int orc_persistent_step(const OrcProblem* p, const double* T, uint32_t it, long long n_slots, double* x, double* s,
                        double* w, const int* band, long long* home, int* due, const uint32_t* n_home_prev,
                        uint32_t* n_home_new, double* R, double* W, double* wall, unsigned long long* counters) {
  if (!valid(p)) return -1;
  Geo g(*p);
  std::vector<double> tmaj, m;
  majorants(*p, g, tmaj);
  cell_m(*p, g, m);
  long long wall_face_off[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int wl = 0; wl < 2 * g.dim; ++wl) {
    int a = wl / 2;
    wall_face_off[wl + 1] = wall_face_off[wl] + (long long)g.n[(a + 1) % 3] * g.n[(a + 2) % 3];
  }
  const long long nbf = wall_face_off[2 * g.dim];
  const long long nh = g.ncells + nbf;  // homes per band
  const long long bc = (long long)p->nb * g.ncells;
  std::fill(R, R + bc, 0.0);
  std::fill(W, W + bc, 0.0);
  std::fill(wall, wall + 2 * p->dim, 0.0);
  std::fill(n_home_new, n_home_new + (long long)p->nb * nh, 0u);
  for (int k = 0; k < 6; ++k) counters[k] = 0;
  for (long long i = 0; i < n_slots; ++i) {
    const int b = band[i];
    Stream st(p->seed, p->instance, (uint32_t)b, it, 0x80000000u, (uint32_t)i);
    double* xi = &x[3 * i];
    double* si = &s[3 * i];
    if (due[i]) {
      const long long h = home[i];
      const double nprev = (double)n_home_prev[(long long)b * nh + h];
      if (h < g.ncells) {  // step (2): re-emission in the cell of the real collision
        const int ci[3] = {(int)(h % g.n[0]), (int)((h / g.n[0]) % g.n[1]), (int)(h / ((long long)g.n[0] * g.n[1]))};
        for (int a = 0; a < g.dim; ++a) xi[a] = (ci[a] + st.uniform()) * g.h[a];
        for (int a = g.dim; a < 3; ++a) xi[a] = 0.0;
        const double u_mu = st.uniform();
        const double u_phi = g.dim >= 2 ? st.uniform() : 0.5;
        thermal_direction(g.dim, u_mu, u_phi, si);
        st.skip_to(emission_uniforms_thermal(g.dim));
        const double te = T[h] + (p->source ? p->source[h] / m[h] : 0.0);
        w[i] = p->C[b] * te * g.V / p->tau[(long long)b * g.ncells + h] / nprev;
      } else {  // re-emission from the boundary face that absorbed it
        const long long bf = h - g.ncells;
        int wl = 0;
        while (bf >= wall_face_off[wl + 1]) ++wl;
        const int a = wl / 2, side = wl % 2, o1 = (a + 1) % 3, o2 = (a + 2) % 3;
        const long long j = bf - wall_face_off[wl];
        int f[3];
        f[a] = side == 0 ? 0 : g.n[a];
        f[o1] = (int)(j % g.n[o1]);
        f[o2] = (int)(j / g.n[o1]);
        int idx[3];
        wall_start(g, a, side, f, st, xi, si, idx);
        const double Tf = p->wall_face_T ? p->wall_face_T[bf] : p->wall_T[wl];
        w[i] = p->C[b] * p->v[b] * g.A[a] * Tf / 4.0 / nprev;
      }
    }
    // step (3): one flight, path length -ln(u) v tau_maj
    counters[0] += 1;
    const double u_path = st.uniform();
    const double u_acc = st.uniform();
    const double ell = -std::log(u_path) * p->v[b] * tmaj[b];
    double tw = INFINITY;
    int wl = -1;
    for (int a = 0; a < g.dim; ++a) {
      if (si[a] == 0.0) continue;
      const double t = si[a] > 0.0 ? (g.L[a] - xi[a]) / si[a] : -xi[a] / si[a];
      if (t < tw) {
        tw = t;
        wl = 2 * a + (si[a] > 0.0 ? 1 : 0);
      }
    }
    if (wl >= 0 && tw < ell) {  // absorbed by the wall it reaches first
      wall[wl] += w[i];
      counters[4] += 1;
      const int a = wl / 2, o1 = (a + 1) % 3, o2 = (a + 2) % 3;
      int j1 = 0, j2 = 0;
      if (o1 < g.dim) j1 = std::min(std::max((int)std::floor((xi[o1] + tw * si[o1]) / g.h[o1]), 0), g.n[o1] - 1);
      if (o2 < g.dim) j2 = std::min(std::max((int)std::floor((xi[o2] + tw * si[o2]) / g.h[o2]), 0), g.n[o2] - 1);
      home[i] = g.ncells + wall_face_off[wl] + (long long)j2 * g.n[o1] + j1;
      due[i] = 1;
      n_home_new[(long long)b * nh + home[i]] += 1;
      continue;
    }
    for (int a = 0; a < g.dim; ++a) xi[a] += ell * si[a];
    int ci[3] = {0, 0, 0};
    for (int a = 0; a < g.dim; ++a) ci[a] = std::min(std::max((int)std::floor(xi[a] / g.h[a]), 0), g.n[a] - 1);
    const long long c = g.cell(ci);
    // steps (4)-(5): candidate at the destination; W from every candidate, W^h and N_rc
    // from real ones
    counters[1] += 1;
    const long long jb = (long long)b * g.ncells + c;
    W[jb] += w[i] * tmaj[b];
    if (u_acc < tmaj[b] / p->tau[jb]) {
      counters[2] += 1;
      R[jb] += w[i];
      home[i] = c;
      due[i] = 1;
      n_home_new[(long long)b * nh + c] += 1;
    } else {
      due[i] = 0;  // step (6): same direction and weight, a new path next iteration
    }
  }
  return 0;
}

}  // extern "C"
