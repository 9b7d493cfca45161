// Device-side building blocks of the IUGKP sweep (sm_103a): counter-based draws,
// particle emission from a cell's or a wall's equilibrium, and the cell-by-cell walk
// with null collisions. Method: Liu, Yang, Zhang, Ji, Xu, arXiv 2506.09465, Sec. 3.1
// (steps (1)-(3), inverse sampling of the free path) and Sec. 3.2 (candidate flights
// at the majorant rate, acceptance sigma / sigma_max).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "layout.h"

namespace iugkp {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds; each round takes
// the high and low halves of two 32x32 products, the key is bumped between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k.x += W0;
      k.y += W1;
    }
    uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Uniform in (0, 1) from the top 23 bits of a word: (2m + 1) 2^-24, exact in float
// and in double, so FP32 and FP64 tracking draw identical values.
template <typename Real>
__device__ __forceinline__ Real word_uniform(uint32_t a) {
  return (Real)((a >> 9) * 2u + 1u) * (Real)(1.0 / 16777216.0);
}

// The same value in FP32 without an integer-to-float conversion (those issue at a fraction
// of the FP32 rate): 1 + m 2^-23 from the mantissa bits, minus 1 - 2^-24, is exactly
// m 2^-23 + 2^-24 = (2m + 1) 2^-24 (representable, so the subtraction is exact).
template <>
__device__ __forceinline__ float word_uniform<float>(uint32_t a) {
  return __int_as_float(0x3F800000u | (a >> 9)) - 0.99999994f;
}

// The uniform stream of one particle: uniform j is word (j mod 4) of block j / 4,
// block k = Philox(counter (k, particle, emitter, band<<24 | epoch), key). Emission
// consumes j0 uniforms (j0 even). The first candidate's path word is made of bits the
// emission leaves unused in block 0 (first), its acceptance word is uniform j0; uniform
// j0 + 1 is not used, and candidate k >= 2 takes the pair (j0 + 2k - 2, j0 + 2k - 1), so
// every later pair lies in one block: one Philox call serves two candidates, and a flight
// whose first candidate needs no acceptance draw needs block 0 alone (2D: thermal and wall
// emission both).
struct Stream {
  uint4 ctr;
  uint2 key;
  uint4 buf;
  uint32_t j;      // index of the next uniform
  uint32_t first;  // the first candidate's path word (init)

  // 23 bits of block 0 that no uniform uses (uniforms take the top 23 bits of a word): the
  // low 9 bits of words x and y and bits 4..8 of word z, placed where word_uniform reads.
  __device__ __forceinline__ static uint32_t spare_word(uint4 b) {
    return (((b.x & 511u) << 14) | ((b.y & 511u) << 5) | ((b.z & 511u) >> 4)) << 9;
  }

  __device__ __forceinline__ void init(unsigned long long seed, uint32_t inst_id, uint32_t band,
                                       uint32_t epoch, uint32_t emitter, uint32_t particle) {
    key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ inst_id);
    ctr = make_uint4(0u, particle, emitter, (band << 24) | (epoch & 0xFFFFFFu));
    buf = philox4x32_10(ctr, key);  // block 0 holds the first emission draws
    first = spare_word(buf);
    j = 0;
  }
  // The same stream with no block computed yet (the first next_pair or load_block does it).
  __device__ __forceinline__ void init_lazy(unsigned long long seed, uint32_t inst_id, uint32_t band,
                                            uint32_t epoch, uint32_t emitter, uint32_t particle) {
    key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ inst_id);
    ctr = make_uint4(0u, particle, emitter, (band << 24) | (epoch & 0xFFFFFFu));
    j = 0;
  }
  __device__ __forceinline__ void load_block(uint32_t blk) {
    uint4 c = ctr;
    c.x = blk;
    buf = philox4x32_10(c, key);
  }
  __device__ __forceinline__ uint32_t word(uint32_t k) const {
    return k == 0 ? buf.x : (k == 1 ? buf.y : (k == 2 ? buf.z : buf.w));
  }
  // Uniform j (even) of the stream: word x of block j / 4, loaded here, or word z of the
  // block already loaded.
  __device__ __forceinline__ uint32_t even_word() {
    if ((j & 3u) == 0u) {
      load_block(j >> 2);
      return buf.x;
    }
    return buf.z;
  }
  // After the emission (j = j0): the first candidate's path and acceptance words.
  __device__ __forceinline__ void first_pair(uint32_t& a, uint32_t& b) {
    a = first;
    b = even_word();
    j += 2;
  }
  // Next (path, accept) pair; j is even.
  __device__ __forceinline__ void next_pair(uint32_t& a, uint32_t& b) {
    if ((j & 3u) == 0u) load_block(j >> 2);
    if (j & 2u) {
      a = buf.z;
      b = buf.w;
    } else {
      a = buf.x;
      b = buf.y;
    }
    j += 2;
  }
};

// Number of uniforms an emission consumes (even): thermal position per axis, mu,
// phi (dim >= 2); wall tangential positions, mu_n, phi (dim >= 2).
__host__ __device__ constexpr int thermal_uniforms(int dim) { return dim == 1 ? 2 : (dim == 2 ? 4 : 6); }
__host__ __device__ constexpr int wall_uniforms(int dim) { return dim == 1 ? 2 : 4; }

// Exact n / d for n < 2^31 and d >= 1 with M = floor((2^32 - 1) / d) from the host: since
// 2^32/d - 1 <= M < 2^32/d, umulhi(n, M) is floor(n/d) or one less, and one comparison of
// the remainder fixes it. Integer operations only (conversions issue at a low rate here).
__device__ __forceinline__ unsigned udiv(unsigned n, unsigned d, unsigned M) {
  unsigned q = __umulhi(n, M);
  q += (n - q * d >= d) ? 1u : 0u;
  return q;
}

template <typename Real>
struct RealTraits;
template <>
struct RealTraits<double> {
  __device__ __forceinline__ static double log_(double x) { return log(x); }
  __device__ __forceinline__ static void sincos2pi(double u, double* s, double* c) {
    double phi = 2.0 * 3.141592653589793 * u;
    sincos(phi, s, c);
  }
  __device__ __forceinline__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
};
template <>
struct RealTraits<float> {
  __device__ __forceinline__ static float log_(float x) { return __logf(x); }
  __device__ __forceinline__ static void sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
  __device__ __forceinline__ static float inf() { return __int_as_float(0x7f800000); }
};

// State of one particle's walk. t = path length from the emission point; tmax[a] =
// path length at which the next face normal to axis a is reached.
template <typename Real, int DIM>
struct Walk {
  int idx[3];
  int cell;  // linear cell index within the instance
  Real tmax[DIM];
  Real tdelta[DIM];
  int step[DIM];
  Real D;    // path length of the next candidate collision
};

// Sets up the DDA from the cell-local fractions xi[a] in [0, 1] and direction s.
template <typename Real, int DIM>
__device__ __forceinline__ void walk_init(Walk<Real, DIM>& w, const InstDesc& in, const Real* xi, const Real* s) {
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    Real h = (Real)in.h[a];
    if (s[a] > (Real)0) {
      w.step[a] = 1;
      w.tdelta[a] = h / s[a];
      w.tmax[a] = ((Real)1 - xi[a]) * h / s[a];
    } else if (s[a] < (Real)0) {
      w.step[a] = -1;
      w.tdelta[a] = h / (-s[a]);
      w.tmax[a] = xi[a] * h / (-s[a]);
    } else {
      w.step[a] = 1;
      w.tdelta[a] = RealTraits<Real>::inf();
      w.tmax[a] = RealTraits<Real>::inf();
    }
  }
  w.cell = w.idx[0] + in.n[0] * (w.idx[1] + in.n[1] * w.idx[2]);
}

// Thermal emission of particle `q` of cell `c` (Sec. 3.1 step (1)): uniform position in
// the cell, isotropic direction s = (mu, sin cos phi, sin sin phi), 1D/2D keep the
// leading components.
template <typename Real, int DIM>
__device__ __forceinline__ void emit_thermal(Walk<Real, DIM>& w, Stream& st, const InstDesc& in, int c) {
  w.idx[0] = c % in.n[0];
  w.idx[1] = (c / in.n[0]) % in.n[1];
  w.idx[2] = c / (in.n[0] * in.n[1]);
  Real xi[3], s[3];
  Real u_mu, u_phi = (Real)0.5;
  if (DIM == 1) {
    xi[0] = word_uniform<Real>(st.buf.x);
    u_mu = word_uniform<Real>(st.buf.y);
  } else if (DIM == 2) {
    xi[0] = word_uniform<Real>(st.buf.x);
    xi[1] = word_uniform<Real>(st.buf.y);
    u_mu = word_uniform<Real>(st.buf.z);
    u_phi = word_uniform<Real>(st.buf.w);
  } else {
    xi[0] = word_uniform<Real>(st.buf.x);
    xi[1] = word_uniform<Real>(st.buf.y);
    xi[2] = word_uniform<Real>(st.buf.z);
    u_mu = word_uniform<Real>(st.buf.w);
    st.load_block(1);
    u_phi = word_uniform<Real>(st.buf.x);
  }
  Real mu = (Real)2 * u_mu - (Real)1;
  s[0] = mu;
  if (DIM >= 2) {
    Real sn = sqrt((Real)1 - mu * mu);
    Real sp, cp;
    RealTraits<Real>::sincos2pi(u_phi, &sp, &cp);
    s[1] = sn * cp;
    s[2] = sn * sp;
  }
  st.j = thermal_uniforms(DIM);
  walk_init<Real, DIM>(w, in, xi, s);
}

// Wall emission of a particle of boundary face (wall, j1, j2): position uniform on the
// face, cosine-weighted direction into the domain (black isothermal wall).
template <typename Real, int DIM>
__device__ __forceinline__ void emit_wall(Walk<Real, DIM>& w, Stream& st, const InstDesc& in, int wall, int j1,
                                          int j2) {
  const int a = wall >> 1, side = wall & 1;
  const int o1 = (a + 1) % 3, o2 = (a + 2) % 3;
  w.idx[a] = side ? in.n[a] - 1 : 0;
  w.idx[o1] = j1;
  w.idx[o2] = j2;
  Real xi[3] = {(Real)0.5, (Real)0.5, (Real)0.5};
  xi[a] = side ? (Real)1 : (Real)0;
  Real u_n, u_phi = (Real)0.5;
  if (DIM == 1) {
    u_n = word_uniform<Real>(st.buf.x);
  } else if (DIM == 2) {
    // the one in-domain tangential axis is the smaller of o1, o2 that is < 2
    int t = (o1 < 2) ? o1 : o2;
    xi[t] = word_uniform<Real>(st.buf.x);
    u_n = word_uniform<Real>(st.buf.y);
    u_phi = word_uniform<Real>(st.buf.z);
  } else {
    int t0 = o1 < o2 ? o1 : o2, t1 = o1 < o2 ? o2 : o1;
    xi[t0] = word_uniform<Real>(st.buf.x);
    xi[t1] = word_uniform<Real>(st.buf.y);
    u_n = word_uniform<Real>(st.buf.z);
    u_phi = word_uniform<Real>(st.buf.w);
  }
  Real s[3];
  Real mn = sqrt(u_n);
  s[a] = side ? -mn : mn;
  if (DIM >= 2) {
    Real st_ = sqrt((Real)1 - u_n);
    Real sp, cp;
    RealTraits<Real>::sincos2pi(u_phi, &sp, &cp);
    s[o1] = st_ * cp;
    s[o2] = st_ * sp;
  } else {
    s[o1] = (Real)0;
    s[o2] = (Real)0;
  }
  st.j = wall_uniforms(DIM);
  walk_init<Real, DIM>(w, in, xi, s);
}

// Index of the face crossed when leaving cell (idx) along axis a with direction step,
// within the instance's face numbering.
template <int DIM>
__device__ __forceinline__ long long face_index(const InstDesc& in, const int* idx, int cell, int a, int step) {
  int up = step > 0 ? 1 : 0;
  if (a == 0) return in.fax_off[0] + (long long)cell + (idx[1] + in.n[1] * idx[2]) + up;
  if (a == 1) return in.fax_off[1] + (long long)cell + (long long)in.n[0] * idx[2] + (long long)in.n[0] * up;
  return in.fax_off[2] + (long long)cell + (long long)in.n[0] * in.n[1] * up;
}

// Resolves a global particle index to its group (binary search over the prefix offsets).
__device__ __forceinline__ int find_group(const Group* g, int n_groups, long long pid) {
  int lo = 0, hi = n_groups - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (g[mid].first_particle <= pid) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

}  // namespace iugkp
