// Work distribution of the staged sweep (sweep_staged.cu), built on the host.
#pragma once

namespace iugkp {

constexpr int STAGED_NT = 1024;                 // threads per persistent block
constexpr int WALK_MIN_LANES = 8;               // 3D per-lane walk: fewest lanes worth a step

// 3D face tallies: the warp tallies the items of the particles that ended together; per warp a
// table of 64 item lists (the x- and y-faces of each lane's particle, 3 int4 of parameters
// each) and their 65 start offsets, in the dynamic shared memory (3D instances keep no face
// window there).
constexpr int COOP3_LISTS = 64;
constexpr int COOP3_INT4_PER_WARP = COOP3_LISTS * 3 + 17;  // parameters, then the starts (65 ints)
constexpr int COOP3_BYTES = (STAGED_NT / 32) * COOP3_INT4_PER_WARP * 16;

// Shared-memory x-face window: one 32-bit word per face holding the low word of a 64-bit
// fixed-point sum in units of w_max 2^-26 (a contribution is below 2^26 units); words start
// at 2^31, and a wrap of the word adds +-2^32 units (= 64 w_max) to the FP64 face at once.
constexpr double WIN_SCALE = 0x1p26;
constexpr double WIN_CARRY = 0x1p6;             // 2^32 units in multiples of w_max
constexpr unsigned WIN_BIAS = 0x80000000u;

// Copies of the two-group exit tally GX (one per block, by block index modulo the count),
// summed when the untallied faces are derived. Exits through one wall pile onto a few hundred
// faces (a single 128 x 128 instance at Kn 10 sends ~4e6 exits to 256 of them); FP64
// atomics to one address serialise at its L2 slice, so one copy made the sweep's time
// depend on which slices those lines landed in.
constexpr int GX_COPIES = 16;

struct StagedArgs {
  int n_inst;
  unsigned long long* inst_next;  // [n_inst] next unclaimed forward particle of each instance
  const long long* inst_end;      // [n_inst] end of each instance's forward particle range
  const double* cost_prefix;      // [n_inst] prefix sums of the estimated cost
  double cost_total;
  const int2* window;             // [n_inst] {first x-face, count} tallied in shared memory
  const double* wmax;             // [n_inst] largest |particle weight| of the sweep
  int warp_grab;                  // particles a warp claims at a time
  int refill;                     // idle lanes that trigger a refill (0: per-instance default)
  int walk_k;                     // crossings per lane between bulk steps
  // division magics M = floor((2^32 - 1) / d) of the divisors d below
  const unsigned* group_mag;      // [forward groups] d = emitters of the group
  const unsigned* mag_n0;         // [n_inst] d = n_x
  const unsigned* mag_n1;         // [n_inst] d = n_y
  const unsigned* mag_wall;       // [n_inst * 3] d = cells along the first tangential axis of each wall
  // compensated FP32 tallies (IUGKP_TALLY_STAGED_K32): {high word, error word} per entry
  float2* R32;                    // [nb * total_cells]
  float2* W32;                    // [nb * total_cells] or null
  float2* F32;                    // [total_faces] face tallies that miss the window, or null
  // Two-group face tallies (2D instances whose faces all fit the window): a particle whose
  // path per cell along x is at least that along y (d_x >= d_y) is in the x-group and
  // tallies the faces normal to x it crosses; the others (y-group) tally the faces normal
  // to y. The untallied faces of each group follow from that group's own power balance.
  double* DY;                     // [total_cells] y-group: absorbed minus emitted power per cell
  double* EY;                     // [total_bfaces] y-group wall emission per boundary face (signed
                                  // flux: + on the low walls, - on the high walls)
  double* GX;                     // [GX_COPIES][total_bfaces] exits of the x-group through the low
                                  // y-wall and of the y-group through the low x-wall (signed flux)
  long long gx_stride;            // total_bfaces: entries per copy of GX
  // Particles whose FP32 walk lies within rounding of a decision of the FP64 walk are left
  // untallied and replayed by the FP64 walk after the sweep (replay_kernel): entry
  // {forward index, (candidates already tallied << 1) | y-group}.
  uint2* defer;                   // [defer_cap]
  unsigned* defer_n;              // entries pushed by this sweep (beyond defer_cap: overflow)
  unsigned defer_cap;
  int* err;                       // device error word (ERR_DEFER on overflow)
#ifdef __CUDACC__
  // this block's copy of GX
  __device__ __forceinline__ double* gx() const {
    return GX + (long long)(blockIdx.x % (unsigned)GX_COPIES) * gx_stride;
  }
#endif
};

}  // namespace iugkp
