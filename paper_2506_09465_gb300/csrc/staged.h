// Work distribution of the staged sweep (sweep_staged.cu), built on the host.
#pragma once

namespace iugkp {

constexpr int STAGED_NT = 1024;                 // threads per persistent block

struct StagedArgs {
  int n_inst;
  unsigned long long* inst_next;  // [n_inst] next unclaimed forward particle of each instance
  const long long* inst_end;      // [n_inst] end of each instance's forward particle range
  const double* cost_prefix;      // [n_inst] prefix sums of the estimated cost
  double cost_total;
  const int* win_fits;            // [n_inst] 1 if all x-faces fit the shared-memory window
  const double* wmax;             // [n_inst] largest |particle weight| of the sweep
  int warp_grab;                  // particles a warp claims at a time
  int refill;                     // idle lanes that trigger a refill (0: per-instance default)
  int walk_k;                     // crossings per lane between bulk steps
  const float* group_rcp;         // [forward groups] 1 / particles per emitter
  const float* rcp_n0;            // [n_inst] 1 / n_x
  const float* rcp_n1;            // [n_inst] 1 / n_y
  const float* rcp_wall;          // [n_inst * 3] 1 / (cells along the first tangential axis of each wall)
  // compensated FP32 tallies (IUGKP_TALLY_STAGED_K32): {high word, error word} per entry
  float2* R32;                    // [nb * total_cells]
  float2* W32;                    // [nb * total_cells] or null
  float2* F32;                    // [total_faces] face tallies that miss the window, or null
};

}  // namespace iugkp
