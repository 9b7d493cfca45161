// Host-side context of the CUDA library and the launchers shared between its
// translation units. Not part of the public ABI (include/iugkp.h is).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/iugkp.h"
#include "layout.h"
#include "staged.h"

namespace iugkp {

// Counts of particles absorbed through one boundary face are spread over this many copies
// (by lane), summed when the face's power is shared out: a wall face receives far more
// absorptions per iteration than a cell receives real collisions, and same-address atomics
// serialise at the L2.
// Fewest emitters per block of the w_max pre-pass of the staged sweep (4 per thread); above
// that the pass takes about two blocks per SM.
constexpr int WMAX_MIN_CHUNK = 1024;

constexpr int PERS_FACE_REPLICAS = 32;

struct InstMG;

// Arguments of the forward and adjoint sweep kernels (all device pointers).
struct SweepArgs {
  const InstDesc* inst;
  const Group* groups;
  int n_groups;
  int nb;
  long long total_particles;
  const double* T;         // [cells] temperature (forward)
  const double* srcshift;  // [cells] Q / m, or null
  const double* coef;      // [bc] C_b V / (tau N_b): weight per unit emission temperature
  const double* ratio64;   // [bc] tau_maj / tau (acceptance probability of a candidate)
  const float* ratio32;
  const float* ratio_nb32; // [bc] largest ratio32 over the cell and its neighbours
  const int* all_real;     // [inst * nb] 1 where tau = tau_maj in every cell (every candidate real)
  const int* perm;         // staged visiting order of the emitters of groups with perm_off >= 0
  const double* taumaj;    // [inst * nb] majorant tau per instance and band
  const double* v;         // [nb] group speed
  const float* vtm32;      // [inst * nb] v_b tau_maj in FP32
  const double* wcoef;     // [inst * nb * 6] C_b v_b A / (4 N_w) per wall
  const double* wallT;     // [walls]
  double* wemit;           // [bc] staged sweep: weight of every thermal emitter (w_max pre-pass)
  const double* wallTf;    // [boundary faces] temperature of every boundary face
  double* R;
  double* W;
  double* F;
  double* wall;
  unsigned long long* counters;
  const double* lambda;    // adjoint: [cells]
  const double* invVm;     // adjoint: [cells] 1 / (V m)
  double* adj_out;         // adjoint: [cells] (A^T lambda)
  double* adj_wall;        // adjoint: [walls]
  unsigned long long seed;
  unsigned epoch;
  long long budget;
  int* err;
  unsigned long long* work_counter;  // persistent schedule: next particle index
  int staged_faces;                  // staged schedule: faces held in shared memory (0 = none)
  int dim;
};

struct Ctx {
  std::string err;
  iugkp_options opt;
  int n_inst = 0, dim = 0, nb = 0;
  long long total_cells = 0, total_faces = 0, total_walls = 0, total_particles = 0;
  int max_inst_faces = 0, max_inst_cells = 0;
  std::vector<InstDesc> h_inst;
  std::vector<Group> h_groups_all;  // every emitter (adjoint)
  std::vector<Group> h_groups_fwd;  // walls at T_w = 0 left out (forward)
  long long fwd_particles = 0;
  std::vector<double> h_wallT;      // [walls]
  std::vector<double> h_wallTf;     // [boundary faces]
  long long total_bfaces = 0;
  std::vector<double> h_C, h_v;
  std::vector<long long> h_nband, h_nwall;
  std::vector<double> h_theta;      // per instance damping of the Newton correction
  std::vector<double> h_Vcell;      // per instance cell volume
  std::vector<iugkp_grid> h_grids;  // the grids the context was created with

  // device buffers
  InstDesc* d_inst = nullptr;
  Group* d_groups_all = nullptr;
  Group* d_groups_fwd = nullptr;
  double* d_coef = nullptr;
  double* d_ratio64 = nullptr;
  float* d_ratio32 = nullptr;
  float* d_ratio_nb32 = nullptr; // [nb * cells] largest FP32 ratio over each cell's neighbourhood
  int* d_perm = nullptr;         // emitter visiting orders of the groups (Group::perm_off)
  int* d_wmax_bpre = nullptr;    // [forward groups + 1] first block of each group in the w_max pre-pass
                                 // (in proportion to its emitters)
  int wmax_blocks = 0;           // blocks of that pass
  int* d_all_real = nullptr;     // [inst * nb] tau = tau_maj in every cell of the band
  bool all_real_all = false;     // ... in every instance and band
  double* d_taumaj = nullptr;
  float* d_vtm32 = nullptr;
  double* d_v = nullptr;
  double* d_wcoef = nullptr;
  double* d_wallT = nullptr;
  double* d_wemit = nullptr;     // [nb * cells] emitter weights of the current sweep
  // two-group face tallies of the staged sweep (2D): group balances and derived faces
  double* d_DY = nullptr;        // [cells]
  double* d_EY = nullptr;        // [total_bfaces]
  double* d_GX = nullptr;        // [GX_COPIES * total_bfaces]
  double* d_Fd = nullptr;        // [total_faces] faces derived from the group balances
  bool any_two_group = false;    // some instance of the context uses the two-group tallies
  bool all_two_group = false;    // ... every instance does (no face follows from a column walk)
  bool sync_ok = false;          // 2D: the pass-synchronous staged kernel applies
  bool sync_partial = false;     // ... and some instance's x-faces exceed the window
  double* d_wallTf = nullptr;    // [total_bfaces]
  double* d_srcshift = nullptr;  // null when no source
  double* d_source = nullptr;    // Q (kept for set_field)
  double* d_m = nullptr;         // [cells] sum_b C_b / tau_b
  double* d_Vm = nullptr;        // [cells] V m
  double* d_invVm = nullptr;     // [cells] 1 / (V m)
  double* d_VC = nullptr;        // [cells] V sum_b C_b
  double* d_theta = nullptr;     // [n_inst] damping of the Newton correction
  double* d_theta_m = nullptr;   // [cells] theta_k m_i (adjoint correction)
  double* d_diag = nullptr;      // [cells] diffusion operator diagonal
  double* d_cx = nullptr;        // [cells] coupling to the +x neighbour (0 at the row end)
  double* d_cy = nullptr;
  double* d_cz = nullptr;
  double* d_pcg = nullptr;       // [5 * cells] x, r, p, q, z
  double* d_work = nullptr;      // [cells] scratch
  double* d_T2 = nullptr;        // [cells] scratch iterate
  double* d_R = nullptr;         // [nb * cells]
  double* d_W = nullptr;
  double* d_F = nullptr;
  double* d_wall = nullptr;
  float2* d_R32 = nullptr;       // compensated FP32 tallies {hi, err} (allocated on first use)
  float2* d_W32 = nullptr;
  float2* d_F32 = nullptr;
  double* d_red = nullptr;       // reduction scratch
  unsigned long long* d_counters = nullptr;
  unsigned long long* d_work_counter = nullptr;
  int* d_err = nullptr;
  int* d_pcg_iters = nullptr;    // [n_inst]
  double* d_scalar = nullptr;    // [8] small results
  double* d_adj = nullptr;       // [4 * cells] adjoint iteration buffers (allocated on first use)
  double* d_m2 = nullptr;        // [cells] averaging: sum of squared deviations (allocated on first use)
  // persistent null-collision population (persistent.cu), allocated by iugkp_persistent_reset
  long long pers_n = 0;          // slots of all instances
  long long pers_homes = 0;      // per-(band, home) counters of all instances
  int pers_parity = 0;           // which half of d_pcount holds the previous iteration
  long long* d_pslot_off = nullptr;
  long long* d_phome_off = nullptr;
  long long* d_pnband = nullptr;  // [n_inst * nb]
  long long* d_pnwall = nullptr;  // [nb]
  double* d_px = nullptr;         // [7 * pers_n] doubles: x, y, z, s_x, s_y, s_z (FP64, or FP32 packed
                                  // at the start), then w at 6 * pers_n
  double* d_phome_w = nullptr;    // [pers_homes] power per re-emitted particle of each home
  int* d_pband = nullptr;
  int* d_phome = nullptr;
  unsigned* d_pcount = nullptr;   // [2 * pers_homes] (cell homes; the entries of face homes stay 0)
  unsigned* d_pfcount = nullptr;  // [2 * PERS_FACE_REPLICAS * face homes] face-home counts, replicated
  double* h_pinned = nullptr;    // [8 + n_inst] host readback
  // multigrid preconditioner of the Newton correction (mg_setup.cu, mgpcg.cu)
  struct InstMG* d_mg = nullptr;
  size_t mg_smem_bytes = 0;      // dynamic shared memory of the PCG kernel (CTA 0's coarse levels)
  float* d_mg_diag = nullptr;
  float* d_mg_dinv = nullptr;
  float* d_mg_cx = nullptr;
  float* d_mg_cy = nullptr;
  float* d_mg_cz = nullptr;
  float* d_mg_cinv = nullptr;
  float* d_mg_b = nullptr;
  float* d_mg_x = nullptr;
  float* d_mg_t = nullptr;
  float* d_mg_r = nullptr;
  float* d_fd_q = nullptr;       // fast diagonalization: eigenvector matrices (FP32)
  float* d_fd_lam = nullptr;     // ... and eigenvalues
  long long mg_level_cells = 0;
  // staged sweep
  long long* d_inst_beg = nullptr;   // [n_inst] forward particle range per instance
  long long* d_inst_end = nullptr;
  unsigned long long* d_inst_next = nullptr;
  double* d_cost_prefix = nullptr;
  double cost_total = 0.0;
  int2* d_window = nullptr;      // [n_inst] {first x-face, count} of the shared-memory window
  unsigned long long* d_wmax = nullptr;  // [n_inst] bit patterns of the largest weight
  unsigned* d_group_mag = nullptr;   // [forward groups] division magic of the emitter count
  double* d_wall_unit = nullptr;     // [n_inst * 6] power entering per face per unit wall T
  // adjoint re-trace over all groups (staged kernel)
  long long* d_all_beg = nullptr;
  long long* d_all_end = nullptr;
  double* d_all_cost_prefix = nullptr;
  double all_cost_total = 0.0;
  unsigned* d_all_group_mag = nullptr;
  int adj_blocks_per_sm = 1;
  // particles the staged FP32 walk left to the FP64 replay (sweep and adjoint re-trace)
  uint2* d_defer = nullptr;
  unsigned* d_defer_n = nullptr;
  unsigned defer_cap = 0;
  unsigned* d_mag = nullptr;         // [n_inst * 5]: division magics of n_x, n_y, n(o1) for walls normal to x, y, z
  int staged_cap = 0;           // x-faces per shared-memory window
  int staged_blocks_per_sm = 1;
  std::vector<double> h_taumean;  // [inst * nb]
  // graph-captured steady iterations
  cudaStream_t graph_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  double* d_res_block = nullptr;  // [2 * GRAPH_ITERS] residual sums of a replay
  int sm_count = 0;
  size_t smem_optin = 0;
};

// Status helpers
iugkp_status fail(Ctx* c, iugkp_status s, const std::string& msg);
iugkp_status cuda_fail(Ctx* c, cudaError_t e, const char* what);

// Launchers (return the cudaError_t of the launch)
cudaError_t launch_sweep(const Ctx* c, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_adjoint(const Ctx* c, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_macro(const Ctx* c, const double* R, const double* W, double* T_half, double* T_E, cudaStream_t s);
cudaError_t launch_newton(const Ctx* c, const double* T_n, double* T_half, const double* R, cudaStream_t s);
cudaError_t launch_adjoint_correction(const Ctx* c, const double* lam, const double* half, double* out,
                                      cudaStream_t s);
cudaError_t launch_residual(const Ctx* c, const double* T0, const double* T1, double dT_ref, double* out_dev,
                            cudaStream_t s);
cudaError_t launch_pcg_check(const Ctx* c, cudaStream_t s);
cudaError_t launch_axpy_grad(const Ctx* c, const double* at, const double* g, double* lam_half, cudaStream_t s);
cudaError_t launch_sweep_staged(const Ctx* c, const SweepArgs& a, cudaStream_t s);
cudaError_t configure_staged(Ctx* c);
cudaError_t launch_adjoint_staged(const Ctx* c, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_replay(const Ctx* c, const SweepArgs& a, const StagedArgs& S, cudaStream_t s);
cudaError_t launch_adjoint_replay(const Ctx* c, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_walk_bounds(unsigned long long* out, cudaStream_t s);
double walk_bound_fraction(const double* measured);
cudaError_t measure_atomic_rate(int sm_count, double* out_rate);
cudaError_t launch_mgpcg(const Ctx* c, const double* rhs, cudaStream_t s);
size_t mg_solo_smem_bytes(const std::vector<InstMG>& h_mg);
cudaError_t configure_mgpcg(Ctx* c, size_t smem);
size_t fd_small_smem_bytes();  // dynamic shared memory of the in-shared-memory fast diagonalization
int fd_small_max_n();          // its largest axis size
iugkp_status build_multigrid(Ctx* c, const std::vector<double>& diag, const std::vector<double>& cx,
                             const std::vector<double>& cy, const std::vector<double>& cz,
                             const std::vector<double>& kap, double cvsum);
cudaError_t launch_grad_source(const Ctx* c, const double* at, double* grad, cudaStream_t s);
cudaError_t launch_persistent_init(Ctx* c, cudaStream_t s);
cudaError_t launch_persistent_step(const Ctx* c, const double* T, unsigned it, double* R, double* W, double* wall,
                                   unsigned long long* counters, cudaStream_t s);
cudaError_t launch_welford(const Ctx* c, const double* x, double* mean, double* m2, long long n, int k,
                           cudaStream_t s);
cudaError_t launch_scale(const Ctx* c, double* x, long long n, double a, cudaStream_t s);

}  // namespace iugkp
