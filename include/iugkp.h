/*
 * iugkp.h -- C ABI of the GB300 (sm_103a) implementation of the implicit unified
 * gas-kinetic particle (IUGKP) steady-state solver for the gray / band-resolved
 * phonon BGK equation (Liu, Yang, Zhang, Ji, Xu, arXiv 2506.09465).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns iugkp_status; none aborts, throws or exits. On failure
 *   iugkp_last_error(ctx) returns a message (valid until the next call on ctx).
 * - Deviational temperature T (T_ref = 0, Sec. 2, Eq. "derivation final
 *   equilibrium"): all temperatures, sources and tallies are linear in T.
 * - Grids are uniform and structured on [0, lx] x [0, ly] x [0, lz]. Cells are
 *   numbered x fastest: i = ix + nx (iy + ny iz). Unused axes have n = 1 and length 1,
 *   so 1D quantities are per unit area and 2D ones per unit depth.
 * - Faces: all x-faces first ((nx+1) ny nz of them, index fx + (nx+1)(iy + ny iz)),
 *   then y-faces (nx (ny+1) nz), then z-faces (nx ny (nz+1)); a dimension's faces
 *   exist only for axes < dim. Boundary faces are included.
 * - Walls: 2*dim per instance in the order -x, +x, -y, +y, -z, +z.
 * - A context holds n_inst >= 1 instances (same dim and band table, any sizes).
 *   Per-cell device arrays are the instances' arrays concatenated; per-(band, cell)
 *   arrays are [instance][band][cell]; faces and walls likewise per instance. Use
 *   iugkp_get_layout() for the offsets.
 * - Pointers named *_dev are caller-owned device memory (contiguous, FP64 unless
 *   stated), read or written on the caller's stream `cuda_stream` (a cudaStream_t;
 *   NULL = the legacy default stream). Host pointers are read during the call only.
 *   Nothing retains a caller pointer after the call returns.
 * - Thread safety: calls on one context must be serialised by the caller; distinct
 *   contexts are independent.
 */
#ifndef IUGKP_H
#define IUGKP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IUGKP_OK = 0,
  IUGKP_EINVAL = 1,   /* invalid argument (sizes, tau <= 0 or not finite, NULL, ...) */
  IUGKP_ENOMEM = 2,   /* device or host allocation failed */
  IUGKP_ECUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error) */
  IUGKP_ENOCONV = 4,  /* an iteration hit its limit before its tolerance */
  IUGKP_EBUDGET = 5,  /* a particle exceeded the per-particle step budget (dropped) */
  IUGKP_EDEVICE = 6   /* a device-side check failed (index out of range, bad state) */
} iugkp_status;

typedef struct iugkp_ctx iugkp_ctx; /* opaque; owned by the library */

/* Uniform structured grid: dim in {1, 2, 3}; n >= 1 and l > 0 on used axes. */
typedef struct {
  int dim, nx, ny, nz;
  double lx, ly, lz;
} iugkp_grid;

/* Band-branch table (host arrays of nb entries): volumetric specific heat C_b > 0
 * and group speed v_b > 0. Gray = one band. (Sec. 2: energy density form; band sums
 * of Eq. "derivation function".) */
typedef struct {
  int nb;
  const double *C;
  const double *v;
} iugkp_bands;

enum { IUGKP_TRACK_FP64 = 0, IUGKP_TRACK_FP32 = 1 };
enum { IUGKP_TALLY_FP64 = 0, IUGKP_TALLY_STAGED = 1, IUGKP_TALLY_STAGED_K32 = 2 };
enum { IUGKP_DRAWS_FRESH = 0, IUGKP_DRAWS_FROZEN = 1 };
enum { IUGKP_SCHED_PLAIN = 0, IUGKP_SCHED_PERSISTENT = 1 };

typedef struct {
  int precision;      /* IUGKP_TRACK_FP64: positions, directions and paths in FP64;
                         IUGKP_TRACK_FP32: in FP32 (weights and tallies stay FP64). */
  int tally;          /* IUGKP_TALLY_FP64: every face / deposit tally is a global FP64
                         atomic; IUGKP_TALLY_STAGED (FP32 tracking only): x-face tallies
                         are exact 64-bit fixed-point sums in a per-block shared-memory
                         window flushed to FP64, last-axis faces and walls follow from
                         per-cell conservation, deposits R, W are FP64 atomics;
                         IUGKP_TALLY_STAGED_K32: as STAGED, but deposits and the face
                         tallies that miss the window are compensated FP32 sums (a high
                         word plus a word that collects each addition's exact rounding
                         error), turned into FP64 after the sweep. Outputs stay FP64. */
  int draws;          /* IUGKP_DRAWS_FRESH: epoch = epoch0 + iteration;
                         IUGKP_DRAWS_FROZEN: epoch = epoch0 every iteration. */
  int newton;         /* 0: plain iteration; 1: inexact-Newton diffusion correction. */
  int schedule;       /* IUGKP_SCHED_PLAIN: one thread per particle;
                         IUGKP_SCHED_PERSISTENT: persistent warps that refill lanes. */
  long long particles_per_cell;       /* N_cell >= nb; split over bands (largest remainder) */
  long long particles_per_wall_face;  /* >= nb; split over bands by C_b v_b */
  unsigned long long seed;            /* Philox key (low, high words) */
  unsigned epoch0;                    /* first epoch (24 bits used) */
  unsigned instance_base;             /* instance k of a batch draws with id base + k */
  double cg_rtol;                     /* PCG relative tolerance (Newton step) */
  int cg_maxit;                       /* PCG iteration cap -> IUGKP_ENOCONV */
  long long step_budget;              /* max crossings + candidates per particle */
  int block_threads;                  /* threads per block of the trace kernel (0 = auto) */
  int blocks_per_sm;                  /* persistent blocks per SM (0 = auto) */
  int refill_lanes;                   /* staged sweep: a warp refills its idle lanes once at
                                         least this many (1..32) are idle; 0 = chosen per
                                         instance from the expected events per particle.
                                         0 or 32 in 2D when every instance's tallied faces
                                         fit the shared-memory window: pass-synchronous
                                         schedule (each pass of a warp emits up to 32
                                         particles, follows each to its end, then tallies
                                         their faces together) */
  int use_graphs;                     /* 1: iugkp_solve_steady with frozen draws replays a
                                         CUDA graph of two iterations (one host readback per
                                         two iterations); 0: plain launches */
  int warp_grab;                      /* staged sweep: particles a warp claims at a time
                                         (0 = 256) */
  int walk_k;                         /* staged sweep: crossings a lane walks between bulk
                                         steps (0 = 16) */
} iugkp_options;

/* Fills *o with defaults: FP32 tracking, staged tallies, frozen draws, Newton on,
 * persistent schedule, 1024 particles per cell and per wall face, seed 0,
 * cg_rtol 1e-3 (the correction is an inexact Newton step: its tolerance changes the
 * iteration count, not the fixed point), cg_maxit 5000, step budget 2^24. */
void iugkp_default_options(iugkp_options *o);

/* Creates a context for one instance (Sec. 4 problem setup).
 *   tau     host [nb][ncells], relaxation time per band and cell, finite and > 0;
 *   wall_T  host [2*dim] deviational wall temperatures;
 *   source  host [ncells] heat source power density, or NULL for none.
 * Device memory for all internal fields is allocated here (cudaMalloc on the
 * current device). EINVAL on bad input, ENOMEM / ECUDA on allocation failure. */
iugkp_status iugkp_create(const iugkp_grid *g, const double *tau, const iugkp_bands *b,
                          const double *wall_T, const double *source, const iugkp_options *o,
                          iugkp_ctx **out);

/* Creates one context holding n instances (same dim and bands); g[k], tau[k],
 * wall_T[k], source[k] (source may be NULL or have NULL entries). Instance k uses
 * Philox id instance_base + k, so it draws exactly what it would draw alone. */
iugkp_status iugkp_create_batch(int n, const iugkp_grid *g, const double *const *tau,
                                const iugkp_bands *b, const double *const *wall_T,
                                const double *const *source, const iugkp_options *o,
                                iugkp_ctx **out);

void iugkp_destroy(iugkp_ctx *ctx);

const char *iugkp_last_error(const iugkp_ctx *ctx);

/* Sizes and offsets of the concatenated arrays. Each array argument may be NULL;
 * *_off arrays have n_inst + 1 entries (prefix sums). */
typedef struct {
  int n_inst, dim, nb;
  long long total_cells, total_faces, total_walls; /* walls = 2*dim per instance */
  long long total_particles;                       /* per sweep, every emitter counted */
  long long total_wall_faces;                      /* boundary faces of all instances */
} iugkp_layout;
iugkp_status iugkp_get_layout(const iugkp_ctx *ctx, iugkp_layout *lay, long long *cell_off,
                              long long *face_off);

/* Replaces a field. which: IUGKP_FIELD_SOURCE ([total_cells] power density),
 * IUGKP_FIELD_WALL_T ([total_walls]: every face of each wall takes its wall's value),
 * IUGKP_FIELD_WALL_FACE_T ([total_wall_faces]: the temperature of every boundary face, for
 * non-uniform walls such as the heated segment of Sec. 4.5; instance-major, walls in the
 * order -x, +x, -y, +y, -z, +z, on the wall normal to axis a the faces run over the axes
 * (a+1)%3 and (a+2)%3, the first fastest). Wall emission per face is C_b v_b T_face A / 4
 * (Sec. 4 black isothermal walls, per face). IUGKP_FIELD_TAU ([instance][band][cell], the
 * layout of iugkp_create_batch's tau: finite and > 0) replaces the relaxation times tau(omega,
 * x) (Sec. 3.2, spatially varying tau): the band split of the particles, the emitter weights,
 * the per-band majorant and acceptance ratios, kappa and the Newton correction's operator and
 * damping, and the source shift are rebuilt exactly as iugkp_create_batch would build them
 * (device buffers are reallocated; the wall temperatures, per-face ones included, the source
 * and the options carry over; a persistent population must be reset again). `data` is host
 * memory unless on_device != 0 (then read back, synchronising cuda_stream). Values must be
 * finite (EINVAL). */
enum { IUGKP_FIELD_SOURCE = 0, IUGKP_FIELD_WALL_T = 1, IUGKP_FIELD_WALL_FACE_T = 2, IUGKP_FIELD_TAU = 3 };
iugkp_status iugkp_set_field(iugkp_ctx *ctx, int which, const double *data, int on_device,
                             void *cuda_stream);

/* One sweep (Sec. 3.1 steps (1)-(3) with the null collisions of Sec. 3.2): every
 * cell emits particles from its equilibrium at T_in_dev (+ source), every wall from
 * its temperature; each particle is traced cell by cell through null candidates to a
 * real collision or a wall. Outputs (overwritten; any may be NULL except R_dev):
 *   R_dev        [inst][band][cell] real-collision power (the paper's W^h);
 *   W_dev        [inst][band][cell] candidate estimator of energy (the paper's W);
 *   F_dev        [total_faces] net power across each face in the +axis direction;
 *   wall_dev     [total_walls] power absorbed by each wall;
 *   counters_dev [6] u64: flights, candidates, real collisions, cell crossings,
 *                wall exits, dropped (step budget).
 * epoch selects the draws (24 bits). Asynchronous on cuda_stream except for the
 * device-error check, which synchronises the stream (EBUDGET / EDEVICE). */
iugkp_status iugkp_sweep(iugkp_ctx *ctx, const double *T_in_dev, unsigned epoch, double *R_dev,
                         double *W_dev, double *F_dev, double *wall_dev,
                         unsigned long long *counters_dev, void *cuda_stream);

/* Macro update (Sec. 3.1 step (3)): T_half = sum_b R_b / (V sum_b C_b / tau_b) and,
 * if T_E_dev != NULL and W_dev != NULL, T_E = sum_b W_b / (V sum_b C_b). */
iugkp_status iugkp_macro(iugkp_ctx *ctx, const double *R_dev, const double *W_dev,
                         double *T_half_dev, double *T_E_dev, void *cuda_stream);

/* Inexact-Newton correction (Sec. 3.3): s = (sum_b R_b - sum_b C_b T_n V / tau_b) / V,
 * solves -div(kappa grad dT) = s to ||s - A dT|| <= cg_rtol ||s|| and sets T_half += theta dT
 * (theta = min(1, 1.5 / cell optical thickness)). Solver: CG preconditioned by one
 * aggregation-multigrid V-cycle in FP32, one thread-block cluster per instance. For
 * cg_rtol >= 1e-5 (the default 1e-3) the CG iterates are FP32 inside FP64 iterative
 * refinement: the solution is accumulated in FP64 and its residual s - A dT is formed and
 * measured in FP64, which is what cg_rtol bounds; below 1e-5 the CG iterates and residual
 * are FP64. Synchronises the stream to read the CG status; *cg_iters_out (may be NULL) gets
 * the largest iteration count over instances. ENOCONV if cg_maxit is reached. */
iugkp_status iugkp_newton_step(iugkp_ctx *ctx, const double *T_n_dev, double *T_half_inout_dev,
                               const double *R_dev, void *cuda_stream, int *cg_iters_out);

/* Statistical averaging after convergence (Sec. 4.4-4.5: the paper adds 100-1500 steps whose
 * results are averaged to reduce the statistical noise). Runs n_steps (>= 1) further
 * iterations from T_inout_dev, each with fresh draws (epoch = epoch_first + step) and the
 * update of iugkp_solve_steady (sweep, macro update, Newton correction when
 * options.newton), and accumulates on the device in FP64 the running mean and, by
 * Welford's update, the sample variance (n - 1 in the denominator; 0 for one step) of the
 * iterates, and the mean net power through every face.
 *   T_inout_dev  device FP64 [total_cells]: start on entry, last iterate on return
 *   T_mean_dev   device FP64 [total_cells] (required)
 *   T_var_dev    device FP64 [total_cells] or NULL
 *   F_mean_dev   device FP64 [total_faces] or NULL (face layout of iugkp_sweep)
 * Successive iterates are correlated: the variance is of the iterates, not of their mean.
 * Enqueued on cuda_stream; synchronises once at the end for the device error check
 * (IUGKP_ENOCONV if a correction solve hit cg_maxit). EINVAL for NULL T or mean, n_steps < 1. */
iugkp_status iugkp_average(iugkp_ctx *ctx, double *T_inout_dev, int n_steps, unsigned epoch_first,
                           double *T_mean_dev, double *T_var_dev, double *F_mean_dev, void *cuda_stream);

/* Persistent null-collision population (Sec. 3.2 steps (1)-(6)): the paper's own form of the
 * variable-tau iteration, next to the stateless sweep of iugkp_sweep. A fixed population
 * (per band, N_b slots per cell numbered q * ncells + cell, then N_w,b per boundary face
 * numbered q * faces + face) makes one candidate
 * flight per iteration. A particle whose flight ended in a real collision (or at a wall) is
 * re-emitted next iteration from that cell (or boundary face) with the home's power shared
 * by the particles that ended there: w = (C_b T_emit V / tau_b) / N in a cell, T_emit = T +
 * Q/m, and (C_b v_b T_face A / 4) / N on a face; a null candidate keeps position, direction
 * and weight. FP64 throughout; state in structure-of-arrays form (7 doubles and 3 ints per
 * slot, allocated by the reset). Draws of slot k (within its instance) in iteration it:
 * Philox counter (block, k, 0x80000000, band << 24 | it), key (seed, seed_hi ^ instance id).
 * iugkp_persistent_reset: (re)builds the population, every slot due for emission from its
 * home and every home counted with its own slots; synchronises cuda_stream.
 * iugkp_persistent_step: one iteration with the macro temperature T_dev (device FP64
 * [total_cells]); writes R_dev (real collisions, required), W_dev (w tau_maj of every
 * candidate), wall_dev (absorbed per wall) and counters_dev {flights, candidates, real, 0,
 * wall exits, 0} (each may be NULL) in the layouts of iugkp_sweep, and *slots_out (may be
 * NULL); enqueued on cuda_stream without synchronising. The macro update and the Newton
 * step are the caller's (iugkp_macro, iugkp_newton_step). EINVAL before a reset. */
iugkp_status iugkp_persistent_reset(iugkp_ctx *ctx, void *cuda_stream);
iugkp_status iugkp_persistent_step(iugkp_ctx *ctx, const double *T_dev, unsigned iteration, double *R_dev,
                                   double *W_dev, double *wall_dev, unsigned long long *counters_dev,
                                   long long *slots_out, void *cuda_stream);

/* Tuning of the staged sweep (no counterpart in the paper; refill, claim size and walk
 * length change speed, not results; the tally mode changes results by rounding only).
 * iugkp_autotune times full sweeps from T_dev (device FP64 [total_cells]) on the caller's
 * stream with CUDA events, searches refill_lanes in {auto, 4, 8, 16, 24}, warp_grab in
 * {128, 256, 512}, walk_k in {8, 16, 32} and, if allow_k32, tally in {STAGED, STAGED_K32}
 * one at a time, stores the fastest in the context's options and reports them in *out
 * (may be NULL). Synchronises the stream. The context must use FP32 tracking with a staged
 * tally mode (EINVAL otherwise). */
typedef struct {
  int refill_lanes, warp_grab, walk_k, tally;
  double sweep_ms;      /* best sweep time found */
  double baseline_ms;   /* sweep time with the options the context had on entry */
} iugkp_tuning;
iugkp_status iugkp_autotune(iugkp_ctx *ctx, const double *T_dev, unsigned epoch, int allow_k32,
                            iugkp_tuning *out, void *cuda_stream);

/* Convergence measure of one iteration (residual definition used by the steady driver):
 * out_dev[0] = sum_i (T1_i - T0_i)^2 and out_dev[1] = sum_i T1_i^2 over all cells of all
 * instances, in a fixed reduction order (deterministic). Asynchronous. */
iugkp_status iugkp_residual(iugkp_ctx *ctx, const double *T0_dev, const double *T1_dev, double *out_dev,
                            void *cuda_stream);

/* FP32 walk and its FP64 replay (no counterpart in the paper: a precision choice). With FP32
 * tracking and a staged tally mode, every decision of a particle's walk (the cell of each
 * candidate, i.e. the faces crossed before it along each axis; whether the first wall comes
 * before it; acceptance with probability tau_maj / tau) is taken in FP32 only when the FP32
 * value lies farther from the decision's boundary than a bound on its difference from the
 * FP64 walk's value. Otherwise the particle is left untallied at that point and, after the
 * sweep, the FP64 walk (the arithmetic of IUGKP_TRACK_FP64) replays it and makes its remaining
 * tallies. Real collisions, wall exits and event counts are therefore those of the FP64 walk;
 * the W tally of a null candidate near a face may sit in the neighbouring cell, and face
 * tallies near a cell corner may swap between two adjacent faces (a few particle weights).
 * iugkp_replayed: the number of particles the FP64 walk replayed in the context's last staged
 *   sweep or adjoint re-trace; synchronises cuda_stream.
 * iugkp_check_fp32_walk: measures on the current device, over every uniform the walk can draw,
 *   the accuracy of the FP32 operations the bound relies on, and writes
 *   out6[0] the largest error of the fast logarithm as a fraction of its allowance (<= 1);
 *   out6[1..4] the largest relative errors, in units of 2^-23, of sincospif, of
 *   sqrtf(1 - mu^2), of sqrtf(u) and sqrtf(1 - u), and of the fast division;
 *   out6[5] the relative bound those imply for the face-count decision, as a fraction of
 *   the one the walk uses (<= 1). Synchronous; errors in iugkp_last_error(NULL). */
iugkp_status iugkp_replayed(iugkp_ctx *ctx, long long *n_out, void *cuda_stream);
iugkp_status iugkp_check_fp32_walk(double *out6);

/* Measurement aid (no counterpart in the paper): the rate of FP64 atomic additions to
 * scattered addresses of an 8 MB (L2-resident) array on the current device, the access
 * pattern of the deposit tallies, in additions per second (best of a warm-up and five
 * timed launches). Allocates and frees its own buffer; synchronous; errors in
 * iugkp_last_error(NULL). */
iugkp_status iugkp_measure_atomics(double *ops_per_s);

/* Steady driver: from the initial T_inout_dev, repeats sweep -> macro -> [Newton]
 * until res = ||T^{n+1} - T^n|| / max(||T^{n+1}||, dT_ref sqrt(ncells)) <= tol over
 * all instances (dT_ref = the wall-temperature span, or max |T_w|, or 1).
 * Writes the final iterate to T_inout_dev; *iters_out, *res_out may be NULL.
 * ENOCONV if max_iter is reached first. */
iugkp_status iugkp_solve_steady(iugkp_ctx *ctx, double *T_inout_dev, double tol, int max_iter,
                                int *iters_out, double *res_out, void *cuda_stream);

/* Adjoint of the frozen-draw steady state (the sweep is linear, Sec. 2 Eq. "sum-g"):
 * with J = sum_i g_i T*_i, solves lambda = A^T lambda + g by re-tracing every
 * particle of epoch epoch0 and gathering lambda at its real-collision cell, with the
 * transposed diffusion correction, to tolerance tol. Outputs:
 *   grad_source_dev [total_cells] dJ/dQ_i (Q = source power density);
 *   grad_wall_dev   [total_walls] dJ/dT_w;
 *   lambda_dev      [total_cells] the adjoint solution (may be NULL).
 * T_star_dev is accepted for interface symmetry and unused (the problem is linear). */
iugkp_status iugkp_adjoint(iugkp_ctx *ctx, const double *T_star_dev, const double *g_dev,
                           double tol, int max_iter, double *grad_source_dev,
                           double *grad_wall_dev, double *lambda_dev, void *cuda_stream);

/* ---------------------------------------------------------------------------------
 * Allocation-free correction solve. The paper has no counterpart; this exists for
 * callers that cannot call cudaMalloc: code whose device memory is owned entirely by
 * another allocator (a framework's caching pool that has already reserved the GPU), or
 * a latency-critical loop that cannot afford the device synchronisation an allocation
 * may cause. The contexts above allocate their buffers in iugkp_create; this function
 * needs no context and allocates nothing.
 *
 * Solves -div(kappa grad x) = rhs on one uniform grid g (the finite-volume operator of
 * iugkp_newton_step: harmonic face kappa, vacuum wall condition with outward flux
 * wall_cv / 2 times the wall value in series with half a cell of conduction) by
 * Jacobi-preconditioned CG in FP64 to ||r|| <= rtol ||rhs||, starting from x = 0.
 *   kappa_dev [cells] conductivity (> 0), rhs_dev [cells], x_dev [cells] output;
 *   wall_cv   sum over bands of C_b v_b (> 0); *iters_out (may be NULL) gets the count.
 * Scratch (stencil, CG vectors) lives in one static device array sized for
 * IUGKP_NOALLOC_MAX_CELLS cells, kept by every GPU that loads the library until the
 * process exits. Larger grids return IUGKP_EINVAL. Every call reuses that array, so
 * calls whose work overlaps on the GPU (two streams, two host threads) race. The first
 * call on a device looks the array's address up once with that device current; make
 * that first call before any stream capture. Every call synchronises cuda_stream to read
 * the iteration count back. IUGKP_ENOCONV if maxit is reached; IUGKP_EINVAL (x_dev then
 * holds no solution) if some kappa is not positive and finite, or if a non-finite value
 * arises from rhs_dev. Errors: iugkp_last_error(NULL). */
#define IUGKP_NOALLOC_MAX_CELLS 65536
iugkp_status iugkp_diffusion_solve_noalloc(const iugkp_grid *g, const double *kappa_dev, double wall_cv,
                                           const double *rhs_dev, double *x_dev, double rtol, int maxit,
                                           int *iters_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* IUGKP_H */
