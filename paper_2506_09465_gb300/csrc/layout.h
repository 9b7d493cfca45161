// Plain-data descriptors shared by host and device code of the CUDA library.
#pragma once

#include <cstdint>

namespace iugkp {

// One instance (geometry and offsets into the concatenated arrays). Device-resident.
struct InstDesc {
  int dim;
  int n[3];           // cells per axis (unused axes: 1)
  int ncells;
  int pad0;
  double h[3];        // cell size per axis (unused axes: 1)
  double V;           // cell volume (per unit area / depth in 1D / 2D)
  long long cell_off; // offset into per-cell arrays
  long long bc_off;   // offset into [band][cell] arrays (= nb * cell_off)
  long long face_off; // offset into per-face arrays
  long long fax_off[3];  // start of each axis's faces within the instance
  long long nfaces;
  int wall_off;       // offset into per-wall arrays (= 2 * dim * k)
  uint32_t inst_id;   // Philox instance id
  float hf[3];        // cell size per axis in FP32 (the FP32 walk)
  int refill;         // staged sweep: refill a warp's lanes once this many are idle
  long long bface_off;   // offset into per-boundary-face arrays
  int wface_off[6];      // start of each wall's faces within the instance (faces of wall
                         // a run over axes (a+1)%3, (a+2)%3, the first fastest)
};

// A run of emitters sharing (instance, band, kind). kind 0 = the instance's cells;
// kind 1 + w = the boundary faces of wall w. Particles of the run are numbered
// emitter-major: local = e * per_emitter + q.
// The staged sweep visits them q-major in the order perm[perm_off + r], r = 0 .. n_emitters-1,
// of emitter ranks (emitters sorted by their cell's majorant ratio class, so that the lanes of
// a warp walk candidate chains of similar length); perm_off = -1: emitter order.
struct Group {
  long long first_particle;
  int inst, band, kind;
  int n_emitters;
  int per_emitter;
  int perm_off;
};

// Counter slots (u64) written by a sweep.
enum { CNT_FLIGHTS = 0, CNT_CANDIDATES, CNT_REAL, CNT_CROSSINGS, CNT_WALL_EXITS, CNT_DROPPED, CNT_N };

// Device error bits.
enum { ERR_BUDGET = 1, ERR_RANGE = 2, ERR_PCG = 4, ERR_WAIT = 8, ERR_DEFER = 16 };

}  // namespace iugkp
