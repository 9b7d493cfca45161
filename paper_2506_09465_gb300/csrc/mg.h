// Multigrid hierarchy descriptor of one instance (device-resident), shared by the host
// set-up (mg_setup.cu) and the cluster PCG kernel (mgpcg.cu).
#pragma once

namespace iugkp {

constexpr int MG_MAXL = 16;
constexpr int MG_COARSE_MAX = 32;  // cells on the coarsest level (dense inverse)

struct InstMG {
  int levels;
  int dim;
  int n[MG_MAXL][3];
  long long nc[MG_MAXL];
  long long off[MG_MAXL];  // offset of each level in the FP32 level arrays
  long long cinv_off;      // offset of the coarsest dense inverse
  long long cell_off;      // offset of the fine level in the per-cell arrays
};

}  // namespace iugkp
