// Multigrid hierarchy descriptor of one instance (device-resident), shared by the host
// set-up (mg_setup.cu) and the cluster PCG kernel (mgpcg.cu).
#pragma once

namespace iugkp {

constexpr int MG_MAXL = 16;
constexpr int MG_COARSE_MAX = 32;  // cells on the coarsest level (dense inverse)
constexpr int FD_MAX_N = 1024;     // largest axis size solved by fast diagonalization

struct InstMG {
  int levels;
  int dim;
  // Separable operator (1D, or 2D with uniform kappa): A = Tx (x) I + I (x) Ty with
  // Tx = Qx diag(lx) Qx^T and Ty = Qy diag(ly) Qy^T; solved by fast diagonalization
  // (mgpcg.cu) instead of the multigrid PCG when direct != 0.
  int direct;               // 0: multigrid PCG; 1: fast diagonalization; 2: the same in shared memory
  int fnx, fny;            // sizes of Tx and Ty (fny = 1 in 1D)
  long long qx_off, qy_off;  // offsets of Qx, Qy (row-major, eigenvectors in columns) in the FP32 array
  long long lx_off, ly_off;  // offsets of the eigenvalues in the FP32 array
  int n[MG_MAXL][3];
  long long nc[MG_MAXL];
  long long off[MG_MAXL];  // offset of each level in the FP32 level arrays
  long long cinv_off;      // offset of the coarsest dense inverse
  long long cell_off;      // offset of the fine level in the per-cell arrays
};

}  // namespace iugkp
