// Multi-determinant trials (Sherman-Morrison-Woodbury updates, Sec. III).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace afqmc {

constexpr int MD_EMAX = 4;               // excitations per spin and determinant
constexpr int MD_MAX_DET_PER_THREAD = 8; // energy kernel: determinants per thread

// One determinant relative to the reference, per spin: E holes at reference
// positions h[0..E) filled in place by active orbitals p[0..E).
struct MdDet {
  int E[2];
  int h[2][MD_EMAX];
  int p[2][MD_EMAX];
  int coff;   // start of this determinant's C rows in the C table (complex values):
              // E[0] rows of n_up for the up spin, then E[1] rows of n_dn
};

struct MdTables {
  int ndet;
  int nact[2];              // active orbitals per spin
  int ctot;                 // complex values in the C table: sum_i E_i^up n_up + E_i^dn n_dn
  const MdDet* dets;        // [ndet], device
  const double2* cconj;     // [ndet] c_i^* (sign of the column order folded in), device
  const int* ract[2];       // [ns] active index of the reference orbital at each position
  const void* CactT[2];     // [nact][M] active orbitals as rows (walker element type)
};

size_t md_step_smem(int M, int nu, int nd, int na_u, int na_d, int ndet, bool f64);
size_t md_energy_smem(int M, int nu, int nd, int na_u, int na_d, int ndet, bool f64);

// Ratios, ln O_T, and Gamma = Theta_0 Lambda per walker (after the overlap
// kernel has produced Theta_0 and the reference log-determinants).
template <typename T>
cudaError_t launch_md_step(cudaStream_t st, const MdTables& tb, int W, int M, int nu, int nd,
                           const T* Theta, long ldt, long dn_off, const double2* logdet0,
                           double2* logO_new, T* Gamma, long ldg, long gdn_off, bool f64);

// Local energy sum_i w_i E_i per walker; LtilA [(G+1)][ldg] holds the
// active orbitals' rotated Cholesky vectors C_act^T L_g and, as row G, C_act^T h1.
template <typename T>
cudaError_t launch_md_energy(cudaStream_t st, const MdTables& tb, int W, int M, int nu, int nd,
                             int G, const T* Theta, long ldt, long dn_off,
                             const double2* logdet0, const T* LtilA, long ldg, long gdn_off,
                             double2* eloc, bool f64);

}  // namespace afqmc
