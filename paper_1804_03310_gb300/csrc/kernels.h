// Launchers of the library's kernels. All take the stream first, return the
// launch error, and read/write device memory only.
//
// Walker layouts (T = double on the FP64 path, float otherwise):
//   Phi    [W][N][2][M]   column j of walker w (j < n_up: spin up), re plane
//                         then im plane, M basis coefficients each
//   Theta  [W][2][ldt]    Theta = Phi (D^H Phi)^-1, re row then im row; each
//                         row holds the up block (n_up*M, column a at a*M)
//                         at 0 and the down block at dn_off, both 16-byte
//                         aligned, zeros in the padding
//   V      [W][2][M][ldV] one-body operator per walker (complex symmetric),
//                         rows padded to ldV >= M
//   X      [nsplit][W][2][ldx]  force-bias contraction partial sums, ldx =
//                         n_chol + 1 (last column: tr(h~ Theta))
//   S      [W][2][ldS]    i sqrt(dt) (x - xbar) per walker, ldS = n_chol
//                         rounded up to a multiple of 4
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace afqmc {

// Opt a kernel in to the largest dynamic shared memory the current device
// allows beside the kernel's static shared memory, and return that limit in
// bytes. The attribute belongs to the device, so the opt-in runs once per
// (kernel, device) pair and is cached; query errors are cleared so they
// cannot surface at a later launch check.
size_t smem_optin(const void* kernel);

template <typename T>
cudaError_t gemm(cudaStream_t st, bool ta, bool tb, int m, int n, int k, T alpha,
                 const T* A, long lda, long sA, const T* B, long ldb, long sB,
                 T beta, T* C, long ldc, long sC, int batch);

// Step counters live in device memory, ctr[0] = completed steps and
// ctr[1] = recorded measurements, so that a block of steps can be captured
// once as a CUDA graph and replayed: the kernels read the step from there.

// K1 + K3: Philox fields, capped force bias, shifted fields and the log of
// the importance factor sum_g (x xbar - xbar^2/2) per walker, at step
// ctr[0]. X holds `nsplit` partial sums (split_stride elements apart) that
// are added in order. With lbar [n_chol] (FP64, else NULL) the mean field is
// subtracted from X before the bias is formed, and lmf[w] receives
// -i sqrt(dt) sum_g (x_g - xbar_g) lbar_g.
template <typename T>
cudaError_t launch_fields(cudaStream_t st, int W, int n_chol, const T* X, long ldx,
                          int nsplit, long split_stride, double sqdt, double cap,
                          uint64_t seed, int run_id, const long long* ctr, T* S, long ldS,
                          T* xbar, double2* lw, const double* lbar, double2* lmf);

// K5 on the CUDA cores: Phi_out = sum_{n<=order} V^n Phi_in / n!, with V
// [W][2][M][ldv].
template <typename T>
cudaError_t launch_taylor(cudaStream_t st, int W, int M, int N, int order,
                          const T* V, long ldv, const T* Phi_in, T* Phi_out);

// K6: A = D^H Phi per spin, inverse by elimination with partial pivoting
// (FP64 arithmetic when fp64_compute, else FP32), ln det A accumulated in
// FP64, Theta = Phi A^-1. PsiT [N][M] holds the reference determinant's
// orbitals as rows (up orbitals then down orbitals). Ainv (optional)
// [W][2][nmax][nmax] double2 receives A^-1 per spin.
template <typename T>
cudaError_t launch_overlap(cudaStream_t st, int W, int M, int n_up, int n_dn,
                           const T* Phi, const T* PsiT, T* Theta, long ldt, long dn_off,
                           double2* logdet, double2* Ainv, bool fp64_compute);

// K7: weight and phaseless cut from the new log-overlap (logO_new, or
// with logO_new NULL the sum of the two spins' log-determinants in
// logdet [W][2]) plus the mean-field scalar lmf (NULL: none); hybrid form
// from the importance log lw, or, with eloc non-NULL, the local-energy form
// from the pre-move local energies. Ends the step (ctr[0] += 1). With
// cap > 0 a weight is capped at cap * (*wref) when *wref > 0.
cudaError_t launch_weights(cudaStream_t st, int W, const double2* logO_new,
                           const double2* logdet, const double2* lw, const double2* lmf,
                           const double2* eloc, double dtau, double e_shift, double cap,
                           const double* wref, double* weight, double2* logO,
                           long long* ctr);

// Sum of the two spins' log-determinants (single-determinant overlap).
cudaError_t launch_logdet_sum(cudaStream_t st, int W, const double2* logdet,
                              double2* out);

// K10: QR orthonormalisation per walker and spin, Phi <- Q with R's
// diagonal real and positive (FP64 arithmetic when fp64_compute, else FP32);
// logO -= ln det R accumulated in FP64. lr [W][2] is scratch.
template <typename T>
cudaError_t launch_qr(cudaStream_t st, int W, int M, int n_up, int n_dn, T* Phi,
                      double2* logO, double* lr, bool fp64_compute);
size_t overlap_smem(int M, int nmax, size_t csize);

// K9 epilogue: E_L = E1 + 1/2 sum X^2 + sum_sigma 1/2 theta^T Yx theta, with
// X split as for launch_fields and Z^sigma = Theta^sigma Yx^sigma per spin
// ([2W][ldz] each, up block first).
template <typename T>
cudaError_t launch_energy_reduce(cudaStream_t st, int W, int M, int n_up, int n_dn,
                                 int n_chol, const T* X, long ldx, int nsplit,
                                 long split_stride, const T* Theta, long ldt, long dn_off,
                                 const T* Z, long ldz_up, long ldz_dn, double2* eloc);

// Weighted mixed estimate sum W Re E / sum W (walkers with W > 0) into
// out[0] and the weight sum into out[1]; with hist, also recorded as
// hist[ctr[1] % hist_len] = (ctr[0], value) and ctr[1] += 1.
cudaError_t launch_mixed_energy(cudaStream_t st, int W, const double* weight,
                                const double2* eloc, long long* ctr, double2* hist,
                                int hist_len, double* out);

// K11: blocked FP64 prefix sum and comb; parent[j] per new walker, the new
// common weight in *wnew; on zero total weight sets bit 1 of *status and
// leaves parent = identity. The comb's uniform is drawn at step ctr[0], or
// at `step` when ctr is NULL.
cudaError_t launch_comb(cudaStream_t st, int W, const double* weight, uint64_t seed,
                        int run_id, const long long* ctr, long step, int* parent,
                        double* scratch, double* wnew, int* status);

// Walker copies after the comb. When the comb succeeded (*wnew = S/n > 0)
// every weight becomes 1, *wref 1, and ln(S/n) is added to *log_scale.
template <typename T>
cudaError_t launch_gather(cudaStream_t st, int W, long phi_elems, long theta_elems,
                          const int* parent, const T* Phi, T* Phi_out,
                          const T* Theta, T* Theta_out, const double2* logO,
                          double2* logO_out, const double* wnew, double* weight,
                          double* wref, double* log_scale);

// Row copies out[j] = in[parent[j]] ([W][elems]).
template <typename T>
cudaError_t launch_gather_rows(cudaStream_t st, int W, long elems, const int* parent,
                               const T* in, T* out);

// Block-diagonal Cholesky vectors. Setup: packed operands Lp [n_chol][nnz]
// and (LpT non-NULL) LpT [nnzp][ldS] from the FP64 L [n_chol][M*M], gidx
// [nnz] holding the i*M+j of each packed entry. Step: the Taylor series of
// the packed V [W][2][nnzp] applied to Pin [W][N][2][M] into Pout, blk
// holding the M int4 {row offset, block size, member base, 0}, M int4 slots
// of which the first nb are the blocks' {first row offset, size, member
// base, 0}, then the M member indices; maxb the largest block.
cudaError_t launch_pack_blocks(cudaStream_t st, int G, long nnz, long nnzp, long ldS, int M,
                               const double* L, const int* gidx, double* Lp, double* LpT);
template <typename T>
cudaError_t launch_taylor_blocks(cudaStream_t st, int W, int M, int N, int order, long nnzp,
                                 int nb, int maxb, const T* V, const void* blk, const T* Pin,
                                 T* Pout);

// Setup helpers (FP64).
cudaError_t launch_h1_remainder(cudaStream_t st, int M, int n_chol, const double* h1,
                                const double* L, const double* lbar, double* h1p);
cudaError_t launch_scale_identity(cudaStream_t st, int M, const double* A, double s,
                                  double* out_I_plus, double* out_scaled);
cudaError_t launch_yx_permute(cudaStream_t st, int n, int M, const double* gram,
                              double* yx, long ldy);
cudaError_t launch_pad_rows(cudaStream_t st, long rows, long Jup, long Jdn,
                            const double* in, double* out, long ld, long dn_off);
cudaError_t launch_transpose(cudaStream_t st, long rows, long cols, const double* in,
                             double* out, long ldo);
// FP64 matrix-vector products: y = A x (rows of A) and y = x^T A (columns).
cudaError_t launch_gemv_rows(cudaStream_t st, long rows, long cols, const double* A, long lda,
                             const double* x, double* y);
cudaError_t launch_gemv_cols(cudaStream_t st, long rows, long cols, const double* A, long lda,
                             const double* x, double* y);
// L [G][M*M] -> out [M*ldv][ldo], out[i ldv + k][g] = L[g][i M + k] (other
// rows untouched).
cudaError_t launch_transpose_pad(cudaStream_t st, long G, int M, long ldv, const double* in,
                                 double* out, long ldo);
template <typename T>
cudaError_t launch_convert(cudaStream_t st, long n, const double* in, T* out);
template <typename T>
cudaError_t launch_init_walkers(cudaStream_t st, int W, int M, int N, const T* PsiT,
                                T* Phi, double* weight);
cudaError_t launch_axpy_d(cudaStream_t st, long n, double a, const double* x,
                          double* y);
cudaError_t launch_add_diag(cudaStream_t st, int M, double* A, double a);

}  // namespace afqmc
