// Batched real GEMM on the CUDA cores (FP64 and FP32 walker paths).
//
//   C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b],   b = 0 .. batch-1
//
// op(A) is A (row-major, m x k, leading dimension lda) or, with TA, the
// transpose of a row-major k x m matrix; the same for B. 64 x 64 output tile
// per 256-thread block, 4 x 4 outputs per thread, K staged through shared
// memory in slabs of 16. Used by the force-bias, one-body-operator,
// B_half and exchange-energy contractions when the step runs on the SIMT
// path, and by the one-time setup in every precision.
#include "kernels.h"

namespace afqmc {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(NT)
gemm_kernel(int m, int n, int k, T alpha, const T* __restrict__ A, long lda,
            long sA, const T* __restrict__ B, long ldb, long sB, T beta,
            T* __restrict__ C, long ldc, long sC) {
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int bz = blockIdx.z;
  A += bz * sA;
  B += bz * sB;
  C += bz * sC;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int idx = tid + r * NT;
      int mm, kk;
      if (TA) { mm = idx % BM; kk = idx / BM; }
      else    { kk = idx % BK; mm = idx / BK; }
      int gm = m0 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < m && gk < k) v = TA ? A[(long)gk * lda + gm] : A[(long)gm * lda + gk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int idx = tid + r * NT;
      int nn, kk;
      if (TB) { kk = idx % BK; nn = idx / BK; }
      else    { nn = idx % BN; kk = idx / BN; }
      int gn = n0 + nn, gk = k0 + kk;
      T v = T(0);
      if (gn < n && gk < k) v = TB ? B[(long)gn * ldb + gk] : B[(long)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty * 4 + i;
    if (gm >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx * 4 + j;
      if (gn >= n) continue;
      T* c = C + (long)gm * ldc + gn;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v += beta * *c;
      *c = v;
    }
  }
}
}  // namespace

template <typename T>
cudaError_t gemm(cudaStream_t st, bool ta, bool tb, int m, int n, int k, T alpha,
                 const T* A, long lda, long sA, const T* B, long ldb, long sB,
                 T beta, T* C, long ldc, long sC, int batch) {
  if (m <= 0 || n <= 0 || batch <= 0) return cudaSuccess;
  dim3 grid((n + BN - 1) / BN, (m + BM - 1) / BM, batch);
  if (grid.y > 65535 || grid.z > 65535) return cudaErrorInvalidConfiguration;
  if (!ta && !tb)
    gemm_kernel<T, false, false><<<grid, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  else if (!ta && tb)
    gemm_kernel<T, false, true><<<grid, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  else if (ta && !tb)
    gemm_kernel<T, true, false><<<grid, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  else
    gemm_kernel<T, true, true><<<grid, NT, 0, st>>>(m, n, k, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC);
  return cudaGetLastError();
}

template cudaError_t gemm<float>(cudaStream_t, bool, bool, int, int, int, float,
                                 const float*, long, long, const float*, long,
                                 long, float, float*, long, long, int);
template cudaError_t gemm<double>(cudaStream_t, bool, bool, int, int, int, double,
                                  const double*, long, long, const double*, long,
                                  long, double, double*, long, long, int);

}  // namespace afqmc
