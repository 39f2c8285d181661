// Tensor-core (tcgen05 + TMA) kernels for the dense contractions of the
// TF32 modes.
#pragma once

#include <cuda_runtime.h>

namespace afqmc {

struct TcCtx;

cudaError_t tc_create(TcCtx** out);
void tc_destroy(TcCtx* t);

// C[m][n] (row stride ldc) = alpha * sum_k A[m][k] B[n][k] + beta * R[m][n].
// A and B are row-major fp32 (K contiguous) with lda, ldb multiples of 4 and
// 16-byte-aligned bases. split3: three TF32 products (hi*hi + hi*lo + lo*hi)
// instead of one. ksplit > 1 splits K into that many ranges and writes
// partial sums to C + s * split_stride (beta must then be 0). bn is the
// output tile width (64 or 128; 0 picks 64 for n <= 64, else 128). A
// device-side wait that times out sets bit 4 of *status.
// With split3 and Blo, B already holds hi = B rounded to TF32 and Blo the
// remainder (see tc_split), so only A is split on the fly. With Clo (ksplit
// 1), the result leaves split the same way: C receives its TF32 hi part and
// Clo (same layout) the remainder. With out_bf16 (Clo set, no R), C and Clo
// are BF16 arrays (row stride ldc elements) receiving the result's BF16 hi
// part and the BF16-rounded remainder.
cudaError_t tc_gemm(TcCtx* t, cudaStream_t st, int m, int n, int k, const float* A,
                    long lda, const float* B, long ldb, float* C, long ldc, float alpha,
                    float beta, const float* R, long ldr, bool split3, int ksplit,
                    long split_stride, int* status, int bn = 0, const float* Blo = nullptr,
                    float* Clo = nullptr, bool out_bf16 = false);

// Self-test of the bounded wait: a kernel waits on an mbarrier nothing
// completes, gives up after limit_cycles and sets bit 4 of *status.
cudaError_t tc_wait_timeout_probe(cudaStream_t st, long long limit_cycles, int* status);

// BF16 hi and lo parts (hi = x rounded, lo = x - hi rounded) of n FP64 values.
cudaError_t tc_split_bf16(cudaStream_t st, long n, const double* x, void* hi, void* lo);

// x <- x rounded to TF32, lo <- the remainder x - hi rounded to TF32, n floats.
cudaError_t tc_split(cudaStream_t st, long n, float* x, float* lo);

// Taylor propagation of W walkers (M <= 64): Pout = sum_{n<=order} V^n Pin / n!
// with V [W][2][M][M] and Pin, Pout [W][N][2][M], on the tensor cores. With a
// half-step image (see tc_bhalf_image) the two half-step factors are applied
// around the series: Pout = B_half exp_T(V) B_half Pin. Pout may be Pin:
// each CTA reads a walker's column chunk completely before writing it, and
// no other CTA touches that chunk. bf16: BF16 hi + lo operands (three
// kind::f16 products per term) instead of TF32 (split3: hi + lo).
cudaError_t tc_taylor(TcCtx* t, cudaStream_t st, int W, int M, int N, int order,
                      const float* V, const float* Pin, float* Pout, const void* bhalf_img,
                      bool split3, bool bf16, int* status);

// Operand image of (B_half - I) (M x M, row-major fp32 in dB) for tc_taylor,
// tc_bhalf_image_bytes(split3, bf16) bytes, 16-byte aligned.
size_t tc_bhalf_image_bytes(bool split3, bool bf16);
cudaError_t tc_bhalf_image(cudaStream_t st, int M, const float* dB, void* img, bool split3,
                           bool bf16);

// B_half exp_T(V) B_half for 64 < M <= 256 (any M <= 256 works), W walkers,
// Pin -> Pout ([W][N][2][M], Pout may be Pin), on the tensor cores with the
// operator streamed from global memory: V [W][2][M][ldV] and dB = B_half - I
// [M][ldV] (ldV >= M, rows 16-byte aligned). TF32X3 (split3): V and dB (FP32)
// hold the TF32 hi parts and Vlo, dBlo the remainders. BF16X3 (bf16): the
// four operands are BF16 arrays of hi and lo parts. A device-side wait that
// times out sets bit 4 of *status.
cudaError_t tc_taylor_wide(TcCtx* t, cudaStream_t st, int W, int M, int N, int order, long ldV,
                           const void* V, const void* Vlo, const void* dB, const void* dBlo,
                           const float* Pin, float* Pout, bool split3, bool bf16, int* status);


}  // namespace afqmc
