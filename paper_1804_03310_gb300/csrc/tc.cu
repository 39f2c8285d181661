// Tensor-core kernels (tcgen05 MMA, TMEM accumulators, TMA operand loads)
// for the dense contractions of the walker step in the TF32 modes:
//
//  * tc_gemm_kernel: C = alpha A B^T + beta R with both operands K-major,
//    128 x BN output tiles, a multi-stage TMA -> MMA pipeline and one
//    accumulator tile in TMEM. Used for the force bias (Theta . L~^T, Sec. II),
//    the one-body operator (S . L, Eq. 3), the exchange-energy contraction
//    (Theta . Yx, Eq. 5) and the half-step propagator (Phi + Phi (B_half - I)).
//  * tc_taylor_kernel: per walker, the Taylor series of exp(V) applied to
//    the orbitals (Sec. II, Thouless propagation by matrix products), with V
//    held on-chip as the real 2M x 2M form [[Vr, -Vi], [Vi, Vr]] and each term
//    t_n = V t_{n-1} / n fed back from TMEM into shared memory.
//
// TF32X3 mode splits each operand x into hi = x rounded to TF32 and
// lo = (x - hi) rounded to TF32, and accumulates hi.hi + hi.lo + lo.hi. The
// remainder is rounded explicitly: fed to the tensor core unrounded, its low
// bits would be truncated, an error of up to 2^-21 |x| of one sign that
// accumulates coherently over long contractions; rounded, x - hi - lo is at
// most 2^-22 |x| and unbiased.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.h"
#include "tc.h"
#include "umma.cuh"

namespace afqmc {

using namespace umma;

struct TcCtx {
  PFN_cuTensorMapEncodeTiled_v12000 encode;
  int num_sms;
};

namespace {

constexpr int BM = 128, BK = 32;
// K tiles (of BK values) the tensor core accumulates before the epilogue
// drains the accumulator into FP32 registers.
constexpr int kGemmChunkTiles = 4;

// x rounded to the nearest TF32 value (10 explicit mantissa bits, the 13
// low bits of the FP32 pattern cleared), so that x - tf32_hi(x) is exact in
// FP32 and at most 2^-11 |x|. One conversion instruction.
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// The second term of the split: (x - hi) rounded to TF32.
__device__ __forceinline__ float tf32_lo(float x, float hi) { return tf32_hi(x - hi); }

__device__ __forceinline__ void flag_timeout(int* status) {
  if (status) atomicOr(status, 4);
}

// ------------------------------------------------------------------ GEMM
// Persistent: each CTA walks work items (output tile, K range) i = blockIdx.x,
// blockIdx.x + gridDim.x, ...; the TMA -> MMA ring of stages runs on across
// items. Within an item the tensor core accumulates at most kc K tiles
// (kc * 32 values) into one TMEM accumulator; the epilogue drains each such
// chunk into FP32 registers (round-to-nearest adds) and stores the item
// after its last chunk. The tensor core's own accumulation rounds with a
// bias that grows with the number of accumulated products (measured: a
// relative error growing linearly with K, 2.3e-5 at K = 3600), which the
// chunking bounds. The accumulator alternates between two TMEM buffers, so
// the draining of one chunk overlaps the products of the next.
// Warps: 0 TMA producer, 1 MMA issuer, 2-5 epilogue (TMEM lane quadrant =
// warp % 4), 6-9 operand split (TF32X3 only).
template <int BN, bool SPLIT3>
struct GemmCfg {
  static constexpr int A_BYTES = BM * BK * 4;
  static constexpr int B_BYTES = BN * BK * 4;
  static constexpr int STAGE_BYTES = (A_BYTES + B_BYTES) * (SPLIT3 ? 2 : 1);
  static constexpr int STAGES = (196 * 1024) / STAGE_BYTES;
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static constexpr int THREADS = SPLIT3 ? 320 : 192;
};

struct GemmWork {
  int mt, nt, ktiles_total, ktiles_per_split, items, kc;
  __device__ void item(int i, int& m0, int& n0, int& z, int& kt0, int& nkt) const {
    const int tn = i % nt;
    const int rest = i / nt;
    const int tm = rest % mt;
    z = rest / mt;
    m0 = tm * BM;
    n0 = tn;            // scaled by BN by the caller
    kt0 = z * ktiles_per_split;
    nkt = max(0, min(ktiles_total, kt0 + ktiles_per_split) - kt0);
  }
};

template <int BN, bool SPLIT3, bool BLO>
__global__ void __launch_bounds__(GemmCfg<BN, SPLIT3>::THREADS, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
               const __grid_constant__ CUtensorMap mapB,
               const __grid_constant__ CUtensorMap mapBlo, int m, int n, GemmWork wk,
               float* __restrict__ C, long ldc, float alpha,
               float beta, const float* __restrict__ R, long ldr, long split_stride,
               int* status, float* __restrict__ Clo, int out_bf16) {
  using Cfg = GemmCfg<BN, SPLIT3>;
  constexpr int S = Cfg::STAGES;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  auto a_hi = [&](int s) { return base + s * Cfg::STAGE_BYTES; };
  auto b_hi = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES; };
  auto a_lo = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES + Cfg::B_BYTES; };
  auto b_lo = [&](int s) {
    return base + s * Cfg::STAGE_BYTES + 2 * Cfg::A_BYTES + Cfg::B_BYTES;
  };
  uint64_t* bars = (uint64_t*)(base + S * Cfg::STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* conv = bars + S;
  uint64_t* empty = bars + 2 * S;
  uint64_t* tfull = bars + 3 * S;       // [2] accumulator ready
  uint64_t* tempty = bars + 3 * S + 2;  // [2] accumulator drained
  uint32_t* tslot = (uint32_t*)(bars + 3 * S + 4);
  __shared__ int s_fail;
  volatile int* fail = &s_fail;       // read afresh: a timed-out role stops the others

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&conv[s]), 128);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&tfull[a]), 1);
      mbar_init(smem_u32(&tempty[a]), 4);
    }
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(tslot), 2 * BN);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int i = blockIdx.x; i < wk.items && !*fail; i += gridDim.x) {
        int m0, tn, z, kt0, nkt;
        wk.item(i, m0, tn, z, kt0, nkt);
        const int n0 = tn * BN;
        for (int k = 0; k < nkt; ++k, ++it) {
          const int s = it % S;
          const uint32_t ph = (uint32_t)(it / S) & 1u;
          if (it >= S && !mbar_wait(smem_u32(&empty[s]), ph ^ 1u)) {
            flag_timeout(status);
            *fail = 1;
            break;
          }
          mbar_arrive_expect_tx(smem_u32(&full[s]),
                                Cfg::A_BYTES + Cfg::B_BYTES * (BLO ? 2 : 1));
          tma_load_2d(smem_u32(a_hi(s)), &mapA, (kt0 + k) * BK, m0, smem_u32(&full[s]));
          tma_load_2d(smem_u32(b_hi(s)), &mapB, (kt0 + k) * BK, n0, smem_u32(&full[s]));
          if (BLO)   // the constant operand arrives already split (hi, lo)
            tma_load_2d(smem_u32(b_lo(s)), &mapBlo, (kt0 + k) * BK, n0, smem_u32(&full[s]));
        }
      }
      // no copy may outlive the CTA: the latest load into each stage has
      // landed before teardown (on the normal path these have long completed)
      for (int j = it - 1; j >= 0 && j >= it - S; --j)
        if (!mbar_wait(smem_u32(&full[j % S]), (uint32_t)(j / S) & 1u)) flag_timeout(status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = idesc_tf32(BM, BN);
      int it = 0, j = 0;                     // j counts accumulation chunks
      uint32_t last_bar = 0, last_par = 0;   // the latest commit, for the drain
      for (int i = blockIdx.x; i < wk.items && !*fail; i += gridDim.x) {
        int m0, tn, z, kt0, nkt;
        wk.item(i, m0, tn, z, kt0, nkt);
        const int nch = nkt > 0 ? (nkt + wk.kc - 1) / wk.kc : 1;
        for (int ch = 0; ch < nch && !*fail; ++ch, ++j) {
          const int acc = j & 1;
          const uint32_t aph = (uint32_t)(j >> 1) & 1u;
          if (j >= 2 && !mbar_wait(smem_u32(&tempty[acc]), aph ^ 1u)) {
            flag_timeout(status);
            *fail = 1;
            break;
          }
          fence_after_sync();
          const uint32_t td = tmem + (uint32_t)(acc * BN);
          const int k_lo = ch * wk.kc, k_hi = min(nkt, k_lo + wk.kc);
          for (int k = k_lo; k < k_hi; ++k, ++it) {
            const int s = it % S;
            const uint32_t ph = (uint32_t)(it / S) & 1u;
            if (!mbar_wait(smem_u32(SPLIT3 ? &conv[s] : &full[s]), ph)) {
              flag_timeout(status);
              *fail = 1;
              break;
            }
            fence_after_sync();
#pragma unroll
            for (int ks = 0; ks < BK / 8; ++ks) {
              const uint64_t ad = desc_sw128(smem_u32(a_hi(s)) + ks * 32);
              const uint64_t bd = desc_sw128(smem_u32(b_hi(s)) + ks * 32);
              mma_tf32(td, ad, bd, id, (k > k_lo || ks > 0) ? 1u : 0u);
              if (SPLIT3) {
                mma_tf32(td, ad, desc_sw128(smem_u32(b_lo(s)) + ks * 32), id, 1u);
                mma_tf32(td, desc_sw128(smem_u32(a_lo(s)) + ks * 32), bd, id, 1u);
              }
            }
            mma_commit(smem_u32(&empty[s]));
            last_bar = smem_u32(&empty[s]);
            last_par = ph;
          }
          if (*fail) break;
          mma_commit(smem_u32(&tfull[acc]));
          last_bar = smem_u32(&tfull[acc]);
          last_par = aph;
        }
      }
      // no MMA may outlive the TMEM allocation: a commit arrives once every
      // earlier MMA of this thread has completed
      if (last_bar && !mbar_wait(last_bar, last_par)) flag_timeout(status);
    }
  } else if (warp < 6) {
    // epilogue: TMEM lane quadrant q = warp % 4 holds rows 32q .. 32q + 31;
    // each chunk's accumulator is added into sum[] (FP32, round to nearest)
    const int q = warp & 3;
    int j = 0;
    float sum[BN];
    for (int i = blockIdx.x; i < wk.items && !*fail; i += gridDim.x) {
      int m0, tn, z, kt0, nkt;
      wk.item(i, m0, tn, z, kt0, nkt);
      const int n0 = tn * BN;
      const int nch = nkt > 0 ? (nkt + wk.kc - 1) / wk.kc : 1;
      bool ok = true;
      for (int ch = 0; ch < nch; ++ch, ++j) {
        const int acc = j & 1;
        const uint32_t aph = (uint32_t)(j >> 1) & 1u;
        if (!mbar_wait(smem_u32(&tfull[acc]), aph)) {
          flag_timeout(status);
          *fail = 1;
          ok = false;
          break;
        }
        fence_after_sync();
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * BN + c0), v);
#pragma unroll
          for (int jj = 0; jj < 32; ++jj) {
            const float x = nkt == 0 ? 0.f : v[jj];
            sum[c0 + jj] = ch == 0 ? x : sum[c0 + jj] + x;
          }
        }
        fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&tempty[acc]));
      }
      if (!ok) break;
      const int row = m0 + 32 * q + lane;
      float* crow = C + (long)z * split_stride + (long)row * ldc;
      float* lrow = Clo ? Clo + (long)row * ldc : nullptr;
      const float* rrow = R ? R + (long)row * ldr : nullptr;
      if (row < m && out_bf16) {
        // split output in BF16: C and Clo are BF16 arrays (hi, lo parts)
        uint16_t* bh = (uint16_t*)C + (long)row * ldc;
        uint16_t* bl = (uint16_t*)Clo + (long)row * ldc;
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
          const int cb = n0 + c0;
          if (cb + 32 <= n && (ldc & 7) == 0 && ((uintptr_t)(bh + cb) & 15) == 0 &&
              ((uintptr_t)(bl + cb) & 15) == 0) {
#pragma unroll
            for (int jj = 0; jj < 32; jj += 8) {
              uint32_t hw[4], lw[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                uint16_t h0, l0, h1, l1;
                bf16_split(alpha * sum[c0 + jj + 2 * u], h0, l0);
                bf16_split(alpha * sum[c0 + jj + 2 * u + 1], h1, l1);
                hw[u] = (uint32_t)h0 | ((uint32_t)h1 << 16);
                lw[u] = (uint32_t)l0 | ((uint32_t)l1 << 16);
              }
              *(uint4*)(bh + cb + jj) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
              *(uint4*)(bl + cb + jj) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int col = cb + jj;
              if (col < n) {
                uint16_t h, l;
                bf16_split(alpha * sum[c0 + jj], h, l);
                bh[col] = h;
                bl[col] = l;
              }
            }
          }
        }
      } else if (row < m) {
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
          const int cb = n0 + c0;
          if (cb + 32 <= n && (ldc & 3) == 0 && (!rrow || (ldr & 3) == 0) &&
              ((uintptr_t)(crow + cb) & 15) == 0 &&
              (!lrow || ((uintptr_t)(lrow + cb) & 15) == 0) &&
              (!rrow || ((uintptr_t)(rrow + cb) & 15) == 0)) {
#pragma unroll
            for (int jj = 0; jj < 32; jj += 4) {
              float4 o;
              o.x = alpha * sum[c0 + jj]; o.y = alpha * sum[c0 + jj + 1];
              o.z = alpha * sum[c0 + jj + 2]; o.w = alpha * sum[c0 + jj + 3];
              if (rrow) {
                float4 r = *(const float4*)(rrow + cb + jj);
                o.x += beta * r.x; o.y += beta * r.y; o.z += beta * r.z; o.w += beta * r.w;
              }
              if (lrow) {   // split output: TF32 hi part here, the remainder in Clo
                float4 h;
                h.x = tf32_hi(o.x); h.y = tf32_hi(o.y); h.z = tf32_hi(o.z); h.w = tf32_hi(o.w);
                float4 l;
                l.x = tf32_lo(o.x, h.x); l.y = tf32_lo(o.y, h.y); l.z = tf32_lo(o.z, h.z); l.w = tf32_lo(o.w, h.w);
                *(float4*)(lrow + cb + jj) = l;
                o = h;
              }
              *(float4*)(crow + cb + jj) = o;
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj) {
              const int col = cb + jj;
              if (col < n) {
                float o = alpha * sum[c0 + jj];
                if (rrow) o += beta * rrow[col];
                if (lrow) {
                  const float h = tf32_hi(o);
                  lrow[col] = tf32_lo(o, h);
                  o = h;
                }
                crow[col] = o;
              }
            }
          }
        }
      }
    }
  } else if (SPLIT3) {
    // operand split: hi = x rounded to TF32 in place, lo = x - hi
    const int t = threadIdx.x - 192;
    int it = 0;
    for (int i = blockIdx.x; i < wk.items && !*fail; i += gridDim.x) {
      int m0, tn, z, kt0, nkt;
      wk.item(i, m0, tn, z, kt0, nkt);
      for (int k = 0; k < nkt; ++k, ++it) {
        const int s = it % S;
        const uint32_t ph = (uint32_t)(it / S) & 1u;
        if (!mbar_wait(smem_u32(&full[s]), ph)) {
          flag_timeout(status);
          *fail = 1;
          break;
        }
        float4* ah = (float4*)a_hi(s);
        float4* al = (float4*)a_lo(s);
        for (int e = t; e < Cfg::A_BYTES / 16; e += 128) {
          float4 x = ah[e], h, l;
          h.x = tf32_hi(x.x); h.y = tf32_hi(x.y); h.z = tf32_hi(x.z); h.w = tf32_hi(x.w);
          l.x = tf32_lo(x.x, h.x); l.y = tf32_lo(x.y, h.y); l.z = tf32_lo(x.z, h.z); l.w = tf32_lo(x.w, h.w);
          ah[e] = h;
          al[e] = l;
        }
        if (!BLO) {
          float4* bh = (float4*)b_hi(s);
          float4* bl = (float4*)b_lo(s);
          for (int e = t; e < Cfg::B_BYTES / 16; e += 128) {
            float4 x = bh[e], h, l;
            h.x = tf32_hi(x.x); h.y = tf32_hi(x.y); h.z = tf32_hi(x.z); h.w = tf32_hi(x.w);
            l.x = tf32_lo(x.x, h.x); l.y = tf32_lo(x.y, h.y); l.z = tf32_lo(x.z, h.z); l.w = tf32_lo(x.w, h.w);
            bh[e] = h;
            bl[e] = l;
          }
        }
        fence_proxy_async();
        mbar_arrive(smem_u32(&conv[s]));
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 2 * BN);
}
// ------------------------------------------------------------------ Taylor
// One CTA of 256 threads per (walker, 64-column chunk) work item, looping
// over items. The chunk's columns form two independent halves of 32 (the
// series acts on every column alone), each run by one warpgroup with its
// own MMA chain, accumulator and barrier, so that one half's products run
// on the tensor core while the other half's epilogue runs on the CUDA
// cores. Thread r of a warpgroup owns row r of the real 2M-row form (r < 64:
// real part of orbital row r; r >= 64: imaginary part of row r - 64) and the
// matching TMEM lane; it keeps the running sum of the series for its row and
// its half's 32 columns in registers.
//
// The operator, in its real form A = [[Vr, -Vi], [Vi, Vr]] (2M x 2M padded to
// 128 x 128), is the MMA's A operand in tensor memory, shared by both halves:
// lane r holds row r, one 32-bit column per K index (TF32X3: hi in columns
// 128..255, lo in 256..383; half h accumulates into columns 64h .. 64h + 63,
// two chains of 32).
// Each thread writes its own row (warpgroup h the K columns 64h..64h+63) with
// tcgen05.st, so the operand needs no shared-memory swizzle and the MMAs read
// only the current term t of their half (the B operand) from shared memory.
//
// With a half-step image (FUSE_B), the symmetric Trotter factors are applied
// on the tensor cores too: t0 = Phi + (B_half - I) Phi before the series and
// out = s + (B_half - I) s after it, the identity part added exactly in FP32
// and (B_half - I) in its real 2M-row form [[dB, 0], [0, dB]] bulk-copied
// once per CTA into shared memory from a pre-swizzled (and pre-split) image.
constexpr int TY_THREADS = 256;
constexpr int TY_A_BYTES = 128 * 128 * 4;     // half-step image, 4 K-blocks
constexpr int TY_H_BYTES = 32 * 128 * 4;      // one half's term t, 32 columns
constexpr int TY_B_BYTES = 2 * TY_H_BYTES;    // both halves
constexpr int TY_V_BYTES = 2 * 64 * 64 * 4;   // raw V of the next walker (TF32X3)
template <bool SPLIT3>
constexpr int taylor_smem() {
  return (TY_A_BYTES + TY_B_BYTES) * (SPLIT3 ? 2 : 1) + 1024 + 128 + (SPLIT3 ? TY_V_BYTES : 0);
}
constexpr uint32_t TY_TMEM_AHI = 128, TY_TMEM_ALO = 256;   // column offsets

// (B_half - I) as the operand image the Taylor kernel copies in: hi tile,
// then (TF32X3) lo tile, each 128 x 128 fp32 in the K-major SW128 layout.
__global__ void bhalf_image_kernel(int M, const float* __restrict__ dB, float* __restrict__ img,
                                   int split3) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 128 * 128) return;
  const int r = e / 128, k = e % 128;
  const int rc = r >> 6, rr = r & 63, kc = k >> 6, kk = k & 63;
  float x = 0.f;
  if (rc == kc && rr < M && kk < M) x = dB[rr * M + kk];
  const uint32_t off = sw128_offset(r, k, 128) / 4;
  if (split3) {
    const float h = tf32_hi(x);
    img[off] = h;
    img[128 * 128 + off] = tf32_lo(x, h);
  } else {
    img[off] = x;
  }
}

// One term column into a half's B operand (32 rows of the K-major SW128
// tile; K index = the thread's row r), hi and (TF32X3) lo parts.
template <bool SPLIT3>
__device__ __forceinline__ void put_term(uint32_t hi, uint32_t lo, int j, int r, float x) {
  const uint32_t off = sw128_offset(j, r, 32);
  if (SPLIT3) {
    const float h = tf32_hi(x);
    st_shared_f32(hi + off, h);
    st_shared_f32(lo + off, tf32_lo(x, h));
  } else {
    st_shared_f32(hi + off, x);
  }
}

// The products of one half run as two independent accumulation chains,
// even and odd K steps into accumulators tD and tD + 32 (summed by the
// epilogue): consecutive MMAs then never wait for each other's accumulator.
//
// D (+)= A B for one half (N = 32) with both operands in shared memory (A =
// the half-step image, 128 rows per K-block; B = the half's term, 32 rows).
template <bool SPLIT3>
__device__ __forceinline__ void issue_half_step(uint32_t tD0, uint32_t Ahi, uint32_t Alo,
                                                uint32_t Bhi, uint32_t Blo, uint32_t id) {
  const uint64_t a0 = desc_sw128(Ahi), b0 = desc_sw128(Bhi);
  const uint64_t al0 = desc_sw128(Alo), bl0 = desc_sw128(Blo);
#pragma unroll
  for (int ks = 0; ks < 16; ++ks) {
    const uint32_t kb = ks >> 2, koff = (ks & 3) * 32;
    const uint32_t tD = tD0 + 32u * (uint32_t)(ks & 1);
    const uint64_t ad = desc_add(a0, kb * 16384 + koff);
    const uint64_t bd = desc_add(b0, kb * 4096 + koff);
    mma_tf32(tD, ad, bd, id, ks > 1 ? 1u : 0u);
    if (SPLIT3) {
      mma_tf32(tD, ad, desc_add(bl0, kb * 4096 + koff), id, 1u);
      mma_tf32(tD, desc_add(al0, kb * 16384 + koff), bd, id, 1u);
    }
  }
}

// D = A B for one half with A in tensor memory (the operator) and B in
// shared memory.
template <bool SPLIT3>
__device__ __forceinline__ void issue_term(uint32_t tD0, uint32_t tAhi, uint32_t tAlo,
                                           uint32_t Bhi, uint32_t Blo, uint32_t id) {
  const uint64_t b0 = desc_sw128(Bhi), bl0 = desc_sw128(Blo);
#pragma unroll
  for (int ks = 0; ks < 16; ++ks) {
    const uint32_t kb = ks >> 2, koff = (ks & 3) * 32;
    const uint32_t tD = tD0 + 32u * (uint32_t)(ks & 1);
    const uint64_t bd = desc_add(b0, kb * 4096 + koff);
    mma_tf32_ts(tD, tAhi + 8 * ks, bd, id, ks > 1 ? 1u : 0u);
    if (SPLIT3) {
      mma_tf32_ts(tD, tAhi + 8 * ks, desc_add(bl0, kb * 4096 + koff), id, 1u);
      mma_tf32_ts(tD, tAlo + 8 * ks, bd, id, 1u);
    }
  }
}

// The sum of a half's two accumulation chains (columns c .. c + 31 and
// c + 32 .. c + 63 of this thread's lane), 8 columns of each at a time.
__device__ __forceinline__ void tmem_ld_sum2(uint32_t taddr, float* v) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    float a[8], b[8];
    tmem_ld8_nowait(taddr + 8u * (uint32_t)g, a);
    tmem_ld8_nowait(taddr + 32u + 8u * (uint32_t)g, b);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 8; ++i) v[8 * g + i] = a[i] + b[i];
  }
}

// Barrier of one warpgroup (ids 1 and 2; 0 is __syncthreads).
__device__ __forceinline__ void group_sync(int h) {
  asm volatile("bar.sync %0, 128;" ::"r"(1 + h) : "memory");
}

template <bool SPLIT3>
__global__ void __launch_bounds__(TY_THREADS, 1)
tc_taylor_kernel(int W, int M, int N, int order, const float* __restrict__ V,
                 const float* Pin, float* Pout,
                 const float* __restrict__ dB_img, int* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  // image hi and lo are adjacent so one bulk copy fills both
  unsigned char* Ihi = base;
  unsigned char* Ilo = base + TY_A_BYTES;
  unsigned char* Bbase = base + TY_A_BYTES * (SPLIT3 ? 2 : 1);   // hi halves, then lo halves
  uint64_t* bar = (uint64_t*)(Bbase + TY_B_BYTES * (SPLIT3 ? 2 : 1));   // [2]: one per half
  uint64_t* lbar = bar + 2;
  uint64_t* vbar = bar + 3;
  uint32_t* tslot = (uint32_t*)(bar + 4);
  // TF32X3 with M even: the next walker's V (2 M^2 floats, contiguous) is
  // bulk-copied into the spare shared memory while this walker's series runs
  float* vst = (float*)(base + (TY_A_BYTES + TY_B_BYTES) * 2 + 128);
  __shared__ int s_fail;
  constexpr uint32_t kCols = SPLIT3 ? 512 : 256;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int h = tid >> 7;                  // half (warpgroup): columns 32h .. 32h + 31
  const int r = tid & 127;                 // embedded row / K index owned
  const int rc = r >> 6, rr = r & 63;      // component (0 re, 1 im), orbital row
  const int nchunk = (N + 63) / 64;
  const int items = W * nchunk;
  const bool fuse_b = dB_img != nullptr;
  const uint32_t img_bytes = (uint32_t)TY_A_BYTES * (SPLIT3 ? 2u : 1u);
  if (tid == 0) {
    s_fail = 0;
    mbar_init(smem_u32(bar), 1);
    mbar_init(smem_u32(bar + 1), 1);
    mbar_init(smem_u32(lbar), 1);
    mbar_init(smem_u32(vbar), 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), kCols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t tAhi = tmem + TY_TMEM_AHI, tAlo = tmem + TY_TMEM_ALO;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
  const uint32_t tD = tmem + 64u * (uint32_t)h;   // this half's two accumulators
  const uint32_t id = idesc_tf32(128, 32);
  const uint32_t sIhi = smem_u32(Ihi), sIlo = smem_u32(Ilo);
  const uint32_t sBhi = smem_u32(Bbase) + (uint32_t)(h * TY_H_BYTES);
  const uint32_t sBlo = smem_u32(Bbase) + (uint32_t)(TY_B_BYTES + h * TY_H_BYTES);
  const uint32_t mybar = smem_u32(bar + h);
  const bool leader = r == 0;              // the half's MMA issuer
  const int MM = M * M;
  uint32_t phase = 0;
  // a wait of this thread that gave up: the thread issues no further MMA
  // (as its half's leader) and waits no more; the leader waits once more,
  // bounded, for that commit before the CTA frees its tensor memory
  bool failed = false;
  uint32_t fail_parity = 0;

  auto wait_mma = [&]() {
    if (!failed && !mbar_wait(mybar, phase)) {
      flag_timeout(status);
      s_fail = 1;
      failed = true;
      fail_parity = phase;
    }
    phase ^= 1u;
    fence_after_sync();
  };
  // the half's term writes are visible to the tensor core before its leader
  // issues, and the previous TMEM reads of the accumulator are complete
  auto sync_half = [&]() {
    fence_proxy_async();
    fence_before_sync();
    group_sync(h);
    fence_after_sync();
  };
  bool img_pending = false;
  if (fuse_b) {                            // the half-step image, once per CTA
    if (tid == 0) {
      mbar_arrive_expect_tx(smem_u32(lbar), img_bytes);
      bulk_load(sIhi, dB_img, img_bytes, smem_u32(lbar));
    }
    img_pending = true;
  }
  const bool vpre = SPLIT3 && (M & 1) == 0;   // rows of 8 M^2 bytes, 16-byte multiples
  const uint32_t vbytes = (uint32_t)(8 * MM);
  uint32_t vphase = 0;
  bool v_inflight = false;
  auto load_v = [&](int it) {             // called by every thread after a barrier
    if (tid == 0) {
      fence_proxy_async();                // earlier generic reads of vst come first
      mbar_arrive_expect_tx(smem_u32(vbar), vbytes);
      bulk_load(smem_u32(vst), V + (long)(it / nchunk) * 2 * MM, vbytes, smem_u32(vbar));
    }
    v_inflight = true;
  };
  if (vpre && (int)blockIdx.x < items) load_v(blockIdx.x);

  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int w = item / nchunk;
    const int j0 = (item - w * nchunk) * 64 + 32 * h;   // this half's first column
    const int nc = max(0, min(32, N - j0));             // and its column count
    const bool active = nc > 0;                          // uniform over the half
    const float* Vw = V + (long)w * 2 * MM;
    // ---- t0 = the half's columns; this thread's row of it seeds the sum
    float acc[32];
    if (active) {
      const float* Pw = Pin + ((long)w * N + j0) * 2 * M;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        acc[j] = (j < nc && rr < M) ? Pw[((long)j * 2 + rc) * M + rr] : 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) put_term<SPLIT3>(sBhi, sBlo, j, r, acc[j]);
    }
    if (fuse_b) {                          // t0 = Phi + dB Phi
      if (img_pending) {
        if (mbar_wait(smem_u32(lbar), 0)) {
          img_pending = false;
        } else {                           // still in flight: drained at teardown
          flag_timeout(status);
          s_fail = 1;
        }
      }
      if (active) {
        sync_half();
        if (leader && !failed) {
          issue_half_step<SPLIT3>(tD, sIhi, sIlo, sBhi, sBlo, id);
          mma_commit(mybar);
        }
        wait_mma();
        float v[32];
        tmem_ld_sum2(tD + lane_base, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          acc[j] += v[j];
          put_term<SPLIT3>(sBhi, sBlo, j, r, acc[j]);
        }
      }
    }
    // ---- the operator into tensor memory: row r of [[Vr, -Vi], [Vi, Vr]],
    // columns 0..63 from plane rc of V, columns 64..127 from the other plane
    // (negated for the real rows), zero beyond M in each half; warpgroup h
    // writes the K columns 64h .. 64h + 63 of its rows
    const float* vsrc = Vw;
    if (vpre) {
      if (mbar_wait(smem_u32(vbar), vphase)) {
        vphase ^= 1u;
        v_inflight = false;
      } else {                             // still in flight: drained at teardown
        flag_timeout(status);
        s_fail = 1;
      }
      vsrc = vst;
    }
    {
      const bool vec = (M & 3) == 0;       // rows 16-byte aligned
#pragma unroll 1
      for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 16) {
        const int half = c0 >> 6, k0 = c0 & 63;
        const int plane = half == 0 ? rc : 1 - rc;
        const float sgn = (rc == 0 && half == 1) ? -1.f : 1.f;
        const float* src = vsrc + (long)plane * MM + (long)rr * M;
        float x[16];
        if (rr < M && vec && k0 + 16 <= M) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 f = *reinterpret_cast<const float4*>(src + k0 + 4 * q);
            x[4 * q] = f.x; x[4 * q + 1] = f.y; x[4 * q + 2] = f.z; x[4 * q + 3] = f.w;
          }
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u) x[u] = (rr < M && k0 + u < M) ? src[k0 + u] : 0.f;
        }
        if (SPLIT3) {
          float hv[16], lv[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            hv[u] = tf32_hi(sgn * x[u]);
            lv[u] = tf32_lo(sgn * x[u], hv[u]);
          }
          tmem_st16(tAhi + lane_base + (uint32_t)c0, hv);
          tmem_st16(tAlo + lane_base + (uint32_t)c0, lv);
        } else {
#pragma unroll
          for (int u = 0; u < 16; ++u) x[u] *= sgn;
          tmem_st16(tAhi + lane_base + (uint32_t)c0, x);
        }
      }
      tmem_wait_st();
    }
    // the whole operator and both halves' terms are in place before either
    // half's series starts; every thread has read vst
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (vpre) {
      const int next = item + (int)gridDim.x;
      if (next < items && !s_fail) load_v(next);
    }
    if (active) {
      for (int term = 1; term <= order; ++term) {
        if (term > 1) sync_half();
        if (leader && !failed) {
          issue_term<SPLIT3>(tD, tAhi, tAlo, sBhi, sBlo, id);
          mma_commit(mybar);
        }
        wait_mma();
        const float inv = 1.0f / (float)term;
        float v[32];
        tmem_ld_sum2(tD + lane_base, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float x = v[j] * inv;
          acc[j] += x;
          if (term < order || fuse_b) put_term<SPLIT3>(sBhi, sBlo, j, r, term < order ? x : acc[j]);
        }
      }
      if (fuse_b) {                        // out = s + dB s
        sync_half();
        if (leader && !failed) {
          issue_half_step<SPLIT3>(tD, sIhi, sIlo, sBhi, sBlo, id);
          mma_commit(mybar);
        }
        wait_mma();
        float v[32];
        tmem_ld_sum2(tD + lane_base, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += v[j];
      }
      if (rr < M) {
        float* Ow = Pout + ((long)w * N + j0) * 2 * M;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (j < nc) Ow[((long)j * 2 + rc) * M + rr] = acc[j];
      }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (s_fail) break;
  }
  if (v_inflight && !mbar_wait(smem_u32(vbar), vphase))   // no copy may outlive the CTA
    flag_timeout(status);
  if (img_pending && !mbar_wait(smem_u32(lbar), 0)) flag_timeout(status);
  if (leader && failed && !mbar_wait(mybar, fail_parity))  // nor an MMA the allocation
    flag_timeout(status);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ------------------------------------------------------ Taylor, BF16X3
// The on-chip series of tc_taylor_kernel (M <= 64, real 2M-row operator in
// tensor memory, one walker chunk of 64 columns per work item, half steps
// fused) with BF16 hi + lo operands and three kind::f16 products per term.
// BF16 halves every operand: the operator's hi and lo parts take 64 TMEM
// columns each (two K values per 32-bit column), the term 16 KB per part in
// shared memory, the half-step image 32 KB per part. With 192 TMEM columns
// and 97 KB of shared memory per CTA, two CTAs share an SM, so one walker's
// products overlap the other's epilogue.
constexpr int TB_A_BYTES = 128 * 128 * 2;     // half-step image part, 2 K-blocks of 64
constexpr int TB_B_BYTES = 64 * 128 * 2;      // term part, 64 columns x 128 K
constexpr int TB_SMEM = 2 * TB_A_BYTES + 2 * TB_B_BYTES + 1024 + 128;
constexpr uint32_t TB_TMEM_AHI = 64, TB_TMEM_ALO = 128, TB_TMEM_COLS = 256;

// (B_half - I) image in BF16: hi part then lo part, 128 x 128 each, K-major
// SW128 with 64 K values per row block.
__global__ void bhalf_image_bf16_kernel(int M, const float* __restrict__ dB,
                                        uint16_t* __restrict__ img) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 128 * 128) return;
  const int r = e / 128, k = e % 128;
  const int rc = r >> 6, rr = r & 63, kc = k >> 6, kk = k & 63;
  float x = 0.f;
  if (rc == kc && rr < M && kk < M) x = dB[rr * M + kk];
  const uint32_t off = sw128_offset_bf16(r, k, 128) / 2;
  uint16_t h, l;
  bf16_split(x, h, l);
  img[off] = h;
  img[128 * 128 + off] = l;
}

__device__ __forceinline__ void put_operand_bf16(uint32_t shi, uint32_t slo, uint32_t off,
                                                 float x) {
  uint16_t h, l;
  bf16_split(x, h, l);
  st_shared_b16(shi + off, h);
  st_shared_b16(slo + off, l);
}

__global__ void __launch_bounds__(128, 2)
tc_taylor_bf16_kernel(int W, int M, int N, int order, const float* __restrict__ V,
                      const float* Pin, float* Pout, const uint16_t* __restrict__ dB_img,
                      int* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* Ihi = base;                      // image hi, lo adjacent (one bulk copy)
  unsigned char* Bhi = base + 2 * TB_A_BYTES;
  unsigned char* Blo = Bhi + TB_B_BYTES;
  uint64_t* bar = (uint64_t*)(Blo + TB_B_BYTES);
  uint64_t* lbar = bar + 1;
  uint32_t* tslot = (uint32_t*)(bar + 2);
  __shared__ int s_fail;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int nchunk = (N + 63) / 64;
  const int items = W * nchunk;
  const bool fuse_b = dB_img != nullptr;
  if (tid == 0) {
    s_fail = 0;
    mbar_init(smem_u32(bar), 1);
    mbar_init(smem_u32(lbar), 1);
    mbar_fence_init();
  }
  if (warp == 0) tmem_alloc(smem_u32(tslot), TB_TMEM_COLS);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t tAhi = tmem + TB_TMEM_AHI, tAlo = tmem + TB_TMEM_ALO;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  const uint32_t id = idesc_bf16(128, 64);
  uint32_t phase = 0;
  const int r = tid;                       // embedded row / K index owned
  const int rc = r >> 6, rr = r & 63;      // component (0 re, 1 im), orbital row
  const uint32_t sIhi = smem_u32(Ihi), sIlo = sIhi + TB_A_BYTES;
  const uint32_t sBhi = smem_u32(Bhi), sBlo = smem_u32(Blo);
  const int MM = M * M;

  // a wait of this thread that gave up: the thread issues no further MMA
  // (as the issuer, thread 0) and waits no more; thread 0 then waits once
  // more, bounded, for that commit before the CTA frees its tensor memory
  bool failed = false;
  uint32_t fail_parity = 0;
  auto wait_mma = [&]() {
    if (!failed && !mbar_wait(smem_u32(bar), phase)) {
      flag_timeout(status);
      s_fail = 1;
      failed = true;
      fail_parity = phase;
    }
    phase ^= 1u;
    fence_after_sync();
  };
  auto sync_for_mma = [&]() {
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
  };
  // D (+)= image x term (both in shared memory), three products per K step
  auto half_products = [&]() {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
      const int kb = ks >> 2, koff = (ks & 3) * 32;
      const uint64_t ad = desc_sw128(sIhi + kb * 16384 + koff);
      const uint64_t bd = desc_sw128(sBhi + kb * 8192 + koff);
      mma_bf16(tmem, ad, bd, id, ks > 0 ? 1u : 0u);
      mma_bf16(tmem, ad, desc_sw128(sBlo + kb * 8192 + koff), id, 1u);
      mma_bf16(tmem, desc_sw128(sIlo + kb * 16384 + koff), bd, id, 1u);
    }
  };
  // D = operator (tensor memory) x term (shared memory)
  auto series_products = [&]() {
#pragma unroll
    for (int ks = 0; ks < 8; ++ks) {
      const int kb = ks >> 2, koff = (ks & 3) * 32;
      const uint64_t bd = desc_sw128(sBhi + kb * 8192 + koff);
      mma_bf16_ts(tmem, tAhi + 8 * ks, bd, id, ks > 0 ? 1u : 0u);
      mma_bf16_ts(tmem, tAhi + 8 * ks, desc_sw128(sBlo + kb * 8192 + koff), id, 1u);
      mma_bf16_ts(tmem, tAlo + 8 * ks, bd, id, 1u);
    }
  };
  bool img_pending = false;
  if (fuse_b) {                            // the half-step image, once per CTA
    if (tid == 0) {
      mbar_arrive_expect_tx(smem_u32(lbar), 2u * TB_A_BYTES);
      bulk_load(sIhi, dB_img, 2u * TB_A_BYTES, smem_u32(lbar));
    }
    img_pending = true;
  }

  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int w = item / nchunk;
    const int j0 = (item - w * nchunk) * 64;
    const int nc = min(64, N - j0);
    const float* Vw = V + (long)w * 2 * MM;
    float acc[64];
    const float* Pw = Pin + ((long)w * N + j0) * 2 * M;
#pragma unroll
    for (int j = 0; j < 64; ++j)
      acc[j] = (j < nc && rr < M) ? Pw[((long)j * 2 + rc) * M + rr] : 0.f;
#pragma unroll
    for (int j = 0; j < 64; ++j)
      put_operand_bf16(sBhi, sBlo, sw128_offset_bf16(j, r, 64), acc[j]);
    if (fuse_b) {                          // t0 = Phi + dB Phi
      if (img_pending) {
        if (mbar_wait(smem_u32(lbar), 0)) {
          img_pending = false;
        } else {                           // still in flight: drained at teardown
          flag_timeout(status);
          s_fail = 1;
        }
      }
      sync_for_mma();
      if (tid == 0 && !failed) {
        half_products();
        mma_commit(smem_u32(bar));
      }
      wait_mma();
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          acc[c0 + j] += v[j];
          put_operand_bf16(sBhi, sBlo, sw128_offset_bf16(c0 + j, r, 64), acc[c0 + j]);
        }
      }
    }
    // the operator into tensor memory: row r of [[Vr, -Vi], [Vi, Vr]] as BF16
    // hi and lo parts, two K values per 32-bit column (lower K in the low half)
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 32) {
      const int half = c0 >> 6, k0 = c0 & 63;
      const int plane = half == 0 ? rc : 1 - rc;
      const float sgn = (rc == 0 && half == 1) ? -1.f : 1.f;
      const float* src = Vw + (long)plane * MM + (long)rr * M;
      float hw[16], lw[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int ka = k0 + 2 * u, kb2 = ka + 1;
        const float xa = (rr < M && ka < M) ? sgn * src[ka] : 0.f;
        const float xb = (rr < M && kb2 < M) ? sgn * src[kb2] : 0.f;
        uint16_t ha, la, hb, lb;
        bf16_split(xa, ha, la);
        bf16_split(xb, hb, lb);
        hw[u] = __uint_as_float((uint32_t)ha | ((uint32_t)hb << 16));
        lw[u] = __uint_as_float((uint32_t)la | ((uint32_t)lb << 16));
      }
      tmem_st16(tAhi + lane_base + (uint32_t)(c0 >> 1), hw);
      tmem_st16(tAlo + lane_base + (uint32_t)(c0 >> 1), lw);
    }
    tmem_wait_st();
    for (int term = 1; term <= order; ++term) {
      sync_for_mma();
      if (tid == 0 && !failed) {
        series_products();
        mma_commit(smem_u32(bar));
      }
      wait_mma();
      const float inv = 1.0f / (float)term;
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float x = v[j] * inv;
          acc[c0 + j] += x;
          if (term < order || fuse_b)
            put_operand_bf16(sBhi, sBlo, sw128_offset_bf16(c0 + j, r, 64),
                             term < order ? x : acc[c0 + j]);
        }
      }
    }
    if (fuse_b) {                          // out = s + dB s
      sync_for_mma();
      if (tid == 0 && !failed) {
        half_products();
        mma_commit(smem_u32(bar));
      }
      wait_mma();
#pragma unroll
      for (int c0 = 0; c0 < 64; c0 += 32) {
        float v[32];
        tmem_ld32(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[c0 + j] += v[j];
      }
    }
    float* Ow = Pout + ((long)w * N + j0) * 2 * M;
    if (rr < M) {
#pragma unroll
      for (int j = 0; j < 64; ++j)
        if (j < nc) Ow[((long)j * 2 + rc) * M + rr] = acc[j];
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (s_fail) break;
  }
  if (img_pending && !mbar_wait(smem_u32(lbar), 0)) flag_timeout(status);   // no copy may outlive the CTA
  if (tid == 0 && failed && !mbar_wait(smem_u32(bar), fail_parity))  // nor an MMA the allocation
    flag_timeout(status);
  fence_before_sync();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TB_TMEM_COLS);
}

// ------------------------------------------------------------ wide Taylor
// B_half exp_T(V) B_half Phi for 64 < M <= 256 (Sec. II, Thouless propagation
// by matrix products), where the operator no longer fits on chip: each CTA
// takes one (walker, column chunk) item at a time and runs it through
// R = order + 2 rounds of products D = A t, A streamed from L2 by TMA in
// 128-row x 32-K tiles and t (the current term) resident in shared memory as
// the B operand:
//   round 0          A = B_half - I (real):   t0 = Phi + D
//   rounds 1..order  A = V (complex):         t_n = D / n, s += t_n
//   round order + 1  A = B_half - I:          out = s + D
// The complex product uses two accumulators per 128-row tile,
// P = Vr [tr | ti] and Q = Vi [tr | ti] (B rows: the chunk's real parts, then
// its imaginary parts), combined in the epilogue as Dr = Pr - Qi,
// Di = Pi + Qr. Rows and K indices past M are zero-filled by the TMA.
// TF32X3: A arrives pre-split (hi and lo planes in global memory); the
// epilogue writes t as hi and lo planes; three products per MMA step.
// BF16X3 (BF): the same with BF16 hi and lo parts (kind::f16 MMAs, 64 K
// values per 128-byte row, so a stage covers twice the K range and the
// streamed operand half the bytes).
// Warps: 0 TMA producer, 1 MMA issuer, 2..9 epilogue (TMEM lane quadrant =
// warp % 4; group (warp - 2) / 4 takes the second row tile, or the second
// half of the columns when there is one row tile).
constexpr int TW_THREADS = 320;
constexpr int TW_TILE_BYTES = 128 * 32 * 4;   // one 128 x 32 fp32 operand tile

template <bool SPLIT3, bool BF>
__global__ void __launch_bounds__(TW_THREADS, 1)
tc_taylor_wide_kernel(const __grid_constant__ CUtensorMap mapV,
                      const __grid_constant__ CUtensorMap mapVlo,
                      const __grid_constant__ CUtensorMap mapB,
                      const __grid_constant__ CUtensorMap mapBlo, int W, int M, int N,
                      int order, int n16, int S, const float* Pin, float* Pout, int* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  constexpr int KBLK = BF ? 64 : 32;                   // K values per 128-byte row
  const int MT = (M + 127) / 128, KB = (M + KBLK - 1) / KBLK;
  const int P = SPLIT3 ? 2 : 1;
  const int kb_bytes = 2 * n16 * 128;                 // one K block of B
  const int b_bytes = KB * kb_bytes;
  unsigned char* Bhi = base;
  unsigned char* Blo = base + b_bytes;                // TF32X3 only
  unsigned char* stages = base + b_bytes * P;
  const int stage_bytes = TW_TILE_BYTES * P;
  uint64_t* bars = (uint64_t*)(stages + S * stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + S;
  uint64_t* bready = bars + 2 * S;   // t for the next round is in shared memory
  uint64_t* aready = bars + 2 * S + 1;   // the round's accumulators are complete
  uint32_t* tslot = (uint32_t*)(bars + 2 * S + 2);
  __shared__ int s_fail;
  volatile int* fail = &s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nchunk = (N + n16 - 1) / n16;
  const int items = W * nchunk;
  const int R = order + 2;
  int cols = 32;
  while (cols < MT * 4 * n16) cols *= 2;
  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(bready), 8);
    mbar_init(smem_u32(aready), 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(smem_u32(tslot), (uint32_t)cols);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  // accumulator (row tile mt, plane p) starts at column (2 mt + p) * 2 n16
  auto acc_col = [&](int mt, int p) { return (uint32_t)((2 * mt + p) * 2 * n16); };

  if (warp == 0) {
    if (lane == 0) {
      int it = 0;
      for (int item = blockIdx.x; item < items && !*fail; item += gridDim.x) {
        const int w = item / nchunk;
        for (int r = 0; r < R && !*fail; ++r) {
          const bool half = (r == 0 || r == R - 1);
          const int planes = half ? 1 : 2;
          for (int mt = 0; mt < MT && !*fail; ++mt)
            for (int kb = 0; kb < KB && !*fail; ++kb)
              for (int pl = 0; pl < planes; ++pl, ++it) {
                const int s = it % S;
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                if (it >= S && !mbar_wait(smem_u32(&empty[s]), ph ^ 1u)) {
                  flag_timeout(status);
                  *fail = 1;
                  break;
                }
                unsigned char* st = stages + s * stage_bytes;
                mbar_arrive_expect_tx(smem_u32(&full[s]), (uint32_t)stage_bytes);
                const int z = half ? 0 : 2 * w + pl;
                tma_load_3d(smem_u32(st), half ? (const void*)&mapB : (const void*)&mapV,
                            kb * KBLK, mt * 128, z, smem_u32(&full[s]));
                if (SPLIT3)
                  tma_load_3d(smem_u32(st + TW_TILE_BYTES),
                              half ? (const void*)&mapBlo : (const void*)&mapVlo, kb * KBLK,
                              mt * 128, z, smem_u32(&full[s]));
              }
        }
      }
      // no copy may outlive the CTA
      for (int j = it - 1; j >= 0 && j >= it - S; --j)
        if (!mbar_wait(smem_u32(&full[j % S]), (uint32_t)(j / S) & 1u)) flag_timeout(status);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id = BF ? idesc_bf16(128, 2 * n16) : idesc_tf32(128, 2 * n16);
      const uint32_t sBhi = smem_u32(Bhi), sBlo = smem_u32(Blo);
      auto mma = [&](uint32_t td, uint64_t a, uint64_t b, uint32_t acc) {
        if (BF) mma_bf16(td, a, b, id, acc);
        else mma_tf32(td, a, b, id, acc);
      };
      int it = 0;
      uint32_t pb = 0, pa = 0;
      uint32_t last_bar = 0, last_par = 0;
      for (int item = blockIdx.x; item < items && !*fail; item += gridDim.x) {
        for (int r = 0; r < R && !*fail; ++r) {
          if (!mbar_wait(smem_u32(bready), pb)) {
            flag_timeout(status);
            *fail = 1;
            break;
          }
          pb ^= 1u;
          fence_after_sync();
          const bool half = (r == 0 || r == R - 1);
          const int planes = half ? 1 : 2;
          for (int mt = 0; mt < MT && !*fail; ++mt)
            for (int kb = 0; kb < KB && !*fail; ++kb)
              for (int pl = 0; pl < planes; ++pl, ++it) {
                const int s = it % S;
                const uint32_t ph = (uint32_t)(it / S) & 1u;
                if (!mbar_wait(smem_u32(&full[s]), ph)) {
                  flag_timeout(status);
                  *fail = 1;
                  break;
                }
                fence_after_sync();
                const uint32_t sa = smem_u32(stages + s * stage_bytes);
                const uint32_t td = tmem + acc_col(mt, pl);
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                  const uint64_t ad = desc_sw128(sa + ks * 32);
                  const uint64_t bd = desc_sw128(sBhi + kb * kb_bytes + ks * 32);
                  mma(td, ad, bd, (kb > 0 || ks > 0) ? 1u : 0u);
                  if (SPLIT3) {
                    mma(td, ad, desc_sw128(sBlo + kb * kb_bytes + ks * 32), 1u);
                    mma(td, desc_sw128(sa + TW_TILE_BYTES + ks * 32), bd, 1u);
                  }
                }
                mma_commit(smem_u32(&empty[s]));
                last_bar = smem_u32(&empty[s]);
                last_par = ph;
              }
          if (*fail) break;
          mma_commit(smem_u32(aready));
          last_bar = smem_u32(aready);
          last_par = pa;
          pa ^= 1u;
        }
      }
      if (last_bar && !mbar_wait(last_bar, last_par)) flag_timeout(status);
    }
  } else {
    // epilogue: rows 32 q + lane of row tile mt, columns [c0, c0 + cp)
    const int g = (warp - 2) >> 2, q = warp & 3;
    const int mt = MT == 2 ? g : 0;
    const int cp = MT == 2 ? n16 : n16 / 2;
    const int c0 = MT == 2 ? 0 : g * cp;
    const int i = mt * 128 + 32 * q + lane;             // orbital row (= K index of B)
    const bool in_b = i < KB * KBLK;
    const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
    uint32_t pa = 0;
    float sr[32], si[32];
    // t into the B operand: real part of column c at B row c, imaginary at
    // B row n16 + c, K index i. Columns go in groups of 8 rows (one swizzle
    // atom): within a group, row u's offset is offu[u]; groups are 1024
    // bytes apart, and K block i / 32 sits at kb * 2 n16 * 128.
    uint32_t offu[8];
    {
      const int kk = i & (KBLK - 1);
      const int elem = BF ? (kk & 7) * 2 : (kk & 3) * 4;   // byte within the 16-byte chunk
      const int chunk = BF ? kk >> 3 : kk >> 2;
      const uint32_t base_i = (uint32_t)((i / KBLK) * 2 * n16 * 128 + elem);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        offu[u] = base_i + (uint32_t)(u * 128) + (uint32_t)(((chunk ^ u) & 7) << 4);
    }
    const uint32_t im_off = (uint32_t)(n16 >> 3) * 1024u;
    const uint32_t sBh = smem_u32(Bhi), sBl = smem_u32(Blo);
    // group gi (columns 8 gi .. 8 gi + 7), member u
    auto put_b = [&](int gi, int u, float xr, float xi) {
      if (!in_b) return;
      const uint32_t o_r = (uint32_t)gi * 1024u + offu[u], o_i = o_r + im_off;
      if (BF) {
        uint16_t hr, lr, hi_, li;
        bf16_split(xr, hr, lr);
        bf16_split(xi, hi_, li);
        st_shared_b16(sBh + o_r, hr);
        st_shared_b16(sBl + o_r, lr);
        st_shared_b16(sBh + o_i, hi_);
        st_shared_b16(sBl + o_i, li);
      } else if (SPLIT3) {
        const float hr = tf32_hi(xr), hi_ = tf32_hi(xi);
        st_shared_f32(sBh + o_r, hr);
        st_shared_f32(sBl + o_r, tf32_lo(xr, hr));
        st_shared_f32(sBh + o_i, hi_);
        st_shared_f32(sBl + o_i, tf32_lo(xi, hi_));
      } else {
        st_shared_f32(sBh + o_r, xr);
        st_shared_f32(sBh + o_i, xi);
      }
    };
    auto signal_b = [&]() {
      fence_proxy_async();          // generic shared-memory writes -> tensor core
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(bready));
    };
    for (int item = blockIdx.x; item < items && !*fail; item += gridDim.x) {
      const int w = item / nchunk;
      const int j0 = (item - w * nchunk) * n16;
      const int nc = min(n16, N - j0);
      const float* Pw = Pin + ((long)w * N + j0) * 2 * M;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c < cp) {
          const int col = c0 + c;
          const bool ok = col < nc && i < M;
          sr[c] = ok ? Pw[((long)col * 2 + 0) * M + i] : 0.f;
          si[c] = ok ? Pw[((long)col * 2 + 1) * M + i] : 0.f;
          put_b(col >> 3, c & 7, sr[c], si[c]);
        }
      }
      signal_b();
      for (int r = 0; r < R; ++r) {
        if (!mbar_wait(smem_u32(aready), pa)) {
          flag_timeout(status);
          *fail = 1;
          break;
        }
        pa ^= 1u;
        fence_after_sync();
        const bool half = (r == 0 || r == R - 1);
        const float inv = half ? 1.f : 1.f / (float)r;
#pragma unroll
        for (int cb = 0; cb < 32; cb += 8) {
          if (cb < cp) {
            float pr[8], pi[8], qr[8], qi[8];
            const uint32_t a0 = lane_addr + acc_col(mt, 0) + (uint32_t)(c0 + cb);
            tmem_ld8_nowait(a0, pr);
            tmem_ld8_nowait(a0 + (uint32_t)n16, pi);
            if (!half) {
              const uint32_t a1 = lane_addr + acc_col(mt, 1) + (uint32_t)(c0 + cb);
              tmem_ld8_nowait(a1, qr);
              tmem_ld8_nowait(a1 + (uint32_t)n16, qi);
            }
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int c = cb + u;
              float dr = pr[u], di = pi[u];
              if (!half) {                      // t_r = V t_{r-1} / r
                dr = (pr[u] - qi[u]) * inv;
                di = (pi[u] + qr[u]) * inv;
              }
              sr[c] += dr;                      // r = 0: t0 = Phi + (B_half - I) Phi;
              si[c] += di;                      // last: out = s + (B_half - I) s
              // the next round's operand: t_r, or the sum before the last half step
              const bool term = !half && r < order;
              pr[u] = term ? dr : sr[c];
              pi[u] = term ? di : si[c];
            }
            if (r < R - 1) {
#pragma unroll
              for (int u = 0; u < 8; ++u) put_b((c0 + cb) >> 3, u, pr[u], pi[u]);
            }
          }
        }
        if (r < R - 1) {
          signal_b();
        } else {
          fence_before_sync();
        }
      }
      if (*fail) break;
      float* Ow = Pout + ((long)w * N + j0) * 2 * M;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const int col = c0 + c;
        if (c < cp && col < nc && i < M) {
          Ow[((long)col * 2 + 0) * M + i] = sr[c];
          Ow[((long)col * 2 + 1) * M + i] = si[c];
        }
      }
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, (uint32_t)cols);
}

template <typename K>
cudaError_t set_smem(K kernel, int bytes) {
  return smem_optin((const void*)kernel) >= (size_t)bytes ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t make_map(TcCtx* t, CUtensorMap* map, const float* ptr, long rows, long k,
                     long ld, int box_rows) {
  if (((uintptr_t)ptr & 15) != 0 || (ld & 3) != 0 || k < 1 || rows < 1)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = t->encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void*)ptr, dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 3-D map of `planes` row-major matrices (rows x k, row stride ld elements,
// plane stride rows * ld elements) with 128-row boxes of 128 bytes along K
// (32 FP32 or 64 BF16 values).
cudaError_t make_map3(TcCtx* t, CUtensorMap* map, const void* ptr, long rows, long k, long ld,
                      long planes, bool bf16 = false) {
  const long es_b = bf16 ? 2 : 4;
  if (((uintptr_t)ptr & 15) != 0 || (ld * es_b) % 16 != 0 || k < 1 || rows < 1 || planes < 1)
    return cudaErrorInvalidValue;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * es_b), (cuuint64_t)(rows * ld * es_b)};
  cuuint32_t box[3] = {bf16 ? 64u : 32u, 128u, 1u};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = t->encode(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                         3, (void*)ptr, dims, strides,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, bool SPLIT3, bool BLO>
cudaError_t launch_gemm(TcCtx* t, cudaStream_t st, int m, int n, int k, const float* A,
                        long lda, const float* B, const float* Blo, long ldb, float* C,
                        long ldc, float alpha, float beta, const float* R, long ldr,
                        int ksplit, long split_stride, int* status, float* Clo,
                        bool out_bf16) {
  using Cfg = GemmCfg<BN, SPLIT3>;
  const cudaError_t attr = set_smem(tc_gemm_kernel<BN, SPLIT3, BLO>, Cfg::SMEM);
  if (attr != cudaSuccess) return attr;
  CUtensorMap ma, mb, mbl;
  cudaError_t e = make_map(t, &ma, A, m, k, lda, BM);
  if (e != cudaSuccess) return e;
  e = make_map(t, &mb, B, n, k, ldb, BN);
  if (e != cudaSuccess) return e;
  if (BLO) {
    e = make_map(t, &mbl, Blo, n, k, ldb, BN);
    if (e != cudaSuccess) return e;
  } else {
    mbl = mb;
  }
  GemmWork wk;
  wk.ktiles_total = (k + BK - 1) / BK;
  wk.ktiles_per_split = (wk.ktiles_total + ksplit - 1) / ksplit;
  wk.kc = kGemmChunkTiles;
  wk.mt = (m + BM - 1) / BM;
  wk.nt = (n + BN - 1) / BN;
  const long items = (long)wk.mt * wk.nt * ksplit;
  if (items > (1L << 30)) return cudaErrorInvalidConfiguration;
  wk.items = (int)items;
  const int grid = wk.items < t->num_sms ? wk.items : t->num_sms;
  tc_gemm_kernel<BN, SPLIT3, BLO><<<grid, Cfg::THREADS, Cfg::SMEM, st>>>(
      ma, mb, mbl, m, n, wk, C, ldc, alpha, beta, R, ldr, split_stride, status, Clo,
      out_bf16 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace

cudaError_t tc_create(TcCtx** out) {
  *out = nullptr;
  TcCtx* t = new TcCtx();
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled",
                                                   (void**)&t->encode, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !t->encode) {
    delete t;
    cudaGetLastError();
    return e != cudaSuccess ? e : cudaErrorNotSupported;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&t->num_sms, cudaDevAttrMultiProcessorCount, dev);
  *out = t;
  return cudaSuccess;
}

void tc_destroy(TcCtx* t) { delete t; }

cudaError_t tc_gemm(TcCtx* t, cudaStream_t st, int m, int n, int k, const float* A, long lda,
                    const float* B, long ldb, float* C, long ldc, float alpha, float beta,
                    const float* R, long ldr, bool split3, int ksplit, long split_stride,
                    int* status, int bn, const float* Blo, float* Clo, bool out_bf16) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (ksplit < 1 || (ksplit > 1 && (R || beta != 0.f))) return cudaErrorInvalidValue;
  if (Clo && ksplit != 1) return cudaErrorInvalidValue;
  if (out_bf16 && (!Clo || R)) return cudaErrorInvalidValue;
  if (bn != 0 && bn != 64 && bn != 128) return cudaErrorInvalidValue;
  if (Blo && !split3) return cudaErrorInvalidValue;
  if (bn == 0) bn = n <= 64 ? 64 : 128;
#define AFQMC_GEMM(BNV, S3, BL)                                                            \
  return launch_gemm<BNV, S3, BL>(t, st, m, n, k, A, lda, B, Blo, ldb, C, ldc, alpha, beta, \
                                  R, ldr, ksplit, split_stride, status, Clo, out_bf16)
  if (bn == 64) {
    if (!split3) AFQMC_GEMM(64, false, false);
    if (Blo) AFQMC_GEMM(64, true, true);
    AFQMC_GEMM(64, true, false);
  }
  if (!split3) AFQMC_GEMM(128, false, false);
  if (Blo) AFQMC_GEMM(128, true, true);
  AFQMC_GEMM(128, true, false);
#undef AFQMC_GEMM
}

// hi (in place, x rounded to TF32) and lo = (x - hi) rounded to TF32.
__global__ void tf32_split_kernel(long n, float* __restrict__ x, float* __restrict__ lo) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float v = x[e], h = tf32_hi(v);
  x[e] = h;
  lo[e] = tf32_lo(v, h);
}

// BF16 hi and lo parts of n FP64 values (setup).
__global__ void bf16_split_f64_kernel(long n, const double* __restrict__ x,
                                      uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  uint16_t h, l;
  bf16_split((float)x[e], h, l);
  hi[e] = h;
  lo[e] = l;
}

cudaError_t tc_split_bf16(cudaStream_t st, long n, const double* x, void* hi, void* lo) {
  if (n <= 0) return cudaSuccess;
  bf16_split_f64_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, (uint16_t*)hi,
                                                                    (uint16_t*)lo);
  return cudaGetLastError();
}

// Self-test of the bounded pipeline wait: one thread initialises an mbarrier
// that nothing ever arrives at and waits on it with the limit given; the
// wait gives up and bit 4 of *status is set, as a timed-out pipeline wait in
// the GEMM and Taylor kernels does. No copy or MMA is issued.
__global__ void wait_timeout_probe_kernel(long long limit_cycles, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(smem_u32(&bar), 1);
  mbar_fence_init();
  if (!mbar_wait(smem_u32(&bar), 0, limit_cycles)) flag_timeout(status);
}

cudaError_t tc_wait_timeout_probe(cudaStream_t st, long long limit_cycles, int* status) {
  wait_timeout_probe_kernel<<<1, 32, 0, st>>>(limit_cycles, status);
  return cudaGetLastError();
}

cudaError_t tc_split(cudaStream_t st, long n, float* x, float* lo) {
  if (n <= 0) return cudaSuccess;
  tf32_split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, lo);
  return cudaGetLastError();
}

cudaError_t tc_taylor(TcCtx* t, cudaStream_t st, int W, int M, int N, int order,
                      const float* V, const float* Pin, float* Pout, const void* bhalf_img,
                      bool split3, bool bf16, int* status) {
  if (M > 64 || M < 1 || N < 1) return cudaErrorInvalidValue;
  if (bhalf_img && ((uintptr_t)bhalf_img & 15)) return cudaErrorInvalidValue;
  const int items = W * ((N + 63) / 64);
  if (bf16) {
    const cudaError_t attr = set_smem(tc_taylor_bf16_kernel, TB_SMEM);
    if (attr != cudaSuccess) return attr;
    int grid = items < 2 * t->num_sms ? items : 2 * t->num_sms;
    tc_taylor_bf16_kernel<<<grid, 128, TB_SMEM, st>>>(W, M, N, order, V, Pin, Pout,
                                                      (const uint16_t*)bhalf_img, status);
    return cudaGetLastError();
  }
  if (split3) {
    const cudaError_t attr = set_smem(tc_taylor_kernel<true>, taylor_smem<true>());
    if (attr != cudaSuccess) return attr;
    int grid = items < t->num_sms ? items : t->num_sms;
    tc_taylor_kernel<true><<<grid, TY_THREADS, taylor_smem<true>(), st>>>(W, M, N, order, V, Pin,
                                                                  Pout, (const float*)bhalf_img,
                                                                  status);
  } else {
    const cudaError_t attr = set_smem(tc_taylor_kernel<false>, taylor_smem<false>());
    if (attr != cudaSuccess) return attr;
    int grid = items < t->num_sms ? items : t->num_sms;   // 256 threads of 152 registers
    tc_taylor_kernel<false><<<grid, TY_THREADS, taylor_smem<false>(), st>>>(W, M, N, order, V, Pin,
                                                                    Pout, (const float*)bhalf_img,
                                                                    status);
  }
  return cudaGetLastError();
}

cudaError_t tc_taylor_wide(TcCtx* t, cudaStream_t st, int W, int M, int N, int order, long ldV,
                           const void* V, const void* Vlo, const void* dB, const void* dBlo,
                           const float* Pin, float* Pout, bool split3, bool bf16, int* status) {
  if (M < 1 || M > 256 || N < 1 || W < 1 || order < 1 || ldV < M || (ldV & (bf16 ? 7 : 3)))
    return cudaErrorInvalidValue;
  if (bf16) split3 = true;
  if (split3 && (!Vlo || !dBlo)) return cudaErrorInvalidValue;
  const int kblk = bf16 ? 64 : 32;
  const int MT = (M + 127) / 128, KB = (M + kblk - 1) / kblk, P = split3 ? 2 : 1;
  const int stage = TW_TILE_BYTES * P;
  const int budget = 227 * 1024 - 1024 - 256;
  int n16 = ((N + 15) / 16) * 16;
  const int n16max = MT == 2 ? 32 : 64;
  if (n16 > n16max) n16 = n16max;
  while (n16 > 16 && KB * 2 * n16 * 128 * P + 3 * stage > budget) n16 -= 16;
  const int b = KB * 2 * n16 * 128 * P;
  int S = (budget - b) / stage;
  if (S > 8) S = 8;
  if (S < 2) return cudaErrorInvalidValue;
  const int smem = 1024 + b + S * stage + 256;
  CUtensorMap mv, mvl, mb, mbl;
  cudaError_t e = make_map3(t, &mv, V, M, M, ldV, 2L * W, bf16);
  if (e == cudaSuccess) e = make_map3(t, &mb, dB, M, M, ldV, 1, bf16);
  if (e == cudaSuccess && split3) e = make_map3(t, &mvl, Vlo, M, M, ldV, 2L * W, bf16);
  if (e == cudaSuccess && split3) e = make_map3(t, &mbl, dBlo, M, M, ldV, 1, bf16);
  if (e != cudaSuccess) return e;
  if (!split3) {
    mvl = mv;
    mbl = mb;
  }
  const long items = (long)W * ((N + n16 - 1) / n16);
  const int grid = items < t->num_sms ? (int)items : t->num_sms;
#define AFQMC_WIDE(S3, BF)                                                                 \
  do {                                                                                     \
    e = set_smem(tc_taylor_wide_kernel<S3, BF>, smem);                                     \
    if (e != cudaSuccess) return e;                                                        \
    tc_taylor_wide_kernel<S3, BF><<<grid, TW_THREADS, smem, st>>>(                         \
        mv, mvl, mb, mbl, W, M, N, order, n16, S, Pin, Pout, status);                      \
  } while (0)
  if (bf16) AFQMC_WIDE(true, true);
  else if (split3) AFQMC_WIDE(true, false);
  else AFQMC_WIDE(false, false);
#undef AFQMC_WIDE
  return cudaGetLastError();
}

size_t tc_bhalf_image_bytes(bool split3, bool bf16) {
  return bf16 ? (size_t)2 * TB_A_BYTES : (size_t)128 * 128 * 4 * (split3 ? 2 : 1);
}

cudaError_t tc_bhalf_image(cudaStream_t st, int M, const float* dB, void* img, bool split3,
                           bool bf16) {
  if (M > 64) return cudaErrorInvalidValue;
  if (bf16)
    bhalf_image_bf16_kernel<<<(128 * 128 + 255) / 256, 256, 0, st>>>(M, dB, (uint16_t*)img);
  else
    bhalf_image_kernel<<<(128 * 128 + 255) / 256, 256, 0, st>>>(M, dB, (float*)img,
                                                                split3 ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace afqmc
