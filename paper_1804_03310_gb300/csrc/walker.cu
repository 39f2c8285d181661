// Per-walker kernels of the ph-AFQMC step: field draw and force-bias shift
// (Sec. II, Eq. 2), Taylor propagation on the CUDA cores (Sec. II, Eq. 3),
// overlap / inverse / Theta (Sec. III), hybrid weight with the phaseless cut
// (Sec. II), the QR orthonormalisation (Sec. IV.A), the local-energy epilogue
// (Sec. III, Eq. 5), and the comb (Sec. V).
#include <float.h>

#include <algorithm>

#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "kernels.h"

namespace afqmc {

size_t smem_optin(const void* kernel) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(kernel, dev);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int optin = 48 * 1024;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  size_t stat = 0;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) stat = fa.sharedSizeBytes;
  size_t dyn = (size_t)optin > stat ? (size_t)optin - stat : 0;
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) !=
      cudaSuccess) {
    const size_t def = 48 * 1024;
    dyn = def > stat ? def - stat : 0;   // the limit without an opt-in
  }
  cudaGetLastError();
  cache[key] = dyn;
  return dyn;
}

namespace {


__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}

// --------------------------------------------------------------- K1 + K3
// Arithmetic type of the field draw: FP64 on the FP64 path, FP32 on the
// reduced paths (the Philox words are the same; only the transform's
// precision differs). The per-walker sum of the importance exponent is
// reduced across the block in FP64.
template <typename T>
struct FieldMath { using type = float; };
template <>
struct FieldMath<double> { using type = double; };

template <typename T>
__global__ void fields_kernel(int n_chol, const T* __restrict__ X, long ldx, int nsplit,
                              long split_stride, double sqdt_d, double cap_d, uint32_t k0,
                              uint32_t k1, int run_id, const long long* __restrict__ ctr,
                              T* __restrict__ S, long ldS, T* __restrict__ xbar,
                              double2* __restrict__ lw, const double* __restrict__ lbar,
                              double2* __restrict__ lmf) {
  using C = typename FieldMath<T>::type;
  __shared__ double red[32];
  const int w = blockIdx.x;
  const uint32_t step = (uint32_t)ctr[0];
  const T* Xr = X + (2L * w) * ldx;
  const T* Xi = Xr + ldx;
  T* Sr = S + (2L * w) * ldS;
  T* Si = Sr + ldS;
  T* Br = xbar + (2L * w) * n_chol;
  T* Bi = Br + n_chol;
  const C sqdt = (C)sqdt_d, cap = (C)cap_d;
  C lre = 0, lim = 0;
  double mre = 0.0, mim = 0.0;   // mean-field scalar, FP64
  const int nq = (n_chol + 3) >> 2;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    // X summed over the K-split partials, in order; the loads are issued
    // before the draw so that their latency overlaps the Philox rounds
    C xr[4] = {0, 0, 0, 0}, xi[4] = {0, 0, 0, 0};
    for (int sp = 0; sp < nsplit; ++sp) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int g = 4 * q + j;
        if (g < n_chol) {
          xr[j] += (C)Xr[sp * split_stride + g];
          xi[j] += (C)Xi[sp * split_stride + g];
        }
      }
    }
    U4 c = {(uint32_t)q, (uint32_t)w, step, (uint32_t)(4 * run_id + kStreamFields)};
    U4 r = philox4x32_10(c, k0, k1);
    C z[4];
    if (sizeof(C) == 8) {
      double a0, a1, a2, a3;
      box_muller(r.x, r.y, a0, a1);
      box_muller(r.z, r.w, a2, a3);
      z[0] = (C)a0; z[1] = (C)a1; z[2] = (C)a2; z[3] = (C)a3;
    } else {
      float a0, a1, a2, a3;
      box_muller_f(r.x, r.y, a0, a1);
      box_muller_f(r.z, r.w, a2, a3);
      z[0] = (C)a0; z[1] = (C)a1; z[2] = (C)a2; z[3] = (C)a3;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int g = 4 * q + j;
      if (g >= n_chol) break;
      // xbar = -i sqrt(dt) X, or -i sqrt(dt) (X - lbar) with the mean field
      // subtracted (lbar real, so only the imaginary part moves)
      const C xre = lbar ? (C)((double)xr[j] - lbar[g]) : xr[j];
      C br = sqdt * xi[j];
      C bi = -sqdt * xre;
      if (!isfinite(br) || !isfinite(bi)) { br = 0; bi = 0; }
      if (cap > 0) {
        const C a = sqrt(br * br + bi * bi);
        if (a > cap) { const C f = cap / a; br *= f; bi *= f; }
      }
      const C x = z[j];
      const C sr = x - br, si = -bi;          // s = x - xbar
      Sr[g] = (T)(-sqdt * si);               // i sqrt(dt) s
      Si[g] = (T)(sqdt * sr);
      Br[g] = (T)br;
      Bi[g] = (T)bi;
      lre += x * br - C(0.5) * (br * br - bi * bi);
      lim += x * bi - br * bi;
      if (lbar) {   // -i sqrt(dt) (x - xbar) lbar
        mre += sqdt_d * (double)si * lbar[g];
        mim -= sqdt_d * (double)sr * lbar[g];
      }
    }
  }
  const double tre = block_sum((double)lre, red);
  const double tim = block_sum((double)lim, red);
  if (threadIdx.x == 0) lw[w] = make_double2(tre, tim);
  if (lbar) {   // uniform over the block
    const double mr = block_sum(mre, red);
    const double mi = block_sum(mim, red);
    if (threadIdx.x == 0) lmf[w] = make_double2(mr, mi);
  }
}

// Complex value of the elimination's compute type R (double or float).
template <typename R>
struct __align__(2 * sizeof(R)) cx {
  R x, y;
};
template <typename R>
__device__ __forceinline__ cx<R> mk(R a, R b) { cx<R> r; r.x = a; r.y = b; return r; }
template <typename R>
__device__ __forceinline__ cx<R> sub_mul(cx<R> a, cx<R> f, cx<R> b) {   // a - f b
  return mk<R>(a.x - (f.x * b.x - f.y * b.y), a.y - (f.x * b.y + f.y * b.x));
}

template <typename R>
__device__ __forceinline__ cx<R> mul_c(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// --------------------------------------------------------------- K5 (SIMT, tiled)
// Asynchronous global -> shared copy of one element (4 or 8 bytes).
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* sdst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gsrc), "n"(BYTES)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

constexpr int kTayKC = 16;           // rows of V per shared-memory chunk
constexpr int kTayMaxThreads = 512;

// Per walker and chunk of NC orbital columns: t_0 = Phi, t_n = V t_{n-1} / n,
// out = sum_n t_n (Sec. II). One thread owns a TR x 4 tile of the M x NC
// output (rows nr apart, columns nc4 apart) for the whole series: the term's
// accumulator and the running sum stay in registers. V (complex symmetric, so
// row k of V is column k) streams through two shared chunks of kTayKC rows
// with cp.async, the next chunk in flight while the current one is used;
// the terms alternate between two shared buffers.
template <typename T, int TR>
__global__ void __launch_bounds__(kTayMaxThreads)
taylor_tiled_kernel(int M, int N, int NC, int order, const T* __restrict__ V, long ldv,
                    const T* __restrict__ Pin, T* __restrict__ Pout) {
  extern __shared__ unsigned char smem_raw[];
  const int ldt = M | 1;
  cx<T>* tb0 = reinterpret_cast<cx<T>*>(smem_raw);    // [NC][ldt]
  cx<T>* tb1 = tb0 + (long)NC * ldt;                  // [NC][ldt]
  T* vbuf = reinterpret_cast<T*>(tb1 + (long)NC * ldt);   // [2 buffers][2 planes][KC][M]
  const int w = blockIdx.x;
  const int j0 = blockIdx.y * NC;
  const int nc = min(NC, N - j0);
  const T* Vw = V + (long)w * 2 * M * ldv;
  const T* Pw = Pin + ((long)w * N + j0) * 2 * M;
  T* Ow = Pout + ((long)w * N + j0) * 2 * M;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nr = (M + TR - 1) / TR, nc4 = (nc + 3) >> 2;
  const bool owner = tid < nr * nc4;
  const int rt = owner ? tid % nr : 0, ct = owner ? tid / nr : 0;
  int rr[TR], cc[4];
#pragma unroll
  for (int u = 0; u < TR; ++u) rr[u] = min(rt + u * nr, M - 1);
#pragma unroll
  for (int v = 0; v < 4; ++v) cc[v] = min(ct + v * nc4, nc - 1);
  const int nchunk = (M + kTayKC - 1) / kTayKC;
  const int total = order * nchunk;
  // copy chunk q % nchunk of V into buffer q & 1 (this thread's share)
  const int per = kTayKC * M;
  auto issue = [&](int q) {
    const int k0 = (q % nchunk) * kTayKC;
    const int kc = min(kTayKC, M - k0);
    T* dst = vbuf + (long)(q & 1) * 2 * per;
    for (int e = tid; e < kc * M; e += nt) {
      const int rk = e / M, ck = e - rk * M;          // V symmetric: rows stand for columns
      const long src = (long)(k0 + rk) * ldv + ck;
      cp_async_elem<sizeof(T)>(dst + e, Vw + src);
      cp_async_elem<sizeof(T)>(dst + per + e, Vw + (long)M * ldv + src);
    }
    cp_async_commit();
  };
  issue(0);
  for (int e = tid; e < nc * 2 * M; e += nt) {        // t_0 from Phi
    const int j = e / (2 * M), r = e - j * 2 * M;
    reinterpret_cast<T*>(&tb0[j * ldt + (r < M ? r : r - M)])[r < M ? 0 : 1] = Pw[e];
  }
  __syncthreads();
  T sr[TR][4], si[TR][4], ar[TR][4], ai[TR][4];
#pragma unroll
  for (int u = 0; u < TR; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const cx<T> x = tb0[cc[v] * ldt + rr[u]];
      sr[u][v] = x.x; si[u][v] = x.y;
      ar[u][v] = T(0); ai[u][v] = T(0);
    }
  cx<T>* tin = tb0;
  cx<T>* tout = tb1;
  for (int q = 0; q < total; ++q) {
    if (q + 1 < total) {
      issue(q + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();                                  // chunk q and the last term are visible
    const int k0 = (q % nchunk) * kTayKC;
    const int kc = min(kTayKC, M - k0);
    const T* vr = vbuf + (long)(q & 1) * 2 * per;
    const T* vi = vr + per;
    if (owner) {
      for (int kk = 0; kk < kc; ++kk) {
        T qr[TR], qi[TR];
        cx<T> x[4];
#pragma unroll
        for (int u = 0; u < TR; ++u) { qr[u] = vr[kk * M + rr[u]]; qi[u] = vi[kk * M + rr[u]]; }
#pragma unroll
        for (int v = 0; v < 4; ++v) x[v] = tin[cc[v] * ldt + k0 + kk];
#pragma unroll
        for (int u = 0; u < TR; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            ar[u][v] = fma(qr[u], x[v].x, fma(-qi[u], x[v].y, ar[u][v]));
            ai[u][v] = fma(qr[u], x[v].y, fma(qi[u], x[v].x, ai[u][v]));
          }
      }
    }
    if (q % nchunk == nchunk - 1) {                   // term n = q / nchunk + 1 complete
      const T inv_n = T(1) / T(q / nchunk + 1);
      if (owner) {
#pragma unroll
        for (int u = 0; u < TR; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const T xr = ar[u][v] * inv_n, xi = ai[u][v] * inv_n;
            sr[u][v] += xr;
            si[u][v] += xi;
            ar[u][v] = T(0);
            ai[u][v] = T(0);
            tout[cc[v] * ldt + rr[u]] = mk<T>(xr, xi);
          }
      }
      cx<T>* t = tin;
      tin = tout;
      tout = t;
    }
    __syncthreads();                                  // buffer q & 1 free for chunk q + 2
  }
  if (owner) {
#pragma unroll
    for (int u = 0; u < TR; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int r = rt + u * nr, j = ct + v * nc4;
        if (r < M && j < nc) {
          Ow[(long)j * 2 * M + r] = sr[u][v];
          Ow[(long)j * 2 * M + M + r] = si[u][v];
        }
      }
  }
}

// --------------------------------------------------------------- K6

// Row stride (in complex values) of a walker block staged as [column][row]:
// odd, so that lanes reading the same row of consecutive columns hit
// distinct banks.
__host__ __device__ __forceinline__ int staged_ld(int M) { return M | 1; }

// Stage the ns orbital columns of one walker's spin block (2M values each:
// the real plane, then the imaginary plane) as complex Q[b][k]. Thread r
// takes plane row r of every column, with kStageU independent loads in
// flight before their stores, so that a block pays a few memory latencies
// instead of one per column.
constexpr int kStageU = 8;
template <typename T, typename R>
__device__ __forceinline__ void stage_columns(const T* __restrict__ Pw, int M, int ns, int ldq,
                                              cx<R>* __restrict__ Q) {
  for (int r = threadIdx.x; r < 2 * M; r += blockDim.x) {
    const int k = r < M ? r : r - M;
    const int part = r < M ? 0 : 1;
    for (int b0 = 0; b0 < ns; b0 += kStageU) {
      T v[kStageU];
#pragma unroll
      for (int u = 0; u < kStageU; ++u)
        v[u] = (b0 + u < ns) ? Pw[(long)(b0 + u) * 2 * M + r] : T(0);
#pragma unroll
      for (int u = 0; u < kStageU; ++u)
        if (b0 + u < ns) reinterpret_cast<R*>(&Q[(b0 + u) * ldq + k])[part] = (R)v[u];
    }
  }
}

// Y = Phi X for one staged walker block: Phi is M x ns with column b at
// Q[b * ldq], X is ns x ns row-major with row stride ldx; store(r, c, y) gets
// every Y_rc. Each thread accumulates a TR x 4 tile whose rows are nr apart
// and whose columns are nc apart, so that the lanes of a warp read
// consecutive rows of Phi (conflict-free) and a few broadcast entries of X.
template <int TR, typename R, typename F>
__device__ __forceinline__ void block_phi_times(int M, int ns, const cx<R>* __restrict__ Q,
                                                int ldq, const cx<R>* __restrict__ X, int ldx,
                                                F store) {
  const int nr = (M + TR - 1) / TR, nc = (ns + 3) >> 2;
  for (int it = threadIdx.x; it < nr * nc; it += blockDim.x) {
    const int rt = it % nr, ct = it / nr;
    int rr[TR], cc[4];
#pragma unroll
    for (int u = 0; u < TR; ++u) rr[u] = min(rt + u * nr, M - 1);
#pragma unroll
    for (int v = 0; v < 4; ++v) cc[v] = min(ct + v * nc, ns - 1);
    R yr[TR][4], yi[TR][4];
#pragma unroll
    for (int u = 0; u < TR; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) { yr[u][v] = R(0); yi[u][v] = R(0); }
    for (int i = 0; i < ns; ++i) {
      cx<R> q[TR], x[4];
#pragma unroll
      for (int u = 0; u < TR; ++u) q[u] = Q[i * ldq + rr[u]];
#pragma unroll
      for (int v = 0; v < 4; ++v) x[v] = X[i * ldx + cc[v]];
#pragma unroll
      for (int u = 0; u < TR; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          yr[u][v] = fma(q[u].x, x[v].x, fma(-q[u].y, x[v].y, yr[u][v]));
          yi[u][v] = fma(q[u].x, x[v].y, fma(q[u].y, x[v].x, yi[u][v]));
        }
    }
#pragma unroll
    for (int u = 0; u < TR; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (rt + u * nr < M && ct + v * nc < ns)
          store(rt + u * nr, ct + v * nc, mk<R>(yr[u][v], yi[u][v]));
  }
}

// Shared-memory bytes of one overlap block: the staged walker columns, two
// ns x ns elimination buffers (the second shares its space with the staged
// trial rows), the pivots and the row permutation.
__host__ __device__ __forceinline__ size_t overlap_region(int M, int ns) {
  const size_t a = (size_t)ns * (ns | 1), d = ((size_t)ns * staged_ld(M) + 1) / 2;
  return a > d ? a : d;
}

// One block per (walker, spin), with the walker's columns of that spin
// staged in shared memory as Q[b][k] (orbital column b, basis row k).
//  1. A = D^T Phi (real trial orbitals), ns x ns.
//  2. Gauss-Jordan elimination with partial pivoting gives (P A)^-1 and the
//     pivots, which are the diagonal of the U in P A = L U; the
//     log-determinant sum_k ln U_kk (+ i pi per odd row-swap count) is
//     accumulated in FP64. Up to 32 electrons per spin one warp eliminates
//     in place with no block barrier (one row per lane, rows left where
//     they are and the pivot order recorded). Above that, all warps share
//     each step: step k reads one buffer and writes the other, so it needs a
//     single block barrier, and the warp that owns column k + 1 picks the
//     next pivot from the values it has just written.
//  3. Theta = Phi A^-1 = (Phi (P A)^-1) P: a block product scattered to the
//     permuted columns. A^-1 itself (for the multi-determinant ratios) is
//     (P A)^-1 with the same column permutation.
template <typename T, typename R, int NT>
__global__ void __launch_bounds__(NT, sizeof(R) == 4 ? (NT == 128 ? 7 : 3) : 1)
overlap_kernel(int M, int n_up, int n_dn, const T* __restrict__ Phi,
                               const T* __restrict__ PsiT, T* __restrict__ Theta,
                               long ldt, long dn_off, double2* __restrict__ logdet,
                               double2* __restrict__ Ainv_out, int nmax) {
  extern __shared__ unsigned char smem_raw[];
  const int w = blockIdx.x, sig = blockIdx.y;
  const int N = n_up + n_dn;
  const int ns = sig ? n_dn : n_up;
  const int j0 = sig ? n_up : 0;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (ns == 0) {
    if (tid == 0) logdet[2 * w + sig] = make_double2(0.0, 0.0);
    return;
  }
  const int ldq = staged_ld(M), lda = ns | 1;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  cx<R>* Q = reinterpret_cast<cx<R>*>(smem_raw);      // [ns][ldq]
  cx<R>* A0 = Q + (long)ns * ldq;                     // [ns][lda]
  cx<R>* A1 = A0 + (long)ns * lda;                    // [ns][lda]
  R* D = reinterpret_cast<R*>(A1);                    // [ns][ldq] trial rows, until step 0
  cx<R>* pvs = A1 + overlap_region(M, ns);            // [ns] pivots
  int* perm = reinterpret_cast<int*>(pvs + ns);       // [ns]
  __shared__ int piv[2], singular, nswap;
  __shared__ cx<R> ipv_s[2];                          // 1 / pivot of the next step
  // lane 0 of the warp that found pivot row bi of column col publishes it
  auto publish = [&](const cx<R>* buf, int col, int bi, R best) {
    if (lane == 0) {
      piv[col & 1] = bi;
      if (!(best > R(0))) {
        singular = 1;
      } else {
        const cx<R> pv = buf[bi * lda + col];
        const R pd = pv.x * pv.x + pv.y * pv.y;
        pvs[col] = pv;
        ipv_s[col & 1] = mk<R>(pv.x / pd, -pv.y / pd);
      }
    }
  };
  const T* Pw = Phi + ((long)w * N + j0) * 2 * M;
  stage_columns<T, R>(Pw, M, ns, ldq, Q);
  for (int k = tid; k < M; k += nt) {                 // trial rows, kStageU loads in flight
    for (int b0 = 0; b0 < ns; b0 += kStageU) {
      T v[kStageU];
#pragma unroll
      for (int u = 0; u < kStageU; ++u)
        v[u] = (b0 + u < ns) ? PsiT[(long)(j0 + b0 + u) * M + k] : T(0);
#pragma unroll
      for (int u = 0; u < kStageU; ++u)
        if (b0 + u < ns) D[(b0 + u) * ldq + k] = (R)v[u];
    }
  }
  if (tid == 0) { nswap = 0; singular = 0; }
  for (int i = tid; i < ns; i += nt) perm[i] = i;
  __syncthreads();
  {                                                   // A = D^T Phi, 2 x 4 tiles
    const int na = (ns + 1) >> 1, nb = (ns + 3) >> 2;
    for (int it = tid; it < na * nb; it += nt) {
      const int ag = it % na, bg = it / na;
      const int a0 = 2 * ag, b0 = 4 * bg;
      const int a1 = min(a0 + 1, ns - 1);
      int bb[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) bb[v] = min(b0 + v, ns - 1);
      R sr[2][4], si[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) { sr[u][v] = R(0); si[u][v] = R(0); }
      for (int k = 0; k < M; ++k) {
        const R d0 = D[a0 * ldq + k], d1 = D[a1 * ldq + k];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const cx<R> q = Q[bb[v] * ldq + k];
          sr[0][v] = fma(d0, q.x, sr[0][v]);
          si[0][v] = fma(d0, q.y, si[0][v]);
          sr[1][v] = fma(d1, q.x, sr[1][v]);
          si[1][v] = fma(d1, q.y, si[1][v]);
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (a0 + u < ns && b0 + v < ns) A0[(a0 + u) * lda + b0 + v] = mk<R>(sr[u][v], si[u][v]);
    }
  }
  __syncthreads();
  cx<R>* cur = A0;
  if (ns <= 32) {
    // One warp eliminates in place, lane i owning row i, with no block
    // barrier: the pivot of column k is the largest |a_ik|^2 among the rows
    // not yet used as pivots (ties to the lower row); every other row i
    // subtracts f_i = a_ik / pivot times the pivot row and keeps -f_i in
    // column k, then the pivot row is scaled by 1 / pivot (1 / pivot in
    // column k). Row p_k (the pivot row of step k) then holds row k of
    // (P A)^-1, where row k of P A is row p_k of A; the pivots are the same
    // U_kk as those of the row-swapping elimination, so ln det A = sum ln U_kk
    // plus i pi when the permutation k -> p_k is odd.
    if (warp == 0) {
      const bool mine = lane < ns;
      cx<R>* arow = A0 + (mine ? lane : 0) * lda;
      bool used = !mine, sing_w = false;
      for (int k = 0; k < ns; ++k) {
        R best = R(-1);
        if (!used) {
          const cx<R> v = arow[k];
          const R m = v.x * v.x + v.y * v.y;
          if (m > best) best = m;                      // a NaN stays out
        }
        int bi = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const R ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > R(0))) {                          // uniform over the warp
          if (lane == 0) singular = 1;
          sing_w = true;
          break;
        }
        const int p = bi;
        const cx<R>* prow = A0 + p * lda;
        const cx<R> pv = prow[k];
        const R pd = pv.x * pv.x + pv.y * pv.y;
        const cx<R> ipv = mk<R>(pv.x / pd, -pv.y / pd);
        if (lane == 0) {
          pvs[k] = pv;
          perm[k] = p;
        }
        if (mine && lane != p) {                       // reads row p, writes row i
          const cx<R> f = mul_c(arow[k], ipv);
          for (int j = 0; j < ns; ++j) arow[j] = sub_mul(arow[j], f, prow[j]);
          arow[k] = mk<R>(-f.x, -f.y);
        }
        __syncwarp();
        if (mine) {                                    // the pivot row, element j = lane
          const cx<R> v = A0[p * lda + lane];
          A0[p * lda + lane] = lane == k ? ipv : mul_c(v, ipv);
        }
        if (lane == p) used = true;
        __syncwarp();
      }
      if (!sing_w) {                                   // parity of k -> p_k by inversions
        int inv = 0;
        if (mine)
          for (int j = lane + 1; j < ns; ++j) inv += perm[j] < perm[lane] ? 1 : 0;
        inv = warp_sum(inv);
        if (lane == 0) nswap = inv & 1;
      }
    }
    __syncthreads();
    if (!singular) {                                   // (P A)^-1 row k = row p_k
      for (int e = tid; e < ns * ns; e += nt) {
        const int k = e / ns, j = e - k * ns;
        A1[k * lda + j] = A0[perm[k] * lda + j];
      }
      cur = A1;
    }
    __syncthreads();
  } else {
    if (warp == 0) {                                    // first pivot: column 0
      R best = R(-1);
      int bi = 0;
      for (int i = lane; i < ns; i += 32) {
        const cx<R> v = A0[i * lda];
        const R m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      publish(A0, 0, bi, best);
    }
    __syncthreads();
    cx<R>* nxt = A1;
    if (!singular) {
      for (int k = 0; k < ns; ++k) {
        const int p = piv[k & 1];
        const cx<R>* prow = cur + p * lda;
        const cx<R> ipv = ipv_s[k & 1];
        if (tid == 0) {
          if (p != k) {
            const int t = perm[k];
            perm[k] = perm[p];
            perm[p] = t;
            nswap ^= 1;
          }
        }
        // rows k and p trade places: row i of the result comes from row src(i)
        // (the new pivot row k is row p scaled: p - (1 - 1/pv) p, one formula for all rows)
        for (int i = lane; i < ns; i += 32) {
          const cx<R>* irow = cur + (i == k ? p : (i == p ? k : i)) * lda;
          cx<R> f, colk;
          if (i == k) {
            f = mk<R>(R(1) - ipv.x, -ipv.y);
            colk = ipv;
          } else {
            f = mul_c(irow[k], ipv);
            colk = mk<R>(-f.x, -f.y);
          }
          cx<R>* orow = nxt + i * lda;
          for (int j = warp; j < ns; j += nwarps)
            orow[j] = (j == k) ? colk : sub_mul(irow[j], f, prow[j]);
        }
        const int jn = k + 1;
        if (jn < ns && jn % nwarps == warp) {           // next pivot, from this warp's own writes
          R best = R(-1);
          int bi = jn;
          for (int i = lane; i < ns; i += 32) {
            if (i < jn) continue;
            const cx<R> v = nxt[i * lda + jn];
            const R m = v.x * v.x + v.y * v.y;
            if (m > best) { best = m; bi = i; }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const R ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          __syncwarp();                                  // the lanes' writes of column jn
          publish(nxt, jn, bi, best);
        }
        __syncthreads();
        cx<R>* t = cur;
        cur = nxt;
        nxt = t;
        if (singular) break;
      }
    }
  }
  const int sing = singular;
  if (tid < 32) {
    double lre = 0.0, lim = 0.0;
    if (!sing) {
      for (int k = tid; k < ns; k += 32) {
        const double px = (double)pvs[k].x, py = (double)pvs[k].y;
        lre += 0.5 * log(px * px + py * py);
        lim += atan2(py, px);
      }
    }
    lre = warp_sum(lre);
    lim = warp_sum(lim);
    if (tid == 0) {
      double2 out = make_double2(lre, lim);
      if (sing) out = make_double2(-INFINITY, 0.0);
      else if (nswap) out.y += 3.141592653589793;
      logdet[2 * w + sig] = out;
    }
  }
  T* Tr = Theta + ((long)w * 2 + 0) * ldt + (sig ? dn_off : 0);
  T* Ti = Theta + ((long)w * 2 + 1) * ldt + (sig ? dn_off : 0);
  if (sing) {
    for (int e = tid; e < ns * M; e += nt) {
      Tr[e] = T(0);
      Ti[e] = T(0);
    }
  } else {
    block_phi_times<2>(M, ns, Q, ldq, cur, lda, [&](int r, int c, cx<R> y) {
      const long o = (long)perm[c] * M + r;
      Tr[o] = (T)y.x;
      Ti[o] = (T)y.y;
    });
  }
  if (Ainv_out) {                                     // A^-1 [r][perm[i]] = (P A)^-1 [r][i]
    double2* Ao = Ainv_out + ((long)w * 2 + sig) * nmax * nmax;
    for (int e = tid; e < ns * ns; e += nt) {
      const int r = e / ns, i = e - r * ns;
      const cx<R> y = sing ? mk<R>(R(0), R(0)) : cur[r * lda + i];
      Ao[(long)r * nmax + (sing ? i : perm[i])] = make_double2((double)y.x, (double)y.y);
    }
  }
}

__global__ void logdet_sum_kernel(int W, const double2* __restrict__ ld,
                                  double2* __restrict__ out) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  out[w] = cadd(ld[2 * w], ld[2 * w + 1]);
}

// --------------------------------------------------------------- K7
// Hybrid form: ln|I| = Re(ln R + lmf) + Re(lw) + dtau e_shift (e_shift
// already holding E_T - E_0); local-energy form (eloc given): ln|I| =
// -dtau (Re E_L - e_shift). Both cut by max(0, cos Im(ln R + lmf)).
__global__ void weights_kernel(int W, const double2* __restrict__ logO_new,
                               const double2* __restrict__ logdet,
                               const double2* __restrict__ lw,
                               const double2* __restrict__ lmf,
                               const double2* __restrict__ eloc, double dtau,
                               double e_shift, double cap, const double* __restrict__ wref,
                               double* __restrict__ weight,
                               double2* __restrict__ logO, long long* __restrict__ ctr) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w == 0) ctr[0] += 1;   // the step is complete once its weights are
  if (w >= W) return;
  const double2 ln = logO_new ? logO_new[w] : cadd(logdet[2 * w], logdet[2 * w + 1]);
  double2 lnR = csub(ln, logO[w]);
  if (lmf) lnR = cadd(lnR, lmf[w]);
  const double lnI_re =
      eloc ? -dtau * (eloc[w].x - e_shift) : lnR.x + lw[w].x + dtau * e_shift;
  double wt = weight[w];
  double out = 0.0;
  if (wt != 0.0) {
    out = wt * exp(lnI_re) * fmax(0.0, cos(lnR.y));
    if (!isfinite(out)) out = 0.0;
    if (cap > 0.0) {
      const double ref = *wref;
      if (ref > 0.0) out = fmin(out, cap * ref);
    }
  }
  weight[w] = out;
  logO[w] = ln;
}

// --------------------------------------------------------------- K10
// QR of each walker's spin block, Phi = Q R with R upper triangular and its
// diagonal real and positive (the factorisation modified Gram-Schmidt
// produces), computed through the Gram matrix: S = Phi^H Phi = R^H R
// (Cholesky), then Q = Phi R^-1 row by row. The route's loss of
// orthogonality grows with cond(Phi)^2; walkers re-orthonormalised every
// step or two stay close to orthonormal (cond(Phi) near 1), where it stays
// at the level of the arithmetic's own rounding (|Q^H Q - I| below 1e-5 in
// FP32 at the H-chain and TM-atom shapes with orthonormalisation every 2
// steps); a larger cadence calls for FP64 arithmetic here (fp64_islands).
// One block per (walker, spin); ln det R =
// sum_j ln R_jj is accumulated in FP64 into lr[w][spin].
template <typename T, typename R>
__global__ void qr_kernel(int M, int n_up, int n_dn, T* __restrict__ Phi,
                          double* __restrict__ lr) {
  extern __shared__ unsigned char smem_raw[];
  const int w = blockIdx.x, sig = blockIdx.y;
  const int N = n_up + n_dn;
  const int ns = sig ? n_dn : n_up;
  const int j0 = sig ? n_up : 0;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (ns == 0) {
    if (tid == 0) lr[2 * w + sig] = 0.0;
    return;
  }
  const int ldq = staged_ld(M);
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  cx<R>* Q = reinterpret_cast<cx<R>*>(smem_raw);      // [ns][ldq]
  cx<R>* S = Q + (long)ns * ldq;                      // [ns][ns], R in the upper part
  T* Pw = Phi + ((long)w * N + j0) * 2 * M;
  stage_columns<T, R>(Pw, M, ns, ldq, Q);
  __syncthreads();
  {                                                   // S_ab = q_a^H q_b, a <= b, 2 x 4 tiles
    const int na = (ns + 1) >> 1, nb = (ns + 3) >> 2;
    for (int it = tid; it < na * nb; it += nt) {
      const int ag = it % na, bg = it / na;
      const int a0 = 2 * ag, b0 = 4 * bg;
      if (a0 > b0 + 3) continue;                      // entirely below the diagonal
      const int a1 = min(a0 + 1, ns - 1);
      int bb[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) bb[v] = min(b0 + v, ns - 1);
      R sr[2][4], si[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) { sr[u][v] = R(0); si[u][v] = R(0); }
      for (int k = 0; k < M; ++k) {
        const cx<R> x0 = Q[a0 * ldq + k], x1 = Q[a1 * ldq + k];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const cx<R> y = Q[bb[v] * ldq + k];
          sr[0][v] = fma(x0.x, y.x, fma(x0.y, y.y, sr[0][v]));
          si[0][v] = fma(x0.x, y.y, fma(-x0.y, y.x, si[0][v]));
          sr[1][v] = fma(x1.x, y.x, fma(x1.y, y.y, sr[1][v]));
          si[1][v] = fma(x1.x, y.y, fma(-x1.y, y.x, si[1][v]));
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (a0 + u < ns && b0 + v < ns && a0 + u <= b0 + v)
            S[(a0 + u) * ns + b0 + v] = mk<R>(sr[u][v], si[u][v]);
    }
  }
  __syncthreads();
  for (int j = 0; j < ns; ++j) {                      // right-looking Cholesky
    const R d = sqrt(S[j * ns + j].x);
    __syncthreads();
    for (int c = j + tid; c < ns; c += nt) {
      const cx<R> v = S[j * ns + c];
      S[j * ns + c] = (c == j) ? mk<R>(d, R(0)) : mk<R>(v.x / d, v.y / d);
    }
    __syncthreads();
    // S_ac -= conj(R_ja) R_jc for j < a <= c; lane = column c, warp = rows a
    for (int c = j + 1 + lane; c < ns; c += 32) {
      const cx<R> y = S[j * ns + c];
      for (int a = j + 1 + warp; a <= c; a += nwarps) {
        const cx<R> x = S[j * ns + a];
        S[a * ns + c] = mk<R>(S[a * ns + c].x - (x.x * y.x + x.y * y.y),
                              S[a * ns + c].y - (x.x * y.y - x.y * y.x));
      }
    }
    __syncthreads();
  }
  for (int k = tid; k < M; k += nt) {                 // q_k R = phi_k (two partial sums)
    for (int j = 0; j < ns; ++j) {
      cx<R> s0 = Q[j * ldq + k], s1 = mk<R>(R(0), R(0));
      int i = 0;
      for (; i + 1 < j; i += 2) {
        s0 = sub_mul(s0, Q[i * ldq + k], S[i * ns + j]);
        s1 = sub_mul(s1, Q[(i + 1) * ldq + k], S[(i + 1) * ns + j]);
      }
      if (i < j) s0 = sub_mul(s0, Q[i * ldq + k], S[i * ns + j]);
      const R d = S[j * ns + j].x;
      Q[j * ldq + k] = mk<R>((s0.x + s1.x) / d, (s0.y + s1.y) / d);
    }
    for (int j = 0; j < ns; ++j) {
      const cx<R> q = Q[j * ldq + k];
      Pw[(long)j * 2 * M + k] = (T)q.x;
      Pw[(long)j * 2 * M + M + k] = (T)q.y;
    }
  }
  if (tid < 32) {
    double l = 0.0;
    for (int j = tid; j < ns; j += 32) l += log((double)S[j * ns + j].x);
    l = warp_sum(l);
    if (tid == 0) lr[2 * w + sig] = l;
  }
}

__global__ void sub_logdet_r_kernel(int W, const double* __restrict__ lr,
                                    double2* __restrict__ logO) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w < W) logO[w].x -= lr[2 * w] + lr[2 * w + 1];
}

// --------------------------------------------------------------- K9 epilogue
template <typename T>
__global__ void energy_reduce_kernel(int M, int n_up, int n_dn, int n_chol,
                                     const T* __restrict__ X, long ldx, int nsplit,
                                     long split_stride, const T* __restrict__ Theta,
                                     long ldt, long dn_off, const T* __restrict__ Z,
                                     long ldz_up, long ldz_dn, int W,
                                     double2* __restrict__ eloc) {
  __shared__ double red[32];
  const int w = blockIdx.x;
  const T* Xr = X + (2L * w) * ldx;
  const T* Xi = Xr + ldx;
  double cr = 0.0, ci = 0.0;
  for (int g = threadIdx.x; g <= n_chol; g += blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) {
      a += (double)Xr[sp * split_stride + g];
      b += (double)Xi[sp * split_stride + g];
    }
    if (g == n_chol) {          // the one-body column tr(h~ Theta)
      cr += a;
      ci += b;
    } else {
      cr += 0.5 * (a * a - b * b);
      ci += a * b;
    }
  }
  double er = 0.0, ei = 0.0;
  long zoff = 0;
  for (int sig = 0; sig < 2; ++sig) {
    const int ns = sig ? n_dn : n_up;
    const long J = (long)ns * M;
    const long ldz = sig ? ldz_dn : ldz_up;
    const T* tr = Theta + (2L * w) * ldt + (sig ? dn_off : 0);
    const T* ti = tr + ldt;
    const T* zr = Z + zoff + (2L * w) * ldz;
    const T* zi = zr + ldz;
    for (long e = threadIdx.x; e < J; e += blockDim.x) {
      double a = tr[e], b = ti[e], p = zr[e], q = zi[e];
      er += 0.5 * (a * p - b * q);
      ei += 0.5 * (a * q + b * p);
    }
    zoff += 2L * W * ldz;
  }
  double tr_ = block_sum(cr + er, red);
  double ti_ = block_sum(ci + ei, red);
  if (threadIdx.x == 0) eloc[w] = make_double2(tr_, ti_);
}

__global__ void mixed_energy_kernel(int W, const double* __restrict__ weight,
                                    const double2* __restrict__ eloc,
                                    long long* __restrict__ ctr, double2* __restrict__ hist,
                                    int hist_len, double* out_scalar) {
  __shared__ double red[32];
  double num = 0.0, den = 0.0;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    double wt = weight[w];
    if (wt > 0.0) {
      num += wt * eloc[w].x;
      den += wt;
    }
  }
  num = block_sum(num, red);
  den = block_sum(den, red);
  if (threadIdx.x == 0) {
    double e = den > 0.0 ? num / den : NAN;
    if (hist) {
      hist[ctr[1] % hist_len] = make_double2((double)ctr[0], e);
      ctr[1] += 1;
    }
    out_scalar[0] = e;
    out_scalar[1] = den;
  }
}

// --------------------------------------------------------------- K11
constexpr int kScanBlock = 32;

__global__ void comb_kernel(int W, const double* __restrict__ weight, uint32_t k0,
                            uint32_t k1, int run_id, const long long* __restrict__ ctr,
                            long long step_val,
                            int* __restrict__ parent, double* __restrict__ C,
                            double* __restrict__ wnew, int* __restrict__ status) {
  extern __shared__ unsigned char smem_raw[];
  double* tot = reinterpret_cast<double*>(smem_raw);   // [nb]
  double* base = tot + ((W + kScanBlock - 1) / kScanBlock);
  __shared__ double S_sh;
  __shared__ int last_sh;
  const int nb = (W + kScanBlock - 1) / kScanBlock;
  if (threadIdx.x == 0) last_sh = -1;
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    double run = 0.0;
    int last = -1;
    for (int k = b * kScanBlock; k < min(W, (b + 1) * kScanBlock); ++k) {
      double wk = weight[k];
      run = __dadd_rn(run, wk);
      C[k] = run;
      if (wk > 0.0) last = k;
    }
    tot[b] = run;
    if (last >= 0) atomicMax(&last_sh, last);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) {
      base[b] = s;
      s = __dadd_rn(s, tot[b]);
    }
    S_sh = s;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    for (int k = b * kScanBlock; k < min(W, (b + 1) * kScanBlock); ++k)
      C[k] = __dadd_rn(base[b], C[k]);
  __syncthreads();
  const double S = S_sh;
  if (!(S > 0.0) || !isfinite(S) || last_sh < 0) {
    for (int j = threadIdx.x; j < W; j += blockDim.x) parent[j] = j;
    if (threadIdx.x == 0) {
      atomicOr(status, 2);
      *wnew = -1.0;
    }
    return;
  }
  const uint32_t step = (uint32_t)(ctr ? ctr[0] : step_val);
  U4 c = {0u, 0u, step, (uint32_t)(4 * run_id + kStreamComb)};
  const double u = open01(philox4x32_10(c, k0, k1).x);
  const double stepw = __ddiv_rn(S, (double)W);
  for (int j = threadIdx.x; j < W; j += blockDim.x) {
    double t = __dmul_rn(__dadd_rn((double)j, u), stepw);
    int lo = 0, hi = W;                 // first index with C > t
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (C[mid] <= t) lo = mid + 1; else hi = mid;
    }
    parent[j] = lo < W ? lo : last_sh;
  }
  if (threadIdx.x == 0) *wnew = stepw;
}

template <typename T>
__global__ void gather_kernel(long phi_elems, long theta_elems,
                              const int* __restrict__ parent, const T* __restrict__ Phi,
                              T* __restrict__ Phi_out, const T* __restrict__ Theta,
                              T* __restrict__ Theta_out, const double2* __restrict__ logO,
                              double2* __restrict__ logO_out,
                              const double* __restrict__ wnew,
                              double* __restrict__ weight, double* __restrict__ wref,
                              double* __restrict__ log_scale) {
  const int j = blockIdx.x;
  const int p = parent[j];
  for (long e = threadIdx.x; e < phi_elems; e += blockDim.x)
    Phi_out[(long)j * phi_elems + e] = Phi[(long)p * phi_elems + e];
  for (long e = threadIdx.x; e < theta_elems; e += blockDim.x)
    Theta_out[(long)j * theta_elems + e] = Theta[(long)p * theta_elems + e];
  if (threadIdx.x == 0) {
    logO_out[j] = logO[p];
    // the common weight S/n is divided out: every walker restarts at 1 and
    // ln(S/n) goes to the log scale (block 0 alone writes the scalars)
    const double wn = *wnew;
    if (wn > 0.0) {
      weight[j] = 1.0;
      if (j == 0) {
        *wref = 1.0;
        *log_scale += log(wn);
      }
    }
  }
}

// --------------------------------------------------------------- setup
template <typename T>
__global__ void gather_rows_kernel(long elems, const int* __restrict__ parent,
                                   const T* __restrict__ in, T* __restrict__ out) {
  const int j = blockIdx.x;
  const int p = parent[j];
  for (long e = threadIdx.x; e < elems; e += blockDim.x)
    out[(long)j * elems + e] = in[(long)p * elems + e];
}

// H1' = h1 - 1/2 sum_g L_g L_g (+ sum_g lbar_g L_g with the mean field
// subtracted, lbar non-null).
__global__ void h1_remainder_kernel(int M, int n_chol, const double* __restrict__ h1,
                                    const double* __restrict__ L,
                                    const double* __restrict__ lbar,
                                    double* __restrict__ h1p) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  int i = e / M, j = e - i * M;
  double s = 0.0, m = 0.0;
  for (int g = 0; g < n_chol; ++g) {
    const double* Lg = L + (long)g * M * M;
    for (int k = 0; k < M; ++k) s = fma(Lg[i * M + k], Lg[k * M + j], s);
    if (lbar) m = fma(lbar[g], Lg[e], m);
  }
  h1p[e] = h1[e] - 0.5 * s + m;
}

__global__ void scale_identity_kernel(int M, const double* __restrict__ A, double s,
                                      double* __restrict__ Ip, double* __restrict__ As) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  int i = e / M, j = e - i * M;
  double a = A[e] * s;
  As[e] = a;
  Ip[e] = a + (i == j ? 1.0 : 0.0);
}

__global__ void yx_permute_kernel(int n, int M, const double* __restrict__ gram,
                                  double* __restrict__ yx, long ldy) {
  // Yx[(a,k)][(b,l)] = -Gram[(b,k)][(a,l)],  J = n * M
  long J = (long)n * M;
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= J * J) return;
  long row = e / J, col = e - row * J;
  int a = (int)(row / M), k = (int)(row - (long)a * M);
  int b = (int)(col / M), l = (int)(col - (long)b * M);
  yx[row * ldy + col] = -gram[((long)b * M + k) * J + (long)a * M + l];
}

// Rows of [rows][Jup + Jdn] into [rows][ld] with the down block at dn_off.
__global__ void pad_rows_kernel(long rows, long Jup, long Jdn, const double* __restrict__ in,
                                double* __restrict__ out, long ld, long dn_off) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long J = Jup + Jdn;
  if (e >= rows * J) return;
  long r = e / J, c = e - r * J;
  out[r * ld + (c < Jup ? c : dn_off + (c - Jup))] = in[e];
}

// L [G][M*M] -> out [M*ldv][ldo]: out[i ldv + k][g] = L[g][i M + k]; the
// rows i ldv + k with k >= M are left as they are (zero).
__global__ void transpose_pad_kernel(long G, int M, long ldv, const double* __restrict__ in,
                                     double* __restrict__ out, long ldo) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long MM = (long)M * M;
  if (e >= G * MM) return;
  const long g = e / MM, r = e - g * MM;
  const long i = r / M, k = r - i * M;
  out[(i * ldv + k) * ldo + g] = in[e];
}

// y[r] = sum_c A[r][c] x[c] (FP64, one block per row).
__global__ void gemv_rows_kernel(long cols, const double* __restrict__ A, long lda,
                                 const double* __restrict__ x, double* __restrict__ y) {
  __shared__ double red[256];
  const long r = blockIdx.x;
  double acc = 0.0;
  for (long c = threadIdx.x; c < cols; c += blockDim.x) acc += A[r * lda + c] * x[c];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) y[r] = red[0];
}

// y[c] = sum_r x[r] A[r][c] (FP64, one thread per column).
__global__ void gemv_cols_kernel(long rows, long cols, const double* __restrict__ A, long lda,
                                 const double* __restrict__ x, double* __restrict__ y) {
  const long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double acc = 0.0;
  for (long r = 0; r < rows; ++r) acc += x[r] * A[r * lda + c];
  y[c] = acc;
}

// out[i][j] = in[j][i] for an rows x cols matrix, into leading dimension ldo.
__global__ void transpose_kernel(long rows, long cols, const double* __restrict__ in,
                                 double* __restrict__ out, long ldo) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  long r = e / cols, c = e - r * cols;
  out[c * ldo + r] = in[e];
}

template <typename T>
__global__ void convert_kernel(long n, const double* __restrict__ in, T* __restrict__ out) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) out[e] = (T)in[e];
}

template <typename T>
__global__ void init_walkers_kernel(int M, int N, const T* __restrict__ PsiT,
                                    T* __restrict__ Phi, double* __restrict__ weight) {
  const int w = blockIdx.x;
  T* Pw = Phi + (long)w * N * 2 * M;
  for (int e = threadIdx.x; e < N * M; e += blockDim.x) {
    int j = e / M, k = e - j * M;
    Pw[(j * 2 + 0) * M + k] = PsiT[(long)j * M + k];
    Pw[(j * 2 + 1) * M + k] = T(0);
  }
  if (threadIdx.x == 0) weight[w] = 1.0;
}

__global__ void add_diag_kernel(int M, double* __restrict__ A, double a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) A[(long)i * M + i] += a;
}

__global__ void axpy_d_kernel(long n, double a, const double* __restrict__ x,
                              double* __restrict__ y) {
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) y[e] += a * x[e];
}

inline unsigned blocks_for(long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// =============================================================== launchers
template <typename T>
cudaError_t launch_fields(cudaStream_t st, int W, int n_chol, const T* X, long ldx,
                          int nsplit, long split_stride, double sqdt, double cap,
                          uint64_t seed, int run_id, const long long* ctr, T* S, long ldS,
                          T* xbar, double2* lw, const double* lbar, double2* lmf) {
  fields_kernel<T><<<W, 128, 0, st>>>(n_chol, X, ldx, nsplit, split_stride, sqdt, cap,
                                      (uint32_t)seed, (uint32_t)(seed >> 32), run_id, ctr,
                                      S, ldS, xbar, lw, lbar, lmf);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_taylor(cudaStream_t st, int W, int M, int N, int order,
                          const T* V, long ldv, const T* Phi_in, T* Phi_out) {
  constexpr int TR = sizeof(T) == 4 ? 4 : 2;
  const size_t cap = smem_optin((const void*)taylor_tiled_kernel<T, TR>);
  if (M < 1 || N < 1) return cudaErrorInvalidValue;
  const int nr = (M + TR - 1) / TR;
  const int ldt = M | 1;
  auto smem_for = [&](int nc) {
    return sizeof(T) * (4 * (size_t)nc * ldt + 4 * (size_t)kTayKC * M);
  };
  int ncmax = 4 * (kTayMaxThreads / nr);             // tiles within one block
  if (ncmax > N) ncmax = N;
  while (ncmax > 1 && smem_for(ncmax) > cap) --ncmax;
  if (ncmax < 1 || nr > kTayMaxThreads || smem_for(ncmax) > cap) return cudaErrorInvalidValue;
  const int pieces = (N + ncmax - 1) / ncmax;        // balanced column chunks
  const int NC = (N + pieces - 1) / pieces;
  const int tiles = nr * ((NC + 3) / 4);
  const int threads = (tiles + 31) / 32 * 32;
  dim3 grid(W, pieces);
  if (ldv < M) return cudaErrorInvalidValue;
  taylor_tiled_kernel<T, TR><<<grid, threads, smem_for(NC), st>>>(M, N, NC, order, V, ldv,
                                                                  Phi_in, Phi_out);
  return cudaGetLastError();
}

size_t overlap_smem(int M, int nmax, size_t csize) {
  return csize * ((size_t)nmax * staged_ld(M) + (size_t)nmax * (nmax | 1) +
                  overlap_region(M, nmax) + nmax) +
         sizeof(int) * nmax;
}

size_t qr_smem(int M, int nmax, size_t csize) {
  return csize * ((size_t)nmax * staged_ld(M) + (size_t)nmax * nmax);
}

template <typename T, typename R, int NT>
cudaError_t launch_overlap_nt(cudaStream_t st, int W, int M, int n_up, int n_dn,
                              const T* Phi, const T* PsiT, T* Theta, long ldt, long dn_off,
                              double2* logdet, double2* Ainv) {
  const int nmax = n_up > n_dn ? n_up : n_dn;
  const size_t cap = smem_optin((const void*)overlap_kernel<T, R, NT>);
  const size_t smem = overlap_smem(M, nmax, sizeof(cx<R>));
  if (smem > cap) return cudaErrorInvalidValue;
  overlap_kernel<T, R, NT><<<dim3(W, 2), NT, smem, st>>>(M, n_up, n_dn, Phi, PsiT, Theta, ldt,
                                                       dn_off, logdet, Ainv, nmax);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_overlap(cudaStream_t st, int W, int M, int n_up, int n_dn,
                           const T* Phi, const T* PsiT, T* Theta, long ldt, long dn_off,
                           double2* logdet, double2* Ainv, bool fp64_compute) {
  if (M > 96)
    return fp64_compute
               ? launch_overlap_nt<T, double, 256>(st, W, M, n_up, n_dn, Phi, PsiT, Theta, ldt,
                                                   dn_off, logdet, Ainv)
               : launch_overlap_nt<T, float, 256>(st, W, M, n_up, n_dn, Phi, PsiT, Theta, ldt,
                                                  dn_off, logdet, Ainv);
  return fp64_compute
             ? launch_overlap_nt<T, double, 128>(st, W, M, n_up, n_dn, Phi, PsiT, Theta, ldt,
                                                 dn_off, logdet, Ainv)
             : launch_overlap_nt<T, float, 128>(st, W, M, n_up, n_dn, Phi, PsiT, Theta, ldt,
                                                dn_off, logdet, Ainv);
}

cudaError_t launch_weights(cudaStream_t st, int W, const double2* logO_new,
                           const double2* logdet, const double2* lw, const double2* lmf,
                           const double2* eloc, double dtau, double e_shift, double cap,
                           const double* wref, double* weight, double2* logO,
                           long long* ctr) {
  weights_kernel<<<blocks_for(W, 256), 256, 0, st>>>(W, logO_new, logdet, lw, lmf, eloc, dtau,
                                                     e_shift, cap, wref, weight, logO, ctr);
  return cudaGetLastError();
}

cudaError_t launch_logdet_sum(cudaStream_t st, int W, const double2* logdet,
                              double2* out) {
  logdet_sum_kernel<<<blocks_for(W, 256), 256, 0, st>>>(W, logdet, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_qr(cudaStream_t st, int W, int M, int n_up, int n_dn, T* Phi,
                      double2* logO, double* lr, bool fp64_compute) {
  const int nmax = n_up > n_dn ? n_up : n_dn;
  const int threads = M > 96 ? 256 : 128;
  dim3 grid(W, 2);
  if (fp64_compute) {
    const size_t cap = smem_optin((const void*)qr_kernel<T, double>);
    const size_t smem = qr_smem(M, nmax, sizeof(double2));
    if (smem > cap) return cudaErrorInvalidValue;
    qr_kernel<T, double><<<grid, threads, smem, st>>>(M, n_up, n_dn, Phi, lr);
  } else {
    const size_t cap = smem_optin((const void*)qr_kernel<T, float>);
    const size_t smem = qr_smem(M, nmax, sizeof(float2));
    if (smem > cap) return cudaErrorInvalidValue;
    qr_kernel<T, float><<<grid, threads, smem, st>>>(M, n_up, n_dn, Phi, lr);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sub_logdet_r_kernel<<<blocks_for(W, 256), 256, 0, st>>>(W, lr, logO);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_energy_reduce(cudaStream_t st, int W, int M, int n_up, int n_dn,
                                 int n_chol, const T* X, long ldx, int nsplit,
                                 long split_stride, const T* Theta, long ldt, long dn_off,
                                 const T* Z, long ldz_up, long ldz_dn, double2* eloc) {
  energy_reduce_kernel<T><<<W, 256, 0, st>>>(M, n_up, n_dn, n_chol, X, ldx, nsplit,
                                             split_stride, Theta, ldt, dn_off, Z, ldz_up,
                                             ldz_dn, W, eloc);
  return cudaGetLastError();
}

cudaError_t launch_mixed_energy(cudaStream_t st, int W, const double* weight,
                                const double2* eloc, long long* ctr, double2* hist,
                                int hist_len, double* out) {
  mixed_energy_kernel<<<1, 1024, 0, st>>>(W, weight, eloc, ctr, hist, hist_len, out);
  return cudaGetLastError();
}

cudaError_t launch_comb(cudaStream_t st, int W, const double* weight, uint64_t seed,
                        int run_id, const long long* ctr, long step, int* parent,
                        double* scratch, double* wnew, int* status) {
  const size_t smem_cap = smem_optin((const void*)comb_kernel);
  int nb = (W + kScanBlock - 1) / kScanBlock;
  size_t smem = sizeof(double) * 2 * (size_t)nb;
  if (smem > smem_cap) return cudaErrorInvalidValue;
  comb_kernel<<<1, 1024, smem, st>>>(W, weight, (uint32_t)seed, (uint32_t)(seed >> 32),
                                     run_id, ctr, (long long)step, parent, scratch, wnew,
                                     status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather(cudaStream_t st, int W, long phi_elems, long theta_elems,
                          const int* parent, const T* Phi, T* Phi_out,
                          const T* Theta, T* Theta_out, const double2* logO,
                          double2* logO_out, const double* wnew, double* weight,
                          double* wref, double* log_scale) {
  gather_kernel<T><<<W, 256, 0, st>>>(phi_elems, theta_elems, parent, Phi, Phi_out,
                                      Theta, Theta_out, logO, logO_out, wnew, weight,
                                      wref, log_scale);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gather_rows(cudaStream_t st, int W, long elems, const int* parent,
                               const T* in, T* out) {
  gather_rows_kernel<T><<<W, 256, 0, st>>>(elems, parent, in, out);
  return cudaGetLastError();
}
template cudaError_t launch_gather_rows<float>(cudaStream_t, int, long, const int*,
                                               const float*, float*);
template cudaError_t launch_gather_rows<double>(cudaStream_t, int, long, const int*,
                                                const double*, double*);
template cudaError_t launch_gather_rows<double2>(cudaStream_t, int, long, const int*,
                                                 const double2*, double2*);

cudaError_t launch_h1_remainder(cudaStream_t st, int M, int n_chol, const double* h1,
                                const double* L, const double* lbar, double* h1p) {
  h1_remainder_kernel<<<blocks_for((long)M * M, 128), 128, 0, st>>>(M, n_chol, h1, L, lbar,
                                                                     h1p);
  return cudaGetLastError();
}

cudaError_t launch_scale_identity(cudaStream_t st, int M, const double* A, double s,
                                  double* out_I_plus, double* out_scaled) {
  scale_identity_kernel<<<blocks_for((long)M * M, 256), 256, 0, st>>>(M, A, s, out_I_plus,
                                                                      out_scaled);
  return cudaGetLastError();
}

cudaError_t launch_yx_permute(cudaStream_t st, int n, int M, const double* gram,
                              double* yx, long ldy) {
  long J = (long)n * M;
  yx_permute_kernel<<<blocks_for(J * J, 256), 256, 0, st>>>(n, M, gram, yx, ldy);
  return cudaGetLastError();
}

cudaError_t launch_pad_rows(cudaStream_t st, long rows, long Jup, long Jdn,
                            const double* in, double* out, long ld, long dn_off) {
  pad_rows_kernel<<<blocks_for(rows * (Jup + Jdn), 256), 256, 0, st>>>(rows, Jup, Jdn, in,
                                                                     out, ld, dn_off);
  return cudaGetLastError();
}

cudaError_t launch_gemv_rows(cudaStream_t st, long rows, long cols, const double* A, long lda,
                             const double* x, double* y) {
  if (rows <= 0) return cudaSuccess;
  gemv_rows_kernel<<<(unsigned)rows, 256, 0, st>>>(cols, A, lda, x, y);
  return cudaGetLastError();
}

cudaError_t launch_gemv_cols(cudaStream_t st, long rows, long cols, const double* A, long lda,
                             const double* x, double* y) {
  if (cols <= 0) return cudaSuccess;
  gemv_cols_kernel<<<blocks_for(cols, 256), 256, 0, st>>>(rows, cols, A, lda, x, y);
  return cudaGetLastError();
}

cudaError_t launch_transpose_pad(cudaStream_t st, long G, int M, long ldv, const double* in,
                                 double* out, long ldo) {
  transpose_pad_kernel<<<blocks_for(G * M * M, 256), 256, 0, st>>>(G, M, ldv, in, out, ldo);
  return cudaGetLastError();
}

cudaError_t launch_transpose(cudaStream_t st, long rows, long cols, const double* in,
                             double* out, long ldo) {
  transpose_kernel<<<blocks_for(rows * cols, 256), 256, 0, st>>>(rows, cols, in, out, ldo);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_convert(cudaStream_t st, long n, const double* in, T* out) {
  if (n <= 0) return cudaSuccess;
  convert_kernel<T><<<blocks_for(n, 256), 256, 0, st>>>(n, in, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_walkers(cudaStream_t st, int W, int M, int N, const T* PsiT,
                                T* Phi, double* weight) {
  init_walkers_kernel<T><<<W, 256, 0, st>>>(M, N, PsiT, Phi, weight);
  return cudaGetLastError();
}

cudaError_t launch_add_diag(cudaStream_t st, int M, double* A, double a) {
  add_diag_kernel<<<blocks_for(M, 128), 128, 0, st>>>(M, A, a);
  return cudaGetLastError();
}

cudaError_t launch_axpy_d(cudaStream_t st, long n, double a, const double* x, double* y) {
  axpy_d_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, a, x, y);
  return cudaGetLastError();
}

// ------------------------------------------- K4 + K5, block-diagonal L_g
namespace {

// Packed Cholesky operands of the block-diagonal form: Lp[g][e] =
// L_g[gidx[e]] ([n_chol][nnz]) and, for the tensor cores, its transpose
// LpT[e][g] ([nnzp][ldS], zero beyond nnz and n_chol). FP64, at setup.
__global__ void pack_blocks_kernel(int G, long nnz, long nnzp, long ldS, long MM,
                                   const double* __restrict__ L, const int* __restrict__ gidx,
                                   double* __restrict__ Lp, double* __restrict__ LpT) {
  const long e = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (e >= nnzp * ldS) return;
  const long r = e / ldS;
  const int g = (int)(e - r * ldS);
  const bool in = r < nnz && g < G;
  const double v = in ? L[(long)g * MM + gidx[r]] : 0.0;
  if (LpT) LpT[e] = v;
  if (in) Lp[(long)g * nnz + r] = v;
}

// K5's series for a block-diagonal V: Pout = sum_{n <= order} V^n Pin / n!,
// V packed [W][2][nnzp] (real entries, then imaginary; each basis index's
// row of its block at tab[p].x, tab[p].y entries long, its block's members
// at members[tab[p].z ..]), Pin / Pout [W][N][2][M]. One block per walker:
// the walker's V and a chunk of jc columns (current term, next term,
// running sum) in shared memory; one thread per (column, row) element.
template <typename T>
__global__ void taylor_blocks_kernel(int M, int N, int order, long nnzp, int jc, size_t tab_off,
                                     const T* __restrict__ V, const int4* __restrict__ tab,
                                     const int* __restrict__ members,
                                     const T* __restrict__ Pin, T* __restrict__ Pout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vr = reinterpret_cast<T*>(smem_raw);
  T* vi = vr + nnzp;
  const long cs = (long)jc * 2 * M;
  T* t = vi + nnzp;
  T* tn = t + cs;
  T* acc = tn + cs;
  int4* tb = reinterpret_cast<int4*>(smem_raw + tab_off);
  int* mem = reinterpret_cast<int*>(tb + M);
  const int w = blockIdx.x;
  const T* Vw = V + (long)w * 2 * nnzp;
  for (long e = threadIdx.x; e < nnzp; e += blockDim.x) {
    vr[e] = Vw[e];
    vi[e] = Vw[nnzp + e];
  }
  for (int p = threadIdx.x; p < M; p += blockDim.x) {
    tb[p] = tab[p];
    mem[p] = members[p];
  }
  for (int j0 = 0; j0 < N; j0 += jc) {
    const int nc = min(jc, N - j0);
    const long ne = (long)nc * 2 * M;
    const T* Pw = Pin + ((long)w * N + j0) * 2 * M;
    __syncthreads();                       // tables ready, the last chunk's reads done
    for (long e = threadIdx.x; e < ne; e += blockDim.x) {
      const T x = Pw[e];
      t[e] = x;
      acc[e] = x;
    }
    T* cur = t;
    T* nxt = tn;
    // this thread's first element (column j, row p); it then steps by
    // blockDim.x elements, (j, p) advanced without a division
    const int e0 = (int)threadIdx.x, step_j = (int)blockDim.x / M, step_p = (int)blockDim.x % M;
    for (int n = 1; n <= order; ++n) {
      __syncthreads();                     // the previous term is complete
      const T inv = T(1) / T(n);
      int j = e0 / M, p = e0 - j * M;
      for (; j < nc;) {
        const int4 d = tb[p];
        const T* cr = cur + j * 2 * M;
        const T* ci = cr + M;
        T sr = T(0), si = T(0);
        for (int q = 0; q < d.y; ++q) {
          const int k = mem[d.z + q];
          const T ar = vr[d.x + q], ai = vi[d.x + q], br = cr[k], bi = ci[k];
          sr = fma(ar, br, fma(-ai, bi, sr));
          si = fma(ar, bi, fma(ai, br, si));
        }
        sr *= inv;
        si *= inv;
        const int o = j * 2 * M + p;
        nxt[o] = sr;
        nxt[o + M] = si;
        acc[o] += sr;
        acc[o + M] += si;
        j += step_j;
        p += step_p;
        if (p >= M) { p -= M; ++j; }
      }
      T* sw = cur;
      cur = nxt;
      nxt = sw;
    }
    __syncthreads();
    T* Ow = Pout + ((long)w * N + j0) * 2 * M;
    for (long e = threadIdx.x; e < ne; e += blockDim.x) Ow[e] = acc[e];
  }
}

// The same series with one thread per (block, column) task, the block's
// piece of the column in registers (blocks of at most MAXB orbitals): tasks
// run column-fastest, so the threads of a warp read the same entries of V
// (broadcast) and nothing else goes through shared memory. btab holds per
// block {offset of its first row in V, size, member base, 0}.
template <typename T, int MAXB>
__global__ void taylor_blocks_reg_kernel(int M, int N, int order, long nnzp, int nb,
                                         const T* __restrict__ V, const int4* __restrict__ btab,
                                         const int* __restrict__ members,
                                         const T* __restrict__ Pin, T* __restrict__ Pout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vr = reinterpret_cast<T*>(smem_raw);
  T* vi = vr + nnzp;
  const int w = blockIdx.x;
  const T* Vw = V + (long)w * 2 * nnzp;
  for (long e = threadIdx.x; e < nnzp; e += blockDim.x) {
    vr[e] = Vw[e];
    vi[e] = Vw[nnzp + e];
  }
  __syncthreads();
  for (int task = threadIdx.x; task < nb * N; task += blockDim.x) {
    const int bl = task / N, j = task - bl * N;
    const int4 d = btab[bl];
    const int b = d.y;
    const T* pr = Pin + ((long)w * N + j) * 2 * M;
    const T* pi = pr + M;
    int mem[MAXB];
    T xr[MAXB], xi[MAXB], sr[MAXB], si[MAXB];
#pragma unroll
    for (int p = 0; p < MAXB; ++p) {
      mem[p] = p < b ? members[d.z + p] : 0;
      xr[p] = p < b ? pr[mem[p]] : T(0);
      xi[p] = p < b ? pi[mem[p]] : T(0);
      sr[p] = xr[p];
      si[p] = xi[p];
    }
    for (int n = 1; n <= order; ++n) {
      const T inv = T(1) / T(n);
      T yr[MAXB], yi[MAXB];
#pragma unroll
      for (int p = 0; p < MAXB; ++p) {
        T ar_ = T(0), ai_ = T(0);
        if (p < b) {
          const T* vrp = vr + d.x + p * b;
          const T* vip = vi + d.x + p * b;
#pragma unroll
          for (int q = 0; q < MAXB; ++q) {
            if (q < b) {
              const T a = vrp[q], c = vip[q];
              ar_ = fma(a, xr[q], fma(-c, xi[q], ar_));
              ai_ = fma(a, xi[q], fma(c, xr[q], ai_));
            }
          }
        }
        yr[p] = ar_ * inv;
        yi[p] = ai_ * inv;
      }
#pragma unroll
      for (int p = 0; p < MAXB; ++p) {
        xr[p] = yr[p];
        xi[p] = yi[p];
        sr[p] += yr[p];
        si[p] += yi[p];
      }
    }
    T* qr = Pout + ((long)w * N + j) * 2 * M;
    T* qi = qr + M;
#pragma unroll
    for (int p = 0; p < MAXB; ++p)
      if (p < b) {
        qr[mem[p]] = sr[p];
        qi[mem[p]] = si[p];
      }
  }
}

}  // namespace

cudaError_t launch_pack_blocks(cudaStream_t st, int G, long nnz, long nnzp, long ldS, int M,
                               const double* L, const int* gidx, double* Lp, double* LpT) {
  const long n = nnzp * ldS;
  pack_blocks_kernel<<<blocks_for(n, 256), 256, 0, st>>>(G, nnz, nnzp, ldS, (long)M * M, L,
                                                         gidx, Lp, LpT);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_taylor_blocks(cudaStream_t st, int W, int M, int N, int order, long nnzp,
                                 int nb, int maxb, const T* V, const void* blk, const T* Pin,
                                 T* Pout) {
  if (W < 1 || M < 1 || N < 1 || order < 0 || nb < 1 || nb > M) return cudaErrorInvalidValue;
  // blk: M int4 rows, M int4 block slots, then the M member indices (every
  // int4 array at a 16-byte multiple)
  const int4* tab = reinterpret_cast<const int4*>(blk);
  const int4* btab = tab + M;
  const int* members = reinterpret_cast<const int*>(tab + 2 * (long)M);
  if (maxb <= 8) {   // registers: one thread per (block, column)
    const size_t smem = 2 * (size_t)nnzp * sizeof(T);
    if (smem > smem_optin((const void*)taylor_blocks_reg_kernel<T, 8>))
      return cudaErrorInvalidValue;
    taylor_blocks_reg_kernel<T, 8><<<W, 256, smem, st>>>(M, N, order, nnzp, nb, V, btab,
                                                          members, Pin, Pout);
    return cudaGetLastError();
  }
  const size_t cap = smem_optin((const void*)taylor_blocks_kernel<T>);
  const size_t tabs = (size_t)M * (sizeof(int4) + sizeof(int));
  const size_t vbytes = 2 * (size_t)nnzp * sizeof(T), per_col = 6 * (size_t)M * sizeof(T);
  if (cap < vbytes + per_col + tabs + 16) return cudaErrorInvalidValue;
  // columns per chunk: all of them if the block stays within 48 KB (several
  // blocks per SM hide the shared-memory latencies), else as many as fit
  const size_t want = std::max<size_t>(48 * 1024, vbytes + per_col + tabs + 16);
  const size_t room = std::min(cap, want) - vbytes - tabs - 16;
  const int jc = (int)std::max<size_t>(1, std::min<size_t>((size_t)N, room / per_col));
  const size_t tab_off = (vbytes + (size_t)jc * per_col + 15) & ~(size_t)15;
  taylor_blocks_kernel<T><<<W, 256, tab_off + tabs, st>>>(M, N, order, nnzp, jc, tab_off, V,
                                                          tab, members, Pin, Pout);
  return cudaGetLastError();
}

#define AFQMC_INST(T)                                                                    \
  template cudaError_t launch_fields<T>(cudaStream_t, int, int, const T*, long, int,    \
                                        long, double, double, uint64_t, int,            \
                                        const long long*, T*, long, T*, double2*,       \
                                        const double*, double2*);                       \
  template cudaError_t launch_taylor<T>(cudaStream_t, int, int, int, int, const T*, long,\
                                        const T*, T*);                                  \
  template cudaError_t launch_overlap<T>(cudaStream_t, int, int, int, int, const T*,    \
                                         const T*, T*, long, long, double2*, double2*,  \
                                         bool);                                         \
  template cudaError_t launch_qr<T>(cudaStream_t, int, int, int, int, T*, double2*,     \
                                    double*, bool);                                     \
  template cudaError_t launch_energy_reduce<T>(cudaStream_t, int, int, int, int, int,   \
                                               const T*, long, int, long, const T*,     \
                                               long, long, const T*, long, long,        \
                                               double2*);                               \
  template cudaError_t launch_gather<T>(cudaStream_t, int, long, long, const int*,      \
                                        const T*, T*, const T*, T*, const double2*,     \
                                        double2*, const double*, double*, double*,      \
                                        double*);                                       \
  template cudaError_t launch_convert<T>(cudaStream_t, long, const double*, T*);        \
  template cudaError_t launch_init_walkers<T>(cudaStream_t, int, int, int, const T*,    \
                                              T*, double*);                             \
  template cudaError_t launch_taylor_blocks<T>(cudaStream_t, int, int, int, int, long,  \
                                               int, int, const T*, const void*, const T*, \
                                               T*);
AFQMC_INST(float)
AFQMC_INST(double)

}  // namespace afqmc
