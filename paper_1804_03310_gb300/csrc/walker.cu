// Per-walker kernels of the ph-AFQMC step: field draw and force-bias shift
// (Sec. II, Eq. 2), Taylor propagation on the CUDA cores (Sec. II, Eq. 3),
// overlap / inverse / Theta (Sec. III), hybrid weight with the phaseless cut
// (Sec. II), modified Gram-Schmidt (Sec. IV.A), the local-energy epilogue
// (Sec. III, Eq. 5), and the comb (Sec. V).
#include <float.h>

#include "common.cuh"
#include "kernels.h"

namespace afqmc {

namespace {


// Opt the kernel in to the largest dynamic shared memory the device allows
// beside its static shared memory; returns that limit in bytes. Errors of
// these queries are cleared so they cannot surface at a later launch check.
template <typename K>
size_t allow_big_smem(K kernel) {
  int dev = 0, optin = 48 * 1024;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  size_t stat = 0;
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) stat = fa.sharedSizeBytes;
  size_t dyn = (size_t)optin > stat ? (size_t)optin - stat : 0;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  cudaGetLastError();
  return dyn;
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
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
                              double2* __restrict__ lw) {
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
  const int nq = (n_chol + 3) >> 2;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
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
      C xr = 0, xi = 0;   // X summed over the K-split partials, in order
      for (int sp = 0; sp < nsplit; ++sp) {
        xr += (C)Xr[sp * split_stride + g];
        xi += (C)Xi[sp * split_stride + g];
      }
      // xbar = -i sqrt(dt) X
      C br = sqdt * xi;
      C bi = -sqdt * xr;
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
    }
  }
  const double tre = block_sum((double)lre, red);
  const double tim = block_sum((double)lim, red);
  if (threadIdx.x == 0) lw[w] = make_double2(tre, tim);
}

// --------------------------------------------------------------- K5 (SIMT)
constexpr int kTaylorThreads = 256;
constexpr int kTaylorKC = 16;
constexpr int kTaylorMaxR = 16;   // outputs per thread: M * NC <= 4096

template <typename T>
__global__ void __launch_bounds__(kTaylorThreads)
taylor_kernel(int M, int N, int NC, int order, const T* __restrict__ V,
              const T* __restrict__ Pin, T* __restrict__ Pout) {
  extern __shared__ unsigned char smem_raw[];
  T* tc = reinterpret_cast<T*>(smem_raw);            // [NC][2][M]
  T* vs = tc + (long)NC * 2 * M;                      // [2][KC][M]
  const int w = blockIdx.x;
  const int j0 = blockIdx.y * NC;
  const int nc = min(NC, N - j0);
  const T* Vw = V + (long)w * 2 * M * M;
  const T* Pw = Pin + ((long)w * N + j0) * 2 * M;
  T* Ow = Pout + ((long)w * N + j0) * 2 * M;
  const int tid = threadIdx.x;
  const int nout = M * nc;
  for (int e = tid; e < NC * 2 * M; e += blockDim.x)
    tc[e] = (e < nc * 2 * M) ? Pw[e] : T(0);
  __syncthreads();
  T ar[kTaylorMaxR], ai[kTaylorMaxR];
#pragma unroll
  for (int r = 0; r < kTaylorMaxR; ++r) {
    int o = tid + r * kTaylorThreads;
    if (o < nout) {
      int i = o % M, jj = o / M;
      ar[r] = tc[(jj * 2 + 0) * M + i];
      ai[r] = tc[(jj * 2 + 1) * M + i];
    } else {
      ar[r] = T(0);
      ai[r] = T(0);
    }
  }
  for (int n = 1; n <= order; ++n) {
    T tr[kTaylorMaxR], ti[kTaylorMaxR];
#pragma unroll
    for (int r = 0; r < kTaylorMaxR; ++r) { tr[r] = T(0); ti[r] = T(0); }
    for (int k0 = 0; k0 < M; k0 += kTaylorKC) {
      const int kc = min(kTaylorKC, M - k0);
      __syncthreads();
      // V is complex symmetric: row k of V is column k.
      for (int e = tid; e < 2 * kTaylorKC * M; e += blockDim.x) {
        int c = e / (kTaylorKC * M);
        int rem = e - c * kTaylorKC * M;
        int kk = rem / M, i = rem - kk * M;
        vs[e] = (kk < kc) ? Vw[((long)c * M + (k0 + kk)) * M + i] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int r = 0; r < kTaylorMaxR; ++r) {
        int o = tid + r * kTaylorThreads;
        if (o >= nout) break;
        int i = o % M, jj = o / M;
        const T* tre = tc + (jj * 2 + 0) * M + k0;
        const T* tim = tc + (jj * 2 + 1) * M + k0;
        T sr = tr[r], si = ti[r];
        for (int kk = 0; kk < kc; ++kk) {
          T vr = vs[kk * M + i], vi = vs[(kTaylorKC + kk) * M + i];
          T xr = tre[kk], xi = tim[kk];
          sr = fma(vr, xr, sr);
          sr = fma(-vi, xi, sr);
          si = fma(vr, xi, si);
          si = fma(vi, xr, si);
        }
        tr[r] = sr;
        ti[r] = si;
      }
    }
    __syncthreads();
    const T inv_n = T(1) / T(n);
#pragma unroll
    for (int r = 0; r < kTaylorMaxR; ++r) {
      int o = tid + r * kTaylorThreads;
      if (o >= nout) break;
      int i = o % M, jj = o / M;
      T xr = tr[r] * inv_n, xi = ti[r] * inv_n;
      tc[(jj * 2 + 0) * M + i] = xr;
      tc[(jj * 2 + 1) * M + i] = xi;
      ar[r] += xr;
      ai[r] += xi;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kTaylorMaxR; ++r) {
    int o = tid + r * kTaylorThreads;
    if (o >= nout) break;
    int i = o % M, jj = o / M;
    Ow[(jj * 2 + 0) * M + i] = ar[r];
    Ow[(jj * 2 + 1) * M + i] = ai[r];
  }
}

// --------------------------------------------------------------- K6
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
__device__ __forceinline__ cx<R> div_c(cx<R> a, cx<R> b) {
  R d = b.x * b.x + b.y * b.y;
  return mk<R>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

template <typename R>
__device__ __forceinline__ cx<R> mul_c(cx<R> a, cx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Row stride (in complex values) of a walker block staged as [column][row]:
// odd, so that lanes reading the same row of consecutive columns hit
// distinct banks.
__host__ __device__ __forceinline__ int staged_ld(int M) { return M | 1; }

// One block per (walker, spin), with the walker's columns of that spin
// staged in shared memory as Q[b][k] (orbital column b, basis row k).
//  1. A = D^T Phi (real trial orbitals), ns x ns.
//  2. LU with partial pivoting, P A = L U, in the compute type R; the
//     log-determinant sum_k ln U_kk (+ i pi per odd row-swap count) is
//     accumulated in FP64.
//  3. Theta = Phi A^-1 = Phi U^-1 L^-1 P row by row: thread k solves
//     z U = phi_k, then y L = z, and scatters theta_k[perm[i]] = y_i.
template <typename T, typename R>
__global__ void overlap_kernel(int M, int n_up, int n_dn, const T* __restrict__ Phi,
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
  const int ldq = staged_ld(M);
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  cx<R>* Q = reinterpret_cast<cx<R>*>(smem_raw);      // [ns][ldq]
  cx<R>* A = Q + (long)ns * ldq;                      // [ns][ns], L and U in place
  R* D = reinterpret_cast<R*>(A + (long)ns * ns);     // [ns][ldq] trial rows
  int* perm = reinterpret_cast<int*>(D + (long)ns * ldq);
  __shared__ int piv, singular, nswap;
  const T* Pw = Phi + ((long)w * N + j0) * 2 * M;
  for (int b = 0; b < ns; ++b) {                      // column b, both planes
    const T* col = Pw + (long)b * 2 * M;
    for (int r = tid; r < 2 * M; r += nt) {
      const R v = (R)col[r];
      if (r < M) Q[b * ldq + r].x = v;
      else Q[b * ldq + r - M].y = v;
    }
    for (int k = tid; k < M; k += nt) D[b * ldq + k] = (R)PsiT[(long)(j0 + b) * M + k];
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
          if (a0 + u < ns && b0 + v < ns) A[(a0 + u) * ns + b0 + v] = mk<R>(sr[u][v], si[u][v]);
    }
  }
  __syncthreads();
  for (int k = 0; k < ns; ++k) {
    if (tid < 32) {
      R best = R(-1);
      int bi = k;
      for (int i = k + tid; i < ns; i += 32) {
        const cx<R> v = A[i * ns + k];
        const R m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        piv = bi;
        if (!(best > R(0))) singular = 1;
      }
    }
    __syncthreads();
    if (singular) break;
    const int p = piv;
    if (p != k) {
      for (int c = tid; c < ns; c += nt) {
        const cx<R> t = A[k * ns + c];
        A[k * ns + c] = A[p * ns + c];
        A[p * ns + c] = t;
      }
      if (tid == 0) {
        const int t = perm[k];
        perm[k] = perm[p];
        perm[p] = t;
        nswap ^= 1;
      }
      __syncthreads();
    }
    const cx<R> pv = A[k * ns + k];
    for (int i = k + 1 + tid; i < ns; i += nt) A[i * ns + k] = div_c(A[i * ns + k], pv);
    __syncthreads();
    // trailing update: lane = column, warp = every nwarps-th row
    for (int j = k + 1 + lane; j < ns; j += 32) {
      const cx<R> ukj = A[k * ns + j];
      for (int i = k + 1 + warp; i < ns; i += nwarps)
        A[i * ns + j] = sub_mul(A[i * ns + j], A[i * ns + k], ukj);
    }
    __syncthreads();
  }
  const int sing = singular;
  if (tid < 32) {
    double lre = 0.0, lim = 0.0;
    if (!sing) {
      for (int k = tid; k < ns; k += 32) {
        const double px = (double)A[k * ns + k].x, py = (double)A[k * ns + k].y;
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
  for (int k = tid; k < M; k += nt) {
    if (sing) {
      for (int a = 0; a < ns; ++a) {
        Tr[(long)a * M + k] = T(0);
        Ti[(long)a * M + k] = T(0);
      }
      continue;
    }
    for (int j = 0; j < ns; ++j) {              // z U = phi_k (two partial sums)
      cx<R> s0 = Q[j * ldq + k], s1 = mk<R>(R(0), R(0));
      int i = 0;
      for (; i + 1 < j; i += 2) {
        s0 = sub_mul(s0, Q[i * ldq + k], A[i * ns + j]);
        s1 = sub_mul(s1, Q[(i + 1) * ldq + k], A[(i + 1) * ns + j]);
      }
      if (i < j) s0 = sub_mul(s0, Q[i * ldq + k], A[i * ns + j]);
      Q[j * ldq + k] = div_c(mk<R>(s0.x + s1.x, s0.y + s1.y), A[j * ns + j]);
    }
    for (int j = ns - 2; j >= 0; --j) {         // y L = z (unit lower L)
      cx<R> s0 = Q[j * ldq + k], s1 = mk<R>(R(0), R(0));
      int i = j + 1;
      for (; i + 1 < ns; i += 2) {
        s0 = sub_mul(s0, Q[i * ldq + k], A[i * ns + j]);
        s1 = sub_mul(s1, Q[(i + 1) * ldq + k], A[(i + 1) * ns + j]);
      }
      if (i < ns) s0 = sub_mul(s0, Q[i * ldq + k], A[i * ns + j]);
      Q[j * ldq + k] = mk<R>(s0.x + s1.x, s0.y + s1.y);
    }
    for (int i = 0; i < ns; ++i) {              // theta_k[perm[i]] = y_i
      const cx<R> y = Q[i * ldq + k];
      Tr[(long)perm[i] * M + k] = (T)y.x;
      Ti[(long)perm[i] * M + k] = (T)y.y;
    }
  }
  if (Ainv_out) {                               // rows of A^-1 = e_r U^-1 L^-1 P
    __syncthreads();
    double2* Ao = Ainv_out + ((long)w * 2 + sig) * nmax * nmax;
    cx<R>* rowbuf = Q;                          // reuse: [ns][ldq] as [i][r]
    for (int r = tid; r < ns; r += nt) {
      for (int j = 0; j < ns; ++j) {
        cx<R> s = mk<R>(j == r ? R(1) : R(0), R(0));
        for (int i = 0; i < j; ++i) s = sub_mul(s, rowbuf[i * ldq + r], A[i * ns + j]);
        rowbuf[j * ldq + r] = sing ? mk<R>(R(0), R(0)) : div_c(s, A[j * ns + j]);
      }
      for (int j = ns - 2; j >= 0; --j) {
        cx<R> s = rowbuf[j * ldq + r];
        for (int i = j + 1; i < ns; ++i) s = sub_mul(s, rowbuf[i * ldq + r], A[i * ns + j]);
        rowbuf[j * ldq + r] = s;
      }
      for (int i = 0; i < ns; ++i) {
        const cx<R> y = rowbuf[i * ldq + r];
        Ao[(long)r * nmax + perm[i]] = make_double2((double)y.x, (double)y.y);
      }
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
__global__ void weights_kernel(int W, const double2* __restrict__ logO_new,
                               const double2* __restrict__ logdet,
                               const double2* __restrict__ lw, double dtau,
                               double e_shift, double cap, const double* __restrict__ wref,
                               double* __restrict__ weight,
                               double2* __restrict__ logO, long long* __restrict__ ctr) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w == 0) ctr[0] += 1;   // the step is complete once its weights are
  if (w >= W) return;
  const double2 ln = logO_new ? logO_new[w] : cadd(logdet[2 * w], logdet[2 * w + 1]);
  double2 lnR = csub(ln, logO[w]);
  double2 l = lw[w];
  double lnI_re = lnR.x + l.x + dtau * e_shift;
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
// (Cholesky), then Q = Phi R^-1 row by row. The walkers are re-orthonormalised
// every few steps, so S stays close to the identity and the Cholesky route is
// as accurate as Gram-Schmidt. One block per (walker, spin); ln det R =
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
  for (int b = 0; b < ns; ++b) {                      // column b, both planes
    const T* col = Pw + (long)b * 2 * M;
    for (int r = tid; r < 2 * M; r += nt) {
      const R v = (R)col[r];
      if (r < M) Q[b * ldq + r].x = v;
      else Q[b * ldq + r - M].y = v;
    }
  }
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
                              double* __restrict__ weight) {
  const int j = blockIdx.x;
  const int p = parent[j];
  for (long e = threadIdx.x; e < phi_elems; e += blockDim.x)
    Phi_out[(long)j * phi_elems + e] = Phi[(long)p * phi_elems + e];
  for (long e = threadIdx.x; e < theta_elems; e += blockDim.x)
    Theta_out[(long)j * theta_elems + e] = Theta[(long)p * theta_elems + e];
  if (threadIdx.x == 0) {
    logO_out[j] = logO[p];
    double wn = *wnew;
    if (wn > 0.0) weight[j] = wn;
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

__global__ void h1_remainder_kernel(int M, int n_chol, const double* __restrict__ h1,
                                    const double* __restrict__ L,
                                    double* __restrict__ h1p) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * M) return;
  int i = e / M, j = e - i * M;
  double s = 0.0;
  for (int g = 0; g < n_chol; ++g) {
    const double* Lg = L + (long)g * M * M;
    for (int k = 0; k < M; ++k) s = fma(Lg[i * M + k], Lg[k * M + j], s);
  }
  h1p[e] = h1[e] - 0.5 * s;
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
                          T* xbar, double2* lw) {
  fields_kernel<T><<<W, 128, 0, st>>>(n_chol, X, ldx, nsplit, split_stride, sqdt, cap,
                                      (uint32_t)seed, (uint32_t)(seed >> 32), run_id, ctr,
                                      S, ldS, xbar, lw);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_taylor(cudaStream_t st, int W, int M, int N, int order,
                          const T* V, const T* Phi_in, T* Phi_out) {
  static const size_t smem_cap = allow_big_smem(taylor_kernel<T>);
  int NC = 4096 / M;
  if (NC > 16) NC = 16;
  if (NC < 1) return cudaErrorInvalidValue;
  if (NC > N) NC = N;
  size_t smem = sizeof(T) * ((size_t)NC * 2 * M + 2 * (size_t)kTaylorKC * M);
  if (smem > smem_cap) return cudaErrorInvalidValue;
  dim3 grid(W, (N + NC - 1) / NC);
  taylor_kernel<T><<<grid, kTaylorThreads, smem, st>>>(M, N, NC, order, V, Phi_in, Phi_out);
  return cudaGetLastError();
}

size_t overlap_smem(int M, int nmax, size_t csize) {
  return csize * ((size_t)nmax * staged_ld(M) + (size_t)nmax * nmax) +
         csize / 2 * (size_t)nmax * staged_ld(M) + sizeof(int) * nmax;
}

template <typename T>
cudaError_t launch_overlap(cudaStream_t st, int W, int M, int n_up, int n_dn,
                           const T* Phi, const T* PsiT, T* Theta, long ldt, long dn_off,
                           double2* logdet, double2* Ainv, bool fp64_compute) {
  const int nmax = n_up > n_dn ? n_up : n_dn;
  const int threads = M > 96 ? 256 : 128;
  dim3 grid(W, 2);
  static const size_t cap64 = allow_big_smem(overlap_kernel<T, double>);
  const size_t smem64 = overlap_smem(M, nmax, sizeof(double2));
  if (fp64_compute) {
    if (smem64 > cap64) return cudaErrorInvalidValue;
    overlap_kernel<T, double><<<grid, threads, smem64, st>>>(M, n_up, n_dn, Phi, PsiT, Theta,
                                                            ldt, dn_off, logdet, Ainv, nmax);
  } else {
    static const size_t cap = allow_big_smem(overlap_kernel<T, float>);
    const size_t smem = overlap_smem(M, nmax, sizeof(float2));
    if (smem > cap) return cudaErrorInvalidValue;
    overlap_kernel<T, float><<<grid, threads, smem, st>>>(M, n_up, n_dn, Phi, PsiT, Theta,
                                                         ldt, dn_off, logdet, Ainv, nmax);
  }
  return cudaGetLastError();
}

cudaError_t launch_weights(cudaStream_t st, int W, const double2* logO_new,
                           const double2* logdet, const double2* lw, double dtau,
                           double e_shift, double cap, const double* wref, double* weight,
                           double2* logO, long long* ctr) {
  weights_kernel<<<blocks_for(W, 256), 256, 0, st>>>(W, logO_new, logdet, lw, dtau, e_shift,
                                                     cap, wref, weight, logO, ctr);
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
    static const size_t cap = allow_big_smem(qr_kernel<T, double>);
    const size_t smem = sizeof(double2) * ((size_t)nmax * staged_ld(M) + (size_t)nmax * nmax);
    if (smem > cap) return cudaErrorInvalidValue;
    qr_kernel<T, double><<<grid, threads, smem, st>>>(M, n_up, n_dn, Phi, lr);
  } else {
    static const size_t cap = allow_big_smem(qr_kernel<T, float>);
    const size_t smem = sizeof(float2) * ((size_t)nmax * staged_ld(M) + (size_t)nmax * nmax);
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
  static const size_t smem_cap = allow_big_smem(comb_kernel);
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
                          double2* logO_out, const double* wnew, double* weight) {
  gather_kernel<T><<<W, 256, 0, st>>>(phi_elems, theta_elems, parent, Phi, Phi_out,
                                      Theta, Theta_out, logO, logO_out, wnew, weight);
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
                                const double* L, double* h1p) {
  h1_remainder_kernel<<<blocks_for((long)M * M, 128), 128, 0, st>>>(M, n_chol, h1, L, h1p);
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

#define AFQMC_INST(T)                                                                    \
  template cudaError_t launch_fields<T>(cudaStream_t, int, int, const T*, long, int,    \
                                        long, double, double, uint64_t, int,            \
                                        const long long*, T*, long, T*, double2*);      \
  template cudaError_t launch_taylor<T>(cudaStream_t, int, int, int, int, const T*,     \
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
                                        double2*, const double*, double*);              \
  template cudaError_t launch_convert<T>(cudaStream_t, long, const double*, T*);        \
  template cudaError_t launch_init_walkers<T>(cudaStream_t, int, int, int, const T*,    \
                                              T*, double*);
AFQMC_INST(float)
AFQMC_INST(double)

}  // namespace afqmc
