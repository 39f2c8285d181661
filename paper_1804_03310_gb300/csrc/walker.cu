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
template <typename T>
__global__ void fields_kernel(int n_chol, const T* __restrict__ X, long ldx,
                              double sqdt, double cap, uint32_t k0, uint32_t k1,
                              int run_id, uint32_t step, T* __restrict__ S,
                              T* __restrict__ xbar, double2* __restrict__ lw) {
  __shared__ double red[32];
  const int w = blockIdx.x;
  const T* Xr = X + (2L * w) * ldx;
  const T* Xi = Xr + ldx;
  T* Sr = S + (2L * w) * n_chol;
  T* Si = Sr + n_chol;
  T* Br = xbar + (2L * w) * n_chol;
  T* Bi = Br + n_chol;
  double lre = 0.0, lim = 0.0;
  const int nq = (n_chol + 3) >> 2;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    U4 c = {(uint32_t)q, (uint32_t)w, step, (uint32_t)(4 * run_id + kStreamFields)};
    U4 r = philox4x32_10(c, k0, k1);
    double z[4];
    box_muller(r.x, r.y, z[0], z[1]);
    box_muller(r.z, r.w, z[2], z[3]);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int g = 4 * q + j;
      if (g >= n_chol) break;
      // xbar = -i sqrt(dt) X
      double br = sqdt * (double)Xi[g];
      double bi = -sqdt * (double)Xr[g];
      if (!isfinite(br) || !isfinite(bi)) { br = 0.0; bi = 0.0; }
      if (cap > 0.0) {
        double a = sqrt(br * br + bi * bi);
        if (a > cap) { double f = cap / a; br *= f; bi *= f; }
      }
      double x = z[j];
      double sr = x - br, si = -bi;          // s = x - xbar
      Sr[g] = (T)(-sqdt * si);               // i sqrt(dt) s
      Si[g] = (T)(sqdt * sr);
      Br[g] = (T)br;
      Bi[g] = (T)bi;
      lre += x * br - 0.5 * (br * br - bi * bi);
      lim += x * bi - br * bi;
    }
  }
  lre = block_sum(lre, red);
  lim = block_sum(lim, red);
  if (threadIdx.x == 0) lw[w] = make_double2(lre, lim);
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
struct cx {
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

// One block per (walker, spin). A = D^T Phi (real trial orbitals) is formed
// and inverted by Gauss-Jordan elimination with partial pivoting in the
// compute type R; the log-determinant (sum of the pivots' logarithms plus
// i pi per row swap) is accumulated in FP64 in every precision.
template <typename T, typename R>
__global__ void overlap_kernel(int M, int n_up, int n_dn, const T* __restrict__ Phi,
                               const T* __restrict__ PsiT, T* __restrict__ Theta,
                               double2* __restrict__ logdet,
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
  cx<R>* aug = reinterpret_cast<cx<R>*>(smem_raw);   // [ns][2 ns]
  cx<R>* fac = aug + (long)ns * 2 * ns;               // [ns]
  __shared__ int piv;
  __shared__ int singular;
  __shared__ double2 ld;
  __shared__ int nswap;
  const int ld2 = 2 * ns;
  const T* Pw = Phi + (long)w * N * 2 * M;
  for (int e = tid; e < ns * ns; e += nt) {
    int a = e / ns, b = e - a * ns;
    const T* d = PsiT + (long)(j0 + a) * M;
    const T* pr = Pw + ((long)(j0 + b) * 2 + 0) * M;
    const T* pi = pr + M;
    R sr = 0, si = 0;
    for (int k = 0; k < M; ++k) {
      R dk = (R)d[k];
      sr = fma(dk, (R)pr[k], sr);
      si = fma(dk, (R)pi[k], si);
    }
    aug[a * ld2 + b] = mk<R>(sr, si);
    aug[a * ld2 + ns + b] = mk<R>(a == b ? R(1) : R(0), R(0));
  }
  if (tid == 0) { ld = make_double2(0.0, 0.0); nswap = 0; singular = 0; }
  __syncthreads();
  for (int k = 0; k < ns; ++k) {
    if (tid < 32) {
      R best = R(-1);
      int bi = k;
      for (int i = k + tid; i < ns; i += 32) {
        cx<R> v = aug[i * ld2 + k];
        R m = v.x * v.x + v.y * v.y;
        if (m > best) { best = m; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        R ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
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
      for (int c = tid; c < ld2; c += nt) {
        cx<R> t = aug[k * ld2 + c];
        aug[k * ld2 + c] = aug[p * ld2 + c];
        aug[p * ld2 + c] = t;
      }
      if (tid == 0) nswap ^= 1;
    }
    __syncthreads();
    const cx<R> pv = aug[k * ld2 + k];
    if (tid == 0) {
      double px = (double)pv.x, py = (double)pv.y;
      ld.x += 0.5 * log(px * px + py * py);
      ld.y += atan2(py, px);
    }
    __syncthreads();
    for (int c = tid; c < ld2; c += nt) aug[k * ld2 + c] = div_c(aug[k * ld2 + c], pv);
    for (int i = tid; i < ns; i += nt) fac[i] = (i == k) ? mk<R>(R(0), R(0)) : aug[i * ld2 + k];
    __syncthreads();
    for (int e = tid; e < ns * ld2; e += nt) {
      int i = e / ld2, c = e - i * ld2;
      if (i == k) continue;
      aug[e] = sub_mul(aug[e], fac[i], aug[k * ld2 + c]);
    }
    __syncthreads();
  }
  const int sing = singular;
  if (tid == 0) {
    double2 out = ld;
    if (sing) out = make_double2(-INFINITY, 0.0);
    else if (nswap) out.y += 3.141592653589793;
    logdet[2 * w + sig] = out;
  }
  if (Ainv_out) {
    double2* Ao = Ainv_out + ((long)w * 2 + sig) * nmax * nmax;
    for (int e = tid; e < ns * ns; e += nt) {
      int a = e / ns, b = e - a * ns;
      cx<R> v = aug[a * ld2 + ns + b];
      Ao[a * nmax + b] = sing ? make_double2(0.0, 0.0) : make_double2((double)v.x, (double)v.y);
    }
  }
  // Theta[:, a] = sum_b Phi[:, b] Ainv[b][a]
  T* Tr = Theta + ((long)w * 2 + 0) * N * M + (long)j0 * M;
  T* Ti = Theta + ((long)w * 2 + 1) * N * M + (long)j0 * M;
  for (int e = tid; e < M * ns; e += nt) {
    int a = e / M, k = e - a * M;
    R sr = 0, si = 0;
    if (!sing) {
      for (int b = 0; b < ns; ++b) {
        const T* pr = Pw + ((long)(j0 + b) * 2 + 0) * M;
        R xr = (R)pr[k], xi = (R)pr[M + k];
        cx<R> iv = aug[b * ld2 + ns + a];
        sr += xr * iv.x - xi * iv.y;
        si += xr * iv.y + xi * iv.x;
      }
    }
    Tr[(long)a * M + k] = (T)sr;
    Ti[(long)a * M + k] = (T)si;
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
                               const double2* __restrict__ lw, double dtau,
                               double e_shift, double* __restrict__ weight,
                               double2* __restrict__ logO) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double2 ln = logO_new[w];
  double2 lnR = csub(ln, logO[w]);
  double2 l = lw[w];
  double lnI_re = lnR.x + l.x + dtau * e_shift;
  double wt = weight[w];
  double out = 0.0;
  if (wt != 0.0) {
    out = wt * exp(lnI_re) * fmax(0.0, cos(lnR.y));
    if (!isfinite(out)) out = 0.0;
  }
  weight[w] = out;
  logO[w] = ln;
}

// --------------------------------------------------------------- K10
// Modified Gram-Schmidt per walker (both spins in turn), right-looking: once
// column j is normalised it is projected out of every later column, one warp
// per column. Arithmetic in R; ln det R = sum_j ln r_jj accumulated in FP64.
template <typename T, typename R>
__global__ void mgs_kernel(int M, int n_up, int n_dn, T* __restrict__ Phi,
                           double2* __restrict__ logO) {
  extern __shared__ unsigned char smem_raw[];
  cx<R>* Q = reinterpret_cast<cx<R>*>(smem_raw);    // [ns][M]
  __shared__ R rjj;
  const int w = blockIdx.x;
  const int N = n_up + n_dn;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  double logr = 0.0;
  for (int sig = 0; sig < 2; ++sig) {
    const int ns = sig ? n_dn : n_up;
    const int j0 = sig ? n_up : 0;
    if (ns == 0) continue;
    T* Pw = Phi + ((long)w * N + j0) * 2 * M;
    __syncthreads();
    for (int e = tid; e < ns * M; e += nt) {
      int b = e / M, k = e - b * M;
      Q[e] = mk<R>((R)Pw[(b * 2 + 0) * M + k], (R)Pw[(b * 2 + 1) * M + k]);
    }
    __syncthreads();
    for (int j = 0; j < ns; ++j) {
      if (wid == 0) {
        R s = 0;
        for (int k = lane; k < M; k += 32) {
          cx<R> q = Q[j * M + k];
          s += q.x * q.x + q.y * q.y;
        }
        s = warp_sum(s);
        if (lane == 0) rjj = sqrt(s);
      }
      __syncthreads();
      const R r = rjj;
      if (tid == 0) logr += log((double)r);
      for (int k = tid; k < M; k += nt) {
        cx<R> q = Q[j * M + k];
        Q[j * M + k] = mk<R>(q.x / r, q.y / r);
      }
      __syncthreads();
      for (int c = j + 1 + wid; c < ns; c += nw) {
        R sr = 0, si = 0;   // r_jc = q_j^H a_c
        for (int k = lane; k < M; k += 32) {
          cx<R> q = Q[j * M + k], a = Q[c * M + k];
          sr += q.x * a.x + q.y * a.y;
          si += q.x * a.y - q.y * a.x;
        }
        sr = warp_sum(sr);
        si = warp_sum(si);
        for (int k = lane; k < M; k += 32) {
          cx<R> q = Q[j * M + k], a = Q[c * M + k];
          Q[c * M + k] = mk<R>(a.x - (sr * q.x - si * q.y), a.y - (sr * q.y + si * q.x));
        }
      }
      __syncthreads();
    }
    for (int e = tid; e < ns * M; e += nt) {
      int b = e / M, k = e - b * M;
      Pw[(b * 2 + 0) * M + k] = (T)Q[e].x;
      Pw[(b * 2 + 1) * M + k] = (T)Q[e].y;
    }
  }
  if (tid == 0) logO[w].x -= logr;
}

// --------------------------------------------------------------- K9 epilogue
template <typename T>
__global__ void energy_reduce_kernel(int M, int n_up, int n_dn, int n_chol,
                                     const T* __restrict__ X, long ldx,
                                     const T* __restrict__ Theta,
                                     const T* __restrict__ Z, int W,
                                     double2* __restrict__ eloc) {
  __shared__ double red[32];
  const int w = blockIdx.x;
  const int N = n_up + n_dn;
  const T* Xr = X + (2L * w) * ldx;
  const T* Xi = Xr + ldx;
  double cr = 0.0, ci = 0.0;
  for (int g = threadIdx.x; g < n_chol; g += blockDim.x) {
    double a = Xr[g], b = Xi[g];
    cr += 0.5 * (a * a - b * b);
    ci += a * b;
  }
  double er = 0.0, ei = 0.0;
  long zoff = 0;
  for (int sig = 0; sig < 2; ++sig) {
    const int ns = sig ? n_dn : n_up;
    const int j0 = sig ? n_up : 0;
    const long J = (long)ns * M;
    const T* tr = Theta + (2L * w) * N * M + (long)j0 * M;
    const T* ti = tr + (long)N * M;
    const T* zr = Z + zoff + (2L * w) * J;
    const T* zi = zr + J;
    for (long e = threadIdx.x; e < J; e += blockDim.x) {
      double a = tr[e], b = ti[e], p = zr[e], q = zi[e];
      er += 0.5 * (a * p - b * q);
      ei += 0.5 * (a * q + b * p);
    }
    zoff += 2L * W * J;
  }
  double tr_ = block_sum(cr + er, red);
  double ti_ = block_sum(ci + ei, red);
  if (threadIdx.x == 0)
    eloc[w] = make_double2(tr_ + (double)Xr[n_chol], ti_ + (double)Xi[n_chol]);
}

__global__ void mixed_energy_kernel(int W, const double* __restrict__ weight,
                                    const double2* __restrict__ eloc, double step,
                                    double2* __restrict__ hist, int slot,
                                    double* out_scalar) {
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
    if (hist) hist[slot] = make_double2(step, e);
    if (out_scalar) *out_scalar = e;
  }
}

// --------------------------------------------------------------- K11
constexpr int kScanBlock = 32;

__global__ void comb_kernel(int W, const double* __restrict__ weight, uint32_t k0,
                            uint32_t k1, int run_id, uint32_t step,
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
                                  double* __restrict__ yx) {
  // Yx[(a,k)][(b,l)] = -Gram[(b,k)][(a,l)],  J = n * M
  long J = (long)n * M;
  long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= J * J) return;
  long row = e / J, col = e - row * J;
  int a = (int)(row / M), k = (int)(row - (long)a * M);
  int b = (int)(col / M), l = (int)(col - (long)b * M);
  yx[e] = -gram[((long)b * M + k) * J + (long)a * M + l];
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
                          double sqdt, double cap, uint64_t seed, int run_id,
                          long step, T* S, T* xbar, double2* lw) {
  fields_kernel<T><<<W, 128, 0, st>>>(n_chol, X, ldx, sqdt, cap, (uint32_t)seed,
                                      (uint32_t)(seed >> 32), run_id, (uint32_t)step,
                                      S, xbar, lw);
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

template <typename T>
cudaError_t launch_overlap(cudaStream_t st, int W, int M, int n_up, int n_dn,
                           const T* Phi, const T* PsiT, T* Theta, double2* logdet,
                           double2* Ainv, bool fp64_compute) {
  int nmax = n_up > n_dn ? n_up : n_dn;
  dim3 grid(W, 2);
  if (fp64_compute) {
    static const size_t cap = allow_big_smem(overlap_kernel<T, double>);
    size_t smem = sizeof(double2) * ((size_t)nmax * 2 * nmax + nmax);
    if (smem > cap) return cudaErrorInvalidValue;
    overlap_kernel<T, double><<<grid, 256, smem, st>>>(M, n_up, n_dn, Phi, PsiT, Theta,
                                                      logdet, Ainv, nmax);
  } else {
    static const size_t cap = allow_big_smem(overlap_kernel<T, float>);
    size_t smem = sizeof(float2) * ((size_t)nmax * 2 * nmax + nmax);
    if (smem > cap) return cudaErrorInvalidValue;
    overlap_kernel<T, float><<<grid, 256, smem, st>>>(M, n_up, n_dn, Phi, PsiT, Theta,
                                                     logdet, Ainv, nmax);
  }
  return cudaGetLastError();
}

cudaError_t launch_weights(cudaStream_t st, int W, const double2* logO_new,
                           const double2* lw, double dtau, double e_shift,
                           double* weight, double2* logO) {
  weights_kernel<<<blocks_for(W, 256), 256, 0, st>>>(W, logO_new, lw, dtau, e_shift,
                                                     weight, logO);
  return cudaGetLastError();
}

cudaError_t launch_logdet_sum(cudaStream_t st, int W, const double2* logdet,
                              double2* out) {
  logdet_sum_kernel<<<blocks_for(W, 256), 256, 0, st>>>(W, logdet, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mgs(cudaStream_t st, int W, int M, int n_up, int n_dn, T* Phi,
                       double2* logO, bool fp64_compute) {
  int nmax = n_up > n_dn ? n_up : n_dn;
  if (fp64_compute) {
    static const size_t cap = allow_big_smem(mgs_kernel<T, double>);
    size_t smem = sizeof(double2) * (size_t)nmax * M;
    if (smem > cap) return cudaErrorInvalidValue;
    mgs_kernel<T, double><<<W, 256, smem, st>>>(M, n_up, n_dn, Phi, logO);
  } else {
    static const size_t cap = allow_big_smem(mgs_kernel<T, float>);
    size_t smem = sizeof(float2) * (size_t)nmax * M;
    if (smem > cap) return cudaErrorInvalidValue;
    mgs_kernel<T, float><<<W, 256, smem, st>>>(M, n_up, n_dn, Phi, logO);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_energy_reduce(cudaStream_t st, int W, int M, int n_up, int n_dn,
                                 int n_chol, const T* X, long ldx, const T* Theta,
                                 const T* Z, double2* eloc) {
  energy_reduce_kernel<T><<<W, 256, 0, st>>>(M, n_up, n_dn, n_chol, X, ldx, Theta, Z,
                                             W, eloc);
  return cudaGetLastError();
}

cudaError_t launch_mixed_energy(cudaStream_t st, int W, const double* weight,
                                const double2* eloc, double step, double2* hist,
                                int slot, double* out_scalar) {
  mixed_energy_kernel<<<1, 1024, 0, st>>>(W, weight, eloc, step, hist, slot, out_scalar);
  return cudaGetLastError();
}

cudaError_t launch_comb(cudaStream_t st, int W, const double* weight, uint64_t seed,
                        int run_id, long step, int* parent, double* scratch,
                        double* wnew, int* status) {
  static const size_t smem_cap = allow_big_smem(comb_kernel);
  int nb = (W + kScanBlock - 1) / kScanBlock;
  size_t smem = sizeof(double) * 2 * (size_t)nb;
  if (smem > smem_cap) return cudaErrorInvalidValue;
  comb_kernel<<<1, 1024, smem, st>>>(W, weight, (uint32_t)seed, (uint32_t)(seed >> 32),
                                     run_id, (uint32_t)step, parent, scratch, wnew,
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
                              double* yx) {
  long J = (long)n * M;
  yx_permute_kernel<<<blocks_for(J * J, 256), 256, 0, st>>>(n, M, gram, yx);
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

cudaError_t launch_axpy_d(cudaStream_t st, long n, double a, const double* x, double* y) {
  axpy_d_kernel<<<blocks_for(n, 256), 256, 0, st>>>(n, a, x, y);
  return cudaGetLastError();
}

#define AFQMC_INST(T)                                                                    \
  template cudaError_t launch_fields<T>(cudaStream_t, int, int, const T*, long, double, \
                                        double, uint64_t, int, long, T*, T*, double2*); \
  template cudaError_t launch_taylor<T>(cudaStream_t, int, int, int, int, const T*,     \
                                        const T*, T*);                                  \
  template cudaError_t launch_overlap<T>(cudaStream_t, int, int, int, int, const T*,    \
                                         const T*, T*, double2*, double2*, bool);       \
  template cudaError_t launch_mgs<T>(cudaStream_t, int, int, int, int, T*, double2*,    \
                                     bool);                                             \
  template cudaError_t launch_energy_reduce<T>(cudaStream_t, int, int, int, int, int,   \
                                               const T*, long, const T*, const T*,      \
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
