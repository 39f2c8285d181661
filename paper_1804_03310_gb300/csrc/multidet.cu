// Multi-determinant trials, |Psi_T> = sum_i c_i |D_i> with orthonormal
// determinants that differ from the reference D_0 by E_i <= 4 excitations per
// spin (Sec. III). With A_0 = D_0^T Phi, Theta_0 = Phi A_0^-1 and
// Omega = C_act^T Theta_0 (active orbitals: every orbital occupied in some
// determinant), the Sherman-Morrison-Woodbury identities of Eq. 4 give, for a
// determinant whose holes h_1..h_E (positions in the reference) are filled
// by particles p_1..p_E:
//   det(A_i) / det(A_0) = det K_i,   K_i[l][m] = Omega[p_l][h_m],
//   Theta_i = Theta_0 - Theta_0[:, h] K_i^-1 (Omega[p, :] - E_h^T).
// The mixed Green's function needed by the force bias is linear in the
// Theta_i, so G^T = C_act Gamma with Gamma = Theta_0 Lambda and
//   Lambda = sum_i w_i [S_i^T - E_h K_i^-1 (Omega[p, :] - E_h^T) S_i^T],
// w_i = c_i^* O_i / O_T, S_i placing determinant i's columns on its orbitals.
// The local energy is not linear in the Theta_i and is summed determinant by
// determinant.
#include "common.cuh"
#include "kernels.h"
#include "multidet.h"

namespace afqmc {

namespace {

constexpr int EMAX = MD_EMAX;

template <typename R>
struct __align__(2 * sizeof(R)) cplx {
  R x, y;
};
template <typename R>
__device__ __forceinline__ cplx<R> cm(R a, R b) {
  cplx<R> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename R>
__device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return cm<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R>
__device__ __forceinline__ cplx<R> cadd(cplx<R> a, cplx<R> b) {
  return cm<R>(a.x + b.x, a.y + b.y);
}
template <typename R>
__device__ __forceinline__ cplx<R> csub(cplx<R> a, cplx<R> b) {
  return cm<R>(a.x - b.x, a.y - b.y);
}
template <typename R>
__device__ __forceinline__ cplx<R> cdiv(cplx<R> a, cplx<R> b) {
  const R d = b.x * b.x + b.y * b.y;
  return cm<R>((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__host__ __device__ __forceinline__ int stage_ld(int M) { return M | 1; }

// det and inverse of an E x E complex matrix (E <= EMAX) by Gauss-Jordan with
// partial pivoting; returns det, writes the inverse (row-major EMAX stride).
template <typename R>
__device__ cplx<R> small_inverse(int E, cplx<R> (&a)[EMAX][EMAX], cplx<R> (&inv)[EMAX][EMAX]) {
  cplx<R> det = cm<R>(R(1), R(0));
  for (int i = 0; i < EMAX; ++i)
    for (int j = 0; j < EMAX; ++j) inv[i][j] = cm<R>(i == j ? R(1) : R(0), R(0));
  for (int k = 0; k < E; ++k) {
    int p = k;
    R best = a[k][k].x * a[k][k].x + a[k][k].y * a[k][k].y;
    for (int i = k + 1; i < E; ++i) {
      const R m = a[i][k].x * a[i][k].x + a[i][k].y * a[i][k].y;
      if (m > best) { best = m; p = i; }
    }
    if (!(best > R(0))) return cm<R>(R(0), R(0));
    if (p != k) {
      for (int j = 0; j < EMAX; ++j) {
        cplx<R> t = a[k][j]; a[k][j] = a[p][j]; a[p][j] = t;
        t = inv[k][j]; inv[k][j] = inv[p][j]; inv[p][j] = t;
      }
      det = cm<R>(-det.x, -det.y);
    }
    const cplx<R> pv = a[k][k];
    det = cmul(det, pv);
    for (int j = 0; j < EMAX; ++j) {
      a[k][j] = cdiv(a[k][j], pv);
      inv[k][j] = cdiv(inv[k][j], pv);
    }
    for (int i = 0; i < E; ++i) {
      if (i == k) continue;
      const cplx<R> f = a[i][k];
      for (int j = 0; j < EMAX; ++j) {
        a[i][j] = csub(a[i][j], cmul(f, a[k][j]));
        inv[i][j] = csub(inv[i][j], cmul(f, inv[k][j]));
      }
    }
  }
  return det;
}

// K_i for one spin from Omega [nact][ns] (smem): K[l][m] = Omega[p_l][h_m];
// returns det K and writes K^-1 (identity and det 1 when E = 0).
template <typename R>
__device__ __noinline__ cplx<R> det_k(int E, const int* p, const int* h, const cplx<R>* Om,
                                      int ns, cplx<R> (&inv)[EMAX][EMAX]) {
  cplx<R> a[EMAX][EMAX];
  for (int l = 0; l < EMAX; ++l)
    for (int m = 0; m < EMAX; ++m)
      a[l][m] = (l < E && m < E) ? Om[p[l] * ns + h[m]] : cm<R>(R(0), R(0));
  return small_inverse<R>(E, a, inv);
}

// Shared layout of the per-walker multi-determinant kernels.
template <typename R>
struct MdSmem {
  cplx<R>* Q[2];    // Theta_0 per spin, [a][ldq] (column a, basis row k)
  cplx<R>* Om[2];   // Omega per spin, [nact][ns]
  cplx<R>* wt;      // normalised determinant weights w_i [ndet]
  double2* term;    // c_i^* r_i^up r_i^dn [ndet]
  __host__ __device__ static size_t bytes(int M, int nu, int nd, int na_u, int na_d, int ndet) {
    const size_t ldq = (size_t)stage_ld(M);
    return sizeof(cplx<R>) * ((size_t)(nu + nd) * ldq + (size_t)na_u * nu + (size_t)na_d * nd +
                              (size_t)ndet) +
           sizeof(double2) * (size_t)ndet + 64;
  }
  __device__ void carve(unsigned char* raw, int M, int nu, int nd, int na_u, int na_d, int ndet) {
    const int ldq = stage_ld(M);
    cplx<R>* p = reinterpret_cast<cplx<R>*>(raw);
    Q[0] = p; p += (long)nu * ldq;
    Q[1] = p; p += (long)nd * ldq;
    Om[0] = p; p += (long)na_u * nu;
    Om[1] = p; p += (long)na_d * nd;
    wt = p; p += ndet;
    uintptr_t u = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    term = reinterpret_cast<double2*>(u);
  }
};

// C = K^-1 (Omega[p] - E_h^T) for one determinant and spin, rows l < E of
// length ns, from the inverse det_k wrote.
template <typename R>
__device__ void fill_c(int E, const int* p, const int* h, const cplx<R>* Om, int ns,
                       const cplx<R> (&inv)[EMAX][EMAX], cplx<R>* C) {
  for (int l = 0; l < E; ++l)
    for (int a = 0; a < ns; ++a) {
      cplx<R> s = cm<R>(R(0), R(0));
      for (int m = 0; m < E; ++m) {
        cplx<R> r = Om[p[m] * ns + a];
        if (a == h[m]) r.x -= R(1);
        s = cadd(s, cmul(inv[l][m], r));
      }
      C[l * ns + a] = s;
    }
}

// Phases shared by the step kernel and the energy kernel: stage Theta_0,
// form Omega, the ratios, O_T and the normalised weights. Returns ln O_T.
// With ctab, also the C table: determinant i's rows for the up spin at
// ctab + coff_i, for the down spin after them.
template <typename T, typename R>
__device__ double2 md_weights(const MdTables& tb, int M, int nu, int nd, const T* Theta,
                              long ldt, long dn_off, const double2* logdet0, int w,
                              MdSmem<R>& sm, double* red, cplx<R>* ctab = nullptr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ldq = stage_ld(M);
  const int nsv[2] = {nu, nd};
  for (int sg = 0; sg < 2; ++sg) {
    const int ns = nsv[sg];
    const T* tr = Theta + (2L * w) * ldt + (sg ? dn_off : 0);
    const T* ti = tr + ldt;
    for (int e = tid; e < ns * M; e += nt) {
      const int a = e / M, k = e - a * M;
      sm.Q[sg][a * ldq + k] = cm<R>((R)tr[(long)a * M + k], (R)ti[(long)a * M + k]);
    }
  }
  __syncthreads();
  for (int sg = 0; sg < 2; ++sg) {                 // Omega = C_act^T Theta_0
    const int ns = nsv[sg], na = tb.nact[sg];
    const T* Ct = (const T*)tb.CactT[sg];
    for (int e = tid; e < na * ns; e += nt) {
      const int q = e / ns, a = e - q * ns;
      const T* cq = Ct + (long)q * M;
      const cplx<R>* th = sm.Q[sg] + a * ldq;
      R sr = 0, si = 0;
      for (int k = 0; k < M; ++k) {
        const R c = (R)cq[k];
        sr = fma(c, th[k].x, sr);
        si = fma(c, th[k].y, si);
      }
      sm.Om[sg][q * ns + a] = cm<R>(sr, si);
    }
  }
  __syncthreads();
  double sr = 0.0, si = 0.0;
  for (int i = tid; i < tb.ndet; i += nt) {        // c_i^* det K_i^up det K_i^dn
    const MdDet d = tb.dets[i];
    cplx<R> inv[EMAX][EMAX];
    const cplx<R> ru = nu ? det_k<R>(d.E[0], d.p[0], d.h[0], sm.Om[0], nu, inv) : cm<R>(R(1), R(0));
    if (ctab && nu) fill_c<R>(d.E[0], d.p[0], d.h[0], sm.Om[0], nu, inv, ctab + d.coff);
    const cplx<R> rd = nd ? det_k<R>(d.E[1], d.p[1], d.h[1], sm.Om[1], nd, inv) : cm<R>(R(1), R(0));
    if (ctab && nd)
      fill_c<R>(d.E[1], d.p[1], d.h[1], sm.Om[1], nd, inv, ctab + d.coff + (long)d.E[0] * nu);
    const double ax = (double)ru.x * rd.x - (double)ru.y * rd.y;
    const double ay = (double)ru.x * rd.y + (double)ru.y * rd.x;
    const double2 cc = tb.cconj[i];
    const double2 t = make_double2(cc.x * ax - cc.y * ay, cc.x * ay + cc.y * ax);
    sm.term[i] = t;
  }
  __syncthreads();
  // fixed-order sums: each thread a strided subset, then the block in order
  for (int i = tid; i < tb.ndet; i += nt) {
    sr += sm.term[i].x;
    si += sm.term[i].y;
  }
  sr = block_sum(sr, red);
  si = block_sum(si, red);
  const double mag2 = sr * sr + si * si;
  for (int i = tid; i < tb.ndet; i += nt) {        // w_i = term_i / S
    const double2 t = sm.term[i];
    sm.wt[i] = cm<R>((R)((t.x * sr + t.y * si) / mag2), (R)((t.y * sr - t.x * si) / mag2));
  }
  __syncthreads();
  double2 lo;
  lo.x = logdet0[2 * w].x + logdet0[2 * w + 1].x + 0.5 * log(mag2);
  lo.y = logdet0[2 * w].y + logdet0[2 * w + 1].y + atan2(si, sr);
  return lo;
}

// ------------------------------------------------------------------ step
// HC: the C_i table fits in shared memory (after Lambda) and the Lambda rows
// read it instead of inverting K_i per row and determinant.
template <typename T, typename R, bool HC>
__global__ void md_step_kernel(MdTables tb, int M, int nu, int nd, const T* __restrict__ Theta,
                               long ldt, long dn_off, const double2* __restrict__ logdet0,
                               double2* __restrict__ logO_new, T* __restrict__ Gamma,
                               long ldg, long gdn_off) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[32];
  MdSmem<R> sm;
  sm.carve(smem_raw, M, nu, nd, tb.nact[0], tb.nact[1], tb.ndet);
  const int w = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  // Lambda rows are accumulated warp by warp (one row of one spin per warp
  // pass, lanes over positions); every entry has a single owning lane, and
  // determinants are visited in order, so the sums are deterministic.
  cplx<R>* Lam = reinterpret_cast<cplx<R>*>(smem_raw + MdSmem<R>::bytes(M, nu, nd, tb.nact[0],
                                                                         tb.nact[1], tb.ndet));
  cplx<R>* Lams[2] = {Lam, Lam + (long)nu * tb.nact[0]};
  cplx<R>* Ctab = Lam + (long)nu * tb.nact[0] + (long)nd * tb.nact[1];
  const double2 lo = md_weights<T, R>(tb, M, nu, nd, Theta, ldt, dn_off, logdet0, w, sm, red,
                                      HC ? Ctab : nullptr);
  if (tid == 0) logO_new[w] = lo;
  const int nsv[2] = {nu, nd};
  for (int e = tid; e < nu * tb.nact[0] + nd * tb.nact[1]; e += nt) Lam[e] = cm<R>(R(0), R(0));
  __syncthreads();
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  if (HC) {
    for (int row = wid; row < nu + nd; row += nw) {
      const int sg = row >= nu;
      const int h = row - (sg ? nu : 0);
      const int ns = nsv[sg], na = tb.nact[sg];
      cplx<R>* Lr = Lams[sg] + (long)h * na;
      const int* ract = tb.ract[sg];
      // determinants without a hole at h add w_i at the reference orbital,
      // an entry no other determinant touches for this row
      cplx<R> wsum = cm<R>(R(0), R(0));
      for (int i = 0; i < tb.ndet; ++i) {
        const MdDet* dp = tb.dets + i;
        const int E = dp->E[sg];
        int l = -1;
        for (int t = 0; t < E; ++t)
          if (dp->h[sg][t] == h) l = t;
        const cplx<R> wi = sm.wt[i];
        if (l < 0) {
          wsum = cadd(wsum, wi);
          continue;
        }
        const cplx<R>* C = Ctab + dp->coff + (sg ? (long)dp->E[0] * nu : 0) + (long)l * ns;
        for (int a = lane; a < ns; a += 32) {
          int q = ract[a];
          for (int m = 0; m < E; ++m)
            if (a == dp->h[sg][m]) q = dp->p[sg][m];
          cplx<R> v = cm<R>(R(0), R(0));
          if (a == h) v = wi;
          v = csub(v, cmul(wi, C[a]));
          Lr[q] = cadd(Lr[q], v);
        }
      }
      if (lane == 0) Lr[ract[h]] = cadd(Lr[ract[h]], wsum);
    }
  }
  for (int row = HC ? nu + nd : wid; row < nu + nd; row += nw) {
    const int sg = row >= nu;
    const int h = row - (sg ? nu : 0);
    const int ns = nsv[sg], na = tb.nact[sg];
    cplx<R>* Lr = Lams[sg] + (long)h * na;
    const cplx<R>* Om = sm.Om[sg];
    const int* ract = tb.ract[sg];
    for (int i = 0; i < tb.ndet; ++i) {
      const MdDet d = tb.dets[i];
      const cplx<R> wi = sm.wt[i];
      const int E = d.E[sg];
      int l = -1;
      for (int t = 0; t < E; ++t)
        if (d.h[sg][t] == h) l = t;
      if (l < 0) {
        if (lane == 0) Lr[ract[h]] = cadd(Lr[ract[h]], wi);
        continue;
      }
      cplx<R> inv[EMAX][EMAX];
      det_k<R>(E, d.p[sg], d.h[sg], Om, ns, inv);
      for (int a = lane; a < ns; a += 32) {
        cplx<R> ca = cm<R>(R(0), R(0));    // sum_m Kinv[l][m] (Omega[p_m][a] - [a == h_m])
        int q = ract[a];
        for (int m = 0; m < E; ++m) {
          cplx<R> r = Om[d.p[sg][m] * ns + a];
          if (a == d.h[sg][m]) {
            r.x -= R(1);
            q = d.p[sg][m];
          }
          ca = cadd(ca, cmul(inv[l][m], r));
        }
        cplx<R> v = cm<R>(R(0), R(0));
        if (a == h) v = wi;
        v = csub(v, cmul(wi, ca));
        Lr[q] = cadd(Lr[q], v);
      }
    }
  }
  __syncthreads();
  // Gamma = Theta_0 Lambda, written per spin at [q][k]
  const int ldq = stage_ld(M);
  for (int sg = 0; sg < 2; ++sg) {
    const int ns = nsv[sg], na = tb.nact[sg];
    T* gr = Gamma + (2L * w) * ldg + (sg ? gdn_off : 0);
    T* gi = gr + ldg;
    for (int e = tid; e < na * M; e += nt) {
      const int q = e / M, k = e - q * M;
      R sr = 0, si = 0;
      for (int a = 0; a < ns; ++a) {
        const cplx<R> th = sm.Q[sg][a * ldq + k];
        const cplx<R> lm = Lams[sg][(long)a * na + q];
        sr += th.x * lm.x - th.y * lm.y;
        si += th.x * lm.y + th.y * lm.x;
      }
      gr[(long)q * M + k] = (T)sr;
      gi[(long)q * M + k] = (T)si;
    }
  }
}

// ------------------------------------------------------------------ energy
// E_L = sum_i w_i E_i with, per spin s and Cholesky vector g,
//   E_i = sum_s tr M_iG + 1/2 sum_g [(sum_s tr M_ig)^2 - sum_s tr M_ig^2],
// M_ig = (L_g Theta_i)[rows of det i's orbitals] (N x N), and g = G the
// one-body matrix. For each g the block forms P = L^act_g Theta_0 (active
// orbital x reference position) and V[q][c] = sum_b P[q][b] P[r_b][c]
// (r_b: reference orbital at position b). With rho(a) det i's orbital at
// position a, C = K_i^-1 (Omega[p] - E_h^T) and B0 = P[rho], B1 = P[rho, h]:
//   M = B0 - B1 C,  tr M^2 = tr B0^2 - 2 tr(C B0 B1) + tr((C B1)^2),
// and every sum over all positions reduces to V plus O(E) corrections, so a
// determinant costs O(N E^2) per g. One thread per determinant.
template <typename T, typename R>
__global__ void md_energy_kernel(MdTables tb, int M, int nu, int nd, int G,
                                 const T* __restrict__ Theta, long ldt, long dn_off,
                                 const double2* __restrict__ logdet0,
                                 const T* __restrict__ LtilA, long ldg, long gdn_off,
                                 double2* __restrict__ eloc) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[32];
  MdSmem<R> sm;
  sm.carve(smem_raw, M, nu, nd, tb.nact[0], tb.nact[1], tb.ndet);
  const int w = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  md_weights<T, R>(tb, M, nu, nd, Theta, ldt, dn_off, logdet0, w, sm, red);
  cplx<R>* P0 = reinterpret_cast<cplx<R>*>(smem_raw + MdSmem<R>::bytes(M, nu, nd, tb.nact[0],
                                                                       tb.nact[1], tb.ndet));
  cplx<R>* Ps[2] = {P0, P0 + (long)tb.nact[0] * nu};
  cplx<R>* V0 = P0 + (long)tb.nact[0] * nu + (long)tb.nact[1] * nd;
  cplx<R>* Vs[2] = {V0, V0 + (long)tb.nact[0] * nu};
  const int nsv[2] = {nu, nd};
  const int ldq = stage_ld(M);
  const int dets_per_thread = (tb.ndet + nt - 1) / nt;
  double e_re[MD_MAX_DET_PER_THREAD], e_im[MD_MAX_DET_PER_THREAD];
  for (int u = 0; u < MD_MAX_DET_PER_THREAD; ++u) { e_re[u] = 0.0; e_im[u] = 0.0; }
  for (int g = 0; g <= G; ++g) {
    __syncthreads();
    for (int sg = 0; sg < 2; ++sg) {               // P = L^act_g Theta_0
      const int ns = nsv[sg], na = tb.nact[sg];
      const T* Lg = LtilA + (long)g * ldg + (sg ? gdn_off : 0);
      for (int e = tid; e < na * ns; e += nt) {
        const int q = e / ns, a = e - q * ns;
        const T* lq = Lg + (long)q * M;
        const cplx<R>* th = sm.Q[sg] + a * ldq;
        R sr = 0, si = 0;
        for (int k = 0; k < M; ++k) {
          const R l = (R)lq[k];
          sr = fma(l, th[k].x, sr);
          si = fma(l, th[k].y, si);
        }
        Ps[sg][q * ns + a] = cm<R>(sr, si);
      }
    }
    __syncthreads();
    if (g < G) {
      for (int sg = 0; sg < 2; ++sg) {             // V[q][c] = sum_b P[q][b] P[r_b][c]
        const int ns = nsv[sg], na = tb.nact[sg];
        const cplx<R>* P = Ps[sg];
        const int* ract = tb.ract[sg];
        for (int e = tid; e < na * ns; e += nt) {
          const int q = e / ns, cc = e - q * ns;
          cplx<R> s = cm<R>(R(0), R(0));
          for (int b = 0; b < ns; ++b) s = cadd(s, cmul(P[q * ns + b], P[ract[b] * ns + cc]));
          Vs[sg][q * ns + cc] = s;
        }
      }
      __syncthreads();
    }
    for (int u = 0; u < dets_per_thread; ++u) {
      const int i = tid + u * nt;
      if (i >= tb.ndet) break;
      const MdDet d = tb.dets[i];
      cplx<R> tr_tot = cm<R>(R(0), R(0));
      cplx<R> sq_tot = cm<R>(R(0), R(0));
      for (int sg = 0; sg < 2; ++sg) {
        const int ns = nsv[sg];
        if (ns == 0) continue;
        const int E = d.E[sg];
        const cplx<R>* P = Ps[sg];
        const cplx<R>* Vm = Vs[sg];
        const cplx<R>* Om = sm.Om[sg];
        const int* ract = tb.ract[sg];
        cplx<R> inv[EMAX][EMAX];
        det_k<R>(E, d.p[sg], d.h[sg], Om, ns, inv);
        cplx<R> trM = cm<R>(R(0), R(0)), trB0sq = cm<R>(R(0), R(0));
        cplx<R> T2 = cm<R>(R(0), R(0));
        cplx<R> CB1[EMAX][EMAX];
        for (int l = 0; l < EMAX; ++l)
          for (int m = 0; m < EMAX; ++m) CB1[l][m] = cm<R>(R(0), R(0));
        for (int a = 0; a < ns; ++a) {
          int ra = ract[a];                          // rho(a)
          for (int m = 0; m < E; ++m)
            if (d.h[sg][m] == a) ra = d.p[sg][m];
          const cplx<R>* Pra = P + ra * ns;
          cplx<R> Ca[EMAX];                          // C[l][a]
          for (int l = 0; l < EMAX; ++l) {
            Ca[l] = cm<R>(R(0), R(0));
            for (int m = 0; m < E; ++m) {
              cplx<R> r = Om[d.p[sg][m] * ns + a];
              if (a == d.h[sg][m]) r.x -= R(1);
              Ca[l] = cadd(Ca[l], cmul(inv[l][m], r));
            }
          }
          // tr M: P[rho a][a] - sum_l P[rho a][h_l] C[l][a]
          cplx<R> v = Pra[a];
          for (int l = 0; l < E; ++l) v = csub(v, cmul(Pra[d.h[sg][l]], Ca[l]));
          trM = cadd(trM, v);
          if (g == G) continue;
          // tr B0^2: V[rho a][a] + sum_m P[rho a][h_m] (P[p_m][a] - P[r_hm][a])
          cplx<R> b2 = Vm[ra * ns + a];
          for (int m = 0; m < E; ++m) {
            const int hm = d.h[sg][m];
            b2 = cadd(b2, cmul(Pra[hm], csub(P[d.p[sg][m] * ns + a], P[ract[hm] * ns + a])));
          }
          trB0sq = cadd(trB0sq, b2);
          for (int l = 0; l < E; ++l) {
            const int hl = d.h[sg][l];
            // (B0 B1)[a][l] = V[rho a][h_l] + sum_m P[rho a][h_m] (P[p_m][h_l] - P[r_hm][h_l])
            cplx<R> bb = Vm[ra * ns + hl];
            for (int m = 0; m < E; ++m) {
              const int hm = d.h[sg][m];
              bb = cadd(bb, cmul(Pra[hm], csub(P[d.p[sg][m] * ns + hl], P[ract[hm] * ns + hl])));
            }
            T2 = cadd(T2, cmul(Ca[l], bb));
            for (int m = 0; m < E; ++m)              // (C B1)[l][m] += C[l][a] P[rho a][h_m]
              CB1[l][m] = cadd(CB1[l][m], cmul(Ca[l], Pra[d.h[sg][m]]));
          }
        }
        tr_tot = cadd(tr_tot, trM);
        if (g < G) {
          cplx<R> sq = csub(trB0sq, cm<R>(R(2) * T2.x, R(2) * T2.y));
          for (int l = 0; l < E; ++l)
            for (int m = 0; m < E; ++m) sq = cadd(sq, cmul(CB1[l][m], CB1[m][l]));
          sq_tot = cadd(sq_tot, sq);
        }
      }
      if (g == G) {
        e_re[u] += (double)tr_tot.x;
        e_im[u] += (double)tr_tot.y;
      } else {
        const double xr = tr_tot.x, xi = tr_tot.y;
        e_re[u] += 0.5 * ((xr * xr - xi * xi) - (double)sq_tot.x);
        e_im[u] += 0.5 * (2.0 * xr * xi - (double)sq_tot.y);
      }
    }
  }
  // E_L = sum_i w_i E_i, in determinant order per thread, then the block
  double sr = 0.0, si = 0.0;
  for (int u = 0; u < dets_per_thread; ++u) {
    const int i = tid + u * nt;
    if (i >= tb.ndet) break;
    const cplx<R> wi = sm.wt[i];
    sr += (double)wi.x * e_re[u] - (double)wi.y * e_im[u];
    si += (double)wi.x * e_im[u] + (double)wi.y * e_re[u];
  }
  sr = block_sum(sr, red);
  si = block_sum(si, red);
  if (tid == 0) eloc[w] = make_double2(sr, si);
}

// One spin's contribution to E_i for one Cholesky vector, with E = the
// determinant's excitation count as a compile-time constant (the arrays stay
// in registers) and C = K_i^-1 (Omega[p] - E_h^T) precomputed ([E][ns]).
// Same quantities as md_energy_kernel: tr M, and (when !last) tr M^2 =
// tr B0^2 - 2 tr(C B0 B1) + tr((C B1)^2). The differences
// D[m][l] = P[p_m][h_l] - P[r_{h_m}][h_l] do not depend on the position a.
template <int E, typename R>
__device__ __forceinline__ void md_spin_terms(const int* __restrict__ h,
                                              const int* __restrict__ p,
                                              const cplx<R>* __restrict__ C,
                                              const cplx<R>* __restrict__ P,
                                              const cplx<R>* __restrict__ Vm,
                                              const int* __restrict__ ract, int ns, bool last,
                                              cplx<R>& trM, cplx<R>& sq) {
  constexpr int E1 = E > 0 ? E : 1;
  int hh[E1], pp[E1], rh[E1];
#pragma unroll
  for (int m = 0; m < E; ++m) { hh[m] = h[m]; pp[m] = p[m]; rh[m] = ract[h[m]]; }
  cplx<R> D[E1][E1];
#pragma unroll
  for (int m = 0; m < E; ++m)
#pragma unroll
    for (int l = 0; l < E; ++l) D[m][l] = csub(P[pp[m] * ns + hh[l]], P[rh[m] * ns + hh[l]]);
  cplx<R> tm = cm<R>(R(0), R(0)), b0 = cm<R>(R(0), R(0)), t2 = cm<R>(R(0), R(0));
  cplx<R> CB1[E1][E1];
#pragma unroll
  for (int l = 0; l < E; ++l)
#pragma unroll
    for (int m = 0; m < E; ++m) CB1[l][m] = cm<R>(R(0), R(0));
  for (int a = 0; a < ns; ++a) {
    int ra = ract[a];                               // rho(a)
#pragma unroll
    for (int m = 0; m < E; ++m)
      if (a == hh[m]) ra = pp[m];
    const cplx<R>* Pra = P + ra * ns;
    cplx<R> ph[E1], Ca[E1];
#pragma unroll
    for (int m = 0; m < E; ++m) { ph[m] = Pra[hh[m]]; Ca[m] = C[m * ns + a]; }
    cplx<R> v = Pra[a];
#pragma unroll
    for (int l = 0; l < E; ++l) v = csub(v, cmul(ph[l], Ca[l]));
    tm = cadd(tm, v);
    if (last) continue;
    cplx<R> b2 = Vm[ra * ns + a];
#pragma unroll
    for (int m = 0; m < E; ++m)
      b2 = cadd(b2, cmul(ph[m], csub(P[pp[m] * ns + a], P[rh[m] * ns + a])));
    b0 = cadd(b0, b2);
#pragma unroll
    for (int l = 0; l < E; ++l) {
      cplx<R> bb = Vm[ra * ns + hh[l]];
#pragma unroll
      for (int m = 0; m < E; ++m) bb = cadd(bb, cmul(ph[m], D[m][l]));
      t2 = cadd(t2, cmul(Ca[l], bb));
#pragma unroll
      for (int m = 0; m < E; ++m) CB1[l][m] = cadd(CB1[l][m], cmul(Ca[l], ph[m]));
    }
  }
  trM = tm;
  if (!last) {
    cplx<R> s = csub(b0, cm<R>(R(2) * t2.x, R(2) * t2.y));
#pragma unroll
    for (int l = 0; l < E; ++l)
#pragma unroll
      for (int m = 0; m < E; ++m) s = cadd(s, cmul(CB1[l][m], CB1[m][l]));
    sq = s;
  } else {
    sq = cm<R>(R(0), R(0));
  }
}

template <typename R>
__device__ __forceinline__ void md_spin_dispatch(int E, const int* h, const int* p,
                                                 const cplx<R>* C, const cplx<R>* P,
                                                 const cplx<R>* Vm, const int* ract, int ns,
                                                 bool last, cplx<R>& trM, cplx<R>& sq) {
  switch (E) {
    case 0: md_spin_terms<0, R>(h, p, C, P, Vm, ract, ns, last, trM, sq); break;
    case 1: md_spin_terms<1, R>(h, p, C, P, Vm, ract, ns, last, trM, sq); break;
    case 2: md_spin_terms<2, R>(h, p, C, P, Vm, ract, ns, last, trM, sq); break;
    case 3: md_spin_terms<3, R>(h, p, C, P, Vm, ract, ns, last, trM, sq); break;
    default: md_spin_terms<4, R>(h, p, C, P, Vm, ract, ns, last, trM, sq); break;
  }
}

// Shared bytes the C_i table takes (determinant i's E_i^up rows of n_up, then
// E_i^dn rows of n_dn, at its offset coff_i) plus one FP64 complex
// accumulator per determinant for the energy kernel.
__host__ __device__ __forceinline__ size_t md_ctab_bytes(int ctot, int ndet, size_t csize) {
  // 15: the accumulators start on a 16-byte address
  return csize * (size_t)ctot + 15 + 16 * (size_t)ndet;
}

// The local energy of md_energy_kernel with the Cholesky-independent parts
// taken out of the loop over g: C_i = K_i^-1 (Omega[p] - E_h^T) per
// determinant and spin is formed once per walker into shared memory, and the
// per-g work runs with the excitation count as a compile-time constant.
template <typename T, typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) md_energy_hoisted_kernel(MdTables tb, int M, int nu, int nd, int G,
                                         const T* __restrict__ Theta, long ldt, long dn_off,
                                         const double2* __restrict__ logdet0,
                                         const T* __restrict__ LtilA, long ldg, long gdn_off,
                                         double2* __restrict__ eloc) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ double red[32];
  MdSmem<R> sm;
  sm.carve(smem_raw, M, nu, nd, tb.nact[0], tb.nact[1], tb.ndet);
  const int w = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;
  cplx<R>* P0 = reinterpret_cast<cplx<R>*>(smem_raw + MdSmem<R>::bytes(M, nu, nd, tb.nact[0],
                                                                       tb.nact[1], tb.ndet));
  cplx<R>* Ps[2] = {P0, P0 + (long)tb.nact[0] * nu};
  cplx<R>* V0 = P0 + (long)tb.nact[0] * nu + (long)tb.nact[1] * nd;
  cplx<R>* Vs[2] = {V0, V0 + (long)tb.nact[0] * nu};
  cplx<R>* Ctab = V0 + (long)tb.nact[0] * nu + (long)tb.nact[1] * nd;
  const size_t cbytes = sizeof(cplx<R>) * (size_t)tb.ctot;
  double2* eacc = reinterpret_cast<double2*>(
      ((uintptr_t)reinterpret_cast<unsigned char*>(Ctab) + cbytes + 15) & ~(uintptr_t)15);
  const int nsv[2] = {nu, nd};
  const int ldq = stage_ld(M);
  // the weights, and C_i = K_i^-1 (Omega[p] - E_h^T) once per walker
  md_weights<T, R>(tb, M, nu, nd, Theta, ldt, dn_off, logdet0, w, sm, red, Ctab);
  for (int i = tid; i < tb.ndet; i += nt) eacc[i] = make_double2(0.0, 0.0);
  MdDet* dets = reinterpret_cast<MdDet*>(eacc + tb.ndet);   // the table, read every pass
  for (int e = tid; e < tb.ndet * (int)(sizeof(MdDet) / sizeof(int)); e += nt)
    reinterpret_cast<int*>(dets)[e] = reinterpret_cast<const int*>(tb.dets)[e];
  for (int g = 0; g <= G; ++g) {
    __syncthreads();
    for (int sg = 0; sg < 2; ++sg) {               // P = L^act_g Theta_0
      const int ns = nsv[sg], na = tb.nact[sg];
      const T* Lg = LtilA + (long)g * ldg + (sg ? gdn_off : 0);
      for (int e = tid; e < na * ns; e += nt) {
        const int q = e / ns, a = e - q * ns;
        const T* lq = Lg + (long)q * M;
        const cplx<R>* th = sm.Q[sg] + a * ldq;
        R sr = 0, si = 0;
        for (int k = 0; k < M; ++k) {
          const R l = (R)lq[k];
          sr = fma(l, th[k].x, sr);
          si = fma(l, th[k].y, si);
        }
        Ps[sg][q * ns + a] = cm<R>(sr, si);
      }
    }
    __syncthreads();
    if (g < G) {
      for (int sg = 0; sg < 2; ++sg) {             // V[q][c] = sum_b P[q][b] P[r_b][c]
        const int ns = nsv[sg], na = tb.nact[sg];
        const cplx<R>* P = Ps[sg];
        const int* ract = tb.ract[sg];
        for (int e = tid; e < na * ns; e += nt) {
          const int q = e / ns, cc = e - q * ns;
          cplx<R> s = cm<R>(R(0), R(0));
          for (int b = 0; b < ns; ++b) s = cadd(s, cmul(P[q * ns + b], P[ract[b] * ns + cc]));
          Vs[sg][q * ns + cc] = s;
        }
      }
      __syncthreads();
    }
    for (int i = tid; i < tb.ndet; i += nt) {
      const MdDet* dp = dets + i;
      cplx<R> tr_tot = cm<R>(R(0), R(0)), sq_tot = cm<R>(R(0), R(0));
      for (int sg = 0; sg < 2; ++sg) {
        const int ns = nsv[sg];
        if (ns == 0) continue;
        cplx<R> trM, sq;
        md_spin_dispatch<R>(dp->E[sg], dp->h[sg], dp->p[sg],
                            Ctab + dp->coff + (sg ? (long)dp->E[0] * nu : 0),
                            Ps[sg], Vs[sg], tb.ract[sg], ns, g == G, trM, sq);
        tr_tot = cadd(tr_tot, trM);
        sq_tot = cadd(sq_tot, sq);
      }
      double2 acc = eacc[i];
      if (g == G) {
        acc.x += (double)tr_tot.x;
        acc.y += (double)tr_tot.y;
      } else {
        const double xr = tr_tot.x, xi = tr_tot.y;
        acc.x += 0.5 * ((xr * xr - xi * xi) - (double)sq_tot.x);
        acc.y += 0.5 * (2.0 * xr * xi - (double)sq_tot.y);
      }
      eacc[i] = acc;
    }
  }
  // E_L = sum_i w_i E_i, in determinant order per thread, then the block
  double sr = 0.0, si = 0.0;
  for (int i = tid; i < tb.ndet; i += nt) {
    const cplx<R> wi = sm.wt[i];
    const double2 e = eacc[i];
    sr += (double)wi.x * e.x - (double)wi.y * e.y;
    si += (double)wi.x * e.y + (double)wi.y * e.x;
  }
  sr = block_sum(sr, red);
  si = block_sum(si, red);
  if (tid == 0) eloc[w] = make_double2(sr, si);
}

}  // namespace

size_t md_step_smem(int M, int nu, int nd, int na_u, int na_d, int ndet, bool f64) {
  const size_t c = f64 ? 16 : 8;
  const size_t base = f64 ? MdSmem<double>::bytes(M, nu, nd, na_u, na_d, ndet)
                          : MdSmem<float>::bytes(M, nu, nd, na_u, na_d, ndet);
  return base + c * ((size_t)nu * na_u + (size_t)nd * na_d);
}

size_t md_energy_smem(int M, int nu, int nd, int na_u, int na_d, int ndet, bool f64) {
  const size_t c = f64 ? 16 : 8;   // P and V per spin
  return md_step_smem(M, nu, nd, na_u, na_d, ndet, f64) +
         c * ((size_t)nu * na_u + (size_t)nd * na_d);
}

template <typename T, typename R>
cudaError_t launch_md_step_r(cudaStream_t st, const MdTables& tb, int W, int M, int nu, int nd,
                             const T* Theta, long ldt, long dn_off, const double2* logdet0,
                             double2* logO_new, T* Gamma, long ldg, long gdn_off) {
  const bool f64 = sizeof(R) == 8;
  const size_t smem = md_step_smem(M, nu, nd, tb.nact[0], tb.nact[1], tb.ndet, f64);
  const size_t smem_h = smem + md_ctab_bytes(tb.ctot, tb.ndet, sizeof(cplx<R>));
  const size_t cap_h = smem_optin((const void*)md_step_kernel<T, R, true>);
  if (smem_h <= cap_h) {
    md_step_kernel<T, R, true><<<W, 256, smem_h, st>>>(tb, M, nu, nd, Theta, ldt, dn_off,
                                                       logdet0, logO_new, Gamma, ldg, gdn_off);
    return cudaGetLastError();
  }
  const size_t cap = smem_optin((const void*)md_step_kernel<T, R, false>);
  if (smem > cap) return cudaErrorInvalidValue;
  md_step_kernel<T, R, false><<<W, 256, smem, st>>>(tb, M, nu, nd, Theta, ldt, dn_off, logdet0,
                                                    logO_new, Gamma, ldg, gdn_off);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_md_step(cudaStream_t st, const MdTables& tb, int W, int M, int nu, int nd,
                           const T* Theta, long ldt, long dn_off, const double2* logdet0,
                           double2* logO_new, T* Gamma, long ldg, long gdn_off, bool f64) {
  return f64 ? launch_md_step_r<T, double>(st, tb, W, M, nu, nd, Theta, ldt, dn_off, logdet0,
                                           logO_new, Gamma, ldg, gdn_off)
             : launch_md_step_r<T, float>(st, tb, W, M, nu, nd, Theta, ldt, dn_off, logdet0,
                                          logO_new, Gamma, ldg, gdn_off);
}

template <typename T>
cudaError_t launch_md_energy(cudaStream_t st, const MdTables& tb, int W, int M, int nu, int nd,
                             int G, const T* Theta, long ldt, long dn_off,
                             const double2* logdet0, const T* LtilA, long ldg, long gdn_off,
                             double2* eloc, bool f64) {
  const size_t smem = md_energy_smem(M, nu, nd, tb.nact[0], tb.nact[1], tb.ndet, f64);
  const int threads = 256;
  // the hoisted kernel when its C_i table fits in shared memory
  const size_t smem_h = smem + md_ctab_bytes(tb.ctot, tb.ndet, f64 ? 16 : 8) +
                        sizeof(MdDet) * (size_t)tb.ndet;
  if (f64) {
    const size_t cap_h = smem_optin((const void*)md_energy_hoisted_kernel<T, double>);
    if (smem_h <= cap_h) {
      md_energy_hoisted_kernel<T, double><<<W, threads, smem_h, st>>>(
          tb, M, nu, nd, G, Theta, ldt, dn_off, logdet0, LtilA, ldg, gdn_off, eloc);
      return cudaGetLastError();
    }
  } else {
    const size_t cap_h = smem_optin((const void*)md_energy_hoisted_kernel<T, float>);
    if (smem_h <= cap_h) {
      md_energy_hoisted_kernel<T, float><<<W, threads, smem_h, st>>>(
          tb, M, nu, nd, G, Theta, ldt, dn_off, logdet0, LtilA, ldg, gdn_off, eloc);
      return cudaGetLastError();
    }
  }
  if ((tb.ndet + threads - 1) / threads > MD_MAX_DET_PER_THREAD) return cudaErrorInvalidValue;
  if (f64) {
    const size_t cap = smem_optin((const void*)md_energy_kernel<T, double>);
    if (smem > cap) return cudaErrorInvalidValue;
    md_energy_kernel<T, double><<<W, threads, smem, st>>>(tb, M, nu, nd, G, Theta, ldt, dn_off,
                                                          logdet0, LtilA, ldg, gdn_off, eloc);
  } else {
    const size_t cap = smem_optin((const void*)md_energy_kernel<T, float>);
    if (smem > cap) return cudaErrorInvalidValue;
    md_energy_kernel<T, float><<<W, threads, smem, st>>>(tb, M, nu, nd, G, Theta, ldt, dn_off,
                                                         logdet0, LtilA, ldg, gdn_off, eloc);
  }
  return cudaGetLastError();
}

#define MD_INST(T)                                                                           \
  template cudaError_t launch_md_step<T>(cudaStream_t, const MdTables&, int, int, int, int,  \
                                         const T*, long, long, const double2*, double2*, T*, \
                                         long, long, bool);                                  \
  template cudaError_t launch_md_energy<T>(cudaStream_t, const MdTables&, int, int, int,     \
                                           int, int, const T*, long, long, const double2*,   \
                                           const T*, long, long, double2*, bool);
MD_INST(float)
MD_INST(double)

}  // namespace afqmc
