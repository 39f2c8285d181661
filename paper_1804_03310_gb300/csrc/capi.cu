// C ABI of the ph-AFQMC walker-step library: context lifetime, setup
// precompute, the per-step schedule and read-out calls. See include/afqmc.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/afqmc.h"
#include "ctx_internal.h"
#include "kernels.h"
#include "multidet.h"
#include "tc.h"

using namespace afqmc;

namespace {

struct TimedPair {
  int id;
  cudaEvent_t a, b;
};

// A captured block of steps: replaying it advances the step counter by its
// length and the measurement counter by `meas`.
struct GraphEntry {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  long meas;
  int64_t launches;
};

struct StateHeader {
  char magic[8];     // "AFQMCST1"
  int32_t M, n_up, n_dn, n_walkers;
  int64_t step;
  uint64_t seed;
  int32_t run_id, n_chol;
};

}  // namespace

struct afqmc_ctx {
  afqmc_params p;
  int M, nu, nd, N, G, W, ndet;
  bool fp64;
  bool fp64_islands;   // Gauss-Jordan (and multi-determinant) arithmetic in FP64
  bool fp64_qr;        // Gram-Schmidt (QR) arithmetic in FP64
  cudaStream_t st;
  bool own_stream;
  long step;
  long n_meas;
  double e_shift;
  std::string err;
  bool poisoned;
  int64_t launches;

  // walker state and step intermediates (element type by precision); the
  // buffers never change roles, so a captured graph stays valid
  void *Phi, *Phi2, *Phi3, *Theta, *Theta2, *V, *X, *S, *xbar, *Z;
  // precomputed operators in the step precision
  void *L, *Ltil, *Bhalf, *PsiT, *Yx_up, *Yx_dn;
  // TF32X3: the constant GEMM operands hold their TF32 hi part, these the
  // remainders (split once at setup)
  void *Ltil_lo, *LT_lo, *Yx_up_lo, *Yx_dn_lo;
  double* PsiT64;
  double *weight, *scan, *wnew, *escalar, *lr;
  double* wref;        // reference weight of the weight cap (1 after a comb)
  double* log_scale;   // sum of ln(S/n) divided out of the weights at the combs
  double2 *logO, *logO2, *logO_new, *logdet, *logdet2, *lw, *eloc, *hist;
  // mean-field subtraction: lbar_g of the reference determinant [G], the
  // per-walker log of the scalar factor it puts on a propagated walker [W],
  // and -E_0 = 1/2 sum_g lbar_g^2
  double* lbar;
  double2* lmf;
  double e_mf;
  // block-diagonal Cholesky vectors: V is built and exponentiated on the
  // blocks' entries only (nnz of them, rows padded to nnzp); blk holds per
  // basis index the int4 {offset of its row of V, block size, start of the
  // block's member list, 0}, then the member lists (M ints)
  bool sparse;
  long nnz, nnzp;
  int nblk, maxblk;
  void* blk;
  std::vector<int> blk_gidx;   // host, during setup: i*M+j of each packed entry
  int *parent, *status;
  double wref_host;   // staging of a restored reference weight
  long long* ctr;   // device step counters: [0] completed steps, [1] measurements
  std::vector<void*> allocs;
  size_t dev_bytes;

  // padded strides (TMA needs 16-byte-aligned rows)
  long ldS;          // S row stride: n_chol rounded up to 4
  long ldx;          // X row stride: n_chol + 1
  long dn_off, ldt;  // Theta: down block offset and row stride
  long Jp[2];        // Yx / Z row strides per spin
  int xsplit;        // K splits of the force-bias contraction
  int xsplit_max;    // partial sums the X buffer holds
  void* LT;          // L transposed [M*ldV][ldS] (tensor-core operand; zero rows pad each
                     // operator row to ldV)
  void* dB;          // B_half - I (tensor-core operand)
  void* bimg;        // (B_half - I) operand image for the fused tensor-core Taylor kernel
  long ldV;          // row stride of V: M, or M rounded up to 4 where the wide
                     // tensor-core Taylor kernel streams V by TMA (M > 64)
  void *Vlo;         // TF32X3, wide kernel: remainders of V (V then holds the TF32 hi parts)
  void *dBp, *dBp_lo;  // B_half - I with rows of ldV (hi, lo) for the wide kernel

  // multi-determinant trial (Sherman-Morrison-Woodbury), unused for one determinant
  bool md;
  const double* ci_h;       // caller's CI coefficients (valid during create only)
  MdTables mdt;
  void *md_dets, *md_cc, *md_r0, *md_r1, *md_ct0, *md_ct1;
  int nact[2];
  long ldg, gdn_off;        // Gamma / LtilA row layout: up block at 0, down at gdn_off
  void *Gamma, *Gamma2, *LtilA;
  std::vector<int> act_h[2];       // host: active orbital indices per spin
  double* CactT64;                 // [nact_up + nact_dn][M] (read-outs)

  // tensor-core resources (TF32 modes)
  TcCtx* tc;
  bool tc_taylor_ok;  // M <= 64: on-chip tensor-core Taylor kernel
  bool tc_bhalf_ok;   // M % 4 == 0: B_half on the tensor cores
  bool tc_wide_ok;    // M > 64: the wide tensor-core Taylor kernel (operator streamed by TMA)
  bool split3;
  bool bf16;          // BF16X3: propagation (series and half steps) in BF16 hi + lo
  int taylor_fused;   // 0: CUDA-core series; 1: fused tensor-core kernel with the
                      // half steps; 2: tensor-core series, half steps as GEMMs;
                      // 3: wide tensor-core kernel with the half steps (M > 64)
  int bn_fb, bn_v, bn_e, bn_b;   // tensor-core tile widths per contraction

  // CUDA graphs of blocks of steps, keyed by (phase in the cadence period, length)
  bool use_graphs;
  long period;        // steps after which the cadence pattern repeats (0: too long)
  std::map<std::pair<long, long>, GraphEntry> graphs;

  bool timing;
  std::vector<TimedPair> pending;
  std::vector<cudaEvent_t> free_events;
  int64_t k_launch[AFQMC_N_KERNEL_IDS];
  double k_ms[AFQMC_N_KERNEL_IDS];
};

namespace {

const int kHist = 4096;
thread_local std::string g_create_err;
}  // namespace

namespace afqmc {
// Error text of calls that have no context (read by afqmc_last_error(NULL)).
void set_global_error(const std::string& msg) { g_create_err = msg; }

cudaError_t ctx_enqueue_readback(afqmc_ctx* c, double* e2, int* status) {
  cudaError_t e = cudaMemcpyAsync(e2, c->escalar, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                  c->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->st);
  return e;
}

long ctx_step(const afqmc_ctx* c) { return c->step; }
}  // namespace afqmc

namespace {

afqmc_status fail(afqmc_ctx* c, afqmc_status s, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (s == AFQMC_E_CUDA) c->poisoned = true;
  } else {
    g_create_err = msg;
  }
  return s;
}

#define CK(expr)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(c, e_ == cudaErrorMemoryAllocation ? AFQMC_E_OOM : AFQMC_E_CUDA,\
                  std::string(#expr) + ": " + cudaGetErrorString(e_));           \
  } while (0)

#define LK(expr)            \
  do {                      \
    CK(expr);               \
    c->launches += 1;       \
  } while (0)

size_t esize(const afqmc_ctx* c) { return c->fp64 ? sizeof(double) : sizeof(float); }

afqmc_status dalloc(afqmc_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(c, AFQMC_E_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  c->allocs.push_back(*p);
  c->dev_bytes += bytes;
  return AFQMC_OK;
}

#define DALLOC(ptr, bytes)                                      \
  do {                                                          \
    void* tmp_ = nullptr;                                       \
    afqmc_status s_ = dalloc(c, &tmp_, (bytes));                \
    if (s_ != AFQMC_OK) return s_;                              \
    ptr = reinterpret_cast<decltype(ptr)>(tmp_);                \
  } while (0)

cudaEvent_t get_event(afqmc_ctx* c) {
  if (!c->free_events.empty()) {
    cudaEvent_t e = c->free_events.back();
    c->free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

struct KTimer {
  afqmc_ctx* c;
  int id;
  cudaEvent_t a;
  KTimer(afqmc_ctx* c_, int id_) : c(c_), id(id_), a(nullptr) {
    if (c->timing) {
      a = get_event(c);
      cudaEventRecord(a, c->st);
    }
  }
  ~KTimer() {
    if (c->timing && a) {
      cudaEvent_t b = get_event(c);
      cudaEventRecord(b, c->st);
      c->pending.push_back({id, a, b});
      c->k_launch[id] += 1;
    }
  }
};

afqmc_status drain_timers(afqmc_ctx* c) {
  if (c->pending.empty()) return AFQMC_OK;
  CK(cudaStreamSynchronize(c->st));
  for (auto& t : c->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    c->k_ms[t.id] += ms;
    c->free_events.push_back(t.a);
    c->free_events.push_back(t.b);
  }
  c->pending.clear();
  return AFQMC_OK;
}

afqmc_status check_status(afqmc_ctx* c) {
  int s = 0;
  CK(cudaMemcpyAsync(&s, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (s & 4) {
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
    return fail(c, AFQMC_E_TIMEOUT, "a tensor-core pipeline wait timed out");
  }
  if (s & 2) {
    CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
    return fail(c, AFQMC_E_POPULATION, "population control found every walker weight zero");
  }
  return AFQMC_OK;
}

// ---------------------------------------------------------------------------
// Step pieces, templated on the walker element type.
// ---------------------------------------------------------------------------

template <typename T>
afqmc_status force_bias_contraction(afqmc_ctx* c) {
  const int W = c->W, G = c->G;
  KTimer t(c, 0);
  // single determinant: X = Theta . L~^T; multi-determinant: X = Gamma . L~act^T
  const bool md = c->md;
  const void* A = md ? c->Gamma : c->Theta;
  const void* B = md ? c->LtilA : c->Ltil;
  const long ld = md ? c->ldg : c->ldt;
  if (c->tc) {
    LK(tc_gemm(c->tc, c->st, 2 * W, G + 1, (int)ld, (const float*)A, ld, (const float*)B, ld,
               (float*)c->X, c->ldx, 1.0f, 0.0f, nullptr, 0, c->split3, c->xsplit,
               2L * W * c->ldx, c->status, c->bn_fb,
               md ? nullptr : (const float*)c->Ltil_lo));
  } else {
    LK(gemm<T>(c->st, false, true, 2 * W, G + 1, (int)ld, T(1), (const T*)A, ld, 0,
               (const T*)B, ld, 0, T(0), (T*)c->X, c->ldx, 0, 1));
  }
  return AFQMC_OK;
}

// Local energies of the current walkers into c->eloc. A single-determinant
// trial needs X from force_bias_contraction at these walkers.
template <typename T>
afqmc_status local_energy_T(afqmc_ctx* c) {
  const int W = c->W, M = c->M, G = c->G;
  KTimer t(c, 7);
  if (c->md) {
    LK(launch_md_energy<T>(c->st, c->mdt, W, M, c->nu, c->nd, G, (const T*)c->Theta, c->ldt,
                           c->dn_off, c->logdet, (const T*)c->LtilA, c->ldg, c->gdn_off,
                           c->eloc, c->fp64_islands));
    return AFQMC_OK;
  }
  {
    long zoff = 0;
    for (int sig = 0; sig < 2; ++sig) {
      const int ns = sig ? c->nd : c->nu;
      const long off = sig ? c->dn_off : 0;
      const long ldz = c->Jp[sig];
      if (ns == 0) continue;
      const long J = (long)ns * M;
      const T* Y = (const T*)(sig ? c->Yx_dn : c->Yx_up);
      if (c->tc) {
        LK(tc_gemm(c->tc, c->st, 2 * W, (int)J, (int)J, (const float*)c->Theta + off, c->ldt,
                   (const float*)Y, ldz, (float*)c->Z + zoff, ldz, 1.0f, 0.0f, nullptr, 0,
                   c->split3, 1, 0, c->status, c->bn_e,
                   (const float*)(sig ? c->Yx_dn_lo : c->Yx_up_lo)));
      } else {
        LK(gemm<T>(c->st, false, false, 2 * W, (int)J, (int)J, T(1),
                   (const T*)c->Theta + off, c->ldt, 0, Y, ldz, 0, T(0), (T*)c->Z + zoff,
                   ldz, 0, 1));
      }
      zoff += 2L * W * ldz;
    }
    LK(launch_energy_reduce<T>(c->st, W, M, c->nu, c->nd, G, (const T*)c->X, c->ldx,
                               c->xsplit, 2L * W * c->ldx, (const T*)c->Theta, c->ldt,
                               c->dn_off, (const T*)c->Z, c->Jp[0], c->Jp[1], c->eloc));
  }
  return AFQMC_OK;
}

template <typename T>
afqmc_status measure_T(afqmc_ctx* c, bool record) {
  afqmc_status s = AFQMC_OK;
  if (!c->md) {
    s = force_bias_contraction<T>(c);
    if (s != AFQMC_OK) return s;
  }
  s = local_energy_T<T>(c);
  if (s != AFQMC_OK) return s;
  LK(launch_mixed_energy(c->st, c->W, c->weight, c->eloc, c->ctr, record ? c->hist : nullptr,
                         kHist, c->escalar));
  if (record) c->n_meas += 1;
  return AFQMC_OK;
}

template <typename T>
afqmc_status mgs_T(afqmc_ctx* c) {
  KTimer t(c, 6);
  LK(launch_qr<T>(c->st, c->W, c->M, c->nu, c->nd, (T*)c->Phi, c->logO, c->lr,
                  c->fp64_qr));
  return AFQMC_OK;
}

template <typename T>
afqmc_status comb_T(afqmc_ctx* c) {
  const int W = c->W;
  KTimer t(c, 8);
  LK(launch_comb(c->st, W, c->weight, c->p.seed, c->p.run_id, c->ctr, 0, c->parent, c->scan,
                 c->wnew, c->status));
  // copies of the parents into the second buffers, then back, so that every
  // buffer keeps its role
  const long pe = (long)c->N * 2 * c->M;
  LK(launch_gather<T>(c->st, W, pe, 2 * c->ldt, c->parent, (const T*)c->Phi, (T*)c->Phi2,
                      (const T*)c->Theta, (T*)c->Theta2, c->logO, c->logO2, c->wnew,
                      c->weight, c->wref, c->log_scale));
  const size_t es = sizeof(T);
  CK(cudaMemcpyAsync(c->Phi, c->Phi2, (size_t)W * pe * es, cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->Theta, c->Theta2, (size_t)W * 2 * c->ldt * es,
                     cudaMemcpyDeviceToDevice, c->st));
  CK(cudaMemcpyAsync(c->logO, c->logO2, (size_t)W * sizeof(double2), cudaMemcpyDeviceToDevice,
                     c->st));
  if (c->md) {
    LK(launch_gather_rows<T>(c->st, W, 2 * c->ldg, c->parent, (const T*)c->Gamma,
                             (T*)c->Gamma2));
    LK(launch_gather_rows<double2>(c->st, W, 2, c->parent, c->logdet, c->logdet2));
    CK(cudaMemcpyAsync(c->Gamma, c->Gamma2, (size_t)W * 2 * c->ldg * es,
                       cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(c->logdet, c->logdet2, (size_t)W * 2 * sizeof(double2),
                       cudaMemcpyDeviceToDevice, c->st));
  }
  return AFQMC_OK;
}

template <typename T>
afqmc_status overlap_T(afqmc_ctx* c, double2* logO_out) {
  LK(launch_overlap<T>(c->st, c->W, c->M, c->nu, c->nd, (const T*)c->Phi,
                       (const T*)c->PsiT, (T*)c->Theta, c->ldt, c->dn_off, c->logdet,
                       nullptr, c->fp64_islands));
  if (c->md) {   // ratios by Sherman-Morrison-Woodbury, ln O_T and Gamma
    LK(launch_md_step<T>(c->st, c->mdt, c->W, c->M, c->nu, c->nd, (const T*)c->Theta, c->ldt,
                         c->dn_off, c->logdet, logO_out, (T*)c->Gamma, c->ldg, c->gdn_off,
                         c->fp64_islands));
  } else if (logO_out != c->logO_new) {   // the step's weight update sums the two spins itself
    LK(launch_logdet_sum(c->st, c->W, c->logdet, logO_out));
  }
  return AFQMC_OK;
}

// K5: out = B_half exp_T(V) B_half Phi. `out` is Phi itself during a step;
// the tuner points it at scratch to time the path without moving walkers.
template <typename T>
afqmc_status propagate_T(afqmc_ctx* c, T* out) {
  const int W = c->W, N = c->N, M = c->M;
  const int rows = W * N * 2;
  if (c->tc && c->taylor_fused == 3) {   // operator streamed by TMA, half steps fused
    LK(tc_taylor_wide(c->tc, c->st, W, M, N, c->p.taylor_order, c->ldV, c->V, c->Vlo, c->dBp,
                      c->dBp_lo, (const float*)c->Phi, (float*)out, c->split3, c->bf16,
                      c->status));
    return AFQMC_OK;
  }
  if (c->tc && c->taylor_fused == 1) {   // B_half exp(V) B_half in one tensor-core kernel, in place
    LK(tc_taylor(c->tc, c->st, W, M, N, c->p.taylor_order, (const float*)c->V,
                 (const float*)c->Phi, (float*)out, c->bimg, c->split3, c->bf16, c->status));
    return AFQMC_OK;
  }
  // Phi2 = B_half Phi
  if (c->tc && c->tc_bhalf_ok) {
    LK(tc_gemm(c->tc, c->st, rows, M, M, (const float*)c->Phi, M, (const float*)c->dB, M,
               (float*)c->Phi2, M, 1.0f, 1.0f, (const float*)c->Phi, M, c->split3, 1, 0,
               c->status, c->bn_b));
  } else if (c->dB) {   // Phi + Phi (B_half - I): the identity part exact in FP32
    CK(cudaMemcpyAsync(c->Phi2, c->Phi, (size_t)rows * M * sizeof(T), cudaMemcpyDeviceToDevice,
                       c->st));
    LK(gemm<T>(c->st, false, true, rows, M, M, T(1), (const T*)c->Phi, M, 0,
               (const T*)c->dB, M, 0, T(1), (T*)c->Phi2, M, 0, 1));
  } else {
    LK(gemm<T>(c->st, false, true, rows, M, M, T(1), (const T*)c->Phi, M, 0,
               (const T*)c->Bhalf, M, 0, T(0), (T*)c->Phi2, M, 0, 1));
  }
  // Phi3 = exp_T(V) Phi2
  if (c->sparse) {
    LK(launch_taylor_blocks<T>(c->st, W, M, N, c->p.taylor_order, c->nnzp, c->nblk,
                               c->maxblk, (const T*)c->V, c->blk, (const T*)c->Phi2,
                               (T*)c->Phi3));
  } else if (c->tc && c->taylor_fused == 2) {
    LK(tc_taylor(c->tc, c->st, W, M, N, c->p.taylor_order, (const float*)c->V,
                 (const float*)c->Phi2, (float*)c->Phi3, nullptr, c->split3, c->bf16,
                 c->status));
  } else {
    LK(launch_taylor<T>(c->st, W, M, N, c->p.taylor_order, (const T*)c->V, c->ldV,
                        (const T*)c->Phi2, (T*)c->Phi3));
  }
  // out = B_half Phi3
  if (c->tc && c->tc_bhalf_ok) {
    LK(tc_gemm(c->tc, c->st, rows, M, M, (const float*)c->Phi3, M, (const float*)c->dB, M,
               (float*)out, M, 1.0f, 1.0f, (const float*)c->Phi3, M, c->split3, 1, 0,
               c->status, c->bn_b));
  } else if (c->dB) {
    CK(cudaMemcpyAsync(out, c->Phi3, (size_t)rows * M * sizeof(T), cudaMemcpyDeviceToDevice,
                       c->st));
    LK(gemm<T>(c->st, false, true, rows, M, M, T(1), (const T*)c->Phi3, M, 0,
               (const T*)c->dB, M, 0, T(1), out, M, 0, 1));
  } else {
    LK(gemm<T>(c->st, false, true, rows, M, M, T(1), (const T*)c->Phi3, M, 0,
               (const T*)c->Bhalf, M, 0, T(0), out, M, 0, 1));
  }
  return AFQMC_OK;
}

template <typename T>
afqmc_status step_T(afqmc_ctx* c) {
  const int W = c->W, M = c->M, G = c->G;
  const double dt = c->p.dtau;
  afqmc_status s = force_bias_contraction<T>(c);
  if (s != AFQMC_OK) return s;
  const bool local = c->p.weight_mode == AFQMC_WEIGHT_LOCAL_ENERGY;
  if (local) {   // the local-energy weight form needs E_L before the move
    s = local_energy_T<T>(c);
    if (s != AFQMC_OK) return s;
  }
  {
    KTimer t(c, 1);
    LK(launch_fields<T>(c->st, W, G, (const T*)c->X, c->ldx, c->xsplit, 2L * W * c->ldx,
                        sqrt(dt), c->p.fb_cap, c->p.seed, c->p.run_id, c->ctr, (T*)c->S,
                        c->ldS, (T*)c->xbar, c->lw, c->lbar, c->lmf));
  }
  if (c->sparse) {   // V on the blocks' entries only, [W][2][nnzp]
    KTimer t(c, 2);
    if (c->tc) {
      LK(tc_gemm(c->tc, c->st, 2 * W, (int)c->nnzp, G, (const float*)c->S, c->ldS,
                 (const float*)c->LT, c->ldS, (float*)c->V, c->nnzp, 1.0f, 0.0f, nullptr, 0,
                 c->split3, 1, 0, c->status, c->bn_v, (const float*)c->LT_lo));
    } else {
      LK(gemm<T>(c->st, false, false, 2 * W, (int)c->nnz, G, T(1), (const T*)c->S, c->ldS, 0,
                 (const T*)c->L, c->nnz, 0, T(0), (T*)c->V, c->nnzp, 0, 1));
    }
  } else {
    KTimer t(c, 2);
    if (c->tc) {
      const long nv = (long)M * c->ldV;
      LK(tc_gemm(c->tc, c->st, 2 * W, (int)nv, G, (const float*)c->S, c->ldS,
                 (const float*)c->LT, c->ldS, (float*)c->V, nv, 1.0f, 0.0f, nullptr, 0,
                 c->split3, 1, 0, c->status, c->bn_v, (const float*)c->LT_lo,
                 c->taylor_fused == 3 && c->split3 ? (float*)c->Vlo : nullptr,
                 c->taylor_fused == 3 && c->bf16));
    } else {
      LK(gemm<T>(c->st, false, false, 2 * W, M * M, G, T(1), (const T*)c->S, c->ldS, 0,
                 (const T*)c->L, (long)M * M, 0, T(0), (T*)c->V, (long)M * M, 0, 1));
    }
  }
  {
    KTimer t(c, 3);
    s = propagate_T<T>(c, (T*)c->Phi);
    if (s != AFQMC_OK) return s;
  }
  {
    KTimer t(c, 4);
    s = overlap_T<T>(c, c->logO_new);
    if (s != AFQMC_OK) return s;
  }
  {
    KTimer t(c, 5);
    LK(launch_weights(c->st, W, c->md ? c->logO_new : nullptr, c->md ? nullptr : c->logdet,
                      c->lw, c->lmf, local ? c->eloc : nullptr, dt,
                      local ? c->e_shift : c->e_shift + c->e_mf, (double)c->p.weight_cap,
                      c->wref, c->weight, c->logO, c->ctr));
  }
  c->step += 1;
  const long n = c->step;
  if (c->p.ortho_every > 0 && n % c->p.ortho_every == 0) {
    s = mgs_T<T>(c);
    if (s != AFQMC_OK) return s;
  }
  if (c->p.measure_every > 0 && n % c->p.measure_every == 0) {
    s = measure_T<T>(c, true);
    if (s != AFQMC_OK) return s;
  }
  if (c->p.pc_every > 0 && n % c->p.pc_every == 0) {
    s = comb_T<T>(c);
    if (s != AFQMC_OK) return s;
  }
  return AFQMC_OK;
}

// ---------------------------------------------------------------------------
// Setup
// ---------------------------------------------------------------------------

// Block structure shared by all Cholesky vectors: the connected components
// of the graph with an edge i - j wherever some L_g,ij is nonzero. Each
// block lists its members in ascending order; blocks are ordered by their
// first member. V = sum_g s_g L_g is block-diagonal in this partition, and
// its packed form holds block b's b x b entries row by row at offset o_b.
struct BlockPlan {
  bool on = false;
  int nb = 0, maxb = 0;
  long nnz = 0;
  std::vector<int> members;             // [M]: block after block
  std::vector<int> vrow, bsize, ibase;  // per basis index
  std::vector<int> gidx;                // [nnz]: i * M + j of each packed entry
};

BlockPlan detect_blocks(const afqmc_params* p, const double* L) {
  BlockPlan B;
  const int M = p->M;
  if (p->block_sparse == 2 || M < 2) return B;
  std::vector<int> up(M);
  for (int i = 0; i < M; ++i) up[i] = i;
  auto root = [&](int i) {
    while (up[i] != i) { up[i] = up[up[i]]; i = up[i]; }
    return i;
  };
  for (long g = 0; g < p->n_chol; ++g) {
    const double* Lg = L + g * M * M;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < i; ++j)
        if (Lg[(long)i * M + j] != 0.0) {
          const int a = root(i), b = root(j);
          if (a != b) up[a < b ? b : a] = a < b ? a : b;
        }
  }
  std::vector<std::vector<int>> blocks;
  std::vector<int> slot(M, -1);
  for (int i = 0; i < M; ++i) {        // ascending i: blocks by first member
    const int r = root(i);
    if (slot[r] < 0) { slot[r] = (int)blocks.size(); blocks.emplace_back(); }
    blocks[slot[r]].push_back(i);
  }
  B.nb = (int)blocks.size();
  for (const auto& b : blocks) {
    B.maxb = std::max(B.maxb, (int)b.size());
    B.nnz += (long)b.size() * (long)b.size();
  }
  if (B.nb < 2 || B.maxb > 32 || B.nnz > (long)M * M / 4) return B;
  B.on = true;
  B.vrow.assign(M, 0);
  B.bsize.assign(M, 0);
  B.ibase.assign(M, 0);
  long off = 0;
  for (const auto& b : blocks) {
    const int n = (int)b.size(), base = (int)B.members.size();
    for (int lp = 0; lp < n; ++lp) {
      const int i = b[lp];
      B.vrow[i] = (int)(off + (long)lp * n);
      B.bsize[i] = n;
      B.ibase[i] = base;
      for (int lq = 0; lq < n; ++lq) B.gidx.push_back(i * M + b[lq]);
    }
    B.members.insert(B.members.end(), b.begin(), b.end());
    off += (long)n * n;
  }
  return B;
}

// Size and option checks that need no matrix data.
afqmc_status validate_sizes(const afqmc_params* p) {
  afqmc_ctx* c = nullptr;
  if (!p) return fail(c, AFQMC_E_INVALID, "null argument");
  if (p->weight_mode != AFQMC_WEIGHT_HYBRID && p->weight_mode != AFQMC_WEIGHT_LOCAL_ENERGY)
    return fail(c, AFQMC_E_INVALID, "weight_mode must be 0 (hybrid) or 1 (local energy)");
  if (p->mf_subtract != 0 && p->mf_subtract != 1)
    return fail(c, AFQMC_E_INVALID, "mf_subtract must be 0 or 1");
  if (p->block_sparse < 0 || p->block_sparse > 2)
    return fail(c, AFQMC_E_INVALID, "block_sparse must be 0 (auto), 1 (required) or 2 (dense)");
  for (int i = 0; i < 3; ++i)
    if (p->reserved[i] != 0) return fail(c, AFQMC_E_INVALID, "reserved fields must be zero");
  if (p->weight_mode == AFQMC_WEIGHT_LOCAL_ENERGY && p->n_det > 1)
    return fail(c, AFQMC_E_INVALID,
                "the local-energy weight form needs a one-determinant trial");
  if (p->cs_group < 0) return fail(c, AFQMC_E_INVALID, "cs_group must be >= 0");
  if (p->cs_group == 0 ? p->cs_size != 0 : (p->cs_size < 2 || p->cs_size > 16))
    return fail(c, AFQMC_E_INVALID, "cs_size must be 2..16 in a correlated-sampling group, else 0");
  if (p->weight_cap < 0) return fail(c, AFQMC_E_INVALID, "weight_cap must be >= 0");
  if ((p->graphs != 0 && p->graphs != 1) || (p->autotune != 0 && p->autotune != 1))
    return fail(c, AFQMC_E_INVALID, "graphs and autotune must be 0 or 1");
  const int M = p->M;
  if (M < 1 || M > 256) return fail(c, AFQMC_E_INVALID, "M must be in 1..256");
  if (p->n_up < 0 || p->n_dn < 0 || p->n_up > M || p->n_dn > M || p->n_up + p->n_dn < 1)
    return fail(c, AFQMC_E_INVALID, "electron counts out of range");
  if (p->n_chol < 1) return fail(c, AFQMC_E_INVALID, "n_chol must be >= 1");
  if (p->n_det < 1 || p->n_det > 256 * MD_MAX_DET_PER_THREAD)
    return fail(c, AFQMC_E_INVALID, "n_det must be in 1..2048");
  if (p->n_walkers < 1 || p->n_walkers > 32768)
    return fail(c, AFQMC_E_INVALID, "n_walkers must be in 1..32768");
  if (!(p->dtau > 0.0)) return fail(c, AFQMC_E_INVALID, "dtau must be > 0");
  if (p->taylor_order < 1 || p->taylor_order > 12)
    return fail(c, AFQMC_E_INVALID, "taylor_order must be in 1..12");
  if (p->precision < AFQMC_FP64 || p->precision > AFQMC_BF16X3)
    return fail(c, AFQMC_E_INVALID, "unknown precision");
  if (p->run_id < 0 || p->run_id >= (1 << 29)) return fail(c, AFQMC_E_INVALID, "run_id out of range");
  if (p->ortho_every < 0 || p->measure_every < 0 || p->pc_every < 0)
    return fail(c, AFQMC_E_INVALID, "cadences must be >= 0");
  if (p->fp64_islands < 0 || p->fp64_islands > 2)
    return fail(c, AFQMC_E_INVALID, "fp64_islands must be 0, 1 or 2");
  const int nmax = p->n_up > p->n_dn ? p->n_up : p->n_dn;
  const bool f64 = p->precision == AFQMC_FP64 || p->fp64_islands;
  if (afqmc::overlap_smem(M, nmax, f64 ? 16 : 8) > 227 * 1024)
    return fail(c, AFQMC_E_INVALID,
                "M x electrons per spin too large for the on-chip overlap and QR in this "
                "precision");
  return AFQMC_OK;
}

afqmc_status validate(const afqmc_params* p, const double* h1, const double* L,
                      const double* Cu, const double* Cd, const int32_t* ou,
                      const int32_t* od, const double* ci) {
  afqmc_ctx* c = nullptr;
  if (!p || !h1 || !L || !Cu || !Cd || !ou || !od || !ci)
    return fail(c, AFQMC_E_INVALID, "null argument");
  afqmc_status s0 = validate_sizes(p);
  if (s0 != AFQMC_OK) return s0;
  const int M = p->M;
  // symmetry of h1 and L
  double scale = 0.0;
  for (long e = 0; e < (long)M * M; ++e) scale = fmax(scale, fabs(h1[e]));
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < i; ++j)
      if (fabs(h1[i * M + j] - h1[j * M + i]) > 1e-12 * (1.0 + scale))
        return fail(c, AFQMC_E_INVALID, "h1 is not symmetric");
  for (long g = 0; g < p->n_chol; ++g) {
    const double* Lg = L + g * M * M;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < i; ++j)
        if (fabs(Lg[i * M + j] - Lg[j * M + i]) > 1e-12 * (1.0 + fabs(Lg[i * M + j])))
          return fail(c, AFQMC_E_INVALID, "L_g is not symmetric (g = " + std::to_string(g) + ")");
  }
  // occupations and orthonormality of the used orbitals
  for (int sig = 0; sig < 2; ++sig) {
    const int ns = sig ? p->n_dn : p->n_up;
    const int32_t* occ = sig ? od : ou;
    const double* C = sig ? Cd : Cu;
    std::vector<char> used(M, 0);
    for (long d = 0; d < p->n_det; ++d) {
      std::vector<char> seen(M, 0);
      for (int a = 0; a < ns; ++a) {
        int o = occ[d * ns + a];
        if (o < 0 || o >= M) return fail(c, AFQMC_E_INVALID, "occupation index out of range");
        if (seen[o]) return fail(c, AFQMC_E_INVALID, "repeated orbital in a determinant");
        seen[o] = 1;
        used[o] = 1;
      }
    }
    for (int a = 0; a < M; ++a) {
      if (!used[a]) continue;
      for (int b = 0; b <= a; ++b) {
        if (!used[b]) continue;
        double s = 0.0;
        for (int k = 0; k < M; ++k) s += C[k * M + a] * C[k * M + b];
        if (fabs(s - (a == b ? 1.0 : 0.0)) > 1e-8)
          return fail(c, AFQMC_E_INVALID, "trial orbitals are not orthonormal");
      }
    }
  }
  if (p->block_sparse == 1 && !detect_blocks(p, L).on)
    return fail(c, AFQMC_E_INVALID,
                "block_sparse = 1, but the Cholesky vectors are not block-diagonal in blocks "
                "of at most 32 orbitals holding at most M^2/4 entries");
  (void)ci;
  return AFQMC_OK;
}

template <typename T>
afqmc_status setup_T(afqmc_ctx* c, const double* h1_h, const double* L_h,
                     const double* Cu, const double* Cd, const int32_t* ou,
                     const int32_t* od) {
  const int M = c->M, N = c->N, G = c->G, W = c->W;
  const long MM = (long)M * M;
  cudaStream_t st = c->st;
  // FP64 staging
  double *h1, *L, *PsiT, *h1p, *Bh, *Ltil, *ta, *tb, *tcur, *tnext;
  std::vector<void*> tmp;
  auto tmalloc = [&](double** p, size_t n) -> afqmc_status {
    cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      for (void* q : tmp) cudaFree(q);
      return fail(c, AFQMC_E_OOM, "setup allocation failed");
    }
    tmp.push_back(*p);
    return AFQMC_OK;
  };
#define TM(p, n) do { afqmc_status s_ = tmalloc(&p, (n)); if (s_ != AFQMC_OK) return s_; } while (0)
  double *Ltil_pad;
  TM(h1, MM); TM(L, (size_t)G * MM); TM(PsiT, (size_t)N * M); TM(h1p, MM); TM(Bh, MM);
  TM(Ltil, (size_t)(G + 1) * N * M); TM(ta, MM); TM(tb, MM); TM(tcur, MM); TM(tnext, MM);
  TM(Ltil_pad, (size_t)(G + 1) * c->ldt);
  std::vector<double> psiT_h((size_t)N * M);
  for (int a = 0; a < N; ++a) {
    const bool up = a < c->nu;
    const double* C = up ? Cu : Cd;
    const int orb = up ? ou[a] : od[a - c->nu];
    for (int k = 0; k < M; ++k) psiT_h[(size_t)a * M + k] = C[(size_t)k * M + orb];
  }
  CK(cudaMemcpyAsync(h1, h1_h, MM * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(L, L_h, (size_t)G * MM * sizeof(double), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(PsiT, psiT_h.data(), psiT_h.size() * sizeof(double),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(c->PsiT64, psiT_h.data(), psiT_h.size() * sizeof(double),
                     cudaMemcpyHostToDevice, st));
  // half-rotated L~_g = D^T L_g (rows: up orbitals, then down), plus D^T h1
  LK(gemm<double>(st, false, false, N, M, M, 1.0, PsiT, M, 0, L, M, MM, 0.0, Ltil, M,
                  (long)N * M, G));
  LK(gemm<double>(st, false, false, N, M, M, 1.0, PsiT, M, 0, h1, M, 0, 0.0,
                  Ltil + (size_t)G * N * M, M, 0, 1));
  // X_g = tr(L~_g D) and tr(h~ D) of the reference determinant (phi = D, so
  // Theta = D and theta = vec(D^T)), FP64: the trial energy's Coulomb and
  // one-body terms and, with mean-field subtraction, lbar_g
  double *et_x, *et_z;
  TM(et_x, G + 1);
  TM(et_z, (size_t)std::max(c->nu, c->nd) * M + 1);
  std::vector<double> et_xh(G + 1);
  LK(launch_gemv_rows(st, G + 1, (long)N * M, Ltil, (long)N * M, PsiT, et_x));
  CK(cudaMemcpyAsync(et_xh.data(), et_x, (G + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (c->lbar)
    CK(cudaMemcpyAsync(c->lbar, et_x, G * sizeof(double), cudaMemcpyDeviceToDevice, st));
  // H1' = h1 - 1/2 sum_g L_g L_g (+ sum_g lbar_g L_g)
  LK(launch_h1_remainder(st, M, G, h1, L, c->lbar, h1p));
  // B_half = exp(-dt/2 H1'): scaling and squaring of a Taylor series
  std::vector<double> hp(MM);
  CK(cudaMemcpyAsync(hp.data(), h1p, MM * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  c->e_mf = 0.0;
  if (c->lbar)
    for (int g = 0; g < G; ++g) c->e_mf += 0.5 * et_xh[g] * et_xh[g];
  double fro = 0.0;
  for (double v : hp) fro += v * v;
  fro = sqrt(fro) * 0.5 * c->p.dtau;
  int sq = 0;
  while (fro / ldexp(1.0, sq) > 0.25 && sq < 60) ++sq;
  const double a = -0.5 * c->p.dtau / ldexp(1.0, sq);
  LK(launch_scale_identity(st, M, h1p, a, Bh, tcur));   // Bh = I + A, tcur = A
  CK(cudaMemcpyAsync(ta, tcur, MM * sizeof(double), cudaMemcpyDeviceToDevice, st));
  for (int k = 2; k <= 24; ++k) {
    LK(gemm<double>(st, false, false, M, M, M, 1.0 / k, tcur, M, 0, ta, M, 0, 0.0, tnext,
                    M, 0, 1));
    LK(launch_axpy_d(st, MM, 1.0, tnext, Bh));
    std::swap(tcur, tnext);
  }
  for (int i = 0; i < sq; ++i) {
    LK(gemm<double>(st, false, false, M, M, M, 1.0, Bh, M, 0, Bh, M, 0, 0.0, tb, M, 0, 1));
    std::swap(Bh, tb);
  }
  // E_T = E_L of the reference determinant in FP64 whatever the step
  // precision: the terms gathered above plus the exchange term
  // 1/2 theta^T Yx theta per spin
  double e_exch = 0.0;
  // exchange part of the Eq. 5 tensor, per spin
  for (int sig = 0; sig < 2; ++sig) {
    const int ns = sig ? c->nd : c->nu;
    const int j0 = sig ? c->nu : 0;
    if (ns == 0) continue;
    const long J = (long)ns * M;
    double *gram, *yx;
    TM(gram, (size_t)J * J);
    TM(yx, (size_t)J * J);
    LK(gemm<double>(st, true, false, (int)J, (int)J, G, 1.0, Ltil + (size_t)j0 * M,
                    (long)N * M, 0, Ltil + (size_t)j0 * M, (long)N * M, 0, 0.0, gram, J, 0, 1));
    CK(cudaMemsetAsync(yx, 0, (size_t)J * J * sizeof(double), st));
    LK(launch_yx_permute(st, ns, M, gram, yx, c->Jp[sig]));
    {   // 1/2 theta^T Yx theta of the reference determinant, FP64
      std::vector<double> zh((size_t)J);
      LK(launch_gemv_cols(st, J, J, yx, c->Jp[sig], PsiT + (size_t)j0 * M, et_z));
      CK(cudaMemcpyAsync(zh.data(), et_z, J * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      double q = 0.0;
      for (long e = 0; e < J; ++e) q += psiT_h[(size_t)j0 * M + e] * zh[e];
      e_exch += 0.5 * q;
    }
    void* dst = sig ? c->Yx_dn : c->Yx_up;
    LK(launch_convert<T>(st, J * c->Jp[sig], yx, (T*)dst));
  }
  if (c->sparse) {   // packed operands of the block-diagonal form
    double *lp, *lpt = nullptr;
    int* gidx;
    TM(lp, (size_t)G * c->nnz);
    if (c->LT) TM(lpt, (size_t)c->nnzp * c->ldS);
    {
      cudaError_t e = cudaMalloc((void**)&gidx, c->nnz * sizeof(int));
      if (e != cudaSuccess) {
        cudaGetLastError();
        for (void* q : tmp) cudaFree(q);
        return fail(c, AFQMC_E_OOM, "setup allocation failed");
      }
      tmp.push_back(gidx);
    }
    CK(cudaMemcpyAsync(gidx, c->blk_gidx.data(), c->nnz * sizeof(int), cudaMemcpyHostToDevice,
                       st));
    LK(launch_pack_blocks(st, G, c->nnz, c->nnzp, c->ldS, M, L, gidx, lp, lpt));
    LK(launch_convert<T>(st, (long)G * c->nnz, lp, (T*)c->L));
    if (c->LT) LK(launch_convert<T>(st, c->nnzp * c->ldS, lpt, (T*)c->LT));
    CK(cudaStreamSynchronize(st));   // the host index list is released below
  } else {
    LK(launch_convert<T>(st, (long)G * MM, L, (T*)c->L));
  }
  CK(cudaMemsetAsync(Ltil_pad, 0, (size_t)(G + 1) * c->ldt * sizeof(double), st));
  LK(launch_pad_rows(st, G + 1, (long)c->nu * M, (long)c->nd * M, Ltil, Ltil_pad, c->ldt,
                     c->dn_off));
  LK(launch_convert<T>(st, (long)(G + 1) * c->ldt, Ltil_pad, (T*)c->Ltil));
  if (c->LT && !c->sparse) {   // L transposed [M*ldV][ldS] for the tensor cores
    double *lt;
    const long nv = (long)M * c->ldV;
    TM(lt, nv * c->ldS);
    CK(cudaMemsetAsync(lt, 0, nv * c->ldS * sizeof(double), st));
    LK(launch_transpose_pad(st, G, M, c->ldV, L, lt, c->ldS));
    LK(launch_convert<T>(st, nv * c->ldS, lt, (T*)c->LT));
  }
  if (c->dB) {   // B_half - I: the reduced modes add the identity part exactly
    CK(cudaMemcpyAsync(tb, Bh, MM * sizeof(double), cudaMemcpyDeviceToDevice, st));
    LK(launch_add_diag(st, M, tb, -1.0));
    LK(launch_convert<T>(st, MM, tb, (T*)c->dB));
    if (c->bimg)
      LK(tc_bhalf_image(st, M, (const float*)c->dB, c->bimg, c->split3, c->bf16));
    if (c->dBp) {   // rows padded to ldV (TMA), then split for TF32X3 / BF16X3
      double* pad;
      TM(pad, (size_t)M * c->ldV);
      CK(cudaMemsetAsync(pad, 0, (size_t)M * c->ldV * sizeof(double), st));
      LK(launch_pad_rows(st, M, M, 0, tb, pad, c->ldV, c->ldV));
      if (c->bf16) {
        LK(tc_split_bf16(st, (long)M * c->ldV, pad, c->dBp, c->dBp_lo));
      } else {
        LK(launch_convert<T>(st, (long)M * c->ldV, pad, (T*)c->dBp));
        if (c->dBp_lo)
          LK(tc_split(st, (long)M * c->ldV, (float*)c->dBp, (float*)c->dBp_lo));
      }
    }
  }
  if (c->split3) {   // the constant operands of the TF32X3 contractions, split once
    LK(tc_split(st, (long)(G + 1) * c->ldt, (float*)c->Ltil, (float*)c->Ltil_lo));
    LK(tc_split(st, c->sparse ? c->nnzp * c->ldS : (long)M * c->ldV * c->ldS, (float*)c->LT,
                (float*)c->LT_lo));
    LK(tc_split(st, (long)c->nu * M * c->Jp[0], (float*)c->Yx_up, (float*)c->Yx_up_lo));
    LK(tc_split(st, (long)c->nd * M * c->Jp[1], (float*)c->Yx_dn, (float*)c->Yx_dn_lo));
  }
  LK(launch_convert<T>(st, MM, Bh, (T*)c->Bhalf));
  LK(launch_convert<T>(st, (long)N * M, PsiT, (T*)c->PsiT));
  if (c->md) {   // C_act^T L_g and C_act^T h1 per spin, [G+1][ldg]
    double* la;
    TM(la, (size_t)(G + 1) * c->ldg);
    CK(cudaMemsetAsync(la, 0, (size_t)(G + 1) * c->ldg * sizeof(double), st));
    for (int sg = 0; sg < 2; ++sg) {
      const int na = c->nact[sg];
      if (na == 0) continue;
      const double* ct = c->CactT64 + (sg ? (size_t)c->nact[0] * M : 0);
      double* dst = la + (sg ? c->gdn_off : 0);
      LK(gemm<double>(st, false, false, na, M, M, 1.0, ct, M, 0, L, M, MM, 0.0, dst, M,
                      c->ldg, G));
      LK(gemm<double>(st, false, false, na, M, M, 1.0, ct, M, 0, h1, M, 0, 0.0,
                      dst + (size_t)G * c->ldg, M, 0, 1));
      LK(launch_convert<T>(st, (long)na * M, ct, (T*)c->mdt.CactT[sg]));
    }
    LK(launch_convert<T>(st, (long)(G + 1) * c->ldg, la, (T*)c->LtilA));
  }
  CK(cudaStreamSynchronize(st));
  for (void* q : tmp) cudaFree(q);
#undef TM
  // walkers start at the reference determinant, weight 1
  LK(launch_init_walkers<T>(st, W, M, N, (const T*)c->PsiT, (T*)c->Phi, c->weight));
  {                                   // reference weight of the weight cap, log scale
    static const double one = 1.0;
    CK(cudaMemcpyAsync(c->wref, &one, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(c->log_scale, 0, sizeof(double), st));
  }
  afqmc_status s = overlap_T<T>(c, c->logO);
  if (s != AFQMC_OK) return s;
  if (isnan(c->p.e_shift)) {
    // E_T: energy of the reference determinant, <D_0|H|D_0>, from the FP64
    // terms gathered above
    double coul = 0.0;
    for (int g = 0; g < G; ++g) coul += et_xh[g] * et_xh[g];
    const double e0 = et_xh[G] + 0.5 * coul + e_exch;
    if (!isfinite(e0)) return fail(c, AFQMC_E_NUMERIC, "trial energy is not finite");
    c->e_shift = e0;
  } else {
    c->e_shift = c->p.e_shift;
  }
  return AFQMC_OK;
}

long round4(long x) { return (x + 3) / 4 * 4; }

// Parity (+1 / -1) of the permutation taking list `from` to list `to`
// (same elements).
int perm_sign(const std::vector<int>& from, const std::vector<int>& to) {
  const int n = (int)from.size();
  std::vector<int> pos(n), seen(n, 0);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      if (from[i] == to[j]) { pos[j] = i; break; }
  int sign = 1;
  for (int j = 0; j < n; ++j) {
    if (seen[j]) continue;
    int len = 0, k = j;
    while (!seen[k]) { seen[k] = 1; k = pos[k]; ++len; }
    if (len % 2 == 0) sign = -sign;
  }
  return sign;
}

// Multi-determinant trial: each determinant as in-place excitations of the
// reference (holes at reference positions, filled by particles in ascending
// order), the column-order sign folded into its coefficient; active orbitals
// per spin are the reference orbitals (in position order) then the others
// occupied anywhere (ascending).
afqmc_status prepare_multidet(afqmc_ctx* c, const int32_t* ou, const int32_t* od,
                              const double* ci, std::vector<MdDet>& dets,
                              std::vector<double2>& cconj) {
  const int nd_ = c->ndet;
  dets.assign(nd_, MdDet());
  cconj.assign(nd_, make_double2(0, 0));
  std::vector<int> sign(nd_, 1);
  for (int sg = 0; sg < 2; ++sg) {
    const int ns = sg ? c->nd : c->nu;
    const int32_t* occ = sg ? od : ou;
    std::vector<int> ref(occ, occ + ns);
    std::vector<int> refpos(c->M, -1);
    for (int a = 0; a < ns; ++a) refpos[ref[a]] = a;
    std::vector<char> used(c->M, 0);
    for (int i = 0; i < nd_; ++i)
      for (int a = 0; a < ns; ++a) used[occ[(size_t)i * ns + a]] = 1;
    std::vector<int>& act = c->act_h[sg];
    act = ref;
    for (int o = 0; o < c->M; ++o)
      if (used[o] && refpos[o] < 0) act.push_back(o);
    std::vector<int> actidx(c->M, -1);
    for (size_t q = 0; q < act.size(); ++q) actidx[act[q]] = (int)q;
    c->nact[sg] = (int)act.size();
    for (int i = 0; i < nd_; ++i) {
      std::vector<int> oi(occ + (size_t)i * ns, occ + (size_t)(i + 1) * ns);
      std::vector<char> in_i(c->M, 0);
      for (int o : oi) in_i[o] = 1;
      std::vector<int> holes, parts;
      for (int a = 0; a < ns; ++a)
        if (!in_i[ref[a]]) holes.push_back(a);
      std::vector<int> sorted_oi = oi;
      std::sort(sorted_oi.begin(), sorted_oi.end());
      for (int o : sorted_oi)
        if (refpos[o] < 0) parts.push_back(o);
      if ((int)holes.size() > MD_EMAX)
        return fail(c, AFQMC_E_INVALID,
                    "a determinant has more than " + std::to_string(MD_EMAX) +
                        " excitations in one spin");
      std::vector<int> t = ref;
      for (size_t l = 0; l < holes.size(); ++l) t[holes[l]] = parts[l];
      sign[i] *= perm_sign(oi, t);
      MdDet& d = dets[i];
      d.E[sg] = (int)holes.size();
      for (int l = 0; l < MD_EMAX; ++l) {
        d.h[sg][l] = l < (int)holes.size() ? holes[l] : 0;
        d.p[sg][l] = l < (int)holes.size() ? actidx[parts[l]] : 0;
      }
    }
  }
  if (dets[0].E[0] != 0 || dets[0].E[1] != 0)
    return fail(c, AFQMC_E_INVALID, "determinant 0 must be the reference");
  for (int i = 0; i < nd_; ++i)
    cconj[i] = make_double2(sign[i] * ci[2 * i], -sign[i] * ci[2 * i + 1]);
  return AFQMC_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: launch shapes of the tensor-core contractions, timed on the
// context's own operands right after setup (the timed launches write only
// scratch: X, V, Z and the spare walker buffers), the fastest kept and cached
// per shape for the rest of the process.
// ---------------------------------------------------------------------------

struct TuneVal {
  int xsplit, bn_fb, bn_v, bn_e, bn_b, fused;
};
using TuneKey = std::tuple<int, int, int, int, int, int, int, int, int, long>;
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;

TuneKey tune_key(const afqmc_ctx* c) {
  return TuneKey(c->M, c->nu, c->nd, c->G, c->W, c->md ? c->nact[0] : -1,
                 c->md ? c->nact[1] : -1, c->p.precision, c->p.taylor_order,
                 c->sparse ? c->nnz : -1L);
}

// Shortest of three timed runs (after one untimed run) of `f`, in ms;
// infinity when a launch fails.
template <typename F>
float best_ms(afqmc_ctx* c, F f) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return INFINITY;
  if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return INFINITY; }
  float best = INFINITY;
  if (f() == AFQMC_OK) {
    for (int r = 0; r < 3; ++r) {
      cudaEventRecord(a, c->st);
      if (f() != AFQMC_OK) { best = INFINITY; break; }
      cudaEventRecord(b, c->st);
      if (cudaEventSynchronize(b) != cudaSuccess) { best = INFINITY; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      best = std::min(best, ms);
    }
  }
  cudaStreamSynchronize(c->st);
  cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

void apply_tune(afqmc_ctx* c, const TuneVal& v) {
  c->xsplit = v.xsplit;
  c->bn_fb = v.bn_fb;
  c->bn_v = v.bn_v;
  c->bn_e = v.bn_e;
  c->bn_b = v.bn_b;
  c->taylor_fused = v.fused;
}

afqmc_status autotune(afqmc_ctx* c) {
  const TuneKey key = tune_key(c);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      apply_tune(c, it->second);
      return AFQMC_OK;
    }
  }
  const int64_t launches0 = c->launches;
  const std::string err0 = c->err;
  const int W = c->W, M = c->M, G = c->G;
  TuneVal v = {c->xsplit, 0, 0, 0, 0, c->taylor_fused};
  const int bns[2] = {64, 128};
  // force bias: K splits x tile width
  {
    const long kdim = (c->md ? c->ldg : c->ldt);
    const long ktiles = (kdim + 31) / 32;
    float best = INFINITY;
    for (int ks = 1; ks <= c->xsplit_max; ++ks) {
      if (ks > 1 && ktiles / ks < 4) break;
      for (int bn : bns) {
        c->xsplit = ks;
        c->bn_fb = bn;
        const float ms = best_ms(c, [&]() { return force_bias_contraction<float>(c); });
        if (ms < best) { best = ms; v.xsplit = ks; v.bn_fb = bn; }
      }
    }
  }
  // one-body operator
  {
    float best = INFINITY;
    for (int bn : bns) {
      const float ms = best_ms(c, [&]() -> afqmc_status {
        const long nv = c->sparse ? c->nnzp : (long)M * c->ldV;
        LK(tc_gemm(c->tc, c->st, 2 * W, (int)nv, G, (const float*)c->S, c->ldS,
                   (const float*)c->LT, c->ldS, (float*)c->V, nv, 1.0f, 0.0f, nullptr, 0,
                   c->split3, 1, 0, c->status, bn, (const float*)c->LT_lo,
                   c->tc_wide_ok && c->split3 && !c->sparse ? (float*)c->Vlo : nullptr,
                   c->tc_wide_ok && c->bf16 && !c->sparse));
        return AFQMC_OK;
      });
      if (ms < best) { best = ms; v.bn_v = bn; }
    }
  }
  // energy contraction (single determinant)
  if (!c->md) {
    float best = INFINITY;
    for (int bn : bns) {
      const float ms = best_ms(c, [&]() -> afqmc_status {
        long zoff = 0;
        for (int sig = 0; sig < 2; ++sig) {
          const int ns = sig ? c->nd : c->nu;
          const long off = sig ? c->dn_off : 0, ldz = c->Jp[sig];
          if (ns == 0) continue;
          const long J = (long)ns * M;
          LK(tc_gemm(c->tc, c->st, 2 * W, (int)J, (int)J, (const float*)c->Theta + off,
                     c->ldt, (const float*)(sig ? c->Yx_dn : c->Yx_up), ldz,
                     (float*)c->Z + zoff, ldz, 1.0f, 0.0f, nullptr, 0, c->split3, 1, 0,
                     c->status, bn, (const float*)(sig ? c->Yx_dn_lo : c->Yx_up_lo)));
          zoff += 2L * W * ldz;
        }
        return AFQMC_OK;
      });
      if (ms < best) { best = ms; v.bn_e = bn; }
    }
  }
  // propagation path (into the spare walker buffer Phi2); the block-diagonal
  // form has one path
  if (!c->sparse) {
    float best = INFINITY;
    for (int fused = c->tc_wide_ok ? 3 : (c->tc_taylor_ok ? 2 : 0); fused >= 0; --fused) {
      if (fused == 3 && !c->tc_wide_ok) continue;
      if ((fused == 1 || fused == 2) && !c->tc_taylor_ok) continue;
      c->taylor_fused = fused;
      for (int bn : bns) {
        if ((fused == 1 || fused == 3) && bn != bns[0]) continue;   // no half-step contraction
        if (fused != 1 && (!c->tc_bhalf_ok || M <= 64) && bn != bns[0]) continue;
        c->bn_b = bn;
        const float ms = best_ms(c, [&]() { return propagate_T<float>(c, (float*)c->Phi2); });
        if (ms < best) { best = ms; v.fused = fused; v.bn_b = (fused == 1 || fused == 3) ? 0 : bn; }
      }
    }
  }
  apply_tune(c, v);
  c->launches = launches0;
  c->err = err0;
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
  CK(cudaStreamSynchronize(c->st));
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.emplace(key, v);
  return AFQMC_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of blocks of steps. The cadence pattern of steps s+1 .. s+len
// depends only on s modulo the period (the lcm of the cadences), so a block
// captured at one phase replays at every later step with that phase.
// ---------------------------------------------------------------------------

long cadence_period(const afqmc_params* p) {
  long P = 1;
  const int ks[3] = {p->ortho_every, p->measure_every, p->pc_every};
  for (int k : ks) {
    if (k <= 0) continue;
    long a = P, b = k;
    while (b) { long t = a % b; a = b; b = t; }
    P = P / a * k;
    if (P > 4096) return 0;
  }
  return P;
}

void drop_graphs(afqmc_ctx* c) {
  for (auto& kv : c->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    cudaGraphDestroy(kv.second.graph);
  }
  c->graphs.clear();
}

afqmc_status step_any(afqmc_ctx* c) { return c->fp64 ? step_T<double>(c) : step_T<float>(c); }

// Capture `len` steps from the current phase. Host counters are left as
// they were. Returns AFQMC_E_STATE (with graphs switched off for the
// context, and no error recorded) when the stream cannot be captured.
afqmc_status capture_block(afqmc_ctx* c, long len, GraphEntry* ge) {
  const long step0 = c->step, meas0 = c->n_meas;
  const int64_t l0 = c->launches;
  const std::string err0 = c->err;
  if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    c->use_graphs = false;
    return AFQMC_E_STATE;
  }
  afqmc_status s = AFQMC_OK;
  for (long i = 0; i < len && s == AFQMC_OK; ++i) s = step_any(c);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->st, &g);
  ge->meas = c->n_meas - meas0;
  ge->launches = c->launches - l0;
  c->step = step0;
  c->n_meas = meas0;
  c->launches = l0;
  cudaGraphExec_t ex = nullptr;
  if (s == AFQMC_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (s != AFQMC_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    c->poisoned = false;
    c->err = err0;
    c->use_graphs = false;
    return AFQMC_E_STATE;
  }
  ge->graph = g;
  ge->exec = ex;
  return AFQMC_OK;
}

afqmc_status block_graph(afqmc_ctx* c, long len, GraphEntry** out) {
  const std::pair<long, long> key(c->step % c->period, len);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    GraphEntry ge;
    afqmc_status s = capture_block(c, len, &ge);
    if (s != AFQMC_OK) return s;
    it = c->graphs.emplace(key, ge).first;
  }
  *out = &it->second;
  return AFQMC_OK;
}

void advance_host(afqmc_ctx* c, long len, const GraphEntry* ge) {
  c->step += len;
  c->n_meas += ge->meas;
  c->launches += ge->launches;
}

// Strides, paths and sizes of a context, from its parameters alone (and the
// active-orbital counts of a multi-determinant trial).
struct Plan {
  int M, nu, nd, N, G, W, ndet, nact[2];
  bool fp64, tcmode, split3, bf16, md, mf, tc_taylor_ok, tc_bhalf_ok, tc_wide_ok;
  size_t es;
  long ldS, ldx, dn_off, ldt, Jp[2], gdn_off, ldg, ldV;
  int xsplit, xsplit_max;
};

Plan make_plan(const afqmc_params* p, int nact_up, int nact_dn) {
  Plan P;
  P.M = p->M; P.nu = p->n_up; P.nd = p->n_dn; P.N = P.nu + P.nd; P.G = p->n_chol;
  P.W = p->n_walkers; P.ndet = p->n_det;
  P.md = P.ndet > 1;
  P.mf = p->mf_subtract != 0;
  P.nact[0] = P.md ? nact_up : P.nu;
  P.nact[1] = P.md ? nact_dn : P.nd;
  P.fp64 = p->precision == AFQMC_FP64;
  P.tcmode = p->precision == AFQMC_TF32 || p->precision == AFQMC_TF32X3 ||
             p->precision == AFQMC_BF16X3;
  P.bf16 = p->precision == AFQMC_BF16X3;
  P.split3 = p->precision == AFQMC_TF32X3 || P.bf16;
  P.tc_taylor_ok = P.tcmode && P.M <= 64;
  P.tc_bhalf_ok = P.tcmode && P.M % 4 == 0;
  P.tc_wide_ok = P.tcmode && P.M > 64;
  // rows of V 16-byte aligned for the TMA: 4 FP32 or 8 BF16 values
  P.ldV = P.tc_wide_ok ? (P.bf16 ? (P.M + 7) / 8 * 8 : round4(P.M)) : P.M;
  P.es = P.fp64 ? sizeof(double) : sizeof(float);
  const int M = P.M, G = P.G, W = P.W;
  P.ldS = round4(G);
  P.ldx = G + 1;
  P.dn_off = round4((long)P.nu * M);
  P.ldt = P.dn_off + round4((long)P.nd * M);
  P.Jp[0] = round4((long)P.nu * M);
  P.Jp[1] = round4((long)P.nd * M);
  P.gdn_off = round4((long)P.nact[0] * M);
  P.ldg = P.gdn_off + round4((long)P.nact[1] * M);
  P.xsplit = 1;
  P.xsplit_max = 1;
  if (P.tcmode) {
    // split K of the force-bias contraction so that its few output tiles
    // still fill the GPU; partial sums are added in order by the consumers
    const long kdim = P.md ? P.ldg : P.ldt;
    const long tiles = ((2L * W + 127) / 128) * ((G + 1 + 127) / 128);
    const long ktiles = (kdim + 31) / 32;
    int ks = (int)(152 / (tiles > 0 ? tiles : 1));
    if (ks > 8) ks = 8;
    while (ks > 1 && ktiles / ks < 4) --ks;
    P.xsplit = ks < 1 ? 1 : ks;
    long mx = ktiles / 4;
    if (mx > 8) mx = 8;
    P.xsplit_max = (int)std::max<long>(mx, P.xsplit);
  }
  return P;
}

struct Buf {
  void** slot;
  size_t bytes;
};

// Every device buffer of a context (slots into c), in allocation order.
std::vector<Buf> buffer_list(afqmc_ctx* c, const Plan& P) {
  const size_t es = P.es, W = P.W, M = P.M, N = P.N, G = P.G;
  const size_t MM = M * M, phi = W * N * 2 * M;
  std::vector<Buf> b;
  auto add = [&](void* slot, size_t bytes) { b.push_back({(void**)slot, bytes ? bytes : 16}); };
  if (P.md) {
    add(&c->Gamma, W * 2 * P.ldg * es);
    add(&c->Gamma2, W * 2 * P.ldg * es);
    add(&c->LtilA, (G + 1) * P.ldg * es);
    add(&c->CactT64, (size_t)(P.nact[0] + P.nact[1]) * M * sizeof(double));
    add(&c->md_ct0, (size_t)P.nact[0] * M * es);
    add(&c->md_ct1, (size_t)P.nact[1] * M * es);
    add(&c->md_dets, sizeof(MdDet) * P.ndet);
    add(&c->md_cc, sizeof(double2) * P.ndet);
    add(&c->md_r0, sizeof(int) * (P.nu + 1));
    add(&c->md_r1, sizeof(int) * (P.nd + 1));
  }
  add(&c->Phi, phi * es);
  add(&c->Phi2, phi * es);
  add(&c->Phi3, phi * es);
  add(&c->Theta, W * 2 * P.ldt * es);
  add(&c->Theta2, W * 2 * P.ldt * es);
  add(&c->V, W * 2 * M * P.ldV * es);
  add(&c->X, (size_t)P.xsplit_max * W * 2 * P.ldx * es);
  add(&c->S, W * 2 * P.ldS * es);
  add(&c->xbar, W * 2 * G * es);
  add(&c->Z, 2 * W * (P.Jp[0] + P.Jp[1]) * es);
  add(&c->L, G * MM * es);
  add(&c->Ltil, (G + 1) * P.ldt * es);
  add(&c->Bhalf, MM * es);
  add(&c->PsiT, N * M * es);
  add(&c->PsiT64, N * M * sizeof(double));
  add(&c->Yx_up, (size_t)P.nu * M * P.Jp[0] * es);
  add(&c->Yx_dn, (size_t)P.nd * M * P.Jp[1] * es);
  if (P.tcmode) add(&c->LT, M * P.ldV * P.ldS * es);
  if (P.split3) {
    add(&c->Ltil_lo, (G + 1) * P.ldt * es);
    add(&c->LT_lo, M * P.ldV * P.ldS * es);
    add(&c->Yx_up_lo, (size_t)P.nu * M * P.Jp[0] * es);
    add(&c->Yx_dn_lo, (size_t)P.nd * M * P.Jp[1] * es);
  }
  if (!P.fp64) add(&c->dB, MM * es);
  if (P.tc_taylor_ok) add(&c->bimg, tc_bhalf_image_bytes(P.split3, P.bf16));
  if (P.tc_wide_ok) {
    add(&c->dBp, M * P.ldV * es);
    if (P.split3) {
      add(&c->dBp_lo, M * P.ldV * es);
      add(&c->Vlo, W * 2 * M * P.ldV * es);
    }
  }
  add(&c->weight, W * sizeof(double));
  add(&c->scan, W * sizeof(double));
  add(&c->lr, 2 * W * sizeof(double));
  add(&c->wnew, sizeof(double));
  add(&c->wref, sizeof(double));
  add(&c->log_scale, sizeof(double));
  add(&c->escalar, 2 * sizeof(double));
  add(&c->logO, W * sizeof(double2));
  add(&c->logO2, W * sizeof(double2));
  add(&c->logO_new, W * sizeof(double2));
  add(&c->logdet, 2 * W * sizeof(double2));
  add(&c->logdet2, 2 * W * sizeof(double2));
  add(&c->lw, W * sizeof(double2));
  add(&c->eloc, W * sizeof(double2));
  add(&c->hist, kHist * sizeof(double2));
  add(&c->blk, (size_t)M * (2 * sizeof(int4) + sizeof(int)));
  if (P.mf) {
    add(&c->lbar, G * sizeof(double));
    add(&c->lmf, W * sizeof(double2));
  }
  add(&c->parent, W * sizeof(int));
  add(&c->status, sizeof(int));
  add(&c->ctr, 2 * sizeof(long long));
  return b;
}

// FP64 staging held by setup_T (all of it until setup ends).
size_t setup_bytes(const Plan& P) {
  const size_t M = P.M, N = P.N, G = P.G, MM = M * M;
  size_t n = 0;
  auto add = [&](size_t k) { n += (k ? k : 1) * sizeof(double); };
  add(MM); add(G * MM); add(N * M); add(MM); add(MM);
  add((G + 1) * N * M); add(MM); add(MM); add(MM); add(MM);
  add((G + 1) * P.ldt);
  add(G + 1);                                   // trial-energy terms
  add((size_t)std::max(P.nu, P.nd) * M + 1);
  for (int sig = 0; sig < 2; ++sig) {
    const size_t ns = sig ? P.nd : P.nu;
    if (ns == 0) continue;
    const size_t J = ns * M;
    add(J * J);
    add(J * J);
  }
  if (P.tcmode) add(M * P.ldV * P.ldS);
  if (P.tc_wide_ok) add(M * P.ldV);
  if (P.md) add((G + 1) * P.ldg);
  return n;
}

// Active-orbital counts of a multi-determinant trial (reference orbitals
// plus every other orbital occupied by some determinant), per spin.
void count_active(const afqmc_params* p, const int32_t* ou, const int32_t* od, int* nact) {
  for (int sg = 0; sg < 2; ++sg) {
    const int ns = sg ? p->n_dn : p->n_up;
    const int32_t* occ = sg ? od : ou;
    std::vector<char> used(p->M, 0);
    int n = 0;
    for (long e = 0; e < (long)p->n_det * ns; ++e) {
      const int o = occ[e];
      if (o >= 0 && o < p->M && !used[o]) { used[o] = 1; ++n; }
    }
    nact[sg] = n;
  }
}

afqmc_status create_impl(afqmc_ctx* c, const double* h1, const double* L,
                         const double* Cu, const double* Cd, const int32_t* ou,
                         const int32_t* od) {
  const int M = c->M;
  c->md = c->ndet > 1;
  std::vector<MdDet> dets_h;
  std::vector<double2> cconj_h;
  c->nact[0] = c->nu;
  c->nact[1] = c->nd;
  if (c->md) {
    afqmc_status s0 = prepare_multidet(c, ou, od, c->ci_h, dets_h, cconj_h);
    if (s0 != AFQMC_OK) return s0;
  }
  const Plan P = make_plan(&c->p, c->nact[0], c->nact[1]);
  c->ldS = P.ldS;
  c->ldx = P.ldx;
  c->dn_off = P.dn_off;
  c->ldt = P.ldt;
  c->Jp[0] = P.Jp[0];
  c->Jp[1] = P.Jp[1];
  c->gdn_off = P.gdn_off;
  c->ldg = P.ldg;
  c->xsplit = P.xsplit;
  c->xsplit_max = P.xsplit_max;
  c->split3 = P.split3;
  c->bf16 = P.bf16;
  c->tc_taylor_ok = P.tc_taylor_ok;
  c->tc_bhalf_ok = P.tc_bhalf_ok;
  c->tc_wide_ok = P.tc_wide_ok;
  c->ldV = P.ldV;
  c->taylor_fused = P.tc_taylor_ok ? 1 : (P.tc_wide_ok ? 3 : 0);
  BlockPlan B = detect_blocks(&c->p, L);
  c->sparse = B.on;
  if (c->sparse) {
    c->nnz = B.nnz;
    c->nnzp = round4(B.nnz);
    c->nblk = B.nb;
    c->maxblk = B.maxb;
    c->taylor_fused = 4;
    c->blk_gidx.swap(B.gidx);
  }
  c->bn_fb = c->bn_v = c->bn_e = c->bn_b = 0;
  if (c->md) {
    const bool f64c = c->fp64_islands;
    if (md_energy_smem(M, c->nu, c->nd, c->nact[0], c->nact[1], c->ndet, f64c) > 227 * 1024)
      return fail(c, AFQMC_E_INVALID,
                  "multi-determinant trial too large for the on-chip energy kernel");
  }
  for (const Buf& b : buffer_list(c, P)) {
    afqmc_status s0 = dalloc(c, b.slot, b.bytes);
    if (s0 != AFQMC_OK) return s0;
  }
  const size_t es = P.es;
  const int W = c->W, G = c->G;
  if (c->md) {
    std::vector<int> ract_u(c->nu + 1), ract_d(c->nd + 1);
    for (int a = 0; a <= c->nu; ++a) ract_u[a] = a;
    for (int a = 0; a <= c->nd; ++a) ract_d[a] = a;
    long ctot = 0;                       // compact C table offsets
    for (MdDet& d : dets_h) {
      d.coff = (int)ctot;
      ctot += (long)d.E[0] * c->nu + (long)d.E[1] * c->nd;
    }
    c->mdt.ctot = (int)ctot;
    CK(cudaMemcpyAsync(c->md_dets, dets_h.data(), sizeof(MdDet) * c->ndet,
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->md_cc, cconj_h.data(), sizeof(double2) * c->ndet,
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->md_r0, ract_u.data(), sizeof(int) * (c->nu + 1),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->md_r1, ract_d.data(), sizeof(int) * (c->nd + 1),
                       cudaMemcpyHostToDevice, c->st));
    // active orbitals as rows, FP64 copy for read-outs
    std::vector<double> cact((size_t)(c->nact[0] + c->nact[1]) * M);
    for (int sg = 0; sg < 2; ++sg) {
      const double* C = sg ? Cd : Cu;
      const size_t off = sg ? (size_t)c->nact[0] * M : 0;
      for (int q = 0; q < c->nact[sg]; ++q)
        for (int k = 0; k < M; ++k)
          cact[off + (size_t)q * M + k] = C[(size_t)k * M + c->act_h[sg][q]];
    }
    CK(cudaMemcpyAsync(c->CactT64, cact.data(), cact.size() * sizeof(double),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->mdt.ndet = c->ndet;
    c->mdt.nact[0] = c->nact[0];
    c->mdt.nact[1] = c->nact[1];
    c->mdt.dets = (const MdDet*)c->md_dets;
    c->mdt.cconj = (const double2*)c->md_cc;
    c->mdt.ract[0] = (const int*)c->md_r0;
    c->mdt.ract[1] = (const int*)c->md_r1;
    c->mdt.CactT[0] = c->md_ct0;
    c->mdt.CactT[1] = c->md_ct1;
  }
  {
    // M int4 rows, M int4 block slots, then the M members (the int4 arrays
    // 16-byte aligned)
    std::vector<int> tab((size_t)M * 9, 0);
    if (c->sparse) {
      int nb = 0;
      for (int i = 0; i < M; ++i) {
        tab[4 * i] = B.vrow[i];
        tab[4 * i + 1] = B.bsize[i];
        tab[4 * i + 2] = B.ibase[i];
        tab[8 * (size_t)M + i] = B.members[i];
      }
      for (int k = 0; k < M; k += B.bsize[B.members[k]], ++nb) {   // blocks in member order
        const int first = B.members[k];
        int* bt = &tab[4 * (size_t)M + 4 * (size_t)nb];
        bt[0] = B.vrow[first];
        bt[1] = B.bsize[first];
        bt[2] = k;
      }
    }
    CK(cudaMemcpyAsync(c->blk, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice,
                       c->st));
    CK(cudaStreamSynchronize(c->st));
  }
  CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->st));
  CK(cudaMemsetAsync(c->ctr, 0, 2 * sizeof(long long), c->st));
  CK(cudaMemsetAsync(c->lw, 0, W * sizeof(double2), c->st));
  CK(cudaMemsetAsync(c->xbar, 0, (size_t)W * 2 * G * es, c->st));
  CK(cudaMemsetAsync(c->S, 0, (size_t)W * 2 * c->ldS * es, c->st));
  CK(cudaMemsetAsync(c->V, 0, (size_t)W * 2 * M * c->ldV * es, c->st));
  if (c->Vlo) CK(cudaMemsetAsync(c->Vlo, 0, (size_t)W * 2 * M * c->ldV * es, c->st));
  CK(cudaMemsetAsync(c->Theta, 0, (size_t)W * 2 * c->ldt * es, c->st));
  CK(cudaMemsetAsync(c->Theta2, 0, (size_t)W * 2 * c->ldt * es, c->st));
  CK(cudaMemsetAsync(c->X, 0, (size_t)c->xsplit_max * W * 2 * c->ldx * es, c->st));
  if (P.tcmode) {
    cudaError_t e = tc_create(&c->tc);
    if (e != cudaSuccess)
      return fail(c, AFQMC_E_CUDA, std::string("tensor-core setup: ") + cudaGetErrorString(e));
  }
  afqmc_status s = c->fp64 ? setup_T<double>(c, h1, L, Cu, Cd, ou, od)
                           : setup_T<float>(c, h1, L, Cu, Cd, ou, od);
  std::vector<int>().swap(c->blk_gidx);
  if (s != AFQMC_OK) return s;
  if (c->tc && c->p.autotune) {
    s = autotune(c);
    if (s != AFQMC_OK) return s;
  }
  CK(cudaStreamSynchronize(c->st));
  return AFQMC_OK;
}

#define GUARD(c)                                                        \
  do {                                                                  \
    if (!(c)) return AFQMC_E_INVALID;                                   \
    if ((c)->poisoned) return fail((c), AFQMC_E_CUDA, "context is poisoned by an earlier CUDA error: " + (c)->err); \
  } while (0)

}  // namespace

extern "C" {

void afqmc_params_default(afqmc_params* p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->n_det = 1;
  p->taylor_order = 6;
  p->fb_cap = 1.0;
  p->e_shift = NAN;
  p->precision = AFQMC_FP64;
  p->ortho_every = 2;
  p->measure_every = 20;
  p->pc_every = 20;
  p->graphs = 1;
  p->autotune = 1;
}

afqmc_status afqmc_create(const afqmc_params* params, const double* h1, const double* L,
                          const double* C_up, const double* C_dn, const int32_t* occ_up,
                          const int32_t* occ_dn, const double* ci, void* stream,
                          afqmc_ctx** out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, AFQMC_E_INVALID, "out is NULL");
  *out = nullptr;
  afqmc_status s = validate(params, h1, L, C_up, C_dn, occ_up, occ_dn, ci);
  if (s != AFQMC_OK) return s;
  afqmc_ctx* c = new afqmc_ctx();
  c->p = *params;
  c->M = params->M;
  c->nu = params->n_up;
  c->nd = params->n_dn;
  c->N = c->nu + c->nd;
  c->G = params->n_chol;
  c->W = params->n_walkers;
  c->ndet = params->n_det;
  c->fp64 = params->precision == AFQMC_FP64;
  c->fp64_islands = c->fp64 || params->fp64_islands == 1;
  c->fp64_qr = c->fp64 || params->fp64_islands != 0;
  c->step = 0;
  c->n_meas = 0;
  c->poisoned = false;
  c->launches = 0;
  c->dev_bytes = 0;
  c->timing = false;
  c->tc = nullptr;
  c->use_graphs = params->graphs != 0;
  c->period = cadence_period(params);
  for (int i = 0; i < AFQMC_N_KERNEL_IDS; ++i) { c->k_launch[i] = 0; c->k_ms[i] = 0.0; }
  if (stream) {
    c->st = (cudaStream_t)stream;
    c->own_stream = false;
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, AFQMC_E_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  c->ci_h = ci;
  s = create_impl(c, h1, L, C_up, C_dn, occ_up, occ_dn);
  c->ci_h = nullptr;
  if (s != AFQMC_OK) {
    g_create_err = c->err;
    afqmc_destroy(c);
    return s;
  }
  *out = c;
  return AFQMC_OK;
}

afqmc_status afqmc_propagate(afqmc_ctx* c, int32_t n_steps) {
  GUARD(c);
  if (n_steps < 0) return fail(c, AFQMC_E_INVALID, "n_steps < 0");
  long n = n_steps;
  // whole periods as graph replays (at least ~32 steps per replay when the
  // period is short), the remainder as plain launches
  while (c->use_graphs && !c->timing && c->period > 0 && n >= c->period) {
    const long per = c->period;
    long k = std::min(n / per, std::max(1L, 32 / per));
    const long len = k * per;
    GraphEntry* ge = nullptr;
    afqmc_status s = block_graph(c, len, &ge);
    if (s == AFQMC_E_STATE) break;   // not capturable: plain launches
    if (s != AFQMC_OK) return s;
    CK(cudaGraphLaunch(ge->exec, c->st));
    advance_host(c, len, ge);
    n -= len;
  }
  for (long i = 0; i < n; ++i) {
    afqmc_status s = step_any(c);
    if (s != AFQMC_OK) return s;
  }
  return AFQMC_OK;
}

afqmc_status afqmc_orthonormalize(afqmc_ctx* c) {
  GUARD(c);
  return c->fp64 ? mgs_T<double>(c) : mgs_T<float>(c);
}

afqmc_status afqmc_population_control(afqmc_ctx* c) {
  GUARD(c);
  afqmc_status s = c->fp64 ? comb_T<double>(c) : comb_T<float>(c);
  if (s != AFQMC_OK) return s;
  return check_status(c);
}

afqmc_status afqmc_local_energy(afqmc_ctx* c, double* e_loc, double* e_mixed) {
  GUARD(c);
  afqmc_status s = c->fp64 ? measure_T<double>(c, false) : measure_T<float>(c, false);
  if (s != AFQMC_OK) return s;
  if (e_loc)
    CK(cudaMemcpyAsync(e_loc, c->eloc, c->W * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
  double em = 0.0;
  CK(cudaMemcpyAsync(&em, c->escalar, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (e_mixed) *e_mixed = em;
  return check_status(c);
}

afqmc_status afqmc_weights(afqmc_ctx* c, double* w, double* log_ovlp) {
  GUARD(c);
  if (w) CK(cudaMemcpyAsync(w, c->weight, c->W * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  if (log_ovlp)
    CK(cudaMemcpyAsync(log_ovlp, c->logO, c->W * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return check_status(c);
}

afqmc_status afqmc_green(afqmc_ctx* c, int32_t walker, double* G_up, double* G_dn) {
  GUARD(c);
  if (walker < 0 || walker >= c->W) return fail(c, AFQMC_E_INVALID, "walker out of range");
  const int M = c->M, N = c->N;
  const size_t es = esize(c);
  std::vector<unsigned char> th(2 * (size_t)c->ldt * es);
  CK(cudaMemcpyAsync(th.data(), (const unsigned char*)c->Theta + (size_t)walker * 2 * c->ldt * es,
                     th.size(), cudaMemcpyDeviceToHost, c->st));
  std::vector<double> psi((size_t)N * M);
  CK(cudaMemcpyAsync(psi.data(), c->PsiT64, psi.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  auto theta = [&](int cc, int a, int k) -> double {
    size_t idx = (size_t)cc * c->ldt + (a < c->nu ? (size_t)a * M
                                                  : c->dn_off + (size_t)(a - c->nu) * M) + k;
    return c->fp64 ? ((const double*)th.data())[idx] : (double)((const float*)th.data())[idx];
  };
  if (c->md) {   // G_ij = sum_q Gamma[q][j] C_act[i][q]
    std::vector<unsigned char> gb(2 * (size_t)c->ldg * es);
    CK(cudaMemcpyAsync(gb.data(), (const unsigned char*)c->Gamma + (size_t)walker * 2 * c->ldg * es,
                       gb.size(), cudaMemcpyDeviceToHost, c->st));
    std::vector<double> ca((size_t)(c->nact[0] + c->nact[1]) * M);
    CK(cudaMemcpyAsync(ca.data(), c->CactT64, ca.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    auto gam = [&](int cc, size_t idx) -> double {
      idx += (size_t)cc * c->ldg;
      return c->fp64 ? ((const double*)gb.data())[idx] : (double)((const float*)gb.data())[idx];
    };
    for (int sig = 0; sig < 2; ++sig) {
      double* G = sig ? G_dn : G_up;
      if (!G) continue;
      const int na = c->nact[sig];
      const size_t goff = sig ? c->gdn_off : 0, coff = sig ? (size_t)c->nact[0] * M : 0;
      for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
          double re = 0.0, im = 0.0;
          for (int q = 0; q < na; ++q) {
            const double cv = ca[coff + (size_t)q * M + i];
            re += gam(0, goff + (size_t)q * M + j) * cv;
            im += gam(1, goff + (size_t)q * M + j) * cv;
          }
          G[2 * ((size_t)i * M + j)] = re;
          G[2 * ((size_t)i * M + j) + 1] = im;
        }
    }
    return AFQMC_OK;
  }
  // G_ij = sum_a Theta_ja D_ia (G^T = Theta D^H, real trial orbitals)
  for (int sig = 0; sig < 2; ++sig) {
    double* G = sig ? G_dn : G_up;
    if (!G) continue;
    const int ns = sig ? c->nd : c->nu, j0 = sig ? c->nu : 0;
    for (int i = 0; i < M; ++i)
      for (int j = 0; j < M; ++j) {
        double re = 0.0, im = 0.0;
        for (int a = 0; a < ns; ++a) {
          double d = psi[(size_t)(j0 + a) * M + i];
          re += theta(0, j0 + a, j) * d;
          im += theta(1, j0 + a, j) * d;
        }
        G[2 * ((size_t)i * M + j)] = re;
        G[2 * ((size_t)i * M + j) + 1] = im;
      }
  }
  return AFQMC_OK;
}

afqmc_status afqmc_selftest_wait_timeout(afqmc_ctx* c, int64_t limit_cycles) {
  GUARD(c);
  if (limit_cycles < 0 || limit_cycles > 4000000000LL)
    return fail(c, AFQMC_E_INVALID, "limit_cycles must be in 0..4e9");
  CK(cudaStreamSynchronize(c->st));
  LK(tc_wait_timeout_probe(c->st, (long long)limit_cycles, c->status));
  return check_status(c);
}

afqmc_status afqmc_energy_shift(afqmc_ctx* c, double* e_shift) {
  GUARD(c);
  if (!e_shift) return fail(c, AFQMC_E_INVALID, "e_shift is NULL");
  *e_shift = c->e_shift;
  return AFQMC_OK;
}

afqmc_status afqmc_log_weight_scale(afqmc_ctx* c, double* log_scale) {
  GUARD(c);
  if (!log_scale) return fail(c, AFQMC_E_INVALID, "log_scale is NULL");
  CK(cudaMemcpyAsync(log_scale, c->log_scale, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return AFQMC_OK;
}

afqmc_status afqmc_force_bias(afqmc_ctx* c, double* xbar) {
  GUARD(c);
  if (!xbar) return fail(c, AFQMC_E_INVALID, "xbar is NULL");
  const size_t n = (size_t)c->W * 2 * c->G;
  std::vector<unsigned char> buf(n * esize(c));
  CK(cudaMemcpyAsync(buf.data(), c->xbar, buf.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int w = 0; w < c->W; ++w)
    for (int cc = 0; cc < 2; ++cc)
      for (int g = 0; g < c->G; ++g) {
        size_t src = ((size_t)w * 2 + cc) * c->G + g;
        double v = c->fp64 ? ((double*)buf.data())[src] : (double)((float*)buf.data())[src];
        xbar[((size_t)w * c->G + g) * 2 + cc] = v;
      }
  return AFQMC_OK;
}

afqmc_status afqmc_energy_history(afqmc_ctx* c, double* out, int32_t max_n, int32_t* n) {
  GUARD(c);
  const long have = c->n_meas < kHist ? c->n_meas : kHist;
  if (n) *n = (int32_t)c->n_meas;
  if (out && max_n > 0) {
    std::vector<double2> h(kHist);
    CK(cudaMemcpyAsync(h.data(), c->hist, kHist * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    long first = c->n_meas - have;
    long cnt = have < max_n ? have : max_n;
    for (long i = 0; i < cnt; ++i) {
      double2 v = h[(first + i) % kHist];
      out[2 * i] = v.x;
      out[2 * i + 1] = v.y;
    }
  }
  return AFQMC_OK;
}

afqmc_status afqmc_get_state(afqmc_ctx* c, void* buf, size_t* bytes) {
  GUARD(c);
  if (!bytes) return fail(c, AFQMC_E_INVALID, "bytes is NULL");
  const int W = c->W, N = c->N, M = c->M;
  const size_t need = sizeof(StateHeader) + (size_t)W * N * M * 16 + (size_t)W * 8 +
                      (size_t)W * 16;
  if (!buf) { *bytes = need; return AFQMC_OK; }
  if (*bytes < need) return fail(c, AFQMC_E_INVALID, "state buffer too small");
  const size_t es = esize(c);
  const size_t phi = (size_t)W * N * 2 * M;
  std::vector<unsigned char> ph(phi * es);
  unsigned char* out = (unsigned char*)buf;
  StateHeader h;
  memcpy(h.magic, "AFQMCST1", 8);
  h.M = M; h.n_up = c->nu; h.n_dn = c->nd; h.n_walkers = W;
  h.step = c->step; h.seed = c->p.seed; h.run_id = c->p.run_id; h.n_chol = c->G;
  memcpy(out, &h, sizeof(h));
  double* z = (double*)(out + sizeof(h));
  double* wt = z + (size_t)W * N * M * 2;
  double* lo = wt + W;
  CK(cudaMemcpyAsync(ph.data(), c->Phi, ph.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(wt, c->weight, W * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(lo, c->logO, W * sizeof(double2), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (size_t w = 0; w < (size_t)W; ++w)
    for (int j = 0; j < N; ++j)
      for (int cc = 0; cc < 2; ++cc)
        for (int k = 0; k < M; ++k) {
          size_t src = ((w * N + j) * 2 + cc) * M + k;
          double v = c->fp64 ? ((double*)ph.data())[src] : (double)((float*)ph.data())[src];
          z[((w * N + j) * M + k) * 2 + cc] = v;
        }
  *bytes = need;
  return AFQMC_OK;
}

afqmc_status afqmc_set_state(afqmc_ctx* c, const void* buf, size_t bytes) {
  GUARD(c);
  const int W = c->W, N = c->N, M = c->M;
  const size_t need = sizeof(StateHeader) + (size_t)W * N * M * 16 + (size_t)W * 8 +
                      (size_t)W * 16;
  if (!buf || bytes < need) return fail(c, AFQMC_E_STATE, "state image too small");
  StateHeader h;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, "AFQMCST1", 8) != 0 || h.M != M || h.n_up != c->nu ||
      h.n_dn != c->nd || h.n_walkers != W || h.n_chol != c->G)
    return fail(c, AFQMC_E_STATE, "state image does not match this context");
  const double* z = (const double*)((const unsigned char*)buf + sizeof(h));
  const double* wt = z + (size_t)W * N * M * 2;
  const double* lo = wt + W;
  const size_t es = esize(c);
  const size_t phi = (size_t)W * N * 2 * M;
  std::vector<unsigned char> ph(phi * es);
  for (size_t w = 0; w < (size_t)W; ++w)
    for (int j = 0; j < N; ++j)
      for (int cc = 0; cc < 2; ++cc)
        for (int k = 0; k < M; ++k) {
          size_t dst = ((w * N + j) * 2 + cc) * M + k;
          double v = z[((w * N + j) * M + k) * 2 + cc];
          if (c->fp64) ((double*)ph.data())[dst] = v;
          else ((float*)ph.data())[dst] = (float)v;
        }
  CK(cudaMemcpyAsync(c->Phi, ph.data(), ph.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->weight, wt, W * sizeof(double), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->logO, lo, W * sizeof(double2), cudaMemcpyHostToDevice, c->st));
  {                                   // reference weight of the weight cap
    double sum = 0.0;
    int live = 0;
    for (int w = 0; w < W; ++w)
      if (wt[w] > 0.0) { sum += wt[w]; ++live; }
    c->wref_host = live ? sum / live : 1.0;
    CK(cudaMemcpyAsync(c->wref, &c->wref_host, sizeof(double), cudaMemcpyHostToDevice, c->st));
    // the image's weights are absolute: the log scale starts again from 0
    CK(cudaMemsetAsync(c->log_scale, 0, sizeof(double), c->st));
  }
  c->step = h.step;
  const long long ctr_h[2] = {(long long)c->step, (long long)c->n_meas};
  CK(cudaMemcpyAsync(c->ctr, ctr_h, sizeof(ctr_h), cudaMemcpyHostToDevice, c->st));
  afqmc_status s = c->fp64 ? overlap_T<double>(c, c->logO_new) : overlap_T<float>(c, c->logO_new);
  if (s != AFQMC_OK) return s;
  CK(cudaStreamSynchronize(c->st));
  return AFQMC_OK;
}

afqmc_status afqmc_synchronize(afqmc_ctx* c) {
  GUARD(c);
  CK(cudaStreamSynchronize(c->st));
  return check_status(c);
}

afqmc_status afqmc_set_kernel_timing(afqmc_ctx* c, int32_t enable) {
  GUARD(c);
  afqmc_status s = drain_timers(c);
  if (s != AFQMC_OK) return s;
  c->timing = enable != 0;
  for (int i = 0; i < AFQMC_N_KERNEL_IDS; ++i) { c->k_launch[i] = 0; c->k_ms[i] = 0.0; }
  return AFQMC_OK;
}

afqmc_status afqmc_kernel_stats(afqmc_ctx* c, int32_t id, int64_t* launches, double* total_ms,
                                double* work, int32_t* is_bytes) {
  GUARD(c);
  if (id < 0 || id >= AFQMC_N_KERNEL_IDS) return fail(c, AFQMC_E_INVALID, "unknown kernel id");
  afqmc_status s = drain_timers(c);
  if (s != AFQMC_OK) return s;
  const double W = c->W, M = c->M, N = c->N, G = c->G, T = c->p.taylor_order;
  const double es = (double)esize(c);
  double wk = 0.0;
  int byt = 0;
  switch (id) {
    case 0: wk = 4.0 * W * G * N * M; break;                         // Theta . L~^T
    case 1: wk = W * 2 * G * es * 3 + W * 16; byt = 1; break;        // X in, S + xbar out
    case 2: wk = 4.0 * W * G * (c->sparse ? (double)c->nnz : M * M); break;   // S . L
    case 3: wk = 8.0 * T * (c->sparse ? (double)c->nnz : M * M) * N * W + 8.0 * M * M * N * W;
      break;
    case 4: {
      double f = 0.0;
      for (int sig = 0; sig < 2; ++sig) {
        double ns = sig ? c->nd : c->nu;
        f += 12.0 * M * ns * ns + 8.0 * ns * ns * ns;
      }
      wk = f * W;
      break;
    }
    case 5: wk = W * (8 + 16 + 16 + 16 + 8 + 16); byt = 1; break;
    case 6: {
      double f = 0.0;
      for (int sig = 0; sig < 2; ++sig) {
        double ns = sig ? c->nd : c->nu;
        f += 8.0 * M * ns * ns;
      }
      wk = f * W;
      break;
    }
    case 7: {
      double f = 0.0;
      for (int sig = 0; sig < 2; ++sig) {
        double J = (sig ? c->nd : c->nu) * M;
        f += 4.0 * J * J;
      }
      wk = f * W;
      break;
    }
    case 8: wk = W * (2.0 * (2 * N * 2 * M * es) + 16 + 8 + 8); byt = 1; break;
  }
  if (launches) *launches = c->k_launch[id];
  if (total_ms) *total_ms = c->k_ms[id];
  if (work) *work = wk;
  if (is_bytes) *is_bytes = byt;
  return AFQMC_OK;
}

int64_t afqmc_launch_count(const afqmc_ctx* c) { return c ? c->launches : 0; }

afqmc_status afqmc_get_tuning(afqmc_ctx* c, afqmc_tuning* out) {
  GUARD(c);
  if (!out) return fail(c, AFQMC_E_INVALID, "out is NULL");
  memset(out, 0, sizeof(*out));
  out->xsplit = c->xsplit;
  if (c->tc) {
    out->bn_force_bias = c->bn_fb ? c->bn_fb : (c->G + 1 <= 64 ? 64 : 128);
    out->bn_one_body = c->bn_v ? c->bn_v : (c->M * c->M <= 64 ? 64 : 128);
    long jmax = (long)std::max(c->nu, c->nd) * c->M;
    out->bn_energy = c->bn_e ? c->bn_e : (jmax <= 64 ? 64 : 128);
    out->bn_half_step = c->bn_b ? c->bn_b : (c->M <= 64 ? 64 : 128);
    out->taylor_fused = c->taylor_fused;
  }
  return AFQMC_OK;
}

afqmc_status afqmc_set_tuning(afqmc_ctx* c, const afqmc_tuning* t) {
  GUARD(c);
  if (!t) return fail(c, AFQMC_E_INVALID, "tuning is NULL");
  if (t->reserved[0] || t->reserved[1]) return fail(c, AFQMC_E_INVALID, "reserved fields must be zero");
  if (!c->tc) {
    if (t->xsplit != 1 || t->bn_force_bias || t->bn_one_body || t->bn_energy ||
        t->bn_half_step || t->taylor_fused)
      return fail(c, AFQMC_E_INVALID, "launch shapes apply to the tensor-core modes only");
    return AFQMC_OK;
  }
  auto bn_ok = [](int b) { return b == 64 || b == 128; };
  if (t->xsplit < 1 || t->xsplit > c->xsplit_max)
    return fail(c, AFQMC_E_INVALID,
                "xsplit must be in 1.." + std::to_string(c->xsplit_max) + " for this system");
  if (!bn_ok(t->bn_force_bias) || !bn_ok(t->bn_one_body) || !bn_ok(t->bn_energy) ||
      !bn_ok(t->bn_half_step))
    return fail(c, AFQMC_E_INVALID, "tile widths must be 64 or 128");
  if (t->taylor_fused < 0 || t->taylor_fused > 4)
    return fail(c, AFQMC_E_INVALID, "taylor_fused must be 0, 1, 2, 3 or 4");
  if ((t->taylor_fused == 4) != c->sparse)
    return fail(c, AFQMC_E_INVALID,
                c->sparse ? "block-diagonal Cholesky vectors: the propagation path is 4"
                          : "taylor_fused = 4 needs block-diagonal Cholesky vectors");
  if ((t->taylor_fused == 1 || t->taylor_fused == 2) && !c->tc_taylor_ok)
    return fail(c, AFQMC_E_INVALID, "the on-chip tensor-core Taylor kernel needs M <= 64");
  if (t->taylor_fused == 3 && !c->tc_wide_ok)
    return fail(c, AFQMC_E_INVALID, "the streamed tensor-core Taylor kernel needs M > 64");
  CK(cudaStreamSynchronize(c->st));
  drop_graphs(c);
  apply_tune(c, TuneVal{t->xsplit, t->bn_force_bias, t->bn_one_body, t->bn_energy,
                        t->bn_half_step, t->taylor_fused});
  return AFQMC_OK;
}

afqmc_status afqmc_footprint(const afqmc_params* p, const int32_t* occ_up,
                             const int32_t* occ_dn, size_t* resident, size_t* setup_peak) {
  g_create_err.clear();
  afqmc_status s = validate_sizes(p);
  if (s != AFQMC_OK) return s;
  int nact[2] = {p->n_up, p->n_dn};
  if (p->n_det > 1) {
    if (!occ_up || !occ_dn)
      return fail(nullptr, AFQMC_E_INVALID, "a multi-determinant footprint needs the occupations");
    count_active(p, occ_up, occ_dn, nact);
    const bool f64c = p->precision == AFQMC_FP64 || p->fp64_islands == 1;
    if (md_energy_smem(p->M, p->n_up, p->n_dn, nact[0], nact[1], p->n_det, f64c) > 227 * 1024)
      return fail(nullptr, AFQMC_E_INVALID,
                  "multi-determinant trial too large for the on-chip energy kernel");
  }
  const Plan P = make_plan(p, nact[0], nact[1]);
  afqmc_ctx dummy;
  size_t total = 0;
  for (const Buf& b : buffer_list(&dummy, P)) total += b.bytes;
  if (resident) *resident = total;
  if (setup_peak) *setup_peak = setup_bytes(P);
  return AFQMC_OK;
}

size_t afqmc_device_bytes(const afqmc_ctx* c) { return c ? c->dev_bytes : 0; }

int32_t afqmc_graph_count(const afqmc_ctx* c) { return c ? (int32_t)c->graphs.size() : 0; }

const char* afqmc_last_error(const afqmc_ctx* c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}

void afqmc_destroy(afqmc_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  for (auto& t : c->pending) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
  for (auto e : c->free_events) cudaEventDestroy(e);
  drop_graphs(c);
  if (c->tc) tc_destroy(c->tc);
  for (void* p : c->allocs) cudaFree(p);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

// ---------------------------------------------------------------------------
// Multi-system batching: one graph launch per block, one branch per member.
// ---------------------------------------------------------------------------

struct afqmc_batch {
  std::vector<afqmc_ctx*> ctx;
  long spb;
  cudaStream_t st;
  cudaEvent_t done;
  std::vector<cudaEvent_t> ready;
  // instantiated batch graphs keyed by the members' phases
  std::map<std::vector<long>, cudaGraphExec_t> execs;
  int64_t launches;
};

afqmc_status afqmc_batch_create(afqmc_ctx* const* ctxs, int32_t n, int32_t steps_per_block,
                                afqmc_batch** out) {
  g_create_err.clear();
  if (!out) return fail(nullptr, AFQMC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1) return fail(nullptr, AFQMC_E_INVALID, "a batch needs at least one context");
  if (steps_per_block < 1) return fail(nullptr, AFQMC_E_INVALID, "steps_per_block must be >= 1");
  for (int i = 0; i < n; ++i) {
    afqmc_ctx* c = ctxs[i];
    if (!c) return fail(nullptr, AFQMC_E_INVALID, "NULL context in the batch");
    if (c->poisoned) return fail(nullptr, AFQMC_E_INVALID, "a member context is poisoned");
    if (c->period <= 0)
      return fail(nullptr, AFQMC_E_INVALID, "a member's cadence period exceeds 4096 steps");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == c) return fail(nullptr, AFQMC_E_INVALID, "a context appears twice");
  }
  afqmc_batch* b = new afqmc_batch();
  b->ctx.assign(ctxs, ctxs + n);
  b->spb = steps_per_block;
  b->launches = 0;
  b->st = nullptr;
  b->done = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ready.push_back(ev);
  }
  if (e != cudaSuccess) {
    afqmc_batch_destroy(b);
    cudaGetLastError();
    return fail(nullptr, AFQMC_E_CUDA, std::string("batch stream: ") + cudaGetErrorString(e));
  }
  *out = b;
  return AFQMC_OK;
}

afqmc_status afqmc_batch_propagate(afqmc_batch* b, int32_t n_blocks) {
  if (!b) return fail(nullptr, AFQMC_E_INVALID, "batch is NULL");
  if (n_blocks < 0) return fail(nullptr, AFQMC_E_INVALID, "n_blocks < 0");
  const size_t n = b->ctx.size();
  for (int blk = 0; blk < n_blocks; ++blk) {
    std::vector<long> key(n);
    std::vector<GraphEntry*> ge(n);
    for (size_t i = 0; i < n; ++i) {
      afqmc_ctx* c = b->ctx[i];
      if (c->poisoned) return fail(nullptr, AFQMC_E_CUDA, "member context poisoned: " + c->err);
      if (c->timing) return fail(nullptr, AFQMC_E_INVALID, "kernel timing is on for a member");
      const bool was = c->use_graphs;
      c->use_graphs = true;
      afqmc_status s = block_graph(c, b->spb, &ge[i]);
      c->use_graphs = was && c->use_graphs;
      if (s == AFQMC_E_STATE)
        return fail(nullptr, AFQMC_E_CUDA, "a member's block could not be captured");
      if (s != AFQMC_OK) return fail(nullptr, s, "member " + std::to_string(i) + ": " + c->err);
      key[i] = c->step % c->period;
    }
    auto it = b->execs.find(key);
    if (it == b->execs.end()) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaGraphCreate(&g, 0);
      for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
        cudaGraphNode_t node;
        e = cudaGraphAddChildGraphNode(&node, g, nullptr, 0, ge[i]->graph);
      }
      cudaGraphExec_t ex = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, AFQMC_E_CUDA, std::string("batch graph: ") + cudaGetErrorString(e));
      }
      it = b->execs.emplace(key, ex).first;
    }
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) {
      e = cudaEventRecord(b->ready[i], b->ctx[i]->st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->ready[i], 0);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(it->second, b->st);
    if (e == cudaSuccess) e = cudaEventRecord(b->done, b->st);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i)
      e = cudaStreamWaitEvent(b->ctx[i]->st, b->done, 0);
    if (e != cudaSuccess)
      return fail(nullptr, AFQMC_E_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    b->launches += 1;
    for (size_t i = 0; i < n; ++i) advance_host(b->ctx[i], b->spb, ge[i]);
  }
  return AFQMC_OK;
}

int64_t afqmc_batch_launches(const afqmc_batch* b) { return b ? b->launches : 0; }

afqmc_status afqmc_batch_synchronize(afqmc_batch* b) {
  if (!b) return fail(nullptr, AFQMC_E_INVALID, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess)
    return fail(nullptr, AFQMC_E_CUDA, std::string("batch: ") + cudaGetErrorString(e));
  for (afqmc_ctx* c : b->ctx) {
    afqmc_status s = check_status(c);
    if (s != AFQMC_OK) return fail(nullptr, s, c->err);
  }
  return AFQMC_OK;
}

void afqmc_batch_destroy(afqmc_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  for (auto& kv : b->execs) cudaGraphExecDestroy(kv.second);
  for (cudaEvent_t ev : b->ready) cudaEventDestroy(ev);
  if (b->done) cudaEventDestroy(b->done);
  if (b->st) cudaStreamDestroy(b->st);
  delete b;
}

}  // extern "C"
