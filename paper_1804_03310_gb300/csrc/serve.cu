// Serving loop: a native scheduler thread that admits independent runs by
// their HBM footprint, keeps their walkers on the device, and overlaps the
// blocks of all admitted runs on one GPU (continuous batching at block
// granularity). See the server section of include/afqmc.h.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/afqmc.h"
#include "ctx_internal.h"

namespace {

constexpr int kDepth = 2;         // blocks kept in flight per run
constexpr int kMaxBypass = 8;     // times the queue head may be overtaken

afqmc_status fail(afqmc_status s, const std::string& msg) {
  afqmc::set_global_error(msg);
  return s;
}

// Page-locked landing area of one block's read-back.
struct Readback {
  double e2[2];
  int status;
  int pad;
};

struct Run {
  int64_t id;
  afqmc_params p;
  std::vector<double> h1, L, Cu, Cd, ci;
  std::vector<int32_t> ou, od;
  int n_blocks, spb;
  size_t resident, setup;
  int bypassed = 0;
  afqmc_run_info info;
  std::vector<afqmc_block_result> blocks;
  // while admitted
  afqmc_ctx* ctx = nullptr;
  int slot = -1;            // index into the server's stream / event / pinned pools
  int enqueued = 0, inflight = 0, head = 0;
  double t_enq[kDepth] = {0, 0};
  long step_end[kDepth] = {0, 0};
  double last_end = 0;
};

}  // namespace

struct afqmc_server {
  afqmc_server_config cfg;
  size_t budget;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::thread thr;
  int64_t next_id = 0;
  std::map<int64_t, std::shared_ptr<Run>> runs;
  std::deque<std::shared_ptr<Run>> queue;
  // correlated-sampling groups: members in submission order; a group is
  // admitted whole once it has cs_size members, and is then closed
  std::map<int32_t, std::vector<std::shared_ptr<Run>>> groups;
  std::map<int32_t, bool> group_admitted;
  std::vector<std::shared_ptr<Run>> active;   // scheduler thread only
  std::vector<int> free_slots;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev;                // [slot][depth][start, end]
  Readback* pinned = nullptr;                 // [slot][depth]
  // accounting (under mu)
  size_t in_use = 0, peak = 0;
  int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, nblocks = 0;
  double walker_steps = 0;
  int max_active_seen = 0;
  std::vector<double> lat_ms;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  cudaEvent_t event(int slot, int d, int which) { return ev[(slot * kDepth + d) * 2 + which]; }
  Readback* rb(int slot, int d) { return pinned + slot * kDepth + d; }
};

namespace {

void finish(afqmc_server* S, Run& r, int state, afqmc_status st, const std::string& msg) {
  if (r.ctx) {
    cudaStreamSynchronize(S->streams[r.slot]);
    afqmc_destroy(r.ctx);
    r.ctx = nullptr;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (r.slot >= 0) {
    S->free_slots.push_back(r.slot);
    S->in_use -= r.resident;
    r.slot = -1;
  }
  r.info.state = state;
  r.info.status = st;
  r.info.t_done = S->now();
  if (!msg.empty()) {
    strncpy(r.info.message, msg.c_str(), sizeof(r.info.message) - 1);
    r.info.message[sizeof(r.info.message) - 1] = 0;
  }
  if (state == AFQMC_RUN_DONE) S->completed += 1; else S->failed += 1;
  S->cv.notify_all();
}

// Issue the run's next block on its stream: start event, the steps (graph
// replays), the read-back copies, end event.
afqmc_status enqueue_block(afqmc_server* S, Run& r) {
  const int d = (r.head + r.inflight) % kDepth;
  Readback* rb = S->rb(r.slot, d);
  cudaStream_t st = S->streams[r.slot];
  if (cudaEventRecord(S->event(r.slot, d, 0), st) != cudaSuccess) return AFQMC_E_CUDA;
  afqmc_status s = afqmc_propagate(r.ctx, r.spb);
  if (s != AFQMC_OK) return s;
  if (afqmc::ctx_enqueue_readback(r.ctx, rb->e2, &rb->status) != cudaSuccess) return AFQMC_E_CUDA;
  if (cudaEventRecord(S->event(r.slot, d, 1), st) != cudaSuccess) return AFQMC_E_CUDA;
  r.t_enq[d] = S->now();
  r.step_end[d] = afqmc::ctx_step(r.ctx);
  r.inflight += 1;
  r.enqueued += 1;
  return AFQMC_OK;
}

// Collect finished blocks of an admitted run; true if anything happened.
bool service(afqmc_server* S, Run& r) {
  bool progress = false;
  while (r.inflight > 0) {
    const int d = r.head;
    cudaError_t q = cudaEventQuery(S->event(r.slot, d, 1));
    if (q == cudaErrorNotReady) break;
    progress = true;
    if (q != cudaSuccess) {
      cudaGetLastError();
      finish(S, r, AFQMC_RUN_FAILED, AFQMC_E_CUDA, std::string("block: ") + cudaGetErrorString(q));
      return true;
    }
    const double t = S->now();
    Readback* rb = S->rb(r.slot, d);
    afqmc_block_result b;
    b.t_start = std::max(r.t_enq[d], r.last_end);
    b.t_end = t;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, S->event(r.slot, d, 0), S->event(r.slot, d, 1));
    b.device_ms = ms;
    b.e_mixed = rb->e2[0];
    b.weight_sum = rb->e2[1];
    b.step = r.step_end[d];
    const int status = rb->status;
    r.last_end = t;
    r.head = (r.head + 1) % kDepth;
    r.inflight -= 1;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r.blocks.push_back(b);
      r.info.blocks_done += 1;
      S->nblocks += 1;
      S->walker_steps += (double)r.p.n_walkers * r.spb;
      S->lat_ms.push_back(1e3 * (b.t_end - b.t_start));
      S->cv.notify_all();
    }
    if (status & 4) {
      finish(S, r, AFQMC_RUN_FAILED, AFQMC_E_TIMEOUT, "a tensor-core pipeline wait timed out");
      return true;
    }
    if (status & 2) {
      finish(S, r, AFQMC_RUN_FAILED, AFQMC_E_POPULATION,
             "population control found every walker weight zero");
      return true;
    }
  }
  if (r.info.blocks_done == r.n_blocks) {
    finish(S, r, AFQMC_RUN_DONE, AFQMC_OK, "");
    return true;
  }
  while (r.inflight < kDepth && r.enqueued < r.n_blocks) {
    afqmc_status s = enqueue_block(S, r);
    if (s != AFQMC_OK) {
      finish(S, r, AFQMC_RUN_FAILED, s, afqmc_last_error(r.ctx));
      return true;
    }
    progress = true;
  }
  return progress;
}

// The runs that admitting queued run r takes with it (under mu): r alone, or
// its whole correlated-sampling group; empty while the group is incomplete.
std::vector<std::shared_ptr<Run>> unit_of(afqmc_server* S, const std::shared_ptr<Run>& r) {
  if (r->p.cs_group == 0) return {r};
  const auto& m = S->groups[r->p.cs_group];
  if ((int)m.size() < r->p.cs_size) return {};
  return m;
}

bool unit_fits(afqmc_server* S, const std::vector<std::shared_ptr<Run>>& u) {
  if (u.empty() || S->free_slots.size() < u.size()) return false;
  size_t need = 0;
  for (const auto& r : u) need += r->resident + r->setup;
  return S->in_use + need <= S->budget;
}

// Pick the next runs to admit (under mu): the queue head's unit if it fits,
// else the first later unit that fits while the head has been overtaken
// fewer than kMaxBypass times. The picked runs leave the queue.
std::vector<std::shared_ptr<Run>> pick(afqmc_server* S) {
  if (S->queue.empty() || S->free_slots.empty()) return {};
  auto take = [&](const std::vector<std::shared_ptr<Run>>& u) {
    for (const auto& r : u) {
      auto it = std::find(S->queue.begin(), S->queue.end(), r);
      if (it != S->queue.end()) S->queue.erase(it);
    }
    if (u.front()->p.cs_group) S->group_admitted[u.front()->p.cs_group] = true;
    return u;
  };
  std::shared_ptr<Run> head = S->queue.front();
  std::vector<std::shared_ptr<Run>> u = unit_of(S, head);
  if (unit_fits(S, u)) return take(u);
  if (head->bypassed >= kMaxBypass) return {};
  for (auto it = S->queue.begin() + 1; it != S->queue.end(); ++it) {
    u = unit_of(S, *it);
    if (unit_fits(S, u)) {
      head->bypassed += 1;
      return take(u);
    }
  }
  return {};
}

bool admit_one(afqmc_server* S) {
  std::vector<std::shared_ptr<Run>> unit;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    unit = pick(S);
    if (unit.empty()) return false;
    for (auto& r : unit) {
      r->slot = S->free_slots.back();
      S->free_slots.pop_back();
      S->in_use += r->resident;
      S->admitted += 1;
      r->info.state = AFQMC_RUN_ACTIVE;
      r->info.t_admit = S->now();
    }
    size_t setup = 0;
    for (auto& r : unit) setup = std::max(setup, r->setup);
    S->peak = std::max(S->peak, S->in_use + setup);
  }
  for (auto& r : unit) {
    afqmc_ctx* ctx = nullptr;
    afqmc_status s = afqmc_create(&r->p, r->h1.data(), r->L.data(), r->Cu.data(),
                                  r->Cd.data(), r->ou.data(), r->od.data(), r->ci.data(),
                                  (void*)S->streams[r->slot], &ctx);
    // the host copies of the inputs are no longer needed
    std::vector<double>().swap(r->h1);
    std::vector<double>().swap(r->L);
    std::vector<double>().swap(r->Cu);
    std::vector<double>().swap(r->Cd);
    std::vector<double>().swap(r->ci);
    if (s != AFQMC_OK) {
      finish(S, *r, AFQMC_RUN_FAILED, s, afqmc_last_error(nullptr));
      continue;
    }
    r->ctx = ctx;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->active.push_back(r);
      S->max_active_seen = std::max(S->max_active_seen, (int)S->active.size());
    }
  }
  for (auto& r : unit)
    if (r->ctx) service(S, *r);
  return true;
}

void scheduler(afqmc_server* S) {
  cudaSetDevice(S->cfg.device);
  while (true) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (S->stop) break;
    }
    bool progress = false;
    std::vector<std::shared_ptr<Run>> act;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      act = S->active;
    }
    for (auto& r : act)
      if (r->ctx) progress |= service(S, *r);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->active.erase(std::remove_if(S->active.begin(), S->active.end(),
                                     [](const std::shared_ptr<Run>& r) { return !r->ctx; }),
                      S->active.end());
    }
    progress |= admit_one(S);
    if (!progress) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(100));
    }
  }
}

}  // namespace

extern "C" {

afqmc_status afqmc_server_create(const afqmc_server_config* cfg, afqmc_server** out) {
  if (!out) return fail(AFQMC_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(AFQMC_E_INVALID, "config is NULL");
  for (int i = 0; i < 4; ++i)
    if (cfg->reserved[i]) return fail(AFQMC_E_INVALID, "reserved fields must be zero");
  const int max_active = cfg->max_active == 0 ? 64 : cfg->max_active;
  if (max_active < 1 || max_active > 256) return fail(AFQMC_E_INVALID, "max_active must be in 1..256");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(AFQMC_E_CUDA, "no CUDA device");
  }
  if (cfg->device < 0 || cfg->device >= ndev) return fail(AFQMC_E_INVALID, "device out of range");
  cudaError_t e = cudaSetDevice(cfg->device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(AFQMC_E_CUDA, std::string("server: ") + cudaGetErrorString(e));
  }
  afqmc_server* S = new afqmc_server();
  S->cfg = *cfg;
  S->cfg.max_active = max_active;
  S->budget = cfg->hbm_budget ? cfg->hbm_budget : (size_t)(0.9 * (double)free_b);
  S->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < max_active && e == cudaSuccess; ++i) {
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) S->streams.push_back(st);
    for (int k = 0; k < 2 * kDepth && e == cudaSuccess; ++k) {
      cudaEvent_t v;
      e = cudaEventCreate(&v);
      if (e == cudaSuccess) S->ev.push_back(v);
    }
    S->free_slots.push_back(max_active - 1 - i);
  }
  if (e == cudaSuccess)
    e = cudaMallocHost((void**)&S->pinned, sizeof(Readback) * max_active * kDepth);
  if (e != cudaSuccess) {
    cudaGetLastError();
    afqmc_server_destroy(S);
    return fail(AFQMC_E_CUDA, std::string("server resources: ") + cudaGetErrorString(e));
  }
  memset(S->pinned, 0, sizeof(Readback) * max_active * kDepth);
  S->thr = std::thread(scheduler, S);
  *out = S;
  return AFQMC_OK;
}

afqmc_status afqmc_server_submit(afqmc_server* S, const afqmc_params* p, const double* h1,
                                 const double* L, const double* C_up, const double* C_dn,
                                 const int32_t* occ_up, const int32_t* occ_dn,
                                 const double* ci, int32_t n_blocks, int32_t steps_per_block,
                                 int64_t* run_id) {
  if (!S || !p || !h1 || !L || !C_up || !C_dn || !occ_up || !occ_dn || !ci || !run_id)
    return fail(AFQMC_E_INVALID, "null argument");
  if (n_blocks < 1 || steps_per_block < 1)
    return fail(AFQMC_E_INVALID, "n_blocks and steps_per_block must be >= 1");
  size_t resident = 0, setup = 0;
  afqmc_status s = afqmc_footprint(p, occ_up, occ_dn, &resident, &setup);
  if (s != AFQMC_OK) return s;
  auto r = std::make_shared<Run>();
  r->p = *p;
  const size_t M = p->M, MM = M * M;
  r->h1.assign(h1, h1 + MM);
  r->L.assign(L, L + (size_t)p->n_chol * MM);
  r->Cu.assign(C_up, C_up + MM);
  r->Cd.assign(C_dn, C_dn + MM);
  r->ci.assign(ci, ci + 2 * (size_t)p->n_det);
  r->ou.assign(occ_up, occ_up + (size_t)p->n_det * p->n_up);
  r->od.assign(occ_dn, occ_dn + (size_t)p->n_det * p->n_dn);
  if (r->ou.empty()) r->ou.push_back(0);
  if (r->od.empty()) r->od.push_back(0);
  r->n_blocks = n_blocks;
  r->spb = steps_per_block;
  r->resident = resident;
  r->setup = setup;
  memset(&r->info, 0, sizeof(r->info));
  r->info.state = AFQMC_RUN_QUEUED;
  r->info.status = AFQMC_OK;
  r->info.n_blocks = n_blocks;
  r->info.t_admit = -1;
  r->info.t_done = -1;
  r->info.footprint = resident + setup;
  std::lock_guard<std::mutex> lk(S->mu);
  if (p->cs_group != 0) {
    if (S->group_admitted.count(p->cs_group))
      return fail(AFQMC_E_INVALID, "correlated-sampling group already admitted");
    auto& m = S->groups[p->cs_group];
    if ((int)m.size() >= p->cs_size)
      return fail(AFQMC_E_INVALID, "correlated-sampling group is full");
    if (!m.empty()) {
      const Run& f = *m.front();
      const afqmc_params& q = f.p;
      if (q.seed != p->seed || q.run_id != p->run_id || q.n_chol != p->n_chol ||
          q.n_walkers != p->n_walkers || q.dtau != p->dtau || q.cs_size != p->cs_size ||
          q.ortho_every != p->ortho_every || q.measure_every != p->measure_every ||
          q.pc_every != p->pc_every || q.taylor_order != p->taylor_order ||
          f.n_blocks != n_blocks || f.spb != steps_per_block)
        return fail(AFQMC_E_INVALID,
                    "correlated-sampling group members must share seed, run_id, n_chol, "
                    "n_walkers, dtau, cadences, taylor_order, cs_size and the block plan");
    }
  }
  r->id = S->next_id++;
  r->info.t_submit = S->now();
  S->runs[r->id] = r;
  S->submitted += 1;
  if (resident + setup > S->budget) {
    r->info.state = AFQMC_RUN_FAILED;
    r->info.status = AFQMC_E_OOM;
    r->info.t_done = r->info.t_submit;
    strncpy(r->info.message, "footprint exceeds the server's HBM budget",
            sizeof(r->info.message) - 1);
    S->failed += 1;
    if (p->cs_group != 0) {   // the group can never be admitted whole: fail it
      S->group_admitted[p->cs_group] = true;
      for (auto& m : S->groups[p->cs_group]) {
        auto it = std::find(S->queue.begin(), S->queue.end(), m);
        if (it != S->queue.end()) S->queue.erase(it);
        m->info.state = AFQMC_RUN_FAILED;
        m->info.status = AFQMC_E_OOM;
        m->info.t_done = S->now();
        strncpy(m->info.message, "a member of its correlated-sampling group exceeds the budget",
                sizeof(m->info.message) - 1);
        S->failed += 1;
      }
    }
  } else {
    S->queue.push_back(r);
    if (p->cs_group != 0) S->groups[p->cs_group].push_back(r);
  }
  *run_id = r->id;
  S->cv.notify_all();
  return AFQMC_OK;
}

afqmc_status afqmc_server_poll(afqmc_server* S, int64_t run_id, afqmc_run_info* info,
                               afqmc_block_result* blocks, int32_t max_blocks) {
  if (!S) return fail(AFQMC_E_INVALID, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->runs.find(run_id);
  if (it == S->runs.end()) return fail(AFQMC_E_INVALID, "unknown run");
  const Run& r = *it->second;
  if (info) *info = r.info;
  if (blocks && max_blocks > 0) {
    const size_t n = std::min<size_t>(max_blocks, r.blocks.size());
    std::copy(r.blocks.begin(), r.blocks.begin() + n, blocks);
  }
  return AFQMC_OK;
}

afqmc_status afqmc_server_wait(afqmc_server* S, int64_t run_id, double timeout_s) {
  if (!S) return fail(AFQMC_E_INVALID, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  if (run_id >= 0 && !S->runs.count(run_id)) return fail(AFQMC_E_INVALID, "unknown run");
  auto finished = [&]() {
    if (run_id >= 0) {
      const int st = S->runs[run_id]->info.state;
      return st == AFQMC_RUN_DONE || st == AFQMC_RUN_FAILED;
    }
    return S->completed + S->failed == S->submitted;
  };
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s);
  while (!finished()) {
    if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && !finished())
      return fail(AFQMC_E_TIMEOUT, "server wait timed out");
  }
  return AFQMC_OK;
}

afqmc_status afqmc_server_stats_get(afqmc_server* S, afqmc_server_stats* out) {
  if (!S || !out) return fail(AFQMC_E_INVALID, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = S->submitted;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->failed = S->failed;
  out->blocks = S->nblocks;
  out->walker_steps = S->walker_steps;
  out->elapsed_s = S->now();
  out->active = (int32_t)S->active.size();
  out->queued = (int32_t)S->queue.size();
  out->max_active_seen = S->max_active_seen;
  out->bytes_in_use = S->in_use;
  out->peak_bytes = S->peak;
  out->p50_ms = out->p99_ms = NAN;
  if (!S->lat_ms.empty()) {
    std::vector<double> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) {   // nearest-rank percentile
      size_t k = (size_t)ceil(f * v.size());
      return v[k ? k - 1 : 0];
    };
    out->p50_ms = q(0.50);
    out->p99_ms = q(0.99);
  }
  return AFQMC_OK;
}

void afqmc_server_destroy(afqmc_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->thr.joinable()) S->thr.join();
  for (auto& r : S->active) {
    if (r->ctx) {
      cudaStreamSynchronize(S->streams[r->slot]);
      afqmc_destroy(r->ctx);
      r->ctx = nullptr;
    }
  }
  for (cudaEvent_t v : S->ev) cudaEventDestroy(v);
  for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
  if (S->pinned) cudaFreeHost(S->pinned);
  delete S;
}

}  // extern "C"
