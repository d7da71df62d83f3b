// Continuous-batching solve server over the HOTRG plans.
//
// Requests (Ising beta, J, h, D_cut, n_steps, want_grad, precision) enter a
// FIFO queue.  A fixed number of slots, each a host worker thread with its own
// CUDA stream, take requests as soon as they are free: a request that arrives
// while others are on the GPU starts when a slot and enough device memory are
// available, and its kernels run concurrently with the other slots' (one
// slot's FP64 eigensolve overlaps another's tensor-core contractions).
//
// Admission by device memory: every live plan is charged its
// hotrg_plan_workspace_bytes against the budget.  Built plans stay in one pool
// shared by all slots (LRU); a slot takes an idle plan of its request's shape
// (re-bound to the slot's stream) or builds one, first freeing idle plans from
// the cold end of the pool and, if the plans in use still leave no room,
// waiting until a running request returns its plan.  A request that could
// never fit the budget is rejected with HOTRG_ENOMEM.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/hotrg.h"
#include <cuda_runtime.h>

namespace {

using Clock = std::chrono::steady_clock;

// Depth of the plans the server builds (requests of up to this many steps
// share them).
constexpr int kPlanSteps = 40;

// Grouped forward: at most kGroupMax requests of one shape per grouped launch,
// for D_cut up to kGroupMaxD.
constexpr int kGroupMax = 4;
constexpr int kGroupMaxD = 32;

struct PlanKey {
  int d_cut, n_steps, want_grad, precision, split_from_step;
  bool operator==(const PlanKey& o) const {
    return d_cut == o.d_cut && n_steps == o.n_steps && want_grad == o.want_grad &&
           precision == o.precision && split_from_step == o.split_from_step;
  }
};

struct PooledPlan {
  PlanKey key;
  hotrg_plan plan;
  size_t bytes;
  bool in_use;
};

struct Job {
  uint64_t ticket;
  hotrg_request req;
  double t_submit;
};

struct SlotGroup {
  PlanKey key;
  hotrg_group group;
  size_t bytes;
};

}  // namespace

struct hotrg_server_s {
  size_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job> queue;
  std::unordered_map<uint64_t, hotrg_result> results;
  std::vector<std::thread> workers;
  std::list<PooledPlan> pool;   // built plans of all slots, front = most recently used
  std::vector<cudaStream_t> streams;   // one per slot; owned by the server, destroyed after
                                       // every pooled plan (plans keep a stream handle)
  std::vector<std::vector<cudaStream_t>> gstreams;   // per slot: the streams of a grouped
                                                     // forward's plans
  int slots = 0;
  std::vector<int> busy;
  size_t bytes_in_use = 0, peak_bytes = 0;
  uint64_t next_ticket = 1, submitted = 0, completed = 0, failed = 0, created = 0, evicted = 0;
  uint64_t admission_waits = 0;   // requests that had to wait for device memory
  uint64_t grouped = 0, groups_run = 0;   // requests run in grouped forwards, and those forwards
  std::vector<std::vector<SlotGroup>> groups;   // per slot: grouped-forward buffers per shape
  int running = 0;
  bool stop = false;
  Clock::time_point t0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Called with the lock held: an idle pooled plan of this key, marked in use
// and moved to the warm end of the pool, or nullptr.
hotrg_plan take_idle(hotrg_server_s* s, const PlanKey& key) {
  for (auto it = s->pool.begin(); it != s->pool.end(); ++it) {
    if (!it->in_use && it->key == key) {
      it->in_use = true;
      s->pool.splice(s->pool.begin(), s->pool, it);
      return s->pool.front().plan;
    }
  }
  return nullptr;
}

// Called with the lock held: free the coldest idle plan; false if none is idle.
bool evict_one(hotrg_server_s* s, std::unique_lock<std::mutex>& lk) {
  for (auto it = s->pool.end(); it != s->pool.begin();) {
    --it;
    if (it->in_use) continue;
    PooledPlan pp = *it;
    s->pool.erase(it);
    s->bytes_in_use -= pp.bytes;
    s->evicted += 1;
    lk.unlock();
    hotrg_plan_destroy(pp.plan);
    lk.lock();
    return true;
  }
  return false;
}

void make_cfg(const hotrg_server_s* s, const hotrg_request& r, int nsteps, hotrg_config* cfg) {
  hotrg_config_default(cfg, 2, r.d_cut, nsteps);
  cfg->precision = r.precision;
  cfg->split_from_step = r.split_from_step > 0 ? r.split_from_step : 1;
  cfg->want_grad = r.want_grad ? 1 : 0;
  // forward-only requests take the randomized subspace eigensolver (the
  // backward's eigensolve adjoint needs all eigenpairs)
  cfg->eigh_mode = r.want_grad ? 0 : 1;
  cfg->eigh_power_iters = 2;
  cfg->eigh_warm_start = r.want_grad ? 0 : 1;
  // with several slots, the contraction GEMMs leave SMs to the other
  // requests' latency-bound eigensolver kernels
  cfg->gemm_sm_reserve = s->slots > 1 ? 16 : 0;
}

// Plans are built for kPlanSteps steps (or the request's depth if larger) and
// run the request's depth (hotrg_plan_set_steps, bit-identical to a plan of
// exactly that depth), so requests of different depths share plans; where
// such a plan does not fit the budget, one of the request's own depth is built.
int plan_steps_of(const hotrg_server_s* s, const hotrg_request& r) {
  int plan_steps = r.n_steps > kPlanSteps ? r.n_steps : kPlanSteps;
  hotrg_config cfg;
  make_cfg(s, r, plan_steps, &cfg);
  size_t bytes = 0;
  if (hotrg_plan_workspace_bytes(&cfg, &bytes) == HOTRG_OK && bytes > s->budget &&
      plan_steps != r.n_steps)
    plan_steps = r.n_steps;
  return plan_steps;
}

PlanKey key_of(const hotrg_server_s* s, const hotrg_request& r) {
  return PlanKey{r.d_cut, plan_steps_of(s, r), r.want_grad ? 1 : 0, r.precision,
                 r.split_from_step};
}

// Called with the lock held (may release it while it builds a plan): a plan of
// this request's key, taken from the pool or built within the budget.  With
// may_wait false it gives up (HOTRG_EBUSY-like: returns HOTRG_EPENDING) instead
// of waiting for a running request to return a plan.
hotrg_status acquire(hotrg_server_s* s, std::unique_lock<std::mutex>& lk, const hotrg_request& r,
                     cudaStream_t stream, bool may_wait, hotrg_plan* out) {
  *out = nullptr;
  const PlanKey key = key_of(s, r);
  hotrg_config cfg;
  make_cfg(s, r, key.n_steps, &cfg);
  size_t bytes = 0;
  hotrg_status st = hotrg_plan_workspace_bytes(&cfg, &bytes);
  if (st != HOTRG_OK) return st;
  hotrg_plan plan = take_idle(s, key);
  if (plan) {
    *out = plan;
    return HOTRG_OK;
  }
  if (bytes > s->budget) return HOTRG_ENOMEM;
  bool waited = false;
  while (!plan && s->bytes_in_use + bytes > s->budget) {
    if (evict_one(s, lk)) {
      plan = take_idle(s, key);   // another slot may have returned one meanwhile
      continue;
    }
    if (!may_wait) return HOTRG_EPENDING;
    // every pooled plan is in use: wait for one to come back
    if (!waited) {
      s->admission_waits += 1;
      waited = true;
    }
    s->cv.wait(lk);
    plan = take_idle(s, key);
  }
  if (!plan) {
    s->bytes_in_use += bytes;
    s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
    lk.unlock();
    st = hotrg_plan_create(&cfg, stream, &plan);
    lk.lock();
    if (st == HOTRG_OK) {
      s->created += 1;
      s->pool.push_front(PooledPlan{key, plan, bytes, true});
    } else {
      s->bytes_in_use -= bytes;
      plan = nullptr;
      s->cv.notify_all();
      return st;
    }
  }
  *out = plan;
  return HOTRG_OK;
}

// Requests that go into a grouped forward: forward only, split precision, at
// most kGroupMaxD (one free-leg chunk per step; at larger D_cut one request's
// stage-2 GEMM already fills the GPU).
bool groupable(const hotrg_request& r) {
  return !r.want_grad && r.precision != HOTRG_FP64 && r.d_cut <= kGroupMaxD &&
         r.n_steps <= kPlanSteps;
}

// Called with the lock held: this slot's group for a key (built on first use,
// charged to the budget), or nullptr if it would not fit.
hotrg_group slot_group(hotrg_server_s* s, std::unique_lock<std::mutex>& lk, int slot,
                       const hotrg_request& r, const PlanKey& key, cudaStream_t stream) {
  for (auto& e : s->groups[slot])
    if (e.key == key) return e.group;
  hotrg_config cfg;
  make_cfg(s, r, key.n_steps, &cfg);
  size_t bytes = 0;
  if (hotrg_group_workspace_bytes(&cfg, kGroupMax, &bytes) != HOTRG_OK) return nullptr;
  if (s->bytes_in_use + bytes > s->budget) return nullptr;
  s->bytes_in_use += bytes;
  s->peak_bytes = std::max(s->peak_bytes, s->bytes_in_use);
  lk.unlock();
  hotrg_group g = nullptr;
  const hotrg_status st = hotrg_group_create(&cfg, kGroupMax, stream, &g);
  lk.lock();
  if (st != HOTRG_OK) {
    s->bytes_in_use -= bytes;
    return nullptr;
  }
  s->groups[slot].push_back(SlotGroup{key, g, bytes});
  return g;
}

void worker(hotrg_server_s* s, int slot) {
  cudaSetDevice(s->device);
  cudaStream_t stream = s->streams[slot];
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (s->stop && s->queue.empty()) break;
    if (s->queue.empty()) {
      s->cv.wait(lk);
      continue;
    }
    std::vector<Job> jobs{s->queue.front()};
    s->queue.pop_front();
    const PlanKey key0 = key_of(s, jobs[0].req);
    // Group only under backlog, when every other slot is busy: on one stream the
    // lockstep runs the plans' eigensolves one after another, while idle slots
    // would overlap them (measured at D_cut = 16-32: a group of four on one
    // stream 1.00-1.01x four solo solves, four concurrent streams 3.2-3.6x).
    int others_busy = 0;
    for (int i = 0; i < s->slots; ++i)
      if (i != slot && s->busy[i]) ++others_busy;
    if (groupable(jobs[0].req) && others_busy == s->slots - 1) {
      // the grouped launch: queued requests of the same shape join this one
      for (auto it = s->queue.begin(); it != s->queue.end() && (int)jobs.size() < kGroupMax;) {
        if (groupable(it->req) && key_of(s, it->req) == key0) {
          jobs.push_back(*it);
          it = s->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    s->busy[slot] = 1;
    s->running += (int)jobs.size();
    std::vector<hotrg_plan> plans(jobs.size(), nullptr);
    std::vector<hotrg_status> sts(jobs.size(), HOTRG_OK);
    sts[0] = acquire(s, lk, jobs[0].req, stream, true, &plans[0]);
    for (size_t i = 1; i < jobs.size(); ++i) {
      sts[i] = acquire(s, lk, jobs[i].req, stream, false, &plans[i]);
      if (sts[i] == HOTRG_EPENDING) {
        // no room for another plan now: the rest go back to the queue
        for (size_t j = jobs.size(); j-- > i;) s->queue.push_front(jobs[j]);
        s->running -= (int)(jobs.size() - i);
        jobs.resize(i);
        plans.resize(i);
        sts.resize(i);
        s->cv.notify_all();
        break;
      }
    }
    std::vector<int> ok;
    for (size_t i = 0; i < jobs.size(); ++i)
      if (sts[i] == HOTRG_OK) ok.push_back((int)i);
    hotrg_group group = nullptr;
    if (ok.size() > 1) group = slot_group(s, lk, slot, jobs[ok[0]].req, key0, stream);
    const double t_start = s->now();
    if (group && ok.size() > 1) {
      s->grouped += ok.size();
      s->groups_run += 1;
    }
    lk.unlock();
    const bool grouped_run = group && ok.size() > 1;
    for (size_t q = 0; q < ok.size(); ++q) {
      const int i = ok[q];
      // a grouped forward's plans run on streams of their own (their eigensolves
      // overlap); the grouped contractions run on the slot's stream
      sts[i] = hotrg_plan_set_stream(plans[i], grouped_run ? s->gstreams[slot][q] : stream);
      if (sts[i] == HOTRG_OK) sts[i] = hotrg_plan_set_steps(plans[i], jobs[i].req.n_steps);
    }
    std::vector<hotrg_result> res(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) {
      memset(&res[i], 0, sizeof(hotrg_result));
      res[i].ticket = jobs[i].ticket;
      res[i].t_submit = jobs[i].t_submit;
      res[i].slot = slot;
      res[i].t_start = t_start;
    }
    if (group && ok.size() > 1) {
      std::vector<hotrg_plan> gp;
      std::vector<double> b, J, h, lnz(ok.size(), 0.0);
      for (int i : ok) {
        gp.push_back(plans[i]);
        b.push_back(jobs[i].req.beta);
        J.push_back(jobs[i].req.J);
        h.push_back(jobs[i].req.h);
      }
      hotrg_status gs = HOTRG_OK;
      for (int i : ok)
        if (sts[i] != HOTRG_OK) gs = sts[i];
      if (gs == HOTRG_OK)
        gs = hotrg_forward_group_ising(group, gp.data(), (int)gp.size(), b.data(), J.data(),
                                       h.data(), lnz.data());
      for (size_t q = 0; q < ok.size(); ++q) {
        sts[ok[q]] = gs;
        res[ok[q]].lnz_per_site = lnz[q];
      }
    } else {
      for (int i : ok) {
        if (sts[i] != HOTRG_OK) continue;
        const hotrg_request& r = jobs[i].req;
        sts[i] = hotrg_forward_ising(plans[i], r.beta, r.J, r.h, &res[i].lnz_per_site, nullptr,
                                     nullptr);
        if (sts[i] == HOTRG_OK && r.want_grad)
          sts[i] = hotrg_backward(plans[i], nullptr, &res[i].dlnz_dbeta);
      }
    }
    lk.lock();
    for (size_t i = 0; i < jobs.size(); ++i) {
      if (plans[i])
        for (auto& pp : s->pool)
          if (pp.plan == plans[i]) pp.in_use = false;
      res[i].status = sts[i];
      res[i].t_finish = s->now();
      s->results[jobs[i].ticket] = res[i];
      s->completed += 1;
      if (sts[i] != HOTRG_OK) s->failed += 1;
    }
    s->busy[slot] = 0;
    s->running -= (int)jobs.size();
    s->cv.notify_all();
  }
  lk.unlock();
  cudaStreamSynchronize(stream);
  for (cudaStream_t g : s->gstreams[slot]) cudaStreamSynchronize(g);
}

}  // namespace

extern "C" {

hotrg_status hotrg_server_create(size_t hbm_budget_bytes, int max_slots, hotrg_server* out) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return HOTRG_EINVAL;
  *out = nullptr;
  hotrg_server_s* s = new hotrg_server_s();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    return HOTRG_ECUDA;
  }
  s->budget = hbm_budget_bytes;
  s->t0 = Clock::now();
  s->slots = max_slots;
  s->busy.assign(max_slots, 0);
  s->groups.assign(max_slots, {});
  s->streams.assign(max_slots, nullptr);
  s->gstreams.assign(max_slots, std::vector<cudaStream_t>(kGroupMax, nullptr));
  bool ok = true;
  for (int i = 0; i < max_slots && ok; ++i) {
    ok = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) == cudaSuccess;
    for (int j = 0; j < kGroupMax && ok; ++j)
      ok = cudaStreamCreateWithFlags(&s->gstreams[i][j], cudaStreamNonBlocking) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    for (int i = 0; i < max_slots; ++i) {
      if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
      for (cudaStream_t g : s->gstreams[i])
        if (g) cudaStreamDestroy(g);
    }
    delete s;
    return HOTRG_ECUDA;
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker, s, i);
  *out = s;
  return HOTRG_OK;
}

hotrg_status hotrg_server_submit(hotrg_server s, const hotrg_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return HOTRG_EINVAL;
  if (r->d_cut < 1 || r->n_steps < 1 || r->n_steps > 200 || r->precision < HOTRG_FP64 ||
      r->precision > HOTRG_BF16X6 || !(r->beta * r->J >= 0))
    return HOTRG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return HOTRG_ESTATE;
  Job j{s->next_ticket++, *r, s->now()};
  s->queue.push_back(j);
  s->submitted += 1;
  *ticket = j.ticket;
  s->cv.notify_all();
  return HOTRG_OK;
}

hotrg_status hotrg_server_poll(hotrg_server s, uint64_t ticket, hotrg_result* out) {
  if (!s || !out) return HOTRG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return ticket < s->next_ticket ? HOTRG_EPENDING : HOTRG_EINVAL;
  *out = it->second;
  return HOTRG_OK;
}

hotrg_status hotrg_server_wait(hotrg_server s, uint64_t ticket, hotrg_result* out) {
  if (!s || !out) return HOTRG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket >= s->next_ticket) return HOTRG_EINVAL;
  s->cv.wait(lk, [&] { return s->results.count(ticket) > 0; });
  *out = s->results[ticket];
  return HOTRG_OK;
}

hotrg_status hotrg_server_drain(hotrg_server s) {
  if (!s) return HOTRG_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait(lk, [&] { return s->queue.empty() && s->running == 0; });
  return HOTRG_OK;
}

hotrg_status hotrg_server_get_stats(hotrg_server s, hotrg_server_stats* o) {
  if (!s || !o) return HOTRG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(o, 0, sizeof(*o));
  o->submitted = s->submitted;
  o->completed = s->completed;
  o->failed = s->failed;
  o->bytes_in_use = s->bytes_in_use;
  o->peak_bytes = s->peak_bytes;
  o->plans_created = s->created;
  o->plans_evicted = s->evicted;
  o->admission_waits = s->admission_waits;
  o->grouped = s->grouped;
  o->groups = s->groups_run;
  o->queue_depth = (int)s->queue.size();
  o->busy_slots = s->running;
  return HOTRG_OK;
}

void hotrg_server_destroy(hotrg_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  for (auto& t : s->workers) t.join();
  // plans first (each waits for its stream), then the streams they were bound to
  for (auto& pp : s->pool) hotrg_plan_destroy(pp.plan);
  s->pool.clear();
  for (auto& v : s->groups)
    for (auto& e : v) hotrg_group_destroy(e.group);
  s->groups.clear();
  for (cudaStream_t st : s->streams)
    if (st) cudaStreamDestroy(st);
  for (auto& v : s->gstreams)
    for (cudaStream_t st : v)
      if (st) cudaStreamDestroy(st);
  delete s;
}

}  // extern "C"
