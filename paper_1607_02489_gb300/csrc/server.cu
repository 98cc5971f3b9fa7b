// Request server (include/emin_amg.h, amg_server_*): continuous batching of
// flexible GMRES solves on one device.
//
// A request is one solve of nrhs right-hand sides on a resident hierarchy.  It
// runs in a slot: a V-cycle clone of its hierarchy (shared matrices, own
// vectors and CUDA graphs), an FGMRES workspace for K = nrhs rounded up to a
// power of two, device copies of b and x, and a stream.  The server advances
// every running request one chunk of device work at a time (an Arnoldi step, a
// cycle end), polling an event per slot, so requests are admitted and retired
// between the steps of the others and their kernels overlap on the device.  A
// request's kernels, K and workspace are those of a blocking solve of the same
// right-hand sides, and every reduction has a fixed order, so its result is the
// same bits whether it runs alone or among others.
//
// Admission is by slots and memory: idle slots of the same (hierarchy, K) are
// reused (their graphs are already captured); a new slot is created while the
// running count is below max_active and its bytes fit the budget, after idle
// slots of other shapes have been released, least recently used first.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <memory>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "hierarchy.hpp"

using namespace emin;

namespace {

thread_local std::string g_server_error;

amg_status sfail(amg_status st, const std::string& msg) {
  g_server_error = msg;
  return st;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Slot {
  amg_hierarchy* h = nullptr;
  int K = 0;
  std::unique_ptr<VCycleIface> vc;
  Krylov ws;
  double* dev_b = nullptr;
  double* dev_x = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  cudaEvent_t wait = nullptr;  // the event the next step of the task waits for (the task's own, or ev)
  size_t bytes = 0;
  std::vector<long long> members;  // requests of the running cohort, empty when idle
  std::unique_ptr<SolveTask> task;
  bool busy() const { return !members.empty(); }
  unsigned long long last_used = 0;

  ~Slot() {
    if (s) cudaStreamSynchronize(s);
    task.reset();
    ws.release();
    vc.reset();
    if (dev_b) cudaFree(dev_b);
    if (dev_x) cudaFree(dev_x);
    if (ev) cudaEventDestroy(ev);
    if (s) cudaStreamDestroy(s);
  }
};

struct Request {
  amg_hierarchy* h = nullptr;
  int nrhs = 0;
  double rtol = 0.0;
  const double* bh = nullptr;
  double* xh = nullptr;
  int state = 0;  // 0 queued, 1 running, 2 done
  int col0 = 0;   // first column of the request in its cohort
  amg_status status = AMG_OK;
  std::vector<int> iters;
  std::vector<double> relres;
  double t_submit = 0.0, t_start = 0.0, t_done = 0.0;
};

size_t slot_bytes(const amg_hierarchy* h, int K, int restart) {
  const bool f32 = h->prm.vcycle_fp32 != 0;
  return h->vc()->clone_bytes(K) + Krylov::bytes_for(h->N, K, restart, f32) + 2 * sizeof(double) * (size_t)h->N * K;
}

}  // namespace

struct amg_server {
  amg_server_params prm{};
  size_t budget = 0;
  size_t bytes = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::deque<long long> queue;
  std::unordered_map<long long, Request> reqs;
  std::deque<long long> completed;  // finished, not yet reported by progress()
  long long next_id = 1;
  unsigned long long tick = 0;
  long long task_launches = 0;      // kernels launched by the solve tasks outside the graphs
  long long retired_vc_launches = 0;  // graph kernels of slots already released
  long long slots_created = 0, slots_released = 0, errors = 0, cohorts = 0;
  std::string last_error;

  int busy_slots() const {
    int n = 0;
    for (const auto& sl : slots) n += sl->busy();
    return n;
  }
  int running_requests() const {
    int n = 0;
    for (const auto& sl : slots) n += (int)sl->members.size();
    return n;
  }

  void release_slot(size_t i) {
    retired_vc_launches += slots[i]->vc ? slots[i]->vc->launches() : 0;
    bytes -= slots[i]->bytes;
    slots.erase(slots.begin() + (long)i);
    ++slots_released;
  }

  void fail_request(long long id, amg_status st, const std::string& err) {
    Request& r = reqs.at(id);
    r.state = 2;
    r.status = st;
    r.t_done = now_s();
    last_error = err;
    ++errors;
    completed.push_back(id);
  }

  // The cohort of a slot is done (st = AMG_OK) or failed (st < 0): report every member.
  void finish(Slot& sl, amg_status st, const std::string& err) {
    const double t = now_s();
    if (st >= 0 && sl.task) {
      int total = 0;
      for (long long id : sl.members) total += reqs.at(id).nrhs;
      std::vector<int> it(total);
      std::vector<double> rel(total);
      sl.task->result(it.data(), rel.data());
      for (long long id : sl.members) {
        Request& r = reqs.at(id);
        r.state = 2;
        r.t_done = t;
        r.status = AMG_OK;
        for (int k = 0; k < r.nrhs; ++k) {
          r.iters[k] = it[r.col0 + k];
          r.relres[k] = rel[r.col0 + k];
          const amg_status cs = sl.task->column_status(r.col0 + k);
          if (cs != AMG_OK && r.status != AMG_BREAKDOWN) r.status = cs;
        }
        completed.push_back(id);
      }
    } else {
      for (long long id : sl.members) fail_request(id, st < 0 ? st : AMG_ERR_CUDA, err);
    }
    sl.members.clear();
    sl.task.reset();
  }

  // Runs the next chunk of a slot's cohort; reports it when the solve finished.
  void step(Slot& sl) {
    try {
      const bool more = sl.task->advance();
      task_launches += sl.task->launches;
      sl.task->launches = 0;
      if (more) {
        sl.wait = sl.task->ready();
        if (!sl.wait) {
          EMIN_CUDA(cudaEventRecord(sl.ev, sl.s));
          sl.wait = sl.ev;
        }
      } else {
        finish(sl, AMG_OK, "");
      }
    } catch (const std::exception& e) {
      finish(sl, AMG_ERR_CUDA, e.what());
    }
  }

  Slot* make_slot(amg_hierarchy* h, int K) {
    std::unique_ptr<Slot> sl(new Slot());
    sl->h = h;
    sl->K = K;
    sl->bytes = slot_bytes(h, K, prm.restart);
    sl->vc.reset(h->vc()->clone(K));
    sl->ws.init(h->N, K, prm.restart, h->prm.vcycle_fp32 != 0);
    if (cudaMalloc(&sl->dev_b, sizeof(double) * (size_t)h->N * K) != cudaSuccess ||
        cudaMalloc(&sl->dev_x, sizeof(double) * (size_t)h->N * K) != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it for the next launch checks
      throw std::runtime_error("cudaMalloc for a request slot's b and x");
    }
    EMIN_CUDA(cudaStreamCreateWithFlags(&sl->s, cudaStreamNonBlocking));
    EMIN_CUDA(cudaEventCreateWithFlags(&sl->ev, cudaEventDisableTiming));
    bytes += sl->bytes;
    ++slots_created;
    slots.push_back(std::move(sl));
    return slots.back().get();
  }

  // Idle slot for (h, K), or a new one if the running count and the budget allow
  // it (after releasing idle slots of other shapes, least recently used first).
  Slot* find_slot(amg_hierarchy* h, int K, bool& no_room) {
    no_room = false;
    for (auto& sl : slots)
      if (!sl->busy() && sl->h == h && sl->K == K) return sl.get();
    if (busy_slots() >= prm.max_active) return nullptr;
    const size_t need = slot_bytes(h, K, prm.restart);
    while (bytes + need > budget) {
      size_t victim = slots.size();
      for (size_t i = 0; i < slots.size(); ++i)
        if (!slots[i]->busy() && (victim == slots.size() || slots[i]->last_used < slots[victim]->last_used))
          victim = i;
      if (victim == slots.size()) break;
      release_slot(victim);
    }
    if (bytes + need > budget) {
      no_room = true;
      return nullptr;
    }
    return make_slot(h, K);
  }

  // Starts queued requests, in submission order, while slots and memory allow.  A
  // request starts together with the later queued requests on the same hierarchy
  // (same rtol) whose columns fit beside its own within merge_k: one cohort, one
  // FGMRES over the stacked columns, one slot of K = columns rounded up.
  void admit() {
    std::vector<long long> q(queue.begin(), queue.end());
    std::vector<char> taken(q.size(), 0);
    // candidate heads: submission order, or smallest work (N x columns) first
    std::vector<size_t> heads(q.size());
    for (size_t a = 0; a < q.size(); ++a) heads[a] = a;
    if (prm.policy == 1)
      std::stable_sort(heads.begin(), heads.end(), [&](size_t x, size_t y) {
        const Request& rx = reqs.at(q[x]);
        const Request& ry = reqs.at(q[y]);
        return (double)rx.h->N * round_k(rx.nrhs) < (double)ry.h->N * round_k(ry.nrhs);
      });
    for (size_t a : heads) {
      if (taken[a]) continue;
      if (busy_slots() >= prm.max_active) break;
      const Request& r = reqs.at(q[a]);
      std::vector<size_t> cohort{a};
      int total = r.nrhs;
      if (prm.merge_k > 1)
        for (size_t b = 0; b < q.size(); ++b) {
          if (b == a || (b < a && prm.policy == 0)) continue;
          if (taken[b]) continue;
          const Request& o = reqs.at(q[b]);
          if (o.h == r.h && o.rtol == r.rtol && total + o.nrhs <= prm.merge_k) {
            cohort.push_back(b);
            total += o.nrhs;
          }
        }
      bool no_room = false;
      Slot* sl = nullptr;
      try {
        sl = find_slot(r.h, round_k(total), no_room);
      } catch (const std::exception& e) {
        // a slot that could not be built: the cohort fails, the server carries on
        const amg_status st =
            std::string(e.what()).find("cudaMalloc") != std::string::npos ? AMG_ERR_OOM : AMG_ERR_CUDA;
        for (size_t idx : cohort) {
          fail_request(q[idx], st, e.what());
          taken[idx] = 1;
        }
        continue;
      }
      if (!sl) {
        if (no_room && busy_slots() == 0 && slots.empty()) {
          // it can never fit: the whole budget is smaller than one slot
          fail_request(q[a], AMG_ERR_OOM, "request needs more device memory than the server's budget");
          taken[a] = 1;
        }
        continue;  // stays queued; a smaller request behind it may still fit
      }
      const double t = now_s();
      std::vector<SolveSegment> segs;
      int col0 = 0;
      sl->members.clear();
      for (size_t idx : cohort) {
        Request& m = reqs.at(q[idx]);
        m.state = 1;
        m.t_start = t;
        m.col0 = col0;
        SolveSegment g;
        g.b = sl->dev_b + (size_t)sl->h->N * col0;
        g.x = sl->dev_x + (size_t)sl->h->N * col0;
        g.b_host = m.bh;
        g.x_host = m.xh;
        g.ncols = m.nrhs;
        segs.push_back(g);
        col0 += m.nrhs;
        sl->members.push_back(q[idx]);
        taken[idx] = 1;
      }
      sl->last_used = ++tick;
      try {
        sl->task = make_solve_task(sl->h, sl->vc.get(), &sl->ws, segs, r.rtol, prm.restart, prm.maxit, sl->s);
      } catch (const std::exception& e) {
        finish(*sl, AMG_ERR_CUDA, e.what());
        continue;
      }
      ++cohorts;
      step(*sl);
    }
    std::deque<long long> rest;
    for (size_t i = 0; i < q.size(); ++i)
      if (!taken[i]) rest.push_back(q[i]);
    queue.swap(rest);
  }

  void poll() {
    for (auto& sl : slots) {
      if (!sl->busy()) continue;
      const cudaError_t e = cudaEventQuery(sl->wait);
      if (e == cudaErrorNotReady) continue;
      if (e != cudaSuccess) {
        finish(*sl, AMG_ERR_CUDA, std::string("cuda: ") + cudaGetErrorString(e));
        continue;
      }
      sl->last_used = ++tick;
      step(*sl);
    }
  }

  long long launches() const {
    long long n = task_launches + retired_vc_launches;
    for (const auto& sl : slots) n += sl->vc ? sl->vc->launches() : 0;
    return n;
  }

  ~amg_server() {
    for (auto& sl : slots)
      if (sl->s) cudaStreamSynchronize(sl->s);
    slots.clear();
  }
};

extern "C" {

void amg_server_params_default(amg_server_params* p) {
  if (!p) return;
  p->max_active = 16;
  p->device_bytes = 0;
  p->restart = 100;
  p->maxit = 500;
  p->merge_k = 8;
  p->policy = 0;
}

const char* amg_server_last_error(amg_server_handle sv) {
  return sv && !sv->last_error.empty() ? sv->last_error.c_str() : g_server_error.c_str();
}

amg_status amg_server_create(const amg_server_params* prm_in, amg_server_handle* out) {
  if (!out) return sfail(AMG_ERR_ARG, "null output handle");
  *out = nullptr;
  amg_server_params prm;
  if (prm_in)
    prm = *prm_in;
  else
    amg_server_params_default(&prm);
  if (prm.max_active < 1 || prm.max_active > 256) return sfail(AMG_ERR_ARG, "max_active must be in 1..256");
  if (prm.restart < 1 || prm.maxit < 1) return sfail(AMG_ERR_ARG, "restart and maxit must be positive");
  if (prm.merge_k < 0 || prm.merge_k > 32) return sfail(AMG_ERR_ARG, "merge_k must be in 0..32");
  if (prm.policy != 0 && prm.policy != 1) return sfail(AMG_ERR_ARG, "policy must be 0 or 1");
  std::unique_ptr<amg_server> sv(new amg_server());
  sv->prm = prm;
  if (prm.device_bytes > 0) {
    sv->budget = prm.device_bytes;
  } else {
    size_t free_b = 0, total_b = 0;
    const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return sfail(AMG_ERR_CUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
    sv->budget = free_b / 10 * 8;
  }
  *out = sv.release();
  return AMG_OK;
}

amg_status amg_server_submit(amg_server_handle sv, amg_handle h, const double* b_host, double* x_host, int nrhs,
                             double rtol, long long* ticket) {
  if (!sv || !h || !b_host || !x_host || !ticket) return sfail(AMG_ERR_ARG, "null argument");
  if (!h->vc()) return sfail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > 32) return sfail(AMG_ERR_ARG, "nrhs must be in 1..32");
  if (!(rtol > 0.0)) return sfail(AMG_ERR_ARG, "rtol must be positive");
  if ((long long)h->N * round_k(nrhs) >= (1LL << 31))
    return sfail(AMG_ERR_ARG, "N * nrhs (rounded up to a power of two) must stay below 2^31");
  Request r;
  r.h = h;
  r.nrhs = nrhs;
  r.rtol = rtol;
  r.bh = b_host;
  r.xh = x_host;
  r.iters.assign(nrhs, 0);
  r.relres.assign(nrhs, 0.0);
  r.t_submit = now_s();
  const long long id = sv->next_id++;
  sv->reqs.emplace(id, std::move(r));
  sv->queue.push_back(id);
  *ticket = id;
  return AMG_OK;
}

amg_status amg_server_reserve(amg_server_handle sv, amg_handle h, int nrhs, int count) {
  if (!sv || !h) return sfail(AMG_ERR_ARG, "null argument");
  if (!h->vc()) return sfail(AMG_ERR_ARG, "hierarchy was built with host_only");
  if (nrhs < 1 || round_k(nrhs) > 32 || count < 0) return sfail(AMG_ERR_ARG, "nrhs must be in 1..32, count >= 0");
  const int K = round_k(nrhs);
  int have = 0;
  for (const auto& sl : sv->slots) have += sl->h == h && sl->K == K;
  try {
    while (have < count) {
      if (sv->bytes + slot_bytes(h, K, sv->prm.restart) > sv->budget)
        return sfail(AMG_ERR_OOM, "reserve: the server's device budget is exhausted");
      Slot* sl = sv->make_slot(h, K);
      sl->last_used = ++sv->tick;
      EMIN_CUDA(sl->vc->prepare(K));
      ++have;
    }
  } catch (const std::exception& e) {
    const std::string m = e.what();
    return sfail(m.find("cudaMalloc") != std::string::npos ? AMG_ERR_OOM : AMG_ERR_CUDA, m);
  }
  return AMG_OK;
}

amg_status amg_server_progress(amg_server_handle sv, long long* done, int cap, int* n_done) {
  if (!sv || (cap > 0 && !done) || cap < 0) return sfail(AMG_ERR_ARG, "null argument or negative cap");
  sv->poll();
  sv->admit();
  int n = 0;
  while (n < cap && !sv->completed.empty()) {
    done[n++] = sv->completed.front();
    sv->completed.pop_front();
  }
  if (n_done) *n_done = n;
  return AMG_OK;
}

amg_status amg_server_result(amg_server_handle sv, long long ticket, int* state, int* iters, double* relres,
                             double* seconds, amg_status* status) {
  if (!sv) return sfail(AMG_ERR_ARG, "null server");
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(AMG_ERR_ARG, "unknown ticket (never issued or already collected)");
  const Request& r = it->second;
  if (state) *state = r.state;
  if (r.state != 2) return AMG_OK;
  if (iters) std::copy(r.iters.begin(), r.iters.end(), iters);
  if (relres) std::copy(r.relres.begin(), r.relres.end(), relres);
  if (seconds) {
    seconds[0] = r.t_start > 0.0 ? r.t_start - r.t_submit : 0.0;
    seconds[1] = r.t_done - r.t_submit;
  }
  if (status) *status = r.status;
  sv->reqs.erase(it);
  return AMG_OK;
}

amg_status amg_server_state(amg_server_handle sv, long long ticket, int* state) {
  if (!sv || !state) return sfail(AMG_ERR_ARG, "null argument");
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(AMG_ERR_ARG, "unknown ticket (never issued or already collected)");
  *state = it->second.state;
  return AMG_OK;
}

amg_status amg_server_get_stats(amg_server_handle sv, amg_server_stats* st) {
  if (!sv || !st) return sfail(AMG_ERR_ARG, "null argument");
  st->queued = (int)sv->queue.size();
  st->running = sv->running_requests();
  st->busy_slots = sv->busy_slots();
  st->cohorts = sv->cohorts;
  st->slots = (int)sv->slots.size();
  st->bytes_in_use = sv->bytes;
  st->budget = sv->budget;
  st->kernel_launches = sv->launches();
  st->slots_created = sv->slots_created;
  st->slots_released = sv->slots_released;
  st->errors = sv->errors;
  return AMG_OK;
}

void amg_server_destroy(amg_server_handle sv) { delete sv; }

}  // extern "C"
