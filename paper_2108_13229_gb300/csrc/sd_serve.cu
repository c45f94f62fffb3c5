// sd_serve.cu -- many independent instances at once: sd_solve_batch (a
// fixed set of handles advanced together: compatible handles in lockstep
// groups that share every launch, the rest each on its own stream) and
// the continuous-batching server (requests admitted FIFO as running slots
// and HBM budget free up, each run keeping its state on the device for all
// its time steps).  Host code on the public C ABI and the lockstep driver;
// instances never share device memory, so every result equals the instance
// run alone.
#include "../../include/sd.h"
#include "sd_internal.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

namespace sdk {
thread_local int t_conc = 0;  // see sd_internal.cuh
}  // namespace sdk

namespace {

using clk = std::chrono::steady_clock;

// DoF of one lockstep group at most.  Measured on GB300 with 10-step runs of
// 64 log-normal instances: 512^2 grids ran fastest one per stream (one 512^2
// grid already fills the GPU, and a group waits for its slowest member),
// 256^2 grids best about eight to a group, 64^2-128^2 grids all in one group
// (1.8-2.4x the one-stream-per-instance rate); 2M DoF per group gives that.
const int64_t kLockstepDof = 2ll << 20;

double ms_between(clk::time_point a, clk::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Job {
  uint64_t id = 0;
  sd_request req;
  std::vector<double> K;
  int64_t est = 0;
  int status = SD_PENDING;
  sd_result res;
  std::vector<double> x;
  clk::time_point t_submit, t_start, t_end;
  // lockstep serving: the run's handle and progress between ticks
  sd_handle* h = nullptr;
  int done = 0, iters = 0;
  int first = SD_OK;  // first non-OK status of a step that still advanced the state
  double maxrel = 0.0;
  int geometry = SD_GEO_SQUARE;  // the server's sd_options.geometry
};

// Lockstep serving: the running requests of one size class (grid, mu, dt)
// advance one time step per tick, each tick's lockstep groups sharing every
// launch; requests join at the next tick after admission and leave when
// their steps are done.
struct SizeClass {
  std::vector<Job*> incoming;  // admitted, handle not yet created
  std::vector<Job*> running;
  std::thread th;
};

}  // namespace

struct sd_server {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<uint64_t> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  int64_t budget = 0, used = 0;
  int max_running = 1, running = 0;
  bool stop = false;
  sd_options opt;
  uint64_t next_id = 1;
  int device = 0;
  int flags = 0;
  bool auto_depth = false;  // created without options: multigrid depth per request
  std::vector<std::thread> workers;
  std::map<std::tuple<int, double, double, int>, std::unique_ptr<SizeClass>> classes;  // (n, mu, dt, depth)
};

namespace {

// A server created without options picks the multigrid depth per request
// from its length: the dense inverse of a 16 x 16 coarsest grid costs about
// 10 ms of setup and some 1,600 dependent launches (which queue behind the
// other runs' work), and saves 0.2-0.3 ms per step, so runs shorter than
// kShortRun steps coarsen to 4 x 4 instead.
const int kShortRun = 40;
// device memory reserved per run beyond its arena (setup temporaries, stream resources)
const int64_t kRunSlack = 4ll << 20;
sd_options run_options(const sd_server* S, const sd_request& req) {
  sd_options o = S->opt;
  o.stream = nullptr;  // each run gets its own stream, so runs overlap on the device
  if (S->auto_depth) o.coarsest = req.nsteps < kShortRun ? 4 : 16;
  return o;
}
sd_options job_options(const sd_server* S, const Job* J) { return run_options(S, J->req); }

void run_job(sd_server* S, Job* J) {
  sd_options o = job_options(S, J);
  sd_handle* h = nullptr;
  int rc = sd_create(&J->req.grid, J->req.mu, J->K.data(), J->req.alpha_bj, J->req.dt, &o, &h);
  std::memset(&J->res, 0, sizeof(J->res));
  J->res.dof = sd_dof_count_geometry(J->req.grid.nx, J->geometry);
  if (rc == SD_OK) {
    std::vector<sd_step_info> info(J->req.nsteps > 0 ? J->req.nsteps : 1);
    rc = sd_step(h, J->req.nsteps, info.data());
    // a CUDA or allocation error ends sd_step early: the handle's step count
    // says how many steps (and info entries) were completed
    int64_t done = 0;
    sd_get_state(h, nullptr, &done, nullptr, nullptr);
    int it = 0;
    double mr = 0.0;
    for (int64_t k = 0; k < done; ++k) {
      it += info[k].iters;
      if (info[k].relres > mr) mr = info[k].relres;
    }
    J->res.steps_done = (int32_t)done;
    J->res.total_iters = it;
    J->res.max_relres = mr;
    if (J->req.keep_fields) {
      J->x.resize((size_t)sd_dof_count_geometry(J->req.grid.nx, J->geometry));
      int r2 = sd_get_state(h, nullptr, nullptr, J->x.data(), nullptr);
      if (rc == SD_OK) rc = r2;
    }
  }
  if (h) sd_destroy(h);
  J->status = rc;
  J->res.status = rc;
}

// grids below this many DoF run in lockstep size classes in the lockstep mode
// (one larger grid already fills the GPU: those keep a worker of their own)
const int64_t kServeLockstepDof = 1ll << 20;

void finish_job(sd_server* S, Job* J) {
  std::lock_guard<std::mutex> lk(S->mu);
  J->t_end = clk::now();
  J->res.queue_ms = ms_between(J->t_submit, J->t_start);
  J->res.run_ms = ms_between(J->t_start, J->t_end);
  J->res.latency_ms = ms_between(J->t_submit, J->t_end);
  S->used -= J->est;
  S->running -= 1;
}

// Close a lockstep-served run: copy its state out if asked (as the one-worker
// path does, also after steps that ended in SD_E_NOCONV or SD_E_NUMERIC),
// release the handle.
void close_job(Job* J, int rc) {
  J->res.dof = sd_dof_count_geometry(J->req.grid.nx, J->geometry);
  J->res.steps_done = J->done;
  J->res.total_iters = J->iters;
  J->res.max_relres = J->maxrel;
  if (J->h && J->req.keep_fields && (rc == SD_OK || rc == SD_E_NOCONV || rc == SD_E_NUMERIC)) {
    J->x.resize((size_t)sd_dof_count_geometry(J->req.grid.nx, J->geometry));
    const int r2 = sd_get_state(J->h, nullptr, nullptr, J->x.data(), nullptr);
    if (rc == SD_OK) rc = r2;
  }
  if (J->h) sd_destroy(J->h);
  J->h = nullptr;
  J->status = rc;
  J->res.status = rc;
}

void class_loop(sd_server* S, SizeClass* C) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<Job*> fresh;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] { return S->stop || !C->incoming.empty() || !C->running.empty(); });
      if (S->stop) return;
      fresh.swap(C->incoming);
    }
    for (Job* J : fresh) {  // joins at this tick
      sd_options o = job_options(S, J);
      const int rc = sd_create(&J->req.grid, J->req.mu, J->K.data(), J->req.alpha_bj, J->req.dt, &o, &J->h);
      if (rc != SD_OK || J->req.nsteps == 0) {
        close_job(J, rc);
        finish_job(S, J);
        S->cv.notify_all();
      } else {
        C->running.push_back(J);
      }
    }
    if (C->running.empty()) continue;
    // one tick: every running request advances one step, in lockstep groups
    std::vector<sd_handle*> hs;
    for (Job* J : C->running) hs.push_back(J->h);
    std::vector<sd_step_info> info(hs.size());
    std::vector<int> rcs(hs.size(), SD_OK);
    const int64_t dof = sd_dof_count_geometry(C->running[0]->req.grid.nx, S->opt.geometry);
    const size_t cap = (size_t)std::max<int64_t>(1, kLockstepDof / dof);
    for (size_t a = 0; a < hs.size(); a += cap) {
      const size_t b = std::min(hs.size(), a + cap);
      std::vector<sd_step_info*> ip;
      for (size_t q = a; q < b; ++q) ip.push_back(&info[q]);
      const int rc = (b - a == 1) ? sd_step(hs[a], 1, ip[0]) : sdk::step_lockstep(&hs[a], (int)(b - a), 1, ip.data());
      for (size_t q = a; q < b; ++q) rcs[q] = (b - a == 1) ? rc : info[q].status;
      if (rc == SD_E_CUDA || rc == SD_E_NOMEM || rc == SD_E_STATE || rc == SD_E_INVAL)
        for (size_t q = a; q < b; ++q) rcs[q] = rc;
    }
    std::vector<Job*> keep;
    for (size_t q = 0; q < hs.size(); ++q) {
      Job* J = C->running[q];
      // a step that ended in SD_E_NOCONV or SD_E_NUMERIC still advanced the
      // state and the run goes on (as in sd_step); a CUDA, allocation or
      // state error returned before the step was taken and ends the run
      const bool advanced = rcs[q] == SD_OK || rcs[q] == SD_E_NOCONV || rcs[q] == SD_E_NUMERIC;
      if (advanced) {
        J->done += 1;
        J->iters += info[q].iters;
        if (info[q].relres > J->maxrel) J->maxrel = info[q].relres;
        if (rcs[q] != SD_OK && J->first == SD_OK) J->first = rcs[q];
      }
      if (!advanced || J->done >= J->req.nsteps) {
        close_job(J, advanced ? J->first : rcs[q]);
        finish_job(S, J);
        S->cv.notify_all();
      } else {
        keep.push_back(J);
      }
    }
    C->running.swap(keep);
  }
}

void worker_loop(sd_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Job* J = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait(lk, [&] {
        if (S->stop) return true;
        if (S->queue.empty() || S->running >= S->max_running) return false;
        Job* head = S->jobs[S->queue.front()].get();
        return S->used + head->est <= S->budget;
      });
      if (S->stop) return;
      J = S->jobs[S->queue.front()].get();
      S->queue.pop_front();
      S->used += J->est;
      S->running += 1;
      J->t_start = clk::now();
      const int n = J->req.grid.nx;
      if ((S->flags & SD_SERVER_LOCKSTEP) && sd_dof_count_geometry(n, S->opt.geometry) < kServeLockstepDof) {
        // hand the run to its size class and go back for the next request
        auto key = std::make_tuple(n, J->req.mu, J->req.dt, job_options(S, J).coarsest);
        auto it = S->classes.find(key);
        if (it == S->classes.end()) {
          std::unique_ptr<SizeClass> c(new SizeClass());
          SizeClass* cp = c.get();
          it = S->classes.emplace(key, std::move(c)).first;
          cp->th = std::thread(class_loop, S, cp);
        }
        it->second->incoming.push_back(J);
        S->cv.notify_all();
        continue;
      }
    }
    run_job(S, J);
    finish_job(S, J);
    S->cv.notify_all();
  }
}

}  // namespace

extern "C" {

int sd_solve_batch_ex(sd_handle* const* hs, int32_t count, const int32_t* nsteps, sd_step_info* const* infos,
                      int32_t max_threads, int32_t flags) {
  if (count < 0 || (count > 0 && (!hs || !nsteps))) return SD_E_INVAL;
  if (count == 0) return SD_OK;
  for (int k = 0; k < count; ++k)
    if (!hs[k] || nsteps[k] < 0) return SD_E_INVAL;
  {  // a handle listed twice would be stepped twice (or by two groups at once)
    std::vector<sd_handle*> order(hs, hs + count);
    std::sort(order.begin(), order.end());
    if (std::adjacent_find(order.begin(), order.end()) != order.end()) return SD_E_INVAL;
  }
  // work items: lockstep groups of compatible handles (same nsteps), or
  // single handles
  std::vector<std::vector<int>> items;
  for (int k = 0; k < count; ++k) {
    bool placed = false;
    if (flags & SD_BATCH_LOCKSTEP) {
      for (auto& it : items) {
        const int a = it[0];
        if (nsteps[a] == nsteps[k] && sdk::can_lockstep(hs[a], hs[k])) {
          it.push_back(k);
          placed = true;
          break;
        }
      }
    }
    if (!placed) items.push_back(std::vector<int>(1, k));
  }
  // split large groups: a group of big grids already fills the GPU with each
  // launch, and smaller groups run concurrently on their own streams and wait
  // for fewer slow instances (lockstep runs every group to its slowest member)
  {
    std::vector<std::vector<int>> split;
    for (auto& it : items) {
      const int64_t dof = sdk::handle_dof(hs[it[0]]);
      const int cap = (int)std::max<int64_t>(1, kLockstepDof / dof);
      for (size_t a = 0; a < it.size(); a += (size_t)cap)
        split.emplace_back(it.begin() + a, it.begin() + std::min(it.size(), a + (size_t)cap));
    }
    items.swap(split);
  }
  if ((flags & SD_BATCH_GRAPH) && (flags & SD_BATCH_LOCKSTEP)) {
    // every group (single handles as groups of one) in one graph per step
    std::vector<std::vector<sd_handle*>> groups;
    std::vector<int> gsteps;
    std::vector<std::vector<sd_step_info*>> ginfos;
    for (auto& it : items) {
      std::vector<sd_handle*> g;
      std::vector<sd_step_info*> gi;
      for (int k : it) {
        g.push_back(hs[k]);
        gi.push_back(infos ? infos[k] : nullptr);
      }
      groups.push_back(g);
      gsteps.push_back(nsteps[it[0]]);
      ginfos.push_back(gi);
    }
    return sdk::step_graph_batch(groups, gsteps, ginfos);
  }
  const int ni = (int)items.size();
  const int nt = (max_threads > 0 && max_threads < ni) ? max_threads : ni;
  int dev = 0;
  cudaGetDevice(&dev);
  std::atomic<int> next(0);
  std::vector<int> rcs(ni, SD_OK);
  auto body = [&]() {
    cudaSetDevice(dev);
    sdk::t_conc = nt > 1 ? 1 : 0;  // the workers' runs share the GPU
    for (;;) {
      const int w = next.fetch_add(1);
      if (w >= ni) return;
      const std::vector<int>& it = items[w];
      if (it.size() == 1) {
        const int k = it[0];
        rcs[w] = sd_step(hs[k], nsteps[k], infos ? infos[k] : nullptr);
      } else {
        std::vector<sd_handle*> g;
        std::vector<sd_step_info*> gi;
        for (int k : it) {
          g.push_back(hs[k]);
          gi.push_back(infos ? infos[k] : nullptr);
        }
        rcs[w] = sdk::step_lockstep(g.data(), (int)g.size(), nsteps[it[0]], gi.data());
      }
    }
  };
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t) th.emplace_back(body);
  for (auto& t : th) t.join();
  for (int w = 0; w < ni; ++w)
    if (rcs[w] != SD_OK) return rcs[w];
  return SD_OK;
}

int sd_solve_batch(sd_handle* const* hs, int32_t count, const int32_t* nsteps, sd_step_info* const* infos,
                   int32_t max_threads) {
  return sd_solve_batch_ex(hs, count, nsteps, infos, max_threads, SD_BATCH_LOCKSTEP);
}

int sd_server_create(int64_t hbm_budget_bytes, int32_t max_running, const sd_options* opt, sd_server** out) {
  return sd_server_create_ex(hbm_budget_bytes, max_running, opt, 0, out);
}

int sd_server_create_ex(int64_t hbm_budget_bytes, int32_t max_running, const sd_options* opt, int32_t flags,
                        sd_server** out) {
  if (!out || hbm_budget_bytes <= 0 || max_running < 1) return SD_E_INVAL;
  sd_server* S = new sd_server();
  sd_options_default(&S->opt);
  if (opt) S->opt = *opt;
  S->auto_depth = opt == nullptr;
  S->budget = hbm_budget_bytes;
  S->max_running = max_running;
  S->flags = flags;
  cudaGetDevice(&S->device);
  for (int k = 0; k < max_running; ++k) S->workers.emplace_back(worker_loop, S);
  *out = S;
  return SD_OK;
}

int sd_submit(sd_server* S, const sd_request* req, uint64_t* ticket) {
  if (!S || !req || !ticket || !req->K || req->nsteps < 0) return SD_E_INVAL;
  // the device memory of the run as it will be created (its own multigrid depth)
  const sd_options ro = run_options(S, *req);
  const int64_t est = sd_memory_estimate(&req->grid, &ro);
  if (est < 0) return SD_E_INVAL;
  // what admission reserves: the arena plus setup temporaries and stream
  // resources; a request accepted here always fits an idle server
  const int64_t need = est + kRunSlack;
  if (need > S->budget) return SD_E_NOMEM;
  const int n = req->grid.nx;
  std::unique_ptr<Job> J(new Job());
  J->geometry = S->opt.geometry;
  J->req = *req;
  J->K.assign(req->K, req->K + (size_t)n * n);
  J->req.K = nullptr;
  J->est = need;
  J->t_submit = clk::now();
  {
    std::lock_guard<std::mutex> lk(S->mu);
    J->id = S->next_id++;
    *ticket = J->id;
    S->queue.push_back(J->id);
    S->jobs[J->id] = std::move(J);
  }
  S->cv.notify_all();
  return SD_OK;
}

int sd_poll(sd_server* S, uint64_t ticket, sd_result* out, double* x) {
  if (!S) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return SD_E_STATE;
  Job* J = it->second.get();
  if (J->t_end == clk::time_point()) {
    if (out) {
      std::memset(out, 0, sizeof(*out));
      out->status = SD_PENDING;
    }
    return SD_PENDING;
  }
  if (out) *out = J->res;
  if (x && !J->x.empty()) std::memcpy(x, J->x.data(), sizeof(double) * J->x.size());
  const int st = J->status;
  S->jobs.erase(it);
  return st;
}

int sd_server_drain(sd_server* S) {
  if (!S) return SD_E_INVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  S->cv.wait(lk, [&] { return S->queue.empty() && S->running == 0; });
  return SD_OK;
}

void sd_server_destroy(sd_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& c : S->classes) {
    if (c.second->th.joinable()) c.second->th.join();
    for (Job* J : c.second->running)
      if (J->h) sd_destroy(J->h);
  }
  delete S;
}

}  // extern "C"
