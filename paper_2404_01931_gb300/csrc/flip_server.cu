// flip_server.cu — continuous-batching step server over resident scenes
// (include/flip_server.h).  Host code only.  A launcher thread admits scenes by
// footprint, forms batches from the requests that have arrived and enqueues them;
// a completer thread waits for each scene's step on the device and completes its
// request.  Two batch slots are in flight at once: as soon as one batch's pressure
// solve has finished on the device, the next batch is formed from the requests
// that arrived meanwhile and enqueued, so its binning and P2G overlap the previous
// batch's G2P and the device does not idle across the host's round trip.  Waiting
// for the solve (rather than enqueueing at once) keeps batches large when the
// device is busy.  The two slots share one stream for their pressure solves, so
// the cooperative solve launches never run concurrently.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "../../include/flip_server.h"

void flip_set_last_error_(const std::string& msg);

namespace flipk {
int batch_step_overlapped(flip_batch* b, flip_handle* const* hs, int n);
cudaStream_t handle_stream(const flip_handle* h);
int* handle_status_word(const flip_handle* h);
int api_status_to_code(int dev_status);
}  // namespace flipk

namespace {

struct Scene {
  flip_params prm{};
  std::vector<float> host[6];  // particle arrays until the scene is admitted
  int64_t np = 0;
  size_t footprint = 0;
  flip_handle* h = nullptr;    // resident when non-null
  int create_status = FLIP_OK; // failure of the admission, if any
  bool remove = false;
  int in_flight = 0;             // batches in flight that step this scene
  int pending = 0;             // requests queued or running
};

struct Request {
  int scene = -1;
  double t_arrival = 0.0, t_start = -1.0, t_done = -1.0;
  int status = FLIP_OK;
  int batch_size = 0;
  bool done = false;
};

constexpr int kSlots = 2;  // batches in flight at once

// A batch enqueued on the device: its requests, their scenes' handles, and one
// event per scene recorded on the scene's stream after its step and after the
// copy of the scene's status word into the slot's pinned status array.
struct InFlight {
  int slot = 0;
  int launch_status = FLIP_OK;
  std::vector<int64_t> tickets;
  std::vector<flip_handle*> hs;
  std::vector<cudaEvent_t> done;
};

}  // namespace

struct flip_server {
  size_t budget = 0;
  int max_batch = 1;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<int, Scene> scenes;
  int next_scene = 0;
  std::deque<int> admit_queue;
  std::map<int64_t, Request> reqs;
  std::deque<int64_t> queue;
  int64_t next_ticket = 0;
  int64_t outstanding = 0;
  size_t used = 0;
  int resident = 0;
  bool stop = false;
  bool launcher_done = false;
  cudaStream_t solve_stream = nullptr;  // shared by the slots' batched solves
  flip_batch* slot[kSlots] = {};
  bool slot_busy[kSlots] = {};
  int* slot_status[kSlots] = {};  // pinned: each scene's status word after its step
  std::vector<cudaEvent_t> event_pool;  // per-scene completion events, reused
  std::deque<InFlight> inflight;
  std::condition_variable cv_inflight;
  cudaEvent_t last_solve = nullptr;  // end of the newest batch's solve, until seen
  bool overlap = true;               // flip_server_set_overlap
  std::thread worker, completer;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // Admits waiting scenes in arrival order while they fit; called with mu held.
  void admit_locked() {
    while (!admit_queue.empty()) {
      const int id = admit_queue.front();
      auto it = scenes.find(id);
      if (it == scenes.end() || it->second.remove) {
        admit_queue.pop_front();
        continue;
      }
      Scene& sc = it->second;
      if (used + sc.footprint > budget) break;
      flip_handle* h = nullptr;
      const int rc = flip_create(&sc.prm, sc.host[0].data(), sc.host[1].data(), sc.host[2].data(),
                                 sc.host[3].data(), sc.host[4].data(), sc.host[5].data(), sc.np,
                                 0, nullptr, nullptr, &h);
      admit_queue.pop_front();
      for (auto& v : sc.host) std::vector<float>().swap(v);
      if (rc != FLIP_OK) {
        sc.create_status = rc;
        continue;
      }
      sc.h = h;
      used += sc.footprint;
      ++resident;
    }
  }

  // Frees removed scenes that have nothing pending; called with mu held.
  bool reap_locked() {
    bool freed = false;
    for (auto it = scenes.begin(); it != scenes.end();) {
      Scene& sc = it->second;
      if (sc.remove && sc.pending == 0) {
        if (sc.h) {
          flip_destroy(sc.h);
          used -= sc.footprint;
          --resident;
          freed = true;
        }
        it = scenes.erase(it);
      } else {
        ++it;
      }
    }
    return freed;
  }

  void complete_locked(int64_t ticket, int status, double t_done, int batch_size) {
    Request& r = reqs[ticket];
    r.status = status;
    r.t_done = t_done;
    r.batch_size = batch_size;
    r.done = true;
    auto it = scenes.find(r.scene);
    if (it != scenes.end()) it->second.pending -= 1;
    outstanding -= 1;
  }

  int free_slot_locked() const {
    for (int k = 0; k < kSlots; ++k)
      if (!slot_busy[k]) return k;
    return -1;
  }

  cudaEvent_t take_event_locked() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }

  // Launcher: forms batches from arrived requests of idle resident scenes and
  // enqueues them on a free slot, without waiting for the device.
  void run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      if (reap_locked()) cv_done.notify_all();
      admit_locked();
      // requests of scenes that failed admission finish with that status
      for (auto q = queue.begin(); q != queue.end();) {
        auto sit = scenes.find(reqs[*q].scene);
        if (sit != scenes.end() && sit->second.create_status != FLIP_OK) {
          complete_locked(*q, sit->second.create_status, now(), 0);
          q = queue.erase(q);
          cv_done.notify_all();
        } else {
          ++q;
        }
      }
      // the next batch is formed once the newest batch's solve is done (its G2P
      // may still run): requests that arrive during the solve join it
      if (!overlap && !inflight.empty()) {  // one batch at a time: wait for its end
        cv_work.wait(lk);
        continue;
      }
      if (last_solve) {
        cudaEvent_t e = last_solve;
        lk.unlock();
        cudaEventSynchronize(e);
        lk.lock();
        event_pool.push_back(e);
        last_solve = nullptr;
        continue;
      }
      const int k = free_slot_locked();
      const double t = now();
      std::vector<int64_t> pick;
      std::vector<flip_handle*> hs;
      std::set<int> in_batch;
      double next_arrival = -1.0;
      for (auto q = queue.begin(); k >= 0 && q != queue.end() && (int)pick.size() < max_batch;) {
        const Request& r = reqs[*q];
        Scene& sc = scenes[r.scene];
        // a scene whose step is still in flight may take part in the next batch
        // in the overlapped mode: its work is ordered on its stream (and the shared
        // solve stream), and each step's status is captured in stream order
        const bool ready = sc.h && (overlap || sc.in_flight == 0) && !in_batch.count(r.scene);
        if (ready && r.t_arrival <= t) {
          pick.push_back(*q);
          hs.push_back(sc.h);
          in_batch.insert(r.scene);
          q = queue.erase(q);
        } else {
          if (ready && (next_arrival < 0.0 || r.t_arrival < next_arrival)) next_arrival = r.t_arrival;
          ++q;
        }
      }
      if (pick.empty()) {
        if (stop && inflight.empty()) {
          // no request can run any more: finish the rest as refused
          for (int64_t q : queue) complete_locked(q, FLIP_E_ARG, now(), 0);
          queue.clear();
          cv_done.notify_all();
          break;
        }
        // woken by a submission, an admission, a completed batch (a free slot or an
        // idle scene) or the next arrival time
        if (k >= 0 && next_arrival >= 0.0)
          cv_work.wait_for(lk, std::chrono::duration<double>(std::max(0.0, next_arrival - t)));
        else
          cv_work.wait(lk);
        continue;
      }
      InFlight f;
      f.slot = k;
      f.tickets = pick;
      f.hs = hs;
      for (size_t q = 0; q < pick.size(); ++q) {
        reqs[pick[q]].t_start = t;
        reqs[pick[q]].batch_size = (int)pick.size();
        scenes[reqs[pick[q]].scene].in_flight += 1;
        f.done.push_back(take_event_locked());
      }
      slot_busy[k] = true;
      cudaEvent_t solved = take_event_locked();
      lk.unlock();
      f.launch_status = flipk::batch_step_overlapped(slot[k], hs.data(), (int)hs.size());
      for (size_t q = 0; q < hs.size(); ++q) {
        // the step's status word, read and cleared in stream order, then its event
        const cudaStream_t hs_q = flipk::handle_stream(hs[q]);
        int* word = flipk::handle_status_word(hs[q]);
        if (!f.done[q] ||
            cudaMemcpyAsync(slot_status[k] + q, word, sizeof(int), cudaMemcpyDeviceToHost,
                            hs_q) != cudaSuccess ||
            cudaMemsetAsync(word, 0, sizeof(int), hs_q) != cudaSuccess ||
            cudaEventRecord(f.done[q], hs_q) != cudaSuccess) {
          cudaGetLastError();
          if (f.launch_status == FLIP_OK) f.launch_status = FLIP_E_CUDA;
        }
      }
      // the solve stream's last work of the call is the batched solve
      if (solved && cudaEventRecord(solved, solve_stream) != cudaSuccess) {
        cudaGetLastError();
        cudaEventDestroy(solved);
        solved = nullptr;
      }
      lk.lock();
      last_solve = solved;
      inflight.push_back(std::move(f));
      cv_inflight.notify_one();
    }
    launcher_done = true;
    cv_inflight.notify_one();
  }

  // Completer: waits for the scenes of the oldest batch in order, each on its own
  // event, and completes each request as soon as its scene's step is done.
  void complete() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      cv_inflight.wait(lk, [&] { return !inflight.empty() || launcher_done; });
      if (inflight.empty()) break;
      InFlight& f = inflight.front();
      lk.unlock();
      std::vector<int> st(f.hs.size(), f.launch_status);
      for (size_t q = 0; q < f.hs.size(); ++q) {
        int s2 = FLIP_E_CUDA;
        if (f.done[q] && cudaEventSynchronize(f.done[q]) == cudaSuccess)
          s2 = flipk::api_status_to_code(slot_status[f.slot][q]);
        cudaGetLastError();
        if (st[q] == FLIP_OK) st[q] = s2;
        const double t_done = now();
        lk.lock();
        scenes[reqs[f.tickets[q]].scene].in_flight -= 1;
        complete_locked(f.tickets[q], st[q], t_done, (int)f.hs.size());
        if (f.done[q]) event_pool.push_back(f.done[q]);
        f.done[q] = nullptr;
        cv_done.notify_all();
        cv_work.notify_one();  // the scene may take part in the next batch
        lk.unlock();
      }
      lk.lock();
      slot_busy[f.slot] = false;
      inflight.pop_front();
      cv_work.notify_one();
    }
  }
};

extern "C" {

int flip_server_create(size_t budget_bytes, int32_t max_batch, flip_server** out) {
  if (!out) return FLIP_E_ARG;
  *out = nullptr;
  if (max_batch < 1 || max_batch > 4096) {
    flip_set_last_error_("max_batch must be in [1, 4096]");
    return FLIP_E_ARG;
  }
  flip_server* s = new (std::nothrow) flip_server();
  if (!s) return FLIP_E_OOM;
  s->budget = budget_bytes;
  s->max_batch = max_batch;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    flip_set_last_error_("no CUDA device");
    return FLIP_E_NOGPU;
  }
  if (cudaStreamCreateWithFlags(&s->solve_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    flip_set_last_error_("cudaStreamCreate failed");
    return FLIP_E_CUDA;
  }
  for (int k = 0; k < kSlots; ++k) {
    int rc = flip_batch_create(max_batch, s->solve_stream, &s->slot[k]);
    if (rc == FLIP_OK &&
        cudaMallocHost((void**)&s->slot_status[k], sizeof(int) * (size_t)max_batch) != cudaSuccess) {
      cudaGetLastError();
      flip_batch_destroy(s->slot[k]);
      rc = FLIP_E_OOM;
    }
    if (rc != FLIP_OK) {
      for (int q = 0; q < k; ++q) {
        flip_batch_destroy(s->slot[q]);
        cudaFreeHost(s->slot_status[q]);
      }
      cudaStreamDestroy(s->solve_stream);
      delete s;
      return rc;
    }
  }
  s->worker = std::thread([s] { s->run(); });
  s->completer = std::thread([s] { s->complete(); });
  *out = s;
  return FLIP_OK;
}

int flip_server_add_scene(flip_server* s, const flip_params* params, const float* x,
                          const float* y, const float* z, const float* u, const float* v,
                          const float* w, int64_t np, int32_t* scene_id) {
  if (!s || !params || !scene_id) return FLIP_E_ARG;
  if (np < 0 || (np > 0 && (!x || !y || !z || !u || !v || !w))) return FLIP_E_ARG;
  const size_t fp = flip_footprint_bytes(params, np);
  if (fp == 0) return FLIP_E_ARG;
  if (fp > s->budget) {
    flip_set_last_error_("the scene's footprint exceeds the server's whole budget");
    return FLIP_E_OOM;
  }
  Scene sc;
  sc.prm = *params;
  sc.np = np;
  sc.footprint = fp;
  const float* src[6] = {x, y, z, u, v, w};
  for (int a = 0; a < 6; ++a) sc.host[a].assign(src[a], src[a] + np);
  std::lock_guard<std::mutex> lk(s->mu);
  const int id = s->next_scene++;
  s->scenes.emplace(id, std::move(sc));
  s->admit_queue.push_back(id);
  *scene_id = id;
  s->cv_work.notify_one();
  return FLIP_OK;
}

int flip_server_submit(flip_server* s, int32_t scene, double t_arrival, int64_t* ticket) {
  if (!s || !ticket) return FLIP_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->scenes.find(scene);
  if (it == s->scenes.end() || it->second.remove) return FLIP_E_ARG;
  const int64_t t = s->next_ticket++;
  Request r;
  r.scene = scene;
  r.t_arrival = t_arrival < 0.0 ? s->now() : t_arrival;
  s->reqs[t] = r;
  s->queue.push_back(t);
  it->second.pending += 1;
  s->outstanding += 1;
  *ticket = t;
  s->cv_work.notify_one();
  return FLIP_OK;
}

int flip_server_wait(flip_server* s, int64_t ticket, flip_request_info* info) {
  if (!s) return FLIP_E_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->reqs.find(ticket) == s->reqs.end()) return FLIP_E_ARG;
  // another waiter on the same ticket may collect it first: then this one ends too
  s->cv_done.wait(lk, [&] {
    auto w = s->reqs.find(ticket);
    return w == s->reqs.end() || w->second.done;
  });
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return FLIP_E_ARG;
  const Request& r = it->second;
  if (info) {
    info->scene = r.scene;
    info->status = r.status;
    info->t_arrival = r.t_arrival;
    info->t_start = r.t_start;
    info->t_done = r.t_done;
    info->batch_size = r.batch_size;
    info->reserved = 0;
  }
  const int st = r.status;
  s->reqs.erase(ticket);
  // the two warnings (the step is committed) read as success; info->status keeps them
  return (st == FLIP_E_NOT_CONVERGED || st == FLIP_E_CAPACITY) ? FLIP_OK : st;
}

int flip_server_drain(flip_server* s) {
  if (!s) return FLIP_E_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_work.notify_one();
  s->cv_done.wait(lk, [&] { return s->outstanding == 0; });
  return FLIP_OK;
}

double flip_server_now(const flip_server* s) { return s ? s->now() : 0.0; }

int flip_server_set_fused(flip_server* s, int32_t enable) {
  if (!s) return FLIP_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);  // the launcher holds mu while it forms a batch
  for (int k = 0; k < kSlots; ++k)
    if (int rc = flip_batch_set_fused(s->slot[k], enable)) return rc;
  return FLIP_OK;
}

int flip_server_set_overlap(flip_server* s, int32_t enable) {
  if (!s) return FLIP_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->overlap = enable != 0;
  s->cv_work.notify_one();
  return FLIP_OK;
}

int flip_server_usage(flip_server* s, int32_t* resident, size_t* bytes) {
  if (!s) return FLIP_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (resident) *resident = s->resident;
  if (bytes) *bytes = s->used;
  return FLIP_OK;
}

int flip_server_scene_handle(flip_server* s, int32_t scene, flip_handle** h) {
  if (!s || !h) return FLIP_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->scenes.find(scene);
  if (it == s->scenes.end() || !it->second.h) return FLIP_E_ARG;
  *h = it->second.h;
  return FLIP_OK;
}

int flip_server_remove_scene(flip_server* s, int32_t scene) {
  if (!s) return FLIP_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->scenes.find(scene);
  if (it == s->scenes.end()) return FLIP_E_ARG;
  it->second.remove = true;
  s->cv_work.notify_one();
  return FLIP_OK;
}

void flip_server_destroy(flip_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_one();
  }
  if (s->worker.joinable()) s->worker.join();
  if (s->completer.joinable()) s->completer.join();
  for (auto& kv : s->scenes)
    if (kv.second.h) flip_destroy(kv.second.h);
  for (int k = 0; k < kSlots; ++k) {
    flip_batch_destroy(s->slot[k]);
    if (s->slot_status[k]) cudaFreeHost(s->slot_status[k]);
  }
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  if (s->solve_stream) {
    cudaStreamSynchronize(s->solve_stream);
    cudaStreamDestroy(s->solve_stream);
  }
  delete s;
}

}  // extern "C"
