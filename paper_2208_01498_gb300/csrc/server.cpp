// Serving loop: continuous batching of amplitude requests on one GPU.
//
// A host thread owns a pool of CUDA streams.  Requests (plan + bitstrings)
// wait in arrival order; the head of the queue is admitted as soon as a
// stream is free and its plan's workspace fits in the caller's device arena
// (first-fit sub-allocation), so requests that arrive while others run start
// as slots and memory free up, and their kernels overlap on the device.  A
// finished request (cudaEvent) frees its bytes and stream for the next one.
// With batching on (tnc_server_set_batching), the waiting requests at the head
// of the queue are admitted together, up to the set number, as one batch of
// tnc_contract_batch (their nodes grouped across requests, wave by wave) on
// one stream; plans with several serial slice groups run alone.
// Every host wait is bounded; device work is plain kernels with no spin.
#include <cuda_runtime_api.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <unordered_map>

#include "tnc_internal.h"

namespace tnc {
int run_request(tnc_plan_t* plan, const uint8_t* host_bits, int batch, void* d_out, void* d_ws,
                size_t ws_bytes, void* stream);
int run_batch(int n, tnc_plan_t* const* plans, const uint8_t* const* bits, const int* batches, void* const* d_outs,
              void* d_ws, size_t ws_bytes, void* stream);
uint64_t batch_ws_bytes(int n, tnc_plan_t* const* plans);
}

using namespace tnc;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
  uint64_t ticket;
  tnc_plan_t* plan;
  std::vector<uint8_t> bits;
  int batch;
  void* d_out;
  uint64_t need;
  Clock::time_point t_submit;
  // running state
  int stream = -1;
  uint64_t arena_off = 0;
  cudaEvent_t done_ev = nullptr;
  uint64_t group = 0;  // batch id shared by the requests of one batch (0: alone)
  bool owner = true;   // holds the stream, the arena block and the event
};

struct Done {
  int status;
  double latency_ms;
};

}  // namespace

struct tnc_server {
  int device = 0;
  char* arena = nullptr;
  size_t arena_bytes = 0;
  std::vector<cudaStream_t> streams;
  std::vector<char> stream_busy;
  std::map<uint64_t, uint64_t> used;  // arena blocks: offset -> size
  std::deque<Request> queue;
  std::vector<Request> running;
  std::unordered_map<uint64_t, Done> done;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  int batching = 1;          // requests admitted together at most
  double batch_max_flops = 0, batch_max_bytes = 0;  // plans batched at most this large (0: any)
  uint64_t next_group = 1;
  size_t max_queue = 1 << 16;
  std::thread worker;

  bool alloc(uint64_t bytes, uint64_t* off) {
    uint64_t cur = 0;
    for (auto& kv : used) {
      if (kv.first >= cur + bytes) break;
      cur = std::max(cur, kv.first + kv.second);
    }
    if (cur + bytes > arena_bytes) return false;
    used[cur] = bytes;
    *off = cur;
    return true;
  }

  // small requests only: their launches, not their work, set their time
  bool batchable(const Request& r) const {
    const tnc_plan_report& rp = r.plan->p.rep;
    return rp.n_slice_groups == 1 && !r.plan->p.profiling && (batch_max_flops <= 0 || rp.real_flops <= batch_max_flops) &&
           (batch_max_bytes <= 0 || rp.bytes <= batch_max_bytes);
  }

  // Admit the batchable requests at the head of the queue (at least two, at
  // most `batching`, as many as fit the arena together) as one batch on
  // stream s; false if that does not apply.
  bool admit_batch(int s) {
    if (batching < 2 || queue.size() < 2) return false;
    std::vector<tnc_plan_t*> plans;
    for (size_t i = 0; i < queue.size() && (int)plans.size() < batching && batchable(queue[i]); ++i)
      plans.push_back(queue[i].plan);
    uint64_t off = 0;
    while (plans.size() >= 2 && !alloc(batch_ws_bytes((int)plans.size(), plans.data()), &off)) plans.pop_back();
    if (plans.size() < 2) return false;
    const size_t n = plans.size();
    const uint64_t need = batch_ws_bytes((int)n, plans.data());
    std::vector<Request> grp;
    for (size_t i = 0; i < n; ++i) {
      grp.push_back(std::move(queue.front()));
      queue.pop_front();
    }
    std::vector<const uint8_t*> bits(n);
    std::vector<int> batches(n);
    std::vector<void*> outs(n);
    for (size_t i = 0; i < n; ++i) bits[i] = grp[i].bits.data(), batches[i] = grp[i].batch, outs[i] = grp[i].d_out;
    const uint64_t gid = next_group++;
    stream_busy[s] = 1;
    int rc = run_batch((int)n, plans.data(), bits.data(), batches.data(), outs.data(), arena + off, need, streams[s]);
    cudaEvent_t ev = nullptr;
    if (rc == TNC_OK) rc = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess ? TNC_OK : TNC_ECUDA;
    if (rc == TNC_OK) rc = cudaEventRecord(ev, streams[s]) == cudaSuccess ? TNC_OK : TNC_ECUDA;
    if (rc != TNC_OK) {
      if (ev) cudaEventDestroy(ev);
      const auto now = Clock::now();
      for (auto& r : grp) done[r.ticket] = {rc, std::chrono::duration<double, std::milli>(now - r.t_submit).count()};
      used.erase(off);
      stream_busy[s] = 0;
      cv_done.notify_all();
      return true;
    }
    for (size_t i = 0; i < n; ++i) {
      grp[i].stream = s;
      grp[i].arena_off = off;
      grp[i].done_ev = ev;
      grp[i].group = gid;
      grp[i].owner = i == 0;
      running.push_back(std::move(grp[i]));
    }
    return true;
  }

  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      // completions: the owner of each finished launch sequence (a request
      // alone, or the first request of a batch) frees its resources, every
      // request of it is done
      for (size_t i = 0; i < running.size(); ++i) {
        Request& r = running[i];
        if (!r.owner) continue;
        cudaError_t q = cudaEventQuery(r.done_ev);
        if (q == cudaErrorNotReady) continue;
        const int status = q == cudaSuccess ? TNC_OK : TNC_ECUDA;
        const auto now = Clock::now();
        const uint64_t grp = r.group, tk = r.ticket;
        used.erase(r.arena_off);
        stream_busy[r.stream] = 0;
        cudaEventDestroy(r.done_ev);
        for (size_t j = 0; j < running.size();) {
          Request& m = running[j];
          if ((grp && m.group == grp) || (!grp && m.ticket == tk)) {
            done[m.ticket] = {status, std::chrono::duration<double, std::milli>(now - m.t_submit).count()};
            running.erase(running.begin() + j);
          } else {
            ++j;
          }
        }
        cv_done.notify_all();
        i = (size_t)-1;  // the vector changed: scan again
      }
      // admissions, in arrival order
      while (!queue.empty() && !stop) {
        int s = -1;
        for (size_t k = 0; k < streams.size(); ++k)
          if (!stream_busy[k]) {
            s = (int)k;
            break;
          }
        if (s < 0) break;
        uint64_t off;
        if (admit_batch(s)) continue;
        Request& r = queue.front();
        if (!alloc(r.need, &off)) break;
        Request req = std::move(queue.front());
        queue.pop_front();
        req.stream = s;
        req.arena_off = off;
        stream_busy[s] = 1;
        int rc = run_request(req.plan, req.bits.data(), req.batch, req.d_out, arena + off, req.need, streams[s]);
        if (rc == TNC_OK) rc = cudaEventCreateWithFlags(&req.done_ev, cudaEventDisableTiming) == cudaSuccess
                                   ? TNC_OK : TNC_ECUDA;
        if (rc == TNC_OK) rc = cudaEventRecord(req.done_ev, streams[s]) == cudaSuccess ? TNC_OK : TNC_ECUDA;
        if (rc != TNC_OK) {
          double ms = std::chrono::duration<double, std::milli>(Clock::now() - req.t_submit).count();
          done[req.ticket] = {rc, ms};
          used.erase(off);
          stream_busy[s] = 0;
          cv_done.notify_all();
          continue;
        }
        running.push_back(std::move(req));
      }
      if (stop && running.empty()) break;
      if (running.empty() && queue.empty()) {
        cv_work.wait_for(lk, std::chrono::milliseconds(50));
      } else {
        // poll completions at a short period without holding the lock
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
};

extern "C" {

int tnc_server_create(void* d_arena, size_t arena_bytes, int n_streams, tnc_server_t** out) {
  if (!out || !d_arena || arena_bytes == 0 || n_streams < 1 || n_streams > 64 || ((uintptr_t)d_arena & 255)) {
    set_error("tnc_server_create: invalid argument");
    return TNC_EINVAL;
  }
  *out = nullptr;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, d_arena) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    set_error("tnc_server_create: arena is not device memory");
    return TNC_EINVAL;
  }
  cudaSetDevice(attr.device);
  auto* s = new tnc_server();
  s->device = attr.device;
  s->arena = (char*)d_arena;
  s->arena_bytes = arena_bytes;
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      delete s;
      set_error("tnc_server_create: cudaStreamCreate: %s", cudaGetErrorString(e));
      return TNC_ECUDA;
    }
    s->streams.push_back(st);
  }
  s->stream_busy.assign(n_streams, 0);
  s->worker = std::thread([s] { s->loop(); });
  *out = s;
  return TNC_OK;
}

int tnc_server_submit(tnc_server_t* s, tnc_plan_t* plan, const uint8_t* bits, int batch, void* d_out,
                      uint64_t* ticket) {
  if (!s || !plan || !bits || !d_out || !ticket || batch < 1 || batch > plan->p.opts.max_batch) {
    set_error("tnc_server_submit: invalid argument");
    return TNC_EINVAL;
  }
  uint64_t need = (plan->p.prog.ws_bytes + 255) & ~(uint64_t)255;
  if (need > s->arena_bytes) {
    set_error("tnc_server_submit: plan needs %llu bytes > arena %zu", (unsigned long long)need, s->arena_bytes);
    return TNC_EBUSY;
  }
  {
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != s->device) cudaSetDevice(s->device);
    int rc = tnc_plan_upload(plan, nullptr);
    if (prev != s->device && prev >= 0) cudaSetDevice(prev);
    if (rc != TNC_OK) return rc;
  }
  Request r;
  r.plan = plan;
  r.bits.assign(bits, bits + (size_t)batch * plan->p.net.n_qubits);
  r.batch = batch;
  r.d_out = d_out;
  r.need = need;
  r.t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    set_error("tnc_server_submit: server is shutting down");
    return TNC_ESTATE;
  }
  if (s->queue.size() >= s->max_queue) {
    set_error("tnc_server_submit: queue full");
    return TNC_EBUSY;
  }
  r.ticket = s->next_ticket++;
  *ticket = r.ticket;
  s->queue.push_back(std::move(r));
  s->cv_work.notify_one();
  return TNC_OK;
}

int tnc_server_set_batching(tnc_server_t* s, int max_requests, double max_request_flops, double max_request_bytes) {
  if (!s || max_requests < 1 || max_requests > 1024 || !(max_request_flops >= 0) || !(max_request_bytes >= 0)) {
    set_error("tnc_server_set_batching: invalid argument");
    return TNC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->batching = max_requests;
  s->batch_max_flops = max_request_flops;
  s->batch_max_bytes = max_request_bytes;
  return TNC_OK;
}

int tnc_server_poll(tnc_server_t* s, uint64_t ticket, int* is_done) {
  if (!s || !is_done) {
    set_error("tnc_server_poll: invalid argument");
    return TNC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    *is_done = 1;
    return it->second.status;
  }
  *is_done = 0;
  for (auto& r : s->queue)
    if (r.ticket == ticket) return TNC_OK;
  for (auto& r : s->running)
    if (r.ticket == ticket) return TNC_OK;
  set_error("tnc_server_poll: unknown ticket %llu", (unsigned long long)ticket);
  return TNC_ENOTFOUND;
}

int tnc_server_wait(tnc_server_t* s, uint64_t ticket, int timeout_ms, double* latency_ms) {
  if (!s) {
    set_error("tnc_server_wait: invalid argument");
    return TNC_EINVAL;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto known = [&]() {
    if (s->done.count(ticket)) return true;
    for (auto& r : s->queue)
      if (r.ticket == ticket) return true;
    for (auto& r : s->running)
      if (r.ticket == ticket) return true;
    return false;
  };
  if (!known()) {
    set_error("tnc_server_wait: unknown ticket %llu", (unsigned long long)ticket);
    return TNC_ENOTFOUND;
  }
  bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                [&] { return s->done.count(ticket) > 0; });
  if (!ok) {
    set_error("tnc_server_wait: ticket %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
    return TNC_ETIMEOUT;
  }
  const Done& d = s->done[ticket];
  if (latency_ms) *latency_ms = d.latency_ms;
  return d.status;
}

int tnc_server_cancel(tnc_server_t* s, uint64_t ticket) {
  if (!s) {
    set_error("tnc_server_cancel: invalid argument");
    return TNC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
    if (it->ticket == ticket) {
      double ms = std::chrono::duration<double, std::milli>(Clock::now() - it->t_submit).count();
      s->done[ticket] = {TNC_ESTATE, ms};
      s->queue.erase(it);
      s->cv_done.notify_all();
      return TNC_OK;
    }
  for (auto& r : s->running)
    if (r.ticket == ticket) {
      set_error("tnc_server_cancel: ticket %llu is already running", (unsigned long long)ticket);
      return TNC_ESTATE;
    }
  if (s->done.count(ticket)) {
    set_error("tnc_server_cancel: ticket %llu is already done", (unsigned long long)ticket);
    return TNC_ESTATE;
  }
  set_error("tnc_server_cancel: unknown ticket %llu", (unsigned long long)ticket);
  return TNC_ENOTFOUND;
}

int tnc_server_destroy(tnc_server_t* s) {
  if (!s) return TNC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& r : s->queue) s->done[r.ticket] = {TNC_ESTATE, 0.0};
    s->queue.clear();
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto st : s->streams) cudaStreamDestroy(st);
  delete s;
  return TNC_OK;
}

}  // extern "C"
