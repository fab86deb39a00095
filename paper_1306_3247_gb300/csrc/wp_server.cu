// Continuous-batching server for propagation requests, built on the public C ABI.
//
// Requests queue in arrival order. wp_server_progress admits queued requests while the
// device-memory budget and a stream slot allow, issues the next chunk of steps for every
// running request whose previous chunk has completed, and reports the requests that
// finished. Each running request owns one stream of the pool, so the kernels of
// different requests overlap on the device; a request's arithmetic is exactly that of
// its handle alone (the result does not depend on the mix).
//
// Device memory: wp_server_create reserves the budget in a CUDA memory pool (its release
// threshold keeps the memory after frees), and every admitted request's handle takes its
// buffers from that pool with stream-ordered allocations (wp_create_pooled), so admission
// and completion call neither cudaMalloc nor cudaFree. Should the pool be too fragmented
// to serve an admission, the request waits in the queue for the next progress call.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "wavepacket_gpu.h"

namespace {

enum JobState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Job {
  int64_t id = 0;
  wp_problem pb{};
  wp_potential pot{};
  double x0[3] = {0, 0, 0}, p0[3] = {0, 0, 0}, sigma[3] = {1, 1, 1};
  int64_t nt = 0, remaining = 0;
  int64_t bytes = 0;
  int slot = -1;
  JobState state = QUEUED;
  wp_status failed = WP_OK;  // admission error, reported by wp_server_fetch
  wp_handle* h = nullptr;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Device bytes a handle of this problem holds (state, scratch, psi0, tables, records).
int64_t job_bytes(const wp_problem& pb) {
  int64_t N = 1, sum_n = 0;
  for (int d = 0; d < pb.ndim; d++) {
    N *= pb.n[d];
    sum_n += pb.n[d];
  }
  const int64_t elem = pb.precision == WP_C64 ? 8 : 16;
  int64_t b = N * elem;                         // state
  if (pb.ndim > 1) b += N * elem + 3 * (N / 4);  // scratch, line records and partials (bounded)
  if (pb.autocorr) b += N * elem;
  b += sum_n * 512 + (1 << 20);                  // per-axis tables and small buffers
  return b;
}

}  // namespace

struct wp_server {
  int64_t budget = 0, in_use = 0;
  int64_t chunk = 50;
  cudaMemPool_t pool = nullptr;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<int64_t> slot_job;  // job id on the slot, -1 when free
  std::deque<int64_t> queue;
  std::map<int64_t, Job> jobs;
  std::string err;
};

namespace {

wp_status sfail(wp_server* s, wp_status st, const std::string& m) {
  if (s) s->err = m;
  return st;
}

wp_status issue_chunk(wp_server* s, Job& j) {
  const int64_t m = j.remaining < s->chunk ? j.remaining : s->chunk;
  wp_status st = wp_step(j.h, m);
  if (st != WP_OK) return sfail(s, st, wp_last_error(j.h));
  j.remaining -= m;
  cudaError_t e = cudaEventRecord(s->events[j.slot], s->streams[j.slot]);
  if (e != cudaSuccess) return sfail(s, WP_ECUDA, cudaGetErrorString(e));
  return WP_OK;
}

wp_status admit(wp_server* s, Job& j, int slot) {
  wp_problem pb = j.pb;
  wp_status st = wp_create_pooled(&pb, s->streams[slot], s->pool, &j.h);
  if (st != WP_OK) return sfail(s, st, wp_last_error(nullptr));
  if ((st = wp_set_potential(j.h, &j.pot)) != WP_OK || (st = wp_init_gaussian(j.h, j.x0, j.p0, j.sigma)) != WP_OK) {
    s->err = wp_last_error(j.h);
    wp_destroy(j.h);
    j.h = nullptr;
    return st;
  }
  j.slot = slot;
  j.state = RUNNING;
  j.t_admit = now_s();
  s->slot_job[slot] = j.id;
  s->in_use += j.bytes;
  return issue_chunk(s, j);
}

}  // namespace

extern "C" {

wp_status wp_server_create(int64_t budget_bytes, int32_t nslots, int64_t chunk_steps, wp_server** out) {
  if (!out || budget_bytes <= 0 || nslots <= 0 || chunk_steps <= 0) return WP_EINVAL;
  *out = nullptr;
  wp_server* s = new (std::nothrow) wp_server();
  if (!s) return WP_ENOMEM;
  s->budget = budget_bytes;
  s->chunk = chunk_steps;
  {
    // the pool of the current device, holding on to up to the budget once reserved
    int dev = 0;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    cudaError_t e = cudaGetDevice(&dev);
    props.location.id = dev;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
    uint64_t keep = (uint64_t)budget_bytes;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    // reserve: one allocation of the whole budget, returned to the pool at once
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&p, (size_t)budget_bytes, s->pool, (cudaStream_t)0);
    if (e == cudaSuccess) e = cudaFreeAsync(p, (cudaStream_t)0);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)0);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      if (s->pool) cudaMemPoolDestroy(s->pool);
      delete s;
      return e == cudaErrorMemoryAllocation ? WP_ENOMEM : WP_ECUDA;
    }
  }
  for (int k = 0; k < nslots; k++) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      for (auto x : s->streams) cudaStreamDestroy(x);
      for (auto x : s->events) cudaEventDestroy(x);
      if (st) cudaStreamDestroy(st);
      cudaMemPoolDestroy(s->pool);
      delete s;
      return WP_ECUDA;
    }
    s->streams.push_back(st);
    s->events.push_back(ev);
    s->slot_job.push_back(-1);
  }
  *out = s;
  return WP_OK;
}

wp_status wp_server_submit(wp_server* s, int64_t id, const wp_problem* pb, const wp_potential* pot,
                           const double x0[3], const double p0[3], const double sigma[3], int64_t nt) {
  if (!s || !pb || !pot || !x0 || !p0 || !sigma) return sfail(s, WP_EINVAL, "NULL argument");
  if (nt < 0) return sfail(s, WP_EINVAL, "nt < 0");
  if (s->jobs.count(id)) return sfail(s, WP_EINVAL, "duplicate request id");
  Job j;
  j.id = id;
  j.pb = *pb;
  j.pot = *pot;
  for (int d = 0; d < 3; d++) {
    j.x0[d] = x0[d];
    j.p0[d] = p0[d];
    j.sigma[d] = sigma[d];
  }
  j.nt = j.remaining = nt;
  j.bytes = job_bytes(*pb);
  if (j.bytes > s->budget) return sfail(s, WP_ENOMEM, "request larger than the memory budget");
  j.t_submit = now_s();
  s->jobs[id] = j;
  s->queue.push_back(id);
  return WP_OK;
}

wp_status wp_server_progress(wp_server* s, int64_t* done_ids, int64_t cap, int64_t* ndone) {
  if (!s || !ndone) return sfail(s, WP_EINVAL, "NULL argument");
  *ndone = 0;
  // running requests: next chunk or completion
  for (size_t k = 0; k < s->slot_job.size(); k++) {
    if (s->slot_job[k] < 0) continue;
    Job& j = s->jobs[s->slot_job[k]];
    if (j.state != RUNNING) continue;
    const cudaError_t q = cudaEventQuery(s->events[k]);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return sfail(s, WP_ECUDA, cudaGetErrorString(q));
    if (j.remaining > 0) {
      wp_status st = issue_chunk(s, j);
      if (st != WP_OK) return st;
    } else {
      j.state = DONE;
      j.t_done = now_s();
      if (*ndone < cap && done_ids) done_ids[*ndone] = j.id;
      (*ndone)++;
    }
  }
  // admission in arrival order while a slot and the budget allow
  while (!s->queue.empty()) {
    Job& j = s->jobs[s->queue.front()];
    if (s->in_use + j.bytes > s->budget) break;
    int slot = -1;
    for (size_t k = 0; k < s->slot_job.size(); k++)
      if (s->slot_job[k] < 0) {
        slot = (int)k;
        break;
      }
    if (slot < 0) break;
    s->queue.pop_front();
    wp_status st = admit(s, j, slot);
    if (st == WP_ENOMEM && j.h == nullptr && s->in_use > 0) {
      // the pool could not serve the buffers now: the request waits for running ones to
      // finish and free theirs (the budget was checked above)
      (void)cudaGetLastError();
      s->queue.push_front(j.id);
      break;
    }
    if (st != WP_OK) {
      // the request cannot run (e.g. an unsupported grid): finish it with its error
      if (j.h) {
        wp_destroy(j.h);
        j.h = nullptr;
      }
      if (j.slot >= 0) {
        s->slot_job[j.slot] = -1;
        s->in_use -= j.bytes;
        j.slot = -1;
      }
      j.failed = st;
      j.state = DONE;
      j.t_admit = j.t_done = now_s();
      if (*ndone < cap && done_ids) done_ids[*ndone] = j.id;
      (*ndone)++;
    }
  }
  return WP_OK;
}

wp_status wp_server_fetch(wp_server* s, int64_t id, void* psi_host, wp_obs* obs, double* times) {
  if (!s) return WP_EINVAL;
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return sfail(s, WP_EINVAL, "unknown request id");
  Job& j = it->second;
  if (j.state != DONE) return sfail(s, WP_EBUSY, "request not finished");
  if (j.failed != WP_OK) {
    if (times) {
      times[0] = j.t_submit;
      times[1] = j.t_admit;
      times[2] = j.t_done;
    }
    const wp_status f = j.failed;
    s->jobs.erase(it);
    return sfail(s, f, "request failed at admission");
  }
  wp_status st = WP_OK;
  if (psi_host) st = wp_get_state(j.h, psi_host, 0);
  if (st == WP_OK && obs) st = wp_observe(j.h, obs);
  if (times) {
    times[0] = j.t_submit;
    times[1] = j.t_admit;
    times[2] = j.t_done;
  }
  if (st != WP_OK) s->err = wp_last_error(j.h);
  wp_destroy(j.h);
  s->in_use -= j.bytes;
  s->slot_job[j.slot] = -1;
  s->jobs.erase(it);
  return st;
}

int64_t wp_server_pending(const wp_server* s) { return s ? (int64_t)s->jobs.size() : 0; }

int64_t wp_server_bytes_in_use(const wp_server* s) { return s ? s->in_use : 0; }

int32_t wp_server_running(const wp_server* s) {
  if (!s) return 0;
  int32_t n = 0;
  for (int64_t v : s->slot_job) n += v >= 0;
  return n;
}

wp_status wp_server_destroy(wp_server* s) {
  if (!s) return WP_OK;
  for (auto& kv : s->jobs)
    if (kv.second.h) wp_destroy(kv.second.h);
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto ev : s->events) cudaEventDestroy(ev);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
  return WP_OK;
}

const char* wp_server_last_error(const wp_server* s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
