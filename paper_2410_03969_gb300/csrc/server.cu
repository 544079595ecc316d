// Continuous-batching server for factorisation jobs (declared in
// include/rpchol.h): a FIFO queue, admission by device memory and slots, one
// context and stream per admitted job, and a worker thread that admits,
// launches and observes completion.  Each job is an ordinary rpchol_run
// (Algorithm 2 of arXiv 2410.03969) on its own context, so its result is
// the one it would have alone; concurrency only overlaps jobs on the GPU.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/rpchol.h"
#include "internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

enum JobState { kWaiting = 0, kRunning = 1, kFinished = 2, kFailed = 3 };

struct Job {
  uint64_t ticket = 0;
  rpchol_job spec{};
  std::vector<unsigned char> X;  // host copy of the points
  int64_t bytes = 0;
  int state = kWaiting;
  rpchol_status status = RPCHOL_OK;
  rpchol_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Clock::time_point t_submit, t_admit, t_done;
  int64_t rank = 0, rounds = 0;
  double trace_error = 0.0;
  int users = 0;  // copy-outs in progress
};

}  // namespace

struct rpchol_server {
  int device = 0;
  int64_t budget = 0;
  int max_slots = 1;
  std::mutex mu;
  std::condition_variable cv_work;  // new job, or memory released
  std::condition_variable cv_done;  // a job finished
  std::deque<Job*> queue;
  std::vector<Job*> running;
  std::map<uint64_t, Job*> jobs;
  uint64_t next_ticket = 1;
  int64_t held_bytes = 0;
  int held_slots = 0;
  bool stop = false;
  std::thread worker;
};

namespace {

void free_job_device(Job* j) {
  if (j->ctx) rpchol_destroy(j->ctx);
  j->ctx = nullptr;
  if (j->done) cudaEventDestroy(j->done);
  j->done = nullptr;
  if (j->stream) cudaStreamDestroy(j->stream);
  j->stream = nullptr;
}

// Admission: context, stream, run.  Called without the lock.
rpchol_status start_job(Job* j) {
  const rpchol_job& q = j->spec;
  cudaError_t e = cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    rpchol::set_last_error("server: stream/event creation failed: %s", cudaGetErrorString(e));
    return RPCHOL_ECUDA;
  }
  const int T = q.T > 0 ? q.T : (int)(q.N < 120 ? q.N : 120);
  rpchol_opts o;
  memset(&o, 0, sizeof(o));
  o.precision = q.precision;
  o.use_graph = 1;
  o.stream = (void*)j->stream;
  rpchol_status s = rpchol_create(q.kind, q.sigma, j->X.data(), q.N, q.d, q.x_dtype, 0, q.k, T,
                                  &o, &j->ctx);
  std::vector<unsigned char>().swap(j->X);  // the context holds the points now
  if (s != RPCHOL_OK) return s;
  s = rpchol_run(j->ctx, q.k, T, q.seed);
  if (s != RPCHOL_OK) return s;
  e = cudaEventRecord(j->done, j->stream);
  if (e != cudaSuccess) {
    rpchol::set_last_error("server: cudaEventRecord: %s", cudaGetErrorString(e));
    return RPCHOL_ECUDA;
  }
  return RPCHOL_OK;
}

void worker_main(rpchol_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    bool progress = false;
    // completions
    for (size_t i = 0; i < sv->running.size();) {
      Job* j = sv->running[i];
      const cudaError_t q = cudaEventQuery(j->done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      j->t_done = Clock::now();
      sv->running.erase(sv->running.begin() + (long)i);
      lk.unlock();
      rpchol_run_stats st;
      rpchol_status s = q == cudaSuccess ? rpchol_stats(j->ctx, &st) : RPCHOL_ECUDA;
      lk.lock();
      if (s == RPCHOL_OK) {
        j->status = (rpchol_status)st.status;
        j->rank = st.rank;
        j->rounds = st.rounds;
        j->trace_error = st.trace_error;
        j->state = st.status == RPCHOL_OK ? kFinished : kFailed;
      } else {
        j->status = s;
        j->state = kFailed;
      }
      progress = true;
      sv->cv_done.notify_all();
    }
    // admission, oldest first
    while (!sv->queue.empty() && !sv->stop) {
      Job* j = sv->queue.front();
      if (sv->held_slots >= sv->max_slots || sv->held_bytes + j->bytes > sv->budget) break;
      sv->queue.pop_front();
      sv->held_slots += 1;
      sv->held_bytes += j->bytes;
      j->t_admit = Clock::now();
      j->state = kRunning;
      lk.unlock();
      const rpchol_status s = start_job(j);
      lk.lock();
      if (s == RPCHOL_OK) {
        sv->running.push_back(j);
      } else {
        j->status = s;
        j->state = kFailed;
        j->t_done = Clock::now();
        sv->cv_done.notify_all();
      }
      progress = true;
    }
    if (sv->stop && sv->running.empty()) break;
    if (!progress) {
      // running jobs are observed by polling their events; otherwise sleep
      // until a submission or a release
      if (sv->running.empty())
        sv->cv_work.wait(lk);
      else
        sv->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

}  // namespace

extern "C" {

rpchol_status rpchol_server_create(int64_t mem_budget_bytes, int32_t max_slots,
                                   rpchol_server** out) {
  if (!out || mem_budget_bytes <= 0 || max_slots < 1) {
    rpchol::set_last_error("invalid argument: budget=%lld slots=%d", (long long)mem_budget_bytes,
                           max_slots);
    return RPCHOL_EINVAL;
  }
  *out = nullptr;
  rpchol_server* sv = new (std::nothrow) rpchol_server();
  if (!sv) return RPCHOL_ENOMEM;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    rpchol::set_last_error("no CUDA device");
    return RPCHOL_ECUDA;
  }
  sv->budget = mem_budget_bytes;
  sv->max_slots = max_slots;
  sv->worker = std::thread(worker_main, sv);
  *out = sv;
  return RPCHOL_OK;
}

rpchol_status rpchol_server_submit(rpchol_server* sv, const rpchol_job* job, uint64_t* ticket) {
  if (!sv || !job || !ticket || !job->X || job->N < 1 || job->d < 1 || job->d > 4096 ||
      job->k < 1 || job->k > job->N || !(job->sigma > 0.0) || job->kind < 0 || job->kind > 4 ||
      job->T < 0 || job->T > 256 ||
      (job->x_dtype != RPCHOL_DT_F32 && job->x_dtype != RPCHOL_DT_F64) ||
      (job->precision != RPCHOL_FP64 && job->precision != RPCHOL_MIXED)) {
    rpchol::set_last_error("invalid job");
    return RPCHOL_EINVAL;
  }
  const int T = job->T > 0 ? job->T : (int)(job->N < 120 ? job->N : 120);
  const int64_t bytes = rpchol_context_bytes(job->N, job->d, job->k, T, job->precision);
  if (bytes > sv->budget) {
    rpchol::set_last_error("job needs %lld bytes, more than the budget", (long long)bytes);
    return RPCHOL_EINVAL;
  }
  Job* j = new (std::nothrow) Job();
  if (!j) return RPCHOL_ENOMEM;
  const size_t xb = (size_t)job->N * (size_t)job->d * (job->x_dtype == RPCHOL_DT_F32 ? 4 : 8);
  try {
    j->X.resize(xb);
  } catch (...) {
    delete j;
    return RPCHOL_ENOMEM;
  }
  memcpy(j->X.data(), job->X, xb);
  j->spec = *job;
  j->spec.X = nullptr;
  j->bytes = bytes;
  j->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> g(sv->mu);
    j->ticket = sv->next_ticket++;
    sv->jobs[j->ticket] = j;
    sv->queue.push_back(j);
  }
  sv->cv_work.notify_one();
  *ticket = j->ticket;
  return RPCHOL_OK;
}

rpchol_status rpchol_server_poll(rpchol_server* sv, uint64_t ticket, int32_t wait_ms,
                                 rpchol_job_result* out) {
  if (!sv || !out) return RPCHOL_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) {
    rpchol::set_last_error("unknown ticket %llu", (unsigned long long)ticket);
    return RPCHOL_EINVAL;
  }
  Job* j = it->second;
  auto finished = [&] { return j->state >= kFinished; };
  if (wait_ms < 0)
    sv->cv_done.wait(lk, finished);
  else if (wait_ms > 0)
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), finished);
  memset(out, 0, sizeof(*out));
  out->state = j->state;
  out->status = j->status;
  out->rank = j->rank;
  out->rounds = j->rounds;
  out->trace_error = j->trace_error;
  out->device_bytes = j->bytes;
  if (j->state >= kRunning) out->queue_ms = ms_between(j->t_submit, j->t_admit);
  if (j->state >= kFinished) {
    out->run_ms = ms_between(j->t_admit, j->t_done);
    out->latency_ms = ms_between(j->t_submit, j->t_done);
  }
  return RPCHOL_OK;
}

rpchol_status rpchol_server_copy_factor(rpchol_server* sv, uint64_t ticket, void* F_out,
                                        int64_t ld_out, int64_t* pivots_out) {
  if (!sv) return RPCHOL_EINVAL;
  Job* j;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return RPCHOL_EINVAL;
    j = it->second;
    if (j->state != kFinished || !j->ctx) return RPCHOL_EBUSY;
    j->users += 1;
  }
  const rpchol_status s = rpchol_copy_factor_raw(j->ctx, F_out, ld_out, pivots_out);
  std::lock_guard<std::mutex> g(sv->mu);
  j->users -= 1;
  return s;
}

rpchol_status rpchol_server_release(rpchol_server* sv, uint64_t ticket) {
  if (!sv) return RPCHOL_EINVAL;
  Job* j;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    auto it = sv->jobs.find(ticket);
    if (it == sv->jobs.end()) return RPCHOL_EINVAL;
    j = it->second;
    if (j->state < kFinished || j->users > 0) return RPCHOL_EBUSY;
    sv->jobs.erase(it);
  }
  free_job_device(j);
  {
    std::lock_guard<std::mutex> g(sv->mu);
    sv->held_bytes -= j->bytes;
    sv->held_slots -= 1;
  }
  delete j;
  sv->cv_work.notify_one();
  return RPCHOL_OK;
}

void rpchol_server_destroy(rpchol_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> g(sv->mu);
    sv->stop = true;
    for (Job* j : sv->queue) {
      j->state = kFailed;
      j->status = RPCHOL_ECANCELLED;
    }
    sv->queue.clear();
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& kv : sv->jobs) {
    free_job_device(kv.second);
    delete kv.second;
  }
  delete sv;
}

}  // extern "C"
