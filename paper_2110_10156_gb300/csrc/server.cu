// Continuous-batching request loop for alignment jobs.
//
// Jobs (a fixed/floating volume pair and a set of candidate rotations, of any
// supported size) arrive at any time.  A worker thread:
//   - admits pending jobs, in arrival order or shortest expected work first
//     (less the time waited), while their device footprint fits the memory
//     budget and an active-job slot is free (device resources are
//     pooled by volume shape, so a finished job's memory serves the next job
//     of that shape without cudaFree / cudaMalloc);
//   - keeps every active job's fixed-volume spectra resident and feeds its
//     rotations to the GPU one launch group at a time on the job's own stream,
//     at most `max_inflight` groups per job, round-robin over the active jobs,
//     so that work of different jobs overlaps on the device and a job that
//     arrives while others run starts as soon as it is admitted;
//   - retires a job when its last group completes, computes the maximum over
//     rotations (Fig. 1) and records its latency.
// Each job's result is the same as scoring it alone: the per-rotation kernels
// do not depend on how rotations are grouped.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/cs_ngf.h"
#include "handle.h"

using csngf::detail::fail;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Slot {                     // device resources of one volume shape
  int32_t dims[3];
  int pad[3];
  float eps, gamma;
  int batch;
  int measure;
  int precision;
  int pad_mode;
  int tensor_cores;
  cs_ngf_fixed* f = nullptr;
  float* dA = nullptr;
  uint8_t* dMA = nullptr;
  float* dB = nullptr;
  uint8_t* dMB = nullptr;
  float* d_score = nullptr;        // per-rotation results of the current job
  int32_t* d_shift = nullptr;
  float* h_score = nullptr;        // pinned copies
  int32_t* h_shift = nullptr;
  int cap = 0;
  size_t bytes = 0;
  bool busy = false;
};

struct Job {
  int64_t id = 0;
  int32_t dims[3] = {0, 0, 0};
  std::vector<float> A, B;
  std::vector<uint8_t> MA, MB;
  std::vector<double> quats;
  int R = 0;
  cs_ngf_config cfg{};
  int pad[3] = {0, 0, 0};
  size_t bytes = 0;
  double est_ms = 0.0;              // estimated device time alone (admission priority)
  Clock::time_point t_submit, t_admit, t_done;
  enum State { PENDING, ACTIVE, DONE } state = PENDING;
  bool cancel = false;
  bool was_admitted = false;
  cs_ngf_status status = CS_NGF_OK;
  std::string error;
  Slot* slot = nullptr;
  cudaStream_t stream = nullptr;
  int cursor = 0;
  // bound-limited padding: rotations in class order (perm[i] = original
  // index; empty = unchanged), class c ends at class_end[c], lengths class_pad
  std::vector<int> perm, class_end, class_pad;
  size_t cls = 0;
  std::deque<cudaEvent_t> inflight;
  cudaEvent_t done_ev = nullptr;
  bool results_enqueued = false;
  std::vector<float> out_score;
  std::vector<int32_t> out_shift;
  float best = -INFINITY;
  int best_index = -1;
  int best_shift[3] = {0, 0, 0};
};

}  // namespace

struct cs_ngf_server {
  cs_ngf_server_config cfg{};
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int64_t next_id = 1;
  std::deque<Job*> pending;
  std::vector<Job*> active;
  std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
  std::vector<std::unique_ptr<Slot>> slots;
  size_t bytes_in_use = 0;
  int64_t admitted = 0, completed = 0;
  std::string worker_error;
};

namespace {

size_t slot_bytes(const int32_t dims[3], const int pad[3], int batch, int measure, int precision,
                  int tensor_cores, int cap) {
  const size_t nvox = (size_t)dims[0] * dims[1] * dims[2];
  return csngf::detail::handle_bytes(dims, pad, batch, measure, precision, tensor_cores) + nvox * 10 +
         (size_t)cap * 16;
}

bool same_shape(const Slot& s, const Job& j) {
  return std::memcmp(s.dims, j.dims, sizeof(s.dims)) == 0 &&
         std::memcmp(s.pad, j.pad, sizeof(s.pad)) == 0 && s.eps == j.cfg.eps &&
         s.gamma == j.cfg.gamma && s.batch == j.cfg.batch && s.measure == j.cfg.measure &&
         s.precision == j.cfg.precision && s.pad_mode == j.cfg.pad_mode &&
         s.tensor_cores == j.cfg.tensor_cores;
}

void free_slot(Slot* s) {
  cs_ngf_release(s->f);
  cudaFree(s->dA);
  cudaFree(s->dMA);
  cudaFree(s->dB);
  cudaFree(s->dMB);
  cudaFree(s->d_score);
  cudaFree(s->d_shift);
  cudaFreeHost(s->h_score);
  cudaFreeHost(s->h_shift);
}

cs_ngf_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CS_NGF_OK;
  return fail(e == cudaErrorMemoryAllocation ? CS_NGF_ENOMEM : CS_NGF_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define SV_CUDA(call) do { if (cs_ngf_status s_ = cuda_status((call), #call)) return s_; } while (0)

// device resources and inputs for an admitted job (worker thread, no lock held)
cs_ngf_status setup_job(cs_ngf_server* sv, Job* j, Slot* slot, bool fresh) {
  if (sv->cfg.inject_admission_failure == j->id)
    return fail(CS_NGF_ENOMEM, "injected admission failure");
  const size_t nvox = (size_t)j->dims[0] * j->dims[1] * j->dims[2];
  SV_CUDA(cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking));
  if (fresh) {
    SV_CUDA(cudaMalloc((void**)&slot->dA, nvox * sizeof(float)));
    SV_CUDA(cudaMalloc((void**)&slot->dMA, nvox));
    SV_CUDA(cudaMalloc((void**)&slot->dB, nvox * sizeof(float)));
    SV_CUDA(cudaMalloc((void**)&slot->dMB, nvox));
  }
  if (j->R > slot->cap) {            // grown only; a shrinking job keeps the larger buffers
    if (slot->d_score) {
      cudaFree(slot->d_score);
      cudaFree(slot->d_shift);
      cudaFreeHost(slot->h_score);
      cudaFreeHost(slot->h_shift);
      slot->d_score = nullptr;
      slot->d_shift = nullptr;
      slot->h_score = nullptr;
      slot->h_shift = nullptr;
    }
    SV_CUDA(cudaMalloc((void**)&slot->d_score, sizeof(float) * j->R));
    SV_CUDA(cudaMalloc((void**)&slot->d_shift, sizeof(int32_t) * 3 * j->R));
    SV_CUDA(cudaMallocHost((void**)&slot->h_score, sizeof(float) * j->R));
    SV_CUDA(cudaMallocHost((void**)&slot->h_shift, sizeof(int32_t) * 3 * j->R));
    slot->cap = j->R;
  }
  cudaStream_t st = j->stream;
  SV_CUDA(cudaMemcpyAsync(slot->dA, j->A.data(), nvox * sizeof(float), cudaMemcpyHostToDevice, st));
  SV_CUDA(cudaMemcpyAsync(slot->dMA, j->MA.data(), nvox, cudaMemcpyHostToDevice, st));
  SV_CUDA(cudaMemcpyAsync(slot->dB, j->B.data(), nvox * sizeof(float), cudaMemcpyHostToDevice, st));
  SV_CUDA(cudaMemcpyAsync(slot->dMB, j->MB.data(), nvox, cudaMemcpyHostToDevice, st));
  if (!slot->f) {
    cs_ngf_config c = j->cfg;
    for (int a = 0; a < 3; ++a) c.pad[a] = j->pad[a];
    if (cs_ngf_status s = cs_ngf_prepare_fixed(slot->dA, slot->dMA, j->dims, &c, st, &slot->f)) return s;
  } else if (cs_ngf_status s = cs_ngf_update_fixed(slot->f, slot->dA, slot->dMA, st)) {
    return s;
  }
  if (cs_ngf_status s = csngf::detail::upload_rotations(slot->f, j->quats.data(), j->R, st)) return s;
  if (cs_ngf_status s = csngf::detail::pack_floating(slot->f, slot->dB, slot->dMB, st)) return s;
  // FFT lengths per class of rotations (bound-limited padding), first class set up
  if (cs_ngf_status s = csngf::detail::plan_classes(slot->f, j->R, st, j->perm, j->class_end,
                                                    j->class_pad))
    return s;
  j->cls = 0;
  return csngf::detail::set_lengths(slot->f, j->class_pad.data(), st);
}

void finish_job(cs_ngf_server* sv, Job* j) {
  // caller holds sv->mu
  j->t_done = Clock::now();
  j->state = Job::DONE;
  if (j->slot) j->slot->busy = false;
  for (cudaEvent_t e : j->inflight) cudaEventDestroy(e);
  j->inflight.clear();
  if (j->done_ev) cudaEventDestroy(j->done_ev);
  j->done_ev = nullptr;
  if (j->stream) cudaStreamDestroy(j->stream);
  j->stream = nullptr;
  // inputs are no longer needed
  std::vector<float>().swap(j->A);
  std::vector<float>().swap(j->B);
  std::vector<uint8_t>().swap(j->MA);
  std::vector<uint8_t>().swap(j->MB);
  ++sv->completed;
  sv->cv_done.notify_all();
}

// pick a slot for the job: an idle slot of the same shape, else a new one
// within the budget (evicting idle slots of other shapes when needed)
Slot* find_slot(cs_ngf_server* sv, Job* j, bool* fresh) {
  for (auto& s : sv->slots)
    if (!s->busy && same_shape(*s, *j)) {
      *fresh = false;
      return s.get();
    }
  const size_t need = j->bytes;
  if (sv->bytes_in_use + need > (size_t)sv->cfg.memory_budget_bytes) {
    std::vector<Slot*> idle;
    for (auto& s : sv->slots)
      if (!s->busy) idle.push_back(s.get());
    std::sort(idle.begin(), idle.end(), [](Slot* a, Slot* b) { return a->bytes > b->bytes; });
    for (Slot* s : idle) {
      if (sv->bytes_in_use + need <= (size_t)sv->cfg.memory_budget_bytes) break;
      free_slot(s);
      sv->bytes_in_use -= s->bytes;
      sv->slots.erase(std::find_if(sv->slots.begin(), sv->slots.end(),
                                   [s](const std::unique_ptr<Slot>& p) { return p.get() == s; }));
    }
    if (sv->bytes_in_use + need > (size_t)sv->cfg.memory_budget_bytes) return nullptr;
  }
  auto s = std::make_unique<Slot>();
  std::memcpy(s->dims, j->dims, sizeof(s->dims));
  std::memcpy(s->pad, j->pad, sizeof(s->pad));
  s->eps = j->cfg.eps;
  s->gamma = j->cfg.gamma;
  s->batch = j->cfg.batch;
  s->measure = j->cfg.measure;
  s->precision = j->cfg.precision;
  s->pad_mode = j->cfg.pad_mode;
  s->tensor_cores = j->cfg.tensor_cores;
  s->bytes = need;
  sv->bytes_in_use += need;
  sv->slots.push_back(std::move(s));
  *fresh = true;
  return sv->slots.back().get();
}

void worker_loop(cs_ngf_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    if (sv->stop && sv->pending.empty() && sv->active.empty()) break;
    bool progress = false;

    // ---- admission: cancelled jobs leave; then arrival order, or shortest
    // expected work less the time waited
    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
      Job* j = *it;
      if (!j->cancel) { ++it; continue; }
      j->status = CS_NGF_ECANCELED;
      j->error = "cancelled before admission";
      it = sv->pending.erase(it);
      finish_job(sv, j);
      progress = true;
    }
    if (sv->cfg.policy == CS_NGF_SERVE_SHORTEST && sv->pending.size() > 1) {
      const Clock::time_point now = Clock::now();
      std::stable_sort(sv->pending.begin(), sv->pending.end(), [&](const Job* a, const Job* b) {
        return a->est_ms - ms_between(a->t_submit, now) < b->est_ms - ms_between(b->t_submit, now);
      });
    }
    for (auto it = sv->pending.begin(); it != sv->pending.end();) {
      Job* j = *it;
      if ((int)sv->active.size() >= sv->cfg.max_active_jobs) break;
      bool fresh = false;
      Slot* slot = find_slot(sv, j, &fresh);
      if (!slot) break;                       // wait for memory to free up
      slot->busy = true;
      it = sv->pending.erase(it);
      j->slot = slot;
      j->was_admitted = true;
      j->t_admit = Clock::now();
      ++sv->admitted;
      lk.unlock();
      cs_ngf_status s = setup_job(sv, j, slot, fresh);
      std::string err = s ? cs_ngf_last_error() : "";
      lk.lock();
      if (s) {
        j->status = s;
        j->error = err;
        if (fresh) {                          // drop a half-built slot
          free_slot(slot);
          sv->bytes_in_use -= slot->bytes;
          sv->slots.erase(std::find_if(sv->slots.begin(), sv->slots.end(),
                                       [slot](const std::unique_ptr<Slot>& p) { return p.get() == slot; }));
          j->slot = nullptr;
        }
        finish_job(sv, j);
      } else {
        j->state = Job::ACTIVE;
        sv->active.push_back(j);
      }
      progress = true;
    }

    // ---- dispatch one launch group per job per round, bounded in flight
    for (Job* j : sv->active) {
      while (!j->inflight.empty() && cudaEventQuery(j->inflight.front()) == cudaSuccess) {
        cudaEventDestroy(j->inflight.front());
        j->inflight.pop_front();
        progress = true;
      }
      if (j->results_enqueued) continue;
      const bool stop_job = j->cancel || j->cursor >= j->R;
      if (!stop_job && (int)j->inflight.size() < sv->cfg.max_inflight) {
        Slot* s = j->slot;
        // launch groups stay inside a class; the next class switches lengths
        // (which waits for this job's groups in flight)
        bool next_class = false;
        while (j->cls + 1 < j->class_end.size() && j->cursor >= j->class_end[j->cls]) {
          ++j->cls;
          next_class = true;
        }
        const int n = std::min(s->f->batch, j->class_end[j->cls] - j->cursor);
        lk.unlock();
        cs_ngf_status st = CS_NGF_OK;
        if (next_class) st = csngf::detail::set_lengths(s->f, j->class_pad.data() + 3 * j->cls, j->stream);
        if (!st) st = csngf::detail::score_range(s->f, j->cursor, n, s->d_score, s->d_shift, j->stream);
        cudaEvent_t ev = nullptr;
        if (!st) st = cuda_status(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
        if (!st) st = cuda_status(cudaEventRecord(ev, j->stream), "event record");
        std::string err = st ? cs_ngf_last_error() : "";
        lk.lock();
        if (st) {
          j->status = st;
          j->error = err;
          j->cancel = true;
          if (ev) cudaEventDestroy(ev);
        } else {
          j->inflight.push_back(ev);
          j->cursor += n;
        }
        progress = true;
      }
      if ((j->cancel || j->cursor >= j->R) && !j->results_enqueued) {
        Slot* s = j->slot;
        const int n = j->cursor;
        cudaError_t e = cudaSuccess;
        if (n > 0) {
          e = cudaMemcpyAsync(s->h_score, s->d_score, sizeof(float) * n, cudaMemcpyDeviceToHost, j->stream);
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->h_shift, s->d_shift, sizeof(int32_t) * 3 * n, cudaMemcpyDeviceToHost,
                                j->stream);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(j->done_ev, j->stream);
        if (e != cudaSuccess && !j->status) {
          j->status = CS_NGF_ECUDA;
          j->error = cudaGetErrorString(e);
        }
        j->results_enqueued = true;
        progress = true;
      }
    }

    // ---- retire finished jobs
    for (auto it = sv->active.begin(); it != sv->active.end();) {
      Job* j = *it;
      if (j->results_enqueued && (!j->done_ev || cudaEventQuery(j->done_ev) != cudaErrorNotReady)) {
        if (j->done_ev && cudaEventQuery(j->done_ev) != cudaSuccess && !j->status) {
          j->status = CS_NGF_ECUDA;
          j->error = "device error while scoring";
        }
        const int n = j->cursor;
        Slot* s = j->slot;
        if (j->perm.empty()) {
          j->out_score.assign(s->h_score, s->h_score + n);
          j->out_shift.assign(s->h_shift, s->h_shift + 3 * (size_t)n);
        } else {                              // back to submission order
          j->out_score.assign((size_t)j->R, -INFINITY);
          j->out_shift.assign(3 * (size_t)j->R, 0);
          for (int i = 0; i < n; ++i) {
            const int r = j->perm[i];
            j->out_score[r] = s->h_score[i];
            for (int a = 0; a < 3; ++a) j->out_shift[3 * (size_t)r + a] = s->h_shift[3 * (size_t)i + a];
          }
        }
        for (int r = 0; r < (int)j->out_score.size(); ++r) {
          const float v = j->out_score[r];
          if (std::isfinite(v) && (j->best_index < 0 || v > j->best)) {
            j->best = v;
            j->best_index = r;
          }
        }
        if (j->best_index >= 0)
          for (int a = 0; a < 3; ++a) j->best_shift[a] = j->out_shift[3 * (size_t)j->best_index + a];
        if (!j->status && j->cancel) {
          j->status = CS_NGF_ECANCELED;
          j->error = "cancelled while running";
        }
        if (!j->status && j->best_index < 0) j->status = CS_NGF_ENOVALID;
        it = sv->active.erase(it);
        finish_job(sv, j);
        progress = true;
      } else {
        ++it;
      }
    }

    if (!progress) sv->cv_work.wait_for(lk, std::chrono::microseconds(100));
  }
}

}  // namespace

extern "C" {

void cs_ngf_server_default_config(cs_ngf_server_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->max_active_jobs = 4;
  cfg->max_inflight = 2;
}

cs_ngf_status cs_ngf_server_create(const cs_ngf_server_config* cfg_in, cs_ngf_server** out) {
  if (!out) return fail(CS_NGF_EINVAL, "out is NULL");
  *out = nullptr;
  cs_ngf_server_config cfg;
  cs_ngf_server_default_config(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.max_active_jobs <= 0 || cfg.max_inflight <= 0)
    return fail(CS_NGF_EINVAL, "max_active_jobs and max_inflight must be positive");
  if (cfg.policy != CS_NGF_SERVE_ARRIVAL && cfg.policy != CS_NGF_SERVE_SHORTEST)
    return fail(CS_NGF_EINVAL, "unknown admission policy");
  auto* sv = new (std::nothrow) cs_ngf_server();
  if (!sv) return fail(CS_NGF_ENOMEM, "host allocation failed");
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return fail(CS_NGF_ECUDA, "no CUDA device");
  }
  if (cfg.memory_budget_bytes <= 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cfg.memory_budget_bytes = (int64_t)(fr * 0.8);
  }
  sv->cfg = cfg;
  try {
    sv->worker = std::thread(worker_loop, sv);
  } catch (...) {
    delete sv;
    return fail(CS_NGF_ENOMEM, "could not start the worker thread");
  }
  *out = sv;
  return CS_NGF_OK;
}

cs_ngf_status cs_ngf_server_submit(cs_ngf_server* sv, const float* A, const uint8_t* maskA,
                                   const float* B, const uint8_t* maskB, const int32_t dims[3],
                                   const double* quats, int32_t R, const cs_ngf_config* cfg_in,
                                   int64_t* job_id) {
  if (!sv || !A || !maskA || !B || !maskB || !dims || !quats || !job_id)
    return fail(CS_NGF_EINVAL, "NULL argument");
  if (R <= 0) return fail(CS_NGF_EINVAL, "R must be positive");
  auto j = std::make_unique<Job>();
  cs_ngf_default_config(&j->cfg);
  if (cfg_in) j->cfg = *cfg_in;
  if (cs_ngf_status s = csngf::detail::resolve_pads(dims, j->cfg, j->pad)) return s;
  if (j->cfg.batch == 0) j->cfg.batch = sv->cfg.batch > 0 ? sv->cfg.batch : 16;
  std::memcpy(j->dims, dims, sizeof(j->dims));
  j->R = R;
  j->est_ms = (double)R * j->pad[0] * j->pad[1] * j->pad[2] * 2.5e-8;
  j->bytes = slot_bytes(dims, j->pad, j->cfg.batch, j->cfg.measure, j->cfg.precision,
                        j->cfg.tensor_cores, R);
  if (j->bytes > (size_t)sv->cfg.memory_budget_bytes)
    return fail(CS_NGF_ENOMEM, "job needs " + std::to_string(j->bytes) + " device bytes, budget is " +
                                   std::to_string(sv->cfg.memory_budget_bytes));
  const size_t nvox = (size_t)dims[0] * dims[1] * dims[2];
  j->A.assign(A, A + nvox);
  j->B.assign(B, B + nvox);
  j->MA.assign(maskA, maskA + nvox);
  j->MB.assign(maskB, maskB + nvox);
  j->quats.assign(quats, quats + 4 * (size_t)R);
  j->t_submit = Clock::now();
  std::lock_guard<std::mutex> lk(sv->mu);
  if (sv->stop) return fail(CS_NGF_EINVAL, "server is shutting down");
  j->id = sv->next_id++;
  *job_id = j->id;
  sv->pending.push_back(j.get());
  sv->jobs[j->id] = std::move(j);
  sv->cv_work.notify_all();
  return CS_NGF_OK;
}

cs_ngf_status cs_ngf_server_cancel(cs_ngf_server* sv, int64_t job_id) {
  if (!sv) return fail(CS_NGF_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(job_id);
  if (it == sv->jobs.end()) return fail(CS_NGF_EINVAL, "unknown job");
  it->second->cancel = true;
  sv->cv_work.notify_all();
  return CS_NGF_OK;
}

cs_ngf_status cs_ngf_server_wait(cs_ngf_server* sv, int64_t job_id, double timeout_s,
                                 cs_ngf_job_result* res, float* best_score, int32_t* best_shift) {
  if (!sv || !res) return fail(CS_NGF_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(job_id);
  if (it == sv->jobs.end()) return fail(CS_NGF_EINVAL, "unknown job");
  Job* j = it->second.get();
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
  while (j->state != Job::DONE) {
    if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && j->state != Job::DONE)
      return fail(CS_NGF_ETIMEOUT, "job not finished within the timeout");
  }
  std::memset(res, 0, sizeof(*res));
  res->status = j->status;
  res->rotations = j->R;
  res->scored = (int32_t)j->cursor;
  res->score = j->best;
  res->rot_index = j->best_index;
  for (int a = 0; a < 3; ++a) res->shift[a] = j->best_shift[a];
  res->latency_ms = ms_between(j->t_submit, j->t_done);
  res->queue_ms = j->was_admitted ? ms_between(j->t_submit, j->t_admit) : res->latency_ms;
  // every rotation: its result, or -inf / (0, 0, 0) if it was not scored
  for (int r = 0; r < j->R; ++r) {
    const bool have = (size_t)r < j->out_score.size();
    if (best_score) best_score[r] = have ? j->out_score[r] : -INFINITY;
    if (best_shift)
      for (int a = 0; a < 3; ++a) best_shift[3 * (size_t)r + a] = have ? j->out_shift[3 * (size_t)r + a] : 0;
  }
  const cs_ngf_status st = j->status;
  if (st) fail(st, j->error);
  sv->jobs.erase(it);
  return CS_NGF_OK;
}

cs_ngf_status cs_ngf_server_stats(cs_ngf_server* sv, cs_ngf_server_info* out) {
  if (!sv || !out) return fail(CS_NGF_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  out->pending = (int32_t)sv->pending.size();
  out->active = (int32_t)sv->active.size();
  out->slots = (int32_t)sv->slots.size();
  out->admitted = sv->admitted;
  out->completed = sv->completed;
  out->bytes_in_use = (int64_t)sv->bytes_in_use;
  out->memory_budget_bytes = sv->cfg.memory_budget_bytes;
  return CS_NGF_OK;
}

void cs_ngf_server_destroy(cs_ngf_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (auto& kv : sv->jobs) kv.second->cancel = true;   // unfinished jobs end as cancelled
    sv->cv_work.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& s : sv->slots) free_slot(s.get());
  delete sv;
}

}  // extern "C"
