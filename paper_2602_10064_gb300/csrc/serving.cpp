// Serving loop: tacaw_submit / tacaw_poll / tacaw_wait / tacaw_cancel.
//
// Requests (a trajectory plus geometry, beam and output) are queued on submission; a worker
// thread admits them while their device-memory footprint fits the context's budget and a
// stream is free, and runs each admitted request's whole path (tacaw_run's pipeline) on its
// own stream, so the kernels of concurrently admitted requests overlap on the GPU.  Requests
// that arrive while others run are admitted as soon as memory and a stream free up
// (continuous batching).  A request that does not fit may be overtaken by later ones that do,
// at most kMaxSkips times; after that nothing is admitted ahead of it.  Per-request host
// timestamps (submission, admission, completion) give latency percentiles.
//
// Requests come in two classes by their work (probes x frames x slices x grid points): small
// ones run on high-priority streams of their own and large ones on normal-priority streams, so
// a small request neither waits for a stream held by a long scan nor, once launched, for the
// long scan's pending blocks.  Each class has "serving_streams" streams.
//
// Requests of the same geometry (parameters, probes, frame and atom counts, species, arithmetic
// and output) that are queued together are coalesced (tacaw_serving_hold queues a batch of
// requests before any of them is admitted), up to the context option "max_coalesce"
// (default 16), into one run: their
// trajectories are stacked along the frame axis, so every slice launch, potential launch and
// time-transform launch covers all of them, and each request's output is copied out of the
// stacked result.  A coalesced request's result is the same, bit for bit, as alone: frames and
// trajectories are independent in every kernel, and the launch grouping does not change the
// arithmetic.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tacaw_api_internal.h"

namespace tacaw {

namespace {
constexpr int kMaxSkips = 8;
constexpr size_t kPinnedMinBlock = (size_t)64 << 10;
constexpr size_t kPinnedCacheBytes = (size_t)4 << 30;

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct Job {
  uint64_t ticket = 0;
  tacaw_params params{};
  tacaw_probe probe{};
  std::vector<double> probe_xy;
  int64_t A = 0, F = 0;
  int32_t precision = 0, reduce = 0;
  const float* pos_dev = nullptr;  // caller's device positions (kept valid by the caller)
  float* pos_pinned = nullptr;     // copy of host positions
  std::vector<int32_t> Z;          // host copy of the species
  float* S_user = nullptr;
  bool S_host = false;
  float* S_pinned = nullptr;
  size_t out_elems = 0;
  uint64_t footprint = 0;
  int skips = 0;
  // run state
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  float* d_pos_tmp = nullptr;
  float* d_S_tmp = nullptr;
  std::vector<std::shared_ptr<Job>> followers;  // coalesced into this request's run
  int cls = 0;                                   // stream class: 1 small (high priority), 0 large
  int batched = 1;                               // requests in the run this request is part of
  int status = TACAW_PENDING;
  bool canceled = false;
  double t_submit = 0, t_admit = 0, t_done = 0;
};

// Page-locked host blocks for the requests' host inputs and outputs, reused across requests:
// allocating or freeing page-locked memory can wait for the whole device, which would hold
// a submission, or the worker finishing a request, behind every running request.  Blocks come
// in power-of-two sizes from 64 KiB; at most kPinnedCacheBytes of free blocks are kept.
struct PinnedPool {
  std::mutex mu;
  std::multimap<size_t, void*> free_blocks;  // block size -> block
  std::unordered_map<void*, size_t> size_of;  // every block handed out or free
  size_t cached = 0;

  cudaError_t get(size_t bytes, void** p) {
    size_t b = kPinnedMinBlock;
    while (b < bytes) b <<= 1;
    std::lock_guard<std::mutex> lk(mu);
    auto it = free_blocks.find(b);
    if (it != free_blocks.end()) {
      *p = it->second;
      free_blocks.erase(it);
      cached -= b;
      return cudaSuccess;
    }
    const cudaError_t e = cudaMallocHost(p, b);
    if (e == cudaSuccess) size_of[*p] = b;
    return e;
  }
  void put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(mu);
    auto it = size_of.find(p);
    if (it == size_of.end()) return;
    if (cached + it->second > kPinnedCacheBytes) {
      cudaFreeHost(p);
      size_of.erase(it);
      return;
    }
    free_blocks.emplace(it->second, p);
    cached += it->second;
  }
  void clear() {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& kv : size_of) cudaFreeHost(kv.first);
    size_of.clear();
    free_blocks.clear();
    cached = 0;
  }
};

struct Serving {
  tacaw_ctx* ctx = nullptr;
  PinnedPool pinned;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::thread worker;
  bool stop = false;
  bool kick = false;  // set by submissions and shutdown: the queue changed
  bool hold = false;  // tacaw_serving_hold: nothing is admitted while set
  std::deque<std::shared_ptr<Job>> queue;
  std::vector<std::shared_ptr<Job>> active;
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<cudaStream_t> free_streams[2];  // per class: 0 large, 1 small (high priority)
  std::vector<cudaStream_t> all_streams;
  uint64_t next_ticket = 1, used = 0;
};

namespace {

void release(Serving& sv, Job& j) {
  sv.pinned.put(j.pos_pinned);
  sv.pinned.put(j.S_pinned);
  j.pos_pinned = j.S_pinned = nullptr;
  if (j.done) cudaEventDestroy(j.done);
  j.done = nullptr;
  if (j.stream) sv.free_streams[j.cls].push_back(j.stream);
  j.stream = nullptr;
}

// Requests whose runs can be stacked along the frame axis: same geometry, beam, probes,
// frame and atom counts, species, arithmetic and output.
bool same_geometry(const Job& a, const Job& b) {
  return std::memcmp(&a.params, &b.params, sizeof(tacaw_params)) == 0 && a.A == b.A && a.F == b.F &&
         a.precision == b.precision && a.reduce == b.reduce && a.probe.alpha_mrad == b.probe.alpha_mrad &&
         a.probe.n_probes == b.probe.n_probes && a.probe.defocus == b.probe.defocus &&
         a.probe.cs_mm == b.probe.cs_mm && a.probe.astig == b.probe.astig &&
         a.probe.astig_angle == b.probe.astig_angle && a.probe.coma == b.probe.coma &&
         a.probe.coma_angle == b.probe.coma_angle && a.probe.psi0 == b.probe.psi0 && a.probe_xy == b.probe_xy &&
         a.Z == b.Z;
}

// Enqueue a run of the leader j and its followers, trajectories stacked along the frame axis
// (no serving lock held): positions gathered into one buffer, one run, each request's output
// [P][F][..] copied out of the stacked [P][R][F][..] result.
int launch_batch(Serving& sv, Job& j) {
  tacaw_ctx* ctx = sv.ctx;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  std::vector<Job*> all{&j};
  for (auto& f : j.followers) all.push_back(f.get());
  const int R = (int)all.size();
  const size_t per_pos = (size_t)j.F * j.A * 3, per_out = j.out_elems / (size_t)j.probe.n_probes;
  const int P = j.probe.n_probes;
  float *d_pos = nullptr, *d_S = nullptr;
  if (j.A > 0) {
    e = cudaMallocAsync((void**)&d_pos, sizeof(float) * per_pos * R, j.stream);
    for (int r = 0; r < R && e == cudaSuccess; ++r) {
      const float* src = all[r]->pos_dev ? all[r]->pos_dev : all[r]->pos_pinned;
      e = cudaMemcpyAsync(d_pos + per_pos * r, src, sizeof(float) * per_pos, cudaMemcpyDefault, j.stream);
    }
    if (e != cudaSuccess) return cuda_err(ctx, e, "coalesced positions");
  }
  e = cudaMallocAsync((void**)&d_S, sizeof(float) * j.out_elems * R, j.stream);
  if (e != cudaSuccess) return cuda_err(ctx, e, "coalesced output");
  int rc = run_impl(ctx, j.params, j.probe, d_pos, j.Z.data(), false, j.A, j.F, j.precision, j.reduce, d_S, j.stream,
                    R);
  for (int r = 0; r < R && rc == TACAW_OK; ++r) {
    float* dst = all[r]->S_host ? all[r]->S_pinned : all[r]->S_user;
    e = copy_rows_out(ctx, dst, per_out, d_S + per_out * r, per_out * R, per_out, (size_t)P, j.stream);
    if (e != cudaSuccess) rc = cuda_err(ctx, e, "coalesced output copy");
  }
  if (d_pos) cudaFreeAsync(d_pos, j.stream);
  cudaFreeAsync(d_S, j.stream);
  if (rc == TACAW_OK) {
    e = cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(j.done, j.stream);
    if (e != cudaSuccess) rc = cuda_err(ctx, e, "request completion event");
  }
  return rc;
}

// Enqueue one admitted request on its stream (no serving lock held).
int launch(Serving& sv, Job& j) {
  if (!j.followers.empty()) return launch_batch(sv, j);
  tacaw_ctx* ctx = sv.ctx;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  const float* d_pos = j.pos_dev;
  if (j.A > 0 && !d_pos) {
    e = cudaMallocAsync((void**)&j.d_pos_tmp, sizeof(float) * j.F * j.A * 3, j.stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(j.d_pos_tmp, j.pos_pinned, sizeof(float) * j.F * j.A * 3, cudaMemcpyHostToDevice, j.stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "request positions");
    d_pos = j.d_pos_tmp;
  }
  float* d_S = j.S_user;
  if (j.S_host) {
    e = cudaMallocAsync((void**)&j.d_S_tmp, sizeof(float) * j.out_elems, j.stream);
    if (e != cudaSuccess) return cuda_err(ctx, e, "request output");
    d_S = j.d_S_tmp;
  }
  int rc = run_impl(ctx, j.params, j.probe, d_pos, j.Z.data(), false, j.A, j.F, j.precision, j.reduce, d_S, j.stream);
  if (rc == TACAW_OK && j.S_host) {
    e = copy_to_host(ctx, j.S_pinned, d_S, j.out_elems, j.stream);
    if (e != cudaSuccess) rc = cuda_err(ctx, e, "request output copy");
  }
  if (j.d_pos_tmp) cudaFreeAsync(j.d_pos_tmp, j.stream);
  if (j.d_S_tmp) cudaFreeAsync(j.d_S_tmp, j.stream);
  j.d_pos_tmp = j.d_S_tmp = nullptr;
  if (rc == TACAW_OK) {
    e = cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(j.done, j.stream);
    if (e != cudaSuccess) rc = cuda_err(ctx, e, "request completion event");
  }
  return rc;
}

void finish(Serving& sv, Job& j, int status) {
  for (auto& f : j.followers) finish(sv, *f, status);
  j.followers.clear();
  if (status == TACAW_OK && j.S_host && !j.canceled) std::memcpy(j.S_user, j.S_pinned, sizeof(float) * j.out_elems);
  j.status = j.canceled ? TACAW_ECANCELED : status;
  j.t_done = now_s();
  sv.used -= j.footprint;
  release(sv, j);
}

void worker_loop(Serving* svp) {
  Serving& sv = *svp;
  cudaSetDevice(sv.ctx->device);
  std::unique_lock<std::mutex> lk(sv.mu);
  while (true) {
    // sleep with the lock released until the queue changes, polling the running requests'
    // completions every 100 us (every 50 ms when nothing runs); a wait whose predicate held
    // from the start would keep the lock, and submissions could not enqueue while any
    // request ran
    const bool busy = !sv.active.empty() || !sv.queue.empty();
    sv.cv.wait_for(lk, busy ? std::chrono::microseconds(100) : std::chrono::microseconds(50000),
                   [&] { return sv.stop || sv.kick; });
    sv.kick = false;
    // completions
    for (size_t i = 0; i < sv.active.size();) {
      Job& j = *sv.active[i];
      const cudaError_t q = cudaEventQuery(j.done);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      finish(sv, j, q == cudaSuccess ? TACAW_OK : TACAW_ECUDA);
      sv.active.erase(sv.active.begin() + i);
      sv.cv_done.notify_all();
    }
    if (sv.stop && sv.active.empty()) break;
    // admissions: in order; one request that does not fit may be overtaken, at most
    // kMaxSkips times, after which nothing is admitted ahead of it
    Job* blocked = nullptr;
    for (auto it = sv.queue.begin();
         !sv.stop && !sv.hold && it != sv.queue.end() && (!sv.free_streams[0].empty() || !sv.free_streams[1].empty());) {
      Job& j = **it;
      if (sv.free_streams[j.cls].empty()) {  // its class's streams are all busy
        ++it;
        continue;
      }
      if (sv.used + j.footprint > sv.ctx->budget) {
        if (blocked || j.skips >= kMaxSkips) break;
        blocked = &j;
        ++it;
        continue;
      }
      if (blocked) ++blocked->skips;
      std::shared_ptr<Job> jp = *it;
      it = sv.queue.erase(it);
      j.stream = sv.free_streams[j.cls].back();
      sv.free_streams[j.cls].pop_back();
      sv.used += j.footprint;
      j.t_admit = now_s();
      // coalesce queued requests of the same geometry that also fit (each reserves its own
      // footprint, an upper bound of its share of the stacked run)
      const int64_t max_batch = sv.ctx->max_coalesce;
      for (auto k = sv.queue.begin(); k != sv.queue.end() && (int64_t)j.followers.size() + 1 < max_batch;) {
        Job& c = **k;
        if (same_geometry(j, c) && sv.used + c.footprint <= sv.ctx->budget) {
          sv.used += c.footprint;
          c.t_admit = j.t_admit;
          j.followers.push_back(*k);
          k = sv.queue.erase(k);
        } else {
          ++k;
        }
      }
      j.batched = 1 + (int)j.followers.size();
      for (auto& f : j.followers) f->batched = j.batched;
      lk.unlock();
      const int rc = launch(sv, j);
      lk.lock();
      if (rc != TACAW_OK) {
        finish(sv, j, rc);
        sv.cv_done.notify_all();
      } else {
        sv.active.push_back(jp);
      }
      it = sv.queue.begin();
      blocked = nullptr;
    }
  }
  // drain: requests still queued at shutdown are cancelled
  for (auto& jp : sv.queue) {
    jp->canceled = true;
    jp->status = TACAW_ECANCELED;
    sv.pinned.put(jp->pos_pinned);
    sv.pinned.put(jp->S_pinned);
    jp->pos_pinned = jp->S_pinned = nullptr;
  }
  sv.queue.clear();
  sv.cv_done.notify_all();
}

Serving* serving_of(tacaw_ctx* ctx, int* rc) {
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  if (ctx->serving) return ctx->serving;
  auto* sv = new Serving();
  sv->ctx = ctx;
  cudaSetDevice(ctx->device);
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  for (int cls = 0; cls < 2; ++cls)
    for (int64_t i = 0; i < ctx->serving_streams; ++i) {
      cudaStream_t s;
      if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, cls ? greatest : least) != cudaSuccess) {
        *rc = set_err(ctx, TACAW_ECUDA, "cannot create serving streams");
        for (cudaStream_t t : sv->all_streams) cudaStreamDestroy(t);
        delete sv;
        return nullptr;
      }
      sv->all_streams.push_back(s);
      sv->free_streams[cls].push_back(s);
    }
  sv->worker = std::thread(worker_loop, sv);
  ctx->serving = sv;
  return sv;
}

void fill(const Job& j, tacaw_result* out) {
  if (!out) return;
  out->status = j.status;
  out->batched = j.batched;
  out->footprint_bytes = j.footprint;
  out->t_submit = j.t_submit;
  out->t_admit = j.t_admit;
  out->t_done = j.t_done;
}

}  // namespace

void serving_shutdown(tacaw_ctx* ctx) {
  Serving* sv = ctx->serving;
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->kick = true;
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (cudaStream_t s : sv->all_streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  sv->pinned.clear();
  ctx->serving = nullptr;
  delete sv;
}

}  // namespace tacaw

using namespace tacaw;

extern "C" {

int tacaw_submit(tacaw_ctx* ctx, const tacaw_request* req, uint64_t* ticket) {
  if (!ctx || !req || !ticket) return TACAW_EINVAL;
  auto j = std::make_shared<Job>();
  int rc = TACAW_OK;
  Serving* sv = serving_of(ctx, &rc);
  if (!sv) return rc;
  PinnedPool& pool = sv->pinned;
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    tacaw_probe pr = req->probe;
    if (pr.n_probes == 0) {
      pr = tacaw_probe{};
      pr.n_probes = 1;
    }
    rc = check_run(ctx, &req->params, pr, req->pos, req->Z, req->n_atoms, req->n_frames, req->precision,
                   req->reduce, req->S_out, true);
    if (rc != TACAW_OK) return rc;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
    j->params = req->params;
    j->A = req->n_atoms;
    j->F = req->n_frames;
    j->precision = req->precision;
    j->reduce = req->reduce;
    const size_t nq = (size_t)req->params.nx * req->params.ny;
    j->out_elems = req->reduce == TACAW_REDUCE_NONE ? (size_t)pr.n_probes * j->F * nq : (size_t)pr.n_probes * j->F;
    if (pr.xy) j->probe_xy.assign(pr.xy, pr.xy + 2 * (size_t)pr.n_probes);
    j->probe = pr;
    j->probe.xy = pr.xy ? j->probe_xy.data() : nullptr;
    // inputs: host data is copied now; device data must stay valid until the request finishes
    cudaPointerAttributes a{};
    const auto on_device = [&](const void* p) {
      if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
    };
    if (j->A > 0) {
      if (on_device(req->pos)) {
        j->pos_dev = req->pos;
      } else {
        e = pool.get(sizeof(float) * j->F * j->A * 3, (void**)&j->pos_pinned);
        if (e != cudaSuccess) return cuda_err(ctx, e, "cudaMallocHost");
        std::memcpy(j->pos_pinned, req->pos, sizeof(float) * j->F * j->A * 3);
      }
      j->Z.resize(j->A);
      if (on_device(req->Z)) e = cudaMemcpy(j->Z.data(), req->Z, sizeof(int32_t) * j->A, cudaMemcpyDeviceToHost);
      else std::memcpy(j->Z.data(), req->Z, sizeof(int32_t) * j->A);
      if (e != cudaSuccess) {
        pool.put(j->pos_pinned);
        return cuda_err(ctx, e, "request species");
      }
      for (int64_t i = 0; i < j->A; ++i) {
        bool known = false;
        for (int32_t z : ctx->ffZ) known |= (z == j->Z[i]);
        if (!known) {
          pool.put(j->pos_pinned);
          return set_err(ctx, TACAW_EINVAL, "atom %lld has Z=%d, not in the form-factor table", (long long)i,
                         j->Z[i]);
        }
      }
    }
    j->S_user = req->S_out;
    j->S_host = !on_device(req->S_out);
    if (j->S_host) {
      e = pool.get(sizeof(float) * j->out_elems, (void**)&j->S_pinned);
      if (e != cudaSuccess) {
        pool.put(j->pos_pinned);
        return cuda_err(ctx, e, "cudaMallocHost");
      }
    }
    const double work = (double)pr.n_probes * j->F * j->params.n_slices * j->params.nx * j->params.ny;
    j->cls = work <= (double)ctx->serving_small_work ? 1 : 0;
    GeoCache* g;
    rc = get_geo(ctx, j->params, &g);
    if (rc == TACAW_OK) {
      j->footprint = run_footprint(ctx, j->params, pr.n_probes, j->F, j->A, j->precision, j->reduce, g);
      if (j->footprint > ctx->budget)
        rc = set_err(ctx, TACAW_ETOOBIG, "request needs %llu bytes, the budget is %llu",
                     (unsigned long long)j->footprint, (unsigned long long)ctx->budget);
    }
    if (rc != TACAW_OK) {
      pool.put(j->pos_pinned);
      pool.put(j->S_pinned);
      return rc;
    }
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    j->ticket = sv->next_ticket++;
    j->t_submit = now_s();
    sv->jobs[j->ticket] = j;
    sv->queue.push_back(j);
    sv->kick = true;
    *ticket = j->ticket;
  }
  sv->cv.notify_all();
  return TACAW_OK;
}

int tacaw_request_footprint(tacaw_ctx* ctx, const tacaw_request* req, uint64_t* bytes) {
  if (!ctx || !req || !bytes) return TACAW_EINVAL;
  std::lock_guard<std::recursive_mutex> lk(ctx->mu);
  tacaw_probe pr = req->probe;
  if (pr.n_probes == 0) {
    pr = tacaw_probe{};
    pr.n_probes = 1;
  }
  int rc = check_run(ctx, &req->params, pr, req->pos, req->Z, req->n_atoms, req->n_frames, req->precision,
                     req->reduce, req->S_out, false);
  if (rc != TACAW_OK) return rc;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  GeoCache* g;
  rc = get_geo(ctx, req->params, &g);
  if (rc != TACAW_OK) return rc;
  *bytes = run_footprint(ctx, req->params, pr.n_probes, req->n_frames, req->n_atoms, req->precision, req->reduce, g);
  if (*bytes > ctx->budget)
    return set_err(ctx, TACAW_ETOOBIG, "request needs %llu bytes, the budget is %llu", (unsigned long long)*bytes,
                   (unsigned long long)ctx->budget);
  return TACAW_OK;
}

int tacaw_poll(tacaw_ctx* ctx, uint64_t ticket, tacaw_result* out) {
  if (!ctx) return TACAW_EINVAL;
  Serving* sv = ctx->serving;
  if (!sv) return TACAW_ENOTFOUND;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return TACAW_ENOTFOUND;
  fill(*it->second, out);
  const int st = it->second->status;
  if (st != TACAW_PENDING) sv->jobs.erase(it);
  return st;
}

int tacaw_wait(tacaw_ctx* ctx, uint64_t ticket, double timeout_s, tacaw_result* out) {
  if (!ctx) return TACAW_EINVAL;
  Serving* sv = ctx->serving;
  if (!sv) return TACAW_ENOTFOUND;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return TACAW_ENOTFOUND;
  std::shared_ptr<Job> j = it->second;
  const double tmo = (timeout_s < 0 || timeout_s > 1e6) ? 1e6 : timeout_s;
  const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(tmo),
                                       [&] { return j->status != TACAW_PENDING; });
  fill(*j, out);
  if (!ok) return TACAW_ETIMEOUT;
  sv->jobs.erase(ticket);
  return j->status;
}

int tacaw_cancel(tacaw_ctx* ctx, uint64_t ticket) {
  if (!ctx) return TACAW_EINVAL;
  Serving* sv = ctx->serving;
  if (!sv) return TACAW_ENOTFOUND;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->jobs.find(ticket);
  if (it == sv->jobs.end()) return TACAW_ENOTFOUND;
  Job& j = *it->second;
  if (j.status != TACAW_PENDING) return TACAW_OK;
  j.canceled = true;
  for (auto q = sv->queue.begin(); q != sv->queue.end(); ++q)
    if ((*q)->ticket == ticket) {
      sv->queue.erase(q);
      j.status = TACAW_ECANCELED;
      j.t_done = now_s();
      sv->pinned.put(j.pos_pinned);
      sv->pinned.put(j.S_pinned);
      j.pos_pinned = j.S_pinned = nullptr;
      sv->cv_done.notify_all();
      break;
    }
  return TACAW_OK;
}

int tacaw_serving_hold(tacaw_ctx* ctx, int32_t hold) {
  if (!ctx) return TACAW_EINVAL;
  int rc = TACAW_OK;
  Serving* sv = serving_of(ctx, &rc);
  if (!sv) return rc;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->hold = hold != 0;
    sv->kick = true;
  }
  sv->cv.notify_all();
  return TACAW_OK;
}

int tacaw_serving_stats(tacaw_ctx* ctx, int64_t* queued, int64_t* active, uint64_t* used_bytes,
                        uint64_t* budget_bytes) {
  if (!ctx) return TACAW_EINVAL;
  Serving* sv = ctx->serving;
  if (budget_bytes) *budget_bytes = ctx->budget;
  if (!sv) {
    if (queued) *queued = 0;
    if (active) *active = 0;
    if (used_bytes) *used_bytes = 0;
    return TACAW_OK;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  if (queued) *queued = (int64_t)sv->queue.size();
  if (active) *active = (int64_t)sv->active.size();
  if (used_bytes) *used_bytes = sv->used;
  return TACAW_OK;
}

}  // extern "C"
