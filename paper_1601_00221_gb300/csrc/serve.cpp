// serve.cpp -- continuously batched evaluation service (gp_server_*).
//
// One server owns: the device copies of every registered run's cases, a
// pool of CUDA streams, a FIFO of submitted requests and a worker thread.
// The worker admits the head of the queue when an in-flight slot and enough
// of the memory budget are free, together with the queued requests of other
// runs of the same kind (float or Boolean) that fit beside it: the programs
// of all of them -- uneven in number, length, case count and inputs -- run in
// one kernel launch (gp_eval_segments, one segment per request, each on its
// own run's resident cases and split by its own run's chunk, so a request's
// result does not depend on what shares its launch).  A head that does not
// fit the free memory may be passed by smaller requests that do, a bounded
// number of times.  The worker copies the programs to the device, launches
// on the next stream, copies the results back and enqueues a host function
// after them.  That host function (run by the CUDA runtime when the stream
// reaches it) copies each request's results into the caller's buffer,
// stamps the completion time and wakes waiters.  No kernel waits on the host
// and the host never spins on the device.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/gpeval.h"
#include "status.h"

namespace {

using Clock = std::chrono::steady_clock;

enum ReqState { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3, Q_CANCELLED = 4 };

struct Run {
  int32_t kind;
  int32_t n_inputs;
  int64_t n_cases;
  int64_t n_units;  // cases (float) or words (Boolean)
  void* d_cases = nullptr;
  void* d_targets = nullptr;
  gp_config cfg;    // fixed per run: the split of the case range depends on n_cases only
};

struct Request {
  uint64_t id;
  int32_t run;
  int32_t n_progs;
  int64_t gpop;
  std::vector<uint32_t> words;
  std::vector<int64_t> offsets;
  std::vector<int32_t> lengths;
  void* result;  // caller's buffer
  int state = Q_QUEUED;
  int status = GP_OK;
  int bypassed = 0;  // times a later request was admitted first
  double t_submit = 0, t_admit = 0, t_done = 0;
};

struct PinnedBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct Launch {
  std::vector<Request*> reqs;
  int32_t run;      // the head's run (its kind decides the interpreter)
  bool segments;    // one segment per request (gp_eval_segments), else one population
  int stream_idx;
  size_t bytes;  // budget charge
  int64_t n_progs;
  PinnedBuf h_in, h_out;
  void* d_in = nullptr;   // words | offsets | lengths
  void* d_out = nullptr;  // results
  size_t in_bytes = 0, out_bytes = 0;
  struct gp_server* srv;
};

}  // namespace

struct gp_server {
  gp_server_opts opts;
  gp_config launch_cfg[2];  // float, Boolean launches
  int device = 0;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  std::deque<Run> runs;  // deque: references stay valid while runs are added
  std::mutex mu;
  std::condition_variable cv_work;  // worker wake-up
  std::condition_variable cv_done;  // request completions
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<Launch*> finished;    // completed launches whose memory the worker frees
  std::vector<PinnedBuf> pinned_pool;
  int inflight = 0;
  int64_t mem_in_use = 0;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  Clock::time_point t0;
  // statistics
  int64_t submitted = 0, completed = 0, failed = 0, cancelled = 0, launches = 0, gpop_done = 0;
  std::vector<double> latencies;
  double first_admit = -1, last_done = -1;

  double now_us() const {
    return std::chrono::duration<double, std::micro>(Clock::now() - t0).count();
  }
};

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// pinned host buffers are recycled: cudaMallocHost is far too slow per request
PinnedBuf take_pinned(gp_server* s, size_t bytes) {  // called with s->mu held
  size_t best = (size_t)-1;
  int bi = -1;
  for (int i = 0; i < (int)s->pinned_pool.size(); ++i)
    if (s->pinned_pool[i].cap >= bytes && s->pinned_pool[i].cap < best) {
      best = s->pinned_pool[i].cap;
      bi = i;
    }
  if (bi >= 0) {
    PinnedBuf b = s->pinned_pool[bi];
    s->pinned_pool.erase(s->pinned_pool.begin() + bi);
    return b;
  }
  return PinnedBuf{};
}

void CUDART_CB on_launch_done(void* arg) {
  // runs on a CUDA runtime thread: no CUDA calls here
  Launch* L = static_cast<Launch*>(arg);
  gp_server* s = L->srv;
  std::lock_guard<std::mutex> lk(s->mu);
  const double t = s->now_us();
  const size_t elem = (s->runs[L->run].kind == GP_RUN_FLOAT) ? sizeof(double) : sizeof(uint64_t);
  size_t off = 0;
  for (Request* r : L->reqs) {
    memcpy(r->result, static_cast<char*>(L->h_out.p) + off, elem * (size_t)r->n_progs);
    off += elem * (size_t)r->n_progs;
    r->state = Q_DONE;
    r->t_done = t;
    s->completed += 1;
    s->gpop_done += r->gpop;
    s->latencies.push_back(r->t_done - r->t_submit);
  }
  s->last_done = t;
  s->inflight -= 1;
  s->mem_in_use -= (int64_t)L->bytes;
  s->finished.push_back(L);
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

void fail_launch(gp_server* s, Launch* L, int status) {  // called with s->mu held
  for (Request* r : L->reqs) {
    r->state = Q_FAILED;
    r->status = status;
    r->t_done = s->now_us();
    s->failed += 1;
  }
  s->inflight -= 1;
  s->mem_in_use -= (int64_t)L->bytes;
  s->finished.push_back(L);
  s->cv_done.notify_all();
}

// Issues one launch (copies, kernel, result copy, completion callback).
// Called without the lock; returns a gp_status.
int issue(gp_server* s, Launch* L) {
  const Run& run = s->runs[L->run];
  cudaStream_t st = s->streams[L->stream_idx];
  int64_t total_words = 0;
  for (Request* r : L->reqs) total_words += (int64_t)r->words.size();
  const size_t w_bytes = round_up(sizeof(uint32_t) * (size_t)total_words, 16);
  const size_t o_bytes = round_up(sizeof(int64_t) * (size_t)L->n_progs, 16);
  const size_t l_bytes = round_up(sizeof(int32_t) * (size_t)L->n_progs, 16);
  L->in_bytes = w_bytes + o_bytes + l_bytes;
  L->out_bytes = round_up(8 * (size_t)L->n_progs, 16);
  cudaError_t e;
  if (!L->h_in.p) {
    e = cudaMallocHost(&L->h_in.p, L->in_bytes);
    if (e != cudaSuccess) return GP_ERR_OOM;
    L->h_in.cap = L->in_bytes;
  }
  if (!L->h_out.p) {
    e = cudaMallocHost(&L->h_out.p, L->out_bytes);
    if (e != cudaSuccess) return GP_ERR_OOM;
    L->h_out.cap = L->out_bytes;
  }
  // concatenate the requests' programs; offsets move by the words before
  char* hin = static_cast<char*>(L->h_in.p);
  uint32_t* hw = reinterpret_cast<uint32_t*>(hin);
  int64_t* ho = reinterpret_cast<int64_t*>(hin + w_bytes);
  int32_t* hl = reinterpret_cast<int32_t*>(hin + w_bytes + o_bytes);
  int64_t wpos = 0, ppos = 0;
  for (Request* r : L->reqs) {
    memcpy(hw + wpos, r->words.data(), sizeof(uint32_t) * r->words.size());
    for (int32_t p = 0; p < r->n_progs; ++p) {
      ho[ppos + p] = r->offsets[p] + wpos;
      hl[ppos + p] = r->lengths[p];
    }
    wpos += (int64_t)r->words.size();
    ppos += r->n_progs;
  }
  e = cudaMallocAsync(&L->d_in, L->in_bytes, st);
  if (e != cudaSuccess) return GP_ERR_OOM;
  e = cudaMallocAsync(&L->d_out, L->out_bytes, st);
  if (e != cudaSuccess) return GP_ERR_OOM;
  e = cudaMemcpyAsync(L->d_in, L->h_in.p, L->in_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return GP_ERR_CUDA;
  char* din = static_cast<char*>(L->d_in);
  const uint32_t* dw = reinterpret_cast<const uint32_t*>(din);
  const int64_t* dofs = reinterpret_cast<const int64_t*>(din + w_bytes);
  const int32_t* dlen = reinterpret_cast<const int32_t*>(din + w_bytes + o_bytes);
  int rc;
  // a Boolean request alone in its launch takes the library's own choice of
  // kernel for its case set (one program per lane, a warp per program, or
  // blocks per program); hit counts are exact whichever kernel runs, so its
  // result is the one it would have in a merged launch
  const bool bool_alone = run.kind == GP_RUN_BOOL && L->reqs.size() == 1;
  if (L->segments && !bool_alone) {
    // one segment per request, each on its own run's cases and chunk
    std::vector<gp_segment> segs;
    int32_t pbeg = 0;
    for (Request* r : L->reqs) {
      const Run& rr = s->runs[r->run];
      gp_segment g;
      g.prog_begin = pbeg;
      g.n_progs = r->n_progs;
      g.cases = rr.d_cases;
      g.n_inputs = rr.n_inputs;
      g.chunk = rr.cfg.chunk_cases;
      g.n_cases = rr.n_cases;
      g.targets = rr.d_targets;
      g.out = static_cast<char*>(L->d_out) + 8 * (size_t)pbeg;
      segs.push_back(g);
      pbeg += r->n_progs;
    }
    gp_config lc = s->launch_cfg[run.kind == GP_RUN_FLOAT ? 0 : 1];
    rc = gp_eval_segments(dw, dofs, dlen, segs.data(), (int32_t)segs.size(), run.kind, &lc, (gp_stream_t)st);
  } else if (run.kind == GP_RUN_FLOAT)
    rc = gp_eval_population_ex(dw, dofs, dlen, (int32_t)L->n_progs, static_cast<const float*>(run.d_cases),
                               run.n_inputs, run.n_cases, static_cast<const float*>(run.d_targets),
                               static_cast<double*>(L->d_out), nullptr, &run.cfg, (gp_stream_t)st);
  else {
    gp_config bc = run.cfg;
    bc.variant = GP_VARIANT_AUTO;
    bc.k = 0;
    bc.block = 0;
    bc.chunk_cases = 0;
    rc = gp_eval_population_bool_ex(dw, dofs, dlen, (int32_t)L->n_progs,
                                    static_cast<const uint32_t*>(run.d_cases), run.n_inputs,
                                    run.n_cases, static_cast<const uint32_t*>(run.d_targets),
                                    static_cast<uint64_t*>(L->d_out), nullptr, &bc, (gp_stream_t)st);
  }
  if (rc != GP_OK) return rc;
  e = cudaMemcpyAsync(L->h_out.p, L->d_out, 8 * (size_t)L->n_progs, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return GP_ERR_CUDA;
  e = cudaLaunchHostFunc(st, on_launch_done, L);
  if (e != cudaSuccess) return GP_ERR_CUDA;
  return GP_OK;
}

void release_launch(gp_server* s, Launch* L) {  // worker thread, lock not held
  cudaStream_t st = s->streams[L->stream_idx];
  if (L->d_in) cudaFreeAsync(L->d_in, st);
  if (L->d_out) cudaFreeAsync(L->d_out, st);
  std::lock_guard<std::mutex> lk(s->mu);
  if (L->h_in.p) s->pinned_pool.push_back(L->h_in);
  if (L->h_out.p) s->pinned_pool.push_back(L->h_out);
  delete L;
}

// Device bytes a request charges against the budget when admitted: its
// share of the launch's buffers (programs, offsets, lengths, results) and of
// the workspace (partial sums of its run's chunks, counters, block order).
size_t request_bytes(const Run& run, const Request* r) {
  const int64_t chunk = std::max<int64_t>(1, run.cfg.chunk_cases);
  const int64_t chunks = std::max<int64_t>(1, (run.n_units + chunk - 1) / chunk);
  return round_up(4 * r->words.size(), 16) + round_up(24 * (size_t)r->n_progs, 16) +
         16 * (size_t)(chunks > 1 ? r->n_progs * chunks : 0) + 4096;
}

// a run whose requests can share a launch with other runs' requests
bool segmentable(const gp_server* s, const Run& run) {
  return run.kind == GP_RUN_BOOL || s->launch_cfg[0].variant == GP_VARIANT_REGISTER;
}

// Takes `group` out of the queue and issues it as one launch (lock held on
// entry and exit; released around the CUDA calls).
void admit(gp_server* s, std::unique_lock<std::mutex>& lk, const std::vector<Request*>& group,
           size_t bytes, bool segments) {
  std::deque<Request*> rest;
  for (Request* r : s->queue)
    if (std::find(group.begin(), group.end(), r) == group.end() && r->state != Q_CANCELLED) rest.push_back(r);
  s->queue.swap(rest);
  int64_t words = 0, progs = 0;
  for (Request* r : group) {
    words += (int64_t)r->words.size();
    progs += r->n_progs;
  }
  Launch* L = new Launch();
  L->reqs = group;
  L->run = group.front()->run;
  L->segments = segments;
  L->srv = s;
  L->bytes = bytes;
  L->n_progs = progs;
  L->stream_idx = s->next_stream;
  s->next_stream = (s->next_stream + 1) % (int)s->streams.size();
  const double t = s->now_us();
  for (Request* r : group) {
    r->state = Q_RUNNING;
    r->t_admit = t;
  }
  if (s->first_admit < 0) s->first_admit = t;
  s->inflight += 1;
  s->mem_in_use += (int64_t)bytes;
  s->launches += 1;
  const size_t in_need = round_up(4 * (size_t)words, 16) + round_up(8 * (size_t)progs, 16) +
                         round_up(4 * (size_t)progs, 16);
  L->h_in = take_pinned(s, in_need);
  L->h_out = take_pinned(s, round_up(8 * (size_t)progs, 16));
  lk.unlock();
  int rc = issue(s, L);
  lk.lock();
  if (rc != GP_OK) fail_launch(s, L, rc);
}

// How many times a queued head may be passed by smaller requests that fit
// the free memory while it does not.
constexpr int kMaxBypass = 8;

// The group a request `lead` heads: `lead`, then the queued requests after
// it that may share its launch -- the same run's requests (any variant), or
// with segment launches any run of the same kind -- up to max_merge
// programs, GP_MAX_SEGMENTS requests and `room` bytes.  Returns its bytes.
size_t gather(gp_server* s, size_t from, std::vector<Request*>& group, int64_t room, bool* segments) {
  Request* lead = s->queue[from];
  const Run& run = s->runs[lead->run];
  *segments = segmentable(s, run);
  group.assign(1, lead);
  size_t bytes = request_bytes(run, lead);
  int64_t progs = lead->n_progs;
  for (size_t i = from + 1; i < s->queue.size() && (int)group.size() < GP_MAX_SEGMENTS; ++i) {
    Request* r = s->queue[i];
    if (r->state == Q_CANCELLED) continue;
    const Run& rr = s->runs[r->run];
    const bool joins = *segments ? (rr.kind == run.kind && segmentable(s, rr)) : r->run == lead->run;
    if (!joins) continue;
    const size_t b = request_bytes(rr, r);
    if (progs + r->n_progs > s->opts.max_merge || (int64_t)(bytes + b) > room) continue;
    group.push_back(r);
    bytes += b;
    progs += r->n_progs;
  }
  return bytes;
}

void worker_main(gp_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // free what completed
    if (!s->finished.empty()) {
      std::vector<Launch*> done;
      done.swap(s->finished);
      lk.unlock();
      for (Launch* L : done) release_launch(s, L);
      lk.lock();
      continue;
    }
    if (s->stop && s->queue.empty() && s->inflight == 0) break;
    // Admit the head of the queue with what may share its launch.  When the
    // head does not fit the free memory (and work is in flight, which will
    // free some), a later request that fits may go first, at most kMaxBypass
    // times per head.
    bool admitted = false;
    while (!s->queue.empty() && s->inflight < s->opts.max_inflight) {
      Request* head = s->queue.front();
      if (head->state == Q_CANCELLED) {
        s->queue.pop_front();
        continue;
      }
      const int64_t room = s->opts.memory_budget - s->mem_in_use;
      std::vector<Request*> group;
      bool segments = false;
      const size_t need = request_bytes(s->runs[head->run], head);
      if ((int64_t)need <= room || s->inflight == 0) {
        const size_t bytes = gather(s, 0, group, std::max<int64_t>(room, (int64_t)need), &segments);
        admit(s, lk, group, bytes, segments);
        admitted = true;
        continue;
      }
      if (head->bypassed >= kMaxBypass) break;  // the head waits for memory
      size_t lead = 0;
      for (size_t i = 1; i < s->queue.size() && !lead; ++i) {
        Request* r = s->queue[i];
        if (r->state != Q_CANCELLED && (int64_t)request_bytes(s->runs[r->run], r) <= room) lead = i;
      }
      if (!lead) break;
      const size_t bytes = gather(s, lead, group, room, &segments);
      head->bypassed += 1;
      admit(s, lk, group, bytes, segments);
      admitted = true;
    }
    if (!admitted) s->cv_work.wait_for(lk, std::chrono::microseconds(200));
  }
}

// Cases (float) or words (Boolean) per block for a run: a function of the
// run's size and configuration only, never of what is merged with it.
int64_t choose_run_chunk(int kind, const gp_config& c) {
  const int64_t per_pass = (int64_t)c.k * c.block;
  const int64_t target = (kind == GP_RUN_FLOAT) ? 32768 : 8192;
  return ((target + per_pass - 1) / per_pass) * per_pass;
}

}  // namespace

extern "C" int gp_server_create(const gp_server_opts* opts, gp_server** out) {
  gp_clear_error();
  if (!out) return gp_fail(GP_ERR_INVALID_ARG, "null server pointer");
  std::unique_ptr<gp_server> s(new gp_server());
  gp_server_opts o{};
  if (opts) o = *opts;
  if (o.n_streams <= 0) o.n_streams = 4;
  if (o.max_inflight <= 0) o.max_inflight = 16;
  if (o.max_queued <= 0) o.max_queued = 65536;
  if (o.max_merge <= 0) o.max_merge = 65536;
  if (o.memory_budget <= 0) o.memory_budget = (int64_t)1 << 30;
  gp_config def;
  gp_get_config(&def);
  if (!o.config.variant) o.config.variant = def.variant;
  if (!o.config.k) o.config.k = def.k;
  if (!o.config.block) o.config.block = def.block;
  if (!o.config.fitness) o.config.fitness = def.fitness;
  if (!o.config.tile_inputs) o.config.tile_inputs = def.tile_inputs;
  o.config.chunk_cases = 0;
  s->opts = o;
  // Float requests of different runs share a launch when the configuration
  // is the register variant (the several-populations kernels); Boolean ones
  // always do, with K = 4 and 64-thread blocks (the staged input tile of
  // many inputs bounds the blocks per multiprocessor), and a Boolean request
  // alone in its launch takes the library's automatic choice
  s->launch_cfg[0] = o.config;
  s->launch_cfg[1] = o.config;
  s->launch_cfg[1].variant = GP_VARIANT_REGISTER;
  s->launch_cfg[1].k = 4;
  s->launch_cfg[1].block = 64;
  s->launch_cfg[1].tile_inputs = 0;
  s->launch_cfg[1].stack_registers = 0;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e != cudaSuccess) return gp_fail(GP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  for (int i = 0; i < o.n_streams; ++i) {
    cudaStream_t st;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      return gp_fail(GP_ERR_CUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
    }
    s->streams.push_back(st);
  }
  s->t0 = Clock::now();
  gp_server* raw = s.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return GP_OK;
}

extern "C" int gp_server_register_run(gp_server* s, int32_t kind, const void* cases, int32_t n_inputs,
                                      int64_t n_cases, const void* targets, int32_t* run_id) {
  gp_clear_error();
  if (!s || !run_id) return gp_fail(GP_ERR_INVALID_ARG, "null argument");
  if (kind != GP_RUN_FLOAT && kind != GP_RUN_BOOL) return gp_fail(GP_ERR_INVALID_ARG, "unknown run kind %d", kind);
  if (n_inputs < 0 || n_cases <= 0) return gp_fail(GP_ERR_INVALID_ARG, "bad run sizes");
  if ((n_inputs > 0 && !cases) || !targets) return gp_fail(GP_ERR_INVALID_ARG, "null case data");
  Run r;
  r.kind = kind;
  r.n_inputs = n_inputs;
  r.n_cases = n_cases;
  r.n_units = (kind == GP_RUN_FLOAT) ? n_cases : (n_cases + 31) / 32;
  const size_t unit = 4;
  const size_t cbytes = unit * (size_t)r.n_units * (size_t)std::max(n_inputs, 1);
  const size_t tbytes = unit * (size_t)r.n_units;
  cudaSetDevice(s->device);
  cudaError_t e = cudaMalloc(&r.d_cases, cbytes);
  if (e == cudaSuccess) e = cudaMalloc(&r.d_targets, tbytes);
  if (e == cudaSuccess && n_inputs > 0)
    e = cudaMemcpy(r.d_cases, cases, unit * (size_t)r.n_units * (size_t)n_inputs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(r.d_targets, targets, tbytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (r.d_cases) cudaFree(r.d_cases);
    if (r.d_targets) cudaFree(r.d_targets);
    return gp_fail(e == cudaErrorMemoryAllocation ? GP_ERR_OOM : GP_ERR_CUDA, "registering run: %s",
                   cudaGetErrorString(e));
  }
  r.cfg = s->launch_cfg[kind == GP_RUN_FLOAT ? 0 : 1];
  r.cfg.chunk_cases = (int32_t)choose_run_chunk(kind, r.cfg);
  std::lock_guard<std::mutex> lk(s->mu);
  s->runs.push_back(r);
  *run_id = (int32_t)s->runs.size() - 1;
  return GP_OK;
}

extern "C" int gp_server_submit(gp_server* s, int32_t run_id, const uint32_t* programs,
                                const int64_t* offsets, const int32_t* lengths, int32_t n_progs,
                                int64_t n_nodes, void* result, uint64_t* req_id) {
  gp_clear_error();
  if (!s || !req_id || !result) return gp_fail(GP_ERR_INVALID_ARG, "null argument");
  if (n_progs <= 0 || !programs || !offsets || !lengths) return gp_fail(GP_ERR_INVALID_ARG, "empty request");
  std::unique_ptr<Request> r(new Request());
  int64_t max_end = 0;
  for (int32_t p = 0; p < n_progs; ++p) {
    if (offsets[p] < 0 || lengths[p] < 4 || (offsets[p] & 3))
      return gp_fail(GP_ERR_INVALID_ARG, "program %d has a bad offset or length", p);
    max_end = std::max<int64_t>(max_end, offsets[p] + lengths[p]);
  }
  r->words.assign(programs, programs + max_end);
  r->words.resize((size_t)round_up((size_t)max_end, 4), 0u);  // the next request's words stay 16-byte aligned
  r->offsets.assign(offsets, offsets + n_progs);
  r->lengths.assign(lengths, lengths + n_progs);
  r->n_progs = n_progs;
  r->result = result;
  std::unique_lock<std::mutex> lk(s->mu);
  if (run_id < 0 || run_id >= (int32_t)s->runs.size()) return gp_fail(GP_ERR_INVALID_ARG, "unknown run %d", run_id);
  const Run& run = s->runs[run_id];
  if ((int64_t)request_bytes(run, r.get()) > s->opts.memory_budget)
    return gp_fail(GP_ERR_OOM, "request needs more than the server's memory budget");
  if ((int64_t)s->queue.size() >= s->opts.max_queued) return gp_fail(GP_ERR_BUSY, "queue full");
  r->run = run_id;
  r->gpop = n_nodes * run.n_cases;
  r->id = s->next_id++;
  r->t_submit = s->now_us();
  Request* raw = r.get();
  s->reqs.emplace(raw->id, std::move(r));
  s->queue.push_back(raw);
  s->submitted += 1;
  *req_id = raw->id;
  s->cv_work.notify_one();
  return GP_OK;
}

static void fill_info(const Request* r, gp_request_info* info) {
  if (!info) return;
  info->status = r->state == Q_DONE ? GP_OK : r->state == Q_CANCELLED ? GP_ERR_CANCELLED : r->status;
  info->n_progs = r->n_progs;
  info->gpop = r->gpop;
  info->t_submit_us = r->t_submit;
  info->t_admit_us = r->t_admit;
  info->t_done_us = r->t_done;
}

extern "C" int gp_server_poll(gp_server* s, uint64_t req_id, gp_request_info* info) {
  gp_clear_error();
  if (!s) return gp_fail(GP_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return gp_fail(GP_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
  const Request* r = it->second.get();
  if (r->state == Q_QUEUED || r->state == Q_RUNNING) return GP_ERR_BUSY;
  fill_info(r, info);
  return GP_OK;
}

extern "C" int gp_server_wait(gp_server* s, uint64_t req_id, int64_t timeout_us, gp_request_info* info) {
  gp_clear_error();
  if (!s) return gp_fail(GP_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return gp_fail(GP_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
  const Request* r = it->second.get();
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
  while (r->state == Q_QUEUED || r->state == Q_RUNNING) {
    if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
        (r->state == Q_QUEUED || r->state == Q_RUNNING))
      return gp_fail(GP_ERR_TIMEOUT, "request %llu not finished after %lld us",
                     (unsigned long long)req_id, (long long)timeout_us);
  }
  fill_info(r, info);
  return GP_OK;
}

extern "C" int gp_server_cancel(gp_server* s, uint64_t req_id) {
  gp_clear_error();
  if (!s) return gp_fail(GP_ERR_INVALID_ARG, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return gp_fail(GP_ERR_INVALID_ARG, "unknown request %llu", (unsigned long long)req_id);
  Request* r = it->second.get();
  if (r->state != Q_QUEUED) return gp_fail(GP_ERR_BUSY, "request %llu already admitted or finished", (unsigned long long)req_id);
  r->state = Q_CANCELLED;
  r->t_done = s->now_us();
  s->cancelled += 1;
  s->cv_done.notify_all();
  return GP_OK;
}

extern "C" int gp_server_get_stats(gp_server* s, gp_server_stats* st) {
  gp_clear_error();
  if (!s || !st) return gp_fail(GP_ERR_INVALID_ARG, "null argument");
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    lat = s->latencies;
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->failed = s->failed;
    st->cancelled = s->cancelled;
    st->launches = s->launches;
    st->gpop_completed = s->gpop_done;
    st->busy_s = (s->first_admit >= 0 && s->last_done >= s->first_admit) ? (s->last_done - s->first_admit) * 1e-6 : 0.0;
  }
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) {
    if (lat.empty()) return 0.0;
    size_t i = (size_t)std::min<double>((double)lat.size() - 1, q * (double)(lat.size() - 1) + 0.5);
    return lat[i];
  };
  st->p50_latency_us = pct(0.50);
  st->p99_latency_us = pct(0.99);
  st->max_latency_us = lat.empty() ? 0.0 : lat.back();
  st->gpop_per_s = st->busy_s > 0 ? (double)st->gpop_completed / st->busy_s : 0.0;
  return GP_OK;
}

extern "C" int gp_server_destroy(gp_server* s) {
  gp_clear_error();
  if (!s) return GP_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (Request* r : s->queue)
      if (r->state == Q_QUEUED) {
        r->state = Q_CANCELLED;
        s->cancelled += 1;
      }
    s->queue.clear();
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (Launch* L : s->finished) delete L;
  for (PinnedBuf& b : s->pinned_pool) cudaFreeHost(b.p);
  for (Run& r : s->runs) {
    if (r.d_cases) cudaFree(r.d_cases);
    if (r.d_targets) cudaFree(r.d_targets);
  }
  delete s;
  return GP_OK;
}
