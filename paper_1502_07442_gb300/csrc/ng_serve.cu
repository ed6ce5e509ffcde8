// Serving runtime (no paper counterpart): a stream of independent force
// evaluations and short integrations, each a full ngravs solve.
//
// Every slot has its own host thread that enqueues its request's kernels, so
// the launch work of concurrent requests is spread over host cores (a 10-step
// request is ~1600 launches) while the polling thread only admits and reaps.
//
// Continuous batching: requests wait in a FIFO host queue and are admitted
// as soon as a slot is free and the device memory the slots hold stays
// within the byte budget. Every slot owns a context (reconfigured per
// request, buffers and cuFFT plans kept), a stream and the request's device
// arrays; an admitted request runs entirely asynchronously on its slot's
// stream (copy in, tree + PM + walk, the KDK steps, copy out, event), so the
// work of all admitted requests overlaps on the GPU. Completion is detected
// by event queries; the status words copied out with the result reveal a
// tree-capacity overflow, after which the request is rerun with more room.
// The host loop never blocks on the device except in bounded waits.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>

#include "ng_internal.cuh"

using namespace ng;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Slot {
  ng_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t first_tree = nullptr;   // the request's first tree is built
  DevBuf pos, vel, acc, type, mass;
  uint32_t* h_status = nullptr;       // pinned copy of the status words
  int64_t req = -1;                   // request in flight (-1: free)
  size_t bytes = 0;                   // device bytes this slot holds (high-water estimate)
  int retries = 0;
  // launch thread: the poller hands it a request, it enqueues the kernels
  std::thread worker;
  std::mutex m;
  std::condition_variable cv;
  bool job = false, quit = false;
  std::atomic<int> launched{0};       // 0 idle, 1 enqueueing, 2 enqueued, 3 launch failed
  int launch_rc = NG_OK;
  struct Req* cur = nullptr;          // request handed to the launch thread
};

struct Req {
  ng_request r;
  ng_result* out;
  int state;                          // 0 queued, 1 running, 2 done, 3 cancelled/failed
};
// (requests live on the heap: the launch threads hold pointers to them while
// the polling thread keeps submitting)

// Device bytes a request needs in a slot: particle arrays, sort buffers, tree
// buffers for a capacity of `nodes` nodes, PM meshes.
size_t request_bytes_nodes(const ng_request& q, size_t nodes) {
  const size_t n = (size_t)q.n, D = (size_t)q.params.D, N = (size_t)q.params.pm_mesh;
  const size_t body = 53 + 100;
  const size_t node = 74 + 52 * D;
  const size_t pm = N ? D * N * N * (N + 2) * 4 * 2 + D * N * N * N * 4 : 0;
  return n * body + nodes * node + pm + (1 << 20);
}

// The admission estimate: a node capacity of n + 1024 (the slot's first try).
size_t request_bytes(const ng_request& q) { return request_bytes_nodes(q, (size_t)q.n + 1024); }

}  // namespace

struct ng_server {
  std::vector<std::unique_ptr<Slot>> slots;
  std::deque<int64_t> queue;
  std::vector<std::unique_ptr<Req>> reqs;
  size_t budget = 0;
  size_t peak_held = 0;        // largest sum of slot bytes seen after an admission or a regrow
  int64_t node_retries = 0;    // requests rerun with a larger tree capacity
  int64_t reconfigs = 0;       // slot contexts reconfigured for new parameters
  int64_t completed = 0;
  std::string err;
};

namespace {

int sfail(ng_server* s, int code, const char* msg) {
  s->err = msg;
  return code;
}

// Message of the last failed ng_serve_create on this thread.
thread_local std::string g_serve_create_err;

// Size the slot for its request on the admitting thread while the slot is
// idle: reconfigure the context if the parameters differ, grow the slot's
// particle arrays and every buffer and cuFFT plan of the context. The slot's
// launch thread then only enqueues work: no device allocation, free or plan
// creation ever runs in a launch thread while other slots' work is in flight.
int prepare_slot(ng_server* s, Slot& sl, const ng_request& r) {
  ng_ctx* c = sl.ctx;
  c->stream = sl.stream;
  const int64_t n = r.n;
  ng_params want = r.params;
  normalize_params(&want);   // compare like with like: the context holds normalised params
  if (std::memcmp(&c->p, &want, sizeof(ng_params)) != 0 || c->h_tab.empty()) {
    NG_TRY(ctx_configure(c, &r.params));
    s->reconfigs++;
  }
  NG_TRY(ensure(c, sl.pos, n * 24));
  NG_TRY(ensure(c, sl.vel, n * 12));
  NG_TRY(ensure(c, sl.acc, n * 12));
  NG_TRY(ensure(c, sl.type, n));
  NG_TRY(ensure(c, sl.mass, n * 4));
  return reserve(c, n);
}

// Restores the full tree depth of a slot's context on every exit path.
struct LevelCapReset {
  ng_ctx* c;
  ~LevelCapReset() { c->level_cap = kMaxLevel; }
};

// Seconds a launch thread waits for its request's first tree.
constexpr double kFirstTreeWait = 120.0;

// Enqueue the whole request on the slot's stream (launch thread; the slot
// was prepared by prepare_slot). For an integration the thread waits (bounded)
// for the first tree only, while the first force runs: the trees of the steps
// then stop two levels below its depth (cells at the cap stay leaves, a valid
// tree; see SF_DEPTH), which saves the launches of the empty deeper levels.
int launch_request(ng_server* s, Slot& sl, Req& q) {
  ng_ctx* c = sl.ctx;
  c->stream = sl.stream;
  LevelCapReset reset_cap{c};
  const uint64_t gen = c->alloc_gen;
  const ng_request& r = q.r;
  const int64_t n = r.n;
  double* pos = as<double>(sl.pos);
  float* vel = as<float>(sl.vel);
  float* acc = as<float>(sl.acc);
  uint8_t* type = as<uint8_t>(sl.type);
  float* mass = as<float>(sl.mass);
  NG_CUDA(c, cudaMemcpyAsync(pos, r.pos, n * 24, cudaMemcpyHostToDevice, sl.stream));
  NG_CUDA(c, cudaMemcpyAsync(type, r.type, n, cudaMemcpyHostToDevice, sl.stream));
  NG_CUDA(c, cudaMemcpyAsync(mass, r.mass, n * 4, cudaMemcpyHostToDevice, sl.stream));
  if (r.kind == NG_REQ_STEPS) {
    if (r.vel) NG_CUDA(c, cudaMemcpyAsync(vel, r.vel, n * 12, cudaMemcpyHostToDevice, sl.stream));
    else NG_CUDA(c, cudaMemsetAsync(vel, 0, n * 12, sl.stream));
  }
  NG_CUDA(c, cudaMemsetAsync(c->status.p, 0, ST_COUNT * 4, sl.stream));
  c->n = n;
  c->aold_n = -1;  // requests are independent: no previous acceleration
  // force at the input positions
  NG_TRY(sort_bodies(c, n, pos, type, mass));
  NG_TRY(tree_stages(c));
  const bool steps = r.kind == NG_REQ_STEPS && r.nsteps > 0;
  if (steps) {
    // the first tree's level counts (read back before the final status copy
    // reuses the buffer)
    NG_CUDA(c, cudaMemcpyAsync(sl.h_status, c->status.p, ST_COUNT * 4, cudaMemcpyDeviceToHost,
                               sl.stream));
    NG_CUDA(c, cudaEventRecord(sl.first_tree, sl.stream));
  }
  NG_TRY(force_stages(c, acc));
  if (r.kind == NG_REQ_STEPS) {
    if (steps) {
      const double t0 = now_s();
      cudaError_t e;
      while ((e = cudaEventQuery(sl.first_tree)) == cudaErrorNotReady) {
        if (now_s() - t0 > kFirstTreeWait) return fail(c, NG_ETIMEOUT, "first tree not built in time");
        std::this_thread::sleep_for(std::chrono::microseconds(20));
      }
      NG_CUDA(c, e);
      int depth = 0;
      for (int l = 0; l <= kMaxLevel; ++l)
        if (sl.h_status[ST_LEVELS + kMaxLevel + 2 + l] > 0) depth = l;
      c->level_cap = std::min(kMaxLevel, depth + kCapturedDepthMargin);
    }
    // a step's closing kick goes with the next step's opening kick and drift
    for (int st = 0; st < r.nsteps; ++st) {
      NG_TRY(launch_kick_drift(c, n, vel, acc, 0.5 * r.dt, st == 0 ? 1 : 2, pos, r.dt));
      NG_TRY(sort_bodies(c, n, pos, type, mass));
      NG_TRY(tree_stages(c));
      NG_TRY(force_stages(c, acc));
    }
    if (r.nsteps > 0) NG_TRY(launch_kick(c, n, vel, acc, 0.5 * r.dt));
    if (r.pos_out) NG_CUDA(c, cudaMemcpyAsync(r.pos_out, pos, n * 24, cudaMemcpyDeviceToHost, sl.stream));
    if (r.vel_out) NG_CUDA(c, cudaMemcpyAsync(r.vel_out, vel, n * 12, cudaMemcpyDeviceToHost, sl.stream));
  }
  if (r.acc_out) NG_CUDA(c, cudaMemcpyAsync(r.acc_out, acc, n * 12, cudaMemcpyDeviceToHost, sl.stream));
  NG_CUDA(c, cudaMemcpyAsync(sl.h_status, c->status.p, ST_COUNT * 4, cudaMemcpyDeviceToHost, sl.stream));
  NG_CUDA(c, cudaEventRecord(sl.done, sl.stream));
  if (c->alloc_gen != gen) return fail(c, NG_ESTATE, "a launch thread grew a device buffer");
  (void)s;
  return NG_OK;
}

size_t held_bytes(const ng_server* s) {
  size_t t = 0;
  for (const auto& sl : s->slots) t += sl->bytes;
  return t;
}

// Hand the slot's request to its launch thread.
void hand_over(Slot& sl, Req* q) {
  {
    std::lock_guard<std::mutex> g(sl.m);
    sl.cur = q;
    sl.launched.store(1);
    sl.job = true;
  }
  sl.cv.notify_one();
}

void worker_loop(ng_server* s, Slot* sl);

// Admit queued requests (FIFO) while a slot is free and the budget holds.
int admit(ng_server* s) {
  while (!s->queue.empty()) {
    const int64_t id = s->queue.front();
    Req& q = *s->reqs[id];
    if (q.state != 0) {
      s->queue.pop_front();
      continue;
    }
    const size_t need = request_bytes(q.r);
    int pick = -1;
    for (size_t k = 0; k < s->slots.size(); ++k) {
      Slot& sl = *s->slots[k];
      if (sl.req >= 0) continue;
      const size_t after = held_bytes(s) - sl.bytes + std::max(sl.bytes, need);
      if (after <= s->budget) {
        pick = (int)k;
        break;
      }
    }
    if (pick < 0) return NG_OK;           // wait for a slot or for memory
    Slot& sl = *s->slots[pick];
    s->queue.pop_front();
    sl.bytes = std::max(sl.bytes, need);
    s->peak_held = std::max(s->peak_held, held_bytes(s));
    q.out->t_admit = now_s();
    const int rc = prepare_slot(s, sl, q.r);
    if (rc != NG_OK) {
      q.state = 3;
      q.out->status = rc;
      q.out->t_done = now_s();
      if (s->err.empty()) s->err = "request " + std::to_string(id) + ": " + sl.ctx->err;
      s->completed++;
      continue;
    }
    sl.req = id;
    sl.retries = 0;
    q.state = 1;
    hand_over(sl, &q);
  }
  return NG_OK;
}

void worker_loop(ng_server* s, Slot* sl) {
  for (;;) {
    {
      std::unique_lock<std::mutex> g(sl->m);
      sl->cv.wait(g, [&] { return sl->job || sl->quit; });
      if (sl->quit) return;
      sl->job = false;
    }
    Req& q = *sl->cur;
    const int rc = launch_request(s, *sl, q);
    sl->launch_rc = rc;
    if (rc != NG_OK) {
      // the slot's stream may hold part of the request: let it drain
      cudaStreamSynchronize(sl->stream);
      cudaGetLastError();
    }
    sl->launched.store(rc == NG_OK ? 2 : 3);
  }
}

// Collect finished requests; returns the number completed by this call.
int reap(ng_server* s) {
  int got = 0;
  for (auto& slp : s->slots) {
    Slot& sl = *slp;
    if (sl.req < 0) continue;
    const int st = sl.launched.load();
    if (st == 1) continue;               // still enqueueing
    Req& q = *s->reqs[sl.req];
    if (st == 3) {
      q.state = 3;
      q.out->status = sl.launch_rc;
      if (s->err.empty()) s->err = "request " + std::to_string(sl.req) + ": " + sl.ctx->err;
      q.out->t_done = now_s();
      sl.req = -1;
      sl.launched.store(0);
      s->completed++;
      got++;
      continue;
    }
    const cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady) continue;
    if (e != cudaSuccess) {
      cudaGetLastError();
      q.out->status = NG_ECUDA;
      sl.ctx->err = std::string("completion event: ") + cudaGetErrorString(e);
    } else if ((sl.h_status[ST_FLAGS] & SF_NODE_OVERFLOW) && sl.retries < 4) {
      // rerun with room for the node count the build reported, if the slot's
      // larger holding still fits the budget beside the other slots
      ng_ctx* c = sl.ctx;
      const int64_t need = (int64_t)sl.h_status[ST_NODES_NEEDED];
      const int64_t cap = std::max<int64_t>(2 * need, 2 * c->cap_nodes);
      const size_t grown = std::max(sl.bytes, request_bytes_nodes(q.r, (size_t)cap));
      if (held_bytes(s) - sl.bytes + grown > s->budget) {
        q.out->status = NG_ENOMEM;
        c->err = "tree capacity for the request exceeds the byte budget";
      } else if (alloc_nodes(c, cap) == NG_OK) {
        sl.bytes = grown;
        s->peak_held = std::max(s->peak_held, held_bytes(s));
        sl.retries++;
        s->node_retries++;
        hand_over(sl, &q);               // rerun on the slot's thread
        continue;
      } else {
        q.out->status = NG_ENOMEM;
      }
    } else {
      q.out->status = sl.h_status[ST_FLAGS] ? check_flags(sl.ctx, sl.h_status[ST_FLAGS]) : NG_OK;
    }
    q.state = q.out->status == NG_OK ? 2 : 3;
    if (q.out->status != NG_OK && s->err.empty())
      s->err = "request " + std::to_string(sl.req) + ": " + sl.ctx->err;
    q.out->t_done = now_s();
    sl.req = -1;
    sl.launched.store(0);
    s->completed++;
    got++;
  }
  return got;
}

}  // namespace

extern "C" {

int ng_serve_create(ng_server** out, int slots, size_t hbm_budget) {
  if (!out || slots < 1 || slots > 256 || hbm_budget == 0) return NG_EINVAL;
  *out = nullptr;
  ng_server* s = new (std::nothrow) ng_server();
  if (!s) return NG_ENOMEM;
  s->budget = hbm_budget;
  ng_params p{};
  p.D = 1;
  p.G[0][0] = 1.0;
  p.eps = 1e-3;
  p.box = 1.0;
  p.asmth = 0.05;
  p.rcut_over_rs = 4.5;
  p.theta = 0.5;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int k = 0; k < slots; ++k) {
    s->slots.emplace_back(new Slot());
    Slot& sl = *s->slots.back();
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.first_tree, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&sl.h_status, ST_COUNT * 4, cudaHostAllocDefault);
    int rc = e == cudaSuccess ? NG_OK : NG_ECUDA;
    if (e != cudaSuccess) {
      g_serve_create_err = std::string("slot ") + std::to_string(k) + ": " + cudaGetErrorString(e);
      cudaGetLastError();
    } else {
      rc = ng_create(&sl.ctx, &p, sl.stream);
      if (rc != NG_OK)
        g_serve_create_err = std::string("slot ") + std::to_string(k) + ": " + ng_last_error(nullptr);
    }
    if (rc != NG_OK) {
      ng_serve_destroy(s);
      return rc;
    }
    Slot* slp = &sl;
    sl.worker = std::thread([s, slp, dev] {
      cudaSetDevice(dev);
      worker_loop(s, slp);
    });
  }
  *out = s;
  return NG_OK;
}

int ng_serve_destroy(ng_server* s) {
  if (!s) return NG_OK;
  for (auto& slp : s->slots) {
    Slot& sl = *slp;
    if (sl.worker.joinable()) {
      // let an enqueueing request finish, then stop the thread
      while (sl.launched.load() == 1) std::this_thread::sleep_for(std::chrono::microseconds(50));
      {
        std::lock_guard<std::mutex> g(sl.m);
        sl.quit = true;
      }
      sl.cv.notify_one();
      sl.worker.join();
    }
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.ctx) {
      release(sl.pos);
      release(sl.vel);
      release(sl.acc);
      release(sl.type);
      release(sl.mass);
      ng_destroy(sl.ctx);
    }
    if (sl.h_status) cudaFreeHost(sl.h_status);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.first_tree) cudaEventDestroy(sl.first_tree);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
  return NG_OK;
}

int ng_serve_submit(ng_server* s, const ng_request* r, ng_result* out, int64_t* id) {
  if (!s || !r || !out) return NG_EINVAL;
  std::memset(out, 0, sizeof(*out));
  out->t_submit = now_s();
  if (r->n < 1 || r->n >= ((int64_t)1 << 31) || !r->pos || !r->type || !r->mass ||
      (r->kind != NG_REQ_FORCE && r->kind != NG_REQ_STEPS) ||
      (r->kind == NG_REQ_STEPS && (r->nsteps < 0 || r->nsteps > 100000)))
    return sfail(s, NG_EINVAL, "malformed request (n, arrays, kind or nsteps)");
  ng_ctx probe;   // host-only validation, no device work
  if (validate(&probe, &r->params) != NG_OK) return sfail(s, NG_EINVAL, probe.err.c_str());
  if (request_bytes(*r) > s->budget)
    return sfail(s, NG_EBUSY, "request larger than the whole device byte budget");
  s->reqs.emplace_back(new Req{*r, out, 0});
  const int64_t k = (int64_t)s->reqs.size() - 1;
  s->queue.push_back(k);
  out->status = 1;                    // pending
  if (id) *id = k;
  return NG_OK;
}

int ng_serve_cancel(ng_server* s, int64_t id) {
  if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return NG_EINVAL;
  Req& q = *s->reqs[id];
  if (q.state != 0) return NG_ESTATE;   // admitted work is not interrupted
  q.state = 3;
  q.out->status = NG_ESTATE;
  q.out->t_done = now_s();
  s->completed++;
  return NG_OK;
}

int ng_serve_poll(ng_server* s, int* ncompleted) {
  if (!s) return NG_EINVAL;
  const int got = reap(s);
  admit(s);
  if (ncompleted) *ncompleted = got;
  return NG_OK;
}

int ng_serve_pending(const ng_server* s) {
  if (!s) return 0;
  return (int)((int64_t)s->reqs.size() - s->completed);
}

int ng_serve_wait(ng_server* s, double timeout_s) {
  if (!s) return NG_EINVAL;
  const double t0 = now_s();
  while (ng_serve_pending(s) > 0) {
    ng_serve_poll(s, nullptr);
    if (ng_serve_pending(s) == 0) break;
    if (now_s() - t0 > timeout_s) return sfail(s, NG_ETIMEOUT, "wait timed out");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  return NG_OK;
}

int ng_serve(ng_server* s, const ng_request* reqs, ng_result* res, int nreq,
             const double* arrival_s, double timeout_s) {
  if (!s || !reqs || !res || nreq < 0) return NG_EINVAL;
  const double t0 = now_s();
  int next = 0;
  while (next < nreq || ng_serve_pending(s) > 0) {
    const double t = now_s() - t0;
    while (next < nreq && (!arrival_s || arrival_s[next] <= t)) {
      const int rc = ng_serve_submit(s, &reqs[next], &res[next], nullptr);
      if (rc != NG_OK) {
        res[next].status = rc;
        res[next].t_done = now_s();
      }
      if (arrival_s) res[next].t_submit = t0 + arrival_s[next];
      ++next;
    }
    int got = 0;
    ng_serve_poll(s, &got);
    if (now_s() - t0 > timeout_s) return sfail(s, NG_ETIMEOUT, "trace timed out");
    if (!got) std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  return NG_OK;
}

const char* ng_serve_last_error(const ng_server* s) {
  return s ? s->err.c_str() : g_serve_create_err.c_str();
}

size_t ng_serve_request_bytes(const ng_request* r) { return r ? request_bytes(*r) : 0; }

int ng_serve_stats(const ng_server* s, size_t* held_bytes_out, size_t* peak_held_bytes,
                   int64_t* node_retries, int64_t* reconfigs) {
  if (!s) return NG_EINVAL;
  if (held_bytes_out) *held_bytes_out = held_bytes(s);
  if (peak_held_bytes) *peak_held_bytes = s->peak_held;
  if (node_retries) *node_retries = s->node_retries;
  if (reconfigs) *reconfigs = s->reconfigs;
  return NG_OK;
}

}  // extern "C"
