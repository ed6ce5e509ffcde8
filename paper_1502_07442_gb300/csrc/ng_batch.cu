// Batched independent simulations (no paper counterpart: the paper runs one
// simulation over MPI ranks; here many small simulations share one GPU).
//
// One batch step = one kick-drift-kick step (Sec. 2.1.1) of every simulation.
// Each simulation's sort, tree and PM stages run on one of several worker
// streams (fork/join inside one captured CUDA graph, so small simulations
// overlap on the device); the short-range walk of all simulations that share
// one law table (one row per distinct law of its members, whatever their
// species counts) is ONE persistent launch whose warps pull (simulation,
// group) items from a single work queue; the closing kick runs per
// simulation. The step is captured once and replayed.
#include <algorithm>
#include <array>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "ng_internal.cuh"

using namespace ng;

struct WalkClass {
  int D = 0;                         // the largest species count of the members
  std::vector<int> members;          // simulation indices
  std::vector<WalkDesc> h;           // host descriptors (kept alive for the graph)
  DevBuf d, pre;                     // device descriptors, group prefix + work counter
  // the class's law table: one row of ncut + 1 segments per distinct law of
  // its members (each member's descriptor maps its species pairs to rows)
  std::vector<std::vector<float>> laws;
  std::vector<float> htab;           // the rows, concatenated (uploaded to tab)
  int ncut = 0;
  double dr = 0;
  DevBuf tab;
};

struct ng_batch {
  std::vector<ng_ctx*> sims;
  cudaStream_t stream = nullptr;     // caller's stream (graph replays go here)
  cudaStream_t cap = nullptr;        // private stream the step is captured on
  std::vector<cudaStream_t> workers;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  std::vector<WalkClass> classes;
  std::vector<std::array<int8_t, kMaxD * kMaxD>> lawmap;   // per simulation: row of pair (s, t)
  cudaGraphExec_t exec = nullptr;
  std::vector<const void*> sig;      // pointers, sizes and dt the graph was captured for
  uint64_t gen = 0;
  uint64_t graph_launches = 0;       // kernels in one captured batch step
  uint64_t replay_launches = 0;      // kernels run by graph replays so far
  std::string err;
};

namespace {

// Worker streams of a batch step: the per-simulation stages are chains of
// small kernels, so more chains keep more SMs busy (batch64: 13.9 ms per
// step with 8 workers, 11.8 with 16, 11.3 with 32).
constexpr int kBatchWorkers = 32;

int bfail(ng_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  b->err = buf;
  return code;
}

// Propagate a member's failure message into the batch.
int from_sim(ng_batch* b, int i, int code) {
  if (code == NG_OK) return NG_OK;
  return bfail(b, code, "simulation %d: %s", i, ng_last_error(b->sims[i]));
}

// Segments per law of a batch class table (those of a D = 4 table), fewer
// when the first member's laws would not fit the table budget.
constexpr int kBatchSegments = 255;
constexpr size_t kClassTableBytes = 64 * 1024;

// A simulation joins a walk class when the cut-off, accumulation and segment
// spacing agree and the class table, with the member's laws not yet in it
// appended, stays within the budget; map receives the rows of the member's
// species pairs.
bool join_class(WalkClass& k, const ng_ctx* rep, const ng_ctx* c, int ncut, double dr,
                const std::vector<float>& rows, std::array<int8_t, kMaxD * kMaxD>& map) {
  if (c->p.accumulate_fp64 != rep->p.accumulate_fp64 || c->rcut != rep->rcut || ncut != k.ncut ||
      dr != k.dr || (c->p.table_size > 0 && c->p.table_size != ncut))
    return false;
  const size_t row = (size_t)(ncut + 1) * 2;
  std::vector<int> id(c->nlaws, -1);
  size_t added = 0;
  for (int u = 0; u < c->nlaws; ++u) {
    const float* r = rows.data() + (size_t)u * row;
    for (size_t v = 0; v < k.laws.size() && id[u] < 0; ++v)
      if (std::equal(r, r + row, k.laws[v].data())) id[u] = (int)v;
    if (id[u] < 0) ++added;
  }
  if ((k.laws.size() + added) * row * sizeof(float) > kClassTableBytes && !k.laws.empty()) return false;
  for (int u = 0; u < c->nlaws; ++u) {
    if (id[u] >= 0) continue;
    const float* r = rows.data() + (size_t)u * row;
    id[u] = (int)k.laws.size();
    k.laws.emplace_back(r, r + row);
    // a law repeated within this member maps to the row just added
    for (int w = u + 1; w < c->nlaws; ++w)
      if (id[w] < 0 && std::equal(r, r + row, rows.data() + (size_t)w * row)) id[w] = id[u];
  }
  map.fill(0);
  for (int s = 0; s < c->p.D; ++s)
    for (int t = 0; t < c->p.D; ++t) map[s * kMaxD + t] = (int8_t)id[c->tabid[s][t]];
  return true;
}

uint64_t alloc_gen(const ng_batch* b) {
  uint64_t g = 0;
  for (const ng_ctx* c : b->sims) g += c->alloc_gen;
  return g;
}

}  // namespace

extern "C" {

int ng_batch_create(ng_batch** out, int nsim, const ng_params* params, void* stream) {
  if (!out || nsim < 1 || !params) return NG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < nsim; ++i)
    if (params[i].pure_tree) return NG_EINVAL;   // batches run the group walk only
  ng_batch* b = new (std::nothrow) ng_batch();
  if (!b) return NG_ENOMEM;
  b->stream = (cudaStream_t)stream;
  for (int i = 0; i < nsim; ++i) {
    ng_ctx* c = nullptr;
    const int r = ng_create(&c, &params[i], stream);
    if (r != NG_OK) {
      ng_batch_destroy(b);
      return r;
    }
    b->sims.push_back(c);
  }
  const int nw = std::min(nsim, kBatchWorkers);
  for (int w = 0; w < nw; ++w) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      ng_batch_destroy(b);
      return NG_ECUDA;
    }
    b->workers.push_back(s);
    b->joins.push_back(e);
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    ng_batch_destroy(b);
    return NG_ECUDA;
  }
  // walk classes: simulations whose laws fit one table laid out for kMaxD
  // lists (largest species counts first, so each class's first member
  // defines its table); one persistent walk launch per class
  std::vector<int> order(nsim);
  for (int i = 0; i < nsim; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->sims[x]->p.D > b->sims[y]->p.D; });
  b->lawmap.resize(nsim);
  for (int i : order) {
    ng_ctx* c = b->sims[i];
    bool placed = false;
    for (WalkClass& k : b->classes) {
      const std::vector<float> rows = law_segments(c, k.ncut, k.dr);
      if (join_class(k, b->sims[k.members[0]], c, k.ncut, k.dr, rows, b->lawmap[i])) {
        k.members.push_back(i);
        placed = true;
        break;
      }
    }
    if (!placed) {
      // a new class, its segment count set by its first member's laws
      int ncut = c->p.table_size > 0 ? c->p.table_size : kBatchSegments;
      if (c->p.table_size <= 0)
        ncut = (int)std::min<size_t>(ncut, kClassTableBytes / (8 * (size_t)c->nlaws) - 1);
      b->classes.emplace_back();
      WalkClass& k = b->classes.back();
      k.D = c->p.D;
      k.ncut = ncut;
      k.dr = c->rcut / (ncut - 0.5);
      k.members.push_back(i);
      join_class(k, c, c, k.ncut, k.dr, law_segments(c, k.ncut, k.dr), b->lawmap[i]);
    }
  }
  for (WalkClass& k : b->classes) {
    std::sort(k.members.begin(), k.members.end());
    for (const std::vector<float>& r : k.laws) k.htab.insert(k.htab.end(), r.begin(), r.end());
    ng_ctx* rep = b->sims[k.members[0]];
    int r = ensure(rep, k.tab, k.htab.size() * sizeof(float));
    if (r == NG_OK &&
        cudaMemcpy(k.tab.p, k.htab.data(), k.htab.size() * sizeof(float), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      cudaGetLastError();
      r = NG_ECUDA;
    }
    if (r != NG_OK) {
      ng_batch_destroy(b);
      return r;
    }
  }
  *out = b;
  return NG_OK;
}

int ng_batch_destroy(ng_batch* b) {
  if (!b) return NG_OK;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (WalkClass& k : b->classes) {
    release(k.d);
    release(k.pre);
    release(k.tab);
  }
  for (cudaStream_t s : b->workers) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (ng_ctx* c : b->sims) ng_destroy(c);
  delete b;
  return NG_OK;
}

int ng_batch_size(const ng_batch* b) { return b ? (int)b->sims.size() : 0; }

int ng_batch_walk_launches(const ng_batch* b) { return b ? (int)b->classes.size() : 0; }

const char* ng_batch_last_error(const ng_batch* b) { return b ? b->err.c_str() : "no batch"; }

int ng_batch_launch_count(const ng_batch* b, uint64_t* out) {
  if (!b || !out) return NG_EINVAL;
  uint64_t s = b->replay_launches;
  for (const ng_ctx* c : b->sims) s += c->launches;
  *out = s;
  return NG_OK;
}

}  // extern "C"

namespace {

// One batch step on the current streams (eager or under capture). acc holds
// the acceleration at the current positions on entry and on exit.
int batch_step_once(ng_batch* b, const int64_t* n, double* const* pos, float* const* vel,
                    const uint8_t* const* type, const float* const* mass, float* const* acc,
                    double dt, cudaStream_t origin) {
  const int S = (int)b->sims.size();
  const int W = (int)b->workers.size();
  if (cudaEventRecord(b->fork, origin) != cudaSuccess) return bfail(b, NG_ECUDA, "fork record");
  for (int w = 0; w < W; ++w)
    if (cudaStreamWaitEvent(b->workers[w], b->fork, 0) != cudaSuccess)
      return bfail(b, NG_ECUDA, "fork wait");
  for (int i = 0; i < S; ++i) {
    ng_ctx* c = b->sims[i];
    cudaStream_t keep = c->stream;
    c->stream = b->workers[i % W];
    int r = launch_kick_drift(c, n[i], vel[i], acc[i], 0.5 * dt, 1, pos[i], dt);
    if (r == NG_OK) r = sort_bodies(c, n[i], pos[i], type[i], mass[i]);
    if (r == NG_OK) r = tree_stages(c);
    if (r == NG_OK) {
      if (c->p.pm_mesh > 0) r = pm_force(c, acc[i], false);
      else if (cudaMemsetAsync(acc[i], 0, 3 * n[i] * sizeof(float), c->stream) != cudaSuccess)
        r = fail(c, NG_ECUDA, "acc clear failed");
    }
    c->stream = keep;
    if (r != NG_OK) return from_sim(b, i, r);
  }
  for (int w = 0; w < W; ++w) {
    if (cudaEventRecord(b->joins[w], b->workers[w]) != cudaSuccess ||
        cudaStreamWaitEvent(origin, b->joins[w], 0) != cudaSuccess)
      return bfail(b, NG_ECUDA, "join failed");
  }
  // one persistent walk per class, accumulating into the long-range part
  for (WalkClass& k : b->classes) {
    ng_ctx* rep = b->sims[k.members[0]];
    cudaStream_t keep = rep->stream;
    rep->stream = origin;
    const int nd = (int)k.members.size();
    int r = NG_OK;
    if (cudaMemcpyAsync(k.d.p, k.h.data(), nd * sizeof(WalkDesc), cudaMemcpyHostToDevice,
                        origin) != cudaSuccess)
      r = fail(rep, NG_ECUDA, "descriptor copy failed");
    uint32_t* pre = as<uint32_t>(k.pre);
    int64_t groups = 0;
    for (int m : k.members) groups += walk_groups_hint(b->sims[m]);
    bool rel = false;   // some member uses the relative criterion
    for (const WalkDesc& h : k.h) rel = rel || h.aold != nullptr;
    WalkTable tab{as<float2>(k.tab), k.ncut, (int)(k.htab.size() / 2)};
    if (r == NG_OK)
      r = launch_walk_descs(rep, origin, as<WalkDesc>(k.d), nd, pre, pre + nd + 1, nullptr, groups,
                            rel, &tab, true);
    rep->stream = keep;
    if (r != NG_OK) return from_sim(b, k.members[0], r);
  }
  for (int i = 0; i < S; ++i) {
    ng_ctx* c = b->sims[i];
    cudaStream_t keep = c->stream;
    c->stream = origin;
    int r = update_aold(c, acc[i]);
    if (r == NG_OK) r = launch_kick(c, n[i], vel[i], acc[i], 0.5 * dt);
    c->stream = keep;
    if (r != NG_OK) return from_sim(b, i, r);
  }
  return NG_OK;
}

}  // namespace

extern "C" {

int ng_batch_step(ng_batch* b, const int64_t* n, double* const* pos, float* const* vel,
                  const uint8_t* const* type, const float* const* mass, float* const* acc,
                  int acc_valid, int nsteps, double dt) {
  if (!b) return NG_EINVAL;
  if (!n || !pos || !vel || !type || !mass || !acc) return bfail(b, NG_EINVAL, "NULL array");
  if (nsteps < 0) return bfail(b, NG_EINVAL, "nsteps < 0");
  const int S = (int)b->sims.size();
  for (int i = 0; i < S; ++i)
    if (n[i] < 1 || n[i] >= ((int64_t)1 << 31) || !pos[i] || !vel[i] || !type[i] || !mass[i] || !acc[i])
      return bfail(b, NG_EINVAL, "simulation %d: bad size or NULL array", i);
  // eager force at the start sizes every buffer of every simulation
  if (!acc_valid) {
    for (int i = 0; i < S; ++i) {
      ng_ctx* c = b->sims[i];
      c->stream = b->stream;
      int r = build_checked(c, n[i], pos[i], type[i], mass[i]);
      if (r == NG_OK) r = force_stages(c, acc[i]);
      if (r != NG_OK) return from_sim(b, i, r);
    }
  }
  if (nsteps == 0) {
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, NG_ECUDA, "sync failed");
    return NG_OK;
  }
  std::vector<const void*> sig;
  for (int i = 0; i < S; ++i) {
    sig.push_back((const void*)n[i]);
    sig.push_back(pos[i]);
    sig.push_back(vel[i]);
    sig.push_back(type[i]);
    sig.push_back(mass[i]);
    sig.push_back(acc[i]);
  }
  double dtv = dt;
  const void* dtp = nullptr;
  std::memcpy(&dtp, &dtv, sizeof(dtp));
  sig.push_back(dtp);
  int done = 0;
  const bool reuse = b->exec && sig == b->sig && b->gen == alloc_gen(b);
  if (!reuse) {
    // one eager step (sizing every buffer with synchronised checks), then capture
    for (int i = 0; i < S; ++i) {
      ng_ctx* c = b->sims[i];
      c->stream = b->stream;
      int r = launch_kick_drift(c, n[i], vel[i], acc[i], 0.5 * dt, 1, pos[i], dt);
      if (r == NG_OK) r = build_checked(c, n[i], pos[i], type[i], mass[i]);
      if (r == NG_OK) r = force_stages(c, acc[i]);
      if (r == NG_OK) r = launch_kick(c, n[i], vel[i], acc[i], 0.5 * dt);
      if (r == NG_OK && c->cap_nodes < c->nnodes + c->nnodes / 4 + 1024) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, NG_ECUDA, "sync");
        r = alloc_nodes(c, c->nnodes + c->nnodes / 4 + 1024);
      }
      if (r != NG_OK) return from_sim(b, i, r);
    }
    done = 1;
    for (WalkClass& k : b->classes) {
      k.h.resize(k.members.size());
      for (size_t j = 0; j < k.members.size(); ++j) {
        ng_ctx* c = b->sims[k.members[j]];
        fill_walk_desc_dr(c, acc[k.members[j]], c->p.pm_mesh > 0, k.dr, &k.h[j]);
        const std::array<int8_t, kMaxD * kMaxD>& m = b->lawmap[k.members[j]];
        for (int ss = 0; ss < kMaxD; ++ss)
          for (int tt = 0; tt < kMaxD; ++tt) k.h[j].tabid[ss][tt] = m[ss * kMaxD + tt];
      }
      ng_ctx* rep = b->sims[k.members[0]];
      int r = ensure(rep, k.d, k.h.size() * sizeof(WalkDesc));
      if (r == NG_OK) r = ensure(rep, k.pre, (k.h.size() + 2) * sizeof(uint32_t));
      if (r != NG_OK) return from_sim(b, k.members[0], r);
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, NG_ECUDA, "sync failed");
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    if (done < nsteps) {
      cudaGraph_t g = nullptr;
      if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, NG_ECUDA, "begin capture failed");
      }
      uint64_t before = 0;
      for (ng_ctx* c : b->sims) {
        before += c->launches;
        // captured trees stop two levels below the deepest one seen so far
        c->level_cap = std::min(kMaxLevel, c->depth_seen + kCapturedDepthMargin);
      }
      const int r = batch_step_once(b, n, pos, vel, type, mass, acc, dt, b->cap);
      uint64_t after = 0;
      for (ng_ctx* c : b->sims) {
        after += c->launches;
        c->level_cap = kMaxLevel;
      }
      b->graph_launches = after - before;
      const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
      cudaGetLastError();
      if (r != NG_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      if (e != cudaSuccess) return bfail(b, NG_ECUDA, "capture failed: %s", cudaGetErrorString(e));
      const cudaError_t ei = cudaGraphInstantiate(&b->exec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return bfail(b, NG_ECUDA, "instantiate: %s", cudaGetErrorString(ei));
      b->sig = sig;
      b->gen = alloc_gen(b);
    }
  }
  for (int i = 0; i < S; ++i)
    if (cudaMemsetAsync(b->sims[i]->status.p, 0, sizeof(uint32_t), b->stream) != cudaSuccess)
      return bfail(b, NG_ECUDA, "flag clear failed");
  for (int s = done; s < nsteps; ++s) {
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, NG_ECUDA, "graph launch failed");
    }
    b->replay_launches += b->graph_launches;
  }
  bool deeper = false;
  for (int i = 0; i < S; ++i) {
    ng_ctx* c = b->sims[i];
    c->stream = b->stream;
    uint32_t st[ST_COUNT];
    int r = read_status(c, st);
    if (r == NG_OK && (st[ST_FLAGS] & SF_DEPTH)) deeper = true;
    if (r == NG_OK) r = check_flags(c, st[ST_FLAGS]);
    if (r != NG_OK) return from_sim(b, i, r);
    c->built = true;
  }
  // a replayed tree outgrew its level cap (still correct): capture deeper next call
  if (deeper && b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return NG_OK;
}

}  // extern "C"
