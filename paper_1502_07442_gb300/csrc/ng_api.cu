// C ABI of the ngravs library: validation, host-built short-range tables,
// the pipeline entry points and the kick-drift-kick step (Sec. 2.1.1).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "ng_internal.cuh"

namespace ng {

int fail(ng_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return code;
}

int ensure(ng_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return NG_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, NG_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  b.p = p;
  b.bytes = bytes;
  if (c) c->alloc_gen++;
  return NG_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// ------------------------------------------------------ short-range laws

// Short-range law tables of the walk. Segment k (k < ncut) of a law is the
// minimax line of T over [(k - 1/2) dr, (k + 1/2) dr] (segment 0 over
// [0, dr/2]) for a locally quadratic T: the chord raised by half its
// deviation at the segment's middle. With t = rho/dr - k it is c0 + t c1,
// stored as {c0 - k c1, c1}; entry ncut is zero (beyond the cut-off, which
// sits at rho = (ncut - 1/2) dr = r_cut). The table depends on the law, r_s
// and r_cut only, not on the softening.
//
// Rows: one row of ncut + 1 float2 segments per distinct law of the context
// (c->tabid[s][t] numbers the law of passive species s and active species
// t). Batch walks read these rows, each lane the row of its own pair, so a
// class table holds each law once: a batch of Newtonian simulations needs
// one row whatever their species counts.
std::vector<float> law_segments(const ng_ctx* c, int ncut, double dr) {
  const ng_params& p = c->p;
  const int D = p.D;
  std::vector<float> h((size_t)c->nlaws * (ncut + 1) * 2, 0.f);
  for (int u = 0; u < c->nlaws && !p.pure_tree; ++u) {
    int si = 0, ti = 0;
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j)
        if (c->tabid[i][j] == u) si = i, ti = j;
    const int kind = p.law[si][ti];
    const bool yk = kind == NG_YUKAWA || kind == NG_YUKAWA_PURE;
    const double ya = yk ? p.yuk_a[si][ti] : 0.0, yl = yk ? p.yuk_l[si][ti] : 0.0;
    float* t = h.data() + (size_t)u * (ncut + 1) * 2;
    auto T = [&](double rho) { return short_law_factor(kind, ya, yl, c->rs, rho); };
    {
      const double lo = T(0.0), hi = T(0.5 * dr);
      t[0] = (float)(lo + 0.5 * (T(0.25 * dr) - 0.5 * (lo + hi)));   // value at t = 0
      t[1] = (float)(2.0 * (hi - lo));
    }
    for (int k = 1; k < ncut; ++k) {
      const double lo = T((k - 0.5) * dr), hi = T((k + 0.5) * dr);
      const double c0 = 0.25 * (lo + hi) + 0.5 * T(k * dr);
      // stored shifted: the walk evaluates (c0 - k c1) + (rho / dr) c1
      t[2 * k] = (float)(c0 - k * (hi - lo));
      t[2 * k + 1] = (float)(hi - lo);
    }
  }
  return h;
}

// Layout of a single simulation's table (walk_tab_pad): one block per active
// species t of the walk's lists, rows k of walk_tab_pad(D) float2 entries,
// entry s of the row holding the law of the pair (passive s, active t). A
// list of species t is evaluated by all lanes at once, each lane with its own
// passive species s and segment k; entry (k, s) lies in the bank pair
// (k * pad + s) mod 16, so lanes of different species never meet in a bank
// (the 2^24 D = 4 walk: 66.9 ms, against 69.9 ms reading one row per law).
std::vector<float> walk_table(const ng_ctx* c, int ncut, double dr) {
  const int D = c->p.D, pad = walk_tab_pad(D);
  const std::vector<float> seg = law_segments(c, ncut, dr);
  std::vector<float> h((size_t)D * (ncut + 1) * pad * 2, 0.f);
  for (int tt = 0; tt < D; ++tt)
    for (int k = 0; k <= ncut; ++k)
      for (int ss = 0; ss < D; ++ss) {
        const float* g = seg.data() + ((size_t)c->tabid[ss][tt] * (ncut + 1) + k) * 2;
        float* o = h.data() + (((size_t)tt * (ncut + 1) + k) * pad + ss) * 2;
        o[0] = g[0];
        o[1] = g[1];
      }
  return h;
}

// Segments per law: as many as 32 KB hold for a D x D block of laws up to
// four species, 64 KB for five or six (4096 for D = 1, 1023 for D = 2, 255
// for D = 3 or 4, 169 for D = 5 or 6). Fewer segments put a warp's lookups on
// fewer distinct entries (fewer bank conflicts): the 2^24 D = 4 walk takes
// 66.2 / 65.9 / 65.2 / 64.9 / 64.4 ms with 511 / 383 / 255 / 191 / 127, while
// the largest deviation from T grows 2.1e-6 / 3.7e-6 / 8.4e-6 / 1.5e-5 /
// 3.4e-5 (of T(0) = 1 for the Newtonian law); 255 stays below the 1.9e-5 of
// the six-species default.
int walk_table_entries(int D, int table_size) {
  if (table_size > 0) return table_size;
  const int pad = D <= 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8;
  const size_t budget = D <= 4 ? 32 * 1024 : 64 * 1024;
  return (int)std::min<size_t>(4096, budget / (sizeof(float) * 2 * D * pad) - 1);
}

int build_tables(ng_ctx* c) {
  const ng_params& p = c->p;
  const int D = p.D;
  struct Law { int kind; double a, l; };
  std::vector<Law> laws;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      const bool yk = p.law[i][j] == NG_YUKAWA || p.law[i][j] == NG_YUKAWA_PURE;
      Law w{p.law[i][j], yk ? p.yuk_a[i][j] : 0.0, yk ? p.yuk_l[i][j] : 0.0};
      int id = -1;
      for (size_t u = 0; u < laws.size(); ++u)
        if (laws[u].kind == w.kind && laws[u].a == w.a && laws[u].l == w.l) id = (int)u;
      if (id < 0) {
        id = (int)laws.size();
        laws.push_back(w);
      }
      c->tabid[i][j] = (int8_t)id;
    }
  c->nlaws = (int)laws.size();
  const int ncut = walk_table_entries(D, p.table_size);
  if (ncut < 16) return fail(c, NG_EINVAL, "table_size %d too small", ncut);
  c->ncut = ncut;
  // pure tree mode evaluates the laws directly: the table is kept (zero) only
  // so that every context has one
  c->dr_phys = p.pure_tree ? 1.0 : c->rcut / (ncut - 0.5);
  // separations in table units must stay below 2^22 for the float-bit index
  if (std::sqrt(3.0) * c->L / c->dr_phys > 4.0e6)
    return fail(c, NG_EINVAL, "box too large relative to the table spacing (box/dr = %.3g)",
                c->L / c->dr_phys);
  std::vector<float> h = walk_table(c, ncut, c->dr_phys);
  c->h_tab = h;
  NG_TRY(ensure(c, c->d_tab, h.size() * sizeof(float)));
  // upload through the context's pinned staging copy: wait until the stream
  // has consumed the previous contents, then copy without a pageable stall
  NG_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->h_tab_pinned_bytes < h.size() * sizeof(float)) {
    if (c->h_tab_pinned) cudaFreeHost(c->h_tab_pinned);
    c->h_tab_pinned = nullptr;
    c->h_tab_pinned_bytes = 0;
    NG_CUDA(c, cudaHostAlloc(&c->h_tab_pinned, h.size() * sizeof(float), cudaHostAllocDefault));
    c->h_tab_pinned_bytes = h.size() * sizeof(float);
  }
  std::memcpy(c->h_tab_pinned, h.data(), h.size() * sizeof(float));
  NG_CUDA(c, cudaMemcpyAsync(c->d_tab.p, c->h_tab_pinned, h.size() * sizeof(float),
                             cudaMemcpyHostToDevice, c->stream));
  c->lattice_grid = 0;
  if (p.pure_tree == 2) {
    std::vector<int> kinds;
    std::vector<double> as, ls;
    for (const Law& w : laws) {
      kinds.push_back(w.kind);
      as.push_back(w.a);
      ls.push_back(w.l);
    }
    NG_TRY(build_lattice(c, (int)laws.size(), kinds.data(), as.data(), ls.data()));
  }
  return NG_OK;
}

// ---------------------------------------------------------------- KDK

__global__ void k_kick(int64_t m, float* __restrict__ vel, const float* __restrict__ acc, float h) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    vel[i] = fmaf(acc[i], h, vel[i]);
}


// Per element: nkick kicks v += a h (each rounded as k_kick), then the FP64
// drift x += v dt with the periodic wrap (in a power-of-two box, x in [+0, L)
// wraps to itself, decided on the bits). One launch for the opening kick and
// drift of a step, or (nkick = 2) for the closing kick of a step with the
// opening kick and drift of the next.
__global__ void k_kick_drift(int64_t m, float* __restrict__ vel, const float* __restrict__ acc,
                             float h, int nkick, double* __restrict__ pos, double dt, double L,
                             double invL, bool pow2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float a = acc[i];
    float v = fmaf(a, h, vel[i]);
    if (nkick == 2) v = fmaf(a, h, v);
    vel[i] = v;
    double x = fma((double)v, dt, pos[i]);
    const long long b = __double_as_longlong(x);
    // the wrap is the rare case: a branch keeps its FP64 floor (and the
    // division of a box that is not a power of two) off the common path
    if (!(pow2 && b >= 0 && b < __double_as_longlong(L))) x -= L * floor(pow2 ? x * invL : x / L);
    pos[i] = x;
  }
}

int launch_kick_drift(ng_ctx* c, int64_t n, float* vel, const float* acc, double h, int nkick,
                      double* pos, double dt) {
  k_kick_drift<<<work_grid(c, 3 * n, 8), 256, 0, c->stream>>>(3 * n, vel, acc, (float)h, nkick, pos,
                                                          dt, c->L, 1.0 / c->L, box_is_pow2(c->L));
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

int launch_kick(ng_ctx* c, int64_t n, float* vel, const float* acc, double h) {
  k_kick<<<work_grid(c, 3 * n, 8), 256, 0, c->stream>>>(3 * n, vel, acc, (float)h);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}


// ------------------------------------------- relative opening criterion

double coupling_max(const ng_ctx* c) {
  double g = 0.0;
  for (int i = 0; i < c->p.D; ++i)
    for (int j = 0; j < c->p.D; ++j) g = std::max(g, c->p.G[i][j]);
  return g > 0.0 ? g : 1.0;
}

bool relative_active(const ng_ctx* c) {
  return c->p.opening == NG_OPEN_RELATIVE && c->n > 0 && c->aold_n == c->n;
}

// |a| per body in FP32, each operation rounded on its own: sqrt((x x + y y) + z z)
__global__ void k_amag(int64_t n, const float* __restrict__ acc, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = acc[i], y = acc[n + i], z = acc[2 * n + i];
    out[i] = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z)));
  }
}

static int set_aold(ng_ctx* c, int64_t n, const float* acc) {
  NG_TRY(ensure(c, c->aold, (size_t)n * sizeof(float)));
  k_amag<<<work_grid(c, n, 8), 256, 0, c->stream>>>(n, acc, as<float>(c->aold));
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  c->aold_n = n;
  return NG_OK;
}

int update_aold(ng_ctx* c, const float* acc) {
  if (c->p.opening != NG_OPEN_RELATIVE) return NG_OK;
  return set_aold(c, c->n, acc);
}

// ------------------------------------------------------------ pipeline

static size_t node_bytes(int D) {
  return 1 + 8 + 4 + 4 + 4 + 1 + 4 + (size_t)D * 32 + (size_t)D * 4 + 16 * 3 + (size_t)D * 16;
}

int alloc_nodes(ng_ctx* c, int64_t cap) {
  const int D = c->p.D;
  NG_TRY(ensure(c, c->n_level, cap));
  NG_TRY(ensure(c, c->n_prefix, cap * 8));
  NG_TRY(ensure(c, c->n_first, cap * 4));
  NG_TRY(ensure(c, c->n_count, cap * 4));
  NG_TRY(ensure(c, c->n_child, cap * 4));
  NG_TRY(ensure(c, c->n_nchild, cap));
  NG_TRY(ensure(c, c->n_tmp, cap * 4));
  NG_TRY(ensure(c, c->n_m64, cap * D * 32));
  NG_TRY(ensure(c, c->n_cnt, cap * D * 4));
  NG_TRY(ensure(c, c->n_geo, cap * 16));
  NG_TRY(ensure(c, c->n_com, cap * 16));
  NG_TRY(ensure(c, c->n_link, cap * 16));
  NG_TRY(ensure(c, c->n_mono, cap * D * 16));
  NG_TRY(ensure(c, c->mono_bins, (3 * kMonoBins + 1) * sizeof(uint32_t)));
  c->cap_nodes = cap;
  (void)node_bytes;
  return NG_OK;
}

int alloc_bodies(ng_ctx* c, int64_t n) {
  NG_TRY(ensure(c, c->body, n * 16));
  NG_TRY(ensure(c, c->bleaf, n * 4));
  NG_TRY(ensure(c, c->groups, n * 8));
  NG_TRY(ensure(c, c->status, ST_COUNT * 4));
  NG_TRY(ensure(c, c->counter, 8));
  return NG_OK;
}

// Every device buffer and cuFFT plan that one force evaluation (and the KDK
// steps of ng_step's stages) of n bodies needs, so that the stages that
// follow allocate nothing.
int reserve(ng_ctx* c, int64_t n) {
  NG_TRY(alloc_bodies(c, n));
  NG_TRY(alloc_nodes(c, std::max<int64_t>(c->cap_nodes, n + 1024)));
  NG_TRY(reserve_sort(c, n));
  NG_TRY(ensure(c, c->gsize, (size_t)n * sizeof(uint32_t)));
  NG_TRY(ensure(c, c->grank, (size_t)n * sizeof(uint32_t)));
  NG_TRY(ensure(c, c->walk_desc, sizeof(WalkDesc)));
  NG_TRY(ensure(c, c->walk_prefix, 4 * sizeof(uint32_t)));
  if (c->p.opening == NG_OPEN_RELATIVE) NG_TRY(ensure(c, c->aold, (size_t)n * sizeof(float)));
  if (c->p.pm_mesh > 0 && !c->pm_stream) {
    if (cudaStreamCreateWithFlags(&c->pm_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, NG_ECUDA, "PM stream creation failed");
    }
  }
  return pm_reserve(c);
}

// Everything after the sort; no host synchronisation.
int tree_stages(ng_ctx* c) {
  NG_TRY(build_octree(c));
  NG_TRY(reduce_monopoles(c));
  NG_TRY(build_groups(c));
  NG_TRY(type_order(c));
  return NG_OK;
}

int read_status(ng_ctx* c, uint32_t* st) {
  NG_CUDA(c, cudaMemcpyAsync(st, c->status.p, ST_COUNT * 4, cudaMemcpyDeviceToHost, c->stream));
  NG_CUDA(c, cudaStreamSynchronize(c->stream));
  return NG_OK;
}

int check_flags(ng_ctx* c, uint32_t flags) {
  flags &= ~(uint32_t)SF_DEPTH;   // a capped tree is valid (see SF_DEPTH)
  if (flags & SF_NODE_OVERFLOW) return fail(c, NG_ENOMEM, "tree node capacity exceeded");
  if (flags & SF_STACK_OVERFLOW) return fail(c, NG_ENOMEM, "walk stack capacity exceeded");
  if (flags & SF_GROUP_OVERFLOW) return fail(c, NG_ENOMEM, "walk group capacity exceeded");
  if (flags & SF_BAD_TYPE) return fail(c, NG_EINVAL, "a species value is >= D");
  if (flags) return fail(c, NG_ECUDA, "device status flags 0x%x", flags);
  return NG_OK;
}

// Sort + tree with capacity sizing (synchronises once per attempt).
int build_checked(ng_ctx* c, int64_t n, const double* pos, const uint8_t* type,
                  const float* mass) {
  c->n = n;
  c->built = false;
  NG_TRY(alloc_bodies(c, n));
  NG_CUDA(c, cudaMemsetAsync(c->status.p, 0, ST_COUNT * 4, c->stream));
  NG_TRY(sort_bodies(c, n, pos, type, mass));
  return tree_checked(c);
}

// The tree stages of the sorted bodies, with the node capacity grown until
// the tree fits (synchronises once per attempt).
int tree_checked(ng_ctx* c) {
  const int64_t n = c->n;
  c->built = false;
  if (c->cap_nodes == 0) {
    const int leaf = std::max(1, c->p.leaf_size);
    NG_TRY(alloc_nodes(c, std::max<int64_t>(4096, 3 * n / leaf + 1024)));
  }
  for (int attempt = 0; attempt < 8; ++attempt) {
    NG_TRY(build_octree(c));
    uint32_t st[ST_COUNT];
    NG_TRY(read_status(c, st));
    if (st[ST_FLAGS] & SF_BAD_TYPE) return check_flags(c, SF_BAD_TYPE);
    if (st[ST_FLAGS] & SF_NODE_OVERFLOW) {
      const int64_t need = (int64_t)st[ST_NODES_NEEDED];
      NG_TRY(alloc_nodes(c, std::max<int64_t>(need + need / 2, 2 * c->cap_nodes)));
      NG_CUDA(c, cudaMemsetAsync(c->status.p, 0, sizeof(uint32_t), c->stream));
      continue;
    }
    c->nnodes = st[ST_LEVELS + kMaxLevel + 1];
    c->depth_seen = 0;
    for (int l = 0; l <= kMaxLevel; ++l)
      if (st[ST_LEVELS + kMaxLevel + 2 + l] > 0) c->depth_seen = l;
    NG_TRY(reduce_monopoles(c));
    NG_TRY(build_groups(c));
    NG_TRY(type_order(c));
    NG_TRY(read_status(c, st));
    NG_TRY(check_flags(c, st[ST_FLAGS]));
    c->ngroups = st[ST_NGROUPS];
    c->ngroups_n = n;
    c->built = true;
    return NG_OK;
  }
  return fail(c, NG_ENOMEM, "tree capacity could not be sized");
}

// Short + long acceleration into acc (no host synchronisation).
int force_stages(ng_ctx* c, float* acc) {
  if (c->p.pm_mesh > 0) {
    NG_TRY(pm_force(c, acc, false));
    NG_TRY(launch_tree_force(c, acc, true, false));
  } else {
    NG_TRY(launch_tree_force(c, acc, false, false));
  }
  NG_TRY(update_aold(c, acc));
  return NG_OK;
}

// The tree stages and the forces of a captured step. The PM stages read only
// the sorted bodies and their type-major order, and the tree stages write
// nothing they read, so PM runs on pm_stream beside the octree, monopoles and
// groups (latency- and FP64-bound launches beside bandwidth-bound ones); the
// walk, which adds the short-range force to the long-range one, waits for it.
int tree_force_overlapped(ng_ctx* c, float* acc) {
  if (c->p.pm_mesh <= 0 || !c->pm_stream) {
    NG_TRY(tree_stages(c));
    return force_stages(c, acc);
  }
  NG_TRY(type_order(c));
  NG_CUDA(c, cudaEventRecord(c->ev_fork, c->stream));
  NG_CUDA(c, cudaStreamWaitEvent(c->pm_stream, c->ev_fork, 0));
  cudaStream_t main = c->stream;
  c->stream = c->pm_stream;
  const int r = pm_force(c, acc, false);
  c->stream = main;
  NG_CUDA(c, cudaEventRecord(c->ev_join, c->pm_stream));
  if (r != NG_OK) {
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);   // a capture stays joined
    return r;
  }
  NG_TRY(build_octree(c));
  NG_TRY(reduce_monopoles(c));
  NG_TRY(build_groups(c));
  NG_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  NG_TRY(launch_tree_force(c, acc, true, false));
  NG_TRY(update_aold(c, acc));
  return NG_OK;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int validate(ng_ctx* c, const ng_params* p) {
  if (!p) return fail(c, NG_EINVAL, "params is NULL");
  if (p->D < 1 || p->D > NG_MAX_SPECIES) return fail(c, NG_EINVAL, "D=%d outside 1..6", p->D);
  if (!(p->box > 0) || !std::isfinite(p->box)) return fail(c, NG_EINVAL, "box must be > 0");
  if (!(p->eps > 0) || !std::isfinite(p->eps)) return fail(c, NG_EINVAL, "eps must be > 0");
  if (!(p->asmth > 0)) return fail(c, NG_EINVAL, "asmth must be > 0");
  if (!(p->rcut_over_rs > 0)) return fail(c, NG_EINVAL, "rcut_over_rs must be > 0");
  if (!(p->theta >= 0) || p->theta > 2.0) return fail(c, NG_EINVAL, "theta must be in [0, 2]");
  if (p->opening != NG_OPEN_GEOMETRIC && p->opening != NG_OPEN_RELATIVE)
    return fail(c, NG_EINVAL, "opening must be NG_OPEN_GEOMETRIC or NG_OPEN_RELATIVE");
  if (p->reserved1 != 0) return fail(c, NG_EINVAL, "reserved1 must be 0");
  if (p->reserved2 != 0) return fail(c, NG_EINVAL, "reserved2 must be 0");
  if (p->accumulate_fp64 != 0 && p->accumulate_fp64 != 1)
    return fail(c, NG_EINVAL, "accumulate_fp64 must be 0 or 1");
  if (p->pure_tree < 0 || p->pure_tree > 2) return fail(c, NG_EINVAL, "pure_tree must be 0, 1 or 2");
  if (p->ignore_nperp != 0 && p->ignore_nperp != 1)
    return fail(c, NG_EINVAL, "ignore_nperp must be 0 or 1");
  if (p->pure_tree && p->pm_mesh != 0) return fail(c, NG_EINVAL, "pure tree mode needs pm_mesh = 0");
  if (p->pure_tree == 2)
    for (int i = 0; i < p->D; ++i)
      for (int j = 0; j < p->D; ++j) {
        if (p->law[i][j] == NG_MAHALO)
          return fail(c, NG_EINVAL, "Mahalo laws have no lattice corrections (pure_tree 1 only)");
        if ((p->law[i][j] == NG_YUKAWA || p->law[i][j] == NG_YUKAWA_PURE) &&
            !(p->yuk_l[i][j] <= p->box / 8))
          return fail(c, NG_EINVAL, "lattice corrections need yuk_l <= box/8 (yuk_l[%d][%d])", i, j);
      }
  if (p->pure_tree) {
    bool mahalo = false;
    for (int i = 0; i < p->D; ++i)
      for (int j = 0; j < p->D; ++j) mahalo = mahalo || p->law[i][j] == NG_MAHALO;
    if (mahalo && (!(p->beta > 0) || !std::isfinite(p->beta)))
      return fail(c, NG_EINVAL, "beta must be > 0 for Mahalo laws");
  }
  if (p->opening == NG_OPEN_RELATIVE && (!(p->alpha > 0) || !std::isfinite(p->alpha)))
    return fail(c, NG_EINVAL, "alpha must be > 0 for the relative criterion");
  if (p->pm_mesh != 0 && (!is_pow2(p->pm_mesh) || p->pm_mesh < 8 || p->pm_mesh > 1024))
    return fail(c, NG_EINVAL, "pm_mesh must be 0 or a power of two in [8, 1024]");
  if (p->leaf_size < 0 || p->leaf_size > 64) return fail(c, NG_EINVAL, "leaf_size must be 0..64");
  if (p->group_size != 0 && p->group_size != 32)
    return fail(c, NG_EINVAL, "group_size must be 0 or 32");
  if (p->table_size < 0 || p->table_size > 8192) return fail(c, NG_EINVAL, "table_size 0..8192");
  if (p->group_cell != 0 && (p->group_cell < 32 || p->group_cell > 4096))
    return fail(c, NG_EINVAL, "group_cell must be 0 or in [32, 4096]");
  for (int i = 0; i < p->D; ++i)
    for (int j = 0; j < p->D; ++j) {
      if (!std::isfinite(p->G[i][j])) return fail(c, NG_EINVAL, "G[%d][%d] not finite", i, j);
      if (p->law[i][j] != NG_NEWTON && p->law[i][j] != NG_YUKAWA &&
          p->law[i][j] != NG_YUKAWA_PURE && p->law[i][j] != NG_MAHALO)
        return fail(c, NG_EINVAL, "law[%d][%d]=%d unknown", i, j, p->law[i][j]);
      if (p->law[i][j] == NG_MAHALO) {
        if (!p->pure_tree) return fail(c, NG_EINVAL, "Mahalo laws need pure tree mode");
        if (p->law[i][i] != NG_MAHALO && p->law[j][j] != NG_MAHALO)
          return fail(c, NG_EINVAL, "Mahalo pair (%d, %d) has no cored species", i, j);
        continue;
      }
      if (p->law[i][j] != NG_NEWTON &&
          (!(p->yuk_l[i][j] > 0) || !std::isfinite(p->yuk_l[i][j]) || !std::isfinite(p->yuk_a[i][j])))
        return fail(c, NG_EINVAL, "Yukawa range yuk_l[%d][%d] must be > 0", i, j);
    }
  const double rs = p->pm_mesh > 0 ? p->asmth * p->box / p->pm_mesh : p->asmth * p->box;
  if (p->pure_tree != 2 && !(p->rcut_over_rs * rs < 0.5 * p->box))
    return fail(c, NG_EINVAL, "r_cut = %.4g must be below box/2", p->rcut_over_rs * rs);
  return NG_OK;
}

void drop_step_graphs(ng_ctx* c) {
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->step_exec_b) cudaGraphExecDestroy(c->step_exec_b);
  c->step_exec = nullptr;
  c->step_exec_b = nullptr;
}

void normalize_params(ng_params* p) {
  if (p->leaf_size == 0) p->leaf_size = 8;
  if (p->group_size == 0) p->group_size = 32;
  if (p->group_cell == 0) p->group_cell = p->group_size;
}

int ctx_configure(ng_ctx* c, const ng_params* p) {
  NG_TRY(validate(c, p));
  c->p = *p;
  normalize_params(&c->p);
  c->L = p->box;
  c->rs = p->pm_mesh > 0 ? p->asmth * p->box / p->pm_mesh : p->asmth * p->box;
  c->rcut = p->pure_tree == 2 ? INFINITY : p->rcut_over_rs * c->rs;
  c->built = false;
  drop_step_graphs(c);
  // node arrays sized by the species count follow a change of D
  if (c->cap_nodes > 0) NG_TRY(alloc_nodes(c, c->cap_nodes));
  return build_tables(c);
}

// ------------------------------------------------ resident state of ng_step

const uint32_t* force_out(const ng_ctx* c) {
  return c->resident ? nullptr : as<uint32_t>(c->vals_a);
}

// Caller arrays into the resident state, caller order (the first step's sort
// permutes them): raw positions, masses, species (checked and clamped as the
// gather of a plain sort does), velocities, caller indices, accelerations.
__global__ void k_resident_load(int64_t n, const double* __restrict__ pos,
                                const float* __restrict__ vel, const uint8_t* __restrict__ type,
                                const float* __restrict__ mass, const float* __restrict__ acc,
                                int D, double* __restrict__ rpos, float* __restrict__ rvel,
                                uint8_t* __restrict__ rtype, float* __restrict__ rmass,
                                uint32_t* __restrict__ rorig, float* __restrict__ racc,
                                uint32_t* status) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      rpos[e * n + i] = pos[e * n + i];
      rvel[e * n + i] = vel[e * n + i];
      racc[e * n + i] = acc[e * n + i];
    }
    const uint8_t t = type[i];
    if (t >= D) atomicOr(&status[ST_FLAGS], (uint32_t)SF_BAD_TYPE);
    rtype[i] = t < D ? t : 0;
    rmass[i] = mass[i];
    rorig[i] = (uint32_t)i;
  }
}

// The resident state back to the caller's order: positions, velocities and
// accelerations scattered to their caller indices.
__global__ void k_resident_store(int64_t n, const uint32_t* __restrict__ rorig,
                                 const double* __restrict__ rpos, const float* __restrict__ rvel,
                                 const float* __restrict__ racc, double* __restrict__ pos,
                                 float* __restrict__ vel, float* __restrict__ acc) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = rorig[k];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      pos[e * n + i] = rpos[e * n + k];
      vel[e * n + i] = rvel[e * n + k];
      acc[e * n + i] = racc[e * n + k];
    }
  }
}

// out[idx[k]] = in[k] (a float per body).
__global__ void k_scatter_f32(int64_t n, const uint32_t* __restrict__ idx,
                              const float* __restrict__ in, float* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[idx[k]] = in[k];
}

int reserve_resident(ng_ctx* c, int64_t n) {
  NG_TRY(reserve(c, n));
  NG_TRY(ensure(c, c->spos_alt, (size_t)n * 24));
  NG_TRY(ensure(c, c->smass_alt, (size_t)n * 4));
  NG_TRY(ensure(c, c->stype_alt, (size_t)n));
  NG_TRY(ensure(c, c->rvel, (size_t)n * 12));
  NG_TRY(ensure(c, c->rvel_alt, (size_t)n * 12));
  NG_TRY(ensure(c, c->rorig, (size_t)n * 4));
  NG_TRY(ensure(c, c->rorig_alt, (size_t)n * 4));
  NG_TRY(ensure(c, c->racc, (size_t)n * 12));
  NG_TRY(ensure(c, c->rtmp, (size_t)n * 4));
  return NG_OK;
}

// Exchange the roles of the two resident sets: the current state moves to
// the *_alt buffers, which the next step reads; the others receive the next
// state.
void swap_resident(ng_ctx* c) {
  std::swap(c->spos, c->spos_alt);
  std::swap(c->smass, c->smass_alt);
  std::swap(c->stype, c->stype_alt);
  std::swap(c->rvel, c->rvel_alt);
  std::swap(c->rorig, c->rorig_alt);
  c->step_parity ^= 1;
}

int resident_load(ng_ctx* c, int64_t n, const double* pos, const float* vel,
                         const uint8_t* type, const float* mass, const float* acc) {
  k_resident_load<<<work_grid(c, n, 8), 256, 0, c->stream>>>(
      n, pos, vel, type, mass, acc, c->p.D, as<double>(c->spos), as<float>(c->rvel),
      as<uint8_t>(c->stype), as<float>(c->smass), as<uint32_t>(c->rorig), as<float>(c->racc),
      as<uint32_t>(c->status));
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  c->resident = true;
  return NG_OK;
}

// Back to caller order; the context's permutation then maps the sorted
// bodies of the last step to caller indices, as after ng_build_tree, and the
// relative criterion's |a_old| returns to caller order.
int resident_store(ng_ctx* c, int64_t n, double* pos, float* vel, float* acc) {
  k_resident_store<<<work_grid(c, n, 8), 256, 0, c->stream>>>(
      n, as<uint32_t>(c->rorig), as<double>(c->spos), as<float>(c->rvel), as<float>(c->racc), pos,
      vel, acc);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  NG_CUDA(c, cudaMemcpyAsync(c->vals_a.p, c->rorig.p, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                             c->stream));
  if (c->aold_n == n) {
    k_scatter_f32<<<work_grid(c, n, 8), 256, 0, c->stream>>>(n, as<uint32_t>(c->rorig),
                                                             as<float>(c->aold), as<float>(c->rtmp));
    c->launches += 1;
    NG_CUDA(c, cudaGetLastError());
    NG_CUDA(c, cudaMemcpyAsync(c->aold.p, c->rtmp.p, (size_t)n * 4, cudaMemcpyDeviceToDevice,
                               c->stream));
  }
  c->resident = false;
  return NG_OK;
}

// One kick-drift-kick step on the resident state (no host synchronisation;
// captured as a graph). The sort's gather takes the state into this step's
// sorted order; the forces are written in that order.
int resident_step_once(ng_ctx* c, int64_t n, double dt, bool checked) {
  swap_resident(c);
  NG_TRY(launch_kick_drift(c, n, as<float>(c->rvel_alt), as<float>(c->racc), 0.5 * dt, 1,
                           as<double>(c->spos_alt), dt));
  NG_TRY(sort_resident(c, n));
  if (checked) {
    NG_TRY(tree_checked(c));
    NG_TRY(force_stages(c, as<float>(c->racc)));
  } else {
    NG_TRY(tree_force_overlapped(c, as<float>(c->racc)));
  }
  NG_TRY(launch_kick(c, n, as<float>(c->rvel), as<float>(c->racc), 0.5 * dt));
  return NG_OK;
}

}  // namespace ng

using namespace ng;

// Message of the last failed ng_create on this thread (read via ng_last_error(NULL)).
static thread_local std::string g_create_err;

extern "C" {

int ng_create(ng_ctx** out, const ng_params* p, void* stream) {
  if (!out) return NG_EINVAL;
  *out = nullptr;
  ng_ctx* c = new (std::nothrow) ng_ctx();
  if (!c) return NG_ENOMEM;
  int r = validate(c, p);
  if (r != NG_OK) {
    g_create_err = c->err;
    delete c;
    return r;
  }
  c->p = *p;
  normalize_params(&c->p);
  c->stream = (cudaStream_t)stream;
  c->L = p->box;
  c->rs = p->pm_mesh > 0 ? p->asmth * p->box / p->pm_mesh : p->asmth * p->box;
  c->rcut = p->pure_tree == 2 ? INFINITY : p->rcut_over_rs * c->rs;
  cudaError_t e = cudaGetDevice(&c->device);
  int v = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, c->device);
  c->nsm = v;
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  c->smem_optin = (size_t)v;
  if (e != cudaSuccess) {
    g_create_err = std::string("device query failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    delete c;
    return NG_ECUDA;
  }
  r = build_tables(c);
  if (r == NG_OK) r = ensure(c, c->status, ST_COUNT * 4);
  if (r == NG_OK) r = ensure(c, c->counter, 8);
  if (r != NG_OK) {
    g_create_err = c->err;
    ng_destroy(c);
    return r;
  }
  *out = c;
  return NG_OK;
}

int ng_destroy(ng_ctx* c) {
  if (!c) return NG_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->h_tab_pinned) cudaFreeHost(c->h_tab_pinned);
  if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
  if (c->step_exec_b) cudaGraphExecDestroy(c->step_exec_b);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->pm_stream) cudaStreamDestroy(c->pm_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  for (int s = 0; s <= NG_NSTAGES; ++s)
    if (c->stage_ev[s]) cudaEventDestroy(c->stage_ev[s]);
  {
    std::lock_guard<std::mutex> lock(g_fft_plan_lock);
    for (const auto& pl : c->plans) {
      cufftDestroy(pl.r2c);
      cufftDestroy(pl.c2r);
    }
  }
  DevBuf* bufs[] = {&c->d_tab, &c->keys_a, &c->keys_b, &c->vals_a, &c->vals_b, &c->blockhist,
                    &c->spos, &c->smass, &c->stype, &c->body, &c->bleaf,
                    &c->tperm, &c->scan_part, &c->n_level, &c->n_prefix, &c->n_first,
                    &c->n_count, &c->n_child, &c->n_nchild, &c->n_tmp, &c->n_m64,
                    &c->n_cnt, &c->n_geo, &c->n_com, &c->n_link, &c->n_mono, &c->mono_bins, &c->groups, &c->gsize, &c->grank,
                    &c->status, &c->counter, &c->aold, &c->io_pos, &c->io_vel, &c->io_type, &c->io_mass,
                    &c->io_acc, &c->lattice, &c->rho, &c->rhok, &c->phi,
                    &c->walk_desc, &c->walk_prefix, &c->spos_alt, &c->smass_alt, &c->stype_alt,
                    &c->rvel, &c->rvel_alt, &c->rorig, &c->rorig_alt, &c->racc, &c->rtmp};
  for (DevBuf* b : bufs) release(*b);
  delete c;
  return NG_OK;
}

int ng_set_stream(ng_ctx* c, void* stream) {
  if (!c) return NG_EINVAL;
  c->stream = (cudaStream_t)stream;
  drop_step_graphs(c);
  return NG_OK;
}

int ng_build_tree(ng_ctx* c, int64_t n, const double* pos, const uint8_t* type,
                  const float* mass, uint64_t* keys_out, uint32_t* perm_out) {
  if (!c) return NG_EINVAL;
  if (n < 1 || n >= (int64_t)1 << 31) return fail(c, NG_EINVAL, "n=%lld outside [1, 2^31)", (long long)n);
  if (!pos || !type || !mass) return fail(c, NG_EINVAL, "pos/type/mass must be device pointers");
  NG_TRY(build_checked(c, n, pos, type, mass));
  if (keys_out)
    NG_CUDA(c, cudaMemcpyAsync(keys_out, c->keys_a.p, n * 8, cudaMemcpyDeviceToDevice, c->stream));
  if (perm_out)
    NG_CUDA(c, cudaMemcpyAsync(perm_out, c->vals_a.p, n * 4, cudaMemcpyDeviceToDevice, c->stream));
  return NG_OK;
}

int ng_tree_force(ng_ctx* c, float* acc_out, uint64_t* interactions_out) {
  if (!c) return NG_EINVAL;
  if (!c->built) return fail(c, NG_ESTATE, "ng_tree_force before ng_build_tree");
  if (!acc_out) return fail(c, NG_EINVAL, "acc_out is NULL");
  if (interactions_out)
    NG_CUDA(c, cudaMemsetAsync(c->counter.p, 0, 8, c->stream));
  NG_TRY(launch_tree_force(c, acc_out, false, interactions_out != nullptr));
  NG_TRY(update_aold(c, acc_out));
  if (interactions_out) {
    unsigned long long v = 0;
    NG_CUDA(c, cudaMemcpyAsync(&v, c->counter.p, 8, cudaMemcpyDeviceToHost, c->stream));
    uint32_t st[ST_COUNT];
    NG_TRY(read_status(c, st));
    NG_TRY(check_flags(c, st[ST_FLAGS]));
    *interactions_out = v;
  }
  return NG_OK;
}

// Largest |a| (FP32, each operation rounded) over n bodies: non-negative
// floats order like their bit patterns, so an unsigned maximum of the bits
// is the maximum of the values.
__global__ void k_amax(int64_t n, const float* __restrict__ acc, unsigned int* out) {
  unsigned int m = 0u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float x = acc[i], y = acc[n + i], z = acc[2 * n + i];
    const float a = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z)));
    const unsigned int b = __float_as_uint(a);
    m = a == a && b > m ? b : m;   // a NaN acceleration is reported through its own check
  }
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// A_max of Eq. (our_timestep): sup over r of |f_ij(r)| r^2 / (G_ij M), times
// G_ij, over all pairs of the context's laws.
static double law_amax(const ng_params& p) {
  double A = 0.0;
  for (int i = 0; i < p.D; ++i)
    for (int j = 0; j < p.D; ++j) {
      // Yukawa factor a (1 + r/l) e^{-r/l} runs over (0, a]
      double s = 1.0;
      if (p.law[i][j] == NG_YUKAWA) s = std::max(1.0, std::fabs(1.0 + p.yuk_a[i][j]));
      if (p.law[i][j] == NG_YUKAWA_PURE) s = std::fabs(p.yuk_a[i][j]);
      A = std::max(A, std::fabs(p.G[i][j]) * s);
    }
  return A;
}

int ng_timestep(ng_ctx* c, int64_t n, const float* acc, double eta, double dt_max,
                double* dt_out, float* amax_out) {
  if (!c) return NG_EINVAL;
  if (n < 1 || n >= (int64_t)1 << 31) return fail(c, NG_EINVAL, "n outside [1, 2^31)");
  if (!acc || !dt_out) return fail(c, NG_EINVAL, "NULL pointer");
  if (!(eta > 0) || !(dt_max > 0) || !std::isfinite(eta) || !std::isfinite(dt_max))
    return fail(c, NG_EINVAL, "eta and dt_max must be > 0");
  NG_TRY(ensure(c, c->counter, 8));
  NG_CUDA(c, cudaMemsetAsync(c->counter.p, 0, 4, c->stream));
  k_amax<<<work_grid(c, n, 8), 256, 0, c->stream>>>(n, acc, as<unsigned int>(c->counter));
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  unsigned int bits = 0;
  NG_CUDA(c, cudaMemcpyAsync(&bits, c->counter.p, 4, cudaMemcpyDeviceToHost, c->stream));
  NG_CUDA(c, cudaStreamSynchronize(c->stream));
  float amax = 0.f;
  std::memcpy(&amax, &bits, 4);
  const double A = law_amax(c->p);
  double dt = dt_max;
  if (amax > 0.f && A > 0.0)
    dt = std::min(dt_max, std::sqrt(2.0 * eta * c->p.eps / (A * (double)amax)));
  *dt_out = dt;
  if (amax_out) *amax_out = amax;
  return NG_OK;
}

int ng_set_acc_old(ng_ctx* c, int64_t n, const float* acc_old) {
  if (!c) return NG_EINVAL;
  if (n < 1 || n >= (int64_t)1 << 31) return fail(c, NG_EINVAL, "n outside [1, 2^31)");
  if (!acc_old) return fail(c, NG_EINVAL, "acc_old is NULL");
  return set_aold(c, n, acc_old);
}

int ng_count_interactions(ng_ctx* c, int64_t* counts_out, uint64_t* total_out) {
  if (!c) return NG_EINVAL;
  if (!c->built) return fail(c, NG_ESTATE, "ng_count_interactions before ng_build_tree");
  NG_TRY(launch_count(c, counts_out));
  unsigned long long v = 0;
  NG_CUDA(c, cudaMemcpyAsync(&v, c->counter.p, 8, cudaMemcpyDeviceToHost, c->stream));
  uint32_t st[ST_COUNT];
  NG_TRY(read_status(c, st));
  NG_TRY(check_flags(c, st[ST_FLAGS]));
  if (total_out) *total_out = v;
  return NG_OK;
}

int ng_pm_force(ng_ctx* c, float* acc_out) {
  if (!c) return NG_EINVAL;
  if (!c->built) return fail(c, NG_ESTATE, "ng_pm_force before ng_build_tree");
  if (!acc_out) return fail(c, NG_EINVAL, "acc_out is NULL");
  return pm_force(c, acc_out, false);
}

int ng_force(ng_ctx* c, float* acc_out) {
  if (!c) return NG_EINVAL;
  if (!c->built) return fail(c, NG_ESTATE, "ng_force before ng_build_tree");
  if (!acc_out) return fail(c, NG_EINVAL, "acc_out is NULL");
  return force_stages(c, acc_out);
}

int ng_stage_times(ng_ctx* c, int64_t n, double* pos, float* vel, const uint8_t* type,
                   const float* mass, float* acc, double dt, float* ms_out) {
  if (!c) return NG_EINVAL;
  if (n < 1 || n >= (int64_t)1 << 31) return fail(c, NG_EINVAL, "n outside [1, 2^31)");
  if (!pos || !vel || !type || !mass || !acc || !ms_out) return fail(c, NG_EINVAL, "NULL array");
  if (!std::isfinite(dt)) return fail(c, NG_EINVAL, "bad dt");
  for (int s = 0; s < NG_NSTAGES; ++s) ms_out[s] = 0.f;
  // untimed: one step sizes every buffer and leaves acc valid at pos
  NG_TRY(ng_step(c, n, pos, vel, type, mass, acc, 0, 1, dt));
  for (int s = 0; s <= NG_NSTAGES; ++s)
    if (!c->stage_ev[s]) NG_CUDA(c, cudaEventCreate(&c->stage_ev[s]));
  NG_TRY(resident_load(c, n, pos, vel, type, mass, acc));
  // one untimed resident step: the timed one then starts, as every replayed
  // step does, from the previous step's sorted order
  NG_TRY(resident_step_once(c, n, dt, false));
  swap_resident(c);
  NG_TRY(launch_kick_drift(c, n, as<float>(c->rvel_alt), as<float>(c->racc), 0.5 * dt, 1,
                           as<double>(c->spos_alt), dt));
  c->stage_seen = 0;
  c->timing = true;
  // the tree depth of a captured step
  c->level_cap = std::min(kMaxLevel, c->depth_seen + kCapturedDepthMargin);
  int r = sort_resident(c, n);
  if (r == NG_OK) r = tree_stages(c);
  c->level_cap = kMaxLevel;
  if (r == NG_OK) r = force_stages(c, as<float>(c->racc));
  c->timing = false;
  if (r != NG_OK) {
    c->resident = false;
    return r;
  }
  NG_CUDA(c, cudaEventRecord(c->stage_ev[NG_NSTAGES], c->stream));
  NG_TRY(launch_kick(c, n, as<float>(c->rvel), as<float>(c->racc), 0.5 * dt));
  NG_TRY(resident_store(c, n, pos, vel, acc));
  NG_CUDA(c, cudaStreamSynchronize(c->stream));
  uint32_t st[ST_COUNT];
  NG_TRY(read_status(c, st));
  NG_TRY(check_flags(c, st[ST_FLAGS]));
  // a stage runs until the next stage that ran (or the final event)
  const uint32_t seen = c->stage_seen;
  for (int s = 0; s < NG_NSTAGES; ++s) {
    if (!(seen >> s & 1u)) continue;
    int e = s + 1;
    while (e < NG_NSTAGES && !(seen >> e & 1u)) ++e;
    float t = 0.f;
    NG_CUDA(c, cudaEventElapsedTime(&t, c->stage_ev[s], c->stage_ev[e]));
    ms_out[s] = t;
  }
  c->built = true;
  return NG_OK;
}

int ng_step(ng_ctx* c, int64_t n, double* pos, float* vel, const uint8_t* type,
            const float* mass, float* acc, int acc_valid, int nsteps, double dt) {
  if (!c) return NG_EINVAL;
  if (n < 1 || n >= (int64_t)1 << 31) return fail(c, NG_EINVAL, "n outside [1, 2^31)");
  if (!pos || !vel || !type || !mass || !acc) return fail(c, NG_EINVAL, "NULL array");
  if (nsteps < 0 || !std::isfinite(dt)) return fail(c, NG_EINVAL, "bad nsteps/dt");
  if (!acc_valid) {
    NG_TRY(build_checked(c, n, pos, type, mass));
    NG_TRY(force_stages(c, acc));
  }
  if (nsteps == 0) {
    NG_CUDA(c, cudaStreamSynchronize(c->stream));
    return NG_OK;
  }
  // the state stays on the device in the previous step's sorted order
  c->n = n;
  NG_TRY(reserve_resident(c, n));
  NG_CUDA(c, cudaMemsetAsync(c->status.p, 0, sizeof(uint32_t), c->stream));
  NG_TRY(resident_load(c, n, pos, vel, type, mass, acc));
  int r = NG_OK;
  int done = 0;
  const bool reuse = c->step_exec && c->step_exec_b && c->graph_n == n && c->graph_dt == dt &&
                     c->graph_gen == c->alloc_gen;
  if (!reuse) {
    // one eager step sizes the tree with synchronised checks, then the step
    // is captured twice, once per assignment of the two resident sets
    r = resident_step_once(c, n, dt, true);
    done = 1;
    if (r == NG_OK && c->cap_nodes < c->nnodes + c->nnodes / 4 + 1024) {
      // headroom for the replayed steps, whose trees cannot regrow; the
      // regrow drops the node arrays, so the tree of the current (sorted)
      // bodies is built again
      r = alloc_nodes(c, c->nnodes + c->nnodes / 4 + 1024);
      if (r == NG_OK) r = tree_checked(c);
    }
    if (r == NG_OK && c->step_exec) {
      cudaGraphExecDestroy(c->step_exec);
      c->step_exec = nullptr;
    }
    if (r == NG_OK && c->step_exec_b) {
      cudaGraphExecDestroy(c->step_exec_b);
      c->step_exec_b = nullptr;
    }
    if (r == NG_OK && done < nsteps) {
      // capture needs a stream other than the legacy default one
      if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        r = fail(c, NG_ECUDA, "capture stream creation failed");
      }
      cudaStream_t user = c->stream;
      // captured trees stop two levels below the deepest one seen so far
      c->level_cap = std::min(kMaxLevel, c->depth_seen + kCapturedDepthMargin);
      // graph k starts from step parity k (the two captures leave the
      // assignment where it was: the captured steps do not run)
      for (int k = 0; k < 2 && r == NG_OK; ++k) {
        cudaGraphExec_t* slot = c->step_parity == 0 ? &c->step_exec : &c->step_exec_b;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
          cudaGetLastError();
          r = fail(c, NG_ECUDA, "begin capture failed");
          break;
        }
        c->stream = c->cap_stream;
        const uint64_t before = c->launches;
        r = resident_step_once(c, n, dt, false);
        c->graph_launches = c->launches - before;
        c->launches = before;
        c->stream = user;
        const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        cudaGetLastError();
        if (r != NG_OK) {
          if (g) cudaGraphDestroy(g);
          break;
        }
        if (e != cudaSuccess) {
          r = fail(c, NG_ECUDA, "step capture failed: %s", cudaGetErrorString(e));
          break;
        }
        const cudaError_t ei = cudaGraphInstantiate(slot, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) r = fail(c, NG_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(ei));
      }
      c->level_cap = kMaxLevel;
      if (r == NG_OK) {
        c->graph_n = n;
        c->graph_dt = dt;
        c->graph_gen = c->alloc_gen;
      }
    }
  }
  for (int s = done; s < nsteps && r == NG_OK; ++s) {
    cudaGraphExec_t g = c->step_parity == 0 ? c->step_exec : c->step_exec_b;
    if (cudaGraphLaunch(g, c->stream) != cudaSuccess) {
      cudaGetLastError();
      r = fail(c, NG_ECUDA, "graph launch failed");
      break;
    }
    swap_resident(c);   // the replayed step's exchange, on the host
    c->launches += c->graph_launches;
  }
  const int rs = resident_store(c, n, pos, vel, acc);
  if (r == NG_OK) r = rs;
  NG_TRY(r);
  uint32_t st[ST_COUNT];
  NG_TRY(read_status(c, st));
  // a replayed tree outgrew the level cap (still correct): capture deeper next call
  if (st[ST_FLAGS] & SF_DEPTH) drop_step_graphs(c);
  NG_TRY(check_flags(c, st[ST_FLAGS]));
  c->built = true;
  return NG_OK;
}

int ng_step_host(ng_ctx* c, int64_t n, double* pos, float* vel, const uint8_t* type,
                 const float* mass, float* acc, int acc_valid, int nsteps, double dt) {
  if (!c) return NG_EINVAL;
  if (n < 1 || n >= (int64_t)1 << 31) return fail(c, NG_EINVAL, "n outside [1, 2^31)");
  if (!pos || !vel || !type || !mass || !acc) return fail(c, NG_EINVAL, "NULL array");
  NG_TRY(ensure(c, c->io_pos, (size_t)n * 24));
  NG_TRY(ensure(c, c->io_vel, (size_t)n * 12));
  NG_TRY(ensure(c, c->io_type, (size_t)n));
  NG_TRY(ensure(c, c->io_mass, (size_t)n * 4));
  NG_TRY(ensure(c, c->io_acc, (size_t)n * 12));
  double* dpos = as<double>(c->io_pos);
  float* dvel = as<float>(c->io_vel);
  float* dacc = as<float>(c->io_acc);
  NG_CUDA(c, cudaMemcpyAsync(dpos, pos, (size_t)n * 24, cudaMemcpyHostToDevice, c->stream));
  NG_CUDA(c, cudaMemcpyAsync(dvel, vel, (size_t)n * 12, cudaMemcpyHostToDevice, c->stream));
  NG_CUDA(c, cudaMemcpyAsync(c->io_type.p, type, (size_t)n, cudaMemcpyHostToDevice, c->stream));
  NG_CUDA(c, cudaMemcpyAsync(c->io_mass.p, mass, (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
  if (acc_valid)
    NG_CUDA(c, cudaMemcpyAsync(dacc, acc, (size_t)n * 12, cudaMemcpyHostToDevice, c->stream));
  NG_TRY(ng_step(c, n, dpos, dvel, as<uint8_t>(c->io_type), as<float>(c->io_mass), dacc,
                 acc_valid, nsteps, dt));
  NG_CUDA(c, cudaMemcpyAsync(pos, dpos, (size_t)n * 24, cudaMemcpyDeviceToHost, c->stream));
  NG_CUDA(c, cudaMemcpyAsync(vel, dvel, (size_t)n * 12, cudaMemcpyDeviceToHost, c->stream));
  NG_CUDA(c, cudaMemcpyAsync(acc, dacc, (size_t)n * 12, cudaMemcpyDeviceToHost, c->stream));
  NG_CUDA(c, cudaStreamSynchronize(c->stream));
  return NG_OK;
}

int ng_tree_export(ng_ctx* c, int64_t* nnodes, int32_t* level, uint64_t* prefix, int64_t* first,
                   int64_t* count, int32_t* nchild, int64_t* child_first, uint32_t* cnt,
                   double* mass, double* com) {
  if (!c || !nnodes) return NG_EINVAL;
  if (!c->built) return fail(c, NG_ESTATE, "no tree built");
  NG_CUDA(c, cudaStreamSynchronize(c->stream));
  const int64_t nn = c->nnodes;
  const int D = c->p.D;
  *nnodes = nn;
  std::vector<uint8_t> u8(nn);
  std::vector<uint32_t> u32(nn);
  if (level) {
    NG_CUDA(c, cudaMemcpy(u8.data(), c->n_level.p, nn, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nn; ++k) level[k] = u8[k];
  }
  if (prefix) NG_CUDA(c, cudaMemcpy(prefix, c->n_prefix.p, nn * 8, cudaMemcpyDeviceToHost));
  if (first) {
    NG_CUDA(c, cudaMemcpy(u32.data(), c->n_first.p, nn * 4, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nn; ++k) first[k] = u32[k];
  }
  if (count) {
    NG_CUDA(c, cudaMemcpy(u32.data(), c->n_count.p, nn * 4, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nn; ++k) count[k] = u32[k];
  }
  std::vector<uint8_t> nch(nn);
  NG_CUDA(c, cudaMemcpy(nch.data(), c->n_nchild.p, nn, cudaMemcpyDeviceToHost));
  if (nchild)
    for (int64_t k = 0; k < nn; ++k) nchild[k] = nch[k];
  if (child_first) {
    NG_CUDA(c, cudaMemcpy(u32.data(), c->n_child.p, nn * 4, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nn; ++k) child_first[k] = nch[k] ? (int64_t)u32[k] : -1;
  }
  if (cnt) NG_CUDA(c, cudaMemcpy(cnt, c->n_cnt.p, nn * D * 4, cudaMemcpyDeviceToHost));
  if (mass || com) {
    std::vector<double> m64((size_t)nn * D * 4);
    NG_CUDA(c, cudaMemcpy(m64.data(), c->n_m64.p, m64.size() * 8, cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < nn; ++k)
      for (int t = 0; t < D; ++t) {
        const double* s = &m64[((size_t)k * D + t) * 4];
        if (mass) mass[k * D + t] = s[0];
        if (com)
          for (int d = 0; d < 3; ++d) com[(k * D + t) * 3 + d] = s[0] > 0 ? s[1 + d] / s[0] * c->L : 0.0;
      }
  }
  return NG_OK;
}

int ng_type_order(ng_ctx* c, int64_t* type_offsets, uint32_t* order_out) {
  if (!c) return NG_EINVAL;
  if (!c->built) return fail(c, NG_ESTATE, "no tree built");
  const int64_t n = c->n;
  const int nblocks = (int)((n + kRadixTile - 1) / kRadixTile);
  if (type_offsets) {
    NG_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int d = 0; d < c->p.D; ++d) {
      uint32_t v = 0;
      NG_CUDA(c, cudaMemcpy(&v, as<uint32_t>(c->blockhist) + (size_t)d * nblocks, 4,
                            cudaMemcpyDeviceToHost));
      type_offsets[d] = v;
    }
    type_offsets[c->p.D] = n;
  }
  if (order_out) {
    // caller indices in type-major order: perm[tperm[j]]
    std::vector<uint32_t> tp(n), pm(n);
    NG_CUDA(c, cudaMemcpy(tp.data(), c->tperm.p, n * 4, cudaMemcpyDeviceToHost));
    NG_CUDA(c, cudaMemcpy(pm.data(), c->vals_a.p, n * 4, cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < n; ++j) tp[j] = pm[tp[j]];
    NG_CUDA(c, cudaMemcpy(order_out, tp.data(), n * 4, cudaMemcpyHostToDevice));
  }
  return NG_OK;
}

int ng_launch_count(const ng_ctx* c, uint64_t* out) {
  if (!c || !out) return NG_EINVAL;
  *out = c->launches;
  return NG_OK;
}

int ng_sort_passes(const ng_ctx* c, int32_t* out) {
  if (!c || !out) return NG_EINVAL;
  *out = c->sort_passes;
  return NG_OK;
}

const char* ng_last_error(const ng_ctx* c) {
  if (!c) return g_create_err.empty() ? "no context" : g_create_err.c_str();
  return c->err.c_str();
}

const char* ng_version(void) { return "ngravs-gb300 0.1 (sm_103a)"; }

}  // extern "C"
