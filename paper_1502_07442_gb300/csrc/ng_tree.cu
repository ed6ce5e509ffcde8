// Tree stage (Sec. 2.2): canonical Morton-prefix octree built breadth-first
// one level per launch (node ranges stay on the device, no host round trip),
// per-node per-species monopoles reduced in double precision (one thread per
// node: every leaf in one launch, then the internal nodes level by level,
// bottom-up), and the walk groups.
//
// Canonical tree: nodes are the non-empty Morton cells reachable from the
// root; a cell is a leaf iff it holds <= leaf_size bodies or is at level 20;
// children are the non-empty octants in octant order; nodes are numbered
// level by level, and within a level in key order. Builds inside captured
// steps stop at a level cap two below the deepest level seen by the step
// before the capture (fewer launches per level-free tail); a cell at the cap
// is then a leaf whatever it holds, and SF_DEPTH says so.
#include <cooperative_groups.h>

#include "ng_internal.cuh"

namespace ng {

struct Levels {
  uint32_t* start;   // [kMaxLevel + 2]: first node of each level, then end
  uint32_t* count;   // [kMaxLevel + 1]: nodes per level
};

__device__ __forceinline__ Levels levels_of(uint32_t* status) {
  return Levels{status + ST_LEVELS, status + ST_LEVELS + kMaxLevel + 2};
}

__global__ void k_tree_init(uint32_t* status, int64_t n, uint8_t* level, uint64_t* prefix,
                            uint32_t* first, uint32_t* count) {
  if (threadIdx.x == 0) {
    Levels lv = levels_of(status);
    for (int l = 0; l <= kMaxLevel + 1; ++l) lv.start[l] = 1;
    for (int l = 0; l <= kMaxLevel; ++l) lv.count[l] = 0;
    lv.start[0] = 0;
    lv.start[1] = 1;
    lv.count[0] = 1;
    status[ST_NODES_NEEDED] = 1;
    status[ST_NGROUPS] = 0;
    level[0] = 0;
    prefix[0] = 0;
    first[0] = 0;
    count[0] = (uint32_t)n;
  }
}

// First index in [lo, hi) whose child octant at shift is >= oct.
__device__ __forceinline__ uint32_t octant_bound(const uint64_t* __restrict__ keys, uint32_t lo,
                                                 uint32_t hi, int shift, uint32_t oct) {
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    const uint32_t o = (uint32_t)((keys[mid] >> (3 + shift)) & 7ull);
    if (o < oct) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Both kernels give each node of level lvl a team of 8 lanes: lane o finds
// where octant o of the node's (sorted) body range starts, all 8 binary
// searches at once, so a level with few large nodes (the top of the tree)
// waits for one search, not eight in a row. Teams of a warp loop together
// (every lane runs the same iterations, so the team shuffles are safe).
struct OctTeam {
  uint32_t start, end;   // octant `sub` of the node: bodies [start, end)
  bool nonempty;
  uint32_t bits;         // non-empty octants of the node, bit o for octant o
};

__device__ __forceinline__ OctTeam octant_team(const uint64_t* __restrict__ keys, bool split,
                                               uint32_t f, uint32_t c, int shift, int sub,
                                               int lane) {
  OctTeam t;
  t.start = (split && sub > 0) ? octant_bound(keys, f, f + c, shift, (uint32_t)sub) : f;
  const uint32_t nxt = __shfl_down_sync(0xffffffffu, t.start, 1, 8);
  t.end = sub == 7 ? f + c : nxt;
  t.nonempty = split && t.end > t.start;
  const uint32_t m = __ballot_sync(0xffffffffu, t.nonempty);
  t.bits = (m >> (lane & 24)) & 0xffu;
  return t;
}

// Count phase of level lvl: each team of 8 lanes (team of teams, warps'
// teams looping together) takes nodes of the level and records their child
// counts in nchild and tmp. lmax: the deepest level the build emits
// (kMaxLevel unless capped); nodes of level lmax are leaves, and one above
// the leaf size raises SF_DEPTH.
__device__ __forceinline__ void tree_count_nodes(int lvl, int lmax, uint32_t* status, int64_t cap,
                                                 int leaf_size, const uint64_t* __restrict__ keys,
                                                 const uint32_t* __restrict__ first,
                                                 const uint32_t* __restrict__ count,
                                                 uint8_t* nchild, uint32_t* child, uint32_t* tmp,
                                                 int64_t team, int64_t teams) {
  Levels lv = levels_of(status);
  const uint32_t s = lv.start[lvl];
  uint32_t e = lv.start[lvl + 1];
  if (e > cap) e = (uint32_t)cap;
  const int nodes = e > s ? (int)(e - s) : 0;
  const int shift = 3 * (kMaxLevel - (lvl + 1));
  const int lane = threadIdx.x & 31, sub = lane & 7;
  for (int64_t base = team & ~(int64_t)3; base < nodes; base += teams) {
    const int64_t j = base + (team & 3);
    const bool valid = j < nodes;
    const uint32_t k = s + (uint32_t)j;
    const uint32_t f = valid ? first[k] : 0u, c = valid ? count[k] : 0u;
    const bool split = valid && (int)c > leaf_size && lvl < lmax;
    const OctTeam t = octant_team(keys, split, f, c, shift, sub, lane);
    if (valid && sub == 0) {
      const uint32_t nch = (uint32_t)__popc(t.bits);
      nchild[k] = (uint8_t)nch;
      tmp[k - s] = nch;
      if (lvl == lmax) {
        child[k] = 0xffffffffu;   // no emit follows the last level
        if ((int)c > leaf_size && lmax < kMaxLevel) atomicOr(&status[ST_FLAGS], (uint32_t)SF_DEPTH);
      }
    }
  }
}

// The start of level lvl + 2 from the child total of level lvl (one thread);
// a node count beyond the capacity raises SF_NODE_OVERFLOW.
__device__ __forceinline__ void tree_level_close(int lvl, uint32_t* status, int64_t cap) {
  Levels lv = levels_of(status);
  const uint64_t end = (uint64_t)lv.start[lvl + 1] + lv.count[lvl + 1];
  lv.start[lvl + 2] = (uint32_t)(end < 0xffffffffull ? end : 0xffffffffull);
  // only levels up to the first overflow are counted correctly: the node
  // estimate is taken there and never from the truncated levels below it
  if (!(status[ST_FLAGS] & SF_NODE_OVERFLOW)) {
    status[ST_NODES_NEEDED] = (uint32_t)(end < 0xffffffffull ? end : 0xffffffffull);
    if (end > (uint64_t)cap) status[ST_FLAGS] |= (uint32_t)SF_NODE_OVERFLOW;
  }
}

// Emit phase of level lvl: the children of each split node, numbered from the
// level's end (next0) by the exclusive scan of the child counts (off).
__device__ __forceinline__ void tree_emit_nodes(int lvl, uint32_t next0, uint32_t* status, int64_t cap,
                                                const uint64_t* __restrict__ keys, uint8_t* level,
                                                uint64_t* prefix, uint32_t* first, uint32_t* count,
                                                const uint8_t* __restrict__ nchild, uint32_t* child,
                                                const uint32_t* __restrict__ off, int64_t team,
                                                int64_t teams) {
  Levels lv = levels_of(status);
  const uint32_t s = lv.start[lvl];
  uint32_t e = next0;
  if (e > cap) e = (uint32_t)cap;
  const int nodes = e > s ? (int)(e - s) : 0;
  const int shift = 3 * (kMaxLevel - (lvl + 1));
  const int lane = threadIdx.x & 31, sub = lane & 7;
  for (int64_t base = team & ~(int64_t)3; base < nodes; base += teams) {
    const int64_t j = base + (team & 3);
    const bool valid = j < nodes;
    const uint32_t k = s + (uint32_t)j;
    const uint32_t nch = valid ? nchild[k] : 0u;
    const bool split = nch > 0;
    const uint32_t f = split ? first[k] : 0u, c = split ? count[k] : 0u;
    const OctTeam t = octant_team(keys, split, f, c, shift, sub, lane);
    if (!split) {
      if (valid && sub == 0) child[k] = 0xffffffffu;
      continue;
    }
    const uint32_t c0 = next0 + off[k - s];
    if (sub == 0) child[k] = c0;
    if (t.nonempty) {
      const uint64_t id = (uint64_t)c0 + (uint32_t)__popc(t.bits & ((1u << sub) - 1u));
      if (id < (uint64_t)cap) {
        level[id] = (uint8_t)(lvl + 1);
        prefix[id] = (prefix[k] << 3) | (uint64_t)sub;
        first[id] = t.start;
        count[id] = t.end - t.start;
      }
    }
  }
}

__global__ void k_tree_count(int lvl, int lmax, uint32_t* status, int64_t cap, int leaf_size,
                             const uint64_t* __restrict__ keys, const uint32_t* __restrict__ first,
                             const uint32_t* __restrict__ count, uint8_t* nchild,
                             uint32_t* child, uint32_t* tmp) {
  const int64_t team = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
  const int64_t teams = ((int64_t)gridDim.x * blockDim.x) >> 3;   // a multiple of 4
  tree_count_nodes(lvl, lmax, status, cap, leaf_size, keys, first, count, nchild, child, tmp, team,
                   teams);
}

__global__ void k_tree_emit(int lvl, uint32_t* status, int64_t cap,
                            const uint64_t* __restrict__ keys, uint8_t* level, uint64_t* prefix,
                            uint32_t* first, uint32_t* count, const uint8_t* __restrict__ nchild,
                            uint32_t* child, const uint32_t* __restrict__ off) {
  const uint32_t next0 = levels_of(status).start[lvl + 1];
  if (blockIdx.x == 0 && threadIdx.x == 0) tree_level_close(lvl, status, cap);
  const int64_t team = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 3;
  const int64_t teams = ((int64_t)gridDim.x * blockDim.x) >> 3;
  tree_emit_nodes(lvl, next0, status, cap, keys, level, prefix, first, count, nchild, child, off,
                  team, teams);
}

// The whole build of a small tree in one launch: one cluster of
// kClusterBlocks blocks (co-scheduled; its barrier is the hardware cluster
// barrier, so no block waits on a flag) runs every level's count, scan and
// emit phases, each the same code as the per-level kernels, with a cluster
// barrier between phases. The child-count scan of a level: each block sums
// its contiguous chunk, the sums go to every block's shared memory, and
// each block scans its chunk from the sum of the chunks before it.
__global__ void __cluster_dims__(kClusterBlocks, 1, 1) __launch_bounds__(1024, 1)
k_tree_cluster(int lmax, uint32_t* status, int64_t n, int64_t cap, int leaf_size,
               const uint64_t* __restrict__ keys, uint8_t* level, uint64_t* prefix, uint32_t* first,
               uint32_t* count, uint8_t* nchild, uint32_t* child, uint32_t* tmp) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  __shared__ uint32_t sums[kClusterBlocks];
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t tile_total;
  const int tid = threadIdx.x, nb = (int)gridDim.x, b = (int)blockIdx.x;
  Levels lv = levels_of(status);
  if (b == 0 && tid == 0) {
    for (int l = 0; l <= kMaxLevel + 1; ++l) lv.start[l] = 1;
    for (int l = 0; l <= kMaxLevel; ++l) lv.count[l] = 0;
    lv.start[0] = 0;
    lv.start[1] = 1;
    lv.count[0] = 1;
    status[ST_NODES_NEEDED] = 1;
    status[ST_NGROUPS] = 0;
    level[0] = 0;
    prefix[0] = 0;
    first[0] = 0;
    count[0] = (uint32_t)n;
  }
  cluster.sync();
  const int64_t team = ((int64_t)b * blockDim.x + tid) >> 3;
  const int64_t teams = ((int64_t)nb * blockDim.x) >> 3;
  for (int l = 0; l <= lmax; ++l) {
    tree_count_nodes(l, lmax, status, cap, leaf_size, keys, first, count, nchild, child, tmp, team,
                     teams);
    cluster.sync();
    if (l == lmax) break;
    // exclusive scan of the level's child counts (tmp, in place)
    const uint32_t s = lv.start[l];
    uint32_t e = lv.start[l + 1];
    if (e > cap) e = (uint32_t)cap;
    const int nodes = e > s ? (int)(e - s) : 0;
    const int chunk = (nodes + nb - 1) / nb;
    const int c0 = min(nodes, b * chunk), c1 = min(nodes, c0 + chunk);
    uint32_t part = 0;
    for (int i = c0 + tid; i < c1; i += blockDim.x) part += tmp[i];
    block_inclusive_scan<1024>(part, warp_tot, &tile_total);
    if (tid < nb) *cluster.map_shared_rank(&sums[b], tid) = tile_total;
    cluster.sync();
    uint32_t carry = 0;
    for (int r = 0; r < b; ++r) carry += sums[r];
    for (int base = c0; base < c1; base += blockDim.x) {
      const int i = base + tid;
      const uint32_t v = i < c1 ? tmp[i] : 0u;
      const uint32_t inc = block_inclusive_scan<1024>(v, warp_tot, &tile_total);
      if (i < c1) tmp[i] = carry + inc - v;
      __syncthreads();
      carry += tile_total;
      __syncthreads();
    }
    if (b == nb - 1 && tid == 0) lv.count[l + 1] = carry;
    cluster.sync();
    const uint32_t next0 = lv.start[l + 1];
    if (b == 0 && tid == 0) tree_level_close(l, status, cap);
    tree_emit_nodes(l, next0, status, cap, keys, level, prefix, first, count, nchild, child, tmp,
                    team, teams);
    cluster.sync();
  }
  if (lmax < kMaxLevel && b == 0 && tid == 0) {
    const uint32_t end = lv.start[lmax + 1];
    for (int l = lmax + 2; l <= kMaxLevel + 1; ++l) lv.start[l] = end;
  }
}

// A build capped at level lmax < kMaxLevel: the levels below it are empty
// (their starts all equal the end of level lmax), as the node total and the
// per-level kernels that follow expect.
__global__ void k_tree_close(uint32_t* status, int lmax) {
  if (threadIdx.x == 0) {
    Levels lv = levels_of(status);
    const uint32_t end = lv.start[lmax + 1];
    for (int l = lmax + 2; l <= kMaxLevel + 1; ++l) lv.start[l] = end;
  }
}

int build_octree(ng_ctx* c) {
  const int64_t n = c->n;
  const int64_t cap = c->cap_nodes;
  uint32_t* st = as<uint32_t>(c->status);
  uint8_t* level = as<uint8_t>(c->n_level);
  uint64_t* prefix = as<uint64_t>(c->n_prefix);
  uint32_t* first = as<uint32_t>(c->n_first);
  uint32_t* count = as<uint32_t>(c->n_count);
  uint8_t* nchild = as<uint8_t>(c->n_nchild);
  uint32_t* child = as<uint32_t>(c->n_child);
  uint32_t* tmp = as<uint32_t>(c->n_tmp);
  const uint64_t* keys = as<uint64_t>(c->keys_a);
  const int leaf = c->p.leaf_size;
  const int lmax = std::min(std::max(c->level_cap, 0), kMaxLevel);
  stage_mark(c, NG_STAGE_OCTREE);
  if (n <= kClusterMaxBodies) {
    k_tree_cluster<<<kClusterBlocks, 1024, 0, c->stream>>>(lmax, st, n, cap, leaf, keys, level,
                                                          prefix, first, count, nchild, child, tmp);
    c->launches += 1;
    NG_CUDA(c, cudaGetLastError());
    return NG_OK;
  }
  k_tree_init<<<1, 32, 0, c->stream>>>(st, n, level, prefix, first, count);
  c->launches += 1 + (lmax + 1) + lmax;   // init, counts, emits (scans count themselves)
  for (int l = 0; l <= lmax; ++l) {
    // grids sized by the most nodes level l can hold (kernels stride over the actual count)
    const int64_t bound = std::min<int64_t>(cap, level_bound(l, c->n));
    const int grid = work_grid(c, 8 * bound, 4);   // 8 lanes per node
    k_tree_count<<<grid, 256, 0, c->stream>>>(l, lmax, st, cap, leaf, keys, first, count, nchild,
                                              child, tmp);
    if (l == lmax) break;
    // children per level: exclusive scan of the per-node child counts
    uint32_t* lvcount = st + ST_LEVELS + kMaxLevel + 2;
    NG_TRY(scan_u32(c, tmp, tmp, bound, lvcount + l, lvcount + l + 1));
    k_tree_emit<<<grid, 256, 0, c->stream>>>(l, st, cap, keys, level, prefix, first, count,
                                             nchild, child, tmp);
  }
  if (lmax < kMaxLevel) {
    k_tree_close<<<1, 32, 0, c->stream>>>(st, lmax);
    c->launches += 1;
  }
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

// --------------------------------------------------------- monopoles


struct MonoArgs {
  const uint8_t* level;
  const uint64_t* prefix;
  const uint32_t* first;
  const uint32_t* count;
  const uint8_t* nchild;
  const uint32_t* child;
  const double* spos;      // [3][n] physical
  const float* smass;
  const uint8_t* stype;
  double* m64;             // [node][D][4]: mass, sum m x, sum m y, sum m z (box units)
  uint32_t* cnt;           // [node][D]
  float4* geo;
  float4* com;
  int4* link;
  float4* mono;            // [node][D]
  float4* body;            // [sorted body]
  uint32_t* bleaf;         // [sorted body] leaf index
  uint32_t* status;
  int64_t n, cap;
  double invL, L;
};

// One thread per node of level lvl (FP64 is ~1/64 of the FP32 rate here, so
// every FP64 operation counts): a leaf adds each body to its own species
// (4 FP64 operations per body, in shared-memory slots chosen by the species)
// and writes the body records (offset from the leaf centre, subtracted in
// FP64 in physical units, scaled to box units in FP32); an internal node adds
// its <= 8 children. The FP32 walk records need no FP64 division: the
// mass-weighted offset sum(m x) - M c is formed with one FP64 FMA and divided
// by M in FP32.
constexpr int kMonoThreads = 128;

// Sums of node k of level lvl (leaf: its bodies; internal node: its <= 8
// children) into the node's FP64 monopoles and FP32 walk records. lacc: the
// calling thread's per-species leaf sums {m, m x, m y, m z} (physical units),
// addressed by the body's species: no FP64 instruction is spent on the
// species a body does not have (predicated per-species sums would issue D
// times as many, and FP64 issues at 1/64 of the FP32 rate here).
template <int D>
__device__ __forceinline__ void mono_node(int lvl, uint32_t k, const MonoArgs& a,
                                          double (*lacc)[4][kMonoThreads], int tid) {
  double cen[3], side;
  node_centre(lvl, a.prefix[k], cen, &side);
  double sm[D], sx[D], sy[D], sz[D];
  uint32_t sc[D];
#pragma unroll
  for (int t = 0; t < D; ++t) { sm[t] = sx[t] = sy[t] = sz[t] = 0.0; sc[t] = 0; }
  const uint32_t nch = a.nchild[k];
  const uint32_t f = a.first[k], c = a.count[k];
  if (nch == 0) {
#pragma unroll
    for (int q = 0; q < D; ++q)
#pragma unroll
      for (int j = 0; j < 4; ++j) lacc[q][j][tid] = 0.0;
    // leaf centre in physical units; body records are offsets from it in box units
    const double cxL = cen[0] * a.L, cyL = cen[1] * a.L, czL = cen[2] * a.L;
    const float invLf = (float)a.invL;
    for (uint32_t b = f; b < f + c; ++b) {
      const double xp = a.spos[b], yp = a.spos[a.n + b], zp = a.spos[2 * a.n + b];
      const float m = a.smass[b];
      const int t = a.stype[b];
      a.body[b] = make_float4((float)(xp - cxL) * invLf, (float)(yp - cyL) * invLf,
                              (float)(zp - czL) * invLf, m);
      a.bleaf[b] = k;
      const double md = (double)m;
      lacc[t][0][tid] += md;
      lacc[t][1][tid] = fma(md, xp, lacc[t][1][tid]);
      lacc[t][2][tid] = fma(md, yp, lacc[t][2][tid]);
      lacc[t][3][tid] = fma(md, zp, lacc[t][3][tid]);
#pragma unroll
      for (int q = 0; q < D; ++q) sc[q] += t == q ? 1u : 0u;
    }
    // to box units (exact when the box is a power of two)
#pragma unroll
    for (int q = 0; q < D; ++q) {
      sm[q] = lacc[q][0][tid];
      sx[q] = lacc[q][1][tid] * a.invL;
      sy[q] = lacc[q][2][tid] * a.invL;
      sz[q] = lacc[q][3][tid] * a.invL;
    }
  } else {
    const uint32_t c0 = a.child[k];
    for (uint32_t j = 0; j < nch; ++j) {
      const uint32_t ch = c0 + j;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const double4_32a v = *reinterpret_cast<const double4_32a*>(a.m64 + ((size_t)ch * D + q) * 4);
        sm[q] += v.x;
        sx[q] += v.y;
        sy[q] += v.z;
        sz[q] += v.w;
        sc[q] += a.cnt[(size_t)ch * D + q];
      }
    }
  }
  double mt = 0, xt = 0, yt = 0, zt = 0;
#pragma unroll
  for (int q = 0; q < D; ++q) {
    // 32-byte records from a cudaMalloc base: one aligned 32-byte access each
    *reinterpret_cast<double4_32a*>(a.m64 + ((size_t)k * D + q) * 4) =
        make_double4_32a(sm[q], sx[q], sy[q], sz[q]);
    a.cnt[(size_t)k * D + q] = sc[q];
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (sm[q] > 0.0) {
      const float im = 1.0f / (float)sm[q];
      r = make_float4((float)fma(-sm[q], cen[0], sx[q]) * im, (float)fma(-sm[q], cen[1], sy[q]) * im,
                      (float)fma(-sm[q], cen[2], sz[q]) * im, (float)sm[q]);
    }
    a.mono[(size_t)k * D + q] = r;
    mt += sm[q];
    xt += sx[q];
    yt += sy[q];
    zt += sz[q];
  }
  a.geo[k] = make_float4((float)cen[0], (float)cen[1], (float)cen[2], (float)(0.5 * side));
  float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
  if (mt > 0.0) {
    const float im = 1.0f / (float)mt;
    r = make_float4((float)fma(-mt, cen[0], xt) * im, (float)fma(-mt, cen[1], yt) * im,
                    (float)fma(-mt, cen[2], zt) * im, (float)mt);
  }
  a.com[k] = r;
  a.link[k] = make_int4(nch ? (int)a.child[k] : -1, (int)nch, (int)f, (int)c);
}

// Trees of kBinnedMonoBodies bodies or more: one thread per node, in an
// order binned by the node's work. A leaf loops over its bodies and an
// internal node over its children, so a warp runs as long as its longest
// loop; FP64 issues at 1/64 of the FP32 rate here and a warp instruction
// costs the same with idle lanes. Taken in level (Morton) order, the leaves
// of a warp hold 1 to leaf_size bodies and a warp ran 2.5 times the
// iterations its bodies need (2^24 clustered bodies, leaf 32); binned, the
// threads of a warp have equal loop counts. All leaves are reduced by one
// launch (a leaf needs no other node), then the internal nodes level by
// level, bottom-up. Each node is still summed by one thread in its own order,
// so the results do not depend on the binning.
static_assert(kMonoBins <= 256, "the bin scan takes one bin per thread of a 256-thread block");

__device__ __forceinline__ int mono_bin(uint32_t lvl, uint32_t nch, uint32_t cnt) {
  return nch == 0 ? (int)min(cnt, (uint32_t)(kLeafBins - 1)) : kLeafBins + (int)lvl * 8 + (int)nch - 1;
}

// bins[0, kMonoBins): nodes per bin (zeroed before the launch)
__global__ void __launch_bounds__(256) k_mono_hist(uint32_t* status, int64_t cap,
                                                   const uint8_t* __restrict__ level,
                                                   const uint8_t* __restrict__ nchild,
                                                   const uint32_t* __restrict__ count, uint32_t* bins) {
  __shared__ uint32_t h[kMonoBins];
  if (status[ST_FLAGS] & SF_NODE_OVERFLOW) return;   // truncated tree: do not read it
  for (int i = threadIdx.x; i < kMonoBins; i += blockDim.x) h[i] = 0;
  __syncthreads();
  uint32_t total = levels_of(status).start[kMaxLevel + 1];
  if (total > cap) total = (uint32_t)cap;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x)
    atomicAdd(&h[mono_bin(level[k], nchild[k], count[k])], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kMonoBins; i += blockDim.x)
    if (h[i]) atomicAdd(&bins[i], h[i]);
}

// order[]: node indices grouped by bin. bins[kMonoBins, 2 kMonoBins): cursors
// (zeroed before the launch); block 0 writes the bin starts to
// bins[2 kMonoBins, 3 kMonoBins] (the last entry: all nodes). Each block
// places one contiguous chunk of nodes, reserving its share of every bin with
// one atomic per bin. Launched with 256 threads.
__global__ void __launch_bounds__(256) k_mono_order(uint32_t* status, int64_t cap,
                                                    const uint8_t* __restrict__ level,
                                                    const uint8_t* __restrict__ nchild,
                                                    const uint32_t* __restrict__ count, uint32_t* bins,
                                                    uint32_t* order) {
  __shared__ uint32_t lh[kMonoBins];
  __shared__ uint32_t base[kMonoBins];
  __shared__ uint32_t warp_tot[8];
  __shared__ uint32_t all;
  if (status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  const int tid = threadIdx.x;
  // bin starts: exclusive scan of the bin counts
  const uint32_t v = tid < kMonoBins ? bins[tid] : 0u;
  const uint32_t inc = block_inclusive_scan<256>(v, warp_tot, &all);
  if (tid < kMonoBins) {
    base[tid] = inc - v;
    lh[tid] = 0;
    if (blockIdx.x == 0) bins[2 * kMonoBins + tid] = inc - v;
  }
  if (blockIdx.x == 0 && tid == 0) bins[3 * kMonoBins] = all;
  __syncthreads();
  uint32_t total = levels_of(status).start[kMaxLevel + 1];
  if (total > cap) total = (uint32_t)cap;
  const uint32_t chunk = (total + gridDim.x - 1) / gridDim.x;
  const uint32_t k0 = min(total, blockIdx.x * chunk), k1 = min(total, k0 + chunk);
  for (uint32_t k = k0 + tid; k < k1; k += blockDim.x)
    atomicAdd(&lh[mono_bin(level[k], nchild[k], count[k])], 1u);
  __syncthreads();
  if (tid < kMonoBins && lh[tid]) base[tid] += atomicAdd(&bins[kMonoBins + tid], lh[tid]);
  __syncthreads();
  for (uint32_t k = k0 + tid; k < k1; k += blockDim.x)
    order[atomicAdd(&base[mono_bin(level[k], nchild[k], count[k])], 1u)] = k;
}

// Trees below kBinnedMonoBodies bodies: one launch per level, bottom-up, one
// thread per node of the level in level order. Their levels hold few nodes,
// so the three launches of the binned order cost more than its convergence
// saves (batches of 2^12..2^18-body simulations: 7.74 against 8.11 ms).
template <int D>
__global__ void __launch_bounds__(kMonoThreads) k_monopoles(int lvl, MonoArgs a) {
  __shared__ double lacc[D][4][kMonoThreads];
  if (a.status[ST_FLAGS] & SF_NODE_OVERFLOW) return;   // truncated tree: do not read it
  Levels lv = levels_of(a.status);
  const uint32_t s = lv.start[lvl];
  uint32_t e = lv.start[lvl + 1];
  if (e > a.cap) e = (uint32_t)a.cap;
  for (uint32_t k = s + blockIdx.x * blockDim.x + threadIdx.x; k < e; k += gridDim.x * blockDim.x)
    mono_node<D>(lvl, k, a, lacc, threadIdx.x);
}

// Every leaf of the tree: order[0, start of the first internal bin).
template <int D>
__global__ void __launch_bounds__(kMonoThreads) k_mono_leaves(MonoArgs a, const uint32_t* __restrict__ bins,
                                                              const uint32_t* __restrict__ order) {
  __shared__ double lacc[D][4][kMonoThreads];
  if (a.status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  const uint32_t e = bins[2 * kMonoBins + kLeafBins];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) {
    const uint32_t k = order[i];
    mono_node<D>(a.level[k], k, a, lacc, threadIdx.x);
  }
}

// The internal nodes of level lvl (their children are done).
template <int D>
__global__ void __launch_bounds__(kMonoThreads) k_mono_internal(int lvl, MonoArgs a,
                                                                const uint32_t* __restrict__ bins,
                                                                const uint32_t* __restrict__ order) {
  __shared__ double lacc[D][4][kMonoThreads];
  if (a.status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  const uint32_t* start = bins + 2 * kMonoBins + kLeafBins + lvl * 8;
  const uint32_t s = start[0], e = start[8];
  for (uint32_t i = s + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x)
    mono_node<D>(lvl, order[i], a, lacc, threadIdx.x);
}

// Every level of a small tree, bottom-up, in one launch: one cluster of
// kClusterBlocks blocks with the hardware cluster barrier between levels.
template <int D>
__global__ void __cluster_dims__(kClusterBlocks, 1, 1) __launch_bounds__(kMonoThreads)
k_monopoles_cluster(int lmax, MonoArgs a) {
  __shared__ double lacc[D][4][kMonoThreads];
  // the flag is read before any level and never written here: every block
  // returns, or none does
  if (a.status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  Levels lv = levels_of(a.status);
  for (int l = lmax; l >= 0; --l) {
    const uint32_t s = lv.start[l];
    uint32_t e = lv.start[l + 1];
    if (e > a.cap) e = (uint32_t)a.cap;
    for (uint32_t k = s + blockIdx.x * blockDim.x + threadIdx.x; k < e; k += gridDim.x * blockDim.x)
      mono_node<D>(l, k, a, lacc, threadIdx.x);
    cluster.sync();
  }
}

int reduce_monopoles(ng_ctx* c) {
  MonoArgs a;
  a.level = as<uint8_t>(c->n_level);
  a.prefix = as<uint64_t>(c->n_prefix);
  a.first = as<uint32_t>(c->n_first);
  a.count = as<uint32_t>(c->n_count);
  a.nchild = as<uint8_t>(c->n_nchild);
  a.child = as<uint32_t>(c->n_child);
  a.spos = as<double>(c->spos);
  a.smass = as<float>(c->smass);
  a.stype = as<uint8_t>(c->stype);
  a.m64 = as<double>(c->n_m64);
  a.cnt = as<uint32_t>(c->n_cnt);
  a.geo = as<float4>(c->n_geo);
  a.com = as<float4>(c->n_com);
  a.link = as<int4>(c->n_link);
  a.mono = as<float4>(c->n_mono);
  a.body = as<float4>(c->body);
  a.bleaf = as<uint32_t>(c->bleaf);
  a.status = as<uint32_t>(c->status);
  a.n = c->n;
  a.cap = c->cap_nodes;
  a.invL = 1.0 / c->L;
  a.L = c->L;
  const int lmax = std::min(std::max(c->level_cap, 0), kMaxLevel);   // deeper levels are empty
  stage_mark(c, NG_STAGE_MONOPOLES);
  if (c->n <= kClusterMaxBodies) {
    switch (c->p.D) {
      case 1: k_monopoles_cluster<1><<<kClusterBlocks, kMonoThreads, 0, c->stream>>>(lmax, a); break;
      case 2: k_monopoles_cluster<2><<<kClusterBlocks, kMonoThreads, 0, c->stream>>>(lmax, a); break;
      case 3: k_monopoles_cluster<3><<<kClusterBlocks, kMonoThreads, 0, c->stream>>>(lmax, a); break;
      case 4: k_monopoles_cluster<4><<<kClusterBlocks, kMonoThreads, 0, c->stream>>>(lmax, a); break;
      case 5: k_monopoles_cluster<5><<<kClusterBlocks, kMonoThreads, 0, c->stream>>>(lmax, a); break;
      default: k_monopoles_cluster<6><<<kClusterBlocks, kMonoThreads, 0, c->stream>>>(lmax, a); break;
    }
    c->launches += 1;
    NG_CUDA(c, cudaGetLastError());
    return NG_OK;
  }
  if (c->n < kBinnedMonoBodies) {
    c->launches += lmax + 1;
    for (int l = lmax; l >= 0; --l) {
      const int64_t nodes = std::min<int64_t>(c->cap_nodes, level_bound(l, c->n));
      const int grid = (int)std::max<int64_t>(
          1, std::min<int64_t>((int64_t)c->nsm * 16, (nodes + kMonoThreads - 1) / kMonoThreads));
      switch (c->p.D) {
        case 1: k_monopoles<1><<<grid, kMonoThreads, 0, c->stream>>>(l, a); break;
        case 2: k_monopoles<2><<<grid, kMonoThreads, 0, c->stream>>>(l, a); break;
        case 3: k_monopoles<3><<<grid, kMonoThreads, 0, c->stream>>>(l, a); break;
        case 4: k_monopoles<4><<<grid, kMonoThreads, 0, c->stream>>>(l, a); break;
        case 5: k_monopoles<5><<<grid, kMonoThreads, 0, c->stream>>>(l, a); break;
        default: k_monopoles<6><<<grid, kMonoThreads, 0, c->stream>>>(l, a); break;
      }
    }
    NG_CUDA(c, cudaGetLastError());
    return NG_OK;
  }
  // the tree build's per-level scratch (n_tmp, one word per node) is free
  // once the tree is built: it holds the binned node order
  uint32_t* bins = as<uint32_t>(c->mono_bins);
  uint32_t* order = as<uint32_t>(c->n_tmp);
  NG_CUDA(c, cudaMemsetAsync(bins, 0, 2 * kMonoBins * sizeof(uint32_t), c->stream));
  const int sgrid = work_grid(c, c->cap_nodes, 4);
  k_mono_hist<<<sgrid, 256, 0, c->stream>>>(a.status, a.cap, a.level, a.nchild, a.count, bins);
  k_mono_order<<<sgrid, 256, 0, c->stream>>>(a.status, a.cap, a.level, a.nchild, a.count, bins, order);
  const int lgrid = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)c->nsm * 16, (c->cap_nodes + kMonoThreads - 1) / kMonoThreads));
  switch (c->p.D) {
    case 1: k_mono_leaves<1><<<lgrid, kMonoThreads, 0, c->stream>>>(a, bins, order); break;
    case 2: k_mono_leaves<2><<<lgrid, kMonoThreads, 0, c->stream>>>(a, bins, order); break;
    case 3: k_mono_leaves<3><<<lgrid, kMonoThreads, 0, c->stream>>>(a, bins, order); break;
    case 4: k_mono_leaves<4><<<lgrid, kMonoThreads, 0, c->stream>>>(a, bins, order); break;
    case 5: k_mono_leaves<5><<<lgrid, kMonoThreads, 0, c->stream>>>(a, bins, order); break;
    default: k_mono_leaves<6><<<lgrid, kMonoThreads, 0, c->stream>>>(a, bins, order); break;
  }
  // nodes at level lmax are leaves
  c->launches += 3 + lmax;
  for (int l = lmax - 1; l >= 0; --l) {
    const int64_t nodes = std::min<int64_t>(c->cap_nodes, level_bound(l, c->n));
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)c->nsm * 16, (nodes + kMonoThreads - 1) / kMonoThreads));
    switch (c->p.D) {
      case 1: k_mono_internal<1><<<grid, kMonoThreads, 0, c->stream>>>(l, a, bins, order); break;
      case 2: k_mono_internal<2><<<grid, kMonoThreads, 0, c->stream>>>(l, a, bins, order); break;
      case 3: k_mono_internal<3><<<grid, kMonoThreads, 0, c->stream>>>(l, a, bins, order); break;
      case 4: k_mono_internal<4><<<grid, kMonoThreads, 0, c->stream>>>(l, a, bins, order); break;
      case 5: k_mono_internal<5><<<grid, kMonoThreads, 0, c->stream>>>(l, a, bins, order); break;
      default: k_mono_internal<6><<<grid, kMonoThreads, 0, c->stream>>>(l, a, bins, order); break;
    }
  }
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

// ------------------------------------------------------------- groups

// Walk groups: runs of consecutive sibling cells holding <= S bodies each
// (and <= S together) whose parent holds more than S, each run cut into
// ceil(c / G) contiguous chunks of balanced size; leaves with more than S
// bodies are cut the same way. Every body lands in exactly one group, so a
// group is named by its first body: gsize[first] = body count (zero
// elsewhere). A flag scan then numbers the groups in body (Morton) order,
// so that warps taking consecutive groups walk neighbouring regions and
// share the nodes they fetch in L2.
__global__ void k_groups(uint32_t* status, int64_t cap, int G, int S,
                         const uint32_t* __restrict__ first,
                         const uint32_t* __restrict__ count, const uint8_t* __restrict__ nchild,
                         const uint32_t* __restrict__ child, uint32_t* gsize) {
  if (status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  Levels lv = levels_of(status);
  uint32_t total = lv.start[kMaxLevel + 1];
  if (total > cap) total = (uint32_t)cap;
  auto emit = [&](uint32_t f, uint32_t c) { gsize[f] = c; };
  auto emit_chunks = [&](uint32_t f, uint32_t c) {
    const uint32_t k = (c + G - 1) / G, base = c / k, rem = c % k;
    for (uint32_t j = 0, o = 0; j < k; ++j) {
      const uint32_t len = base + (j < rem ? 1u : 0u);
      emit(f + o, len);
      o += len;
    }
  };
  const uint32_t SS = (uint32_t)S;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += gridDim.x * blockDim.x) {
    const uint32_t c = count[k];
    if (k == 0 && c <= SS) { emit_chunks(first[0], c); continue; }
    if (c <= SS) continue;
    const uint32_t nch = nchild[k];
    if (nch == 0) {
      if (k == 0) emit_chunks(first[0], c);
      continue;
    }
    uint32_t bf = 0, bc = 0;
    for (uint32_t j = 0; j < nch; ++j) {
      const uint32_t ch = child[k] + j;
      const uint32_t cc = count[ch];
      if (cc > SS) {
        if (bc) { emit_chunks(bf, bc); bc = 0; }
        if (nchild[ch] == 0) emit_chunks(first[ch], cc);
        continue;
      }
      if (bc + cc > SS) { emit_chunks(bf, bc); bc = 0; }
      if (bc == 0) bf = first[ch];
      bc += cc;
    }
    if (bc) emit_chunks(bf, bc);
  }
}

// groups[rank[b]] = (b, gsize[b]) for every group start b.
__global__ void k_group_compact(int64_t n, const uint32_t* __restrict__ gsize,
                                const uint32_t* __restrict__ rank, int2* __restrict__ groups) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n;
       b += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t s = gsize[b];
    if (s) groups[rank[b]] = make_int2((int)b, (int)s);
  }
}

int build_groups(ng_ctx* c) {
  const int64_t n = c->n;
  NG_TRY(ensure(c, c->groups, (size_t)n * sizeof(int2)));
  NG_TRY(ensure(c, c->gsize, (size_t)n * sizeof(uint32_t)));
  NG_TRY(ensure(c, c->grank, (size_t)n * sizeof(uint32_t)));
  uint32_t* gsize = as<uint32_t>(c->gsize);
  uint32_t* grank = as<uint32_t>(c->grank);
  stage_mark(c, NG_STAGE_GROUPS);
  NG_CUDA(c, cudaMemsetAsync(gsize, 0, (size_t)n * sizeof(uint32_t), c->stream));
  c->launches += 2;   // groups, compaction (the flag scan counts itself)
  k_groups<<<work_grid(c, std::min<int64_t>(c->cap_nodes, 2 * n + 64), 4), 256, 0, c->stream>>>(
      as<uint32_t>(c->status), c->cap_nodes, c->p.group_size, c->p.group_cell,
      as<uint32_t>(c->n_first),
      as<uint32_t>(c->n_count), as<uint8_t>(c->n_nchild), as<uint32_t>(c->n_child), gsize);
  NG_CUDA(c, cudaGetLastError());
  NG_TRY(scan_u32_flags(c, gsize, grank, n, as<uint32_t>(c->status) + ST_NGROUPS));
  k_group_compact<<<work_grid(c, n, 8), 256, 0, c->stream>>>(n, gsize, grank,
                                                          as<int2>(c->groups));
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

}  // namespace ng
