// Internal declarations of the ngravs CUDA library (not part of the ABI).
#pragma once

#include <cmath>

#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <string>
#include <mutex>
#include <vector>

#include "../../include/ngravs.h"

namespace ng {

// ----------------------------------------------------------------- limits
constexpr int kMaxD = NG_MAX_SPECIES;
constexpr int kMaxLevel = 20;           // 20 Morton bits per axis
constexpr int kCapturedDepthMargin = 2;  // captured steps build this far below the depth seen
// Trees of at most kClusterMaxBodies bodies are built, and their monopoles
// reduced, by one launch each: a cluster of kClusterBlocks blocks that runs
// every level with the hardware cluster barrier between levels (larger trees:
// one launch per level and phase, over the whole GPU).
constexpr int kClusterBlocks = 8;
constexpr int64_t kClusterMaxBodies = 32768;
// Monopoles of trees of kBinnedMonoBodies bodies or more are reduced in an
// order binned by the work of a node: leaves by body count (0..64, one more
// bin for the larger leaves of a tree stopped at a level cap), internal nodes
// by level and child count.
constexpr int kLeafBins = 66;
constexpr int kMonoBins = kLeafBins + (kMaxLevel + 1) * 8;
constexpr int64_t kBinnedMonoBodies = 1 << 20;   // smaller trees: level order
constexpr int kWarp = 32;

// Status words in device memory (ctx->status).
enum StatusSlot {
  ST_FLAGS = 0,          // bit flags below
  ST_NODES_NEEDED = 1,   // node count the last build asked for
  ST_NGROUPS = 2,        // walk groups of the last build
  ST_WORK = 3,           // walk work-queue counter
  ST_LEVELS = 8,         // 22 level starts (levels 0..20, then end) + 21 level counts
  ST_COUNT = 64
};
enum StatusFlag {
  SF_NODE_OVERFLOW = 1,
  SF_STACK_OVERFLOW = 2,
  SF_GROUP_OVERFLOW = 4,
  SF_BAD_TREE = 8,
  SF_BAD_TYPE = 16,
  // not an error: a build with a level cap (captured steps) kept a node at
  // the cap whose body count is above the leaf size as a leaf. The tree is
  // valid (leaves of any size are walked, summed and grouped) but not the
  // canonical one; the caller captures its steps again, deeper.
  SF_DEPTH = 32
};
static_assert(ST_LEVELS + (kMaxLevel + 2) + (kMaxLevel + 1) <= ST_COUNT, "status block too small");

// Growable device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Walk tuning constants.
constexpr int kStackCap = 384;          // node stack entries per warp
constexpr int kStackReserve = 7 * kMaxLevel + 8 + 32;   // depth-first descent + push-backs
constexpr int kWalkMaxWarps = 32;
// Warps per walk block by species count: as many as the per-warp lists and a
// 64 KB law table leave room for in 227 KB of shared memory; the register
// budget follows (65536 / threads).
// Every third bit of v, from bit 0, packed into the low 21 bits: one axis
// of a Morton key or node prefix (x from v >> 2, y from v >> 1, z from v).
__device__ __forceinline__ uint32_t morton_compact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (uint32_t)v;
}

// (2 i + 1) 2^-(lvl + 1), the centre of cell i of level lvl in box units:
// exact in FP64, and formed from its bits with integer operations only
// (FP64 issues at 1/64 of the FP32 rate here).
__device__ __forceinline__ double cell_centre(uint32_t i, int lvl) {
  const uint32_t v = 2u * i + 1u;            // odd, below 2^22
  const int p = 31 - __clz(v);               // v = 1.f 2^p
  const uint64_t mant = ((uint64_t)v << (52 - p)) & ((1ull << 52) - 1);
  return __longlong_as_double((long long)(((uint64_t)(1023 + p - (lvl + 1)) << 52) | mant));
}

// Centre (box units) and side 2^-lvl of a node from its level and Morton prefix.
__device__ __forceinline__ void node_centre(int lvl, uint64_t pre, double c[3], double* side) {
  c[0] = cell_centre(morton_compact3(pre >> 2), lvl);
  c[1] = cell_centre(morton_compact3(pre >> 1), lvl);
  c[2] = cell_centre(morton_compact3(pre), lvl);
  *side = __longlong_as_double((long long)(1023 - lvl) << 52);
}

// A box-unit offset wrapped to its nearest periodic image, rounded once.
__device__ __forceinline__ double nearest_image_unit(double d) { return __dsub_rn(d, rint(d)); }

// ------------------------------------------------------------------ keys
// Wrap, quantisation and interleaving of the sort keys (Sec. 2.4), shared by
// every kernel that forms keys so that all of them round identically.

// x / L rounded once. For a power-of-two L the product with 1/L is the same
// number (both exact), and FP64 division costs ~10 FP64 operations here.
__device__ __forceinline__ double div_box(double x, double L, double invL, bool pow2) {
  return pow2 ? __dmul_rn(x, invL) : __ddiv_rn(x, L);
}

// Periodic wrap x - L floor(x / L) with each operation rounded separately
// (no fused multiply-add), so that the host reference rounds identically.
// FP64 issues at 1/64 of the FP32 rate here, so for a power-of-two box the
// common case is decided on the bits: a non-negative double orders like its
// bit pattern, and for x in [+0, L) x / L is exact and below 1, so the wrap
// returns x itself.
__device__ __forceinline__ double wrap_box(double x, double L, double invL, bool pow2) {
  if (pow2) {
    const long long b = __double_as_longlong(x);
    if (b >= 0 && b < __double_as_longlong(L)) return x;
  }
  const double f = floor(div_box(x, L, invL, pow2));
  return __dsub_rn(x, __dmul_rn(L, f));
}

// floor(w / L * 2^20) clamped to [0, 2^20 - 1]. For a box L = 2^ebox the
// scaled value is w * 2^(20 - ebox) exactly, and its integer part is read
// from the exponent and mantissa bits (the same number the FP64 formula
// gives, without FP64 instructions).
__device__ __forceinline__ uint64_t quantise20(double w, double L, double invL, bool pow2,
                                               int ebox) {
  if (pow2) {
    const long long b = __double_as_longlong(w);
    const int e = (int)((b >> 52) & 0x7ff);
    if (b <= 0) return 0;                        // +0, -0 and negative w
    if (e != 0x7ff) {                            // finite w > 0
      const int sh = e - 1023 + 20 - ebox;      // w * 2^(20 - ebox) = 1.m * 2^sh
      if (sh < 0) return 0;
      if (sh >= 20) return 1048575;
      const uint64_t m = ((uint64_t)b & ((1ull << 52) - 1)) | (1ull << 52);
      return m >> (52 - sh);
    }
  }
  double q = floor(__dmul_rn(div_box(w, L, invL, pow2), 1048576.0));
  q = q < 0.0 ? 0.0 : q;
  q = q > 1048575.0 ? 1048575.0 : q;
  return (uint64_t)q;
}

// Spread the low 21 bits of v to every third bit.
__device__ __forceinline__ uint64_t spread3(uint64_t v) {
  v &= 0x1fffffull;
  v = (v | (v << 32)) & 0x1f00000000ffffull;
  v = (v | (v << 16)) & 0x1f0000ff0000ffull;
  v = (v | (v << 8)) & 0x100f00f00f00f00full;
  v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
  v = (v | (v << 2)) & 0x1249249249249249ull;
  return v;
}

// The sort key of one body: (Morton(q_x, q_y, q_z) << 3) | species, x most
// significant, q = floor((x mod L) / L * 2^20) clamped to [0, 2^20 - 1].
__device__ __forceinline__ uint64_t sort_key(double x, double y, double z, uint8_t type, double L,
                                             double invL, bool pow2, int ebox) {
  const uint64_t qx = quantise20(wrap_box(x, L, invL, pow2), L, invL, pow2, ebox);
  const uint64_t qy = quantise20(wrap_box(y, L, invL, pow2), L, invL, pow2, ebox);
  const uint64_t qz = quantise20(wrap_box(z, L, invL, pow2), L, invL, pow2, ebox);
  const uint64_t m = (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
  return (m << 3) | (uint64_t)(type & 7);
}

// Keys per block of the radix sort; the per-block digit histograms (and the
// type offsets read back from the last pass's) are laid out by it.
constexpr int kRadixTile = 2048;

// Entries per row of a single simulation's law table: the passive species
// count rounded up to a power of two (a row of the table of list species t
// holds the law of every passive species s; see walk_table).
__host__ __device__ constexpr int walk_tab_pad(int D) { return D <= 1 ? 1 : D == 2 ? 2 : D <= 4 ? 4 : 8; }
__host__ __device__ constexpr int walk_tab_shift(int D) { return D <= 1 ? 0 : D == 2 ? 1 : D <= 4 ? 2 : 3; }

// Warps per walk block (one block per SM): registers and the per-warp lists
// bound them. The variable-species instance of batches, laid out for six
// species, runs 24 warps when its law table is small (a few distinct laws).
__host__ __device__ constexpr int walk_warps(int D) { return D <= 3 ? 24 : D == 4 ? 24 : D == 5 ? 20 : 16; }
constexpr int kVardWarps = 24;
// Records per species list per warp: as many as fit beside the default law
// table at the walk's warp count. A list is evaluated once the next round of
// up to 32 appends could overflow it, so longer lists spread each
// evaluation's fixed cost over more records (the 2^24 D = 4 walk: 65.8 ms
// with 64, 64.7 ms with 80); the variable-species instance of batches,
// laid out for six species at 24 warps, keeps 64.
__host__ __device__ constexpr int walk_list_cap(int D, bool vard) {
  return vard ? 64 : D <= 2 ? 128 : D == 3 ? 96 : D == 4 ? 80 : D == 5 ? 64 : 72;
}

// Per-simulation inputs of the walk (device memory, one per simulation).
// The law table of a walk launch (device copy).
// (batch classes: one row of segments per distinct law of the members)
struct WalkTable {
  const float2* tab;        // [law][ncut + 1] segments {c0 - k c1, c1}
  int ncut;
  int count;                // float2 entries
};

struct __align__(16) WalkDesc {
  const float4* geo;        // [node] centre (box units), half side
  const float4* com;        // [node] all-species centre of mass - centre, total mass
  const int4* link;         // [node] child_first, nchild, body_first, body_count
  const float4* mono;       // [node][D] species com - centre, species mass
  const float4* body;       // [sorted body] offset from its leaf centre, mass
  const uint8_t* btype;     // [sorted body] species
  const uint32_t* bleaf;    // [sorted body] leaf node holding the body
  const int2* groups;       // [group] first body, count
  const uint32_t* perm;     // sorted -> caller index (previous accelerations are read there)
  const uint32_t* out;      // sorted -> output index of acc (nullptr: sorted order)
  uint32_t* status;         // device status words of the simulation
  float* acc;               // [3][n] output order
  int64_t n;
  int accumulate;           // add into acc instead of overwriting
  float s_tab;              // table units per box unit
  float rcut_box;           // cut-off in box units
  float theta2;
  float eps2_tab;           // softening^2 in table units^2
  float out_scale;          // converts accumulated table-unit sums to acceleration
  int8_t tabid[kMaxD][kMaxD];
  float G[kMaxD][kMaxD];
  const float* aold;        // relative criterion: |a_old| per caller index (nullptr: geometric)
  float rel_scale;          // alpha L^2 / G_max (box units)
  int D;                    // species of the simulation (launches over several species counts)
};

// Kernel parameters of one walk launch over one or more simulations that
// share the species count and the law table.
struct WalkLaunch {
  const WalkDesc* descs;
  int ndesc;
  const uint32_t* gprefix;  // [ndesc + 1] group prefix
  uint32_t* work;           // work-queue counter
  // law table, segments {c0 - k c1, c1}: single simulations
  // [list species t][ncut + 1][walk_tab_pad(D)] (entry s: passive species s);
  // variable-species launches [law][ncut + 1] (a lane's row: tabid[s][t])
  const float2* tab;
  int tab_entries;          // ncut + 1
  int ncut;
  int tab_count;            // float2 entries of the whole table
  unsigned long long* counter;  // executed interaction counter (optional)
};

}  // namespace ng

// Opaque context (defined here, declared in the public header).
struct ng_ctx {
  ng_params p{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int nsm = 0;
  size_t smem_optin = 0;
  std::string err;

  // derived geometry
  double L = 1.0, rs = 0, rcut = 0;

  // short-range tables
  int nlaws = 0, ncut = 0;
  int8_t tabid[ng::kMaxD][ng::kMaxD]{};
  double dr_phys = 0;                 // table spacing (physical length)
  ng::DevBuf d_tab;
  std::vector<float> h_tab;           // host copy (tables of a batch are matched on it)
  void* h_tab_pinned = nullptr;       // pinned staging copy of the table upload
  size_t h_tab_pinned_bytes = 0;

  // particles of the last build
  int64_t n = 0;
  bool built = false;
  ng::DevBuf keys_a, keys_b, vals_a, vals_b, blockhist;
  ng::DevBuf spos, smass, stype, body, bleaf, tperm, scan_part;

  // tree
  int64_t cap_nodes = 0, nnodes = 0;
  int level_cap = ng::kMaxLevel;   // deepest level a build emits (captured steps: depth_seen + 2)
  int depth_seen = ng::kMaxLevel;  // deepest non-empty level of the last checked build
  int sort_passes = 0;             // radix passes of the last key sort
  int64_t ngroups = 0, ngroups_n = -1;   // walk groups of the last checked build, for n = ngroups_n
  ng::DevBuf n_level, n_prefix, n_first, n_count, n_child, n_nchild, n_tmp;
  ng::DevBuf n_m64, n_cnt, n_geo, n_com, n_link, n_mono;
  ng::DevBuf mono_bins;   // uint32[3 kMonoBins + 1]: nodes, cursors and starts per monopole bin
  ng::DevBuf groups;
  ng::DevBuf gsize, grank;          // group size at its first body, rank of each group start
  ng::DevBuf status;     // uint32[ST_COUNT]
  ng::DevBuf walk_desc, walk_prefix;
  ng::DevBuf counter;    // unsigned long long
  ng::DevBuf io_pos, io_vel, io_type, io_mass, io_acc;   // device copies for ng_step_host
  ng::DevBuf lattice;    // float4[nlaws][(N+1)^3] lattice corrections (pure tree mode 2)
  int lattice_grid = 0;  // N of the lattice tables (0: none)
  ng::DevBuf aold;       // float[n] |previous acceleration| per body (caller order)
  int64_t aold_n = -1;   // bodies aold holds (-1: none)

  // resident state of ng_step: between steps the bodies stay in the sorted
  // order of the previous step. (spos, smass, stype) with rvel, rorig (the
  // caller index of each body) and racc hold the current state; each step
  // swaps them with their *_alt partners, gathers the previous state into
  // sorted order and writes the forces in that order.
  bool resident = false;
  ng::DevBuf spos_alt, smass_alt, stype_alt, rvel, rvel_alt, rorig, rorig_alt, racc, rtmp;
  cudaGraphExec_t step_exec_b = nullptr;   // the step with the buffer roles exchanged
  int step_parity = 0;

  // PM: cuFFT plans cached per (mesh, species count); a context reused for
  // requests of other sizes keeps its plans
  struct Plan { int N, D; cufftHandle r2c, c2r; };
  std::vector<Plan> plans;
  cufftHandle plan_r2c = 0, plan_c2r = 0;   // the plans of the current (mesh, D)
  ng::DevBuf rho, rhok, phi;

  // stage timer of ng_stage_times: when on, each stage records its start event
  bool timing = false;
  uint32_t stage_seen = 0;       // stages marked during the current measurement
  cudaEvent_t stage_ev[NG_NSTAGES + 1]{};

  // kernels this library has launched (host-side count)
  uint64_t launches = 0;
  uint64_t graph_launches = 0;     // kernels in one captured step

  // step graph (captured on a private stream, replayed on the caller's)
  cudaStream_t cap_stream = nullptr;
  // captured steps run the PM stages on pm_stream beside the tree stages
  // (fork after the type-major order, join before the walk)
  cudaStream_t pm_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  uint64_t alloc_gen = 0;          // bumped whenever a device buffer is (re)allocated
  uint64_t graph_gen = 0;
  cudaGraphExec_t step_exec = nullptr;
  int64_t graph_n = -1;
  double graph_dt = 0;
};

namespace ng {

// Stage timer: record the start of stage s on the context's stream (a no-op
// unless ng_stage_times is measuring).
inline void stage_mark(ng_ctx* c, int s) {
  if (!c->timing) return;
  cudaEventRecord(c->stage_ev[s], c->stream);
  c->stage_seen |= 1u << s;
}

// Error helpers: record a message on ctx and return a code.
int fail(ng_ctx* c, int code, const char* fmt, ...);
#define NG_CUDA(c, call)                                                             \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      cudaGetLastError(); /* leave no stale error for the next call */               \
      return ::ng::fail((c), NG_ECUDA, "%s failed: %s (%s:%d)", #call,               \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                 \
    }                                                                                \
  } while (0)
#define NG_TRY(expr)                 \
  do {                               \
    int r_ = (expr);                 \
    if (r_ != NG_OK) return r_;      \
  } while (0)

// Ensure buf holds at least bytes (grows, contents not kept).
int ensure(ng_ctx* c, DevBuf& buf, size_t bytes);
void release(DevBuf& buf);

template <class T>
inline T* as(const DevBuf& b) { return static_cast<T*>(b.p); }

// Device-wide exclusive scan of uint32 values; len read from *d_len when
// d_len != nullptr (then len is an upper bound), total written to *d_total
// when non-null. Needs ctx->scan_part scratch.
int scan_u32_flags(ng_ctx* c, const uint32_t* in, uint32_t* out, int64_t len, uint32_t* d_total);
int scan_u32(ng_ctx* c, const uint32_t* in, uint32_t* out, int64_t len,
             const uint32_t* d_len, uint32_t* d_total);

// Stages of the pipeline (each enqueues on c->stream, no host sync).
int sort_bodies(ng_ctx* c, int64_t n, const double* pos, const uint8_t* type,
                const float* mass);
// Resident step's sort: keys of the state in *_alt, gather of positions,
// masses, species, velocities and caller indices into sorted order.
int sort_resident(ng_ctx* c, int64_t n);
// Output index of the force kernels: the caller order, or the sorted order
// while ng_step keeps the state resident.
const uint32_t* force_out(const ng_ctx* c);
// Resident state of ng_step (ng_api.cu).
int reserve_resident(ng_ctx* c, int64_t n);
void swap_resident(ng_ctx* c);
int resident_load(ng_ctx* c, int64_t n, const double* pos, const float* vel, const uint8_t* type,
                  const float* mass, const float* acc);
int resident_store(ng_ctx* c, int64_t n, double* pos, float* vel, float* acc);
int resident_step_once(ng_ctx* c, int64_t n, double dt, bool checked);
int build_octree(ng_ctx* c);                  // needs sorted bodies
int reduce_monopoles(ng_ctx* c);              // needs octree
int build_groups(ng_ctx* c);                  // needs octree
int launch_walk(ng_ctx* c, float* acc, bool accumulate, bool count);
void fill_walk_desc(ng_ctx* c, float* acc, bool accumulate, WalkDesc* d);
int64_t walk_groups_hint(const ng_ctx* c);
// One walk launch over ndesc simulations sharing the law table `tab` (the
// context's own when nullptr); vard: their species counts differ (the
// variable-D instance with lists and table for 6 species).
int launch_walk_descs(ng_ctx* c, cudaStream_t stream, const WalkDesc* d_descs, int ndesc,
                      uint32_t* d_prefix, uint32_t* d_work, unsigned long long* counter,
                      int64_t groups, bool rel, const WalkTable* tab = nullptr, bool vard = false);
// Walk descriptor with the table spacing of another table (batch classes).
void fill_walk_desc_dr(ng_ctx* c, float* acc, bool accumulate, double dr, WalkDesc* d);
int launch_count(ng_ctx* c, int64_t* counts);  // per-particle walk counts
// Direct mode (theta = 0, geometric opening, TreePM split): every pair within
// r_cut summed in FP64 (ng_direct.cu).
int launch_direct64(ng_ctx* c, float* acc, bool accumulate, bool count);
bool direct_mode(const ng_ctx* c);
// Pure tree mode: per-particle walk with the full laws (incl. Mahalo).
int launch_walk_exact(ng_ctx* c, float* acc, bool accumulate, bool count);
// The tree force of a context: the group walk, or in pure tree mode the exact walk.
int launch_tree_force(ng_ctx* c, float* acc, bool accumulate, bool count);
// Lattice-correction tables of pure tree mode 2, one per distinct law.
int build_lattice(ng_ctx* c, int nlaws, const int* kind, const double* a, const double* l);
// Relative opening criterion: active when the context asks for it and holds
// |a_old| for its current bodies; G_max of the law table; |acc| -> aold.
bool relative_active(const ng_ctx* c);
double coupling_max(const ng_ctx* c);
int update_aold(ng_ctx* c, const float* acc);
int pm_force(ng_ctx* c, float* acc, bool accumulate);
int pm_reserve(ng_ctx* c);                     // meshes and cuFFT plans of the context's mesh
int reserve_sort(ng_ctx* c, int64_t n);        // sort buffers for n bodies
// Every buffer and plan a force evaluation of n bodies needs (allocates on the
// calling thread; the stages that follow then allocate nothing).
int reserve(ng_ctx* c, int64_t n);
extern std::mutex g_fft_plan_lock;   // see pm_setup
int type_order(ng_ctx* c);

// Host short-range law tables (double precision closed forms).
int build_tables(ng_ctx* c);
// The linear segments of a context's distinct laws, [law][ncut + 1] float2
// (c->tabid numbers the laws), ncut segments of dr.
std::vector<float> law_segments(const ng_ctx* c, int ncut, double dr);
// The same segments laid out for the walk of a single simulation:
// [list species t][ncut + 1][walk_tab_pad(D)], entry s the law of (s, t).
std::vector<float> walk_table(const ng_ctx* c, int ncut, double dr);
int walk_table_entries(int D, int table_size);   // default segments per law for D species

// Short-range force factor T(rho) of Sec. 2.4.1 in FP64: the acceleration from
// a source of active mass M is G M T(rho) d / rho^3. Newtonian part:
// -rho^2 d/drho [erfc(rho / 2 r_s) / rho]. Yukawa part (Eq. (yukawa), C = 1,
// Sec. 3.2 long-range kernel scaled by exp(-mu^2 r_s^2)): the remaining
// real-space potential -a S(rho)/rho with
//   S = [e^{-mu rho} erfc(v - mu r_s) + e^{mu rho} erfc(v + mu r_s)] / 2,
// v = rho / 2 r_s, contributes a (S - rho dS/drho). The pure Yukawa law
// (C = 0, Sec. 3.2) has that part alone. The same function fills the host
// tables of the FP32 walk and evaluates the FP64 direct-mode sum.
__host__ __device__ inline double short_law_factor(int law, double a, double l, double rs,
                                                   double rho) {
  const double v = rho / (2.0 * rs);
  const double gauss = ::exp(-v * v);
  double T = law == NG_YUKAWA_PURE ? 0.0 : ::erfc(v) + (2.0 / ::sqrt(M_PI)) * v * gauss;
  if (law == NG_YUKAWA || law == NG_YUKAWA_PURE) {
    const double mu = 1.0 / l;
    const double lo = ::exp(-mu * rho) * ::erfc(v - mu * rs);
    const double ec = ::erfc(v + mu * rs);
    const double hi = ec > 0.0 ? ::exp(mu * rho + ::log(ec)) : 0.0;
    const double S = 0.5 * (lo + hi);
    const double dS = 0.5 * mu * (hi - lo) - gauss * ::exp(-mu * mu * rs * rs) / (rs * ::sqrt(M_PI));
    T += a * (S - rho * dS);
  }
  return T;
}

// Inclusive scan of one value per thread over a block of THREADS threads
// (warp shuffles, then the warp totals); *total receives the block's sum.

template <int THREADS>
__device__ __forceinline__ uint32_t block_inclusive_scan(uint32_t v, uint32_t* warp_tot,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < THREADS / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < THREADS / 32) warp_tot[lane] = w;
    if (lane == THREADS / 32 - 1) *total = w;
  }
  __syncthreads();
  if (wid > 0) v += warp_tot[wid - 1];
  return v;
}

// Blocks of 256 threads for a grid-stride kernel over `items` items: enough
// to cover them, at most per_sm blocks per SM, at least one.
int work_grid(ng_ctx* c, int64_t items, int per_sm);
// Upper bound on the nodes of tree level l: 8^l and the body count.
int64_t level_bound(int l, int64_t n);

// Pipeline pieces shared by the single-simulation calls and the batch
// runtime (ng_api.cu).
int build_checked(ng_ctx* c, int64_t n, const double* pos, const uint8_t* type, const float* mass);
int tree_checked(ng_ctx* c);                   // tree stages of the sorted bodies, capacity grown
int tree_stages(ng_ctx* c);
int force_stages(ng_ctx* c, float* acc);
int tree_force_overlapped(ng_ctx* c, float* acc);
int launch_kick(ng_ctx* c, int64_t n, float* vel, const float* acc, double h);
// nkick (1 or 2) kicks of h, then the drift (one launch, same rounding as the two)
int launch_kick_drift(ng_ctx* c, int64_t n, float* vel, const float* acc, double h, int nkick,
                      double* pos, double dt);
int alloc_nodes(ng_ctx* c, int64_t cap);
int read_status(ng_ctx* c, uint32_t* st);      // synchronises c->stream
int alloc_bodies(ng_ctx* c, int64_t n);
// (Re)configure an existing context for new parameters: validation and the
// law tables (uploaded on c->stream); buffers and cuFFT plans are kept.
int ctx_configure(ng_ctx* c, const ng_params* p);
// Host-only validation of a parameter block (message on c).
int validate(ng_ctx* c, const ng_params* p);
// Fill the defaults of a parameter block (leaf size, group size, group cell).
void normalize_params(ng_params* p);
void drop_step_graphs(ng_ctx* c);   // the captured steps of ng_step
int check_flags(ng_ctx* c, uint32_t flags);
bool box_is_pow2(double L);   // L = 2^k: x / L == x * (1 / L) exactly

}  // namespace ng
