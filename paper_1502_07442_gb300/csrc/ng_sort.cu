// Sort stage (Sec. 2.4): periodic wrap, 63-bit Morton+type keys, stable LSD
// radix sort, one gather of the particle data into sorted order, and the
// type-major order (bodies grouped by type, each type in key order).
#include <cmath>
#include <cstdarg>
#include <cstdio>

#include "ng_internal.cuh"

namespace ng {

constexpr int kScanThreads = 1024;
constexpr int kScanBlocks = 256;

__device__ __forceinline__ int64_t scan_len(int64_t bound, const uint32_t* d_len) {
  if (!d_len) return bound;
  const int64_t l = (int64_t)*d_len;
  return l < bound ? l : bound;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_partial(const uint32_t* __restrict__ in, int64_t bound, const uint32_t* d_len,
               uint32_t* part, int as_flags) {
  const int64_t len = scan_len(bound, d_len);
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < len ? b0 + chunk : len;
  uint32_t s = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += as_flags ? (in[i] != 0u) : in[i];
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ uint32_t ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < blockDim.x / 32 ? ws[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_final(const uint32_t* in, uint32_t* out, int64_t bound, const uint32_t* d_len,
             const uint32_t* __restrict__ part, uint32_t* d_total, int as_flags) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t tile_total;
  __shared__ uint32_t off;
  const int64_t len = scan_len(bound, d_len);
  const int64_t chunk = (len + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * chunk;
  const int64_t b1 = b0 + chunk < len ? b0 + chunk : len;
  if (threadIdx.x < 32) {
    uint32_t s = 0;
    for (int j = threadIdx.x; j < (int)blockIdx.x; j += 32) s += part[j];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) off = s;
  }
  __syncthreads();
  uint32_t carry = off;
  for (int64_t base = b0; base < b1; base += kScanThreads) {
    const int64_t i = base + threadIdx.x;
    uint32_t v = i < b1 ? in[i] : 0u;
    if (as_flags) v = v != 0u;
    const uint32_t inc = block_inclusive_scan<kScanThreads>(v, warp_tot, &tile_total);
    if (i < b1) out[i] = carry + inc - v;
    __syncthreads();
    carry += tile_total;
    __syncthreads();
  }
  if (d_total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *d_total = carry;
}

static int scan_blocks(int64_t len) {
  return (int)std::max<int64_t>(
      1, std::min<int64_t>(kScanBlocks, (len + 4 * kScanThreads - 1) / (4 * kScanThreads)));
}

int scan_u32(ng_ctx* c, const uint32_t* in, uint32_t* out, int64_t len, const uint32_t* d_len,
             uint32_t* d_total) {
  NG_TRY(ensure(c, c->scan_part, kScanBlocks * sizeof(uint32_t)));
  uint32_t* part = as<uint32_t>(c->scan_part);
  // blocks for at most 4 tiles each; both kernels split the range by gridDim
  const int blocks = scan_blocks(len);
  // one block needs no partial sums (its offset is zero)
  if (blocks > 1) k_scan_partial<<<blocks, kScanThreads, 0, c->stream>>>(in, len, d_len, part, 0);
  k_scan_final<<<blocks, kScanThreads, 0, c->stream>>>(in, out, len, d_len, part, d_total, 0);
  c->launches += blocks > 1 ? 2 : 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

// Exclusive scan of the flags (in[i] != 0): out[i] = number of non-zero
// entries before i; *d_total = number of non-zero entries.
int scan_u32_flags(ng_ctx* c, const uint32_t* in, uint32_t* out, int64_t len, uint32_t* d_total) {
  NG_TRY(ensure(c, c->scan_part, kScanBlocks * sizeof(uint32_t)));
  uint32_t* part = as<uint32_t>(c->scan_part);
  const int blocks = scan_blocks(len);
  if (blocks > 1) k_scan_partial<<<blocks, kScanThreads, 0, c->stream>>>(in, len, nullptr, part, 1);
  k_scan_final<<<blocks, kScanThreads, 0, c->stream>>>(in, out, len, nullptr, part, d_total, 1);
  c->launches += blocks > 1 ? 2 : 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

// --------------------------------------------------------------- keys

__global__ void k_keys(int64_t n, const double* __restrict__ pos, const uint8_t* __restrict__ type,
                       double L, double invL, bool pow2, int ebox, uint64_t* __restrict__ keys,
                       uint32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = sort_key(pos[i], pos[n + i], pos[2 * n + i], type[i], L, invL, pow2, ebox);
    idx[i] = (uint32_t)i;
  }
}

// ---------------------------------------------------------- radix sort

constexpr int kRsThreads = 256;
constexpr int kRsItems = 8;                        // keys per lane
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsTile = kRsThreads * kRsItems;     // 2048 keys per block
static_assert(kRsTile == kRadixTile, "radix tile and histogram layout disagree");

__global__ void __launch_bounds__(kRsThreads)
k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t mask,
          uint32_t* __restrict__ hist, int nblocks) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kRsTile;
  for (int j = threadIdx.x; j < kRsTile; j += kRsThreads) {
    const int64_t i = t0 + j;
    if (i < n) atomicAdd(&cnt[(uint32_t)(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one digit. Each warp ranks its contiguous sub-tile in
// order (match_any groups equal digits); warps are ordered per digit. The
// tile is then reordered by digit in shared memory and written out by
// consecutive threads, so each digit's run of the tile (16 keys on average)
// leaves as one contiguous segment instead of one sector per key.
__global__ void __launch_bounds__(kRsThreads)
k_rs_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
             uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
             uint32_t mask, const uint32_t* __restrict__ offs, int nblocks) {
  __shared__ uint32_t wcnt[kRsWarps][256];   // per warp and digit: count, then tile position
  __shared__ uint32_t dstart[256];           // tile position of each digit's run
  __shared__ uint32_t gdst[256];             // global position of each digit's run
  __shared__ uint64_t tk[kRsTile];
  __shared__ uint32_t tv[kRsTile];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < kRsWarps * 256; j += kRsThreads) (&wcnt[0][0])[j] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kRsTile;
  const int64_t sub0 = t0 + (int64_t)w * (kRsTile / kRsWarps);
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t k[kRsItems];
  uint32_t v[kRsItems], rank[kRsItems];
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int64_t i = sub0 + it * 32 + lane;
    const bool valid = i < n;
    k[it] = valid ? kin[i] : 0ull;
    v[it] = valid ? vin[i] : 0u;
    const uint32_t d = (uint32_t)(k[it] >> shift) & mask;
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? d : 0xffffffffu);
    uint32_t prior = 0;
    if (valid) prior = wcnt[w][d];
    __syncwarp();
    rank[it] = prior + __popc(peers & lt);
    if (valid && (peers & lt) == 0) wcnt[w][d] = prior + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    // thread d: the digit's total in the tile, its run's tile start (block
    // scan over digits) and the warps' positions inside the run
    const int d = threadIdx.x;
    uint32_t total = 0;
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ++ww) total += wcnt[ww][d];
    uint32_t incl = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    __shared__ uint32_t wsum[kRsWarps];
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int ww = 0; ww < w; ++ww) wbase += wsum[ww];
    uint32_t run = wbase + incl - total;
    dstart[d] = run;
    gdst[d] = offs[(int64_t)d * nblocks + blockIdx.x];
#pragma unroll
    for (int ww = 0; ww < kRsWarps; ++ww) {
      const uint32_t t = wcnt[ww][d];
      wcnt[ww][d] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int64_t i = sub0 + it * 32 + lane;
    if (i < n) {
      const uint32_t d = (uint32_t)(k[it] >> shift) & mask;
      const uint32_t pos = wcnt[w][d] + rank[it];
      tk[pos] = k[it];
      tv[pos] = v[it];
    }
  }
  __syncthreads();
  const int valid = (int)((n - t0) < kRsTile ? (n - t0) : kRsTile);
  for (int p = threadIdx.x; p < valid; p += kRsThreads) {
    const uint64_t key = tk[p];
    const uint32_t d = (uint32_t)(key >> shift) & mask;
    const uint32_t dst = gdst[d] + ((uint32_t)p - dstart[d]);
    kout[dst] = key;
    vout[dst] = tv[p];
  }
}

static int radix_pass(ng_ctx* c, const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                      uint32_t* vout, int64_t n, int shift, uint32_t mask) {
  const int nblocks = (int)((n + kRsTile - 1) / kRsTile);
  uint32_t* hist = as<uint32_t>(c->blockhist);
  k_rs_hist<<<nblocks, kRsThreads, 0, c->stream>>>(kin, n, shift, mask, hist, nblocks);
  NG_TRY(scan_u32(c, hist, hist, (int64_t)256 * nblocks, nullptr, nullptr));
  k_rs_scatter<<<nblocks, kRsThreads, 0, c->stream>>>(kin, vin, kout, vout, n, shift, mask, hist,
                                                     nblocks);
  c->launches += 2;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

// -------------------------------------------------------------- gather

__global__ void k_gather(int64_t n, const uint32_t* __restrict__ perm,
                         const double* __restrict__ pos, const uint8_t* __restrict__ type,
                         const float* __restrict__ mass, double L, double invL, bool pow2,
                         int D, double* __restrict__ spos, float* __restrict__ smass,
                         uint8_t* __restrict__ stype, uint32_t* status) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = perm[k];
    spos[k] = wrap_box(pos[i], L, invL, pow2);
    spos[n + k] = wrap_box(pos[n + i], L, invL, pow2);
    spos[2 * n + k] = wrap_box(pos[2 * n + i], L, invL, pow2);
    smass[k] = mass[i];
    const uint8_t ti = type[i];
    if (ti >= D) atomicOr(&status[ST_FLAGS], (uint32_t)SF_BAD_TYPE);
    stype[k] = ti < D ? ti : 0;    // out-of-range species: flagged, never used as an index
  }
}

// The resident step's gather: the previous state (positions already wrapped
// by the drift, masses, species, velocities and caller indices, in the
// previous step's sorted order) into this step's sorted order. The bodies
// move little from step to step, so perm is close to the identity and every
// read is close to sequential.
__global__ void k_gather_resident(int64_t n, const uint32_t* __restrict__ perm,
                                  const double* __restrict__ xpos, const float* __restrict__ xmass,
                                  const uint8_t* __restrict__ xtype, const float* __restrict__ xvel,
                                  const uint32_t* __restrict__ xorig, double* __restrict__ ypos,
                                  float* __restrict__ ymass, uint8_t* __restrict__ ytype,
                                  float* __restrict__ yvel, uint32_t* __restrict__ yorig) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t i = perm[k];
    ypos[k] = xpos[i];
    ypos[n + k] = xpos[n + i];
    ypos[2 * n + k] = xpos[2 * n + i];
    yvel[k] = xvel[i];
    yvel[n + k] = xvel[n + i];
    yvel[2 * n + k] = xvel[2 * n + i];
    ymass[k] = xmass[i];
    ytype[k] = xtype[i];
    yorig[k] = xorig[i];
  }
}

__global__ void k_iota(int64_t n, uint32_t* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (uint32_t)k;
}


int work_grid(ng_ctx* c, int64_t items, int per_sm) {
  const int64_t need = (items + 255) / 256;
  const int64_t most = (int64_t)c->nsm * per_sm;
  return (int)std::max<int64_t>(1, std::min(need, most));
}

int64_t level_bound(int l, int64_t n) {
  return l >= 21 ? n : std::min<int64_t>(n, (int64_t)1 << (3 * l));
}

bool box_is_pow2(double L) {
  int e = 0;
  return std::frexp(L, &e) == 0.5;
}

int reserve_sort(ng_ctx* c, int64_t n) {
  const int nblocks = (int)((n + kRsTile - 1) / kRsTile);
  NG_TRY(ensure(c, c->keys_a, n * 8));
  NG_TRY(ensure(c, c->keys_b, n * 8));
  NG_TRY(ensure(c, c->vals_a, n * 4));
  NG_TRY(ensure(c, c->vals_b, n * 4));
  NG_TRY(ensure(c, c->blockhist, (size_t)256 * nblocks * 4));
  NG_TRY(ensure(c, c->spos, n * 24));
  NG_TRY(ensure(c, c->smass, n * 4));
  NG_TRY(ensure(c, c->stype, n));
  NG_TRY(ensure(c, c->tperm, n * 4));
  NG_TRY(ensure(c, c->scan_part, kScanBlocks * sizeof(uint32_t)));
  return NG_OK;
}

// Keys of the bodies at pos and their stable sort: sorted keys in keys_a,
// the permutation (sorted index -> input index) in vals_a.
static int sort_keys(ng_ctx* c, int64_t n, const double* pos, const uint8_t* type) {
  uint64_t *ka = as<uint64_t>(c->keys_a), *kb = as<uint64_t>(c->keys_b);
  uint32_t *va = as<uint32_t>(c->vals_a), *vb = as<uint32_t>(c->vals_b);
  const int grid = work_grid(c, n, 8);
  const bool pow2 = box_is_pow2(c->L);
  stage_mark(c, NG_STAGE_KEYS);
  k_keys<<<grid, 256, 0, c->stream>>>(n, pos, type, c->L, 1.0 / c->L, pow2,
                                      pow2 ? std::ilogb(c->L) : 0, ka, va);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  // 8 passes of 8 bits: the result returns to (ka, va). A tree capped at
  // level_cap reads the Morton bits of its levels only (bits >= 3 + 3 (20 -
  // cap)), so the passes below them are skipped, keeping an even number of
  // passes: bodies that share those bits keep their previous relative order,
  // and every cell down to the cap is still one contiguous range.
  int first = 0;
  if (c->level_cap < kMaxLevel) {
    first = (3 + 3 * (kMaxLevel - std::max(c->level_cap, 0))) / 8;
    if ((8 - first) & 1) --first;
  }
  c->sort_passes = 8 - first;
  stage_mark(c, NG_STAGE_RADIX);
  for (int pass = first; pass < 8; ++pass) {
    const bool even = ((pass - first) & 1) == 0;
    NG_TRY(radix_pass(c, even ? ka : kb, even ? va : vb, even ? kb : ka, even ? vb : va, n,
                      8 * pass, 0xffu));
  }
  return NG_OK;
}

int sort_resident(ng_ctx* c, int64_t n) {
  NG_TRY(sort_keys(c, n, as<double>(c->spos_alt), as<uint8_t>(c->stype_alt)));
  stage_mark(c, NG_STAGE_GATHER);
  k_gather_resident<<<work_grid(c, n, 8), 256, 0, c->stream>>>(
      n, as<uint32_t>(c->vals_a), as<double>(c->spos_alt), as<float>(c->smass_alt),
      as<uint8_t>(c->stype_alt), as<float>(c->rvel_alt), as<uint32_t>(c->rorig_alt),
      as<double>(c->spos), as<float>(c->smass), as<uint8_t>(c->stype), as<float>(c->rvel),
      as<uint32_t>(c->rorig));
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

int sort_bodies(ng_ctx* c, int64_t n, const double* pos, const uint8_t* type, const float* mass) {
  NG_TRY(reserve_sort(c, n));
  uint32_t* va = as<uint32_t>(c->vals_a);
  const int grid = work_grid(c, n, 8);
  const bool pow2 = box_is_pow2(c->L);
  NG_TRY(sort_keys(c, n, pos, type));
  c->launches += 1;   // gather
  stage_mark(c, NG_STAGE_GATHER);
  k_gather<<<grid, 256, 0, c->stream>>>(n, va, pos, type, mass, c->L, 1.0 / c->L, pow2, c->p.D,
                                        as<double>(c->spos), as<float>(c->smass),
                                        as<uint8_t>(c->stype), as<uint32_t>(c->status));
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

// Type-major order: one stable radix pass on the species bits of the sorted
// keys. tperm[j] = sorted index of the j-th body in type-major order.
int type_order(ng_ctx* c) {
  const int64_t n = c->n;
  const int grid = work_grid(c, n, 8);
  uint64_t *ka = as<uint64_t>(c->keys_a), *kb = as<uint64_t>(c->keys_b);
  uint32_t* vb = as<uint32_t>(c->vals_b);
  stage_mark(c, NG_STAGE_TYPE_ORDER);
  k_iota<<<grid, 256, 0, c->stream>>>(n, vb);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  NG_TRY(radix_pass(c, ka, vb, kb, as<uint32_t>(c->tperm), n, 0, 7u));
  return NG_OK;
}

}  // namespace ng
