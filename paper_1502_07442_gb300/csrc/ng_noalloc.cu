// Key sort that allocates nothing, for callers that must not call cudaMalloc.
//
// Some hosts of this library cannot allocate device memory on their own
// schedule: code that runs while a memory pool is locked by another
// framework, real-time loops whose allocator calls would stall or
// synchronise the device, or embedding programs that hand the library only
// the buffers they own. ng_build_tree grows its scratch with cudaMalloc;
// ng_sort_keys_noalloc computes the same sorted keys and permutation with
// its scratch in one fixed device array that exists from the moment the
// library is loaded.
//
// The scratch lives in a file-scope __device__ array (kNoAllocMaxBodies
// bodies, about 3.4 MB on every GPU that loads the library, held until the
// process exits). Host code cannot pass the array's name to a kernel (on the
// host it is only a stand-in symbol), so every call looks up the array's
// device address with cudaGetSymbolAddress on the current device. The first
// call on a device may load the library's device code there; make that
// first call before any stream capture. The address is not cached, so a
// device reset (which can move the array) leaves no stale pointer behind.
// Every call shares the one array: calls whose work overlaps on the GPU (two
// streams, or two host threads) race on it. No part of the scratch has to
// start at zero: every pass writes each word before it is read.
#include <cmath>

#include "ng_internal.cuh"

namespace {

constexpr int64_t kNoAllocMaxBodies = int64_t(1) << 18;   // 262144 bodies
constexpr int kNaThreads = 256;
constexpr int kNaItems = 4;
constexpr int kNaTile = kNaThreads * kNaItems;            // keys per block and pass
constexpr int kNaMaxBlocks = (int)(kNoAllocMaxBodies / kNaTile);
constexpr int kNaWarps = kNaThreads / 32;

struct NaScratch {
  uint64_t keys[kNoAllocMaxBodies];                      // ping-pong partner of keys_out
  uint32_t vals[kNoAllocMaxBodies];                      // ping-pong partner of perm_out
  uint32_t hist[256 * kNaMaxBlocks];                     // digit-major block histograms
};

static __device__ __align__(256) NaScratch g_na_scratch;

// The keys of ng_build_tree (the same device function forms both).
__global__ void k_na_keys(int64_t n, const double* __restrict__ pos,
                          const uint8_t* __restrict__ type, double L, double invL, bool pow2,
                          int ebox, uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = ng::sort_key(pos[i], pos[n + i], pos[2 * n + i], type[i], L, invL, pow2, ebox);
    idx[i] = (uint32_t)i;
  }
}

__global__ void __launch_bounds__(kNaThreads)
k_na_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, uint32_t* __restrict__ hist,
          int nblocks) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kNaTile;
  for (int j = threadIdx.x; j < kNaTile; j += kNaThreads)
    if (t0 + j < n) atomicAdd(&cnt[(uint32_t)(keys[t0 + j] >> shift) & 255u], 1u);
  __syncthreads();
  hist[threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// One block scans the 256 * nblocks digit-major counts in place.
__global__ void __launch_bounds__(1024) k_na_scan(uint32_t* hist, int len) {
  __shared__ uint32_t part[1024];
  const int per = (len + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  uint32_t s = 0;
  for (int i = b0; i < b0 + per && i < len; ++i) s += hist[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int t = 0; t < 1024; ++t) {
      const uint32_t v = part[t];
      part[t] = run;
      run += v;
    }
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (int i = b0; i < b0 + per && i < len; ++i) {
    const uint32_t v = hist[i];
    hist[i] = run;
    run += v;
  }
}

// Stable scatter of one 8-bit digit (warps rank their contiguous slices in
// order, then take their places after the earlier warps of the block).
__global__ void __launch_bounds__(kNaThreads)
k_na_scatter(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
             uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n, int shift,
             const uint32_t* __restrict__ offs, int nblocks) {
  __shared__ uint32_t wcnt[kNaWarps][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < kNaWarps * 256; j += kNaThreads) (&wcnt[0][0])[j] = 0;
  __syncthreads();
  const int64_t sub0 = (int64_t)blockIdx.x * kNaTile + (int64_t)w * (kNaTile / kNaWarps);
  const uint32_t lt = (1u << lane) - 1u;
  uint64_t k[kNaItems];
  uint32_t v[kNaItems], rank[kNaItems];
#pragma unroll
  for (int it = 0; it < kNaItems; ++it) {
    const int64_t i = sub0 + it * 32 + lane;
    const bool valid = i < n;
    k[it] = valid ? kin[i] : 0ull;
    v[it] = valid ? vin[i] : 0u;
    const uint32_t d = (uint32_t)(k[it] >> shift) & 255u;
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
    uint32_t run = offs[threadIdx.x * nblocks + blockIdx.x];
    for (int ww = 0; ww < kNaWarps; ++ww) {
      const uint32_t t = wcnt[ww][threadIdx.x];
      wcnt[ww][threadIdx.x] = run;
      run += t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kNaItems; ++it) {
    const int64_t i = sub0 + it * 32 + lane;
    if (i < n) {
      const uint32_t dst = wcnt[w][(uint32_t)(k[it] >> shift) & 255u] + rank[it];
      kout[dst] = k[it];
      vout[dst] = v[it];
    }
  }
}

// Device address of the scratch array on the current device.
int na_scratch(NaScratch** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_na_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return NG_ECUDA;
  }
  *out = static_cast<NaScratch*>(p);
  return NG_OK;
}

// The launch just made failed to start: report it as this call's error.
int na_launched() {
  if (cudaGetLastError() != cudaSuccess) return NG_ECUDA;
  return NG_OK;
}

}  // namespace

extern "C" int ng_sort_keys_noalloc(int64_t n, const double* pos, const uint8_t* type, double box,
                                    uint64_t* keys_out, uint32_t* perm_out, void* stream) {
  if (n < 1 || n > kNoAllocMaxBodies) return NG_EINVAL;   // at most 2^18 bodies
  if (!pos || !type || !keys_out || !perm_out || !(box > 0)) return NG_EINVAL;
  NaScratch* sc = nullptr;
  const int r = na_scratch(&sc);
  if (r != NG_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const bool pow2 = ng::box_is_pow2(box);
  const int ebox = pow2 ? std::ilogb(box) : 0;     // box = 2^ebox
  k_na_keys<<<(int)((n + 255) / 256), 256, 0, st>>>(n, pos, type, box, 1.0 / box, pow2, ebox,
                                                   keys_out, perm_out);
  if (na_launched() != NG_OK) return NG_ECUDA;
  const int nblocks = (int)((n + kNaTile - 1) / kNaTile);
  // 8 passes of 8 bits; the sorted result returns to (keys_out, perm_out)
  for (int pass = 0; pass < 8; ++pass) {
    const bool even = (pass & 1) == 0;
    const uint64_t* kin = even ? keys_out : sc->keys;
    const uint32_t* vin = even ? perm_out : sc->vals;
    uint64_t* kout = even ? sc->keys : keys_out;
    uint32_t* vout = even ? sc->vals : perm_out;
    k_na_hist<<<nblocks, kNaThreads, 0, st>>>(kin, n, 8 * pass, sc->hist, nblocks);
    k_na_scan<<<1, 1024, 0, st>>>(sc->hist, 256 * nblocks);
    k_na_scatter<<<nblocks, kNaThreads, 0, st>>>(kin, vin, kout, vout, n, 8 * pass, sc->hist,
                                                 nblocks);
    if (na_launched() != NG_OK) return NG_ECUDA;
  }
  return NG_OK;
}
