// Short-range tree walk (Sec. 2.2) with the TreePM short-range laws of
// Sec. 2.4.1, evaluated in FP32 on group-relative offsets.
//
// One warp walks the tree for one group of up to 32 spatially compact bodies
// (one body per lane). Nodes are popped 32 at a time from a warp stack in
// shared memory and classified against the group's bounding box:
//   skip    the node cube lies >= r_cut from the box;
//   accept  l < theta * d, d = distance from the box to the node's
//           all-species centre of mass (and the box is outside the cube):
//           its D species monopoles go to D per-species record lists;
//   leaf    a rejected leaf: its bodies go to the list of their species;
//   open    a rejected internal node: its children are pushed.
// A record (monopole or body) that lies r_cut or more from the box is not
// appended: it would contribute exactly zero to every body of the group.
// A list that may overflow is evaluated: every lane interacts its body with
// every record. Records and bodies are float4 {x, y, z, m} in
// table units relative to a dyadic group origin, so node-centre offsets are
// exact in FP32 and no FP64 enters the inner loop.
//
// Inner loop per (body, record): q = |d|^2 + eps^2, inv = rsqrt(q); the
// table index k = rint(rho), rho = q * inv, is read from the float bits of
// q*inv + 2^23; the table holds linear segments per law (laid out per list
// species with one entry per passive species; in variable-species launches
// one row per distinct law), stored as {c0 - k c1, c1} so that its value is
// (c0 - k c1) + rho c1 (zero past the cut-off); the force is m * value * inv^3 * d, summed over one species list;
// each list's sum is scaled by the coupling G[s][t] of the body's species s
// and the list's species t and added to one accumulator per body.
#include <type_traits>

#include "ng_internal.cuh"

namespace ng {

template <int D, int CAP>
struct __align__(16) WarpSmem {
  WalkDesc desc;              // batched launches: the current item's simulation
  // records per active species, table units, one float array per component
  // (x[CAP], y[CAP], z[CAP], m[CAP]): consecutive records
  // of one component are one 8- or 16-byte load, so the inner loop forms
  // (record j, record j + 1) pairs for the packed FP32x2 instructions
  float4 list[D][CAP];
  float4 leafc[32];           // opened leaves: centre offset from the origin (box units)
  int2 leafb[32];             // opened leaves: first body, body count
  int leafo[32];              // opened leaves: exclusive prefix of body counts
  int stack[kStackCap];
};

constexpr float kMagic = 8388608.0f;   // 2^23
constexpr int kMagicBits = 0x4B000000;

__device__ __forceinline__ float wrap_unit(float d) { return d - rintf(d); }

// A record at p (box units, relative to the group origin) can reach some body
// of the group only if it lies within r_cut of the group box (half extents g
// around the origin); records beyond contribute exactly zero for every body.
__device__ __forceinline__ bool near_box(float px, float py, float pz, float gx, float gy,
                                         float gz, float r2) {
  const float ex = fmaxf(0.f, fabsf(px) - gx), ey = fmaxf(0.f, fabsf(py) - gy),
              ez = fmaxf(0.f, fabsf(pz) - gz);
  return fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < r2;
}

// Append one record at `slot` of a component-major list.
template <int CAP>
__device__ __forceinline__ void put_rec(float4* list, int slot, float x, float y, float z,
                                        float m) {
  float* c = reinterpret_cast<float*>(list);
  c[slot] = x;
  c[CAP + slot] = y;
  c[2 * CAP + slot] = z;
  c[3 * CAP + slot] = m;
}

// 8-byte shared-memory load from a 32-bit shared address
__device__ __forceinline__ float2 lds_f2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
  return v;
}

// Each warp copies its item's descriptor (one per simulation) from device
// memory into shared memory and reads the fields from there.
#define DESC(f) (ws->desc.f)

// ACC64: the FP64-accumulated variant (each evaluated list's FP32 sum is
// added into an FP64 per-body accumulator); otherwise FP32 throughout.
// REL: some simulation of the launch may use the relative criterion (an
// instance without it carries none of that code).
// VARD: the simulations of the launch may have different species counts; D
// is then the largest (lists for D species, the law table laid out for D),
// and each work item uses its simulation's own count DESC(D) <= D.
template <int D, bool ACC64, bool REL, bool VARD>
__global__ void __launch_bounds__((VARD ? kVardWarps : walk_warps(D)) * 32, 1) k_walk(WalkLaunch L) {
  using Acc = typename std::conditional<ACC64, double, float>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tab = reinterpret_cast<float2*>(smem_raw);
  const int ntab = L.tab_count;
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) tab[i] = L.tab[i];
  const size_t tab_bytes = ((size_t)ntab * sizeof(float2) + 15) & ~(size_t)15;
  constexpr int CAP = walk_list_cap(D, VARD);
  WarpSmem<D, CAP>* ws = reinterpret_cast<WarpSmem<D, CAP>*>(smem_raw + tab_bytes) + (threadIdx.x >> 5);
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t total_groups = L.gprefix[L.ndesc];
  const int clampbits = kMagicBits + L.ncut;
  unsigned long long nint = 0;

  while (true) {
    // one work item = one group of one simulation (all simulations of the
    // launch share the law table and the species count)
    uint32_t g = 0;
    if (lane == 0) g = atomicAdd(L.work, 1u);
    g = __shfl_sync(0xffffffffu, g, 0);
    if (g >= total_groups) break;
    int lo_s = 0, hi_s = L.ndesc - 1;
    while (lo_s < hi_s) {
      const int mid = (lo_s + hi_s + 1) >> 1;
      if (L.gprefix[mid] <= g) lo_s = mid; else hi_s = mid - 1;
    }
    __syncwarp();
    {
      const int4* src = reinterpret_cast<const int4*>(L.descs + lo_s);
      int4* dst = reinterpret_cast<int4*>(&ws->desc);
      for (int i = lane; i < (int)(sizeof(WalkDesc) / 16); i += 32) dst[i] = src[i];
    }
    __syncwarp();
    const uint32_t nnodes = DESC(status)[ST_LEVELS + kMaxLevel + 1];
    const int DR = VARD ? DESC(D) : D;   // species of this item's simulation
    const float rc2 = DESC(rcut_box) * DESC(rcut_box);
    const float rc2_keep = rc2 * 1.0001f;   // margin for FP32 rounding of the offsets
    const float s_tab = DESC(s_tab);
    const float eps2 = DESC(eps2_tab);
    const int2 gr = DESC(groups)[g - L.gprefix[lo_s]];
    const int nact = gr.y;
    const bool active = lane < nact;
    const int64_t p = gr.x + (active ? lane : 0);
    const int s = DESC(btype)[p];
    float ox, oy, oz, gx, gy, gz;
    const float4 lg = DESC(geo)[DESC(bleaf)[p]];
    const float4 bd = DESC(body)[p];
    {
      // bounding box (box units, FP32; no FP64 in the walk) relative to the
      // leaf centre of the group's first body; group bodies lie in one cell
      // far smaller than the box, so no wrap is needed inside the group
      const float rx = __shfl_sync(0xffffffffu, lg.x, 0), ry = __shfl_sync(0xffffffffu, lg.y, 0),
                  rz = __shfl_sync(0xffffffffu, lg.z, 0);
      float lo[3] = {(lg.x - rx) + bd.x, (lg.y - ry) + bd.y, (lg.z - rz) + bd.z};
      float hi[3] = {lo[0], lo[1], lo[2]};
#pragma unroll
      for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
          hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
      }
      // dyadic origin (a multiple of 2^-21, exact in FP32) at the box centre
      const float s21 = 2097152.0f, i21 = 1.0f / 2097152.0f;
      ox = rintf((rx + 0.5f * (lo[0] + hi[0])) * s21) * i21;
      oy = rintf((ry + 0.5f * (lo[1] + hi[1])) * s21) * i21;
      oz = rintf((rz + 0.5f * (lo[2] + hi[2])) * s21) * i21;
      const float pad = 1.0f / 1048576.0f;
      gx = 0.5f * (hi[0] - lo[0]) + pad;
      gy = 0.5f * (hi[1] - lo[1]) + pad;
      gz = 0.5f * (hi[2] - lo[2]) + pad;
    }
    // relative criterion: the group accepts a node only when every body of it
    // would, so it uses the smallest |a_old| of the group
    const bool rel = REL && DESC(aold) != nullptr;
    float thr = 0.f;
    if (rel) {
      float a = active ? DESC(aold)[DESC(perm)[p]] : 3.0e38f;
#pragma unroll
      for (int o = 16; o; o >>= 1) a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
      thr = DESC(rel_scale) * a;
    }
    // the body's own position is formed exactly as its record in the lists
    // (leaf centre offset + body offset, then scaled), so the self term has
    // d = 0 exactly and contributes nothing
    const float xr = (wrap_unit(lg.x - ox) + bd.x) * s_tab;
    const float yr = (wrap_unit(lg.y - oy) + bd.y) * s_tab;
    const float zr = (wrap_unit(lg.z - oz) + bd.z) * s_tab;

    Acc ax = 0, ay = 0, az = 0;   // per-body accumulator
    int lc[D];                      // records per species list (same in every lane)
#pragma unroll
    for (int t = 0; t < D; ++t) lc[t] = 0;

    if (lane == 0) ws->stack[0] = 0;
    int size = 1;
    int qtotal = 0, qdone = 0, nl = 0;   // queued bodies of opened leaves
    bool overflow = false;
    uint32_t visits = 0;            // a tree has nnodes nodes: more visits means corruption
    __syncwarp();
    while (true) {
      // ---- the single evaluation site: lists that could overflow on the
      // next round of (<= 32 per species) appends, or everything at the end
      const bool drain = size == 0 && qdone >= qtotal;
      uint32_t fmask = 0;   // lists to evaluate now (the same in every lane)
#pragma unroll
      for (int q = 0; q < D; ++q)
        if (lc[q] > CAP - 32 || (drain && lc[q] > 0)) fmask |= 1u << q;
#pragma unroll 1
      while (fmask) {
        const int t = __ffs(fmask) - 1;
        fmask &= fmask - 1;
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < D; ++q) cnt = (q == t) ? lc[q] : cnt;
        {
          // shared address of segment k of this lane's law (passive s,
          // active t) is tb + 8 pad * (float bits of k + 2^23), mod 2^32, so
          // the index needs no subtraction (pad = 1 for the one-row-per-law
          // table of variable-species launches)
          constexpr int kRowShift = 3 + (VARD ? 0 : walk_tab_shift(D));
          const float2* row = VARD ? tab + DESC(tabid)[s][t] * L.tab_entries
                                   : tab + (t * L.tab_entries << walk_tab_shift(D)) + s;
          const uint32_t tb =
              (uint32_t)__cvta_generic_to_shared(row) - ((uint32_t)kMagicBits << kRowShift);
          float* lt4 = reinterpret_cast<float*>(ws->list[t]);
          // pad to an even count with a massless record (zero force); full
          // quads of records, then at most one pair
          const int cnt2 = (cnt + 1) & ~1;
          const int nq = cnt2 & ~3;
          if (lane < cnt2 - cnt) put_rec<CAP>(ws->list[t], cnt + lane, 0.f, 0.f, 0.f, 0.f);
          __syncwarp();
          // (record j, record j + 1) in the two halves of packed FP32x2
          // operations; each half rounds exactly as the scalar operation
          const float2 nx = make_float2(-xr, -xr), ny = make_float2(-yr, -yr),
                       nz = make_float2(-zr, -zr), e2 = make_float2(eps2, eps2),
                       mg = make_float2(kMagic, kMagic);
          float2 sx2 = make_float2(0.f, 0.f), sy2 = sx2, sz2 = sx2;
          auto pair = [&](float2 rx, float2 ry, float2 rz, float2 rm) {
            const float2 dx = __fadd2_rn(rx, nx), dy = __fadd2_rn(ry, ny), dz = __fadd2_rn(rz, nz);
            const float2 qq = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, e2)));
            const float2 inv = make_float2(rsqrtf(qq.x), rsqrtf(qq.y));
            const float2 fi = __ffma2_rn(qq, inv, mg);
            const int b0 = min(__float_as_int(fi.x), clampbits);
            const int b1 = min(__float_as_int(fi.y), clampbits);
            const float2 rho = __fmul2_rn(qq, inv);
            const float2 t0 = lds_f2(tb + ((uint32_t)b0 << kRowShift));
            const float2 t1 = lds_f2(tb + ((uint32_t)b1 << kRowShift));
            const float2 gg = make_float2(fmaf(rho.x, t0.y, t0.x), fmaf(rho.y, t1.y, t1.x));
            const float2 inv2 = __fmul2_rn(inv, inv);
            const float2 f = __fmul2_rn(__fmul2_rn(rm, gg), __fmul2_rn(inv2, inv));
            sx2 = __ffma2_rn(f, dx, sx2);
            sy2 = __ffma2_rn(f, dy, sy2);
            sz2 = __ffma2_rn(f, dz, sz2);
          };
          // four records of each component per 16-byte load; four loop
          // bodies per iteration give the scheduler loads to hoist
#pragma unroll 4
          for (int j = 0; j < nq; j += 4) {
            const float4 X = *reinterpret_cast<const float4*>(lt4 + j);
            const float4 Y = *reinterpret_cast<const float4*>(lt4 + CAP + j);
            const float4 Z = *reinterpret_cast<const float4*>(lt4 + 2 * CAP + j);
            const float4 M = *reinterpret_cast<const float4*>(lt4 + 3 * CAP + j);
            pair(make_float2(X.x, X.y), make_float2(Y.x, Y.y), make_float2(Z.x, Z.y),
                 make_float2(M.x, M.y));
            pair(make_float2(X.z, X.w), make_float2(Y.z, Y.w), make_float2(Z.z, Z.w),
                 make_float2(M.z, M.w));
          }
          if (cnt2 != nq) {
            const float2 X = *reinterpret_cast<const float2*>(lt4 + nq);
            const float2 Y = *reinterpret_cast<const float2*>(lt4 + CAP + nq);
            const float2 Z = *reinterpret_cast<const float2*>(lt4 + 2 * CAP + nq);
            const float2 M = *reinterpret_cast<const float2*>(lt4 + 3 * CAP + nq);
            pair(X, Y, Z, M);
          }
          const float sx = sx2.x + sx2.y, sy = sy2.x + sy2.y, sz = sz2.x + sz2.y;
          __syncwarp();
          const float G = DESC(G[s][t]);
          if constexpr (ACC64) {
            ax = fma((double)G, (double)sx, ax);
            ay = fma((double)G, (double)sy, ay);
            az = fma((double)G, (double)sz, az);
          } else {
            ax = fmaf(G, sx, ax);
            ay = fmaf(G, sy, ay);
            az = fmaf(G, sz, az);
          }
#pragma unroll
          for (int q = 0; q < D; ++q) lc[q] = (q == t) ? 0 : lc[q];
          nint += (unsigned long long)cnt * (unsigned long long)nact;
        }
      }
      if (drain) break;

      if (qdone < qtotal) {
        // ---- one chunk of up to 32 queued leaf bodies into the lists of their species
        const int f = qdone + lane;
        const bool has = f < qtotal;
        // leaf holding queued body f: the number of leaf starts <= f, minus
        // one. Lane j holds the start of leaf j; the starts inside this chunk
        // become one bit mask, those before it one count (no search)
        const int sj = lane < nl ? ws->leafo[lane] : 0x7fffffff;
        const uint32_t starts = __reduce_or_sync(
            0xffffffffu, sj >= qdone && sj < qdone + 32 ? 1u << (sj - qdone) : 0u);
        const int before = __popc(__ballot_sync(0xffffffffu, sj < qdone));
        const uint32_t upto = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;
        const int lo = before + __popc(starts & upto) - 1;
        const int lstart = __shfl_sync(0xffffffffu, sj, lo & 31);
        float4 rec = make_float4(0.f, 0.f, 0.f, 0.f);
        int bt = -1;
        if (has) {
          const int b = ws->leafb[lo].x + (f - lstart);
          const float4 lc4 = ws->leafc[lo];
          const float4 bb = DESC(body)[b];
          const float px = lc4.x + bb.x, py = lc4.y + bb.y, pz = lc4.z + bb.z;
          bt = near_box(px, py, pz, gx, gy, gz, rc2_keep) ? (int)DESC(btype)[b] : -1;
          rec = make_float4(px * s_tab, py * s_tab, pz * s_tab, bb.w);
        }
        // each body goes to the list of its species: its slot is taken while
        // the list counts advance, then one append per lane
        int slot = 0;
#pragma unroll
        for (int t = 0; t < D; ++t) {
          if (VARD && t >= DR) break;
          const uint32_t m = __ballot_sync(0xffffffffu, bt == t);
          if (bt == t) slot = lc[t] + __popc(m & lt);
          lc[t] += __popc(m);
        }
        // (bt = -1: beyond r_cut of the box; the gather stores only species < D)
        if ((unsigned)bt < (unsigned)D) put_rec<CAP>(ws->list[bt], slot, rec.x, rec.y, rec.z, rec.w);
        qdone += 32;
        __syncwarp();
        continue;
      }

      // ---- pop the top min(32, size) nodes. Their children may use `avail`
      // slots of the breadth area (kStackCap - kStackReserve); an opened
      // node whose children do not fit is pushed back and popped again
      // later (lane 0 always fits: avail >= 8). When fewer than 8 slots are
      // left, pop one node (depth-first) whose children go into the reserve.
      // A breadth round leaves at most (kStackCap - kStackReserve) + 31
      // entries, and depth-first descent adds at most 7 per level below
      // that, so the stack stays below kStackCap - 7.
      if (size + 7 > kStackCap || visits > nnodes) { overflow = true; break; }
      int k = min(32, size);
      int avail = (kStackCap - kStackReserve) - (size - k);
      if (avail < 8) {
        k = 1;
        avail = kStackCap - (size - 1);
      }
      visits += k;
      const int node = lane < k ? ws->stack[size - k + lane] : -1;
      size -= k;
      __syncwarp();
      // classify: the three node records are fetched together
      int cls = 0;   // 0 skip, 1 accept, 2 leaf, 3 open
      float dcx = 0.f, dcy = 0.f, dcz = 0.f;
      int4 lk = make_int4(0, 0, 0, 0);
      if (node >= 0) {
        const float4 ge = DESC(geo)[node];
        const float4 cm = DESC(com)[node];
        lk = DESC(link)[node];
        // the species monopoles are read only if the node is accepted;
        // start moving them into L1 now
        const char* mp = reinterpret_cast<const char*>(DESC(mono) + (size_t)node * DR);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(mp));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(mp + DR * 16 - 1));
        dcx = wrap_unit(ge.x - ox);
        dcy = wrap_unit(ge.y - oy);
        dcz = wrap_unit(ge.z - oz);
        const float hx = fmaxf(0.f, fabsf(dcx) - ge.w - gx);
        const float hy = fmaxf(0.f, fabsf(dcy) - ge.w - gy);
        const float hz = fmaxf(0.f, fabsf(dcz) - ge.w - gz);
        const float d2min = hx * hx + hy * hy + hz * hz;
        if (d2min < rc2) {
          const float ex = fmaxf(0.f, fabsf(dcx + cm.x) - gx);
          const float ey = fmaxf(0.f, fabsf(dcy + cm.y) - gy);
          const float ez = fmaxf(0.f, fabsf(dcz + cm.z) - gz);
          const float dd2 = ex * ex + ey * ey + ez * ez;
          const float side = 2.f * ge.w;
          bool take;
          if (rel) {
            // the box lies outside the cube of side 1.2 l about the node centre,
            // and G_max M l^2 <= alpha |a_old| d^4 at the box's closest point
            const float lim = 0.6f * side;
            const bool outside = fabsf(dcx) - gx >= lim || fabsf(dcy) - gy >= lim ||
                                 fabsf(dcz) - gz >= lim;
            take = outside && cm.w * (side * side) <= thr * (dd2 * dd2);
          } else {
            take = d2min > 0.f && side * side < DESC(theta2) * dd2;
          }
          if (take) cls = 1;
          else cls = lk.y == 0 ? 2 : 3;
        }
      }
      // accepted nodes: one record per species with mass
      if (__any_sync(0xffffffffu, cls == 1)) {
#pragma unroll
        for (int t = 0; t < D; ++t) {
          if (VARD && t >= DR) break;
          float4 mo = make_float4(0.f, 0.f, 0.f, 0.f);
          if (cls == 1) mo = DESC(mono)[(size_t)node * DR + t];
          const float px = dcx + mo.x, py = dcy + mo.y, pz = dcz + mo.z;
          const bool has = mo.w > 0.f && near_box(px, py, pz, gx, gy, gz, rc2_keep);
          const uint32_t b = __ballot_sync(0xffffffffu, has);
          if (has) put_rec<CAP>(ws->list[t], lc[t] + __popc(b & lt), px * s_tab, py * s_tab, pz * s_tab, mo.w);
          lc[t] += __popc(b);
        }
      }
      // rejected internal nodes: push children, in lane order while they
      // fit in `avail`; the remaining opened nodes are pushed back
      {
        const int nch = cls == 3 ? lk.y : 0;
        int incl = nch;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const bool fit = incl <= avail;
        const uint32_t back = __ballot_sync(0xffffffffu, cls == 3 && !fit);
        const int used = (int)__reduce_max_sync(0xffffffffu, fit ? (unsigned)incl : 0u);
        if (fit) {
          const int base = size + incl - nch;
          for (int cc = 0; cc < nch; ++cc) ws->stack[base + cc] = lk.x + cc;
        } else if (cls == 3) {
          ws->stack[size + used + __popc(back & lt)] = node;
        }
        size += used + __popc(back);
        visits -= __popc(back);
      }
      // rejected leaves: queue their bodies (drained 32 per iteration above)
      {
        const uint32_t lm = __ballot_sync(0xffffffffu, cls == 2);
        if (lm) {
          const int nb = cls == 2 ? lk.w : 0;
          int incl = nb;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
          }
          qtotal = __shfl_sync(0xffffffffu, incl, 31);
          qdone = 0;
          nl = __popc(lm);
          if (cls == 2) {
            // the queued bodies are read in the next chunks; start moving
            // their records into L1 now
            const char* bp = reinterpret_cast<const char*>(DESC(body) + lk.z);
            for (int o = 0; o < lk.w * 16; o += 128) asm volatile("prefetch.global.L1 [%0];" ::"l"(bp + o));
            const int pos = __popc(lm & lt);
            ws->leafc[pos] = make_float4(dcx, dcy, dcz, 0.f);
            ws->leafb[pos] = make_int2(lk.z, lk.w);
            ws->leafo[pos] = incl - nb;
          }
        }
      }
      __syncwarp();
    }
    __syncwarp();
    if (overflow) {
      if (lane == 0) atomicOr(&DESC(status)[ST_FLAGS], (uint32_t)SF_STACK_OVERFLOW);
      continue;
    }
    if (active) {
      const Acc sc = (Acc)DESC(out_scale);
      const float fx = (float)(ax * sc), fy = (float)(ay * sc), fz = (float)(az * sc);
      const uint32_t i = DESC(out) ? DESC(out)[p] : (uint32_t)p;
      float* acc = DESC(acc);
      const int64_t nb = DESC(n);
      if (DESC(accumulate)) {
        acc[i] += fx;
        acc[nb + i] += fy;
        acc[2 * nb + i] += fz;
      } else {
        acc[i] = fx;
        acc[nb + i] = fy;
        acc[2 * nb + i] = fz;
      }
    }
  }
  if (L.counter && lane == 0 && nint) atomicAdd(L.counter, nint);
}

#undef DESC

// Group-count prefix over the descriptors of one launch; zero work counter.
// Simulations whose tree overflowed contribute no groups.
__global__ void __launch_bounds__(1024) k_walk_prep(const WalkDesc* __restrict__ descs, int ndesc,
                                                    uint32_t* gprefix, uint32_t* work) {
  __shared__ uint32_t part[1024];
  const int per = (ndesc + 1023) / 1024;
  const int b0 = threadIdx.x * per;
  uint32_t sum = 0;
  for (int i = b0; i < b0 + per && i < ndesc; ++i) {
    const uint32_t* st = descs[i].status;
    uint32_t ng = st[ST_NGROUPS];
    if (ng > (uint64_t)descs[i].n) ng = (uint32_t)descs[i].n;
    if (st[ST_FLAGS] & SF_NODE_OVERFLOW) ng = 0;
    sum += ng;
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int t = 0; t < 1024; ++t) {
      const uint32_t v = part[t];
      part[t] = run;
      run += v;
    }
    gprefix[ndesc] = run;
    *work = 0;
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (int i = b0; i < b0 + per && i < ndesc; ++i) {
    gprefix[i] = run;
    const uint32_t* st = descs[i].status;
    uint32_t ng = st[ST_NGROUPS];
    if (ng > (uint64_t)descs[i].n) ng = (uint32_t)descs[i].n;
    if (st[ST_FLAGS] & SF_NODE_OVERFLOW) ng = 0;
    run += ng;
  }
}

template <int D, bool VARD>
static size_t walk_smem(int tab_count, int nwarps) {
  const size_t tab_bytes = ((size_t)tab_count * sizeof(float2) + 15) & ~(size_t)15;
  return tab_bytes + (size_t)nwarps * sizeof(WarpSmem<D, walk_list_cap(D, VARD)>);
}

template <int D, bool ACC64, bool REL, bool VARD>
static int launch_walk_d(ng_ctx* c, cudaStream_t stream, const WalkLaunch& L, int64_t groups) {
  int nwarps = VARD ? kVardWarps : walk_warps(D);
  while (nwarps > 1 && walk_smem<D, VARD>(L.tab_count, nwarps) > c->smem_optin) --nwarps;
  const size_t smem = walk_smem<D, VARD>(L.tab_count, nwarps);
  if (smem > c->smem_optin)
    return fail(c, NG_ENOMEM, "walk needs %zu B shared memory (max %zu)", smem, c->smem_optin);
  // the attribute is a per-function ceiling shared by every thread that
  // launches the walk: always raise it to the device maximum, never lower it
  NG_CUDA(c, cudaFuncSetAttribute(k_walk<D, ACC64, REL, VARD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)c->smem_optin));
  int per_sm = 0;
  NG_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk<D, ACC64, REL, VARD>, nwarps * 32,
                                                           smem));
  if (per_sm < 1) per_sm = 1;
  // persistent warps take groups from a counter: no more blocks than the
  // expected groups need, so small problems leave SMs to concurrent work
  const int64_t want = (std::max<int64_t>(groups, 1) + nwarps - 1) / nwarps;
  const int grid = (int)std::min<int64_t>((int64_t)c->nsm * per_sm, want);
  k_walk<D, ACC64, REL, VARD><<<grid, nwarps * 32, smem, stream>>>(L);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

void fill_walk_desc(ng_ctx* c, float* acc, bool accumulate, WalkDesc* d) {
  fill_walk_desc_dr(c, acc, accumulate, c->dr_phys, d);
}

void fill_walk_desc_dr(ng_ctx* c, float* acc, bool accumulate, double dr, WalkDesc* d) {
  d->geo = as<float4>(c->n_geo);
  d->com = as<float4>(c->n_com);
  d->link = as<int4>(c->n_link);
  d->mono = as<float4>(c->n_mono);
  d->body = as<float4>(c->body);
  d->btype = as<uint8_t>(c->stype);
  d->bleaf = as<uint32_t>(c->bleaf);
  d->groups = as<int2>(c->groups);
  d->perm = as<uint32_t>(c->vals_a);
  d->out = force_out(c);
  d->status = as<uint32_t>(c->status);
  d->acc = acc;
  d->n = c->n;
  d->accumulate = accumulate ? 1 : 0;
  d->s_tab = (float)(c->L / dr);
  d->rcut_box = (float)(c->rcut / c->L);
  d->theta2 = (float)(c->p.theta * c->p.theta);
  const double eps_tab = c->p.eps / dr;
  d->eps2_tab = (float)(eps_tab * eps_tab);
  d->out_scale = (float)(1.0 / (dr * dr));
  d->D = c->p.D;
  for (int i = 0; i < kMaxD; ++i)
    for (int j = 0; j < kMaxD; ++j) {
      d->tabid[i][j] = c->tabid[i][j];
      d->G[i][j] = (float)c->p.G[i][j];
    }
  d->aold = relative_active(c) ? as<float>(c->aold) : nullptr;
  d->rel_scale = (float)(c->p.alpha * c->L * c->L / coupling_max(c));
}

template <bool ACC64, bool REL>
static int dispatch_walk_acc(ng_ctx* c, cudaStream_t stream, const WalkLaunch& L, int64_t groups,
                             bool vard) {
  if (vard) return launch_walk_d<kMaxD, ACC64, REL, true>(c, stream, L, groups);
  switch (c->p.D) {
    case 1: return launch_walk_d<1, ACC64, REL, false>(c, stream, L, groups);
    case 2: return launch_walk_d<2, ACC64, REL, false>(c, stream, L, groups);
    case 3: return launch_walk_d<3, ACC64, REL, false>(c, stream, L, groups);
    case 4: return launch_walk_d<4, ACC64, REL, false>(c, stream, L, groups);
    case 5: return launch_walk_d<5, ACC64, REL, false>(c, stream, L, groups);
    default: return launch_walk_d<6, ACC64, REL, false>(c, stream, L, groups);
  }
}

static int dispatch_walk(ng_ctx* c, cudaStream_t stream, const WalkLaunch& L, int64_t groups,
                         bool rel, bool vard) {
  if (c->p.accumulate_fp64)
    return rel ? dispatch_walk_acc<true, true>(c, stream, L, groups, vard)
               : dispatch_walk_acc<true, false>(c, stream, L, groups, vard);
  return rel ? dispatch_walk_acc<false, true>(c, stream, L, groups, vard)
             : dispatch_walk_acc<false, false>(c, stream, L, groups, vard);
}

int64_t walk_groups_hint(const ng_ctx* c) {
  // the group count of the last checked build of this size, else a guess
  // from the body count (grids only size the launch, every group is walked)
  return c->ngroups_n == c->n && c->ngroups > 0 ? c->ngroups : (c->n + 15) / 16;
}

// The walk of one launch over descriptors already in device memory (their
// group prefix and the work counter ready).
static int launch_walk_ready(ng_ctx* c, cudaStream_t stream, const WalkDesc* d_descs, int ndesc,
                             uint32_t* d_prefix, uint32_t* d_work, unsigned long long* counter,
                             int64_t groups, bool rel, const WalkTable* tab, bool vard) {
  WalkLaunch L;
  L.descs = d_descs;
  L.ndesc = ndesc;
  L.gprefix = d_prefix;
  L.work = d_work;
  if (tab) {
    L.tab = tab->tab;
    L.tab_entries = tab->ncut + 1;
    L.ncut = tab->ncut;
    L.tab_count = tab->count;
  } else {
    L.tab = as<float2>(c->d_tab);
    L.tab_entries = c->ncut + 1;
    L.ncut = c->ncut;
    L.tab_count = c->p.D * (c->ncut + 1) * walk_tab_pad(c->p.D);
  }
  L.counter = counter;
  return dispatch_walk(c, stream, L, groups, rel, vard);
}

int launch_walk_descs(ng_ctx* c, cudaStream_t stream, const WalkDesc* d_descs, int ndesc,
                      uint32_t* d_prefix, uint32_t* d_work, unsigned long long* counter,
                      int64_t groups, bool rel, const WalkTable* tab, bool vard) {
  k_walk_prep<<<1, 1024, 0, stream>>>(d_descs, ndesc, d_prefix, d_work);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return launch_walk_ready(c, stream, d_descs, ndesc, d_prefix, d_work, counter, groups, rel, tab,
                           vard);
}

// One simulation: the descriptor travels as a kernel argument (captured by
// value, also in graphs) and one thread stores it to device memory with the
// group prefix and the zeroed work counter, so no host buffer has to outlive
// the launch and no pageable copy stalls the stream.
__global__ void k_walk_prep1(const WalkDesc d, WalkDesc* out, uint32_t* gprefix, uint32_t* work) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *out = d;
    uint32_t ng = d.status[ST_NGROUPS];
    if (ng > (uint64_t)d.n) ng = (uint32_t)d.n;
    if (d.status[ST_FLAGS] & SF_NODE_OVERFLOW) ng = 0;
    gprefix[0] = 0;
    gprefix[1] = ng;
    *work = 0;
  }
}

int launch_walk(ng_ctx* c, float* acc, bool accumulate, bool count) {
  NG_TRY(ensure(c, c->walk_desc, sizeof(WalkDesc)));
  NG_TRY(ensure(c, c->walk_prefix, 4 * sizeof(uint32_t)));
  WalkDesc d;
  fill_walk_desc(c, acc, accumulate, &d);
  uint32_t* pre = as<uint32_t>(c->walk_prefix);
  k_walk_prep1<<<1, 32, 0, c->stream>>>(d, as<WalkDesc>(c->walk_desc), pre, pre + 2);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return launch_walk_ready(c, c->stream, as<WalkDesc>(c->walk_desc), 1, pre, pre + 2,
                           count ? as<unsigned long long>(c->counter) : nullptr,
                           walk_groups_hint(c), d.aold != nullptr, nullptr, false);
}

// ------------------------------------------------ per-particle count walk

// The algorithm's own unit of work: the per-particle walk with the geometric
// criterion evaluated in double precision (each operation rounded on its
// own, in the order of the definition). One thread per sorted body.
struct CountArgs {
  const uint8_t* level;
  const uint64_t* prefix;
  const uint32_t* first;
  const uint32_t* count;
  const uint8_t* nchild;
  const uint32_t* child;
  const double* m64;       // [node][D][4]
  const double* spos;
  const uint32_t* perm;
  int64_t n;
  int D;
  double invL, rcut2, theta;
  int64_t* out;            // [caller index] or nullptr
  unsigned long long* total;
  uint32_t* status;
  const float* aold;       // relative criterion: |a_old| per caller index
  double alphaL2, gmax;    // alpha L^2 (box units), largest coupling
  int relative;
};

constexpr int kCountStack = 192;

__global__ void __launch_bounds__(128) k_count(CountArgs a) {
  if (a.status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  unsigned long long mine = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x[3] = {a.spos[k] * a.invL, a.spos[a.n + k] * a.invL, a.spos[2 * a.n + k] * a.invL};
    uint32_t stack[kCountStack];
    int sp = 0;
    stack[sp++] = 0;
    long long cnt = 0;
    uint32_t visits = 0;
    const uint32_t nnodes = a.status[ST_LEVELS + kMaxLevel + 1];
    while (sp > 0) {
      if (++visits > nnodes) {
        atomicOr(&a.status[ST_FLAGS], (uint32_t)SF_BAD_TREE);
        break;
      }
      const uint32_t nd = stack[--sp];
      const int lvl = a.level[nd];
      const uint64_t pre = a.prefix[nd];
      const double side = 1.0 / (double)(1u << lvl);
      const double c[3] = {((double)morton_compact3(pre >> 2) + 0.5) * side,
                           ((double)morton_compact3(pre >> 1) + 0.5) * side,
                           ((double)morton_compact3(pre) + 0.5) * side};
      const double half = __dmul_rn(0.5, side);
      double g2 = 0.0, dcs[3];
      bool inside = true;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const double dc = nearest_image_unit(__dsub_rn(c[e], x[e]));
        dcs[e] = dc;
        double gap = __dsub_rn(fabs(dc), half);
        gap = gap > 0.0 ? gap : 0.0;
        g2 = __dadd_rn(g2, __dmul_rn(gap, gap));
        if (fabs(dc) > half) inside = false;
      }
      if (g2 >= a.rcut2) continue;
      const uint32_t nch = a.nchild[nd];
      if (!inside) {
        double mt = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        int nspec = 0;
        for (int t = 0; t < a.D; ++t) {
          const double* m = a.m64 + ((size_t)nd * a.D + t) * 4;
          mt += m[0];
          sx += m[1];
          sy += m[2];
          sz += m[3];
          nspec += m[0] > 0.0;
        }
        const double com[3] = {sx / mt, sy / mt, sz / mt};
        double dd2 = 0.0;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          const double v = nearest_image_unit(__dsub_rn(com[e], x[e]));
          dd2 = __dadd_rn(dd2, __dmul_rn(v, v));
        }
        bool accept;
        if (a.relative) {
          // outside the cube of side 1.2 l about the centre, and
          // G_max M l^2 <= alpha |a_old| r^4 (box units: alpha L^2)
          const double lim = __dmul_rn(0.6, side);
          bool near = true;
#pragma unroll
          for (int e = 0; e < 3; ++e)
            if (!(fabs(dcs[e]) < lim)) near = false;
          const double lhs = __dmul_rn(__dmul_rn(a.gmax, mt), __dmul_rn(side, side));
          const double rhs = __dmul_rn(__dmul_rn(a.alphaL2, (double)a.aold[a.perm[k]]),
                                       __dmul_rn(dd2, dd2));
          accept = !near && lhs <= rhs;
        } else {
          accept = side < __dmul_rn(a.theta, sqrt(dd2));
        }
        if (accept) {
          cnt += nspec;
          continue;
        }
      }
      if (nch == 0) {
        const uint32_t f = a.first[nd], c2 = a.count[nd];
        cnt += c2;
        if ((uint64_t)k >= f && (uint64_t)k < (uint64_t)f + c2) cnt -= 1;
      } else {
        if (sp + (int)nch > kCountStack) {
          atomicOr(&a.status[ST_FLAGS], (uint32_t)SF_STACK_OVERFLOW);
          break;
        }
        for (int ch = (int)nch - 1; ch >= 0; --ch) stack[sp++] = a.child[nd] + ch;
      }
    }
    if (a.out) a.out[a.perm[k]] = cnt;
    mine += (unsigned long long)cnt;
  }
  for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.total, mine);
}

int launch_count(ng_ctx* c, int64_t* counts) {
  CountArgs a;
  a.level = as<uint8_t>(c->n_level);
  a.prefix = as<uint64_t>(c->n_prefix);
  a.first = as<uint32_t>(c->n_first);
  a.count = as<uint32_t>(c->n_count);
  a.nchild = as<uint8_t>(c->n_nchild);
  a.child = as<uint32_t>(c->n_child);
  a.m64 = as<double>(c->n_m64);
  a.spos = as<double>(c->spos);
  a.perm = as<uint32_t>(c->vals_a);
  a.n = c->n;
  a.D = c->p.D;
  a.invL = 1.0 / c->L;
  const double rc = c->rcut / c->L;
  a.rcut2 = rc * rc;
  a.theta = c->p.theta;
  a.relative = relative_active(c) ? 1 : 0;
  a.aold = as<float>(c->aold);
  a.alphaL2 = c->p.alpha * c->L * c->L;
  a.gmax = coupling_max(c);
  a.out = counts;
  a.total = as<unsigned long long>(c->counter);
  a.status = as<uint32_t>(c->status);
  NG_CUDA(c, cudaMemsetAsync(a.total, 0, sizeof(unsigned long long), c->stream));
  const int blocks = (int)std::min<int64_t>((c->n + 127) / 128, (int64_t)c->nsm * 16);
  k_count<<<blocks, 128, 0, c->stream>>>(a);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

}  // namespace ng
