// Pure tree mode (no TreePM split, no PM): the per-particle walk with the
// full laws, including the accumulator ("Mahalo") laws of Sec. 3.3 whose
// force depends on the number N_perp of bodies behind a monopole and on the
// passive mass, so it cannot be read from a table of separations.
//
// One thread per sorted body walks the tree with the criterion of the
// per-particle count (geometric or relative, decisions in FP64 as there),
// and evaluates every accepted species monopole and every body of an opened
// leaf with the pair's law in FP32 (FP64 offsets rounded once to FP32; the
// cut-off decided in FP64):
//   Newton         f = 1
//   Yukawa (C=1)   f = 1 + a (1 + r/l) e^{-r/l}
//   pure Yukawa    f = a (1 + r/l) e^{-r/l}
//   Mahalo         f = (2/pi) [atan(x) - x / (1 + x^2)], x = 4 pi beta r / s,
//                  s = (active cored ? M / N_perp : 0) + (passive cored ? m : 0)
// and the acceleration G M f(rho) d / rho^3 at the softened separation rho,
// for rho < r_cut (minimum image, r_cut < L/2). A species is cored when its
// own pair law is the Mahalo law.
//
// Pure tree mode 2 (Sec. 2.3 lattice corrections): no cut-off, and every
// term adds the force of all other periodic images of its source, read by
// trilinear interpolation from a table of the correction over [0, L/2]^3
// (one per distinct law; each component odd in its own axis, even in the
// others). The tables are computed here in FP64: an Ewald sum for the
// Newtonian part, an image sum for Yukawa parts (yuk_l <= L/8).
#include "ng_internal.cuh"

namespace ng {

namespace {

struct ExactArgs {
  const uint8_t* level;
  const uint64_t* prefix;
  const uint32_t* first;
  const uint32_t* count;
  const uint8_t* nchild;
  const uint32_t* child;
  const double* m64;       // [node][D][4]: M, sum m x, sum m y, sum m z (box units)
  const uint32_t* cnt;     // [node][D]: N_perp
  const double* spos;      // [3][n] sorted, physical
  const float* smass;      // [n] sorted
  const uint8_t* stype;    // [n] sorted
  const uint32_t* perm;    // sorted -> caller (previous accelerations)
  const uint32_t* out;     // sorted -> output index (nullptr: sorted order)
  int64_t n;
  int D;
  double invL, L;
  double rcut2_box;        // cut-off^2 in box units (node skipping)
  double theta;
  const float* aold;
  double alphaL2, gmax;
  int relative;
  int ignore_nperp;
  double rcut2, eps2;           // physical units (cut-off decided in FP64, as the oracle)
  float beta4pi;
  int8_t kind[kMaxD][kMaxD];
  float G[kMaxD][kMaxD], ya[kMaxD][kMaxD], inv_l[kMaxD][kMaxD];
  uint8_t cored[kMaxD];
  const float4* lattice;   // [law][(N+1)^3] corrections per unit G M (box units), or nullptr
  int lat_n;               // N
  float lat_scale;         // 2 N / L
  float lat_inv_l2;        // 1 / L^2
  int8_t tabid[kMaxD][kMaxD];
  float* acc;              // [3][n] output order
  int accumulate;
  unsigned long long* counter;   // executed terms (optional)
  uint32_t* status;
};

constexpr int kExactStack = 192;

// One term: passive species s of mass mp, active species t of mass M behind
// which stand np bodies, offset d (physical, source - target). The cut-off
// rho < r_cut is decided in FP64 with the oracle's operation order; the law
// is evaluated in FP32.
__device__ __forceinline__ void exact_term(const ExactArgs& a, int s, int t, float M, float np,
                                           float mp, const double d[3], float& ax, float& ay,
                                           float& az) {
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                              __dmul_rn(d[2], d[2]));
  const double q64 = __dadd_rn(r2, a.eps2);
  if (!(q64 < a.rcut2)) return;
  const float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
  const float q = (float)q64;
  const float rho = sqrtf(q);
  float f;
  const int kind = a.kind[s][t];
  if (kind == NG_MAHALO) {
    const float npu = a.ignore_nperp ? 1.f : np;
    const float scale = (a.cored[t] ? M / npu : 0.f) + (a.cored[s] ? mp : 0.f);
    const float x = a.beta4pi * rho / scale;
    f = 0.63661977236758134f * (atanf(x) - x / fmaf(x, x, 1.f));
  } else {
    f = kind == NG_YUKAWA_PURE ? 0.f : 1.f;
    if (kind == NG_YUKAWA || kind == NG_YUKAWA_PURE) {
      const float u = rho * a.inv_l[s][t];
      f = fmaf(a.ya[s][t] * (1.f + u), expf(-u), f);
    }
  }
  const float g = a.G[s][t] * M * f / (q * rho);
  ax = fmaf(g, dx, ax);
  ay = fmaf(g, dy, ay);
  az = fmaf(g, dz, az);
  if (a.lattice) {
    // all other images: trilinear interpolation at |d|, signs per axis
    const int N = a.lat_n, P = N + 1;
    const float4* T = a.lattice + (size_t)a.tabid[s][t] * P * P * P;
    const float dv[3] = {dx, dy, dz};
    int i0[3];
    float fr[3];
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const float u = fminf(fabsf(dv[e]) * a.lat_scale, (float)N);
      i0[e] = min((int)u, N - 1);
      fr[e] = u - (float)i0[e];
    }
    float cx = 0.f, cy = 0.f, cz = 0.f;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      const int bx = corner >> 2, by = (corner >> 1) & 1, bz = corner & 1;
      const float w = (bx ? fr[0] : 1.f - fr[0]) * (by ? fr[1] : 1.f - fr[1]) *
                      (bz ? fr[2] : 1.f - fr[2]);
      const float4 v = __ldg(T + ((size_t)(i0[0] + bx) * P + (i0[1] + by)) * P + (i0[2] + bz));
      cx = fmaf(w, v.x, cx);
      cy = fmaf(w, v.y, cy);
      cz = fmaf(w, v.z, cz);
    }
    const float gc = a.G[s][t] * M * a.lat_inv_l2;
    // the table holds d_e >= 0; the component flips with the sign of d_e
    ax = fmaf(gc, dx < 0.f ? -cx : cx, ax);
    ay = fmaf(gc, dy < 0.f ? -cy : cy, ay);
    az = fmaf(gc, dz < 0.f ? -cz : cz, az);
  }
}

__global__ void __launch_bounds__(128) k_walk_exact(ExactArgs a) {
  if (a.status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  unsigned long long mine = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x[3] = {a.spos[k] * a.invL, a.spos[a.n + k] * a.invL,
                         a.spos[2 * a.n + k] * a.invL};
    const int s = a.stype[k];
    const float mp = a.smass[k];
    float ax = 0.f, ay = 0.f, az = 0.f;
    uint32_t stack[kExactStack];
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
      const uint64_t pre = a.prefix[nd];
      double c[3], side;
      node_centre(a.level[nd], pre, c, &side);
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
      if (g2 >= a.rcut2_box) continue;
      const uint32_t nch = a.nchild[nd];
      if (!inside) {
        double mt = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        for (int t = 0; t < a.D; ++t) {
          const double* m = a.m64 + ((size_t)nd * a.D + t) * 4;
          mt += m[0];
          sx += m[1];
          sy += m[2];
          sz += m[3];
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
          for (int t = 0; t < a.D; ++t) {
            const double* m = a.m64 + ((size_t)nd * a.D + t) * 4;
            if (!(m[0] > 0.0)) continue;
            const double d[3] = {nearest_image_unit(__dsub_rn(m[1] / m[0], x[0])) * a.L,
                                 nearest_image_unit(__dsub_rn(m[2] / m[0], x[1])) * a.L,
                                 nearest_image_unit(__dsub_rn(m[3] / m[0], x[2])) * a.L};
            exact_term(a, s, t, (float)m[0], (float)a.cnt[(size_t)nd * a.D + t], mp, d, ax, ay,
                       az);
            ++cnt;
          }
          continue;
        }
      }
      if (nch == 0) {
        const uint32_t f = a.first[nd], c2 = a.count[nd];
        for (uint32_t b = f; b < f + c2; ++b) {
          if ((int64_t)b == k) continue;
          const double d[3] = {nearest_image_unit(__dsub_rn(a.spos[b] * a.invL, x[0])) * a.L,
                               nearest_image_unit(__dsub_rn(a.spos[a.n + b] * a.invL, x[1])) * a.L,
                               nearest_image_unit(__dsub_rn(a.spos[2 * a.n + b] * a.invL, x[2])) * a.L};
          exact_term(a, s, a.stype[b], a.smass[b], 1.f, mp, d, ax, ay, az);
          ++cnt;
        }
      } else {
        if (sp + (int)nch > kExactStack) {
          atomicOr(&a.status[ST_FLAGS], (uint32_t)SF_STACK_OVERFLOW);
          break;
        }
        for (int ch = (int)nch - 1; ch >= 0; --ch) stack[sp++] = a.child[nd] + ch;
      }
    }
    const uint32_t i = a.out ? a.out[k] : (uint32_t)k;
    if (a.accumulate) {
      a.acc[i] += ax;
      a.acc[a.n + i] += ay;
      a.acc[2 * a.n + i] += az;
    } else {
      a.acc[i] = ax;
      a.acc[a.n + i] = ay;
      a.acc[2 * a.n + i] = az;
    }
    mine += (unsigned long long)cnt;
  }
  if (a.counter) {
    for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.counter, mine);
  }
}

}  // namespace

int launch_walk_exact(ng_ctx* c, float* acc, bool accumulate, bool count) {
  ExactArgs a{};
  a.level = as<uint8_t>(c->n_level);
  a.prefix = as<uint64_t>(c->n_prefix);
  a.first = as<uint32_t>(c->n_first);
  a.count = as<uint32_t>(c->n_count);
  a.nchild = as<uint8_t>(c->n_nchild);
  a.child = as<uint32_t>(c->n_child);
  a.m64 = as<double>(c->n_m64);
  a.cnt = as<uint32_t>(c->n_cnt);
  a.spos = as<double>(c->spos);
  a.smass = as<float>(c->smass);
  a.stype = as<uint8_t>(c->stype);
  a.perm = as<uint32_t>(c->vals_a);
  a.out = force_out(c);
  a.n = c->n;
  a.D = c->p.D;
  a.L = c->L;
  a.invL = 1.0 / c->L;
  const double rc = c->rcut / c->L;
  a.rcut2_box = rc * rc;
  a.theta = c->p.theta;
  a.relative = relative_active(c) ? 1 : 0;
  a.aold = as<float>(c->aold);
  a.alphaL2 = c->p.alpha * c->L * c->L;
  a.gmax = coupling_max(c);
  a.ignore_nperp = c->p.ignore_nperp;
  a.rcut2 = c->rcut * c->rcut;
  a.eps2 = c->p.eps * c->p.eps;
  a.beta4pi = (float)(4.0 * M_PI * c->p.beta);
  for (int i = 0; i < kMaxD; ++i) {
    a.cored[i] = i < c->p.D && c->p.law[i][i] == NG_MAHALO ? 1 : 0;
    for (int j = 0; j < kMaxD; ++j) {
      const bool in = i < c->p.D && j < c->p.D;
      a.kind[i][j] = (int8_t)(in ? c->p.law[i][j] : NG_NEWTON);
      a.G[i][j] = in ? (float)c->p.G[i][j] : 0.f;
      a.ya[i][j] = in ? (float)c->p.yuk_a[i][j] : 0.f;
      a.inv_l[i][j] = in && c->p.yuk_l[i][j] > 0 ? (float)(1.0 / c->p.yuk_l[i][j]) : 0.f;
    }
  }
  a.lattice = c->lattice_grid > 0 ? as<float4>(c->lattice) : nullptr;
  a.lat_n = c->lattice_grid;
  a.lat_scale = (float)(2.0 * c->lattice_grid / c->L);
  a.lat_inv_l2 = (float)(1.0 / (c->L * c->L));
  for (int i = 0; i < kMaxD; ++i)
    for (int j = 0; j < kMaxD; ++j) a.tabid[i][j] = c->tabid[i][j];
  a.acc = acc;
  a.accumulate = accumulate ? 1 : 0;
  a.counter = count ? as<unsigned long long>(c->counter) : nullptr;
  a.status = as<uint32_t>(c->status);
  const int blocks = (int)std::min<int64_t>((c->n + 127) / 128, (int64_t)c->nsm * 16);
  k_walk_exact<<<blocks, 128, 0, c->stream>>>(a);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

// ------------------------------------------------ lattice-correction tables

// Correction of one law at grid point (i, j, k) of [0, 1/2]^3 (box units,
// L = 1), per unit G M, FP64: all images but the nearest. Newtonian part by
// Ewald summation (splitting 2; real-space images |n_i| <= 3, reciprocal
// vectors |m_i| <= 5); Yukawa part a (1 + mu r) e^{-mu r} / r^2 by images
// |n_i| <= 4.
__global__ void k_lattice_table(int kind, double ya, double mu, int N, float4* out) {
  const int P = N + 1;
  const int64_t total = (int64_t)P * P * P;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(g / ((int64_t)P * P)), j = (int)((g / P) % P), k = (int)(g % P);
    const double d[3] = {0.5 * i / N, 0.5 * j / N, 0.5 * k / N};
    double acc[3] = {0.0, 0.0, 0.0};
    if (kind != NG_YUKAWA_PURE) {
      const double al = 2.0;
      for (int nx = -3; nx <= 3; ++nx)
        for (int ny = -3; ny <= 3; ++ny)
          for (int nz = -3; nz <= 3; ++nz) {
            const double v[3] = {d[0] + nx, d[1] + ny, d[2] + nz};
            const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (r == 0.0) continue;
            const double f = (erfc(al * r) + 2.0 * al * r * 0.56418958354775628 *
                                                 exp(-al * al * r * r)) / (r * r * r);
            for (int e = 0; e < 3; ++e) acc[e] += f * v[e];
          }
      for (int mx = -5; mx <= 5; ++mx)
        for (int my = -5; my <= 5; ++my)
          for (int mz = -5; mz <= 5; ++mz) {
            if (mx == 0 && my == 0 && mz == 0) continue;
            const double kv[3] = {2.0 * M_PI * mx, 2.0 * M_PI * my, 2.0 * M_PI * mz};
            const double k2 = kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2];
            const double w = 4.0 * M_PI / k2 * exp(-k2 / (4.0 * al * al)) *
                             sin(kv[0] * d[0] + kv[1] * d[1] + kv[2] * d[2]);
            for (int e = 0; e < 3; ++e) acc[e] += w * kv[e];
          }
      const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      if (r > 0.0)
        for (int e = 0; e < 3; ++e) acc[e] -= d[e] / (r * r * r);
    }
    if (kind == NG_YUKAWA || kind == NG_YUKAWA_PURE) {
      for (int nx = -4; nx <= 4; ++nx)
        for (int ny = -4; ny <= 4; ++ny)
          for (int nz = -4; nz <= 4; ++nz) {
            if (nx == 0 && ny == 0 && nz == 0) continue;
            const double v[3] = {d[0] + nx, d[1] + ny, d[2] + nz};
            const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            const double f = ya * (1.0 + mu * r) * exp(-mu * r) / (r * r * r);
            for (int e = 0; e < 3; ++e) acc[e] += f * v[e];
          }
    }
    out[g] = make_float4((float)acc[0], (float)acc[1], (float)acc[2], 0.f);
  }
}

int build_lattice(ng_ctx* c, int nlaws, const int* kind, const double* a, const double* l) {
  constexpr int N = 64;
  const size_t P3 = (size_t)(N + 1) * (N + 1) * (N + 1);
  NG_TRY(ensure(c, c->lattice, (size_t)nlaws * P3 * sizeof(float4)));
  for (int u = 0; u < nlaws; ++u) {
    const bool yk = kind[u] == NG_YUKAWA || kind[u] == NG_YUKAWA_PURE;
    k_lattice_table<<<work_grid(c, (int64_t)P3, 4), 256, 0, c->stream>>>(
        kind[u], yk ? a[u] : 0.0, yk ? c->L / l[u] : 0.0, N, as<float4>(c->lattice) + u * P3);
    c->launches += 1;
    NG_CUDA(c, cudaGetLastError());
  }
  c->lattice_grid = N;
  return NG_OK;
}

// The short-range (or, in pure tree mode, the whole) tree force of a context:
// the exact-law walk in pure tree mode, the FP64 pair sum in direct mode
// (theta = 0), the FP32 group walk otherwise.
int launch_tree_force(ng_ctx* c, float* acc, bool accumulate, bool count) {
  stage_mark(c, NG_STAGE_WALK);
  if (c->p.pure_tree) return launch_walk_exact(c, acc, accumulate, count);
  if (direct_mode(c)) return launch_direct64(c, acc, accumulate, count);
  return launch_walk(c, acc, accumulate, count);
}

}  // namespace ng
