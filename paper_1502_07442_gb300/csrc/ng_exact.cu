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
  const uint32_t* perm;    // sorted -> caller
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
  float* acc;              // [3][n] caller order
  int accumulate;
  unsigned long long* counter;   // executed terms (optional)
  uint32_t* status;
};

__device__ __forceinline__ uint32_t xcompact3(uint64_t v) {
  v &= 0x1249249249249249ull;
  v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
  v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
  v = (v ^ (v >> 8)) & 0x1f0000ff0000ffull;
  v = (v ^ (v >> 16)) & 0x1f00000000ffffull;
  v = (v ^ (v >> 32)) & 0x1fffffull;
  return (uint32_t)v;
}

__device__ __forceinline__ double ximage(double d) { return __dsub_rn(d, rint(d)); }

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
      const double side = 1.0 / (double)(1u << a.level[nd]);
      const double c[3] = {((double)xcompact3(pre >> 2) + 0.5) * side,
                           ((double)xcompact3(pre >> 1) + 0.5) * side,
                           ((double)xcompact3(pre) + 0.5) * side};
      const double half = __dmul_rn(0.5, side);
      double g2 = 0.0, dcs[3];
      bool inside = true;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        const double dc = ximage(__dsub_rn(c[e], x[e]));
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
          const double v = ximage(__dsub_rn(com[e], x[e]));
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
            const double d[3] = {ximage(__dsub_rn(m[1] / m[0], x[0])) * a.L,
                                 ximage(__dsub_rn(m[2] / m[0], x[1])) * a.L,
                                 ximage(__dsub_rn(m[3] / m[0], x[2])) * a.L};
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
          const double d[3] = {ximage(__dsub_rn(a.spos[b] * a.invL, x[0])) * a.L,
                               ximage(__dsub_rn(a.spos[a.n + b] * a.invL, x[1])) * a.L,
                               ximage(__dsub_rn(a.spos[2 * a.n + b] * a.invL, x[2])) * a.L};
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
    const uint32_t i = a.perm[k];
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

// The short-range (or, in pure tree mode, the whole) tree force of a context.
int launch_tree_force(ng_ctx* c, float* acc, bool accumulate, bool count) {
  return c->p.pure_tree ? launch_walk_exact(c, acc, accumulate, count)
                        : launch_walk(c, acc, accumulate, count);
}

}  // namespace ng
