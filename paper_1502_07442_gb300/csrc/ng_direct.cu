// Direct mode (opening angle theta = 0): the short-range sum of Eq. (map)
// with N_perp = 1 over every pair closer than r_cut, in FP64.
//
// With theta = 0 the geometric criterion accepts no node, so the walk opens
// every leaf the cut-off lets through and the tree only serves as a cell
// list. The FP32 group walk carries about 1e-6 relative error per term (table
// chords, FP32 offsets); where the terms of a body cancel, that error is
// large against the body's net force. Direct mode is the accuracy reference
// of the method, so here every term is formed in FP64: the minimum-image
// offset from the FP64 sorted positions, the closed-form short-range factor
// (the function that fills the walk's tables), and an FP64 sum per body,
// rounded once to FP32 at the end.
//
// One thread per sorted body walks the tree with the cut-off test of the
// per-particle count (the gap between the body and the node cube, FP64) and
// visits the bodies of every leaf it reaches, in Morton order, so that the
// threads of a warp walk neighbouring nodes.
#include "ng_internal.cuh"

namespace ng {

namespace {

struct DirectArgs {
  const uint8_t* level;
  const uint64_t* prefix;
  const uint32_t* count;
  const uint32_t* first;
  const uint8_t* nchild;
  const uint32_t* child;
  const double* spos;      // [3][n] sorted, physical
  const float* smass;      // [n] sorted
  const uint8_t* stype;    // [n] sorted
  const uint32_t* out;     // sorted -> output index (nullptr: sorted order)
  int64_t n;
  double L, invL;
  double rcut2_box;        // cut-off^2 in box units (node skipping)
  double rcut2, eps2, rs;  // physical units
  double G[kMaxD][kMaxD], ya[kMaxD][kMaxD], yl[kMaxD][kMaxD];
  int law[kMaxD][kMaxD];
  float* acc;              // [3][n] output order
  int accumulate;
  unsigned long long* counter;   // terms of opened leaves (optional)
  uint32_t* status;
};

constexpr int kDirectStack = 192;

__global__ void __launch_bounds__(128) k_direct64(DirectArgs a) {
  if (a.status[ST_FLAGS] & SF_NODE_OVERFLOW) return;
  unsigned long long mine = 0;
  const uint32_t nnodes = a.status[ST_LEVELS + kMaxLevel + 1];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double x[3] = {a.spos[k] * a.invL, a.spos[a.n + k] * a.invL,
                         a.spos[2 * a.n + k] * a.invL};
    const int s = a.stype[k];
    double ax = 0.0, ay = 0.0, az = 0.0;
    uint32_t stack[kDirectStack];
    int sp = 0;
    stack[sp++] = 0;
    long long cnt = 0;
    uint32_t visits = 0;
    while (sp > 0) {
      if (++visits > nnodes) {
        atomicOr(&a.status[ST_FLAGS], (uint32_t)SF_BAD_TREE);
        break;
      }
      const uint32_t nd = stack[--sp];
      const uint64_t pre = a.prefix[nd];
      double c[3], side;
      node_centre(a.level[nd], pre, c, &side);
      const double half = 0.5 * side;
      double g2 = 0.0;
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        double gap = fabs(nearest_image_unit(c[e] - x[e])) - half;
        gap = gap > 0.0 ? gap : 0.0;
        g2 += gap * gap;
      }
      if (g2 >= a.rcut2_box) continue;
      const uint32_t nch = a.nchild[nd];
      if (nch == 0) {
        const uint32_t f = a.first[nd], c2 = a.count[nd];
        for (uint32_t b = f; b < f + c2; ++b) {
          if ((int64_t)b == k) continue;
          ++cnt;
          const double dx = nearest_image_unit(a.spos[b] * a.invL - x[0]) * a.L;
          const double dy = nearest_image_unit(a.spos[a.n + b] * a.invL - x[1]) * a.L;
          const double dz = nearest_image_unit(a.spos[2 * a.n + b] * a.invL - x[2]) * a.L;
          const double q = dx * dx + dy * dy + dz * dz + a.eps2;
          if (!(q < a.rcut2)) continue;
          const int t = a.stype[b];
          const double rho = sqrt(q);
          const double T = short_law_factor(a.law[s][t], a.ya[s][t], a.yl[s][t], a.rs, rho);
          const double g = a.G[s][t] * (double)a.smass[b] * T / (q * rho);
          ax = fma(g, dx, ax);
          ay = fma(g, dy, ay);
          az = fma(g, dz, az);
        }
      } else {
        if (sp + (int)nch > kDirectStack) {
          atomicOr(&a.status[ST_FLAGS], (uint32_t)SF_STACK_OVERFLOW);
          break;
        }
        for (int ch = (int)nch - 1; ch >= 0; --ch) stack[sp++] = a.child[nd] + ch;
      }
    }
    const uint32_t i = a.out ? a.out[k] : (uint32_t)k;
    if (a.accumulate) {
      a.acc[i] = (float)((double)a.acc[i] + ax);
      a.acc[a.n + i] = (float)((double)a.acc[a.n + i] + ay);
      a.acc[2 * a.n + i] = (float)((double)a.acc[2 * a.n + i] + az);
    } else {
      a.acc[i] = (float)ax;
      a.acc[a.n + i] = (float)ay;
      a.acc[2 * a.n + i] = (float)az;
    }
    mine += (unsigned long long)cnt;
  }
  if (a.counter) {
    for (int o = 16; o; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(a.counter, mine);
  }
}

}  // namespace

bool direct_mode(const ng_ctx* c) {
  return c->p.theta == 0.0 && c->p.opening == NG_OPEN_GEOMETRIC && c->p.pure_tree == 0;
}

int launch_direct64(ng_ctx* c, float* acc, bool accumulate, bool count) {
  DirectArgs a{};
  a.level = as<uint8_t>(c->n_level);
  a.prefix = as<uint64_t>(c->n_prefix);
  a.first = as<uint32_t>(c->n_first);
  a.count = as<uint32_t>(c->n_count);
  a.nchild = as<uint8_t>(c->n_nchild);
  a.child = as<uint32_t>(c->n_child);
  a.spos = as<double>(c->spos);
  a.smass = as<float>(c->smass);
  a.stype = as<uint8_t>(c->stype);
  a.out = force_out(c);
  a.n = c->n;
  a.L = c->L;
  a.invL = 1.0 / c->L;
  const double rc = c->rcut / c->L;
  a.rcut2_box = rc * rc;
  a.rcut2 = c->rcut * c->rcut;
  a.eps2 = c->p.eps * c->p.eps;
  a.rs = c->rs;
  for (int i = 0; i < kMaxD; ++i)
    for (int j = 0; j < kMaxD; ++j) {
      const bool in = i < c->p.D && j < c->p.D;
      a.law[i][j] = in ? c->p.law[i][j] : NG_NEWTON;
      a.G[i][j] = in ? c->p.G[i][j] : 0.0;
      const bool yk = in && (c->p.law[i][j] == NG_YUKAWA || c->p.law[i][j] == NG_YUKAWA_PURE);
      a.ya[i][j] = yk ? c->p.yuk_a[i][j] : 0.0;
      a.yl[i][j] = yk ? c->p.yuk_l[i][j] : 1.0;
    }
  a.acc = acc;
  a.accumulate = accumulate ? 1 : 0;
  a.counter = count ? as<unsigned long long>(c->counter) : nullptr;
  a.status = as<uint32_t>(c->status);
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((c->n + 127) / 128, (int64_t)c->nsm * 16));
  k_direct64<<<blocks, 128, 0, c->stream>>>(a);
  c->launches += 1;
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

}  // namespace ng
