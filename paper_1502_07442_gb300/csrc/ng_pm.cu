// Long-range PM step (Sec. 2.4; Sec. 2.4.1 split; Sec. 3.2 Yukawa filter).
//
// Per active species j the CIC-deposited mass mesh rho_j is transformed
// (cuFFT R2C, D transforms in one batched plan); every mode is then mapped
// in place to phi_i(k) = sum_j K_ij(k) rho_j(k) for all passive species i at
// once (the paper's D^2 passes, fused: each mode is read and written once);
// D inverse transforms give phi_i, and each particle of passive species i
// interpolates -grad phi_i (4-point differences at the 8 CIC corners).
//
// K_ij(k) = -4 pi G_ij [C_ij/k^2 + a_ij e^{-mu^2 r_s^2}/(k^2 + mu^2)] e^{-k^2 r_s^2}
//           / W(k)^2 / L^3,   W = prod_d sinc^2(pi n_d / N), K(0) = 0,
// with C_ij = 0 for the pure Yukawa law and 1 otherwise.
// The 1/L^3 folds the cell volume of the density and the 1/N^3 of the
// unnormalised inverse transform.
#include <cmath>

#include <mutex>

#include "ng_internal.cuh"

namespace ng {

struct PmLaw {
  float G[kMaxD][kMaxD];
  float yfac[kMaxD][kMaxD];   // a_ij exp(-mu^2 r_s^2), 0 for Newtonian pairs
  float mu2[kMaxD][kMaxD];
  float cnew[kMaxD][kMaxD];   // C of Eq. (yukawa): 1, or 0 for the pure Yukawa law
};

__global__ void k_cic_deposit(int64_t n, const uint32_t* __restrict__ order,
                              const double* __restrict__ spos, const float* __restrict__ smass,
                              const uint8_t* __restrict__ stype, int N, double cells_per_len,
                              float* __restrict__ rho) {
  const size_t N3 = (size_t)N * N * N;
  const int mask = N - 1;
  const int lane = threadIdx.x & 31;
  const uint32_t below = (1u << lane) - 1u;
  // whole warps step together (the shuffles below need every lane)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n;
       base += stride) {
    const int64_t j = base + lane;
    const bool valid = j < n;
    const uint32_t k = valid ? order[j] : 0u;
    const double ux = spos[k] * cells_per_len, uy = spos[n + k] * cells_per_len,
                 uz = spos[2 * n + k] * cells_per_len;
    const double fx0 = floor(ux), fy0 = floor(uy), fz0 = floor(uz);
    const float fx = (float)(ux - fx0), fy = (float)(uy - fy0), fz = (float)(uz - fz0);
    const int ix = (int)fx0 & mask, iy = (int)fy0 & mask, iz = (int)fz0 & mask;
    const int jx = (ix + 1) & mask, jy = (iy + 1) & mask, jz = (iz + 1) & mask;
    const size_t off = (size_t)stype[k] * N3;
    const float m = valid ? smass[k] : 0.f;
    const float wx0 = 1.f - fx, wy0 = 1.f - fy, wz0 = 1.f - fz;
    const size_t X0 = (size_t)ix * N * N, X1 = (size_t)jx * N * N;
    const size_t Y0 = (size_t)iy * N, Y1 = (size_t)jy * N;
    float w[8] = {m * wx0 * wy0 * wz0, m * wx0 * wy0 * fz, m * wx0 * fy * wz0, m * wx0 * fy * fz,
                  m * fx * wy0 * wz0,  m * fx * wy0 * fz,  m * fx * fy * wz0,  m * fx * fy * fz};
    // bodies in type-major Morton order: the bodies of one mesh cell and
    // species are consecutive, so consecutive lanes with the same cell form
    // runs; each run's weights are summed in registers and its last lane
    // adds them (one atomic per corner and run instead of per body)
    const size_t cell = valid ? off + X0 + Y0 + iz : ~(size_t)lane;
    const size_t prev = __shfl_up_sync(0xffffffffu, cell, 1);
    const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || prev != cell);
    bool tail = true;
    if (heads != 0xffffffffu) {
      const int head = 31 - __clz(heads & (below | (1u << lane)));
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float t = __shfl_up_sync(0xffffffffu, w[c], d);
          if (lane - d >= head) w[c] += t;
        }
      }
      tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    }
    if (valid && tail) {
      float* r = rho + off;
      atomicAdd(r + X0 + Y0 + iz, w[0]);
      atomicAdd(r + X0 + Y0 + jz, w[1]);
      atomicAdd(r + X0 + Y1 + iz, w[2]);
      atomicAdd(r + X0 + Y1 + jz, w[3]);
      atomicAdd(r + X1 + Y0 + iz, w[4]);
      atomicAdd(r + X1 + Y0 + jz, w[5]);
      atomicAdd(r + X1 + Y1 + iz, w[6]);
      atomicAdd(r + X1 + Y1 + jz, w[7]);
    }
  }
}

__device__ __forceinline__ float sinc_pi(int nd, int N) {
  if (nd == 0) return 1.f;
  const float x = 3.14159265358979f * (float)nd / (float)N;
  return sinf(x) / x;
}

template <int D>
__global__ void k_kspace(cufftComplex* __restrict__ mesh, int N, float kf, float rs2,
                         float pref, PmLaw law) {
  const int Nz = N / 2 + 1;
  const size_t modes = (size_t)N * N * Nz;
  for (size_t m = blockIdx.x * (size_t)blockDim.x + threadIdx.x; m < modes;
       m += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(m % Nz);
    const int y = (int)((m / Nz) % N);
    const int x = (int)(m / ((size_t)Nz * N));
    const int nx = x <= N / 2 ? x : x - N;
    const int ny = y <= N / 2 ? y : y - N;
    const int nz = z;
    cufftComplex in[D];
#pragma unroll
    for (int j = 0; j < D; ++j) in[j] = mesh[(size_t)j * modes + m];
    const float k2 = kf * kf * (float)(nx * nx + ny * ny + nz * nz);
    if (k2 == 0.f) {
#pragma unroll
      for (int i = 0; i < D; ++i) mesh[(size_t)i * modes + m] = make_cuComplex(0.f, 0.f);
      continue;
    }
    const float sx = sinc_pi(nx, N), sy = sinc_pi(ny, N), sz = sinc_pi(nz, N);
    const float w = sx * sx * sy * sy * sz * sz;
    const float filt = expf(-k2 * rs2) / (w * w) * pref;
    const float inv_k2 = 1.f / k2;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float re = 0.f, im = 0.f;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float K = law.cnew[i][j] * inv_k2;
        if (law.yfac[i][j] != 0.f) K += law.yfac[i][j] / (k2 + law.mu2[i][j]);
        K *= law.G[i][j] * filt;
        re = fmaf(K, in[j].x, re);
        im = fmaf(K, in[j].y, im);
      }
      mesh[(size_t)i * modes + m] = make_cuComplex(re, im);
    }
  }
}

// -grad phi_i by 4-point central differences at the 8 CIC corners of each
// particle of passive species i, interpolated with the CIC weights; written
// at perm[k] (caller order) or, with perm == nullptr, at k (sorted order).
// The three stencils of the 8 corners touch 56 distinct mesh points: along
// each axis, for each of the 4 corner lines, the 6 points from -2 to +3
// around the cell, the 2x2x2 corner block shared by the three axes. Each is
// loaded once (56 loads instead of 96).
__global__ void k_pm_interp(int64_t n, const double* __restrict__ spos,
                            const uint8_t* __restrict__ stype, const uint32_t* __restrict__ perm,
                            const float* __restrict__ phi, int N, double cells_per_len,
                            float inv_h, float* __restrict__ acc, int accumulate) {
  const size_t N3 = (size_t)N * N * N;
  const int mask = N - 1;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double ux = spos[k] * cells_per_len, uy = spos[n + k] * cells_per_len,
                 uz = spos[2 * n + k] * cells_per_len;
    const double fx0 = floor(ux), fy0 = floor(uy), fz0 = floor(uz);
    const float f[3] = {(float)(ux - fx0), (float)(uy - fy0), (float)(uz - fz0)};
    const int i0[3] = {(int)fx0, (int)fy0, (int)fz0};
    const float* P = phi + (size_t)stype[k] * N3;
    // wrapped offsets of the mesh points -2..+3 along each axis
    size_t ox[6], oy[6];
    int oz[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      ox[d] = (size_t)((i0[0] + d - 2) & mask) * N * N;
      oy[d] = (size_t)((i0[1] + d - 2) & mask) * N;
      oz[d] = (i0[2] + d - 2) & mask;
    }
    // X[b][e][j]: the x line at y offset b, z offset e (j = x offset + 2);
    // Y[a][e][j], Z[a][b][j] likewise; indices 2 and 3 are the corner block
    float X[2][2][6], Y[2][2][6], Z[2][2][6];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int j = 0; j < 6; ++j) X[b][e][j] = __ldg(P + ox[j] + oy[2 + b] + oz[2 + e]);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int j = 0; j < 6; ++j)
          Y[a][e][j] = (j == 2 || j == 3) ? X[j - 2][e][2 + a]
                                          : __ldg(P + ox[2 + a] + oy[j] + oz[2 + e]);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int j = 0; j < 6; ++j)
          Z[a][b][j] = (j == 2 || j == 3) ? X[b][j - 2][2 + a]
                                          : __ldg(P + ox[2 + a] + oy[2 + b] + oz[j]);
    float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float w = (a ? f[0] : 1.f - f[0]) * (b ? f[1] : 1.f - f[1]) * (e ? f[2] : 1.f - f[2]);
          const float* x = X[b][e];
          const float* y = Y[a][e];
          const float* z = Z[a][b];
          const float gx = (2.f / 3.f) * (x[a + 3] - x[a + 1]) - (1.f / 12.f) * (x[a + 4] - x[a]);
          const float gy = (2.f / 3.f) * (y[b + 3] - y[b + 1]) - (1.f / 12.f) * (y[b + 4] - y[b]);
          const float gz = (2.f / 3.f) * (z[e + 3] - z[e + 1]) - (1.f / 12.f) * (z[e + 4] - z[e]);
          g[0] = fmaf(w, gx, g[0]);
          g[1] = fmaf(w, gy, g[1]);
          g[2] = fmaf(w, gz, g[2]);
        }
    const uint32_t i = perm ? perm[k] : (uint32_t)k;
    const float s = -inv_h;
    if (accumulate) {
      acc[i] += s * g[0];
      acc[n + i] += s * g[1];
      acc[2 * n + i] += s * g[2];
    } else {
      acc[i] = s * g[0];
      acc[n + i] = s * g[1];
      acc[2 * n + i] = s * g[2];
    }
  }
}

// cuFFT plan creation and destruction are serialised across host threads
// (serving slots create plans concurrently); executing different plans from
// different threads needs no lock.
std::mutex g_fft_plan_lock;

static int pm_setup(ng_ctx* c) {
  const int N = c->p.pm_mesh, D = c->p.D;
  const size_t N3 = (size_t)N * N * N;
  const size_t modes = (size_t)N * N * (N / 2 + 1);
  NG_TRY(ensure(c, c->rho, (size_t)D * N3 * sizeof(float)));
  NG_TRY(ensure(c, c->rhok, (size_t)D * modes * sizeof(cufftComplex)));
  NG_TRY(ensure(c, c->phi, (size_t)D * N3 * sizeof(float)));
  for (const auto& pl : c->plans)
    if (pl.N == N && pl.D == D) {
      c->plan_r2c = pl.r2c;
      c->plan_c2r = pl.c2r;
      return NG_OK;
    }
  int dims[3] = {N, N, N};
  ng_ctx::Plan pl{N, D, 0, 0};
  std::lock_guard<std::mutex> lock(g_fft_plan_lock);
  if (cufftPlanMany(&pl.r2c, 3, dims, nullptr, 1, (int)N3, nullptr, 1, (int)modes,
                    CUFFT_R2C, D) != CUFFT_SUCCESS ||
      cufftPlanMany(&pl.c2r, 3, dims, nullptr, 1, (int)modes, nullptr, 1, (int)N3,
                    CUFFT_C2R, D) != CUFFT_SUCCESS) {
    if (pl.r2c) cufftDestroy(pl.r2c);
    return fail(c, NG_ECUDA, "cuFFT plan creation failed for a %d^3 mesh, batch %d", N, D);
  }
  c->plans.push_back(pl);
  c->plan_r2c = pl.r2c;
  c->plan_c2r = pl.c2r;
  return NG_OK;
}

int pm_reserve(ng_ctx* c) { return c->p.pm_mesh > 0 ? pm_setup(c) : NG_OK; }

int pm_force(ng_ctx* c, float* acc, bool accumulate) {
  const int N = c->p.pm_mesh, D = c->p.D;
  if (N <= 0) return fail(c, NG_ESTATE, "pm_mesh is 0: no long-range step configured");
  NG_TRY(pm_setup(c));
  const size_t N3 = (size_t)N * N * N;
  const double L = c->L;
  stage_mark(c, NG_STAGE_DEPOSIT);
  NG_CUDA(c, cudaMemsetAsync(c->rho.p, 0, (size_t)D * N3 * sizeof(float), c->stream));
  const int grid = work_grid(c, c->n, 8);
  const int kgrid = work_grid(c, (int64_t)N * N * (N / 2 + 1), 8);
  c->launches += 3;   // deposit, k-space, interpolation (cuFFT kernels are the library's)
  k_cic_deposit<<<grid, 256, 0, c->stream>>>(c->n, as<uint32_t>(c->tperm), as<double>(c->spos),
                                            as<float>(c->smass), as<uint8_t>(c->stype), N,
                                            (double)N / L, as<float>(c->rho));
  NG_CUDA(c, cudaGetLastError());
  if (cufftSetStream(c->plan_r2c, c->stream) != CUFFT_SUCCESS ||
      cufftSetStream(c->plan_c2r, c->stream) != CUFFT_SUCCESS)
    return fail(c, NG_ECUDA, "cufftSetStream failed");
  stage_mark(c, NG_STAGE_FFT_FWD);
  if (cufftExecR2C(c->plan_r2c, as<cufftReal>(c->rho), as<cufftComplex>(c->rhok)) != CUFFT_SUCCESS)
    return fail(c, NG_ECUDA, "cufftExecR2C failed");
  PmLaw law{};
  for (int i = 0; i < kMaxD; ++i)
    for (int j = 0; j < kMaxD; ++j) {
      law.G[i][j] = (float)c->p.G[i][j];
      law.cnew[i][j] = i < D && j < D && c->p.law[i][j] == NG_YUKAWA_PURE ? 0.f : 1.f;
      if (i < D && j < D && (c->p.law[i][j] == NG_YUKAWA || c->p.law[i][j] == NG_YUKAWA_PURE)) {
        const double mu = 1.0 / c->p.yuk_l[i][j];
        law.mu2[i][j] = (float)(mu * mu);
        law.yfac[i][j] = (float)(c->p.yuk_a[i][j] * std::exp(-mu * mu * c->rs * c->rs));
      }
    }
  const float kf = (float)(2.0 * M_PI / L);
  const float pref = (float)(-4.0 * M_PI / (L * L * L));
  const float rs2 = (float)(c->rs * c->rs);
  cufftComplex* mk = as<cufftComplex>(c->rhok);
  stage_mark(c, NG_STAGE_KSPACE);
  switch (D) {
    case 1: k_kspace<1><<<kgrid, 256, 0, c->stream>>>(mk, N, kf, rs2, pref, law); break;
    case 2: k_kspace<2><<<kgrid, 256, 0, c->stream>>>(mk, N, kf, rs2, pref, law); break;
    case 3: k_kspace<3><<<kgrid, 256, 0, c->stream>>>(mk, N, kf, rs2, pref, law); break;
    case 4: k_kspace<4><<<kgrid, 256, 0, c->stream>>>(mk, N, kf, rs2, pref, law); break;
    case 5: k_kspace<5><<<kgrid, 256, 0, c->stream>>>(mk, N, kf, rs2, pref, law); break;
    default: k_kspace<6><<<kgrid, 256, 0, c->stream>>>(mk, N, kf, rs2, pref, law); break;
  }
  NG_CUDA(c, cudaGetLastError());
  stage_mark(c, NG_STAGE_FFT_INV);
  if (cufftExecC2R(c->plan_c2r, mk, as<cufftReal>(c->phi)) != CUFFT_SUCCESS)
    return fail(c, NG_ECUDA, "cufftExecC2R failed");
  stage_mark(c, NG_STAGE_INTERP);
  k_pm_interp<<<grid, 256, 0, c->stream>>>(c->n, as<double>(c->spos), as<uint8_t>(c->stype),
                                          force_out(c), as<float>(c->phi), N,
                                          (double)N / L, (float)(N / L), acc, accumulate ? 1 : 0);
  NG_CUDA(c, cudaGetLastError());
  return NG_OK;
}

}  // namespace ng
