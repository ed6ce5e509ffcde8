/*
 * FP64 CPU ORACLE for the multi-species TreePM force of "ngravs: Distinct
 * gravitational interactions in GADGET-2" (Croker, arXiv:1502.07442).
 *
 * THIS FILE IS TEST INFRASTRUCTURE. Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. The product library never
 * links, includes or calls it, and it shares no code with the CUDA path.
 *
 * Everything is plain double precision, written from the paper's definitions
 * in the order the paper states them, with no blocking or reordering beyond
 * what the definitions need. OpenMP only spreads independent targets over
 * cores. Built with -ffp-contract=off so that the integer-producing steps
 * (periodic wrap, Morton quantisation) round the same way on every host.
 *
 * Readings of the paper that these routines take:
 *  - Sec. 2, Eq. (map): f_ij with i the passive and j the active species;
 *    G is stored [passive][active].
 *  - Eq. (yukawa) with C = 1: phi_ij(r) = -G_ij M (1 + a_ij exp(-r/l_ij)) / r;
 *    and with C = 0 (Sec. 3.2, the pure Yukawa interaction of the transition
 *    test): phi_ij(r) = -G_ij M a_ij exp(-r/l_ij) / r.
 *  - Sec. 2.4.1: Gaussian split exp(-k^2 r_s^2) in k-space, erfc(r / 2 r_s)
 *    in real space; r_s = a_smth L / N_m (the printed "2 pi a_smth / L" is
 *    not a length and is read as garbled).
 *  - Sec. 3.2: the Yukawa k-space Green's function of the long-range part is
 *    scaled by exp(-mu^2 r_s^2), mu = 1 / l_ij. Its short-range complement
 *    is the closed form coded in short_factor() below.
 *  - Sec. 2 (D^2 softenings, kind unspecified): one Plummer length eps; the
 *    radial law F(r)/r is evaluated at rho = sqrt(r^2 + eps^2) and the
 *    vector is F(rho)/rho * r_vec. The cut-off (not given by the paper) is
 *    applied to the same argument: a term contributes iff rho < r_cut,
 *    i.e. r^2 + eps^2 < r_cut^2 (strict).
 *  - Sec. 2.2 tree: canonical Morton-prefix octree; a cell is a leaf iff it
 *    holds <= leaf_size bodies or sits at level 20. Per node and species:
 *    mass, centre of mass and body count (N_perp).
 *  - Sec. 2.2 walk: geometric opening with angle theta on the all-species
 *    centre of mass (accept iff side < theta * d and the target is not inside
 *    the cell); accepted nodes contribute one monopole per species with
 *    nonzero mass; rejected leaves are opened into bodies.
 *  - Sec. 2.4 PM: CIC deposit per active species, D forward FFTs, per-pair
 *    Green's functions (the paper's D^2 passes, equal by linearity), D
 *    inverse FFTs, 4-point finite-difference gradient, CIC interpolation to
 *    passive particles; CIC window divided out twice; k = 0 mode zeroed.
 *  - Sec. 2.1.1: kick-drift-kick leapfrog at fixed dt.
 *  - Sec. 2.3 lattice corrections (pure tree mode 2): the force of a source
 *    and all its periodic images is the nearest image's plus a correction
 *    that is smooth inside the cube |d_i| <= L/2; it is tabulated once per
 *    law on a grid over [0, L/2]^3 (Ewald summation for the Newtonian part,
 *    a plain image sum for the exponentially decaying Yukawa part) and
 *    interpolated trilinearly, with the sign of each component following its
 *    own axis. Softening applies to the nearest image only.
 *  - Sec. 3.3 accumulator ("Mahalo") laws, pure tree mode only: a species j
 *    is cored when law[j][j] is the Mahalo law; a Mahalo pair (passive i,
 *    active j) has phi = -(2 M m / (pi r)) atan(4 pi beta r / s) with the
 *    core scale s = (j cored ? M / N_perp : 0) + (i cored ? m : 0), N_perp the
 *    number of bodies of species j behind the monopole (1 for a body). This
 *    is Eq. (bambam) for i = j cored and Eq. (01) for a point passive
 *    species; for a cored passive and point active species it gives
 *    atan(4 pi beta r / m), where the printed Eq. (10) also carries N_perp
 *    (read as a misprint: the softening scale is the cored object's alone,
 *    and only then is the monopole exact for N_perp coincident bodies).
 *
 * Parity notes: every routine is pinned by tests/test_oracle_*.py against a
 * route that does not go through this file (closed forms, numerical
 * quadrature of Eq. (short_accel), brute force, Ewald sums, numpy FFT).
 */
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <deque>
#include <numeric>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

/* Parameters of one force evaluation (the oracle's own layout). */
typedef struct {
  int32_t D;            /* number of species, 1..6 */
  int32_t leaf_size;    /* canonical octree leaf capacity */
  int32_t pm_mesh;      /* N_m; 0 disables the PM part */
  int32_t pad0;
  double box;           /* periodic box side L */
  double eps;           /* Plummer softening length */
  double rs;            /* split scale r_s */
  double rcut;          /* short-range cut-off radius */
  double theta;         /* opening angle; 0 = open everything (direct) */
  double G[6][6];       /* coupling, [passive][active] */
  int32_t law[6][6];    /* 0 = Newtonian, 1 = Newtonian + Yukawa (C = 1) */
  double ya[6][6];      /* Yukawa strength alpha */
  double yl[6][6];      /* Yukawa range lambda */
  int32_t opening;      /* 0 geometric (theta), 1 relative (alpha, previous |a|) */
  int32_t pad1;
  double alpha;         /* relative criterion tolerance */
  int32_t pure_tree;    /* 1: no split, full laws truncated at rcut, no PM;
                           2: no split, every image: nearest image plus the
                           tabulated lattice correction, no cut-off, no PM */
  int32_t ignore_nperp; /* 1: Mahalo monopoles as single objects (N_perp := 1) */
  double beta;          /* Mahalo scale beta (Sec. 3.3) */
} or_params;

enum { OR_NEWTON = 0, OR_YUKAWA = 1, OR_YUKAWA_PURE = 2, OR_MAHALO = 3 };

/* ------------------------------------------------------------------ laws */

/* Newtonian short-range factor of Sec. 2.4.1: -r^2 d/dr[erfc(r/2r_s)/r]. */
static double newton_short(double r, double rs) {
  const double u = r / (2.0 * rs);
  return std::erfc(u) + (2.0 * u / std::sqrt(M_PI)) * std::exp(-u * u);
}

/* exp(x) * erfc(y) without overflow for large x (erfc underflows first). */
static double exp_erfc(double x, double y) {
  const double e = std::erfc(y);
  if (e <= 0.0) return 0.0;
  return std::exp(x + std::log(e));
}

/*
 * Dimensionless short-range factor T_ij(rho): the short-range acceleration
 * from a source of active mass M at separation vector r_vec is
 * G_ij M T_ij(rho) r_vec / rho^3.
 *
 * Newtonian part: erfc(u) + 2u/sqrt(pi) exp(-u^2), u = rho / 2 r_s.
 * Yukawa part (C = 1, alpha = a, lambda = l, mu = 1/l): the long-range
 * Fourier kernel 4 pi a exp(-(k^2 + mu^2) r_s^2) / (k^2 + mu^2) leaves the
 * real-space potential  -a S(r)/r  with
 *   S(r) = 1/2 [ e^{-mu r} erfc(u - mu r_s) + e^{mu r} erfc(u + mu r_s) ],
 * whose force factor is S - r S'. The pure Yukawa law (C = 0) has the Yukawa
 * part alone.
 */
double or_short_factor(int law, double a, double l, double rs, double rho) {
  double T = law == OR_YUKAWA_PURE ? 0.0 : newton_short(rho, rs);
  if (law == OR_YUKAWA || law == OR_YUKAWA_PURE) {
    const double mu = 1.0 / l;
    const double u = rho / (2.0 * rs);
    const double em = std::exp(-mu * rho) * std::erfc(u - mu * rs);
    const double ep = exp_erfc(mu * rho, u + mu * rs);
    const double S = 0.5 * (em + ep);
    const double dS = 0.5 * mu * (ep - em)
                    - std::exp(-u * u - mu * mu * rs * rs) / (rs * std::sqrt(M_PI));
    T += a * (S - rho * dS);
  }
  return T;
}

/* Unsplit force factor of Eq. (yukawa): |F| r^2 / (G M m). */
double or_full_factor(int law, double a, double l, double r) {
  double F = law == OR_YUKAWA_PURE ? 0.0 : 1.0;
  if (law == OR_YUKAWA || law == OR_YUKAWA_PURE) F += a * (1.0 + r / l) * std::exp(-r / l);
  return F;
}

/* Long-range k-space kernel without the -4 pi G factor and the CIC window:
 * [C/k^2 + a exp(-mu^2 r_s^2)/(k^2 + mu^2)] exp(-k^2 r_s^2), C = 0 for the
 * pure Yukawa law, else 1; 0 at k = 0. */
double or_long_kernel(int law, double a, double l, double rs, double k2) {
  if (k2 <= 0.0) return 0.0;
  double K = law == OR_YUKAWA_PURE ? 0.0 : 1.0 / k2;
  if (law == OR_YUKAWA || law == OR_YUKAWA_PURE) {
    const double mu = 1.0 / l;
    K += a * std::exp(-mu * mu * rs * rs) / (k2 + mu * mu);
  }
  return K * std::exp(-k2 * rs * rs);
}

/* ------------------------------------------------------------ geometry */

static double wrap_coord(double x, double L) {
  return x - L * std::floor(x / L);
}

static double min_image(double d, double L) {
  return d - L * std::nearbyint(d / L);
}

/* ------------------------------------------------- lattice corrections */

enum { kEwaldGrid = 64 };   /* grid intervals per axis over [0, L/2] */

/* Periodic acceleration toward a unit source and all its images at offset d
 * (source - target, box units, L = 1) minus the nearest image's d/|d|^3:
 * Ewald summation with splitting alpha = 2, real-space images |n_i| <= 3
 * (the first left out is >= 3.1 L away: erfc(6.2) ~ 1e-18), reciprocal
 * vectors |m_i| <= 5 (the first left out has exp(-k^2/4 alpha^2) ~ 1e-39). */
static void ewald_newton_correction(const double d[3], double out[3]) {
  const double alpha = 2.0;
  double a[3] = {0, 0, 0};
  for (int nx = -3; nx <= 3; ++nx)
    for (int ny = -3; ny <= 3; ++ny)
      for (int nz = -3; nz <= 3; ++nz) {
        const double v[3] = {d[0] + nx, d[1] + ny, d[2] + nz};
        const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (r == 0.0) continue;
        const double f = (std::erfc(alpha * r) +
                          2.0 * alpha * r / std::sqrt(M_PI) * std::exp(-alpha * alpha * r * r)) /
                         (r * r * r);
        for (int e = 0; e < 3; ++e) a[e] += f * v[e];
      }
  for (int mx = -5; mx <= 5; ++mx)
    for (int my = -5; my <= 5; ++my)
      for (int mz = -5; mz <= 5; ++mz) {
        if (mx == 0 && my == 0 && mz == 0) continue;
        const double k[3] = {2 * M_PI * mx, 2 * M_PI * my, 2 * M_PI * mz};
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        const double w = 4.0 * M_PI / k2 * std::exp(-k2 / (4.0 * alpha * alpha)) *
                         std::sin(k[0] * d[0] + k[1] * d[1] + k[2] * d[2]);
        for (int e = 0; e < 3; ++e) a[e] += w * k[e];
      }
  const double r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  for (int e = 0; e < 3; ++e) out[e] = a[e] - (r > 0.0 ? d[e] / (r * r * r) : 0.0);
}

/* Images other than the nearest of the Yukawa force a (1 + mu r) e^{-mu r} / r^2
 * (box units), |n_i| <= 4; the library requires mu >= 8 / L. */
static void yukawa_image_correction(double a, double mu, const double d[3], double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  for (int nx = -4; nx <= 4; ++nx)
    for (int ny = -4; ny <= 4; ++ny)
      for (int nz = -4; nz <= 4; ++nz) {
        if (nx == 0 && ny == 0 && nz == 0) continue;
        const double v[3] = {d[0] + nx, d[1] + ny, d[2] + nz};
        const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        const double f = a * (1.0 + mu * r) * std::exp(-mu * r) / (r * r * r);
        for (int e = 0; e < 3; ++e) out[e] += f * v[e];
      }
}

/* Lattice correction of law (kind, a, l) at offset d in box units (L = 1),
 * per unit G M: the Newtonian part (C = 1) by Ewald, the Yukawa part by
 * images. Exported for the tests. */
void or_lattice_correction(int kind, double a, double l_box, const double d[3], double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (kind != OR_YUKAWA_PURE) ewald_newton_correction(d, out);
  if (kind == OR_YUKAWA || kind == OR_YUKAWA_PURE) {
    double y[3];
    yukawa_image_correction(a, 1.0 / l_box, d, y);
    for (int e = 0; e < 3; ++e) out[e] += y[e];
  }
}

struct LatticeTable {
  int kind;
  double a, l_box;
  std::vector<double> v;   /* [(N+1)^3][3] over [0, 1/2]^3, box units */
};

static std::deque<LatticeTable>& lattice_cache() {   /* references stay valid */
  static std::deque<LatticeTable> cache;
  return cache;
}

static const LatticeTable& lattice_table(int kind, double a, double l_box) {
  auto& cache = lattice_cache();
  for (const auto& t : cache)
    if (t.kind == kind && t.a == a && t.l_box == l_box) return t;
  LatticeTable t{kind, a, l_box, {}};
  const int N = kEwaldGrid, P = N + 1;
  t.v.assign((size_t)P * P * P * 3, 0.0);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < P; ++i)
    for (int j = 0; j < P; ++j)
      for (int k = 0; k < P; ++k) {
        const double d[3] = {0.5 * i / N, 0.5 * j / N, 0.5 * k / N};
        or_lattice_correction(kind, a, l_box, d, &t.v[(((size_t)i * P + j) * P + k) * 3]);
      }
  cache.push_back(std::move(t));
  return cache.back();
}

/* The table of pair (s, t); built beforehand by prepare_lattice (the walks
 * and sums call this from parallel loops, which only read the cache). */
static const LatticeTable& pair_table(const or_params* p, int s, int t) {
  const int law = p->law[s][t];
  return lattice_table(law, law == OR_NEWTON ? 0.0 : p->ya[s][t],
                       law == OR_NEWTON ? 0.0 : p->yl[s][t] / p->box);
}

static void prepare_lattice(const or_params* p) {
  if (p->pure_tree != 2) return;
  for (int s = 0; s < p->D; ++s)
    for (int t = 0; t < p->D; ++t) pair_table(p, s, t);
}

/* Trilinear interpolation of the table at offset d (physical, min image),
 * returned per unit G M in physical units. */
static void lattice_interp(const LatticeTable& t, double L, const double d[3], double out[3]) {
  const int N = kEwaldGrid, P = N + 1;
  int i0[3];
  double f[3], sg[3];
  for (int e = 0; e < 3; ++e) {
    const double u = std::fabs(d[e]) / L * 2.0 * N;
    const double uc = std::min(u, (double)N);
    i0[e] = std::min((int)std::floor(uc), N - 1);
    f[e] = uc - i0[e];
    sg[e] = d[e] < 0.0 ? -1.0 : 1.0;
  }
  double c[3] = {0, 0, 0};
  for (int corner = 0; corner < 8; ++corner) {
    const int bx = corner >> 2, by = (corner >> 1) & 1, bz = corner & 1;
    const double w = (bx ? f[0] : 1 - f[0]) * (by ? f[1] : 1 - f[1]) * (bz ? f[2] : 1 - f[2]);
    const double* v = &t.v[((((size_t)(i0[0] + bx)) * P + (i0[1] + by)) * P + (i0[2] + bz)) * 3];
    for (int e = 0; e < 3; ++e) c[e] += w * v[e];
  }
  for (int e = 0; e < 3; ++e) out[e] = sg[e] * c[e] / (L * L);
}

/* Mahalo force factor |F| r^2 / (G M m) of phi = -(2 M m/(pi r)) atan(r/a),
 * a = s / (4 pi beta): (2/pi) [atan(x) - x / (1 + x^2)], x = r / a. */
double or_mahalo_factor(double beta, double scale, double r) {
  const double x = 4.0 * M_PI * beta * r / scale;
  return (2.0 / M_PI) * (std::atan(x) - x / (1.0 + x * x));
}

/* Force factor of pair (s, t) at (softened) separation rho: the short-range
 * part of the law, or in pure tree mode the whole law. nperp and mpass enter
 * only the Mahalo law: bodies behind the monopole, passive mass. */
static double pair_factor(const or_params* p, int s, int t, double M, double nperp,
                          double mpass, double rho) {
  const int law = p->law[s][t];
  if (!p->pure_tree) return or_short_factor(law, p->ya[s][t], p->yl[s][t], p->rs, rho);
  if (law != OR_MAHALO) return or_full_factor(law, p->ya[s][t], p->yl[s][t], rho);
  const double np = p->ignore_nperp ? 1.0 : nperp;
  const double scale = (p->law[t][t] == OR_MAHALO ? M / np : 0.0) +
                       (p->law[s][s] == OR_MAHALO ? mpass : 0.0);
  return or_mahalo_factor(p->beta, scale, rho);
}

/* Acceleration on a passive particle of species s and mass mpass from a point
 * of active mass M and species t standing for nperp bodies, at min-image
 * separation d (source - target); mag (optional) accumulates the magnitude
 * of the term. */
static void pair_accel(const or_params* p, int s, int t, double M, double nperp, double mpass,
                       const double d[3], double acc[3], double* mag = nullptr) {
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double q = r2 + p->eps * p->eps;
  if (p->pure_tree == 2) {
    double cv[3];
    lattice_interp(pair_table(p, s, t), p->box, d, cv);
    for (int e = 0; e < 3; ++e) acc[e] += p->G[s][t] * M * cv[e];
  } else if (!(q < p->rcut * p->rcut)) {
    return;
  }
  const double rho = std::sqrt(q);
  const double T = pair_factor(p, s, t, M, nperp, mpass, rho);
  const double f = p->G[s][t] * M * T / (rho * rho * rho);
  acc[0] += f * d[0];
  acc[1] += f * d[1];
  acc[2] += f * d[2];
  if (mag) *mag += std::fabs(f) * std::sqrt(r2);
}

/* --------------------------------------------------------- Morton keys */

/* Sec. 2.4 sort key: periodic wrap, 20-bit quantisation per axis, 3-way bit
 * interleave (x most significant), species in the low 3 bits. */
void or_keys(int64_t n, const double* pos, const uint8_t* type, double L,
             uint64_t* keys) {
  for (int64_t i = 0; i < n; ++i) {
    uint64_t q[3];
    for (int d = 0; d < 3; ++d) {
      const double w = wrap_coord(pos[d * n + i], L);
      double c = std::floor((w / L) * 1048576.0);
      if (c < 0.0) c = 0.0;
      if (c > 1048575.0) c = 1048575.0;
      q[d] = (uint64_t)c;
    }
    uint64_t m = 0;
    for (int b = 0; b < 20; ++b) {
      m |= ((q[0] >> b) & 1ull) << (3 * b + 2);
      m |= ((q[1] >> b) & 1ull) << (3 * b + 1);
      m |= ((q[2] >> b) & 1ull) << (3 * b);
    }
    keys[i] = (m << 3) | (uint64_t)(type[i] & 7);
  }
}

/* Stable sort of the keys: perm[k] = original index of the k-th body. */
void or_sort_perm(int64_t n, const uint64_t* keys, uint32_t* perm) {
  std::vector<uint32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0u);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](uint32_t a, uint32_t b) { return keys[a] < keys[b]; });
  std::copy(idx.begin(), idx.end(), perm);
}

/* ------------------------------------------------------------ the tree */

struct Node {
  int level;
  uint64_t prefix;
  int64_t first, count;
  int64_t child_first;
  int nchild;
};

struct Tree {
  std::vector<Node> nodes;
  std::vector<double> mass;     /* [node][D] */
  std::vector<double> com;      /* [node][D][3] absolute */
  std::vector<uint32_t> cnt;    /* [node][D] */
  std::vector<double> mtot;     /* [node] */
  std::vector<double> comtot;   /* [node][3] */
};

static void node_geometry(const Node& nd, double L, double c[3], double* side) {
  uint64_t ix = 0, iy = 0, iz = 0;
  for (int b = 0; b < nd.level; ++b) {
    iz |= ((nd.prefix >> (3 * b)) & 1ull) << b;
    iy |= ((nd.prefix >> (3 * b + 1)) & 1ull) << b;
    ix |= ((nd.prefix >> (3 * b + 2)) & 1ull) << b;
  }
  const double s = L / (double)(1ull << nd.level);
  c[0] = ((double)ix + 0.5) * s;
  c[1] = ((double)iy + 0.5) * s;
  c[2] = ((double)iz + 0.5) * s;
  *side = s;
}

/* Canonical octree over the sorted Morton codes (breadth-first, children in
 * octant order). spos/smass/stype are the sorted, wrapped body arrays. */
static void build_tree(const or_params* p, int64_t n, const uint64_t* skeys,
                       const double* spos, const float* smass,
                       const uint8_t* stype, Tree& T) {
  T.nodes.clear();
  if (n <= 0) return;
  T.nodes.push_back(Node{0, 0, 0, n, -1, 0});
  for (size_t idx = 0; idx < T.nodes.size(); ++idx) {
    Node nd = T.nodes[idx];
    if (nd.count <= p->leaf_size || nd.level == 20) continue;
    const int shift = 3 * (20 - (nd.level + 1));
    int64_t b = nd.first;
    const int64_t end = nd.first + nd.count;
    T.nodes[idx].child_first = (int64_t)T.nodes.size();
    int nch = 0;
    while (b < end) {
      const uint64_t oct = ((skeys[b] >> 3) >> shift) & 7ull;
      int64_t e = b;
      while (e < end && ((((skeys[e] >> 3) >> shift) & 7ull) == oct)) ++e;
      T.nodes.push_back(Node{nd.level + 1, (nd.prefix << 3) | oct, b, e - b, -1, 0});
      ++nch;
      b = e;
    }
    T.nodes[idx].nchild = nch;
  }
  const int D = p->D;
  const size_t nn = T.nodes.size();
  T.mass.assign(nn * D, 0.0);
  T.com.assign(nn * D * 3, 0.0);
  T.cnt.assign(nn * D, 0u);
  T.mtot.assign(nn, 0.0);
  T.comtot.assign(nn * 3, 0.0);
  /* monopoles: direct sums over each node's body range (Sec. 2.2) */
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t k = 0; k < (int64_t)nn; ++k) {
    const Node& nd = T.nodes[k];
    double msum[6] = {0}, xs[6][3] = {{0}}, mt = 0, xt[3] = {0, 0, 0};
    for (int64_t b = nd.first; b < nd.first + nd.count; ++b) {
      const int t = stype[b];
      const double m = smass[b];
      msum[t] += m;
      T.cnt[k * D + t] += 1;
      mt += m;
      for (int d = 0; d < 3; ++d) {
        xs[t][d] += m * spos[d * n + b];
        xt[d] += m * spos[d * n + b];
      }
    }
    for (int t = 0; t < D; ++t) {
      T.mass[k * D + t] = msum[t];
      for (int d = 0; d < 3; ++d)
        T.com[(k * D + t) * 3 + d] = msum[t] > 0 ? xs[t][d] / msum[t] : 0.0;
    }
    T.mtot[k] = mt;
    for (int d = 0; d < 3; ++d) T.comtot[k * 3 + d] = mt > 0 ? xt[d] / mt : 0.0;
  }
}

/* Sort + gather into sorted, wrapped arrays. */
static void sort_bodies(const or_params* p, int64_t n, const double* pos,
                        const uint8_t* type, const float* mass,
                        std::vector<uint64_t>& skeys, std::vector<uint32_t>& perm,
                        std::vector<double>& spos, std::vector<float>& smass,
                        std::vector<uint8_t>& stype) {
  std::vector<uint64_t> keys(n);
  or_keys(n, pos, type, p->box, keys.data());
  perm.resize(n);
  or_sort_perm(n, keys.data(), perm.data());
  skeys.resize(n);
  spos.resize(3 * n);
  smass.resize(n);
  stype.resize(n);
  for (int64_t k = 0; k < n; ++k) {
    const uint32_t i = perm[k];
    skeys[k] = keys[i];
    for (int d = 0; d < 3; ++d) spos[d * n + k] = wrap_coord(pos[d * n + i], p->box);
    smass[k] = mass[i];
    stype[k] = type[i];
  }
}

/*
 * Export the canonical tree. Returns the node count; when the output
 * pointers are non-null (sized for at least cap nodes) it fills, per node in
 * canonical order: level, prefix, first, count, child_first (-1 for leaves),
 * nchild, per-species counts [node][D], masses [node][D] and centres of mass
 * [node][D][3].
 */
int64_t or_tree(const or_params* p, int64_t n, const double* pos,
                const uint8_t* type, const float* mass, int64_t cap,
                int32_t* level, uint64_t* prefix, int64_t* first,
                int64_t* count, int64_t* child_first, int32_t* nchild,
                uint32_t* cnt, double* msp, double* comsp) {
  std::vector<uint64_t> skeys;
  std::vector<uint32_t> perm;
  std::vector<double> spos;
  std::vector<float> smass;
  std::vector<uint8_t> stype;
  sort_bodies(p, n, pos, type, mass, skeys, perm, spos, smass, stype);
  Tree T;
  build_tree(p, n, skeys.data(), spos.data(), smass.data(), stype.data(), T);
  const int64_t nn = (int64_t)T.nodes.size();
  if (level && cap >= nn) {
    const int D = p->D;
    for (int64_t k = 0; k < nn; ++k) {
      level[k] = T.nodes[k].level;
      prefix[k] = T.nodes[k].prefix;
      first[k] = T.nodes[k].first;
      count[k] = T.nodes[k].count;
      child_first[k] = T.nodes[k].child_first;
      nchild[k] = T.nodes[k].nchild;
      for (int t = 0; t < D; ++t) {
        cnt[k * D + t] = T.cnt[k * D + t];
        msp[k * D + t] = T.mass[k * D + t];
        for (int d = 0; d < 3; ++d) comsp[(k * D + t) * 3 + d] = T.com[(k * D + t) * 3 + d];
      }
    }
  }
  return nn;
}

/* ---------------------------------------------------- short-range forces */

void or_direct_mag(const or_params* p, int64_t n, const double* pos,
                   const uint8_t* type, const float* mass, int64_t ntgt,
                   const int64_t* tgt, double* acc, double* mag);

/* Brute-force direct short-range sum (Eq. (map) with N_perp = 1) for the
 * targets listed in tgt (original indices); acc is [3][ntgt]. */
void or_direct(const or_params* p, int64_t n, const double* pos,
               const uint8_t* type, const float* mass, int64_t ntgt,
               const int64_t* tgt, double* acc) {
  or_direct_mag(p, n, pos, type, mass, ntgt, tgt, acc, nullptr);
}

/* The same sum; mag (optional, [ntgt]) receives sum_k |a_k|, the scale of
 * the rounding error any finite-precision evaluation of the sum carries. */
void or_direct_mag(const or_params* p, int64_t n, const double* pos,
                   const uint8_t* type, const float* mass, int64_t ntgt,
                   const int64_t* tgt, double* acc, double* mag) {
  const double L = p->box;
  prepare_lattice(p);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < ntgt; ++q) {
    const int64_t i = tgt[q];
    double a[3] = {0, 0, 0}, m = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      if (k == i) continue;
      double d[3];
      for (int c = 0; c < 3; ++c) d[c] = min_image(pos[c * n + k] - pos[c * n + i], L);
      pair_accel(p, type[i], type[k], mass[k], 1.0, mass[i], d, a, &m);
    }
    for (int c = 0; c < 3; ++c) acc[c * ntgt + q] = a[c];
    if (mag) mag[q] = m;
  }
}

/* The same sum through a periodic cell list (cells of side >= r_cut). */
void or_direct_cells(const or_params* p, int64_t n, const double* pos,
                     const uint8_t* type, const float* mass, int64_t ntgt,
                     const int64_t* tgt, double* acc) {
  const double L = p->box;
  prepare_lattice(p);
  const int nc = p->pure_tree == 2 ? 0 : (int)std::floor(L / p->rcut);
  if (nc < 3) {
    or_direct(p, n, pos, type, mass, ntgt, tgt, acc);
    return;
  }
  const double h = L / nc;
  auto cell_of = [&](int64_t k, int c) {
    int v = (int)std::floor(wrap_coord(pos[c * n + k], L) / h);
    return std::min(std::max(v, 0), nc - 1);
  };
  std::vector<int64_t> head((size_t)nc * nc * nc, -1), next(n, -1);
  for (int64_t k = 0; k < n; ++k) {
    const int64_t cid = ((int64_t)cell_of(k, 0) * nc + cell_of(k, 1)) * nc + cell_of(k, 2);
    next[k] = head[cid];
    head[cid] = k;
  }
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < ntgt; ++q) {
    const int64_t i = tgt[q];
    double a[3] = {0, 0, 0};
    const int ci[3] = {cell_of(i, 0), cell_of(i, 1), cell_of(i, 2)};
    for (int dx = -1; dx <= 1; ++dx)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dz = -1; dz <= 1; ++dz) {
          const int cx = (ci[0] + dx + nc) % nc, cy = (ci[1] + dy + nc) % nc,
                    cz = (ci[2] + dz + nc) % nc;
          for (int64_t k = head[((int64_t)cx * nc + cy) * nc + cz]; k >= 0; k = next[k]) {
            if (k == i) continue;
            double d[3];
            for (int c = 0; c < 3; ++c) d[c] = min_image(pos[c * n + k] - pos[c * n + i], L);
            pair_accel(p, type[i], type[k], mass[k], 1.0, mass[i], d, a);
          }
        }
    for (int c = 0; c < 3; ++c) acc[c * ntgt + q] = a[c];
  }
}

/*
 * Per-particle Barnes-Hut walk (Sec. 2.2) over the canonical tree for the
 * targets in tgt (original indices). acc is [3][ntgt]; counts[q] receives the
 * number of evaluated terms: one per (accepted node, species with M > 0) and
 * one per body of an opened leaf (the target itself excluded).
 */
static double wall_seconds() {
#ifdef _OPENMP
  return omp_get_wtime();
#else
  return 0.0;
#endif
}

static void tree_walk(const or_params* p, int64_t n, const double* pos, const uint8_t* type,
                      const float* mass, const float* aold, int64_t ntgt, const int64_t* tgt,
                      double* acc, int64_t* counts, double* times);

void or_tree_walk(const or_params* p, int64_t n, const double* pos,
                  const uint8_t* type, const float* mass, int64_t ntgt,
                  const int64_t* tgt, double* acc, int64_t* counts) {
  tree_walk(p, n, pos, type, mass, nullptr, ntgt, tgt, acc, counts, nullptr);
}

/* The same walk; times (optional, 2 doubles) receives the wall seconds of the
 * sort + tree build and of the walk itself. */
void or_tree_walk_timed(const or_params* p, int64_t n, const double* pos,
                        const uint8_t* type, const float* mass, int64_t ntgt,
                        const int64_t* tgt, double* acc, int64_t* counts, double* times) {
  tree_walk(p, n, pos, type, mass, nullptr, ntgt, tgt, acc, counts, times);
}

/* The walk with the relative opening criterion when p->opening == 1:
 * aold[i] is the magnitude of body i's previous acceleration (original
 * order). Sec. 2.2: ngravs keeps GADGET-2's Newtonian relative criterion in
 * its single vectorised walk. A node of side l, total mass M and all-species
 * centre of mass at distance r is accepted iff the target lies outside the
 * cube of side 1.2 l about the node centre and G_max M l^2 <= alpha |a_old|
 * r^4, G_max the largest coupling (the Newtonian estimate bounds every
 * species' term). Without aold the geometric criterion is used, as for the
 * first force of a run. */
void or_tree_walk_aold(const or_params* p, int64_t n, const double* pos, const uint8_t* type,
                       const float* mass, const float* aold, int64_t ntgt, const int64_t* tgt,
                       double* acc, int64_t* counts) {
  tree_walk(p, n, pos, type, mass, aold, ntgt, tgt, acc, counts, nullptr);
}

static void tree_walk(const or_params* p, int64_t n, const double* pos, const uint8_t* type,
                      const float* mass, const float* aold, int64_t ntgt, const int64_t* tgt,
                      double* acc, int64_t* counts, double* times) {
  prepare_lattice(p);
  const double t0 = wall_seconds();
  std::vector<uint64_t> skeys;
  std::vector<uint32_t> perm;
  std::vector<double> spos;
  std::vector<float> smass;
  std::vector<uint8_t> stype;
  sort_bodies(p, n, pos, type, mass, skeys, perm, spos, smass, stype);
  Tree T;
  build_tree(p, n, skeys.data(), spos.data(), smass.data(), stype.data(), T);
  std::vector<int64_t> rank(n);
  for (int64_t k = 0; k < n; ++k) rank[perm[k]] = k;
  const double t1 = wall_seconds();
  const double L = p->box;
  const int D = p->D;
  const double rc2 = p->pure_tree == 2 ? INFINITY : p->rcut * p->rcut;
  const bool relative = p->opening == 1 && aold != nullptr;
  double gmax = 0.0;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) gmax = std::max(gmax, p->G[i][j]);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < ntgt; ++q) {
    const int64_t i = tgt[q];
    const double a_old = relative ? (double)aold[i] : 0.0;
    const int64_t si = rank[i];
    const int s = type[i];
    double x[3];
    for (int c = 0; c < 3; ++c) x[c] = spos[c * n + si];
    double a[3] = {0, 0, 0};
    int64_t cntq = 0;
    std::vector<int64_t> stack;
    stack.push_back(0);
    while (!stack.empty()) {
      const int64_t k = stack.back();
      stack.pop_back();
      const Node& nd = T.nodes[k];
      double c[3], side;
      node_geometry(nd, L, c, &side);
      const double half = 0.5 * side;
      double dc[3], g2 = 0.0;
      bool inside = true;
      for (int e = 0; e < 3; ++e) {
        dc[e] = min_image(c[e] - x[e], L);
        const double gap = std::max(0.0, std::fabs(dc[e]) - half);
        g2 += gap * gap;
        if (std::fabs(dc[e]) > half) inside = false;
      }
      if (g2 >= rc2) continue;
      if (!inside) {
        double dd2 = 0.0;
        for (int e = 0; e < 3; ++e) {
          const double v = min_image(T.comtot[k * 3 + e] - x[e], L);
          dd2 += v * v;
        }
        bool accept;
        if (relative) {
          const double lim = 0.6 * side;
          bool near = true;
          for (int e = 0; e < 3; ++e)
            if (!(std::fabs(dc[e]) < lim)) near = false;
          const double lhs = (gmax * T.mtot[k]) * (side * side);
          const double rhs = (p->alpha * a_old) * (dd2 * dd2);
          accept = !near && lhs <= rhs;
        } else {
          accept = side < p->theta * std::sqrt(dd2);
        }
        if (accept) {
          for (int t = 0; t < D; ++t) {
            const double M = T.mass[k * D + t];
            if (!(M > 0.0)) continue;
            double d[3];
            for (int e = 0; e < 3; ++e) d[e] = min_image(T.com[(k * D + t) * 3 + e] - x[e], L);
            pair_accel(p, s, t, M, (double)T.cnt[k * D + t], smass[si], d, a);
            ++cntq;
          }
          continue;
        }
      }
      if (nd.nchild == 0) {
        for (int64_t b = nd.first; b < nd.first + nd.count; ++b) {
          if (b == si) continue;
          double d[3];
          for (int e = 0; e < 3; ++e) d[e] = min_image(spos[e * n + b] - x[e], L);
          pair_accel(p, s, stype[b], smass[b], 1.0, smass[si], d, a);
          ++cntq;
        }
      } else {
        for (int ch = nd.nchild - 1; ch >= 0; --ch) stack.push_back(nd.child_first + ch);
      }
    }
    for (int c = 0; c < 3; ++c) acc[c * ntgt + q] = a[c];
    if (counts) counts[q] = cntq;
  }
  if (times) {
    times[0] = t1 - t0;
    times[1] = wall_seconds() - t1;
  }
}

/* ------------------------------------------------------------------- PM */

typedef std::complex<double> cplx;

/* In-place radix-2 complex FFT of length m (power of two); sign -1 forward. */
void or_fft1d(int64_t m, double* re, double* im, int sign) {
  for (int64_t i = 1, j = 0; i < m; ++i) {
    int64_t bit = m >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      std::swap(re[i], re[j]);
      std::swap(im[i], im[j]);
    }
  }
  for (int64_t len = 2; len <= m; len <<= 1) {
    for (int64_t i = 0; i < m; i += len) {
      for (int64_t k = 0; k < len / 2; ++k) {
        const double ang = sign * 2.0 * M_PI * (double)k / (double)len;
        const double wr = std::cos(ang), wi = std::sin(ang);
        const int64_t a = i + k, b = i + k + len / 2;
        const double xr = re[b] * wr - im[b] * wi;
        const double xi = re[b] * wi + im[b] * wr;
        re[b] = re[a] - xr;
        im[b] = im[a] - xi;
        re[a] += xr;
        im[a] += xi;
      }
    }
  }
}

/* 3D FFT of an N^3 complex mesh (index (x*N + y)*N + z) along each axis. */
static void fft3d(int64_t N, std::vector<cplx>& a, int sign) {
  std::vector<double> re(N), im(N);
  for (int axis = 0; axis < 3; ++axis) {
    for (int64_t u = 0; u < N; ++u)
      for (int64_t v = 0; v < N; ++v) {
        auto at = [&](int64_t w) -> cplx& {
          if (axis == 0) return a[(w * N + u) * N + v];
          if (axis == 1) return a[(u * N + w) * N + v];
          return a[(u * N + v) * N + w];
        };
        for (int64_t w = 0; w < N; ++w) {
          re[w] = at(w).real();
          im[w] = at(w).imag();
        }
        or_fft1d(N, re.data(), im.data(), sign);
        for (int64_t w = 0; w < N; ++w) at(w) = cplx(re[w], im[w]);
      }
  }
}

/* 3D FFT of an N^3 complex mesh given as separate re/im arrays. */
void or_fft3d(int64_t N, double* re, double* im, int sign) {
  std::vector<cplx> a(N * N * N);
  for (int64_t i = 0; i < N * N * N; ++i) a[i] = cplx(re[i], im[i]);
  fft3d(N, a, sign);
  for (int64_t i = 0; i < N * N * N; ++i) {
    re[i] = a[i].real();
    im[i] = a[i].imag();
  }
}

static double sinc(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }

/*
 * Long-range PM acceleration (Sec. 2.4) on every particle; acc is [3][n].
 * Mesh points sit at integer multiples of h = L / N_m.
 */
void or_pm(const or_params* p, int64_t n, const double* pos, const uint8_t* type,
           const float* mass, double* acc) {
  const int64_t N = p->pm_mesh;
  const int D = p->D;
  const double L = p->box, h = L / (double)N;
  const int64_t N3 = N * N * N;
  auto cell = [&](int64_t x, int64_t y, int64_t z) {
    return (((x % N + N) % N) * N + ((y % N + N) % N)) * N + ((z % N + N) % N);
  };
  /* CIC deposit per active species, as density */
  std::vector<std::vector<cplx>> rhok(D, std::vector<cplx>(N3, cplx(0, 0)));
  for (int64_t k = 0; k < n; ++k) {
    double u[3];
    int64_t i0[3];
    double f[3];
    for (int c = 0; c < 3; ++c) {
      u[c] = wrap_coord(pos[c * n + k], L) / h;
      i0[c] = (int64_t)std::floor(u[c]);
      f[c] = u[c] - (double)i0[c];
    }
    const double m = mass[k] / (h * h * h);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b)
        for (int c = 0; c < 2; ++c) {
          const double w = (a ? f[0] : 1 - f[0]) * (b ? f[1] : 1 - f[1]) * (c ? f[2] : 1 - f[2]);
          rhok[type[k]][cell(i0[0] + a, i0[1] + b, i0[2] + c)] += w * m;
        }
  }
  for (int j = 0; j < D; ++j) fft3d(N, rhok[j], -1);
  /* potential per passive species: phi_i = sum_j K_ij rho_j */
  std::vector<std::vector<cplx>> phik(D, std::vector<cplx>(N3, cplx(0, 0)));
  for (int64_t x = 0; x < N; ++x)
    for (int64_t y = 0; y < N; ++y)
      for (int64_t z = 0; z < N; ++z) {
        const int64_t nx = x <= N / 2 ? x : x - N;
        const int64_t ny = y <= N / 2 ? y : y - N;
        const int64_t nz = z <= N / 2 ? z : z - N;
        const double kf = 2.0 * M_PI / L;
        const double k2 = kf * kf * (double)(nx * nx + ny * ny + nz * nz);
        if (k2 == 0.0) continue;
        const double W = std::pow(sinc(M_PI * nx / (double)N), 2) *
                         std::pow(sinc(M_PI * ny / (double)N), 2) *
                         std::pow(sinc(M_PI * nz / (double)N), 2);
        const int64_t id = (x * N + y) * N + z;
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) {
            const double K = -4.0 * M_PI * p->G[i][j] *
                             or_long_kernel(p->law[i][j], p->ya[i][j], p->yl[i][j], p->rs, k2) /
                             (W * W);
            phik[i][id] += K * rhok[j][id];
          }
      }
  for (int i = 0; i < D; ++i) fft3d(N, phik[i], +1);
  /* 4-point finite-difference force mesh and CIC interpolation */
  std::vector<int> used(D, 0);
  for (int64_t k = 0; k < n; ++k) used[type[k]] = 1;
  std::vector<double> F(3 * N3);
  for (int i = 0; i < D; ++i) {
    if (!used[i]) continue;
    auto phi = [&](int64_t x, int64_t y, int64_t z) {
      return phik[i][cell(x, y, z)].real() / (double)N3;
    };
    for (int64_t x = 0; x < N; ++x)
      for (int64_t y = 0; y < N; ++y)
        for (int64_t z = 0; z < N; ++z) {
          const int64_t id = (x * N + y) * N + z;
          F[0 * N3 + id] = -((2.0 / 3.0) * (phi(x + 1, y, z) - phi(x - 1, y, z)) -
                             (1.0 / 12.0) * (phi(x + 2, y, z) - phi(x - 2, y, z))) / h;
          F[1 * N3 + id] = -((2.0 / 3.0) * (phi(x, y + 1, z) - phi(x, y - 1, z)) -
                             (1.0 / 12.0) * (phi(x, y + 2, z) - phi(x, y - 2, z))) / h;
          F[2 * N3 + id] = -((2.0 / 3.0) * (phi(x, y, z + 1) - phi(x, y, z - 1)) -
                             (1.0 / 12.0) * (phi(x, y, z + 2) - phi(x, y, z - 2))) / h;
        }
    for (int64_t k = 0; k < n; ++k) {
      if (type[k] != i) continue;
      double u[3], f[3];
      int64_t i0[3];
      for (int c = 0; c < 3; ++c) {
        u[c] = wrap_coord(pos[c * n + k], L) / h;
        i0[c] = (int64_t)std::floor(u[c]);
        f[c] = u[c] - (double)i0[c];
      }
      double a[3] = {0, 0, 0};
      for (int aa = 0; aa < 2; ++aa)
        for (int b = 0; b < 2; ++b)
          for (int c = 0; c < 2; ++c) {
            const double w = (aa ? f[0] : 1 - f[0]) * (b ? f[1] : 1 - f[1]) * (c ? f[2] : 1 - f[2]);
            const int64_t id = cell(i0[0] + aa, i0[1] + b, i0[2] + c);
            for (int e = 0; e < 3; ++e) a[e] += w * F[e * N3 + id];
          }
      for (int e = 0; e < 3; ++e) acc[e * n + k] = a[e];
    }
  }
}

/* ------------------------------------------------------ full force + KDK */

/* Total acceleration on every particle: short range (tree walk, or direct
 * when theta == 0) plus PM long range when pm_mesh > 0. acc is [3][n]. */
void or_force(const or_params* p, int64_t n, const double* pos, const uint8_t* type,
              const float* mass, double* acc) {
  std::vector<int64_t> all(n);
  std::iota(all.begin(), all.end(), (int64_t)0);
  if (p->theta > 0.0)
    or_tree_walk(p, n, pos, type, mass, n, all.data(), acc, nullptr);
  else
    or_direct_cells(p, n, pos, type, mass, n, all.data(), acc);
  if (p->pm_mesh > 0) {
    std::vector<double> al(3 * n, 0.0);
    or_pm(p, n, pos, type, mass, al.data());
    for (int64_t i = 0; i < 3 * n; ++i) acc[i] += al[i];
  }
}

/*
 * Kick-drift-kick leapfrog (Sec. 2.1.1) at fixed dt: the acceleration at the
 * initial positions is computed first, then each step is
 * v += a dt/2; x += v dt; wrap; a = a(x); v += a dt/2.
 * pos, vel are [3][n] and updated in place; acc receives the final a.
 */
void or_kdk(const or_params* p, int64_t n, double* pos, double* vel,
            const uint8_t* type, const float* mass, int nsteps, double dt,
            double* acc) {
  std::vector<double> a(3 * n);
  or_force(p, n, pos, type, mass, a.data());
  for (int s = 0; s < nsteps; ++s) {
    for (int64_t i = 0; i < 3 * n; ++i) vel[i] += 0.5 * dt * a[i];
    for (int64_t i = 0; i < 3 * n; ++i) pos[i] = wrap_coord(pos[i] + dt * vel[i], p->box);
    or_force(p, n, pos, type, mass, a.data());
    for (int64_t i = 0; i < 3 * n; ++i) vel[i] += 0.5 * dt * a[i];
  }
  if (acc) std::copy(a.begin(), a.end(), acc);
}

int or_set_threads(int nt) {
#ifdef _OPENMP
  if (nt > 0) omp_set_num_threads(nt);
  return omp_get_max_threads();
#else
  (void)nt;
  return 1;
#endif
}

}  /* extern "C" */
