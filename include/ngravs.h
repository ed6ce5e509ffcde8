/*
 * ngravs — GB300-native multi-species TreePM force (C ABI).
 *
 * The problem (Croker, "ngravs: Distinct gravitational interactions in
 * GADGET-2", arXiv:1502.07442):
 *   D <= 6 gravitating species; a particle of passive species i feels a
 *   source of active species j through its own force law f_ij (Sec. 2,
 *   Eq. (map)), here Newtonian or Newtonian + Yukawa (Eq. (yukawa), C = 1).
 *   The force is split TreePM-style (Sec. 2.4.1): a short-range part
 *   evaluated by a Barnes-Hut walk whose nodes carry one monopole per species
 *   (Sec. 2.2), plus a long-range part from a particle-mesh step that deposits
 *   active masses per species and applies D x D Fourier kernels (Sec. 2.4).
 *
 * Conventions shared by every call:
 *  - Memory: every particle array is a DEVICE pointer owned by the caller,
 *    laid out structure-of-arrays: positions double[3][n] (x block, y block,
 *    z block), velocities float[3][n], accelerations float[3][n], species
 *    uint8[n] with values < D, masses float[n]. The library owns its own
 *    scratch (tree, tables, meshes), allocated with cudaMalloc on the device
 *    that is current when ng_create is called, and freed by ng_destroy.
 *  - Order: outputs are in the caller's particle order; the sorted order is
 *    exposed only through perm_out.
 *  - Streams: work is enqueued on the stream given to ng_create (or
 *    ng_set_stream) and is asynchronous unless a call says otherwise.
 *  - Errors: every call returns NG_OK (0) or a negative NG_E* code; no C++
 *    exception crosses the ABI. ng_last_error gives a message for the last
 *    failure on that context. A context is not thread-safe.
 *  - Coordinates: periodic box [0, L)^3; inputs outside are wrapped.
 */
#ifndef NGRAVS_H
#define NGRAVS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NG_MAX_SPECIES 6

enum {
  NG_OK = 0,
  NG_EINVAL = -1,    /* bad argument: D, n, box, law table, pointer */
  NG_ENOMEM = -2,    /* device allocation failed or a capacity was exceeded */
  NG_ECUDA = -3,     /* a CUDA or cuFFT call failed */
  NG_ETIMEOUT = -4,  /* a bounded device wait ran out */
  NG_EBUSY = -5,     /* serving admission refused (byte budget) */
  NG_ESTATE = -6     /* call out of order (e.g. force before build) */
};

enum { NG_NEWTON = 0, NG_YUKAWA = 1, NG_YUKAWA_PURE = 2, NG_MAHALO = 3 };
enum { NG_OPEN_GEOMETRIC = 0, NG_OPEN_RELATIVE = 1 };

/*
 * Parameters of one simulation (Sec. 2, Eq. (map); Sec. 2.4.1).
 *  G[i][j]        coupling for passive species i and active species j.
 *  law[i][j]      NG_NEWTON, or NG_YUKAWA for Eq. (yukawa) with C = 1:
 *                 phi_ij(r) = -G_ij M (1 + yuk_a[i][j] exp(-r / yuk_l[i][j])) / r,
 *                 or NG_YUKAWA_PURE for C = 0 (the pure Yukawa interaction of
 *                 Sec. 3.2): phi_ij(r) = -G_ij M yuk_a[i][j] exp(-r / yuk_l[i][j]) / r.
 *                 Both Yukawa kinds need yuk_l > 0; their long-range k-space
 *                 part carries the factor exp(-r_s^2 / yuk_l^2) of Sec. 3.2.
 *                 NG_MAHALO (pure tree mode only): the accumulator laws of
 *                 Sec. 3.3, phi_ij(r) = -G_ij (2 M m / (pi r)) atan(4 pi beta r / s)
 *                 with s = (j cored ? M / N_perp : 0) + (i cored ? m : 0), where
 *                 species k is cored when law[k][k] == NG_MAHALO, M and N_perp
 *                 are the active mass and body count behind a monopole (N_perp =
 *                 1 for a body) and m the passive mass (Eqs. (bambam), (01);
 *                 for a cored passive and point active species the scale is m
 *                 alone). At least one of i, j must be cored.
 *  eps            Plummer softening length (> 0): the radial law is
 *                 evaluated at rho = sqrt(r^2 + eps^2).
 *  box            periodic box side L.
 *  pm_mesh        PM mesh points per side N_m (power of two, 0 = no PM).
 *  asmth          split scale in mesh cells: r_s = asmth * L / N_m; when
 *                 pm_mesh == 0, r_s = asmth * L (short-range law still split).
 *  rcut_over_rs   short-range cut-off r_cut = rcut_over_rs * r_s (< L/2);
 *                 a term contributes iff rho < r_cut.
 *  theta          opening angle: a node of side l is used as D monopoles when
 *                 l < theta * d (d from the target group to the node's centre
 *                 of mass); theta = 0 opens every node (direct summation).
 *  opening        NG_OPEN_GEOMETRIC (theta) or NG_OPEN_RELATIVE: the Newtonian
 *                 relative criterion GADGET-2 uses and ngravs keeps (Sec. 2.2):
 *                 a node of side l, total mass M and centre of mass at
 *                 distance r is used when the target lies outside the cube of
 *                 side 1.2 l about the node centre and
 *                 G_max M l^2 <= alpha |a_old| r^4, G_max = max G[i][j] and
 *                 |a_old| the magnitude of the target's previous acceleration
 *                 (see ng_set_acc_old). Until a context holds |a_old| for its
 *                 bodies, the geometric criterion with theta is used.
 *  alpha          relative criterion tolerance (> 0 when opening is relative).
 *  pure_tree      1: pure tree mode (needs pm_mesh == 0): no TreePM split, every
 *                 law is evaluated whole, truncated at r_cut = rcut_over_rs *
 *                 asmth * L (< L/2, minimum image), by a per-particle walk.
 *                 2: periodic pure tree mode with the lattice corrections of
 *                 Sec. 2.3: no cut-off; every term is the nearest image's
 *                 plus the force of all other images of its source, tabulated
 *                 per law on a 64^3 grid over [0, L/2]^3 (Ewald sum for the
 *                 Newtonian part, image sum for Yukawa parts, which need
 *                 yuk_l <= L/8) and interpolated; not with Mahalo laws. The
 *                 tables are computed on the device when the context is
 *                 configured.
 *  ignore_nperp   1: Mahalo monopoles are treated as single objects (N_perp = 1),
 *                 the "without tracking" comparison of Sec. 3.3.
 *  beta           Mahalo scale beta (> 0 when a Mahalo law is used).
 *  accumulate_fp64  1: the group walk adds each evaluated list's FP32 sum into
 *                 an FP64 per-body accumulator (the FP64-accumulated variant);
 *                 0: FP32 accumulation throughout (default).
 *  leaf_size      maximum bodies per tree leaf (1..64, 0 = 8).
 *  group_size     particles per walk group (32 or 64, 0 = 32).
 *  table_size     short-range table entries per law (0 = automatic).
 *  group_cell     walk groups: runs of sibling cells of at most this many
 *                 bodies are cut into balanced chunks of <= group_size
 *                 (>= group_size, <= 4096; 0 = 32).
 */
typedef struct {
  int32_t D;
  int32_t pm_mesh;
  int32_t leaf_size;
  int32_t group_size;
  int32_t table_size;
  int32_t group_cell;
  double G[NG_MAX_SPECIES][NG_MAX_SPECIES];
  int32_t law[NG_MAX_SPECIES][NG_MAX_SPECIES];
  double yuk_a[NG_MAX_SPECIES][NG_MAX_SPECIES];
  double yuk_l[NG_MAX_SPECIES][NG_MAX_SPECIES];
  double eps;
  double box;
  double asmth;
  double rcut_over_rs;
  double theta;
  int32_t opening;
  int32_t reserved1;   /* must be 0 */
  double alpha;
  int32_t pure_tree;
  int32_t ignore_nperp;
  double beta;
  int32_t accumulate_fp64;
  int32_t reserved2;   /* must be 0 */
} ng_params;

typedef struct ng_ctx ng_ctx;

/*
 * Create a context for one simulation on the current CUDA device.
 * stream: a cudaStream_t passed as void* (NULL = legacy default stream).
 * Validates p (NG_EINVAL with a message on failure) and builds the
 * short-range tables on the host in double precision. *out is owned by the
 * caller and released with ng_destroy.
 */
int ng_create(ng_ctx** out, const ng_params* p, void* stream);
int ng_destroy(ng_ctx* ctx);
int ng_set_stream(ng_ctx* ctx, void* stream);

/*
 * Sort and tree build (Sec. 2.4 sort by Peano-Hilbert-type key and type,
 * Sec. 2.2 tree with per-species monopoles and N_perp counts).
 * Wraps positions into the box, forms 63-bit keys (20-bit Morton per axis,
 * x most significant, species in the low 3 bits), stable-sorts them, builds
 * the canonical octree (a cell is a leaf iff it holds <= leaf_size bodies or
 * is at level 20; children in octant order; nodes numbered breadth-first) and
 * reduces per-node per-species mass, centre of mass (double precision) and
 * body count. n >= 1; pos/type/mass are device arrays of n entries and are
 * only read. keys_out (uint64[n], sorted keys) and perm_out (uint32[n];
 * perm_out[k] = caller index of the k-th sorted body) are optional device
 * outputs. The tree stays valid until the next ng_build_tree on ctx.
 * Synchronises the stream once to size the tree (grows capacity as needed).
 */
int ng_build_tree(ng_ctx* ctx, int64_t n, const double* pos, const uint8_t* type,
                  const float* mass, uint64_t* keys_out, uint32_t* perm_out);

/*
 * Short-range tree force (Sec. 2.2 walk, Sec. 2.4.1 short-range law) on the
 * bodies of the last build: acc_out (device float[3][n], caller order) is
 * overwritten with the short-range acceleration. interactions_out (host,
 * optional) receives the number of particle-term evaluations the group walk
 * executed (synchronises the stream when non-NULL).
 */
int ng_tree_force(ng_ctx* ctx, float* acc_out, uint64_t* interactions_out);

/*
 * Previous accelerations for the relative opening criterion (Sec. 2.2): the
 * context keeps |a| of acc_old (device float[3][n], caller order; |a| formed
 * in FP32 as sqrt((x*x + y*y) + z*z), each operation rounded on its own).
 * With opening == NG_OPEN_RELATIVE every force evaluation of this context
 * on n bodies then uses these magnitudes, and afterwards replaces them with
 * the magnitudes of the acceleration it computed (the short-range part for
 * ng_tree_force, the total for ng_step and batches), as GADGET-2 does from
 * step to step. Served requests are independent and start without them.
 * NG_EINVAL for a NULL pointer or n outside [1, 2^31).
 */
int ng_set_acc_old(ng_ctx* ctx, int64_t n, const float* acc_old);

/*
 * Synchronous time step of Sec. 2.1.1, Eq. (our_timestep):
 *   dt = min(dt_max, sqrt(2 eta eps / (A_max |a|_max))),
 * the smallest of the per-particle steps, with |a|_max the largest |a| of acc
 * (device float[3][n]; |a| in FP32 as sqrt((x*x + y*y) + z*z)) and A_max the
 * bound |f_ij(r)| r^2 <= A_max M over the context's laws: G_ij for Newtonian
 * pairs, G_ij max(1, |1 + yuk_a|) for NG_YUKAWA, G_ij |yuk_a| for
 * NG_YUKAWA_PURE (maximum over i, j < D). dt_max > 0 and eta > 0; dt = dt_max
 * when every acceleration is zero. Writes the host double *dt_out and the
 * optional *amax_out (host, |a|_max). Synchronises the stream.
 */
int ng_timestep(ng_ctx* ctx, int64_t n, const float* acc, double eta, double dt_max,
                double* dt_out, float* amax_out);

/*
 * Per-particle walk interaction count (Sec. 2.2, the context's opening
 * criterion per target particle, double precision decisions): the number
 * of (accepted node, species with mass > 0) terms plus bodies of opened
 * leaves, the target excluded, summed over all bodies. This is the
 * algorithm's unit of work for throughput reports; it evaluates no force.
 * counts_out (device int64[n], caller order) is optional; *total_out (host)
 * receives the sum. Synchronises the stream.
 */
int ng_count_interactions(ng_ctx* ctx, int64_t* counts_out, uint64_t* total_out);

/*
 * Long-range PM acceleration (Sec. 2.4): CIC deposit of active masses per
 * species, D forward FFTs (cuFFT), the D x D Gaussian-filtered Green's
 * functions (Yukawa part scaled by exp(-mu^2 r_s^2), Sec. 3.2; CIC window
 * divided out twice; k = 0 removed), D inverse FFTs, 4-point
 * finite-difference gradient and CIC interpolation to each passive particle.
 * Uses the bodies of the last build; acc_out (device float[3][n], caller
 * order) is overwritten. NG_ESTATE when pm_mesh == 0.
 */
int ng_pm_force(ng_ctx* ctx, float* acc_out);

/*
 * Total acceleration of the bodies of the last build (Sec. 2.4.1: the TreePM
 * split of every law into a short-range part summed by the tree walk and a
 * long-range part from the mesh): the PM acceleration of ng_pm_force when
 * pm_mesh > 0, plus the short-range tree acceleration of ng_tree_force,
 * summed on the device into acc_out (device float[3][n], caller order,
 * overwritten). With pm_mesh == 0 it is the tree force alone. With the
 * relative criterion, |a_old| is then replaced by the magnitude of this
 * total. NG_ESTATE before ng_build_tree. Asynchronous on the stream.
 */
int ng_force(ng_ctx* ctx, float* acc_out);

/*
 * Kick-drift-kick leapfrog (Sec. 2.1.1) at fixed dt for nsteps steps:
 *   v += a dt/2 (float); x += v dt (double); wrap; a = a_short + a_long; v += a dt/2.
 * pos (double[3][n]) and vel (float[3][n]) are updated in place; acc
 * (float[3][n]) must hold the acceleration at pos when acc_valid != 0,
 * otherwise it is computed first; on return it holds the acceleration at the
 * final positions. Between steps the state stays in library buffers in the
 * previous step's sorted order (the caller's arrays are read once at the
 * start and written once at the end); each step after the first is replayed
 * from a captured CUDA graph. Synchronises the stream at the end to report
 * device errors.
 */
int ng_step(ng_ctx* ctx, int64_t n, double* pos, float* vel, const uint8_t* type,
            const float* mass, float* acc, int acc_valid, int nsteps, double dt);

/*
 * Export the canonical tree of the last build (for inspection and tests).
 * Returns the node count in *nnodes. Each array is optional (NULL skips it)
 * and is a HOST array of at least *nnodes (times D where stated) entries:
 * level int32, prefix uint64 (3*level Morton bits), first/count int64 (body
 * range in sorted order), nchild int32 (0 = leaf), child_first int64,
 * cnt uint32[node][D] (N_perp per species), mass double[node][D],
 * com double[node][D][3]. Synchronises the stream.
 */
/*
 * ng_step on host arrays (Sec. 2.1.1): the same integration for callers that
 * hold the particles in host memory (page-locked memory, e.g. from
 * cudaHostAlloc, copies at full link speed; pageable memory works but is
 * staged). pos (double[3][n]), vel (float[3][n]) and acc (float[3][n]) are
 * read and written back; type (uint8[n]) and mass (float[n]) are read. The
 * context keeps device copies of the arrays between calls (so a repeated call
 * with the same n replays the captured step). Synchronises the stream.
 */
int ng_step_host(ng_ctx* ctx, int64_t n, double* pos, float* vel, const uint8_t* type,
                 const float* mass, float* acc, int acc_valid, int nsteps, double dt);

int ng_tree_export(ng_ctx* ctx, int64_t* nnodes, int32_t* level, uint64_t* prefix,
                   int64_t* first, int64_t* count, int32_t* nchild, int64_t* child_first,
                   uint32_t* cnt, double* mass, double* com);

/*
 * Type-major order of the last build (Sec. 2.4: bodies grouped by type, each
 * type in key order): type_offsets (host int64[D+1]) and, optionally,
 * order_out (device uint32[n]; order_out[k] = caller index of the k-th body in
 * type-major order). Synchronises the stream.
 */
int ng_type_order(ng_ctx* ctx, int64_t* type_offsets, uint32_t* order_out);

/* ------------------------------------------------------------ batches
 *
 * Many independent simulations (uneven n, D, couplings) advanced together
 * on one GPU. The paper has no counterpart (it runs one simulation over MPI
 * ranks); each simulation still follows ng_step exactly. Within one batch
 * step every simulation's sort, tree and PM stages run on one of several
 * worker streams, and the short-range walk of all simulations that share the
 * species count and the law table is one persistent kernel launch whose
 * warps take (simulation, group) items from one work queue. The step is
 * captured once as a CUDA graph and replayed.
 */
typedef struct ng_batch ng_batch;

/* nsim >= 1 parameter blocks (validated as in ng_create; pure tree mode is
 * not batched: NG_EINVAL); stream as in ng_create. *out is released with
 * ng_batch_destroy. */
int ng_batch_create(ng_batch** out, int nsim, const ng_params* params, void* stream);
int ng_batch_destroy(ng_batch* b);

/*
 * nsteps kick-drift-kick steps of every simulation. Each argument is a HOST
 * array of nsim entries; the pointers in it are DEVICE arrays laid out as for
 * ng_step (n[i] bodies of simulation i). acc_valid as for ng_step. The first
 * call (and any call whose pointers, sizes or dt differ from the captured
 * ones) runs one step eagerly to size every buffer and captures the next.
 * Synchronises the stream at the end and reports device errors.
 */
int ng_batch_step(ng_batch* b, const int64_t* n, double* const* pos, float* const* vel,
                  const uint8_t* const* type, const float* const* mass, float* const* acc,
                  int acc_valid, int nsteps, double dt);

/* Number of simulations; number of walk launches per step: one per class of
 * simulations whose laws fit one law table laid out for 6 species (any
 * species counts; simulations whose laws agree on their species pairs, cut-off
 * and table spacing share a class). */
int ng_batch_size(const ng_batch* b);
int ng_batch_walk_launches(const ng_batch* b);
/* Kernels launched by all member contexts so far (see ng_launch_count). */
int ng_batch_launch_count(const ng_batch* b, uint64_t* out);
const char* ng_batch_last_error(const ng_batch* b);

/* ------------------------------------------------------------ serving
 *
 * A stream of independent requests (force evaluations and short
 * integrations, each a full solve as above; no paper counterpart). Requests
 * wait in a FIFO queue and are admitted while a slot is free and the device
 * memory the slots hold stays within the byte budget; every admitted request
 * runs asynchronously on its slot's own stream, so admitted requests overlap
 * on the GPU (continuous batching). The host never blocks on the device
 * except in ng_serve_wait / ng_serve, whose waits are bounded.
 */
enum { NG_REQ_FORCE = 0, NG_REQ_STEPS = 1 };

typedef struct {
  int32_t kind;          /* NG_REQ_FORCE: acceleration at pos; NG_REQ_STEPS: nsteps KDK steps */
  int32_t nsteps;
  double dt;
  ng_params params;
  int64_t n;
  /* HOST arrays (pinned memory lets the copies overlap), layouts as above;
   * they must stay valid until the request completes. vel may be NULL
   * (zero velocities). */
  const double* pos;
  const float* vel;
  const uint8_t* type;
  const float* mass;
  /* HOST outputs, each optional: acc_out float[3][n] (acceleration at the
   * final positions); pos_out / vel_out (NG_REQ_STEPS only). */
  double* pos_out;
  float* vel_out;
  float* acc_out;
} ng_request;

typedef struct {
  int32_t status;        /* 1 pending, NG_OK done, or an NG_E* code */
  int32_t reserved;
  double t_submit;       /* seconds on a monotonic clock */
  double t_admit;
  double t_done;
} ng_result;

typedef struct ng_server ng_server;

/* slots: concurrent requests (1..256); hbm_budget: bytes the slots may hold. */
int ng_serve_create(ng_server** out, int slots, size_t hbm_budget);
int ng_serve_destroy(ng_server* s);
/* Queue a request (validated on the host: NG_EINVAL; NG_EBUSY if it alone
 * exceeds the budget). *out is owned by the caller and updated in place. */
int ng_serve_submit(ng_server* s, const ng_request* r, ng_result* out, int64_t* id);
/* Cancel a request that has not been admitted yet (NG_ESTATE otherwise). */
int ng_serve_cancel(ng_server* s, int64_t id);
/* Non-blocking: collect finished requests, admit queued ones. */
int ng_serve_poll(ng_server* s, int* ncompleted);
/* Requests submitted and not finished. */
int ng_serve_pending(const ng_server* s);
/* Poll until nothing is pending or timeout_s elapses (NG_ETIMEOUT). */
int ng_serve_wait(ng_server* s, double timeout_s);
/* Run a trace: request k is submitted arrival_s[k] seconds after the call
 * starts (NULL: all at once), then everything is polled to completion within
 * timeout_s (NG_ETIMEOUT). res[k] receives each request's status and times
 * (t_submit = scheduled arrival). */
int ng_serve(ng_server* s, const ng_request* reqs, ng_result* res, int nreq,
             const double* arrival_s, double timeout_s);
const char* ng_serve_last_error(const ng_server* s);
/* Device bytes the server budgets for a request (particle arrays, sort and
 * tree buffers, PM meshes). */
size_t ng_serve_request_bytes(const ng_request* r);
/* Bookkeeping (no paper counterpart): bytes the slots hold now, the largest
 * sum seen after any admission or tree regrow (never above the budget), the
 * number of requests rerun with a larger tree capacity, and the number of
 * admissions that reconfigured a slot's context (parameters other than the
 * slot's previous request's, defaults filled in before comparing). A request
 * whose tree outgrows the slot is rerun only if the slot's larger holding
 * fits the budget beside the other slots; otherwise it fails with NG_ENOMEM.
 * Every device buffer and cuFFT plan a request needs is sized when it is
 * admitted, on the thread that admits it; the slots' launch threads only
 * enqueue work. Any output pointer may be NULL. */
int ng_serve_stats(const ng_server* s, size_t* held_bytes, size_t* peak_held_bytes,
                   int64_t* node_retries, int64_t* reconfigs);

/*
 * Stages of one force evaluation, in execution order (ng_stage_times):
 * Morton+type keys, the 8 radix passes, the gather into sorted order, the
 * octree levels, the monopoles, the walk groups, the type-major order, the
 * PM deposit (mesh clear + CIC), forward FFTs, k-space kernels, inverse
 * FFTs, gradient + interpolation, and the short-range tree force.
 */
enum {
  NG_STAGE_KEYS = 0, NG_STAGE_RADIX, NG_STAGE_GATHER, NG_STAGE_OCTREE, NG_STAGE_MONOPOLES,
  NG_STAGE_GROUPS, NG_STAGE_TYPE_ORDER, NG_STAGE_DEPOSIT, NG_STAGE_FFT_FWD, NG_STAGE_KSPACE,
  NG_STAGE_FFT_INV, NG_STAGE_INTERP, NG_STAGE_WALK, NG_NSTAGES
};

/*
 * Measurement (no paper counterpart): advances the n bodies (device arrays as
 * in ng_step) by two ng_step steps, untimed, which size every buffer and
 * bring the state into sorted order; then by one more step exactly as a
 * replayed ng_step step runs (resident sorted order), with a
 * CUDA event recorded on the context's stream before each stage of its sort,
 * tree build and force evaluation and after the last, and writes each
 * stage's milliseconds to ms_out[NG_NSTAGES] (host; 0 for stages the
 * context's mode does not run, e.g. the PM stages when pm_mesh == 0; the
 * kicks and the drift are not timed). pos, vel and acc hold the state after
 * the three steps on return. Synchronises the stream. Not to be called during
 * stream capture.
 */
int ng_stage_times(ng_ctx* ctx, int64_t n, double* pos, float* vel, const uint8_t* type,
                   const float* mass, float* acc, double dt, float* ms_out);

/*
 * Number of CUDA kernels this context has launched so far (host-side count,
 * library kernels only; cuFFT's own kernels are not included). A captured
 * step counts once when it is captured; each replay of the step graph adds
 * the kernels of one step. Used to report launches per timed region.
 */
int ng_launch_count(const ng_ctx* ctx, uint64_t* out);

/*
 * Radix passes (8 key bits each) of the context's last key sort: 8 for a
 * canonical build; fewer in steps whose trees stop at a level cap (captured
 * steps, served integrations), which sort only the Morton bits of their
 * levels. Sizes the sort's bytes in per-stage bandwidth figures.
 */
int ng_sort_passes(const ng_ctx* ctx, int32_t* out);

/*
 * Sorted keys and permutation without any allocation (the paper has no
 * counterpart: this is for callers that cannot call cudaMalloc, e.g. code
 * running while another framework holds the memory pool, or a host that
 * only lends the library its own buffers). Computes exactly the keys_out /
 * perm_out of ng_build_tree (same wrap, 63-bit key, stable order) for
 * 1 <= n <= 2^18 bodies, with its scratch in one fixed device array of about
 * 3.4 MB that every GPU loading the library holds until the process exits.
 * pos (double[3][n]), type (uint8[n]), keys_out (uint64[n]) and perm_out
 * (uint32[n]) are caller DEVICE arrays; stream as in ng_create. Returns
 * NG_EINVAL for n outside [1, 2^18], NULL arrays or box <= 0, NG_ECUDA if a
 * CUDA call or launch fails. Every call looks the scratch address up on the
 * current device (cudaGetSymbolAddress, never cached); the first call on a
 * device may load the library's device code there and should come before
 * any stream capture. All calls share the one scratch array: calls whose
 * work overlaps on the GPU (other streams or host threads) race on it.
 * Asynchronous on the stream.
 */
int ng_sort_keys_noalloc(int64_t n, const double* pos, const uint8_t* type, double box,
                         uint64_t* keys_out, uint32_t* perm_out, void* stream);

/* Message describing the last error on ctx (never NULL); with ctx == NULL,
 * the message of the last failed ng_create on the calling thread. */
const char* ng_last_error(const ng_ctx* ctx);

/* Library version string. */
const char* ng_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NGRAVS_H */
