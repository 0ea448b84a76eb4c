/*
 * dao.h - C ABI of libdao.so: column-generation direct aperture optimisation
 * (DAO) for IMRT on one NVIDIA GB300 (sm_103a).
 *
 * Method: Men, Jia & Jiang, "GPU-based ultra-fast direct aperture optimization
 * for online adaptive radiation therapy" (arXiv:1003.5402).
 *   - model: dose z_j = sum_k D_kj y_k, y >= 0 (Sec. 2.1, Eqs. 1, 2, 6, 7);
 *   - objective: one-sided quadratic under/over-dose penalties per structure,
 *     weights divided by the structure's voxel count (Sec. 4, Eqs. 9-10, the
 *     per-structure form of Eqs. 3-5);
 *   - column generation: a master problem over the current aperture pool and a
 *     pricing sub-problem (Sec. 2.2-2.3, Eq. 8) solved row by row over the MLC.
 *
 * Conventions for every call below
 *   - Beamlet i of beam b, MLC row r, column c is i = off_b + r * cols[b] + c,
 *     off_b = sum_{b' < b} rows[b'] * cols[b'] (beam-major, row, column).
 *   - An aperture is given per MLC row of its beam as a half-open range
 *     [L, R) of open beamlets, 0 <= L <= R <= cols[b]; a closed row is (0, 0).
 *     leaf_lr arrays hold 2 * rows[b] int32: L_0, R_0, L_1, R_1, ...
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the context's device.  Every call is synchronous with
 *     respect to host outputs: when it returns, host outputs are written.
 *   - Errors: calls return a dao_status; no exception or abort crosses the
 *     ABI.  dao_last_error() gives a message for the calling thread's last
 *     failed call.  A failed call leaves the context usable unless it returns
 *     DAO_ECUDA (device state is then undefined; destroy the context) or
 *     DAO_ETIMEOUT from a solve (the device pool may hold rounds the host
 *     did not record; dao_reset the context).
 *   - A context is not thread-safe; different contexts are independent.
 */
#ifndef DAO_H
#define DAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dao_status {
    DAO_OK = 0,
    DAO_OPTIMAL = 1,      /* pricing found no aperture with a negative reduced cost (Sec. 2.2) */
    DAO_DUPLICATE = 2,    /* pricing returned an aperture already in the pool */
    DAO_EINVAL = -1,      /* invalid argument; nothing changed */
    DAO_ENOMEM = -2,      /* device or host allocation failed; nothing changed */
    DAO_ECUDA = -3,       /* a CUDA call failed; destroy the context */
    DAO_ETIMEOUT = -4,    /* a bounded device-side wait gave up; dao_reset the plan */
    DAO_EBUSY = -5,       /* no free slot / not enough free device memory */
    DAO_ESTATE = -6       /* call not valid in the current state (e.g. pool full) */
} dao_status;

/* D_ij of Eq. 2: voxel-major CSR (row j = voxel, column i = beamlet), host
 * memory, column indices strictly increasing within a row, values finite.
 * row_ptr has n_voxels + 1 entries, row_ptr[0] = 0, row_ptr[n_voxels] = nnz. */
typedef struct dao_csr {
    int32_t n_voxels;
    int32_t n_beamlets;
    int64_t nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* val;
} dao_csr;

/* MLC geometry: beam b has rows[b] MLC rows of cols[b] beamlets (host).
 * sum_b rows[b] * cols[b] must equal n_beamlets; 1 <= cols[b] <= 32. */
typedef struct dao_geometry {
    int32_t n_beams;
    const int32_t* rows;
    const int32_t* cols;
} dao_geometry;

/* Structures of Sec. 4: voxel_struct[j] in [0, n_structures) labels each voxel
 * with one structure (overlaps resolved by the caller); is_target[s] != 0
 * marks the targets T (under-dose term of Eq. 9 applies), all structures get
 * the over-dose term of Eq. 10.  n_structures <= 64.  Host memory. */
typedef struct dao_structures {
    int32_t n_structures;
    const int32_t* voxel_struct;
    const uint8_t* is_target;
} dao_structures;

/* Penalty weights of Eqs. 9-10 per structure (host): under_w = alpha_s,
 * over_w = beta_s, over_thresh = T_s^+.  When normalize_by_volume != 0 the
 * weights are divided by |v_s| (Eqs. 9-10); otherwise they are the per-voxel
 * alpha_j, beta_j of Eqs. 3-4.  Weights must be >= 0 and finite. */
typedef struct dao_weights {
    const double* under_w;
    const double* over_w;
    const double* over_thresh;
    int32_t normalize_by_volume;
} dao_weights;

enum { DAO_PREC_FP32 = 0, DAO_PREC_FP16 = 1, DAO_PREC_BF16 = 2 };

/* MLC hardware constraint of the pricing sub-problem (Sec. 4, last
 * paragraph).  Every mode keeps each row's open beamlets consecutive; the
 * paper's own pricing (Sec. 2.3) is DAO_MLC_CONSECUTIVE.
 *   DAO_MLC_INTERDIGITATION: the leaves of adjacent rows may not cross,
 *     L_r <= R_{r+1} and L_{r+1} <= R_r in boundary positions 0..cols, a
 *     closed row keeping its two leaves together at some position p that
 *     takes part in the constraint;
 *   DAO_MLC_CONNECTED: the open rows form one contiguous block of rows;
 *   DAO_MLC_JAWS: the aperture is a rectangle, one column range open in a
 *     contiguous block of rows (jaws-only delivery).
 * The constrained modes need at most 64 MLC rows per beam.  Their per-row
 * outputs (dao_k_price's row_best) hold the beam's value at the beam's first
 * row and 0 at the others. */
enum { DAO_MLC_CONSECUTIVE = 0, DAO_MLC_INTERDIGITATION = 1, DAO_MLC_CONNECTED = 2, DAO_MLC_JAWS = 3 };

/* Solver options; dao_options_default() fills every field. */
typedef struct dao_options {
    int32_t k_max;             /* aperture pool capacity, 1..64 (default 64) */
    int32_t max_master_iters;  /* projected-Newton iterations per master solve (default 50) */
    double master_tol;         /* stop when every |y_k - P(y_k - g_k)| <= master_tol * max|g(start)|
                                * + 64 u sum_j |S_jk pi_j| (u = 2^-24: FP32 rounding of g) (1e-6) */
    double price_tol;          /* optimal when reduced cost >= -price_tol * max(D) * ||grad F(0)||_1 (1e-7) */
    int32_t precision;         /* DAO_PREC_FP32 (default), DAO_PREC_FP16 or DAO_PREC_BF16 storage of D;
                                * 16-bit storage keeps beamlet indices in 16 bits (n_beamlets <= 65536) */
    int32_t device;            /* CUDA device ordinal (default 0) */
    void* stream;              /* cudaStream_t to run on; NULL = a stream owned by the context */
    int32_t use_graphs;        /* 1 (default): dao_solve runs on the device without host synchronisation
                                * between rounds: with the persistent master one CUDA graph per context
                                * whose device-side while node runs every round, else one graph per round;
                                * 0: host-driven launches */
    int32_t master_persistent; /* 1 (default): each master solve is one cooperative kernel whose blocks
                                * iterate together (bounded grid barriers); 0, or where a cooperative
                                * launch is not available: one launch per evaluation kernel */
    int32_t mlc_constraint;    /* DAO_MLC_* of the pricing (default DAO_MLC_CONSECUTIVE) */
    int32_t master_blocks;     /* blocks of the persistent master solve; 0 (default): two per SM, the whole
                                * GPU; fewer (raised to the least whose per-block working set fits shared
                                * memory) leave room for other plans' solves to run side by side */
    int32_t dt_threads;        /* threads per beamlet row of the transposed SpMV: 0 (default: 64, or the
                                * autotuner's choice), 64, 128 or 256 */
    int32_t dt_map;            /* form of the transposed SpMV: 0 (default: DAO_DT_CONSECUTIVE, or the
                                * autotuner's choice); DAO_DT_GROUPED (a block per beamlet row, a thread per
                                * 4 or 8 consecutive entries, 16-byte loads), DAO_DT_CONSECUTIVE (a block per
                                * row, consecutive entries on consecutive threads: the pi gathers of a warp
                                * fall on few cache lines) or DAO_DT_SPLIT (all entries split evenly over a
                                * fixed set of warps, consecutive entries on consecutive lanes; a row covered
                                * by several warps adds their partial sums in warp order; falls back to
                                * DAO_DT_CONSECUTIVE where a row is shorter than 32 entries) */
    int32_t dose_form;         /* form of the dose SpMV: 0 (default: DAO_DOSE_UNITS where its shared memory
                                * fits, or the autotuner's choice), DAO_DOSE_LANES (4 to 32 lanes per voxel
                                * row), DAO_DOSE_UNITS (one warp per 32 consecutive rows, their entries
                                * requested at once) or DAO_DOSE_MERGE (the merge of the stored entries and
                                * the row ends split evenly over a fixed set of warps, entries requested
                                * before any row offset; a row across two warps' stretches is finished by
                                * the later of the two) */
    int32_t column_lanes;      /* the aperture column (a4): 0 (default, or the autotuner's choice): one lane per
                                * voxel row over a copy of D stored by beams (each beam's part of every row in
                                * one contiguous range); 1, 2, 4, 8 or 16: lanes per voxel row over the row's
                                * segment of the beam in D */
    int32_t split_warps;       /* warps of the forms that split D's or D^T's stored entries evenly over warps
                                * (DAO_DOSE_MERGE, DAO_DT_SPLIT): 0 (default: 32 per SM) or any positive count
                                * (fewer warps take longer chunks; the dose form's chunk stays longer than
                                * the longest row and at most 1024 groups) */
} dao_options;

enum { DAO_DT_GROUPED = 1, DAO_DT_CONSECUTIVE = 2, DAO_DT_SPLIT = 3 };
enum { DAO_DOSE_LANES = 1, DAO_DOSE_UNITS = 2, DAO_DOSE_MERGE = 3 };

typedef struct dao_ctx dao_ctx;

void dao_options_default(dao_options* opt);

/* Create a plan context: validates the inputs (DAO_EINVAL on a malformed CSR,
 * geometry, labels or weights, or on a D whose rows, padded to 4 entries (8
 * with 16-bit storage), or whose transpose's rows, hold 2^31 entries or more:
 * the device offsets are 32-bit), copies D to the device in its own layout,
 * builds the transpose D^T (beamlet-major) used by pricing, and expands the
 * per-structure criteria.  prescriptions[s] is T_s^- for target s (ignored
 * for non-targets).  The caller keeps ownership of every input; *out is owned
 * by the caller and released with dao_destroy.  The pool starts empty
 * (y = [], z = 0). */
dao_status dao_create(const dao_csr* D, const dao_geometry* g, const dao_structures* s,
                      const dao_weights* w, const double* prescriptions,
                      const dao_options* opt, dao_ctx** out);

/* Re-optimisation mode (Sec. 4): the criteria of Eqs. 3-4 with a weight and a
 * threshold per voxel instead of per structure.  The paper re-plans on the
 * day's anatomy with alpha_j = beta_j = 1 and T_j = the planned dose deformed
 * onto that anatomy, so that the new plan reproduces the original dose.
 * Voxel j contributes under_w[j] max(0, under_t[j] - z_j)^2 +
 * over_w[j] max(0, z_j - over_t[j])^2 to F (Eq. 5); the weights are used as
 * given (no division by a structure volume).  The paper's mode is under_w = 1
 * on target voxels (Eq. 3 applies to V_T only; 0 elsewhere), over_w = 1 and
 * under_t = over_t = T_j.  Arrays: host double[n_voxels], weights >= 0 and
 * finite, thresholds finite (DAO_EINVAL otherwise); on the device each voxel
 * keeps FP32 weights and its thresholds as FP32 hi + lo pairs. */
typedef struct dao_voxel_terms {
    const double* under_w;
    const double* under_t;
    const double* over_w;
    const double* over_t;
} dao_voxel_terms;

/* As dao_create, with the objective of dao_voxel_terms in place of structures,
 * weights and prescriptions.  Every other call works on the context as on one
 * made by dao_create. */
dao_status dao_create_voxelwise(const dao_csr* D, const dao_geometry* g, const dao_voxel_terms* t,
                                const dao_options* opt, dao_ctx** out);

/* ---- D generated on the device from a pencil-beam model ----
 * The paper obtains D_ij (Eq. 2) from its GPU pencil-beam dose engine
 * (Sec. 1); generating D on the device removes its upload from a re-plan.
 * Model, for beam b of n_beams coplanar beams at gantry angle 2 pi b / n_beams
 * about the z axis (direction (sin, -cos), leaf travel along (cos, sin)), a
 * grid of rows x cols beamlets of pitch beamlet_mm centred on iso, and voxel j
 * at p = voxel_xyz[j] - iso (mm):
 *   D_ij = exp(-mu_per_mm depth_j) L(dv) L(du), du / dv the voxel's offsets
 *   from the beamlet's central axis, depth_j the distance along the beam from
 *   the body's z-invariant cross-section (DAO_BODY_BOX: half-widths
 *   body_size; DAO_BODY_ECYL: semi-axes body_size; centred at body_center) to
 *   the voxel; L(d) = exp(-d^2 / (2 sigma^2)) (DAO_PB_GAUSS) or a strip of
 *   width beamlet_mm blurred by that Gaussian, normalised to 1 on the axis
 *   (DAO_PB_STRIP);
 *   kept when above 1e-12 and at least cutoff times the beamlet's largest
 *   coefficient, then multiplied by 1 + jitter (2 U - 1), U the SplitMix64 draw
 *   of counter j n_beamlets + i in stream jitter_stream (0 jitter: none), and
 *   rounded to FP32.  Beamlet i = b rows cols + r cols + c.
 * FP64 throughout, every product and sum rounded on its own.  The search range
 * of a voxel is the window of beamlets within ceil(sigma sqrt(2 ln 1e7) /
 * beamlet_mm) + 1 of its own (at most 16 per axis, else DAO_EINVAL). */
enum { DAO_PB_GAUSS = 0, DAO_PB_STRIP = 1 };
enum { DAO_BODY_BOX = 0, DAO_BODY_ECYL = 1 };
typedef struct dao_pencil_beam {
    int32_t n_voxels;
    const float* voxel_xyz;      /* host float[n_voxels][3], mm */
    double iso[3];
    int32_t n_beams, rows, cols;  /* 1 <= cols <= 32 */
    double beamlet_mm, sigma_mm, mu_per_mm, cutoff;
    int32_t profile;              /* DAO_PB_* */
    int32_t body_kind;            /* DAO_BODY_* */
    double body_center[2];        /* x, y */
    double body_size[2];
    double jitter;                /* in [0, 1) */
    uint64_t jitter_stream;
} dao_pencil_beam;

/* Generate D on device `device` and copy it to host buffers: voxel-major CSR,
 * columns increasing.  *nnz (host) receives the entry count; row_ptr
 * (int64[n_voxels + 1]), col (int32[*nnz]) and val (float[*nnz]) may be NULL
 * (call once with NULL buffers to learn *nnz, then with buffers of that size:
 * the generation is deterministic).  Device memory is temporary. */
dao_status dao_pencil_generate(const dao_pencil_beam* pb, int32_t device, int64_t* nnz, int64_t* row_ptr,
                               int32_t* col, float* val);

/* As dao_create, with D generated on the context's device from the pencil-beam
 * model instead of a host CSR (n_beams beams of rows x cols beamlets). */
dao_status dao_create_pencil(const dao_pencil_beam* pb, const dao_structures* s, const dao_weights* w,
                             const double* prescriptions, const dao_options* opt, dao_ctx** out);

/* Release a context.  Its device memory goes back to a process-wide
 * stream-ordered pool on its device, which keeps up to min(16 GiB, 1/16 of the
 * device) of freed memory mapped for the contexts created after it; its small
 * page-locked staging block goes to a process-wide free list (at most 64 MiB). */
void dao_destroy(dao_ctx* ctx);

/* Return the cached memory of device `device` to the system: the pool is
 * trimmed to the memory of live contexts and the page-locked free list is
 * emptied.  Safe to call at any time; contexts stay valid. */
dao_status dao_release_cached_memory(int32_t device);

/* Diagnostic of the bounded device waits (no context needed): a cooperative
 * launch of two blocks in which one block never arrives at the grid barrier
 * the persistent master solve uses.  The other block must give up after the
 * barrier's poll limit (seconds at most) and mark the barrier broken.
 * Returns DAO_ETIMEOUT when that happened (the expected outcome; *gave_up and
 * *passed count the blocks of each kind), DAO_ESTATE if the wait did not give
 * up, DAO_ECUDA on a CUDA error.  The device stays usable either way. */
dao_status dao_check_bounded_wait(int32_t device, int32_t* gave_up, int32_t* passed);

/* Empty the aperture pool (y = [], z = 0) keeping D on the device. */
dao_status dao_reset(dao_ctx* ctx);

/* Append n apertures to the pool and solve the master problem once (Sec. 2.3)
 * over the enlarged pool: re-planning from a saved pool (dao_apertures,
 * dao_intensities of an earlier context) on this context's D, or resuming a
 * solve.  beams[n] and leaf_lr[n][2 * max rows] (host; rows past a beam's
 * own count are ignored) as dao_add_aperture takes them; their dose columns
 * come from this context's D.  y_start[n] (host, >= 0, or NULL for zeros)
 * starts the master on the new apertures, the last of them at 0 as for every
 * added aperture; the apertures already in the pool start from their current
 * intensities.  *objective (host, may be NULL) receives F at the master
 * optimum.  Everything is checked before the pool changes (DAO_EINVAL);
 * DAO_ESTATE if the pool would exceed k_max.  n = 0 changes nothing. */
dao_status dao_import_apertures(dao_ctx* ctx, int32_t n, const int32_t* beams, const int32_t* leaf_lr,
                                const double* y_start, double* objective);

/* Pricing sub-problem (Eq. 8, Sec. 2.3) at the current master optimum:
 * pi = grad F(z), w = D^T pi, per-MLC-row minimum-sum consecutive interval,
 * per-beam sum, beam with the smallest sum (lowest index on ties).  Outputs
 * (host): *beam, leaf_lr[2 * rows[*beam]] (caller allocates 2 * max rows),
 * *reduced_cost (FP64 sum of the rows' best values).  Returns DAO_OPTIMAL
 * when the reduced cost is not below -tau, DAO_OK otherwise; the pool is not
 * changed. */
dao_status dao_price(dao_ctx* ctx, int32_t* beam, int32_t* leaf_lr, double* reduced_cost);

/* Add aperture (beam, leaf_lr host) to the pool: its dose column D_kj (Eq. 2)
 * is formed on the device and the master problem is re-solved warm-started
 * (previous intensities, 0 for the new one).  *objective (host, optional)
 * receives F at the new master solution.  DAO_ESTATE when the pool is full,
 * DAO_EINVAL for an invalid aperture. */
dao_status dao_add_aperture(dao_ctx* ctx, int32_t beam, const int32_t* leaf_lr, double* objective);

/* Column generation (Sec. 2.2-2.3, Fig. 1): up to n_apertures rounds of
 * pricing + add + master.  *n_done (host) receives the pool size reached;
 * objective_trace (host, optional, n_apertures entries) receives F after each
 * added aperture.  Returns DAO_OPTIMAL / DAO_DUPLICATE if pricing stopped
 * early, DAO_OK otherwise. */
dao_status dao_solve(dao_ctx* ctx, int32_t n_apertures, int32_t* n_done, double* objective_trace);

/* Beamlet-level fluence map optimisation, min over x >= 0 of F(D x): the model
 * the paper calls mathematically the same as DAO with the beamlets as the
 * decision variables (Sec. 2.2), solved, as the paper solves its FMO, by
 * gradient projection on the GPU (Sec. 2.3).  Its optimum bounds every DAO
 * objective of the same problem from below.  Method: projected Newton with an
 * epsilon-active set, the free beamlets' Newton system solved inexactly by
 * conjugate gradients (each product one dose SpMV and one transposed SpMV on
 * the context's D and D^T, in its storage precision), and an Armijo rule along
 * the projection arc.  Stops when every |x_i - P(x_i - g_i)| is within tol times
 * the largest such residual at x = 0 plus 64 u (D^T |grad F|)_i (u = 2^-24,
 * the FP32 rounding of g_i), or after max_iters Newton steps.  Outputs (host, each optional):
 * x_out double[n_beamlets], *objective = F(D x) (FP64 sum of the FP32 dose
 * epilogue), *iters Newton steps, *cg_iters CG iterations in all.  Returns
 * DAO_OK when the tolerance was met, DAO_ESTATE when the iteration cap or a
 * failed arc search (the FP32 noise floor) stopped it first.  The aperture
 * pool is not changed. */
dao_status dao_fmo(dao_ctx* ctx, int32_t max_iters, double tol, double* x_out, double* objective, int32_t* iters,
                   int32_t* cg_iters);

/* Final dose z = D x with x_i = sum_{k in K_i} y_k (Eqs. 1, 7) computed by the
 * full dose SpMV; dose (host, n_voxels floats, optional), *objective (host,
 * optional) = F(z) of Eq. 5. */
dao_status dao_dose(dao_ctx* ctx, float* dose, double* objective);

/* Current pool: y (host, FP64, capacity k_max), beams (host int32 [K]),
 * leaf_lr (host int32 [K][2 * max rows], row-padded with (0, 0)), *k = K. */
dao_status dao_intensities(dao_ctx* ctx, double* y, int32_t* k);
dao_status dao_apertures(dao_ctx* ctx, int32_t* beams, int32_t* leaf_lr, int32_t* k);

/* Problem sizes: voxels, beamlets, beams, total MLC rows, the widest row
 * count of any beam, stored nnz of D (after row padding), and the pool
 * capacity. */
dao_status dao_sizes(const dao_ctx* ctx, int32_t* n_voxels, int32_t* n_beamlets, int32_t* n_beams,
                     int32_t* n_mlc_rows, int32_t* max_rows, int64_t* nnz_stored, int32_t* k_max);

/* ---- kernel-level entry points (device vectors, for parity tests and the
 * bandwidth benchmark).  All run on the context's stream and read the
 * context's device copy of D / D^T.  Device pointers are caller-owned memory
 * of the context's device holding at least the stated number of elements; the
 * library cannot check either, and a shorter buffer is read or written out of
 * bounds. ---- */

/* Step a1: z = D x (device float[n_beamlets] -> float[n_voxels]) with the
 * objective epilogue: grad (device, optional) = grad F(z) (Sec. 2.3's pi) and
 * *objective (host, optional) = F(z) in FP64 (Eqs. 5, 9, 10). */
dao_status dao_k_dose(dao_ctx* ctx, const float* x, float* z, float* grad, double* objective);

/* Step a2: w = D^T pi (device float[n_voxels] -> float[n_beamlets]), the
 * bracketed sum of Eq. 8, from the stored transpose (no atomics). */
dao_status dao_k_beamlet_prices(dao_ctx* ctx, const float* pi, float* w);

/* Step a3: pricing on a given w (device float[n_beamlets]); outputs as
 * dao_price plus, when non-NULL, row_best (host double[n_mlc_rows]: each
 * row's best interval sum v*) and row_lr (host int32[2 * n_mlc_rows]). */
dao_status dao_k_price(dao_ctx* ctx, const float* w, int32_t* beam, int32_t* leaf_lr,
                       double* reduced_cost, double* row_best, int32_t* row_lr);

/* Step a4: column D_kj = sum_{i in A_k} D_ij (Eq. 2) of aperture
 * (beam, leaf_lr host) into out (device float[n_voxels]). */
dao_status dao_k_aperture_column(dao_ctx* ctx, int32_t beam, const int32_t* leaf_lr, float* out);

/* Current pi = grad F(z) and z of the last master solution (device outputs,
 * float[n_voxels] each). */
dao_status dao_k_state(dao_ctx* ctx, float* z, float* pi);

/* Average device time in microseconds (*us_per_launch, host) of `reps`
 * back-to-back launches of one kernel class on the context's current data,
 * between two CUDA events on the context's stream: DAO_KC_MASTER_PASS (the
 * slab pass at pool size K, 1 <= K <= current pool size), DAO_KC_MASTER_HESS
 * (the curvature kernel on the last pass's active voxels), DAO_KC_DT,
 * DAO_KC_DOSE, DAO_KC_COLUMN (first aperture of the pool), DAO_KC_PRICE.
 * Results and the pool are unchanged; scratch buffers are overwritten. */
dao_status dao_k_time(dao_ctx* ctx, int32_t kc, int32_t K, int32_t reps, double* us_per_launch);
/* Cold-cache device time of one launch of DAO_KC_DOSE, DAO_KC_DT or
 * DAO_KC_PRICE: `reps` (1..1024) repetitions of [read all flush_bytes of the
 * caller's device buffer `flush` (make it larger than L2; reading leaves only
 * clean lines, so no write-back overlaps the kernel), event, launch, event]
 * captured into one CUDA graph and replayed once; *us_median (host) receives
 * the median in microseconds.  K is ignored.  Synchronises. */
dao_status dao_k_time_cold(dao_ctx* ctx, int32_t kc, int32_t K, int32_t reps, void* flush, int64_t flush_bytes,
                           double* us_median);

/* ---- instrumentation: per-kernel-class CUDA-event timing on the context's
 * stream (off by default).  While it is on, dao_solve uses host-driven
 * launches so that every kernel can be bracketed by events. ---- */
enum {
    DAO_KC_DOSE = 0,           /* a1 dose SpMV + epilogue */
    DAO_KC_DT = 1,             /* a2 transposed SpMV */
    DAO_KC_PRICE = 2,          /* a3 pricing (row scan + beam reduction) */
    DAO_KC_COLUMN = 3,         /* a4 aperture column */
    DAO_KC_MASTER_PASS = 4,    /* a5 slab pass: z, pi, h, F and the active-voxel list */
    DAO_KC_MASTER_REDUCE = 5,  /* a5 partial reduction: now part of DAO_KC_MASTER_STEP, never counted */
    DAO_KC_MASTER_STEP = 6,    /* a5 partial reduction + Newton step / line search control */
    DAO_KC_MASTER_HESS = 7,    /* a5 curvature matrix and gradient over the active voxels */
    DAO_KC_OTHER = 8,
    DAO_KC_MASTER_SOLVE = 9,   /* a5 the whole master solve as one persistent kernel */
    DAO_KC_COUNT = 10
};
dao_status dao_profile_enable(dao_ctx* ctx, int32_t enable);
/* launches, summed device milliseconds and the kernel launches counted for
 * class kc since the last dao_profile_enable(ctx, 1); synchronises. */
dao_status dao_profile_read(dao_ctx* ctx, int32_t kc, int64_t* launches, double* total_ms);
/* Every kernel launched by this context since creation (all classes). */
int64_t dao_launch_count(const dao_ctx* ctx);

/* Per master solve since the last reset, in pool order (host arrays of k_max
 * entries, each optional): evals = fused slab passes evaluated, status = 1
 * converged / 2 iteration cap / 3 line search stalled, kkt = final
 * ||y - P(y - g)||_inf divided by max|g| at the warm start; *k = solves. */
dao_status dao_master_stats(const dao_ctx* ctx, int32_t* evals, int32_t* status, double* kkt, int32_t* k);

/* ---- batched plans (many instances at once) ----
 * Column generation (Sec. 2.3, Fig. 1) for n independent contexts in one call:
 * the same work as dao_solve(ctxs[i], n_apertures, ...) for every i, with every
 * context's rounds run as its own CUDA graphs on its own stream and launched
 * round-interleaved, so that the GPU overlaps the instances' small kernels.
 * The instances share no device state: each one's apertures, intensities,
 * objective trace and dose are bitwise those of solving it alone.
 *   ctxs: n distinct contexts on one device, created with use_graphs and with
 *         profiling off; contexts that share a stream run one after another;
 *   n_done: int32[n] or NULL, each instance's pool size afterwards;
 *   traces: double[n][n_apertures] or NULL, each instance's objective after
 *         each aperture it added (as dao_solve's trace);
 *   status: int32[n] or NULL, each instance's dao_solve status (DAO_OK,
 *         DAO_OPTIMAL, DAO_DUPLICATE, or DAO_ESTATE for a full pool).
 * Returns DAO_EINVAL for invalid arguments (nothing runs), DAO_ECUDA on a CUDA
 * error, else DAO_OK with the per-instance outcome in status.  Synchronous. */
dao_status dao_batch_solve(dao_ctx* const* ctxs, int32_t n, int32_t n_apertures, int32_t* n_done, double* traces,
                           int32_t* status);

/* Column generation for n independent contexts with one persistent master
 * launch per round for all of them: the plans' master solves run side by side
 * in one cooperative kernel, each on its own group of blocks (two blocks per SM
 * shared out evenly; each group with its own grid barrier, solver state and
 * stopping), while every plan's D^T kernel and beam decision with the new
 * column run on its own stream before it.  The rounds are captured once into
 * a CUDA graph for the list of contexts and the round count, kept for the
 * next call with the same list (at most four such graphs; a graph goes with
 * its contexts' dao_destroy).  Arguments and results as dao_batch_solve; a
 * plan's results are those of solving it alone with a persistent master of
 * the same group size.  DAO_EINVAL when two blocks per SM do not give every
 * plan a block (n > 2 x SMs).  Synchronous. */
dao_status dao_batch_solve_persistent(dao_ctx* const* ctxs, int32_t n, int32_t n_apertures, int32_t* n_done,
                                      double* traces, int32_t* status);

/* Blocks per plan of dao_batch_solve_persistent for n plans on device `device` (0 when n plans do not fit one launch): a plan
 * created with this master_blocks solves alone exactly as it does in the
 * batch. */
int32_t dao_batch_group_size(int32_t n, int32_t device);

/* ---- autotuner of the SpMV launch shapes ----
 * Times the dose SpMV (a1: the lane form with 4/8/16/32 lanes per voxel row,
 * 16-bit storage up to 16, and the unit form), the transposed SpMV (a2, threads
 * per beamlet row: 64/128/256, each with both lane mappings, and the split
 * form) and the
 * aperture column (a4: D by beams, or 1/2/4/8/16 lanes per voxel row over D) on the context's own
 * matrices (10 launches per candidate, each after a read of a buffer twice the
 * L2 size, so that it runs on a cold cache as in a plan; median of the
 * per-launch event times) and keeps the fastest of each for this context.
 * Needs 2 x L2 bytes of device memory for the duration of the call.  cache_path (or
 * NULL): a text file of "key dose column dt form map" lines, key = device name,
 * precision and the log2 size class of voxels, beamlets and the mean row
 * lengths of D and D^T; a matching entry is applied without timing, a new
 * choice is appended.  out (or NULL) receives the choice and whether it came
 * from the cache.  Cached round graphs are rebuilt on the next solve.  Results
 * are unchanged up to the FP32 summation order of the SpMVs. */
typedef struct {
    int32_t dose_lanes;    /* a1 lanes per voxel row (lane form) */
    int32_t column_lanes;  /* a4: 0 D by beams, else lanes per voxel row over D */
    int32_t dt_threads;    /* a2 threads per beamlet row */
    int32_t from_cache;    /* 1 when read from cache_path, 0 when timed */
    int32_t dose_form;     /* a1 form: DAO_DOSE_LANES, DAO_DOSE_UNITS or DAO_DOSE_MERGE */
    int32_t dt_map;        /* a2 form: DAO_DT_GROUPED, DAO_DT_CONSECUTIVE or DAO_DT_SPLIT */
} dao_tuning;
dao_status dao_autotune(dao_ctx* ctx, const char* cache_path, dao_tuning* out);

/* The SpMV forms and launch shapes the context's kernels run with now (after
 * options, the autotuner's choice and the fallbacks: the unit form of a1 where
 * its shared memory fits, the split form of a2 where every row of D^T has at
 * least 32 entries); dt_threads is 0 for the split form; from_cache is 0.
 * Host only, no CUDA call. */
dao_status dao_kernel_forms(const dao_ctx* ctx, dao_tuning* out);

/* ---- re-plan serving (continuous batching) ----
 * A server plans requests as they arrive (the paper's motivation: re-planning
 * fast enough to adapt a treatment to the day's anatomy, Sec. 1 and Sec. 4).
 * One host worker thread admits queued requests in arrival order while a slot
 * is free and the request's device footprint fits (free device memory minus
 * hbm_reserve_bytes, or the hbm_budget_bytes budget minus the footprints of the
 * running plans); an admitted request gets its own context and stream, all its
 * column-generation rounds are queued as CUDA graphs at once, and it runs
 * alongside the plans already on the GPU; the worker retires each plan as soon
 * as its last round completes, copies the results into the request's output
 * buffers and admits the next request, without waiting for the other plans.
 * A request that can never fit is rejected (DAO_ENOMEM) instead of blocking the
 * queue; an invalid one fails with dao_create's status.
 * Simulation (simulate_ms_per_aperture > 0): a host-only stand-in for the GPU
 * used to test the scheduler; no CUDA call is made, no plan is computed, a
 * request "runs" for simulate_ms_per_aperture * n_apertures milliseconds and
 * reports status DAO_OK, n_apertures apertures and a NaN objective; free
 * memory is hbm_budget_bytes, which must then be > 0. */
typedef struct dao_server dao_server;
typedef struct {
    int32_t max_slots;             /* plans on the GPU at once (>= 1) */
    int32_t queue_capacity;        /* queued requests beyond which submit returns DAO_EBUSY (>= 1) */
    int64_t hbm_reserve_bytes;     /* device memory left free when admitting */
    int64_t hbm_budget_bytes;      /* 0: admit by free device memory; > 0: admit while the
                                      footprints of the running plans stay within it */
    int32_t device;
    double simulate_ms_per_aperture;
    dao_options plan_options;      /* options of every plan; stream and device are ignored */
    int64_t prewarm_bytes;         /* device memory taken into the library's memory pool, and page-locked
                                      staging blocks for max_slots + 2 plans, when the server starts, so that
                                      admitted plans do not wait for the pool to grow or for host pages to be
                                      locked (default 2 GiB; 0: none) */
    int32_t solve_slots;           /* plans whose column-generation rounds are on the GPU at once: 0 (default)
                                      as many as max_slots; n > 0: admitted requests create their contexts
                                      (upload, checks, device build) alongside the running plans, then queue
                                      their rounds in admission order, at most n plans' rounds at a time */
} dao_server_options;
void dao_server_options_default(dao_server_options* opt);

/* One request: dao_create's arguments, the apertures to add, and caller-owned
 * output buffers (each may be NULL).  Every array, input or output, must stay
 * valid until dao_server_poll or dao_server_wait has reported the request. */
typedef struct {
    dao_csr D;
    dao_geometry geometry;
    dao_structures structures;
    dao_weights weights;
    const double* prescriptions;
    int32_t n_apertures;
    float* dose_out;               /* [n_voxels] planned dose */
    double* intensities_out;       /* [plan_options.k_max] y */
    int32_t* beams_out;            /* [plan_options.k_max] aperture beams */
    int32_t* leaves_out;           /* [plan_options.k_max][2 * max rows] half-open [L, R) per row */
} dao_request;

typedef struct {
    int32_t status;        /* dao_solve's status, or the error that stopped the request */
    int32_t n_apertures;   /* apertures in the plan */
    double objective;      /* F of the final plan (Eqs. 9-10) */
    double queue_ms;       /* submission to admission */
    double run_ms;         /* admission to results in the output buffers */
    double latency_ms;     /* submission to results */
    double create_ms;      /* of run_ms: the plan's context created (upload, checks, device build) */
    double solve_ms;       /* of run_ms: rounds queued until the worker saw them complete */
    double finish_ms;      /* of run_ms: results copied out and the context released */
    double gpu_wait_ms;    /* of run_ms: created, waiting for its turn to queue its rounds (solve_slots) */
    char error[256];       /* message of a failed request */
} dao_result;

typedef struct {
    int64_t submitted, completed, failed, rejected;
    int32_t active, queued, max_active;
    int64_t bytes_in_use;  /* footprints of the running plans */
} dao_server_stats;

dao_status dao_server_create(const dao_server_options* opt, dao_server** out);
/* Queues a request (DAO_EBUSY when the queue is full, DAO_ESTATE after
 * shutdown); *id identifies it. */
dao_status dao_server_submit(dao_server* srv, const dao_request* req, int64_t* id);
/* DAO_OK and *out once the request has finished (each id is reported once),
 * DAO_EBUSY while it is queued or running, DAO_EINVAL for an unknown id. */
dao_status dao_server_poll(dao_server* srv, int64_t id, dao_result* out);
/* As poll, blocking up to timeout_ms (< 0: no limit); DAO_ETIMEOUT if it ran out. */
dao_status dao_server_wait(dao_server* srv, int64_t id, double timeout_ms, dao_result* out);
dao_status dao_server_stats_get(dao_server* srv, dao_server_stats* out);
/* Device bytes a request's plan holds at its peak, the temporaries of its
 * device build included: the admission footprint. */
int64_t dao_server_footprint(const dao_request* req, const dao_options* plan_options);
/* Cancels queued requests (status DAO_ESTATE), waits for the running plans,
 * stops the worker and frees the server. */
void dao_server_destroy(dao_server* srv);

/* ---- allocation-free dose with objective (the paper has no counterpart) ----
 * For callers that must not allocate device memory while they run, e.g. a
 * re-planning service that reserves every device buffer before an online
 * adaptive fraction (so that the fraction cannot fail on an allocation or stall
 * on the synchronisation cudaMalloc / cudaFree may imply), or an application
 * whose own allocator owns the device.  Without a context and without
 * allocating (no cudaMalloc, cudaFree or allocating library routine) it
 * computes the dose z = D x of a fluence x, the derivative of the objective
 * with respect to each voxel's dose, and the objective itself, for one-sided
 * quadratic voxel penalties: a voxel of structure s contributes
 * a_s max(0, t_s - z)^2 + b_s max(0, z - u_s)^2, with the weights and
 * thresholds given per structure in `terms`.  It is what dao_k_dose computes
 * for a context, in a standalone form.
 *   D: voxel-major CSR on the device, int32 row_ptr[n_voxels + 1], col[nnz],
 *      float val[nnz] (rows need no padding), columns in [0, n_beamlets);
 *      x: device float[n_beamlets];
 *   voxel_struct: device int32[n_voxels], labels in [0, n_structures); a voxel
 *      with a label outside that range gets a NaN derivative and makes the
 *      objective NaN (its dose is still written);
 *   terms: host double[n_structures][4] = a_s, t_s, b_s, u_s;
 *   z: device float[n_voxels]; grad: device float[n_voxels] or NULL (then only
 *      z and the objective are computed);
 *   objective: device double; stream: cudaStream_t or NULL (legacy stream).
 * Every device buffer and the stream must belong to the CUDA device that is
 * current on the calling thread: the kernels run there.  A stream of another
 * device is refused (DAO_EINVAL); buffers cannot be checked, and buffers of
 * another device, or shorter than stated, or column indices outside
 * [0, n_beamlets), are read or written out of bounds.
 * Limits: n_voxels <= 4,194,304 and n_structures <= 64, else DAO_EINVAL with a
 * message.  Scratch: the per-block partial sums of the objective live in a
 * 32 KiB file-scope device array that every GPU loading the library keeps until
 * the process exits; every block overwrites its own entry on each call, so
 * nothing needs clearing, and the array keeps the last call's contents.  All
 * calls on a device share that array: calls whose kernels overlap on the GPU
 * (for example on different streams) race and give wrong objectives.  The
 * first call on a device looks up the array's device address with that device
 * current and keeps it for the life of the process; make that first call
 * before any stream capture, and do not call this entry point again after a
 * cudaDeviceReset of that device.  Asynchronous: results are ready when the
 * stream reaches them. */
dao_status dao_dose_objective_noalloc(int32_t n_voxels, int32_t n_beamlets, const int32_t* row_ptr,
                                      const int32_t* col, const float* val, const float* x,
                                      const int32_t* voxel_struct, int32_t n_structures, const double* terms,
                                      float* z, float* grad, double* objective, void* stream);

const char* dao_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DAO_H */
