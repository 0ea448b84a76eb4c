// Internal declarations shared by the libdao.so translation units.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dao.h"

namespace dao {

// Record the calling thread's error message for dao_last_error(); returns s.
dao_status set_error(dao_status s, const std::string& msg);

// Host-only validation of dao_create's arguments (no CUDA call).
dao_status check_inputs(const dao_csr* D, const dao_geometry* g, const dao_structures* s, const dao_weights* w,
                        const double* rx, const dao_options* opt);
// Graph path without waiting: launch up to n_apertures rounds on the context's
// stream and record `done` after them; solve_async_end reads the outcome back
// once `done` has completed.
dao_status solve_async_begin(dao_ctx* c, int n_apertures, cudaEvent_t done);
dao_status solve_async_end(dao_ctx* c, int n_apertures, int32_t* n_done, dao_status* result);

constexpr int KMAX = 64;        // aperture pool capacity (master problem size)
constexpr int SMAX = 64;        // structures
constexpr int CMAX = 32;        // beamlets per MLC row (one warp lane each)
constexpr int MASTER_TILE = 256;  // voxels per tile of the master evaluation (= block size)
constexpr int KROW = KMAX + 4;    // row stride (floats) of the active-voxel rows (odd float4 count)

// Per-structure objective terms (Eqs. 9-10): a = alpha_s/|v_s| (0 for
// non-targets), tu = T_s^-, b = beta_s/|v_s|, to = T_s^+.
struct StructTermsF { float a, tu, b, to; };
struct StructTermsD { double a, tu, b, to; };
// FP32 terms of the dose epilogue with each threshold split into hi + lo floats,
// so that T - z is exact near the threshold.
struct StructTermsS { float a, tu_hi, tu_lo, b, to_hi, to_lo, pad0, pad1; };

// Every kernel that reads objective terms takes (labels, terms, S): with S >= 0
// voxel j's terms are terms[labels[j]] (S structures, staged in shared
// memory); with S < 0 (per-voxel weights and thresholds, the re-optimisation
// form of Eqs. 3-4) they are terms[j] and the labels are not read.
__device__ __forceinline__ StructTermsF voxel_terms(const StructTermsF* __restrict__ tf, int j) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(tf) + j);
    return StructTermsF{v.x, v.y, v.z, v.w};
}

// Device copy of a CSR matrix whose rows are padded to a multiple of four
// entries (padding: value 0, column = the row's last real column), so every
// row starts on a 16-byte boundary for int4/float4 loads.
struct DevCSR {
    int n_rows = 0;
    int n_cols = 0;
    int64_t nnz_stored = 0;
    int prec = 0;            // DAO_PREC_FP32 / FP16 / BF16
    int* rowptr = nullptr;   // n_rows + 1; multiples of 4 (FP32) or 8 (16-bit values)
    int* col = nullptr;      // FP32 layout, and the voxel indices of a 16-bit D^T
    float* val = nullptr;    // FP32 values
    unsigned short* col16 = nullptr;  // 16-bit layout of D: beamlet indices
    unsigned short* val16 = nullptr;  // 16-bit values D_ij / s_i (FP16 or BF16 bits)
    const float* scale = nullptr;     // 16-bit layout: per-beamlet scale s_i (length n_beamlets)
    const int* order = nullptr;       // D^T: rows by decreasing length (block b takes row order[b])
    // launch shape chosen by the autotuner (0: built-in rule): lanes per row of the
    // dose SpMV and of the aperture column (D), threads per row of the transposed
    // SpMV (D^T)
    int tune_dose_g = 0;
    int tune_col_g = 0;
    int tune_dt_threads = 0;
    // form of the dose SpMV (DOSE_FORM_*) and lane mapping of the transposed
    // SpMV (DT_MAP_*); 0: the built-in rule
    int tune_dose_form = 0;
    int tune_dt_map = 0;
    // D: the most groups (8 entries of 16-bit storage, 4 of FP32) in one unit of
    // 32 consecutive rows; sizes the unit form's shared partials (0: not known)
    int unit_groups_max = 0;
    // D^T split over warps by entries (DT_MAP_SPLIT, rows of at least 32
    // entries): warp v takes entries [v chunk, (v + 1) chunk), split_row[v] is
    // the row holding its first entry; a row covered by several warps adds their
    // partial sums (split_part, split_ps slots per row) in warp order, on a
    // per-row ticket (split_cnt, zero between launches)
    // D by beams (the aperture column's layout): beam b's part of row j is
    // entries [beam_rowptr[b (V + 1) + j], beam_rowptr[b (V + 1) + j + 1]) of
    // beam_col (beamlet index within the beam) and beam_val32 (FP32) or
    // beam_val16 (16-bit values, as in D); nullptr: not built
    int* beam_rowptr = nullptr;
    unsigned short* beam_col = nullptr;
    float* beam_val32 = nullptr;
    unsigned short* beam_val16 = nullptr;
    // D split over warps along the merge path of its groups and row ends
    // (DOSE_FORM_MERGE): warp v takes the stretch between merge_path[v] and
    // merge_path[v + 1] (rows finished, groups consumed), merge_chunk items,
    // more than the longest row; a row crossing the boundary before warp v is
    // finished from merge_slot[2v], merge_slot[2v + 1] on the ticket
    // merge_cnt[v] (zero between launches)
    int merge_chunk = 0;     // items per warp (its most groups); 0: the merge form is not available
    int merge_warps = 0;
    const int2* merge_path = nullptr;
    float* merge_slot = nullptr;
    int* merge_cnt = nullptr;
    int split_chunk = 0;     // 0: the split form is not available
    int split_warps = 0;
    int split_ps = 0;
    const int* split_row = nullptr;
    float* split_part = nullptr;
    int* split_cnt = nullptr;
};

// Forms of the dose SpMV (a1): G lanes per voxel row over the row's groups,
// or one warp per unit of 32 rows (the default where its shared memory fits).
enum { DOSE_FORM_LANES = DAO_DOSE_LANES, DOSE_FORM_UNITS = DAO_DOSE_UNITS, DOSE_FORM_MERGE = DAO_DOSE_MERGE };
// Warps of the merge form of a1 per SM (blocks of 8 warps), and its most
// groups per warp.
constexpr int MERGE_WARPS_PER_SM = 32;
constexpr int MERGE_CHUNK_MAX = 1024;
// Lane mappings of the transposed SpMV (a2): a thread per group of 4 or 8
// consecutive entries, or consecutive entries on consecutive threads (default).
enum { DT_MAP_GROUPED = DAO_DT_GROUPED, DT_MAP_CONSECUTIVE = DAO_DT_CONSECUTIVE, DT_MAP_SPLIT = DAO_DT_SPLIT };
// Warps of the split form of a2 per SM (blocks of 8 warps).
constexpr int SPLIT_WARPS_PER_SM = 32;

// Launch shapes the autotuner may choose from.
constexpr int TUNE_DOSE_G[] = {4, 8, 16, 32};
constexpr int TUNE_COL_G[] = {0, 1, 2, 4, 8, 16};  // 0: D by beams, one lane per voxel row
constexpr int TUNE_DT_THREADS[] = {64, 128, 256};

// Projected-Newton master state (device memory, one per context).
struct MasterDev {
    double y[KMAX];       // accepted intensities
    double yt[KMAX];      // trial point evaluated by the next fused pass
    double d[KMAX];       // search direction
    double g[KMAX];       // gradient at y
    double gt[KMAX];      // gradient at the trial point (written by the reduction)
    float Ht[KMAX * KMAX];   // curvature matrix at the trial point (full, symmetric; FP64 sums
                             // rounded once to FP32, the precision of the factorisation)
    float gn[KMAX];       // sum_j |S_jk pi_j| at the trial point: the rounding scale of g_k
    double F;             // objective at y
    double Ft;            // objective at the trial point
    double alpha;         // step length along d
    double tol;           // absolute KKT tolerance of this solve
    double res;           // KKT residual at y
    int K;                // pool size
    int iter;             // Newton iterations taken
    int phase;            // 0: evaluating the warm start, 1: line search
    int done;             // 1 once converged / stalled / out of iterations
    int status;           // MASTER_*
    int n_eval;           // fused passes evaluated
    int err;              // set when a tile copy of an evaluation never completed
    unsigned ticket;      // blocks of the reduce + step kernel that finished their share (0 between launches)
    int final_pending;    // the solve stopped at an accepted point other than the last one evaluated
    int inc_G;            // persistent solve: group size whose kept partial H and voxel states are valid (0: none)
    int inc_K;            // the pool size they were kept at
};

enum { MASTER_RUNNING = 0, MASTER_CONVERGED = 1, MASTER_MAXITER = 2, MASTER_STALLED = 3, MASTER_ERROR = 4 };

// Result of the device-side pricing (step a3).
struct PriceDev {
    double rc;            // reduced cost of the best beam
    int beam;             // b*
    int pad;
};

// Device-side column-generation state of a graph-driven solve.
struct CGDev {
    int K;                // pool size reached
    int done;             // 0 running, 1 no negative reduced cost, 2 duplicate aperture
    int K_end;            // a device-driven solve stops when the pool reaches this size
    int stop;             // done set or K_end reached: later rounds skip D^T and pricing
    int idle;             // this round added no aperture: its column and master solve skip
    int rs_K;             // K and stop as the round's D^T kernel found them: the fused
    int rs_stop;          //   commit kernel reads these while its block 0 updates K and stop
    int pad;
    double trace[KMAX];   // F after each added aperture
    double res[KMAX];     // final KKT residual of each master solve
    double tol[KMAX];     // its absolute tolerance
    int evals[KMAX];      // fused passes of each master solve
    int status[KMAX];     // MASTER_* of each master solve
};

// ---- kernel launchers (all on `stream`; return the launch error) ----------

// a1: z = D x, optional grad F(z), FP64 F partials (one per block) reduced into *F_out.
cudaError_t launch_dose(const DevCSR& D, const float* x, const uint8_t* vstruct,
                        const StructTermsF* tf, const StructTermsS* ts, int S,
                        float* z, float* grad, double* F_part, int F_blocks, double* F_out,
                        int num_sms, cudaStream_t stream, int* launches);
int dose_grid(int n_rows, int num_sms);
// The unit form of a1 fits shared memory for this matrix.
bool dose_units_available(const DevCSR& D);
// The form of a1 a launch takes (DOSE_FORM_*), and the objective partial
// slots the merge form writes (0 when it is not available).
int dose_form_effective(const DevCSR& D);
int dose_merge_f_slots(const DevCSR& D);
// Process-wide dynamic shared-memory limits of the SpMV kernels (set once per
// device, to a fixed size).
cudaError_t spmv_configure();

// a2: w = D^T pi over the beamlet-major transpose (skipped when *skip != 0).
cudaError_t launch_dt(const DevCSR& Dt, const float* pi, float* w, const int* skip, cudaStream_t stream,
                      int* launches);

// a4: out[j * stride] = sum over beam b's entries of row j with mask[col - base] (0/1);
// seg: the (B + 1) x V beam segments of D's rows.
cudaError_t launch_column(const DevCSR& D, const int* seg, int b, int base, int n_beamlets_b, const float* mask,
                          float* out, int stride, int num_sms, cudaStream_t stream, int* launches);

// a4 for the aperture the device just committed at pool index K-1 (graph
// path), written to column K-1 of the slab (column stride ld).
cudaError_t launch_column_dev(const DevCSR& D, const int* seg, const int* ap_beam, int K, const int* beam_off,
                              const int* rows, const int* cols, int max_nb, const float* mask, float* slab, int ld,
                              const CGDev* cg, int num_sms, cudaStream_t stream, int* launches);

// x_i = sum_{k in K_i} y_k (Eq. 7) from the aperture table.
cudaError_t launch_fluence(const int* ap_beam, const int* ap_lr, int lr_stride, const double* y, int K,
                           const int4* beamlet_info, int N, float* x, cudaStream_t stream, int* launches);

// a3: per-row scan (one warp per MLC row) and the per-beam sum / argmin.
cudaError_t launch_price(const float* w, const int4* row_info, int n_rows, const int* beam_row0,
                         int n_beams, double* row_v, int2* row_lr, PriceDev* out, const int* skip,
                         cudaStream_t stream, int* launches);
// Graph path: stop the solve when the reduced cost is not below -tau or the
// aperture repeats one in the pool; otherwise record it as aperture K-1 and
// write its open-beamlet mask.
// Graph path: the row scans, then the beam argmin fused with the commit.
cudaError_t launch_price_rows(const float* w, const int4* row_info, int n_rows, double* row_v, int2* row_lr,
                              const int* skip, cudaStream_t stream, int* launches);
// Sets cg->idle (0 when it added aperture K - 1) and cg->stop (done, or the
// pool reached cg->K_end).
cudaError_t launch_price_commit(const double* row_v, const int* beam_row0, int n_beams, PriceDev* pr,
                                const int2* row_lr, const int* rows, const int* cols, double tau, int K, int lr_stride,
                                int* ap_beam, int* ap_lr, float* mask, CGDev* cg, cudaStream_t stream, int* launches);

// Only the per-beam sums of row_v and their argmin (k_price_beams).
cudaError_t launch_price_beams(const double* row_v, const int* beam_row0, int n_beams, PriceDev* out,
                               const int* skip, cudaStream_t stream, int* launches);
// a3 under an MLC constraint (mlc.cu): one block per beam writes row_v (the
// beam's value at its first row, 0 at the others) and row_lr; smem bytes from
// mlc_smem_bytes for the largest beam, after mlc_configure with that size.
size_t mlc_smem_bytes(int mode, int max_rows, int max_cols);
cudaError_t mlc_configure(int mode, size_t smem);
cudaError_t launch_price_mlc(int mode, const float* w, const int* beam_off, const int* rows, const int* cols,
                             const int* beam_row0, int n_beams, size_t smem, double* row_v, int2* row_lr,
                             const int* skip, cudaStream_t stream, int* launches);

// Beamlet-level FMO (fmo.cu): the scalars that steer the host loop and the
// one-block vector kernels on the N beamlets (FP64 values).
struct FmoScalars {
    double res;       // KKT residual ||x - P(x - g)||_inf of the current x
    double res_x;     // its part beyond the FP32 rounding of g (the stopping test)
    double rr;        // r^T r of the current CG iterate
    double bb;        // g_F^T g_F (the CG right-hand side's norm squared)
    double eta;       // CG forcing term
    double gdx;       // g^T (x_trial - x)
    int cg_done;      // the CG of this Newton step has stopped
    int cg_iters;     // CG iterations of this Newton step
};
cudaError_t fmo_kkt(int N, const double* x, const float* g, const float* gn, FmoScalars* st, cudaStream_t s);
cudaError_t fmo_abs(int V, const float* pi, float* out, int num_sms, cudaStream_t s);
cudaError_t fmo_cg_init(int N, const double* x, const float* g, double eps, double eta, unsigned char* free_,
                        double* r, double* p, float* p32, double* dF, FmoScalars* st, cudaStream_t s);
cudaError_t fmo_hmul(int V, const float* z, float* u, const uint8_t* vstruct, const StructTermsF* tf, int S,
                     int num_sms, cudaStream_t s);
cudaError_t fmo_cg_step(int N, const float* Ap, const unsigned char* free_, double* r, double* p, float* p32,
                        double* dF, FmoScalars* st, cudaStream_t s);
cudaError_t fmo_trial(int N, const double* x, const float* g, const unsigned char* free_, const double* dF, double a,
                      double* xt, float* xt32, FmoScalars* st, cudaStream_t s);

// D from the pencil-beam model on the device (pencil.cu): argument checks, and
// the voxel-major CSR (int64 row offsets, int32 columns, FP32 values) in
// stream-ordered pool memory that the caller frees with pool_free.
dao_status pencil_check(const dao_pencil_beam* pb);
cudaError_t pencil_generate(const dao_pencil_beam* pb, int device, cudaStream_t s, int64_t** rp, int** col,
                            float** val, int64_t* nnz);

// The device-driven round (one graph for every round of a solve):
//  - D^T with the MLC-row search fused: the block that completes the last
//    beamlet of an MLC row (a per-row ticket) runs that row's search; block 0
//    snapshots cg->K and cg->stop into rs_K and rs_stop;
//  - the beam decision fused with the new aperture's column: every block takes
//    the same decision from the row results, block 0 commits aperture
//    rs_K (pool size rs_K + 1), writes cg->K, idle, stop, done and the
//    while-node handle (!stop), and every block computes its share of the
//    column into the slab.
struct RowTicket {
    const int4* binfo;      // per beamlet: beam, MLC row within the beam, column
    const int* beam_row0;   // first global MLC row of each beam
    const int* cols;        // beamlets per MLC row of each beam
    const int4* row_info;   // per MLC row: beam, first beamlet, columns, row
    int* row_cnt;           // per MLC row: beamlets done this round (the row's last block resets it)
    double* row_v;
    int2* row_lr;
    CGDev* cg;
};
cudaError_t launch_dt_rows(const DevCSR& Dt, const float* pi, float* w, const RowTicket& rt, cudaStream_t stream,
                           int* launches);
struct CommitArgs {
    const double* row_v;
    const int2* row_lr;
    const int* beam_row0;
    const int* rows;
    const int* cols;
    const int* beam_off;
    const int* seg;         // (B + 1) x V beam segments of D's rows
    int n_beams;
    int lr_stride;
    double tau;
    int* ap_beam;
    int* ap_lr;
    float* slab;
    int ld;
    CGDev* cg;
    cudaGraphConditionalHandle cond;
    int use_cond;           // 0: no conditional node around the kernel (cond unused)
};
cudaError_t launch_commit_column(const DevCSR& D, const CommitArgs& ca, int max_nb, int num_sms, cudaStream_t stream,
                                 int* launches);

// a5: projected-Newton master problem kernels.
// Counters of the grid barrier of the persistent master solve (zeroed memory;
// count returns to 0 after every barrier, gen only increases).
// Device-scope acquire-release atomic add and acquire load.  After a
// __syncthreads(), thread 0's release covers the writes of every thread of
// its block (PTX causality order runs through bar.sync); after thread 0's
// acquire and a __syncthreads(), every thread of the block sees what was
// released to it.  This is the pattern of the grid barrier and of the
// last-block tickets; it replaces a full fence (fence.sc) per thread before
// the atomic and after it.
__device__ __forceinline__ unsigned atom_add_acq_rel_gpu(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of the persistent master solve: a monotonic arrival counter
// (zeroed by the host before each solve) and a flag a block sets when a wait
// ran out, after which the solve's later launches return at entry.
struct GridBar {
    unsigned count;
    unsigned broken;
    unsigned pad[2];
};

struct MasterBuffers {
    MasterDev* st = nullptr;
    float* act_rows = nullptr;  // [n_tiles * MASTER_TILE][KROW]: rows of the active voxels, per tile slot
    float2* act_hp = nullptr;   // [n_tiles * MASTER_TILE]: their curvature and gradient
    int* act_count = nullptr;   // [n_tiles]
    int n_tiles = 0;
    float* H_part = nullptr;    // [KMAX*(KMAX+1)/2][GH]
    double* g_part = nullptr;   // [KMAX][GH]
    float* gn_part = nullptr;   // [KMAX][GH]
    double* F_part = nullptr;   // [max evaluation grid]
    int GH = 0;                 // blocks of the curvature kernel
    GridBar* bar = nullptr;     // grid barrier of the persistent solve
    int GP = 0;                 // blocks of the persistent solve (co-resident), 0: not available
    int grid[KMAX + 1] = {};    // blocks of the evaluation kernel for each pool size
    CUtensorMap tmap[KMAX / 4 + 1];  // slab tile maps, indexed by columns / 4
    CUtensorMap tmap_p[2];           // slab maps of the persistent solve: boxes of 128 voxels x 16, x 4 columns
    uint8_t* vstate = nullptr;       // [V] persistent solve: each voxel's curvature state at the last evaluation
    float* H_keep = nullptr;         // [GH][KMAX*(KMAX+1)/2] persistent solve: each block's kept partial H
};
enum { PASS_EVAL = 0, PASS_FINAL = 1, PASS_TIMING = 2 };
__host__ __device__ int master_kw(int K);
__host__ __device__ int master_lanes(int K);
__host__ __device__ int persist_lanes(int K);
int master_grid(int V, int num_sms, int K);
int master_grid_max(int num_sms);
int master_hess_grid(int num_sms);
size_t master_eval_smem(int K);
cudaError_t master_configure();
// skip (nullable): device flag that turns the launch into a no-op (graph path).
// cond / use_cond: while-node handle the step kernel sets to "not done".
cudaError_t launch_master_init(MasterDev* st, int K, const int* skip, cudaGraphConditionalHandle cond,
                               int use_cond, cudaStream_t stream, int* launches, GridBar* gb = nullptr);
cudaError_t launch_master_eval(const MasterBuffers& mb, int V, int K, const uint8_t* vstruct,
                               const StructTermsF* tf, int S, float* z_out, float* pi_out, int mode,
                               const int* skip, cudaStream_t stream, int* launches);
cudaError_t launch_master_hess(const MasterBuffers& mb, int K, int mode, cudaStream_t stream, int* launches);
// Read-only pass over a buffer larger than L2 (cold-cache timing).
cudaError_t launch_l2_evict(const void* buf, size_t bytes, float* sink, int num_sms, cudaStream_t stream);

// NVTX range for the duration of a scope: the host phases of the library
// (create, device build, solve, batch, dose, import, autotune) show up on a
// profiler's timeline; without a profiler attached the calls do nothing.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

// Process-wide memory caches (memory.cu): a stream-ordered device pool per
// device that keeps up to POOL_KEEP_MAX bytes (at most 1/16 of the device) of
// freed memory for reuse, and a free list of page-locked host blocks.
constexpr unsigned long long POOL_KEEP_MAX = 16ull << 30;
cudaError_t pool_alloc(void** p, size_t bytes, int device, cudaStream_t s);
cudaError_t pool_free(void* p, cudaStream_t s);
// *bytes_io: requested size in, size of the block handed out back.
cudaError_t pinned_alloc(void** p, size_t* bytes_io);
void pinned_release(void* p, size_t bytes);
cudaError_t release_cached_memory(int device);

// Result of the device-side input checks: the first bad CSR row and the first
// bad structure label as V - index (0: none), the padded entry count of D and
// the voxels of each structure.
struct BuildCheck {
    int bad_row;
    int bad_label;
    long long padded;
    int count[SMAX];
};

// Device-side construction of the matrices (build.cu).
// Checks rows and labels, writes the labels as bytes, and the padded row
// offsets prow[0..V] of D (rows rounded up to pad entries; clamped to INT_MAX,
// the exact total in chk->padded).  plen: V int64, bsum: check_scan_blocks(V)
// int64 of scratch.
int check_scan_blocks(int V);
cudaError_t build_check(const int64_t* rp, const int* col, const float* val, int64_t nnz, int V, int N,
                        const int* label, int S, int pad, int64_t* plen, int64_t* bsum, uint8_t* vs8, int* prow,
                        BuildCheck* chk, cudaStream_t s);
// Chunk counts C (relative slots after the call), entries per beamlet cnt,
// per-beamlet scales (smax, in place) and the largest |D_ij| (dmax).
cudaError_t build_stats(const int64_t* rp, const int* col, const float* val, int V, int CH, int N, int n_ch,
                        int* C, int* cnt, unsigned* smax, unsigned* dmax, int num_sms, cudaStream_t s);
cudaError_t build_fill_d(int prec, const int64_t* rp, const int* col, const float* val, const int* prow, int V,
                         const float* scale, DevCSR& D, cudaStream_t s);
cudaError_t build_seg(const int64_t* rp, const int* col, const int* prow, int V, const int* beam_off, int B, int* seg,
                      cudaStream_t s);
// The most groups of epg entries in one unit of 32 consecutive rows of the
// padded D (row offsets prow) into out[0], the most in one row into out[1]
// (both zeroed by the call).
cudaError_t build_unit_max(const int* prow, int V, int epg, int* out, cudaStream_t s);
// D by beams: the row offsets of every beam's part (B x (V + 1), from the beam
// segments seg), then the entries (beamlet index within the beam, value).
// tmp: B x beam_scan_tiles(V) ints of scratch.
int beam_scan_tiles(int V);
cudaError_t build_beam_rows(const int* seg, int V, int B, int* brp, int* tmp, cudaStream_t s);
cudaError_t build_beam_fill(int prec, const int* seg, int V, int B, const int* beam_off, const DevCSR& D,
                            cudaStream_t s);
// Merge-path splits of the merge form: out[v] = (rows done, groups consumed)
// at diagonal min(v * chunk, V + groups), rows finished as soon as their groups
// are (prow in entries, epg entries per group), v = 0 .. n_warps.
cudaError_t build_merge_path(const int* prow, int V, int epg, int chunk, int n_warps, int2* out, cudaStream_t s);
cudaError_t build_transpose_place(int prec, const int64_t* rp, const int* col, const float* val, int V, int CH, int N,
                                  int n_ch, int* C, const int* cnt, const float* scale, DevCSR& Dt, float* tval,
                                  int num_sms, cudaStream_t s);

// One plan's persistent master solve as the kernel reads it: the solver state,
// the slab and its partial arrays (stride GS), the objective terms, the
// round's skip flag and outputs, and the device-side round state (pool size).
struct MasterTask {
    CUtensorMap tmap[2];  // the slab in boxes of 128 voxels x 16, x 4 columns (MasterBuffers::tmap_p)
    const float* slab;
    int ld, V, GS, S, max_iter;
    MasterDev* st;
    GridBar* gb;
    float* H_part;
    double* g_part;
    float* gn_part;
    double* F_part;
    const uint8_t* vstruct;
    const StructTermsF* tf;
    double tol_rel;
    const int* skip;
    float* z_out;
    float* pi_out;
    CGDev* cg;
    uint8_t* vstate;      // MasterBuffers::vstate
    float* H_keep;        // MasterBuffers::H_keep
};
// Several plans' master solves in one cooperative launch, GB blocks each
// (master_batch_group: the most for n_tasks plans with two blocks per SM);
// tasks in device memory; max_V the largest voxel count.
int master_batch_group(int n_tasks, int num_sms);
cudaError_t launch_master_persist_batch(const MasterTask* tasks, int n_tasks, int GB, int max_V, cudaStream_t stream,
                                        int* launches);

// The whole master solve as one cooperative launch (GP blocks), after
// launch_master_init; dynamic shared memory per master_persist_smem.
size_t master_persist_smem(int V, int G);
// Diagnostic: a cooperative launch whose block `absent` never arrives at the
// grid barrier; out[0] counts the blocks whose bounded wait gave up, out[1]
// those that passed.
cudaError_t launch_barrier_check(GridBar* gb, int blocks, int absent, int* out, cudaStream_t stream);
int master_persist_grid(int V, int num_sms, int want = 0);
// Includes k_master_init's warm start, writes z and pi of the final point, and
// (cg != nullptr) the round's record.  K = 0: the pool size is read from
// cg->K when the kernel runs.
cudaError_t launch_master_persist(const MasterBuffers& mb, const float* slab, int ld, int V, int K,
                                  const uint8_t* vstruct, const StructTermsF* tf, int S, int max_iter, double tol_rel,
                                  const int* skip, float* z_out, float* pi_out, CGDev* cg, cudaStream_t stream,
                                  int* launches);

// Reduction of the partial sums and the projected-Newton step, one launch.
cudaError_t launch_master_step(int K, const MasterBuffers& mb, int max_iter, double tol_rel,
                               cudaGraphConditionalHandle cond, int use_cond, cudaStream_t stream, int* launches);
cudaError_t launch_cg_record(const MasterDev* st, CGDev* cg, int K, cudaStream_t stream, int* launches);

}  // namespace dao
