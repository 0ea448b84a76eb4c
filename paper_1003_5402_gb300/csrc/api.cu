// Host side of libdao.so: input validation, the device data layout, the
// column-generation driver (Sec. 2.2-2.3 of arXiv:1003.5402, Fig. 1) and the
// C ABI declared in include/dao.h.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dao_internal.h"

using namespace dao;

namespace {

thread_local std::string g_err;

dao_status fail(dao_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define DAO_CU(call)                                                                                    \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess) return fail(DAO_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define DAO_TRY(expr)                    \
    do {                                 \
        dao_status s_ = (expr);          \
        if (s_ != DAO_OK) return s_;     \
    } while (0)

inline int64_t round4(int64_t n) { return (n + 3) / 4 * 4; }
inline int64_t round_up(int64_t n, int m) { return (n + m - 1) / m * m; }

}  // namespace

dao_status dao::set_error(dao_status s, const std::string& msg) { return fail(s, msg); }

struct ProfRecord {
    int kc;
    cudaEvent_t start, stop;
    int launches;
};

struct dao_ctx {
    uint64_t uid = 0;                // unique for the life of the process (batch graph cache key)
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    dao_options opt{};

    int V = 0, N = 0, B = 0, R_tot = 0, max_rows = 0, S = 0;
    int64_t nnz = 0;
    std::vector<int> rows, cols, beam_off, beam_row0;
    double tau = 0.0;  // absolute pricing tolerance

    DevCSR D, Dt;
    int* seg = nullptr;              // (B + 1) x V: start of beam b's entries in row j; [B] = end of real entries
    uint8_t* vstruct = nullptr;
    StructTermsF* tf = nullptr;
    StructTermsS* ts = nullptr;      // FP32 dose-epilogue terms, thresholds split hi + lo
    int4* row_info = nullptr;        // per MLC row: beam, first beamlet, columns, row within beam
    int* beam_row0_d = nullptr;
    int4* binfo = nullptr;           // per beamlet: beam, row, column
    int* rows_d = nullptr;           // per beam: MLC rows, beamlets per row, first beamlet
    int* cols_d = nullptr;
    int* beam_off_d = nullptr;
    int* row_cnt = nullptr;          // per MLC row: tickets of the fused D^T + row search
    int max_nb = 0;                  // largest rows * cols of a beam
    size_t mlc_smem = 0;             // shared memory of the MLC-constrained pricing kernel (0: consecutive rows)

    // beamlet-level FMO (dao_fmo), allocated on its first call
    double *fx = nullptr, *fxt = nullptr, *fr = nullptr, *fp = nullptr, *fdF = nullptr;
    float *fx32 = nullptr, *fp32 = nullptr, *fg = nullptr, *fAp = nullptr;
    float *fz = nullptr, *fzt = nullptr, *fpi = nullptr, *fpit = nullptr, *fu = nullptr;
    unsigned char* ffree = nullptr;
    FmoScalars* fst = nullptr;

    // column-generation state
    int K = 0, K_cap = 0, ld = 0;
    int async_K0 = 0, async_K1 = 0;  // rounds launched by solve_async_begin
    float* slab = nullptr;           // K_cap x ld, column k = dose of aperture k (Eq. 2)
    std::vector<int> ap_beam_h, ap_lr_h;
    int* ap_beam = nullptr;
    int* ap_lr = nullptr;            // K_cap x 2*max_rows
    float* z = nullptr;
    float* pi = nullptr;
    float* w = nullptr;
    float* x = nullptr;
    float* dose = nullptr;
    float* mask = nullptr;
    double* row_v = nullptr;
    int2* row_lr = nullptr;
    PriceDev* price = nullptr;
    MasterBuffers mb;
    CGDev* cg = nullptr;             // device-side state of graph-driven solves
    std::vector<cudaGraph_t> round_graph;       // per pool size K: one column-generation round
    std::vector<cudaGraphExec_t> round_exec;
    // persistent master: one graph for every solve, a while node over rounds
    // whose kernels read the pool size from the device
    cudaGraph_t solve_graph = nullptr;
    cudaGraphExec_t solve_exec = nullptr;
    bool solve_tried = false;
    double* F_part = nullptr;
    int F_blocks = 0;
    double* F_dev = nullptr;

    // pinned staging
    unsigned char* pinned = nullptr;
    size_t off_small = 0, off_rows = 0, off_mask = 0, off_master = 0, off_cg = 0, off_bar = 0, pinned_bytes = 0;
    size_t pinned_block = 0;  // size of the cached block behind pinned

    // per master solve: evaluations (fused passes), final status, KKT residual / max|g(start)|
    std::vector<int> stat_evals, stat_status;
    std::vector<double> stat_kkt;

    std::vector<void*> dev_allocs;
    int launches_i = 0;
    int64_t launches_total = 0;

    // instrumentation
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<ProfRecord> recs;
    int open_kc = -1;
    cudaEvent_t open_start = nullptr;
    int open_launch0 = 0;

    template <class T>
    dao_status dalloc(T** p, size_t n) {
        void* q = nullptr;
        const size_t bytes = std::max<size_t>(n, 1) * sizeof(T);
        cudaError_t e = pool_alloc(&q, bytes, device, stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(DAO_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " +
                                        cudaGetErrorString(e));
        }
        dev_allocs.push_back(q);
        *p = static_cast<T*>(q);
        return DAO_OK;
    }

    cudaEvent_t event() {
        if (ev_used == ev_pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            ev_pool.push_back(e);
        }
        return ev_pool[ev_used++];
    }
    void prof_begin(int kc) {
        if (!prof_on) return;
        open_kc = kc;
        open_start = event();
        open_launch0 = launches_i;
        if (open_start) cudaEventRecord(open_start, stream);
    }
    void prof_end() {
        if (!prof_on || open_kc < 0) return;
        cudaEvent_t stop = event();
        if (open_start && stop) {
            cudaEventRecord(stop, stream);
            recs.push_back({open_kc, open_start, stop, launches_i - open_launch0});
        }
        open_kc = -1;
    }
    void count_launches() {
        launches_total += launches_i;
        launches_i = 0;
    }
};

namespace {

// Cached batch graphs that name a context are released with it (defined with the batch solve).
void batch_graphs_forget(uint64_t uid);

dao_status check_ctx(dao_ctx* c) {
    if (c == nullptr) return fail(DAO_EINVAL, "null context");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(DAO_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return DAO_OK;
}

dao_status sync(dao_ctx* c) {
    DAO_CU(cudaStreamSynchronize(c->stream));
    return DAO_OK;
}

// ---- validation ---------------------------------------------------------------

// Message for CSR row j of D (the device check found it to be the first bad
// row): the first of its faults in entry order.
std::string row_error(const dao_csr* D, int j) {
    const int64_t p0 = D->row_ptr[j], p1 = D->row_ptr[j + 1];
    if (p1 < p0 || p0 < 0 || p1 > D->nnz) return "row_ptr decreases or leaves [0, nnz] at row " + std::to_string(j);
    for (int64_t p = p0; p < p1; ++p) {
        const int32_t c = D->col[p];
        if (c < 0 || c >= D->n_beamlets) return "column index out of range at entry " + std::to_string(p);
        if (p > p0 && c <= D->col[p - 1]) return "columns not strictly increasing in row " + std::to_string(j);
        if (!std::isfinite(D->val[p])) return "non-finite value at entry " + std::to_string(p);
    }
    return "invalid row " + std::to_string(j);
}

// Host checks of everything but the per-entry and per-voxel arrays, which the
// device checks while it builds the plan's layout (build_check).
dao_status validate(const dao_csr* D, const dao_geometry* g, const dao_structures* s, const dao_weights* w,
                    const double* rx, const dao_options* opt) {
    if (!D || !g || !s || !w || !rx || !opt) return fail(DAO_EINVAL, "null argument");
    if (D->n_voxels < 1 || D->n_beamlets < 1) return fail(DAO_EINVAL, "need at least one voxel and one beamlet");
    const bool generated = D->nnz == -1 && !D->row_ptr && !D->col && !D->val;  // D made on the device
    if (!generated) {
        if (!D->row_ptr || !D->col || !D->val) return fail(DAO_EINVAL, "null CSR array");
        if (D->row_ptr[0] != 0 || D->row_ptr[D->n_voxels] != D->nnz || D->nnz < 0)
            return fail(DAO_EINVAL, "row_ptr[0] must be 0 and row_ptr[n_voxels] must equal nnz");
    }
    if (g->n_beams < 1 || !g->rows || !g->cols) return fail(DAO_EINVAL, "geometry needs at least one beam");
    int64_t total = 0;
    for (int b = 0; b < g->n_beams; ++b) {
        if (g->rows[b] < 1) return fail(DAO_EINVAL, "beam with no MLC rows");
        if (g->cols[b] < 1 || g->cols[b] > CMAX)
            return fail(DAO_EINVAL, "beamlets per MLC row must be in [1, 32]");
        total += (int64_t)g->rows[b] * g->cols[b];
    }
    if (total != D->n_beamlets) return fail(DAO_EINVAL, "sum of rows*cols differs from n_beamlets");
    if (s->n_structures < 1 || s->n_structures > SMAX || !s->voxel_struct || !s->is_target)
        return fail(DAO_EINVAL, "n_structures must be in [1, 64]");
    if (!w->under_w || !w->over_w || !w->over_thresh) return fail(DAO_EINVAL, "null weight array");
    for (int k = 0; k < s->n_structures; ++k) {
        if (!(w->under_w[k] >= 0) || !std::isfinite(w->under_w[k]) || !(w->over_w[k] >= 0) ||
            !std::isfinite(w->over_w[k]) || !std::isfinite(w->over_thresh[k]))
            return fail(DAO_EINVAL, "weights must be finite and >= 0, thresholds finite");
        if (s->is_target[k] && !std::isfinite(rx[k])) return fail(DAO_EINVAL, "non-finite prescription");
    }
    if (opt->k_max < 1 || opt->k_max > KMAX) return fail(DAO_EINVAL, "k_max must be in [1, 64]");
    if (opt->max_master_iters < 1) return fail(DAO_EINVAL, "max_master_iters must be >= 1");
    if (!(opt->master_tol > 0) || !(opt->price_tol >= 0)) return fail(DAO_EINVAL, "tolerances must be positive");
    if (opt->precision != DAO_PREC_FP32 && opt->precision != DAO_PREC_FP16 && opt->precision != DAO_PREC_BF16)
        return fail(DAO_EINVAL, "precision must be DAO_PREC_FP32, DAO_PREC_FP16 or DAO_PREC_BF16");
    if (opt->master_blocks < 0) return fail(DAO_EINVAL, "master_blocks must be >= 0");
    if (opt->dt_threads != 0 && opt->dt_threads != 64 && opt->dt_threads != 128 && opt->dt_threads != 256)
        return fail(DAO_EINVAL, "dt_threads must be 0, 64, 128 or 256");
    if (opt->dt_map < 0 || opt->dt_map > DT_MAP_SPLIT)
        return fail(DAO_EINVAL, "dt_map must be 0, DAO_DT_GROUPED, DAO_DT_CONSECUTIVE or DAO_DT_SPLIT");
    if (opt->dose_form < 0 || opt->dose_form > DOSE_FORM_MERGE)
        return fail(DAO_EINVAL, "dose_form must be 0, DAO_DOSE_LANES, DAO_DOSE_UNITS or DAO_DOSE_MERGE");
    if (opt->column_lanes != 0 && opt->column_lanes != 1 && opt->column_lanes != 2 && opt->column_lanes != 4 &&
        opt->column_lanes != 8 && opt->column_lanes != 16)  // 0: D by beams, one lane per voxel row
        return fail(DAO_EINVAL, "column_lanes must be 0, 1, 2, 4, 8 or 16");
    if (opt->split_warps < 0) return fail(DAO_EINVAL, "split_warps must be >= 0");
    if (opt->mlc_constraint < DAO_MLC_CONSECUTIVE || opt->mlc_constraint > DAO_MLC_JAWS)
        return fail(DAO_EINVAL, "mlc_constraint must be one of DAO_MLC_*");
    if (opt->mlc_constraint != DAO_MLC_CONSECUTIVE)
        for (int b = 0; b < g->n_beams; ++b)
            if (g->rows[b] > 64) return fail(DAO_EINVAL, "the MLC-constrained pricing takes at most 64 rows per beam");
    if (opt->precision != DAO_PREC_FP32 && D->n_beamlets > 65536)
        return fail(DAO_EINVAL, "16-bit storage keeps beamlet indices in 16 bits: at most 65536 beamlets");
    return DAO_OK;
}

// ---- device data layout -------------------------------------------------------

template <class T>
dao_status upload(dao_ctx* c, T** dst, const T* src, size_t n) {
    // ordered on the context's stream (a non-blocking stream does not wait for
    // copies on the legacy default stream); build() synchronises before the
    // host arrays go out of scope
    DAO_TRY(c->dalloc(dst, n));
    if (n) DAO_CU(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return DAO_OK;
}

// D already on the device (pool memory that build() takes over and frees).
struct DeviceCSR {
    int64_t* rp = nullptr;
    int* col = nullptr;
    float* val = nullptr;
    int64_t nnz = 0;
};

dao_status build(dao_ctx* c, const dao_csr* Din, const dao_geometry* g, const dao_structures* s,
                 const dao_weights* w, const double* rx, const dao_voxel_terms* vt, DeviceCSR* din) {
    const int V = c->V, N = c->N, B = c->B;
    // beam geometry
    c->rows.assign(g->rows, g->rows + B);
    c->cols.assign(g->cols, g->cols + B);
    c->beam_off.assign(B + 1, 0);
    c->beam_row0.assign(B + 1, 0);
    for (int b = 0; b < B; ++b) {
        c->beam_off[b + 1] = c->beam_off[b] + c->rows[b] * c->cols[b];
        c->beam_row0[b + 1] = c->beam_row0[b] + c->rows[b];
        c->max_rows = std::max(c->max_rows, c->rows[b]);
    }
    c->R_tot = c->beam_row0[B];
    std::vector<int4> ri(c->R_tot), bi(N);
    for (int b = 0; b < B; ++b)
        for (int r = 0; r < c->rows[b]; ++r) {
            ri[c->beam_row0[b] + r] = make_int4(b, c->beam_off[b] + r * c->cols[b], c->cols[b], r);
            for (int q = 0; q < c->cols[b]; ++q) bi[c->beam_off[b] + r * c->cols[b] + q] = make_int4(b, r, q, 0);
        }

    // D (voxel-major) with per-row beam segments, and D^T, built on the device
    // from the caller's CSR (uploaded as is) after the device has checked it.
    // Rows are padded to 4 entries (one float4 / int4 load) or, with 16-bit
    // values, to 8 entries (one 16-byte load of values and of 16-bit columns).
    const int prec = c->opt.precision;
    const int pad_m = prec == DAO_PREC_FP32 ? 4 : 8;
    const int64_t nnz = din ? din->nnz : Din->nnz;
    const int S = s->n_structures;
    c->S = S;
    // rows of D per chunk of the transpose: the chunk-by-beamlet counters stay under 16M
    const int CH = (int)std::max<int64_t>(256, ((int64_t)V * N / (16 << 20) + 31) / 32 * 32);
    const int n_ch = (V + CH - 1) / CH;
    cudaStream_t st = c->stream;
    // temporaries, stream-ordered
    int64_t* t_rp = nullptr;
    int* t_col = nullptr;
    float* t_val = nullptr;
    int* t_lab = nullptr;
    int64_t* t_plen = nullptr;
    int64_t* t_bsum = nullptr;
    BuildCheck* t_chk = nullptr;
    int* t_C = nullptr;
    int* t_cnt = nullptr;
    unsigned* t_dmax = nullptr;
    int* t_umax = nullptr;
    int* t_bscan = nullptr;
    float* t_tval = nullptr;
    auto free_temps = [&]() {
        for (void* q : {(void*)t_rp, (void*)t_col, (void*)t_val, (void*)t_lab, (void*)t_plen, (void*)t_bsum,
                        (void*)t_chk, (void*)t_C, (void*)t_cnt, (void*)t_dmax, (void*)t_umax, (void*)t_bscan,
                        (void*)(prec == DAO_PREC_FP32 ? nullptr : t_tval)})
            if (q) pool_free(q, st);
    };
    auto talloc = [&](auto** q, size_t bytes) -> dao_status {
        void* v = nullptr;
        const cudaError_t e = pool_alloc(&v, bytes, c->device, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            free_temps();
            return fail(DAO_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
        }
        *q = static_cast<std::remove_pointer_t<decltype(q)>>(v);
        return DAO_OK;
    };
    auto cu = [&](cudaError_t e, const char* what) -> dao_status {
        if (e == cudaSuccess) return DAO_OK;
        free_temps();
        return fail(DAO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    if (din) {  // generated on the device: taken over, freed with the other temporaries
        t_rp = din->rp;
        t_col = din->col;
        t_val = din->val;
        *din = DeviceCSR{};
    } else {
        DAO_TRY(talloc(&t_rp, sizeof(int64_t) * (V + 1)));
        DAO_TRY(talloc(&t_col, sizeof(int) * nnz));
        DAO_TRY(talloc(&t_val, sizeof(float) * nnz));
    }
    DAO_TRY(talloc(&t_lab, sizeof(int) * V));
    DAO_TRY(talloc(&t_plen, sizeof(int64_t) * V));
    DAO_TRY(talloc(&t_bsum, sizeof(int64_t) * check_scan_blocks(V)));
    DAO_TRY(talloc(&t_chk, sizeof(BuildCheck)));
    if (Din->row_ptr) {
        DAO_TRY(cu(cudaMemcpyAsync(t_rp, Din->row_ptr, sizeof(int64_t) * (V + 1), cudaMemcpyHostToDevice, st),
                   "upload"));
        DAO_TRY(cu(cudaMemcpyAsync(t_col, Din->col, sizeof(int) * nnz, cudaMemcpyHostToDevice, st), "upload"));
        DAO_TRY(cu(cudaMemcpyAsync(t_val, Din->val, sizeof(float) * nnz, cudaMemcpyHostToDevice, st), "upload"));
    }
    DAO_TRY(cu(cudaMemcpyAsync(t_lab, s->voxel_struct, sizeof(int) * V, cudaMemcpyHostToDevice, st), "upload"));
    DAO_TRY(c->dalloc(&c->D.rowptr, (size_t)V + 1));
    DAO_TRY(c->dalloc(&c->vstruct, V));
    // checks of every row and label, padded row offsets, voxels per structure
    TraceRange range("device checks and layout");
    BuildCheck chk{};
    DAO_TRY(cu(build_check(t_rp, t_col, t_val, nnz, V, N, t_lab, S, pad_m, t_plen, t_bsum, c->vstruct, c->D.rowptr,
                           t_chk, st), "input checks"));
    DAO_TRY(cu(cudaMemcpyAsync(&chk, t_chk, sizeof(BuildCheck), cudaMemcpyDeviceToHost, st), "check read-back"));
    DAO_TRY(cu(cudaStreamSynchronize(st), "input checks"));
    if (chk.bad_row > 0) {
        free_temps();
        return fail(DAO_EINVAL, Din->row_ptr ? row_error(Din, V - chk.bad_row)
                                             : "invalid generated row " + std::to_string(V - chk.bad_row));
    }
    if (chk.bad_label > 0) {
        free_temps();
        return fail(DAO_EINVAL, "voxel structure label out of range at voxel " + std::to_string(V - chk.bad_label));
    }
    const int64_t padded = chk.padded;
    if (padded >= (int64_t)1 << 31) {
        free_temps();
        return fail(DAO_EINVAL, "D too large for 32-bit row offsets");
    }
    DAO_TRY(talloc(&t_C, sizeof(int) * (size_t)n_ch * N));
    DAO_TRY(talloc(&t_cnt, sizeof(int) * N));
    DAO_TRY(talloc(&t_dmax, sizeof(unsigned)));
    DAO_TRY(talloc(&t_umax, 2 * sizeof(int)));
    c->D.n_rows = V;
    c->D.n_cols = N;
    c->D.nnz_stored = padded;
    c->D.prec = prec;
    c->Dt.n_rows = N;
    c->Dt.n_cols = V;
    c->Dt.prec = prec;
    c->Dt.tune_dt_threads = c->opt.dt_threads;
    c->Dt.tune_dt_map = c->opt.dt_map;
    c->D.tune_dose_form = c->opt.dose_form;
    c->D.tune_col_g = c->opt.column_lanes;
    float* scale = nullptr;
    DAO_TRY(c->dalloc(&scale, N));
    c->D.scale = scale;
    c->Dt.scale = scale;
    DAO_TRY(upload(c, &c->beam_off_d, c->beam_off.data(), c->beam_off.size()));
    DAO_TRY(c->dalloc(&c->seg, (size_t)(B + 1) * V));
    if (prec == DAO_PREC_FP32) {
        DAO_TRY(c->dalloc(&c->D.col, padded));
        DAO_TRY(c->dalloc(&c->D.val, padded));
    } else {
        DAO_TRY(c->dalloc(&c->D.col16, padded));
        DAO_TRY(c->dalloc(&c->D.val16, padded));
    }
    DAO_TRY(cu(build_stats(t_rp, t_col, t_val, V, CH, N, n_ch, t_C, t_cnt, reinterpret_cast<unsigned*>(scale), t_dmax,
                           c->num_sms, st), "transpose counts and scales"));
    DAO_TRY(cu(build_fill_d(prec, t_rp, t_col, t_val, c->D.rowptr, V, scale, c->D, st), "padded D"));
    DAO_TRY(cu(build_seg(t_rp, t_col, c->D.rowptr, V, c->beam_off_d, B, c->seg, st), "beam segments"));
    // D by beams for the aperture column (a4): each beam's part of every row
    // in one contiguous range
    DAO_TRY(c->dalloc(&c->D.beam_rowptr, (size_t)B * (V + 1)));
    DAO_TRY(c->dalloc(&c->D.beam_col, (size_t)nnz));
    if (prec == DAO_PREC_FP32)
        DAO_TRY(c->dalloc(&c->D.beam_val32, (size_t)nnz));
    else
        DAO_TRY(c->dalloc(&c->D.beam_val16, (size_t)nnz));
    DAO_TRY(talloc(&t_bscan, sizeof(int) * (size_t)B * beam_scan_tiles(V)));
    DAO_TRY(cu(build_beam_rows(c->seg, V, B, c->D.beam_rowptr, t_bscan, st), "beam rows"));
    DAO_TRY(cu(build_beam_fill(prec, c->seg, V, B, c->beam_off_d, c->D, st), "beam layout"));
    DAO_TRY(cu(build_unit_max(c->D.rowptr, V, pad_m, t_umax, st), "row units"));
    // counts, the largest |D_ij| and the largest row unit back to the host: row
    // offsets of D^T, tau, the dose SpMV's shared partials
    std::vector<int> cnt(N);
    unsigned dmax_bits = 0;
    int umax[2] = {0, 0};
    DAO_TRY(cu(cudaMemcpyAsync(cnt.data(), t_cnt, sizeof(int) * N, cudaMemcpyDeviceToHost, st), "counts"));
    DAO_TRY(cu(cudaMemcpyAsync(&dmax_bits, t_dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "max"));
    DAO_TRY(cu(cudaMemcpyAsync(umax, t_umax, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "units"));
    DAO_TRY(cu(cudaStreamSynchronize(st), "device build"));
    c->D.unit_groups_max = std::max(umax[0], 1);
    {
        // the merge form of a1: the merge of D's groups and row ends in equal
        // stretches (longer than the longest row) over a fixed set of warps
        const int64_t items = padded / pad_m + V;
        const int64_t warps =
            c->opt.split_warps > 0 ? (int64_t)c->opt.split_warps : (int64_t)c->num_sms * MERGE_WARPS_PER_SM;
        int64_t chunk = std::max<int64_t>((items + warps - 1) / warps, (int64_t)umax[1] + 1);
        if (chunk > MERGE_CHUNK_MAX) chunk = std::max<int64_t>(MERGE_CHUNK_MAX, (int64_t)umax[1] + 1);
        if (padded > 0 && chunk <= MERGE_CHUNK_MAX) {
            const int nw = (int)((items + chunk - 1) / chunk);
            int2* mp = nullptr;
            DAO_TRY(c->dalloc(&mp, (size_t)nw + 1));
            DAO_TRY(c->dalloc(&c->D.merge_slot, 2 * (size_t)nw));
            DAO_TRY(c->dalloc(&c->D.merge_cnt, (size_t)nw));
            DAO_TRY(cu(cudaMemsetAsync(c->D.merge_cnt, 0, sizeof(int) * (size_t)nw, st), "merge tickets"));
            DAO_TRY(cu(build_merge_path(c->D.rowptr, V, pad_m, (int)chunk, nw, mp, st), "merge path"));
            c->D.merge_path = mp;
            c->D.merge_chunk = (int)chunk;
            c->D.merge_warps = nw;
        }
    }
    std::vector<int> trow(N + 1, 0);
    int64_t tpadded = 0;
    for (int i = 0; i < N; ++i) {
        trow[i] = (int)std::min<int64_t>(tpadded, INT32_MAX);
        tpadded += round_up(cnt[i], pad_m);
    }
    if (tpadded >= (int64_t)1 << 31) {
        free_temps();
        return fail(DAO_EINVAL, "D^T too large for 32-bit row offsets");
    }
    trow[N] = (int)tpadded;
    c->Dt.nnz_stored = tpadded;
    DAO_TRY(upload(c, &c->Dt.rowptr, trow.data(), trow.size()));
    // rows of D^T by decreasing length (ties by index) for the transposed SpMV;
    // the host copy lives until build() has synchronised
    std::vector<int> order(N);
    for (int i = 0; i < N; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] > cnt[b]; });
    {
        int* od = nullptr;
        DAO_TRY(upload(c, &od, order.data(), order.size()));
        c->Dt.order = od;
    }
    // the split form of a2 (every row of D^T at least 32 stored entries): the
    // entries in equal chunks (multiples of 32) over a fixed set of warps, the
    // row holding each chunk's first entry, and the most warps one row spans
    std::vector<int> srow;
    {
        int min_len = INT32_MAX;
        for (int i = 0; i < N; ++i) min_len = std::min(min_len, trow[i + 1] - trow[i]);
        const int64_t warps =
            c->opt.split_warps > 0 ? (int64_t)c->opt.split_warps : (int64_t)c->num_sms * SPLIT_WARPS_PER_SM;
        if (N > 0 && min_len >= 32 && tpadded > 0) {
            const int64_t chunk = std::max<int64_t>(32, ((tpadded + warps - 1) / warps + 31) / 32 * 32);
            const int nw = (int)((tpadded + chunk - 1) / chunk);
            srow.resize(nw);
            int ps = 1;
            for (int v = 0, r = 0; v < nw; ++v) {
                const int64_t e = (int64_t)v * chunk;
                while (trow[r + 1] <= e) ++r;
                srow[v] = r;
            }
            for (int i = 0; i < N; ++i)
                ps = std::max(ps, (int)((trow[i + 1] - 1) / chunk - trow[i] / chunk + 1));
            int* sr = nullptr;
            DAO_TRY(upload(c, &sr, srow.data(), srow.size()));
            DAO_TRY(c->dalloc(&c->Dt.split_part, (size_t)N * ps));
            DAO_TRY(c->dalloc(&c->Dt.split_cnt, (size_t)N));
            DAO_CU(cudaMemsetAsync(c->Dt.split_cnt, 0, sizeof(int) * (size_t)N, st));
            c->Dt.split_row = sr;
            c->Dt.split_chunk = (int)chunk;
            c->Dt.split_warps = nw;
            c->Dt.split_ps = ps;
        }
    }
    DAO_TRY(c->dalloc(&c->Dt.col, tpadded));
    if (prec == DAO_PREC_FP32) {
        DAO_TRY(c->dalloc(&c->Dt.val, tpadded));
        t_tval = c->Dt.val;
    } else {
        DAO_TRY(c->dalloc(&c->Dt.val16, tpadded));
        DAO_TRY(talloc(&t_tval, sizeof(float) * tpadded));
    }
    DAO_TRY(cu(build_transpose_place(prec, t_rp, t_col, t_val, V, CH, N, n_ch, t_C, t_cnt, scale, c->Dt, t_tval,
                                     c->num_sms, st),
               "transpose"));
    free_temps();
    float dmax = 0.f;
    std::memcpy(&dmax, &dmax_bits, sizeof(float));

    // objective terms per structure (Eqs. 9-10); voxel counts from the device check
    std::vector<StructTermsD> tdh(S);
    std::vector<StructTermsF> tfh(S);
    std::vector<StructTermsS> tsh(S);
    double pi0_l1 = 0.0;
    for (int k = 0; k < S; ++k) {
        const int64_t count = chk.count[k];
        const double vol = (w->normalize_by_volume && count > 0) ? (double)count : 1.0;
        const bool tgt = s->is_target[k] != 0;
        tdh[k].a = tgt ? w->under_w[k] / vol : 0.0;
        tdh[k].tu = tgt ? rx[k] : 0.0;
        tdh[k].b = w->over_w[k] / vol;
        tdh[k].to = w->over_thresh[k];
        tfh[k] = {(float)tdh[k].a, (float)tdh[k].tu, (float)tdh[k].b, (float)tdh[k].to};
        const float tu_hi = (float)tdh[k].tu, to_hi = (float)tdh[k].to;
        tsh[k] = {(float)tdh[k].a, tu_hi, (float)(tdh[k].tu - (double)tu_hi), (float)tdh[k].b, to_hi,
                  (float)(tdh[k].to - (double)to_hi), 0.f, 0.f};
        // |grad F(0)| summed over the structure's voxels
        pi0_l1 += (double)count * (2.0 * tdh[k].a * std::max(0.0, tdh[k].tu) + 2.0 * tdh[k].b * std::max(0.0, -tdh[k].to));
    }
    if (vt != nullptr) {
        // re-optimisation form of Eqs. 3-4: every voxel its own weights and
        // thresholds (the kernels read terms[j] when S < 0); no volume division
        tfh.assign(V, StructTermsF{});
        tsh.assign(V, StructTermsS{});
        pi0_l1 = 0.0;
        for (int j = 0; j < V; ++j) {
            const double a = vt->under_w[j], tu = vt->under_t[j], b = vt->over_w[j], to = vt->over_t[j];
            tfh[j] = {(float)a, (float)tu, (float)b, (float)to};
            const float tu_hi = (float)tu, to_hi = (float)to;
            tsh[j] = {(float)a, tu_hi, (float)(tu - (double)tu_hi), (float)b, to_hi, (float)(to - (double)to_hi),
                      0.f, 0.f};
            pi0_l1 += 2.0 * a * std::max(0.0, tu) + 2.0 * b * std::max(0.0, -to);
        }
        c->S = -1;
    }
    c->tau = c->opt.price_tol * (double)dmax * pi0_l1;

    DAO_TRY(upload(c, &c->tf, tfh.data(), tfh.size()));
    DAO_TRY(upload(c, &c->ts, tsh.data(), tsh.size()));
    DAO_TRY(upload(c, &c->row_info, ri.data(), ri.size()));
    DAO_TRY(upload(c, &c->beam_row0_d, c->beam_row0.data(), c->beam_row0.size()));
    DAO_TRY(upload(c, &c->binfo, bi.data(), bi.size()));
    DAO_TRY(upload(c, &c->rows_d, c->rows.data(), c->rows.size()));
    DAO_TRY(upload(c, &c->cols_d, c->cols.data(), c->cols.size()));
    DAO_TRY(sync(c));
    return DAO_OK;
}

// 2-D tensor maps over the column-major slab (column k = aperture k, stride
// ld floats): box = (MASTER_TILE voxels, KP columns), one map per KP.
dao_status make_tensor_maps(dao_ctx* c) {
    typedef CUresult (*encode_fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    DAO_CU(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (fn == nullptr || q != cudaDriverEntryPointSuccess) return fail(DAO_ECUDA, "cuTensorMapEncodeTiled unavailable");
    encode_fn encode = reinterpret_cast<encode_fn>(fn);
    std::memset(c->mb.tmap, 0, sizeof(c->mb.tmap));
    for (int kp = 4; kp <= KMAX; kp += 4) {
        const cuuint64_t dims[2] = {(cuuint64_t)c->ld, (cuuint64_t)KMAX};
        const cuuint64_t strides[1] = {(cuuint64_t)c->ld * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)MASTER_TILE, (cuuint32_t)kp};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&c->mb.tmap[kp / 4], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->slab, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(DAO_ECUDA, "cuTensorMapEncodeTiled failed with " + std::to_string((int)r));
    }
    for (int m = 0; m < 2; ++m) {  // the persistent solve's maps: boxes of 128 voxels x 16, x 4 columns
        const cuuint64_t dims[2] = {(cuuint64_t)c->ld, (cuuint64_t)KMAX};
        const cuuint64_t strides[1] = {(cuuint64_t)c->ld * sizeof(float)};
        const cuuint32_t box[2] = {128u, m == 0 ? 16u : 4u};
        const cuuint32_t estr[2] = {1, 1};
        CUresult r = encode(&c->mb.tmap_p[m], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, c->slab, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(DAO_ECUDA, "cuTensorMapEncodeTiled failed with " + std::to_string((int)r));
    }
    return DAO_OK;
}

dao_status alloc_state(dao_ctx* c) {
    c->K_cap = c->opt.k_max;
    c->mb.n_tiles = (c->V + MASTER_TILE - 1) / MASTER_TILE;
    c->ld = c->mb.n_tiles * MASTER_TILE;  // column stride: voxels zero padded to whole tiles
    DAO_TRY(c->dalloc(&c->slab, (size_t)c->ld * KMAX));
    DAO_CU(cudaMemsetAsync(c->slab, 0, (size_t)c->ld * KMAX * sizeof(float), c->stream));
    DAO_TRY(make_tensor_maps(c));
    DAO_TRY(c->dalloc(&c->ap_beam, c->K_cap));
    DAO_TRY(c->dalloc(&c->ap_lr, (size_t)c->K_cap * 2 * c->max_rows));
    DAO_TRY(c->dalloc(&c->z, c->V));
    DAO_TRY(c->dalloc(&c->pi, c->V));
    DAO_TRY(c->dalloc(&c->dose, c->V));
    DAO_TRY(c->dalloc(&c->w, c->N));
    DAO_TRY(c->dalloc(&c->x, c->N));
    int nbmax = 0;
    for (int b = 0; b < c->B; ++b) nbmax = std::max(nbmax, c->rows[b] * c->cols[b]);
    DAO_TRY(c->dalloc(&c->mask, nbmax));
    c->max_nb = nbmax;
    DAO_TRY(c->dalloc(&c->cg, 1));
    DAO_CU(cudaMemsetAsync(c->cg, 0, sizeof(CGDev), c->stream));
    c->round_graph.assign(c->K_cap + 1, nullptr);
    c->round_exec.assign(c->K_cap + 1, nullptr);
    DAO_TRY(c->dalloc(&c->row_v, c->R_tot));
    DAO_TRY(c->dalloc(&c->row_lr, c->R_tot));
    DAO_TRY(c->dalloc(&c->row_cnt, c->R_tot));
    DAO_CU(cudaMemsetAsync(c->row_cnt, 0, (size_t)std::max(c->R_tot, 1) * sizeof(int), c->stream));
    DAO_TRY(c->dalloc(&c->price, 1));
    if (c->opt.mlc_constraint != DAO_MLC_CONSECUTIVE) {
        int max_cols = 0;
        for (int b = 0; b < c->B; ++b) max_cols = std::max(max_cols, c->cols[b]);
        c->mlc_smem = mlc_smem_bytes(c->opt.mlc_constraint, c->max_rows, max_cols);
        DAO_CU(mlc_configure(c->opt.mlc_constraint, c->mlc_smem));
    }
    for (int k = 0; k <= KMAX; ++k) c->mb.grid[k] = master_grid(c->V, c->num_sms, k);
    c->mb.GH = master_hess_grid(c->num_sms);
    DAO_TRY(c->dalloc(&c->mb.bar, 1));
    DAO_TRY(c->dalloc(&c->mb.vstate, (size_t)std::max(c->V, 1)));
    DAO_CU(cudaMemsetAsync(c->mb.bar, 0, sizeof(GridBar), c->stream));
    c->mb.GP = c->opt.master_persistent ? master_persist_grid(c->V, c->num_sms, c->opt.master_blocks) : 0;
    if (c->mb.GP > c->mb.GH) c->mb.GP = c->mb.GH;  // the partial arrays have GH columns
    DAO_TRY(c->dalloc(&c->mb.st, 1));
    DAO_TRY(c->dalloc(&c->mb.act_rows, (size_t)c->ld * KROW));
    DAO_TRY(c->dalloc(&c->mb.act_hp, (size_t)c->ld));
    DAO_TRY(c->dalloc(&c->mb.act_count, (size_t)c->mb.n_tiles));
    DAO_CU(cudaMemsetAsync(c->mb.act_count, 0, (size_t)c->mb.n_tiles * sizeof(int), c->stream));
    DAO_TRY(c->dalloc(&c->mb.H_part, (size_t)KMAX * (KMAX + 1) / 2 * c->mb.GH));
    DAO_TRY(c->dalloc(&c->mb.g_part, (size_t)KMAX * c->mb.GH));
    DAO_TRY(c->dalloc(&c->mb.gn_part, (size_t)KMAX * c->mb.GH));
    DAO_TRY(c->dalloc(&c->mb.H_keep, (size_t)KMAX * (KMAX + 1) / 2 * c->mb.GH));
    DAO_TRY(c->dalloc(&c->mb.F_part, (size_t)master_grid_max(c->num_sms)));
    c->F_blocks = std::max(dose_grid(c->V, c->num_sms), dose_merge_f_slots(c->D));
    DAO_TRY(c->dalloc(&c->F_part, c->F_blocks));
    DAO_TRY(c->dalloc(&c->F_dev, 1));
    DAO_CU(cudaMemsetAsync(c->mb.st, 0, sizeof(MasterDev), c->stream));
    DAO_CU(cudaMemsetAsync(c->ap_lr, 0, (size_t)c->K_cap * 2 * c->max_rows * sizeof(int), c->stream));
    c->off_small = 0;
    c->off_rows = 256;
    c->off_mask = c->off_rows + round4((int64_t)c->R_tot * 2) * sizeof(int);
    c->off_master = round4(c->off_mask + (size_t)nbmax * sizeof(float) + 64) + 64;
    c->off_master = (c->off_master + 255) / 256 * 256;
    c->off_cg = (c->off_master + sizeof(MasterDev) + 255) / 256 * 256;
    c->off_bar = (c->off_cg + sizeof(CGDev) + 15) / 16 * 16;
    c->pinned_bytes = c->off_bar + sizeof(GridBar);
    void* p = nullptr;
    size_t got = c->pinned_bytes;
    DAO_CU(pinned_alloc(&p, &got));
    c->pinned = static_cast<unsigned char*>(p);
    c->pinned_block = got;
    return DAO_OK;
}

// ---- the column-generation steps ------------------------------------------------

// The per-row part of pricing on w (row_v, row_lr): the paper's row search per
// MLC row, or the beams priced under the context's MLC constraint.
cudaError_t price_rows_any(dao_ctx* c, const float* w, const int* skip, cudaStream_t s, int* n) {
    if (c->opt.mlc_constraint == DAO_MLC_CONSECUTIVE)
        return launch_price_rows(w, c->row_info, c->R_tot, c->row_v, c->row_lr, skip, s, n);
    return launch_price_mlc(c->opt.mlc_constraint, w, c->beam_off_d, c->rows_d, c->cols_d, c->beam_row0_d, c->B,
                            c->mlc_smem, c->row_v, c->row_lr, skip, s, n);
}

// Both parts of pricing: row results, beam sums and their argmin into c->price.
cudaError_t price_any(dao_ctx* c, const float* w, const int* skip, cudaStream_t s, int* n) {
    if (c->opt.mlc_constraint == DAO_MLC_CONSECUTIVE)
        return launch_price(w, c->row_info, c->R_tot, c->beam_row0_d, c->B, c->row_v, c->row_lr, c->price, skip, s,
                            n);
    cudaError_t e = price_rows_any(c, w, skip, s, n);
    if (e != cudaSuccess) return e;
    return launch_price_beams(c->row_v, c->beam_row0_d, c->B, c->price, skip, s, n);
}

// pi = grad F(z) and z at the current pool's accepted intensities (final pass).
dao_status refresh_state(dao_ctx* c) {
    c->prof_begin(DAO_KC_MASTER_PASS);
    DAO_CU(launch_master_eval(c->mb, c->V, c->K, c->vstruct, c->tf, c->S, c->z, c->pi, PASS_FINAL, nullptr, c->stream,
                              &c->launches_i));
    c->prof_end();
    return DAO_OK;
}

dao_status master_solve(dao_ctx* c, double* F_out) {
    const size_t tail = sizeof(MasterDev) - offsetof(MasterDev, F);
    MasterDev* shadow = reinterpret_cast<MasterDev*>(c->pinned + c->off_master - offsetof(MasterDev, F));
    if (c->mb.GP > 0) {  // the whole solve as one cooperative launch (warm start, z and pi included)
        DAO_CU(cudaMemsetAsync(c->mb.bar, 0, sizeof(GridBar), c->stream));
        c->prof_begin(DAO_KC_MASTER_SOLVE);
        DAO_CU(launch_master_persist(c->mb, c->slab, c->ld, c->V, c->K, c->vstruct, c->tf, c->S,
                                     c->opt.max_master_iters, c->opt.master_tol, nullptr, c->z, c->pi, nullptr,
                                     c->stream, &c->launches_i));
        c->prof_end();
        DAO_CU(cudaMemcpyAsync(&shadow->F, &c->mb.st->F, tail, cudaMemcpyDeviceToHost, c->stream));
        DAO_TRY(sync(c));
        if (shadow->err == 2) return fail(DAO_ETIMEOUT, "a grid barrier of the master solve timed out");
        if (shadow->status == MASTER_ERROR) return fail(DAO_ETIMEOUT, "the master solve stopped on an error");
        if (!shadow->done) return fail(DAO_ETIMEOUT, "master problem did not stop");
        c->stat_evals.push_back(shadow->n_eval);
        c->stat_status.push_back(shadow->status);
        c->stat_kkt.push_back(shadow->res / (shadow->tol > 0 ? shadow->tol / c->opt.master_tol : 1.0));
        if (F_out) *F_out = shadow->F;
        return DAO_OK;
    }
    DAO_CU(launch_master_init(c->mb.st, c->K, nullptr, 0, 0, c->stream, &c->launches_i, c->mb.bar));
    const int unroll = 4;
    const int max_passes = c->opt.max_master_iters + 80;
    int passes = 0;
    for (;;) {
        for (int u = 0; u < unroll; ++u) {
            c->prof_begin(DAO_KC_MASTER_PASS);
            DAO_CU(launch_master_eval(c->mb, c->V, c->K, c->vstruct, c->tf, c->S, nullptr, nullptr, PASS_EVAL, nullptr,
                                      c->stream, &c->launches_i));
            c->prof_end();
            c->prof_begin(DAO_KC_MASTER_HESS);
            DAO_CU(launch_master_hess(c->mb, c->K, PASS_EVAL, c->stream, &c->launches_i));
            c->prof_end();
            c->prof_begin(DAO_KC_MASTER_STEP);
            DAO_CU(launch_master_step(c->K, c->mb, c->opt.max_master_iters, c->opt.master_tol, 0, 0, c->stream,
                                      &c->launches_i));
            c->prof_end();
        }
        passes += unroll;
        DAO_CU(cudaMemcpyAsync(&shadow->F, &c->mb.st->F, tail, cudaMemcpyDeviceToHost, c->stream));
        DAO_TRY(sync(c));
        if (shadow->done) break;
        if (passes > max_passes) return fail(DAO_ETIMEOUT, "master problem did not stop within its evaluation cap");
    }
    DAO_TRY(refresh_state(c));
    if (shadow->status == MASTER_ERROR) return fail(DAO_ETIMEOUT, "a slab tile copy did not complete");
    c->stat_evals.push_back(shadow->n_eval);
    c->stat_status.push_back(shadow->status);
    c->stat_kkt.push_back(shadow->res / (shadow->tol > 0 ? shadow->tol / c->opt.master_tol : 1.0));
    if (F_out) *F_out = shadow->F;
    return DAO_OK;
}

// pricing on the vector w already on the device; fills host outputs
dao_status price_on_w(dao_ctx* c, const float* w, int32_t* beam, int32_t* leaf_lr, double* rc, double* row_best,
                      int32_t* row_lr_out) {
    c->prof_begin(DAO_KC_PRICE);
    DAO_CU(price_any(c, w, nullptr, c->stream, &c->launches_i));
    c->prof_end();
    PriceDev* pd = reinterpret_cast<PriceDev*>(c->pinned + c->off_small + 16);
    int* lr = reinterpret_cast<int*>(c->pinned + c->off_rows);
    DAO_CU(cudaMemcpyAsync(pd, c->price, sizeof(PriceDev), cudaMemcpyDeviceToHost, c->stream));
    DAO_CU(cudaMemcpyAsync(lr, c->row_lr, sizeof(int2) * c->R_tot, cudaMemcpyDeviceToHost, c->stream));
    if (row_best) DAO_CU(cudaMemcpyAsync(row_best, c->row_v, sizeof(double) * c->R_tot, cudaMemcpyDeviceToHost, c->stream));
    DAO_TRY(sync(c));
    const int b = pd->beam;
    if (beam) *beam = b;
    if (rc) *rc = pd->rc;
    if (leaf_lr)
        for (int r = 0; r < c->rows[b]; ++r) {
            leaf_lr[2 * r] = lr[2 * (c->beam_row0[b] + r)];
            leaf_lr[2 * r + 1] = lr[2 * (c->beam_row0[b] + r) + 1];
        }
    if (row_lr_out) std::memcpy(row_lr_out, lr, sizeof(int) * 2 * c->R_tot);
    return DAO_OK;
}

dao_status validate_aperture(const dao_ctx* c, int beam, const int32_t* lr) {
    if (beam < 0 || beam >= c->B || lr == nullptr) return fail(DAO_EINVAL, "invalid beam index");
    for (int r = 0; r < c->rows[beam]; ++r) {
        const int L = lr[2 * r], R = lr[2 * r + 1];
        if (L < 0 || R < L || R > c->cols[beam])
            return fail(DAO_EINVAL, "leaf range out of bounds in row " + std::to_string(r));
    }
    return DAO_OK;
}

bool is_duplicate(const dao_ctx* c, int beam, const int32_t* lr) {
    const int stride = 2 * c->max_rows;
    for (int k = 0; k < c->K; ++k) {
        if (c->ap_beam_h[k] != beam) continue;
        bool same = true;
        for (int r = 0; r < c->rows[beam] && same; ++r) {
            int L = lr[2 * r], R = lr[2 * r + 1];
            if (L == R) L = R = 0;
            same = c->ap_lr_h[(size_t)k * stride + 2 * r] == L && c->ap_lr_h[(size_t)k * stride + 2 * r + 1] == R;
        }
        if (same) return true;
    }
    return false;
}

// form the new column (Eq. 2) into slab column K, record the aperture
// The mask goes through the context's pinned staging block: the caller
// synchronises before the next call refills it.
dao_status add_column(dao_ctx* c, int beam, const int32_t* lr, float* out, int stride) {
    const int nb = c->rows[beam] * c->cols[beam];
    float* m = reinterpret_cast<float*>(c->pinned + c->off_mask);
    for (int i = 0; i < nb; ++i) m[i] = 0.f;
    for (int r = 0; r < c->rows[beam]; ++r)
        for (int q = lr[2 * r]; q < lr[2 * r + 1]; ++q) m[r * c->cols[beam] + q] = 1.f;
    DAO_CU(cudaMemcpyAsync(c->mask, m, sizeof(float) * nb, cudaMemcpyHostToDevice, c->stream));
    c->prof_begin(DAO_KC_COLUMN);
    DAO_CU(launch_column(c->D, c->seg, beam, c->beam_off[beam], nb, c->mask, out, stride, c->num_sms, c->stream,
                         &c->launches_i));
    c->prof_end();
    return DAO_OK;
}

// Column and table entry of aperture (beam, lr) at pool index K; no master solve.
dao_status append_aperture(dao_ctx* c, int beam, const int32_t* lr) {
    DAO_TRY(add_column(c, beam, lr, c->slab + (size_t)c->K * c->ld, 1));
    const int stride = 2 * c->max_rows;
    c->ap_beam_h.push_back(beam);
    c->ap_lr_h.resize((size_t)(c->K + 1) * stride, 0);
    for (int r = 0; r < c->rows[beam]; ++r) {
        int L = lr[2 * r], R = lr[2 * r + 1];
        if (L == R) L = R = 0;
        c->ap_lr_h[(size_t)c->K * stride + 2 * r] = L;
        c->ap_lr_h[(size_t)c->K * stride + 2 * r + 1] = R;
    }
    DAO_CU(cudaMemcpyAsync(c->ap_beam + c->K, &c->ap_beam_h[c->K], sizeof(int), cudaMemcpyHostToDevice, c->stream));
    DAO_CU(cudaMemcpyAsync(c->ap_lr + (size_t)c->K * stride, &c->ap_lr_h[(size_t)c->K * stride], sizeof(int) * stride,
                           cudaMemcpyHostToDevice, c->stream));
    c->K += 1;
    return DAO_OK;
}

dao_status add_aperture(dao_ctx* c, int beam, const int32_t* lr, double* F) {
    if (c->K >= c->K_cap) return fail(DAO_ESTATE, "aperture pool is full (k_max)");
    DAO_TRY(append_aperture(c, beam, lr));
    return master_solve(c, F);
}

// ---- graph-driven column generation ---------------------------------------------

// One round for pool size K as a CUDA graph: pricing (a2, a3), the device-side
// commit of the priced aperture, its column (a4), the master problem (a5) as a
// while node whose body is one evaluation, and the final pass.  Every node
// becomes a no-op once an earlier round has stopped the solve, so rounds can be
// queued without waiting on the host.
// Persistent variant: one captured sequence, the master solve one cooperative
// kernel node.
dao_status build_round_graph_persist(dao_ctx* c, int K) {
    cudaStream_t cs = c->stream;
    int n = 0;
    const int* stop = &c->cg->stop;  // D^T and pricing skip once the solve has stopped
    const int* skip = &c->cg->idle;  // the master solve skips a round that added nothing
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    auto check = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    if (e == cudaSuccess) {
        check(launch_dt(c->Dt, c->pi, c->w, stop, cs, &n));
        check(price_rows_any(c, c->w, stop, cs, &n));
        check(launch_price_commit(c->row_v, c->beam_row0_d, c->B, c->price, c->row_lr, c->rows_d, c->cols_d, c->tau,
                                  K, 2 * c->max_rows, c->ap_beam, c->ap_lr, c->mask, c->cg, cs, &n));
        check(launch_column_dev(c->D, c->seg, c->ap_beam, K, c->beam_off_d, c->rows_d, c->cols_d, c->max_nb, c->mask,
                                c->slab, c->ld, c->cg, c->num_sms, cs, &n));
        check(launch_master_persist(c->mb, c->slab, c->ld, c->V, K, c->vstruct, c->tf, c->S, c->opt.max_master_iters,
                                    c->opt.master_tol, skip, c->z, c->pi, c->cg, cs, &n));
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return fail(DAO_ECUDA, std::string("building the round graph: ") + cudaGetErrorString(e));
        }
        c->round_graph[K] = g;
        c->round_exec[K] = ex;
        return DAO_OK;
    }
    cudaGetLastError();
    return fail(DAO_ECUDA, std::string("building the round graph: ") + cudaGetErrorString(e));
}

// Every round of a solve in one graph: a while node whose body is
// ROUNDS_PER_ITER rounds of three kernels (D^T with the MLC-row search, the
// beam decision with the new aperture's column, the persistent master solve),
// which read the pool size from the device.  The decision kernel ends the loop
// when pricing stops the solve or the pool reaches cg->K_end.  Returns false
// (and leaves nothing behind) where the driver does not take this form.
constexpr int ROUNDS_PER_ITER = 4;

bool build_solve_graph_persist(dao_ctx* c) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaStream_t cs = c->stream;
    int n = 0;
    const int* skip = &c->cg->idle;
    cudaError_t e = cudaSuccess;
    auto check = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    cudaGraphConditionalHandle h = 0;
    check(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cnode = nullptr;
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        check(cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &cp));
    }
    if (e == cudaSuccess) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) {
            // ROUNDS_PER_ITER rounds per iteration: the while node's relaunch costs
            // about as much as a few kernels, and rounds after the stop return at entry
            // with an MLC constraint the D^T kernel only takes the round's snapshot, and
            // the beams are priced by their own kernel before the decision
            const bool mlc = c->opt.mlc_constraint != DAO_MLC_CONSECUTIVE;
            const RowTicket rt{c->binfo, c->beam_row0_d, c->cols_d, c->row_info, mlc ? nullptr : c->row_cnt,
                               c->row_v, c->row_lr, c->cg};
            CommitArgs ca{};
            ca.row_v = c->row_v;
            ca.row_lr = c->row_lr;
            ca.beam_row0 = c->beam_row0_d;
            ca.rows = c->rows_d;
            ca.cols = c->cols_d;
            ca.beam_off = c->beam_off_d;
            ca.seg = c->seg;
            ca.n_beams = c->B;
            ca.lr_stride = 2 * c->max_rows;
            ca.tau = c->tau;
            ca.ap_beam = c->ap_beam;
            ca.ap_lr = c->ap_lr;
            ca.slab = c->slab;
            ca.ld = c->ld;
            ca.cg = c->cg;
            ca.cond = h;
            ca.use_cond = 1;
            for (int u = 0; u < ROUNDS_PER_ITER; ++u) {
                check(launch_dt_rows(c->Dt, c->pi, c->w, rt, cs, &n));
                if (mlc) check(price_rows_any(c, c->w, &c->cg->stop, cs, &n));
                check(launch_commit_column(c->D, ca, c->max_nb, c->num_sms, cs, &n));
                check(launch_master_persist(c->mb, c->slab, c->ld, c->V, 0, c->vstruct, c->tf, c->S,
                                            c->opt.max_master_iters, c->opt.master_tol, skip, c->z, c->pi, c->cg,
                                            cs, &n));
            }
            cudaGraph_t out = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
            check(e2);
        }
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) check(cudaGraphInstantiate(&ex, g, 0));
    if (e != cudaSuccess) {
        cudaStreamCaptureStatus cst;
        if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
        }
        cudaGetLastError();
        cudaGraphDestroy(g);
        return false;
    }
    c->solve_graph = g;
    c->solve_exec = ex;
    return true;
}

dao_status build_round_graph(dao_ctx* c, int K) {
    if (c->mb.GP > 0) return build_round_graph_persist(c, K);
    cudaGraph_t g = nullptr;
    DAO_CU(cudaGraphCreate(&g, 0));
    cudaStream_t cs = c->stream;
    int n = 0;
    const int* stop = &c->cg->stop;
    const int* skip = &c->cg->idle;
    cudaError_t e = cudaSuccess;
    cudaGraphConditionalHandle h = 0;
    std::vector<cudaGraphNode_t> deps;
    cudaGraphNode_t cnode = nullptr;
    auto check = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    check(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    if (e == cudaSuccess) {
        check(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) {
            check(launch_dt(c->Dt, c->pi, c->w, stop, cs, &n));
            check(price_rows_any(c, c->w, stop, cs, &n));
            check(launch_price_commit(c->row_v, c->beam_row0_d, c->B, c->price, c->row_lr, c->rows_d, c->cols_d,
                                      c->tau, K, 2 * c->max_rows, c->ap_beam, c->ap_lr, c->mask, c->cg, cs, &n));
            check(launch_column_dev(c->D, c->seg, c->ap_beam, K, c->beam_off_d, c->rows_d, c->cols_d, c->max_nb,
                                    c->mask, c->slab, c->ld, c->cg, c->num_sms, cs, &n));
            check(launch_master_init(c->mb.st, K, skip, h, 1, cs, &n));
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t* d = nullptr;
            size_t nd = 0;
            check(cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &d, nullptr, &nd));
            if (e == cudaSuccess) deps.assign(d, d + nd);
            cudaGraph_t out = nullptr;
            check(cudaStreamEndCapture(cs, &out));
        }
    }
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        check(cudaGraphAddNode(&cnode, g, deps.data(), nullptr, deps.size(), &cp));
        if (e == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            check(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            if (e == cudaSuccess) {
                // two evaluations per iteration of the while node: the node's own
                // relaunch costs about as much as a kernel, and once the solve is
                // done the kernels of the second evaluation return at entry
                for (int u = 0; u < 2; ++u) {
                    check(launch_master_eval(c->mb, c->V, K, c->vstruct, c->tf, c->S, nullptr, nullptr, PASS_EVAL,
                                             nullptr, cs, &n));
                    check(launch_master_hess(c->mb, K, PASS_EVAL, cs, &n));
                    check(launch_master_step(K, c->mb, c->opt.max_master_iters, c->opt.master_tol, h, 1, cs, &n));
                }
                cudaGraph_t out = nullptr;
                check(cudaStreamEndCapture(cs, &out));
            }
        }
    }
    if (e == cudaSuccess) {
        check(cudaStreamBeginCaptureToGraph(cs, g, &cnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) {
            check(launch_master_eval(c->mb, c->V, K, c->vstruct, c->tf, c->S, c->z, c->pi, PASS_FINAL, skip, cs, &n));
            check(launch_cg_record(c->mb.st, c->cg, K, cs, &n));
            cudaGraph_t out = nullptr;
            check(cudaStreamEndCapture(cs, &out));
        }
    }
    cudaGraphExec_t ex = nullptr;
    if (e == cudaSuccess) check(cudaGraphInstantiate(&ex, g, 0));
    if (e != cudaSuccess) {
        cudaStreamCaptureStatus cst;
        if (cudaStreamIsCapturing(cs, &cst) == cudaSuccess && cst != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(cs, &junk);
        }
        cudaGetLastError();
        cudaGraphDestroy(g);
        return fail(DAO_ECUDA, std::string("building the round graph: ") + cudaGetErrorString(e));
    }
    c->round_graph[K] = g;
    c->round_exec[K] = ex;
    return DAO_OK;
}

// Rounds K_old+1 .. K_new queued back to back; one synchronisation at the end.
// Graph path in three parts so that a batch can interleave the launches of
// several contexts: prepare (graphs, device-side round state), launch one
// round, finish (read back, bookkeeping).
struct GraphSolve {
    int K0 = 0, K1 = 0;
};

// The device-side round state of a solve of rounds K0+1 .. K1 (copied on the
// context's stream); the barrier counter of the persistent master zeroed.
dao_status solve_state_begin(dao_ctx* c, const GraphSolve* gs);

dao_status solve_graph_begin(dao_ctx* c, int n_apertures, GraphSolve* gs) {
    gs->K0 = c->K;
    gs->K1 = std::min(c->K_cap, c->K + n_apertures);
    if (c->mb.GP > 0 && !c->solve_tried) {
        c->solve_tried = true;
        build_solve_graph_persist(c);  // else: one graph per round below
    }
    if (c->solve_exec == nullptr)
        for (int k = gs->K0 + 1; k <= gs->K1; ++k)
            if (c->round_exec[k] == nullptr) DAO_TRY(build_round_graph(c, k));
    return solve_state_begin(c, gs);
}

dao_status solve_state_begin(dao_ctx* c, const GraphSolve* gs) {
    CGDev* h = reinterpret_cast<CGDev*>(c->pinned + c->off_cg);
    h->K = gs->K0;
    h->done = 0;
    h->K_end = gs->K1;
    h->stop = 0;
    h->idle = 0;
    h->rs_K = gs->K0;
    h->rs_stop = 0;
    DAO_CU(cudaMemcpyAsync(c->cg, h, offsetof(CGDev, pad), cudaMemcpyHostToDevice, c->stream));
    DAO_CU(cudaMemsetAsync(c->mb.bar, 0, sizeof(GridBar), c->stream));  // barrier counter
    return DAO_OK;
}

// Round k (K0 < k <= K1) of a prepared solve; with the single solve graph the
// first round launches every round.
dao_status launch_round(dao_ctx* c, const GraphSolve& gs, int k) {
    if (k <= gs.K0 || k > gs.K1) return DAO_OK;
    if (c->solve_exec != nullptr) {
        if (k == gs.K0 + 1) DAO_CU(cudaGraphLaunch(c->solve_exec, c->stream));
        return DAO_OK;
    }
    DAO_CU(cudaGraphLaunch(c->round_exec[k], c->stream));
    return DAO_OK;
}

dao_status solve_graph_end(dao_ctx* c, const GraphSolve& gs, int n_apertures, int32_t* n_done, double* trace,
                           dao_status* result, bool count = true) {
    const int K0 = gs.K0, K1 = gs.K1;
    CGDev* h = reinterpret_cast<CGDev*>(c->pinned + c->off_cg);
    GridBar* hb = reinterpret_cast<GridBar*>(c->pinned + c->off_bar);
    DAO_CU(cudaMemcpyAsync(h, c->cg, sizeof(CGDev), cudaMemcpyDeviceToHost, c->stream));
    if (c->mb.GP > 0) DAO_CU(cudaMemcpyAsync(hb, c->mb.bar, sizeof(GridBar), cudaMemcpyDeviceToHost, c->stream));
    DAO_TRY(sync(c));
    // a barrier of a cooperative master solve gave up: the rounds after it returned
    // at entry, so the device pool no longer matches the host's
    if (c->mb.GP > 0 && hb->broken)
        return fail(DAO_ETIMEOUT, "a grid barrier of the master solve timed out; reset the plan");
    const int K = h->K;
    const int stride = 2 * c->max_rows;
    if (K > K0) {
        c->ap_beam_h.resize(K);
        c->ap_lr_h.resize((size_t)K * stride);
        DAO_CU(cudaMemcpy(c->ap_beam_h.data() + K0, c->ap_beam + K0, sizeof(int) * (K - K0), cudaMemcpyDeviceToHost));
        DAO_CU(cudaMemcpy(c->ap_lr_h.data() + (size_t)K0 * stride, c->ap_lr + (size_t)K0 * stride,
                          sizeof(int) * (size_t)(K - K0) * stride, cudaMemcpyDeviceToHost));
        for (int k = K0; k < K; ++k) {  // rows beyond the beam's own count are not part of the aperture
            const int b = c->ap_beam_h[k];
            for (int r = c->rows[b]; r < c->max_rows; ++r) {
                c->ap_lr_h[(size_t)k * stride + 2 * r] = 0;
                c->ap_lr_h[(size_t)k * stride + 2 * r + 1] = 0;
            }
        }
    }
    // kernels the graphs ran: per round D^T, row scans, argmin + commit, column, and then
    // the persistent solve, or init, the final pass, the record and, per pair of
    // evaluations, pass, curvature and reduce + step
    const bool persist = c->mb.GP > 0;
    if (!count) {
    } else if (c->solve_exec != nullptr) {
        // the while node ran the rounds that grew the pool and, when pricing
        // stopped the solve, the round that found it, ROUNDS_PER_ITER to an iteration
        const int rounds = K - K0 + (h->done != 0 ? 1 : 0);
        const int per_round = c->opt.mlc_constraint != DAO_MLC_CONSECUTIVE ? 4 : 3;
        c->launches_i += per_round * ROUNDS_PER_ITER * ((rounds + ROUNDS_PER_ITER - 1) / ROUNDS_PER_ITER);
    } else {
        // every queued round launches its kernels (a stopped solve's rounds return at entry)
        c->launches_i += (persist ? 5 : 7) * (K1 - K0);
    }
    for (int k = K0; k < K; ++k) {
        if (!persist && count) c->launches_i += 6 * ((h->evals[k] + 1) / 2);  // two evaluations per while iteration
        c->stat_evals.push_back(h->evals[k]);
        c->stat_status.push_back(h->status[k]);
        c->stat_kkt.push_back(h->res[k] / (h->tol[k] > 0 ? h->tol[k] / c->opt.master_tol : 1.0));
        if (trace) trace[k - K0] = h->trace[k];
    }
    c->K = K;
    if (n_done) *n_done = K;
    *result = h->done == 1 ? DAO_OPTIMAL : h->done == 2 ? DAO_DUPLICATE : DAO_OK;
    if (*result == DAO_OK && K0 + n_apertures > c->K_cap) *result = fail(DAO_ESTATE, "aperture pool is full (k_max)");
    return DAO_OK;
}

dao_status solve_graph(dao_ctx* c, int n_apertures, int32_t* n_done, double* trace, dao_status* result) {
    GraphSolve gs;
    DAO_TRY(solve_graph_begin(c, n_apertures, &gs));
    for (int k = gs.K0 + 1; k <= gs.K1; ++k) DAO_TRY(launch_round(c, gs, k));
    return solve_graph_end(c, gs, n_apertures, n_done, trace, result);
}

// Round graphs embed the launch shapes they were captured with: drop them when
// the shapes change.
void drop_round_graphs(dao_ctx* c) {
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    if (c->solve_graph) cudaGraphDestroy(c->solve_graph);
    c->solve_exec = nullptr;
    c->solve_graph = nullptr;
    c->solve_tried = false;
    for (size_t k = 0; k < c->round_exec.size(); ++k) {
        if (c->round_exec[k]) cudaGraphExecDestroy(c->round_exec[k]);
        if (c->round_graph[k]) cudaGraphDestroy(c->round_graph[k]);
        c->round_exec[k] = nullptr;
        c->round_graph[k] = nullptr;
    }
}

dao_status reset_state(dao_ctx* c) {
    c->K = 0;
    c->stat_evals.clear();
    c->stat_status.clear();
    c->stat_kkt.clear();
    c->ap_beam_h.clear();
    c->ap_lr_h.clear();
    DAO_CU(cudaMemsetAsync(c->mb.st, 0, sizeof(MasterDev), c->stream));
    DAO_TRY(refresh_state(c));
    DAO_TRY(sync(c));
    return DAO_OK;
}

}  // namespace

// ============================ internal hooks (serve.cu) ===========================
namespace dao {

dao_status check_inputs(const dao_csr* D, const dao_geometry* g, const dao_structures* s, const dao_weights* w,
                        const double* rx, const dao_options* opt) {
    dao_options o;
    dao_options_default(&o);
    if (opt) o = *opt;
    return validate(D, g, s, w, rx, &o);
}

dao_status solve_async_begin(dao_ctx* c, int n_apertures, cudaEvent_t done) {
    DAO_TRY(check_ctx(c));
    if (!c->opt.use_graphs || c->prof_on) return fail(DAO_EINVAL, "asynchronous solve needs use_graphs, profiling off");
    GraphSolve gs;
    DAO_TRY(solve_graph_begin(c, n_apertures, &gs));
    for (int k = gs.K0 + 1; k <= gs.K1; ++k) DAO_TRY(launch_round(c, gs, k));
    DAO_CU(cudaEventRecord(done, c->stream));
    c->async_K0 = gs.K0;
    c->async_K1 = gs.K1;
    return DAO_OK;
}

dao_status solve_async_end(dao_ctx* c, int n_apertures, int32_t* n_done, dao_status* result) {
    DAO_TRY(check_ctx(c));
    GraphSolve gs;
    gs.K0 = c->async_K0;
    gs.K1 = c->async_K1;
    DAO_TRY(solve_graph_end(c, gs, n_apertures, n_done, nullptr, result));
    c->count_launches();
    return DAO_OK;
}

}  // namespace dao

// ================================ C ABI ==========================================

extern "C" {

void dao_options_default(dao_options* opt) {
    if (!opt) return;
    opt->k_max = KMAX;
    opt->max_master_iters = 50;
    opt->master_tol = 1e-6;
    opt->price_tol = 1e-7;
    opt->precision = DAO_PREC_FP32;
    opt->device = 0;
    opt->stream = nullptr;
    opt->use_graphs = 1;
    opt->master_persistent = 1;
    opt->mlc_constraint = DAO_MLC_CONSECUTIVE;
    opt->master_blocks = 0;
    opt->dt_threads = 0;
    opt->dt_map = 0;
    opt->dose_form = 0;
    opt->column_lanes = 0;
    opt->split_warps = 0;
}

const char* dao_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {
dao_status create_common(const dao_csr* D, const dao_geometry* g, const dao_structures* s, const dao_weights* w,
                         const double* prescriptions, const dao_voxel_terms* vt, const dao_options* opt_in,
                         dao_ctx** out, const dao_pencil_beam* pb = nullptr) {
    if (!out) return fail(DAO_EINVAL, "null output pointer");
    *out = nullptr;
    dao_options opt;
    dao_options_default(&opt);
    if (opt_in) opt = *opt_in;
    DAO_TRY(validate(D, g, s, w, prescriptions, &opt));
    dao_ctx* c = new (std::nothrow) dao_ctx();
    if (!c) return fail(DAO_ENOMEM, "host allocation failed");
    {
        static std::atomic<uint64_t> next_uid{1};
        c->uid = next_uid++;
    }
    c->opt = opt;
    c->device = opt.device;
    c->V = D->n_voxels;
    c->N = D->n_beamlets;
    c->B = g->n_beams;
    c->nnz = D->nnz;
    dao_status st = DAO_OK;
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) st = fail(DAO_ECUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    if (st == DAO_OK) {
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
        if (opt.stream) {
            c->stream = static_cast<cudaStream_t>(opt.stream);
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) st = fail(DAO_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
            c->own_stream = true;
        }
    }
    if (st == DAO_OK) {
        e = master_configure();
        if (e == cudaSuccess) e = spmv_configure();
        if (e != cudaSuccess) st = fail(DAO_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
    }
    DeviceCSR gen;
    if (st == DAO_OK && pb) {  // D from the pencil-beam model, on the device
        TraceRange range("pencil-beam D");
        e = pencil_generate(pb, c->device, c->stream, &gen.rp, &gen.col, &gen.val, &gen.nnz);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = fail(e == cudaErrorMemoryAllocation ? DAO_ENOMEM : DAO_ECUDA,
                      std::string("pencil-beam generation: ") + cudaGetErrorString(e));
        }
        c->nnz = gen.nnz;
    }
    if (st == DAO_OK) st = build(c, D, g, s, w, prescriptions, vt, pb ? &gen : nullptr);
    for (void* q : {(void*)gen.rp, (void*)gen.col, (void*)gen.val})  // left over when build did not run
        if (q) pool_free(q, c->stream);
    if (st == DAO_OK) st = alloc_state(c);
    if (st == DAO_OK) st = reset_state(c);
    if (st != DAO_OK) {
        std::string keep = g_err;
        dao_destroy(c);
        g_err = keep;
        return st;
    }
    c->count_launches();
    *out = c;
    return DAO_OK;
}
}  // namespace

extern "C" {

dao_status dao_create(const dao_csr* D, const dao_geometry* g, const dao_structures* s, const dao_weights* w,
                      const double* prescriptions, const dao_options* opt_in, dao_ctx** out) {
    TraceRange trace("dao_create");
    return create_common(D, g, s, w, prescriptions, nullptr, opt_in, out);
}

dao_status dao_create_voxelwise(const dao_csr* D, const dao_geometry* g, const dao_voxel_terms* t,
                                const dao_options* opt_in, dao_ctx** out) {
    TraceRange trace("dao_create_voxelwise");
    if (!out) return fail(DAO_EINVAL, "null output pointer");
    *out = nullptr;
    if (!D || !t) return fail(DAO_EINVAL, "null argument");
    if (!t->under_w || !t->under_t || !t->over_w || !t->over_t) return fail(DAO_EINVAL, "null voxel term array");
    if (D->n_voxels < 1) return fail(DAO_EINVAL, "need at least one voxel and one beamlet");
    for (int j = 0; j < D->n_voxels; ++j) {
        if (!(t->under_w[j] >= 0) || !std::isfinite(t->under_w[j]) || !(t->over_w[j] >= 0) ||
            !std::isfinite(t->over_w[j]))
            return fail(DAO_EINVAL, "voxel weights must be finite and >= 0 (voxel " + std::to_string(j) + ")");
        if (!std::isfinite(t->under_t[j]) || !std::isfinite(t->over_t[j]))
            return fail(DAO_EINVAL, "voxel thresholds must be finite (voxel " + std::to_string(j) + ")");
    }
    // one structure that every voxel belongs to: the labels and per-structure
    // weights the common path checks; the terms themselves come from t
    std::vector<int32_t> labels((size_t)D->n_voxels, 0);
    const uint8_t tgt = 0;
    const double zero = 0.0;
    const dao_structures s{1, labels.data(), &tgt};
    const dao_weights w{&zero, &zero, &zero, 0};
    return create_common(D, g, &s, &w, &zero, t, opt_in, out);
}

dao_status dao_create_pencil(const dao_pencil_beam* pb, const dao_structures* s, const dao_weights* w,
                             const double* prescriptions, const dao_options* opt_in, dao_ctx** out) {
    TraceRange trace("dao_create_pencil");
    if (!out) return fail(DAO_EINVAL, "null output pointer");
    *out = nullptr;
    DAO_TRY(pencil_check(pb));
    std::vector<int32_t> rows(pb->n_beams, pb->rows), cols(pb->n_beams, pb->cols);
    const dao_geometry g{pb->n_beams, rows.data(), cols.data()};
    dao_csr D{};
    D.n_voxels = pb->n_voxels;
    D.n_beamlets = pb->n_beams * pb->rows * pb->cols;
    D.nnz = -1;  // generated on the device
    return create_common(&D, &g, s, w, prescriptions, nullptr, opt_in, out, pb);
}

dao_status dao_pencil_generate(const dao_pencil_beam* pb, int32_t device, int64_t* nnz, int64_t* row_ptr,
                               int32_t* col, float* val) {
    TraceRange trace("dao_pencil_generate");
    DAO_TRY(pencil_check(pb));
    int n = 0;
    DAO_CU(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(DAO_EINVAL, "no such device");
    DAO_CU(cudaSetDevice(device));
    cudaStream_t s = nullptr;
    DAO_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int64_t* rp = nullptr;
    int* c = nullptr;
    float* v = nullptr;
    int64_t m = 0;
    cudaError_t e = pencil_generate(pb, device, s, &rp, &c, &v, &m);
    if (e == cudaSuccess && row_ptr)
        e = cudaMemcpyAsync(row_ptr, rp, sizeof(int64_t) * ((size_t)pb->n_voxels + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && col && m > 0) e = cudaMemcpyAsync(col, c, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && val && m > 0) e = cudaMemcpyAsync(val, v, sizeof(float) * (size_t)m, cudaMemcpyDeviceToHost, s);
    for (void* q : {(void*)rp, (void*)c, (void*)v})
        if (q) pool_free(q, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return fail(DAO_ECUDA, std::string("dao_pencil_generate: ") + cudaGetErrorString(e));
    if (nnz) *nnz = m;
    return DAO_OK;
}

void dao_destroy(dao_ctx* c) {
    if (!c) return;
    batch_graphs_forget(c->uid);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_round_graphs(c);
    // back to the process-wide caches, ordered after the context's last work
    for (void* p : c->dev_allocs) pool_free(p, c->stream);
    for (cudaEvent_t ev : c->ev_pool) cudaEventDestroy(ev);
    if (c->pinned) pinned_release(c->pinned, c->pinned_block);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

dao_status dao_release_cached_memory(int32_t device) {
    int n = 0;
    DAO_CU(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(DAO_EINVAL, "no such device");
    DAO_CU(cudaSetDevice(device));
    DAO_CU(release_cached_memory(device));
    return DAO_OK;
}

dao_status dao_check_bounded_wait(int32_t device, int32_t* gave_up, int32_t* passed) {
    int n = 0;
    DAO_CU(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return fail(DAO_EINVAL, "no such device");
    DAO_CU(cudaSetDevice(device));
    cudaStream_t s = nullptr;
    DAO_CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    GridBar* gb = nullptr;
    int* out = nullptr;
    cudaError_t e = cudaMalloc(&gb, sizeof(GridBar));
    if (e == cudaSuccess) e = cudaMalloc(&out, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(gb, 0, sizeof(GridBar), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(out, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = launch_barrier_check(gb, 2, 0, out, s);
    int h[2] = {0, 0};
    GridBar hb{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hb, gb, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (out) cudaFree(out);
    if (gb) cudaFree(gb);
    cudaStreamDestroy(s);
    if (e != cudaSuccess) return fail(DAO_ECUDA, std::string("barrier check: ") + cudaGetErrorString(e));
    if (gave_up) *gave_up = h[0];
    if (passed) *passed = h[1];
    if (h[0] > 0 && hb.broken) return fail(DAO_ETIMEOUT, "a grid barrier wait gave up as bounded");
    return fail(DAO_ESTATE, "the bounded barrier wait did not give up");
}

dao_status dao_reset(dao_ctx* c) {
    DAO_TRY(check_ctx(c));
    dao_status st = reset_state(c);
    c->count_launches();
    return st;
}

dao_status dao_sizes(const dao_ctx* c, int32_t* V, int32_t* N, int32_t* B, int32_t* R, int32_t* max_rows,
                     int64_t* nnz_stored, int32_t* k_max) {
    if (!c) return fail(DAO_EINVAL, "null context");
    if (V) *V = c->V;
    if (N) *N = c->N;
    if (B) *B = c->B;
    if (R) *R = c->R_tot;
    if (max_rows) *max_rows = c->max_rows;
    if (nnz_stored) *nnz_stored = c->D.nnz_stored;
    if (k_max) *k_max = c->K_cap;
    return DAO_OK;
}

dao_status dao_price(dao_ctx* c, int32_t* beam, int32_t* leaf_lr, double* rc) {
    DAO_TRY(check_ctx(c));
    c->prof_begin(DAO_KC_DT);
    DAO_CU(launch_dt(c->Dt, c->pi, c->w, nullptr, c->stream, &c->launches_i));
    c->prof_end();
    double r = 0.0;
    dao_status st = price_on_w(c, c->w, beam, leaf_lr, &r, nullptr, nullptr);
    c->count_launches();
    if (st != DAO_OK) return st;
    if (rc) *rc = r;
    return r < -c->tau ? DAO_OK : DAO_OPTIMAL;
}

dao_status dao_import_apertures(dao_ctx* c, int32_t n, const int32_t* beams, const int32_t* leaf_lr,
                                const double* y_start, double* objective) {
    TraceRange range("dao_import_apertures");
    DAO_TRY(check_ctx(c));
    if (n < 0 || (n > 0 && (beams == nullptr || leaf_lr == nullptr)))
        return fail(DAO_EINVAL, "n >= 0 apertures with their beams and leaves");
    if (c->K + n > c->K_cap) return fail(DAO_ESTATE, "aperture pool is full (k_max)");
    const int stride = 2 * c->max_rows;
    for (int i = 0; i < n; ++i) {  // all checked before the pool changes
        DAO_TRY(validate_aperture(c, beams[i], leaf_lr + (size_t)i * stride));
        if (y_start != nullptr && !(y_start[i] >= 0.0 && std::isfinite(y_start[i])))
            return fail(DAO_EINVAL, "starting intensities must be finite and >= 0");
    }
    const int K0 = c->K;
    for (int i = 0; i < n; ++i) {
        DAO_TRY(append_aperture(c, beams[i], leaf_lr + (size_t)i * stride));
        DAO_TRY(sync(c));  // the column's mask is staged in one pinned buffer, refilled by the next aperture
    }
    if (n > 0) {
        // the master starts from y_start on the imported apertures (the last at 0,
        // as for every added aperture) and from the current optimum on the rest
        std::vector<double> y0(n, 0.0);
        if (y_start != nullptr) y0.assign(y_start, y_start + n);
        DAO_CU(cudaMemcpyAsync(c->mb.st->y + K0, y0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        const dao_status st = master_solve(c, objective);
        c->count_launches();
        return st;
    }
    return DAO_OK;  // n = 0: nothing changes, *objective is not written
}

dao_status dao_add_aperture(dao_ctx* c, int32_t beam, const int32_t* leaf_lr, double* objective) {
    DAO_TRY(check_ctx(c));
    DAO_TRY(validate_aperture(c, beam, leaf_lr));
    dao_status st = add_aperture(c, beam, leaf_lr, objective);
    c->count_launches();
    return st;
}

dao_status dao_solve(dao_ctx* c, int32_t n_apertures, int32_t* n_done, double* trace) {
    TraceRange range("dao_solve");
    DAO_TRY(check_ctx(c));
    if (n_apertures < 0) return fail(DAO_EINVAL, "negative aperture count");
    if (c->opt.use_graphs && !c->prof_on) {
        if (c->K >= c->K_cap && n_apertures > 0) return fail(DAO_ESTATE, "aperture pool is full (k_max)");
        dao_status result = DAO_OK;
        dao_status st = solve_graph(c, n_apertures, n_done, trace, &result);
        c->count_launches();
        return st != DAO_OK ? st : result;
    }
    std::vector<int32_t> lr(2 * c->max_rows);
    dao_status result = DAO_OK;
    for (int k = 0; k < n_apertures; ++k) {
        if (c->K >= c->K_cap) {
            result = fail(DAO_ESTATE, "aperture pool is full (k_max)");
            break;
        }
        c->prof_begin(DAO_KC_DT);
        DAO_CU(launch_dt(c->Dt, c->pi, c->w, nullptr, c->stream, &c->launches_i));
        c->prof_end();
        int32_t beam = 0;
        double rc = 0.0;
        DAO_TRY(price_on_w(c, c->w, &beam, lr.data(), &rc, nullptr, nullptr));
        if (!(rc < -c->tau)) {
            result = DAO_OPTIMAL;
            break;
        }
        if (is_duplicate(c, beam, lr.data())) {
            result = DAO_DUPLICATE;
            break;
        }
        double F = 0.0;
        DAO_TRY(add_aperture(c, beam, lr.data(), &F));
        if (trace) trace[k] = F;
    }
    if (n_done) *n_done = c->K;
    c->count_launches();
    return result;
}

dao_status dao_dose(dao_ctx* c, float* dose, double* objective) {
    TraceRange range("dao_dose");
    DAO_TRY(check_ctx(c));
    DAO_CU(launch_fluence(c->ap_beam, c->ap_lr, 2 * c->max_rows, c->mb.st->y, c->K, c->binfo, c->N, c->x, c->stream,
                          &c->launches_i));
    c->prof_begin(DAO_KC_DOSE);
    DAO_CU(launch_dose(c->D, c->x, c->vstruct, c->tf, c->ts, c->S, c->dose, nullptr, c->F_part, c->F_blocks, c->F_dev,
                       c->num_sms, c->stream, &c->launches_i));
    c->prof_end();
    double* f = reinterpret_cast<double*>(c->pinned + c->off_small + 8);
    DAO_CU(cudaMemcpyAsync(f, c->F_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if (dose) DAO_CU(cudaMemcpyAsync(dose, c->dose, sizeof(float) * c->V, cudaMemcpyDeviceToHost, c->stream));
    DAO_TRY(sync(c));
    if (objective) *objective = *f;
    c->count_launches();
    return DAO_OK;
}

dao_status dao_intensities(dao_ctx* c, double* y, int32_t* k) {
    DAO_TRY(check_ctx(c));
    if (y && c->K > 0) {
        DAO_CU(cudaMemcpyAsync(y, c->mb.st->y, sizeof(double) * c->K, cudaMemcpyDeviceToHost, c->stream));
        DAO_TRY(sync(c));
    }
    if (k) *k = c->K;
    return DAO_OK;
}

dao_status dao_apertures(dao_ctx* c, int32_t* beams, int32_t* leaf_lr, int32_t* k) {
    if (!c) return fail(DAO_EINVAL, "null context");
    if (beams) std::memcpy(beams, c->ap_beam_h.data(), sizeof(int) * c->K);
    if (leaf_lr) std::memcpy(leaf_lr, c->ap_lr_h.data(), sizeof(int) * c->K * 2 * c->max_rows);
    if (k) *k = c->K;
    return DAO_OK;
}

dao_status dao_fmo(dao_ctx* c, int32_t max_iters, double tol, double* x_out, double* objective, int32_t* iters,
                   int32_t* cg_iters) {
    TraceRange range("dao_fmo");
    DAO_TRY(check_ctx(c));
    if (max_iters < 1 || !(tol > 0)) return fail(DAO_EINVAL, "max_iters >= 1 and tol > 0 are required");
    const int N = c->N, V = c->V;
    if (c->fst == nullptr) {
        DAO_TRY(c->dalloc(&c->fx, N));
        DAO_TRY(c->dalloc(&c->fxt, N));
        DAO_TRY(c->dalloc(&c->fr, N));
        DAO_TRY(c->dalloc(&c->fp, N));
        DAO_TRY(c->dalloc(&c->fdF, N));
        DAO_TRY(c->dalloc(&c->fx32, N));
        DAO_TRY(c->dalloc(&c->fp32, N));
        DAO_TRY(c->dalloc(&c->fg, N));
        DAO_TRY(c->dalloc(&c->fAp, N));
        DAO_TRY(c->dalloc(&c->ffree, N));
        DAO_TRY(c->dalloc(&c->fz, V));
        DAO_TRY(c->dalloc(&c->fzt, V));
        DAO_TRY(c->dalloc(&c->fpi, V));
        DAO_TRY(c->dalloc(&c->fpit, V));
        DAO_TRY(c->dalloc(&c->fu, V));
        DAO_TRY(c->dalloc(&c->fst, 1));
    }
    cudaStream_t s = c->stream;
    FmoScalars* h = reinterpret_cast<FmoScalars*>(c->pinned + c->off_master);  // the master shadow is idle here
    double* hF = reinterpret_cast<double*>(c->pinned + c->off_small + 8);
    int* n = &c->launches_i;
    // F, z and pi of x: the a1 kernel with its epilogue; g = D^T pi: the a2 kernel
    auto evaluate = [&](const float* x32, float* z, float* pi) -> dao_status {
        DAO_CU(launch_dose(c->D, x32, c->vstruct, c->tf, c->ts, c->S, z, pi, c->F_part, c->F_blocks, c->F_dev,
                           c->num_sms, s, n));
        DAO_CU(cudaMemcpyAsync(hF, c->F_dev, sizeof(double), cudaMemcpyDeviceToHost, s));
        return DAO_OK;
    };
    auto read_scalars = [&]() -> dao_status {
        DAO_CU(cudaMemcpyAsync(h, c->fst, sizeof(FmoScalars), cudaMemcpyDeviceToHost, s));
        return sync(c);
    };
    DAO_CU(cudaMemsetAsync(c->fx, 0, sizeof(double) * N, s));
    DAO_CU(cudaMemsetAsync(c->fx32, 0, sizeof(float) * N, s));
    // g = D^T pi, its rounding scale D^T |pi| (into the CG's Ap buffer) and the KKT test
    auto gradient = [&]() -> dao_status {
        DAO_CU(launch_dt(c->Dt, c->fpi, c->fg, nullptr, s, n));
        DAO_CU(fmo_abs(V, c->fpi, c->fu, c->num_sms, s));
        ++*n;
        DAO_CU(launch_dt(c->Dt, c->fu, c->fAp, nullptr, s, n));
        DAO_CU(fmo_kkt(N, c->fx, c->fg, c->fAp, c->fst, s));
        ++*n;
        return read_scalars();
    };
    DAO_TRY(evaluate(c->fx32, c->fz, c->fpi));
    DAO_TRY(gradient());
    double F = *hF;
    const double res0 = h->res;
    double res = res0, res_x = h->res_x;
    int it = 0, cg_total = 0;
    constexpr int CG_BATCH = 8, CG_MAX = 400;
    for (; it < max_iters && res_x > tol * res0; ++it) {
        const double eps = std::min(1e-3, res), eta = std::min(0.1, std::sqrt(res / res0));
        DAO_CU(fmo_cg_init(N, c->fx, c->fg, eps, eta, c->ffree, c->fr, c->fp, c->fp32, c->fdF, c->fst, s));
        // CG on the free beamlets: u = D p, u *= h(z), Ap = D^T u; batches of
        // CG_BATCH iterations between reads of the stop flag (after it the
        // SpMVs run on p = 0 and the step kernel returns at entry)
        for (int k = 0; k < CG_MAX; k += CG_BATCH) {
            for (int q = 0; q < CG_BATCH; ++q) {
                DAO_CU(launch_dose(c->D, c->fp32, c->vstruct, c->tf, c->ts, c->S, c->fu, nullptr, nullptr, 0,
                                   nullptr, c->num_sms, s, n));
                DAO_CU(fmo_hmul(V, c->fz, c->fu, c->vstruct, c->tf, c->S, c->num_sms, s));
                ++*n;
                DAO_CU(launch_dt(c->Dt, c->fu, c->fAp, nullptr, s, n));
                DAO_CU(fmo_cg_step(N, c->fAp, c->ffree, c->fr, c->fp, c->fp32, c->fdF, c->fst, s));
                ++*n;
            }
            DAO_TRY(read_scalars());
            if (h->cg_done) break;
        }
        cg_total += h->cg_iters;
        // Armijo rule along the projection arc
        bool accepted = false;
        double a = 1.0;
        for (int ls = 0; ls < 60 && !accepted; ++ls, a *= 0.5) {
            DAO_CU(fmo_trial(N, c->fx, c->fg, c->ffree, c->fdF, a, c->fxt, c->fx32, c->fst, s));
            ++*n;
            DAO_TRY(evaluate(c->fx32, c->fzt, c->fpit));
            DAO_TRY(read_scalars());
            accepted = *hF <= F + 1e-4 * h->gdx;
        }
        if (!accepted) break;  // no decrease along the arc: the FP32 noise floor
        F = *hF;
        std::swap(c->fx, c->fxt);
        std::swap(c->fz, c->fzt);
        std::swap(c->fpi, c->fpit);
        DAO_TRY(gradient());
        res = h->res;
        res_x = h->res_x;
    }
    if (x_out) {
        DAO_CU(cudaMemcpyAsync(x_out, c->fx, sizeof(double) * N, cudaMemcpyDeviceToHost, s));
        DAO_TRY(sync(c));
    }
    if (objective) *objective = F;
    if (iters) *iters = it;
    if (cg_iters) *cg_iters = cg_total;
    c->count_launches();
    return res_x <= tol * res0 ? DAO_OK : DAO_ESTATE;
}

dao_status dao_k_dose(dao_ctx* c, const float* x, float* z, float* grad, double* objective) {
    DAO_TRY(check_ctx(c));
    if (!x || !z) return fail(DAO_EINVAL, "null vector");
    c->prof_begin(DAO_KC_DOSE);
    DAO_CU(launch_dose(c->D, x, c->vstruct, c->tf, c->ts, c->S, z, grad, objective ? c->F_part : nullptr, c->F_blocks,
                       c->F_dev, c->num_sms, c->stream, &c->launches_i));
    c->prof_end();
    if (objective) {
        double* f = reinterpret_cast<double*>(c->pinned + c->off_small + 8);
        DAO_CU(cudaMemcpyAsync(f, c->F_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        DAO_TRY(sync(c));
        *objective = *f;
    } else {
        DAO_TRY(sync(c));
    }
    c->count_launches();
    return DAO_OK;
}

dao_status dao_k_beamlet_prices(dao_ctx* c, const float* pi, float* w) {
    DAO_TRY(check_ctx(c));
    if (!pi || !w) return fail(DAO_EINVAL, "null vector");
    c->prof_begin(DAO_KC_DT);
    DAO_CU(launch_dt(c->Dt, pi, w, nullptr, c->stream, &c->launches_i));
    c->prof_end();
    DAO_TRY(sync(c));
    c->count_launches();
    return DAO_OK;
}

dao_status dao_k_price(dao_ctx* c, const float* w, int32_t* beam, int32_t* leaf_lr, double* rc, double* row_best,
                       int32_t* row_lr) {
    DAO_TRY(check_ctx(c));
    if (!w) return fail(DAO_EINVAL, "null vector");
    double r = 0.0;
    dao_status st = price_on_w(c, w, beam, leaf_lr, &r, row_best, row_lr);
    c->count_launches();
    if (st != DAO_OK) return st;
    if (rc) *rc = r;
    return r < -c->tau ? DAO_OK : DAO_OPTIMAL;
}

dao_status dao_k_aperture_column(dao_ctx* c, int32_t beam, const int32_t* leaf_lr, float* out) {
    DAO_TRY(check_ctx(c));
    DAO_TRY(validate_aperture(c, beam, leaf_lr));
    if (!out) return fail(DAO_EINVAL, "null vector");
    DAO_TRY(add_column(c, beam, leaf_lr, out, 1));
    DAO_TRY(sync(c));
    c->count_launches();
    return DAO_OK;
}

dao_status dao_k_state(dao_ctx* c, float* z, float* pi) {
    DAO_TRY(check_ctx(c));
    if (z) DAO_CU(cudaMemcpyAsync(z, c->z, sizeof(float) * c->V, cudaMemcpyDeviceToDevice, c->stream));
    if (pi) DAO_CU(cudaMemcpyAsync(pi, c->pi, sizeof(float) * c->V, cudaMemcpyDeviceToDevice, c->stream));
    DAO_TRY(sync(c));
    return DAO_OK;
}

}  // extern "C"

namespace {
// One launch of kernel class kc for dao_k_time.
cudaError_t time_one(dao_ctx* c, int kc, int K, cudaStream_t s, int* n) {
    switch (kc) {
        case DAO_KC_MASTER_PASS:
            return launch_master_eval(c->mb, c->V, K, c->vstruct, c->tf, c->S, nullptr, nullptr, PASS_TIMING, nullptr,
                                      s, n);
        case DAO_KC_MASTER_HESS:
            return launch_master_hess(c->mb, K, PASS_TIMING, s, n);
        case DAO_KC_DT:
            return launch_dt(c->Dt, c->pi, c->w, nullptr, s, n);
        case DAO_KC_DOSE:
            return launch_dose(c->D, c->x, c->vstruct, c->tf, c->ts, c->S, c->dose, nullptr, nullptr, 0, nullptr,
                               c->num_sms, s, n);
        case DAO_KC_COLUMN: {
            const int b = c->ap_beam_h[0];
            return launch_column(c->D, c->seg, b, c->beam_off[b], c->rows[b] * c->cols[b], c->mask, c->dose, 1,
                                 c->num_sms, s, n);
        }
        case DAO_KC_PRICE:
            return price_any(c, c->w, nullptr, s, n);
    }
    return cudaErrorInvalidValue;
}
// Average microseconds of one launch: reps launches captured into a CUDA graph
// (so that they run back to back on the device, without host launch gaps), one
// warm replay, one replay timed with events on the context's stream.
template <class F>
dao_status time_graph(dao_ctx* c, int reps, F&& launch, double* us, const char* what) {
    DAO_TRY(sync(c));
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    int n = 0;
    DAO_CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch(&n);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    cudaEvent_t e0 = c->event(), e1 = c->event();
    float ms = 0.f;
    if (e == cudaSuccess && (!e0 || !e1)) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->stream);  // warm
    if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    if (e0 && e1) c->ev_used -= 2;
    if (e != cudaSuccess) return fail(DAO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    c->launches_i += 2 * n;
    c->count_launches();
    *us = 1e3 * ms / reps;
    return DAO_OK;
}

// Cold timing of `launch` as the plan meets it: before each of reps launches a
// read of a buffer twice the L2 size (clean lines only) leaves none of the
// kernel's data in L2; the median of the per-launch event times (graph replay,
// external event records).  The buffer is stream-ordered pool memory, freed
// before the return.
template <class F>
dao_status time_cold(dao_ctx* c, int reps, F&& launch, double* us, const char* what) {
    DAO_TRY(sync(c));
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) != cudaSuccess || l2 <= 0) {
        cudaGetLastError();
        l2 = 128 << 20;
    }
    const size_t fbytes = (size_t)2 * l2;
    void* flush = nullptr;
    DAO_CU(pool_alloc(&flush, fbytes, c->device, c->stream));
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    int n = 0;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = launch_l2_evict(flush, fbytes, c->w, c->num_sms, c->stream);
            if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2 * r], c->stream, cudaEventRecordExternal);
            if (e == cudaSuccess) e = launch(&n);
            if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2 * r + 1], c->stream, cudaEventRecordExternal);
        }
        const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    std::vector<float> ms(reps, 0.f);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaEventElapsedTime(&ms[r], ev[2 * r], ev[2 * r + 1]);
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    pool_free(flush, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DAO_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
    }
    c->launches_i += 2 * n;
    c->count_launches();
    std::sort(ms.begin(), ms.end());
    *us = 1e3 * ms[reps / 2];
    return DAO_OK;
}

// Autotuner cache key: device, storage and the size class of the problem
// (log2 buckets of voxels, beamlets and the mean row lengths of D and D^T).
std::string tune_key(const dao_ctx* c) {
    cudaDeviceProp prop;
    std::string dev = cudaGetDeviceProperties(&prop, c->device) == cudaSuccess ? prop.name : "unknown";
    for (char& ch : dev)
        if (ch == ' ' || ch == '\t') ch = '_';
    auto lb = [](double v) { return (int)std::lround(std::log2(std::max(v, 1.0))); };
    const double row_d = c->V > 0 ? (double)c->nnz / c->V : 0.0, row_t = c->N > 0 ? (double)c->nnz / c->N : 0.0;
    return dev + "|prec=" + std::to_string(c->opt.precision) + "|V=" + std::to_string(lb(c->V)) + "|N=" +
           std::to_string(lb(c->N)) + "|rowD=" + std::to_string(lb(row_d)) + "|rowDt=" + std::to_string(lb(row_t)) +
           "|cold|forms";
}

// One line per choice: "key dose_lanes column_lanes dt_threads dose_form dt_map".
bool tune_cache_read(const char* path, const std::string& key, int* dose_g, int* col_g, int* dt_t, int* form,
                     int* map) {
    if (!path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {  // the last entry for a key wins
        char k[400];
        int a = 0, b = 0, t = 0, fm = 0, mp = 0;
        if (std::sscanf(line, "%399s %d %d %d %d %d", k, &a, &b, &t, &fm, &mp) == 6 && key == k) {
            *dose_g = a;
            *col_g = b;
            *dt_t = t;
            *form = fm;
            *map = mp;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

template <size_t M>
bool tune_allowed(const int (&set)[M], int v) {
    for (size_t i = 0; i < M; ++i)
        if (set[i] == v) return true;
    return false;
}

}  // namespace

extern "C" {

dao_status dao_k_time(dao_ctx* c, int32_t kc, int32_t K, int32_t reps, double* us_per_launch) {
    DAO_TRY(check_ctx(c));
    if (reps < 1 || !us_per_launch) return fail(DAO_EINVAL, "reps must be >= 1 and the output non-null");
    if ((kc == DAO_KC_MASTER_PASS || kc == DAO_KC_MASTER_HESS) && (K < 1 || K > c->K))
        return fail(DAO_EINVAL, "master kernel timing needs 1 <= K <= the current pool size");
    if (kc == DAO_KC_COLUMN && c->K < 1) return fail(DAO_EINVAL, "column timing needs an aperture in the pool");
    if (kc != DAO_KC_MASTER_PASS && kc != DAO_KC_MASTER_HESS && kc != DAO_KC_DT && kc != DAO_KC_DOSE &&
        kc != DAO_KC_COLUMN && kc != DAO_KC_PRICE)
        return fail(DAO_EINVAL, "kernel class cannot be timed on its own");
    double us = 0.0;
    DAO_TRY(time_graph(c, reps, [&](int* n) { return time_one(c, kc, K, c->stream, n); }, &us, "dao_k_time"));
    *us_per_launch = us;
    return DAO_OK;
}

dao_status dao_k_time_cold(dao_ctx* c, int32_t kc, int32_t K, int32_t reps, void* flush, int64_t flush_bytes,
                           double* us_median) {
    DAO_TRY(check_ctx(c));
    if (reps < 1 || reps > 1024 || !us_median || !flush || flush_bytes < 1)
        return fail(DAO_EINVAL, "reps in [1, 1024], a flush buffer and an output are required");
    if (kc == DAO_KC_MASTER_PASS || kc == DAO_KC_MASTER_HESS || kc == DAO_KC_COLUMN ||
        (kc != DAO_KC_DT && kc != DAO_KC_DOSE && kc != DAO_KC_PRICE))
        return fail(DAO_EINVAL, "cold timing covers DAO_KC_DOSE, DAO_KC_DT and DAO_KC_PRICE");
    DAO_TRY(sync(c));
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreate(&x);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    int n = 0;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // per repetition: read a buffer larger than L2 (clean lines only, so no
        // write-back overlaps the kernel), then the kernel between two events
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
            e = launch_l2_evict(flush, (size_t)flush_bytes, c->w, c->num_sms, c->stream);
            // external records: event nodes that the host can time after the replay
            if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2 * r], c->stream, cudaEventRecordExternal);
            if (e == cudaSuccess) e = time_one(c, kc, K, c->stream, &n);
            if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev[2 * r + 1], c->stream, cudaEventRecordExternal);
        }
        cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(ex, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    std::vector<float> ms(reps, 0.f);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = cudaEventElapsedTime(&ms[r], ev[2 * r], ev[2 * r + 1]);
    if (ex) cudaGraphExecDestroy(ex);
    if (g) cudaGraphDestroy(g);
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    if (e != cudaSuccess) return fail(DAO_ECUDA, std::string("dao_k_time_cold: ") + cudaGetErrorString(e));
    c->launches_i += n;
    c->count_launches();
    std::sort(ms.begin(), ms.end());
    *us_median = 1e3 * (reps % 2 ? ms[reps / 2] : 0.5 * (ms[reps / 2 - 1] + ms[reps / 2]));
    return DAO_OK;
}

dao_status dao_profile_enable(dao_ctx* c, int32_t enable) {
    DAO_TRY(check_ctx(c));
    DAO_TRY(sync(c));
    c->prof_on = enable != 0;
    c->recs.clear();
    c->ev_used = 0;
    return DAO_OK;
}

dao_status dao_profile_read(dao_ctx* c, int32_t kc, int64_t* launches, double* total_ms) {
    DAO_TRY(check_ctx(c));
    if (kc < 0 || kc >= DAO_KC_COUNT) return fail(DAO_EINVAL, "unknown kernel class");
    DAO_TRY(sync(c));
    int64_t n = 0;
    double ms = 0.0;
    for (const ProfRecord& r : c->recs) {
        if (r.kc != kc) continue;
        float t = 0.f;
        DAO_CU(cudaEventElapsedTime(&t, r.start, r.stop));
        ms += t;
        n += r.launches;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = ms;
    return DAO_OK;
}

int64_t dao_launch_count(const dao_ctx* c) { return c ? c->launches_total + c->launches_i : 0; }

dao_status dao_master_stats(const dao_ctx* c, int32_t* evals, int32_t* status, double* kkt, int32_t* k) {
    if (!c) return fail(DAO_EINVAL, "null context");
    const int n = (int)c->stat_evals.size();
    for (int i = 0; i < n; ++i) {
        if (evals) evals[i] = c->stat_evals[i];
        if (status) status[i] = c->stat_status[i];
        if (kkt) kkt[i] = c->stat_kkt[i];
    }
    if (k) *k = n;
    return DAO_OK;
}

dao_status dao_batch_solve(dao_ctx* const* ctxs, int32_t n, int32_t n_apertures, int32_t* n_done, double* traces,
                           int32_t* status) {
    TraceRange range("dao_batch_solve");
    if (n < 0 || n_apertures < 0 || (n > 0 && ctxs == nullptr))
        return fail(DAO_EINVAL, "dao_batch_solve: n >= 0, n_apertures >= 0 and a context array are required");
    for (int i = 0; i < n; ++i) {
        if (ctxs[i] == nullptr) return fail(DAO_EINVAL, "dao_batch_solve: null context " + std::to_string(i));
        if (!ctxs[i]->opt.use_graphs || ctxs[i]->prof_on)
            return fail(DAO_EINVAL, "dao_batch_solve: every context needs use_graphs and profiling off");
        if (ctxs[i]->device != ctxs[0]->device)
            return fail(DAO_EINVAL, "dao_batch_solve: the contexts must be on one device");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(DAO_EINVAL, "dao_batch_solve: context listed twice");
    }
    if (n == 0) return DAO_OK;
    DAO_TRY(check_ctx(ctxs[0]));
    std::vector<GraphSolve> gs(n);
    std::vector<char> run(n, 0);
    int rounds = 0;
    for (int i = 0; i < n; ++i) {
        dao_ctx* c = ctxs[i];
        if (status) status[i] = DAO_OK;
        if (n_done) n_done[i] = c->K;
        if (c->K >= c->K_cap && n_apertures > 0) {
            if (status) status[i] = DAO_ESTATE;
            continue;
        }
        DAO_TRY(solve_graph_begin(c, n_apertures, &gs[i]));
        run[i] = 1;
        rounds = std::max(rounds, gs[i].K1 - gs[i].K0);
    }
    // interleaved: round r of every instance before round r + 1 of any, each on
    // its own stream, so that the GPU overlaps the instances' kernels
    for (int r = 0; r < rounds; ++r)
        for (int i = 0; i < n; ++i) {
            if (!run[i]) continue;
            const int k = gs[i].K0 + 1 + r;
            DAO_TRY(launch_round(ctxs[i], gs[i], k));
        }
    for (int i = 0; i < n; ++i) {
        if (!run[i]) continue;
        dao_status res = DAO_OK;
        DAO_TRY(solve_graph_end(ctxs[i], gs[i], n_apertures, n_done ? n_done + i : nullptr,
                                traces ? traces + (size_t)i * n_apertures : nullptr, &res));
        ctxs[i]->count_launches();
        if (status) status[i] = res;
    }
    return DAO_OK;
}

}  // extern "C"

// ---- batched plans with one persistent master launch per round -----------------
namespace {

// An instantiated graph of R unrolled rounds over a fixed list of contexts:
// per round every plan's D^T kernel (with its MLC-row search) and beam
// decision with the new column on the plan's own stream, then all the plans'
// master solves in one cooperative launch (GB blocks each).
struct BatchGraph {
    std::vector<uint64_t> key;  // the contexts' ids, then R
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    MasterTask* tasks = nullptr;  // device copies of the plans' master tasks
    std::vector<cudaEvent_t> events;
    int GB = 0;
};
std::mutex g_batch_mu;
std::vector<BatchGraph*> g_batch_graphs;  // most recently used first
constexpr size_t BATCH_GRAPHS_KEPT = 4;

void batch_graph_free(BatchGraph* bg) {
    cudaSetDevice(bg->device);
    if (bg->stream) cudaStreamSynchronize(bg->stream);
    if (bg->exec) cudaGraphExecDestroy(bg->exec);
    if (bg->graph) cudaGraphDestroy(bg->graph);
    if (bg->tasks) pool_free(bg->tasks, bg->stream);
    for (cudaEvent_t e : bg->events) cudaEventDestroy(e);
    if (bg->stream) {
        cudaStreamSynchronize(bg->stream);
        cudaStreamDestroy(bg->stream);
    }
    delete bg;
}

// Graphs that name a context are dropped with it.
void batch_graphs_forget(uint64_t uid) {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batch_graphs.size();) {
        BatchGraph* bg = g_batch_graphs[i];
        if (std::find(bg->key.begin(), bg->key.end() - 1, uid) != bg->key.end() - 1) {
            batch_graph_free(bg);
            g_batch_graphs.erase(g_batch_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

dao_status build_batch_graph(dao_ctx* const* ctxs, int n, int R, BatchGraph* bg) {
    dao_ctx* c0 = ctxs[0];
    bg->device = c0->device;
    bg->GB = master_batch_group(n, c0->num_sms);
    if (bg->GB < 1) return fail(DAO_EINVAL, "too many plans for one persistent launch (two blocks per SM each)");
    DAO_CU(cudaStreamCreateWithFlags(&bg->stream, cudaStreamNonBlocking));
    std::vector<MasterTask> tasks(n);
    int max_V = 0;
    for (int i = 0; i < n; ++i) {
        dao_ctx* c = ctxs[i];
        MasterTask& t = tasks[i];
        t = MasterTask{};
        t.slab = c->slab;
        t.ld = c->ld;
        t.V = c->V;
        t.GS = c->mb.GH;
        t.S = c->S;
        t.max_iter = c->opt.max_master_iters;
        t.st = c->mb.st;
        t.gb = c->mb.bar;
        t.H_part = c->mb.H_part;
        t.g_part = c->mb.g_part;
        t.gn_part = c->mb.gn_part;
        t.F_part = c->mb.F_part;
        t.vstruct = c->vstruct;
        t.tf = c->tf;
        t.tol_rel = c->opt.master_tol;
        t.skip = &c->cg->idle;
        t.z_out = c->z;
        t.pi_out = c->pi;
        t.cg = c->cg;
        t.tmap[0] = c->mb.tmap_p[0];
        t.tmap[1] = c->mb.tmap_p[1];
        t.vstate = c->mb.vstate;
        t.H_keep = c->mb.H_keep;
        max_V = std::max(max_V, c->V);
    }
    void* tp = nullptr;
    DAO_CU(pool_alloc(&tp, sizeof(MasterTask) * n, bg->device, bg->stream));
    bg->tasks = static_cast<MasterTask*>(tp);
    DAO_CU(cudaMemcpyAsync(bg->tasks, tasks.data(), sizeof(MasterTask) * n, cudaMemcpyHostToDevice, bg->stream));
    DAO_CU(cudaStreamSynchronize(bg->stream));
    bg->events.assign(n + 1, nullptr);
    for (auto& e : bg->events) DAO_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaError_t e = cudaStreamBeginCapture(bg->stream, cudaStreamCaptureModeThreadLocal);
    auto check = [&](cudaError_t x) {
        if (e == cudaSuccess && x != cudaSuccess) e = x;
    };
    int nl = 0;
    for (int r = 0; r < R && e == cudaSuccess; ++r) {
        check(cudaEventRecord(bg->events[n], bg->stream));
        for (int i = 0; i < n; ++i) {
            dao_ctx* c = ctxs[i];
            cudaStream_t cs = c->stream;
            check(cudaStreamWaitEvent(cs, bg->events[n], 0));
            const bool mlc = c->opt.mlc_constraint != DAO_MLC_CONSECUTIVE;
            const RowTicket rt{c->binfo, c->beam_row0_d, c->cols_d, c->row_info, mlc ? nullptr : c->row_cnt,
                               c->row_v, c->row_lr, c->cg};
            check(launch_dt_rows(c->Dt, c->pi, c->w, rt, cs, &nl));
            if (mlc) check(price_rows_any(c, c->w, &c->cg->stop, cs, &nl));
            CommitArgs ca{};
            ca.row_v = c->row_v;
            ca.row_lr = c->row_lr;
            ca.beam_row0 = c->beam_row0_d;
            ca.rows = c->rows_d;
            ca.cols = c->cols_d;
            ca.beam_off = c->beam_off_d;
            ca.seg = c->seg;
            ca.n_beams = c->B;
            ca.lr_stride = 2 * c->max_rows;
            ca.tau = c->tau;
            ca.ap_beam = c->ap_beam;
            ca.ap_lr = c->ap_lr;
            ca.slab = c->slab;
            ca.ld = c->ld;
            ca.cg = c->cg;
            ca.use_cond = 0;
            check(launch_commit_column(c->D, ca, c->max_nb, c->num_sms, cs, &nl));
            check(cudaEventRecord(bg->events[i], cs));
            check(cudaStreamWaitEvent(bg->stream, bg->events[i], 0));
        }
        check(launch_master_persist_batch(bg->tasks, n, bg->GB, max_V, bg->stream, &nl));
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(bg->stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&bg->exec, g, 0);
    bg->graph = g;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DAO_ECUDA, std::string("building the batch graph: ") + cudaGetErrorString(e));
    }
    return DAO_OK;
}

}  // namespace

extern "C" {

int32_t dao_batch_group_size(int32_t n, int32_t device) {
    int sms = 0;
    if (n < 1 || cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return master_batch_group(n, sms);
}

dao_status dao_batch_solve_persistent(dao_ctx* const* ctxs, int32_t n, int32_t n_apertures, int32_t* n_done,
                                      double* traces, int32_t* status) {
    TraceRange range("dao_batch_solve_persistent");
    if (n < 0 || n_apertures < 0 || (n > 0 && ctxs == nullptr))
        return fail(DAO_EINVAL, "n >= 0, n_apertures >= 0 and a context array are required");
    for (int i = 0; i < n; ++i) {
        if (ctxs[i] == nullptr) return fail(DAO_EINVAL, "null context " + std::to_string(i));
        if (ctxs[i]->prof_on) return fail(DAO_EINVAL, "every context needs profiling off");
        if (ctxs[i]->device != ctxs[0]->device) return fail(DAO_EINVAL, "the contexts must be on one device");
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return fail(DAO_EINVAL, "context listed twice");
    }
    if (n == 0) return DAO_OK;
    DAO_TRY(check_ctx(ctxs[0]));
    std::vector<GraphSolve> gs(n);
    int R = 0;
    for (int i = 0; i < n; ++i) {
        gs[i].K0 = ctxs[i]->K;
        gs[i].K1 = std::min(ctxs[i]->K_cap, ctxs[i]->K + n_apertures);
        R = std::max(R, gs[i].K1 - gs[i].K0);
        if (status) status[i] = DAO_OK;
        if (n_done) n_done[i] = ctxs[i]->K;
    }
    std::vector<uint64_t> key;
    for (int i = 0; i < n; ++i) key.push_back(ctxs[i]->uid);
    key.push_back((uint64_t)R);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchGraph* bg = nullptr;
    for (size_t i = 0; i < g_batch_graphs.size(); ++i)
        if (g_batch_graphs[i]->key == key) {
            bg = g_batch_graphs[i];
            g_batch_graphs.erase(g_batch_graphs.begin() + i);
            break;
        }
    if (bg == nullptr && R > 0) {
        bg = new (std::nothrow) BatchGraph();
        if (!bg) return fail(DAO_ENOMEM, "host allocation failed");
        bg->key = key;
        const dao_status st = build_batch_graph(ctxs, n, R, bg);
        if (st != DAO_OK) {
            const std::string msg = g_err;
            batch_graph_free(bg);
            return fail(st, msg);
        }
    }
    if (bg != nullptr) {
        g_batch_graphs.insert(g_batch_graphs.begin(), bg);
        while (g_batch_graphs.size() > BATCH_GRAPHS_KEPT) {
            batch_graph_free(g_batch_graphs.back());
            g_batch_graphs.pop_back();
        }
        // every plan's round state on its stream, then the graph after all of them,
        // then every plan's stream after the graph
        for (int i = 0; i < n; ++i) {
            DAO_TRY(solve_state_begin(ctxs[i], &gs[i]));
            DAO_CU(cudaEventRecord(bg->events[i], ctxs[i]->stream));
            DAO_CU(cudaStreamWaitEvent(bg->stream, bg->events[i], 0));
        }
        DAO_CU(cudaGraphLaunch(bg->exec, bg->stream));
        DAO_CU(cudaEventRecord(bg->events[n], bg->stream));
        for (int i = 0; i < n; ++i) DAO_CU(cudaStreamWaitEvent(ctxs[i]->stream, bg->events[n], 0));
    }
    for (int i = 0; i < n; ++i) {
        dao_ctx* c = ctxs[i];
        dao_status res = DAO_OK;
        DAO_TRY(solve_graph_end(c, gs[i], n_apertures, n_done ? n_done + i : nullptr,
                                traces ? traces + (size_t)i * n_apertures : nullptr, &res, false));
        const int per_round = c->opt.mlc_constraint != DAO_MLC_CONSECUTIVE ? 3 : 2;
        c->launches_i += per_round * R + (i == 0 ? R : 0);  // its round kernels; the master launches on the first
        c->count_launches();
        if (status) status[i] = res;
    }
    return DAO_OK;
}

dao_status dao_kernel_forms(const dao_ctx* c, dao_tuning* out) {
    if (!c || !out) return fail(DAO_EINVAL, "null argument");
    const DevCSR& D = c->D;
    const DevCSR& Dt = c->Dt;
    const bool split = Dt.tune_dt_map == DT_MAP_SPLIT && Dt.split_chunk > 0;
    out->dose_form = dose_form_effective(D);
    out->dose_lanes = D.tune_dose_g;
    out->column_lanes = D.tune_col_g;  // 0: the beam layout
    out->dt_map = split ? DT_MAP_SPLIT : Dt.tune_dt_map == DT_MAP_GROUPED ? DT_MAP_GROUPED : DT_MAP_CONSECUTIVE;
    out->dt_threads = split ? 0 : (Dt.tune_dt_threads ? Dt.tune_dt_threads : 64);
    out->from_cache = 0;
    return DAO_OK;
}

dao_status dao_autotune(dao_ctx* c, const char* cache_path, dao_tuning* out) {
    TraceRange range("dao_autotune");
    DAO_TRY(check_ctx(c));
    const std::string key = tune_key(c);
    int dg = 0, cg = 0, dt = 0, form = 0, map = 0;
    const bool units_ok = dose_units_available(c->D);
    bool cached = tune_cache_read(cache_path, key, &dg, &cg, &dt, &form, &map) && tune_allowed(TUNE_DOSE_G, dg) &&
                  tune_allowed(TUNE_COL_G, cg) && tune_allowed(TUNE_DT_THREADS, dt) &&
                  (form == DOSE_FORM_LANES || (form == DOSE_FORM_UNITS && units_ok) ||
                   (form == DOSE_FORM_MERGE && c->D.merge_chunk > 0)) &&
                  (map == DT_MAP_GROUPED || map == DT_MAP_CONSECUTIVE ||
                   (map == DT_MAP_SPLIT && c->Dt.split_chunk > 0));
    if (cached && c->opt.precision != DAO_PREC_FP32 && dg > 16) cached = false;
    if (!cached) {
        const int reps = 10;
        auto time_dose = [&](double* us) {
            return time_cold(c, reps, [&](int* nl) {
                return launch_dose(c->D, c->x, c->vstruct, c->tf, c->ts, c->S, c->dose, nullptr, nullptr, 0, nullptr,
                                   c->num_sms, c->stream, nl);
            }, us, "dao_autotune");
        };
        // a1: lanes per voxel row of the lane form (the lane count is kept for
        // the aperture column's defaults), then the unit form against the best
        double best = 1e300;
        c->D.tune_dose_form = DOSE_FORM_LANES;
        for (int g : TUNE_DOSE_G) {
            if (c->opt.precision != DAO_PREC_FP32 && g > 16) continue;
            c->D.tune_dose_g = g;
            double us = 0.0;
            DAO_TRY(time_dose(&us));
            if (us < best) {
                best = us;
                dg = g;
            }
        }
        form = DOSE_FORM_LANES;
        for (int f : {DOSE_FORM_UNITS, DOSE_FORM_MERGE}) {
            c->D.tune_dose_form = f;
            if (dose_form_effective(c->D) != f) continue;  // not available for this matrix
            double us = 0.0;
            DAO_TRY(time_dose(&us));
            if (us < best) {
                best = us;
                form = f;
            }
        }
        best = 1e300;
        if (c->Dt.split_chunk > 0) {  // a2: the split form, then a block per row in both lane mappings
            c->Dt.tune_dt_map = DT_MAP_SPLIT;
            double us = 0.0;
            DAO_TRY(time_cold(c, reps,
                              [&](int* nl) { return launch_dt(c->Dt, c->pi, c->w, nullptr, c->stream, nl); }, &us,
                              "dao_autotune"));
            best = us;
            dt = 64;
            map = DT_MAP_SPLIT;
        }
        for (int m : {DT_MAP_GROUPED, DT_MAP_CONSECUTIVE})
            for (int t : TUNE_DT_THREADS) {
                c->Dt.tune_dt_threads = t;
                c->Dt.tune_dt_map = m;
                double us = 0.0;
                DAO_TRY(time_cold(c, reps,
                                  [&](int* nl) { return launch_dt(c->Dt, c->pi, c->w, nullptr, c->stream, nl); }, &us,
                                  "dao_autotune"));
                if (us < best) {
                    best = us;
                    dt = t;
                    map = m;
                }
            }
        best = 1e300;
        for (int g : TUNE_COL_G) {  // a4: the beam layout (0), or lanes per voxel row over beam 0's segment
            c->D.tune_col_g = g;
            double us = 0.0;
            DAO_TRY(time_cold(c, reps, [&](int* nl) {
                return launch_column(c->D, c->seg, 0, c->beam_off[0], c->rows[0] * c->cols[0], c->mask, c->dose, 1,
                                     c->num_sms, c->stream, nl);
            }, &us, "dao_autotune"));
            if (us < best) {
                best = us;
                cg = g;
            }
        }
        if (cache_path) {
            FILE* f = std::fopen(cache_path, "a");
            if (f) {
                std::fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), dg, cg, dt, form, map);
                std::fclose(f);
            }
        }
    }
    c->D.tune_dose_g = dg;
    c->D.tune_dose_form = form;
    c->D.tune_col_g = cg;
    c->Dt.tune_dt_threads = dt;
    c->Dt.tune_dt_map = map;
    drop_round_graphs(c);
    if (out) {
        out->dose_lanes = dg;
        out->column_lanes = cg;
        out->dt_threads = dt;
        out->from_cache = cached ? 1 : 0;
        out->dose_form = form;
        out->dt_map = map;
    }
    return DAO_OK;
}

}  // extern "C"
