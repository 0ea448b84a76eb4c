// Internal declarations shared by the libdao.so translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "dao.h"

namespace dao {

constexpr int KMAX = 64;        // aperture pool capacity (master problem size)
constexpr int SMAX = 64;        // structures
constexpr int CMAX = 32;        // beamlets per MLC row (one warp lane each)
constexpr int MASTER_TILE = 256;  // voxels per tile of the fused master pass (= block size)

// Per-structure objective terms (Eqs. 9-10): a = alpha_s/|v_s| (0 for
// non-targets), tu = T_s^-, b = beta_s/|v_s|, to = T_s^+.
struct StructTermsF { float a, tu, b, to; };
struct StructTermsD { double a, tu, b, to; };

// Device copy of a CSR matrix whose rows are padded to a multiple of four
// entries (padding: value 0, column = the row's last real column), so every
// row starts on a 16-byte boundary for int4/float4 loads.
struct DevCSR {
    int n_rows = 0;
    int n_cols = 0;
    int64_t nnz_stored = 0;
    int* rowptr = nullptr;   // n_rows + 1, multiples of 4
    int* col = nullptr;
    float* val = nullptr;
};

// Projected-Newton master state (device memory, one per context).
struct MasterDev {
    double y[KMAX];       // accepted intensities
    double yt[KMAX];      // trial point evaluated by the next fused pass
    double d[KMAX];       // search direction
    double g[KMAX];       // gradient at y
    double gt[KMAX];      // gradient at the trial point (written by the reduction)
    double Ht[KMAX * KMAX];  // curvature matrix at the trial point (full, symmetric)
    double F;             // objective at y
    double Ft;            // objective at the trial point
    double alpha;         // step length along d
    double tol;           // absolute KKT tolerance of this solve
    double res;           // KKT residual at y
    float yf[KMAX];       // FP32 copy of the point the fused pass evaluates
    int K;                // pool size
    int iter;             // Newton iterations taken
    int phase;            // 0: evaluating the warm start, 1: line search
    int done;             // 1 once converged / stalled / out of iterations
    int status;           // MASTER_*
    int n_eval;           // fused passes evaluated
};

enum { MASTER_RUNNING = 0, MASTER_CONVERGED = 1, MASTER_MAXITER = 2, MASTER_STALLED = 3 };

// Result of the device-side pricing (step a3).
struct PriceDev {
    double rc;            // reduced cost of the best beam
    int beam;             // b*
    int pad;
};

// ---- kernel launchers (all on `stream`; return the launch error) ----------

// a1: z = D x, optional grad F(z), FP64 F partials (one per block) reduced into *F_out.
cudaError_t launch_dose(const DevCSR& D, const float* x, const uint8_t* vstruct,
                        const StructTermsF* tf, const StructTermsD* td, int S,
                        float* z, float* grad, double* F_part, int F_blocks, double* F_out,
                        int num_sms, cudaStream_t stream, int* launches);
int dose_grid(int n_rows, int num_sms);

// a2: w = D^T pi over the beamlet-major transpose.
cudaError_t launch_dt(const DevCSR& Dt, const float* pi, float* w, cudaStream_t stream, int* launches);

// a4: out_j = sum over beam b's entries of row j with mask[col - base] (0/1).
cudaError_t launch_column(const DevCSR& D, const int* seg_lo, const int* seg_hi, int base,
                          int n_beamlets_b, const float* mask, float* out, int num_sms,
                          cudaStream_t stream, int* launches);

// x_i = sum_{k in K_i} y_k (Eq. 7) from the aperture table.
cudaError_t launch_fluence(const int* ap_beam, const int* ap_lr, int lr_stride, const double* y, int K,
                           const int4* beamlet_info, int N, float* x, cudaStream_t stream, int* launches);

// a3: per-row scan (one warp per MLC row) and the per-beam sum / argmin.
cudaError_t launch_price(const float* w, const int4* row_info, int n_rows, const int* beam_row0,
                         int n_beams, double* row_v, int2* row_lr, PriceDev* out,
                         cudaStream_t stream, int* launches);

// a5: projected-Newton master problem kernels.
struct MasterBuffers {
    MasterDev* st = nullptr;
    float* H_part = nullptr;    // [KMAX*KMAX][G]
    double* g_part = nullptr;   // [KMAX][G]
    double* F_part = nullptr;   // [G]
    int G = 0;
};
cudaError_t launch_master_init(MasterDev* st, int K, cudaStream_t stream, int* launches);
cudaError_t launch_master_pass(const float* slab, int V, int ld, int K, const MasterBuffers& mb,
                               const uint8_t* vstruct, const StructTermsF* tf, const StructTermsD* td,
                               int S, float* z_out, float* pi_out, int final_pass,
                               cudaStream_t stream, int* launches);
cudaError_t launch_master_reduce(int K, const MasterBuffers& mb, cudaStream_t stream, int* launches);
cudaError_t launch_master_step(const MasterBuffers& mb, int max_iter, double tol_rel,
                               cudaStream_t stream, int* launches);
size_t master_pass_smem(int K);
cudaError_t master_configure();

}  // namespace dao
