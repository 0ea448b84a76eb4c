// Pricing sub-problem of column-generation DAO (arXiv:1003.5402, Eq. 8 and the
// one-pass MLC-row search of Sec. 2.3), re-designed as one warp per MLC row.
//
// For row w_1..w_n (n <= 32, lane c holds w_{c+1}) the paper's sequential loop
// keeps the running sum v = S_r, the largest running sum vbar = max(0, S_1..S_r)
// with its earliest position l, and the best value v* = min_r (S_r - vbar_r)
// with the earliest r.  The warp computes the same quantities:
//   1. S_r by lane-serial replay: lane r-1 adds w_1, ..., w_r in that order in
//      FP64, which is exactly the rounding sequence of the sequential loop;
//   2. (vbar_r, l_r) by an inclusive shuffle scan whose operator keeps the
//      earlier element unless the later one is strictly larger (the strict ">"
//      of the loop), seeded with the empty prefix (0, 0);
//   3. S_r - vbar_r per lane (the same subtraction as the loop), then a
//      butterfly minimum that prefers the smaller r on equal values (the
//      strict "<").
// The result equals the sequential loop bit for bit for the same FP32 inputs.
// The per-beam sum adds the rows' v* in row order, and the beam argmin keeps
// the lowest beam index on ties.
#include "dao_internal.h"

namespace dao {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// row_info[g] = (beam, first beamlet index, columns, row within the beam)
__global__ void __launch_bounds__(256) k_price_rows(const float* __restrict__ w, const int4* __restrict__ row_info,
                                                    int n_rows, double* __restrict__ row_v,
                                                    int2* __restrict__ row_lr, const int* __restrict__ skip) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= n_rows) return;  // uniform per warp
    if (skip != nullptr && *skip) return;
    const int4 ri = row_info[g];
    const int n = ri.z;
    const double wv = lane < n ? (double)w[ri.y + lane] : 0.0;

    // 1. prefix sums in the sequential order
    double s = 0.0;
    for (int q = 0; q < n; ++q) {
        const double t = __shfl_sync(FULL, wv, q);
        if (q <= lane) s = s + t;
    }

    // 2. running maximum with the earliest position (1-based prefix index)
    double m = lane < n ? s : -INFINITY;
    int mi = lane + 1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double om = __shfl_up_sync(FULL, m, o);
        const int omi = __shfl_up_sync(FULL, mi, o);
        if (lane >= o && !(m > om)) {
            m = om;
            mi = omi;
        }
    }
    if (!(m > 0.0)) {  // the empty prefix S_0 = 0 at l = 0 comes first
        m = 0.0;
        mi = 0;
    }

    // 3. best (most negative) S_r - vbar_r, earliest r on ties
    double bd = lane < n ? s - m : INFINITY;
    int br = lane + 1;
    int bl = mi;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(FULL, bd, o);
        const int orr = __shfl_xor_sync(FULL, br, o);
        const int ol = __shfl_xor_sync(FULL, bl, o);
        if (od < bd || (od == bd && orr < br)) {
            bd = od;
            br = orr;
            bl = ol;
        }
    }
    if (lane == 0) {
        if (bd < 0.0) {
            row_v[g] = bd;
            row_lr[g] = make_int2(bl, br);  // open beamlets [l*, r* - 1) in 0-based half-open form
        } else {
            row_v[g] = 0.0;
            row_lr[g] = make_int2(0, 0);
        }
    }
}

// One block: thread b sums beam b's rows in row order; thread 0 takes the argmin.
__global__ void __launch_bounds__(256) k_price_beams(const double* __restrict__ row_v,
                                                     const int* __restrict__ beam_row0, int n_beams,
                                                     PriceDev* __restrict__ out, const int* __restrict__ skip) {
    extern __shared__ double s_sum[];
    if (skip != nullptr && *skip) return;
    for (int b = threadIdx.x; b < n_beams; b += blockDim.x) {
        double t = 0.0;
        for (int r = beam_row0[b]; r < beam_row0[b + 1]; ++r) t = t + row_v[r];
        s_sum[b] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        for (int b = 1; b < n_beams; ++b)
            if (s_sum[b] < s_sum[best]) best = b;
        out->beam = best;
        out->rc = n_beams > 0 ? s_sum[best] : 0.0;
    }
}

// The beam sums and their argmin (as k_price_beams) in one block with the
// stop tests and the new aperture (the graph path).
__global__ void __launch_bounds__(256) k_price_commit(const double* __restrict__ row_v,
                                                      const int* __restrict__ beam_row0, int n_beams,
                                                      PriceDev* __restrict__ pr, const int2* __restrict__ row_lr,
                                                      const int* __restrict__ rows, const int* __restrict__ cols,
                                                      double tau, int K, int lr_stride, int* __restrict__ ap_beam,
                                                      int* __restrict__ ap_lr, float* __restrict__ mask,
                                                      CGDev* __restrict__ cg, cudaGraphConditionalHandle cond,
                                                      int use_cond) {
    extern __shared__ double s_sum[];
    __shared__ int s_best, s_dup;
    __shared__ double s_rc;
    const int tid = threadIdx.x;
    // idle: this round's column and master solve skip; stop: later rounds skip
    // (the enclosing while node, if any, ends)
    auto finish = [&](int idle, int stop) {
        if (tid == 0) {
            cg->idle = idle;
            cg->stop = stop;
            if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
        }
    };
    if (cg->stop) {
        finish(1, 1);
        return;
    }
    if (K <= 0) K = cg->K + 1;
    for (int b = tid; b < n_beams; b += blockDim.x) {
        double t = 0.0;
        for (int r = beam_row0[b]; r < beam_row0[b + 1]; ++r) t = t + row_v[r];
        s_sum[b] = t;
    }
    __syncthreads();
    if (tid == 0) {
        int best = 0;
        for (int b = 1; b < n_beams; ++b)
            if (s_sum[b] < s_sum[best]) best = b;
        s_best = best;
        s_rc = n_beams > 0 ? s_sum[best] : 0.0;
        pr->beam = best;
        pr->rc = s_rc;
        s_dup = 0;
    }
    __syncthreads();
    const int b = s_best;
    if (!(s_rc < -tau)) {
        if (tid == 0) cg->done = 1;
        finish(1, 1);
        return;
    }
    const int R = rows[b], C = cols[b], r0 = beam_row0[b];
    for (int k = tid; k < K - 1; k += blockDim.x) {
        if (ap_beam[k] != b) continue;
        bool same = true;
        for (int r = 0; r < R && same; ++r) {
            const int2 lr = row_lr[r0 + r];
            same = ap_lr[k * lr_stride + 2 * r] == lr.x && ap_lr[k * lr_stride + 2 * r + 1] == lr.y;
        }
        if (same) s_dup = 1;
    }
    __syncthreads();
    if (s_dup) {
        if (tid == 0) cg->done = 2;
        finish(1, 1);
        return;
    }
    if (tid == 0) ap_beam[K - 1] = b;
    for (int r = tid; r < R; r += blockDim.x) {
        const int2 lr = row_lr[r0 + r];
        ap_lr[(K - 1) * lr_stride + 2 * r] = lr.x;
        ap_lr[(K - 1) * lr_stride + 2 * r + 1] = lr.y;
    }
    for (int i = tid; i < R * C; i += blockDim.x) {
        const int2 lr = row_lr[r0 + i / C];
        const int c = i % C;
        mask[i] = (c >= lr.x && c < lr.y) ? 1.f : 0.f;
    }
    if (tid == 0) cg->K = K;
    finish(0, K >= cg->K_end ? 1 : 0);
}

}  // namespace

cudaError_t launch_price_rows(const float* w, const int4* row_info, int n_rows, double* row_v, int2* row_lr,
                              const int* skip, cudaStream_t stream, int* launches) {
    if (n_rows == 0) return cudaSuccess;
    k_price_rows<<<n_rows, 32, 0, stream>>>(w, row_info, n_rows, row_v, row_lr, skip);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_price_commit(const double* row_v, const int* beam_row0, int n_beams, PriceDev* pr,
                                const int2* row_lr, const int* rows, const int* cols, double tau, int K, int lr_stride,
                                int* ap_beam, int* ap_lr, float* mask, CGDev* cg, cudaGraphConditionalHandle cond,
                                int use_cond, cudaStream_t stream, int* launches) {
    k_price_commit<<<1, 256, (size_t)(n_beams > 0 ? n_beams : 1) * sizeof(double), stream>>>(
        row_v, beam_row0, n_beams, pr, row_lr, rows, cols, tau, K, lr_stride, ap_beam, ap_lr, mask, cg, cond,
        use_cond);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_price(const float* w, const int4* row_info, int n_rows, const int* beam_row0, int n_beams,
                         double* row_v, int2* row_lr, PriceDev* out, const int* skip, cudaStream_t stream,
                         int* launches) {
    // one warp per block: the FP64 prefix sums of a row issue at 1/64 of the FP32
    // rate, so the rows are spread over every SM rather than packed 8 to a block
    const int warps_per_block = 1;
    const int grid = (n_rows + warps_per_block - 1) / warps_per_block;
    if (grid > 0) {
        k_price_rows<<<grid, 32 * warps_per_block, 0, stream>>>(w, row_info, n_rows, row_v, row_lr, skip);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_price_beams<<<1, 256, (size_t)(n_beams > 0 ? n_beams : 1) * sizeof(double), stream>>>(row_v, beam_row0,
                                                                                           n_beams, out, skip);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace dao
