// Pricing sub-problem of column-generation DAO (arXiv:1003.5402, Eq. 8 and the
// one-pass MLC-row search of Sec. 2.3), re-designed as one warp per MLC row;
// the row search and the beam decision are in pricing.cuh.
#include "pricing.cuh"

namespace dao {

namespace {


// row_info[g] = (beam, first beamlet index, columns, row within the beam)
__global__ void __launch_bounds__(256) k_price_rows(const float* __restrict__ w, const int4* __restrict__ row_info,
                                                    int n_rows, double* __restrict__ row_v,
                                                    int2* __restrict__ row_lr, const int* __restrict__ skip) {
    const int g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= n_rows) return;  // uniform per warp
    if (skip != nullptr && *skip) return;
    pricing::row_best(w, row_info[g], g, row_v, row_lr);
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
// stop tests and the new aperture K - 1 (the per-round graphs).  Sets cg->idle
// (0 when it added an aperture) and cg->stop (the solve stopped, or the pool
// reached cg->K_end).
__global__ void __launch_bounds__(256) k_price_commit(const double* __restrict__ row_v,
                                                      const int* __restrict__ beam_row0, int n_beams,
                                                      PriceDev* __restrict__ pr, const int2* __restrict__ row_lr,
                                                      const int* __restrict__ rows, const int* __restrict__ cols,
                                                      double tau, int K, int lr_stride, int* __restrict__ ap_beam,
                                                      int* __restrict__ ap_lr, float* __restrict__ mask,
                                                      CGDev* __restrict__ cg) {
    extern __shared__ double s_sum[];
    const int tid = threadIdx.x;
    auto finish = [&](int idle, int stop) {
        if (tid == 0) {
            cg->idle = idle;
            cg->stop = stop;
        }
    };
    if (cg->stop) {
        finish(1, 1);
        return;
    }
    int b = 0;
    double rc = 0.0;
    const int outcome = pricing::decide(row_v, beam_row0, n_beams, row_lr, rows, tau, K, lr_stride, ap_beam, ap_lr,
                                        s_sum, &b, &rc);
    if (tid == 0) {
        pr->beam = b;
        pr->rc = rc;
    }
    if (outcome != pricing::OUTCOME_NEW) {
        if (tid == 0) cg->done = outcome;
        finish(1, 1);
        return;
    }
    const int R = rows[b], C = cols[b], r0 = beam_row0[b];
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
                                int* ap_beam, int* ap_lr, float* mask, CGDev* cg, cudaStream_t stream, int* launches) {
    k_price_commit<<<1, 256, (size_t)(n_beams > 0 ? n_beams : 1) * sizeof(double), stream>>>(
        row_v, beam_row0, n_beams, pr, row_lr, rows, cols, tau, K, lr_stride, ap_beam, ap_lr, mask, cg);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_price_beams(const double* row_v, const int* beam_row0, int n_beams, PriceDev* out,
                               const int* skip, cudaStream_t stream, int* launches) {
    k_price_beams<<<1, 256, (size_t)(n_beams > 0 ? n_beams : 1) * sizeof(double), stream>>>(row_v, beam_row0,
                                                                                           n_beams, out, skip);
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
