// Device pieces of the pricing sub-problem (arXiv:1003.5402, Eq. 8 and the
// one-pass MLC-row search of Sec. 2.3) shared by the stand-alone pricing
// kernels (price.cu) and the fused kernels of the device-driven round
// (spmv.cu).
//
// row_best: for row w_1..w_n (n <= 32, lane c holds w_{c+1}) the paper's
// sequential loop keeps the running sum v = S_r, the largest running sum
// vbar = max(0, S_1..S_r) with its earliest position l, and the best value
// v* = min_r (S_r - vbar_r) with the earliest r.  The warp computes the same
// quantities:
//   1. S_r by lane-serial replay: lane r-1 adds w_1, ..., w_r in that order in
//      FP64, which is exactly the rounding sequence of the sequential loop;
//   2. (vbar_r, l_r) by an inclusive shuffle scan whose operator keeps the
//      earlier element unless the later one is strictly larger (the strict ">"
//      of the loop), seeded with the empty prefix (0, 0);
//   3. S_r - vbar_r per lane (the same subtraction as the loop), then a
//      butterfly minimum that prefers the smaller r on equal values (the
//      strict "<").
// The result equals the sequential loop bit for bit for the same FP32 inputs.
//
// decide: the per-beam sum adds the rows' v* in row order, the beam argmin
// keeps the lowest beam index on ties; then the stop test (reduced cost not
// below -tau) and the duplicate test against the pool.
#pragma once

#include "dao_internal.h"

namespace dao {
namespace pricing {

constexpr unsigned WARP_ALL = 0xffffffffu;

// One full warp: MLC row g with row_info ri = (beam, first beamlet, columns,
// row within the beam).  w is read through L2: in the fused round other
// blocks of the same launch wrote it.
__device__ __forceinline__ void row_best(const float* __restrict__ w, int4 ri, int g, double* __restrict__ row_v,
                                         int2* __restrict__ row_lr) {
    const int lane = threadIdx.x & 31;
    const int n = ri.z;
    const double wv = lane < n ? (double)__ldcg(w + ri.y + lane) : 0.0;

    // 1. prefix sums in the sequential order
    double s = 0.0;
    for (int q = 0; q < n; ++q) {
        const double t = __shfl_sync(WARP_ALL, wv, q);
        if (q <= lane) s = s + t;
    }

    // 2. running maximum with the earliest position (1-based prefix index)
    double m = lane < n ? s : -INFINITY;
    int mi = lane + 1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double om = __shfl_up_sync(WARP_ALL, m, o);
        const int omi = __shfl_up_sync(WARP_ALL, mi, o);
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
        const double od = __shfl_xor_sync(WARP_ALL, bd, o);
        const int orr = __shfl_xor_sync(WARP_ALL, br, o);
        const int ol = __shfl_xor_sync(WARP_ALL, bl, o);
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

enum { OUTCOME_NEW = 0, OUTCOME_OPTIMAL = 1, OUTCOME_DUPLICATE = 2 };

// Whole block (every thread calls it): beam sums into s_sum (n_beams doubles
// of shared memory), argmin, stop test, then the duplicate test against the
// K - 1 apertures of the pool.  Every thread returns the same outcome, beam
// and reduced cost.
__device__ __forceinline__ int decide(const double* __restrict__ row_v, const int* __restrict__ beam_row0,
                                      int n_beams, const int2* __restrict__ row_lr, const int* __restrict__ rows,
                                      double tau, int K, int lr_stride, const int* __restrict__ ap_beam,
                                      const int* __restrict__ ap_lr, double* s_sum, int* beam_out,
                                      double* rc_out) {
    __shared__ int s_best, s_dup;
    __shared__ double s_rc;
    const int tid = threadIdx.x;
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
        s_dup = 0;
    }
    __syncthreads();
    const int b = s_best;
    *beam_out = b;
    *rc_out = s_rc;
    if (!(s_rc < -tau)) return OUTCOME_OPTIMAL;
    const int R = rows[b], r0 = beam_row0[b];
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
    return s_dup ? OUTCOME_DUPLICATE : OUTCOME_NEW;
}

}  // namespace pricing
}  // namespace dao
