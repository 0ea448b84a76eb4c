// Pricing under MLC hardware constraints (arXiv:1003.5402, Sec. 4, last
// paragraph: besides the consecutiveness of each row's open beamlets the
// method handles interdigitation, connectedness and jaws-only delivery).
//
// One block per beam.  Every mode works on the FP64 prefix sums of the beam's
// rows, P_r[0] = 0, P_r[c + 1] = P_r[c] + w_c (column order), an interval's
// sum being P_r[R] - P_r[L]; the arithmetic and the tie rules below are fixed
// so that the result is reproducible bit for bit:
//   - interdigitation (adjacent rows' leaves may not cross: L_r <= R_{r+1} and
//     L_{r+1} <= R_r, a closed row's leaves together at some position p):
//     dynamic programme over the rows on the leaf states (L, R), 0 <= L <= R
//     <= C, f_0(s) = I_0(s), f_r(s') = I_r(s') + min over compatible s of
//     f_{r-1}(s); the minimum over the compatible states {L <= R', R >= L'} is
//     read from a two-dimensional running minimum (a suffix minimum over R,
//     then a prefix minimum over L) that keeps the smallest state index on
//     equal values, so every choice, and the trace back from the smallest
//     final state, takes the smallest index among equal values;
//   - connectedness (the open rows form one contiguous block): each row's
//     best non-empty interval (smallest (L, R) in L-major order on ties), then
//     the paper's one-pass search over those row values picks the block;
//   - jaws-only (a rectangle): for every column range [L, R) the paper's
//     one-pass search over the rows' interval sums, then the smallest value
//     over the column ranges, the earliest range on ties.
// A beam whose best value is not negative is closed (value 0).  The beam's
// value is written at its first MLC row of row_v and 0 at the others, so that
// the beam decision, which sums row_v over a beam's rows in row order, sees
// exactly the beam's value; closed rows are written as (0, 0).
#include <climits>

#include "dao_internal.h"

namespace dao {

namespace {

constexpr int MLC_THREADS = 256;

__device__ __forceinline__ bool mlc_better(double v, int i, double bv, int bi) {
    return v < bv || (v == bv && i < bi);
}

// index of the leaf state (L, R), 0 <= L <= R <= C (C1 = C + 1), L-major
__device__ __forceinline__ int mlc_state(int L, int R, int C1) { return L * C1 - L * (L - 1) / 2 + (R - L); }

// The paper's one-pass search (Sec. 2.3) over n values v(1..n): running sum,
// largest running sum with its earliest position, best difference with the
// earliest end; returns v* and the block [a, b) (v* = 0: none).
template <class Get>
__device__ __forceinline__ double mlc_row_search(int n, Get get, int* a, int* b) {
    double s = 0.0, vbar = 0.0, best = 0.0;
    int l = 0, ls = 0, rs = 1;
    for (int r = 1; r <= n; ++r) {
        s = s + get(r - 1);
        if (s > vbar) {
            vbar = s;
            l = r;
        }
        if (s - vbar < best) {
            best = s - vbar;
            ls = l;
            rs = r + 1;
        }
    }
    *a = ls;
    *b = rs - 1;
    return best;
}

template <int MODE>
__global__ void __launch_bounds__(MLC_THREADS) k_price_mlc(const float* __restrict__ w,
                                                           const int* __restrict__ beam_off,
                                                           const int* __restrict__ rows,
                                                           const int* __restrict__ cols,
                                                           const int* __restrict__ beam_row0,
                                                           double* __restrict__ row_v, int2* __restrict__ row_lr,
                                                           const int* __restrict__ skip) {
    extern __shared__ __align__(16) double sm[];
    if (skip != nullptr && *skip) return;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int R = rows[b], C = cols[b], C1 = C + 1, off = beam_off[b], r0 = beam_row0[b];
    double* P = sm;  // [R][C1]
    for (int r = tid; r < R; r += blockDim.x) {
        double acc = 0.0;
        P[r * C1] = 0.0;
        for (int c = 0; c < C; ++c) {
            acc = acc + (double)w[off + r * C + c];
            P[r * C1 + c + 1] = acc;
        }
    }
    __syncthreads();
    __shared__ double s_val;
    __shared__ int s_a, s_b, s_L, s_R;

    if constexpr (MODE == DAO_MLC_INTERDIGITATION) {
        const int NS = C1 * (C1 + 1) / 2;
        double* fa = P + R * C1;
        double* fb = fa + NS;
        double* Gv = fb + NS;                                                   // [C1][C1]
        int* Gi = reinterpret_cast<int*>(Gv + C1 * C1);                         // [C1][C1]
        unsigned short* back = reinterpret_cast<unsigned short*>(Gi + C1 * C1);  // [R][NS]
        unsigned char* sL = reinterpret_cast<unsigned char*>(back + R * NS);     // [NS]
        unsigned char* sR = sL + NS;                                            // [NS]
        for (int L = tid; L <= C; L += blockDim.x)
            for (int Rr = L; Rr <= C; ++Rr) {
                const int s = mlc_state(L, Rr, C1);
                sL[s] = (unsigned char)L;
                sR[s] = (unsigned char)Rr;
            }
        __syncthreads();
        for (int s = tid; s < NS; s += blockDim.x) fa[s] = P[sR[s]] - P[sL[s]];
        __syncthreads();
        for (int r = 1; r < R; ++r) {
            // H[a][x] = min over R >= max(a, x) of f(a, R)
            for (int a = tid; a <= C; a += blockDim.x) {
                double m = INFINITY;
                int mi = INT_MAX;
                for (int Rr = C; Rr >= a; --Rr) {
                    const int s = mlc_state(a, Rr, C1);
                    if (mlc_better(fa[s], s, m, mi)) {
                        m = fa[s];
                        mi = s;
                    }
                    Gv[a * C1 + Rr] = m;
                    Gi[a * C1 + Rr] = mi;
                }
                for (int x = a - 1; x >= 0; --x) {
                    Gv[a * C1 + x] = m;
                    Gi[a * C1 + x] = mi;
                }
            }
            __syncthreads();
            // G[a][x] = min over a' <= a of H[a'][x]: min over L <= a, R >= x
            for (int x = tid; x <= C; x += blockDim.x) {
                double m = INFINITY;
                int mi = INT_MAX;
                for (int a = 0; a <= C; ++a) {
                    if (mlc_better(Gv[a * C1 + x], Gi[a * C1 + x], m, mi)) {
                        m = Gv[a * C1 + x];
                        mi = Gi[a * C1 + x];
                    }
                    Gv[a * C1 + x] = m;
                    Gi[a * C1 + x] = mi;
                }
            }
            __syncthreads();
            // the states compatible with (L', R') are {L <= R', R >= L'}: G[R'][L']
            const double* Pr = P + r * C1;
            for (int s = tid; s < NS; s += blockDim.x) {
                const int L = sL[s], Rr = sR[s];
                fb[s] = (Pr[Rr] - Pr[L]) + Gv[Rr * C1 + L];
                back[r * NS + s] = (unsigned short)Gi[Rr * C1 + L];
            }
            __syncthreads();
            double* t = fa;
            fa = fb;
            fb = t;
        }
        if (tid == 0) {
            int best = 0;
            for (int s = 1; s < NS; ++s)
                if (fa[s] < fa[best]) best = s;
            const double v = fa[best];
            const bool open = v < 0.0;
            row_v[r0] = open ? v : 0.0;
            int s = best;
            for (int r = R - 1; r >= 0; --r) {
                const int L = sL[s], Rr = sR[s];
                row_lr[r0 + r] = (open && L < Rr) ? make_int2(L, Rr) : make_int2(0, 0);
                if (r > 0) row_v[r0 + r] = 0.0;
                if (r > 0) s = back[r * NS + s];
            }
        }
    } else if constexpr (MODE == DAO_MLC_CONNECTED) {
        double* m = P + R * C1;                                  // [R]
        int* lr = reinterpret_cast<int*>(m + R);                 // [R][2]
        for (int r = tid; r < R; r += blockDim.x) {
            const double* Pr = P + r * C1;
            double best = INFINITY;
            int bl = 0, br = 0;
            for (int L = 0; L < C; ++L)
                for (int Rr = L + 1; Rr <= C; ++Rr) {
                    const double v = Pr[Rr] - Pr[L];
                    if (v < best) {
                        best = v;
                        bl = L;
                        br = Rr;
                    }
                }
            m[r] = best;
            lr[2 * r] = bl;
            lr[2 * r + 1] = br;
        }
        __syncthreads();
        if (tid == 0) {
            int a = 0, e = 0;
            const double v = mlc_row_search(R, [&](int q) { return m[q]; }, &a, &e);
            const bool open = v < 0.0;
            row_v[r0] = open ? v : 0.0;
            for (int r = 0; r < R; ++r) {
                if (r > 0) row_v[r0 + r] = 0.0;
                row_lr[r0 + r] = (open && r >= a && r < e) ? make_int2(lr[2 * r], lr[2 * r + 1]) : make_int2(0, 0);
            }
        }
    } else {  // DAO_MLC_JAWS
        const int NP = C * C1 / 2;                               // column ranges L < R
        double* pv = P + R * C1;                                 // [NP]
        int* pab = reinterpret_cast<int*>(pv + NP);              // [NP][2]
        for (int p = tid; p < NP; p += blockDim.x) {
            int L = 0, q = p;
            while (q >= C - L) {
                q -= C - L;
                ++L;
            }
            const int Rr = L + 1 + q;
            int a = 0, e = 0;
            pv[p] = mlc_row_search(R, [&](int k) { return P[k * C1 + Rr] - P[k * C1 + L]; }, &a, &e);
            pab[2 * p] = a;
            pab[2 * p + 1] = e;
        }
        __syncthreads();
        if (tid == 0) {
            int best = 0;
            for (int p = 1; p < NP; ++p)
                if (pv[p] < pv[best]) best = p;
            const double v = pv[best];
            const bool open = v < 0.0;
            int L = 0, q = best;
            while (q >= C - L) {
                q -= C - L;
                ++L;
            }
            s_val = v;
            s_L = L;
            s_R = L + 1 + q;
            s_a = open ? pab[2 * best] : 0;
            s_b = open ? pab[2 * best + 1] : 0;
            row_v[r0] = open ? v : 0.0;
        }
        __syncthreads();
        for (int r = tid; r < R; r += blockDim.x) {
            if (r > 0) row_v[r0 + r] = 0.0;
            row_lr[r0 + r] = (r >= s_a && r < s_b) ? make_int2(s_L, s_R) : make_int2(0, 0);
        }
    }
}

template <int MODE>
cudaError_t mlc_launch(const float* w, const int* beam_off, const int* rows, const int* cols, const int* beam_row0,
                       int n_beams, size_t smem, double* row_v, int2* row_lr, const int* skip, cudaStream_t stream) {
    k_price_mlc<MODE><<<n_beams, MLC_THREADS, smem, stream>>>(w, beam_off, rows, cols, beam_row0, row_v, row_lr,
                                                              skip);
    return cudaGetLastError();
}

}  // namespace

size_t mlc_smem_bytes(int mode, int max_rows, int max_cols) {
    const size_t R = (size_t)max_rows, C = (size_t)max_cols, C1 = C + 1;
    switch (mode) {
        case DAO_MLC_INTERDIGITATION: {
            const size_t NS = C1 * (C1 + 1) / 2;
            return 8 * (R * C1 + 2 * NS + C1 * C1) + 4 * C1 * C1 + 2 * R * NS + 2 * NS;
        }
        case DAO_MLC_CONNECTED:
            return 8 * (R * C1 + R) + 8 * R;
        case DAO_MLC_JAWS: {
            const size_t NP = C * C1 / 2;
            return 8 * (R * C1 + NP) + 8 * NP;
        }
    }
    return 0;
}

cudaError_t mlc_configure(int mode, size_t smem) {
    // the attribute is process-wide and plans may be created from several threads
    // at once: the largest size of any plan (64 rows of 32 beamlets), never this
    // plan's own, which another thread's smaller plan could otherwise lower
    if (smem > mlc_smem_bytes(mode, 64, 32)) return cudaErrorInvalidValue;
    smem = mlc_smem_bytes(mode, 64, 32);
    switch (mode) {
        case DAO_MLC_INTERDIGITATION:
            return cudaFuncSetAttribute(k_price_mlc<DAO_MLC_INTERDIGITATION>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        case DAO_MLC_CONNECTED:
            return cudaFuncSetAttribute(k_price_mlc<DAO_MLC_CONNECTED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
        case DAO_MLC_JAWS:
            return cudaFuncSetAttribute(k_price_mlc<DAO_MLC_JAWS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_price_mlc(int mode, const float* w, const int* beam_off, const int* rows, const int* cols,
                             const int* beam_row0, int n_beams, size_t smem, double* row_v, int2* row_lr,
                             const int* skip, cudaStream_t stream, int* launches) {
    if (n_beams == 0) return cudaSuccess;
    cudaError_t e = cudaErrorInvalidValue;
    switch (mode) {
        case DAO_MLC_INTERDIGITATION:
            e = mlc_launch<DAO_MLC_INTERDIGITATION>(w, beam_off, rows, cols, beam_row0, n_beams, smem, row_v, row_lr,
                                                    skip, stream);
            break;
        case DAO_MLC_CONNECTED:
            e = mlc_launch<DAO_MLC_CONNECTED>(w, beam_off, rows, cols, beam_row0, n_beams, smem, row_v, row_lr, skip,
                                              stream);
            break;
        case DAO_MLC_JAWS:
            e = mlc_launch<DAO_MLC_JAWS>(w, beam_off, rows, cols, beam_row0, n_beams, smem, row_v, row_lr, skip,
                                         stream);
            break;
    }
    ++*launches;
    return e;
}

}  // namespace dao
