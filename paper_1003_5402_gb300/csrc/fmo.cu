// Beamlet-level fluence map optimisation (FMO), min_{x >= 0} F(D x): the model
// the paper calls mathematically the same as DAO with the beamlet intensities
// as the decision variables (arXiv:1003.5402, Sec. 2.2), solved, as the paper
// says of its own FMO (Sec. 2.3), by gradient projection on the GPU.  Its
// optimum is a lower bound on every DAO objective of the same problem.
//
// Method: projected Newton (Bertsekas 1982) with the Newton system of the free
// beamlets solved inexactly by conjugate gradients.  Per outer iteration:
//   - g = D^T grad F(D x) (the a2 kernel on pi = grad F from the a1 epilogue)
//     and the KKT residual ||x - P(x - g)||_inf;
//   - the epsilon-active set {x_i <= eps, g_i > 0}, eps = min(1e-3, residual),
//     takes the gradient step; the free beamlets take d_F from
//     (D_F^T diag(h) D_F) d_F = -g_F, h the curvature of F at the current dose,
//     by CG until ||r|| <= eta ||g_F|| with eta = min(0.1, sqrt(res / res_0));
//     each CG product is one dose SpMV (a1 without epilogue), a curvature
//     scaling, and one transposed SpMV (a2);
//   - an Armijo rule along the projection arc, F(P(x + a d)) <= F(x) +
//     sigma g^T (P(x + a d) - x), a = 1, 1/2, ...
// Every vector operation on the N beamlets runs in one block with FP64 values
// and fixed-order reductions; the host sequences the launches and reads the
// few scalars that steer the loop (KKT residual, CG stop flag, F, g^T dx).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "dao_internal.h"

namespace dao {

namespace {

constexpr int FV_T = 1024;  // threads of the one-block vector kernels


__device__ __forceinline__ double fv_block_sum(double v, double* s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = s_red[threadIdx.x];  // FV_T / 32 == 32 warps
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) s_red[32] = t;
    }
    __syncthreads();
    t = s_red[32];
    __syncthreads();
    return t;
}

__device__ __forceinline__ double fv_block_max(double v, double* s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = s_red[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (threadIdx.x == 0) s_red[32] = t;
    }
    __syncthreads();
    t = s_red[32];
    __syncthreads();
    return t;
}

// KKT residual ||x - P(x - g)||_inf, and its part beyond the FP32 rounding of
// g: max_i (|x_i - P(x_i - g_i)| - 64 u gn_i), gn = D^T |pi| (u = 2^-24).
__global__ void __launch_bounds__(FV_T) k_fmo_kkt(int N, const double* __restrict__ x, const float* __restrict__ g,
                                                  const float* __restrict__ gn, FmoScalars* __restrict__ st) {
    __shared__ double s_red[33];
    double m = 0.0, mx = 0.0;
    for (int i = threadIdx.x; i < N; i += FV_T) {
        const double r = fabs(x[i] - fmax(x[i] - (double)g[i], 0.0));
        m = fmax(m, r);
        mx = fmax(mx, r - 64.0 * 5.9604644775390625e-08 * (double)gn[i]);
    }
    m = fv_block_max(m, s_red);
    mx = fv_block_max(mx, s_red);
    if (threadIdx.x == 0) {
        st->res = m;
        st->res_x = mx;
    }
}

// |pi| for the rounding scale of g.
__global__ void __launch_bounds__(256) k_fmo_abs(int V, const float* __restrict__ pi, float* __restrict__ out) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < V; j += gridDim.x * blockDim.x) out[j] = fabsf(pi[j]);
}

// The free set {not (x_i <= eps and g_i > 0)}, r = -g_F, p = r, d_F = 0.
__global__ void __launch_bounds__(FV_T) k_fmo_cg_init(int N, const double* __restrict__ x,
                                                      const float* __restrict__ g, double eps, double eta,
                                                      unsigned char* __restrict__ free_, double* __restrict__ r,
                                                      double* __restrict__ p, float* __restrict__ p32,
                                                      double* __restrict__ dF, FmoScalars* __restrict__ st) {
    __shared__ double s_red[33];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += FV_T) {
        const bool fr = !(x[i] <= eps && g[i] > 0.f);
        free_[i] = fr ? 1 : 0;
        const double ri = fr ? -(double)g[i] : 0.0;
        r[i] = ri;
        p[i] = ri;
        p32[i] = (float)ri;
        dF[i] = 0.0;
        s += ri * ri;
    }
    s = fv_block_sum(s, s_red);
    if (threadIdx.x == 0) {
        st->rr = s;
        st->bb = s;
        st->eta = eta;
        st->cg_done = s > 0.0 ? 0 : 1;
        st->cg_iters = 0;
    }
}

// u_j <- h_j u_j, h the curvature of F at the dose z (Eqs. 3-4: 2 alpha below
// the under-dose threshold, 2 beta above the over-dose threshold).
__global__ void __launch_bounds__(256) k_fmo_hmul(int V, const float* __restrict__ z, float* __restrict__ u,
                                                  const uint8_t* __restrict__ vstruct,
                                                  const StructTermsF* __restrict__ tf, int S) {
    __shared__ StructTermsF s_tf[SMAX];
    for (int i = threadIdx.x; i < S; i += blockDim.x) s_tf[i] = tf[i];
    __syncthreads();
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < V; j += gridDim.x * blockDim.x) {
        const StructTermsF t = S >= 0 ? s_tf[vstruct[j]] : voxel_terms(tf, j);
        const float zj = z[j];
        const float h = 2.f * ((zj < t.tu ? t.a : 0.f) + (zj > t.to ? t.b : 0.f));
        u[j] = h * u[j];
    }
}

// One CG iteration on the free set given Ap = D^T diag(h) D p (FP32 SpMVs).
__global__ void __launch_bounds__(FV_T) k_fmo_cg_step(int N, const float* __restrict__ Ap,
                                                      const unsigned char* __restrict__ free_,
                                                      double* __restrict__ r, double* __restrict__ p,
                                                      float* __restrict__ p32, double* __restrict__ dF,
                                                      FmoScalars* __restrict__ st) {
    __shared__ double s_red[33];
    if (st->cg_done) return;  // uniform
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += FV_T)
        if (free_[i]) s += p[i] * (double)Ap[i];
    const double pAp = fv_block_sum(s, s_red);
    const double rr = st->rr;
    if (!(pAp > 0.0)) {  // no curvature left along p: keep d_F as it is
        if (threadIdx.x == 0) st->cg_done = 1;
        return;
    }
    const double alpha = rr / pAp;
    s = 0.0;
    for (int i = threadIdx.x; i < N; i += FV_T) {
        if (!free_[i]) continue;
        dF[i] += alpha * p[i];
        const double ri = r[i] - alpha * (double)Ap[i];
        r[i] = ri;
        s += ri * ri;
    }
    const double rn = fv_block_sum(s, s_red);
    const bool done = sqrt(rn) <= st->eta * sqrt(st->bb);
    const double beta = rn / rr;
    for (int i = threadIdx.x; i < N; i += FV_T) {
        const double pi_ = free_[i] ? r[i] + beta * p[i] : 0.0;
        p[i] = pi_;
        p32[i] = done ? 0.f : (float)pi_;
    }
    if (threadIdx.x == 0) {
        st->rr = rn;
        st->cg_iters += 1;
        st->cg_done = done ? 1 : 0;
    }
}

// Trial point on the projection arc: x_t = max(x + a d, 0) with d = d_F on the
// free set and -g on the active set; g^T (x_t - x).
__global__ void __launch_bounds__(FV_T) k_fmo_trial(int N, const double* __restrict__ x,
                                                    const float* __restrict__ g,
                                                    const unsigned char* __restrict__ free_,
                                                    const double* __restrict__ dF, double a,
                                                    double* __restrict__ xt, float* __restrict__ xt32,
                                                    FmoScalars* __restrict__ st) {
    __shared__ double s_red[33];
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += FV_T) {
        const double d = free_[i] ? dF[i] : -(double)g[i];
        const double v = fmax(x[i] + a * d, 0.0);
        xt[i] = v;
        xt32[i] = (float)v;
        s += (double)g[i] * (v - x[i]);
    }
    s = fv_block_sum(s, s_red);
    if (threadIdx.x == 0) st->gdx = s;
}

}  // namespace

cudaError_t fmo_kkt(int N, const double* x, const float* g, const float* gn, FmoScalars* st, cudaStream_t s) {
    k_fmo_kkt<<<1, FV_T, 0, s>>>(N, x, g, gn, st);
    return cudaGetLastError();
}
cudaError_t fmo_abs(int V, const float* pi, float* out, int num_sms, cudaStream_t s) {
    k_fmo_abs<<<num_sms * 4, 256, 0, s>>>(V, pi, out);
    return cudaGetLastError();
}
cudaError_t fmo_cg_init(int N, const double* x, const float* g, double eps, double eta, unsigned char* free_,
                        double* r, double* p, float* p32, double* dF, FmoScalars* st, cudaStream_t s) {
    k_fmo_cg_init<<<1, FV_T, 0, s>>>(N, x, g, eps, eta, free_, r, p, p32, dF, st);
    return cudaGetLastError();
}
cudaError_t fmo_hmul(int V, const float* z, float* u, const uint8_t* vstruct, const StructTermsF* tf, int S,
                     int num_sms, cudaStream_t s) {
    k_fmo_hmul<<<num_sms * 4, 256, 0, s>>>(V, z, u, vstruct, tf, S);
    return cudaGetLastError();
}
cudaError_t fmo_cg_step(int N, const float* Ap, const unsigned char* free_, double* r, double* p, float* p32,
                        double* dF, FmoScalars* st, cudaStream_t s) {
    k_fmo_cg_step<<<1, FV_T, 0, s>>>(N, Ap, free_, r, p, p32, dF, st);
    return cudaGetLastError();
}
cudaError_t fmo_trial(int N, const double* x, const float* g, const unsigned char* free_, const double* dF, double a,
                      double* xt, float* xt32, FmoScalars* st, cudaStream_t s) {
    k_fmo_trial<<<1, FV_T, 0, s>>>(N, x, g, free_, dF, a, xt, xt32, st);
    return cudaGetLastError();
}

}  // namespace dao
