// Master problem of column-generation DAO (arXiv:1003.5402, Sec. 2.2-2.3):
// min_y F(S y) subject to y >= 0 over the current aperture pool, where column k
// of the slab S (V x K, FP32, column-major) is the aperture dose D_kj of Eq. 2.
//
// The paper uses gradient projection and gives no step or stopping rule.  This
// is a scaled gradient projection, the projected Newton method of Bertsekas
// (1982): variables with y_k <= eps and g_k > 0 take the plain gradient step,
// the others a Newton step on H = S_F^T diag(h) S_F (h = generalised second
// derivative of the piecewise-quadratic F), with Armijo backtracking along the
// projection arc.  Each evaluation is three kernels:
//   k_master_pass    one fused pass over the slab at the trial point: z = S y,
//                    pi = grad F(z), h, F (FP64), and per-block partials of
//                    g = S^T pi (FP64) and H (FP32);
//   k_master_reduce  fixed-order reduction of the partials (one warp per entry);
//   k_master_step    one block: Armijo test, KKT residual, Cholesky (FP64) of
//                    the free block of H, next trial point.
// Every kernel returns at once after the state is marked done, so the host can
// queue several evaluations ahead and poll the flag.
#include "dao_internal.h"

#include <cmath>

namespace dao {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TILE = MASTER_TILE;
constexpr int LDA = TILE + 1;  // padded stride of the shared slab tile (bank spread)

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__global__ void k_master_init(MasterDev* __restrict__ st, int K) {
    const int t = threadIdx.x;
    if (t < K) {
        const double v = t < K - 1 ? st->y[t] : 0.0;  // warm start: previous optimum, new aperture at 0
        st->yt[t] = v;
        st->yf[t] = (float)v;
        st->d[t] = 0.0;
    }
    if (t == 0) {
        st->K = K;
        st->iter = 0;
        st->phase = 0;
        st->done = 0;
        st->status = MASTER_RUNNING;
        st->alpha = 1.0;
        st->n_eval = 0;
    }
}

__global__ void __launch_bounds__(TILE) k_master_pass(const float* __restrict__ slab, int V, int ld, int K, int KP,
                                                      MasterDev* __restrict__ st, float* __restrict__ H_part,
                                                      double* __restrict__ g_part, double* __restrict__ F_part, int G,
                                                      const uint8_t* __restrict__ vstruct,
                                                      const StructTermsF* __restrict__ tf,
                                                      const StructTermsD* __restrict__ td, int S,
                                                      float* __restrict__ z_out, float* __restrict__ pi_out,
                                                      int final_pass) {
    if (!final_pass && st->done) return;
    extern __shared__ float As[];  // [KP][LDA]
    __shared__ float s_y[KMAX];
    __shared__ float s_h[TILE];
    __shared__ float s_p[TILE];
    __shared__ StructTermsF s_tf[SMAX];
    __shared__ StructTermsD s_td[SMAX];
    __shared__ double s_red[TILE / 32];
    const int tid = threadIdx.x;
    if (tid < K) s_y[tid] = final_pass ? (float)st->y[tid] : st->yf[tid];
    for (int i = tid; i < S; i += TILE) {
        s_tf[i] = tf[i];
        s_td[i] = td[i];
    }
    // thread roles of the curvature / gradient phase: 4x4 blocks of the upper
    // triangle of H, then one thread per gradient entry
    const int KB = KP / 4;
    const int nb = KB * (KB + 1) / 2;
    int rb = -1, cb = -1;
    if (!final_pass && tid < nb) {
        int r = 0, rem = tid;
        while (rem >= KB - r) {
            rem -= KB - r;
            ++r;
        }
        rb = r;
        cb = r + rem;
    }
    const int gk = (!final_pass && tid >= nb && tid < nb + K) ? tid - nb : -1;
    __syncthreads();

    float hs[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) hs[q] = 0.f;
    double gsum = 0.0, facc = 0.0;
    const int n_tiles = (V + TILE - 1) / TILE;
    for (int tile = blockIdx.x; tile < n_tiles; tile += G) {
        const int j = tile * TILE + tid;
        const bool valid = j < V;
        float z = 0.f;
        for (int k = 0; k < K; ++k) {
            const float a = valid ? __ldg(slab + (size_t)k * ld + j) : 0.f;
            As[k * LDA + tid] = a;
            z = fmaf(a, s_y[k], z);
        }
        for (int k = K; k < KP; ++k) As[k * LDA + tid] = 0.f;
        float h = 0.f, p = 0.f;
        if (valid) {
            const int s = vstruct[j];
            const StructTermsF t = s_tf[s];
            const float u = fmaxf(0.f, t.tu - z);
            const float o = fmaxf(0.f, z - t.to);
            p = 2.f * (t.b * o - t.a * u);
            h = 2.f * ((z < t.tu ? t.a : 0.f) + (z > t.to ? t.b : 0.f));
            const StructTermsD td_ = s_td[s];
            const double zd = z;
            const double ud = fmax(0.0, td_.tu - zd);
            const double od = fmax(0.0, zd - td_.to);
            facc += td_.a * ud * ud + td_.b * od * od;
            if (final_pass) {
                z_out[j] = z;
                pi_out[j] = p;
            }
        }
        if (!final_pass) {
            s_h[tid] = h;
            s_p[tid] = p;
            __syncthreads();
            if (rb >= 0) {
                const float* r0 = As + (4 * rb) * LDA;
                const float* c0 = As + (4 * cb) * LDA;
                for (int t = 0; t < TILE; ++t) {
                    const float hv = s_h[t];
                    const float a0 = r0[t] * hv, a1 = r0[LDA + t] * hv, a2 = r0[2 * LDA + t] * hv,
                                a3 = r0[3 * LDA + t] * hv;
                    const float b0 = c0[t], b1 = c0[LDA + t], b2 = c0[2 * LDA + t], b3 = c0[3 * LDA + t];
                    hs[0] = fmaf(a0, b0, hs[0]);
                    hs[1] = fmaf(a0, b1, hs[1]);
                    hs[2] = fmaf(a0, b2, hs[2]);
                    hs[3] = fmaf(a0, b3, hs[3]);
                    hs[4] = fmaf(a1, b0, hs[4]);
                    hs[5] = fmaf(a1, b1, hs[5]);
                    hs[6] = fmaf(a1, b2, hs[6]);
                    hs[7] = fmaf(a1, b3, hs[7]);
                    hs[8] = fmaf(a2, b0, hs[8]);
                    hs[9] = fmaf(a2, b1, hs[9]);
                    hs[10] = fmaf(a2, b2, hs[10]);
                    hs[11] = fmaf(a2, b3, hs[11]);
                    hs[12] = fmaf(a3, b0, hs[12]);
                    hs[13] = fmaf(a3, b1, hs[13]);
                    hs[14] = fmaf(a3, b2, hs[14]);
                    hs[15] = fmaf(a3, b3, hs[15]);
                }
            } else if (gk >= 0) {
                const float* a = As + gk * LDA;
                float ga = 0.f;
                for (int t = 0; t < TILE; ++t) ga = fmaf(a[t], s_p[t], ga);
                gsum += (double)ga;
            }
            __syncthreads();
        }
    }
    if (!final_pass) {
        if (rb >= 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int r = 4 * rb + q, cc = 4 * cb + c;
                    if (r < K && cc < K && r <= cc) H_part[(size_t)(r * KMAX + cc) * G + blockIdx.x] = hs[q * 4 + c];
                }
        }
        if (gk >= 0) g_part[(size_t)gk * G + blockIdx.x] = gsum;
        double v = warp_sum_f64(facc);
        if ((tid & 31) == 0) s_red[tid >> 5] = v;
        __syncthreads();
        if (tid < 32) {
            double t = tid < TILE / 32 ? s_red[tid] : 0.0;
            t = warp_sum_f64(t);
            if (tid == 0) F_part[blockIdx.x] = t;
        }
    }
}

// One warp per output: H entries (r <= c), then g, then F.
__global__ void __launch_bounds__(256) k_master_reduce(const float* __restrict__ H_part,
                                                       const double* __restrict__ g_part,
                                                       const double* __restrict__ F_part, int G,
                                                       MasterDev* __restrict__ st) {
    if (st->done) return;
    const int K = st->K;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nH = K * K;
    if (warp < nH) {
        const int r = warp / K, c = warp % K;
        if (r > c) return;
        double s = 0.0;
        const float* src = H_part + (size_t)(r * KMAX + c) * G;
        for (int i = lane; i < G; i += 32) s += (double)src[i];
        s = warp_sum_f64(s);
        if (lane == 0) {
            st->Ht[r * KMAX + c] = s;
            st->Ht[c * KMAX + r] = s;
        }
    } else if (warp < nH + K) {
        const int k = warp - nH;
        double s = 0.0;
        const double* src = g_part + (size_t)k * G;
        for (int i = lane; i < G; i += 32) s += src[i];
        s = warp_sum_f64(s);
        if (lane == 0) st->gt[k] = s;
    } else if (warp == nH + K) {
        double s = 0.0;
        for (int i = lane; i < G; i += 32) s += F_part[i];
        s = warp_sum_f64(s);
        if (lane == 0) st->Ft = s;
    }
}

__global__ void __launch_bounds__(256) k_master_step(MasterDev* __restrict__ st, int max_iter, double tol_rel,
                                                     double sigma) {
    __shared__ double L[KMAX][KMAX + 1];
    __shared__ double rhs[KMAX];
    __shared__ int fidx[KMAX];
    __shared__ int s_nf, s_ok, s_accept, s_stop;
    __shared__ double s_lam, s_maxdiag;
    if (st->done) return;
    const int K = st->K;
    const int tid = threadIdx.x;
    if (tid == 0) {
        ++st->n_eval;
        s_stop = 0;
        s_nf = 0;
        bool accept;
        if (st->iter >= max_iter + 64) {  // hard cap on evaluations, whatever the line search does
            st->status = MASTER_MAXITER;
            s_stop = 1;
            accept = false;
        } else if (st->phase == 0) {
            accept = true;
        } else {
            double dec = 0.0;
            for (int k = 0; k < K; ++k) dec += st->g[k] * (st->yt[k] - st->y[k]);
            accept = st->Ft <= st->F + sigma * dec;
        }
        s_accept = accept ? 1 : 0;
        if (accept) {
            double res = 0.0, gmax = 0.0;
            for (int k = 0; k < K; ++k) {
                const double y = st->yt[k], g = st->gt[k];
                st->y[k] = y;
                st->g[k] = g;
                res = fmax(res, fabs(y - fmax(y - g, 0.0)));
                gmax = fmax(gmax, fabs(g));
            }
            st->F = st->Ft;
            if (st->phase == 0) st->tol = tol_rel * fmax(gmax, 1e-300);
            st->res = res;
            if (res <= st->tol) {
                st->status = MASTER_CONVERGED;
                s_stop = 1;
            } else if (st->iter >= max_iter) {
                st->status = MASTER_MAXITER;
                s_stop = 1;
            } else {
                const double eps = fmin(1e-3, res);
                int nf = 0;
                for (int k = 0; k < K; ++k) {
                    if (st->y[k] <= eps && st->g[k] > 0.0) {
                        st->d[k] = -st->g[k];
                    } else {
                        fidx[nf++] = k;
                    }
                }
                s_nf = nf;
            }
        } else if (!s_stop) {
            st->alpha *= 0.5;
            if (st->alpha < 1e-12) {
                st->status = MASTER_STALLED;
                s_stop = 1;
            }
        }
    }
    __syncthreads();
    if (s_stop) {
        if (tid == 0) st->done = 1;
        return;
    }
    if (s_accept) {
        const int nf = s_nf;
        for (int idx = tid; idx < nf * nf; idx += blockDim.x) {
            const int i = idx / nf, j = idx % nf;
            L[i][j] = st->Ht[fidx[i] * KMAX + fidx[j]];
        }
        __syncthreads();
        if (tid == 0) {
            double md = 0.0;
            for (int i = 0; i < nf; ++i) md = fmax(md, L[i][i]);
            s_maxdiag = md;
            s_lam = 1e-10 * md;
            s_ok = 0;
        }
        __syncthreads();
        for (int attempt = 0; attempt < 8; ++attempt) {
            if (attempt > 0) {
                for (int idx = tid; idx < nf * nf; idx += blockDim.x) {
                    const int i = idx / nf, j = idx % nf;
                    L[i][j] = st->Ht[fidx[i] * KMAX + fidx[j]];
                }
                __syncthreads();
            }
            for (int i = tid; i < nf; i += blockDim.x) L[i][i] += s_lam;
            if (tid == 0) s_ok = 1;
            __syncthreads();
            for (int j = 0; j < nf; ++j) {
                if (tid == 0) {
                    const double p = L[j][j];
                    if (!(p > 0.0) || !isfinite(p))
                        s_ok = 0;
                    else
                        L[j][j] = sqrt(p);
                }
                __syncthreads();
                if (!s_ok) break;
                const double ljj = L[j][j];
                for (int i = j + 1 + tid; i < nf; i += blockDim.x) L[i][j] /= ljj;
                __syncthreads();
                const int m = nf - j - 1;
                for (int idx = tid; idx < m * m; idx += blockDim.x) {
                    const int i = j + 1 + idx / m, k = j + 1 + idx % m;
                    if (k <= i) L[i][k] -= L[i][j] * L[k][j];
                }
                __syncthreads();
            }
            if (s_ok) break;
            __syncthreads();
            if (tid == 0) s_lam = fmax(s_lam * 100.0, 1e-12 * s_maxdiag + 1e-300);
            __syncthreads();
        }
        if (s_ok) {
            for (int i = tid; i < nf; i += blockDim.x) rhs[i] = -st->g[fidx[i]];
            __syncthreads();
            for (int j = 0; j < nf; ++j) {  // L u = -g_F
                if (tid == 0) rhs[j] /= L[j][j];
                __syncthreads();
                for (int i = j + 1 + tid; i < nf; i += blockDim.x) rhs[i] -= L[i][j] * rhs[j];
                __syncthreads();
            }
            for (int j = nf - 1; j >= 0; --j) {  // L^T d = u
                if (tid == 0) rhs[j] /= L[j][j];
                __syncthreads();
                for (int i = tid; i < j; i += blockDim.x) rhs[i] -= L[j][i] * rhs[j];
                __syncthreads();
            }
            for (int i = tid; i < nf; i += blockDim.x) st->d[fidx[i]] = rhs[i];
        } else {
            // no factorisation: diagonally scaled gradient step on the free set
            for (int i = tid; i < nf; i += blockDim.x) {
                const int k = fidx[i];
                const double hk = st->Ht[k * KMAX + k];
                st->d[k] = -st->g[k] / (hk > 0.0 ? hk : 1.0);
            }
        }
        if (tid == 0) st->alpha = 1.0;
        __syncthreads();
    }
    if (tid < K) {
        const double yt = fmax(st->y[tid] + st->alpha * st->d[tid], 0.0);
        st->yt[tid] = yt;
        st->yf[tid] = (float)yt;
    }
    if (tid == 0) {
        st->iter += 1;
        st->phase = 1;
    }
}

}  // namespace

size_t master_pass_smem(int K) {
    const int KP = (K + 3) / 4 * 4;
    return (size_t)KP * LDA * sizeof(float);
}

cudaError_t master_configure() {
    return cudaFuncSetAttribute(k_master_pass, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)master_pass_smem(KMAX));
}

cudaError_t launch_master_init(MasterDev* st, int K, cudaStream_t stream, int* launches) {
    k_master_init<<<1, KMAX, 0, stream>>>(st, K);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_master_pass(const float* slab, int V, int ld, int K, const MasterBuffers& mb,
                               const uint8_t* vstruct, const StructTermsF* tf, const StructTermsD* td, int S,
                               float* z_out, float* pi_out, int final_pass, cudaStream_t stream, int* launches) {
    const int KP = (K + 3) / 4 * 4;
    k_master_pass<<<mb.G, TILE, master_pass_smem(K), stream>>>(slab, V, ld, K, KP, mb.st, mb.H_part, mb.g_part,
                                                               mb.F_part, mb.G, vstruct, tf, td, S, z_out, pi_out,
                                                               final_pass);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_master_reduce(int K, const MasterBuffers& mb, cudaStream_t stream, int* launches) {
    const int warps = K * K + K + 1;
    k_master_reduce<<<(warps + 7) / 8, 256, 0, stream>>>(mb.H_part, mb.g_part, mb.F_part, mb.G, mb.st);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_master_step(const MasterBuffers& mb, int max_iter, double tol_rel, cudaStream_t stream,
                               int* launches) {
    k_master_step<<<1, 256, 0, stream>>>(mb.st, max_iter, tol_rel, 1e-4);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace dao
