// Master problem of column-generation DAO (arXiv:1003.5402, Sec. 2.2-2.3):
// min_y F(S y) subject to y >= 0 over the current aperture pool, where column k
// of the slab S (V x K, FP32, column-major with stride ld) is the aperture dose
// D_kj of Eq. 2.
//
// The paper uses gradient projection and gives no step or stopping rule.  This
// is a scaled gradient projection, the projected Newton method of Bertsekas
// (1982): variables with y_k <= eps and g_k > 0 take the plain gradient step,
// the others a Newton step on H = S_F^T diag(h) S_F (h = generalised second
// derivative of the piecewise-quadratic F), with Armijo backtracking along the
// projection arc.  One evaluation is four kernels:
//   k_master_eval   streams the slab in tiles of TILE voxels (2-D TMA bulk
//                   copies completing on an mbarrier) and computes z = S y as a
//                   compensated FP32 dot product (Ogita, Rump & Oishi,
//                   "Accurate sum and dot product", 2005; y split into two
//                   floats), pi = grad F(z), h and F; voxels with h > 0 are the
//                   only ones that contribute to g and H, and their rows, h and
//                   pi are written compacted, per tile, to an active list;
//   k_master_hess   the active list split evenly over the blocks: per-block
//                   partials of H (FP32), g and the rounding scale of g;
//   k_master_reduce fixed-order reduction of the partials;
//   k_master_step   one block: KKT test at the trial point, Armijo test, damped
//                   FP32 Cholesky of the free block of H, next trial point.
// Every kernel returns at once after the state is marked done, so evaluations
// can be queued ahead (or looped on the device by a graph while node).
//
// Stopping rule: |y_k - max(y_k - g_k, 0)| <= tol_rel * max|g(start)| +
// NOISE * u * sum_j |S_jk pi_j| for every k (u = 2^-24), i.e. KKT up to the
// FP32 rounding level of g.  A trial point that meets it is accepted without
// the Armijo test: near the optimum the objective's change is below its own
// rounding and the test would reject an optimal point.
#include <algorithm>

#include "dao_internal.h"

#include <cmath>

namespace dao {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int TILE = MASTER_TILE;   // voxels per evaluation tile = threads per block
constexpr int CH = 128;             // active voxels per Hessian sub-chunk
constexpr float U32 = 5.9604645e-8f;  // 2^-24
constexpr double NOISE = 64.0;
constexpr int WAIT_LIMIT = 1 << 20;   // mbarrier polls before a copy is declared lost
constexpr int HSTRIDE = KMAX * (KMAX + 1) / 2;  // packed curvature entries per block of the kept partial H

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// ---- TMA / mbarrier (sm_90+ PTX) ----------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false if it never completed.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    const unsigned a = smem_addr(bar);
    for (int i = 0; i < WAIT_LIMIT; ++i) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// 2-D tiled bulk copy of box (x, y) of the tensor map into shared memory.
__device__ __forceinline__ void tma_load_2d(float* dst, const CUtensorMap* map, int x, int y,
                                            unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// TwoSum accumulation of a product a*y (y = yh + yl) into the pair (s, c).
__device__ __forceinline__ void dot2_step(float& s, float& c, float a, float yh, float yl) {
    const float p = a * yh;
    float pe = fmaf(a, yh, -p);  // a*yh = p + pe exactly
    pe = fmaf(a, yl, pe);
    const float t2 = s + p;      // TwoSum(s, p)
    const float bb = t2 - s;
    const float e = (s - (t2 - bb)) + (p - bb);
    s = t2;
    c += e + pe;
}

// (rb, cb) of the eb-th 4x4 block of the upper triangle, row-major
__device__ __forceinline__ void block_of(int eb, int KB, int& rb, int& cb) {
    int r = 0, rem = eb;
    while (rem >= KB - r) {
        rem -= KB - r;
        ++r;
    }
    rb = r;
    cb = r + rem;
}

// Packed index of entry (r, c), r <= c, of the upper triangle, column by column:
// c (c + 1) / 2 + r, the same for every pool size K (a partial H kept from one
// pool size to the next keeps its entries in place).
__device__ __forceinline__ int tri_index(int r, int c, int K) {
    (void)K;
    return c * (c + 1) / 2 + r;
}

__global__ void k_master_init(MasterDev* __restrict__ st, int K, const int* __restrict__ skip,
                              cudaGraphConditionalHandle cond, int use_cond, GridBar* __restrict__ gb) {
    const int t = threadIdx.x;
    if (t == 0 && gb != nullptr) {  // a barrier left by an aborted solve starts empty
        gb->count = 0;
        gb->broken = 0;
    }
    if (skip != nullptr && *skip) {  // the solve stopped before this round: nothing to iterate
        if (t == 0) {
            st->done = 1;
            if (use_cond) cudaGraphSetConditional(cond, 0u);
        }
        return;
    }
    if (t < K) {
        const double v = t < K - 1 ? st->y[t] : 0.0;  // warm start: previous optimum, new aperture at 0
        st->yt[t] = v;
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
        st->err = 0;
        st->ticket = 0;
        st->final_pending = 0;
        if (use_cond) cudaGraphSetConditional(cond, 1u);
    }
}

// Graph path: keep the statistics of the master solve that just finished.
__global__ void k_cg_record(const MasterDev* __restrict__ st, CGDev* __restrict__ cg, int K) {
    if (threadIdx.x != 0 || cg->idle) return;
    cg->trace[K - 1] = st->F;
    cg->res[K - 1] = st->res;
    cg->tol[K - 1] = st->tol;
    cg->evals[K - 1] = st->n_eval;
    cg->status[K - 1] = st->status;
}

// ---- evaluation: one slab tile per iteration --------------------------------
// The slab is column-major (column k = the doses of aperture k over all voxels,
// stride ld); a tile is the box of KP columns x TILE voxels, landing in shared
// memory as [KP][TILE].
__global__ void __launch_bounds__(TILE, 3) k_master_eval(const __grid_constant__ CUtensorMap tmap, int V, int K,
                                                         int KP, MasterDev* __restrict__ st,
                                                         float* __restrict__ act_rows, float2* __restrict__ act_hp,
                                                         int* __restrict__ act_count, double* __restrict__ F_part,
                                                         const uint8_t* __restrict__ vstruct,
                                                         const StructTermsF* __restrict__ tf, int S,
                                                         float* __restrict__ z_out, float* __restrict__ pi_out,
                                                         int mode, const int* __restrict__ skip) {
    if (skip != nullptr && *skip) return;
    if (mode == PASS_EVAL && st->done) return;
    const bool final_pass = mode == PASS_FINAL;
    extern __shared__ __align__(128) float As[];  // [KP][TILE]
    __shared__ __align__(8) unsigned long long bar;
    __shared__ float s_yh[KMAX], s_yl[KMAX];
    __shared__ int s_wcount[TILE / 32];
    __shared__ StructTermsF s_tf[SMAX];
    __shared__ float s_red[TILE / 32];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if (tid < KMAX) {
        const double yv = tid < K ? (final_pass ? st->y[tid] : st->yt[tid]) : 0.0;
        const float hi = (float)yv;
        s_yh[tid] = hi;
        s_yl[tid] = (float)(yv - (double)hi);
    }
    for (int i = tid; i < S; i += TILE) s_tf[i] = tf[i];
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    float facc = 0.f;  // this thread's voxels: a few terms, FP32 is enough before the FP64 block sum
    unsigned parity = 0;
    bool lost = false;
    const int n_tiles = (V + TILE - 1) / TILE;
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        __syncthreads();  // every thread is done with the previous tile's buffers
        if (tid == 0 && KP > 0) {
            mbar_expect_tx(&bar, (unsigned)(TILE * KP * sizeof(float)));
            tma_load_2d(As, &tmap, tile * TILE, 0, &bar);
        }
        if (KP > 0) {
            if (!mbar_wait(&bar, parity)) {
                lost = true;
                break;
            }
            parity ^= 1u;
        }
        const int j = tile * TILE + tid;
        // ---- compensated z from this voxel's column of the tile, four chains
        float sc[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int k = 0; k < KP; k += 4) {  // doses of columns K..KP-1 meet y = 0
            dot2_step(sc[0], cc[0], As[k * TILE + tid], s_yh[k], s_yl[k]);
            dot2_step(sc[1], cc[1], As[(k + 1) * TILE + tid], s_yh[k + 1], s_yl[k + 1]);
            dot2_step(sc[2], cc[2], As[(k + 2) * TILE + tid], s_yh[k + 2], s_yl[k + 2]);
            dot2_step(sc[3], cc[3], As[(k + 3) * TILE + tid], s_yh[k + 3], s_yl[k + 3]);
        }
        float s = sc[0], c = cc[0];
#pragma unroll
        for (int q = 1; q < 4; ++q) {
            const float t2 = s + sc[q];
            const float bb = t2 - s;
            const float e = (s - (t2 - bb)) + (sc[q] - bb);
            s = t2;
            c += e + cc[q];
        }
        float h = 0.f, p = 0.f;
        if (j < V) {
            const StructTermsF t = S >= 0 ? s_tf[vstruct[j]] : voxel_terms(tf, j);
            const float du = (t.tu - s) - c;   // T^- - z, exact subtraction near the threshold
            const float dov = (s - t.to) + c;  // z - T^+
            const float u = fmaxf(du, 0.f), o = fmaxf(dov, 0.f);
            p = 2.f * (t.b * o - t.a * u);
            h = 2.f * ((du > 0.f ? t.a : 0.f) + (dov > 0.f ? t.b : 0.f));
            facc = fmaf(t.a * u, u, fmaf(t.b * o, o, facc));
            if (final_pass) {
                z_out[j] = s + c;
                pi_out[j] = p;
            }
        }
        if (final_pass) continue;
        // ---- compact the voxels with non-zero curvature into this tile's slots
        const bool act = h > 0.f;
        const unsigned bal = __ballot_sync(FULL, act);
        if (lane == 0) s_wcount[warp] = __popc(bal);
        __syncthreads();
        int base = 0, n_act = 0;
#pragma unroll
        for (int w = 0; w < TILE / 32; ++w) {
            const int cnt = s_wcount[w];
            base += w < warp ? cnt : 0;
            n_act += cnt;
        }
        if (act) {
            const size_t slot = (size_t)tile * TILE + base + __popc(bal & ((1u << lane) - 1u));
            float4* dst = reinterpret_cast<float4*>(act_rows + slot * KROW);
            for (int k = 0; k < KP; k += 4)
                dst[k / 4] = make_float4(As[k * TILE + tid], As[(k + 1) * TILE + tid], As[(k + 2) * TILE + tid],
                                         As[(k + 3) * TILE + tid]);
            act_hp[slot] = make_float2(h, p);
        }
        if (tid == 0) act_count[tile] = n_act;
    }
    if (lost) {  // a tile copy never arrived: report it, the step kernel stops the solve
        if (tid == 0) st->err = 1;
        return;
    }
    if (final_pass) return;
    // F: FP32 within a warp (32 voxel terms), FP64 across the block's warps
    // (FP64 runs at 1/64 of the FP32 rate here: keep it to a few lanes)
    const float fw = warp_sum_f32(facc);
    if (lane == 0) s_red[warp] = fw;
    __syncthreads();
    if (tid < 32) {
        double t = tid < TILE / 32 ? (double)s_red[tid] : 0.0;
#pragma unroll
        for (int o = TILE / 64; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
        if (tid == 0) F_part[blockIdx.x] = t;
    }
}

// ---- curvature and gradient over the active list ----------------------------
// Block b takes active voxels [M b / G, M (b + 1) / G) in tile order, in
// sub-chunks of CH voxels copied to shared memory as rows of KW floats; thread
// (eb, v) accumulates the 4x4 block eb of H over voxel lane v, and the diagonal
// blocks also g and sum |S_jk pi_j|.
__global__ void __launch_bounds__(256) k_master_hess(const float* __restrict__ act_rows,
                                                     const float2* __restrict__ act_hp,
                                                     const int* __restrict__ act_count, int n_tiles, int K, int KW,
                                                     int NV, MasterDev* __restrict__ st, float* __restrict__ H_part,
                                                     double* __restrict__ g_part, float* __restrict__ gn_part, int G,
                                                     int mode) {
    if (mode == PASS_EVAL && st->done) return;
    // the partial arrays are overwritten: the persistent solve's kept partial H is gone
    if (blockIdx.x == 0 && threadIdx.x == 0) st->inc_G = 0;
    extern __shared__ __align__(16) float smem[];
    int* s_pref = reinterpret_cast<int*>(smem);                        // [n_tiles + 1]
    float* Ac = smem + ((n_tiles + 1 + 3) / 4) * 4;                    // [CH][KW]
    float* s_h = Ac + CH * KW;                                         // [CH]
    float* s_p = s_h + CH;                                             // [CH]
    __shared__ float s_scr[8 * 24];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    // exclusive prefix of the per-tile active counts (integer sums: exact in any
    // order): contiguous chunks per thread, then a scan of the chunk totals
    __shared__ int s_wsum[8];
    {
        const int per = (n_tiles + 255) / 256;
        const int t0 = tid * per, t1 = min(n_tiles, t0 + per);
        int mine = 0;
        for (int t = t0; t < t1; ++t) mine += act_count[t];
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        int before = incl - mine;
        for (int w = 0; w < warp; ++w) before += s_wsum[w];
        for (int t = t0; t < t1; ++t) {
            s_pref[t] = before;
            before += act_count[t];
        }
        if (tid == 255) s_pref[n_tiles] = before;
    }
    const int KP = (K + 3) / 4 * 4;
    const int KB = KP / 4;
    const int nb = KB * (KB + 1) / 2;
    int rb = -1, cb = -1;
    const int v = tid % NV;
    if (tid < nb * NV) block_of(tid / NV, KB, rb, cb);
    __syncthreads();
    const int M = s_pref[n_tiles];
    const int m0 = (int)((long long)M * blockIdx.x / G), m1 = (int)((long long)M * (blockIdx.x + 1) / G);
    const int nq = KP / 4;
    float hs[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) hs[q] = 0.f;
    float gs[4] = {0.f, 0.f, 0.f, 0.f}, gns[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c0 = m0; c0 < m1; c0 += CH) {
        const int n = min(CH, m1 - c0);
        __syncthreads();
        // copy the sub-chunk: two threads per voxel, alternate float4 groups
        {
            const int i = tid >> 1, half = tid & 1;
            if (i < n) {
                const int m = c0 + i;
                int lo = 0, hi = n_tiles;  // last tile with pref <= m
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_pref[mid] <= m) lo = mid; else hi = mid;
                }
                const size_t slot = (size_t)lo * TILE + (m - s_pref[lo]);
                const float4* src = reinterpret_cast<const float4*>(act_rows + slot * KROW);
                float4* dst = reinterpret_cast<float4*>(Ac + i * KW);
                for (int q = half; q < nq; q += 2) dst[q] = src[q];
                if (half == 0) {
                    const float2 hp = act_hp[slot];
                    s_h[i] = hp.x;
                    s_p[i] = hp.y;
                }
            }
        }
        __syncthreads();
        if (rb >= 0) {
            for (int i = v; i < n; i += NV) {
                const float4 ra = *reinterpret_cast<const float4*>(Ac + i * KW + 4 * rb);
                const float4 rc = *reinterpret_cast<const float4*>(Ac + i * KW + 4 * cb);
                const float hv = s_h[i];
                const float a0 = ra.x * hv, a1 = ra.y * hv, a2 = ra.z * hv, a3 = ra.w * hv;
                hs[0] = fmaf(a0, rc.x, hs[0]);
                hs[1] = fmaf(a0, rc.y, hs[1]);
                hs[2] = fmaf(a0, rc.z, hs[2]);
                hs[3] = fmaf(a0, rc.w, hs[3]);
                hs[4] = fmaf(a1, rc.x, hs[4]);
                hs[5] = fmaf(a1, rc.y, hs[5]);
                hs[6] = fmaf(a1, rc.z, hs[6]);
                hs[7] = fmaf(a1, rc.w, hs[7]);
                hs[8] = fmaf(a2, rc.x, hs[8]);
                hs[9] = fmaf(a2, rc.y, hs[9]);
                hs[10] = fmaf(a2, rc.z, hs[10]);
                hs[11] = fmaf(a2, rc.w, hs[11]);
                hs[12] = fmaf(a3, rc.x, hs[12]);
                hs[13] = fmaf(a3, rc.y, hs[13]);
                hs[14] = fmaf(a3, rc.z, hs[14]);
                hs[15] = fmaf(a3, rc.w, hs[15]);
                if (rb == cb) {
                    const float pv = s_p[i], pa = fabsf(pv);
                    gs[0] = fmaf(ra.x, pv, gs[0]);
                    gs[1] = fmaf(ra.y, pv, gs[1]);
                    gs[2] = fmaf(ra.z, pv, gs[2]);
                    gs[3] = fmaf(ra.w, pv, gs[3]);
                    gns[0] = fmaf(fabsf(ra.x), pa, gns[0]);
                    gns[1] = fmaf(fabsf(ra.y), pa, gns[1]);
                    gns[2] = fmaf(fabsf(ra.z), pa, gns[2]);
                    gns[3] = fmaf(fabsf(ra.w), pa, gns[3]);
                }
            }
        }
    }
    // fold the NV voxel lanes of each entry block (consecutive threads) with a
    // fixed shuffle tree, then across warps through shared memory when NV > 32
    float vals[24];
#pragma unroll
    for (int q = 0; q < 16; ++q) vals[q] = hs[q];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        vals[16 + q] = gs[q];
        vals[20 + q] = gns[q];
    }
    const int span = NV < 32 ? NV : 32;
    for (int o = span / 2; o > 0; o >>= 1)
#pragma unroll
        for (int q = 0; q < 24; ++q) vals[q] += __shfl_xor_sync(FULL, vals[q], o);
    if (NV > 32 && lane == 0)
#pragma unroll
        for (int q = 0; q < 24; ++q) s_scr[warp * 24 + q] = vals[q];
    __syncthreads();
    if ((tid % NV) == 0 && tid < nb * NV) {
        if (NV > 32) {
            const int w0 = tid >> 5, nw = NV >> 5;
#pragma unroll
            for (int q = 0; q < 24; ++q) {
                float t = 0.f;
                for (int w = 0; w < nw; ++w) t += s_scr[(w0 + w) * 24 + q];
                vals[q] = t;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int r = 4 * rb + q, col = 4 * cb + e;
                if (r < K && col < K && r <= col) H_part[(size_t)tri_index(r, col, K) * G + blockIdx.x] = vals[q * 4 + e];
            }
        if (rb == cb) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = 4 * rb + q;
                if (r < K) {
                    g_part[(size_t)r * G + blockIdx.x] = (double)vals[16 + q];
                    gn_part[(size_t)r * G + blockIdx.x] = vals[20 + q];
                }
            }
        }
    }
}

// Reduction of the partial sums: one warp per output (packed H entries, then g,
// then the g rounding scale, then F), outputs strided over the grid's warps;
// lanes read the blocks' partials (contiguous per output) and combine them with
// a fixed shuffle tree in FP64.
// Lane's share src[lane], src[lane + 32], ... of n partial sums, added in that
// order (as a plain loop would), with the loads of up to RP_LANE of them issued
// before the first add: in-order issue would otherwise wait for each load at
// its add.  Through L2: the partials were written by other blocks.
constexpr int RP_LANE = 12;
template <class T>
__device__ __forceinline__ T lane_sum_strided(const T* __restrict__ src, int n, int lane) {
    T s = T(0);
    for (int b0 = 0; b0 < n; b0 += 32 * RP_LANE) {
        T v[RP_LANE];
#pragma unroll
        for (int q = 0; q < RP_LANE; ++q) {
            const int b = b0 + lane + 32 * q;
            v[q] = b < n ? __ldcg(src + b) : T(0);
        }
#pragma unroll
        for (int q = 0; q < RP_LANE; ++q) s += v[q];
    }
    return s;
}

// The partial arrays hold GC columns (the blocks that wrote them) at stride GH.
__device__ __forceinline__ void master_reduce_part(const float* __restrict__ H_part,
                                                   const double* __restrict__ g_part,
                                                   const float* __restrict__ gn_part,
                                                   const double* __restrict__ F_part, int GH, int GC, int GE, int K,
                                                   MasterDev* __restrict__ st, int bid, int nblocks) {
    const int E = K * (K + 1) / 2;
    const int lane = threadIdx.x & 31;
    const int n_out = E + 2 * K + 1;
    for (int o = (bid * (int)blockDim.x + (int)threadIdx.x) >> 5; o < n_out; o += (nblocks * (int)blockDim.x) >> 5) {
        if (o < E) {  // the factorisation is FP32: so is this sum
            float s = lane_sum_strided(H_part + (size_t)o * GH, GC, lane);
            s = warp_sum_f32(s);
            if (lane == 0) {  // o = c (c + 1) / 2 + r, r <= c
                int c = (int)((sqrtf(8.f * (float)o + 1.f) - 1.f) * 0.5f);
                while ((c + 1) * (c + 2) / 2 <= o) ++c;
                while (c * (c + 1) / 2 > o) --c;
                const int r = o - c * (c + 1) / 2;
                st->Ht[r * KMAX + c] = s;
                st->Ht[c * KMAX + r] = s;
            }
        } else if (o < E + K) {
            const int k = o - E;
            double s = lane_sum_strided(g_part + (size_t)k * GH, GC, lane);
            s = warp_sum_f64(s);
            if (lane == 0) st->gt[k] = s;
        } else if (o < E + 2 * K) {
            const int k = o - E - K;
            float s = lane_sum_strided(gn_part + (size_t)k * GH, GC, lane);
            s = warp_sum_f32(s);
            if (lane == 0) st->gn[k] = s;
        } else {
            double s = lane_sum_strided(F_part, GE, lane);
            s = warp_sum_f64(s);
            if (lane == 0) st->Ft = s;
        }
    }
}

// Block-wide reductions over STEP_T threads with a fixed order.
constexpr int STEP_T = 256;
constexpr int STEP_W = STEP_T / 32;
// Thread roles in a panel of the step's factorisation: warps 0-5 update the
// rows of the trailing tiles, warp 6 writes the panel's final columns and
// pivots, warp 7 eliminates the right-hand side.
constexpr int FACT_TILE_T = 192, FACT_COLW = 192, FACT_RHSW = 224;
static_assert(STEP_T == 256 && KMAX == 64, "the step kernel maps a 16 x 16 thread grid onto 64 x 64 entries");

// Maximum over the warp of non-negative doubles: their IEEE bit patterns order
// like their values, so a 64-bit integer maximum is exact and stays off the
// FP64 pipe (1/64 of the FP32 rate on this part).  A NaN counts as 0, as
// fmax would skip it.
__device__ __forceinline__ long long nonneg_bits(double v) { return __double_as_longlong(v == v ? v : 0.0); }
__device__ __forceinline__ double warp_max_nonneg(double v) {
    long long b = nonneg_bits(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b = max(b, __shfl_xor_sync(FULL, b, o));
    return __longlong_as_double(b);
}

__device__ __forceinline__ float blk_max_f32(float v, float* sw) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = sw[0];
#pragma unroll
    for (int w = 1; w < STEP_W; ++w) t = fmaxf(t, sw[w]);
    return t;
}


// One block: thread k < K owns variable k; all threads share the factorisation.
__device__ __forceinline__ void master_step_body(MasterDev* __restrict__ st, int max_iter, double tol_rel,
                                                 double sigma) {
    __shared__ __align__(16) float A[KMAX][KMAX + 4];   // working lower triangle
    __shared__ __align__(16) float Lw[KMAX][KMAX + 4];  // final panel columns, L_ik d_k
    __shared__ __align__(16) float u[KMAX];             // right-hand side being eliminated
    __shared__ __align__(16) float ye[KMAX];            // eliminated right-hand side
    __shared__ float piv[KMAX];
    __shared__ float rd[KMAX];
    __shared__ float rhs[KMAX];
    __shared__ float sg[KMAX];                          // FP32 gradient at the accepted point
    __shared__ float swf[STEP_W];
    __shared__ int fidx[KMAX];
    __shared__ double sw[STEP_W];
    __shared__ double sw2[STEP_W];
    __shared__ double sw3[STEP_W];
    __shared__ int swi[STEP_W];
    // every value the step reads is loaded up front (independent loads, one round
    // trip); gt, gn, Ft and Ht were written by other blocks of this launch and
    // are read through L2 (__ldcg), never from a possibly stale L1 line
    const int k = threadIdx.x;
    const int kk = k < KMAX ? k : KMAX - 1;
    // (all through L2: a persistent solve runs the step in whichever block
    // finishes last, so no L1 line of another iteration may be trusted)
    const int done = __ldcg(&st->done), err = __ldcg(&st->err), K = __ldcg(&st->K), phase = __ldcg(&st->phase);
    const int iter0 = __ldcg(&st->iter);
    const double tol0 = __ldcg(&st->tol), F0 = __ldcg(&st->F), Ft = __ldcg(&st->Ft);
    const double yt_ = __ldcg(&st->yt[kk]), gt_ = __ldcg(&st->gt[kk]), gn_ = (double)__ldcg(&st->gn[kk]);
    const double y_ = __ldcg(&st->y[kk]), g_ = __ldcg(&st->g[kk]);
    // the curvature matrix, requested now so that its latency passes behind the
    // reductions below; stored to shared memory once the free set is known
    // (entry 256 m + k of the row-major KMAX x KMAX array)
    float hpre[KMAX * KMAX / STEP_T];
#pragma unroll
    for (int m = 0; m < KMAX * KMAX / STEP_T; ++m) hpre[m] = __ldcg(&st->Ht[m * STEP_T + k]);
    if (done) return;
    if (err) {  // a tile copy was lost in an evaluation: stop with the last accepted point
        if (threadIdx.x == 0) {
            st->status = MASTER_ERROR;
            st->final_pending = 1;
            st->done = 1;
        }
        return;
    }
    const bool own = k < K;
    // only the first nw warps hold variables (K <= 64): they alone run the FP64
    // reductions, which issue at 1/64 of the FP32 rate on this part
    const int nw = (K + 31) >> 5;
    const bool vwarp = (k >> 5) < nw;
    const double yt = own ? yt_ : 0.0, gt = own ? gt_ : 0.0, gn = own ? gn_ : 0.0;
    const double y = own ? y_ : 0.0, g = own ? g_ : 0.0;
    // tolerance of this solve from the gradient at the warm start
    double tol = tol0;
    if (phase == 0) {
        if (vwarp) {
            const double m = warp_max_nonneg(own ? fabs(gt) : 0.0);
            if ((k & 31) == 0) sw3[k >> 5] = m;
        }
        __syncthreads();
        long long mb = nonneg_bits(sw3[0]);
        for (int w = 1; w < nw; ++w) mb = max(mb, nonneg_bits(sw3[w]));
        tol = tol_rel * fmax(__longlong_as_double(mb), 1e-300);
        if (k == 0) st->tol = tol;
    }
    // KKT violation flag, residual and Armijo decrease in one reduction
    double rmax = 0.0, dec = 0.0;
    int viol = 0;
    if (vwarp) {
        const double rt = own ? fabs(yt - fmax(yt - gt, 0.0)) : 0.0;
        viol = __any_sync(FULL, own && rt > tol + NOISE * (double)U32 * gn) ? 1 : 0;
        rmax = warp_max_nonneg(rt);
        dec = own ? g * (yt - y) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dec += __shfl_xor_sync(FULL, dec, o);
        if ((k & 31) == 0) {
            sw[k >> 5] = rmax;
            sw2[k >> 5] = dec;
            swi[k >> 5] = viol;
        }
    }
    __syncthreads();
    long long rb = nonneg_bits(sw[0]);
    dec = sw2[0];
    viol = swi[0];
    for (int w = 1; w < nw; ++w) {
        rb = max(rb, nonneg_bits(sw[w]));
        dec += sw2[w];
        viol |= swi[w];
    }
    rmax = __longlong_as_double(rb);
    const bool cap = iter0 >= max_iter + 64;
    const bool accept = !cap && (phase == 0 || !viol || Ft <= F0 + sigma * dec);
    if (k == 0) st->n_eval = __ldcg(&st->n_eval) + 1;
    if (cap) {
        if (k == 0) {
            st->status = MASTER_MAXITER;
            st->final_pending = 1;
            st->done = 1;
        }
        return;
    }
    if (!accept) {
        const double alpha = __ldcg(&st->alpha) * 0.5;
        if (alpha < 9.3e-10) {  // 2^-30: the line search found no decrease
            if (k == 0) {
                st->status = MASTER_STALLED;
                st->final_pending = 1;
                st->done = 1;
            }
            return;
        }
        if (own) st->yt[k] = fmax(y + alpha * __ldcg(&st->d[k]), 0.0);
        if (k == 0) {
            st->alpha = alpha;
            st->iter = iter0 + 1;
            st->phase = 1;
        }
        return;
    }
    // accept the trial point
    if (own) {
        st->y[k] = yt;
        st->g[k] = gt;
    }
    if (k == 0) {
        st->F = Ft;
        st->res = rmax;
    }
    if (!viol || iter0 >= max_iter) {
        if (k == 0) {
            st->status = viol ? MASTER_MAXITER : MASTER_CONVERGED;
            st->done = 1;
        }
        return;
    }
    // epsilon-active set, free variables compacted in order
    bool active = false;
    if (vwarp) {
        const double eps = fmin(1e-3, rmax);
        active = own && yt <= eps && gt > 0.0;
    }
    const bool fr = own && !active;
    const unsigned bal = __ballot_sync(FULL, fr);
    __syncthreads();
    if ((k & 31) == 0) swi[k >> 5] = __popc(bal);
    __syncthreads();
    int nf = 0, pos = 0;
#pragma unroll
    for (int w = 0; w < STEP_W; ++w) {
        pos += w < (k >> 5) ? swi[w] : 0;
        nf += swi[w];
    }
    pos += __popc(bal & ((1u << (k & 31)) - 1u));
    if (fr) fidx[pos] = k;
#pragma unroll
    for (int m = 0; m < KMAX * KMAX / STEP_T; ++m) {  // H into Lw (overwritten later by the factorisation)
        const int idx = m * STEP_T + k;
        Lw[idx / KMAX][idx % KMAX] = hpre[m];
    }
    if (k < KMAX) sg[k] = (float)gt;
    double d = active ? -gt : 0.0;
    __syncthreads();
    // Damped FP32 L D L^T factorisation of H_FF with the forward solve folded in,
    // by panels of 4 columns with one barrier per panel.  The working lower
    // triangle A lives in shared memory.  For panel p (columns c0 = 4p .. c0+3)
    // the threads that need it factor the 4 x 4 diagonal block themselves
    // (identical arithmetic everywhere) and map rows through it, w = x L11^-T:
    //   - work item 4 t + a < 4 nb(nb+1)/2 (threads below FACT_TILE_T, strided)
    //     takes row a of trailing tile t = (r, s), s <= r, and subtracts
    //     w_R D^-1 w_Q^T from it (the trailing part shrinks, so do the items);
    //   - threads FACT_COLW + r' write the panel's final column entries w
    //     (unscaled: L_ik d_k) of row block r' into Lw, and the pivots d and
    //     their reciprocals;
    //   - thread FACT_RHSW writes the eliminated right-hand side of the panel
    //     into ye, threads FACT_RHSW + r subtract its contribution from row
    //     block r of u.
    // Rows nf .. 4*panels-1 are padding with only the shift on the diagonal.  The
    // pivots are checked once at the end; one that is not in [2^-126, 2^126]
    // (non-positive, or outside the range of the reciprocal approximation)
    // restarts the factorisation with a 100x larger shift.  Then L^T x = D^-1 ye
    // is solved by warp 0 with the unit lower factor L_ik = Lw_ik / d_k.
    const int ti = k >> 4, tq = k & 15;
    const int n_panels = (nf + 3) >> 2;
    const int n4 = 4 * n_panels;
    float Hr[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = ti + 16 * a, q = tq + 16 * b;
            Hr[a][b] = (i < nf && q <= i) ? Lw[fidx[i]][fidx[q]] : 0.f;
        }
    const float bk = k < nf ? -sg[fidx[k]] : 0.f;
    float dg = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) dg = fmaxf(dg, (ti == tq) ? Hr[a][a] : 0.f);
    const float maxdiag = blk_max_f32(dg, swf);
    float lam = 1e-6f * maxdiag + 1e-30f;
    bool ok = false;
    for (int attempt = 0; attempt < 6 && !ok; ++attempt) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = ti + 16 * a, q = tq + 16 * b;
                A[i][q] = Hr[a][b] + ((i == q && i < n4) ? lam : 0.f);
            }
        if (k < KMAX) u[k] = bk;
        __syncthreads();
        for (int p = 0; p < n_panels; ++p) {
            const int c0 = 4 * p;
            const int nb = n_panels - p - 1;
            const int ntile4 = 2 * nb * (nb + 1);  // rows of the nb (nb + 1) / 2 trailing tiles
            const bool tilew = k < FACT_TILE_T && k < ntile4;
            const bool colw = k >= FACT_COLW && k <= FACT_COLW + nb;
            const bool rhsw = k >= FACT_RHSW && k <= FACT_RHSW + nb;
            if (tilew || colw || rhsw) {
                const float4 a0 = *reinterpret_cast<const float4*>(&A[c0][c0]);
                const float4 a1 = *reinterpret_cast<const float4*>(&A[c0 + 1][c0]);
                const float4 a2 = *reinterpret_cast<const float4*>(&A[c0 + 2][c0]);
                const float4 a3 = *reinterpret_cast<const float4*>(&A[c0 + 3][c0]);
                // the pivot reciprocals on the chain of every panel: the hardware
                // approximation (__fdividef, within 2 ulp for pivots in
                // [2^-126, 2^126]; a pivot outside that range fails the check
                // below and the factorisation restarts with a larger shift)
                const float d0 = a0.x, i0 = __fdividef(1.f, d0);
                const float l10 = a1.x * i0;
                const float d1 = a1.y - l10 * a1.x, i1 = __fdividef(1.f, d1);
                const float l20 = a2.x * i0, w21 = a2.y - l10 * a2.x, l21 = w21 * i1;
                const float d2 = a2.z - l20 * a2.x - l21 * w21, i2 = __fdividef(1.f, d2);
                const float l30 = a3.x * i0, w31 = a3.y - l10 * a3.x, l31 = w31 * i1;
                const float w32 = a3.z - l20 * a3.x - l21 * w31, l32 = w32 * i2;
                const float d3 = a3.w - l30 * a3.x - l31 * w31 - l32 * w32, i3 = __fdividef(1.f, d3);
                auto xform = [&](float4 x) {
                    float4 w;
                    w.x = x.x;
                    w.y = x.y - l10 * w.x;
                    w.z = x.z - l20 * w.x - l21 * w.y;
                    w.w = x.w - l30 * w.x - l31 * w.y - l32 * w.z;
                    return w;
                };
                if (tilew) {
                    // one row a of trailing tile t per work item; the four rows of
                    // a tile run in parallel
                    for (int it = k; it < ntile4; it += FACT_TILE_T) {
                        const int t = it >> 2, a = it & 3;
                        int r = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
                        while ((r + 1) * (r + 2) / 2 <= t) ++r;
                        while (r * (r + 1) / 2 > t) --r;
                        const int R = c0 + 4 + 4 * r, Q = c0 + 4 + 4 * (t - r * (r + 1) / 2);
                        float4 wq[4];
#pragma unroll
                        for (int b = 0; b < 4; ++b) wq[b] = xform(*reinterpret_cast<const float4*>(&A[Q + b][c0]));
                        float4 w = xform(*reinterpret_cast<const float4*>(&A[R + a][c0]));
                        w.x *= i0;
                        w.y *= i1;
                        w.z *= i2;
                        w.w *= i3;
                        float4 tt = *reinterpret_cast<const float4*>(&A[R + a][Q]);
                        tt.x -= w.x * wq[0].x + w.y * wq[0].y + w.z * wq[0].z + w.w * wq[0].w;
                        tt.y -= w.x * wq[1].x + w.y * wq[1].y + w.z * wq[1].z + w.w * wq[1].w;
                        tt.z -= w.x * wq[2].x + w.y * wq[2].y + w.z * wq[2].z + w.w * wq[2].w;
                        tt.w -= w.x * wq[3].x + w.y * wq[3].y + w.z * wq[3].z + w.w * wq[3].w;
                        *reinterpret_cast<float4*>(&A[R + a][Q]) = tt;
                    }
                } else if (colw) {
                    const int R = c0 + 4 * (k - FACT_COLW);
#pragma unroll
                    for (int a = 0; a < 4; ++a)
                        *reinterpret_cast<float4*>(&Lw[R + a][c0]) =
                            xform(*reinterpret_cast<const float4*>(&A[R + a][c0]));
                    if (k == FACT_COLW) {
                        piv[c0] = d0;
                        piv[c0 + 1] = d1;
                        piv[c0 + 2] = d2;
                        piv[c0 + 3] = d3;
                        rd[c0] = i0;
                        rd[c0 + 1] = i1;
                        rd[c0 + 2] = i2;
                        rd[c0 + 3] = i3;
                    }
                } else {
                    const float4 e = xform(*reinterpret_cast<const float4*>(&u[c0]));
                    if (k == FACT_RHSW) {
                        *reinterpret_cast<float4*>(&ye[c0]) = e;
                    } else {
                        const int R = c0 + 4 * (k - FACT_RHSW);
                        const float e0 = e.x * i0, e1 = e.y * i1, e2 = e.z * i2, e3 = e.w * i3;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const float4 w = xform(*reinterpret_cast<const float4*>(&A[R + a][c0]));
                            u[R + a] -= w.x * e0 + w.y * e1 + w.z * e2 + w.w * e3;
                        }
                    }
                }
            }
            __syncthreads();
        }
        const float pk = k < n4 ? piv[k] : 1.f, rk = k < n4 ? rd[k] : 1.f;
        ok = __syncthreads_and(pk >= 1.17549435e-38f && pk <= 8.50705917e37f && isfinite(rk)) != 0;
        lam *= 100.f;
    }
    if (ok) {
        if (k >= nf && k < KMAX) rd[k] = 0.f;  // padding rows
        __syncthreads();
        // L^T x = D^-1 ye by warp 0, one pivot at a time from the last, with
        // L_ik = Lw_ik / d_k: lanes keep b_r = ye_r - sum_{i > r, done} Lw_ir x_i
        // for rows r = lane and lane + 32; x_j = b_j / d_j is broadcast from its
        // lane and every row above j takes its term (one shuffle and one FMA
        // per pivot on the dependent chain)
        if (k < 32) {
            float b0 = k < n4 ? ye[k] : 0.f, b1 = k + 32 < n4 ? ye[k + 32] : 0.f;
            const float r0 = rd[k], r1 = rd[k + 32];
            for (int j = nf - 1; j >= 0; --j) {
                const float xj = __shfl_sync(FULL, j < 32 ? b0 * r0 : b1 * r1, j & 31);
                if (k == (j & 31)) {
                    if (j < 32)
                        b0 = xj;
                    else
                        b1 = xj;
                }
                if (k < j) b0 = fmaf(-Lw[j][k], xj, b0);
                if (k + 32 < j) b1 = fmaf(-Lw[j][k + 32], xj, b1);
            }
            rhs[k] = b0;
            rhs[k + 32] = b1;
        }
        __syncthreads();
        if (fr) d = (double)rhs[pos];
    } else if (fr) {
        const double hk = (double)__ldcg(&st->Ht[k * KMAX + k]);
        d = -gt / (hk > 0.0 ? hk : 1.0);
    }
    if (own) {
        st->d[k] = d;
        st->yt[k] = fmax(yt + d, 0.0);
    }
    if (k == 0) {
        st->alpha = 1.0;
        st->iter = iter0 + 1;
        st->phase = 1;
    }
}

// Reduction of the evaluation's partial sums, then the step: every block reduces
// its share of the outputs, and the block that finishes last (a ticket taken
// after a memory fence, so all outputs are visible to it) takes the step.  No
// block waits for another.  The while-node condition is set to "not done" on
// every path that continues; the evaluation cap inside the step guarantees that
// done is reached.
__global__ void __launch_bounds__(STEP_T, 1) k_master_reduce_step(const float* __restrict__ H_part,
                                                               const double* __restrict__ g_part,
                                                               const float* __restrict__ gn_part,
                                                               const double* __restrict__ F_part, int GH, int GE,
                                                               MasterDev* __restrict__ st, int max_iter,
                                                               double tol_rel, double sigma,
                                                               cudaGraphConditionalHandle cond, int use_cond) {
    __shared__ int s_last;
    if (st->done) {  // the same for every block: only the last block of a launch changes it
        if (use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    master_reduce_part(H_part, g_part, gn_part, F_part, GH, GH, GE, st->K, st, blockIdx.x, gridDim.x);
    __syncthreads();
    if (threadIdx.x == 0) s_last = atom_add_acq_rel_gpu(&st->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    if (threadIdx.x == 0) st->ticket = 0;
    master_step_body(st, max_iter, tol_rel, sigma);
    if (use_cond && threadIdx.x == 0) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// ---- the master solve as one persistent cooperative kernel -------------------
// All blocks are co-resident (cooperative launch).  Block b owns the chunks of
// CHV = 128 voxels b, b + G, b + 2G, ... of the slab (interleaved, so the active
// voxels of a compact target spread evenly over the blocks).  Per Newton
// iteration:
//   A. the chunk's slab columns arrive in shared memory by TMA (boxes of 128
//      voxels x 16 columns, one mbarrier; the next chunk's copy is in flight
//      while the current one is folded in, and the block's first chunk is
//      fetched again for the next iteration as soon as its last one has been
//      read: the slab does not change during a solve); warps 0-3 (lane = voxel)
//      compute the compensated z, then pi, h, F, and copy the rows of the
//      voxels with h > 0 to a compacted row-major buffer; every thread then
//      accumulates its 4x4 block of the partial H (and g and the rounding
//      scale of g) over those rows; after its chunks the block writes its
//      partials to column b of the partial arrays;
//   grid barrier;
//   B. every block reduces its share of the outputs in a fixed order; the block
//      that finishes last (ticket after a fence) takes the Newton step;
//   grid barrier; stop when the step marked the solve done.
// Every barrier wait is bounded: after GRID_WAIT_LIMIT polls the block reports
// st->err = 2, marks the barrier broken (later launches of the solve return at
// entry) and every block leaves at the next barrier or check.
constexpr int PT = STEP_T;         // threads per block (the step body's layout)
constexpr int PW = PT / 32;
constexpr int CHV = 128;           // voxels per chunk of the persistent pass
constexpr int BOXC = 16;           // slab columns per TMA box of the persistent pass
constexpr int NST_MAX = 4;         // copies in flight per block (when the pool is small enough)
enum { MODE_FULL = 0, MODE_EXT = 1, MODE_INC = 2 };  // the kept partial H: rebuilt, extended by a column, updated
constexpr int GRID_WAIT_LIMIT = 1 << 22;
constexpr size_t PERSIST_SMEM_MAX = 150 * 1024;  // dynamic shared memory the kernel is configured for

// Barrier over the blocks of one cooperative launch with one acquire-release
// atomic per arrival.  The counter only grows: barrier e of a launch completes when it
// reaches base + (e + 1) G.  base, the counter at launch, is a multiple of G
// (each completed barrier adds exactly G), and every block reads it before its
// first arrival, when fewer than G arrivals can have happened, so
// base = c - c % G for whatever value c it reads.  Waiters poll the counter.
// The host zeroes it before each solve; a solve's barriers stay far below
// 2^32 arrivals.  *s_target is the block's next target.
__device__ __forceinline__ bool grid_sync(GridBar* gb, unsigned nblocks, unsigned* s_target, int* s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = *s_target + nblocks;
        *s_target = target;
        // release: the block's writes (ordered by the __syncthreads above)
        // before the arrival; acquire: the other blocks' writes after it
        const unsigned arrived = atom_add_acq_rel_gpu(&gb->count, 1u) + 1u;
        int ok = 1;
        if (arrived != target) {
            int i = 0;
            while ((int)(ld_acquire_gpu(&gb->count) - target) < 0 && ++i < GRID_WAIT_LIMIT) __nanosleep(64);
            ok = i < GRID_WAIT_LIMIT;
            if (!ok) atomicExch(&gb->broken, 1u);
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// BATCH: one launch for several plans, blocks [g GB, (g + 1) GB) solving the
// master problem of tasks[g] with its own barrier and partial arrays (the
// plans' solves run side by side, each on GB blocks); otherwise one plan, t1,
// on the whole grid.  Every other difference is the block's index within its
// group (bid) and the group's size (G).
// The master solve of one plan (a task) by a group of G co-resident blocks, bid
// the block's index in it; pm the dynamic shared memory, s_target / s_flag the
// group barrier's shared state (s_target: the block's next target, already
// based on the barrier counter).  Every block of the group calls it with the
// same K.
__device__ __forceinline__ void master_solve_group(
    const float* __restrict__ slab, const CUtensorMap* tmap, int ld, int V, int GS, int S, int max_iter,
    MasterDev* __restrict__ st,
    GridBar* __restrict__ gb, float* __restrict__ H_part, double* __restrict__ g_part, float* __restrict__ gn_part,
    double* __restrict__ F_part, const uint8_t* __restrict__ vstruct, const StructTermsF* __restrict__ tf,
    double tol_rel, float* __restrict__ z_out, float* __restrict__ pi_out, CGDev* __restrict__ cg,
    uint8_t* __restrict__ vstate, float* __restrict__ H_keep, int bid, int G, int K, int KP, int KW, int NV,
    double sigma, float* pm,
    unsigned* s_target, int* s_flag) {
    float* stage = pm;                                // [KMAX][CHV] slab columns of a chunk (TMA, 128-byte aligned)
    float* Arow = stage + KMAX * CHV;                 // [CHV][KW] rows of the chunk's active voxels
    float* s_ch = Arow + CHV * KW;                    // [CHV] their change of h
    float* s_cp = s_ch + CHV;                         // [CHV] their pi
    float* s_ho = s_cp + CHV;                         // [CHV] their previous h (first evaluation after a new column)
    int* s_dl = reinterpret_cast<int*>(s_ho + CHV);   // [CHV] slots of the rows whose h changed
    __shared__ float s_zs[CHV], s_zc[CHV];
    __shared__ unsigned s_bu[CHV / 32], s_bd[CHV / 32];
    __shared__ float s_ga[PT], s_gna[PT], s_ea[PT];  // [lane set][column]
    __shared__ int s_mode0;
    __shared__ __align__(8) unsigned long long s_bars[NST_MAX];
    __shared__ float s_yh[KMAX], s_yl[KMAX];
    __shared__ StructTermsF s_tf[SMAX];
    __shared__ float s_red[PW];
    __shared__ float s_scr[8 * 24];
    __shared__ int s_last, s_stop;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < S; i += PT) s_tf[i] = tf[i];
    const int KB = KP / 4;
    const int nb = KB * (KB + 1) / 2;
    int rb = -1, cb = -1;
    const int vl = tid % NV;
    if (tid < nb * NV) block_of(tid / NV, KB, rb, cb);
    const int n32 = (V + 31) / 32;
    const int tiles_b = bid < n32 ? (n32 - 1 - bid) / G + 1 : 0;
    // the block's chunks: bid, bid + G, bid + 2G, ...
    const int n_ch = (V + CHV - 1) / CHV;
    const int chunks_b = bid < n_ch ? (n_ch - 1 - bid) / G + 1 : 0;
    auto chunk_of = [&](int m) { return bid + m * G; };
    // copies in flight: nst stages of nbox boxes each, copy n (n = 0, 1, ... over
    // the launch) holding position n mod chunks_b in stage n mod nst
    // a copy: KP / 16 boxes of 16 columns, then (KP mod 16) / 4 of 4 columns
    const int nbox = KP / BOXC, nbox4 = (KP % BOXC) / 4;
    const int nst = max(1, min(NST_MAX, KMAX / KP));
    const int stage_floats = KP * CHV;
    int n_use = 0, n_iss = 0;  // copies consumed (every thread), issued (thread 0)
    bool lost = false;
    // z by column halves: thread (half, v), columns [k0h, k1h); g by column kq
    // and lane set ls (PT / KP lane sets: the fewer the columns, the more rows
    // each column's sums are split over)
    const int half = tid / CHV, v = tid % CHV;
    const int KH = KP / 8 * 4;
    const int k0h = half ? KH : 0, k1h = half ? KP : KH;
    const int nls = PT / KP;
    const int kq = tid % KP, ls = tid / KP;
    int n_ev = 0;  // evaluations of this solve so far
    auto issue = [&](int n) {  // thread 0
        const int sidx = n % nst;
        float* dst = stage + sidx * stage_floats;
        mbar_expect_tx(&s_bars[sidx], (unsigned)(stage_floats * sizeof(float)));
        const int c = chunk_of(n % chunks_b);
        for (int q = 0; q < nbox; ++q) tma_load_2d(dst + q * BOXC * CHV, tmap, c * CHV, q * BOXC, &s_bars[sidx]);
        for (int q = 0; q < nbox4; ++q)
            tma_load_2d(dst + (nbox * BOXC + 4 * q) * CHV, tmap + 1, c * CHV, nbox * BOXC + 4 * q, &s_bars[sidx]);
    };
    // warm start (every block computes it; block 0 also writes the solver
    // state): the previous optimum, the new aperture K - 1 at 0
    if (tid < KMAX) {
        const double yv = tid < K - 1 ? __ldcg(&st->y[tid]) : 0.0;
        const float hi = (float)yv;
        s_yh[tid] = hi;
        s_yl[tid] = (float)(yv - (double)hi);
        if (bid == 0 && tid < K) {
            st->yt[tid] = yv;
            st->d[tid] = 0.0;
        }
    }
    if (bid == 0 && tid == 0) {
        st->K = K;
        st->iter = 0;
        st->phase = 0;
        st->done = 0;
        st->status = MASTER_RUNNING;
        st->alpha = 1.0;
        st->n_eval = 0;
        st->err = 0;
        st->ticket = 0;
        st->final_pending = 0;
    }
    if (tid < NST_MAX) mbar_init(&s_bars[tid], 1);
    if (tid == 0) {  // the kept partial H: extend it by the new column, keep it, or rebuild it
        const int iG = __ldcg(&st->inc_G), iK = __ldcg(&st->inc_K);
        s_mode0 = iG == G && iK == K - 1 ? MODE_EXT : iG == G && iK == K ? MODE_INC : MODE_FULL;
    }
    __syncthreads();
    if (tid == 0 && chunks_b > 0)  // the first nst copies; the slab does not change during the solve
        for (; n_iss < nst; ++n_iss) issue(n_iss);
    const int mode0 = s_mode0;
    bool first = true;
    for (;;) {
        if (!first) {  // the state of the previous step (all blocks read it after the barrier)
            if (tid == 0) s_stop = __ldcg(&st->done) | __ldcg(&st->err);
            if (tid < KMAX) {
                const double yv = tid < K ? __ldcg(&st->yt[tid]) : 0.0;
                const float hi = (float)yv;
                s_yh[tid] = hi;
                s_yl[tid] = (float)(yv - (double)hi);
            }
            __syncthreads();
            if (s_stop) break;
        }
        first = false;
        // ---- A. the block's chunks of CHV voxels in turn.  The chunk's slab
        // columns arrive in a stage buffer ([16 q][CHV] per box of 16 columns,
        // TMA, copies in flight ahead).  Per chunk:
        //   z: thread (half, v) takes the compensated products of voxel v over
        //      its half of the columns (four chains); half 1 hands its pair to
        //      half 0, which forms z, pi, h, F and the voxel's curvature state;
        //   rows: the rows of the voxels with h > 0 now or at the previous
        //      evaluation go, compacted, to Arow (each half copies its own
        //      columns), with pi, the change of h and (first evaluation after a
        //      new column) the previous h; then the next copy is issued;
        //   every thread folds the rows in: g, the rounding scale of g and the
        //      new column's curvature row by column (four lane sets), and the
        //      change of H by 4x4 blocks over the rows whose h changed.
        // The block's partial H is kept from one evaluation to the next (it is
        // updated by the changes of h only); the first evaluation of a solve
        // extends it by the new column, or rebuilds it when it is not valid.
        const int mode = n_ev == 0 ? mode0 : MODE_INC;
        float facc = 0.f;
        float hs[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) hs[q] = 0.f;
        float ga = 0.f, gna = 0.f, ea = 0.f;
        int nd_blk = 0;  // rows of the block whose h changed (uniform)
        // the voxel's label and curvature state, one chunk ahead (their latency
        // passes behind the previous chunk's work)
        auto voxel_in = [&](int m, int& lab_, unsigned& osv_) {
            const int jj = chunk_of(m) * CHV + v;
            const bool own = !half && m < chunks_b && jj < V;
            lab_ = own && S >= 0 ? (int)vstruct[jj] : 0;
            osv_ = own && mode != MODE_FULL ? (unsigned)vstate[jj] : 0u;
        };
        int lab_n = 0;
        unsigned osv_n = 0u;
        voxel_in(0, lab_n, osv_n);
        for (int m = 0; m < chunks_b && !lost; ++m) {
            const int sidx = n_use % nst;
            const float* stage_c = stage + sidx * stage_floats;
            const int j = chunk_of(m) * CHV + v;
            const int lab = lab_n;
            const unsigned osv = osv_n;
            voxel_in(m + 1, lab_n, osv_n);
            const bool got = mbar_wait(&s_bars[sidx], (unsigned)((n_use / nst) & 1));
            float sc[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = k0h; k < k1h; k += 4) {  // columns K..KP-1 are zero and meet y = 0
                dot2_step(sc[0], cc[0], stage_c[k * CHV + v], s_yh[k], s_yl[k]);
                dot2_step(sc[1], cc[1], stage_c[(k + 1) * CHV + v], s_yh[k + 1], s_yl[k + 1]);
                dot2_step(sc[2], cc[2], stage_c[(k + 2) * CHV + v], s_yh[k + 2], s_yl[k + 2]);
                dot2_step(sc[3], cc[3], stage_c[(k + 3) * CHV + v], s_yh[k + 3], s_yl[k + 3]);
            }
            float s = sc[0], c = cc[0];
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                const float t2 = s + sc[q];
                const float bb = t2 - s;
                const float e = (s - (t2 - bb)) + (sc[q] - bb);
                s = t2;
                c += e + cc[q];
            }
            if (half) {
                s_zs[v] = s;
                s_zc[v] = c;
            }
            if (__syncthreads_or(!got)) {  // a copy never arrived: stop issuing, report it
                lost = true;
                break;
            }
            float p = 0.f, dh = 0.f, hold = 0.f;
            bool uni = false;
            if (!half) {
                {  // TwoSum of the halves' sums
                    const float s1 = s_zs[v];
                    const float t2 = s + s1;
                    const float bb = t2 - s;
                    const float e = (s - (t2 - bb)) + (s1 - bb);
                    s = t2;
                    c += e + s_zc[v];
                }
                float h = 0.f;
                if (j < V) {
                    const StructTermsF t = S >= 0 ? s_tf[lab] : voxel_terms(tf, j);
                    const float du = (t.tu - s) - c;
                    const float dov = (s - t.to) + c;
                    const float u = fmaxf(du, 0.f), o = fmaxf(dov, 0.f);
                    p = 2.f * (t.b * o - t.a * u);
                    h = 2.f * ((du > 0.f ? t.a : 0.f) + (dov > 0.f ? t.b : 0.f));
                    facc = fmaf(t.a * u, u, fmaf(t.b * o, o, facc));
                    z_out[j] = s + c;  // the state of the round when this point is the final one
                    pi_out[j] = p;
                    const unsigned nsv = (du > 0.f ? 1u : 0u) | (dov > 0.f ? 2u : 0u);
                    hold = 2.f * (((osv & 1u) ? t.a : 0.f) + ((osv & 2u) ? t.b : 0.f));
                    dh = h - hold;
                    if (nsv != osv || mode == MODE_FULL) vstate[j] = (uint8_t)nsv;
                }
                uni = h > 0.f || hold > 0.f;
                const unsigned bu = __ballot_sync(FULL, uni);
                const unsigned bd = __ballot_sync(FULL, uni && dh != 0.f);
                if (lane == 0) {
                    s_bu[warp] = bu;
                    s_bd[warp] = bd;
                }
            }
            __syncthreads();
            int n_u = 0, base = 0, n_d = 0, based = 0;
            const int wv = v >> 5;  // the voxel's warp in half 0
#pragma unroll
            for (int w = 0; w < CHV / 32; ++w) {
                const int cu = __popc(s_bu[w]), cd = __popc(s_bd[w]);
                base += w < wv ? cu : 0;
                based += w < wv ? cd : 0;
                n_u += cu;
                n_d += cd;
            }
            const unsigned lt = (1u << lane) - 1u;
            if ((s_bu[wv] >> lane) & 1u) {
                const int slot = base + __popc(s_bu[wv] & lt);
                float4* dst = reinterpret_cast<float4*>(Arow + slot * KW);
                for (int q = k0h / 4; q < k1h / 4; ++q)
                    dst[q] = make_float4(stage_c[(4 * q) * CHV + v], stage_c[(4 * q + 1) * CHV + v],
                                         stage_c[(4 * q + 2) * CHV + v], stage_c[(4 * q + 3) * CHV + v]);
                if (!half) {
                    s_cp[slot] = p;
                    s_ch[slot] = dh;
                    s_ho[slot] = mode == MODE_EXT ? hold : 0.f;
                    if ((s_bd[wv] >> lane) & 1u) s_dl[based + __popc(s_bd[wv] & lt)] = slot;
                }
            }
            __syncthreads();  // the stage is free, the chunk's rows are in Arow
            if (tid == 0) issue(n_iss++);  // copy n_use + nst into the freed stage
            ++n_use;
            nd_blk += n_d;
            // g, the rounding scale of g and the new column's curvature row
            if (kq < K && ls < nls) {
                if (mode == MODE_EXT) {
                    for (int i = ls; i < n_u; i += nls) {
                        const float a = Arow[i * KW + kq], pv = s_cp[i];
                        ga = fmaf(a, pv, ga);
                        gna = fmaf(fabsf(a), fabsf(pv), gna);
                        ea = fmaf(a * s_ho[i], Arow[i * KW + K - 1], ea);
                    }
                } else {
                    for (int i = ls; i < n_u; i += nls) {
                        const float a = Arow[i * KW + kq], pv = s_cp[i];
                        ga = fmaf(a, pv, ga);
                        gna = fmaf(fabsf(a), fabsf(pv), gna);
                    }
                }
            }
            // the change of H over the rows whose h changed
            if (rb >= 0) {
                for (int ii = vl; ii < n_d; ii += NV) {
                    const int i = s_dl[ii];
                    const float4 ra = *reinterpret_cast<const float4*>(Arow + i * KW + 4 * rb);
                    const float4 rc = *reinterpret_cast<const float4*>(Arow + i * KW + 4 * cb);
                    const float hv = s_ch[i];
                    const float a0 = ra.x * hv, a1 = ra.y * hv, a2 = ra.z * hv, a3 = ra.w * hv;
                    hs[0] = fmaf(a0, rc.x, hs[0]);
                    hs[1] = fmaf(a0, rc.y, hs[1]);
                    hs[2] = fmaf(a0, rc.z, hs[2]);
                    hs[3] = fmaf(a0, rc.w, hs[3]);
                    hs[4] = fmaf(a1, rc.x, hs[4]);
                    hs[5] = fmaf(a1, rc.y, hs[5]);
                    hs[6] = fmaf(a1, rc.z, hs[6]);
                    hs[7] = fmaf(a1, rc.w, hs[7]);
                    hs[8] = fmaf(a2, rc.x, hs[8]);
                    hs[9] = fmaf(a2, rc.y, hs[9]);
                    hs[10] = fmaf(a2, rc.z, hs[10]);
                    hs[11] = fmaf(a2, rc.w, hs[11]);
                    hs[12] = fmaf(a3, rc.x, hs[12]);
                    hs[13] = fmaf(a3, rc.y, hs[13]);
                    hs[14] = fmaf(a3, rc.z, hs[14]);
                    hs[15] = fmaf(a3, rc.w, hs[15]);
                }
            }
            // Arow and the lists are next written after the next chunk's first two
            // barriers, which every thread reaches only when done with this chunk
        }
        ++n_ev;
        // ---- the block's partials: F; g, the rounding scale of g and the new
        // column's curvature row (lane sets added in order); H in place
        const float fw = warp_sum_f32(facc);
        if (lane == 0) s_red[warp] = fw;
        if (ls < nls) {
            s_ga[ls * KP + kq] = ga;
            s_gna[ls * KP + kq] = gna;
            s_ea[ls * KP + kq] = ea;
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < PW; ++w) t += (double)s_red[w];
            F_part[bid] = t;
            if (lost) st->err = 1;  // the step stops the solve at the last accepted point
        }
        if (tid < K) {
            float g4 = 0.f, gn4 = 0.f, ext = 0.f;  // lane sets in order
            for (int l = 0; l < nls; ++l) {
                g4 += s_ga[l * KP + tid];
                gn4 += s_gna[l * KP + tid];
                ext += s_ea[l * KP + tid];
            }
            g_part[(size_t)tid * GS + bid] = (double)g4;
            gn_part[(size_t)tid * GS + bid] = gn4;
            if (mode == MODE_EXT) {
                H_keep[(size_t)bid * HSTRIDE + tri_index(tid, K - 1, K)] = ext;
                if (nd_blk == 0) H_part[(size_t)tri_index(tid, K - 1, K) * GS + bid] = ext;
            }
        }
        __syncthreads();  // the new column's row is in place before the changes are added
        if (mode == MODE_FULL || nd_blk > 0) {
            const int span = NV < 32 ? NV : 32;
            for (int o = span / 2; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < 16; ++q) hs[q] += __shfl_xor_sync(FULL, hs[q], o);
            if (NV > 32 && lane == 0)
#pragma unroll
                for (int q = 0; q < 16; ++q) s_scr[warp * 24 + q] = hs[q];
            __syncthreads();
            if ((tid % NV) == 0 && tid < nb * NV) {
                if (NV > 32) {
                    const int w0 = tid >> 5, nw = NV >> 5;
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        float t = 0.f;
                        for (int w = 0; w < nw; ++w) t += s_scr[(w0 + w) * 24 + q];
                        hs[q] = t;
                    }
                }
                float old[16];
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int r = 4 * rb + q, cl = 4 * cb + e;
                        old[q * 4 + e] = mode != MODE_FULL && r < K && cl < K && r <= cl
                                             ? H_keep[(size_t)bid * HSTRIDE + tri_index(r, cl, K)]
                                             : 0.f;
                    }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int r = 4 * rb + q, cl = 4 * cb + e;
                        if (r < K && cl < K && r <= cl) {
                            const float nv = old[q * 4 + e] + hs[q * 4 + e];
                            H_keep[(size_t)bid * HSTRIDE + tri_index(r, cl, K)] = nv;
                            H_part[(size_t)tri_index(r, cl, K) * GS + bid] = nv;
                        }
                    }
            }
        }
        if (!grid_sync(gb, G, s_target, s_flag)) {
            if (tid == 0) st->err = 2;
            break;
        }
        // ---- B. reduction by every block, the step by the last one to finish
        master_reduce_part(H_part, g_part, gn_part, F_part, GS, G, G, K, st, bid, G);
        __syncthreads();
        if (tid == 0) s_last = atom_add_acq_rel_gpu(&st->ticket, 1u) == (unsigned)G - 1u;
        __syncthreads();
        if (s_last) {
            if (tid == 0) st->ticket = 0;
            master_step_body(st, max_iter, tol_rel, sigma);
        }
        if (!grid_sync(gb, G, s_target, s_flag)) {
            if (tid == 0) st->err = 2;
            break;
        }
    }
    if (tid == 0) {
        // no copy of this block outlives the launch (a lost one is not waited for again)
        for (int n = lost ? n_use + 1 : n_use; n < n_iss; ++n) mbar_wait(&s_bars[n % nst], (unsigned)((n / nst) & 1));
        s_stop = __ldcg(&st->err) == 2;
        if (bid == 0) {  // the kept partial H and voxel states are those of the last evaluation
            st->inc_G = __ldcg(&st->err) == 0 ? G : 0;
            st->inc_K = K;
        }
    }
    __syncthreads();
    if (s_stop) return;  // a barrier timed out: the host reports it
    // the solve stopped at an accepted point other than the last one evaluated:
    // z and pi of that point
    if (__ldcg(&st->final_pending)) {
        if (tid < KMAX) {
            const double yv = tid < K ? __ldcg(&st->y[tid]) : 0.0;
            const float hi = (float)yv;
            s_yh[tid] = hi;
            s_yl[tid] = (float)(yv - (double)hi);
        }
        __syncthreads();
        for (int i = warp; i < tiles_b; i += PW) {
            const int j = (bid + i * G) * 32 + lane;
            const bool in = j < V;
            float sc[4] = {0.f, 0.f, 0.f, 0.f}, cc[4] = {0.f, 0.f, 0.f, 0.f};
            const float* col = slab + (in ? j : 0);
            for (int k = 0; k < KP; k += 4) {
                dot2_step(sc[0], cc[0], __ldcg(col + (size_t)k * ld), s_yh[k], s_yl[k]);
                dot2_step(sc[1], cc[1], __ldcg(col + (size_t)(k + 1) * ld), s_yh[k + 1], s_yl[k + 1]);
                dot2_step(sc[2], cc[2], __ldcg(col + (size_t)(k + 2) * ld), s_yh[k + 2], s_yl[k + 2]);
                dot2_step(sc[3], cc[3], __ldcg(col + (size_t)(k + 3) * ld), s_yh[k + 3], s_yl[k + 3]);
            }
            float s = sc[0], c = cc[0];
#pragma unroll
            for (int q = 1; q < 4; ++q) {
                const float t2 = s + sc[q];
                const float bb = t2 - s;
                const float e = (s - (t2 - bb)) + (sc[q] - bb);
                s = t2;
                c += e + cc[q];
            }
            if (in) {
                const StructTermsF t = S >= 0 ? s_tf[vstruct[j]] : voxel_terms(tf, j);
                const float u = fmaxf((t.tu - s) - c, 0.f), o = fmaxf((s - t.to) + c, 0.f);
                z_out[j] = s + c;
                pi_out[j] = 2.f * (t.b * o - t.a * u);
            }
        }
    }
    if (cg != nullptr && bid == 0 && tid == 0) {  // the round's record
        cg->trace[K - 1] = __ldcg(&st->F);
        cg->res[K - 1] = __ldcg(&st->res);
        cg->tol[K - 1] = __ldcg(&st->tol);
        cg->evals[K - 1] = __ldcg(&st->n_eval);
        cg->status[K - 1] = __ldcg(&st->status);
    }
}


template <bool BATCH>
__global__ void __launch_bounds__(PT, 2) k_master_persist(const __grid_constant__ MasterTask t1,
                                                          const MasterTask* __restrict__ tasks,
                                                       int GB, int K, int KP, int KW, int NV, double sigma) {
#define DAO_TASK(f) (BATCH ? tasks[blockIdx.x / GB].f : t1.f)
    const float* __restrict__ slab = DAO_TASK(slab);
    const int ld = DAO_TASK(ld), V = DAO_TASK(V), GS = DAO_TASK(GS), S = DAO_TASK(S), max_iter = DAO_TASK(max_iter);
    const CUtensorMap* tmap = BATCH ? tasks[blockIdx.x / GB].tmap : t1.tmap;
    MasterDev* __restrict__ st = DAO_TASK(st);
    GridBar* __restrict__ gb = DAO_TASK(gb);
    float* __restrict__ H_part = DAO_TASK(H_part);
    double* __restrict__ g_part = DAO_TASK(g_part);
    float* __restrict__ gn_part = DAO_TASK(gn_part);
    double* __restrict__ F_part = DAO_TASK(F_part);
    const uint8_t* __restrict__ vstruct = DAO_TASK(vstruct);
    const StructTermsF* __restrict__ tf = DAO_TASK(tf);
    const double tol_rel = DAO_TASK(tol_rel);
    const int* __restrict__ skip = DAO_TASK(skip);
    float* __restrict__ z_out = DAO_TASK(z_out);
    float* __restrict__ pi_out = DAO_TASK(pi_out);
    CGDev* __restrict__ cg = DAO_TASK(cg);
    uint8_t* __restrict__ vstate = DAO_TASK(vstate);
    float* __restrict__ H_keep = DAO_TASK(H_keep);
#undef DAO_TASK
    const int bid = BATCH ? (int)(blockIdx.x % GB) : (int)blockIdx.x;
    if (K <= 0) {  // pool size from the device (one graph for every round); KW sets the layout below
        K = __ldcg(&cg->K);
        KP = (K + 3) / 4 * 4;
        KW = master_kw(K);
        NV = persist_lanes(K);
    }
    extern __shared__ __align__(128) float pm[];
    __shared__ int s_flag, s_stop0;
    __shared__ unsigned s_target;
    if (skip != nullptr && *skip) return;  // the same for every block
    const int G = BATCH ? GB : (int)gridDim.x;
    if (threadIdx.x == 0) {  // barrier base; a solve whose barrier broke runs no further master solve
        const unsigned c = *reinterpret_cast<volatile unsigned*>(&gb->count);
        s_target = c - c % (unsigned)G;
        s_stop0 = *reinterpret_cast<volatile unsigned*>(&gb->broken) != 0;
    }
    __syncthreads();
    if (s_stop0) return;
    master_solve_group(slab, tmap, ld, V, GS, S, max_iter, st, gb, H_part, g_part, gn_part, F_part, vstruct, tf,
                       tol_rel, z_out, pi_out, cg, vstate, H_keep, bid, G, K, KP, KW, NV, sigma, pm, &s_target,
                       &s_flag);
}


}  // namespace

__host__ __device__ int master_kw(int K) {
    const int KP = (K + 3) / 4 * 4;
    int kw = KP < 4 ? 4 : KP;
    if (((kw / 4) & 1) == 0) kw += 4;  // odd float4 count per row: conflict-free row-per-thread loads
    return kw;
}

size_t master_eval_smem(int K) {
    const int KP = (K + 3) / 4 * 4;
    return (size_t)TILE * (KP > 0 ? KP : 4) * sizeof(float);
}

size_t master_hess_smem(int K, int n_tiles) {
    return (size_t)((n_tiles + 1 + 3) / 4 * 4) * sizeof(int) + (size_t)CH * master_kw(K) * sizeof(float) +
           2 * CH * sizeof(float);
}

// Voxel lanes per 4x4 block of H in the persistent solve: the most (a power of
// two) for which every block of the triangle has its lanes among the 256 threads.
__host__ __device__ int persist_lanes(int K) {
    const int KP = (K + 3) / 4 * 4;
    const int KB = KP / 4;
    const int nb = KB * (KB + 1) / 2;
    int nv = 1;
    while (nb > 0 && nv * 2 * nb <= PT) nv *= 2;
    return nv;
}

__host__ __device__ int master_lanes(int K) {
    const int KP = (K + 3) / 4 * 4;
    const int KB = KP / 4;
    const int nb = KB * (KB + 1) / 2;
    int nv = 1;
    while (nb > 0 && nv * 2 * nb <= 256) nv *= 2;
    return nv;
}

// Blocks of the evaluation kernel for pool size K: all resident at once.
int master_grid(int V, int num_sms, int K) {
    const int n_tiles = (V + TILE - 1) / TILE;
    int occ = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_master_eval, TILE, master_eval_smem(K)) != cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    const int gmax = num_sms * (occ < 4 ? occ : 4);
    return n_tiles < gmax ? (n_tiles > 0 ? n_tiles : 1) : gmax;
}

int master_grid_max(int num_sms) { return 4 * num_sms; }

int master_hess_grid(int num_sms) { return 2 * num_sms; }

// Diagnostic of the bounded barrier wait: a cooperative launch of `blocks`
// blocks meets at grid_sync, except block `absent`, which leaves without
// arriving.  The others must give up after GRID_WAIT_LIMIT polls, mark the
// barrier broken and report (out[0] = blocks that gave up, out[1] = blocks
// that passed).  Nothing faults and every wait ends.
__global__ void k_barrier_check(GridBar* gb, int absent, int* out) {
    __shared__ unsigned s_target;
    __shared__ int s_flag;
    if (threadIdx.x == 0) s_target = 0;
    if ((int)blockIdx.x == absent) return;  // the whole block leaves: it never arrives
    const bool ok = grid_sync(gb, gridDim.x, &s_target, &s_flag);
    if (threadIdx.x == 0) atomicAdd(&out[ok ? 1 : 0], 1);
}

cudaError_t launch_barrier_check(GridBar* gb, int blocks, int absent, int* out, cudaStream_t stream) {
    void* args[] = {(void*)&gb, (void*)&absent, (void*)&out};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(32);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, (const void*)k_barrier_check, args);
}

cudaError_t master_configure() {
    cudaError_t e = cudaFuncSetAttribute(k_master_eval, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)master_eval_smem(KMAX));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_master_persist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)PERSIST_SMEM_MAX);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_master_persist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)PERSIST_SMEM_MAX);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_master_hess, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_master_init(MasterDev* st, int K, const int* skip, cudaGraphConditionalHandle cond,
                               int use_cond, cudaStream_t stream, int* launches, GridBar* gb) {
    k_master_init<<<1, KMAX, 0, stream>>>(st, K, skip, cond, use_cond, gb);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_master_eval(const MasterBuffers& mb, int V, int K, const uint8_t* vstruct, const StructTermsF* tf,
                               int S, float* z_out, float* pi_out, int mode, const int* skip, cudaStream_t stream,
                               int* launches) {
    const int KP = (K + 3) / 4 * 4;
    k_master_eval<<<mb.grid[K], TILE, master_eval_smem(K), stream>>>(
        mb.tmap[KP / 4], V, K, KP, mb.st, mb.act_rows, mb.act_hp, mb.act_count, mb.F_part, vstruct, tf, S, z_out,
        pi_out, mode, skip);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_master_hess(const MasterBuffers& mb, int K, int mode, cudaStream_t stream, int* launches) {
    k_master_hess<<<mb.GH, 256, master_hess_smem(K, mb.n_tiles), stream>>>(
        mb.act_rows, mb.act_hp, mb.act_count, mb.n_tiles, K, master_kw(K), master_lanes(K), mb.st, mb.H_part,
        mb.g_part, mb.gn_part, mb.GH, mode);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_master_step(int K, const MasterBuffers& mb, int max_iter, double tol_rel,
                               cudaGraphConditionalHandle cond, int use_cond, cudaStream_t stream, int* launches) {
    const int outs = K * (K + 1) / 2 + 2 * K + 1;
    k_master_reduce_step<<<(outs + STEP_W - 1) / STEP_W, STEP_T, 0, stream>>>(
        mb.H_part, mb.g_part, mb.gn_part, mb.F_part, mb.GH, mb.grid[K], mb.st, max_iter, tol_rel, 1e-4, cond,
        use_cond);
    ++*launches;
    return cudaGetLastError();
}

// Dynamic shared memory of the persistent solve, the same for every voxel count
// and grid size: the TMA stage (KMAX columns of a chunk), the chunk's active
// rows at the widest row stride, their h and pi.
size_t master_persist_smem(int V, int G) {
    (void)V;
    (void)G;
    return (size_t)KMAX * CHV * sizeof(float) + (size_t)CHV * master_kw(KMAX) * sizeof(float) +
           4 * (size_t)CHV * sizeof(float);
}

// Co-resident blocks of the persistent solve: 2 per SM when they fit, else 1;
// 0 when a cooperative launch is not possible.  want > 0: that many blocks, or
// the least number whose per-block working set fits the shared memory, if
// more (at most the full count).
int master_persist_grid(int V, int num_sms, int want) {
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return 0;
    }
    if (want > 0) {
        int occ = 0;
        for (int G = want; G <= 2 * num_sms; ++G) {
            const size_t smem = master_persist_smem(V, G);
            if (smem > PERSIST_SMEM_MAX) continue;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_master_persist<false>, PT, smem) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            if (occ >= 1 && G <= occ * num_sms) return G;
        }
    }
    for (int per = 2; per >= 1; --per) {
        const int G = per * num_sms;
        const size_t smem = master_persist_smem(V, G);
        if (smem > PERSIST_SMEM_MAX) continue;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_master_persist<false>, PT, smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (occ >= per) return G;
    }
    return 0;
}

cudaError_t launch_master_persist(const MasterBuffers& mb, const float* slab, int ld, int V, int K,
                                  const uint8_t* vstruct, const StructTermsF* tf, int S, int max_iter, double tol_rel,
                                  const int* skip, float* z_out, float* pi_out, CGDev* cg, cudaStream_t stream,
                                  int* launches) {
    const int G = mb.GP;
    if (G < 1) return cudaErrorInvalidConfiguration;
    if (K <= 0 && cg == nullptr) return cudaErrorInvalidValue;
    int KP = K > 0 ? (K + 3) / 4 * 4 : 0;
    int KW = K > 0 ? master_kw(K) : 0, NV = K > 0 ? persist_lanes(K) : 0;
    MasterTask t{};
    t.tmap[0] = mb.tmap_p[0];
    t.tmap[1] = mb.tmap_p[1];
    t.vstate = mb.vstate;
    t.H_keep = mb.H_keep;
    t.slab = slab;
    t.ld = ld;
    t.V = V;
    t.GS = mb.GH;  // partial arrays: stride GH >= G
    t.S = S;
    t.max_iter = max_iter;
    t.st = mb.st;
    t.gb = mb.bar;
    t.H_part = mb.H_part;
    t.g_part = mb.g_part;
    t.gn_part = mb.gn_part;
    t.F_part = mb.F_part;
    t.vstruct = vstruct;
    t.tf = tf;
    t.tol_rel = tol_rel;
    t.skip = skip;
    t.z_out = z_out;
    t.pi_out = pi_out;
    t.cg = cg;
    const MasterTask* none = nullptr;
    int GB = 0;
    double sigma = 1e-4;
    void* args[] = {(void*)&t, (void*)&none, (void*)&GB, (void*)&K, (void*)&KP, (void*)&KW, (void*)&NV,
                    (void*)&sigma};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = master_persist_smem(V, G);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, (const void*)k_master_persist<false>, args);
    ++*launches;
    return e;
}

int master_batch_group(int n_tasks, int num_sms) {
    // two co-resident blocks per SM (the shared memory per block is capped)
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_master_persist<true>, PT, master_persist_smem(0, 0)) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    occ = std::min(occ, 2);
    return n_tasks > 0 ? occ * num_sms / n_tasks : 0;
}

cudaError_t launch_master_persist_batch(const MasterTask* tasks, int n_tasks, int GB, int max_V, cudaStream_t stream,
                                        int* launches) {
    if (n_tasks < 1 || GB < 1) return cudaErrorInvalidConfiguration;
    int K = 0, KP = 0, KW = 0, NV = 0;  // each group reads its pool size from its plan's device state
    MasterTask none{};
    double sigma = 1e-4;
    void* args[] = {(void*)&none, (void*)&tasks, (void*)&GB, (void*)&K, (void*)&KP, (void*)&KW, (void*)&NV,
                    (void*)&sigma};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_tasks * GB);
    cfg.blockDim = dim3(PT);
    cfg.dynamicSmemBytes = master_persist_smem(max_V, GB);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, (const void*)k_master_persist<true>, args);
    ++*launches;
    return e;
}

cudaError_t launch_cg_record(const MasterDev* st, CGDev* cg, int K, cudaStream_t stream, int* launches) {
    k_cg_record<<<1, 32, 0, stream>>>(st, cg, K);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace dao
