// Sparse dose kernels of column-generation DAO (arXiv:1003.5402):
//   a1  z = D x with the objective epilogue (Eqs. 1, 5, 7, 9, 10),
//   a2  w = D^T pi from the stored transpose (the bracketed sum of Eq. 8),
//   a4  the dose column of a new aperture, D_kj = sum_{i in A_k} D_ij (Eq. 2),
//   and the beamlet fluence x_i = sum_{k in K_i} y_k (Eq. 7).
// All reductions have a fixed order (per-lane sequential, then a fixed
// shuffle tree, then fixed-order shared-memory combination), so every result
// is bitwise reproducible for a given launch shape.  No atomic accumulation:
// the forms that split rows between warps add the warps' partial sums in a
// fixed order, whichever warp takes the row's last ticket (an atomic counter).
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dao_internal.h"
#include "pricing.cuh"
#include "spmv_body.cuh"

namespace dao {

namespace {

constexpr unsigned FULL = 0xffffffffu;

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

// Sum of one double per thread over the block; the result is valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum_f64(double v, double* s_red) {
    v = warp_sum_f64(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < NT / 32 ? s_red[lane] : 0.0;
        t = warp_sum_f64(t);
    }
    return t;
}

// ---- a1 ---------------------------------------------------------------------
// G lanes per voxel row, rows_per_warp = 32 / G rows per warp; every lane of a
// warp runs the same number of tile iterations so the shuffles stay converged.
template <int G, bool SMEM_X>
__global__ void __launch_bounds__(256) k_dose(const int* __restrict__ rowptr, const int4* __restrict__ col4,
                                              const float4* __restrict__ val4, int V,
                                              const float* __restrict__ x, int N,
                                              const uint8_t* __restrict__ vstruct,
                                              const StructTermsS* __restrict__ ts, int S,
                                              float* __restrict__ z, float* __restrict__ grad,
                                              double* __restrict__ F_part) {
    extern __shared__ float sx[];
    __shared__ StructTermsS s_ts[SMAX];
    __shared__ double s_red[8];
    if (SMEM_X)
        for (int i = threadIdx.x; i < N; i += blockDim.x) sx[i] = x[i];
    for (int i = threadIdx.x; i < S; i += blockDim.x) s_ts[i] = ts[i];
    __syncthreads();
    const float* xs = SMEM_X ? sx : x;
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    constexpr int RPW = 32 / G;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int n_tiles = (V + RPW - 1) / RPW;
    float facc = 0.f;
    for (int t = warp_global; t < n_tiles; t += n_warps) {
        const int row = t * RPW + lane / G;
        float acc = 0.f;
        if (row < V) {
            const int p0 = rowptr[row] >> 2, p1 = rowptr[row + 1] >> 2;
            // two groups of the lane (p, p + G) requested together, summed in order
            for (int p = p0 + sub; p < p1; p += 2 * G) {
                const bool two = p + G < p1;
                const int4 c = __ldg(col4 + p);
                const float4 v = __ldg(val4 + p);
                int4 c2 = make_int4(0, 0, 0, 0);
                float4 v2 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (two) {
                    c2 = __ldg(col4 + p + G);
                    v2 = __ldg(val4 + p + G);
                }
                acc = fmaf(v.x, xs[c.x], acc);
                acc = fmaf(v.y, xs[c.y], acc);
                acc = fmaf(v.z, xs[c.z], acc);
                acc = fmaf(v.w, xs[c.w], acc);
                if (two) {
                    acc = fmaf(v2.x, xs[c2.x], acc);
                    acc = fmaf(v2.y, xs[c2.y], acc);
                    acc = fmaf(v2.z, xs[c2.z], acc);
                    acc = fmaf(v2.w, xs[c2.w], acc);
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (row < V && sub == 0) {
            z[row] = acc;
            if (grad != nullptr || F_part != nullptr) {
                // FP32 epilogue (FP64 issues at 1/64 of the FP32 rate here)
                const StructTermsS tt = S >= 0 ? s_ts[vstruct[row]] : ts[row];
                const float u = fmaxf((tt.tu_hi - acc) + tt.tu_lo, 0.f);  // T^- - z
                const float o = fmaxf((acc - tt.to_hi) - tt.to_lo, 0.f);  // z - T^+
                if (grad != nullptr) grad[row] = 2.f * (tt.b * o - tt.a * u);
                facc = fmaf(tt.a * u, u, fmaf(tt.b * o, o, facc));
            }
        }
    }
    if (F_part != nullptr) {
        const double s = block_sum_mixed<256>(facc, s_red);
        if (threadIdx.x == 0) F_part[blockIdx.x] = s;
    }
}

// Fixed-order sum of n doubles by one block.
__global__ void __launch_bounds__(256) k_sum_f64(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double s_red[8];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) v += part[i];
    const double s = block_sum_f64<256>(v, s_red);
    if (threadIdx.x == 0) *out = s;
}

// ---- a2 ---------------------------------------------------------------------
// The device-driven round (rt.cg != nullptr): block 0 snapshots the pool
// size and the stop flag for the fused commit kernel that follows.
__device__ __forceinline__ void dt_round_snapshot(const RowTicket& rt) {
    if (rt.cg != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
        rt.cg->rs_K = rt.cg->K;
        rt.cg->rs_stop = rt.cg->stop;
    }
}

// The fused MLC-row search: thread 0 has published w[row]; it takes the ticket
// of the row's MLC row, and the block that holds the MLC row's last beamlet
// runs the row search (warp 0) on the row's w, read through L2.
__device__ __forceinline__ void dt_row_ticket(const RowTicket& rt, int row, const float* w) {
    if (rt.row_cnt == nullptr) return;  // uniform
    __shared__ int s_row;
    if (threadIdx.x == 0) {
        const int4 bi = rt.binfo[row];
        const int g = rt.beam_row0[bi.x] + bi.y;
        // release: w[row] before the ticket; acquire: the row's other prices
        const bool last = (int)atom_add_acq_rel_gpu(reinterpret_cast<unsigned*>(&rt.row_cnt[g]), 1u) ==
                          rt.cols[bi.x] - 1;
        if (last) rt.row_cnt[g] = 0;  // every other beamlet of the row has taken its ticket
        s_row = last ? g : -1;
    }
    __syncthreads();
    const int g = s_row;
    // every other block of the row released its w with its ticket; row_best
    // reads w through L2
    if (g >= 0 && threadIdx.x < 32) pricing::row_best(w, rt.row_info[g], g, rt.row_v, rt.row_lr);
}

// One block per beamlet row of D^T; int4/float4 loads of (voxel, value),
// gathered pi from L2; FP32 products, FP64 combination across threads.
// LC: consecutive entries on consecutive threads (dt_row_sum_lc), else groups of
// four entries per thread (dt_row_sum).
template <int BT, bool LC>
__global__ void __launch_bounds__(BT) k_dt(const int* __restrict__ rowptr, const int4* __restrict__ col4,
                                           const float4* __restrict__ val4, int N,
                                           const int* __restrict__ order,
                                           const float* __restrict__ pi, float* __restrict__ w,
                                           const int* __restrict__ skip, RowTicket rt) {
    __shared__ double s_red[BT / 32];
    dt_round_snapshot(rt);
    if (skip != nullptr && *skip) return;
    const int row = order[blockIdx.x];  // longest rows first: they start in the first wave
    const float s = LC ? dt_row_sum_lc<BT>(rowptr, reinterpret_cast<const int*>(col4),
                                           reinterpret_cast<const float*>(val4), row, pi, s_red)
                       : dt_row_sum<BT>(rowptr, col4, val4, row, pi, s_red);
    if (threadIdx.x == 0) w[row] = s;
    dt_row_ticket(rt, row, w);
}

// The fused MLC-row search taken by one warp (all lanes): lane 0 has published
// w[row]; as dt_row_ticket, with the warp's lanes ordered by __syncwarp.
__device__ __forceinline__ void dt_row_ticket_warp(const RowTicket& rt, int row, const float* w) {
    if (rt.row_cnt == nullptr) return;  // uniform
    int g = -1;
    if ((threadIdx.x & 31) == 0) {
        const int4 bi = rt.binfo[row];
        const int gg = rt.beam_row0[bi.x] + bi.y;
        const bool last = (int)atom_add_acq_rel_gpu(reinterpret_cast<unsigned*>(&rt.row_cnt[gg]), 1u) ==
                          rt.cols[bi.x] - 1;
        if (last) rt.row_cnt[gg] = 0;
        g = last ? gg : -1;
    }
    g = __shfl_sync(FULL, g, 0);
    __syncwarp();
    if (g >= 0) pricing::row_best(w, rt.row_info[g], g, rt.row_v, rt.row_lr);
}

// a2 with D^T's entries split evenly over a fixed set of warps: warp v takes
// the entries [v chunk, (v + 1) chunk) in steps of 32 consecutive entries
// (lane l the entry t + l, U steps requested ahead of their pi gathers), so
// every warp streams the same number of bytes whatever the row lengths, and
// the 32 gathers of a step fall on a few cache lines.  Every row has at least
// 32 entries, so a step crosses at most one row end.  At a row end the warp
// sums its lanes (fixed butterfly): a row within the warp's range is final
// (lane 0 writes w[row], times the beamlet scale for 16-bit values); a row
// covered by warps v0 .. v1 stores this warp's sum at slot v - v0.  Only after
// its range does the warp take the tickets of its rows (an acquire-release
// atomic waits for the warp's loads in flight, so none is taken while the
// stream runs): the last of a row's warps adds the slots in order in FP64 and
// writes w[row]; then the fused MLC-row ticket.
constexpr int SPLIT_THREADS = 256;

template <int VK>  // 0: FP32 values, 1: FP16, 2: BF16
__global__ void __launch_bounds__(SPLIT_THREADS) k_dt_split(
    const int* __restrict__ rowptr, const int* __restrict__ col, const void* __restrict__ valv,
    const float* __restrict__ scale, int N, int E, int chunk, int n_warps, const int* __restrict__ split_row,
    float* __restrict__ part, int PS, int* __restrict__ cnt, const float* __restrict__ pi, float* __restrict__ w,
    const int* __restrict__ skip, RowTicket rt) {
    constexpr int U = 4;
    dt_round_snapshot(rt);
    if (skip != nullptr && *skip) return;
    const int lane = threadIdx.x & 31;
    const int wg = blockIdx.x * (SPLIT_THREADS / 32) + (threadIdx.x >> 5);
    if (wg >= n_warps) return;  // uniform per warp
    const int e_begin = wg * chunk;
    const int e_end = min(e_begin + chunk, E);
    auto loadv = [&](int e) -> float {
        if constexpr (VK == 0)
            return __ldg(static_cast<const float*>(valv) + e);
        else
            return unpack1<VK == 2>(__ldg(static_cast<const unsigned short*>(valv) + e));
    };
    auto finish = [&](int r, double tot) {
        w[r] = VK == 0 ? (float)tot : (float)(tot * (double)__ldg(scale + r));
    };
    // three stages in flight: the indices and values of batch k + 2, the pi
    // gathers of batch k + 1, the products of batch k
    int c1[U], c2[U];
    float v0[U], v1[U], v2[U], a0[U], a1[U];
    auto load_batch = [&](int s0, int* cc, float* vv) {
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int e = s0 + 32 * q + lane;
            cc[q] = e < e_end ? __ldg(col + e) : -1;
            vv[q] = e < e_end ? loadv(e) : 0.f;
        }
    };
    auto gather = [&](const int* cc, float* aa) {
#pragma unroll
        for (int q = 0; q < U; ++q) aa[q] = cc[q] >= 0 ? __ldg(pi + cc[q]) : 0.f;
    };
    {
        int c0[U];
        load_batch(e_begin, c0, v0);
        load_batch(e_begin + 32 * U, c1, v1);
        gather(c0, a0);
    }
    // a window of 32 row offsets, lane l holding rowptr[rbase + l]
    const int r_first = __ldg(split_row + wg);
    int rbase = r_first;
    int rp = __ldg(rowptr + min(rbase + lane, N));
    int ri = 0;
    int rstart = __shfl_sync(FULL, rp, 0);
    int rend = __shfl_sync(FULL, rp, 1);
    // a row's sum over this warp's entries: final, or this warp's slot
    auto store = [&](int r, int rs, int re, float a) {
        const float p = warp_sum_f32(a);
        if (lane == 0) {
            const int wa = rs / chunk, wb = (re - 1) / chunk;  // the row's first and last warps
            if (wb > wa)
                part[(size_t)r * PS + (wg - wa)] = p;
            else
                finish(r, (double)p);
        }
    };
    float acc = 0.f;
    for (int s0 = e_begin; s0 < e_end; s0 += 32 * U) {
        load_batch(s0 + 64 * U, c2, v2);
        gather(c1, a1);
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int t = s0 + 32 * q;
            if (t >= e_end) break;  // uniform
            if (rend >= t + 32 || rend >= e_end) {
                acc = fmaf(v0[q], a0[q], acc);  // lanes past e_end add 0 * 0
            } else {
                // the row ends inside this step: lanes below rend finish it
                const int e = t + lane;
                if (e < rend) acc = fmaf(v0[q], a0[q], acc);
                store(rbase + ri, rstart, rend, acc);
                if (++ri == 31) {  // next window of row offsets
                    rbase += 31;
                    rp = __ldg(rowptr + min(rbase + lane, N));
                    ri = 0;
                }
                rstart = rend;
                rend = __shfl_sync(FULL, rp, ri + 1);
                acc = (e >= rstart && e < e_end) ? fmaf(v0[q], a0[q], 0.f) : 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            v0[q] = v1[q];
            a0[q] = a1[q];
            c1[q] = c2[q];
            v1[q] = v2[q];
        }
    }
    const int r_last = rbase + ri;
    store(r_last, rstart, rend, acc);  // the row this warp's range ends in
    // tickets of the rows, in order
    for (int r = r_first; r <= r_last; ++r) {
        int fin = -1;
        if (lane == 0) {
            const int rs = __ldg(rowptr + r), re = __ldg(rowptr + r + 1);
            const int wa = rs / chunk, wb = (re - 1) / chunk;
            bool done = true;
            if (wb > wa) {
                done = (int)atom_add_acq_rel_gpu(reinterpret_cast<unsigned*>(cnt + r), 1u) == wb - wa;
                if (done) {
                    cnt[r] = 0;  // every warp of the row has taken its ticket
                    double tot = 0.0;
                    for (int k = 0; k <= wb - wa; ++k) tot += (double)__ldcg(part + (size_t)r * PS + k);
                    finish(r, tot);
                }
            }
            fin = done ? r : -1;
        }
        fin = __shfl_sync(FULL, fin, 0);
        if (fin >= 0) dt_row_ticket_warp(rt, fin, w);
    }
}

template <int G>
__global__ void __launch_bounds__(256) k_column(const int* __restrict__ col, const float* __restrict__ val,
                                                const int* __restrict__ seg_lo, const int* __restrict__ seg_hi,
                                                int V, int base, int nb, const float* __restrict__ mask,
                                                float* __restrict__ out, int stride) {
    extern __shared__ float smask[];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) smask[i] = mask[i];
    __syncthreads();
    column_body<G>(col, val, seg_lo, seg_hi, V, base, smask, out, stride, (int)(blockIdx.x * blockDim.x), (int)(gridDim.x * blockDim.x));
}

// The same for the aperture at pool index K-1 of the device table, into
// column K-1 of the slab.
template <int G>
__global__ void __launch_bounds__(256) k_column_dev(const int* __restrict__ col, const float* __restrict__ val,
                                                    const int* __restrict__ seg, int V,
                                                    const int* __restrict__ ap_beam, int K,
                                                    const int* __restrict__ beam_off, const int* __restrict__ rows,
                                                    const int* __restrict__ cols, const float* __restrict__ mask,
                                                    float* __restrict__ slab, int ld, const CGDev* __restrict__ cg) {
    extern __shared__ float smask[];
    if (cg->idle) return;
    const int b = ap_beam[K - 1];
    const int nb = rows[b] * cols[b];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) smask[i] = mask[i];
    __syncthreads();
    column_body<G>(col, val, seg + (size_t)b * V, seg + (size_t)(b + 1) * V, V, beam_off[b], smask,
                   slab + (size_t)(K - 1) * ld, 1, (int)(blockIdx.x * blockDim.x), (int)(gridDim.x * blockDim.x));
}

// a4 from D by beams, for beam b (b_dev: the beam read from the device's
// aperture table, the graph path's k_column_dev).
template <bool W16, bool BF>
__global__ void __launch_bounds__(256) k_column_beam(const int* __restrict__ brp_all,
                                                     const unsigned short* __restrict__ bcol,
                                                     const float* __restrict__ bval32,
                                                     const unsigned short* __restrict__ bval16, int V, int b, int nb,
                                                     int base, const int* __restrict__ ap_beam, int K,
                                                     const int* __restrict__ beam_off, const int* __restrict__ rows,
                                                     const int* __restrict__ cols, const float* __restrict__ mask,
                                                     const float* __restrict__ scale, float* __restrict__ out,
                                                     int stride, int ld, const CGDev* __restrict__ cg) {
    extern __shared__ float smask[];
    if (cg != nullptr) {  // the device-table form: aperture K - 1 into column K - 1 of the slab
        if (cg->idle) return;
        b = ap_beam[K - 1];
        nb = rows[b] * cols[b];
        base = beam_off[b];
        out += (size_t)(K - 1) * ld;
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) smask[i] = W16 ? mask[i] * scale[base + i] : mask[i];
    __syncthreads();
    column_beam_body<W16, BF>(brp_all + (size_t)b * (V + 1), beam_entry_base(brp_all, V, b), bcol, bval32, bval16, V,
                              smask, out, stride, (int)(blockIdx.x * blockDim.x), (int)(gridDim.x * blockDim.x));
}

// ---- Eq. 7 ------------------------------------------------------------------
__global__ void k_fluence(const int* __restrict__ ap_beam, const int* __restrict__ ap_lr, int lr_stride,
                          const double* __restrict__ y, int K, const int4* __restrict__ binfo, int N,
                          float* __restrict__ x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int4 bi = binfo[i];  // beam, MLC row within the beam, column, unused
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        if (ap_beam[k] != bi.x) continue;
        const int L = ap_lr[k * lr_stride + 2 * bi.y];
        const int R = ap_lr[k * lr_stride + 2 * bi.y + 1];
        if (bi.z >= L && bi.z < R) s += y[k];
    }
    x[i] = (float)s;
}

// ---- 16-bit storage (a6): values D_ij / s_i in FP16 or BF16, per-beamlet FP32
// scale s_i, FP32 accumulation ------------------------------------------------
// a1 with rows padded to 8 entries: uint4 loads of 8 uint16 columns and 8 values;
// x pre-multiplied by the beamlet scale in shared memory (or, when N floats do
// not fit in 48 KB, the product formed from global memory per entry).
template <int G, bool BF, bool SMEM_X>
__global__ void __launch_bounds__(256) k_dose16(const int* __restrict__ rowptr, const uint4* __restrict__ col8,
                                                const uint4* __restrict__ val8, int V, const float* __restrict__ x,
                                                const float* __restrict__ scale, int N,
                                                const uint8_t* __restrict__ vstruct,
                                                const StructTermsS* __restrict__ ts, int S, float* __restrict__ z,
                                                float* __restrict__ grad, double* __restrict__ F_part) {
    extern __shared__ float sx[];
    __shared__ StructTermsS s_ts[SMAX];
    __shared__ double s_red[8];
    if (SMEM_X)
        for (int i = threadIdx.x; i < N; i += blockDim.x) sx[i] = x[i] * scale[i];
    for (int i = threadIdx.x; i < S; i += blockDim.x) s_ts[i] = ts[i];
    __syncthreads();
    auto xs = [&](unsigned c) -> float { return SMEM_X ? sx[c] : __ldg(x + c) * __ldg(scale + c); };
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    constexpr int RPW = 32 / G;
    const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int n_warps = (gridDim.x * blockDim.x) >> 5;
    const int n_tiles = (V + RPW - 1) / RPW;
    float facc = 0.f;
    for (int t = warp_global; t < n_tiles; t += n_warps) {
        const int row = t * RPW + lane / G;
        float acc = 0.f;
        if (row < V) {
            const int p0 = rowptr[row] >> 3, p1 = rowptr[row + 1] >> 3;
            // two groups of the lane (p, p + G) requested together, summed in order
            for (int p = p0 + sub; p < p1; p += 2 * G) {
                const bool two = p + G < p1;
                const uint4 cw = __ldg(col8 + p);
                const uint4 vw = __ldg(val8 + p);
                uint4 cw2 = make_uint4(0u, 0u, 0u, 0u), vw2 = make_uint4(0u, 0u, 0u, 0u);
                if (two) {
                    cw2 = __ldg(col8 + p + G);
                    vw2 = __ldg(val8 + p + G);
                }
                const unsigned cs[8] = {cw.x, cw.y, cw.z, cw.w, cw2.x, cw2.y, cw2.z, cw2.w};
                const unsigned vs[8] = {vw.x, vw.y, vw.z, vw.w, vw2.x, vw2.y, vw2.z, vw2.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 v2 = unpack2<BF>(vs[q]);
                    acc = fmaf(v2.x, xs(cs[q] & 0xffffu), acc);
                    acc = fmaf(v2.y, xs(cs[q] >> 16), acc);
                }
                if (two)
#pragma unroll
                    for (int q = 4; q < 8; ++q) {
                        const float2 v2 = unpack2<BF>(vs[q]);
                        acc = fmaf(v2.x, xs(cs[q] & 0xffffu), acc);
                        acc = fmaf(v2.y, xs(cs[q] >> 16), acc);
                    }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (row < V && sub == 0) {
            z[row] = acc;
            if (grad != nullptr || F_part != nullptr) {
                // FP32 epilogue (FP64 issues at 1/64 of the FP32 rate here)
                const StructTermsS tt = S >= 0 ? s_ts[vstruct[row]] : ts[row];
                const float u = fmaxf((tt.tu_hi - acc) + tt.tu_lo, 0.f);  // T^- - z
                const float o = fmaxf((acc - tt.to_hi) - tt.to_lo, 0.f);  // z - T^+
                if (grad != nullptr) grad[row] = 2.f * (tt.b * o - tt.a * u);
                facc = fmaf(tt.a * u, u, fmaf(tt.b * o, o, facc));
            }
        }
    }
    if (F_part != nullptr) {
        const double sres = block_sum_mixed<256>(facc, s_red);
        if (threadIdx.x == 0) F_part[blockIdx.x] = sres;
    }
}

// ---- a1 in units of 32 voxel rows ------------------------------------------
// One warp per unit of 32 consecutive rows (grid-stride over the units, every
// block resident): the unit's entries are one contiguous range of groups (8
// entries of 16-bit storage, 4 of FP32), which the lanes request together,
// lane l the groups l, l + 32, ..., up to UB per lane at a time, so that the
// whole unit is in flight at once and every request is a full 512-byte
// warp access.  Each lane forms the dot product of its groups with x (staged
// in shared memory, pre-multiplied by the beamlet scale) and writes it to
// the warp's row of shared partials; then lane r sums row r's partials in
// group order and applies the epilogue, so z, grad F and the labels are
// accessed as 32 consecutive words.  The next unit's row offsets and labels
// are requested before this unit's entries.  Fixed summation order: a row's
// z is its groups' sequential FMA chains (from 0) summed in group order, the
// same whichever warp or block computes it.
constexpr int UNIT_ROWS = 32;
constexpr int UNIT_THREADS = 512;

template <bool L16, bool BF>
__device__ __forceinline__ float group_dot(const uint4 c, const uint4 v, const float* __restrict__ sx) {
    float p = 0.f;
    if constexpr (L16) {
        const unsigned cs[4] = {c.x, c.y, c.z, c.w};
        const unsigned vs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = unpack2<BF>(vs[q]);
            p = fmaf(f.x, sx[cs[q] & 0xffffu], p);
            p = fmaf(f.y, sx[cs[q] >> 16], p);
        }
    } else {
        p = fmaf(__uint_as_float(v.x), sx[c.x], p);
        p = fmaf(__uint_as_float(v.y), sx[c.y], p);
        p = fmaf(__uint_as_float(v.z), sx[c.z], p);
        p = fmaf(__uint_as_float(v.w), sx[c.w], p);
    }
    return p;
}

template <bool L16, bool BF>
__global__ void __launch_bounds__(UNIT_THREADS, 2) k_dose_units(
    const int* __restrict__ rowptr, const uint4* __restrict__ colg, const uint4* __restrict__ valg, int V,
    const float* __restrict__ x, const float* __restrict__ scale, int N, const uint8_t* __restrict__ vstruct,
    const StructTermsS* __restrict__ ts, int S, float* __restrict__ z, float* __restrict__ grad,
    double* __restrict__ F_part, int part_cap) {
    constexpr int EPG = L16 ? 8 : 4;  // entries per group (one 16-byte load of columns and of values)
    constexpr int UB = 4;             // groups per lane in flight
    constexpr int NW = UNIT_THREADS / 32;
    extern __shared__ __align__(16) float s_dyn_units[];
    __shared__ StructTermsS s_ts[SMAX];
    __shared__ double s_red[NW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* sx = s_dyn_units;
    float* spart = s_dyn_units + ((N + 3) & ~3) + wib * part_cap;
    const int n_units = (V + UNIT_ROWS - 1) / UNIT_ROWS;
    const int W = gridDim.x * NW;
    int u = blockIdx.x * NW + wib;
    // this unit's row offsets and labels first, so that they are in flight
    // while x is staged
    int rs = 0, re = 0, lab = 0;
    auto meta = [&](int uu, int& a, int& b, int& l) {
        const int row = uu * UNIT_ROWS + lane;
        a = b = 0;
        l = 0;
        if (uu < n_units && row < V) {
            a = __ldg(rowptr + row);
            b = __ldg(rowptr + row + 1);
            if (S >= 0) l = __ldg(vstruct + row);
        }
    };
    meta(u, rs, re, lab);
    for (int i = threadIdx.x; i < N; i += UNIT_THREADS) sx[i] = L16 ? __ldg(x + i) * __ldg(scale + i) : __ldg(x + i);
    for (int i = threadIdx.x; i < S; i += UNIT_THREADS) s_ts[i] = ts[i];
    __syncthreads();
    float facc = 0.f;
    for (; u < n_units; u += W) {
        const int row0 = u * UNIT_ROWS;
        const int nrow = min(UNIT_ROWS, V - row0);
        const int e0 = __shfl_sync(FULL, rs, 0);
        const int e1 = __shfl_sync(FULL, re, nrow - 1);
        int rs_n, re_n, lab_n;
        meta(u + W, rs_n, re_n, lab_n);
        const int g0 = e0 / EPG, ng = (e1 - e0) / EPG;
        float acc = 0.f;
        if (ng <= part_cap) {
            for (int k0 = 0; k0 < ng; k0 += 32 * UB) {
                uint4 c[UB], v[UB];
#pragma unroll
                for (int q = 0; q < UB; ++q) {
                    const int g = k0 + q * 32 + lane;
                    if (g < ng) {
                        c[q] = __ldg(colg + g0 + g);
                        v[q] = __ldg(valg + g0 + g);
                    }
                }
#pragma unroll
                for (int q = 0; q < UB; ++q) {
                    const int g = k0 + q * 32 + lane;
                    if (g < ng) spart[g] = group_dot<L16, BF>(c[q], v[q], sx);
                }
            }
            __syncwarp();
            if (lane < nrow)
                for (int g = (rs - e0) / EPG, gh = (re - e0) / EPG; g < gh; ++g) acc += spart[g];
            __syncwarp();  // the partials are rewritten by the next unit
        } else if (lane < nrow) {
            // a unit larger than the partial row (not produced by a plan's
            // layout, whose largest unit sizes part_cap): the same sums, the
            // groups read by the row's own lane
            for (int g = rs / EPG, gh = re / EPG; g < gh; ++g) acc += group_dot<L16, BF>(__ldg(colg + g), __ldg(valg + g), sx);
        }
        if (lane < nrow) {
            const int row = row0 + lane;
            z[row] = acc;
            if (grad != nullptr || F_part != nullptr) {
                const StructTermsS tt = S >= 0 ? s_ts[lab] : ts[row];
                const float uu = fmaxf((tt.tu_hi - acc) + tt.tu_lo, 0.f);  // T^- - z
                const float o = fmaxf((acc - tt.to_hi) - tt.to_lo, 0.f);   // z - T^+
                if (grad != nullptr) grad[row] = 2.f * (tt.b * o - tt.a * uu);
                facc = fmaf(tt.a * uu, uu, fmaf(tt.b * o, o, facc));
            }
        }
        rs = rs_n;
        re = re_n;
        lab = lab_n;
    }
    if (F_part != nullptr) {
        const double sres = block_sum_mixed<UNIT_THREADS>(facc, s_red);
        if (threadIdx.x == 0) F_part[blockIdx.x] = sres;
    }
}

// ---- a1 split evenly over warps along the merge path ------------------------
// The work of a1 is the merge of two sequences, D's groups of stored entries
// (8 per group with 16-bit storage, 4 with FP32) and the row ends (a row is
// done once its groups are): warp v takes the stretch of that merge between
// the splits path[v] = (rows done, groups consumed) and path[v + 1], the
// same number of items for every warp (Merrill & Garland's merge-path
// split), so empty rows (one item each) spread over the warps like entries.
// The warp requests its first UB groups per lane as soon as it has its
// split, puts each group's dot product with x (staged in shared memory) in its
// row of shared partials, and finishes the rows that end in its stretch: lane
// l sums row l's partials in group order and applies the epilogue, 32 rows at
// a time.  Every stretch is longer than the longest row, so a row has groups
// in at most two stretches: the earlier warp stores the sum of the row's
// groups it holds (slot 0 of the boundary), the warp that finishes the row
// the sum of the rest (slot 1), and the second of the two to take the
// boundary's ticket forms z = slot 0 + slot 1, applies the epilogue and writes
// the row's objective term to F_part[F_stride + boundary] (0 where no row
// crosses the boundary), so that F is a fixed-order sum whichever warp
// finishes first.
constexpr int MERGE_THREADS = 256;

template <bool L16, bool BF>
__global__ void __launch_bounds__(MERGE_THREADS, 4) k_dose_merge(
    const int* __restrict__ rowptr, const uint4* __restrict__ colg, const uint4* __restrict__ valg, int V,
    const float* __restrict__ x, const float* __restrict__ scale, int N, const uint8_t* __restrict__ vstruct,
    const StructTermsS* __restrict__ ts, int S, float* __restrict__ z, float* __restrict__ grad,
    double* __restrict__ F_part, int F_stride, int cap, int n_warps, const int2* __restrict__ path,
    float* __restrict__ slot, int* __restrict__ cnt) {
    constexpr int EPG = L16 ? 8 : 4;
    constexpr int UB = 4;
    constexpr int NW = MERGE_THREADS / 32;
    extern __shared__ __align__(16) float s_dyn_merge[];
    __shared__ StructTermsS s_ts[SMAX];
    __shared__ double s_red[NW];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wg = blockIdx.x * NW + wib;
    const bool active = wg < n_warps;  // uniform per warp; idle warps still meet the block barrier
    float* sx = s_dyn_merge;
    float* spart = s_dyn_merge + ((N + 3) & ~3) + wib * cap;
    int2 p0 = make_int2(0, 0), p1 = make_int2(0, 0);
    if (active) {
        p0 = __ldg(path + wg);
        p1 = __ldg(path + wg + 1);
    }
    const int r0 = p0.x, r1 = p1.x, g_begin = p0.y, ng = p1.y - p0.y;
    uint4 c[UB], v[UB];
    auto load_batch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < UB; ++q) {
            const int g = k0 + q * 32 + lane;
            if (g < ng) {
                c[q] = __ldg(colg + g_begin + g);
                v[q] = __ldg(valg + g_begin + g);
            }
        }
    };
    load_batch(0);
    // the rows this warp finishes (r0 .. r1 - 1), 32 at a time, and the row it
    // leaves unfinished (r1, when it holds some of its groups)
    int rs = 0, re = 0, lab = 0;
    auto row_meta = [&](int r) {
        rs = re = 0;
        lab = 0;
        if (r < r1) {
            rs = __ldg(rowptr + r);
            re = __ldg(rowptr + r + 1);
            if (S >= 0) lab = __ldg(vstruct + r);
        }
    };
    row_meta(r0 + lane);
    const int rs_out = active && r1 < V ? __ldg(rowptr + r1) : 0;
    for (int i = threadIdx.x; i < N; i += MERGE_THREADS) sx[i] = L16 ? __ldg(x + i) * __ldg(scale + i) : __ldg(x + i);
    for (int i = threadIdx.x; i < S; i += MERGE_THREADS) s_ts[i] = ts[i];
    __syncthreads();
    for (int k0 = 0; k0 < ng; k0 += 32 * UB) {
        if (k0 > 0) load_batch(k0);
#pragma unroll
        for (int q = 0; q < UB; ++q) {
            const int g = k0 + q * 32 + lane;
            if (g < ng) spart[g] = group_dot<L16, BF>(c[q], v[q], sx);
        }
    }
    __syncwarp();
    // epilogue of row r at z = acc; returns its objective term
    auto epilogue = [&](int r, float acc, int l) -> float {
        z[r] = acc;
        float f = 0.f;
        if (grad != nullptr || F_part != nullptr) {
            const StructTermsS tt = S >= 0 ? s_ts[l] : ts[r];
            const float uu = fmaxf((tt.tu_hi - acc) + tt.tu_lo, 0.f);  // T^- - z
            const float o = fmaxf((acc - tt.to_hi) - tt.to_lo, 0.f);   // z - T^+
            if (grad != nullptr) grad[r] = 2.f * (tt.b * o - tt.a * uu);
            f = fmaf(tt.a * uu, uu, tt.b * o * o);
        }
        return f;
    };
    // a row across boundary b: this lane's part into slot s; the second to arrive finishes the row
    auto cross = [&](int b, int s, float part_sum, int r, int l) {
        slot[2 * b + s] = part_sum;
        if ((int)atom_add_acq_rel_gpu(reinterpret_cast<unsigned*>(cnt + b), 1u) == 1) {
            cnt[b] = 0;
            const float a0 = s == 0 ? part_sum : __ldcg(slot + 2 * b);
            const float a1 = s == 1 ? part_sum : __ldcg(slot + 2 * b + 1);
            const float f = epilogue(r, a0 + a1, l);
            if (F_part != nullptr) F_part[F_stride + b] = (double)f;
        }
    };
    float facc = 0.f;
    bool crossed_in = false;  // (lane 0) the first row began in the previous stretch
    for (int rb = r0; rb < r1; rb += 32) {
        const int r = rb + lane;
        const int crs = rs, cre = re, cl = lab;
        if (rb + 32 < r1) row_meta(rb + 32 + lane);  // the next 32 rows
        if (r < r1) {
            const int gs = max(crs / EPG - g_begin, 0), ge = cre / EPG - g_begin;
            float acc = 0.f;
            for (int g = gs; g < ge; ++g) acc += spart[g];
            if (crs / EPG < g_begin) {  // only the first row: its other groups are the previous warp's
                crossed_in = true;
                cross(wg, 1, acc, r, cl);
            } else {
                facc += epilogue(r, acc, cl);
            }
        }
    }
    if (active && lane == 0) {
        if (!crossed_in && F_part != nullptr) F_part[F_stride + wg] = 0.0;  // no row crosses into this stretch
        if (r1 < V && rs_out / EPG < g_begin + ng) {
            // row r1 continues in the next stretch: the sum of its groups here
            float a = 0.f;
            for (int g = rs_out / EPG - g_begin; g < ng; ++g) a += spart[g];
            cross(wg + 1, 0, a, r1, S >= 0 ? __ldg(vstruct + r1) : 0);
        }
    }
    if (F_part != nullptr) {
        const double sres = block_sum_mixed<MERGE_THREADS>(facc, s_red);
        if (threadIdx.x == 0) F_part[blockIdx.x] = sres;
    }
}

// a2 with rows padded to 8 entries: two int4 loads of voxel indices and one uint4
// of values per 8 entries (LC: consecutive entries on consecutive threads);
// the row's scale is applied once at the end.
template <int BT, bool BF, bool LC>
__global__ void __launch_bounds__(BT) k_dt16(const int* __restrict__ rowptr, const int4* __restrict__ col4,
                                             const uint4* __restrict__ val8, const float* __restrict__ scale, int N,
                                             const int* __restrict__ order,
                                             const float* __restrict__ pi, float* __restrict__ w,
                                             const int* __restrict__ skip, RowTicket rt) {
    __shared__ double s_red[BT / 32];
    dt_round_snapshot(rt);
    if (skip != nullptr && *skip) return;
    const int row = order[blockIdx.x];  // longest rows first
    const float s = LC ? dt16_row_sum_lc<BT, BF>(rowptr, reinterpret_cast<const int*>(col4),
                                                 reinterpret_cast<const unsigned short*>(val8), scale, row, pi, s_red)
                       : dt16_row_sum<BT, BF>(rowptr, col4, val8, scale, row, pi, s_red);
    if (threadIdx.x == 0) w[row] = s;
    dt_row_ticket(rt, row, w);
}

template <int G, bool BF>
__global__ void __launch_bounds__(256) k_column16(const unsigned short* __restrict__ col,
                                                  const unsigned short* __restrict__ val,
                                                  const int* __restrict__ seg_lo, const int* __restrict__ seg_hi,
                                                  int V, int base, int nb, const float* __restrict__ mask,
                                                  const float* __restrict__ scale, float* __restrict__ out,
                                                  int stride) {
    extern __shared__ float smask[];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) smask[i] = mask[i] * scale[base + i];
    __syncthreads();
    column16_body<G, BF>(col, val, seg_lo, seg_hi, V, base, smask, out, stride, (int)(blockIdx.x * blockDim.x), (int)(gridDim.x * blockDim.x));
}

template <int G, bool BF>
__global__ void __launch_bounds__(256) k_column16_dev(const unsigned short* __restrict__ col,
                                                      const unsigned short* __restrict__ val,
                                                      const int* __restrict__ seg, int V,
                                                      const int* __restrict__ ap_beam, int K,
                                                      const int* __restrict__ beam_off,
                                                      const int* __restrict__ rows, const int* __restrict__ cols,
                                                      const float* __restrict__ mask, const float* __restrict__ scale,
                                                      float* __restrict__ slab, int ld,
                                                      const CGDev* __restrict__ cg) {
    extern __shared__ float smask[];
    if (cg->idle) return;
    const int b = ap_beam[K - 1];
    const int nb = rows[b] * cols[b];
    const int base = beam_off[b];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) smask[i] = mask[i] * scale[base + i];
    __syncthreads();
    column16_body<G, BF>(col, val, seg + (size_t)b * V, seg + (size_t)(b + 1) * V, V, base, smask,
                         slab + (size_t)(K - 1) * ld, 1, (int)(blockIdx.x * blockDim.x),
                         (int)(gridDim.x * blockDim.x));
}

// The device-driven round's beam decision fused with the new aperture's
// column (a4): every block takes the same decision from the row results of
// the D^T kernel (pricing::decide); block 0 commits aperture rs_K, writes
// cg->K, idle, stop, done and the while-node handle; every block then builds
// the open-beamlet mask from the rows' leaf positions and computes its rows of
// the column, with the arithmetic of column_body / column16_body.  Blocks read
// the round state only from rs_K and rs_stop, which no block of this launch
// writes.
template <int G, int PREC>
__global__ void __launch_bounds__(256) k_commit_column(const int* __restrict__ col, const float* __restrict__ val,
                                                       const unsigned short* __restrict__ col16,
                                                       const unsigned short* __restrict__ val16,
                                                       const float* __restrict__ scale, int V, CommitArgs ca,
                                                       const int* __restrict__ brp_all,
                                                       const unsigned short* __restrict__ bcol,
                                                       const float* __restrict__ bval32,
                                                       const unsigned short* __restrict__ bval16) {
    extern __shared__ double s_dyn[];
    double* s_sum = s_dyn;                                        // n_beams
    float* smask = reinterpret_cast<float*>(s_dyn + ca.n_beams);  // max_nb
    CGDev* cg = ca.cg;
    const int tid = threadIdx.x;
    const bool lead = blockIdx.x == 0 && tid == 0;
    auto finish = [&](int idle, int stop) {
        if (lead) {
            cg->idle = idle;
            cg->stop = stop;
            if (ca.use_cond) cudaGraphSetConditional(ca.cond, stop ? 0u : 1u);
        }
    };
    if (__ldcg(&cg->rs_stop)) {
        finish(1, 1);
        return;
    }
    const int K = __ldcg(&cg->rs_K) + 1;  // pool size with the new aperture
    int b = 0;
    double rc = 0.0;
    const int outcome = pricing::decide(ca.row_v, ca.beam_row0, ca.n_beams, ca.row_lr, ca.rows, ca.tau, K,
                                        ca.lr_stride, ca.ap_beam, ca.ap_lr, s_sum, &b, &rc);
    if (outcome != pricing::OUTCOME_NEW) {
        if (lead) cg->done = outcome;
        finish(1, 1);
        return;
    }
    const int R = ca.rows[b], C = ca.cols[b], r0 = ca.beam_row0[b], base = ca.beam_off[b];
    if (blockIdx.x == 0) {
        if (tid == 0) ca.ap_beam[K - 1] = b;
        for (int r = tid; r < R; r += blockDim.x) {
            const int2 lr = ca.row_lr[r0 + r];
            ca.ap_lr[(K - 1) * ca.lr_stride + 2 * r] = lr.x;
            ca.ap_lr[(K - 1) * ca.lr_stride + 2 * r + 1] = lr.y;
        }
        if (tid == 0) cg->K = K;
        finish(0, K >= __ldcg(&cg->K_end) ? 1 : 0);
    }
    for (int i = tid; i < R * C; i += blockDim.x) {
        const int2 lr = ca.row_lr[r0 + i / C];
        const int c = i % C;
        const float m = (c >= lr.x && c < lr.y) ? 1.f : 0.f;
        if constexpr (PREC == DAO_PREC_FP32)
            smask[i] = m;
        else
            smask[i] = m * scale[base + i];
    }
    __syncthreads();
    float* out = ca.slab + (size_t)(K - 1) * ca.ld;
    const int* seg_lo = ca.seg + (size_t)b * V;
    const int* seg_hi = ca.seg + (size_t)(b + 1) * V;
    if constexpr (G == 0)  // D by beams
        column_beam_body<PREC != DAO_PREC_FP32, PREC == DAO_PREC_BF16>(
            brp_all + (size_t)b * (V + 1), beam_entry_base(brp_all, V, b), bcol, bval32, bval16, V, smask, out, 1,
            (int)(blockIdx.x * blockDim.x), (int)(gridDim.x * blockDim.x));
    else if constexpr (PREC == DAO_PREC_FP32)
        column_body<G>(col, val, seg_lo, seg_hi, V, base, smask, out, 1, (int)(blockIdx.x * blockDim.x), (int)(gridDim.x * blockDim.x));
    else
        column16_body<G, PREC == DAO_PREC_BF16>(col16, val16, seg_lo, seg_hi, V, base, smask, out, 1, (int)(blockIdx.x * blockDim.x), (int)(gridDim.x * blockDim.x));
}

// Blocks of a grid-stride kernel that are all resident at once (every block
// runs the same number of row tiles, so a second wave would double the time),
// capped at `cap`.
template <class Kern>
int resident_grid(Kern kern, size_t smem, int num_sms, int cap) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, smem) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    return std::min(cap, occ * num_sms);
}

template <int G, bool BF>
cudaError_t dose16_g(const DevCSR& D, const float* x, const uint8_t* vstruct, const StructTermsS* ts, int S,
                     float* z, float* grad, double* F_part, int& grid, int num_sms, cudaStream_t stream) {
    const size_t smem = (size_t)D.n_cols * sizeof(float);
    if (smem <= 48 * 1024)
        grid = resident_grid(k_dose16<G, BF, true>, smem, num_sms, grid);
    else
        grid = resident_grid(k_dose16<G, BF, false>, 0, num_sms, grid);
    if (smem <= 48 * 1024)
        k_dose16<G, BF, true><<<grid, 256, smem, stream>>>(
            D.rowptr, reinterpret_cast<const uint4*>(D.col16), reinterpret_cast<const uint4*>(D.val16), D.n_rows, x,
            D.scale, D.n_cols, vstruct, ts, S, z, grad, F_part);
    else
        k_dose16<G, BF, false><<<grid, 256, 0, stream>>>(
            D.rowptr, reinterpret_cast<const uint4*>(D.col16), reinterpret_cast<const uint4*>(D.val16), D.n_rows, x,
            D.scale, D.n_cols, vstruct, ts, S, z, grad, F_part);
    return cudaGetLastError();
}

// Dynamic shared memory of the unit form: x (N floats) and one row of
// part_cap partials per warp.
constexpr int UNITS_SMEM_MAX = 200 * 1024;
size_t units_smem(int N, int part_cap) {
    return (size_t)((N + 3) & ~3) * sizeof(float) + (size_t)(UNIT_THREADS / 32) * part_cap * sizeof(float);
}

template <bool L16, bool BF>
cudaError_t dose_units(const DevCSR& D, const float* x, const uint8_t* vstruct, const StructTermsS* ts, int S,
                       float* z, float* grad, double* F_part, int& grid, int num_sms, cudaStream_t stream) {
    const size_t smem = units_smem(D.n_cols, D.unit_groups_max);
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dose_units<L16, BF>, UNIT_THREADS, smem) !=
            cudaSuccess ||
        occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    grid = std::min(grid, occ * num_sms);
    const void* colp = L16 ? static_cast<const void*>(D.col16) : static_cast<const void*>(D.col);
    const void* valp = L16 ? static_cast<const void*>(D.val16) : static_cast<const void*>(D.val);
    k_dose_units<L16, BF><<<grid, UNIT_THREADS, smem, stream>>>(
        D.rowptr, static_cast<const uint4*>(colp), static_cast<const uint4*>(valp), D.n_rows, x, D.scale, D.n_cols,
        vstruct, ts, S, z, grad, F_part, D.unit_groups_max);
    return cudaGetLastError();
}

template <int G>
cudaError_t dose_g(const DevCSR& D, const float* x, const uint8_t* vstruct, const StructTermsS* ts, int S,
                   float* z, float* grad, double* F_part, int& grid, int num_sms, cudaStream_t stream) {
    const size_t smem = (size_t)D.n_cols * sizeof(float);
    if (smem <= 48 * 1024)
        grid = resident_grid(k_dose<G, true>, smem, num_sms, grid);
    else
        grid = resident_grid(k_dose<G, false>, 0, num_sms, grid);
    if (smem <= 48 * 1024) {
        k_dose<G, true><<<grid, 256, smem, stream>>>(D.rowptr, reinterpret_cast<const int4*>(D.col),
                                                     reinterpret_cast<const float4*>(D.val), D.n_rows, x,
                                                     D.n_cols, vstruct, ts, S, z, grad, F_part);
    } else {
        k_dose<G, false><<<grid, 256, 0, stream>>>(D.rowptr, reinterpret_cast<const int4*>(D.col),
                                                   reinterpret_cast<const float4*>(D.val), D.n_rows, x,
                                                   D.n_cols, vstruct, ts, S, z, grad, F_part);
    }
    return cudaGetLastError();
}

}  // namespace

int dose_grid(int n_rows, int num_sms) {
    (void)n_rows;
    return num_sms * 8;
}

namespace {

// lanes per voxel row of the dose SpMV: the autotuner's choice, else by the mean
// stored row length (16-bit rows hold 8 entries per load, FP32 rows 4)
int dose_lanes(const DevCSR& D) {
    const double mean = D.n_rows > 0 ? (double)D.nnz_stored / (double)D.n_rows : 0.0;
    int g = D.tune_dose_g;
    if (g == 0) {
        if (D.prec != DAO_PREC_FP32)
            g = mean <= 48.0 ? 4 : mean <= 128.0 ? 8 : 16;
        else
            g = mean <= 24.0 ? 4 : mean <= 64.0 ? 8 : mean <= 160.0 ? 16 : 32;
    }
    if (D.prec != DAO_PREC_FP32 && g > 16) g = 16;
    return g;
}

template <bool BF>
cudaError_t dose16_any(int g, const DevCSR& D, const float* x, const uint8_t* vstruct, const StructTermsS* ts,
                       int S, float* z, float* grad, double* F_part, int& grid, int num_sms, cudaStream_t stream) {
    switch (g) {
        case 4: return dose16_g<4, BF>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
        case 8: return dose16_g<8, BF>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
        default: return dose16_g<16, BF>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    }
}

template <int BT, bool LC>
void dt_launch(const DevCSR& Dt, const float* pi, float* w, const int* skip, const RowTicket& rt,
               cudaStream_t stream) {
    if (Dt.prec == DAO_PREC_FP16)
        k_dt16<BT, false, LC><<<Dt.n_rows, BT, 0, stream>>>(Dt.rowptr, reinterpret_cast<const int4*>(Dt.col),
                                                            reinterpret_cast<const uint4*>(Dt.val16), Dt.scale,
                                                            Dt.n_rows, Dt.order, pi, w, skip, rt);
    else if (Dt.prec == DAO_PREC_BF16)
        k_dt16<BT, true, LC><<<Dt.n_rows, BT, 0, stream>>>(Dt.rowptr, reinterpret_cast<const int4*>(Dt.col),
                                                           reinterpret_cast<const uint4*>(Dt.val16), Dt.scale,
                                                           Dt.n_rows, Dt.order, pi, w, skip, rt);
    else
        k_dt<BT, LC><<<Dt.n_rows, BT, 0, stream>>>(Dt.rowptr, reinterpret_cast<const int4*>(Dt.col),
                                                    reinterpret_cast<const float4*>(Dt.val), Dt.n_rows, Dt.order, pi,
                                                    w, skip, rt);
}

template <int BT>
void dt_launch_map(const DevCSR& Dt, const float* pi, float* w, const int* skip, const RowTicket& rt,
                   cudaStream_t stream) {
    if (Dt.tune_dt_map == DT_MAP_GROUPED)
        dt_launch<BT, false>(Dt, pi, w, skip, rt, stream);
    else
        dt_launch<BT, true>(Dt, pi, w, skip, rt, stream);
}

template <int G>
void column_launch(const DevCSR& D, const int* seg_lo, const int* seg_hi, int base, int nb, const float* mask,
                   float* out, int stride, int grid, cudaStream_t stream) {
    const size_t sm = (size_t)nb * sizeof(float);
    if (D.prec == DAO_PREC_FP16)
        k_column16<G, false><<<grid, 256, sm, stream>>>(D.col16, D.val16, seg_lo, seg_hi, D.n_rows, base, nb, mask,
                                                         D.scale, out, stride);
    else if (D.prec == DAO_PREC_BF16)
        k_column16<G, true><<<grid, 256, sm, stream>>>(D.col16, D.val16, seg_lo, seg_hi, D.n_rows, base, nb, mask,
                                                        D.scale, out, stride);
    else
        k_column<G><<<grid, 256, sm, stream>>>(D.col, D.val, seg_lo, seg_hi, D.n_rows, base, nb, mask, out, stride);
}

template <int G>
void column_dev_launch(const DevCSR& D, const int* seg, const int* ap_beam, int K, const int* beam_off,
                       const int* rows, const int* cols, int max_nb, const float* mask, float* slab, int ld,
                       const CGDev* cg, int grid, cudaStream_t stream) {
    const size_t sm = (size_t)max_nb * sizeof(float);
    if (D.prec == DAO_PREC_FP16)
        k_column16_dev<G, false><<<grid, 256, sm, stream>>>(D.col16, D.val16, seg, D.n_rows, ap_beam, K, beam_off,
                                                             rows, cols, mask, D.scale, slab, ld, cg);
    else if (D.prec == DAO_PREC_BF16)
        k_column16_dev<G, true><<<grid, 256, sm, stream>>>(D.col16, D.val16, seg, D.n_rows, ap_beam, K, beam_off,
                                                            rows, cols, mask, D.scale, slab, ld, cg);
    else
        k_column_dev<G><<<grid, 256, sm, stream>>>(D.col, D.val, seg, D.n_rows, ap_beam, K, beam_off, rows, cols,
                                                    mask, slab, ld, cg);
}

}  // namespace

size_t merge_smem(int N, int cap) {
    return (size_t)((N + 3) & ~3) * sizeof(float) + (size_t)(MERGE_THREADS / 32) * cap * sizeof(float);
}

template <bool L16, bool BF>
cudaError_t dose_merge(const DevCSR& D, const float* x, const uint8_t* vstruct, const StructTermsS* ts, int S,
                       float* z, float* grad, double* F_part, int& grid, int& F_used, cudaStream_t stream) {
    const size_t smem = merge_smem(D.n_cols, D.merge_chunk);
    grid = (D.merge_warps + MERGE_THREADS / 32 - 1) / (MERGE_THREADS / 32);
    F_used = grid + D.merge_warps;
    const void* colp = L16 ? static_cast<const void*>(D.col16) : static_cast<const void*>(D.col);
    const void* valp = L16 ? static_cast<const void*>(D.val16) : static_cast<const void*>(D.val);
    k_dose_merge<L16, BF><<<grid, MERGE_THREADS, smem, stream>>>(
        D.rowptr, static_cast<const uint4*>(colp), static_cast<const uint4*>(valp), D.n_rows, x, D.scale, D.n_cols,
        vstruct, ts, S, z, grad, F_part, grid, D.merge_chunk, D.merge_warps, D.merge_path, D.merge_slot,
        D.merge_cnt);
    return cudaGetLastError();
}

bool dose_merge_available(const DevCSR& D) {
    return D.merge_chunk > 0 && merge_smem(D.n_cols, D.merge_chunk) <= (size_t)UNITS_SMEM_MAX;
}

int dose_merge_f_slots(const DevCSR& D) {
    return D.merge_chunk > 0 ? (D.merge_warps + MERGE_THREADS / 32 - 1) / (MERGE_THREADS / 32) + D.merge_warps : 0;
}

bool dose_units_available(const DevCSR& D) {
    return D.unit_groups_max > 0 && units_smem(D.n_cols, D.unit_groups_max) <= (size_t)UNITS_SMEM_MAX;
}

int dose_form_effective(const DevCSR& D) {
    const int f = D.tune_dose_form;
    if (f == DOSE_FORM_MERGE && dose_merge_available(D)) return DOSE_FORM_MERGE;
    if (f != DOSE_FORM_LANES && dose_units_available(D)) return DOSE_FORM_UNITS;
    return DOSE_FORM_LANES;
}

cudaError_t spmv_configure() {
    cudaError_t e = cudaSuccess;
    for (const void* k : {(const void*)k_dose_units<false, false>, (const void*)k_dose_units<true, false>,
                          (const void*)k_dose_units<true, true>, (const void*)k_dose_merge<false, false>,
                          (const void*)k_dose_merge<true, false>, (const void*)k_dose_merge<true, true>})
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, UNITS_SMEM_MAX);
    return e;
}

cudaError_t launch_dose(const DevCSR& D, const float* x, const uint8_t* vstruct, const StructTermsF* tf,
                        const StructTermsS* ts, int S, float* z, float* grad, double* F_part, int F_blocks,
                        double* F_out, int num_sms, cudaStream_t stream, int* launches) {
    (void)tf;
    int grid = dose_grid(D.n_rows, num_sms);  // at most this many; resident_grid trims it
    const int form = dose_form_effective(D);
    if (F_part != nullptr && form != DOSE_FORM_MERGE && F_blocks < grid) return cudaErrorInvalidValue;
    const int g = dose_lanes(D);
    const bool units = form == DOSE_FORM_UNITS;
    cudaError_t e;
    if (form == DOSE_FORM_MERGE) {
        int F_used = dose_merge_f_slots(D);
        if (F_part != nullptr && F_blocks < F_used) return cudaErrorInvalidValue;  // sized at creation
        if (D.prec == DAO_PREC_FP32)
            e = dose_merge<false, false>(D, x, vstruct, ts, S, z, grad, F_part, grid, F_used, stream);
        else if (D.prec == DAO_PREC_FP16)
            e = dose_merge<true, false>(D, x, vstruct, ts, S, z, grad, F_part, grid, F_used, stream);
        else
            e = dose_merge<true, true>(D, x, vstruct, ts, S, z, grad, F_part, grid, F_used, stream);
        ++*launches;
        if (e != cudaSuccess || F_part == nullptr || F_out == nullptr) return e;
        k_sum_f64<<<1, 256, 0, stream>>>(F_part, F_used, F_out);
        ++*launches;
        return cudaGetLastError();
    }
    if (units && D.prec == DAO_PREC_FP32)
        e = dose_units<false, false>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else if (units && D.prec == DAO_PREC_FP16)
        e = dose_units<true, false>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else if (units)
        e = dose_units<true, true>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else if (D.prec == DAO_PREC_BF16)
        e = dose16_any<true>(g, D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else if (D.prec == DAO_PREC_FP16)
        e = dose16_any<false>(g, D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else if (g == 4)
        e = dose_g<4>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else if (g == 8)
        e = dose_g<8>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else if (g == 16)
        e = dose_g<16>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    else
        e = dose_g<32>(D, x, vstruct, ts, S, z, grad, F_part, grid, num_sms, stream);
    ++*launches;
    if (e != cudaSuccess || F_part == nullptr || F_out == nullptr) return e;
    k_sum_f64<<<1, 256, 0, stream>>>(F_part, grid, F_out);
    ++*launches;
    return cudaGetLastError();
}

static cudaError_t dt_dispatch(const DevCSR& Dt, const float* pi, float* w, const int* skip, const RowTicket& rt,
                        cudaStream_t stream, int* launches) {
    if (Dt.n_rows == 0) return cudaSuccess;
    if (Dt.tune_dt_map == DT_MAP_SPLIT && Dt.split_chunk > 0) {
        const int grid = (Dt.split_warps + SPLIT_THREADS / 32 - 1) / (SPLIT_THREADS / 32);
        const int E = (int)Dt.nnz_stored;
        if (Dt.prec == DAO_PREC_FP16)
            k_dt_split<1><<<grid, SPLIT_THREADS, 0, stream>>>(Dt.rowptr, Dt.col, Dt.val16, Dt.scale, Dt.n_rows, E,
                                                              Dt.split_chunk, Dt.split_warps, Dt.split_row,
                                                              Dt.split_part, Dt.split_ps, Dt.split_cnt, pi, w, skip,
                                                              rt);
        else if (Dt.prec == DAO_PREC_BF16)
            k_dt_split<2><<<grid, SPLIT_THREADS, 0, stream>>>(Dt.rowptr, Dt.col, Dt.val16, Dt.scale, Dt.n_rows, E,
                                                              Dt.split_chunk, Dt.split_warps, Dt.split_row,
                                                              Dt.split_part, Dt.split_ps, Dt.split_cnt, pi, w, skip,
                                                              rt);
        else
            k_dt_split<0><<<grid, SPLIT_THREADS, 0, stream>>>(Dt.rowptr, Dt.col, Dt.val, Dt.scale, Dt.n_rows, E,
                                                              Dt.split_chunk, Dt.split_warps, Dt.split_row,
                                                              Dt.split_part, Dt.split_ps, Dt.split_cnt, pi, w, skip,
                                                              rt);
        ++*launches;
        return cudaGetLastError();
    }
    // one block per beamlet row; 64 threads by default, so that up to 32 blocks
    // per SM keep every row resident in one wave
    switch (Dt.tune_dt_threads) {
        case 128: dt_launch_map<128>(Dt, pi, w, skip, rt, stream); break;
        case 256: dt_launch_map<256>(Dt, pi, w, skip, rt, stream); break;
        default: dt_launch_map<64>(Dt, pi, w, skip, rt, stream); break;
    }
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_dt(const DevCSR& Dt, const float* pi, float* w, const int* skip, cudaStream_t stream,
                      int* launches) {
    return dt_dispatch(Dt, pi, w, skip, RowTicket{}, stream, launches);
}

cudaError_t launch_dt_rows(const DevCSR& Dt, const float* pi, float* w, const RowTicket& rt, cudaStream_t stream,
                           int* launches) {
    if (rt.cg == nullptr) return cudaErrorInvalidValue;  // row_cnt null: the snapshot without the row search
    return dt_dispatch(Dt, pi, w, &rt.cg->stop, rt, stream, launches);
}

// The aperture column runs on D by beams when the launch shape is 0 (the
// default) and the layout was built.
static bool column_by_beams(const DevCSR& D) { return D.tune_col_g == 0 && D.beam_rowptr != nullptr; }

// b, nb, base: the beam, its beamlets and its first beamlet (cg == nullptr);
// else the beam of aperture K - 1 of the device table, into column K - 1 of
// the slab (stride ld).
static void column_beam_launch(const DevCSR& D, int b, int nb, int base, const int* ap_beam, int K,
                               const int* beam_off, const int* rows, const int* cols, int max_nb, const float* mask,
                               float* out, int stride, int ld, const CGDev* cg, int grid, cudaStream_t stream) {
    const size_t sm = (size_t)std::max(max_nb, 1) * sizeof(float);
    if (D.prec == DAO_PREC_FP16)
        k_column_beam<true, false><<<grid, 256, sm, stream>>>(D.beam_rowptr, D.beam_col, nullptr, D.beam_val16,
                                                               D.n_rows, b, nb, base, ap_beam, K, beam_off, rows,
                                                               cols, mask, D.scale, out, stride, ld, cg);
    else if (D.prec == DAO_PREC_BF16)
        k_column_beam<true, true><<<grid, 256, sm, stream>>>(D.beam_rowptr, D.beam_col, nullptr, D.beam_val16,
                                                              D.n_rows, b, nb, base, ap_beam, K, beam_off, rows,
                                                              cols, mask, D.scale, out, stride, ld, cg);
    else
        k_column_beam<false, false><<<grid, 256, sm, stream>>>(D.beam_rowptr, D.beam_col, D.beam_val32, nullptr,
                                                                D.n_rows, b, nb, base, ap_beam, K, beam_off, rows,
                                                                cols, mask, D.scale, out, stride, ld, cg);
}

cudaError_t launch_column(const DevCSR& D, const int* seg, int b, int base, int nb, const float* mask, float* out,
                          int stride, int num_sms, cudaStream_t stream, int* launches) {
    if (D.n_rows == 0) return cudaSuccess;
    const int grid = num_sms * 8;
    const int V = D.n_rows;
    const int* seg_lo = seg + (size_t)b * V;
    const int* seg_hi = seg + (size_t)(b + 1) * V;
    if (column_by_beams(D)) {
        column_beam_launch(D, b, nb, base, nullptr, 0, nullptr, nullptr, nullptr, nb, mask, out, stride, 0, nullptr,
                           grid, stream);
        ++*launches;
        return cudaGetLastError();
    }
    switch (D.tune_col_g) {
        case 1: column_launch<1>(D, seg_lo, seg_hi, base, nb, mask, out, stride, grid, stream); break;
        case 2: column_launch<2>(D, seg_lo, seg_hi, base, nb, mask, out, stride, grid, stream); break;
        case 4: column_launch<4>(D, seg_lo, seg_hi, base, nb, mask, out, stride, grid, stream); break;
        case 16: column_launch<16>(D, seg_lo, seg_hi, base, nb, mask, out, stride, grid, stream); break;
        default: column_launch<8>(D, seg_lo, seg_hi, base, nb, mask, out, stride, grid, stream); break;
    }
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_column_dev(const DevCSR& D, const int* seg, const int* ap_beam, int K, const int* beam_off,
                              const int* rows, const int* cols, int max_nb, const float* mask, float* slab, int ld,
                              const CGDev* cg, int num_sms, cudaStream_t stream, int* launches) {
    if (D.n_rows == 0) return cudaSuccess;
    const int grid = num_sms * 8;
    if (column_by_beams(D)) {
        column_beam_launch(D, 0, 0, 0, ap_beam, K, beam_off, rows, cols, max_nb, mask, slab, 1, ld, cg, grid,
                           stream);
        ++*launches;
        return cudaGetLastError();
    }
    switch (D.tune_col_g) {
        case 1:
            column_dev_launch<1>(D, seg, ap_beam, K, beam_off, rows, cols, max_nb, mask, slab, ld, cg, grid, stream);
            break;
        case 2:
            column_dev_launch<2>(D, seg, ap_beam, K, beam_off, rows, cols, max_nb, mask, slab, ld, cg, grid, stream);
            break;
        case 4:
            column_dev_launch<4>(D, seg, ap_beam, K, beam_off, rows, cols, max_nb, mask, slab, ld, cg, grid, stream);
            break;
        case 16:
            column_dev_launch<16>(D, seg, ap_beam, K, beam_off, rows, cols, max_nb, mask, slab, ld, cg, grid, stream);
            break;
        default:
            column_dev_launch<8>(D, seg, ap_beam, K, beam_off, rows, cols, max_nb, mask, slab, ld, cg, grid, stream);
            break;
    }
    ++*launches;
    return cudaGetLastError();
}

template <int G>
static void commit_column_launch(const DevCSR& D, const CommitArgs& ca, size_t sm, int grid, cudaStream_t stream) {
    if (D.prec == DAO_PREC_FP16)
        k_commit_column<G, DAO_PREC_FP16><<<grid, 256, sm, stream>>>(nullptr, nullptr, D.col16, D.val16, D.scale,
                                                                      D.n_rows, ca, D.beam_rowptr, D.beam_col,
                                                                      nullptr, D.beam_val16);
    else if (D.prec == DAO_PREC_BF16)
        k_commit_column<G, DAO_PREC_BF16><<<grid, 256, sm, stream>>>(nullptr, nullptr, D.col16, D.val16, D.scale,
                                                                      D.n_rows, ca, D.beam_rowptr, D.beam_col,
                                                                      nullptr, D.beam_val16);
    else
        k_commit_column<G, DAO_PREC_FP32><<<grid, 256, sm, stream>>>(D.col, D.val, nullptr, nullptr, D.scale,
                                                                      D.n_rows, ca, D.beam_rowptr, D.beam_col,
                                                                      D.beam_val32, nullptr);
}

cudaError_t launch_commit_column(const DevCSR& D, const CommitArgs& ca, int max_nb, int num_sms, cudaStream_t stream,
                                 int* launches) {
    if (D.n_rows == 0 || ca.cg == nullptr) return cudaErrorInvalidValue;
    const int grid = num_sms * 8;
    const size_t sm = (size_t)std::max(ca.n_beams, 1) * sizeof(double) + (size_t)std::max(max_nb, 1) * sizeof(float);
    if (column_by_beams(D)) {
        commit_column_launch<0>(D, ca, sm, grid, stream);
        ++*launches;
        return cudaGetLastError();
    }
    switch (D.tune_col_g) {
        case 1: commit_column_launch<1>(D, ca, sm, grid, stream); break;
        case 2: commit_column_launch<2>(D, ca, sm, grid, stream); break;
        case 4: commit_column_launch<4>(D, ca, sm, grid, stream); break;
        case 16: commit_column_launch<16>(D, ca, sm, grid, stream); break;
        default: commit_column_launch<8>(D, ca, sm, grid, stream); break;
    }
    ++*launches;
    return cudaGetLastError();
}

namespace {
// Reads a buffer larger than L2 so that L2 holds only clean lines of it
// (overwriting it instead would leave dirty lines whose write-back overlaps
// whatever runs next); `sink` is written only for an impossible sum.
__global__ void __launch_bounds__(256) k_l2_evict(const float4* __restrict__ buf, size_t n, float* __restrict__ sink) {
    float a = 0.f;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float4 v = buf[i];  // default caching: the lines replace what L2 held
        a += v.x + v.y + v.z + v.w;
    }
    if (a == -1.2345e37f) *sink = a;
}
}  // namespace

cudaError_t launch_l2_evict(const void* buf, size_t bytes, float* sink, int num_sms, cudaStream_t stream) {
    k_l2_evict<<<num_sms * 8, 256, 0, stream>>>(static_cast<const float4*>(buf), bytes / sizeof(float4), sink);
    return cudaGetLastError();
}

cudaError_t launch_fluence(const int* ap_beam, const int* ap_lr, int lr_stride, const double* y, int K,
                           const int4* binfo, int N, float* x, cudaStream_t stream, int* launches) {
    if (N == 0) return cudaSuccess;
    k_fluence<<<(N + 255) / 256, 256, 0, stream>>>(ap_beam, ap_lr, lr_stride, y, K, binfo, N, x);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace dao
