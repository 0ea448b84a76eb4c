// Device bodies of the sparse kernels of spmv.cu (the stand-alone kernels and
// the fused kernels of the device-driven round): the block sum of the
// transposed SpMV, one beamlet row of D^T (a2, the bracketed sum of Eq. 8),
// the aperture column over a beam's segment of each voxel row (a4, Eq. 2),
// and the 16-bit unpacking.  Fixed summation orders: a row's result depends
// only on the block size (a2) or on the lanes per voxel row (a4), not on
// which block or warp computes it.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dao_internal.h"

namespace dao {
namespace {

// Sum over a block: FP32 within each warp, FP64 across the warps (FP64 issues
// at 1/64 of the FP32 rate on this part, so it is kept to one lane per warp).
template <int NT>
__device__ __forceinline__ double block_sum_mixed(float v, double* s_red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_red[warp] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t += s_red[w];
    return t;
}

template <bool BF>
__device__ __forceinline__ float2 unpack2(unsigned w) {
    if (BF) {
        __nv_bfloat162 h;
        *reinterpret_cast<unsigned*>(&h) = w;
        return __bfloat1622float2(h);
    } else {
        __half2 h;
        *reinterpret_cast<unsigned*>(&h) = w;
        return __half22float2(h);
    }
}

template <bool BF>
__device__ __forceinline__ float unpack1(unsigned short b) {
    if (BF) {
        __nv_bfloat16 h;
        *reinterpret_cast<unsigned short*>(&h) = b;
        return __bfloat162float(h);
    } else {
        __half h;
        *reinterpret_cast<unsigned short*>(&h) = b;
        return __half2float(h);
    }
}

// a2, one beamlet row of D^T by a block of BT threads (every thread calls it);
// the result is valid in thread 0.  Software pipeline: the next group's indices
// and values (DRAM) are in flight while the current group's pi gathers (L2)
// and products run.
template <int BT>
__device__ __forceinline__ float dt_row_sum(const int* __restrict__ rowptr, const int4* __restrict__ col4,
                                            const float4* __restrict__ val4, int row, const float* __restrict__ pi,
                                            double* s_red) {
    const int p0 = rowptr[row] >> 2, p1 = rowptr[row + 1] >> 2;
    float acc = 0.f;
    int p = p0 + (int)threadIdx.x;
    int4 cn = make_int4(0, 0, 0, 0);
    float4 vn = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p < p1) {
        cn = __ldg(col4 + p);
        vn = __ldg(val4 + p);
    }
    while (p < p1) {
        const int4 c = cn;
        const float4 v = vn;
        p += BT;
        if (p < p1) {
            cn = __ldg(col4 + p);
            vn = __ldg(val4 + p);
        }
        const float a0 = __ldg(pi + c.x), a1 = __ldg(pi + c.y),
                    a2 = __ldg(pi + c.z), a3 = __ldg(pi + c.w);
        acc = fmaf(v.x, a0, acc);
        acc = fmaf(v.y, a1, acc);
        acc = fmaf(v.z, a2, acc);
        acc = fmaf(v.w, a3, acc);
    }
    return (float)block_sum_mixed<BT>(acc, s_red);
}

// a2 with rows padded to 8 entries: two int4 loads of voxel indices and one uint4
// of values per 8 entries; the row's scale is applied once at the end.
template <int BT, bool BF>
__device__ __forceinline__ float dt16_row_sum(const int* __restrict__ rowptr, const int4* __restrict__ col4,
                                              const uint4* __restrict__ val8, const float* __restrict__ scale, int row,
                                              const float* __restrict__ pi, double* s_red) {
    const int p0 = rowptr[row] >> 3, p1 = rowptr[row + 1] >> 3;
    float acc = 0.f;
    for (int p = p0 + (int)threadIdx.x; p < p1; p += BT) {
        const int4 c0 = __ldg(col4 + 2 * p);
        const int4 c1 = __ldg(col4 + 2 * p + 1);
        const uint4 vw = __ldg(val8 + p);
        const float2 a = unpack2<BF>(vw.x), b = unpack2<BF>(vw.y), c = unpack2<BF>(vw.z), d = unpack2<BF>(vw.w);
        acc = fmaf(a.x, __ldg(pi + c0.x), acc);
        acc = fmaf(a.y, __ldg(pi + c0.y), acc);
        acc = fmaf(b.x, __ldg(pi + c0.z), acc);
        acc = fmaf(b.y, __ldg(pi + c0.w), acc);
        acc = fmaf(c.x, __ldg(pi + c1.x), acc);
        acc = fmaf(c.y, __ldg(pi + c1.y), acc);
        acc = fmaf(d.x, __ldg(pi + c1.z), acc);
        acc = fmaf(d.y, __ldg(pi + c1.w), acc);
    }
    const double sres = block_sum_mixed<BT>(acc, s_red);
    return (float)(sres * (double)scale[row]);
}

// a2 with consecutive entries on consecutive threads: thread t takes entries
// e0 + t, e0 + t + BT, ... of the row, U at a time, the next U requested while
// the current U's pi gathers run (a deeper pipeline needs more registers, and
// then the 64-thread blocks of every row no longer fit one wave).  A row of D^T
// lists its voxels in increasing
// order, so the 32 gathers of one warp instruction fall on a few cache lines
// (the grouped form above spreads them over 8 x 32 entries).  Scalar loads of
// the voxel index (and the 16-bit value); padding entries (value 0, a valid
// voxel) are summed like the others.
template <int BT, int U, class LoadV>
__device__ __forceinline__ float dt_row_consecutive(int e0, int e1, const int* __restrict__ col, LoadV loadv,
                                                    const float* __restrict__ pi) {
    float acc = 0.f;
    int e = e0 + (int)threadIdx.x;
    int cn[U];
    float vn[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
        const int p = e + q * BT;
        cn[q] = p < e1 ? __ldg(col + p) : -1;
        vn[q] = p < e1 ? loadv(p) : 0.f;
    }
    while (e < e1) {
        int c[U];
        float v[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            c[q] = cn[q];
            v[q] = vn[q];
        }
        e += BT * U;
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const int p = e + q * BT;
            cn[q] = p < e1 ? __ldg(col + p) : -1;
            vn[q] = p < e1 ? loadv(p) : 0.f;
        }
        float a[U];
#pragma unroll
        for (int q = 0; q < U; ++q) a[q] = c[q] >= 0 ? __ldg(pi + c[q]) : 0.f;
#pragma unroll
        for (int q = 0; q < U; ++q) acc = fmaf(v[q], a[q], acc);
    }
    return acc;
}

template <int BT>
__device__ __forceinline__ float dt_row_sum_lc(const int* __restrict__ rowptr, const int* __restrict__ col,
                                               const float* __restrict__ val, int row, const float* __restrict__ pi,
                                               double* s_red) {
    const float acc = dt_row_consecutive<BT, 4>(rowptr[row], rowptr[row + 1], col,
                                                [&](int p) { return __ldg(val + p); }, pi);
    return (float)block_sum_mixed<BT>(acc, s_red);
}

template <int BT, bool BF>
__device__ __forceinline__ float dt16_row_sum_lc(const int* __restrict__ rowptr, const int* __restrict__ col,
                                                 const unsigned short* __restrict__ val,
                                                 const float* __restrict__ scale, int row,
                                                 const float* __restrict__ pi, double* s_red) {
    const float acc = dt_row_consecutive<BT, 4>(rowptr[row], rowptr[row + 1], col,
                                                [&](int p) { return unpack1<BF>(__ldg(val + p)); }, pi);
    const double sres = block_sum_mixed<BT>(acc, s_red);
    return (float)(sres * (double)scale[row]);
}

// ---- a4 ---------------------------------------------------------------------
// The first entry of beam b in D by beams: the totals of the beams before it.
__device__ __forceinline__ int beam_entry_base(const int* __restrict__ brp_all, int V, int b) {
    int e = 0;
    for (int bb = 0; bb < b; ++bb) e += __ldg(brp_all + (size_t)bb * (V + 1) + V);
    return e;
}

// a4 from D by beams: one lane per voxel row over the row's part of beam b
// (entries e_base + brp[j] .. e_base + brp[j + 1] - 1, one contiguous range, so the lanes of a
// warp read consecutive bytes), summed in order from 0 as the one-lane form
// over D's segments sums them; the mask is pre-multiplied by the scales for
// 16-bit values.  Four entries requested ahead of their products.
template <bool W16, bool BF>
__device__ __forceinline__ void column_beam_body(const int* __restrict__ brp, int e_base,
                                                 const unsigned short* __restrict__ bcol,
                                                 const float* __restrict__ bval32,
                                                 const unsigned short* __restrict__ bval16, int V,
                                                 const float* smask, float* __restrict__ out, int stride, int wbase,
                                                 int wcount) {
    for (int j = wbase + (int)threadIdx.x; j < V; j += wcount) {
        const int p0 = __ldg(brp + j) + e_base, p1 = __ldg(brp + j + 1) + e_base;
        float acc = 0.f;
        for (int p = p0; p < p1; p += 4) {
            unsigned short c[4];
            float v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool in = p + q < p1;
                c[q] = in ? __ldg(bcol + p + q) : (unsigned short)0;
                if constexpr (W16)
                    v[q] = in ? unpack1<BF>(__ldg(bval16 + p + q)) : 0.f;
                else
                    v[q] = in ? __ldg(bval32 + p + q) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (p + q < p1) acc = fmaf(v[q], smask[c[q]], acc);
        }
        out[(size_t)j * stride] = acc;
    }
}

// The caller's threads are [wbase, wbase + blockDim) of wcount threads sharing
// the rows (a grid, or a group of blocks).
// G lanes per voxel row over the row's segment of beam b (columns base ..
// base + nb - 1); mask[c] in {0, 1} marks the aperture's open beamlets.
template <int G>
__device__ __forceinline__ void column_body(const int* __restrict__ col, const float* __restrict__ val,
                                            const int* __restrict__ seg_lo, const int* __restrict__ seg_hi,
                                            int V, int base, const float* smask, float* __restrict__ out,
                                            int stride, int wbase, int wcount) {
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    constexpr int RPW = 32 / G;
    const int warp_global = (wbase + (int)threadIdx.x) >> 5;
    const int n_warps = wcount >> 5;
    const int n_tiles = (V + RPW - 1) / RPW;
    // the next tile's segment bounds are loaded while this tile's entries are
    int row = warp_global * RPW + lane / G;
    int lo = 0, hi = 0;
    if (warp_global < n_tiles && row < V) {
        lo = seg_lo[row];
        hi = seg_hi[row];
    }
    for (int t = warp_global; t < n_tiles; t += n_warps) {
        const int row_c = row, lo_c = lo, hi_c = hi;
        row = (t + n_warps) * RPW + lane / G;
        lo = hi = 0;
        if (t + n_warps < n_tiles && row < V) {
            lo = seg_lo[row];
            hi = seg_hi[row];
        }
        float acc = 0.f;
        for (int p = lo_c + sub; p < hi_c; p += G) acc = fmaf(__ldg(val + p), smask[__ldg(col + p) - base], acc);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (row_c < V && sub == 0) out[(size_t)row_c * stride] = acc;
    }
}

// a4 over beam b's segment of each row; the mask is pre-multiplied by the scales.
template <int G, bool BF>
__device__ __forceinline__ void column16_body(const unsigned short* __restrict__ col,
                                              const unsigned short* __restrict__ val,
                                              const int* __restrict__ seg_lo, const int* __restrict__ seg_hi, int V,
                                              int base, const float* smask, float* __restrict__ out, int stride,
                                              int wbase, int wcount) {
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    constexpr int RPW = 32 / G;
    const int warp_global = (wbase + (int)threadIdx.x) >> 5;
    const int n_warps = wcount >> 5;
    const int n_tiles = (V + RPW - 1) / RPW;
    // the next tile's segment bounds are loaded while this tile's entries are
    int row = warp_global * RPW + lane / G;
    int lo = 0, hi = 0;
    if (warp_global < n_tiles && row < V) {
        lo = seg_lo[row];
        hi = seg_hi[row];
    }
    for (int t = warp_global; t < n_tiles; t += n_warps) {
        const int row_c = row, lo_c = lo, hi_c = hi;
        row = (t + n_warps) * RPW + lane / G;
        lo = hi = 0;
        if (t + n_warps < n_tiles && row < V) {
            lo = seg_lo[row];
            hi = seg_hi[row];
        }
        float acc = 0.f;
        for (int p = lo_c + sub; p < hi_c; p += G)
            acc = fmaf(unpack1<BF>(__ldg(val + p)), smask[__ldg(col + p) - base], acc);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (row_c < V && sub == 0) out[(size_t)row_c * stride] = acc;
    }
}

}  // namespace
}  // namespace dao
