// Device-side construction of a plan's matrices from the caller's CSR of D
// (uploaded as is): the checks of the caller's rows and labels, the padded
// row offsets (a scan), the padded voxel-major layout, the per-row beam segments,
// the per-beamlet scales of the 16-bit storage, and the beamlet-major
// transpose D^T by a stable counting sort.
//
// The transpose keeps every row of D^T in increasing voxel order, the order a
// sequential counting sort gives, without sorting: the voxel rows are cut into
// chunks; C[chunk][i] counts chunk's entries of beamlet i (integer atomics, so
// the counts are exact); a scan over chunks turns the counts into each chunk's
// first slot in every row of D^T; then one warp per chunk walks its voxels in
// order and places each entry at its beamlet's next slot.  Entries of one voxel
// have distinct beamlets, so the lanes of a warp never share a slot counter.
#include <climits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dao_internal.h"

namespace dao {

namespace {

constexpr unsigned FULL = 0xffffffffu;

template <int PREC>
__device__ __forceinline__ unsigned short to16(float r) {
    if (PREC == DAO_PREC_FP16) return __half_as_ushort(__float2half_rn(r));
    return __bfloat16_as_ushort(__float2bfloat16_rn(r));
}

// s_i = max_j |D_ij| as the bits of a non-negative float (ordered like the
// floats), and the overall maximum for the pricing tolerance.
__global__ void k_colmax(const int* __restrict__ col, const float* __restrict__ val, int64_t nnz,
                         unsigned* __restrict__ smax) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        atomicMax(&smax[col[p]], __float_as_uint(fabsf(val[p])));
}

// scale_i = s_i, or 1 for a beamlet without entries; dmax = max_i s_i.
__global__ void k_scale_fix(unsigned* __restrict__ smax, int N, unsigned* __restrict__ dmax) {
    __shared__ unsigned s_m[8];
    unsigned m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const unsigned b = smax[i];
        m = max(m, b);
        const float s = __uint_as_float(b);
        reinterpret_cast<float*>(smax)[i] = s > 0.f ? s : 1.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = max(t, s_m[w]);
        atomicMax(dmax, t);
    }
}

// Padded voxel-major D, one warp per voxel row; padding repeats the row's last
// column with value 0.
template <int PREC>
__global__ void k_fill_d(const int64_t* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ val,
                         const int* __restrict__ prow, int V, const float* __restrict__ scale,
                         int* __restrict__ dcol, float* __restrict__ dval, unsigned short* __restrict__ dcol16,
                         unsigned short* __restrict__ dval16) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= V) return;
    const int64_t p0 = rp[j];
    const int len = (int)(rp[j + 1] - p0);
    const int q0 = prow[j], n = prow[j + 1] - q0;
    const int last = len > 0 ? col[p0 + len - 1] : 0;
    for (int t = lane; t < n; t += 32) {
        const int c = t < len ? col[p0 + t] : last;
        const float v = t < len ? val[p0 + t] : 0.f;
        if (PREC == DAO_PREC_FP32) {
            dcol[q0 + t] = c;
            dval[q0 + t] = v;
        } else {
            dcol16[q0 + t] = (unsigned short)c;
            dval16[q0 + t] = to16<PREC>(v / scale[c]);
        }
    }
}

// seg[b][j] = first padded position of row j with column >= beam_off[b];
// seg[B][j] = the end of row j's real entries.
__global__ void k_seg(const int64_t* __restrict__ rp, const int* __restrict__ col, const int* __restrict__ prow,
                      int V, const int* __restrict__ beam_off, int B, int* __restrict__ seg) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= V) return;
    const int64_t p0 = rp[j];
    const int len = (int)(rp[j + 1] - p0);
    const int q0 = prow[j];
    int t = 0;
    for (int b = 0; b < B; ++b) {
        const int lo = beam_off[b];
        while (t < len && col[p0 + t] < lo) ++t;
        seg[(size_t)b * V + j] = q0 + t;
    }
    seg[(size_t)B * V + j] = q0 + len;
}

// C[chunk][i] += entries of beamlet i in the chunk's voxel rows (warp per row).
__global__ void k_chunk_count(const int64_t* __restrict__ rp, const int* __restrict__ col, int V, int CH, int N,
                              int* __restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= V) return;
    int* Cc = C + (size_t)(j / CH) * N;
    for (int64_t p = rp[j] + lane; p < rp[j + 1]; p += 32) atomicAdd(&Cc[col[p]], 1);
}

// cnt[i] = entries of beamlet i (column of D, row of D^T).
__global__ void k_col_total(const int* __restrict__ C, int n_ch, int N, int* __restrict__ cnt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int s = 0;
    for (int ch = 0; ch < n_ch; ++ch) s += C[(size_t)ch * N + i];
    cnt[i] = s;
}

// C[chunk][i] becomes the chunk's first slot in row i of D^T.
__global__ void k_chunk_scan(int* __restrict__ C, int n_ch, int N, const int* __restrict__ trow) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int run = trow[i];
    for (int ch = 0; ch < n_ch; ++ch) {
        const int t = C[(size_t)ch * N + i];
        C[(size_t)ch * N + i] = run;
        run += t;
    }
}

// One warp per chunk, voxel rows in increasing order: each entry goes to its
// beamlet's next slot.
__global__ void k_chunk_place(const int64_t* __restrict__ rp, const int* __restrict__ col,
                              const float* __restrict__ val, int V, int CH, int N, int n_ch, int* __restrict__ C,
                              int* __restrict__ tcol, float* __restrict__ tval) {
    const int lane = threadIdx.x & 31;
    const int ch = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (ch >= n_ch) return;
    int* Cc = C + (size_t)ch * N;
    const int j1 = min(V, (ch + 1) * CH);
    for (int j = ch * CH; j < j1; ++j) {
        for (int64_t p = rp[j] + lane; p < rp[j + 1]; p += 32) {
            const int c = col[p];
            const int pos = Cc[c];
            Cc[c] = pos + 1;
            tcol[pos] = j;
            tval[pos] = val[p];
        }
        __syncwarp();
    }
}

// Padding of the rows of D^T: the row's last voxel with value 0.
__global__ void k_pad_t(const int* __restrict__ trow, const int* __restrict__ cnt, int N, int* __restrict__ tcol,
                        float* __restrict__ tval) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const int q0 = trow[i], real = cnt[i], q1 = trow[i + 1];
    const int last = real > 0 ? tcol[q0 + real - 1] : 0;
    for (int q = q0 + real + lane; q < q1; q += 32) {
        tcol[q] = last;
        tval[q] = 0.f;
    }
}

// 16-bit values of D^T, row i scaled by 1 / s_i.
template <int PREC>
__global__ void k_quant_t(const float* __restrict__ tval, const int* __restrict__ trow, int N,
                          const float* __restrict__ scale, unsigned short* __restrict__ tval16) {
    const int lane = threadIdx.x & 31;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= N) return;
    const float s = scale[i];
    for (int q = trow[i] + lane; q < trow[i + 1]; q += 32) tval16[q] = to16<PREC>(tval[q] / s);
}

// The caller's CSR and labels, one warp per voxel row j: row bounds inside
// [0, nnz], columns in [0, N) and strictly increasing, finite values, label in
// [0, S).  A bad row or label is recorded as V - j under atomicMax (so the
// lowest index wins); a good row writes its padded length, a good label its
// byte and one count for its structure.  Every read of col / val is inside the
// row's checked bounds.
__global__ void k_check(const int64_t* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ val,
                        int64_t nnz, int V, int N, const int* __restrict__ label, int S, int pad,
                        int64_t* __restrict__ plen, uint8_t* __restrict__ vs8, BuildCheck* __restrict__ chk) {
    __shared__ int s_cnt[SMAX];
    for (int k = threadIdx.x; k < SMAX; k += blockDim.x) s_cnt[k] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int j = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (j < V) {
        const int64_t p0 = rp[j], p1 = rp[j + 1];
        bool ok = p0 >= 0 && p1 >= p0 && p1 <= nnz;
        if (ok) {
            bool bad = false;
            for (int64_t p = p0 + lane; p < p1; p += 32) {
                const int c = col[p];
                bad |= c < 0 || c >= N || !isfinite(val[p]);
                if (p > p0) bad |= c <= col[p - 1];
            }
            ok = !__any_sync(FULL, bad);
        }
        if (lane == 0) {
            plen[j] = ok ? (p1 - p0 + pad - 1) / pad * pad : 0;
            if (!ok) atomicMax(&chk->bad_row, V - j);
            const int l = label[j];
            if (l < 0 || l >= S) {
                atomicMax(&chk->bad_label, V - j);
            } else {
                vs8[j] = (uint8_t)l;
                atomicAdd(&s_cnt[l], 1);
            }
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < S; k += blockDim.x)
        if (s_cnt[k]) atomicAdd(&chk->count[k], s_cnt[k]);
}

// Exclusive scan of plen in three steps: block totals, a scan of the totals
// (one block), then each block's scan plus its offset.  SCAN_T threads with
// SCAN_E consecutive elements each per block.
constexpr int SCAN_T = 1024, SCAN_E = 4, SCAN_B = SCAN_T * SCAN_E;

// Exclusive scan of one value per thread across the block; returns the block total.
__device__ __forceinline__ int64_t block_exscan(int64_t v, int64_t* ex) {
    __shared__ int64_t s_w[SCAN_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < SCAN_T / 32 ? s_w[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_T / 32) s_w[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = wid > 0 ? s_w[wid - 1] : 0;
    *ex = before + x - v;
    const int64_t total = s_w[SCAN_T / 32 - 1];
    __syncthreads();  // s_w reused by the next call
    return total;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_totals(const int64_t* __restrict__ plen, int V,
                                                         int64_t* __restrict__ bsum) {
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_E;
    int64_t v = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e)
        if (i0 + e < V) v += plen[i0 + e];
    int64_t ex;
    const int64_t t = block_exscan(v, &ex);
    if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

// One block: bsum becomes exclusive; the grand total goes to chk->padded and
// (clamped) to prow[V].
__global__ void __launch_bounds__(SCAN_T) k_scan_offsets(int64_t* __restrict__ bsum, int nb, int V,
                                                          int* __restrict__ prow, BuildCheck* __restrict__ chk) {
    int64_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += SCAN_T) {
        const int b = b0 + threadIdx.x;
        const int64_t v = b < nb ? bsum[b] : 0;
        int64_t ex;
        const int64_t t = block_exscan(v, &ex);
        if (b < nb) bsum[b] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0) {
        chk->padded = carry;
        prow[V] = (int)min(carry, (int64_t)INT_MAX);
    }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_apply(const int64_t* __restrict__ plen, int V,
                                                        const int64_t* __restrict__ bsum, int* __restrict__ prow) {
    const int64_t i0 = (int64_t)blockIdx.x * SCAN_B + (int64_t)threadIdx.x * SCAN_E;
    int64_t v[SCAN_E], tot = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e) {
        v[e] = i0 + e < V ? plen[i0 + e] : 0;
        tot += v[e];
    }
    int64_t ex;
    block_exscan(tot, &ex);
    int64_t run = bsum[blockIdx.x] + ex;
#pragma unroll
    for (int e = 0; e < SCAN_E; ++e)
        if (i0 + e < V) {
            prow[i0 + e] = (int)min(run, (int64_t)INT_MAX);
            run += v[e];
        }
}

inline unsigned blocks_for(int64_t threads, int bs) { return (unsigned)((threads + bs - 1) / bs); }

}  // namespace

int check_scan_blocks(int V) { return (int)blocks_for(V, SCAN_B); }

cudaError_t build_check(const int64_t* rp, const int* col, const float* val, int64_t nnz, int V, int N,
                        const int* label, int S, int pad, int64_t* plen, int64_t* bsum, uint8_t* vs8, int* prow,
                        BuildCheck* chk, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(chk, 0, sizeof(BuildCheck), s);
    if (e != cudaSuccess) return e;
    k_check<<<blocks_for((int64_t)V * 32, 256), 256, 0, s>>>(rp, col, val, nnz, V, N, label, S, pad, plen, vs8, chk);
    const int nb = check_scan_blocks(V);
    k_scan_totals<<<nb, SCAN_T, 0, s>>>(plen, V, bsum);
    k_scan_offsets<<<1, SCAN_T, 0, s>>>(bsum, nb, V, prow, chk);
    k_scan_apply<<<nb, SCAN_T, 0, s>>>(plen, V, bsum, prow);
    return cudaGetLastError();
}

cudaError_t build_scales(const int* col, const float* val, int64_t nnz, int N, unsigned* smax, unsigned* dmax,
                         int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(smax, 0, sizeof(unsigned) * N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    if (nnz > 0) k_colmax<<<num_sms * 8, 256, 0, s>>>(col, val, nnz, smax);
    k_scale_fix<<<num_sms, 256, 0, s>>>(smax, N, dmax);
    return cudaGetLastError();
}

cudaError_t build_fill_d(int prec, const int64_t* rp, const int* col, const float* val, const int* prow, int V,
                         const float* scale, DevCSR& D, cudaStream_t s) {
    const unsigned g = blocks_for((int64_t)V * 32, 256);
    if (prec == DAO_PREC_FP32)
        k_fill_d<DAO_PREC_FP32><<<g, 256, 0, s>>>(rp, col, val, prow, V, scale, D.col, D.val, nullptr, nullptr);
    else if (prec == DAO_PREC_FP16)
        k_fill_d<DAO_PREC_FP16><<<g, 256, 0, s>>>(rp, col, val, prow, V, scale, nullptr, nullptr, D.col16, D.val16);
    else
        k_fill_d<DAO_PREC_BF16><<<g, 256, 0, s>>>(rp, col, val, prow, V, scale, nullptr, nullptr, D.col16, D.val16);
    return cudaGetLastError();
}

cudaError_t build_seg(const int64_t* rp, const int* col, const int* prow, int V, const int* beam_off, int B, int* seg,
                      cudaStream_t s) {
    k_seg<<<blocks_for(V, 256), 256, 0, s>>>(rp, col, prow, V, beam_off, B, seg);
    return cudaGetLastError();
}

cudaError_t build_transpose_count(const int64_t* rp, const int* col, int V, int CH, int N, int n_ch, int* C, int* cnt,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(C, 0, sizeof(int) * (size_t)n_ch * N, s);
    if (e != cudaSuccess) return e;
    k_chunk_count<<<blocks_for((int64_t)V * 32, 256), 256, 0, s>>>(rp, col, V, CH, N, C);
    k_col_total<<<blocks_for(N, 256), 256, 0, s>>>(C, n_ch, N, cnt);
    return cudaGetLastError();
}

cudaError_t build_transpose_place(int prec, const int64_t* rp, const int* col, const float* val, int V, int CH, int N,
                                  int n_ch, int* C, const int* cnt, const float* scale, DevCSR& Dt, float* tval,
                                  cudaStream_t s) {
    k_chunk_scan<<<blocks_for(N, 256), 256, 0, s>>>(C, n_ch, N, Dt.rowptr);
    k_chunk_place<<<blocks_for((int64_t)n_ch * 32, 256), 256, 0, s>>>(rp, col, val, V, CH, N, n_ch, C, Dt.col, tval);
    k_pad_t<<<blocks_for((int64_t)N * 32, 256), 256, 0, s>>>(Dt.rowptr, cnt, N, Dt.col, tval);
    if (prec == DAO_PREC_FP16)
        k_quant_t<DAO_PREC_FP16><<<blocks_for((int64_t)N * 32, 256), 256, 0, s>>>(tval, Dt.rowptr, N, scale,
                                                                                   Dt.val16);
    else if (prec == DAO_PREC_BF16)
        k_quant_t<DAO_PREC_BF16><<<blocks_for((int64_t)N * 32, 256), 256, 0, s>>>(tval, Dt.rowptr, N, scale,
                                                                                   Dt.val16);
    return cudaGetLastError();
}

}  // namespace dao
