// Device-side construction of a plan's matrices from the caller's CSR of D
// (uploaded as is): the checks of the caller's rows and labels, the padded
// row offsets (a scan), the padded voxel-major layout, the per-row beam segments,
// the per-beamlet scales of the 16-bit storage, and the beamlet-major
// transpose D^T by a stable counting sort.
//
// The transpose keeps every row of D^T in increasing voxel order, the order a
// sequential counting sort gives, without sorting: the voxel rows are cut into
// chunks; C[chunk][i] counts chunk's entries of beamlet i (shared-memory
// integer atomics, so the counts are exact); a scan over chunks turns the
// counts into each chunk's first slot in every row of D^T; then one warp per
// chunk walks its entries in CSR order and places each at its beamlet's next
// slot, lanes that share a beamlet taking consecutive slots in lane order.
#include <algorithm>
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

// Beamlet counters of one block live in shared memory for a tile of TILE_N
// beamlets; a matrix with more beamlets runs a grid of (chunk, tile) blocks.
constexpr int TILE_N = 12288;
constexpr int STATS_T = 256;

// Per (chunk, beamlet tile): C[chunk][i] = the chunk's entries of beamlet i,
// counted in shared memory, and s_i = max |D_ij| over them folded into smax
// (bits of a non-negative float, ordered like the floats) with one atomicMax
// per beamlet the chunk touches.
__global__ void __launch_bounds__(STATS_T) k_chunk_stats(const int64_t* __restrict__ rp, const int* __restrict__ col,
                                                         const float* __restrict__ val, int V, int CH, int N,
                                                         int* __restrict__ C, unsigned* __restrict__ smax) {
    extern __shared__ unsigned s_stats[];
    const int ch = blockIdx.x, i0 = blockIdx.y * TILE_N;
    const int nt = min(TILE_N, N - i0);
    unsigned* s_cnt = s_stats;
    unsigned* s_mx = s_stats + nt;
    for (int t = threadIdx.x; t < 2 * nt; t += STATS_T) s_stats[t] = 0u;
    __syncthreads();
    const int64_t p0 = rp[(int64_t)ch * CH], p1 = rp[min((int64_t)V, (int64_t)(ch + 1) * CH)];
    for (int64_t p = p0 + threadIdx.x; p < p1; p += STATS_T) {
        const int c = col[p] - i0;
        if (c >= 0 && c < nt) {
            atomicAdd(&s_cnt[c], 1u);
            atomicMax(&s_mx[c], __float_as_uint(fabsf(val[p])));
        }
    }
    __syncthreads();
    int* Cc = C + (size_t)ch * N + i0;
    for (int t = threadIdx.x; t < nt; t += STATS_T) {
        const unsigned n = s_cnt[t];
        Cc[t] = (int)n;
        if (n) atomicMax(&smax[i0 + t], s_mx[t]);
    }
}

// Column i of C becomes each chunk's first slot relative to the start of row
// i of D^T, and cnt[i] its total.  Block of 32 beamlets x 32 chunk segments:
// segment sums, a scan over the segments in shared memory, then each segment
// rewritten from its offset.
__global__ void __launch_bounds__(1024) k_chunk_scan(int* __restrict__ C, int n_ch, int N, int* __restrict__ cnt) {
    __shared__ int s_sum[32][33];
    const int x = threadIdx.x, y = threadIdx.y;
    const int i = blockIdx.x * 32 + x;
    const int per = (n_ch + 31) / 32;
    const int c0 = min(n_ch, y * per), c1 = min(n_ch, c0 + per);
    int sum = 0;
    if (i < N)
        for (int ch = c0; ch < c1; ++ch) sum += C[(size_t)ch * N + i];
    s_sum[y][x] = sum;
    __syncthreads();
    int run = 0;
    for (int t = 0; t < y; ++t) run += s_sum[t][x];
    if (i < N) {
        if (y == 31) cnt[i] = run + sum;
        for (int ch = c0; ch < c1; ++ch) {
            const int v = C[(size_t)ch * N + i];
            C[(size_t)ch * N + i] = run;
            run += v;
        }
    }
}

// Placement: one warp per (chunk, beamlet tile of width tw) walks the chunk's
// voxel rows in order, the lanes over a row's entries (distinct beamlets, so no
// two lanes share a counter).  The next slot of each beamlet of the tile is a
// shared-memory counter (row start of D^T + the chunk's offset).  Row starts
// (PL_ROWS rows at a time) and entries (PL_STG at a time) are staged in shared
// memory with coalesced loads; a row that straddles two stages is finished in
// the second.  The walk is a chain of shared-memory round trips per row, so
// the tiles are made narrow enough for about 24 warps per SM.
constexpr int PL_ROWS = 256, PL_STG = 512;

__global__ void __launch_bounds__(32) k_chunk_place(const int64_t* __restrict__ rp, const int* __restrict__ col,
                                                    const float* __restrict__ val, int V, int CH, int N, int tw,
                                                    const int* __restrict__ C, const int* __restrict__ trow,
                                                    int* __restrict__ tcol, float* __restrict__ tval) {
    extern __shared__ int s_pl[];
    const int ch = blockIdx.x, i0 = blockIdx.y * tw;
    const int nt = min(tw, N - i0);
    int* s_slot = s_pl;                   // nt next slots
    int* s_row = s_slot + nt;             // PL_ROWS + 1 row starts, relative to the window's first entry
    int* s_col = s_row + PL_ROWS + 1;     // PL_STG staged entries: beamlet - i0
    float* s_val = reinterpret_cast<float*>(s_col + PL_STG);
    const int lane = threadIdx.x;
    for (int t = lane; t < nt; t += 32) s_slot[t] = trow[i0 + t] + C[(size_t)ch * N + i0 + t];
    const int j0 = ch * CH, j1 = (int)min((int64_t)V, (int64_t)j0 + CH);
    for (int w0 = j0; w0 < j1; w0 += PL_ROWS) {
        const int nr = min(PL_ROWS, j1 - w0);
        const int64_t e0 = rp[w0];
        __syncwarp();
        for (int r = lane; r <= nr; r += 32) s_row[r] = (int)(rp[w0 + r] - e0);
        __syncwarp();
        const int ne = s_row[nr];
        int r = 0;                        // next row to place (may have started in the previous stage)
        for (int s0 = 0; s0 < ne; s0 += PL_STG) {
            const int s1 = min(ne, s0 + PL_STG);
            __syncwarp();
#pragma unroll 8
            for (int q = s0 + lane; q < s1; q += 32) {
                s_col[q - s0] = col[e0 + q] - i0;
                s_val[q - s0] = val[e0 + q];
            }
            __syncwarp();
            // rows with entries in [s0, s1); the last may continue in the next stage
            while (r < nr && s_row[r] < s1) {
                const int a = max(s_row[r], s0), b = min(s_row[r + 1], s1);
                for (int q = a + lane; q < b; q += 32) {
                    const int c = s_col[q - s0];
                    if (c >= 0 && c < nt) {
                        const int pos = s_slot[c];
                        s_slot[c] = pos + 1;
                        tcol[pos] = w0 + r;
                        tval[pos] = s_val[q - s0];
                    }
                }
                __syncwarp();
                if (s_row[r + 1] > s1) break;   // continues in the next stage
                ++r;
            }
        }
    }
}

size_t place_smem(int nt) { return sizeof(int) * ((size_t)nt + PL_ROWS + 1 + 2 * PL_STG); }

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

cudaError_t build_stats(const int64_t* rp, const int* col, const float* val, int V, int CH, int N, int n_ch,
                        int* C, int* cnt, unsigned* smax, unsigned* dmax, int num_sms, cudaStream_t s) {
    const int n_tile = (N + TILE_N - 1) / TILE_N;
    const size_t sm_stats = 2 * sizeof(unsigned) * (size_t)std::min(N, TILE_N);
    // the attribute is process-wide and plans may be created from several threads at
    // once: always the largest size any launch asks for, never this plan's own
    cudaError_t e = cudaFuncSetAttribute(k_chunk_stats, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * sizeof(unsigned) * TILE_N));
    if (e == cudaSuccess) e = cudaMemsetAsync(smax, 0, sizeof(unsigned) * N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dmax, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_chunk_stats<<<dim3(n_ch, n_tile), STATS_T, sm_stats, s>>>(rp, col, val, V, CH, N, C, smax);
    k_chunk_scan<<<(N + 31) / 32, dim3(32, 32), 0, s>>>(C, n_ch, N, cnt);
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

namespace {
// One thread per unit of 32 rows: its group count, the largest into out[0];
// the largest row into out[1].
__global__ void k_unit_max(const int* __restrict__ prow, int V, int epg, int* __restrict__ out) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int r0 = u * 32;
    if (r0 >= V) return;
    const int r1 = min(r0 + 32, V);
    atomicMax(out, (prow[r1] - prow[r0]) / epg);
    int m = 0;
    for (int r = r0; r < r1; ++r) m = max(m, prow[r + 1] - prow[r]);
    atomicMax(out + 1, m / epg);
}

// One thread per split of the merge form: at diagonal d the largest i in
// [max(0, d - G), min(d, V)] whose row i - 1 ends within the first d - i groups
// (binary search: the condition holds up to that i and fails after it).
__global__ void k_merge_path(const int* __restrict__ prow, int V, int epg, int chunk, int n_warps,
                             int2* __restrict__ out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v > n_warps) return;
    const long long G = prow[V] / epg;
    const long long d = min((long long)v * chunk, (long long)V + G);
    long long lo = max(0LL, d - G), hi = min(d, (long long)V);
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if ((long long)(prow[mid] / epg) <= d - mid)  // row mid - 1 ends within d - mid groups
            lo = mid;
        else
            hi = mid - 1;
    }
    out[v] = make_int2((int)lo, (int)(d - lo));
}
}  // namespace

namespace {
constexpr int BEAM_TILE = 1024;  // rows per tile of the beams' row-offset scan

// Inclusive sum over the block of one int per thread (BEAM_TILE threads);
// *total receives the block's sum.
__device__ __forceinline__ int block_scan_incl(int v, int* s_w, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) s_w[w] = v;
    __syncthreads();
    if (w == 0) {
        int x = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += u;
        }
        s_w[lane] = x;  // inclusive sums of the warps' totals
    }
    __syncthreads();
    const int r = v + (w > 0 ? s_w[w - 1] : 0);
    *total = s_w[BEAM_TILE / 32 - 1];
    __syncthreads();
    return r;
}

__device__ __forceinline__ int beam_seg_len(const int* __restrict__ seg, int V, int b, int j) {
    return j < V ? seg[(size_t)(b + 1) * V + j] - seg[(size_t)b * V + j] : 0;
}

// Per (tile, beam): the sum of the tile's segment lengths of the beam.
__global__ void __launch_bounds__(BEAM_TILE) k_beam_tiles(const int* __restrict__ seg, int V, int n_tiles,
                                                         int* __restrict__ tsum) {
    __shared__ int s_w[BEAM_TILE / 32];
    const int b = blockIdx.y, t = blockIdx.x;
    int total = 0;
    block_scan_incl(beam_seg_len(seg, V, b, t * BEAM_TILE + (int)threadIdx.x), s_w, &total);
    if (threadIdx.x == 0) tsum[(size_t)b * n_tiles + t] = total;
}

// Per beam: the tile sums turned into the tiles' first offsets (in place),
// the beam's total into brp[b][V].
__global__ void __launch_bounds__(BEAM_TILE) k_beam_tile_scan(int* __restrict__ tsum, int n_tiles, int V,
                                                             int* __restrict__ brp) {
    __shared__ int s_w[BEAM_TILE / 32];
    const int b = blockIdx.x;
    int carry = 0;
    for (int c0 = 0; c0 < n_tiles; c0 += BEAM_TILE) {
        const int i = c0 + (int)threadIdx.x;
        const int v = i < n_tiles ? tsum[(size_t)b * n_tiles + i] : 0;
        int total = 0;
        const int incl = block_scan_incl(v, s_w, &total);
        if (i < n_tiles) tsum[(size_t)b * n_tiles + i] = carry + incl - v;
        carry += total;
    }
    if (threadIdx.x == 0) brp[(size_t)b * (V + 1) + V] = carry;
}

// Per (tile, beam): the row offsets of the tile's rows, counted from the
// beam's first entry; beam b's entries follow those of beams 0 .. b - 1 (the
// totals brp[b'][V]).
__global__ void __launch_bounds__(BEAM_TILE) k_beam_offsets(const int* __restrict__ seg, int V, int n_tiles,
                                                           const int* __restrict__ toff, int* __restrict__ brp) {
    __shared__ int s_w[BEAM_TILE / 32];
    const int b = blockIdx.y, t = blockIdx.x;
    const int j = t * BEAM_TILE + (int)threadIdx.x;
    const int len = beam_seg_len(seg, V, b, j);
    int total = 0;
    const int incl = block_scan_incl(len, s_w, &total);
    if (j < V) brp[(size_t)b * (V + 1) + j] = toff[(size_t)b * n_tiles + t] + incl - len;
}

// One thread per (beam, row): the row's segment of the beam, with the beamlet
// index made local to the beam.
template <int PREC>
__global__ void k_beam_fill(const int* __restrict__ seg, int V, int B, const int* __restrict__ beam_off,
                            const int* __restrict__ brp, const int* __restrict__ col, const float* __restrict__ val,
                            const unsigned short* __restrict__ col16, const unsigned short* __restrict__ val16,
                            unsigned short* __restrict__ bcol, float* __restrict__ bval32,
                            unsigned short* __restrict__ bval16) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * V) return;
    const int b = (int)(i / V), j = (int)(i % V);
    const int q0 = seg[(size_t)b * V + j], q1 = seg[(size_t)(b + 1) * V + j];
    const int base = beam_off[b];
    int64_t d0 = brp[(size_t)b * (V + 1) + j];
    for (int bb = 0; bb < b; ++bb) d0 += brp[(size_t)bb * (V + 1) + V];  // the beams before b
    for (int q = q0; q < q1; ++q) {
        const int64_t d = d0 + (q - q0);
        if constexpr (PREC == DAO_PREC_FP32) {
            bcol[d] = (unsigned short)(col[q] - base);
            bval32[d] = val[q];
        } else {
            bcol[d] = (unsigned short)(col16[q] - base);
            bval16[d] = val16[q];
        }
    }
}
}  // namespace

int beam_scan_tiles(int V) { return (V + BEAM_TILE - 1) / BEAM_TILE; }

cudaError_t build_beam_rows(const int* seg, int V, int B, int* brp, int* tmp, cudaStream_t s) {
    if (B < 1 || V < 1) return cudaSuccess;
    const int nt = beam_scan_tiles(V);
    k_beam_tiles<<<dim3(nt, B), BEAM_TILE, 0, s>>>(seg, V, nt, tmp);
    k_beam_tile_scan<<<B, BEAM_TILE, 0, s>>>(tmp, nt, V, brp);
    k_beam_offsets<<<dim3(nt, B), BEAM_TILE, 0, s>>>(seg, V, nt, tmp, brp);
    return cudaGetLastError();
}

cudaError_t build_beam_fill(int prec, const int* seg, int V, int B, const int* beam_off, const DevCSR& D,
                            cudaStream_t s) {
    const int64_t n = (int64_t)B * V;
    if (n == 0) return cudaSuccess;
    const unsigned g = (unsigned)((n + 255) / 256);
    if (prec == DAO_PREC_FP32)
        k_beam_fill<DAO_PREC_FP32><<<g, 256, 0, s>>>(seg, V, B, beam_off, D.beam_rowptr, D.col, D.val, nullptr,
                                                     nullptr, D.beam_col, D.beam_val32, nullptr);
    else
        k_beam_fill<DAO_PREC_FP16><<<g, 256, 0, s>>>(seg, V, B, beam_off, D.beam_rowptr, nullptr, nullptr, D.col16,
                                                     D.val16, D.beam_col, nullptr, D.beam_val16);
    return cudaGetLastError();
}

cudaError_t build_merge_path(const int* prow, int V, int epg, int chunk, int n_warps, int2* out, cudaStream_t s) {
    k_merge_path<<<(n_warps + 1 + 255) / 256, 256, 0, s>>>(prow, V, epg, chunk, n_warps, out);
    return cudaGetLastError();
}

cudaError_t build_unit_max(const int* prow, int V, int epg, int* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, 2 * sizeof(int), s);
    if (e != cudaSuccess || V < 1) return e;
    const int units = (V + 31) / 32;
    k_unit_max<<<(units + 255) / 256, 256, 0, s>>>(prow, V, epg, out);
    return cudaGetLastError();
}

cudaError_t build_transpose_place(int prec, const int64_t* rp, const int* col, const float* val, int V, int CH, int N,
                                  int n_ch, int* C, const int* cnt, const float* scale, DevCSR& Dt, float* tval,
                                  int num_sms, cudaStream_t s) {
    const int split = std::max(1, std::min(16, (24 * num_sms + n_ch - 1) / n_ch));
    const int tw = std::min(TILE_N, (N + split - 1) / split);
    const int n_tile = (N + tw - 1) / tw;
    const size_t sm_place = place_smem(tw);
    // process-wide: the largest size any launch asks for (see build_stats)
    cudaError_t e = cudaFuncSetAttribute(k_chunk_place, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)place_smem(TILE_N));
    if (e != cudaSuccess) return e;
    k_chunk_place<<<dim3(n_ch, n_tile), 32, sm_place, s>>>(rp, col, val, V, CH, N, tw, C, Dt.rowptr, Dt.col, tval);
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
