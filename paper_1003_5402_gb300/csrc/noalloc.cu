// Allocation-free dose SpMV with the objective epilogue.
//
// Some callers cannot allocate device memory at call time.  One example is a
// re-planning service that reserves and pins every device buffer before an
// online adaptive fraction starts, so that a fraction can neither fail on an
// out-of-memory error nor stall on the device-wide synchronisation that
// cudaMalloc and cudaFree may imply.  Another is an application whose own
// allocator owns the whole device.  This entry point computes the same
// quantities as dao_k_dose (z = D x, grad F(z) and F(z)) without a context
// and without any allocation: the caller passes the inputs and outputs, and
// the only scratch memory, the per-block partial sums of F, lives in a
// file-scope device array that every GPU loading the library keeps until the
// process exits.
#include <mutex>

#include "dao_internal.h"

namespace {

constexpr int NA_ROWS_PER_BLOCK = 1024;  // voxel rows per block
constexpr int NA_MAX_BLOCKS = 4096;      // size of the scratch array
constexpr int NA_THREADS = 256;
constexpr int NA_LANES = 8;              // lanes per voxel row
constexpr int NA_MAX_DEVICES = 64;
constexpr int SMAX_TERMS = dao::SMAX;

// Per-block FP64 partial sums of the objective (32 KiB per device).
static __device__ __align__(256) double dao_noalloc_scratch[NA_MAX_BLOCKS];

struct NoallocTerms {
    double t[SMAX_TERMS][4];  // alpha_s / |v_s|, T_s^-, beta_s / |v_s|, T_s^+
};

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One block per NA_ROWS_PER_BLOCK rows; NA_LANES lanes per row with scalar
// loads of an unpadded CSR; the block's FP64 objective sum goes to partial[b].
__global__ void __launch_bounds__(NA_THREADS) k_dose_noalloc(int V, const int* __restrict__ rowptr,
                                                            const int* __restrict__ col,
                                                            const float* __restrict__ val,
                                                            const float* __restrict__ x,
                                                            const int* __restrict__ vstruct, int S,
                                                            const NoallocTerms terms, float* __restrict__ z,
                                                            float* __restrict__ grad, double* __restrict__ partial) {
    __shared__ double s_red[NA_THREADS / 32];
    const int lane = threadIdx.x & 31;
    const int sub = lane % NA_LANES;
    constexpr int RPW = 32 / NA_LANES;
    const int warp = threadIdx.x >> 5;
    const int r0 = blockIdx.x * NA_ROWS_PER_BLOCK;
    const int r1 = min(V, r0 + NA_ROWS_PER_BLOCK);
    double facc = 0.0;
    for (int base = r0 + warp * RPW; base < r1; base += (NA_THREADS / 32) * RPW) {
        const int row = base + lane / NA_LANES;
        float acc = 0.f;
        if (row < r1) {
            const int p1 = rowptr[row + 1];
            for (int p = rowptr[row] + sub; p < p1; p += NA_LANES) acc = fmaf(__ldg(val + p), __ldg(x + col[p]), acc);
        }
#pragma unroll
        for (int o = NA_LANES / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (row < r1 && sub == 0) {
            z[row] = acc;
            const int lab = vstruct[row];
            if ((unsigned)lab >= (unsigned)S) {  // no such structure: flagged, never read
                if (grad != nullptr) grad[row] = __int_as_float(0x7fc00000);
                facc += __longlong_as_double(0x7ff8000000000000ll);  // the objective becomes NaN
                continue;
            }
            const double* tt = terms.t[lab];
            const double zd = acc;
            const double u = fmax(0.0, tt[1] - zd);
            const double o = fmax(0.0, zd - tt[3]);
            if (grad != nullptr) grad[row] = (float)(2.0 * (tt[2] * o - tt[0] * u));
            facc += tt[0] * u * u + tt[2] * o * o;
        }
    }
    facc = na_warp_sum(facc);
    if (lane == 0) s_red[warp] = facc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < NA_THREADS / 32 ? s_red[threadIdx.x] : 0.0;
        t = na_warp_sum(t);
        if (threadIdx.x == 0) partial[blockIdx.x] = t;
    }
}

// Fixed-order sum of the n block partials into *out.
__global__ void __launch_bounds__(NA_THREADS) k_sum_noalloc(const double* __restrict__ partial, int n,
                                                           double* __restrict__ out) {
    __shared__ double s_red[NA_THREADS / 32];
    double v = 0.0;
    for (int i = threadIdx.x; i < n; i += NA_THREADS) v += partial[i];
    v = na_warp_sum(v);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < NA_THREADS / 32 ? s_red[threadIdx.x] : 0.0;
        t = na_warp_sum(t);
        if (threadIdx.x == 0) *out = t;
    }
}

std::mutex g_mu;
double* g_scratch_ptr[NA_MAX_DEVICES] = {};

dao_status na_fail(dao_status s, const std::string& m) { return dao::set_error(s, m); }

}  // namespace

extern "C" {

dao_status dao_dose_objective_noalloc(int32_t n_voxels, int32_t n_beamlets, const int32_t* row_ptr,
                                      const int32_t* col, const float* val, const float* x,
                                      const int32_t* voxel_struct, int32_t n_structures, const double* terms,
                                      float* z, float* grad, double* objective, void* stream) {
    if (n_voxels < 1 || n_beamlets < 1 || !row_ptr || !col || !val || !x || !voxel_struct || !terms || !z ||
        !objective)
        return na_fail(DAO_EINVAL, "null pointer or empty problem");
    const long long blocks = ((long long)n_voxels + NA_ROWS_PER_BLOCK - 1) / NA_ROWS_PER_BLOCK;
    if (blocks > NA_MAX_BLOCKS)
        return na_fail(DAO_EINVAL, "n_voxels exceeds the allocation-free limit of " +
                                       std::to_string((long long)NA_MAX_BLOCKS * NA_ROWS_PER_BLOCK) + " voxels");
    if (n_structures < 1 || n_structures > SMAX_TERMS)
        return na_fail(DAO_EINVAL, "n_structures must be in [1, " + std::to_string(SMAX_TERMS) + "]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(DAO_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return na_fail(DAO_EINVAL, "device ordinal out of range");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (st != nullptr) {  // the kernels run on the current device: the stream must belong to it
        int sdev = -1;
        e = cudaStreamGetDevice(st, &sdev);
        if (e != cudaSuccess) return na_fail(DAO_EINVAL, std::string("cudaStreamGetDevice: ") + cudaGetErrorString(e));
        if (sdev != dev)
            return na_fail(DAO_EINVAL, "the stream belongs to device " + std::to_string(sdev) +
                                           ", not to the current device " + std::to_string(dev));
    }
    double* scratch = nullptr;
    {
        // set-up, once per device with that device current: the device address of
        // the file-scope array (its name is only a host-side stand-in).  The
        // address belongs to the device's primary context as it was at that first
        // call; after a cudaDeviceReset it is stale, and a caller that resets the
        // device must not call this entry point again in the same process.
        std::lock_guard<std::mutex> lock(g_mu);
        if (g_scratch_ptr[dev] == nullptr) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, dao_noalloc_scratch);
            if (e != cudaSuccess)
                return na_fail(DAO_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    NoallocTerms t;
    for (int s = 0; s < SMAX_TERMS; ++s)
        for (int q = 0; q < 4; ++q) t.t[s][q] = s < n_structures ? terms[4 * s + q] : 0.0;
    k_dose_noalloc<<<(unsigned)blocks, NA_THREADS, 0, st>>>(n_voxels, row_ptr, col, val, x, voxel_struct,
                                                          n_structures, t, z, grad, scratch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(DAO_ECUDA, std::string("k_dose_noalloc: ") + cudaGetErrorString(e));
    k_sum_noalloc<<<1, NA_THREADS, 0, st>>>(scratch, (int)blocks, objective);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(DAO_ECUDA, std::string("k_sum_noalloc: ") + cudaGetErrorString(e));
    return DAO_OK;
}

}  // extern "C"
