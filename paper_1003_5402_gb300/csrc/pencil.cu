// The dose-deposition coefficients D_ij (arXiv:1003.5402, Eq. 2) generated on
// the device from a pencil-beam model, so that a re-plan needs no host-built D
// (the paper computes D with its own GPU pencil-beam engine, Sec. 1).
//
// Model, for beam b of B coplanar beams at gantry angle 2 pi b / B about z
// (direction e = (sin, -cos), lateral axis u = (cos, sin)), R x C beamlets of
// pitch w centred on the isocentre, and voxel j at p = xyz_j - iso:
//   D_ij = exp(-mu depth_j) * L(dv) * L(du),
//   depth_j = distance along e from the body's z-invariant cross-section (box or
//   elliptic cylinder) to the voxel, du / dv the voxel's offsets from the
//   beamlet's central axis, L the Gaussian profile exp(-d^2 / 2 sigma^2) or a
//   strip of width w blurred by that Gaussian; a coefficient is kept when it
//   exceeds 1e-12 and is at least cutoff times the beamlet's largest, then
//   multiplied by 1 + jitter (2 U - 1), U the SplitMix64 draw (Steele, Lea &
//   Flood 2014, used as a counter-based generator) of counter j N + i, and
//   rounded to FP32.
// The search range of a voxel is a window of rows and columns r0 - W .. r0 + W
// + 1 around the beamlet it projects into, W = ceil(sigma sqrt(2 ln 1e7) / w)
// + 1: outside it the lateral factor of the Gaussian profile is below 1e-7;
// inside, the 1e-12 floor and the cutoff decide.
// Every product and sum is rounded on its own (no fused multiply-add), so the
// coefficients equal a sequential FP64 evaluation of the same expressions up to
// the last bits of exp / erf.
//
// Three passes over (voxel, beam): the beamlets' maxima (atomic maximum on
// the bits of positive doubles, order independent), the kept entries per voxel
// row, and the entries themselves in column order (beam, row, column), which
// is the order the CSR needs; between the last two an exclusive scan of the
// row counts.
#include <cmath>

#include "dao_internal.h"

namespace dao {

namespace {

constexpr int PB_WMAX = 16;  // window entries per axis (2 W + 2)
constexpr int PB_T = 256;

struct PBParams {
    int V, B, R, C, N;
    double iso0, iso1, iso2;
    double w, sigma, mu, cutoff, jitter;
    int profile, body_kind;
    double bc0, bc1, bs0, bs1;
    unsigned long long stream;
    int win;
    double strip_norm;  // erf(w k / 2) of the strip profile
};

__device__ __forceinline__ double pb_lateral(const PBParams& q, double d) {
    if (q.profile == DAO_PB_GAUSS) {
        // exp(-(d * d) / (2 sigma sigma))
        const double num = -__dmul_rn(d, d);
        const double den = __dmul_rn(__dmul_rn(2.0, q.sigma), q.sigma);
        return exp(__ddiv_rn(num, den));
    }
    const double k = __ddiv_rn(1.0, __dmul_rn(sqrt(2.0), q.sigma));
    const double hw = __dmul_rn(0.5, q.w);
    const double a = erf(__dmul_rn(__dadd_rn(d, hw), k));
    const double b = erf(__dmul_rn(__dsub_rn(d, hw), k));
    return __ddiv_rn(__dmul_rn(0.5, __dsub_rn(a, b)), q.strip_norm);
}

// Smallest s with (px, py) + s (ex, ey) inside the body cross-section.
__device__ __forceinline__ double pb_entry(const PBParams& q, double px, double py, double ex, double ey) {
    const double qx = __dsub_rn(px, q.bc0), qy = __dsub_rn(py, q.bc1);
    if (q.body_kind == DAO_BODY_BOX) {
        double s = -INFINITY;
        if (fabs(ex) >= 1e-12) {
            const double t1 = __ddiv_rn(__dsub_rn(-q.bs0, qx), ex), t2 = __ddiv_rn(__dsub_rn(q.bs0, qx), ex);
            s = fmax(s, fmin(t1, t2));
        }
        if (fabs(ey) >= 1e-12) {
            const double t1 = __ddiv_rn(__dsub_rn(-q.bs1, qy), ey), t2 = __ddiv_rn(__dsub_rn(q.bs1, qy), ey);
            s = fmax(s, fmin(t1, t2));
        }
        return s;
    }
    const double a = q.bs0, b = q.bs1;
    const double ea = __ddiv_rn(ex, a), eb = __ddiv_rn(ey, b);
    const double A = __dadd_rn(__dmul_rn(ea, ea), __dmul_rn(eb, eb));
    const double Bq = __dmul_rn(2.0, __dadd_rn(__ddiv_rn(__dmul_rn(qx, ex), __dmul_rn(a, a)),
                                               __ddiv_rn(__dmul_rn(qy, ey), __dmul_rn(b, b))));
    const double qa = __ddiv_rn(qx, a), qb = __ddiv_rn(qy, b);
    const double Cq = __dsub_rn(__dadd_rn(__dmul_rn(qa, qa), __dmul_rn(qb, qb)), 1.0);
    const double disc = fmax(__dsub_rn(__dmul_rn(Bq, Bq), __dmul_rn(__dmul_rn(4.0, A), Cq)), 0.0);
    return __ddiv_rn(__dsub_rn(-Bq, sqrt(disc)), __dmul_rn(2.0, A));
}

// The window of voxel j in beam b: attenuation times the row factor for each
// window row (0 outside the grid), the column factor for each window column,
// and the first row / column of the window.
struct PBWindow {
    double av[PB_WMAX];  // exp(-mu depth) * L(dv) per window row
    double gu[PB_WMAX];  // L(du) per window column
    int r0, c0, n;
};

__device__ __forceinline__ void pb_window(const PBParams& q, const float* __restrict__ xyz, int j, int b,
                                          PBWindow& W) {
    const double th = __ddiv_rn(__dmul_rn(__dmul_rn(2.0, M_PI), (double)b), (double)q.B);
    const double ex = sin(th), ey = -cos(th);
    const double ux = cos(th), uy = sin(th);
    const double x0 = (double)xyz[3 * j], x1 = (double)xyz[3 * j + 1], x2 = (double)xyz[3 * j + 2];
    const double p0 = __dsub_rn(x0, q.iso0), p1 = __dsub_rn(x1, q.iso1), p2 = __dsub_rn(x2, q.iso2);
    const double u = __dadd_rn(__dmul_rn(p0, ux), __dmul_rn(p1, uy));
    const double v = p2;
    const double depth = fmax(-pb_entry(q, x0, x1, ex, ey), 0.0);
    const double att = exp(__dmul_rn(-q.mu, depth));
    const double cf = __dsub_rn(__dadd_rn(__ddiv_rn(u, q.w), __dmul_rn(0.5, (double)q.C)), 0.5);
    const double rf = __dsub_rn(__dadd_rn(__ddiv_rn(v, q.w), __dmul_rn(0.5, (double)q.R)), 0.5);
    W.c0 = (int)floor(cf) - q.win;
    W.r0 = (int)floor(rf) - q.win;
    W.n = 2 * q.win + 2;
    for (int k = 0; k < W.n; ++k) {
        const int r = W.r0 + k, c = W.c0 + k;
        W.av[k] = 0.0;
        W.gu[k] = 0.0;
        if (r >= 0 && r < q.R) {
            const double ctr = __dmul_rn(__dsub_rn(__dadd_rn((double)r, 0.5), __dmul_rn(0.5, (double)q.R)), q.w);
            W.av[k] = __dmul_rn(att, pb_lateral(q, __dsub_rn(v, ctr)));
        }
        if (c >= 0 && c < q.C) {
            const double ctr = __dmul_rn(__dsub_rn(__dadd_rn((double)c, 0.5), __dmul_rn(0.5, (double)q.C)), q.w);
            W.gu[k] = pb_lateral(q, __dsub_rn(u, ctr));
        }
    }
}

__global__ void __launch_bounds__(PB_T) k_pb_bmax(PBParams q, const float* __restrict__ xyz,
                                                  unsigned long long* __restrict__ bmax) {
    const long long t = (long long)blockIdx.x * PB_T + threadIdx.x;
    if (t >= (long long)q.V * q.B) return;
    const int j = (int)(t / q.B), b = (int)(t % q.B);
    PBWindow W;
    pb_window(q, xyz, j, b, W);
    for (int kr = 0; kr < W.n; ++kr) {
        if (W.av[kr] == 0.0) continue;
        for (int kc = 0; kc < W.n; ++kc) {
            const double val = __dmul_rn(W.av[kr], W.gu[kc]);
            if (val > 1e-12) {
                const int i = b * q.R * q.C + (W.r0 + kr) * q.C + (W.c0 + kc);
                atomicMax(bmax + i, (unsigned long long)__double_as_longlong(val));
            }
        }
    }
}

// pass 2 (write == false): kept entries of each voxel row; pass 3: the entries.
template <bool WRITE>
__global__ void __launch_bounds__(PB_T) k_pb_rows(PBParams q, const float* __restrict__ xyz,
                                                  const unsigned long long* __restrict__ bmax,
                                                  long long* __restrict__ cnt, const long long* __restrict__ rp,
                                                  int* __restrict__ col, float* __restrict__ val) {
    const int j = blockIdx.x * PB_T + threadIdx.x;
    if (j >= q.V) return;
    long long n = 0, p = WRITE ? rp[j] : 0;
    for (int b = 0; b < q.B; ++b) {
        PBWindow W;
        pb_window(q, xyz, j, b, W);
        for (int kr = 0; kr < W.n; ++kr) {
            if (W.av[kr] == 0.0) continue;
            for (int kc = 0; kc < W.n; ++kc) {
                const double v = __dmul_rn(W.av[kr], W.gu[kc]);
                if (!(v > 1e-12)) continue;
                const int i = b * q.R * q.C + (W.r0 + kr) * q.C + (W.c0 + kc);
                if (!(v >= __dmul_rn(q.cutoff, __longlong_as_double((long long)bmax[i])))) continue;
                if (WRITE) {
                    double x = v;
                    if (q.jitter > 0.0) {
                        // SplitMix64: mix(stream + (counter + 1) * gamma), top 53 bits
                        unsigned long long z = q.stream + ((unsigned long long)j * (unsigned long long)q.N +
                                                           (unsigned long long)i + 1ull) * 0x9E3779B97F4A7C15ull;
                        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                        z = z ^ (z >> 31);
                        const double uu = __dmul_rn((double)(z >> 11), 1.0 / 9007199254740992.0);
                        x = __dmul_rn(v, __dadd_rn(1.0, __dmul_rn(q.jitter, __dsub_rn(__dmul_rn(2.0, uu), 1.0))));
                    }
                    col[p] = i;
                    val[p] = __double2float_rn(x);
                    ++p;
                } else {
                    ++n;
                }
            }
        }
    }
    if (!WRITE) cnt[j] = n;
}

// Exclusive scan of V int64 counts in three launches (block totals, their scan
// in one block, the blocks' prefixes); the total goes to rp[V].
constexpr int PS_T = 1024;
__device__ __forceinline__ long long pb_block_exscan(long long v, long long* s_w, long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long t = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        s_w[lane] = t;
    }
    __syncthreads();
    const long long before = wid > 0 ? s_w[wid - 1] : 0;
    *total = s_w[31];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(PS_T) k_pb_scan_totals(const long long* __restrict__ cnt, int V,
                                                         long long* __restrict__ bsum) {
    __shared__ long long s_w[32];
    const int i = blockIdx.x * PS_T + threadIdx.x;
    long long tot;
    pb_block_exscan(i < V ? cnt[i] : 0, s_w, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(PS_T) k_pb_scan_blocks(long long* __restrict__ bsum, int nb,
                                                         long long* __restrict__ rpV) {
    __shared__ long long s_w[32];
    long long carry = 0;
    for (int b0 = 0; b0 < nb; b0 += PS_T) {
        const int b = b0 + threadIdx.x;
        long long tot;
        const long long ex = pb_block_exscan(b < nb ? bsum[b] : 0, s_w, &tot);
        if (b < nb) bsum[b] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *rpV = carry;
}

__global__ void __launch_bounds__(PS_T) k_pb_scan_apply(const long long* __restrict__ cnt, int V,
                                                        const long long* __restrict__ bsum,
                                                        long long* __restrict__ rp) {
    __shared__ long long s_w[32];
    const int i = blockIdx.x * PS_T + threadIdx.x;
    long long tot;
    const long long ex = pb_block_exscan(i < V ? cnt[i] : 0, s_w, &tot);
    if (i < V) rp[i] = bsum[blockIdx.x] + ex;
}

}  // namespace

dao_status pencil_check(const dao_pencil_beam* pb) {
    if (!pb) return set_error(DAO_EINVAL, "null pencil-beam description");
    if (pb->n_voxels < 1 || !pb->voxel_xyz) return set_error(DAO_EINVAL, "pencil beam: need voxels and coordinates");
    if (pb->n_beams < 1 || pb->rows < 1 || pb->cols < 1 || pb->cols > CMAX)
        return set_error(DAO_EINVAL, "pencil beam: n_beams >= 1, rows >= 1, 1 <= cols <= 32");
    if ((int64_t)pb->n_beams * pb->rows * pb->cols > (1 << 30))
        return set_error(DAO_EINVAL, "pencil beam: too many beamlets");
    if (!(pb->beamlet_mm > 0) || !(pb->sigma_mm > 0) || !(pb->mu_per_mm >= 0) || !(pb->cutoff >= 0) ||
        !(pb->cutoff < 1) || !(pb->jitter >= 0) || !(pb->jitter < 1) || !std::isfinite(pb->beamlet_mm) ||
        !std::isfinite(pb->sigma_mm) || !std::isfinite(pb->mu_per_mm))
        return set_error(DAO_EINVAL, "pencil beam: pitch, sigma > 0, mu >= 0, cutoff and jitter in [0, 1)");
    if (pb->profile != DAO_PB_GAUSS && pb->profile != DAO_PB_STRIP)
        return set_error(DAO_EINVAL, "pencil beam: profile must be DAO_PB_GAUSS or DAO_PB_STRIP");
    if (pb->body_kind != DAO_BODY_BOX && pb->body_kind != DAO_BODY_ECYL)
        return set_error(DAO_EINVAL, "pencil beam: body must be DAO_BODY_BOX or DAO_BODY_ECYL");
    if (!(pb->body_size[0] > 0) || !(pb->body_size[1] > 0))
        return set_error(DAO_EINVAL, "pencil beam: body sizes must be positive");
    const double reach = pb->sigma_mm * std::sqrt(2.0 * std::log(1e7));
    const int win = (int)std::ceil(reach / pb->beamlet_mm) + 1;
    if (2 * win + 2 > PB_WMAX)
        return set_error(DAO_EINVAL, "pencil beam: sigma too wide for the pitch (window above 16 beamlets)");
    return DAO_OK;
}

cudaError_t pencil_generate(const dao_pencil_beam* pb, int device, cudaStream_t s, int64_t** rp_out, int** col_out,
                            float** val_out, int64_t* nnz_out) {
    PBParams q{};
    q.V = pb->n_voxels;
    q.B = pb->n_beams;
    q.R = pb->rows;
    q.C = pb->cols;
    q.N = q.B * q.R * q.C;
    q.iso0 = pb->iso[0];
    q.iso1 = pb->iso[1];
    q.iso2 = pb->iso[2];
    q.w = pb->beamlet_mm;
    q.sigma = pb->sigma_mm;
    q.mu = pb->mu_per_mm;
    q.cutoff = pb->cutoff;
    q.jitter = pb->jitter;
    q.profile = pb->profile;
    q.body_kind = pb->body_kind;
    q.bc0 = pb->body_center[0];
    q.bc1 = pb->body_center[1];
    q.bs0 = pb->body_size[0];
    q.bs1 = pb->body_size[1];
    q.stream = (unsigned long long)pb->jitter_stream;
    q.win = (int)std::ceil(q.sigma * std::sqrt(2.0 * std::log(1e7)) / q.w) + 1;
    q.strip_norm = std::erf(0.5 * q.w * (1.0 / (std::sqrt(2.0) * q.sigma)));
    *rp_out = nullptr;
    *col_out = nullptr;
    *val_out = nullptr;
    float* xyz = nullptr;
    unsigned long long* bmax = nullptr;
    long long* cnt = nullptr;
    long long* bsum = nullptr;
    long long* rp = nullptr;
    const int nb = (q.V + PS_T - 1) / PS_T;
    auto release = [&]() {
        for (void* p : {(void*)xyz, (void*)bmax, (void*)cnt, (void*)bsum})
            if (p) pool_free(p, s);
    };
    cudaError_t e = pool_alloc((void**)&xyz, sizeof(float) * 3 * (size_t)q.V, device, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&bmax, sizeof(unsigned long long) * (size_t)q.N, device, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&cnt, sizeof(long long) * (size_t)q.V, device, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&bsum, sizeof(long long) * (size_t)nb, device, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&rp, sizeof(long long) * ((size_t)q.V + 1), device, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(xyz, pb->voxel_xyz, sizeof(float) * 3 * (size_t)q.V, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bmax, 0, sizeof(unsigned long long) * (size_t)q.N, s);
    if (e == cudaSuccess) {
        const long long pairs = (long long)q.V * q.B;
        k_pb_bmax<<<(unsigned)((pairs + PB_T - 1) / PB_T), PB_T, 0, s>>>(q, xyz, bmax);
        k_pb_rows<false><<<(q.V + PB_T - 1) / PB_T, PB_T, 0, s>>>(q, xyz, bmax, cnt, nullptr, nullptr, nullptr);
        k_pb_scan_totals<<<nb, PS_T, 0, s>>>(cnt, q.V, bsum);
        k_pb_scan_blocks<<<1, PS_T, 0, s>>>(bsum, nb, rp + q.V);
        k_pb_scan_apply<<<nb, PS_T, 0, s>>>(cnt, q.V, bsum, rp);
        e = cudaGetLastError();
    }
    long long nnz = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nnz, rp + q.V, sizeof(long long), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int* col = nullptr;
    float* val = nullptr;
    if (e == cudaSuccess) e = pool_alloc((void**)&col, sizeof(int) * (size_t)std::max(nnz, 1ll), device, s);
    if (e == cudaSuccess) e = pool_alloc((void**)&val, sizeof(float) * (size_t)std::max(nnz, 1ll), device, s);
    if (e == cudaSuccess) {
        k_pb_rows<true><<<(q.V + PB_T - 1) / PB_T, PB_T, 0, s>>>(q, xyz, bmax, nullptr, rp, col, val);
        e = cudaGetLastError();
    }
    release();
    if (e != cudaSuccess) {
        for (void* p : {(void*)rp, (void*)col, (void*)val})
            if (p) pool_free(p, s);
        return e;
    }
    *rp_out = reinterpret_cast<int64_t*>(rp);
    *col_out = col;
    *val_out = val;
    *nnz_out = nnz;
    return cudaSuccess;
}

}  // namespace dao
