// indexing.cu -- step (a6): the look-up table and Eq. 3 matching, and step
// (a7): Gauss-Newton orientation refinement on a bilinear elevation-azimuth
// reference image, with forward and backward kernels for automatic
// differentiation.
//
// Supplement "Indexing algorithm": the reference signature of a candidate is
// normalised, its n_hat strongest nodes are kept, every test orientation g
// rotates them, and the look-up table holds the measured-image node nearest
// to each rotated reference node; Eq. 3 scores g by the sum of squared
// differences of the image values there.  Rotations map crystal to lab.
#include <math.h>

#include "common.cuh"

namespace aptidx {

namespace {

// ---- rotations (FP64, fixed operation order, no contraction) ----------------

struct M3 {
    double a[9];
};

__device__ __forceinline__ M3 quat_to_matrix(double w, double x, double y, double z) {
    const double xx = __dmul_rn(x, x), yy = __dmul_rn(y, y), zz = __dmul_rn(z, z);
    const double xy = __dmul_rn(x, y), xz = __dmul_rn(x, z), yz = __dmul_rn(y, z);
    const double wx = __dmul_rn(w, x), wy = __dmul_rn(w, y), wz = __dmul_rn(w, z);
    M3 m;
    m.a[0] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(yy, zz)));
    m.a[1] = __dmul_rn(2.0, __dsub_rn(xy, wz));
    m.a[2] = __dmul_rn(2.0, __dadd_rn(xz, wy));
    m.a[3] = __dmul_rn(2.0, __dadd_rn(xy, wz));
    m.a[4] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, zz)));
    m.a[5] = __dmul_rn(2.0, __dsub_rn(yz, wx));
    m.a[6] = __dmul_rn(2.0, __dsub_rn(xz, wy));
    m.a[7] = __dmul_rn(2.0, __dadd_rn(yz, wx));
    m.a[8] = __dsub_rn(1.0, __dmul_rn(2.0, __dadd_rn(xx, yy)));
    return m;
}

__device__ __forceinline__ void quat_mul(const double* a, const double* b, double* o) {
    const double r0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    const double r1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    const double r2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    const double r3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = r0;
    o[1] = r1;
    o[2] = r2;
    o[3] = r3;
}

__device__ __forceinline__ void exp_quat(const double* d, double* q) {
    const double th = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (th < 1e-300) {
        q[0] = 1.0;
        q[1] = q[2] = q[3] = 0.0;
        return;
    }
    const double s = sin(0.5 * th) / th;
    q[0] = cos(0.5 * th);
    q[1] = s * d[0];
    q[2] = s * d[1];
    q[3] = s * d[2];
}

// ---- strongest reference nodes (bitonic sort of packed keys, one block) -----

__device__ __forceinline__ uint32_t ordered_f32(float f) {
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// key = (descending value, ascending index); padding sorts last
__global__ void __launch_bounds__(1024) k_top_nodes(const float* __restrict__ sig, int32_t nv, int32_t npow2,
                                                    uint64_t* keys, int32_t n_hat, int32_t* top, float* top_val) {
    for (int i = threadIdx.x; i < npow2; i += blockDim.x)
        keys[i] = i < nv ? ((uint64_t)(~ordered_f32(sig[i])) << 32) | (uint32_t)i : ~0ull;
    __syncthreads();
    for (int k = 2; k <= npow2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < npow2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const uint64_t a = keys[i], b = keys[l];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        keys[i] = b;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n_hat; i += blockDim.x) {
        const int32_t idx = (int32_t)(keys[i] & 0xFFFFFFFFu);
        top[i] = idx;
        top_val[i] = sig[idx];
    }
}

// ---- look-up table ---------------------------------------------------------------

constexpr int kLutThreads = 256;
constexpr int kLutPer = 4;                       // queries per thread
constexpr int kLutTile = 2048;                   // nodes per shared-memory tile

// lut_t[k * ng_pad + g] = argmax_p u_p . r with r = (float)(R(q_g) n_top[k])
// (FP64 products summed left to right), the dot product by the FP32 contract
// fma(u_z, r_z, fma(u_y, r_y, u_x r_x)); ties resolve to the lowest index.
// IdxT is uint16_t when every node index fits (nv <= 65536), else int32_t.
template <typename IdxT>
__global__ void __launch_bounds__(kLutThreads) k_build_lut(const float4* __restrict__ dirs, int32_t nv,
                                                           const int32_t* __restrict__ top, int32_t n_hat,
                                                           const double* __restrict__ quats, int64_t ng,
                                                           int64_t ng_pad, IdxT* lut_t) {
    __shared__ float4 tile[kLutTile];
    const int64_t nq = ng * n_hat;
    const int64_t q0 = (int64_t)blockIdx.x * kLutThreads * kLutPer;
    float rx[kLutPer], ry[kLutPer], rz[kLutPer], best[kLutPer];
    int32_t bi[kLutPer];
    int64_t qi[kLutPer];
#pragma unroll
    for (int j = 0; j < kLutPer; ++j) {
        const int64_t q = q0 + (int64_t)j * kLutThreads + threadIdx.x;
        qi[j] = q;
        best[j] = -INFINITY;
        bi[j] = 0;
        rx[j] = ry[j] = rz[j] = 0.f;
        if (q < nq) {
            const int64_t g = q / n_hat;
            const int k = (int)(q % n_hat);
            const M3 R = quat_to_matrix(quats[4 * g], quats[4 * g + 1], quats[4 * g + 2], quats[4 * g + 3]);
            const float4 n = dirs[top[k]];
            const double nx = n.x, ny = n.y, nz = n.z;
            rx[j] = __double2float_rn(__dadd_rn(__dadd_rn(__dmul_rn(R.a[0], nx), __dmul_rn(R.a[1], ny)), __dmul_rn(R.a[2], nz)));
            ry[j] = __double2float_rn(__dadd_rn(__dadd_rn(__dmul_rn(R.a[3], nx), __dmul_rn(R.a[4], ny)), __dmul_rn(R.a[5], nz)));
            rz[j] = __double2float_rn(__dadd_rn(__dadd_rn(__dmul_rn(R.a[6], nx), __dmul_rn(R.a[7], ny)), __dmul_rn(R.a[8], nz)));
        }
    }
    for (int p0 = 0; p0 < nv; p0 += kLutTile) {
        const int cnt = min(kLutTile, nv - p0);
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kLutThreads) tile[i] = dirs[p0 + i];
        __syncthreads();
        for (int i = 0; i < cnt; ++i) {
            const float4 u = tile[i];
#pragma unroll
            for (int j = 0; j < kLutPer; ++j) {
                const float d = __fmaf_rn(u.z, rz[j], __fmaf_rn(u.y, ry[j], __fmul_rn(u.x, rx[j])));
                if (d > best[j]) {
                    best[j] = d;
                    bi[j] = p0 + i;
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kLutPer; ++j) {
        const int64_t q = qi[j];
        if (q < nq) {
            const int64_t g = q / n_hat;
            const int k = (int)(q % n_hat);
            lut_t[(int64_t)k * ng_pad + g] = (IdxT)bi[j];
        }
    }
}

// ---- Eq. 3 -----------------------------------------------------------------------

// One CTA per ROI (persistent): the ROI's signature row in shared memory,
// Delta(g) = sum_k (S[lut[k, g]] - ref[k])^2 accumulated in FP32 in k order,
// argmin with ties to the lowest g.  The table streams from L2 once per ROI:
// each thread reads 16 bytes of a table row per k (G = 16 / sizeof(IdxT)
// consecutive orientations) and keeps kMatchDepth rows in flight.
constexpr int kMatchDepth = 8;   // table rows in flight per thread

template <typename IdxT>
__device__ __forceinline__ uint4 lut_load(const IdxT* p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

template <typename IdxT>
__device__ __forceinline__ void lut_accumulate(const uint4 w, const float* row, float rk, float* acc) {
    if (sizeof(IdxT) == 2) {
        const float d0 = row[w.x & 0xFFFFu] - rk, d1 = row[w.x >> 16] - rk;
        const float d2 = row[w.y & 0xFFFFu] - rk, d3 = row[w.y >> 16] - rk;
        const float d4 = row[w.z & 0xFFFFu] - rk, d5 = row[w.z >> 16] - rk;
        const float d6 = row[w.w & 0xFFFFu] - rk, d7 = row[w.w >> 16] - rk;
        acc[0] = fmaf(d0, d0, acc[0]);
        acc[1] = fmaf(d1, d1, acc[1]);
        acc[2] = fmaf(d2, d2, acc[2]);
        acc[3] = fmaf(d3, d3, acc[3]);
        acc[4] = fmaf(d4, d4, acc[4]);
        acc[5] = fmaf(d5, d5, acc[5]);
        acc[6] = fmaf(d6, d6, acc[6]);
        acc[7] = fmaf(d7, d7, acc[7]);
    } else {
        const float d0 = row[w.x] - rk, d1 = row[w.y] - rk, d2 = row[w.z] - rk, d3 = row[w.w] - rk;
        acc[0] = fmaf(d0, d0, acc[0]);
        acc[1] = fmaf(d1, d1, acc[1]);
        acc[2] = fmaf(d2, d2, acc[2]);
        acc[3] = fmaf(d3, d3, acc[3]);
    }
}

// With scores_out, weight x Delta(g) of ROI r also goes to scores_out[r * ng
// + g] (accumulate: added to the value there, for sums over signature
// channels).
template <typename IdxT>
__global__ void __launch_bounds__(1024, 1) k_match(const float* __restrict__ S, int64_t nroi, int32_t nv,
                                                const IdxT* __restrict__ lut_t, int64_t ng, int64_t ng_pad,
                                                const float* __restrict__ top_val, int32_t n_hat, int32_t* best,
                                                float* score, float* scores_out, bool accumulate, float weight) {
    constexpr int G = 16 / (int)sizeof(IdxT);
    extern __shared__ float sm[];
    float* row = sm;                     // nv
    float* ref = sm + nv;                // n_hat
    __shared__ float red_v[32];
    __shared__ int32_t red_g[32];
    const int nwarps = blockDim.x >> 5;
    for (int i = threadIdx.x; i < n_hat; i += blockDim.x) ref[i] = top_val[i];
    for (int64_t r = blockIdx.x; r < nroi; r += gridDim.x) {
        __syncthreads();
        const float* src = S + r * (int64_t)nv;
        for (int i = threadIdx.x; i < nv; i += blockDim.x) row[i] = src[i];
        __syncthreads();
        float bv = INFINITY;
        int32_t bg = 0x7FFFFFFF;
        for (int64_t g0 = (int64_t)threadIdx.x * G; g0 < ng; g0 += (int64_t)blockDim.x * G) {
            float acc[G];
#pragma unroll
            for (int e = 0; e < G; ++e) acc[e] = 0.f;
            const IdxT* lp = lut_t + g0;
            int k = 0;
            for (; k + kMatchDepth <= n_hat; k += kMatchDepth) {
                uint4 w[kMatchDepth];
#pragma unroll
                for (int j = 0; j < kMatchDepth; ++j) w[j] = lut_load(lp + (int64_t)(k + j) * ng_pad);
#pragma unroll
                for (int j = 0; j < kMatchDepth; ++j) lut_accumulate<IdxT>(w[j], row, ref[k + j], acc);
            }
            for (; k < n_hat; ++k) lut_accumulate<IdxT>(lut_load(lp + (int64_t)k * ng_pad), row, ref[k], acc);
#pragma unroll
            for (int e = 0; e < G; ++e)
                if (g0 + e < ng && acc[e] < bv) {
                    bv = acc[e];
                    bg = (int32_t)(g0 + e);
                }
            if (scores_out) {
#pragma unroll
                for (int e = 0; e < G; ++e)
                    if (g0 + e < ng) {
                        float* o = scores_out + r * ng + g0 + e;
                        *o = accumulate ? fmaf(weight, acc[e], *o) : weight * acc[e];
                    }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int32_t og = __shfl_xor_sync(0xffffffffu, bg, o);
            if (ov < bv || (ov == bv && og < bg)) {
                bv = ov;
                bg = og;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            red_v[threadIdx.x >> 5] = bv;
            red_g[threadIdx.x >> 5] = bg;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < nwarps; ++w)
                if (red_v[w] < bv || (red_v[w] == bv && red_g[w] < bg)) {
                    bv = red_v[w];
                    bg = red_g[w];
                }
            if (best) best[r] = bg;
            if (score) score[r] = bv;
        }
    }
}

// ---- the topk smallest Delta(g) of a ROI (ties: lower g), ascending ----------
// One CTA per ROI: radix select of the topk-th smallest key (Delta >= 0, so
// its FP32 bit pattern orders like the value) over four 8-bit digits, then
// every g below that key plus the lowest-g ones equal to it, then a bitonic
// sort of the (key, g) pairs.
constexpr int kTopkThreads = 256;

__global__ void __launch_bounds__(kTopkThreads) k_topk(const float* __restrict__ scores, int64_t ng, int64_t nroi,
                                                       int32_t topk, int32_t* best, float* score) {
    __shared__ uint32_t hist[256];
    __shared__ uint64_t sel[APTIDX_MAX_TOPK];
    __shared__ uint32_t s_prefix, s_remaining, s_count;
    __shared__ uint32_t warp_cnt[kTopkThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int kp = 1;
    while (kp < topk) kp <<= 1;
    for (int64_t r = blockIdx.x; r < nroi; r += gridDim.x) {
        const uint32_t* key = reinterpret_cast<const uint32_t*>(scores + r * ng);
        if (tid == 0) {
            s_prefix = 0;
            s_remaining = (uint32_t)topk;
        }
        // 1. radix select: the topk-th smallest key
        for (int pass = 3; pass >= 0; --pass) {
            for (int i = tid; i < 256; i += kTopkThreads) hist[i] = 0;
            __syncthreads();
            const uint32_t prefix = s_prefix;
            const uint32_t hmask = pass == 3 ? 0u : (0xFFFFFFFFu << (8 * (pass + 1)));
            for (int64_t g = tid; g < ng; g += kTopkThreads) {
                const uint32_t k = key[g];
                if ((k & hmask) == (prefix & hmask)) atomicAdd(&hist[(k >> (8 * pass)) & 255u], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t rem = s_remaining, d = 0;
                while (hist[d] < rem) {
                    rem -= hist[d];
                    ++d;
                }
                s_remaining = rem;
                s_prefix = prefix | (d << (8 * pass));
            }
            __syncthreads();
        }
        const uint32_t kth = s_prefix;
        const uint32_t need_eq = s_remaining;   // how many keys equal to kth are kept
        const uint32_t n_less = (uint32_t)topk - need_eq;
        // 2. every key below kth (any order), then the lowest-g keys equal to it
        if (tid == 0) s_count = 0;
        for (int i = tid; i < kp; i += kTopkThreads) sel[i] = ~0ull;
        __syncthreads();
        for (int64_t g = tid; g < ng; g += kTopkThreads) {
            const uint32_t k = key[g];
            if (k < kth) sel[atomicAdd(&s_count, 1u)] = ((uint64_t)k << 32) | (uint32_t)g;
        }
        __syncthreads();
        uint32_t taken = 0;
        for (int64_t g0 = 0; g0 < ng && taken < need_eq; g0 += kTopkThreads) {
            const int64_t g = g0 + tid;
            const bool eq = g < ng && key[g] == kth;
            const uint32_t bal = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) warp_cnt[warp] = __popc(bal);
            __syncthreads();
            uint32_t before = 0, total = 0;
            for (int w = 0; w < kTopkThreads / 32; ++w) {
                if (w < warp) before += warp_cnt[w];
                total += warp_cnt[w];
            }
            const uint32_t rank = taken + before + __popc(bal & ((1u << lane) - 1u));
            if (eq && rank < need_eq) sel[n_less + rank] = ((uint64_t)kth << 32) | (uint32_t)g;
            taken += total;
            __syncthreads();
        }
        __syncthreads();
        // 3. bitonic sort of the kp slots (unused slots hold ~0)
        for (int size = 2; size <= kp; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < kp; i += kTopkThreads) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const bool up = (i & size) == 0;
                        const uint64_t a = sel[i], b = sel[j];
                        if ((a > b) == up) {
                            sel[i] = b;
                            sel[j] = a;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i < topk; i += kTopkThreads) {
            const uint64_t v = sel[i];
            if (best) best[r * topk + i] = (int32_t)(uint32_t)v;
            if (score) score[r * topk + i] = __uint_as_float((uint32_t)(v >> 32));
        }
        __syncthreads();
    }
}

// ---- refinement ----------------------------------------------------------------------

constexpr int kRefThreads = 256;
constexpr float kPoleDeg = 89.0f;
constexpr float kRad2Deg = 57.295779513082320876f;

// atan(t) for t in [0, 1] as t * P(t^2), P of degree 7 with coefficients that
// minimise the maximum error on [0, 1] (Lawson's iteratively reweighted least
// squares; atan_fit.py regenerates them): |error| < 4e-8 rad in exact
// arithmetic, < 2e-7 rad with FP32 Horner steps.
__device__ __forceinline__ float atan01(float t) {
    const float s = t * t;
    float p = -4.054556496e-03f;
    p = fmaf(p, s, 2.186292078e-02f);
    p = fmaf(p, s, -5.591227578e-02f);
    p = fmaf(p, s, 9.642193788e-02f);
    p = fmaf(p, s, -1.390862825e-01f);
    p = fmaf(p, s, 1.994656541e-01f);
    p = fmaf(p, s, -3.332986076e-01f);
    p = fmaf(p, s, 9.999993356e-01f);
    return t * p;
}

// atan2(y, x) in degrees, (-180, 180]: octant reduction to atan01 of
// min(|x|, |y|) / max(|x|, |y|) (a 2-ulp quotient).  NaN when x = y = 0.
__device__ __forceinline__ float atan2_deg(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    float a = atan01(__fdividef(fminf(ax, ay), fmaxf(ax, ay)));
    if (ay > ax) a = 1.57079632679489662f - a;
    if (x < 0.f) a = 3.14159265358979324f - a;
    if (y < 0.f) a = -a;
    return a * kRad2Deg;
}

struct DirTerm {
    bool ok;
    float r;       // residual S - I
    float J[3];    // d r / d delta
};

// residual and its derivative with respect to the lab-frame perturbation delta
// of R = exp([delta]x) R(q) for one direction: c = R^T u, (alpha, beta) of c,
// bilinear sample of the image, r = s - I, J = -(R grad_c I) x u
// = -R (grad_c I x c); kCrystalJ returns grad_c I x c instead.
template <bool kCrystalJ = false>
__device__ __forceinline__ DirTerm dir_term(const float* Rf, float ux, float uy, float uz, float s,
                                            const float4* __restrict__ img4, bool want_j) {
    DirTerm t;
    const float cx = Rf[0] * ux + Rf[3] * uy + Rf[6] * uz;
    const float cy = Rf[1] * ux + Rf[4] * uy + Rf[7] * uz;
    const float cz = Rf[2] * ux + Rf[5] * uy + Rf[8] * uz;
    const float rho2 = cx * cx + cy * cy;
    const float inv_rho = rsqrtf(rho2);
    const float rho = rho2 * inv_rho;
    const float alpha = atan2_deg(cz, rho);
    t.ok = fabsf(alpha) <= kPoleDeg;   // also false for NaN at the exact poles
    if (!t.ok) return t;
    float beta = atan2_deg(cy, cx);
    if (beta < 0.f) beta += 360.f;
    const float fi = alpha + 90.f;
    int i0 = (int)floorf(fi);
    i0 = min(max(i0, 0), kImgRows - 2);
    const float fj0 = floorf(beta);
    const float ti = fi - (float)i0;
    const float tj = beta - fj0;
    int j0 = (int)fj0;
    j0 = j0 >= kImgCols ? j0 - kImgCols : j0;
    j0 = min(max(j0, 0), kImgCols - 1);
    // the cell's four taps (I[i0][j0], I[i0][j0 + 1], I[i0 + 1][j0], I[i0 + 1][j0 + 1],
    // the column index mod 360) in one read
    const float4 cell = __ldg(img4 + i0 * kImgCols + j0);
    const float I00 = cell.x, I01 = cell.y, I10 = cell.z, I11 = cell.w;
    const float v = (1.f - ti) * ((1.f - tj) * I00 + tj * I01) + ti * ((1.f - tj) * I10 + tj * I11);
    t.r = s - v;
    if (want_j) {
        const float dfi = (1.f - tj) * (I10 - I00) + tj * (I11 - I01);
        const float dfj = (1.f - ti) * (I01 - I00) + ti * (I11 - I10);
        // partial derivatives of (alpha, beta) in radians; the 2-ulp
        // reciprocals are far inside the FP32 error of the sums they feed
        const float n2 = rho2 + cz * cz;
        const float inv_n2 = __fdividef(1.f, n2);
        const float inv_rho2 = inv_rho * inv_rho;
        const float t_a = -cz * inv_n2 * inv_rho;
        const float da0 = t_a * cx, da1 = t_a * cy, da2 = rho * inv_n2;
        const float db0 = -cy * inv_rho2, db1 = cx * inv_rho2;
        const float g0 = kRad2Deg * (dfi * da0 + dfj * db0);
        const float g1 = kRad2Deg * (dfi * da1 + dfj * db1);
        const float g2 = kRad2Deg * (dfi * da2);
        if (kCrystalJ) {
            // J = -R (g x c): keep g x c; the caller rotates the sums once
            t.J[0] = g1 * cz - g2 * cy;
            t.J[1] = g2 * cx - g0 * cz;
            t.J[2] = g0 * cy - g1 * cx;
        } else {
            const float ax = Rf[0] * g0 + Rf[1] * g1 + Rf[2] * g2;
            const float ay = Rf[3] * g0 + Rf[4] * g1 + Rf[5] * g2;
            const float az = Rf[6] * g0 + Rf[7] * g1 + Rf[8] * g2;
            t.J[0] = -(ay * uz - az * uy);
            t.J[1] = -(az * ux - ax * uz);
            t.J[2] = -(ax * uy - ay * ux);
        }
    }
    return t;
}

// direction and signature reads stream past L1 so that L1 holds the reference
// image cells (180 x 360 x 16 B, reused by neighbouring directions and ROIs)
// for the bilinear gathers
__device__ __forceinline__ float4 ld_stream4(const float4* p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

__device__ __forceinline__ float ld_stream(const float* p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// coherent read that skips L1 (for data this kernel writes)
__device__ __forceinline__ float ld_l2(const float* p) {
    float v;
    asm volatile("ld.global.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}

// block sum of n FP32 partials per thread into FP64 totals (thread 0 holds them)
template <int N>
__device__ __forceinline__ void block_sum(float* v, double* out, double* scratch /* [N * 32] */) {
    double d[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        d[i] = (double)v[i];
        for (int o = 16; o > 0; o >>= 1) d[i] += __shfl_xor_sync(0xffffffffu, d[i], o);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) scratch[i * 32 + w] = d[i];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) {
            double s = 0.0;
            for (int k = 0; k < nw; ++k) s += scratch[i * 32 + k];
            out[i] = s;
        }
}

// Current rotation of ROI r: q = exp(omega) (x) q0 when omega is given.
__device__ __forceinline__ void roi_quat(const double* q0, const double* omega, int64_t r, double* q) {
    const double* a = q0 + 4 * r;
    if (omega) {
        double e[4];
        exp_quat(omega + 3 * r, e);
        quat_mul(e, a, q);
    } else {
        q[0] = a[0];
        q[1] = a[1];
        q[2] = a[2];
        q[3] = a[3];
    }
    const double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) q[i] /= n;
}

__device__ __forceinline__ void matrix_f32(const double* q, float* Rf) {
    const M3 R = quat_to_matrix(q[0], q[1], q[2], q[3]);
    for (int i = 0; i < 9; ++i) Rf[i] = (float)R.a[i];
}

// Forward (loss) and backward (gradient) of L = sum_v (S_v - I(R^T u_v))^2.
// With omega, the gradient is with respect to omega (rotation exp([omega]x)
// R(q0)): dL/domega = J_l(omega)^T dL/ddelta, J_l the left Jacobian of SO(3).
template <bool kGrad>
__global__ void __launch_bounds__(kRefThreads) k_refine_eval(const float* __restrict__ S, const float4* __restrict__ dirs,
                                                             int32_t nv, const float4* __restrict__ img,
                                                             const double* __restrict__ q0, const double* __restrict__ omega,
                                                             int64_t nroi, float* loss, float* grad) {
    __shared__ double scratch[4 * 32];
    __shared__ double tot[4];
    __shared__ float Rs[9];
    for (int64_t r = blockIdx.x; r < nroi; r += gridDim.x) {
        if (threadIdx.x == 0) {
            double q[4];
            roi_quat(q0, omega, r, q);
            matrix_f32(q, Rs);
        }
        __syncthreads();
        float Rf[9];
        for (int i = 0; i < 9; ++i) Rf[i] = Rs[i];
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const float* srow = S + r * (int64_t)nv;
        for (int v = threadIdx.x; v < nv; v += kRefThreads) {
            const float4 u = ld_stream4(dirs + v);
            const DirTerm t = dir_term(Rf, u.x, u.y, u.z, ld_stream(srow + v), img, kGrad);
            if (!t.ok) continue;
            acc[0] = fmaf(t.r, t.r, acc[0]);
            if (kGrad) {
                acc[1] = fmaf(2.f * t.r, t.J[0], acc[1]);
                acc[2] = fmaf(2.f * t.r, t.J[1], acc[2]);
                acc[3] = fmaf(2.f * t.r, t.J[2], acc[3]);
            }
        }
        block_sum<4>(acc, tot, scratch);
        if (threadIdx.x == 0) {
            if (loss) loss[r] = (float)tot[0];
            if (kGrad && grad) {
                double g[3] = {tot[1], tot[2], tot[3]};
                if (omega) {
                    // g_omega = J_l(omega)^T g_delta
                    const double* w = omega + 3 * r;
                    const double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                    const double th = sqrt(th2);
                    double A, B;
                    if (th < 1e-4) {
                        A = 0.5 - th2 / 24.0;
                        B = 1.0 / 6.0 - th2 / 120.0;
                    } else {
                        A = (1.0 - cos(th)) / th2;
                        B = (th - sin(th)) / (th2 * th);
                    }
                    // J_l = I + A [w]x + B [w]x^2;  J_l^T g = g - A (w x g) + B (w x (w x g))
                    const double c1[3] = {w[1] * g[2] - w[2] * g[1], w[2] * g[0] - w[0] * g[2], w[0] * g[1] - w[1] * g[0]};
                    const double c2[3] = {w[1] * c1[2] - w[2] * c1[1], w[2] * c1[0] - w[0] * c1[2], w[0] * c1[1] - w[1] * c1[0]};
                    for (int i = 0; i < 3; ++i) g[i] = g[i] - A * c1[i] + B * c2[i];
                }
                grad[3 * r] = (float)g[0];
                grad[3 * r + 1] = (float)g[1];
                grad[3 * r + 2] = (float)g[2];
            }
        }
        __syncthreads();
    }
}

// `iters` Gauss-Newton steps per ROI in one CTA: per step the direction terms
// give J^T J and J^T r (FP32 partials, FP64 block sums), thread 0 solves
// (J^T J + lambda I) delta = -J^T r with lambda = 1e-6 tr(J^T J) in FP64 and
// updates q <- exp(delta) q with FP64 renormalisation.  The directions are
// walked in the spatial order of `dsort` (w = index into the signature row),
// so that neighbouring lanes sample neighbouring pixels of the image; the
// CTA first gathers the ROI's row into that order in its own scratch row
// (global memory, L2-resident while the steps run).
constexpr int kGnThreads = 256;

__global__ void __launch_bounds__(kGnThreads) k_refine_gn(const float* __restrict__ S, const float4* __restrict__ dsort,
                                                          int32_t nv, const float4* __restrict__ img,
                                                          const double* __restrict__ q0,
                                                          const int32_t* __restrict__ best,
                                                          const double* __restrict__ quats, int64_t nroi, int iters,
                                                          float* scratch, double* q_out, float* loss_out) {
    __shared__ double red[10 * 32];
    __shared__ double tot[10];
    __shared__ double qs[4];
    __shared__ float Rs[9];
    float* srow = scratch + (int64_t)blockIdx.x * nv;
    for (int64_t r = blockIdx.x; r < nroi; r += gridDim.x) {
        __syncthreads();   // the previous ROI is done with srow
        {
            const float* src = S + r * (int64_t)nv;
            for (int i = threadIdx.x; i < nv; i += blockDim.x) srow[i] = src[__float_as_int(__ldg(&dsort[i].w))];
        }
        if (threadIdx.x == 0) {
            const double* qa = best ? quats + 4 * (int64_t)best[r] : q0 + 4 * r;
            double n = 0.0;
            for (int i = 0; i < 4; ++i) n += qa[i] * qa[i];
            n = sqrt(n);
            for (int i = 0; i < 4; ++i) qs[i] = qa[i] / n;
        }
        for (int it = 0; it <= iters; ++it) {
            const bool last = it == iters;   // final pass: loss only
            if (threadIdx.x == 0) matrix_f32(qs, Rs);
            __syncthreads();
            float Rf[9];
            for (int i = 0; i < 9; ++i) Rf[i] = Rs[i];
            float acc[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // L, Jtr[3], JtJ[6]
            for (int v = threadIdx.x; v < nv; v += blockDim.x) {
                const float4 u = ld_stream4(dsort + v);
                const DirTerm t = dir_term<true>(Rf, u.x, u.y, u.z, ld_l2(srow + v), img, !last);
                if (!t.ok) continue;
                acc[0] = fmaf(t.r, t.r, acc[0]);
                if (!last) {
                    acc[1] = fmaf(t.J[0], t.r, acc[1]);
                    acc[2] = fmaf(t.J[1], t.r, acc[2]);
                    acc[3] = fmaf(t.J[2], t.r, acc[3]);
                    acc[4] = fmaf(t.J[0], t.J[0], acc[4]);
                    acc[5] = fmaf(t.J[0], t.J[1], acc[5]);
                    acc[6] = fmaf(t.J[0], t.J[2], acc[6]);
                    acc[7] = fmaf(t.J[1], t.J[1], acc[7]);
                    acc[8] = fmaf(t.J[1], t.J[2], acc[8]);
                    acc[9] = fmaf(t.J[2], t.J[2], acc[9]);
                }
            }
            block_sum<10>(acc, tot, red);
            if (threadIdx.x == 0) {
                if (last) {
                    if (loss_out) loss_out[r] = (float)tot[0];
                } else {
                    double H[9] = {tot[4], tot[5], tot[6], tot[5], tot[7], tot[8], tot[6], tot[8], tot[9]};
                    const double lam = 1e-6 * (H[0] + H[4] + H[8]);
                    H[0] += lam;
                    H[4] += lam;
                    H[8] += lam;
                    // crystal-frame sums: J = -R j with j = g x c, so the lab system
                    // (R H_c R^T + lambda I) delta = R sum(j r) is solved as
                    // delta = R (H_c + lambda I)^-1 sum(j r)
                    const double b[3] = {tot[1], tot[2], tot[3]};
                    const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                                       H[2] * (H[3] * H[7] - H[4] * H[6]);
                    double d[3] = {0.0, 0.0, 0.0};
                    if (fabs(det) > 0.0) {
                        for (int c = 0; c < 3; ++c) {
                            double Bm[9];
                            for (int i = 0; i < 9; ++i) Bm[i] = H[i];
                            Bm[c] = b[0];
                            Bm[3 + c] = b[1];
                            Bm[6 + c] = b[2];
                            d[c] = (Bm[0] * (Bm[4] * Bm[8] - Bm[5] * Bm[7]) - Bm[1] * (Bm[3] * Bm[8] - Bm[5] * Bm[6]) +
                                    Bm[2] * (Bm[3] * Bm[7] - Bm[4] * Bm[6])) / det;
                        }
                    }
                    const M3 Rq = quat_to_matrix(qs[0], qs[1], qs[2], qs[3]);
                    const double dl[3] = {Rq.a[0] * d[0] + Rq.a[1] * d[1] + Rq.a[2] * d[2],
                                          Rq.a[3] * d[0] + Rq.a[4] * d[1] + Rq.a[5] * d[2],
                                          Rq.a[6] * d[0] + Rq.a[7] * d[1] + Rq.a[8] * d[2]};
                    double e[4], qn[4];
                    exp_quat(dl, e);
                    quat_mul(e, qs, qn);
                    const double n = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
                    for (int i = 0; i < 4; ++i) qs[i] = qn[i] / n;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double sgn = qs[0] < 0.0 ? -1.0 : 1.0;
            for (int i = 0; i < 4; ++i) q_out[4 * r + i] = sgn * qs[i];
        }
        __syncthreads();
    }
}

// k-major table to g-major int32
template <typename IdxT>
__global__ void k_lut_transpose(const IdxT* __restrict__ lut_t, int64_t ng, int64_t ng_pad, int32_t n_hat,
                                int32_t* out) {
    const int64_t n = ng * n_hat;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = i / n_hat;
        const int k = (int)(i % n_hat);
        out[i] = (int32_t)lut_t[(int64_t)k * ng_pad + g];
    }
}

}  // namespace

cudaError_t launch_lut_export(Ctx* c, Reference* r, int32_t* out) {
    const int64_t n = r->ng * r->n_hat;
    const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, 8192);
    if (r->lut_bytes == 2)
        k_lut_transpose<<<grid, 256, 0, c->stream>>>(static_cast<const uint16_t*>(r->d_lut), r->ng, r->ng_pad,
                                                     r->n_hat, out);
    else
        k_lut_transpose<<<grid, 256, 0, c->stream>>>(static_cast<const int32_t*>(r->d_lut), r->ng, r->ng_pad,
                                                     r->n_hat, out);
    return cudaGetLastError();
}

// ---- launches ------------------------------------------------------------------------

cudaError_t launch_top_nodes(Ctx* c, Reference* r) {
    int32_t npow2 = 1;
    while (npow2 < c->nv) npow2 <<= 1;
    uint64_t* keys = nullptr;
    if (dev_alloc(c, (void**)&keys, (size_t)npow2 * sizeof(uint64_t))) return cudaErrorMemoryAllocation;
    k_top_nodes<<<1, 1024, 0, c->stream>>>(r->d_node_sig, c->nv, npow2, keys, r->n_hat, r->d_top, r->d_top_val);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(keys);
    return e;
}

cudaError_t launch_build_lut(Ctx* c, Reference* r, const double* d_quats, int64_t ng) {
    const int64_t nq = ng * r->n_hat;
    const int64_t per = (int64_t)kLutThreads * kLutPer;
    const unsigned grid = (unsigned)((nq + per - 1) / per);
    if (r->lut_bytes == 2)
        k_build_lut<<<grid, kLutThreads, 0, c->stream>>>(c->d_dirs, c->nv, r->d_top, r->n_hat, d_quats, ng, r->ng_pad,
                                                         static_cast<uint16_t*>(r->d_lut));
    else
        k_build_lut<<<grid, kLutThreads, 0, c->stream>>>(c->d_dirs, c->nv, r->d_top, r->n_hat, d_quats, ng, r->ng_pad,
                                                         static_cast<int32_t*>(r->d_lut));
    return cudaGetLastError();
}

template <typename IdxT>
static cudaError_t launch_match_t(Ctx* c, Reference* r, const float* S, int64_t nroi, int32_t* best, float* score,
                                  float* scores_out, bool accumulate, float weight) {
    constexpr int G = 16 / (int)sizeof(IdxT);
    const size_t smem = ((size_t)c->nv + r->n_hat) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_match<IdxT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // one thread per G orientations, whole warps, at most 1024 threads
    const int64_t want = (r->ng + G - 1) / G;
    const int threads = (int)std::min<int64_t>(1024, std::max<int64_t>(32, (want + 31) / 32 * 32));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<IdxT>, threads, smem);
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>((int64_t)c->sm_count * per_sm, nroi);
    k_match<IdxT><<<(unsigned)grid, threads, smem, c->stream>>>(S, nroi, c->nv, static_cast<const IdxT*>(r->d_lut),
                                                                r->ng, r->ng_pad, r->d_top_val, r->n_hat, best, score,
                                                                scores_out, accumulate, weight);
    return cudaGetLastError();
}

cudaError_t launch_match(Ctx* c, Reference* r, const float* S, int64_t nroi, int32_t* best, float* score,
                         float* scores_out, bool accumulate, float weight) {
    return r->lut_bytes == 2 ? launch_match_t<uint16_t>(c, r, S, nroi, best, score, scores_out, accumulate, weight)
                             : launch_match_t<int32_t>(c, r, S, nroi, best, score, scores_out, accumulate, weight);
}

// Phase decision: candidate c's summed channel scores divided by its channel
// count n_c (in place), then phase[r] = the candidate of the lowest score
// (ties: lowest c).
__global__ void k_phase(float* score, const int32_t* n_ch, int32_t n_cand, int64_t nroi, int32_t* phase) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nroi; r += (int64_t)gridDim.x * blockDim.x) {
        float bs = INFINITY;
        int32_t bc = 0;
        for (int c = 0; c < n_cand; ++c) {
            const float v = score[(int64_t)c * nroi + r] / (float)n_ch[c];
            score[(int64_t)c * nroi + r] = v;
            if (v < bs) {
                bs = v;
                bc = c;
            }
        }
        if (phase) phase[r] = bc;
    }
}

cudaError_t launch_phase(Ctx* c, float* score, const int32_t* n_ch, int32_t n_cand, int64_t nroi, int32_t* phase) {
    const int64_t grid = std::min<int64_t>((nroi + 255) / 256, (int64_t)c->sm_count * 8);
    k_phase<<<(unsigned)grid, 256, 0, c->stream>>>(score, n_ch, n_cand, nroi, phase);
    return cudaGetLastError();
}

cudaError_t launch_topk(Ctx* c, const float* scores, int64_t ng, int64_t nroi, int32_t topk, int32_t* best,
                        float* score) {
    const int64_t grid = std::min<int64_t>((int64_t)c->sm_count * 8, nroi);
    k_topk<<<(unsigned)grid, kTopkThreads, 0, c->stream>>>(scores, ng, nroi, topk, best, score);
    return cudaGetLastError();
}

cudaError_t launch_refine_eval(Ctx* c, Reference* r, const float* S, const double* q0, const double* omega,
                               int64_t nroi, float* loss, float* grad) {
    const int64_t grid = std::min<int64_t>((int64_t)c->sm_count * 8, nroi);
    if (grad)
        k_refine_eval<true><<<(unsigned)grid, kRefThreads, 0, c->stream>>>(S, c->d_dirs, c->nv, r->d_img4, q0, omega,
                                                                          nroi, loss, grad);
    else
        k_refine_eval<false><<<(unsigned)grid, kRefThreads, 0, c->stream>>>(S, c->d_dirs, c->nv, r->d_img4, q0, omega,
                                                                           nroi, loss, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_refine_gn(Ctx* c, Reference* r, const float* S, const double* q0, const int32_t* best,
                             int64_t nroi, int iters, double* q_out, float* loss) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_refine_gn, kGnThreads, 0);
    const int64_t grid = std::min<int64_t>((int64_t)c->sm_count * std::max(per_sm, 1), nroi);
    const size_t need = (size_t)grid * c->nv * sizeof(float);
    if (need > c->gn_scratch_bytes) {
        dev_free(c->d_gn_scratch);
        c->d_gn_scratch = nullptr;
        c->gn_scratch_bytes = 0;
        if (dev_alloc(c, (void**)&c->d_gn_scratch, need)) return cudaErrorMemoryAllocation;
        c->gn_scratch_bytes = need;
    }
    k_refine_gn<<<(unsigned)grid, kGnThreads, 0, c->stream>>>(S, c->d_dirs_sorted, c->nv, r->d_img4, q0, best,
                                                              r->d_quats, nroi, iters, c->d_gn_scratch, q_out, loss);
    return cudaGetLastError();
}

}  // namespace aptidx
