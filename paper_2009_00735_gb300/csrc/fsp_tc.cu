// fsp_tc.cu -- the reciprocal-space signature (Eq. 2, the FSP method of
// Section 2.2 after Vurpillot et al.): |F(k)| with
//   F(k) = sum_w exp(-2 pi i k . x_w)
// over the centred positions x_w of a ROI, on the cubic grid
// k_a = -k_max + i_a dk (i_a < L, dk = 2 k_max / (L - 1)), as tensor-core
// GEMMs.  The exponential factorises per axis, E_a[i, w] = exp(-2 pi i k_i a_w),
// so with P[(ix, iy), w] = E_x[ix, w] E_y[iy, w]:
//   F[(ix, iy), iz] = sum_w P[(ix, iy), w] E_z[iz, w],
// a complex GEMM of M = L^2 rows, N = L columns and K = N_w.  It runs as the
// real GEMM [P_r | P_i] x [[E_r, E_i], [-E_i, E_r]] (K = 2 N_w, N = 2 L)
// whose two column halves are Re F and Im F, on tcgen05 with fp16 operands
// and FP32 accumulators in tensor memory.
//
// Work item = (ROI, 8 consecutive ix) = 512 rows = 4 M tiles of 128, their
// accumulators filling the 512 tensor-memory columns.  Per chunk of 32 atoms
// (K = 64: the 32 real parts, then the 32 imaginary parts) four table warps
// tabulate E_x (8 rows), E_y and E_z (64 rows each) in fp16 pairs (E_y, E_z by
// recurrence E[i + 1] = E[i] exp(-2 pi i dk a) over 16-row segments whose
// starts come from the hardware sine and cosine after an exact range
// reduction) into one of two table sets, ten builder warps turn the other
// set into the A stage (P = E_x E_y in fp16 pair arithmetic, 4 tiles) and
// the B stage in the K-major 128-byte-swizzled layout, and two issuer
// threads run the 16 MMAs (M = 128, N = 128, K = 16) of the previous stage.
#include <cuda_fp16.h>

#include "tcgen05.cuh"

namespace aptidx {

namespace {

constexpr int kL = APTIDX_FSP_L;                    // grid points per axis
constexpr int kN = 2 * kL;                          // MMA N: [Re F | Im F] over iz
constexpr int kTileRows = 128;                      // MMA M
constexpr int kTiles = 4;                           // M tiles per item
constexpr int kIxItem = kTiles * kTileRows / kL;    // 8 values of ix per item
constexpr int kItemsRoi = kL / kIxItem;             // 8 items per ROI
constexpr int kWc = 32;                             // atoms per chunk (K = 64)
constexpr int kThreadsF = 512;
constexpr int kIss = 2;                             // issuer warps 0, 1: tiles 0-1 and 2-3
constexpr int kTab0 = kIss * 32;                    // table warps 2..5
constexpr int kTabThreads = 128;
constexpr int kBld0 = kTab0 + kTabThreads;          // builder warps 6..15
constexpr int kBld = kThreadsF - kBld0;             // 320 builder threads
constexpr int kStageA = kTiles * kTileRows * 128;   // 64 KB
constexpr int kStageB = kN * 128;                   // 16 KB
constexpr int kStage = kStageA + kStageB;           // 80 KB
// table rows of 32 atoms as fp16 pairs: words 0..15 = (Re a_2j, Re a_2j+1),
// words 16..31 = (Im a_2j, Im a_2j+1); 36-word stride spreads rows over banks
constexpr int kTabRowH = kWc + 4;
constexpr int kTabSet = (kIxItem + 2 * kL) * kTabRowH * 4;   // one table set: E_x, E_y, E_z
constexpr int kTabBytes = 2 * kTabSet;              // double buffered
constexpr int kSeg = 16;                            // recurrence segment (rows)

static_assert(kL == 64, "the tiling assumes L = 64");

struct FspParams {
    const float4* atoms;   // centred ROI atoms, CSR by off
    const int64_t* off;
    const int32_t* nw;
    int64_t nroi;
    float kmax, dk;
    float* out;            // nroi x L^3 amplitudes, iz fastest
    int32_t* counter;
    int* status;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bld_sync() { asm volatile("bar.sync 1, %0;" ::"r"(kBld) : "memory"); }
__device__ __forceinline__ void tab_sync() { asm volatile("bar.sync 2, %0;" ::"r"(kTabThreads) : "memory"); }

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// exp(-i pi x) for x = 2 k a (so exp(-2 pi i k a)): x reduced exactly to
// [-1, 1] (x - 2 rint(x / 2) is exact in FP32 for |x| < 2^22), then the
// hardware sine and cosine of pi x_r, absolute error a few 1e-7 on [-pi, pi]
__device__ __forceinline__ float2 cexp_m2pi(float two_ka) {
    const float xr = two_ka - 2.f * rintf(0.5f * two_ka);
    float s, c;
    __sincosf(3.14159265358979324f * xr, &s, &c);
    return make_float2(c, -s);
}

__device__ __forceinline__ __half2 u2h2(uint32_t v) { return *reinterpret_cast<const __half2*>(&v); }
__device__ __forceinline__ uint32_t h22u(__half2 h) { return *reinterpret_cast<const uint32_t*>(&h); }

__device__ __forceinline__ uint32_t pack_h2(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// byte offset of 16-byte chunk j of row r in a K-major 128-byte-swizzled
// operand (rows of 64 fp16, atoms of 8 rows x 128 bytes)
__device__ __forceinline__ uint32_t sw128_off(int r, int j) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}

__global__ void __launch_bounds__(kThreadsF, 1) k_fsp_tc(FspParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* tabs = smem + 2 * kStage;   // two table sets: E_x, E_y, E_z as fp16 pairs
    uint64_t* bars = reinterpret_cast<uint64_t*>(tabs + kTabBytes);
    uint64_t* full = bars;          // [2] stage built -> issuers
    uint64_t* empty = bars + 2;     // [2] stage's MMAs completed -> builders
    uint64_t* accum = bars + 4;     // all MMAs of the item completed
    uint64_t* tfull = bars + 5;     // [2] table set filled -> builders
    uint64_t* tempty = bars + 7;    // [2] table set consumed -> table warps
    int64_t* item_s = reinterpret_cast<int64_t*>(bars + 9);
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(bars + 10);
    int* fail_s = reinterpret_cast<int*>(bars + 11);
    const volatile int* vfail = fail_s;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], kIss);
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 1);
        }
        mbar_init(accum, kIss);
        *fail_s = 0;
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(tmem_s, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t st_addr = smem_u32(smem);
    const uint32_t idesc = idesc_f16_mk(kTileRows, kN, false);

    uint32_t cg = 0;      // chunks handled so far by this CTA (stage and table-set ring position)
    uint32_t nitem = 0;   // items finished so far (accumulator barrier phase)
    const int64_t n_items = p.nroi * kItemsRoi;
    for (;;) {
        if (tid == 0) *item_s = atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t item = *item_s;
        const int failed = *fail_s;
        __syncthreads();
        if (item >= n_items || failed) break;
        const int64_t roi = item / kItemsRoi;
        const int g = (int)(item % kItemsRoi);
        const int nw = p.nw[roi];
        const float4* A = p.atoms + p.off[roi];
        const int nch = max(1, (nw + kWc - 1) / kWc);

        if (warp < kIss) {
            // ---- issuers: warp 0 tiles 0-1, warp 1 tiles 2-3 ----
            if (lane == 0) {
                bool ok = true;
                for (int c = 0; c < nch && ok; ++c) {
                    const uint32_t s = (cg + c) & 1u, u = (cg + c) >> 1;
                    ok = mbar_wait_bounded(&full[s], u & 1u, p.status);
                    if (!ok) {
                        *fail_s = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = st_addr + s * kStage;
                    const uint32_t b_base = a_base + kStageA;
#pragma unroll
                    for (int tt = 0; tt < 2; ++tt) {
                        const int t = warp * 2 + tt;
                        const uint64_t ad = sdesc_sw128(a_base + (uint32_t)t * (kTileRows * 128), 16u, 1024u);
                        const uint64_t bd = sdesc_sw128(b_base, 16u, 1024u);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)   // K = 16 per MMA: +32 bytes along the row
                            mma_f16(tmem + (uint32_t)t * 128u, ad + 2u * kk, bd + 2u * kk, idesc,
                                    (c > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(&empty[s]);
                }
                mma_commit(accum);   // also after a failure: the epilogue then waits on what was issued
            }
            __syncwarp();
        } else if (warp < kBld0 / 32) {
            // ---- table warps: E_x (8 rows), E_y, E_z (64 rows each) of the
            // chunk's 32 atoms into table set (chunk & 1), running up to two
            // chunks ahead of the builders.  E_y, E_z by recurrence
            // E[i + 1] = E[i] exp(-2 pi i dk a) over 16-row segments in FP32,
            // stored as fp16 pairs; lane = atom, neighbouring lanes pair up ----
            const int tt = tid - kTab0;
            const bool even = (lane & 1) == 0;
            const uint32_t sel = even ? 0x5410u : 0x3276u;   // (own Re, other Re) | (other Im, own Im)
            const int col = (lane >> 1) + (even ? 0 : kWc / 2);
            for (int c = 0; c < nch; ++c) {
                const uint32_t cc = cg + c, b = cc & 1u, u = cc >> 1;
                if (tt == 0 && u >= 1 && !*vfail && !mbar_wait_bounded(&tempty[b], (u - 1) & 1u, p.status)) *fail_s = 1;
                tab_sync();
                uint32_t* Exh = reinterpret_cast<uint32_t*>(tabs + b * kTabSet);
                uint32_t* Eyh = Exh + kIxItem * kTabRowH;
                uint32_t* Ezh = Eyh + kL * kTabRowH;
                const int w = c * kWc + lane;
                const bool valid = w < nw;
                const float4 at = valid ? A[w] : make_float4(0.f, 0.f, 0.f, 0.f);
                auto put = [&](uint32_t* row, float2 e) {
                    const uint32_t own = valid ? pack_h2(e.x, e.y) : 0u;
                    const uint32_t oth = __shfl_xor_sync(0xffffffffu, own, 1);
                    row[col] = __byte_perm(own, oth, sel);
                };
                const int i0 = (tt >> 5) * kSeg;
                const float k0 = fmaf((float)i0, p.dk, -p.kmax);
                float2 ey = cexp_m2pi(2.f * k0 * at.y), ez = cexp_m2pi(2.f * k0 * at.z);
                const float2 dy = cexp_m2pi(2.f * p.dk * at.y), dz = cexp_m2pi(2.f * p.dk * at.z);
#pragma unroll 4
                for (int j = 0; j < kSeg; ++j) {
                    put(Eyh + (i0 + j) * kTabRowH, ey);
                    put(Ezh + (i0 + j) * kTabRowH, ez);
                    ey = cmul(ey, dy);
                    ez = cmul(ez, dz);
                }
#pragma unroll
                for (int rep = 0; rep < 2; ++rep) {
                    const int ixl = (tt >> 5) + 4 * rep;
                    const float k = fmaf((float)(g * kIxItem + ixl), p.dk, -p.kmax);
                    put(Exh + ixl * kTabRowH, cexp_m2pi(2.f * k * at.x));
                }
                tab_sync();
                if (tt == 0) mbar_arrive(&tfull[b]);
            }
        } else {
            // ---- builders: the A stage (P = E_x E_y, 4 tiles) and the B stage ----
            const int bt = tid - kBld0;
            for (int c = 0; c < nch; ++c) {
                const uint32_t cc = cg + c, s = cc & 1u, u = cc >> 1;
                if (bt == 0 && !*vfail) {   // after a timeout the rest of the item runs unsynchronised
                    if (u >= 1 && !mbar_wait_bounded(&empty[s], (u - 1) & 1u, p.status)) *fail_s = 1;
                    if (!*vfail && !mbar_wait_bounded(&tfull[s], u & 1u, p.status)) *fail_s = 1;
                }
                bld_sync();
                const uint32_t* Exh = reinterpret_cast<const uint32_t*>(tabs + s * kTabSet);
                const uint32_t* Eyh = Exh + kIxItem * kTabRowH;
                const uint32_t* Ezh = Eyh + kL * kTabRowH;
                unsigned char* stA = smem + s * kStage;
                unsigned char* stB = stA + kStageA;
                if (bt < kL * 4) {
                    // A: row m = ixl * 64 + iy, K = [Re P of the 32 atoms | Im P];
                    // unit (iy, q): E_y of atoms 8q .. 8q+7 in registers, all 8
                    // values of ix (E_x reads are broadcasts); P in fp16 pairs
                    const int iy = bt & (kL - 1), q = bt / kL;
                    const uint4 yr4 = *reinterpret_cast<const uint4*>(Eyh + iy * kTabRowH + 4 * q);
                    const uint4 yi4 = *reinterpret_cast<const uint4*>(Eyh + iy * kTabRowH + kWc / 2 + 4 * q);
                    const __half2 yr[4] = {u2h2(yr4.x), u2h2(yr4.y), u2h2(yr4.z), u2h2(yr4.w)};
                    const __half2 yi[4] = {u2h2(yi4.x), u2h2(yi4.y), u2h2(yi4.z), u2h2(yi4.w)};
#pragma unroll 4
                    for (int ixl = 0; ixl < kIxItem; ++ixl) {
                        const uint4 xr4 = *reinterpret_cast<const uint4*>(Exh + ixl * kTabRowH + 4 * q);
                        const uint4 xi4 = *reinterpret_cast<const uint4*>(Exh + ixl * kTabRowH + kWc / 2 + 4 * q);
                        const __half2 xr[4] = {u2h2(xr4.x), u2h2(xr4.y), u2h2(xr4.z), u2h2(xr4.w)};
                        const __half2 xi[4] = {u2h2(xi4.x), u2h2(xi4.y), u2h2(xi4.z), u2h2(xi4.w)};
                        uint32_t re[4], im[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            re[j] = h22u(__hfma2(xr[j], yr[j], __hneg2(__hmul2(xi[j], yi[j]))));
                            im[j] = h22u(__hfma2(xr[j], yi[j], __hmul2(xi[j], yr[j])));
                        }
                        const int m = ixl * kL + iy, t = m >> 7, r = m & 127;
                        unsigned char* rowt = stA + t * (kTileRows * 128);
                        *reinterpret_cast<uint4*>(rowt + sw128_off(r, q)) = make_uint4(re[0], re[1], re[2], re[3]);
                        *reinterpret_cast<uint4*>(rowt + sw128_off(r, q + 4)) =
                            make_uint4(im[0], im[1], im[2], im[3]);
                    }
                } else {
                    // B: row n < L: [Re E_z | -Im E_z] of iz = n; n >= L:
                    // [Im E_z | Re E_z] of iz = n - L (fp16 pairs moved as bits,
                    // the sign flipped in the bits)
                    for (int e = bt - kL * 4; e < kN * 4; e += kBld - kL * 4) {
                        const int n = e & (kN - 1), q = e / kN, z = n & (kL - 1);   // 8 lanes: 8 rows, one q
                        const uint4 zr = *reinterpret_cast<const uint4*>(Ezh + z * kTabRowH + 4 * q);
                        const uint4 zi = *reinterpret_cast<const uint4*>(Ezh + z * kTabRowH + kWc / 2 + 4 * q);
                        const uint32_t f = 0x80008000u;
                        const uint4 v0 = n < kL ? zr : zi;
                        const uint4 v1 = n < kL ? make_uint4(zi.x ^ f, zi.y ^ f, zi.z ^ f, zi.w ^ f) : zr;
                        *reinterpret_cast<uint4*>(stB + sw128_off(n, q)) = v0;
                        *reinterpret_cast<uint4*>(stB + sw128_off(n, q + 4)) = v1;
                    }
                }
                fence_proxy_async_smem();
                bld_sync();
                if (bt == 0) {
                    mbar_arrive(&full[s]);
                    mbar_arrive(&tempty[s]);
                }
            }
        }
        cg += (uint32_t)nch;

        // ---- epilogue: |F| = sqrt(Re^2 + Im^2); warp w reads TMEM lane
        // quadrant w % 4 of tile w / 4 ----
        if (tid == 0 && !mbar_wait_bounded(accum, nitem & 1u, p.status)) *fail_s = 1;
        ++nitem;
        __syncthreads();
        tc_fence_after();
        if (!*fail_s) {
            const int qd = warp & 3, t = warp >> 2;
            const int m = t * kTileRows + qd * 32 + lane;
            const int ix = g * kIxItem + (m >> 6), iy = m & (kL - 1);
            float* dst = p.out + (((int64_t)roi * kL + ix) * kL + iy) * kL;
            const uint32_t tb = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)t * 128u;
            for (int h = 0; h < 2; ++h) {
                float re[32], im[32];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    tmem_ld8(tb + (uint32_t)(h * 32 + 8 * i), re + 8 * i);
                    tmem_ld8(tb + (uint32_t)(kL + h * 32 + 8 * i), im + 8 * i);
                }
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 32; i += 4) {
                    float4 v;
                    v.x = sqrtf(re[i] * re[i] + im[i] * im[i]);
                    v.y = sqrtf(re[i + 1] * re[i + 1] + im[i + 1] * im[i + 1]);
                    v.z = sqrtf(re[i + 2] * re[i + 2] + im[i + 2] * im[i + 2]);
                    v.w = sqrtf(re[i + 3] * re[i + 3] + im[i + 3] * im[i + 3]);
                    *reinterpret_cast<float4*>(dst + h * 32 + i) = v;
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace

size_t fsp_smem_bytes() { return 1024 + 2 * (size_t)kStage + kTabBytes + 128; }

cudaError_t launch_fsp_tc(Ctx* c, double kmax, float* out) {
    const size_t smem = fsp_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_fsp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FspParams p;
    p.atoms = c->d_atoms;
    p.off = c->d_off;
    p.nw = c->d_nw;
    p.nroi = c->nroi;
    p.kmax = (float)kmax;
    p.dk = (float)(2.0 * kmax / (double)(kL - 1));
    p.out = out;
    p.counter = c->d_counter + 2;
    p.status = c->d_status;
    if ((e = cudaMemsetAsync(p.counter, 0, sizeof(int32_t), c->stream)) != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>((int64_t)c->sm_count, c->nroi * kItemsRoi);
    if (grid < 1) return cudaSuccess;
    k_fsp_tc<<<(unsigned)grid, kThreadsF, smem, c->stream>>>(p);
    return cudaGetLastError();
}

}  // namespace aptidx
