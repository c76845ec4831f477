// fsp_tc.cu -- the reciprocal-space signature (Eq. 2, the FSP method of
// Section 2.2 after Vurpillot et al.): |F(k)| with
//   F(k) = sum_w exp(-2 pi i k . x_w)
// over the centred positions x_w of a ROI, on the cubic grid
// k_a = -k_max + i_a dk (i_a < L, dk = 2 k_max / (L - 1)), as tensor-core
// GEMMs.  The exponential factorises per axis, E_a[i, w] = exp(-2 pi i k_i a_w),
// so with P[(ix, iy), w] = E_x[ix, w] E_y[iy, w]:
//   F[(ix, iy), iz] = sum_w P[(ix, iy), w] E_z[iz, w],
// a complex GEMM of M = L^2 rows, N = L columns and K = N_w.  It runs
// transposed as the real GEMM
//   [[Re F^T], [Im F^T]] = [[E_r, -E_i], [E_i, E_r]] x [P_r | P_i]^T
// (rows: Re F then Im F over iz; columns (ix, iy); K = 2 N_w), on tcgen05
// with fp16 operands and FP32 accumulators in tensor memory.
//
// Work item = (ROI, 64 values of iz, 8 of ix, 64 of iy): M = 128 rows of
// the E_z block matrix times 512 columns of P, two MMAs of N = 256 per K
// step, the accumulators filling the 512 tensor-memory columns; L is any
// multiple of 64 up to 512 (L^3 / 32768 items per ROI).  Per chunk of 32
// atoms (K = 64: the 32 real parts, then the 32 imaginary parts):
//   four table warps tabulate E_x (8 rows) and E_y (64 rows) as fp16 pairs
//     into one of two table sets (E_y by the recurrence
//     E[i + 1] = E[i] exp(-2 pi i dk a) over runs of 4 rows, whose starts
//     come from the hardware sine and cosine after an exact range
//     reduction);
//   four warps compute E_z (recurrence of step 2 dk over 8 rows) and write
//     the A operand (the E_z block matrix, 16 KB) straight into the stage;
//   eight builder warps form the B operand P = E_x E_y in fp16 pair
//     arithmetic (512 rows, 64 KB);
//   two issuer threads run the 8 MMAs (M = 128, N = 256, K = 16) of the
//     previous stage.
// Both operands are K-major with the 128-byte swizzle.  The epilogue pairs
// the Re and Im lanes through shared memory and writes |F| with iz fastest.
#include <cuda_fp16.h>

#include "tcgen05.cuh"

namespace aptidx {

namespace {

constexpr int kL = 64;                              // grid points per block of iy and of iz
constexpr int kN = 2 * kL;                          // rows of the E_z block matrix: Re F, Im F over iz
constexpr int kTileRows = 128;
constexpr int kTiles = 4;                           // 512 (ix, iy) columns per item
constexpr int kIxItem = kTiles * kTileRows / kL;    // 8 values of ix per item
constexpr int kWc = 32;                             // atoms per chunk (K = 64)
constexpr int kThreadsF = 576;                      // 18 warps, every role spread over the 4 SM sub-partitions
constexpr int kIss = 2;                             // issuer warps 0, 1: N halves 0 and 1
constexpr int kTab0 = kIss * 32;                    // E_x, E_y table warps 2..5
constexpr int kTabThreads = 128;
constexpr int kZ0 = kTab0 + kTabThreads;            // E_z warps 6..9
constexpr int kZThreads = 128;
constexpr int kBld0 = kZ0 + kZThreads;              // B-operand builder warps 10..17
constexpr int kBld = kThreadsF - kBld0;             // 256 builder threads
constexpr int kNHalf = kTiles * kTileRows / 2;      // 256 P rows per MMA
constexpr int kStageP = kTiles * kTileRows * 128;   // 64 KB: P, the B operand
constexpr int kStageZ = kN * 128;                   // 16 KB: the E_z block matrix, the A operand
constexpr int kStage = kStageP + kStageZ;           // 80 KB
// table rows of 32 atoms as fp16 pairs: words 0..15 = (Re a_2j, Re a_2j+1),
// words 16..31 = (Im a_2j, Im a_2j+1); 36-word stride spreads rows over banks
constexpr int kTabRowH = kWc + 4;
constexpr int kTabSet = (kIxItem + kL) * kTabRowH * 4;   // one table set: E_x, E_y
constexpr int kTabBytes = 2 * kTabSet;              // double buffered
constexpr int kRowsHw = 8;   // E_y / E_z rows per half warp and chunk (recurrence length)

static_assert(kL == 64 && APTIDX_FSP_L_MIN == kL && APTIDX_FSP_L_MAX % kL == 0, "the tiling assumes 64-blocks");

struct FspParams {
    const float4* atoms;   // centred ROI atoms, CSR by off
    const int64_t* off;
    const int32_t* nw;
    int64_t nroi;
    float kmax, dk;
    int L;                 // grid points per axis, a multiple of 64
    int nxb, nyb;          // blocks of 8 ix and of 64 iy per axis
    int items_roi;         // (L / 64) blocks of iz x nxb x nyb
    float* out;            // nroi x L^3 amplitudes, iz fastest
    int32_t* counter;
    int* status;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bld_sync() { asm volatile("bar.sync 1, %0;" ::"r"(kBld) : "memory"); }
__device__ __forceinline__ void tab_sync() { asm volatile("bar.sync 2, %0;" ::"r"(kTabThreads) : "memory"); }
__device__ __forceinline__ void z_sync() { asm volatile("bar.sync 3, %0;" ::"r"(kZThreads) : "memory"); }

// centred position of atom w of the chunk, zero past the ROI's end
__device__ __forceinline__ float4 atom_or_zero(const float4* A, int w, int nw) {
    return w < nw ? A[w] : make_float4(0.f, 0.f, 0.f, 0.f);
}
// the four warps of one epilogue column group (named barriers 4..7)
__device__ __forceinline__ void grp_sync(int grp) { asm volatile("bar.sync %0, 128;" ::"r"(4 + grp) : "memory"); }

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
// operand (rows of 64 fp16, atoms of 8 rows x 128 bytes, 1024 bytes apart)
__device__ __forceinline__ uint32_t sw128_off(int r, int j) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
}

__global__ void __launch_bounds__(kThreadsF, 1) k_fsp_tc(FspParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* tabs = smem + 2 * kStage;   // two table sets: E_x, E_y as fp16 pairs
    uint64_t* bars = reinterpret_cast<uint64_t*>(tabs + kTabBytes);
    uint64_t* full = bars;          // [2] stage written (E_z warps, builders) -> issuers
    uint64_t* empty = bars + 2;     // [2] stage's MMAs completed -> E_z warps, builders
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
            mbar_init(&full[i], 2);
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
    const uint32_t idesc = idesc_f16_mk(kTileRows, kNHalf, false);

    uint32_t cg = 0;      // chunks handled so far by this CTA (stage and table-set ring position)
    uint32_t nitem = 0;   // items finished so far (accumulator barrier phase)
    const int64_t n_items = p.nroi * p.items_roi;
    for (;;) {
        if (tid == 0) *item_s = atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t item = *item_s;
        const int failed = *fail_s;
        __syncthreads();
        if (item >= n_items || failed) break;
        // item = (ROI, 64-block of iz, 8-block of ix, 64-block of iy)
        const int64_t roi = item / p.items_roi;
        int rest = (int)(item % p.items_roi);
        const int iy0 = (rest % p.nyb) * kL;
        rest /= p.nyb;
        const int ix0 = (rest % p.nxb) * kIxItem;
        const int iz0 = (rest / p.nxb) * kL;
        const int nw = p.nw[roi];
        const float4* A = p.atoms + p.off[roi];
        const int nch = max(1, (nw + kWc - 1) / kWc);

        if (warp < kIss) {
            // ---- issuers: warp h runs N half h (P rows 256h .. 256h + 255
            // into tensor-memory columns 256h ..) ----
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
                    const uint32_t base = st_addr + s * kStage;
                    const uint64_t ad = sdesc_sw128(base + kStageP, 16u, 1024u);
                    const uint64_t bd = sdesc_sw128(base + (uint32_t)warp * (kNHalf * 128), 16u, 1024u);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)   // K = 16 per MMA: +32 bytes along the row
                        mma_f16(tmem + (uint32_t)warp * kNHalf, ad + 2u * kk, bd + 2u * kk, idesc,
                                (c > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                mma_commit(accum);   // also after a failure: the epilogue then waits on what was issued
            }
            __syncwarp();
        } else if (tid < kZ0) {
            // ---- table warps: E_x (8 rows) and E_y (64 rows) of the chunk's
            // 32 atoms into table set (chunk & 1), up to two chunks ahead of
            // the builders.  Lane (hw, pl) = (lane / 16, lane % 16) holds
            // atoms 2 pl, 2 pl + 1; warp tw, half hw: E_y rows
            // 16 tw + 4 hw + {0..3} and 16 tw + 4 hw + 8 + {0..3} (two
            // recurrences of step dk), E_x row tw + 4 hw.  The halves' rows
            // are 4 apart, so a store's two 16-word halves fall in disjoint
            // banks (36-word rows) ----
            const int tw = (tid - kTab0) >> 5, hw = lane >> 4, pl = lane & 15;
            const int r0 = 16 * tw + 4 * hw, ixl = tw + 4 * hw;
            const float kx = fmaf((float)(ix0 + ixl), p.dk, -p.kmax);
            const float ky0 = fmaf((float)(iy0 + r0), p.dk, -p.kmax);
            const float ky1 = fmaf((float)(iy0 + r0 + 8), p.dk, -p.kmax);
            float4 na = atom_or_zero(A, 2 * pl, nw), nb = atom_or_zero(A, 2 * pl + 1, nw);
            for (int c = 0; c < nch; ++c) {
                const uint32_t cc = cg + c, b = cc & 1u, u = cc >> 1;
                const float4 xa = na, xb = nb;
                if (c + 1 < nch) {
                    na = atom_or_zero(A, (c + 1) * kWc + 2 * pl, nw);
                    nb = atom_or_zero(A, (c + 1) * kWc + 2 * pl + 1, nw);
                }
                if (tid == kTab0 && u >= 1 && !*vfail && !mbar_wait_bounded(&tempty[b], (u - 1) & 1u, p.status))
                    *fail_s = 1;
                tab_sync();
                uint32_t* Exh = reinterpret_cast<uint32_t*>(tabs + b * kTabSet);
                uint32_t* Eyh = Exh + kIxItem * kTabRowH;
                {   // atoms past the ROI's end get E_x = 0, so their columns of P vanish
                    const float2 z2 = make_float2(0.f, 0.f);
                    const float2 ea = c * kWc + 2 * pl < nw ? cexp_m2pi(2.f * kx * xa.x) : z2;
                    const float2 eb = c * kWc + 2 * pl + 1 < nw ? cexp_m2pi(2.f * kx * xb.x) : z2;
                    Exh[ixl * kTabRowH + pl] = pack_h2(ea.x, eb.x);
                    Exh[ixl * kTabRowH + kWc / 2 + pl] = pack_h2(ea.y, eb.y);
                }
                float2 ea = cexp_m2pi(2.f * ky0 * xa.y), eb = cexp_m2pi(2.f * ky0 * xb.y);
                float2 fa = cexp_m2pi(2.f * ky1 * xa.y), fb = cexp_m2pi(2.f * ky1 * xb.y);
                const float2 da = cexp_m2pi(2.f * p.dk * xa.y), db = cexp_m2pi(2.f * p.dk * xb.y);
#pragma unroll
                for (int j = 0; j < kRowsHw / 2; ++j) {
                    uint32_t* row = Eyh + (r0 + j) * kTabRowH;
                    row[pl] = pack_h2(ea.x, eb.x);
                    row[kWc / 2 + pl] = pack_h2(ea.y, eb.y);
                    row += 8 * kTabRowH;
                    row[pl] = pack_h2(fa.x, fb.x);
                    row[kWc / 2 + pl] = pack_h2(fa.y, fb.y);
                    ea = cmul(ea, da);
                    eb = cmul(eb, db);
                    fa = cmul(fa, da);
                    fb = cmul(fb, db);
                }
                tab_sync();
                if (tid == kTab0) mbar_arrive(&tfull[b]);
            }
        } else if (tid < kBld0) {
            // ---- E_z warps: the A operand of the stage directly.  Row n < L:
            // [Re E_z | -Im E_z] of iz = n; row n + L: [Im E_z | Re E_z].
            // Lane (hw, pl) holds atoms 2 pl, 2 pl + 1; warp zw, half hw: iz =
            // 16 zw + hw + 2 j (j < 8).  The two halves write rows n, n + 1
            // (the same swizzle phase) and take the two words of a row in
            // opposite order, so a store touches 32 distinct banks ----
            const int zw = (tid - kZ0) >> 5, hw = lane >> 4, pl = lane & 15;
            const int n0 = 16 * zw + hw;
            const float kz0 = fmaf((float)(iz0 + n0), p.dk, -p.kmax);
            const uint32_t wofs_lo = (uint32_t)(pl & 3) * 4u, c_lo = (uint32_t)(pl >> 2), c_hi = c_lo + 4u;
            const uint32_t c0 = hw ? c_hi : c_lo, c1 = hw ? c_lo : c_hi;   // this half's first and second word
            float4 na = atom_or_zero(A, 2 * pl, nw), nb = atom_or_zero(A, 2 * pl + 1, nw);
            for (int c = 0; c < nch; ++c) {
                const uint32_t cc = cg + c, s = cc & 1u, u = cc >> 1;
                const float4 xa = na, xb = nb;
                if (c + 1 < nch) {
                    na = atom_or_zero(A, (c + 1) * kWc + 2 * pl, nw);
                    nb = atom_or_zero(A, (c + 1) * kWc + 2 * pl + 1, nw);
                }
                if (tid == kZ0 && u >= 1 && !*vfail && !mbar_wait_bounded(&empty[s], (u - 1) & 1u, p.status))
                    *fail_s = 1;
                z_sync();
                unsigned char* stZ = smem + s * kStage + kStageP;
                float2 ea = cexp_m2pi(2.f * kz0 * xa.z), eb = cexp_m2pi(2.f * kz0 * xb.z);
                const float2 da = cexp_m2pi(4.f * p.dk * xa.z), db = cexp_m2pi(4.f * p.dk * xb.z);
#pragma unroll
                for (int j = 0; j < kRowsHw; ++j) {
                    const int n = n0 + 2 * j;
                    const uint32_t r7 = (uint32_t)(n & 7);
                    const uint32_t re = pack_h2(ea.x, eb.x), im = pack_h2(ea.y, eb.y);
                    unsigned char* row = stZ + (n >> 3) * 1024 + r7 * 128 + wofs_lo;
                    // word pl (chunk c_lo): K = 2 pl, 2 pl + 1; word 16 + pl (chunk c_hi): K = 32 + 2 pl, ..
                    unsigned char* p0 = row + ((c0 ^ r7) << 4);
                    unsigned char* p1 = row + ((c1 ^ r7) << 4);
                    const uint32_t nim = im ^ 0x80008000u;
                    *reinterpret_cast<uint32_t*>(p0) = hw ? nim : re;            // row n: [Re | -Im]
                    *reinterpret_cast<uint32_t*>(p1) = hw ? re : nim;
                    *reinterpret_cast<uint32_t*>(p0 + 8 * 1024) = hw ? re : im;  // row n + L: [Im | Re]
                    *reinterpret_cast<uint32_t*>(p1 + 8 * 1024) = hw ? im : re;
                    ea = cmul(ea, da);
                    eb = cmul(eb, db);
                }
                fence_proxy_async_smem();
                z_sync();
                if (tid == kZ0) mbar_arrive(&full[s]);
            }
        } else {
            // ---- builders: the B operand, row m = ixl * 64 + iy of P with
            // K = [Re P of the 32 atoms | Im P]; thread (iy, q) keeps E_y of
            // atoms 8q .. 8q+7 in registers across the item's 8 values of ix
            // (E_x reads are broadcasts) ----
            const int bt = tid - kBld0;
            const int iy = bt & (kL - 1), q = bt / kL;
            for (int c = 0; c < nch; ++c) {
                const uint32_t cc = cg + c, s = cc & 1u, u = cc >> 1;
                if (bt == 0 && !*vfail) {   // after a timeout the rest of the item runs unsynchronised
                    if (u >= 1 && !mbar_wait_bounded(&empty[s], (u - 1) & 1u, p.status)) *fail_s = 1;
                    if (!*vfail && !mbar_wait_bounded(&tfull[s], u & 1u, p.status)) *fail_s = 1;
                }
                bld_sync();
                const uint32_t* Exh = reinterpret_cast<const uint32_t*>(tabs + s * kTabSet);
                const uint32_t* Eyh = Exh + kIxItem * kTabRowH;
                unsigned char* stP = smem + s * kStage;
                const uint4 yr4 = *reinterpret_cast<const uint4*>(Eyh + iy * kTabRowH + 4 * q);
                const uint4 yi4 = *reinterpret_cast<const uint4*>(Eyh + iy * kTabRowH + kWc / 2 + 4 * q);
                const __half2 yr[4] = {u2h2(yr4.x), u2h2(yr4.y), u2h2(yr4.z), u2h2(yr4.w)};
                const __half2 yi[4] = {u2h2(yi4.x), u2h2(yi4.y), u2h2(yi4.z), u2h2(yi4.w)};
#pragma unroll
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
                    const int m = ixl * kL + iy;
                    *reinterpret_cast<uint4*>(stP + sw128_off(m, q)) = make_uint4(re[0], re[1], re[2], re[3]);
                    *reinterpret_cast<uint4*>(stP + sw128_off(m, q + 4)) = make_uint4(im[0], im[1], im[2], im[3]);
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

        // ---- epilogue: tensor-memory lane n holds Re F (n < 64) or Im F
        // (n >= 64) of iz = iz0 + n mod 64, column j the grid point
        // (ix0 + j / 64, iy0 + j % 64).
        // Warp w reads lane quadrant qd = w % 4 of column group w / 4; the
        // Re and Im quadrants of the same iz (qd, qd ^ 2) meet in shared
        // memory (the idle stage), taking turns at forming |F| ----
        if (tid == 0 && !mbar_wait_bounded(accum, nitem & 1u, p.status)) *fail_s = 1;
        ++nitem;
        __syncthreads();
        tc_fence_after();
        if (!*fail_s && warp < 16) {
            const int qd = warp & 3, grp = warp >> 2, pair = qd & 1;
            const bool is_im = qd >= 2;
            float* slab = reinterpret_cast<float*>(smem) + (grp * 2 + pair) * 32 * 32;
            const uint32_t tl = tmem + ((uint32_t)(qd * 32) << 16);
            const int64_t L = p.L;
            float* dst = p.out + ((roi * L + ix0) * L + iy0) * L + iz0 + pair * 32 + lane;
            for (int bb = 0; bb < 4; ++bb) {
                const int c0 = grp * 128 + bb * 32;
                float v[32];
#pragma unroll
                for (int i = 0; i < 4; ++i) tmem_ld8(tl + (uint32_t)(c0 + 8 * i), v + 8 * i);
                tmem_wait_ld();
                const bool sender = (bb & 1) ? !is_im : is_im;
                if (sender) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) slab[j * 32 + lane] = v[j];
                }
                grp_sync(grp);
                if (!sender) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float o = slab[j * 32 + lane];
                        const float a2 = fmaf(v[j], v[j], o * o);
                        const int m = c0 + j;   // (ix, iy) = (ix0 + m / 64, iy0 + m % 64)
                        dst[((m >> 6) * L + (m & (kL - 1))) * L] = a2 * rsqrtf(fmaxf(a2, 1e-30f));   // |F|, 0 at a2 = 0
                    }
                }
                grp_sync(grp);
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

cudaError_t launch_fsp_tc(Ctx* c, int L, double kmax, float* out) {
    const size_t smem = fsp_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_fsp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    FspParams p;
    p.atoms = c->d_atoms;
    p.off = c->d_off;
    p.nw = c->d_nw;
    p.nroi = c->nroi;
    p.kmax = (float)kmax;
    p.dk = (float)(2.0 * kmax / (double)(L - 1));
    p.L = L;
    p.nxb = L / kIxItem;
    p.nyb = L / kL;
    p.items_roi = (L / kL) * p.nxb * p.nyb;
    p.out = out;
    p.counter = c->d_counter + 2;
    p.status = c->d_status;
    if ((e = cudaMemsetAsync(p.counter, 0, sizeof(int32_t), c->stream)) != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>((int64_t)c->sm_count, c->nroi * p.items_roi);
    if (grid < 1) return cudaSuccess;
    k_fsp_tc<<<(unsigned)grid, kThreadsF, smem, c->stream>>>(p);
    return cudaGetLastError();
}

}  // namespace aptidx
