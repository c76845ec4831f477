// signature_tc.cu -- steps (a2)-(a5) with the band spectrum on the tcgen05
// tensor cores: X = H x T, H the [64 directions x bins] histogram tile and T
// the [bins x band columns] DFT matrix (cos and sin of 2 pi k n / 2^m),
// accumulated in FP32 in tensor memory (Section 2.2: the Fourier amplitude
// spectrum of every SDM; the paper notes that the SDMs of a ROI share one
// bin count, which permits batching their transforms).
//
// The histogram of a tile is built in chunks of at most 1024 bins (2^m <= 1024:
// one chunk; m = 11, 12: two or four) and over blocks of at most 2048 atoms,
// so that every count of a block is exact in fp16; every (block, chunk) pass is
// contracted into the same tensor-memory accumulators.  The contraction of a
// pass runs as M = 128 rows: rows 0-63 are the 64 directions over the chunk's
// first half of bins, rows 64-127 the same directions over its second half.
// Both halves use the twiddles of the first half, since
// w^(k (n + h)) = w^(k h) w^(k n) for w = exp(-2 pi i / 2^m) and the half
// offset h = 2^(m-1) (one chunk: w^(k h) = (-1)^k) or h = 512 (chunks of 1024);
// the epilogue forms X(k) = D_lo(k) + w^(k h) D_hi(k).
//
// Antipodal pairs: when the direction set holds u and -u, only u is projected;
// -u gets the same signature value and frequency bin (its histogram is the
// mirror image of u's, whose spectrum has the same amplitudes), provided no
// atom's bin product along u is an exact integer, which the histogram pass
// checks exactly (common.cuh).  A tile with such an atom runs a second pass
// over the negated directions and writes their signatures from their own
// histograms.
//
// Wide bands (more frequency groups than one B batch holds) run in their own
// kernel instance (kWide): the chunk's bins split into quarters, only the
// first quarter's twiddles stream from L2 through four shared-memory stages,
// and each stage feeds two M = 128 MMAs per K step (bin quarters 0 | 2 and
// 1 | 3); the epilogue applies the quarter factor w^(k NBc / 4).
//
// Per 64-direction tile of a ROI and (block, chunk) pass:
//   1. histograms by shared-memory atomics (bank-private columns, as in the
//      FP32 path); counts c <= 2048, so the u16 bit pattern of c is the fp16
//      value c * 2^-24 exactly (fp16 is linear through its subnormal range up
//      to 0x0800) and the histogram is the A operand as it stands;
//   2. an in-place permutation of 16-byte chunks gives the MN-major 128-byte
//      swizzled layout (chunk c of bin row k moves to c ^ (k & 7));
//   3. up to four issuer threads issue the bins / 32 tcgen05.mma of the chunk
//      (M = 128, K = 16, N = 16 per group of 4 frequencies: 8 hi columns, then
//      8 lo columns, where T = T_hi + T_lo with both parts fp16) into FP32
//      accumulators in TMEM;
//   4. after the last pass, warps 0-7 read the accumulators (tcgen05.ld), add
//      the partials, hi and lo parts and the two bin halves (one exchange in
//      shared memory), scale by 2^24 and keep the band maximum of |X(k)|,
//      while warps 8-15 zero the histogram for the next pass.
#include <cuda_fp16.h>

#include "tcgen05.cuh"

namespace aptidx {

namespace {

constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kDirs = kTileDirs;     // 64 directions per tile
constexpr int kRows = 2 * kDirs;     // MMA M: (direction, bin half)
constexpr int kBtBytes = 32 * 1024;  // shared-memory budget of the B operand (narrow bands)
constexpr int kWideStage = 16 * 1024;   // wide bands: one of four twiddle stream stages
constexpr int kExBytes = kDirs * 8 * 4;   // epilogue exchange: one group's (re, im) x 4 per direction
constexpr int kIssuers = 4;          // at most this many warps issue MMAs, one TMEM partial accumulator each
constexpr int kChunkBins = 1024;     // bins per histogram chunk (128 KB of words)

struct TcParams {
    const float4* atoms;
    const int64_t* off;
    const int32_t* nw;
    const int32_t* order;
    const float4* dirs;     // direction slots, padded to whole tiles with (1, 0, 0)
    const int2* slot_idx;   // per slot: (output direction, antipodal partner or -1); NULL: slot = direction
    int32_t nv;
    int32_t tiles_per_roi;
    int32_t tiles_per_item;
    int32_t items_per_roi;
    int64_t nroi;
    const float* scale;
    const int32_t* band;
    int m;
    int32_t kbase;          // frequency of column group 0
    const uint8_t* twb;     // global B: [chunk][hi|lo][group][k-block] x 1 KB
    const uint8_t* twk;     // global B, streamed layout: [chunk][32-bin block of the first quarter][hi|lo]
                            // [group] x 512 B, 64-byte swizzle (wide bands), ng_total + 1 groups per run,
                            // the last one zero
    int32_t bt_bytes;       // shared-memory bytes of the B region (kBtBytes, or 4 kWideStage)
    int32_t ng_total;
    int32_t gb;             // groups per shared-memory batch
    uint32_t tmem_cols;
    float* S;
    uint16_t* argk;
    uint16_t* hist_out;
    int64_t single_roi;
    int32_t* counter;
    int* status;
    int atom_cap;           // atoms per block (<= 2048)
    int n_iss;              // MMA issuer warps (1 .. kIssuers)
    BandSet bands;
};

// instruction descriptor: A MN-major (the histogram), B K-major, M = 128
__device__ __forceinline__ uint32_t idesc_f16(int n) { return idesc_f16_mk(kRows, n, true); }

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}

// Debug export of one (block, chunk) pass: adds the counts of rows
// [0, nbc) to h_out[v * 2^m + bc * nbc + row] (the caller zeroes h_out).
__device__ __forceinline__ void hist_export_add(const uint32_t* H, int nbc, int NB, int bc, int tile, int nv,
                                                uint16_t* h_out, int tid, int nthreads) {
    for (int i = tid; i < nbc * 32; i += nthreads) {
        const int b = i >> 5, l = i & 31;
        const uint32_t w = H[i];
        const int64_t v0 = (int64_t)tile * 64 + 2 * l;
        const int64_t col = (int64_t)bc * nbc + b;
        if (v0 < nv) h_out[v0 * NB + col] = (uint16_t)(h_out[v0 * NB + col] + (w & 0xFFFFu));
        if (v0 + 1 < nv) h_out[(v0 + 1) * NB + col] = (uint16_t)(h_out[(v0 + 1) * NB + col] + (w >> 16));
    }
}

// v += (-i)^(R0 + q) u for the n complex pairs (re, im) of v and u, where a
// pair (r, i) stands for r - i i: multiplying by -i maps it to (-i, r), by -1
// to (-r, -i), by i to (i, -r)
template <int R0>
__device__ __forceinline__ void quarter_rot(float* v, const float* u, int n) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        if (q < n) {
            const int ph = (R0 + q) & 3;   // constant once unrolled
            const float ur = u[2 * q], ui = u[2 * q + 1];
            v[2 * q] += ph == 0 ? ur : ph == 1 ? -ui : ph == 2 ? -ur : ui;
            v[2 * q + 1] += ph == 0 ? ui : ph == 1 ? ur : ph == 2 ? -ui : -ur;
        }
    }
}

// ---- the kernel ----------------------------------------------------------------

// kNB: band slots of the epilogue (1: the ROI's own band; APTIDX_MAX_BANDS:
// the pass's BandSet, aptidx_compute_signatures_multi); kWide: the instance
// that streams the twiddles of bands wider than one B batch (the narrow-band
// instance is compiled without that code)
template <int kNB, bool kWide>
__global__ void __launch_bounds__(kThreads, 1) k_sig_tc(TcParams p) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment for the swizzled operands; offset arithmetic on the
    // shared array keeps the pointers in the shared address space
    unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int NB = 1 << p.m;
    const int NBc = NB < kChunkBins ? NB : kChunkBins;   // bins per chunk
    const int nchunk = NB / NBc;
    const uint32_t cmask = (uint32_t)(nchunk - 1);
    const int KB = NBc / 128;   // 1 KB K-blocks of the B operand per chunk (K = NBc / 2 rows)
    uint32_t* H = reinterpret_cast<uint32_t*>(smem);
    unsigned char* BT = smem + (size_t)NBc * 128;
    float* EX = reinterpret_cast<float*>(BT + p.bt_bytes);   // [kDirs][8]
    float4* A = reinterpret_cast<float4*>(BT + p.bt_bytes + kExBytes);
    float4* DB = A + p.atom_cap;   // [2][kDirs]: this tile's directions and the next tile's
    int2* DI = reinterpret_cast<int2*>(DB + 2 * kDirs);   // [2][kDirs]: (output, partner) of those slots
    float* EX2 = reinterpret_cast<float*>(DI + 2 * kDirs);   // [128 TMEM lanes][8]: partials 2, 3
    // barriers: [0] atoms, [1] B operand, [2 .. 2 + kIssuers) MMA completion per
    // issuer, then the wide-band stream: four stage loads, four stage MMA completions
    constexpr int kBars = 2 + kIssuers + 8;
    uint64_t* bars = reinterpret_cast<uint64_t*>(EX2 + 128 * 8);
    uint64_t* wbar = bars + 2 + kIssuers;
    int* flag = reinterpret_cast<int*>(bars + kBars);
    int64_t* item_s = reinterpret_cast<int64_t*>(bars + kBars + 1);
    uint32_t* tmem_s = reinterpret_cast<uint32_t*>(bars + kBars + 2);
    int* iss_ok = reinterpret_cast<int*>(bars + kBars + 3);   // [kIssuers]
    unsigned* r2max_s = reinterpret_cast<unsigned*>(iss_ok + kIssuers);   // largest |x|^2 of the item's atoms
    int* prod_ok = reinterpret_cast<int*>(r2max_s + 1);                      // wide-band stream producer

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < kBars; ++i) mbar_init(&bars[i], 1);
        fence_barrier_init();
    }
    for (int i = tid; i < NBc * 8; i += kThreads) reinterpret_cast<uint4*>(H)[i] = make_uint4(0, 0, 0, 0);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_s)),
                     "r"(p.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_s;
    const uint32_t h_addr = smem_u32(H);
    const uint32_t bt_addr = smem_u32(BT);

    uint32_t ph_atoms = 0, ph_b = 0, ph_mma = 0;   // ph_mma: this warp's issuer barrier
    uint32_t wph = 0u, wdph = 0u;   // wide stream parity bits (bit i: buffer i): stage loads (thread 0), stage MMAs (thread 32)
    int cur_g0 = -1, cur_nb = -1, cur_bc = -1;     // B operand held in shared memory
    const float magic = bin_magic(p.m);
    const bool sym = p.slot_idx != nullptr;
    const int64_t n_items = (p.single_roi >= 0 ? 1 : p.nroi) * (int64_t)p.items_per_roi;
    bool failed = false;

    for (;;) {
        if (tid == 0) *item_s = atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t item = *item_s;
        __syncthreads();
        if (item >= n_items) break;
        const int64_t roi = p.single_roi >= 0 ? p.single_roi : (int64_t)p.order[item / p.items_per_roi];
        const int grp = (int)(item % p.items_per_roi);
        const int nw = p.nw[roi];
        const int64_t abase = p.off[roi];
        const float scale = p.scale[roi];
        const int klo = p.band[2 * roi], khi = p.band[2 * roi + 1];
        const int fg0 = (klo - p.kbase) >> 2, fg1 = (khi - p.kbase) >> 2;
        const int ng = fg1 - fg0 + 1;
        const int nbatch = (ng + p.gb - 1) / p.gb;
        const int t0 = grp * p.tiles_per_item;
        const int t1 = min(t0 + p.tiles_per_item, p.tiles_per_roi);
        const int nblk = max(1, (nw + p.atom_cap - 1) / p.atom_cap);   // atom blocks
        if (nblk == 1) {
            if (tid == 0) *r2max_s = 0u;
            if (!stage_atoms(A, p.atoms + abase, nw, &bars[0], ph_atoms, p.status, flag)) {
                failed = true;
                break;
            }
            pair_atoms(A, nw, tid, kThreads, r2max_s);
        }
        // the first tile's directions (later tiles' arrive while the tile
        // before them runs)
        if (tid < kDirs) {
            cp_async16(DB + (t0 & 1) * kDirs + tid, p.dirs + (int64_t)t0 * kDirs + tid);
            if (sym) cp_async8(DI + (t0 & 1) * kDirs + tid, p.slot_idx + (int64_t)t0 * kDirs + tid);
        }
        cp_async_wait_all();
        __syncthreads();
        // with one atom block and no nonzero integer product possible, the
        // antipodal check only looks for s = 0 (a product per lane instead of
        // an exact count)
        const bool zero_check = sym && nblk == 1 && !nonzero_integer_products_possible(scale, __uint_as_float(*r2max_s));

        for (int tile = t0; tile < t1 && !failed; ++tile) {
            const int cur = tile & 1;
            float4 d0 = DB[cur * kDirs + 2 * lane];
            float4 d1 = DB[cur * kDirs + 2 * lane + 1];
            const int pt0 = sym ? DI[cur * kDirs + 2 * lane].y : -1;
            const int pt1 = sym ? DI[cur * kDirs + 2 * lane + 1].y : -1;
            if (tile + 1 < t1 && tid < kDirs) {
                cp_async16(DB + (cur ^ 1) * kDirs + tid, p.dirs + (int64_t)(tile + 1) * kDirs + tid);
                if (sym) cp_async8(DI + (cur ^ 1) * kDirs + tid, p.slot_idx + (int64_t)(tile + 1) * kDirs + tid);
            }
            int tile_bad = 0;
            for (int pass = 0; pass < 2 && !failed; ++pass) {
                if (pass == 1) {
                    if (!tile_bad) break;
                    // the partners -u of this tile's directions, from their own histograms
                    d0 = make_float4(-d0.x, -d0.y, -d0.z, d0.w);
                    d1 = make_float4(-d1.x, -d1.y, -d1.z, d1.w);
                }
                const bool count = sym && pass == 0;
                uint32_t c0 = 0, c1 = 0;
                uint64_t zp = f2_dup(1.f);
                int handled = 0;
                const int n_sub = nblk * nchunk;
                for (int sub = 0; sub < n_sub && !failed; ++sub) {
                    const int blk = sub / nchunk, bc = sub % nchunk;
                    const int cn = min(p.atom_cap, nw - blk * p.atom_cap);
                    const bool last = sub == n_sub - 1;
                    if (nblk > 1 && bc == 0) {
                        if (!stage_atoms(A, p.atoms + abase + (int64_t)blk * p.atom_cap, cn, &bars[0], ph_atoms,
                                         p.status, flag)) {
                            failed = true;
                            break;
                        }
                        pair_atoms(A, cn, tid, kThreads);
                        __syncthreads();
                    }
                    // ---- 1. histograms (H is zero here) ----
                    if (nchunk == 1) {
                        if (count && zero_check)
                            handled += hist_tile_pairs2<kWarps, 2, false>(H, A, cn, warp, lane, d0, d1, scale, magic,
                                                                          0u, 0u, c0, c1, zp);
                        else if (count)
                            handled += hist_tile_pairs2<kWarps, 1, false>(H, A, cn, warp, lane, d0, d1, scale, magic,
                                                                          0u, 0u, c0, c1, zp);
                        else
                            hist_tile_pairs2<kWarps, 0, false>(H, A, cn, warp, lane, d0, d1, scale, magic, 0u, 0u,
                                                               c0, c1, zp);
                    } else {
                        if (count && bc == 0 && zero_check)
                            handled += hist_tile_pairs2<kWarps, 2, true>(H, A, cn, warp, lane, d0, d1, scale, magic,
                                                                         (uint32_t)bc, cmask, c0, c1, zp);
                        else if (count && bc == 0)
                            handled += hist_tile_pairs2<kWarps, 1, true>(H, A, cn, warp, lane, d0, d1, scale, magic,
                                                                         (uint32_t)bc, cmask, c0, c1, zp);
                        else
                            hist_tile_pairs2<kWarps, 0, true>(H, A, cn, warp, lane, d0, d1, scale, magic,
                                                              (uint32_t)bc, cmask, c0, c1, zp);
                    }
                    __syncthreads();
                    if (p.hist_out) {
                        hist_export_add(H, NBc, NB, bc, tile, p.nv, p.hist_out, tid, kThreads);
                        __syncthreads();   // every row is read before the permutation moves it
                    }

                    // ---- 2. swizzle: every warp brings bin rows into the MN-major
                    // 128-byte swizzled layout in place (a warp holds four rows, 512
                    // contiguous bytes, one 16-byte chunk per lane, and writes chunk c
                    // of row k to chunk c ^ (k & 7); rows with k & 7 == 0 stay).  The
                    // pass runs at the shared-memory bandwidth; interleaving it with
                    // the MMAs below slows both, so the two run one after the other.
                    // ---- 3. contraction: lane 0 of warps 0 .. n_iss-1 issues every
                    // n_iss-th K step into its own partial accumulator (a single
                    // tcgen05.mma costs the issuing warp ~75 cycles whatever its N;
                    // several issuers overlap that cost); every pass after the first
                    // accumulates onto the result so far.
                    // Wide bands (more frequency groups than one B batch holds):
                    // the chunk's bins split into four quarters, and the twiddles of
                    // the first quarter, all the ROI's groups, stream through four
                    // 16 KB shared-memory stages, one per (32-bin K block, hi|lo
                    // part), in the 64-byte-swizzled K-major layout.  Each stage
                    // feeds two M = 128 MMAs per K step: block 0 (rows 0-63 the first
                    // quarter's bins, rows 64-127 the third's) into tensor-memory
                    // columns 8 g .. 8 g + 7 of group g, block 1 (second and fourth
                    // quarters) into the same columns from bo1 on; hi and lo products
                    // accumulate into the same columns, one MMA of N = 8 x groups per
                    // block and K step.  Twiddle row n serves bin n + j NBc / 4 of
                    // quarter j up to the factor w^(f j NBc / 4) the epilogue applies,
                    // so a stage's bytes feed twice the tensor work of the bin-half
                    // split alone.  Thread 0 issues the MMAs as stages land; thread 32
                    // refills a stage once its MMAs are done, three stages ahead.
                    const bool wide = kWide && nbatch > 1;
                    const int n_iss = wide ? 1 : p.n_iss;
                    const uint32_t sbo_b = (uint32_t)KB * 1024u;
                    const bool issuer = lane == 0 && warp < n_iss;
                    const uint32_t acc0 = sub > 0 ? 1u : 0u;
                    // N = 8 x groups must be a multiple of 16 (M = 128): an odd group
                    // count takes one more group of twiddles (zeros past the last
                    // group), whose columns are never read
                    const int ngw = (ng + 1) & ~1;
                    const uint32_t bo1 = (uint32_t)((8 * ngw + 31) & ~31);   // block 1's first column
                    const uint32_t wbytes = (uint32_t)ngw * 512u;
                    const int KB4 = NBc / 128;      // 32-bin K blocks of the chunk's first quarter
                    const int S = 2 * KB4;          // stages: (block, part)
                    auto wide_load = [&](int s) {   // stage s = 2 x block + part, into buffer s & 3
                        const int kb = s >> 1, part = s & 1, bf = s & 3;
                        mbar_arrive_expect_tx(&wbar[bf], wbytes);
                        bulk_g2s(BT + (size_t)bf * kWideStage,
                                 p.twk + ((((size_t)bc * KB4 + kb) * 2 + part) * (p.ng_total + 1) + fg0) * 512, wbytes,
                                 &wbar[bf]);
                    };
                    int ok = 1;
                    if (tid == 0) {
                        if (wide) {
                            // the first two stages load while the histogram is swizzled
                            // (the epilogue before wrote the B region through the
                            // generic proxy)
                            fence_proxy_async_smem();
                            for (int st = 0; st < 4; ++st) wide_load(st);
                            cur_g0 = -1;   // the narrow-band B operand is overwritten
                            *prod_ok = 1;
                        } else {
                            // B operand of the band for this chunk (kept across tiles while
                            // the ROI band and the chunk allow)
                            const int nb0 = fg1 + 1 - fg0;
                            if (fg0 != cur_g0 || nb0 != cur_nb || bc != cur_bc) {
                                const uint32_t part = (uint32_t)nb0 * KB * 1024u;
                                fence_proxy_async_smem();
                                mbar_arrive_expect_tx(&bars[1], 2 * part);
                                bulk_g2s(BT, p.twb + ((size_t)(2 * bc) * p.ng_total + fg0) * KB * 1024, part, &bars[1]);
                                bulk_g2s(BT + part, p.twb + ((size_t)(2 * bc + 1) * p.ng_total + fg0) * KB * 1024, part,
                                         &bars[1]);
                                ok = mbar_wait_bounded(&bars[1], ph_b, p.status) ? 1 : 0;
                                if (!ok) mbar_wait_bounded(&bars[1], ph_b, p.status, 1u << 20);
                                ph_b ^= 1u;
                                cur_g0 = ok ? fg0 : -1;
                                cur_nb = nb0;
                                cur_bc = bc;
                            }
                        }
                        *flag = ok;
                    }
                    // two groups of four rows per pass, 64 rows apart (same k & 7;
                    // the chunk's rows are a multiple of 128)
                    for (int r0 = warp * 4; r0 < NBc; r0 += kWarps * 8) {
                        const int k = r0 + (lane >> 3), c = lane & 7, sw = k & 7;
                        uint4* row = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(H) + (size_t)k * 128);
                        uint4* row2 = row + kWarps * 4 * 8;   // row k + 64
                        uint4 x, x2;
                        if (sw) {
                            x = row[c];
                            x2 = row2[c];
                        }
                        __syncwarp();
                        if (sw) {
                            row[c ^ sw] = x;
                            row2[c ^ sw] = x2;
                        }
                    }
                    fence_proxy_async_smem();
                    tc_fence_before();
                    __syncthreads();
                    ok = *flag;
                    // A: rows 64-127 (second bin half) one swizzle atom along M
                    // away, NBc / 2 bin rows of 128 bytes
                    const uint64_t a0 = sdesc_sw128(h_addr, (uint32_t)NBc * 64u, 1024u);
                    if (issuer && ok && wide) {
                        // the consumer: MMAs of each stage as it lands
                        tc_fence_after();
                        const uint32_t idw = idesc_f16(8 * ngw);
                        for (int s = 0; s < S && ok; ++s) {
                            const int kb = s >> 1, bf = s & 3;
                            if (!mbar_wait_bounded(&wbar[bf], (wph >> bf) & 1u, p.status)) {
                                mbar_wait_bounded(&wbar[bf], (wph >> bf) & 1u, p.status, 1u << 20);
                                ok = 0;
                            }
                            wph ^= 1u << bf;
                            if (!ok) break;
                            tc_fence_after();
                            // B: 8 x groups rows (4 frequencies x cos, sin per group) of
                            // 32 bins, 512 bytes per 8 rows; 32 bytes per K step.  A:
                            // block 0 from bin 0, block 1 from bin NBc / 4 (NBc x 32
                            // bytes on), the other half NBc / 2 bins away in both
                            const uint64_t b0 = sdesc_sw64(bt_addr + (uint32_t)bf * kWideStage, 16u, 512u);
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const uint64_t ad = a0 + (uint64_t)((2 * kb + kk) * 128);
                                const uint64_t bd = b0 + (uint64_t)(kk * 2);
                                const uint32_t acc = (s > 0 || kk > 0) ? 1u : acc0;
                                mma_f16(tmem, ad, bd, idw, acc);
                                mma_f16(tmem + bo1, ad + (uint64_t)(NBc * 2), bd, idw, acc);
                            }
                            mma_commit(&wbar[4 + bf]);
                        }
                    } else if (wide && tid == 32 && ok) {
                        // the producer: a stage's buffer takes the stage four later
                        // once its MMAs are done; then the last four stages' MMAs
                        int pok = 1;
                        for (int s = 4; s < S + 4 && pok; ++s) {
                            const int bf = s & 3;
                            if (!mbar_wait_bounded(&wbar[4 + bf], (wdph >> bf) & 1u, p.status)) {
                                mbar_wait_bounded(&wbar[4 + bf], (wdph >> bf) & 1u, p.status, 1u << 20);
                                pok = 0;
                            }
                            wdph ^= 1u << bf;
                            if (pok && s < S) wide_load(s);
                        }
                        *prod_ok = pok;
                    } else if (issuer && ok) {
                        tc_fence_after();
                        const int nb0 = fg1 + 1 - fg0;
                        const uint32_t idesc = idesc_f16(16 * nb0);
                        const uint32_t dcol = tmem + (uint32_t)warp * (uint32_t)(16 * p.gb);
                        const uint64_t b0 = sdesc_sw128(bt_addr, 16u, sbo_b);
                        // descriptors advance by constant steps: A by 2 KB per K step,
                        // B by 32 bytes inside a 128-byte row and 1 KB per 64-bin
                        // block (the address field counts 16-byte units)
                        for (int kk = warp; kk < NBc / 32; kk += n_iss) {
                            const uint64_t ad = a0 + (uint64_t)(kk * 128);
                            const uint64_t bd = b0 + (uint64_t)((kk >> 2) * 64 + (kk & 3) * 2);
                            mma_f16(dcol, ad, bd, idesc, (kk >= n_iss) ? 1u : acc0);
                        }
                    }
                    if (issuer) {
                        int mine = ok;
                        if (mine && !wide) {
                            mma_commit(&bars[2 + warp]);
                            mine = mbar_wait_bounded(&bars[2 + warp], ph_mma, p.status) ? 1 : 0;
                            if (!mine) mbar_wait_bounded(&bars[2 + warp], ph_mma, p.status, 1u << 20);
                            ph_mma ^= 1u;
                        }
                        iss_ok[warp] = mine;
                    }
                    // the non-integer counts are complete once the last pass's
                    // histogram is in: a partner whose count falls short of the
                    // atoms this warp handled needs its own histogram
                    const int bad = count && last &&
                                    (zero_check ? (pt0 >= 0 || pt1 >= 0) && (f2_lo(zp) == 0.f || f2_hi(zp) == 0.f)
                                                : ((pt0 >= 0 && c0 != (uint32_t)handled) ||
                                                   (pt1 >= 0 && c1 != (uint32_t)handled)));
                    const int any_bad = __syncthreads_or(bad);
                    if (last) tile_bad = any_bad;
                    {
                        int all = wide ? *prod_ok : 1;
                        for (int i = 0; i < n_iss; ++i) all &= iss_ok[i];
                        if (!all) {
                            failed = true;
                            break;
                        }
                    }
                    tc_fence_after();
                    if (!last) {
                        // H is read by the MMAs above; zero it for the next pass
                        for (int i = tid; i < NBc * 8; i += kThreads)
                            reinterpret_cast<uint4*>(H)[i] = make_uint4(0, 0, 0, 0);
                        __syncthreads();
                    }
                }
                if (failed) break;

                // ---- 4. epilogue: |X(k)| and the band maximum; the warps from zw0 on
                // zero H for the next tile meanwhile.  With four partial
                // accumulators and one frequency group (the common case), warps
                // 0-7 each read two partials of one TMEM lane quadrant and warps
                // 0, 1 combine the four contributions of their directions after a
                // single exchange; otherwise warps 0-3 (one per quadrant) read
                // every partial and exchange per frequency group ----
                // warps 0, 1: pass 0 writes the slot's direction (and its partner
                // when the tile's mirror images are exact); pass 1 the partners
                auto write_out = [&](const float* best, const int* bk, int dir) {
                    const int slot = tile * kDirs + dir;
                    int v0, v1;
                    if (sym) {
                        const int2 si = DI[cur * kDirs + dir];
                        v0 = pass == 0 ? si.x : si.y;
                        v1 = (pass == 0 && !tile_bad) ? si.y : -1;
                    } else {
                        v0 = slot < p.nv ? slot : -1;
                        v1 = -1;
                    }
                    const int64_t rb = (p.single_roi >= 0 ? 0 : roi) * (int64_t)p.nv;
#pragma unroll
                    for (int b = 0; b < kNB; ++b) {
                        if (b < band_count_t<kNB>(p.bands)) {
                            const int64_t ob = band_off_t<kNB>(p.bands, b) + rb;
                            if (v0 >= 0) {
                                p.S[ob + v0] = best[b];
                                if (p.argk) p.argk[ob + v0] = (uint16_t)bk[b];
                            }
                            if (v1 >= 0) {
                                p.S[ob + v1] = best[b];
                                if (p.argk) p.argk[ob + v1] = (uint16_t)bk[b];
                            }
                        }
                    }
                };
                const bool quad = nbatch == 1 && p.n_iss == kIssuers && fg1 == fg0;
                const int zw0 = (quad || (kWide && nbatch > 1)) ? 8 : 4;   // first zeroing warp
                if (warp >= zw0) {
                    for (int i = tid - zw0 * 32; i < NBc * 8; i += kThreads - zw0 * 32)
                        reinterpret_cast<uint4*>(H)[i] = make_uint4(0, 0, 0, 0);
                } else if (quad) {
                    // warp w: partials 2 (w >> 2) and 2 (w >> 2) + 1 (hi and lo
                    // columns) of lane quadrant w & 3; warps 2-7 leave their sums
                    // in shared memory (EX: warps 2, 3; EX2: warps 4-7)
                    const uint32_t cols_b = (uint32_t)(16 * p.gb);
                    const uint32_t c0 = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(2 * (warp >> 2)) * cols_b;
                    float a[8], b[8], c[8], d[8], x[8];
                    tmem_ld8(c0, a);
                    tmem_ld8(c0 + 8u, b);
                    tmem_ld8(c0 + cols_b, c);
                    tmem_ld8(c0 + cols_b + 8u, d);
                    tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = (a[i] + b[i]) + (c[i] + d[i]);
                    if (warp >= 2) {
                        float4* xs = reinterpret_cast<float4*>((warp < 4 ? EX + (warp - 2) * 32 * 8 : EX2 + (warp - 4) * 32 * 8) +
                                                               lane * 8);
                        xs[0] = make_float4(x[0], x[1], x[2], x[3]);
                        xs[1] = make_float4(x[4], x[5], x[6], x[7]);
                    }
                    asm volatile("bar.sync 2, 256;" ::: "memory");
                    if (warp < 2) {
                        // direction dir: rows dir (first bin half: this warp, partials
                        // 0-1; warp 4 + warp, partials 2-3) and 64 + dir (second half:
                        // warp 2 + warp, partials 0-1; warp 6 + warp, partials 2-3)
                        const int dir = warp * 32 + lane;
                        const float4* pl = reinterpret_cast<const float4*>(EX2 + (warp * 32 + lane) * 8);
                        const float4* ph = reinterpret_cast<const float4*>(EX + (warp * 32 + lane) * 8);
                        const float4* ph2 = reinterpret_cast<const float4*>(EX2 + ((2 + warp) * 32 + lane) * 8);
                        const float4 l0 = pl[0], l1 = pl[1], h0 = ph[0], h1 = ph[1], g0 = ph2[0], g1 = ph2[1];
                        const float lo[8] = {x[0] + l0.x, x[1] + l0.y, x[2] + l0.z, x[3] + l0.w,
                                             x[4] + l1.x, x[5] + l1.y, x[6] + l1.z, x[7] + l1.w};
                        const float hv[8] = {h0.x + g0.x, h0.y + g0.y, h0.z + g0.z, h0.w + g0.w,
                                             h1.x + g1.x, h1.y + g1.y, h1.z + g1.z, h1.w + g1.w};
                        float best[kNB];
                        int bk[kNB];
                        band_init_t<kNB>(p.bands, klo, best, bk);
                        // the band maximum on |X|^2 (its root is the maximum
                        // amplitude); the second half's factor w^(f h) is (-1)^f for
                        // one chunk (a branch outside the frequency loop, so that the
                        // loop carries no predicated sincos)
                        const int f0 = p.kbase + 4 * fg0;
                        if (nchunk == 1) {
                            const float sg0 = (f0 & 1) ? -1.f : 1.f;
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const float sg = (q & 1) ? -sg0 : sg0;
                                const float xr = lo[2 * q] + sg * hv[2 * q], xi = lo[2 * q + 1] + sg * hv[2 * q + 1];
                                band_update_t<kNB>(p.bands, klo, khi, f0 + q, xr * xr + xi * xi, best, bk);
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int f = f0 + q;
                                float fs, fc;   // w^(f h) = fc - i fs, h = 512
                                sincospif((float)f * (float)NBc / (float)NB, &fs, &fc);
                                const float xr = lo[2 * q] + fc * hv[2 * q] - fs * hv[2 * q + 1];
                                const float xi = lo[2 * q + 1] + fs * hv[2 * q] + fc * hv[2 * q + 1];
                                band_update_t<kNB>(p.bands, klo, khi, f, xr * xr + xi * xi, best, bk);
                            }
                        }
#pragma unroll
                        for (int b = 0; b < kNB; ++b)
                            if (best[b] >= 0.f) best[b] = sqrtf(best[b]) * 16777216.0f;
                        write_out(best, bk, dir);
                    }
                } else if (kWide && nbatch > 1) {
                    // Wide bands, warps 0-7: the 64 directions form two groups
                    // (32 p .. 32 p + 31, p = warp & 1); a group's first-half rows are
                    // lane quadrant p (warps p, p + 4), its second-half rows quadrant
                    // 2 + p (warps p + 2, p + 6).  The 4-group column batches split
                    // into four frequency quarters, one per warp of the group
                    // (quarter 0: warp p, 1: p + 4, 2: p + 2, 3: p + 6).  Each warp
                    // first hands the warp of quarter qi ^ 2 (the other bin half)
                    // its own rows of that quarter through the (now idle) B region
                    // as [column][direction], then forms X = D_lo + w^(f h) D_hi over
                    // its quarter and keeps the band maximum of |X|^2 (its root is
                    // the maximum amplitude); quarters 1-3 pass their maxima to
                    // quarter 0 through EX and EX2, which keeps a higher quarter's
                    // value only when strictly greater (lowest-k ties).
                    float best[kNB];
                    int bk[kNB];
                    band_init_t<kNB>(p.bands, klo, best, bk);
                    const int q4 = warp & 3;
                    const uint32_t lane_base = tmem + ((uint32_t)(q4 * 32) << 16);
                    const int dir = (warp & 1) * 32 + lane;
                    const bool first = q4 < 2;                       // first bin half
                    const int qi = (first ? 0 : 2) + (warp >> 2);    // frequency quarter
                    float* xw = reinterpret_cast<float*>(BT);        // [8 x 32 groups][kDirs]
                    const int nb32 = (ng + 3) >> 2;
                    auto qb = [&](int j) { return (j * nb32 + 3) >> 2; };   // quarter j = batches [qb(j), qb(j + 1))
                    const uint32_t bo1 = (uint32_t)((8 * ((ng + 1) & ~1) + 31) & ~31);
                    // columns [c, c + 2 n) of batch b (n frequencies from f0, cos and
                    // sin) over this lane quadrant's bin half: D = D_a + w^(f NBc / 4)
                    // D_b from blocks 0 and 1; w^(f N / 4) = (-i)^f for one chunk,
                    // whose exponent mod 4 follows from kbase mod 4 (a permutation
                    // with signs, fixed per unrolled frequency)
                    auto quarter_add = [&](float* v, const float* u, int n, int f0) {
                        if (nchunk == 1) {
                            switch (p.kbase & 3) {
                                case 0: quarter_rot<0>(v, u, n); break;
                                case 1: quarter_rot<1>(v, u, n); break;
                                case 2: quarter_rot<2>(v, u, n); break;
                                default: quarter_rot<3>(v, u, n); break;
                            }
                        } else {
                            for (int q = 0; q < n; ++q) {
                                float fs, fc;   // w^(f NBc / 4) = fc - i fs
                                sincospif((float)(f0 + q) * (float)NBc / (float)(2 * NB), &fs, &fc);
                                const float ur = u[2 * q], ui = u[2 * q + 1];
                                v[2 * q] += fc * ur - fs * ui;
                                v[2 * q + 1] += fs * ur + fc * ui;
                            }
                        }
                    };
                    for (int b = qb(qi ^ 2); b < qb((qi ^ 2) + 1); ++b) {
                        float v[32], u[32];
                        const uint32_t col = lane_base + (uint32_t)(32 * b);
                        tmem_ld16(col, v);
                        tmem_ld16(col + 16u, v + 16);
                        tmem_ld16(col + bo1, u);
                        tmem_ld16(col + bo1 + 16u, u + 16);
                        tmem_wait_ld();
                        quarter_add(v, u, 16, p.kbase + 4 * (fg0 + 4 * b));
#pragma unroll
                        for (int i = 0; i < 32; ++i) xw[(32 * b + i) * kDirs + dir] = v[i];
                    }
                    asm volatile("bar.sync 1, 256;" ::: "memory");
                    for (int b = qb(qi); b < qb(qi + 1); ++b) {
                        float v[32];
                        {
                            float u[32];
                            const uint32_t col = lane_base + (uint32_t)(32 * b);
                            tmem_ld16(col, v);
                            tmem_ld16(col + 16u, v + 16);
                            tmem_ld16(col + bo1, u);
                            tmem_ld16(col + bo1 + 16u, u + 16);
                            tmem_wait_ld();
                            quarter_add(v, u, 16, p.kbase + 4 * (fg0 + 4 * b));
                        }
                        const int f0 = p.kbase + 4 * (fg0 + 4 * b);
                        const float* xo = xw + 32 * b * kDirs + dir;
                        // the second half's factor w^(f h): (-1)^f for one chunk (a
                        // branch outside the frequency loop, so that the loop carries
                        // no predicated sincos), else cos and sin of pi f h 2 / 2^m
                        if (nchunk == 1) {
                            const float sg0 = (f0 & 1) ? -1.f : 1.f;
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const float orr = xo[(2 * q) * kDirs], ori = xo[(2 * q + 1) * kDirs];
                                const float lr = first ? v[2 * q] : orr, li = first ? v[2 * q + 1] : ori;
                                const float hr = first ? orr : v[2 * q], hs = first ? ori : v[2 * q + 1];
                                const float sg = (q & 1) ? -sg0 : sg0;
                                const float xr = lr + sg * hr, xi = li + sg * hs;
                                band_update_t<kNB>(p.bands, klo, khi, f0 + q, xr * xr + xi * xi, best, bk);
                            }
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const int f = f0 + q;
                                const float orr = xo[(2 * q) * kDirs], ori = xo[(2 * q + 1) * kDirs];
                                const float lr = first ? v[2 * q] : orr, li = first ? v[2 * q + 1] : ori;
                                const float hr = first ? orr : v[2 * q], hs = first ? ori : v[2 * q + 1];
                                float fs, fc;   // w^(f h) = fc - i fs, h = 512
                                sincospif((float)f * (float)NBc / (float)NB, &fs, &fc);
                                const float xr = lr + fc * hr - fs * hs, xi = li + fs * hr + fc * hs;
                                band_update_t<kNB>(p.bands, klo, khi, f, xr * xr + xi * xi, best, bk);
                            }
                        }
                    }
                    // maxima of quarters 1-3: slot ((qi - 1) x 64 + dir) x 8 of EX
                    // (first 512 floats) and EX2
                    auto mx = [&](int qq, int k) -> float& {
                        const int f = ((qq - 1) * kDirs + dir) * 8 + k;
                        return f < kDirs * 8 ? EX[f] : EX2[f - kDirs * 8];
                    };
                    if (qi > 0) {
#pragma unroll
                        for (int b = 0; b < kNB; ++b) {
                            mx(qi, 2 * b) = best[b];
                            mx(qi, 2 * b + 1) = __int_as_float(bk[b]);
                        }
                    }
                    asm volatile("bar.sync 1, 256;" ::: "memory");
                    if (qi == 0) {
#pragma unroll
                        for (int b = 0; b < kNB; ++b) {
                            for (int qq = 1; qq < 4; ++qq) {
                                const float ob = mx(qq, 2 * b);
                                if (ob > best[b]) {
                                    best[b] = ob;
                                    bk[b] = __float_as_int(mx(qq, 2 * b + 1));
                                }
                            }
                            if (best[b] >= 0.f) best[b] = sqrtf(best[b]) * 16777216.0f;
                        }
                        write_out(best, bk, dir);
                    }
                } else {
                    // warps 0, 1 hold rows 0-63 (the first half of the chunk's
                    // bins), warps 2, 3 rows 64-127; per frequency group the
                    // second-half warps hand their sums over through shared memory
                    float best[kNB];
                    int bk[kNB];
                    band_init_t<kNB>(p.bands, klo, best, bk);
                    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
                    const int n_iss = p.n_iss;
                    const uint32_t cols_b = (uint32_t)(16 * p.gb);
                    const int dir = (warp & 1) * 32 + lane;
                    {
                        const int g0 = fg0;
                        const int nb = ng;
                        for (int j = 0; j < nb; ++j) {
                            float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
                            for (int i = 0; i < n_iss; ++i) {
                                const uint32_t dcol = lane_base + (uint32_t)i * cols_b;
                                float hi[8], lo[8];
                                tmem_ld8(dcol + (uint32_t)(8 * j), hi);
                                tmem_ld8(dcol + (uint32_t)(8 * nb + 8 * j), lo);
                                tmem_wait_ld();
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    re[q] += hi[2 * q] + lo[2 * q];
                                    im[q] += hi[2 * q + 1] + lo[2 * q + 1];
                                }
                            }
                            if (warp >= 2) {
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    EX[dir * 8 + 2 * q] = re[q];
                                    EX[dir * 8 + 2 * q + 1] = im[q];
                                }
                            }
                            asm volatile("bar.sync 1, 128;" ::: "memory");
                            if (warp < 2) {
#pragma unroll
                                for (int q = 0; q < 4; ++q) {
                                    const int f = p.kbase + 4 * (g0 + j) + q;
                                    // re = sum h cos, im = sum h sin over a half;
                                    // X = D_lo + w^(f h) D_hi with D = re - i im
                                    const float hr = EX[dir * 8 + 2 * q], hs = EX[dir * 8 + 2 * q + 1];
                                    float xr, xi;
                                    if (nchunk == 1) {
                                        const float sg = (f & 1) ? -1.f : 1.f;
                                        xr = re[q] + sg * hr;
                                        xi = im[q] + sg * hs;
                                    } else {
                                        float fs, fc;   // w^(f h) = fc - i fs, h = 512
                                        sincospif((float)f * (float)NBc / (float)NB, &fs, &fc);
                                        xr = re[q] + fc * hr - fs * hs;
                                        xi = im[q] + fs * hr + fc * hs;
                                    }
                                    band_update_t<kNB>(p.bands, klo, khi, f, sqrtf(xr * xr + xi * xi) * 16777216.0f,
                                                       best, bk);
                                }
                            }
                            asm volatile("bar.sync 1, 128;" ::: "memory");
                        }
                    }
                    if (warp < 2) write_out(best, bk, dir);
                }
                tc_fence_before();
                // the next tile's directions have landed (this thread's copies;
                // the barrier publishes them), H is zero and the accumulators
                // are read before the next pass or tile
                cp_async_wait_all();
                __syncthreads();
                tc_fence_after();
            }
        }
        if (failed) break;
    }
    // teardown: warp 0 frees the tensor memory
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(p.tmem_cols) : "memory");
    }
}

// ---- the global B operand: DFT matrix columns, fp16 hi + lo, K-major SW128 ----

// Chunk bc covers bins [bc nbc, bc nbc + nbc) with nbc = min(2^m, 1024); its K
// rows are the first half of those bins, n = bc nbc + kr, kr < nbc / 2.
// Layout [chunk][hi|lo][group][64-row K block] x 1 KB, 128-byte swizzle
// (narrow bands: a batch of groups is one contiguous run per part), or with
// `streamed` the first nbc / 4 rows only, [chunk][32-row K block][hi|lo][group]
// x 512 B, 64-byte swizzle, with ng + 1 groups per run, the last left as the
// caller's zeros (wide bands: one K block of one part over a run of groups is
// contiguous).
__global__ void k_build_twb(uint8_t* twb, int m, int kbase, int ng, bool streamed) {
    const int NB = 1 << m;
    const int NBc = NB < kChunkBins ? NB : kChunkBins;
    const int nchunk = NB / NBc;
    const int NK = streamed ? NBc / 4 : NBc / 2;
    const int KB = NBc / 128;
    const int64_t total = (int64_t)nchunk * 2 * ng * NK * 8;   // chunks x [hi|lo] x groups x K rows x 8 columns
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i & 7);
        const int64_t t = i >> 3;
        const int k = (int)(t % NK);
        const int64_t t2 = t / NK;
        const int g = (int)(t2 % ng);
        const int64_t t3 = t2 / ng;
        const int part = (int)(t3 % 2);   // 0 hi, 1 lo
        const int bc = (int)(t3 / 2);
        const int f = kbase + 4 * g + (r >> 1);
        const int64_t n = (int64_t)bc * NBc + k;
        const int jn = (int)(((int64_t)f * n) % NB);
        double sn, cs;
        sincospi(2.0 * (double)jn / (double)NB, &sn, &cs);
        const double v = (r & 1) ? sn : cs;
        const __half hi = __double2half(v);
        const __half lo = __double2half(v - (double)__half2float(hi));
        size_t off;
        if (streamed) {
            const int kb = k >> 5, kin = k & 31;
            const size_t blk = ((size_t)(bc * KB + kb) * 2 + part) * (ng + 1) + g;
            off = blk * 512 + (size_t)r * 64 + (size_t)(((kin >> 3) ^ ((r >> 1) & 3)) << 4) + (size_t)(kin & 7) * 2;
        } else {
            const int kb = k >> 6, kin = k & 63;
            const size_t blk = (size_t)((2 * bc + part) * ng + g) * KB + kb;
            off = blk * 1024 + (size_t)r * 128 + (size_t)(((kin >> 3) ^ r) << 4) + (size_t)(kin & 7) * 2;
        }
        *reinterpret_cast<__half*>(twb + off) = part ? lo : hi;
    }
}

}  // namespace

bool tc_supported(Ctx* c) {
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
    return major == 10 && minor == 3;
}

static size_t tc_smem_bytes(int m, int atom_cap, size_t bt_bytes) {
    const size_t nbc = std::min<size_t>((size_t)1 << m, kChunkBins);
    return 1024 + nbc * 128 + bt_bytes + kExBytes + (size_t)atom_cap * 16 + 2 * kDirs * 16 + 2 * kDirs * 8 +
           128 * 8 * 4 + 256;
}

// Build the B operand for the current ROI bands and pick the TMEM size.
int prepare_tc(Ctx* c) {
    if (!tc_supported(c)) return set_error(c, APTIDX_E_INVALID_ARG, "tensor-core path needs an sm_103 device");
    const int NB = 1 << c->m;
    const int NBc = std::min(NB, kChunkBins);
    const int nchunk = NB / NBc;
    const int KB = NBc / 128;   // 1 KB blocks of 64 K rows per chunk, K = NBc / 2
    const int kbase = c->band_min;
    const int ng = (c->band_max - kbase) / 4 + 1;
    const int gb = kBtBytes / (2 * KB * 1024);
    int ng_roi_max = 1;
    for (int64_t r = 0; r < c->nroi; ++r) {
        const int g0 = (c->h_band[2 * r] - kbase) >> 2, g1 = (c->h_band[2 * r + 1] - kbase) >> 2;
        ng_roi_max = std::max(ng_roi_max, g1 - g0 + 1);
    }
    // accumulators: kIssuers partials of 16 columns per group for bands that fit
    // one B batch; wider bands stream their twiddles and accumulate 8 columns per
    // group in each of two blocks (bin quarters 0 and 2, 1 and 3), all groups in
    // one MMA of N = 8 x groups <= 256 per block
    const bool wide = ng_roi_max > gb;
    if (wide && ng_roi_max > 32)
        return set_error(c, APTIDX_E_INVALID_ARG,
                         "tensor-core path: a ROI band spans %d frequency groups (4 frequencies each); at most 32",
                         ng_roi_max);
    // (wide: two blocks of 8 x groups columns, the second from a multiple of 32)
    const int wcols = 8 * ((ng_roi_max + 1) & ~1);
    const uint32_t need = (uint32_t)std::max(kIssuers * 16 * gb, wide ? ((wcols + 31) & ~31) + wcols : 0);
    uint32_t cols = 32;
    while (cols < need) cols <<= 1;
    if (c->twb_key[0] != c->m || c->twb_key[1] != kbase || c->twb_key[2] != ng) {
        dev_free(c->d_twb);
        c->d_twb = nullptr;
        c->twb_key[0] = c->twb_key[1] = c->twb_key[2] = -1;
        // both layouts of the same twiddles: [narrow | streamed (one zero group more per run)]
        const size_t bytes = (size_t)nchunk * 2 * ng * KB * 1024;
        const size_t sbytes = (size_t)nchunk * 2 * (ng + 1) * KB * 512;
        int rc = dev_alloc(c, &c->d_twb, bytes + sbytes);
        if (rc) return rc;
        cudaError_t e0 = cudaMemsetAsync((uint8_t*)c->d_twb + bytes, 0, sbytes, c->stream);
        if (e0 != cudaSuccess) return cuda_check(c, e0, "twiddle operand");
        for (int streamed = 0; streamed < 2; ++streamed) {
            k_build_twb<<<(unsigned)std::min<int64_t>(((int64_t)nchunk * ng * NBc * 8 + 255) / 256, 4096), 256, 0,
                          c->stream>>>((uint8_t*)c->d_twb + streamed * bytes, c->m, kbase, ng, streamed != 0);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_check(c, e, "twiddle operand");
            c->launches += 1;
        }
        c->twb_bytes = bytes;
        c->twb_key[0] = c->m;
        c->twb_key[1] = kbase;
        c->twb_key[2] = ng;
    }
    c->tc_gb = gb;
    c->tc_ng = ng;
    c->tc_tmem_cols = cols;
    c->tc_wide = wide;
    return APTIDX_OK;
}

cudaError_t launch_signatures_tc(Ctx* c, float* S, uint16_t* argk, uint16_t* hist_out, int64_t hist_roi) {
    cudaError_t e;
    static int max_optin = -1;
    if (max_optin < 0) cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    const size_t bt_bytes = c->tc_wide ? 4 * (size_t)kWideStage : (size_t)kBtBytes;
    const size_t base = tc_smem_bytes(c->m, 0, bt_bytes);
    int cap = (int)(((size_t)max_optin - base) / 16);
    cap = std::min(cap, kTcMaxAtoms) & ~15;
    if (cap < 256) return cudaErrorInvalidConfiguration;
    const size_t smem = tc_smem_bytes(c->m, cap, bt_bytes);
    const bool multi = !hist_out && c->multi.n > 0;
    // the wide-band stream lives in its own instances, so that the narrow-band
    // kernel compiles without it
    auto kern = multi ? (c->tc_wide ? k_sig_tc<APTIDX_MAX_BANDS, true> : k_sig_tc<APTIDX_MAX_BANDS, false>)
                      : (c->tc_wide ? k_sig_tc<1, true> : k_sig_tc<1, false>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    // antipodal pairs (one projection per pair) unless switched off or exporting
    const bool pairs = !hist_out && c->use_pairs && c->d_slot_idx;
    TcParams p;
    p.atoms = c->d_atoms;
    p.off = c->d_off;
    p.nw = c->d_nw;
    p.order = c->d_order;
    p.dirs = pairs ? c->d_slot_dirs : c->d_dirs;
    p.slot_idx = pairs ? c->d_slot_idx : nullptr;
    p.nv = c->nv;
    p.tiles_per_roi = (pairs ? c->nslot_pad : c->nv_pad) / kDirs;
    p.tiles_per_item = std::min(std::max(c->tune_tpi[1], 1), p.tiles_per_roi);
    p.items_per_roi = (p.tiles_per_roi + p.tiles_per_item - 1) / p.tiles_per_item;
    p.nroi = c->rank_limit > 0 ? std::min<int64_t>(c->nroi, c->rank_limit) : c->nroi;
    p.scale = c->d_scale;
    p.band = c->d_band;
    p.m = c->m;
    p.kbase = c->band_min;
    p.twb = (const uint8_t*)c->d_twb;
    p.twk = (const uint8_t*)c->d_twb + c->twb_bytes;
    p.bt_bytes = (int32_t)bt_bytes;
    p.ng_total = c->tc_ng;
    p.gb = c->tc_gb;
    p.tmem_cols = c->tc_tmem_cols;
    p.S = S;
    p.argk = argk;
    p.hist_out = hist_out;
    p.single_roi = hist_out ? hist_roi : -1;
    p.counter = c->d_counter + 2;
    p.status = c->d_status;
    p.atom_cap = cap;
    p.n_iss = std::min(std::max(c->tune_iss, 1), kIssuers);
    p.bands = hist_out ? BandSet() : c->multi;
    if ((e = cudaMemsetAsync(p.counter, 0, sizeof(int32_t), c->stream)) != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    per_sm = std::max(1, std::min(per_sm, (int)(512 / p.tmem_cols)));
    const int64_t items = (hist_out ? 1 : p.nroi) * (int64_t)p.items_per_roi;
    const int64_t grid = std::min<int64_t>((int64_t)c->sm_count * per_sm, items);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kThreads, smem, c->stream>>>(p);
    c->launches += hist_out ? 0 : 1;
    return cudaGetLastError();
}

}  // namespace aptidx
