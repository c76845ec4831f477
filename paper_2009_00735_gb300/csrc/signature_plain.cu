// signature_plain.cu -- steps (a2)-(a5) on CUDA cores, FP32: projection (Eq. 1
// dot product), binning into 2^m-bin histograms, the band of the DFT
// amplitude spectrum (Section 2.2), and the per-direction band maximum (the
// signature value, supplement "Al bicrystal").
//
// Work item = (ROI, group of 64-direction tiles).  A persistent grid claims
// items from a global counter, ROIs in longest-first order.  Per item the
// ROI's centred atoms are copied into shared memory once (bulk copy on the
// TMA engine).  Per tile every warp walks a strided subset of the atoms; lane
// l owns directions 2l and 2l+1 and adds 1 to 16-bit halves of the word
// H[b * 32 + l].  A lane's words sit in bank l whatever the bin, so the
// shared-memory atomics of one warp instruction never conflict.
// The band spectrum X(k) = sum_n h[n] e^{-2 pi i k n / 2^m} is then
// accumulated in FP32 against a (cos, sin) table; the twiddle index is
// uniform across a warp, so table reads are broadcasts.
#include <mutex>

#include "common.cuh"

namespace aptidx {

namespace {

constexpr int kWarps = 16;
constexpr int kThreads = kWarps * 32;
constexpr int kDirs = kTileDirs;        // 64 directions per tile
constexpr int kWords = kDirs / 2;       // u32 words per bin
constexpr int kKpw = 4;                 // frequencies per warp unit
constexpr int kPartBytes = kWarps * kKpw * kDirs * 8;
constexpr int kChunkBins = 1024;        // bins per histogram chunk (128 KB of words)
constexpr int kBlockAtoms = 65535;      // atoms per block: every 16-bit count of a block is exact

// Histograms of one tile for bin chunk bc over `cn` staged atoms (the
// multi-pass path: 2^m > 1024 bins, or a ROI above kBlockAtoms atoms): the bin
// is masked to m bits and only bins of [1024 bc, 1024 bc + 1024) are added,
// at row b - 1024 bc.
template <int W>
__device__ __forceinline__ void hist_tile_chunk(uint32_t* H, const float4* A, int cn, int warp, int lane, float4 d0,
                                                float4 d1, float scale, float magic, uint32_t nbm1, uint32_t bc) {
    const uint32_t hb = smem_u32(H) + 4u * (uint32_t)lane;
    for (int j = warp; j < cn; j += W) {
        const float4 a = A[j];
        const uint32_t b0 = __float_as_uint(__fmaf_rd(project_f32(d0.x, d0.y, d0.z, a), scale, magic)) & nbm1;
        const uint32_t b1 = __float_as_uint(__fmaf_rd(project_f32(d1.x, d1.y, d1.z, a), scale, magic)) & nbm1;
        if ((b0 >> 10) == bc)
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(hb + ((b0 & 1023u) << 7)), "r"(1u) : "memory");
        if ((b1 >> 10) == bc)
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(hb + ((b1 & 1023u) << 7)), "r"(0x10000u) : "memory");
    }
}

// Debug export of one pass: adds the counts of rows [0, nbc) to
// h_out[v * 2^m + bc * nbc + row] (the caller zeroes h_out).
__device__ __forceinline__ void hist_export_add_p(const uint32_t* H, int nbc, int NB, int bc, int tile, int nv,
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

struct SigParams {
    const float4* atoms;
    const int64_t* off;
    const int32_t* nw;
    const int32_t* order;
    const float4* dirs;
    int32_t nv;
    int32_t tiles_per_roi;
    int32_t tiles_per_item;
    int32_t items_per_roi;
    int64_t n_items;
    const float* scale;
    const int32_t* band;
    int m;
    const float2* tw;
    float* S;
    uint16_t* argk;
    uint16_t* hist_out;
    int64_t single_roi;
    int32_t* counter;
    int* status;
    int atom_cap;
    const int32_t* n_big;
    int rank_mode;
    int64_t nroi;
    BandSet bands;
};

// kNB: band slots of the epilogue (1: the ROI's own band; APTIDX_MAX_BANDS:
// the pass's BandSet)
template <int kNB>
__global__ void __launch_bounds__(kThreads, 1) k_sig_plain(SigParams p) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int NB = 1 << p.m;
    const int nbm1 = NB - 1;
    const int NBc = NB < kChunkBins ? NB : kChunkBins;   // histogram rows held at once
    const int nchunk = NB / NBc;
    uint32_t* H = reinterpret_cast<uint32_t*>(smem);
    float2* TW = reinterpret_cast<float2*>(smem + (size_t)NBc * kWords * 4);
    float4* A = reinterpret_cast<float4*>(smem + (size_t)NBc * kWords * 4 + (size_t)NB * 8);
    float2* PART = reinterpret_cast<float2*>(A + p.atom_cap);
    uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(PART) + kPartBytes);
    int* flag = reinterpret_cast<int*>(bar + 1);
    int64_t* item_s = reinterpret_cast<int64_t*>(bar + 2);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int j = tid; j < NB; j += kThreads) TW[j] = p.tw[j];
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const float magic = bin_magic(p.m);
    int64_t rank_lo = 0, n_items = p.n_items;
    if (p.single_roi < 0 && p.rank_mode != kRanksAll) {
        const int64_t nb = *p.n_big;
        rank_lo = p.rank_mode == kRanksBig ? 0 : nb;
        const int64_t rank_hi = p.rank_mode == kRanksBig ? nb : p.nroi;
        n_items = (rank_hi - rank_lo) * p.items_per_roi;
    }

    for (;;) {
        if (tid == 0) *item_s = atomicAdd(p.counter, 1);
        __syncthreads();
        const int64_t item = *item_s;
        __syncthreads();
        if (item >= n_items) break;
        const int64_t roi_rank = rank_lo + item / p.items_per_roi;
        const int grp = (int)(item % p.items_per_roi);
        const int64_t roi = p.single_roi >= 0 ? p.single_roi : (int64_t)p.order[roi_rank];
        const int nw = p.nw[roi];
        const int64_t abase = p.off[roi];
        const float scale = p.scale[roi];
        const int klo = p.band[2 * roi], khi = p.band[2 * roi + 1];
        const int t0 = grp * p.tiles_per_item;
        const int t1 = min(t0 + p.tiles_per_item, p.tiles_per_roi);
        const bool one_chunk = nw <= p.atom_cap;
        if (one_chunk && !stage_atoms(A, p.atoms + abase, nw, bar, phase, p.status, flag)) return;

        if (nchunk > 1 || nw > kBlockAtoms) {
            // ---- multi-pass path: the histogram of a tile in passes over atom
            // blocks of at most kBlockAtoms and bin chunks of 1024; each warp
            // unit (4 frequencies x a span of the chunk's bins) accumulates its
            // partial DFT in registers across the passes.  Bands of more than
            // kWarps groups of frequencies run in rounds of kWarps groups.
            const int K = khi - klo + 1;
            const int G = (K + kKpw - 1) / kKpw;
            const int nblk = (nw + kBlockAtoms - 1) / kBlockAtoms;
            const int64_t out_base = (p.single_roi >= 0 ? 0 : roi) * (int64_t)p.nv;
            for (int tile = t0; tile < t1; ++tile) {
                const float4 d0 = p.dirs[(int64_t)tile * kDirs + 2 * lane];
                const float4 d1 = p.dirs[(int64_t)tile * kDirs + 2 * lane + 1];
                float best[kNB];
                int bk[kNB];
                if (tid < kDirs) band_init_t<kNB>(p.bands, klo, best, bk);
                for (int g_lo = 0; g_lo < G; g_lo += kWarps) {
                    const int Gr = min(kWarps, G - g_lo);
                    int nsplit = 1;
                    while (Gr * nsplit * 2 <= kWarps && nsplit * 2 <= NBc / 32) nsplit *= 2;
                    const int span = NBc / nsplit;
                    const bool unit = warp < Gr * nsplit;
                    const int g = g_lo + warp / nsplit, sp = warp % nsplit;
                    const int k0 = klo + g * kKpw;
                    float re[kKpw][2], im[kKpw][2];
#pragma unroll
                    for (int q = 0; q < kKpw; ++q) re[q][0] = re[q][1] = im[q][0] = im[q][1] = 0.f;
                    for (int blk = 0; blk < max(nblk, 1); ++blk) {
                        const int b0 = blk * kBlockAtoms, bn = max(0, min(kBlockAtoms, nw - b0));
                        for (int bc = 0; bc < nchunk; ++bc) {
                            uint4* H4 = reinterpret_cast<uint4*>(H);
                            for (int i = tid; i < NBc * kWords / 4; i += kThreads) H4[i] = make_uint4(0, 0, 0, 0);
                            __syncthreads();
                            for (int c0 = 0; c0 < bn; c0 += p.atom_cap) {
                                const int cn = min(p.atom_cap, bn - c0);
                                if (!one_chunk) {
                                    if (!stage_atoms(A, p.atoms + abase + b0 + c0, cn, bar, phase, p.status, flag))
                                        return;
                                }
                                hist_tile_chunk<kWarps>(H, A, cn, warp, lane, d0, d1, scale, magic, (uint32_t)nbm1,
                                                        (uint32_t)bc);
                                if (!one_chunk) __syncthreads();
                            }
                            __syncthreads();
                            if (p.hist_out && g_lo == 0) {
                                hist_export_add_p(H, NBc, NB, bc, tile, p.nv, p.hist_out, tid, kThreads);
                                __syncthreads();
                            }
                            if (unit) {
                                const int n0 = bc * NBc + sp * span;
                                unsigned idx[kKpw];
#pragma unroll
                                for (int q = 0; q < kKpw; ++q)
                                    idx[q] = (unsigned)(((int64_t)(k0 + q) * n0) & (int64_t)nbm1);
                                for (int n = 0; n < span; ++n) {
                                    const uint32_t w = H[(sp * span + n) * kWords + lane];
                                    const float f0 = u23_to_float(w & 0xFFFFu), f1 = u23_to_float(w >> 16);
#pragma unroll
                                    for (int q = 0; q < kKpw; ++q) {
                                        const float2 t = TW[idx[q]];
                                        re[q][0] = fmaf(f0, t.x, re[q][0]);
                                        im[q][0] = fmaf(f0, t.y, im[q][0]);
                                        re[q][1] = fmaf(f1, t.x, re[q][1]);
                                        im[q][1] = fmaf(f1, t.y, im[q][1]);
                                        idx[q] = (idx[q] + (unsigned)(k0 + q)) & (unsigned)nbm1;
                                    }
                                }
                            }
                            __syncthreads();   // H is read before the next pass zeroes it
                        }
                    }
                    if (unit) {
#pragma unroll
                        for (int q = 0; q < kKpw; ++q) {
                            PART[((size_t)warp * kKpw + q) * kDirs + 2 * lane] = make_float2(re[q][0], im[q][0]);
                            PART[((size_t)warp * kKpw + q) * kDirs + 2 * lane + 1] = make_float2(re[q][1], im[q][1]);
                        }
                    }
                    __syncthreads();
                    if (tid < kDirs) {
                        for (int kk = g_lo * kKpw; kk < min(K, (g_lo + Gr) * kKpw); ++kk) {
                            const int gg = kk / kKpw - g_lo, q = kk % kKpw;
                            float sr = 0.f, si = 0.f;
                            for (int s2 = 0; s2 < nsplit; ++s2) {
                                const float2 t = PART[((size_t)(gg * nsplit + s2) * kKpw + q) * kDirs + tid];
                                sr += t.x;
                                si += t.y;
                            }
                            band_update_t<kNB>(p.bands, klo, khi, klo + kk, sqrtf(sr * sr + si * si), best, bk);
                        }
                    }
                    __syncthreads();
                }
                if (tid < kDirs) {
                    const int64_t v = (int64_t)tile * kDirs + tid;
                    if (v < p.nv) {
#pragma unroll
                        for (int b = 0; b < kNB; ++b) {
                            if (b < band_count_t<kNB>(p.bands)) {
                                p.S[band_off_t<kNB>(p.bands, b) + out_base + v] = best[b];
                                if (p.argk) p.argk[band_off_t<kNB>(p.bands, b) + out_base + v] = (uint16_t)bk[b];
                            }
                        }
                    }
                }
            }
            continue;
        }

        for (int tile = t0; tile < t1; ++tile) {
            uint4* H4 = reinterpret_cast<uint4*>(H);
            for (int i = tid; i < NB * kWords / 4; i += kThreads) H4[i] = make_uint4(0, 0, 0, 0);
            const float4 d0 = p.dirs[(int64_t)tile * kDirs + 2 * lane];
            const float4 d1 = p.dirs[(int64_t)tile * kDirs + 2 * lane + 1];
            __syncthreads();
            for (int c0 = 0; c0 < nw; c0 += p.atom_cap) {
                const int cn = min(p.atom_cap, nw - c0);
                if (!one_chunk && !stage_atoms(A, p.atoms + abase + c0, cn, bar, phase, p.status, flag)) return;
                hist_tile<kWarps, true>(H, A, cn, warp, lane, d0, d1, scale, magic, nbm1);
                if (!one_chunk) __syncthreads();
            }
            __syncthreads();

            if (p.hist_out) hist_export_add_p(H, NB, NB, 0, tile, p.nv, p.hist_out, tid, kThreads);

            // ---- band spectrum (FP32) and band maximum ----
            const int K = khi - klo + 1;
            const int G = (K + kKpw - 1) / kKpw;   // frequency groups of kKpw
            const int64_t out_base = (p.single_roi >= 0 ? 0 : roi) * (int64_t)p.nv + (int64_t)tile * kDirs;
            if (G <= kWarps) {
                int nsplit = 1;
                while (G * nsplit * 2 <= kWarps && nsplit * 2 <= NB / 32) nsplit *= 2;
                const int span = NB / nsplit;
                const int units = G * nsplit;
                if (warp < units) {
                    const int g = warp / nsplit, sp = warp % nsplit;
                    const int k0 = klo + g * kKpw;
                    float re[kKpw][2], im[kKpw][2];
                    unsigned idx[kKpw];
                    const int n0 = sp * span;
#pragma unroll
                    for (int q = 0; q < kKpw; ++q) {
                        re[q][0] = re[q][1] = im[q][0] = im[q][1] = 0.f;
                        idx[q] = (unsigned)((k0 + q) * n0) & (unsigned)nbm1;
                    }
                    for (int n = n0; n < n0 + span; ++n) {
                        const uint32_t w = H[n * kWords + lane];
                        const float f0 = u23_to_float(w & 0xFFFFu), f1 = u23_to_float(w >> 16);
#pragma unroll
                        for (int q = 0; q < kKpw; ++q) {
                            const float2 t = TW[idx[q]];
                            re[q][0] = fmaf(f0, t.x, re[q][0]);
                            im[q][0] = fmaf(f0, t.y, im[q][0]);
                            re[q][1] = fmaf(f1, t.x, re[q][1]);
                            im[q][1] = fmaf(f1, t.y, im[q][1]);
                            idx[q] = (idx[q] + (unsigned)(k0 + q)) & (unsigned)nbm1;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kKpw; ++q) {
                        PART[((size_t)warp * kKpw + q) * kDirs + 2 * lane] = make_float2(re[q][0], im[q][0]);
                        PART[((size_t)warp * kKpw + q) * kDirs + 2 * lane + 1] = make_float2(re[q][1], im[q][1]);
                    }
                }
                __syncthreads();
                if (tid < kDirs) {
                    const int64_t v = (int64_t)tile * kDirs + tid;
                    float best[kNB];
                    int bk[kNB];
                    band_init_t<kNB>(p.bands, klo, best, bk);
                    for (int kk = 0; kk < K; ++kk) {
                        const int g = kk / kKpw, q = kk % kKpw;
                        float sr = 0.f, si = 0.f;
                        for (int sp = 0; sp < nsplit; ++sp) {
                            const float2 t = PART[((size_t)(g * nsplit + sp) * kKpw + q) * kDirs + tid];
                            sr += t.x;
                            si += t.y;
                        }
                        band_update_t<kNB>(p.bands, klo, khi, klo + kk, sqrtf(sr * sr + si * si), best, bk);
                    }
                    if (v < p.nv) {
#pragma unroll
                        for (int b = 0; b < kNB; ++b) {
                            if (b < band_count_t<kNB>(p.bands)) {
                                p.S[band_off_t<kNB>(p.bands, b) + out_base + tid] = best[b];
                                if (p.argk) p.argk[band_off_t<kNB>(p.bands, b) + out_base + tid] = (uint16_t)bk[b];
                            }
                        }
                    }
                }
            } else {
                float b0[kNB], b1[kNB];
                int bk0[kNB], bk1[kNB];
                band_init_t<kNB>(p.bands, klo, b0, bk0);
                band_init_t<kNB>(p.bands, klo, b1, bk1);
                for (int g = warp; g < G; g += kWarps) {
                    const int k0 = klo + g * kKpw;
                    float re[kKpw][2], im[kKpw][2];
                    unsigned idx[kKpw];
#pragma unroll
                    for (int q = 0; q < kKpw; ++q) {
                        re[q][0] = re[q][1] = im[q][0] = im[q][1] = 0.f;
                        idx[q] = 0;
                    }
                    for (int n = 0; n < NB; ++n) {
                        const uint32_t w = H[n * kWords + lane];
                        const float f0 = u23_to_float(w & 0xFFFFu), f1 = u23_to_float(w >> 16);
#pragma unroll
                        for (int q = 0; q < kKpw; ++q) {
                            const float2 t = TW[idx[q]];
                            re[q][0] = fmaf(f0, t.x, re[q][0]);
                            im[q][0] = fmaf(f0, t.y, im[q][0]);
                            re[q][1] = fmaf(f1, t.x, re[q][1]);
                            im[q][1] = fmaf(f1, t.y, im[q][1]);
                            idx[q] = (idx[q] + (unsigned)(k0 + q)) & (unsigned)nbm1;
                        }
                    }
#pragma unroll
                    for (int q = 0; q < kKpw; ++q) {
                        if (k0 + q > khi) break;
                        const float a0 = sqrtf(re[q][0] * re[q][0] + im[q][0] * im[q][0]);
                        const float a1 = sqrtf(re[q][1] * re[q][1] + im[q][1] * im[q][1]);
                        band_update_t<kNB>(p.bands, klo, khi, k0 + q, a0, b0, bk0);
                        band_update_t<kNB>(p.bands, klo, khi, k0 + q, a1, b1, bk1);
                    }
                }
                // per band, each warp's best over its frequency groups; the
                // band's slab of PART holds kWarps x kDirs (value, k) pairs
#pragma unroll
                for (int b = 0; b < kNB; ++b) {
                    if (b < band_count_t<kNB>(p.bands)) {
                        PART[((size_t)b * kWarps + warp) * kDirs + 2 * lane] = make_float2(b0[b], __int_as_float(bk0[b]));
                        PART[((size_t)b * kWarps + warp) * kDirs + 2 * lane + 1] =
                            make_float2(b1[b], __int_as_float(bk1[b]));
                    }
                }
                __syncthreads();
                if (tid < kDirs) {
                    const int64_t v = (int64_t)tile * kDirs + tid;
                    for (int b = 0; b < band_count_t<kNB>(p.bands); ++b) {
                        float best = -1.f;
                        int bk = kNB == 1 ? klo : p.bands.lo[b];
                        for (int w = 0; w < kWarps; ++w) {
                            const float2 t = PART[((size_t)b * kWarps + w) * kDirs + tid];
                            const int k = __float_as_int(t.y);
                            if (t.x > best || (t.x == best && k < bk)) {
                                best = t.x;
                                bk = k;
                            }
                        }
                        if (v < p.nv) {
                            p.S[band_off_t<kNB>(p.bands, b) + out_base + tid] = best;
                            if (p.argk) p.argk[band_off_t<kNB>(p.bands, b) + out_base + tid] = (uint16_t)bk;
                        }
                    }
                }
            }
            __syncthreads();
        }
    }
}

// per-ROI normalisation (supplement "Indexing algorithm", step 1): S / max_v S
__global__ void __launch_bounds__(256) k_normalise(float* S, int32_t nv) {
    __shared__ float red[8];
    float* row = S + (int64_t)blockIdx.x * nv;
    float mx = 0.f;
    for (int v = threadIdx.x; v < nv; v += 256) mx = fmaxf(mx, row[v]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
    const float inv = mx > 0.f ? 1.0f / mx : 0.f;
    for (int v = threadIdx.x; v < nv; v += 256) row[v] = mx > 0.f ? row[v] * inv : 0.f;
}

}  // namespace

cudaError_t launch_normalise(Ctx* c, float* S, int64_t rows) {
    if (rows < 0) rows = c->nroi;
    if (rows <= 0) return cudaSuccess;
    k_normalise<<<(unsigned)rows, 256, 0, c->stream>>>(S, c->nv);
    return cudaGetLastError();
}

size_t plain_smem_bytes(int m, int atom_cap) {
    const size_t NB = (size_t)1 << m;
    const size_t NBc = NB < (size_t)kChunkBins ? NB : (size_t)kChunkBins;
    return NBc * kWords * 4 + NB * 8 + (size_t)atom_cap * 16 + kPartBytes + 64;
}

cudaError_t launch_signatures_plain(Ctx* c, float* S, uint16_t* argk, uint16_t* hist_out, int64_t hist_roi,
                                    int rank_mode) {
    static int max_optin = -1;
    if (max_optin < 0) {
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    }
    const size_t base = plain_smem_bytes(c->m, 0);
    int cap = (int)(((size_t)max_optin - base) / 16);
    cap = min(cap, 4096) & ~15;
    if (cap < 256) return cudaErrorInvalidConfiguration;
    const size_t smem = plain_smem_bytes(c->m, cap);
    const bool multi = !hist_out && c->multi.n > 0;
    auto kern = multi ? k_sig_plain<APTIDX_MAX_BANDS> : k_sig_plain<1>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;

    SigParams p;
    p.atoms = c->d_atoms;
    p.off = c->d_off;
    p.nw = c->d_nw;
    p.order = c->d_order;
    p.dirs = c->d_dirs;
    p.nv = c->nv;
    p.tiles_per_roi = c->nv_pad / kDirs;
    p.tiles_per_item = min(max(c->tune_tpi[0], 1), p.tiles_per_roi);
    p.items_per_roi = (p.tiles_per_roi + p.tiles_per_item - 1) / p.tiles_per_item;
    const int64_t nroi_lim = c->rank_limit > 0 ? tmin<int64_t>(c->nroi, c->rank_limit) : c->nroi;
    const int64_t nroi_eff = hist_out ? 1 : nroi_lim;
    p.n_items = nroi_eff * p.items_per_roi;
    p.scale = c->d_scale;
    p.band = c->d_band;
    p.m = c->m;
    p.tw = c->d_tw;
    p.S = S;
    p.argk = argk;
    p.hist_out = hist_out;
    p.single_roi = hist_out ? hist_roi : -1;
    p.counter = c->d_counter;
    p.status = c->d_status;
    p.atom_cap = cap;
    p.n_big = c->d_counter + 1;
    p.rank_mode = hist_out ? kRanksAll : rank_mode;
    p.nroi = nroi_lim;
    p.bands = hist_out ? BandSet() : c->multi;
    if ((e = cudaMemsetAsync(c->d_counter, 0, sizeof(int32_t), c->stream)) != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    per_sm = max(per_sm, 1);
    int64_t grid = tmin<int64_t>((int64_t)c->sm_count * per_sm, p.n_items);
    if (rank_mode == kRanksBig && !hist_out) grid = tmin<int64_t>(grid, (int64_t)c->sm_count);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kThreads, smem, c->stream>>>(p);
    return cudaGetLastError();
}

// -----------------------------------------------------------------------------
// No-allocation variant (aptidx_signatures_noalloc).  Everything a call derives
// from its inputs -- padded directions, per-ROI scale, band, atom count and
// order, the twiddle table, the work counter -- lives in one fixed scratch
// array in device memory, so the call allocates nothing.  Every GPU that loads
// the library holds the array until the process exits; all calls share it.
// -----------------------------------------------------------------------------
namespace {

constexpr int64_t kNaMaxRoi = APTIDX_NOALLOC_MAX_ROIS;
constexpr int64_t kNaMaxDirs = APTIDX_NOALLOC_MAX_DIRS;
// byte offsets inside the scratch array
constexpr size_t kNaDirs = 0;                                        // float4 [kNaMaxDirs]
constexpr size_t kNaTw = kNaDirs + 16 * (size_t)kNaMaxDirs;          // float2 [2^APTIDX_MAX_M]
constexpr size_t kNaScale = kNaTw + 8 * ((size_t)1 << APTIDX_MAX_M);  // float  [kNaMaxRoi]
constexpr size_t kNaBand = kNaScale + 4 * (size_t)kNaMaxRoi;         // int32  [2 kNaMaxRoi]
constexpr size_t kNaNw = kNaBand + 8 * (size_t)kNaMaxRoi;            // int32  [kNaMaxRoi]
constexpr size_t kNaOrder = kNaNw + 4 * (size_t)kNaMaxRoi;           // int32  [kNaMaxRoi]
constexpr size_t kNaCounter = kNaOrder + 4 * (size_t)kNaMaxRoi;      // int32  [4]
constexpr size_t kNaStatus = kNaCounter + 16;                        // int    [1]
constexpr size_t kNaEnd = kNaStatus + 16;
static_assert(kNaEnd <= APTIDX_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[APTIDX_NOALLOC_SCRATCH_BYTES];

// Per-call set-up: counts, scales, bands and identity order per ROI; padded
// float4 directions; the twiddle table.  Flags ROIs above 65535 atoms
// (overflow), radii outside [1e-6, 1e6] nm and directions that are not unit
// vectors (invalid input); a flagged ROI gets zero atoms, so its row of S is
// zero.
__global__ void k_noalloc_setup(unsigned char* scr, const int64_t* __restrict__ off, const double* __restrict__ radii,
                                int64_t nroi, const float* __restrict__ u, int32_t nv, int32_t nv_pad, int m,
                                int32_t k_lo, int32_t k_hi, int* status) {
    float4* dirs = reinterpret_cast<float4*>(scr + kNaDirs);
    float2* tw = reinterpret_cast<float2*>(scr + kNaTw);
    float* scale = reinterpret_cast<float*>(scr + kNaScale);
    int32_t* band = reinterpret_cast<int32_t*>(scr + kNaBand);
    int32_t* nw = reinterpret_cast<int32_t*>(scr + kNaNw);
    int32_t* order = reinterpret_cast<int32_t*>(scr + kNaOrder);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int half = 1 << (m - 1);
    for (int64_t r = t0; r < nroi; r += stride) {
        int64_t n = off[r + 1] - off[r];
        if (n < 0 || n > APTIDX_MAX_ATOMS_PER_ROI) {
            atomicOr(status, kStatusOverflow);
            n = 0;
        }
        const double R = radii[r];
        if (!(R >= 1e-6 && R <= 1e6)) {   // also false for NaN
            atomicOr(status, kStatusInvalid);
            n = 0;
        }
        nw[r] = (int32_t)n;
        scale[r] = n > 0 ? __double2float_rn((double)(half - 1) / R) : 0.f;
        band[2 * r] = k_lo;
        band[2 * r + 1] = k_hi;
        order[r] = (int32_t)r;
    }
    for (int64_t v = t0; v < nv_pad; v += stride) {
        float4 d = make_float4(1.f, 0.f, 0.f, 0.f);
        if (v < nv) {
            d = make_float4(u[3 * v], u[3 * v + 1], u[3 * v + 2], 0.f);
            const double n2 = (double)d.x * d.x + (double)d.y * d.y + (double)d.z * d.z;
            if (!(fabs(sqrt(n2) - 1.0) <= 1e-5)) atomicOr(status, kStatusInvalid);
        }
        dirs[v] = d;
    }
    for (int64_t j = t0; j < (int64_t)(1 << m); j += stride) {
        double sn, cs;
        sincospi(2.0 * (double)j / (double)(1 << m), &sn, &cs);
        tw[j] = make_float2((float)cs, (float)sn);
    }
}

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

}  // namespace

}  // namespace aptidx

extern "C" int aptidx_signatures_noalloc(const float* xc4, const int64_t* off, const double* radii, int64_t nroi,
                                         const float* u, int32_t nv, int m, int32_t k_lo, int32_t k_hi, float* S,
                                         int* status, void* cuda_stream) {
    using namespace aptidx;
    if (nroi < 0 || nroi > kNaMaxRoi || nv <= 0 || nv > kNaMaxDirs) return APTIDX_E_INVALID_ARG;
    if (m < APTIDX_MIN_M || m > APTIDX_MAX_M) return APTIDX_E_INVALID_ARG;
    if (k_lo < 0 || k_hi < k_lo || k_hi > (1 << (m - 1))) return APTIDX_E_INVALID_ARG;
    if (nroi == 0) return APTIDX_OK;
    if (!xc4 || !off || !radii || !u || !S) return APTIDX_E_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(xc4) & 15u) != 0) return APTIDX_E_INVALID_ARG;   // bulk copies need 16-byte rows
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return APTIDX_E_CUDA;
    }
    void* scr = nullptr;
    {
        // set-up, once per device, with that device current: the host-side
        // name of the array is not a device address
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return APTIDX_E_CUDA;
            }
            g_noalloc_ptr[dev] = ptr;
        }
        scr = g_noalloc_ptr[dev];
    }
    unsigned char* base = static_cast<unsigned char*>(scr);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int* st = status ? status : reinterpret_cast<int*>(base + kNaStatus);
    int32_t* counter = reinterpret_cast<int32_t*>(base + kNaCounter);
    const int32_t nv_pad = (nv + kTileDirs - 1) / kTileDirs * kTileDirs;
    int sm_count = 0, max_optin = 0;
    if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return APTIDX_E_CUDA;
    }
    // the work counter must start at zero; the rest is rewritten by the set-up kernel
    if (cudaMemsetAsync(counter, 0, 16, s) != cudaSuccess) return APTIDX_E_CUDA;
    const int64_t work = std::max<int64_t>(nroi, (int64_t)nv_pad);
    k_noalloc_setup<<<(unsigned)std::min<int64_t>((work + 255) / 256, 1024), 256, 0, s>>>(base, off, radii, nroi, u, nv,
                                                                                       nv_pad, m, k_lo, k_hi, st);
    if (cudaGetLastError() != cudaSuccess) return APTIDX_E_CUDA;
    const size_t smem_base = plain_smem_bytes(m, 0);
    int cap = (int)(((size_t)max_optin - smem_base) / 16);
    cap = std::min(cap, 4096) & ~15;
    if (cap < 256) return APTIDX_E_CUDA;
    const size_t smem = plain_smem_bytes(m, cap);
    if (cudaFuncSetAttribute(k_sig_plain<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return APTIDX_E_CUDA;
    }
    SigParams p;
    p.atoms = reinterpret_cast<const float4*>(xc4);
    p.off = off;
    p.nw = reinterpret_cast<const int32_t*>(base + kNaNw);
    p.order = reinterpret_cast<const int32_t*>(base + kNaOrder);
    p.dirs = reinterpret_cast<const float4*>(base + kNaDirs);
    p.nv = nv;
    p.tiles_per_roi = nv_pad / kDirs;
    p.tiles_per_item = std::min(16, p.tiles_per_roi);
    p.items_per_roi = (p.tiles_per_roi + p.tiles_per_item - 1) / p.tiles_per_item;
    p.n_items = nroi * p.items_per_roi;
    p.scale = reinterpret_cast<const float*>(base + kNaScale);
    p.band = reinterpret_cast<const int32_t*>(base + kNaBand);
    p.m = m;
    p.tw = reinterpret_cast<const float2*>(base + kNaTw);
    p.S = S;
    p.argk = nullptr;
    p.hist_out = nullptr;
    p.single_roi = -1;
    p.counter = counter;
    p.status = st;
    p.atom_cap = cap;
    p.n_big = counter + 1;
    p.rank_mode = kRanksAll;
    p.nroi = nroi;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sig_plain<1>, kThreads, smem);
    per_sm = std::max(per_sm, 1);
    const int64_t grid = std::min<int64_t>((int64_t)sm_count * per_sm, p.n_items);
    k_sig_plain<1><<<(unsigned)grid, kThreads, smem, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? APTIDX_OK : APTIDX_E_CUDA;
}
