// common.cuh -- device helpers shared by the aptidx kernels: the binning
// contract of Eq. 1, bounded mbarrier waits, bulk (TMA) copies.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace aptidx {

template <typename T>
__host__ __device__ __forceinline__ T tmin(T a, T b) { return a < b ? a : b; }
template <typename T>
__host__ __device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// -----------------------------------------------------------------------------
// Eq. 1, the bin of a projected atom.  With dR = R / (2^(m-1) - 1) (Fig. 2
// caption) Eq. 1 is b = floor(2^(m-1) + s (2^(m-1) - 1) / R).  The library
// evaluates s in FP32 with a fixed fma order and takes the floor of the exact
// product s * scale: one fma rounding toward -inf onto the integer grid of
// [2^23, 2^24), whose bit pattern is 0x4B000000 + integer part.
// -----------------------------------------------------------------------------
__device__ __forceinline__ float project_f32(float ux, float uy, float uz, float4 a) {
    return __fmaf_rn(uz, a.z, __fmaf_rn(uy, a.y, __fmul_rn(ux, a.x)));
}

// magic = 2^23 + 2^(m-1) as float
__host__ __device__ __forceinline__ float bin_magic(int m) {
    return 8388608.0f + (float)(1 << (m - 1));
}

__device__ __forceinline__ int bin_of(float s, float scale, float magic, int nb_minus_1) {
    int b = __float_as_int(__fmaf_rd(s, scale, magic)) - 0x4B000000;
    return min(max(b, 0), nb_minus_1);
}

// The same bin without the clamp, for the histogram loops.  For inputs the
// library accepts (|u| within 1e-5 of 1, |x| <= R by the FP64 membership
// test, m <= 10) |s * scale| < 2^(m-1) - 1 + 0.01, so the exact bin lies in
// [0, 2^m - 1] and the clamp of the contract never acts; the fma result is
// then 2^23 + b exactly and its low m bits are b.  The mask keeps every
// shared-memory index in range whatever the input.
__device__ __forceinline__ uint32_t bin_of_valid(float s, float scale, float magic, uint32_t nb_minus_1) {
    return __float_as_uint(__fmaf_rd(s, scale, magic)) & nb_minus_1;
}

// exact small non-negative integer (< 2^23) to float with one integer op and
// one FP32 add (no conversion-pipe instruction)
__device__ __forceinline__ float u23_to_float(uint32_t c) {
    return __int_as_float(0x4B000000 | c) - 8388608.0f;
}

// One atom into the histograms of a 64-direction tile: lane l owns
// directions 2l (low 16 bits) and 2l + 1 (high 16 bits) of the word
// H[b * 32 + l].  The word of a lane lies in bank l for every bin b, so the
// 32 atomics of one warp instruction never share a bank.  `hbase` is the
// shared address of H plus 4 * lane.
//   kMasked: the bin is masked to m bits (memory-safe for any input).
//   otherwise: the inputs are known to give bins in range (the library's own
//   gather and validated directions and radii), and the word address is one
//   multiply-add of the fma result's bit pattern 0x4B000000 + b.
template <bool kMasked>
__device__ __forceinline__ void hist_add_atom(uint32_t hbase, float4 a, float4 d0, float4 d1, float scale,
                                              float magic, int nbm1) {
    const float s0 = project_f32(d0.x, d0.y, d0.z, a);
    const float s1 = project_f32(d1.x, d1.y, d1.z, a);
    const uint32_t t0 = __float_as_uint(__fmaf_rd(s0, scale, magic));
    const uint32_t t1 = __float_as_uint(__fmaf_rd(s1, scale, magic));
    uint32_t w0, w1;
    if (kMasked) {
        w0 = hbase + ((t0 & (uint32_t)nbm1) << 7);
        w1 = hbase + ((t1 & (uint32_t)nbm1) << 7);
    } else {
        // (t - 0x4B000000) * 128 + hbase, in wrapping 32-bit arithmetic
        w0 = t0 * 128u + (hbase - 0x80000000u);
        w1 = t1 * 128u + (hbase - 0x80000000u);
    }
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(w0), "r"(1u) : "memory");
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(w1), "r"(0x10000u) : "memory");
}

// Histograms of one 64-direction tile over `cn` staged atoms; warp w takes
// atoms w, w + W, w + 2W, ...
template <int W, bool kMasked>
__device__ __forceinline__ void hist_tile(uint32_t* H, const float4* A, int cn, int warp, int lane, float4 d0,
                                          float4 d1, float scale, float magic, int nbm1) {
    const uint32_t hbase = smem_u32(H) + 4u * (uint32_t)lane;
    int j = warp;
    if (j + 3 * W < cn) {
        // groups of four atoms, the next group's loads issued before the
        // current group's increments
        float4 a0 = A[j], a1 = A[j + W], a2 = A[j + 2 * W], a3 = A[j + 3 * W];
        for (; j + 7 * W < cn; j += 4 * W) {
            const float4 b0 = A[j + 4 * W], b1 = A[j + 5 * W], b2 = A[j + 6 * W], b3 = A[j + 7 * W];
            hist_add_atom<kMasked>(hbase, a0, d0, d1, scale, magic, nbm1);
            hist_add_atom<kMasked>(hbase, a1, d0, d1, scale, magic, nbm1);
            hist_add_atom<kMasked>(hbase, a2, d0, d1, scale, magic, nbm1);
            hist_add_atom<kMasked>(hbase, a3, d0, d1, scale, magic, nbm1);
            a0 = b0;
            a1 = b1;
            a2 = b2;
            a3 = b3;
        }
        hist_add_atom<kMasked>(hbase, a0, d0, d1, scale, magic, nbm1);
        hist_add_atom<kMasked>(hbase, a1, d0, d1, scale, magic, nbm1);
        hist_add_atom<kMasked>(hbase, a2, d0, d1, scale, magic, nbm1);
        hist_add_atom<kMasked>(hbase, a3, d0, d1, scale, magic, nbm1);
        j += 4 * W;
    }
    for (; j < cn; j += W) hist_add_atom<kMasked>(hbase, A[j], d0, d1, scale, magic, nbm1);
}

// Packed FP32 pairs (f32x2): each half is one IEEE FP32 operation with the
// stated rounding, so a pair gives bit for bit the two scalar results.
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma_rd(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_fma_ru(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t d;
    asm("fma.rp.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ float f2_lo(uint64_t x) { return __uint_as_float((uint32_t)x); }
__device__ __forceinline__ float f2_hi(uint64_t x) { return __uint_as_float((uint32_t)(x >> 32)); }
__device__ __forceinline__ uint64_t f2_dup(float v) {
    return ((uint64_t)__float_as_uint(v) << 32) | (uint64_t)__float_as_uint(v);
}

// Rearranges staged atoms in place for the paired histogram loop: the
// 32-byte block of atoms 2p, 2p + 1 becomes (x_a, x_b, y_a, y_b | z_a, z_b,
// w_a, w_b), so that one 16-byte and one 8-byte load give the coordinates
// of both atoms as FP32 pairs.  A trailing odd atom keeps its layout.  With
// r2max, the largest x^2 + y^2 + z^2 (FP32) of the atoms goes to *r2max by
// atomicMax on its bit pattern (the caller zeroes it).
__device__ __forceinline__ void pair_atoms(float4* A, int n, int tid, int nthreads, unsigned* r2max = nullptr) {
    float m = 0.f;
    for (int q = tid; q < (n >> 1); q += nthreads) {
        const float4 a = A[2 * q], b = A[2 * q + 1];
        A[2 * q] = make_float4(a.x, b.x, a.y, b.y);
        A[2 * q + 1] = make_float4(a.z, b.z, a.w, b.w);
        m = fmaxf(m, fmaxf(a.x * a.x + a.y * a.y + a.z * a.z, b.x * b.x + b.y * b.y + b.z * b.z));
    }
    if (r2max) {
        if ((n & 1) && tid == 0) {
            const float4 a = A[n - 1];
            m = fmaxf(m, a.x * a.x + a.y * a.y + a.z * a.z);
        }
        atomicMax(r2max, __float_as_uint(m));
    }
}

// Whether, along any direction of norm <= 1 + 1e-5, a projection s of an atom
// with |x|^2 <= r2max can make s * scale an exact nonzero integer.  With
// scale = J 2^E (J odd) and s = j 2^e (j odd), s * scale = j J 2^(e + E) is an
// integer only if e >= -E, i.e. |s| >= 2^-E.  |s| <= |u| |x| (1 + 4 2^-24)
// and r2max carries at most ~2e-7 relative rounding, so |s| stays below 2^-E
// when r2max (1 + 5e-5) < 2^-2E.  Otherwise only s = 0 gives an integer product.
__device__ __forceinline__ bool nonzero_integer_products_possible(float scale, float r2max) {
    const uint32_t bits = __float_as_uint(scale);
    const int ex = (int)((bits >> 23) & 0xFFu);
    if (ex == 0 || ex == 0xFF) return true;   // subnormal or not finite: no claim
    const uint32_t mant = (bits & 0x7FFFFFu) | 0x800000u;
    const int E = ex - 150 + (__ffs((int)mant) - 1);
    if (-2 * E >= 126) return false;
    return !(r2max * 1.00005f < ldexpf(1.0f, -2 * E));
}

// Per-lane constants of the paired loop: the lane's two directions and the
// binning scale and magic, each duplicated into both halves of a pair.
struct PairDirs {
    uint64_t x0, y0, z0, x1, y1, z1, sc, mg;
};

__device__ __forceinline__ PairDirs pair_dirs(float4 d0, float4 d1, float scale, float magic) {
    PairDirs q;
    q.x0 = f2_dup(d0.x);
    q.y0 = f2_dup(d0.y);
    q.z0 = f2_dup(d0.z);
    q.x1 = f2_dup(d1.x);
    q.y1 = f2_dup(d1.y);
    q.z1 = f2_dup(d1.z);
    q.sc = f2_dup(scale);
    q.mg = f2_dup(magic);
    return q;
}

// Two atoms (one paired block) into the histograms of a 64-direction tile:
// the projections and the binning of Eq. 1 in the scalar order (x, then
// y, then z; fma rounding down for the bin) on FP32 pairs, then the four
// increments of hist_add_atom's unmasked form.
__device__ __forceinline__ void hist_add_pair(uint32_t hbase, ulonglong2 xy, uint64_t zz, const PairDirs& q) {
    const uint64_t s0 = f2_fma(zz, q.z0, f2_fma(xy.y, q.y0, f2_mul(xy.x, q.x0)));
    const uint64_t s1 = f2_fma(zz, q.z1, f2_fma(xy.y, q.y1, f2_mul(xy.x, q.x1)));
    const uint64_t t0 = f2_fma_rd(s0, q.sc, q.mg);
    const uint64_t t1 = f2_fma_rd(s1, q.sc, q.mg);
    const uint32_t base = hbase - 0x80000000u;   // (t - 0x4B000000) * 128 + hbase, wrapping
    const uint32_t wa0 = (uint32_t)t0 * 128u + base, wb0 = (uint32_t)(t0 >> 32) * 128u + base;
    const uint32_t wa1 = (uint32_t)t1 * 128u + base, wb1 = (uint32_t)(t1 >> 32) * 128u + base;
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wa0), "r"(1u) : "memory");
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wb0), "r"(1u) : "memory");
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wa1), "r"(0x10000u) : "memory");
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wb1), "r"(0x10000u) : "memory");
}

// hist_tile<W, false> over atoms staged by pair_atoms: warp w takes the
// pairs w, w + W, w + 2W, ...; the odd trailing atom goes to warp
// (cn / 2) % W.
template <int W>
__device__ __forceinline__ void hist_tile_pairs(uint32_t* H, const float4* A, int cn, int warp, int lane,
                                                float4 d0, float4 d1, float scale, float magic) {
    const uint32_t hbase = smem_u32(H) + 4u * (uint32_t)lane;
    const PairDirs q = pair_dirs(d0, d1, scale, magic);
    const int np = cn >> 1;
    int j = warp;
    auto ld_xy = [&](int i) { return *reinterpret_cast<const ulonglong2*>(A + 2 * i); };
    auto ld_z = [&](int i) { return *reinterpret_cast<const uint64_t*>(A + 2 * i + 1); };
    if (j + W < np) {
        // two pairs at a time, the next two pairs' loads issued first
        ulonglong2 xa = ld_xy(j), xb = ld_xy(j + W);
        uint64_t za = ld_z(j), zb = ld_z(j + W);
        for (; j + 3 * W < np; j += 2 * W) {
            const ulonglong2 nxa = ld_xy(j + 2 * W), nxb = ld_xy(j + 3 * W);
            const uint64_t nza = ld_z(j + 2 * W), nzb = ld_z(j + 3 * W);
            hist_add_pair(hbase, xa, za, q);
            hist_add_pair(hbase, xb, zb, q);
            xa = nxa;
            xb = nxb;
            za = nza;
            zb = nzb;
        }
        hist_add_pair(hbase, xa, za, q);
        hist_add_pair(hbase, xb, zb, q);
        j += 2 * W;
    }
    for (; j < np; j += W) hist_add_pair(hbase, ld_xy(j), ld_z(j), q);
    if ((cn & 1) && warp == np % W) {
        const float4 d0s = d0, d1s = d1;
        hist_add_atom<false>(hbase, A[cn - 1], d0s, d1s, scale, magic, 0);
    }
}

// -----------------------------------------------------------------------------
// Histogram pass of the general tensor-core path: bin chunks, and the count of
// atoms whose bin product is not an integer.
//
// Bin chunks (m > 10): the 2^m bins are split into chunks of 1024 bins (128 KB
// of histogram words); the pass for chunk bc adds only atoms whose bin lies in
// [1024 bc, 1024 bc + 1024), at row b - 1024 bc.  The bin fma's bit pattern is
// 0x4B000000 + b, so the chunk of b is bits 10.. of the pattern.
//
// Antipodal directions: along -u the projection is exactly -s (round to
// nearest is symmetric), so the bin of -u is 2^m - 1 - b(u) whenever the exact
// product x = s * scale is not an integer, and 2^m - b(u) when it is.  With the
// product rounded down (t_rd) and up (t_ru) onto the integer grid of
// [2^23, 2^24), t_ru - t_rd is 1 for a non-integer x and 0 for an integer x; a
// lane sums it over its atoms (kCount), so the histogram of -u is the mirror
// image of the histogram of u exactly when that sum equals the lane's atom
// count.
// -----------------------------------------------------------------------------
template <int kCount, bool kChunked>
__device__ __forceinline__ void hist_add_pair2(uint32_t hb, ulonglong2 xy, uint64_t zz, const PairDirs& q,
                                               uint32_t bc, uint32_t cmask, uint32_t& c0, uint32_t& c1,
                                               uint64_t& zp) {
    const uint64_t s0 = f2_fma(zz, q.z0, f2_fma(xy.y, q.y0, f2_mul(xy.x, q.x0)));
    const uint64_t s1 = f2_fma(zz, q.z1, f2_fma(xy.y, q.y1, f2_mul(xy.x, q.x1)));
    const uint64_t t0 = f2_fma_rd(s0, q.sc, q.mg);
    const uint64_t t1 = f2_fma_rd(s1, q.sc, q.mg);
    if (kCount == 2) {
        zp = f2_mul(zp, f2_mul(s0, s1));
    } else if (kCount == 1) {
        const uint64_t u0 = f2_fma_ru(s0, q.sc, q.mg);
        const uint64_t u1 = f2_fma_ru(s1, q.sc, q.mg);
        c0 += ((uint32_t)u0 - (uint32_t)t0) + ((uint32_t)(u0 >> 32) - (uint32_t)(t0 >> 32));
        c1 += ((uint32_t)u1 - (uint32_t)t1) + ((uint32_t)(u1 >> 32) - (uint32_t)(t1 >> 32));
    }
    // (t - 0x4B000000 - 1024 bc) * 128 + H + 4 lane, in wrapping 32-bit arithmetic
    const uint32_t wa0 = (uint32_t)t0 * 128u + hb, wb0 = (uint32_t)(t0 >> 32) * 128u + hb;
    const uint32_t wa1 = (uint32_t)t1 * 128u + hb, wb1 = (uint32_t)(t1 >> 32) * 128u + hb;
    if (kChunked) {
        if ((((uint32_t)t0 >> 10) & cmask) == bc) asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wa0), "r"(1u) : "memory");
        if ((((uint32_t)(t0 >> 32) >> 10) & cmask) == bc)
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wb0), "r"(1u) : "memory");
        if ((((uint32_t)t1 >> 10) & cmask) == bc)
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wa1), "r"(0x10000u) : "memory");
        if ((((uint32_t)(t1 >> 32) >> 10) & cmask) == bc)
            asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wb1), "r"(0x10000u) : "memory");
    } else {
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wa0), "r"(1u) : "memory");
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wb0), "r"(1u) : "memory");
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wa1), "r"(0x10000u) : "memory");
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(wb1), "r"(0x10000u) : "memory");
    }
}

template <int kCount, bool kChunked>
__device__ __forceinline__ void hist_add_one2(uint32_t hb, float4 a, float4 d0, float4 d1, float scale, float magic,
                                              uint32_t bc, uint32_t cmask, uint32_t& c0, uint32_t& c1, uint64_t& zp) {
    const float s0 = project_f32(d0.x, d0.y, d0.z, a);
    const float s1 = project_f32(d1.x, d1.y, d1.z, a);
    const uint32_t t0 = __float_as_uint(__fmaf_rd(s0, scale, magic));
    const uint32_t t1 = __float_as_uint(__fmaf_rd(s1, scale, magic));
    if (kCount == 2) {
        zp = (zp & 0xFFFFFFFF00000000ull) | (uint64_t)__float_as_uint(__uint_as_float((uint32_t)zp) * s0 * s1);
    } else if (kCount == 1) {
        c0 += __float_as_uint(__fmaf_ru(s0, scale, magic)) - t0;
        c1 += __float_as_uint(__fmaf_ru(s1, scale, magic)) - t1;
    }
    if (!kChunked || ((t0 >> 10) & cmask) == bc)
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(t0 * 128u + hb), "r"(1u) : "memory");
    if (!kChunked || ((t1 >> 10) & cmask) == bc)
        asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(t1 * 128u + hb), "r"(0x10000u) : "memory");
}

// Histograms of one 64-direction tile over `cn` atoms staged by pair_atoms, for
// bin chunk bc (kChunked) or all bins; warp w takes pairs w, w + W, ...
// Returns the number of atoms this warp handled.  kCount == 1: c0, c1
// accumulate the lane's non-integer counts of its two directions; kCount ==
// 2 (only s = 0 can give an integer product): zp multiplies the projections
// of the lane's atoms along both directions, so a zero half means an atom
// with s = 0 (a product of the ~70 factors |s| <= R a lane sees per tile
// stays above ~1e-20 at four standard deviations, far from FP32's 1e-45; an
// underflow would only cost the tile a second pass).
template <int W, int kCount, bool kChunked>
__device__ __forceinline__ int hist_tile_pairs2(uint32_t* H, const float4* A, int cn, int warp, int lane, float4 d0,
                                                float4 d1, float scale, float magic, uint32_t bc, uint32_t cmask,
                                                uint32_t& c0, uint32_t& c1, uint64_t& zp) {
    const uint32_t hb = smem_u32(H) + 4u * (uint32_t)lane - 0x80000000u - (bc << 17);
    const PairDirs q = pair_dirs(d0, d1, scale, magic);
    const int np = cn >> 1;
    int j = warp;
    auto ld_xy = [&](int i) { return *reinterpret_cast<const ulonglong2*>(A + 2 * i); };
    auto ld_z = [&](int i) { return *reinterpret_cast<const uint64_t*>(A + 2 * i + 1); };
    // four independent atom pairs per step (their loads first)
    for (; j + 3 * W < np; j += 4 * W) {
        const ulonglong2 x0 = ld_xy(j), x1 = ld_xy(j + W), x2 = ld_xy(j + 2 * W), x3 = ld_xy(j + 3 * W);
        const uint64_t z0 = ld_z(j), z1 = ld_z(j + W), z2 = ld_z(j + 2 * W), z3 = ld_z(j + 3 * W);
        hist_add_pair2<kCount, kChunked>(hb, x0, z0, q, bc, cmask, c0, c1, zp);
        hist_add_pair2<kCount, kChunked>(hb, x1, z1, q, bc, cmask, c0, c1, zp);
        hist_add_pair2<kCount, kChunked>(hb, x2, z2, q, bc, cmask, c0, c1, zp);
        hist_add_pair2<kCount, kChunked>(hb, x3, z3, q, bc, cmask, c0, c1, zp);
    }
    for (; j < np; j += W) hist_add_pair2<kCount, kChunked>(hb, ld_xy(j), ld_z(j), q, bc, cmask, c0, c1, zp);
    int handled = warp < np ? 2 * ((np - warp + W - 1) / W) : 0;
    if ((cn & 1) && warp == np % W) {
        hist_add_one2<kCount, kChunked>(hb, A[cn - 1], d0, d1, scale, magic, bc, cmask, c0, c1, zp);
        handled += 1;
    }
    return handled;
}

// Debug export of a tile's histograms: h_out[v * 2^m + b] for v < nv.
__device__ __forceinline__ void hist_export(const uint32_t* H, int NB, int tile, int nv, uint16_t* h_out, int tid,
                                            int nthreads) {
    for (int i = tid; i < NB * 32; i += nthreads) {
        const int b = i >> 5, l = i & 31;
        const uint32_t w = H[i];
        const int64_t v0 = (int64_t)tile * 64 + 2 * l;
        if (v0 < nv) h_out[v0 * NB + b] = (uint16_t)(w & 0xFFFFu);
        if (v0 + 1 < nv) h_out[(v0 + 1) * NB + b] = (uint16_t)(w >> 16);
    }
}

// Band maxima of one direction: frequency f with amplitude a updates every
// band holding f (strictly greater, so with f ascending ties keep the lowest
// f).  bs.n == 0: the single band [klo, khi] of the ROI.
__device__ __forceinline__ int band_count(const BandSet& bs) { return bs.n == 0 ? 1 : bs.n; }

__device__ __forceinline__ void band_init(const BandSet& bs, int klo, float* best, int* bk) {
#pragma unroll
    for (int b = 0; b < APTIDX_MAX_BANDS; ++b) {
        best[b] = -1.f;
        bk[b] = bs.n == 0 ? klo : bs.lo[b];
    }
}

__device__ __forceinline__ void band_update(const BandSet& bs, int klo, int khi, int f, float a, float* best,
                                            int* bk) {
    const int nb = band_count(bs);
#pragma unroll
    for (int b = 0; b < APTIDX_MAX_BANDS; ++b) {
        const int lo = bs.n == 0 ? klo : bs.lo[b], hi = bs.n == 0 ? khi : bs.hi[b];
        if (b < nb && f >= lo && f <= hi && a > best[b]) {
            best[b] = a;
            bk[b] = f;
        }
    }
}

// The same with the slot count fixed at compile time: kNB == 1 is the
// single-band kernel (the ROI's band [klo, khi]; the BandSet is not read).
template <int kNB>
__device__ __forceinline__ void band_init_t(const BandSet& bs, int klo, float* best, int* bk) {
    if (kNB == 1) {
        best[0] = -1.f;
        bk[0] = klo;
    } else {
        band_init(bs, klo, best, bk);
    }
}

template <int kNB>
__device__ __forceinline__ void band_update_t(const BandSet& bs, int klo, int khi, int f, float a, float* best,
                                              int* bk) {
    if (kNB == 1) {
        if (f >= klo && f <= khi && a > best[0]) {
            best[0] = a;
            bk[0] = f;
        }
    } else {
        band_update(bs, klo, khi, f, a, best, bk);
    }
}

template <int kNB>
__device__ __forceinline__ int band_count_t(const BandSet& bs) { return kNB == 1 ? 1 : band_count(bs); }

template <int kNB>
__device__ __forceinline__ int64_t band_off_t(const BandSet& bs, int b) { return kNB == 1 ? 0 : bs.off[b]; }

// ROI rank ranges of a signature launch (ranks index the longest-first order)
constexpr int kRanksAll = 0;       // [0, nroi)
constexpr int kRanksBig = 1;       // [0, n_big): ROIs above 2048 atoms
constexpr int kRanksSmall = 2;     // [n_big, nroi)
constexpr int kTcMaxAtoms = 2048;  // fp16 carries every count <= 2048 exactly

// -----------------------------------------------------------------------------
// status word
// -----------------------------------------------------------------------------
__device__ __forceinline__ void raise_status(int* status, int bit) {
    atomicOr(status, bit);
}

// -----------------------------------------------------------------------------
// shared-memory addresses, mbarriers and bulk copies (inline PTX)
// -----------------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, at most `limit` polls.  Returns
// false (and raises the timeout status bit) if the phase never completed.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int* status,
                                                  uint32_t limit = (1u << 22)) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    raise_status(status, kStatusTimeout);
    return false;
}

// 1-D bulk copy global -> shared (TMA engine), completion counted in bytes on
// `bar`.  dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte asynchronous copy global -> shared (no L1 allocation); completion
// by cp_async_wait_all of the issuing thread.  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Stage `n` float4 atoms from global into shared memory with one bulk copy
// issued by thread 0, then make them visible to the whole CTA.  `phase` is
// the barrier's parity bit, toggled per use.  Returns false on a timeout
// (every thread of the CTA returns the same value).
__device__ __forceinline__ bool stage_atoms(float4* dst, const float4* src, int n, uint64_t* bar,
                                            uint32_t& phase, int* status, int* flag_smem) {
    if (threadIdx.x == 0) {
        int ok = 1;
        if (n > 0) {
            fence_proxy_async_smem();   // earlier generic reads of dst before the async write
            mbar_arrive_expect_tx(bar, (uint32_t)n * 16u);
            bulk_g2s(dst, src, (uint32_t)n * 16u, bar);
            ok = mbar_wait_bounded(bar, phase, status) ? 1 : 0;
            if (!ok) mbar_wait_bounded(bar, phase, status, 1u << 20);   // let an in-flight copy land
            phase ^= 1u;
        }
        *flag_smem = ok;
    }
    __syncthreads();
    int ok = *flag_smem;
    if (threadIdx.x != 0 && n > 0) phase ^= 1u;
    __syncthreads();   // flag_smem is rewritten by the next call
    return ok != 0;
}

}  // namespace aptidx
