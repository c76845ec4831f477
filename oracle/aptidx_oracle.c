/*
 * aptidx_oracle.c -- plain, slow, FP64 CPU oracle of the real-space (RSP)
 * signature method of Kuehbach et al., arXiv 2009.00735.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library
 * never calls it.
 *
 * Every function states the passage of the paper it writes out.  The
 * arithmetic is FP64 unless the function emulates the library's published
 * FP32 binning contract, which is stated where it is used.
 *
 * Readings of passages that the paper leaves open (each also listed in the
 * design notes):
 *   - membership is the closed ball |p - p_c| <= R, evaluated in FP64 as
 *     (dx*dx + dy*dy) + dz*dz without fused multiply-add;
 *   - Eq. 1 with Delta R = R / (2^(m-1) - 1) (Fig. 2 caption) gives
 *     b = floor(2^(m-1) + s (2^(m-1) - 1) / R), bins clamped to [0, 2^m - 1];
 *   - the spectrum is the unnormalised one-sided DFT amplitude of the
 *     histogram with a rectangular window (Section 2.2, Fig. 2 caption,
 *     supplement "Controlled windowing"), X(0) = N_w;
 *   - the signature value is the largest amplitude inside a fixed band of
 *     frequency bins [k_lo, k_hi]; ties resolve to the lowest k;
 *   - normalisation divides a signature by its largest value;
 *   - Eq. 3 matching: q maps crystal to lab, so reference node n rotates to
 *     R(q) n, and the look-up table holds its nearest measured node.
 *
 * Parity unpinned: none (every function below has a pin in the CPU tests).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* Test-only mutation points.  A build with -DORC_MUTATION=k plants the k-th
 * plausible mistake listed in tests/test_oracle_mutations.py (a dropped term,
 * an off-by-one, a transposed operand, ...), so that the test can check that
 * the pins of tests/test_oracle_pins.py catch it.  The default build
 * (ORC_MUTATION = 0) contains none of them. */
#ifndef ORC_MUTATION
#define ORC_MUTATION 0
#endif
/* MUT(k, wrong, right): the planted mistake k in a mutant build, the
 * definition otherwise (a compile-time choice; the default build evaluates
 * `right` only). */
#define MUT(k, wrong, right) ((ORC_MUTATION == (k)) ? (wrong) : (right))

/* ------------------------------------------------------------------------ */
/* Section 2.2 / SI cost O_Proj: atoms of the ROI                            */
/* ------------------------------------------------------------------------ */

static int orc_selected(const uint8_t* types, int64_t i, uint32_t type_mask)
{
    if (!types) return 1;
    unsigned t = types[i] + MUT(19, 1u, 0u);
    return t < 32u && ((type_mask >> t) & 1u);
}

/* Atoms i with |p_i - p_c| <= R (closed ball, FP64).  Brute force over all
 * atoms.  Writes their indices (ascending) and the centred coordinates
 * x_i = (float)(p_i - p_c) when the output pointers are not NULL.  Returns
 * the count N_w. */
int64_t orc_gather(const float* xyz, int64_t n, const uint8_t* types, uint32_t type_mask,
                   const double* c, double R, int64_t* idx, float* xc)
{
    int64_t k = 0;
    const double R2 = R * R;
    for (int64_t i = 0; i < n; ++i) {
        if (!orc_selected(types, i, type_mask)) continue;
        double dx = (double)xyz[3 * i + MUT(6, 1, 0)] - c[0];
        double dy = (double)xyz[3 * i + 1] - c[1];
        double dz = (double)xyz[3 * i + 2] - c[2];
        double xx = dx * dx;
        double yy = dy * dy;
        double zz = dz * dz;
        double d2 = (xx + yy) + zz;
        if (d2 <= R2) {
            if (idx) idx[k] = i;
            if (xc) {
                xc[3 * k + 0] = (float)dx;
                xc[3 * k + 1] = (float)dy;
                xc[3 * k + 2] = (float)dz;
            }
            ++k;
        }
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* Eq. 1: the bin of a projected atom                                        */
/* ------------------------------------------------------------------------ */

static int64_t orc_clamp_bin(double f, int m)
{
    const int64_t nb = (int64_t)1 << m;
    if (!(f > -1e300)) return 0;            /* NaN or -inf */
    if (f < 0.0) return 0;
    if (f > (double)(nb - 1)) return nb - 1;
    return (int64_t)f;
}

/* Eq. 1 written out in FP64: b = floor((s + R + dR) 2^m / (dR + 2R + dR))
 * with s = d . (p - p_c) and dR = R / (2^(m-1) - 1). */
int orc_bin_eq1(const double* u, const double* x, int m, double R)
{
    const double dR = R / (double)((1 << (m - 1)) - 1);
    const double s = (u[0] * x[0] + u[1] * x[1]) + u[2] * x[2];
    const double t = MUT(4, (s + R) * (double)(1 << m) / (2.0 * R),
                            (s + R + dR) * (double)(1 << m) / (dR + 2.0 * R + dR));
    return (int)orc_clamp_bin(floor(t), m);
}

/* The binning contract the library computes bit-exactly (FP32 inputs):
 *   s     = fma(u_z, x_z, fma(u_y, x_y, u_x * x_x))     each step FP32, RN
 *   scale = (float)((2^(m-1) - 1) / R)                  from FP64
 *   b     = clamp(2^(m-1) + floor(s * scale), 0, 2^m - 1)
 * where s * scale is the exact real product (two FP32 numbers multiply
 * exactly in FP64).  Algebraically this is Eq. 1 with dR = R/(2^(m-1)-1),
 * since (R + dR) 2^m / (2R + 2dR) = 2^(m-1) and 2^m / (2R + 2dR) =
 * (2^(m-1) - 1) / R. */
float orc_bin_scale(int m, double R)
{
    return (float)((double)((1 << (m - 1)) - 1) / R);
}

float orc_project_f32(const float* u, const float* x)
{
    float p = u[0] * x[0];
    float a = fmaf(u[1], x[1], p);
    return MUT(1, a, fmaf(u[2], x[2], a));
}

int orc_bin_contract(const float* u, const float* x, int m, double R)
{
    const float s = orc_project_f32(u, x);
    const float scale = orc_bin_scale(m, R);
    const double prod = (double)s * (double)scale;   /* exact */
    const double f = (double)((1 << (m - 1)) - MUT(2, 1, 0)) + floor(prod);
    return (int)orc_clamp_bin(f, m);
}

/* One SDM per direction (Section 2.2): h[v * 2^m + b] = number of atoms
 * whose contract bin along direction v is b.  h is overwritten. */
void orc_histograms(const float* xc, int64_t nw, const float* u, int64_t nv, int m, double R,
                    int32_t* h)
{
    const int64_t nb = (int64_t)1 << m;
    memset(h, 0, sizeof(int32_t) * (size_t)(nv * nb));
    for (int64_t v = 0; v < nv; ++v)
        for (int64_t i = 0; i < nw; ++i)
            h[v * nb + orc_bin_contract(u + 3 * v, xc + 3 * i, m, R)] += 1;
}

/* Same, with the FP64 Eq. 1 bins (the exact form); used by the tests that
 * count boundary atoms where the FP32 contract and Eq. 1 disagree. */
void orc_histograms_eq1(const float* xc, int64_t nw, const float* u, int64_t nv, int m, double R,
                        int32_t* h)
{
    const int64_t nb = (int64_t)1 << m;
    memset(h, 0, sizeof(int32_t) * (size_t)(nv * nb));
    for (int64_t v = 0; v < nv; ++v) {
        double ud[3] = {u[3 * v], u[3 * v + 1], u[3 * v + 2]};
        for (int64_t i = 0; i < nw; ++i) {
            double xd[3] = {xc[3 * i], xc[3 * i + 1], xc[3 * i + 2]};
            h[v * nb + orc_bin_eq1(ud, xd, m, R)] += 1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Section 2.2: amplitude spectrum of one SDM, band-limited                  */
/* ------------------------------------------------------------------------ */

/* cos/sin of 2 pi j / N_b for j < N_b; the angle index is reduced exactly
 * in integers before the FP64 trigonometric call. */
static void orc_twiddles(int m, double* cs, double* sn)
{
    const int64_t nb = (int64_t)1 << m;
    for (int64_t j = 0; j < nb; ++j) {
        double th = 2.0 * ORC_PI * (double)j / (double)(nb - MUT(21, 1, 0));
        cs[j] = cos(th);
        sn[j] = sin(th);
    }
}

/* X(k) = sum_n h[n] exp(-2 pi i k n / N_b) for k in [k_lo, k_hi];
 * amp[k - k_lo] = |X(k)|. */
static void orc_band_amplitudes_tw(const int32_t* h, int m, int k_lo, int k_hi,
                                   const double* cs, const double* sn, double* amp)
{
    const int64_t nb = (int64_t)1 << m;
    for (int k = k_lo; k <= k_hi; ++k) {
        double re = 0.0, im = 0.0;
        for (int64_t n = 0; n < nb; ++n) {
            if (!h[n]) continue;
            int64_t j = ((int64_t)(k + MUT(3, 1, 0)) * n) % nb;
            re += (double)h[n] * cs[j];
            im -= (double)h[n] * sn[j];
        }
        amp[k - k_lo] = sqrt(re * re + im * im);
    }
}

void orc_band_amplitudes(const int32_t* h, int m, int k_lo, int k_hi, double* amp)
{
    const int64_t nb = (int64_t)1 << m;
    double* cs = (double*)malloc(sizeof(double) * (size_t)nb);
    double* sn = (double*)malloc(sizeof(double) * (size_t)nb);
    orc_twiddles(m, cs, sn);
    orc_band_amplitudes_tw(h, m, k_lo, k_hi, cs, sn, amp);
    free(cs);
    free(sn);
}

/* ------------------------------------------------------------------------ */
/* Section 2.2 + supplement (Al bicrystal): signature of one ROI             */
/* ------------------------------------------------------------------------ */

/* S[v] = max_{k_lo <= k <= k_hi} |X_v(k)|, argk[v] = the lowest k attaining it. */
void orc_roi_signature(const float* xc, int64_t nw, const float* u, int64_t nv, int m, double R,
                       int k_lo, int k_hi, double* S, int32_t* argk)
{
    const int64_t nb = (int64_t)1 << m;
    const int nk = k_hi - k_lo + 1;
    int32_t* h = (int32_t*)malloc(sizeof(int32_t) * (size_t)nb);
    double* amp = (double*)malloc(sizeof(double) * (size_t)(nk > 0 ? nk : 1));
    double* cs = (double*)malloc(sizeof(double) * (size_t)nb);
    double* sn = (double*)malloc(sizeof(double) * (size_t)nb);
    orc_twiddles(m, cs, sn);
    for (int64_t v = 0; v < nv; ++v) {
        memset(h, 0, sizeof(int32_t) * (size_t)nb);
        for (int64_t i = 0; i < nw; ++i)
            h[orc_bin_contract(u + 3 * v, xc + 3 * i, m, R)] += 1;
        orc_band_amplitudes_tw(h, m, k_lo, k_hi, cs, sn, amp);
        double best = -1.0;
        int bk = k_lo;
        for (int k = 0; k < nk; ++k)
            if (MUT(8, amp[k] >= best, amp[k] > best)) { best = amp[k]; bk = k_lo + k; }
        S[v] = nk > 0 ? best : 0.0;
        if (argk) argk[v] = bk;
    }
    free(h); free(amp); free(cs); free(sn);
}

/* All ROIs: gather (brute force), then per-ROI signature.  Optional outputs
 * may be NULL.  band_lo/band_hi are per ROI.  Runs ROIs in parallel on
 * `threads` OpenMP threads (<= 0: the runtime default). */
int orc_signatures(const float* xyz, int64_t n, const uint8_t* types, uint32_t type_mask,
                   const double* centres, const double* radii, int64_t nroi,
                   const int32_t* band_lo, const int32_t* band_hi,
                   const float* u, int64_t nv, int m,
                   double* S, int32_t* argk, int64_t* nw_out, int threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int64_t r = 0; r < nroi; ++r) {
        int64_t nw = orc_gather(xyz, n, types, type_mask, centres + 3 * r, radii[r], NULL, NULL);
        float* xc = (float*)malloc(sizeof(float) * 3 * (size_t)(nw > 0 ? nw : 1));
        orc_gather(xyz, n, types, type_mask, centres + 3 * r, radii[r], NULL, xc);
        orc_roi_signature(xc, nw, u, nv, m, radii[r], band_lo[r], band_hi[r], S + r * nv,
                          argk ? argk + r * nv : NULL);
        if (nw_out) nw_out[r] = nw;
        free(xc);
    }
    return 0;
}

/* Indexing step 1 (supplement "Indexing algorithm"): divide a signature by
 * its largest value, giving intensities in [0, 1]. */
void orc_normalise(double* S, int64_t nroi, int64_t nv)
{
    for (int64_t r = 0; r < nroi; ++r) {
        double mx = 0.0;
        for (int64_t v = 0; v < nv; ++v) {
            const double s = S[r * nv + v];
            mx = MUT(13, mx + s, s > mx ? s : mx);
        }
        for (int64_t v = 0; v < nv; ++v) S[r * nv + v] = mx > 0.0 ? S[r * nv + v] / mx : 0.0;
    }
}

/* Band of frequency bins for a plane-spacing interval [d_min, d_max]:
 * frequency bin k has period W / k with W = 2^m dR = 2 (R + dR)
 * (Fig. 2 caption: f_s = L / (2 (R + dR))), so
 * k_lo = ceil(W / d_max), k_hi = floor(W / d_min). */
void orc_band_for_spacing(double d_min, double d_max, double R, int m, int32_t* k_lo, int32_t* k_hi)
{
    const double dR = R / (double)((1 << (m - 1)) - 1);
    const double W = 2.0 * (R + dR);
    *k_lo = (int32_t)MUT(16, floor(W / d_max), ceil(W / d_max));
    *k_hi = (int32_t)MUT(16, ceil(W / d_min), floor(W / d_min));
}

/* ------------------------------------------------------------------------ */
/* Rotations (FP64)                                                          */
/* ------------------------------------------------------------------------ */

static void orc_transpose3(double* M)
{
    double t;
    t = M[1]; M[1] = M[3]; M[3] = t;
    t = M[2]; M[2] = M[6]; M[6] = t;
    t = M[5]; M[5] = M[7]; M[7] = t;
}

/* Rotation matrix of a unit quaternion q = (w, x, y, z); maps crystal to lab.
 * No fused multiply-add, fixed evaluation order. */
void orc_quat_to_matrix(const double* q, double* M)
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double xx = x * x, yy = y * y, zz = z * z;
    const double xy = x * y, xz = x * z, yz = y * z;
    const double wx = w * x, wy = w * y, wz = w * z;
    M[0] = 1.0 - 2.0 * (yy + zz); M[1] = 2.0 * (xy - wz);       M[2] = 2.0 * (xz + wy);
    M[3] = 2.0 * (xy + wz);       M[4] = 1.0 - 2.0 * (xx + zz); M[5] = 2.0 * (yz - wx);
    M[6] = 2.0 * (xz - wy);       M[7] = 2.0 * (yz + wx);       M[8] = 1.0 - 2.0 * (xx + yy);
    if (MUT(14, 1, 0)) orc_transpose3(M);
}

static void orc_quat_mul(const double* a, const double* b, double* o)
{
    double r0 = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    double r1 = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    double r2 = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    double r3 = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3;
}

/* The 24 proper rotations of m-3m as quaternions (Section 2.3,
 * supplement "test orientations"): identity, 9 rotations about <100>
 * (90, 180, 270 deg), 8 about <111> (120, 240 deg), 6 about <110> (180 deg). */
static void orc_cubic_symmetry(double q[24][4])
{
    const double h = sqrt(0.5);
    const double t[24][4] = {
        {1, 0, 0, 0},
        {h, h, 0, 0}, {0, 1, 0, 0}, {h, -h, 0, 0},
        {h, 0, h, 0}, {0, 0, 1, 0}, {h, 0, -h, 0},
        {h, 0, 0, h}, {0, 0, 0, 1}, {h, 0, 0, -h},
        {0.5, 0.5, 0.5, 0.5}, {0.5, -0.5, -0.5, -0.5},
        {0.5, -0.5, 0.5, 0.5}, {0.5, 0.5, -0.5, -0.5},
        {0.5, 0.5, -0.5, 0.5}, {0.5, -0.5, 0.5, -0.5},
        {0.5, 0.5, 0.5, -0.5}, {0.5, -0.5, -0.5, 0.5},
        {0, h, h, 0}, {0, h, -h, 0}, {0, h, 0, h}, {0, h, 0, -h}, {0, 0, h, h}, {0, 0, h, -h},
    };
    memcpy(q, t, sizeof(t));
}

/* Disorientation angle (degrees) between two cubic orientations: the
 * smallest rotation angle of q1^-1 q2 s over the 24 proper cubic rotations s
 * (the supplement defines the disorientation as the symmetry-equivalent
 * misorientation of least rotation angle). */
double orc_disorientation_deg(const double* q1, const double* q2)
{
    double sym[24][4];
    orc_cubic_symmetry(sym);
    double inv[4] = {q1[0], -q1[1], -q1[2], -q1[3]};
    double d[4];
    orc_quat_mul(inv, q2, d);
    double best = 0.0;
    for (int s = 0; s < 24 - MUT(12, 1, 0); ++s) {
        double e[4];
        orc_quat_mul(d, sym[s], e);
        double w = fabs(e[0]) / sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3]);
        if (w > best) best = w;
    }
    if (best > 1.0) best = 1.0;
    return 2.0 * acos(best) * 180.0 / ORC_PI;
}

/* ------------------------------------------------------------------------ */
/* Supplement "Indexing algorithm" and Eq. 3                                 */
/* ------------------------------------------------------------------------ */

/* Indices of the n_hat strongest reference nodes, strongest first; equal
 * values order by ascending node index. */
typedef struct { float v; int32_t i; } orc_vi;
static int orc_vi_cmp(const void* a, const void* b)
{
    const orc_vi* x = (const orc_vi*)a;
    const orc_vi* y = (const orc_vi*)b;
    if (x->v > y->v) return -1;
    if (x->v < y->v) return 1;
    return MUT(10, (x->i < y->i) - (x->i > y->i), (x->i > y->i) - (x->i < y->i));
}

void orc_top_nodes(const float* sig, int64_t nv, int n_hat, int32_t* out)
{
    orc_vi* a = (orc_vi*)malloc(sizeof(orc_vi) * (size_t)nv);
    for (int64_t v = 0; v < nv; ++v) { a[v].v = sig[v]; a[v].i = (int32_t)v; }
    qsort(a, (size_t)nv, sizeof(orc_vi), orc_vi_cmp);
    for (int k = 0; k < n_hat; ++k) out[k] = a[k].i;
    free(a);
}

/* The rotated node direction, as FP32: r = (float)(R(q) n), FP64 products
 * summed left to right. */
void orc_rotate_node(const double* q, const float* nrm, float* r)
{
    double M[9];
    orc_quat_to_matrix(q, M);
    for (int i = 0; i < 3; ++i) {
        const int st = MUT(20, 3, 1), rs = MUT(20, 1, 3);
        double a = M[rs * i + 0 * st] * (double)nrm[0];
        double b = M[rs * i + 1 * st] * (double)nrm[1];
        double c = M[rs * i + 2 * st] * (double)nrm[2];
        r[i] = (float)((a + b) + c);
    }
}

/* Nearest node: argmax_p u_p . r (dot product as the FP32 contract above),
 * ties to the lowest index. */
int32_t orc_nearest_node(const float* u, int64_t nv, const float* r)
{
    int32_t best = 0;
    float bd = MUT(11, INFINITY, -INFINITY);
    for (int64_t p = 0; p < nv; ++p) {
        float d = orc_project_f32(u + 3 * p, r);
        if (MUT(11, d < bd, d > bd)) { bd = d; best = (int32_t)p; }
    }
    return best;
}

/* Look-up table p^g_v for every test orientation g and strongest node v:
 * lut[g * n_hat + k] = nearest node to R(q_g) n_{top[k]}. */
void orc_lut(const float* u, int64_t nv, const int32_t* top, int n_hat,
             const double* quats, int64_t ng, int32_t* lut, int threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int64_t g = 0; g < ng; ++g)
        for (int k = 0; k < n_hat; ++k) {
            float r[3];
            orc_rotate_node(quats + 4 * g, u + 3 * (int64_t)top[k], r);
            lut[g * n_hat + k] = orc_nearest_node(u, nv, r);
        }
}

/* Eq. 3: Delta(g) = sum_k (S_msr[lut[g, k]] - S_ref[top[k]])^2 (FP64 sum),
 * best[r] = argmin_g (ties: lowest g).  scores may be NULL or [nroi x ng]. */
void orc_match(const float* S_msr, int64_t nroi, int64_t nv, const float* S_ref,
               const int32_t* top, int n_hat, const int32_t* lut, int64_t ng,
               int32_t* best, double* best_score, double* scores, int threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int64_t r = 0; r < nroi; ++r) {
        const float* s = S_msr + r * nv;
        double bs = INFINITY;
        int32_t bg = 0;
        for (int64_t g = 0; g < ng; ++g) {
            double acc = 0.0;
            for (int k = 0; k < n_hat; ++k) {
                double d = (double)s[lut[g * n_hat + k]] - (double)S_ref[top[k]];
                acc += MUT(5, fabs(d), d * d);
            }
            if (scores) scores[r * ng + g] = acc;
            if (acc < bs) { bs = acc; bg = (int32_t)g; }
        }
        best[r] = bg;
        if (best_score) best_score[r] = bs;
    }
}

/* Phase and orientation from several signatures per candidate (Section 2.3
 * "Indexing": every ROI's signatures are compared with the rotated references
 * of every crystal-structure candidate; the supplement's Al-Li-Mg-Ag case
 * compares three reference patterns, one for pure Al and one for each
 * sub-lattice of Al3Li).  Candidate c owns the signature channels
 * j in [off[c], off[c+1]); channel j compares the measured signatures
 * S + sig[j] * nroi * nv (layout [signature][roi][node]) with reference j:
 * values S_ref + j * nv, strongest nodes top + j * n_hat, look-up table
 * lut + j * ng * n_hat, all tables on one set of ng test orientations.
 *   Delta_c(g) = (1 / n_c) sum_j Delta_j(g) / E_j,  n_c = off[c+1] - off[c],
 * with Delta_j of Eq. 3 (FP64) and E_j = sum_k S_ref_j(top_j[k])^2, the Eq. 3
 * difference of an empty signature against reference j.  The paper compares
 * image differences across candidates without fixing how; relative to E_j a
 * channel scores 0 for a perfect match and 1 for no signal, whatever the
 * number and strength of its reference's peaks.  E_j > 0 is assumed.
 * best[c * nroi + r] = argmin_g Delta_c(g) (ties: lowest g), score[c * nroi
 * + r] = Delta_c(best); phase[r] = the candidate of the lowest score (ties:
 * lowest c). */
void orc_match_phase(const float* S, int64_t nroi, int64_t nv, int n_cand, const int32_t* off, const int32_t* sig,
                     const float* S_ref, const int32_t* top, int n_hat, const int32_t* lut, int64_t ng,
                     int32_t* phase, int32_t* best, double* score, int threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int64_t r = 0; r < nroi; ++r) {
        double bsc = INFINITY;
        int32_t bc = 0;
        for (int c = 0; c < n_cand; ++c) {
            const int nc = off[c + 1] - off[c];
            double bs = INFINITY;
            int32_t bg = 0;
            for (int64_t g = 0; g < ng; ++g) {
                double tot = 0.0;
                for (int j = off[c]; j < off[c + 1]; ++j) {
                    const float* s = S + ((int64_t)sig[MUT(23, off[c], j)] * nroi + r) * nv;
                    const float* ref = S_ref + (int64_t)j * nv;
                    const int32_t* tp = top + (int64_t)j * n_hat;
                    const int32_t* lt = lut + ((int64_t)j * ng + g) * n_hat;
                    double acc = 0.0, e = 0.0;
                    for (int k = 0; k < n_hat; ++k) {
                        const double d = (double)s[lt[k]] - (double)ref[tp[k]];
                        acc += d * d;
                        e += (double)ref[tp[k]] * (double)ref[tp[k]];
                    }
                    tot += MUT(24, acc, acc / e);
                }
                const double dc = MUT(22, tot, tot / (double)nc);
                if (dc < bs) { bs = dc; bg = (int32_t)g; }
            }
            best[(int64_t)c * nroi + r] = bg;
            score[(int64_t)c * nroi + r] = bs;
            if (bs < bsc) { bsc = bs; bc = c; }
        }
        phase[r] = bc;
    }
}

/* ------------------------------------------------------------------------ */
/* Orientation refinement (Gauss-Newton on a bilinear elevation-azimuth      */
/* reference image).  The paper motivates refining the indexing (Section     */
/* 3.3); the steps below are the workload's definition:                      */
/*   residual r_v = S_msr(u_v) - I(alpha, beta of c_v),  c_v = R^T u_v,      */
/*   R <- exp([delta]x) R,  delta = -(J^T J + lambda I)^-1 J^T r,            */
/*   lambda = 1e-6 tr(J^T J).                                                */
/* Image rows: alpha_i = -90 + i deg (i = 0..180); columns beta_j = j deg    */
/* (j = 0..359, periodic).  Directions whose crystal-frame elevation        */
/* exceeds 89 deg in magnitude are left out of the loss.                     */
/* ------------------------------------------------------------------------ */

#define ORC_IMG_NA 181
#define ORC_IMG_NB 360
#define ORC_POLE_DEG 89.0

/* Bilinear sample of the image at crystal-frame direction c, and the
 * gradient of the sample with respect to c.  Returns 0 when c is inside the
 * pole cap that is left out, 1 otherwise.  cell (may be NULL) receives
 * (i0, j0). */
int orc_bilinear(const float* img, const double* c, double* val, double* grad, int32_t* cell)
{
    const double rho2 = c[0] * c[0] + c[1] * c[1];
    const double rho = sqrt(rho2);
    const double alpha = atan2(c[2], rho) * 180.0 / ORC_PI;
    if (fabs(alpha) > ORC_POLE_DEG) return 0;
    double beta = atan2(c[1], c[0]) * 180.0 / ORC_PI;
    if (beta < 0.0) beta += 360.0;
    double fi = alpha + 90.0;
    double fj = beta;
    int i0 = (int)floor(fi);
    if (i0 > ORC_IMG_NA - 2) i0 = ORC_IMG_NA - 2;
    if (i0 < 0) i0 = 0;
    int j0 = (int)floor(fj);
    double ti = fi - (double)i0;
    double tj = fj - (double)j0;
    tj = MUT(15, 1.0 - tj, tj);
    j0 %= ORC_IMG_NB;
    int j1 = (j0 + 1) % ORC_IMG_NB;
    const double I00 = img[i0 * ORC_IMG_NB + j0], I01 = img[i0 * ORC_IMG_NB + j1];
    const double I10 = img[(i0 + 1) * ORC_IMG_NB + j0], I11 = img[(i0 + 1) * ORC_IMG_NB + j1];
    *val = (1 - ti) * (1 - tj) * I00 + (1 - ti) * tj * I01 + ti * (1 - tj) * I10 + ti * tj * I11;
    if (cell) { cell[0] = i0; cell[1] = j0; }
    if (grad) {
        const double dfi = (1 - tj) * (I10 - I00) + tj * (I11 - I01);   /* per degree of alpha */
        const double dfj = (1 - ti) * (I01 - I00) + ti * (I11 - I10);   /* per degree of beta */
        const double n2 = rho2 + c[2] * c[2];
        const double k = 180.0 / ORC_PI;
        /* d alpha / d c and d beta / d c (radians), from the atan2 forms */
        const double da0 = -c[2] * c[0] / (rho * n2), da1 = -c[2] * c[1] / (rho * n2), da2 = rho / n2;
        const double db0 = -c[1] / rho2, db1 = c[0] / rho2;
        grad[0] = k * (dfi * da0 + dfj * db0);
        grad[1] = k * (dfi * da1 + dfj * db1);
        grad[2] = k * (dfi * da2);
    }
    return 1;
}

/* Loss L = sum_v w_v r_v^2 at orientation q and its gradient with respect
 * to the lab-frame perturbation delta of R = exp([delta]x) R(q) at delta = 0.
 * Optionally J^T J (3x3) and J^T r.  w (may be NULL) weights directions. */
void orc_refine_eval(const float* img, const float* S_msr, const float* u, int64_t nv,
                     const double* q, const double* w, double* loss, double* grad,
                     double* JtJ, double* Jtr)
{
    double M[9];
    orc_quat_to_matrix(q, M);
    double L = 0.0, g[3] = {0, 0, 0}, H[9] = {0}, b[3] = {0, 0, 0};
    for (int64_t v = 0; v < nv; ++v) {
        const double ux = u[3 * v], uy = u[3 * v + 1], uz = u[3 * v + 2];
        double c[3];   /* c = R^T u */
        c[0] = (M[0] * ux + M[3] * uy) + M[6] * uz;
        c[1] = (M[1] * ux + M[4] * uy) + M[7] * uz;
        c[2] = (M[2] * ux + M[5] * uy) + M[8] * uz;
        double f, gc[3];
        if (!orc_bilinear(img, c, &f, gc, NULL)) continue;
        const double wv = w ? w[v] : 1.0;
        if (wv == 0.0) continue;
        const double r = (double)S_msr[v] - f;
        /* a = R gc (lab frame); dr/ddelta = -(a x u) */
        double a[3];
        a[0] = (M[0] * gc[0] + M[1] * gc[1]) + M[2] * gc[2];
        a[1] = (M[3] * gc[0] + M[4] * gc[1]) + M[5] * gc[2];
        a[2] = (M[6] * gc[0] + M[7] * gc[1]) + M[8] * gc[2];
        double J[3];
        const double sj = MUT(9, 1.0, -1.0);   /* times -1.0 is an exact negation */
        J[0] = sj * (a[1] * uz - a[2] * uy);
        J[1] = sj * (a[2] * ux - a[0] * uz);
        J[2] = sj * (a[0] * uy - a[1] * ux);
        L += wv * r * r;
        for (int i = 0; i < 3; ++i) {
            g[i] += wv * 2.0 * r * J[i];
            b[i] += wv * J[i] * r;
            for (int j = 0; j < 3; ++j) H[3 * i + j] += wv * J[i] * J[j];
        }
    }
    if (loss) *loss = L;
    if (grad) for (int i = 0; i < 3; ++i) grad[i] = g[i];
    if (JtJ) for (int i = 0; i < 9; ++i) JtJ[i] = H[i];
    if (Jtr) for (int i = 0; i < 3; ++i) Jtr[i] = b[i];
}

/* exp([delta]x) as a quaternion. */
static void orc_exp_quat(const double* d, double* q)
{
    const double th = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (th < 1e-300) { q[0] = 1; q[1] = q[2] = q[3] = 0; return; }
    const double s = sin(0.5 * th) / th;
    q[0] = cos(0.5 * th); q[1] = s * d[0]; q[2] = s * d[1]; q[3] = s * d[2];
}

/* Solve the symmetric 3x3 system A x = b by Cramer's rule (FP64). */
static int orc_solve3(const double* A, const double* b, double* x)
{
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6])
                     + A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(fabs(det) > 0.0)) { x[0] = x[1] = x[2] = 0; return 0; }
    for (int c = 0; c < 3; ++c) {
        double B[9];
        memcpy(B, A, sizeof(B));
        B[c] = b[0]; B[3 + c] = b[1]; B[6 + c] = b[2];
        x[c] = (B[0] * (B[4] * B[8] - B[5] * B[7]) - B[1] * (B[3] * B[8] - B[5] * B[6])
              + B[2] * (B[3] * B[7] - B[4] * B[6])) / det;
    }
    return 1;
}

/* `iters` Gauss-Newton steps from q0; q_out receives the final unit
 * quaternion (w >= 0) and loss_out the loss at it. */
void orc_refine(const float* img, const float* S_msr, const float* u, int64_t nv,
                const double* q0, int iters, double* q_out, double* loss_out)
{
    double q[4] = {q0[0], q0[1], q0[2], q0[3]};
    for (int it = 0; it < iters; ++it) {
        double H[9], b[3], L;
        orc_refine_eval(img, S_msr, u, nv, q, NULL, &L, NULL, H, b);
        const double lam = 1e-6 * (H[0] + H[4] + H[8]);
        H[0] += lam; H[4] += lam; H[8] += lam;
        double d[3];
        const double sg = MUT(18, 1.0, -1.0);
        double nb[3] = {sg * b[0], sg * b[1], sg * b[2]};
        orc_solve3(H, nb, d);
        double e[4], qn[4];
        orc_exp_quat(d, e);
        orc_quat_mul(e, q, qn);
        const double n = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int i = 0; i < 4; ++i) q[i] = qn[i] / n;
    }
    if (q[0] < 0) for (int i = 0; i < 4; ++i) q[i] = -q[i];
    for (int i = 0; i < 4; ++i) q_out[i] = q[i];
    if (loss_out) orc_refine_eval(img, S_msr, u, nv, q, NULL, loss_out, NULL, NULL, NULL);
}

/* Batch of ROIs (OpenMP over ROIs). */
void orc_refine_batch(const float* img, const float* S_msr, const float* u, int64_t nv, int64_t nroi,
                      const double* q0, int iters, double* q_out, double* loss_out, int threads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads > 0 ? threads : omp_get_max_threads())
#endif
    for (int64_t r = 0; r < nroi; ++r)
        orc_refine(img, S_msr + r * nv, u, nv, q0 + 4 * r, iters, q_out + 4 * r,
                   loss_out ? loss_out + r : NULL);
}

int orc_openmp_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Reciprocal-space signature (Eq. 2, the FSP method after Vurpillot et al.) */
/* F(k) = sum_w exp(-2 pi i k . x_w) over the centred positions x_w of a ROI */
/* on the cubic grid k_a = -k_max + i_a dk, i_a < L, dk = 2 k_max / (L - 1)   */
/* (the reciprocal-space cube [-k_max, k_max]^3 of the supplement's cost     */
/* section, L_D points per axis).  out[p] = |F(k_p)| for the grid points     */
/* given as flat indices (ix L + iy) L + iz; FP64 throughout.                */
/* ------------------------------------------------------------------------ */
void orc_fsp(const float* xc, int64_t nw, int L, double kmax, const int64_t* pts, int64_t npts, double* out)
{
    const double dk = 2.0 * kmax / (double)MUT(17, L, L - 1);
    for (int64_t p = 0; p < npts; ++p) {
        const int64_t f = pts[p];
        const int iz = (int)(f % L), iy = (int)((f / L) % L), ix = (int)(f / ((int64_t)L * L));
        const double kx = -kmax + ix * dk, ky = -kmax + iy * dk, kz = -kmax + iz * dk;
        double re = 0.0, im = 0.0;
        for (int64_t w = 0; w < nw; ++w) {
            const double ka = MUT(7, ky, kx), kb = MUT(7, kx, ky);
            const double ph = 2.0 * ORC_PI * (ka * (double)xc[3 * w] + kb * (double)xc[3 * w + 1] +
                                               kz * (double)xc[3 * w + 2]);
            re += cos(ph);
            im -= sin(ph);
        }
        out[p] = sqrt(re * re + im * im);
    }
}
