// cher_kernels.cu -- the hot path (steps a1-a5) as one fused kernel per tile
// of track steps, in FP64 and in FP32-bulk precision.
//
// A CTA owns a tile of `BLOCK` consecutive steps:
//   phase A  one thread per step: Cherenkov yield (CERENK, paper section
//            3.2; the FP32 path screens it in FP32 and takes the FP64 chain
//            wherever the count or the photons per bunch would not be
//            certain), bunch count nb = ceil(N / B), per-step constants
//            staged in shared memory; a CTA-wide exclusive scan of nb gives
//            every bunch of the tile a slot;
//   phase B  the CTA's threads stride over the tile's bunches (the paper's
//            sub-step loop, Appendix A, unrolled across threads): Philox
//            randoms, emission point / azimuth / wavelength, the rare
//            conditions first (Algorithm 2's hoisting becomes a per-lane
//            predicate), Snell + one fine-table index for n(h) and one
//            (height, sin^2) cell for both refraction corrections (the
//            single-search refactor of section 3.3.1 and the repeated-call
//            hoisting of Algorithm 3), the ground point and arrival time
//            (RAYBND, Appendix B listing), candidate spheres from the ground
//            grid, and warp-aggregated compaction of the crossings (TELOUT;
//            the hits kernels queue their crossings per warp and record
//            them 32 at a time, see flush_ring).
// In the persistent variant CTAs pull tiles from an atomic queue, so showers
// of very uneven size share one launch (the paper's independent-shower
// parallelism, section 2, inside one GPU).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "cher_device.cuh"
#include "cher_internal.h"

namespace cher {
namespace {

using namespace dev;

// ------------------------------------------------------------------------
// Per-step constants staged in shared memory for the bunch loop.
// ------------------------------------------------------------------------
template <class R>
struct alignas(16) Seg {
    R ux, uy, uz, L;
    R e1x, e1y, e2x, e2y;
    R e2z, cosc, sinc, inv_nb;
    R x0, y0, dz0, tseg;   // dz0 = z0 - h_obs, tseg = t0 - t_ref (FP64 differences)
    R inv_bc, w;
    // FP32 path: the low parts of tseg and dz0 (tseg + tseg_lo and dz0 +
    // dz0_lo are their FP64 values to ~2^-48), for the arrival time's
    // float-float sum (unused in FP64)
    float tseg_lo, dz0_lo;
    // the parts of the first two Philox rounds that depend on the step only
    // (philox_bunch)
    uint32_t ph_a, ph_b, ph_c, ph_d;
};

// ------------------------------------------------------------------------
// a1 in the FP32 path: the yield evaluated in single precision with a bound
// E on the rounding error of q = N / B.  When no integer lies within
// [q - E, q + E] the bunch count ceil(q) is certain and equals the FP64
// result; when the Cherenkov-threshold cancellation in the numerator is
// strong, or an integer is within reach, the exact FP64 chain decides.
// ------------------------------------------------------------------------
struct YieldF {
    int nb;
    bool valid;
    float g, eta, s2, N;
};

// The FP32 screen keeps its photon count only where the Cherenkov-threshold
// cancellation in the numerator loses at most a factor ~10 (num >= 0.1 of
// its terms) and the midpoint's cell of the fine table holds no layer
// boundary (there the density jumps, and the FP32 height's rounding would
// move eta by up to the jump times ~1e-4): its rounding then leaves the
// photons per bunch within ~5e-6 of the FP64 chain (a few 1e-7 of eta times
// A / num <= 11, plus the FP32 operations); elsewhere the FP64 chain
// computes them.  (Deferring only the photons of those steps to the hit
// path, with the count kept from the screen, measured slower: the FP64 chain
// there made the bunch loop spill.)
constexpr float kMildCancel = 0.1f;

// sign and zero tests on the bit pattern (no FP64 instruction)
__device__ __forceinline__ bool d_negative(double v) {
    const long long b = __double_as_longlong(v);
    return b < 0 && (b & 0x7fffffffffffffffLL) != 0;
}
__device__ __forceinline__ bool d_not_positive(double v) {
    const long long b = __double_as_longlong(v);
    return b < 0 || b == 0;
}

// The FP32 radial midpoint height in a curved atmosphere (xyf = {x0, y0,
// ux, uy}); its rounding (a few ulp of the correction) joins the bound.
__device__ __forceinline__ float curved_midpoint_f(const KParams &p, float hm, float L,
                                                   const float *xyf, float &err) {
    const float half = 0.5f * L;
    const float xm = xyf[0] + half * xyf[2], ym = xyf[1] + half * xyf[3];
    const float rho2 = xm * xm + ym * ym;
    const float Rp = hm + p.f.earth_radius;
    const float corr = rho2 / (sqrtf(rho2 + Rp * Rp) + Rp);
    err = 32.0f * 5.9604645e-8f * corr;
    return hm + corr;
}

__device__ __forceinline__ void step_yield_screened(const KParams &p, bool others_valid,
                                                    double z0, double len, double ekin, float uz,
                                                    YieldF &y, const float *xyf = nullptr,
                                                    const double *xyd = nullptr) {
    y.nb = 0;
    y.valid = false;
    y.g = y.eta = y.s2 = y.N = 0.0f;
    if (!others_valid || !finite_d(z0) || !finite_d(len) || !finite_d(ekin) || !finite_f(uz) ||
        d_negative(len) || d_not_positive(ekin))
        return;
    y.valid = true;
    const float u = 5.9604645e-8f;                       // 2^-24
    const float e = d2f_rn(ekin), L = d2f_rn(len);
    const float z = d2f_rn(z0);
    const float g = e * p.f.inv_me;
    const float gam = 1.0f + g, gam2 = gam * gam;
    float hm = z + (0.5f * L) * uz;
    float curv_err = 0.0f;
    if (xyf) hm = curved_midpoint_f(p, hm, L, xyf, curv_err);
    float hc = fminf(fmaxf(hm, 0.0f), p.f.h_max);
    const float x = hc * p.f.inv_dh;
    int k = static_cast<int>(x);
    k = k > p.n_fine - 2 ? p.n_fine - 2 : k;
    k = dbg_index(p, k, p.n_fine - 1, DBG_ETA);
    const float f = x - static_cast<float>(k);
    const float t0 = __ldg(p.eta32 + k), t1 = __ldg(p.eta32 + k + 1);
    const float eta = t0 + f * (t1 - t0);
    const float np1 = 1.0f + eta, np1sq = np1 * np1;
    const float a = eta * (2.0f + eta);
    const float A = a * gam2;
    const float num = A - np1sq;
    const float bg2 = g * (2.0f + g);
    const float den = bg2 * np1sq;
    const float s2 = num / den;
    const float KL = p.f.K * L;
    const float q = KL * s2 * p.f.inv_B;
    // rounding-error bound (first order, each term padded)
    const float d_eta = p.f.eta_slope * (6.0f * u * (fabsf(z) + L + p.f.dh) + curv_err) +
                        5.0f * u * eta;
    const float d_a = (2.0f + 2.0f * eta) * d_eta + 3.0f * u * a;
    const float d_A = gam2 * (d_a + 10.0f * u * a);
    const float d_B = 2.0f * np1 * d_eta + 3.0f * u * np1sq;
    const float d_num = d_A + d_B + u * (A + np1sq);
    const float d_s2 = d_num / den + fabsf(s2) * (12.0f * u + 2.0f * d_eta);
    const float E = 4.0f * (KL * p.f.inv_B * d_s2 + fabsf(q) * 8.0f * u) + 1e-30f;
    const float lo = q - E, hi = q + E;
    if (hi <= 0.0f) return;                              // below threshold for sure
    if (lo > 0.0f && ceilf(lo) == ceilf(hi) && num >= kMildCancel * (A + np1sq) &&
        fabsf(t1 - t0) <= p.f.eta_jump * t0 && hi < 4.0e6f) {
        y.nb = static_cast<int>(ceilf(hi));
        y.g = g;
        y.eta = eta;
        y.s2 = s2;
        y.N = KL * s2;
        return;
    }
    // exact FP64 chain (rare)
    Yield yd;
    step_yield(p, true, z0, len, ekin, static_cast<double>(uz), yd, xyd);
    y.valid = yd.valid;
    y.nb = yd.nb;
    y.g = static_cast<float>(yd.g);
    y.eta = static_cast<float>(yd.eta);
    y.s2 = static_cast<float>(yd.s2);
    y.N = static_cast<float>(yd.N);
}

// ------------------------------------------------------------------------
// a1 with a wavelength-dependent index, n(u) = 1 + eta kappa(u) with kappa
// linear in the wavenumber u = 1/lambda between nodes.  On each piece the
// Frank-Tamm integral of 1 - 1/(beta n)^2 is exact in closed form,
//     width (1 - 1/(beta^2 n_a n_b)) = width [e gamma^2 - (1 + e)] / [g (2 + g) (1 + e)],
//     e = e_a + e_b + e_a e_b,  e_a = eta kappa_a,
// and the Cherenkov threshold eta kappa = x_th = 1 / (gamma^2 beta (1 + beta))
// cuts at most one piece (kappa falls along the nodes), whose radiating
// fraction (e_a - x_th) / (e_a - e_b) ends at the threshold.  The step keeps
// the cumulative shares of the pieces for the bunches' wavelengths.
// ------------------------------------------------------------------------
template <class R>
struct alignas(16) SegD {
    R cdf[kDispMax - 1];     // cumulative shares (integral / piece width)
    R eta, beta;             // at the step midpoint
    R x_th;                  // the threshold's eta kappa, 1/beta - 1
    R frac_cut;              // the piece the threshold cuts: its radiating fraction
    int m_cut, pad;          // and index (disp_k - 1: none)
};

__device__ __forceinline__ double disp_piece(double x, double y, double gam2, double bg2) {
    const double xy = __dmul_rn(x, y);
    const double xpy = __dadd_rn(x, y);
    const double e = __dadd_rn(xpy, xy);
    const double np = __dadd_rn(1.0, e);
    const double A = __dmul_rn(e, gam2);
    const double num = __dsub_rn(A, np);
    const double den = __dmul_rn(bg2, np);
    const double S = __ddiv_rn(num, den);
    return S > 0.0 ? S : 0.0;
}

// the exact FP64 chain (same operation order as the oracle)
template <class R>
__device__ __forceinline__ void step_yield_disp(const KParams &p, bool others_valid, double z0,
                                                double len, double ekin, double uz, Yield &y,
                                                SegD<R> &D, const double *xy = nullptr) {
    y.nb = 0;
    y.valid = false;
    y.N = y.s2 = y.g = y.gam = y.eta = 0.0;
    if (!others_valid || !finite_d(z0) || !finite_d(len) || !finite_d(ekin) || !finite_d(uz) ||
        len < 0.0 || ekin <= 0.0)
        return;
    const double g = __dmul_rn(ekin, p.inv_me);
    const double gam = __dadd_rn(1.0, g);
    const double gam2 = __dmul_rn(gam, gam);
    const double half_len = __dmul_rn(0.5, len);
    const double dz = __dmul_rn(half_len, uz);
    double hm = __dadd_rn(z0, dz);
    if (xy) hm = curved_midpoint(p, hm, half_len, xy);
    const double eta = eta_exact_lookup(p, hm);
    const double two_g = __dadd_rn(2.0, g);
    const double bg2 = __dmul_rn(g, two_g);
    const double beta = __ddiv_rn(__dsqrt_rn(bg2), gam);
    const double onepb = __dadd_rn(1.0, beta);
    const double gb = __dmul_rn(gam2, beta);
    const double gbb = __dmul_rn(gb, onepb);
    const double x_th = __ddiv_rn(1.0, gbb);
    y.g = g;
    y.gam = gam;
    y.eta = eta;
    y.valid = true;
    double sum = 0.0, frac_cut = 1.0;
    int m_cut = p.disp_k - 1;
#pragma unroll
    for (int m = 0; m < kDispMax - 1; ++m) {
        if (m + 1 < p.disp_k) {
            const double ea = __dmul_rn(eta, p.kap[m]);
            const double eb = __dmul_rn(eta, p.kap[m + 1]);
            double v = 0.0;
            if (ea > x_th) {
                if (eb >= x_th) {
                    v = disp_piece(ea, eb, gam2, bg2);
                } else {
                    const double f = __ddiv_rn(__dsub_rn(ea, x_th), __dsub_rn(ea, eb));
                    v = __dmul_rn(f, disp_piece(ea, x_th, gam2, bg2));
                    m_cut = m;
                    frac_cut = f;
                }
            }
            sum = __dadd_rn(sum, v);
            D.cdf[m] = static_cast<R>(sum);
        }
    }
    D.eta = static_cast<R>(eta);
    D.beta = static_cast<R>(beta);
    D.x_th = static_cast<R>(x_th);
    D.frac_cut = static_cast<R>(frac_cut);
    D.m_cut = m_cut;
    if (!(sum > 0.0)) return;                  // below threshold over the whole band
    const double Ks = __dmul_rn(p.disp_Kd, sum);
    const double N = __dmul_rn(len, Ks);
    const double q = __dmul_rn(N, p.inv_B);
    if (!(q < 4194304.0)) {
        y.valid = false;
        return;
    }
    y.nb = static_cast<int>(ceil(q));
    y.N = N;
    y.s2 = sum;
}

// The FP32 screen: every piece whole (every node clearly above the
// threshold) and ceil(q) certain under the rounding bound, or every node
// clearly below it; anything else (a cut piece, strong cancellation, an
// integer within reach) takes the exact chain.
__device__ __forceinline__ void step_yield_screened_disp(const KParams &p, bool others_valid,
                                                         double z0, double len, double ekin,
                                                         float uz, YieldF &y, SegD<float> &D,
                                                         const float *xyf = nullptr,
                                                         const double *xyd = nullptr) {
    y.nb = 0;
    y.valid = false;
    y.g = y.eta = y.s2 = y.N = 0.0f;
    if (!others_valid || !finite_d(z0) || !finite_d(len) || !finite_d(ekin) || !finite_f(uz) ||
        d_negative(len) || d_not_positive(ekin))
        return;
    y.valid = true;
    const float u = 5.9604645e-8f;                       // 2^-24
    const float e = d2f_rn(ekin), L = d2f_rn(len);
    const float z = d2f_rn(z0);
    const float g = e * p.f.inv_me;
    const float gam = 1.0f + g, gam2 = gam * gam;
    float hm = z + (0.5f * L) * uz;
    float curv_err = 0.0f;
    if (xyf) hm = curved_midpoint_f(p, hm, L, xyf, curv_err);
    float hc = fminf(fmaxf(hm, 0.0f), p.f.h_max);
    const float x = hc * p.f.inv_dh;
    int k = static_cast<int>(x);
    k = k > p.n_fine - 2 ? p.n_fine - 2 : k;
    k = dbg_index(p, k, p.n_fine - 1, DBG_ETA);
    const float f = x - static_cast<float>(k);
    const float t0 = __ldg(p.eta32 + k), t1 = __ldg(p.eta32 + k + 1);
    const float eta = t0 + f * (t1 - t0);
    const float bg2 = g * (2.0f + g);
    const float beta = sqrtf(bg2) / gam;
    const float x_th = 1.0f / (gam2 * beta * (1.0f + beta));
    const float d_eta = p.f.eta_slope * (6.0f * u * (fabsf(z) + L + p.f.dh) + curv_err) +
                        5.0f * u * eta;
    const float tol_x = 64.0f * u * x_th;
    const float e_hi = eta * p.f.kap[0], e_lo = eta * p.f.kap_lo;
    const int K = p.disp_k;
    if (e_hi + p.f.kap[0] * d_eta + 4.0f * u * e_hi < x_th - tol_x) return;   // below, surely
    if (e_lo - p.f.kap_lo * d_eta - 4.0f * u * e_lo > x_th + tol_x) {
        float sum = 0.0f, dsum = 0.0f;
        bool mild = true;
#pragma unroll
        for (int m = 0; m < kDispMax - 1; ++m) {
            if (m + 1 < K) {
                const float ka = p.f.kap[m], kb = p.f.kap[m + 1];
                const float ea = eta * ka, eb = eta * kb;
                const float ee = (ea + eb) + ea * eb;
                const float B = 1.0f + ee, A = ee * gam2;
                const float num = A - B, den = bg2 * B;
                const float S = num / den;
                const float d_e = (ka + kb) * (1.0f + ee) * d_eta + 4.0f * u * ee;
                const float d_A = gam2 * (d_e + 10.0f * u * ee);
                const float d_B = d_e + 3.0f * u * B;
                const float d_num = d_A + d_B + u * (A + B);
                dsum += d_num / den + fabsf(S) * (12.0f * u + 2.0f * d_eta);
                mild = mild && num >= kMildCancel * (A + B);
                sum += S;
                D.cdf[m] = sum;
            }
        }
        const float KL = p.f.disp_Kd * L;
        const float q = KL * sum * p.f.inv_B;
        const float E = 4.0f * (KL * p.f.inv_B * dsum +
                                fabsf(q) * (8.0f + static_cast<float>(K)) * u) + 1e-30f;
        const float lo = q - E, hi = q + E;
        if (lo > 0.0f && ceilf(lo) == ceilf(hi) && mild && fabsf(t1 - t0) <= p.f.eta_jump * t0 &&
            hi < 4.0e6f) {
            y.nb = static_cast<int>(ceilf(hi));
            y.g = g;
            y.eta = eta;
            y.s2 = sum;
            y.N = KL * sum;
            D.eta = eta;
            D.beta = beta;
            D.x_th = x_th;
            D.frac_cut = 1.0f;
            D.m_cut = K - 1;
            return;
        }
    }
    Yield yd;
    step_yield_disp<float>(p, true, z0, len, ekin, static_cast<double>(uz), yd, D, xyd);
    y.valid = yd.valid;
    y.nb = yd.nb;
    y.g = static_cast<float>(yd.g);
    y.eta = static_cast<float>(yd.eta);
    y.s2 = static_cast<float>(yd.s2);
    y.N = static_cast<float>(yd.N);
}

// A bunch's wavelength from its step's spectrum (density 1 - 1/(beta n)^2
// in u over the radiating part of the band) by inversion of u2 from the
// band's short end: the piece m whose cumulative share first exceeds
// u2 * total, then the fraction t of its radiating width where
//     G(t) = t - t / (beta^2 n_a n(t)),  n(t) = n_a + b t
// equals the remaining share D' (the quadratic b t^2 + (n_a s_a^2 - D' b) t
// - D' n_a = 0, root 2 D' n_a / (P + sqrt(P^2 + 4 b D' n_a)), P = n_a s_a^2 -
// D' b >= 0 since b <= 0).  Returns lambda, kappa and the cone of the
// bunch's index at the step midpoint.  Near the threshold 1 - 1/(beta n)^2
// cancels; with beta n - 1 = beta (eta kappa - x_th), x_th = 1/beta - 1,
//     s^2 = b_d (2 + b_d) / (1 + b_d)^2,  cos = 1 - b_d / (1 + b_d),
//     b_d = beta (eta kappa - x_th),
// neither does, and the cosine keeps half an ulp through approximate
// divisions.
template <class R>
__device__ __forceinline__ void disp_sample(const KParams &p, const SegD<R> &D, R u2, R &lam,
                                            R &kap, R &cosc, R &sinc) {
    const int K = p.disp_k;
    const R T = u2 * D.cdf[K - 2];
    int m = 0;
#pragma unroll
    for (int i = 0; i < kDispMax - 2; ++i) m += (i < K - 2 && !(T < D.cdf[i]));
    const R acc = m > 0 ? D.cdf[m - 1] : R(0);
    const bool cut = m == D.m_cut;
    const R frac = cut ? D.frac_cut : R(1);
    R ka, kb, u1, du;
    if constexpr (std::is_same<R, float>::value) {
        ka = __ldg(p.kap32 + m);
        kb = __ldg(p.kap32 + m + 1);
        u1 = p.f.disp_u1;
        du = p.f.disp_du;
    } else {
        ka = __ldg(p.kap64 + m);
        kb = __ldg(p.kap64 + m + 1);
        u1 = p.disp_u1;
        du = p.disp_du;
    }
    const R ea = D.eta * ka;
    const R x_end = cut ? D.x_th : D.eta * kb;
    R Dl = T - acc;
    Dl = Dl > R(0) ? Dl : R(0);
    const R Dp = cut ? (frac > R(0) ? Dl / frac : R(0)) : Dl;
    const R na = R(1) + ea;
    const R bda = D.beta * (ea - D.x_th);
    R s2a = bda * (R(2) + bda) / ((R(1) + bda) * (R(1) + bda));
    s2a = s2a > R(0) ? s2a : R(0);
    const R b = x_end - ea;
    const R P = na * s2a - Dp * b;
    R disc = P * P + R(4) * b * Dp * na;
    disc = disc > R(0) ? disc : R(0);
    const R den = P + sqrt(disc);
    R t = den > R(0) ? (R(2) * Dp * na) / den : R(0);
    t = t < R(1) ? t : R(1);
    t = t > R(0) ? t : R(0);
    const R sm = t * frac;
    kap = ka + sm * (kb - ka);
    lam = R(1) / (u1 - (static_cast<R>(m) + sm) * du);
    const R bd = D.beta * (D.eta * kap - D.x_th);
    R s2 = bd * (R(2) + bd) / ((R(1) + bd) * (R(1) + bd));
    s2 = s2 > R(0) ? s2 : R(0);
    sinc = sqrt(s2);
    cosc = R(1) - bd / (R(1) + bd);
}

template <class R>
__device__ __forceinline__ R load_dir(const void *p, int64_t i) {
    return __ldg(static_cast<const R *>(p) + i);
}

template <class R, class Y>
__device__ __forceinline__ void prep_step(const KParams &p, int64_t i, const Y &y, Seg<R> &S) {
    const R ux = load_dir<R>(p.ux, i);
    const R uy = load_dir<R>(p.uy, i);
    const R uz = load_dir<R>(p.uz, i);
    double t_ref = 0.0;
    if (p.t_ref) {
        const uint32_t sh = p.shower ? __ldg(p.shower + i) : 0u;
        if (static_cast<int32_t>(sh) < p.n_showers) t_ref = __ldg(p.t_ref + sh);
    }
    {
        // counter (lo(g), hi(g), j, 0): round 1 multiplies word 0 (the step's)
        // and word 2 (j); round 2 multiplies round 1's word 2, which is the
        // step's again
        const uint64_t g = static_cast<uint64_t>(p.track_base + i);
        const uint32_t glo = static_cast<uint32_t>(g), ghi = static_cast<uint32_t>(g >> 32);
        const uint32_t lo0 = 0xD2511F53u * glo, hi0 = __umulhi(0xD2511F53u, glo);
        const uint32_t w2 = hi0 ^ p.rk1[0];                      // c1.z (c.w = 0)
        const uint32_t lo1 = 0xCD9E8D57u * w2, hi1 = __umulhi(0xCD9E8D57u, w2);
        S.ph_a = ghi ^ p.rk0[0];         // round 1: c1.x = hi(M1 j) ^ ph_a
        S.ph_b = hi1 ^ p.rk0[1];         // round 2: c2.x = ph_b ^ c1.y
        S.ph_c = lo1;                    //          c2.y
        S.ph_d = lo0 ^ p.rk1[1];         //          c2.z = hi(M0 c1.x) ^ ph_d
    }
    S.ux = ux;
    S.uy = uy;
    S.uz = uz;
    // the two absolute differences stay in FP64 (tens of km, ~1e5 ns); the
    // FP32 path rounds to float on the integer pipes (GB300's FP64 pipe,
    // which converts too, runs at 1/64 of the FP32 rate)
    if constexpr (std::is_same<R, float>::value) {
        S.L = d2f_rn(__ldg(p.len + i));
        S.x0 = d2f_rn(__ldg(p.x0 + i));
        S.y0 = d2f_rn(__ldg(p.y0 + i));
        d2f_split(__ldg(p.z0 + i) - p.h_obs, S.dz0, S.dz0_lo);
        d2f_split(__ldg(p.t0 + i) - t_ref, S.tseg, S.tseg_lo);
    } else {
        S.L = __ldg(p.len + i);
        S.x0 = __ldg(p.x0 + i);
        S.y0 = __ldg(p.y0 + i);
        S.dz0 = __ldg(p.z0 + i) - p.h_obs;
        S.tseg = __ldg(p.t0 + i) - t_ref;
        S.tseg_lo = S.dz0_lo = 0.0f;
    }
    // azimuth basis around the step: e1 horizontal, e2 = d x e1
    R e1x, e1y;
    const R rho2 = ux * ux + uy * uy;
    if (rho2 > R(1e-20)) {
        const R inv = R(1) / sqrt(rho2);
        e1x = -uy * inv;
        e1y = ux * inv;
    } else {
        e1x = R(1);
        e1y = R(0);
    }
    S.e1x = e1x;
    S.e1y = e1y;
    S.e2x = -uz * e1y;
    S.e2y = uz * e1x;
    S.e2z = ux * e1y - uy * e1x;
    if (y.nb > 0) {
        // beta = sqrt(g (2 + g)) / gamma ; cos = 1 / (beta n) ; sin = sqrt(s2)
        const R g = static_cast<R>(y.g);
        const R beta = sqrt(g * (R(2) + g)) / (R(1) + g);
        const R inv_nb = R(1) / static_cast<R>(y.nb);
        if constexpr (std::is_same<R, float>::value) {
            // cos = 1/(beta n) = 1 - b_d / (1 + b_d), b_d = beta n - 1 = beta (eta - x_th),
            // x_th = 1/beta - 1 = 1 / (gamma^2 beta (1 + beta)): half an ulp through the
            // approximate divisions and square roots (1/(beta n) directly: ~6 ulp, which
            // the arrival time at large zenith, ~1e5 ns of path, feels)
            const float gam = 1.0f + g;
            const float x_th = 1.0f / (gam * gam * beta * (1.0f + beta));
            const float bd = beta * (y.eta - x_th);
            S.cosc = 1.0f - bd / (1.0f + bd);
        } else {
            S.cosc = R(1) / (beta * (R(1) + static_cast<R>(y.eta)));
        }
        S.sinc = sqrt(static_cast<R>(y.s2));
        S.inv_nb = inv_nb;
        S.inv_bc = R(1) / (beta * R(kC));
        if constexpr (std::is_same<R, float>::value)
            S.w = static_cast<float>(y.N) * inv_nb;
        else
            S.w = y.N / static_cast<double>(y.nb);
    } else {
        S.cosc = S.sinc = S.inv_nb = S.inv_bc = S.w = R(0);
    }
}

// ------------------------------------------------------------------------
// Longitudinal production profile (CERLDE, paper section 4).  A step's
// photons are spread uniformly along its path and counted at the depth of
// their emission point, X = T(h) / cos(axis zenith); the step adds to each
// depth bin its photons times the fraction of its path inside the bin.
// Depth falls monotonically with height, so the fractions are differences
// of bin-edge heights, from the inverse of the layer formula.
// ------------------------------------------------------------------------
__device__ __forceinline__ float atm_thickness(const KParams &p, float h) {
    if (!(h < p.f.hb[5])) return 0.0f;
    float a = p.f.a[0], b = p.f.b[0], ic = p.f.inv_c[0];
#pragma unroll
    for (int l = 1; l < 5; ++l)
        if (h >= p.f.hb[l]) { a = p.f.a[l]; b = p.f.b[l]; ic = p.f.inv_c[l]; }
    return a + b * __expf(-(h * ic));
}

__device__ __forceinline__ double atm_thickness(const KParams &p, double h) {
    if (!(h < p.atm.hb[5])) return 0.0;
    double a = p.atm.a[0], b = p.atm.b[0], c = p.atm.c[0];
#pragma unroll
    for (int l = 1; l < 5; ++l)
        if (h >= p.atm.hb[l]) { a = p.atm.a[l]; b = p.atm.b[l]; c = p.atm.c[l]; }
    return a + b * exp(-(h / c));
}

// the height in [lo, hi] where the thickness is tau: the lowest layer whose
// top thickness is <= tau holds it (tau below the last layer's top: the
// jump to T = 0 at the top of the atmosphere)
__device__ __forceinline__ float atm_height(const KParams &p, float tau, float lo, float hi) {
    float h = p.f.hb[5];
    if (tau >= p.f.t_top[4]) {
        float a = p.f.a[4], b = p.f.b[4], c = p.f.c[4], h0 = p.f.hb[4], h1 = p.f.hb[5];
#pragma unroll
        for (int l = 3; l >= 0; --l)
            if (tau >= p.f.t_top[l]) {
                a = p.f.a[l]; b = p.f.b[l]; c = p.f.c[l]; h0 = p.f.hb[l]; h1 = p.f.hb[l + 1];
            }
        h = fminf(fmaxf(-c * __logf((tau - a) / b), h0), h1);
    }
    return fminf(fmaxf(h, lo), hi);
}

__device__ __forceinline__ double atm_height(const KParams &p, double tau, double lo, double hi) {
    double h = p.atm.hb[5];
    if (tau >= p.atm.t_top[4]) {
        double a = p.atm.a[4], b = p.atm.b[4], c = p.atm.c[4], h0 = p.atm.hb[4],
               h1 = p.atm.hb[5];
#pragma unroll
        for (int l = 3; l >= 0; --l)
            if (tau >= p.atm.t_top[l]) {
                a = p.atm.a[l]; b = p.atm.b[l]; c = p.atm.c[l]; h0 = p.atm.hb[l];
                h1 = p.atm.hb[l + 1];
            }
        h = fmin(fmax(-c * log((tau - a) / b), h0), h1);
    }
    return fmin(fmax(h, lo), hi);
}

// One FP64 atomic per bin the step touches (one for most steps: 20 m of
// path is ~2 g/cm^2 at 8 km).  Combining equal bins across the warp first
// measured slower (+14 % against +6 % of the launch).
template <class R>
__device__ __forceinline__ void profile_step(const KParams &p, int64_t i, R N) {
    const uint32_t sh = p.shower ? __ldg(p.shower + i) : 0u;
    if (sh >= static_cast<uint32_t>(p.prof_rows)) return;
    const R uz = load_dir<R>(p.uz, i);
    const R za = static_cast<R>(__ldg(p.z0 + i));
    const R zb = za + static_cast<R>(__ldg(p.len + i)) * uz;
    const R lo = za < zb ? za : zb, hi = za < zb ? zb : za;
    const R cz = p.prof_cos ? static_cast<R>(__ldg(p.prof_cos + sh)) : R(1);
    R dx, inv_dx;
    if constexpr (std::is_same<R, float>::value) {
        dx = p.f.prof_dx;
        inv_dx = p.f.prof_inv_dx;
    } else {
        dx = p.prof_dx;
        inv_dx = p.prof_inv_dx;
    }
    const R kt = floor(atm_thickness(p, hi) / cz * inv_dx);   // shallowest point's bin
    const R kb = floor(atm_thickness(p, lo) / cz * inv_dx);   // deepest point's bin
    const R nbins = static_cast<R>(p.prof_bins);
    if (!(kt >= R(0) && kt < nbins)) return;
    double *row = p.prof + static_cast<int64_t>(sh) * p.prof_bins;
    if (!(hi > lo) || kt == kb) {
        atomicAdd(row + static_cast<int>(kt), static_cast<double>(N));
        return;
    }
    const int k_last = static_cast<int>(kb < nbins - R(1) ? kb : nbins - R(1));
    const R inv_span = R(1) / (hi - lo);
    R h_up = hi;
    for (int k = static_cast<int>(kt); k <= k_last; ++k) {
        const R h_dn = static_cast<R>(k) == kb
                           ? lo
                           : atm_height(p, static_cast<R>(k + 1) * dx * cz, lo, hi);
        atomicAdd(row + k, static_cast<double>(N * ((h_up - h_dn) * inv_span)));
        h_up = h_dn;
    }
}

// ------------------------------------------------------------------------
// Atmospheric transmission: the vertical optical depth tau(lambda, h)
// interpolated bilinearly in its table (clamped to the nodes).
// ------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ R trans_tau(const KParams &p, R lam, R h) {
    R xl, xh;
    if constexpr (std::is_same<R, float>::value) {
        xl = (lam - p.f.trans_l0) * p.f.trans_lscale;
        xh = (h - p.f.trans_h0) * p.f.trans_hscale;
    } else {
        xl = (lam - p.trans_l0) * p.trans_lscale;
        xh = (h - p.trans_h0) * p.trans_hscale;
    }
    const int nl = p.trans_nl, nh = p.trans_nh;
    xl = fmin(fmax(xl, R(0)), static_cast<R>(nl - 1));
    xh = fmin(fmax(xh, R(0)), static_cast<R>(nh - 1));
    const int a = min(static_cast<int>(xl), nl - 2), b = min(static_cast<int>(xh), nh - 2);
    const R s = xl - static_cast<R>(a), t = xh - static_cast<R>(b);
    const R *T = static_cast<const R *>(p.trans) + a * nh + b;
    const R t00 = __ldg(T), t01 = __ldg(T + 1), t10 = __ldg(T + nh), t11 = __ldg(T + nh + 1);
    return (R(1) - s) * ((R(1) - t) * t00 + t * t01) + s * ((R(1) - t) * t10 + t * t11);
}

// ------------------------------------------------------------------------
// a2 + a3: one bunch, from the Philox block to the ground.
// ------------------------------------------------------------------------
template <class R>
struct BunchOut {
    R X, Y, cx, cy, cz, t, he, lam;
    R kap;               // (n - 1) scale at the bunch's wavelength
    R c2;                // cos^2 of the arrival zenith (queued fallback bunches)
    R zg;                // arrival z - h_obs (curved atmosphere; 0 in flat layers)
    R tsec;              // FP32 hits path: 1 / cos(theta_obs), t holds the time's
                         // small part (the float-float sum is formed on the hit path)
    int status;
};

// The FP32 arrival time at h_obs minus t_ref, summed in float-float.  With
// Lp = sec (dz0 + m) the optical path (m = fl u_z + A_l sec^2, the part
// beyond the step's own height above h_obs) the time is
//     t = tseg + fl / (beta c) + Lp / c
//       = [tseg + (sec dz0) / c] + [fl / (beta c) + sec m / c],
// two large terms of opposite sign (tens of km of path against the step's
// time before the shower front, ~1e5 ns each) and a small one r.  The large
// ones are formed exactly: tseg and dz0 come as float pairs split from their
// FP64 values (prep_step), 1/c as a float pair, the products sec dz0 and
// (sec dz0) (1/c) with their FMA-exact rounding errors, their sum with tseg
// by Knuth's two-sum; the rounding errors, the low parts and r are added
// last.  r is formed where the bunch is propagated.  (Explicitly rounded
// operations: no contraction into FMAs may touch the error-free
// transforms.)
constexpr double kInvC = 1.0 / kC;
constexpr float kInvC_hi = static_cast<float>(kInvC);
constexpr float kInvC_lo = static_cast<float>(kInvC - static_cast<double>(kInvC_hi));

__device__ __forceinline__ float arrival_time_ff(const Seg<float> &S, float sec, float r) {
    const float P = __fmul_rn(sec, S.dz0);
    const float Pe = fmaf(sec, S.dz0, -P);
    const float Q = __fmul_rn(P, kInvC_hi);
    const float Qe = fmaf(P, kInvC_hi, -Q);
    const float s = __fadd_rn(S.tseg, Q);
    const float bb = __fsub_rn(s, S.tseg);
    const float se = __fadd_rn(__fsub_rn(S.tseg, __fsub_rn(s, bb)), __fsub_rn(Q, bb));
    const float lo = (P * kInvC_lo + (Pe + sec * S.dz0_lo) * kInvC_hi) + S.tseg_lo;
    return s + (((se + Qe) + lo) + r);
}

template <class R>
struct Consts {
    R h_obs, dH_max, eta_o, inv_np1o, q_max, inv_dht, inv_dq, inv_dh, lam_inv1, lam_dinv;
    R gx0[2], gy0[2], inv_gcs[2], q_band, fb_q;
    int H, Z, n_fine;
};

template <class R>
__device__ __forceinline__ R eta_at(const KParams &p, const Consts<R> &c, R h) {
    R x = h * c.inv_dh;
    x = x < R(0) ? R(0) : x;
    int k = static_cast<int>(x);
    k = k > c.n_fine - 2 ? c.n_fine - 2 : k;
    k = dbg_index(p, k, p.n_fine - 1, DBG_ETA);
    const R f = x - static_cast<R>(k);
    R t0, t1;
    if constexpr (std::is_same<R, float>::value) {
        t0 = __ldg(p.eta32 + k);
        t1 = __ldg(p.eta32 + k + 1);
    } else {
        t0 = __ldg(p.eta64 + k);
        t1 = __ldg(p.eta64 + k + 1);
    }
    return t0 + f * (t1 - t0);
}

// the per-launch constants of the bunch loop in the path's precision
template <class R>
__device__ __forceinline__ void make_consts(const KParams &p, Consts<R> &c, R &np1o) {
    if constexpr (std::is_same<R, float>::value) {
        c.h_obs = p.f.h_obs;
        c.dH_max = p.f.dH_max;
        c.eta_o = p.f.eta_o;
        c.inv_np1o = p.f.inv_np1o;
        c.q_max = p.f.q_max;
        c.inv_dht = p.f.inv_dht;
        c.inv_dq = p.f.inv_dq;
        c.inv_dh = p.f.inv_dh;
        c.lam_inv1 = p.f.lam_inv1;
        c.lam_dinv = p.f.lam_dinv;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            c.gx0[g] = p.f.gx0[g];
            c.gy0[g] = p.f.gy0[g];
            c.inv_gcs[g] = p.f.inv_gcs[g];
        }
        c.q_band = p.f.q_band;
        c.fb_q = p.f.fb_q;
        np1o = p.f.np1o;
    } else {
        c.h_obs = p.h_obs;
        c.dH_max = p.h_max - p.h_obs;
        c.eta_o = p.eta_obs;
        c.inv_np1o = 1.0 / (1.0 + p.eta_obs);
        c.q_max = p.q_max;
        c.inv_dht = p.inv_dht;
        c.inv_dq = p.inv_dq;
        c.inv_dh = p.inv_dh;
        c.lam_inv1 = p.lam_inv1;
        c.lam_dinv = p.lam_dinv;
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            c.gx0[g] = p.grid[g].x0;
            c.gy0[g] = p.grid[g].y0;
            c.inv_gcs[g] = p.grid[g].inv_cs;
        }
        c.q_band = p.q_band;
        c.fb_q = p.fb_q;
        np1o = 1.0 + p.eta_obs;
    }
    c.H = p.H;
    c.Z = p.Z;
    c.n_fine = p.n_fine;
}

// ------------------------------------------------------------------------
// Beyond-table fallback (the paper's scalar path for the photons that do
// not fit the vectorised one, section 3.3.1): the ray integrals
//   D = int tan(theta(h)) dh,  L = int n(h) / cos(theta(h)) dh  over
//   [h_obs, h_e], n(h) sin(theta(h)) = n_obs sin(theta_obs),
// in FP64 with the exact layered n(h), 12-point Gauss-Legendre on each
// layer's part of the interval (the integrands are smooth inside a layer).
// ------------------------------------------------------------------------
__device__ __forceinline__ double eta_layer(const KParams &p, double h) {
    if (!(h < p.atm.hb[5])) return 0.0;
    double e = p.atm.eta_coef[0], ic = p.atm.inv_c[0];
#pragma unroll
    for (int l = 1; l < 5; ++l)
        if (h >= p.atm.hb[l]) { e = p.atm.eta_coef[l]; ic = p.atm.inv_c[l]; }
    return e * exp(-(h * ic));
}

__device__ void ray_integrals(const KParams &p, double h_e, double s_obs, double kap, double &D,
                              double &L) {
    const double K = (1.0 + kap * eta_layer(p, p.h_obs)) * s_obs;
    D = 0.0;
    L = 0.0;
    double a = p.h_obs;
    for (int l = 0; l < 5 && a < h_e; ++l) {
        const double top = l < 4 ? p.atm.hb[l + 1] : h_e;
        if (!(top > a)) continue;
        const double b = top < h_e ? top : h_e;
        const double half = 0.5 * (b - a), mid = 0.5 * (a + b);
        for (int q = 0; q < 12; ++q) {
            const double n = 1.0 + kap * eta_layer(p, mid + half * p.gl_x[q]);
            const double sn = K / n;
            const double inv_c = rsqrt(1.0 - sn * sn);
            D += p.gl_w[q] * half * sn * inv_c;
            L += p.gl_w[q] * half * n * inv_c;
        }
        a = b;
    }
}

// The same integrals for the FP32 path, in FP32: the straight line at the
// observation-level zenith plus the integrals of the corrections,
//   D = dh tan(theta_o) + int (tan(theta) - tan(theta_o)),
//   L = dh / cos(theta_o) + int (n / cos(theta) - 1 / cos(theta_o)),
// whose integrands are small and written without cancellation: with
// delta = (n_o - n) / n, sin(theta) = s_o (1 + delta) and
//   cos_o - cos = s_o^2 delta (2 + delta) / (cos_o + cos),
//   tan - tan_o = s_o [delta cos_o + (cos_o - cos)] / (cos cos_o),
//   n / cos - 1 / cos_o = [(n - 1) cos_o + (cos_o - cos)] / (cos cos_o).
// cos_o^2 comes in as computed from the vertical cosine (full relative
// precision at large zenith).
__device__ __forceinline__ float eta_layer_f(const KParams &p, float h) {
    if (!(h < p.f.hb[5])) return 0.0f;
    float e = p.f.eta_coef[0], ic = p.f.inv_c[0];
#pragma unroll
    for (int l = 1; l < 5; ++l)
        if (h >= p.f.hb[l]) { e = p.f.eta_coef[l]; ic = p.f.inv_c[l]; }
    return e * __expf(-(h * ic));
}

__device__ void ray_integrals_f(const KParams &p, float dh, float s_o, float c2o, float kap,
                                float &D, float &L) {
    const float c_o = sqrtf(c2o);
    const float inv_co = 1.0f / c_o;
    const float s2o = s_o * s_o;
    const float eta_o = kap * eta_layer_f(p, p.f.h_obs);
    const float h_e = p.f.h_obs + dh;
    float Dc = 0.0f, Lc = 0.0f;
    float a = p.f.h_obs;
    for (int l = 0; l < 5 && a < h_e; ++l) {
        const float top = l < 4 ? p.f.hb[l + 1] : h_e;
        if (!(top > a)) continue;
        const float b = top < h_e ? top : h_e;
        const float half = 0.5f * (b - a), mid = 0.5f * (a + b);
        float sx = 0.0f, sl = 0.0f;
#pragma unroll 4
        for (int q = 0; q < 12; ++q) {
            const float eh = kap * eta_layer_f(p, mid + half * p.f.gl_x[q]);
            const float del = (eta_o - eh) / (1.0f + eh);
            const float g = s2o * (del * (2.0f + del));
            const float c = sqrtf(c2o - g);
            const float dc = g / (c_o + c);                 // cos_o - cos
            const float inv = 1.0f / (c * c_o);
            sx += p.f.gl_w[q] * ((s_o * (del * c_o + dc)) * inv);
            sl += p.f.gl_w[q] * ((eh * c_o + dc) * inv);
        }
        Dc += half * sx;
        Lc += half * sl;
        a = b;
    }
    D = dh * s_o * inv_co + Dc;
    L = dh * inv_co + Lc;
}

// One queued bunch: its emission point and time, the horizontal direction,
// sine and squared cosine of its observation-level zenith, wavelength, its
// index's scale kappa, photons and key.
template <class R>
struct alignas(16) FbEntry {
    R xe, ye, he, dh, te, hx, hy, s_obs, c2, lam, w, kap;   // dh = h_e - h_obs
    uint64_t key;                                  // the record key (step << 32 | j)
    uint32_t step_hi;                              // bits 32.. of the global step index
};

// ------------------------------------------------------------------------
// a3 in a curved atmosphere (spherical shells around C = (0, 0, -R_E) in the
// core frame, Bouguer's invariant n r sin(zeta)): the emission point's
// radial height and local vertical; the photon's angle to it (sine as
// |p x r^|, exact at small angles); sin(zeta_o) = sin(zeta_e) (r_e / r_o)
// (n_e / n_o); the central angle and optical path of the straight line that
// arrives at zeta_o (closed forms, below) plus the tables' corrections
// (central angle; (n - 1) and geometric parts of the optical path, each
// times the path average of its first-order factor along that line); the
// arrival point x_e + (r_o cos(phi) - r_e) r^ + r_o sin(phi) t^ and
// direction -cos(zeta_o) r^_o + sin(zeta_o) t^_o in the plane of the centre.
// Every difference of nearly equal terms is written out: h_e - h_obs =
// (z - h_obs) + rho^2 / (r_e + z + R_E), 1 - u = (h_e - h_obs) / r_e,
// cos_e'^2 = cos_o^2 + sin_o^2 (1 - u)(1 + u), 1 - cos(phi) = sin^2 / (1 + cos).
// ------------------------------------------------------------------------
template <class R, bool TR, bool DS>
__device__ __forceinline__ void propagate_curved(const KParams &p, const Consts<R> &c,
                                                 const Seg<R> &S, R fl, R px, R py, R pz,
                                                 uint32_t w3, BunchOut<R> &o) {
    R r_o, inv_ro, inv_dsec;
    if constexpr (std::is_same<R, float>::value) {
        r_o = p.f.r_o;
        inv_ro = p.f.inv_ro;
        inv_dsec = p.f.inv_dsec;
    } else {
        r_o = p.r_o;
        inv_ro = p.inv_ro;
        inv_dsec = p.inv_dsec;
    }
    const R xe = S.x0 + fl * S.ux, ye = S.y0 + fl * S.uy;
    const R dze = S.dz0 + fl * S.uz;                     // z - h_obs in the core frame
    const R Rp = dze + r_o;
    const R rho2 = xe * xe + ye * ye;
    const R r_e = sqrt(rho2 + Rp * Rp);
    const R dH = dze + rho2 / (r_e + Rp);                // radial height above h_obs
    o.he = c.h_obs + dH;
    const R inv_re = R(1) / r_e;
    const R rx = xe * inv_re, ry = ye * inv_re, rz = Rp * inv_re;
    const R ce = px * rx + py * ry + pz * rz;           // cosine to the upward vertical
    if (!(ce < R(0))) { o.status = ST_UPWARD; return; }
    if (!(dH >= R(0))) { o.status = ST_BELOW; return; }
    if (!(dH <= c.dH_max)) { o.status = ST_ABOVE; return; }
    const R wx = py * rz - pz * ry, wy = pz * rx - px * rz, wz = px * ry - py * rx;
    const R se2 = wx * wx + wy * wy + wz * wz;
    const R eta_e = eta_at<R>(p, c, o.he);
    R rm1;
    if constexpr (DS)
        rm1 = o.kap * (eta_e - c.eta_o) / (R(1) + o.kap * c.eta_o);
    else
        rm1 = (eta_e - c.eta_o) * c.inv_np1o;
    const R gb = (R(1) + dH * inv_ro) * (R(1) + rm1);
    const R q = se2 * gb * gb;                           // sin^2(zeta_o)
    if (!(q <= c.q_max)) { o.status = ST_ANGLE; return; }
    const R omq = R(1) - q;
    const R sec = rsqrt(omq);
    const R co = omq * sec;
    const R so = sqrt(q);
    // one cell: heights in rows, zeniths uniform in sec
    const R fj = dH * c.inv_dht;
    int jj = static_cast<int>(fj);
    jj = jj > c.H - 2 ? c.H - 2 : jj;
    const R a = fj - static_cast<R>(jj);
    const R fk = (sec - R(1)) * inv_dsec;
    int kk = static_cast<int>(fk);
    kk = kk > c.Z - 2 ? c.Z - 2 : kk;
    const R b = fk - static_cast<R>(kk);
    const size_t e0 = dbg_index(p, static_cast<size_t>(jj) * (c.Z - 1) + kk,
                                int64_t(c.H - 1) * (c.Z - 1), DBG_TAB);
    const size_t e1 = dbg_index(p, e0 + (c.Z - 1), int64_t(c.H) * (c.Z - 1), DBG_TAB);
    R v[2][6];                  // rows jj, jj + 1: ax_k, al_k, ax_k1, al_k1, ag_k, ag_k1
    if constexpr (std::is_same<R, float>::value) {
        const float4 *T = static_cast<const float4 *>(DS ? p.tabd : p.tab);
        const int per = DS ? 4 : 2;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const size_t e = r ? e1 : e0;
            float4 A = __ldg(T + per * e), B = __ldg(T + per * e + 1);
            if constexpr (DS) {
                const float wk = (o.kap - p.f.kap_lo) * p.f.kap_winv;
                const float4 A2 = __ldg(T + per * e + 2), B2 = __ldg(T + per * e + 3);
                A = make_float4(A.x + wk * (A2.x - A.x), A.y + wk * (A2.y - A.y),
                                A.z + wk * (A2.z - A.z), A.w + wk * (A2.w - A.w));
                B = make_float4(B.x + wk * (B2.x - B.x), B.y + wk * (B2.y - B.y), 0.0f, 0.0f);
            }
            v[r][0] = A.x; v[r][1] = A.y; v[r][2] = A.z; v[r][3] = A.w;
            v[r][4] = B.x; v[r][5] = B.y;
        }
    } else {
        const double2 *T = static_cast<const double2 *>(DS ? p.tabd : p.tab);
        const int per = DS ? 8 : 4;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const size_t e = r ? e1 : e0;
            double2 A = __ldg(T + per * e), B = __ldg(T + per * e + 1);
            double2 C = __ldg(T + per * e + 2);
            if constexpr (DS) {
                const double wk = (o.kap - p.kap_lo) * p.kap_winv;
                const double2 A2 = __ldg(T + per * e + 4), B2 = __ldg(T + per * e + 5);
                const double2 C2 = __ldg(T + per * e + 6);
                A = make_double2(A.x + wk * (A2.x - A.x), A.y + wk * (A2.y - A.y));
                B = make_double2(B.x + wk * (B2.x - B.x), B.y + wk * (B2.y - B.y));
                C = make_double2(C.x + wk * (C2.x - C.x), C.y + wk * (C2.y - C.y));
            }
            v[r][0] = A.x; v[r][1] = A.y; v[r][2] = B.x; v[r][3] = B.y;
            v[r][4] = C.x; v[r][5] = C.y;
        }
    }
    R t3[6];
#pragma unroll
    for (int m = 0; m < 6; ++m) t3[m] = v[0][m] + a * (v[1][m] - v[0][m]);
    const R Ax = t3[0] + b * (t3[2] - t3[0]);
    const R A1 = t3[1] + b * (t3[3] - t3[1]);
    const R A2 = t3[4] + b * (t3[5] - t3[4]);
    // the straight line arriving at zeta_o
    const R u = R(1) / (R(1) + dH * inv_ro);            // r_o / r_e
    const R omu = dH * inv_re;                           // 1 - u
    const R ce2 = sqrt(omq + q * omu * (R(1) + u));     // its cosine at r_e
    const R g1 = (R(1) + u) / (ce2 + u * co);
    const R gphi = u * so * g1 / (co * ce2);
    const R g2 = g1 * q * u / (ce2 * co);
    const R dphi = Ax * gphi * inv_ro;
    const R L = dH * g1 + A1 * g1 + A2 * g2;
    const R sps = so * omu * g1;                         // sin of its central angle
    const R cps = ce2 * co + q * u;
    const R hd = R(0.5) * dphi * dphi;
    const R sphi = sps * (R(1) - hd) + cps * dphi;
    const R cphi = cps * (R(1) - hd) - sps * dphi;
    const R omc = sphi * sphi / (R(1) + cphi);
    // the horizontal direction of travel at the emission point
    const R rse = rsqrt(se2 > R(1e-30) ? se2 : R(1e-30));
    const R tx = (px - ce * rx) * rse, ty = (py - ce * ry) * rse, tz = (pz - ce * rz) * rse;
    const R dr = -dH - r_o * omc;                        // r_o cos(phi) - r_e
    const R dtn = r_o * sphi;
    o.X = xe + (dr * rx + dtn * tx);
    o.Y = ye + (dr * ry + dtn * ty);
    o.zg = dze + (dr * rz + dtn * tz);
    o.t = S.tseg + fl * S.inv_bc + L * R(1.0 / kC);
    const R rox = cphi * rx + sphi * tx, roy = cphi * ry + sphi * ty, roz = cphi * rz + sphi * tz;
    const R tox = cphi * tx - sphi * rx, toy = cphi * ty - sphi * ry, toz = cphi * tz - sphi * rz;
    o.cx = so * tox - co * rox;
    o.cy = so * toy - co * roy;
    o.cz = so * toz - co * roz;
    if constexpr (TR) {
        const R tau = trans_tau<R>(p, o.lam, o.he);
        R P, u3;
        if constexpr (std::is_same<R, float>::value) {
            P = __expf(-(tau * sec));
            u3 = u01f(w3);
        } else {
            P = exp(-(tau / co));
            u3 = u01d(w3);
        }
        if (!(u3 < P)) {
            o.status = ST_ABSORBED;
            return;
        }
    }
    o.status = ST_GROUND;
}

// Philox4x32-10 of the bunch's counter (lo(g), hi(g), j, 0), g the global
// step index, with the step's share of the first two rounds taken from the
// step constants (prep_step): round 1 multiplies counter word 0 (the
// step's) and word 2 (j); round 2 multiplies round 1's word 2, which is the
// step's again.  Same words as philox4x32_10; each product is taken whole
// (64 bits) so that its two halves come from one multiply.
template <class R>
__device__ __forceinline__ uint4 philox_bunch(const KParams &p, const Seg<R> &S, uint32_t j) {
    const uint64_t w1 = static_cast<uint64_t>(0xCD9E8D57u) * j;
    const uint32_t c1x = static_cast<uint32_t>(w1 >> 32) ^ S.ph_a, c1y = static_cast<uint32_t>(w1);
    const uint64_t w0 = static_cast<uint64_t>(0xD2511F53u) * c1x;
    uint4 c = make_uint4(S.ph_b ^ c1y, S.ph_c, static_cast<uint32_t>(w0 >> 32) ^ S.ph_d,
                         static_cast<uint32_t>(w0));
#pragma unroll
    for (int r = 2; r < 10; ++r) {
        const uint64_t m0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t m1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        c = make_uint4(static_cast<uint32_t>(m1 >> 32) ^ c.y ^ p.rk0[r], static_cast<uint32_t>(m1),
                       static_cast<uint32_t>(m0 >> 32) ^ c.w ^ p.rk1[r], static_cast<uint32_t>(m0));
    }
    return c;
}

template <class R, bool TR, int FB, bool DS, bool CV = false, bool LAZY = false>
__device__ __forceinline__ void bunch(const KParams &p, const Consts<R> &c, const Seg<R> &S,
                                      const SegD<R> *SD, int j, BunchOut<R> &o) {
    const uint4 x = philox_bunch<R>(p, S, static_cast<uint32_t>(j));
    R u0, u1, u2;
    if constexpr (std::is_same<R, float>::value) {
        u0 = u01f(x.x);
        u1 = u01f(x.y);
        u2 = u01f(x.z);
    } else {
        u0 = u01d(x.x);
        u1 = u01d(x.y);
        u2 = u01d(x.z);
    }
    // sub-step j, emission point uniform inside it
    const R f = (static_cast<R>(j) + u0) * S.inv_nb;
    const R fl = f * S.L;
    R sp, cp;
    if constexpr (std::is_same<R, float>::value) {
        // phi = 2 pi u1 = a + pi with a in (-pi, pi), where the hardware
        // sine and cosine are accurate to 2^-21 (direction error < 1e-8)
        float sa, ca;
        __sincosf((u1 - 0.5f) * 6.28318530717958647692f, &sa, &ca);
        sp = -sa;
        cp = -ca;
    } else {
        sincospi(2.0 * u1, &sp, &cp);
    }
    R cosc = S.cosc, sinc = S.sinc;
    o.kap = R(1);
    if constexpr (DS) {
        disp_sample<R>(p, *SD, u2, o.lam, o.kap, cosc, sinc);
    } else if constexpr (LAZY) {
        // the deviate; the record forms lambda (the hit path only)
        o.lam = u2;
    } else {
        // 1/lambda^2 spectrum by inversion
        o.lam = R(1) / (c.lam_inv1 - u2 * c.lam_dinv);
    }
    const R px = cosc * S.ux + sinc * (cp * S.e1x + sp * S.e2x);
    const R py = cosc * S.uy + sinc * (cp * S.e1y + sp * S.e2y);
    const R pz = cosc * S.uz + sinc * (sp * S.e2z);
    o.zg = R(0);
    if constexpr (CV) {
        propagate_curved<R, TR, DS>(p, c, S, fl, px, py, pz, x.w, o);
        return;
    }
    const R dH = S.dz0 + fl * S.uz;                 // h_e - h_obs
    o.he = c.h_obs + dH;
    // rare conditions first (paper Alg. 2)
    if (!(pz < R(0))) { o.status = ST_UPWARD; return; }
    if (!(dH >= R(0))) { o.status = ST_BELOW; return; }
    if (!(dH <= c.dH_max)) { o.status = ST_ABOVE; return; }
    // Snell: sin_obs = sin_em (1 + kappa eta_e) / (1 + kappa eta_o)
    const R eta_e = eta_at<R>(p, c, o.he);
    R rm1;                                          // rat - 1
    if constexpr (DS)
        rm1 = o.kap * (eta_e - c.eta_o) / (R(1) + o.kap * c.eta_o);
    else
        rm1 = (eta_e - c.eta_o) * c.inv_np1o;
    const R rat = R(1) + rm1;
    const R se2 = px * px + py * py;
    const R q = se2 * rat * rat;                    // sin^2(theta_obs)
    if (!(q <= c.q_max)) {
        if constexpr (FB != 0) {
            if (q <= c.fb_q) {
                // past the tables' range: the ray integrals, queued (FB 1,
                // the hits kernel) or in place (FB 2, the trace kernel);
                // a queued bunch carries emission point, time, horizontal
                // direction and sin(theta_obs) in X, Y, t, cx, cy, cz, and
                // h_e - h_obs in he
                const R rse = rsqrt(se2 > R(1e-30) ? se2 : R(1e-30));
                const R hx = px * rse, hy = py * rse, s_obs = sqrt(q);
                const R c2 = R(1) - q;                                     // cos^2
                const R xe = S.x0 + fl * S.ux, ye = S.y0 + fl * S.uy;
                const R te = S.tseg + fl * S.inv_bc;
                if constexpr (FB == 1) {
                    o.X = xe; o.Y = ye; o.t = te; o.cx = hx; o.cy = hy; o.cz = s_obs;
                    o.he = dH;
                    o.c2 = c2;
                    o.status = ST_DEFER;
                } else {
                    R Df, Lf;
                    if constexpr (std::is_same<R, float>::value) {
                        ray_integrals_f(p, dH, s_obs, c2, o.kap, Df, Lf);
                    } else {
                        ray_integrals(p, p.h_obs + dH, s_obs, o.kap, Df, Lf);
                    }
                    const R co_fb = sqrt(c2);
                    o.X = xe + Df * hx;
                    o.Y = ye + Df * hy;
                    o.t = te + Lf * R(1.0 / kC);
                    o.cx = s_obs * hx;
                    o.cy = s_obs * hy;
                    o.cz = -co_fb;
                    o.status = ST_GROUND;
                    if constexpr (TR) {
                        const R tau = trans_tau<R>(p, o.lam, o.he);
                        R P, u3;
                        if constexpr (std::is_same<R, float>::value) {
                            P = __expf(-(tau / co_fb));
                            u3 = u01f(x.w);
                        } else {
                            P = exp(-(tau / co_fb));
                            u3 = u01d(x.w);
                        }
                        if (!(u3 < P)) o.status = ST_ABSORBED;
                    }
                }
                return;
            }
        }
        o.status = ST_ANGLE;
        return;
    }
    const R omq = R(1) - q;
    const R sec = rsqrt(omq);              // 1 / cos(theta_obs)
    const R co = omq * sec;
    // one cell of the (height, sin^2) tables serves both corrections
    const R fj = dH * c.inv_dht;
    int jj = static_cast<int>(fj);
    jj = jj > c.H - 2 ? c.H - 2 : jj;
    const R a = fj - static_cast<R>(jj);
    const R fk = q * c.inv_dq;
    int kk = static_cast<int>(fk);
    kk = kk > c.Z - 2 ? c.Z - 2 : kk;
    const R b = fk - static_cast<R>(kk);
    R Ax, Al;
    if constexpr (DS) {
        // the tables of the band's two ends, linear in kappa
        const size_t e0 = dbg_index(p, static_cast<size_t>(jj) * (c.Z - 1) + kk,
                                    int64_t(c.H - 1) * (c.Z - 1), DBG_TAB);
        const size_t e1 = dbg_index(p, e0 + (c.Z - 1), int64_t(c.H) * (c.Z - 1), DBG_TAB);
        if constexpr (std::is_same<R, float>::value) {
            const float wk = (o.kap - p.f.kap_lo) * p.f.kap_winv;
            const float4 *T = static_cast<const float4 *>(p.tabd);
            const float4 a0 = __ldg(T + 2 * e0), b0 = __ldg(T + 2 * e0 + 1);
            const float4 a1 = __ldg(T + 2 * e1), b1 = __ldg(T + 2 * e1 + 1);
            const float4 t0 = make_float4(a0.x + wk * (b0.x - a0.x), a0.y + wk * (b0.y - a0.y),
                                          a0.z + wk * (b0.z - a0.z), a0.w + wk * (b0.w - a0.w));
            const float4 t1 = make_float4(a1.x + wk * (b1.x - a1.x), a1.y + wk * (b1.y - a1.y),
                                          a1.z + wk * (b1.z - a1.z), a1.w + wk * (b1.w - a1.w));
            const float x0 = t0.x + a * (t1.x - t0.x), x1 = t0.z + a * (t1.z - t0.z);
            const float l0 = t0.y + a * (t1.y - t0.y), l1 = t0.w + a * (t1.w - t0.w);
            Ax = x0 + b * (x1 - x0);
            Al = l0 + b * (l1 - l0);
        } else {
            const double wk = (o.kap - p.kap_lo) * p.kap_winv;
            const double2 *T = static_cast<const double2 *>(p.tabd);
            double v[2][4];
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const size_t e = r ? e1 : e0;
                const double2 la = __ldg(T + 4 * e), lb = __ldg(T + 4 * e + 1);
                const double2 ha = __ldg(T + 4 * e + 2), hb = __ldg(T + 4 * e + 3);
                v[r][0] = la.x + wk * (ha.x - la.x);
                v[r][1] = la.y + wk * (ha.y - la.y);
                v[r][2] = lb.x + wk * (hb.x - lb.x);
                v[r][3] = lb.y + wk * (hb.y - lb.y);
            }
            const double x0 = v[0][0] + a * (v[1][0] - v[0][0]), x1 = v[0][2] + a * (v[1][2] - v[0][2]);
            const double l0 = v[0][1] + a * (v[1][1] - v[0][1]), l1 = v[0][3] + a * (v[1][3] - v[0][3]);
            Ax = x0 + b * (x1 - x0);
            Al = l0 + b * (l1 - l0);
        }
    } else if constexpr (std::is_same<R, float>::value) {
        // the cell's four nodes of the per-node table (H <= 65536, Z <= 4096:
        // the node index fits 32 bits; measured on GB300 0.4-1 % faster than
        // two 16-byte loads of the pair-interleaved entries, twice the bytes)
        const int n0 = dbg_index(p, jj * c.Z + kk, int64_t(c.H - 1) * c.Z - 1, DBG_TAB);
        const float2 *T = static_cast<const float2 *>(p.tab);
        const float2 a0 = __ldg(T + n0), a1 = __ldg(T + n0 + 1);
        const float2 b0 = __ldg(T + n0 + c.Z), b1 = __ldg(T + n0 + c.Z + 1);
        const float x0 = a0.x + a * (b0.x - a0.x), x1 = a1.x + a * (b1.x - a1.x);
        const float l0 = a0.y + a * (b0.y - a0.y), l1 = a1.y + a * (b1.y - a1.y);
        Ax = x0 + b * (x1 - x0);
        Al = l0 + b * (l1 - l0);
    } else {
        const int n0 = dbg_index(p, jj * c.Z + kk, int64_t(c.H - 1) * c.Z - 1, DBG_TAB);
        const double2 *T = static_cast<const double2 *>(p.tab);
        const double2 a0 = __ldg(T + n0), a1 = __ldg(T + n0 + 1);
        const double2 b0 = __ldg(T + n0 + c.Z), b1 = __ldg(T + n0 + c.Z + 1);
        const double x0 = a0.x + a * (b0.x - a0.x), x1 = a1.x + a * (b1.x - a1.x);
        const double l0 = a0.y + a * (b0.y - a0.y), l1 = a1.y + a * (b1.y - a1.y);
        Ax = x0 + b * (x1 - x0);
        Al = l0 + b * (l1 - l0);
    }
    const R sec2 = sec * sec;
    // horizontal unit vector and sin(theta_obs); a vertical photon (se2 = 0)
    // gets hx = hy = so = 0 through the clamp
    const R rse = rsqrt(se2 > R(1e-30) ? se2 : R(1e-30));
    const R hx = px * rse, hy = py * rse, so = se2 * rse * rat;
    const R tn = so * sec;
    const R D = tn * (dH + Ax * sec2);              // horizontal offset
    o.X = S.x0 + fl * S.ux + D * hx;
    o.Y = S.y0 + fl * S.uy + D * hy;
    if constexpr (std::is_same<R, float>::value) {
        // the time's small part here, its float-float sum on the hit path
        // (LAZY) or now
        const float r = fl * S.inv_bc + (sec * (fl * S.uz + Al * sec2)) * static_cast<float>(1.0 / kC);
        if constexpr (LAZY) {
            o.t = r;
            o.tsec = sec;
        } else {
            o.t = arrival_time_ff(S, sec, r);
        }
    } else {
        const R Lp = sec * (dH + Al * sec2);        // optical path
        o.t = S.tseg + fl * S.inv_bc + Lp * R(1.0 / kC);
    }
    o.cx = so * hx;
    o.cy = so * hy;
    o.cz = -co;
    if constexpr (TR) {
        // survive the atmosphere when u3 < exp(-tau / cos(theta_obs))
        const R tau = trans_tau<R>(p, o.lam, o.he);
        R P, u3;
        if constexpr (std::is_same<R, float>::value) {
            P = __expf(-(tau * sec));
            u3 = u01f(x.w);
        } else {
            P = exp(-(tau / co));
            u3 = u01d(x.w);
        }
        if (!(u3 < P)) {
            o.status = ST_ABSORBED;
            return;
        }
    }
    o.status = ST_GROUND;
}

// Candidate spheres of the bunch's grid cell: bit m of the mask is cell
// entry s0 + m of grid g (chosen by the arrival zenith).
template <class R, bool CV = false>
__device__ __forceinline__ unsigned sphere_hits(const KParams &p, const Consts<R> &c,
                                                const BunchOut<R> &o, int &s0,
                                                int &g) {
    s0 = 0;
    g = 0;
    if (o.status != ST_GROUND) return 0u;
    g = (o.cx * o.cx + o.cy * o.cy <= c.q_band) ? 0 : 1;
    // (selects, not indexing: the small arrays stay in registers)
    const R gx = (o.X - (g ? c.gx0[1] : c.gx0[0])) * (g ? c.inv_gcs[1] : c.inv_gcs[0]);
    const R gy = (o.Y - (g ? c.gy0[1] : c.gy0[0])) * (g ? c.inv_gcs[1] : c.inv_gcs[0]);
    const int nx = g ? p.grid[1].nx : p.grid[0].nx;
    const int ny = g ? p.grid[1].ny : p.grid[0].ny;
    // range check on the truncated indices (unsigned: negatives fail); a
    // point just below a grid edge truncates into the first row or column,
    // whose candidates it cannot hit: the grid covers every telescope's reach
    const int ix = static_cast<int>(gx), iy = static_cast<int>(gy);
    if (static_cast<unsigned>(ix) >= static_cast<unsigned>(nx) ||
        static_cast<unsigned>(iy) >= static_cast<unsigned>(ny))
        return 0u;
    const int cell = dbg_index(p, iy * nx + ix, int64_t(nx) * ny, DBG_GRID);
    unsigned mask = 0u;
    if constexpr (std::is_same<R, float>::value) {
        // (the first entry and the count packed in one word measured slower
        // than the two neighbouring starts)
        const int32_t *cs = g ? p.grid[1].cell_start : p.grid[0].cell_start;
        const float4 *cd = static_cast<const float4 *>(g ? p.grid[1].cand32 : p.grid[0].cand32);
        s0 = __ldg(cs + cell);
        const int s1 = __ldg(cs + cell + 1);
        const int nc = g ? p.grid[1].n_cand : p.grid[0].n_cand;
        auto crosses = [&](int m) {
            const float4 T = __ldg(cd + dbg_index(p, m, nc, DBG_GRID));
            const float dx = T.x - o.X, dy = T.y - o.Y, dz = CV ? T.z - o.zg : T.z;
            const float q0 = dy * o.cz - dz * o.cy;
            const float q1 = dz * o.cx - dx * o.cz;
            const float q2 = dx * o.cy - dy * o.cx;
            return q0 * q0 + q1 * q1 + q2 * q2 <= T.w;
        };
        // most cells hold none or one candidate: the first one is tested
        // straight-line, the loop only takes the rest (measured on GB300:
        // 2-3 % less time per launch than one loop over all of them)
        if (s1 > s0) {
            mask = crosses(s0) ? 1u : 0u;
            for (int m = s0 + 1; m < s1; ++m)
                if (crosses(m)) mask |= 1u << (m - s0);
        }
    } else {
        const int32_t *cs = g ? p.grid[1].cell_start : p.grid[0].cell_start;
        s0 = __ldg(cs + cell);
        const int s1 = __ldg(cs + cell + 1);
        const double2 *T = static_cast<const double2 *>(g ? p.grid[1].cand64 : p.grid[0].cand64);
        for (int m = s0; m < s1; ++m) {
            const int mc = dbg_index(p, m, g ? p.grid[1].n_cand : p.grid[0].n_cand, DBG_GRID);
            const double2 A = __ldg(T + 2 * mc), B = __ldg(T + 2 * mc + 1);
            const double dx = A.x - o.X, dy = A.y - o.Y, dz = CV ? B.x - o.zg : B.x;
            const double q0 = dy * o.cz - dz * o.cy;
            const double q1 = dz * o.cx - dx * o.cz;
            const double q2 = dx * o.cy - dy * o.cx;
            if (q0 * q0 + q1 * q1 + q2 * q2 <= B.y) mask |= 1u << (m - s0);
        }
    }
    return mask;
}

// telescope index and centre of entry m of grid g
template <class R>
__device__ __forceinline__ int cand_info(const KParams &p, int g, int m, R &tx, R &ty, R &tz) {
    if constexpr (std::is_same<R, float>::value) {
        const float4 T = __ldg(static_cast<const float4 *>(g ? p.grid[1].cand32 : p.grid[0].cand32) + m);
        tx = T.x; ty = T.y; tz = T.z;
        return __ldg((g ? p.grid[1].cand_tel : p.grid[0].cand_tel) + m);
    } else {
        const double2 *T = static_cast<const double2 *>(g ? p.grid[1].cand64 : p.grid[0].cand64);
        const double2 A = __ldg(T + 2 * m), B = __ldg(T + 2 * m + 1);
        tx = A.x; ty = A.y; tz = B.x;
        return __ldg((g ? p.grid[1].cand_tel : p.grid[0].cand_tel) + m);
    }
}

template <class R>
__device__ __forceinline__ void tel_xyz(const KParams &p, int k, R &tx, R &ty, R &tz) {
    if constexpr (std::is_same<R, float>::value) {
        const float4 T = __ldg(static_cast<const float4 *>(p.tel) + k);
        tx = T.x; ty = T.y; tz = T.z;
    } else {
        const double2 *T = static_cast<const double2 *>(p.tel);
        const double2 A = __ldg(T + 2 * k), B = __ldg(T + 2 * k + 1);
        tx = A.x; ty = A.y; tz = B.x;
    }
}

template <class R>
__device__ __forceinline__ void store4(void *base, int64_t r, R a, R b, R c, R d) {
    if constexpr (std::is_same<R, float>::value) {
        static_cast<float4 *>(base)[r] = make_float4(a, b, c, d);
    } else {
        double2 *q = static_cast<double2 *>(base) + 2 * r;
        q[0] = make_double2(a, b);
        q[1] = make_double2(c, d);
    }
}

// ask L2 for a line this CTA reads soon (no result, nothing waits on it)
__device__ __forceinline__ void prefetch_l2(const void *ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// warp-wide sum of a counter, one atomic per warp
__device__ __forceinline__ void flush_stat(unsigned long long *stats, int idx, unsigned v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(stats + idx, static_cast<unsigned long long>(v));
}

// the same for a counter whose per-thread part may be negative
__device__ __forceinline__ void flush_stat_signed(unsigned long long *stats, int idx, int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v)
        atomicAdd(stats + idx, static_cast<unsigned long long>(static_cast<long long>(v)));
}

// Warp-aggregated compaction into the per-telescope buffers: per (warp,
// telescope) one atomicAdd reserves the slots; the record is the crossing
// of the arrival line with the horizontal plane through the sphere centre.
// All 32 lanes call it (hm = 0 on lanes without a crossing).  The photon
// weight, record key, wavelength and arrival time at h_obs come from
// weight_key(w, key, lambda, t), called on the hit path only.  The fallback
// pass records through it; the fused kernel queues its crossings and
// records them with flush_ring, the same steps one crossing per lane.
template <class R, class KW>
__device__ __forceinline__ void record_hits(const KParams &p, const BunchOut<R> &o, unsigned hm,
                                            int s0, int gsel, KW weight_key, R np1o, int lane,
                                            unsigned &st_hits, unsigned &st_over) {
    for (;;) {
        if (!__any_sync(kFull, hm != 0u)) break;
        int tel = -1;
        R tx = R(0), ty = R(0), tz = R(0);
        if (hm) {
            const int bit = __ffs(hm) - 1;
            hm &= hm - 1u;
            tel = cand_info<R>(p, gsel,
                               dbg_index(p, s0 + bit, gsel ? p.grid[1].n_cand : p.grid[0].n_cand,
                                         DBG_GRID),
                               tx, ty, tz);
            ++st_hits;
        }
        const unsigned grp = __match_any_sync(kFull, tel);
        if (tel >= 0) {
            const int leader = __ffs(grp) - 1;
            const unsigned rank = __popc(grp & ((1u << lane) - 1u));
            unsigned long long slot0 = 0;
            if (lane == leader)
                slot0 = atomicAdd(p.count + tel, static_cast<unsigned long long>(__popc(grp)));
            slot0 = __shfl_sync(grp, slot0, leader);
            const unsigned long long slot = slot0 + rank;
            if (slot < static_cast<unsigned long long>(p.cap)) {
                R w, lam, tg;
                uint64_t key;
                weight_key(w, key, lam, tg);   // only on the (rare) hit path
                const R sl = (tz - o.zg) / o.cz;   // to the plane through the centre
                const int64_t r = dbg_index(p, static_cast<int64_t>(tel) * p.cap +
                                                   static_cast<int64_t>(slot),
                                            int64_t(p.n_tel) * p.cap, DBG_OUT);
                store4<R>(p.pos, r, o.X + sl * o.cx - tx, o.Y + sl * o.cy - ty, o.cx, o.cy);
                store4<R>(p.tim, r, tg + sl * np1o * R(1.0 / kC), o.he, w, lam);
                p.key[r] = key;
            } else {
                ++st_over;
            }
        }
    }
}

// The hits kernels record their crossings from a per-warp queue instead of
// in the window where they are found.  About 1-2 % of bunches cross a
// sphere, so a window usually holds none or one, and recording it there
// keeps 31 of 32 lanes idle through the record's ~70 instructions.  The
// window queues each (bunch, candidate) pair as 8 bytes (step in tile and
// bunch index; grid and candidate entry) in a ring of 64 in shared memory;
// once 32 are queued, and at the end of the tile while its step constants
// are still in shared memory, each lane takes one pair, computes its bunch
// again (the same function on the same inputs, so the same values) and
// writes the record with the per-(warp, telescope) atomics of record_hits.
// Measured on GB300: 4-8 % less time per launch of the plain FP32 path,
// 5-7 % with the transmission draw, 1-2 % with spectra, 12-14 % in FP64
// (where the record's division and products run on the FP64 pipe).
constexpr int kRing = 64;

template <class R, int BLOCK, bool TR, int FB, bool DS, bool CV>
__device__ __forceinline__ void flush_ring(const KParams &p, const Consts<R> &c, R np1o,
                                           const Seg<R> *seg, const SegD<R> *segd,
                                           const uint2 *ring, int head, int n, int64_t base,
                                           int lane, unsigned &st_over) {
    // the plain instantiation leaves wavelength and time's large part to here
    constexpr bool kLazy = !TR && FB == 0 && !DS && !CV;
    int tel = -1;
    R tx = R(0), ty = R(0), tz = R(0);
    BunchOut<R> o;
    o.status = -1;
    o.zg = R(0);
    int s = 0, j = 0;
    if (lane < n) {
        const uint2 e = ring[(head + lane) & (kRing - 1)];
        s = dbg_index(p, static_cast<int>(e.x >> 22), BLOCK, DBG_SMEM);
        j = static_cast<int>(e.x & 0x3fffffu);
        bunch<R, TR, FB, DS, CV, kLazy>(p, c, seg[s], DS ? segd + s : nullptr, j, o);
        const int g = static_cast<int>(e.y >> 31);
        const int m = static_cast<int>(e.y & 0x7fffffffu);
        tel = cand_info<R>(p, g, dbg_index(p, m, g ? p.grid[1].n_cand : p.grid[0].n_cand,
                                           DBG_GRID), tx, ty, tz);
    }
    // from here on as record_hits, one crossing per lane
    const unsigned grp = __match_any_sync(kFull, tel);
    if (tel >= 0) {
        const int leader = __ffs(grp) - 1;
        const unsigned rank = __popc(grp & ((1u << lane) - 1u));
        unsigned long long slot0 = 0;
        if (lane == leader)
            slot0 = atomicAdd(p.count + tel, static_cast<unsigned long long>(__popc(grp)));
        slot0 = __shfl_sync(grp, slot0, leader);
        const unsigned long long slot = slot0 + rank;
        if (slot < static_cast<unsigned long long>(p.cap)) {
            const Seg<R> &S = seg[s];
            const int64_t gstep = p.track_base + base + s;
            const uint64_t key = (static_cast<uint64_t>(gstep) << 32) | static_cast<uint32_t>(j);
            R lam, tg;
            if constexpr (kLazy) {
                lam = R(1) / (c.lam_inv1 - o.lam * c.lam_dinv);
                if constexpr (std::is_same<R, float>::value)
                    tg = arrival_time_ff(S, o.tsec, o.t);
                else
                    tg = o.t;
            } else {
                lam = o.lam;
                tg = o.t;
            }
            const R np1 = DS ? R(1) + o.kap * c.eta_o : np1o;
            const R sl = (tz - o.zg) / o.cz;   // to the plane through the centre
            const int64_t r = dbg_index(p, static_cast<int64_t>(tel) * p.cap +
                                               static_cast<int64_t>(slot),
                                        int64_t(p.n_tel) * p.cap, DBG_OUT);
            store4<R>(p.pos, r, o.X + sl * o.cx - tx, o.Y + sl * o.cy - ty, o.cx, o.cy);
            store4<R>(p.tim, r, tg + sl * np1 * R(1.0 / kC), o.he, S.w, lam);
            p.key[r] = key;
        } else {
            ++st_over;
        }
    }
}

// ------------------------------------------------------------------------
// The fused kernel.
// ------------------------------------------------------------------------
// TR: the atmospheric transmission draw is compiled in (a separate
// instantiation: present but switched off it cost 2 % of the launch).
// FB: bunches past the tables' zenith range are queued for the fallback
// pass (1, hits) or integrated in place (2, trace).
// DS: the index depends on the wavelength (per-step spectra in shared memory).
template <class R, int BLOCK>
__host__ __device__ constexpr size_t segd_offset() {
    return (sizeof(Seg<R>) * BLOCK + sizeof(int) * (BLOCK + 1 + 32) + 15) & ~size_t(15);
}

// the crossing queue of the hits kernels, after the spectra (DS)
template <class R, int BLOCK, bool DS>
__host__ __device__ constexpr size_t ring_offset() {
    return segd_offset<R, BLOCK>() + (DS ? sizeof(SegD<R>) * BLOCK : 0);
}

// CV: a curved atmosphere (radial heights, spherical shells).
template <class R, int BLOCK, int MODE, bool TR, int FB, bool DS, bool CV>
__device__ __forceinline__ void gen_prop(const KParams &p) {
    extern __shared__ __align__(16) unsigned char smem[];
    Seg<R> *seg = reinterpret_cast<Seg<R> *>(smem);
    int *off = reinterpret_cast<int *>(seg + BLOCK);          // BLOCK + 1
    int *wsum = off + BLOCK + 1;                                // BLOCK / 32
    SegD<R> *segd = reinterpret_cast<SegD<R> *>(smem + segd_offset<R, BLOCK>());   // DS only
    // the hits kernels queue their crossings (flush_ring) in a ring after
    // the spectra (the entry packs the step in the tile in 10 bits above the
    // bunch index in 22: a step has at most 2^22 bunches)
    constexpr bool kQueue = MODE == MODE_HITS;
    static_assert(BLOCK <= 1024, "the queue entry holds the step in the tile in 10 bits");
    __shared__ unsigned long long s_tile;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint2 *ring = reinterpret_cast<uint2 *>(smem + ring_offset<R, BLOCK, DS>()) + warp * kRing;
    int q_tail = 0, q_cnt = 0;       // (warp-uniform)
    // the candidate grids (a few KB) are read through L1; their sizes and
    // pointers come straight from the kernel parameters (selects, nothing
    // held in registers across the bunch loop)

    Consts<R> c;
    R np1o;
    make_consts<R>(p, c, np1o);

    unsigned st_steps = 0, st_emit = 0, st_inval = 0, st_bunch = 0, st_up = 0, st_below = 0,
             st_above = 0, st_angle = 0, st_absorb = 0, st_hits = 0, st_over = 0;

    // Persistent CTAs claim their next tile one tile ahead, during the scan
    // (its barriers publish the claim), and prefetch that tile's step
    // arrays into L2 while they work through the current tile's bunches; one
    // barrier per tile separates its bunch loop from the next phase A.
    int64_t tile = blockIdx.x;
    if (p.tile_counter) {
        __syncthreads();
        if (tid == 0) s_tile = atomicAdd(p.tile_counter, 1ull);
        __syncthreads();
        tile = static_cast<int64_t>(s_tile);
    }
    for (;;) {
        if (tile >= p.n_tiles) break;
        const int64_t base = tile * BLOCK;

        // ---- phase A: one step per thread ----------------------------------
        const int64_t i = base + tid;
        int nb = 0;
        if (i < p.n) {
            // the FP32 path screens the yield in FP32 (same bunch counts as FP64)
            using YT = typename std::conditional<std::is_same<R, float>::value, YieldF,
                                                 Yield>::type;
            YT y;
            // in a curved atmosphere the yield needs the midpoint's horizontal place
            double xyd[4];
            float xyf[4];
            if constexpr (CV) {
                xyd[0] = __ldg(p.x0 + i);
                xyd[1] = __ldg(p.y0 + i);
                xyd[2] = static_cast<double>(load_dir<R>(p.ux, i));
                xyd[3] = static_cast<double>(load_dir<R>(p.uy, i));
                xyf[0] = d2f_rn(xyd[0]);
                xyf[1] = d2f_rn(xyd[1]);
                xyf[2] = static_cast<float>(load_dir<R>(p.ux, i));
                xyf[3] = static_cast<float>(load_dir<R>(p.uy, i));
            }
            const double *pxyd = CV ? xyd : nullptr;
            const float *pxyf = CV ? xyf : nullptr;
            if constexpr (DS) {
                if constexpr (std::is_same<YT, YieldF>::value)
                    step_yield_screened_disp(p, step_valid<R>(p, i), __ldg(p.z0 + i),
                                             __ldg(p.len + i), __ldg(p.ekin + i),
                                             load_dir<float>(p.uz, i), y, segd[tid], pxyf, pxyd);
                else
                    step_yield_disp<R>(p, step_valid<R>(p, i), __ldg(p.z0 + i), __ldg(p.len + i),
                                       __ldg(p.ekin + i), static_cast<double>(load_dir<R>(p.uz, i)),
                                       y, segd[tid], pxyd);
            } else if constexpr (std::is_same<YT, YieldF>::value) {
                step_yield_screened(p, step_valid<R>(p, i), __ldg(p.z0 + i), __ldg(p.len + i),
                                    __ldg(p.ekin + i), load_dir<float>(p.uz, i), y, pxyf, pxyd);
            } else {
                step_yield(p, step_valid<R>(p, i), __ldg(p.z0 + i), __ldg(p.len + i),
                           __ldg(p.ekin + i), static_cast<double>(load_dir<R>(p.uz, i)), y, pxyd);
            }
            if constexpr (MODE == MODE_SCREEN) {
                // the adjoint freezes the sub-step structure
                const int nf = __ldg(p.nb_frozen + i);
                y.nb = (y.s2 > 0.0 && nf > 0) ? nf : 0;
            }
            nb = y.nb;
            if constexpr (MODE == MODE_HITS) {
                if (p.prof && nb > 0) profile_step<R>(p, i, static_cast<R>(y.N));
            }
            ++st_steps;
            st_emit += (nb > 0);
            st_inval += !y.valid;
            if constexpr (MODE == MODE_YIELD) {
                p.y_nb[i] = nb;
                p.y_w[i] = nb > 0 ? static_cast<double>(y.N) / static_cast<double>(nb) : 0.0;
            } else {
                prep_step<R>(p, i, y, seg[tid]);
            }
        }
        if constexpr (MODE == MODE_YIELD) {
            if (!p.tile_counter) break;
            __syncthreads();
            if (tid == 0) s_tile = atomicAdd(p.tile_counter, 1ull);
            __syncthreads();
            tile = static_cast<int64_t>(s_tile);
            continue;
        }
        st_bunch += nb;

        // ---- CTA exclusive scan of nb ---------------------------------------
        int v = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) wsum[warp] = v;
        if (tid == 0 && p.tile_counter) s_tile = atomicAdd(p.tile_counter, 1ull);
        __syncthreads();
        const int64_t next = p.tile_counter ? static_cast<int64_t>(s_tile) : p.n_tiles;
        if (warp == 0) {
            int w = lane < BLOCK / 32 ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, w, o);
                if (lane >= o) w += t;
            }
            if (lane < BLOCK / 32) wsum[lane] = w;   // inclusive warp totals
        }
        __syncthreads();
        const int excl = v - nb + (warp > 0 ? wsum[warp - 1] : 0);
        off[tid] = excl;
        if (tid == BLOCK - 1) off[BLOCK] = excl + nb;
        __syncthreads();
        const int total = off[BLOCK];
        if (next < p.n_tiles) {
            const int64_t ni = next * BLOCK + tid;
            if (ni < p.n) {
                prefetch_l2(p.x0 + ni);
                prefetch_l2(p.y0 + ni);
                prefetch_l2(p.z0 + ni);
                prefetch_l2(p.t0 + ni);
                prefetch_l2(p.len + ni);
                prefetch_l2(p.ekin + ni);
                prefetch_l2(static_cast<const R *>(p.ux) + ni);
                prefetch_l2(static_cast<const R *>(p.uy) + ni);
                prefetch_l2(static_cast<const R *>(p.uz) + ni);
                if (p.shower) prefetch_l2(p.shower + ni);
            }
        }

        // ---- phase B: the tile's bunches -------------------------------------
        // Each warp takes an even share of contiguous 32-bunch windows (shares
        // differ by at most one window).  The step of a window's first bunch
        // comes from the previous window (one search per warp and tile);
        // inside a window a lane's step is the last step whose first bunch is
        // <= its own, counted from the at most 32 step starts that follow with
        // one ballot and a few shuffles.
        const int nwin = (total + 31) >> 5;
        const int w_lo = (warp * nwin) / (BLOCK / 32);
        const int w_hi = ((warp + 1) * nwin) / (BLOCK / 32);
        int s_cur = 0;
        if (w_lo < w_hi) {
            int lo = 0, hi = BLOCK;
            const int b_first = w_lo * 32;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (off[mid] <= b_first) lo = mid; else hi = mid;
            }
            s_cur = lo;
        }
        for (int win = w_lo; win < w_hi; ++win) {
            const int bidx = win * 32 + lane;
            const bool live = bidx < total;
            int s = s_cur;
            for (int batch = s_cur;; batch += 32) {
                const int idx = batch + 1 + lane;
                const int v = (idx <= BLOCK ? off[idx] : 0x7fffffff) - win * 32;
                const int k = __popc(__ballot_sync(kFull, v <= 31));
                for (int q = 0; q < k; ++q) s += (__shfl_sync(kFull, v, q) <= lane);
                if (k < 32) break;
            }
            s_cur = __shfl_sync(kFull, s, 31);
            BunchOut<R> o;
            o.status = -1;
            o.zg = R(0);
            int j = 0;
            if (live) {
                s = dbg_index(p, s, BLOCK, DBG_SMEM);
                j = bidx - off[s];
                constexpr bool kLazy = MODE == MODE_HITS && !TR && FB == 0 && !DS && !CV;
                bunch<R, TR, FB, DS, CV, kLazy>(p, c, seg[s], DS ? segd + s : nullptr, j, o);
                if (o.status != ST_GROUND) {       // rare: the drops
                    st_up += o.status == ST_UPWARD;
                    st_below += o.status == ST_BELOW;
                    st_above += o.status == ST_ABOVE;
                    st_angle += o.status == ST_ANGLE;
                    st_absorb += o.status == ST_ABSORBED;
                }
            }
            if constexpr (MODE == MODE_SCREEN) {
                // list the bunch if it lands near a telescope centre
                if (live && o.status == ST_GROUND) {
                    const R rc2 = std::is_same<R, float>::value ? static_cast<R>(p.f.rcut2)
                                                                : static_cast<R>(p.rcut2);
                    for (int k = 0; k < p.n_tel; ++k) {
                        R tx, ty, tz;
                        tel_xyz<R>(p, k, tx, ty, tz);
                        const R dx = o.X - tx, dy = o.Y - ty;
                        if (dx * dx + dy * dy < rc2) {
                            const unsigned long long at = atomicAdd(p.list_count, 1ull);
                            if (at < static_cast<unsigned long long>(p.list_cap))
                                p.list[at] = (static_cast<uint64_t>(base + s) << 32) |
                                             static_cast<uint32_t>(j);
                            break;
                        }
                    }
                }
                continue;
            }
            if constexpr (MODE == MODE_HITS && FB == 1) {
                // past the tables' range: queue for the fallback pass
                const bool dq = live && o.status == ST_DEFER;
                const unsigned qm = __ballot_sync(kFull, dq);
                if (qm) {
                    const int leader = __ffs(qm) - 1;
                    unsigned long long at0 = 0;
                    if (lane == leader) at0 = atomicAdd(p.fb_count, static_cast<unsigned long long>(__popc(qm)));
                    at0 = __shfl_sync(kFull, at0, leader);
                    const unsigned long long at = at0 + __popc(qm & ((1u << lane) - 1u));
                    if (dq && at < static_cast<unsigned long long>(p.fb_cap)) {
                        FbEntry<R> e;
                        e.xe = o.X; e.ye = o.Y; e.he = c.h_obs + o.he; e.dh = o.he; e.te = o.t;
                        e.hx = o.cx; e.hy = o.cy; e.s_obs = o.cz; e.c2 = o.c2; e.lam = o.lam;
                        e.w = seg[s].w;
                        e.kap = o.kap;
                        const int64_t gstep = p.track_base + base + s;
                        e.key = (static_cast<uint64_t>(gstep) << 32) | static_cast<uint32_t>(j);
                        e.step_hi = static_cast<uint32_t>(static_cast<uint64_t>(gstep) >> 32);
                        static_cast<FbEntry<R> *>(p.fb_list)[dbg_index(
                            p, static_cast<int64_t>(at), p.fb_cap, DBG_FB)] = e;
                    }
                }
            }
            int s0 = 0, gsel = 0;
            unsigned hm = live ? sphere_hits<R, CV>(p, c, o, s0, gsel) : 0u;
            if constexpr (MODE == MODE_TRACE) {
                st_hits += __popc(hm);
                if (live) {
                    const int64_t gb =
                        dbg_index(p, __ldg(p.bunch_off + base + s) + j, p.t_nbunch, DBG_TRACE);
                    const R w = seg[s].w;
                    if (o.status == ST_GROUND) {
                        store4<R>(p.pos, gb, o.X, o.Y, o.cx, o.cy);
                        store4<R>(p.tim, gb, o.t, o.he, w, o.lam);
                    } else {
                        store4<R>(p.pos, gb, R(0), R(0), R(0), R(0));
                        store4<R>(p.tim, gb, R(0), o.he, w, o.lam);
                    }
                    p.t_status[gb] = o.status;
                    p.t_nhit[gb] = __popc(hm);
                    int first = -1;
                    for (unsigned mm = hm; mm; mm &= mm - 1u) {      // lowest telescope index
                        R tx, ty, tz;
                        const int k = cand_info<R>(p, gsel, s0 + __ffs(mm) - 1, tx, ty, tz);
                        first = (first < 0 || k < first) ? k : first;
                    }
                    p.t_first[gb] = first;
                }
            } else if constexpr (kQueue) {
                // one pair per lane and round (a lane with several crossings
                // takes several rounds), so at most 32 join a ring of < 32
                for (;;) {
                    const unsigned has = __ballot_sync(kFull, hm != 0u);
                    if (!has) break;
                    if (hm) {
                        const int bit = __ffs(hm) - 1;
                        hm &= hm - 1u;
                        const int slot =
                            (q_tail + __popc(has & ((1u << lane) - 1u))) & (kRing - 1);
                        ring[slot] = make_uint2(
                            (static_cast<uint32_t>(s) << 22) | static_cast<uint32_t>(j),
                            (static_cast<uint32_t>(gsel) << 31) | static_cast<uint32_t>(s0 + bit));
                        ++st_hits;
                    }
                    q_tail = (q_tail + __popc(has)) & (kRing - 1);
                    q_cnt += __popc(has);
                    if (q_cnt >= 32) {
                        __syncwarp();
                        flush_ring<R, BLOCK, TR, FB, DS, CV>(p, c, np1o, seg, segd, ring,
                                                             (q_tail - q_cnt) & (kRing - 1), 32,
                                                             base, lane, st_over);
                        q_cnt -= 32;
                        __syncwarp();
                    }
                }
            }
        }
        if constexpr (kQueue) {
            // the rest of the queue, while the tile's step constants are there
            __syncwarp();
            if (q_cnt > 0) {
                flush_ring<R, BLOCK, TR, FB, DS, CV>(p, c, np1o, seg, segd, ring,
                                                     (q_tail - q_cnt) & (kRing - 1), q_cnt, base,
                                                     lane, st_over);
                q_cnt = 0;
            }
            __syncwarp();
        }
        if (!p.tile_counter) break;
        // every warp is done with this tile's step constants and offsets
        // before the next tile's phase A and scan overwrite them
        __syncthreads();
        tile = next;
    }

    unsigned long long *S = p.stats;
    if (S) {
        flush_stat(S, CHER_STAT_STEPS, st_steps);
        flush_stat(S, CHER_STAT_EMITTING, st_emit);
        flush_stat(S, CHER_STAT_INVALID, st_inval);
        if (MODE != MODE_YIELD) {
            flush_stat(S, CHER_STAT_BUNCHES, st_bunch);
            flush_stat(S, CHER_STAT_UPWARD, st_up);
            flush_stat(S, CHER_STAT_BELOW_OBS, st_below);
            flush_stat(S, CHER_STAT_ABOVE_MAX, st_above);
            flush_stat(S, CHER_STAT_ANGLE, st_angle);
            flush_stat(S, CHER_STAT_ABSORBED, st_absorb);
            // reached the ground = generated - dropped (a per-thread partial
            // may be negative; the sum modulo 2^64 is exact)
            flush_stat_signed(S, CHER_STAT_GROUND,
                              static_cast<int>(st_bunch) -
                                  static_cast<int>(st_up + st_below + st_above + st_angle + st_absorb));
            flush_stat(S, CHER_STAT_HITS, st_hits);
            flush_stat(S, CHER_STAT_OVERFLOW, st_over);
        }
    }
}

// The kernels: every instantiation at the register budget of 1024 / BLOCK
// threads per SM (FP32) or of one CTA (FP64), and the plain FP32 hits
// instantiation also at 9 and 10 CTAs of 128 threads per SM (56 and 48
// registers): more resident warps hide more of the table and grid load
// latency, at the cost of a few spilled values (measured on GB300: -0.5 to
// -3 % by workload; 12 CTAs at 40 registers spilled too much, +2 to +5 %).
template <class R, int BLOCK, int MODE, bool TR, int FB, bool DS, bool CV>
__global__ void __launch_bounds__(BLOCK, std::is_same<R, float>::value ? 1024 / BLOCK : 1)
    k_gen_prop(const KParams p) {
    gen_prop<R, BLOCK, MODE, TR, FB, DS, CV>(p);
}

template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_gen_prop_occ(const KParams p) {
    gen_prop<float, 128, MODE_HITS, false, 0, false, false>(p);
}

// ------------------------------------------------------------------------
// The fallback pass: one thread per queued bunch (warps walk the queue 32
// entries at a time so that the compaction stays warp-synchronous).
// ------------------------------------------------------------------------
template <class R, bool TR, bool DS>
__global__ void __launch_bounds__(128) k_fallback(const KParams p) {
    Consts<R> c;
    R np1o;
    make_consts<R>(p, c, np1o);
    const int lane = threadIdx.x & 31;
    const unsigned long long queued = *p.fb_count;
    const unsigned long long cap = static_cast<unsigned long long>(p.fb_cap);
    const int64_t n = static_cast<int64_t>(queued < cap ? queued : cap);
    unsigned st_fb = 0, st_absorb = 0, st_hits = 0, st_over = 0;
    const int64_t warps = static_cast<int64_t>(gridDim.x) * (blockDim.x >> 5);
    const int64_t wid = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int64_t first = wid * 32; first < n; first += warps * 32) {
        const int64_t e = first + lane;
        const bool live = e < n;
        BunchOut<R> o;
        o.status = -1;
        o.zg = R(0);
        R w = R(0);
        uint64_t key = 0;
        if (live) {
            const FbEntry<R> E =
                static_cast<const FbEntry<R> *>(p.fb_list)[dbg_index(p, e, p.fb_cap, DBG_FB)];
            R D, L;
            if constexpr (std::is_same<R, float>::value)
                ray_integrals_f(p, E.dh, E.s_obs, E.c2, DS ? E.kap : 1.0f, D, L);
            else
                ray_integrals(p, p.h_obs + E.dh, E.s_obs, DS ? E.kap : 1.0, D, L);
            const R co = sqrt(E.c2);
            o.X = E.xe + D * E.hx;
            o.Y = E.ye + D * E.hy;
            o.t = E.te + L * R(1.0 / kC);
            o.cx = E.s_obs * E.hx;
            o.cy = E.s_obs * E.hy;
            o.cz = -co;
            o.he = E.he;
            o.lam = E.lam;
            o.kap = DS ? E.kap : R(1);
            o.status = ST_GROUND;
            w = E.w;
            key = E.key;
            const uint32_t step_hi = E.step_hi;
            ++st_fb;
            if constexpr (TR) {
                // the bunch's fourth Philox word decides, as in the main pass
                const uint4 x = philox4x32_10(
                    make_uint4(static_cast<uint32_t>(key >> 32), step_hi, static_cast<uint32_t>(key),
                               0u),
                    p.key0, p.key1);
                const R tau = trans_tau<R>(p, o.lam, o.he);
                R P, u3;
                if constexpr (std::is_same<R, float>::value) {
                    P = __expf(-(tau / co));
                    u3 = u01f(x.w);
                } else {
                    P = exp(-(tau / co));
                    u3 = u01d(x.w);
                }
                if (!(u3 < P)) {
                    o.status = ST_ABSORBED;
                    ++st_absorb;
                }
            }
        }
        int s0 = 0, gsel = 0;
        unsigned hm = live ? sphere_hits<R>(p, c, o, s0, gsel) : 0u;
        const R np1 = DS ? R(1) + o.kap * c.eta_o : np1o;
        const R lam_o = o.lam, t_o = o.t;
        record_hits<R>(p, o, hm, s0, gsel,
                       [w, key, lam_o, t_o](R &w_, uint64_t &k_, R &l_, R &t_) {
                           w_ = w;
                           k_ = key;
                           l_ = lam_o;
                           t_ = t_o;
                       },
                       np1, lane, st_hits, st_over);
    }
    unsigned long long *S = p.stats;
    if (S) {
        // the main pass counted the queued bunches as reaching the ground
        flush_stat(S, CHER_STAT_FALLBACK, st_fb);
        flush_stat(S, CHER_STAT_ABSORBED, st_absorb);
        flush_stat_signed(S, CHER_STAT_GROUND, -static_cast<int>(st_absorb));
        flush_stat(S, CHER_STAT_HITS, st_hits);
        flush_stat(S, CHER_STAT_OVERFLOW, st_over);
        if (blockIdx.x == 0 && threadIdx.x == 0 && queued > cap) {
            atomicAdd(S + CHER_STAT_FB_LOST, queued - cap);
            atomicAdd(S + CHER_STAT_GROUND, ~(queued - cap) + 1ull);     // minus the lost
        }
    }
}

template <class R, int BLOCK>
size_t smem_bytes(const KParams &p) {
    size_t b = segd_offset<R, BLOCK>();
    if (p.disp_k > 0) b += sizeof(SegD<R>) * BLOCK;
    // every launch reserves the crossing queue (the hits kernels use it;
    // 2 KB per 128 threads)
    b += sizeof(uint2) * kRing * (BLOCK / 32);
    return b;
}

template <class R, int BLOCK, int MODE, bool DS, bool CV>
const void *kernel_ptr_ds(bool tr, bool fb) {
    if constexpr (MODE == MODE_YIELD || MODE == MODE_SCREEN) {
        if constexpr (MODE == MODE_YIELD)
            return reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, false, 0, DS, CV>);
        else
            return tr ? reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, true, 0, DS, CV>)
                      : reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, false, 0, DS, CV>);
    } else if constexpr (CV) {
        // the curved atmosphere has no beyond-table fallback
        if (fb) return nullptr;
        return tr ? reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, true, 0, DS, CV>)
                  : reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, false, 0, DS, CV>);
    } else {
        constexpr int F = MODE == MODE_HITS ? 1 : 2;
        if (fb)
            return tr ? reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, true, F, DS, CV>)
                      : reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, false, F, DS, CV>);
        return tr ? reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, true, 0, DS, CV>)
                  : reinterpret_cast<const void *>(&k_gen_prop<R, BLOCK, MODE, false, 0, DS, CV>);
    }
}

template <class R, int BLOCK, int MODE>
const void *kernel_ptr(bool tr, bool fb, bool ds, bool cv) {
    if (ds || cv) {
        // the wavelength-dependent index and the curved atmosphere: 128-step
        // tiles, no adjoint screening
        if constexpr (BLOCK == kDispBlock && MODE != MODE_SCREEN) {
            if (cv)
                return ds ? kernel_ptr_ds<R, BLOCK, MODE, true, true>(tr, fb)
                          : kernel_ptr_ds<R, BLOCK, MODE, false, true>(tr, fb);
            return kernel_ptr_ds<R, BLOCK, MODE, true, false>(tr, fb);
        } else {
            return nullptr;
        }
    }
    return kernel_ptr_ds<R, BLOCK, MODE, false, false>(tr, fb);
}

template <class R, int MODE>
const void *pick(int block, bool tr, bool fb, bool ds, bool cv) {
    switch (block) {
    case 128: return kernel_ptr<R, 128, MODE>(tr, fb, ds, cv);
    case 256: return kernel_ptr<R, 256, MODE>(tr, fb, ds, cv);
    case 512: return kernel_ptr<R, 512, MODE>(tr, fb, ds, cv);
    }
    return nullptr;
}

// mode: a Mode, plus kTransBit / kFbBit / kDispBit / kCurvBit for the
// instantiations with the transmission draw / the beyond-table fallback /
// the wavelength-dependent index / the curved atmosphere
const void *pick_kernel(bool fp32, int block, int mode) {
    const int occ = (mode & kOccMask) >> kOccShift;
    mode &= ~kOccMask;
    if (occ && fp32 && block == 128 && mode == MODE_HITS) {
        return occ == 1 ? reinterpret_cast<const void *>(&k_gen_prop_occ<9>)
                        : reinterpret_cast<const void *>(&k_gen_prop_occ<10>);
    }
    const bool tr = (mode & kTransBit) != 0;
    const bool fb = (mode & kFbBit) != 0;
    const bool ds = (mode & kDispBit) != 0;
    const bool cv = (mode & kCurvBit) != 0;
    mode &= ~(kTransBit | kFbBit | kDispBit | kCurvBit);
    if (fp32) {
        switch (mode) {
        case MODE_HITS: return pick<float, MODE_HITS>(block, tr, fb, ds, cv);
        case MODE_TRACE: return pick<float, MODE_TRACE>(block, tr, fb, ds, cv);
        case MODE_YIELD: return pick<float, MODE_YIELD>(block, tr, fb, ds, cv);
        case MODE_SCREEN: return pick<float, MODE_SCREEN>(block, tr, fb, ds, cv);
        }
    } else {
        switch (mode) {
        case MODE_HITS: return pick<double, MODE_HITS>(block, tr, fb, ds, cv);
        case MODE_TRACE: return pick<double, MODE_TRACE>(block, tr, fb, ds, cv);
        case MODE_YIELD: return pick<double, MODE_YIELD>(block, tr, fb, ds, cv);
        case MODE_SCREEN: return pick<double, MODE_SCREEN>(block, tr, fb, ds, cv);
        }
    }
    return nullptr;
}

}  // namespace

void fill_float_constants(KParams &p) {
    p.f.h_obs = static_cast<float>(p.h_obs);
    p.f.dH_max = static_cast<float>(p.h_max - p.h_obs);
    p.f.eta_o = static_cast<float>(p.eta_obs);
    p.f.inv_np1o = static_cast<float>(1.0 / (1.0 + p.eta_obs));
    p.f.np1o = static_cast<float>(1.0 + p.eta_obs);
    p.f.q_max = static_cast<float>(p.q_max);
    p.f.inv_dht = static_cast<float>(p.inv_dht);
    p.f.inv_dq = static_cast<float>(p.inv_dq);
    p.f.inv_dh = static_cast<float>(p.inv_dh);
    p.f.lam_inv1 = static_cast<float>(p.lam_inv1);
    p.f.lam_dinv = static_cast<float>(p.lam_dinv);
    for (int g = 0; g < 2; ++g) {
        p.f.gx0[g] = static_cast<float>(p.grid[g].x0);
        p.f.gy0[g] = static_cast<float>(p.grid[g].y0);
        p.f.inv_gcs[g] = static_cast<float>(p.grid[g].inv_cs);
    }
    p.f.q_band = static_cast<float>(p.q_band);
    p.f.inv_me = static_cast<float>(p.inv_me);
    p.f.K = static_cast<float>(p.K);
    p.f.inv_B = static_cast<float>(p.inv_B);
    p.f.h_max = static_cast<float>(p.h_max);
    p.f.dh = static_cast<float>(1.0 / p.inv_dh);
    p.f.eta_slope = static_cast<float>(p.eta_slope * 1.01);
    p.f.eta_jump = static_cast<float>(p.eta_jump);
    p.f.rcut2 = static_cast<float>(p.rcut2);
    p.f.fb_q = static_cast<float>(p.fb_q);
    p.f.trans_l0 = static_cast<float>(p.trans_l0);
    p.f.trans_lscale = static_cast<float>(p.trans_lscale);
    p.f.trans_h0 = static_cast<float>(p.trans_h0);
    p.f.trans_hscale = static_cast<float>(p.trans_hscale);
    p.f.prof_dx = static_cast<float>(p.prof_dx);
    p.f.prof_inv_dx = static_cast<float>(p.prof_inv_dx);
    for (int m = 0; m < kDispMax; ++m) p.f.kap[m] = static_cast<float>(p.kap[m]);
    p.f.disp_Kd = static_cast<float>(p.disp_Kd);
    p.f.disp_u1 = static_cast<float>(p.disp_u1);
    p.f.disp_du = static_cast<float>(p.disp_du);
    p.f.kap_lo = static_cast<float>(p.kap_lo);
    p.f.kap_winv = static_cast<float>(p.kap_winv);
    for (int l = 0; l < 5; ++l) p.f.eta_coef[l] = static_cast<float>(p.atm.eta_coef[l]);
    p.f.earth_radius = static_cast<float>(p.earth_radius);
    p.f.r_o = static_cast<float>(p.r_o);
    p.f.inv_ro = static_cast<float>(p.inv_ro);
    p.f.inv_dsec = static_cast<float>(p.inv_dsec);
    for (int q = 0; q < 12; ++q) {
        p.f.gl_x[q] = static_cast<float>(p.gl_x[q]);
        p.f.gl_w[q] = static_cast<float>(p.gl_w[q]);
    }
    for (int l = 0; l < 6; ++l) p.f.hb[l] = static_cast<float>(p.atm.hb[l]);
    for (int l = 0; l < 5; ++l) {
        p.f.a[l] = static_cast<float>(p.atm.a[l]);
        p.f.b[l] = static_cast<float>(p.atm.b[l]);
        p.f.c[l] = static_cast<float>(p.atm.c[l]);
        p.f.inv_c[l] = static_cast<float>(p.atm.inv_c[l]);
        p.f.t_top[l] = static_cast<float>(p.atm.t_top[l]);
    }
}

namespace {
__global__ void k_round_to_float(const double *in, float *out, float *lo, int64_t n) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n;
         i += int64_t(gridDim.x) * blockDim.x) {
        if (lo)
            d2f_split(in[i], out[i], lo[i]);
        else
            out[i] = d2f_rn(in[i]);
    }
}
}  // namespace

size_t fallback_record_bytes(bool fp32) {
    static_assert(sizeof(FbEntry<float>) == 64 && sizeof(FbEntry<double>) == 112,
                  "fallback queue records");
    return fp32 ? sizeof(FbEntry<float>) : sizeof(FbEntry<double>);
}

template <class R>
void fallback_r(bool tr, bool disp, const KParams &p, int grid, cudaStream_t st) {
    if (disp) {
        if (tr) k_fallback<R, true, true><<<grid, 128, 0, st>>>(p);
        else k_fallback<R, false, true><<<grid, 128, 0, st>>>(p);
    } else {
        if (tr) k_fallback<R, true, false><<<grid, 128, 0, st>>>(p);
        else k_fallback<R, false, false><<<grid, 128, 0, st>>>(p);
    }
}

cudaError_t launch_fallback(bool fp32, bool tr, bool disp, const KParams &p, int num_sms,
                            void *stream) {
    const int grid = num_sms * 8;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (fp32) fallback_r<float>(tr, disp, p, grid, st);
    else fallback_r<double>(tr, disp, p, grid, st);
    return cudaGetLastError();
}

cudaError_t round_to_float(const double *in, float *out, float *lo, int64_t n, int num_sms,
                           void *stream) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, int64_t(num_sms) * 8);
    k_round_to_float<<<static_cast<int>(blocks), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        in, out, lo, n);
    return cudaGetLastError();
}

size_t kernel_smem_bytes(bool fp32, int block, const KParams &p) {
    if (fp32) {
        switch (block) {
        case 128: return smem_bytes<float, 128>(p);
        case 256: return smem_bytes<float, 256>(p);
        case 512: return smem_bytes<float, 512>(p);
        }
    } else {
        switch (block) {
        case 128: return smem_bytes<double, 128>(p);
        case 256: return smem_bytes<double, 256>(p);
        case 512: return smem_bytes<double, 512>(p);
        }
    }
    return 0;
}

cudaError_t kernel_prepare(bool fp32, int block, int mode, size_t smem) {
    const void *k = pick_kernel(fp32, block, mode);
    if (!k) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem));
}

int kernel_max_ctas_per_sm(bool fp32, int block, int mode, size_t smem) {
    const void *k = pick_kernel(fp32, block, mode);
    int n = 0;
    if (!k || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem) != cudaSuccess)
        return 0;
    return n;
}

cudaError_t kernel_launch(bool fp32, int block, int mode, int grid, size_t smem,
                          const KParams &p, void *stream) {
    const void *k = pick_kernel(fp32, block, mode);
    if (!k) return cudaErrorInvalidValue;
    void *args[] = {const_cast<KParams *>(&p)};
    return cudaLaunchKernel(k, dim3(grid), dim3(block), args, smem,
                            static_cast<cudaStream_t>(stream));
}

}  // namespace cher
