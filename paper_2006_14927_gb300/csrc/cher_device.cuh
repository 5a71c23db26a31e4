// cher_device.cuh -- device helpers shared by the fused kernel and the
// adjoint kernels: Philox4x32-10, uniform deviates, finiteness tests and the
// FP64 per-step yield whose rounding decides the bunch count.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "cher_internal.h"

namespace cher {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

// ------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Counter (lo(i), hi(i), j, 0), key
// (lo(seed), hi(seed)).
// ------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// uniform deviates in (0, 1)
__device__ __forceinline__ double u01d(uint32_t x) {
    return (static_cast<double>(x) + 0.5) * (1.0 / 4294967296.0);
}
__device__ __forceinline__ float u01f(uint32_t x) {
    // top 24 bits, centred: exactly representable, never 0 or 1
    return __uint2float_rz(x >> 8) * (1.0f / 16777216.0f) + (1.0f / 33554432.0f);
}

// ------------------------------------------------------------------------
// a1: per-step yield, FP64, one IEEE operation per statement in a fixed
// order (the bunch count must not depend on the precision of the rest).
// ------------------------------------------------------------------------
struct Yield {
    int nb;
    bool valid;
    double N, s2, g, gam, eta;
};

// finiteness from the exponent bits: integer ops only (GB300's FP64 pipe is
// about 1/64 of the FP32 rate, so the per-step code keeps off it where it can)
__device__ __forceinline__ bool finite_d(double v) {
    return (__double2hiint(v) & 0x7ff00000) != 0x7ff00000;
}
__device__ __forceinline__ bool finite_f(float v) {
    return (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u;
}

// double -> float with round-to-nearest-even (IEEE 754), on the integer
// pipes: keep the top 23 fraction bits, round on the 29 dropped ones, let a
// carry run into the exponent.  Results below the smallest normal float
// flush to zero (the FP32 path runs with flush-to-zero), results beyond the
// largest float become infinities, NaN stays NaN.
__device__ __forceinline__ float d2f_rn(double d) {
    const unsigned hi = static_cast<unsigned>(__double2hiint(d));
    const unsigned lo = static_cast<unsigned>(__double2loint(d));
    const unsigned sign = hi & 0x80000000u;
    const unsigned ex = (hi >> 20) & 0x7ffu;
    const int e = static_cast<int>(ex) - 1023 + 127;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    unsigned r = (static_cast<unsigned>(e) << 23) + m + up;
    r = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : r);
    if (ex == 0x7ffu && ((hi & 0xfffffu) | lo)) r = 0x7fc00000u;
    return __uint_as_float(r | sign);
}

// A double as an unevaluated float pair, hi + lo, on the integer pipes:
// hi = d2f_rn(d), and lo the float nearest to d - hi, which is the 29
// fraction bits hi dropped minus the rounding carry, R = rem - up 2^29,
// times 2^(E - 52) for the double's exponent E: R is converted to float and
// E - 52 added to its exponent field (|lo| <= ulp(hi) / 2, so hi + lo
// carries 48 bits).  lo is 0 where it would not be a normal float, and for
// zero, subnormal, infinite or NaN d.
__device__ __forceinline__ void d2f_split(double d, float &hi, float &lo) {
    hi = d2f_rn(d);
    const unsigned h = static_cast<unsigned>(__double2hiint(d));
    const unsigned l = static_cast<unsigned>(__double2loint(d));
    const unsigned ex = (h >> 20) & 0x7ffu;
    const unsigned m = ((h & 0xfffffu) << 3) | (l >> 29);
    const unsigned rem = l & 0x1fffffffu;
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    const int R = static_cast<int>(rem) - static_cast<int>(up << 29);
    const unsigned vb = __float_as_uint(static_cast<float>(R));
    const int ve = static_cast<int>((vb >> 23) & 0xffu);
    const int ne = ve + static_cast<int>(ex) - (1023 + 52);
    const bool ok = ve != 0 && ne > 0 && ne < 255 && ex != 0u && ex != 0x7ffu;
    const float a = ok ? __uint_as_float((vb & 0x807fffffu) | (static_cast<unsigned>(ne) << 23))
                       : 0.0f;
    lo = (h & 0x80000000u) ? -a : a;
}

// The bounds-checked build (compiled with CHER_DEBUG): an index about to be
// used is checked against its array; a bad one sets `bit` in
// stats[CHER_STAT_DEBUG] and is replaced by 0, so the access stays inside
// the array and nothing traps.  The regular build compiles the check away.
template <class I>
__device__ __forceinline__ I dbg_index(const KParams &p, I i, int64_t n, unsigned bit) {
#ifdef CHER_DEBUG
    if (i < 0 || static_cast<int64_t>(i) >= n) {
        if (p.stats) atomicOr(p.stats + CHER_STAT_DEBUG, static_cast<unsigned long long>(bit));
        return I(0);
    }
#else
    (void)p;
    (void)n;
    (void)bit;
#endif
    return i;
}
enum : unsigned { DBG_ETA = 1u, DBG_TAB = 2u, DBG_GRID = 4u, DBG_OUT = 8u, DBG_TRACE = 16u,
                  DBG_SMEM = 32u, DBG_FB = 64u };

__device__ __forceinline__ double eta_exact_lookup(const KParams &p, double h) {
    double hc = h;
    if (hc < 0.0) hc = 0.0;
    if (hc > p.h_max) hc = p.h_max;
    const double x = __dmul_rn(hc, p.inv_dh);
    int k = static_cast<int>(x);
    if (k > p.n_fine - 2) k = p.n_fine - 2;
    const double f = __dsub_rn(x, static_cast<double>(k));
    k = dbg_index(p, k, p.n_fine - 1, DBG_ETA);
    const double t0 = __ldg(p.eta64 + k), t1 = __ldg(p.eta64 + k + 1);
    const double d = __dsub_rn(t1, t0);
    const double fd = __dmul_rn(f, d);
    return __dadd_rn(t0, fd);
}

// A step emits only if every field is finite, len >= 0 and ekin > 0.
template <class R>
__device__ __forceinline__ bool finite_r(R v) {
    if constexpr (std::is_same<R, float>::value) return finite_f(v);
    else return finite_d(v);
}

template <class R>
__device__ __forceinline__ bool step_valid(const KParams &p, int64_t i) {
    return finite_d(__ldg(p.x0 + i)) && finite_d(__ldg(p.y0 + i)) && finite_d(__ldg(p.t0 + i)) &&
           finite_r<R>(__ldg(static_cast<const R *>(p.ux) + i)) &&
           finite_r<R>(__ldg(static_cast<const R *>(p.uy) + i));
}

// In a curved atmosphere the index is taken at the radial height of the
// step's midpoint, |x_m - C| - R_E = h_m + rho^2 / (sqrt(rho^2 + (h_m + R_E)^2) + h_m + R_E),
// in the oracle's order.  xy = {x0, y0, ux, uy}.
__device__ __forceinline__ double curved_midpoint(const KParams &p, double hm, double half_len,
                                                  const double *xy) {
    const double dx = __dmul_rn(half_len, xy[2]);
    const double xm = __dadd_rn(xy[0], dx);
    const double dy = __dmul_rn(half_len, xy[3]);
    const double ym = __dadd_rn(xy[1], dy);
    const double xx = __dmul_rn(xm, xm);
    const double yy = __dmul_rn(ym, ym);
    const double rho2 = __dadd_rn(xx, yy);
    const double Rp = __dadd_rn(hm, p.earth_radius);
    const double RR = __dmul_rn(Rp, Rp);
    const double r2 = __dadd_rn(rho2, RR);
    const double r = __dsqrt_rn(r2);
    const double den = __dadd_rn(r, Rp);
    const double corr = __ddiv_rn(rho2, den);
    return __dadd_rn(hm, corr);
}

__device__ __forceinline__ void step_yield(const KParams &p, bool others_valid, double z0,
                                           double len, double ekin, double uz, Yield &y,
                                           const double *xy = nullptr) {
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
    const double np1 = __dadd_rn(1.0, eta);
    const double np1sq = __dmul_rn(np1, np1);
    const double two_eta = __dadd_rn(2.0, eta);
    const double a = __dmul_rn(eta, two_eta);
    const double b = __dmul_rn(a, gam2);
    const double num = __dsub_rn(b, np1sq);
    const double two_g = __dadd_rn(2.0, g);
    const double bg2 = __dmul_rn(g, two_g);
    const double den = __dmul_rn(bg2, np1sq);
    const double s2 = __ddiv_rn(num, den);
    y.g = g;
    y.gam = gam;
    y.eta = eta;
    y.valid = true;
    if (!(s2 > 0.0)) return;
    const double Ks2 = __dmul_rn(p.K, s2);
    const double N = __dmul_rn(len, Ks2);
    const double q = __dmul_rn(N, p.inv_B);
    if (!(q < 4194304.0)) {                    // more than 2^22 bunches: invalid
        y.valid = false;
        return;
    }
    y.nb = static_cast<int>(ceil(q));
    y.N = N;
    y.s2 = s2;
}

}  // namespace dev
}  // namespace cher
