// cher_adjoint.cu -- gradients of the telescope read-out with respect to the
// atmosphere and the track steps (no counterpart in the paper: the paper's
// path is a forward simulation; this is its differentiable extension).
//
// Read-out, per telescope k (sigma the smoothing length):
//   S_k = sum_b w_b G(r_bk),  U_k = sum_b w_b G(r_bk) t_b,
//   G(r) = exp(-r^2 / 2 sigma^2) / (2 pi sigma^2) for r < 6 sigma,
//   D_k = S_k (photon density), Tbar_k = U_k / S_k (mean arrival time),
// with r_bk the distance in the observation plane from bunch b's ground point
// to the telescope centre, and the bunch counts nb frozen.
// Loss L = sum_k dL/dD_k D_k + dL/dTbar_k Tbar_k (the caller's upstream
// gradients).
//
// Only the bunches that land within 6 sigma of a centre contribute.  The
// fused kernel (screen mode) lists them in one FP32 pass over all bunches;
// here one thread per listed bunch recomputes that bunch from its Philox
// counter (no stored intermediates) in forward-mode dual numbers with 11
// tangents -- the six step inputs (x0, y0, z0, ux, uy, uz) and five
// "channels" through which the atmosphere enters (n at the step midpoint, n
// at the emission point, n at the observation level, and the two refraction
// corrections) -- and turns dL/d(X, Y, t, w) into gradients, accumulated in
// FP64 with atomics.  The atmosphere gradient chains the channels through
// the sensitivity tables d(table)/d(b_i, c_i) built on the host; n does not
// depend on a_i, whose gradient is exactly zero.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "cher_device.cuh"
#include "cher_internal.h"

namespace cher {
namespace {

using namespace dev;

constexpr int NT = 11;   // tangents
enum { T_X0 = 0, T_Y0, T_Z0, T_UX, T_UY, T_UZ, C_ETA_M, C_ETA_E, C_ETA_O, C_AX, C_AL };

template <class T>
struct Dual {
    T v;
    T d[NT];
};

template <class T>
__device__ __forceinline__ Dual<T> cst(T v) {
    Dual<T> r;
    r.v = v;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = T(0);
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> var(T v, int idx) {
    Dual<T> r = cst<T>(v);
    r.d[idx] = T(1);
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator+(const Dual<T> &a, const Dual<T> &b) {
    Dual<T> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator-(const Dual<T> &a, const Dual<T> &b) {
    Dual<T> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator-(const Dual<T> &a) {
    Dual<T> r;
    r.v = -a.v;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = -a.d[i];
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator*(const Dual<T> &a, const Dual<T> &b) {
    Dual<T> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator*(T s, const Dual<T> &a) {
    Dual<T> r;
    r.v = s * a.v;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = s * a.d[i];
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator+(T s, const Dual<T> &a) {
    Dual<T> r = a;
    r.v = s + a.v;
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> operator/(const Dual<T> &a, const Dual<T> &b) {
    Dual<T> r;
    const T inv = T(1) / b.v;
    r.v = a.v * inv;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * inv;
    return r;
}
template <class T>
__device__ __forceinline__ Dual<T> dsqrt(const Dual<T> &a) {
    Dual<T> r;
    r.v = sqrt(a.v);
    const T h = T(0.5) / r.v;
#pragma unroll
    for (int i = 0; i < NT; ++i) r.d[i] = a.d[i] * h;
    return r;
}

template <class T>
__device__ __forceinline__ T tdir(const void *p, int64_t i) {
    return __ldg(static_cast<const T *>(p) + i);
}

// fine-table eta at a dual height: value, slope along the height, plus the
// tangent of its own atmosphere channel
template <class T>
__device__ __forceinline__ Dual<T> eta_dual(const KParams &p, const Dual<T> &h, int channel,
                                            int &k_out, T &f_out) {
    T hc = h.v;
    if (hc < T(0)) hc = T(0);
    if (hc > T(p.h_max)) hc = T(p.h_max);
    const T x = hc * T(p.inv_dh);
    int k = static_cast<int>(x);
    k = k > p.n_fine - 2 ? p.n_fine - 2 : k;
    const T f = x - static_cast<T>(k);
    T t0, t1;
    if constexpr (std::is_same<T, float>::value) {
        t0 = __ldg(p.eta32 + k);
        t1 = __ldg(p.eta32 + k + 1);
    } else {
        t0 = __ldg(p.eta64 + k);
        t1 = __ldg(p.eta64 + k + 1);
    }
    const bool inside = h.v > T(0) && h.v < T(p.h_max);
    const T slope = inside ? (t1 - t0) * T(p.inv_dh) : T(0);
    Dual<T> r = slope * h;
    r.v = t0 + f * (t1 - t0);
    r.d[channel] += T(1);
    k_out = k;
    f_out = f;
    return r;
}

// d eta / d p of the fine-table value at node position (k, f): the nodes'
// analytic sensitivities, interpolated like the values
__device__ __forceinline__ void eta_sens(const AdjParams &a, int k, double f, double *d) {
    for (int q = 0; q < 10; ++q) d[q] = 0.0;
    for (int side = 0; side < 2; ++side) {
        const int kk = k + side;
        const double wgt = side ? f : 1.0 - f;
        const double h = static_cast<double>(kk) * a.dh_fine;
        if (h >= a.hb[5]) continue;
        int i = 0;
        while (i < 4 && h >= a.hb[i + 1]) ++i;
        const double e = __ldg(a.k.eta64 + kk) * wgt;
        d[i] += e / a.b[i];
        d[a.layer0] -= e / a.b[a.layer0];
        d[5 + i] += e * (h - a.c[i]) / (a.c[i] * a.c[i]);
        d[5 + a.layer0] += e / a.c[a.layer0];
    }
}

// one listed bunch, recomputed in dual numbers; returns false if it does not
// reach the ground
template <class T>
struct BunchDual {
    Dual<T> X, Y, t, w;
    // table cell for the sensitivities
    int jj, kk, km, ke;
    T a, b, fm, fe;
    double hm, he;
};

template <class T>
__device__ bool bunch_dual(const AdjParams &A, int64_t i, int j, BunchDual<T> &o) {
    const KParams &p = A.k;
    const int nb = __ldg(A.nb + i);
    const Dual<T> x0 = var<T>(static_cast<T>(__ldg(p.x0 + i)), T_X0);
    const Dual<T> y0 = var<T>(static_cast<T>(__ldg(p.y0 + i)), T_Y0);
    const Dual<T> z0 = var<T>(static_cast<T>(__ldg(p.z0 + i)), T_Z0);
    const Dual<T> ux = var<T>(tdir<T>(p.ux, i), T_UX);
    const Dual<T> uy = var<T>(tdir<T>(p.uy, i), T_UY);
    const Dual<T> uz = var<T>(tdir<T>(p.uz, i), T_UZ);
    const T len = static_cast<T>(__ldg(p.len + i));
    const double ekin = __ldg(p.ekin + i);
    double t_ref = 0.0;
    if (p.t_ref) {
        const uint32_t sh = p.shower ? __ldg(p.shower + i) : 0u;
        if (static_cast<int32_t>(sh) < p.n_showers) t_ref = __ldg(p.t_ref + sh);
    }
    // yield at the step midpoint (a1), nb frozen
    const T g = static_cast<T>(ekin * p.inv_me);
    const T gam = T(1) + g;
    const T gam2 = gam * gam;
    const Dual<T> hm = z0 + (T(0.5) * len) * uz;
    const Dual<T> eta_m = eta_dual<T>(p, hm, C_ETA_M, o.km, o.fm);
    o.hm = static_cast<double>(hm.v);
    const Dual<T> np1 = T(1) + eta_m;
    const Dual<T> np1sq = np1 * np1;
    const Dual<T> num = gam2 * (eta_m * (T(2) + eta_m)) - np1sq;
    const T bg2 = g * (T(2) + g);
    const Dual<T> s2 = num / (bg2 * np1sq);
    if (!(s2.v > T(0)) || nb <= 0) return false;
    const Dual<T> w = (static_cast<T>(p.K) * len / static_cast<T>(nb)) * s2;
    const T beta = sqrt(bg2) / gam;
    const Dual<T> cosc = cst<T>(T(1)) / (beta * np1);
    const Dual<T> sinc = dsqrt(s2);
    // azimuth basis around the step
    const Dual<T> rho2 = ux * ux + uy * uy;
    Dual<T> e1x, e1y;
    if (rho2.v > T(1e-20)) {
        const Dual<T> r = dsqrt(rho2);
        e1x = -uy / r;
        e1y = ux / r;
    } else {
        e1x = cst<T>(T(1));
        e1y = cst<T>(T(0));
    }
    const Dual<T> e2x = -(uz * e1y), e2y = uz * e1x, e2z = ux * e1y - uy * e1x;
    // randoms (a2)
    const int64_t gi = p.track_base + i;
    const uint4 x = philox4x32_10(
        make_uint4(static_cast<uint32_t>(gi), static_cast<uint32_t>(static_cast<uint64_t>(gi) >> 32),
                   static_cast<uint32_t>(j), 0u),
        p.key0, p.key1);
    T u0, u1;
    if constexpr (std::is_same<T, float>::value) {
        u0 = u01f(x.x);
        u1 = u01f(x.y);
    } else {
        u0 = u01d(x.x);
        u1 = u01d(x.y);
    }
    const T fl = (static_cast<T>(j) + u0) / static_cast<T>(nb) * len;
    T sp, cp;
    if constexpr (std::is_same<T, float>::value) sincospif(2.0f * u1, &sp, &cp);
    else sincospi(2.0 * u1, &sp, &cp);
    const Dual<T> px = cosc * ux + sinc * (cp * e1x + sp * e2x);
    const Dual<T> py = cosc * uy + sinc * (cp * e1y + sp * e2y);
    const Dual<T> pz = cosc * uz + sinc * (sp * e2z);
    const Dual<T> xe = x0 + fl * ux, ye = y0 + fl * uy, he = z0 + fl * uz;
    const T te = static_cast<T>(__ldg(p.t0 + i) - t_ref) + fl / (beta * T(kC));
    // rare conditions (a3)
    if (!(pz.v < T(0)) || !(he.v >= T(p.h_obs)) || !(he.v <= T(p.h_max))) return false;
    const Dual<T> eta_e = eta_dual<T>(p, he, C_ETA_E, o.ke, o.fe);
    o.he = static_cast<double>(he.v);
    Dual<T> eta_o = cst<T>(static_cast<T>(p.eta_obs));
    eta_o.d[C_ETA_O] = T(1);
    const Dual<T> se2 = px * px + py * py;
    if (!(se2.v > T(0))) return false;
    const Dual<T> sin_em = dsqrt(se2);
    const Dual<T> rat = (T(1) + eta_e) / (T(1) + eta_o);
    const Dual<T> sin_obs = sin_em * rat;
    const Dual<T> q = sin_obs * sin_obs;
    if (!(q.v <= static_cast<T>(p.q_max))) return false;
    const Dual<T> cos_obs = dsqrt(cst<T>(T(1)) - q);
    const Dual<T> dH = he - cst<T>(static_cast<T>(p.h_obs));
    // table cell: value, slopes along dH and q, plus the table channels
    const T fj = dH.v * static_cast<T>(p.inv_dht);
    int jj = static_cast<int>(fj);
    jj = jj > p.H - 2 ? p.H - 2 : jj;
    jj = jj < 0 ? 0 : jj;
    const T a = fj - static_cast<T>(jj);
    const T fk = q.v * static_cast<T>(p.inv_dq);
    int kk = static_cast<int>(fk);
    kk = kk > p.Z - 2 ? p.Z - 2 : kk;
    kk = kk < 0 ? 0 : kk;
    const T b = fk - static_cast<T>(kk);
    T c00x, c01x, c10x, c11x, c00l, c01l, c10l, c11l;
    {
        if constexpr (std::is_same<T, float>::value) {
            // (flat layers: one float2 (ax, al) per node)
            const float2 *Tb = static_cast<const float2 *>(p.tab);
            const int n0 = jj * p.Z + kk;
            const float2 a0 = __ldg(Tb + n0), a1 = __ldg(Tb + n0 + 1);
            const float2 b0 = __ldg(Tb + n0 + p.Z), b1 = __ldg(Tb + n0 + p.Z + 1);
            c00x = a0.x; c00l = a0.y; c01x = a1.x; c01l = a1.y;
            c10x = b0.x; c10l = b0.y; c11x = b1.x; c11l = b1.y;
        } else {
            const double2 *Tb = static_cast<const double2 *>(p.tab);
            const int n0 = jj * p.Z + kk;
            const double2 a0 = __ldg(Tb + n0), a1 = __ldg(Tb + n0 + 1);
            const double2 b0 = __ldg(Tb + n0 + p.Z), b1 = __ldg(Tb + n0 + p.Z + 1);
            c00x = a0.x; c00l = a0.y; c01x = a1.x; c01l = a1.y;
            c10x = b0.x; c10l = b0.y; c11x = b1.x; c11l = b1.y;
        }
    }
    auto cell = [&](T v00, T v01, T v10, T v11, int channel) {
        const T v0 = v00 + a * (v10 - v00), v1 = v01 + a * (v11 - v01);
        const T dvdh = ((T(1) - b) * (v10 - v00) + b * (v11 - v01)) * static_cast<T>(p.inv_dht);
        const T dvdq = ((T(1) - a) * (v01 - v00) + a * (v11 - v10)) * static_cast<T>(p.inv_dq);
        Dual<T> r = dvdh * dH + dvdq * q;
        r.v = v0 + b * (v1 - v0);
        r.d[channel] += T(1);
        return r;
    };
    const Dual<T> Ax = cell(c00x, c01x, c10x, c11x, C_AX);
    const Dual<T> Al = cell(c00l, c01l, c10l, c11l, C_AL);
    const Dual<T> sec = cst<T>(T(1)) / cos_obs;
    const Dual<T> sec2 = sec * sec;
    const Dual<T> tn = sin_obs * sec;
    const Dual<T> Dh = dH * tn + Ax * tn * sec2;
    const Dual<T> Lp = dH * sec + Al * sec2 * sec;
    const Dual<T> hx = px / sin_em, hy = py / sin_em;
    o.X = xe + Dh * hx;
    o.Y = ye + Dh * hy;
    o.t = static_cast<T>(1.0 / kC) * Lp;
    o.t.v += te;
    o.w = w;
    o.jj = jj;
    o.kk = kk;
    o.a = a;
    o.b = b;
    return true;
}

// Sums that many pairs add to the same few addresses (S_k, U_k per
// telescope; the ten atmosphere gradients) are combined per CTA in shared
// memory first, then added to global memory once per CTA: the pairs of a
// shower crowd around a handful of telescopes.
constexpr int kSmemTel = 512;     // telescopes whose S, U are combined in smem

template <class T, int MODE>
__global__ void __launch_bounds__(128) k_adj_pairs(const AdjParams A) {
    __shared__ double s_sum[MODE == 0 ? 2 * kSmemTel : 10];
    const int n_tel = A.k.n_tel;
    const bool smem_su = MODE == 0 && n_tel <= kSmemTel;
    const int n_red = MODE == 0 ? (smem_su ? 2 * n_tel : 0) : 10;
    for (int q = threadIdx.x; q < n_red; q += blockDim.x) s_sum[q] = 0.0;
    __syncthreads();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < A.n_list;
         e += stride) {
        const uint64_t ent = A.list[e];
        const int64_t i = static_cast<int64_t>(ent >> 32);
        const int j = static_cast<int>(ent & 0xffffffffu);
        BunchDual<T> o;
        if (!bunch_dual<T>(A, i, j, o)) continue;
        const double X = o.X.v, Y = o.Y.v, t = o.t.v, w = o.w.v;
        double gX = 0, gY = 0, gt = 0, gw = 0;
        bool any = false;
        for (int k = 0; k < A.k.n_tel; ++k) {
            double tx, ty;
            if constexpr (std::is_same<T, float>::value) {
                const float4 Tt = __ldg(static_cast<const float4 *>(A.k.tel) + k);
                tx = Tt.x;
                ty = Tt.y;
            } else {
                const double2 Tt = __ldg(static_cast<const double2 *>(A.k.tel) + 2 * k);
                tx = Tt.x;
                ty = Tt.y;
            }
            const double dx = X - tx, dy = Y - ty;
            const double r2 = dx * dx + dy * dy;
            if (!(r2 < A.rcut2)) continue;
            const double G = A.norm * exp(-r2 * A.inv_2s2);
            if constexpr (MODE == 0) {
                if (smem_su) {
                    atomicAdd(s_sum + k, w * G);
                    atomicAdd(s_sum + n_tel + k, w * G * t);
                } else {
                    atomicAdd(A.S + k, w * G);
                    atomicAdd(A.U + k, w * G * t);
                }
            } else {
                const double S = __ldg(A.S + k), U = __ldg(A.U + k);
                double dLdS = __ldg(A.gD + k), dLdU = 0.0;
                if (S > 0.0) {
                    const double gT = __ldg(A.gT + k);
                    dLdS -= gT * (U / S) / S;
                    dLdU = gT / S;
                }
                const double q = dLdS + dLdU * t;        // dL / d(w G)
                gw += G * q;
                gt += w * G * dLdU;
                const double dGr = -G * A.inv_2s2;         // dG / d(r^2)
                gX += w * q * dGr * 2.0 * dx;
                gY += w * q * dGr * 2.0 * dy;
                any = true;
            }
        }
        if constexpr (MODE == 1) {
            if (!any) continue;
            double gl[NT];
#pragma unroll
            for (int c = 0; c < NT; ++c)
                gl[c] = gX * static_cast<double>(o.X.d[c]) + gY * static_cast<double>(o.Y.d[c]) +
                        gt * static_cast<double>(o.t.d[c]) + gw * static_cast<double>(o.w.d[c]);
            for (int m = 0; m < 6; ++m) atomicAdd(A.grad_tracks + m * A.k.n + i, gl[m]);
            // atmosphere: the five channels through their sensitivities
            double dm[10], de[10], dob[10];
            eta_sens(A, o.km, static_cast<double>(o.fm), dm);
            eta_sens(A, o.ke, static_cast<double>(o.fe), de);
            eta_sens(A, A.ko, A.fo, dob);
            const double *s00 = A.sens + (static_cast<size_t>(o.jj) * A.k.Z + o.kk) * 20;
            const double *s01 = s00 + 20;
            const double *s10 = s00 + static_cast<size_t>(A.k.Z) * 20;
            const double *s11 = s10 + 20;
            const double aa = o.a, bb = o.b;
            for (int q = 0; q < 10; ++q) {
                double tab[2];
                for (int m = 0; m < 2; ++m) {
                    const int idx = m * 10 + q;
                    const double v0 = __ldg(s00 + idx) + aa * (__ldg(s10 + idx) - __ldg(s00 + idx));
                    const double v1 = __ldg(s01 + idx) + aa * (__ldg(s11 + idx) - __ldg(s01 + idx));
                    tab[m] = v0 + bb * (v1 - v0);
                }
                const double gp = gl[C_ETA_M] * dm[q] + gl[C_ETA_E] * de[q] +
                                  gl[C_ETA_O] * dob[q] + gl[C_AX] * tab[0] + gl[C_AL] * tab[1];
                atomicAdd(s_sum + q, gp);            // b_i at 5 + i, c_i at 10 + i
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < n_red; q += blockDim.x) {
        const double v = s_sum[q];
        if (v == 0.0) continue;
        if constexpr (MODE == 0)
            atomicAdd(q < n_tel ? A.S + q : A.U + (q - n_tel), v);
        else
            atomicAdd(A.grad_atm + 5 + q, v);
    }
}

template <class T, int MODE>
cudaError_t launch_pairs(const AdjParams &A, void *stream) {
    if (A.n_list == 0) return cudaSuccess;
    const int block = 128;
    const int64_t want = (A.n_list + block - 1) / block;
    const int grid = static_cast<int>(want < 4096 ? want : 4096);
    k_adj_pairs<T, MODE><<<grid, block, 0, static_cast<cudaStream_t>(stream)>>>(A);
    return cudaGetLastError();
}

}  // namespace

cudaError_t adjoint_pairs(bool fp32, int mode, const AdjParams &A, void *stream) {
    if (fp32) return mode == 0 ? launch_pairs<float, 0>(A, stream) : launch_pairs<float, 1>(A, stream);
    return mode == 0 ? launch_pairs<double, 0>(A, stream) : launch_pairs<double, 1>(A, stream);
}

}  // namespace cher
