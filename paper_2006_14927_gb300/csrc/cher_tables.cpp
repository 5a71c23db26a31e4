// cher_tables.cpp -- step a0: atmosphere tables and the telescope grid,
// built once per context on the host in double precision.
//
// * Fine table of eta = n - 1 at n_fine uniformly spaced heights on
//   [0, h_max]: the paper's "fast interpolation" (section 3.3.2), which
//   replaces the per-call binary search over ~55 tabulated altitudes
//   (section 3.3.1) by an index computed from a uniform step.
// * Refraction-correction tables (section 3.3.1: "coefficients for air
//   refraction correction"; section 3.3.2 extends fast interpolation to them)
//   over uniform heights and uniform squared sines of the observation-level
//   zenith angle.  For a ray that reaches the observation level at zenith
//   theta_o, Snell's law in flat layers (n(h) sin theta(h) = n_o sin theta_o)
//   gives its horizontal offset x(h) and optical path l(h) between h_obs and
//   h.  The tables store the differences to the straight line at theta_o,
//   divided by their leading angular factors:
//       ax = (x - dH tan theta_o) cos^3 theta_o / sin theta_o
//       al = (l - dH / cos theta_o) cos^3 theta_o
//   so that bilinear interpolation stays accurate up to the largest angles.
//   The integrals are split at layer boundaries (the density jumps there)
//   and done with fixed 12-point Gauss-Legendre rules on each piece, with
//   the integrands rewritten so that no difference of nearly equal numbers
//   is formed.
// * Ground grid: every telescope is listed in each cell its conservative
//   reach disc touches, so a bunch only tests the spheres of its own cell.
#include <algorithm>
#include <cmath>
#include <thread>

#include "cher_internal.h"

namespace cher {
namespace {

struct Layered {
    double hb[6], a[5], b[5], c[5], n0m1, rho0;
};

int layer_of(const Layered &A, double h) {
    int i = 0;
    while (i < 4 && h >= A.hb[i + 1]) ++i;
    return i;
}

// rho(h) = (b_i / c_i) exp(-h / c_i); zero above the top of the atmosphere.
double rho(const Layered &A, double h) {
    if (h >= A.hb[5]) return 0.0;
    const int i = layer_of(A, h);
    const double r = A.b[i] / A.c[i];
    const double e = std::exp(-(h / A.c[i]));
    return r * e;
}

// eta = n0_minus_1 * rho / rho(0), evaluated in this order (the bunch count
// depends on the exact rounding of the fine-table entries).
double eta_of(const Layered &A, double h) {
    const double r = rho(A, h);
    const double q = r / A.rho0;
    return A.n0m1 * q;
}

Layered make_layered(const cher_atmosphere &atm) {
    Layered A;
    for (int i = 0; i < 6; ++i) A.hb[i] = atm.h_bound[i];
    for (int i = 0; i < 5; ++i) { A.a[i] = atm.a[i]; A.b[i] = atm.b[i]; A.c[i] = atm.c[i]; }
    A.n0m1 = atm.n0_minus_1;
    A.rho0 = 1.0;
    A.rho0 = rho(A, 0.0);
    return A;
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n.
struct GaussLegendre {
    static constexpr int N = 12;
    double x[N], w[N];
    GaussLegendre() {
        for (int i = 0; i < N; ++i) {
            double z = std::cos(kPi * (i + 0.75) / (N + 0.5));
            for (int it = 0; it < 100; ++it) {
                double p0 = 1.0, p1 = 0.0;
                for (int k = 1; k <= N; ++k) {
                    const double p2 = p1;
                    p1 = p0;
                    p0 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p2) / k;
                }
                const double dp = N * (z * p0 - p1) / (z * z - 1.0);
                const double dz = p0 / dp;
                z -= dz;
                if (std::fabs(dz) < 1e-16) {
                    x[i] = z;
                    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
                    break;
                }
                x[i] = z;
                w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
            }
        }
    }
};

// Integrands of ax and al at height h for a ray with observation sine so,
// cosine co (co = sqrt(1 - so^2)).  With r = n_o / n(h) = (1 + eta_o)/(1 + eta),
// s = so r and c = sqrt(1 - s^2):
//   tan(theta) - tan(theta_o) = so (r - 1)(r + 1) / ((r co + c) c co)
//   1/c - 1/co                = so^2 (r - 1)(r + 1) / ((co + c) c co)
// so that, after the normalisation,
//   d(ax)/dh = (r - 1)(r + 1) co^2 / ((r co + c) c)
//   d(al)/dh = eta co^3 / c + so^2 (r - 1)(r + 1) co^2 / ((co + c) c)
// with r - 1 = (eta_o - eta) / (1 + eta) formed without cancellation.
struct RayIntegrand {
    const Layered *A;
    double eta_o, so, co;
    void operator()(double h, double &gx, double &gl) const {
        const double eta = eta_of(*A, h);
        const double rm1 = (eta_o - eta) / (1.0 + eta);
        const double r = 1.0 + rm1;
        const double s = so * r;
        const double c = std::sqrt((1.0 - s) * (1.0 + s));
        const double rr = rm1 * (r + 1.0);
        const double co2 = co * co;
        gx = rr * co2 / ((r * co + c) * c);
        gl = eta * co2 * co / c + so * so * rr * co2 / ((co + c) * c);
    }
};

// The curved atmosphere's integrands (spherical shells, Bouguer's
// invariant n r sin(zeta) = n_o r_o s_o): at height h, with w = r_o / r and
// v = n_o / n (v - 1 = (eta_o - eta) / (1 + eta)), the ray's sine is
// s = s_o v w and the straight reference line's s_s = s_o w, and
//   tan(zeta) - tan(zeta_s) = s_o w [(v - 1) c_s + (c_s - c)] / (c c_s),
//   1/c - 1/c_s = (c_s - c) / (c c_s),  c_s - c = s_o^2 w^2 (v - 1)(v + 1) / (c_s + c),
// so the three corrections (central angle times r_o, the (n - 1) part and
// the geometric part of the optical path) are free of cancellation:
//   g_phi = w (tan - tan_s),  g_1 = (n - 1) / c,  g_2 = 1/c - 1/c_s.
// At s_o = 0 the tables hold their limits divided by s_o and s_o^2:
//   w^2 (v - 1)  and  w^2 (v - 1)(v + 1) / 2.
struct CurvedIntegrand {
    const Layered *A;
    double R_E, r_o, eta_o, so;
    void operator()(double h, double &gp, double &g1, double &g2) const {
        const double eta = eta_of(*A, h);
        const double vm1 = (eta_o - eta) / (1.0 + eta);
        const double v = 1.0 + vm1;
        const double w = r_o / (R_E + h);
        if (so == 0.0) {
            gp = w * w * vm1;
            g1 = eta;
            g2 = 0.5 * w * w * vm1 * (v + 1.0);
            return;
        }
        const double ss = so * w, s = ss * v;
        const double cs = std::sqrt((1.0 - ss) * (1.0 + ss));
        const double c = std::sqrt((1.0 - s) * (1.0 + s));
        const double dc = so * so * w * w * vm1 * (v + 1.0) / (cs + c);   // c_s - c
        gp = w * so * w * (vm1 * cs + dc) / (c * cs);
        g1 = eta / c;
        g2 = dc / (c * cs);
    }
};

// Path averages of the three first-order factors along the straight line
// that arrives at r_o with sine s_o, up to r_e (u = r_o / r_e, c_e' its
// cosine at r_e, from c_e'^2 = c_o^2 + s_o^2 (1 - u)(1 + u)):
//   G_phi = u s_o (1 + u) / ((c_e' + u c_o) c_o c_e'),  G_1 = (1 + u) / (c_e' + u c_o),
//   G_2 = G_1 s_o^2 u / (c_e' c_o).
void curved_factors(double r_o, double r_e, double so, double co, double &g_phi, double &g_1,
                    double &g_2) {
    const double u = r_o / r_e;
    const double ce = std::sqrt(co * co + so * so * ((r_e - r_o) / r_e) * (1.0 + u));
    g_1 = (1.0 + u) / (ce + u * co);
    g_phi = u * so * g_1 / (co * ce);
    g_2 = g_1 * so * so * u / (ce * co);
}

void integrate_piece_c(const CurvedIntegrand &f, const GaussLegendre &gl, double lo, double hi,
                       double &ip, double &i1, double &i2) {
    const double m = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
    double sp = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < GaussLegendre::N; ++i) {
        double gp, g1, g2;
        f(m + hw * gl.x[i], gp, g1, g2);
        sp += gl.w[i] * gp;
        s1 += gl.w[i] * g1;
        s2 += gl.w[i] * g2;
    }
    ip = sp * hw;
    i1 = s1 * hw;
    i2 = s2 * hw;
}

void integrate_c(const CurvedIntegrand &f, const GaussLegendre &gl, double lo, double hi,
                 double &ip, double &i1, double &i2) {
    ip = i1 = i2 = 0.0;
    double a = lo;
    for (int i = 1; i <= 5; ++i) {
        const double hb = f.A->hb[i];
        if (hb > a && hb < hi) {
            double p, q1, q2;
            integrate_piece_c(f, gl, a, hb, p, q1, q2);
            ip += p; i1 += q1; i2 += q2;
            a = hb;
        }
    }
    double p, q1, q2;
    integrate_piece_c(f, gl, a, hi, p, q1, q2);
    ip += p; i1 += q1; i2 += q2;
}

void integrate_piece(const RayIntegrand &f, const GaussLegendre &gl, double lo, double hi,
                     double &ix, double &il) {
    const double m = 0.5 * (lo + hi), hw = 0.5 * (hi - lo);
    double sx = 0.0, sl = 0.0;
    for (int i = 0; i < GaussLegendre::N; ++i) {
        double gx, gL;
        f(m + hw * gl.x[i], gx, gL);
        sx += gl.w[i] * gx;
        sl += gl.w[i] * gL;
    }
    ix = sx * hw;
    il = sl * hw;
}

// integral over [lo, hi], split at the layer boundaries inside it
void integrate(const RayIntegrand &f, const GaussLegendre &gl, double lo, double hi,
               double &ix, double &il) {
    ix = il = 0.0;
    double a = lo;
    for (int i = 1; i <= 5; ++i) {
        const double hb = f.A->hb[i];
        if (hb > a && hb < hi) {
            double px, pl;
            integrate_piece(f, gl, a, hb, px, pl);
            ix += px;
            il += pl;
            a = hb;
        }
    }
    double px, pl;
    integrate_piece(f, gl, a, hi, px, pl);
    ix += px;
    il += pl;
}

bool atm_valid(const cher_atmosphere &atm) {
    for (int i = 0; i < 5; ++i) {
        if (!(atm.c[i] > 0.0) || !(atm.b[i] >= 0.0) || !std::isfinite(atm.a[i]) ||
            !std::isfinite(atm.b[i]) || !std::isfinite(atm.c[i]))
            return false;
        if (!(atm.h_bound[i + 1] > atm.h_bound[i])) return false;
    }
    if (!std::isfinite(atm.h_bound[0]) || !std::isfinite(atm.h_bound[5])) return false;
    if (!(atm.n0_minus_1 >= 0.0 && atm.n0_minus_1 < 0.01)) return false;
    if (!(atm.b[0] > 0.0)) return false;
    return true;
}

}  // namespace

double eta_lookup(const HostTables &t, double h) {
    double hc = h;
    if (hc < 0.0) hc = 0.0;
    if (hc > t.h_max) hc = t.h_max;
    const double x = hc * t.inv_dh;
    int k = static_cast<int>(x);
    if (k > t.n_fine - 2) k = t.n_fine - 2;
    const double f = x - static_cast<double>(k);
    const double d = t.eta[k + 1] - t.eta[k];
    const double fd = f * d;
    return t.eta[k] + fd;
}

cher_status build_tables(const cher_atmosphere &atm, double h_obs, int32_t n_fine, int32_t H,
                         int32_t Z, double theta_max, double h_max, HostTables &T,
                         double earth_radius) {
    if (!atm_valid(atm)) return CHER_EINVAL;
    if (n_fine < 2 || n_fine > (1 << 20)) return CHER_EINVAL;
    if (H < 2 || H > 65536 || Z < 2 || Z > 4096) return CHER_EINVAL;
    if (!(theta_max > 0.0) || !(theta_max < 85.0 * kPi / 180.0)) return CHER_EINVAL;
    if (!std::isfinite(h_obs) || !(h_max > h_obs) || !(h_max <= atm.h_bound[5]) ||
        !(h_max > 0.0) || h_obs < 0.0)
        return CHER_EINVAL;
    const Layered A = make_layered(atm);
    if (!(A.rho0 > 0.0)) return CHER_EINVAL;

    // fine eta table: h_k = k * dh
    T.n_fine = n_fine;
    T.h_max = h_max;
    T.dh = h_max / static_cast<double>(n_fine - 1);
    T.inv_dh = 1.0 / T.dh;
    T.eta.assign(n_fine, 0.0);
    for (int k = 0; k < n_fine; ++k) {
        const double h = static_cast<double>(k) * T.dh;
        T.eta[k] = eta_of(A, h);
    }

    // refraction tables
    T.H = H;
    T.Z = Z;
    T.theta_max = theta_max;
    T.dht = (h_max - h_obs) / static_cast<double>(H - 1);
    T.inv_dht = 1.0 / T.dht;
    const double smax = std::sin(theta_max);
    T.q_max = smax * smax;
    T.dq = T.q_max / static_cast<double>(Z - 1);
    T.inv_dq = 1.0 / T.dq;
    T.ax.assign(static_cast<size_t>(H) * Z, 0.0);
    T.al.assign(static_cast<size_t>(H) * Z, 0.0);
    const double eta_o = eta_of(A, h_obs);
    static const GaussLegendre gl;
    T.earth_radius = earth_radius;
    if (earth_radius > 0.0) {
        T.dsec = (1.0 / std::cos(theta_max) - 1.0) / static_cast<double>(Z - 1);
        T.inv_dsec = 1.0 / T.dsec;
        T.ag.assign(static_cast<size_t>(H) * Z, 0.0);
    }

    auto column_curved = [&](int k) {
        const double co = 1.0 / (1.0 + static_cast<double>(k) * T.dsec);
        const double so = std::sqrt((1.0 - co) * (1.0 + co));
        const double r_o = earth_radius + h_obs;
        CurvedIntegrand f{&A, earth_radius, r_o, eta_o, k == 0 ? 0.0 : so};
        double cp = 0.0, c1 = 0.0, c2 = 0.0;
        for (int j = 1; j < H; ++j) {
            const double lo = h_obs + static_cast<double>(j - 1) * T.dht;
            const double hi = h_obs + static_cast<double>(j) * T.dht;
            double ip, i1, i2;
            integrate_c(f, gl, lo, hi, ip, i1, i2);
            cp += ip;
            c1 += i1;
            c2 += i2;
            const double r_e = earth_radius + hi;
            const size_t a = static_cast<size_t>(j) * Z + k;
            if (k == 0) {
                // the limits at s_o = 0: G_phi / s_o, G_2 / s_o^2 -> u, G_1 -> 1
                T.ax[a] = cp * (r_e / r_o);
                T.al[a] = c1;
                T.ag[a] = c2 * (r_e / r_o);
            } else {
                double g_phi, g_1, g_2;
                curved_factors(r_o, r_e, so, co, g_phi, g_1, g_2);
                T.ax[a] = cp / g_phi;
                T.al[a] = c1 / g_1;
                T.ag[a] = c2 / g_2;
            }
        }
    };

    auto column = [&](int k) {
        if (earth_radius > 0.0) {
            column_curved(k);
            return;
        }
        const double q = static_cast<double>(k) * T.dq;
        const double so = std::sqrt(q);
        RayIntegrand f{&A, eta_o, so, std::sqrt((1.0 - so) * (1.0 + so))};
        double cx = 0.0, cl = 0.0;
        for (int j = 1; j < H; ++j) {
            const double lo = h_obs + static_cast<double>(j - 1) * T.dht;
            const double hi = h_obs + static_cast<double>(j) * T.dht;
            double ix, il;
            integrate(f, gl, lo, hi, ix, il);
            cx += ix;
            cl += il;
            T.ax[static_cast<size_t>(j) * Z + k] = cx;
            T.al[static_cast<size_t>(j) * Z + k] = cl;
        }
    };
    unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    nthr = std::min<unsigned>(nthr, static_cast<unsigned>(Z));
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nthr; ++t)
        pool.emplace_back([&, t] {
            for (int k = static_cast<int>(t); k < Z; k += static_cast<int>(nthr)) column(k);
        });
    for (auto &th : pool) th.join();
    return CHER_OK;
}

// ---------------------------------------------------------------------------
// Sensitivities for the adjoint (no counterpart in the paper).  eta depends
// on the atmosphere only through rho(h)/rho(0) = (b_i/c_i) e^{-h/c_i} /
// (b_0/c_0): d ln eta / d b_i = [layer(h) = i] / b_i - [layer(0) = i] / b_i,
// d ln eta / d c_i = [layer(h) = i] (h - c_i) / c_i^2 + [layer(0) = i] / c_i,
// and not on a_i at all.  Parameter index p: b_0..b_4 then c_0..c_4.
// ---------------------------------------------------------------------------
namespace {

void dlneta_dp(const Layered &A, double h, double *d /*[10]*/) {
    for (int q = 0; q < 10; ++q) d[q] = 0.0;
    if (h >= A.hb[5]) return;
    const int i = layer_of(A, h), i0 = layer_of(A, 0.0);
    d[i] += 1.0 / A.b[i];
    d[i0] -= 1.0 / A.b[i0];
    d[5 + i] += (h - A.c[i]) / (A.c[i] * A.c[i]);
    d[5 + i0] += 1.0 / A.c[i0];
}

// d(integrand)/d(eta at h) and d(integrand)/d(eta_o) of ax and al.
struct RaySensitivity {
    const Layered *A;
    double eta_o, so, co;
    void operator()(double h, double &gx_e, double &gx_o, double &gl_e, double &gl_o,
                    double &eta) const {
        eta = eta_of(*A, h);
        const double np1 = 1.0 + eta;
        const double rm1 = (eta_o - eta) / np1;
        const double r = 1.0 + rm1;
        const double s = so * r;
        const double c = std::sqrt((1.0 - s) * (1.0 + s));
        const double dc = -so * so * r / c;                 // dc/dr
        const double Aq = rm1 * (r + 1.0);                  // r^2 - 1
        const double co2 = co * co;
        const double E = (r * co + c) * c;
        const double dE = (co + dc) * c + (r * co + c) * dc;
        const double dgx = co2 * (2.0 * r * E - Aq * dE) / (E * E);
        const double F = (co + c) * c;
        const double dF = dc * (2.0 * c + co);
        const double dgl = -eta * co2 * co * dc / (c * c) + so * so * co2 * (2.0 * r * F - Aq * dF) / (F * F);
        const double dr_de = -r / np1, dr_do = 1.0 / np1;
        gx_e = dgx * dr_de;
        gx_o = dgx * dr_do;
        gl_e = co2 * co / c + dgl * dr_de;
        gl_o = dgl * dr_do;
    }
};

}  // namespace

void eta_sensitivity(const cher_atmosphere &atm, double h, double *d /*[10]*/) {
    const Layered A = make_layered(atm);
    dlneta_dp(A, h, d);
    const double e = eta_of(A, h);
    for (int q = 0; q < 10; ++q) d[q] *= e;
}

cher_status build_sensitivity(const cher_atmosphere &atm, double h_obs, const HostTables &T,
                              std::vector<double> &out) {
    const Layered A = make_layered(atm);
    const int H = T.H, Z = T.Z;
    out.assign(static_cast<size_t>(H) * Z * 20, 0.0);
    const double eta_o = eta_of(A, h_obs);
    double deo[10];
    dlneta_dp(A, h_obs, deo);
    for (int q = 0; q < 10; ++q) deo[q] *= eta_o;
    static const GaussLegendre gl;
    auto column = [&](int k) {
        const double q2 = static_cast<double>(k) * T.dq;
        const double so = std::sqrt(q2);
        RaySensitivity f{&A, eta_o, so, std::sqrt((1.0 - so) * (1.0 + so))};
        double acc[20] = {0};
        for (int j = 1; j < H; ++j) {
            const double lo = h_obs + static_cast<double>(j - 1) * T.dht;
            const double hi = h_obs + static_cast<double>(j) * T.dht;
            // pieces split at the layer boundaries, 12-point Gauss-Legendre
            double a = lo;
            for (int pi = 1; pi <= 6; ++pi) {
                double b = hi;
                if (pi <= 5) {
                    const double hb = A.hb[pi];
                    if (!(hb > a && hb < hi)) continue;
                    b = hb;
                }
                const double m = 0.5 * (a + b), hw = 0.5 * (b - a);
                for (int g = 0; g < GaussLegendre::N; ++g) {
                    const double h = m + hw * gl.x[g];
                    double gxe, gxo, gle, glo, eta;
                    f(h, gxe, gxo, gle, glo, eta);
                    double de[10];
                    dlneta_dp(A, h, de);
                    const double wgt = gl.w[g] * hw;
                    for (int q = 0; q < 10; ++q) {
                        const double dep = de[q] * eta;
                        acc[q] += wgt * (gxe * dep + gxo * deo[q]);
                        acc[10 + q] += wgt * (gle * dep + glo * deo[q]);
                    }
                }
                a = b;
                if (pi > 5) break;
            }
            double *dst = &out[(static_cast<size_t>(j) * Z + k) * 20];
            for (int q = 0; q < 20; ++q) dst[q] = acc[q];
        }
    };
    unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    nthr = std::min<unsigned>(nthr, static_cast<unsigned>(Z));
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nthr; ++t)
        pool.emplace_back([&, t] {
            for (int k = static_cast<int>(t); k < Z; k += static_cast<int>(nthr)) column(k);
        });
    for (auto &th : pool) th.join();
    return CHER_OK;
}

cher_status build_grid(const cher_telescope *tel, int32_t n_tel, double theta_max,
                       HostGrid &g) {
    // A line that crosses sphere k with zenith at most theta_max reaches h_obs
    // at a horizontal distance of at most |z| tan(theta_max) + r / cos(theta_max)
    // from the centre (the distance from the centre to the line is at least
    // cos(theta) times the horizontal distance in the plane of the centre); a
    // margin covers single-precision ground points.  Cells of half the largest
    // reach (fewer false candidates per cell than cells of the full reach, and
    // the grid still fits L1), or of the full reach where half would pass the
    // cell limit; a sphere is listed in every cell its reach disc touches.
    std::vector<double> reach(n_tel);
    double rmax = 0.0, xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int k = 0; k < n_tel; ++k) {
        const double mag = std::fabs(tel[k].x) + std::fabs(tel[k].y);
        reach[k] = std::fabs(tel[k].z) * std::tan(theta_max) + tel[k].r / std::cos(theta_max) +
                   0.5 + 1e-5 * mag;
        rmax = std::max(rmax, reach[k]);
        xmin = std::min(xmin, tel[k].x - reach[k]);
        xmax = std::max(xmax, tel[k].x + reach[k]);
        ymin = std::min(ymin, tel[k].y - reach[k]);
        ymax = std::max(ymax, tel[k].y + reach[k]);
    }
    double cs = rmax * 0.5;
    bool widened = false;
    for (int attempt = 0; attempt < 24; ++attempt) {
        const double ex = xmax - xmin, ey = ymax - ymin;
        const double nxd = std::ceil(ex / cs), nyd = std::ceil(ey / cs);
        if (nxd * nyd > double(1 << 22)) {
            // too many cells of half the reach for this extent: cells of the
            // full reach, once (the same limit then applies as to them)
            if (!widened && cs < rmax) {
                cs = rmax;
                widened = true;
                continue;
            }
            return CHER_ERANGE;
        }
        g.nx = std::max(1, static_cast<int>(nxd));
        g.ny = std::max(1, static_cast<int>(nyd));
        g.x0 = xmin;
        g.y0 = ymin;
        g.cs = cs;
        g.inv_cs = 1.0 / cs;
        const size_t nc = static_cast<size_t>(g.nx) * g.ny;
        std::vector<std::vector<int32_t>> cells(nc);
        for (int k = 0; k < n_tel; ++k) {
            const int cx0 = std::max(0, static_cast<int>(std::floor((tel[k].x - reach[k] - g.x0) * g.inv_cs)));
            const int cx1 = std::min(g.nx - 1, static_cast<int>(std::floor((tel[k].x + reach[k] - g.x0) * g.inv_cs)));
            const int cy0 = std::max(0, static_cast<int>(std::floor((tel[k].y - reach[k] - g.y0) * g.inv_cs)));
            const int cy1 = std::min(g.ny - 1, static_cast<int>(std::floor((tel[k].y + reach[k] - g.y0) * g.inv_cs)));
            for (int cy = cy0; cy <= cy1; ++cy)
                for (int cx = cx0; cx <= cx1; ++cx) {
                    // distance from the centre to the cell rectangle
                    const double rx0 = g.x0 + cx * cs, rx1 = rx0 + cs;
                    const double ry0 = g.y0 + cy * cs, ry1 = ry0 + cs;
                    const double dx = std::max({rx0 - tel[k].x, 0.0, tel[k].x - rx1});
                    const double dy = std::max({ry0 - tel[k].y, 0.0, tel[k].y - ry1});
                    if (dx * dx + dy * dy <= reach[k] * reach[k])
                        cells[static_cast<size_t>(cy) * g.nx + cx].push_back(k);
                }
        }
        size_t worst = 0;
        for (auto &c : cells) worst = std::max(worst, c.size());
        if (worst <= static_cast<size_t>(kMaxCandPerCell)) {
            g.cell_start.assign(nc + 1, 0);
            g.cell_tel.clear();
            for (size_t c = 0; c < nc; ++c) {
                g.cell_start[c] = static_cast<int32_t>(g.cell_tel.size());
                g.cell_tel.insert(g.cell_tel.end(), cells[c].begin(), cells[c].end());
            }
            g.cell_start[nc] = static_cast<int32_t>(g.cell_tel.size());
            if (g.cell_tel.empty()) g.cell_tel.push_back(0);
            return CHER_OK;
        }
        cs *= 0.5;   // too many spheres share a cell: refine
        if (cs < 1e-3) break;
    }
    return CHER_ERANGE;
}

// Greisen profile of a shower of y = ln(E0 / E_c), up to a constant factor,
// and its CDF on n_cdf uniform nodes of [0, t_g], normalised to 1 (the
// device step generator inverts it); Gauss-Legendre on each node interval.
namespace {
double greisen(double t, double y) {
    if (t <= 0.0) return 1.0;
    const double s = 3.0 * t / (t + 2.0 * y);
    return std::exp(t * (1.0 - 1.5 * std::log(s)));
}
}  // namespace

void gauss_legendre12(double *x, double *w) {
    static const GaussLegendre gl;
    static_assert(GaussLegendre::N == 12, "the fallback integrator takes 12 nodes");
    for (int q = 0; q < GaussLegendre::N; ++q) {
        x[q] = gl.x[q];
        w[q] = gl.w[q];
    }
}

void greisen_cdf_host(double y, double t_g, int n_cdf, std::vector<double> &cdf) {
    static const GaussLegendre gl;
    cdf.assign(n_cdf, 0.0);
    const double dt = t_g / (n_cdf - 1);
    for (int k = 1; k < n_cdf; ++k) {
        const double half = 0.5 * dt, mid = (k - 1) * dt + half;
        double sum = 0.0;
        for (int q = 0; q < GaussLegendre::N; ++q) sum += gl.w[q] * greisen(mid + half * gl.x[q], y);
        cdf[k] = cdf[k - 1] + half * sum;
    }
    const double tot = cdf[n_cdf - 1];
    for (double &v : cdf) v /= tot;
}

}  // namespace cher
