// cher_internal.h -- private structures shared by the library's translation
// units (host table builder, C ABI, CUDA kernels).  Not installed, not part
// of the ABI.
#pragma once

#include <cuda_runtime_api.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/cher.h"

namespace cher {

// Physical constants (CODATA 2018; c exact by the SI definition).
constexpr double kC = 0.299792458;          // m/ns
constexpr double kMe = 0.51099895000;       // electron mass, MeV
constexpr double kAlpha = 7.2973525693e-3;  // fine-structure constant
constexpr double kPi = 3.14159265358979323846;

// Bunch status codes (the rare branches of the paper's Algorithm 1).
enum : int32_t {
    ST_GROUND = 0, ST_UPWARD = 1, ST_BELOW = 2, ST_ABOVE = 3, ST_ANGLE = 4, ST_ABSORBED = 5,
    ST_DEFER = 6    // internal: past the tables' zenith range, queued for the fallback pass
};

constexpr int kMaxCandPerCell = 32;   // telescope candidates in one grid cell
constexpr int kDispMax = 9;           // nodes of a wavelength-dependent index

// Host-side tables, all FP64 (step a0).
struct HostTables {
    int32_t n_fine = 0;
    double h_max = 0, dh = 0, inv_dh = 0;
    std::vector<double> eta;             // [n_fine]
    int32_t H = 0, Z = 0;
    double theta_max = 0, dht = 0, inv_dht = 0, q_max = 0, dq = 0, inv_dq = 0;
    std::vector<double> ax, al;          // [H][Z]
    // curved atmosphere (earth_radius > 0): zenith nodes uniform in sec,
    // sec_k = 1 + k dsec, and a third table (the geometric part of the
    // optical-path correction); ax, al, ag normalised by the path averages
    // of their first-order factors along the straight reference line
    double earth_radius = 0, dsec = 0, inv_dsec = 0;
    std::vector<double> ag;              // [H][Z]
};

// Ground grid of telescope candidates (step a4).
struct HostGrid {
    double x0 = 0, y0 = 0, cs = 1, inv_cs = 1;
    int32_t nx = 1, ny = 1;
    std::vector<int32_t> cell_start;     // [nx * ny + 1]
    std::vector<int32_t> cell_tel;       // candidates
};

// Build eta, ax, al (table definitions in cher_tables.cpp).
cher_status build_tables(const cher_atmosphere &atm, double h_obs, int32_t n_fine,
                         int32_t H, int32_t Z, double theta_max, double h_max,
                         HostTables &out, double earth_radius = 0.0);
// Eta lookup in the fine table, one IEEE operation per statement (the same
// rounding as the device lookup that decides the bunch count).
double eta_lookup(const HostTables &t, double h);
cher_status build_grid(const cher_telescope *tel, int32_t n_tel, double theta_max,
                       HostGrid &g);
// Adjoint support: d eta(h) / d p and the refraction-table sensitivities
// [H][Z][20] = {d ax / d p (10), d al / d p (10)}, p = b_0..b_4, c_0..c_4.
void eta_sensitivity(const cher_atmosphere &atm, double h, double *d);
cher_status build_sensitivity(const cher_atmosphere &atm, double h_obs, const HostTables &T,
                              std::vector<double> &out);

// Everything a kernel launch needs, passed by value.
struct KParams {
    // tracks
    const double *x0, *y0, *z0, *t0, *len, *ekin;
    const void *ux, *uy, *uz;
    const uint32_t *shower;
    const double *t_ref;
    int32_t n_showers;
    int64_t n, track_base;
    uint32_t key0, key1;
    // Philox round keys, rk0[r] = key0 + r W0 and rk1[r] = key1 + r W1: uniform
    // over the launch, so the bunch loop (philox_bunch) reads them from the
    // parameter bank instead of advancing the key every round
    uint32_t rk0[10], rk1[10];
    // yield constants (FP64, same rounding as the host)
    double inv_me, K, inv_B;
    // fine eta table
    int32_t n_fine;
    double h_max, inv_dh;
    const double *eta64;
    const float *eta32;
    double eta_slope;                     // max |eta[k+1] - eta[k]| / dh
    double eta_jump;                      // 1.5 x max |eta[k+1] - eta[k]| / eta[k] over
                                          // the cells that hold no layer boundary
    // observation level
    double h_obs, eta_obs;
    // refraction tables, pair-interleaved: entry (j, k), k < Z-1, holds
    // {ax[j][k], al[j][k], ax[j][k+1], al[j][k+1]}
    int32_t H, Z;
    double inv_dht, inv_dq, q_max;
    // flat layers: one (ax, al) pair per node [H][Z] (double2 or float2);
    // curved atmosphere: entry (j, k < Z-1) = {ax_k, al_k, ax_k+1, al_k+1},
    // {ag_k, ag_k+1, 0, 0} (double, or rounded to float)
    const void *tab;
    // wavelength band in 1/nm
    double lam_inv1, lam_dinv;
    // telescopes and two ground grids of candidate spheres: grid 0 serves
    // photons arriving with sin^2(zenith) <= q_band (small reach), grid 1
    // the rest (reach of the largest zenith)
    int32_t n_tel;
    const void *tel;                      // float4 / double4: x, y, z, r^2
    struct Grid {
        int32_t nx, ny, n_cand;
        double x0, y0, inv_cs;
        const int32_t *cell_start;        // [nx * ny + 1]
        const int32_t *cand_tel;          // telescope of each entry
        const void *cand32;               // float4 per entry: x, y, z, r^2
        const void *cand64;               // double4 per entry
    } grid[2];
    double q_band;
    // outputs
    void *pos, *tim;
    uint64_t *key;
    int64_t cap;
    unsigned long long *count, *stats;
    // trace mode
    const int64_t *bunch_off;
    int32_t *t_status, *t_nhit, *t_first;
    int64_t t_nbunch;                     // entries of the trace arrays
    // yield-only mode
    int32_t *y_nb;
    double *y_w;
    // scheduling
    unsigned long long *tile_counter;     // NULL: one CTA per tile
    int64_t n_tiles;
    // adjoint screening: frozen bunch counts, list of (step, bunch) pairs
    // that land within the read-out radius of a telescope centre
    const int32_t *nb_frozen;
    uint64_t *list;
    unsigned long long *list_count;
    int64_t list_cap;
    double rcut2;
    // longitudinal production profile: rows of n_bins per shower (NULL:
    // off); the layered thickness T(h) = a + b exp(-h / c) per layer, with
    // the thickness at each layer's top from its own formula (the inverse
    // picks the layer by it)
    double *prof;
    const double *prof_cos;
    int32_t prof_bins, prof_rows;
    double prof_dx, prof_inv_dx;
    struct Layers {
        double hb[6], a[5], b[5], c[5], inv_c[5], t_top[5];
        double eta_coef[5];      // n - 1 = eta_coef * exp(-h / c) in each layer
    } atm;
    // beyond-table fallback (fb_q = 0: off): bunches with the tables'
    // q_max < sin^2(zenith) <= fb_q are queued (fb_list, FbEntry records,
    // fb_count appended atomically, fb_cap entries) and propagated by the
    // ray integrals (12-point Gauss-Legendre per layer) in a second pass
    double fb_q;
    void *fb_list;
    unsigned long long *fb_count;
    int64_t fb_cap;
    double gl_x[12], gl_w[12];
    // atmospheric transmission (NULL: off): vertical optical depth on a
    // uniform (lambda, h) grid, [nl][nh], float (FP32) or double (FP64);
    // index = (value - first node) * scale
    const void *trans;
    int32_t trans_nl, trans_nh;
    double trans_l0, trans_lscale, trans_h0, trans_hscale;
    // wavelength-dependent index (disp_k = 0: off): n - 1 = eta(h) kappa,
    // kappa at disp_k nodes uniform in 1/lambda from 1/lambda_min (node 0),
    // linear between them; the yield's band factor per piece disp_Kd =
    // 2 pi alpha du (du in 1/m); tabd: the refraction tables of kappa at the
    // band's two ends, entry (j, k) = {entry of kap_lo, entry of kap_hi} in
    // the pair-interleaved layout of tab; weight (kappa - kap_lo) kap_winv
    int32_t disp_k;
    double kap[kDispMax];
    const double *kap64;
    const float *kap32;
    double disp_Kd, disp_u1, disp_du, kap_lo, kap_winv;
    const void *tabd;
    // curved atmosphere (earth_radius = 0: flat layers): r_o = R_E + h_obs;
    // the tables' zenith axis is uniform in sec (inv_dsec) and an entry holds
    // two more values (the geometric part of the optical path): entry (j, k)
    // = {ax_k, al_k, ax_k+1, al_k+1}, {ag_k, ag_k+1, 0, 0} (and with kappa,
    // that pair for kap_lo then for kap_hi)
    double earth_radius, r_o, inv_ro, inv_dsec;
    // the per-launch constants of the bunch loop, rounded to float on the
    // host: the FP32 path converts nothing from double on the device
    struct {
        float h_obs, dH_max, eta_o, inv_np1o, np1o, q_max, inv_dht, inv_dq, inv_dh;
        float lam_inv1, lam_dinv, rcut2, q_band;
        // FP32 screen of the yield: constants and the table's largest slope
        float inv_me, K, inv_B, h_max, dh, eta_slope, eta_jump;
        float gx0[2], gy0[2], inv_gcs[2];
        float prof_dx, prof_inv_dx;
        float trans_l0, trans_lscale, trans_h0, trans_hscale;
        float fb_q;
        float hb[6], a[5], b[5], c[5], inv_c[5], t_top[5];
        float kap[kDispMax], disp_Kd, disp_u1, disp_du, kap_lo, kap_winv;
        float eta_coef[5], gl_x[12], gl_w[12];
        float earth_radius, r_o, inv_ro, inv_dsec;
    } f;
};

// Adjoint pass over the listed bunches (cher_adjoint.cu).
struct AdjParams {
    KParams k;
    const uint64_t *list;
    int64_t n_list;
    const int32_t *nb;
    double sigma, inv_2s2, norm, rcut2;
    double *S, *U;                 // [n_tel] read-out sums
    const double *gD, *gT;         // [n_tel] upstream gradients
    double *grad_atm;              // [15]: a_0..a_4, b_0..b_4, c_0..c_4
    double *grad_tracks;           // [6][n]: x0, y0, z0, ux, uy, uz
    const double *sens;            // [H][Z][20] table sensitivities
    double hb[6], b[5], c[5];
    int layer0;                    // layer of h = 0 (rho(0))
    double dh_fine;
    int ko;                        // fine-table position of h_obs
    double fo;
};
cudaError_t adjoint_pairs(bool fp32, int mode, const AdjParams &A, void *stream);

// Fill KParams::f from the double fields.
void fill_float_constants(KParams &p);

enum Mode : int { MODE_HITS = 0, MODE_TRACE = 1, MODE_YIELD = 2, MODE_SCREEN = 3 };
// added to a Mode when the launch applies the transmission draw, and when
// it queues (hits) or integrates in place (trace) the bunches past the
// tables' zenith range
constexpr int kTransBit = 4;
constexpr int kFbBit = 8;
// and when the index depends on the wavelength, and in a curved atmosphere
// (both instantiated for 128-step tiles and the hits, trace and yield modes
// only; the curved atmosphere without the beyond-table fallback)
constexpr int kDispBit = 16;
constexpr int kCurvBit = 32;
// The plain FP32 hits kernel also comes in builds for more resident CTAs per
// SM (128 threads each, fewer registers per thread): 9 or 10; the launch
// shape's CTAs per SM picks one (kOccShift: 2 bits of the mode word).
constexpr int kOccShift = 6;
constexpr int kOccMask = 3 << kOccShift;
inline int occupancy_bits(bool fp32, int block, int ctas_per_sm) {
    if (!fp32 || block != 128 || ctas_per_sm <= 8) return 0;
    return (ctas_per_sm <= 9 ? 1 : 2) << kOccShift;
}
constexpr int kDispBlock = 128;
inline int kernel_mode(int mode, const KParams &p) {
    int m = mode;
    if (p.trans && mode != MODE_YIELD) m |= kTransBit;
    if (p.fb_q > 0.0 && (mode == MODE_HITS || mode == MODE_TRACE)) m |= kFbBit;
    if (p.disp_k > 0) m |= kDispBit;
    if (p.earth_radius > 0.0) m |= kCurvBit;
    return m;
}
// The fallback pass over the queued bunches (after a MODE_HITS launch with
// fb_q > 0, on the same stream; reads the queue's count on the device).
cudaError_t launch_fallback(bool fp32, bool tr, bool disp, const KParams &p, int num_sms,
                            void *stream);
// Bytes of one fallback queue record.
size_t fallback_record_bytes(bool fp32);
// The 12-point Gauss-Legendre rule on [-1, 1] (host).
void gauss_legendre12(double *x, double *w);

// Launchers (cher_kernels.cu).  fp32 selects CHER_FP32_BULK.
size_t kernel_smem_bytes(bool fp32, int block, const KParams &p);
// Device step generator (cher_generator.cu): per-shower constants in float.
struct GenShower {
    float ax, ay, az;            // axis (downward)
    float b1x, b1y, b1z, b2x, b2y, b2z;   // transverse basis
    float cz, x0cz;              // cos zenith, X0 cos zenith (g/cm^2)
    float core_x, core_y, s_ref, dt;      // s_ref: m; dt: CDF node spacing
};
struct GenParams {
    const GenShower *showers;
    const int64_t *first;        // [n_showers + 1] first global step of each shower
    int32_t n_showers, n_cdf;
    const float *cdf;            // [n_showers][n_cdf]
    uint32_t key0, key1;
    float h_obs;
    int64_t n;
    double *x0, *y0, *z0, *t0, *len, *ekin;
    void *ux, *uy, *uz;
    bool dirs_fp32;
    uint32_t *shower;
};
cudaError_t generate_steps(const GenParams &g, int num_sms, void *stream);
// The Greisen profile's CDF on n_cdf uniform nodes of [0, t_g] (host, FP64).
void greisen_cdf_host(double y, double t_g, int n_cdf, std::vector<double> &cdf);

// The records of every telescope packed contiguously (cher_pack.cu).
cudaError_t pack_records(bool fp32, const void *pos, const void *tim, const uint64_t *key,
                         const unsigned long long *count, int64_t cap, int n_tel, int64_t max_rec,
                         void *dpos, void *dtim, uint64_t *dkey, int64_t *off, int num_sms,
                         void *stream);

// The FP32 path's double -> float rounding over an array (grid-stride).
cudaError_t round_to_float(const double *in, float *out, float *lo, int64_t n, int num_sms,
                           void *stream);
cudaError_t kernel_prepare(bool fp32, int block, int mode, size_t smem);
cudaError_t kernel_launch(bool fp32, int block, int mode, int grid, size_t smem,
                          const KParams &p, void *stream);
int kernel_max_ctas_per_sm(bool fp32, int block, int mode, size_t smem);

}  // namespace cher
