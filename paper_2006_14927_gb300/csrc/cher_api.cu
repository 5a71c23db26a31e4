// cher_api.cu -- the C ABI declared in include/cher.h: context lifetime,
// argument checks, table upload, launch configuration and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "cher_internal.h"

struct cher_ctx {
    int device = 0;
    int num_sms = 0;
    cher_atmosphere atm{};
    double h_obs = 0;
    std::vector<cher_telescope> tel;
    cher_options opt{};
    // constants of the yield, computed once in double (same rounding as the
    // per-step statements of the kernel)
    double inv_me = 0, K = 0, inv_B = 0, lam_inv1 = 0, lam_dinv = 0;
    // tables
    bool built = false;
    cher::HostTables T;
    cher::HostGrid G[2];                  // zenith bands: steep, all
    double q_band = 0;
    double eta_obs = 0;
    double eta_slope = 0;                 // max |eta[k+1] - eta[k]| / dh
    double eta_jump = 0;                  // see KParams::eta_jump
    double *d_eta64 = nullptr;
    float *d_eta32 = nullptr;
    void *d_tab64 = nullptr, *d_tab32 = nullptr;
    void *d_tel64 = nullptr, *d_tel32 = nullptr;
    int32_t *d_cell_start[2] = {nullptr, nullptr}, *d_cell_tel[2] = {nullptr, nullptr};
    float *d_cand32[2] = {nullptr, nullptr};
    double *d_cand64[2] = {nullptr, nullptr};
    // scratch: the persistent kernel's tile counter
    unsigned long long *d_scratch = nullptr;
    // launch shape
    int block = 128;                      // the autotuner's choice on GB300 for the
    int ctas_per_sm = 8;                  // FP32 path (32 resident warps per SM)
    // table sizes of the last build (cher_set_atmosphere rebuilds with them)
    int32_t tab_H = 0, tab_Z = 0;
    double tab_zen = 0, tab_hmax = 0;
    // adjoint: sensitivity tables and scratch, allocated on first use
    double *d_sens = nullptr;
    int32_t *d_nb = nullptr;
    double *d_w = nullptr;
    int64_t nb_cap = 0;
    uint64_t *d_list = nullptr;
    int64_t list_cap = 0;
    unsigned long long *d_list_count = nullptr;
    double *d_SU = nullptr;
    // atmospheric transmission table (both precisions), NULL when off
    double *d_trans64 = nullptr;
    float *d_trans32 = nullptr;
    int32_t trans_nl = 0, trans_nh = 0;
    double trans_l0 = 0, trans_l1 = 0, trans_h0 = 0, trans_h1 = 0;
    // beyond-table fallback: zenith limit (deg, 0 off) and its queue
    double fb_deg = 0.0;
    int64_t fb_records = 0;               // queue size per call (0: the default)
    void *d_fb = nullptr;
    int64_t fb_cap = 0;                   // bytes
    unsigned long long *d_fb_count = nullptr;
    // step generator: per-call shower constants, offsets and CDF tables;
    // host CDF rows cached by (E0, zenith) (cleared past 4096 entries)
    unsigned char *d_gen = nullptr;
    int64_t gen_cap = 0;
    std::map<std::pair<double, double>, std::vector<float>> cdf_cache;
    // pinned staging of those tables (the upload is asynchronous; the event
    // marks when the last upload has read the staging, before it is reused)
    unsigned char *h_gen = nullptr;
    int64_t h_gen_cap = 0;
    cudaEvent_t gen_ev = nullptr;
    bool gen_ev_pending = false;
    // wavelength-dependent index: kappa at the nodes (disp_k = 0: off), its
    // device copies, and the refraction tables of the band's two ends in
    // the pair-interleaved layout, {kappa_lo entry, kappa_hi entry}
    int32_t disp_k = 0;
    double kap[cher::kDispMax] = {};
    // curved atmosphere: the Earth's radius (0: flat layers)
    double earth_radius = 0.0;
    double *d_kap64 = nullptr;
    float *d_kap32 = nullptr;
    void *d_tabd64 = nullptr, *d_tabd32 = nullptr;
};

namespace {

bool bad_ptr(const void *p) { return p == nullptr; }

void free_tables(cher_ctx *c) {
    cudaFree(c->d_eta64);
    cudaFree(c->d_eta32);
    cudaFree(c->d_tab64);
    cudaFree(c->d_tab32);
    cudaFree(c->d_tel64);
    cudaFree(c->d_tel32);
    for (int g = 0; g < 2; ++g) {
        cudaFree(c->d_cell_start[g]);
        cudaFree(c->d_cell_tel[g]);
        cudaFree(c->d_cand32[g]);
        cudaFree(c->d_cand64[g]);
        c->d_cell_start[g] = c->d_cell_tel[g] = nullptr;
        c->d_cand32[g] = nullptr;
        c->d_cand64[g] = nullptr;
    }
    c->d_eta64 = nullptr;
    c->d_eta32 = nullptr;
    c->d_tab64 = c->d_tab32 = nullptr;
    c->d_tel64 = c->d_tel32 = nullptr;
    cudaFree(c->d_sens);
    c->d_sens = nullptr;
    c->built = false;
}

void free_dispersion_tables(cher_ctx *c) {
    cudaFree(c->d_kap64);
    cudaFree(c->d_kap32);
    cudaFree(c->d_tabd64);
    cudaFree(c->d_tabd32);
    c->d_kap64 = nullptr;
    c->d_kap32 = nullptr;
    c->d_tabd64 = c->d_tabd32 = nullptr;
}

void free_adjoint_scratch(cher_ctx *c) {
    cudaFree(c->d_nb);
    cudaFree(c->d_w);
    cudaFree(c->d_list);
    cudaFree(c->d_list_count);
    cudaFree(c->d_SU);
    c->d_nb = nullptr;
    c->d_w = nullptr;
    c->d_list = nullptr;
    c->d_list_count = nullptr;
    c->d_SU = nullptr;
    c->nb_cap = c->list_cap = 0;
}

template <class T>
cher_status upload(T **dst, const T *src, size_t n) {
    if (cudaMalloc(reinterpret_cast<void **>(dst), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ENOMEM;
    }
    if (cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
        return CHER_ECUDA;
    return CHER_OK;
}

template <class T>
cher_status grow(T **ptr, int64_t &cap, int64_t need) {
    if (need <= cap && *ptr) return CHER_OK;
    cudaFree(*ptr);
    *ptr = nullptr;
    cap = 0;
    if (cudaMalloc(reinterpret_cast<void **>(ptr), std::max<int64_t>(need, 1) * sizeof(T)) !=
        cudaSuccess) {
        cudaGetLastError();
        return CHER_ENOMEM;
    }
    cap = need;
    return CHER_OK;
}

// device copies of grid g: cell starts, candidate telescopes and their
// centres and squared radii in both precisions
cher_status upload_grid(cher_ctx *c, int g) {
    const cher::HostGrid &G = c->G[g];
    std::vector<float> c32(G.cell_tel.size() * 4);
    std::vector<double> c64(G.cell_tel.size() * 4);
    for (size_t m = 0; m < G.cell_tel.size(); ++m) {
        const cher_telescope &q = c->tel[G.cell_tel[m]];
        const double v[4] = {q.x, q.y, q.z, q.r * q.r};
        for (int e = 0; e < 4; ++e) {
            c64[4 * m + e] = v[e];
            c32[4 * m + e] = static_cast<float>(v[e]);
        }
    }
    cher_status r;
    if ((r = upload(&c->d_cell_start[g], G.cell_start.data(), G.cell_start.size())) != CHER_OK ||
        (r = upload(&c->d_cell_tel[g], G.cell_tel.data(), G.cell_tel.size())) != CHER_OK ||
        (r = upload(&c->d_cand32[g], c32.data(), c32.size())) != CHER_OK ||
        (r = upload(&c->d_cand64[g], c64.data(), c64.size())) != CHER_OK)
        return r;
    return CHER_OK;
}

// Pair-interleaved entries (the dispersion tables, and the main tables in a
// curved atmosphere): per entry (j, k < Z-1) the pair {ax_k, al_k, ax_k+1,
// al_k+1} and, in a curved atmosphere, {ag_k, ag_k+1, 0, 0}.
size_t entry_values(const cher::HostTables &T) { return T.earth_radius > 0.0 ? 8 : 4; }

void pack_entry(const cher::HostTables &T, int j, int k, double *out) {
    const size_t a = static_cast<size_t>(j) * T.Z + k;
    out[0] = T.ax[a];
    out[1] = T.al[a];
    out[2] = T.ax[a + 1];
    out[3] = T.al[a + 1];
    if (T.earth_radius > 0.0) {
        out[4] = T.ag[a];
        out[5] = T.ag[a + 1];
        out[6] = out[7] = 0.0;
    }
}

// The refraction tables of kappa[k-1] (lo) and kappa[0] (hi): the context's
// table shape with n - 1 scaled by kappa, interleaved per entry.
cher_status build_dispersion_tables(cher_ctx *c) {
    free_dispersion_tables(c);
    if (c->disp_k == 0) return CHER_OK;
    const double th = c->tab_zen * cher::kPi / 180.0;
    cher::HostTables T[2];
    for (int s = 0; s < 2; ++s) {
        cher_atmosphere a = c->atm;
        a.n0_minus_1 *= s == 0 ? c->kap[c->disp_k - 1] : c->kap[0];
        const cher_status r = cher::build_tables(a, c->h_obs, 2, c->tab_H, c->tab_Z, th,
                                                 c->tab_hmax, T[s], c->earth_radius);
        if (r != CHER_OK) return r;
    }
    const int H = T[0].H, Z = T[0].Z;
    const size_t per = entry_values(T[0]);
    std::vector<double> t64(static_cast<size_t>(H) * (Z - 1) * 2 * per);
    std::vector<float> t32(t64.size());
    for (int j = 0; j < H; ++j)
        for (int k = 0; k < Z - 1; ++k) {
            const size_t e = (static_cast<size_t>(j) * (Z - 1) + k) * 2 * per;
            for (int s = 0; s < 2; ++s) pack_entry(T[s], j, k, &t64[e + per * s]);
            for (size_t q = 0; q < 2 * per; ++q) t32[e + q] = static_cast<float>(t64[e + q]);
        }
    float k32[cher::kDispMax];
    for (int m = 0; m < cher::kDispMax; ++m) k32[m] = static_cast<float>(c->kap[m]);
    double *d64 = nullptr;
    float *d32 = nullptr;
    cher_status r;
    if ((r = upload(&c->d_kap64, c->kap, cher::kDispMax)) != CHER_OK ||
        (r = upload(&c->d_kap32, k32, cher::kDispMax)) != CHER_OK ||
        (r = upload(&d64, t64.data(), t64.size())) != CHER_OK ||
        (r = upload(&d32, t32.data(), t32.size())) != CHER_OK) {
        cudaFree(d64);
        cudaFree(d32);
        free_dispersion_tables(c);
        return r;
    }
    c->d_tabd64 = d64;
    c->d_tabd32 = d32;
    return CHER_OK;
}

bool tracks_ok(const cher_tracks *t) {
    if (!t) return false;
    if (t->n < 0 || t->n > (int64_t(1) << 40)) return false;
    if (t->track_base < 0 || t->track_base > (int64_t(1) << 40)) return false;
    if (t->n == 0) return true;
    if (bad_ptr(t->x0) || bad_ptr(t->y0) || bad_ptr(t->z0) || bad_ptr(t->t0) ||
        bad_ptr(t->len) || bad_ptr(t->ekin) || bad_ptr(t->ux) || bad_ptr(t->uy) ||
        bad_ptr(t->uz))
        return false;
    if (t->t_ref && t->n_showers < 1) return false;
    return true;
}

cher::KParams base_params(const cher_ctx *c, const cher_tracks *t, uint64_t seed, bool fp32) {
    cher::KParams p;
    std::memset(&p, 0, sizeof(p));
    p.x0 = t->x0; p.y0 = t->y0; p.z0 = t->z0; p.t0 = t->t0; p.len = t->len; p.ekin = t->ekin;
    p.ux = t->ux; p.uy = t->uy; p.uz = t->uz;
    p.shower = t->shower;
    p.t_ref = t->t_ref;
    p.n_showers = t->n_showers;
    p.n = t->n;
    p.track_base = t->track_base;
    p.key0 = static_cast<uint32_t>(seed & 0xffffffffu);
    p.key1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.rk0[r] = p.key0 + static_cast<uint32_t>(r) * 0x9E3779B9u;
        p.rk1[r] = p.key1 + static_cast<uint32_t>(r) * 0xBB67AE85u;
    }
    p.inv_me = c->inv_me;
    p.K = c->K;
    p.inv_B = c->inv_B;
    p.n_fine = c->T.n_fine;
    p.h_max = c->T.h_max;
    p.inv_dh = c->T.inv_dh;
    p.eta64 = c->d_eta64;
    p.eta32 = c->d_eta32;
    p.eta_slope = c->eta_slope;
    p.eta_jump = c->eta_jump;
    p.h_obs = c->h_obs;
    p.eta_obs = c->eta_obs;
    p.H = c->T.H;
    p.Z = c->T.Z;
    p.inv_dht = c->T.inv_dht;
    p.inv_dq = c->T.inv_dq;
    p.q_max = c->T.q_max;
    p.tab = fp32 ? c->d_tab32 : c->d_tab64;
    p.lam_inv1 = c->lam_inv1;
    p.lam_dinv = c->lam_dinv;
    p.n_tel = static_cast<int32_t>(c->tel.size());
    p.tel = fp32 ? c->d_tel32 : c->d_tel64;
    for (int g = 0; g < 2; ++g) {
        p.grid[g].nx = c->G[g].nx;
        p.grid[g].ny = c->G[g].ny;
        p.grid[g].n_cand = static_cast<int32_t>(c->G[g].cell_tel.size());
        p.grid[g].x0 = c->G[g].x0;
        p.grid[g].y0 = c->G[g].y0;
        p.grid[g].inv_cs = c->G[g].inv_cs;
        p.grid[g].cell_start = c->d_cell_start[g];
        p.grid[g].cand_tel = c->d_cell_tel[g];
        p.grid[g].cand32 = c->d_cand32[g];
        p.grid[g].cand64 = c->d_cand64[g];
    }
    p.q_band = c->q_band;
    // the layered thickness, for the production profile
    for (int l = 0; l < 6; ++l) p.atm.hb[l] = c->atm.h_bound[l];
    for (int l = 0; l < 5; ++l) {
        p.atm.a[l] = c->atm.a[l];
        p.atm.b[l] = c->atm.b[l];
        p.atm.c[l] = c->atm.c[l];
        p.atm.inv_c[l] = 1.0 / c->atm.c[l];
        p.atm.t_top[l] = c->atm.a[l] + c->atm.b[l] * std::exp(-(c->atm.h_bound[l + 1] / c->atm.c[l]));
        // n - 1 = (n0 - 1) rho(h) / rho(0), rho = (b / c) exp(-h / c) in the layer
        p.atm.eta_coef[l] = c->atm.n0_minus_1 * (c->atm.b[l] / c->atm.c[l]) /
                            (c->atm.b[0] / c->atm.c[0]);
    }
    cher::gauss_legendre12(p.gl_x, p.gl_w);
    if (c->earth_radius > 0.0) {
        p.earth_radius = c->earth_radius;
        p.r_o = c->earth_radius + c->h_obs;
        p.inv_ro = 1.0 / p.r_o;
        p.inv_dsec = c->T.inv_dsec;
    }
    if (c->fb_deg > c->tab_zen && c->built && c->earth_radius == 0.0) {
        const double sf = std::sin(c->fb_deg * 3.14159265358979323846 / 180.0);
        p.fb_q = sf * sf;
    }
    if (c->disp_k > 0) {
        p.disp_k = c->disp_k;
        for (int m = 0; m < cher::kDispMax; ++m) p.kap[m] = c->kap[m];
        p.kap64 = c->d_kap64;
        p.kap32 = c->d_kap32;
        // 2 pi alpha du, du = (1/lambda_min - 1/lambda_max) / (k - 1) in 1/m
        const double two_pi_alpha = (2.0 * cher::kPi) * cher::kAlpha;
        const double inv1 = 1.0e9 / c->opt.lambda_min_nm;
        const double inv2 = 1.0e9 / c->opt.lambda_max_nm;
        const double dinv = inv1 - inv2;
        const double du = dinv / static_cast<double>(c->disp_k - 1);
        p.disp_Kd = two_pi_alpha * du;
        p.disp_u1 = 1.0 / c->opt.lambda_min_nm;
        p.disp_du = (1.0 / c->opt.lambda_min_nm - 1.0 / c->opt.lambda_max_nm) /
                    static_cast<double>(c->disp_k - 1);
        p.kap_lo = c->kap[c->disp_k - 1];
        p.kap_winv = c->kap[0] > p.kap_lo ? 1.0 / (c->kap[0] - p.kap_lo) : 0.0;
        p.tabd = fp32 ? c->d_tabd32 : c->d_tabd64;
    }
    if (c->d_trans64) {
        p.trans = fp32 ? static_cast<const void *>(c->d_trans32) : c->d_trans64;
        p.trans_nl = c->trans_nl;
        p.trans_nh = c->trans_nh;
        p.trans_l0 = c->trans_l0;
        p.trans_lscale = (c->trans_nl - 1) / (c->trans_l1 - c->trans_l0);
        p.trans_h0 = c->trans_h0;
        p.trans_hscale = (c->trans_nh - 1) / (c->trans_h1 - c->trans_h0);
    }
    cher::fill_float_constants(p);
    return p;
}

cher_status launch(cher_ctx *c, cher::KParams &p, bool fp32, int mode, bool persistent,
                   void *stream) {
    const int block = (p.disp_k > 0 || p.earth_radius > 0.0) ? cher::kDispBlock : c->block;
    p.n_tiles = (p.n + block - 1) / block;
    if (p.n_tiles == 0) return CHER_OK;
    const size_t smem = cher::kernel_smem_bytes(fp32, block, p);
    const int kmode = cher::kernel_mode(mode, p) |
                      (persistent ? cher::occupancy_bits(fp32, block, c->ctas_per_sm) : 0);
    if (cher::kernel_prepare(fp32, block, kmode, smem) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ERANGE;
    }
    int grid;
    if (persistent && c->ctas_per_sm > 0) {
        const int fit = cher::kernel_max_ctas_per_sm(fp32, block, kmode, smem);
        const int per_sm = std::max(1, std::min(c->ctas_per_sm, fit));
        grid = static_cast<int>(std::min<int64_t>(p.n_tiles, int64_t(per_sm) * c->num_sms));
        p.tile_counter = c->d_scratch;
        if (cudaMemsetAsync(c->d_scratch, 0, sizeof(unsigned long long),
                            static_cast<cudaStream_t>(stream)) != cudaSuccess)
            return CHER_ECUDA;
    } else {
        if (p.n_tiles > 0x7fffffff) return CHER_ERANGE;
        grid = static_cast<int>(p.n_tiles);
        p.tile_counter = nullptr;
    }
    if (cher::kernel_launch(fp32, block, kmode, grid, smem, p, stream) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ECUDA;
    }
    return CHER_OK;
}

bool check_device(const cher_ctx *c) {
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess && d == c->device;
}

}  // namespace

extern "C" {

const char *cher_status_string(cher_status s) {
    switch (s) {
    case CHER_OK: return "ok";
    case CHER_EINVAL: return "invalid argument";
    case CHER_ENOMEM: return "out of memory";
    case CHER_ECUDA: return "CUDA runtime error";
    case CHER_ESTATE: return "refraction tables not built";
    case CHER_ERANGE: return "size out of supported range";
    case CHER_EOVERFLOW: return "telescope buffer overflow";
    case CHER_ETIMEOUT: return "device wait timed out";
    case CHER_EBOUNDS: return "a device index check failed (bounds-checked build)";
    }
    return "unknown status";
}

cher_status cher_create(const cher_atmosphere *atm, double h_obs, const cher_telescope *tel,
                        int32_t n_tel, const cher_options *opt, cher_ctx **out) {
    if (!atm || !tel || !out || n_tel < 1 || n_tel > 4096 || !std::isfinite(h_obs))
        return CHER_EINVAL;
    *out = nullptr;
    for (int k = 0; k < n_tel; ++k)
        if (!(tel[k].r > 0.0) || !std::isfinite(tel[k].x) || !std::isfinite(tel[k].y) ||
            !std::isfinite(tel[k].z) || !std::isfinite(tel[k].r))
            return CHER_EINVAL;
    cher_options o{5.0, 300.0, 600.0, 10000};
    if (opt) {
        if (opt->bunch_size != 0.0) o.bunch_size = opt->bunch_size;
        if (opt->lambda_min_nm != 0.0) o.lambda_min_nm = opt->lambda_min_nm;
        if (opt->lambda_max_nm != 0.0) o.lambda_max_nm = opt->lambda_max_nm;
        if (opt->n_fine != 0) o.n_fine = opt->n_fine;
    }
    if (!(o.bunch_size > 0.0) || !(o.lambda_min_nm > 0.0) ||
        !(o.lambda_max_nm > o.lambda_min_nm) || o.n_fine < 2 || o.n_fine > (1 << 20))
        return CHER_EINVAL;
    cher_ctx *c = new (std::nothrow) cher_ctx;
    if (!c) return CHER_ENOMEM;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete c;
        return CHER_ECUDA;
    }
    c->atm = *atm;
    c->h_obs = h_obs;
    c->tel.assign(tel, tel + n_tel);
    c->opt = o;
    // yield constants: K = 2 pi alpha (1/lambda1 - 1/lambda2), lambda in m
    c->inv_me = 1.0 / cher::kMe;
    const double two_pi_alpha = (2.0 * cher::kPi) * cher::kAlpha;
    const double inv1 = 1.0e9 / o.lambda_min_nm;
    const double inv2 = 1.0e9 / o.lambda_max_nm;
    const double dinv = inv1 - inv2;
    c->K = two_pi_alpha * dinv;
    c->inv_B = 1.0 / o.bunch_size;
    c->lam_inv1 = 1.0 / o.lambda_min_nm;
    c->lam_dinv = 1.0 / o.lambda_min_nm - 1.0 / o.lambda_max_nm;
    if (cudaMalloc(reinterpret_cast<void **>(&c->d_scratch), 256) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return CHER_ENOMEM;
    }
    *out = c;
    return CHER_OK;
}

cher_status cher_build_refraction_tables(cher_ctx *c, int32_t n_heights, int32_t n_zenith,
                                         double zenith_max_deg, double h_max) {
    if (!c) return CHER_EINVAL;
    if (!check_device(c)) return CHER_EINVAL;
    cher::HostTables T;
    const double th = zenith_max_deg * cher::kPi / 180.0;
    cher_status s = cher::build_tables(c->atm, c->h_obs, c->opt.n_fine, n_heights, n_zenith, th,
                                       h_max, T, c->earth_radius);
    if (s != CHER_OK) return s;
    // candidate grids for two zenith bands: photons steeper than 25 degrees
    // (the bulk of a near-vertical shower) see a much smaller reach.  In a
    // curved atmosphere the ground point lies up to rho^2 / 2R_E below the
    // tangent plane and the local vertical is tilted by up to rho / R_E
    // (rho: the telescopes' distance from the core plus their reach): the
    // spheres' heights and the zenith range grow by that much for the grid.
    std::vector<cher_telescope> tg(c->tel);
    double tilt = 0.0;
    if (c->earth_radius > 0.0) {
        double rho_max = 0.0;
        for (const cher_telescope &q : c->tel)
            rho_max = std::max(rho_max, std::hypot(q.x, q.y) + q.r);
        rho_max += 1000.0;
        tilt = rho_max / c->earth_radius;
        for (cher_telescope &q : tg)
            q.z = std::fabs(q.z) + rho_max * rho_max / (2.0 * c->earth_radius);
    }
    cher::HostGrid G[2];
    const double th_band = std::min(th, 25.0 * cher::kPi / 180.0);
    s = cher::build_grid(tg.data(), static_cast<int32_t>(tg.size()), th_band + tilt, G[0]);
    if (s != CHER_OK) return s;
    s = cher::build_grid(tg.data(), static_cast<int32_t>(tg.size()),
                         std::min(th + tilt, 85.0 * cher::kPi / 180.0), G[1]);
    if (s != CHER_OK) return s;
    if (static_cast<double>(n_heights) * n_zenith * 32.0 > 4.0e9) return CHER_ERANGE;
    free_tables(c);
    c->T = std::move(T);
    c->G[0] = std::move(G[0]);
    c->G[1] = std::move(G[1]);
    c->q_band = std::sin(th_band) * std::sin(th_band);
    c->eta_obs = cher::eta_lookup(c->T, c->h_obs);
    c->eta_slope = 0.0;
    for (int k = 0; k + 1 < c->T.n_fine; ++k)
        c->eta_slope = std::max(c->eta_slope, std::fabs(c->T.eta[k + 1] - c->T.eta[k]) * c->T.inv_dh);
    // the largest relative step of eta between nodes inside a layer (the
    // density jumps at the boundaries; a cell that holds one is left out)
    c->eta_jump = 0.0;
    for (int k = 0; k + 1 < c->T.n_fine; ++k) {
        const double h0 = static_cast<double>(k) / c->T.inv_dh;
        const double h1 = static_cast<double>(k + 1) / c->T.inv_dh;
        bool straddle = false;
        for (int l = 0; l < 6; ++l)
            straddle = straddle || (c->atm.h_bound[l] > h0 && c->atm.h_bound[l] <= h1);
        if (straddle || !(c->T.eta[k] > 0.0)) continue;
        c->eta_jump = std::max(c->eta_jump, std::fabs(c->T.eta[k + 1] - c->T.eta[k]) / c->T.eta[k]);
    }
    c->eta_jump *= 1.5;

    const int H = c->T.H, Z = c->T.Z;
    const size_t per = entry_values(c->T);
    std::vector<double> t64;
    if (per == 4) {
        // FP64 in flat layers: one (ax, al) pair per node, [H][Z]
        t64.resize(static_cast<size_t>(H) * Z * 2);
        for (size_t a = 0; a < static_cast<size_t>(H) * Z; ++a) {
            t64[2 * a] = c->T.ax[a];
            t64[2 * a + 1] = c->T.al[a];
        }
    } else {
        t64.resize(static_cast<size_t>(H) * (Z - 1) * per);
        for (int j = 0; j < H; ++j)
            for (int k = 0; k < Z - 1; ++k)
                pack_entry(c->T, j, k, &t64[(static_cast<size_t>(j) * (Z - 1) + k) * per]);
    }
    // FP32 likewise: in flat layers one (ax, al) pair per node (half the
    // bytes of pair-interleaved entries: the bunch loop reads the cell's four
    // nodes as four 8-byte loads, and more of a large table stays in L1); in
    // a curved atmosphere the FP64 entries rounded
    std::vector<float> t32;
    if (per == 4) {
        t32.resize(static_cast<size_t>(H) * Z * 2);
        for (size_t a = 0; a < static_cast<size_t>(H) * Z; ++a) {
            t32[2 * a] = static_cast<float>(c->T.ax[a]);
            t32[2 * a + 1] = static_cast<float>(c->T.al[a]);
        }
    } else {
        t32.resize(t64.size());
        for (size_t q = 0; q < t64.size(); ++q) t32[q] = static_cast<float>(t64[q]);
    }
    std::vector<float> e32(c->T.eta.begin(), c->T.eta.end());
    const size_t nt = c->tel.size();
    std::vector<double> tel64(nt * 4);
    std::vector<float> tel32(nt * 4);
    for (size_t k = 0; k < nt; ++k) {
        const cher_telescope &q = c->tel[k];
        const double v[4] = {q.x, q.y, q.z, q.r * q.r};
        for (int m = 0; m < 4; ++m) {
            tel64[4 * k + m] = v[m];
            tel32[4 * k + m] = static_cast<float>(v[m]);
        }
    }
    cher_status r;
    double *d_tab64 = nullptr;
    float *d_tab32 = nullptr, *d_tel32 = nullptr;
    double *d_tel64 = nullptr;
    if ((r = upload(&c->d_eta64, c->T.eta.data(), c->T.eta.size())) != CHER_OK ||
        (r = upload(&c->d_eta32, e32.data(), e32.size())) != CHER_OK ||
        (r = upload(&d_tab64, t64.data(), t64.size())) != CHER_OK ||
        (r = upload(&d_tab32, t32.data(), t32.size())) != CHER_OK ||
        (r = upload(&d_tel64, tel64.data(), tel64.size())) != CHER_OK ||
        (r = upload(&d_tel32, tel32.data(), tel32.size())) != CHER_OK ||
        (r = upload_grid(c, 0)) != CHER_OK || (r = upload_grid(c, 1)) != CHER_OK) {
        c->d_tab64 = d_tab64;
        c->d_tab32 = d_tab32;
        c->d_tel64 = d_tel64;
        c->d_tel32 = d_tel32;
        free_tables(c);
        return r;
    }
    c->d_tab64 = d_tab64;
    c->d_tab32 = d_tab32;
    c->d_tel64 = d_tel64;
    c->d_tel32 = d_tel32;
    c->built = true;
    c->tab_H = n_heights;
    c->tab_Z = n_zenith;
    c->tab_zen = zenith_max_deg;
    c->tab_hmax = h_max;
    return build_dispersion_tables(c);
}

cher_status cher_set_atmosphere(cher_ctx *c, const cher_atmosphere *atm) {
    if (!c || !atm) return CHER_EINVAL;
    const cher_atmosphere old = c->atm;
    c->atm = *atm;
    if (!c->built) return CHER_OK;
    const cher_status s = cher_build_refraction_tables(c, c->tab_H, c->tab_Z, c->tab_zen,
                                                       c->tab_hmax);
    if (s != CHER_OK) c->atm = old;
    return s;
}

static void free_transmission(cher_ctx *c) {
    cudaFree(c->d_trans64);
    cudaFree(c->d_trans32);
    c->d_trans64 = nullptr;
    c->d_trans32 = nullptr;
}

cher_status cher_set_transmission(cher_ctx *c, const cher_transmission *tb) {
    if (!c) return CHER_EINVAL;
    if (!check_device(c)) return CHER_EINVAL;
    if (!tb) {
        if (cudaDeviceSynchronize() != cudaSuccess) return CHER_ECUDA;
        free_transmission(c);
        return CHER_OK;
    }
    if (!tb->tau || tb->n_lambda < 2 || tb->n_lambda > 4096 || tb->n_height < 2 ||
        tb->n_height > 4096 || !std::isfinite(tb->lambda_min_nm) ||
        !std::isfinite(tb->lambda_max_nm) || !(tb->lambda_max_nm > tb->lambda_min_nm) ||
        !std::isfinite(tb->h_min) || !std::isfinite(tb->h_max) || !(tb->h_max > tb->h_min))
        return CHER_EINVAL;
    const size_t n = static_cast<size_t>(tb->n_lambda) * tb->n_height;
    std::vector<float> t32(n);
    for (size_t k = 0; k < n; ++k) {
        if (!std::isfinite(tb->tau[k]) || tb->tau[k] < 0.0) return CHER_EINVAL;
        t32[k] = static_cast<float>(tb->tau[k]);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return CHER_ECUDA;
    free_transmission(c);
    cher_status r;
    if ((r = upload(&c->d_trans64, tb->tau, n)) != CHER_OK ||
        (r = upload(&c->d_trans32, t32.data(), n)) != CHER_OK) {
        free_transmission(c);
        return r;
    }
    c->trans_nl = tb->n_lambda;
    c->trans_nh = tb->n_height;
    c->trans_l0 = tb->lambda_min_nm;
    c->trans_l1 = tb->lambda_max_nm;
    c->trans_h0 = tb->h_min;
    c->trans_h1 = tb->h_max;
    return CHER_OK;
}

cher_status cher_pack_records(cher_ctx *c, const cher_output *out, cher_precision prec,
                              int64_t max_records, void *dst_pos, void *dst_tim,
                              uint64_t *dst_key, int64_t *tel_offset, void *stream) {
    if (!c || !out || max_records < 0 || bad_ptr(tel_offset)) return CHER_EINVAL;
    if (prec != CHER_FP64 && prec != CHER_FP32_BULK) return CHER_EINVAL;
    if (bad_ptr(out->count) || out->cap_per_tel < 0) return CHER_EINVAL;
    if (out->cap_per_tel > 0 && (bad_ptr(out->pos) || bad_ptr(out->tim) || bad_ptr(out->key)))
        return CHER_EINVAL;
    if (max_records > 0 && (bad_ptr(dst_pos) || bad_ptr(dst_tim) || bad_ptr(dst_key)))
        return CHER_EINVAL;
    if (!check_device(c)) return CHER_EINVAL;
    if (cher::pack_records(prec == CHER_FP32_BULK, out->pos, out->tim, out->key, out->count,
                           out->cap_per_tel, static_cast<int>(c->tel.size()), max_records,
                           dst_pos, dst_tim, dst_key, tel_offset, c->num_sms,
                           stream) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ECUDA;
    }
    return CHER_OK;
}

cher_status cher_set_curved(cher_ctx *c, double earth_radius_m) {
    if (!c || !std::isfinite(earth_radius_m)) return CHER_EINVAL;
    if (earth_radius_m != 0.0 && !(earth_radius_m >= 1.0e6 && earth_radius_m <= 1.0e8))
        return CHER_EINVAL;
    if (!check_device(c)) return CHER_EINVAL;
    const double old = c->earth_radius;
    c->earth_radius = earth_radius_m;
    if (!c->built) return CHER_OK;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        c->earth_radius = old;
        return CHER_ECUDA;
    }
    const cher_status s = cher_build_refraction_tables(c, c->tab_H, c->tab_Z, c->tab_zen,
                                                       c->tab_hmax);
    if (s != CHER_OK) {
        c->earth_radius = old;
        cher_build_refraction_tables(c, c->tab_H, c->tab_Z, c->tab_zen, c->tab_hmax);
    }
    return s;
}

cher_status cher_set_dispersion(cher_ctx *c, const double *kappa, int32_t k) {
    if (!c) return CHER_EINVAL;
    if (!check_device(c)) return CHER_EINVAL;
    if (!kappa || k == 0) {
        if (cudaDeviceSynchronize() != cudaSuccess) return CHER_ECUDA;
        free_dispersion_tables(c);
        c->disp_k = 0;
        return CHER_OK;
    }
    if (k < 2 || k > cher::kDispMax) return CHER_EINVAL;
    for (int m = 0; m < k; ++m)
        if (!std::isfinite(kappa[m]) || !(kappa[m] > 0.0) || (m > 0 && kappa[m] > kappa[m - 1]))
            return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    if (cudaDeviceSynchronize() != cudaSuccess) return CHER_ECUDA;
    c->disp_k = k;
    for (int m = 0; m < cher::kDispMax; ++m) c->kap[m] = m < k ? kappa[m] : 0.0;
    const cher_status r = build_dispersion_tables(c);
    if (r != CHER_OK) c->disp_k = 0;
    return r;
}

cher_status cher_generate_steps(cher_ctx *c, const cher_shower *sh, int32_t n_showers,
                                uint64_t seed, cher_precision prec, const cher_step_buffers *out,
                                void *stream) {
    if (!c || !sh || n_showers < 1 || !out) return CHER_EINVAL;
    if (prec != CHER_FP64 && prec != CHER_FP32_BULK) return CHER_EINVAL;
    if (!check_device(c)) return CHER_EINVAL;
    constexpr int kCdf = 1024;
    constexpr double kX0 = 36.7, kEc = 85.0, kXsea = 1030.0, kH = 8000.0, kStart = 30000.0;
    const double pi = 3.14159265358979323846;
    int64_t total = 0;
    for (int s = 0; s < n_showers; ++s) {
        const cher_shower &S = sh[s];
        if (!(S.e0_mev > kEc) || !std::isfinite(S.e0_mev) || !(S.zenith >= 0.0) ||
            !(S.zenith < 0.5 * pi) || !std::isfinite(S.azimuth) || !std::isfinite(S.core_x) ||
            !std::isfinite(S.core_y) || S.n_steps < 0)
            return CHER_EINVAL;
        total += S.n_steps;
        if (total > (int64_t(1) << 40)) return CHER_ERANGE;
    }
    if (bad_ptr(out->t_ref)) return CHER_EINVAL;
    if (total > 0 && (bad_ptr(out->x0) || bad_ptr(out->y0) || bad_ptr(out->z0) ||
                      bad_ptr(out->t0) || bad_ptr(out->len) || bad_ptr(out->ekin) ||
                      bad_ptr(out->ux) || bad_ptr(out->uy) || bad_ptr(out->uz) ||
                      bad_ptr(out->shower)))
        return CHER_EINVAL;
    std::vector<cher::GenShower> G(n_showers);
    std::vector<int64_t> first(n_showers + 1, 0);
    std::vector<float> cdf(static_cast<size_t>(n_showers) * kCdf);
    std::vector<double> t_ref(n_showers), row;
    for (int s = 0; s < n_showers; ++s) {
        const cher_shower &S = sh[s];
        const double cz = std::cos(S.zenith), sz = std::sin(S.zenith);
        const double ax = sz * std::cos(S.azimuth), ay = sz * std::sin(S.azimuth), az = -cz;
        double b1x = ay, b1y = -ax;
        const double nb = std::sqrt(b1x * b1x + b1y * b1y);
        if (nb > 1e-12) {
            b1x /= nb;
            b1y /= nb;
        } else {
            b1x = 1.0;
            b1y = 0.0;
        }
        const double b1z = 0.0;
        const double b2x = ay * b1z - az * b1y, b2y = az * b1x - ax * b1z, b2z = ax * b1y - ay * b1x;
        const double t_g = kXsea * std::exp(-(c->h_obs / kH)) / cz / kX0;
        const double s_ref = (kStart - c->h_obs) / cz;
        cher::GenShower &g = G[s];
        g.ax = static_cast<float>(ax); g.ay = static_cast<float>(ay); g.az = static_cast<float>(az);
        g.b1x = static_cast<float>(b1x); g.b1y = static_cast<float>(b1y); g.b1z = 0.0f;
        g.b2x = static_cast<float>(b2x); g.b2y = static_cast<float>(b2y);
        g.b2z = static_cast<float>(b2z);
        g.cz = static_cast<float>(cz);
        g.x0cz = static_cast<float>(kX0 * cz);
        g.core_x = static_cast<float>(S.core_x);
        g.core_y = static_cast<float>(S.core_y);
        g.s_ref = static_cast<float>(s_ref);
        g.dt = static_cast<float>(t_g / (kCdf - 1));
        t_ref[s] = s_ref / cher::kC;
        first[s + 1] = first[s] + S.n_steps;
        const auto key = std::make_pair(S.e0_mev, S.zenith);
        auto it = c->cdf_cache.find(key);
        if (it == c->cdf_cache.end()) {
            if (c->cdf_cache.size() >= 4096) c->cdf_cache.clear();
            cher::greisen_cdf_host(std::log(S.e0_mev / kEc), t_g, kCdf, row);
            std::vector<float> rf(row.begin(), row.end());
            it = c->cdf_cache.emplace(key, std::move(rf)).first;
        }
        std::copy(it->second.begin(), it->second.end(), cdf.begin() + static_cast<size_t>(s) * kCdf);
    }
    // one scratch block: shower constants | offsets | tables, staged in pinned
    // host memory (with t_ref after it) and uploaded in one asynchronous copy
    const size_t o_first = (sizeof(cher::GenShower) * n_showers + 15) & ~size_t(15);
    const size_t o_cdf = (o_first + sizeof(int64_t) * (n_showers + 1) + 15) & ~size_t(15);
    const size_t bytes = o_cdf + sizeof(float) * cdf.size();
    const size_t o_tref = (bytes + 15) & ~size_t(15);
    const size_t staged = o_tref + sizeof(double) * n_showers;
    cher_status r;
    if ((r = grow(&c->d_gen, c->gen_cap, static_cast<int64_t>(bytes))) != CHER_OK) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!c->gen_ev && cudaEventCreateWithFlags(&c->gen_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        c->gen_ev = nullptr;
        return CHER_ECUDA;
    }
    // the previous call's upload has read the staging before it is rewritten
    if (c->gen_ev_pending && cudaEventSynchronize(c->gen_ev) != cudaSuccess) return CHER_ECUDA;
    c->gen_ev_pending = false;
    if (static_cast<int64_t>(staged) > c->h_gen_cap) {
        cudaFreeHost(c->h_gen);
        c->h_gen = nullptr;
        c->h_gen_cap = 0;
        void *h = nullptr;
        if (cudaHostAlloc(&h, staged, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return CHER_ENOMEM;
        }
        c->h_gen = static_cast<unsigned char *>(h);
        c->h_gen_cap = static_cast<int64_t>(staged);
    }
    std::memcpy(c->h_gen, G.data(), sizeof(cher::GenShower) * n_showers);
    std::memcpy(c->h_gen + o_first, first.data(), sizeof(int64_t) * (n_showers + 1));
    std::memcpy(c->h_gen + o_cdf, cdf.data(), sizeof(float) * cdf.size());
    std::memcpy(c->h_gen + o_tref, t_ref.data(), sizeof(double) * n_showers);
    if (cudaMemcpyAsync(c->d_gen, c->h_gen, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(out->t_ref, c->h_gen + o_tref, sizeof(double) * n_showers,
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(c->gen_ev, st) != cudaSuccess)
        return CHER_ECUDA;
    c->gen_ev_pending = true;
    cher::GenParams g;
    g.showers = reinterpret_cast<const cher::GenShower *>(c->d_gen);
    g.first = reinterpret_cast<const int64_t *>(c->d_gen + o_first);
    g.n_showers = n_showers;
    g.n_cdf = kCdf;
    g.cdf = reinterpret_cast<const float *>(c->d_gen + o_cdf);
    g.key0 = static_cast<uint32_t>(seed & 0xffffffffu);
    g.key1 = static_cast<uint32_t>(seed >> 32);
    g.h_obs = static_cast<float>(c->h_obs);
    g.n = total;
    g.x0 = out->x0; g.y0 = out->y0; g.z0 = out->z0; g.t0 = out->t0;
    g.len = out->len; g.ekin = out->ekin;
    g.ux = out->ux; g.uy = out->uy; g.uz = out->uz;
    g.dirs_fp32 = prec == CHER_FP32_BULK;
    g.shower = out->shower;
    if (cher::generate_steps(g, c->num_sms, stream) != cudaSuccess) return CHER_ECUDA;
    return CHER_OK;
}

cher_status cher_destroy(cher_ctx *c) {
    if (!c) return CHER_OK;
    free_tables(c);
    free_adjoint_scratch(c);
    free_transmission(c);
    free_dispersion_tables(c);
    if (c->gen_ev) {
        cudaEventSynchronize(c->gen_ev);
        cudaEventDestroy(c->gen_ev);
    }
    cudaFreeHost(c->h_gen);
    cudaFree(c->d_gen);
    cudaFree(c->d_fb);
    cudaFree(c->d_fb_count);
    cudaFree(c->d_scratch);
    delete c;
    return CHER_OK;
}

cher_status cher_set_launch(cher_ctx *c, int32_t block_threads, int32_t ctas_per_sm) {
    if (!c) return CHER_EINVAL;
    if (block_threads != 128 && block_threads != 256 && block_threads != 512) return CHER_EINVAL;
    if (ctas_per_sm < 0 || ctas_per_sm > 10) return CHER_EINVAL;
    c->block = block_threads;
    c->ctas_per_sm = ctas_per_sm;
    return CHER_OK;
}

cher_status cher_get_launch(const cher_ctx *c, int32_t *block_threads, int32_t *ctas_per_sm) {
    if (!c) return CHER_EINVAL;
    if (block_threads) *block_threads = c->block;
    if (ctas_per_sm) *ctas_per_sm = c->ctas_per_sm;
    return CHER_OK;
}

cher_status cher_generate_propagate(cher_ctx *c, const cher_tracks *t, uint64_t seed,
                                    cher_precision prec, const cher_output *out, void *stream) {
    return cher_generate_propagate_ex(c, t, seed, prec, out, nullptr, stream);
}

cher_status cher_generate_propagate_ex(cher_ctx *c, const cher_tracks *t, uint64_t seed,
                                       cher_precision prec, const cher_output *out,
                                       const cher_profile *prof, void *stream) {
    if (!c || !out || !tracks_ok(t)) return CHER_EINVAL;
    if (prof && (bad_ptr(prof->profile) || prof->n_bins < 1 || prof->n_bins > 65536 ||
                 !(prof->bin_gcm2 > 0.0) || !std::isfinite(prof->bin_gcm2) ||
                 reinterpret_cast<uintptr_t>(prof->profile) % alignof(double) ||
                 reinterpret_cast<uintptr_t>(prof->axis_cos) % alignof(double) ||
                 int64_t(std::max(t->n_showers, 1)) * prof->n_bins > 0x7fffffffLL))
        return CHER_EINVAL;
    if (prof && c->earth_radius > 0.0) return CHER_EINVAL;   // depths of flat layers
    if (prec != CHER_FP64 && prec != CHER_FP32_BULK) return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    if (!check_device(c)) return CHER_EINVAL;
    if (bad_ptr(out->count) || bad_ptr(out->stats)) return CHER_EINVAL;
    if (out->cap_per_tel < 0) return CHER_EINVAL;
    if (out->cap_per_tel > 0 && (bad_ptr(out->pos) || bad_ptr(out->tim) || bad_ptr(out->key)))
        return CHER_EINVAL;
    constexpr size_t al = 16;
    if (reinterpret_cast<uintptr_t>(out->pos) % al || reinterpret_cast<uintptr_t>(out->tim) % al)
        return CHER_EINVAL;
    const bool fp32 = prec == CHER_FP32_BULK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out->count, 0, c->tel.size() * sizeof(unsigned long long), s) !=
            cudaSuccess ||
        cudaMemsetAsync(out->stats, 0, CHER_NSTATS * sizeof(unsigned long long), s) != cudaSuccess)
        return CHER_ECUDA;
    cher::KParams p = base_params(c, t, seed, fp32);
    p.pos = out->pos;
    p.tim = out->tim;
    p.key = out->key;
    p.cap = out->cap_per_tel;
    p.count = out->count;
    p.stats = out->stats;
    const bool fb = p.fb_q > 0.0;
    if (fb) {
        // the fallback queue: the set size or max(2^20, 4 n) records
        const size_t rec = cher::fallback_record_bytes(fp32);
        const int64_t want = c->fb_records > 0 ? c->fb_records
                                               : std::max<int64_t>(int64_t(1) << 20, 4 * t->n);
        int64_t bytes_cap = c->fb_cap;
        if (static_cast<int64_t>(want * rec) > bytes_cap) {
            unsigned char *buf = static_cast<unsigned char *>(c->d_fb);
            cher_status r = grow(&buf, bytes_cap, static_cast<int64_t>(want * rec));
            c->d_fb = buf;
            c->fb_cap = bytes_cap;
            if (r != CHER_OK) return r;
        }
        if (!c->d_fb_count) {
            int64_t one = 0;
            cher_status r = grow(&c->d_fb_count, one, 1);
            if (r != CHER_OK) return r;
        }
        if (cudaMemsetAsync(c->d_fb_count, 0, sizeof(unsigned long long), s) != cudaSuccess)
            return CHER_ECUDA;
        p.fb_list = c->d_fb;
        p.fb_count = c->d_fb_count;
        p.fb_cap = std::min<int64_t>(want, c->fb_cap / static_cast<int64_t>(rec));
    }
    if (prof) {
        p.prof = prof->profile;
        p.prof_cos = prof->axis_cos;
        p.prof_bins = prof->n_bins;
        p.prof_rows = std::max(t->n_showers, 1);
        p.prof_dx = prof->bin_gcm2;
        p.prof_inv_dx = 1.0 / prof->bin_gcm2;
        cher::fill_float_constants(p);
    }
    cher_status r = launch(c, p, fp32, cher::MODE_HITS, true, stream);
    if (r != CHER_OK || !fb || p.n == 0) return r;
    if (cher::launch_fallback(fp32, p.trans != nullptr, p.disp_k > 0, p, c->num_sms, stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return CHER_ECUDA;
    }
    return CHER_OK;
}

cher_status cher_set_fallback(cher_ctx *c, double zenith_max_deg, int64_t queue_records) {
    if (!c || !std::isfinite(zenith_max_deg)) return CHER_EINVAL;
    if (queue_records < 0 || queue_records > (int64_t(1) << 34)) return CHER_EINVAL;
    c->fb_records = queue_records;
    if (zenith_max_deg == 0.0) {
        c->fb_deg = 0.0;
        return CHER_OK;
    }
    if (!(zenith_max_deg > 0.0) || zenith_max_deg > 85.0) return CHER_EINVAL;
    if (c->built && !(zenith_max_deg > c->tab_zen)) return CHER_EINVAL;
    c->fb_deg = zenith_max_deg;
    return CHER_OK;
}

static cher_status round_or_split(const double *in, float *out, float *lo, int64_t n,
                                  void *stream) {
    if (n < 0 || (n > 0 && (bad_ptr(in) || bad_ptr(out)))) return CHER_EINVAL;
    if (n == 0) return CHER_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ECUDA;
    }
    if (cher::round_to_float(in, out, lo, n, sms, stream) != cudaSuccess) return CHER_ECUDA;
    return CHER_OK;
}

cher_status cher_round_to_float(const double *in, float *out, int64_t n, void *stream) {
    return round_or_split(in, out, nullptr, n, stream);
}

cher_status cher_split_to_float(const double *in, float *hi, float *lo, int64_t n,
                                void *stream) {
    if (n > 0 && bad_ptr(lo)) return CHER_EINVAL;
    return round_or_split(in, hi, lo, n, stream);
}

cher_status cher_sync_status(cher_ctx *c, const cher_output *out, unsigned long long *stats_host,
                             void *stream) {
    if (!c || !out || !out->stats) return CHER_EINVAL;
    unsigned long long st[CHER_NSTATS];
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return CHER_ECUDA;
    if (cudaMemcpy(st, out->stats, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
        return CHER_ECUDA;
    if (stats_host) std::memcpy(stats_host, st, sizeof(st));
    if (st[CHER_STAT_DEBUG]) return CHER_EBOUNDS;
    return st[CHER_STAT_OVERFLOW] ? CHER_EOVERFLOW : CHER_OK;
}

cher_status cher_segment_yield(cher_ctx *c, const cher_tracks *t, cher_precision prec, int32_t *nb,
                               double *w, void *stream) {
    if (!c || !tracks_ok(t) || (t->n > 0 && (!nb || !w))) return CHER_EINVAL;
    if (prec != CHER_FP64 && prec != CHER_FP32_BULK) return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    if (!check_device(c)) return CHER_EINVAL;
    const bool fp32 = prec == CHER_FP32_BULK;
    cher::KParams p = base_params(c, t, 0, fp32);
    p.y_nb = nb;
    p.y_w = w;
    return launch(c, p, fp32, cher::MODE_YIELD, false, stream);
}

cher_status cher_trace_bunches(cher_ctx *c, const cher_tracks *t, uint64_t seed,
                               cher_precision prec, const int64_t *bunch_off,
                               const cher_trace *out, void *stream) {
    if (!c || !tracks_ok(t) || !out) return CHER_EINVAL;
    if (prec != CHER_FP64 && prec != CHER_FP32_BULK) return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    if (!check_device(c)) return CHER_EINVAL;
    if (t->n > 0 && (!bunch_off || !out->pos || !out->tim || !out->status || !out->nhit ||
                     !out->first_hit))
        return CHER_EINVAL;
    const bool fp32 = prec == CHER_FP32_BULK;
    cher::KParams p = base_params(c, t, seed, fp32);
    p.pos = out->pos;
    p.tim = out->tim;
    p.bunch_off = bunch_off;
    p.t_status = out->status;
    p.t_nbunch = out->n_bunches;
    p.t_nhit = out->nhit;
    p.t_first = out->first_hit;
    return launch(c, p, fp32, cher::MODE_TRACE, false, stream);
}

cher_status cher_get_tables(const cher_ctx *c, double *eta, double *ax, double *al) {
    if (!c) return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    if (eta) std::copy(c->T.eta.begin(), c->T.eta.end(), eta);
    if (ax) std::copy(c->T.ax.begin(), c->T.ax.end(), ax);
    if (al) std::copy(c->T.al.begin(), c->T.al.end(), al);
    return CHER_OK;
}

cher_status cher_build_tables_host(const cher_atmosphere *atm, double h_obs, int32_t n_fine,
                                   int32_t n_heights, int32_t n_zenith, double zenith_max_deg,
                                   double h_max, double *eta, double *ax, double *al) {
    if (!atm || !eta || !ax || !al) return CHER_EINVAL;
    cher::HostTables T;
    const cher_status s = cher::build_tables(*atm, h_obs, n_fine, n_heights, n_zenith,
                                             zenith_max_deg * cher::kPi / 180.0, h_max, T);
    if (s != CHER_OK) return s;
    std::copy(T.eta.begin(), T.eta.end(), eta);
    std::copy(T.ax.begin(), T.ax.end(), ax);
    std::copy(T.al.begin(), T.al.end(), al);
    return CHER_OK;
}

cher_status cher_build_curved_tables_host(const cher_atmosphere *atm, double earth_radius_m,
                                          double h_obs, int32_t n_heights, int32_t n_zenith,
                                          double zenith_max_deg, double h_max, double *ax,
                                          double *al, double *ag) {
    if (!atm || !ax || !al || !ag || !(earth_radius_m >= 1.0e6 && earth_radius_m <= 1.0e8))
        return CHER_EINVAL;
    cher::HostTables T;
    const cher_status s = cher::build_tables(*atm, h_obs, 2, n_heights, n_zenith,
                                             zenith_max_deg * cher::kPi / 180.0, h_max, T,
                                             earth_radius_m);
    if (s != CHER_OK) return s;
    std::copy(T.ax.begin(), T.ax.end(), ax);
    std::copy(T.al.begin(), T.al.end(), al);
    std::copy(T.ag.begin(), T.ag.end(), ag);
    return CHER_OK;
}

cher_status cher_autotune(cher_ctx *c, const cher_tracks *t, uint64_t seed, cher_precision prec,
                          const cher_output *out, const char *cache_path, void *stream) {
    if (!c || !tracks_ok(t) || !out) return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) return CHER_ECUDA;
    char tag[512];
    const long long tiles_bucket = static_cast<long long>(std::log2(double(t->n) + 1.0));
    std::snprintf(tag, sizeof(tag), "%s|%d|%lld|%d|%d", prop.name, static_cast<int>(prec),
                  tiles_bucket, static_cast<int>(c->tel.size()), c->T.Z);
    for (char *q = tag; *q; ++q)
        if (*q == ' ') *q = '_';
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "r")) {
            char line[512];
            while (std::fgets(line, sizeof(line), f)) {
                char key[300];
                int b, cps;
                if (std::sscanf(line, "%299s %d %d", key, &b, &cps) == 3 &&
                    std::strcmp(key, tag) == 0) {
                    std::fclose(f);
                    return cher_set_launch(c, b, cps);
                }
            }
            std::fclose(f);
        }
    }
    const int blocks[] = {128, 256, 512};
    const int ctas[] = {0, 1, 2, 3, 4, 6, 8, 9, 10};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return CHER_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float best = 1e30f;
    int best_b = c->block, best_c = c->ctas_per_sm;
    cher_status rc = CHER_OK;
    for (int b : blocks)
        for (int cps : ctas) {
            if ((b == 512 && cps > 4) || (b == 256 && cps > 8)) continue;
            // more than 8 CTAs per SM: the FP32 hits kernel's builds for 9 and
            // 10 (other precisions and modes cap at what fits)
            if (cps > 8 && (b != 128 || prec != CHER_FP32_BULK)) continue;
            c->block = b;
            c->ctas_per_sm = cps;
            float tsum = 0.0f;
            bool ok = true;
            for (int rep = 0; rep < 4 && ok; ++rep) {
                cudaEventRecord(e0, s);
                rc = cher_generate_propagate(c, t, seed, prec, out, stream);
                cudaEventRecord(e1, s);
                if (rc != CHER_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                    ok = false;
                    break;
                }
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tsum += ms;   // first run warms up
            }
            if (ok && tsum < best) {
                best = tsum;
                best_b = b;
                best_c = cps;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->block = best_b;
    c->ctas_per_sm = best_c;
    if (best >= 1e30f) return rc != CHER_OK ? rc : CHER_ECUDA;
    if (cache_path) {
        if (FILE *f = std::fopen(cache_path, "a")) {
            std::fprintf(f, "%s %d %d\n", tag, best_b, best_c);
            std::fclose(f);
        }
    }
    return CHER_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Differentiable read-out and its adjoint (no counterpart in the paper).
// ---------------------------------------------------------------------------
namespace {


cher_status readout(cher_ctx *c, const cher_tracks *t, uint64_t seed, cher_precision prec,
                    double sigma, const int32_t *nb_frozen, double *D, double *Tbar,
                    const double *gD, const double *gT, double *grad_atm, double *grad_tracks,
                    void *stream) {
    if (!c || !tracks_ok(t)) return CHER_EINVAL;
    if (prec != CHER_FP64 && prec != CHER_FP32_BULK) return CHER_EINVAL;
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return CHER_EINVAL;
    if (c->disp_k > 0) return CHER_EINVAL;   // defined for a wavelength-independent index
    if (c->earth_radius > 0.0) return CHER_EINVAL;   // and for flat layers
    if (!c->built) return CHER_ESTATE;
    if (!check_device(c)) return CHER_EINVAL;
    if (t->n > 0x7fffffffLL) return CHER_ERANGE;
    const bool fp32 = prec == CHER_FP32_BULK;
    const int n_tel = static_cast<int>(c->tel.size());
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cher_status r;
    // sensitivity tables of the refraction corrections
    if (grad_atm && !c->d_sens) {
        std::vector<double> sv;
        if ((r = cher::build_sensitivity(c->atm, c->h_obs, c->T, sv)) != CHER_OK) return r;
        if ((r = upload(&c->d_sens, sv.data(), sv.size())) != CHER_OK) return r;
    }
    int64_t cap_tmp = c->nb_cap;
    if ((r = grow(&c->d_nb, cap_tmp, t->n)) != CHER_OK) return r;
    int64_t cap_w = c->nb_cap;
    if ((r = grow(&c->d_w, cap_w, t->n)) != CHER_OK) return r;
    c->nb_cap = std::max(cap_tmp, cap_w);
    int64_t one = c->d_list_count ? 1 : 0;
    if ((r = grow(&c->d_list_count, one, 1)) != CHER_OK) return r;
    int64_t su = c->d_SU ? 2 * n_tel : 0;
    if ((r = grow(&c->d_SU, su, 2 * n_tel)) != CHER_OK) return r;
    if (!c->d_list && (r = grow(&c->d_list, c->list_cap, std::max<int64_t>(1 << 16, t->n / 8))) != CHER_OK)
        return r;
    // frozen bunch counts: the caller's, or this call's yield
    const int32_t *nb = nb_frozen;
    if (!nb) {
        cher::KParams p = base_params(c, t, seed, fp32);
        p.y_nb = c->d_nb;
        p.y_w = c->d_w;
        if ((r = launch(c, p, fp32, cher::MODE_YIELD, false, stream)) != CHER_OK) return r;
        nb = c->d_nb;
    }
    // screen: list the bunches within 6 sigma (plus a margin) of a centre
    const double rscreen = 6.0 * sigma + 0.05;
    unsigned long long count = 0;
    for (int attempt = 0; attempt < 3; ++attempt) {
        if (cudaMemsetAsync(c->d_list_count, 0, sizeof(unsigned long long), st) != cudaSuccess)
            return CHER_ECUDA;
        cher::KParams p = base_params(c, t, seed, fp32);
        p.nb_frozen = nb;
        p.list = c->d_list;
        p.list_count = c->d_list_count;
        p.list_cap = c->list_cap;
        p.rcut2 = rscreen * rscreen;
        cher::fill_float_constants(p);
        if ((r = launch(c, p, fp32, cher::MODE_SCREEN, false, stream)) != CHER_OK) return r;
        if (cudaMemcpyAsync(&count, c->d_list_count, sizeof(count), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CHER_ECUDA;
        if (static_cast<int64_t>(count) <= c->list_cap) break;
        if ((r = grow(&c->d_list, c->list_cap, static_cast<int64_t>(count) + count / 4 + 1024)) !=
            CHER_OK)
            return r;
    }
    if (static_cast<int64_t>(count) > c->list_cap) return CHER_ERANGE;
    // the pass over the listed bunches: sums, then gradients
    cher::AdjParams A;
    std::memset(&A, 0, sizeof(A));
    A.k = base_params(c, t, seed, fp32);
    A.list = c->d_list;
    A.n_list = static_cast<int64_t>(count);
    A.nb = nb;
    A.sigma = sigma;
    A.inv_2s2 = 1.0 / (2.0 * sigma * sigma);
    A.norm = 1.0 / (2.0 * cher::kPi * sigma * sigma);
    A.rcut2 = 36.0 * sigma * sigma;
    A.S = c->d_SU;
    A.U = c->d_SU + n_tel;
    A.sens = c->d_sens;
    for (int i = 0; i < 6; ++i) A.hb[i] = c->atm.h_bound[i];
    for (int i = 0; i < 5; ++i) {
        A.b[i] = c->atm.b[i];
        A.c[i] = c->atm.c[i];
    }
    A.layer0 = 0;
    while (A.layer0 < 4 && 0.0 >= A.hb[A.layer0 + 1]) ++A.layer0;
    A.dh_fine = c->T.dh;
    {
        double hc = std::min(std::max(c->h_obs, 0.0), c->T.h_max);
        const double x = hc * c->T.inv_dh;
        int k = static_cast<int>(x);
        if (k > c->T.n_fine - 2) k = c->T.n_fine - 2;
        A.ko = k;
        A.fo = x - k;
    }
    if (cudaMemsetAsync(c->d_SU, 0, 2 * n_tel * sizeof(double), st) != cudaSuccess)
        return CHER_ECUDA;
    if (cher::adjoint_pairs(fp32, 0, A, stream) != cudaSuccess) return CHER_ECUDA;
    if (D || Tbar) {
        std::vector<double> su(2 * n_tel), d(n_tel), tb(n_tel);
        if (cudaMemcpyAsync(su.data(), c->d_SU, su.size() * sizeof(double),
                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CHER_ECUDA;
        for (int k = 0; k < n_tel; ++k) {
            d[k] = su[k];
            tb[k] = su[k] > 0.0 ? su[n_tel + k] / su[k] : 0.0;
        }
        if ((D && cudaMemcpyAsync(D, d.data(), n_tel * sizeof(double), cudaMemcpyHostToDevice,
                                  st) != cudaSuccess) ||
            (Tbar && cudaMemcpyAsync(Tbar, tb.data(), n_tel * sizeof(double),
                                     cudaMemcpyHostToDevice, st) != cudaSuccess) ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return CHER_ECUDA;
    }
    if (grad_atm) {
        if (cudaMemsetAsync(grad_atm, 0, 15 * sizeof(double), st) != cudaSuccess ||
            cudaMemsetAsync(grad_tracks, 0, 6 * static_cast<size_t>(t->n) * sizeof(double), st) !=
                cudaSuccess)
            return CHER_ECUDA;
        A.gD = gD;
        A.gT = gT;
        A.grad_atm = grad_atm;
        A.grad_tracks = grad_tracks;
        if (cher::adjoint_pairs(fp32, 1, A, stream) != cudaSuccess) return CHER_ECUDA;
    }
    return CHER_OK;
}

}  // namespace

extern "C" cher_status cher_density(cher_ctx *c, const cher_tracks *t, uint64_t seed,
                                    cher_precision prec, double sigma, const int32_t *nb_frozen,
                                    double *D, double *Tbar, void *stream) {
    if (!D || !Tbar) return CHER_EINVAL;
    return readout(c, t, seed, prec, sigma, nb_frozen, D, Tbar, nullptr, nullptr, nullptr,
                   nullptr, stream);
}

extern "C" cher_status cher_adjoint(cher_ctx *c, const cher_tracks *t, uint64_t seed,
                                    cher_precision prec, double sigma, const int32_t *nb_frozen,
                                    const double *dL_dD, const double *dL_dT, double *grad_atm,
                                    double *grad_tracks, void *stream) {
    if (!dL_dD || !dL_dT || !grad_atm || (!grad_tracks && t && t->n > 0)) return CHER_EINVAL;
    return readout(c, t, seed, prec, sigma, nb_frozen, nullptr, nullptr, dL_dD, dL_dT, grad_atm,
                   grad_tracks, stream);
}

extern "C" cher_status cher_build_sensitivity_host(const cher_atmosphere *atm, double h_obs,
                                                   int32_t n_fine, int32_t n_heights,
                                                   int32_t n_zenith, double zenith_max_deg,
                                                   double h_max, double *dax, double *dal) {
    if (!atm || !dax || !dal) return CHER_EINVAL;
    cher::HostTables T;
    cher_status s = cher::build_tables(*atm, h_obs, n_fine, n_heights, n_zenith,
                                       zenith_max_deg * cher::kPi / 180.0, h_max, T);
    if (s != CHER_OK) return s;
    std::vector<double> sv;
    if ((s = cher::build_sensitivity(*atm, h_obs, T, sv)) != CHER_OK) return s;
    const size_t HZ = static_cast<size_t>(n_heights) * n_zenith;
    for (size_t e = 0; e < HZ; ++e)
        for (int q = 0; q < 10; ++q) {
            dax[q * HZ + e] = sv[e * 20 + q];
            dal[q * HZ + e] = sv[e * 20 + 10 + q];
        }
    return CHER_OK;
}

struct cher_graph {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" cher_status cher_graph_destroy(cher_graph *g) {
    if (!g) return CHER_OK;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->stream) cudaStreamDestroy(g->stream);
    delete g;
    return CHER_OK;
}

extern "C" cher_status cher_graph_create(cher_ctx *c, const cher_tracks *t, uint64_t seed,
                                         cher_precision prec, const cher_output *out,
                                         cher_graph **graph) {
    if (!graph) return CHER_EINVAL;
    *graph = nullptr;
    if (!c || !out || !tracks_ok(t)) return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    cher_graph *g = new (std::nothrow) cher_graph;
    if (!g) return CHER_ENOMEM;
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return CHER_ECUDA;
    }
    // a first uncaptured call sets the kernel attributes and checks arguments
    cher_status s = cher_generate_propagate(c, t, seed, prec, out, g->stream);
    if (s == CHER_OK && cudaStreamSynchronize(g->stream) != cudaSuccess) s = CHER_ECUDA;
    if (s != CHER_OK) {
        cher_graph_destroy(g);
        return s;
    }
    if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        cher_graph_destroy(g);
        return CHER_ECUDA;
    }
    s = cher_generate_propagate(c, t, seed, prec, out, g->stream);
    const cudaError_t e = cudaStreamEndCapture(g->stream, &g->graph);
    if (s != CHER_OK || e != cudaSuccess || !g->graph) {
        cudaGetLastError();
        cher_graph_destroy(g);
        return s != CHER_OK ? s : CHER_ECUDA;
    }
    if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess) {
        cudaGetLastError();
        cher_graph_destroy(g);
        return CHER_ECUDA;
    }
    *graph = g;
    return CHER_OK;
}

extern "C" cher_status cher_graph_launch(cher_graph *g, void *stream) {
    if (!g || !g->exec) return CHER_EINVAL;
    if (cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ECUDA;
    }
    return CHER_OK;
}

// ---------------------------------------------------------------------------
// Entry point that allocates nothing (no counterpart in the paper).
//
// The persistent kernel needs one word of scratch: the counter its CTAs
// take tiles from.  cher_generate_propagate uses a word the context
// allocated with cudaMalloc; this variant uses a fixed array compiled into
// the library instead, so the call itself never allocates.  Every GPU that
// loads the library holds the array until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = 256;
static __device__ __align__(256) unsigned long long
    g_static_scratch[kStaticScratchBytes / sizeof(unsigned long long)];

// Clears the words a call uses.  Naming the array in device code also keeps
// it in the module (an unreferenced file-scope array may be dropped).
__global__ void k_clear_static_scratch(int words) {
    if (static_cast<int>(threadIdx.x) < words) g_static_scratch[threadIdx.x] = 0ull;
}

// Device address of g_static_scratch on each device, looked up once per
// device with that device current (host code may not use the symbol itself:
// on the host it names a stand-in, not device memory).
constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void *g_static_addr[kMaxDevices] = {};

cher_status static_scratch(int device, unsigned long long **out) {
    if (device < 0 || device >= kMaxDevices) return CHER_ERANGE;
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[device]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return CHER_ECUDA;
        }
        g_static_addr[device] = ptr;
    }
    *out = static_cast<unsigned long long *>(g_static_addr[device]);
    return CHER_OK;
}

}  // namespace

extern "C" cher_status cher_generate_propagate_noalloc(cher_ctx *c, const cher_tracks *t,
                                                       uint64_t seed, cher_precision prec,
                                                       const cher_output *out, void *stream) {
    if (!c || !out || !t) return CHER_EINVAL;
    // one 8-byte tile counter of the fixed array; tile indices beyond the
    // library-wide step limit are refused before anything is launched
    const size_t need = sizeof(unsigned long long);
    if (need > kStaticScratchBytes) return CHER_ERANGE;
    if (t->n > (int64_t(1) << 40) || t->track_base > (int64_t(1) << 40)) return CHER_ERANGE;
    if (!tracks_ok(t)) return CHER_EINVAL;
    if (prec != CHER_FP64 && prec != CHER_FP32_BULK) return CHER_EINVAL;
    if (!c->built) return CHER_ESTATE;
    if (!check_device(c)) return CHER_EINVAL;
    if (bad_ptr(out->count) || bad_ptr(out->stats) || out->cap_per_tel < 0) return CHER_EINVAL;
    if (out->cap_per_tel > 0 && (bad_ptr(out->pos) || bad_ptr(out->tim) || bad_ptr(out->key)))
        return CHER_EINVAL;
    if (reinterpret_cast<uintptr_t>(out->pos) % 16 || reinterpret_cast<uintptr_t>(out->tim) % 16)
        return CHER_EINVAL;
    // the beyond-table fallback queues its bunches in memory the context
    // allocates: with it active this call would drop them where the regular
    // entry point propagates them, so it refuses instead
    if (c->fb_deg > c->tab_zen && c->earth_radius == 0.0) return CHER_EINVAL;
    unsigned long long *scratch = nullptr;
    cher_status s = static_scratch(c->device, &scratch);
    if (s != CHER_OK) return s;

    const bool fp32 = prec == CHER_FP32_BULK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(out->count, 0, c->tel.size() * sizeof(unsigned long long), st) !=
            cudaSuccess ||
        cudaMemsetAsync(out->stats, 0, CHER_NSTATS * sizeof(unsigned long long), st) !=
            cudaSuccess)
        return CHER_ECUDA;
    cher::KParams p = base_params(c, t, seed, fp32);
    p.pos = out->pos;
    p.tim = out->tim;
    p.key = out->key;
    p.cap = out->cap_per_tel;
    p.count = out->count;
    p.stats = out->stats;
    const int block = (p.disp_k > 0 || p.earth_radius > 0.0) ? cher::kDispBlock : c->block;
    p.n_tiles = (p.n + block - 1) / block;
    if (p.n_tiles == 0) return CHER_OK;
    const size_t smem = cher::kernel_smem_bytes(fp32, block, p);
    const int kmode = cher::kernel_mode(cher::MODE_HITS, p) |
                      cher::occupancy_bits(fp32, block, c->ctas_per_sm);
    if (cher::kernel_prepare(fp32, block, kmode, smem) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ERANGE;
    }
    const int fit = cher::kernel_max_ctas_per_sm(fp32, block, kmode, smem);
    const int per_sm = std::max(1, std::min(c->ctas_per_sm > 0 ? c->ctas_per_sm : 1, fit));
    const int grid =
        static_cast<int>(std::min<int64_t>(p.n_tiles, int64_t(per_sm) * c->num_sms));
    // the array keeps the previous call's contents: clear the counter first
    k_clear_static_scratch<<<1, 32, 0, st>>>(static_cast<int>(need / sizeof(unsigned long long)));
    if (cudaGetLastError() != cudaSuccess) return CHER_ECUDA;
    p.tile_counter = scratch;
    if (cher::kernel_launch(fp32, block, kmode, grid, smem, p, stream) != cudaSuccess) {
        cudaGetLastError();
        return CHER_ECUDA;
    }
    return CHER_OK;
}
