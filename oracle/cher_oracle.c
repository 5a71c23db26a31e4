/*
 * cher_oracle.c -- plain, slow FP64 CPU oracle for Cherenkov photon-bunch
 * generation and propagation (Arrabito et al., "Optimizing Cherenkov photons
 * generation and propagation in CORSIKA for CTA Monte-Carlo simulations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * What it computes, in the order the paper describes it (Appendix A):
 *   per track step   : Cherenkov yield (CERENK, paper section 3.2), split
 *                      into sub-steps, one bunch of about five photons each;
 *   per bunch        : emission point, azimuth and wavelength from a
 *                      counter-based Philox4x32-10 stream keyed by
 *                      (seed, track, bunch), so every code version draws the
 *                      same random sequence (paper section 5.2);
 *                      refraction and propagation to the observation level
 *                      (RAYBND, paper section 3.2 and the Appendix B listing:
 *                      the horizontal direction is rescaled by
 *                      sin(theta_obs)/sin(theta_em), the vertical cosine is
 *                      recomputed from sin(theta_obs), the ground point moves
 *                      by the horizontal offset along the horizontal
 *                      direction and the travel time is added);
 *                      atmosphere lookups through uniform fine tables built
 *                      once (fast interpolation, paper section 3.3.2, 10000
 *                      points for the index of refraction);
 *                      the fiducial-sphere test of every telescope (paper
 *                      section 2: only photons crossing a sphere are kept).
 * The paper prints no formulas; the physics is textbook (Frank-Tamm yield,
 * Cherenkov angle cos(theta_c) = 1/(beta n), Snell's law in a flat layered
 * atmosphere) and every choice the paper leaves open is listed, as a
 * "reading", in the design notes of the repository.
 *
 * Two propagation variants:
 *   (T) table variant: refraction corrections interpolated bilinearly from
 *       tables over (height, squared sine of the observation zenith angle)
 *       that this file builds by numerical integration.  This is the parity
 *       reference.
 *   (B) brute-force variant: the ray integral itself, with no tables, used to
 *       pin (T) on tiny inputs.
 *
 * Floating point: FP64 throughout, compiled with -ffp-contract=off so that no
 * multiply-add is fused; the photon-yield chain and the index-of-refraction
 * table lookup are written one IEEE operation per statement because the
 * integer bunch count nb = ceil(N/B) depends on their exact rounding.
 *
 * Units: lengths in m, heights above sea level with z up, times in ns,
 * energies in MeV, wavelengths in nm.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------------- */
/* Physical constants (CODATA 2018 / SI definition)                         */
/* ----------------------------------------------------------------------- */
#define ORC_C_M_PER_NS 0.299792458       /* speed of light, m/ns (exact)     */
#define ORC_ME_MEV 0.51099895000         /* electron mass, MeV               */
#define ORC_ALPHA 7.2973525693e-3        /* fine-structure constant          */
#define ORC_PI 3.14159265358979323846

/* drop / status codes of a bunch (paper Alg. 1: the rare branches) */
#define ORC_ST_GROUND 0      /* reached the observation level               */
#define ORC_ST_UPWARD 1      /* photon direction not downward               */
#define ORC_ST_BELOW_OBS 2   /* emitted below the observation level         */
#define ORC_ST_ABOVE_MAX 3   /* emitted above the top of the tables         */
#define ORC_ST_ANGLE 4       /* zenith at the observation level > table max */
#define ORC_ST_ABSORBED 5    /* reached the ground level, then lost to the  */
                             /* atmospheric transmission draw              */

#define ORC_MAX_HITS 4       /* telescopes recorded per bunch               */
#define ORC_DISP_MAX 9       /* nodes of a wavelength-dependent index       */

/* Layered atmosphere: thickness T(h) = a_i + b_i exp(-h/c_i) in layer i,
 * h in [h_bound[i], h_bound[i+1]); density rho = -dT/dh; above h_bound[5]
 * there is no air.  n(h) - 1 = n0_minus_1 * rho(h) / rho(0). */
typedef struct {
    double h_bound[6];
    double a[5], b[5], c[5];
    double n0_minus_1;
} orc_atm;

/* Everything the per-bunch computation needs, set up by the caller. */
typedef struct {
    orc_atm atm;
    double h_obs;            /* observation level, m a.s.l.                */
    double h_max;            /* top of the tables, m a.s.l.                */
    /* fine table of eta = n - 1 on [0, h_max], n_fine points              */
    int n_fine;
    const double *eta_tab;
    /* refraction tables [H][Z]: h in [h_obs, h_max], sin^2 in [0, sin^2 tmax] */
    int H, Z;
    double theta_max;        /* rad                                        */
    const double *ax, *al;
    /* bunching and wavelength band                                        */
    double bunch_size;
    double lambda1_nm, lambda2_nm;
    /* telescopes: x, y, z (relative to h_obs), r                          */
    int n_tel;
    const double *tel;
    /* per-shower reference time (ns); NULL means zero                      */
    const double *t_ref;
    int n_showers;
    double bf_tol;           /* absolute tolerance of the (B) integrals    */
    uint32_t philox_key[2];  /* set from the seed by the entry points      */
    /* atmospheric transmission (NULL tau: off): vertical optical depth     */
    /* between height h and h_obs at wavelength lambda, on the uniform      */
    /* nodes lambda_a = l0 + a (l1 - l0)/(nl - 1), h_b = h0 + b (h1 - h0)/(nh - 1), */
    /* tau[a * nh + b]                                                      */
    int trans_nl, trans_nh;
    double trans_l0, trans_l1, trans_h0, trans_h1;
    const double *trans_tau;
    /* beyond-table fallback (0: off): bunches whose observation-level      */
    /* sin^2(zenith) exceeds the tables' range but not fb_sin2_max are      */
    /* propagated by the ray integrals themselves (variant (B))            */
    double fb_sin2_max;
    /* wavelength-dependent index (disp_k = 0: off):                       */
    /*   n(h, lambda) - 1 = eta(h) kappa(lambda),                           */
    /* kappa linear in the wavenumber 1/lambda between disp_k nodes, node m */
    /* at 1/lambda_m = 1/lambda1 - m (1/lambda1 - 1/lambda2)/(disp_k - 1),  */
    /* so node 0 is the short end of the band; kappa is positive and does   */
    /* not increase with m (normal dispersion).  The refraction tables are  */
    /* then (ax, al) for kappa[disp_k - 1] and (ax_hi, al_hi) for kappa[0], */
    /* interpolated linearly in kappa.                                      */
    int disp_k;
    const double *disp_kappa;
    const double *ax_hi, *al_hi;
    /* curved atmosphere (earth_radius = 0: flat layers).  Positions are   */
    /* Cartesian in the core frame (z up, z = height a.s.l. on the core's   */
    /* vertical); the Earth's centre is (0, 0, -earth_radius); a point's    */
    /* height is its radial height |x - C| - earth_radius; rays keep        */
    /* Bouguer's invariant n r sin(zeta) (zeta from the local vertical);   */
    /* the observation level is the sphere r_o = earth_radius + h_obs.  The */
    /* refraction tables are then the curved ones (orc_build_curved_tables). */
    double earth_radius;
    /* curved: the third table (the geometric part of the optical path),   */
    /* and its twin at kappa[0] with a wavelength-dependent index          */
    const double *ag, *ag_hi;
} orc_cfg;

typedef struct {
    const double *x0, *y0, *z0, *t0, *len, *ekin;
    const double *ux, *uy, *uz;
    const uint32_t *shower;  /* NULL: every track belongs to shower 0      */
    int64_t n;
    int64_t track_base;      /* global index of track 0 (Philox counter)   */
} orc_tracks;

/* One entry per bunch, indexed by bunch_off[i] + j. */
typedef struct {
    int32_t *status;
    double *xe, *ye, *he, *te;        /* emission point and time           */
    double *px, *py, *pz;             /* emission direction                */
    double *X, *Y, *t;                /* ground point and arrival time     */
    double *cx, *cy, *cz;             /* direction at the observation level */
    double *lam, *w;                  /* wavelength (nm), photons          */
    int32_t *nhit;                    /* telescopes crossed                */
    int32_t *hit_tel;                 /* [ORC_MAX_HITS] per bunch          */
    double *hit_x, *hit_y, *hit_t;    /* record in the telescope frame     */
    double *tr_margin;                /* u3 - P of the transmission draw (NaN */
                                      /* where none), optional              */
    double *Zg;                       /* arrival z - h_obs (curved), optional */
} orc_bunch_out;

/* ======================================================================= */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random      */
/* numbers: as easy as 1, 2, 3").  Each round multiplies counter words 0   */
/* and 2 by the two round multipliers, takes the 64-bit products apart and */
/* mixes the high halves with the other counter words and the key; the key */
/* is advanced by the two Weyl constants between rounds.                   */
/* ======================================================================= */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* n consecutive blocks for counters (lo(i), hi(i), j0 + m, 0), m < n, under
 * the key (lo(seed), hi(seed)): 4 n words into out. */
void orc_philox_fill(uint64_t seed, uint64_t i, uint32_t j0, int64_t n, uint32_t *out)
{
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    for (int64_t m = 0; m < n; ++m) {
        uint32_t ctr[4] = { (uint32_t)(i & 0xffffffffu), (uint32_t)(i >> 32),
                            j0 + (uint32_t)m, 0u };
        orc_philox4x32_10(ctr, key, out + 4 * m);
    }
}

/* A 32-bit word to a uniform deviate in (0, 1): (x + 1/2) / 2^32, exact. */
static double orc_u01(uint32_t x)
{
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

/* ======================================================================= */
/* Atmosphere (paper section 3.3.1: density, thickness and refractive index */
/* as functions of altitude)                                                */
/* ======================================================================= */
static int orc_layer(const orc_atm *A, double h)
{
    int i = 0;
    while (i < 4 && h >= A->h_bound[i + 1]) ++i;
    return i;
}

double orc_thickness(const orc_atm *A, double h)
{
    if (h >= A->h_bound[5]) return 0.0;
    int i = orc_layer(A, h);
    return A->a[i] + A->b[i] * exp(-(h / A->c[i]));
}

double orc_rho(const orc_atm *A, double h)
{
    if (h >= A->h_bound[5]) return 0.0;
    int i = orc_layer(A, h);
    double r = A->b[i] / A->c[i];
    double e = exp(-(h / A->c[i]));
    return r * e;
}

/* eta(h) = n(h) - 1 = n0_minus_1 * rho(h) / rho(0), from the formula. */
double orc_eta_exact(const orc_atm *A, double h)
{
    double rho0 = orc_rho(A, 0.0);
    double rho = orc_rho(A, h);
    double q = rho / rho0;
    return A->n0_minus_1 * q;
}

/* Fine table (fast interpolation, paper section 3.3.2): eta at the
 * n uniformly spaced heights h_k = k * dh, dh = h_max / (n - 1). */
int orc_build_eta_table(const orc_atm *A, double h_max, int n, double *tab)
{
    if (n < 2 || !(h_max > 0.0)) return -1;
    double dh = h_max / (double)(n - 1);
    for (int k = 0; k < n; ++k) {
        double h = (double)k * dh;
        tab[k] = orc_eta_exact(A, h);
    }
    return 0;
}

/* Lookup in the fine table: no search, index from the uniform step; the
 * height is clamped to [0, h_max].  One IEEE operation per statement. */
double orc_eta_lookup(const double *tab, int n, double h_max, double h)
{
    double dh = h_max / (double)(n - 1);
    double inv_dh = 1.0 / dh;
    double hc = h;
    if (hc < 0.0) hc = 0.0;
    if (hc > h_max) hc = h_max;
    double x = hc * inv_dh;
    int k = (int)x;
    if (k > n - 2) k = n - 2;
    double f = x - (double)k;
    double d = tab[k + 1] - tab[k];
    double fd = f * d;
    return tab[k] + fd;
}

/* ======================================================================= */
/* Per-step photon yield (CERENK, paper section 3.2 and Appendix A)         */
/* ======================================================================= */
/* Frank-Tamm for a singly charged particle with n independent of the
 * wavelength: dN/dL = 2 pi alpha sin^2(theta_c) (1/lambda1 - 1/lambda2).
 * sin^2(theta_c) = 1 - 1/(beta n)^2 is written without cancellation using
 * g = E_kin / m_e (gamma = 1 + g, beta^2 gamma^2 = g (2 + g)):
 *     sin^2 = [eta (2 + eta) gamma^2 - (1 + eta)^2] / [g (2 + g) (1 + eta)^2].
 * n is taken at the midpoint of the step.  nb = ceil(N / B) bunches share
 * the photons equally: w = N / nb. */
typedef struct {
    int64_t nb;
    double w, N, s2, beta, eta;
    /* with a wavelength-dependent index: gamma^2, beta^2 gamma^2, and per  */
    /* piece of the band its share of the yield (integral / piece width)    */
    /* and the radiating fraction of its width                              */
    double gam2, bg2, psum, x_th;
    double piece[ORC_DISP_MAX - 1], frac[ORC_DISP_MAX - 1];
} orc_yield;

static double orc_band_factor(const orc_cfg *C)
{
    /* 2 pi alpha (1/lambda1 - 1/lambda2), lambda in m */
    double two_pi_alpha = (2.0 * ORC_PI) * ORC_ALPHA;
    double inv1 = 1.0e9 / C->lambda1_nm;
    double inv2 = 1.0e9 / C->lambda2_nm;
    double dinv = inv1 - inv2;
    return two_pi_alpha * dinv;
}

static int orc_finite(double v) { return v == v && v - v == 0.0; }

/* Height of a point in a curved atmosphere: |x - C| - R_E with the centre
 * C = (0, 0, -R_E), written without cancellation:
 *     sqrt(rho^2 + (z + R_E)^2) - R_E = z + rho^2 / (sqrt(rho^2 + (z + R_E)^2) + z + R_E). */
static double orc_radial_height(double R_E, double x, double y, double z)
{
    double rho2 = x * x + y * y;
    double Rp = z + R_E;
    double r = sqrt(rho2 + Rp * Rp);
    double den = r + Rp;
    return z + rho2 / den;
}

/* The height at which a step's index is taken: its midpoint's (reading:
 * the radial height in a curved atmosphere).  One IEEE operation per
 * statement, like the rest of the yield. */
static double orc_midpoint_height(const orc_cfg *C, const orc_tracks *T, int64_t i)
{
    double half_len = 0.5 * T->len[i];
    double dz = half_len * T->uz[i];
    double hm = T->z0[i] + dz;
    if (C->earth_radius > 0.0) {
        double dx = half_len * T->ux[i];
        double xm = T->x0[i] + dx;
        double dy = half_len * T->uy[i];
        double ym = T->y0[i] + dy;
        double xx = xm * xm;
        double yy = ym * ym;
        double rho2 = xx + yy;
        double Rp = hm + C->earth_radius;
        double RR = Rp * Rp;
        double r2 = rho2 + RR;
        double r = sqrt(r2);
        double den = r + Rp;
        double corr = rho2 / den;
        hm = hm + corr;
    }
    return hm;
}

/* the yield of a step whose fields are all valid */
static int orc_step_yield_valid(const orc_cfg *C, double hm, double len, double ekin,
                                orc_yield *Y)
{
    double inv_me = 1.0 / ORC_ME_MEV;
    double K = orc_band_factor(C);
    double inv_B = 1.0 / C->bunch_size;

    double g = ekin * inv_me;               /* gamma - 1                   */
    double gam = 1.0 + g;
    double gam2 = gam * gam;
    double eta = orc_eta_lookup(C->eta_tab, C->n_fine, C->h_max, hm);
    double np1 = 1.0 + eta;
    double np1sq = np1 * np1;
    double two_eta = 2.0 + eta;
    double a = eta * two_eta;
    double b = a * gam2;
    double num = b - np1sq;                 /* gamma^2 ((beta n)^2 - 1)   */
    double two_g = 2.0 + g;
    double bg2 = g * two_g;                 /* beta^2 gamma^2              */
    double den = bg2 * np1sq;               /* gamma^2 (beta n)^2         */
    double s2 = num / den;
    Y->eta = eta;
    Y->beta = sqrt(bg2) / gam;
    if (!(s2 > 0.0)) return 0;              /* below threshold             */
    double Ks2 = K * s2;
    double N = len * Ks2;
    double q = N * inv_B;
    double nbd = ceil(q);
    Y->s2 = s2;
    Y->N = N;
    Y->nb = (int64_t)nbd;
    Y->w = (Y->nb > 0) ? N / nbd : 0.0;
    return 0;
}

/* Frank-Tamm with a wavelength-dependent index (an extension: the paper's
 * CERENK takes n independent of the wavelength).  Per unit path,
 *     dN/dL = 2 pi alpha int (1 - 1/(beta n(u))^2)_+ du,   u = 1/lambda.
 * On a piece of the band where n(u) = 1 + eta kappa(u) is linear in u the
 * integral has a closed form (the antiderivative of 1/(A + B u)^2 is
 * -1/(B (A + B u))):
 *     int_piece (1 - 1/(beta n)^2) du = width (1 - 1/(beta^2 n_a n_b)),
 * n_a, n_b the index at the ends, and with e = n_a n_b - 1 = e_a + e_b + e_a e_b
 * (e_a = eta kappa_a) the bracket is the cancellation-free
 *     [e gamma^2 - (1 + e)] / [g (2 + g) (1 + e)],
 * the constant-index sin^2 form with eta (2 + eta) replaced by e.  Only the
 * part of the band where beta n > 1 radiates, i.e. eta kappa > x_th with
 *     x_th = 1/beta - 1 = 1 / (gamma^2 beta (1 + beta));
 * kappa falls along the nodes, so at most one piece is cut: its radiating
 * part is the fraction (e_a - x_th) / (e_a - e_b) at its short-wavelength
 * end, where the index runs from n_a down to 1/beta (e_b replaced by x_th).
 *     N = L 2 pi alpha du sum_m frac_m S_m,  du = (1/lambda1 - 1/lambda2)/(k - 1),
 * and nb = ceil(N / B) as for the constant index. */
static double orc_disp_piece(double x, double y, double gam2, double bg2)
{
    double xy = x * y;
    double xpy = x + y;
    double e = xpy + xy;
    double np = 1.0 + e;
    double A = e * gam2;
    double num = A - np;
    double den = bg2 * np;
    double S = num / den;
    return (S > 0.0) ? S : 0.0;
}

static double orc_disp_band_factor(const orc_cfg *C)
{
    double two_pi_alpha = (2.0 * ORC_PI) * ORC_ALPHA;
    double inv1 = 1.0e9 / C->lambda1_nm;
    double inv2 = 1.0e9 / C->lambda2_nm;
    double dinv = inv1 - inv2;
    double du = dinv / (double)(C->disp_k - 1);
    return two_pi_alpha * du;
}

static int orc_step_yield_disp(const orc_cfg *C, double hm, double len, double ekin,
                               orc_yield *Y)
{
    double inv_me = 1.0 / ORC_ME_MEV;
    double Kd = orc_disp_band_factor(C);
    double inv_B = 1.0 / C->bunch_size;

    double g = ekin * inv_me;
    double gam = 1.0 + g;
    double gam2 = gam * gam;
    double eta = orc_eta_lookup(C->eta_tab, C->n_fine, C->h_max, hm);
    double two_g = 2.0 + g;
    double bg2 = g * two_g;
    double beta = sqrt(bg2) / gam;
    double onepb = 1.0 + beta;
    double gb = gam2 * beta;
    double gbb = gb * onepb;
    double x_th = 1.0 / gbb;
    Y->eta = eta;
    Y->beta = beta;
    Y->gam2 = gam2;
    Y->bg2 = bg2;
    Y->x_th = x_th;
    double sum = 0.0;
    for (int m = 0; m + 1 < C->disp_k; ++m) {
        double ea = eta * C->disp_kappa[m];
        double eb = eta * C->disp_kappa[m + 1];
        double frac = 0.0, S = 0.0;
        if (ea > x_th) {
            if (eb >= x_th) {
                frac = 1.0;
                S = orc_disp_piece(ea, eb, gam2, bg2);
            } else {
                double d1 = ea - x_th;
                double d2 = ea - eb;
                frac = d1 / d2;
                S = orc_disp_piece(ea, x_th, gam2, bg2);
            }
        }
        double v = frac * S;
        Y->frac[m] = frac;
        Y->piece[m] = v;
        sum = sum + v;
    }
    Y->psum = sum;
    if (!(sum > 0.0)) return 0;             /* below threshold everywhere  */
    double Ks = Kd * sum;
    double N = len * Ks;
    double q = N * inv_B;
    double nbd = ceil(q);
    Y->s2 = sum / (double)(C->disp_k - 1);  /* band-averaged sin^2         */
    Y->N = N;
    Y->nb = (int64_t)nbd;
    Y->w = (Y->nb > 0) ? N / nbd : 0.0;
    return 0;
}

/* A step is valid when every field is finite, its length is not negative
 * and its kinetic energy is positive; an invalid step emits nothing. */
static int orc_step_valid(const orc_tracks *T, int64_t i)
{
    return orc_finite(T->x0[i]) && orc_finite(T->y0[i]) && orc_finite(T->z0[i])
        && orc_finite(T->t0[i]) && orc_finite(T->len[i]) && orc_finite(T->ekin[i])
        && orc_finite(T->ux[i]) && orc_finite(T->uy[i]) && orc_finite(T->uz[i])
        && T->len[i] >= 0.0 && T->ekin[i] > 0.0;
}

/* returns 0 for a valid step, -1 for an invalid one (nb = 0 then) */
static int orc_step_yield(const orc_cfg *C, const orc_tracks *T, int64_t i, orc_yield *Y)
{
    Y->nb = 0; Y->w = 0.0; Y->N = 0.0; Y->s2 = 0.0; Y->beta = 0.0; Y->eta = 0.0;
    Y->psum = 0.0;
    if (!orc_step_valid(T, i)) return -1;
    double hm = orc_midpoint_height(C, T, i);
    if (C->disp_k > 0)
        return orc_step_yield_disp(C, hm, T->len[i], T->ekin[i], Y);
    return orc_step_yield_valid(C, hm, T->len[i], T->ekin[i], Y);
}

/* Per-step yield for every step: nb (bunches), w (photons per bunch),
 * s2 (sin^2 of the Cherenkov angle) and a validity flag (1 valid). */
void orc_segment_yield(const orc_cfg *C, const orc_tracks *T, int64_t *nb, double *w,
                       double *s2, int32_t *valid)
{
    for (int64_t i = 0; i < T->n; ++i) {
        orc_yield Y;
        int ok = orc_step_yield(C, T, i, &Y);
        nb[i] = Y.nb;
        if (w) w[i] = Y.w;
        if (s2) s2[i] = Y.s2;
        if (valid) valid[i] = (ok == 0);
    }
}

/* ======================================================================= */
/* Ray integrals in a flat layered atmosphere (RAYBND's refraction,        */
/* paper section 3.2).  With n(h) sin(theta(h)) = n_obs sin(theta_obs)     */
/* (Snell), a ray seen at zenith theta_obs at the observation level has    */
/*   horizontal displacement x(h) = int_{h_obs}^{h} tan(theta(h')) dh'     */
/*   optical path            l(h) = int_{h_obs}^{h} n(h') / cos(theta(h')) dh' */
/* The integrands are smooth inside a layer and jump at layer boundaries,   */
/* so every integral is split there and done by adaptive Simpson.          */
/* ======================================================================= */
typedef struct {
    const orc_atm *A;
    double np1_obs;   /* n at the observation level                        */
    double s_obs;     /* sin(theta_obs)                                    */
    double c_obs;     /* cos(theta_obs)                                    */
    int which;        /* integrand selector                                */
    double floor;     /* relative noise floor of the adaptive rule         */
} orc_ray;

enum { F_TAN = 0, F_OPT = 1, F_TAN_CORR = 2, F_OPT_CORR = 3, F_RATIO = 4 };

static double orc_integrand(const orc_ray *R, double h)
{
    double eta = orc_eta_exact(R->A, h);
    double np1 = 1.0 + eta;
    double s = R->np1_obs * R->s_obs / np1;
    double c = sqrt(1.0 - s * s);
    switch (R->which) {
    case F_TAN: return s / c;
    case F_OPT: return np1 / c;
    case F_TAN_CORR: return s / c - R->s_obs / R->c_obs;
    case F_OPT_CORR: return np1 / c - 1.0 / R->c_obs;
    case F_RATIO: return R->np1_obs / np1 - 1.0;
    }
    return 0.0;
}

/* Adaptive Simpson stops refining once the two estimates agree to the
 * rounding noise of the integrand: the correction integrands of the tables
 * (tan - tan_o) are differences of terms up to ~1/cos^3 larger, whose
 * rounding at large zenith reaches ~1e-10 of the correction (80 degrees);
 * a tolerance halved below that recurses towards the depth limit without
 * gaining anything.  The floor, `rel` of the integrand's size over the
 * interval (1e-9 for the tables' corrections, 1e-13 for the full integrands
 * of the brute-force variant), changes an integral by at most `rel` of its
 * size. */
static double orc_noise_floor(double rel, double a, double b, double fa, double fm, double fb)
{
    return rel * (fabs(fa) + fabs(fm) + fabs(fb)) * (b - a);
}

static double orc_simpson_rec(const orc_ray *R, double a, double b, double fa,
                              double fm, double fb, double whole, double tol,
                              int depth)
{
    double m = 0.5 * (a + b);
    double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = orc_integrand(R, lm), frm = orc_integrand(R, rm);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double delta = left + right - whole;
    if (depth <= 0 || fabs(delta) <= 15.0 * tol || fabs(delta) <= orc_noise_floor(R->floor, a, b, fa, fm, fb))
        return left + right + delta / 15.0;
    return orc_simpson_rec(R, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1)
         + orc_simpson_rec(R, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

static double orc_simpson(const orc_ray *R, double a, double b, double tol)
{
    if (b <= a) return 0.0;
    double fa = orc_integrand(R, a), fb = orc_integrand(R, b);
    double m = 0.5 * (a + b), fm = orc_integrand(R, m);
    double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
    return orc_simpson_rec(R, a, b, fa, fm, fb, whole, tol, 48);
}

/* integral over [lo, hi] split at the layer boundaries inside it */
static double orc_integrate(const orc_ray *R, double lo, double hi, double tol)
{
    double sum = 0.0, a = lo;
    for (int i = 1; i <= 5; ++i) {
        double hb = R->A->h_bound[i];
        if (hb > a && hb < hi) {
            sum += orc_simpson(R, a, hb, tol);
            a = hb;
        }
    }
    sum += orc_simpson(R, a, hi, tol);
    return sum;
}

/* (B): x and l of the ray that arrives at zenith asin(sin_obs), from the
 * observation level up to h_e, with the exact n(h). */
int orc_brute_ray(const orc_atm *A, double h_obs, double h_e, double sin_obs,
                  double tol, double *x_out, double *l_out)
{
    if (!(sin_obs >= 0.0 && sin_obs < 1.0) || h_e < h_obs) return -1;
    orc_ray R;
    R.A = A;
    R.floor = 1e-13;
    R.np1_obs = 1.0 + orc_eta_exact(A, h_obs);
    R.s_obs = sin_obs;
    R.c_obs = sqrt(1.0 - sin_obs * sin_obs);
    R.which = F_TAN;
    *x_out = orc_integrate(&R, h_obs, h_e, tol);
    R.which = F_OPT;
    *l_out = orc_integrate(&R, h_obs, h_e, tol);
    return 0;
}

/* Refraction tables over heights h_j = h_obs + j dht (j < H, dht =
 * (h_max - h_obs)/(H-1)) and observation-level zeniths theta_k whose squared
 * sines are uniform: sin^2(theta_k) = k dq (k < Z, dq = sin^2(theta_max)/(Z-1)).
 * They hold the corrections to the straight line at theta_k,
 *     dx = x(h_j) - (h_j - h_obs) tan(theta_k),
 *     dl = l(h_j) - (h_j - h_obs) / cos(theta_k),
 * divided by their leading angular dependence so that interpolation stays
 * accurate at large zenith angles (to first order in n - 1, ax does not
 * depend on the angle and al is linear in sin^2(theta)):
 *     ax[j][k] = dx cos^3(theta_k) / sin(theta_k)   (k > 0),
 *     ax[j][0] = int (n_obs / n(h') - 1) dh'         (the limit theta -> 0),
 *     al[j][k] = dl cos^3(theta_k).
 * Each column is accumulated interval by interval. */
int orc_build_refraction_tables(const orc_atm *A, double h_obs, double h_max,
                                int H, int Z, double theta_max, double tol,
                                double *ax, double *al)
{
    if (H < 2 || Z < 2 || !(h_max > h_obs) || !(theta_max > 0.0)
        || !(theta_max < 0.5 * ORC_PI))
        return -1;
    double dht = (h_max - h_obs) / (double)(H - 1);
    double smax = sin(theta_max);
    double dq = smax * smax / (double)(Z - 1);
    double np1_obs = 1.0 + orc_eta_exact(A, h_obs);
    for (int k = 0; k < Z; ++k) {
        double q = (double)k * dq;
        double so = sqrt(q), co = sqrt(1.0 - so * so);
        orc_ray R;
        R.A = A; R.np1_obs = np1_obs; R.s_obs = so; R.c_obs = co;
        R.floor = 1e-9;
        double dx = 0.0, dl = 0.0;
        ax[(size_t)0 * Z + k] = 0.0;
        al[(size_t)0 * Z + k] = 0.0;
        for (int j = 1; j < H; ++j) {
            double lo = h_obs + (double)(j - 1) * dht;
            double hi = h_obs + (double)j * dht;
            R.which = (k == 0) ? F_RATIO : F_TAN_CORR;
            dx += orc_integrate(&R, lo, hi, tol);
            R.which = F_OPT_CORR;
            dl += orc_integrate(&R, lo, hi, tol);
            double c3 = co * co * co;
            ax[(size_t)j * Z + k] = (k == 0) ? dx : dx * c3 / so;
            al[(size_t)j * Z + k] = dl * c3;
        }
    }
    return 0;
}

/* ======================================================================= */
/* Curved atmosphere (an extension: the flat layers of RAYBND become       */
/* spherical shells, for large zenith angles).  A ray in a spherically     */
/* stratified medium stays in the plane through the Earth's centre and     */
/* keeps Bouguer's invariant n(r) r sin(zeta(r)) = K, zeta the angle to the */
/* local vertical.  Between the observation sphere r_o and the emission    */
/* radius r_e it turns through the central angle and has the optical path  */
/*     phi = int tan(zeta) / r dr,   L = int n / cos(zeta) dr,             */
/* r = R_E + h, integrated over h layer by layer (adaptive Simpson).       */
/* The tables hold corrections to the straight line that arrives at the    */
/* same zenith (impact parameter b = r_o sin(zeta_o), sin(zeta_s) = b / r): */
/*     dphi = int (tan(zeta) - tan(zeta_s)) / r dr,                        */
/*     L - l_s = int (n - 1) / cos(zeta) dr + int (1/cos(zeta) - 1/cos(zeta_s)) dr, */
/* three quantities, each divided by the path average along that line of   */
/* its first-order angular factor (b r_o / (r^2 cos^3), 1 / cos and        */
/* sin^2 / cos^3 of zeta_s), all closed forms (orc_curved_factors), so that */
/* to first order in n - 1 each table is the path average of n_o / n - 1,  */
/* n - 1 or n_o / n - 1: nearly independent of the angle.  The zenith axis */
/* is uniform in sec(zeta_o) from 1 to sec(theta_max): what the path       */
/* averages leave (the weights n - 1 are not uniform along a path whose    */
/* zenith changes, by ~2 sin^2 h / r_o in cos^2) varies near grazing like  */
/* 1 / cos^2, far from linear in sin^2 but near linear in sec.  For        */
/* R_E -> infinity the three factors become tan / cos^2, 1 / cos and       */
/* sin^2 / cos^3, the flat tables' normalisation.                          */
/* ======================================================================= */
typedef struct {
    const orc_atm *A;
    double R_E, K, b, no_ro;   /* invariant, reference impact parameter, n_o r_o */
    double r_o;
    int which;
    double floor;
} orc_cray;

enum { C_PHI = 0, C_OPT = 1, C_PHI_CORR = 2, C_OPT_N1 = 3, C_OPT_GEO = 4, C_RATIO = 5,
       C_RATIO_GEO = 6 };

static double orc_cintegrand(const orc_cray *R, double h)
{
    double r = R->R_E + h;
    double n = 1.0 + orc_eta_exact(R->A, h);
    double s = R->K / (n * r);
    double c = sqrt(1.0 - s * s);
    double ss = R->b / r;
    double cs = sqrt(1.0 - ss * ss);
    switch (R->which) {
    /* the central-angle integrands carry a factor r_o (metres of arc at the
     * observation level), so that the absolute tolerance means the same as
     * for the flat tables */
    case C_PHI: return s / c * (R->r_o / r);
    case C_OPT: return n / c;
    case C_PHI_CORR: return (s / c - ss / cs) * (R->r_o / r);
    case C_OPT_N1: return (n - 1.0) / c;
    case C_OPT_GEO: return (s * s - ss * ss) / (c * cs * (c + cs));   /* 1/c - 1/cs */
    case C_RATIO: return (R->no_ro / (n * r) - R->r_o / r) * R->r_o / r;
    case C_RATIO_GEO: {                       /* small-angle limit of C_OPT_GEO / sin^2 */
        double v = R->no_ro / (n * R->r_o);   /* n_o / n */
        return 0.5 * (v * v - 1.0) * (R->r_o / r) * (R->r_o / r);
    }
    }
    return 0.0;
}

static double orc_csimpson_rec(const orc_cray *R, double a, double b, double fa, double fm,
                               double fb, double whole, double tol, int depth)
{
    double m = 0.5 * (a + b);
    double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = orc_cintegrand(R, lm), frm = orc_cintegrand(R, rm);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double delta = left + right - whole;
    if (depth <= 0 || fabs(delta) <= 15.0 * tol || fabs(delta) <= orc_noise_floor(R->floor, a, b, fa, fm, fb))
        return left + right + delta / 15.0;
    return orc_csimpson_rec(R, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1)
         + orc_csimpson_rec(R, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1);
}

static double orc_cintegrate(const orc_cray *R, double lo, double hi, double tol)
{
    double sum = 0.0, a = lo;
    for (int i = 1; i <= 5; ++i) {
        double hb = R->A->h_bound[i];
        if (hb > a && hb < hi) {
            double fa = orc_cintegrand(R, a), fb = orc_cintegrand(R, hb);
            double m = 0.5 * (a + hb), fm = orc_cintegrand(R, m);
            sum += orc_csimpson_rec(R, a, hb, fa, fm, fb, (hb - a) / 6.0 * (fa + 4.0 * fm + fb),
                                    tol, 48);
            a = hb;
        }
    }
    if (hi > a) {
        double fa = orc_cintegrand(R, a), fb = orc_cintegrand(R, hi);
        double m = 0.5 * (a + hi), fm = orc_cintegrand(R, m);
        sum += orc_csimpson_rec(R, a, hi, fa, fm, fb, (hi - a) / 6.0 * (fa + 4.0 * fm + fb),
                                tol, 48);
    }
    return sum;
}

/* The path averages, along the straight line that arrives at the
 * observation sphere (radius r_o) with sine s_o, between r_o and r_e
 * (dH = r_e - r_o), of b r_o / (r^2 cos^3), 1 / cos and sin^2 / cos^3 of
 * its zenith (u = r_o / r_e, c_e' its cosine at r_e, c_o at r_o):
 *     G_phi = r_o (tan(zeta_o) - tan(zeta_e')) / dH
 *           = r_o s_o (1 + u) / (r_e (c_e' + u c_o) c_o c_e'),
 *     G_1   = (r_e c_e' - r_o c_o) / dH = (r_e + r_o) / (r_e c_e' + r_o c_o),
 *     G_2   = G_1 s_o^2 u / (c_e' c_o)
 * (from d tan/dr = -b / (r^2 cos^3), d (r cos)/dr = 1 / cos and
 * d (r (1 - 2 sin^2) / cos)/dr = 1 / cos^3, written without cancellation;
 * G_2 vanishes with s_o like s_o^2). */
static void orc_curved_factors(double r_o, double r_e, double s_o, double *g_phi,
                               double *g_1, double *g_2)
{
    double u = r_o / r_e;
    double c_o = sqrt(1.0 - s_o * s_o);
    double se = s_o * u;
    double ce = sqrt(1.0 - se * se);
    *g_phi = r_o * s_o * (1.0 + u) / (r_e * (ce + u * c_o) * c_o * ce);
    *g_1 = (r_e + r_o) / (r_e * ce + r_o * c_o);
    *g_2 = *g_1 * s_o * s_o * u / (ce * c_o);
}

/* (B), curved: central angle phi and optical path L of the ray that arrives
 * at the observation sphere at local zenith asin(sin_obs), up to h_e. */
int orc_brute_ray_curved(const orc_atm *A, double R_E, double h_obs, double h_e,
                         double sin_obs, double tol, double *phi_out, double *l_out)
{
    if (!(sin_obs >= 0.0 && sin_obs < 1.0) || h_e < h_obs || !(R_E > 0.0)) return -1;
    orc_cray R;
    R.A = A;
    R.floor = 1e-13;
    R.R_E = R_E;
    R.r_o = R_E + h_obs;
    R.no_ro = (1.0 + orc_eta_exact(A, h_obs)) * R.r_o;
    R.K = R.no_ro * sin_obs;
    R.b = R.r_o * sin_obs;
    R.which = C_PHI;
    *phi_out = orc_cintegrate(&R, h_obs, h_e, tol) / R.r_o;
    R.which = C_OPT;
    *l_out = orc_cintegrate(&R, h_obs, h_e, tol);
    return 0;
}

/* Curved tables over heights h_j (as the flat ones) and observation-level
 * zeniths with sec(zeta_k) = 1 + k dsec, dsec = (sec(theta_max) - 1)/(Z-1),
 * accumulated interval by interval. */
int orc_build_curved_tables(const orc_atm *A, double R_E, double h_obs, double h_max,
                            int H, int Z, double theta_max, double tol, double *ax,
                            double *al, double *ag)
{
    if (H < 2 || Z < 2 || !(h_max > h_obs) || !(theta_max > 0.0)
        || !(theta_max < 0.5 * ORC_PI) || !(R_E > 0.0))
        return -1;
    double dht = (h_max - h_obs) / (double)(H - 1);
    double dsec = (1.0 / cos(theta_max) - 1.0) / (double)(Z - 1);
    double r_o = R_E + h_obs;
    double no_ro = (1.0 + orc_eta_exact(A, h_obs)) * r_o;
    for (int k = 0; k < Z; ++k) {
        double co = 1.0 / (1.0 + (double)k * dsec);
        double so = sqrt((1.0 - co) * (1.0 + co));
        orc_cray R;
        R.A = A; R.R_E = R_E; R.r_o = r_o; R.no_ro = no_ro;
        R.floor = 1e-9;
        R.K = no_ro * so; R.b = r_o * so;
        double dphi = 0.0, d1 = 0.0, d2 = 0.0;
        ax[(size_t)0 * Z + k] = 0.0;
        al[(size_t)0 * Z + k] = 0.0;
        ag[(size_t)0 * Z + k] = 0.0;
        for (int j = 1; j < H; ++j) {
            double lo = h_obs + (double)(j - 1) * dht;
            double hi = h_obs + (double)j * dht;
            R.which = (k == 0) ? C_RATIO : C_PHI_CORR;
            dphi += orc_cintegrate(&R, lo, hi, tol);
            R.which = C_OPT_N1;
            d1 += orc_cintegrate(&R, lo, hi, tol);
            R.which = (k == 0) ? C_RATIO_GEO : C_OPT_GEO;
            d2 += orc_cintegrate(&R, lo, hi, tol);
            double r_e = R_E + hi;
            double g_phi, g_1, g_2;
            orc_curved_factors(r_o, r_e, so, &g_phi, &g_1, &g_2);
            /* dphi carries r_o; at k = 0 the small-angle limits' integrals,
             * divided by G_phi / s_o -> r_o / r_e and G_2 / s_o^2 -> r_o / r_e */
            ax[(size_t)j * Z + k] = (k == 0) ? dphi * (r_e / r_o) : dphi / g_phi;
            al[(size_t)j * Z + k] = d1 / g_1;
            ag[(size_t)j * Z + k] = (k == 0) ? d2 * (r_e / r_o) : d2 / g_2;
        }
    }
    return 0;
}

/* bilinear interpolation in a [H][Z] table at fractional indices */
static double orc_bilinear(const double *T, int Z, int j, int k, double a, double b)
{
    double t00 = T[(size_t)j * Z + k], t01 = T[(size_t)j * Z + k + 1];
    double t10 = T[(size_t)(j + 1) * Z + k], t11 = T[(size_t)(j + 1) * Z + k + 1];
    double v0 = t00 + a * (t10 - t00);
    double v1 = t01 + a * (t11 - t01);
    return v0 + b * (v1 - v0);
}

/* ======================================================================= */
/* Propagation of one photon bunch to the observation level (RAYBND).      */
/* variant 0 = (T) tables, 1 = (B) brute force.  kappa scales n - 1 at the */
/* bunch's wavelength (1 for a wavelength-independent index).               */
/* out: X, Y, t, cx, cy, cz of the arrival, its z relative to h_obs (0 in  */
/* flat layers), the cosine of its zenith to the local vertical, and the   */
/* emission height.  Returns the status code.                               */
/* ======================================================================= */
static int orc_propagate_curved(const orc_cfg *C, int variant, double kappa, double xe,
                                double ye, double ze, double te, double px, double py,
                                double pz, double *out);

int orc_propagate_photon_k(const orc_cfg *C, int variant, double kappa, double xe,
                           double ye, double he, double te, double px, double py,
                           double pz, double *out)
{
    if (C->earth_radius > 0.0)
        return orc_propagate_curved(C, variant, kappa, xe, ye, he, te, px, py, pz, out);
    out[6] = 0.0;
    out[8] = he;
    /* rare conditions first (paper Alg. 2), each a counted drop */
    if (pz >= 0.0) return ORC_ST_UPWARD;
    if (he < C->h_obs) return ORC_ST_BELOW_OBS;
    if (he > C->h_max) return ORC_ST_ABOVE_MAX;

    double sin_em = sqrt(px * px + py * py);
    double eta_e, eta_o;
    if (variant == 0) {
        eta_e = orc_eta_lookup(C->eta_tab, C->n_fine, C->h_max, he);
        eta_o = orc_eta_lookup(C->eta_tab, C->n_fine, C->h_max, C->h_obs);
    } else {
        eta_e = orc_eta_exact(&C->atm, he);
        eta_o = orc_eta_exact(&C->atm, C->h_obs);
    }
    eta_e = kappa * eta_e;
    eta_o = kappa * eta_o;
    /* the atmosphere at this wavelength, for the ray integrals */
    orc_atm Ak = C->atm;
    Ak.n0_minus_1 = kappa * C->atm.n0_minus_1;
    /* Snell in flat layers: n(h_e) sin(theta_em) = n_obs sin(theta_obs) */
    double sin_obs = sin_em * (1.0 + eta_e) / (1.0 + eta_o);
    double q = sin_obs * sin_obs;
    double smax = sin(C->theta_max);
    double q_max = smax * smax;
    /* the paper's rare-case fallback (section 3.3.1: the few photons that do
     * not fit the vectorised path take the scalar code): beyond the tables'
     * zenith range, up to fb_sin2_max, the ray integrals themselves */
    int fallback = 0;
    if (q > q_max) {
        if (!(C->fb_sin2_max > 0.0) || !(q <= C->fb_sin2_max)) return ORC_ST_ANGLE;
        fallback = 1;
    }
    double cos_obs = sqrt(1.0 - q);
    double dH = he - C->h_obs;

    double hx = 0.0, hy = 0.0;        /* horizontal unit direction        */
    if (sin_em > 0.0) { hx = px / sin_em; hy = py / sin_em; }

    double D, L;                      /* horizontal offset, optical path  */
    if (variant == 0 && !fallback) {
        double dht = (C->h_max - C->h_obs) / (double)(C->H - 1);
        double dq = q_max / (double)(C->Z - 1);
        double fj = dH / dht;
        int j = (int)fj;
        if (j > C->H - 2) j = C->H - 2;
        double a = fj - (double)j;
        double fk = q / dq;
        int k = (int)fk;
        if (k > C->Z - 2) k = C->Z - 2;
        double b = fk - (double)k;
        double Ax = orc_bilinear(C->ax, C->Z, j, k, a, b);
        double Al = orc_bilinear(C->al, C->Z, j, k, a, b);
        if (C->disp_k > 0) {
            /* linear in kappa between the tables of the band's two ends */
            double k_lo = C->disp_kappa[C->disp_k - 1], k_hi = C->disp_kappa[0];
            double wk = (k_hi > k_lo) ? (kappa - k_lo) / (k_hi - k_lo) : 0.0;
            double Bx = orc_bilinear(C->ax_hi, C->Z, j, k, a, b);
            double Bl = orc_bilinear(C->al_hi, C->Z, j, k, a, b);
            Ax = Ax + wk * (Bx - Ax);
            Al = Al + wk * (Bl - Al);
        }
        /* dx = Ax tan sec^2, dl = Al sec^3 (see the table definition) */
        double sec = 1.0 / cos_obs;
        double tn = sin_obs * sec;
        double sec2 = sec * sec;
        D = dH * tn + Ax * tn * sec2;
        L = dH * sec + Al * sec2 * sec;
    } else {
        if (orc_brute_ray(&Ak, C->h_obs, he, sin_obs, C->bf_tol, &D, &L) != 0)
            return ORC_ST_ANGLE;
    }
    out[0] = xe + D * hx;
    out[1] = ye + D * hy;
    out[2] = te + L / ORC_C_M_PER_NS;
    out[3] = sin_obs * hx;
    out[4] = sin_obs * hy;
    out[5] = -cos_obs;
    out[7] = cos_obs;
    return ORC_ST_GROUND;
}

/* Curved: the emission point's radial height and local vertical r^ (from
 * the Earth's centre); cos and sin of the photon's angle to it (the sine as
 * |p x r^|, exact at small angles); Bouguer's invariant for the arrival
 * zenith, sin(zeta_o) = n_e r_e sin(zeta_e) / (n_o r_o); the central angle
 * and optical path from the tables (corrections to the straight line of the
 * same arrival zenith, whose central angle and length are closed forms) or
 * from the integrals; then the arrival point
 *     x_e + (r_o cos(phi) - r_e) r^ + r_o sin(phi) t^,
 * t^ the horizontal direction of travel at the emission point, and the
 * arrival direction -cos(zeta_o) r^_o + sin(zeta_o) t^_o in the rotated
 * frame.  The same rare conditions, with radial heights and the outward
 * cosine for "upward". */
static int orc_propagate_curved(const orc_cfg *C, int variant, double kappa, double xe,
                                double ye, double ze, double te, double px, double py,
                                double pz, double *out)
{
    double R_E = C->earth_radius;
    double Rp = ze + R_E;
    double rho2 = xe * xe + ye * ye;
    double r_e = sqrt(rho2 + Rp * Rp);
    double he = ze + rho2 / (r_e + Rp);
    out[8] = he;
    double rx = xe / r_e, ry = ye / r_e, rz = Rp / r_e;
    double ce = px * rx + py * ry + pz * rz;          /* cosine to the upward vertical */
    if (ce >= 0.0) return ORC_ST_UPWARD;
    if (he < C->h_obs) return ORC_ST_BELOW_OBS;
    if (he > C->h_max) return ORC_ST_ABOVE_MAX;
    double wx = py * rz - pz * ry, wy = pz * rx - px * rz, wz = px * ry - py * rx;
    double se = sqrt(wx * wx + wy * wy + wz * wz);
    double eta_e, eta_o;
    if (variant == 0) {
        eta_e = orc_eta_lookup(C->eta_tab, C->n_fine, C->h_max, he);
        eta_o = orc_eta_lookup(C->eta_tab, C->n_fine, C->h_max, C->h_obs);
    } else {
        eta_e = orc_eta_exact(&C->atm, he);
        eta_o = orc_eta_exact(&C->atm, C->h_obs);
    }
    eta_e = kappa * eta_e;
    eta_o = kappa * eta_o;
    orc_atm Ak = C->atm;
    Ak.n0_minus_1 = kappa * C->atm.n0_minus_1;
    double r_o = R_E + C->h_obs;
    double dH = he - C->h_obs;
    double s_o = se * (r_e / r_o) * ((1.0 + eta_e) / (1.0 + eta_o));
    double q = s_o * s_o;
    double smax = sin(C->theta_max);
    double q_max = smax * smax;
    int fallback = 0;
    if (q > q_max) {
        if (!(C->fb_sin2_max > 0.0) || !(q <= C->fb_sin2_max)) return ORC_ST_ANGLE;
        fallback = 1;
    }
    double c_o = sqrt(1.0 - q);
    double sphi, cphi, L;
    if (variant == 0 && !fallback) {
        double dht = (C->h_max - C->h_obs) / (double)(C->H - 1);
        double dsec = (1.0 / cos(C->theta_max) - 1.0) / (double)(C->Z - 1);
        double fj = dH / dht;
        int j = (int)fj;
        if (j > C->H - 2) j = C->H - 2;
        double a = fj - (double)j;
        double fk = (1.0 / c_o - 1.0) / dsec;
        int k = (int)fk;
        if (k > C->Z - 2) k = C->Z - 2;
        double b = fk - (double)k;
        double Ax = orc_bilinear(C->ax, C->Z, j, k, a, b);
        double A1 = orc_bilinear(C->al, C->Z, j, k, a, b);
        double A2 = orc_bilinear(C->ag, C->Z, j, k, a, b);
        if (C->disp_k > 0) {
            double k_lo = C->disp_kappa[C->disp_k - 1], k_hi = C->disp_kappa[0];
            double wk = (k_hi > k_lo) ? (kappa - k_lo) / (k_hi - k_lo) : 0.0;
            Ax = Ax + wk * (orc_bilinear(C->ax_hi, C->Z, j, k, a, b) - Ax);
            A1 = A1 + wk * (orc_bilinear(C->al_hi, C->Z, j, k, a, b) - A1);
            A2 = A2 + wk * (orc_bilinear(C->ag_hi, C->Z, j, k, a, b) - A2);
        }
        double g_phi, g_1, g_2;
        orc_curved_factors(r_o, r_e, s_o, &g_phi, &g_1, &g_2);
        double dphi = Ax * g_phi / r_o;
        double dL = A1 * g_1 + A2 * g_2;
        /* the straight line arriving at zeta_o: at r_e its angle to the
         * vertical has sine s_o u, u = r_o / r_e; it turns through
         * sin(phi_s) = s_o (1 - u^2) / (cos_e' + c_o u) and is
         * dH (r_e + r_o) / (r_e cos_e' + r_o c_o) long */
        double u = r_o / r_e;
        double se2 = s_o * u;
        double ce2 = sqrt(1.0 - se2 * se2);
        double omu2 = (dH / r_e) * (1.0 + u);
        double sps = s_o * omu2 / (ce2 + c_o * u);
        double cps = ce2 * c_o + se2 * s_o;
        double lref = dH * (r_e + r_o) / (r_e * ce2 + r_o * c_o);
        sphi = sps * cos(dphi) + cps * sin(dphi);
        cphi = cps * cos(dphi) - sps * sin(dphi);
        L = lref + dL;
    } else {
        double phi;
        if (orc_brute_ray_curved(&Ak, R_E, C->h_obs, he, s_o, C->bf_tol, &phi, &L) != 0)
            return ORC_ST_ANGLE;
        sphi = sin(phi);
        cphi = cos(phi);
    }
    double tx = 0.0, ty = 0.0, tz = 0.0;              /* horizontal direction of travel */
    if (se > 0.0) {
        tx = (px - ce * rx) / se;
        ty = (py - ce * ry) / se;
        tz = (pz - ce * rz) / se;
    }
    double omc = sphi * sphi / (1.0 + cphi);          /* 1 - cos(phi) */
    double dr = -dH - r_o * omc;                      /* r_o cos(phi) - r_e */
    double dtn = r_o * sphi;
    out[0] = xe + (dr * rx + dtn * tx);
    out[1] = ye + (dr * ry + dtn * ty);
    out[6] = (ze - C->h_obs) + (dr * rz + dtn * tz);
    out[2] = te + L / ORC_C_M_PER_NS;
    double rox = cphi * rx + sphi * tx, roy = cphi * ry + sphi * ty, roz = cphi * rz + sphi * tz;
    double tox = cphi * tx - sphi * rx, toy = cphi * ty - sphi * ry, toz = cphi * tz - sphi * rz;
    out[3] = -c_o * rox + s_o * tox;
    out[4] = -c_o * roy + s_o * toy;
    out[5] = -c_o * roz + s_o * toz;
    out[7] = c_o;
    return ORC_ST_GROUND;
}

int orc_propagate_photon(const orc_cfg *C, int variant, double xe, double ye,
                         double he, double te, double px, double py, double pz,
                         double *out)
{
    return orc_propagate_photon_k(C, variant, 1.0, xe, ye, he, te, px, py, pz, out);
}

/* ======================================================================= */
/* Fiducial telescope spheres (TELOUT, paper sections 2 and Appendix A).    */
/* The line through the ground point along the arrival direction crosses   */
/* sphere k iff |(C_k - P0) x D|^2 <= R_k^2 (inclusive).  The record is    */
/* taken where the line crosses the horizontal plane through the centre,   */
/* relative to the centre; its time moves at c/n_obs along the line.       */
/* ======================================================================= */
static int orc_telescopes(const orc_cfg *C, double X, double Y, double Zg, double t,
                          double cx, double cy, double cz, double np1_obs,
                          int32_t *tel, double *rx, double *ry, double *rt)
{
    int nh = 0;
    for (int k = 0; k < C->n_tel; ++k) {
        double tx = C->tel[4 * k + 0], ty = C->tel[4 * k + 1];
        double tz = C->tel[4 * k + 2], tr = C->tel[4 * k + 3];
        double dx = tx - X, dy = ty - Y, dz = tz - Zg;
        double q0 = dy * cz - dz * cy;
        double q1 = dz * cx - dx * cz;
        double q2 = dx * cy - dy * cx;
        double d2 = q0 * q0 + q1 * q1 + q2 * q2;
        if (d2 <= tr * tr) {
            if (nh < ORC_MAX_HITS) {
                double s = dz / cz;
                tel[nh] = k;
                rx[nh] = X + s * cx - tx;
                ry[nh] = Y + s * cy - ty;
                rt[nh] = t + s * np1_obs / ORC_C_M_PER_NS;
            }
            ++nh;
        }
    }
    return nh;
}

/* ======================================================================= */
/* One bunch: emission (a2) and propagation (a3) of bunch j of step i,      */
/* given the step's yield and the bunch count in use.                       */
/* ======================================================================= */
typedef struct {
    int status;
    double xe, ye, he, te, px, py, pz, lam;
    double r[9];                      /* X, Y, t (before t_ref), cx, cy, cz, */
                                      /* z - h_obs, local cos, emission height */
    double tr_margin;                 /* u3 - P of the transmission draw, or NaN */
    double kappa;                     /* (n - 1) scale at the bunch's wavelength */
} orc_bunch1;

/* The wavelength of a bunch under a wavelength-dependent index, from the
 * step's spectrum (density 1 - 1/(beta n(u))^2 in u = 1/lambda over the
 * radiating part of the band) by inversion of the deviate u2, counted from
 * the short end of the band like the constant-index inversion: the piece m
 * whose cumulative share first exceeds u2 * psum, then inside it the
 * fraction t of its radiating width where
 *     G(t) = t - t / (beta^2 n_a n(t)),  n(t) = n_a + b t,  b = n_end - n_a
 * (the density's integral over [0, t] in units of that width) equals the
 * remaining share D' = D / frac.  That is the quadratic
 *     b t^2 + (n_a s_a^2 - D' b) t - D' n_a = 0,  s_a^2 = 1 - 1/(beta n_a)^2,
 * whose root in [0, 1] is taken as t = 2 D' n_a / (P + sqrt(P^2 + 4 b D' n_a)),
 * P = n_a s_a^2 - D' b (b <= 0, so P >= 0 and nothing cancels).  kappa and
 * the wavenumber follow linearly; the Cherenkov angle is that of the
 * bunch's index at the step midpoint: cos = 1/(beta n), sin^2 in the
 * cancellation-free form. */
static void orc_disp_sample(const orc_cfg *C, const orc_yield *Y, double u2, double *lam,
                            double *kap, double *cos_c, double *sin_c)
{
    int K = C->disp_k;
    double T = u2 * Y->psum;
    int m = 0;
    double acc = 0.0;
    while (m < K - 2) {
        double nxt = acc + Y->piece[m];
        if (T < nxt) break;
        acc = nxt;
        ++m;
    }
    double eta = Y->eta;
    double frac = Y->frac[m];
    double ka = C->disp_kappa[m], kb = C->disp_kappa[m + 1];
    double ea = eta * ka;
    double x_end = (frac < 1.0) ? Y->x_th : eta * kb;
    double D = T - acc;
    if (D < 0.0) D = 0.0;
    double Dp = (frac > 0.0) ? D / frac : 0.0;
    double na = 1.0 + ea;
    double eaa = ea * (2.0 + ea);
    double s2a = (eaa * Y->gam2 - (1.0 + eaa)) / (Y->bg2 * (1.0 + eaa));
    if (!(s2a > 0.0)) s2a = 0.0;
    double b = x_end - ea;
    double P = na * s2a - Dp * b;
    double disc = P * P + 4.0 * b * Dp * na;
    if (!(disc > 0.0)) disc = 0.0;
    double den = P + sqrt(disc);
    double t = (den > 0.0) ? (2.0 * Dp * na) / den : 0.0;
    if (t > 1.0) t = 1.0;
    if (!(t > 0.0)) t = 0.0;
    double sm = t * frac;                 /* position inside the whole piece */
    double k = ka + sm * (kb - ka);
    double inv1 = 1.0 / C->lambda1_nm, inv2 = 1.0 / C->lambda2_nm;
    double du = (inv1 - inv2) / (double)(K - 1);
    double u = inv1 - ((double)m + sm) * du;
    *lam = 1.0 / u;
    *kap = k;
    double e = eta * k;
    double ee = e * (2.0 + e);
    double s2 = (ee * Y->gam2 - (1.0 + ee)) / (Y->bg2 * (1.0 + ee));
    if (!(s2 > 0.0)) s2 = 0.0;
    *sin_c = sqrt(s2);
    *cos_c = 1.0 / (Y->beta * (1.0 + e));
}

/* ======================================================================= */
/* Atmospheric transmission (an extension: the paper's RAYBND only bends   */
/* and times the photons; CORSIKA's IACT option can also drop photons that */
/* the atmosphere absorbs or scatters, using external transmission         */
/* profiles).  Reading: a bunch that reaches the observation level survives */
/* with probability P = exp(-tau_v(lambda, h_e) / cos(theta_obs))          */
/* (Beer-Lambert along a straight line at the observation-level zenith     */
/* through a flat atmosphere), tau_v from a table interpolated bilinearly  */
/* in (lambda, h) and clamped to its range; the draw is the fourth Philox  */
/* word of the bunch: it survives when u3 < P.                            */
/* ======================================================================= */
static double orc_trans_tau(const orc_cfg *C, double lam, double h)
{
    double xl = (lam - C->trans_l0) / (C->trans_l1 - C->trans_l0) * (double)(C->trans_nl - 1);
    double xh = (h - C->trans_h0) / (C->trans_h1 - C->trans_h0) * (double)(C->trans_nh - 1);
    if (xl < 0.0) xl = 0.0;
    if (xl > (double)(C->trans_nl - 1)) xl = (double)(C->trans_nl - 1);
    if (xh < 0.0) xh = 0.0;
    if (xh > (double)(C->trans_nh - 1)) xh = (double)(C->trans_nh - 1);
    int a = (int)xl, b = (int)xh;
    if (a > C->trans_nl - 2) a = C->trans_nl - 2;
    if (b > C->trans_nh - 2) b = C->trans_nh - 2;
    double s = xl - (double)a, t = xh - (double)b;
    const double *T = C->trans_tau;
    int nh = C->trans_nh;
    double t00 = T[a * nh + b], t01 = T[a * nh + b + 1];
    double t10 = T[(a + 1) * nh + b], t11 = T[(a + 1) * nh + b + 1];
    return (1.0 - s) * ((1.0 - t) * t00 + t * t01) + s * ((1.0 - t) * t10 + t * t11);
}

static void orc_one_bunch(const orc_cfg *C, const orc_tracks *Tk, int64_t i, int64_t j,
                          int64_t nb, const orc_yield *Y, int variant, orc_bunch1 *B)
{
    double ux = Tk->ux[i], uy = Tk->uy[i], uz = Tk->uz[i];
    double cos_c = 0.0, sin_c = 0.0;
    if (C->disp_k == 0) {
        cos_c = 1.0 / (Y->beta * (1.0 + Y->eta));
        sin_c = sqrt(Y->s2);
    }
    /* azimuth basis around the step direction */
    double e1x, e1y, e1z = 0.0;
    double rho2 = ux * ux + uy * uy;
    if (rho2 > 1e-20) {
        double r = sqrt(rho2);
        e1x = -uy / r; e1y = ux / r;
    } else {
        e1x = 1.0; e1y = 0.0;
    }
    double e2x = uy * e1z - uz * e1y;
    double e2y = uz * e1x - ux * e1z;
    double e2z = ux * e1y - uy * e1x;
    int64_t gi = Tk->track_base + i;
    uint32_t ctr[4] = { (uint32_t)((uint64_t)gi & 0xffffffffu),
                        (uint32_t)((uint64_t)gi >> 32), (uint32_t)j, 0u };
    uint32_t x[4];
    orc_philox4x32_10(ctr, C->philox_key, x);
    double u0 = orc_u01(x[0]), u1 = orc_u01(x[1]), u2 = orc_u01(x[2]);
    /* sub-step j, emission point uniform inside it */
    double f = ((double)j + u0) / (double)nb;
    double phi = 2.0 * ORC_PI * u1;
    B->kappa = 1.0;
    if (C->disp_k > 0) {
        orc_disp_sample(C, Y, u2, &B->lam, &B->kappa, &cos_c, &sin_c);
    } else {
        /* 1/lambda^2 spectrum on [lambda1, lambda2] by inversion */
        double inv1 = 1.0 / C->lambda1_nm, inv2 = 1.0 / C->lambda2_nm;
        B->lam = 1.0 / (inv1 - u2 * (inv1 - inv2));
    }
    double cp = cos(phi), sp = sin(phi);
    B->px = cos_c * ux + sin_c * (cp * e1x + sp * e2x);
    B->py = cos_c * uy + sin_c * (cp * e1y + sp * e2y);
    B->pz = cos_c * uz + sin_c * (cp * e1z + sp * e2z);
    double fl = f * Tk->len[i];
    double inv_bc = 1.0 / (Y->beta * ORC_C_M_PER_NS);
    B->xe = Tk->x0[i] + fl * ux;
    B->ye = Tk->y0[i] + fl * uy;
    B->he = Tk->z0[i] + fl * uz;
    B->te = Tk->t0[i] + fl * inv_bc;
    B->status = orc_propagate_photon_k(C, variant, B->kappa, B->xe, B->ye, B->he, B->te,
                                       B->px, B->py, B->pz, B->r);
    /* the emission height: radial in a curved atmosphere */
    if (C->earth_radius > 0.0)
        B->he = orc_radial_height(C->earth_radius, B->xe, B->ye, B->he);
    B->tr_margin = NAN;
    if (B->status == ORC_ST_GROUND && C->trans_tau) {
        double tau = orc_trans_tau(C, B->lam, B->he);
        double cos_obs = B->r[7];
        double P = exp(-(tau / cos_obs));
        double u3 = orc_u01(x[3]);
        B->tr_margin = u3 - P;
        if (!(u3 < P)) B->status = ORC_ST_ABSORBED;
    }
}

static double orc_t_ref(const orc_cfg *C, const orc_tracks *Tk, int64_t i)
{
    uint32_t sh = Tk->shower ? Tk->shower[i] : 0u;
    return (C->t_ref && (int)sh < C->n_showers) ? C->t_ref[sh] : 0.0;
}

/* ======================================================================= */
/* Whole path for a set of steps: every bunch of every step.               */
/* bunch_off[i] is the index of the first bunch of step i (a prefix sum of */
/* nb from orc_segment_yield).  variant 0 = (T), 1 = (B).                  */
/* Returns 0, or -1 on bad arguments.                                       */
/* ======================================================================= */
int orc_bunches(const orc_cfg *C, const orc_tracks *Tk, uint64_t seed,
                const int64_t *bunch_off, int variant, orc_bunch_out *O)
{
    if (!C || !Tk || !bunch_off || !O) return -1;
    orc_cfg Cs = *C;
    Cs.philox_key[0] = (uint32_t)(seed & 0xffffffffu);
    Cs.philox_key[1] = (uint32_t)(seed >> 32);
    double eta_obs_T = orc_eta_lookup(C->eta_tab, C->n_fine, C->h_max, C->h_obs);
    double eta_obs_B = orc_eta_exact(&C->atm, C->h_obs);
    double eta_obs = (variant == 0) ? eta_obs_T : eta_obs_B;

#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < Tk->n; ++i) {
        orc_yield Y;
        if (orc_step_yield(&Cs, Tk, i, &Y) != 0)
            continue;
        if (Y.nb == 0) continue;
        double t_ref = orc_t_ref(&Cs, Tk, i);
        for (int64_t j = 0; j < Y.nb; ++j) {
            int64_t bidx = bunch_off[i] + j;
            orc_bunch1 B;
            orc_one_bunch(&Cs, Tk, i, j, Y.nb, &Y, variant, &B);
            O->xe[bidx] = B.xe; O->ye[bidx] = B.ye; O->he[bidx] = B.he; O->te[bidx] = B.te;
            O->px[bidx] = B.px; O->py[bidx] = B.py; O->pz[bidx] = B.pz;
            O->lam[bidx] = B.lam; O->w[bidx] = Y.w;
            O->status[bidx] = B.status;
            O->nhit[bidx] = 0;
            if (O->tr_margin) O->tr_margin[bidx] = B.tr_margin;
            if (B.status != ORC_ST_GROUND) {
                O->X[bidx] = O->Y[bidx] = O->t[bidx] = 0.0;
                if (O->Zg) O->Zg[bidx] = 0.0;
                O->cx[bidx] = O->cy[bidx] = O->cz[bidx] = 0.0;
                continue;
            }
            double t = B.r[2] - t_ref;
            O->X[bidx] = B.r[0]; O->Y[bidx] = B.r[1]; O->t[bidx] = t;
            O->cx[bidx] = B.r[3]; O->cy[bidx] = B.r[4]; O->cz[bidx] = B.r[5];
            double np1_obs = 1.0 + B.kappa * eta_obs;
            if (O->Zg) O->Zg[bidx] = B.r[6];
            O->nhit[bidx] = orc_telescopes(&Cs, B.r[0], B.r[1], B.r[6], t, B.r[3], B.r[4], B.r[5],
                                           np1_obs,
                                           O->hit_tel + ORC_MAX_HITS * bidx,
                                           O->hit_x + ORC_MAX_HITS * bidx,
                                           O->hit_y + ORC_MAX_HITS * bidx,
                                           O->hit_t + ORC_MAX_HITS * bidx);
        }
    }
    return 0;
}

/* ======================================================================= */
/* Gaussian-smoothed photon density and mean arrival time at the telescope  */
/* centres, the quantities whose gradient the adjoint computes (the paper   */
/* has no counterpart: this is the differentiable read-out of the path):    */
/*   S_k = sum_b w_b G(r_bk),   U_k = sum_b w_b G(r_bk) t_b,                */
/*   G(r) = exp(-r^2 / (2 sigma^2)) / (2 pi sigma^2) for r < 6 sigma, else 0, */
/* r_bk the distance in the observation plane between the ground point of   */
/* bunch b and the centre (x_k, y_k) of telescope k; only bunches reaching  */
/* the ground count.  The density is D_k = S_k and the mean arrival time    */
/* Tbar_k = U_k / S_k.  nb_frozen fixes the bunch counts (the sub-step      */
/* structure) so that the sums are smooth in the parameters: w = N / nb.    */
/* Table variant (T).  S, U: n_tel entries each, overwritten.               */
/* ======================================================================= */
int orc_density(const orc_cfg *C, const orc_tracks *Tk, uint64_t seed, const int32_t *nb_frozen,
                double sigma, double *S, double *U)
{
    if (!C || !Tk || !nb_frozen || !S || !U || !(sigma > 0.0)) return -1;
    orc_cfg Cs = *C;
    Cs.philox_key[0] = (uint32_t)(seed & 0xffffffffu);
    Cs.philox_key[1] = (uint32_t)(seed >> 32);
    double norm = 1.0 / (2.0 * ORC_PI * sigma * sigma);
    double rcut2 = 36.0 * sigma * sigma;
    for (int k = 0; k < C->n_tel; ++k) { S[k] = 0.0; U[k] = 0.0; }
    for (int64_t i = 0; i < Tk->n; ++i) {
        orc_yield Y;
        if (orc_step_yield(&Cs, Tk, i, &Y) != 0) continue;
        int64_t nb = nb_frozen[i];
        if (nb <= 0 || !(Y.s2 > 0.0)) continue;
        double w = Y.N / (double)nb;
        double t_ref = orc_t_ref(&Cs, Tk, i);
        for (int64_t j = 0; j < nb; ++j) {
            orc_bunch1 B;
            orc_one_bunch(&Cs, Tk, i, j, nb, &Y, 0, &B);
            if (B.status != ORC_ST_GROUND) continue;
            double t = B.r[2] - t_ref;
            for (int k = 0; k < C->n_tel; ++k) {
                double dx = B.r[0] - C->tel[4 * k + 0];
                double dy = B.r[1] - C->tel[4 * k + 1];
                double r2 = dx * dx + dy * dy;
                if (!(r2 < rcut2)) continue;
                double G = norm * exp(-r2 / (2.0 * sigma * sigma));
                S[k] += w * G;
                U[k] += w * G * t;
            }
        }
    }
    return 0;
}

/* ======================================================================= */
/* Longitudinal profile of Cherenkov production (CERLDE, paper section 4:   */
/* the simulation can keep the number of photons produced versus           */
/* atmospheric depth, which follows the density profile).                  */
/* The paper gives no formula; the reading used here:                      */
/*  - a step emits its N photons uniformly along its straight path (its    */
/*    yield per unit length is one number, taken at the midpoint);         */
/*  - a photon is counted at the atmospheric depth of its emission point,  */
/*    X = T(h) / cos_axis (vertical depth when cos_axis = 1, the slant      */
/*    depth of a flat atmosphere along a shower axis of zenith            */
/*    acos(cos_axis) otherwise), in g/cm^2;                                */
/*  - bin k holds the depths [k dX, (k + 1) dX); photons deeper than the   */
/*    last bin are not counted.                                            */
/* Step i therefore adds N_i times the fraction of its path whose depth     */
/* lies in bin k.  Depth decreases monotonically with height, so that       */
/* fraction is the overlap of the bin's height interval with the step's     */
/* height interval, divided by the latter; the heights of the bin edges     */
/* come from bisection on T.  A horizontal step puts all its photons in     */
/* the bin of its depth.  Steps emitting no bunch, and steps whose shower  */
/* index has no row, add nothing.                                          */
/* prof: n_showers (at least 1) x n_bins, overwritten.                      */
/* ======================================================================= */
static double orc_height_of_thickness(const orc_atm *A, double target, double lo, double hi)
{
    /* T is non-increasing in h and T(hi) <= target <= T(lo) */
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (orc_thickness(A, mid) >= target) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

int orc_profile(const orc_cfg *C, const orc_tracks *Tk, const double *axis_cos,
                double bin_gcm2, int n_bins, double *prof)
{
    if (!C || !Tk || !prof || !(bin_gcm2 > 0.0) || n_bins < 1) return -1;
    int ns = C->n_showers > 0 ? C->n_showers : 1;
    for (int64_t q = 0; q < (int64_t)ns * n_bins; ++q) prof[q] = 0.0;
    for (int64_t i = 0; i < Tk->n; ++i) {
        orc_yield Y;
        if (orc_step_yield(C, Tk, i, &Y) != 0 || Y.nb <= 0) continue;
        int64_t s = Tk->shower ? (int64_t)Tk->shower[i] : 0;
        if (s >= ns) continue;                               /* no row: not counted */
        double cz = axis_cos ? axis_cos[s] : 1.0;
        double za = Tk->z0[i];
        double zb = za + Tk->len[i] * Tk->uz[i];
        double lo = za < zb ? za : zb;
        double hi = za < zb ? zb : za;
        double X_top = orc_thickness(&C->atm, hi) / cz;     /* shallowest point */
        double X_bot = orc_thickness(&C->atm, lo) / cz;     /* deepest point    */
        double *row = prof + (int64_t)s * n_bins;
        if (hi == lo) {
            double kd = floor(X_top / bin_gcm2);
            if (kd >= 0.0 && kd < (double)n_bins) row[(int)kd] += Y.N;
            continue;
        }
        for (int k = 0; k < n_bins; ++k) {
            double e0 = (double)k * bin_gcm2;
            double e1 = (double)(k + 1) * bin_gcm2;
            if (!(X_top < e1) || !(X_bot >= e0)) continue;  /* no overlap */
            double h_up = X_top >= e0 ? hi : orc_height_of_thickness(&C->atm, e0 * cz, lo, hi);
            double h_dn = X_bot < e1 ? lo : orc_height_of_thickness(&C->atm, e1 * cz, lo, hi);
            double frac = (h_up - h_dn) / (hi - lo);
            row[k] += Y.N * frac;
        }
    }
    return 0;
}

/* ======================================================================= */
/* Shower steps from a parameterised electromagnetic shower (an extension: */
/* the paper's input are the EGS4 electron/positron steps that CORSIKA      */
/* hands to CERENK; this generator stands in for them on the device).      */
/* Per shower: primary energy E0 (MeV), axis zenith and azimuth, core      */
/* (x, y) at h_obs, n steps at global indices first .. first + n - 1.       */
/* Per step g, eight deviates u0..u7 from Philox4x32-10 keyed by the seed, */
/* counters (g_lo, g_hi, 0, 1) and (g_lo, g_hi, 1, 1):                     */
/*   depth  t (radiation lengths) from the Greisen profile                  */
/*          N(t) ~ exp(t (1 - 1.5 ln s)) / sqrt(y), s = 3t/(t + 2y),        */
/*          y = ln(E0/E_c), E_c = 85 MeV, on (0, t_g], t_g the slant depth  */
/*          of h_obs (isothermal air, X(h) = 1030 exp(-h/8000 m) g/cm^2,    */
/*          X0 = 36.7 g/cm^2), by inverting the CDF tabulated on n_cdf      */
/*          uniform nodes (linear between them) at u0;                      */
/*   height h = 8000 ln(1030 / (t X0 cos(zenith))), at most 29999 m, and    */
/*          s = (h - h_obs)/cos(zenith) up the axis from the core;          */
/*   lateral offset r = -50 ln(u1) m (exponential, mean 50 m) at azimuth    */
/*          2 pi u2 in the plane normal to the axis (basis b1, b2);         */
/*   kinetic energy E = 20 MeV (5000/20)^u3 (log-uniform 20 MeV - 5 GeV);   */
/*   direction: axis + sigma (n1 b1 + n2 b2), normalised, with             */
/*          sigma = 3 deg * 50 MeV / E and (n1, n2) standard normals by     */
/*          Box-Muller from (u4, u5);                                       */
/*   start time (s_ref - s)/c with s_ref = (30000 m - h_obs)/cos(zenith);   */
/*   length 1 + 19 u6 m.                                                    */
/* The reference time of the shower is s_ref / c.                          */
/* ======================================================================= */
typedef struct {
    double e0_mev, zenith, azimuth, core_x, core_y;
    int64_t first, n;
} orc_shower;

static double orc_greisen(double t, double y)
{
    if (t <= 0.0) return 1.0 / sqrt(y);
    double s = 3.0 * t / (t + 2.0 * y);
    return exp(t * (1.0 - 1.5 * log(s))) / sqrt(y);
}

static double orc_simpson_greisen(double a, double b, double y, double fa, double fm, double fb,
                                  double whole, double tol, int depth)
{
    double m = 0.5 * (a + b);
    double lm = orc_greisen(0.5 * (a + m), y), rm = orc_greisen(0.5 * (m + b), y);
    double left = (m - a) / 6.0 * (fa + 4.0 * lm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * rm + fb);
    if (depth <= 0 || fabs(left + right - whole) <= 15.0 * tol)
        return left + right + (left + right - whole) / 15.0;
    return orc_simpson_greisen(a, m, y, fa, lm, fm, left, 0.5 * tol, depth - 1) +
           orc_simpson_greisen(m, b, y, fm, rm, fb, right, 0.5 * tol, depth - 1);
}

/* cdf[0 .. n_cdf-1] on t_k = k t_g / (n_cdf - 1), normalised to 1 */
static void orc_greisen_cdf(double y, double t_g, int n_cdf, double *cdf)
{
    double dt = t_g / (double)(n_cdf - 1);
    cdf[0] = 0.0;
    for (int k = 1; k < n_cdf; ++k) {
        double a = (double)(k - 1) * dt, b = (double)k * dt;
        double fa = orc_greisen(a, y), fb = orc_greisen(b, y), fm = orc_greisen(0.5 * (a + b), y);
        double whole = (b - a) / 6.0 * (fa + 4.0 * fm + fb);
        cdf[k] = cdf[k - 1] + orc_simpson_greisen(a, b, y, fa, fm, fb, whole, 1e-15 * fabs(whole) + 1e-300, 40);
    }
    double tot = cdf[n_cdf - 1];
    for (int k = 0; k < n_cdf; ++k) cdf[k] /= tot;
}

int orc_generate_steps(const orc_shower *S, int n_showers, double h_obs, uint64_t seed,
                       int n_cdf, double *x0, double *y0, double *z0, double *t0, double *len,
                       double *ekin, double *ux, double *uy, double *uz, uint32_t *shower,
                       double *t_ref)
{
    const double c_light = ORC_C_M_PER_NS, X0 = 36.7, E_c = 85.0, X_sea = 1030.0, H = 8000.0;
    const double h_start = 30000.0;
    if (!S || n_showers < 1 || n_cdf < 2) return -1;
    double *cdf = (double *)malloc(sizeof(double) * (size_t)n_cdf);
    if (!cdf) return -1;
    uint32_t key[2] = { (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) };
    for (int sh = 0; sh < n_showers; ++sh) {
        const orc_shower *P = S + sh;
        double cz = cos(P->zenith);
        if (!(P->e0_mev > E_c) || !(cz > 0.0)) { free(cdf); return -1; }
        double y = log(P->e0_mev / E_c);
        double t_g = X_sea * exp(-(h_obs / H)) / cz / X0;
        orc_greisen_cdf(y, t_g, n_cdf, cdf);
        double dt = t_g / (double)(n_cdf - 1);
        double sz = sin(P->zenith);
        double ax = sz * cos(P->azimuth), ay = sz * sin(P->azimuth), az = -cz;
        /* b1 = axis x z (normalised), b2 = axis x b1 */
        double b1x = ay, b1y = -ax, b1z = 0.0;
        double nb = sqrt(b1x * b1x + b1y * b1y);
        if (nb > 1e-12) { b1x /= nb; b1y /= nb; } else { b1x = 1.0; b1y = 0.0; }
        double b2x = ay * b1z - az * b1y, b2y = az * b1x - ax * b1z, b2z = ax * b1y - ay * b1x;
        double s_ref = (h_start - h_obs) / cz;
        t_ref[sh] = s_ref / c_light;
        for (int64_t k = 0; k < P->n; ++k) {
            int64_t g = P->first + k;
            uint32_t c0[4] = { (uint32_t)((uint64_t)g & 0xffffffffu), (uint32_t)((uint64_t)g >> 32), 0u, 1u };
            uint32_t c1[4] = { c0[0], c0[1], 1u, 1u };
            uint32_t w0[4], w1[4];
            orc_philox4x32_10(c0, key, w0);
            orc_philox4x32_10(c1, key, w1);
            double u[8];
            for (int q = 0; q < 4; ++q) { u[q] = orc_u01(w0[q]); u[4 + q] = orc_u01(w1[q]); }
            /* depth: the node interval holding u0, then linear inside it */
            int lo = 0, hi = n_cdf - 1;
            while (hi - lo > 1) {
                int mid = (lo + hi) / 2;
                if (cdf[mid] <= u[0]) lo = mid; else hi = mid;
            }
            double t = (double)lo * dt + (u[0] - cdf[lo]) / (cdf[lo + 1] - cdf[lo]) * dt;
            double h = H * log(X_sea / (t * X0 * cz));
            if (h > h_start - 1.0) h = h_start - 1.0;
            double sa = (h - h_obs) / cz;
            double r = -50.0 * log(u[1]);
            double psi = 2.0 * ORC_PI * u[2];
            double lx = r * cos(psi), ly = r * sin(psi);
            x0[g] = P->core_x - sa * ax + lx * b1x + ly * b2x;
            y0[g] = P->core_y - sa * ay + lx * b1y + ly * b2y;
            z0[g] = h_obs - sa * az + lx * b1z + ly * b2z;
            double e = 20.0 * exp(u[3] * log(5000.0 / 20.0));
            ekin[g] = e;
            double sig = (3.0 * ORC_PI / 180.0) * (50.0 / e);
            double rho = sqrt(-2.0 * log(u[4]));
            double n1 = rho * cos(2.0 * ORC_PI * u[5]), n2 = rho * sin(2.0 * ORC_PI * u[5]);
            double dx = ax + sig * (n1 * b1x + n2 * b2x);
            double dy = ay + sig * (n1 * b1y + n2 * b2y);
            double dz = az + sig * (n1 * b1z + n2 * b2z);
            double dn = sqrt(dx * dx + dy * dy + dz * dz);
            ux[g] = dx / dn; uy[g] = dy / dn; uz[g] = dz / dn;
            t0[g] = (s_ref - sa) / c_light;
            len[g] = 1.0 + 19.0 * u[6];
            shower[g] = (uint32_t)sh;
        }
    }
    free(cdf);
    return 0;
}

int orc_max_hits(void) { return ORC_MAX_HITS; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The number of OpenMP threads of the next parallel loops (timing only; no
 * effect without OpenMP). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ======================================================================= */
/* Reference gradient of the read-out by forward-mode dual numbers (no     */
/* counterpart in the paper: the reference for the library's adjoint).    */
/* Every quantity carries its value and its derivatives with respect to    */
/* ORC_NG inputs: the six of the step it belongs to (x0, y0, z0, u_x, u_y, */
/* u_z) and the ten atmosphere parameters n depends on (b_0..b_4,          */
/* c_0..c_4; n does not depend on a_i, so dL/da_i = 0).  The arithmetic is */
/* the table variant's (T), statement by statement and in the same order,  */
/* so the values are the oracle's own: the derivative of an adaptive       */
/* integral is that of the quadrature it chose (the same nodes), the       */
/* derivative of a table lookup that of the interpolation inside the cell  */
/* it chose; the bunch counts are frozen (w = N / nb).  For                */
/*   L = sum_k gD_k S_k + gT_k Tbar_k,  Tbar_k = U_k / S_k,               */
/* dL/dS_k = gD_k - gT_k U_k / S_k^2 and dL/dU_k = gT_k / S_k.             */
/* Flat layers, constant index.                                             */
/* ======================================================================= */
#define ORC_NG 16
enum { ORC_G_X0 = 0, ORC_G_Y0, ORC_G_Z0, ORC_G_UX, ORC_G_UY, ORC_G_UZ, ORC_G_B0 = 6,
       ORC_G_C0 = 11 };

typedef struct {
    double v;
    double d[ORC_NG];
} orc_dual;

static orc_dual od_c(double v)
{
    orc_dual r;
    r.v = v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = 0.0;
    return r;
}

static orc_dual od_var(double v, int i)
{
    orc_dual r = od_c(v);
    r.d[i] = 1.0;
    return r;
}

static orc_dual od_add(orc_dual a, orc_dual b)
{
    orc_dual r;
    r.v = a.v + b.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}

static orc_dual od_sub(orc_dual a, orc_dual b)
{
    orc_dual r;
    r.v = a.v - b.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}

static orc_dual od_mul(orc_dual a, orc_dual b)
{
    orc_dual r;
    r.v = a.v * b.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
    return r;
}

/* a / b: d(a/b) = (da - (a/b) db) / b */
static orc_dual od_div(orc_dual a, orc_dual b)
{
    orc_dual r;
    r.v = a.v / b.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
    return r;
}

/* constant on the left of a product, a sum, a quotient; quotient by a constant */
static orc_dual od_cmul(double s, orc_dual a)
{
    orc_dual r;
    r.v = s * a.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = s * a.d[i];
    return r;
}

static orc_dual od_cadd(double s, orc_dual a)
{
    orc_dual r = a;
    r.v = s + a.v;
    return r;
}

static orc_dual od_csub(double s, orc_dual a)
{
    orc_dual r;
    r.v = s - a.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = -a.d[i];
    return r;
}

static orc_dual od_subc(orc_dual a, double s)
{
    orc_dual r = a;
    r.v = a.v - s;
    return r;
}

static orc_dual od_divc(orc_dual a, double s)
{
    orc_dual r;
    r.v = a.v / s;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = a.d[i] / s;
    return r;
}

static orc_dual od_cdiv(double s, orc_dual b)
{
    orc_dual r;
    r.v = s / b.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = -r.v * b.d[i] / b.v;
    return r;
}

static orc_dual od_neg(orc_dual a)
{
    orc_dual r;
    r.v = -a.v;
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = -a.d[i];
    return r;
}

static orc_dual od_sqrt(orc_dual a)
{
    orc_dual r;
    r.v = sqrt(a.v);
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
    return r;
}

static orc_dual od_exp(orc_dual a)
{
    orc_dual r;
    r.v = exp(a.v);
    for (int i = 0; i < ORC_NG; ++i) r.d[i] = r.v * a.d[i];
    return r;
}

/* rho(h) = (b_i / c_i) exp(-h / c_i) in layer i, b_i and c_i as variables */
static orc_dual od_rho(const orc_atm *A, orc_dual h)
{
    if (h.v >= A->h_bound[5]) return od_c(0.0);
    int i = orc_layer(A, h.v);
    orc_dual b = od_var(A->b[i], ORC_G_B0 + i);
    orc_dual c = od_var(A->c[i], ORC_G_C0 + i);
    orc_dual r = od_div(b, c);
    orc_dual e = od_exp(od_neg(od_div(h, c)));
    return od_mul(r, e);
}

/* eta(h) = n0_minus_1 rho(h) / rho(0) */
static orc_dual od_eta_exact(const orc_atm *A, orc_dual h)
{
    orc_dual rho0 = od_rho(A, od_c(0.0));
    orc_dual rho = od_rho(A, h);
    orc_dual q = od_div(rho, rho0);
    return od_cmul(A->n0_minus_1, q);
}

static orc_dual od_eta_lookup(const orc_dual *tab, int n, double h_max, orc_dual h)
{
    double dh = h_max / (double)(n - 1);
    double inv_dh = 1.0 / dh;
    orc_dual hc = h;
    if (hc.v < 0.0) hc = od_c(0.0);
    if (hc.v > h_max) hc = od_c(h_max);
    orc_dual x = od_cmul(inv_dh, hc);
    int k = (int)x.v;
    if (k > n - 2) k = n - 2;
    orc_dual f = od_subc(x, (double)k);
    orc_dual d = od_sub(tab[k + 1], tab[k]);
    orc_dual fd = od_mul(f, d);
    return od_add(tab[k], fd);
}

/* the ray-integral integrands of the tables (orc_integrand) in duals */
typedef struct {
    const orc_atm *A;
    orc_dual np1_obs;
    double s_obs, c_obs;
    int which;
    double floor;
} orc_dray;

static orc_dual od_integrand(const orc_dray *R, double h)
{
    orc_dual eta = od_eta_exact(R->A, od_c(h));
    orc_dual np1 = od_cadd(1.0, eta);
    orc_dual s = od_div(od_mul(R->np1_obs, od_c(R->s_obs)), np1);
    orc_dual c = od_sqrt(od_csub(1.0, od_mul(s, s)));
    switch (R->which) {
    case F_TAN_CORR: return od_subc(od_div(s, c), R->s_obs / R->c_obs);
    case F_OPT_CORR: return od_subc(od_div(np1, c), 1.0 / R->c_obs);
    case F_RATIO: return od_subc(od_div(R->np1_obs, np1), 1.0);
    }
    return od_c(0.0);
}

/* adaptive Simpson in duals: every decision on the values, as orc_simpson_rec */
static orc_dual od_simpson_rec(const orc_dray *R, double a, double b, orc_dual fa, orc_dual fm,
                               orc_dual fb, orc_dual whole, double tol, int depth)
{
    double m = 0.5 * (a + b);
    double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    orc_dual flm = od_integrand(R, lm), frm = od_integrand(R, rm);
    orc_dual left = od_cmul((m - a) / 6.0, od_add(od_add(fa, od_cmul(4.0, flm)), fm));
    orc_dual right = od_cmul((b - m) / 6.0, od_add(od_add(fm, od_cmul(4.0, frm)), fb));
    orc_dual delta = od_sub(od_add(left, right), whole);
    if (depth <= 0 || fabs(delta.v) <= 15.0 * tol
        || fabs(delta.v) <= orc_noise_floor(R->floor, a, b, fa.v, fm.v, fb.v))
        return od_add(od_add(left, right), od_divc(delta, 15.0));
    return od_add(od_simpson_rec(R, a, m, fa, flm, fm, left, 0.5 * tol, depth - 1),
                  od_simpson_rec(R, m, b, fm, frm, fb, right, 0.5 * tol, depth - 1));
}

static orc_dual od_simpson(const orc_dray *R, double a, double b, double tol)
{
    if (b <= a) return od_c(0.0);
    orc_dual fa = od_integrand(R, a), fb = od_integrand(R, b);
    double m = 0.5 * (a + b);
    orc_dual fm = od_integrand(R, m);
    orc_dual whole = od_cmul((b - a) / 6.0, od_add(od_add(fa, od_cmul(4.0, fm)), fb));
    return od_simpson_rec(R, a, b, fa, fm, fb, whole, tol, 48);
}

static orc_dual od_integrate(const orc_dray *R, double lo, double hi, double tol)
{
    orc_dual sum = od_c(0.0);
    double a = lo;
    for (int i = 1; i <= 5; ++i) {
        double hb = R->A->h_bound[i];
        if (hb > a && hb < hi) {
            sum = od_add(sum, od_simpson(R, a, hb, tol));
            a = hb;
        }
    }
    return od_add(sum, od_simpson(R, a, hi, tol));
}

/* orc_build_refraction_tables in duals */
static void od_build_tables(const orc_atm *A, double h_obs, double h_max, int H, int Z,
                            double theta_max, double tol, orc_dual *ax, orc_dual *al)
{
    double dht = (h_max - h_obs) / (double)(H - 1);
    double smax = sin(theta_max);
    double dq = smax * smax / (double)(Z - 1);
    orc_dual np1_obs = od_cadd(1.0, od_eta_exact(A, od_c(h_obs)));
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < Z; ++k) {
        double q = (double)k * dq;
        double so = sqrt(q), co = sqrt(1.0 - so * so);
        orc_dray R;
        R.A = A; R.np1_obs = np1_obs; R.s_obs = so; R.c_obs = co;
        R.floor = 1e-9;
        orc_dual dx = od_c(0.0), dl = od_c(0.0);
        ax[(size_t)0 * Z + k] = od_c(0.0);
        al[(size_t)0 * Z + k] = od_c(0.0);
        for (int j = 1; j < H; ++j) {
            double lo = h_obs + (double)(j - 1) * dht;
            double hi = h_obs + (double)j * dht;
            R.which = (k == 0) ? F_RATIO : F_TAN_CORR;
            dx = od_add(dx, od_integrate(&R, lo, hi, tol));
            R.which = F_OPT_CORR;
            dl = od_add(dl, od_integrate(&R, lo, hi, tol));
            double c3 = co * co * co;
            ax[(size_t)j * Z + k] = (k == 0) ? dx : od_divc(od_cmul(c3, dx), so);
            al[(size_t)j * Z + k] = od_cmul(c3, dl);
        }
    }
}

static orc_dual od_bilinear(const orc_dual *T, int Z, int j, int k, orc_dual a, orc_dual b)
{
    orc_dual t00 = T[(size_t)j * Z + k], t01 = T[(size_t)j * Z + k + 1];
    orc_dual t10 = T[(size_t)(j + 1) * Z + k], t11 = T[(size_t)(j + 1) * Z + k + 1];
    orc_dual v0 = od_add(t00, od_mul(a, od_sub(t10, t00)));
    orc_dual v1 = od_add(t01, od_mul(a, od_sub(t11, t01)));
    return od_add(v0, od_mul(b, od_sub(v1, v0)));
}

typedef struct {
    const orc_dual *eta, *ax, *al;
    orc_dual eta_obs;
} orc_dtabs;

/* One bunch in duals (orc_one_bunch + the (T) propagation, flat layers):
 * its ground point X, Y, arrival time t (before t_ref) and photons w.
 * Returns 1 when it reaches the ground. */
static int od_bunch(const orc_cfg *C, const orc_dtabs *D, const orc_tracks *Tk, int64_t i,
                    int64_t j, int64_t nb, orc_dual *X, orc_dual *Y, orc_dual *t, orc_dual *w)
{
    orc_dual x0 = od_var(Tk->x0[i], ORC_G_X0), y0 = od_var(Tk->y0[i], ORC_G_Y0);
    orc_dual z0 = od_var(Tk->z0[i], ORC_G_Z0);
    orc_dual ux = od_var(Tk->ux[i], ORC_G_UX), uy = od_var(Tk->uy[i], ORC_G_UY);
    orc_dual uz = od_var(Tk->uz[i], ORC_G_UZ);
    double len = Tk->len[i];
    /* the yield (orc_step_yield_valid), nb frozen */
    double inv_me = 1.0 / ORC_ME_MEV;
    double K = orc_band_factor(C);
    double g = Tk->ekin[i] * inv_me;
    double gam = 1.0 + g;
    double gam2 = gam * gam;
    double half_len = 0.5 * len;
    orc_dual hm = od_add(z0, od_cmul(half_len, uz));
    orc_dual eta = od_eta_lookup(D->eta, C->n_fine, C->h_max, hm);
    orc_dual np1 = od_cadd(1.0, eta);
    orc_dual np1sq = od_mul(np1, np1);
    orc_dual two_eta = od_cadd(2.0, eta);
    orc_dual a = od_mul(eta, two_eta);
    orc_dual b = od_mul(a, od_c(gam2));
    orc_dual num = od_sub(b, np1sq);
    double two_g = 2.0 + g;
    double bg2 = g * two_g;
    orc_dual den = od_cmul(bg2, np1sq);
    orc_dual s2 = od_div(num, den);
    if (!(s2.v > 0.0)) return 0;
    double beta = sqrt(bg2) / gam;
    orc_dual N = od_cmul(len, od_cmul(K, s2));
    *w = od_divc(N, (double)nb);
    /* emission (orc_one_bunch) */
    orc_dual cos_c = od_cdiv(1.0, od_cmul(beta, od_cadd(1.0, eta)));
    orc_dual sin_c = od_sqrt(s2);
    orc_dual e1x, e1y, e1z = od_c(0.0);
    orc_dual rho2 = od_add(od_mul(ux, ux), od_mul(uy, uy));
    if (rho2.v > 1e-20) {
        orc_dual r = od_sqrt(rho2);
        e1x = od_div(od_neg(uy), r);
        e1y = od_div(ux, r);
    } else {
        e1x = od_c(1.0);
        e1y = od_c(0.0);
    }
    orc_dual e2x = od_sub(od_mul(uy, e1z), od_mul(uz, e1y));
    orc_dual e2y = od_sub(od_mul(uz, e1x), od_mul(ux, e1z));
    orc_dual e2z = od_sub(od_mul(ux, e1y), od_mul(uy, e1x));
    int64_t gi = Tk->track_base + i;
    uint32_t ctr[4] = { (uint32_t)((uint64_t)gi & 0xffffffffu),
                        (uint32_t)((uint64_t)gi >> 32), (uint32_t)j, 0u };
    uint32_t xw[4];
    orc_philox4x32_10(ctr, C->philox_key, xw);
    double u0 = orc_u01(xw[0]), u1 = orc_u01(xw[1]);
    double f = ((double)j + u0) / (double)nb;
    double phi = 2.0 * ORC_PI * u1;
    double cp = cos(phi), sp = sin(phi);
    orc_dual px = od_add(od_mul(cos_c, ux),
                         od_mul(sin_c, od_add(od_cmul(cp, e1x), od_cmul(sp, e2x))));
    orc_dual py = od_add(od_mul(cos_c, uy),
                         od_mul(sin_c, od_add(od_cmul(cp, e1y), od_cmul(sp, e2y))));
    orc_dual pz = od_add(od_mul(cos_c, uz),
                         od_mul(sin_c, od_add(od_cmul(cp, e1z), od_cmul(sp, e2z))));
    double fl = f * len;
    double inv_bc = 1.0 / (beta * ORC_C_M_PER_NS);
    orc_dual xe = od_add(x0, od_cmul(fl, ux));
    orc_dual ye = od_add(y0, od_cmul(fl, uy));
    orc_dual he = od_add(z0, od_cmul(fl, uz));
    double te = Tk->t0[i] + fl * inv_bc;
    /* propagation (orc_propagate_photon_k, variant (T), kappa = 1) */
    if (pz.v >= 0.0 || he.v < C->h_obs || he.v > C->h_max) return 0;
    orc_dual sin_em = od_sqrt(od_add(od_mul(px, px), od_mul(py, py)));
    orc_dual eta_e = od_eta_lookup(D->eta, C->n_fine, C->h_max, he);
    orc_dual sin_obs = od_div(od_mul(sin_em, od_cadd(1.0, eta_e)), od_cadd(1.0, D->eta_obs));
    orc_dual q = od_mul(sin_obs, sin_obs);
    double smax = sin(C->theta_max);
    double q_max = smax * smax;
    if (q.v > q_max) return 0;
    orc_dual cos_obs = od_sqrt(od_csub(1.0, q));
    orc_dual dH = od_subc(he, C->h_obs);
    orc_dual hx = od_c(0.0), hy = od_c(0.0);
    if (sin_em.v > 0.0) { hx = od_div(px, sin_em); hy = od_div(py, sin_em); }
    double dht = (C->h_max - C->h_obs) / (double)(C->H - 1);
    double dq = q_max / (double)(C->Z - 1);
    orc_dual fj = od_divc(dH, dht);
    int jj = (int)fj.v;
    if (jj > C->H - 2) jj = C->H - 2;
    orc_dual aa = od_subc(fj, (double)jj);
    orc_dual fk = od_divc(q, dq);
    int kk = (int)fk.v;
    if (kk > C->Z - 2) kk = C->Z - 2;
    orc_dual bb = od_subc(fk, (double)kk);
    orc_dual Ax = od_bilinear(D->ax, C->Z, jj, kk, aa, bb);
    orc_dual Al = od_bilinear(D->al, C->Z, jj, kk, aa, bb);
    orc_dual sec = od_cdiv(1.0, cos_obs);
    orc_dual tn = od_mul(sin_obs, sec);
    orc_dual sec2 = od_mul(sec, sec);
    orc_dual Dh = od_add(od_mul(dH, tn), od_mul(od_mul(Ax, tn), sec2));
    orc_dual Lp = od_add(od_mul(dH, sec), od_mul(od_mul(Al, sec2), sec));
    *X = od_add(xe, od_mul(Dh, hx));
    *Y = od_add(ye, od_mul(Dh, hy));
    *t = od_cadd(te, od_divc(Lp, ORC_C_M_PER_NS));
    return 1;
}

/* S, U of the read-out and the gradients of L: grad_atm[15] (a_0..a_4,
 * b_0..b_4, c_0..c_4), grad_steps[6 n] (dL/dx0, dL/dy0, dL/dz0, dL/dux,
 * dL/duy, dL/duz, six arrays of n).  table_tol is the tolerance the tables
 * were built with.  Returns 0, or -1 on bad arguments or a configuration it
 * does not cover (curved, dispersion, fallback, transmission). */
int orc_density_grad(const orc_cfg *C, const orc_tracks *Tk, uint64_t seed,
                     const int32_t *nb_frozen, double sigma, const double *gD,
                     const double *gT, double table_tol, double *S, double *U,
                     double *grad_atm, double *grad_steps)
{
    if (!C || !Tk || !nb_frozen || !gD || !gT || !S || !U || !grad_atm || !grad_steps
        || !(sigma > 0.0) || C->earth_radius > 0.0 || C->disp_k > 0 || C->fb_sin2_max > 0.0
        || C->trans_tau)
        return -1;
    orc_cfg Cs = *C;
    Cs.philox_key[0] = (uint32_t)(seed & 0xffffffffu);
    Cs.philox_key[1] = (uint32_t)(seed >> 32);
    size_t nt = (size_t)C->H * C->Z;
    orc_dual *eta = malloc(sizeof(orc_dual) * (size_t)C->n_fine);
    orc_dual *ax = malloc(sizeof(orc_dual) * nt), *al = malloc(sizeof(orc_dual) * nt);
    int n_tel = C->n_tel;
    orc_dual *SU = malloc(sizeof(orc_dual) * 2 * (size_t)(n_tel > 0 ? n_tel : 1));
    if (!eta || !ax || !al || !SU) {
        free(eta); free(ax); free(al); free(SU);
        return -1;
    }
    double dh = C->h_max / (double)(C->n_fine - 1);
    for (int k = 0; k < C->n_fine; ++k) eta[k] = od_eta_exact(&C->atm, od_c((double)k * dh));
    od_build_tables(&C->atm, C->h_obs, C->h_max, C->H, C->Z, C->theta_max, table_tol, ax, al);
    orc_dtabs D;
    D.eta = eta; D.ax = ax; D.al = al;
    D.eta_obs = od_eta_lookup(eta, C->n_fine, C->h_max, od_c(C->h_obs));
    double norm = 1.0 / (2.0 * ORC_PI * sigma * sigma);
    double rcut2 = 36.0 * sigma * sigma;
    for (int k = 0; k < 2 * n_tel; ++k) SU[k] = od_c(0.0);
    /* pass 1: S and U with their atmosphere tangents (the step tangents of
     * different steps are different variables and are not summed here) */
    for (int pass = 0; pass < 2; ++pass) {
        double dLdS[4096], dLdU[4096];
        if (pass == 1) {
            if (n_tel > 4096) break;
            for (int k = 0; k < n_tel; ++k) {
                double s = SU[k].v, u = SU[n_tel + k].v;
                dLdS[k] = gD[k];
                dLdU[k] = 0.0;
                if (s > 0.0) {
                    dLdS[k] = gD[k] - gT[k] * u / (s * s);
                    dLdU[k] = gT[k] / s;
                }
            }
            for (int q = 0; q < 15; ++q) grad_atm[q] = 0.0;
            for (int q = 0; q < 10; ++q) {
                double gq = 0.0;
                for (int k = 0; k < n_tel; ++k)
                    gq += dLdS[k] * SU[k].d[ORC_G_B0 + q] + dLdU[k] * SU[n_tel + k].d[ORC_G_B0 + q];
                grad_atm[5 + q] = gq;
            }
        }
        for (int64_t i = 0; i < Tk->n; ++i) {
            double gs[6] = { 0, 0, 0, 0, 0, 0 };
            int64_t nb = nb_frozen[i];
            orc_yield Yv;
            if (nb > 0 && orc_step_yield(&Cs, Tk, i, &Yv) == 0 && Yv.s2 > 0.0) {
                double t_ref = orc_t_ref(&Cs, Tk, i);
                for (int64_t j = 0; j < nb; ++j) {
                    /* the bunch's values first (the same arithmetic): the
                     * dual numbers only where it lands within the cut of a
                     * centre, as nothing else contributes */
                    orc_bunch1 B;
                    orc_one_bunch(&Cs, Tk, i, j, nb, &Yv, 0, &B);
                    if (B.status != ORC_ST_GROUND) continue;
                    int near = 0;
                    for (int k = 0; k < n_tel && !near; ++k) {
                        double ex = B.r[0] - C->tel[4 * k + 0], ey = B.r[1] - C->tel[4 * k + 1];
                        near = ex * ex + ey * ey < rcut2;
                    }
                    if (!near) continue;
                    orc_dual X, Y, t, w;
                    if (!od_bunch(&Cs, &D, Tk, i, j, nb, &X, &Y, &t, &w)) continue;
                    t = od_subc(t, t_ref);
                    for (int k = 0; k < n_tel; ++k) {
                        orc_dual dx = od_subc(X, C->tel[4 * k + 0]);
                        orc_dual dy = od_subc(Y, C->tel[4 * k + 1]);
                        orc_dual r2 = od_add(od_mul(dx, dx), od_mul(dy, dy));
                        if (!(r2.v < rcut2)) continue;
                        orc_dual G = od_cmul(norm, od_exp(od_divc(od_neg(r2), 2.0 * sigma * sigma)));
                        orc_dual wG = od_mul(w, G);
                        orc_dual wGt = od_mul(wG, t);
                        if (pass == 0) {
                            SU[k] = od_add(SU[k], wG);
                            SU[n_tel + k] = od_add(SU[n_tel + k], wGt);
                        } else {
                            for (int m = 0; m < 6; ++m)
                                gs[m] += dLdS[k] * wG.d[m] + dLdU[k] * wGt.d[m];
                        }
                    }
                }
            }
            if (pass == 1)
                for (int m = 0; m < 6; ++m) grad_steps[(size_t)m * (size_t)Tk->n + (size_t)i] = gs[m];
        }
    }
    int ok = n_tel <= 4096;
    for (int k = 0; k < n_tel; ++k) { S[k] = SU[k].v; U[k] = SU[n_tel + k].v; }
    free(eta); free(ax); free(al); free(SU);
    return ok ? 0 : -1;
}
