/*
 * mcd_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of the representative-particle dust
 * coagulation step of mcdust (Vaikundaraman, Gurrutxaga & Drazkowska 2025,
 * "mcdust: A 2D Monte Carlo code for dust coagulation in protoplanetary
 * disks", Summary section): a static, vertically isothermal power-law gas disk
 * (Benchmark table) or one tabulated in radius, swarms of identical particles followed through one
 * representative each (Zsom & Dullemond 2008, cited in the Summary), sticking,
 * fragmentation and erosion outcomes (Summary), radial and vertical transport
 * (Summary), and an adaptive grid whose cells hold equal numbers of
 * representatives (Summary).
 *
 * The paper prints no formulas; every formula below is the standard published
 * form of the physics the Summary names, and each is marked "reading" where a
 * choice was made.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library.  It shares no code,
 * header, table or constant generator with the CUDA library; it is compiled
 * with -ffp-contract=off so that no multiply-add is fused behind its back.
 *
 * Parity status: every function here is pinned by a test in tests/ against a
 * closed form, an invariant, brute force, a library routine or a numerical
 * integral (the gas state at 1 AU against textbook definitions and printed
 * closed-form numbers; the Ormel & Cuzzi closed forms against quadratures of
 * their eddy-class integrals), except the absolute physical outcome of full
 * disk runs (the paper prints no numbers for them), which is "parity
 * unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- constants (CGS).  The paper states none of them (reading). ---------- */
#define ORC_GM_SUN 1.32712440018e26 /* G * M_sun [cm^3 s^-2] */
#define ORC_AU 1.495978707e13       /* astronomical unit [cm] */
#define ORC_YR 3.15576e7            /* Julian year [s] */
#define ORC_KB 1.380649e-16         /* Boltzmann constant [erg/K] */
#define ORC_MP 1.67262192e-24       /* proton mass [g] */
#define ORC_PI 3.141592653589793
#define ORC_YA 1.6                  /* Ormel & Cuzzi (2007) y_a */

/* status codes (same meaning as the library's, own definitions) */
#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENAN -4
#define ORC_ETIMEOUT -5

/* domain tags of the counter-based random stream (4th counter word) */
#define ORC_TAG_INIT 1ULL
#define ORC_TAG_COLLIDE 2ULL
#define ORC_TAG_TRANSPORT 3ULL

/* relative-velocity term switches */
#define ORC_DV_BM 1
#define ORC_DV_TURB 2
#define ORC_DV_RAD 4
#define ORC_DV_PHI 8
#define ORC_DV_SET 16

/* transport switches */
#define ORC_TR_RADIAL 1
#define ORC_TR_VERTICAL 2
#define ORC_TR_ST_MIDPLANE 4

typedef struct {
    /* Benchmark table of the paper */
    double sigma0;        /* gas surface density at 1 AU [g cm^-2] */
    double p;             /* Sigma_g ~ r^-p */
    double T0;            /* temperature at 1 AU [K] */
    double q;             /* T ~ r^-q */
    double alpha;         /* turbulence strength */
    double v_frag;        /* fragmentation velocity [cm/s] */
    double erosion_ratio; /* mass ratio at and above which erosion happens */
    /* workload parameters the paper does not give */
    double dust_to_gas, r_in, r_out, m_star, rho_s, a_mono;
    /* readings */
    double mu, sigma_h2, dm_group, frag_xi, erosion_chi;
    /* constant-kernel (0D) mode and initial state overrides */
    double K_const, V_const, m_init, M_total;
    /* fragmentation probability ramp: relative width below v_frag (reading) */
    double frag_ramp;
    int32_t kernel_mode; /* 0 physical, 1 constant kernel */
    int32_t settle_form; /* 0: v_z = -z Omega St ; 1: -z Omega St/(1+St) */
    int32_t dv_flags;    /* ORC_DV_* mask */
    int32_t tr_flags;    /* ORC_TR_* mask */
    /* a tabulated (non-power-law) gas disk, reading: gas_n knots r_k, Sigma_k,
       T_k at gas_tab[3k .. 3k+2], r_k increasing; 0 knots: the power laws */
    const double *gas_tab;
    int32_t gas_n;
} orc_params;

/* ======================================================================== */
/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11, "Parallel random      */
/* numbers: as easy as 1, 2, 3"), written from the published round function. */
/* ======================================================================== */
static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        orc_mulhilo64(M0, c0, &hi0, &lo0);
        orc_mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform on (0,1): the top 53 bits plus one half, times 2^-53 */
static double orc_u01(uint64_t x) { return ((double)(x >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

static void orc_draw(uint64_t seed, uint64_t disk, uint64_t c0, uint64_t c1, uint64_t c2, uint64_t tag, double u[4])
{
    uint64_t ctr[4] = {c0, c1, c2, tag}, key[2] = {seed, disk}, x[4];
    orc_philox4x64_10(ctr, key, x);
    for (int k = 0; k < 4; ++k) u[k] = orc_u01(x[k]);
}

/* ======================================================================== */
/* Gas disk: static power law, vertically isothermal (Summary; Benchmark).  */
/* ======================================================================== */
typedef struct {
    double Sigma, T, cs, Omega, H, rho, vth, lambda, nu, etavk, D, vg2, St_eta, asw;
    double p, q; /* local slopes -dln Sigma/dln r, -dln T/dln r */
} orc_gas;

/* Knot k's ln Sigma, ln T and the slopes p_k = -(ln Sigma_{k+1} - ln Sigma_k) /
 * (ln r_{k+1} - ln r_k), q_k likewise, of segment [r_k, r_{k+1}) (the last
 * segment's slopes are repeated at the last knot).  Between knots Sigma and T
 * are linear in log-log: Sigma(r) = exp(ln Sigma_k - p_k (ln r - ln r_k)) with
 * k the last knot not above r (the first below r_0); beyond the ends the end
 * segments extend.  A power law is therefore reproduced exactly. */
void orc_gas_table_prep(int32_t n, const double *tab, double *lnr, double *lnS, double *lnT, double *ps, double *qs)
{
    for (int32_t k = 0; k < n; ++k) {
        lnr[k] = log(tab[3 * k]);
        lnS[k] = log(tab[3 * k + 1]);
        lnT[k] = log(tab[3 * k + 2]);
    }
    for (int32_t k = 0; k + 1 < n; ++k) {
        const double dl = lnr[k + 1] - lnr[k];
        ps[k] = -(lnS[k + 1] - lnS[k]) / dl;
        qs[k] = -(lnT[k + 1] - lnT[k]) / dl;
    }
    ps[n - 1] = ps[n - 2];
    qs[n - 1] = qs[n - 2];
}

/* Sigma, T and the local slopes at r from the table */
static void orc_gas_table(const orc_params *P, double r, double *Sigma, double *T, double *p, double *q)
{
    const int32_t n = P->gas_n;
    double lnr[n], lnS[n], lnT[n], ps[n], qs[n];
    orc_gas_table_prep(n, P->gas_tab, lnr, lnS, lnT, ps, qs);
    int32_t k = 0;
    while (k + 2 < n && P->gas_tab[3 * (k + 1)] <= r) ++k; /* segment [r_k, r_k+1), ends extended */
    const double dl = log(r) - lnr[k];
    *Sigma = exp(lnS[k] - ps[k] * dl);
    *T = exp(lnT[k] - qs[k] * dl);
    *p = ps[k];
    *q = qs[k];
}

static orc_gas orc_gas_at(const orc_params *P, double r, double z)
{
    orc_gas g;
    if (P->gas_n >= 2) {
        orc_gas_table(P, r, &g.Sigma, &g.T, &g.p, &g.q);
    } else {
        double x = r / ORC_AU;
        g.Sigma = P->sigma0 * pow(x, -P->p);
        g.T = P->T0 * pow(x, -P->q);
        g.p = P->p;
        g.q = P->q;
    }
    g.cs = sqrt(ORC_KB * g.T / (P->mu * ORC_MP));
    g.Omega = sqrt(P->m_star * ORC_GM_SUN / (r * r * r));
    g.H = g.cs / g.Omega;
    double rho_mid = g.Sigma / (sqrt(2.0 * ORC_PI) * g.H);
    g.rho = rho_mid * exp(-z * z / (2.0 * g.H * g.H));
    g.vth = sqrt(8.0 / ORC_PI) * g.cs;
    g.lambda = P->mu * ORC_MP / (g.rho * P->sigma_h2);
    g.nu = 0.5 * g.vth * g.lambda;
    /* eta v_K = -(1/2) c_s^2/(Omega r) dlnP/dlnr with the midplane pressure
       P ~ r^-(p + (3+q)/2) (reading: midplane gradient at every height). */
    g.etavk = 0.5 * g.cs * g.cs / (g.Omega * r) * (g.p + 0.5 * (3.0 + g.q));
    g.D = P->alpha * g.cs * g.H;              /* Schmidt number 1 (reading) */
    g.vg2 = 1.5 * P->alpha * g.cs * g.cs;     /* Ormel & Cuzzi V_g^2 (reading) */
    g.St_eta = 1.0 / sqrt(g.D / g.nu);        /* Re^-1/2, Re = alpha c_s H / nu */
    g.asw = 2.25 * g.lambda;                  /* Epstein/Stokes switch a = 9 lambda/4 */
    return g;
}

/* ======================================================================== */
/* Particle: radius and Stokes number (Epstein below 9 lambda/4, Stokes at   */
/* and above it).                                                            */
/* ======================================================================== */
typedef struct {
    double m, a, St;
    int stokes; /* 1 when a >= 9 lambda / 4 */
} orc_part;

static double orc_radius(const orc_params *P, double m) { return cbrt(3.0 * m / (4.0 * ORC_PI * P->rho_s)); }

static orc_part orc_particle(const orc_params *P, const orc_gas *g, double m)
{
    orc_part q;
    q.m = m;
    q.a = orc_radius(P, m);
    if (q.a < g->asw) {
        q.stokes = 0;
        q.St = P->rho_s * q.a / (g->rho * g->vth) * g->Omega;
    } else {
        q.stokes = 1;
        q.St = 2.0 * P->rho_s * q.a * q.a / (9.0 * g->nu * g->rho) * g->Omega;
    }
    return q;
}

/* |St_i - St_j| without subtracting two nearly equal Stokes numbers.
 * a_i - a_j = (3/(4 pi rho_s)) (m_i - m_j) / (a_i^2 + a_i a_j + a_j^2) is the
 * factored difference of cubes; the Stokes-law and mixed cases follow from
 * St = C_ep a (Epstein) and St = C_st a^2 (Stokes) with C_ep = C_st * 9 lambda/4. */
static double orc_dst(const orc_params *P, const orc_gas *g, const orc_part *x, const orc_part *y)
{
    const double cm = 3.0 / (4.0 * ORC_PI * P->rho_s);
    const double Cep = P->rho_s / (g->rho * g->vth) * g->Omega;
    const double Cst = 2.0 * P->rho_s / (9.0 * g->nu * g->rho) * g->Omega;
    double da = cm * fabs(x->m - y->m) / ((x->a * x->a + y->a * y->a) + x->a * y->a);
    if (!x->stokes && !y->stokes) return Cep * da;
    if (x->stokes && y->stokes) return Cst * (x->a + y->a) * da;
    const orc_part *s = x->stokes ? x : y; /* the Stokes-law particle, a_s >= a_sw */
    double asw = g->asw;
    double msw = 4.0 * ORC_PI * P->rho_s / 3.0 * asw * asw * asw;
    double da_sw = cm * (s->m - msw) / (s->a * s->a + s->a * asw + asw * asw);
    return Cst * (s->a * da_sw + asw * da);
}

/* Ormel & Cuzzi (2007) turbulent relative velocity squared, closed forms of
 * the three regimes with St1 the larger Stokes number (reading: V_g^2 =
 * 3/2 alpha c_s^2, St_eta = Re^-1/2, boundaries taken with ">="). */
static double orc_dv2_turb(const orc_gas *g, double Si, double Sj, double D)
{
    double S1 = Si > Sj ? Si : Sj, S2 = Si > Sj ? Sj : Si;
    if (S1 < g->St_eta) {
        double s = S1 + S2;
        if (s <= 0.0) return 0.0;
        /* vg2 (S1-S2)/(S1+S2) [S1^2/(S1+St_eta) - S2^2/(S2+St_eta)], factored */
        return g->vg2 * D * D * (S1 * S2 + g->St_eta * s) / (s * (S1 + g->St_eta) * (S2 + g->St_eta));
    } else if (S1 < 1.0) {
        double eps = S2 / S1;
        return g->vg2 * S1 *
               (2.0 * ORC_YA - (1.0 + eps) +
                2.0 / (1.0 + eps) * (1.0 / (1.0 + ORC_YA) + eps * eps * eps / (ORC_YA + eps)));
    } else {
        return g->vg2 * (1.0 / (1.0 + S1) + 1.0 / (1.0 + S2));
    }
}

/* Relative velocity of a pair at the cell centre (r_c, z_c) from Brownian
 * motion, turbulence, radial drift, azimuthal drift and settling, summed in
 * quadrature; all differences in the factored forms. */
static double orc_dv_pair(const orc_params *P, const orc_gas *g, double zc, const orc_part *x, const orc_part *y,
                          double terms[5])
{
    double D = orc_dst(P, g, x, y);
    double Si = x->St, Sj = y->St;
    double den = (1.0 + Si * Si) * (1.0 + Sj * Sj);
    double t[5];
    t[0] = 8.0 * ORC_KB * g->T / ORC_PI * (1.0 / x->m + 1.0 / y->m);
    t[1] = orc_dv2_turb(g, Si, Sj, D);
    double vr = 2.0 * g->etavk * D * (1.0 - Si * Sj) / den;
    t[2] = vr * vr;
    double vp = g->etavk * D * (Si + Sj) / den;
    t[3] = vp * vp;
    double vz = g->Omega * fabs(zc) * D;
    if (P->settle_form == 1) vz = vz / ((1.0 + Si) * (1.0 + Sj));
    t[4] = vz * vz;
    double s = 0.0;
    for (int k = 0; k < 5; ++k) {
        if (!(P->dv_flags & (1 << k))) t[k] = 0.0;
        s += t[k];
        if (terms) terms[k] = t[k];
    }
    return sqrt(s);
}

/* Collision kernel K = pi (a_i + a_j)^2 dv (constant mode: K_const). */
static double orc_kernel(const orc_params *P, const orc_gas *g, double zc, const orc_part *x, const orc_part *y,
                         double *dv_out)
{
    if (P->kernel_mode == 1) {
        if (dv_out) *dv_out = 0.0;
        return P->K_const;
    }
    double dv = orc_dv_pair(P, g, zc, x, y, NULL);
    if (dv_out) *dv_out = dv;
    double s = x->a + y->a;
    return ORC_PI * s * s * dv;
}

/* Zsom & Dullemond weight: swarm j's number density M_j/(m_j V) times the
 * grouping factor min(1, m_j/(dm m_i)); dm = 0 switches grouping off. */
static double orc_weight(const orc_params *P, double V, double mi, double mj, double Mj)
{
    double inv = 1.0 / mj;
    if (P->dm_group > 0.0) {
        double g = 1.0 / (P->dm_group * mi);
        if (g < inv) inv = g;
    }
    return Mj / V * inv;
}

/* ======================================================================== */
/* Exported probes (for the tests)                                          */
/* ======================================================================== */
/* 14 gas quantities per (r, z): Sigma T cs Omega H rho vth lambda nu etavk D vg2 St_eta asw */
void orc_gas_probe(const orc_params *P, int64_t n, const double *r, const double *z, double *out)
{
    for (int64_t k = 0; k < n; ++k) {
        orc_gas g = orc_gas_at(P, r[k], z[k]);
        double v[14] = {g.Sigma, g.T, g.cs, g.Omega, g.H, g.rho, g.vth, g.lambda, g.nu, g.etavk, g.D, g.vg2, g.St_eta, g.asw};
        memcpy(out + 14 * k, v, sizeof v);
    }
}

/* radius, Stokes number and regime flag of masses m at gas position (r, z) */
void orc_particle_probe(const orc_params *P, double r, double z, int64_t n, const double *m, double *a, double *St,
                        int32_t *stokes)
{
    orc_gas g = orc_gas_at(P, r, z);
    for (int64_t k = 0; k < n; ++k) {
        orc_part q = orc_particle(P, &g, m[k]);
        a[k] = q.a;
        St[k] = q.St;
        stokes[k] = q.stokes;
    }
}

/* pair quantities at the cell centre: dv, K, and the five squared terms */
void orc_pair_probe(const orc_params *P, double rc, double zc, int64_t n, const double *mi, const double *mj,
                    double *dv, double *K, double *terms, double *dst)
{
    orc_gas g = orc_gas_at(P, rc, zc);
    for (int64_t k = 0; k < n; ++k) {
        orc_part x = orc_particle(P, &g, mi[k]), y = orc_particle(P, &g, mj[k]);
        double t[5];
        dv[k] = orc_dv_pair(P, &g, zc, &x, &y, t);
        K[k] = orc_kernel(P, &g, zc, &x, &y, NULL);
        if (terms) memcpy(terms + 5 * k, t, sizeof t);
        if (dst) dst[k] = orc_dst(P, &g, &x, &y);
    }
}

/* full rate matrix r_ij (row-major n x n) and row sums of one cell */
void orc_rate_matrix(const orc_params *P, double rc, double zc, double V, int64_t n, const double *m,
                     const double *M, double *rate, double *R)
{
    orc_gas g = orc_gas_at(P, rc, zc);
    if (P->kernel_mode == 1) V = P->V_const;
    for (int64_t i = 0; i < n; ++i) {
        orc_part x = orc_particle(P, &g, m[i]);
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            orc_part y = orc_particle(P, &g, m[j]);
            double v = orc_kernel(P, &g, zc, &x, &y, NULL) * orc_weight(P, V, m[i], m[j], M[j]);
            if (rate) rate[i * n + j] = v;
            s += v;
        }
        if (R) R[i] = s;
    }
}

/* mass-weighted fragment draw on [m0, mmax] from n(m) ~ m^-xi: the inverse of
   the CDF (m^e - m0^e)/(mmax^e - m0^e), e = 2 - xi, written as
   m = m0 [1 + u ((mmax/m0)^e - 1)]^(1/e) with expm1/log1p so that it keeps
   its relative precision when mmax is close to m0 */
static double orc_fragment(const orc_params *P, double m0, double mmax, double u)
{
    if (mmax <= m0) return m0;
    double e = 2.0 - P->frag_xi, L = log(mmax / m0);
    if (fabs(e) < 1e-12) return m0 * exp(u * L);
    return m0 * exp(log1p(u * expm1(e * L)) / e);
}

double orc_fragment_probe(const orc_params *P, double m0, double mmax, double u) { return orc_fragment(P, m0, mmax, u); }

static double orc_outcome(const orc_params *P, double mi, double mj, double dv, double m0, double u, int *kind);
double orc_outcome_probe(const orc_params *P, double mi, double mj, double dv, double m0, double u, int32_t *kind)
{
    int k = 0;
    const double mn = orc_outcome(P, mi, mj, dv, m0, u, &k);
    *kind = k;
    return mn;
}

static double orc_monomer_mass(const orc_params *P)
{
    if (P->m_init > 0.0) return P->m_init;
    return 4.0 * ORC_PI / 3.0 * P->rho_s * P->a_mono * P->a_mono * P->a_mono;
}

/* ======================================================================== */
/* One cell: the event-driven Zsom & Dullemond loop from t0 to t_end.       */
/* ======================================================================== */
typedef struct {
    int32_t i, j, outcome; /* outcome: 0 stick, 1 fragment, 2 erode */
    double t, m_new;
} orc_event;

/* outcome of representative i meeting a particle of swarm j; returns m_i new */
/* Outcome of representative i meeting a particle of swarm j at relative
 * velocity dv, u the event's fourth uniform.  Below v_frag the pair sticks;
 * with frag_ramp = delta > 0 (reading: a linear ramp, the paper names the
 * outcomes but not their parameters) the fragmentation probability rises
 * linearly from 0 at v_lo = v_frag (1 - delta) to 1 at v_frag, decided by
 * u < p, and u / p (uniform again) then draws the fragment. */
static double orc_outcome(const orc_params *P, double mi, double mj, double dv, double m0, double u, int *kind)
{
    double gain = mj;
    if (P->dm_group > 0.0 && P->dm_group * mi > mj) gain = P->dm_group * mi; /* N_g m_j */
    const double vlo = P->v_frag * (1.0 - P->frag_ramp);
    int stick = P->kernel_mode == 1 || dv < vlo;
    if (!stick && dv < P->v_frag) {
        const double p = (dv - vlo) / (P->v_frag - vlo);
        if (u < p)
            u = u / p;
        else
            stick = 1;
    }
    if (stick) {
        *kind = 0;
        return mi + gain;
    }
    double big = mi > mj ? mi : mj, small = mi > mj ? mj : mi;
    if (big >= P->erosion_ratio * small) {
        *kind = 2;
        if (mi >= mj) {
            double mnew = mi - P->erosion_chi * gain;
            return mnew > m0 ? mnew : m0;
        }
        return orc_fragment(P, m0, mi, u);
    }
    *kind = 1;
    return orc_fragment(P, m0, big, u);
}

/* A tracked property of each swarm (a composition fraction q), carried by its
 * representative particle (the particle histories of the Statement of Need
 * section; reading, the paper gives no rule): sticking mixes by mass, q_i <- (m_i q_i + g q_j) /
 * (m_i + g), g = N_g m_j the absorbed mass; fragmentation gives the pair's
 * mass-weighted mixture; erosion leaves the larger body's q as it was and turns
 * the smaller one into debris of itself and the chipped mass, chi times its own:
 * (q_i + chi q_j) / (1 + chi).  mi, mj before the event; mnew after it. */
double orc_tracer_update(const orc_params *P, double mi, double mj, double qi, double qj, double mnew, int32_t kind)
{
    if (kind == 0) {
        double gain = mj;
        if (P->dm_group > 0.0 && P->dm_group * mi > mj) gain = P->dm_group * mi;
        return (mi * qi + gain * qj) / mnew;
    }
    if (kind == 1) return (mi * qi + mj * qj) / (mi + mj);
    if (mi >= mj) return qi;
    return (qi + P->erosion_chi * qj) / (1.0 + P->erosion_chi);
}

static int orc_collide_cell_impl(const orc_params *P, double rc, double zc, double V, int64_t n, double *m,
                                 const double *M, double *q, double t0, double t_end, uint64_t seed, uint64_t disk,
                                 uint64_t step, uint64_t cell, int64_t max_events, int64_t rebuild_every,
                                 int64_t *events_out, double *R_out, orc_event *evlog, int64_t log_cap)
{
    int status = ORC_OK;
    int64_t ev = 0;
    if (events_out) *events_out = 0;
    if (n <= 0) return ORC_OK;
    if (P->kernel_mode == 1) V = P->V_const;
    if (rebuild_every <= 0) rebuild_every = 4 * n; /* reading: full rebuild every 4n events */
    orc_gas g = orc_gas_at(P, rc, zc);
    double m0 = orc_monomer_mass(P);
    orc_part *pt = (orc_part *)malloc(sizeof(orc_part) * n);
    double *R = (double *)malloc(sizeof(double) * n);
    double *row = (double *)malloc(sizeof(double) * n);   /* r_ik, i fixed */
    double *colo = (double *)malloc(sizeof(double) * n);  /* r_ki before the event */
    for (int64_t k = 0; k < n; ++k) pt[k] = orc_particle(P, &g, m[k]);

#define ORC_REBUILD()                                                                     \
    for (int64_t a_ = 0; a_ < n; ++a_) {                                                  \
        double s_ = 0.0;                                                                  \
        for (int64_t b_ = 0; b_ < n; ++b_)                                                \
            s_ += orc_kernel(P, &g, zc, &pt[a_], &pt[b_], NULL) *                         \
                  orc_weight(P, V, pt[a_].m, pt[b_].m, M[b_]);                            \
        R[a_] = s_;                                                                       \
    }
    ORC_REBUILD();
    double t = t0;
    for (;;) {
        double Rtot = 0.0;
        for (int64_t k = 0; k < n; ++k) Rtot += R[k];
        if (!(Rtot > 0.0)) break; /* idle cell */
        if (ev >= max_events) {
            status = ORC_ETIMEOUT;
            break;
        }
        double u[4];
        orc_draw(seed, disk, (uint64_t)ev, cell, step, ORC_TAG_COLLIDE, u);
        double tau = -log(u[0]) / Rtot;
        if (t + tau >= t_end) break; /* memoryless: the crossing event is discarded */
        t += tau;
        /* choose i: first k whose inclusive prefix exceeds u1 R_tot */
        double target = u[1] * Rtot, acc = 0.0;
        int64_t i = -1, lastpos = -1;
        for (int64_t k = 0; k < n; ++k) {
            acc += R[k];
            if (R[k] > 0.0) lastpos = k;
            if (acc > target) { i = k; break; }
        }
        if (i < 0) i = lastpos;
        /* row i and column i before the event */
        double Ri = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double K = orc_kernel(P, &g, zc, &pt[i], &pt[k], NULL);
            row[k] = K * orc_weight(P, V, pt[i].m, pt[k].m, M[k]);
            colo[k] = K * orc_weight(P, V, pt[k].m, pt[i].m, M[i]);
            Ri += row[k];
        }
        /* choose j: first k whose inclusive prefix over row i exceeds u2 R_i */
        target = u[2] * Ri;
        acc = 0.0;
        int64_t j = -1;
        lastpos = -1;
        for (int64_t k = 0; k < n; ++k) {
            acc += row[k];
            if (row[k] > 0.0) lastpos = k;
            if (acc > target) { j = k; break; }
        }
        if (j < 0) j = lastpos;
        double dv = 0.0;
        orc_kernel(P, &g, zc, &pt[i], &pt[j], &dv);
        int kind = 0;
        double mnew = orc_outcome(P, pt[i].m, pt[j].m, dv, m0, u[3], &kind);
        if (evlog && ev < log_cap) {
            evlog[ev].i = (int32_t)i; evlog[ev].j = (int32_t)j; evlog[ev].outcome = kind;
            evlog[ev].t = t; evlog[ev].m_new = mnew;
        }
        if (q) q[i] = orc_tracer_update(P, pt[i].m, pt[j].m, q[i], q[j], mnew, kind);
        pt[i] = orc_particle(P, &g, mnew);
        /* only row i and column i change: R_k += r_ki(new) - r_ki(old), R_i afresh */
        double Rin = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            double K = orc_kernel(P, &g, zc, &pt[i], &pt[k], NULL);
            Rin += K * orc_weight(P, V, pt[i].m, pt[k].m, M[k]);
            if (k != i) {
                double cn = K * orc_weight(P, V, pt[k].m, pt[i].m, M[i]);
                R[k] += cn - colo[k];
            }
        }
        R[i] = Rin;
        ++ev;
        if (ev % rebuild_every == 0) { ORC_REBUILD(); }
    }
#undef ORC_REBUILD
    for (int64_t k = 0; k < n; ++k) m[k] = pt[k].m;
    if (R_out) memcpy(R_out, R, sizeof(double) * n);
    if (events_out) *events_out = ev;
    free(pt); free(R); free(row); free(colo);
    return status;
}

int orc_collide_cell(const orc_params *P, double rc, double zc, double V, int64_t n, double *m, const double *M,
                     double t0, double t_end, uint64_t seed, uint64_t disk, uint64_t step, uint64_t cell,
                     int64_t max_events, int64_t rebuild_every, int64_t *events_out, double *R_out,
                     orc_event *evlog, int64_t log_cap)
{
    return orc_collide_cell_impl(P, rc, zc, V, n, m, M, NULL, t0, t_end, seed, disk, step, cell, max_events,
                                 rebuild_every, events_out, R_out, evlog, log_cap);
}

/* the same with the tracer column q (updated in place) */
int orc_collide_cell_q(const orc_params *P, double rc, double zc, double V, int64_t n, double *m, const double *M,
                       double *q, double t0, double t_end, uint64_t seed, uint64_t disk, uint64_t step, uint64_t cell,
                       int64_t max_events, int64_t rebuild_every, int64_t *events_out, double *R_out,
                       orc_event *evlog, int64_t log_cap)
{
    return orc_collide_cell_impl(P, rc, zc, V, n, m, M, q, t0, t_end, seed, disk, step, cell, max_events,
                                 rebuild_every, events_out, R_out, evlog, log_cap);
}

/* ======================================================================== */
/* Initial state (workload recipe): equal swarm masses, r drawn from the    */
/* dust-mass CDF ~ r^(2-p), z ~ N(0, H_g(r)), monomers.  The draw follows   */
/* the power-law disk even when a gas table is set (reading).              */
/* ======================================================================== */
double orc_disk_dust_mass(const orc_params *P)
{
    if (P->M_total > 0.0) return P->M_total;
    double e = 2.0 - P->p, ri = P->r_in / ORC_AU, ro = P->r_out / ORC_AU;
    double I = fabs(e) < 1e-12 ? log(ro / ri) : (pow(ro, e) - pow(ri, e)) / e; /* in AU^2 */
    return P->dust_to_gas * 2.0 * ORC_PI * P->sigma0 * I * ORC_AU * ORC_AU;
}

void orc_init_disk(const orc_params *P, int64_t N, uint64_t seed, uint64_t disk, double *m, double *M, double *r,
                   double *z, uint32_t *id)
{
    double m0 = orc_monomer_mass(P), Mi = orc_disk_dust_mass(P) / (double)N;
    double e = 2.0 - P->p;
    for (int64_t k = 0; k < N; ++k) {
        double u[4];
        orc_draw(seed, disk, (uint64_t)k, 0, 0, ORC_TAG_INIT, u);
        double rr;
        if (fabs(e) < 1e-12)
            rr = P->r_in * exp(u[0] * log(P->r_out / P->r_in));
        else {
            double lo = pow(P->r_in, e), hi = pow(P->r_out, e);
            rr = pow(lo + u[0] * (hi - lo), 1.0 / e);
        }
        double xi = sqrt(-2.0 * log(u[1])) * cos(2.0 * ORC_PI * u[2]);
        orc_params Pw = *P;
        Pw.gas_n = 0;
        orc_gas g = orc_gas_at(&Pw, rr, 0.0);
        r[k] = rr;
        z[k] = g.H * xi;
        m[k] = m0;
        M[k] = Mi;
        id[k] = (uint32_t)k;
    }
}

/* ======================================================================== */
/* Equal-count regrid: radial zones by (r, id) rank, cells by (z, id) rank. */
/* ======================================================================== */
typedef struct {
    double key;
    uint32_t id;
    int64_t src;
} orc_key;

static int orc_cmp_key(const void *a, const void *b)
{
    const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* count of group k when N items are split into G groups of equal count,
   the first N mod G groups taking one extra */
static int64_t orc_group_size(int64_t N, int64_t G, int64_t k) { return N / G + (k < N % G ? 1 : 0); }

/* Reorders (m, M, r, z, id) in place into cell order (cells radial-major,
 * z-minor; dead particles, r = +inf, at the tail ordered by id).
 * Outputs: perm[new] = old index, cell_off[n_r*n_z+1], cell_b[6 per cell:
 * r_lo r_hi z_lo z_hi r_c z_c], cell_V, and the alive count. */
int orc_regrid(const orc_params *P, int32_t n_r, int32_t n_z, int64_t N, double *m, double *M, double *r, double *z,
               uint32_t *id, int64_t *perm, int64_t *cell_off, double *cell_b, double *cell_V, int64_t *n_alive)
{
    if (n_r <= 0 || n_z <= 0) return ORC_EINVAL;
    for (int64_t k = 0; k < N; ++k) {
        if (isnan(r[k]) || isnan(z[k])) return ORC_ENAN;
        if (r[k] == 0.0) r[k] = 0.0; /* -0.0 -> +0.0 */
        if (z[k] == 0.0) z[k] = 0.0;
    }
    orc_key *kr = (orc_key *)malloc(sizeof(orc_key) * (N > 0 ? N : 1));
    for (int64_t k = 0; k < N; ++k) { kr[k].key = r[k]; kr[k].id = id[k]; kr[k].src = k; }
    qsort(kr, (size_t)N, sizeof(orc_key), orc_cmp_key);
    int64_t Na = 0;
    while (Na < N && isfinite(kr[Na].key)) ++Na;
    int64_t ncell = (int64_t)n_r * n_z;
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (N > 0 ? N : 1));
    orc_key *kz = (orc_key *)malloc(sizeof(orc_key) * (N > 0 ? N : 1));
    int64_t zone_start = 0, pos = 0;
    int64_t nonempty_r = Na < n_r ? Na : n_r;
    for (int64_t zk = 0; zk < n_r; ++zk) {
        int64_t nk = orc_group_size(Na, n_r, zk);
        /* radial bounds of zone zk from the global (r, id)-sorted sequence */
        double rlo = 0.0, rhi = 0.0;
        if (nk > 0) {
            double rf = kr[zone_start].key, rl = kr[zone_start + nk - 1].key;
            if (Na == 1) {
                orc_gas g = orc_gas_at(P, rf, 0.0);
                rlo = rf - 0.5 * g.H;
                rhi = rf + 0.5 * g.H;
            } else {
                if (zk == 0) rlo = rf - (kr[1].key - rf) * 0.5;
                else rlo = (kr[zone_start - 1].key + rf) * 0.5;
                if (zk + 1 < nonempty_r) rhi = (rl + kr[zone_start + nk].key) * 0.5;
                else rhi = rl + (rl - kr[Na - 2].key) * 0.5;
            }
        }
        double rcen = (rlo + rhi) * 0.5;
        /* sort the zone by (z, id) */
        for (int64_t s = 0; s < nk; ++s) {
            int64_t src = kr[zone_start + s].src;
            kz[s].key = z[src]; kz[s].id = id[src]; kz[s].src = src;
        }
        qsort(kz, (size_t)nk, sizeof(orc_key), orc_cmp_key);
        int64_t nonempty_z = nk < n_z ? nk : n_z, cs = 0;
        for (int64_t c = 0; c < n_z; ++c) {
            int64_t cell = zk * n_z + c, nc = orc_group_size(nk, n_z, c);
            cell_off[cell] = pos + cs;
            double zlo = 0.0, zhi = 0.0;
            if (nc > 0) {
                double zf = kz[cs].key, zl = kz[cs + nc - 1].key;
                if (nk == 1) {
                    orc_gas g = orc_gas_at(P, rcen, 0.0);
                    zlo = zf - 0.5 * g.H;
                    zhi = zf + 0.5 * g.H;
                } else {
                    if (c == 0) zlo = zf - (kz[1].key - zf) * 0.5;
                    else zlo = (kz[cs - 1].key + zf) * 0.5;
                    if (c + 1 < nonempty_z) zhi = (zl + kz[cs + nc].key) * 0.5;
                    else zhi = zl + (zl - kz[nk - 2].key) * 0.5;
                }
            }
            double *b = cell_b + 6 * cell;
            b[0] = nc > 0 ? rlo : 0.0;
            b[1] = nc > 0 ? rhi : 0.0;
            b[2] = zlo;
            b[3] = zhi;
            b[4] = (b[0] + b[1]) * 0.5;
            b[5] = (zlo + zhi) * 0.5;
            double A = b[1] * b[1] - b[0] * b[0];
            cell_V[cell] = ORC_PI * A * (zhi - zlo);
            cs += nc;
        }
        for (int64_t s = 0; s < nk; ++s) order[pos + s] = kz[s].src;
        pos += nk;
        zone_start += nk;
    }
    cell_off[ncell] = pos;
    for (int64_t k = Na; k < N; ++k) order[k] = kr[k].src; /* dead, by id */
    double *tmp = (double *)malloc(sizeof(double) * (N > 0 ? N : 1));
    uint32_t *tid = (uint32_t *)malloc(sizeof(uint32_t) * (N > 0 ? N : 1));
#define ORC_PERMUTE(arr)                                   \
    for (int64_t k = 0; k < N; ++k) tmp[k] = arr[order[k]]; \
    memcpy(arr, tmp, sizeof(double) * N);
    ORC_PERMUTE(m);
    ORC_PERMUTE(M);
    ORC_PERMUTE(r);
    ORC_PERMUTE(z);
#undef ORC_PERMUTE
    for (int64_t k = 0; k < N; ++k) tid[k] = id[order[k]];
    memcpy(id, tid, sizeof(uint32_t) * N);
    if (perm) memcpy(perm, order, sizeof(int64_t) * N);
    if (n_alive) *n_alive = Na;
    free(kr); free(kz); free(order); free(tmp); free(tid);
    return ORC_OK;
}

/* ======================================================================== */
/* Transport of one particle over dt: radial Ito drift + diffusion kick and */
/* an exact Ornstein-Uhlenbeck step in z for frozen coefficients (reading). */
/* ======================================================================== */
static void orc_transport_one(const orc_params *P, double *r, double *z, double m, uint32_t idv, double dt,
                              uint64_t seed, uint64_t disk, uint64_t step, int *removed)
{
    double u[4];
    orc_draw(seed, disk, (uint64_t)idv, 0, step, ORC_TAG_TRANSPORT, u);
    double rho_bm = sqrt(-2.0 * log(u[0]));
    double xi1 = rho_bm * cos(2.0 * ORC_PI * u[1]);
    double xi2 = rho_bm * sin(2.0 * ORC_PI * u[1]);
    double r0 = *r, z0 = *z;
    orc_gas g = orc_gas_at(P, r0, z0);
    orc_gas gs = (P->tr_flags & ORC_TR_ST_MIDPLANE) ? orc_gas_at(P, r0, 0.0) : g;
    orc_part q = orc_particle(P, &gs, m);
    double St = q.St;
    double rn = r0, zn = z0;
    if (P->tr_flags & ORC_TR_RADIAL) {
        double vr = -2.0 * g.etavk * St / (1.0 + St * St);
        /* (1/(r rho_g)) d/dr (r D rho_g) for D ~ r^(3/2-q), rho_g(r, z) */
        double vD = g.D / r0 * (1.0 - g.p - 0.5 * g.q + z0 * z0 / (g.H * g.H) * 0.5 * (3.0 - g.q));
        rn = r0 + (vr + vD) * dt + sqrt(2.0 * g.D * dt) * xi1;
    }
    if (P->tr_flags & ORC_TR_VERTICAL) {
        double sv = P->settle_form == 1 ? St / (1.0 + St) : St;
        double k = g.Omega * (sv + P->alpha);
        double e = exp(-k * dt);
        zn = z0 * e + sqrt(g.D * (-expm1(-2.0 * k * dt)) / k) * xi2;
    }
    *removed = 0;
    if (rn < P->r_in) {
        *removed = 1;
        rn = INFINITY;
    } else if (rn > P->r_out) {
        rn = 2.0 * P->r_out - rn;
    }
    *r = rn;
    *z = zn;
}

/* transport every alive particle; removed ones get r = +inf and their swarm
   mass is added to *accreted */
void orc_transport(const orc_params *P, int64_t N, double *r, double *z, const double *m, const double *M,
                   const uint32_t *id, double dt, uint64_t seed, uint64_t disk, uint64_t step, double *accreted)
{
    double acc = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        if (!isfinite(r[k])) continue;
        int rem = 0;
        orc_transport_one(P, &r[k], &z[k], m[k], id[k], dt, seed, disk, step, &rem);
        if (rem) acc += M[k];
    }
    if (accreted) *accreted += acc;
}

/* ---- adaptive time step (reading; the paper states no rule) -------------
 * dt = min(dt_max, C min_c (r_hi - r_lo)_c / max_i |v_r,i|): a drifting
 * particle crosses at most the fraction C of the narrowest cell in one step.
 * The minimum runs over the cells that hold particles, the maximum over the
 * live particles, with v_r = -2 eta v_K St / (1 + St^2) the radial drift of the
 * transport step (St at the particle, or at the midplane with
 * ORC_TR_ST_MIDPLANE).  Without radial transport (or in the constant-kernel
 * mode) nothing drifts and dt = dt_max. */
double orc_adaptive_dt(const orc_params *P, int64_t ncell, const int64_t *cell_off, const double *cell_b,
                       int64_t N, const double *m, const double *r, const double *z, double dt_max, double courant)
{
    if (P->kernel_mode != 0 || !(P->tr_flags & ORC_TR_RADIAL)) return dt_max;
    double dr_min = INFINITY, v_max = 0.0;
    for (int64_t c = 0; c < ncell; ++c)
        if (cell_off[c + 1] > cell_off[c]) {
            double w = cell_b[6 * c + 1] - cell_b[6 * c];
            if (w < dr_min) dr_min = w;
        }
    for (int64_t k = 0; k < N; ++k) {
        if (!isfinite(r[k])) continue;
        orc_gas g = orc_gas_at(P, r[k], z[k]);
        orc_gas gs = (P->tr_flags & ORC_TR_ST_MIDPLANE) ? orc_gas_at(P, r[k], 0.0) : g;
        double St = orc_particle(P, &gs, m[k]).St;
        double v = fabs(-2.0 * g.etavk * St / (1.0 + St * St));
        if (v > v_max) v_max = v;
    }
    if (!(v_max > 0.0)) return dt_max;
    double dt = courant * dr_min / v_max;
    return dt < dt_max ? dt : dt_max;
}

/* ======================================================================== */
/* Whole-disk driver: regrid -> collide every cell to t + dt -> transport.  */
/* ======================================================================== */
static int orc_collide_all_impl(const orc_params *P, int32_t n_r, int32_t n_z, const int64_t *cell_off,
                                const double *cell_b, const double *cell_V, double *m, const double *M, double *q,
                                double t0, double t_end, uint64_t seed, uint64_t disk, uint64_t step,
                                int64_t max_events, int64_t rebuild_every, int64_t *cell_events, int32_t nthreads)
{
    int64_t ncell = (int64_t)n_r * n_z;
    int status = ORC_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t c = 0; c < ncell; ++c) {
        int64_t off = cell_off[c], n = cell_off[c + 1] - cell_off[c], ev = 0;
        int st = orc_collide_cell_impl(P, cell_b[6 * c + 4], cell_b[6 * c + 5], cell_V[c], n, m + off, M + off,
                                       q ? q + off : NULL, t0, t_end, seed, disk, step, (uint64_t)c, max_events,
                                       rebuild_every, &ev, NULL, NULL, 0);
        if (cell_events) cell_events[c] = ev;
        if (st != ORC_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
            status = st;
        }
    }
    return status;
}

int orc_collide_all(const orc_params *P, int32_t n_r, int32_t n_z, const int64_t *cell_off, const double *cell_b,
                    const double *cell_V, double *m, const double *M, double t0, double t_end, uint64_t seed,
                    uint64_t disk, uint64_t step, int64_t max_events, int64_t rebuild_every, int64_t *cell_events,
                    int32_t nthreads)
{
    return orc_collide_all_impl(P, n_r, n_z, cell_off, cell_b, cell_V, m, M, NULL, t0, t_end, seed, disk, step,
                                max_events, rebuild_every, cell_events, nthreads);
}

/* n_steps steps of length dt from time t0 and step index step0; q (or NULL)
 * is the tracer column, reordered with the particles by every regrid */
static int orc_run_impl(const orc_params *P, int32_t n_r, int32_t n_z, int64_t N, double *m, double *M, double *r,
                        double *z, uint32_t *id, double *q, double t0, double dt, int64_t step0, int64_t n_steps,
                        uint64_t seed, uint64_t disk, int64_t max_events, int64_t rebuild_every, double *accreted,
                        int64_t *events_total, int32_t nthreads, double dt_max, double courant, double *dts)
{
    int64_t ncell = (int64_t)n_r * n_z;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (ncell + 1));
    double *cb = (double *)malloc(sizeof(double) * 6 * ncell);
    double *cv = (double *)malloc(sizeof(double) * ncell);
    int64_t *ce = (int64_t *)malloc(sizeof(int64_t) * ncell);
    int64_t *perm = q ? (int64_t *)malloc(sizeof(int64_t) * N) : NULL;
    double *qt = q ? (double *)malloc(sizeof(double) * N) : NULL;
    int status = ORC_OK;
    double t = t0;
    for (int64_t s = 0; s < n_steps && status == ORC_OK; ++s) {
        uint64_t step = (uint64_t)(step0 + s);
        int64_t na = 0;
        status = orc_regrid(P, n_r, n_z, N, m, M, r, z, id, perm, off, cb, cv, &na);
        if (status != ORC_OK) break;
        if (q) {
            for (int64_t k = 0; k < N; ++k) qt[k] = q[perm[k]];
            memcpy(q, qt, sizeof(double) * N);
        }
        /* dt <= 0: the adaptive step, from the cells just made */
        const double h = dt > 0.0 ? dt : orc_adaptive_dt(P, ncell, off, cb, N, m, r, z, dt_max, courant);
        if (dts) dts[s] = h;
        status = orc_collide_all_impl(P, n_r, n_z, off, cb, cv, m, M, q, t, t + h, seed, disk, step, max_events,
                                      rebuild_every, ce, nthreads);
        for (int64_t c = 0; c < ncell; ++c)
            if (events_total) *events_total += ce[c];
        if (P->kernel_mode == 0 && (P->tr_flags & (ORC_TR_RADIAL | ORC_TR_VERTICAL)))
            orc_transport(P, N, r, z, m, M, id, h, seed, disk, step, accreted);
        t += h;
    }
    free(off); free(cb); free(cv); free(ce); free(perm); free(qt);
    return status;
}

int orc_run(const orc_params *P, int32_t n_r, int32_t n_z, int64_t N, double *m, double *M, double *r, double *z,
            uint32_t *id, double t0, double dt, int64_t step0, int64_t n_steps, uint64_t seed, uint64_t disk,
            int64_t max_events, int64_t rebuild_every, double *accreted, int64_t *events_total, int32_t nthreads)
{
    return orc_run_impl(P, n_r, n_z, N, m, M, r, z, id, NULL, t0, dt, step0, n_steps, seed, disk, max_events,
                        rebuild_every, accreted, events_total, nthreads, 0.0, 0.0, NULL);
}

int orc_run_q(const orc_params *P, int32_t n_r, int32_t n_z, int64_t N, double *m, double *M, double *r, double *z,
              uint32_t *id, double *q, double t0, double dt, int64_t step0, int64_t n_steps, uint64_t seed,
              uint64_t disk, int64_t max_events, int64_t rebuild_every, double *accreted, int64_t *events_total,
              int32_t nthreads)
{
    return orc_run_impl(P, n_r, n_z, N, m, M, r, z, id, q, t0, dt, step0, n_steps, seed, disk, max_events,
                        rebuild_every, accreted, events_total, nthreads, 0.0, 0.0, NULL);
}

/* n_steps with the adaptive step (dt_max, courant); dts[n_steps] receives each step's dt; q may be NULL */
int orc_run_adaptive(const orc_params *P, int32_t n_r, int32_t n_z, int64_t N, double *m, double *M, double *r,
                     double *z, uint32_t *id, double *q, double t0, double dt_max, double courant, int64_t step0,
                     int64_t n_steps, uint64_t seed, uint64_t disk, int64_t max_events, int64_t rebuild_every,
                     double *accreted, int64_t *events_total, int32_t nthreads, double *dts)
{
    return orc_run_impl(P, n_r, n_z, N, m, M, r, z, id, q, t0, 0.0, step0, n_steps, seed, disk, max_events,
                        rebuild_every, accreted, events_total, nthreads, dt_max, courant, dts);
}

/* ---- diagnostics --------------------------------------------------------
 * The mass distribution versus distance (the Results compare mcdust and
 * dustpy by the dust surface density per mass and radius), summarised per
 * radial bin: over the particles whose r lies in [edges[b], edges[b+1]) the
 * swarm-mass-weighted sums S0 = sum M, S_k = sum M m^k (k = 1..3) and the
 * count, each by Neumaier's compensated summation in particle order.  A
 * particle outside [edges[0], edges[nbins]) -- a removed one has r = +inf --
 * counts nowhere.  out: nbins x 5, (S0, S1, S2, S3, count) per bin.  The
 * mass-weighted moments of the representative mass are S_k / S0. */
static void orc_nsum(double *s, double *c, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x))
        *c += (*s - t) + x;
    else
        *c += (x - t) + *s;
    *s = t;
}

void orc_moments(int64_t N, const double *m, const double *M, const double *r, int32_t nbins, const double *edges,
                 double *out)
{
    double *acc = (double *)calloc((size_t)nbins * 10, sizeof(double)); /* (sum, compensation) x 5 */
    for (int64_t i = 0; i < N; ++i) {
        if (!(r[i] >= edges[0] && r[i] < edges[nbins])) continue;
        int32_t b = 0;
        while (b + 1 < nbins && edges[b + 1] <= r[i]) ++b; /* the last edge not above r */
        const double w = M[i], x = m[i];
        const double v[5] = {w, w * x, w * x * x, w * x * x * x, 1.0};
        for (int k = 0; k < 5; ++k) orc_nsum(&acc[10 * b + 2 * k], &acc[10 * b + 2 * k + 1], v[k]);
    }
    for (int32_t b = 0; b < nbins; ++b)
        for (int k = 0; k < 5; ++k) out[5 * b + k] = acc[10 * b + 2 * k] + acc[10 * b + 2 * k + 1];
    free(acc);
}

/* The map itself (Benchmark section: the dust surface density as a function
 * of particle mass and distance from the star): per (radial bin b, mass bin q)
 * the swarm mass sum M over the particles with r in [r_edges[b], r_edges[b+1])
 * and m in [m_edges[q], m_edges[q+1]), by compensated summation in particle
 * order.  out: nr x nm, radial bin major.  sigma_d per logarithmic mass
 * interval is out / (pi (r_hi^2 - r_lo^2) ln(m_hi / m_lo)). */
void orc_sigma_map(int64_t N, const double *m, const double *M, const double *r, int32_t nr, const double *r_edges,
                   int32_t nm, const double *m_edges, double *out)
{
    double *acc = (double *)calloc((size_t)nr * nm * 2, sizeof(double));
    for (int64_t i = 0; i < N; ++i) {
        if (!(r[i] >= r_edges[0] && r[i] < r_edges[nr])) continue;
        if (!(m[i] >= m_edges[0] && m[i] < m_edges[nm])) continue;
        int32_t b = 0, q = 0;
        while (b + 1 < nr && r_edges[b + 1] <= r[i]) ++b;
        while (q + 1 < nm && m_edges[q + 1] <= m[i]) ++q;
        const int64_t k = (int64_t)b * nm + q;
        orc_nsum(&acc[2 * k], &acc[2 * k + 1], M[i]);
    }
    for (int64_t k = 0; k < (int64_t)nr * nm; ++k) out[k] = acc[2 * k] + acc[2 * k + 1];
    free(acc);
}

int orc_abi_version(void) { return 1; }
