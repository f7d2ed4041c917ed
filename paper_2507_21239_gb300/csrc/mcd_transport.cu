// mcd_transport.cu -- initial particles and particle transport (Summary of the
// mcdust paper: "transport in the vertical and radial directions" in a static
// power-law gas disk).
//
// Transport of one particle over dt (reading, Ciesla-type Monte Carlo
// diffusion): radial Ito step r += [v_r + (1/(r rho_g)) d(r D rho_g)/dr] dt
// + sqrt(2 D dt) xi_1 with v_r = -2 eta v_K St/(1+St^2), and an exact
// Ornstein-Uhlenbeck step in z with rate k = Omega (St + alpha) and
// stationary variance D/k, i.e. H_d = H_g sqrt(alpha/(alpha+St)).  Particles
// below r_in are removed (swarm mass accreted); beyond r_out reflected.
//
// One thread per particle slot over the structure-of-arrays state; reads
// r, z, m, M, id and writes r, z (about 44 algorithmic bytes per particle).
// The FP64 path evaluates everything in FP64; the mixed path evaluates the
// gas, drag and displacements in FP32 and adds them to FP64 positions.
#include <math.h>

#include "mcd_internal.cuh"

namespace mcd {

__device__ __forceinline__ int find_disk(const DiskDev *disks, int nd, int64_t s)
{
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (disks[mid].p_off <= s) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- initial state ---------------------------------------------------------------
__global__ void k_init(const mcd_disk_params *params, const DiskDev *disks, int nd, const double *Mswarm,
                       uint64_t seed, int64_t N, double *m, double *M, double *r, double *z, uint32_t *id)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int d = find_disk(disks, nd, s);
    const mcd_disk_params &P = params[d];
    int64_t k = s - disks[d].p_off;
    U4 x = philox((uint64_t)k, 0, 0, kTagInit, seed, (uint64_t)d);
    double u0 = u01d(x.x[0]), u1 = u01d(x.x[1]), u2 = u01d(x.x[2]);
    double e = 2.0 - P.p, rr;
    if (fabs(e) < 1e-12) {
        rr = P.r_in * exp(u0 * log(P.r_out / P.r_in));
    } else {
        double lo = pow(P.r_in, e), hi = pow(P.r_out, e);
        rr = pow(lo + u0 * (hi - lo), 1.0 / e);
    }
    double xi = sqrt(-2.0 * log(u1)) * cos(2.0 * kPI * u2);
    Gas<double> g = gas_at<double>(P, rr, 0.0);
    r[s] = rr;
    z[s] = g.H * xi;
    m[s] = monomer_mass(P);
    M[s] = Mswarm[d];
    id[s] = (uint32_t)k;
}

// ---- transport -------------------------------------------------------------------------
__device__ __forceinline__ void transport_fp64(const mcd_disk_params &P, GasTab tab, double &r, double &z,
                                               double m, double dt, U4 x, bool &removed)
{
    double rho_bm = sqrt(-2.0 * log(u01d(x.x[0])));
    double ang = 2.0 * kPI * u01d(x.x[1]);
    double xi1 = rho_bm * cos(ang), xi2 = rho_bm * sin(ang);
    double r0 = r, z0 = z;
    Gas<double> g = gas_at<double>(P, tab, r0, z0);
    double rho_s = P.rho_s;
    double rho_st = g.rho, vth = g.vth, nu = g.nu, asw = g.asw;
    if (P.tr_flags & MCD_TR_ST_MIDPLANE) {
        Gas<double> g0 = gas_at<double>(P, tab, r0, 0.0);
        rho_st = g0.rho, vth = g0.vth, nu = g0.nu, asw = g0.asw;
    }
    double a = cbrt(3.0 * m / (4.0 * kPI * rho_s));
    double St = a < asw ? rho_s * a / (rho_st * vth) * g.Omega : 2.0 * rho_s * a * a / (9.0 * nu * rho_st) * g.Omega;
    double rn = r0, zn = z0;
    if (P.tr_flags & MCD_TR_RADIAL) {
        double vr = -2.0 * g.etavk * St / (1.0 + St * St);
        double s2 = z0 / g.H;
        double vD = g.D / r0 * (1.0 - g.p - 0.5 * g.q + s2 * s2 * 0.5 * (3.0 - g.q));
        rn = r0 + (vr + vD) * dt + sqrt(2.0 * g.D * dt) * xi1;
    }
    if (P.tr_flags & MCD_TR_VERTICAL) {
        double sv = P.settle_form == 1 ? St / (1.0 + St) : St;
        double k = g.Omega * (sv + P.alpha);
        zn = z0 * exp(-k * dt) + sqrt(g.D * (-expm1(-2.0 * k * dt)) / k) * xi2;
    }
    removed = false;
    if (rn < P.r_in) {
        removed = true;
        rn = INFINITY;
    } else if (rn > P.r_out) {
        rn = 2.0 * P.r_out - rn;
    }
    r = rn;
    z = zn;
}

__device__ __forceinline__ void transport_mixed(const mcd_disk_params &P, GasTab tab, double &r, double &z,
                                                double m, double dt, U4 x, bool &removed)
{
    float rho_bm = sqrtf(-2.0f * logf(u01f(x.x[0])));
    float sn, cs;
    sincospif(2.0f * u01f(x.x[1]), &sn, &cs);
    float xi1 = rho_bm * cs, xi2 = rho_bm * sn;
    double r0 = r, z0 = z;
    Gas<float> g = gas_at<float>(P, tab, r0, z0);
    float rho_s = (float)P.rho_s;
    float rho_st = g.rho, vth = g.vth, nu = g.nu, asw = g.asw;
    if (P.tr_flags & MCD_TR_ST_MIDPLANE) {
        Gas<float> g0 = gas_at<float>(P, tab, r0, 0.0);
        rho_st = g0.rho, vth = g0.vth, nu = g0.nu, asw = g0.asw;
    }
    float a = cbrtf((float)(m * (3.0 / (4.0 * kPI * P.rho_s))));
    float St = a < asw ? rho_s * a / (rho_st * vth) * g.Omega : 2.0f * rho_s * a * a / (9.0f * nu * rho_st) * g.Omega;
    float dtf = (float)dt;
    double rn = r0, zn = z0;
    if (P.tr_flags & MCD_TR_RADIAL) {
        float vr = -2.0f * g.etavk * St / (1.0f + St * St);
        float s2 = (float)z0 / g.H;
        float vD = g.D / (float)r0 * (1.0f - g.p - 0.5f * g.q + s2 * s2 * 0.5f * (3.0f - g.q));
        rn = r0 + (double)((vr + vD) * dtf + sqrtf(2.0f * g.D * dtf) * xi1);
    }
    if (P.tr_flags & MCD_TR_VERTICAL) {
        float sv = P.settle_form == 1 ? St / (1.0f + St) : St;
        float k = g.Omega * (sv + (float)P.alpha);
        float em1 = expm1f(-k * dtf);
        zn = z0 + (double)((float)z0 * em1 + sqrtf(g.D * (-expm1f(-2.0f * k * dtf)) / k) * xi2);
    }
    removed = false;
    if (rn < P.r_in) {
        removed = true;
        rn = INFINITY;
    } else if (rn > P.r_out) {
        rn = 2.0 * P.r_out - rn;
    }
    r = rn;
    z = zn;
}

// TABLE: some disk has a gas table (the variant without one reads none)
template <bool MIXED, bool TABLE>
__global__ void __launch_bounds__(256) k_transport(const mcd_disk_params *params, const GasKnot *gas_knots,
                                                   const int32_t *gas_n, const DiskDev *disks, int nd,
                                                   uint64_t seed, const StepState *state, int64_t N, double *r,
                                                   double *z, const double *m, const double *M, const uint32_t *id,
                                                   double *accreted)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    double rs = r[s];
    if (!isfinite(rs)) return;
    int d = find_disk(disks, nd, s);
    const mcd_disk_params &P = params[d];
    if (P.kernel_mode == 1 || !(P.tr_flags & (MCD_TR_RADIAL | MCD_TR_VERTICAL))) return;
    double zs = z[s];
    U4 x = philox((uint64_t)id[s], 0, (uint64_t)state->step, kTagTransport, seed, (uint64_t)d);
    bool removed;
    const GasTab tab = TABLE ? gas_tab(gas_knots, gas_n, d) : GasTab{nullptr, 0};
    if (MIXED)
        transport_mixed(P, tab, rs, zs, m[s], state->dt, x, removed);
    else
        transport_fp64(P, tab, rs, zs, m[s], state->dt, x, removed);
    r[s] = rs;
    z[s] = zs;
    if (removed) atomicAdd(&accreted[d], M[s]);
}

__global__ void k_set_clock(StepState *st, double t, int set_t, double dt, int set_dt)
{
    if (set_t) st->t = t;
    if (set_dt) st->dt = dt;
}

__global__ void k_advance_clock(StepState *st, int add_dt_to_t)
{
    if (add_dt_to_t) st->t += st->dt;
    st->step += 1;
}

cudaError_t launch_init(mcd_ctx *c, const double *d_Mswarm)
{
    if (c->N == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((c->N + 255) / 256);
    k_init<<<blocks, 256, 0, c->stream>>>(c->d_params, c->d_disks, c->n_disks, d_Mswarm, c->seed, c->N,
                                          c->m[c->cur], c->M[c->cur], c->r[c->cur], c->z[c->cur], c->id[c->cur]);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_transport(mcd_ctx *c)
{
    if (c->N == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((c->N + 255) / 256);
    int b = c->cur;
    auto go = [&](auto kernel) {
        kernel<<<blocks, 256, 0, c->stream>>>(c->d_params, c->gas_knots, c->gas_n, c->d_disks, c->n_disks, c->seed,
                                              c->state, c->N, c->r[b], c->z[b], c->m[b], c->M[b], c->id[b],
                                              c->accreted);
    };
    const bool mixed = c->prec == MCD_MIXED, table = c->gas_tables > 0;
    if (mixed)
        table ? go(k_transport<true, true>) : go(k_transport<true, false>);
    else
        table ? go(k_transport<false, true>) : go(k_transport<false, false>);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_set_clock(mcd_ctx *c, double t, int set_t, double dt, int set_dt)
{
    k_set_clock<<<1, 1, 0, c->stream>>>(c->state, t, set_t, dt, set_dt);
    c->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_advance_clock(mcd_ctx *c, int add_dt_to_t)
{
    k_advance_clock<<<1, 1, 0, c->stream>>>(c->state, add_dt_to_t);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace mcd
