// mcd_step.cu -- the adaptive time step (a reading; the paper states no rule):
// after the regrid, dt = min(dt_max, C min_c (r_hi - r_lo)_c / max_i |v_r,i|)
// per disk, over the cells that hold particles and the live particles, v_r =
// -2 eta v_K St / (1 + St^2) the radial drift of the transport step (St at
// the particle, or at the midplane with MCD_TR_ST_MIDPLANE).  A disk without
// radial transport (or in the constant-kernel mode) does not drift and asks
// for dt_max.  The disks of a context share one clock, so the step is the
// smallest of their steps.
//
// One launch: a block of particle slots or of cells reduces its extrema and
// merges them into per-disk accumulators with integer atomics.  |v_r| and the
// widths are non-negative, so their IEEE bit patterns order like the values
// and the extrema are exact whatever the order of the atomics.  The last block
// to finish turns the accumulators into dt, writes it into the step state and
// re-arms them for the next step.
#include "mcd_internal.cuh"

namespace mcd {

constexpr int kDtThreads = 256;
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;  // +inf

// |v_r| of a live particle: the drift of the transport step, FP64
__device__ __forceinline__ double drift_speed_fp64(const mcd_disk_params &P, GasTab tab, double r, double z,
                                                   double m)
{
    Gas<double> g = gas_at<double>(P, tab, r, z);
    double rho_st = g.rho, vth = g.vth, nu = g.nu, asw = g.asw;
    if (P.tr_flags & MCD_TR_ST_MIDPLANE) {
        Gas<double> g0 = gas_at<double>(P, tab, r, 0.0);
        rho_st = g0.rho, vth = g0.vth, nu = g0.nu, asw = g0.asw;
    }
    const double a = cbrt(3.0 * m / (4.0 * kPI * P.rho_s));
    const double St = a < asw ? P.rho_s * a / (rho_st * vth) * g.Omega
                              : 2.0 * P.rho_s * a * a / (9.0 * nu * rho_st) * g.Omega;
    return fabs(-2.0 * g.etavk * St / (1.0 + St * St));
}

// the same in FP32, as the mixed transport evaluates it
__device__ __forceinline__ double drift_speed_mixed(const mcd_disk_params &P, GasTab tab, double r, double z,
                                                    double m)
{
    Gas<float> g = gas_at<float>(P, tab, r, z);
    float rho_st = g.rho, vth = g.vth, nu = g.nu, asw = g.asw;
    if (P.tr_flags & MCD_TR_ST_MIDPLANE) {
        Gas<float> g0 = gas_at<float>(P, tab, r, 0.0);
        rho_st = g0.rho, vth = g0.vth, nu = g0.nu, asw = g0.asw;
    }
    const float rho_s = (float)P.rho_s;
    const float a = cbrtf((float)(m * (3.0 / (4.0 * kPI * P.rho_s))));
    const float St = a < asw ? rho_s * a / (rho_st * vth) * g.Omega
                             : 2.0f * rho_s * a * a / (9.0f * nu * rho_st) * g.Omega;
    return (double)fabsf(-2.0f * g.etavk * St / (1.0f + St * St));
}

__device__ __forceinline__ bool drifts(const mcd_disk_params &P)
{
    return P.kernel_mode == 0 && (P.tr_flags & MCD_TR_RADIAL);
}

struct DtArgs {
    const mcd_disk_params *params;
    const GasKnot *gas_knots;
    const int32_t *gas_n;
    const int32_t *slot_disk, *cell_disk;
    const double *r, *z, *m;
    const int32_t *cell_n;
    const double *cell_b;
    int64_t N, C;
    int nd;
    unsigned p_blocks;  // blocks [0, p_blocks) take particle slots, the rest cells
    double dt_max, courant;
    unsigned long long *vmax, *wmin;  // per disk: bits of max |v_r| and of min cell width
    unsigned *done;                   // blocks finished this launch
    StepState *state;
};

// block-wide max (want_max) or min of non-negative bit patterns; every thread gets the result
__device__ __forceinline__ unsigned long long block_ext(unsigned long long x, bool want_max, unsigned long long *sh)
{
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = want_max ? (y > x ? y : x) : (y < x ? y : x);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();  // sh may still be read from an earlier call
    if (l == 0) sh[w] = x;
    __syncthreads();
    x = sh[0];
    for (int k = 1; k < kDtThreads / 32; ++k) x = want_max ? (sh[k] > x ? sh[k] : x) : (sh[k] < x ? sh[k] : x);
    return x;
}

template <bool MIXED, bool TABLE>
__global__ void __launch_bounds__(kDtThreads) k_adaptive_dt(DtArgs A)
{
    __shared__ unsigned long long sh[kDtThreads / 32];
    __shared__ bool last;
    const bool cells = blockIdx.x >= A.p_blocks;
    const int64_t base = (int64_t)(cells ? blockIdx.x - A.p_blocks : blockIdx.x) * kDtThreads;
    const int64_t n = cells ? A.C : A.N;
    const int64_t i = base + threadIdx.x;
    const int32_t *owner = cells ? A.cell_disk : A.slot_disk;
    // slots and cells are stored disk by disk: a block whose ends share a disk holds one disk only
    const int64_t hi = (base + kDtThreads < n ? base + kDtThreads : n) - 1;
    const int d0 = owner[base], d1 = owner[hi];
    int d = d0;
    unsigned long long x = cells ? kInfBits : 0ull;
    if (i < n) {
        d = owner[i];
        const mcd_disk_params &P = A.params[d];
        if (drifts(P)) {
            if (cells) {
                if (A.cell_n[i] > 0) {
                    const double w = A.cell_b[6 * i + 1] - A.cell_b[6 * i];
                    x = __double_as_longlong(w > 0.0 ? w : 0.0);
                }
            } else {
                const double ri = A.r[i];
                if (ri < INFINITY) {
                    const GasTab tab = TABLE ? gas_tab(A.gas_knots, A.gas_n, d) : GasTab{nullptr, 0};
                    const double v = MIXED ? drift_speed_mixed(P, tab, ri, A.z[i], A.m[i])
                                           : drift_speed_fp64(P, tab, ri, A.z[i], A.m[i]);
                    x = __double_as_longlong(v);
                }
            }
        }
    }
    unsigned long long *acc = cells ? A.wmin : A.vmax;
    if (d0 == d1) {
        x = block_ext(x, !cells, sh);
        if (threadIdx.x == 0) {
            if (cells)
                atomicMin(&acc[d0], x);
            else
                atomicMax(&acc[d0], x);
        }
    } else if (i < n) {  // a block across disks (one per disk boundary at most): per thread
        if (cells)
            atomicMin(&acc[d], x);
        else
            atomicMax(&acc[d], x);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(A.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    // the last block: every other block's atomics are visible (fence before the count)
    __threadfence();
    double dt = A.dt_max;
    for (int k = threadIdx.x; k < A.nd; k += kDtThreads) {
        volatile unsigned long long *vv = A.vmax, *ww = A.wmin;
        const double v = __longlong_as_double((long long)vv[k]), w = __longlong_as_double((long long)ww[k]);
        if (drifts(A.params[k]) && v > 0.0 && w < INFINITY) {
            const double h = A.courant * w / v;
            if (h < dt) dt = h;
        }
        vv[k] = 0ull;
        ww[k] = kInfBits;
    }
    const unsigned long long b = block_ext(__double_as_longlong(dt), false, sh);
    if (threadIdx.x == 0) {
        A.state->dt = __longlong_as_double((long long)b);
        *A.done = 0u;
    }
}

cudaError_t launch_adaptive_dt(mcd_ctx *c)
{
    const int b = c->cur;
    DtArgs A;
    A.params = c->d_params;
    A.gas_knots = c->gas_knots;
    A.gas_n = c->gas_n;
    A.slot_disk = c->slot_disk;
    A.cell_disk = c->cell_disk;
    A.r = c->r[b];
    A.z = c->z[b];
    A.m = c->m[b];
    A.cell_n = c->cell_n;
    A.cell_b = c->cell_b;
    A.N = c->N;
    A.C = c->C;
    A.nd = c->n_disks;
    A.p_blocks = (unsigned)((c->N + kDtThreads - 1) / kDtThreads);
    A.dt_max = c->dt_max;
    A.courant = c->courant;
    A.vmax = c->dt_acc;
    A.wmin = c->dt_acc + c->n_disks;
    A.done = reinterpret_cast<unsigned *>(c->dt_acc + 2 * c->n_disks);
    A.state = c->state;
    const unsigned blocks = A.p_blocks + (unsigned)((c->C + kDtThreads - 1) / kDtThreads);
    if (blocks == 0) return cudaSuccess;
    const bool mixed = c->prec == MCD_MIXED, table = c->gas_tables > 0;
    if (mixed)
        table ? k_adaptive_dt<true, true><<<blocks, kDtThreads, 0, c->stream>>>(A)
              : k_adaptive_dt<true, false><<<blocks, kDtThreads, 0, c->stream>>>(A);
    else
        table ? k_adaptive_dt<false, true><<<blocks, kDtThreads, 0, c->stream>>>(A)
              : k_adaptive_dt<false, false><<<blocks, kDtThreads, 0, c->stream>>>(A);
    c->launches += 1;
    return cudaGetLastError();
}

// the accumulators' resting state: no speed, no width, no block finished
std::vector<unsigned long long> adaptive_dt_rest(int32_t n_disks)
{
    std::vector<unsigned long long> v(2 * (size_t)n_disks + 1, 0ull);
    for (int32_t k = 0; k < n_disks; ++k) v[n_disks + k] = kInfBits;
    return v;
}

}  // namespace mcd
