// mcd_internal.cuh -- shared device helpers and the host context of libmcd.
//
// Physics follows the Summary section of the mcdust paper (static power-law,
// vertically isothermal gas disk; Epstein/Stokes drag; relative velocities
// from Brownian motion, turbulence, radial and azimuthal drift and settling;
// Zsom & Dullemond representative particles).  The paper prints no formulas:
// each form here is the standard published one, the same reading as the
// project's written design.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "mcd.h"

namespace mcd {

// ---- constants (CGS) -------------------------------------------------------
constexpr double kGMsun = 1.32712440018e26;  // G M_sun [cm^3 s^-2]
constexpr double kAU = 1.495978707e13;       // [cm]
constexpr double kKB = 1.380649e-16;         // [erg/K]
constexpr double kMP = 1.67262192e-24;       // [g]
constexpr double kPI = 3.141592653589793;
constexpr double kYA = 1.6;                  // Ormel & Cuzzi (2007) y_a

constexpr uint64_t kTagInit = 1, kTagCollide = 2, kTagTransport = 3;

// status bits latched on the device (mapped to MCD_* codes on the host)
constexpr int kStNaN = 1, kStTimeout = 2, kStEmpty = 4, kStBadCell = 8;

// ---- Philox4x64-10 (Salmon et al., SC'11) ---------------------------------
struct U4 {
    uint64_t x[4];
};

__host__ __device__ inline void mulhilo(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo)
{
#if defined(__CUDA_ARCH__)
    hi = __umul64hi(a, b);
    lo = a * b;
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
#endif
}

__host__ __device__ inline U4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0,
                                     uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint64_t h0, l0, h1, l1;
        mulhilo(M0, c0, h0, l0);
        mulhilo(M1, c2, h1, l1);
        uint64_t n0 = h1 ^ c1 ^ k0, n2 = h0 ^ c3 ^ k1;
        c0 = n0;
        c1 = l1;
        c2 = n2;
        c3 = l0;
        k0 += W0;
        k1 += W1;
    }
    U4 o;
    o.x[0] = c0;
    o.x[1] = c1;
    o.x[2] = c2;
    o.x[3] = c3;
    return o;
}

// (0,1) from the top 53 bits; the float version rounds that same 53-bit value
// (relative precision 2^-24 at every magnitude, so log u stays accurate near 0)
__host__ __device__ inline double u01d(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }
__host__ __device__ inline float u01f(uint64_t x)
{
    // ((x >> 11) + 0.5) 2^-53 from two 32-bit conversions (a 64-bit integer
    // conversion would run on the slow FP64 unit)
    uint32_t hi = (uint32_t)(x >> 32), lo = ((uint32_t)x) >> 11;
    return (float)hi * 0x1.0p-32f + ((float)lo + 0.5f) * 0x1.0p-53f;
}

// ---- gas disk at (r, z) ------------------------------------------------------
template <class T>
struct Gas {
    T Sigma, T_, cs, Omega, H, rho, vth, lambda, nu, etavk, D, vg2, St_eta, asw;
    T p, q;  // local slopes -dln Sigma/dln r, -dln T/dln r
};

// A disk's gas table (mcd_set_gas_table), prepared on the host: knot k holds
// r_k, ln r_k, ln Sigma_k, ln T_k, Sigma_k, T_k and the slopes p_k, q_k of
// segment [r_k, r_{k+1}).  n < 2: the power laws.
struct GasKnot {
    double r, lnr, lnS, lnT, S, T, p, q;
};
struct GasTab {
    const GasKnot *k;
    int n;
};
constexpr int kMaxGasKnots = MCD_MAX_GAS_KNOTS;

__device__ __forceinline__ GasTab gas_tab(const GasKnot *pool, const int32_t *gas_n, int d)
{
    return gas_n ? GasTab{pool + (int64_t)d * kMaxGasKnots, gas_n[d]} : GasTab{nullptr, 0};
}

// the segment holding r: the last k <= n - 2 with r_k <= r, 0 below r_1 (the
// end segments extend beyond the table)
__device__ __forceinline__ int gas_segment(const GasTab &t, double r)
{
    int lo = 0, hi = t.n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (t.k[mid].r <= r)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__device__ inline double mpow(double x, double y) { return pow(x, y); }
__device__ inline float mpow(float x, float y) { return powf(x, y); }
__device__ inline double mexp(double x) { return exp(x); }
__device__ inline float mexp(float x) { return expf(x); }
__device__ inline double msqrt(double x) { return sqrt(x); }
__device__ inline float msqrt(float x) { return sqrtf(x); }
__device__ inline double mcbrt(double x) { return cbrt(x); }
__device__ inline float mcbrt(float x) { return cbrtf(x); }
__device__ inline double mlog(double x) { return log(x); }
__device__ inline float mlog(float x) { return logf(x); }
__device__ inline double mexpm1(double x) { return expm1(x); }
__device__ inline float mexpm1(float x) { return expm1f(x); }

// all quantities of the static, vertically isothermal disk: power laws in r,
// or log-log interpolation of the disk's gas table
template <class T>
__device__ inline Gas<T> gas_at(const mcd_disk_params &P, GasTab tab, double r, double z)
{
    Gas<T> g;
    T rr = (T)r, zz = (T)z;
    if (tab.n >= 2) {
        const GasKnot &K = tab.k[gas_segment(tab, r)];
        if constexpr (sizeof(T) == 8) {
            const double dl = log(r) - K.lnr;
            g.Sigma = exp(K.lnS - K.p * dl);
            g.T_ = exp(K.lnT - K.q * dl);
        } else {
            // ln(r / r_k) from the ratio: exact to a few float ulps of a small number
            const float dl = logf((float)r / (float)K.r);
            g.Sigma = (float)K.S * expf(-(float)K.p * dl);
            g.T_ = (float)K.T * expf(-(float)K.q * dl);
        }
        g.p = (T)K.p;
        g.q = (T)K.q;
    } else {
        T x = (T)r * (T)(1.0 / kAU);
        g.Sigma = (T)P.sigma0 * mpow(x, -(T)P.p);
        g.T_ = (T)P.T0 * mpow(x, -(T)P.q);
        g.p = (T)P.p;
        g.q = (T)P.q;
    }
    g.cs = msqrt((T)kKB * g.T_ / ((T)P.mu * (T)kMP));
    g.Omega = msqrt((T)(P.m_star * kGMsun) / rr / rr / rr);
    g.H = g.cs / g.Omega;
    T rho_mid = g.Sigma / ((T)2.5066282746310002 * g.H);  // sqrt(2 pi)
    T s = zz / g.H;
    g.rho = rho_mid * mexp((T)-0.5 * s * s);
    g.vth = (T)1.5957691216057308 * g.cs;  // sqrt(8/pi)
    g.lambda = ((T)P.mu * (T)kMP / (T)P.sigma_h2) / g.rho;
    g.nu = (T)0.5 * g.vth * g.lambda;
    g.etavk = (T)0.5 * g.cs * g.cs / (g.Omega * rr) * (g.p + (T)0.5 * ((T)3 + g.q));
    g.D = (T)P.alpha * g.cs * g.H;
    g.vg2 = (T)1.5 * (T)P.alpha * g.cs * g.cs;
    g.St_eta = (T)1 / msqrt(g.D / g.nu);
    g.asw = (T)2.25 * g.lambda;
    return g;
}

template <class T>
__device__ inline Gas<T> gas_at(const mcd_disk_params &P, double r, double z)
{
    return gas_at<T>(P, GasTab{nullptr, 0}, r, z);
}

__host__ __device__ inline double monomer_mass(const mcd_disk_params &P)
{
    return P.m_init > 0.0 ? P.m_init : 4.0 * kPI / 3.0 * P.rho_s * P.a_mono * P.a_mono * P.a_mono;
}

// ---- per-disk tables ---------------------------------------------------------
struct DiskDev {
    int64_t p_off, n0;       // particle slots [p_off, p_off + n0)
    int64_t c_off;           // first global cell
    int64_t z_off;           // first global radial zone
    int64_t t_off, n_tiles;  // radix tiles
    int32_t n_r, n_z;
};

struct StepState {
    double t, dt;
    int64_t step;
};

// the r sort's fix-up: runs of equal upper key words longer than this are
// listed (so a list of N / (kRunShortMax + 1) + 1 entries always suffices)
constexpr int kRunShortMax = 64;

// radix sort tile: 256 threads x 16 keys
constexpr int kRadixThreads = 256, kRadixItems = 8, kRadixTile = kRadixThreads * kRadixItems;
constexpr int kRadixBins = 256, kRadixPasses = 8;
constexpr int kRadixUpperPasses = 4;  // the r sort runs the passes of the keys' upper four bytes

// largest cell population the collide kernel takes (one thread per swarm)
constexpr int kMaxCell = 512;

// largest radial zone the regrid sorts in shared memory: (z, id, source)
// elements of 16 bytes, 224 KB
constexpr int64_t kZoneCap = 14336;

// bytes reserved per cell for its gas/drag constants
constexpr int kCellKBytes = 384;

// Collide runs the cells in classes by particles per cell (each disk's
// per_cell picks its class); every class has its own thread count, swarms per
// thread and dv-matrix store, and its own launch on its own stream, so that
// heavy chains of different classes run side by side.
constexpr int kMaxClasses = 5;
constexpr int kMaxTrials = 12;
struct CollideClass {
    int32_t n_lo = 0, n_hi = 0;  // particles per cell of the class's disks
    int64_t cells = 0, qoff = 0; // its cells and their first queue position (class-major queue)
    int32_t rows = 0, W = 0;     // stored matrix: rows (= n_hi) x W entries per cell (circulant half form)
    int32_t smem_fits = 0;       // FP32: the shared-memory matrix fits one CTA
    int32_t reserve = 0;         // the plan reserves the class's matrices in the workspace
    void *dvg = nullptr;         // those matrices (null: not reserved)
    int32_t S = 1, store = 0;    // swarms per thread; 0 recompute row i, 1 shared matrix, 2 workspace matrix
    int32_t ws = 0;              // 1: the control-warp variant (one worker thread per swarm)
    int32_t tuned = 0, n_trials = 0;
    float trial_us[kMaxTrials] = {};  // per candidate: trial time per event on the class's largest cells
    int32_t trial_S[kMaxTrials] = {}, trial_store[kMaxTrials] = {}, trial_ws[kMaxTrials] = {};
};

// row width of a circulant half matrix for cells of up to n swarms: at least
// n/2 + 1, and 2 mod 4 (even for conflict-free reads, W/2 odd for the build)
inline int32_t sym_width(int32_t n)
{
    int32_t w = n / 2 + 1;
    while (w % 4 != 2) ++w;
    return w;
}

}  // namespace mcd

// ---- host context ------------------------------------------------------------
struct mcd_ctx {
    int32_t n_disks = 0, prec = 0;
    cudaStream_t stream = nullptr;
    uint64_t seed = 0;
    std::vector<mcd_disk_params> hp;
    std::vector<mcd_grid> hg;
    std::vector<mcd::DiskDev> hd;
    int64_t N = 0, C = 0, Z = 0, n_tiles = 0;
    int32_t n_max = 0;  // largest possible cell population
    int64_t zone_max = 0, n0_max = 0;  // largest radial zone (n_z * per_cell) and disk (particles)

    mcd_disk_params *d_params = nullptr;
    mcd::DiskDev *d_disks = nullptr;
    int32_t *slot_disk = nullptr;  // disk of each particle slot [N]
    int32_t *cell_disk = nullptr;  // disk of each global cell [C]
    int32_t *zone_disk = nullptr;  // disk of each global zone [Z]
    int32_t *tile_disk = nullptr;  // disk of each radix tile [n_tiles]

    double *m[2] = {}, *M[2] = {}, *r[2] = {}, *z[2] = {};
    uint32_t *id[2] = {};
    int cur = 0;

    uint64_t *key[2] = {};
    uint32_t *val[2] = {};
    uint32_t *hist = nullptr;      // [n_tiles * 256] in (disk, digit, tile) order
    uint32_t *scan_part = nullptr; // block partials of the histogram scan
    int64_t *rfix_longs = nullptr; // the r sort's long runs of equal upper key words (first position each)
    int32_t *rfix_count = nullptr; // [0] long runs listed, [1] the fix-up CTAs' ticket
    int32_t n_sm_regrid = 0;       // SMs of the device (the long-run fix-up's grid)

    int64_t *cell_start = nullptr;  // global particle slot of each cell's first particle
    int32_t *cell_n = nullptr;
    double *cell_b = nullptr;  // 6 per cell: r_lo r_hi z_lo z_hi r_c z_c
    double *cell_V = nullptr;
    unsigned char *cellk = nullptr;  // per-cell constants, kCellKBytes each
    std::vector<mcd::CollideClass> cls;  // collide classes (mcd_init_disk)
    std::vector<int32_t> cell_class_host;  // class of each cell
    int32_t *cell_class = nullptr;         // the same on the device [C]
    int32_t *queue_static = nullptr;       // class-major cell order without the work estimate [C]
    int32_t *qheads = nullptr;             // persistent CTAs: one ticket counter per class
    double *Rtot = nullptr;                // per cell: the total rate of the last scan (MCD_OPT_DUMP_R)
    unsigned long long *tune_scr = nullptr;  // the trial's events and status words
    cudaStream_t cls_stream[mcd::kMaxClasses] = {};  // classes after the first run on these
    cudaEvent_t cls_fork = nullptr, cls_join[mcd::kMaxClasses] = {};
    int32_t n_sm = 0;

    int64_t *cell_events = nullptr;
    uint32_t *cell_cost = nullptr;
    int32_t *queue = nullptr;
    int32_t *qcount = nullptr;  // [64 bins + head]
    int64_t *n_alive = nullptr;
    double *accreted = nullptr;
    unsigned long long *events_total = nullptr;
    double *Rdump = nullptr;
    int32_t *log_ijo = nullptr;
    double *log_t = nullptr, *log_m = nullptr;
    unsigned long long *log_n = nullptr;
    int32_t *status = nullptr;
    mcd::StepState *state = nullptr;
    double *d_Mswarm = nullptr;  // per-disk initial swarm mass
    double *q[2] = {nullptr, nullptr};  // tracer column, double-buffered like the particle columns
    double *diag_edges = nullptr, *diag_out = nullptr;  // diagnostics: bin edges, per-bin sums
    unsigned long long *map_acc = nullptr;  // sigma map: per-bin unit counts, then the unit's exponent
    double *map_redges = nullptr, *map_medges = nullptr, *map_out = nullptr;
    mcd::GasKnot *gas_knots = nullptr;  // [n_disks][MCD_MAX_GAS_KNOTS] gas tables
    int32_t *gas_n = nullptr;           // knots per disk (0: the power laws)
    static constexpr int64_t kLogCap = 1 << 16;

    // options
    int64_t max_events = 10000000;  // per cell per collide call; bounds every event loop
    int32_t cap_stops = 0;
    int64_t rebuild_every = 0;
    int32_t use_graph = 1, dump_R = 0, lpt = 1, threads = 0, exclusive = 1;
    int32_t dv_matrix = -1;  // -1 chosen by the trial; 0 recompute; 1 stored (shared, else workspace); 2 workspace
    int32_t spt = 0;         // swarms per thread: 0 chosen by the trial, 1 or 2
    int32_t control_warp = -1;  // MCD_MIXED: 1 the control-warp variant, 0 the block variants, -1 the trial decides
    int32_t persistent = 0;  // 1: persistent collide CTAs take cells by atomic ticket
    int32_t autotune = 1;    // 1: the first collide times the candidate variants of each class
    int32_t exact_total = 0; // MCD_MIXED: the compensated total rate (one helper warp per cell)
    bool tuned = false;
    int32_t smem_optin = 0;  // dynamic shared memory a collide CTA may request (the device's opt-in limit)
    int32_t ramp = 0;        // some disk has a fragmentation ramp (frag_ramp > 0)
    int32_t tracer = 0;      // the swarms carry the tracer column (MCD_OPT_TRACER / mcd_set_tracer)
    int32_t gas_tables = 0;  // disks with a gas table (mcd_set_gas_table)
    unsigned long long *dt_acc = nullptr;  // adaptive step: per-disk max |v_r| and min width bits, block count
    double dt_max = 3.15576e7, courant = 0.5;  // the adaptive step's cap [s] and C (MCD_OPT_DT_MAX / COURANT)
    int32_t graph_adaptive = 0;             // the captured step graphs choose dt on the device
    bool t_known = true;                    // t_host is the device clock (false after an adaptive step)
    std::vector<int32_t> gas_n_host;  // knots per disk, as on the device
    int64_t log_cell = -1;

    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int64_t graph_launches[2] = {0, 0};  // kernels per replay of each graph
    int64_t launches = 0;                // kernels launched so far
    int32_t trace = 0;
    cudaEvent_t tev[5] = {};
    cudaStream_t cap_stream = nullptr;  // private stream the step graph is captured on
    bool cells_valid = false;
    double t_host = 0.0;
    int64_t step_host = 0;
};

// ---- launchers (defined across the translation units) ----------------------------
namespace mcd {
cudaError_t launch_init(mcd_ctx *c, const double *d_Mswarm);
cudaError_t launch_transport(mcd_ctx *c);  // reads dt and step from the device state
cudaError_t launch_regrid(mcd_ctx *c);     // gathers into buffer 1 - cur; caller flips cur
cudaError_t launch_lpt(mcd_ctx *c);
cudaError_t launch_collide_impl(mcd_ctx *c, int t_end_from_state, double t_end);
cudaError_t launch_set_clock(mcd_ctx *c, double t, int set_t, double dt, int set_dt);
cudaError_t launch_advance_clock(mcd_ctx *c, int add_dt_to_t);
cudaError_t launch_adaptive_dt(mcd_ctx *c);  // writes dt into the device state
std::vector<unsigned long long> adaptive_dt_rest(int32_t n_disks);
cudaError_t prepare_collide(mcd_ctx *c);
cudaError_t tune_collide(mcd_ctx *c);  // the timed trial (once per context, before the first collide)
void collide_shape(const mcd_ctx *c, int q, int32_t *S, int32_t *store, int32_t *threads,
                   int32_t *control_warp);  // class q's launch
int plan_classes(const mcd_grid *g, int32_t nd, int32_t prec, std::vector<CollideClass> &cls,
                 std::vector<int32_t> &disk_class);
size_t class_matrix_bytes(const CollideClass &k, int32_t prec);  // 0: no workspace matrix for the class
cudaError_t prepare_zone(mcd_ctx *c);
cudaError_t launch_moments(mcd_ctx *c, int disk, int nbins);
cudaError_t launch_sigma_map(mcd_ctx *c, int disk, int nr, int nm);
cudaError_t launch_pair_probe(const mcd_disk_params &p, int prec, double rc, double zc, int64_t n,
                              const double *mi, const double *mj, double *dv, double *K, cudaStream_t s);
cudaError_t launch_rate_probe(const mcd_disk_params &p, int prec, double rc, double zc, double V, int n,
                              const double *m, const double *M, double *rate, double *R, cudaStream_t s);
}  // namespace mcd
