// mcd_collide.cu -- the representative-particle collision step (Summary of
// the mcdust paper; Zsom & Dullemond 2008): per cell, the rate of swarm i
// meeting a particle of swarm j is r_ij = K_ij n_j g_ij with
// K_ij = pi (a_i + a_j)^2 dv_ij, n_j = M_j / (m_j V) and the grouping factor
// g_ij = min(1, m_j / (dm m_i)); events follow with exponential waiting times
// from R_tot = sum_i R_i, i chosen by R_i and j by r_ij, and only row and
// column i change after an event.
//
// GB300 layout: one CTA per cell, one thread per swarm (n <= kMaxCell).  The
// per-swarm cache (radius, Stokes number, drag-law flags, 1/m, M/V, ...) sits
// in shared memory; each thread keeps its own row sum R_k in registers.  One
// event costs two block scans (choose i, choose j), two row evaluations (n
// kernel entries each, one per thread) and one block reduction.
//
// Precision (template T): T = double is the plain FP64 path.  T = float is
// the mixed path: dv, sigma, K and the rates in FP32; masses, the cell clock
// and sticking additions in FP64; row sums R_k as compensated FP32 pairs.
// Differences of Stokes numbers use a factored difference of cubes over
// masses split into (hi, lo) FP32 pairs, so close masses lose no digits, and
// drag-law and turbulence regimes are decided by FP64 mass thresholds.
#include <float.h>
#include <math.h>

#include "mcd_internal.cuh"

namespace mcd {

// ---- per-swarm cache -----------------------------------------------------------
template <class T>
struct alignas(16) Part {
    T a, S, p, q;      // radius, Stokes number, 1/(1+S^2), 1/(1+S)
    T im, mh, ml, ad;  // 1/m, mass as hi+lo, (a - a_sw) for Stokes-law swarms
    T Mv, gi;          // M/V (times the cell's rate scale), 1/(dm m) (inf: no grouping)
    T Sl;              // low part of S (FP32 path: S = S + Sl to ~2^-44)
    int32_t fl;        // turbulence regime (0,1,2) | stokes << 2
};

// ---- per-cell constants ----------------------------------------------------------
template <class T>
struct CellK {
    T Cep, Cst, cm, asw, vg2, Se, cbm, e4, e1, oz2, Kc, pi;
    int32_t kmode, settle;
    double m_sw, m_eta, m_one, m0, V, sc, invVsc, vfrag, ratio, chi, dm, fe, cm_d;
    T Cep_lo, Cst_lo;  // FP32 path: low parts of the drag constants
};

template <class T>
__device__ CellK<T> make_cell(const mcd_disk_params &P, double rc, double zc, double V, double Mref)
{
    CellK<T> c;
    Gas<double> g = gas_at<double>(P, rc, zc);
    double Cep = P.rho_s / (g.rho * g.vth) * g.Omega;
    double Cst = 2.0 * P.rho_s / (9.0 * g.nu * g.rho) * g.Omega;
    double cm = 3.0 / (4.0 * kPI * P.rho_s);
    c.m_sw = g.asw * g.asw * g.asw / cm;
    // mass at which the Stokes number reaches S (Epstein below the switch)
    auto m_at = [&](double S) {
        double a = S / Cep;
        if (a >= g.asw) a = sqrt(S / Cst);
        return a * a * a / cm;
    };
    c.m_eta = m_at(g.St_eta);
    c.m_one = m_at(1.0);
    int f = P.dv_flags;
    c.Cep = (T)Cep;
    c.Cst = (T)Cst;
    c.cm = (T)cm;
    c.cm_d = cm;
    c.asw = (T)g.asw;
    c.vg2 = (f & MCD_DV_TURB) ? (T)g.vg2 : (T)0;
    c.Se = (T)g.St_eta;
    c.cbm = (f & MCD_DV_BM) ? (T)(8.0 * kKB * g.T_ / kPI) : (T)0;
    c.e4 = (f & MCD_DV_RAD) ? (T)(4.0 * g.etavk * g.etavk) : (T)0;
    c.e1 = (f & MCD_DV_PHI) ? (T)(g.etavk * g.etavk) : (T)0;
    double oz = g.Omega * fabs(zc);
    c.oz2 = (f & MCD_DV_SET) ? (T)(oz * oz) : (T)0;
    c.Kc = (T)P.K_const;
    c.pi = (T)kPI;
    c.kmode = P.kernel_mode;
    c.settle = P.settle_form;
    c.V = P.kernel_mode == 1 ? P.V_const : V;
    if (sizeof(T) == 4 && Mref > 0.0 && c.V > 0.0) {
        // power-of-two rate scale keeping M/V near 1 in FP32
        c.sc = ldexp(1.0, -ilogb(Mref / c.V));
    } else {
        c.sc = 1.0;
    }
    c.invVsc = c.V > 0.0 ? c.sc / c.V : 0.0;
    c.m0 = monomer_mass(P);
    c.vfrag = P.v_frag;
    c.ratio = P.erosion_ratio;
    c.chi = P.erosion_chi;
    c.dm = P.dm_group;
    c.fe = 2.0 - P.frag_xi;
    c.Cep_lo = (T)(Cep - (double)c.Cep);
    c.Cst_lo = (T)(Cst - (double)c.Cst);
    return c;
}

template <class T>
__device__ __forceinline__ Part<T> make_part(const CellK<T> &c, double m, double M);

template <>
__device__ __forceinline__ Part<double> make_part<double>(const CellK<double> &c, double m, double M)
{
    Part<double> q;
    bool stk = m >= c.m_sw;
    int cls = m < c.m_eta ? 0 : (m < c.m_one ? 1 : 2);
    q.mh = m;
    q.ml = 0.0;
    q.a = cbrt(c.cm_d * m);
    q.S = stk ? c.Cst * q.a * q.a : c.Cep * q.a;
    q.p = 1.0 / (1.0 + q.S * q.S);
    q.q = 1.0 / (1.0 + q.S);
    q.im = 1.0 / m;
    q.ad = stk ? c.cm_d * (m - c.m_sw) / ((q.a * q.a + c.asw * c.asw) + q.a * c.asw) : 0.0;
    q.Mv = M * c.invVsc;
    q.gi = c.dm > 0.0 ? 1.0 / (c.dm * m) : (double)INFINITY;
    q.fl = cls | ((int)stk << 2);
    q.Sl = 0.0;
    return q;
}

template <>
__device__ __forceinline__ Part<float> make_part<float>(const CellK<float> &c, double m, double M)
{
    Part<float> q;
    bool stk = m >= c.m_sw;
    int cls = m < c.m_eta ? 0 : (m < c.m_one ? 1 : 2);
    q.mh = (float)m;
    q.ml = (float)(m - (double)q.mh);
    // a = cbrt(cm m) to about 2^-44: FP32 cube root plus one Newton step on the
    // residual x - a0^3 taken exactly with fused multiply-adds
    double xd = c.cm_d * m;
    float xh = (float)xd, xl = (float)(xd - (double)xh);
    float a0 = cbrtf(xh);
    float p2 = a0 * a0, p2e = fmaf(a0, a0, -p2);   // a0^2 = p2 + p2e
    float p3 = p2 * a0, p3e = fmaf(p2, a0, -p3);   // p2 a0 = p3 + p3e
    float res = (((xh - p3) - p3e) - p2e * a0) + xl; // x - a0^3
    float alo = res / (3.0f * p2);
    q.a = a0;
    float Sh, Se;
    if (stk) {  // S = Cst a^2 = Cst (p2 + p2e + 2 a0 alo)
        Sh = c.Cst * p2;
        Se = fmaf(c.Cst, p2, -Sh) + c.Cst * (p2e + 2.0f * a0 * alo) + c.Cst_lo * p2;
    } else {    // S = Cep a
        Sh = c.Cep * a0;
        Se = fmaf(c.Cep, a0, -Sh) + c.Cep * alo + c.Cep_lo * a0;
    }
    q.S = Sh + Se;
    q.Sl = Se - (q.S - Sh);
    q.p = 1.0f / (1.0f + q.S * q.S);
    q.q = 1.0f / (1.0f + q.S);
    q.im = 1.0f / q.mh;
    q.ad = stk ? (float)(c.cm_d * (m - c.m_sw)) / ((q.a * q.a + c.asw * c.asw) + q.a * c.asw) : 0.0f;
    q.Mv = (float)(M * c.invVsc);
    q.gi = c.dm > 0.0 ? 1.0f / ((float)c.dm * q.mh) : INFINITY;
    q.fl = cls | ((int)stk << 2);
    return q;
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Relative velocity of a pair (symmetric in its arguments bit for bit):
// Brownian motion, Ormel & Cuzzi (2007) turbulence, radial and azimuthal
// drift and settling, summed in quadrature.  Returns dv; K via *K.
template <class T>
__device__ __forceinline__ T pair_dv(const CellK<T> &c, const Part<T> &u, const Part<T> &v, T *K)
{
    if (c.kmode == 1) {
        *K = c.Kc;
        return (T)0;
    }
    // |St_u - St_v| from the factored difference of cubes
    T dm = fabs((u.mh - v.mh) + (u.ml - v.ml));
    T den = fma(u.a, v.a, mul_rn(u.a, u.a) + mul_rn(v.a, v.a));
    T da = c.cm * dm / den;
    int su = u.fl >> 2, sv = v.fl >> 2;
    T D;
    if (su & sv) {
        D = c.Cst * (u.a + v.a) * da;
    } else if (su | sv) {
        T as = su ? u.a : v.a, ads = su ? u.ad : v.ad;
        D = c.Cst * fma(as, ads, c.asw * da);
    } else {
        D = c.Cep * da;
    }
    T S1 = fmax(u.S, v.S), S2 = fmin(u.S, v.S);
    int cls = max(u.fl & 3, v.fl & 3);
    T tv;
    if (cls == 0) {
        T s = S1 + S2;
        tv = s > (T)0 ? c.vg2 * D * D * fma(S1, S2, c.Se * s) / (s * (S1 + c.Se) * (S2 + c.Se)) : (T)0;
    } else if (cls == 1) {
        T eps = S2 / S1, ope = (T)1 + eps;
        tv = c.vg2 * S1 *
             (((T)(2.0 * kYA) - ope) + (T)2 / ope * ((T)(1.0 / (1.0 + kYA)) + eps * eps * eps / ((T)kYA + eps)));
    } else {
        tv = c.vg2 * (u.q + v.q);
    }
    T pp = u.p * v.p;
    // 1 - S_u S_v with the product taken exactly and the low parts added
    T om = fma(-u.S, v.S, (T)1) - (mul_rn(u.S, v.Sl) + mul_rn(u.Sl, v.S));
    T sp = S1 + S2;
    T D2 = D * D;
    T rp = D2 * pp * pp * (c.e4 * om * om + c.e1 * sp * sp);
    T sz = c.oz2 * D2;
    if (c.settle) {
        T qq = u.q * v.q;
        sz *= qq * qq;
    }
    T dv = msqrt(c.cbm * (u.im + v.im) + tv + rp + sz);
    T s2 = u.a + v.a;
    *K = c.pi * s2 * s2 * dv;
    return dv;
}

// rate of swarm `self` meeting a particle of swarm `other`: K M_o/V min(1/m_o, 1/(dm m_self))
template <class T>
__device__ __forceinline__ T weight(const Part<T> &self, const Part<T> &other)
{
    return other.Mv * fmin(other.im, self.gi);
}

// ---- block scan --------------------------------------------------------------
template <class V>
__device__ __forceinline__ void block_scan(V x, V *buf, V &incl, V &excl, V &total)
{
    const unsigned FULL = 0xffffffffu;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V wi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V y = __shfl_up_sync(FULL, wi, o);
        if (lane >= o) wi += y;
    }
    V we = __shfl_up_sync(FULL, wi, 1);
    if (lane == 0) we = (V)0;
    if (lane == 31) buf[w] = wi;
    __syncthreads();
    V off = (V)0, tot = (V)0;
    for (int k = 0; k < nw; ++k) {
        V b = buf[k];
        if (k < w) off += b;
        tot += b;
    }
    incl = off + wi;
    excl = off + we;
    total = tot;
}

// ---- fragments -----------------------------------------------------------------
// mass-weighted draw on [m0, mmax] from n(m) ~ m^-xi, e = 2 - xi:
// m = m0 [1 + u ((mmax/m0)^e - 1)]^(1/e), in expm1/log1p form (relative
// precision kept when mmax is close to m0)
__device__ double frag_draw(double m0, double fe, double mmax, double u, bool fp32)
{
    if (mmax <= m0) return m0;
    double m;
    if (fp32) {
        float L = logf((float)(mmax / m0)), e = (float)fe;
        m = fabs(fe) < 1e-12 ? m0 * (double)expf((float)u * L)
                             : m0 * (double)expf(log1pf((float)u * expm1f(e * L)) / e);
    } else {
        double L = log(mmax / m0);
        m = fabs(fe) < 1e-12 ? m0 * exp(u * L) : m0 * exp(log1p(u * expm1(fe * L)) / fe);
    }
    return fmin(fmax(m, m0), mmax);
}

template <class T>
__device__ double outcome(const CellK<T> &c, double mi, double mj, double dv, double u3, int &kind)
{
    double gain = (c.dm > 0.0 && c.dm * mi > mj) ? c.dm * mi : mj;
    if (c.kmode == 1 || dv < c.vfrag) {
        kind = 0;
        return mi + gain;
    }
    double big = fmax(mi, mj), small = fmin(mi, mj);
    if (big >= c.ratio * small) {
        kind = 2;
        if (mi >= mj) {
            double mn = mi - c.chi * gain;
            return mn > c.m0 ? mn : c.m0;
        }
        return frag_draw(c.m0, c.fe, mi, u3, sizeof(T) == 4);
    }
    kind = 1;
    return frag_draw(c.m0, c.fe, big, u3, sizeof(T) == 4);
}

// ---- accumulators: FP64 sum, or a compensated FP32 pair ------------------------
template <class T>
struct Acc;
template <>
struct Acc<double> {
    double s;
    __device__ void zero() { s = 0.0; }
    __device__ void add(double x) { s += x; }
    __device__ double hi() const { return s; }
    __device__ double value() const { return s; }
    __device__ void set(double x) { s = x; }
};
template <>
struct Acc<float> {
    float s, c;  // running sum and its compensation (TwoSum)
    __device__ void zero() { s = 0.0f, c = 0.0f; }
    __device__ void add(float x)
    {
        float t = s + x;
        float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ float hi() const { return s + c; }
    __device__ double value() const { return (double)s + (double)c; }
    __device__ void set(float x) { s = x, c = 0.0f; }
};

struct CollideArgs {
    const mcd_disk_params *params;
    const DiskDev *disks;
    const int32_t *cell_disk;
    const int64_t *cell_start;
    const int32_t *cell_n;
    const double *cell_b, *cell_V;
    const int32_t *queue;  // block -> cell (null: identity)
    double *m;
    const double *M;
    int64_t *cell_events;
    unsigned long long *events_total;
    const StepState *state;
    double t_end_fixed;  // used when t_end_from_state == 0
    int t_end_from_state;
    uint64_t seed;
    int64_t max_events, rebuild_every;
    int cap_stops;
    int32_t *status;
    double *Rdump;
    int64_t log_cell;
    int32_t *log_ijo;
    double *log_t, *log_m;
    unsigned long long *log_n;
    int64_t log_cap;
    int64_t n_cells;
};

template <class T>
struct Shared {
    CellK<T> c;
    T scan[4][32];
    int sel[4];
    double ring[32][4];  // -log u0, u1, u2, u3
    double mnew;
    int i_ev, j_ev;
};

template <class T>
__global__ void __launch_bounds__(kMaxCell) k_collide(CollideArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<T> sh;
    const int nmax = blockDim.x;
    Part<T> *parts = reinterpret_cast<Part<T> *>(smem_raw);
    double *msh = reinterpret_cast<double *>(parts + nmax);
    T *dvrow = reinterpret_cast<T *>(msh + nmax);

    const int64_t cell = A.queue ? (int64_t)A.queue[blockIdx.x] : (int64_t)blockIdx.x;
    if (cell >= A.n_cells) return;
    const int n = A.cell_n[cell];
    const int k = threadIdx.x;
    if (n <= 0) {
        if (k == 0) A.cell_events[cell] = 0;
        return;
    }
    if (n > nmax) {
        if (k == 0) atomicOr(A.status, kStBadCell);
        return;
    }
    const int disk = A.cell_disk[cell];
    const mcd_disk_params &P = A.params[disk];
    const int64_t off = A.cell_start[cell];
    const double t0 = A.state->t;
    const double t_end = A.t_end_from_state ? t0 + A.state->dt : A.t_end_fixed;
    const uint64_t step = (uint64_t)A.state->step;

    if (k == 0) {
        const double *b = A.cell_b + 6 * cell;
        sh.c = make_cell<T>(P, b[4], b[5], A.cell_V[cell], A.M[off]);
    }
    __syncthreads();
    const CellK<T> &c = sh.c;
    const bool active = k < n;
    Part<T> pk;
    if (active) {
        double mk = A.m[off + k];
        msh[k] = mk;
        pk = make_part<T>(c, mk, A.M[off + k]);
        parts[k] = pk;
    }
    __syncthreads();


    Acc<T> R;
    auto rebuild = [&]() {
        R.zero();
        if (active) {
            for (int j = 0; j < n; ++j) {
                Part<T> pj = parts[j];
                T K;
                pair_dv<T>(c, pk, pj, &K);
                R.add(K * weight<T>(pk, pj));
            }
        }
    };
    rebuild();

    const int64_t reb = A.rebuild_every > 0 ? A.rebuild_every : (int64_t)n;
    // the random stream is keyed by (seed, disk) and counted by
    // (event, disk-local cell, step, domain tag)
    const uint64_t dcell = (uint64_t)(cell - A.disks[disk].c_off);
    double t = t0;
    int64_t ev = 0;
    int sb = 0;  // scan buffer rotation
    const bool logging = (cell == A.log_cell);
    const double sc = c.sc;
    for (;;) {
        if ((ev & 31) == 0) {
            if (k < 32) {
                U4 x = philox((uint64_t)(ev + k), dcell, step, kTagCollide, A.seed, (uint64_t)disk);
                sh.ring[k][0] = -log(u01d(x.x[0]));
                sh.ring[k][1] = u01d(x.x[1]);
                sh.ring[k][2] = u01d(x.x[2]);
                sh.ring[k][3] = u01d(x.x[3]);
            }
            __syncthreads();
        }
        const int slot = (int)(ev & 31);
        // choose i: first k whose inclusive prefix of R exceeds u1 R_tot
        T val = active ? (T)R.hi() : (T)0;
        T incl, excl, tot;
        if (k == 0) sh.sel[(sb + 1) & 3] = -1;  // ordered before any hit by the scan's barrier
        block_scan<T>(val, sh.scan[sb], incl, excl, tot);
        sb = (sb + 1) & 3;
        if (!(tot > (T)0)) break;
        if (ev >= A.max_events) {
            if (!A.cap_stops && k == 0) atomicOr(A.status, kStTimeout);
            break;
        }
        double tau = sh.ring[slot][0] * sc / (double)tot;
        if (t + tau >= t_end) break;
        t += tau;
        T target = (T)sh.ring[slot][1] * tot;
        if (target >= tot) target = tot * (T)(1.0 - 1e-7);
        if (active && excl <= target && target < incl) sh.sel[sb] = k;
        __syncthreads();
        int i = sh.sel[sb];
        if (i < 0) i = n - 1;  // no prefix bracket (non-finite rates): stay in bounds
        sb = (sb + 1) & 3;
        const Part<T> pi = parts[i];
        // row i (i meets k) and column i (k meets i) before the event
        T Kold, dvik = (T)0;
        T row = (T)0, colo = (T)0;
        if (active) {
            dvik = pair_dv<T>(c, pk, pi, &Kold);
            row = Kold * weight<T>(pi, pk);
            colo = Kold * weight<T>(pk, pi);
            dvrow[k] = dvik;
        }
        if (k == 0) sh.sel[(sb + 1) & 3] = -1;
        block_scan<T>(row, sh.scan[sb], incl, excl, tot);
        sb = (sb + 1) & 3;
        T target2 = (T)sh.ring[slot][2] * tot;
        if (target2 >= tot) target2 = tot * (T)(1.0 - 1e-7);
        if (active && excl <= target2 && target2 < incl) sh.sel[sb] = k;
        __syncthreads();
        int j = sh.sel[sb];
        if (j < 0) j = n - 1;
        sb = (sb + 1) & 3;
        if (k == 0) {
            int kind = 0;
            double mnew = outcome<T>(c, msh[i], msh[j], (double)dvrow[j], sh.ring[slot][3], kind);
            msh[i] = mnew;
            parts[i] = make_part<T>(c, mnew, A.M[off + i]);
            if (logging && ev < A.log_cap) {
                A.log_ijo[3 * ev] = i;
                A.log_ijo[3 * ev + 1] = j;
                A.log_ijo[3 * ev + 2] = kind;
                A.log_t[ev] = t;
                A.log_m[ev] = mnew;
            }
        }
        __syncthreads();
        const Part<T> pn = parts[i];
        if (k == i) pk = pn;
        T rown = (T)0;
        if (active) {
            T Knew;
            pair_dv<T>(c, pk, pn, &Knew);
            rown = Knew * weight<T>(pn, pk);
            if (k != i) {
                T coln = Knew * weight<T>(pk, pn);
                if (sizeof(T) == 8) {
                    R.add(coln - colo);
                } else {
                    R.add(coln);
                    R.add(-colo);
                }
            }
        }
        block_scan<T>(rown, sh.scan[sb], incl, excl, tot);
        sb = (sb + 1) & 3;
        if (k == i) R.set(tot);
        ++ev;
        if (ev % reb == 0) rebuild();
    }
    if (active) {
        A.m[off + k] = msh[k];
        if (A.Rdump) A.Rdump[off + k] = R.value() / sc;
    }
    if (k == 0) {
        A.cell_events[cell] = ev;
        atomicAdd(&A.events_total[disk], (unsigned long long)ev);
        if (logging) *A.log_n = (unsigned long long)(ev < A.log_cap ? ev : A.log_cap);
    }
}

// ---- probes ------------------------------------------------------------------------
template <class T>
__global__ void k_pair_probe(mcd_disk_params P, double rc, double zc, int64_t n, const double *mi,
                             const double *mj, double *dv, double *K)
{
    __shared__ CellK<T> c;
    if (threadIdx.x == 0) c = make_cell<T>(P, rc, zc, 1.0, 0.0);
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        Part<T> a = make_part<T>(c, mi[q], 0.0), b = make_part<T>(c, mj[q], 0.0);
        T Kq;
        T d = pair_dv<T>(c, a, b, &Kq);
        dv[q] = (double)d;
        K[q] = (double)Kq;
    }
}

template <class T>
__global__ void k_rate_probe(mcd_disk_params P, double rc, double zc, double V, int n, const double *m,
                             const double *M, double *rate, double *R)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Part<T> *parts = reinterpret_cast<Part<T> *>(smem_raw);
    __shared__ CellK<T> c;
    if (threadIdx.x == 0) c = make_cell<T>(P, rc, zc, V, M[0]);
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) parts[q] = make_part<T>(c, m[q], M[q]);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        Acc<T> acc;
        acc.zero();
        Part<T> pi = parts[i];
        for (int j = 0; j < n; ++j) {
            Part<T> pj = parts[j];
            T K;
            pair_dv<T>(c, pi, pj, &K);
            T rij = K * weight<T>(pi, pj);
            acc.add(rij);
            rate[(int64_t)i * n + j] = (double)rij / c.sc;
        }
        R[i] = acc.value() / c.sc;
    }
}

// ---- launchers -----------------------------------------------------------------------
template <class T>
static cudaError_t collide_impl(mcd_ctx *cx, int from_state, double t_end)
{
    int nthr = cx->threads > 0 ? cx->threads : ((cx->n_max + 31) / 32) * 32;
    if (nthr < 32) nthr = 32;
    if (nthr > kMaxCell || nthr < cx->n_max) return cudaErrorInvalidValue;
    size_t smem = (size_t)nthr * (sizeof(Part<T>) + sizeof(double) + sizeof(T));
    CollideArgs A;
    A.params = cx->d_params;
    A.disks = cx->d_disks;
    A.cell_disk = cx->cell_disk;
    A.cell_start = cx->cell_start;
    A.cell_n = cx->cell_n;
    A.cell_b = cx->cell_b;
    A.cell_V = cx->cell_V;
    A.queue = cx->lpt ? cx->queue : nullptr;
    A.m = cx->m[cx->cur];
    A.M = cx->M[cx->cur];
    A.cell_events = cx->cell_events;
    A.events_total = cx->events_total;
    A.state = cx->state;
    A.t_end_fixed = t_end;
    A.t_end_from_state = from_state;
    A.seed = cx->seed;
    A.max_events = cx->max_events;
    A.rebuild_every = cx->rebuild_every;
    A.cap_stops = cx->cap_stops;
    A.status = cx->status;
    A.Rdump = cx->dump_R ? cx->Rdump : nullptr;
    A.log_cell = cx->log_cell;
    A.log_ijo = cx->log_ijo;
    A.log_t = cx->log_t;
    A.log_m = cx->log_m;
    A.log_n = cx->log_n;
    A.log_cap = mcd_ctx::kLogCap;
    A.n_cells = cx->C;
    if (cx->C == 0) return cudaSuccess;
    k_collide<T><<<(unsigned)cx->C, nthr, smem, cx->stream>>>(A);
    cx->launches += 1;
    return cudaGetLastError();
}

// ---- largest-work-first cell order -------------------------------------------------
// Work of a cell ~ n^2 (rate build) + 2 n x (events in the previous step, same
// cell index).  Cells go into 64 log2 bins, heaviest first; CTAs start in
// block order, so the long event chains begin early.
__global__ void k_lpt_bin(int64_t C, const int32_t *cell_n, const int64_t *cell_events, uint32_t *bin,
                          int32_t *qcount)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    double n = (double)cell_n[c];
    double w = n * n + 2.0 * n * (double)cell_events[c] + 1.0;
    int b = 63 - min(63, ilogb(w));
    bin[c] = (uint32_t)b;
    atomicAdd(&qcount[b], 1);
}

__global__ void k_lpt_scan(int32_t *qcount)
{
    int32_t run = 0;
    for (int b = 0; b < 64; ++b) {
        int32_t x = qcount[b];
        qcount[b] = run;
        run += x;
    }
}

__global__ void k_lpt_place(int64_t C, const uint32_t *bin, int32_t *qcount, int32_t *queue)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    int pos = atomicAdd(&qcount[bin[c]], 1);
    queue[pos] = (int32_t)c;
}

cudaError_t launch_lpt(mcd_ctx *c)
{
    if (c->C == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(c->qcount, 0, 64 * sizeof(int32_t), c->stream);
    if (e != cudaSuccess) return e;
    unsigned g = (unsigned)((c->C + 255) / 256);
    k_lpt_bin<<<g, 256, 0, c->stream>>>(c->C, c->cell_n, c->cell_events, c->cell_cost, c->qcount);
    k_lpt_scan<<<1, 1, 0, c->stream>>>(c->qcount);
    k_lpt_place<<<g, 256, 0, c->stream>>>(c->C, c->cell_cost, c->qcount, c->queue);
    c->launches += 3;
    return cudaGetLastError();
}

template <class T>
static cudaError_t prepare_impl()
{
    size_t smem = (size_t)kMaxCell * (sizeof(Part<T>) + sizeof(double) + sizeof(T));
    return cudaFuncSetAttribute(k_collide<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t prepare_collide(mcd_ctx *c)
{
    cudaError_t e = c->prec == MCD_MIXED ? prepare_impl<float>() : prepare_impl<double>();
    if (e != cudaSuccess) return e;
    size_t sm = (size_t)1024 * sizeof(Part<double>);
    e = cudaFuncSetAttribute(k_rate_probe<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rate_probe<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(1024 * sizeof(Part<float>)));
}

cudaError_t launch_collide_impl(mcd_ctx *cx, int from_state, double t_end)
{
    return cx->prec == MCD_MIXED ? collide_impl<float>(cx, from_state, t_end)
                                 : collide_impl<double>(cx, from_state, t_end);
}

cudaError_t launch_pair_probe(const mcd_disk_params &p, int prec, double rc, double zc, int64_t n,
                              const double *mi, const double *mj, double *dv, double *K, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    unsigned blocks = (unsigned)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (prec == MCD_MIXED)
        k_pair_probe<float><<<blocks, 256, 0, s>>>(p, rc, zc, n, mi, mj, dv, K);
    else
        k_pair_probe<double><<<blocks, 256, 0, s>>>(p, rc, zc, n, mi, mj, dv, K);
    return cudaGetLastError();
}

cudaError_t launch_rate_probe(const mcd_disk_params &p, int prec, double rc, double zc, double V, int n,
                              const double *m, const double *M, double *rate, double *R, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (prec == MCD_MIXED) {
        size_t sm = (size_t)n * sizeof(Part<float>);
        cudaFuncSetAttribute(k_rate_probe<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(1024 * sizeof(Part<float>)));
        k_rate_probe<float><<<1, 256, sm, s>>>(p, rc, zc, V, n, m, M, rate, R);
    } else {
        size_t sm = (size_t)n * sizeof(Part<double>);
        cudaFuncSetAttribute(k_rate_probe<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(1024 * sizeof(Part<double>)));
        k_rate_probe<double><<<1, 256, sm, s>>>(p, rc, zc, V, n, m, M, rate, R);
    }
    return cudaGetLastError();
}

}  // namespace mcd
