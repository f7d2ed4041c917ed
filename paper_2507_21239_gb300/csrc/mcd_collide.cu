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
// in shared memory; each thread keeps its own row sum R_k in registers.  The
// per-cell gas constants come from a separate one-thread-per-cell kernel.
// One event = a block scan that chooses i (and folds in the previous event's
// fresh R_i), row/column i before the event (read from the cell's stored dv
// matrix, or one kernel entry per thread), a block scan whose bracketing lane
// chooses j and applies the outcome itself, and one kernel entry per thread
// for the new row/column i: four block barriers.
//
// Precision (template T): T = double is the plain FP64 path.  T = float is
// the mixed path: dv, sigma, K, rates, waiting times and partner choice in
// FP32; masses and the cell clock in FP64 (touched by one lane per event,
// because an FP64 instruction costs ~64 cycles on GB300);
// row sums R_k as compensated FP32 pairs.  Stokes-number differences use a
// factored difference of cubes over masses split into (hi, lo) FP32 pairs and
// St itself is carried as a (hi, lo) pair, so close masses lose no digits;
// drag-law and turbulence regimes are decided by mass thresholds held as
// (hi, lo) pairs of the FP64 values.
#include <float.h>
#include <math.h>

#include <type_traits>

#include "mcd_internal.cuh"

namespace mcd {

// ---- per-swarm cache -----------------------------------------------------------
template <class T>
struct alignas(16) Part {
    T a, S, p, q;      // radius, Stokes number, 1/(1+S^2), 1/(1+S)
    T im, mh, ml, ad;  // 1/m, mass as hi+lo, (a - a_sw) for Stokes-law swarms
    T Mv, gi;          // M/V (times the cell's rate scale), 1/(dm m) (inf: no grouping)
    T Sl;              // low part of S (FP32 path: S + Sl to ~2^-44)
    int32_t fl;        // turbulence regime (0,1,2) | stokes << 2
};

// ---- per-cell constants ----------------------------------------------------------
template <class T>
struct CellK {
    T Cep, Cst, cm, asw, vg2, Se, cbm, e4, e1, oz2, Kc, pi;
    T Cep_lo, Cst_lo, cm_lo;                         // low parts (FP32 path)
    T msw_h, msw_l, meta_h, meta_l, mone_h, mone_l;  // mass thresholds as hi + lo
    T invVsc_t, dm_t, vfrag_t, m0_t, fe_t;
    int32_t kmode, settle, fe_zero;
    double m_sw, m_eta, m_one, m0, V, sc, invVsc, vfrag, ratio, chi, dm, fe, cm_d;
};
static_assert(sizeof(CellK<double>) <= kCellKBytes && sizeof(CellK<float>) <= kCellKBytes, "cell constants");

template <class T>
__device__ __forceinline__ void split(double x, T &h, T &l)
{
    h = (T)x;
    l = (T)(x - (double)h);
}

template <class T>
__device__ CellK<T> make_cell(const mcd_disk_params &P, GasTab tab, double rc, double zc, double V, double Mref)
{
    CellK<T> c;
    Gas<double> g = gas_at<double>(P, tab, rc, zc);
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
    split(Cep, c.Cep, c.Cep_lo);
    split(Cst, c.Cst, c.Cst_lo);
    split(cm, c.cm, c.cm_lo);
    split(c.m_sw, c.msw_h, c.msw_l);
    split(c.m_eta, c.meta_h, c.meta_l);
    split(c.m_one, c.mone_h, c.mone_l);
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
    // FP32 path: a power-of-two rate scale keeping M/V near 1
    c.sc = (sizeof(T) == 4 && Mref > 0.0 && c.V > 0.0) ? ldexp(1.0, -ilogb(Mref / c.V)) : 1.0;
    c.invVsc = c.V > 0.0 ? c.sc / c.V : 0.0;
    c.invVsc_t = (T)c.invVsc;
    c.m0 = monomer_mass(P);
    c.m0_t = (T)c.m0;
    c.vfrag = P.v_frag;
    c.vfrag_t = (T)P.v_frag;
    c.ratio = P.erosion_ratio;
    c.chi = P.erosion_chi;
    c.dm = P.dm_group;
    c.dm_t = (T)P.dm_group;
    c.fe = 2.0 - P.frag_xi;
    c.fe_t = (T)c.fe;
    c.fe_zero = fabs(c.fe) < 1e-12;
    return c;
}

// (float)m and (float)(m - (double)(float)m) for a double in [2^-74, 2^126)
// (mass_splits), on the integer unit: an f64 <-> f32 conversion costs ~70 cycles of
// latency on GB300, this whole split ~40.  The 53-bit significand is rounded to
// 24 bits, to nearest with ties to even (a carry rolls into the exponent
// field), and the remainder, exact as a signed 30-bit integer, is rounded to
// float and scaled by the exponent.  (No fallback branch: the compiler would
// predicate it and wait for the FP64 route.)
__device__ __forceinline__ bool mass_splits(double m) { return (unsigned)(__double_as_longlong(m) >> 52) - 949u <= 200u; }
__device__ __forceinline__ void split_f64(double m, float &h, float &l)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(m);
    const unsigned lo = (unsigned)b, E = (unsigned)(b >> 52);
    const unsigned up = ((lo >> 28) & 1u) & (((lo & 0x0FFFFFFFu) != 0u) | ((lo >> 29) & 1u));
    h = __uint_as_float((unsigned)(b >> 29) - (896u << 23) + up);  // exponent rebiased mod 2^32
    const int D = (int)(lo & 0x1FFFFFFFu) - (int)(up << 29);
    l = __int2float_rn(D) * __uint_as_float((E - 948u) << 23);  // D 2^(E-1075), E-1075 >= -126
}

// (double)f for a positive normal float, on the integer unit
__device__ __forceinline__ double f2d_pos(float f)
{
    const unsigned x = __float_as_uint(f);
    if ((x >> 23) - 1u >= 254u) return (double)f;  // zero, subnormal, inf, NaN or negative
    return __longlong_as_double((long long)((((unsigned long long)(x >> 23) + 896ull) << 52) |
                                            ((unsigned long long)(x & 0x7FFFFFu) << 29)));
}

// MUFU base-2 exponential and logarithm (flush-to-zero forms; arguments here
// are normal)
__device__ __forceinline__ float ex2_mufu(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_mufu(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// (ah, al) < (bh, bl) for normalised hi + lo pairs
__device__ __forceinline__ bool pair_lt(float ah, float al, float bh, float bl) { return ah < bh || (ah == bh && al < bl); }

// Per-swarm cache from the mass and the swarm's M/V (times the rate scale).
template <class T>
__device__ __forceinline__ Part<T> make_part(const CellK<T> &c, double m, T Mv);

template <>
__device__ __forceinline__ Part<double> make_part<double>(const CellK<double> &c, double m, double Mv)
{
    Part<double> q;
    bool stk = m >= c.m_sw;
    int cls = m < c.m_eta ? 0 : (m < c.m_one ? 1 : 2);
    q.mh = m;
    q.ml = 0.0;
    q.a = cbrt(c.cm_d * m);
    q.S = stk ? c.Cst * q.a * q.a : c.Cep * q.a;
    q.Sl = 0.0;
    q.p = 1.0 / (1.0 + q.S * q.S);
    q.q = 1.0 / (1.0 + q.S);
    q.im = 1.0 / m;
    q.ad = stk ? c.cm_d * (m - c.m_sw) / ((q.a * q.a + c.asw * c.asw) + q.a * c.asw) : 0.0;
    q.Mv = Mv;
    q.gi = c.dm > 0.0 ? 1.0 / (c.dm * m) : (double)INFINITY;
    q.fl = cls | ((int)stk << 2);
    return q;
}

// FP32 path: no FP64 instruction (masses within the split's range).
template <>
__device__ __forceinline__ Part<float> make_part<float>(const CellK<float> &c, double m, float Mv)
{
    Part<float> q;
    float mh, ml;
    split_f64(m, mh, ml);
    q.mh = mh;
    q.ml = ml;
    bool stk = !pair_lt(mh, ml, c.msw_h, c.msw_l);
    int cls = pair_lt(mh, ml, c.meta_h, c.meta_l) ? 0 : (pair_lt(mh, ml, c.mone_h, c.mone_l) ? 1 : 2);
    // x = cm m as a (hi, lo) pair, then a = cbrt(x) to about 2^-44: FP32 cube
    // root plus one Newton step on the residual x - a0^3 taken exactly
    float xh = c.cm * mh;
    float xl = fmaf(c.cm, mh, -xh) + c.cm * ml + c.cm_lo * mh;
    const float l3 = lg2_mufu(xh) * (1.0f / 3.0f);
    float a0 = ex2_mufu(l3);        // refined to full precision below
    const float ia = ex2_mufu(-l3);  // 1/a0 to a few ulp, alongside a0
    float p2 = a0 * a0, p2e = fmaf(a0, a0, -p2);     // a0^2 = p2 + p2e
    float p3 = p2 * a0, p3e = fmaf(p2, a0, -p3);     // p2 a0 = p3 + p3e
    float res = (((xh - p3) - p3e) - p2e * a0) + xl;  // x - a0^3
    float alo = res * (ia * ia * (1.0f / 3.0f));      // res / (3 a0^2): a correction, few digits needed
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
    q.p = __fdividef(1.0f, 1.0f + q.S * q.S);
    q.q = __fdividef(1.0f, 1.0f + q.S);
    q.im = __fdividef(1.0f, mh);
    // a - a_sw = cm (m - m_sw) / (a^2 + a a_sw + a_sw^2), m - m_sw from the pairs
    float dsw = (mh - c.msw_h) + (ml - c.msw_l);
    q.ad = stk ? c.cm * dsw * __fdividef(1.0f, (a0 * a0 + c.asw * c.asw) + a0 * c.asw) : 0.0f;
    q.Mv = Mv;
    q.gi = c.dm_t > 0.0f ? __fdividef(1.0f, c.dm_t * mh) : INFINITY;
    q.fl = cls | ((int)stk << 2);
    return q;
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// The constants one kernel entry reads; the FP32 path keeps them in registers
// (read from shared memory at every entry they would sit on the critical path).
template <class T>
struct PairK {
    T Cep, Cst, cm, asw, vg2, Se, cbm, e4, e1, oz2, Kc, pi;
    int32_t kmode, settle;
};

template <class T>
__device__ __forceinline__ PairK<T> pair_consts(const CellK<T> &c)
{
    PairK<T> p;
    p.Cep = c.Cep, p.Cst = c.Cst, p.cm = c.cm, p.asw = c.asw, p.vg2 = c.vg2, p.Se = c.Se;
    p.cbm = c.cbm, p.e4 = c.e4, p.e1 = c.e1, p.oz2 = c.oz2, p.Kc = c.Kc, p.pi = c.pi;
    p.kmode = c.kmode, p.settle = c.settle;
    return p;
}

// Coagulation kernel from a pair's relative velocity: K = pi (a_u + a_v)^2 dv
// (the constant kernel in the 0D test mode).  The same expression serves the
// fresh evaluation and the stored-dv path, so both give the same bits.
template <class T, class C>
__device__ __forceinline__ T kern_of(const C &c, T au, T av, T dv)
{
    if (c.kmode == 1) return c.Kc;
    T s2 = au + av;
    return c.pi * s2 * s2 * dv;
}

// Relative velocity of a pair (symmetric in its arguments bit for bit):
// Brownian motion, Ormel & Cuzzi (2007) turbulence, radial and azimuthal
// drift and settling, summed in quadrature.  Returns dv; K via *K.  C is
// CellK<T> or PairK<T>.
template <class T, class C>
__device__ __forceinline__ T pair_dv(const C &c, const Part<T> &u, const Part<T> &v, T *K)
{
    if (c.kmode == 1) {
        *K = c.Kc;
        return (T)0;
    }
    // |St_u - St_v| from the factored difference of cubes
    T dm = fabs((u.mh - v.mh) + (u.ml - v.ml));
    T den = fma(u.a, v.a, mul_rn(u.a, u.a) + mul_rn(v.a, v.a));
    T da = fdiv(c.cm * dm, den);
    int su = u.fl >> 2, sv = v.fl >> 2;
    T S1 = fmax(u.S, v.S), S2 = fmin(u.S, v.S);
    int cls = max(u.fl & 3, v.fl & 3);
    T D, tv;
    if (sizeof(T) == 4) {
        // FP32: every case evaluated and selected, so the lanes of a warp
        // never diverge (the regimes mix freely within a cell).  dv^2 is
        // factored as t0 + D^2 coef: everything but D (including the regime-I
        // division) is computed alongside D's own division.
        T as = su ? u.a : v.a, ads = su ? u.ad : v.ad;
        T D_st = c.Cst * (u.a + v.a) * da, D_mx = c.Cst * fma(as, ads, c.asw * da), D_ep = c.Cep * da;
        D = (su & sv) ? D_st : ((su | sv) ? D_mx : D_ep);
        T s = S1 + S2;
        T g1 = fdiv(c.vg2 * fma(S1, S2, c.Se * s), s * (S1 + c.Se) * (S2 + c.Se));  // regime I: D^2 g1
        // regime II with eps = S2/S1 cleared from the fractions (one division):
        // vg2 [(2 y_a - 1) S1 - S2 + 2((y_a S1 + S2) S1^2/(1+y_a) + S2^3) / ((S1+S2)(y_a S1 + S2))],
        // every term positive (S2 <= S1, S1 < 1 where this regime applies)
        T A1 = fma((T)kYA, S1, S2);
        T num = fma(A1 * (S1 * S1), (T)(1.0 / (1.0 + kYA)), S2 * S2 * S2);
        T t2 = c.vg2 * (fma((T)(2.0 * kYA - 1.0), S1, -S2) + fdiv((T)2 * num, s * A1));
        T t3 = c.vg2 * (u.q + v.q);
        T pp = u.p * v.p;
        T om = fma(-u.S, v.S, (T)1) - (mul_rn(u.S, v.Sl) + mul_rn(u.Sl, v.S));
        T sp = S1 + S2;
        T qq = c.settle ? (u.q * v.q) * (u.q * v.q) : (T)1;
        T coef = pp * pp * (c.e4 * om * om + c.e1 * sp * sp) + c.oz2 * qq + ((cls == 0 && s > (T)0) ? g1 : (T)0);
        T t0 = c.cbm * (u.im + v.im) + (cls == 1 ? t2 : (cls == 2 ? t3 : (T)0));
        T dv2 = fma(D * D, coef, t0);
        T dv = dv2 > (T)0 ? dv2 * rsqrtf(dv2) : (T)0;
        *K = kern_of<T>(c, u.a, v.a, dv);
        return dv;
    } else {
        if (su & sv) {
            D = c.Cst * (u.a + v.a) * da;
        } else if (su | sv) {
            T as = su ? u.a : v.a, ads = su ? u.ad : v.ad;
            D = c.Cst * fma(as, ads, c.asw * da);
        } else {
            D = c.Cep * da;
        }
        if (cls == 0) {
            T s = S1 + S2;
            tv = s > (T)0 ? fdiv(c.vg2 * D * D * fma(S1, S2, c.Se * s), s * (S1 + c.Se) * (S2 + c.Se)) : (T)0;
        } else if (cls == 1) {
            // vg2 S1 [2 y_a - (1+e) + 2/(1+e) (1/(1+y_a) + e^3/(y_a+e))], the last
            // term over one common denominator
            T eps = fdiv(S2, S1), ope = (T)1 + eps, yae = (T)kYA + eps;
            T last = fdiv((T)2 * (yae * (T)(1.0 / (1.0 + kYA)) + eps * eps * eps), ope * yae);
            tv = c.vg2 * S1 * (((T)(2.0 * kYA) - ope) + last);
        } else {
            tv = c.vg2 * (u.q + v.q);
        }
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
    *K = kern_of<T>(c, u.a, v.a, dv);
    return dv;
}

// rate of swarm `self` meeting a particle of swarm `other`: K M_o/V min(1/m_o, 1/(dm m_self))
template <class T>
__device__ __forceinline__ T weight(const Part<T> &self, const Part<T> &other)
{
    return other.Mv * fmin(other.im, self.gi);
}

// ---- partner choice ----------------------------------------------------------
// Choose k with probability x_k / total: the first k whose inclusive prefix
// exceeds u * total.  With FUSE the scan also sums y over the block (the
// previous event's new row) and folds that sum in as element pend's value
// (x_pend is then 0).  A shuffle scan within each warp, then a shuffle scan of
// the warp totals held one per lane; every warp knows the range [lo, hi) of
// the prefix it covers, lo of warp w+1 bit-identical to hi of warp w, so
// exactly one warp brackets the target and finds the element by a ballot.
// block_bracket returns the element in that warp's lane 0 and -1 in every
// other lane (one barrier); block_choose broadcasts it through shared memory
// (a second barrier).
template <class V, bool FUSE>
__device__ __forceinline__ int block_bracket(V x, V y, V u, int pend, V *buf, V &total, V &ysum)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V wi = x, ys = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        V a = __shfl_up_sync(FULL, wi, o);
        if (lane >= o) wi += a;
        if (FUSE) ys += __shfl_xor_sync(FULL, ys, o);
    }
    if (lane == 31) {
        buf[2 * w] = wi;
        buf[2 * w + 1] = ys;
    }
    __syncthreads();
    // lane q holds warp q's total (q < nw <= 16); scan them in registers
    V bt = lane < nw ? buf[2 * lane] : (V)0;
    V by = (FUSE && lane < nw) ? buf[2 * lane + 1] : (V)0;
    V bs = bt;
#pragma unroll
    for (int o = 1; o < kMaxCell / 32; o <<= 1) {
        if (o >= nw) break;  // (block-uniform) log2(nw) rounds
        V a = __shfl_up_sync(FULL, bs, o);
        if (lane >= o) bs += a;
        if (FUSE) by += __shfl_xor_sync(FULL, by, o);
    }
    const V tot = __shfl_sync(FULL, bs, nw - 1);
    const V prev = __shfl_sync(FULL, bs, w > 0 ? w - 1 : 0);
    const V off = w > 0 ? prev : (V)0;
    const V hib = __shfl_sync(FULL, bs, w);
    const V Rp = (FUSE && pend >= 0) ? __shfl_sync(FULL, by, 0) : (V)0;
    total = tot + Rp;
    ysum = Rp;
    V target = u * total;
    if (target >= total) target = total * (V)(1.0 - 1e-7);
    const int k = threadIdx.x;
    const V P = (off + wi) + ((pend >= 0 && k >= pend) ? Rp : (V)0);
    const V lo = off + ((pend >= 0 && 32 * w > pend) ? Rp : (V)0);
    const V hi = hib + ((pend >= 0 && 32 * w + 31 >= pend) ? Rp : (V)0);
    const unsigned bal = __ballot_sync(FULL, P > target);
    // (a tree scan may leave lane 31's prefix an ulp below hi: then lane 31)
    return (lane == 0 && lo <= target && target < hi) ? 32 * w + __ffs(bal | 0x80000000u) - 1 : -1;
}

template <class V, bool FUSE>
__device__ __forceinline__ int block_choose(V x, V y, V u, int pend, V *buf, int *sel, V &total, V &ysum)
{
    const int f = block_bracket<V, FUSE>(x, y, u, pend, buf, total, ysum);
    if (f >= 0) *sel = f;
    __syncthreads();
    return *sel;
}

// ---- outcomes ----------------------------------------------------------------
// order of positive finite doubles through their bit patterns (integer unit);
// a negative value (sign bit set) orders below every positive one
__device__ __forceinline__ bool dgt(double a, double b) { return __double_as_longlong(a) > __double_as_longlong(b); }

// mass-weighted draw on [m0, mmax] from n(m) ~ m^-xi, e = 2 - xi:
// m = m0 [1 + u ((mmax/m0)^e - 1)]^(1/e), in expm1/log1p form (relative
// precision kept when mmax is close to m0); the clamp to [m0, mmax] by dgt
template <class T>
struct Frag;
template <>
struct Frag<double> {
    static __device__ double draw(const CellK<double> &c, double mmax, double, double u)
    {
        if (!dgt(mmax, c.m0)) return c.m0;
        const double L = log(mmax / c.m0);
        double m = c.fe_zero ? c.m0 * exp(u * L) : c.m0 * exp(log1p(u * expm1(c.fe * L)) / c.fe);
        m = dgt(c.m0, m) ? c.m0 : m;
        return dgt(m, mmax) ? mmax : m;
    }
};
// FP32 path: L and the draw in FP32 from the float images of mmax (its cache
// hi part) and m0; m0 times the draw in FP64
template <>
struct Frag<float> {
    static __device__ double draw(const CellK<float> &c, double mmax, float mmax_h, float u)
    {
        if (!dgt(mmax, c.m0)) return c.m0;
        const float L = logf(__fdividef(mmax_h, c.m0_t)), e = c.fe_t;
        const float f = c.fe_zero ? expf(u * L) : expf(log1pf(u * expm1f(e * L)) / e);
        double m = c.m0 * f2d_pos(f);
        m = dgt(c.m0, m) ? c.m0 : m;
        return dgt(m, mmax) ? mmax : m;
    }
};

// new mass of representative i after meeting a particle of swarm j; dmmi is
// dm m_i (0 when grouping is off), computed ahead by the caller; mih, mjh the
// hi parts of the masses (FP32 path).  u3 draws a fragment's mass.
template <class T>
__device__ __forceinline__ double outcome(const CellK<T> &c, double mi, double mj, T mih, T mjh, double dmmi, T dv,
                                          T u3, int &kind)
{
    const double gain = dgt(dmmi, mj) ? dmmi : mj;  // N_g m_j
    if (c.kmode == 1 || dv < (sizeof(T) == 4 ? (T)c.vfrag_t : (T)c.vfrag)) {
        kind = 0;
        return mi + gain;
    }
    const bool igt = dgt(mi, mj);
    const double big = igt ? mi : mj, small = igt ? mj : mi;
    if (big >= c.ratio * small) {
        kind = 2;
        if (!dgt(mj, mi)) {
            const double mn = mi - c.chi * gain;
            return dgt(mn, c.m0) ? mn : c.m0;
        }
        return Frag<T>::draw(c, mi, mih, u3);
    }
    kind = 1;
    return Frag<T>::draw(c, big, igt ? mih : mjh, u3);
}

// The same with a fragmentation ramp below v_frag: the probability of
// fragmenting rises linearly from 0 at vlo = v_frag (1 - frag_ramp) to 1 at
// v_frag, decided by u3 < p; u3 / p (uniform again) then draws the fragment.
template <class T>
__device__ __forceinline__ double outcome_ramp(const CellK<T> &c, double mi, double mj, T mih, T mjh, double dmmi,
                                               T dv, T u3, T vlo, int &kind)
{
    const T vfr = sizeof(T) == 4 ? (T)c.vfrag_t : (T)c.vfrag;
    if (c.kmode != 1 && dv < vfr && !(dv < vlo)) {  // inside the ramp
        const T p = fdiv(dv - vlo, vfr - vlo);
        if (u3 < p) return outcome<T>(c, mi, mj, mih, mjh, dmmi, vfr, fdiv(u3, p), kind);  // fragments as at v_frag
    }
    return outcome<T>(c, mi, mj, mih, mjh, dmmi, dv, u3, kind);
}

// The tracer of representative i after an event of the given kind: sticking
// mixes by mass, (m_i q_i + g q_j) / m_new with g the absorbed mass;
// fragmentation gives the pair's mass-weighted mixture; erosion leaves the
// larger body's q and makes the smaller one debris of itself and chi times its
// mass chipped from the other, (q_i + chi q_j) / (1 + chi).  FP64, explicitly
// rounded (no fused multiply-add), like the plain CPU evaluation.
__device__ __forceinline__ double tracer_update(double mi, double mj, double qi, double qj, double gain, double mnew,
                                                int kind, double chi)
{
    if (kind == 0) return __ddiv_rn(__dadd_rn(__dmul_rn(mi, qi), __dmul_rn(gain, qj)), mnew);
    if (kind == 1) return __ddiv_rn(__dadd_rn(__dmul_rn(mi, qi), __dmul_rn(mj, qj)), __dadd_rn(mi, mj));
    if (!(mi < mj)) return qi;
    return __ddiv_rn(__dadd_rn(qi, __dmul_rn(chi, qj)), __dadd_rn(1.0, chi));
}

// ---- accumulators: FP64 sum, or a compensated FP32 pair ------------------------
template <class T>
struct Acc;
template <>
struct Acc<double> {
    double s;
    __device__ void zero() { s = 0.0; }
    __device__ void add(double x) { s += x; }
    __device__ void update(double n, double o) { s += n - o; }
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
        float t = __fadd_rn(s, x);
        float bp = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
        s = t;
    }
    __device__ void update(float n, float o)
    {
        add(n);
        add(-o);
    }
    __device__ float hi() const { return __fadd_rn(s, c); }
    __device__ double value() const { return (double)s + (double)c; }
    __device__ void set(float x) { s = x, c = 0.0f; }
};

// random numbers of one event: -log(u0) (times the rate scale), u1, u2, u3
template <class T>
struct Draw {
    T L, u1, u2, u3;
};

__device__ __forceinline__ Draw<float> make_draw(const U4 &x, float sc)
{
    Draw<float> d;
    d.L = -logf(u01f(x.x[0])) * sc;
    d.u1 = u01f(x.x[1]);
    d.u2 = u01f(x.x[2]);
    d.u3 = u01f(x.x[3]);
    return d;
}

__device__ __forceinline__ Draw<double> make_draw(const U4 &x, double sc)
{
    Draw<double> d;
    d.L = -log(u01d(x.x[0])) * sc;
    d.u1 = u01d(x.x[1]);
    d.u2 = u01d(x.x[2]);
    d.u3 = u01d(x.x[3]);
    return d;
}

struct CollideArgs {
    const mcd_disk_params *params;
    const DiskDev *disks;
    const int32_t *cell_disk;
    const int64_t *cell_start;
    const int32_t *cell_n;
    const double *cell_b, *cell_V;
    const unsigned char *cellk;  // per-cell constants, kCellKBytes each
    const int32_t *queue;        // block -> cell (null: identity)
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
    int dv_ld;  // row stride of the stored dv matrix (odd; STORE path)
    double *q;  // the tracer column (TRACER variants)
    double *dvg;  // FP64 stored matrices in global memory, ld x ld per cell (STORE, FP64)
};

template <class T>
struct Shared {
    CellK<T> c;
    T scan[2][64];
    int sel;
    Draw<T> ring[32];
    double t;  // the cell clock
    int stop;  // 0 event applied, 1 crossing t_end, 2 no partner bracketed
};

// per-cell constants: one thread per cell, all SMs (the FP64 gas evaluation is
// long; done here it leaves the collide CTAs' critical path)
template <class T>
__global__ void k_cellconst(const mcd_disk_params *params, const GasKnot *gas_knots, const int32_t *gas_n,
                            const int32_t *cell_disk, const int64_t *cell_start, const int32_t *cell_n,
                            const double *cell_b, const double *cell_V, const double *M, unsigned char *cellk,
                            int64_t C)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C || cell_n[c] <= 0) return;
    const double *b = cell_b + 6 * c;
    const int d = cell_disk[c];
    *reinterpret_cast<CellK<T> *>(cellk + c * kCellKBytes) =
        make_cell<T>(params[d], gas_tab(gas_knots, gas_n, d), b[4], b[5], cell_V[c], M[cell_start[c]]);
}

// STORE (FP32 only): the cell's dv matrix lives in shared memory (row stride
// A.dv_ld, odd, so a column walk is free of bank conflicts).  Row i before an
// event is then read, not recomputed, and later full rebuilds sum stored
// entries; pair_dv is symmetric bit for bit, so the results are those of the
// recomputing path.
// TRACER: the swarms carry a tracer column (shared-memory copy after the dv
// row, before the matrix), updated on every event.
template <class T, bool STORE, bool RAMP, bool TRACER>
__global__ void __launch_bounds__(kMaxCell) k_collide(CollideArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<T> sh;
    const int nmax = blockDim.x;
    Part<T> *parts = reinterpret_cast<Part<T> *>(smem_raw);
    double *msh = reinterpret_cast<double *>(parts + nmax);
    T *dvrow = reinterpret_cast<T *>(msh + nmax);
    double *qsh = reinterpret_cast<double *>(dvrow + nmax);  // TRACER
    T *Dm = TRACER ? reinterpret_cast<T *>(qsh + nmax) : dvrow + nmax;  // STORE: dv_kj at Dm[k * ld + j], ld x ld
    const int ld = A.dv_ld;

    const int64_t cell = A.queue ? (int64_t)A.queue[blockIdx.x] : (int64_t)blockIdx.x;
    if (cell >= A.n_cells) return;
    if constexpr (STORE && sizeof(T) == 8) Dm = reinterpret_cast<T *>(A.dvg) + (size_t)cell * ld * ld;
    const int n = A.cell_n[cell];
    const int k = threadIdx.x;
    if (n <= 0) {
        if (k == 0) A.cell_events[cell] = 0;
        return;
    }
    if (n > nmax || (STORE && n > ld)) {
        if (k == 0) atomicOr(A.status, kStBadCell);
        return;
    }
    const int disk = A.cell_disk[cell];
    const int64_t off = A.cell_start[cell];
    if (k == 0) sh.c = *reinterpret_cast<const CellK<T> *>(A.cellk + cell * kCellKBytes);
    __syncthreads();
    const CellK<T> &c = sh.c;
    // FP32: the entry constants in registers; FP64: read in place (register budget)
    typedef typename std::conditional<sizeof(T) == 4, PairK<T>, const CellK<T> &>::type PK;
    PK pc = [&]() -> PK {
        if constexpr (sizeof(T) == 4) return pair_consts<T>(sh.c); else return sh.c;
    }();
    const bool active = k < n;
    Part<T> pk;
    if (active) {
        double mk = A.m[off + k];
        // FP32 path: every mass the event loop can reach lies between the
        // monomer mass and the disk's dust mass, inside the split's range
        if (sizeof(T) == 4 && !mass_splits(mk)) atomicOr(A.status, kStBadCell);
        msh[k] = mk;
        if (TRACER) qsh[k] = A.q[off + k];
        pk = make_part<T>(c, mk, (T)(A.M[off + k] * c.invVsc));
        parts[k] = pk;
    }
    __syncthreads();

    Acc<T> R;
    // R_k = sum_j r_kj in j order; four independent kernel entries in flight
    // (STORE: the dv entries go to row k of the matrix)
    auto rebuild = [&]() {
        R.zero();
        if (active) {
            int j = 0;
            // (FP64: no unrolling; its register budget is spent on the wider values)
            for (; sizeof(T) == 4 && j + 4 <= n; j += 4) {
                T K0, K1, K2, K3;
                const Part<T> p0 = parts[j], p1 = parts[j + 1], p2 = parts[j + 2], p3 = parts[j + 3];
                T d0 = pair_dv<T>(pc, pk, p0, &K0);
                T d1 = pair_dv<T>(pc, pk, p1, &K1);
                T d2 = pair_dv<T>(pc, pk, p2, &K2);
                T d3 = pair_dv<T>(pc, pk, p3, &K3);
                if (STORE) {
                    Dm[k * ld + j] = d0;
                    Dm[k * ld + j + 1] = d1;
                    Dm[k * ld + j + 2] = d2;
                    Dm[k * ld + j + 3] = d3;
                }
                R.add(K0 * weight<T>(pk, p0));
                R.add(K1 * weight<T>(pk, p1));
                R.add(K2 * weight<T>(pk, p2));
                R.add(K3 * weight<T>(pk, p3));
            }
            for (; j < n; ++j) {
                const Part<T> pj = parts[j];
                T K;
                T d = pair_dv<T>(pc, pk, pj, &K);
                if (STORE) Dm[k * ld + j] = d;
                R.add(K * weight<T>(pk, pj));
            }
        }
    };
    // STORE: the same sums from the stored row k (entries written by other
    // threads since the last barrier are made visible first)
    auto rebuild_stored = [&]() {
        __syncthreads();
        R.zero();
        if (active)
            for (int j = 0; j < n; ++j) {
                const Part<T> pj = parts[j];
                R.add(kern_of<T>(pc, pk.a, pj.a, Dm[k * ld + j]) * weight<T>(pk, pj));
            }
    };
    rebuild();

    // the random stream is keyed by (seed, disk) and counted by
    // (event, disk-local cell, step, domain tag)
    const uint64_t dcell = (uint64_t)(cell - A.disks[disk].c_off);
    const uint64_t step = (uint64_t)A.state->step;
    const double t_end = A.t_end_from_state ? A.state->t + A.state->dt : A.t_end_fixed;
    const int64_t reb = A.rebuild_every > 0 ? A.rebuild_every : 4 * (int64_t)n;
    int64_t until_rebuild = reb;  // events left before the next full rebuild
    const bool logging = (cell == A.log_cell);
    const T sc = (T)c.sc;
    if (k == 0) sh.t = A.state->t;  // (visible after the first ring barrier)
    const int lane = k & 31;
    int64_t ev = 0;
    int pend = -1;          // swarm whose fresh row sum rides on the next scan
    T rown = (T)0;          // this thread's entry of that row
    for (;;) {
        if ((ev & 31) == 0) {
            if (k < 32)
                sh.ring[k] = make_draw(philox((uint64_t)(ev + k), dcell, step, kTagCollide, A.seed, (uint64_t)disk), sc);
            __syncthreads();
        }
        const Draw<T> dr = sh.ring[ev & 31];
        // (1) choose i: first k whose inclusive prefix of R exceeds u1 R_tot;
        //     the previous event's R_i (sum of its new row) is folded in here
        T val = (active && k != pend) ? (T)R.hi() : (T)0;
        T tot, Rp;
        if (k == 0) sh.sel = -1;
        int i = block_choose<T, true>(val, rown, dr.u1, pend, sh.scan[0], &sh.sel, tot, Rp);
        if (pend >= 0 && k == pend) R.set(Rp);
        if (!(tot > (T)0)) break;
        if (ev >= A.max_events) {
            if (!A.cap_stops && k == 0) atomicOr(A.status, kStTimeout);
            break;
        }
        if (i < 0 || i >= n) i = n - 1;  // no bracket (non-finite rates): stay in bounds
        // the lane that brackets j applies the event (lane 0 of some warp): every
        // warp's lane 0 reads m_i and forms dm m_i ahead (FP64 latency, off the path)
        double mi = 0.0, dmmi = 0.0;
        if (lane == 0) {
            mi = msh[i];
            dmmi = c.dm * mi;
        }
        if (k == 0) sh.stop = 2;
        // (2) row i (i meets k) and column i (k meets i) before the event
        const Part<T> pi = parts[i];
        T Kold, row = (T)0, colo = (T)0;
        if (active) {
            if (STORE) {
                Kold = kern_of<T>(pc, pk.a, pi.a, Dm[i * ld + k]);
            } else {
                T dvik = pair_dv<T>(pc, pk, pi, &Kold);
                dvrow[k] = dvik;
            }
            row = Kold * weight<T>(pi, pk);
            colo = Kold * weight<T>(pk, pi);
        }
        // (3) choose j by the row's prefix; (4) the lane that finds j advances
        //     the clock and, unless the event would cross t_end (memoryless:
        //     discarded), applies the outcome and the new cache of i (FP64 masses)
        T tot2, unused;
        int j = block_bracket<T, false>(row, (T)0, dr.u2, -1, sh.scan[1], tot2, unused);
        if (j >= 0) {
            if (j >= n) j = n - 1;  // (lane 31 fallback in a partly idle warp)
            // the clock, the outcome and the new cache are independent chains;
            // only the stores wait for the crossing test
            const double tn = sh.t + (double)fdiv(dr.L, tot);
            int kind = 0;
            double mnew;
            if constexpr (RAMP) {  // the ramp's foot as the plain FP64 evaluation forms it
                const mcd_disk_params &P = A.params[disk];
                mnew = outcome_ramp<T>(c, mi, msh[j], pi.mh, parts[j].mh, dmmi, STORE ? Dm[i * ld + j] : dvrow[j],
                                       dr.u3, (T)(P.v_frag * (1.0 - P.frag_ramp)), kind);
            } else {
                mnew = outcome<T>(c, mi, msh[j], pi.mh, parts[j].mh, dmmi, STORE ? Dm[i * ld + j] : dvrow[j], dr.u3,
                                  kind);
            }
            const Part<T> pnew = make_part<T>(c, mnew, pi.Mv);
            const int stop = tn >= t_end;
            if (!stop) {
                if constexpr (TRACER) {
                    const double mj = msh[j];
                    qsh[i] = tracer_update(mi, mj, qsh[i], qsh[j], dgt(dmmi, mj) ? dmmi : mj, mnew, kind, c.chi);
                }
                msh[i] = mnew;
                parts[i] = pnew;
                sh.t = tn;
                if (logging && ev < A.log_cap) {
                    A.log_ijo[3 * ev] = i;
                    A.log_ijo[3 * ev + 1] = j;
                    A.log_ijo[3 * ev + 2] = kind;
                    A.log_t[ev] = tn;
                    A.log_m[ev] = mnew;
                }
            }
            sh.stop = stop;
        }
        __syncthreads();
        if (sh.stop) {
            // no lane bracketed j: the row's prefix sums are not finite
            if (sh.stop == 2 && k == 0) atomicOr(A.status, kStNaN);
            break;
        }
        // (5) new row and column i: R_k += r_ki(new) - r_ki(old); R_i afresh
        const Part<T> pn = parts[i];
        if (k == i) pk = pn;
        rown = (T)0;
        if (active) {
            T Knew;
            T dvn = pair_dv<T>(pc, pk, pn, &Knew);
            if (STORE) {
                Dm[i * ld + k] = dvn;
                Dm[k * ld + i] = dvn;
            }
            rown = Knew * weight<T>(pn, pk);
            if (k != i) R.update(Knew * weight<T>(pk, pn), colo);
        }
        pend = i;
        ++ev;
        if (--until_rebuild == 0) {
            if (STORE) rebuild_stored(); else rebuild();
            pend = -1;
            rown = (T)0;
            until_rebuild = reb;
        }
    }
    if (active) {
        A.m[off + k] = msh[k];
        if (TRACER) A.q[off + k] = qsh[k];
        if (A.Rdump) A.Rdump[off + k] = R.value() / c.sc;
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
    if (threadIdx.x == 0) c = make_cell<T>(P, GasTab{nullptr, 0}, rc, zc, 1.0, 0.0);
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        Part<T> a = make_part<T>(c, mi[q], (T)0), b = make_part<T>(c, mj[q], (T)0);
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
    if (threadIdx.x == 0) c = make_cell<T>(P, GasTab{nullptr, 0}, rc, zc, V, M[0]);
    __syncthreads();
    for (int q = threadIdx.x; q < n; q += blockDim.x) parts[q] = make_part<T>(c, m[q], (T)(M[q] * c.invVsc));
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

// ---- launchers -----------------------------------------------------------------------
constexpr size_t kExclusiveSmem = 120 * 1024;  // > half of an SM's shared memory

template <class T>
static size_t collide_smem(int nthr)
{
    return (size_t)nthr * (sizeof(Part<T>) + sizeof(double) + sizeof(T));
}

template <class T>
static cudaError_t collide_impl(mcd_ctx *cx, int from_state, double t_end)
{
    int nthr = cx->threads > 0 ? cx->threads : ((cx->n_max + 31) / 32) * 32;
    if (nthr < 32) nthr = 32;
    if (nthr > kMaxCell || nthr < cx->n_max) return cudaErrorInvalidValue;
    if (cx->C == 0) return cudaSuccess;
    const int b = cx->cur;
    k_cellconst<T><<<(unsigned)((cx->C + 127) / 128), 128, 0, cx->stream>>>(
        cx->d_params, cx->gas_knots, cx->gas_n, cx->cell_disk, cx->cell_start, cx->cell_n, cx->cell_b, cx->cell_V,
        cx->M[b], cx->cellk, cx->C);
    CollideArgs A;
    A.params = cx->d_params;
    A.disks = cx->d_disks;
    A.cell_disk = cx->cell_disk;
    A.cell_start = cx->cell_start;
    A.cell_n = cx->cell_n;
    A.cell_b = cx->cell_b;
    A.cell_V = cx->cell_V;
    A.cellk = cx->cellk;
    A.queue = cx->lpt ? cx->queue : nullptr;
    A.m = cx->m[b];
    A.M = cx->M[b];
    A.q = cx->tracer ? cx->q[b] : nullptr;
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
    // exclusive: request more than half an SM's shared memory so that no two
    // collide CTAs share an SM (the heaviest cells, launched first, run alone)
    size_t smem = collide_smem<T>(nthr);
    if (cx->exclusive && smem < kExclusiveSmem) smem = kExclusiveSmem;
    // FP32: the dv matrix (ld x ld, ld = n_max rounded up to odd) when it fits
    const int ld = cx->n_max | 1;
    const size_t smem_store = collide_smem<T>(nthr) + (size_t)ld * ld * sizeof(T) +
                              (cx->tracer ? (size_t)nthr * sizeof(double) : 0);
    // FP64: the matrices live in the workspace (when it holds them), not in shared memory
    const bool store = cx->dv_matrix && (sizeof(T) == 4 ? smem_store <= (size_t)cx->smem_optin : cx->dvg != nullptr);
    A.dv_ld = ld;
    A.dvg = cx->dvg;
    // a fragmentation ramp in any disk, or the tracer, selects the kernel variant with its branch
    auto go = [&](auto kernel, size_t bytes) {
        kernel<<<(unsigned)cx->C, nthr, bytes, cx->stream>>>(A);
        cx->launches += 2;
        return cudaGetLastError();
    };
    const size_t tq = cx->tracer ? (size_t)nthr * sizeof(double) : 0;  // the tracer's shared-memory copy
    if (store) {
        const size_t b = sizeof(T) == 4 ? (smem_store > smem + tq ? smem_store : smem + tq) : smem + tq;
        if (cx->tracer)
            return cx->ramp ? go(k_collide<T, true, true, true>, b) : go(k_collide<T, true, false, true>, b);
        return cx->ramp ? go(k_collide<T, true, true, false>, b) : go(k_collide<T, true, false, false>, b);
    }
    if (cx->tracer)
        return cx->ramp ? go(k_collide<T, false, true, true>, smem + tq) : go(k_collide<T, false, false, true>, smem + tq);
    return cx->ramp ? go(k_collide<T, false, true, false>, smem) : go(k_collide<T, false, false, false>, smem);
}

// the dynamic shared memory each variant may request; for the stored-matrix
// variants, what the device lets a block opt in to beyond its static part
template <class T, bool STORE>
static cudaError_t set_smem(int bytes)
{
    cudaError_t e = cudaSuccess;
    auto one = [&](auto kernel) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    };
    one(k_collide<T, STORE, false, false>);
    one(k_collide<T, STORE, true, false>);
    one(k_collide<T, STORE, false, true>);
    one(k_collide<T, STORE, true, true>);
    return e;
}

template <class T>
static cudaError_t prepare_impl(mcd_ctx *c)
{
    const size_t need = collide_smem<T>(kMaxCell);
    cudaError_t e = set_smem<T, false>((int)((need > kExclusiveSmem ? need : kExclusiveSmem) +
                                             (size_t)kMaxCell * sizeof(double)));  // + the tracer's copy
    c->smem_optin = 0;
    if constexpr (sizeof(T) != 4) {
        // the FP64 stored-matrix variants keep their matrices in global memory
        if (e == cudaSuccess)
            e = set_smem<T, true>((int)((need > kExclusiveSmem ? need : kExclusiveSmem) +
                                        (size_t)kMaxCell * sizeof(double)));
        return e;
    } else {
        if (e != cudaSuccess) return e;
        int dev = 0, optin = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
            return e;
        int st = 0;
        auto stat = [&](auto kernel) {
            cudaFuncAttributes fa;
            if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
            if (e == cudaSuccess && (int)fa.sharedSizeBytes > st) st = (int)fa.sharedSizeBytes;
        };
        stat(k_collide<T, true, false, false>);
        stat(k_collide<T, true, true, false>);
        stat(k_collide<T, true, false, true>);
        stat(k_collide<T, true, true, true>);
        if (e != cudaSuccess) return e;
        const int dyn = optin - st;
        if (dyn <= 0) return cudaSuccess;
        e = set_smem<T, true>(dyn);
        if (e == cudaSuccess) c->smem_optin = dyn;
        return e;
    }
}

cudaError_t prepare_collide(mcd_ctx *c)
{
    cudaError_t e = c->prec == MCD_MIXED ? prepare_impl<float>(c) : prepare_impl<double>(c);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rate_probe<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(1024 * sizeof(Part<double>)));
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
    cudaError_t e = cudaFuncSetAttribute(k_rate_probe<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(1024 * sizeof(Part<double>)));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_rate_probe<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(1024 * sizeof(Part<float>)));
    if (e != cudaSuccess) return e;
    if (prec == MCD_MIXED)
        k_rate_probe<float><<<1, 256, (size_t)n * sizeof(Part<float>), s>>>(p, rc, zc, V, n, m, M, rate, R);
    else
        k_rate_probe<double><<<1, 256, (size_t)n * sizeof(Part<double>), s>>>(p, rc, zc, V, n, m, M, rate, R);
    return cudaGetLastError();
}

}  // namespace mcd
