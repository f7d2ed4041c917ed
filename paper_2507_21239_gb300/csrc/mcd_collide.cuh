// mcd_collide.cuh -- the representative-particle collision step (Summary of
// the mcdust paper; Zsom & Dullemond 2008): per cell, the rate of swarm i
// meeting a particle of swarm j is r_ij = K_ij n_j g_ij with
// K_ij = pi (a_i + a_j)^2 dv_ij, n_j = M_j / (m_j V) and the grouping factor
// g_ij = min(1, m_j / (dm m_i)); events follow with exponential waiting times
// from R_tot = sum_i R_i, i chosen by R_i and j by r_ij, and only row and
// column i change after an event.
//
// GB300 layout: one CTA per cell, S swarms per thread (S = 1 or 2; swarm k is
// owned by thread k / S).  The per-swarm cache (radius, Stokes number,
// drag-law flags, 1/m, M/V, ...) sits in shared memory; each thread keeps the
// row sums R_k of its swarms in registers.  The per-cell gas constants come
// from a separate one-thread-per-cell kernel.  One event = a block scan that
// chooses i (and folds in the previous event's fresh R_i), row/column i
// before the event (read from the cell's stored dv matrix, or one kernel
// entry per swarm), a block scan whose bracketing lane chooses j and applies
// the outcome itself, and one kernel entry per swarm for the new row/column
// i: four block barriers.  A launch either takes one cell per CTA, or runs
// persistent CTAs that pull cells from the largest-work-first queue with an
// atomic ticket.
//
// The stored dv matrix is symmetric (dv_ij = dv_ji bit for bit) and is kept
// in circulant half form: row i holds the partners j = i + d (mod n) for
// 0 <= d < n/2, and d = n/2 when i < j, so each unordered pair is stored once
// and a full build evaluates n(n+1)/2 kernel entries.  It lives in shared
// memory (FP32, when it fits) or in the workspace (FP64; FP32 for cells too
// large for shared memory).
//
// Precision (template T): T = double is the plain FP64 path.  T = float is
// the mixed path: dv, sigma, K, rates, waiting times and partner choice in
// FP32; masses and the cell clock in FP64 (touched by one lane per event,
// because an FP64 instruction costs ~64 cycles on GB300); row sums R_k as
// compensated FP32 pairs.  The total rate R_tot (which sets the waiting time)
// and the fresh R_i are block sums of the row sums' leading parts, a tree of
// at most 9 levels of FP32 additions (relative error below 10 ulp, formed
// afresh every event, so nothing drifts); with the exact_total option they
// are compensated sums (TwoSum) formed by one extra warp that holds no swarm,
// from the row sums every thread posts to shared memory, while the other
// warps read row i.  Stokes-number
// differences use a factored difference of cubes over masses split into
// (hi, lo) FP32 pairs and St itself is carried as a (hi, lo) pair, so close
// masses lose no digits; drag-law and turbulence regimes are decided by mass
// thresholds held as (hi, lo) pairs of the FP64 values.
#pragma once
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

// ---- the cell's symmetric dv matrix in circulant half form ---------------------------
// Position of the unordered pair {i, j} of an n-swarm cell in rows of width W:
// row i holds d = (j - i) mod n for 2d < n, and for 2d = n when i < j; the
// other pairs sit in row j at n - d.  With W even, a warp reading row i
// (lane k: the pair {i, k}) touches consecutive words in row i and words
// W - 1 apart in the lanes' own rows, so shared-memory reads do not conflict.
__device__ __forceinline__ int sym_at(int i, int j, int n, int W)
{
    int d = j - i;
    if (d < 0) d += n;
    const int d2 = 2 * d;
    return (d2 < n || (d2 == n && i < j)) ? i * W + d : j * W + (n - d);
}

// ---- partner choice ----------------------------------------------------------
// Choose element k with probability x_k / total: the first k whose inclusive
// prefix exceeds u * total.  Thread t holds elements S t .. S t + S - 1.  With
// FUSE the scan also sums y over the block (the previous event's new row) and
// folds that sum in as element pend's value (x_pend is then 0).  A shuffle
// scan of the threads' sums within each warp, then a shuffle scan of the warp
// totals held one per lane; every warp knows the range [lo, hi) of the prefix
// it covers, lo of warp w+1 bit-identical to hi of warp w, so exactly one warp
// brackets the target and finds the thread by a ballot (and the element
// within the thread from the previous thread's prefix).  block_bracket returns
// the element in that warp's lane 0 and -1 in every other lane (one barrier).
// A passive warp (no elements) skips its own scan.
template <class V, int S, bool FUSE>
__device__ __forceinline__ int block_bracket(const V (&x)[S], const V (&y)[S], V u, int pend, V *buf, V &total,
                                             V &ysum, bool passive = false)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    V wi = x[0], ys = FUSE ? y[0] : (V)0;
    if (!passive) {  // (warp-uniform: a warp without elements skips its own scan)
#pragma unroll
        for (int s = 1; s < S; ++s) {
            wi += x[s];
            if (FUSE) ys += y[s];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const V a = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += a;
            if (FUSE) ys += __shfl_xor_sync(FULL, ys, o);
        }
    }
    if (lane == 31) {
        buf[2 * w] = wi;
        buf[2 * w + 1] = ys;
    }
    __syncthreads();
    // lane q holds warp q's total (q < nw <= 16); scan them in registers
    V bs = lane < nw ? buf[2 * lane] : (V)0;
    V by = (FUSE && lane < nw) ? buf[2 * lane + 1] : (V)0;
#pragma unroll
    for (int o = 1; o < kMaxCell / 32; o <<= 1) {
        if (o >= nw) break;  // (block-uniform) log2(nw) rounds
        const V a = __shfl_up_sync(FULL, bs, o);
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
    const int e0 = S * (int)threadIdx.x;
    const V P = (off + wi) + ((pend >= 0 && e0 + S - 1 >= pend) ? Rp : (V)0);
    const V lo = off + ((pend >= 0 && S * 32 * w > pend) ? Rp : (V)0);
    const V hi = hib + ((pend >= 0 && S * 32 * (w + 1) - 1 >= pend) ? Rp : (V)0);
    const unsigned bal = __ballot_sync(FULL, P > target);
    // (a tree scan may leave lane 31's prefix an ulp below hi: then lane 31)
    const int l = __ffs(bal | 0x80000000u) - 1;
    int sub = 0;
    if constexpr (S > 1) {
        // the element of this thread that brackets: the first whose prefix,
        // counted on from the previous thread's, exceeds the target (an element
        // of zero weight is never taken)
        V e = __shfl_up_sync(FULL, P, 1);
        if (lane == 0) e = lo;
        int first = -1, last = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const V v = x[s] + ((pend >= 0 && e0 + s == pend) ? Rp : (V)0);
            e += v;
            if (v > (V)0) {
                last = s;
                if (first < 0 && e > target) first = s;
            }
        }
        sub = __shfl_sync(FULL, first >= 0 ? first : last, l);
    }
    return (lane == 0 && lo <= target && target < hi) ? S * (32 * w + l) + sub : -1;
}

// ---- compensated FP32 sums ---------------------------------------------------------
// a + b = s + *err exactly (Knuth's TwoSum; no fused operations)
__device__ __forceinline__ float two_sum(float a, float b, float *err)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    *err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
// a compensated pair (h, e) plus x: h takes the rounded sum, e gathers the errors
__device__ __forceinline__ void comp_add(float &h, float &e, float x)
{
    float r;
    h = two_sum(h, x, &r);
    e = __fadd_rn(e, r);
}
// the compensated sum of (h, e) over the warp, in every lane (the same bits:
// each addition is commutative and its error exact)
__device__ __forceinline__ void warp_comp_sum(float &h, float &e)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), oe = __shfl_xor_sync(0xffffffffu, e, o);
        float r;
        h = two_sum(h, oh, &r);
        e = __fadd_rn(__fadd_rn(e, oe), r);
    }
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
    __device__ void set2(double h, double l) { s = h + l; }
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
    __device__ void set2(float h, float l) { s = h, c = l; }
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
    const unsigned char *cellk;  // per-cell constants, kCellKBytes each
    const int32_t *queue;        // this launch's part of the queue: entry -> cell (null: entry = cell)
    int64_t n_queue;             // entries in this launch
    int32_t *qhead;              // persistent CTAs: the ticket counter (zero at launch); null: one CTA per entry
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
    double *Rdump;  // per particle: the row sums at the end (null: off)
    double *Rtot;   // per cell: the total rate of the last choice scan (with Rdump)
    int64_t log_cell;
    int32_t *log_ijo;
    double *log_t, *log_m;
    unsigned long long *log_n;
    int64_t log_cap;
    int dv_w;         // row width of the stored matrix (STORE)
    int dv_rows;      // rows per cell of the stored matrix (the class's largest cell)
    double *q;        // the tracer column (TRACER variants)
    void *dvg;        // STORE == 2: the class's matrices in the workspace, dv_rows x dv_w entries of T per queue entry
};

template <class T>
struct Shared {
    CellK<T> c;
    T scan[2][64];
    float tot_h, tot_e, y_h, y_e;  // FP32: the helper warp's compensated total rate and fresh row sum
    int sel;
    Draw<T> ring[32];
    double t;    // the cell clock
    int stop;    // 0 event applied, 1 crossing t_end, 2 no partner bracketed
    int ticket;  // persistent CTAs: the queue entry taken
};

// One cell's event chain.  STORE: 0 recompute row i before every event, 1 the
// circulant half matrix in shared memory, 2 in the workspace.  TRACER: the
// swarms carry a tracer column (shared-memory copy after the dv row), updated
// on every event.  RAMP: a fragmentation probability ramp below v_frag.
// entry: the cell's position in this launch's queue, which also picks its
// slot of the launch's workspace matrices (STORE == 2; rebuilt at every start)
template <class T, int S, int STORE, bool RAMP, bool TRACER, bool EXACT>
__device__ __forceinline__ void cell_chain(const CollideArgs &A, const int64_t cell, const int64_t entry,
                                           Shared<T> &sh, unsigned char *smem_raw)
{
    const int nslot = blockDim.x * S;
    Part<T> *parts = reinterpret_cast<Part<T> *>(smem_raw);
    double *msh = reinterpret_cast<double *>(parts + nslot);
    T *dvrow = reinterpret_cast<T *>(msh + nslot);
    double *qsh = reinterpret_cast<double *>(dvrow + nslot);  // TRACER
    constexpr bool COMP = sizeof(T) == 4 && EXACT;
    // (exact total) every swarm's row sum (s, c) and new-row entry, posted for the helper warp
    float4 *post = reinterpret_cast<float4 *>(TRACER ? reinterpret_cast<unsigned char *>(qsh + nslot)
                                                     : reinterpret_cast<unsigned char *>(qsh));
    T *Dm = reinterpret_cast<T *>(COMP ? reinterpret_cast<unsigned char *>(post + nslot)
                                       : reinterpret_cast<unsigned char *>(post));  // STORE == 1
    const int W = A.dv_w;
    if constexpr (STORE == 2) Dm = reinterpret_cast<T *>(A.dvg) + (size_t)entry * A.dv_rows * W;
    const int k0 = S * (int)threadIdx.x;  // this thread's first swarm
    const int lane = threadIdx.x & 31;
    // FP32 with the compensated total (EXACT): the last warp holds no swarm; it
    // sums the posted row sums into the compensated total rate while the others
    // form row i
    constexpr bool comp = COMP;
    const bool helper = comp && (int)(threadIdx.x >> 5) == (int)(blockDim.x >> 5) - 1;
    const int n = A.cell_n[cell];
    if (n <= 0) {
        if (threadIdx.x == 0) A.cell_events[cell] = 0;
        return;
    }
    if (n > nslot || (STORE && (n > A.dv_rows || n / 2 >= W))) {
        if (threadIdx.x == 0) atomicOr(A.status, kStBadCell);
        return;
    }
    const int disk = A.cell_disk[cell];
    const int64_t off = A.cell_start[cell];
    if (threadIdx.x == 0) sh.c = *reinterpret_cast<const CellK<T> *>(A.cellk + cell * kCellKBytes);
    __syncthreads();
    const CellK<T> &c = sh.c;
    // FP32: the entry constants in registers; FP64: read in place (register budget)
    typedef typename std::conditional<sizeof(T) == 4, PairK<T>, const CellK<T> &>::type PK;
    PK pc = [&]() -> PK {
        if constexpr (sizeof(T) == 4) return pair_consts<T>(sh.c); else return sh.c;
    }();
    bool act[S];
    Part<T> pk[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int k = k0 + s;
        act[s] = k < n;
        if (act[s]) {
            const double mk = A.m[off + k];
            // FP32 path: every mass the event loop can reach lies between the
            // monomer mass and the disk's dust mass, inside the split's range
            if (sizeof(T) == 4 && !mass_splits(mk)) atomicOr(A.status, kStBadCell);
            msh[k] = mk;
            if (TRACER) qsh[k] = A.q[off + k];
            pk[s] = make_part<T>(c, mk, (T)(A.M[off + k] * c.invVsc));
            parts[k] = pk[s];
        }
    }
    __syncthreads();

    Acc<T> R[S];
    // R_k = sum_j r_kj in j order, from the stored matrix
    auto row_sums_stored = [&]() {
#pragma unroll
        for (int s = 0; s < S; ++s) {
            R[s].zero();
            if (act[s]) {
                const int k = k0 + s;
                for (int j = 0; j < n; ++j) {
                    const Part<T> pj = parts[j];
                    R[s].add(kern_of<T>(pc, pk[s].a, pj.a, Dm[sym_at(k, j, n, W)]) * weight<T>(pk[s], pj));
                }
            }
        }
    };
    // full build of the row sums.  STORE: every unordered pair once (warp w
    // takes rows w, w + nw, ...; its lanes consecutive offsets d, so the
    // stores are consecutive words), then the sums from the stored entries.
    // Otherwise every swarm's full row, four independent entries in flight.
    auto build = [&]() {
        if constexpr (STORE != 0) {
            const int nw = blockDim.x >> 5, w = threadIdx.x >> 5;
            for (int rr = w; rr < n; rr += nw) {
                const Part<T> pr = parts[rr];
                const int dmax = (n - 1) / 2 + (((n & 1) == 0 && rr < n / 2) ? 1 : 0);
                for (int d = lane; d <= dmax; d += 32) {
                    int j = rr + d;
                    if (j >= n) j -= n;
                    T K;
                    Dm[rr * W + d] = pair_dv<T>(pc, pr, parts[j], &K);
                }
            }
            __syncthreads();
            row_sums_stored();
        } else {
#pragma unroll
            for (int s = 0; s < S; ++s) {
                R[s].zero();
                if (act[s]) {
                    int j = 0;
                    // (FP64: no unrolling; its register budget is spent on the wider values)
                    for (; sizeof(T) == 4 && j + 4 <= n; j += 4) {
                        T K0, K1, K2, K3;
                        const Part<T> p0 = parts[j], p1 = parts[j + 1], p2 = parts[j + 2], p3 = parts[j + 3];
                        pair_dv<T>(pc, pk[s], p0, &K0);
                        pair_dv<T>(pc, pk[s], p1, &K1);
                        pair_dv<T>(pc, pk[s], p2, &K2);
                        pair_dv<T>(pc, pk[s], p3, &K3);
                        R[s].add(K0 * weight<T>(pk[s], p0));
                        R[s].add(K1 * weight<T>(pk[s], p1));
                        R[s].add(K2 * weight<T>(pk[s], p2));
                        R[s].add(K3 * weight<T>(pk[s], p3));
                    }
                    for (; j < n; ++j) {
                        const Part<T> pj = parts[j];
                        T K;
                        pair_dv<T>(pc, pk[s], pj, &K);
                        R[s].add(K * weight<T>(pk[s], pj));
                    }
                }
            }
        }
    };
    build();

    // the random stream is keyed by (seed, disk) and counted by
    // (event, disk-local cell, step, domain tag)
    const uint64_t dcell = (uint64_t)(cell - A.disks[disk].c_off);
    const uint64_t step = (uint64_t)A.state->step;
    const double t_end = A.t_end_from_state ? A.state->t + A.state->dt : A.t_end_fixed;
    const int64_t reb = A.rebuild_every > 0 ? A.rebuild_every : 4 * (int64_t)n;
    int64_t until_rebuild = reb;  // events left before the next full rebuild
    const bool logging = (cell == A.log_cell);
    const T sc = (T)c.sc;
    if (threadIdx.x == 0) sh.t = A.state->t;  // (visible after the first ring barrier)
    int64_t ev = 0;
    int pend = -1;  // swarm whose fresh row sum rides on the next scan
    T rown[S], colo[S], row[S], zero[S];
#pragma unroll
    for (int s = 0; s < S; ++s) rown[s] = colo[s] = row[s] = zero[s] = (T)0;
    T last_tot = (T)0;  // the total rate of the last choice scan (rate-scaled)
    float last_e = 0.0f; // (exact total) its compensation
    for (;;) {
        if ((ev & 31) == 0) {
            if (threadIdx.x < 32)
                sh.ring[threadIdx.x] = make_draw(
                    philox((uint64_t)(ev + threadIdx.x), dcell, step, kTagCollide, A.seed, (uint64_t)disk), sc);
            __syncthreads();
        }
        const Draw<T> dr = sh.ring[ev & 31];
        // (1) choose i: first k whose inclusive prefix of R exceeds u1 R_tot;
        //     the previous event's R_i (sum of its new row) is folded in here
        T val[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const bool live = act[s] && k0 + s != pend;
            val[s] = live ? (T)R[s].hi() : (T)0;
            if constexpr (COMP)  // (the helper reads these after the choice)
                if (act[s])
                    post[k0 + s] = make_float4(live ? R[s].s : 0.0f, live ? R[s].c : 0.0f, rown[s], 0.0f);
        }
        T tot, Rp;
        if (threadIdx.x == 0) sh.sel = -1;
        {
            const int f = block_bracket<T, S, true>(val, rown, dr.u1, pend, sh.scan[0], tot, Rp, helper);
            if (f >= 0) sh.sel = f;
            __syncthreads();
        }
        int i = sh.sel;
        if constexpr (COMP) {
            if (helper) {
                // the compensated sums of the posted row sums (their own
                // compensations added alongside) and of the new row: the total
                // rate that sets the waiting time, and the fresh row sum of the
                // previous i
                float h = 0.0f, e = 0.0f, yh = 0.0f, ye = 0.0f;
                for (int k = lane; k < n; k += 32) {
                    const float4 v = post[k];
                    comp_add(h, e, v.x);
                    e = __fadd_rn(e, v.y);
                    comp_add(yh, ye, v.z);
                }
                warp_comp_sum(h, e);
                warp_comp_sum(yh, ye);
                if (lane == 0) {
                    if (pend < 0) yh = ye = 0.0f;
                    float r;
                    sh.tot_h = two_sum(h, yh, &r);
                    sh.tot_e = __fadd_rn(__fadd_rn(e, ye), r);
                    sh.y_h = yh;
                    sh.y_e = ye;
                }
            }
        }
        last_tot = tot;
#pragma unroll
        for (int s = 0; s < S; ++s)
            if (pend >= 0 && k0 + s == pend) R[s].set(Rp);  // (its compensated value follows after the event)
        if (!(tot > (T)0) || ev >= A.max_events) {
            if (ev >= A.max_events && tot > (T)0 && !A.cap_stops && threadIdx.x == 0) atomicOr(A.status, kStTimeout);
            if (comp && A.Rtot) {  // (uniform branch)
                __syncthreads();
                if (threadIdx.x == 0) {
                    last_tot = sh.tot_h;
                    last_e = sh.tot_e;
                }
            }
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
        if (threadIdx.x == 0) sh.stop = 2;
        // (2) row i (i meets k) and column i (k meets i) before the event
        const Part<T> pi = parts[i];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            row[s] = colo[s] = (T)0;
            if (act[s]) {
                const int k = k0 + s;
                T Kold;
                if constexpr (STORE != 0) {
                    const T dvik = Dm[sym_at(i, k, n, W)];
                    if (STORE == 2) dvrow[k] = dvik;  // (the outcome reads it from shared memory)
                    Kold = kern_of<T>(pc, pk[s].a, pi.a, dvik);
                } else {
                    dvrow[k] = pair_dv<T>(pc, pk[s], pi, &Kold);
                }
                row[s] = Kold * weight<T>(pi, pk[s]);
                colo[s] = Kold * weight<T>(pk[s], pi);
            }
        }
        // (3) choose j by the row's prefix; (4) the lane that finds j advances
        //     the clock and, unless the event would cross t_end (memoryless:
        //     discarded), applies the outcome and the new cache of i (FP64 masses)
        T tot2, unused;
        int j = block_bracket<T, S, false>(row, zero, dr.u2, -1, sh.scan[1], tot2, unused, helper);
        if (j >= 0) {
            if (j >= n) j = n - 1;  // (lane 31 fallback in a partly idle warp)
            // the clock, the outcome and the new cache are independent chains;
            // only the stores wait for the crossing test.  FP32: the total rate
            // is the helper warp's compensated sum
            T Rt = tot;
            if constexpr (COMP)
                if (comp) Rt = __fadd_rn(sh.tot_h, sh.tot_e);
            const double tn = sh.t + (double)fdiv(dr.L, Rt);
            int kind = 0;
            double mnew;
            const T dvij = STORE == 1 ? Dm[sym_at(i, j, n, W)] : dvrow[j];
            if constexpr (RAMP) {  // the ramp's foot as the plain FP64 evaluation forms it
                const mcd_disk_params &P = A.params[disk];
                mnew = outcome_ramp<T>(c, mi, msh[j], pi.mh, parts[j].mh, dmmi, dvij, dr.u3,
                                       (T)(P.v_frag * (1.0 - P.frag_ramp)), kind);
            } else {
                mnew = outcome<T>(c, mi, msh[j], pi.mh, parts[j].mh, dmmi, dvij, dr.u3, kind);
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
        if (comp && A.Rtot && threadIdx.x == 0) {
            last_tot = sh.tot_h;
            last_e = sh.tot_e;
        }
        if (sh.stop) {
            // no lane bracketed j: the row's prefix sums are not finite
            if (sh.stop == 2 && threadIdx.x == 0) atomicOr(A.status, kStNaN);
            break;
        }
        if constexpr (COMP) {
            if (comp)
#pragma unroll
                for (int s = 0; s < S; ++s)
                    if (pend >= 0 && k0 + s == pend) R[s].set2(sh.y_h, sh.y_e);  // the compensated fresh row sum
        }
        // (5) new row and column i: R_k += r_ki(new) - r_ki(old); R_i afresh
        const Part<T> pn = parts[i];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const int k = k0 + s;
            if (k == i) pk[s] = pn;
            rown[s] = (T)0;
            if (act[s]) {
                T Knew;
                const T dvn = pair_dv<T>(pc, pk[s], pn, &Knew);
                if constexpr (STORE != 0) Dm[sym_at(i, k, n, W)] = dvn;
                rown[s] = Knew * weight<T>(pn, pk[s]);
                if (k != i) R[s].update(Knew * weight<T>(pk[s], pn), colo[s]);
            }
        }
        pend = i;
        ++ev;
        if (--until_rebuild == 0) {
            if constexpr (STORE != 0) {
                __syncthreads();  // (entries written by other threads since the last barrier)
                row_sums_stored();
            } else {
                build();
            }
            pend = -1;
#pragma unroll
            for (int s = 0; s < S; ++s) rown[s] = (T)0;
            until_rebuild = reb;
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (act[s]) {
            const int k = k0 + s;
            A.m[off + k] = msh[k];
            if (TRACER) A.q[off + k] = qsh[k];
            if (A.Rdump) A.Rdump[off + k] = R[s].value() / c.sc;
        }
    if (threadIdx.x == 0) {
        A.cell_events[cell] = ev;
        atomicAdd(&A.events_total[disk], (unsigned long long)ev);
        if (logging) *A.log_n = (unsigned long long)(ev < A.log_cap ? ev : A.log_cap);
        if (A.Rtot) A.Rtot[cell] = ((double)last_tot + (double)last_e) / c.sc;
    }
}

// One CTA per queue entry, or (qhead set) persistent CTAs that take entries
// by an atomic ticket until the queue is exhausted.
template <class T, int S, int STORE, bool RAMP, bool TRACER, bool EXACT>
__global__ void __launch_bounds__(kMaxCell / S) k_collide(CollideArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<T> sh;
    int64_t entry = blockIdx.x;
    for (;;) {
        if (A.qhead) {
            __syncthreads();  // the previous cell's shared data is no longer read
            if (threadIdx.x == 0) sh.ticket = atomicAdd(A.qhead, 1);
            __syncthreads();
            entry = sh.ticket;
        }
        if (entry >= A.n_queue) return;
        const int64_t cell = A.queue ? (int64_t)A.queue[entry] : entry;
        cell_chain<T, S, STORE, RAMP, TRACER, EXACT>(A, cell, entry, sh, smem_raw);
        if (!A.qhead) return;
    }
}

// dynamic shared memory of a collide CTA of nthr threads (S swarms each):
// caches, masses, the dv row, the tracer copy and (FP32, exact total) the
// posted row sums; plus the stored matrix (STORE == 1) of rows x W entries
template <class T>
inline size_t collide_smem_bytes(int nthr, int S, bool tracer, int store, int rows, int W, bool exact)
{
    const size_t slots = (size_t)nthr * S;
    size_t b = slots * (sizeof(Part<T>) + sizeof(double) + sizeof(T)) + (tracer ? slots * sizeof(double) : 0) +
               (sizeof(T) == 4 && exact ? slots * sizeof(float4) : 0);
    if (store == 1) b += (size_t)rows * W * sizeof(T);
    return b;
}

// the variants' host entry points, one translation unit per (T, S, EXACT): op 0
// launches the (store, ramp, tracer) variant; op 1 sets every ramp/tracer
// variant of that store's dynamic shared-memory limit to `smem`; op 2 writes
// the largest static shared memory of those variants to *out; op 3 writes the
// variant's resident CTAs per SM at (nthr, smem) to *out
template <class T, int S, bool EXACT>
cudaError_t collide_variant(int op, int store, bool ramp, bool tracer, unsigned grid, int nthr, size_t smem,
                            cudaStream_t st, const CollideArgs *A, int *out);

template <class T, int S, int STORE, bool EXACT>
cudaError_t collide_variant_store(int op, bool ramp, bool tracer, unsigned grid, int nthr, size_t smem,
                                  cudaStream_t st, const CollideArgs *A, int *out)
{
    void (*ks[4])(CollideArgs) = {
        k_collide<T, S, STORE, false, false, EXACT>, k_collide<T, S, STORE, true, false, EXACT>,
        k_collide<T, S, STORE, false, true, EXACT>, k_collide<T, S, STORE, true, true, EXACT>};
    if (op == 0) {
        ks[(ramp ? 1 : 0) + (tracer ? 2 : 0)]<<<grid, nthr, smem, st>>>(*A);
        return cudaGetLastError();
    }
    if (op == 3) {  // resident CTAs per SM of the launch shape (nthr, smem)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, ks[(ramp ? 1 : 0) + (tracer ? 2 : 0)], nthr, smem);
    }
    cudaError_t e = cudaSuccess;
    int mx = 0;
    for (int v = 0; v < 4 && e == cudaSuccess; ++v) {
        if (op == 1) {
            e = cudaFuncSetAttribute(ks[v], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        } else {
            cudaFuncAttributes fa;
            e = cudaFuncGetAttributes(&fa, ks[v]);
            if (e == cudaSuccess && (int)fa.sharedSizeBytes > mx) mx = (int)fa.sharedSizeBytes;
        }
    }
    if (op == 2 && out) *out = mx;
    return e;
}

}  // namespace mcd
