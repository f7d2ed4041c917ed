// mcd_diag.cu -- diagnostics: the dust mass distribution versus distance (the
// Benchmark section compares the codes by the dust surface density as a
// function of particle mass and distance from the star), in summary form:
// per radial bin [edges[b], edges[b+1]), the swarm-mass-weighted sums of the
// representative mass's first three powers and the particle count.
//
// One CTA per bin scans the disk's particles; every thread keeps Neumaier-
// compensated sums over a fixed stride of them and the CTA combines the
// threads' sums in a fixed tree, so the result does not depend on scheduling.
// Products and sums are explicitly rounded (no fused multiply-add), like the
// plain CPU evaluation they are compared with.
#include "mcd_internal.cuh"

namespace mcd {

constexpr int kDiagThreads = 256;

struct NSum {
    double s, c;
    __device__ void add(double x)
    {
        const double t = __dadd_rn(s, x);
        c = fabs(s) >= fabs(x) ? __dadd_rn(c, __dadd_rn(__dsub_rn(s, t), x))
                               : __dadd_rn(c, __dadd_rn(__dsub_rn(x, t), s));
        s = t;
    }
};

__global__ void __launch_bounds__(kDiagThreads) k_moments(const double *m, const double *M, const double *r,
                                                          int64_t n, const double *edges, double *out)
{
    __shared__ double ss[5][kDiagThreads], cs[5][kDiagThreads];
    const int b = blockIdx.x, k = threadIdx.x;
    const double lo = edges[b], hi = edges[b + 1];
    NSum acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q].s = acc[q].c = 0.0;
    for (int64_t i = k; i < n; i += kDiagThreads) {
        const double ri = r[i];
        if (!(ri >= lo && ri < hi)) continue;
        const double w = M[i], x = m[i];
        const double w1 = __dmul_rn(w, x), w2 = __dmul_rn(w1, x), w3 = __dmul_rn(w2, x);
        acc[0].add(w);
        acc[1].add(w1);
        acc[2].add(w2);
        acc[3].add(w3);
        acc[4].add(1.0);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        ss[q][k] = acc[q].s;
        cs[q][k] = acc[q].c;
    }
    __syncthreads();
    for (int h = kDiagThreads / 2; h > 0; h >>= 1) {
        if (k < h) {
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                NSum a{ss[q][k], cs[q][k]};
                a.add(ss[q][k + h]);
                ss[q][k] = a.s;
                cs[q][k] = __dadd_rn(a.c, cs[q][k + h]);
            }
        }
        __syncthreads();
    }
    if (k < 5) out[5 * b + k] = __dadd_rn(ss[k][0], cs[k][0]);
}

// ---- sigma_d(m, r) map: swarm mass per (radial bin, mass bin) --------------
// Every particle's M enters as a 64-bit integer count of a power-of-two unit
// 2^(e-62), 2^e at least the disk's total live swarm mass, so no sum can
// overflow and integer atomics make the sums independent of the order of
// the additions.  M times a power of two is exact; each M is rounded once, to
// the nearest unit (2^-61 of the total at most).

// e = the exponent of the unit's 2^62 multiple; the sum is compensated and
// combined in a fixed order (one CTA)
__global__ void __launch_bounds__(kDiagThreads) k_map_unit(const double *M, const double *r, int64_t n, int *e_out)
{
    __shared__ double ss[kDiagThreads], cs[kDiagThreads];
    const int k = threadIdx.x;
    NSum a{0.0, 0.0};
    for (int64_t i = k; i < n; i += kDiagThreads)
        if (r[i] < INFINITY) a.add(M[i]);
    ss[k] = a.s;
    cs[k] = a.c;
    __syncthreads();
    for (int h = kDiagThreads / 2; h > 0; h >>= 1) {
        if (k < h) {
            NSum b{ss[k], cs[k]};
            b.add(ss[k + h]);
            ss[k] = b.s;
            cs[k] = __dadd_rn(b.c, cs[k + h]);
        }
        __syncthreads();
    }
    if (k == 0) {
        const double tot = __dadd_rn(ss[0], cs[0]);
        *e_out = tot > 0.0 ? ilogb(tot) + 2 : 0;  // 2^e > tot with a margin for the rounding of the sum
    }
}

// the last edge not above v, for e[0] <= v < e[n] (non-decreasing edges)
__device__ __forceinline__ int last_not_above(const double *e, int n, double v)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (e[mid] <= v)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_map_add(const double *m, const double *M, const double *r, int64_t n, const double *re, int nr,
                          const double *me, int nm, const int *e_unit, unsigned long long *acc)
{
    const int sh = 62 - *e_unit;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ri = r[i], mi = m[i];
        if (!(ri >= re[0] && ri < re[nr]) || !(mi >= me[0] && mi < me[nm])) continue;
        const int b = last_not_above(re, nr, ri), q = last_not_above(me, nm, mi);
        atomicAdd(&acc[(int64_t)b * nm + q], __double2ull_rn(scalbn(M[i], sh)));
    }
}

__global__ void k_map_out(const unsigned long long *acc, int64_t nb, const int *e_unit, double *out)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < nb) out[k] = scalbn(__ull2double_rn(acc[k]), *e_unit - 62);
}

cudaError_t launch_sigma_map(mcd_ctx *c, int disk, int nr, int nm)
{
    const DiskDev &D = c->hd[disk];
    const int b = c->cur;
    const int64_t nb = (int64_t)nr * nm;
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(c->map_acc);
    int *e_unit = reinterpret_cast<int *>(c->map_acc + nb);
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * nb, c->stream);
    if (e != cudaSuccess) return e;
    k_map_unit<<<1, kDiagThreads, 0, c->stream>>>(c->M[b] + D.p_off, c->r[b] + D.p_off, D.n0, e_unit);
    unsigned g = (unsigned)((D.n0 + 255) / 256);
    if (g > 1216) g = 1216;
    if (g == 0) g = 1;
    k_map_add<<<g, 256, 0, c->stream>>>(c->m[b] + D.p_off, c->M[b] + D.p_off, c->r[b] + D.p_off, D.n0,
                                        c->map_redges, nr, c->map_medges, nm, e_unit, acc);
    k_map_out<<<(unsigned)((nb + 255) / 256), 256, 0, c->stream>>>(acc, nb, e_unit, c->map_out);
    c->launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_moments(mcd_ctx *c, int disk, int nbins)
{
    const DiskDev &D = c->hd[disk];
    const int b = c->cur;
    k_moments<<<(unsigned)nbins, kDiagThreads, 0, c->stream>>>(c->m[b] + D.p_off, c->M[b] + D.p_off,
                                                              c->r[b] + D.p_off, D.n0, c->diag_edges, c->diag_out);
    c->launches += 1;
    return cudaGetLastError();
}

}  // namespace mcd
