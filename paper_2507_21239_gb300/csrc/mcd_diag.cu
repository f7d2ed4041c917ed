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
