// mcd_capi.cu -- the C ABI of libmcd.so (declared in include/mcd.h): context,
// workspace carving, argument checks, the step sequence and its CUDA graph.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "mcd_internal.cuh"


using namespace mcd;

namespace {

struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <class T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

struct Sizes {
    int64_t N = 0, C = 0, Z = 0, T = 0;
    int32_t n_max = 0;
    std::vector<DiskDev> disks;
    std::vector<CollideClass> cls;
    std::vector<int32_t> disk_class;
};

int plan(const mcd_disk_params *p, const mcd_grid *g, int32_t nd, int32_t prec, Sizes &S)
{
    if (!p || !g || nd <= 0) return MCD_EINVAL;
    S.disks.resize(nd);
    for (int d = 0; d < nd; ++d) {
        const mcd_grid &G = g[d];
        const mcd_disk_params &P = p[d];
        if (G.n_r <= 0 || G.n_z <= 0 || G.per_cell <= 0) return MCD_EINVAL;
        if (G.per_cell > kMaxCell) return MCD_EINVAL;
        if ((int64_t)G.n_z * G.per_cell > kZoneCap) return MCD_EINVAL;
        if (!(P.frag_ramp >= 0.0 && P.frag_ramp < 1.0)) return MCD_EINVAL;
        if (P.kernel_mode == 1) {
            if (!(P.V_const > 0.0) || !(P.m_init > 0.0)) return MCD_EINVAL;
        } else if (P.kernel_mode == 0) {
            if (!(P.r_in > 0.0) || !(P.r_out > P.r_in) || !(P.rho_s > 0.0) || !(P.a_mono > 0.0 || P.m_init > 0.0) ||
                !(P.m_star > 0.0) || !(P.mu > 0.0) || !(P.sigma_h2 > 0.0) || !(P.sigma0 > 0.0) || !(P.T0 > 0.0) ||
                !(P.alpha > 0.0) || !(P.dm_group >= 0.0) || !(P.frag_xi < 2.0 + 1e-12 || P.frag_xi > 2.0))
                return MCD_EINVAL;
        } else {
            return MCD_EINVAL;
        }
        DiskDev &D = S.disks[d];
        D.n_r = G.n_r;
        D.n_z = G.n_z;
        D.n0 = (int64_t)G.n_r * G.n_z * G.per_cell;
        D.p_off = S.N;
        D.c_off = S.C;
        D.z_off = S.Z;
        D.t_off = S.T;
        D.n_tiles = (D.n0 + kRadixTile - 1) / kRadixTile;
        S.N += D.n0;
        S.C += (int64_t)G.n_r * G.n_z;
        S.Z += G.n_r;
        S.T += D.n_tiles;
        if (G.per_cell > S.n_max) S.n_max = G.per_cell;
    }
    if (S.N >= ((int64_t)1 << 31)) return MCD_EINVAL;
    return plan_classes(g, nd, prec, S.cls, S.disk_class);
}

size_t carve(mcd_ctx *c, void *base, Sizes &S, int32_t nd, int32_t prec)
{
    Carver cv(base);
    mcd_ctx tmp;
    mcd_ctx *x = c ? c : &tmp;
    x->d_params = cv.take<mcd_disk_params>(nd);
    x->d_disks = cv.take<DiskDev>(nd);
    x->slot_disk = cv.take<int32_t>(S.N);
    x->cell_disk = cv.take<int32_t>(S.C);
    x->zone_disk = cv.take<int32_t>(S.Z);
    x->tile_disk = cv.take<int32_t>(S.T);
    for (int b = 0; b < 2; ++b) {
        x->m[b] = cv.take<double>(S.N);
        x->M[b] = cv.take<double>(S.N);
        x->r[b] = cv.take<double>(S.N);
        x->z[b] = cv.take<double>(S.N);
        x->id[b] = cv.take<uint32_t>(S.N);
        x->key[b] = cv.take<uint64_t>(S.N);
        x->val[b] = cv.take<uint32_t>(S.N);
        x->q[b] = cv.take<double>(S.N);
    }
    int64_t H = 256 * S.T;
    x->hist = cv.take<uint32_t>(H);
    x->scan_part = cv.take<uint32_t>(H / 4096 + 2);
    x->rfix_longs = cv.take<int64_t>(S.N / (kRunShortMax + 1) + 1);
    x->rfix_count = cv.take<int32_t>(2);
    x->cell_start = cv.take<int64_t>(S.C);
    x->cell_n = cv.take<int32_t>(S.C);
    x->cell_b = cv.take<double>(6 * S.C);
    x->cell_V = cv.take<double>(S.C);
    x->cellk = cv.take<unsigned char>((size_t)S.C * kCellKBytes);
    x->cell_events = cv.take<int64_t>(S.C);
    x->cell_cost = cv.take<uint32_t>(S.C);
    x->queue = cv.take<int32_t>(S.C);
    x->queue_static = cv.take<int32_t>(S.C);
    x->cell_class = cv.take<int32_t>(S.C);
    x->qcount = cv.take<int32_t>(kMaxClasses * 64 + 8);
    x->qheads = cv.take<int32_t>(kMaxClasses);
    x->Rtot = cv.take<double>(S.C);
    x->tune_scr = cv.take<unsigned long long>((size_t)nd + 2);
    x->n_alive = cv.take<int64_t>(nd);
    x->accreted = cv.take<double>(nd);
    x->events_total = cv.take<unsigned long long>(nd);
    x->Rdump = cv.take<double>(S.N);
    x->log_ijo = cv.take<int32_t>(3 * mcd_ctx::kLogCap);
    x->log_t = cv.take<double>(mcd_ctx::kLogCap);
    x->log_m = cv.take<double>(mcd_ctx::kLogCap);
    x->log_n = cv.take<unsigned long long>(1);
    x->status = cv.take<int32_t>(1);
    x->state = cv.take<StepState>(1);
    x->d_Mswarm = cv.take<double>(nd);
    x->diag_edges = cv.take<double>(MCD_MAX_BINS + 1);
    x->diag_out = cv.take<double>(5 * MCD_MAX_BINS);
    x->map_acc = cv.take<unsigned long long>(MCD_MAX_MAP_BINS + 1);
    x->map_redges = cv.take<double>(MCD_MAX_MAP_EDGES + 1);
    x->map_medges = cv.take<double>(MCD_MAX_MAP_EDGES + 1);
    x->map_out = cv.take<double>(MCD_MAX_MAP_BINS);
    x->gas_knots = cv.take<GasKnot>((size_t)nd * kMaxGasKnots);
    x->gas_n = cv.take<int32_t>(nd);
    x->dt_acc = cv.take<unsigned long long>(2 * (size_t)nd + 1);
    // the classes' stored dv matrices (where the plan reserves them)
    for (CollideClass &k : S.cls) k.dvg = k.reserve ? cv.take<unsigned char>(class_matrix_bytes(k, prec)) : nullptr;
    if (c) c->cls = S.cls;
    return (cv.off + 255) & ~(size_t)255;
}

double disk_dust_mass(const mcd_disk_params &P)
{
    if (P.M_total > 0.0) return P.M_total;
    double e = 2.0 - P.p, ri = P.r_in / kAU, ro = P.r_out / kAU;
    double I = fabs(e) < 1e-12 ? log(ro / ri) : (pow(ro, e) - pow(ri, e)) / e;
    return P.dust_to_gas * 2.0 * kPI * P.sigma0 * I * kAU * kAU;
}

int cuda_code(cudaError_t e) { return e == cudaSuccess ? MCD_OK : MCD_ECUDA; }

int status_code(int32_t st)
{
    if (st & kStNaN) return MCD_ENAN;
    if (st & kStBadCell) return MCD_EINVAL;
    if (st & kStTimeout) return MCD_ETIMEOUT;
    if (st & kStEmpty) return MCD_EEMPTY;
    return MCD_OK;
}

void drop_graphs(mcd_ctx *c)
{
    for (int k = 0; k < 2; ++k)
        if (c->gexec[k]) {
            cudaGraphExecDestroy(c->gexec[k]);
            c->gexec[k] = nullptr;
        }
}

// the context's streams, events and graphs, then the context
void destroy(mcd_ctx *c)
{
    drop_graphs(c);
    for (int k = 0; k < 5; ++k)
        if (c->tev[k]) cudaEventDestroy(c->tev[k]);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->cls_fork) cudaEventDestroy(c->cls_fork);
    for (int q = 0; q < kMaxClasses; ++q) {
        if (c->cls_stream[q]) cudaStreamDestroy(c->cls_stream[q]);
        if (c->cls_join[q]) cudaEventDestroy(c->cls_join[q]);
    }
    delete c;
}

cudaError_t enqueue_regrid(mcd_ctx *c)
{
    cudaError_t e = launch_regrid(c);
    c->cur ^= 1;
    return e;
}

cudaError_t mark(mcd_ctx *c, int k)
{
    return c->trace ? cudaEventRecordWithFlags(c->tev[k], c->stream, cudaEventRecordExternal) : cudaSuccess;
}

cudaError_t enqueue_step_body(mcd_ctx *c)
{
    cudaError_t e = mark(c, 0);
    if (e == cudaSuccess) e = enqueue_regrid(c);
    if (e == cudaSuccess) e = mark(c, 1);
    if (e == cudaSuccess && c->lpt) e = launch_lpt(c);
    if (e == cudaSuccess) e = mark(c, 2);
    if (e == cudaSuccess && c->graph_adaptive) e = launch_adaptive_dt(c);
    if (e == cudaSuccess) e = launch_collide_impl(c, 1, 0.0);
    if (e == cudaSuccess) e = mark(c, 3);
    if (e == cudaSuccess) e = launch_transport(c);
    if (e == cudaSuccess) e = launch_advance_clock(c, 1);
    if (e == cudaSuccess) e = mark(c, 4);
    return e;
}

}  // namespace

extern "C" {

int mcd_workspace_size(const mcd_disk_params *p, const mcd_grid *g, int32_t n_disks, int32_t prec, size_t *bytes)
{
    if (!bytes || (prec != MCD_FP64 && prec != MCD_MIXED)) return MCD_EINVAL;
    Sizes S;
    int rc = plan(p, g, n_disks, prec, S);
    if (rc) return rc;
    *bytes = carve(nullptr, nullptr, S, n_disks, prec);
    return MCD_OK;
}

int mcd_init_disk(mcd_ctx **out, const mcd_disk_params *p, const mcd_grid *g, int32_t n_disks, uint64_t seed,
                  int32_t prec, void *ws, size_t ws_bytes, void *stream)
{
    if (!out || !ws || (prec != MCD_FP64 && prec != MCD_MIXED)) return MCD_EINVAL;
    if (((uintptr_t)ws & 255) != 0) return MCD_EINVAL;
    *out = nullptr;
    Sizes S;
    int rc = plan(p, g, n_disks, prec, S);
    if (rc) return rc;
    size_t need = carve(nullptr, nullptr, S, n_disks, prec);
    if (ws_bytes < need) return MCD_ENOMEM;
    mcd_ctx *c = new (std::nothrow) mcd_ctx();
    if (!c) return MCD_ENOMEM;
    c->n_disks = n_disks;
    c->prec = prec;
    c->stream = (cudaStream_t)stream;
    c->seed = seed;
    c->hp.assign(p, p + n_disks);
    for (int32_t d = 0; d < n_disks; ++d)
        if (p[d].frag_ramp > 0.0) c->ramp = 1;
    c->hg.assign(g, g + n_disks);
    c->gas_n_host.assign(n_disks, 0);
    c->hd = S.disks;
    c->N = S.N;
    c->C = S.C;
    c->Z = S.Z;
    c->n_tiles = S.T;
    c->n_max = S.n_max;
    for (int32_t d = 0; d < n_disks; ++d) {
        const int64_t zc = (int64_t)g[d].n_z * g[d].per_cell;
        c->zone_max = c->zone_max > zc ? c->zone_max : zc;
        c->n0_max = c->n0_max > (int64_t)g[d].n_r * zc ? c->n0_max : (int64_t)g[d].n_r * zc;
    }
    carve(c, ws, S, n_disks, prec);
    double *d_Mswarm = c->d_Mswarm;

    // host-built tables
    std::vector<int32_t> cell_disk(S.C), zone_disk(S.Z), tile_disk(S.T), slot_disk(S.N);
    std::vector<double> Msw(n_disks);
    for (int d = 0; d < n_disks; ++d) {
        const DiskDev &D = S.disks[d];
        for (int64_t k = 0; k < (int64_t)D.n_r * D.n_z; ++k) cell_disk[D.c_off + k] = d;
        for (int64_t k = 0; k < D.n_r; ++k) zone_disk[D.z_off + k] = d;
        for (int64_t k = 0; k < D.n_tiles; ++k) tile_disk[D.t_off + k] = d;
        for (int64_t k = 0; k < D.n0; ++k) slot_disk[D.p_off + k] = d;
        Msw[d] = disk_dust_mass(p[d]) / (double)D.n0;
    }
    // collide classes: each cell's class, and the class-major cell order
    c->cell_class_host.assign(S.C, 0);
    for (int d = 0; d < n_disks; ++d) {
        const DiskDev &D = S.disks[d];
        for (int64_t k = 0; k < (int64_t)D.n_r * D.n_z; ++k) c->cell_class_host[D.c_off + k] = S.disk_class[d];
    }
    std::vector<int32_t> qstatic(S.C);
    std::vector<int64_t> fill(c->cls.size(), 0);
    for (int64_t x = 0; x < S.C; ++x) {
        const int q = c->cell_class_host[x];
        qstatic[c->cls[q].qoff + fill[q]++] = (int32_t)x;
    }
    cudaStream_t st = c->stream;
    cudaError_t e = cudaSuccess;
    if (c->cls.size() > 1) e = cudaEventCreateWithFlags(&c->cls_fork, cudaEventDisableTiming);
    for (size_t q = 1; q < c->cls.size() && e == cudaSuccess; ++q) {
        e = cudaStreamCreateWithFlags(&c->cls_stream[q], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->cls_join[q], cudaEventDisableTiming);
    }
    auto cp = [&](void *dst, const void *src, size_t n) {
        if (e == cudaSuccess && n) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, st);
    };
    cp(c->cell_class, c->cell_class_host.data(), 4 * S.C);
    cp(c->queue_static, qstatic.data(), 4 * S.C);
    cp(c->d_params, p, sizeof(mcd_disk_params) * n_disks);
    cp(c->d_disks, S.disks.data(), sizeof(DiskDev) * n_disks);
    cp(c->cell_disk, cell_disk.data(), 4 * S.C);
    cp(c->zone_disk, zone_disk.data(), 4 * S.Z);
    cp(c->tile_disk, tile_disk.data(), 4 * S.T);
    cp(c->slot_disk, slot_disk.data(), 4 * S.N);
    cp(d_Mswarm, Msw.data(), 8 * n_disks);
    StepState s0 = {0.0, 0.0, 0};
    cp(c->state, &s0, sizeof s0);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->status, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->accreted, 0, 8 * n_disks, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->events_total, 0, 8 * n_disks, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->cell_events, 0, 8 * S.C, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->log_n, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->gas_n, 0, 4 * n_disks, st);  // the power laws
    const std::vector<unsigned long long> rest = adaptive_dt_rest(n_disks);
    cp(c->dt_acc, rest.data(), 8 * rest.size());
    for (int b = 0; b < 2; ++b)  // the tracer starts at zero (uniform: its order does not matter)
        if (e == cudaSuccess) e = cudaMemsetAsync(c->q[b], 0, 8 * S.N, st);
    if (e == cudaSuccess) e = prepare_collide(c);
    if (e == cudaSuccess) e = prepare_zone(c);
    if (e == cudaSuccess) e = launch_init(c, d_Mswarm);
    if (e == cudaSuccess) e = enqueue_regrid(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        destroy(c);
        return MCD_ECUDA;
    }
    c->cells_valid = true;
    *out = c;
    return MCD_OK;
}

int mcd_regrid(mcd_ctx *c)
{
    if (!c) return MCD_EINVAL;
    int rc = cuda_code(enqueue_regrid(c));
    if (rc == MCD_OK) c->cells_valid = true;
    return rc;
}

int mcd_collide(mcd_ctx *c, double t_end)
{
    if (!c) return MCD_EINVAL;
    if (!c->t_known) {  // after adaptive steps the clock lives on the device
        StepState s;
        if (cudaMemcpyAsync(&s, c->state, sizeof s, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess)
            return MCD_ECUDA;
        c->t_host = s.t;
        c->t_known = true;
    }
    if (!(t_end >= c->t_host)) return MCD_EINVAL;
    if (!c->cells_valid) return MCD_ESTATE;
    cudaError_t e = tune_collide(c);
    if (e == cudaSuccess && c->lpt) e = launch_lpt(c);
    if (e == cudaSuccess) e = launch_collide_impl(c, 0, t_end);
    if (e == cudaSuccess) e = launch_set_clock(c, t_end, 1, 0.0, 0);
    if (e == cudaSuccess) c->t_host = t_end;
    return cuda_code(e);
}

int mcd_transport(mcd_ctx *c, double dt)
{
    if (!c || !(dt > 0.0) || !isfinite(dt)) return MCD_EINVAL;
    cudaError_t e = launch_set_clock(c, 0.0, 0, dt, 1);
    if (e == cudaSuccess) e = launch_transport(c);
    if (e == cudaSuccess) e = launch_advance_clock(c, 0);
    if (e == cudaSuccess) {
        c->step_host += 1;
        c->cells_valid = false;
    }
    return cuda_code(e);
}

int mcd_step(mcd_ctx *c, double dt)
{
    if (!c || !isfinite(dt)) return MCD_EINVAL;
    const int32_t adaptive = dt > 0.0 ? 0 : 1;  // dt <= 0: chosen on the device after the regrid
    if (adaptive != c->graph_adaptive) {
        drop_graphs(c);
        c->graph_adaptive = adaptive;
    }
    cudaError_t e = tune_collide(c);  // (the first collide's timed trial, before any capture)
    if (e == cudaSuccess && !adaptive) e = launch_set_clock(c, 0.0, 0, dt, 1);
    if (e != cudaSuccess) return MCD_ECUDA;
    if (c->use_graph) {
        int p = c->cur;
        if (!c->gexec[p]) {
            // capture on a private stream (capture is illegal on the legacy
            // default stream); the graph is then launched on the caller's stream
            if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
                return MCD_ECUDA;
            cudaGraph_t gr = nullptr;
            const int64_t l0 = c->launches;
            cudaStream_t user = c->stream;
            c->stream = c->cap_stream;
            e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                c->stream = user;
                return MCD_ECUDA;
            }
            cudaError_t eb = enqueue_step_body(c);
            e = cudaStreamEndCapture(c->stream, &gr);
            c->stream = user;
            c->cur = p;  // the capture only recorded; the state did not change
            c->graph_launches[p] = c->launches - l0;
            c->launches = l0;
            if (eb != cudaSuccess || e != cudaSuccess) {
                if (gr) cudaGraphDestroy(gr);
                return MCD_ECUDA;
            }
            e = cudaGraphInstantiate(&c->gexec[p], gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) {
                c->gexec[p] = nullptr;
                return MCD_ECUDA;
            }
        }
        e = cudaGraphLaunch(c->gexec[p], c->stream);
        if (e != cudaSuccess) return MCD_ECUDA;
        c->launches += c->graph_launches[p];
        c->cur = p ^ 1;
    } else {
        e = enqueue_step_body(c);
        if (e != cudaSuccess) return MCD_ECUDA;
    }
    if (adaptive)
        c->t_known = false;
    else
        c->t_host += dt;
    c->step_host += 1;
    c->cells_valid = false;
    return MCD_OK;
}

int mcd_get_particles(mcd_ctx *c, int32_t disk, double *m, double *M, double *r, double *z, uint32_t *id,
                      int64_t *count, int32_t where)
{
    if (!c || disk < 0 || disk >= c->n_disks || (where != MCD_HOST && where != MCD_DEVICE)) return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    const int b = c->cur;
    cudaMemcpyKind kind = where == MCD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t n) {
        if (dst && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n, kind, c->stream);
    };
    cp(m, c->m[b] + D.p_off, 8 * D.n0);
    cp(M, c->M[b] + D.p_off, 8 * D.n0);
    cp(r, c->r[b] + D.p_off, 8 * D.n0);
    cp(z, c->z[b] + D.p_off, 8 * D.n0);
    cp(id, c->id[b] + D.p_off, 4 * D.n0);
    if (count) *count = D.n0;
    if (e == cudaSuccess && where == MCD_HOST) e = cudaStreamSynchronize(c->stream);
    return cuda_code(e);
}

int mcd_moments(mcd_ctx *c, int32_t disk, int32_t nbins, const double *edges, double *out)
{
    if (!c || disk < 0 || disk >= c->n_disks || nbins <= 0 || nbins > MCD_MAX_BINS || !edges || !out)
        return MCD_EINVAL;
    for (int32_t b = 0; b <= nbins; ++b)
        if (edges[b] != edges[b] || (b > 0 && edges[b] < edges[b - 1])) return MCD_EINVAL;  // NaN or descending
    cudaError_t e = cudaMemcpyAsync(c->diag_edges, edges, sizeof(double) * (nbins + 1), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = launch_moments(c, disk, nbins);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, c->diag_out, sizeof(double) * 5 * nbins, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_code(e);
}

int mcd_get_tracer(mcd_ctx *c, int32_t disk, double *q, int32_t where)
{
    if (!c || disk < 0 || disk >= c->n_disks || !q || (where != MCD_HOST && where != MCD_DEVICE)) return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    cudaError_t e = cudaMemcpyAsync(q, c->q[c->cur] + D.p_off, 8 * D.n0,
                                    where == MCD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && where == MCD_HOST) e = cudaStreamSynchronize(c->stream);
    return cuda_code(e);
}

int mcd_set_tracer(mcd_ctx *c, int32_t disk, const double *q, int32_t where)
{
    if (!c || disk < 0 || disk >= c->n_disks || !q || (where != MCD_HOST && where != MCD_DEVICE)) return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    cudaError_t e = cudaMemcpyAsync(c->q[c->cur] + D.p_off, q, 8 * D.n0,
                                    where == MCD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && where == MCD_HOST) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return MCD_ECUDA;
    if (!c->tracer) {
        c->tracer = 1;
        drop_graphs(c);
    }
    return MCD_OK;
}

int mcd_set_gas_table(mcd_ctx *c, int32_t disk, int32_t n, const double *r, const double *Sigma, const double *T)
{
    if (!c || disk < 0 || disk >= c->n_disks || n < 0 || n == 1 || n > kMaxGasKnots) return MCD_EINVAL;
    if (n > 0 && (!r || !Sigma || !T)) return MCD_EINVAL;
    std::vector<GasKnot> k((size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        if (!(r[i] > 0.0 && r[i] < INFINITY) || !(Sigma[i] > 0.0 && Sigma[i] < INFINITY) ||
            !(T[i] > 0.0 && T[i] < INFINITY) || (i > 0 && !(r[i] > r[i - 1])))
            return MCD_EINVAL;
        k[i].r = r[i];
        k[i].S = Sigma[i];
        k[i].T = T[i];
        k[i].lnr = log(r[i]);
        k[i].lnS = log(Sigma[i]);
        k[i].lnT = log(T[i]);
    }
    // slopes of segment [r_i, r_i+1): -d ln Sigma / d ln r, -d ln T / d ln r
    for (int32_t i = 0; i + 1 < n; ++i) {
        const double dl = k[i + 1].lnr - k[i].lnr;
        k[i].p = -(k[i + 1].lnS - k[i].lnS) / dl;
        k[i].q = -(k[i + 1].lnT - k[i].lnT) / dl;
    }
    if (n > 0) {
        k[n - 1].p = k[n - 2].p;
        k[n - 1].q = k[n - 2].q;
    }
    cudaError_t e = cudaSuccess;
    if (n > 0)
        e = cudaMemcpyAsync(c->gas_knots + (int64_t)disk * kMaxGasKnots, k.data(), sizeof(GasKnot) * n,
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->gas_n + disk, &n, 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_code(e);
    // transport has a variant that reads no table: a captured step graph is
    // rebuilt when the first table comes or the last one goes
    const int32_t before = c->gas_tables;
    c->gas_n_host[disk] = n;
    c->gas_tables = 0;
    for (int32_t k : c->gas_n_host) c->gas_tables += k > 0;
    if ((before > 0) != (c->gas_tables > 0)) drop_graphs(c);
    return MCD_OK;
}

int mcd_sigma_map(mcd_ctx *c, int32_t disk, int32_t nr, const double *r_edges, int32_t nm, const double *m_edges,
                  double *out)
{
    if (!c || disk < 0 || disk >= c->n_disks || nr <= 0 || nm <= 0 || nr > MCD_MAX_MAP_EDGES ||
        nm > MCD_MAX_MAP_EDGES || (int64_t)nr * nm > MCD_MAX_MAP_BINS || !r_edges || !m_edges || !out)
        return MCD_EINVAL;
    for (int32_t b = 0; b <= nr; ++b)
        if (r_edges[b] != r_edges[b] || (b > 0 && r_edges[b] < r_edges[b - 1])) return MCD_EINVAL;
    for (int32_t q = 0; q <= nm; ++q)
        if (m_edges[q] != m_edges[q] || (q > 0 && m_edges[q] < m_edges[q - 1])) return MCD_EINVAL;
    cudaError_t e = cudaMemcpyAsync(c->map_redges, r_edges, sizeof(double) * (nr + 1), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->map_medges, m_edges, sizeof(double) * (nm + 1), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_sigma_map(c, disk, nr, nm);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, c->map_out, sizeof(double) * nr * nm, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_code(e);
}

namespace {

// Staged replacement of one disk's particles: the new columns sit in the
// disk's range of the inactive state buffer (free between steps), the ids are
// counted there (each must occur exactly once and be below n0), and only a
// clean count lets the columns into the live buffer.
__global__ void k_ids_count(const uint32_t *id, int64_t n, uint32_t *cnt, int32_t *bad)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint32_t v = id[k];
    if ((int64_t)v >= n)
        atomicOr(bad, 1);
    else
        atomicAdd(&cnt[v], 1u);
}

__global__ void k_ids_verify(const uint32_t *cnt, int64_t n, int32_t *bad)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n && cnt[k] != 1u) atomicOr(bad, 1);
}

__global__ void k_ids_commit(const int32_t *bad, int64_t n, const double *m, const double *M, const double *r,
                             const double *z, const uint32_t *id, double *m1, double *M1, double *r1, double *z1,
                             uint32_t *id1, int32_t *status)
{
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (*bad) {
        if (k == 0 && status) atomicOr(status, kStBadCell);
        return;
    }
    if (k >= n) return;
    m1[k] = m[k];
    M1[k] = M[k];
    r1[k] = r[k];
    z1[k] = z[k];
    id1[k] = id[k];
}

}  // namespace

int mcd_set_particles(mcd_ctx *c, int32_t disk, const double *m, const double *M, const double *r, const double *z,
                      const uint32_t *id, int64_t count, int32_t where)
{
    if (!c || disk < 0 || disk >= c->n_disks || (where != MCD_HOST && where != MCD_DEVICE)) return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    if (count != D.n0 || !m || !M || !r || !z || !id) return MCD_EINVAL;
    const int b = c->cur, sb = 1 - c->cur;  // live buffer, staging buffer
    const int64_t o = D.p_off, n = D.n0;
    cudaMemcpyKind kind = where == MCD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, kind, c->stream);
    };
    cp(c->m[sb] + o, m, 8 * n);
    cp(c->M[sb] + o, M, 8 * n);
    cp(c->r[sb] + o, r, 8 * n);
    cp(c->z[sb] + o, z, 8 * n);
    cp(c->id[sb] + o, id, 4 * n);
    // the id counts go to the sort's value buffer, the check's result to its histogram
    // (both free between regrids)
    uint32_t *cnt = c->val[1] + o;
    int32_t *bad = reinterpret_cast<int32_t *>(c->hist);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4 * n, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 4, c->stream);
    const unsigned g = (unsigned)((n + 255) / 256);
    if (e == cudaSuccess && n > 0) {
        k_ids_count<<<g, 256, 0, c->stream>>>(c->id[sb] + o, n, cnt, bad);
        k_ids_verify<<<g, 256, 0, c->stream>>>(cnt, n, bad);
        k_ids_commit<<<g, 256, 0, c->stream>>>(bad, n, c->m[sb] + o, c->M[sb] + o, c->r[sb] + o, c->z[sb] + o,
                                               c->id[sb] + o, c->m[b] + o, c->M[b] + o, c->r[b] + o, c->z[b] + o,
                                               c->id[b] + o, where == MCD_DEVICE ? c->status : nullptr);
        c->launches += 3;
        e = cudaGetLastError();
    }
    c->cells_valid = false;
    if (e != cudaSuccess) return MCD_ECUDA;
    if (where == MCD_HOST) {
        // host arrays: the caller may reuse them on return, and learns of bad ids now
        int32_t hb = 0;
        e = cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return MCD_ECUDA;
        if (hb) return MCD_EINVAL;  // the live state is untouched
    }
    return MCD_OK;
}

int mcd_get_cells(mcd_ctx *c, int32_t disk, int64_t *cell_off, double *bounds, double *V, int32_t where)
{
    if (!c || disk < 0 || disk >= c->n_disks || where != MCD_HOST) return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    int64_t nc = (int64_t)D.n_r * D.n_z;
    std::vector<int64_t> start(nc);
    std::vector<int32_t> n(nc);
    cudaError_t e = cudaMemcpyAsync(start.data(), c->cell_start + D.c_off, 8 * nc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(n.data(), c->cell_n + D.c_off, 4 * nc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && bounds)
        e = cudaMemcpyAsync(bounds, c->cell_b + 6 * D.c_off, 48 * nc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && V) e = cudaMemcpyAsync(V, c->cell_V + D.c_off, 8 * nc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return MCD_ECUDA;
    if (cell_off) {
        for (int64_t k = 0; k < nc; ++k) cell_off[k] = start[k] - D.p_off;
        cell_off[nc] = nc ? cell_off[nc - 1] + n[nc - 1] : 0;
    }
    return MCD_OK;
}

int mcd_get_rates(mcd_ctx *c, int32_t disk, double *R, int32_t where)
{
    if (!c || disk < 0 || disk >= c->n_disks || !R || (where != MCD_HOST && where != MCD_DEVICE)) return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    cudaError_t e = cudaMemcpyAsync(R, c->Rdump + D.p_off, 8 * D.n0,
                                    where == MCD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && where == MCD_HOST) e = cudaStreamSynchronize(c->stream);
    return cuda_code(e);
}

int mcd_get_total_rates(mcd_ctx *c, int32_t disk, double *Rtot, int32_t where)
{
    if (!c || !Rtot || disk < 0 || disk >= c->n_disks || (where != MCD_HOST && where != MCD_DEVICE))
        return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    cudaError_t e = cudaMemcpyAsync(Rtot, c->Rtot + D.c_off, 8 * (size_t)D.n_r * D.n_z,
                                    where == MCD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && where == MCD_HOST) e = cudaStreamSynchronize(c->stream);
    return cuda_code(e);
}

int mcd_get_collide_classes(mcd_ctx *c, mcd_collide_class *out, int32_t cap, int32_t *count)
{
    if (!c || !count || (cap > 0 && !out)) return MCD_EINVAL;
    *count = (int32_t)c->cls.size();
    for (int32_t q = 0; q < cap && q < (int32_t)c->cls.size(); ++q) {
        const CollideClass &k = c->cls[q];
        mcd_collide_class &o = out[q];
        memset(&o, 0, sizeof o);
        o.n_lo = k.n_lo;
        o.n_hi = k.n_hi;
        o.cells = k.cells;
        collide_shape(c, q, &o.swarms_per_thread, &o.store, &o.threads, &o.control_warp);
        o.persistent = c->persistent;
        o.tuned = k.tuned;
        o.n_trials = k.n_trials;
        for (int t = 0; t < k.n_trials && t < MCD_MAX_TRIALS; ++t) {
            o.trial_swarms[t] = k.trial_S[t];
            o.trial_store[t] = k.trial_store[t];
            o.trial_control_warp[t] = k.trial_ws[t];
            o.trial_us_per_event[t] = k.trial_us[t];
        }
    }
    return MCD_OK;
}

int mcd_get_cell_events(mcd_ctx *c, int32_t disk, int64_t *events, int32_t where)
{
    if (!c || disk < 0 || disk >= c->n_disks || !events || (where != MCD_HOST && where != MCD_DEVICE))
        return MCD_EINVAL;
    const DiskDev &D = c->hd[disk];
    cudaError_t e = cudaMemcpyAsync(events, c->cell_events + D.c_off, 8 * (int64_t)D.n_r * D.n_z,
                                    where == MCD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && where == MCD_HOST) e = cudaStreamSynchronize(c->stream);
    return cuda_code(e);
}

int mcd_get_event_log(mcd_ctx *c, int32_t *ijo, double *t, double *m_new, int64_t cap, int64_t *n)
{
    if (!c || !n || cap < 0) return MCD_EINVAL;
    unsigned long long ln = 0;
    cudaError_t e = cudaMemcpyAsync(&ln, c->log_n, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return MCD_ECUDA;
    int64_t k = (int64_t)ln < cap ? (int64_t)ln : cap;
    if (k > 0) {
        if (ijo) e = cudaMemcpyAsync(ijo, c->log_ijo, 12 * k, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && t) e = cudaMemcpyAsync(t, c->log_t, 8 * k, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && m_new) e = cudaMemcpyAsync(m_new, c->log_m, 8 * k, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    *n = (int64_t)ln;
    return cuda_code(e);
}

int mcd_get_stats(mcd_ctx *c, int32_t disk, mcd_stats *out)
{
    if (!c || !out || disk < 0 || disk >= c->n_disks) return MCD_EINVAL;
    int64_t na = 0;
    double acc = 0.0;
    unsigned long long ev = 0;
    int32_t st = 0;
    StepState s;
    cudaError_t e = cudaMemcpyAsync(&na, c->n_alive + disk, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&acc, c->accreted + disk, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ev, c->events_total + disk, 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&st, c->status, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&s, c->state, sizeof s, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return MCD_ECUDA;
    out->t = s.t;
    out->step = s.step;
    out->events = (int64_t)ev;
    out->n_alive = na;
    out->accreted_mass = acc;
    out->status = status_code(st);
    out->reserved = 0;
    return MCD_OK;
}

int mcd_set_option(mcd_ctx *c, int32_t key, double v)
{
    if (!c) return MCD_EINVAL;
    switch (key) {
    case MCD_OPT_MAX_EVENTS:
        if (!(v >= 0)) return MCD_EINVAL;
        c->max_events = (int64_t)v;
        break;
    case MCD_OPT_CAP_STOPS: c->cap_stops = v != 0.0; break;
    case MCD_OPT_REBUILD_EVERY:
        if (!(v >= 0)) return MCD_EINVAL;
        c->rebuild_every = (int64_t)v;
        break;
    case MCD_OPT_USE_GRAPH: c->use_graph = v != 0.0; break;
    case MCD_OPT_DUMP_R: c->dump_R = v != 0.0; break;
    case MCD_OPT_LOG_CELL: c->log_cell = (int64_t)v; break;
    case MCD_OPT_LPT: c->lpt = v != 0.0; break;
    case MCD_OPT_EXCLUSIVE: c->exclusive = v != 0.0; break;
    case MCD_OPT_TRACER:
        if (c->tracer && v == 0.0) {  // switched off: the column is cleared, not left stale
            for (int b = 0; b < 2; ++b)
                if (cudaMemsetAsync(c->q[b], 0, 8 * c->N, c->stream) != cudaSuccess) return MCD_ECUDA;
        }
        c->tracer = v != 0.0;
        break;
    case MCD_OPT_DV_MATRIX:
        if (!(v == -1.0 || v == 0.0 || v == 1.0 || v == 2.0)) return MCD_EINVAL;
        c->dv_matrix = (int32_t)v;
        break;
    case MCD_OPT_SWARMS_PER_THREAD:
        if (!(v == 0.0 || v == 1.0 || (v == 2.0 && c->prec == MCD_MIXED))) return MCD_EINVAL;
        c->spt = (int32_t)v;
        break;
    case MCD_OPT_PERSISTENT: c->persistent = v != 0.0; break;
    case MCD_OPT_CONTROL_WARP:
        if (!(v == -1.0 || v == 0.0 || (v == 1.0 && c->prec == MCD_MIXED))) return MCD_EINVAL;
        c->control_warp = (int32_t)v;
        break;
    case MCD_OPT_EXACT_TOTAL: c->exact_total = v != 0.0; break;
    case MCD_OPT_AUTOTUNE:
        c->autotune = v != 0.0;
        if (c->autotune) c->tuned = false;  // the next collide runs the trial again
        break;
    case MCD_OPT_DT_MAX:
        if (!(v > 0.0) || !isfinite(v)) return MCD_EINVAL;
        c->dt_max = v;
        break;
    case MCD_OPT_COURANT:
        if (!(v > 0.0) || !isfinite(v)) return MCD_EINVAL;
        c->courant = v;
        break;
    case MCD_OPT_THREADS:  // (MCD_MIXED with MCD_OPT_EXACT_TOTAL adds one helper warp to these)
        if (v != 0.0 && (v < c->n_max || v > kMaxCell || ((int)v % 32) != 0)) return MCD_EINVAL;
        c->threads = (int32_t)v;
        break;
    default: return MCD_EINVAL;
    }
    drop_graphs(c);
    return MCD_OK;
}

int mcd_trace(mcd_ctx *c, int32_t on)
{
    if (!c) return MCD_EINVAL;
    if (on && !c->tev[0])
        for (int k = 0; k < 5; ++k)
            if (cudaEventCreate(&c->tev[k]) != cudaSuccess) return MCD_ECUDA;
    c->trace = on ? 1 : 0;
    drop_graphs(c);
    return MCD_OK;
}

int mcd_trace_read(mcd_ctx *c, float *ms)
{
    if (!c || !ms || !c->tev[0]) return MCD_EINVAL;
    if (cudaEventSynchronize(c->tev[4]) != cudaSuccess) return MCD_ECUDA;
    for (int k = 0; k < 4; ++k)
        if (cudaEventElapsedTime(&ms[k], c->tev[k], c->tev[k + 1]) != cudaSuccess) return MCD_ECUDA;
    return MCD_OK;
}

int mcd_get_launch_count(mcd_ctx *c, int64_t *launches)
{
    if (!c || !launches) return MCD_EINVAL;
    *launches = c->launches;
    return MCD_OK;
}

namespace {
// the resumed clock, step counter and a disk's counters, passed by value
__global__ void k_restore_clock(mcd::StepState *st, double t, int64_t step)
{
    st->t = t;
    st->step = step;
}
__global__ void k_restore_counters(unsigned long long *events, double *accreted, unsigned long long ev, double acc)
{
    *events = ev;
    *accreted = acc;
}
}  // namespace

int mcd_set_clock(mcd_ctx *c, double t, int64_t step)
{
    if (!c || !isfinite(t) || t < 0.0 || step < 0) return MCD_EINVAL;
    k_restore_clock<<<1, 1, 0, c->stream>>>(c->state, t, step);
    c->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return MCD_ECUDA;
    c->t_host = t;
    c->t_known = true;
    c->step_host = step;
    return MCD_OK;
}

int mcd_set_counters(mcd_ctx *c, int32_t disk, int64_t events, double accreted_mass)
{
    if (!c || disk < 0 || disk >= c->n_disks || events < 0 || !isfinite(accreted_mass) || accreted_mass < 0.0)
        return MCD_EINVAL;
    k_restore_counters<<<1, 1, 0, c->stream>>>(c->events_total + disk, c->accreted + disk,
                                                (unsigned long long)events, accreted_mass);
    c->launches += 1;
    return cudaGetLastError() == cudaSuccess ? MCD_OK : MCD_ECUDA;
}

int mcd_sync(mcd_ctx *c)
{
    if (!c) return MCD_EINVAL;
    int32_t st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, c->status, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return MCD_ECUDA;
    return status_code(st);
}

int mcd_free(mcd_ctx *c)
{
    if (!c) return MCD_EINVAL;
    cudaStreamSynchronize(c->stream);
    destroy(c);
    return MCD_OK;
}

const char *mcd_strerror(int code)
{
    switch (code) {
    case MCD_OK: return "ok";
    case MCD_EINVAL: return "invalid argument";
    case MCD_ENOMEM: return "workspace too small";
    case MCD_ECUDA: return "CUDA runtime error";
    case MCD_ENAN: return "NaN in particle positions";
    case MCD_ETIMEOUT: return "a cell reached the event cap";
    case MCD_EEMPTY: return "every particle of a disk was removed";
    case MCD_ESTATE: return "call out of order";
    default: return "unknown status";
    }
}

int mcd_pair_probe(const mcd_disk_params *p, int32_t prec, double rc, double zc, int64_t n, const double *mi,
                   const double *mj, double *dv, double *K, void *stream)
{
    if (!p || n < 0 || (n > 0 && (!mi || !mj || !dv || !K)) || (prec != MCD_FP64 && prec != MCD_MIXED))
        return MCD_EINVAL;
    return cuda_code(launch_pair_probe(*p, prec, rc, zc, n, mi, mj, dv, K, (cudaStream_t)stream));
}

int mcd_rate_probe(const mcd_disk_params *p, int32_t prec, double rc, double zc, double V, int32_t n,
                   const double *m, const double *M, double *rate, double *R, void *stream)
{
    if (!p || n < 0 || n > 1024 || (n > 0 && (!m || !M || !rate || !R)) || (prec != MCD_FP64 && prec != MCD_MIXED))
        return MCD_EINVAL;
    return cuda_code(launch_rate_probe(*p, prec, rc, zc, V, n, m, M, rate, R, (cudaStream_t)stream));
}

}  // extern "C"
