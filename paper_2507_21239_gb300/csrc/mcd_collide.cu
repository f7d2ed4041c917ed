// mcd_collide.cu -- host side of the collision step: the per-cell constants,
// the largest-work-first queue, the cell classes and their launches, the
// timed trial that picks each class's variant, and the probes.  The kernels
// themselves are in mcd_collide.cuh, instantiated per (precision, swarms per
// thread, exact total) in mcd_collide_f32s1.cu, mcd_collide_f32s2.cu,
// mcd_collide_f32s1x.cu, mcd_collide_f32s2x.cu and mcd_collide_f64.cu, and the
// control-warp variants in mcd_collide_ws.cuh (mcd_collide_f32ws4.cu,
// mcd_collide_f32ws10.cu).
#include <algorithm>

#include "mcd_collide_ws.cuh"

namespace mcd {

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
// cell index).  Cells go into 64 log2 bins per class, heaviest first, classes
// in order: each class's cells then take one contiguous part of the queue in
// largest-work-first order; CTAs start in block order, so the long event
// chains begin early.
constexpr int kLptBins = 64;

__global__ void k_lpt_bin(int64_t C, const int32_t *cell_n, const int64_t *cell_events, const int32_t *cell_class,
                          uint32_t *bin, int32_t *qcount)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= C) return;
    double n = (double)cell_n[c];
    double w = n * n + 2.0 * n * (double)cell_events[c] + 1.0;
    int b = cell_class[c] * kLptBins + (kLptBins - 1 - min(kLptBins - 1, ilogb(w)));
    bin[c] = (uint32_t)b;
    atomicAdd(&qcount[b], 1);
}

__global__ void k_lpt_scan(int32_t *qcount, int nbins)
{
    int32_t run = 0;
    for (int b = 0; b < nbins; ++b) {
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
    const int nbins = (int)c->cls.size() * kLptBins;
    cudaError_t e = cudaMemsetAsync(c->qcount, 0, nbins * sizeof(int32_t), c->stream);
    if (e != cudaSuccess) return e;
    unsigned g = (unsigned)((c->C + 255) / 256);
    k_lpt_bin<<<g, 256, 0, c->stream>>>(c->C, c->cell_n, c->cell_events, c->cell_class, c->cell_cost, c->qcount);
    k_lpt_scan<<<1, 1, 0, c->stream>>>(c->qcount, nbins);
    k_lpt_place<<<g, 256, 0, c->stream>>>(c->C, c->cell_cost, c->qcount, c->queue);
    c->launches += 3;
    return cudaGetLastError();
}

// ---- cell classes ----------------------------------------------------------------------
// GB300: up to 227 KB of shared memory per CTA (opt-in); a few KB are kept for
// the kernel's static shared memory
constexpr size_t kSmemOptinMax = 232448;
constexpr size_t kStaticReserve = 4096;
constexpr size_t kExclusiveSmem = 120 * 1024;  // > half of an SM's shared memory
// workspace budgets for the stored matrices
constexpr size_t kFp64MatrixCap = (size_t)8 << 30;
constexpr size_t kFp32MatrixCap = (size_t)16 << 30;

static int round32(int x) { return ((x + 31) / 32) * 32; }

static int class_threads(int n_hi, int S) { return std::max(32, round32((n_hi + S - 1) / S)); }

// threads of a collide CTA: the swarms' threads, plus (FP32 with the exact
// total) the helper warp that sums the compensated total rate
template <class T>
static int block_threads(int swarm_threads, bool exact)
{
    return swarm_threads + (sizeof(T) == 4 && exact ? 32 : 0);
}

// the FP32 shared-memory matrix of cells of up to n swarms fits one CTA (with
// the tracer's copy, which may be switched on after the plan; the exact
// total's helper warp and posted sums may push it out, and the launch then
// falls back to the next store)
static bool smem_matrix_fits(int n)
{
    for (int S = 1; S <= 2; ++S)
        if (collide_smem_bytes<float>(class_threads(n, S), S, true, 1, n, sym_width(n), false) + kStaticReserve >
            kSmemOptinMax)
            return false;
    return true;
}

size_t class_matrix_bytes(const CollideClass &k, int32_t prec)
{
    return (size_t)k.cells * k.rows * k.W * (prec == MCD_FP64 ? sizeof(double) : sizeof(float));
}

int plan_classes(const mcd_grid *g, int32_t nd, int32_t prec, std::vector<CollideClass> &cls,
                 std::vector<int32_t> &disk_class)
{
    // class bounds: 64, 128, 224, the largest cell whose FP32 matrix fits in
    // shared memory, kMaxCell
    int nfit = 224;
    while (nfit < kMaxCell && smem_matrix_fits(nfit + 1)) ++nfit;
    const int bounds[kMaxClasses] = {64, 128, 224, nfit, kMaxCell};
    CollideClass all[kMaxClasses];
    std::vector<int32_t> raw(nd);
    for (int32_t d = 0; d < nd; ++d) {
        int b = 0;
        while (b < kMaxClasses - 1 && g[d].per_cell > bounds[b]) ++b;
        raw[d] = b;
        CollideClass &k = all[b];
        k.n_lo = k.cells ? std::min(k.n_lo, g[d].per_cell) : g[d].per_cell;
        k.n_hi = std::max(k.n_hi, g[d].per_cell);
        k.cells += (int64_t)g[d].n_r * g[d].n_z;
    }
    cls.clear();
    int map[kMaxClasses];
    for (int b = 0; b < kMaxClasses; ++b) {
        map[b] = -1;
        if (all[b].cells == 0) continue;
        CollideClass k = all[b];
        k.qoff = cls.empty() ? 0 : cls.back().qoff + cls.back().cells;
        k.rows = k.n_hi;
        k.W = sym_width(k.n_hi);
        k.smem_fits = prec == MCD_MIXED && smem_matrix_fits(k.n_hi);
        map[b] = (int)cls.size();
        cls.push_back(k);
    }
    disk_class.assign(nd, 0);
    for (int32_t d = 0; d < nd; ++d) disk_class[d] = map[raw[d]];
    // workspace matrices: FP64 for every class, FP32 for the classes whose
    // matrix does not fit in shared memory, within the budgets (all or none)
    size_t total = 0;
    for (const CollideClass &k : cls)
        if (prec == MCD_FP64 || !k.smem_fits) total += class_matrix_bytes(k, prec);
    const bool reserve = total <= (prec == MCD_FP64 ? kFp64MatrixCap : kFp32MatrixCap);
    for (CollideClass &k : cls) {
        k.reserve = reserve && (prec == MCD_FP64 || !k.smem_fits);
        k.dvg = nullptr;
    }
    return MCD_OK;
}

// ---- launches ------------------------------------------------------------------------
template <class T>
static cudaError_t variant(int op, int S, int store, bool ramp, bool tracer, bool exact, unsigned grid, int nthr,
                           size_t smem, cudaStream_t st, const CollideArgs *A, int *out)
{
    if constexpr (sizeof(T) == 8) {
        if (S != 1 || store == 1 || exact) return cudaErrorInvalidValue;
        return collide_variant<double, 1, false>(op, store, ramp, tracer, grid, nthr, smem, st, A, out);
    } else {
        if (exact)
            return S == 2 ? collide_variant<float, 2, true>(op, store, ramp, tracer, grid, nthr, smem, st, A, out)
                          : collide_variant<float, 1, true>(op, store, ramp, tracer, grid, nthr, smem, st, A, out);
        return S == 2 ? collide_variant<float, 2, false>(op, store, ramp, tracer, grid, nthr, smem, st, A, out)
                      : collide_variant<float, 1, false>(op, store, ramp, tracer, grid, nthr, smem, st, A, out);
    }
}

// the control-warp variants: swarms per control lane for cells of up to n
// swarms (0: none fits)
static int ws_pl(int n)
{
    for (int pl : {4, 7, 10, 16})
        if (32 * pl >= n) return pl;
    return 0;
}

static cudaError_t ws_variant(int op, int pl, int store, bool ramp, bool tracer, unsigned grid, int nthr, size_t smem,
                              cudaStream_t st, const CollideArgs *A, int *out)
{
    switch (pl) {
    case 4: return collide_ws_variant<4>(op, store, ramp, tracer, grid, nthr, smem, st, A, out);
    case 7: return collide_ws_variant<7>(op, store, ramp, tracer, grid, nthr, smem, st, A, out);
    case 10: return collide_ws_variant<10>(op, store, ramp, tracer, grid, nthr, smem, st, A, out);
    case 16: return collide_ws_variant<16>(op, store, ramp, tracer, grid, nthr, smem, st, A, out);
    default: return cudaErrorInvalidValue;
    }
}

// the store a class can use: 1 needs the FP32 shared matrix to fit, 2 a
// reserved workspace matrix; otherwise recompute
template <class T>
static int usable_store(const CollideClass &k, int want)
{
    if (want == 1 && sizeof(T) == 4 && k.smem_fits) return 1;
    if (want == 1 || want == 2) return k.dvg ? 2 : 0;
    return 0;
}

struct ClassLaunch {
    int S, store, nthr;
    size_t smem;
    int ws, pl;  // the control-warp variant and its swarms per control lane
};

// whether class k runs the control-warp variant: MCD_MIXED without the exact
// total or a thread count, forced by the option (cw 0 or 1), else the class's
// choice unless swarms per thread are set
template <class T>
static bool class_ws(const CollideClass &k, int threads, int spt, int cw, int exact)
{
    if (sizeof(T) == 8 || threads || exact || !ws_pl(k.n_hi)) return false;
    if (cw >= 0) return cw == 1;
    return !spt && k.ws;
}

// the launch shape of class k: the options' swarms per thread and store when
// set (spt, dv_matrix >= 0), else the class's chosen ones
template <class T>
static ClassLaunch class_launch(const CollideClass &k, int threads, int spt, int dv_matrix, int exclusive, int tracer,
                                int exact, int smem_optin, int ws)
{
    ClassLaunch L;
    L.ws = ws;
    L.pl = ws ? ws_pl(k.n_hi) : 0;
    if (ws) {
        L.S = 1;
        L.store = usable_store<T>(k, dv_matrix >= 0 ? dv_matrix : k.store);
        L.nthr = 32 + round32(k.n_hi);
        L.smem = collide_ws_smem_bytes(L.pl, tracer != 0, L.store, k.rows, k.W);
        if (L.store == 1 && L.smem > (size_t)smem_optin) {
            L.store = usable_store<T>(k, 2);
            L.smem = collide_ws_smem_bytes(L.pl, tracer != 0, L.store, k.rows, k.W);
        }
        if (exclusive && k.n_hi > 64 && L.smem < kExclusiveSmem) L.smem = kExclusiveSmem;
        return L;
    }
    L.S = (sizeof(T) == 8 || threads) ? 1 : (spt ? spt : k.S);
    // (FP32: one swarm per thread leaves no room for the helper warp above 480 swarms)
    if (sizeof(T) == 4 && !threads && block_threads<T>(class_threads(k.n_hi, 1), exact) > kMaxCell) L.S = 2;
    L.store = usable_store<T>(k, dv_matrix >= 0 ? dv_matrix : k.store);
    L.nthr = block_threads<T>(threads ? threads : class_threads(k.n_hi, L.S), exact);
    L.smem = collide_smem_bytes<T>(L.nthr, L.S, tracer != 0, L.store, k.rows, k.W, exact);
    if (L.store == 1 && L.smem > (size_t)smem_optin) {  // (the shared matrix no longer fits)
        L.store = usable_store<T>(k, 2);
        L.smem = collide_smem_bytes<T>(L.nthr, L.S, tracer != 0, L.store, k.rows, k.W, exact);
    }
    // exclusive: request more than half an SM's shared memory so that no two
    // collide CTAs of classes that can carry long chains share an SM (the
    // heaviest cells, launched first, run alone)
    if (exclusive && k.n_hi > 64 && L.smem < kExclusiveSmem) L.smem = kExclusiveSmem;
    return L;
}

template <class T>
static ClassLaunch class_launch(const mcd_ctx *cx, const CollideClass &k)
{
    return class_launch<T>(k, cx->threads, cx->spt, cx->dv_matrix, cx->exclusive, cx->tracer, cx->exact_total,
                           cx->smem_optin, class_ws<T>(k, cx->threads, cx->spt, cx->control_warp, cx->exact_total));
}

void collide_shape(const mcd_ctx *c, int q, int32_t *S, int32_t *store, int32_t *threads, int32_t *control_warp)
{
    const ClassLaunch L = c->prec == MCD_MIXED ? class_launch<float>(c, c->cls[q]) : class_launch<double>(c, c->cls[q]);
    *S = L.S;
    *store = L.store;
    *threads = L.nthr;
    *control_warp = L.ws;
}

// one launch-time operation (variant op codes) of a class launch shape
template <class T>
static cudaError_t launch_op(int op, const ClassLaunch &L, bool ramp, bool tracer, bool exact, unsigned grid,
                             cudaStream_t st, const CollideArgs *A, int *out)
{
    if (L.ws) return ws_variant(op, L.pl, L.store, ramp, tracer, grid, L.nthr, L.smem, st, A, out);
    return variant<T>(op, L.S, L.store, ramp, tracer, exact, grid, L.nthr, L.smem, st, A, out);
}

template <class T>
static void common_args(mcd_ctx *cx, CollideArgs &A, int from_state, double t_end)
{
    const int b = cx->cur;
    A.params = cx->d_params;
    A.disks = cx->d_disks;
    A.cell_disk = cx->cell_disk;
    A.cell_start = cx->cell_start;
    A.cell_n = cx->cell_n;
    A.cellk = cx->cellk;
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
    A.Rtot = cx->dump_R ? cx->Rtot : nullptr;
    A.log_cell = cx->log_cell;
    A.log_ijo = cx->log_ijo;
    A.log_t = cx->log_t;
    A.log_m = cx->log_m;
    A.log_n = cx->log_n;
    A.log_cap = mcd_ctx::kLogCap;
    A.qhead = nullptr;
}

template <class T>
static cudaError_t cellconst(mcd_ctx *cx)
{
    k_cellconst<T><<<(unsigned)((cx->C + 127) / 128), 128, 0, cx->stream>>>(
        cx->d_params, cx->gas_knots, cx->gas_n, cx->cell_disk, cx->cell_start, cx->cell_n, cx->cell_b, cx->cell_V,
        cx->M[cx->cur], cx->cellk, cx->C);
    cx->launches += 1;
    return cudaGetLastError();
}

template <class T>
static cudaError_t collide_impl(mcd_ctx *cx, int from_state, double t_end)
{
    if (cx->C == 0) return cudaSuccess;
    cudaError_t e = cellconst<T>(cx);
    if (e != cudaSuccess) return e;
    CollideArgs A;
    common_args<T>(cx, A, from_state, t_end);
    const int ncls = (int)cx->cls.size();
    const bool exact = sizeof(T) == 4 && cx->exact_total;
    if (ncls > 1 && (e = cudaEventRecord(cx->cls_fork, cx->stream)) != cudaSuccess) return e;
    for (int q = 0; q < ncls && e == cudaSuccess; ++q) {
        const CollideClass &k = cx->cls[q];
        const ClassLaunch L = class_launch<T>(cx, k);
        if (L.ws ? (L.nthr - 32 < k.n_hi || 32 * L.pl < k.n_hi || L.nthr > 32 + 32 * L.pl)
                 : (L.nthr - block_threads<T>(0, cx->exact_total) < (k.n_hi + L.S - 1) / L.S ||
                    L.nthr > kMaxCell / L.S))
            return cudaErrorInvalidValue;
        if (L.smem > (size_t)cx->smem_optin) return cudaErrorInvalidValue;
        cudaStream_t st = q == 0 ? cx->stream : cx->cls_stream[q];
        if (q > 0 && (e = cudaStreamWaitEvent(st, cx->cls_fork, 0)) != cudaSuccess) return e;
        A.queue = (cx->lpt ? cx->queue : cx->queue_static) + k.qoff;
        A.n_queue = k.cells;
        A.dv_w = k.W;
        A.dv_rows = k.rows;
        A.dvg = L.store == 2 ? k.dvg : nullptr;
        unsigned grid = (unsigned)k.cells;
        A.qhead = nullptr;
        if (cx->persistent) {
            int per_sm = 0;
            e = launch_op<T>(3, L, cx->ramp != 0, cx->tracer != 0, exact, 0, st, &A, &per_sm);
            if (e != cudaSuccess) return e;
            const int64_t cap = (int64_t)std::max(per_sm, 1) * cx->n_sm;
            grid = (unsigned)std::min<int64_t>(k.cells, cap);
            A.qhead = cx->qheads + q;
            if ((e = cudaMemsetAsync(A.qhead, 0, sizeof(int32_t), st)) != cudaSuccess) return e;
        }
        e = launch_op<T>(0, L, cx->ramp != 0, cx->tracer != 0, exact, grid, st, &A, nullptr);
        cx->launches += 1;
        if (e == cudaSuccess && q > 0) {
            e = cudaEventRecord(cx->cls_join[q], st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cx->stream, cx->cls_join[q], 0);
        }
    }
    return e;
}

// every variant's dynamic shared-memory limit: what the device lets a block
// opt in to beyond the variant's static part
template <class T>
static cudaError_t prepare_impl(mcd_ctx *c)
{
    cudaError_t e;
    int dev = 0, optin = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    int smin = optin;
    for (int exact = 0; exact <= (sizeof(T) == 4 ? 1 : 0); ++exact)
        for (int S = 1; S <= (sizeof(T) == 4 ? 2 : 1); ++S)
            for (int store = 0; store <= 2; ++store) {
                if (sizeof(T) == 8 && store == 1) continue;
                int st = 0;
                if ((e = variant<T>(2, S, store, false, false, exact, 0, 0, 0, nullptr, nullptr, &st)) != cudaSuccess)
                    return e;
                const int dyn = optin - st;
                if (dyn <= 0) return cudaErrorInvalidValue;
                if ((e = variant<T>(1, S, store, false, false, exact, 0, 0, (size_t)dyn, nullptr, nullptr,
                                    nullptr)) != cudaSuccess)
                    return e;
                smin = std::min(smin, dyn);
            }
    if (sizeof(T) == 4)  // the control-warp variants
        for (int pl : {4, 7, 10, 16})
            for (int store = 0; store <= 2; ++store) {
                int st = 0;
                if ((e = ws_variant(2, pl, store, false, false, 0, 0, 0, nullptr, nullptr, &st)) != cudaSuccess)
                    return e;
                const int dyn = optin - st;
                if (dyn <= 0) return cudaErrorInvalidValue;
                if ((e = ws_variant(1, pl, store, false, false, 0, 0, (size_t)dyn, nullptr, nullptr, nullptr)) !=
                    cudaSuccess)
                    return e;
                smin = std::min(smin, dyn);
            }
    c->smem_optin = smin;
    return cudaSuccess;
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

// ---- the timed trial ---------------------------------------------------------------------
// For every class with more than one candidate (swarms per thread 1 or 2 where
// 2 takes fewer warps, or the control warp; the shared, workspace or no
// matrix), up to 8 of the class's largest cells run kTrialEvents events each
// from the current masses, into scratch copies (the particle and tracer
// buffers the next regrid overwrites, the row-sum dump and a scratch status),
// once to warm up and kTrialRuns times timed with CUDA events; the candidate
// with the smallest median time is kept.  The state of the context does not change.  The options MCD_OPT_SWARMS_PER_THREAD
// and MCD_OPT_DV_MATRIX, when set, take the choice out of the trial.
constexpr int kTrialEvents = 512, kTrialCells = 8, kTrialRuns = 5;

template <class T>
static cudaError_t tune_impl(mcd_ctx *c)
{
    cudaStream_t st = c->stream;
    std::vector<int32_t> n(c->C);
    cudaError_t e = cudaMemcpyAsync(n.data(), c->cell_n, 4 * c->C, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const int b = c->cur;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if ((e = cudaEventCreate(&t0)) != cudaSuccess) return e;
    if ((e = cudaEventCreate(&t1)) != cudaSuccess) {
        cudaEventDestroy(t0);
        return e;
    }
    bool cc_done = false;
    for (size_t q = 0; q < c->cls.size() && e == cudaSuccess; ++q) {
        CollideClass &k = c->cls[q];
        struct Cand {
            int S, store, ws;
        };
        std::vector<Cand> cand;
        // the control-warp variant: when the options leave it open (or ask for it)
        const bool ws_ok = sizeof(T) == 4 && !c->threads && !c->exact_total && ws_pl(k.n_hi) &&
                           (c->control_warp == 1 || (c->control_warp < 0 && !c->spt));
        for (int ws = 0; ws <= 1; ++ws) {
            if (ws ? !ws_ok : c->control_warp == 1 && ws_ok) continue;
            for (int S = 1; S <= (sizeof(T) == 4 && !ws ? 2 : 1); ++S) {
                if (!ws && c->spt && S != c->spt) continue;
                if (!ws && S == 2 && class_threads(k.n_hi, 2) >= class_threads(k.n_hi, 1)) continue;  // no fewer warps
                if (!ws && S == 1 && block_threads<T>(class_threads(k.n_hi, 1), c->exact_total) > kMaxCell) continue;
                for (int store : {1, 2, 0}) {
                    if (c->dv_matrix >= 0 && usable_store<T>(k, c->dv_matrix) != store) continue;
                    if (usable_store<T>(k, store) != store) continue;
                    cand.push_back({S, store, ws});
                }
            }
        }
        if (cand.empty()) continue;
        k.S = cand[0].S;
        k.store = cand[0].store;
        k.ws = cand[0].ws;
        if (cand.size() < 2 || !c->autotune) continue;
        // the class's largest cells
        std::vector<int32_t> pick;
        int nbest = 0;
        for (int64_t x = 0; x < c->C; ++x)
            if (c->cell_class_host[x] == (int32_t)q) nbest = std::max(nbest, n[x]);
        for (int64_t x = 0; x < c->C && (int)pick.size() < kTrialCells; ++x)
            if (c->cell_class_host[x] == (int32_t)q && n[x] == nbest && nbest > 1) pick.push_back((int32_t)x);
        if (pick.empty()) continue;
        if (!cc_done) {
            if ((e = cellconst<T>(c)) != cudaSuccess) break;
            cc_done = true;
        }
        int32_t *tq = reinterpret_cast<int32_t *>(c->cell_cost);
        e = cudaMemcpyAsync(tq, pick.data(), 4 * pick.size(), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        CollideArgs A;
        common_args<T>(c, A, 0, 1e300);
        A.m = c->m[1 - b];
        A.q = c->tracer ? c->q[1 - b] : nullptr;
        A.cell_events = reinterpret_cast<int64_t *>(c->Rdump);
        A.events_total = c->tune_scr;
        A.status = reinterpret_cast<int32_t *>(c->tune_scr + c->n_disks);
        A.Rdump = nullptr;
        A.Rtot = nullptr;
        A.log_cell = -1;
        A.max_events = kTrialEvents;
        A.cap_stops = 1;
        A.queue = tq;
        A.n_queue = (int64_t)pick.size();
        A.dv_w = k.W;
        A.dv_rows = k.rows;
        k.n_trials = 0;
        float best = 3.0e38f;
        for (const auto &cs : cand) {
            const ClassLaunch L = class_launch<T>(k, c->threads, cs.S, cs.store, c->exclusive, c->tracer,
                                                  c->exact_total, c->smem_optin, cs.ws);
            if (L.S != cs.S || L.store != cs.store) continue;  // (the launch would not run this candidate)
            if (L.smem > (size_t)c->smem_optin) continue;
            A.dvg = L.store == 2 ? k.dvg : nullptr;
            float ms[kTrialRuns + 1] = {};
            for (int rep = 0; rep <= kTrialRuns && e == cudaSuccess; ++rep) {
                e = cudaMemcpyAsync(A.m, c->m[b], 8 * c->N, cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess && A.q) e = cudaMemcpyAsync(A.q, c->q[b], 8 * c->N, cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess) e = cudaEventRecord(t0, st);
                if (e == cudaSuccess)
                    e = launch_op<T>(0, L, c->ramp != 0, c->tracer != 0, sizeof(T) == 4 && c->exact_total,
                                     (unsigned)pick.size(), st, &A, nullptr);
                c->launches += 1;
                if (e == cudaSuccess) e = cudaEventRecord(t1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[rep], t0, t1);
            }
            if (e != cudaSuccess) break;
            std::sort(ms + 1, ms + kTrialRuns + 1);
            const float us = 1e3f * ms[1 + kTrialRuns / 2] / kTrialEvents;
            if (k.n_trials < kMaxTrials) {
                k.trial_us[k.n_trials] = us;
                k.trial_S[k.n_trials] = cs.S;
                k.trial_store[k.n_trials] = cs.store;
                k.trial_ws[k.n_trials] = cs.ws;
                ++k.n_trials;
            }
            if (us < best) {
                best = us;
                k.S = cs.S;
                k.store = cs.store;
                k.ws = cs.ws;
            }
        }
        k.tuned = 1;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return e;
}

cudaError_t tune_collide(mcd_ctx *c)
{
    if (c->tuned) return cudaSuccess;
    c->tuned = true;
    return c->prec == MCD_MIXED ? tune_impl<float>(c) : tune_impl<double>(c);
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
