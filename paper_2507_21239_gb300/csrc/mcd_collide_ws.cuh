// mcd_collide_ws.cuh -- the collision chain of one cell with a control warp
// (mixed precision).  Same method as cell_chain in mcd_collide.cuh (Zsom &
// Dullemond's representative-particle scheme, Summary of the mcdust paper):
// waiting time from R_tot, i by R_i, j by r_ij, outcome, row and column i
// renewed.  What differs is the division of labour inside the CTA:
//
//  * warp 0, the control warp, keeps every row sum R_k in registers (lane l
//    owns swarms PL l .. PL l + PL - 1) and makes both choices with warp-wide
//    shuffle scans: no cross-warp scan, no barrier inside a choice;
//  * warps 1.., the workers, own one swarm each (swarm k = thread - 32): they
//    form row and column i before the event and, after it, the new row and
//    column, and post what the control warp needs in shared memory;
//  * control lane 0 applies the outcome once j is known (FP64 masses and
//    clock on one lane, as in the block variant).
//
// Per event there are four hand-overs (block barriers): i chosen -> row i
// formed -> j chosen and the event applied -> new row and column formed.
// The control warp's choice scans sum each lane's PL swarms in order, then
// scan the 32 lane sums (Kogge-Stone); the fresh R_i of the last event's
// swarm is the same per-lane sum of its new row, reduced over the lanes by
// a butterfly (every lane gets the same bits).
#pragma once
#include "mcd_collide.cuh"

namespace mcd {

// shared memory of the control-warp chain: caches, masses, row i, the new
// row, the column updates, the dv row, the tracer copy, the rebuilt row sums;
// plus the stored matrix (STORE == 1)
inline size_t collide_ws_smem_bytes(int PL, bool tracer, int store, int rows, int W)
{
    const size_t slots = (size_t)32 * PL;
    size_t b = slots * (sizeof(Part<float>) + sizeof(double) + 3 * sizeof(float) + sizeof(float2) + sizeof(float2)) +
               (tracer ? slots * sizeof(double) : 0);
    if (store == 1) b += (size_t)rows * W * sizeof(float);
    return b;
}

// warp-wide choice over the PL values each lane holds: the first element
// (in lane-major order, lane l holding elements PL l ..) whose inclusive
// prefix exceeds u * total, where element pend (if >= 0) carries the extra
// value Rp on top of its x (0).  Returns the element in every lane, -1 when
// the target is not bracketed (non-finite sums).  total is written.
template <int PL>
__device__ __forceinline__ int warp_choose(const float (&x)[PL], float u, int pend, float Rp, float &total)
{
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float wi = x[0];
#pragma unroll
    for (int s = 1; s < PL; ++s) wi += x[s];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float a = __shfl_up_sync(FULL, wi, o);
        if (lane >= o) wi += a;
    }
    const float tot = __shfl_sync(FULL, wi, 31) + (pend >= 0 ? Rp : 0.0f);
    total = tot;
    float target = u * tot;
    if (target >= tot) target = tot * (float)(1.0 - 1e-7);
    const int e0 = PL * lane;
    const float P = wi + ((pend >= 0 && e0 + PL - 1 >= pend) ? Rp : 0.0f);
    const unsigned bal = __ballot_sync(FULL, P > target);
    // (lane 31's prefix is the total itself, so it brackets whenever the total does)
    const int l = __ffs(bal | 0x80000000u) - 1;
    float e = __shfl_up_sync(FULL, P, 1);
    if (lane == 0) e = 0.0f;
    int first = -1, last = 0;
#pragma unroll
    for (int s = 0; s < PL; ++s) {
        const float v = x[s] + ((pend >= 0 && e0 + s == pend) ? Rp : 0.0f);
        e += v;
        if (v > 0.0f) {
            last = s;
            if (first < 0 && e > target) first = s;
        }
    }
    const int sub = __shfl_sync(FULL, first >= 0 ? first : last, l);
    return (0.0f <= target && target < tot) ? PL * l + sub : -1;
}

template <int PL, int STORE, bool RAMP, bool TRACER>
__device__ __forceinline__ void cell_chain_ws(const CollideArgs &A, const int64_t cell, const int64_t entry,
                                              Shared<float> &sh, unsigned char *smem_raw)
{
    typedef float T;
    const unsigned FULL = 0xffffffffu;
    constexpr int nslot = 32 * PL;
    Part<T> *parts = reinterpret_cast<Part<T> *>(smem_raw);
    double *msh = reinterpret_cast<double *>(parts + nslot);
    float2 *upd = reinterpret_cast<float2 *>(msh + nslot);  // per swarm: (r_ki new, r_ki old)
    float2 *Rs = upd + nslot;                                // rebuilt row sums (s, c)
    T *rowv = reinterpret_cast<T *>(Rs + nslot);            // row i before the event
    T *rnew = rowv + nslot;                                  // row i after the event
    T *dvrow = rnew + nslot;                                 // dv_ik before the event (STORE != 1)
    double *qsh = reinterpret_cast<double *>(dvrow + nslot); // TRACER
    T *Dm = reinterpret_cast<T *>(TRACER ? reinterpret_cast<unsigned char *>(qsh + nslot)
                                         : reinterpret_cast<unsigned char *>(qsh));  // STORE == 1
    const int W = A.dv_w;
    if constexpr (STORE == 2) Dm = reinterpret_cast<T *>(A.dvg) + (size_t)entry * A.dv_rows * W;
    const int lane = threadIdx.x & 31;
    const bool ctl = threadIdx.x < 32;
    const int k = (int)threadIdx.x - 32;  // a worker's swarm
    const int n = A.cell_n[cell];
    if (n <= 0) {
        if (threadIdx.x == 0) A.cell_events[cell] = 0;
        return;
    }
    if (n > nslot || n > (int)blockDim.x - 32 || (STORE && (n > A.dv_rows || n / 2 >= W))) {
        if (threadIdx.x == 0) atomicOr(A.status, kStBadCell);
        return;
    }
    const bool act = k >= 0 && k < n;
    const int disk = A.cell_disk[cell];
    const int64_t off = A.cell_start[cell];
    if (threadIdx.x == 0) sh.c = *reinterpret_cast<const CellK<T> *>(A.cellk + cell * kCellKBytes);
    __syncthreads();
    const CellK<T> &c = sh.c;
    const PairK<T> pc = pair_consts<T>(sh.c);
    Part<T> pk;
    if (act) {
        const double mk = A.m[off + k];
        if (!mass_splits(mk)) atomicOr(A.status, kStBadCell);
        msh[k] = mk;
        if (TRACER) qsh[k] = A.q[off + k];
        pk = make_part<T>(c, mk, (T)(A.M[off + k] * c.invVsc));
        parts[k] = pk;
    }
    __syncthreads();

    // row sums: the workers sum their swarm's row (j order) and post them; the
    // control warp takes them into registers
    Acc<T> R[PL];
    auto worker_row_sum = [&]() {
        Acc<T> a;
        a.zero();
        if constexpr (STORE != 0) {
            for (int j = 0; j < n; ++j) {
                const Part<T> pj = parts[j];
                a.add(kern_of<T>(pc, pk.a, pj.a, Dm[sym_at(k, j, n, W)]) * weight<T>(pk, pj));
            }
        } else {
            int j = 0;
            for (; j + 4 <= n; j += 4) {
                T K0, K1, K2, K3;
                const Part<T> p0 = parts[j], p1 = parts[j + 1], p2 = parts[j + 2], p3 = parts[j + 3];
                pair_dv<T>(pc, pk, p0, &K0);
                pair_dv<T>(pc, pk, p1, &K1);
                pair_dv<T>(pc, pk, p2, &K2);
                pair_dv<T>(pc, pk, p3, &K3);
                a.add(K0 * weight<T>(pk, p0));
                a.add(K1 * weight<T>(pk, p1));
                a.add(K2 * weight<T>(pk, p2));
                a.add(K3 * weight<T>(pk, p3));
            }
            for (; j < n; ++j) {
                const Part<T> pj = parts[j];
                T K;
                pair_dv<T>(pc, pk, pj, &K);
                a.add(K * weight<T>(pk, pj));
            }
        }
        Rs[k] = make_float2(a.s, a.c);
    };
    auto rebuild = [&]() {  // entered by every thread after a barrier
        if (act) worker_row_sum();
        __syncthreads();
        if (ctl) {
#pragma unroll
            for (int s = 0; s < PL; ++s) {
                const int kk = PL * lane + s;
                const float2 v = kk < n ? Rs[kk] : make_float2(0.0f, 0.0f);
                R[s].set2(v.x, v.y);
            }
        }
    };
    if constexpr (STORE != 0) {  // every unordered pair once, all warps (warp w rows w, w + nw, ...)
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
    }
    rebuild();

    const uint64_t dcell = (uint64_t)(cell - A.disks[disk].c_off);
    const uint64_t step = (uint64_t)A.state->step;
    const double t_end = A.t_end_from_state ? A.state->t + A.state->dt : A.t_end_fixed;
    const int64_t reb = A.rebuild_every > 0 ? A.rebuild_every : 4 * (int64_t)n;
    int64_t until_rebuild = reb;
    const bool logging = (cell == A.log_cell);
    const T sc = (T)c.sc;
    if (threadIdx.x == 0) sh.t = A.state->t;
    int64_t ev = 0;
    int pend = -1;
    T colo = (T)0, last_tot = (T)0;
    for (;;) {
        // (1) control: fold in the last event's column updates and choose i
        if (ctl) {
            if ((ev & 31) == 0) {
                sh.ring[lane] = make_draw(
                    philox((uint64_t)(ev + lane), dcell, step, kTagCollide, A.seed, (uint64_t)disk), sc);
                __syncwarp();
            }
            T val[PL], y[PL];
#pragma unroll
            for (int s = 0; s < PL; ++s) {
                const int kk = PL * lane + s;
                y[s] = (T)0;
                if (pend >= 0 && kk < n) {
                    y[s] = rnew[kk];
                    if (kk != pend) {
                        const float2 u = upd[kk];
                        R[s].update(u.x, u.y);
                    }
                }
                val[s] = (kk < n && kk != pend) ? R[s].hi() : (T)0;
            }
            // the fresh R_i of the last event's swarm: its new row summed
            T Rp = (T)0;
            if (pend >= 0) {
                Rp = y[0];
#pragma unroll
                for (int s = 1; s < PL; ++s) Rp += y[s];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) Rp += __shfl_xor_sync(FULL, Rp, o);
            }
            const Draw<T> dr = sh.ring[ev & 31];
            T tot;
            int i = warp_choose<PL>(val, dr.u1, pend, Rp, tot);
#pragma unroll
            for (int s = 0; s < PL; ++s)
                if (pend >= 0 && PL * lane + s == pend) R[s].set(Rp);
            last_tot = tot;
            const bool stop = !(tot > (T)0) || ev >= A.max_events;
            if (lane == 0) {
                if (stop && ev >= A.max_events && tot > (T)0 && !A.cap_stops) atomicOr(A.status, kStTimeout);
                if (i < 0 || i >= n) i = n - 1;  // no bracket (non-finite rates): stay in bounds
                sh.sel = i;
                sh.stop = stop ? 3 : 0;
            }
        }
        __syncthreads();  // (H1) i chosen
        if (sh.stop) break;
        const int i = sh.sel;
        // (2) workers: row i (i meets k) and column i (k meets i) before the event
        if (act) {
            const Part<T> pi = parts[i];
            T Kold;
            if constexpr (STORE != 0) {
                const T dvik = Dm[sym_at(i, k, n, W)];
                if (STORE == 2) dvrow[k] = dvik;
                Kold = kern_of<T>(pc, pk.a, pi.a, dvik);
            } else {
                dvrow[k] = pair_dv<T>(pc, pk, pi, &Kold);
            }
            rowv[k] = Kold * weight<T>(pi, pk);
            colo = Kold * weight<T>(pk, pi);
        }
        __syncthreads();  // (H2) row i formed
        // (3) control: choose j; lane 0 advances the clock and, unless the event
        //     would cross t_end (discarded: the process is memoryless), applies
        //     the outcome and the new cache of i (FP64 masses)
        if (ctl) {
            T x[PL];
#pragma unroll
            for (int s = 0; s < PL; ++s) {
                const int kk = PL * lane + s;
                x[s] = kk < n ? rowv[kk] : (T)0;
            }
            // what the outcome needs of i and the clock, ahead of the scan (FP64
            // latency off the chain)
            const Draw<T> dr = sh.ring[ev & 31];
            const double mi = msh[i];
            const double dmmi = c.dm * mi;
            const double tn = sh.t + (double)fdiv(dr.L, last_tot);
            const Part<T> pi = parts[i];
            T tot2;
            int j = warp_choose<PL>(x, dr.u2, -1, (T)0, tot2);
            if (lane == 0) {
                if (j < 0) {
                    sh.stop = 2;
                } else {
                    if (j >= n) j = n - 1;  // (a lane without swarms bracketing by a rounding of the scan)
                    const double mj = msh[j];
                    const T dvij = STORE == 1 ? Dm[sym_at(i, j, n, W)] : dvrow[j];
                    int kind = 0;
                    double mnew;
                    if constexpr (RAMP) {
                        const mcd_disk_params &P = A.params[disk];
                        mnew = outcome_ramp<T>(c, mi, mj, pi.mh, parts[j].mh, dmmi, dvij, dr.u3,
                                               (T)(P.v_frag * (1.0 - P.frag_ramp)), kind);
                    } else {
                        mnew = outcome<T>(c, mi, mj, pi.mh, parts[j].mh, dmmi, dvij, dr.u3, kind);
                    }
                    const Part<T> pnew = make_part<T>(c, mnew, pi.Mv);
                    const int stop = tn >= t_end;
                    if (!stop) {
                        if constexpr (TRACER)
                            qsh[i] = tracer_update(mi, mj, qsh[i], qsh[j], dgt(dmmi, mj) ? dmmi : mj, mnew, kind, c.chi);
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
            }
        }
        __syncthreads();  // (H3) the event applied
        if (sh.stop) {
            if (sh.stop == 2 && threadIdx.x == 0) atomicOr(A.status, kStNaN);  // row i's prefix not finite
            break;
        }
        // (4) workers: the new row and column i; R_k += r_ki(new) - r_ki(old) is
        //     applied by the control warp, R_i summed afresh from the new row
        if (act) {
            const Part<T> pn = parts[i];
            if (k == i) pk = pn;
            T Knew;
            const T dvn = pair_dv<T>(pc, pk, pn, &Knew);
            if constexpr (STORE != 0) Dm[sym_at(i, k, n, W)] = dvn;
            rnew[k] = Knew * weight<T>(pn, pk);
            upd[k] = make_float2(Knew * weight<T>(pk, pn), colo);
        }
        pend = i;
        ++ev;
        __syncthreads();  // (H4) new row and column posted
        if (--until_rebuild == 0) {  // every row sum afresh (the pending updates are superseded)
            rebuild();
            pend = -1;
            until_rebuild = reb;
        }
    }
    __syncthreads();
    if (act) {
        A.m[off + k] = msh[k];
        if (TRACER) A.q[off + k] = qsh[k];
    }
    if (ctl) {
        if (A.Rdump)
#pragma unroll
            for (int s = 0; s < PL; ++s) {
                const int kk = PL * lane + s;
                if (kk < n) A.Rdump[off + kk] = R[s].value() / c.sc;
            }
        if (lane == 0) {
            A.cell_events[cell] = ev;
            atomicAdd(&A.events_total[disk], (unsigned long long)ev);
            if (logging) *A.log_n = (unsigned long long)(ev < A.log_cap ? ev : A.log_cap);
            if (A.Rtot) A.Rtot[cell] = (double)last_tot / c.sc;
        }
    }
}

template <int PL, int STORE, bool RAMP, bool TRACER>
__global__ void __launch_bounds__(32 + 32 * PL) k_collide_ws(CollideArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Shared<float> sh;
    int64_t entry = blockIdx.x;
    for (;;) {
        if (A.qhead) {
            __syncthreads();
            if (threadIdx.x == 0) sh.ticket = atomicAdd(A.qhead, 1);
            __syncthreads();
            entry = sh.ticket;
        }
        if (entry >= A.n_queue) return;
        const int64_t cell = A.queue ? (int64_t)A.queue[entry] : entry;
        cell_chain_ws<PL, STORE, RAMP, TRACER>(A, cell, entry, sh, smem_raw);
        if (!A.qhead) return;
    }
}


template <int PL, int STORE>
cudaError_t collide_ws_variant_store(int op, bool ramp, bool tracer, unsigned grid, int nthr, size_t smem,
                                     cudaStream_t st, const CollideArgs *A, int *out)
{
    void (*ks[4])(CollideArgs) = {k_collide_ws<PL, STORE, false, false>, k_collide_ws<PL, STORE, true, false>,
                                  k_collide_ws<PL, STORE, false, true>, k_collide_ws<PL, STORE, true, true>};
    if (op == 0) {
        ks[(ramp ? 1 : 0) + (tracer ? 2 : 0)]<<<grid, nthr, smem, st>>>(*A);
        return cudaGetLastError();
    }
    if (op == 3) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, ks[(ramp ? 1 : 0) + (tracer ? 2 : 0)], nthr, smem);
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

// host entry of the control-warp variants of one PL (same ops as
// collide_variant), instantiated in mcd_collide_f32ws4.cu (PL 4, 7) and
// mcd_collide_f32ws10.cu (PL 10, 16)
template <int PL>
cudaError_t collide_ws_variant(int op, int store, bool ramp, bool tracer, unsigned grid, int nthr, size_t smem,
                               cudaStream_t st, const CollideArgs *A, int *out)
{
    switch (store) {
    case 0: return collide_ws_variant_store<PL, 0>(op, ramp, tracer, grid, nthr, smem, st, A, out);
    case 1: return collide_ws_variant_store<PL, 1>(op, ramp, tracer, grid, nthr, smem, st, A, out);
    case 2: return collide_ws_variant_store<PL, 2>(op, ramp, tracer, grid, nthr, smem, st, A, out);
    default: return cudaErrorInvalidValue;
    }
}
extern template cudaError_t collide_ws_variant<4>(int, int, bool, bool, unsigned, int, size_t, cudaStream_t,
                                                  const CollideArgs *, int *);
extern template cudaError_t collide_ws_variant<7>(int, int, bool, bool, unsigned, int, size_t, cudaStream_t,
                                                  const CollideArgs *, int *);
extern template cudaError_t collide_ws_variant<10>(int, int, bool, bool, unsigned, int, size_t, cudaStream_t,
                                                   const CollideArgs *, int *);
extern template cudaError_t collide_ws_variant<16>(int, int, bool, bool, unsigned, int, size_t, cudaStream_t,
                                                   const CollideArgs *, int *);

}  // namespace mcd
