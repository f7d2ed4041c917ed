/*
 * mcd.h -- C ABI of libmcd.so, a GB300 (sm_103a) implementation of the hot
 * path of mcdust (Vaikundaraman, Gurrutxaga & Drazkowska 2025, "mcdust: A 2D
 * Monte Carlo code for dust coagulation in protoplanetary disks").
 *
 * The path, per time step (Summary section): particles binned into an
 * adaptive grid whose cells hold equal numbers of representative particles
 * (mcd_regrid); in every cell, the representative-particle Monte Carlo
 * collision chain of Zsom & Dullemond (2008) with sticking, fragmentation and
 * erosion outcomes (mcd_collide); then radial and vertical transport of the
 * particles in a static, vertically isothermal power-law gas disk, or one
 * tabulated in radius (mcd_set_gas_table) (mcd_transport).  mcd_step runs the
 * three in that order.
 *
 * Conventions for every call:
 *  - CGS units; times in seconds.
 *  - Every call returns an int: MCD_OK (0) or a negative MCD_E* code.  No C++
 *    exception crosses this boundary.  Device-side failures (NaN positions,
 *    an event-count cap reached) latch into a status word that mcd_sync and
 *    mcd_get_stats return.
 *  - Work is enqueued on the CUDA stream given to mcd_init_disk and calls
 *    return without waiting, except those that copy to host memory
 *    (mcd_get_*, mcd_sync), which synchronise that stream.
 *  - The caller owns the device workspace (its size from mcd_workspace_size)
 *    and every host array passed in; the library owns the context and never
 *    allocates device memory after mcd_init_disk.
 *  - Disks are independent: arrays of n_disks parameter sets and grids run
 *    together in one set of launches.
 */
#ifndef MCD_H
#define MCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MCD_OK 0
#define MCD_EINVAL -1   /* invalid argument (sizes, pointers, parameters) */
#define MCD_ENOMEM -2   /* workspace smaller than mcd_workspace_size */
#define MCD_ECUDA -3    /* a CUDA runtime call failed */
#define MCD_ENAN -4     /* NaN met in particle positions */
#define MCD_ETIMEOUT -5 /* a cell reached the per-call event cap */
#define MCD_EEMPTY -6   /* every particle of a disk has been removed */
#define MCD_ESTATE -7   /* call out of order (e.g. collide before regrid) */

/* ---- precision of the collision arithmetic ------------------------------ */
#define MCD_FP64 0  /* everything in FP64 */
#define MCD_MIXED 1 /* dv, sigma, K and rates in FP32; masses, clock and the
                       running row sums in FP64 / compensated FP32 */

/* ---- where a pointer lives ---------------------------------------------- */
#define MCD_HOST 0
#define MCD_DEVICE 1

/* ---- switches ------------------------------------------------------------ */
#define MCD_DV_BM 1    /* Brownian motion */
#define MCD_DV_TURB 2  /* turbulence (Ormel & Cuzzi 2007 closed forms) */
#define MCD_DV_RAD 4   /* radial drift */
#define MCD_DV_PHI 8   /* azimuthal drift */
#define MCD_DV_SET 16  /* vertical settling */
#define MCD_TR_RADIAL 1
#define MCD_TR_VERTICAL 2
#define MCD_TR_ST_MIDPLANE 4 /* transport uses the midplane Stokes number */

/*
 * One disk.  The first seven fields are the paper's Benchmark table (gas
 * surface density and temperature at 1 AU, alpha, v_frag, erosion mass ratio,
 * p, q).  The rest are not given by the paper and are readings: dust-to-gas
 * ratio, radial extent, stellar mass [M_sun], monomer density and radius,
 * mean molecular weight, H2 cross-section, the Zsom & Dullemond grouping
 * ratio dm_group (0 = off), the fragment mass slope frag_xi (n(m) ~ m^-xi),
 * the eroded-mass factor erosion_chi, and overrides for the 0D
 * constant-kernel test problem (kernel_mode = 1: K = K_const, V = V_const,
 * always sticking).  m_init > 0 overrides the monomer mass, M_total > 0 the
 * disk dust mass.  settle_form 0: v_z = -z Omega St; 1: -z Omega St/(1+St).
 */
typedef struct {
    double sigma0, p, T0, q, alpha, v_frag, erosion_ratio;
    double dust_to_gas, r_in, r_out, m_star, rho_s, a_mono;
    double mu, sigma_h2, dm_group, frag_xi, erosion_chi;
    double K_const, V_const, m_init, M_total;
    double frag_ramp; /* fragmentation probability: 0 below v_frag (1 - frag_ramp), 1 from v_frag, linear
                         between (0 = the sharp threshold); 0 <= frag_ramp < 1 */
    int32_t kernel_mode, settle_form, dv_flags, tr_flags;
} mcd_disk_params;

/* n_r radial zones x n_z cells per zone, per_cell particles per cell at start */
typedef struct {
    int32_t n_r, n_z, per_cell, reserved;
} mcd_grid;

typedef struct {
    double t;             /* clock [s] */
    int64_t step;         /* steps (transport calls) taken */
    int64_t events;       /* collision events, cumulative */
    int64_t n_alive;      /* particles not yet removed at r_in */
    double accreted_mass; /* swarm mass removed at r_in [g] */
    int32_t status;       /* latched device status, an MCD_* code */
    int32_t reserved;
} mcd_stats;

typedef struct mcd_ctx mcd_ctx;

/* ---- options (mcd_set_option) -------------------------------------------- */
#define MCD_OPT_MAX_EVENTS 1    /* per cell per collide call; reaching it latches MCD_ETIMEOUT (default 1e7) */
#define MCD_OPT_CAP_STOPS 2     /* 1: reaching MAX_EVENTS stops the cell without an error (tests) */
#define MCD_OPT_REBUILD_EVERY 3 /* events between full row-sum rebuilds; 0 = 4n of the cell (default) */
#define MCD_OPT_USE_GRAPH 4     /* 1: mcd_step replays a captured CUDA graph (default 1) */
#define MCD_OPT_DUMP_R 5        /* 1: keep each particle's row sum after collide (mcd_get_rates) */
#define MCD_OPT_LOG_CELL 6      /* global cell index whose events are logged; -1 off (default) */
#define MCD_OPT_LPT 7           /* 1: order cells by descending work estimate (default 1) */
#define MCD_OPT_THREADS 8       /* threads per cell in collide; 0 = auto */
#define MCD_OPT_EXCLUSIVE 9     /* 1: one collide CTA per SM, so long event chains share no SM (default 1) */
#define MCD_OPT_DV_MATRIX 10    /* where each cell's symmetric dv_ij matrix is kept (circulant half form,
                                   each pair once): 1 MCD_MIXED in shared memory when it fits (cells of up
                                   to ~314 particles), else in the workspace when reserved; 2 in the
                                   workspace when reserved (MCD_FP64: every class, when all matrices
                                   together take at most 8 GiB; MCD_MIXED: the classes whose matrix does
                                   not fit in shared memory, within 16 GiB); 0 recompute row i at every
                                   event; -1 (default) chosen per class by the timed trial.  All give
                                   bit-identical results */
#define MCD_OPT_TRACER 11       /* 1: every swarm carries the tracer column (mcd_get_tracer); 0 (default)
                                   clears it.  mcd_set_tracer switches it on. */
#define MCD_OPT_DT_MAX 12       /* the largest step mcd_step(dt <= 0) takes [s] (default one year) */
#define MCD_OPT_COURANT 13      /* C of the adaptive step (default 0.5) */
#define MCD_OPT_SWARMS_PER_THREAD 14 /* collide threads own 1 or 2 swarms (MCD_MIXED only for 2); 0 (default)
                                   chosen per class by the timed trial.  The mixed path's trajectories
                                   depend on it at the level of FP32 rounding in the choice scans (the
                                   FP64 path runs 1) */
#define MCD_OPT_PERSISTENT 15   /* 1: persistent collide CTAs (resident ones only) take cells from the
                                   largest-work-first queue by an atomic ticket; 0 (default) one CTA per
                                   cell.  Results are identical */
#define MCD_OPT_EXACT_TOTAL 17  /* MCD_MIXED, 1: the total rate that sets each waiting time, and the fresh row
                                   sum of the last event's swarm, are compensated (TwoSum) sums of the
                                   compensated row sums, formed by one extra warp per cell (MCD_OPT_THREADS
                                   must then leave room for it); 0 (default): block sums of the row sums'
                                   leading parts, relative error below 10 ulp, formed afresh each event */
#define MCD_OPT_AUTOTUNE 16     /* 1 (default): before its first collide the context times the candidate
                                   variants of each cell class (swarms per thread, control warp, dv-matrix
                                   store) on the class's largest cells and keeps the fastest
                                   (mcd_get_collide_classes); setting it to 1 again repeats the trial at the
                                   next collide */
#define MCD_OPT_CONTROL_WARP 18 /* MCD_MIXED: 1 runs every class with a control warp (one warp keeps the row
                                   sums in registers and makes both choices with warp-wide scans; one worker
                                   thread per swarm forms the rows); 0 the block variants (every thread
                                   holds its swarms' row sums, block-wide scans); -1 (default) the timed
                                   trial decides per class, unless MCD_OPT_SWARMS_PER_THREAD is set.  The
                                   trajectories differ from the block variants' at the level of FP32
                                   rounding in the choice scans */

/*
 * Bytes of device workspace needed for n_disks disks at precision prec.
 * p[n_disks], g[n_disks] host arrays.  Returns MCD_EINVAL on a bad grid.
 * The stored dv matrices add, per cell class (disks grouped by particles per
 * cell: up to 64, 128, 224, ~314, 512), cells x n_hi x W entries (W about
 * n_hi / 2 + 1; n_hi the class's largest per_cell): MCD_FP64 for every class
 * when all take at most 8 GiB, MCD_MIXED for the classes whose matrix does not
 * fit in shared memory when those take at most 16 GiB.
 */
int mcd_workspace_size(const mcd_disk_params *p, const mcd_grid *g, int32_t n_disks, int32_t prec, size_t *bytes);

/*
 * Create a context and the initial particles (workload recipe of the paper's
 * Benchmark: equal swarm masses summing to the disk's dust mass, r drawn from
 * the dust-mass distribution, z ~ N(0, H_g(r)), monomers), then bin them
 * (mcd_regrid).  Random numbers come from Philox4x64-10 keyed by (seed, disk).
 * device_workspace: caller-owned device memory of ws_bytes >= the size from
 * mcd_workspace_size, 256-byte aligned; it must outlive the context.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 */
int mcd_init_disk(mcd_ctx **out, const mcd_disk_params *p, const mcd_grid *g, int32_t n_disks, uint64_t seed,
                  int32_t prec, void *device_workspace, size_t ws_bytes, void *cuda_stream);

/*
 * Advance every cell's clock to t_end with the representative-particle
 * event chain (Summary: sticking, fragmentation, erosion; Zsom & Dullemond
 * 2008): waiting times from the total rate, partner selection by rate
 * weight, only row and column i of the rate matrix updated per event.
 * Requires current cells (mcd_regrid after the last transport).
 */
int mcd_collide(mcd_ctx *ctx, double t_end);

/*
 * Move every particle over dt (Summary: transport in the radial and vertical
 * directions): radial drift plus turbulent diffusion, settling plus mixing.
 * Particles crossing r_in are removed (their swarm mass is accreted); those
 * crossing r_out are reflected.  Increments the step counter.
 */
int mcd_transport(mcd_ctx *ctx, double dt);

/*
 * Re-bin particles into equal-count cells (Summary: adaptive grid): n_r
 * radial zones of equal count by (r, id), then n_z cells of equal count per
 * zone by (z, id); particle arrays are reordered into cell order.
 */
int mcd_regrid(mcd_ctx *ctx);

/*
 * One step: regrid, collide to t + dt, transport dt (Summary section: binning,
 * collisional evolution, transport).  dt > 0: that step.  dt <= 0: the step is
 * chosen on the device after the regrid (a reading; the paper gives no rule):
 * per disk min(dt_max, C min_c (r_hi - r_lo)_c / max_i |v_r,i|) over the cells
 * that hold particles and the live particles, v_r = -2 eta v_K St / (1 + St^2)
 * the radial drift of the transport step; a disk without radial transport asks
 * for dt_max.  The disks of a context share one clock, so the step is the
 * smallest of theirs.  dt_max and C are MCD_OPT_DT_MAX and MCD_OPT_COURANT;
 * the mixed path evaluates v_r in FP32 like its transport.  The host learns
 * the clock from mcd_get_stats (t); the first mcd_collide after adaptive steps
 * synchronises once to read it.  NaN or infinite dt: MCD_EINVAL.
 */
int mcd_step(mcd_ctx *ctx, double dt);

/*
 * A tracked property per swarm (a particle history such as a composition
 * fraction, Statement of Need section), carried by the representative particle through the
 * regrid and updated at every collision (a reading: the paper names no rule):
 * sticking mixes by mass, (m_i q_i + g q_j) / (m_i + g) with g the absorbed
 * mass; fragmentation gives the pair's mass-weighted mixture; erosion leaves the
 * larger body's q and makes the smaller one debris of itself and erosion_chi
 * times its mass chipped from the other, (q_i + chi q_j) / (1 + chi).  It starts
 * at 0 and costs nothing while off.  q: disk `disk`'s n0 values in the order
 * mcd_get_particles returns; where = MCD_HOST (synchronises) or MCD_DEVICE.
 * mcd_set_tracer switches the tracer on; mcd_set_particles leaves the column
 * as it is, slot by slot.
 */
int mcd_get_tracer(mcd_ctx *ctx, int32_t disk, double *q, int32_t where);
int mcd_set_tracer(mcd_ctx *ctx, int32_t disk, const double *q, int32_t where);

/*
 * Copy disk `disk`'s particles in cell order (dead ones, r = +inf, last).
 * Arrays of at least the disk's initial particle count; any may be NULL.
 * where = MCD_HOST (synchronises) or MCD_DEVICE (device pointers, async).
 */
int mcd_get_particles(mcd_ctx *ctx, int32_t disk, double *m, double *M, double *r, double *z, uint32_t *id,
                      int64_t *count, int32_t where);

/*
 * Replace disk `disk`'s particles (count must equal its initial particle
 * count; ids a permutation of 0..count-1; r = +inf marks a removed particle).
 * Cells become stale: call mcd_regrid before mcd_collide.
 * The columns are staged on the device and the ids checked there; only a
 * permutation replaces the live state, which bad ids leave untouched.
 * where = MCD_HOST: host arrays, synchronises, returns MCD_EINVAL for bad ids.
 * where = MCD_DEVICE: device arrays, asynchronous; bad ids latch MCD_EINVAL
 * in the status word (mcd_sync / mcd_get_stats).
 */
int mcd_set_particles(mcd_ctx *ctx, int32_t disk, const double *m, const double *M, const double *r,
                      const double *z, const uint32_t *id, int64_t count, int32_t where);

/*
 * Cells of disk `disk` after the last regrid: cell_off[n_r*n_z+1] particle
 * offsets within the disk, bounds[6 per cell] = r_lo r_hi z_lo z_hi r_c z_c,
 * V[n_r*n_z] volumes.  Any pointer may be NULL.
 */
int mcd_get_cells(mcd_ctx *ctx, int32_t disk, int64_t *cell_off, double *bounds, double *V, int32_t where);

/* Per-particle row sums R_i after the last collide (needs MCD_OPT_DUMP_R). */
int mcd_get_rates(mcd_ctx *ctx, int32_t disk, double *R, int32_t where);

/*
 * Per cell of the disk (n_r * n_z values, cell order): the total rate R_tot of
 * the last choice scan of the last collide, the value that set the waiting
 * time there (Zsom & Dullemond's event loop, Summary section; MCD_MIXED: the
 * compensated FP32 sum of the compensated row sums, as a double).  Needs
 * MCD_OPT_DUMP_R; with MCD_OPT_MAX_EVENTS 0 and MCD_OPT_CAP_STOPS 1 it is the
 * total of the rebuilt row sums that mcd_get_rates returns.
 */
int mcd_get_total_rates(mcd_ctx *ctx, int32_t disk, double *Rtot, int32_t where);

/*
 * The collide's cell classes (disks grouped by particles per cell) and the
 * variant each runs: threads per cell, swarms per thread, control warp,
 * dv-matrix store, and the timed trial's candidates (the time per event of
 * each, the median of five runs of 512 events on up to 8 of the class's
 * largest cells, after one warm-up run).  Host memory; up to cap records, *count the number of
 * classes.  This is the implementation's scheduling, not the paper's method.
 */
#define MCD_MAX_TRIALS 12
typedef struct {
    int32_t n_lo, n_hi;          /* particles per cell of the class's disks */
    int64_t cells;               /* cells in the class */
    int32_t threads;             /* threads per cell */
    int32_t swarms_per_thread;   /* 1 or 2 (the control-warp variant: 1 per worker thread) */
    int32_t store;               /* dv matrix: 0 row i recomputed, 1 shared memory, 2 workspace */
    int32_t persistent;          /* persistent CTAs take cells by atomic ticket */
    int32_t control_warp;        /* 1: the control-warp variant (MCD_OPT_CONTROL_WARP) */
    int32_t tuned;               /* 1: chosen by the timed trial */
    int32_t n_trials;            /* candidates timed (at most MCD_MAX_TRIALS) */
    int32_t trial_swarms[MCD_MAX_TRIALS], trial_store[MCD_MAX_TRIALS], trial_control_warp[MCD_MAX_TRIALS];
    float trial_us_per_event[MCD_MAX_TRIALS]; /* the trial's time per event [us] */
} mcd_collide_class;
int mcd_get_collide_classes(mcd_ctx *ctx, mcd_collide_class *out, int32_t cap, int32_t *count);

/* Per-cell event counts of the last collide, n_r*n_z entries. */
int mcd_get_cell_events(mcd_ctx *ctx, int32_t disk, int64_t *events, int32_t where);

/*
 * Event log of the cell chosen with MCD_OPT_LOG_CELL: up to cap records of
 * (i, j, outcome) as int32 triples and the event time t and new mass of i.
 * outcome 0 stick, 1 fragment, 2 erode.  Returns the number logged in *n.
 */
int mcd_get_event_log(mcd_ctx *ctx, int32_t *ijo, double *t, double *m_new, int64_t cap, int64_t *n);

int mcd_get_stats(mcd_ctx *ctx, int32_t disk, mcd_stats *out);

/*
 * Checkpoint and resume (the paper describes none; the random streams are
 * keyed by (seed, disk) and counted by step, cell and event or particle id,
 * so a resumed run repeats the checkpointed one bit for bit).  mcd_set_clock
 * sets the context's clock t [s] and its step counter; mcd_set_counters sets
 * a disk's collision-event count and accreted swarm mass [g], as
 * mcd_get_stats read them from the checkpointed context.  To resume, create a
 * context with the same parameters, grids, seed and precision, then call
 * mcd_set_particles (and mcd_set_tracer, mcd_set_gas_table and the options
 * the checkpointed context had) for every disk, mcd_set_clock once and
 * mcd_set_counters per disk.  On MCD_MIXED the collide variant must be the
 * same one (pin MCD_OPT_SWARMS_PER_THREAD, or MCD_OPT_CONTROL_WARP): the
 * variants' choice scans sum in different orders.  Asynchronous (the values
 * reach the device as kernel arguments); MCD_EINVAL for a non-finite or
 * negative time, a negative step or count, or a bad disk.
 */
int mcd_set_clock(mcd_ctx *ctx, double t, int64_t step);
int mcd_set_counters(mcd_ctx *ctx, int32_t disk, int64_t events, double accreted_mass);

/* Diagnostics (Benchmark section: the dust surface density as a function of
 * particle mass and distance from the star, here summarised per radial bin).
 * For every bin b = [edges[b], edges[b+1]) of disk `disk`, over the particles
 * whose r lies in it (a removed particle has r = +inf and counts nowhere):
 *   out[5b + 0] = sum M_i, out[5b + 1] = sum M_i m_i, out[5b + 2] = sum M_i m_i^2,
 *   out[5b + 3] = sum M_i m_i^3, out[5b + 4] = the number of particles.
 * The mass-weighted moments of the representative mass are out[5b+k]/out[5b].
 * Sums are compensated (Neumaier) and combined in a fixed order, so repeated
 * calls give the same bits.  edges: host, nbins + 1 non-decreasing values [cm]
 * (a particle on an interior edge belongs to the bin above it); out: host,
 * 5 * nbins doubles, filled when the call returns (it synchronises the
 * context's stream).  1 <= nbins <= MCD_MAX_BINS; NaN or descending edges give
 * MCD_EINVAL. */
#define MCD_MAX_BINS 1024
int mcd_moments(mcd_ctx *ctx, int32_t disk, int32_t nbins, const double *edges, double *out);

/* The sigma_d(m, r) map (Benchmark section: the dust surface density as a
 * function of particle mass and distance from the star): out[b * nm + q] =
 * the swarm mass sum M_i [g] over disk `disk`'s particles with r in
 * [r_edges[b], r_edges[b+1]) and m in [m_edges[q], m_edges[q+1]).  Divided by
 * pi (r_hi^2 - r_lo^2) and ln(m_hi / m_lo) it is sigma_d per logarithmic mass
 * interval.  Each M_i enters rounded to a power-of-two unit of at most 2^-61 of
 * the disk's live swarm mass and the sums are integer, so repeated calls give
 * the same bits.  Edges: host, non-decreasing, no NaN (MCD_EINVAL otherwise);
 * out: host, nr * nm doubles, filled when the call returns (it synchronises
 * the context's stream).  nr, nm <= MCD_MAX_MAP_EDGES, nr * nm <=
 * MCD_MAX_MAP_BINS. */
#define MCD_MAX_MAP_EDGES 4096
#define MCD_MAX_MAP_BINS 65536
int mcd_sigma_map(mcd_ctx *ctx, int32_t disk, int32_t nr, const double *r_edges, int32_t nm, const double *m_edges,
                  double *out);
int mcd_set_option(mcd_ctx *ctx, int32_t key, double value);

/* A gas disk tabulated in radius in place of the power laws Sigma0 (r/AU)^-p,
 * T0 (r/AU)^-q: the azimuthally averaged profile of a hydrodynamic snapshot
 * that the method post-processes (Statement of Need section).  n knots r[k] [cm],
 * Sigma[k] [g cm^-2], T[k] [K] (host arrays): r strictly increasing, every
 * value finite and positive.  Between knots Sigma and T are linear in
 * ln r - ln Sigma (ln T), and the first and last segments extend beyond the
 * ends, so a table sampled from a power law gives that power law back; the
 * pressure-gradient speed eta v_K and the radial diffusion drift take the
 * logarithmic slopes of the segment holding r.  The disk stays vertically
 * isothermal with a Gaussian profile.  n = 0 restores the power laws; n = 1,
 * n > MCD_MAX_GAS_KNOTS or a bad value give MCD_EINVAL and leave the table
 * as it was.  The table is read by every later collide, transport and regrid
 * (a captured step graph stays valid); the initial draw of mcd_init_disk, the
 * probes and mcd_regrid_noalloc use the power laws.  The host arrays may be
 * released when the call returns (it synchronises the context's stream). */
#define MCD_MAX_GAS_KNOTS 1024
int mcd_set_gas_table(mcd_ctx *ctx, int32_t disk, int32_t n, const double *r, const double *Sigma,
                      const double *T);

/*
 * Phase tracing.  With on = 1 every later mcd_step records CUDA events on the
 * context's stream before the regrid, after the regrid, after the cell
 * ordering, after the collisions and after the transport (inside the step's
 * CUDA graph when graphs are on).  mcd_trace_read waits for the last traced
 * step and writes its four phase durations [regrid, order, collide,
 * transport] in milliseconds to ms[4].
 */
int mcd_trace(mcd_ctx *ctx, int32_t on);
int mcd_trace_read(mcd_ctx *ctx, float *ms);

/* Number of kernels this context has launched so far (graph replays count
   every kernel node). */
int mcd_get_launch_count(mcd_ctx *ctx, int64_t *launches);

/* Synchronise the context's stream; returns the latched device status. */
int mcd_sync(mcd_ctx *ctx);

/* Release the context (not the caller's workspace). */
int mcd_free(mcd_ctx *ctx);

const char *mcd_strerror(int code);

/*
 * Pair probe (parity tests): relative velocity and collision kernel of n
 * pairs (m_i[k], m_j[k]) in the gas at cell centre (r_c, z_c), computed by
 * the device functions the collide kernel uses, at precision prec.
 * m_i, m_j, dv, K: device arrays of n doubles.  Asynchronous on stream.
 */
int mcd_pair_probe(const mcd_disk_params *p, int32_t prec, double r_c, double z_c, int64_t n, const double *m_i,
                   const double *m_j, double *dv, double *K, void *cuda_stream);

/*
 * Rate-matrix probe: rate[i*n+j] = K_ij (M_j/V) min(1/m_j, 1/(dm m_i)) and
 * the row sums R[i] of one cell of n <= 1024 swarms, computed by the collide
 * kernel's build phase at precision prec.  Device arrays; asynchronous.
 */
int mcd_rate_probe(const mcd_disk_params *p, int32_t prec, double r_c, double z_c, double V, int32_t n,
                   const double *m, const double *M, double *rate, double *R, void *cuda_stream);

/*
 * Regrid of one disk that allocates nothing (the paper has no counterpart;
 * this is a service entry point).  For callers that cannot call cudaMalloc:
 * code that runs inside another framework's memory pool or arena (which owns
 * every allocation), real-time loops where an allocation would stall, and
 * embedded users with a fixed memory budget.  It does what mcd_regrid does
 * for one disk, without a context: the
 * caller passes the particle arrays (n_r * n_z * per_cell of each, device
 * pointers; ids a permutation of 0..count-1, r = +inf for removed particles)
 * and receives the arrays in cell order (m_out .. id_out), each cell's first
 * slot and count (cell_start[n_r*n_z], cell_n[n_r*n_z]), bounds[6 per cell]
 * (r_lo r_hi z_lo z_hi r_c z_c), volumes V[n_r*n_z], the alive count
 * (*n_alive) and a device status code (*status: MCD_OK, MCD_ENAN for NaN
 * positions, MCD_EINVAL for invalid ids, MCD_EEMPTY for an emptied disk), all
 * device pointers, enqueued on cuda_stream.
 *
 * Its scratch (sort keys and values, histograms, tables, status bits) is one
 * fixed device array of about 2.1 MB that every GPU loading the library holds
 * until the process exits; hence at most MCD_NOALLOC_MAX_PARTICLES particles
 * (MCD_EINVAL beyond, and when one radial zone holds more than 14,336).  The
 * first call on a device looks the array's device address up; make it before
 * any stream capture.  All calls share the array and it keeps the previous
 * call's contents (the status bits are cleared at the start of each call):
 * calls that overlap on the GPU race on it and must be serialised by the
 * caller.  It calls no cudaMalloc, cudaFree or allocating library routine;
 * its disk tables reach the device as kernel arguments, not host copies.
 */
#define MCD_NOALLOC_MAX_PARTICLES 65536
int mcd_regrid_noalloc(const mcd_disk_params *p, const mcd_grid *g, const double *m, const double *M,
                       const double *r, const double *z, const uint32_t *id, double *m_out, double *M_out,
                       double *r_out, double *z_out, uint32_t *id_out, int64_t *cell_start, int32_t *cell_n,
                       double *bounds, double *V, int64_t *n_alive, int32_t *status, void *cuda_stream);

/*
 * Microbenchmarks of this GPU (measurement only; the paper has no
 * counterpart): shared-memory read bandwidth (conflict-free 16-byte loads,
 * two 1024-thread CTAs per SM), FP32 and FP64 FMA throughput (eight
 * independent chains per thread), each the median of three CUDA-event-timed
 * runs on cuda_stream after a warm-up run; plus the SM count, the SM clock the
 * device reports, the L2 size and the shared memory per SM.  These are the
 * denominators of the collide kernel's rooflines.  Synchronous; allocates
 * nothing.
 */
typedef struct {
    double smem_gbs;      /* shared-memory read bandwidth, all SMs [GB/s] */
    double fp32_tflops;   /* FP32 FMA throughput (2 flops per FMA) [TFLOP/s] */
    double fp64_tflops;   /* FP64 FMA throughput [TFLOP/s] */
    int32_t sm_count, sm_clock_mhz, l2_bytes, smem_per_sm_bytes;
    float ms_smem, ms_fp32, ms_fp64;  /* the timed runs' medians [ms] */
} mcd_peaks;
int mcd_probe_peaks(mcd_peaks *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MCD_H */
