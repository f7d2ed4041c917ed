// mcd_regrid.cu -- the adaptive equal-count grid (Summary of the mcdust paper:
// "each cell has equal number of representative particles").
//
// Rule (reading): particles are ranked by (r, id); radial zone k of n_r takes
// the next floor(N/n_r) of them, the first N mod n_r zones one extra; within a
// zone particles are ranked by (z, id) and split into n_z cells the same way.
// Interior cell edges are midpoints of neighbouring sorted positions, outer
// edges extend by half the first / last spacing, V = pi (r_hi^2 - r_lo^2)
// (z_hi - z_lo).  Removed particles (r = +inf) stay at the tail in id order.
//
// GB300 design:
//  1. keys: each particle's order-preserving 64-bit r key is written at
//     position (disk offset + id), so a stable sort by r alone breaks ties by id;
//  2. a segmented LSD radix sort of the keys' upper four bytes (sign, exponent
//     and 20 mantissa bits), 4 passes of 8 bits, all disks in one launch
//     sequence (tiles never straddle disks; the histogram is laid out disk-major,
//     digit, tile so one exclusive scan yields every scatter offset), then every
//     run of equal upper words put in (r, id) order (k_rfix, k_rfix_long);
//  3. one CTA per radial zone loads its (z, id) keys into shared memory, sorts
//     them (radix on the upper words with the same run fix-up, or a bitonic
//     network that needs no padding: every compare is ascending, absent
//     elements act as +inf), computes cell bounds with explicitly rounded FP64
//     operations (no fused multiply-add, so they are bit-identical to a plain
//     CPU evaluation), and gathers the particle columns into cell order.
#include <math.h>

#include "mcd_internal.cuh"

namespace mcd {

__device__ __forceinline__ uint64_t order_key(double x)
{
    if (x == 0.0) x = 0.0;  // -0.0 -> +0.0
    uint64_t b = (uint64_t)__double_as_longlong(x);
    return (b & 0x8000000000000000ULL) ? ~b : (b | 0x8000000000000000ULL);
}

__device__ __forceinline__ double key_value(uint64_t k)
{
    uint64_t b = (k & 0x8000000000000000ULL) ? (k & 0x7FFFFFFFFFFFFFFFULL) : ~k;
    return __longlong_as_double((long long)b);
}

constexpr uint64_t kInfKey = 0xFFF0000000000000ULL;  // order_key(+inf)

__global__ void k_regrid_keys(const DiskDev *disks, const int32_t *slot_disk, int64_t N, const double *r,
                              const double *z, const uint32_t *id, uint64_t *key, uint32_t *val, int32_t *status)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int d = slot_disk[s];
    double rs = r[s];
    if (isnan(rs) || isnan(z[s])) {
        atomicOr(status, kStNaN);
        rs = INFINITY;
    }
    uint32_t k = id[s];
    if ((int64_t)k >= disks[d].n0) {
        atomicOr(status, kStBadCell);
        return;
    }
    int64_t dst = disks[d].p_off + k;
    key[dst] = order_key(rs);
    val[dst] = (uint32_t)(s - disks[d].p_off);
}

// Lanes of the warp holding the same 8-bit digit as this lane, among the lanes
// with ok set (an empty lane gets 0): the AND over the digit's bits of each
// bit's ballot or its complement.  Nine independent ballots; a warp match
// costs more once the lanes hold many distinct values.
__device__ __forceinline__ unsigned digit_peers(int digit, bool ok)
{
    unsigned peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (digit >> b) & 1;
        const unsigned m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
    }
    return ok ? peers : 0u;
}

// histogram index of (tile t of disk d, digit b)
__device__ __forceinline__ int64_t hidx(const DiskDev &D, int64_t t, int b)
{
    return 256 * D.t_off + (int64_t)b * D.n_tiles + (t - D.t_off);
}

__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const DiskDev *disks, const int32_t *tile_disk,
                                                              const uint64_t *key, int shift, uint32_t *hist)
{
    __shared__ uint32_t h[kRadixBins];
    int64_t t = blockIdx.x;
    const DiskDev D = disks[tile_disk[t]];
    int64_t start = D.p_off + (t - D.t_off) * kRadixTile;
    int64_t end = min(start + kRadixTile, D.p_off + D.n0);
    h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t q = start + threadIdx.x; q < end; q += kRadixThreads) atomicAdd(&h[(key[q] >> shift) & 255], 1u);
    __syncthreads();
    hist[hidx(D, t, threadIdx.x)] = h[threadIdx.x];
}

constexpr int kScanThreads = 1024, kScanItems = 4, kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t x, uint32_t *wsum, uint32_t &total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) wsum[w] = v;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < nw ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) wsum[lane] = s;
    }
    __syncthreads();
    total = wsum[nw - 1];
    uint32_t res = v - x + (w > 0 ? wsum[w - 1] : 0);
    __syncthreads();
    return res;
}

// exclusive scan of each block of kScanBlock entries in place; block totals to part
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(uint32_t *a, int64_t n, uint32_t *part)
{
    __shared__ uint32_t wsum[32];
    int64_t base = blockIdx.x * (int64_t)kScanBlock + threadIdx.x * kScanItems;
    uint32_t v[kScanItems], s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = base + i < n ? a[base + i] : 0;
        s += v[i];
    }
    uint32_t tot;
    uint32_t ex = block_excl_scan_u32(s, wsum, tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) a[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// exclusive scan of the block totals (one CTA, any length)
__global__ void __launch_bounds__(kScanThreads) k_scan_parts(uint32_t *part, int64_t n)
{
    __shared__ uint32_t wsum[32];
    uint32_t carry = 0;
    for (int64_t base = 0; base < n; base += kScanThreads) {
        int64_t q = base + threadIdx.x;
        uint32_t x = q < n ? part[q] : 0, tot;
        uint32_t ex = block_excl_scan_u32(x, wsum, tot);
        if (q < n) part[q] = ex + carry;
        carry += tot;
    }
}

constexpr size_t kScatterStage = (size_t)kRadixTile * (sizeof(uint64_t) + sizeof(uint32_t));

// One tile: rank every key within its digit (warp match, then a prefix over
// warps), stage the tile in shared memory in digit order, and write it out
// run by run, so consecutive threads store consecutive addresses of a digit's
// destination range.  Tiles of 2,048 keys and four resident CTAs per SM (64
// registers): a disk's tiles spread over the SMs in one wave with little
// imbalance between SMs.
__global__ void __launch_bounds__(kRadixThreads, 4) k_radix_scatter(const DiskDev *disks, const int32_t *tile_disk,
                                                                 const uint64_t *ksrc, const uint32_t *vsrc,
                                                                 uint64_t *kdst, uint32_t *vdst, int shift,
                                                                 const uint32_t *hist, const uint32_t *part)
{
    __shared__ uint32_t wcnt[kRadixThreads / 32][kRadixBins];
    __shared__ uint32_t toff[kRadixBins], loff[kRadixBins], wsum[32];
    extern __shared__ __align__(16) unsigned char stage_raw[];  // kScatterStage bytes
    uint64_t *skey = reinterpret_cast<uint64_t *>(stage_raw);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + kRadixTile);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t t = blockIdx.x;
    const DiskDev D = disks[tile_disk[t]];
    int64_t start = D.p_off + (t - D.t_off) * kRadixTile;
    int64_t end = min(start + kRadixTile, D.p_off + D.n0);
    const int nvalid = (int)(end - start);
    {
        int64_t hi = hidx(D, t, threadIdx.x);
        toff[threadIdx.x] = hist[hi] + part[hi / kScanBlock];
    }
    for (int q = threadIdx.x; q < (kRadixThreads / 32) * kRadixBins; q += kRadixThreads) (&wcnt[0][0])[q] = 0;
    // every load of the tile issued before the first use
    uint64_t kk[kRadixItems];
    uint32_t vv[kRadixItems], rk[kRadixItems];
    int dg[kRadixItems];
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        const int lq = w * (32 * kRadixItems) + it * 32 + lane;
        const bool ok = lq < nvalid;
        kk[it] = ok ? ksrc[start + lq] : 0;
        vv[it] = ok ? vsrc[start + lq] : 0;
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        const int lq = w * (32 * kRadixItems) + it * 32 + lane;
        const bool ok = lq < nvalid;
        const int digit = (int)((kk[it] >> shift) & 255);
        dg[it] = ok ? digit : 256;
        const unsigned peers = digit_peers(digit, ok);
        const int leader = ok ? __ffs(peers) - 1 : lane;
        uint32_t old = 0;
        if (lane == leader && ok) {
            old = wcnt[w][digit];
            wcnt[w][digit] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        rk[it] = old + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps within it, and the tile's count of it
    uint32_t cnt;
    {
        const int b = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int ww = 0; ww < kRadixThreads / 32; ++ww) {
            uint32_t c = wcnt[ww][b];
            wcnt[ww][b] = run;
            run += c;
        }
        cnt = run;
    }
    // exclusive scan of the digit counts: the digit's first slot in the staged tile
    {
        uint32_t v = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) wsum[w] = v;
        __syncthreads();
        uint32_t off = 0;
#pragma unroll
        for (int ww = 0; ww < kRadixThreads / 32; ++ww) off += ww < w ? wsum[ww] : 0u;
        loff[threadIdx.x] = off + v - cnt;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRadixItems; ++it) {
        if (dg[it] < 256) {
            const uint32_t pos = loff[dg[it]] + wcnt[w][dg[it]] + rk[it];
            skey[pos] = kk[it];
            sval[pos] = vv[it];
        }
    }
    __syncthreads();
    // write out in staged order: position p of digit d goes to toff[d] + (p - loff[d])
    for (int p = threadIdx.x; p < nvalid; p += kRadixThreads) {
        const uint64_t k = skey[p];
        const int d = (int)((k >> shift) & 255);
        const uint32_t g = toff[d] + ((uint32_t)p - loff[d]);
        kdst[g] = k;
        vdst[g] = sval[p];
    }
}

// a zone element in shared memory: (z key lo, z key hi, id, source slot)
__device__ __forceinline__ uint64_t el_key(const uint4 &e) { return ((uint64_t)e.y << 32) | e.x; }
__device__ __forceinline__ bool zless(const uint4 &a, const uint4 &b)
{
    const uint64_t ka = el_key(a), kb = el_key(b);
    return ka < kb || (ka == kb && a.z < b.z);
}

// Bitonic sort of el[0, n) in shared memory by (key, id) (zless); every
// compare ascending, i < j, j < n (32-bit indices; strides are powers of two,
// so / and % are shifts).  Pair p of a stage touches positions inside an
// aligned block of 2^(lt+1); with nw warps each warp owns the aligned chunk of
// 2^lwb positions whose pairs are p in [w 2^(lwb-1), (w+1) 2^(lwb-1)), so the
// stages with lt < lwb need only the warp's own synchronisation.  blockDim.x
// is a power-of-two multiple of 32; every thread of the block calls it.
__device__ void block_bitonic(uint4 *el, int n)
{
    int lg = 0;
    while ((1 << lg) < n) ++lg;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int lgw = 31 - __clz((int)(blockDim.x >> 5));
    const int lwb = lg - lgw;
    auto stage = [&](int ls, int lt, int p) {
        const int stride = 1 << lt;
        int i, j;
        if (lt == ls - 1) {  // first step of a merge: mirror compare
            const int blk = p >> lt, off = p & (stride - 1);
            i = (blk << ls) + off;
            j = (blk << ls) + (1 << ls) - 1 - off;
        } else {
            i = ((p >> lt) << (lt + 1)) + (p & (stride - 1));
            j = i + stride;
        }
        if (j < n) {
            const uint4 a = el[i], b = el[j];
            if (zless(b, a)) {
                el[i] = b;
                el[j] = a;
            }
        }
    };
    for (int ls = 1; ls <= lg; ++ls) {         // merge size 2^ls
        for (int lt = ls - 1; lt >= 0; --lt) {  // compare stride 2^lt
            if (lt >= lwb) {  // pairs span warps
                for (int p = threadIdx.x; p < (1 << (lg - 1)); p += blockDim.x) stage(ls, lt, p);
                __syncthreads();
            } else {
                const int p1 = (w + 1) << (lwb - 1);
                for (int p = (w << (lwb - 1)) + lane; p < p1; p += 32) stage(ls, lt, p);
                __syncwarp();
            }
        }
        // a merge that ended in warp-local stages is followed by a block barrier
        // when the next merge opens with a cross-warp stage, and at the end
        if (lwb >= 1 && (ls >= lwb || ls == lg)) __syncthreads();
    }
}

constexpr int kZoneThreads = 512;  // two zones per SM

// ---- the r sort's fix-up --------------------------------------------------------
// The radix passes sort the r keys by their upper 32 bits only (sign, exponent
// and 20 mantissa bits), stably, so positions with equal upper words hold their
// keys in id order.  Each such run is then put in (full key, id) order: runs of
// up to kRunShort by the thread at their start (insertion sort, stable, in
// place), longer ones are listed for k_rfix_long.  Runs are disjoint and a
// permutation inside a run leaves its upper words unchanged, so the threads'
// run tests do not race with the sorts.  The removed particles' run (+inf) is
// already in order.
constexpr int kRunShort = kRunShortMax;

__global__ void k_rfix(const DiskDev *disks, const int32_t *slot_disk, int64_t N, uint64_t *key, uint32_t *val,
                       int64_t *longs, int32_t *n_long, int64_t *n_alive, int32_t *status)
{
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const int d = slot_disk[s];
    const DiskDev D = disks[d];
    const int64_t end = D.p_off + D.n0;
    // the disk's live count: the last finite key's position + 1 (removed particles, +inf, sort last; a run
    // never mixes finite and +inf keys, so the fix-up below does not move this boundary)
    const bool fin = key[s] < kInfKey;
    if (fin && (s + 1 == end || !(key[s + 1] < kInfKey))) n_alive[d] = s + 1 - D.p_off;
    if (!fin && s == D.p_off) {
        n_alive[d] = 0;
        atomicOr(status, kStEmpty);
    }
    const uint32_t hi = (uint32_t)(key[s] >> 32);
    if (hi == (uint32_t)(kInfKey >> 32)) return;
    if (s + 1 >= end || (uint32_t)(key[s + 1] >> 32) != hi) return;
    if (s > D.p_off && (uint32_t)(key[s - 1] >> 32) == hi) return;  // not the run's first position
    int64_t e = s + 1;
    while (e + 1 < end && e - s < kRunShort && (uint32_t)(key[e + 1] >> 32) == hi) ++e;
    if (e - s + 1 > kRunShort) {
        longs[atomicAdd(n_long, 1)] = s;  // (at most N / (kRunShort + 1) of them)
        return;
    }
    for (int64_t i = s + 1; i <= e; ++i) {
        const uint64_t k = key[i];
        const uint32_t v = val[i];
        int64_t j = i - 1;
        while (j >= s && key[j] > k) {
            key[j + 1] = key[j];
            val[j + 1] = val[j];
            --j;
        }
        key[j + 1] = k;
        val[j + 1] = v;
    }
}

// the listed long runs, one CTA each (taken by an atomic ticket): the run's
// length, nothing to do when all its full keys are equal, else a bitonic sort
// by (key, id) -- in shared memory up to kZoneCap positions, in place in
// global memory beyond (inputs that put more than 14,336 particles within a
// relative 2^-20 of one radius and not all at the same one)
__global__ void __launch_bounds__(kZoneThreads) k_rfix_long(const DiskDev *disks, const int32_t *slot_disk,
                                                           uint64_t *key, uint32_t *val, const uint32_t *id0,
                                                           const int64_t *longs, const int32_t *n_long,
                                                           int32_t *ticket)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint4 *el = reinterpret_cast<uint4 *>(smem_raw);
    __shared__ int64_t s_sh;
    __shared__ unsigned long long len_sh;
    __shared__ int diff_sh;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int t = atomicAdd(ticket, 1);
            s_sh = t < *n_long ? longs[t] : -1;
        }
        __syncthreads();
        const int64_t s = s_sh;
        if (s < 0) return;
        const DiskDev D = disks[slot_disk[s]];
        const int64_t end = D.p_off + D.n0;
        const uint64_t k0 = key[s];
        const uint32_t hi = (uint32_t)(k0 >> 32);
        if (threadIdx.x == 0) {
            len_sh = (unsigned long long)(end - s);
            diff_sh = 0;
        }
        __syncthreads();
        for (int64_t q = s + 1 + threadIdx.x; q < end; q += blockDim.x)
            if ((uint32_t)(key[q] >> 32) != hi) {
                atomicMin(&len_sh, (unsigned long long)(q - s));
                break;
            }
        __syncthreads();
        const int64_t L = (int64_t)len_sh;
        for (int64_t q = threadIdx.x; q < L; q += blockDim.x)
            if (key[s + q] != k0) diff_sh = 1;
        __syncthreads();
        if (!diff_sh) continue;  // equal keys: already in id order
        if (L <= kZoneCap) {
            for (int64_t q = threadIdx.x; q < L; q += blockDim.x) {
                const uint64_t k = key[s + q];
                const uint32_t v = val[s + q];  // (a source slot outside the disk: ids were not a permutation)
                el[q] = make_uint4((uint32_t)k, (uint32_t)(k >> 32), id0[D.p_off + (v < D.n0 ? v : 0)], v);
            }
            __syncthreads();
            block_bitonic(el, (int)L);
            __syncthreads();
            for (int64_t q = threadIdx.x; q < L; q += blockDim.x) {
                key[s + q] = el_key(el[q]);
                val[s + q] = el[q].w;
            }
        } else {
            int lg = 0;
            while ((1LL << lg) < L) ++lg;
            auto idk = [&](int64_t q) {
                const uint32_t v = val[s + q];
                return id0[D.p_off + (v < D.n0 ? v : 0)];
            };
            for (int ls = 1; ls <= lg; ++ls)
                for (int lt = ls - 1; lt >= 0; --lt) {
                    const int64_t stride = 1LL << lt;
                    for (int64_t p = threadIdx.x; p < (1LL << (lg - 1)); p += blockDim.x) {
                        int64_t i, j;
                        if (lt == ls - 1) {
                            const int64_t blk = p >> lt, off = p & (stride - 1);
                            i = (blk << ls) + off;
                            j = (blk << ls) + (1LL << ls) - 1 - off;
                        } else {
                            i = ((p >> lt) << (lt + 1)) + (p & (stride - 1));
                            j = i + stride;
                        }
                        if (j < L) {
                            const uint64_t ka = key[s + i], kb = key[s + j];
                            if (kb < ka || (kb == ka && idk(j) < idk(i))) {
                                const uint32_t va = val[s + i];
                                key[s + i] = kb;
                                key[s + j] = ka;
                                val[s + i] = val[s + j];
                                val[s + j] = va;
                            }
                        }
                    }
                    __syncthreads();
                }
        }
    }
}

constexpr int kZoneItems = 8;      // radix path: elements per lane, zones up to 16 x 32 x 8 = 4,096
constexpr int kZoneRadixMax = (kZoneThreads / 32) * 32 * kZoneItems;
constexpr int kTieRun = 64;  // longest run of equal heights the radix path orders by id in place

// digit of element e in pass p: the first id_passes take the id's bytes, the
// next ones the z key's from byte zb0 up (least significant first)
__device__ __forceinline__ int zdigit(const uint4 &e, int p, int id_passes, int zb0)
{
    return p < id_passes ? (int)((e.z >> (8 * p)) & 255u)
                         : (int)((el_key(e) >> (8 * (zb0 + p - id_passes))) & 255u);
}

// Stable LSD radix sort of a[0, n): id_passes passes over the id's bytes,
// then the z key's bytes from byte zb0 up (zb0 = 0 and all id bytes: by
// (z key, id); zb0 = 4 and no id pass: by the key's upper word, stably).
// Each pass ranks a warp's items by ballots (item order it, lane within a
// warp; warps in order), offsets every (warp, digit) run and scatters into the
// other buffer.
// Returns the buffer that holds the result.  n <= kZoneRadixMax.  The
// counters live in the radix path's own part of the dynamic shared memory
// (kZoneRadixScratch bytes after the two buffers), so the bitonic path keeps
// the whole allocation for its one buffer.
constexpr size_t kZoneRadixScratch = sizeof(uint16_t) * (kZoneThreads / 32) * kRadixBins + sizeof(uint32_t) * (kRadixBins + 8);
__device__ uint4 *zone_radix(uint4 *a, uint4 *b, int n, int id_passes, int zb0, unsigned char *scratch)
{
    uint16_t(*wcnt)[kRadixBins] = reinterpret_cast<uint16_t(*)[kRadixBins]>(scratch);
    uint32_t *doff = reinterpret_cast<uint32_t *>(scratch + sizeof(uint16_t) * (kZoneThreads / 32) * kRadixBins);
    uint32_t *wsum = doff + kRadixBins;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int per_warp = ((n + nw - 1) / nw + 31) & ~31;
    const unsigned below = (1u << lane) - 1u;
    for (int p = 0; p < id_passes + 8 - zb0; ++p) {
        for (int q = threadIdx.x; q < nw * kRadixBins; q += blockDim.x) (&wcnt[0][0])[q] = 0;
        __syncthreads();
        uint32_t dr[kZoneItems];  // digit | rank << 9
#pragma unroll
        for (int it = 0; it < kZoneItems; ++it) {
            const int q = w * per_warp + it * 32 + lane;
            const bool ok = it * 32 < per_warp && q < n;
            const int d = ok ? zdigit(a[q], p, id_passes, zb0) : 256;
            const unsigned peers = digit_peers(d & 255, ok);
            const int leader = ok ? __ffs(peers) - 1 : lane;
            uint32_t old = 0;
            if (lane == leader && ok) {
                old = wcnt[w][d];
                wcnt[w][d] = (uint16_t)(old + __popc(peers));
            }
            old = __shfl_sync(0xffffffffu, old, leader);
            dr[it] = (uint32_t)d | ((old + __popc(peers & below)) << 9);
            __syncwarp();
        }
        __syncthreads();
        // per digit: the warps' offsets within it, then the digits' offsets
        if (threadIdx.x < kRadixBins) {
            const int d = threadIdx.x;
            uint32_t tot = 0;
            for (int ww = 0; ww < nw; ++ww) {
                const uint32_t c = wcnt[ww][d];
                wcnt[ww][d] = (uint16_t)tot;
                tot += c;
            }
            uint32_t v = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            if (lane == 31) wsum[w] = v;
            doff[d] = v - tot;  // exclusive within the warp; warp offsets added below
        }
        __syncthreads();
        if (threadIdx.x < kRadixBins) {
            uint32_t o = 0;
            for (int ww = 0; ww < w; ++ww) o += wsum[ww];
            doff[threadIdx.x] += o;
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < kZoneItems; ++it) {
            const int q = w * per_warp + it * 32 + lane;
            const int d = (int)(dr[it] & 511u);
            if (d < 256) b[doff[d] + wcnt[w][d] + (dr[it] >> 9)] = a[q];
        }
        __syncthreads();
        uint4 *t = a;
        a = b;
        b = t;
    }
    return a;
}

struct ZoneArgs {
    const mcd_disk_params *params;
    const DiskDev *disks;
    const int32_t *zone_disk;
    const int64_t *n_alive;
    const uint64_t *rkey;  // sorted r keys
    const uint32_t *rsrc;  // disk-local source slot of each sorted position
    const double *m0, *M0, *r0, *z0;
    const uint32_t *id0;
    double *m1, *M1, *r1, *z1;
    uint32_t *id1;
    const double *q0;  // the tracer column, or null
    double *q1;
    int64_t *cell_start;
    int32_t *cell_n;
    double *cell_b, *cell_V;
    int32_t *status;
    int64_t zcap;   // elements per buffer (the largest zone)
    int radix;      // 1: radix sort in two buffers (zcap <= kZoneRadixMax); 0: bitonic in one
    int id_passes;  // radix path: bytes of the largest id
    const GasKnot *gas_knots;  // gas tables (a single particle's cell spans H_g)
    const int32_t *gas_n;
};

__global__ void __launch_bounds__(kZoneThreads, 2) k_zone(ZoneArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int zg = blockIdx.x;
    const int d = A.zone_disk[zg];
    const DiskDev D = A.disks[d];
    const int64_t k = zg - D.z_off;
    const int64_t Na = A.n_alive[d];
    const int64_t nr = D.n_r, nz = D.n_z;
    const int64_t base = Na / nr, rem = Na % nr;
    const int64_t nk = base + (k < rem ? 1 : 0);
    const int64_t zs = k * base + (k < rem ? k : rem);
    const int64_t c0 = D.c_off + k * nz;
    uint4 *el = reinterpret_cast<uint4 *>(smem_raw);
    const uint64_t *rk = A.rkey + D.p_off;

    // (1) load this zone's (z, id, source) triples
    auto load = [&]() {
        for (int64_t q = threadIdx.x; q < nk; q += blockDim.x) {
            uint32_t src = A.rsrc[D.p_off + zs + q];
            if ((int64_t)src >= D.n0) {  // ids were not a permutation
                atomicOr(A.status, kStBadCell);
                src = 0;
            }
            int64_t gs = D.p_off + src;
            double zz = A.z0[gs];
            if (isnan(zz)) {
                atomicOr(A.status, kStNaN);
                zz = INFINITY;
            }
            const uint64_t kz = order_key(zz);
            el[q] = make_uint4((uint32_t)kz, (uint32_t)(kz >> 32), A.id0[gs], src);
        }
        __syncthreads();
    };
    load();
    // (2) sort by (z, id)
    if (A.radix) {
        // The upper four bytes of the z key alone (sign, exponent and 20
        // mantissa bits): a stable sort by them, then each run of equal upper
        // words is put in (full z key, id) order by the thread at its start
        // (runs are disjoint; inside a run only the lower words and ids differ).
        // Such runs are rare for continuous heights and short; a run longer
        // than kTieRun redoes the sort with the id passes and all eight z passes.
        uint4 *const base = el;
        unsigned char *const scratch = reinterpret_cast<unsigned char *>(base + 2 * A.zcap);
        el = zone_radix(base, base + A.zcap, (int)nk, 0, 4, scratch);
        __shared__ int long_run;
        if (threadIdx.x == 0) long_run = 0;
        __syncthreads();
        const int n32 = (int)nk;
        for (int q = threadIdx.x; q + 1 < n32; q += blockDim.x) {
            const uint32_t kq = el[q].y;
            if (el[q + 1].y != kq || (q > 0 && el[q - 1].y == kq)) continue;
            int e = q + 1;
            while (e + 1 < n32 && el[e + 1].y == kq) ++e;
            if (e - q + 1 > kTieRun) {
                long_run = 1;
                continue;
            }
            for (int i = q + 1; i <= e; ++i) {  // insertion sort of el[q..e] by (z key, id)
                const uint4 x = el[i];
                int j = i - 1;
                while (j >= q && zless(x, el[j])) {
                    el[j + 1] = el[j];
                    --j;
                }
                el[j + 1] = x;
            }
        }
        __syncthreads();
        if (long_run) {
            el = base;
            load();
            el = zone_radix(base, base + A.zcap, (int)nk, A.id_passes, 0, scratch);
        }
    } else {
        block_bitonic(el, (int)nk);
    }
    // (3) bounds: radial edges of the zone, then one thread per cell
    __shared__ double rlo_s, rhi_s;
    if (threadIdx.x == 0) {
        double rlo = 0.0, rhi = 0.0;
        if (nk > 0) {
            double rf = key_value(rk[zs]), rl = key_value(rk[zs + nk - 1]);
            int64_t nonempty = Na < nr ? Na : nr;
            if (Na == 1) {
                double H = gas_at<double>(A.params[d], gas_tab(A.gas_knots, A.gas_n, d), rf, 0.0).H;
                rlo = __dsub_rn(rf, __dmul_rn(0.5, H));
                rhi = __dadd_rn(rf, __dmul_rn(0.5, H));
            } else {
                if (k == 0)
                    rlo = __dsub_rn(rf, __dmul_rn(__dsub_rn(key_value(rk[1]), rf), 0.5));
                else
                    rlo = __dmul_rn(__dadd_rn(key_value(rk[zs - 1]), rf), 0.5);
                if (k + 1 < nonempty)
                    rhi = __dmul_rn(__dadd_rn(rl, key_value(rk[zs + nk])), 0.5);
                else
                    rhi = __dadd_rn(rl, __dmul_rn(__dsub_rn(rl, key_value(rk[Na - 2])), 0.5));
            }
        }
        rlo_s = rlo;
        rhi_s = rhi;
    }
    __syncthreads();
    const double rlo = rlo_s, rhi = rhi_s;
    const double rcen = __dmul_rn(__dadd_rn(rlo, rhi), 0.5);
    const int64_t zb = nk / nz, zr = nk % nz, nonempty_z = nk < nz ? nk : nz;
    for (int64_t c = threadIdx.x; c < nz; c += blockDim.x) {
        int64_t nc = zb + (c < zr ? 1 : 0), cs = c * zb + (c < zr ? c : zr);
        double zlo = 0.0, zhi = 0.0;
        if (nc > 0) {
            double zf = key_value(el_key(el[cs])), zl = key_value(el_key(el[cs + nc - 1]));
            if (nk == 1) {
                double H = gas_at<double>(A.params[d], gas_tab(A.gas_knots, A.gas_n, d), rcen, 0.0).H;
                zlo = __dsub_rn(zf, __dmul_rn(0.5, H));
                zhi = __dadd_rn(zf, __dmul_rn(0.5, H));
            } else {
                if (c == 0)
                    zlo = __dsub_rn(zf, __dmul_rn(__dsub_rn(key_value(el_key(el[1])), zf), 0.5));
                else
                    zlo = __dmul_rn(__dadd_rn(key_value(el_key(el[cs - 1])), zf), 0.5);
                if (c + 1 < nonempty_z)
                    zhi = __dmul_rn(__dadd_rn(zl, key_value(el_key(el[cs + nc]))), 0.5);
                else
                    zhi = __dadd_rn(zl, __dmul_rn(__dsub_rn(zl, key_value(el_key(el[nk - 2]))), 0.5));
            }
        }
        double b0 = nc > 0 ? rlo : 0.0, b1 = nc > 0 ? rhi : 0.0;
        double *b = A.cell_b + 6 * (c0 + c);
        b[0] = b0;
        b[1] = b1;
        b[2] = zlo;
        b[3] = zhi;
        b[4] = __dmul_rn(__dadd_rn(b0, b1), 0.5);
        b[5] = __dmul_rn(__dadd_rn(zlo, zhi), 0.5);
        double Ar = __dsub_rn(__dmul_rn(b1, b1), __dmul_rn(b0, b0));
        A.cell_V[c0 + c] = __dmul_rn(__dmul_rn(kPI, Ar), __dsub_rn(zhi, zlo));
        A.cell_start[c0 + c] = D.p_off + zs + cs;
        A.cell_n[c0 + c] = (int32_t)nc;
    }
    // (4) gather the particle columns into cell order
#pragma unroll 4
    for (int64_t q = threadIdx.x; q < nk; q += blockDim.x) {
        const uint4 e = el[q];
        int64_t gs = D.p_off + e.w, gd = D.p_off + zs + q;
        A.m1[gd] = A.m0[gs];
        A.M1[gd] = A.M0[gs];
        A.r1[gd] = A.r0[gs];
        A.z1[gd] = key_value(el_key(e));
        A.id1[gd] = e.z;
        if (A.q0) A.q1[gd] = A.q0[gs];
    }
}

// removed particles: sorted positions [n_alive, n0) of each disk, in id order
__global__ void k_dead_tail(const DiskDev *disks, const int32_t *slot_disk, int64_t N, const int64_t *n_alive,
                            const uint32_t *rsrc, const double *m0, const double *M0, const double *r0,
                            const double *z0, const uint32_t *id0, double *m1, double *M1, double *r1, double *z1,
                            uint32_t *id1, const double *q0, double *q1)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= N) return;
    int d = slot_disk[s];
    const DiskDev D = disks[d];
    if (s - D.p_off < n_alive[d]) return;
    int64_t gs = D.p_off + ((int64_t)rsrc[s] < D.n0 ? rsrc[s] : 0);
    m1[s] = m0[gs];
    M1[s] = M0[gs];
    r1[s] = r0[gs];
    z1[s] = z0[gs];
    id1[s] = id0[gs];
    if (q0) q1[s] = q0[gs];
}

// the zone sort: the largest zone's size, the path (radix when the zone fits
// its item count; both paths hold 16-byte elements, the radix path twice) and
// the dynamic shared memory it takes
struct ZonePlan {
    int64_t zcap;
    int radix, id_passes;
    size_t smem;
};
static ZonePlan zone_plan(const mcd_ctx *c)
{
    ZonePlan z{c->zone_max, 0, 0, 0};
    z.radix = z.zcap <= kZoneRadixMax;
    for (int64_t idmax = c->n0_max - 1; idmax > 0; idmax >>= 8) ++z.id_passes;
    z.smem = (size_t)z.zcap * sizeof(uint4) * (z.radix ? 2 : 1) + (z.radix ? kZoneRadixScratch : 0);
    return z;
}

// The zone sort's shared-memory limit is a property of the kernel, shared by
// every context and caller in the process: it is set to what the largest
// zone of either path takes, never to one caller's need, so that no later
// set-up lowers it below what another context launches with.
constexpr size_t kZoneSmemRadixMax = (size_t)kZoneRadixMax * sizeof(uint4) * 2 + kZoneRadixScratch;
constexpr size_t kZoneSmemBitonicMax = (size_t)kZoneCap * sizeof(uint4);
constexpr size_t kZoneSmemMax = kZoneSmemRadixMax > kZoneSmemBitonicMax ? kZoneSmemRadixMax : kZoneSmemBitonicMax;

cudaError_t prepare_zone(mcd_ctx *c)
{
    cudaError_t e = cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScatterStage);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rfix_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kZoneSmemBitonicMax);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&c->n_sm_regrid, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_zone, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kZoneSmemMax);
}

cudaError_t launch_regrid(mcd_ctx *c)
{
    if (c->N == 0) return cudaSuccess;
    cudaStream_t st = c->stream;
    const int b = c->cur, nb = 1 - c->cur;
    unsigned gN = (unsigned)((c->N + 255) / 256);
    k_regrid_keys<<<gN, 256, 0, st>>>(c->d_disks, c->slot_disk, c->N, c->r[b], c->z[b], c->id[b], c->key[0],
                                      c->val[0], c->status);
    const int64_t H = 256 * c->n_tiles;
    const unsigned nsb = (unsigned)((H + kScanBlock - 1) / kScanBlock);
    // the upper four bytes of the keys (an even number of passes: the result is back in buffer 0)
    for (int pass = kRadixPasses - kRadixUpperPasses; pass < kRadixPasses; ++pass) {
        const int shift = 8 * pass, src = pass & 1, dst = src ^ 1;
        k_radix_hist<<<(unsigned)c->n_tiles, kRadixThreads, 0, st>>>(c->d_disks, c->tile_disk, c->key[src], shift,
                                                                     c->hist);
        k_scan_blocks<<<nsb, kScanThreads, 0, st>>>(c->hist, H, c->scan_part);
        k_scan_parts<<<1, kScanThreads, 0, st>>>(c->scan_part, nsb);
        k_radix_scatter<<<(unsigned)c->n_tiles, kRadixThreads, kScatterStage, st>>>(
            c->d_disks, c->tile_disk, c->key[src], c->val[src], c->key[dst], c->val[dst], shift, c->hist,
            c->scan_part);
    }
    // runs of equal upper words into (key, id) order
    cudaError_t e = cudaMemsetAsync(c->rfix_count, 0, 2 * sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    k_rfix<<<gN, 256, 0, st>>>(c->d_disks, c->slot_disk, c->N, c->key[0], c->val[0], c->rfix_longs, c->rfix_count,
                               c->n_alive, c->status);
    k_rfix_long<<<(unsigned)std::max(1, std::min(c->n_sm_regrid, 1024)), kZoneThreads, kZoneSmemBitonicMax, st>>>(
        c->d_disks, c->slot_disk, c->key[0], c->val[0], c->id[b], c->rfix_longs, c->rfix_count, c->rfix_count + 1);
    ZoneArgs A;
    A.params = c->d_params;
    A.disks = c->d_disks;
    A.zone_disk = c->zone_disk;
    A.n_alive = c->n_alive;
    A.rkey = c->key[0];
    A.rsrc = c->val[0];
    A.m0 = c->m[b]; A.M0 = c->M[b]; A.r0 = c->r[b]; A.z0 = c->z[b]; A.id0 = c->id[b];
    A.m1 = c->m[nb]; A.M1 = c->M[nb]; A.r1 = c->r[nb]; A.z1 = c->z[nb]; A.id1 = c->id[nb];
    A.q0 = c->tracer ? c->q[b] : nullptr;
    A.q1 = c->tracer ? c->q[nb] : nullptr;
    A.cell_start = c->cell_start;
    A.cell_n = c->cell_n;
    A.cell_b = c->cell_b;
    A.cell_V = c->cell_V;
    A.status = c->status;
    const ZonePlan zp = zone_plan(c);
    A.zcap = zp.zcap;
    A.radix = zp.radix;
    A.id_passes = zp.id_passes;
    A.gas_knots = c->gas_knots;
    A.gas_n = c->gas_n;
    k_zone<<<(unsigned)c->Z, kZoneThreads, zp.smem, st>>>(A);
    k_dead_tail<<<gN, 256, 0, st>>>(c->d_disks, c->slot_disk, c->N, c->n_alive, c->val[0], c->m[b], c->M[b], c->r[b],
                                    c->z[b], c->id[b], c->m[nb], c->M[nb], c->r[nb], c->z[nb], c->id[nb],
                                    c->tracer ? c->q[b] : nullptr, c->tracer ? c->q[nb] : nullptr);
    c->launches += 5 + 4 * kRadixUpperPasses;
    return cudaGetLastError();
}

}  // namespace mcd
