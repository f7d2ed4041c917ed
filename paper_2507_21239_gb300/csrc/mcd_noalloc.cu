// mcd_noalloc.cu -- mcd_regrid_noalloc: the equal-count regrid of one disk for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another
// framework's memory pool or arena (which owns every allocation and forbids
// side allocations), real-time loops where an allocation would stall, and
// embedded users with a fixed memory budget.  This entry point takes the
// caller's input and output arrays and keeps its own scratch (sort keys and
// values, the digit histogram, the disk tables, the alive count and the status
// bits) in one file-scope device array of fixed size, so it allocates nothing,
// on the device or on the host.
//
// The array lives on every GPU that loads the library until the process
// exits.  All calls share it and it keeps the previous call's contents, so
// the status bits are cleared at the start of every call, and calls that
// overlap on the GPU (different streams, or different host threads) race on
// it: serialise them.  The first call on a device looks the array's device
// address up (host code cannot use the symbol itself, which on the host is
// only a stand-in); make that first call before any stream capture.
#include <string.h>

#include <mutex>

#include "mcd_internal.cuh"

namespace {

constexpr int64_t kNoAllocMax = MCD_NOALLOC_MAX_PARTICLES;
constexpr int64_t kTiles = (kNoAllocMax + mcd::kRadixTile - 1) / mcd::kRadixTile;
constexpr int64_t kScanParts = (256 * kTiles) / 4096 + 2;

// byte layout of the scratch array (each block 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffParams = 0;
constexpr size_t kOffDisk = align256(kOffParams + sizeof(mcd_disk_params));
constexpr size_t kOffSlot = align256(kOffDisk + sizeof(mcd::DiskDev));
constexpr size_t kOffZone = align256(kOffSlot + 4 * kNoAllocMax);
constexpr size_t kOffTile = align256(kOffZone + 4 * kNoAllocMax);
constexpr size_t kOffKey0 = align256(kOffTile + 4 * kTiles);
constexpr size_t kOffKey1 = align256(kOffKey0 + 8 * kNoAllocMax);
constexpr size_t kOffVal0 = align256(kOffKey1 + 8 * kNoAllocMax);
constexpr size_t kOffVal1 = align256(kOffVal0 + 4 * kNoAllocMax);
constexpr size_t kOffHist = align256(kOffVal1 + 4 * kNoAllocMax);
constexpr size_t kOffPart = align256(kOffHist + 4 * 256 * kTiles);
constexpr size_t kOffLongs = align256(kOffPart + 4 * kScanParts);
constexpr size_t kOffRfix = align256(kOffLongs + 8 * (kNoAllocMax / (mcd::kRunShortMax + 1) + 1));
constexpr size_t kOffAlive = align256(kOffRfix + 8);
constexpr size_t kOffStatus = align256(kOffAlive + 8);
constexpr size_t kScratchBytes = align256(kOffStatus + 4);

static __device__ __align__(256) unsigned char g_regrid_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
unsigned char *g_scratch_ptr[kMaxDevices] = {};  // per device, null until looked up

// device address of the scratch array on the current device
int scratch_address(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MCD_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return MCD_ECUDA;
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_regrid_scratch) != cudaSuccess || !p) return MCD_ECUDA;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return MCD_OK;
}

// the one disk's parameter and layout tables, passed by value (nothing is
// copied from host memory), and a clean status word
__global__ void k_noalloc_tables(mcd_disk_params p, mcd::DiskDev D, mcd_disk_params *dp, mcd::DiskDev *dd,
                                 int32_t *status)
{
    *dp = p;
    *dd = D;
    *status = 0;
}

__global__ void k_status_code(const int32_t *bits, int32_t *code)
{
    int32_t b = *bits;
    *code = (b & mcd::kStNaN) ? MCD_ENAN : (b & mcd::kStBadCell) ? MCD_EINVAL : (b & mcd::kStEmpty) ? MCD_EEMPTY : MCD_OK;
}

}  // namespace

extern "C" int mcd_regrid_noalloc(const mcd_disk_params *p, const mcd_grid *g, const double *m, const double *M,
                                  const double *r, const double *z, const uint32_t *id, double *m_out,
                                  double *M_out, double *r_out, double *z_out, uint32_t *id_out,
                                  int64_t *cell_start, int32_t *cell_n, double *bounds, double *V,
                                  int64_t *n_alive, int32_t *status, void *cuda_stream)
{
    if (!p || !g || !m || !M || !r || !z || !id || !m_out || !M_out || !r_out || !z_out || !id_out || !cell_start ||
        !cell_n || !bounds || !V || !n_alive || !status)
        return MCD_EINVAL;
    if (g->n_r <= 0 || g->n_z <= 0 || g->per_cell <= 0) return MCD_EINVAL;
    const int64_t N = (int64_t)g->n_r * g->n_z * g->per_cell;
    if (N > kNoAllocMax) return MCD_EINVAL;                     // beyond the fixed scratch
    if ((int64_t)g->n_z * g->per_cell > mcd::kZoneCap) return MCD_EINVAL;  // one zone must fit in shared memory
    if (p->kernel_mode == 0 && !(p->r_in > 0.0)) return MCD_EINVAL;
    unsigned char *s = nullptr;
    int rc = scratch_address(&s);
    if (rc != MCD_OK) return rc;

    // a context on the stack whose buffers are the caller's arrays and the
    // scratch (its host-side tables stay empty: nothing is allocated)
    mcd_ctx c;
    c.n_disks = 1;
    c.stream = (cudaStream_t)cuda_stream;
    mcd::DiskDev D;
    D.p_off = 0;
    D.n0 = N;
    D.c_off = 0;
    D.z_off = 0;
    D.t_off = 0;
    D.n_tiles = (N + mcd::kRadixTile - 1) / mcd::kRadixTile;
    D.n_r = g->n_r;
    D.n_z = g->n_z;
    c.N = N;
    c.zone_max = (int64_t)g->n_z * g->per_cell;
    c.n0_max = N;
    c.C = (int64_t)g->n_r * g->n_z;
    c.Z = g->n_r;
    c.n_tiles = D.n_tiles;
    c.n_max = g->per_cell;
    c.d_params = reinterpret_cast<mcd_disk_params *>(s + kOffParams);
    c.d_disks = reinterpret_cast<mcd::DiskDev *>(s + kOffDisk);
    c.slot_disk = reinterpret_cast<int32_t *>(s + kOffSlot);
    c.zone_disk = reinterpret_cast<int32_t *>(s + kOffZone);
    c.tile_disk = reinterpret_cast<int32_t *>(s + kOffTile);
    c.key[0] = reinterpret_cast<uint64_t *>(s + kOffKey0);
    c.key[1] = reinterpret_cast<uint64_t *>(s + kOffKey1);
    c.val[0] = reinterpret_cast<uint32_t *>(s + kOffVal0);
    c.val[1] = reinterpret_cast<uint32_t *>(s + kOffVal1);
    c.hist = reinterpret_cast<uint32_t *>(s + kOffHist);
    c.scan_part = reinterpret_cast<uint32_t *>(s + kOffPart);
    c.rfix_longs = reinterpret_cast<int64_t *>(s + kOffLongs);
    c.rfix_count = reinterpret_cast<int32_t *>(s + kOffRfix);
    c.n_alive = reinterpret_cast<int64_t *>(s + kOffAlive);
    c.status = reinterpret_cast<int32_t *>(s + kOffStatus);
    c.m[0] = const_cast<double *>(m);  // read only
    c.M[0] = const_cast<double *>(M);
    c.r[0] = const_cast<double *>(r);
    c.z[0] = const_cast<double *>(z);
    c.id[0] = const_cast<uint32_t *>(id);
    c.m[1] = m_out;
    c.M[1] = M_out;
    c.r[1] = r_out;
    c.z[1] = z_out;
    c.id[1] = id_out;
    c.cur = 0;
    c.cell_start = cell_start;
    c.cell_n = cell_n;
    c.cell_b = bounds;
    c.cell_V = V;

    // tables for one disk (all indices 0) and a clean status word
    cudaStream_t st = c.stream;
    k_noalloc_tables<<<1, 1, 0, st>>>(*p, D, c.d_params, c.d_disks, c.status);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(c.slot_disk, 0, 4 * N, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.zone_disk, 0, 4 * c.Z, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c.tile_disk, 0, 4 * c.n_tiles, st);
    if (e == cudaSuccess) e = mcd::prepare_zone(&c);
    if (e == cudaSuccess) e = mcd::launch_regrid(&c);
    if (e == cudaSuccess) e = cudaMemcpyAsync(n_alive, c.n_alive, 8, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        k_status_code<<<1, 1, 0, st>>>(c.status, status);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? MCD_OK : MCD_ECUDA;
}
