// mcd_collide_f32s2.cu -- the mixed-precision collide variants with 2 swarms per thread
// (every dv-matrix store, with and without the fragmentation ramp and the
// tracer), in a translation unit of their own so that the build compiles the
// variants in parallel.
#include "mcd_collide.cuh"

namespace mcd {

template <>
cudaError_t collide_variant<float, 2, false>(int op, int store, bool ramp, bool tracer, unsigned grid, int nthr,
                                        size_t smem, cudaStream_t st, const CollideArgs *A, int *out)
{
    switch (store) {
    case 0: return collide_variant_store<float, 2, 0, false>(op, ramp, tracer, grid, nthr, smem, st, A, out);
    case 1: return collide_variant_store<float, 2, 1, false>(op, ramp, tracer, grid, nthr, smem, st, A, out);
    case 2: return collide_variant_store<float, 2, 2, false>(op, ramp, tracer, grid, nthr, smem, st, A, out);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace mcd
