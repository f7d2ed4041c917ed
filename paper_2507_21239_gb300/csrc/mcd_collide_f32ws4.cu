// mcd_collide_f32ws4.cu -- the mixed-precision collide variants with a control warp
// (mcd_collide_ws.cuh) for cells of up to 32 PL swarms, PL = 4 and 7: every
// dv-matrix store, with and without the fragmentation ramp and the tracer,
// in a translation unit of their own so that the build compiles them in
// parallel.
#include "mcd_collide_ws.cuh"

namespace mcd {

template cudaError_t collide_ws_variant<4>(int, int, bool, bool, unsigned, int, size_t, cudaStream_t,
                                            const CollideArgs *, int *);
template cudaError_t collide_ws_variant<7>(int, int, bool, bool, unsigned, int, size_t, cudaStream_t,
                                            const CollideArgs *, int *);

}  // namespace mcd
