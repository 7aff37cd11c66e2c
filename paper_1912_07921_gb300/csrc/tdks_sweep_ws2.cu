// Warp-specialised TMA sweep, tile shape 2 (see WsShape in tdks_tma.cuh), compiled on its
// own so that the shapes build in parallel.
#include "tdks_tma.cuh"

namespace tdks {
template cudaError_t launch_ws_shape<2>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                          cudaStream_t);
template cudaError_t launch_ws_batch_shape<2>(int, int, int, const BatchSweepArgs &, cudaStream_t);
}  // namespace tdks
