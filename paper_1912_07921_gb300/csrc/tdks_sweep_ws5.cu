// Warp-specialised TMA sweep, tile shape 5 (complex64 with one complex value per thread
// vector; see WsShape in tdks_tma.cuh), compiled on its own so that the shapes build in
// parallel.  Its complex128 and periodic-cell launches use shape 2, compiled elsewhere.
#include "tdks_tma.cuh"

namespace tdks {
extern template cudaError_t launch_ws_shape<2>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                                 cudaStream_t);
extern template cudaError_t launch_ws_batch_shape<2>(int, int, int, const BatchSweepArgs &, cudaStream_t);
template cudaError_t launch_ws_shape<5>(int, int, int, int, const SweepMaps &, const SweepParams &, int,
                                          cudaStream_t);
template cudaError_t launch_ws_batch_shape<5>(int, int, int, const BatchSweepArgs &, cudaStream_t);
}  // namespace tdks
