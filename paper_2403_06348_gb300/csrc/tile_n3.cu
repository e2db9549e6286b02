// In-tile output-oriented MTTKRP kernels specialised for 3 modes.
#include "tile.cuh"

namespace alto {
template cudaError_t launch_mttkrp_tile_nt<3>(const MttkrpArgs &, int, bool, bool, int, cudaStream_t);
}  // namespace alto
