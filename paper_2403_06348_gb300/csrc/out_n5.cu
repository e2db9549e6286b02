// Output-oriented MTTKRP and Phi kernels specialised for 5 modes.
#include "outorder.cuh"

namespace alto {
template cudaError_t launch_mttkrp_out_nt<5>(const MttkrpArgs &, int, bool, size_t, int, cudaStream_t);
template cudaError_t launch_phi_out_nt<5>(const MttkrpArgs &, bool, size_t, int, cudaStream_t);
}  // namespace alto
