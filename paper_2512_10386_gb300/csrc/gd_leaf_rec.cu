// gd_leaf_rec.cu -- the instantiation of the fused per-leaf kernel that also
// writes the debug and training tensors (denoise_run_debug, training mode).
#include "gd_leaf_kernel.cuh"

namespace gd {

int launch_leaf_rec(const LeafArgs &a, int num_sms, cudaStream_t st) { return launch_kmax<true, false>(a, num_sms, st); }

}  // namespace gd
