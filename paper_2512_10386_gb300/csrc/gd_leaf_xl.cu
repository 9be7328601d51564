// gd_leaf_xl.cu -- the instantiations of the fused per-leaf kernel that run the
// phases of the cross-leaf kNN variant (voxel gate only; gate, median, score and
// selection on the cross-leaf neighbours), with and without the debug / training
// outputs.  Kept apart so that the plain path carries none of their code.
#include "gd_leaf_kernel.cuh"

namespace gd {

int launch_leaf_xl(const LeafArgs &a, int num_sms, cudaStream_t st) {
  return (a.use_dbg || a.use_train) ? launch_kmax<true, true>(a, num_sms, st) : launch_kmax<false, true>(a, num_sms, st);
}

}  // namespace gd
