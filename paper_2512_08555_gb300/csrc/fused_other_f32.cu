// FP32 residual, FAS right-hand side, halo dump and transposed ghost fill (instantiations).
#include "kernels_fused.cuh"

namespace mrp {

template void launch_residual_fused<float>(float*, const float*, const float*, const float*, LevelView, LevelView, int,
                                           int, double, int, cudaStream_t);
template void launch_fas_fused<float>(float*, float*, const float*, const float*, LevelView, LevelView, int, int, double,
                                      int, cudaStream_t);
template void launch_halo_dump<float>(float*, const float*, LevelView, LevelView, int, int, cudaStream_t);
template void launch_ghost_T_fused<float>(float*, float*, LevelView, LevelView, int, int, cudaStream_t);

}  // namespace mrp
