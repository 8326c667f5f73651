// FP32 Gauss-Seidel sweep with the fused ghost layer (instantiations).
#include "kernels_fused.cuh"

namespace mrp {

template void launch_smooth_fused<float>(float*, const float*, const float*, const float*, LevelView, LevelView, int, int,
                                         double, int, cudaStream_t);

}  // namespace mrp
