// FP64 residual, FAS right-hand side, halo dump and transposed ghost fill (instantiations).
#include "kernels_fused.cuh"

namespace mrp {

template void launch_residual_fused<double>(double*, const double*, const double*, const double*, LevelView, LevelView,
                                            int, int, double, int, cudaStream_t);
template void launch_fas_fused<double>(double*, double*, const double*, const double*, LevelView, LevelView, int, int,
                                       double, int, cudaStream_t);
template void launch_halo_dump<double>(double*, const double*, LevelView, LevelView, int, int, cudaStream_t);
template void launch_ghost_T_fused<double>(double*, double*, LevelView, LevelView, int, int, cudaStream_t);

size_t fused_smem_bytes(int n, int M, int el) {
    return el == 8 ? fused_smem<double>(n, M + 2) : fused_smem<float>(n, M + 2);
}

}  // namespace mrp
