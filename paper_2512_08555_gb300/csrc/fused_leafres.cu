// FP64 leaf residual of the refinement and the stop rule.
#include "kernels_fused.cuh"

namespace mrp {

void launch_leafres_fused(float* R, const double* U, const double* F, const double* Uc, const int* blocks, int nblocks,
                          LevelView lk, LevelView lc, int n, int M, double inv_h2, unsigned long long* out, int nt,
                          cudaStream_t s) {
    if (nblocks == 0) return;
    attrs_leafres();
    const size_t sm = fused_smem<double>(n, M + 2);
    const int ct = cta_size_fixed(n, nt, true);
    if (M == 2) leafres_m<2>(R, U, F, Uc, blocks, nblocks, lk, n, inv_h2 / LW<2>::den, out, ct, sm, s);
    if (M == 4) leafres_m<4>(R, U, F, Uc, blocks, nblocks, lk, n, inv_h2 / LW<4>::den, out, ct, sm, s);
    if (M == 6) leafres_m<6>(R, U, F, Uc, blocks, nblocks, lk, n, inv_h2 / LW<6>::den, out, ct, sm, s);
}

}  // namespace mrp
