// FP64 leaf residual of the refinement and the stop rule; f* = R^M f with its ghost layer (M = 2, 4).
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

void launch_rhs_fused(double* F, const double* Af, const double* Ac, const int* blocks, int nblocks, LevelView lk,
                             int n, int M, unsigned long long* fmax_out, cudaStream_t s) {
    if (nblocks == 0) return;
    static std::once_flag done[MAX_DEVICES];
    once_per_device(done, [] {
        allow(k_rhs_fused<2, 4, NC_FIXED>); allow(k_rhs_fused<2, 4, 0>);
        allow(k_rhs_fused<4, 6, NC_FIXED>); allow(k_rhs_fused<4, 6, 0>);
    });
    const size_t sm = fused_smem<double>(n, M + 2);
    if (M == 2) rhs_fused_m<2>(F, Af, Ac, blocks, nblocks, lk, n, fmax_out, sm, s);
    if (M == 4) rhs_fused_m<4>(F, Af, Ac, blocks, nblocks, lk, n, fmax_out, sm, s);
}

}  // namespace mrp
