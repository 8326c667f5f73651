// Gradient of the converged solve on the device: f-bar = S^T w, where
// u_leaf = S f is the composite solution the V-cycles of Alg. 1 converge to.
//
// S factors as f* = B f (Sec. 3.2, with f ghosts), 0 = c(f*) - K x (the
// composite leaf system: leaf rows f* - L_k u at levels >= 1, and on covered
// level-0 nodes the mismatch (h0^2 G * f0 - inject u_1) / h0^2), and
// u_leaf = E(x, f*) (level-0 leaves from the convolution).  Hence
//     f-bar = B^T (E_f^T w + c^T lambda),   K^T lambda = E_x^T w.
// K^T lambda = g is solved by FP64 refinement, lambda += M^T (g - K^T lambda),
// with M^T the transposed correction V-cycle; I - M^T K^T = (I - K M)^T has
// the spectrum of the forward cycle's error propagator, so the refinement
// contracts at the forward rate.  No state of a forward solve is needed: all
// of these maps are linear and fixed by the forest and the order.
//
// Vectors of the unknown / residual space hold [nb_k][n^3] per level k at
// offset xoff[k]: levels >= 1 use their leaf blocks, level 0 its covered
// blocks; every other entry stays zero.
#include "mrp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mrp {

static int adj_alloc(double*& p, size_t count) {
    if (cudaMalloc(&p, sizeof(double) * (count ? count : 1)) != cudaSuccess) return MRP_ERR_OOM;
    if (cudaMemset(p, 0, sizeof(double) * (count ? count : 1)) != cudaSuccess) return MRP_ERR_CUDA;
    return MRP_OK;
}

int adjoint_setup(Handle& h) {
    if (!h.adj.empty()) return MRP_OK;
    const size_t n = h.n, S = n + 2, S4 = n + 4, nn = n * n * n;
    h.adj.resize(h.L + 1);
    h.xoff.assign(h.L + 2, 0);
    int rc;
    for (int k = 0; k <= h.L; ++k) {
        const size_t nb = h.lv[k].nb;
        Handle::AdjLevel& a = h.adj[k];
        if ((rc = adj_alloc(a.Ub, nb * S * S * S))) return rc;
        if ((rc = adj_alloc(a.Fb, nb * nn))) return rc;
        if ((rc = adj_alloc(a.Rb, nb * nn))) return rc;
        if ((rc = adj_alloc(a.Hb, nb * nn))) return rc;
        if ((rc = adj_alloc(a.Rawb, nb * S4 * S4 * S4))) return rc;
        h.xoff[k + 1] = h.xoff[k] + nb * nn;
    }
    const size_t len = h.xoff[h.L + 1];
    for (double** p : {&h.lam, &h.rho, &h.gvec, &h.xb, &h.fsb, &h.wl})
        if ((rc = adj_alloc(*p, len))) return rc;
    size_t C = 0, D = 0;
    for (const Problem& p : h.pr) {
        C = std::max(C, (size_t)(p.n0[0] + 2) * (p.n0[1] + 2) * (p.n0[2] + 2));
        D = std::max(D, (size_t)p.n0[0] * p.n0[1] * p.n0[2]);
    }
    if ((rc = adj_alloc(h.cube, C))) return rc;
    if ((rc = adj_alloc(h.dense, D))) return rc;
    if ((rc = adj_alloc(h.off0b, (size_t)h.lv[0].nb * nn))) return rc;
    if (h.mixed) {
        auto alloc32 = [](float*& p, size_t count) {
            if (cudaMalloc(&p, sizeof(float) * (count ? count : 1)) != cudaSuccess) return MRP_ERR_OOM;
            return cudaMemset(p, 0, sizeof(float) * (count ? count : 1)) == cudaSuccess ? MRP_OK : MRP_ERR_CUDA;
        };
        h.adj32.resize(h.L + 1);
        for (int k = 0; k <= h.L; ++k) {
            const size_t nb = h.lv[k].nb;
            Handle::AdjLevel32& a = h.adj32[k];
            if ((rc = alloc32(a.Ub, nb * S * S * S))) return rc;
            if ((rc = alloc32(a.Fb, nb * nn))) return rc;
            if ((rc = alloc32(a.Rb, nb * nn))) return rc;
            if ((rc = alloc32(a.Hb, nb * nn))) return rc;
        }
        if ((rc = alloc32(h.cube32, C))) return rc;
        if ((rc = alloc32(h.dense32, D))) return rc;
        if ((rc = alloc32(h.off0b32, (size_t)h.lv[0].nb * nn))) return rc;
    }
    return MRP_OK;
}

void adjoint_release(Handle& h) {
    for (auto& a : h.adj) { cudaFree(a.Ub); cudaFree(a.Fb); cudaFree(a.Rb); cudaFree(a.Hb); cudaFree(a.Rawb); }
    h.adj.clear();
    for (auto& a : h.adj32) { cudaFree(a.Ub); cudaFree(a.Fb); cudaFree(a.Rb); cudaFree(a.Hb); }
    h.adj32.clear();
    for (float* p : {h.cube32, h.dense32, h.off0b32}) cudaFree(p);
    h.cube32 = h.dense32 = h.off0b32 = nullptr;
    for (double* p : {h.lam, h.rho, h.gvec, h.xb, h.fsb, h.wl, h.cube, h.dense, h.off0b}) cudaFree(p);
    h.lam = h.rho = h.gvec = h.xb = h.fsb = h.wl = h.cube = h.dense = h.off0b = nullptr;
}

static size_t xlen(const Handle& h) { return h.xoff[h.L + 1]; }
template <typename T = double>
static size_t box_bytes(const Handle& h, int k, int g) {
    const size_t S = h.n + 2 * g;
    return sizeof(T) * h.lv[k].nb * S * S * S;
}

// Per-level adjoint fields and level-0 scratch of one working precision.
template <typename T> struct AdjF { T *Ub, *Fb, *Rb, *Hb; };
template <typename T> static AdjF<T> af(Handle& h, int k) {
    if constexpr (sizeof(T) == 8) return AdjF<T>{h.adj[k].Ub, h.adj[k].Fb, h.adj[k].Rb, h.adj[k].Hb};
    else return AdjF<T>{h.adj32[k].Ub, h.adj32[k].Fb, h.adj32[k].Rb, h.adj32[k].Hb};
}
template <typename T> static T* cube_of(Handle& h) {
    if constexpr (sizeof(T) == 8) return h.cube; else return h.cube32;
}
template <typename T> static T* dense_of(Handle& h) {
    if constexpr (sizeof(T) == 8) return h.dense; else return h.dense32;
}
template <typename T> static T* off0b_of(Handle& h) {
    if constexpr (sizeof(T) == 8) return h.off0b; else return h.off0b32;
}

// Transpose of the ghost fill of level k (u layout, halo 1), including the
// injection of level k into the covered level-(k-1) nodes that precedes it.
template <typename T>
static void ghost_fill_T(Handle& h, int k, cudaStream_t s) {
    PhaseScope ps(h, s, ph<T>(PH_GHOST), h.lv[k].nb * n3(h), k >= 1 ? 2 : 1);
    launch_ghost_T_fused<T>(af<T>(h, k).Ub, k >= 1 ? af<T>(h, k - 1).Ub : nullptr, h.lv[k].view(),
                            view_or_empty(h, k - 1), h.n, h.M, s);
    if (k >= 1) launch_inject_T<T>(af<T>(h, k).Ub, 1, af<T>(h, k - 1).Ub, 1, h.lv[k].view(), h.n, s);
}

// Transpose of problem p's level-0 convolution read on its level-0 boxes:
// the adjoint of every box (interior and exterior ring) -> the dense source
// adjoint of that problem.
template <typename T>
static void conv_T(Handle& h, const Problem& p, const T* U0bar, cudaStream_t s) {
    PhaseScope ps(h, s, ph<T>(PH_COARSE), (int64_t)p.n0[0] * p.n0[1] * p.n0[2], 6);
    const size_t S = h.n + 2;
    launch_window_T<T>(cube_of<T>(h), U0bar + (size_t)p.base0 * S * S * S, h.n, p.nb0, s);
    launch_conv_transpose<T>(h, p, cube_of<T>(h), dense_of<T>(h), s);
}

// The dense source adjoint of problem p -> per-block arrays of its covered
// (cov = true) or leaf level-0 blocks, added or set.
template <typename T>
static void dense_to(Handle& h, const Problem& p, T* out, bool cov, bool add, cudaStream_t s) {
    const Level& l0 = h.lv[0];
    const int* list = cov ? l0.cov_blocks + p.cov0_lo : l0.leaf_blocks + p.leaf0_lo;
    const int cnt = cov ? p.cov0_hi - p.cov0_lo : p.leaf0_hi - p.leaf0_lo;
    launch_dense_to_blocks<T>(out, dense_of<T>(h), list, cnt, l0.coords, h.n, p.n0, add, s);
}

// res^T lambda -> x-bar (into xb); with fsb, also adds c^T lambda (the f*-bar
// of the leaf rows and of the level-0 convolution) into fsb.
static void res_T(Handle& h, const double* lam, double* xb, double* fsb, cudaStream_t s) {
    const int L = h.L, n = h.n;
    Level& l0 = h.lv[0];
    const double ih02 = 1.0 / (h.h0 * h.h0);
    for (int k = 0; k <= L; ++k) cudaMemsetAsync(h.adj[k].Ub, 0, box_bytes(h, k, 1), s);
    {
        PhaseScope ps(h, s, PH_RESIDUAL, h.leaf_nodes, 1 + L);
        // covered level-0 rows: (conv - inject u_1) / h0^2
        launch_interior_add(h.adj[0].Ub, 1, lam + h.xoff[0], l0.cov_blocks, l0.ncov, n, -ih02, s);
        // leaf rows of levels >= 1: f* - L_k u
        for (int k = 1; k <= L; ++k) {
            const double hk = level_h(h, k);
            launch_stencil_T(h.adj[k].Ub, lam + h.xoff[k], fsb ? fsb + h.xoff[k] : nullptr, h.lv[k].leaf_blocks,
                             h.lv[k].nleaf, n, h.M, -1.0 / (hk * hk), s);
        }
    }
    // the ghost fills of levels L..1 (each with its injection), reversed
    for (int k = 1; k <= L; ++k) ghost_fill_T<double>(h, k, s);
    {
        PhaseScope ps(h, s, PH_OTHER, l0.ncov * n3(h), 1);
        launch_interior_add(h.adj[0].Ub, 1, lam + h.xoff[0], l0.cov_blocks, l0.ncov, n, ih02, s);
    }
    for (const Problem& p : h.pr) {
        conv_T<double>(h, p, h.adj[0].Ub, s);
        PhaseScope ps(h, s, PH_OTHER, (int64_t)l0.nb * n3(h), fsb ? 2 : 1);
        dense_to<double>(h, p, xb + h.xoff[0], true, false, s);
        if (fsb) dense_to<double>(h, p, fsb + h.xoff[0], false, true, s);
    }
    {
        PhaseScope ps(h, s, PH_OTHER, h.total_nodes, L + (L >= 2 ? L - 1 : 0));
        // the injections of levels L..2 that set the covered nodes first, reversed
        for (int k = 2; k <= L; ++k) launch_inject_T(h.adj[k].Ub, 1, h.adj[k - 1].Ub, 1, h.lv[k].view(), n, s);
        for (int k = 1; k <= L; ++k)
            launch_interior_get(xb + h.xoff[k], h.adj[k].Ub, 1, h.lv[k].leaf_blocks, h.lv[k].nleaf, n, 1.0, s);
    }
}

// E^T: leaf adjoint w (caller layout) -> g = E_x^T w (into gvec) and E_f^T w (into fsb, which it sets).
static void out_T(Handle& h, const double* w, cudaStream_t s) {
    const int L = h.L, n = h.n;
    Level& l0 = h.lv[0];
    const size_t len = xlen(h);
    cudaMemsetAsync(h.wl, 0, sizeof(double) * len, s);
    cudaMemsetAsync(h.fsb, 0, sizeof(double) * len, s);
    {
        PhaseScope ps(h, s, PH_OTHER, h.leaf_nodes, 2);
        LevelPtrs lp{};
        for (int k = 0; k <= L; ++k) lp.p[k] = h.wl + h.xoff[k];
        launch_scatter_leaves_to(h, w, lp, 0, false, s);
        cudaMemcpyAsync(h.gvec, h.wl, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(h.gvec, 0, sizeof(double) * h.xoff[1], s);
        cudaMemsetAsync(h.adj[0].Ub, 0, box_bytes(h, 0, 1), s);
        launch_interior_add(h.adj[0].Ub, 1, h.wl, l0.leaf_blocks, l0.nleaf, n, 1.0, s);
    }
    for (const Problem& p : h.pr) {
        conv_T<double>(h, p, h.adj[0].Ub, s);
        PhaseScope ps(h, s, PH_OTHER, l0.nb * n3(h), 2);
        dense_to<double>(h, p, h.gvec, true, false, s);
        dense_to<double>(h, p, h.fsb, false, false, s);
    }
}

// B^T: f*-bar (leaf blocks, per level) -> f-bar (caller layout).
static void rhs_T(Handle& h, const double* fsb, double* fbar, cudaStream_t s) {
    const int L = h.L, n = h.n;
    {
        PhaseScope ps(h, s, PH_OTHER, h.leaf_nodes, L + 1);
        for (int k = 0; k <= L; ++k) {
            cudaMemsetAsync(h.adj[k].Rawb, 0, box_bytes(h, k, 2), s);
            launch_rstencil_T(h.adj[k].Rawb, fsb + h.xoff[k], h.lv[k].leaf_blocks, h.lv[k].nleaf, n, h.M, s);
        }
    }
    PhaseScope ps(h, s, PH_GHOST, h.total_nodes, 2 * L + 1 + L + 1);
    for (int k = L; k >= 0; --k) {
        launch_ghost_T(h.adj[k].Rawb, 2, k >= 1 ? h.adj[k - 1].Rawb : nullptr, 2, h.lv[k].view(), view_or_empty(h, k - 1),
                       n, h.M, s);
        if (k >= 1) launch_inject_T(h.adj[k].Rawb, 2, h.adj[k - 1].Rawb, 2, h.lv[k].view(), n, s);
    }
    for (int k = 0; k < L; ++k) launch_inject_T(h.adj[k + 1].Rawb, 2, h.adj[k].Rawb, 2, h.lv[k + 1].view(), n, s);
    LevelPtrs lp{};
    for (int k = 0; k <= L; ++k) lp.p[k] = h.adj[k].Rawb;
    launch_gather_leaves_from(h, fbar, lp, 2, true, s);
}

// M^T: the transposed correction V-cycle in precision T (FP64, or FP32 on a
// mixed-precision handle), x-space vector xin -> residual-space rout (both FP64).
template <typename T>
static void cycle_T(Handle& h, const double* xin, double* rout, cudaStream_t s) {
    const int L = h.L, n = h.n;
    Level& l0 = h.lv[0];
    for (int k = 0; k <= L; ++k) {
        cudaMemsetAsync(af<T>(h, k).Ub, 0, box_bytes<T>(h, k, 1), s);
        cudaMemsetAsync(af<T>(h, k).Fb, 0, sizeof(T) * h.lv[k].nb * n3(h), s);
        cudaMemsetAsync(af<T>(h, k).Hb, 0, sizeof(T) * h.lv[k].nb * n3(h), s);
    }
    {
        PhaseScope ps(h, s, ph<T>(PH_OTHER), h.leaf_nodes, L + 1);
        for (int k = 1; k <= L; ++k)
            launch_interior_add<T, double>(af<T>(h, k).Ub, 1, xin + h.xoff[k], h.lv[k].leaf_blocks, h.lv[k].nleaf, n,
                                           1.0, s);
        launch_block_copy<T, double>(af<T>(h, 0).Fb, xin, l0.cov_blocks, l0.ncov, n, 1.0, s);
    }
    auto smooth_T = [&](int k) {
        PhaseScope ps(h, s, ph<T>(PH_SMOOTH), h.lv[k].nb * n3(h), 1);
        const double hk = level_h(h, k);
        launch_smooth_T<T>(af<T>(h, k).Ub, af<T>(h, k).Fb, h.lv[k].nb, n, h.M, hk * hk, s);
    };
    // coarse-to-fine half, reversed
    for (int k = L; k >= 1; --k) {
        for (int i = 0; i < h.nu2; ++i) { smooth_T(k); ghost_fill_T<T>(h, k, s); }
        PhaseScope ps(h, s, ph<T>(PH_PROLONG), h.lv[k].nb * n3(h), 1);
        launch_prolong_T<T>(af<T>(h, k - 1).Ub, af<T>(h, k - 1).Hb, af<T>(h, k).Ub, h.lv[k].view(), h.lv[k - 1].view(),
                            n, s);
    }
    // level-0 solve: the source adjoint gains the convolution transpose of u_0's adjoint
    for (const Problem& p : h.pr) {
        conv_T<T>(h, p, af<T>(h, 0).Ub, s);
        PhaseScope ps(h, s, ph<T>(PH_COARSE), l0.nb * n3(h), 2);
        dense_to<T>(h, p, af<T>(h, 0).Fb, true, true, s);
        dense_to<T>(h, p, af<T>(h, 0).Fb, false, true, s);
    }
    cudaMemsetAsync(af<T>(h, 0).Ub, 0, box_bytes<T>(h, 0, 1), s);
    // fine-to-coarse half, reversed
    for (int k = 1; k <= L; ++k) {
        Level& c = h.lv[k - 1];
        Level& f = h.lv[k];
        const AdjF<T> ac = af<T>(h, k - 1), a = af<T>(h, k);
        {
            PhaseScope ps(h, s, ph<T>(PH_RESTRICT), c.nb * n3(h), 2);
            const double hc = level_h(h, k - 1);
            // uhat_{k-1} = u_{k-1}; f_{k-1} += L u_{k-1} on covered blocks
            launch_interior_add<T, T>(ac.Ub, 1, ac.Hb, c.order, c.nb, n, 1.0, s);
            cudaMemsetAsync(ac.Hb, 0, sizeof(T) * c.nb * n3(h), s);
            launch_stencil_T<T>(ac.Ub, ac.Fb, nullptr, c.cov_blocks, c.ncov, n, h.M, 1.0 / (hc * hc), s);
        }
        ghost_fill_T<T>(h, k - 1, s);
        {
            PhaseScope ps(h, s, ph<T>(PH_RESTRICT), f.nb * n3(h), 3 + (k == 1 ? 1 : 0));
            // f_{k-1} = FW r_k on covered blocks
            launch_fw_T<T>(a.Rb, ac.Fb, f.view(), n, s);
            launch_block_zero<T>(ac.Fb, c.cov_blocks, c.ncov, n, s);
            // u_{k-1} = inject u_k (+ the level-0 offset carrying the covered level-0 rows)
            if (k == 1) launch_interior_get<T, T>(off0b_of<T>(h), af<T>(h, 0).Ub, 1, l0.cov_blocks, l0.ncov, n, 1.0, s);
            launch_inject_T<T>(a.Ub, 1, ac.Ub, 1, f.view(), n, s);
        }
        {
            PhaseScope ps(h, s, ph<T>(PH_RESIDUAL), f.nb * n3(h), 1);
            const double hk = level_h(h, k);
            launch_stencil_T<T>(a.Ub, a.Rb, a.Fb, f.order, f.nb, n, h.M, -1.0 / (hk * hk), s);
        }
        ghost_fill_T<T>(h, k, s);
        for (int i = 0; i < h.nu1; ++i) { smooth_T(k); ghost_fill_T<T>(h, k, s); }
    }
    PhaseScope ps(h, s, ph<T>(PH_OTHER), h.leaf_nodes, L + 1);
    for (int k = 1; k <= L; ++k)
        launch_block_copy<double, T>(rout + h.xoff[k], af<T>(h, k).Fb, h.lv[k].leaf_blocks, h.lv[k].nleaf, n, 1.0, s);
    launch_block_copy<double, T>(rout, off0b_of<T>(h), l0.cov_blocks, l0.ncov, n, -h.h0 * h.h0, s);
}

// Per-problem max |v| over an unknown-space vector into slot 2.
static void xnorm_launch(Handle& h, const double* v, cudaStream_t s) {
    cudaMemsetAsync(h.slot(2), 0, sizeof(unsigned long long) * h.nprob(), s);
    PhaseScope ps(h, s, PH_NORM, h.total_nodes, h.L + 1);
    for (int k = 0; k <= h.L; ++k)
        launch_absmax(v + h.xoff[k], h.lv[k].order, h.lv[k].nb, h.n, h.slot(2), h.lv[k].prob, s);
}

// The whole gradient.  Returns MRP_OK, MRP_ERR_NOT_CONVERGED (fbar still
// written) or an error status; *rel_out is the worst problem's relative residual.
int solve_adjoint(Handle& h, const double* w, double* fbar, cudaStream_t s, int* cycles_out, double* rel_out) {
    int rc = adjoint_setup(h);
    if (rc) return rc;
    const size_t len = xlen(h);
    const int np = h.nprob();
    out_T(h, w, s);
    cudaMemsetAsync(h.lam, 0, sizeof(double) * len, s);
    cudaMemcpyAsync(h.rho, h.gvec, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
    xnorm_launch(h, h.rho, s);
    std::vector<double> gmax(np), r(np);
    if ((rc = read_max(h, s, gmax.data(), 2))) return rc;
    auto worst = [&](const std::vector<double>& v) {
        double m = 0.0;
        for (int p = 0; p < np; ++p) m = std::max(m, v[p] / (gmax[p] > 0.0 ? gmax[p] : 1.0));
        return m;
    };
    double rel = worst(gmax);
    int cycles = 0;
    while (rel >= h.tol && cycles < h.max_cycles) {
        if (h.mixed) cycle_T<float>(h, h.rho, h.xb, s);
        else cycle_T<double>(h, h.rho, h.xb, s);
        ++cycles;
        {
            PhaseScope ps(h, s, PH_NORM, (int64_t)len, 1);
            launch_lincomb(h.lam, 1.0, h.lam, 1.0, h.xb, len, nullptr, s);
        }
        res_T(h, h.lam, h.xb, nullptr, s);
        {
            // rho = g - K^T lambda = g + x-bar
            PhaseScope ps(h, s, PH_NORM, (int64_t)len, 1);
            launch_lincomb(h.rho, 1.0, h.gvec, 1.0, h.xb, len, nullptr, s);
        }
        xnorm_launch(h, h.rho, s);
        if ((rc = read_max(h, s, r.data(), 2))) return rc;
        rel = worst(r);
        if (!std::isfinite(rel)) { *cycles_out = cycles; *rel_out = rel; return MRP_ERR_NUMERICAL; }
    }
    res_T(h, h.lam, h.xb, h.fsb, s);
    rhs_T(h, h.fsb, fbar, s);
    if (cudaGetLastError() != cudaSuccess) return MRP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
    harvest(h);
    *cycles_out = cycles;
    *rel_out = rel;
    return rel < h.tol ? MRP_OK : MRP_ERR_NOT_CONVERGED;
}

// Single transposed operators for parity checks (see mrp_adjoint_op).
int adjoint_op(Handle& h, int op, const double* in, double* out, cudaStream_t s) {
    int rc = adjoint_setup(h);
    if (rc) return rc;
    const size_t len = xlen(h);
    switch (op) {
        case MRP_ADJ_CYCLE_T:
            cudaMemcpyAsync(h.rho, in, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            cudaMemsetAsync(h.xb, 0, sizeof(double) * len, s);
            cycle_T<double>(h, h.rho, h.xb, s);
            cudaMemcpyAsync(out, h.xb, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            break;
        case MRP_ADJ_RES_T:
            cudaMemcpyAsync(h.lam, in, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            cudaMemsetAsync(h.xb, 0, sizeof(double) * len, s);
            cudaMemsetAsync(h.fsb, 0, sizeof(double) * len, s);
            res_T(h, h.lam, h.xb, h.fsb, s);
            cudaMemcpyAsync(out, h.xb, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(out + len, h.fsb, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            break;
        case MRP_ADJ_OUT_T:
            out_T(h, in, s);
            cudaMemcpyAsync(out, h.gvec, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(out + len, h.fsb, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            break;
        case MRP_ADJ_RHS_T:
            cudaMemcpyAsync(h.fsb, in, sizeof(double) * len, cudaMemcpyDeviceToDevice, s);
            rhs_T(h, h.fsb, out, s);
            break;
        default:
            return MRP_ERR_INVALID_ARG;
    }
    if (cudaGetLastError() != cudaSuccess) return MRP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
    harvest(h);
    return MRP_OK;
}

}  // namespace mrp
