// Stencil, ghosting and grid-transfer kernels of the adaptive V-cycle.
//
// Every kernel works on whole blocks: one CTA per block, the block's nodes
// enumerated by the CTA's threads.  Fields are [block][z][y][x] with a halo
// of g layers (U: g = 1, raw f: g = 2).
#include "mrp_internal.h"

namespace mrp {

// ----------------------------------------------------------------------------
// Stencil weights (arXiv 2512.08555, Fig. stencils / Sec. 3.2), unit spacing,
// as integers over a common denominator:  L u = (c u0 + f Sum_faces + e Sum_edges
// + k Sum_corners) / den / h^2.
template <int M> struct LhsW;
template <> struct LhsW<2> { static constexpr double den = 1, c = -6, f = 1, e = 0, k = 0; };
template <> struct LhsW<4> { static constexpr double den = 6, c = -24, f = 2, e = 1, k = 0; };
template <> struct LhsW<6> { static constexpr double den = 30, c = -128, f = 14, e = 3, k = 1; };

// Weighted sum of the 26 off-centre neighbours of node o in an array with
// strides (1, S, S2).
template <int M, typename T>
__device__ __forceinline__ T offcentre(const T* __restrict__ a, int o, int S, int S2) {
    using W = LhsW<M>;
    T sf = (a[o - 1] + a[o + 1]) + (a[o - S] + a[o + S]) + (a[o - S2] + a[o + S2]);
    T acc = T(W::f) * sf;
    if (W::e != 0) {
        T se = (a[o - 1 - S] + a[o + 1 - S]) + (a[o - 1 + S] + a[o + 1 + S])
             + (a[o - 1 - S2] + a[o + 1 - S2]) + (a[o - 1 + S2] + a[o + 1 + S2])
             + (a[o - S - S2] + a[o + S - S2]) + (a[o - S + S2] + a[o + S + S2]);
        acc += T(W::e) * se;
    }
    if (W::k != 0) {
        T sc = (a[o - 1 - S - S2] + a[o + 1 - S - S2]) + (a[o - 1 + S - S2] + a[o + 1 + S - S2])
             + (a[o - 1 - S + S2] + a[o + 1 - S + S2]) + (a[o - 1 + S + S2] + a[o + 1 + S + S2]);
        acc += T(W::k) * sc;
    }
    return acc;
}

// L u at node o (times h^2 * den).
template <int M, typename T>
__device__ __forceinline__ T lhs_scaled(const T* __restrict__ a, int o, int S, int S2) {
    return T(LhsW<M>::c) * a[o] + offcentre<M>(a, o, S, S2);
}

// Midpoint Lagrange weights of I = M + 2 points (Sec. 2.1: interpolation of
// order M + 2 at resolution jumps); node offsets -(I-1)/2 .. (I-1)/2.
struct InterpW { int I; double w[8]; };
static InterpW interp_weights(int M) {
    InterpW r{};
    r.I = M + 2;
    if (r.I == 4) { const double w[4] = {-1, 9, 9, -1}; for (int i = 0; i < 4; ++i) r.w[i] = w[i] / 16.0; }
    if (r.I == 6) { const double w[6] = {3, -25, 150, 150, -25, 3}; for (int i = 0; i < 6; ++i) r.w[i] = w[i] / 256.0; }
    if (r.I == 8) { const double w[8] = {-5, 49, -245, 1225, 1225, -245, 49, -5}; for (int i = 0; i < 8; ++i) r.w[i] = w[i] / 2048.0; }
    return r;
}

// ----------------------------------------------------------------------------
// Injection of level-k values into the covered nodes of their parent block
// (Alg. 1, restriction of u; also the coarse representation of the fine
// blocks that ghosting at a resolution jump reads).
template <typename T>
__global__ void k_inject_to_parent(T* __restrict__ coarse, int gc, const T* __restrict__ fine, int gf,
                                   LevelView lf, int n, const T* __restrict__ off) {
    const int B = blockIdx.x;
    const int P = lf.parent[B];
    const int o = lf.octant[B];
    const int h = n >> 1;
    const int Sf = n + 2 * gf, Sc = n + 2 * gc;
    const T* src = fine + (size_t)B * Sf * Sf * Sf;
    T* dst = coarse + (size_t)P * Sc * Sc * Sc;
    const T* ob = off ? off + (size_t)P * n * n * n : nullptr;
    const int ox = (o & 1) * h, oy = ((o >> 1) & 1) * h, oz = ((o >> 2) & 1) * h;
    for (int t = threadIdx.x; t < h * h * h; t += blockDim.x) {
        const int i = t % h, j = (t / h) % h, l = t / (h * h);
        T v = src[((gf + 2 * l) * Sf + gf + 2 * j) * Sf + gf + 2 * i];
        if (ob) v += ob[((oz + l) * n + oy + j) * n + ox + i];
        dst[((gc + oz + l) * Sc + gc + oy + j) * Sc + gc + ox + i] = v;
    }
}

template <typename T>
void launch_inject_to_parent(T* coarse, int gc, const T* fine, int gf, LevelView lf, int n, const T* off, cudaStream_t s) {
    if (lf.nb == 0) return;
    k_inject_to_parent<T><<<lf.nb, 256, 0, s>>>(coarse, gc, fine, gf, lf, n, off);
}
template void launch_inject_to_parent<double>(double*, int, const double*, int, LevelView, int, const double*, cudaStream_t);
template void launch_inject_to_parent<float>(float*, int, const float*, int, LevelView, int, const float*, cudaStream_t);

// ----------------------------------------------------------------------------
// Ghosting (Sec. 2.1).  Halo node of block b in direction d: copied from the
// level-k neighbour when it exists; outside the domain left alone or zeroed;
// otherwise the I-point tensor-product Lagrange interpolant of level k-1
// (identity along axes where the node coincides with a coarse node).  The
// coarse nodes lie in the 27-neighbourhood of b's parent.
template <typename T>
__global__ void k_ghost_fill(T* __restrict__ A, int g, const T* __restrict__ Ac, int gc, LevelView lk,
                             LevelView lc, int n, InterpW iw, bool zero_outside) {
    const int b = blockIdx.x;
    const int S = n + 2 * g, S2 = S * S, S3 = S2 * S;
    const int Sc = n + 2 * gc, Sc2 = Sc * Sc, Sc3 = Sc2 * Sc;
    const int* nbr = lk.nbr + b * 27;
    T* Ab = A + (size_t)b * S3;
    const int bx = lk.coords[3 * b], by = lk.coords[3 * b + 1], bz = lk.coords[3 * b + 2];
    for (int t = threadIdx.x; t < S3; t += blockDim.x) {
        const int x = t % S, y = (t / S) % S, z = t / S2;
        const int dx = x < g ? -1 : (x >= g + n ? 1 : 0);
        const int dy = y < g ? -1 : (y >= g + n ? 1 : 0);
        const int dz = z < g ? -1 : (z >= g + n ? 1 : 0);
        if ((dx | dy | dz) == 0) continue;
        const int j = nbr[dir27(dx, dy, dz)];
        if (j >= 0) {
            Ab[t] = A[(size_t)j * S3 + (size_t)((z - dz * n) * S + (y - dy * n)) * S + (x - dx * n)];
            continue;
        }
        if (j == NBR_OUTSIDE) {
            if (zero_outside) Ab[t] = T(0);
            continue;
        }
        // interpolation from level k-1
        const int P = lk.parent[b];
        const int* cnbr = lc.nbr + P * 27;
        const int p[3] = {bx * n + x - g, by * n + y - g, bz * n + z - g};
        const int porig[3] = {(bx >> 1) * n, (by >> 1) * n, (bz >> 1) * n};
        int cnt[3], c0[3];
        for (int a = 0; a < 3; ++a) {
            if ((p[a] & 1) == 0) { cnt[a] = 1; c0[a] = (p[a] >> 1) - porig[a]; }
            else { cnt[a] = iw.I; c0[a] = ((p[a] - 1) >> 1) - iw.I / 2 + 1 - porig[a]; }
        }
        T accz = T(0);
        for (int mz = 0; mz < cnt[2]; ++mz) {
            const int rz = c0[2] + mz;
            const int ddz = rz < 0 ? -1 : (rz >= n ? 1 : 0);
            const int lz = rz - ddz * n;
            T accy = T(0);
            for (int my = 0; my < cnt[1]; ++my) {
                const int ry = c0[1] + my;
                const int ddy = ry < 0 ? -1 : (ry >= n ? 1 : 0);
                const int ly = ry - ddy * n;
                T accx = T(0);
                for (int mx = 0; mx < cnt[0]; ++mx) {
                    const int rx = c0[0] + mx;
                    const int ddx = rx < 0 ? -1 : (rx >= n ? 1 : 0);
                    const int lx = rx - ddx * n;
                    const int cb = cnbr[dir27(ddx, ddy, ddz)];
                    const T v = Ac[(size_t)cb * Sc3 + (size_t)((gc + lz) * Sc + gc + ly) * Sc + gc + lx];
                    accx += (cnt[0] == 1 ? T(1) : T(iw.w[mx])) * v;
                }
                accy += (cnt[1] == 1 ? T(1) : T(iw.w[my])) * accx;
            }
            accz += (cnt[2] == 1 ? T(1) : T(iw.w[mz])) * accy;
        }
        Ab[t] = accz;
    }
}

void launch_ghost_fill(double* A, int g, const double* Ac, int gc, LevelView lk, LevelView lkm1, int n, int M,
                       bool zero_outside, cudaStream_t s) {
    if (lk.nb == 0) return;
    k_ghost_fill<double><<<lk.nb, 256, 0, s>>>(A, g, Ac, gc, lk, lkm1, n, interp_weights(M), zero_outside);
}

// ----------------------------------------------------------------------------
// Leaf scatter / gather between the caller's layout (leaf i at element
// offset src[i], n^3 values, x fastest) and the per-level halo layout
// (halo g); values are multiplied by scale[i] when a scale table is given.
__global__ void k_scatter_leaves(const double* __restrict__ f, const int* __restrict__ leaf_level,
                                 const int* __restrict__ leaf_block, const int64_t* __restrict__ src_off,
                                 const double* __restrict__ scale, LevelPtrs dst, int n, int g) {
    const int i = blockIdx.x;
    const int S = n + 2 * g;
    double* d = dst.p[leaf_level[i]] + (size_t)leaf_block[i] * S * S * S;
    const double* src = f + src_off[i];
    const double a = scale ? scale[i] : 1.0;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        d[((z + g) * S + y + g) * S + x + g] = a * src[t];
    }
}

__global__ void k_gather_leaves(double* __restrict__ u, const int* __restrict__ leaf_level,
                                const int* __restrict__ leaf_block, const int64_t* __restrict__ dst_off,
                                const double* __restrict__ scale, LevelPtrs src, int n, int g) {
    const int i = blockIdx.x;
    const int S = n + 2 * g;
    const double* s = src.p[leaf_level[i]] + (size_t)leaf_block[i] * S * S * S;
    double* d = u + dst_off[i];
    const double a = scale ? scale[i] : 1.0;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        d[t] = a * s[((z + g) * S + y + g) * S + x + g];
    }
}

void launch_scatter_leaves(Handle& h, const double* f, cudaStream_t s) {
    LevelPtrs lp{};
    for (int k = 0; k <= h.L; ++k) lp.p[k] = h.lv[k].Fraw;
    k_scatter_leaves<<<h.n_leaves, 256, 0, s>>>(f, h.leaf_level, h.leaf_block, h.leaf_src, h.leaf_scale, lp, h.n, 2);
}

void launch_gather_leaves(Handle& h, double* u, cudaStream_t s) {
    LevelPtrs lp{};
    for (int k = 0; k <= h.L; ++k) lp.p[k] = h.lv[k].U;
    k_gather_leaves<<<h.n_leaves, 256, 0, s>>>(u, h.leaf_level, h.leaf_block, h.leaf_src, nullptr, lp, h.n, 1);
}

void launch_scatter_leaves_to(const Handle& h, const double* f, const LevelPtrs& dst, int g, bool scaled, cudaStream_t s) {
    k_scatter_leaves<<<h.n_leaves, 256, 0, s>>>(f, h.leaf_level, h.leaf_block, h.leaf_src, scaled ? h.leaf_scale : nullptr,
                                                dst, h.n, g);
}

void launch_gather_leaves_from(const Handle& h, double* u, const LevelPtrs& src, int g, bool scaled, cudaStream_t s) {
    k_gather_leaves<<<h.n_leaves, 256, 0, s>>>(u, h.leaf_level, h.leaf_block, h.leaf_src, scaled ? h.leaf_scale : nullptr,
                                               src, h.n, g);
}

// ----------------------------------------------------------------------------
// f* = R^M f on leaf blocks (Sec. 3.2; R^6 reaches two nodes along the axes).
template <int M>
__global__ void k_rhs_star(double* __restrict__ F, const double* __restrict__ Fraw, const int* __restrict__ blocks,
                           int n) {
    const int b = blocks[blockIdx.x];
    const int S = n + 4, S2 = S * S;
    const double* a = Fraw + (size_t)b * S2 * S;
    double* out = F + (size_t)b * n * n * n;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        const int o = ((z + 2) * S + y + 2) * S + x + 2;
        double v;
        if (M == 2) {
            v = a[o];
        } else {
            const double sf = (a[o - 1] + a[o + 1]) + (a[o - S] + a[o + S]) + (a[o - S2] + a[o + S2]);
            if (M == 4) {
                v = 0.5 * a[o] + sf / 12.0;
            } else {
                const double se = (a[o - 1 - S] + a[o + 1 - S]) + (a[o - 1 + S] + a[o + 1 + S])
                                + (a[o - 1 - S2] + a[o + 1 - S2]) + (a[o - 1 + S2] + a[o + 1 + S2])
                                + (a[o - S - S2] + a[o + S - S2]) + (a[o - S + S2] + a[o + S + S2]);
                const double s2 = (a[o - 2] + a[o + 2]) + (a[o - 2 * S] + a[o + 2 * S]) + (a[o - 2 * S2] + a[o + 2 * S2]);
                v = (67.0 / 120.0) * a[o] + sf / 18.0 + se / 90.0 - s2 / 240.0;
            }
        }
        out[t] = v;
    }
}

void launch_rhs_star(double* F, const double* Fraw, const int* leaf_blocks, int nleaf, int n, int M, cudaStream_t s) {
    if (nleaf == 0) return;
    if (M == 2) k_rhs_star<2><<<nleaf, 256, 0, s>>>(F, Fraw, leaf_blocks, n);
    if (M == 4) k_rhs_star<4><<<nleaf, 256, 0, s>>>(F, Fraw, leaf_blocks, n);
    if (M == 6) k_rhs_star<6><<<nleaf, 256, 0, s>>>(F, Fraw, leaf_blocks, n);
}

// ----------------------------------------------------------------------------
// One Gauss-Seidel iteration (Sec. 3.1) on every block: the block with its
// frozen ghost layer is staged in shared memory, nodes are updated colour by
// colour (c = (x&1) + 2(y&1) + 4(z&1), c = 0..7) with
//   u <- (den h^2 f - offcentre) / c,
// the same-colour nodes of one colour being independent for a 27-point stencil.
template <int M, typename T>
__global__ void k_smooth(T* __restrict__ U, const T* __restrict__ F, int n, T h2den) {
    extern __shared__ unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    const int S = n + 2, S2 = S * S, S3 = S2 * S;
    const int b = blockIdx.x;
    T* Ub = U + (size_t)b * S3;
    const T* Fb = F + (size_t)b * n * n * n;
    for (int t = threadIdx.x; t < S3; t += blockDim.x) s[t] = Ub[t];
    __syncthreads();
    const int h = n >> 1, h3 = h * h * h;
    const T inv_c = T(1) / T(LhsW<M>::c);
    for (int col = 0; col < 8; ++col) {
        const int cx = col & 1, cy = (col >> 1) & 1, cz = (col >> 2) & 1;
        for (int q = threadIdx.x; q < h3; q += blockDim.x) {
            const int x = 2 * (q % h) + cx, y = 2 * ((q / h) % h) + cy, z = 2 * (q / (h * h)) + cz;
            const int o = ((z + 1) * S + y + 1) * S + x + 1;
            s[o] = (h2den * Fb[(z * n + y) * n + x] - offcentre<M>(s, o, S, S2)) * inv_c;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        const int o = ((z + 1) * S + y + 1) * S + x + 1;
        Ub[o] = s[o];
    }
}

template <typename T>
static void smooth_attributes() {
    static bool done = false;
    if (done) return;
    const int mx = MAX_DYN_SMEM;
    cudaFuncSetAttribute(k_smooth<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_smooth<4, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(k_smooth<6, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    done = true;
}

template <typename T>
void launch_smooth(T* U, const T* F, int nb, int n, int M, double h2, cudaStream_t s) {
    if (nb == 0) return;
    smooth_attributes<T>();
    const size_t sm = sizeof(T) * (n + 2) * (n + 2) * (n + 2);
    if (M == 2) k_smooth<2, T><<<nb, 256, sm, s>>>(U, F, n, T(h2 * LhsW<2>::den));
    if (M == 4) k_smooth<4, T><<<nb, 256, sm, s>>>(U, F, n, T(h2 * LhsW<4>::den));
    if (M == 6) k_smooth<6, T><<<nb, 256, sm, s>>>(U, F, n, T(h2 * LhsW<6>::den));
}
template void launch_smooth<double>(double*, const double*, int, int, int, double, cudaStream_t);
template void launch_smooth<float>(float*, const float*, int, int, int, double, cudaStream_t);

// ----------------------------------------------------------------------------
// r = f - L u on every node of every block (Alg. 1).
template <int M, typename T>
__global__ void k_residual(T* __restrict__ R, const T* __restrict__ U, const T* __restrict__ F, int n, T scale) {
    const int S = n + 2, S2 = S * S;
    const int b = blockIdx.x;
    const T* Ub = U + (size_t)b * S2 * S;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        const int o = ((z + 1) * S + y + 1) * S + x + 1;
        R[(size_t)b * n * n * n + t] = F[(size_t)b * n * n * n + t] - scale * lhs_scaled<M>(Ub, o, S, S2);
    }
}

template <typename T>
void launch_residual(T* R, const T* U, const T* F, int nb, int n, int M, double inv_h2, cudaStream_t s) {
    if (nb == 0) return;
    if (M == 2) k_residual<2, T><<<nb, 256, 0, s>>>(R, U, F, n, T(inv_h2 / LhsW<2>::den));
    if (M == 4) k_residual<4, T><<<nb, 256, 0, s>>>(R, U, F, n, T(inv_h2 / LhsW<4>::den));
    if (M == 6) k_residual<6, T><<<nb, 256, 0, s>>>(R, U, F, n, T(inv_h2 / LhsW<6>::den));
}
template void launch_residual<double>(double*, const double*, const double*, int, int, int, double, cudaStream_t);
template void launch_residual<float>(float*, const float*, const float*, int, int, int, double, cudaStream_t);

// ----------------------------------------------------------------------------
// Restriction from level k to the covered blocks of level k-1 (Alg. 1):
// u_{k-1} = injection of u_k;  r_{k-1} = full weighting (1/4)[1 2 1]^3 of r_k,
// or injection where the 27-point stencil reaches outside Omega_k.  The
// restricted residual is left in F_{k-1}; k_fas_snapshot adds L u_{k-1}.
template <typename T>
__global__ void k_restrict(T* __restrict__ Uc, T* __restrict__ Fc, const T* __restrict__ Uf, const T* __restrict__ Rf,
                           const int* __restrict__ cov, LevelView lc, LevelView lf, int n, const T* __restrict__ off) {
    const int P = cov[blockIdx.x];
    const int S = n + 2, S3 = S * S * S, n3 = n * n * n, h = n >> 1;
    const int* kids = lc.children + 8 * P;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, l = t / (n * n);
        const int ox = i >= h, oy = j >= h, oz = l >= h;
        const int c = kids[ox + 2 * oy + 4 * oz];
        const int fx = 2 * i - ox * n, fy = 2 * j - oy * n, fz = 2 * l - oz * n;
        Uc[(size_t)P * S3 + ((l + 1) * S + j + 1) * S + i + 1] = Uf[(size_t)c * S3 + ((fz + 1) * S + fy + 1) * S + fx + 1]
                                                               + (off ? off[(size_t)P * n3 + t] : T(0));
        const int* cn = lf.nbr + 27 * c;
        T acc = T(0);
        bool inside = true;
        for (int dz = -1; dz <= 1 && inside; ++dz) {
            const int zz = fz + dz, ez = zz < 0 ? -1 : 0;
            T accy = T(0);
            for (int dy = -1; dy <= 1 && inside; ++dy) {
                const int yy = fy + dy, ey = yy < 0 ? -1 : 0;
                T accx = T(0);
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = fx + dx, ex = xx < 0 ? -1 : 0;
                    const int blk = cn[dir27(ex, ey, ez)];
                    if (blk < 0) { inside = false; break; }
                    const T v = Rf[(size_t)blk * n3 + ((zz - ez * n) * n + yy - ey * n) * n + xx - ex * n];
                    accx += T(2 - (dx < 0 ? -dx : dx)) * v;
                }
                accy += T(2 - (dy < 0 ? -dy : dy)) * accx;
            }
            acc += T(2 - (dz < 0 ? -dz : dz)) * accy;
        }
        Fc[(size_t)P * n3 + t] = inside ? acc * T(1.0 / 64.0) : Rf[(size_t)c * n3 + (fz * n + fy) * n + fx];
    }
}

template <typename T>
void launch_restrict(T* Uc, T* Fc, const T* Uf, const T* Rf, const int* cov, int ncov, LevelView lc, LevelView lf, int n,
                     const T* off, cudaStream_t s) {
    if (ncov == 0) return;
    k_restrict<T><<<ncov, 256, 0, s>>>(Uc, Fc, Uf, Rf, cov, lc, lf, n, off);
}
template void launch_restrict<double>(double*, double*, const double*, const double*, const int*, int, LevelView, LevelView,
                                      int, const double*, cudaStream_t);
template void launch_restrict<float>(float*, float*, const float*, const float*, const int*, int, LevelView, LevelView,
                                     int, const float*, cudaStream_t);

// F += L u on covered blocks; u-hat = u on every block of the level (Alg. 1).
template <int M, typename T>
__global__ void k_fas_snapshot(T* __restrict__ F, T* __restrict__ H, const T* __restrict__ U, const uint8_t* __restrict__ is_leaf,
                               int n, T scale) {
    const int b = blockIdx.x;
    const int S = n + 2, S2 = S * S, n3 = n * n * n;
    const T* Ub = U + (size_t)b * S2 * S;
    const bool cov = !is_leaf[b];
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        const int o = ((z + 1) * S + y + 1) * S + x + 1;
        if (cov) F[(size_t)b * n3 + t] += scale * lhs_scaled<M>(Ub, o, S, S2);
        H[(size_t)b * n3 + t] = Ub[o];
    }
}

template <typename T>
void launch_fas_snapshot(T* F, T* H, const T* U, const uint8_t* is_leaf, int nb, int n, int M, double inv_h2, cudaStream_t s) {
    if (nb == 0) return;
    if (M == 2) k_fas_snapshot<2, T><<<nb, 256, 0, s>>>(F, H, U, is_leaf, n, T(inv_h2 / LhsW<2>::den));
    if (M == 4) k_fas_snapshot<4, T><<<nb, 256, 0, s>>>(F, H, U, is_leaf, n, T(inv_h2 / LhsW<4>::den));
    if (M == 6) k_fas_snapshot<6, T><<<nb, 256, 0, s>>>(F, H, U, is_leaf, n, T(inv_h2 / LhsW<6>::den));
}
template void launch_fas_snapshot<double>(double*, double*, const double*, const uint8_t*, int, int, int, double, cudaStream_t);
template void launch_fas_snapshot<float>(float*, float*, const float*, const uint8_t*, int, int, int, double, cudaStream_t);

// ----------------------------------------------------------------------------
// Coarse-grid correction (Alg. 1): eps = u_{k-1} - uhat_{k-1} on the coarse
// nodes of the fine block's extent plus the next coarse node on each upper
// side, then u_k += trilinear(eps).
template <typename T>
__global__ void k_prolong(T* __restrict__ Uf, const T* __restrict__ Uc, const T* __restrict__ Hc, LevelView lf,
                          LevelView lc, int n) {
    extern __shared__ unsigned char smem_raw[];
    T* e = reinterpret_cast<T*>(smem_raw);
    const int B = blockIdx.x;
    const int P = lf.parent[B], o = lf.octant[B];
    const int h = n >> 1, E = h + 1;
    const int S = n + 2, S3 = S * S * S, n3 = n * n * n;
    const int ox = (o & 1) * h, oy = ((o >> 1) & 1) * h, oz = ((o >> 2) & 1) * h;
    const int* cn = lc.nbr + 27 * P;
    for (int t = threadIdx.x; t < E * E * E; t += blockDim.x) {
        const int i = t % E, j = (t / E) % E, l = t / (E * E);
        const int cx = ox + i, cy = oy + j, cz = oz + l;
        const int ex = cx >= n, ey = cy >= n, ez = cz >= n;
        const int blk = cn[dir27(ex, ey, ez)];
        const int lx = cx - ex * n, ly = cy - ey * n, lz = cz - ez * n;
        e[t] = Uc[(size_t)blk * S3 + ((lz + 1) * S + ly + 1) * S + lx + 1] - Hc[(size_t)blk * n3 + (lz * n + ly) * n + lx];
    }
    __syncthreads();
    T* Ub = Uf + (size_t)B * S3;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        const int ax = x >> 1, ay = y >> 1, az = z >> 1;
        const int bx = x & 1, by = y & 1, bz = z & 1;
        T acc = T(0);
        for (int mz = 0; mz <= bz; ++mz) {
            T accy = T(0);
            for (int my = 0; my <= by; ++my) {
                T accx = T(0);
                for (int mx = 0; mx <= bx; ++mx) accx += e[((az + mz) * E + ay + my) * E + ax + mx];
                accy += (bx ? T(0.5) : T(1)) * accx;
            }
            acc += (by ? T(0.5) : T(1)) * accy;
        }
        Ub[((z + 1) * S + y + 1) * S + x + 1] += (bz ? T(0.5) : T(1)) * acc;
    }
}

template <typename T>
void launch_prolong(T* Uf, const T* Uc, const T* Hc, LevelView lf, LevelView lc, int n, cudaStream_t s) {
    if (lf.nb == 0) return;
    const int E = n / 2 + 1;
    k_prolong<T><<<lf.nb, 256, sizeof(T) * E * E * E, s>>>(Uf, Uc, Hc, lf, lc, n);
}
template void launch_prolong<double>(double*, const double*, const double*, LevelView, LevelView, int, cudaStream_t);
template void launch_prolong<float>(float*, const float*, const float*, LevelView, LevelView, int, cudaStream_t);

// ----------------------------------------------------------------------------
// Max-norm reductions: warp shuffle, then one atomicMax per CTA on the bit
// pattern of a non-negative double (monotone in the value).  NaN is mapped
// to +Inf so that it cannot hide below a finite maximum.
__device__ __forceinline__ void block_max_atomic(double v, unsigned long long* out) {
    __shared__ double red[32];
    if (v != v) v = __longlong_as_double(0x7ff0000000000000ULL);
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (lane == 0) atomicMax(out, (unsigned long long)__double_as_longlong(v));
    }
}

// max |F| over the listed blocks into out[prob[b]] (out[0] without a problem table).
__global__ void k_absmax(const double* __restrict__ F, const int* __restrict__ blocks, int n, unsigned long long* out,
                         const int* __restrict__ prob) {
    const int b = blocks[blockIdx.x];
    const int n3 = n * n * n;
    double m = 0.0;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const double v = F[(size_t)b * n3 + t];
        m = (v != v) ? __longlong_as_double(0x7ff0000000000000ULL) : fmax(m, fabs(v));
    }
    block_max_atomic(m, out + (prob ? prob[b] : 0));
}

void launch_absmax(const double* F, const int* blocks, int nblocks, int n, unsigned long long* out, const int* prob,
                   cudaStream_t s) {
    if (nblocks == 0) return;
    k_absmax<<<nblocks, 256, 0, s>>>(F, blocks, n, out, prob);
}

}  // namespace mrp
