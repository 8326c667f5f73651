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
//
// Interface blocks first stage, in shared memory, every coarse node their
// interpolants can touch: parent-local indices [pb, pb + PL) per axis with
// pb = (b&1) n/2 - (g+1)/2 - I/2 and PL = n/2 + g + I + 1 (nodes of missing
// coarse blocks, which no interpolant uses, read as 0).
template <int I>
__global__ void k_ghost_fill(double* __restrict__ A, int g, const double* __restrict__ Ac, int gc, LevelView lk,
                             LevelView lc, int n, InterpW iw, bool zero_outside) {
    extern __shared__ double gpatch[];
    __shared__ int snbr[27], cnbr[27];
    __shared__ double sw[8];
    __shared__ int interp;
    const int b = blockIdx.x;
    const int S = n + 2 * g, S2 = S * S, S3 = S2 * S;
    const int Sc = n + 2 * gc, Sc2 = Sc * Sc, Sc3 = Sc2 * Sc;
    const int h = n >> 1;
    const int P = lk.parent[b];
    if (threadIdx.x < 27) {
        snbr[threadIdx.x] = lk.nbr[27 * b + threadIdx.x];
        cnbr[threadIdx.x] = P >= 0 ? lc.nbr[27 * P + threadIdx.x] : -1;
    }
    if (threadIdx.x < I) sw[threadIdx.x] = iw.w[threadIdx.x];
    if (threadIdx.x == 0) interp = 0;
    __syncthreads();
    if (threadIdx.x < 27 && threadIdx.x != 13 && snbr[threadIdx.x] == NBR_MISSING) interp = 1;
    __syncthreads();
    double* Ab = A + (size_t)b * S3;
    const int bx = lk.coords[3 * b], by = lk.coords[3 * b + 1], bz = lk.coords[3 * b + 2];
    const int PL = h + g + I + 1, PL2 = PL * PL;
    const int pb[3] = {(bx & 1) * h - (g + 1) / 2 - I / 2, (by & 1) * h - (g + 1) / 2 - I / 2,
                       (bz & 1) * h - (g + 1) / 2 - I / 2};
    if (interp) {
        for (int t = threadIdx.x; t < PL2 * PL; t += blockDim.x) {
            const int r[3] = {pb[0] + t % PL, pb[1] + (t / PL) % PL, pb[2] + t / PL2};
            int e[3], l[3];
            for (int a = 0; a < 3; ++a) { e[a] = r[a] < 0 ? -1 : (r[a] >= n ? 1 : 0); l[a] = r[a] - e[a] * n; }
            const int cb = cnbr[dir27(e[0], e[1], e[2])];
            gpatch[t] = cb >= 0 ? Ac[(size_t)cb * Sc3 + (size_t)((gc + l[2]) * Sc + gc + l[1]) * Sc + gc + l[0]] : 0.0;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < S3; t += blockDim.x) {
        const int x = t % S, y = (t / S) % S, z = t / S2;
        const int dx = x < g ? -1 : (x >= g + n ? 1 : 0);
        const int dy = y < g ? -1 : (y >= g + n ? 1 : 0);
        const int dz = z < g ? -1 : (z >= g + n ? 1 : 0);
        if ((dx | dy | dz) == 0) continue;
        const int j = snbr[dir27(dx, dy, dz)];
        if (j >= 0) {
            Ab[t] = A[(size_t)j * S3 + (size_t)((z - dz * n) * S + (y - dy * n)) * S + (x - dx * n)];
            continue;
        }
        if (j == NBR_OUTSIDE) {
            if (zero_outside) Ab[t] = 0.0;
            continue;
        }
        // interpolation from level k-1 (parent-local coarse indices, then patch indices)
        const int p[3] = {bx * n + x - g, by * n + y - g, bz * n + z - g};
        const int porig[3] = {(bx >> 1) * n, (by >> 1) * n, (bz >> 1) * n};
        int cnt[3], c0[3];
        for (int a = 0; a < 3; ++a) {
            if ((p[a] & 1) == 0) { cnt[a] = 1; c0[a] = (p[a] >> 1) - porig[a] - pb[a]; }
            else { cnt[a] = I; c0[a] = ((p[a] - 1) >> 1) - I / 2 + 1 - porig[a] - pb[a]; }
        }
        double accz = 0.0;
        for (int mz = 0; mz < cnt[2]; ++mz) {
            double accy = 0.0;
            for (int my = 0; my < cnt[1]; ++my) {
                const double* row = gpatch + ((c0[2] + mz) * PL + c0[1] + my) * PL + c0[0];
                double accx;
                if (cnt[0] == 1) {
                    accx = row[0];
                } else {
                    double v[I];
#pragma unroll
                    for (int mx = 0; mx < I; ++mx) v[mx] = row[mx];
                    accx = 0.0;
#pragma unroll
                    for (int mx = 0; mx < I; ++mx) accx += sw[mx] * v[mx];
                }
                accy += (cnt[1] == 1 ? 1.0 : sw[my]) * accx;
            }
            accz += (cnt[2] == 1 ? 1.0 : sw[mz]) * accy;
        }
        Ab[t] = accz;
    }
}

// Separable form of the same ghost layer: the interpolant is evaluated over
// the whole (n+2g)^3 box in three passes from the staged patch, along x
// (fine x, coarse y, z), along y (fine x, y, coarse z) and along z (fine
// nodes of the interpolated regions only); the sums nest in the tensor
// kernel's order (x innermost, then y, then z).  Each pass takes its items
// with the parity of the interpolated coordinate slowest, so the lanes of a
// warp share the stencil length (I points at an odd fine coordinate, one
// coincident node at an even one).  Work arrays: wa (patch, then the y pass)
// and wb (the x pass).
__host__ __device__ inline int gsep_wa(int n, int g, int I) {
    const int S = n + 2 * g, PL = n / 2 + g + I + 1;
    return PL * PL * PL > S * S * PL ? PL * PL * PL : S * S * PL;
}
__host__ __device__ inline int gsep_wb(int n, int g, int I) {
    const int S = n + 2 * g, PL = n / 2 + g + I + 1;
    return S * PL * PL;
}

template <int I>
__global__ void k_ghost_fill_sep(double* __restrict__ A, int g, const double* __restrict__ Ac, int gc, LevelView lk,
                                 LevelView lc, int n, InterpW iw, bool zero_outside) {
    extern __shared__ double gsm[];
    __shared__ int snbr[27], cnbr[27];
    __shared__ int interp;
    const int b = blockIdx.x;
    const int S = n + 2 * g, S2 = S * S, S3 = S2 * S;
    const int Sc = n + 2 * gc, Sc2 = Sc * Sc, Sc3 = Sc2 * Sc;
    const int h = n >> 1, Sh = S >> 1;
    const int P = lk.parent[b];
    if (threadIdx.x < 27) {
        snbr[threadIdx.x] = lk.nbr[27 * b + threadIdx.x];
        cnbr[threadIdx.x] = P >= 0 ? lc.nbr[27 * P + threadIdx.x] : -1;
    }
    if (threadIdx.x == 0) interp = 0;
    __syncthreads();
    if (threadIdx.x < 27 && threadIdx.x != 13 && snbr[threadIdx.x] == NBR_MISSING) interp = 1;
    double w[I];
#pragma unroll
    for (int m = 0; m < I; ++m) w[m] = iw.w[m];
    double* Ab = A + (size_t)b * S3;
    const unsigned mS = magic_of(S), mSh = magic_of(Sh);
    // copied and outside regions
    for (int t = threadIdx.x; t < S3; t += blockDim.x) {
        const int zy = fdiv(t, mS), x = t - zy * S, z = fdiv(zy, mS), y = zy - z * S;
        const int dx = x < g ? -1 : (x >= g + n ? 1 : 0);
        const int dy = y < g ? -1 : (y >= g + n ? 1 : 0);
        const int dz = z < g ? -1 : (z >= g + n ? 1 : 0);
        if ((dx | dy | dz) == 0) continue;
        const int j = snbr[dir27(dx, dy, dz)];
        if (j >= 0) Ab[t] = A[(size_t)j * S3 + (size_t)((z - dz * n) * S + (y - dy * n)) * S + (x - dx * n)];
        else if (j == NBR_OUTSIDE && zero_outside) Ab[t] = 0.0;
    }
    __syncthreads();
    if (!interp) return;
    const int bx = lk.coords[3 * b], by = lk.coords[3 * b + 1], bz = lk.coords[3 * b + 2];
    const int PL = h + g + I + 1, PL2 = PL * PL;
    const int pb0 = (bx & 1) * h - (g + 1) / 2 - I / 2, pb1 = (by & 1) * h - (g + 1) / 2 - I / 2,
              pb2 = (bz & 1) * h - (g + 1) / 2 - I / 2;
    double* wa = gsm;
    double* wb = gsm + gsep_wa(n, g, I);
    const unsigned mPL = magic_of(PL);
    for (int t = threadIdx.x; t < PL2 * PL; t += blockDim.x) {
        const int q = fdiv(t, mPL), px = t - q * PL, pz = fdiv(q, mPL), py = q - pz * PL;
        const int r0 = pb0 + px, r1 = pb1 + py, r2 = pb2 + pz;
        const int e0 = r0 < 0 ? -1 : (r0 >= n ? 1 : 0), e1 = r1 < 0 ? -1 : (r1 >= n ? 1 : 0),
                  e2 = r2 < 0 ? -1 : (r2 >= n ? 1 : 0);
        const int cb = cnbr[dir27(e0, e1, e2)];
        wa[t] = cb >= 0 ? Ac[(size_t)cb * Sc3 + (size_t)((gc + r2 - e2 * n) * Sc + gc + r1 - e1 * n) * Sc + gc + r0 - e0 * n]
                        : 0.0;
    }
    __syncthreads();
    // Patch index of the first stencil node of box coordinate X on an axis
    // whose block origin is bo (fine) and patch base pb: fine coordinate
    // p = bo + X - g; even p: node p/2, odd p: I nodes from (p-1)/2 - I/2 + 1;
    // both relative to the parent's origin (bo >> 1 rounded to the parent) and pb.
    auto start = [&](int bo, int X, int pbase) {
        const int p = bo + X - g, porig = ((bo / n) >> 1) * n;
        return ((p & 1) == 0 ? (p >> 1) : ((p - 1) >> 1) - I / 2 + 1) - porig - pbase;
    };
    // x pass: wb[(cz PL + cy) S + X]
    for (int t = threadIdx.x; t < S * PL2; t += blockDim.x) {
        const int par = t >= Sh * PL2;
        const int e = t - par * Sh * PL2;
        const int q = fdiv(e, mSh), Xh = e - q * Sh;          // q = cz PL + cy
        const int X = 2 * Xh + par;
        const double* row = wa + q * PL + start(bx * n, X, pb0);
        double acc;
        if (!par) acc = row[0];
        else {
            acc = 0.0;
#pragma unroll
            for (int m = 0; m < I; ++m) acc += w[m] * row[m];
        }
        wb[q * S + X] = acc;
    }
    __syncthreads();
    // y pass: wa[(cz S + Y) S + X]
    for (int t = threadIdx.x; t < S2 * PL; t += blockDim.x) {
        const int par = t >= Sh * S * PL;
        const int e = t - par * Sh * S * PL;
        const int q = fdiv(e, mS), X = e - q * S;               // q = cz Sh + Yh
        const int cz = fdiv(q, mSh), Yh = q - cz * Sh;
        const int Y = 2 * Yh + par;
        const double* col = wb + (cz * PL + start(by * n, Y, pb1)) * S + X;
        double acc;
        if (!par) acc = col[0];
        else {
            acc = 0.0;
#pragma unroll
            for (int m = 0; m < I; ++m) acc += w[m] * col[m * S];
        }
        wa[(cz * S + Y) * S + X] = acc;
    }
    __syncthreads();
    // z pass on the interpolated regions
    for (int t = threadIdx.x; t < S3; t += blockDim.x) {
        const int par = t >= Sh * S2;
        const int e = t - par * Sh * S2;
        const int q = fdiv(e, mS), X = e - q * S;               // q = Zh S + Y
        const int Zh = fdiv(q, mS), Y = q - Zh * S;
        const int Z = 2 * Zh + par;
        const int dx = X < g ? -1 : (X >= g + n ? 1 : 0);
        const int dy = Y < g ? -1 : (Y >= g + n ? 1 : 0);
        const int dz = Z < g ? -1 : (Z >= g + n ? 1 : 0);
        if ((dx | dy | dz) == 0 || snbr[dir27(dx, dy, dz)] != NBR_MISSING) continue;
        const double* col = wa + start(bz * n, Z, pb2) * S2 + Y * S + X;
        double acc;
        if (!par) acc = col[0];
        else {
            acc = 0.0;
#pragma unroll
            for (int m = 0; m < I; ++m) acc += w[m] * col[m * S2];
        }
        Ab[(Z * S + Y) * S + X] = acc;
    }
}

void launch_ghost_fill(double* A, int g, const double* Ac, int gc, LevelView lk, LevelView lkm1, int n, int M,
                       bool zero_outside, cudaStream_t s) {
    if (lk.nb == 0) return;
    {
        const int I = M + 2;
        const size_t sm = sizeof(double) * ((size_t)gsep_wa(n, g, I) + (size_t)gsep_wb(n, g, I));
        if (g % 2 == 0 && sm <= (size_t)MAX_DYN_SMEM) {
            static std::once_flag attr_sep[MAX_DEVICES];
            once_per_device(attr_sep, [] {
                cudaFuncSetAttribute(k_ghost_fill_sep<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
                cudaFuncSetAttribute(k_ghost_fill_sep<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
                cudaFuncSetAttribute(k_ghost_fill_sep<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
            });
            const InterpW iw = interp_weights(M);
            if (I == 4) k_ghost_fill_sep<4><<<lk.nb, 256, sm, s>>>(A, g, Ac, gc, lk, lkm1, n, iw, zero_outside);
            if (I == 6) k_ghost_fill_sep<6><<<lk.nb, 256, sm, s>>>(A, g, Ac, gc, lk, lkm1, n, iw, zero_outside);
            if (I == 8) k_ghost_fill_sep<8><<<lk.nb, 256, sm, s>>>(A, g, Ac, gc, lk, lkm1, n, iw, zero_outside);
            return;
        }
    }
    if (lk.nb == 0) return;
    const InterpW iw = interp_weights(M);
    const int PL = n / 2 + g + iw.I + 1;
    const size_t sm = sizeof(double) * PL * PL * PL;
    static std::once_flag attr[MAX_DEVICES];
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_ghost_fill<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_ghost_fill<6>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_ghost_fill<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    });
    if (iw.I == 4) k_ghost_fill<4><<<lk.nb, 256, sm, s>>>(A, g, Ac, gc, lk, lkm1, n, iw, zero_outside);
    if (iw.I == 6) k_ghost_fill<6><<<lk.nb, 256, sm, s>>>(A, g, Ac, gc, lk, lkm1, n, iw, zero_outside);
    if (iw.I == 8) k_ghost_fill<8><<<lk.nb, 256, sm, s>>>(A, g, Ac, gc, lk, lkm1, n, iw, zero_outside);
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
    // one thread per (x, y) column walking z; the weights are multiplied
    // (reciprocals of 12, 18, 90, 240 rounded once), not divided
    for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
        const int y = c / n, x = c - y * n;
        for (int z = 0; z < n; ++z) {
            const int o = ((z + 2) * S + y + 2) * S + x + 2;
            double v;
            if (M == 2) {
                v = a[o];
            } else {
                const double sf = (a[o - 1] + a[o + 1]) + (a[o - S] + a[o + S]) + (a[o - S2] + a[o + S2]);
                if (M == 4) {
                    v = 0.5 * a[o] + sf * (1.0 / 12.0);
                } else {
                    const double se = (a[o - 1 - S] + a[o + 1 - S]) + (a[o - 1 + S] + a[o + 1 + S])
                                    + (a[o - 1 - S2] + a[o + 1 - S2]) + (a[o - 1 + S2] + a[o + 1 + S2])
                                    + (a[o - S - S2] + a[o + S - S2]) + (a[o - S + S2] + a[o + S + S2]);
                    const double s2 =
                        (a[o - 2] + a[o + 2]) + (a[o - 2 * S] + a[o + 2 * S]) + (a[o - 2 * S2] + a[o + 2 * S2]);
                    v = (67.0 / 120.0) * a[o] + sf * (1.0 / 18.0) + se * (1.0 / 90.0) - s2 * (1.0 / 240.0);
                }
            }
            out[(z * n + y) * n + x] = v;
        }
    }
}

void launch_rhs_star(double* F, const double* Fraw, const int* leaf_blocks, int nleaf, int n, int M, cudaStream_t s) {
    if (nleaf == 0) return;
    if (M == 2) k_rhs_star<2><<<nleaf, 256, 0, s>>>(F, Fraw, leaf_blocks, n);
    if (M == 4) k_rhs_star<4><<<nleaf, 256, 0, s>>>(F, Fraw, leaf_blocks, n);
    if (M == 6) k_rhs_star<6><<<nleaf, 256, 0, s>>>(F, Fraw, leaf_blocks, n);
}

// ----------------------------------------------------------------------------
// Restriction from level k to the covered blocks of level k-1 (Alg. 1):
// u_{k-1} = injection of u_k;  r_{k-1} = full weighting (1/4)[1 2 1]^3 of r_k,
// or injection where the 27-point stencil reaches outside Omega_k.  The
// restricted residual is left in F_{k-1}; the FAS kernel adds L u_{k-1}.
// One CTA per level-k block B computes the (n/2)^3 coarse nodes whose fine
// image 2X lies in B: it stages r_k on B's nodes and on the planes just below
// them (local coordinates -1 .. n-1, from the lower neighbours); the window
// of X is complete when those neighbours exist along the axes where 2X sits
// on B's lower face (the upper side always lies in B).
// Row stride of the restriction's residual window: at least n + 1 (the
// n/2 + 1 even and n/2 odd columns of a row), and 4 (mod 16), so that a warp
// of 8 consecutive coarse i by 4 consecutive j reads 32 distinct banks.
__host__ __device__ inline int restrict_row(int n) {
    int r = n + 1;
    while (r % 16 != 4) ++r;
    return r;
}

template <typename T, int NC>
__global__ void k_restrict(T* __restrict__ Uc, T* __restrict__ Fc, const T* __restrict__ Uf, const T* __restrict__ Rf,
                           LevelView lf, int n_arg, const T* __restrict__ off) {
    const int n = NC ? NC : n_arg;    // NC: block size fixed at compile time (0: runtime)
    extern __shared__ __align__(16) unsigned char rs_raw[];
    T* sr = reinterpret_cast<T*>(rs_raw);
    __shared__ int nb27[27];
    __shared__ int ins[8];
    const int B = blockIdx.x;
    if (threadIdx.x < 27) nb27[threadIdx.x] = lf.nbr[27 * B + threadIdx.x];
    __syncthreads();
    if (threadIdx.x < 8) {
        const int m = threadIdx.x;
        int ok = 1;
        for (int sz = 0; sz <= ((m >> 2) & 1); ++sz)
            for (int sy = 0; sy <= ((m >> 1) & 1); ++sy)
                for (int sx = 0; sx <= (m & 1); ++sx)
                    if (nb27[dir27(-sx, -sy, -sz)] < 0) ok = 0;
        ins[m] = ok;
    }
    const int N1 = n + 1, n3 = n * n * n, h = n >> 1;
    // the residual window, fine nodes [-1, n)^3 (window coordinates X = x + 1
    // etc.), split by the parity of X within each row (see restrict_rows), so
    // that the full weighting's reads at X = 2i, 2i + 1, 2i + 2 of a warp's
    // consecutive i are consecutive words; one thread per (X, Y) column walking
    // Z (cp.async); nodes of missing neighbours read as 0
    const int RR = restrict_row(n), OE = h + 1, PR = RR * N1;
    auto wi = [&](int X, int Y, int Z) { return Z * PR + Y * RR + (X & 1) * OE + (X >> 1); };
    for (int c = threadIdx.x; c < N1 * N1; c += blockDim.x) {
        const int Y = c / N1, X = c - Y * N1, x = X - 1, y = Y - 1;
        const int ex = x < 0 ? -1 : 0, ey = y < 0 ? -1 : 0;
        T* dcol = sr + wi(X, Y, 0);
        for (int ez = -1; ez <= 0; ++ez) {
            const int blk = nb27[dir27(ex, ey, ez)];
            const int z0 = ez < 0 ? -1 : 0, z1 = ez < 0 ? 0 : n;
            const T* scol = Rf + (blk >= 0 ? (size_t)blk * n3 + (size_t)((y - ey * n) * n + (x - ex * n)) : 0);
            for (int z = z0; z < z1; ++z) {
                if (blk >= 0) cp_async_el(dcol + (z + 1) * PR, scol + (size_t)(z - ez * n) * n * n);
                else dcol[(z + 1) * PR] = T(0);
            }
        }
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    const int P = lf.parent[B], o = lf.octant[B];
    const int ox = (o & 1) * h, oy = ((o >> 1) & 1) * h, oz = ((o >> 2) & 1) * h;
    const int S = n + 2, S3 = S * S * S;
    const unsigned mh = magic_of(h);
    for (int q = threadIdx.x; q < h * h * h; q += blockDim.x) {
        const int q1 = NC ? q / h : fdiv(q, mh), i = q - q1 * h, l = NC ? q1 / h : fdiv(q1, mh), j = q1 - l * h;
        const int fx = 2 * i, fy = 2 * j, fz = 2 * l;
        const int cidx = ((oz + l) * n + oy + j) * n + ox + i;
        Uc[(size_t)P * S3 + ((oz + l + 1) * S + oy + j + 1) * S + ox + i + 1] =
            Uf[(size_t)B * S3 + ((fz + 1) * S + fy + 1) * S + fx + 1] + (off ? off[(size_t)P * n3 + cidx] : T(0));
        // window X = fx + 1 = 2i + 1 (odd half, index i); its x neighbours are
        // X = 2i, 2i + 2 (even half, indices i, i + 1)
        const T* c = sr + wi(fx + 1, fy + 1, fz + 1);
        const T* ce = sr + wi(fx, fy + 1, fz + 1);
        T v;
        if (ins[(fx == 0) | ((fy == 0) << 1) | ((fz == 0) << 2)]) {
            T acc = T(0);
            for (int dz = -1; dz <= 1; ++dz) {
                T accy = T(0);
                for (int dy = -1; dy <= 1; ++dy) {
                    const int d = dz * PR + dy * RR;
                    accy += T(2 - (dy < 0 ? -dy : dy)) * (ce[d] + T(2) * c[d] + ce[d + 1]);
                }
                acc += T(2 - (dz < 0 ? -dz : dz)) * accy;
            }
            v = acc * T(1.0 / 64.0);
        } else {
            v = c[0];
        }
        Fc[(size_t)P * n3 + cidx] = v;
    }
}

template <typename T>
void launch_restrict(T* Uc, T* Fc, const T* Uf, const T* Rf, LevelView lf, int n, const T* off, cudaStream_t s) {
    if (lf.nb == 0) return;
    static std::once_flag attr[MAX_DEVICES];
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_restrict<T, NC_FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_restrict<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    });
    const size_t sm = sizeof(T) * (size_t)restrict_row(n) * (n + 1) * (n + 1);
    if (n == NC_FIXED) k_restrict<T, NC_FIXED><<<lf.nb, 256, sm, s>>>(Uc, Fc, Uf, Rf, lf, n, off);
    else k_restrict<T, 0><<<lf.nb, 256, sm, s>>>(Uc, Fc, Uf, Rf, lf, n, off);
}
template void launch_restrict<double>(double*, double*, const double*, const double*, LevelView, int, const double*,
                                      cudaStream_t);
template void launch_restrict<float>(float*, float*, const float*, const float*, LevelView, int, const float*, cudaStream_t);

// ----------------------------------------------------------------------------
// Coarse-grid correction (Alg. 1): eps = u_{k-1} - uhat_{k-1} on the coarse
// nodes of the fine block's extent plus the next coarse node on each upper
// side, then u_k += trilinear(eps).
template <typename T, int NC>
__global__ void k_prolong(T* __restrict__ Uf, const T* __restrict__ Uc, const T* __restrict__ Hc, LevelView lf,
                          LevelView lc, int n_arg) {
    const int n = NC ? NC : n_arg;    // NC: block size fixed at compile time (0: runtime)
    extern __shared__ unsigned char smem_raw[];
    T* e = reinterpret_cast<T*>(smem_raw);
    const int B = blockIdx.x;
    const int P = lf.parent[B], o = lf.octant[B];
    const int h = n >> 1, E = h + 1;
    const int S = n + 2, S3 = S * S * S, n3 = n * n * n;
    const int ox = (o & 1) * h, oy = ((o >> 1) & 1) * h, oz = ((o >> 2) & 1) * h;
    const int* cn = lc.nbr + 27 * P;
    const unsigned mE = magic_of(E);
    for (int t = threadIdx.x; t < E * E * E; t += blockDim.x) {
        const int t1 = NC ? t / E : fdiv(t, mE), i = t - t1 * E, l = NC ? t1 / E : fdiv(t1, mE), j = t1 - l * E;
        const int cx = ox + i, cy = oy + j, cz = oz + l;
        const int ex = cx >= n, ey = cy >= n, ez = cz >= n;
        const int blk = cn[dir27(ex, ey, ez)];
        const int lx = cx - ex * n, ly = cy - ey * n, lz = cz - ez * n;
        e[t] = Uc[(size_t)blk * S3 + ((lz + 1) * S + ly + 1) * S + lx + 1] - Hc[(size_t)blk * n3 + (lz * n + ly) * n + lx];
    }
    __syncthreads();
    // one thread per fine (x, y) column: the x-then-y interpolant of each
    // coarse plane, then z (coincident plane, or the midpoint of two)
    T* Ub = Uf + (size_t)B * S3;
    const int S2 = S * S;
    for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
        const int y = c / n, x = c - y * n;
        const int ax = x >> 1, ay = y >> 1, bx = x & 1, by = y & 1;
        // bilinear value at (x, y): rows ay and ay + by, columns ax and ax + bx;
        // on a coincident axis both indices are equal and the halving undoes
        // the doubling exactly
        auto plane = [&](int az) {
            const T* r0 = e + (az * E + ay) * E + ax;
            const T* r1 = r0 + by * E;
            return T(0.25) * ((r0[0] + r0[bx]) + (r1[0] + r1[bx]));
        };
        T cur = plane(0);
        if constexpr (sizeof(T) == 4) {
            // FP32: the corrections go to shared memory first (below)
            T* cc = e + E * E * E + c;
            for (int az = 0; az < h; ++az) {
                const T nxt = plane(az + 1);
                cc[(2 * az) * n * n] = cur;
                cc[(2 * az + 1) * n * n] = T(0.5) * (cur + nxt);
                cur = nxt;
            }
        } else {
            T* col = Ub + (y + 1) * S + x + 1;
            for (int az = 0; az < h; ++az) {
                const T nxt = plane(az + 1);
                col[(2 * az + 1) * S2] += cur;
                col[(2 * az + 2) * S2] += T(0.5) * (cur + nxt);
                cur = nxt;
            }
        }
    }
    if constexpr (sizeof(T) == 4) {
        // FP32: u += correction over the whole planes z = 1..n of the block's
        // box with 16-byte accesses (S^2 is a multiple of 4 for even n), whole
        // 32-byte sectors and independent loads; ghost entries add nothing
        __syncthreads();
        const T* corr = e + E * E * E;
        float4* p = reinterpret_cast<float4*>(Ub + S2);
        auto add = [&](float& v, int X, int Y, int Zr) {
            if (X >= 1 && X <= n && Y >= 1 && Y <= n) v += corr[(Zr * n + Y - 1) * n + X - 1];
        };
        const int NV = n * S2 / 4;
        for (int t = threadIdx.x; t < NV; t += blockDim.x) {
            const int q = 4 * t, Zr = q / S2, r = q - Zr * S2, Y = r / S, X = r - Y * S;
            float4 v = p[t];
            add(v.x, X, Y, Zr);
            add(v.y, X + 1, Y, Zr);
            if (X + 2 < S) {
                add(v.z, X + 2, Y, Zr);
                add(v.w, X + 3, Y, Zr);
            } else {             // the row ends: columns 0 and 1 of the next row (never the next plane)
                add(v.z, 0, Y + 1, Zr);
                add(v.w, 1, Y + 1, Zr);
            }
            p[t] = v;
        }
    }
}

template <typename T>
void launch_prolong(T* Uf, const T* Uc, const T* Hc, LevelView lf, LevelView lc, int n, cudaStream_t s) {
    if (lf.nb == 0) return;
    const int E = n / 2 + 1;
    // FP32 adds an n^3 buffer of corrections (64 KB at n = 24: opt-in size)
    const size_t sm = sizeof(T) * ((size_t)E * E * E + (sizeof(T) == 4 ? (size_t)n * n * n : 0));
    static std::once_flag attr[MAX_DEVICES];
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_prolong<T, NC_FIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_prolong<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    });
    if (n == NC_FIXED) k_prolong<T, NC_FIXED><<<lf.nb, 256, sm, s>>>(Uf, Uc, Hc, lf, lc, n);
    else k_prolong<T, 0><<<lf.nb, 256, sm, s>>>(Uf, Uc, Hc, lf, lc, n);
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
    // max |v| on bit patterns (integer pipe): ordered like the values for
    // non-negative doubles; NaN patterns sort above +Inf and become +Inf
    unsigned long long mb = 0;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const unsigned long long v = (unsigned long long)__double_as_longlong(F[(size_t)b * n3 + t]) & 0x7fffffffffffffffULL;
        mb = v > mb ? v : mb;
    }
    const double m = mb > 0x7ff0000000000000ULL ? __longlong_as_double(0x7ff0000000000000ULL) : __longlong_as_double((long long)mb);
    block_max_atomic(m, out + (prob ? prob[b] : 0));
}

void launch_absmax(const double* F, const int* blocks, int nblocks, int n, unsigned long long* out, const int* prob,
                   cudaStream_t s) {
    if (nblocks == 0) return;
    k_absmax<<<nblocks, 256, 0, s>>>(F, blocks, n, out, prob);
}

}  // namespace mrp
