// Ghosting of u (one ghost layer), arXiv 2512.08555 Sec. 2.1.
//
// One CTA per level-k block.  Halo regions whose same-level neighbour exists
// are copied from it.  The others are reconstructed from level k-1 by the
// I-point (I = M + 2) tensor-product Lagrange interpolant, evaluated
// separably: the coarse patch around the block is staged in shared memory,
// each interpolated region is first reduced along its normal axes (a plane
// for a face, a line for an edge, a value for a corner), then each ghost node
// takes the tangential interpolant of that reduced array.  The covered coarse
// nodes of the patch hold the injection of the current fine values (the
// caller injects first).
//
// Patch coordinates: patch index 4 + floor(q/2) is the coarse node left of
// (or at) fine local coordinate q of this block, q in [-1, n]; the patch
// spans n/2 + 9 coarse nodes per axis.
#include "mrp_internal.h"

namespace mrp {

// Midpoint weights of the I-point Lagrange interpolant (I = M + 2).
template <int I> struct MidW;
template <> struct MidW<4> {
    static __device__ double w(int m) { return (m == 0 || m == 3 ? -1.0 : 9.0) / 16.0; }
};
template <> struct MidW<6> {
    static __device__ double w(int m) { return (m == 0 || m == 5 ? 3.0 : (m == 1 || m == 4 ? -25.0 : 150.0)) / 256.0; }
};
template <> struct MidW<8> {
    static __device__ double w(int m) {
        const int k = m < 4 ? m : 7 - m;
        return (k == 0 ? -5.0 : (k == 1 ? 49.0 : (k == 2 ? -245.0 : 1225.0))) / 2048.0;
    }
};

// Shell enumeration of an S^3 box without its (S-2)^3 interior.
__device__ __forceinline__ void shell_xyz(int t, int S, int& x, int& y, int& z) {
    const int S2 = S * S;
    if (t < S2) { z = 0; y = t / S; x = t % S; return; }
    t -= S2;
    if (t < S2) { z = S - 1; y = t / S; x = t % S; return; }
    t -= S2;
    const int ring = 4 * S - 4;
    z = 1 + t / ring;
    int r = t % ring;
    if (r < S) { y = 0; x = r; return; }
    r -= S;
    if (r < S) { y = S - 1; x = r; return; }
    r -= S;
    y = 1 + (r >> 1);
    x = (r & 1) ? S - 1 : 0;
}

template <typename T, int I>
__global__ void __launch_bounds__(256) k_ghost_u(T* __restrict__ A, const T* __restrict__ Ac, LevelView lk, LevelView lc, int n) {
    extern __shared__ unsigned char smem_raw[];
    T* patch = reinterpret_cast<T*>(smem_raw);
    __shared__ int snbr[27];
    __shared__ int cnbr[27];
    __shared__ int off[27];
    __shared__ T sw[8];
    const int b = blockIdx.x;
    if (threadIdx.x < I) sw[threadIdx.x] = T(MidW<I>::w(threadIdx.x));
    const int S = n + 2, S2 = S * S, S3 = S2 * S;
    const int C = n / 2 + 9, C2 = C * C, C3 = C2 * C;
    if (threadIdx.x < 27) snbr[threadIdx.x] = lk.nbr[27 * b + threadIdx.x];
    __syncthreads();
    bool interp = false;
    for (int d = 0; d < 27; ++d) interp |= (d != 13 && snbr[d] == NBR_MISSING);
    T* Ab = A + (size_t)b * S3;
    const int shell = S3 - n * n * n;
    // same-level copies
    for (int t = threadIdx.x; t < shell; t += blockDim.x) {
        int x, y, z;
        shell_xyz(t, S, x, y, z);
        const int dx = x == 0 ? -1 : (x == S - 1 ? 1 : 0);
        const int dy = y == 0 ? -1 : (y == S - 1 ? 1 : 0);
        const int dz = z == 0 ? -1 : (z == S - 1 ? 1 : 0);
        const int j = snbr[dir27(dx, dy, dz)];
        if (j >= 0) Ab[(z * S + y) * S + x] = A[(size_t)j * S3 + ((z - dz * n) * S + (y - dy * n)) * S + (x - dx * n)];
    }
    if (!interp) return;
    // stage the coarse patch
    const int P = lk.parent[b];
    if (threadIdx.x < 27) cnbr[threadIdx.x] = lc.nbr[27 * P + threadIdx.x];
    if (threadIdx.x == 0) {
        int o = C3;
        for (int d = 0; d < 27; ++d) {
            off[d] = o;
            if (d == 13 || snbr[d] != NBR_MISSING) continue;
            const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
            const int nt = (dx == 0) + (dy == 0) + (dz == 0);
            o += nt == 2 ? C2 : (nt == 1 ? C : 1);
        }
    }
    __syncthreads();
    const int bx = lk.coords[3 * b], by = lk.coords[3 * b + 1], bz = lk.coords[3 * b + 2];
    const int h = n >> 1;
    const int basex = (bx & 1) * h - 4, basey = (by & 1) * h - 4, basez = (bz & 1) * h - 4;
    const int Sc = n + 2, Sc3 = Sc * Sc * Sc;
    for (int t = threadIdx.x; t < C3; t += blockDim.x) {
        const int px = t % C, py = (t / C) % C, pz = t / C2;
        const int rx = basex + px, ry = basey + py, rz = basez + pz;
        const int ex = rx < 0 ? -1 : (rx >= n ? 1 : 0);
        const int ey = ry < 0 ? -1 : (ry >= n ? 1 : 0);
        const int ez = rz < 0 ? -1 : (rz >= n ? 1 : 0);
        const int blk = cnbr[dir27(ex, ey, ez)];
        patch[t] = Ac[(size_t)blk * Sc3 + ((rz - ez * n + 1) * Sc + (ry - ey * n + 1)) * Sc + (rx - ex * n + 1)];
    }
    __syncthreads();
    // phase 1: reduce every interpolated region along its normal axes
    constexpr int lo = 4 - I / 2;              // first patch index of the stencil around fine local -1
    const int up = 4 + h;                      // patch index coincident with fine local n
    for (int d = 0; d < 27; ++d) {
        if (d == 13 || snbr[d] != NBR_MISSING) continue;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        const int nt = (dx == 0) + (dy == 0) + (dz == 0);
        const int size = nt == 2 ? C2 : (nt == 1 ? C : 1);
        T* R = patch + off[d];
        for (int e = threadIdx.x; e < size; e += blockDim.x) {
            // tangential patch coordinates in x, y, z order
            int tc[3] = {0, 0, 0};
            int rem = e;
            if (dx == 0) { tc[0] = rem % C; rem /= C; }
            if (dy == 0) { tc[1] = rem % C; rem /= C; }
            if (dz == 0) { tc[2] = rem % C; }
            const int cntx = dx < 0 ? I : 1, cnty = dy < 0 ? I : 1, cntz = dz < 0 ? I : 1;
            const int x0 = dx < 0 ? lo : (dx > 0 ? up : tc[0]);
            const int y0 = dy < 0 ? lo : (dy > 0 ? up : tc[1]);
            const int z0 = dz < 0 ? lo : (dz > 0 ? up : tc[2]);
            T acc = T(0);
            for (int mz = 0; mz < cntz; ++mz) {
                T ay = T(0);
                for (int my = 0; my < cnty; ++my) {
                    T ax = T(0);
                    const T* row = patch + ((z0 + mz) * C + y0 + my) * C + x0;
                    for (int mx = 0; mx < cntx; ++mx) ax += (cntx == 1 ? T(1) : sw[mx]) * row[mx];
                    ay += (cnty == 1 ? T(1) : sw[my]) * ax;
                }
                acc += (cntz == 1 ? T(1) : sw[mz]) * ay;
            }
            R[e] = acc;
        }
    }
    __syncthreads();
    // phase 2: tangential interpolation from the reduced arrays
    for (int t = threadIdx.x; t < shell; t += blockDim.x) {
        int x, y, z;
        shell_xyz(t, S, x, y, z);
        const int dx = x == 0 ? -1 : (x == S - 1 ? 1 : 0);
        const int dy = y == 0 ? -1 : (y == S - 1 ? 1 : 0);
        const int dz = z == 0 ? -1 : (z == S - 1 ? 1 : 0);
        const int d = dir27(dx, dy, dz);
        if (snbr[d] != NBR_MISSING) continue;
        const T* R = patch + off[d];
        // tangential axes: (start patch index, count) and stride in R
        int st[2] = {0, 0}, cn[2] = {1, 1}, sd[2] = {0, 0};
        int nt = 0, stride = 1;
        const int q[3] = {x - 1, y - 1, z - 1};
        const int dd[3] = {dx, dy, dz};
        for (int a = 0; a < 3; ++a) {
            if (dd[a] != 0) continue;
            const int qa = q[a];
            if (qa & 1) { st[nt] = 4 + ((qa - 1) >> 1) - I / 2 + 1; cn[nt] = I; }
            else { st[nt] = 4 + (qa >> 1); cn[nt] = 1; }
            sd[nt] = stride;
            stride *= C;
            ++nt;
        }
        T acc = T(0);
        for (int m1 = 0; m1 < cn[1]; ++m1) {
            T a0 = T(0);
            const int base = (st[1] + m1) * sd[1] + st[0] * sd[0];
            for (int m0 = 0; m0 < cn[0]; ++m0) a0 += (cn[0] == 1 ? T(1) : sw[m0]) * R[base + m0 * sd[0]];
            acc += (cn[1] == 1 ? T(1) : sw[m1]) * a0;
        }
        Ab[(z * S + y) * S + x] = acc;
    }
}

template <typename T>
static size_t ghost_u_smem(int n) {
    const int C = n / 2 + 9;
    return sizeof(T) * ((size_t)C * C * C + 6 * C * C + 12 * C + 8);
}

template <typename T>
void launch_ghost_u(T* A, const T* Ac, LevelView lk, LevelView lkm1, int n, int M, cudaStream_t s) {
    if (lk.nb == 0) return;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_ghost_u<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_ghost_u<T, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_ghost_u<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        attr = true;
    }
    const size_t sm = ghost_u_smem<T>(n);
    if (M == 2) k_ghost_u<T, 4><<<lk.nb, 256, sm, s>>>(A, Ac, lk, lkm1, n);
    if (M == 4) k_ghost_u<T, 6><<<lk.nb, 256, sm, s>>>(A, Ac, lk, lkm1, n);
    if (M == 6) k_ghost_u<T, 8><<<lk.nb, 256, sm, s>>>(A, Ac, lk, lkm1, n);
}
template void launch_ghost_u<double>(double*, const double*, LevelView, LevelView, int, int, cudaStream_t);
template void launch_ghost_u<float>(float*, const float*, LevelView, LevelView, int, int, cudaStream_t);

}  // namespace mrp
