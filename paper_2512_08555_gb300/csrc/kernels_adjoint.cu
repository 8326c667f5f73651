// Transposed operators for the gradient of the converged solve (FP64).
//
// The converged map f -> u_leaf is linear, and so is one correction V-cycle
// (Alg. 1 started from u = 0).  Their transposes are built from the
// transposes of the elementary steps, applied in reverse order:
//   stencil application       -> gather of the (symmetric) weights over the rows
//   Gauss-Seidel sweep         -> colours 7..0, each colour's update transposed
//   ghost fill (Sec. 2.1)      -> each ghost adjoint is added back to its sources
//                                 (same-level interior node, or the I-point
//                                 Lagrange coarse stencil), then cleared
//   injection into covered coarse nodes -> coarse adjoint moved to the
//                                 coincident fine node, then cleared
//   full weighting             -> its transpose (a trilinear-type spread)
//   trilinear correction       -> its transpose (a full-weighting-type gather)
//   level-0 convolution        -> the convolution with source and target exchanged
// Scatters across blocks (ghost and correction transposes) use FP64 atomics.
#include "mrp_internal.h"

namespace mrp {

// LHS weights of the order-M stencil as integers over den (Sec. 3.2).
template <int M> struct LWa;
template <> struct LWa<2> { static constexpr double den = 1, c = -6, f = 1, e = 0, k = 0; };
template <> struct LWa<4> { static constexpr double den = 6, c = -24, f = 2, e = 1, k = 0; };
template <> struct LWa<6> { static constexpr double den = 30, c = -128, f = 14, e = 3, k = 1; };

// Weight of the neighbour with m non-zero offsets (m = 0 centre, 1 face, 2 edge, 3 corner).
template <int M>
__device__ __forceinline__ double lhs_w(int m) {
    using W = LWa<M>;
    return m == 0 ? W::c : (m == 1 ? W::f : (m == 2 ? W::e : W::k));
}

template <int M>
__device__ __forceinline__ double rhs_weight(int dx, int dy, int dz) {
    const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
    if (M == 2) return (ax | ay | az) == 0 ? 1.0 : 0.0;
    if (ax > 1 || ay > 1 || az > 1) {
        if (M == 4) return 0.0;
        const int nz = (ax != 0) + (ay != 0) + (az != 0);     // axis +-2 terms of R^6
        return (nz == 1 && (ax == 2 || ay == 2 || az == 2)) ? -1.0 / 240.0 : 0.0;
    }
    const int o = (ax != 0) + (ay != 0) + (az != 0);
    if (M == 4) return o == 0 ? 0.5 : (o == 1 ? 1.0 / 12.0 : 0.0);
    return o == 0 ? 67.0 / 120.0 : (o == 1 ? 1.0 / 18.0 : (o == 2 ? 1.0 / 90.0 : 0.0));
}

// ---------------------------------------------------------------- stencils
// out[b] (halo layout, g = 1) += scale * L^T lam[b] on the listed blocks: every
// node q of the (n+2)^3 box gathers the weights of the interior rows p with
// |p - q| <= 1.  With fadd, also fadd[b] += lam[b] (the f-part of r = f - L u).
// The weights are symmetric, so this is the stencil applied to lam extended by
// zeros: lam goes to shared memory with a two-node zero border, and one thread
// per box column (x, y) walks z with plane sums (for the plane at z,
// P = f u + e c + k d is what it gives a neighbouring plane and
// Q = c_w u + f c + e d what it gives its own, c and d the sums of the 4 face
// and the 4 diagonal neighbours in (x, y)), so L lam(z) = P(z - 1) + P(z + 1)
// + Q(z); a warp's threads take consecutive x, so its global accesses are
// contiguous.
template <int M, typename T>
__global__ void k_stencil_T(T* __restrict__ out, const T* __restrict__ lam, T* __restrict__ fadd,
                            const int* __restrict__ blocks, int n, T scale) {
    using W = LWa<M>;
    extern __shared__ __align__(16) unsigned char sl_raw[];
    T* lp = reinterpret_cast<T*>(sl_raw);
    const int b = blocks[blockIdx.x];
    const int S = n + 2, S2 = S * S, S3 = S2 * S, n3 = n * n * n, A = n + 4, A2 = A * A, A3 = A2 * A;
    const T* lb = lam + (size_t)b * n3;
    for (int t = threadIdx.x; t < A3; t += blockDim.x) lp[t] = T(0);
    __syncthreads();
    const unsigned mn = magic_of(n), mn2 = magic_of(n * n), mS = magic_of(S);
    __shared__ unsigned s_emax;
    if (threadIdx.x == 0) s_emax = 0u;
    unsigned em = 0;                  // largest exponent field of the staged values (FP64)
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int z = fdiv(t, mn2), r = t - z * n * n, y = fdiv(r, mn), x = r - y * n;
        const T v = lb[t];
        lp[(z + 2) * A2 + (y + 2) * A + x + 2] = v;
        if constexpr (sizeof(T) == 8) em = max(em, ((unsigned)__double2hiint(v) >> 20) & 0x7FFu);
    }
    __syncthreads();
    T* ob = out + (size_t)b * S3;
    if constexpr (sizeof(T) == 8) {
        // The same plane sums in 64-bit fixed point (as the FP64 leaf
        // residual's): every staged value becomes trunc(lambda 2^s) with s set
        // by the largest exponent field E, so that the integer weights (their
        // magnitudes summing to at most 2^G) cannot overflow; the exact sum is
        // rounded once to double and scaled by 2^-s, one FP64 operation per
        // node.  Blocks with Inf or NaN, only zeros, or extreme exponents keep
        // the FP64 sums below.
        constexpr int G = M == 6 ? 8 : 6;
        em = __reduce_max_sync(0xffffffffu, em);
        if ((threadIdx.x & 31) == 0) atomicMax(&s_emax, em);
        __syncthreads();
        const int E = (int)s_emax;
        if (E >= 128 && E <= 1900) {
            const int shb = 9 - G - E;
            for (int t = threadIdx.x; t < n3; t += blockDim.x) {
                const int z = fdiv(t, mn2), r = t - z * n * n, y = fdiv(r, mn), x = r - y * n;
                T* a = lp + (z + 2) * A2 + (y + 2) * A + x + 2;
                *a = __longlong_as_double(to_fixed(__double_as_longlong(*a), shb));
            }
            __syncthreads();
            const double scale2 = (double)scale * __longlong_as_double((long long)(E + G - 1084 + 1023) << 52);
            constexpr long long wc = (long long)W::c, wf = (long long)W::f, we = (long long)W::e, wk = (long long)W::k;
            for (int r = threadIdx.x; r < S2; r += blockDim.x) {
                const int Y = fdiv(r, mS), X = r - Y * S;
                const T* c0 = lp + (Y + 1) * A + X + 1;
                auto ld = [&](const T* q) { return __double_as_longlong(*q); };
                auto plane = [&](int a, long long& P, long long& Q) {
                    const T* q0 = c0 + a * A2;
                    const long long u = ld(q0);
                    const long long c = (ld(q0 - 1) + ld(q0 + 1)) + (ld(q0 - A) + ld(q0 + A));
                    long long p = wf * u, q = wc * u + wf * c;
                    if (we != 0 || wk != 0) {
                        const long long d = (ld(q0 - 1 - A) + ld(q0 + 1 - A)) + (ld(q0 - 1 + A) + ld(q0 + 1 + A));
                        p += we * c + wk * d;
                        q += we * d;
                    }
                    P = p;
                    Q = q;
                };
                long long P0, P1, Q1, Qg;
                plane(0, P0, Qg);
                plane(1, P1, Q1);
                T* ocol = ob + Y * S + X;
                for (int Z = 0; Z < S; ++Z) {
                    long long P2, Q2;
                    plane(Z + 2, P2, Q2);
                    T* o = ocol + (size_t)Z * S2;
                    *o = fma(scale2, i64_to_double_rn((P0 + P2) + Q1), *o);
                    P0 = P1;
                    P1 = P2;
                    Q1 = Q2;
                }
            }
            if (fadd)
                for (int t = threadIdx.x; t < n3; t += blockDim.x) fadd[(size_t)b * n3 + t] += lb[t];
            return;
        }
    }
    for (int r = threadIdx.x; r < S2; r += blockDim.x) {
        const int Y = fdiv(r, mS), X = r - Y * S;
        // padded coordinates of box node (X, Y, Z): (X + 1, Y + 1, Z + 1)
        const T* c0 = lp + (Y + 1) * A + X + 1;
        auto plane = [&](int a, T& P, T& Q) {
            const T* q0 = c0 + a * A2;
            const T u = q0[0];
            const T c = (q0[-1] + q0[1]) + (q0[-A] + q0[A]);
            const T d = (q0[-1 - A] + q0[1 - A]) + (q0[-1 + A] + q0[1 + A]);
            T p = T(W::f) * u, q = T(W::c) * u + T(W::f) * c;
            if (W::e != 0) { p += T(W::e) * c; q += T(W::e) * d; }
            if (W::k != 0) p += T(W::k) * d;
            P = p;
            Q = q;
        };
        T P0, P1, Q1, Qg;
        plane(0, P0, Qg);
        plane(1, P1, Q1);
        T* ocol = ob + Y * S + X;
        for (int Z = 0; Z < S; ++Z) {
            T P2, Q2;
            plane(Z + 2, P2, Q2);
            ocol[(size_t)Z * S2] += scale * ((P0 + P2) + Q1);
            P0 = P1;
            P1 = P2;
            Q1 = Q2;
        }
    }
    if (fadd)
        for (int t = threadIdx.x; t < n3; t += blockDim.x) fadd[(size_t)b * n3 + t] += lb[t];
}

template <typename T>
void launch_stencil_T(T* out, const T* lam, T* fadd, const int* blocks, int nblocks, int n, int M, double inv_h2,
                      cudaStream_t s) {
    if (nblocks == 0) return;
    static std::once_flag attr[MAX_DEVICES];
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_stencil_T<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_stencil_T<4, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_stencil_T<6, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    });
    const size_t sm = sizeof(T) * (size_t)(n + 4) * (n + 4) * (n + 4);
    if (M == 2) k_stencil_T<2, T><<<nblocks, 256, sm, s>>>(out, lam, fadd, blocks, n, T(inv_h2 / LWa<2>::den));
    if (M == 4) k_stencil_T<4, T><<<nblocks, 256, sm, s>>>(out, lam, fadd, blocks, n, T(inv_h2 / LWa<4>::den));
    if (M == 6) k_stencil_T<6, T><<<nblocks, 256, sm, s>>>(out, lam, fadd, blocks, n, T(inv_h2 / LWa<6>::den));
}
template void launch_stencil_T<double>(double*, const double*, double*, const int*, int, int, int, double, cudaStream_t);
template void launch_stencil_T<float>(float*, const float*, float*, const int*, int, int, int, double, cudaStream_t);

// out[b] (raw-f layout, g = 2) = R^T fsb[b] on the listed blocks.
template <int M>
__global__ void k_rstencil_T(double* __restrict__ out, const double* __restrict__ fsb, const int* __restrict__ blocks, int n) {
    const int b = blocks[blockIdx.x];
    const int S = n + 4, S3 = S * S * S, n3 = n * n * n;
    const double* lb = fsb + (size_t)b * n3;
    for (int t = threadIdx.x; t < S3; t += blockDim.x) {
        const int qx = t % S - 2, qy = (t / S) % S - 2, qz = t / (S * S) - 2;
        double acc = 0.0;
        for (int dz = -2; dz <= 2; ++dz) {
            const int pz = qz + dz;
            if (pz < 0 || pz >= n) continue;
            for (int dy = -2; dy <= 2; ++dy) {
                const int py = qy + dy;
                if (py < 0 || py >= n) continue;
                for (int dx = -2; dx <= 2; ++dx) {
                    const int px = qx + dx;
                    if (px < 0 || px >= n) continue;
                    const double w = rhs_weight<M>(dx, dy, dz);
                    if (w != 0.0) acc += w * lb[(pz * n + py) * n + px];
                }
            }
        }
        out[(size_t)b * S3 + t] = acc;
    }
}

void launch_rstencil_T(double* out, const double* fsb, const int* blocks, int nblocks, int n, int M, cudaStream_t s) {
    if (nblocks == 0) return;
    if (M == 2) k_rstencil_T<2><<<nblocks, 256, 0, s>>>(out, fsb, blocks, n);
    if (M == 4) k_rstencil_T<4><<<nblocks, 256, 0, s>>>(out, fsb, blocks, n);
    if (M == 6) k_rstencil_T<6><<<nblocks, 256, 0, s>>>(out, fsb, blocks, n);
}

// ---------------------------------------------------------------- Gauss-Seidel sweep
// Transpose of one 8-colour sweep with frozen halo (forward: nodes p of colour
// c take (den h^2 f_p - sum_q w_q u_q) / w_c).  Colours run 7..0.  With x the
// adjoint restricted to the colour-c interior nodes, colour c's transposed
// update is u-bar -= (1 / w_c) N x on every node of the box (halo included:
// it is scattered afterwards by the ghost transpose), N the off-centre
// stencil; then the colour-c nodes pass den h^2 / w_c of their adjoint to f
// and clear it.  N x vanishes on colour c itself, and a node whose parity
// differs from c in m axes has exactly the colour-c neighbours q +- 1 in those
// axes (2^m of them, all of weight w_m).
//
// Layout: the (n+2)^3 box in shared memory split by the parity of its box
// coordinates (8 sub-arrays of H^3, H = n/2 + 1, at X >> 1 etc.), so that a
// colour is one sub-array; x goes to a copy of that sub-array with a zero
// border (and zeros where the colour's positions are halo), so the gathers
// need no bounds tests.  Along an axis where a destination of box parity p
// differs from the colour, its two sources sit at split offsets p - 1 and p.
// One destination sub-array's gathers: every position subtracts coef times the
// sum of its CNT colour-c values in the bordered copy xs, at uniform offsets
// from its own place (z, y, x order, ascending).
template <int CNT, typename T>
__device__ __forceinline__ void gather_T(T* __restrict__ sd, const T* __restrict__ xs, const int* __restrict__ ptab,
                                         int o0, int hi, int lo, int E, int E2, T coef, int H3) {
    for (int pos = threadIdx.x; pos < H3; pos += blockDim.x) {
        const T* g = xs + (ptab[pos] & 0xFFF) + o0;
        T acc;
        if (CNT == 2) acc = g[0] + g[lo];
        else if (CNT == 4) acc = ((g[0] + g[lo]) + g[hi]) + g[hi + lo];
        else acc = ((((((g[0] + g[1]) + g[E]) + g[E + 1]) + g[E2]) + g[E2 + 1]) + g[E2 + E]) + g[E2 + E + 1];
        sd[pos] -= coef * acc;
    }
}

template <int M, typename T>
__global__ void __launch_bounds__(256) k_smooth_T(T* __restrict__ U, T* __restrict__ F, int n, T h2den) {
    extern __shared__ __align__(16) unsigned char st_raw[];
    const int S = n + 2, S2 = S * S, S3 = S2 * S, n3 = n * n * n;
    const int H = n / 2 + 1, H2 = H * H, H3 = H2 * H;
    const int E = H + 2, E2 = E * E;
    T* su = reinterpret_cast<T*>(st_raw);
    T* xs = su + 8 * H3;                  // E^3, zero border
    // per position of a sub-array: its place in xs (12 bits) and i, j, l (4 bits each)
    int* ptab = reinterpret_cast<int*>(xs + E2 * E);
    const int b = blockIdx.x;
    T* Ub = U + (size_t)b * S3;
    T* Fb = F + (size_t)b * n3;
    const unsigned mH = magic_of(H), mH2 = magic_of(H2), mH3 = magic_of(H3);
    for (int t = threadIdx.x; t < E2 * E; t += blockDim.x) xs[t] = T(0);
    for (int t = threadIdx.x; t < H3; t += blockDim.x) {
        const int l = fdiv(t, mH2), r = t - l * H2, j = fdiv(r, mH), i = r - j * H;
        ptab[t] = ((l + 1) * E2 + (j + 1) * E + i + 1) | (i << 12) | (j << 16) | (l << 20);
    }
    __syncthreads();
    // global box index of split position pos of sub-array d (box parity d)
    auto boxidx = [&](int d, int pos) {
        const int pt = ptab[pos];
        const int X = 2 * ((pt >> 12) & 15) + (d & 1), Y = 2 * ((pt >> 16) & 15) + ((d >> 1) & 1),
                  Z = 2 * ((pt >> 20) & 15) + (d >> 2);
        return (Z * S + Y) * S + X;
    };
    for (int t = threadIdx.x; t < 8 * H3; t += blockDim.x) {
        const int d = fdiv(t, mH3);
        su[t] = Ub[boxidx(d, t - d * H3)];
    }
    __syncthreads();
    const T inv_c = T(1.0 / LWa<M>::c), fscale = h2den * inv_c;
    for (int col = 7; col >= 0; --col) {
        // colour col in interior coordinates; its box parity is the opposite
        const int cs = col ^ 7;
        const int px = cs & 1, py = (cs >> 1) & 1, pz = (cs >> 2) & 1;
        // split index of the colour's halo positions along each axis
        const int hx = px ? H - 1 : 0, hy = py ? H - 1 : 0, hz = pz ? H - 1 : 0;
        T* sc = su + cs * H3;
        for (int t = threadIdx.x; t < H3; t += blockDim.x) {
            const int pt = ptab[t];
            const int i = (pt >> 12) & 15, j = (pt >> 16) & 15, l = (pt >> 20) & 15;
            const bool in = i != hx && j != hy && l != hz;
            const T v = in ? sc[t] : T(0);
            xs[pt & 0xFFF] = v;
            if (in) {
                sc[t] = T(0);
                Fb[((2 * l + pz - 1) * n + 2 * j + py - 1) * n + 2 * i + px - 1] += fscale * v;
            }
        }
        __syncthreads();
        for (int q = 0; q < 7; ++q) {
            const int d = q < cs ? q : q + 1;           // destination sub-array (box parity)
            const int D = d ^ cs;                       // axes in which it differs from the colour
            const int m = (D & 1) + ((D >> 1) & 1) + ((D >> 2) & 1);
            const T w = T(lhs_w<M>(m));
            if (w == T(0)) continue;
            // along an axis where it differs, the sources sit at split offsets p - 1 and p
            // (p its parity bit); o0 is the first (all axes at p - 1), hi and lo the
            // strides of the differing axes (the larger first; one axis: lo only)
            const int o0 = ((D & 4) ? (((d >> 2) & 1) - 1) * E2 : 0) + ((D & 2) ? (((d >> 1) & 1) - 1) * E : 0) +
                           ((D & 1) ? (d & 1) - 1 : 0);
            const int hi = (D & 4) ? E2 : E;
            const int lo = (D & 1) ? 1 : ((D & 2) ? E : E2);
            T* sd = su + d * H3;
            const T coef = w * inv_c;
            if (m == 1) gather_T<2>(sd, xs, ptab, o0, hi, lo, E, E2, coef, H3);
            else if (m == 2) gather_T<4>(sd, xs, ptab, o0, hi, lo, E, E2, coef, H3);
            else gather_T<8>(sd, xs, ptab, o0, hi, lo, E, E2, coef, H3);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < 8 * H3; t += blockDim.x) {
        const int d = fdiv(t, mH3);
        Ub[boxidx(d, t - d * H3)] = su[t];
    }
}

template <typename T>
void launch_smooth_T(T* U, T* F, int nb, int n, int M, double h2, cudaStream_t s) {
    if (nb == 0) return;
    static std::once_flag attr[MAX_DEVICES];
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_smooth_T<2, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_smooth_T<4, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
        cudaFuncSetAttribute(k_smooth_T<6, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM);
    });
    const size_t H = n / 2 + 1, E = H + 2;
    const size_t sm = sizeof(T) * (8 * H * H * H + E * E * E) + sizeof(int) * H * H * H;
    if (M == 2) k_smooth_T<2, T><<<nb, 256, sm, s>>>(U, F, n, T(h2 * LWa<2>::den));
    if (M == 4) k_smooth_T<4, T><<<nb, 256, sm, s>>>(U, F, n, T(h2 * LWa<4>::den));
    if (M == 6) k_smooth_T<6, T><<<nb, 256, sm, s>>>(U, F, n, T(h2 * LWa<6>::den));
}
template void launch_smooth_T<double>(double*, double*, int, int, int, double, cudaStream_t);
template void launch_smooth_T<float>(float*, float*, int, int, int, double, cudaStream_t);

// ---------------------------------------------------------------- ghosts and injection
// Transpose of the ghost fill of level k (halo g): every ghost adjoint goes
// back to its sources, then the ghost layer is cleared.  Outside the domain
// it is dropped (f is zero there; u's exterior ring is not an input).
template <int I>
__global__ void k_ghost_T(double* __restrict__ A, int g, double* __restrict__ Ac, int gc, LevelView lk, LevelView lc, int n) {
    __shared__ int snbr[27], cnbr[27];
    __shared__ double sw[8];
    const int b = blockIdx.x;
    const int par = lk.parent ? lk.parent[b] : -1;
    if (threadIdx.x < 27) {
        snbr[threadIdx.x] = lk.nbr[27 * b + threadIdx.x];
        cnbr[threadIdx.x] = par >= 0 ? lc.nbr[27 * par + threadIdx.x] : -1;
    }
    if (threadIdx.x < I) {
        const int m = threadIdx.x;
        double w;
        if (I == 4) w = (m == 0 || m == 3 ? -1.0 : 9.0) / 16.0;
        else if (I == 6) w = (m == 0 || m == 5 ? 3.0 : (m == 1 || m == 4 ? -25.0 : 150.0)) / 256.0;
        else { const int q = m < 4 ? m : 7 - m; w = (q == 0 ? -5.0 : (q == 1 ? 49.0 : (q == 2 ? -245.0 : 1225.0))) / 2048.0; }
        sw[m] = w;
    }
    __syncthreads();
    const int S = n + 2 * g, S2 = S * S, S3 = S2 * S;
    const int Sc = n + 2 * gc, Sc3 = Sc * Sc * Sc;
    double* Ab = A + (size_t)b * S3;
    const int bx = lk.coords[3 * b], by = lk.coords[3 * b + 1], bz = lk.coords[3 * b + 2];
    for (int t = threadIdx.x; t < S3; t += blockDim.x) {
        const int x = t % S, y = (t / S) % S, z = t / S2;
        const int dx = x < g ? -1 : (x >= g + n ? 1 : 0);
        const int dy = y < g ? -1 : (y >= g + n ? 1 : 0);
        const int dz = z < g ? -1 : (z >= g + n ? 1 : 0);
        if ((dx | dy | dz) == 0) continue;
        const double a = Ab[t];
        Ab[t] = 0.0;
        if (a == 0.0) continue;
        const int j = snbr[dir27(dx, dy, dz)];
        if (j >= 0) {
            atomicAdd(&A[(size_t)j * S3 + (size_t)((z - dz * n) * S + (y - dy * n)) * S + (x - dx * n)], a);
            continue;
        }
        if (j != NBR_MISSING || par < 0) continue;
        // level-k node p; even coordinates coincide with a coarse node, odd ones
        // take the I-point midpoint interpolant; coarse nodes are addressed in
        // the parent's 27-neighbourhood
        const int p[3] = {bx * n + x - g, by * n + y - g, bz * n + z - g};
        const int porig[3] = {(bx >> 1) * n, (by >> 1) * n, (bz >> 1) * n};
        int cnt[3], c0[3];
        for (int q = 0; q < 3; ++q) {
            if ((p[q] & 1) == 0) { cnt[q] = 1; c0[q] = (p[q] >> 1) - porig[q]; }
            else { cnt[q] = I; c0[q] = ((p[q] - 1) >> 1) - I / 2 + 1 - porig[q]; }
        }
        for (int mz = 0; mz < cnt[2]; ++mz) {
            const int rz = c0[2] + mz, ez = rz < 0 ? -1 : (rz >= n ? 1 : 0), lz = rz - ez * n;
            const double wz = cnt[2] == 1 ? 1.0 : sw[mz];
            for (int my = 0; my < cnt[1]; ++my) {
                const int ry = c0[1] + my, ey = ry < 0 ? -1 : (ry >= n ? 1 : 0), ly = ry - ey * n;
                const double wy = cnt[1] == 1 ? 1.0 : sw[my];
                for (int mx = 0; mx < cnt[0]; ++mx) {
                    const int rx = c0[0] + mx, ex = rx < 0 ? -1 : (rx >= n ? 1 : 0), lx = rx - ex * n;
                    const double wx = cnt[0] == 1 ? 1.0 : sw[mx];
                    const int cb = cnbr[dir27(ex, ey, ez)];
                    if (cb < 0) continue;   // unreachable in a 2:1 balanced forest
                    atomicAdd(&Ac[(size_t)cb * Sc3 + (size_t)((gc + lz) * Sc + gc + ly) * Sc + gc + lx], wx * wy * wz * a);
                }
            }
        }
    }
}

void launch_ghost_T(double* A, int g, double* Ac, int gc, LevelView lk, LevelView lc, int n, int M, cudaStream_t s) {
    if (lk.nb == 0) return;
    if (M == 2) k_ghost_T<4><<<lk.nb, 256, 0, s>>>(A, g, Ac, gc, lk, lc, n);
    if (M == 4) k_ghost_T<6><<<lk.nb, 256, 0, s>>>(A, g, Ac, gc, lk, lc, n);
    if (M == 6) k_ghost_T<8><<<lk.nb, 256, 0, s>>>(A, g, Ac, gc, lk, lc, n);
}

// Transpose of the injection of level k into its parents' covered nodes
// (one CTA per level-k block; the covered interiors are disjoint).
template <typename T>
__global__ void k_inject_T(T* __restrict__ fine, int gf, T* __restrict__ coarse, int gc, LevelView lf, int n) {
    const int B = blockIdx.x;
    const int P = lf.parent[B], o = lf.octant[B];
    const int h = n >> 1;
    const int Sf = n + 2 * gf, Sc = n + 2 * gc;
    T* fb = fine + (size_t)B * Sf * Sf * Sf;
    T* cb = coarse + (size_t)P * Sc * Sc * Sc;
    const int ox = (o & 1) * h, oy = ((o >> 1) & 1) * h, oz = ((o >> 2) & 1) * h;
    for (int t = threadIdx.x; t < h * h * h; t += blockDim.x) {
        const int i = t % h, j = (t / h) % h, l = t / (h * h);
        const size_t c = ((size_t)(gc + oz + l) * Sc + gc + oy + j) * Sc + gc + ox + i;
        fb[((gf + 2 * l) * Sf + gf + 2 * j) * Sf + gf + 2 * i] += cb[c];
        cb[c] = T(0);
    }
}

template <typename T>
void launch_inject_T(T* fine, int gf, T* coarse, int gc, LevelView lf, int n, cudaStream_t s) {
    if (lf.nb == 0) return;
    k_inject_T<T><<<lf.nb, 256, 0, s>>>(fine, gf, coarse, gc, lf, n);
}
template void launch_inject_T<double>(double*, int, double*, int, LevelView, int, cudaStream_t);
template void launch_inject_T<float>(float*, int, float*, int, LevelView, int, cudaStream_t);

// ---------------------------------------------------------------- grid transfers
// Transpose of u_k += trilinear(u_{k-1} - uhat_{k-1}): the (n/2+1)^3 coarse
// window of block B (its parent's part plus the next coarse node on each
// upper side) gathers the fine adjoints with weights 1 (coincident) and 1/2
// (midpoint neighbours); it is added to u_{k-1} and subtracted from uhat_{k-1}.
template <typename T>
__global__ void k_prolong_T(T* __restrict__ Uc, T* __restrict__ Hc, const T* __restrict__ Uf, LevelView lf, LevelView lc,
                            int n) {
    const int B = blockIdx.x;
    const int P = lf.parent[B], o = lf.octant[B];
    const int h = n >> 1, E = h + 1;
    const int S = n + 2, S3 = S * S * S, n3 = n * n * n;
    const int ox = (o & 1) * h, oy = ((o >> 1) & 1) * h, oz = ((o >> 2) & 1) * h;
    const int* cn = lc.nbr + 27 * P;
    const T* Ub = Uf + (size_t)B * S3;
    for (int t = threadIdx.x; t < E * E * E; t += blockDim.x) {
        const int i = t % E, j = (t / E) % E, l = t / (E * E);
        T acc = T(0);
        for (int dz = -1; dz <= 1; ++dz) {
            const int z = 2 * l + dz;
            if (z < 0 || z >= n) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int y = 2 * j + dy;
                if (y < 0 || y >= n) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x = 2 * i + dx;
                    if (x < 0 || x >= n) continue;
                    // 1 or 1/2 per axis: exact, without FP64 arithmetic
                    const T w = T(1.0 / 8.0) * T(1 << ((dx == 0) + (dy == 0) + (dz == 0)));
                    acc += w * Ub[((z + 1) * S + y + 1) * S + x + 1];
                }
            }
        }
        if (acc == T(0)) continue;
        const int cx = ox + i, cy = oy + j, cz = oz + l;
        const int ex = cx >= n, ey = cy >= n, ez = cz >= n;
        const int blk = cn[dir27(ex, ey, ez)];
        const int lx = cx - ex * n, ly = cy - ey * n, lz = cz - ez * n;
        atomicAdd(&Uc[(size_t)blk * S3 + ((lz + 1) * S + ly + 1) * S + lx + 1], acc);
        atomicAdd(&Hc[(size_t)blk * n3 + (lz * n + ly) * n + lx], -acc);
    }
}

template <typename T>
void launch_prolong_T(T* Uc, T* Hc, const T* Uf, LevelView lf, LevelView lc, int n, cudaStream_t s) {
    if (lf.nb == 0) return;
    k_prolong_T<T><<<lf.nb, 256, 0, s>>>(Uc, Hc, Uf, lf, lc, n);
}
template void launch_prolong_T<double>(double*, double*, const double*, LevelView, LevelView, int, cudaStream_t);
template void launch_prolong_T<float>(float*, float*, const float*, LevelView, LevelView, int, cudaStream_t);

// Transpose of the restriction of r (full weighting (1/4)[1 2 1]^3, or
// injection where the 27-point window of the coarse node leaves Omega_k):
// each node p of level-k block B gathers from the covered coarse nodes X
// with |2X - p| <= 1.  The fine image 2X lies in B or in B's upper
// neighbours; X's window is complete when the level-k blocks below 2X exist
// along the axes where 2X sits on the block's lower face.  Writes Rf[B].
// The neighbour tables those tests need are read once per block into shared
// memory: for each upper neighbour e in {0, 1}^3 (the block holding 2X), its
// index, parent and octant, and for each pattern m of axes on which 2X lies on
// its lower face, whether the window is complete.
template <typename T>
__global__ void k_fw_T(T* __restrict__ Rf, const T* __restrict__ Fc, LevelView lf, int n) {
    __shared__ int cblk[8], cpar[8], coct[8];
    __shared__ unsigned char ins[8][8];
    const int B = blockIdx.x;
    if (threadIdx.x < 8) {
        const int e = threadIdx.x;
        const int c = lf.nbr[27 * B + dir27(e & 1, (e >> 1) & 1, (e >> 2) & 1)];
        cblk[e] = c;
        cpar[e] = c >= 0 ? lf.parent[c] : 0;
        coct[e] = c >= 0 ? lf.octant[c] : 0;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int e = threadIdx.x >> 3, m = threadIdx.x & 7, c = cblk[e];
        bool inside = c >= 0;
        for (int sz = 0; sz <= ((m >> 2) & 1) && inside; ++sz)
            for (int sy = 0; sy <= ((m >> 1) & 1); ++sy)
                for (int sx = 0; sx <= (m & 1); ++sx)
                    if (lf.nbr[27 * c + dir27(-sx, -sy, -sz)] < 0) inside = false;
        ins[e][m] = inside;
    }
    __syncthreads();
    const int h = n >> 1, n3 = n * n * n;
    const unsigned mn = magic_of(n), mn2 = magic_of(n * n);
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int pz = fdiv(t, mn2), r = t - pz * n * n, py = fdiv(r, mn), px = r - py * n;
        // odd coordinates reach the coarse nodes at p - 1 and p + 1, even ones the node at p
        const int lx = px & 1 ? -1 : 0, ly = py & 1 ? -1 : 0, lz = pz & 1 ? -1 : 0;
        T acc = T(0);
        for (int dz = lz; dz <= -lz; dz += 2)
            for (int dy = ly; dy <= -ly; dy += 2)
                for (int dx = lx; dx <= -lx; dx += 2) {
                    const int vx = px + dx, vy = py + dy, vz = pz + dz;      // 0..n, even
                    const int ex = vx >= n, ey = vy >= n, ez = vz >= n;
                    const int e = ex | (ey << 1) | (ez << 2);
                    if (cblk[e] < 0) continue;                  // 2X not in Omega_k: X is not covered
                    const int qx = vx - ex * n, qy = vy - ey * n, qz = vz - ez * n;
                    const int m = (qx == 0) | ((qy == 0) << 1) | ((qz == 0) << 2);
                    const int o = coct[e];
                    const int X = (o & 1) * h + (qx >> 1), Y = ((o >> 1) & 1) * h + (qy >> 1),
                              Z = ((o >> 2) & 1) * h + (qz >> 1);
                    const T v = Fc[(size_t)cpar[e] * n3 + (Z * n + Y) * n + X];
                    if (ins[e][m]) {
                        // (1 or 2 per axis) / 64: exact, without FP64 arithmetic
                        const T w = T(((dx == 0) + 1) * ((dy == 0) + 1) * ((dz == 0) + 1)) * T(1.0 / 64.0);
                        acc += w * v;
                    } else if ((dx | dy | dz) == 0) {
                        acc += v;
                    }
                }
        Rf[(size_t)B * n3 + t] = acc;
    }
}

template <typename T>
void launch_fw_T(T* Rf, const T* Fc, LevelView lf, int n, cudaStream_t s) {
    if (lf.nb == 0) return;
    k_fw_T<T><<<lf.nb, 256, 0, s>>>(Rf, Fc, lf, n);
}
template void launch_fw_T<double>(double*, const double*, LevelView, int, cudaStream_t);
template void launch_fw_T<float>(float*, const float*, LevelView, int, cudaStream_t);

// ---------------------------------------------------------------- level 0
// Transpose of the write of the level-0 target cube [-1, N0]^3 into every
// level-0 block's (n+2)^3 box: each cube node sums the boxes that hold it.
template <typename T>
__global__ void k_window_T(T* __restrict__ cube, const T* __restrict__ U0, int n, int nbx, int nby, int nbz) {
    const int Cx = nbx * n + 2, Cy = nby * n + 2, Cz = nbz * n + 2;
    const size_t total = (size_t)Cx * Cy * Cz;
    const int S = n + 2, S3 = S * S * S;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int tx = (int)(t % Cx) - 1, ty = (int)((t / Cx) % Cy) - 1, tz = (int)(t / ((size_t)Cx * Cy)) - 1;
        T acc = T(0);
        for (int bz = (tz - 1 < 0 ? -1 : (tz - 1) / n); bz <= (tz + 1) / n; ++bz) {
            if (bz < 0 || bz >= nbz || tz < bz * n - 1 || tz > bz * n + n) continue;
            for (int by = (ty - 1 < 0 ? -1 : (ty - 1) / n); by <= (ty + 1) / n; ++by) {
                if (by < 0 || by >= nby || ty < by * n - 1 || ty > by * n + n) continue;
                for (int bx = (tx - 1 < 0 ? -1 : (tx - 1) / n); bx <= (tx + 1) / n; ++bx) {
                    if (bx < 0 || bx >= nbx || tx < bx * n - 1 || tx > bx * n + n) continue;
                    const int blk = (bz * nby + by) * nbx + bx;
                    acc += U0[(size_t)blk * S3 + ((tz - bz * n + 1) * S + ty - by * n + 1) * S + tx - bx * n + 1];
                }
            }
        }
        cube[t] = acc;
    }
}

template <typename T>
void launch_window_T(T* cube, const T* U0, int n, const int* nb0, cudaStream_t s) {
    k_window_T<T><<<4 * 152, 256, 0, s>>>(cube, U0, n, nb0[0], nb0[1], nb0[2]);
}
template void launch_window_T<double>(double*, const double*, int, const int*, cudaStream_t);
template void launch_window_T<float>(float*, const float*, int, const int*, cudaStream_t);

// Dense level-0 source array [0, N0)^3 -> per-block n^3 arrays of the listed blocks (add or set).
template <typename T>
__global__ void k_dense_to_blocks(T* __restrict__ out, const T* __restrict__ dense, const int* __restrict__ blocks,
                                  const int* __restrict__ coords, int n, int N0x, int N0y, bool add) {
    const int b = blocks[blockIdx.x];
    const int cx = coords[3 * b] * n, cy = coords[3 * b + 1] * n, cz = coords[3 * b + 2] * n;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        const T v = dense[((size_t)(cz + z) * N0y + cy + y) * N0x + cx + x];
        if (add) out[(size_t)b * n * n * n + t] += v;
        else out[(size_t)b * n * n * n + t] = v;
    }
}

template <typename T>
void launch_dense_to_blocks(T* out, const T* dense, const int* blocks, int nblocks, const int* coords, int n, const int* n0,
                            bool add, cudaStream_t s) {
    if (nblocks == 0) return;
    k_dense_to_blocks<T><<<nblocks, 256, 0, s>>>(out, dense, blocks, coords, n, n0[0], n0[1], add);
}
template void launch_dense_to_blocks<double>(double*, const double*, const int*, int, const int*, int, const int*, bool,
                                             cudaStream_t);
template void launch_dense_to_blocks<float>(float*, const float*, const int*, int, const int*, int, const int*, bool,
                                            cudaStream_t);

// ---------------------------------------------------------------- block and vector helpers
// scale * v in the output's type: a scale of 1 is a plain conversion, and
// float to float stays in FP32 (GB300's FP64 pipe is the scarce one).
template <typename TO, typename TI>
__device__ __forceinline__ TO scaled(TI v, double scale, bool unit) {
    if (unit) return TO(v);
    if constexpr (sizeof(TO) == 4 && sizeof(TI) == 4) return TO(float(scale) * v);
    else return TO(scale * (double)v);
}

// out[b] = scale * interior of A[b] (halo g) for the listed blocks.
template <typename TO, typename TI>
__global__ void k_interior_get(TO* __restrict__ out, const TI* __restrict__ A, int g, const int* __restrict__ blocks, int n,
                               double scale) {
    const int b = blocks[blockIdx.x];
    const int S = n + 2 * g;
    const bool unit = scale == 1.0;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        out[(size_t)b * n * n * n + t] = scaled<TO>(A[(size_t)b * S * S * S + ((z + g) * S + y + g) * S + x + g], scale, unit);
    }
}

template <typename TO, typename TI>
void launch_interior_get(TO* out, const TI* A, int g, const int* blocks, int nblocks, int n, double scale, cudaStream_t s) {
    if (nblocks == 0) return;
    k_interior_get<TO, TI><<<nblocks, 256, 0, s>>>(out, A, g, blocks, n, scale);
}
template void launch_interior_get<double, double>(double*, const double*, int, const int*, int, int, double, cudaStream_t);
template void launch_interior_get<float, float>(float*, const float*, int, const int*, int, int, double, cudaStream_t);

// interior of A[b] (halo g) += scale * v[b] for the listed blocks.
template <typename TA, typename TV>
__global__ void k_interior_add(TA* __restrict__ A, int g, const TV* __restrict__ v, const int* __restrict__ blocks, int n,
                               double scale) {
    const int b = blocks[blockIdx.x];
    const int S = n + 2 * g;
    const bool unit = scale == 1.0;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        A[(size_t)b * S * S * S + ((z + g) * S + y + g) * S + x + g] += scaled<TA>(v[(size_t)b * n * n * n + t], scale, unit);
    }
}

template <typename TA, typename TV>
void launch_interior_add(TA* A, int g, const TV* v, const int* blocks, int nblocks, int n, double scale, cudaStream_t s) {
    if (nblocks == 0) return;
    k_interior_add<TA, TV><<<nblocks, 256, 0, s>>>(A, g, v, blocks, n, scale);
}
template void launch_interior_add<double, double>(double*, int, const double*, const int*, int, int, double, cudaStream_t);
template void launch_interior_add<float, float>(float*, int, const float*, const int*, int, int, double, cudaStream_t);
template void launch_interior_add<float, double>(float*, int, const double*, const int*, int, int, double, cudaStream_t);

// out[b] = scale * in[b] (n^3 arrays) for the listed blocks; in may be null (zero).
template <typename TO, typename TI>
__global__ void k_block_copy(TO* __restrict__ out, const TI* __restrict__ in, const int* __restrict__ blocks, int n,
                             double scale) {
    const int b = blocks[blockIdx.x];
    const bool unit = scale == 1.0;
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x)
        out[(size_t)b * n * n * n + t] = in ? scaled<TO>(in[(size_t)b * n * n * n + t], scale, unit) : TO(0);
}

template <typename TO, typename TI>
void launch_block_copy(TO* out, const TI* in, const int* blocks, int nblocks, int n, double scale, cudaStream_t s) {
    if (nblocks == 0) return;
    k_block_copy<TO, TI><<<nblocks, 256, 0, s>>>(out, in, blocks, n, scale);
}
template void launch_block_copy<double, double>(double*, const double*, const int*, int, int, double, cudaStream_t);
template void launch_block_copy<float, double>(float*, const double*, const int*, int, int, double, cudaStream_t);
template void launch_block_copy<double, float>(double*, const float*, const int*, int, int, double, cudaStream_t);

template <typename T>
void launch_block_zero(T* out, const int* blocks, int nblocks, int n, cudaStream_t s) {
    if (nblocks == 0) return;
    k_block_copy<T, T><<<nblocks, 256, 0, s>>>(out, nullptr, blocks, n, 0.0);
}
template void launch_block_zero<double>(double*, const int*, int, int, cudaStream_t);
template void launch_block_zero<float>(float*, const int*, int, int, cudaStream_t);

// out = a x + b y over a flat vector (out may alias x or y); optionally
// max |out| into *absmax (bit pattern of a non-negative double, NaN mapped to +Inf).
__global__ void k_lincomb(double* out, double a, const double* x, double b, const double* y, size_t len,
                          unsigned long long* absmax) {
    __shared__ double red[32];
    // max |v| on bit patterns (integer pipe; NaN patterns sort above +Inf and
    // are mapped to +Inf below), and a plain add for a = b = 1: the FP64 pipe
    // would otherwise bound this memory-bound loop
    unsigned long long mb = 0;
    const bool add = a == 1.0 && b == 1.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
        const double v = add ? x[i] + y[i] : a * x[i] + b * y[i];
        out[i] = v;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
        mb = bits > mb ? bits : mb;
    }
    if (!absmax) return;
    double m = mb > 0x7ff0000000000000ULL ? __longlong_as_double(0x7ff0000000000000ULL) : __longlong_as_double((long long)mb);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[w] = m;
    __syncthreads();
    if (w == 0) {
        m = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0) atomicMax(absmax, (unsigned long long)__double_as_longlong(m));
    }
}

void launch_lincomb(double* out, double a, const double* x, double b, const double* y, size_t len,
                    unsigned long long* absmax, cudaStream_t s) {
    if (len == 0) return;
    k_lincomb<<<4 * 152, 256, 0, s>>>(out, a, x, b, y, len, absmax);
}

}  // namespace mrp
