// Stencil kernels that build their block's ghost layer in shared memory
// (arXiv 2512.08555, Sec. 2.1 ghosting fused into the Sec. 3.1 smoother,
// residual and FAS right-hand side).
//
// Each CTA handles one block of level k.  build_halo() stages the block and a
// one-node ghost layer in shared memory:
//  * interior: the block's own values;
//  * ghost regions whose same-level neighbour exists: that neighbour's values;
//  * ghost regions outside the domain (level 0 only): the block's stored ghost
//    layer, i.e. the exterior ring written by the level-0 solve;
//  * the other ghost regions: the I-point (I = M + 2) tensor-product Lagrange
//    interpolant of level k-1, evaluated separably (reduction along the
//    region's normal axes into a small array, then the tangential stencil).
//    A coarse node covered by level k takes the value of its coincident
//    level-k node (the injection of the current fine values), read from the
//    fine level directly.
// All values are read from the input buffers, which no CTA of the launch
// writes: ghost layers are frozen for the duration of a sweep, which writes
// its result to a second buffer.
//
// This header holds the device code and the launcher templates; the
// fused_*.cu translation units instantiate them by family and precision, so
// that they compile in parallel.
#pragma once

#include "mrp_internal.h"

namespace mrp {

template <int M> struct LW;
template <> struct LW<2> { static constexpr double den = 1, c = -6, f = 1, e = 0, k = 0; };
template <> struct LW<4> { static constexpr double den = 6, c = -24, f = 2, e = 1, k = 0; };
template <> struct LW<6> { static constexpr double den = 30, c = -128, f = 14, e = 3, k = 1; };

// ---------------------------------------------------------------- parity-split box
// The block's (n+2)^3 box (ghost layer included) is kept in shared memory as
// 8 sub-arrays by the parity of the box coordinates (X, Y, Z):
//     at(X, Y, Z) = ((Z&1)*4 + (Y&1)*2 + (X&1)) * H3p + (Z>>1) Hp + (Y>>1) H + (X>>1),
// H = (n+2)/2, plane stride Hp >= H^2, sub-array stride H3p >= H Hp with
// H3p = 16 (mod 32).  In one Gauss-Seidel colour every stencil neighbour of
// the colour's nodes lies in one sub-array per offset.  A warp's lanes take
// the colour's nodes with x fastest, then z (see cset_init), so a load
// touches rows (Y) of h consecutive words at plane distance Hp apart; for
// FP32, Hp is the value in [H^2, H^2 + 32) that minimises the shared-memory
// wavefronts of such loads over a colour; block size 16 uses node pairs with
// their own lane order (pair_of) and Hp = 84, whose four rows of one z parity
// fall in disjoint 8-bank windows (no conflicts).  The two x-parities of a row
// fall 16 banks apart.
struct Split {
    int H, H2, H3p;      // H2: plane stride Hp
    __device__ __forceinline__ int at(int X, int Y, int Z) const {
        return (((Z & 1) << 2) | ((Y & 1) << 1) | (X & 1)) * H3p + (Z >> 1) * H2 + (Y >> 1) * H + (X >> 1);
    }
};
__host__ __device__ inline int split_hp(int n, int el) {
    const int H = n / 2 + 1;
    if (el != 4) return H * H;
    switch (n) {
        case 10: return 59;
        case 12: return 70;
        case 14: return 71;
        case 16: return 84;
        case 18: return 105;
        case 20: return 138;
        case 22: return 171;
        case 24: return 172;
        default: return H * H;
    }
}
__host__ __device__ inline int split_h3p(int n, int el) {
    const int H = n / 2 + 1, H3 = H * split_hp(n, el);
    return H3 + ((16 - H3 % 32) % 32 + 32) % 32;
}
template <typename T>
__device__ __forceinline__ Split split_of(int n) {
    Split sp;
    sp.H = n / 2 + 1;
    sp.H2 = split_hp(n, (int)sizeof(T));
    sp.H3p = split_h3p(n, (int)sizeof(T));
    return sp;
}

// A staged right-hand side uses the same colour split without a ghost layer:
//     fat(x, y, z) = ((z&1)*4 + (y&1)*2 + (x&1)) * F3 + (z>>1) Fp + (y>>1) Fr + (x>>1),
// h = n/2, F3 >= h Fp.  FP32 strides minimise the wavefronts of a colour's
// loads: for n = 16 (node pairs along x, see pair_of) Fr = 9, Fp = 76;
// otherwise Fr = h and Fp is the best value in [h^2, h^2 + 32); FP64 keeps
// Fr = h, Fp = h^2.
__host__ __device__ inline int split_fp(int n, int el) {
    const int h = n / 2;
    if (el != 4) return h * h;
    switch (n) {
        case 8: return 24;
        case 10: return 27;
        case 12: return 38;
        case 14: return 71;
        case 16: return 76;
        case 18: return 105;
        case 20: return 106;
        case 22: return 139;
        case 24: return 172;
        default: return h * h;
    }
}
__host__ __device__ inline int split_fr(int n, int el) { return (el == 4 && n == 16) ? 9 : n / 2; }
// Colour sub-array stride: FP32 pads h Fp to 16 (mod 32) words, so that the
// two x-parities of a column copy fall 16 banks apart; block size 16 pads to
// 8 (mod 32), which puts the x-parities 8 banks and the y-parities 16 banks
// apart (a warp's column copy of two rows is then conflict-free) with less
// shared memory.
__host__ __device__ inline int split_f3(int n, int el) {
    const int f = (n / 2) * split_fp(n, el);
    if (el == 4 && n == 16) return f + ((8 - f % 32) % 32 + 32) % 32;
    return el == 4 ? f + ((16 - f % 32) % 32 + 32) % 32 : f;
}

// The thread's nodes of one colour: node q = tid + k * nt (k < KMAX) of the
// (n/2)^3 nodes (i, j, l) of a colour, q = i + h (l + h j), packed
// i | j << 10 | l << 20; a colour c = (cx, cy, cz) places it at interior
// coordinates (2i+cx, 2j+cy, 2l+cz).
constexpr int KMAX = 8;
struct Cset { int cnt; int q[KMAX]; };
__device__ __forceinline__ void cset_init(Cset& cs, int h) {
    const int h3 = h * h * h;
    cs.cnt = 0;
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
        const int q = threadIdx.x + k * blockDim.x;
        cs.q[k] = 0;
        if (q < h3) {
            const int i = q % h, l = (q / h) % h, j = q / (h * h);
            cs.q[k] = i | (j << 10) | (l << 20);
            cs.cnt = k + 1;
        }
    }
}

// Offsets of colour col: cb = sub-array of the (-1,-1,-1) neighbour; dX, dY,
// dZ = step from a (-1) neighbour to the centre along each axis (the (+1)
// neighbour is 1, H, Hp past the (-1) one); fo / go = natural interior /
// box offsets of the colour.
struct Col { int cb, dX, dY, dZ, fo, go; };
__device__ __forceinline__ Col colour(int col, const Split& sp, int n) {
    const int cx = col & 1, cy = (col >> 1) & 1, cz = (col >> 2) & 1;
    const int S = n + 2;
    Col c;
    c.cb = sp.H3p * (4 * cz + 2 * cy + cx);
    c.dX = sp.H3p * (1 - 2 * cx) + cx;
    c.dY = 2 * sp.H3p * (1 - 2 * cy) + sp.H * cy;
    c.dZ = 4 * sp.H3p * (1 - 2 * cz) + sp.H2 * cz;
    c.fo = (cz * n + cy) * n + cx;
    c.go = (cz * S + cy) * S + cx;
    return c;
}

// Per node of a colour: split index of its (-1,-1,-1) neighbour, natural
// interior index and natural box index (each before the colour's offsets).
struct Node { int b0, f, g, fs; };
__device__ __forceinline__ Node node_of(int packed, const Split& sp, int n, int fp = 0, int fr = 0) {
    const int i = packed & 1023, j = (packed >> 10) & 1023, l = packed >> 20;
    const int S = n + 2;
    Node d;
    d.b0 = l * sp.H2 + j * sp.H + i;
    d.fs = l * fp + j * fr + i;
    d.f = ((2 * l) * n + 2 * j) * n + 2 * i;
    d.g = ((2 * l + 1) * S + 2 * j + 1) * S + 2 * i + 1;
    return d;
}

// Weighted sum of the 26 off-centre neighbours (integer weights of LW<M>) of
// the node whose (-1,-1,-1) neighbour sits at split index b0.
template <int M, typename T>
__device__ __forceinline__ T offc_s(const T* __restrict__ a, int b0, int dX, int dY, int dZ, int H, int H2) {
    using W = LW<M>;
    T acc = T(W::f) * ((a[b0 + dY + dZ] + a[b0 + 1 + dY + dZ]) + (a[b0 + dX + dZ] + a[b0 + dX + H + dZ])
                       + (a[b0 + dX + dY] + a[b0 + dX + dY + H2]));
    if (W::e != 0)
        acc += T(W::e) * ((a[b0 + dZ] + a[b0 + 1 + dZ]) + (a[b0 + H + dZ] + a[b0 + 1 + H + dZ])
                          + (a[b0 + dY] + a[b0 + 1 + dY]) + (a[b0 + dY + H2] + a[b0 + 1 + dY + H2])
                          + (a[b0 + dX] + a[b0 + dX + H]) + (a[b0 + dX + H2] + a[b0 + dX + H + H2]));
    if (W::k != 0)
        acc += T(W::k) * ((a[b0] + a[b0 + 1]) + (a[b0 + H] + a[b0 + 1 + H])
                          + (a[b0 + H2] + a[b0 + 1 + H2]) + (a[b0 + H + H2] + a[b0 + 1 + H + H2]));
    return acc;
}

// Packed FP32 pairs (Blackwell's f32x2 arithmetic: one instruction applies
// the same IEEE operation, round to nearest, to both halves).  A node pair of
// the fixed block size 16 runs the same operations on neighbour values one
// word apart, so its two stencils are evaluated as one packed stencil.
typedef unsigned long long f2_t;
__device__ __forceinline__ f2_t f2pk(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2up(f2_t v, float& a, float& b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f2_t f2add(f2_t a, f2_t b) {
    f2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2sub(f2_t a, f2_t b) {
    f2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2mul(f2_t a, f2_t b) {
    f2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2_t f2fma(f2_t a, f2_t b, f2_t c) {
    f2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2_t f2splat(float a) { return f2pk(a, a); }

// offc_s for the nodes with (-1,-1,-1) neighbours at b0 and b0 + 1 at once
// (packed: low half the first node, high half the second), same sums in the
// same order.
template <int M>
__device__ __forceinline__ f2_t offc2(const float* __restrict__ a, int b0, int dX, int dY, int dZ, int H, int H2) {
    using W = LW<M>;
    auto L = [&](int o) { return f2pk(a[b0 + o], a[b0 + 1 + o]); };
    f2_t acc = f2mul(f2splat(float(W::f)),
                     f2add(f2add(f2add(L(dY + dZ), L(1 + dY + dZ)), f2add(L(dX + dZ), L(dX + H + dZ))),
                           f2add(L(dX + dY), L(dX + dY + H2))));
    if (W::e != 0) {
        const f2_t e = f2add(f2add(f2add(f2add(f2add(f2add(L(dZ), L(1 + dZ)), f2add(L(H + dZ), L(1 + H + dZ))),
                                                   f2add(L(dY), L(1 + dY))),
                                             f2add(L(dY + H2), L(1 + dY + H2))),
                                       f2add(L(dX), L(dX + H))),
                                 f2add(L(dX + H2), L(dX + H + H2)));
        acc = W::e == 1 ? f2add(acc, e) : f2fma(f2splat(float(W::e)), e, acc);
    }
    if (W::k != 0) {
        const f2_t k = f2add(f2add(f2add(L(0), L(1)), f2add(L(H), L(1 + H))),
                             f2add(f2add(L(H2), L(1 + H2)), f2add(L(H + H2), L(1 + H + H2))));
        acc = W::k == 1 ? f2add(acc, k) : f2fma(f2splat(float(W::k)), k, acc);
    }
    return acc;
}

template <int I> __device__ __forceinline__ double midw(int m);
template <> __device__ __forceinline__ double midw<4>(int m) { return (m == 0 || m == 3 ? -1.0 : 9.0) / 16.0; }
template <> __device__ __forceinline__ double midw<6>(int m) {
    return (m == 0 || m == 5 ? 3.0 : (m == 1 || m == 4 ? -25.0 : 150.0)) / 256.0;
}
template <> __device__ __forceinline__ double midw<8>(int m) {
    const int k = m < 4 ? m : 7 - m;
    return (k == 0 ? -5.0 : (k == 1 ? 49.0 : (k == 2 ? -245.0 : 1225.0))) / 2048.0;
}

// Reduced-array extent per tangential axis: patch indices [tlo, tlo + TN)
// cover every tangential stencil of fine coordinates 0..n-1.  Patch index
// 4 + floor(q/2) is the coarse node at or left of fine coordinate q.
template <int I> __device__ __forceinline__ int tan_lo() { return 4 - I / 2 + 1; }
__host__ __device__ inline int tan_n(int n, int I) { return n / 2 + I - 1; }

// Coordinates of shell node t of an S^3 box without its (S-2)^3 interior:
// the z = 0 and z = S-1 planes, then the ring of each inner z plane.
__device__ __forceinline__ void shell_coords(int t, int S, int& x, int& y, int& z) {
    const int S2 = S * S;
    if (t < S2) { z = 0; y = t / S; x = t % S; return; }
    t -= S2;
    if (t < S2) { z = S - 1; y = t / S; x = t % S; return; }
    t -= S2;
    const int ring = 4 * S - 4;
    z = 1 + t / ring;
    int q = t % ring;
    if (q < S) { y = 0; x = q; return; }
    q -= S;
    if (q < S) { y = S - 1; x = q; return; }
    q -= S;
    y = 1 + (q >> 1);
    x = (q & 1) ? S - 1 : 0;
}

// Shared scratch of build_halo besides the block itself: the block's
// neighbourhood record.
struct __align__(16) HaloSmem {
    int rec[REC_INTS];
};
// Shared scratch of the transposed ghost fill.
template <typename T>
struct HaloSmemT {
    int snbr[27], cnbr[27], cleaf[27], cch[27 * 8], off[27], rdir[27], rstart[27];
    T sw[8];
    int interp, outside, nreg, ntot;
};

__host__ __device__ inline int pool_size(int n, int I) {
    const int TN = tan_n(n, I);
    return 6 * TN * TN + 12 * TN + 8;
}



// Per-axis description of one interpolated ghost region d: its tangential
// axes ta0 < ta1 (x, y, z order) with their patch strides, the patch strides
// of the normal axes on a -1 side (I-point midpoint stencils) and the patch
// offset of its element 0 (a +1 side is the coincident coarse node, patch
// index `up`; a tangential axis starts at patch index 1).  All fields are
// scalars so that the region stays in registers.
struct Region {
    int d0, d1, d2;            // side per axis: -1, 0 (tangential), +1
    int nt, nn, ta0, ta1;
    int ts0, ts1, ns0, ns1, ns2, p0;
};
__device__ __forceinline__ Region region_of(int d, int PL, int up) {
    Region g;
    g.d0 = d % 3 - 1; g.d1 = (d / 3) % 3 - 1; g.d2 = d / 9 - 1;
    g.nt = 0; g.nn = 0; g.ta0 = 0; g.ta1 = 0;
    g.ts0 = 0; g.ts1 = 0; g.ns0 = 0; g.ns1 = 0; g.ns2 = 0; g.p0 = 0;
    const int dd[3] = {g.d0, g.d1, g.d2};
    int st = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (dd[a] == 0) {
            if (g.nt == 0) { g.ta0 = a; g.ts0 = st; } else { g.ta1 = a; g.ts1 = st; }
            ++g.nt;
            g.p0 += st;
        } else if (dd[a] < 0) {
            if (g.nn == 0) g.ns0 = st; else if (g.nn == 1) g.ns1 = st; else g.ns2 = st;
            ++g.nn;
        } else {
            g.p0 += up * st;
        }
        st *= PL;
    }
    return g;
}
// Box coordinate on axis a of the region's ghost node with tangential box
// coordinates u1 (axis ta0) and v1 (axis ta1).
__device__ __forceinline__ int box_coord(int side, int a, const Region& g, int S, int u1, int v1) {
    return side != 0 ? (side < 0 ? 0 : S - 1) : (a == g.ta0 ? u1 : v1);
}

// Starts the copy of block b's neighbourhood record into shared memory (one
// cp.async group, committed); the caller waits for it.
__device__ __forceinline__ void load_record(HaloSmem& hs, const LevelView& lk, int b) {
    for (int c = threadIdx.x; c < REC_INTS / 4; c += blockDim.x)
        cp_async16(&hs.rec[4 * c], lk.rec + (size_t)b * REC_INTS + 4 * c);
    cp_async_commit();
}

// Starts the copy of block b's n^3 right-hand side into shared memory in the
// split layout (one thread per (x, y) column walking z, cp.async), and
// commits a cp.async group.
template <typename T>
__device__ __forceinline__ void load_rhs(T* __restrict__ fs, const T* __restrict__ F, int b, int n) {
    const int h = n >> 1, Fp = split_fp(n, (int)sizeof(T)), Fr = split_fr(n, (int)sizeof(T));
    const int F3 = split_f3(n, (int)sizeof(T));
    const T* Fb = F + (size_t)b * n * n * n;
    for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
        const int y = c / n, x = c - y * n;
        T* dcol = fs + (((y & 1) << 1) | (x & 1)) * F3 + (y >> 1) * Fr + (x >> 1);
        const T* scol = Fb + c;
        for (int m = 0; m < h; ++m) {
            cp_async_el(dcol + m * Fp, scol + (size_t)(2 * m) * n * n);
            cp_async_el(dcol + 4 * F3 + m * Fp, scol + (size_t)(2 * m + 1) * n * n);
        }
    }
    cp_async_commit();
}

// Builds the block's (n+2)^3 box in shared memory (parity-split layout).
// Expects the block's record in hs (complete and visible: the caller waited
// for its copy and synchronised).  Waits for every cp.async group of the
// thread, so a right-hand side staged by the caller is complete on return.
//  1. Copied values, one thread per (X, Y) column of the box, walking Z: the
//     block's own interior, same-level neighbours' interiors, and the stored
//     ghost layer where the region lies outside the domain (cp.async).
//  2. Interpolated regions (no same-level neighbour), separably:
//     a. stage the coarse patch over the hull of the regions' stencils
//        (cp.async, issued with the box copies);
//     b. reduce each region along its normal axes (one value per coarse
//        tangential node);
//     c. faces: interpolate along the first tangential axis into fine x
//        coarse rows; edges and corners: final values;
//     d. faces: interpolate along the second tangential axis.
//     Work items are ordered so that the lanes of a warp share the parity of
//     the interpolated coordinate (the same stencil length).
// Issues the cp.async copies of block b's box (step 1 below) and, for a block
// with interpolated regions, of its coarse patch (step 2a) without committing
// them; the caller commits, waits and synchronises before halo_interpolate.
template <typename T, int I, bool INTERP = true, bool OWN = false>
__device__ __forceinline__ void halo_issue(T* __restrict__ su, T* __restrict__ patch, const int* __restrict__ rec,
                                           const T* __restrict__ Uk, const T* __restrict__ Uc, const LevelView& lk,
                                           int b, int n, const Split& sp) {
    const int S = n + 2, S2 = S * S, S3 = S2 * S;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int H = sp.H, H2 = sp.H2, H3p = sp.H3p;
    const int h = n >> 1;
    const int* __restrict__ snbr = rec + REC_SNBR;
    // 1. copied values
    for (int c = tid; c < S2; c += nth) {
        const int Y = c / S, X = c - Y * S;
        const int rx = X == 0 ? -1 : (X == S - 1 ? 1 : 0);
        const int ry = Y == 0 ? -1 : (Y == S - 1 ? 1 : 0);
        T* dcol = su + ((((Y & 1) << 1) | (X & 1)) * H3p + (Y >> 1) * H + (X >> 1));
#pragma unroll
        for (int rz = -1; rz <= 1; ++rz) {
            if (OWN && (rx | ry | rz) == 0) continue;     // the block's own interior: issued by own_box_issue()
            const int j = snbr[dir27(rx, ry, rz)];
            if (j == NBR_MISSING) continue;
            // source column: same-level block j (shifted into its own box), or this block's stored ghost layer
            const T* col = Uk + (j >= 0 ? (size_t)j * S3 + (size_t)((Y - ry * n) * S + X - rx * n)
                                        : (size_t)b * S3 + (size_t)(Y * S + X));
            if (rz != 0) {
                const int Z = rz < 0 ? 0 : S - 1;
                const int Zs = j >= 0 ? Z - rz * n : Z;
                cp_async_el(dcol + (Z & 1) * 4 * H3p + (Z >> 1) * H2, col + (size_t)Zs * S2);
            } else {
                // Z = 2m + 1 (odd sub-array, index m) and Z = 2m + 2 (even sub-array, index m + 1)
                for (int m = 0; m < h; ++m) {
                    cp_async_el(dcol + 4 * H3p + m * H2, col + (size_t)(2 * m + 1) * S2);
                    cp_async_el(dcol + (m + 1) * H2, col + (size_t)(2 * m + 2) * S2);
                }
            }
        }
    }
    if constexpr (INTERP) {
        const int nreg = rec[REC_NREG];
        constexpr int plo = 4 - I / 2;
        const int PL = h + I, PL2 = PL * PL;
        const int* __restrict__ pnbr = rec + REC_PNBR;
        const int* __restrict__ pch = rec + REC_PCH;
        // 2a. coarse patch over the hull, copied together with the box; patch
        //     index p on an axis is coarse coordinate base + p relative to the
        //     parent's origin.  A covered coarse node takes its coincident fine
        //     node from the input level (for this block too: the box holds the
        //     same values until the caller changes it).
        if (nreg > 0) {
            const int bx = lk.coords[3 * b], by = lk.coords[3 * b + 1], bz = lk.coords[3 * b + 2];
            const int bs0 = (bx & 1) * h - 4 + plo, bs1 = (by & 1) * h - 4 + plo, bs2 = (bz & 1) * h - 4 + plo;
            const int lo0 = rec[REC_LO], lo1 = rec[REC_LO + 1], z0 = rec[REC_LO + 2];
            const int L0 = rec[REC_HI] - lo0, L1 = rec[REC_HI + 1] - lo1, z1 = rec[REC_HI + 2];
            for (int c = tid; c < L0 * L1; c += nth) {
                const int q1 = c / L0, q0 = c - q1 * L0;
                const int px = lo0 + q0, py = lo1 + q1;
                const int rx = bs0 + px, ry = bs1 + py;
                const int ex = rx < 0 ? -1 : (rx >= n ? 1 : 0), ey = ry < 0 ? -1 : (ry >= n ? 1 : 0);
                const int lx = rx - ex * n, ly = ry - ey * n;
                const int ox = lx >= h, oy = ly >= h;
                const int FX = 2 * lx - ox * n + 1, FY = 2 * ly - oy * n + 1;
                T* pcol = patch + py * PL + px;
                for (int pz = z0; pz < z1; ++pz) {
                    const int rz = bs2 + pz;
                    const int ez = rz < 0 ? -1 : (rz >= n ? 1 : 0);
                    const int lz = rz - ez * n;
                    const int d = dir27(ex, ey, ez);
                    const int oz = lz >= h;
                    const int ch = pch[8 * d + ox + 2 * oy + 4 * oz];
                    if (pch[8 * d] < 0) {
                        // leaf coarse block
                        cp_async_el(pcol + pz * PL2, Uc + ((size_t)pnbr[d] * S3 + (size_t)(((lz + 1) * S + ly + 1) * S + lx + 1)));
                    } else {
                        // covered coarse node: the coincident fine node of the current level
                        const int FZ = 2 * lz - oz * n + 1;
                        cp_async_el(pcol + pz * PL2, Uk + ((size_t)ch * S3 + (size_t)((FZ * S + FY) * S + FX)));
                    }
                }
            }
        }
    }
}

// Steps 2b-2d below for block b, whose box and coarse patch copies are
// complete and visible; returns after a barrier (at once without
// interpolated regions).
template <typename T, int I>
__device__ __forceinline__ void halo_interpolate(T* __restrict__ su, T* __restrict__ pool, T* __restrict__ patch,
                                                 const int* __restrict__ rec, const LevelView& lk, int b, int n,
                                                 const Split& sp) {
    const int S = n + 2;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int h = n >> 1;
    const int nreg = rec[REC_NREG];
    constexpr int plo = 4 - I / 2;
    const int TN = tan_n(n, I);
    const int PL = h + I;
    const int up = 4 + h - plo;          // patch index coincident with fine coordinate n
    if (nreg == 0) return;
    T w[I];
#pragma unroll
    for (int m = 0; m < I; ++m) w[m] = T(midw<I>(m));
    const unsigned mTN = magic_of(TN);
    const int* __restrict__ rdir = rec + REC_RDIR;
    const int* __restrict__ roff = rec + REC_ROFF;
    const int* __restrict__ raoff = rec + REC_RAOFF;
    const int* __restrict__ coff = rec + REC_COFF;
    const int* __restrict__ doff = rec + REC_DOFF;
    // Each pass is one flat loop over the items of all regions; the region of
    // item f is the last one whose first item is <= f.
    auto region_at = [&](const int* __restrict__ off, int f) {
        int lo = 0, hi = nreg;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (off[mid] <= f) lo = mid;
            else hi = mid;
        }
        return lo;
    };
    // 2b. reduction along the normal axes: one value per coarse tangential node
    const int nB = rec[REC_NTOT], nC = rec[REC_NTOT + 1], nD = rec[REC_NTOT + 2];
    for (int f = tid; f < nB; f += nth) {
        const int r = region_at(roff, f);
        const Region g = region_of(rdir[r], PL, up);
        const int e = f - roff[r];
        const int e1 = g.nt == 2 ? fdiv(e, mTN) : 0, e0 = e - e1 * TN;
        const T* p = patch + g.p0 + e0 * g.ts0 + e1 * g.ts1;
        const int s0 = g.ns0, s1 = g.ns1, s2 = g.ns2;
        T acc = T(0);
        if (g.nn == 0) {
            acc = p[0];
        } else if (g.nn == 1) {
#pragma unroll
            for (int m = 0; m < I; ++m) acc += w[m] * p[m * s0];
        } else if (g.nn == 2) {
#pragma unroll
            for (int m1 = 0; m1 < I; ++m1) {
                T a = T(0);
#pragma unroll
                for (int m = 0; m < I; ++m) a += w[m] * p[m * s0 + m1 * s1];
                acc += w[m1] * a;
            }
        } else {
#pragma unroll 1
            for (int m2 = 0; m2 < I; ++m2) {
                T a2 = T(0);
#pragma unroll 1
                for (int m1 = 0; m1 < I; ++m1) {
                    T a = T(0);
#pragma unroll
                    for (int m = 0; m < I; ++m) a += w[m] * p[m * s0 + m1 * s1 + m2 * s2];
                    a2 += T(midw<I>(m1)) * a;
                }
                acc += T(midw<I>(m2)) * a2;
            }
        }
        pool[f] = acc;
    }
    __syncthreads();
    // 2c. faces: along the first tangential axis into A[v'][u] (fine u, coarse
    //     v'); edges and corners: their ghost values.  A reuses the patch.
    //     Reduced-array start of the stencil of fine coordinate q: q/2 + I/2 - 1
    //     (q even, one point) or (q - 1)/2 (q odd, I points).  A face's items
    //     run over even u first, then odd u.
    T* A = patch;
    const unsigned mh = magic_of(h), mn = magic_of(n);
    for (int f = tid; f < nC; f += nth) {
        const int r = region_at(coff, f);
        const Region g = region_of(rdir[r], PL, up);
        const int e = f - coff[r];
        const T* R = pool + roff[r];
        if (g.nt == 2) {
            const int par = e >= h * TN;
            const int e2 = e - par * h * TN;
            const int v = fdiv(e2, mh), u = 2 * (e2 - v * h) + par;
            T acc = T(0);
            if (!par) {
                acc = R[v * TN + u / 2 + I / 2 - 1];
            } else {
                const T* q = R + v * TN + (u - 1) / 2;
#pragma unroll
                for (int m = 0; m < I; ++m) acc += w[m] * q[m];
            }
            A[raoff[r] + v * n + u] = acc;
        } else if (g.nt == 1) {
            const int u = e;
            T acc = T(0);
            if (!(u & 1)) {
                acc = R[u / 2 + I / 2 - 1];
            } else {
#pragma unroll
                for (int m = 0; m < I; ++m) acc += w[m] * R[(u - 1) / 2 + m];
            }
            su[sp.at(box_coord(g.d0, 0, g, S, u + 1, 0), box_coord(g.d1, 1, g, S, u + 1, 0),
                     box_coord(g.d2, 2, g, S, u + 1, 0))] = acc;
        } else {
            su[sp.at(box_coord(g.d0, 0, g, S, 0, 0), box_coord(g.d1, 1, g, S, 0, 0), box_coord(g.d2, 2, g, S, 0, 0))] =
                R[0];
        }
    }
    __syncthreads();
    // 2d. faces: along the second tangential axis (fine v), rows of fine u,
    //     even v first
    for (int f = tid; f < nD; f += nth) {
        const int r = region_at(doff, f);
        const Region g = region_of(rdir[r], PL, up);
        const int e = f - doff[r];
        const T* Ar = A + raoff[r];
        const int row = fdiv(e, mn), u = e - row * n;
        const int par = row >= h;
        const int v = 2 * (row - par * h) + par;
        T acc = T(0);
        if (!par) {
            acc = Ar[(v / 2 + I / 2 - 1) * n + u];
        } else {
            const T* q = Ar + ((v - 1) / 2) * n + u;
#pragma unroll
            for (int m = 0; m < I; ++m) acc += w[m] * q[m * n];
        }
        su[sp.at(box_coord(g.d0, 0, g, S, u + 1, v + 1), box_coord(g.d1, 1, g, S, u + 1, v + 1),
                 box_coord(g.d2, 2, g, S, u + 1, v + 1))] = acc;
    }
    __syncthreads();
}

template <typename T, int I, bool INTERP = true, bool OWN = false>
__device__ __forceinline__ void build_halo(T* __restrict__ su, T* __restrict__ pool, T* __restrict__ patch,
                                           const int* __restrict__ rec, const T* __restrict__ Uk, const T* __restrict__ Uc,
                                           const LevelView& lk, int b, int n, const Split& sp) {
    halo_issue<T, I, INTERP, OWN>(su, patch, rec, Uk, Uc, lk, b, n, sp);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    if constexpr (INTERP) halo_interpolate<T, I>(su, pool, patch, rec, lk, b, n, sp);
}

__host__ __device__ inline int patch_size(int n, int I) {
    const int PL = n / 2 + I;
    return PL * PL * PL;
}

// Dynamic shared memory of the fused kernels: the split box, then the
// reduced array and the patch of the interpolation.  The smoother stages the
// block's right-hand side in one of two ways (fmode):
//   1: over that second area, once the ghost layer is built;
//   2: in an area of its own after it, copied together with the box (more
//      shared memory, one memory round trip less on interface blocks).
// Both areas start at 16-byte boundaries (the split box is a multiple of 32
// elements).
__host__ __device__ inline size_t rhs_offset(int n, size_t el) { return el * 8 * (size_t)split_h3p(n, (int)el); }
__host__ __device__ inline size_t rhs_offset2(int n, int I, size_t el) {
    const size_t e = rhs_offset(n, el) + el * ((size_t)pool_size(n, I) + (size_t)patch_size(n, I));
    return (e + 15) / 16 * 16;
}
template <typename T>
__host__ __device__ inline size_t fused_smem(int n, int I, int fmode = 0) {
    const size_t interp = (size_t)pool_size(n, I) + (size_t)patch_size(n, I), f = 8 * (size_t)split_f3(n, sizeof(T));
    if (fmode == 2) return rhs_offset2(n, I, sizeof(T)) + sizeof(T) * f;
    return rhs_offset(n, sizeof(T)) + sizeof(T) * (fmode == 1 && f > interp ? f : interp);
}


// The copies of block b's own interior into its split box (the part of the
// box that needs no record: z = 1..n of its own columns), one thread per
// (x, y) column walking z; not committed.
template <typename T>
__device__ __forceinline__ void own_box_issue(T* __restrict__ su, const T* __restrict__ Uk, int b, int n, const Split& sp) {
    const int S = n + 2, S2 = S * S, h = n >> 1;
    const T* Ub = Uk + (size_t)b * S2 * S;
    for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
        const int y = c / n, x = c - y * n;
        const int X = x + 1, Y = y + 1;
        T* dcol = su + ((((Y & 1) << 1) | (X & 1)) * sp.H3p + (Y >> 1) * sp.H + (X >> 1));
        const T* col = Ub + (Y * S + X);
        for (int m = 0; m < h; ++m) {
            cp_async_el(dcol + 4 * sp.H3p + m * sp.H2, col + (size_t)(2 * m + 1) * S2);
            cp_async_el(dcol + (m + 1) * sp.H2, col + (size_t)(2 * m + 2) * S2);
        }
    }
}

// Prologue of the fused kernels: the block's record, complete and visible on
// return.  With OWN, the copy of the block's own interior from Uk, which
// needs no record, is in flight behind it (build_halo<..., OWN = true> copies
// the rest and waits for both), so that the record's memory round trip
// overlaps the largest copy.  FP64 boxes take OWN; FP32 boxes measured
// slightly slower with it and keep the record first.
template <typename T, bool OWN = (sizeof(T) == 8)>
__device__ __forceinline__ void record_prologue_own(HaloSmem& hs, const LevelView& lk, int b, T* __restrict__ su,
                                                    const T* __restrict__ Uk, int n, const Split& sp) {
    load_record(hs, lk, b);
    if constexpr (OWN) {
        own_box_issue(su, Uk, b, n, sp);
        cp_async_commit();
        cp_async_wait<1>();
    } else {
        cp_async_wait<0>();
    }
    __syncthreads();
}


// Pair p (0 <= p < 256) of a colour's nodes for the fixed block size 16
// (h = 8): split indices (i, j, l) and (i + 1, j, l) with i = 2 (p & 3),
// l = 2 ((p >> 2) & 3) + (p >> 7), j = ((p >> 4) & 1) + 2 ((p >> 5) & 3).  A
// warp's lanes take i-pairs fastest (4), then 4 z rows of one parity
// (l = 0, 2, 4, 6 or 1, 3, 5, 7), then 2 y rows; with the FP32 plane strides
// Hp = 84 (box) and Fp = 76 (staged right-hand side) and row strides 9, its
// loads fall in 32 distinct banks.  Pairs p and p + 128 are z-adjacent (l and
// l + 1): a thread that takes both shares between their stencils the plane
// that lies between them.
struct Pair { int i, j, l; };
__device__ __forceinline__ Pair pair_of(int p) {
    Pair q;
    q.i = 2 * (p & 3);
    q.l = 2 * ((p >> 2) & 3) + (p >> 7);
    q.j = ((p >> 4) & 1) + 2 * ((p >> 5) & 3);
    return q;
}

// Writes planes Z = 1..16 of a block-size-16 FP32 box, ghost rows and
// columns included, from the split box in shared memory to the block's 18^3
// array: one contiguous run of 16 x 18^2 floats that starts on a 16-byte
// boundary (18^3 and 18^2 are multiples of 4), written with 16-byte stores,
// so that every 32-byte sector is written whole (no read-modify-write of
// partly written sectors in DRAM).  On levels >= 1 nothing reads the stored
// ghost layer of a field (the stencil kernels rebuild it from the
// neighbours' interiors and the coarse level, the prolongation reads the
// neighbours' interiors), so the halo values stored there are harmless.
__device__ __forceinline__ void store_planes16(float* __restrict__ Ub, const float* __restrict__ su, const Split& sp,
                                               int nthreads) {
    // A float4 starts at an even x (S is even): its elements x, x+1, x+2, x+3
    // sit at a, a + H3p, a + 1, a + H3p + 1 of the split box (a = at(x, y, z)),
    // except at x = 16, where the last two start the next row.
    constexpr int S = 18, S2 = S * S, NV = 16 * S2 / 4;
    float4* __restrict__ dst = reinterpret_cast<float4*>(Ub + S2);
    for (int t = threadIdx.x; t < NV; t += nthreads) {
        const int q = 4 * t;
        const int Zr = q / S2, r = q - Zr * S2, Y = r / S, X = r - Y * S;
        const int a = sp.at(X, Y, Zr + 1);
        // x + 2 at a + 1, or (x = 16) column 0 of the next row, never in the
        // next plane (x = 16 in a plane's last row has 4 t = 2 (mod 4))
        const int a2 = X < S - 2 ? a + 1 : sp.at(0, Y + 1, Zr + 1);
        float4 v;
        v.x = su[a];
        v.y = su[a + sp.H3p];
        v.z = su[a2];
        v.w = su[a2 + sp.H3p];
        dst[t] = v;
    }
}

// ---------------------------------------------------------------- smoother
// One Gauss-Seidel iteration (Sec. 3.1): 8 colours c = (x&1) + 2(y&1) + 4(z&1),
// u <- (den h^2 f - offcentre) / c; reads Uin, writes the interior to Uout.
template <int M, typename T, int I, int NC>
__global__ void __launch_bounds__(512) k_smooth_fused(T* __restrict__ Uout, const T* __restrict__ Uin,
                                                      const T* __restrict__ F, const T* __restrict__ Uc, LevelView lk,
                                                      int n_arg, T h2den, const int* __restrict__ order, int fmode) {
    const int n = NC ? NC : n_arg;    // NC: block size fixed at compile time (0: runtime)
    extern __shared__ __align__(16) unsigned char fz_smem[];
    T* su = reinterpret_cast<T*>(fz_smem);
    const Split sp = split_of<T>(n);
    T* pool = su + 8 * sp.H3p;
    T* patch = pool + pool_size(n, I);
    // staged right-hand side (fmode 1: over the interpolation scratch; 2: its own area)
    T* fs = fmode == 2 ? reinterpret_cast<T*>(fz_smem + rhs_offset2(n, I, sizeof(T))) : pool;
    __shared__ HaloSmem hs;
    Cset cs;
    cset_init(cs, n >> 1);
    const int b = order ? order[blockIdx.x] : blockIdx.x;
    record_prologue_own(hs, lk, b, su, Uin, n, sp);
    // the right-hand side copy overlaps the box copy (build_halo waits for
    // both); in fmode 1 it goes over the interpolation scratch, so an
    // interface block, which needs that scratch first, reads its right-hand
    // side from global memory instead (fm = 0)
    const int fm = (fmode == 1 && hs.rec[REC_NREG] != 0) ? 0 : fmode;
    if (fm) load_rhs(fs, F, b, n);
    build_halo<T, I, true, sizeof(T) == 8>(su, pool, patch, hs.rec, Uin, Uc, lk, b, n, sp);
    const T* Fb = F + (size_t)b * n * n * n;
    const int Fp = split_fp(n, (int)sizeof(T)), Fr = split_fr(n, (int)sizeof(T)), F3 = split_f3(n, (int)sizeof(T));
    const T inv_c = T(1) / T(LW<M>::c);
    if constexpr (NC != 0 && sizeof(T) == 4) {
        // Fixed block size, FP32: each work item is a pair of a colour's nodes
        // adjacent along x (split indices i, i + 1), whose stencils share the
        // values of the fine plane between them (the +x neighbours of the
        // first are the -x neighbours of the second); lane order: pair_of.
        // A 128-thread CTA gives each thread the z-adjacent pairs p and
        // p + 128 and loads all four stencils before it stores, so that the
        // plane between the pairs is loaded once.
        constexpr int hh = NC / 2, NP = hh * hh * hh / 2, NU = NP / 2;
        static_assert(hh == 8, "the pair lane order assumes h = 8");
#pragma unroll
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
            if (blockDim.x == NU) {
                const Pair q = pair_of(threadIdx.x);
                const int b0 = c.cb + q.l * sp.H2 + q.j * sp.H + q.i, b1 = b0 + sp.H2;
                T fa0, fb0, fa1, fb1;
                if (fm) {
                    const int fi = col * F3 + q.l * Fp + q.j * Fr + q.i;
                    fa0 = fs[fi]; fb0 = fs[fi + 1];
                    fa1 = fs[fi + Fp]; fb1 = fs[fi + Fp + 1];
                } else {
                    const int fi = ((2 * q.l) * n + 2 * q.j) * n + 2 * q.i + c.fo;
                    fa0 = Fb[fi]; fb0 = Fb[fi + 2];
                    fa1 = Fb[fi + 2 * n * n]; fb1 = Fb[fi + 2 * n * n + 2];
                }
                const f2_t s0 = offc2<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2);
                const f2_t s1 = offc2<M>(su, b1, c.dX, c.dY, c.dZ, sp.H, sp.H2);
                const f2_t hd = f2splat(h2den), ic = f2splat(inv_c);
                const f2_t v0 = f2mul(f2sub(f2mul(hd, f2pk(fa0, fb0)), s0), ic);
                const f2_t v1 = f2mul(f2sub(f2mul(hd, f2pk(fa1, fb1)), s1), ic);
                const int d = c.dX + c.dY + c.dZ;
                f2up(v0, su[b0 + d], su[b0 + 1 + d]);
                f2up(v1, su[b1 + d], su[b1 + 1 + d]);
                __syncthreads();
                continue;
            }
            for (int p = threadIdx.x; p < NP; p += blockDim.x) {
                const Pair q = pair_of(p);
                const int i = q.i, j = q.j, l = q.l;
                const int b0 = c.cb + l * sp.H2 + j * sp.H + i;
                T fa, fb;
                if (fm) {
                    const int fi = col * F3 + l * Fp + j * Fr + i;
                    fa = fs[fi];
                    fb = fs[fi + 1];
                } else {
                    const int fi = ((2 * l) * n + 2 * j) * n + 2 * i + c.fo;
                    fa = Fb[fi];
                    fb = Fb[fi + 2];
                }
                const f2_t sab = offc2<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2);
                const f2_t v = f2mul(f2sub(f2mul(f2splat(h2den), f2pk(fa, fb)), sab), f2splat(inv_c));
                f2up(v, su[b0 + c.dX + c.dY + c.dZ], su[b0 + 1 + c.dX + c.dY + c.dZ]);
            }
            __syncthreads();
        }
    } else {
        // (colour loop not unrolled: the FP64 sweep is bound by its arithmetic, and
        // the runtime-size build has no constant offsets to gain)
#pragma unroll 1
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < cs.cnt) {
                    const Node d = node_of(cs.q[k], sp, n, Fp, Fr);
                    const int b0 = c.cb + d.b0;
                    const T fv = fm ? fs[col * F3 + d.fs] : Fb[d.f + c.fo];
                    su[b0 + c.dX + c.dY + c.dZ] =
                        (h2den * fv - offc_s<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2)) * inv_c;
                }
            __syncthreads();
        }
    }
    const int S = n + 2, S2 = S * S;
    T* Ob = Uout + (size_t)b * S2 * S;
    if constexpr (NC == 16 && sizeof(T) == 4) {
        store_planes16(reinterpret_cast<float*>(Ob), reinterpret_cast<const float*>(su), sp, blockDim.x);
        return;
    }
    // interior back to global, one thread per (x, y) column
    for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
        const int y = c / n, x = c - y * n;
        const int X = x + 1, Y = y + 1;
        const T* scol = su + ((((Y & 1) << 1) | (X & 1)) * sp.H3p + (Y >> 1) * sp.H + (X >> 1));
        T* gcol = Ob + (Y * S + X);
        for (int m = 0; m < (n >> 1); ++m) {
            gcol[(2 * m + 1) * S2] = scol[4 * sp.H3p + m * sp.H2];
            gcol[(2 * m + 2) * S2] = scol[(m + 1) * sp.H2];
        }
    }
}

// ---------------------------------------------------------------- residual r = f - L u (all nodes)
template <int M, typename T, int I, int NC>
__global__ void __launch_bounds__(512) k_residual_fused(T* __restrict__ R, const T* __restrict__ U,
                                                        const T* __restrict__ F, const T* __restrict__ Uc, LevelView lk,
                                                        int n_arg, T scale, const int* __restrict__ order, int stage) {
    const int n = NC ? NC : n_arg;    // NC: block size fixed at compile time (0: runtime)
    extern __shared__ __align__(16) unsigned char fz_smem[];
    T* su = reinterpret_cast<T*>(fz_smem);
    const Split sp = split_of<T>(n);
    T* pool = su + 8 * sp.H3p;
    T* patch = pool + pool_size(n, I);
    __shared__ HaloSmem hs;
    Cset cs;
    cset_init(cs, n >> 1);
    const int b = order ? order[blockIdx.x] : blockIdx.x;
    record_prologue_own(hs, lk, b, su, U, n, sp);
    const size_t n3 = (size_t)n * n * n;
    if constexpr (NC != 0 && sizeof(T) == 4) {
        const int Fp = split_fp(n, 4), Fr = split_fr(n, 4), F3 = split_f3(n, 4);
        constexpr int NP = (NC / 2) * (NC / 2) * (NC / 2) / 2, NU = NP / 2;
        auto lpair = [&](const Col& c, int b0, T& la, T& lb) {
            const int d = c.dX + c.dY + c.dZ;
            const f2_t l = f2fma(f2splat(float(LW<M>::c)), f2pk(su[b0 + d], su[b0 + 1 + d]),
                                 offc2<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2));
            f2up(l, la, lb);
        };
        if (!stage) {
            // F read and R written in global memory by the pairs themselves
            // (no staging round trip; the same arithmetic as below)
            build_halo<T, I, true, false>(su, pool, patch, hs.rec, U, Uc, lk, b, n, sp);
            const T* Fb = F + b * n3;
            T* Rb = R + b * n3;
#pragma unroll
            for (int col = 0; col < 8; ++col) {
                const Col c = colour(col, sp, n);
                for (int p = threadIdx.x; p < NP; p += blockDim.x) {
                    const Pair q = pair_of(p);
                    T la, lb;
                    lpair(c, c.cb + q.l * sp.H2 + q.j * sp.H + q.i, la, lb);
                    const int gi = ((2 * q.l) * n + 2 * q.j) * n + 2 * q.i + c.fo;
                    Rb[gi] = Fb[gi] - scale * la;
                    Rb[gi + 2] = Fb[gi + 2] - scale * lb;
                }
            }
            return;
        }
        // F staged in shared memory in the colour split (as the smoother's),
        // over the interpolation scratch: copied with the box where the block
        // has no interpolated regions, after the ghost layer otherwise.  Each
        // pair's residual replaces its F there; the block's R then goes out by
        // columns (whole 64-byte rows).  Pairs of nodes adjacent along x as in
        // the smoother (two z-adjacent pairs per thread in a 128-thread CTA).
        T* fs = pool;
        const bool early = hs.rec[REC_NREG] == 0;
        if (early) load_rhs(fs, F, b, n);
        build_halo<T, I, true, sizeof(T) == 8>(su, pool, patch, hs.rec, U, Uc, lk, b, n, sp);
        if (!early) {
            load_rhs(fs, F, b, n);
            cp_async_wait<0>();
            __syncthreads();
        }
#pragma unroll
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
            if (blockDim.x == NU) {
                const Pair q = pair_of(threadIdx.x);
                const int b0 = c.cb + q.l * sp.H2 + q.j * sp.H + q.i;
                T la0, lb0, la1, lb1;
                lpair(c, b0, la0, lb0);
                lpair(c, b0 + sp.H2, la1, lb1);
                const int fi = col * F3 + q.l * Fp + q.j * Fr + q.i, fj = fi + Fp;
                fs[fi] = fs[fi] - scale * la0;
                fs[fi + 1] = fs[fi + 1] - scale * lb0;
                fs[fj] = fs[fj] - scale * la1;
                fs[fj + 1] = fs[fj + 1] - scale * lb1;
                continue;
            }
            for (int p = threadIdx.x; p < NP; p += blockDim.x) {
                const Pair q = pair_of(p);
                const int b0 = c.cb + q.l * sp.H2 + q.j * sp.H + q.i;
                T la, lb;
                lpair(c, b0, la, lb);
                const int fi = col * F3 + q.l * Fp + q.j * Fr + q.i;
                fs[fi] = fs[fi] - scale * la;
                fs[fi + 1] = fs[fi + 1] - scale * lb;
            }
        }
        __syncthreads();
        // R by (x, y) columns walking z, the inverse of load_rhs's copy
        T* Rb = R + b * n3;
        for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
            const int y = c / n, x = c - y * n;
            const T* scol = fs + (((y & 1) << 1) | (x & 1)) * F3 + (y >> 1) * Fr + (x >> 1);
            T* gcol = Rb + c;
#pragma unroll
            for (int m = 0; m < NC / 2; ++m) {
                gcol[(size_t)(2 * m) * n * n] = scol[m * Fp];
                gcol[(size_t)(2 * m + 1) * n * n] = scol[4 * F3 + m * Fp];
            }
        }
    } else {
        build_halo<T, I, true, sizeof(T) == 8>(su, pool, patch, hs.rec, U, Uc, lk, b, n, sp);
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < cs.cnt) {
                    const Node d = node_of(cs.q[k], sp, n);
                    const int b0 = c.cb + d.b0;
                    const T l = T(LW<M>::c) * su[b0 + c.dX + c.dY + c.dZ] + offc_s<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2);
                    const size_t fi = b * n3 + d.f + c.fo;
                    R[fi] = F[fi] - scale * l;
                }
        }
    }
}

// ---------------------------------------------------------------- FAS RHS and u-hat (Alg. 1)
// F += L u on covered blocks; H = u on every block.
template <int M, typename T, int I, int NC>
__global__ void __launch_bounds__(512) k_fas_fused(T* __restrict__ F, T* __restrict__ H, const T* __restrict__ U,
                                                   const T* __restrict__ Uc, LevelView lk, int n_arg, T scale,
                                                   const int* __restrict__ order) {
    const int n = NC ? NC : n_arg;    // NC: block size fixed at compile time (0: runtime)
    extern __shared__ __align__(16) unsigned char fz_smem[];
    T* su = reinterpret_cast<T*>(fz_smem);
    const Split sp = split_of<T>(n);
    T* pool = su + 8 * sp.H3p;
    T* patch = pool + pool_size(n, I);
    __shared__ HaloSmem hs;
    const int S = n + 2, S3 = S * S * S;
    const size_t n3 = (size_t)n * n * n;
    const int b = order ? order[blockIdx.x] : blockIdx.x;
    Cset cs;
    cset_init(cs, n >> 1);
    const bool cov = !lk.is_leaf[b];
    if (!cov) {
        const T* Ub = U + (size_t)b * S3;
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < cs.cnt) {
                    const Node d = node_of(cs.q[k], sp, n);
                    H[b * n3 + d.f + c.fo] = Ub[d.g + c.go];
                }
        }
        return;
    }
    record_prologue_own(hs, lk, b, su, U, n, sp);
    if constexpr (NC != 0 && sizeof(T) == 4) {
        // F staged in shared memory over the interpolation scratch as in the
        // residual kernel, updated in place and written back by columns;
        // node pairs adjacent along x as in the smoother
        T* fs = pool;
        const bool early = hs.rec[REC_NREG] == 0;
        if (early) load_rhs(fs, F, b, n);
        build_halo<T, I, true, sizeof(T) == 8>(su, pool, patch, hs.rec, U, Uc, lk, b, n, sp);
        if (!early) {
            load_rhs(fs, F, b, n);
            cp_async_wait<0>();
            __syncthreads();
        }
        const int Fp = split_fp(n, 4), Fr = split_fr(n, 4), F3 = split_f3(n, 4);
        constexpr int NP = (NC / 2) * (NC / 2) * (NC / 2) / 2;
#pragma unroll
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
            for (int p = threadIdx.x; p < NP; p += blockDim.x) {
                const Pair q = pair_of(p);
                const int b0 = c.cb + q.l * sp.H2 + q.j * sp.H + q.i;
                const T ua = su[b0 + c.dX + c.dY + c.dZ], ub = su[b0 + 1 + c.dX + c.dY + c.dZ];
                T la, lb;
                f2up(f2fma(f2splat(float(LW<M>::c)), f2pk(ua, ub), offc2<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2)),
                     la, lb);
                const int si = col * F3 + q.l * Fp + q.j * Fr + q.i;
                fs[si] += scale * la;
                fs[si + 1] += scale * lb;
                const size_t fi = b * n3 + ((2 * q.l) * n + 2 * q.j) * n + 2 * q.i + c.fo;
                H[fi] = ua;
                H[fi + 2] = ub;
            }
        }
        __syncthreads();
        T* Fb = F + b * n3;
        for (int c = threadIdx.x; c < n * n; c += blockDim.x) {
            const int y = c / n, x = c - y * n;
            const T* scol = fs + (((y & 1) << 1) | (x & 1)) * F3 + (y >> 1) * Fr + (x >> 1);
            T* gcol = Fb + c;
#pragma unroll
            for (int m = 0; m < NC / 2; ++m) {
                gcol[(size_t)(2 * m) * n * n] = scol[m * Fp];
                gcol[(size_t)(2 * m + 1) * n * n] = scol[4 * F3 + m * Fp];
            }
        }
    } else {
        build_halo<T, I, true, sizeof(T) == 8>(su, pool, patch, hs.rec, U, Uc, lk, b, n, sp);
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < cs.cnt) {
                    const Node d = node_of(cs.q[k], sp, n);
                    const int b0 = c.cb + d.b0;
                    const T u = su[b0 + c.dX + c.dY + c.dZ];
                    const size_t fi = b * n3 + d.f + c.fo;
                    F[fi] += scale * (T(LW<M>::c) * u + offc_s<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2));
                    H[fi] = u;
                }
        }
    }
}

// ---------------------------------------------------------------- leaf residual (FP64 stop rule / outer residual)
__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) { return a > b ? a : b; }
__device__ __forceinline__ void bmax_atomic(double v, unsigned long long* out) {
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

// The FP64 box of a fixed block size NC in 64-bit fixed point, in place: its
// largest exponent field E (a block-wide max held in *emax, zero on entry)
// fixes the scale 2^s, s = 1084 - G - E, so that every |u 2^s| < 2^(62 - G);
// each value becomes trunc(u 2^s) (to_fixed) as the bit pattern of its
// double slot.  Returns E, or -1 with the box unchanged where the box holds
// Inf or NaN, only zeros and subnormals, or exponents whose scales 2^-s
// would leave the normal range (E < 128 or E > 1900).  Ends with a barrier.
template <int NC, int G>
__device__ __forceinline__ int box_to_fixed(double* __restrict__ su, const Split& sp, unsigned* emax) {
    constexpr int H3 = (NC / 2 + 1) * (NC / 2 + 1) * (NC / 2 + 1);
    unsigned em = 0;
    for (int t = threadIdx.x; t < 8 * H3; t += blockDim.x) {
        const int q = t / H3, i = t - q * H3;
        em = max(em, ((unsigned)__double2hiint(su[q * sp.H3p + i]) >> 20) & 0x7FFu);
    }
    em = __reduce_max_sync(0xffffffffu, em);
    if ((threadIdx.x & 31) == 0) atomicMax(emax, em);
    __syncthreads();
    const int E = (int)*emax;
    if (E < 128 || E > 1900) return -1;
    const int shb = 9 - G - E;
    for (int t = threadIdx.x; t < 8 * H3; t += blockDim.x) {
        const int q = t / H3, i = t - q * H3;
        double* a = su + q * sp.H3p + i;
        *a = __longlong_as_double(to_fixed(__double_as_longlong(*a), shb));
    }
    __syncthreads();
    return E;
}

template <int M, int I, int NC>
__global__ void __launch_bounds__(512) k_leafres_fused(float* __restrict__ R, const double* __restrict__ U,
                                                       const double* __restrict__ F, const double* __restrict__ Uc,
                                                       const int* __restrict__ blocks, LevelView lk, int n_arg,
                                                       double scale, unsigned long long* out) {
    const int n = NC ? NC : n_arg;
    extern __shared__ __align__(16) unsigned char fz_smem[];
    double* su = reinterpret_cast<double*>(fz_smem);
    const Split sp = split_of<double>(n);
    double* pool = su + 8 * sp.H3p;
    double* patch = pool + pool_size(n, I);
    __shared__ HaloSmem hs;
    __shared__ unsigned s_emax;       // largest exponent field in the box
    Cset cs;
    cset_init(cs, n >> 1);
    const int b = blocks[blockIdx.x];
    if (threadIdx.x == 0) s_emax = 0u;
    record_prologue_own(hs, lk, b, su, U, n, sp);
    build_halo<double, I, true, true>(su, pool, patch, hs.rec, U, Uc, lk, b, n, sp);
    const size_t n3 = (size_t)n * n * n;
    unsigned long long mb = 0;        // max |r| as a bit pattern
    if constexpr (NC != 0) {
        // Fixed block size: one thread per interior (y, z) row walking x.
        // Per box plane X it forms the centre value u, the sum c of the 4
        // face-adjacent (y, z) neighbours and the sum d of the 4 diagonal
        // ones; a node's faces are u(X-1) + u(X+1) + c(X), its edges c(X-1) +
        // c(X+1) + d(X), its corners d(X-1) + d(X+1).  So with the plane's
        // weighted sums P = w_f u + w_e c + w_k d (what a neighbouring plane
        // contributes) and Q = w_c u + w_f c + w_e d (what the node's own plane
        // contributes), L u(X) = P(X-1) + P(X+1) + Q(X): each plane's sums are
        // formed once for three nodes.
        //
        // L u in 64-bit fixed point.  Every box value becomes the integer
        // trunc(u 2^s), with s set by the box's largest exponent field E so
        // that |u 2^s| < 2^(62 - G) and the stencil's weights (integers whose
        // absolute values sum to at most 2^G) cannot overflow; the stencil sum
        // is then exact, rounded once to double and scaled by 2^-s.  A value
        // loses only bits below 2^(E - 1084 + G) (2^-55 of the box's largest
        // magnitude for G = 6), less than the rounding of a double stencil
        // sum, and the integer sums cost a fraction of the FP64 operations
        // they replace.  Boxes with Inf or NaN, only zeros, or extreme
        // exponents take the FP64 sums below.
        constexpr int G = M == 6 ? 8 : 6;
        const int E = box_to_fixed<NC, G>(su, sp, &s_emax);
        if (E >= 0) {
            const double scale2 = scale * __longlong_as_double((long long)(E + G - 1084 + 1023) << 52);
            constexpr long long wc = (long long)LW<M>::c, wf = (long long)LW<M>::f, we = (long long)LW<M>::e,
                                wk = (long long)LW<M>::k;
            constexpr int nn = NC;
            const int H = sp.H, Hp = sp.H2, H3p = sp.H3p;
            for (int r = threadIdx.x; r < nn * nn; r += blockDim.x) {
                const int z = r / nn, y = r - z * nn;
                const int Y = y + 1, Z = z + 1;
                auto rowb = [&](int dy, int dz) {
                    const int YY = Y + dy, ZZ = Z + dz;
                    return (((ZZ & 1) << 2) | ((YY & 1) << 1)) * H3p + (ZZ >> 1) * Hp + (YY >> 1) * H;
                };
                const int r00 = rowb(0, 0), rm0 = rowb(-1, 0), rp0 = rowb(1, 0), r0m = rowb(0, -1), r0p = rowb(0, 1);
                const int rmm = rowb(-1, -1), rpm = rowb(1, -1), rmp = rowb(-1, 1), rpp = rowb(1, 1);
                auto ld = [&](int i) { return __double_as_longlong(su[i]); };
                auto plane = [&](int X, long long& P, long long& Q) {
                    const int o = (X & 1) * H3p + (X >> 1);
                    const long long u = ld(r00 + o);
                    const long long c = (ld(rm0 + o) + ld(rp0 + o)) + (ld(r0m + o) + ld(r0p + o));
                    long long p = wf * u, q = wc * u + wf * c;
                    if (we != 0 || wk != 0) {
                        const long long d = (ld(rmm + o) + ld(rpm + o)) + (ld(rmp + o) + ld(rpp + o));
                        p += we * c + wk * d;
                        q += we * d;
                    }
                    P = p;
                    Q = q;
                };
                long long P0, P1, Q1, Qg;
                plane(0, P0, Qg);
                plane(1, P1, Q1);
                const size_t rowf = b * n3 + (size_t)r * nn;
#pragma unroll
                for (int X = 1; X <= nn; ++X) {
                    long long P2, Q2;
                    plane(X + 1, P2, Q2);
                    const double l = i64_to_double_rn((P0 + P2) + Q1);
                    const size_t fi = rowf + (X - 1);
                    const double res = fma(-scale2, l, F[fi]);
                    if (R) R[fi] = narrow_rn(res);
                    mb = umax64(mb, (unsigned long long)__double_as_longlong(res) & 0x7fffffffffffffffULL);
                    P0 = P1;
                    P1 = P2; Q1 = Q2;
                }
            }
            bmax_atomic(__longlong_as_double((long long)mb), out + (lk.prob ? lk.prob[b] : 0));
            return;
        }
        // The same plane sums in FP64.
        constexpr int nn = NC;
        const int H = sp.H, Hp = sp.H2, H3p = sp.H3p;
        for (int r = threadIdx.x; r < nn * nn; r += blockDim.x) {
            const int z = r / nn, y = r - z * nn;
            const int Y = y + 1, Z = z + 1;
            auto rowb = [&](int dy, int dz) {
                const int YY = Y + dy, ZZ = Z + dz;
                return (((ZZ & 1) << 2) | ((YY & 1) << 1)) * H3p + (ZZ >> 1) * Hp + (YY >> 1) * H;
            };
            const int r00 = rowb(0, 0), rm0 = rowb(-1, 0), rp0 = rowb(1, 0), r0m = rowb(0, -1), r0p = rowb(0, 1);
            const int rmm = rowb(-1, -1), rpm = rowb(1, -1), rmp = rowb(-1, 1), rpp = rowb(1, 1);
            auto plane = [&](int X, double& P, double& Q) {
                const int o = (X & 1) * H3p + (X >> 1);
                const double u = su[r00 + o];
                const double c = (su[rm0 + o] + su[rp0 + o]) + (su[r0m + o] + su[r0p + o]);
                const double d = (su[rmm + o] + su[rpm + o]) + (su[rmp + o] + su[rpp + o]);
                double p = LW<M>::f * u, q = LW<M>::c * u + LW<M>::f * c;
                if (LW<M>::e != 0) { p += LW<M>::e * c; q += LW<M>::e * d; }
                if (LW<M>::k != 0) p += LW<M>::k * d;
                P = p;
                Q = q;
            };
            double P0, P1, Q1, Qg;
            plane(0, P0, Qg);             // (the ghost plane's own-plane sum is not needed)
            plane(1, P1, Q1);
            const size_t rowf = b * n3 + (size_t)r * nn;
#pragma unroll
            for (int X = 1; X <= nn; ++X) {
                double P2, Q2;
                plane(X + 1, P2, Q2);
                const double l = (P0 + P2) + Q1;
                const size_t fi = rowf + (X - 1);
                const double res = F[fi] - scale * l;
                if (R) R[fi] = narrow_rn(res);
                // |res| as its bit pattern (sign cleared): ordered like the
                // value for non-negative doubles, NaN above +Inf
                mb = umax64(mb, (unsigned long long)__double_as_longlong(res) & 0x7fffffffffffffffULL);
                P0 = P1;
                P1 = P2; Q1 = Q2;
            }
        }
    } else {
        for (int col = 0; col < 8; ++col) {
            const Col c = colour(col, sp, n);
#pragma unroll
            for (int k = 0; k < KMAX; ++k)
                if (k < cs.cnt) {
                    const Node d = node_of(cs.q[k], sp, n);
                    const int b0 = c.cb + d.b0;
                    const double l =
                        LW<M>::c * su[b0 + c.dX + c.dY + c.dZ] + offc_s<M>(su, b0, c.dX, c.dY, c.dZ, sp.H, sp.H2);
                    const size_t fi = b * n3 + d.f + c.fo;
                    const double r = F[fi] - scale * l;
                    if (R) R[fi] = (float)r;
                    mb = umax64(mb, (unsigned long long)__double_as_longlong(r) & 0x7fffffffffffffffULL);
                }
        }
    }
    bmax_atomic(__longlong_as_double((long long)mb), out + (lk.prob ? lk.prob[b] : 0));
}

// ---------------------------------------------------------------- f* = R^M f (M = 2, 4), fused with its ghost layer
// Raw f of level k in the (n+2)^3 box layout (Af; the level-(k-1) array Ac
// holds f on covered nodes by injection): build_halo() builds the one ghost
// layer R^2 and R^4 read (same-level copies, I-point interpolation at
// resolution jumps, zero outside the domain from the stored ghost layer,
// which nothing writes), then f* = R^M f on the listed leaf blocks (Sec. 3.2;
// the arithmetic of k_rhs_star).
template <int M, int I, int NC>
__global__ void __launch_bounds__(512) k_rhs_fused(double* __restrict__ F, const double* __restrict__ Af,
                                                   const double* __restrict__ Ac, const int* __restrict__ blocks,
                                                   LevelView lk, int n_arg, unsigned long long* fmax_out) {
    static_assert(M == 2 || M == 4, "R^6 reads two ghost layers");
    const int n = NC ? NC : n_arg;
    extern __shared__ __align__(16) unsigned char fz_smem[];
    double* su = reinterpret_cast<double*>(fz_smem);
    const Split sp = split_of<double>(n);
    double* pool = su + 8 * sp.H3p;
    double* patch = pool + pool_size(n, I);
    __shared__ HaloSmem hs;
    __shared__ unsigned s_emax;       // largest exponent field in the box
    const int b = blocks[blockIdx.x];
    if (threadIdx.x == 0) s_emax = 0u;
    record_prologue_own(hs, lk, b, su, Af, n, sp);
    build_halo<double, I, true, true>(su, pool, patch, hs.rec, Af, Ac, lk, b, n, sp);
    double* out = F + (size_t)b * n * n * n;
    unsigned long long mb = 0;        // max |f*| as a bit pattern
    if constexpr (NC != 0) {
        // Fixed block size: one thread per interior (y, z) row walking x, the
        // row's x neighbours kept in registers.
        const int H = sp.H, Hp = sp.H2, H3p = sp.H3p;
        if constexpr (M == 4) {
            // f* = (6 f + the sum of the 6 face neighbours) / 12 with the sum
            // exact in 64-bit fixed point (weights 6 and 1: at most 2^4 in
            // all), rounded once to double and scaled by 2^-s / 12; boxes
            // box_to_fixed() turns down take the FP64 sums below.
            constexpr int G = 4;
            const int E = box_to_fixed<NC, G>(su, sp, &s_emax);
            if (E >= 0) {
                const double sc = (1.0 / 12.0) * __longlong_as_double((long long)(E + G - 1084 + 1023) << 52);
                for (int r = threadIdx.x; r < NC * NC; r += blockDim.x) {
                    const int z = r / NC, y = r - z * NC;
                    const int Y = y + 1, Z = z + 1;
                    auto rowb = [&](int dy, int dz) {
                        const int YY = Y + dy, ZZ = Z + dz;
                        return (((ZZ & 1) << 2) | ((YY & 1) << 1)) * H3p + (ZZ >> 1) * Hp + (YY >> 1) * H;
                    };
                    const int r00 = rowb(0, 0), rm0 = rowb(-1, 0), rp0 = rowb(1, 0), r0m = rowb(0, -1), r0p = rowb(0, 1);
                    auto at = [&](int rb, int X) { return __double_as_longlong(su[rb + (X & 1) * H3p + (X >> 1)]); };
                    long long um = at(r00, 0), uc = at(r00, 1);
                    double* orow = out + (size_t)r * NC;
#pragma unroll
                    for (int X = 1; X <= NC; ++X) {
                        const long long up = at(r00, X + 1);
                        const long long S = 6 * uc + (um + up) + (at(rm0, X) + at(rp0, X)) + (at(r0m, X) + at(r0p, X));
                        const double v = sc * i64_to_double_rn(S);
                        orow[X - 1] = v;
                        mb = umax64(mb, (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL);
                        um = uc;
                        uc = up;
                    }
                }
                bmax_atomic(__longlong_as_double((long long)mb), fmax_out + (lk.prob ? lk.prob[b] : 0));
                return;
            }
        }
        for (int r = threadIdx.x; r < NC * NC; r += blockDim.x) {
            const int z = r / NC, y = r - z * NC;
            const int Y = y + 1, Z = z + 1;
            auto rowb = [&](int dy, int dz) {
                const int YY = Y + dy, ZZ = Z + dz;
                return (((ZZ & 1) << 2) | ((YY & 1) << 1)) * H3p + (ZZ >> 1) * Hp + (YY >> 1) * H;
            };
            const int r00 = rowb(0, 0), rm0 = rowb(-1, 0), rp0 = rowb(1, 0), r0m = rowb(0, -1), r0p = rowb(0, 1);
            auto at = [&](int rb, int X) { return su[rb + (X & 1) * H3p + (X >> 1)]; };
            double um = at(r00, 0), uc = at(r00, 1);
            double* orow = out + (size_t)r * NC;
#pragma unroll
            for (int X = 1; X <= NC; ++X) {
                const double up = at(r00, X + 1);
                double v = uc;
                if (M == 4) {
                    const double sf = (um + up) + (at(rm0, X) + at(rp0, X)) + (at(r0m, X) + at(r0p, X));
                    v = 0.5 * uc + sf * (1.0 / 12.0);
                }
                orow[X - 1] = v;
                mb = umax64(mb, (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL);
                um = uc;
                uc = up;
            }
        }
        bmax_atomic(__longlong_as_double((long long)mb), fmax_out + (lk.prob ? lk.prob[b] : 0));
        return;
    }
    for (int t = threadIdx.x; t < n * n * n; t += blockDim.x) {
        const int x = t % n, y = (t / n) % n, z = t / (n * n);
        const int X = x + 1, Y = y + 1, Z = z + 1;
        double v = su[sp.at(X, Y, Z)];
        if (M == 4) {
            const double sf = (su[sp.at(X - 1, Y, Z)] + su[sp.at(X + 1, Y, Z)]) +
                              (su[sp.at(X, Y - 1, Z)] + su[sp.at(X, Y + 1, Z)]) +
                              (su[sp.at(X, Y, Z - 1)] + su[sp.at(X, Y, Z + 1)]);
            v = 0.5 * v + sf * (1.0 / 12.0);
        }
        out[t] = v;
        mb = umax64(mb, (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL);
    }
    // max |f*| over the leaves (the stop rule's scale), per problem
    bmax_atomic(__longlong_as_double((long long)mb), fmax_out + (lk.prob ? lk.prob[b] : 0));
}

// ---------------------------------------------------------------- halo dump (step API)
// Writes the ghost layer build_halo() produces into the block's stored ghost layer.
template <typename T, int I>
__global__ void __launch_bounds__(512) k_halo_dump(T* __restrict__ U, const T* __restrict__ Uc, LevelView lk, int n) {
    extern __shared__ __align__(16) unsigned char fz_smem[];
    T* su = reinterpret_cast<T*>(fz_smem);
    const Split sp = split_of<T>(n);
    T* pool = su + 8 * sp.H3p;
    T* patch = pool + pool_size(n, I);
    __shared__ HaloSmem hs;
    const int S = n + 2, S3 = S * S * S;
    const int b = blockIdx.x;
    record_prologue_own(hs, lk, b, su, U, n, sp);
    build_halo<T, I, true, sizeof(T) == 8>(su, pool, patch, hs.rec, U, Uc, lk, b, n, sp);
    for (int t = threadIdx.x; t < S3 - n * n * n; t += blockDim.x) {
        int x, y, z;
        shell_coords(t, S, x, y, z);
        U[(size_t)b * S3 + (z * S + y) * S + x] = su[sp.at(x, y, z)];
    }
}

// ---------------------------------------------------------------- launchers
template <typename K>
static void allow(K kern) { cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, MAX_DYN_SMEM); }

// ---------------------------------------------------------------- ghost fill, transposed (FP64)
// Exact transpose of the ghost layer build_halo() produces for block b
// (halo 1): the adjoints on b's ghost layer A[b] are sent back to their
// sources, then the ghost layer is cleared.  Copied regions add to the
// same-level neighbour's interior; interpolated regions run the two
// separable passes of build_halo() backwards in shared memory (tangential,
// then normal, with shared atomics) into the coarse patch, whose entries add
// to the coarse level's interior (leaf coarse blocks) or to the coincident
// node of the current level (covered coarse blocks, which the forward reads
// from the fine level); outside the domain the adjoint is dropped.  Global
// writes are atomic and land only on interiors, never on ghost layers, so
// blocks of one launch do not interfere.
template <typename T, int I>
__global__ void __launch_bounds__(256) k_ghost_T_fused(T* __restrict__ A, T* __restrict__ Ac, LevelView lk, LevelView lc,
                                                       int n) {
    extern __shared__ __align__(16) unsigned char fz_smem[];
    T* pool = reinterpret_cast<T*>(fz_smem);
    __shared__ HaloSmemT<T> hs;
    const int S = n + 2, S2 = S * S, S3 = S2 * S, n3 = n * n * n;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int b = blockIdx.x;
    if (tid < 27) hs.snbr[tid] = lk.nbr[27 * b + tid];
    if (tid < I) hs.sw[tid] = T(midw<I>(tid));
    __syncthreads();
    if (tid == 0) {
        int any = 0, out = 0;
        for (int d = 0; d < 27; ++d) {
            any |= (d != 13 && hs.snbr[d] == NBR_MISSING);
            out |= (d != 13 && hs.snbr[d] == NBR_OUTSIDE);
        }
        hs.interp = any;
        hs.outside = out;
    }
    T* Ab = A + (size_t)b * S3;
    const int shell = S3 - n3;
    // copied regions: K ghost nodes per thread and round, all loads issued
    // before the stores and atomics (which could alias them as far as the
    // compiler knows), so that their latencies overlap
    constexpr int K = 4;
    for (int t0 = tid; t0 < shell; t0 += K * nth) {
        T a[K];
        int o[K];
        long long to[K];                  // target index in A, or -1
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int t = t0 + k * nth;
            to[k] = -1;
            o[k] = 0;
            a[k] = T(0);
            if (t < shell) {
                int x, y, z;
                shell_coords(t, S, x, y, z);
                const int dx = x == 0 ? -1 : (x == S - 1 ? 1 : 0);
                const int dy = y == 0 ? -1 : (y == S - 1 ? 1 : 0);
                const int dz = z == 0 ? -1 : (z == S - 1 ? 1 : 0);
                const int j = hs.snbr[dir27(dx, dy, dz)];
                if (j >= 0) {
                    o[k] = (z * S + y) * S + x;
                    to[k] = (long long)j * S3 + ((z - dz * n) * S + (y - dy * n)) * S + (x - dx * n);
                    a[k] = Ab[o[k]];
                }
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (to[k] < 0) continue;
            Ab[o[k]] = T(0);
            if (a[k] != T(0)) atomicAdd(&A[to[k]], a[k]);
        }
    }
    __syncthreads();
    if (!hs.interp) {
        // outside-domain ghosts: dropped (the copied ones are clear already)
        if (hs.outside)
            for (int t = tid; t < shell; t += nth) {
                int x, y, z;
                shell_coords(t, S, x, y, z);
                Ab[(z * S + y) * S + x] = T(0);
            }
        return;
    }
    const int P = lk.parent[b];
    if (tid < 27) {
        const int cb = lc.nbr[27 * P + tid];
        hs.cnbr[tid] = cb;
        hs.cleaf[tid] = cb >= 0 ? (int)lc.is_leaf[cb] : 1;
        for (int o = 0; o < 8; ++o) hs.cch[8 * tid + o] = (cb >= 0 && !hs.cleaf[tid]) ? lc.children[8 * cb + o] : -1;
    }
    const int TN = tan_n(n, I), TN2 = TN * TN;
    if (tid == 0) {
        int o = 0, nr = 0;
        for (int d = 0; d < 27; ++d) {
            hs.off[d] = o;
            if (d == 13 || hs.snbr[d] != NBR_MISSING) continue;
            const int nt = (d % 3 == 1) + ((d / 3) % 3 == 1) + (d / 9 == 1);
            hs.rdir[nr] = d;
            hs.rstart[nr] = o;
            ++nr;
            o += nt == 2 ? TN2 : (nt == 1 ? TN : 1);
        }
        hs.nreg = nr;
        hs.ntot = o;
    }
    const int h = n >> 1;
    constexpr int plo = 4 - I / 2;
    const int PL = h + I, PL2 = PL * PL, PL3 = PL2 * PL;
    T* patch = pool + pool_size(n, I);
    for (int t = tid; t < pool_size(n, I) + PL3; t += nth) pool[t] = T(0);
    __syncthreads();
    // phase 2 transposed: each interpolated ghost node spreads over its region's reduced array
    for (int t = tid; t < shell; t += nth) {
        int x, y, z;
        shell_coords(t, S, x, y, z);
        const int dx = x == 0 ? -1 : (x == S - 1 ? 1 : 0);
        const int dy = y == 0 ? -1 : (y == S - 1 ? 1 : 0);
        const int dz = z == 0 ? -1 : (z == S - 1 ? 1 : 0);
        const int d = dir27(dx, dy, dz);
        const int o = (z * S + y) * S + x;
        if (hs.snbr[d] != NBR_MISSING) {
            if (hs.snbr[d] == NBR_OUTSIDE) Ab[o] = T(0);
            continue;
        }
        const T a = Ab[o];
        Ab[o] = T(0);
        if (a == T(0)) continue;
        T* R = pool + hs.off[d];
        int st0 = 0, st1 = 0, cn0 = 1, cn1 = 1, sd0 = 0, sd1 = 0, nt = 0, stride = 1;
        const int q[3] = {x - 1, y - 1, z - 1};
        const int dd[3] = {dx, dy, dz};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            if (dd[ax] != 0) continue;
            const int qa = q[ax];
            const int st = (qa & 1) ? 4 + ((qa - 1) >> 1) - I / 2 + 1 - tan_lo<I>() : 4 + (qa >> 1) - tan_lo<I>();
            const int cn = (qa & 1) ? I : 1;
            if (nt == 0) { st0 = st; cn0 = cn; sd0 = stride; }
            else { st1 = st; cn1 = cn; sd1 = stride; }
            stride *= TN;
            ++nt;
        }
        for (int m1 = 0; m1 < cn1; ++m1) {
            const T a1 = (cn1 == 1 ? T(1) : hs.sw[m1]) * a;
            const int rb = (st1 + m1) * sd1 + st0 * sd0;
            for (int m0 = 0; m0 < cn0; ++m0) atomicAdd(&R[rb + m0 * sd0], (cn0 == 1 ? T(1) : hs.sw[m0]) * a1);
        }
    }
    __syncthreads();
    // phase 1 transposed: each reduced element spreads along its region's normal axes into the patch
    const int lo = 0, up = 4 + h - plo, tlo = tan_lo<I>() - plo;
    for (int f = tid; f < hs.ntot; f += nth) {
        int r = 0;
        while (r + 1 < hs.nreg && hs.rstart[r + 1] <= f) ++r;
        const int d = hs.rdir[r];
        const int e = f - hs.rstart[r];
        const T a = pool[f];
        if (a == T(0)) continue;
        const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        int tc[3] = {0, 0, 0};
        int rem = e;
        if (dx == 0) { tc[0] = tlo + rem % TN; rem /= TN; }
        if (dy == 0) { tc[1] = tlo + rem % TN; rem /= TN; }
        if (dz == 0) { tc[2] = tlo + rem % TN; }
        const int cx = dx < 0 ? I : 1, cy = dy < 0 ? I : 1, cz = dz < 0 ? I : 1;
        const int x0 = dx < 0 ? lo : (dx > 0 ? up : tc[0]);
        const int y0 = dy < 0 ? lo : (dy > 0 ? up : tc[1]);
        const int z0 = dz < 0 ? lo : (dz > 0 ? up : tc[2]);
        for (int mz = 0; mz < cz; ++mz) {
            const T az = (cz == 1 ? T(1) : hs.sw[mz]) * a;
            for (int my = 0; my < cy; ++my) {
                const T ay = (cy == 1 ? T(1) : hs.sw[my]) * az;
                T* row = patch + ((z0 + mz) * PL + y0 + my) * PL + x0;
                for (int mx = 0; mx < cx; ++mx) atomicAdd(&row[mx], (cx == 1 ? T(1) : hs.sw[mx]) * ay);
            }
        }
    }
    __syncthreads();
    // the patch back to its sources
    const int bx = lk.coords[3 * b], by = lk.coords[3 * b + 1], bz = lk.coords[3 * b + 2];
    const int base[3] = {(bx & 1) * h - 4 + plo, (by & 1) * h - 4 + plo, (bz & 1) * h - 4 + plo};
    for (int t = tid; t < PL3; t += nth) {
        const T a = patch[t];
        if (a == T(0)) continue;
        const int px = t % PL, py = (t / PL) % PL, pz = t / PL2;
        const int rx = base[0] + px, ry = base[1] + py, rz = base[2] + pz;
        const int ex = rx < 0 ? -1 : (rx >= n ? 1 : 0);
        const int ey = ry < 0 ? -1 : (ry >= n ? 1 : 0);
        const int ez = rz < 0 ? -1 : (rz >= n ? 1 : 0);
        const int d = dir27(ex, ey, ez);
        const int lx = rx - ex * n, ly = ry - ey * n, lz = rz - ez * n;
        if (hs.cleaf[d]) {
            if (hs.cnbr[d] >= 0) atomicAdd(&Ac[(size_t)hs.cnbr[d] * S3 + ((lz + 1) * S + ly + 1) * S + lx + 1], a);
        } else {
            const int ox = lx >= h, oy = ly >= h, oz = lz >= h;
            const int ch = hs.cch[8 * d + ox + 2 * oy + 4 * oz];
            const int FX = 2 * lx - ox * n + 1, FY = 2 * ly - oy * n + 1, FZ = 2 * lz - oz * n + 1;
            atomicAdd(&A[(size_t)ch * S3 + (FZ * S + FY) * S + FX], a);
        }
    }
}

template <typename T>
void launch_ghost_T_fused(T* A, T* Ac, LevelView lk, LevelView lc, int n, int M, cudaStream_t s) {
    if (lk.nb == 0) return;
    const int I = M + 2, PL = n / 2 + I;
    const size_t sm = sizeof(T) * ((size_t)pool_size(n, I) + (size_t)PL * PL * PL);
    static std::once_flag attr[MAX_DEVICES];
    once_per_device(attr, [] {
        allow(k_ghost_T_fused<T, 4>); allow(k_ghost_T_fused<T, 6>); allow(k_ghost_T_fused<T, 8>);
    });
    if (M == 2) k_ghost_T_fused<T, 4><<<lk.nb, 256, sm, s>>>(A, Ac, lk, lc, n);
    if (M == 4) k_ghost_T_fused<T, 6><<<lk.nb, 256, sm, s>>>(A, Ac, lk, lc, n);
    if (M == 6) k_ghost_T_fused<T, 8><<<lk.nb, 256, sm, s>>>(A, Ac, lk, lc, n);
}

// CTA size actually launched: the requested one, raised (in warps) until each
// thread holds at most KMAX nodes of a colour.
inline int cta_size(int n, int nt) {
    const int h3 = (n / 2) * (n / 2) * (n / 2);
    while (nt < 512 && nt * KMAX < h3) nt += 32;
    return nt;
}
// Kernels whose fixed-size build has 256 work items per phase (FP32 node
// pairs, FP64 leaf-residual rows) take at most 256 threads: more would idle.
inline int cta_size_fixed(int n, int nt, bool fixed_items) {
    const int c = cta_size(n, nt);
    return (fixed_items && n == 16 && c > 256) ? 256 : c;
}

// Per-family shared-memory attributes, set once per device (each family's
// instantiations live in one translation unit).
template <typename T>
static void attrs_smooth() {
    static std::once_flag done[MAX_DEVICES];
    once_per_device(done, [] {
        allow(k_smooth_fused<2, T, 4, NC_FIXED>); allow(k_smooth_fused<2, T, 4, 0>);
        allow(k_smooth_fused<4, T, 6, NC_FIXED>); allow(k_smooth_fused<4, T, 6, 0>);
        allow(k_smooth_fused<6, T, 8, NC_FIXED>); allow(k_smooth_fused<6, T, 8, 0>);
    });
}
template <typename T>
static void attrs_residual() {
    static std::once_flag done[MAX_DEVICES];
    once_per_device(done, [] {
        allow(k_residual_fused<2, T, 4, NC_FIXED>); allow(k_residual_fused<2, T, 4, 0>);
        allow(k_residual_fused<4, T, 6, NC_FIXED>); allow(k_residual_fused<4, T, 6, 0>);
        allow(k_residual_fused<6, T, 8, NC_FIXED>); allow(k_residual_fused<6, T, 8, 0>);
    });
}
template <typename T>
static void attrs_fas() {
    static std::once_flag done[MAX_DEVICES];
    once_per_device(done, [] {
        allow(k_fas_fused<2, T, 4, NC_FIXED>); allow(k_fas_fused<2, T, 4, 0>);
        allow(k_fas_fused<4, T, 6, NC_FIXED>); allow(k_fas_fused<4, T, 6, 0>);
        allow(k_fas_fused<6, T, 8, NC_FIXED>); allow(k_fas_fused<6, T, 8, 0>);
    });
}
inline void attrs_leafres() {
    static std::once_flag done[MAX_DEVICES];
    once_per_device(done, [] {
        allow(k_leafres_fused<2, 4, NC_FIXED>); allow(k_leafres_fused<2, 4, 0>);
        allow(k_leafres_fused<4, 6, NC_FIXED>); allow(k_leafres_fused<4, 6, 0>);
        allow(k_leafres_fused<6, 8, NC_FIXED>); allow(k_leafres_fused<6, 8, 0>);
    });
}
template <typename T>
static void attrs_halo_dump() {
    static std::once_flag done[MAX_DEVICES];
    once_per_device(done, [] {
        allow(k_halo_dump<T, 4>); allow(k_halo_dump<T, 6>); allow(k_halo_dump<T, 8>);
    });
}

template <int M, typename T>
static void smooth_m(T* Uout, const T* Uin, const T* F, const T* Uc, const LevelView& lk, int nblocks, int n, T h2den,
                     int fst, int ct, size_t sm, cudaStream_t s) {
    constexpr int I = M + 2;
    if (nblocks == 0) return;
    if (n == NC_FIXED) k_smooth_fused<M, T, I, NC_FIXED><<<nblocks, ct, sm, s>>>(Uout, Uin, F, Uc, lk, n, h2den, lk.order, fst);
    else k_smooth_fused<M, T, I, 0><<<nblocks, ct, sm, s>>>(Uout, Uin, F, Uc, lk, n, h2den, lk.order, fst);
}
template <int M, typename T>
static void residual_m(T* R, const T* U, const T* F, const T* Uc, const LevelView& lk, int n, T scale, int ct, size_t sm,
                       int stage, cudaStream_t s) {
    constexpr int I = M + 2;
    if (n == NC_FIXED) k_residual_fused<M, T, I, NC_FIXED><<<lk.nb, ct, sm, s>>>(R, U, F, Uc, lk, n, scale, lk.order, stage);
    else k_residual_fused<M, T, I, 0><<<lk.nb, ct, sm, s>>>(R, U, F, Uc, lk, n, scale, lk.order, stage);
}
template <int M, typename T>
static void fas_m(T* F, T* H, const T* U, const T* Uc, const LevelView& lk, int n, T scale, int ct, size_t sm,
                  cudaStream_t s) {
    constexpr int I = M + 2;
    if (n == NC_FIXED) k_fas_fused<M, T, I, NC_FIXED><<<lk.nb, ct, sm, s>>>(F, H, U, Uc, lk, n, scale, lk.order);
    else k_fas_fused<M, T, I, 0><<<lk.nb, ct, sm, s>>>(F, H, U, Uc, lk, n, scale, lk.order);
}
template <int M>
static void leafres_m(float* R, const double* U, const double* F, const double* Uc, const int* blocks, int nblocks,
                      const LevelView& lk, int n, double scale, unsigned long long* out, int ct, size_t sm,
                      cudaStream_t s) {
    constexpr int I = M + 2;
    if (n == NC_FIXED) k_leafres_fused<M, I, NC_FIXED><<<nblocks, ct, sm, s>>>(R, U, F, Uc, blocks, lk, n, scale, out);
    else k_leafres_fused<M, I, 0><<<nblocks, ct, sm, s>>>(R, U, F, Uc, blocks, lk, n, scale, out);
}

template <typename T>
void launch_smooth_fused(T* Uout, const T* Uin, const T* F, const T* Uc, LevelView lk, LevelView lc, int n, int M,
                         double h2, int nt, cudaStream_t s) {
    if (lk.nb == 0) return;
    attrs_smooth<T>();
    // The block's right-hand side goes to shared memory where it fits: in its
    // own area when the launch fits in one wave at the CTAs per SM that this
    // leaves, else over the interpolation scratch.
    int nsm = 1, dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm < 1)
        nsm = 1;
    int fmode = 0;
    if (!(nt & SMOOTH_NOSTAGE)) {
        if (fused_smem<T>(n, M + 2, 1) <= (size_t)MAX_DYN_SMEM) fmode = 1;
        const size_t s2 = fused_smem<T>(n, M + 2, 2);
        const size_t per_sm = 228 * 1024, per_cta = s2 + sizeof(HaloSmem) + 1024;
        if (s2 <= (size_t)MAX_DYN_SMEM && (size_t)lk.nb <= (size_t)nsm * (per_sm / per_cta)) fmode = 2;
    }
    const int fst = fmode;
    const size_t sm = fused_smem<T>(n, M + 2, fmode);
    const int ct = cta_size_fixed(n, nt & SMOOTH_NT_MASK, sizeof(T) == 4);
    if (M == 2) smooth_m<2, T>(Uout, Uin, F, Uc, lk, lk.nb, n, T(h2 * LW<2>::den), fst, ct, sm, s);
    if (M == 4) smooth_m<4, T>(Uout, Uin, F, Uc, lk, lk.nb, n, T(h2 * LW<4>::den), fst, ct, sm, s);
    if (M == 6) smooth_m<6, T>(Uout, Uin, F, Uc, lk, lk.nb, n, T(h2 * LW<6>::den), fst, ct, sm, s);
}

template <typename T>
void launch_residual_fused(T* R, const T* U, const T* F, const T* Uc, LevelView lk, LevelView lc, int n, int M,
                           double inv_h2, int nt, cudaStream_t s) {
    if (lk.nb == 0) return;
    attrs_residual<T>();
    // FP32 block size 16 stages F over the interpolation scratch (fmode-1
    // sizing), unless the CTA choice carries SMOOTH_NOSTAGE (F read and R
    // written in global memory by the pairs)
    const int stage = (sizeof(T) == 4 && n == NC_FIXED && !(nt & SMOOTH_NOSTAGE)) ? 1 : 0;
    const size_t sm = fused_smem<T>(n, M + 2, stage);
    const int ct = cta_size_fixed(n, nt & SMOOTH_NT_MASK, sizeof(T) == 4);
    if (M == 2) residual_m<2, T>(R, U, F, Uc, lk, n, T(inv_h2 / LW<2>::den), ct, sm, stage, s);
    if (M == 4) residual_m<4, T>(R, U, F, Uc, lk, n, T(inv_h2 / LW<4>::den), ct, sm, stage, s);
    if (M == 6) residual_m<6, T>(R, U, F, Uc, lk, n, T(inv_h2 / LW<6>::den), ct, sm, stage, s);
}

template <typename T>
void launch_fas_fused(T* F, T* H, const T* U, const T* Uc, LevelView lk, LevelView lc, int n, int M, double inv_h2,
                      int nt, cudaStream_t s) {
    if (lk.nb == 0) return;
    attrs_fas<T>();
    // FP32 block size 16 stages F over the interpolation scratch (fmode-1 sizing)
    const size_t sm = fused_smem<T>(n, M + 2, (sizeof(T) == 4 && n == NC_FIXED) ? 1 : 0);
    const int ct = cta_size_fixed(n, nt, sizeof(T) == 4);
    if (M == 2) fas_m<2, T>(F, H, U, Uc, lk, n, T(inv_h2 / LW<2>::den), ct, sm, s);
    if (M == 4) fas_m<4, T>(F, H, U, Uc, lk, n, T(inv_h2 / LW<4>::den), ct, sm, s);
    if (M == 6) fas_m<6, T>(F, H, U, Uc, lk, n, T(inv_h2 / LW<6>::den), ct, sm, s);
}


template <int M>
static void rhs_fused_m(double* F, const double* Af, const double* Ac, const int* blocks, int nblocks, const LevelView& lk,
                        int n, unsigned long long* fmax_out, size_t sm, cudaStream_t s) {
    constexpr int I = M + 2;
    if (n == NC_FIXED) k_rhs_fused<M, I, NC_FIXED><<<nblocks, 256, sm, s>>>(F, Af, Ac, blocks, lk, n, fmax_out);
    else k_rhs_fused<M, I, 0><<<nblocks, 256, sm, s>>>(F, Af, Ac, blocks, lk, n, fmax_out);
}

template <typename T>
void launch_halo_dump(T* U, const T* Uc, LevelView lk, LevelView lc, int n, int M, cudaStream_t s) {
    if (lk.nb == 0) return;
    attrs_halo_dump<T>();
    const size_t sm = fused_smem<T>(n, M + 2);
    if (M == 2) k_halo_dump<T, 4><<<lk.nb, 256, sm, s>>>(U, Uc, lk, n);
    if (M == 4) k_halo_dump<T, 6><<<lk.nb, 256, sm, s>>>(U, Uc, lk, n);
    if (M == 6) k_halo_dump<T, 8><<<lk.nb, 256, sm, s>>>(U, Uc, lk, n);
}

}  // namespace mrp
