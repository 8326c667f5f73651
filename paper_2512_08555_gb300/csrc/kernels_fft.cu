// Level-0 direct solve: zero-padded FFT convolution with the lattice Green's
// function of the multigrid operator (arXiv 2512.08555, Sec. 2.2 and 3.3),
// and the FP64 tabulation of that Green's function.
//
// Padded lattice: P_a >= 2 N0_a + 1 per axis (a 2,3,5,7-smooth length), so
// the circular convolution equals the linear one on the target cube
// [-1, N0]^3 (level-0 nodes plus a one-node exterior ring).
//
// Spectral buffer layout: spec[z][y][kx], kx in [0, Px/2], complex FP64.
// Passes (each a batch of 1-D mixed-radix Stockham FFTs in shared memory):
//   A  x: real -> half spectrum, lines (y, z) < N0 only (the rest is zero padding)
//   B  y: forward, lines z < N0 only; input y < N0 only
//   C  z: forward, times G-hat, inverse; input z < N0, output z targets only
//   B' y: inverse on target z planes, output y targets only
//   A' x: half spectrum -> real on target (y, z) lines, written into the
//         level-0 blocks' interiors and ghost layers.
#include "mrp_internal.h"

#include <cmath>
#include <vector>

namespace mrp {

// Complex type of each real type.
template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

// One line length with its radix sequence.  Per stage st: ns[st] = product of
// the earlier radices, nsm[st] = floor(2^32 / ns) + 1 (so that j / ns =
// umulhi(j, nsm) for j, ns < 2^16; ns = 1 is handled apart), tstep[st] =
// P / (ns * rad) (the twiddle stride of one butterfly index).
template <typename R>
struct FftLine {
    int P, nrad;
    int rad[MAX_RADIX_STAGES];
    int ns[MAX_RADIX_STAGES], tstep[MAX_RADIX_STAGES];
    unsigned nsm[MAX_RADIX_STAGES];
    const typename Cx<R>::T* tw;
};

// The descriptor a CTA works with: twiddles and the stage table in shared
// memory (st[0..S) radices, st[S..2S) Ns, st[2S..3S) twiddle strides,
// st[3S..4S) Ns reciprocals, S = MAX_RADIX_STAGES), read there by index.
template <typename R>
struct FftDev {
    int P, nrad;
    const int* st;
    const typename Cx<R>::T* tw;
};
constexpr int FFT_STAGE_BYTES = 4 * MAX_RADIX_STAGES * 4;

template <typename R>
static FftLine<R> line_of(const FftAxis& a) {
    FftLine<R> l{};
    const int* rad = sizeof(R) == 8 ? a.rad : a.rad32;
    l.P = a.P;
    l.nrad = sizeof(R) == 8 ? a.nrad : a.nrad32;
    int ns = 1;
    for (int i = 0; i < l.nrad; ++i) {
        l.rad[i] = rad[i];
        l.ns[i] = ns;
        l.nsm[i] = ns > 1 ? (unsigned)((1ULL << 32) / (unsigned long long)ns + 1ULL) : 0u;
        l.tstep[i] = a.P / (ns * rad[i]);
        ns *= rad[i];
    }
    if constexpr (sizeof(R) == 8) l.tw = a.tw;
    else l.tw = a.tw32;
    return l;
}

template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) { return C{a.x * s, a.y * s}; }
// i * s * a
template <typename C, typename R> __device__ __forceinline__ C cmuli(C a, R s) { return C{-a.y * s, a.x * s}; }

// exp(sign * 2 pi i m / P) from the table exp(-2 pi i m / P).
template <typename C> __device__ __forceinline__ C twiddle(const C* tw, int m, int sign) {
    C w = tw[m];
    if (sign > 0) w.y = -w.y;
    return w;
}

// Small DFTs X_k = sum_j v_j w^(sign j k), w = exp(2 pi i / R), in registers.
template <int RAD, typename R> struct Dft;
template <typename R> struct Dft<2, R> {
    template <typename C> static __device__ __forceinline__ void run(C* v, int) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};
template <typename R> struct Dft<3, R> {
    template <typename C> static __device__ __forceinline__ void run(C* v, int sign) {
        const R c = R(-0.5), sn = R(0.86602540378443864676);   // cos, sin of 2 pi / 3
        const C a = cadd(v[1], v[2]), b = csub(v[1], v[2]);
        const C m = cadd(v[0], cscale(a, c));
        const C t = cmuli(b, R(sign) * sn);
        v[0] = cadd(v[0], a);
        v[1] = cadd(m, t);
        v[2] = csub(m, t);
    }
};
template <typename R> struct Dft<4, R> {
    template <typename C> static __device__ __forceinline__ void run(C* v, int sign) {
        const C a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
        const C c = cadd(v[1], v[3]), d = cmuli(csub(v[1], v[3]), R(sign));
        v[0] = cadd(a, c);
        v[2] = csub(a, c);
        v[1] = cadd(b, d);
        v[3] = csub(b, d);
    }
};
template <typename R> struct Dft<5, R> {
    template <typename C> static __device__ __forceinline__ void run(C* v, int sign) {
        const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);   // cos(2pi/5), cos(4pi/5)
        const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);    // sin(2pi/5), sin(4pi/5)
        const C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        const C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        const C m1 = cadd(v[0], cadd(cscale(a1, c1), cscale(a2, c2)));
        const C m2 = cadd(v[0], cadd(cscale(a1, c2), cscale(a2, c1)));
        const C t1 = cmuli(cadd(cscale(b1, s1), cscale(b2, s2)), R(sign));
        const C t2 = cmuli(csub(cscale(b1, s2), cscale(b2, s1)), R(sign));
        v[0] = cadd(v[0], cadd(a1, a2));
        v[1] = cadd(m1, t1);
        v[4] = csub(m1, t1);
        v[2] = cadd(m2, t2);
        v[3] = csub(m2, t2);
    }
};

template <typename R> struct Dft<7, R> {
    // symmetric pairs (j, 7 - j): a_j = v_j + v_{7-j}, b_j = v_j - v_{7-j};
    // X_k = v_0 + sum_j a_j cos(2 pi j k / 7) + i sign sum_j b_j sin(2 pi j k / 7)
    template <typename C> static __device__ __forceinline__ void run(C* v, int sign) {
        const R c1 = R(0.62348980185873353053), c2 = R(-0.22252093395631440429), c3 = R(-0.90096886790241912624);
        const R s1 = R(0.78183148246802980871), s2 = R(0.97492791218182360702), s3 = R(0.43388373911755812048);
        const C a1 = cadd(v[1], v[6]), b1 = csub(v[1], v[6]);
        const C a2 = cadd(v[2], v[5]), b2 = csub(v[2], v[5]);
        const C a3 = cadd(v[3], v[4]), b3 = csub(v[3], v[4]);
        const C m1 = cadd(v[0], cadd(cadd(cscale(a1, c1), cscale(a2, c2)), cscale(a3, c3)));
        const C m2 = cadd(v[0], cadd(cadd(cscale(a1, c2), cscale(a2, c3)), cscale(a3, c1)));
        const C m3 = cadd(v[0], cadd(cadd(cscale(a1, c3), cscale(a2, c1)), cscale(a3, c2)));
        const C t1 = cmuli(cadd(cadd(cscale(b1, s1), cscale(b2, s2)), cscale(b3, s3)), R(sign));
        const C t2 = cmuli(csub(csub(cscale(b1, s2), cscale(b2, s3)), cscale(b3, s1)), R(sign));
        const C t3 = cmuli(cadd(csub(cscale(b1, s3), cscale(b2, s1)), cscale(b3, s2)), R(sign));
        v[0] = cadd(v[0], cadd(cadd(a1, a2), a3));
        v[1] = cadd(m1, t1);
        v[6] = csub(m1, t1);
        v[2] = cadd(m2, t2);
        v[5] = csub(m2, t2);
        v[3] = cadd(m3, t3);
        v[4] = csub(m3, t3);
    }
};

// Composite R = A B points in registers (Cooley-Tukey inside one butterfly):
// with j = j1 + A j2 and k = k2 + B k1,
//   X[k2 + B k1] = sum_j1 w_A^(j1 k1) w_R^(j1 k2) sum_j2 w_B^(j2 k2) v[j1 + A j2],
// w_n = exp(sign 2 pi i / n).  One shared-memory round trip of a Stockham
// stage then does the work of two.  unit_root<R>(m) = (cos, sin)(2 pi m / R);
// the loops are unrolled, so every m is a constant.
template <int RR> __device__ __forceinline__ double2 unit_root(int m);
template <> __device__ __forceinline__ double2 unit_root<8>(int m) {
    switch (m) {
        case 0: return double2{1.0, 0.0};
        case 1: return double2{0.707106781186547524401, 0.707106781186547524401};
        case 2: return double2{0.0, 1.0};
        case 3: return double2{-0.707106781186547524401, 0.707106781186547524401};
        case 4: return double2{-1.0, 0.0};
        case 5: return double2{-0.707106781186547524401, -0.707106781186547524401};
        case 6: return double2{0.0, -1.0};
        case 7: return double2{0.707106781186547524401, -0.707106781186547524401};
        default: return double2{1.0, 0.0};
    }
}
template <> __device__ __forceinline__ double2 unit_root<9>(int m) {
    switch (m) {
        case 0: return double2{1.0, 0.0};
        case 1: return double2{0.766044443118978035202, 0.642787609686539326323};
        case 2: return double2{0.173648177666930348852, 0.984807753012208059367};
        case 3: return double2{-0.5, 0.866025403784438646764};
        case 4: return double2{-0.939692620785908384054, 0.342020143325668733044};
        case 5: return double2{-0.939692620785908384054, -0.342020143325668733044};
        case 6: return double2{-0.5, -0.866025403784438646764};
        case 7: return double2{0.173648177666930348852, -0.984807753012208059367};
        case 8: return double2{0.766044443118978035202, -0.642787609686539326323};
        default: return double2{1.0, 0.0};
    }
}
template <> __device__ __forceinline__ double2 unit_root<14>(int m) {
    switch (m) {
        case 0: return double2{1.0, 0.0};
        case 1: return double2{0.900968867902419126236, 0.433883739117558120476};
        case 2: return double2{0.623489801858733530525, 0.781831482468029808708};
        case 3: return double2{0.222520933956314404289, 0.974927912181823607018};
        case 4: return double2{-0.222520933956314404289, 0.974927912181823607018};
        case 5: return double2{-0.623489801858733530525, 0.781831482468029808708};
        case 6: return double2{-0.900968867902419126236, 0.433883739117558120476};
        case 7: return double2{-1.0, 0.0};
        case 8: return double2{-0.900968867902419126236, -0.433883739117558120476};
        case 9: return double2{-0.623489801858733530525, -0.781831482468029808708};
        case 10: return double2{-0.222520933956314404289, -0.974927912181823607018};
        case 11: return double2{0.222520933956314404289, -0.974927912181823607018};
        case 12: return double2{0.623489801858733530525, -0.781831482468029808708};
        case 13: return double2{0.900968867902419126236, -0.433883739117558120476};
        default: return double2{1.0, 0.0};
    }
}
template <> __device__ __forceinline__ double2 unit_root<15>(int m) {
    switch (m) {
        case 0: return double2{1.0, 0.0};
        case 1: return double2{0.913545457642600895502, 0.406736643075800207754};
        case 2: return double2{0.669130606358858213826, 0.743144825477394235015};
        case 3: return double2{0.309016994374947424102, 0.951056516295153572116};
        case 4: return double2{-0.1045284632676534714, 0.994521895368273336923};
        case 5: return double2{-0.5, 0.866025403784438646764};
        case 6: return double2{-0.809016994374947424102, 0.587785252292473129169};
        case 7: return double2{-0.978147600733805637929, 0.207911690817759337102};
        case 8: return double2{-0.978147600733805637929, -0.207911690817759337102};
        case 9: return double2{-0.809016994374947424102, -0.587785252292473129169};
        case 10: return double2{-0.5, -0.866025403784438646764};
        case 11: return double2{-0.1045284632676534714, -0.994521895368273336923};
        case 12: return double2{0.309016994374947424102, -0.951056516295153572116};
        case 13: return double2{0.669130606358858213826, -0.743144825477394235015};
        case 14: return double2{0.913545457642600895502, -0.406736643075800207754};
        default: return double2{1.0, 0.0};
    }
}
template <> __device__ __forceinline__ double2 unit_root<16>(int m) {
    switch (m) {
        case 0: return double2{1.0, 0.0};
        case 1: return double2{0.923879532511286756128, 0.382683432365089771728};
        case 2: return double2{0.707106781186547524401, 0.707106781186547524401};
        case 3: return double2{0.382683432365089771728, 0.923879532511286756128};
        case 4: return double2{0.0, 1.0};
        case 5: return double2{-0.382683432365089771728, 0.923879532511286756128};
        case 6: return double2{-0.707106781186547524401, 0.707106781186547524401};
        case 7: return double2{-0.923879532511286756128, 0.382683432365089771728};
        case 8: return double2{-1.0, 0.0};
        case 9: return double2{-0.923879532511286756128, -0.382683432365089771728};
        case 10: return double2{-0.707106781186547524401, -0.707106781186547524401};
        case 11: return double2{-0.382683432365089771728, -0.923879532511286756128};
        case 12: return double2{0.0, -1.0};
        case 13: return double2{0.382683432365089771728, -0.923879532511286756128};
        case 14: return double2{0.707106781186547524401, -0.707106781186547524401};
        case 15: return double2{0.923879532511286756128, -0.382683432365089771728};
        default: return double2{1.0, 0.0};
    }
}

template <> __device__ __forceinline__ double2 unit_root<18>(int m) {
    switch (m) {
        case 0: return double2{1.0, 0.0};
        case 1: return double2{0.939692620785908384054, 0.342020143325668733044};
        case 2: return double2{0.766044443118978035202, 0.642787609686539326323};
        case 3: return double2{0.5, 0.866025403784438646764};
        case 4: return double2{0.173648177666930348852, 0.984807753012208059367};
        case 5: return double2{-0.173648177666930348852, 0.984807753012208059367};
        case 6: return double2{-0.5, 0.866025403784438646764};
        case 7: return double2{-0.766044443118978035202, 0.642787609686539326323};
        case 8: return double2{-0.939692620785908384054, 0.342020143325668733044};
        case 9: return double2{-1.0, 0.0};
        case 10: return double2{-0.939692620785908384054, -0.342020143325668733044};
        case 11: return double2{-0.766044443118978035202, -0.642787609686539326323};
        case 12: return double2{-0.5, -0.866025403784438646764};
        case 13: return double2{-0.173648177666930348852, -0.984807753012208059367};
        case 14: return double2{0.173648177666930348852, -0.984807753012208059367};
        case 15: return double2{0.5, -0.866025403784438646764};
        case 16: return double2{0.766044443118978035202, -0.642787609686539326323};
        case 17: return double2{0.939692620785908384054, -0.342020143325668733044};
        default: return double2{1.0, 0.0};
    }
}
template <> __device__ __forceinline__ double2 unit_root<27>(int m) {
    switch (m) {
        case 0: return double2{1.0, 0.0};
        case 1: return double2{0.973044870579823838833, 0.23061587074244017845};
        case 2: return double2{0.893632640323412248193, 0.448799180200462172785};
        case 3: return double2{0.766044443118978035202, 0.642787609686539326323};
        case 4: return double2{0.597158591702786164852, 0.802123192755043785083};
        case 5: return double2{0.396079766039156823696, 0.918216106880274014759};
        case 6: return double2{0.173648177666930348852, 0.984807753012208059367};
        case 7: return double2{-0.058144828910475828539, 0.998308158271268208048};
        case 8: return double2{-0.286803232711090253103, 0.957989512315488874437};
        case 9: return double2{-0.5, 0.866025403784438646764};
        case 10: return double2{-0.68624163786873358573, 0.727373641573048695987};
        case 11: return double2{-0.835487811412936419654, 0.549508978070806035263};
        case 12: return double2{-0.939692620785908384054, 0.342020143325668733044};
        case 13: return double2{-0.993238357741942988548, 0.116092914125230229676};
        case 14: return double2{-0.993238357741942988548, -0.116092914125230229676};
        case 15: return double2{-0.939692620785908384054, -0.342020143325668733044};
        case 16: return double2{-0.835487811412936419654, -0.549508978070806035263};
        case 17: return double2{-0.68624163786873358573, -0.727373641573048695987};
        case 18: return double2{-0.5, -0.866025403784438646764};
        case 19: return double2{-0.286803232711090253103, -0.957989512315488874437};
        case 20: return double2{-0.058144828910475828539, -0.998308158271268208048};
        case 21: return double2{0.173648177666930348852, -0.984807753012208059367};
        case 22: return double2{0.396079766039156823696, -0.918216106880274014759};
        case 23: return double2{0.597158591702786164852, -0.802123192755043785083};
        case 24: return double2{0.766044443118978035202, -0.642787609686539326323};
        case 25: return double2{0.893632640323412248193, -0.448799180200462172785};
        case 26: return double2{0.973044870579823838833, -0.23061587074244017845};
        default: return double2{1.0, 0.0};
    }
}

template <int A, int B, typename R> struct DftAB {
    template <typename C> static __device__ __forceinline__ void run(C* v, int sign) {
        constexpr int RR = A * B;
#pragma unroll
        for (int j1 = 0; j1 < A; ++j1) {
            C t[B];
#pragma unroll
            for (int j2 = 0; j2 < B; ++j2) t[j2] = v[j1 + A * j2];
            Dft<B, R>::run(t, sign);
#pragma unroll
            for (int k2 = 0; k2 < B; ++k2) {
                const int m = (j1 * k2) % RR;
                C x = t[k2];
                if (m != 0) {
                    if ((4 * m) % RR == 0) {             // w = i^q: a swap and sign changes
                        const int q = 4 * m / RR;
                        x = q == 2 ? C{-x.x, -x.y} : cmuli(x, R(q == 1 ? sign : -sign));
                    } else {
                        const double2 w = unit_root<RR>(m);
                        x = cmul(x, C{R(w.x), R(sign) * R(w.y)});
                    }
                }
                v[j1 + A * k2] = x;
            }
        }
        C out[RR];
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) {
            C t[A];
#pragma unroll
            for (int j1 = 0; j1 < A; ++j1) t[j1] = v[j1 + A * k2];
            Dft<A, R>::run(t, sign);
#pragma unroll
            for (int k1 = 0; k1 < A; ++k1) out[k2 + B * k1] = t[k1];
        }
#pragma unroll
        for (int k = 0; k < RR; ++k) v[k] = out[k];
    }
};
template <typename R> struct Dft<8, R> : DftAB<2, 4, R> {};
template <typename R> struct Dft<9, R> : DftAB<3, 3, R> {};
template <typename R> struct Dft<14, R> : DftAB<2, 7, R> {};
template <typename R> struct Dft<15, R> : DftAB<3, 5, R> {};
template <typename R> struct Dft<16, R> : DftAB<4, 4, R> {};
template <typename R> struct Dft<18, R> : DftAB<2, 9, R> {};
template <typename R> struct Dft<27, R> : DftAB<3, 9, R> {};

// One Stockham stage of radix RAD: butterfly j reads a[j + r P/RAD], twiddles
// by w^{(j mod Ns) r P/(Ns RAD)}, applies the RAD-point DFT and writes
// b[(j / Ns) Ns RAD + (j mod Ns) + r Ns].
// In the first stage (Ns = 1, FIRST) every twiddle is 1; if moreover only
// a[0 .. nz) can be nonzero and nz <= P / RAD (a zero-padded input), each
// butterfly sees one nonzero input and all its outputs equal it.
template <int RAD, bool FIRST, typename R, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ a, C* __restrict__ b, int P, int Ns, unsigned nsm,
                                               int tstep, const C* tw, int sign, int nz) {
    const int PR = P / RAD;
    if (FIRST && nz <= PR) {
        for (int j = threadIdx.x; j < PR; j += blockDim.x) {
            const C x = a[j];
#pragma unroll
            for (int r = 0; r < RAD; ++r) b[j * RAD + r] = x;
        }
        return;
    }
    for (int j = threadIdx.x; j < PR; j += blockDim.x) {
        const int qd = FIRST ? j : (int)__umulhi((unsigned)j, nsm);       // j / Ns
        const int k = j - qd * Ns;                                         // j % Ns
        const int step = tstep * k;
        C v[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) {
            const C x = a[j + r * PR];
            v[r] = (r == 0 || FIRST) ? x : cmul(x, twiddle(tw, step * r, sign));
        }
        Dft<RAD, R>::run(v, sign);
        const int base = qd * Ns * RAD + k;
#pragma unroll
        for (int r = 0; r < RAD; ++r) b[base + r * Ns] = v[r];
    }
}

// Threads per line and lines per CTA (shared memory (2 LY + 1) P complex
// values).  FP32 runs one warp per line, 8 lines, with warp barriers between
// stages; FP64, bound by its arithmetic, keeps 64 threads per line, 4 lines.
template <typename R> __host__ __device__ constexpr int fft_tx() { return sizeof(R) == 4 ? 32 : 64; }
template <typename R> __host__ __device__ constexpr int fft_ly() { return sizeof(R) == 4 ? 8 : 4; }

// Four-step transform of one line of length P = P1 P2 (P1, P2 <= 32; one
// warp per line).  With n = P2 n1 + n2 and k = k1 + P1 k2,
//   X[k1 + P1 k2] = sum_n2 w_P2^(n2 k2) w_P^(n2 k1) sum_n1 w_P1^(n1 k1) x[P2 n1 + n2],
// w_m = exp(sign 2 pi i / m).  Lane n2 < P2 forms the inner P1-point
// transform in registers and writes it, twiddled, to b[k1 P2 + n2]; after a
// warp barrier lane k1 < P1 forms the outer P2-point transform of
// b[k1 P2 + ...] and writes X in natural order to a.  Two shared-memory
// round trips in all, where a Stockham plan takes one per radix stage.
// a[nz ..) is zero and not read.  Returns a.
template <int P1, int P2, typename R, typename C>
__device__ C* fft_4step(C* a, C* b, const FftDev<R>& L, int sign, int nz) {
    const int t = threadIdx.x;
    if (t < P2) {
        C v[P1];
#pragma unroll
        for (int n1 = 0; n1 < P1; ++n1) {
            const int i = P2 * n1 + t;
            v[n1] = i < nz ? a[i] : C{R(0), R(0)};
        }
        Dft<P1, R>::run(v, sign);
        b[t] = v[0];
#pragma unroll
        for (int k1 = 1; k1 < P1; ++k1) b[k1 * P2 + t] = cmul(v[k1], twiddle(L.tw, t * k1, sign));
    }
    __syncwarp();
    if (t < P1) {
        C u[P2];
#pragma unroll
        for (int n2 = 0; n2 < P2; ++n2) u[n2] = b[t * P2 + n2];
        Dft<P2, R>::run(u, sign);
#pragma unroll
        for (int k2 = 0; k2 < P2; ++k2) a[t + P1 * k2] = u[k2];
    }
    __syncwarp();
    return a;
}

// One line of length P in a[], b[] as scratch (a[nz ..) known to be zero);
// the fft_tx<R>() threads with the same threadIdx.y cooperate.  With one warp per line the stages are
// separated by warp barriers, else by CTA barriers (every thread of the CTA
// must then call this).  Returns the buffer that holds the result (Stockham
// autosort, mixed radix).
// The z pass of the convolution on a four-step line: forward transform,
// product with the Green's function spectrum (lane k1 < P1 brings its
// values gk[k2] = G(k1 + P1 k2) in registers), inverse transform, with
// the spectrum kept in registers between the two.  The forward transform
// leaves X[k1 + P1 k2] in lane k1 (k2 = 0 .. P2-1), which is the inner
// transform's input of the inverse taken as P = P2 P1 (index P1 n1' + n2',
// lane n2' = k1): that lane multiplies by gk, transforms over n1', twiddles
// and writes to a[k1' P1 + n2']; after a warp barrier lane k1' < P2 forms
// the outer P1-point transform and writes the result in natural order to b.
// Three shared-memory round trips instead of four (and of two per radix
// stage in a Stockham plan).  Returns b.
template <int P1, int P2, typename R, typename C>
__device__ C* fft_conv_4step(C* a, C* b, const FftDev<R>& L, int nz, const R (&gk)[P2]) {
    const int t = threadIdx.x;
    if (t < P2) {
        C v[P1];
#pragma unroll
        for (int n1 = 0; n1 < P1; ++n1) {
            const int i = P2 * n1 + t;
            v[n1] = i < nz ? a[i] : C{R(0), R(0)};
        }
        Dft<P1, R>::run(v, -1);
        b[t] = v[0];
#pragma unroll
        for (int k1 = 1; k1 < P1; ++k1) b[k1 * P2 + t] = cmul(v[k1], twiddle(L.tw, t * k1, -1));
    }
    __syncwarp();
    if (t < P1) {
        C u[P2];
#pragma unroll
        for (int n2 = 0; n2 < P2; ++n2) u[n2] = b[t * P2 + n2];
        Dft<P2, R>::run(u, -1);
#pragma unroll
        for (int k2 = 0; k2 < P2; ++k2) {
            u[k2] = C{u[k2].x * gk[k2], u[k2].y * gk[k2]};
        }
        Dft<P2, R>::run(u, +1);
        a[t] = u[0];
#pragma unroll
        for (int k = 1; k < P2; ++k) a[k * P1 + t] = cmul(u[k], twiddle(L.tw, t * k, +1));
    }
    __syncwarp();
    if (t < P2) {
        C w[P1];
#pragma unroll
        for (int n = 0; n < P1; ++n) w[n] = a[t * P1 + n];
        Dft<P1, R>::run(w, +1);
#pragma unroll
        for (int k = 0; k < P1; ++k) b[t + P2 * k] = w[k];
    }
    __syncwarp();
    return b;
}

// PLAN: 0 a Stockham plan of prime radices (and 4), 1 one with composite
// radices, P1 * 100 + P2 the four-step transform of P = P1 P2 (FP32 lines).
template <typename R, int PLAN, typename C>
__device__ C* fft_line(C* a, C* b, const FftDev<R>& L, int sign, int nz) {
    if constexpr (PLAN >= 100) return fft_4step<PLAN / 100, PLAN % 100, R>(a, b, L, sign, nz);
    constexpr bool CMP = PLAN == 1;
    const int P = L.P;
    constexpr int MS = MAX_RADIX_STAGES;
    for (int st = 0; st < L.nrad; ++st) {
        const int RAD = L.st[st], Ns = L.st[MS + st], ts = L.st[2 * MS + st];
        const unsigned nsm = (unsigned)L.st[3 * MS + st];
        if constexpr (!CMP) {
            // plans of prime radices (and 4): 2 first for even P
            if (st == 0) {
                switch (RAD) {
                    case 2: stockham_stage<2, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                    case 3: stockham_stage<3, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                    case 4: stockham_stage<4, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                    case 5: stockham_stage<5, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                    default: stockham_stage<7, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                }
            } else {
                switch (RAD) {
                    case 2: stockham_stage<2, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                    case 3: stockham_stage<3, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                    case 4: stockham_stage<4, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                    case 5: stockham_stage<5, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                    default: stockham_stage<7, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                }
            }
        } else if (st == 0) {
            // plans with composite radices (a separate build, so that the
            // prime-radix lines keep their smaller code): the first radix is 2
            // for even P, else an odd one
            switch (RAD) {
                case 2: stockham_stage<2, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                case 3: stockham_stage<3, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                case 5: stockham_stage<5, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                case 7: stockham_stage<7, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                case 9: stockham_stage<9, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
                default: stockham_stage<15, true, R>(a, b, P, Ns, nsm, ts, L.tw, sign, nz); break;
            }
        } else {
            switch (RAD) {
                case 2: stockham_stage<2, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 3: stockham_stage<3, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 4: stockham_stage<4, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 5: stockham_stage<5, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 7: stockham_stage<7, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 8: stockham_stage<8, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 9: stockham_stage<9, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 14: stockham_stage<14, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                case 15: stockham_stage<15, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
                default: stockham_stage<16, false, R>(a, b, P, Ns, nsm, ts, L.tw, sign, P); break;
            }
        }
        if constexpr (fft_tx<R>() == 32) __syncwarp();
        else __syncthreads();
        C* t = a; a = b; b = t;
    }
    return a;
}


// Copies the line's twiddle table and stage table into shared memory (after
// the CTA's line buffers) and returns the descriptor that reads them from
// there; both are complete when the next __syncthreads() of the caller has
// passed.
template <typename R>
__device__ __forceinline__ FftDev<R> stage_twiddles(const FftLine<R>& Lg, typename Cx<R>::T* stw) {
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    for (int j = tid; j < Lg.P; j += nth) stw[j] = Lg.tw[j];
    int* sst = reinterpret_cast<int*>(stw + Lg.P);
    constexpr int MS = MAX_RADIX_STAGES;
    if (tid < MS) {
        sst[tid] = Lg.rad[tid];
        sst[MS + tid] = Lg.ns[tid];
        sst[2 * MS + tid] = Lg.tstep[tid];
        sst[3 * MS + tid] = (int)Lg.nsm[tid];
    }
    FftDev<R> L;
    L.P = Lg.P;
    L.nrad = Lg.nrad;
    L.st = sst;
    L.tw = stw;
    return L;
}

// Geometry of one convolution: padded lengths, half spectrum, and the input
// (source) and output (target) node ranges per axis (x, y, z).  A node i of a
// range sits at padded index (i + P) mod P.  The circular convolution equals
// the linear one when in_n + out_n - 1 <= P on every axis.
struct Geo {
    int n, nbx, nby, nbz;
    int Px, Py, Pz, Kx, Ky, Kz;
    int in_lo[3], in_n[3], out_lo[3], out_n[3];
    int dense_in, dense_out;   // 0: level-0 block layouts, 1: dense arrays over the ranges
};

// Padded index of a lattice coordinate i in [-P, 2P) (every range here lies inside).
__device__ __forceinline__ int pidx(int i, int P) { return i < 0 ? i + P : (i >= P ? i - P : i); }

// Copies elements e = 0 .. n-1 of the CTA's lines from global into shared
// memory (value src(e), stored by dst(e, v)) with B loads of a thread in
// flight before their stores: the passes are bound by memory latency, and
// with a run-time loop bound one load at a time would be in flight.
// The elements are spread over the whole CTA (WARP = false) or over the
// threads of one line (WARP = true: threadIdx.x).
template <int B, typename C, bool WARP = false, typename S, typename D>
__device__ __forceinline__ void gather_lines(int n, const S& src, const D& dst) {
    const int tid = WARP ? (int)threadIdx.x : (int)(threadIdx.y * blockDim.x + threadIdx.x);
    const int nth = WARP ? (int)blockDim.x : (int)(blockDim.x * blockDim.y);
    for (int e0 = tid; e0 < n; e0 += B * nth) {
        C v[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int e = e0 + i * nth;
            v[i] = e < n ? src(e) : C{};
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            const int e = e0 + i * nth;
            if (e < n) dst(e, v[i]);
        }
    }
}

// ---------------------------------------------------------------- pass A (x, real -> half spectrum)
// lines: input (y, z) range; x input range.  Each warp transforms two real
// lines at once as one complex line z = a + i b; with Z = FFT(z) and
// Z' = conj(Z[(P - k) mod P]), the halves are A = (Z + Z') / 2 and
// B = (Z - Z') / (2 i).
template <typename R, int PLAN>
__global__ void k_fft_x_fwd(typename Cx<R>::T* __restrict__ spec, const R* __restrict__ src, Geo g, FftLine<R> Lg) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char fsm[];
    C* sm = reinterpret_cast<C*>(fsm);
    const FftDev<R> L = stage_twiddles<R>(Lg, sm + fft_ly<R>() * 2 * Lg.P);
    const int nlines = g.in_n[1] * g.in_n[2];
    const int line0 = 2 * (blockIdx.x * fft_ly<R>() + threadIdx.y);
    C* a = sm + threadIdx.y * 2 * L.P;
    C* b = a + L.P;
    for (int j = threadIdx.x; j < L.P; j += blockDim.x) a[j] = C{R(0), R(0)};
    __syncthreads();
    int ty[2], tz[2];
    bool live[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int line = line0 + h;
        live[h] = line < nlines;
        ty[h] = live[h] ? line % g.in_n[1] : 0;
        tz[h] = live[h] ? line / g.in_n[1] : 0;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!live[h]) continue;
        const int y = g.in_lo[1] + ty[h], z = g.in_lo[2] + tz[h];
        gather_lines<8, R, true>(
            g.in_n[0],
            [&](int tx) {
                if (g.dense_in) return src[((size_t)tz[h] * g.in_n[1] + ty[h]) * g.in_n[0] + tx];
                const int x = g.in_lo[0] + tx;
                const int bx = x / g.n, lx = x % g.n, by = y / g.n, ly = y % g.n, bz = z / g.n, lz = z % g.n;
                const int blk = (bz * g.nby + by) * g.nbx + bx;
                return src[(size_t)blk * g.n * g.n * g.n + (lz * g.n + ly) * g.n + lx];
            },
            [&](int tx, R v) {
                const int x = g.in_lo[0] + tx;
                if (h == 0) a[pidx(x, L.P)].x = v;
                else a[pidx(x, L.P)].y = v;
            });
    }
    __syncthreads();
    C* r = fft_line<R, PLAN>(a, b, L, -1, g.in_lo[0] == 0 ? g.in_n[0] : L.P);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!live[h]) continue;
        const int y = g.in_lo[1] + ty[h], z = g.in_lo[2] + tz[h];
        const size_t row = ((size_t)pidx(z, g.Pz) * g.Py + pidx(y, g.Py)) * g.Kx;
        for (int k = threadIdx.x; k < g.Kx; k += blockDim.x) {
            const C zk = r[k], zm = r[k == 0 ? 0 : L.P - k];
            spec[row + k] = h == 0 ? C{R(0.5) * (zk.x + zm.x), R(0.5) * (zk.y - zm.y)}
                                   : C{R(0.5) * (zk.y + zm.y), R(0.5) * (zm.x - zk.x)};
        }
    }
}

// The y and z passes take LY = fft_ly<R>() lines of consecutive kx per CTA.
// Their global loads and stores walk the lines' elements with kx fastest
// across the CTA's threads (element e: line e % LY, position e / LY), so that
// a warp touches whole sectors; the transforms themselves run per line.

// ---------------------------------------------------------------- pass B (y, forward), lines (input z, kx)
template <typename R, int PLAN>
__global__ void k_fft_y_fwd(typename Cx<R>::T* __restrict__ spec, Geo g, FftLine<R> Lg) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char fsm[];
    C* sm = reinterpret_cast<C*>(fsm);
    const FftDev<R> L = stage_twiddles<R>(Lg, sm + fft_ly<R>() * 2 * Lg.P);
    const int P = L.P, P2 = 2 * P;
    const int zi = pidx(g.in_lo[2] + (int)blockIdx.y, g.Pz);
    const int kx0 = blockIdx.x * fft_ly<R>();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    C* a = sm + threadIdx.y * P2;
    C* b = a + P;
    // (four-step lines read only a[0 .. nz), the input itself where it starts at 0)
    if (PLAN < 100 || g.in_lo[1] != 0) {
        for (int j = threadIdx.x; j < P; j += blockDim.x) a[j] = C{R(0), R(0)};
        __syncthreads();
    }
    gather_lines<8, C>(
        fft_ly<R>() * g.in_n[1],
        [&](int e) {
            const int ly = e % fft_ly<R>(), j = pidx(g.in_lo[1] + e / fft_ly<R>(), g.Py);
            return kx0 + ly < g.Kx ? spec[((size_t)zi * g.Py + j) * g.Kx + kx0 + ly] : C{R(0), R(0)};
        },
        [&](int e, C v) { sm[(e % fft_ly<R>()) * P2 + pidx(g.in_lo[1] + e / fft_ly<R>(), g.Py)] = v; });
    __syncthreads();
    const int roff = (int)(fft_line<R, PLAN>(a, b, L, -1, g.in_lo[1] == 0 ? g.in_n[1] : P) - a);
    __syncthreads();
    for (int e = tid; e < fft_ly<R>() * P; e += nth) {
        const int ly = e % fft_ly<R>(), y = e / fft_ly<R>();
        if (kx0 + ly < g.Kx) spec[((size_t)zi * g.Py + y) * g.Kx + kx0 + ly] = sm[ly * P2 + roff + y];
    }
}

// ---------------------------------------------------------------- pass C (z forward, x G-hat, z inverse), lines (ky, kx)
template <typename R, int PLAN>
__device__ __forceinline__ void z_conv_body(typename Cx<R>::T* __restrict__ spec, const R* __restrict__ ghat, Geo g,
                                            FftLine<R> Lg) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char fsm[];
    C* sm = reinterpret_cast<C*>(fsm);
    const FftDev<R> L = stage_twiddles<R>(Lg, sm + fft_ly<R>() * 2 * Lg.P);
    const int P = L.P, P2 = 2 * P;
    const int ky = blockIdx.y;
    const int kx0 = blockIdx.x * fft_ly<R>();
    const int kx = kx0 + threadIdx.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    C* a = sm + threadIdx.y * P2;
    C* b = a + P;
    const bool live = kx < g.Kx;
    // (four-step lines read only a[0 .. nz), the input itself where it starts at 0)
    if (PLAN < 100 || g.in_lo[2] != 0) {
        for (int j = threadIdx.x; j < P; j += blockDim.x) a[j] = C{R(0), R(0)};
        __syncthreads();
    }
    gather_lines<8, C>(
        fft_ly<R>() * g.in_n[2],
        [&](int e) {
            const int ly = e % fft_ly<R>(), j = pidx(g.in_lo[2] + e / fft_ly<R>(), g.Pz);
            return kx0 + ly < g.Kx ? spec[((size_t)j * g.Py + ky) * g.Kx + kx0 + ly] : C{R(0), R(0)};
        },
        [&](int e, C v) { sm[(e % fft_ly<R>()) * P2 + pidx(g.in_lo[2] + e / fft_ly<R>(), g.Pz)] = v; });
    // the line's G-hat values, fetched now so that their latency overlaps the
    // input's (the first GPRE per thread in registers, the rest later)
    constexpr int GPRE = sizeof(R) == 4 ? 8 : 4;
    const int fy = ky <= g.Py - ky ? ky : g.Py - ky;
    auto ghat_at = [&](int kz) {
        const int fz = kz <= g.Pz - kz ? kz : g.Pz - kz;
        return live ? ghat[((size_t)fz * g.Ky + fy) * g.Kx + kx] : R(0);
    };
    int qoff;
    if constexpr (PLAN >= 100) {
        // the G-hat values of lane k1 (k = k1 + P1 k2), fetched with the input
        constexpr int P1 = PLAN / 100, P2 = PLAN % 100;
        R gk[P2];
#pragma unroll
        for (int k2 = 0; k2 < P2; ++k2) gk[k2] = threadIdx.x < P1 ? ghat_at(threadIdx.x + P1 * k2) : R(0);
        __syncthreads();
        qoff = (int)(fft_conv_4step<P1, P2, R>(a, b, L, g.in_lo[2] == 0 ? g.in_n[2] : P, gk) - a);
        __syncthreads();
    } else {
    R gpre[GPRE];
#pragma unroll
    for (int m = 0; m < GPRE; ++m) {
        const int kz = threadIdx.x + m * blockDim.x;
        gpre[m] = kz < P ? ghat_at(kz) : R(0);
    }
    __syncthreads();
    C* r = fft_line<R, PLAN>(a, b, L, -1, g.in_lo[2] == 0 ? g.in_n[2] : P);
#pragma unroll
    for (int m = 0; m < GPRE; ++m) {
        const int kz = threadIdx.x + m * blockDim.x;
        if (kz < P) r[kz] = C{r[kz].x * gpre[m], r[kz].y * gpre[m]};
    }
    for (int kz = threadIdx.x + GPRE * blockDim.x; kz < P; kz += blockDim.x) {
        const R gv = ghat_at(kz);
        r[kz] = C{r[kz].x * gv, r[kz].y * gv};
    }
    __syncthreads();
    C* other = (r == a) ? b : a;
    qoff = (int)(fft_line<R, PLAN>(r, other, L, +1, P) - a);
    __syncthreads();
    }
    for (int e = tid; e < fft_ly<R>() * g.out_n[2]; e += nth) {
        const int ly = e % fft_ly<R>(), t = e / fft_ly<R>();
        if (kx0 + ly >= g.Kx) continue;
        const int z = pidx(g.out_lo[2] + t, g.Pz);
        spec[((size_t)z * g.Py + ky) * g.Kx + kx0 + ly] = sm[ly * P2 + qoff + z];
    }
}

// Registers capped for 3 CTAs of 256 threads per SM (the FP32 shared-memory
// limit): the pass is bound by memory latency.
template <typename R, int PLAN>
__global__ void __launch_bounds__(256, 3)
k_fft_z_conv(typename Cx<R>::T* __restrict__ spec, const R* __restrict__ ghat, Geo g, FftLine<R> Lg) {
    z_conv_body<R, PLAN>(spec, ghat, g, Lg);
}

// ---------------------------------------------------------------- pass B' (y inverse), lines (output z, kx)
template <typename R, int PLAN>
__global__ void k_fft_y_inv(typename Cx<R>::T* __restrict__ spec, Geo g, FftLine<R> Lg) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char fsm[];
    C* sm = reinterpret_cast<C*>(fsm);
    const FftDev<R> L = stage_twiddles<R>(Lg, sm + fft_ly<R>() * 2 * Lg.P);
    const int P = L.P, P2 = 2 * P;
    const int z = pidx(g.out_lo[2] + (int)blockIdx.y, g.Pz);
    const int kx0 = blockIdx.x * fft_ly<R>();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
    C* a = sm + threadIdx.y * P2;
    C* b = a + P;
    gather_lines<8, C>(
        fft_ly<R>() * P,
        [&](int e) {
            const int ly = e % fft_ly<R>(), y = e / fft_ly<R>();
            return kx0 + ly < g.Kx ? spec[((size_t)z * g.Py + y) * g.Kx + kx0 + ly] : C{R(0), R(0)};
        },
        [&](int e, C v) { sm[(e % fft_ly<R>()) * P2 + e / fft_ly<R>()] = v; });
    __syncthreads();
    const int roff = (int)(fft_line<R, PLAN>(a, b, L, +1, P) - a);
    __syncthreads();
    for (int e = tid; e < fft_ly<R>() * g.out_n[1]; e += nth) {
        const int ly = e % fft_ly<R>(), t = e / fft_ly<R>();
        if (kx0 + ly >= g.Kx) continue;
        const int y = pidx(g.out_lo[1] + t, g.Py);
        spec[((size_t)z * g.Py + y) * g.Kx + kx0 + ly] = sm[ly * P2 + roff + y];
    }
}

// ---------------------------------------------------------------- pass A' (x inverse, half spectrum -> real)
// lines: output (y, z) range.  Each warp inverts two Hermitian lines at once
// as one complex line A + i B, whose real and imaginary parts are the two
// real outputs.  Block mode writes node (x, y, z) into every level-0 block
// whose (n+2)^3 box holds it (interior or ghost layer); dense mode writes the
// dense output range.
template <typename R, int PLAN>
__global__ void k_fft_x_inv(R* __restrict__ dst, const typename Cx<R>::T* __restrict__ spec, Geo g, FftLine<R> Lg) {
    using C = typename Cx<R>::T;
    extern __shared__ __align__(16) unsigned char fsm[];
    C* sm = reinterpret_cast<C*>(fsm);
    const FftDev<R> L = stage_twiddles<R>(Lg, sm + fft_ly<R>() * 2 * Lg.P);
    const int nlines = g.out_n[1] * g.out_n[2];
    const int line0 = 2 * (blockIdx.x * fft_ly<R>() + threadIdx.y);
    C* a = sm + threadIdx.y * 2 * L.P;
    C* b = a + L.P;
    int oy[2], oz[2];
    bool live[2];
    const C* src[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int line = line0 + h;
        live[h] = line < nlines;
        oy[h] = live[h] ? line % g.out_n[1] : 0;
        oz[h] = live[h] ? line / g.out_n[1] : 0;
        src[h] = spec + ((size_t)pidx(g.out_lo[2] + oz[h], g.Pz) * g.Py + pidx(g.out_lo[1] + oy[h], g.Py)) * g.Kx;
    }
    gather_lines<8, C, true>(
        L.P,
        [&](int k) {
            C v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                v[h] = C{R(0), R(0)};
                if (live[h]) {
                    if (k < g.Kx) v[h] = src[h][k];
                    else { v[h] = src[h][L.P - k]; v[h].y = -v[h].y; }
                }
            }
            return C{v[0].x - v[1].y, v[0].y + v[1].x};
        },
        [&](int k, C v) { a[k] = v; });
    __syncthreads();
    C* r = fft_line<R, PLAN>(a, b, L, +1, L.P);
    const int S = g.n + 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (!live[h]) continue;
        const int ty = g.out_lo[1] + oy[h], tz = g.out_lo[2] + oz[h];
        if (g.dense_out) {
            for (int ox = threadIdx.x; ox < g.out_n[0]; ox += blockDim.x) {
                const C w = r[pidx(g.out_lo[0] + ox, g.Px)];
                dst[((size_t)oz[h] * g.out_n[1] + oy[h]) * g.out_n[0] + ox] = h == 0 ? w.x : w.y;
            }
            continue;
        }
        for (int ox = threadIdx.x; ox < g.out_n[0]; ox += blockDim.x) {
            const int tx = g.out_lo[0] + ox;
            const C w = r[pidx(tx, g.Px)];
            const R val = h == 0 ? w.x : w.y;
            for (int bz = (tz - 1 < 0 ? -1 : (tz - 1) / g.n); bz <= (tz + 1) / g.n; ++bz) {
                if (bz < 0 || bz >= g.nbz || tz < bz * g.n - 1 || tz > bz * g.n + g.n) continue;
                for (int by = (ty - 1 < 0 ? -1 : (ty - 1) / g.n); by <= (ty + 1) / g.n; ++by) {
                    if (by < 0 || by >= g.nby || ty < by * g.n - 1 || ty > by * g.n + g.n) continue;
                    for (int bx = (tx - 1 < 0 ? -1 : (tx - 1) / g.n); bx <= (tx + 1) / g.n; ++bx) {
                        if (bx < 0 || bx >= g.nbx || tx < bx * g.n - 1 || tx > bx * g.n + g.n) continue;
                        const int blk = (bz * g.nby + by) * g.nbx + bx;
                        const int lx = tx - bx * g.n + 1, ly = ty - by * g.n + 1, lz = tz - bz * g.n + 1;
                        dst[(size_t)blk * S * S * S + (lz * S + ly) * S + lx] = val;
                    }
                }
            }
        }
    }
}

// Forward geometry of problem p: sources on level-0 nodes [0, N0), targets [-1, N0].
static Geo geo_of(const Handle& h, const Problem& p) {
    Geo g{};
    g.n = h.n;
    g.nbx = p.nb0[0]; g.nby = p.nb0[1]; g.nbz = p.nb0[2];
    g.Px = p.ax[0].P; g.Py = p.ax[1].P; g.Pz = p.ax[2].P;
    g.Kx = p.gK[0]; g.Ky = p.gK[1]; g.Kz = p.gK[2];
    for (int a = 0; a < 3; ++a) {
        g.in_lo[a] = 0; g.in_n[a] = p.n0[a];
        g.out_lo[a] = -1; g.out_n[a] = p.n0[a] + 2;
    }
    return g;
}

// Whether a line's plan holds a composite radix (8, 9, 14, 15, 16).
template <typename R>
static bool has_composite(const FftLine<R>& l) {
    for (int i = 0; i < l.nrad; ++i)
        if (l.rad[i] > 7) return true;
    return false;
}

// FP32 line lengths with a four-step build (P1 * 100 + P2, P = P1 P2), else 0:
// the solver's own level-0 lattice (N0 = 96, P = 196), the 240^3 lattice
// (P = 486) and a smaller one (P = 144).
static int fourstep_plan(int P) {
    switch (P) {
        case 144: return 916;
        case 196: return 1414;
        case 486: return 1827;
        default: return 0;
    }
}

template <typename R>
static void conv_passes(const Problem& p, const Geo& g, typename Cx<R>::T* spec, const R* ghat, const R* src, R* dst,
                        cudaStream_t s) {
    using C = typename Cx<R>::T;
    const dim3 blk(fft_tx<R>(), fft_ly<R>());
    const FftLine<R> Lx = line_of<R>(p.ax[0]), Ly = line_of<R>(p.ax[1]), Lz = line_of<R>(p.ax[2]);
    const size_t smx = sizeof(C) * (2 * fft_ly<R>() + 1) * g.Px + FFT_STAGE_BYTES;
    const size_t smy = sizeof(C) * (2 * fft_ly<R>() + 1) * g.Py + FFT_STAGE_BYTES;
    const size_t smz = sizeof(C) * (2 * fft_ly<R>() + 1) * g.Pz + FFT_STAGE_BYTES;
    const int kxb = (g.Kx + fft_ly<R>() - 1) / fft_ly<R>();
    const int lx2 = 2 * fft_ly<R>();   // lines per CTA in the x passes (two per warp)
    // FP32 lines take the four-step build where their length has one, else
    // the composite-radix build where their plan holds a composite radix
    constexpr bool F32 = sizeof(R) == 4;
#define MRP_FFT_LAUNCH(KERN, LINE, GRID, SM, ...)                                      \
    do {                                                                               \
        if constexpr (F32) {                                                           \
            const int fs = fourstep_plan(LINE.P);                                      \
            if (fs == 916) KERN<R, 916><<<GRID, blk, SM, s>>>(__VA_ARGS__);            \
            else if (fs == 1414) KERN<R, 1414><<<GRID, blk, SM, s>>>(__VA_ARGS__);     \
            else if (fs == 1827) KERN<R, 1827><<<GRID, blk, SM, s>>>(__VA_ARGS__);     \
            else if (has_composite(LINE)) KERN<R, 1><<<GRID, blk, SM, s>>>(__VA_ARGS__); \
            else KERN<R, 0><<<GRID, blk, SM, s>>>(__VA_ARGS__);                        \
        } else {                                                                       \
            KERN<R, 0><<<GRID, blk, SM, s>>>(__VA_ARGS__);                             \
        }                                                                              \
    } while (0)
    MRP_FFT_LAUNCH(k_fft_x_fwd, Lx, (g.in_n[1] * g.in_n[2] + lx2 - 1) / lx2, smx, spec, src, g, Lx);
    MRP_FFT_LAUNCH(k_fft_y_fwd, Ly, dim3(kxb, g.in_n[2]), smy, spec, g, Ly);
    {
        const int fz = F32 ? fourstep_plan(Lz.P) : 0;
        const dim3 gz(kxb, g.Py);
        if constexpr (F32) {
            if (fz == 916) k_fft_z_conv<R, 916><<<gz, blk, smz, s>>>(spec, ghat, g, Lz);
            else if (fz == 1414) k_fft_z_conv<R, 1414><<<gz, blk, smz, s>>>(spec, ghat, g, Lz);
            else if (fz == 1827) k_fft_z_conv<R, 1827><<<gz, blk, smz, s>>>(spec, ghat, g, Lz);
            else if (has_composite(Lz)) k_fft_z_conv<R, 1><<<gz, blk, smz, s>>>(spec, ghat, g, Lz);
            else k_fft_z_conv<R, 0><<<gz, blk, smz, s>>>(spec, ghat, g, Lz);
        } else {
            k_fft_z_conv<R, 0><<<gz, blk, smz, s>>>(spec, ghat, g, Lz);
        }
    }
    MRP_FFT_LAUNCH(k_fft_y_inv, Ly, dim3(kxb, g.out_n[2]), smy, spec, g, Ly);
    MRP_FFT_LAUNCH(k_fft_x_inv, Lx, (g.out_n[1] * g.out_n[2] + lx2 - 1) / lx2, smx, dst, spec, g, Lx);
#undef MRP_FFT_LAUNCH
}

// Level-0 solve of every problem of the handle, one after another on s (they
// share the spectral buffer); problem p's level-0 blocks start at block base0.
template <typename T>
void launch_coarse_solve_t(const Handle& h, const T* F0, T* U0, cudaStream_t s) {
    const size_t n3 = (size_t)h.n * h.n * h.n, S3 = (size_t)(h.n + 2) * (h.n + 2) * (h.n + 2);
    for (const Problem& p : h.pr) {
        if constexpr (sizeof(T) == 8)
            conv_passes<double>(p, geo_of(h, p), h.spec, p.ghat, F0 + p.base0 * n3, U0 + p.base0 * S3, s);
        else
            conv_passes<float>(p, geo_of(h, p), h.spec32, p.ghat32, F0 + p.base0 * n3, U0 + p.base0 * S3, s);
    }
}
template void launch_coarse_solve_t<double>(const Handle&, const double*, double*, cudaStream_t);
template void launch_coarse_solve_t<float>(const Handle&, const float*, float*, cudaStream_t);

// Same five passes for problem 0 with the spectral buffer, source and output
// given by the caller (spec must hold Pz * Py * (Px/2+1) complex values).
void launch_coarse_solve_ext(const Handle& h, double2* spec, const double* F0, double* U0, cudaStream_t s) {
    const Problem& p = h.pr[0];
    conv_passes<double>(p, geo_of(h, p), spec, p.ghat, F0, U0, s);
}

// Transpose of problem p's level-0 convolution: dense adjoint on the target
// cube [-1, N0]^3 -> dense adjoint on the sources [0, N0)^3 (FP64, or FP32
// with the FP32 spectrum of a mixed-precision handle).  The kernel is even,
// so this is the convolution with the two ranges exchanged.
template <typename T>
void launch_conv_transpose(const Handle& h, const Problem& p, const T* cube_in, T* src_out, cudaStream_t s) {
    Geo g = geo_of(h, p);
    for (int a = 0; a < 3; ++a) {
        g.in_lo[a] = -1; g.in_n[a] = p.n0[a] + 2;
        g.out_lo[a] = 0; g.out_n[a] = p.n0[a];
    }
    g.dense_in = 1;
    g.dense_out = 1;
    if constexpr (sizeof(T) == 8) conv_passes<double>(p, g, h.spec, p.ghat, cube_in, src_out, s);
    else conv_passes<float>(p, g, h.spec32, p.ghat32, cube_in, src_out, s);
}
template void launch_conv_transpose<double>(const Handle&, const Problem&, const double*, double*, cudaStream_t);
template void launch_conv_transpose<float>(const Handle&, const Problem&, const float*, float*, cudaStream_t);

// ============================================================================
// Lattice Green's function (FP64).  G[n] = (2pi)^-3 int cos(k.n) / sigma(k) dk
// with sigma the symbol of the unit-spacing LHS stencil.  sigma is affine in
// s3 = 4 sin^2(k3/2): sigma = -(c0 + c1 s3), so the k3 integral is closed:
// (1/2pi) int cos(n3 k3)/(a - b cos k3) = rho^|n3| / sqrt(a^2 - b^2),
// a = c0 + 2 c1, b = 2 c1, rho = b / (a + sqrt(a^2 - b^2)).  The (k1, k2)
// integral over [0,pi]^2 is split into the triangles k2 <= k1 and k1 <= k2
// and Duffy-mapped (k1, k2) = (u, u v), which removes the 1/|k| singularity;
// composite Gauss-Legendre in u and v.
//
// Per u-node i:   B[i][n2][n3] = sum_j cos(n2 u_i v_j) W_ij rho_ij^n3
// then            A[n1][n2][n3] = sum_i cos(n1 u_i) B[i][n2][n3]
//                 G = -(A + A^T(n1<->n2)) / pi^2.
constexpr int LGF_JT = 32;

__global__ void k_lgf_B(double* __restrict__ Bout, const double* __restrict__ u, const double* __restrict__ v,
                        const double* __restrict__ W, const double* __restrict__ rho, int Qv, int nn) {
    extern __shared__ double lsm[];
    double* ct = lsm;                    // [nn][JT]
    double* pt = lsm + nn * LGF_JT;      // [nn][JT]
    const int i = blockIdx.x;
    const double ui = u[i];
    double* Bi = Bout + (size_t)i * nn * nn;
    for (int t = threadIdx.x; t < nn * nn; t += blockDim.x) Bi[t] = 0.0;
    for (int j0 = 0; j0 < Qv; j0 += LGF_JT) {
        const int jn = min(LGF_JT, Qv - j0);
        __syncthreads();
        for (int t = threadIdx.x; t < nn * LGF_JT; t += blockDim.x) {
            const int n2 = t / LGF_JT, jj = t % LGF_JT;
            ct[t] = jj < jn ? cos((double)n2 * (ui * v[j0 + jj])) : 0.0;
        }
        for (int jj = threadIdx.x; jj < LGF_JT; jj += blockDim.x) {
            double p = jj < jn ? W[(size_t)i * Qv + j0 + jj] : 0.0;
            const double r = jj < jn ? rho[(size_t)i * Qv + j0 + jj] : 0.0;
            for (int n3 = 0; n3 < nn; ++n3) { pt[n3 * LGF_JT + jj] = p; p *= r; }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nn * nn; t += blockDim.x) {
            const int n2 = t / nn, n3 = t % nn;
            double acc = 0.0;
            for (int jj = 0; jj < LGF_JT; ++jj) acc += ct[n2 * LGF_JT + jj] * pt[n3 * LGF_JT + jj];
            Bi[t] += acc;
        }
    }
}

__global__ void k_lgf_A(double* __restrict__ A, const double* __restrict__ B, const double* __restrict__ C1,
                        int Qu, int nn) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nn * nn * nn) return;
    const int n1 = (int)(t / ((size_t)nn * nn));
    const size_t r = t % ((size_t)nn * nn);
    double acc = 0.0;
    for (int i = 0; i < Qu; ++i) acc += C1[(size_t)n1 * Qu + i] * B[(size_t)i * nn * nn + r];
    A[t] = acc;
}

__global__ void k_lgf_sym(double* __restrict__ G, const double* __restrict__ A, int nn) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)nn * nn * nn) return;
    const int n1 = (int)(t / ((size_t)nn * nn)), n2 = (int)((t / nn) % nn), n3 = (int)(t % nn);
    const double pi = 3.14159265358979323846;
    G[t] = -(A[t] + A[((size_t)n2 * nn + n1) * nn + n3]) / (pi * pi);
}

// Spectrum of the even padded kernel g[i] = G[min(i, P-i)] by separable
// cosine sums; out[kz][ky][kx] over the octant k_a in [0, P_a/2].
// pass 1: T1[dz][dy][kx] = sum_ix G[dz][dy][d(ix)] cos(2 pi kx ix / Px)
__global__ void k_ghat_x(double* __restrict__ T1, const double* __restrict__ G, int nn, const double* __restrict__ cx,
                         int Px, int Dz, int Dy, int Kx) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)Dz * Dy * Kx) return;
    const int kx = (int)(t % Kx), dy = (int)((t / Kx) % Dy), dz = (int)(t / ((size_t)Kx * Dy));
    const double* g = G + ((size_t)dz * nn + dy) * nn;
    double acc = 0.0;
    for (int i = 0; i < Px; ++i) acc += g[i <= Px - i ? i : Px - i] * cx[((size_t)kx * i) % Px];
    T1[t] = acc;
}
// pass 2: T2[dz][ky][kx] = sum_iy T1[dz][d(iy)][kx] cos(2 pi ky iy / Py)
__global__ void k_ghat_y(double* __restrict__ T2, const double* __restrict__ T1, const double* __restrict__ cy,
                         int Py, int Dz, int Dy, int Ky, int Kx) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)Dz * Ky * Kx) return;
    const int kx = (int)(t % Kx), ky = (int)((t / Kx) % Ky), dz = (int)(t / ((size_t)Kx * Ky));
    double acc = 0.0;
    for (int i = 0; i < Py; ++i)
        acc += T1[((size_t)dz * Dy + (i <= Py - i ? i : Py - i)) * Kx + kx] * cy[((size_t)ky * i) % Py];
    T2[t] = acc;
}
// pass 3: ghat[kz][ky][kx] = scale * sum_iz T2[d(iz)][ky][kx] cos(2 pi kz iz / Pz)
__global__ void k_ghat_z(double* __restrict__ out, const double* __restrict__ T2, const double* __restrict__ cz,
                         int Pz, int Kz, int Ky, int Kx, double scale) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)Kz * Ky * Kx) return;
    const int kx = (int)(t % Kx), ky = (int)((t / Kx) % Ky), kz = (int)(t / ((size_t)Kx * Ky));
    double acc = 0.0;
    for (int i = 0; i < Pz; ++i)
        acc += T2[((size_t)(i <= Pz - i ? i : Pz - i) * Ky + ky) * Kx + kx] * cz[((size_t)kz * i) % Pz];
    out[t] = scale * acc;
}

// ---------------------------------------------------------------- host side of the tabulation
// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_q.
static void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
    x.resize(q);
    w.resize(q);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < q; ++i) {
        double z = std::cos(pi * (i + 0.75) / (q + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= q; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            // p1 = P_q(z), p0 = P_{q-1}(z)
            const double dp = q * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                double a0 = 1.0, a1 = z;
                for (int k = 2; k <= q; ++k) { const double a2 = ((2 * k - 1) * z * a1 - (k - 1) * a0) / k; a0 = a1; a1 = a2; }
                const double d = q * (z * a1 - a0) / (z * z - 1.0);
                x[i] = -z;
                w[i] = 2.0 / ((1.0 - z * z) * d * d);
                break;
            }
        }
    }
}

static void composite(int q, double a, double b, int panels, std::vector<double>& xs, std::vector<double>& ws) {
    std::vector<double> x, w;
    gauss_legendre(q, x, w);
    xs.clear();
    ws.clear();
    for (int p = 0; p < panels; ++p) {
        const double lo = a + (b - a) * p / panels, hi = a + (b - a) * (p + 1) / panels;
        for (int i = 0; i < q; ++i) {
            xs.push_back(0.5 * (hi - lo) * x[i] + 0.5 * (hi + lo));
            ws.push_back(0.5 * (hi - lo) * w[i]);
        }
    }
}

#define CK(call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { goto fail; } } while (0)

// Spectrum of problem p's padded kernel, scaled by h0^2 / (Px Py Pz) with the handle's h0.
static int ghat_build(const Handle& h, Problem& p, cudaStream_t s) {
    const double pi = 3.14159265358979323846;
    const int nn = h.lgf_nmax + 1;
    const int Kx = p.gK[0], Ky = p.gK[1], Kz = p.gK[2];
    const int Dz = p.ax[2].P / 2 + 1, Dy = p.ax[1].P / 2 + 1;
    double *dc[3] = {nullptr, nullptr, nullptr}, *T1 = nullptr, *T2 = nullptr;
    int rc = MRP_ERR_CUDA;
    double scale;
    for (int a = 0; a < 3; ++a) {
        const int P = p.ax[a].P;
        std::vector<double> c(P);
        for (int m = 0; m < P; ++m) c[m] = std::cos(2.0 * pi * (double)m / (double)P);
        CK(cudaMalloc(&dc[a], sizeof(double) * P));
        CK(cudaMemcpyAsync(dc[a], c.data(), sizeof(double) * P, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    CK(cudaMalloc(&T1, sizeof(double) * (size_t)Dz * Dy * Kx));
    CK(cudaMalloc(&T2, sizeof(double) * (size_t)Dz * Ky * Kx));
    CK(cudaMalloc(&p.ghat, sizeof(double) * (size_t)Kz * Ky * Kx));
    k_ghat_x<<<(unsigned)(((size_t)Dz * Dy * Kx + 255) / 256), 256, 0, s>>>(T1, h.lgf, nn, dc[0], p.ax[0].P, Dz, Dy, Kx);
    k_ghat_y<<<(unsigned)(((size_t)Dz * Ky * Kx + 255) / 256), 256, 0, s>>>(T2, T1, dc[1], p.ax[1].P, Dz, Dy, Ky, Kx);
    scale = h.h0 * h.h0 / ((double)p.ax[0].P * p.ax[1].P * p.ax[2].P);
    k_ghat_z<<<(unsigned)(((size_t)Kz * Ky * Kx + 255) / 256), 256, 0, s>>>(p.ghat, T2, dc[2], p.ax[2].P, Kz, Ky, Kx, scale);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    rc = MRP_OK;
fail:
    cudaFree(T1); cudaFree(T2);
    for (int a = 0; a < 3; ++a) cudaFree(dc[a]);
    return rc;
}

int lgf_build(Handle& h, cudaStream_t s) {
    const double pi = 3.14159265358979323846;
    int nmax = 0;
    for (const Problem& p : h.pr)
        for (int a = 0; a < 3; ++a) nmax = std::max(nmax, p.ax[a].P / 2);
    const int nn = nmax + 1;
    // quadrature: 32-point rules on 8 + nmax/16 panels in u and 4 + nmax/32 panels in v
    std::vector<double> u, wu, v, wv;
    composite(32, 0.0, pi, 8 + nmax / 16, u, wu);
    composite(32, 0.0, 1.0, 4 + nmax / 32, v, wv);
    const int Qu = (int)u.size(), Qv = (int)v.size();
    std::vector<double> W((size_t)Qu * Qv), rho((size_t)Qu * Qv), C1((size_t)nn * Qu);
    for (int i = 0; i < Qu; ++i)
        for (int j = 0; j < Qv; ++j) {
            const double k1 = u[i], k2 = u[i] * v[j];
            const double s1 = 4.0 * std::sin(0.5 * k1) * std::sin(0.5 * k1);
            const double s2 = 4.0 * std::sin(0.5 * k2) * std::sin(0.5 * k2);
            double c0, c1;
            if (h.M == 2) { c0 = s1 + s2; c1 = 1.0; }
            else {
                c0 = s1 + s2 - s1 * s2 / 6.0;
                c1 = 1.0 - (s1 + s2) / 6.0;
                if (h.M == 6) c1 += s1 * s2 / 30.0;
            }
            const double sq = std::sqrt(c0 * (c0 + 4.0 * c1));
            rho[(size_t)i * Qv + j] = 2.0 * c1 / (c0 + 2.0 * c1 + sq);
            W[(size_t)i * Qv + j] = wu[i] * wv[j] * u[i] / sq;
        }
    for (int n1 = 0; n1 < nn; ++n1)
        for (int i = 0; i < Qu; ++i) C1[(size_t)n1 * Qu + i] = std::cos(n1 * u[i]);
    double *du = nullptr, *dv = nullptr, *dW = nullptr, *drho = nullptr, *dC1 = nullptr, *dB = nullptr, *dA = nullptr;
    int rc = MRP_ERR_CUDA;
    size_t total;
    h.lgf_nmax = nmax;
    CK(cudaMalloc(&h.lgf, sizeof(double) * nn * nn * nn));
    CK(cudaMalloc(&du, sizeof(double) * Qu));
    CK(cudaMalloc(&dv, sizeof(double) * Qv));
    CK(cudaMalloc(&dW, sizeof(double) * Qu * Qv));
    CK(cudaMalloc(&drho, sizeof(double) * Qu * Qv));
    CK(cudaMalloc(&dC1, sizeof(double) * nn * Qu));
    CK(cudaMalloc(&dB, sizeof(double) * (size_t)Qu * nn * nn));
    CK(cudaMalloc(&dA, sizeof(double) * (size_t)nn * nn * nn));
    CK(cudaMemcpyAsync(du, u.data(), sizeof(double) * Qu, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dv, v.data(), sizeof(double) * Qv, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dW, W.data(), sizeof(double) * Qu * Qv, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(drho, rho.data(), sizeof(double) * Qu * Qv, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dC1, C1.data(), sizeof(double) * nn * Qu, cudaMemcpyHostToDevice, s));
    CK(cudaFuncSetAttribute(k_lgf_B, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * nn * LGF_JT * (int)sizeof(double)));
    k_lgf_B<<<Qu, 256, 2 * nn * LGF_JT * sizeof(double), s>>>(dB, du, dv, dW, drho, Qv, nn);
    total = (size_t)nn * nn * nn;
    k_lgf_A<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(dA, dB, dC1, Qu, nn);
    k_lgf_sym<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(h.lgf, dA, nn);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    rc = MRP_OK;
    for (Problem& p : h.pr)
        if ((rc = ghat_build(h, p, s)) != MRP_OK) break;
fail:
    cudaFree(du); cudaFree(dv); cudaFree(dW); cudaFree(drho); cudaFree(dC1); cudaFree(dB); cudaFree(dA);
    return rc;
}

// ---------------------------------------------------------------- FFT plan
// Radices of P: a single 2 first when P is even (the first stage of a
// zero-padded forward line then only copies, since the padding takes at
// least half the line); then, where the stage still gives every thread of a
// line a butterfly (P / R >= minb), two prime factors per stage with a
// composite butterfly (16, 8, 9, 15, 14: one shared-memory round trip instead
// of two); then 4, and the primes left.
static bool factor(int P, int* rad, int& nrad, int minb) {
    nrad = 0;
    const int P0 = P;
    if (P % 2 == 0) { rad[nrad++] = 2; P /= 2; }
    int c2 = 0, c3 = 0, c5 = 0, c7 = 0;
    while (P % 2 == 0) { ++c2; P /= 2; }
    while (P % 3 == 0) { ++c3; P /= 3; }
    while (P % 5 == 0) { ++c5; P /= 5; }
    while (P % 7 == 0) { ++c7; P /= 7; }
    if (P != 1) return false;
    std::vector<int> r;
    auto ok = [&](int R) { return P0 / R >= minb; };
    for (; c2 >= 4 && ok(16); c2 -= 4) r.push_back(16);
    for (; c2 >= 3 && ok(8); c2 -= 3) r.push_back(8);
    for (; c3 >= 2 && ok(9); c3 -= 2) r.push_back(9);
    for (; c3 >= 1 && c5 >= 1 && ok(15); --c3, --c5) r.push_back(15);
    for (; c2 >= 1 && c7 >= 1 && ok(14); --c2, --c7) r.push_back(14);
    for (; c2 >= 2; c2 -= 2) r.push_back(4);
    for (; c2 >= 1; --c2) r.push_back(2);
    for (; c3 >= 1; --c3) r.push_back(3);
    for (; c5 >= 1; --c5) r.push_back(5);
    for (; c7 >= 1; --c7) r.push_back(7);
    if (nrad + (int)r.size() > MAX_RADIX_STAGES) return false;
    for (int x : r) rad[nrad++] = x;
    return true;
}

static int smooth_length(int need) {
    for (int P = need;; ++P) {
        int m = P;
        for (int r : {2, 3, 5, 7}) while (m % r == 0) m /= r;
        if (m == 1) return P;
    }
}

int fft_plan(Handle& h) {
    const double pi = 3.14159265358979323846;
    size_t ns = 0;
    for (Problem& p : h.pr) {
        for (int a = 0; a < 3; ++a) {
            FftAxis& ax = p.ax[a];
            ax.P = smooth_length(2 * p.n0[a] + 1);
            ax.K = ax.P / 2 + 1;
            // FP64 lines (bound by their arithmetic) keep one prime per stage; FP32
            // lines take the composite radices that leave a butterfly per thread
            if (!factor(ax.P, ax.rad, ax.nrad, ax.P + 1) || !factor(ax.P, ax.rad32, ax.nrad32, fft_tx<float>()))
                return MRP_ERR_UNSUPPORTED;
            // a CTA holds (2 LY + 1) P complex values of its lines and twiddles, and the stage table
            if (sizeof(double2) * (2 * fft_ly<double>() + 1) * (size_t)ax.P + FFT_STAGE_BYTES > (size_t)MAX_DYN_SMEM ||
                sizeof(float2) * (2 * fft_ly<float>() + 1) * (size_t)ax.P + FFT_STAGE_BYTES > (size_t)MAX_DYN_SMEM)
                return MRP_ERR_UNSUPPORTED;
            std::vector<double2> tw(ax.P);
            for (int m = 0; m < ax.P; ++m) {
                const double ang = 2.0 * pi * (double)m / (double)ax.P;
                tw[m] = make_double2(std::cos(ang), -std::sin(ang));
            }
            if (cudaMalloc(&ax.tw, sizeof(double2) * ax.P) != cudaSuccess) return MRP_ERR_OOM;
            if (cudaMemcpy(ax.tw, tw.data(), sizeof(double2) * ax.P, cudaMemcpyHostToDevice) != cudaSuccess)
                return MRP_ERR_CUDA;
            p.gK[a] = ax.K;
        }
        ns = std::max(ns, (size_t)p.ax[2].P * p.ax[1].P * p.ax[0].K);
    }
    if (cudaMalloc(&h.spec, sizeof(double2) * ns) != cudaSuccess) return MRP_ERR_OOM;
    const int mx = MAX_DYN_SMEM;
#define MRP_FFT_KERNELS(K)                                                                           \
    (const void*)K<double, 0>, (const void*)K<float, 0>, (const void*)K<float, 1>, (const void*)K<float, 916>, \
        (const void*)K<float, 1414>, (const void*)K<float, 1827>
    const void* kernels[] = {MRP_FFT_KERNELS(k_fft_x_fwd), MRP_FFT_KERNELS(k_fft_y_fwd), (const void*)k_fft_z_conv<double, 0>,
                             (const void*)k_fft_z_conv<float, 0>, (const void*)k_fft_z_conv<float, 1>,
                             (const void*)k_fft_z_conv<float, 916>, (const void*)k_fft_z_conv<float, 1414>,
                             (const void*)k_fft_z_conv<float, 1827>,
                             MRP_FFT_KERNELS(k_fft_y_inv), MRP_FFT_KERNELS(k_fft_x_inv)};
#undef MRP_FFT_KERNELS
    for (const void* k : kernels) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    return MRP_OK;
}

}  // namespace mrp
