// Kernels of the FP64 iterative-refinement loop around FP32 V-cycles, and of
// the Cauchy stop rule.
//
// The FP64 state is u at every node of levels >= 1 and the level-0 source f0
// (f* on level-0 leaves, the unknown source s on level-0 nodes covered by
// level 1); the level-0 field is always the FP64 free-space convolution of
// f0.  The outer residual of the composite system has two parts: the leaf
// equations f* - L_k u of levels >= 1, and c0 = u0(X) - u1(2X) on covered
// level-0 nodes (the injection the converged multigrid state satisfies).
#include "mrp_internal.h"

#include <algorithm>

namespace mrp {

template <int M> struct LhsW64;
template <> struct LhsW64<2> { static constexpr double den = 1, c = -6, f = 1, e = 0, k = 0; };
template <> struct LhsW64<4> { static constexpr double den = 6, c = -24, f = 2, e = 1, k = 0; };
template <> struct LhsW64<6> { static constexpr double den = 30, c = -128, f = 14, e = 3, k = 1; };

template <int M>
__device__ __forceinline__ double lhs64(const double* __restrict__ a, int o, int S, int S2) {
    using W = LhsW64<M>;
    double acc = W::c * a[o];
    acc += W::f * ((a[o - 1] + a[o + 1]) + (a[o - S] + a[o + S]) + (a[o - S2] + a[o + S2]));
    if (W::e != 0)
        acc += W::e * ((a[o - 1 - S] + a[o + 1 - S]) + (a[o - 1 + S] + a[o + 1 + S])
                       + (a[o - 1 - S2] + a[o + 1 - S2]) + (a[o - 1 + S2] + a[o + 1 + S2])
                       + (a[o - S - S2] + a[o + S - S2]) + (a[o - S + S2] + a[o + S + S2]));
    if (W::k != 0)
        acc += W::k * ((a[o - 1 - S - S2] + a[o + 1 - S - S2]) + (a[o - 1 + S - S2] + a[o + 1 + S - S2])
                       + (a[o - 1 - S + S2] + a[o + 1 - S + S2]) + (a[o - 1 + S + S2] + a[o + 1 + S + S2]));
    return acc;
}

__device__ __forceinline__ void block_max_atomic64(double v, unsigned long long* out) {
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

// c0 = u0(X) - u1(2X) on covered level-0 blocks; off32 = -c0 (FP32); max |c0| / h0^2
// into out[prob[P]] (out[0] without a problem table).
__global__ void k_c0(double* __restrict__ c0, float* __restrict__ off32, const double* __restrict__ U0,
                     const double* __restrict__ U1, const int* __restrict__ cov0, const int* __restrict__ children0, int n,
                     double inv_h2, unsigned long long* out, const int* __restrict__ prob) {
    const int P = cov0[blockIdx.x];
    const int S = n + 2, S3 = S * S * S, n3 = n * n * n, h = n >> 1;
    double m = 0.0;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) {
        const int i = t % n, j = (t / n) % n, l = t / (n * n);
        const int ox = i >= h, oy = j >= h, oz = l >= h;
        const int c = children0[8 * P + ox + 2 * oy + 4 * oz];
        const int fx = 2 * i - ox * n, fy = 2 * j - oy * n, fz = 2 * l - oz * n;
        const double v = U0[(size_t)P * S3 + ((l + 1) * S + j + 1) * S + i + 1]
                       - U1[(size_t)c * S3 + ((fz + 1) * S + fy + 1) * S + fx + 1];
        c0[(size_t)P * n3 + t] = v;
        off32[(size_t)P * n3 + t] = (float)(-v);
        const double a = fabs(v) * inv_h2;
        m = (v != v) ? __longlong_as_double(0x7ff0000000000000ULL) : fmax(m, a);
    }
    block_max_atomic64(m, out + (prob ? prob[P] : 0));
}

void launch_c0(double* c0, float* off32, const double* U0, const double* U1, const int* cov0, int ncov0, const int* children0,
               int n, double inv_h2, unsigned long long* out, const int* prob, cudaStream_t s) {
    if (ncov0 == 0) return;
    k_c0<<<ncov0, 256, 0, s>>>(c0, off32, U0, U1, cov0, children0, n, inv_h2, out, prob);
}

// FP32 right-hand side of the correction cycles: the FP64 leaf residual (or 0).
__global__ void k_cast_rhs(float* __restrict__ F32, const double* __restrict__ R64, const int* __restrict__ blocks, int n,
                           bool zero) {
    const int b = blocks[blockIdx.x];
    const int n3 = n * n * n;
    for (int t = threadIdx.x; t < n3; t += blockDim.x)
        F32[(size_t)b * n3 + t] = zero ? 0.0f : (float)R64[(size_t)b * n3 + t];
}

void launch_cast_rhs(float* F32, const double* R64, const int* leaf_blocks, int nleaf, int n, bool zero, cudaStream_t s) {
    if (nleaf == 0) return;
    k_cast_rhs<<<nleaf, 256, 0, s>>>(F32, R64, leaf_blocks, n, zero);
}


// U64 += U32 on the interior of every block of a level.
__global__ void k_accumulate_u(double* __restrict__ U64, const float* __restrict__ U32, int n) {
    const int b = blockIdx.x;
    const int S = n + 2, S2 = S * S, S3 = S2 * S, nn = n * n, n3 = nn * n;
    const unsigned mnn = magic_of(nn), mn = magic_of(n);
    const size_t base = (size_t)b * S3 + S2 + S + 1;     // interior node (0, 0, 0)
    // K nodes per thread and round, all loads issued before the stores (the
    // stores could alias later loads as far as the compiler knows)
    constexpr int K = 4;
    for (int t0 = threadIdx.x; t0 < n3; t0 += K * blockDim.x) {
        double u[K];
        float v[K];
        size_t o[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int t = t0 + k * blockDim.x;
            const int z = fdiv(t, mnn), r = t - z * nn, y = fdiv(r, mn), x = r - y * n;
            o[k] = base + (size_t)z * S2 + y * S + x;
            if (t < n3) {
                u[k] = U64[o[k]];
                v[k] = U32[o[k]];
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (t0 + k * blockDim.x < n3) U64[o[k]] = u[k] + widen_exact(v[k]);
    }
}

void launch_accumulate_u(double* U64, const float* U32, int nb, int n, cudaStream_t s) {
    if (nb == 0) return;
    k_accumulate_u<<<nb, 256, 0, s>>>(U64, U32, n);
}

// F64 += F32 on the given blocks (level-0 source on covered nodes).
__global__ void k_accumulate_f(double* __restrict__ F64, const float* __restrict__ F32, const int* __restrict__ blocks, int n) {
    const int b = blocks[blockIdx.x];
    const int n3 = n * n * n;
    for (int t = threadIdx.x; t < n3; t += blockDim.x) F64[(size_t)b * n3 + t] += widen_exact(F32[(size_t)b * n3 + t]);
}

void launch_accumulate_f(double* F64, const float* F32, const int* blocks, int nblocks, int n, cudaStream_t s) {
    if (nblocks == 0) return;
    k_accumulate_f<<<nblocks, 256, 0, s>>>(F64, F32, blocks, n);
}

// Cauchy stop rule (Sec. 3): over the interiors of the given leaf blocks,
// max |u - u_prev| into num[prob] and max |u| into den[prob]; then u_prev = u.
__global__ void k_cauchy(double* __restrict__ Uprev, const double* __restrict__ U, const int* __restrict__ blocks, int n,
                         unsigned long long* num, unsigned long long* den, const int* __restrict__ prob) {
    const int b = blocks[blockIdx.x];
    const int S = n + 2, S2 = S * S, S3 = S2 * S, n3 = n * n * n;
    double md = 0.0, mu = 0.0;
    for (int c = threadIdx.x; c < n * n; c += blockDim.x) {       // one thread per (x, y) column
        const int y = c / n, x = c - y * n;
        const size_t o = (size_t)b * S3 + (size_t)((y + 1) * S + x + 1);
        for (int z = 0; z < n; ++z) {
            const double u = U[o + (size_t)(z + 1) * S2];
            const size_t q = (size_t)b * n3 + (size_t)z * n * n + c;
            const double d = fabs(u - Uprev[q]);
            Uprev[q] = u;
            md = (d != d) ? __longlong_as_double(0x7ff0000000000000ULL) : fmax(md, d);
            mu = (u != u) ? __longlong_as_double(0x7ff0000000000000ULL) : fmax(mu, fabs(u));
        }
    }
    const int p = prob ? prob[b] : 0;
    block_max_atomic64(md, num + p);
    __syncthreads();                 // the reduction's shared scratch is reused
    block_max_atomic64(mu, den + p);
}

void launch_cauchy(double* Uprev, const double* U, const int* leaf_blocks, int nleaf, int n, unsigned long long* num,
                   unsigned long long* den, const int* prob, cudaStream_t s) {
    if (nleaf == 0) return;
    k_cauchy<<<nleaf, 256, 0, s>>>(Uprev, U, leaf_blocks, n, num, den, prob);
}

}  // namespace mrp

namespace mrp {
__global__ void k_convert_check(const double* __restrict__ d_in, float* __restrict__ f_out, const float* __restrict__ f_in,
                                double* __restrict__ d_out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        f_out[i] = narrow_rn(d_in[i]);
        d_out[i] = widen_exact(f_in[i]);
    }
}
}  // namespace mrp

namespace mrp {
__global__ void k_fixed_check(const double* __restrict__ u_in, int shb, long long* __restrict__ fx_out,
                              const long long* __restrict__ i_in, double* __restrict__ d_out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        fx_out[i] = to_fixed(__double_as_longlong(u_in[i]), shb);
        d_out[i] = i64_to_double_rn(i_in[i]);
    }
}
}  // namespace mrp

extern "C" int mrp_fixed_check(const double* u_in, int32_t shb, int64_t* fx_out, const int64_t* i_in, double* d_out,
                               int64_t n, void* stream) {
    if (n < 0 || shb > 0 || (n > 0 && (!u_in || !fx_out || !i_in || !d_out))) return MRP_ERR_INVALID_ARG;
    if (n == 0) return MRP_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    mrp::k_fixed_check<<<grid, 256, 0, (cudaStream_t)stream>>>(u_in, shb, reinterpret_cast<long long*>(fx_out),
                                                              reinterpret_cast<const long long*>(i_in), d_out,
                                                              (long long)n);
    return cudaGetLastError() == cudaSuccess ? MRP_OK : MRP_ERR_CUDA;
}

extern "C" int mrp_convert_check(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n,
                                 void* stream) {
    if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out))) return MRP_ERR_INVALID_ARG;
    if (n == 0) return MRP_OK;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 4096);
    mrp::k_convert_check<<<grid, 256, 0, (cudaStream_t)stream>>>(d_in, f_out, f_in, d_out, (long long)n);
    return cudaGetLastError() == cudaSuccess ? MRP_OK : MRP_ERR_CUDA;
}
