// Internal declarations shared by the translation units of libmrp.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <vector>
#include <string>
#include <memory>
#include <mutex>

#include "mrp.h"
#include "mrp_steps.h"

namespace mrp {

// 27 neighbour directions, index = (dz+1)*9 + (dy+1)*3 + (dx+1); 13 is the block itself.
__host__ __device__ inline int dir27(int dx, int dy, int dz) { return (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); }

// x / d for 0 <= x < 2^16 and 2 <= d < 2^16, with m = magic_of(d): the
// product x m = x (2^32 + e) / d with 0 <= e < d, so its high word is
// floor(x / d) while x e < 2^32.
#ifdef __CUDACC__
__device__ __forceinline__ unsigned magic_of(int d) { return 0xFFFFFFFFu / (unsigned)d + 1u; }
__device__ __forceinline__ int fdiv(int x, unsigned m) { return (int)__umulhi((unsigned)x, m); }

// (double)v for a float v without the conversion instruction, which runs on
// GB300's scarce FP64 pipe: a normal float's exponent is rebiased (+896 =
// 1023 - 127) and its 23-bit fraction moved to the top of the 52-bit one,
// which is exact; zeros, subnormals, Inf and NaN take the plain conversion.
__device__ __forceinline__ double widen_exact(float v) {
    const unsigned long long u = __float_as_uint(v);
    const unsigned e = (unsigned)(u >> 23) & 0xFFu;
    if (e - 1u < 254u)
        return __longlong_as_double((long long)(((u & 0x80000000ull) << 32) | ((unsigned long long)(e + 896u) << 52) |
                                                ((u & 0x7FFFFFull) << 29)));
    return (double)v;
}

// (float)d, rounded to nearest with ties to even, without the conversion
// instruction (it runs on GB300's scarce FP64 pipe): for results in the
// normal float range the 52-bit fraction is cut to 23 bits and rounded on the
// 29 bits dropped; a carry out of the fraction moves into the exponent, which
// is the correct rounding (up to +-Inf past the largest float).  Zeros,
// subnormal results, overflow before rounding, Inf and NaN take the plain
// conversion.
__device__ __forceinline__ float narrow_rn(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((u >> 52) & 0x7FF) - 896;         // float exponent field (1023 - 127 = 896)
    if (e >= 1 && e <= 254) {
        unsigned keep = (unsigned)((u >> 29) & 0x7FFFFFu);
        const unsigned rem = (unsigned)(u & 0x1FFFFFFFu), half = 0x10000000u;
        keep += (rem > half || (rem == half && (keep & 1u))) ? 1u : 0u;
        return __uint_as_float((((unsigned)(u >> 32)) & 0x80000000u) + ((unsigned)e << 23) + keep);
    }
    return (float)d;
}

// Fixed-point form of a double: trunc(u 2^(shb + 1075)) as a 64-bit integer,
// the 53-bit significand (hidden bit included; a subnormal's exponent field
// counts as 1) shifted by (exponent field + shb) and the sign applied.  The
// caller picks shb so that the left shifts stay small (box_to_fixed: at most
// 9 - G bits, for every value of the box whose largest exponent field fixed
// shb).
__device__ __forceinline__ long long to_fixed(long long bits, int shb) {
    const int e = (int)((bits >> 52) & 0x7FF);
    const unsigned long long m = ((unsigned long long)bits & 0xFFFFFFFFFFFFFULL) | (e ? (1ULL << 52) : 0ULL);
    const int sh = (e ? e : 1) + shb;
    const unsigned long long a = sh >= 0 ? m << sh : (sh > -64 ? m >> -sh : 0ULL);
    return bits < 0 ? -(long long)a : (long long)a;
}

// (double)v, rounded to nearest with ties to even, with integer operations:
// |v| is normalised so that its top bit is bit 63, the 53 bits from there are
// the significand (hidden bit included) and the 11 bits below decide the
// rounding; a carry out of the significand moves into the exponent.
__device__ __forceinline__ double i64_to_double_rn(long long v) {
    const unsigned long long sgn = (unsigned long long)v & 0x8000000000000000ULL;
    unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
    if (a == 0) return 0.0;
    const int lz = __clzll((long long)a);
    a <<= lz;
    unsigned long long keep = a >> 11;
    const unsigned rem = (unsigned)(a & 0x7FFu);
    keep += (rem > 0x400u || (rem == 0x400u && (keep & 1ULL))) ? 1ULL : 0ULL;
    return __longlong_as_double((long long)(sgn | ((((unsigned long long)(1085 - lz)) << 52) + keep)));
}

// Asynchronous global -> shared copies (cp.async): one element, or 16 bytes;
// a thread's copies complete at cp_async_wait<N>() (all but its N most recent
// committed groups), and are visible to the CTA after the next barrier.
template <typename T>
__device__ __forceinline__ void cp_async_el(T* sdst, const T* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    if constexpr (sizeof(T) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// Read-only global load issued where it stands (volatile: not moved past the
// copies and barriers that follow), for values prefetched into registers.
__device__ __forceinline__ float ldg_now(const float* p) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];\n" : "=f"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
#endif

// Runs fn once per device (the current one) for each distinct flags array,
// thread-safe: kernel attributes such as the opt-in shared-memory size are
// per device, and several host threads may create handles at once.
constexpr int MAX_DEVICES = 64;
template <typename Fn>
inline void once_per_device(std::once_flag (&flags)[MAX_DEVICES], Fn&& fn) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) { fn(); return; }
    std::call_once(flags[dev], fn);
}

// Codes stored in the neighbour table besides block indices.
constexpr int NBR_MISSING = -1;   // no block of this level there: interpolate from level k-1
constexpr int NBR_OUTSIDE = -2;   // outside the domain (level 0 only)

// Device view of one level's block tables (passed by value to kernels).
struct LevelView {
    int nb;
    const int* coords;     // [nb][3] x y z
    const int* nbr;        // [nb][27]
    const int* parent;     // [nb] block index at level k-1 (-1 at level 0)
    const int* octant;     // [nb] child octant o = ox + 2 oy + 4 oz inside the parent
    const int* children;   // [nb][8] (-1 for leaves)
    const uint8_t* is_leaf;
    const int* order;      // [nb] launch order: blocks with interpolated ghosts first
    const int* prob;       // [nb] problem of each block (per-problem norms of a batched handle)
    const int* rec;        // [nb][REC_INTS] neighbourhood records (below)
    int nint;              // blocks with interpolated ghost regions; they come first in `order`
};

// Per-block neighbourhood record, REC_INTS ints, which the fused stencil
// kernels copy to shared memory in 16-byte chunks: the same-level
// neighbours, the ghost regions to interpolate (offsets of their work
// arrays and the hull of their coarse stencils), the parent's neighbours and
// the children of each (everything the ghost layer needs besides values).
constexpr int REC_SNBR = 0;      // [27] same-level neighbour per direction (or NBR_*)
constexpr int REC_NREG = 27;     // number of interpolated regions (0: none)
constexpr int REC_PNBR = 28;     // [27] the parent's neighbours at level k-1
constexpr int REC_RDIR = 56;     // [26] direction of each interpolated region
constexpr int REC_ROFF = 82;     // [26] its offset in the normal-reduced array
constexpr int REC_RAOFF = 108;   // [26] its offset in the face array (faces only)
constexpr int REC_LO = 134;      // [3] coarse patch hull per axis: [lo, hi)
constexpr int REC_HI = 137;      // [3]
constexpr int REC_PCH = 140;     // [27][8] children of each parent neighbour (-1: leaf, or no block)
constexpr int REC_COFF = 356;    // [26] each region's first item in the tangential pass (faces n TN, edges n, corners 1)
constexpr int REC_DOFF = 382;    // [26] each region's first item in the second face pass (faces n^2, others 0)
constexpr int REC_NTOT = 408;    // [3] items of the normal reduction, the tangential pass and the second face pass
constexpr int REC_INTS = 412;    // a multiple of 4

// Host + device tables of one level, plus its FP64 fields.
struct Level {
    int nb = 0, nleaf = 0, ncov = 0;
    int nint = 0;                     // blocks with interpolated ghost regions (first in h_order)
    std::vector<int> h_coords, h_nbr, h_parent, h_octant, h_children, h_leaf_blocks, h_cov_blocks, h_order;
    std::vector<uint8_t> h_is_leaf;
    std::vector<int> h_prob, h_rec;
    int *coords = nullptr, *nbr = nullptr, *parent = nullptr, *octant = nullptr, *children = nullptr;
    int *leaf_blocks = nullptr, *cov_blocks = nullptr, *order = nullptr, *prob = nullptr, *rec = nullptr;
    uint8_t* is_leaf = nullptr;
    double *U = nullptr, *F = nullptr, *R = nullptr, *H = nullptr, *Fraw = nullptr;
    double* Ualt = nullptr;           // second u buffer: a sweep reads U and writes Ualt, then they swap
    double* Uprev = nullptr;          // [nb][n^3] leaf values of the previous iterate (Cauchy stop rule only)
    float *U32 = nullptr, *F32 = nullptr, *R32 = nullptr, *H32 = nullptr;   // mixed precision inner cycles
    float* U32alt = nullptr;
    LevelView view() const { return LevelView{nb, coords, nbr, parent, octant, children, is_leaf, order, prob, rec, nint}; }
};

// One padded FFT axis: length, radix sequence, twiddles exp(-2 pi i m / P).
struct FftAxis {
    int P = 0, K = 0;                 // K = P/2 + 1 (half spectrum along x)
    int nrad = 0, nrad32 = 0;
    int rad[16], rad32[16];           // radix sequences of the FP64 and FP32 lines
    double2* tw = nullptr;            // device [P]
    float2* tw32 = nullptr;           // device [P], FP32 copy
};

constexpr int MAX_RADIX_STAGES = 16;
// Opt-in dynamic shared memory per CTA requested for the large-tile kernels
// (below the 227 KB limit so that their small static arrays still fit).
constexpr int MAX_DYN_SMEM = 225 * 1024;   // dynamic shared memory per CTA (227 KB opt-in less static use)
// The block kernels come in two builds: block size 16 fixed at compile time
// (constant strides, offsets and divisions) and any block size at run time.
constexpr int NC_FIXED = 16;

// One problem of a handle: a forest, or one component of a forest's vector
// right-hand side.  Its blocks are contiguous in every level's pool; it has
// its own level-0 lattice and FFT.  All problems of a handle share the block
// size n, the order and one reference spacing h0: a problem of spacing h0_p
// enters with f scaled by (h0_p / h0)^2, which leaves u unchanged since the
// discrete operator at every level scales as 1/h^2 and the level-0 solve as h^2.
struct Problem {
    int forest = 0, comp = 0;
    int nb0[3] = {0, 0, 0}, n0[3] = {0, 0, 0};   // level-0 blocks and nodes per axis
    double h0 = 0.0, scale = 1.0;
    int L = 0;                        // finest level
    int base0 = 0;                    // first level-0 block
    int cov0_lo = 0, cov0_hi = 0;     // range in level 0's covered-block list
    int leaf0_lo = 0, leaf0_hi = 0;   // range in level 0's leaf-block list
    FftAxis ax[3];
    int gK[3] = {0, 0, 0};
    double* ghat = nullptr;           // [Kz][Ky][Kx] real spectrum of G, scaled by h0^2 / (Px Py Pz) (handle's h0)
    float* ghat32 = nullptr;          // FP32 copy
};

struct Handle {
    // forest: the problems' blocks pooled per level
    int n, L;                         // block size; finest level over all problems
    double h0;                        // reference level-0 spacing (problem 0's)
    std::vector<Problem> pr;
    int M, nu1, nu2, max_cycles, stop_rule;
    double tol;
    std::vector<Level> lv;
    int n_leaves;                     // leaves over all problems
    int* leaf_level = nullptr;        // device [n_leaves]
    int* leaf_block = nullptr;        // device [n_leaves]
    int64_t* leaf_src = nullptr;      // device [n_leaves] element offset of the leaf in the caller's f / u
    double* leaf_scale = nullptr;     // device [n_leaves] scale of the leaf's problem
    std::vector<int> h_leaf_level, h_leaf_block;
    std::vector<int64_t> h_leaf_src;
    std::vector<double> h_leaf_scale;
    // coarse solve (spectral buffers sized for the largest lattice; problems run one after another)
    double2* spec = nullptr;          // [Pz][Py][Kx]
    float2* spec32 = nullptr;         // FP32 spectral buffer
    // mixed precision
    bool mixed = false;
    int inner_cycles = 4, max_ir = 12;
    double* c0 = nullptr;             // [nb0 blocks][n^3] injection mismatch on covered level-0 nodes (FP64)
    float* off32 = nullptr;           // [nb0 blocks][n^3] -c0 in FP32 (offset of the level-1 -> 0 injection)
    int lgf_nmax = 0;
    double* lgf = nullptr;            // [(nmax+1)^3]
    // max-norm reductions: slot s of problem p at dmax[s * nprob + p] (s < 4)
    unsigned long long* dmax = nullptr;
    unsigned long long* hmax = nullptr;   // pinned host mirror
    int nprob() const { return (int)pr.size(); }
    unsigned long long* slot(int s) const { return dmax + (size_t)s * pr.size(); }
    int64_t leaf_nodes = 0, total_nodes = 0;
    std::vector<double> fstar;        // max |f*| per problem
    double fstar_max = 0.0;
    bool have_forward = false;
    // launch accounting and optional per-phase event timing
    int64_t launches = 0;
    bool prof = false;
    std::vector<cudaEvent_t> ev;          // pool, 2 events per timed phase
    int ev_used = 0;
    struct Pending { int phase, e0; int64_t nodes; };
    std::vector<Pending> pend;
    double prof_ms[16] = {};
    int64_t prof_cnt[16] = {}, prof_nodes[16] = {};
    // CTA sizes of the fused stencil kernels per precision (0 FP64, 1 FP32) and
    // level, chosen by timing at the first solve (autotune in solver.cu)
    static constexpr int MAXL = 32;
    int nt_smooth[2][MAXL], nt_res[2][MAXL], nt_fas[2][MAXL], nt_leafres[MAXL];
    bool tuned = false;
    int launch_override = 0;          // mrp_options.launch (0: autotune)
    // device-side loop control of the graph-captured solve (graph.cu)
    int* loop_ctr = nullptr;          // [4]: cycles, refinement steps, status, unused
    double* loop_rel = nullptr;       // [nprob] relative residuals
    int64_t gl_pro = 0, gl_body = 0, gl_epi = 0;   // kernels in the graph's prologue, loop body, epilogue
    // gradient of the converged solve (adjoint.cu), allocated at its first call
    struct AdjLevel { double *Ub = nullptr, *Fb = nullptr, *Rb = nullptr, *Hb = nullptr, *Rawb = nullptr; };
    std::vector<AdjLevel> adj;
    std::vector<size_t> xoff;         // level k's offset in the vectors below, which hold [nb_k][n^3] per level
    double *lam = nullptr, *rho = nullptr, *gvec = nullptr, *xb = nullptr, *fsb = nullptr, *wl = nullptr;
    double *cube = nullptr, *dense = nullptr, *off0b = nullptr;
    struct AdjLevel32 { float *Ub = nullptr, *Fb = nullptr, *Rb = nullptr, *Hb = nullptr; };
    std::vector<AdjLevel32> adj32;    // FP32 transposed cycles of a mixed-precision handle
    float *cube32 = nullptr, *dense32 = nullptr, *off0b32 = nullptr;
};

inline double level_h(const Handle& h, int k) { return h.h0 / (double)(1 << k); }
inline int64_t n3(const Handle& h) { return (int64_t)h.n * h.n * h.n; }
inline LevelView view_or_empty(const Handle& h, int k) {
    return k >= 0 ? h.lv[k].view()
                  : LevelView{0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0};
}

// Per-level base pointers, passed by value to the leaf scatter / gather kernels.
struct LevelPtrs { double* p[32]; };

enum Phase { PH_GHOST = 0, PH_SMOOTH = 1, PH_RESIDUAL = 2, PH_RESTRICT = 3, PH_COARSE = 4, PH_PROLONG = 5,
             PH_NORM = 6, PH_OTHER = 7 };
// Phases of FP32 work are counted separately, at index + 8.
template <typename T> constexpr int ph(int p) { return p + (sizeof(T) == 4 ? 8 : 0); }

// Phase names (NVTX ranges), index as in Phase, FP32 work at index + 8.
inline const char* phase_name(int p) {
    static const char* names[16] = {"ghost_f64", "smooth_f64", "residual_f64", "restrict_f64", "coarse_fft_f64",
                                    "prolong_f64", "norm_f64", "other_f64", "ghost_f32", "smooth_f32", "residual_f32",
                                    "restrict_f32", "coarse_fft_f32", "prolong_f32", "norm_f32", "other_f32"};
    return (p >= 0 && p < 16) ? names[p] : "phase";
}

// Per-phase accounting: counts launches; opens an NVTX range named for the
// phase around its launches (host side; a profiler attached to the process
// shows each phase's launches under it); with profiling on, records a CUDA
// event pair around the phase (harvested at the next host synchronisation).
struct PhaseScope {
    Handle& h;
    cudaStream_t s;
    int phase, e0 = -1, launches;
    int64_t nodes;
    PhaseScope(Handle& hh, cudaStream_t ss, int ph, int64_t nd, int nl) : h(hh), s(ss), phase(ph), launches(nl), nodes(nd) {
        nvtxRangePushA(phase_name(phase));
        if (h.prof && h.ev_used + 2 <= (int)h.ev.size()) {
            e0 = h.ev_used;
            h.ev_used += 2;
            cudaEventRecord(h.ev[e0], s);
        }
    }
    ~PhaseScope() {
        nvtxRangePop();
        h.launches += launches;
        if (e0 >= 0) {
            cudaEventRecord(h.ev[e0 + 1], s);
            h.pend.push_back(Handle::Pending{phase, e0, nodes});
        }
    }
};
void harvest(Handle& h);
// Copies the per-problem max-norms of slot `slot` to out[0 .. nprob); synchronises s.
int read_max(Handle& h, cudaStream_t s, double* out, int slot);

// ---------------------------------------------------------------- host side
// One problem to build: forest, component, and the caller-layout element
// offset of its first leaf.
struct ProblemDesc { const mrp_forest* f; int forest, comp; int64_t src_off; };
int build_forest(Handle& h, const std::vector<ProblemDesc>& list, std::string& why);
int upload_tables(Handle& h);
int lgf_build(Handle& h, cudaStream_t s);   // tabulate G and the scaled spectrum
int fft_plan(Handle& h);
// pieces of a solve (solver.cu), also captured into the solve graph (graph.cu)
template <typename T> void vcycle(Handle& h, cudaStream_t s);
void solve_begin(Handle& h, const double* f, cudaStream_t s);
void leaf_residual_launch(Handle& h, cudaStream_t s);
void cauchy_launch(Handle& h, cudaStream_t s);   // Cauchy stop rule into slots 2 (num) and 3 (den)
void outer_residual_launch(Handle& h, cudaStream_t s);
void first_step_launch(Handle& h, cudaStream_t s);   // mixed precision: FP32 cycles on the problem itself, from u = 0
void correction_launch(Handle& h, cudaStream_t s);
void solve_end(Handle& h, double* u, cudaStream_t s);
int autotune(Handle& h, cudaStream_t s);
// gradient of the converged solve (adjoint.cu)
int adjoint_setup(Handle& h);
void adjoint_release(Handle& h);
int solve_adjoint(Handle& h, const double* w, double* fbar, cudaStream_t s, int* cycles_out, double* rel_out);
int adjoint_op(Handle& h, int op, const double* in, double* out, cudaStream_t s);
}  // namespace mrp
struct mrp_handle;
namespace mrp {
// the solve graph (graph.cu)
void graph_release(mrp_handle* H);

// ---------------------------------------------------------------- launches (kernels_*.cu)
// Templated launchers are instantiated for double (FP64 path, outer refinement)
// and float (inner cycles of the mixed-precision path).
template <typename T>
void launch_inject_to_parent(T* coarse, int gc, const T* fine, int gf, LevelView fine_lv, int n, const T* off, cudaStream_t s);
template <typename T>
void launch_restrict(T* Uc, T* Fc, const T* Uf, const T* Rf, LevelView lf, int n, const T* off, cudaStream_t s);
template <typename T>
void launch_prolong(T* Uf, const T* Uc, const T* Hc, LevelView lf, LevelView lc, int n, cudaStream_t s);
template <typename T>
void launch_coarse_solve_t(const Handle& h, const T* F0, T* U0, cudaStream_t s);
// stencil kernels with the ghost layer built in shared memory (kernels_fused.cuh, fused_*.cu);
// Smoother and residual launch choice (the `nt` argument of
// launch_smooth_fused and launch_residual_fused): the CTA size in the low
// bits; SMOOTH_NOSTAGE reads the right-hand side from global memory where it
// is used instead of staging it in shared memory (less shared memory per
// CTA, so more CTAs per SM; the FP32 residual also writes R there).
constexpr int SMOOTH_NT_MASK = 0xFFF, SMOOTH_NOSTAGE = 1 << 12;
// fused_smem_bytes: their dynamic shared memory for block size n, order M and
// element size el (bytes), without a staged right-hand side
size_t fused_smem_bytes(int n, int M, int el);
template <typename T>
void launch_smooth_fused(T* Uout, const T* Uin, const T* F, const T* Uc, LevelView lk, LevelView lc, int n, int M,
                         double h2, int nt, cudaStream_t s);
template <typename T>
void launch_residual_fused(T* R, const T* U, const T* F, const T* Uc, LevelView lk, LevelView lc, int n, int M,
                           double inv_h2, int nt, cudaStream_t s);
template <typename T>
void launch_fas_fused(T* F, T* H, const T* U, const T* Uc, LevelView lk, LevelView lc, int n, int M, double inv_h2,
                      int nt, cudaStream_t s);
template <typename T>
void launch_halo_dump(T* U, const T* Uc, LevelView lk, LevelView lc, int n, int M, cudaStream_t s);
void launch_leafres_fused(float* R, const double* U, const double* F, const double* Uc, const int* blocks, int nblocks,
                          LevelView lk, LevelView lc, int n, int M, double inv_h2, unsigned long long* out, int nt,
                          cudaStream_t s);

void launch_ghost_fill(double* A, int g, const double* Ac, int gc, LevelView lk, LevelView lkm1, int n, int M,
                       bool zero_outside, cudaStream_t s);
void launch_scatter_leaves(Handle& h, const double* f, cudaStream_t s);
void launch_gather_leaves(Handle& h, double* u, cudaStream_t s);
void launch_rhs_star(double* F, const double* Fraw, const int* leaf_blocks, int nleaf, int n, int M, cudaStream_t s);
// f* = R^M f (M = 2, 4) on the listed leaf blocks of level k, the one ghost layer built in the kernel from raw f
// in the (n+2)^3 box layout (Af: level k; Ac: level k-1, covered nodes injected); max |f*| per problem into
// fmax_out[prob] (atomic max on the bit pattern, NaN as +Inf)
void launch_rhs_fused(double* F, const double* Af, const double* Ac, const int* blocks, int nblocks, LevelView lk, int n,
                      int M, unsigned long long* fmax_out, cudaStream_t s);
void launch_absmax(const double* F, const int* blocks, int nblocks, int n, unsigned long long* out, const int* prob,
                   cudaStream_t s);
void launch_coarse_solve_ext(const Handle& h, double2* spec, const double* F0, double* U0, cudaStream_t s);
template <typename T>
void launch_conv_transpose(const Handle& h, const Problem& p, const T* cube_in, T* src_out, cudaStream_t s);
void launch_scatter_leaves_to(const Handle& h, const double* f, const LevelPtrs& dst, int g, bool scaled, cudaStream_t s);
void launch_gather_leaves_from(const Handle& h, double* u, const LevelPtrs& src, int g, bool scaled, cudaStream_t s);
// transposed operators (kernels_adjoint.cu); T = double, or float for the FP32 transposed cycles
template <typename T>
void launch_stencil_T(T* out, const T* lam, T* fadd, const int* blocks, int nblocks, int n, int M, double inv_h2,
                      cudaStream_t s);
void launch_rstencil_T(double* out, const double* fsb, const int* blocks, int nblocks, int n, int M, cudaStream_t s);
void launch_ghost_T(double* A, int g, double* Ac, int gc, LevelView lk, LevelView lc, int n, int M, cudaStream_t s);
template <typename T>
void launch_ghost_T_fused(T* A, T* Ac, LevelView lk, LevelView lc, int n, int M, cudaStream_t s);
template <typename T>
void launch_inject_T(T* fine, int gf, T* coarse, int gc, LevelView lf, int n, cudaStream_t s);
template <typename T>
void launch_smooth_T(T* U, T* F, int nb, int n, int M, double h2, cudaStream_t s);
template <typename T>
void launch_prolong_T(T* Uc, T* Hc, const T* Uf, LevelView lf, LevelView lc, int n, cudaStream_t s);
template <typename T>
void launch_fw_T(T* Rf, const T* Fc, LevelView lf, int n, cudaStream_t s);
template <typename T>
void launch_window_T(T* cube, const T* U0, int n, const int* nb0, cudaStream_t s);
template <typename T>
void launch_dense_to_blocks(T* out, const T* dense, const int* blocks, int nblocks, const int* coords, int n, const int* n0,
                            bool add, cudaStream_t s);
template <typename TO, typename TI>
void launch_interior_get(TO* out, const TI* A, int g, const int* blocks, int nblocks, int n, double scale, cudaStream_t s);
template <typename TA, typename TV>
void launch_interior_add(TA* A, int g, const TV* v, const int* blocks, int nblocks, int n, double scale, cudaStream_t s);
template <typename TO, typename TI>
void launch_block_copy(TO* out, const TI* in, const int* blocks, int nblocks, int n, double scale, cudaStream_t s);
template <typename T>
void launch_block_zero(T* out, const int* blocks, int nblocks, int n, cudaStream_t s);
void launch_lincomb(double* out, double a, const double* x, double b, const double* y, size_t len,
                    unsigned long long* absmax, cudaStream_t s);
// mixed precision helpers (kernels_mixed.cu)
void launch_c0(double* c0, float* off32, const double* U0, const double* U1, const int* cov0, int ncov0, const int* children0,
               int n, double inv_h2, unsigned long long* out, const int* prob, cudaStream_t s);
void launch_cast_rhs(float* F32, const double* R64, const int* leaf_blocks, int nleaf, int n, bool zero, cudaStream_t s);
void launch_accumulate_u(double* U64, const float* U32, int nb, int n, cudaStream_t s);
void launch_accumulate_f(double* F64, const float* F32, const int* blocks, int nblocks, int n, cudaStream_t s);
// Cauchy stop rule: max |u - u_prev| and max |u| over leaf interiors per problem; u_prev = u
void launch_cauchy(double* Uprev, const double* U, const int* leaf_blocks, int nleaf, int n, unsigned long long* num,
                   unsigned long long* den, const int* prob, cudaStream_t s);
}  // namespace mrp

// Opaque handle of the C ABI: one internal handle per block size; the
// problems of one block size share its pooled levels.
struct mrp_handle {
    std::vector<std::unique_ptr<mrp::Handle>> g;
    std::vector<cudaStream_t> gs;     // one stream per group when there are several
    std::vector<cudaEvent_t> ev;      // fork event, then one join event per group
    int64_t elems = 0;                // doubles of f (and u): every forest, component and leaf
    // the whole solve as one CUDA graph (mrp_solve_graph), built for one (f, u) pair
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t cap = nullptr;       // capture stream
    const double* gf = nullptr;
    double* gu = nullptr;
    // device copies of f and u for mrp_solve_host, allocated at its first call
    double* host_f = nullptr;
    double* host_u = nullptr;
};
