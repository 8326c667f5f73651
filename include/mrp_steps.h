/*
 * Step-level entry points of mrp: run one stage of the solve on the
 * handle's internal per-level fields, and copy those fields in and out.
 * They exist so that each kernel of the path can be compared with a CPU
 * implementation of the same stage; mrp_solve is the composition of these
 * stages (Alg. 1 of arXiv 2512.08555).
 *
 * Internal layout (FP64).  Level k holds nb_k blocks (leaves of level k and
 * parents of level-(k+1) blocks), ordered by block coordinates with z
 * slowest, then y, then x.  Per block:
 *   MRP_FIELD_U     (n+2)^3   u with one ghost layer
 *   MRP_FIELD_F     n^3       right-hand side (f* on leaves, FAS RHS on covered blocks)
 *   MRP_FIELD_R     n^3       residual f - L u
 *   MRP_FIELD_UHAT  n^3       stored approximation u-hat (Alg. 1)
 *   MRP_FIELD_FRAW  (n+4)^3   raw source f with two ghost layers (order 6 only; other
 *                             orders keep raw f in the U arrays during
 *                             MRP_STEP_PREPARE_RHS and return MRP_ERR_UNSUPPORTED)
 * All arrays are [block][z][y][x], x fastest.
 */
#ifndef MRP_STEPS_H
#define MRP_STEPS_H

#include <stdint.h>
#include "mrp.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MRP_FIELD_U = 0, MRP_FIELD_F = 1, MRP_FIELD_R = 2, MRP_FIELD_UHAT = 3, MRP_FIELD_FRAW = 4
};

enum {
    MRP_STEP_PREPARE_RHS = 0,  /* f (leaf layout, arg) -> raw f on every level (FRAW with two ghost layers for
                                  M = 6; for M = 2, 4 the interiors of U, which it overwrites, with zero ghost
                                  layers) -> F = R^M f on leaves (Sec. 3.2) */
    MRP_STEP_GHOST_U = 1,      /* level k: inject U_k into covered U_{k-1}, then write into U_k's stored
                                  ghost layer the ghosts the stencil kernels build (Sec. 2.1) */
    MRP_STEP_SMOOTH = 2,       /* level k: one 8-colour Gauss-Seidel sweep with the ghost layer built from
                                  the current neighbours and frozen during the sweep (Sec. 3.1); the
                                  stored ghost layer of U_k is not updated */
    MRP_STEP_RESIDUAL = 3,     /* level k: R = F - L U on every node, ghosts built in the kernel (Alg. 1) */
    MRP_STEP_RESTRICT = 4,     /* level k -> k-1: injection of u, full weighting of r, FAS RHS on covered
                                  blocks (ghosts of U_{k-1} built in the kernel), u-hat (Alg. 1) */
    MRP_STEP_COARSE_SOLVE = 5, /* level 0: U = h0^2 G * F on all nodes and the exterior ring (Sec. 2.2) */
    MRP_STEP_PROLONG = 6,      /* level k: U_k += trilinear(U_{k-1} - UHAT_{k-1}) (Alg. 1) */
    MRP_STEP_VCYCLE = 7,       /* one full V(nu1,nu2) cycle (level argument ignored) */
    MRP_STEP_COARSE_SOLVE_F32 = 8  /* level 0 of a mixed-precision handle: the FP32 level-0 solve of its
                                      correction cycles (Sec. 2.2 in FP32): F rounded to FP32, the FP32
                                      zero-padded convolution, and its result widened into U (interiors
                                      and exterior ring); MRP_ERR_UNSUPPORTED on an FP64 handle */
};

/* Number of levels (max leaf level + 1). */
int mrp_level_count(mrp_handle* h, int32_t* levels);

/* Blocks of level k; coords ([nb][3], x y z) and is_leaf ([nb]) are host
 * buffers and may be NULL. */
int mrp_level_info(mrp_handle* h, int32_t level, int32_t* nb, int32_t* coords, uint8_t* is_leaf);

/* Copy a whole per-level field between the handle and a device buffer
 * (to_handle = 1: buf -> handle; 0: handle -> buf).  buf holds the internal
 * layout above.  Ordered on stream. */
int mrp_field_copy(mrp_handle* h, int32_t field, int32_t level, double* buf, int32_t to_handle, void* stream);

/* Run one step.  f_leaf is used by MRP_STEP_PREPARE_RHS only (device,
 * leaf layout of mrp_solve). */
int mrp_step(mrp_handle* h, int32_t step, int32_t level, const double* f_leaf, void* stream);

/* Copy the tabulated lattice Green's function G[n1][n2][n3],
 * 0 <= n_i <= nmax, to a host buffer of (nmax+1)^3 doubles; nmax must not
 * exceed the handle's table (returned by mrp_lgf_extent). */
int mrp_lgf_extent(mrp_handle* h, int32_t* nmax);
int mrp_lgf_copy(mrp_handle* h, int32_t nmax, double* out_host);

/* Padded FFT lattice of level 0 (per axis, x y z). */
int mrp_fft_shape(mrp_handle* h, int32_t* P);

/* The level-0 solve of MRP_STEP_COARSE_SOLVE, for callers that cannot
 * allocate device memory when they call it (while capturing a stream into a
 * CUDA graph, inside a host whose own pool owns all device memory, in loops
 * that must not synchronise).  The paper has no counterpart: this is a
 * deployment variant of the same computation.
 *
 * f0: device, level-0 source in the internal F layout ([block][z][y][x],
 * n^3 doubles per level-0 block); u0: device, level-0 result in the internal
 * U layout ((n+2)^3 per block, interior and ghost layer including the
 * exterior ring).  Both are the caller's.  The handle supplies only
 * read-only tables (Green's-function spectrum, twiddles).
 *
 * Scratch: a fixed 48 MiB device array inside the library (every GPU that
 * loads the library holds it until exit); it fits level-0 lattices with
 * Pz * Py * (Px/2 + 1) <= 3,145,728 complex values (e.g. P = 162 per axis);
 * larger ones return MRP_ERR_TOO_LARGE.  Nothing is allocated or freed.
 * The first call on a device looks the array's address up (a runtime call
 * that is not a stream operation): make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's
 * contents; every entry a call reads was written earlier in the same call,
 * so nothing needs clearing.  Calls whose GPU work overlaps (other streams,
 * other threads, other handles) race on the array: serialise them.
 * Returns MRP_ERR_CUDA if a launch error is pending after the launches; the
 * error is left pending (not cleared), so the caller still sees an error
 * its own earlier work may have left. */
int mrp_coarse_solve_noalloc(mrp_handle* h, const double* f0, double* u0, void* stream);

/* The factors of mrp_solve_adjoint one at a time (for parity checks).
 * Vectors of the unknown / residual space have *len = total_nodes doubles:
 * [nb_k][n^3] per level k = 0..L in level order, blocks in the order of
 * mrp_level_info; levels >= 1 carry values on their leaf blocks, level 0 on
 * its covered blocks, and every other entry must be zero (outputs keep them
 * zero).  in / out: device.  Allocates the adjoint workspace on first use;
 * synchronises the stream.
 *   MRP_ADJ_CYCLE_T  in: x-space vector -> out: M^T in (residual space), M the
 *                    correction V-cycle of Alg. 1 from u = 0 (leaf rows drive
 *                    the leaf blocks, covered level-0 rows the offset of the
 *                    injection into level 0); reads the handle's nu1, nu2
 *   MRP_ADJ_RES_T    in: lambda -> out[0, len): x-bar of res^T lambda,
 *                    out[len, 2 len): f*-bar (leaf blocks of every level)
 *   MRP_ADJ_OUT_T    in: w (leaf layout) -> out[0, len): E_x^T w,
 *                    out[len, 2 len): E_f^T w
 *   MRP_ADJ_RHS_T    in: f*-bar (len, leaf blocks) -> out: B^T f*-bar (leaf layout) */
/* Measured FMA throughput of the current device in TFLOP/s (2 flops per
 * FMA): precision MRP_FP64 times FP64 FMAs, MRP_MIXED FP32 FMAs.  Every
 * thread of a grid of 8 CTAs per SM runs 8 independent FMA chains; the best
 * of 3 launches timed with CUDA events on stream counts.  It is the
 * measured denominator of the FP64 stencil kernels' roofline (their flops
 * per byte lie far above this GPU's FP64 ridge).  Allocates and frees a few
 * bytes; synchronises the stream.  The paper has no counterpart (a
 * measurement aid). */
int mrp_fma_peak(int32_t precision, double* tflops, void* stream);

/* The two float/double conversions of the mixed-precision path, for their
 * tests: f_out[i] = d_in[i] rounded to float (nearest, ties to even) as the
 * FP64 leaf residual writes the FP32 right-hand side, and d_out[i] = f_in[i]
 * widened to double as the FP32 corrections are added to u.  Both are done
 * with integer operations where the result is a normal number (GB300's FP64
 * pipe is the scarce unit) and must equal the IEEE conversions bit for bit.
 * Device buffers of n elements (any may be NULL when n == 0), ordered on
 * stream.  The paper has no counterpart (an implementation detail). */
int mrp_convert_check(const double* d_in, float* f_out, const float* f_in, double* d_out, int64_t n, void* stream);

/* The two conversions of the FP64 leaf residual's fixed-point stencil sum,
 * for their tests: fx_out[i] = trunc(u_in[i] 2^(shb + 1075)) as a 64-bit
 * integer (the caller keeps it below 2^62 in magnitude: shb + the exponent
 * field of every u_in[i] <= 9), and d_out[i] = i_in[i] rounded to double
 * (nearest, ties to even).  Both use integer operations only; the second
 * must equal the IEEE conversion bit for bit.  Device buffers of n elements
 * (any may be NULL when n == 0), ordered on stream.  Returns
 * MRP_ERR_INVALID_ARG for n < 0, a NULL buffer with n > 0, or shb > 0.  The
 * paper has no counterpart (an implementation detail). */
int mrp_fixed_check(const double* u_in, int32_t shb, int64_t* fx_out, const int64_t* i_in, double* d_out, int64_t n,
                    void* stream);

enum { MRP_ADJ_CYCLE_T = 0, MRP_ADJ_RES_T = 1, MRP_ADJ_OUT_T = 2, MRP_ADJ_RHS_T = 3 };
int mrp_adjoint_len(mrp_handle* h, int64_t* len);
int mrp_adjoint_op(mrp_handle* h, int32_t op, const double* in, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif
