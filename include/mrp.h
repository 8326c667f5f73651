/*
 * mrp: free-space (unbounded) Poisson solver on a block-structured adaptive
 * forest, by an adaptive FAS multigrid V-cycle coupled to a zero-padded FFT
 * lattice-Green's-function convolution on the uniform level 0.
 *
 * Method: arXiv 2512.08555 -- Alg. 1 (adaptive V(nu1,nu2) FAS cycle),
 * Sec. 3.2 Eqs. cross_discr2 / mehrstellen_discr4 / mehrstellen_discr6
 * (compact stencils of order 2, 4, 6 and the RHS operator R^M),
 * Sec. 2.1 (ghosting with polynomial interpolation of order M+2 at
 * resolution jumps), Sec. 3.1 (injection, full weighting, trilinear
 * prolongation, Gauss-Seidel smoothing), Sec. 2.2 and 3.3 (the level-0
 * direct solve is the convolution with the lattice Green's function of the
 * multigrid operator).
 *
 * The problem solved is  nabla^2 u = f  (Eq. 1) with u -> 0 at infinity.
 *
 * Geometry.  Level 0 is a grid of nb0[0] x nb0[1] x nb0[2] cubic blocks of
 * n^3 nodes, spacing h0, lower corner origin.  A block at level k with block
 * coordinates (bx, by, bz) holds the nodes origin + (b*n + i) * h0/2^k,
 * i = 0..n-1 per axis (vertex-centred, half-open).  A forest is given by its
 * leaves; every leaf is (level, bx, by, bz).  Constraints (checked by
 * mrp_create, MRP_ERR_INVALID_FOREST otherwise): leaves tile the domain
 * without overlap; 2:1 balance across faces, edges and corners; level-0
 * blocks that touch the domain boundary are leaves (Sec. 3.3); n even,
 * 8 <= n <= 24.
 *
 * Field layout.  f and u are [leaf, in the order given to mrp_create][z][y][x]
 * with x fastest, n^3 doubles per leaf.
 *
 * Errors.  Every entry point returns an int status (MRP_OK = 0); no
 * exception or abort crosses this interface.  mrp_error_string maps a
 * status to a static string.
 *
 * Threading.  A handle is not thread-safe; use it from one host thread and
 * one stream at a time.
 */
#ifndef MRP_H
#define MRP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MRP_OK = 0,
    MRP_ERR_INVALID_ARG = 1,     /* null pointer, bad option value */
    MRP_ERR_INVALID_FOREST = 2,  /* forest violates a constraint listed above */
    MRP_ERR_CUDA = 3,            /* a CUDA runtime call failed */
    MRP_ERR_OOM = 4,             /* device allocation failed */
    MRP_ERR_NOT_CONVERGED = 5,   /* max_cycles reached before the tolerance */
    MRP_ERR_TIMEOUT = 6,         /* a bounded device wait ran out (reserved: no kernel of this
                                    library waits on a device flag; waits are stream order only) */
    MRP_ERR_NUMERICAL = 7,       /* NaN or Inf in the stop-rule norm */
    /* 8 is not used */
    MRP_ERR_UNSUPPORTED = 9,     /* option combination not built */
    MRP_ERR_TOO_LARGE = 10       /* problem exceeds a fixed-size scratch array */
};

enum { MRP_FP64 = 0, MRP_MIXED = 1 };
enum { MRP_STOP_RESIDUAL = 0, MRP_STOP_CAUCHY = 1 };
/* Flag of mrp_options.launch (see there). */
enum { MRP_LAUNCH_NOSTAGE = 4096 };

typedef struct {
    int32_t nb0[3];              /* level-0 blocks per axis (x, y, z) */
    int32_t n;                   /* nodes per block edge */
    double origin[3];            /* position of level-0 node (0,0,0) */
    double h0;                   /* level-0 node spacing */
    int32_t n_leaves;
    const int32_t* leaf_level;   /* host, [n_leaves] */
    const int32_t* leaf_ijk;     /* host, [n_leaves][3] block coords (x, y, z) at the leaf's level */
    int32_t ncomp;               /* right-hand sides sharing this forest (>= 1) */
} mrp_forest;

typedef struct {
    int32_t order;               /* M = 2, 4 or 6 */
    double tol;                  /* stop when the rule below falls under tol */
    int32_t stop_rule;           /* MRP_STOP_RESIDUAL: max|f* - L u| / max|f*| over leaf nodes
                                    (Sec. 3.1).
                                    MRP_STOP_CAUCHY: max|u^n - u^{n+1}| / max|u^{n+1}| over leaf
                                    nodes between successive iterates (Sec. 3, the criterion for
                                    problems whose residual stalls).  MRP_FP64: an iterate is the
                                    state after a V-cycle, u^0 = 0.  MRP_MIXED: an iterate is the
                                    state after a refinement step, u^0 = 0.  A zero iterate
                                    divides by 1.  Keeps one more FP64 copy of the leaf values
                                    (8 bytes per leaf node). */
    int32_t max_cycles;          /* >= 1 */
    int32_t nu1, nu2;            /* pre- and post-smoothing sweeps, >= 0 */
    int32_t precision;           /* MRP_FP64: every stage in FP64.
                                    MRP_MIXED: FP64 outer refinement (Green's function, outer
                                    residual, level-0 convolution of the accumulated source,
                                    correction accumulation) around FP32 V-cycles; tol then
                                    bounds the relative residual of the composite system.
                                    The first refinement step starts from u = 0, so its FP32
                                    cycles solve the problem itself (f* on every level's
                                    leaves); each step ends with an FP64 outer residual and
                                    the stop check, so at least one step runs */
    int32_t inner_cycles;        /* MRP_MIXED: FP32 V-cycles per refinement step (0 = 4) */
    int32_t max_outer;           /* MRP_MIXED: refinement steps at most (0 = 12) */
    int32_t launch;              /* 0: the CTA size of each stencil kernel and level is chosen by
                                    timing at the first solve.  Otherwise that size (128, 256 or
                                    512) for every kernel and level; 128 or 256 may carry
                                    MRP_LAUNCH_NOSTAGE, with which the Gauss-Seidel sweep and the
                                    FP32 residual of block size 16 read the right-hand side from
                                    global memory instead of staging it in shared memory.
                                    Results do not depend on this choice. */
} mrp_options;


typedef struct {
    int32_t cycles;              /* V-cycles run */
    int32_t ir_steps;            /* outer refinement steps (0 for MRP_FP64) */
    double residual;             /* final relative residual (stop rule RESIDUAL; MRP_MIXED also
                                    under CAUCHY, where the outer residual is computed anyway;
                                    0 when not computed) */
    double cauchy;               /* final relative increment (stop rule CAUCHY, else 0) */
    double fstar_max;            /* max |f*| over leaf nodes */
    int64_t leaf_nodes;          /* unknowns of the composite grid */
    int64_t total_nodes;         /* nodes over all levels */
    int64_t launches;            /* kernels launched by this call */
} mrp_stats;

typedef struct mrp_handle mrp_handle;

/* Build a solver for n_forests independent forests, each with ncomp
 * right-hand sides (a batch: every (forest, component) pair is one problem,
 * and one call solves them all; the caller layout of f and u is then
 * [forest][component][leaf][z][y][x]).  Forests may differ in every field;
 * those that share a block size n share pooled per-level block arrays, one
 * group per block size.  Validates each forest, builds per-level block
 * tables and the ghost plan, allocates every device workspace, tabulates the
 * lattice Green's function of the order-M operator in FP64 on the device
 * (Sec. 2.2, 3.3) and each problem's spectrum on its padded level-0 lattice.
 * Uses the current CUDA device.  On failure *out is NULL and nothing is
 * leaked. */
int mrp_create(mrp_handle** out, const mrp_forest* forests, int32_t n_forests, const mrp_options* opt);

/* Solve nabla^2 u = f from u = 0.  f, u: device pointers, layout above.
 * stream: a cudaStream_t (NULL = legacy default stream).  Allocates nothing;
 * synchronises the stream once per cycle to read the stop criterion.
 * st may be NULL.  Returns MRP_ERR_NOT_CONVERGED (u still written) when
 * max_cycles ran out. */
int mrp_solve(mrp_handle* h, const double* f, double* u, void* stream, mrp_stats* st);

/* The same solve as mrp_solve, run as one CUDA graph launch with no host
 * synchronisation inside: per block-size group, a prologue (f*, norms,
 * u = 0), a device-controlled WHILE loop over cycles (MRP_FP64) or
 * refinement steps (MRP_MIXED) whose last kernel compares every problem's
 * relative residual with tol and sets the loop condition, and the gather of
 * u; the groups' chains are independent branches of the graph and run
 * concurrently.  The graph is built (captured and instantiated) on the first
 * call and again whenever f or u differ from the previous call's: such a call
 * synchronises the stream first and allocates; other calls launch the graph
 * and synchronise the stream once at the end to read the statistics.  Same
 * results and status as mrp_solve (st->launches counts the kernels the
 * graph ran). */
int mrp_solve_graph(mrp_handle* h, const double* f, double* u, void* stream, mrp_stats* st);

/* The mrp_solve_graph solve end to end from host memory: copies f_host to a
 * device buffer the handle owns, launches the solve graph, copies the result
 * into u_host, all ordered on stream, and returns once u_host is written.
 * f_host, u_host: host pointers in the layout above (pinned memory, from
 * cudaHostAlloc or cudaHostRegister, lets the copies run asynchronously at
 * full bandwidth; pageable memory also works).  The caller keeps ownership.
 * The first call allocates the two device buffers (8 bytes per element of f
 * each) and builds the graph; later calls allocate nothing.  Same status and
 * statistics as mrp_solve_graph; u_host is written also under
 * MRP_ERR_NOT_CONVERGED and MRP_ERR_NUMERICAL. */
int mrp_solve_host(mrp_handle* h, const double* f_host, double* u_host, void* stream, mrp_stats* st);

/* Gradient of the converged solve: fbar = S^T w, where u = S f is the
 * composite solution mrp_solve converges to (the map is linear).  S
 * factors as f* = B f (Sec. 3.2 with f ghosts), 0 = c(f*) - K x (the
 * composite leaf system: L_k u = f* at leaves of levels >= 1, and on level-0
 * nodes covered by level 1 the level-0 field h0^2 G * f0 of Sec. 2.2 equal to
 * the injection of level 1) and u = E(x, f*); so fbar = B^T (E_f^T w +
 * c^T lambda) with K^T lambda = E_x^T w.  Every factor is the exact
 * transpose of the forward stage (ghost fill, injection, stencils, level-0
 * convolution).  K^T lambda = E_x^T w is solved in FP64 by refinement with the
 * transposed correction V-cycle (Gauss-Seidel colours reversed, full
 * weighting and trilinear correction exchanged, ghost fills turned into
 * scatters); it stops when max|E_x^T w - K^T lambda| / max|E_x^T w| < tol or
 * after max_cycles transposed cycles (MRP_ERR_NOT_CONVERGED, fbar still
 * written).  w, fbar: device pointers in the leaf layout of f and u.  Needs
 * no earlier mrp_solve (no forward state enters: every factor is linear and
 * independent of the forward iterates).  The first call allocates the
 * adjoint workspace (about 5 fields per level plus 6 vectors of total_nodes
 * doubles); later calls allocate nothing.  The refinement residual
 * E_x^T w - K^T lambda and the accumulation of lambda are FP64 on both
 * precision options; the transposed cycles M^T run in FP64 on an MRP_FP64
 * handle and in FP32 on an MRP_MIXED one.  The stop rule is always the
 * residual above (stop_rule is ignored).  st->cycles = st->ir_steps =
 * transposed cycles, st->residual = the final relative residual above. */
int mrp_solve_adjoint(mrp_handle* h, const double* w, double* fbar, void* stream, mrp_stats* st);

/* Release every resource of h (NULL is allowed). */
int mrp_destroy(mrp_handle* h);

const char* mrp_error_string(int status);

/* Per-phase device timing (CUDA events around every kernel launch of the
 * solve), off by default.  Phases: 0 ghosting, 1 smoothing, 2 residual,
 * 3 restriction + FAS RHS, 4 level-0 FFT solve, 5 prolongation,
 * 6 residual norms, 7 right-hand-side preparation and other; FP64 work at
 * these indices, FP32 work (inner cycles of MRP_MIXED) at index + 8.
 * mrp_profile_read copies n (<= 16) accumulated milliseconds, launch counts
 * and node-updates (nodes processed, summed over launches) to host arrays
 * (any may be NULL) and, if reset != 0, clears the accumulators. */
int mrp_profile_enable(mrp_handle* h, int32_t enable);
int mrp_profile_read(mrp_handle* h, int32_t n, double* ms, int64_t* launches, int64_t* nodes, int32_t reset);

#ifdef __cplusplus
}
#endif

#endif
