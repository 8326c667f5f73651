// The whole solve as one CUDA graph: one launch runs every problem of the
// handle to convergence with no host synchronisation.
//
// Per block-size group the graph holds a chain
//     prologue:  right-hand side f*, its per-problem norms, u = 0
//                (mixed precision: also the first refinement step, FP32
//                cycles on the problem itself, its FP64 outer residual and a
//                check, which may skip the loop)
//     WHILE loop (conditional node): one V-cycle (FP64), or one refinement
//                step (FP32 correction cycles + FP64 accumulation + FP64 outer
//                residual), then a check kernel that compares every
//                problem's relative residual with tol, counts cycles and sets
//                the loop condition (cudaGraphSetConditional)
//     epilogue:  leaf values into u
// The chains of different groups are independent branches of the graph, so
// the runtime runs them concurrently.  The graph is built for one (f, u)
// pair and rebuilt when either pointer changes.
#include "mrp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mrp {

// Loop control of one group (single thread).  res / fstar: per-problem
// max-norm bit patterns of the stop rule's numerator and denominator (slots
// 1 and 0 for the residual rule, 2 and 3 for the Cauchy rule); ctr: cycles,
// refinement steps, status.
__global__ void k_loop_check(const unsigned long long* __restrict__ res, const unsigned long long* __restrict__ fstar,
                             int np, double tol, int* __restrict__ ctr, double* __restrict__ rel_out, int mixed, int inner,
                             int max_cycles, int max_ir, int count_step, cudaGraphConditionalHandle hc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool all = true, bad = false;
    for (int p = 0; p < np; ++p) {
        const double f = __longlong_as_double((long long)fstar[p]);
        const double r = __longlong_as_double((long long)res[p]);
        const double rel = r / (f > 0.0 ? f : 1.0);
        rel_out[p] = rel;
        if (!(rel < tol)) all = false;
        if (!isfinite(rel)) bad = true;
    }
    if (count_step) {
        if (mixed) { ctr[0] += inner; ctr[1] += 1; }
        else ctr[0] += 1;
    }
    if (bad) ctr[2] = MRP_ERR_NUMERICAL;
    const bool stop = all || bad || (!mixed && ctr[0] >= max_cycles) || (mixed && (ctr[1] >= max_ir || ctr[0] >= max_cycles));
    cudaGraphSetConditional(hc, stop ? 0u : 1u);
}

#define GK(call) do { if ((call) != cudaSuccess) return MRP_ERR_CUDA; } while (0)

// Ping-pong buffers of every level and precision (a sweep swaps them on the host).
struct Ptrs { std::vector<double*> u64, a64; std::vector<float*> u32, a32; };
static Ptrs ptrs_of(Handle& h) {
    Ptrs p;
    for (Level& lv : h.lv) {
        p.u64.push_back(lv.U); p.a64.push_back(lv.Ualt);
        p.u32.push_back(lv.U32); p.a32.push_back(lv.U32alt);
    }
    return p;
}

// After capturing a loop body whose sweeps left a level's buffers swapped,
// copy the current buffer into the original one (inside the body) and swap
// the host pointers back, so that every iteration starts from the same buffers.
static void restore_buffers(Handle& h, const Ptrs& p0, cudaStream_t s) {
    const size_t S = h.n + 2;
    for (size_t k = 0; k < h.lv.size(); ++k) {
        Level& lv = h.lv[k];
        const size_t cnt = (size_t)lv.nb * S * S * S;
        if (lv.U != p0.u64[k]) {
            cudaMemcpyAsync(p0.u64[k], lv.U, sizeof(double) * cnt, cudaMemcpyDeviceToDevice, s);
            std::swap(lv.U, lv.Ualt);
        }
        if (lv.U32 != p0.u32[k]) {
            cudaMemcpyAsync(p0.u32[k], lv.U32, sizeof(float) * cnt, cudaMemcpyDeviceToDevice, s);
            std::swap(lv.U32, lv.U32alt);
        }
    }
}

// Capture of the current stream tail: its last nodes.
static int tail_of(cudaStream_t s, std::vector<cudaGraphNode_t>& out) {
    cudaStreamCaptureStatus st;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    GK(cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &deps, nullptr, &nd));
    out.assign(deps, deps + nd);
    return MRP_OK;
}

static int build_group(Handle& h, cudaGraph_t G, cudaStream_t cs, const double* f, double* u) {
    const int np = h.nprob();
    if (!h.loop_ctr) {
        GK(cudaMalloc(&h.loop_ctr, sizeof(int) * 4));
        GK(cudaMalloc(&h.loop_rel, sizeof(double) * np));
    }
    cudaGraphConditionalHandle hc;
    GK(cudaGraphConditionalHandleCreate(&hc, G, 1, cudaGraphCondAssignDefault));
    int64_t l0 = h.launches;
    // prologue
    GK(cudaStreamBeginCaptureToGraph(cs, G, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaMemsetAsync(h.loop_ctr, 0, sizeof(int) * 4, cs);
    solve_begin(h, f, cs);
    const bool cauchy = h.stop_rule == MRP_STOP_CAUCHY;
    const unsigned long long* num = h.slot(cauchy ? 2 : 1);
    const unsigned long long* den = h.slot(cauchy ? 3 : 0);
    if (h.mixed) {
        // (one level: no FP32 cycles; the FP64 level-0 convolution is the answer)
        if (h.L >= 1) first_step_launch(h, cs);
        outer_residual_launch(h, cs);
        if (cauchy) cauchy_launch(h, cs);
        k_loop_check<<<1, 32, 0, cs>>>(num, den, np, h.tol, h.loop_ctr, h.loop_rel, 1, h.inner_cycles,
                                       h.max_cycles, h.max_ir, h.L >= 1 ? 1 : 0, hc);
    }
    std::vector<cudaGraphNode_t> deps;
    int rc = tail_of(cs, deps);
    cudaGraph_t dummy = nullptr;
    if (cudaStreamEndCapture(cs, &dummy) != cudaSuccess || rc) return MRP_ERR_CUDA;
    h.gl_pro = h.launches - l0 + (h.mixed ? 1 : 0);
    l0 = h.launches;
    // the loop
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode;
    GK(cudaGraphAddNode(&wnode, G, deps.data(), nullptr, deps.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    GK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const Ptrs p0 = ptrs_of(h);
    if (h.mixed) {
        correction_launch(h, cs);
        outer_residual_launch(h, cs);
        if (cauchy) cauchy_launch(h, cs);
    } else {
        vcycle<double>(h, cs);
        if (cauchy) cauchy_launch(h, cs);
        else leaf_residual_launch(h, cs);
    }
    k_loop_check<<<1, 32, 0, cs>>>(num, den, np, h.tol, h.loop_ctr, h.loop_rel, h.mixed ? 1 : 0,
                                   h.inner_cycles, h.max_cycles, h.max_ir, 1, hc);
    restore_buffers(h, p0, cs);
    if (cudaStreamEndCapture(cs, &dummy) != cudaSuccess) return MRP_ERR_CUDA;
    h.gl_body = h.launches - l0 + 1;
    l0 = h.launches;
    // epilogue
    GK(cudaStreamBeginCaptureToGraph(cs, G, &wnode, nullptr, 1, cudaStreamCaptureModeRelaxed));
    solve_end(h, u, cs);
    if (cudaStreamEndCapture(cs, &dummy) != cudaSuccess) return MRP_ERR_CUDA;
    h.gl_epi = h.launches - l0;
    return MRP_OK;
}

int graph_build(mrp_handle* H, const double* f, double* u) {
    if (H->gexec) { cudaGraphExecDestroy(H->gexec); H->gexec = nullptr; }
    if (H->graph) { cudaGraphDestroy(H->graph); H->graph = nullptr; }
    if (!H->cap) GK(cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking));
    for (auto& g : H->g)
        if (autotune(*g, H->cap)) return MRP_ERR_CUDA;
    GK(cudaGraphCreate(&H->graph, 0));
    for (auto& g : H->g) {
        const bool prof = g->prof;
        g->prof = false;                 // no event records inside the graph
        const int rc = build_group(*g, H->graph, H->cap, f, u);
        g->prof = prof;
        if (rc) {
            cudaGetLastError();
            return rc;
        }
    }
    GK(cudaGraphInstantiate(&H->gexec, H->graph, 0));
    H->gf = f;
    H->gu = u;
    return MRP_OK;
}

void graph_release(mrp_handle* H) {
    if (H->gexec) cudaGraphExecDestroy(H->gexec);
    if (H->graph) cudaGraphDestroy(H->graph);
    if (H->cap) cudaStreamDestroy(H->cap);
    H->gexec = nullptr;
    H->graph = nullptr;
    H->cap = nullptr;
    cudaFree(H->host_f);
    cudaFree(H->host_u);
    H->host_f = nullptr;
    H->host_u = nullptr;
    for (auto& g : H->g) {
        cudaFree(g->loop_ctr);
        cudaFree(g->loop_rel);
        g->loop_ctr = nullptr;
        g->loop_rel = nullptr;
    }
}

}  // namespace mrp

using namespace mrp;

extern "C" int mrp_solve_graph(mrp_handle* H, const double* f, double* u, void* stream, mrp_stats* st) {
    if (!H || !f || !u) return MRP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!H->gexec || H->gf != f || H->gu != u) {
        // the graph reads nothing that a call on another stream may still be writing
        if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
        const int rc = graph_build(H, f, u);
        if (rc) return rc;
    }
    if (cudaGraphLaunch(H->gexec, s) != cudaSuccess) return MRP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
    int status = MRP_OK;
    bool converged = true;
    if (st) std::memset(st, 0, sizeof(*st));
    for (auto& gp : H->g) {
        Handle& h = *gp;
        const int np = h.nprob();
        int ctr[4];
        std::vector<double> rel(np);
        if (cudaMemcpy(ctr, h.loop_ctr, sizeof(ctr), cudaMemcpyDeviceToHost) != cudaSuccess) return MRP_ERR_CUDA;
        if (cudaMemcpy(rel.data(), h.loop_rel, sizeof(double) * np, cudaMemcpyDeviceToHost) != cudaSuccess)
            return MRP_ERR_CUDA;
        if (read_max(h, s, h.fstar.data(), 0)) return MRP_ERR_CUDA;
        h.fstar_max = *std::max_element(h.fstar.begin(), h.fstar.end());
        h.have_forward = true;
        double worst = 0.0;
        for (double r : rel) worst = std::max(worst, r);
        if (!(worst < h.tol)) converged = false;
        if (ctr[2] && !status) status = ctr[2];
        if (st) {
            st->cycles = std::max(st->cycles, ctr[0]);
            st->ir_steps = std::max(st->ir_steps, ctr[1]);
            if (h.stop_rule == MRP_STOP_CAUCHY) {
                st->cauchy = std::max(st->cauchy, worst);
                if (h.mixed) {       // the last outer residual, relative to max |f*|
                    std::vector<double> r(np);
                    if (read_max(h, s, r.data(), 1)) return MRP_ERR_CUDA;
                    for (int p = 0; p < np; ++p)
                        st->residual = std::max(st->residual, r[p] / (h.fstar[p] > 0.0 ? h.fstar[p] : 1.0));
                }
            } else {
                st->residual = std::max(st->residual, worst);
            }
            st->fstar_max = std::max(st->fstar_max, h.fstar_max);
            st->leaf_nodes += h.leaf_nodes;
            st->total_nodes += h.total_nodes;
            st->launches += h.gl_pro + (int64_t)(h.mixed ? ctr[1] : ctr[0]) * h.gl_body + h.gl_epi;
        }
    }
    if (status) return status;
    return converged ? MRP_OK : MRP_ERR_NOT_CONVERGED;
}

extern "C" int mrp_solve_host(mrp_handle* H, const double* f_host, double* u_host, void* stream, mrp_stats* st) {
    if (!H || !f_host || !u_host) return MRP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = sizeof(double) * (size_t)H->elems;
    if (!H->host_f) {
        if (cudaMalloc(&H->host_f, bytes) != cudaSuccess) { cudaGetLastError(); return MRP_ERR_OOM; }
        if (cudaMalloc(&H->host_u, bytes) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(H->host_f);
            H->host_f = nullptr;
            return MRP_ERR_OOM;
        }
    }
    if (cudaMemcpyAsync(H->host_f, f_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return MRP_ERR_CUDA;
    const int rc = mrp_solve_graph(H, H->host_f, H->host_u, stream, st);
    if (rc != MRP_OK && rc != MRP_ERR_NOT_CONVERGED && rc != MRP_ERR_NUMERICAL) return rc;
    if (cudaMemcpyAsync(u_host, H->host_u, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return MRP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MRP_ERR_CUDA;
    return rc;
}
