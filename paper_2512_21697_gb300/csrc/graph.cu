// graph.cu -- the persistent multi-step driver: the whole Crank-Nicolson time loop (Eq. solPsi)
// captured once into a CUDA graph whose data-dependent loops are conditional WHILE nodes
//   steps -> { pulse + assembly, b = A_- psi, guess,
//              solve: FP64 BiCGSTAB with true-residual restarts, or refinement with inner
//              complex64 BiCGSTAB (precision >= 1),
//              history shift }
// so one graph launch advances n_steps with no host round trip.  Loop conditions are set on the
// device (cudaGraphSetConditional) from the BiCGSTAB state; every loop has an iteration cap.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "device.h"
#include "kernels.h"
#include "op.h"

namespace dg {

struct StepCtl {
    double t_start, dt, t_off;   // evaluation time of step s: t_start + s dt + t_off
    int step, n_steps;
    int hist_n;                  // valid history entries (0..hist_max)
    int hist_max;                // 2, or 3 with the learned guess
    int status;                  // first failing status, 0 while all steps succeed
    int accepted, restarts, outer, total_it;
    int max_restarts, max_outer;
};

struct GraphDriver {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* psi = nullptr;
    const void* hist = nullptr;
    StepCtl* ctl = nullptr;
    int* its = nullptr;
    double* res = nullptr;
    int cap = 0;                 // capacity of its/res
    cudaStream_t cap_stream = nullptr;
    int gen = -1;                // op->config_gen the graph was captured with
    StepCtl* h_ctl = nullptr;    // pinned host copies of the results (asynchronous read-back)
    int* h_its = nullptr;
    double* h_res = nullptr;
};

__global__ void k_set_ctl(StepCtl* c, StepCtl v) { *c = v; }

__global__ void k_ctl_begin_step(StepCtl* c, double* t_eval, cudaGraphConditionalHandle h_solve)
{
    *t_eval = step_time(c->t_start, c->step, c->dt, c->t_off);
    c->accepted = 0;
    c->restarts = 0;
    c->outer = 0;
    c->total_it = 0;
    cudaGraphSetConditional(h_solve, 1);
}

// x = extrapolated guess from psi and the valid history (guess option >= 1), else psi; skipped when
// the learned guess produced x this step (*skip set)
__global__ void k_guess(const StepCtl* c, int use_hist, int64_t n, const double2* psi, const double2* h1,
                        const double2* h2, double2* x, const int* skip)
{
    if (skip && *skip) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int nh = use_hist ? min(c->hist_n, 2) : 0;
    double2 p = psi[i], a = nh >= 1 ? h1[i] : p, b = nh >= 2 ? h2[i] : p;
    x[i] = make_double2(extrapolate(nh, p.x, a.x, b.x), extrapolate(nh, p.y, a.y, b.y));
}

// learned guess of this step: field factors at t_start + (step + 1) dt, and the gate (three past states)
__global__ void k_ctl_guess_prep(const StepCtl* c, PulseView P, float* F, int* gate)
{
    guess_field_at(P, next_time(c->t_start, c->step, c->dt), F);
    *gate = c->hist_n >= 3 ? 1 : 0;
}

// after r = b - A x: accept on the true residual, else iterate
__global__ void k_ctl_after_begin(StepCtl* c, const KState* ks, cudaGraphConditionalHandle h_iter)
{
    int it = 0;
    if (ks->status) {
        c->status = ks->status;
        c->accepted = 1;
    } else if (ks->done) {
        c->accepted = 1;
    } else {
        it = 1;
    }
    cudaGraphSetConditional(h_iter, it);
}

__global__ void k_ctl_iter_cond(const KState* ks, cudaGraphConditionalHandle h_iter)
{
    cudaGraphSetConditional(h_iter, ks->done ? 0 : 1);
}

// after an iteration run of the FP64 solve: restart (breakdown or recursive-residual drift, then
// the next begin checks the true residual) or stop
__global__ void k_ctl_after_solve(StepCtl* c, const KState* ks, cudaGraphConditionalHandle h_solve)
{
    int again = 0;
    if (!c->accepted) {
        c->total_it += ks->it;
        if (ks->status == 5 && c->restarts < 2) {
            c->restarts++;
            again = 1;
        } else if (ks->status) {
            c->status = ks->status;
        } else if (++c->restarts > c->max_restarts) {
            c->status = 4;
        } else {
            again = 1;
        }
    }
    cudaGraphSetConditional(h_solve, again);
}

// refinement: after the accurate residual; done when it meets tol, else one inner solve and
// another refinement pass
__global__ void k_ctl_after_outer(StepCtl* c, const KState* ks, cudaGraphConditionalHandle h_inner,
                                  cudaGraphConditionalHandle h_solve)
{
    int go = 0;
    if (ks->status) {
        c->status = ks->status;
        c->accepted = 1;
    } else if (ks->done) {
        c->accepted = 1;
    } else if (c->outer++ >= c->max_outer) {
        c->status = 4;
        c->accepted = 1;
    } else {
        go = 1;
    }
    cudaGraphSetConditional(h_inner, go);
    cudaGraphSetConditional(h_solve, go);
}

__global__ void k_ctl_after_inner(StepCtl* c, const KState* ki)
{
    c->total_it += ki->it;
    if (ki->status && ki->status != 4) c->status = ki->status;
}

// end of a refinement pass (same graph level as the refinement loop): stop on a failure
__global__ void k_ctl_after_pass(const StepCtl* c, cudaGraphConditionalHandle h_solve)
{
    if (c->status) cudaGraphSetConditional(h_solve, 0);
}

__global__ void k_ctl_end_step(StepCtl* c, const KState* ks, int* its, double* res,
                               cudaGraphConditionalHandle h_step)
{
    int s = c->step;
    its[s] = c->total_it;
    res[s] = sqrt(ks->rnorm2 / (ks->bnorm2 > 0 ? ks->bnorm2 : 1.0));
    c->hist_n = c->hist_n < c->hist_max ? c->hist_n + 1 : c->hist_max;
    c->step = s + 1;
    cudaGraphSetConditional(h_step, (c->step < c->n_steps && c->status == 0) ? 1 : 0);
}

// b = a when at least `need` history entries are valid
__global__ void k_copy_if_hist(const StepCtl* c, int need, int64_t n, const double2* a, double2* b)
{
    if (c->hist_n < need) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i];
}

// ---- capture helpers --------------------------------------------------------------------------

#define G_TRY(call)                                                                              \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            set_error(std::string("dirac_run: ") + #call + ": " + cudaGetErrorString(e_));      \
            return DIRAC_E_CUDA;                                                                 \
        }                                                                                        \
    } while (0)

// Append a conditional node (WHILE or IF) at the current capture point of `s`; returns its body.
static dirac_status add_cond(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                             cudaGraph_t* body)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    G_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams p{};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    G_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    *body = p.conditional.phGraph_out[0];
    G_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return DIRAC_OK;
}

static dirac_status current_graph(cudaStream_t s, cudaGraph_t* g)
{
    cudaStreamCaptureStatus cs;
    G_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, g, nullptr, nullptr, nullptr));
    return DIRAC_OK;
}

// Capture `fill` into `body` on a private stream (the op's launches are redirected to it).
template <class F>
static dirac_status capture_into(dirac_op* op, cudaGraph_t body, F fill)
{
    cudaStream_t s;
    G_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaStream_t saved = op->st;
    cudaError_t e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        set_error(std::string("dirac_run: cudaStreamBeginCaptureToGraph: ") + cudaGetErrorString(e));
        return DIRAC_E_CUDA;
    }
    op->st = s;
    dirac_status st = fill(s);
    op->st = saved;
    cudaGraph_t out;
    e = cudaStreamEndCapture(s, &out);
    cudaStreamDestroy(s);
    if (st) return st;
    if (e != cudaSuccess) {
        set_error(std::string("dirac_run: cudaStreamEndCapture: ") + cudaGetErrorString(e));
        return DIRAC_E_CUDA;
    }
    return DIRAC_OK;
}

// Body of the FP64 solve loop: begin (true residual), then iterations while not done.
static dirac_status fill_solve64(dirac_op* op, GraphDriver* gd, cudaStream_t s, cudaGraphConditionalHandle h_solve)
{
    Krylov& K = op->k64;
    const dirac_solver_opts& o = op->opts;
    bicgstab_begin(op, K, o.max_iter);
    cudaGraph_t g;
    dirac_status st = current_graph(s, &g);
    if (st) return st;
    cudaGraphConditionalHandle h_iter;
    G_TRY(cudaGraphConditionalHandleCreate(&h_iter, g, 0, 0));
    k_ctl_after_begin<<<1, 1, 0, s>>>(gd->ctl, K.ks, h_iter);
    cudaGraph_t body;
    st = add_cond(s, h_iter, cudaGraphCondTypeWhile, &body);
    if (st) return st;
    st = capture_into(op, body, [&](cudaStream_t s2) {
        dirac_status e = bicgstab_iteration(op, K, o.max_iter, false);
        if (e) return e;
        k_ctl_iter_cond<<<1, 1, 0, s2>>>(K.ks, h_iter);
        return check_launch("dirac_run iteration");
    });
    if (st) return st;
    k_ctl_after_solve<<<1, 1, 0, s>>>(gd->ctl, K.ks, h_solve);
    return check_launch("dirac_run solve");
}

// Body of the refinement loop: accurate residual; unless accepted, one inner complex64 solve
// (begin + iterations) and x += ||r|| d.
static dirac_status fill_refine(dirac_op* op, GraphDriver* gd, cudaStream_t s, cudaGraphConditionalHandle h_solve,
                                const double2* psi)
{
    Krylov& K = op->k64;
    Krylov& I = op->k32;
    const dirac_solver_opts& o = op->opts;
    residual_accurate(op, psi);
    cudaGraph_t g;
    dirac_status st = current_graph(s, &g);
    if (st) return st;
    cudaGraphConditionalHandle h_inner;
    G_TRY(cudaGraphConditionalHandleCreate(&h_inner, g, 0, 0));
    k_ctl_after_outer<<<1, 1, 0, s>>>(gd->ctl, K.ks, h_inner, h_solve);
    cudaGraph_t inner;
    st = add_cond(s, h_inner, cudaGraphCondTypeIf, &inner);
    if (st) return st;
    st = capture_into(op, inner, [&](cudaStream_t s2) {
        int npv = op->nparts_vec;
        k_to_float_scaled<<<npv, 256, 0, s2>>>(op->n, (const double2*)K.r, K.ks, (float2*)I.b);
        k_zero32<<<npv, 256, 0, s2>>>(op->n, (float2*)I.x);
        bicgstab_begin(op, I, o.max_iter, true);
        cudaGraph_t g2;
        dirac_status e = current_graph(s2, &g2);
        if (e) return e;
        cudaGraphConditionalHandle h_iter;
        G_TRY(cudaGraphConditionalHandleCreate(&h_iter, g2, 0, 0));
        k_ctl_iter_cond<<<1, 1, 0, s2>>>(I.ks, h_iter);
        cudaGraph_t body;
        e = add_cond(s2, h_iter, cudaGraphCondTypeWhile, &body);
        if (e) return e;
        e = capture_into(op, body, [&](cudaStream_t s3) {
            dirac_status e3 = bicgstab_iteration(op, I, o.max_iter, false);
            if (e3) return e3;
            k_ctl_iter_cond<<<1, 1, 0, s3>>>(I.ks, h_iter);
            return check_launch("dirac_run inner iteration");
        });
        if (e) return e;
        k_add_float_scaled<<<npv, 256, 0, s2>>>(op->n, (const float2*)I.x, K.ks, (double2*)K.x);
        k_ctl_after_inner<<<1, 1, 0, s2>>>(gd->ctl, I.ks);
        return check_launch("dirac_run inner");
    });
    if (st) return st;
    k_ctl_after_pass<<<1, 1, 0, s>>>(gd->ctl, h_solve);
    return check_launch("dirac_run refinement");
}

static dirac_status build_graph(dirac_op* op, GraphDriver* gd, double2* psi, double2* h1, double2* h2)
{
    if (gd->exec) { cudaGraphExecDestroy(gd->exec); gd->exec = nullptr; }
    if (gd->graph) { cudaGraphDestroy(gd->graph); gd->graph = nullptr; }
    G_TRY(cudaGraphCreate(&gd->graph, 0));
    cudaGraphConditionalHandle h_step;
    G_TRY(cudaGraphConditionalHandleCreate(&h_step, gd->graph, 1, cudaGraphCondAssignDefault));
    bool prof = op->profiling;
    op->profiling = false;   // event records are not allowed inside conditional bodies
    int64_t launches = op->launches;
    dirac_status st = capture_into(op, gd->graph, [&](cudaStream_t s0) {
        cudaGraph_t step_body;
        dirac_status e = add_cond(s0, h_step, cudaGraphCondTypeWhile, &step_body);
        if (e) return e;
        return capture_into(op, step_body, [&](cudaStream_t s1) {
            Krylov& K = op->k64;
            const dirac_solver_opts& o = op->opts;
            cudaGraph_t g;
            dirac_status e1 = current_graph(s1, &g);
            if (e1) return e1;
            cudaGraphConditionalHandle h_solve;
            G_TRY(cudaGraphConditionalHandleCreate(&h_solve, g, 0, 0));
            k_ctl_begin_step<<<1, 1, 0, s1>>>(gd->ctl, op->t_eval, h_solve);
            launch_assemble(op);
            if (o.precision == 0) {
                apply_accurate(op, -1, psi, K.b, nullptr, op->part_n);
                finish(op, K.ks, 0, op->nparts_apply, nullptr, op->part_n, o.max_iter);
            } else {
                rhs_accurate(op, psi);
            }
            int npv = op->nparts_vec;
            const bool learned = o.guess == 2 && op->net;
            if (learned) {
                k_ctl_guess_prep<<<1, 1, 0, s1>>>(gd->ctl, op->pv, op->gfield, op->ggate);
                e1 = guess_into(op, psi, h1, h2, h1 + 2 * op->n, 0.0, 0, (double2*)K.x, op->ggate, s1, op->gfield);
                if (e1) return e1;
            }
            k_guess<<<npv, 256, 0, s1>>>(gd->ctl, o.guess >= 1, op->n, psi, h1, h2, (double2*)K.x,
                                         learned ? op->ggate : nullptr);
            cudaGraph_t solve_body;
            e1 = add_cond(s1, h_solve, cudaGraphCondTypeWhile, &solve_body);
            if (e1) return e1;
            e1 = capture_into(op, solve_body, [&](cudaStream_t s2) {
                return o.precision == 0 ? fill_solve64(op, gd, s2, h_solve) : fill_refine(op, gd, s2, h_solve, psi);
            });
            if (e1) return e1;
            if (learned) k_copy_if_hist<<<npv, 256, 0, s1>>>(gd->ctl, 2, op->n, h2, h1 + 2 * op->n);
            k_copy_if_hist<<<npv, 256, 0, s1>>>(gd->ctl, 1, op->n, h1, h2);
            k_copy64<<<npv, 256, 0, s1>>>(op->n, psi, h1);
            k_copy64<<<npv, 256, 0, s1>>>(op->n, (const double2*)K.x, psi);
            k_ctl_end_step<<<1, 1, 0, s1>>>(gd->ctl, K.ks, gd->its, gd->res, h_step);
            return check_launch("dirac_run step");
        });
    });
    op->profiling = prof;
    op->launches = launches;
    if (st) {
        // a graph whose capture was invalidated part-way through a conditional body is dropped, not
        // destroyed: it is never launched, and tearing down its half-captured bodies is not relied on
        gd->graph = nullptr;
        return st;
    }
    G_TRY(cudaGraphInstantiate(&gd->exec, gd->graph, 0));
    gd->psi = psi;
    gd->hist = h1;
    return DIRAC_OK;
}

void graph_free(dirac_op* op)
{
    GraphDriver* gd = op->graph;
    if (!gd) return;
    if (gd->exec) cudaGraphExecDestroy(gd->exec);
    if (gd->graph) cudaGraphDestroy(gd->graph);
    cudaFree(gd->ctl);
    cudaFree(gd->its);
    cudaFree(gd->res);
    cudaFreeHost(gd->h_ctl);
    cudaFreeHost(gd->h_its);
    cudaFreeHost(gd->h_res);
    delete gd;
    op->graph = nullptr;
}


// Enqueue n_steps of the captured driver on the op's stream (graph built or rebuilt as needed) and
// the asynchronous read-back of its results into pinned host memory.  Nothing waits for the GPU.
dirac_status run_launch(dirac_op* op, double2* psi, double2* h1, int n_hist, int n_steps, double t_start)
{
    if (!op->graph) op->graph = new GraphDriver();
    GraphDriver* gd = op->graph;
    double2* h2 = h1 + op->n;
    bool rebuild = !gd->exec || gd->psi != psi || gd->hist != h1 || gd->gen != op->config_gen;
    if (!gd->ctl) G_TRY(cudaMalloc(&gd->ctl, sizeof(StepCtl)));
    if (!gd->h_ctl) G_TRY(cudaMallocHost(&gd->h_ctl, sizeof(StepCtl)));
    if (gd->cap < n_steps) {
        cudaFree(gd->its);
        cudaFree(gd->res);
        cudaFreeHost(gd->h_its);
        cudaFreeHost(gd->h_res);
        gd->its = nullptr;
        gd->res = nullptr;
        gd->h_its = nullptr;
        gd->h_res = nullptr;
        int cap = std::max(n_steps, 256);
        G_TRY(cudaMalloc(&gd->its, sizeof(int) * cap));
        G_TRY(cudaMalloc(&gd->res, sizeof(double) * cap));
        G_TRY(cudaMallocHost(&gd->h_its, sizeof(int) * cap));
        G_TRY(cudaMallocHost(&gd->h_res, sizeof(double) * cap));
        gd->cap = cap;
        rebuild = true;
    }
    if (rebuild) {
        dirac_status st = build_graph(op, gd, psi, h1, h2);
        if (st) return st;
        gd->gen = op->config_gen;
    }
    const dirac_solver_opts& o = op->opts;
    StepCtl c{};
    c.t_start = t_start;
    c.dt = o.dt;
    c.t_off = o.time_eval ? o.dt : 0.5 * o.dt;
    c.n_steps = n_steps;
    c.hist_max = (o.guess == 2 && op->net) ? 3 : 2;
    c.hist_n = std::max(0, std::min(c.hist_max, n_hist));
    c.max_restarts = 8;
    c.max_outer = o.max_outer;
    k_set_ctl<<<1, 1, 0, op->st>>>(gd->ctl, c);
    G_TRY(cudaGetLastError());
    G_TRY(cudaGraphLaunch(gd->exec, op->st));
    G_TRY(cudaMemcpyAsync(gd->h_ctl, gd->ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, op->st));
    G_TRY(cudaMemcpyAsync(gd->h_its, gd->its, sizeof(int) * n_steps, cudaMemcpyDeviceToHost, op->st));
    G_TRY(cudaMemcpyAsync(gd->h_res, gd->res, sizeof(double) * n_steps, cudaMemcpyDeviceToHost, op->st));
    op->launches += 2;   // the control upload and one graph launch (its kernels are not counted)
    return DIRAC_OK;
}

// Wait for the op's stream and report the results of the last run_launch.
dirac_status run_collect(dirac_op* op, int n_steps, int* n_hist, int* iters_out, double* resid_out, const char* who)
{
    GraphDriver* gd = op->graph;
    cudaError_t e = cudaStreamSynchronize(op->st);
    if (e != cudaSuccess) {
        set_error(std::string(who) + ": " + cudaGetErrorString(e));
        return DIRAC_E_CUDA;
    }
    const StepCtl& c = *gd->h_ctl;
    for (int s = 0; s < c.step && s < n_steps; s++) {
        if (iters_out) iters_out[s] = gd->h_its[s];
        if (resid_out) resid_out[s] = gd->h_res[s];
    }
    if (n_hist) *n_hist = c.hist_n;
    dirac_status de = check_dev_err(op, who);
    if (de) return de;
    if (c.status) {
        set_error(std::string(who) + ": step " + std::to_string(c.step - 1) + " failed with status " +
                  std::to_string(c.status));
        return (dirac_status)c.status;
    }
    return DIRAC_OK;
}

}  // namespace dg

using namespace dg;

extern "C" dirac_status dirac_run(dirac_op* op, void* psi_dev, void* hist_dev, int* n_hist, int n_steps,
                                  double t_start, int* iters_out, double* resid_out)
{
    if (!op || !psi_dev || !hist_dev || n_steps < 0) {
        set_error("dirac_run: bad argument (psi and the 2n history buffer are required)");
        return DIRAC_E_ARG;
    }
    if (n_steps == 0) return DIRAC_OK;
    dirac_status st = run_launch(op, (double2*)psi_dev, (double2*)hist_dev, n_hist ? *n_hist : 0, n_steps, t_start);
    if (st) return st;
    return run_collect(op, n_steps, n_hist, iters_out, resid_out, "dirac_run");
}

// Many independent instances (their own basis, pulse and radial size), each advanced by its own
// captured driver on its own stream, so their kernels overlap on the GPU: the small, latency-bound
// parts of one instance (preconditioner sweeps, reductions, control) fill the gaps of the others.
// window > 0 keeps at most `window` instances in flight (instance i starts when i - window is done).
extern "C" dirac_status dirac_solve_batch(dirac_op* const* ops, int n_inst, void* const* psi_dev,
                                          void* const* hist_dev, int* n_hist, int n_steps, const double* t_start,
                                          int window, int* iters_out, double* resid_out)
{
    if (!ops || !psi_dev || !hist_dev || !t_start || n_inst < 0 || n_steps < 0 || window < 0) {
        set_error("dirac_solve_batch: bad argument");
        return DIRAC_E_ARG;
    }
    for (int i = 0; i < n_inst; i++) {
        if (!ops[i] || !psi_dev[i] || !hist_dev[i]) {
            set_error("dirac_solve_batch: instance " + std::to_string(i) + " has a NULL op, state or history");
            return DIRAC_E_ARG;
        }
        if (ops[i]->device != ops[0]->device) {
            set_error("dirac_solve_batch: instances on different devices");
            return DIRAC_E_ARG;
        }
        for (int j = 0; j < i; j++)
            if (ops[j] == ops[i]) {
                set_error("dirac_solve_batch: the same op appears twice");
                return DIRAC_E_ARG;
            }
    }
    if (n_inst == 0 || n_steps == 0) return DIRAC_OK;
    std::vector<cudaEvent_t> ev(n_inst, nullptr);
    dirac_status first = DIRAC_OK;
    int launched = 0;
    for (int i = 0; i < n_inst; i++) {
        dirac_op* op = ops[i];
        if (window > 0 && i >= window) {
            if (cudaStreamWaitEvent(op->st, ev[i - window], 0) != cudaSuccess) {
                set_error("dirac_solve_batch: cudaStreamWaitEvent failed");
                first = DIRAC_E_CUDA;
                break;
            }
        }
        dirac_status st = run_launch(op, (double2*)psi_dev[i], (double2*)hist_dev[i], n_hist ? n_hist[i] : 0, n_steps,
                                     t_start[i]);
        if (st) { first = st; break; }
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventRecord(ev[i], op->st) != cudaSuccess) {
            set_error("dirac_solve_batch: event record failed");
            first = DIRAC_E_CUDA;
            launched = i + 1;
            break;
        }
        launched = i + 1;
    }
    std::string msg = first ? dirac_last_error() : std::string();
    for (int i = 0; i < launched; i++) {
        dirac_status st = run_collect(ops[i], n_steps, n_hist ? &n_hist[i] : nullptr,
                                      iters_out ? iters_out + (size_t)i * n_steps : nullptr,
                                      resid_out ? resid_out + (size_t)i * n_steps : nullptr, "dirac_solve_batch");
        if (st && !first) {
            first = st;
            msg = "instance " + std::to_string(i) + ": " + dirac_last_error();
        }
    }
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    if (first) set_error(msg);
    return first;
}

// Schedule autotuner of the batch: times one step of every instance for each candidate window
// (instances in flight) and each inner-preconditioner schedule (one lane or one warp per channel;
// the warp schedule is the best available: rotated lanes, else staged, else plain),
// on saved copies of the states, restores the states and histories, and leaves every op on the
// fastest preconditioner schedule.  Returns the best window and, per tried configuration, the
// milliseconds (ms_out[v * ncand + c], v = 0 lanes, 1 warps), when ms_out is given.
extern "C" dirac_status dirac_batch_tune(dirac_op* const* ops, int n_inst, void* const* psi_dev, void* const* hist_dev,
                                         const int* n_hist, const double* t_start, const int* cand, int ncand,
                                         int* best_window, double* ms_out)
{
    if (!ops || !psi_dev || !hist_dev || !t_start || !cand || ncand <= 0 || n_inst <= 0 || !best_window) {
        set_error("dirac_batch_tune: bad argument");
        return DIRAC_E_ARG;
    }
    for (int c = 0; c < ncand; c++)
        if (cand[c] < 0) { set_error("dirac_batch_tune: negative window"); return DIRAC_E_ARG; }
    std::vector<void*> save(n_inst, nullptr);
    std::vector<int> nh(n_inst), nh0(n_inst);
    dirac_status first = DIRAC_OK;
    for (int i = 0; i < n_inst && !first; i++) {
        if (!ops[i] || !psi_dev[i] || !hist_dev[i]) { set_error("dirac_batch_tune: NULL instance"); first = DIRAC_E_ARG; break; }
        size_t b = sizeof(double2) * 3 * (size_t)ops[i]->n;
        if (cudaMalloc(&save[i], b) != cudaSuccess) { set_error("dirac_batch_tune: cudaMalloc failed"); first = DIRAC_E_NOMEM; break; }
        size_t bn = sizeof(double2) * (size_t)ops[i]->n;
        cudaMemcpyAsync(save[i], psi_dev[i], bn, cudaMemcpyDeviceToDevice, ops[i]->st);
        cudaMemcpyAsync((char*)save[i] + bn, hist_dev[i], 2 * bn, cudaMemcpyDeviceToDevice, ops[i]->st);
        nh0[i] = n_hist ? n_hist[i] : 0;
    }
    int nsaved = 0;
    for (int i = 0; i < n_inst; i++) nsaved += save[i] != nullptr;
    auto restore = [&]() {
        if (nsaved != n_inst) return;   // a save failed: nothing ran, nothing to restore
        for (int i = 0; i < n_inst; i++) {
            size_t bn = sizeof(double2) * (size_t)ops[i]->n;
            cudaMemcpyAsync(psi_dev[i], save[i], bn, cudaMemcpyDeviceToDevice, ops[i]->st);
            cudaMemcpyAsync(hist_dev[i], (char*)save[i] + bn, 2 * bn, cudaMemcpyDeviceToDevice, ops[i]->st);
            nh[i] = nh0[i];
        }
    };
    double best = 1e300;
    int bw = cand[0], bv = 0;
    auto sched_of = [](const dirac_op* op, int v) {
        if (v == 0) return 0;
        return op->prec_rot_ok ? 3 : op->prec_sm_ok ? 2 : 1;
    };
    for (int v = 0; v < 2 && !first; v++) {
        for (int i = 0; i < n_inst; i++) {
            ops[i]->prec_sched32 = sched_of(ops[i], v);
            ops[i]->config_gen++;
        }
        restore();
        first = dirac_solve_batch(ops, n_inst, psi_dev, hist_dev, nh.data(), 1, t_start, 0, nullptr, nullptr);   // warm-up
        for (int c = 0; c < ncand && !first; c++) {
            restore();
            for (int i = 0; i < n_inst; i++) cudaStreamSynchronize(ops[i]->st);
            auto t0 = std::chrono::steady_clock::now();
            first = dirac_solve_batch(ops, n_inst, psi_dev, hist_dev, nh.data(), 1, t_start, cand[c], nullptr, nullptr);
            double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            if (ms_out) ms_out[v * ncand + c] = ms;
            if (!first && ms < best) { best = ms; bw = cand[c]; bv = v; }
        }
    }
    restore();
    for (int i = 0; i < n_inst; i++) {
        if (ops[i]) {
            ops[i]->prec_sched32 = sched_of(ops[i], bv);
            ops[i]->config_gen++;
            if (ops[i]->st) cudaStreamSynchronize(ops[i]->st);
        }
        if (save[i]) cudaFree(save[i]);
    }
    *best_window = bw;
    return first;
}
