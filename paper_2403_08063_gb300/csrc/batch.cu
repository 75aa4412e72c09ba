// Batches of independent problems with different block sizes (many uneven octree forests solved together).
//
// Problems sharing a block size n live in one multi-problem forest (its blocks carry a problem id; neighbours,
// octet merging, norms and the block-diagonal coarsest inverse are per problem).  The batch owns one such forest
// per distinct n, all on one stream, reading and writing the caller's arrays in place through per-leaf offsets.
// With FP32 cycles, one defect-correction step of every group (m FP32 V-cycles, the FP64 update, the next FP64
// residual and its per-problem norms) is captured once in a CUDA graph and replayed until every problem meets rtol.
// Each group runs on a stream of its own, forked from and joined back to the batch stream, so the graph holds one
// branch per group and the latency-bound launches of small groups overlap the bandwidth-bound ones of large groups.
#include <algorithm>
#include <cmath>
#include <map>

#include "forest_state.h"

struct mg_batch {
    mg_config cfg{};
    cudaStream_t user = nullptr;  // caller's stream (may be the legacy default stream)
    cudaStream_t st = nullptr;    // batch stream (non-blocking; graphs are captured on it)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int np = 0;
    int64_t total_cells = 0;
    std::vector<mg_forest *> groups;
    std::vector<int32_t> gn;                  // block size per group
    std::vector<std::vector<int32_t>> gprob;  // batch problem ids per group (local id = position)
    std::vector<cudaStream_t> gst;            // one stream per group (the group forest's stream)
    std::vector<cudaEvent_t> gev;             // join events, one per group
    cudaEvent_t ev_fork = nullptr;
    int *flag = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_m = 0;
    std::vector<int> graph_tails;  // the groups' tail levels (and the tail mode, last) when the graph was captured
    bool rhs_set = false;
    bool tails_tuned = false;
    // persistent tails: 0 every level launched, 1 each group's own tail, 2 one joint tail per V-cycle
    int tail_mode = 0;
    std::vector<int> tuned_tails;         // each group's tuned tail level (-1: none)
    cudaEvent_t ev_joint = nullptr;       // the joint tail done (groups[0]'s stream), awaited by the other groups
    octmg::TailArgs *jt_args = nullptr;   // device: every group's tail arguments
    octmg::BatchEntry *jt_entries = nullptr;
    int jt_ne = 0, jt_cap = 0;
    unsigned *jt_bar = nullptr;
    int64_t jt_need = 1;
};

namespace octmg {
namespace {

__global__ void k_check_batch(const double *__restrict__ f, const double *__restrict__ k, int64_t n,
                              int *__restrict__ bad) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (!isfinite(f[i])) atomicOr(bad, 1);
        if (k && !(isfinite(k[i]) && k[i] > 0.0)) atomicOr(bad, 2);
    }
}

void destroy_batch(mg_batch *B) {
    if (!B) return;
    if (B->st) cudaStreamSynchronize(B->st);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    for (cudaStream_t s : B->gst) cudaStreamSynchronize(s);
    for (mg_forest *F : B->groups) mg_forest_destroy(F);
    for (cudaEvent_t e : B->gev) cudaEventDestroy(e);
    for (cudaStream_t s : B->gst) cudaStreamDestroy(s);
    if (B->ev_fork) cudaEventDestroy(B->ev_fork);
    if (B->ev_joint) cudaEventDestroy(B->ev_joint);
    if (B->jt_args) cudaFree(B->jt_args);
    if (B->jt_entries) cudaFree(B->jt_entries);
    if (B->jt_bar) cudaFree(B->jt_bar);
    if (B->flag) cudaFree(B->flag);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->st) cudaStreamDestroy(B->st);
    delete B;
}

// Order the batch stream after the caller's stream on entry, and the caller's after the batch's on exit.
mg_status enter(mg_batch *B) {
    MG_CUDA(cudaEventRecord(B->ev_in, B->user));
    MG_CUDA(cudaStreamWaitEvent(B->st, B->ev_in, 0));
    return MG_OK;
}
mg_status leave(mg_batch *B) {
    MG_CUDA(cudaEventRecord(B->ev_out, B->st));
    MG_CUDA(cudaStreamWaitEvent(B->user, B->ev_out, 0));
    return MG_OK;
}

// Group streams start after the batch stream's work so far (fork) and the batch stream waits for all of them (join).
mg_status fork(mg_batch *B) {
    MG_CUDA(cudaEventRecord(B->ev_fork, B->st));
    for (cudaStream_t s : B->gst) MG_CUDA(cudaStreamWaitEvent(s, B->ev_fork, 0));
    return MG_OK;
}
mg_status join(mg_batch *B) {
    for (size_t g = 0; g < B->gst.size(); ++g) {
        MG_CUDA(cudaEventRecord(B->gev[g], B->gst[g]));
        MG_CUDA(cudaStreamWaitEvent(B->st, B->gev[g], 0));
    }
    return MG_OK;
}

// The joint tail's entry list: phase i of every group that has one, then a grid barrier (groups with a recorded
// tail only; their phase lists are aligned from the first phase).  Uploaded with the groups' tail arguments.
mg_status build_joint_tail(mg_batch *B) {
    std::vector<TailArgs> args;
    std::vector<BatchEntry> e;
    size_t longest = 0;
    B->jt_need = 1;
    for (mg_forest *F : B->groups) {
        args.push_back(tail_args(F));
        if (F->tail_level >= 0) {
            longest = std::max(longest, F->tail_ph_host.size());
            B->jt_need += tail_ctas(F);
        }
    }
    for (size_t i = 0; i < longest; ++i) {
        const size_t first = e.size();
        for (size_t g = 0; g < B->groups.size(); ++g) {
            const mg_forest *F = B->groups[g];
            if (F->tail_level >= 0 && i < F->tail_ph_host.size())
                e.push_back({static_cast<int32_t>(g), 0, F->tail_ph_host[i]});
        }
        if (e.size() > first) e.back().last = 1;
    }
    if (!B->jt_args) {
        MG_CUDA(cudaMalloc(&B->jt_args, B->groups.size() * sizeof(TailArgs)));
        MG_CUDA(cudaMalloc(&B->jt_bar, 2 * sizeof(unsigned)));
    }
    if (static_cast<int>(e.size()) > B->jt_cap) {
        if (B->jt_entries) cudaFree(B->jt_entries);
        B->jt_entries = nullptr;
        MG_CUDA(cudaMalloc(&B->jt_entries, std::max<size_t>(1, e.size()) * sizeof(BatchEntry)));
        B->jt_cap = static_cast<int>(e.size());
    }
    MG_CUDA(cudaMemcpyAsync(B->jt_args, args.data(), args.size() * sizeof(TailArgs), cudaMemcpyHostToDevice, B->st));
    if (!e.empty())
        MG_CUDA(cudaMemcpyAsync(B->jt_entries, e.data(), e.size() * sizeof(BatchEntry), cudaMemcpyHostToDevice, B->st));
    MG_CUDA(cudaStreamSynchronize(B->st));
    B->jt_ne = static_cast<int>(e.size());
    return MG_OK;
}

// groups[0]'s stream waits for every other group's work so far; it then runs the joint tail, and the other groups'
// streams wait for it.
mg_status enqueue_joint_tail(mg_batch *B) {
    mg_forest *F0 = B->groups[0];
    for (size_t g = 1; g < B->groups.size(); ++g) {
        MG_CUDA(cudaEventRecord(B->gev[g], B->gst[g]));
        MG_CUDA(cudaStreamWaitEvent(B->gst[0], B->gev[g], 0));
    }
    if (B->jt_ne > 0) {
        Prof p(F0, P_TAIL32, 1);
        MG_TRY(launch_batch_tail32(B->groups.data(), B->jt_args, B->jt_entries, B->jt_ne, B->jt_bar, B->jt_need));
    }
    MG_CUDA(cudaEventRecord(B->ev_joint, B->gst[0]));
    for (size_t g = 1; g < B->groups.size(); ++g) MG_CUDA(cudaStreamWaitEvent(B->gst[g], B->ev_joint, 0));
    return MG_OK;
}

// One FP32 defect-correction step of every group with unconverged problems is enqueued (no synchronisation).  With
// the joint tail every V-cycle is three stages: each group's steps down to its tail level (on its own stream), the
// joint tail of all groups (one cooperative launch), each group's steps back up.
mg_status enqueue_step(mg_batch *B, int m) {
    MG_TRY(fork(B));
    if (B->tail_mode == 2) {
        for (mg_forest *F : B->groups) MG_TRY(enqueue_done(F));
        for (int c = 0; c < m; ++c) {
            for (mg_forest *F : B->groups) vcycle32_part(F, 1);
            MG_TRY(enqueue_joint_tail(B));
            for (mg_forest *F : B->groups) vcycle32_part(F, 2);
        }
        for (mg_forest *F : B->groups) {
            MG_TRY(enqueue_update_mixed(F));
            MG_TRY(enqueue_scales(F));
            MG_TRY(enqueue_residual(F));
            MG_TRY(enqueue_problem_sums(F));
        }
        return join(B);
    }
    for (mg_forest *F : B->groups) {
        MG_TRY(enqueue_done(F));
        MG_TRY(enqueue_fp32_step(F, m));
        MG_TRY(enqueue_scales(F));
        MG_TRY(enqueue_residual(F));
        MG_TRY(enqueue_problem_sums(F));
    }
    return join(B);
}

// Tail mode 0 / 1 / 2 with the tuned tail levels (mode 0 turns every group's tail off).
mg_status apply_tail_mode(mg_batch *B, int mode) {
    for (size_t g = 0; g < B->groups.size(); ++g) {
        mg_forest *F = B->groups[g];
        const int lt = mode == 0 ? -1 : B->tuned_tails[g];
        if (lt >= 0 && F->tail_for != lt) MG_TRY(record_tail(F, lt));
        F->tail_level = lt;
    }
    B->tail_mode = mode;
    if (mode == 2) MG_TRY(build_joint_tail(B));
    return MG_OK;
}

// The groups' tail levels were tuned one group at a time; run concurrently, a cooperative tail launch may wait for
// other groups' kernels to leave the SMs it needs.  So the batch times one defect-correction step of all groups in
// each tail mode -- every level launched, each group's own tail, one joint tail per V-cycle -- (one untimed and two
// timed steps each, on the groups' pools, which are dead between solves) and keeps the fastest, a persistent mode
// when it is within 1 % of it.
mg_status tune_batch_tails(mg_batch *B) {
    B->tuned_tails.clear();
    bool any = false;
    for (mg_forest *F : B->groups) {
        B->tuned_tails.push_back(F->tail_level);
        any = any || F->tail_level >= 0;
        set_scales_host(F, std::vector<double>(F->np, 1.0));
    }
    if (!any) return apply_tail_mode(B, 0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    MG_CUDA(cudaEventCreate(&e0));
    MG_CUDA(cudaEventCreate(&e1));
    float ms[3] = {0.0f, 0.0f, 0.0f};
    const int m = std::max(1, B->cfg.inner_cycles);
    mg_status st = MG_OK;
    for (int v = 0; v < 3 && st == MG_OK; ++v) {
        if ((st = apply_tail_mode(B, v)) != MG_OK) break;
        if ((st = enqueue_step(B, m)) != MG_OK) break;
        if (cudaEventRecord(e0, B->st) != cudaSuccess) st = MG_ERR_CUDA;
        for (int r = 0; r < 2 && st == MG_OK; ++r) st = enqueue_step(B, m);
        if (st == MG_OK && (cudaEventRecord(e1, B->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms[v], e0, e1) != cudaSuccess))
            st = MG_ERR_CUDA;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != MG_OK) {
        if (st == MG_ERR_CUDA) set_error("timing the batch tails failed");
        return st;
    }
    // the fastest, except that the persistent modes (fewer launches, less host work per step) win ties within 1 %
    int best = 0;
    for (int v = 1; v < 3; ++v)
        if (ms[v] < ms[best]) best = v;
    for (int v = 2; v > best; --v)
        if (ms[v] <= 1.01f * ms[best]) {
            best = v;
            break;
        }
    MG_TRY(apply_tail_mode(B, best));
    for (mg_forest *F : B->groups) MG_TRY(check_kernel_waits(F));
    return MG_OK;
}

bool profiling(const mg_batch *B) {
    for (const mg_forest *F : B->groups)
        if (F->prof) return true;
    return false;
}

mg_status batch_solve(mg_batch *B, double *u_dev, double rtol, int max_cycles, int32_t *cycles_out,
                      double *rel_out) {
    if (!B->rhs_set) {
        set_error("mg_batch_set_rhs has not been called");
        return MG_ERR_STATE;
    }
    if (B->cfg.precision != 1) {
        set_error("batched solves run FP32 cycles inside FP64 defect correction (precision = 1)");
        return MG_ERR_INVALID_ARG;
    }
    MG_TRY(enter(B));
    MG_TRY(fork(B));
    const size_t G = B->groups.size();
    for (mg_forest *F : B->groups) reset_done(F);
    std::vector<std::vector<double>> fn(G), mult(G), rel(G), rr(G);
    std::vector<std::vector<int32_t>> met(G);
    for (size_t g = 0; g < G; ++g) {
        mg_forest *F = B->groups[g];
        bool zero_guess = false;
        MG_TRY(pack_initial_guess(F, u_dev, &zero_guess));
        fn[g].resize(F->np);
        mult[g].resize(F->np);
        rel[g].assign(F->np, -1.0);
        rr[g].assign(F->np, 0.0);
        met[g].assign(F->np, -1);
        for (int p = 0; p < F->np; ++p) {
            fn[g][p] = F->fnorm_p[p] > 0.0 ? F->fnorm_p[p] : 1.0;
            mult[g][p] = pow2_near(1.0 / fn[g][p]);
        }
        set_scales_host(F, mult[g]);
        MG_TRY(enqueue_scales(F));
        MG_TRY(enqueue_residual(F, zero_guess));  // a zero guess needs no operator: r = f
        MG_TRY(enqueue_problem_sums(F));
    }
    MG_TRY(join(B));
    int done = 0;
    bool all = false, finite = true;
    const int inner = std::max(1, B->cfg.inner_cycles);
    for (;;) {
        MG_CUDA(cudaStreamSynchronize(B->st));
        all = true;
        for (size_t g = 0; g < G; ++g) {
            mg_forest *F = B->groups[g];
            for (int p = 0; p < F->np; ++p) {
                if (F->pdone_h[p]) continue;  // masked out since it met rtol: keeps that residual
                rr[g][p] = F->psum_h[p] / (mult[g][p] * mult[g][p]);
                rel[g][p] = std::sqrt(rr[g][p]) / fn[g][p];
                if (!std::isfinite(rel[g][p])) finite = false;
                if (rel[g][p] <= rtol && met[g][p] < 0) {
                    met[g][p] = done;
                    F->pdone_h[p] = 1;  // copied to the device at the start of the next step
                }
                if (!(rel[g][p] <= rtol)) all = false;
            }
        }
        if (all || !finite || done >= max_cycles) break;
        const int m = std::min(inner, max_cycles - done);
        // scales of the next residual; the update of this step still uses the previous ones (device pinv)
        for (size_t g = 0; g < G; ++g) {
            for (int p = 0; p < B->groups[g]->np; ++p)
                if (!B->groups[g]->pdone_h[p]) mult[g][p] = pow2_near(1.0 / std::sqrt(rr[g][p]));
        }
        // the update reads pinv on the device before the captured copies overwrite it: keep host copies of the
        // new scales until the step is enqueued
        if (m == inner && !profiling(B)) {
            std::vector<int> tails;
            for (mg_forest *F : B->groups) tails.push_back(F->tail_level);
            tails.push_back(B->tail_mode);
            if (!B->graph || B->graph_m != m || B->graph_tails != tails) {
                if (B->graph) cudaGraphExecDestroy(B->graph);
                B->graph = nullptr;
                cudaGraph_t graph = nullptr;
                MG_CUDA(cudaStreamBeginCapture(B->st, cudaStreamCaptureModeThreadLocal));
                mg_status es = enqueue_step(B, m);
                cudaError_t ce = cudaStreamEndCapture(B->st, &graph);
                if (es != MG_OK) return es;
                if (ce != cudaSuccess) {
                    set_error(std::string("graph capture: ") + cudaGetErrorString(ce));
                    return MG_ERR_CUDA;
                }
                ce = cudaGraphInstantiate(&B->graph, graph, 0);
                cudaGraphDestroy(graph);
                if (ce != cudaSuccess) {
                    set_error(std::string("graph instantiate: ") + cudaGetErrorString(ce));
                    return MG_ERR_CUDA;
                }
                B->graph_m = m;
                B->graph_tails = tails;
            }
            for (size_t g = 0; g < G; ++g) set_scales_host(B->groups[g], mult[g]);
            MG_CUDA(cudaGraphLaunch(B->graph, B->st));
        } else {
            for (size_t g = 0; g < G; ++g) set_scales_host(B->groups[g], mult[g]);
            MG_TRY(enqueue_step(B, m));
        }
        done += m;
    }
    MG_TRY(fork(B));
    for (size_t g = 0; g < G; ++g) {
        mg_forest *F = B->groups[g];
        DevLevel &d = F->L[0];
        k_unpack<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(u_dev, d.u64, d.g, F->leaf_off);
        for (int p = 0; p < F->np; ++p) {
            const int32_t bp = B->gprob[g][p];
            if (cycles_out) cycles_out[bp] = met[g][p] >= 0 ? met[g][p] : done;
            if (rel_out) rel_out[bp] = rel[g][p];
        }
    }
    for (mg_forest *F : B->groups) reset_done(F);
    MG_TRY(join(B));
    MG_CUDA(cudaGetLastError());
    MG_TRY(leave(B));
    MG_CUDA(cudaStreamSynchronize(B->st));
    for (mg_forest *F : B->groups) MG_TRY(check_kernel_waits(F));
    if (!finite) {
        set_error("residual is not finite");
        return MG_ERR_NOT_CONVERGED;
    }
    if (!all) {
        set_error("some problems did not reach rtol within " + std::to_string(done) + " cycles");
        return MG_ERR_NOT_CONVERGED;
    }
    return MG_OK;
}

}  // namespace
}  // namespace octmg

using namespace octmg;

extern "C" {

mg_status mg_batch_create(const mg_config *cfg, const int32_t *problem_n, mg_batch **out) {
    if (out) *out = nullptr;
    if (!cfg || !out || !cfg->leaves || cfg->n_leaves <= 0) {
        set_error("null config, output or leaves");
        return MG_ERR_INVALID_ARG;
    }
    const int np = std::max(1, cfg->n_problems);
    std::vector<int32_t> pn(np, cfg->n);
    if (problem_n)
        for (int p = 0; p < np; ++p) pn[p] = problem_n[p];
    for (int p = 0; p < np; ++p)
        if (pn[p] < 4 || (pn[p] & (pn[p] - 1)) != 0 || pn[p] > 1024) {
            set_error("problem " + std::to_string(p) + ": block size must be a power of two in 4..1024");
            return MG_ERR_BLOCK_SIZE;
        }
    mg_batch *B = new (std::nothrow) mg_batch();
    if (!B) return MG_ERR_OOM;
    B->cfg = *cfg;
    B->cfg.leaves = nullptr;
    B->np = np;
    B->user = static_cast<cudaStream_t>(cfg->stream);
    auto fail = [&](mg_status s) {
        destroy_batch(B);
        return s;
    };
    if (cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_joint, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&B->flag, sizeof(int)) != cudaSuccess) {
        set_error("batch stream / event / flag allocation failed");
        return fail(MG_ERR_CUDA);
    }
    // leaf offsets in the caller's layout (leaves in order, each n_p^3 cells), groups by block size
    std::vector<int64_t> off(cfg->n_leaves);
    int64_t run = 0;
    for (int i = 0; i < cfg->n_leaves; ++i) {
        const int32_t p = cfg->leaves[5 * static_cast<int64_t>(i)];
        if (p < 0 || p >= np) {
            set_error("leaf problem index outside 0..n_problems-1");
            return fail(MG_ERR_INVALID_ARG);
        }
        off[i] = run;
        run += static_cast<int64_t>(pn[p]) * pn[p] * pn[p];
    }
    B->total_cells = run;
    std::map<int32_t, std::vector<int32_t>> byn;
    for (int p = 0; p < np; ++p) byn[pn[p]].push_back(p);
    for (auto &kv : byn) {
        std::vector<int32_t> local(np, -1);
        for (size_t q = 0; q < kv.second.size(); ++q) local[kv.second[q]] = static_cast<int32_t>(q);
        std::vector<int32_t> rows;
        std::vector<int64_t> goff;
        for (int i = 0; i < cfg->n_leaves; ++i) {
            const int32_t *r = cfg->leaves + 5 * static_cast<int64_t>(i);
            if (local[r[0]] < 0) continue;
            rows.insert(rows.end(), {local[r[0]], r[1], r[2], r[3], r[4]});
            goff.push_back(off[i]);
        }
        mg_config gc = *cfg;
        gc.n = kv.first;
        gc.n_leaves = static_cast<int32_t>(goff.size());
        gc.leaves = rows.data();
        gc.n_problems = static_cast<int32_t>(kv.second.size());
        cudaStream_t gs = nullptr;
        cudaEvent_t ge = nullptr;
        if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess) {
            set_error("group stream creation failed");
            return fail(MG_ERR_CUDA);
        }
        B->gst.push_back(gs);
        if (cudaEventCreateWithFlags(&ge, cudaEventDisableTiming) != cudaSuccess) {
            set_error("group event creation failed");
            return fail(MG_ERR_CUDA);
        }
        B->gev.push_back(ge);
        gc.stream = gs;
        mg_forest *F = nullptr;
        mg_status st = create(&gc, &F);
        if (st != MG_OK) return fail(st);
        B->groups.push_back(F);
        B->gn.push_back(kv.first);
        B->gprob.push_back(kv.second);
        F->batch_member = true;
        void *p = nullptr;
        if ((st = forest_alloc(F, &p, static_cast<int64_t>(goff.size() * sizeof(int64_t)))) != MG_OK) return fail(st);
        F->leaf_off = static_cast<int64_t *>(p);
        // same stream as the zero-fill of the allocation, then wait: the host vector dies at the end of the loop
        if (cudaMemcpyAsync(F->leaf_off, goff.data(), goff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, F->st) !=
                cudaSuccess ||
            cudaStreamSynchronize(F->st) != cudaSuccess) {
            set_error("leaf offset upload failed");
            return fail(MG_ERR_CUDA);
        }
    }
    *out = B;
    return MG_OK;
}

void mg_batch_destroy(mg_batch *B) { destroy_batch(B); }

mg_status mg_batch_set_rhs(mg_batch *B, const double *f_dev, const double *k_dev) {
    if (!B || !f_dev || (B->cfg.coeff && !k_dev)) {
        set_error("null batch, f, or k for a coefficient problem");
        return MG_ERR_INVALID_ARG;
    }
    MG_TRY(enter(B));
    MG_CUDA(cudaMemsetAsync(B->flag, 0, sizeof(int), B->st));
    k_check_batch<<<grid_for(B->total_cells), kThreads, 0, B->st>>>(f_dev, B->cfg.coeff ? k_dev : nullptr,
                                                                   B->total_cells, B->flag);
    int hbad = 0;
    MG_CUDA(cudaMemcpyAsync(&hbad, B->flag, sizeof(int), cudaMemcpyDeviceToHost, B->st));
    MG_CUDA(cudaStreamSynchronize(B->st));
    if (hbad) {
        set_error(hbad & 2 ? "k must be finite and > 0" : "f has a non-finite entry");
        return MG_ERR_NONFINITE;
    }
    MG_TRY(fork(B));
    for (mg_forest *F : B->groups) MG_TRY(set_rhs(F, f_dev, k_dev));
    MG_TRY(join(B));
    if (!B->tails_tuned && B->cfg.precision == 1) {
        MG_TRY(tune_batch_tails(B));
        B->tails_tuned = true;
    } else if (B->tail_mode == 2) {
        MG_TRY(build_joint_tail(B));  // the groups' set-up may have moved what the tail arguments point to
    }
    B->rhs_set = true;
    MG_TRY(leave(B));
    return MG_OK;
}

mg_status mg_batch_solve(mg_batch *B, double *u_dev, double rtol, int32_t max_cycles, int32_t *cycles_out,
                         double *rel_res_out) {
    if (!B || !u_dev || max_cycles < 0 || !(rtol >= 0.0)) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    return batch_solve(B, u_dev, rtol, max_cycles, cycles_out, rel_res_out);
}

mg_status mg_batch_info(const mg_batch *B, int32_t *n_groups, int64_t *total_cells, int32_t *group_n,
                        int32_t *group_problems) {
    if (!B || !n_groups) {
        set_error("null argument");
        return MG_ERR_INVALID_ARG;
    }
    *n_groups = static_cast<int32_t>(B->groups.size());
    if (total_cells) *total_cells = B->total_cells;
    for (size_t g = 0; g < B->groups.size(); ++g) {
        if (group_n) group_n[g] = B->gn[g];
        if (group_problems) group_problems[g] = static_cast<int32_t>(B->gprob[g].size());
    }
    return MG_OK;
}

mg_status mg_batch_profile(mg_batch *B, int32_t enable) {
    if (!B) {
        set_error("null batch");
        return MG_ERR_INVALID_ARG;
    }
    for (mg_forest *F : B->groups) MG_TRY(mg_profile(F, enable));
    return MG_OK;
}

mg_status mg_batch_set_tail_mode(mg_batch *B, int32_t mode) {
    if (!B || mode < 0 || mode > 2) {
        set_error("null batch or tail mode outside 0..2");
        return MG_ERR_INVALID_ARG;
    }
    if (!B->tails_tuned) {
        set_error("mg_batch_set_rhs has not been called (the tail levels are tuned there)");
        return MG_ERR_STATE;
    }
    MG_TRY(apply_tail_mode(B, mode));
    for (mg_forest *F : B->groups) MG_TRY(check_kernel_waits(F));
    return MG_OK;
}

mg_status mg_batch_get_tail_mode(const mg_batch *B, int32_t *mode) {
    if (!B || !mode) {
        set_error("null argument");
        return MG_ERR_INVALID_ARG;
    }
    *mode = B->tail_mode;
    return MG_OK;
}

mg_forest *mg_batch_group(mg_batch *B, int32_t g) {
    if (!B || g < 0 || g >= static_cast<int32_t>(B->groups.size())) return nullptr;
    return B->groups[g];
}

}  // extern "C"
