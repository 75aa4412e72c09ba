// The persistent tail of the FP32 V-cycle: every level from `tail_level` down to the coarsest, and back up to the
// end of that level's post-smoothing, in one cooperative launch.  The coarse levels of a V-cycle are small (a few
// thousand to a few hundred thousand cells) and their kernels last a few microseconds each, so launching them one
// by one is latency-bound; here the CTAs stay resident and walk a phase list recorded from the same schedule as the
// launched V-cycle (smoothing half-sweeps, interface and full exchanges, restriction, prolongation, coarsest
// solve), separated by grid barriers.  Every phase runs the same device code as the corresponding kernel (loads of
// data written by earlier phases go through L2), so results are bit-identical to the launched V-cycle.  No
// counterpart in the paper, whose generated code runs the cycle level by level (Sec. 4).
#include "forest_state.h"
#include "kernels.cuh"

namespace octmg {

constexpr int kTailThreads = 256;

// Grid barrier for a cooperative launch: arrive on a counter, the last CTA resets it and advances the generation,
// the others poll the generation (no sleep: a phase of the tail lasts microseconds).  The wait is bounded by the SM
// clock (2^30 cycles, about half a second): it then sets *err and returns false (the kernel stops; the host
// reports MG_ERR_TIMEOUT).
__device__ bool grid_barrier(unsigned *count, unsigned *gen, int *err, unsigned expected) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *vg = gen;
        const unsigned g0 = *vg;
        __threadfence();
        if (atomicAdd(count, 1u) == expected - 1) {
            atomicExch(count, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vg == g0) {
                if (clock64() - t0 > (1LL << 30)) {
                    atomicOr(err, 2);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <int MODE, int LG>
__device__ __forceinline__ void tail_smooth(const TailLevel &d, int colour, Skip skip, int64_t t0, int64_t ts) {
    const int64_t work = d.g.nb * (int64_t(1) << (3 * LG - 1));
    for (int64_t t = t0; t < work; t += ts)
        smooth32_column<MODE, LG, 1, true>(d.u, d.f, d.kap, d.h2, d.g.bs, colour, d.nbr6, skip, t, d.ax, d.ay, d.az);
}

template <int MODE, int LG>
__device__ __forceinline__ void tail_restrict(const TailLevel &d, const TailLevel &c, Skip skip, int64_t t0,
                                              int64_t ts) {
    residual_restrict32_body<MODE, LG, true>(d.u, d.f, d.kap, d.ih2, d.g.bs, c.f, c.u, d.xfer, c.g.nb, c.g.bs, skip,
                                             t0, ts, d.ax, d.ay, d.az);
}

// The phases that read the level's coefficients (smoothing, conservative fine-to-coarse ghosts, residual +
// restriction), in coefficient mode M; the others do not depend on it.
template <int M>
__device__ __forceinline__ void tail_coef_phase(const TailArgs &a, const TailPhase &P, const TailLevel &d, Skip skip,
                                                int64_t t0, int64_t ts) {
    const Coef cf{nullptr, nullptr, nullptr, nullptr, nullptr, d.kap, d.ax, d.ay, d.az};
    switch (P.op) {
        case T_SMOOTH0:
        case T_SMOOTH1: {
            const int colour = P.op == T_SMOOTH1;
            switch (d.g.lg) {
                case 2: tail_smooth<M, 2>(d, colour, skip, t0, ts); break;
                case 3: tail_smooth<M, 3>(d, colour, skip, t0, ts); break;
                case 4: tail_smooth<M, 4>(d, colour, skip, t0, ts); break;
                case 5: tail_smooth<M, 5>(d, colour, skip, t0, ts); break;
                case 6: tail_smooth<M, 6>(d, colour, skip, t0, ts); break;
                default: tail_smooth<M, 7>(d, colour, skip, t0, ts); break;
            }
            break;
        }
        case T_SEGS:
            if (a.flux)
                exchange_segs_body<float, M, true, true>(d.u, cf, d.segs, d.nsegs, d.g, skip, t0, ts);
            else
                exchange_segs_body<float, M, false, true>(d.u, cf, d.segs, d.nsegs, d.g, skip, t0, ts);
            break;
        default: {  // T_RESTRICT
            const TailLevel &c = a.L[P.level + 1];
            const Skip cs{c.bprob, a.done};
            if (d.fast) {
                switch (d.g.lg) {
                    case 3: tail_restrict<M, 3>(d, c, cs, t0, ts); break;
                    case 4: tail_restrict<M, 4>(d, c, cs, t0, ts); break;
                    case 5: tail_restrict<M, 5>(d, c, cs, t0, ts); break;
                    case 6: tail_restrict<M, 6>(d, c, cs, t0, ts); break;
                    default: tail_restrict<M, 7>(d, c, cs, t0, ts); break;
                }
            } else {
                residual_restrict_body<float, M, true>(d.u, d.f, cf, d.ih2, d.g, c.f, c.u, d.xfer, c.g, cs, t0, ts);
            }
            break;
        }
    }
}

template <int LG>
__device__ __forceinline__ void tail_prolong(const TailLevel &d, const TailLevel &c, Skip skip, int64_t t0,
                                             int64_t ts) {
    prolong32_body<LG, true>(d.u, d.g.bs, c.u, d.xfer, c.g.nb, c.g.bs, d.nbr6, skip, t0, ts);
}

// One phase of a recorded tail, over every thread of the grid (thread t0 of ts).
template <int MODE>
__device__ __forceinline__ void tail_phase(const TailArgs &a, const TailPhase &P, int64_t t0, int64_t ts) {
    const TailLevel &d = a.L[P.level];
    const Skip skip{d.bprob, a.done};
    switch (P.op) {
        case T_SMOOTH0:
        case T_SMOOTH1:
        case T_SEGS:
        case T_RESTRICT:
            if (MODE == 2 && d.face32) tail_coef_phase<3>(a, P, d, skip, t0, ts);
            else tail_coef_phase<MODE>(a, P, d, skip, t0, ts);
            break;
        case T_FACES_IFACE:
            exchange_faces_body<float, false, true>(d.u, d.ifaces, d.nifaces, d.g, skip, t0, ts);
            break;
        case T_FACES_FULL:
            exchange_faces_body<float, false, true>(d.u, d.faces, d.nfaces, d.g, skip, t0, ts);
            break;
        case T_PROLONG: {
            const TailLevel &c = a.L[P.level + 1];
            const Skip cs{c.bprob, a.done};
            if (d.fast) {
                switch (d.g.lg) {
                    case 3: tail_prolong<3>(d, c, cs, t0, ts); break;
                    case 4: tail_prolong<4>(d, c, cs, t0, ts); break;
                    case 5: tail_prolong<5>(d, c, cs, t0, ts); break;
                    case 6: tail_prolong<6>(d, c, cs, t0, ts); break;
                    default: tail_prolong<7>(d, c, cs, t0, ts); break;
                }
            } else {
                prolong_body<float, true>(d.u, d.g, c.u, d.xfer, c.g, cs, t0, ts);
            }
            break;
        }
        default: {  // T_COARSE: one warp per coarsest unknown
            const int lane = threadIdx.x & 31;
            const int64_t w0 = t0 >> 5, wn = ts >> 5;
            for (int64_t w = w0; w < a.Nc; w += wn)
                coarse_solve_row<float, true>(d.u, d.f, a.Ainv, a.cmap32, a.uprob, a.ustart, a.moff, a.done,
                                              static_cast<int>(w), lane);
            break;
        }
    }
}

template <int MODE>
static __global__ void __launch_bounds__(kTailThreads) k_tail32(TailArgs a) {
    const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t ts = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int p = 0; p < a.nph; ++p) {
        tail_phase<MODE>(a, a.ph[p], t0, ts);
        if (!grid_barrier(a.bar, a.bar + 1, a.err, gridDim.x)) return;
    }
}

// The joint tail of a batch: the recorded tails of several forests (one per block size) in one launch.  Entries
// between two barriers are phases of different forests, which share no data, so the grid runs them back to back
// and synchronises once; each forest's own phases keep their order, each followed by a barrier as in k_tail32.
template <int MODE>
static __global__ void __launch_bounds__(kTailThreads) k_batch_tail32(const TailArgs *__restrict__ ga,
                                                                      const BatchEntry *__restrict__ e, int ne,
                                                                      unsigned *bar, int *err) {
    const int64_t t0 = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    const int64_t ts = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int i = 0; i < ne; ++i) {
        const BatchEntry E = e[i];
        tail_phase<MODE>(ga[E.group], E.P, t0, ts);
        if (E.last && !grid_barrier(bar, bar + 1, err, gridDim.x)) return;
    }
}

TailArgs tail_args(mg_forest *F) {
    return TailArgs{F->tail_L, F->tail_ph, F->tail_nph, F->cfg.interface_flux, F->Ainv, F->cmap32, F->uprob,
                    F->ustart, F->moff, F->Nc, F->pdone, F->tail_bar, F->kerr};
}

// CTAs the largest phase of F's recorded tail can use (one thread per updated cell of a half-sweep).
int64_t tail_ctas(mg_forest *F) {
    int64_t need = 1;
    for (int l = std::max(0, F->tail_level); l < static_cast<int>(F->L.size()); ++l)
        need = std::max<int64_t>(need, (F->L[l].cells() / 2 + kTailThreads - 1) / kTailThreads);
    return need;
}

// Cooperative launch of `fn` with one TailArgs-like argument list; grid: `need` CTAs, at most two per SM (all must
// be resident together).
static mg_status launch_cooperative(const void *fn, int slot, int64_t need, cudaStream_t st, void **args) {
    static int per_sm[4] = {-1, -1, -1, -1}, sms = 0;
    if (per_sm[slot] < 0) {
        int dev = 0, v = 0, sm = 0;
        MG_CUDA(cudaGetDevice(&dev));
        MG_CUDA(cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev));
        MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, fn, kTailThreads, 0));
        sms = sm;
        per_sm[slot] = std::max(1, std::min(v, 2));
    }
    const int grid = static_cast<int>(std::min<int64_t>(need, static_cast<int64_t>(per_sm[slot]) * sms));
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    MG_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    return MG_OK;
}

// Enqueues the recorded tail on the forest's stream (capturable: a memset and a cooperative kernel launch).
mg_status launch_tail32(mg_forest *F) {
    const int mi = F->cfg.coeff ? 1 : 0;
    const void *fn = mi ? reinterpret_cast<const void *>(k_tail32<2>) : reinterpret_cast<const void *>(k_tail32<0>);
    TailArgs a = tail_args(F);
    MG_CUDA(cudaMemsetAsync(F->tail_bar, 0, 2 * sizeof(unsigned), F->st));
    void *args[] = {&a};
    return launch_cooperative(fn, mi, tail_ctas(F), F->st, args);
}

// Enqueues a batch's joint tail on groups[0]'s stream (capturable), after that stream has waited for the others.
mg_status launch_batch_tail32(mg_forest *const *groups, const TailArgs *args, const BatchEntry *entries, int ne,
                              unsigned *bar, int64_t need) {
    mg_forest *F = groups[0];
    const int mi = F->cfg.coeff ? 1 : 0;
    const void *fn =
        mi ? reinterpret_cast<const void *>(k_batch_tail32<2>) : reinterpret_cast<const void *>(k_batch_tail32<0>);
    MG_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), F->st));
    int *err = F->kerr;
    void *kargs[] = {&args, &entries, &ne, &bar, &err};
    return launch_cooperative(fn, 2 + mi, need, F->st, kargs);
}

// Self-test of the bounded waits (mg_selftest_waits): one CTA waits for something that never happens and must give up
// with its error bit set.  which = 0: an mbarrier phase that no thread or copy completes (the wait of the staged
// smoother's copies, bit 1); which = 1: a grid barrier that expects one more CTA than the grid has (the persistent
// tail's, bit 2).
static __global__ void k_selftest_wait(int which, unsigned *bar, int *err) {
    __shared__ uint64_t mb;
    if (which == 0) {
        if (threadIdx.x == 0) {
            mbar_init(&mb, 1);
            mbar_init_fence();
        }
        __syncthreads();
        if (threadIdx.x == 0 && !mbar_wait(&mb, 0)) atomicOr(err, 1);
    } else {
        grid_barrier(bar, bar + 1, err, gridDim.x + 1);
    }
}

mg_status launch_selftest_wait(mg_forest *F, int which) {
    MG_CUDA(cudaMemsetAsync(F->tail_bar, 0, 2 * sizeof(unsigned), F->st));
    k_selftest_wait<<<1, 32, 0, F->st>>>(which, F->tail_bar, F->kerr);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

}  // namespace octmg
