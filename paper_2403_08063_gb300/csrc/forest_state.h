// Forest state shared by the solver translation units: device level structures and the opaque mg_forest.
#pragma once
#include <algorithm>
#include <cstdio>
#include <string>
#include <utility>
#include <array>
#include <vector>

#include <cuda_runtime.h>

#include "kernels.cuh"
#include "octmg_internal.h"

namespace octmg {

#define MG_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                     \
            return MG_ERR_CUDA;                                                                \
        }                                                                                      \
    } while (0)

#define MG_TRY(expr)                      \
    do {                                  \
        mg_status s_ = (expr);            \
        if (s_ != MG_OK) return s_;       \
    } while (0)

constexpr int kMaxGrid = 152 * 32;  // grid-stride loops: at most 32 CTAs of 256 threads per SM

inline int grid_for(int64_t total) {
    int64_t g = (total + kThreads - 1) / kThreads;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, kMaxGrid)));
}

struct DevLevel {
    LevelGeom g{};
    FaceItem *faces = nullptr;
    int nfaces = 0;
    SegItem *segs = nullptr;
    int nsegs = 0;
    XferItem *xfer = nullptr;  // from this level to the next (per block of the next level)
    double *h2_64 = nullptr, *ih2_64 = nullptr, *vol_64 = nullptr;  // per block h^2, 1/h^2, h^3
    float *h2_32 = nullptr, *ih2_32 = nullptr, *vol_32 = nullptr;
    double *u64 = nullptr, *f64 = nullptr;
    double *u64b = nullptr;  // second FP64 iterate pool (damped Jacobi)
    float *u32 = nullptr, *f32 = nullptr;
    double *k64 = nullptr, *tx = nullptr, *ty = nullptr, *tz = nullptr, *dg = nullptr, *dinv = nullptr;
    float *kap = nullptr;
    int32_t *bprob = nullptr;  // problem of each block
    int32_t *nbr6 = nullptr;   // per block face: same-level neighbour, -1 boundary, -2 refinement interface
    FaceItem *ifaces = nullptr;  // the C2F faces alone (interface-only exchange)
    int nifaces = 0;
    int8_t *fkind = nullptr;   // per block face (b * 6 + 2 * axis + side): 0 boundary, 1 same, 2 C2F, 3 F2C
    bool all_halve = false;  // every block of the next level is a halved block of this one
    // FP32 smoother launch shape (kind, parameters): {1, ZC, threads, 0, 0} k_smooth32, {2, TY, TZ, D, R}
    // k_smooth32t; kind 0 = not chosen yet
    std::array<int32_t, 5> s32{0, 0, 0, 0, 0};
    // adjoint work pools (allocated by the first adjoint call)
    double *a_ub = nullptr, *a_fb = nullptr, *a_z = nullptr, *a_tmp = nullptr;
    // FP32 transposed cycles (forests with FP32 forward cycles): natural-layout pools and rounded coefficients
    float *a32_ub = nullptr, *a32_fb = nullptr, *a32_z = nullptr, *a32_tmp = nullptr;
    float *a32_tx = nullptr, *a32_ty = nullptr, *a32_tz = nullptr, *a32_dg = nullptr, *a32_dinv = nullptr;
    // FP32 cycles on a face-averaged coarse level: its halved face coefficients (colour-split) and mode 3
    float *ax32 = nullptr, *ay32 = nullptr, *az32 = nullptr;
    bool face32 = false;
    DiagItem *edges = nullptr, *corners = nullptr;  // trilinear prolongation: edge / corner items of every block
    int nedges = 0, ncorners = 0;
    Coef c64() const { return Coef{tx, ty, tz, dg, dinv, nullptr, nullptr, nullptr, nullptr}; }
    Coef c32() const { return Coef{nullptr, nullptr, nullptr, nullptr, nullptr, kap, ax32, ay32, az32}; }
    int64_t pool_elems() const { return static_cast<int64_t>(g.nb) * g.bs; }
    int64_t cells() const { return static_cast<int64_t>(g.nb) << (3 * g.lg); }
};

// One FP32 level as the persistent tail kernel sees it.
struct TailLevel {
    LevelGeom g;
    float *u, *f;
    const float *kap, *h2, *ih2;
    const FaceItem *faces, *ifaces;
    const SegItem *segs;
    const XferItem *xfer;  // to the next level
    const int32_t *nbr6, *bprob;
    int nfaces, nifaces, nsegs;
    int fast;  // the transfers to the next level use the specialised kernels (every block halves, edge 8..128)
    const float *ax, *ay, *az;  // halved face coefficients of a face-averaged coarse level (mode 3)
    int face32;                 // 1: this level's smoothing, ghosts and restriction use them
};

// One step of the tail's V-cycle; every step is followed by a grid barrier.
enum TailOp : int32_t {
    T_SMOOTH0 = 0, T_SMOOTH1, T_FACES_IFACE, T_FACES_FULL, T_SEGS, T_RESTRICT, T_PROLONG, T_COARSE
};
struct TailPhase {
    int32_t op, level;
};

// Everything the tail kernel reads of one forest (its level descriptors, phase list, coarsest inverse, done-mask and
// the barrier and error words of its launch).
struct TailArgs {
    const TailLevel *L;
    const TailPhase *ph;
    int nph;
    int flux;  // conservative F2C ghosts
    const double *Ainv;
    const int64_t *cmap32;
    const int32_t *uprob;
    const int64_t *ustart, *moff;
    int Nc;
    const uint8_t *done;
    unsigned *bar;  // [count, generation]
    int *err;
};

// One entry of a batch's joint tail: phase P of group `group`'s recorded tail; a grid barrier follows the entry when
// `last` is set (the entries between two barriers belong to different groups and are independent).
struct BatchEntry {
    int32_t group, last;
    TailPhase P;
};

}  // namespace octmg

struct mg_forest {
    mg_config cfg{};
    cudaStream_t st = nullptr;
    octmg::HostHierarchy H;
    std::vector<octmg::DevLevel> L;
    std::vector<void *> allocs;
    double *Ainv = nullptr;
    int64_t *cmap = nullptr;    // coarsest unknowns' offsets in the FP64 pools (natural layout)
    int64_t *cmap32 = nullptr;  // ... and in the colour-split FP32 pools
    int Nc = 0;
    double *partial = nullptr;  // 2 * kMaxGrid
    double *sums = nullptr;     // 2 doubles on the device
    double *pinned = nullptr;   // 2 doubles, host pinned
    double *s64a = nullptr, *s64b = nullptr;  // level-0 FP64 scratch pools
    double *coarse_r = nullptr;               // coarsest-level scratch pool (operator assembly)
    int *flag = nullptr;                      // input-check flag
    double *gb = nullptr;                     // 2 g on the finest level's boundary faces (mg_set_boundary), or null
    double *gb_pool = nullptr;                // its storage (kept when g is reset to 0)
    double omega = 0.8;                       // damping of the Jacobi smoother
    int *kerr = nullptr;                      // set by a device wait that gave up (staged smoother)
    double *AinvT = nullptr;                  // transpose of the coarsest inverses (adjoint cycles)
    int32_t *gj_piv = nullptr, *gj_src = nullptr;  // device Gauss-Jordan: pivot rows, column permutation
    double *gj_pinv = nullptr;                 // and the current pivot's reciprocal, per problem
    cudaGraphExec_t coarse_graph = nullptr;    // recorded coarsest-level probe + inversion (assemble_coarse)
    int coarse_runs = 0;                       // calls of assemble_coarse so far
    bool coarse_nograph = false;               // its recording failed: launched directly
    cudaStream_t cap_st = nullptr;             // private stream: graph recording, host-input copies
    cudaGraphExec_t v64_graph = nullptr;       // one recorded FP64 V-cycle (vcycle64_step), replayed per cycle
    int v64_runs = 0;                          // FP64 V-cycles run so far (recording starts at the second)
    bool v64_nograph = false;                  // the recording failed or is not replayable: launched directly
    double *hst_f = nullptr, *hst_k = nullptr, *hst_u = nullptr;  // mg_solve_host staging buffers (user layout)
    cudaEvent_t hst_ev = nullptr;              // orders the staging copies against the forest's stream
    int8_t *pcol = nullptr;                    // colour probe (interface-free coarsest level): colour per unknown
    int32_t *pnbu = nullptr;                   // and the unknowns of its 7-point neighbourhood (-1: outside)
    // several independent problems: per-problem reductions, scales, block-diagonal coarsest inverse
    int np = 1;
    int32_t *pstart = nullptr, *pblk = nullptr;  // level-0 blocks of problem p: pblk[pstart[p] .. pstart[p+1])
    double *bsum = nullptr;                      // per-CTA partial sums of h^3 x^2 over level 0, bsum_cpb per block
    int bsum_cpb = 1;
    double *psum = nullptr, *psum_h = nullptr;   // per-problem sums (device, pinned host)
    float *pscale = nullptr, *pscale_h = nullptr;  // per-problem power-of-two residual scale (device, pinned host)
    double *pinv = nullptr, *pinv_h = nullptr;     // its inverse in FP64
    uint8_t *pdone = nullptr, *pdone_h = nullptr;  // per problem: met rtol in the running solve (device, pinned host)
    int32_t *uprob = nullptr;                    // coarsest unknown -> problem
    int64_t *ustart = nullptr, *moff = nullptr;  // coarsest unknowns / inverse offsets per problem
    std::vector<int64_t> ustart_h, moff_h;
    std::vector<double> fnorm_p;                 // ||f|| per problem
    int64_t *leaf_off = nullptr;                 // optional: start of every leaf in the user arrays (elements)
    bool batch_member = false;                   // inputs are checked by the owning batch
    double *a_g = nullptr, *a_lam = nullptr;  // adjoint right-hand side and solution (level 0)
    bool rhs_set = false;
    double fnorm = 0.0;
    // per-kernel-family launch counters (always on) and CUDA-event timing (mg_profile)
    bool prof = false;
    int64_t nlaunch[32] = {};
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> recs;  // (family, index of the start event; stop = +1)
    // persistent tail: the FP32 V-cycle from level tail_level down is one cooperative launch (tail_level < 0: off)
    int tail_level = -1;
    bool tail_tuned = false;
    octmg::TailLevel *tail_L = nullptr;  // device copy of the level descriptors
    octmg::TailPhase *tail_ph = nullptr;  // device phase list
    int tail_nph = 0, tail_for = -2;      // phases recorded, and for which tail level
    unsigned *tail_bar = nullptr;          // grid-barrier counter and generation
    std::vector<octmg::TailPhase> tail_ph_host;  // host copy of the phase list (merged into a batch's joint tail)
};


namespace octmg {
// Kernel families for launch counting and timing.
enum ProfCat {
    P_EXCH64 = 0, P_EXCH32, P_SMOOTH64, P_SMOOTH32, P_RESTR64, P_RESTR32, P_PROL64, P_PROL32, P_COARSE64,
    P_COARSE32, P_RESID64, P_UPDATE, P_LAYOUT, P_ADJ, P_SMOOTH64_L0, P_SMOOTH32_L0, P_TAIL32, P_NCAT
};
template <typename T> constexpr int cat_of(int cat64) { return sizeof(T) == 8 ? cat64 : cat64 + 1; }

cudaEvent_t next_event(mg_forest *F);

// RAII scope around the launches of one kernel family (a negative family: no accounting).
struct Prof {
    mg_forest *F;
    int cat;
    size_t start = 0;
    bool on = false;
    Prof(mg_forest *f, int c, int launches) : F(f), cat(c) {  // c < 0: inside another family's scope, not counted
        if (c < 0) return;
        F->nlaunch[c] += launches;
        if (F->prof) {
            cudaEvent_t a = next_event(F), b = next_event(F);
            if (a && b) {
                start = F->ev_used - 2;
                cudaEventRecord(a, F->st);
                on = true;
            }
        }
    }
    ~Prof() {
        if (on) {
            cudaEventRecord(F->ev_pool[start + 1], F->st);
            F->recs.emplace_back(cat, start);
        }
    }
};

inline std::string fmt_e(double v) {
    char b[32];
    std::snprintf(b, sizeof(b), "%.3e", v);
    return b;
}

// FP64 operator application A u on a level (ghosts of u already exchanged), defined in solver.cu.
void apply64(mg_forest *F, DevLevel &d, const double *u, double *out);

// FP64 ghost exchange of one level on a pool laid out like the level's pools (defined in solver.cu).
void exchange_any64(mg_forest *F, DevLevel &d, double *u);
// Device allocation owned by the forest (freed by mg_forest_destroy), zero-filled (defined in solver.cu).
mg_status forest_alloc(mg_forest *F, void **p, int64_t bytes);
mg_status check_ready(mg_forest *F);
mg_status check_kernel_waits(mg_forest *F);
mg_status launch_tail32(mg_forest *F);  // tail.cu
octmg::TailArgs tail_args(mg_forest *F);  // tail.cu: the forest's recorded tail as the kernel reads it
// tail.cu: a batch's joint tail, one cooperative launch on groups[0]'s stream walking `ne` entries (device) over the
// groups' tail arguments (device), with a grid of at most `need` CTAs
mg_status launch_batch_tail32(mg_forest *const *groups, const octmg::TailArgs *args, const octmg::BatchEntry *entries,
                              int ne, unsigned *bar, int64_t need);
int64_t tail_ctas(mg_forest *F);  // tail.cu: CTAs the largest phase of F's tail can use
// solver.cu: one FP32 V-cycle in two parts around a joint tail: part 1 the steps down to the tail level's entry,
// part 2 the steps after the tail (0: the whole cycle, its tail launched as usual)
void vcycle32_part(mg_forest *F, int part);
mg_status enqueue_update_mixed(mg_forest *F);  // solver.cu: u64 += e32 / scale_p
mg_status record_tail(mg_forest *F, int l);   // solver.cu
mg_status launch_selftest_wait(mg_forest *F, int which);  // tail.cu (F->tail_bar allocated)
void reset_done(mg_forest *F);
mg_status enqueue_done(mg_forest *F);
mg_status reference_norms(mg_forest *F);
mg_status ensure_scratch64(mg_forest *F);
mg_status create(const mg_config *cfg, mg_forest **out);
mg_status set_rhs(mg_forest *F, const double *f_dev, const double *k_dev);
double pow2_near(double x);
void set_scales_host(mg_forest *F, const std::vector<double> &mult);
mg_status enqueue_scales(mg_forest *F);
// FP64 residual -> FP32 scaled rhs, zeroed correction, per-block sums (zero_u: u is zero, r = f)
mg_status enqueue_residual(mg_forest *F, bool zero_u = false);
mg_status pack_initial_guess(mg_forest *F, const double *u_dev, bool *zero);
mg_status enqueue_problem_sums(mg_forest *F);  // per-problem sums -> pinned psum_h (no synchronisation)
mg_status enqueue_fp32_step(mg_forest *F, int cycles);  // `cycles` FP32 V-cycles and the FP64 update

mg_status ensure_fp64_coefficients(mg_forest *F);
}  // namespace octmg
