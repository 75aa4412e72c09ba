// The forest object, the V-cycle driver and the C-ABI entry points (include/octmg.h).
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "forest_state.h"
#include "kernels.cuh"
#include "octmg_internal.h"

namespace octmg {

thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

template <typename T>
mg_status dalloc(mg_forest *F, T **p, int64_t count, bool zero = true) {
    void *q = nullptr;
    const size_t bytes = static_cast<size_t>(std::max<int64_t>(count, 1)) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA;
    }
    F->allocs.push_back(q);
    if (zero) MG_CUDA(cudaMemsetAsync(q, 0, bytes, F->st));
    *p = static_cast<T *>(q);
    return MG_OK;
}

template <typename T>
mg_status upload(mg_forest *F, T **p, const std::vector<T> &v) {
    MG_TRY(dalloc(F, p, static_cast<int64_t>(v.size()), false));
    if (!v.empty()) MG_CUDA(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));  // host vectors may die after return
    return MG_OK;
}

const char *const kProfNames[P_NCAT] = {"exchange_f64", "exchange_f32", "smooth_f64", "smooth_f32",
                                         "residual_restrict_f64", "residual_restrict_f32", "prolong_f64",
                                         "prolong_f32", "coarse_f64", "coarse_f32", "residual_f64",
                                         "update_mixed", "layout", "adjoint", "smooth_f64_finest",
                                         "smooth_f32_finest", "tail_f32"};

cudaEvent_t next_event(mg_forest *F) {
    if (F->ev_used == F->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        F->ev_pool.push_back(e);
    }
    return F->ev_pool[F->ev_used++];
}

mg_status forest_alloc(mg_forest *F, void **p, int64_t bytes) {
    char *q = nullptr;
    MG_TRY(dalloc(F, &q, bytes));
    *p = q;
    return MG_OK;
}

int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// ---------------------------------------------------------------------------------------------------------------
// Level operations
// ---------------------------------------------------------------------------------------------------------------
template <typename T> T *ufield(DevLevel &d);
template <> double *ufield<double>(DevLevel &d) { return d.u64; }
template <> float *ufield<float>(DevLevel &d) { return d.u32; }
template <typename T> T *ffield(DevLevel &d);
template <> double *ffield<double>(DevLevel &d) { return d.f64; }
template <> float *ffield<float>(DevLevel &d) { return d.f32; }
template <typename T> const T *h2_of(const DevLevel &d);
template <> const double *h2_of<double>(const DevLevel &d) { return d.h2_64; }
template <> const float *h2_of<float>(const DevLevel &d) { return d.h2_32; }
template <typename T> const T *ih2_of(const DevLevel &d);
template <> const double *ih2_of<double>(const DevLevel &d) { return d.ih2_64; }
template <> const float *ih2_of<float>(const DevLevel &d) { return d.ih2_32; }
template <typename T> Coef coef_of(const DevLevel &d);
template <> Coef coef_of<double>(const DevLevel &d) { return d.c64(); }
template <> Coef coef_of<float>(const DevLevel &d) { return d.c32(); }

// The done-mask view of a level for its kernels (all problems active outside a solve).
Skip skip_of(mg_forest *F, const DevLevel &d) { return Skip{d.bprob, F->pdone}; }

// Ghost exchange of a level: every face (full), or only the refinement-interface faces (C2F and F2C), whose
// ghosts the smoother's write-through does not maintain.
template <typename T, int MODE>
void exchange(mg_forest *F, DevLevel &d, T *u, bool interface_only = false, bool prof = true) {
    const FaceItem *items = interface_only ? d.ifaces : d.faces;
    const int nitems = interface_only ? d.nifaces : d.nfaces;
    if (!nitems && !d.nsegs) return;
    Prof p(F, prof ? cat_of<T>(P_EXCH64) : -1, (nitems ? 1 : 0) + (d.nsegs ? 1 : 0));
    const T *gb = nullptr;  // inhomogeneous Dirichlet data: FP64 finest level only
    if constexpr (sizeof(T) == 8)
        if (&d == &F->L[0]) gb = F->gb;
    if (nitems && interface_only) {  // C2F faces only: one CTA per fine face, shared intermediate extrapolations
        const int w = d.g.n / 2 + 2, threads = d.g.n <= 8 ? 32 : (d.g.n <= 32 ? 128 : 256);
        k_exchange_c2f_smem<T><<<nitems, threads, static_cast<size_t>(w) * w * sizeof(T), F->st>>>(
            u, items, d.g, skip_of(F, d), F->cfg.c2f_variant);
    }
    else if (nitems)
        k_exchange_faces<T, false><<<grid_for(static_cast<int64_t>(nitems) * d.g.n * d.g.n), kThreads, 0, F->st>>>(
            u, items, nitems, d.g, skip_of(F, d), F->cfg.c2f_variant, gb);
    if (d.nsegs) {
        const int64_t tot = static_cast<int64_t>(d.nsegs) * (d.g.n / 2) * (d.g.n / 2);
        if (F->cfg.interface_flux)
            k_exchange_segs<T, MODE, true><<<grid_for(tot), kThreads, 0, F->st>>>(u, coef_of<T>(d), d.segs, d.nsegs, d.g,
                                                                                skip_of(F, d));
        else
            k_exchange_segs<T, MODE, false><<<grid_for(tot), kThreads, 0, F->st>>>(u, coef_of<T>(d), d.segs, d.nsegs,
                                                                                 d.g, skip_of(F, d));
    }
}

void exchange_any64(mg_forest *F, DevLevel &d, double *u) {
    if (F->cfg.coeff) exchange<double, 1>(F, d, u);
    else exchange<double, 0>(F, d, u);
}

// Coefficient exchange: boundary copy, same-level copy, C2F injection, F2C mean (either interface variant).
void exchange_k(mg_forest *F, DevLevel &d) {
    if (d.nfaces)
        k_exchange_faces<double, true><<<grid_for(static_cast<int64_t>(d.nfaces) * d.g.n * d.g.n), kThreads, 0, F->st>>>(
            d.k64, d.faces, d.nfaces, d.g);
    if (d.nsegs)
        k_exchange_segs<double, 0, false><<<grid_for(static_cast<int64_t>(d.nsegs) * (d.g.n / 2) * (d.g.n / 2)), kThreads, 0,
                                             F->st>>>(d.k64, Coef{}, d.segs, d.nsegs, d.g);
}

// FP32 smoothers specialised for block edges 4..128.  Two kernels and their launch shapes (kind, parameters):
//   {1, ZC, threads, 0, 0}: k_smooth32, one column of ZC in {1, 2, 4} cells per thread, 128 / 256 / 512 threads;
//   {2, TY, TZ, D, R}:      k_smooth32t (edges 32..128), a CTA per TY rows x TZ planes of a block, other-colour planes
//                           staged in shared memory D + 1 ahead, R rows per thread (consumer threads = n/2 TY / R in
//                           128..512, plus one producer warp,
//                           TZ in {8, 16, 32, 64} up to n, D in {2, 4}, R in {1, 2, 4}).
// A shape only changes which thread updates a cell, never the arithmetic, so every shape gives identical bits.
using Shape = std::array<int32_t, 5>;
using Smooth32Fn = void (*)(float *, const float *, const float *, const float *, int64_t, int64_t, int,
                            const int32_t *, Skip, const float *, const float *, const float *);
#define OCTMG_S32(K, M, L) {K<M, L, 1>, K<M, L, 2>, K<M, L, 4>}
// [coefficient mode 0, 2, 3][block edge 2^2 .. 2^7][column length 1, 2, 4]
const Smooth32Fn kSmooth32[3][6][3] = {
    {OCTMG_S32(k_smooth32, 0, 2), OCTMG_S32(k_smooth32, 0, 3), OCTMG_S32(k_smooth32, 0, 4),
     OCTMG_S32(k_smooth32, 0, 5), OCTMG_S32(k_smooth32, 0, 6), OCTMG_S32(k_smooth32, 0, 7)},
    {OCTMG_S32(k_smooth32, 2, 2), OCTMG_S32(k_smooth32, 2, 3), OCTMG_S32(k_smooth32, 2, 4),
     OCTMG_S32(k_smooth32, 2, 5), OCTMG_S32(k_smooth32, 2, 6), OCTMG_S32(k_smooth32, 2, 7)},
    {OCTMG_S32(k_smooth32, 3, 2), OCTMG_S32(k_smooth32, 3, 3), OCTMG_S32(k_smooth32, 3, 4),
     OCTMG_S32(k_smooth32, 3, 5), OCTMG_S32(k_smooth32, 3, 6), OCTMG_S32(k_smooth32, 3, 7)}};
using Smooth32tFn = void (*)(float *, const float *, const float *, const float *, int64_t, int, const int32_t *, int,
                             int, int, int *, Skip, const float *, const float *, const float *);
// [coefficient mode 0, 2, 3][block edge 2^5 .. 2^7][rows per thread 1, 2, 4]
const Smooth32tFn kSmooth32t[3][3][3] = {
    {OCTMG_S32(k_smooth32t, 0, 5), OCTMG_S32(k_smooth32t, 0, 6), OCTMG_S32(k_smooth32t, 0, 7)},
    {OCTMG_S32(k_smooth32t, 2, 5), OCTMG_S32(k_smooth32t, 2, 6), OCTMG_S32(k_smooth32t, 2, 7)},
    {OCTMG_S32(k_smooth32t, 3, 5), OCTMG_S32(k_smooth32t, 3, 6), OCTMG_S32(k_smooth32t, 3, 7)}};
#undef OCTMG_S32

bool smooth32_specialised(const DevLevel &d) { return d.g.lg >= 2 && d.g.lg <= 7; }

size_t smooth32t_smem(int lg, int mode, int TY, int D) {
    return s32t_smem_bytes(s32t_plan(lg, s32t_arrays(mode), TY, D));
}

int ridx(int v) { return v == 4 ? 2 : (v == 2 ? 1 : 0); }

// FP32 coefficient mode of a level: 0 constant k, 2 1/k with harmonic means on the fly, 3 stored halved face
// coefficients (face-averaged coarse levels); and its index into the kernel tables.
int mode32(const mg_forest *F, const DevLevel &d) { return !F->cfg.coeff ? 0 : (d.face32 ? 3 : 2); }
int mode_index(int mode) { return mode == 3 ? 2 : (mode == 2 ? 1 : 0); }

// The shapes a level may use (the tuner's candidates): column kernels, and for edges 32..128 the staged kernel
// (1/k, or the three stored face arrays of mode 3, staged with u and f).
std::vector<Shape> smooth32_shapes(const DevLevel &d, int mode) {
    std::vector<Shape> v;
    const int n = d.g.n;
    for (int zc : {1, 2, 4})
        for (int th : {128, 256, 512})
            if (zc <= n) v.push_back({1, zc, th, 0, 0});
    if (d.g.lg >= 5)
        for (int R : {1, 2, 4})
            for (int th : {128, 256, 512})
                for (int tz : {8, 16, 32, 64})
                    for (int D : {2, 4}) {
                        const int TY = th * R / (n / 2);
                        if (TY >= R && TY <= n && tz <= n && smooth32t_smem(d.g.lg, mode, TY, D) <= 200 * 1024)
                            v.push_back({2, TY, tz, D, R});
                    }
    return v;
}

bool smooth32_shape_ok(const DevLevel &d, int mode, const Shape &sh) {
    for (const auto &c : smooth32_shapes(d, mode))
        if (c == sh) return true;
    return false;
}

void launch_smooth32(mg_forest *F, DevLevel &d, int colour, const Shape &sh, cudaStream_t st) {
    const int mode = mode32(F, d), mi = mode_index(mode);
    if (sh[0] == 2) {
        const int TY = sh[1], TZ = sh[2], D = sh[3], R = sh[4], n = d.g.n;
        const size_t smem = smooth32t_smem(d.g.lg, mode, TY, D);
        Smooth32tFn fn = kSmooth32t[mi][d.g.lg - 5][ridx(R)];
        static std::once_flag once[3][3][3];
        std::call_once(once[mi][d.g.lg - 5][ridx(R)], [&] {
            cudaFuncSetAttribute(reinterpret_cast<const void *>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
        });
        const int64_t grid = static_cast<int64_t>(d.g.nb) * (n / TY) * (n / TZ);
        fn<<<static_cast<unsigned>(grid), (n / 2) * TY / R + 32, smem, st>>>(d.u32, d.f32, d.kap, d.h2_32, d.g.bs, colour,
                                                                         d.nbr6, TY, TZ, D, F->kerr, skip_of(F, d),
                                                                         d.ax32, d.ay32, d.az32);
        return;
    }
    const int zc = sh[0] == 1 ? sh[1] : 1, threads = sh[0] == 1 ? sh[2] : kThreads;
    const int64_t work = (d.cells() / 2) >> ridx(zc);  // one thread per column of zc cells
    const int64_t grid = (work + threads - 1) / threads;
    kSmooth32[mode_index(mode)][d.g.lg - 2][ridx(zc)]<<<static_cast<unsigned>(grid), threads, 0, st>>>(
        d.u32, d.f32, d.kap, d.h2_32, work, d.g.bs, colour, d.nbr6, skip_of(F, d), d.ax32, d.ay32, d.az32);
}

// Reads and clears the device error word of bounded waits.
mg_status check_kernel_waits(mg_forest *F) {
    int h = 0;
    MG_CUDA(cudaMemcpyAsync(&h, F->kerr, sizeof(int), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (h) {
        MG_CUDA(cudaMemsetAsync(F->kerr, 0, sizeof(int), F->st));
        set_error(h & 1   ? "a staged smoother gave up waiting for its shared-memory copies"
                  : h & 4 ? "a staged restriction gave up waiting for its shared-memory copies"
                          : "the persistent tail kernel gave up waiting at a grid barrier");
        return MG_ERR_TIMEOUT;
    }
    return MG_OK;
}

// Launch-shape autotuner of the FP32 smoother: on every level with at least 2^18 cells, time both colours of each
// candidate shape (one untimed pair, then three timed pairs between CUDA events on the forest's stream) and keep
// the fastest.  It runs on the level's own FP32 pools, whose contents are dead between solves (each correction
// cycle rewrites f and zeroes u before reading them).  Choices are cached for the process per (device,
// coefficient mode, n, blocks); smaller levels, and every level while the stream is being captured, take
// {1, 1, 256, 0}.
mg_status tune_smooth32(mg_forest *F) {
    static std::mutex mu;
    static std::map<std::array<int64_t, 4>, Shape> cache;
    int dev = 0;
    MG_CUDA(cudaGetDevice(&dev));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MG_CUDA(cudaStreamIsCapturing(F->st, &cap));
    for (DevLevel &d : F->L) {
        if (!smooth32_specialised(d) || !d.u32 || d.s32[0]) continue;
        if (d.cells() < (int64_t(1) << 18) || cap != cudaStreamCaptureStatusNone) {
            d.s32 = {1, 1, kThreads, 0, 0};
            continue;
        }
        const std::array<int64_t, 4> key{dev, mode32(F, d), d.g.n, d.g.nb};
        {
            std::lock_guard<std::mutex> lk(mu);
            auto it = cache.find(key);
            if (it != cache.end()) {
                d.s32 = it->second;
                continue;
            }
        }
        cudaEvent_t e0 = next_event(F), e1 = next_event(F);
        if (!e0 || !e1) {
            set_error("cudaEventCreate failed");
            return MG_ERR_CUDA;
        }
        float best = 0.0f;
        Shape pick{1, 1, kThreads, 0, 0};
        for (const auto &sh : smooth32_shapes(d, mode32(F, d))) {
            launch_smooth32(F, d, 0, sh, F->st);
            launch_smooth32(F, d, 1, sh, F->st);
            MG_CUDA(cudaEventRecord(e0, F->st));
            for (int rep = 0; rep < 3; ++rep) {
                launch_smooth32(F, d, 0, sh, F->st);
                launch_smooth32(F, d, 1, sh, F->st);
            }
            MG_CUDA(cudaEventRecord(e1, F->st));
            MG_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (best == 0.0f || ms < best) {
                best = ms;
                pick = sh;
            }
        }
        F->ev_used -= 2;
        MG_CUDA(cudaGetLastError());
        MG_TRY(check_kernel_waits(F));
        d.s32 = pick;
        std::lock_guard<std::mutex> lk(mu);
        cache[key] = pick;
    }
    return MG_OK;
}

// FP32 residual + restriction and prolongation specialised for levels whose blocks all halve, fine edges 8..128.
bool transfer32_specialised(const DevLevel &d) { return d.all_halve && d.g.lg >= 3 && d.g.lg <= 7; }

using Restrict32Fn = void (*)(const float *, const float *, const float *, const float *, int64_t, float *, float *,
                              const XferItem *, int32_t, int64_t, Skip, const float *, const float *, const float *);
// [coefficient mode 0, 2, 3][fine block edge 2^3 .. 2^7]
const Restrict32Fn kRestrict32[3][5] = {
    {k_residual_restrict32<0, 3>, k_residual_restrict32<0, 4>, k_residual_restrict32<0, 5>,
     k_residual_restrict32<0, 6>, k_residual_restrict32<0, 7>},
    {k_residual_restrict32<2, 3>, k_residual_restrict32<2, 4>, k_residual_restrict32<2, 5>,
     k_residual_restrict32<2, 6>, k_residual_restrict32<2, 7>},
    {k_residual_restrict32<3, 3>, k_residual_restrict32<3, 4>, k_residual_restrict32<3, 5>,
     k_residual_restrict32<3, 6>, k_residual_restrict32<3, 7>}};
using Prolong32Fn = void (*)(float *, int64_t, const float *, const XferItem *, int32_t, int64_t,
                             const int32_t *, Skip);
const Prolong32Fn kProlong32[5] = {k_prolong32<3>, k_prolong32<4>, k_prolong32<5>, k_prolong32<6>, k_prolong32<7>};
// fine block edges 32, 64, 128: one thread per segment of kProlongZC coarse cells of a z-column
constexpr int kProlongZC = 2;
const Prolong32Fn kProlong32z[3] = {k_prolong32z<5, kProlongZC>, k_prolong32z<6, kProlongZC>,
                                    k_prolong32z<7, kProlongZC>};

using Restrict32tFn = void (*)(const float *, const float *, const float *, const float *, int64_t, float *, float *,
                               const XferItem *, int32_t, int64_t, Skip, const float *, const float *, const float *,
                               int, int, int, int *);
// staged residual + restriction: [coefficient mode 0, 2, 3][fine block edge 2^6, 2^7]
const Restrict32tFn kRestrict32t[3][2] = {{k_residual_restrict32t<0, 6>, k_residual_restrict32t<0, 7>},
                                          {k_residual_restrict32t<2, 6>, k_residual_restrict32t<2, 7>},
                                          {k_residual_restrict32t<3, 6>, k_residual_restrict32t<3, 7>}};

// Tile of the staged residual + restriction of a fine level {TY, TZ, D} (fine rows and planes per CTA, planes
// staged beyond the four a coarse plane reads), or {0, 0, 0} for the cell-per-thread kernel: fine edges 64 and 128,
// eight fine rows (128 or 256 consumer threads), 32 planes, one plane pair ahead.  At 512^3 (64^3 blocks) this tile
// took the level-0 restriction from 4.13 to 3.85 ms per solve; 16 rows, 16 or 64 planes or two pairs ahead were
// slower than the cell-per-thread kernel.
std::array<int, 3> restrict32t_shape(const DevLevel &d) {
    if (d.g.lg == 6 || d.g.lg == 7) return {8, 32, 1};
    return {0, 0, 0};
}

size_t restrict32t_smem(int lg, int mode, int TY, int TZ, int D) {
    return r32t_smem_bytes(r32t_plan(lg, mode, TY, TZ, D));
}

void launch_residual_restrict32(mg_forest *F, DevLevel &d, DevLevel &c) {
    const std::array<int, 3> sh = restrict32t_shape(d);
    if (sh[0]) {
        const int TY = sh[0], TZ = sh[1], D = sh[2], n = d.g.n, mode = mode32(F, d), mi = mode_index(mode);
        const Restrict32tFn fn = kRestrict32t[mi][d.g.lg - 6];
        static std::once_flag once[3][2];
        std::call_once(once[mi][d.g.lg - 6], [&] {
            cudaFuncSetAttribute(reinterpret_cast<const void *>(fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024);
        });
        const int64_t grid = static_cast<int64_t>(c.g.nb) * (n / TY) * (n / TZ);
        fn<<<static_cast<unsigned>(grid), (n / 2) * (TY / 2) + 32, restrict32t_smem(d.g.lg, mode, TY, TZ, D), F->st>>>(
            d.u32, d.f32, d.kap, d.ih2_32, d.g.bs, c.f32, c.u32, d.xfer, c.g.nb, c.g.bs, skip_of(F, c), d.ax32, d.ay32,
            d.az32, TY, TZ, D, F->kerr);
        return;
    }
    // one coarse cell per thread (no grid-stride loop): its load chain xf -> fine block -> 64 loads is latency-bound
    const auto grid = static_cast<unsigned>((c.cells() + kThreads - 1) / kThreads);
    kRestrict32[mode_index(mode32(F, d))][d.g.lg - 3]<<<grid, kThreads, 0, F->st>>>(
        d.u32, d.f32, d.kap, d.ih2_32, d.g.bs, c.f32, c.u32, d.xfer, c.g.nb, c.g.bs, skip_of(F, c), d.ax32, d.ay32,
        d.az32);
}

void launch_prolong32(mg_forest *F, DevLevel &d, DevLevel &c) {
    if (d.g.lg >= 5) {
        const auto grid = static_cast<unsigned>((c.cells() / kProlongZC + kThreads - 1) / kThreads);
        kProlong32z[d.g.lg - 5]<<<grid, kThreads, 0, F->st>>>(d.u32, d.g.bs, c.u32, d.xfer, c.g.nb, c.g.bs, d.nbr6,
                                                              skip_of(F, c));
        return;
    }
    kProlong32[d.g.lg - 3]<<<grid_for(c.cells()), kThreads, 0, F->st>>>(d.u32, d.g.bs, c.u32, d.xfer, c.g.nb, c.g.bs,
                                                                          d.nbr6, skip_of(F, c));
}

template <typename T, int MODE>
void smooth(mg_forest *F, DevLevel &d, int colour) {
    Prof p(F, &d == &F->L[0] ? cat_of<T>(P_SMOOTH64_L0) : cat_of<T>(P_SMOOTH64), 1);
    if constexpr (sizeof(T) == 4 && MODE != 1) {
        if (smooth32_specialised(d)) {
            launch_smooth32(F, d, colour, d.s32[0] ? d.s32 : Shape{1, 1, kThreads, 0, 0}, F->st);
            return;
        }
    }
    const T *gb = nullptr;
    if constexpr (sizeof(T) == 8)
        if (&d == &F->L[0]) gb = F->gb;
    k_smooth<T, MODE><<<grid_for(d.cells() / 2), kThreads, 0, F->st>>>(ufield<T>(d), ffield<T>(d), coef_of<T>(d),
                                                                       h2_of<T>(d), d.g, colour, d.nbr6, skip_of(F, d),
                                                                       gb);
}

// V(nu1, nu2) on level l.  Exchange schedule: at level entry a full exchange, unless the ghosts are known to be
// current (`entry`: ENTRY_FULL, ENTRY_INTERFACE = only refinement-interface ghosts may be stale, ENTRY_NONE = the
// correction and all its face ghosts were just zeroed); before each later half-sweep and before the restriction
// only the refinement-interface ghosts (the smoothers write same-level and boundary ghosts through); after the
// prolongation a full exchange, or only the interface one after a prolongation that writes through.
enum { ENTRY_FULL = 0, ENTRY_INTERFACE = 1, ENTRY_NONE = 2 };

// The schedule of V(nu1, nu2) from level l, walked with an executor: LaunchExec launches each step's kernels,
// RecordExec writes the steps down as the phase list of the persistent tail kernel (tail.cu), so both follow one
// schedule.
template <typename T, int MODE, typename E>
void vcycle_walk(mg_forest *F, int l, int entry, E &ex) {
    const int last = static_cast<int>(F->L.size()) - 1;
    if (ex.tail(l, entry)) return;
    if (l == last) {
        ex.coarse(l);
        ex.exchange(l, false);
        return;
    }
    if (entry != ENTRY_NONE) ex.exchange(l, entry == ENTRY_INTERFACE);
    const bool jac = F->cfg.smoother == 1;  // damped Jacobi (FP64): no write-through, a full exchange per sweep
    for (int i = 0; i < F->cfg.nu1; ++i) {
        if (jac) {
            if (i) ex.exchange(l, false);
            ex.jacobi(l);
            continue;
        }
        if (i) ex.exchange(l, true);
        ex.smooth(l, 0);
        ex.exchange(l, true);
        ex.smooth(l, 1);
    }
    if (F->cfg.nu1) ex.exchange(l, !jac);
    const bool fast = sizeof(T) == 4 && MODE != 1 && transfer32_specialised(F->L[l]);
    ex.restrict_to(l, fast);
    vcycle_walk<T, MODE>(F, l + 1, fast ? ENTRY_NONE : ENTRY_FULL, ex);
    if (l + 1 != last) ex.exchange(l + 1, !jac);  // Jacobi sweeps write no ghosts through
    const bool fast_p = fast && F->cfg.prolongation == 0;  // the trilinear prolongation writes no ghost through
    ex.prolong_from(l, fast_p);
    ex.exchange(l, fast_p);
    for (int i = 0; i < F->cfg.nu2; ++i) {
        if (jac) {
            if (i) ex.exchange(l, false);
            ex.jacobi(l);
            continue;
        }
        if (i) ex.exchange(l, true);
        ex.smooth(l, 0);
        ex.exchange(l, true);
        ex.smooth(l, 1);
    }
}

// How level l is entered in an FP32 V-cycle (level 0 from vcycle32, deeper levels from the restriction above).
int entry32(mg_forest *F, int l) {
    if (l == 0) return ENTRY_INTERFACE;
    return transfer32_specialised(F->L[l - 1]) ? ENTRY_NONE : ENTRY_FULL;
}

// Edge and corner ghosts of a level (trilinear prolongation; the face ghosts are current): edges, then corners.
template <typename T>
void exchange_diag(mg_forest *F, DevLevel &d, T *u) {
    if (!d.nedges) return;
    k_exchange_diag<T><<<grid_for(static_cast<int64_t>(d.nedges) * d.g.n), kThreads, 0, F->st>>>(
        u, d.edges, d.nedges, d.g, false, skip_of(F, d));
    k_exchange_diag<T><<<grid_for(d.ncorners), kThreads, 0, F->st>>>(u, d.corners, d.ncorners, d.g, true,
                                                                     skip_of(F, d));
}

template <typename T, int MODE>
struct LaunchExec {
    mg_forest *F;
    bool tail(int l, int entry) {
        if constexpr (sizeof(T) == 4) {
            if (F->tail_level >= 0 && l == F->tail_level && F->tail_for == l && entry == entry32(F, l)) {
                Prof p(F, P_TAIL32, 1);
                launch_tail32(F);
                return true;
            }
        }
        return false;
    }
    void exchange(int l, bool iface) {
        if constexpr (sizeof(T) == 4 && MODE == 2) {
            if (F->L[l].face32) {  // face-averaged coarse level: its conservative ghosts read the stored faces
                octmg::exchange<float, 3>(F, F->L[l], F->L[l].u32, iface);
                return;
            }
        }
        octmg::exchange<T, MODE>(F, F->L[l], ufield<T>(F->L[l]), iface);
    }
    void smooth(int l, int colour) { octmg::smooth<T, MODE>(F, F->L[l], colour); }
    void jacobi(int l, bool prof = true) {
        if constexpr (sizeof(T) == 8) {
            DevLevel &d = F->L[l];
            Prof p(F, prof ? cat_of<T>(l == 0 ? P_SMOOTH64_L0 : P_SMOOTH64) : -1, 1);
            k_jacobi64<MODE><<<grid_for(d.cells()), kThreads, 0, F->st>>>(d.u64, d.u64b, d.f64, d.c64(), d.h2_64, d.g,
                                                                          F->omega, skip_of(F, d));
            std::swap(d.u64, d.u64b);  // the new iterate; its ghosts are refreshed by the next exchange
        }
    }
    void coarse(int l) {
        DevLevel &d = F->L[l];
        if (F->cfg.coarse_iters > 0) {  // damped Jacobi sweeps from zero (the paper's coarsest solver)
            const DevLevel &d = F->L[l];
            Prof p(F, cat_of<T>(P_COARSE64), F->cfg.coarse_iters * (1 + (d.nfaces > 0) + (d.nsegs > 0)));
            for (int it = 0; it < F->cfg.coarse_iters; ++it) {
                octmg::exchange<T, MODE>(F, F->L[l], ufield<T>(F->L[l]), false, false);
                jacobi(l, false);
            }
            return;
        }
        Prof p(F, cat_of<T>(P_COARSE64), 1);
        k_coarse_solve<T><<<(F->Nc * 32 + kThreads - 1) / kThreads, kThreads, 0, F->st>>>(
            ufield<T>(d), ffield<T>(d), F->Ainv, sizeof(T) == 4 ? F->cmap32 : F->cmap, F->uprob, F->ustart, F->moff,
            F->Nc, F->pdone);
    }
    void restrict_to(int l, bool fast) {
        DevLevel &d = F->L[l], &c = F->L[l + 1];
        Prof p(F, cat_of<T>(P_RESTR64), 1);
        if (fast)
            launch_residual_restrict32(F, d, c);
        else if (sizeof(T) == 4 && d.face32)
            k_residual_restrict<float, 3><<<grid_for(c.cells()), kThreads, 0, F->st>>>(
                d.u32, d.f32, d.c32(), d.ih2_32, d.g, c.f32, c.u32, d.xfer, c.g, skip_of(F, c));
        else
            k_residual_restrict<T, MODE><<<grid_for(c.cells()), kThreads, 0, F->st>>>(
                ufield<T>(d), ffield<T>(d), coef_of<T>(d), ih2_of<T>(d), d.g, ffield<T>(c), ufield<T>(c), d.xfer, c.g,
                skip_of(F, c));
    }
    void prolong_from(int l, bool fast) {
        DevLevel &d = F->L[l], &c = F->L[l + 1];
        if (F->cfg.prolongation == 1) {  // trilinear: the coarse correction's edge and corner ghosts first
            Prof p(F, cat_of<T>(P_PROL64), 3);
            exchange_diag<T>(F, c, ufield<T>(c));
            k_prolong_tri<T><<<grid_for(c.cells()), kThreads, 0, F->st>>>(ufield<T>(d), d.g, ufield<T>(c), d.xfer,
                                                                          c.g, skip_of(F, c));
            return;
        }
        Prof p(F, cat_of<T>(P_PROL64), 1);
        if (fast)
            launch_prolong32(F, d, c);
        else
            k_prolong<T><<<grid_for(c.cells()), kThreads, 0, F->st>>>(ufield<T>(d), d.g, ufield<T>(c), d.xfer, c.g,
                                                                      skip_of(F, c));
    }
};

struct RecordExec {
    mg_forest *F;
    std::vector<TailPhase> ph;
    bool tail(int, int) { return false; }
    void exchange(int l, bool iface) {
        const DevLevel &d = F->L[l];
        if ((iface ? d.nifaces : d.nfaces) > 0) ph.push_back({iface ? T_FACES_IFACE : T_FACES_FULL, l});
        if (d.nsegs > 0) ph.push_back({T_SEGS, l});
    }
    void smooth(int l, int colour) { ph.push_back({colour ? T_SMOOTH1 : T_SMOOTH0, l}); }
    void jacobi(int) {}  // FP64 only; the tail runs FP32 cycles
    void coarse(int l) { ph.push_back({T_COARSE, l}); }
    void restrict_to(int l, bool) { ph.push_back({T_RESTRICT, l}); }
    void prolong_from(int l, bool) { ph.push_back({T_PROLONG, l}); }
};

template <typename T, int MODE>
void vcycle(mg_forest *F, int l, int entry) {
    LaunchExec<T, MODE> ex{F};
    vcycle_walk<T, MODE>(F, l, entry, ex);
}

// One part of an FP32 V-cycle around a tail that another launch runs (a batch's joint tail): the same schedule, with
// the steps before the tail level's entry launched in part 1 and those after the tail in part 2.  A forest without a
// recorded tail runs its whole cycle in part 1.
template <int MODE>
struct PartExec {
    LaunchExec<float, MODE> in;
    int part;
    bool past = false;
    bool on() const { return (part == 1) != past; }
    bool tail(int l, int entry) {
        mg_forest *F = in.F;
        if (F->tail_level >= 0 && l == F->tail_level && F->tail_for == l && entry == entry32(F, l)) {
            past = true;
            return true;
        }
        return false;
    }
    void exchange(int l, bool iface) {
        if (on()) in.exchange(l, iface);
    }
    void smooth(int l, int colour) {
        if (on()) in.smooth(l, colour);
    }
    void jacobi(int l) {
        if (on()) in.jacobi(l);
    }
    void coarse(int l) {
        if (on()) in.coarse(l);
    }
    void restrict_to(int l, bool fast) {
        if (on()) in.restrict_to(l, fast);
    }
    void prolong_from(int l, bool fast) {
        if (on()) in.prolong_from(l, fast);
    }
};

// Levels from which the tail kernel can run the rest of an FP32 V-cycle: every deeper level has a specialised
// column smoother (edge 4..128).
bool tail_possible(mg_forest *F, int l) {
    if (F->cfg.precision != 1 || F->cfg.prolongation != 0 || l < 0 || l >= static_cast<int>(F->L.size()))
        return false;
    for (int m = l; m < static_cast<int>(F->L.size()); ++m)
        if (F->L[m].g.lg < 2 || F->L[m].g.lg > 7) return false;
    return true;
}

// Records the tail's phase list from level l and uploads it with the level descriptors.
mg_status record_tail(mg_forest *F, int l) {
    RecordExec rec{F, {}};
    if (F->cfg.coeff) vcycle_walk<float, 2>(F, l, entry32(F, l), rec);
    else vcycle_walk<float, 0>(F, l, entry32(F, l), rec);
    if (!F->tail_L) {
        std::vector<TailLevel> tl(F->L.size());
        for (size_t m = 0; m < F->L.size(); ++m) {
            const DevLevel &d = F->L[m];
            tl[m] = TailLevel{d.g, d.u32, d.f32, d.kap, d.h2_32, d.ih2_32, d.faces, d.ifaces, d.segs, d.xfer, d.nbr6,
                              d.bprob, d.nfaces, d.nifaces, d.nsegs, transfer32_specialised(d) ? 1 : 0,
                              d.ax32, d.ay32, d.az32, d.face32 ? 1 : 0};
        }
        MG_TRY(upload(F, &F->tail_L, tl));
        MG_TRY(dalloc(F, &F->tail_bar, 2));
    }
    if (static_cast<int>(rec.ph.size()) > F->tail_nph || !F->tail_ph) MG_TRY(dalloc(F, &F->tail_ph, rec.ph.size()));
    MG_CUDA(cudaMemcpyAsync(F->tail_ph, rec.ph.data(), rec.ph.size() * sizeof(TailPhase), cudaMemcpyHostToDevice,
                            F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    F->tail_nph = static_cast<int>(rec.ph.size());
    F->tail_ph_host = rec.ph;
    F->tail_for = l;
    return MG_OK;
}

// CTA chunks per block for the per-block reductions: about 2048 cells per CTA.
int chunks_per_block(const DevLevel &d) { return std::max(1, static_cast<int>(d.cells() / d.g.nb) / 2048); }

// Per-problem sums of the per-block sums to the host (pinned psum_h), synchronising the stream.
mg_status read_problem_sums(mg_forest *F) {
    k_problem_sums<<<F->np, kSumThreads, 0, F->st>>>(F->bsum, F->bsum_cpb, F->pstart, F->pblk, F->np, F->psum);
    MG_CUDA(cudaMemcpyAsync(F->psum_h, F->psum, F->np * sizeof(double), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    return MG_OK;
}

// Per-problem residual scales (powers of two, exact in FP32 and FP64): host pinned copies, then the device copies.
void set_scales_host(mg_forest *F, const std::vector<double> &mult) {
    for (int p = 0; p < F->np; ++p) {
        F->pscale_h[p] = static_cast<float>(mult[p]);
        F->pinv_h[p] = 1.0 / mult[p];
    }
}

mg_status enqueue_scales(mg_forest *F) {
    MG_CUDA(cudaMemcpyAsync(F->pscale, F->pscale_h, F->np * sizeof(float), cudaMemcpyHostToDevice, F->st));
    MG_CUDA(cudaMemcpyAsync(F->pinv, F->pinv_h, F->np * sizeof(double), cudaMemcpyHostToDevice, F->st));
    return MG_OK;
}

// The done-mask to the device (pinned host copy read when the copy runs, also inside a replayed graph).
mg_status enqueue_done(mg_forest *F) {
    MG_CUDA(cudaMemcpyAsync(F->pdone, F->pdone_h, F->np, cudaMemcpyHostToDevice, F->st));
    return MG_OK;
}

// Clears the per-problem done-mask (host and device): outside a solve no problem is skipped.
void reset_done(mg_forest *F) {
    std::memset(F->pdone_h, 0, F->np);
    cudaMemsetAsync(F->pdone, 0, F->np, F->st);
}


mg_status upload_scales(mg_forest *F, const std::vector<double> &mult) {
    set_scales_host(F, mult);
    return enqueue_scales(F);
}

mg_status enqueue_problem_sums(mg_forest *F) {
    k_problem_sums<<<F->np, kSumThreads, 0, F->st>>>(F->bsum, F->bsum_cpb, F->pstart, F->pblk, F->np, F->psum);
    MG_CUDA(cudaMemcpyAsync(F->psum_h, F->psum, F->np * sizeof(double), cudaMemcpyDeviceToHost, F->st));
    return MG_OK;
}

// Level-0 FP64 residual r = f - A u (exchange first); optionally written as FP32 r * scale_p with the FP32
// correction zeroed; returns ||r_p||^2 (volume-weighted, per problem) to rr when rr is not null.  scale_p (set by
// upload_scales, mult) is a power of two close to 1 / ||r_p|| so the FP32 values stay near unit size.
template <int MODE>
mg_status residual64(mg_forest *F, double *u, const double *f, float *out, float *zero_out,
                     const std::vector<double> &mult, std::vector<double> *rr, bool zero_u = false) {
    DevLevel &d = F->L[0];
    if (!zero_u) exchange<double, MODE>(F, d, u);
    const int cpb = chunks_per_block(d);
    MG_CUDA(cudaMemsetAsync(F->bsum, 0, static_cast<size_t>(d.g.nb) * cpb * sizeof(double), F->st));
    {
        Prof p(F, P_RESID64, 1);
        if (zero_u)
            k_residual_norm<MODE, true><<<d.g.nb * cpb, kThreads, 0, F->st>>>(
                u, f, d.c64(), d.ih2_64, d.vol_32, d.g, cpb, out, F->pscale, d.bprob, F->bsum, zero_out,
                skip_of(F, d));
        else
            k_residual_norm<MODE><<<d.g.nb * cpb, kThreads, 0, F->st>>>(u, f, d.c64(), d.ih2_64, d.vol_32, d.g, cpb,
                                                                        out, F->pscale, d.bprob, F->bsum, zero_out,
                                                                        skip_of(F, d));
    }
    if (rr) {
        MG_TRY(read_problem_sums(F));
        rr->resize(F->np);
        for (int p = 0; p < F->np; ++p) (*rr)[p] = F->psum_h[p] / (mult[p] * mult[p]);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

mg_status residual64_any(mg_forest *F, double *u, const double *f, const std::vector<double> &mult,
                         std::vector<double> *rr) {
    if (F->cfg.coeff) return residual64<1>(F, u, f, nullptr, nullptr, mult, rr);
    return residual64<0>(F, u, f, nullptr, nullptr, mult, rr);
}

void apply64(mg_forest *F, DevLevel &d, const double *u, double *out) {
    if (F->cfg.coeff)
        k_apply64<1><<<grid_for(d.cells()), kThreads, 0, F->st>>>(u, d.c64(), d.ih2_64, d.g, out);
    else
        k_apply64<0><<<grid_for(d.cells()), kThreads, 0, F->st>>>(u, d.c64(), d.ih2_64, d.g, out);
}

// The device part of assemble_coarse: the columns A e_m of every problem's coarsest operator (FP64 kernels on unit
// vectors, all problems probed at once), then Gauss-Jordan on the device into Ainv and AinvT (transposes).
void enqueue_coarse_inverse(mg_forest *F, DevLevel &d, int N, int maxN) {
    double *r = F->coarse_r;
    // the columns go to the buffer that makes the eliminated matrix end up in AinvT after maxN steps
    double *Adev = maxN % 2 == 0 ? F->AinvT : F->Ainv;
    cudaMemsetAsync(d.u64, 0, d.pool_elems() * sizeof(double), F->st);
    if (F->pcol) {  // no refinement interface: 27 colour probes
        cudaMemsetAsync(Adev, 0, F->moff_h[F->np] * sizeof(double), F->st);
        for (int C = 0; C < 27; ++C) {
            k_set_colour<<<(N + 255) / 256, 256, 0, F->st>>>(d.u64, F->cmap, F->pcol, N, C);
            exchange_any64(F, d, d.u64);
            apply64(F, d, d.u64, r);
            k_gather_colour<<<(N + 255) / 256, 256, 0, F->st>>>(r, F->cmap, F->uprob, F->ustart, F->moff, F->pcol,
                                                                F->pnbu, N, Adev, C);
        }
    } else {  // one unit vector per column
        for (int m = 0; m < maxN; ++m) {
            k_set_units<<<(F->np + 127) / 128, 128, 0, F->st>>>(d.u64, F->cmap, F->ustart, F->np, m);
            exchange_any64(F, d, d.u64);
            apply64(F, d, d.u64, r);
            k_gather_columns<<<(N + 255) / 256, 256, 0, F->st>>>(r, F->cmap, F->uprob, F->ustart, F->moff, N, Adev,
                                                                 m);
        }
    }
    cudaMemsetAsync(F->flag, 0, sizeof(int), F->st);
    const dim3 grid(static_cast<unsigned>(std::min<int64_t>(1024, (static_cast<int64_t>(maxN) * maxN + 255) / 256)),
                    static_cast<unsigned>(F->np));
    double *X = Adev, *Y = Adev == F->Ainv ? F->AinvT : F->Ainv;
    for (int c = 0; c < maxN; ++c) {
        k_gj_pivot<<<(F->np * 32 + 255) / 256, 256, 0, F->st>>>(X, F->moff, F->ustart, F->np, c, F->gj_piv,
                                                                F->gj_pinv, maxN, F->flag);
        k_gj_step<<<grid, 256, 0, F->st>>>(X, Y, F->moff, F->ustart, c, F->gj_piv, F->gj_pinv, maxN);
        std::swap(X, Y);
    }
    k_gj_perm<<<(F->np + 127) / 128, 128, 0, F->st>>>(F->gj_piv, F->ustart, F->np, F->gj_src, maxN);
    k_gj_unpermute<<<grid, 256, 0, F->st>>>(F->AinvT, F->Ainv, F->moff, F->ustart, F->gj_src, maxN);
    k_gj_transpose<<<grid, 256, 0, F->st>>>(F->Ainv, F->AinvT, F->moff, F->ustart);
    cudaMemsetAsync(d.u64, 0, d.pool_elems() * sizeof(double), F->st);
}

// Coarsest-level dense operators and their inverses (and transposes), every problem's block at once.  The device
// part is a few thousand small launches; outside a stream capture it is recorded as a CUDA graph at the second call
// and replayed by later ones (the pointers it uses never change).
mg_status assemble_coarse(mg_forest *F) {
    const int l = static_cast<int>(F->L.size()) - 1;
    DevLevel &d = F->L[l];
    const HostLevel &hl = F->H.levels[l];
    const int N = static_cast<int>(d.cells());
    const int cells = d.g.n * d.g.n * d.g.n;
    F->Nc = N;
    if (!F->cmap) {
        std::vector<std::vector<int32_t>> blocks(F->np);
        for (int b = 0; b < d.g.nb; ++b) blocks[hl.keys[b].p].push_back(b);
        std::vector<int64_t> cmap, cmap32;
        std::vector<int32_t> uprob;
        F->ustart_h.assign(F->np + 1, 0);
        F->moff_h.assign(F->np + 1, 0);
        const int n = d.g.n;
        for (int p = 0; p < F->np; ++p) {
            F->ustart_h[p] = static_cast<int64_t>(cmap.size());
            for (int b : blocks[p])
                for (int z = 0; z < n; ++z)
                    for (int y = 0; y < n; ++y)
                        for (int x = 0; x < n; ++x) {
                            cmap.push_back(b * d.g.bs + off3(x + 1, y + 1, z + 1, d.g.P));
                            cmap32.push_back(Lay<float>::at(d.g, b, x + 1, y + 1, z + 1));
                            uprob.push_back(p);
                        }
            const int64_t Np = static_cast<int64_t>(blocks[p].size()) * cells;
            F->moff_h[p + 1] = F->moff_h[p] + Np * Np;
        }
        F->ustart_h[F->np] = static_cast<int64_t>(cmap.size());
        MG_TRY(upload(F, &F->cmap, cmap));
        MG_TRY(upload(F, &F->cmap32, cmap32));
        MG_TRY(upload(F, &F->uprob, uprob));
        MG_TRY(upload(F, &F->ustart, F->ustart_h));
        MG_TRY(upload(F, &F->moff, F->moff_h));
        MG_TRY(dalloc(F, &F->Ainv, F->moff_h[F->np]));
        MG_TRY(dalloc(F, &F->AinvT, F->moff_h[F->np]));
        if (d.nifaces == 0 && d.nsegs == 0) {
            // colours and the 7-point neighbourhoods of the unknowns for the colour probe; every block of a problem
            // is then at one refinement level (face neighbours share it), so key * n + local is a global coordinate
            std::vector<int64_t> first(d.g.nb, -1);  // unknown index of each block's first cell
            for (int p = 0; p < F->np; ++p) {
                int64_t at = F->ustart_h[p];
                for (int b : blocks[p]) {
                    first[b] = at;
                    at += cells;
                }
            }
            std::vector<int32_t> nb6(static_cast<size_t>(d.g.nb) * 6, -2);
            for (const FaceItem &fi : hl.faces)
                nb6[static_cast<size_t>(fi.blk) * 6 + 2 * fi.axis + fi.side] =
                    fi.kind == FK_SAME ? fi.nbr : (fi.kind == FK_BND ? -1 : -2);
            std::vector<int8_t> col(N);
            std::vector<int32_t> nbu(static_cast<size_t>(N) * 7, -1);
            bool ok = true;
            for (int b = 0; b < d.g.nb && ok; ++b) {
                const Key &kb = hl.keys[b];
                for (int z = 0; z < n; ++z)
                    for (int y = 0; y < n; ++y)
                        for (int x = 0; x < n; ++x) {
                            const int64_t i = first[b] + (static_cast<int64_t>(z) * n + y) * n + x;
                            const int64_t gx = static_cast<int64_t>(kb.i) * n + x, gy = static_cast<int64_t>(kb.j) * n + y,
                                          gz = static_cast<int64_t>(kb.k) * n + z;
                            col[i] = static_cast<int8_t>(gx % 3 + 3 * (gy % 3) + 9 * (gz % 3));
                            nbu[i * 7] = static_cast<int32_t>(i);
                            const int c[3] = {x, y, z};
                            for (int axis = 0; axis < 3; ++axis)
                                for (int side = 0; side < 2; ++side) {
                                    int cc[3] = {c[0], c[1], c[2]};
                                    cc[axis] += side ? 1 : -1;
                                    int bb = b;
                                    if (cc[axis] < 0 || cc[axis] >= n) {
                                        bb = nb6[static_cast<size_t>(b) * 6 + 2 * axis + side];
                                        if (bb == -2) ok = false;
                                        if (bb < 0) continue;
                                        cc[axis] = side ? 0 : n - 1;
                                    }
                                    nbu[i * 7 + 1 + 2 * axis + side] =
                                        static_cast<int32_t>(first[bb] + (static_cast<int64_t>(cc[2]) * n + cc[1]) * n + cc[0]);
                                }
                        }
            }
            if (ok && N < (int64_t(1) << 31)) {
                MG_TRY(upload(F, &F->pcol, col));
                MG_TRY(upload(F, &F->pnbu, nbu));
            }
        }
    }
    if (!F->coarse_r) MG_TRY(dalloc(F, &F->coarse_r, d.pool_elems()));
    int maxN = 0;
    for (int p = 0; p < F->np; ++p) maxN = std::max<int>(maxN, static_cast<int>(F->ustart_h[p + 1] - F->ustart_h[p]));
    if (!F->gj_piv) {
        MG_TRY(dalloc(F, &F->gj_piv, static_cast<int64_t>(F->np) * maxN));
        MG_TRY(dalloc(F, &F->gj_src, static_cast<int64_t>(F->np) * maxN));
        MG_TRY(dalloc(F, &F->gj_pinv, F->np));
    }
    // the probe must see the homogeneous operator: no boundary data, no profiling events inside a recorded graph
    double *const gb = F->gb;
    const bool prof = F->prof;
    F->gb = nullptr;
    F->prof = false;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ce = cudaStreamIsCapturing(F->st, &cap);
    // recorded from the second call on (the first one loads every kernel the sequence uses, which a capture does not
    // allow); a recording that fails is abandoned for good and the sequence launched directly
    if (ce == cudaSuccess && cap == cudaStreamCaptureStatusNone && F->coarse_runs++ > 0 && !F->coarse_graph &&
        !F->coarse_nograph) {
        // recorded on a private stream (the forest's stream may be the legacy default stream, which cannot be
        // captured); the graph is then launched on the forest's stream
        cudaGraph_t graph = nullptr;
        cudaError_t e1 = F->cap_st ? cudaSuccess : cudaStreamCreateWithFlags(&F->cap_st, cudaStreamNonBlocking);
        if (e1 == cudaSuccess) e1 = cudaStreamBeginCapture(F->cap_st, cudaStreamCaptureModeThreadLocal);
        if (e1 == cudaSuccess) {
            cudaStream_t own = F->st;
            F->st = F->cap_st;
            enqueue_coarse_inverse(F, d, N, maxN);
            F->st = own;
            e1 = cudaStreamEndCapture(F->cap_st, &graph);
        }
        if (e1 == cudaSuccess && graph) e1 = cudaGraphInstantiate(&F->coarse_graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e1 != cudaSuccess || !F->coarse_graph) {
            F->coarse_graph = nullptr;
            F->coarse_nograph = true;
            cudaGetLastError();
        }
    }
    if (ce == cudaSuccess) {
        if (F->coarse_graph && cap == cudaStreamCaptureStatusNone) {
            ce = cudaGraphLaunch(F->coarse_graph, F->st);
        } else {
            enqueue_coarse_inverse(F, d, N, maxN);
            ce = cudaGetLastError();
        }
    }
    F->gb = gb;
    F->prof = prof;
    if (ce != cudaSuccess) {
        set_error(std::string("coarsest-level inverse: ") + cudaGetErrorString(ce));
        return MG_ERR_CUDA;
    }
    int hbad = 0;
    MG_CUDA(cudaMemcpyAsync(&hbad, F->flag, sizeof(int), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (hbad) {
        set_error("a coarsest-level operator is singular");
        return MG_ERR_INVALID_ARG;
    }
    return MG_OK;
}

// Coefficient pyramid: k with ghosts on every level, face coefficients (FP64) and 1/k (FP32).
mg_status build_coefficients(mg_forest *F) {
    for (size_t l = 0; l < F->L.size(); ++l) {
        DevLevel &d = F->L[l];
        if (l > 0) {
            DevLevel &p = F->L[l - 1];
            k_restrict_field<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(p.k64, p.g, d.k64, p.xfer, d.g);
        }
        exchange_k(F, d);
        const bool averaged = l > 0 && F->cfg.coarse_coef == 1 && d.tx;
        // harmonic means of k on the finest level (and on every level when rediscretised); 1/k for the FP32 cycles
        k_face_coefs<<<grid_for(d.pool_elems()), kThreads, 0, F->st>>>(d.k64, d.ih2_64, d.g, averaged ? nullptr : d.tx,
                                                                        averaged ? nullptr : d.ty,
                                                                        averaged ? nullptr : d.tz, d.kap);
        if (averaged) {
            DevLevel &p = F->L[l - 1];
            k_average_faces64<<<grid_for(static_cast<int64_t>(d.g.nb) * 3 * (d.g.n + 1) * d.g.n * d.g.n), kThreads, 0,
                                F->st>>>(p.tx, p.ty, p.tz, p.g, d.tx, d.ty, d.tz, p.xfer, d.g);
        }
        if (d.dg) k_diag<<<grid_for(d.cells()), kThreads, 0, F->st>>>(d.tx, d.ty, d.tz, d.g, d.dg, d.dinv);
        if (d.face32)
            k_face_half32<<<grid_for(d.pool_elems()), kThreads, 0, F->st>>>(d.tx, d.ty, d.tz, d.h2_64, d.g, d.ax32,
                                                                             d.ay32, d.az32);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

template <typename T>
mg_status pack_user(mg_forest *F, DevLevel &d, T *pool, const double *user) {
    Prof p(F, P_LAYOUT, 1);
    k_pack<T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(pool, user, d.g, &d == &F->L[0] ? F->leaf_off : nullptr);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

template <typename T>
mg_status unpack_user(mg_forest *F, DevLevel &d, double *user, const T *pool) {
    Prof p(F, P_LAYOUT, 1);
    k_unpack<T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(user, pool, d.g,
                                                             &d == &F->L[0] ? F->leaf_off : nullptr);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

// One FP64 V-cycle on level 0.
void vcycle64(mg_forest *F) {
    if (F->cfg.coeff) vcycle<double, 1>(F, 0, ENTRY_FULL);
    else vcycle<double, 0>(F, 0, ENTRY_FULL);
}
// One FP64 V-cycle on level 0, replayed from a recorded CUDA graph: the cycle's launch sequence depends only on the
// forest, so it is recorded once, on the private stream (from the second cycle on: the first one loads the kernels,
// which a capture does not allow), and each later cycle is one graph launch instead of one launch per step, which
// is what small, launch-bound forests need.  Launched directly while profiling (per-family events), while the
// caller's stream is being captured, and when the recorded cycle would not leave the damped-Jacobi ping-pong pools
// as it found them (an odd number of sweeps per level) or the recording fails.  mg_set_boundary drops the graph.
mg_status vcycle64_step(mg_forest *F) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MG_CUDA(cudaStreamIsCapturing(F->st, &cap));
    if (F->prof || F->v64_nograph || cap != cudaStreamCaptureStatusNone || F->v64_runs++ == 0) {
        vcycle64(F);
        return MG_OK;
    }
    if (!F->v64_graph) {
        std::vector<std::pair<double *, double *>> before;
        for (const DevLevel &d : F->L) before.emplace_back(d.u64, d.u64b);
        cudaGraph_t graph = nullptr;
        cudaError_t e = F->cap_st ? cudaSuccess : cudaStreamCreateWithFlags(&F->cap_st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(F->cap_st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaStream_t own = F->st;
            F->st = F->cap_st;
            vcycle64(F);
            F->st = own;
            e = cudaStreamEndCapture(F->cap_st, &graph);
        }
        bool same = true;  // nothing ran during the recording: the iterate is still where it was
        for (size_t i = 0; i < F->L.size(); ++i) {
            same = same && F->L[i].u64 == before[i].first;
            F->L[i].u64 = before[i].first;
            F->L[i].u64b = before[i].second;
        }
        if (e == cudaSuccess && graph && same) e = cudaGraphInstantiate(&F->v64_graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess || !same || !F->v64_graph) {
            F->v64_graph = nullptr;
            F->v64_nograph = true;
            cudaGetLastError();
            vcycle64(F);
            return MG_OK;
        }
    }
    MG_CUDA(cudaGraphLaunch(F->v64_graph, F->st));
    return MG_OK;
}

// The FP32 correction on level 0 either was just zeroed with its face ghosts (k_residual_norm) or ends a previous
// FP32 V-cycle whose last half-sweeps wrote its same-level and boundary ghosts through.
void vcycle32(mg_forest *F) {
    if (F->cfg.coeff) vcycle<float, 2>(F, 0, ENTRY_INTERFACE);
    else vcycle<float, 0>(F, 0, ENTRY_INTERFACE);
}

void vcycle32_part(mg_forest *F, int part) {
    if (part == 0) {
        vcycle32(F);
    } else if (F->cfg.coeff) {
        PartExec<2> ex{{F}, part};
        vcycle_walk<float, 2>(F, 0, ENTRY_INTERFACE, ex);
    } else {
        PartExec<0> ex{{F}, part};
        vcycle_walk<float, 0>(F, 0, ENTRY_INTERFACE, ex);
    }
}

// Picks the persistent tail's level: every level l whose own and deeper levels have at most 2^20 cells (and
// specialised smoothers) is a candidate; each candidate and "off" is timed over five FP32 V-cycles (after two
// untimed ones) on the FP32 pools, which are dead between solves, and the fastest is kept.  Skipped (off) while the
// stream is being captured.
mg_status tune_tail(mg_forest *F) {
    if (F->tail_tuned || F->cfg.precision != 1) return MG_OK;
    F->tail_tuned = true;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MG_CUDA(cudaStreamIsCapturing(F->st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return MG_OK;
    const int last = static_cast<int>(F->L.size()) - 1;
    std::vector<int> cand{-1};
    for (int l = last - 1; l >= 0; --l) {
        if (F->L[l].cells() > (int64_t(1) << 20) || !tail_possible(F, l)) break;
        cand.push_back(l);
    }
    if (cand.size() == 1) return MG_OK;
    cudaEvent_t e0 = next_event(F), e1 = next_event(F);
    if (!e0 || !e1) {
        set_error("cudaEventCreate failed");
        return MG_ERR_CUDA;
    }
    float best = 0.0f;
    int pick = -1;
    for (int lt : cand) {
        if (lt >= 0) MG_TRY(record_tail(F, lt));
        F->tail_level = lt;
        for (int w = 0; w < 2; ++w) vcycle32(F);
        MG_CUDA(cudaEventRecord(e0, F->st));
        for (int w = 0; w < 5; ++w) vcycle32(F);
        MG_CUDA(cudaEventRecord(e1, F->st));
        MG_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        MG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (lt == -1 || ms < best) {
            best = ms;
            pick = lt;
        }
    }
    F->ev_used -= 2;
    MG_CUDA(cudaGetLastError());
    MG_TRY(check_kernel_waits(F));
    if (pick >= 0) MG_TRY(record_tail(F, pick));
    F->tail_level = pick;
    return MG_OK;
}

// The power of two nearest to x, kept inside the binary32 normal range (the kernels apply it on exponent bits).
double pow2_near(double x) {
    if (!(x > 0.0) || !std::isfinite(x)) return 1.0;
    const long e = std::lround(std::log2(x));
    return std::ldexp(1.0, static_cast<int>(std::min(126L, std::max(-126L, e))));
}

// Mixed precision, first half of a defect-correction step: r64 = f - A u (FP64), stored as FP32 r * scale_p
// with the FP32 correction zeroed; per-problem ||r||^2 to rr.
mg_status mixed_step(mg_forest *F, const std::vector<double> &mult, std::vector<double> *rr, bool zero_u) {
    DevLevel &d = F->L[0];
    MG_TRY(upload_scales(F, mult));
    if (F->cfg.coeff)
        MG_TRY((residual64<1>(F, d.u64, d.f64, d.f32, d.u32, mult, rr, zero_u)));
    else
        MG_TRY((residual64<0>(F, d.u64, d.f64, d.f32, d.u32, mult, rr, zero_u)));
    return MG_OK;
}

// The residual half of a defect-correction step without host synchronisation (graph-capturable).
mg_status enqueue_residual(mg_forest *F, bool zero_u) {
    DevLevel &d = F->L[0];
    static const std::vector<double> none;
    if (F->cfg.coeff) return residual64<1>(F, d.u64, d.f64, d.f32, d.u32, none, nullptr, zero_u);
    return residual64<0>(F, d.u64, d.f64, d.f32, d.u32, none, nullptr, zero_u);
}

// Packs the caller's u into the level-0 FP64 pool and reports whether it is all zero (one read-back).
mg_status pack_initial_guess(mg_forest *F, const double *u_dev, bool *zero) {
    DevLevel &d = F->L[0];
    MG_CUDA(cudaMemsetAsync(F->flag, 0, sizeof(int), F->st));
    {
        Prof p(F, P_LAYOUT, 1);
        k_pack<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(d.u64, u_dev, d.g, F->leaf_off, F->flag);
    }
    int h = 1;
    MG_CUDA(cudaMemcpyAsync(&h, F->flag, sizeof(int), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    *zero = h == 0;
    return MG_OK;
}

// Second half: `cycles` FP32 V-cycles on the scaled residual, then u64 += e32 / scale_p (exact).
mg_status enqueue_update_mixed(mg_forest *F) {
    DevLevel &d = F->L[0];
    Prof p(F, P_UPDATE, 1);
    k_update_mixed<<<grid_for(d.cells()), kThreads, 0, F->st>>>(d.u64, d.u32, F->pinv, d.bprob, d.g, skip_of(F, d));
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

mg_status finish_mixed_cycle(mg_forest *F, int cycles) {
    for (int i = 0; i < cycles; ++i) vcycle32(F);
    return enqueue_update_mixed(F);
}

// Level-0 FP64 scratch pools (operator application, gradients), allocated on first use.
mg_status ensure_scratch64(mg_forest *F) {
    if (!F->s64a) MG_TRY(dalloc(F, &F->s64a, F->L[0].pool_elems()));
    if (!F->s64b) MG_TRY(dalloc(F, &F->s64b, F->L[0].pool_elems()));
    return MG_OK;
}

// FP64 coefficient arrays (scaled faces, diagonal, inverse diagonal) on every level, for the FP64 paths a forest
// with FP32 cycles does not allocate at creation (adjoint cycles, the debug exchange of intermediate levels).
mg_status ensure_fp64_coefficients(mg_forest *F) {
    if (!F->cfg.coeff) return MG_OK;
    bool added = false;
    for (DevLevel &d : F->L) {
        const int64_t pe = d.pool_elems();
        if (!d.tx) {
            MG_TRY(dalloc(F, &d.tx, pe));
            MG_TRY(dalloc(F, &d.ty, pe));
            MG_TRY(dalloc(F, &d.tz, pe));
            MG_TRY(dalloc(F, &d.dg, pe));
            added = true;
        }
        if (!d.dinv) {
            MG_TRY(dalloc(F, &d.dinv, pe));
            added = true;
        }
    }
    if (added && F->rhs_set) MG_TRY(build_coefficients(F));
    return MG_OK;
}

mg_status enqueue_fp32_step(mg_forest *F, int cycles) { return finish_mixed_cycle(F, cycles); }

mg_status check_ready(mg_forest *F) {
    if (!F) {
        set_error("null forest");
        return MG_ERR_INVALID_ARG;
    }
    if (!F->rhs_set) {
        set_error("mg_set_rhs has not been called");
        return MG_ERR_STATE;
    }
    return MG_OK;
}

// Runs cycles until every problem has rel <= rtol (rtol < 0: exactly max_cycles).  u_dev in/out.  Per problem,
// cycles_out gets the cycle count at which it first met rtol (else the total) and rel_out its final residual.
mg_status run_cycles(mg_forest *F, double *u_dev, double rtol, int max_cycles, int32_t *cycles_out,
                     double *rel_out) {
    MG_TRY(check_ready(F));
    DevLevel &d = F->L[0];
    const int np = F->np;
    bool zero_guess = false;
    MG_TRY(pack_initial_guess(F, u_dev, &zero_guess));
    reset_done(F);
    std::vector<double> fn(np), rel(np, -1.0), mult(np), rr(np, 0.0);
    std::vector<int32_t> met(np, -1);
    for (int p = 0; p < np; ++p) {
        fn[p] = F->fnorm_p[p] > 0.0 ? F->fnorm_p[p] : 1.0;
        mult[p] = pow2_near(1.0 / fn[p]);
    }
    // A problem that meets rtol is masked out of every later kernel (its u stays where it converged, its residual
    // is no longer computed and keeps the value that met rtol).
    auto update_rel = [&](int done) {
        bool all = true, finite = true, changed = false;
        for (int p = 0; p < np; ++p) {
            if (F->pdone_h[p]) continue;
            rel[p] = std::sqrt(rr[p]) / fn[p];
            if (!std::isfinite(rel[p])) finite = false;
            if (rtol >= 0.0 && rel[p] <= rtol && met[p] < 0) {
                met[p] = done;
                F->pdone_h[p] = 1;
                changed = true;
            }
            if (!(rtol >= 0.0 && rel[p] <= rtol)) all = false;
            mult[p] = pow2_near(1.0 / std::sqrt(rr[p]));
        }
        if (changed && !all) enqueue_done(F);
        return std::make_pair(all, finite);
    };
    int done = 0;
    bool finite = true;
    if (F->cfg.precision == 0) {
        while (done < max_cycles) {
            MG_TRY(vcycle64_step(F));
            ++done;
            if (rtol >= 0.0 || done == max_cycles) {
                MG_TRY(upload_scales(F, mult));
                MG_TRY(residual64_any(F, d.u64, d.f64, mult, &rr));
                auto st = update_rel(done);
                finite = st.second;
                if (!finite || st.first) break;
            }
        }
    } else {
        MG_TRY(mixed_step(F, mult, &rr, zero_guess && !F->gb));  // a zero guess (g = 0) needs no operator: r = f
        auto st = update_rel(0);
        finite = st.second;
        const int inner = std::max(1, F->cfg.inner_cycles);
        while (finite && done < max_cycles && !st.first) {
            const int m = std::min(inner, max_cycles - done);
            MG_TRY(finish_mixed_cycle(F, m));
            done += m;
            MG_TRY(mixed_step(F, mult, &rr, false));
            st = update_rel(done);
            finite = st.second;
        }
    }
    MG_TRY(unpack_user<double>(F, d, u_dev, d.u64));
    reset_done(F);
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (F->cfg.precision == 1) MG_TRY(check_kernel_waits(F));
    for (int p = 0; p < np; ++p) {
        if (cycles_out) cycles_out[p] = met[p] >= 0 ? met[p] : done;
        if (rel_out) rel_out[p] = rel[p];
    }
    if (!finite) {
        set_error("residual is not finite");
        return MG_ERR_NOT_CONVERGED;
    }
    if (rtol >= 0.0) {
        for (int p = 0; p < np; ++p)
            if (!(rel[p] <= rtol)) {
                set_error("problem " + std::to_string(p) + ": relative residual " + fmt_e(rel[p]) +
                          " above rtol after " + std::to_string(done) + " cycles");
                return MG_ERR_NOT_CONVERGED;
            }
    }
    return MG_OK;
}

mg_status create(const mg_config *cfg, mg_forest **out) {
    if (!cfg || !out || !cfg->leaves || cfg->n_leaves <= 0) {
        set_error("null config, output or leaves");
        return MG_ERR_INVALID_ARG;
    }
    if (cfg->coeff < 0 || cfg->coeff > 1 || cfg->precision < 0 || cfg->precision > 1 || cfg->nu1 < 0 || cfg->nu2 < 0 ||
        cfg->nu1 + cfg->nu2 == 0 || cfg->interface_flux < 0 || cfg->interface_flux > 1) {
        set_error("bad coeff / precision / nu1 / nu2 / interface_flux");
        return MG_ERR_INVALID_ARG;
    }
    if (cfg->c2f_variant < 0 || cfg->c2f_variant > 2 || cfg->smoother < 0 || cfg->smoother > 1 ||
        cfg->coarse_iters < 0 || !(cfg->omega < 2.0) || std::isnan(cfg->omega)) {
        set_error("bad c2f_variant (0..2) / smoother (0, 1) / coarse_iters (>= 0) / omega (< 2)");
        return MG_ERR_INVALID_ARG;
    }
    if (cfg->coarse_coef < 0 || cfg->coarse_coef > 1) {
        set_error("bad coarse_coef (0 rediscretised from k, 1 face-averaged)");
        return MG_ERR_INVALID_ARG;
    }
    if (cfg->prolongation < 0 || cfg->prolongation > 1) {
        set_error("bad prolongation (0 face-neighbour linear, 1 trilinear)");
        return MG_ERR_INVALID_ARG;
    }

    if ((cfg->smoother == 1 || cfg->coarse_iters > 0) && cfg->precision != 0) {
        set_error("the damped Jacobi smoother and coarsest solver run FP64 cycles (precision 0)");
        return MG_ERR_INVALID_ARG;
    }
    const int np = std::max(1, cfg->n_problems);
    std::vector<Key> leaves(cfg->n_leaves);
    for (int i = 0; i < cfg->n_leaves; ++i) {
        const int32_t *r = cfg->leaves + 5 * static_cast<int64_t>(i);
        leaves[i] = Key{r[0], r[1], r[2], r[3], r[4]};
    }
    mg_forest *F = new (std::nothrow) mg_forest();
    if (!F) return MG_ERR_OOM;
    F->cfg = *cfg;
    F->cfg.leaves = nullptr;
    if (F->cfg.max_coarse <= 0) F->cfg.max_coarse = 512;
    F->st = static_cast<cudaStream_t>(cfg->stream);
    F->omega = cfg->omega > 0.0 ? cfg->omega : 0.8;
    F->np = np;
    F->cfg.n_problems = np;
    std::string err;
    mg_status st = build_hierarchy(cfg->roots, cfg->n, np, leaves, F->cfg.max_coarse, F->H, err);
    if (st != MG_OK) {
        set_error(err);
        delete F;
        return st;
    }
    auto fail = [&](mg_status s) {
        mg_forest_destroy(F);
        return s;
    };
    const size_t nl = F->H.levels.size();
    F->L.resize(nl);
    for (size_t l = 0; l < nl; ++l) {
        const HostLevel &h = F->H.levels[l];
        DevLevel &d = F->L[l];
        d.g.nb = static_cast<int32_t>(h.keys.size());
        d.g.n = h.n;
        d.g.lg = ilog2(h.n);
        d.g.P = h.n + 2;
        d.g.bs = block_stride(d.g.P);
        d.nfaces = static_cast<int>(h.faces.size());
        d.nsegs = static_cast<int>(h.segs.size());
        if ((st = upload(F, &d.faces, h.faces)) != MG_OK) return fail(st);
        {
            std::vector<int8_t> fk(static_cast<size_t>(h.keys.size()) * 6, 0);
            for (const FaceItem &fi : h.faces) fk[static_cast<size_t>(fi.blk) * 6 + 2 * fi.axis + fi.side] = fi.kind;
            for (const SegItem &si : h.segs) fk[static_cast<size_t>(si.coarse) * 6 + 2 * si.axis + si.side] = 3;
            if ((st = upload(F, &d.fkind, fk)) != MG_OK) return fail(st);
        }
        if ((st = upload(F, &d.segs, h.segs)) != MG_OK) return fail(st);
        {
            std::vector<int32_t> bp(h.keys.size());
            for (size_t b = 0; b < bp.size(); ++b) bp[b] = h.keys[b].p;
            if ((st = upload(F, &d.bprob, bp)) != MG_OK) return fail(st);
            std::vector<int32_t> nb6(h.keys.size() * 6, -2);
            std::vector<FaceItem> itf;
            for (const FaceItem &fi : h.faces) {
                int32_t &slot = nb6[static_cast<size_t>(fi.blk) * 6 + 2 * fi.axis + fi.side];
                if (fi.kind == FK_SAME) slot = fi.nbr;
                else if (fi.kind == FK_BND) slot = -1;
                else itf.push_back(fi);
            }
            if ((st = upload(F, &d.nbr6, nb6)) != MG_OK) return fail(st);
            d.nifaces = static_cast<int>(itf.size());
            if (!itf.empty() && (st = upload(F, &d.ifaces, itf)) != MG_OK) return fail(st);
        }
        if (!h.to_next.empty() && (st = upload(F, &d.xfer, h.to_next)) != MG_OK) return fail(st);
        if (F->cfg.prolongation == 1) {  // edge and corner ghosts for the trilinear prolongation
            build_diagonal(F->H.R, F->H.levels[l]);
            d.nedges = static_cast<int>(h.edges.size());
            d.ncorners = static_cast<int>(h.corners.size());
            if ((st = upload(F, &d.edges, h.edges)) != MG_OK) return fail(st);
            if ((st = upload(F, &d.corners, h.corners)) != MG_OK) return fail(st);
        }
        d.all_halve = !h.to_next.empty() &&
                      std::all_of(h.to_next.begin(), h.to_next.end(), [](const XferItem &x) { return x.kind == XF_HALVE; });
        std::vector<double> h2(h.h.size()), ih2(h.h.size()), vol(h.h.size());
        std::vector<float> h2f(h.h.size()), ih2f(h.h.size()), volf(h.h.size());
        for (size_t b = 0; b < h2.size(); ++b) {
            h2[b] = h.h[b] * h.h[b];
            ih2[b] = 1.0 / h2[b];
            vol[b] = h2[b] * h.h[b];
            h2f[b] = static_cast<float>(h2[b]);
            ih2f[b] = static_cast<float>(ih2[b]);
            volf[b] = static_cast<float>(vol[b]);
        }
        if ((st = upload(F, &d.h2_64, h2)) != MG_OK) return fail(st);
        if ((st = upload(F, &d.ih2_64, ih2)) != MG_OK) return fail(st);
        if ((st = upload(F, &d.vol_64, vol)) != MG_OK) return fail(st);
        if ((st = upload(F, &d.h2_32, h2f)) != MG_OK) return fail(st);
        if ((st = upload(F, &d.ih2_32, ih2f)) != MG_OK) return fail(st);
        if ((st = upload(F, &d.vol_32, volf)) != MG_OK) return fail(st);
        // FP32 cycles need FP64 pools only on the finest level (outer residual, solution) and the coarsest (operator
        // assembly); the FP64 smoother's inverse diagonal only exists for FP64 cycles.  The adjoint and the debug
        // exchange add the missing FP64 coefficient arrays on first use (ensure_fp64_coefficients).
        const int64_t pe = d.pool_elems();
        const bool mixed = cfg->precision == 1;
        const bool fp64 = !mixed || l == 0 || l + 1 == nl;
        if (fp64 && (st = dalloc(F, &d.u64, pe)) != MG_OK) return fail(st);
        if (fp64 && (st = dalloc(F, &d.f64, pe)) != MG_OK) return fail(st);
        const bool jacobi_level = cfg->smoother == 1 || (cfg->coarse_iters > 0 && l + 1 == nl);
        if (jacobi_level && (st = dalloc(F, &d.u64b, pe)) != MG_OK) return fail(st);
        if (mixed) {
            if ((st = dalloc(F, &d.u32, pe)) != MG_OK) return fail(st);
            if ((st = dalloc(F, &d.f32, pe)) != MG_OK) return fail(st);
        }
        if (cfg->coeff) {
            if ((st = dalloc(F, &d.k64, pe)) != MG_OK) return fail(st);
            if (fp64 || cfg->coarse_coef == 1) {  // face-averaged coarse levels derive from every level's FP64 faces
                if ((st = dalloc(F, &d.tx, pe)) != MG_OK) return fail(st);
                if ((st = dalloc(F, &d.ty, pe)) != MG_OK) return fail(st);
                if ((st = dalloc(F, &d.tz, pe)) != MG_OK) return fail(st);
                if ((st = dalloc(F, &d.dg, pe)) != MG_OK) return fail(st);
            }
            if (!mixed && (st = dalloc(F, &d.dinv, pe)) != MG_OK) return fail(st);
            if (mixed && (st = dalloc(F, &d.kap, pe)) != MG_OK) return fail(st);
            if (mixed && cfg->coarse_coef == 1 && l > 0) {  // FP32 cycles on face-averaged coarse levels: mode 3
                if ((st = dalloc(F, &d.ax32, pe)) != MG_OK) return fail(st);
                if ((st = dalloc(F, &d.ay32, pe)) != MG_OK) return fail(st);
                if ((st = dalloc(F, &d.az32, pe)) != MG_OK) return fail(st);
                d.face32 = true;
            }
        }
    }
    if ((st = dalloc(F, &F->partial, 2 * kMaxGrid)) != MG_OK) return fail(st);
    if ((st = dalloc(F, &F->sums, 2)) != MG_OK) return fail(st);
    if ((st = dalloc(F, &F->flag, 1)) != MG_OK) return fail(st);
    if ((st = dalloc(F, &F->kerr, 1)) != MG_OK) return fail(st);
    {
        const HostLevel &h0 = F->H.levels[0];
        std::vector<int32_t> pstart(np + 1, 0), pblk(h0.keys.size());
        for (const Key &k : h0.keys) pstart[k.p + 1] += 1;
        for (int p = 0; p < np; ++p) pstart[p + 1] += pstart[p];
        std::vector<int32_t> fill(pstart.begin(), pstart.end() - 1);
        for (size_t b = 0; b < h0.keys.size(); ++b) pblk[fill[h0.keys[b].p]++] = static_cast<int32_t>(b);
        if ((st = upload(F, &F->pstart, pstart)) != MG_OK) return fail(st);
        if ((st = upload(F, &F->pblk, pblk)) != MG_OK) return fail(st);
        F->bsum_cpb = chunks_per_block(F->L[0]);
        if ((st = dalloc(F, &F->bsum, static_cast<int64_t>(h0.keys.size()) * F->bsum_cpb)) != MG_OK) return fail(st);
        if ((st = dalloc(F, &F->psum, np)) != MG_OK) return fail(st);
        if ((st = dalloc(F, &F->pscale, np)) != MG_OK) return fail(st);
        if ((st = dalloc(F, &F->pinv, np)) != MG_OK) return fail(st);
        if ((st = dalloc(F, &F->pdone, np)) != MG_OK) return fail(st);
        if (cudaMallocHost(&F->psum_h, np * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&F->pscale_h, np * sizeof(float)) != cudaSuccess ||
            cudaMallocHost(&F->pinv_h, np * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&F->pdone_h, np) != cudaSuccess)
            return fail(MG_ERR_OOM);
        std::memset(F->pdone_h, 0, np);
        F->fnorm_p.assign(np, 0.0);
    }
    if (cudaMallocHost(&F->pinned, 2 * sizeof(double)) != cudaSuccess) return fail(MG_ERR_OOM);
    if (!cfg->coeff && (st = assemble_coarse(F)) != MG_OK) return fail(st);
    if (cudaStreamSynchronize(F->st) != cudaSuccess) {
        set_error("stream error during forest creation");
        return fail(MG_ERR_CUDA);
    }
    *out = F;
    return MG_OK;
}

__global__ void k_check_inputs(const double *__restrict__ f, const double *__restrict__ k, int64_t n,
                               int *__restrict__ bad) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (f && !isfinite(f[i])) atomicOr(bad, 1);
        if (k && !(isfinite(k[i]) && k[i] > 0.0)) atomicOr(bad, 2);
    }
}

// Per-problem reference norms of relative residuals: ||f|| (volume-weighted) with g = 0, else the norm of the residual
// of u = 0, i.e. of f plus the boundary data's contribution.
mg_status reference_norms(mg_forest *F) {
    DevLevel &d = F->L[0];
    std::vector<double> sums(F->np, 0.0);
    if (!F->gb) {
        const int cpb = chunks_per_block(d);
        k_block_norm64<<<d.g.nb * cpb, kThreads, 0, F->st>>>(d.f64, d.vol_64, d.g, cpb, F->bsum);
        MG_TRY(read_problem_sums(F));
        for (int p = 0; p < F->np; ++p) sums[p] = F->psum_h[p];
    } else {
        MG_TRY(ensure_scratch64(F));
        MG_CUDA(cudaMemsetAsync(F->s64a, 0, d.pool_elems() * sizeof(double), F->st));
        const std::vector<double> ones(F->np, 1.0);
        MG_TRY(upload_scales(F, ones));
        MG_TRY(residual64_any(F, F->s64a, d.f64, ones, &sums));
    }
    double total = 0.0;
    for (int p = 0; p < F->np; ++p) {
        F->fnorm_p[p] = std::sqrt(sums[p]);
        total += sums[p];
    }
    F->fnorm = std::sqrt(total);
    return MG_OK;
}

__global__ void k_twice(double *__restrict__ out, const double *__restrict__ in, int64_t n) {
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[i] = 2.0 * in[i];
}

// Finite f and finite positive k (either may be null), read back on the host.
mg_status check_inputs(mg_forest *F, const double *f_dev, const double *k_dev) {
    if (F->batch_member) return MG_OK;  // the batch checks its whole fields once
    DevLevel &d = F->L[0];
    MG_CUDA(cudaMemsetAsync(F->flag, 0, sizeof(int), F->st));
    k_check_inputs<<<grid_for(d.cells()), kThreads, 0, F->st>>>(f_dev, k_dev, d.cells(), F->flag);
    int hbad = 0;
    MG_CUDA(cudaMemcpyAsync(&hbad, F->flag, sizeof(int), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (hbad) {
        set_error(hbad & 2 ? "k must be finite and > 0" : "f has a non-finite entry");
        return MG_ERR_NONFINITE;
    }
    return MG_OK;
}

// The k part of mg_set_rhs: coefficient pyramid and coarsest inverse (inputs already checked).
mg_status set_rhs_k(mg_forest *F, const double *k_dev) {
    MG_TRY(pack_user<double>(F, F->L[0], F->L[0].k64, k_dev));
    MG_TRY(build_coefficients(F));
    return assemble_coarse(F);
}

// The f part: the right-hand side, its reference norms and (first call) the launch-shape and tail tuning.
mg_status set_rhs_f(mg_forest *F, const double *f_dev) {
    MG_TRY(pack_user<double>(F, F->L[0], F->L[0].f64, f_dev));
    MG_TRY(reference_norms(F));
    if (F->cfg.precision == 1) {
        MG_TRY(tune_smooth32(F));
        MG_TRY(tune_tail(F));
    }
    F->rhs_set = true;
    return MG_OK;
}

mg_status set_rhs(mg_forest *F, const double *f_dev, const double *k_dev) {
    if (!F || !f_dev) {
        set_error("null forest or f");
        return MG_ERR_INVALID_ARG;
    }
    if (F->cfg.coeff && !k_dev) {
        set_error("coeff == 1 needs k");
        return MG_ERR_INVALID_ARG;
    }
    MG_TRY(check_inputs(F, f_dev, F->cfg.coeff ? k_dev : nullptr));
    if (F->cfg.coeff) MG_TRY(set_rhs_k(F, k_dev));
    return set_rhs_f(F, f_dev);
}

// mg_solve_host: inputs from host buffers through device staging buffers.  k goes first on the forest's stream and
// its set-up (coefficient pyramid, coarsest inverse) runs while f and the initial guess cross on the private copy
// stream; the forest's stream waits for them before the f part.  u comes back on the forest's stream.
mg_status solve_host(mg_forest *F, const double *f_host, const double *k_host, const double *u0_host,
                     double *u_host, double rtol, int32_t max_cycles, int32_t *cycles_out, double *rel_out) {
    if (!F || !f_host || !u_host || (F->cfg.coeff && !k_host) || max_cycles < 0 || !(rtol >= 0.0)) {
        set_error("mg_solve_host: null forest, f or u, k missing with coeff == 1, or bad rtol / max_cycles");
        return MG_ERR_INVALID_ARG;
    }
    if (F->batch_member) {
        set_error("mg_solve_host: not for a batch member forest");
        return MG_ERR_STATE;
    }
    const int64_t cells = F->L[0].cells();
    const size_t bytes = static_cast<size_t>(cells) * sizeof(double);
    if (!F->hst_f) {
        MG_TRY(dalloc(F, &F->hst_f, cells, false));
        MG_TRY(dalloc(F, &F->hst_u, cells, false));
        if (F->cfg.coeff) MG_TRY(dalloc(F, &F->hst_k, cells, false));
    }
    if (!F->cap_st) MG_CUDA(cudaStreamCreateWithFlags(&F->cap_st, cudaStreamNonBlocking));
    if (!F->hst_ev) MG_CUDA(cudaEventCreateWithFlags(&F->hst_ev, cudaEventDisableTiming));
    // the copy stream must not overtake work still queued on the forest's stream that uses the staging buffers
    MG_CUDA(cudaEventRecord(F->hst_ev, F->st));
    MG_CUDA(cudaStreamWaitEvent(F->cap_st, F->hst_ev, 0));
    if (F->cfg.coeff) MG_CUDA(cudaMemcpyAsync(F->hst_k, k_host, bytes, cudaMemcpyHostToDevice, F->st));
    MG_CUDA(cudaMemcpyAsync(F->hst_f, f_host, bytes, cudaMemcpyHostToDevice, F->cap_st));
    if (u0_host) MG_CUDA(cudaMemcpyAsync(F->hst_u, u0_host, bytes, cudaMemcpyHostToDevice, F->cap_st));
    else MG_CUDA(cudaMemsetAsync(F->hst_u, 0, bytes, F->cap_st));
    MG_CUDA(cudaEventRecord(F->hst_ev, F->cap_st));
    if (F->cfg.coeff) {
        mg_status st = check_inputs(F, nullptr, F->hst_k);
        if (st == MG_OK) st = set_rhs_k(F, F->hst_k);
        if (st != MG_OK) {
            cudaStreamSynchronize(F->cap_st);  // the staging copies still read the caller's buffers
            return st;
        }
    }
    MG_CUDA(cudaStreamWaitEvent(F->st, F->hst_ev, 0));
    MG_TRY(check_inputs(F, F->hst_f, nullptr));
    MG_TRY(set_rhs_f(F, F->hst_f));
    MG_TRY(run_cycles(F, F->hst_u, rtol, max_cycles, cycles_out, rel_out));
    MG_CUDA(cudaMemcpyAsync(u_host, F->hst_u, bytes, cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    return MG_OK;
}

mg_status apply_op(mg_forest *F, const double *u_dev, double *Au_dev) {
    if (!F || !u_dev || !Au_dev) {
        set_error("null argument");
        return MG_ERR_INVALID_ARG;
    }
    if (F->cfg.coeff && !F->rhs_set) {
        set_error("mg_set_rhs (k) has not been called");
        return MG_ERR_STATE;
    }
    DevLevel &d = F->L[0];
    MG_TRY(ensure_scratch64(F));
    MG_TRY(pack_user<double>(F, d, F->s64a, u_dev));
    exchange_any64(F, d, F->s64a);
    apply64(F, d, F->s64a, F->s64b);
    MG_TRY(unpack_user<double>(F, d, Au_dev, F->s64b));
    return MG_OK;
}

}  // namespace octmg

using namespace octmg;

extern "C" {

mg_status mg_forest_create(const mg_config *cfg, mg_forest **out) {
    if (out) *out = nullptr;
    return create(cfg, out);
}

void mg_forest_destroy(mg_forest *F) {
    if (!F) return;
    cudaStreamSynchronize(F->st);
    for (void *p : F->allocs) cudaFree(p);
    for (cudaEvent_t e : F->ev_pool) cudaEventDestroy(e);
    if (F->pinned) cudaFreeHost(F->pinned);
    if (F->psum_h) cudaFreeHost(F->psum_h);
    if (F->pscale_h) cudaFreeHost(F->pscale_h);
    if (F->pinv_h) cudaFreeHost(F->pinv_h);
    if (F->pdone_h) cudaFreeHost(F->pdone_h);
    if (F->coarse_graph) cudaGraphExecDestroy(F->coarse_graph);
    if (F->v64_graph) cudaGraphExecDestroy(F->v64_graph);
    if (F->cap_st) cudaStreamDestroy(F->cap_st);
    if (F->hst_ev) cudaEventDestroy(F->hst_ev);
    delete F;
}

mg_status mg_forest_levels(const mg_forest *F, int32_t *n_levels, int32_t *nb_per_level, int32_t *n_per_level) {
    if (!F || !n_levels) {
        set_error("null argument");
        return MG_ERR_INVALID_ARG;
    }
    *n_levels = static_cast<int32_t>(F->L.size());
    for (size_t l = 0; l < F->L.size(); ++l) {
        if (nb_per_level) nb_per_level[l] = F->L[l].g.nb;
        if (n_per_level) n_per_level[l] = F->L[l].g.n;
    }
    return MG_OK;
}

mg_status mg_level_keys(const mg_forest *F, int32_t level, int32_t *keys_host) {
    if (!F || !keys_host || level < 0 || level >= static_cast<int32_t>(F->L.size())) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    const HostLevel &h = F->H.levels[level];
    for (size_t b = 0; b < h.keys.size(); ++b) {
        keys_host[4 * b + 0] = h.keys[b].lev;
        keys_host[4 * b + 1] = h.keys[b].i;
        keys_host[4 * b + 2] = h.keys[b].j;
        keys_host[4 * b + 3] = h.keys[b].k;
    }
    return MG_OK;
}

mg_status mg_set_rhs(mg_forest *F, const double *f_dev, const double *k_dev) { return set_rhs(F, f_dev, k_dev); }

mg_status mg_vcycle(mg_forest *F, double *u_dev, int32_t ncycles, double *rel_res_out) {
    if (!F || !u_dev || ncycles < 0) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    return run_cycles(F, u_dev, -1.0, ncycles, nullptr, rel_res_out);
}

mg_status mg_solve(mg_forest *F, double *u_dev, double rtol, int32_t max_cycles, int32_t *cycles_out,
                   double *rel_res_out) {
    if (!F || !u_dev || max_cycles < 0 || !(rtol >= 0.0)) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    return run_cycles(F, u_dev, rtol, max_cycles, cycles_out, rel_res_out);
}

mg_status mg_solve_host(mg_forest *F, const double *f_host, const double *k_host, const double *u0_host,
                        double *u_host, double rtol, int32_t max_cycles, int32_t *cycles_out, double *rel_res_out) {
    return solve_host(F, f_host, k_host, u0_host, u_host, rtol, max_cycles, cycles_out, rel_res_out);
}

mg_status mg_apply(mg_forest *F, const double *u_dev, double *Au_dev) { return apply_op(F, u_dev, Au_dev); }

mg_status mg_exchange_level(mg_forest *F, int32_t level, const double *u_dev, double *padded_dev) {
    if (!F || !u_dev || !padded_dev || level < 0 || level >= static_cast<int32_t>(F->L.size())) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    if (F->cfg.coeff && !F->rhs_set) {
        set_error("mg_set_rhs (k) has not been called");
        return MG_ERR_STATE;
    }
    MG_TRY(ensure_fp64_coefficients(F));
    DevLevel &d = F->L[level];
    double *pool = nullptr;
    MG_CUDA(cudaStreamSynchronize(F->st));
    MG_CUDA(cudaMalloc(&pool, d.pool_elems() * sizeof(double)));
    cudaMemsetAsync(pool, 0, d.pool_elems() * sizeof(double), F->st);
    k_pack<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(pool, u_dev, d.g);
    exchange_any64(F, d, pool);
    if (F->cfg.prolongation == 1) exchange_diag<double>(F, d, pool);
    const size_t per = static_cast<size_t>(d.g.P) * d.g.P * d.g.P;
    cudaMemcpy2DAsync(padded_dev, per * sizeof(double), pool, d.g.bs * sizeof(double), per * sizeof(double), d.g.nb,
                      cudaMemcpyDeviceToDevice, F->st);
    cudaError_t e = cudaStreamSynchronize(F->st);
    cudaFree(pool);
    if (e != cudaSuccess) {
        set_error(std::string("exchange_level: ") + cudaGetErrorString(e));
        return MG_ERR_CUDA;
    }
    return MG_OK;
}

mg_status mg_get_smoother_shape(const mg_forest *F, int32_t level, int32_t *shape) {
    if (!F || level < 0 || level >= static_cast<int32_t>(F->L.size()) || !shape) {
        set_error("null forest or output, or level out of range");
        return MG_ERR_INVALID_ARG;
    }
    const DevLevel &d = F->L[level];
    const bool used = F->cfg.precision == 1 && smooth32_specialised(d);
    for (int i = 0; i < 5; ++i) shape[i] = used ? d.s32[i] : 0;
    return MG_OK;
}

mg_status mg_set_smoother_shape(mg_forest *F, int32_t level, const int32_t *shape) {
    if (!F || level < 0 || level >= static_cast<int32_t>(F->L.size()) || !shape) {
        set_error("null forest or shape, or level out of range");
        return MG_ERR_INVALID_ARG;
    }
    DevLevel &d = F->L[level];
    if (F->cfg.precision != 1 || !smooth32_specialised(d)) {
        set_error("level " + std::to_string(level) + " has no specialised FP32 smoother");
        return MG_ERR_INVALID_ARG;
    }
    const Shape sh{shape[0], shape[1], shape[2], shape[3], shape[4]};
    if (!smooth32_shape_ok(d, mode32(F, d), sh)) {
        set_error("smoother shape not offered for this level (see mg_smoother_shapes)");
        return MG_ERR_INVALID_ARG;
    }
    d.s32 = sh;
    return MG_OK;
}

mg_status mg_set_boundary(mg_forest *F, const double *g_dev) {
    if (!F) {
        set_error("null forest");
        return MG_ERR_INVALID_ARG;
    }
    if (F->v64_graph) {  // the recorded FP64 cycle holds the boundary-data pointer it was recorded with
        MG_CUDA(cudaStreamSynchronize(F->st));
        cudaGraphExecDestroy(F->v64_graph);
        F->v64_graph = nullptr;
    }
    DevLevel &d = F->L[0];
    if (!g_dev) {
        F->gb = nullptr;
    } else {
        const int64_t cnt = static_cast<int64_t>(d.g.nb) * 6 * d.g.n * d.g.n;
        if (!F->gb_pool) MG_TRY(dalloc(F, &F->gb_pool, cnt));
        MG_CUDA(cudaMemsetAsync(F->flag, 0, sizeof(int), F->st));
        k_check_inputs<<<grid_for(cnt), kThreads, 0, F->st>>>(g_dev, nullptr, cnt, F->flag);
        int hbad = 0;
        MG_CUDA(cudaMemcpyAsync(&hbad, F->flag, sizeof(int), cudaMemcpyDeviceToHost, F->st));
        MG_CUDA(cudaStreamSynchronize(F->st));
        if (hbad) {
            set_error("g has a non-finite entry");
            return MG_ERR_NONFINITE;
        }
        k_twice<<<grid_for(cnt), kThreads, 0, F->st>>>(F->gb_pool, g_dev, cnt);
        F->gb = F->gb_pool;
    }
    if (F->rhs_set) MG_TRY(reference_norms(F));
    MG_CUDA(cudaStreamSynchronize(F->st));
    return MG_OK;
}

mg_status mg_selftest_waits(mg_forest *F, int32_t which) {
    if (!F || (which != 0 && which != 1)) {
        set_error("mg_selftest_waits: null forest or which not in {0, 1}");
        return MG_ERR_INVALID_ARG;
    }
    if (!F->tail_bar) MG_TRY(dalloc(F, &F->tail_bar, 2));
    MG_TRY(launch_selftest_wait(F, which));
    return check_kernel_waits(F);
}

mg_status mg_get_tail(const mg_forest *F, int32_t *level) {
    if (!F || !level) {
        set_error("null forest or output");
        return MG_ERR_INVALID_ARG;
    }
    *level = F->tail_level;
    return MG_OK;
}

mg_status mg_set_tail(mg_forest *F, int32_t level) {
    if (!F) {
        set_error("null forest");
        return MG_ERR_INVALID_ARG;
    }
    if (level < 0) {
        F->tail_level = -1;
        F->tail_tuned = true;
        return MG_OK;
    }
    if (!tail_possible(F, level)) {
        set_error("no persistent tail from level " + std::to_string(level) +
                  " (FP32 cycles and block edges 4..128 on every deeper level required)");
        return MG_ERR_INVALID_ARG;
    }
    MG_TRY(record_tail(F, level));
    F->tail_level = level;
    F->tail_tuned = true;
    return MG_OK;
}

mg_status mg_smoother_shapes(const mg_forest *F, int32_t level, int32_t max_shapes, int32_t *shapes,
                             int32_t *n_shapes) {
    if (!F || level < 0 || level >= static_cast<int32_t>(F->L.size()) || !n_shapes || max_shapes < 0) {
        set_error("null forest or output, or level out of range");
        return MG_ERR_INVALID_ARG;
    }
    const DevLevel &d = F->L[level];
    std::vector<Shape> v;
    if (F->cfg.precision == 1 && smooth32_specialised(d)) v = smooth32_shapes(d, mode32(F, d));
    *n_shapes = static_cast<int32_t>(v.size());
    for (int i = 0; i < static_cast<int>(v.size()) && i < max_shapes && shapes; ++i)
        for (int k = 0; k < 5; ++k) shapes[5 * i + k] = v[i][k];
    return MG_OK;
}

mg_status mg_staged_copy_plan(int32_t lg, int32_t coeff, int32_t colour, int32_t shape_index, int32_t *shape,
                              int32_t *n_shapes, int64_t *smem_bytes, int64_t *block_bytes, int64_t max_records,
                              int64_t *records, int64_t *n_records) {
    if (lg < 5 || lg > 7 || coeff < 0 || coeff > 2 || colour < 0 || colour > 1 || shape_index < 0 || !n_shapes ||
        !n_records || max_records < 0) {
        set_error("mg_staged_copy_plan: lg 5..7, coeff 0..2, colour 0 or 1, shape_index >= 0, outputs not null");
        return MG_ERR_INVALID_ARG;
    }
    const int mode = coeff == 2 ? 3 : (coeff ? 2 : 0);
    DevLevel d;
    d.g.n = 1 << lg;
    d.g.lg = lg;
    d.g.P = d.g.n + 2;
    std::vector<Shape> staged;
    for (const Shape &sh : smooth32_shapes(d, mode))
        if (sh[0] == 2) staged.push_back(sh);
    *n_shapes = static_cast<int32_t>(staged.size());
    *n_records = 0;
    if (shape_index >= static_cast<int32_t>(staged.size())) return MG_OK;
    const Shape sh = staged[shape_index];
    if (shape)
        for (int k = 0; k < 5; ++k) shape[k] = sh[k];
    const int TY = sh[1], TZ = sh[2], D = sh[3], n = d.g.n;
    const S32tPlan plan = s32t_plan(lg, s32t_arrays(mode), TY, D);
    const int64_t half = static_cast<int64_t>(plan.P) * plan.P * plan.H;
    const int64_t bs = block_stride(d.g.P);
    if (smem_bytes) *smem_bytes = static_cast<int64_t>(smooth32t_smem(lg, mode, TY, D));
    if (block_bytes) *block_bytes = 4 * bs;
    // the kernel's halves: the colour being updated is stored in half s = colour ^ 1, the other one in half colour
    const int64_t own = (colour ^ 1) * half, other = static_cast<int64_t>(colour) * half;
    struct HostSink {
        int64_t *rec, cap, *cnt, tile, group, other, own;
        const S32tPlan *p;
        void put(const int64_t (&v)[10]) {
            if (*cnt < cap && rec)
                for (int i = 0; i < 10; ++i) rec[10 * *cnt + i] = v[i];
            ++*cnt;
        }
        void arm(int bi, uint32_t bytes) { put({tile, 0, bi, group, -1, -1, -1, static_cast<int64_t>(bytes), -1, -1}); }
        void copy(int dst, int array, int off, int lead, uint32_t bytes, int bi) {
            const bool oth = array < 2 || array == 4 || array == 5;
            const int64_t src = (oth ? other : own) + off;
            const int len = oth ? p->lo : p->lw;
            put({tile, 1, bi, group, 4 * static_cast<int64_t>(dst), array, 4 * src, static_cast<int64_t>(bytes), lead,
                 len});
        }
    };
    HostSink sink{records, max_records, n_records, 0, -1, other, own, &plan};
    for (int tz = 0; tz < n / TZ; ++tz)
        for (int ty = 0; ty < n / TY; ++ty) {
            sink.tile = static_cast<int64_t>(tz) * (n / TY) + ty;
            const int y0 = ty * TY, z0 = tz * TZ;
            sink.group = -1;
            s32t_issue_first(plan, z0, y0, sink);
            for (int g = 0; g < TZ; ++g) {
                sink.group = g;
                s32t_issue_group(plan, z0, y0, g, sink);
            }
        }
    return MG_OK;
}

mg_status mg_restrict_copy_plan(int32_t lg, int32_t coeff, int32_t *shape, int64_t *smem_bytes,
                                int64_t *block_bytes, int64_t max_records, int64_t *records, int64_t *n_records) {
    if (lg < 6 || lg > 7 || coeff < 0 || coeff > 2 || !shape || !n_records || max_records < 0) {
        set_error("mg_restrict_copy_plan: lg 6 or 7, coeff 0..2, shape and n_records not null");
        return MG_ERR_INVALID_ARG;
    }
    DevLevel d;
    d.g.n = 1 << lg;
    d.g.lg = lg;
    d.g.P = d.g.n + 2;
    const int n = d.g.n, mode = coeff == 2 ? 3 : (coeff ? 2 : 0);
    if (shape[0] == 0) {
        const std::array<int, 3> sh = restrict32t_shape(d);
        for (int k = 0; k < 3; ++k) shape[k] = sh[k];
    }
    const int TY = shape[0], TZ = shape[1], D = shape[2];
    if (TY < 2 || TY > n || (TY & 1) || n % TY || (n / 2) * (TY / 2) + 32 > 544 || TZ < 2 || TZ > n || (TZ & 1) ||
        n % TZ || D < 0 || D > 4 || restrict32t_smem(lg, mode, TY, TZ, D) > 200 * 1024) {
        set_error("mg_restrict_copy_plan: TY, TZ even divisors of the block edge, at most 544 threads, D 0..4, "
                  "at most 200 KB of shared memory");
        return MG_ERR_INVALID_ARG;
    }
    const R32tPlan plan = r32t_plan(lg, mode, TY, TZ, D);
    const int64_t half = static_cast<int64_t>(plan.P) * plan.P * plan.H;
    if (smem_bytes) *smem_bytes = static_cast<int64_t>(r32t_smem_bytes(plan));
    if (block_bytes) *block_bytes = 4 * block_stride(d.g.P);
    struct HostSink {
        int64_t *rec, cap, *cnt, tile, plane, half;
        const R32tPlan *p;
        void put(const int64_t (&v)[11]) {
            if (*cnt < cap && rec)
                for (int i = 0; i < 11; ++i) rec[11 * *cnt + i] = v[i];
            ++*cnt;
        }
        void arm(int slot, uint32_t bytes) { put({tile, 0, slot, plane, -1, -1, -1, -1, static_cast<int64_t>(bytes), -1, -1}); }
        void copy(int dst, int array, int h, int off, int lead, uint32_t bytes, int slot) {
            put({tile, 1, slot, plane, 4 * static_cast<int64_t>(dst), array, h, 4 * (h * half + off),
                 static_cast<int64_t>(bytes), lead, array < p->NU ? p->lo : p->lw});
        }
    };
    *n_records = 0;
    HostSink sink{records, max_records, n_records, 0, 0, half, &plan};
    for (int tz = 0; tz < n / TZ; ++tz)
        for (int ty = 0; ty < n / TY; ++ty) {
            sink.tile = static_cast<int64_t>(tz) * (n / TY) + ty;
            for (int q = 0; q < TZ + 2; ++q) {
                sink.plane = q;
                r32t_issue_plane(plan, tz * TZ, ty * TY, q, sink);
            }
        }
    return MG_OK;
}

mg_status mg_profile(mg_forest *F, int32_t enable) {
    if (!F) {
        set_error("null forest");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (enable) {
        F->recs.clear();
        F->ev_used = 0;
        for (int c = 0; c < P_NCAT; ++c) F->nlaunch[c] = 0;
    }
    F->prof = enable != 0;
    return MG_OK;
}

mg_status mg_profile_read(mg_forest *F, int32_t max_families, char *names, double *ms, int64_t *launches,
                          int32_t *n_families) {
    if (!F || !n_families || max_families < 0) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaStreamSynchronize(F->st));
    double acc[P_NCAT] = {};
    for (auto &r : F->recs) {
        float t = 0.0f;
        MG_CUDA(cudaEventElapsedTime(&t, F->ev_pool[r.second], F->ev_pool[r.second + 1]));
        acc[r.first] += t;
    }
    *n_families = P_NCAT;
    for (int c = 0; c < P_NCAT && c < max_families; ++c) {
        if (names) {
            std::strncpy(names + 32 * c, kProfNames[c], 31);
            names[32 * c + 31] = 0;
        }
        if (ms) ms[c] = acc[c];
        if (launches) launches[c] = F->nlaunch[c];
    }
    return MG_OK;
}

const char *mg_last_error(void) { return g_err.c_str(); }

}  // extern "C"

