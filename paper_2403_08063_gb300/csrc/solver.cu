// The forest object, the V-cycle driver and the C-ABI entry points (include/octmg.h).
#include <algorithm>
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
                                         "update_mixed", "layout", "adjoint"};

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

template <typename T, int MODE>
void exchange(mg_forest *F, DevLevel &d, T *u) {
    Prof p(F, cat_of<T>(P_EXCH64), (d.nfaces ? 1 : 0) + (d.nsegs ? 1 : 0));
    if (d.nfaces)
        k_exchange_faces<T, false><<<grid_for(static_cast<int64_t>(d.nfaces) * d.g.n * d.g.n), kThreads, 0, F->st>>>(
            u, d.faces, d.nfaces, d.g);
    if (d.nsegs) {
        const int64_t tot = static_cast<int64_t>(d.nsegs) * (d.g.n / 2) * (d.g.n / 2);
        if (F->cfg.interface_flux)
            k_exchange_segs<T, MODE, true><<<grid_for(tot), kThreads, 0, F->st>>>(u, coef_of<T>(d), d.segs, d.nsegs, d.g);
        else
            k_exchange_segs<T, MODE, false><<<grid_for(tot), kThreads, 0, F->st>>>(u, coef_of<T>(d), d.segs, d.nsegs, d.g);
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

template <typename T, int MODE>
void smooth(mg_forest *F, DevLevel &d, int colour) {
    Prof p(F, cat_of<T>(P_SMOOTH64), 1);
    k_smooth<T, MODE><<<grid_for(d.cells() / 2), kThreads, 0, F->st>>>(ufield<T>(d), ffield<T>(d), coef_of<T>(d),
                                                                       h2_of<T>(d), d.g, colour);
}

template <typename T, int MODE>
void vcycle(mg_forest *F, int l) {
    DevLevel &d = F->L[l];
    const int last = static_cast<int>(F->L.size()) - 1;
    if (l == last) {
        Prof p(F, cat_of<T>(P_COARSE64), 1);
        k_coarse_solve<T><<<(F->Nc * 32 + kThreads - 1) / kThreads, kThreads, 0, F->st>>>(ufield<T>(d), ffield<T>(d),
                                                                                          F->Ainv, F->cmap, F->Nc);
        return;
    }
    for (int i = 0; i < F->cfg.nu1; ++i) {
        exchange<T, MODE>(F, d, ufield<T>(d));
        smooth<T, MODE>(F, d, 0);
        exchange<T, MODE>(F, d, ufield<T>(d));
        smooth<T, MODE>(F, d, 1);
    }
    exchange<T, MODE>(F, d, ufield<T>(d));
    DevLevel &c = F->L[l + 1];
    {
        Prof p(F, cat_of<T>(P_RESTR64), 1);
        k_residual_restrict<T, MODE><<<grid_for(c.cells()), kThreads, 0, F->st>>>(
            ufield<T>(d), ffield<T>(d), coef_of<T>(d), ih2_of<T>(d), d.g, ffield<T>(c), ufield<T>(c), d.xfer, c.g);
    }
    vcycle<T, MODE>(F, l + 1);
    exchange<T, MODE>(F, c, ufield<T>(c));
    {
        Prof p(F, cat_of<T>(P_PROL64), 1);
        k_prolong<T><<<grid_for(c.cells()), kThreads, 0, F->st>>>(ufield<T>(d), d.g, ufield<T>(c), d.xfer, c.g);
    }
    for (int i = 0; i < F->cfg.nu2; ++i) {
        exchange<T, MODE>(F, d, ufield<T>(d));
        smooth<T, MODE>(F, d, 0);
        exchange<T, MODE>(F, d, ufield<T>(d));
        smooth<T, MODE>(F, d, 1);
    }
}

// Level-0 FP64 residual r = f - A u (exchange first); optionally written as FP32 r * scale with the FP32
// correction zeroed; returns ||r||^2 (volume-weighted) to the host when rr is not null.  scale is a power of two
// close to 1 / ||r|| so the FP32 values stay near unit size.
template <int MODE>
mg_status residual64(mg_forest *F, double *u, const double *f, float *out, double scale, float *zero_out,
                     double *rr) {
    DevLevel &d = F->L[0];
    exchange<double, MODE>(F, d, u);
    const int grid = grid_for(d.cells());
    {
        Prof p(F, P_RESID64, 2);
        k_residual_norm<MODE><<<grid, kThreads, 0, F->st>>>(u, f, d.c64(), d.ih2_64, d.vol_32, d.g, out,
                                                            static_cast<float>(scale), F->partial, zero_out);
        k_sum_partials<<<1, kThreads, 0, F->st>>>(F->partial, grid, F->sums);
    }
    if (rr) {
        MG_CUDA(cudaMemcpyAsync(F->pinned, F->sums, sizeof(double), cudaMemcpyDeviceToHost, F->st));
        MG_CUDA(cudaStreamSynchronize(F->st));
        *rr = F->pinned[0] / (scale * scale);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

mg_status residual64_any(mg_forest *F, double *u, const double *f, double scale, double *rr) {
    if (F->cfg.coeff) return residual64<1>(F, u, f, nullptr, scale, nullptr, rr);
    return residual64<0>(F, u, f, nullptr, scale, nullptr, rr);
}

void apply64(mg_forest *F, DevLevel &d, const double *u, double *out) {
    if (F->cfg.coeff)
        k_apply64<1><<<grid_for(d.cells()), kThreads, 0, F->st>>>(u, d.c64(), d.ih2_64, d.g, out);
    else
        k_apply64<0><<<grid_for(d.cells()), kThreads, 0, F->st>>>(u, d.c64(), d.ih2_64, d.g, out);
}

// Coarsest-level dense operator (FP64 kernels on unit vectors), inverted on the host, uploaded.
mg_status assemble_coarse(mg_forest *F) {
    const int l = static_cast<int>(F->L.size()) - 1;
    DevLevel &d = F->L[l];
    const int N = static_cast<int>(d.cells());
    F->Nc = N;
    if (!F->cmap) {
        std::vector<int64_t> cmap(N);
        const int n = d.g.n;
        for (int b = 0, m = 0; b < d.g.nb; ++b)
            for (int z = 0; z < n; ++z)
                for (int y = 0; y < n; ++y)
                    for (int x = 0; x < n; ++x) cmap[m++] = b * d.g.bs + off3(x + 1, y + 1, z + 1, d.g.P);
        MG_TRY(upload(F, &F->cmap, cmap));
        MG_TRY(dalloc(F, &F->Ainv, static_cast<int64_t>(N) * N));
    }
    if (!F->coarse_r) MG_TRY(dalloc(F, &F->coarse_r, d.pool_elems()));
    double *r = F->coarse_r, *Adev = F->Ainv;
    for (int m = 0; m < N; ++m) {
        MG_CUDA(cudaMemsetAsync(d.u64, 0, d.pool_elems() * sizeof(double), F->st));
        k_set_unit<<<1, 32, 0, F->st>>>(d.u64, F->cmap, m);
        exchange_any64(F, d, d.u64);
        apply64(F, d, d.u64, r);
        k_gather_column<<<(N + 255) / 256, 256, 0, F->st>>>(r, F->cmap, N, Adev, m);
    }
    MG_CUDA(cudaGetLastError());
    std::vector<double> A(static_cast<size_t>(N) * N);
    MG_CUDA(cudaMemcpyAsync(A.data(), Adev, A.size() * sizeof(double), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (!invert_dense(A, N)) {
        set_error("coarsest-level operator is singular");
        return MG_ERR_INVALID_ARG;
    }
    MG_CUDA(cudaMemcpyAsync(Adev, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, F->st));
    {
        std::vector<double> At(A.size());
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) At[static_cast<size_t>(j) * N + i] = A[static_cast<size_t>(i) * N + j];
        if (!F->AinvT) MG_TRY(dalloc(F, &F->AinvT, static_cast<int64_t>(N) * N));
        MG_CUDA(cudaMemcpyAsync(F->AinvT, At.data(), At.size() * sizeof(double), cudaMemcpyHostToDevice, F->st));
        MG_CUDA(cudaStreamSynchronize(F->st));
    }
    MG_CUDA(cudaMemsetAsync(d.u64, 0, d.pool_elems() * sizeof(double), F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
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
        k_face_coefs<<<grid_for(d.pool_elems()), kThreads, 0, F->st>>>(d.k64, d.ih2_64, d.g, d.tx, d.ty, d.tz,
                                                                        d.kap);
        k_diag<<<grid_for(d.cells()), kThreads, 0, F->st>>>(d.tx, d.ty, d.tz, d.g, d.dg, d.dinv);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

template <typename T>
mg_status pack_user(mg_forest *F, DevLevel &d, T *pool, const double *user) {
    Prof p(F, P_LAYOUT, 1);
    k_pack<T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(pool, user, d.g);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

template <typename T>
mg_status unpack_user(mg_forest *F, DevLevel &d, double *user, const T *pool) {
    Prof p(F, P_LAYOUT, 1);
    k_unpack<T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(user, pool, d.g);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

// One FP64 V-cycle on level 0.
void vcycle64(mg_forest *F) {
    if (F->cfg.coeff) vcycle<double, 1>(F, 0);
    else vcycle<double, 0>(F, 0);
}
void vcycle32(mg_forest *F) {
    if (F->cfg.coeff) vcycle<float, 2>(F, 0);
    else vcycle<float, 0>(F, 0);
}

double pow2_near(double x) {
    if (!(x > 0.0) || !std::isfinite(x)) return 1.0;
    return std::ldexp(1.0, static_cast<int>(std::lround(std::log2(x))));
}

// Mixed precision: r64 = f - A u (FP64), written as FP32 r / s; FP32 V-cycle; u += s e.  `iters` outer steps;
// returns the relative residual measured before the last update when `final_rel` is requested afterwards.
mg_status mixed_step(mg_forest *F, double scale, double *rr) {
    DevLevel &d = F->L[0];
    if (F->cfg.coeff)
        MG_TRY((residual64<1>(F, d.u64, d.f64, d.f32, scale, d.u32, rr)));
    else
        MG_TRY((residual64<0>(F, d.u64, d.f64, d.f32, scale, d.u32, rr)));
    return MG_OK;
}

// `cycles` FP32 V-cycles on the scaled residual, then u64 += e32 / mult (mult a power of two: exact).
mg_status finish_mixed_cycle(mg_forest *F, double inv_mult, int cycles) {
    DevLevel &d = F->L[0];
    for (int i = 0; i < cycles; ++i) vcycle32(F);
    Prof p(F, P_UPDATE, 1);
    k_update_mixed<<<grid_for(d.cells()), kThreads, 0, F->st>>>(d.u64, d.u32, inv_mult, d.g);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

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

// Runs cycles until rel <= rtol (rtol < 0: exactly max_cycles).  u_dev in/out.
mg_status run_cycles(mg_forest *F, double *u_dev, double rtol, int max_cycles, int *cycles_out, double *rel_out) {
    MG_TRY(check_ready(F));
    DevLevel &d = F->L[0];
    MG_TRY(pack_user<double>(F, d, d.u64, u_dev));
    const double fn = F->fnorm > 0.0 ? F->fnorm : 1.0;
    int done = 0;
    double rel = -1.0;
    double mult = pow2_near(1.0 / fn);  // FP32 values of residuals are scaled by a power of two near 1/||r||
    if (F->cfg.precision == 0) {
        for (; done < max_cycles; ++done) {
            if (rtol >= 0.0 && done > 0 && rel <= rtol) break;
            vcycle64(F);
            double rr = 0.0;
            if (rtol >= 0.0 || rel_out || done + 1 == max_cycles) {
                MG_TRY(residual64_any(F, d.u64, d.f64, mult, &rr));
                rel = std::sqrt(rr) / fn;
                mult = pow2_near(1.0 / std::sqrt(rr));
                if (!std::isfinite(rel)) {
                    set_error("residual is not finite");
                    ++done;
                    break;
                }
            }
        }
    } else {
        double rr = 0.0;
        MG_TRY(mixed_step(F, mult, &rr));
        rel = std::sqrt(rr) / fn;
        const int inner = std::max(1, F->cfg.inner_cycles);
        while (done < max_cycles) {
            if (rtol >= 0.0 && rel <= rtol) break;
            const int m = std::min(inner, max_cycles - done);
            MG_TRY(finish_mixed_cycle(F, 1.0 / mult, m));
            done += m;
            mult = pow2_near(1.0 / std::sqrt(rr));
            MG_TRY(mixed_step(F, mult, &rr));
            rel = std::sqrt(rr) / fn;
            if (!std::isfinite(rel)) {
                set_error("residual is not finite");
                break;
            }
        }
    }
    MG_TRY(unpack_user<double>(F, d, u_dev, d.u64));
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (cycles_out) *cycles_out = done;
    if (rel_out) *rel_out = rel;
    if (!std::isfinite(rel)) return MG_ERR_NOT_CONVERGED;
    if (rtol >= 0.0 && !(rel <= rtol)) {
        set_error("relative residual " + fmt_e(rel) + " above rtol after " + std::to_string(done) + " cycles");
        return MG_ERR_NOT_CONVERGED;
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
    std::vector<Key> leaves(cfg->n_leaves);
    for (int i = 0; i < cfg->n_leaves; ++i) {
        const int32_t *r = cfg->leaves + 5 * static_cast<int64_t>(i);
        if (r[0] != 0) {
            set_error("leaf problem index must be 0 for a single forest");
            return MG_ERR_INVALID_ARG;
        }
        leaves[i] = Key{r[1], r[2], r[3], r[4]};
    }
    mg_forest *F = new (std::nothrow) mg_forest();
    if (!F) return MG_ERR_OOM;
    F->cfg = *cfg;
    F->cfg.leaves = nullptr;
    if (F->cfg.max_coarse <= 0) F->cfg.max_coarse = 512;
    F->st = static_cast<cudaStream_t>(cfg->stream);
    std::string err;
    mg_status st = build_hierarchy(cfg->roots, cfg->n, leaves, F->cfg.max_coarse, F->H, err);
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
        const int64_t per = static_cast<int64_t>(d.g.P) * d.g.P * d.g.P;
        d.g.bs = (per + 31) / 32 * 32;
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
        if (!h.to_next.empty() && (st = upload(F, &d.xfer, h.to_next)) != MG_OK) return fail(st);
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
        const int64_t pe = d.pool_elems();
        if ((st = dalloc(F, &d.u64, pe)) != MG_OK) return fail(st);
        if ((st = dalloc(F, &d.f64, pe)) != MG_OK) return fail(st);
        if (cfg->precision == 1) {
            if ((st = dalloc(F, &d.u32, pe)) != MG_OK) return fail(st);
            if ((st = dalloc(F, &d.f32, pe)) != MG_OK) return fail(st);
        }
        if (cfg->coeff) {
            if ((st = dalloc(F, &d.k64, pe)) != MG_OK) return fail(st);
            if ((st = dalloc(F, &d.tx, pe)) != MG_OK) return fail(st);
            if ((st = dalloc(F, &d.ty, pe)) != MG_OK) return fail(st);
            if ((st = dalloc(F, &d.tz, pe)) != MG_OK) return fail(st);
            if ((st = dalloc(F, &d.dg, pe)) != MG_OK) return fail(st);
            if ((st = dalloc(F, &d.dinv, pe)) != MG_OK) return fail(st);
            if (cfg->precision == 1 && (st = dalloc(F, &d.kap, pe)) != MG_OK) return fail(st);
        }
    }
    if ((st = dalloc(F, &F->partial, 2 * kMaxGrid)) != MG_OK) return fail(st);
    if ((st = dalloc(F, &F->sums, 2)) != MG_OK) return fail(st);
    if ((st = dalloc(F, &F->flag, 1)) != MG_OK) return fail(st);
    if ((st = dalloc(F, &F->s64a, F->L[0].pool_elems())) != MG_OK) return fail(st);
    if ((st = dalloc(F, &F->s64b, F->L[0].pool_elems())) != MG_OK) return fail(st);
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
        if (!isfinite(f[i])) atomicOr(bad, 1);
        if (k && !(isfinite(k[i]) && k[i] > 0.0)) atomicOr(bad, 2);
    }
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
    DevLevel &d = F->L[0];
    int *bad = F->flag;
    MG_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), F->st));
    k_check_inputs<<<grid_for(d.cells()), kThreads, 0, F->st>>>(f_dev, F->cfg.coeff ? k_dev : nullptr, d.cells(), bad);
    int hbad = 0;
    MG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (hbad) {
        set_error(hbad & 2 ? "k must be finite and > 0" : "f has a non-finite entry");
        return MG_ERR_NONFINITE;
    }
    MG_TRY(pack_user<double>(F, d, d.f64, f_dev));
    if (F->cfg.coeff) {
        MG_TRY(pack_user<double>(F, d, d.k64, k_dev));
        MG_TRY(build_coefficients(F));
        MG_TRY(assemble_coarse(F));
    }
    const int grid = grid_for(d.cells());
    k_norm64<<<grid, kThreads, 0, F->st>>>(d.f64, d.vol_64, d.g, F->partial);
    k_sum_partials<<<1, kThreads, 0, F->st>>>(F->partial, grid, F->sums);
    MG_CUDA(cudaMemcpyAsync(F->pinned, F->sums, sizeof(double), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    F->fnorm = std::sqrt(F->pinned[0]);
    F->rhs_set = true;
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
    DevLevel &d = F->L[level];
    double *pool = nullptr;
    MG_CUDA(cudaStreamSynchronize(F->st));
    MG_CUDA(cudaMalloc(&pool, d.pool_elems() * sizeof(double)));
    cudaMemsetAsync(pool, 0, d.pool_elems() * sizeof(double), F->st);
    k_pack<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(pool, u_dev, d.g);
    exchange_any64(F, d, pool);
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

