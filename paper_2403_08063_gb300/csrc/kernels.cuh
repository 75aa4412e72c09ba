// Device kernels of the octree-block multigrid (arXiv 2403.08063), written for sm_103a.
//
// Storage: every block of a level is a padded (n+2)^3 array, x fastest (padded coordinate = interior + 1), one
// ghost layer per face (Sec. 3.3: one layer suffices for the quadratic C2F / linear F2C schemes).  The blocks of
// a level are contiguous with a stride `bs` (elements) rounded up to 256 bytes.
//
// Coefficient modes (template parameter MODE):
//   0  constant coefficient, -Laplace: every face coefficient T_f = 1;
//   1  variable k in FP64, face coefficients precomputed and scaled by the block's 1/h^2:
//      tx/ty/tz[idx] = T_f / h^2 of the face between padded cells idx - stride and idx along that axis
//      (T_f the harmonic mean 2 k_a k_b / (k_a + k_b)), dg[idx] = their sum over the six faces, dinv = 1 / dg;
//      the residual is then f + sum_f T~_f u_f - dg u, seven FMAs per cell;
//   2  variable k in FP32: kap[idx] = 1/k with ghosts; T_f = 2 / (kap_i + kap_nb) evaluated with rcp.approx.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "octmg_internal.h"

namespace octmg {

constexpr int kThreads = 256;

struct LevelGeom {
    int32_t nb;     // blocks
    int32_t n;      // interior cells per edge (power of two)
    int32_t lg;     // log2(n)
    int32_t P;      // n + 2
    int64_t bs;     // block stride in elements
};

struct Coef {       // coefficient arrays of one level (unused members are null)
    const double *tx, *ty, *tz, *dg, *dinv;  // MODE 1
    const float *kap;                        // MODE 2
};

__host__ __device__ inline int64_t off3(int X, int Y, int Z, int P) {
    return (static_cast<int64_t>(Z) * P + Y) * P + X;
}

__device__ inline int axis_stride(int axis, int P) { return axis == 0 ? 1 : (axis == 1 ? P : P * P); }

// Offset, inside one padded block, of the cell at `depth` from face (axis, side) (depth 0 = ghost layer,
// 1 = first interior layer) and interior tangential coordinates (i1, i2) along t1 < t2, the other two axes.
__device__ inline int face_off(int axis, int side, int depth, int i1, int i2, int n, int P) {
    const int t1 = axis == 0 ? 1 : 0;
    const int t2 = axis == 2 ? 1 : 2;
    const int a = side ? (n + 1 - depth) : depth;
    return a * axis_stride(axis, P) + (1 + i1) * axis_stride(t1, P) + (1 + i2) * axis_stride(t2, P);
}

// ------------------------------------------------------------------------------------------------------------
// Quadratic coarse-to-fine weights (Sec. 3.3.2).  Lagrange basis through three coarse bases evaluated at the
// fine-ghost target; distances in coarse cells.
//   Normal step: bases = current cell and the two cells inward (0, 1, 2); target 1/4 outward (-1/4):
//     w = (45, -18, 5) / 32.
//   Orthogonal step, bases {-1, 0, +1} (case 0), targets -1/4 (downwind fine cell) and +1/4 (upwind):
//     (5, 30, -3) / 32 and (-3, 30, 5) / 32.
//   Downwind neighbour in the ghost region, remapped to +2 (case 1, bases {0, 1, 2}):
//     (45, -18, 5) / 32 and (21, 14, -3) / 32.
//   Upwind neighbour remapped to -2 (case 2, bases {-2, -1, 0}):
//     (-3, 14, 21) / 32 and (5, -18, 45) / 32.
// ------------------------------------------------------------------------------------------------------------
static __constant__ double c_wn[3] = {45.0 / 32, -18.0 / 32, 5.0 / 32};
static __constant__ double c_wt[3][2][3] = {
    {{5.0 / 32, 30.0 / 32, -3.0 / 32}, {-3.0 / 32, 30.0 / 32, 5.0 / 32}},
    {{45.0 / 32, -18.0 / 32, 5.0 / 32}, {21.0 / 32, 14.0 / 32, -3.0 / 32}},
    {{-3.0 / 32, 14.0 / 32, 21.0 / 32}, {5.0 / 32, -18.0 / 32, 45.0 / 32}}};
static __constant__ int c_base[3][3] = {{-1, 0, 1}, {0, 1, 2}, {-2, -1, 0}};
static __constant__ float c_wn_f[3] = {45.0f / 32, -18.0f / 32, 5.0f / 32};
static __constant__ float c_wt_f[3][2][3] = {
    {{5.0f / 32, 30.0f / 32, -3.0f / 32}, {-3.0f / 32, 30.0f / 32, 5.0f / 32}},
    {{45.0f / 32, -18.0f / 32, 5.0f / 32}, {21.0f / 32, 14.0f / 32, -3.0f / 32}},
    {{-3.0f / 32, 14.0f / 32, 21.0f / 32}, {5.0f / 32, -18.0f / 32, 45.0f / 32}}};

template <typename T> __device__ inline T w_normal(int a);
template <> __device__ inline double w_normal<double>(int a) { return c_wn[a]; }
template <> __device__ inline float w_normal<float>(int a) { return c_wn_f[a]; }
template <typename T> __device__ inline T w_tang(int c, int al, int b);
template <> __device__ inline double w_tang<double>(int c, int al, int b) { return c_wt[c][al][b]; }
template <> __device__ inline float w_tang<float>(int c, int al, int b) { return c_wt_f[c][al][b]; }

__device__ inline float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Face coefficient of the face between depth 0 and depth 1 of a block face, stored (MODE 1) or evaluated (MODE 2)
// at the cell with the larger padded coordinate along the axis: `loc`; `other` is the cell across the face.
template <typename T, int MODE>
__device__ inline T face_coef(const Coef &c, int64_t loc, int64_t other, int axis) {
    if (MODE == 0) return T(1);
    if (MODE == 1) {
        const double *t = axis == 0 ? c.tx : (axis == 1 ? c.ty : c.tz);
        return T(t[loc]);
    }
    return T(2.0f * frcp(c.kap[loc] + c.kap[other]));
}

// MODE 1: init + sum_f T~_f u_f over the six faces of padded cell g.
__device__ inline double sten1(const double *__restrict__ u, const Coef &c, int64_t g, int P, double init) {
    const int64_t PP = static_cast<int64_t>(P) * P;
    double a = fma(c.tx[g], u[g - 1], init);
    a = fma(c.tx[g + 1], u[g + 1], a);
    a = fma(c.ty[g], u[g - P], a);
    a = fma(c.ty[g + P], u[g + P], a);
    a = fma(c.tz[g], u[g - PP], a);
    a = fma(c.tz[g + PP], u[g + PP], a);
    return a;
}

// MODE 0: plain sum of the six neighbours.
template <typename T>
__device__ inline T sten0(const T *__restrict__ u, int64_t g, int P) {
    const int64_t PP = static_cast<int64_t>(P) * P;
    return ((u[g - 1] + u[g + 1]) + (u[g - P] + u[g + P])) + (u[g - PP] + u[g + PP]);
}

// MODE 2: S = sum_f T_f u_f and D = sum_f T_f with T_f = 2 / (kap_i + kap_f), in FP32.
__device__ inline void sten2(const float *__restrict__ u, const float *__restrict__ kap, int64_t g, int P, float &S,
                             float &D) {
    const int64_t PP = static_cast<int64_t>(P) * P;
    const float k0 = kap[g];
    const float a0 = frcp(k0 + kap[g - 1]), a1 = frcp(k0 + kap[g + 1]);
    const float b0 = frcp(k0 + kap[g - P]), b1 = frcp(k0 + kap[g + P]);
    const float c0 = frcp(k0 + kap[g - PP]), c1 = frcp(k0 + kap[g + PP]);
    float s = a0 * u[g - 1];
    s = fmaf(a1, u[g + 1], s);
    s = fmaf(b0, u[g - P], s);
    s = fmaf(b1, u[g + P], s);
    s = fmaf(c0, u[g - PP], s);
    s = fmaf(c1, u[g + PP], s);
    S = 2.0f * s;
    D = 2.0f * (((a0 + a1) + (b0 + b1)) + (c0 + c1));
}

// Point-form residual r = f - A u at padded cell g (ih2 = 1/h^2 of the block; unused in MODE 1).
template <typename T, int MODE>
__device__ inline T residual_at(const T *__restrict__ u, const T *__restrict__ f, const Coef &cf, int64_t g, int P,
                                T ih2) {
    const T fv = f ? f[g] : T(0);
    if constexpr (MODE == 1) {
        return fma(-cf.dg[g], u[g], sten1(u, cf, g, P, fv));
    } else if constexpr (MODE == 0) {
        const T S = sten0<T>(u, g, P);
        return fma(fma(T(-6), u[g], S), ih2, fv);
    } else {
        float S, D;
        sten2(reinterpret_cast<const float *>(u), cf.kap, g, P, S, D);
        return T(fmaf(fmaf(-D, float(u[g]), S), float(ih2), float(fv)));
    }
}

// A u at padded cell g (FP64 operator application; f = 0).
template <int MODE>
__device__ inline double apply_at(const double *__restrict__ u, const Coef &cf, int64_t g, int P, double ih2) {
    return -residual_at<double, MODE>(u, nullptr, cf, g, P, ih2);
}

// ------------------------------------------------------------------------------------------------------------
// Ghost exchange, part 1: whole faces filled from one source block (boundary, same level, C2F).
// KIND_K = false: solution-type field (Dirichlet reflection ghost = -u_i; quadratic C2F extrapolation).
// KIND_K = true:  coefficient field k (ghost = k_i at the boundary; fine ghosts inject the covering coarse k).
// One thread per ghost cell; n is a power of two, so items and cells decode with shifts.
// ------------------------------------------------------------------------------------------------------------
template <typename T, bool KIND_K>
static __global__ void k_exchange_faces(T *__restrict__ u, const FaceItem *__restrict__ items, int nitems, LevelGeom g) {
    const int n = g.n, P = g.P, lg = g.lg, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int it = static_cast<int>(t >> (2 * lg));
        const int r = static_cast<int>(t) & ((1 << (2 * lg)) - 1);
        const int i1 = r & (n - 1), i2 = r >> lg;
        const FaceItem F = items[it];
        T *ub = u + F.blk * g.bs;
        T val;
        if (F.kind == FK_BND) {
            const T in = ub[face_off(F.axis, F.side, 1, i1, i2, n, P)];
            val = KIND_K ? in : -in;
        } else if (F.kind == FK_SAME) {
            val = u[F.nbr * g.bs + face_off(F.axis, 1 - F.side, 1, i1, i2, n, P)];
        } else {
            const T *uc = u + F.nbr * g.bs;
            const int yc = F.seg1 * h + (i1 >> 1), zc = F.seg2 * h + (i2 >> 1);
            if (KIND_K) {
                val = uc[face_off(F.axis, 1 - F.side, 1, yc, zc, n, P)];
            } else {
                const int a1 = i1 & 1, a2 = i2 & 1;
                const int cy = yc == 0 ? 1 : (yc == n - 1 ? 2 : 0);
                const int cz = zc == 0 ? 1 : (zc == n - 1 ? 2 : 0);
                T acc = T(0);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T accb = T(0);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const int y = yc + c_base[cy][b], z = zc + c_base[cz][c];
                        T e = w_normal<T>(0) * uc[face_off(F.axis, 1 - F.side, 1, y, z, n, P)];
                        e = fma(w_normal<T>(1), uc[face_off(F.axis, 1 - F.side, 2, y, z, n, P)], e);
                        e = fma(w_normal<T>(2), uc[face_off(F.axis, 1 - F.side, 3, y, z, n, P)], e);
                        accb = fma(w_tang<T>(cy, a1, b), e, accb);
                    }
                    acc = fma(w_tang<T>(cz, a2, c), accb, acc);
                }
                val = acc;
            }
        }
        ub[face_off(F.axis, F.side, 0, i1, i2, n, P)] = val;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Ghost exchange, part 2: coarse ghost segments next to finer neighbours.
// FLUX = false: F2C mean of the 2x2x2 fine inner cells overlapping each coarse ghost cell (Sec. 3.3.1).
// FLUX = true:  conservative coarse ghost G with T_C (u_C - G) = 1/2 sum_j T_j (g_j - u_j) over the four fine
//               sub-faces j, g_j the fine ghosts (C2F, part 1 must have run), u_j the first fine layer.  With the
//               1/h^2-scaled coefficients of MODE 1, T_j / (2 T_C) = T~_j / (8 T~_C) since h_C = 2 h_j.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE, bool FLUX>
static __global__ void k_exchange_segs(T *__restrict__ u, Coef cf, const SegItem *__restrict__ items, int nitems,
                                LevelGeom g) {
    const int n = g.n, P = g.P, lgh = g.lg - 1, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lgh);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int it = static_cast<int>(t >> (2 * lgh));
        const int r = static_cast<int>(t) & ((1 << (2 * lgh)) - 1);
        const int p = r & (h - 1), q = r >> lgh;
        const SegItem S = items[it];
        const int64_t cb = S.coarse * g.bs, fb = S.fine * g.bs;
        const int fs = 1 - S.side;
        const int yc = S.s1 * h + p, zc = S.s2 * h + q;
        T val;
        if (!FLUX) {
            T s = T(0);
#pragma unroll
            for (int d = 1; d <= 2; ++d)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int a = 0; a < 2; ++a) s += u[fb + face_off(S.axis, fs, d, 2 * p + a, 2 * q + b, n, P)];
            val = T(0.125) * s;
        } else {
            const int64_t gC = cb + face_off(S.axis, S.side, 1, yc, zc, n, P);
            const int64_t g0c = cb + face_off(S.axis, S.side, 0, yc, zc, n, P);
            const T uC = u[gC];
            T flux = T(0);
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int64_t g0 = fb + face_off(S.axis, fs, 0, 2 * p + a, 2 * q + b, n, P);
                    const int64_t g1 = fb + face_off(S.axis, fs, 1, 2 * p + a, 2 * q + b, n, P);
                    const T Tj = face_coef<T, MODE>(cf, fs ? g0 : g1, fs ? g1 : g0, S.axis);
                    flux = fma(Tj, u[g0] - u[g1], flux);
                }
            const T Tc = face_coef<T, MODE>(cf, S.side ? g0c : gC, S.side ? gC : g0c, S.axis);
            val = uC - flux / (T(MODE == 1 ? 8 : 2) * Tc);
        }
        u[cb + face_off(S.axis, S.side, 0, yc, zc, n, P)] = val;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep of one colour ((x+y+z) mod 2 of the block-local interior index; red = 0):
//     u_i = (h^2 f_i + sum_f T_f u_f) / sum_f T_f
// over every block of the level, ghosts as left by the last exchange.  One thread per updated cell.
// h2 is h^2 per block in the field's precision (unused in MODE 1, whose coefficients carry 1/h^2).
// ------------------------------------------------------------------------------------------------------------
// nbr6 (optional): per block face (b * 6 + 2 * axis + side) the same-level neighbour block, -1 on the domain
// boundary, -2 on a refinement interface.  When given, every updated cell on a block face also writes its new value
// into the neighbour's ghost cell that mirrors it (or the reflected -u into its own boundary ghost), so same-level and
// boundary ghosts stay current without an exchange launch; interface ghosts are left to the exchange kernels.  The
// ghost cells written have the colour being updated, which no cell of this half-sweep reads (its neighbours all
// have the other colour), so the writes cannot race with the reads.
template <typename T, int MODE>
static __global__ void k_smooth(T *__restrict__ u, const T *__restrict__ f, Coef cf, const T *__restrict__ h2,
                                LevelGeom g, int colour, const int32_t *__restrict__ nbr6) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg - 1);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int m = static_cast<int>(t & ((n >> 1) - 1));
        const int y = static_cast<int>((t >> (lg - 1)) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg - 1)) & (n - 1));
        const int64_t b = t >> (3 * lg - 1);
        const int x = 2 * m + ((y + z + colour) & 1);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        T val;
        if constexpr (MODE == 1) {
            val = sten1(u, cf, gi, P, f[gi]) * cf.dinv[gi];
        } else if constexpr (MODE == 0) {
            val = fma(h2[b], f[gi], sten0<T>(u, gi, P)) * T(1.0 / 6.0);
        } else {
            float S, D;
            sten2(reinterpret_cast<const float *>(u), cf.kap, gi, P, S, D);
            val = T(fmaf(float(h2[b]), float(f[gi]), S) * frcp(D));
        }
        u[gi] = val;
        if (nbr6 && (x == 0 || x == n - 1 || y == 0 || y == n - 1 || z == 0 || z == n - 1)) {
            const int c[3] = {x, y, z};
#pragma unroll
            for (int axis = 0; axis < 3; ++axis) {
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (c[axis] != (side ? n - 1 : 0)) continue;
                    const int nb = nbr6[b * 6 + 2 * axis + side];
                    const int i1 = axis == 0 ? y : x, i2 = axis == 2 ? y : z;
                    if (nb >= 0)
                        u[static_cast<int64_t>(nb) * g.bs + face_off(axis, 1 - side, 0, i1, i2, n, P)] = val;
                    else if (nb == -1)
                        u[b * g.bs + face_off(axis, side, 0, i1, i2, n, P)] = -val;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Residual of the fine level restricted to the next level (mean of the 8 children), written as the coarse
// right-hand side; the coarse solution's interior is zeroed (coarse-grid correction starts from 0).
// One thread per coarse cell.  ih2f: 1/h^2 per fine block.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE>
static __global__ void k_residual_restrict(const T *__restrict__ u, const T *__restrict__ f, Coef cf,
                                    const T *__restrict__ ih2f, LevelGeom gf, T *__restrict__ fc,
                                    T *__restrict__ uc, const XferItem *__restrict__ xf, LevelGeom gc) {
    const int lgc = gc.lg, nc = gc.n;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int X = static_cast<int>(t & (nc - 1));
        const int Y = static_cast<int>((t >> lgc) & (nc - 1));
        const int Z = static_cast<int>((t >> (2 * lgc)) & (nc - 1));
        const int64_t B = t >> (3 * lgc);
        const XferItem xi = xf[B];
        const int64_t gcell = B * gc.bs + off3(X + 1, Y + 1, Z + 1, gc.P);
        uc[gcell] = T(0);
        if (xi.kind == XF_COPY) {
            const int64_t b = xi.src[0];
            fc[gcell] = residual_at<T, MODE>(u, f, cf, b * gf.bs + off3(X + 1, Y + 1, Z + 1, gf.P), gf.P, ih2f[b]);
            continue;
        }
        int64_t b;
        int x0, y0, z0;
        if (xi.kind == XF_HALVE) {
            b = xi.src[0];
            x0 = 2 * X;
            y0 = 2 * Y;
            z0 = 2 * Z;
        } else {
            const int hc = nc >> 1;
            const int ox = X >= hc, oy = Y >= hc, oz = Z >= hc;
            b = xi.src[ox + 2 * oy + 4 * oz];
            x0 = 2 * X - ox * nc;
            y0 = 2 * Y - oy * nc;
            z0 = 2 * Z - oz * nc;
        }
        const T ih2 = ih2f[b];
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    s += residual_at<T, MODE>(u, f, cf, b * gf.bs + off3(x0 + a + 1, y0 + bb + 1, z0 + c + 1, gf.P),
                                              gf.P, ih2);
        fc[gcell] = T(0.125) * s;
    }
}

// Restriction of a plain field (mean of the 8 children; copy for carried-over blocks), e.g. the coefficient k.
template <typename T>
static __global__ void k_restrict_field(const T *__restrict__ xf_in, LevelGeom gf, T *__restrict__ xc,
                                 const XferItem *__restrict__ xf, LevelGeom gc) {
    const int lgc = gc.lg, nc = gc.n;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int X = static_cast<int>(t & (nc - 1));
        const int Y = static_cast<int>((t >> lgc) & (nc - 1));
        const int Z = static_cast<int>((t >> (2 * lgc)) & (nc - 1));
        const int64_t B = t >> (3 * lgc);
        const XferItem xi = xf[B];
        const int64_t gcell = B * gc.bs + off3(X + 1, Y + 1, Z + 1, gc.P);
        if (xi.kind == XF_COPY) {
            xc[gcell] = xf_in[xi.src[0] * gf.bs + off3(X + 1, Y + 1, Z + 1, gf.P)];
            continue;
        }
        int64_t b;
        int x0, y0, z0;
        if (xi.kind == XF_HALVE) {
            b = xi.src[0];
            x0 = 2 * X;
            y0 = 2 * Y;
            z0 = 2 * Z;
        } else {
            const int hc = nc >> 1;
            const int ox = X >= hc, oy = Y >= hc, oz = Z >= hc;
            b = xi.src[ox + 2 * oy + 4 * oz];
            x0 = 2 * X - ox * nc;
            y0 = 2 * Y - oy * nc;
            z0 = 2 * Z - oz * nc;
        }
        T s = T(0);
        for (int c = 0; c < 2; ++c)
            for (int bb = 0; bb < 2; ++bb)
                for (int a = 0; a < 2; ++a) s += xf_in[b * gf.bs + off3(x0 + a + 1, y0 + bb + 1, z0 + c + 1, gf.P)];
        xc[gcell] = T(0.125) * s;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Prolongation + correction: u_f += 1/4 (e_C + e_{C+sx} + e_{C+sy} + e_{C+sz}), s_d pointing to the child's side
// along axis d (face-neighbour linear interpolation, exact for linear functions; coarse ghosts exchanged).
// One thread per coarse cell, writing its 8 children.
// ------------------------------------------------------------------------------------------------------------
template <typename T>
static __global__ void k_prolong(T *__restrict__ uf, LevelGeom gf, const T *__restrict__ ec,
                          const XferItem *__restrict__ xf, LevelGeom gc) {
    const int lgc = gc.lg, nc = gc.n, Pc = gc.P;
    const int64_t PPc = static_cast<int64_t>(Pc) * Pc;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int X = static_cast<int>(t & (nc - 1));
        const int Y = static_cast<int>((t >> lgc) & (nc - 1));
        const int Z = static_cast<int>((t >> (2 * lgc)) & (nc - 1));
        const int64_t B = t >> (3 * lgc);
        const XferItem xi = xf[B];
        const int64_t gcell = B * gc.bs + off3(X + 1, Y + 1, Z + 1, Pc);
        const T e0 = ec[gcell];
        if (xi.kind == XF_COPY) {
            uf[xi.src[0] * gf.bs + off3(X + 1, Y + 1, Z + 1, gf.P)] += e0;
            continue;
        }
        const T ex[2] = {ec[gcell - 1], ec[gcell + 1]};
        const T ey[2] = {ec[gcell - Pc], ec[gcell + Pc]};
        const T ez[2] = {ec[gcell - PPc], ec[gcell + PPc]};
        int64_t b;
        int x0, y0, z0;
        if (xi.kind == XF_HALVE) {
            b = xi.src[0];
            x0 = 2 * X;
            y0 = 2 * Y;
            z0 = 2 * Z;
        } else {
            const int hc = nc >> 1;
            const int ox = X >= hc, oy = Y >= hc, oz = Z >= hc;
            b = xi.src[ox + 2 * oy + 4 * oz];
            x0 = 2 * X - ox * nc;
            y0 = 2 * Y - oy * nc;
            z0 = 2 * Z - oz * nc;
        }
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int64_t gfc = b * gf.bs + off3(x0 + a + 1, y0 + bb + 1, z0 + c + 1, gf.P);
                    uf[gfc] += T(0.25) * ((e0 + ex[a]) + (ey[bb] + ez[c]));
                }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Coarsest level: u = A_c^{-1} f with the dense FP64 inverse of every problem (block-diagonal: the unknowns of
// problem p are cmap[ustart[p] .. ustart[p+1]), its inverse is the row-major N_p x N_p matrix at Ainv + moff[p]).
// One warp per unknown; f gathered from the padded pool through cmap.
// ------------------------------------------------------------------------------------------------------------
template <typename T>
static __global__ void k_coarse_solve(T *__restrict__ u, const T *__restrict__ f, const double *__restrict__ Ainv,
                                      const int64_t *__restrict__ cmap, const int32_t *__restrict__ uprob,
                                      const int64_t *__restrict__ ustart, const int64_t *__restrict__ moff, int N) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int p = uprob[warp];
    const int64_t base = ustart[p];
    const int Np = static_cast<int>(ustart[p + 1] - base);
    const double *row = Ainv + moff[p] + static_cast<int64_t>(warp - base) * Np;
    double s = 0.0;
    for (int j = lane; j < Np; j += 32) s = fma(row[j], static_cast<double>(f[cmap[base + j]]), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) u[cmap[warp]] = T(s);
}

// ------------------------------------------------------------------------------------------------------------
// FP64 residual over the finest level, r = f - A u, written as FP32 r * scale_p (scale_p a power of two per
// problem, so the scaling is exact), with the FP32 correction field zeroed, and per-block sums of h^3 (r scale_p)^2.
// Grid: nb * cpb CTAs, CTA (b, c) covers the c-th of cpb contiguous chunks of block b, so each CTA adds one value
// to its block's sum.  The squared norm is accumulated in FP32 per thread (it decides convergence and is reported
// to ~1e-6 relative) and in FP64 across threads.  out / zero_out may be null.
// ------------------------------------------------------------------------------------------------------------
template <int MODE>
static __global__ void k_residual_norm(const double *__restrict__ u, const double *__restrict__ f, Coef cf,
                                       const double *__restrict__ ih2, const float *__restrict__ vol, LevelGeom g,
                                       int cpb, float *__restrict__ out, const float *__restrict__ pscale,
                                       const int32_t *__restrict__ bprob, double *__restrict__ bsum,
                                       float *__restrict__ zero_out) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t b = blockIdx.x / cpb;
    const int chunk = blockIdx.x - static_cast<int>(b * cpb);
    const int per = (1 << (3 * lg)) / cpb;
    const float scale = pscale[bprob[b]];
    const double ihb = MODE == 1 ? 0.0 : ih2[b];
    float acc = 0.0f;
    for (int c = chunk * per + threadIdx.x; c < (chunk + 1) * per; c += blockDim.x) {
        const int x = c & (n - 1), y = (c >> lg) & (n - 1), z = c >> (2 * lg);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        const double r = residual_at<double, MODE>(u, f, cf, gi, P, ihb);
        const float rs = static_cast<float>(r) * scale;
        if (out) out[gi] = rs;
        if (zero_out) zero_out[gi] = 0.0f;
        acc = fmaf(rs, rs, acc);
    }
    __shared__ double sm[kThreads / 32];
    double a = static_cast<double>(acc) * vol[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sm[w];
        atomicAdd(&bsum[b], s);
    }
}

// Per-block sums of h^3 x^2 over the interior of an FP64 field (same grid shape as k_residual_norm).
static __global__ void k_block_norm64(const double *__restrict__ x, const double *__restrict__ vol, LevelGeom g,
                                      int cpb, double *__restrict__ bsum) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t b = blockIdx.x / cpb;
    const int chunk = blockIdx.x - static_cast<int>(b * cpb);
    const int per = (1 << (3 * lg)) / cpb;
    double acc = 0.0;
    for (int c = chunk * per + threadIdx.x; c < (chunk + 1) * per; c += blockDim.x) {
        const int xx = c & (n - 1), y = (c >> lg) & (n - 1), z = c >> (2 * lg);
        const double v = x[b * g.bs + off3(xx + 1, y + 1, z + 1, P)];
        acc = fma(v, v, acc);
    }
    __shared__ double sm[kThreads / 32];
    acc *= vol[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sm[w];
        atomicAdd(&bsum[b], s);
    }
}

// Per-problem sums of the per-block sums, blocks of problem p listed in pblk[pstart[p] .. pstart[p+1]).
static __global__ void k_problem_sums(const double *__restrict__ bsum, const int32_t *__restrict__ pstart,
                                      const int32_t *__restrict__ pblk, int np, double *__restrict__ psum) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    double s = 0.0;
    for (int i = pstart[p]; i < pstart[p + 1]; ++i) s += bsum[pblk[i]];
    psum[p] = s;
}

// A u over a whole level in FP64 (operator application; ghosts already exchanged).
template <int MODE>
static __global__ void k_apply64(const double *__restrict__ u, Coef cf, const double *__restrict__ ih2, LevelGeom g,
                          double *__restrict__ out) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        out[gi] = apply_at<MODE>(u, cf, gi, P, MODE == 1 ? 0.0 : ih2[b]);
    }
}

// Per-CTA partial sums of h^3 x^2 over the interior of a padded FP64 field (vol = h^3 per block, FP64).
static __global__ void k_norm64(const double *__restrict__ x, const double *__restrict__ vol, LevelGeom g,
                         double *__restrict__ partial) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    double acc = 0.0;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int xx = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const double v = x[b * g.bs + off3(xx + 1, y + 1, z + 1, P)];
        acc = fma(vol[b] * v, v, acc);
    }
    __shared__ double sm[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sm[w];
        partial[blockIdx.x] = s;
    }
}

// Deterministic sum of the per-CTA partials (fixed order for a fixed grid).
static __global__ void k_sum_partials(const double *__restrict__ partial, int nparts, double *__restrict__ out) {
    __shared__ double sa[kThreads];
    double a = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += partial[i];
    sa[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sa[threadIdx.x] += sa[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sa[0];
}

// ------------------------------------------------------------------------------------------------------------
// Layout moves and small updates.
// ------------------------------------------------------------------------------------------------------------
// user layout (n_leaves, n^3) FP64 <-> padded pool of type T (interior only)
// Leaf b of the user array starts at element off[b] (or b * n^3 when off is null).
template <typename T>
static __global__ void k_pack(T *__restrict__ pool, const double *__restrict__ user, LevelGeom g,
                              const int64_t *__restrict__ off = nullptr) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t src = off ? off[b] + (t & ((int64_t(1) << (3 * lg)) - 1)) : t;
        pool[b * g.bs + off3(x + 1, y + 1, z + 1, g.P)] = T(user[src]);
    }
}

template <typename T>
static __global__ void k_unpack(double *__restrict__ user, const T *__restrict__ pool, LevelGeom g,
                                const int64_t *__restrict__ off = nullptr) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t dst = off ? off[b] + (t & ((int64_t(1) << (3 * lg)) - 1)) : t;
        user[dst] = static_cast<double>(pool[b * g.bs + off3(x + 1, y + 1, z + 1, g.P)]);
    }
}

// u64 += e32 / scale_p over the interior (mixed-precision defect correction update; pinv = 1 / scale_p per problem)
static __global__ void k_update_mixed(double *__restrict__ u, const float *__restrict__ e,
                                      const double *__restrict__ pinv, const int32_t *__restrict__ bprob,
                                      LevelGeom g) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, g.P);
        u[gi] = fma(pinv[bprob[b]], static_cast<double>(e[gi]), u[gi]);
    }
}

// Face coefficients of a level from k with ghosts: MODE 1 arrays (harmonic mean times the block's 1/h^2) and
// 1/k for FP32 (MODE 2).  tx at padded (X, Y, Z) is the face between X-1 and X, for X in 1..n+1 and interior
// Y, Z (same for ty, tz).
static __global__ void k_face_coefs(const double *__restrict__ k, const double *__restrict__ ih2, LevelGeom g,
                             double *__restrict__ tx, double *__restrict__ ty, double *__restrict__ tz,
                             float *__restrict__ kap) {
    const int P = g.P, n = g.n;
    const int64_t per = static_cast<int64_t>(P) * P * P;
    const int64_t total = static_cast<int64_t>(g.nb) * per;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = t / per;
        const int r = static_cast<int>(t - b * per);
        const int X = r % P, Y = (r / P) % P, Z = r / (P * P);
        const int64_t gi = b * g.bs + r;
        const double kc = k[gi], s = ih2[b];
        const bool inY = Y >= 1 && Y <= n, inZ = Z >= 1 && Z <= n, inX = X >= 1 && X <= n;
        const auto harm = [](double a, double c) { return 2.0 * a * c / (a + c); };
        if (tx && X >= 1 && inY && inZ) tx[gi] = harm(k[gi - 1], kc) * s;
        if (ty && Y >= 1 && inX && inZ) ty[gi] = harm(k[gi - P], kc) * s;
        if (tz && Z >= 1 && inX && inY) tz[gi] = harm(k[gi - static_cast<int64_t>(P) * P], kc) * s;
        const bool face_or_interior = (inX && inY) || (inX && inZ) || (inY && inZ);
        if (kap && face_or_interior && kc > 0.0) kap[gi] = static_cast<float>(1.0 / kc);
    }
}

// Diagonal (sum of the six scaled face coefficients) and its inverse, interior cells.
static __global__ void k_diag(const double *__restrict__ tx, const double *__restrict__ ty, const double *__restrict__ tz,
                       LevelGeom g, double *__restrict__ dg, double *__restrict__ dinv) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t PP = static_cast<int64_t>(P) * P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        const double D = ((tx[gi] + tx[gi + 1]) + (ty[gi] + ty[gi + P])) + (tz[gi] + tz[gi + PP]);
        dg[gi] = D;
        if (dinv) dinv[gi] = 1.0 / D;
    }
}

}  // namespace octmg

namespace octmg {
// Unit entry m of every problem with more than m coarsest unknowns.
static __global__ void k_set_units(double *__restrict__ u, const int64_t *__restrict__ cmap,
                                   const int64_t *__restrict__ ustart, int np, int m) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < np && ustart[p] + m < ustart[p + 1]) u[cmap[ustart[p] + m]] = 1.0;
}
// Column m of every problem's block: A_p[i, m] = (A e_m)[cmap[ustart[p] + i]].
static __global__ void k_gather_columns(const double *__restrict__ r, const int64_t *__restrict__ cmap,
                                        const int32_t *__restrict__ uprob, const int64_t *__restrict__ ustart,
                                        const int64_t *__restrict__ moff, int N, double *__restrict__ A, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int p = uprob[i];
    const int64_t base = ustart[p];
    const int64_t Np = ustart[p + 1] - base;
    if (m < Np) A[moff[p] + (i - base) * Np + m] = r[cmap[i]];
}
}  // namespace octmg
