// Device kernels of the octree-block multigrid (arXiv 2403.08063), written for sm_103a.
//
// Storage: every block of a level is a padded (n+2)^3 array, x fastest (padded coordinate = interior + 1), one
// ghost layer per face (Sec. 3.3: one layer suffices for the quadratic C2F / linear F2C schemes).  The blocks of
// a level are contiguous with a stride `bs` (elements) rounded up to 256 bytes.
//
// Coefficient modes (template parameter MODE):
//   0  constant coefficient, -Laplace: every face coefficient T_f = 1;
//   1  variable k, face coefficients precomputed in FP64: tx/ty/tz[idx] hold T of the face between padded
//      cells idx - stride and idx along that axis (harmonic mean 2 k_a k_b / (k_a + k_b)), dinv[idx] = 1 / sum_f T_f;
//   2  variable k in FP32: kap[idx] = 1/k with ghosts; T_f = 2 / (kap_i + kap_nb) evaluated with rcp.approx.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "octmg_internal.h"

namespace octmg {

constexpr int kThreads = 256;

struct LevelGeom {
    int32_t nb;     // blocks
    int32_t n;      // interior cells per edge
    int32_t lg;     // log2(n)
    int32_t P;      // n + 2
    int64_t bs;     // block stride in elements
};

struct Coef {       // coefficient arrays of one level (unused members are null)
    const double *tx, *ty, *tz, *dinv;  // MODE 1
    const float *kap;                   // MODE 2
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
__constant__ double c_wn[3] = {45.0 / 32, -18.0 / 32, 5.0 / 32};
__constant__ double c_wt[3][2][3] = {
    {{5.0 / 32, 30.0 / 32, -3.0 / 32}, {-3.0 / 32, 30.0 / 32, 5.0 / 32}},
    {{45.0 / 32, -18.0 / 32, 5.0 / 32}, {21.0 / 32, 14.0 / 32, -3.0 / 32}},
    {{-3.0 / 32, 14.0 / 32, 21.0 / 32}, {5.0 / 32, -18.0 / 32, 45.0 / 32}}};
__constant__ int c_base[3][3] = {{-1, 0, 1}, {0, 1, 2}, {-2, -1, 0}};

__device__ inline float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Face coefficient between padded cells idx and idx + s*stride(axis) (s = -1 or +1) of one block.
template <typename T, int MODE>
__device__ inline T face_T(const Coef &c, int64_t gidx, int axis, int s, int P) {
    if (MODE == 0) return T(1);
    const int st = axis_stride(axis, P);
    if (MODE == 1) {
        const double *t = axis == 0 ? c.tx : (axis == 1 ? c.ty : c.tz);
        return T(t[s > 0 ? gidx + st : gidx]);
    }
    const float a = c.kap[gidx], b = c.kap[gidx + (s > 0 ? st : -st)];
    return T(2.0f * frcp(a + b));
}

// sum_f T_f u_f and sum_f T_f at padded cell gidx.
template <typename T, int MODE>
__device__ inline void stencil(const T *__restrict__ u, const Coef &c, int64_t g, int P, T &S, T &D) {
    const int64_t PP = static_cast<int64_t>(P) * P;
    if (MODE == 0) {
        S = ((u[g - 1] + u[g + 1]) + (u[g - P] + u[g + P])) + (u[g - PP] + u[g + PP]);
        D = T(6);
    } else if (MODE == 1) {
        const T a0 = T(c.tx[g]), a1 = T(c.tx[g + 1]), b0 = T(c.ty[g]), b1 = T(c.ty[g + P]);
        const T c0 = T(c.tz[g]), c1 = T(c.tz[g + PP]);
        S = a0 * u[g - 1];
        S = fma(a1, u[g + 1], S);
        S = fma(b0, u[g - P], S);
        S = fma(b1, u[g + P], S);
        S = fma(c0, u[g - PP], S);
        S = fma(c1, u[g + PP], S);
        D = ((a0 + a1) + (b0 + b1)) + (c0 + c1);
    } else {
        const float k0 = c.kap[g];
        const float a0 = frcp(k0 + c.kap[g - 1]), a1 = frcp(k0 + c.kap[g + 1]);
        const float b0 = frcp(k0 + c.kap[g - P]), b1 = frcp(k0 + c.kap[g + P]);
        const float c0 = frcp(k0 + c.kap[g - PP]), c1 = frcp(k0 + c.kap[g + PP]);
        float s = a0 * float(u[g - 1]);
        s = fmaf(a1, float(u[g + 1]), s);
        s = fmaf(b0, float(u[g - P]), s);
        s = fmaf(b1, float(u[g + P]), s);
        s = fmaf(c0, float(u[g - PP]), s);
        s = fmaf(c1, float(u[g + PP]), s);
        S = T(2.0f * s);
        D = T(2.0f * (((a0 + a1) + (b0 + b1)) + (c0 + c1)));
    }
}

// ------------------------------------------------------------------------------------------------------------
// Ghost exchange, part 1: whole faces filled from one source block (boundary, same level, C2F).
// KIND_K = false: solution-type field (Dirichlet reflection ghost = -u_i; quadratic C2F extrapolation).
// KIND_K = true:  coefficient field k (ghost = k_i at the boundary; fine ghosts inject the covering coarse k).
// ------------------------------------------------------------------------------------------------------------
template <typename T, bool KIND_K>
__global__ void k_exchange_faces(T *__restrict__ u, const FaceItem *__restrict__ items, int nitems, LevelGeom g) {
    const int n = g.n, P = g.P, nn = n * n, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) * nn;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int it = static_cast<int>(t / nn);
        const int r = static_cast<int>(t - static_cast<int64_t>(it) * nn);
        const int i1 = r % n, i2 = r / n;
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
                        T e = T(c_wn[0]) * uc[face_off(F.axis, 1 - F.side, 1, y, z, n, P)];
                        e = fma(T(c_wn[1]), uc[face_off(F.axis, 1 - F.side, 2, y, z, n, P)], e);
                        e = fma(T(c_wn[2]), uc[face_off(F.axis, 1 - F.side, 3, y, z, n, P)], e);
                        accb = fma(T(c_wt[cy][a1][b]), e, accb);
                    }
                    acc = fma(T(c_wt[cz][a2][c]), accb, acc);
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
//               sub-faces j, g_j the fine ghosts (C2F, part 1 must have run), u_j the first fine layer.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE, bool FLUX>
__global__ void k_exchange_segs(T *__restrict__ u, Coef cf, const SegItem *__restrict__ items, int nitems,
                                LevelGeom g) {
    const int n = g.n, P = g.P, h = n >> 1, hh = h * h;
    const int64_t total = static_cast<int64_t>(nitems) * hh;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int it = static_cast<int>(t / hh);
        const int r = static_cast<int>(t - static_cast<int64_t>(it) * hh);
        const int p = r % h, q = r / h;
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
            // The face coefficient between depth 0 and depth 1 of a face sits at depth 1 (minus face) or at the
            // ghost (plus face), i.e. at the cell with the larger padded coordinate.
            const int64_t gC = cb + face_off(S.axis, S.side, 1, yc, zc, n, P);
            const T uC = u[gC];
            T flux = T(0);
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int64_t g0 = fb + face_off(S.axis, fs, 0, 2 * p + a, 2 * q + b, n, P);
                    const int64_t g1 = fb + face_off(S.axis, fs, 1, 2 * p + a, 2 * q + b, n, P);
                    const T Tj = face_T<T, MODE>(cf, fs ? g0 : g1, S.axis, -1, P);
                    flux = fma(Tj, u[g0] - u[g1], flux);
                }
            const int64_t g0c = cb + face_off(S.axis, S.side, 0, yc, zc, n, P);
            const T Tc = face_T<T, MODE>(cf, S.side ? g0c : gC, S.axis, -1, P);
            val = uC - flux / (T(2) * Tc);
        }
        u[cb + face_off(S.axis, S.side, 0, yc, zc, n, P)] = val;
    }
}

// ------------------------------------------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep of one colour ((x+y+z) mod 2 of the block-local interior index; red = 0):
//     u_i = (h^2 f_i + sum_f T_f u_f) / sum_f T_f
// over every block of the level, ghosts as left by the last exchange.  One thread per updated cell.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void k_smooth(T *__restrict__ u, const T *__restrict__ f, Coef cf, const double *__restrict__ h2,
                         LevelGeom g, int colour) {
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
        T S, D;
        stencil<T, MODE>(u, cf, gi, P, S, D);
        const T rhs = fma(T(h2[b]), f[gi], S);
        if (MODE == 1)
            u[gi] = rhs * T(cf.dinv[gi]);
        else if (MODE == 0)
            u[gi] = rhs * T(1.0 / 6.0);
        else
            u[gi] = T(float(rhs) * frcp(float(D)));
    }
}

// Point-form residual r = f - (D u - S) / h^2 at padded cell gi of block b.
template <typename T, int MODE>
__device__ inline T residual_at(const T *__restrict__ u, const T *__restrict__ f, const Coef &cf, int64_t gi,
                                int P, T inv_h2) {
    T S, D;
    stencil<T, MODE>(u, cf, gi, P, S, D);
    return (f ? f[gi] : T(0)) - (D * u[gi] - S) * inv_h2;
}

// ------------------------------------------------------------------------------------------------------------
// Residual of the fine level restricted to the next level (mean of the 8 children), written as the coarse
// right-hand side; the coarse solution's interior is zeroed (coarse-grid correction starts from 0).
// One thread per coarse cell.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void k_residual_restrict(const T *__restrict__ u, const T *__restrict__ f, Coef cf,
                                    const double *__restrict__ h2f, LevelGeom gf, T *__restrict__ fc,
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
            fc[gcell] = residual_at<T, MODE>(u, f, cf, b * gf.bs + off3(X + 1, Y + 1, Z + 1, gf.P), gf.P,
                                             T(1.0 / h2f[b]));
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
        const T ih2 = T(1.0 / h2f[b]);
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
__global__ void k_restrict_field(const T *__restrict__ xf_in, LevelGeom gf, T *__restrict__ xc,
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
__global__ void k_prolong(T *__restrict__ uf, LevelGeom gf, const T *__restrict__ ec,
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
// Coarsest level: u = A_c^{-1} f with the dense FP64 inverse (one warp per unknown; f gathered from the padded
// pool through cmap, the padded offset of every unknown).
// ------------------------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_coarse_solve(T *__restrict__ u, const T *__restrict__ f, const double *__restrict__ Ainv,
                               const int64_t *__restrict__ cmap, int N) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const double *row = Ainv + static_cast<int64_t>(warp) * N;
    double s = 0.0;
    for (int j = lane; j < N; j += 32) s = fma(row[j], static_cast<double>(f[cmap[j]]), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) u[cmap[warp]] = T(s);
}

// ------------------------------------------------------------------------------------------------------------
// Residual over a whole level into an interior-shaped output, optionally scaled and cast, plus per-CTA partial
// sums of h^3 r^2 (volume-weighted squared norm) and of h^3 f^2.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE, typename TO>
__global__ void k_residual_full(const T *__restrict__ u, const T *__restrict__ f, Coef cf,
                                const double *__restrict__ h2, LevelGeom g, TO *__restrict__ out, double scale,
                                double *__restrict__ partial, TO *__restrict__ zero_out) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    double acc_r = 0.0, acc_f = 0.0;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        const double hb2 = h2[b];
        const T r = residual_at<T, MODE>(u, f, cf, gi, P, T(1.0 / hb2));
        if (out) out[gi] = TO(static_cast<double>(r) * scale);
        if (zero_out) zero_out[gi] = TO(0);
        const double vol = hb2 * sqrt(hb2);
        const double fv = f ? double(f[gi]) : 0.0;
        acc_r = fma(vol * double(r), double(r), acc_r);
        acc_f = fma(vol * fv, fv, acc_f);
    }
    if (!partial) return;
    __shared__ double sr[kThreads / 32], sf[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc_r += __shfl_xor_sync(0xffffffffu, acc_r, o);
        acc_f += __shfl_xor_sync(0xffffffffu, acc_f, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sr[threadIdx.x >> 5] = acc_r;
        sf[threadIdx.x >> 5] = acc_f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            a += sr[w];
            b += sf[w];
        }
        partial[2 * blockIdx.x] = a;
        partial[2 * blockIdx.x + 1] = b;
    }
}

__global__ void k_sum_partials(const double *__restrict__ partial, int nparts, double *__restrict__ out) {
    __shared__ double sa[kThreads], sb[kThreads];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sa[threadIdx.x] += sa[threadIdx.x + s];
            sb[threadIdx.x] += sb[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sa[0];
        out[1] = sb[0];
    }
}

// ------------------------------------------------------------------------------------------------------------
// Layout moves and small updates.
// ------------------------------------------------------------------------------------------------------------
// user layout (n_leaves, n^3) FP64 <-> padded pool of type T (interior only)
template <typename T>
__global__ void k_pack(T *__restrict__ pool, const double *__restrict__ user, LevelGeom g) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        pool[b * g.bs + off3(x + 1, y + 1, z + 1, g.P)] = T(user[t]);
    }
}

template <typename T>
__global__ void k_unpack(double *__restrict__ user, const T *__restrict__ pool, LevelGeom g) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        user[t] = static_cast<double>(pool[b * g.bs + off3(x + 1, y + 1, z + 1, g.P)]);
    }
}

// u64 += s * e32 over the interior (mixed-precision defect correction update)
__global__ void k_update_mixed(double *__restrict__ u, const float *__restrict__ e, double s, LevelGeom g) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, g.P);
        u[gi] = fma(s, static_cast<double>(e[gi]), u[gi]);
    }
}

// Face coefficients of a level from k with ghosts (MODE 1 arrays) and 1/k for FP32 (MODE 2).
// tx at padded (X, Y, Z) = harmonic mean of k at X-1 and X, for X in 1..n+1 and interior Y, Z (same for ty, tz).
__global__ void k_face_coefs(const double *__restrict__ k, LevelGeom g, double *__restrict__ tx,
                             double *__restrict__ ty, double *__restrict__ tz, float *__restrict__ kap) {
    const int P = g.P, n = g.n;
    const int64_t per = static_cast<int64_t>(P) * P * P;
    const int64_t total = static_cast<int64_t>(g.nb) * per;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = t / per;
        const int r = static_cast<int>(t - b * per);
        const int X = r % P, Y = (r / P) % P, Z = r / (P * P);
        const int64_t gi = b * g.bs + r;
        const double kc = k[gi];
        const bool inY = Y >= 1 && Y <= n, inZ = Z >= 1 && Z <= n, inX = X >= 1 && X <= n;
        const auto harm = [](double a, double c) { return 2.0 * a * c / (a + c); };
        if (X >= 1 && inY && inZ) tx[gi] = harm(k[gi - 1], kc);
        if (Y >= 1 && inX && inZ) ty[gi] = harm(k[gi - P], kc);
        if (Z >= 1 && inX && inY) tz[gi] = harm(k[gi - static_cast<int64_t>(P) * P], kc);
        const bool face_or_interior = (inX && inY) || (inX && inZ) || (inY && inZ);
        if (kap && face_or_interior && kc > 0.0) kap[gi] = static_cast<float>(1.0 / kc);
    }
}

__global__ void k_diag_inv(const double *__restrict__ tx, const double *__restrict__ ty,
                           const double *__restrict__ tz, LevelGeom g, double *__restrict__ dinv) {
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
        dinv[gi] = 1.0 / D;
    }
}

}  // namespace octmg

namespace octmg {
__global__ void k_set_unit(double *__restrict__ u, const int64_t *__restrict__ cmap, int m) {
    if (threadIdx.x == 0 && blockIdx.x == 0) u[cmap[m]] = 1.0;
}
// A[i, m] = -r[cmap[i]]: column m of the operator from the residual of a unit vector with f = 0
__global__ void k_gather_column(const double *__restrict__ r, const int64_t *__restrict__ cmap, int N,
                                double *__restrict__ A, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) A[static_cast<int64_t>(i) * N + m] = -r[cmap[i]];
}
}  // namespace octmg
