// Adjoint of the octree-block multigrid solve (FP64): the transposed operator, the exact transpose of the forward
// V-cycle, the adjoint solve by defect correction, and dL/dk.  The paper has no adjoint; every step here is the
// transpose of a forward step that cites its passage.
//
// A = S E: E fills ghosts from interiors (reflection, copy, C2F extrapolation of Sec. 3.3.2, F2C mean of Sec. 3.3.1
// or the conservative flux ghost), S is the 7-point stencil.  A^T = E^T S^T: S^T y is the stencil applied to y with
// zero ghosts plus, at every ghost next to an interior cell i, the ghost adjoint -T_f y_i / h_i^2; E^T adds every
// ghost adjoint into the interior cells that ghost was computed from (FP64 atomics), in the reverse order of the
// forward exchange.  The forward V-cycle is a linear map M of its right-hand side; its transpose M^T runs the cycle's
// steps backwards, each transposed, so lambda += M^T (g - A^T lambda) converges at the forward cycle's rate.
#include <cmath>

#include "forest_state.h"

namespace octmg {
namespace {

__device__ inline void decode_cell(int64_t t, int lg, int &x, int &y, int &z, int64_t &b) {
    const int n = 1 << lg;
    x = static_cast<int>(t & (n - 1));
    y = static_cast<int>((t >> lg) & (n - 1));
    z = static_cast<int>((t >> (2 * lg)) & (n - 1));
    b = t >> (3 * lg);
}

#define GRID_STRIDE(total) \
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < (total); \
         t += static_cast<int64_t>(gridDim.x) * blockDim.x)

// The operator's coefficients as the transposed cycle reads them, in its working precision T (natural layout):
// scaled face coefficients T_f / h^2 (x-, y-, z-faces, stored at the cell with the larger coordinate), their sum
// (the diagonal) and its inverse.  FP64: the forest's arrays; FP32: rounded copies made by the first adjoint call.
template <typename T>
struct ACoef {
    const T *tx, *ty, *tz, *dg, *dinv;
};

// Scaled face coefficient T_f / h^2 between depth 0 and depth 1 of face (axis, side) at those two cells.
template <int MODE, typename T>
__device__ inline T face_ts(const ACoef<T> &cf, const T *ih2, int64_t b, int64_t g0, int64_t g1, int axis, int side) {
    if (MODE == 0) return ih2[b];
    const T *t = axis == 0 ? cf.tx : (axis == 1 ? cf.ty : cf.tz);
    return t[side ? g0 : g1];
}

// Ghost adjoints of the transposed stencil: G[ghost] = -T~ y[adjacent interior], every face of every block.
template <int MODE, typename T>
__global__ void k_at_ghosts(const T *__restrict__ y, T *__restrict__ G, ACoef<T> cf, const T *__restrict__ ih2,
                            LevelGeom g) {
    const int n = g.n, lg = g.lg, P = g.P;
    const int64_t total = static_cast<int64_t>(g.nb) * 6 << (2 * lg);
    GRID_STRIDE(total) {
        const int cell = static_cast<int>(t & ((1 << (2 * lg)) - 1));
        const int64_t rest = t >> (2 * lg);
        const int f = static_cast<int>(rest % 6);
        const int64_t b = rest / 6;
        const int axis = f >> 1, side = f & 1;
        const int i1 = cell & (n - 1), i2 = cell >> lg;
        const int64_t g0 = b * g.bs + face_off(axis, side, 0, i1, i2, n, P);
        const int64_t g1 = b * g.bs + face_off(axis, side, 1, i1, i2, n, P);
        G[g0] = -face_ts<MODE>(cf, ih2, b, g0, g1, axis, side) * y[g1];
    }
}

// E^T of the conservative coarse ghosts G = u_C - c sum_j (g_j - u_j), c = T_j / (2 T_C) (T~_j / (8 T~_C) scaled).
template <int MODE, typename T>
__global__ void k_et_segs_flux(T *__restrict__ G, ACoef<T> cf, const T *__restrict__ ih2,
                               const SegItem *__restrict__ items, int nitems, LevelGeom g) {
    const int n = g.n, P = g.P, lgh = g.lg - 1, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lgh);
    GRID_STRIDE(total) {
        const int it = static_cast<int>(t >> (2 * lgh));
        const int r = static_cast<int>(t) & ((1 << (2 * lgh)) - 1);
        const int p = r & (h - 1), q = r >> lgh;
        const SegItem S = items[it];
        const int64_t cb = S.coarse * g.bs, fb = S.fine * g.bs;
        const int fs = 1 - S.side;
        const int yc = S.s1 * h + p, zc = S.s2 * h + q;
        const int64_t g0c = cb + face_off(S.axis, S.side, 0, yc, zc, n, P);
        const int64_t gC = cb + face_off(S.axis, S.side, 1, yc, zc, n, P);
        const T a = G[g0c];
        atomicAdd(&G[gC], a);
        const T Tc = face_ts<MODE>(cf, ih2, S.coarse, g0c, gC, S.axis, S.side);
        const T fac = MODE == 1 ? T(8) : T(2);
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                const int64_t g0 = fb + face_off(S.axis, fs, 0, 2 * p + aa, 2 * q + bb, n, P);
                const int64_t g1 = fb + face_off(S.axis, fs, 1, 2 * p + aa, 2 * q + bb, n, P);
                const T Tj = MODE == 0 ? T(1) : face_ts<MODE>(cf, ih2, S.fine, g0, g1, S.axis, fs);
                const T c = (MODE == 0 ? T(1) : Tj) / (fac * (MODE == 0 ? T(1) : Tc)) * a;
                atomicAdd(&G[g0], -c);
                atomicAdd(&G[g1], c);
            }
    }
}

// E^T of whole faces: reflection (ghost = -u_i), copy from the neighbour, quadratic C2F (27 coarse cells).
template <typename T>
__global__ void k_et_faces(T *__restrict__ G, const FaceItem *__restrict__ items, int nitems, LevelGeom g) {
    const int n = g.n, P = g.P, lg = g.lg, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lg);
    GRID_STRIDE(total) {
        const int it = static_cast<int>(t >> (2 * lg));
        const int r = static_cast<int>(t) & ((1 << (2 * lg)) - 1);
        const int i1 = r & (n - 1), i2 = r >> lg;
        const FaceItem F = items[it];
        const int64_t base = F.blk * g.bs;
        const T a = G[base + face_off(F.axis, F.side, 0, i1, i2, n, P)];
        if (F.kind == FK_BND) {
            atomicAdd(&G[base + face_off(F.axis, F.side, 1, i1, i2, n, P)], -a);
        } else if (F.kind == FK_SAME) {
            atomicAdd(&G[F.nbr * g.bs + face_off(F.axis, 1 - F.side, 1, i1, i2, n, P)], a);
        } else {
            const int64_t cbase = F.nbr * g.bs;
            const int yc = F.seg1 * h + (i1 >> 1), zc = F.seg2 * h + (i2 >> 1);
            const int a1 = i1 & 1, a2 = i2 & 1;
            const int cy = yc == 0 ? 1 : (yc == n - 1 ? 2 : 0);
            const int cz = zc == 0 ? 1 : (zc == n - 1 ? 2 : 0);
            for (int c = 0; c < 3; ++c)
                for (int bb = 0; bb < 3; ++bb) {
                    const T wt = w_tang<T>(0, cz, a2, c) * w_tang<T>(0, cy, a1, bb) * a;
                    const int y = yc + c_base[cy][bb], z = zc + c_base[cz][c];
                    for (int d = 0; d < 3; ++d)
                        atomicAdd(&G[cbase + face_off(F.axis, 1 - F.side, 1 + d, y, z, n, P)], w_normal<T>(0, d) * wt);
                }
        }
    }
}

// E^T of the F2C mean: each of the 8 fine cells receives 1/8 of the coarse ghost adjoint.
template <typename T>
__global__ void k_et_segs_mean(T *__restrict__ G, const SegItem *__restrict__ items, int nitems, LevelGeom g) {
    const int n = g.n, P = g.P, lgh = g.lg - 1, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lgh);
    GRID_STRIDE(total) {
        const int it = static_cast<int>(t >> (2 * lgh));
        const int r = static_cast<int>(t) & ((1 << (2 * lgh)) - 1);
        const int p = r & (h - 1), q = r >> lgh;
        const SegItem S = items[it];
        const int fs = 1 - S.side;
        const T a = T(0.125) * G[S.coarse * g.bs + face_off(S.axis, S.side, 0, S.s1 * h + p, S.s2 * h + q, n, P)];
        for (int d = 1; d <= 2; ++d)
            for (int bb = 0; bb < 2; ++bb)
                for (int aa = 0; aa < 2; ++aa)
                    atomicAdd(&G[S.fine * g.bs + face_off(S.axis, fs, d, 2 * p + aa, 2 * q + bb, n, P)], a);
    }
}

// One transposed smoother step on colour c: z = Pi_c D^-1 ubar (D the diagonal the forward half-sweep divides by),
// fbar += z.  z is written on every interior cell (0 off the colour); its ghosts stay 0.
template <int MODE, typename T>
__global__ void k_adj_colour(const T *__restrict__ ub, T *__restrict__ fb, T *__restrict__ z, ACoef<T> cf,
                             const T *__restrict__ h2, LevelGeom g, int colour) {
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int x, y, zz;
        int64_t b;
        decode_cell(t, g.lg, x, y, zz, b);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, zz + 1, g.P);
        T v = T(0);
        if (((x + y + zz) & 1) == colour) {
            if constexpr (MODE == 1) v = ub[gi] * cf.dinv[gi];
            else if constexpr (sizeof(T) == 8) v = ub[gi] * (h2[b] * (1.0 / 6.0));
            else v = div6(ub[gi] * h2[b]);  // FP32: without the bias of the rounded 1/6
            fb[gi] += v;
        }
        z[gi] = v;
    }
}

// y += a x over the interior.
template <typename T>
__global__ void k_axpy(T *__restrict__ y, const T *__restrict__ x, T a, LevelGeom g) {
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int xx, yy, zz;
        int64_t b;
        decode_cell(t, g.lg, xx, yy, zz, b);
        const int64_t gi = b * g.bs + off3(xx + 1, yy + 1, zz + 1, g.P);
        y[gi] = fma(a, x[gi], y[gi]);
    }
}

// Transposed prolongation: the fine adjoint of u_f += 1/4 (e_C + e_{C+sx} + e_{C+sy} + e_{C+sz}) scattered into the
// coarse padded adjoint (ghost positions included; the transposed coarse exchange follows).
template <typename T>
__global__ void k_prolong_T(const T *__restrict__ ubf, LevelGeom gf, T *__restrict__ Ec,
                            const XferItem *__restrict__ xf, LevelGeom gc) {
    const int lgc = gc.lg, nc = gc.n, Pc = gc.P;
    const int64_t PPc = static_cast<int64_t>(Pc) * Pc;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    GRID_STRIDE(total) {
        int X, Y, Z;
        int64_t B;
        decode_cell(t, lgc, X, Y, Z, B);
        const XferItem xi = xf[B];
        const int64_t gcell = B * gc.bs + off3(X + 1, Y + 1, Z + 1, Pc);
        if (xi.kind == XF_COPY) {
            atomicAdd(&Ec[gcell], ubf[xi.src[0] * gf.bs + off3(X + 1, Y + 1, Z + 1, gf.P)]);
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
        T all = T(0), sx[2] = {T(0), T(0)}, sy[2] = {T(0), T(0)}, sz[2] = {T(0), T(0)};
        for (int c = 0; c < 2; ++c)
            for (int bb = 0; bb < 2; ++bb)
                for (int a = 0; a < 2; ++a) {
                    const T v = T(0.25) * ubf[b * gf.bs + off3(x0 + a + 1, y0 + bb + 1, z0 + c + 1, gf.P)];
                    all += v;
                    sx[a] += v;
                    sy[bb] += v;
                    sz[c] += v;
                }
        atomicAdd(&Ec[gcell], all);
        atomicAdd(&Ec[gcell - 1], sx[0]);
        atomicAdd(&Ec[gcell + 1], sx[1]);
        atomicAdd(&Ec[gcell - Pc], sy[0]);
        atomicAdd(&Ec[gcell + Pc], sy[1]);
        atomicAdd(&Ec[gcell - PPc], sz[0]);
        atomicAdd(&Ec[gcell + PPc], sz[1]);
    }
}

// Transposed restriction: every fine cell receives 1/8 of its parent's adjoint (carried-over blocks: all of it).
template <typename T>
__global__ void k_restrict_T(const T *__restrict__ fbc, LevelGeom gc, T *__restrict__ rf,
                             const XferItem *__restrict__ xf, LevelGeom gf) {
    const int lgc = gc.lg, nc = gc.n;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    GRID_STRIDE(total) {
        int X, Y, Z;
        int64_t B;
        decode_cell(t, lgc, X, Y, Z, B);
        const XferItem xi = xf[B];
        const T v = fbc[B * gc.bs + off3(X + 1, Y + 1, Z + 1, gc.P)];
        if (xi.kind == XF_COPY) {
            rf[xi.src[0] * gf.bs + off3(X + 1, Y + 1, Z + 1, gf.P)] = v;
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
        for (int c = 0; c < 2; ++c)
            for (int bb = 0; bb < 2; ++bb)
                for (int a = 0; a < 2; ++a) rf[b * gf.bs + off3(x0 + a + 1, y0 + bb + 1, z0 + c + 1, gf.P)] = T(0.125) * v;
    }
}

// A u in the working precision T on a natural-layout level (ghosts of u filled): the 7-point rows
// (1/h^2) sum_f T_f (u_i - u_f), written as dg u_i - sum_f T~_f u_f with the scaled coefficients (MODE 1) or
// (6 u_i - sum_f u_f) / h^2 (MODE 0).  The FP32 transposed cycle's S^T (the stencil part of A^T y with zero ghosts).
template <typename T, int MODE>
__global__ void k_apply_nat(const T *__restrict__ u, ACoef<T> cf, const T *__restrict__ ih2, LevelGeom g,
                            T *__restrict__ out) {
    const int P = g.P;
    const int64_t PP = static_cast<int64_t>(P) * P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int x, y, z;
        int64_t b;
        decode_cell(t, g.lg, x, y, z, b);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        if constexpr (MODE == 1) {
            T a = cf.tx[gi] * u[gi - 1];
            a = fma(cf.tx[gi + 1], u[gi + 1], a);
            a = fma(cf.ty[gi], u[gi - P], a);
            a = fma(cf.ty[gi + P], u[gi + P], a);
            a = fma(cf.tz[gi], u[gi - PP], a);
            a = fma(cf.tz[gi + PP], u[gi + PP], a);
            out[gi] = fma(cf.dg[gi], u[gi], -a);
        } else {
            const T S = ((u[gi - 1] + u[gi + 1]) + (u[gi - P] + u[gi + P])) + (u[gi - PP] + u[gi + PP]);
            out[gi] = fma(T(6), u[gi], -S) * ih2[b];
        }
    }
}

// FP32 copy of an FP64 array (the coefficient arrays of the FP32 transposed cycle), every element.
__global__ void k_round32(const double *__restrict__ src, float *__restrict__ dst, int64_t count) {
    GRID_STRIDE(count) dst[t] = static_cast<float>(src[t]);
}

// FP32 right-hand side of a transposed correction cycle: r32 = s r over the interior (s a power of two: exact up to
// the rounding to FP32).
__global__ void k_scaled32(const double *__restrict__ r, float *__restrict__ r32, double s, LevelGeom g) {
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int x, y, z;
        int64_t b;
        decode_cell(t, g.lg, x, y, z, b);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, g.P);
        r32[gi] = static_cast<float>(s * r[gi]);
    }
}

// lambda += e32 / s over the interior, in FP64.
__global__ void k_add_from32(double *__restrict__ lam, const float *__restrict__ e32, double inv_s, LevelGeom g) {
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int x, y, z;
        int64_t b;
        decode_cell(t, g.lg, x, y, z, b);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, g.P);
        lam[gi] = fma(static_cast<double>(e32[gi]), inv_s, lam[gi]);
    }
}

// r = g - q over the interior, with per-CTA partials of h^3 r^2.
__global__ void k_sub_norm(const double *__restrict__ gvec, const double *__restrict__ q, double *__restrict__ r,
                           const double *__restrict__ vol, LevelGeom g, double *__restrict__ partial) {
    double acc = 0.0;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int x, y, z;
        int64_t b;
        decode_cell(t, g.lg, x, y, z, b);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, g.P);
        const double v = gvec[gi] - q[gi];
        r[gi] = v;
        acc = fma(vol[b] * v, v, acc);
    }
    __shared__ double sm[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sm[w];
        partial[blockIdx.x] = s;
    }
}

// dL/dk, face terms: for every interior cell i and face f (except coarse sides of refinement interfaces in the
// conservative variant), the row term (1/h^2) T(k_i, k_f) (u_i - u_f) contributes -lambda_i (u_i - u_f) / h^2 times
// dT/dk_i to k_i and times dT/dk_f to the k at the neighbour or ghost position (gadj).  T = 2 a b / (a + b):
// dT/da = 2 b^2 / (a + b)^2.
__global__ void k_gradk_faces(const double *__restrict__ u, const double *__restrict__ lam,
                              const double *__restrict__ k, const double *__restrict__ ih2,
                              const int8_t *__restrict__ fkind, int skip_f2c, LevelGeom g, double *__restrict__ grad,
                              double *__restrict__ gadj) {
    const int n = g.n, P = g.P;
    const int64_t PP = static_cast<int64_t>(P) * P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int x, y, z;
        int64_t b;
        decode_cell(t, g.lg, x, y, z, b);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        const double w0 = -lam[gi] * ih2[b];
        const double ki = k[gi], ui = u[gi];
        const int c[3] = {x, y, z};
        const int64_t st[3] = {1, P, PP};
        double acc = 0.0;
        for (int axis = 0; axis < 3; ++axis)
            for (int side = 0; side < 2; ++side) {
                const bool at_face = side ? (c[axis] == n - 1) : (c[axis] == 0);
                if (at_face && skip_f2c && fkind[b * 6 + 2 * axis + side] == 3) continue;
                const int64_t gn = gi + (side ? st[axis] : -st[axis]);
                const double kg = k[gn];
                const double d = ui - u[gn];
                const double inv = 1.0 / ((ki + kg) * (ki + kg));
                acc += w0 * d * 2.0 * kg * kg * inv;
                atomicAdd(&gadj[gn], w0 * d * 2.0 * ki * ki * inv);
            }
        grad[gi] = acc;
    }
}

// Interior positions of gadj are the neighbours' own k.
__global__ void k_gradk_merge(double *__restrict__ grad, const double *__restrict__ gadj, LevelGeom g) {
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * g.lg);
    GRID_STRIDE(total) {
        int x, y, z;
        int64_t b;
        decode_cell(t, g.lg, x, y, z, b);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, g.P);
        grad[gi] += gadj[gi];
    }
}

// Ghost positions of gadj through the ghost-k maps: k_g = k_i (boundary), neighbour copy, injection of the
// covering coarse k (fine ghosts).
__global__ void k_gradk_ghost_faces(double *__restrict__ grad, const double *__restrict__ gadj,
                                    const FaceItem *__restrict__ items, int nitems, LevelGeom g) {
    const int n = g.n, P = g.P, lg = g.lg, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lg);
    GRID_STRIDE(total) {
        const int it = static_cast<int>(t >> (2 * lg));
        const int r = static_cast<int>(t) & ((1 << (2 * lg)) - 1);
        const int i1 = r & (n - 1), i2 = r >> lg;
        const FaceItem F = items[it];
        const double a = gadj[F.blk * g.bs + face_off(F.axis, F.side, 0, i1, i2, n, P)];
        if (F.kind == FK_BND)
            atomicAdd(&grad[F.blk * g.bs + face_off(F.axis, F.side, 1, i1, i2, n, P)], a);
        else if (F.kind == FK_SAME)
            atomicAdd(&grad[F.nbr * g.bs + face_off(F.axis, 1 - F.side, 1, i1, i2, n, P)], a);
        else
            atomicAdd(&grad[F.nbr * g.bs + face_off(F.axis, 1 - F.side, 1, F.seg1 * h + (i1 >> 1), F.seg2 * h + (i2 >> 1),
                                                     n, P)],
                      a);
    }
}

// Coarse ghost k = mean of the 8 fine k (ghost-only variant): 1/8 of the ghost adjoint to each fine cell.
__global__ void k_gradk_ghost_segs(double *__restrict__ grad, const double *__restrict__ gadj,
                                   const SegItem *__restrict__ items, int nitems, LevelGeom g) {
    const int n = g.n, P = g.P, lgh = g.lg - 1, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lgh);
    GRID_STRIDE(total) {
        const int it = static_cast<int>(t >> (2 * lgh));
        const int r = static_cast<int>(t) & ((1 << (2 * lgh)) - 1);
        const int p = r & (h - 1), q = r >> lgh;
        const SegItem S = items[it];
        const int fs = 1 - S.side;
        const double a =
            0.125 * gadj[S.coarse * g.bs + face_off(S.axis, S.side, 0, S.s1 * h + p, S.s2 * h + q, n, P)];
        for (int d = 1; d <= 2; ++d)
            for (int bb = 0; bb < 2; ++bb)
                for (int aa = 0; aa < 2; ++aa)
                    atomicAdd(&grad[S.fine * g.bs + face_off(S.axis, fs, d, 2 * p + aa, 2 * q + bb, n, P)], a);
    }
}

// Conservative coarse rows: (1/h_C^2) 1/2 sum_j T(k_j, k_C) (g_j - u_j) with weight -lambda_C.
__global__ void k_gradk_flux_rows(double *__restrict__ grad, const double *__restrict__ u,
                                  const double *__restrict__ lam, const double *__restrict__ k,
                                  const double *__restrict__ ih2, const SegItem *__restrict__ items, int nitems,
                                  LevelGeom g) {
    const int n = g.n, P = g.P, lgh = g.lg - 1, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lgh);
    GRID_STRIDE(total) {
        const int it = static_cast<int>(t >> (2 * lgh));
        const int r = static_cast<int>(t) & ((1 << (2 * lgh)) - 1);
        const int p = r & (h - 1), q = r >> lgh;
        const SegItem S = items[it];
        const int fs = 1 - S.side;
        const int64_t gC = S.coarse * g.bs + face_off(S.axis, S.side, 1, S.s1 * h + p, S.s2 * h + q, n, P);
        const double lC = lam[gC] * ih2[S.coarse], kC = k[gC];
        double accC = 0.0;
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                const int64_t g0 = S.fine * g.bs + face_off(S.axis, fs, 0, 2 * p + aa, 2 * q + bb, n, P);
                const int64_t g1 = S.fine * g.bs + face_off(S.axis, fs, 1, 2 * p + aa, 2 * q + bb, n, P);
                const double kj = k[g1];
                const double w = -lC * 0.5 * (u[g0] - u[g1]);
                const double inv = 1.0 / ((kj + kC) * (kj + kC));
                atomicAdd(&grad[g1], w * 2.0 * kC * kC * inv);
                accC += w * 2.0 * kj * kj * inv;
            }
        atomicAdd(&grad[gC], accC);
    }
}

// ---------------------------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------------------------
// The transposed cycle's pools and coefficients in its working precision.
template <typename T>
struct APools {
    T *ub, *fb, *z, *tmp;
};
template <typename T> APools<T> apools(DevLevel &d);
template <> APools<double> apools<double>(DevLevel &d) { return {d.a_ub, d.a_fb, d.a_z, d.a_tmp}; }
template <> APools<float> apools<float>(DevLevel &d) { return {d.a32_ub, d.a32_fb, d.a32_z, d.a32_tmp}; }
template <typename T> ACoef<T> acoef(const DevLevel &d);
template <> ACoef<double> acoef<double>(const DevLevel &d) { return {d.tx, d.ty, d.tz, d.dg, d.dinv}; }
template <> ACoef<float> acoef<float>(const DevLevel &d) {
    return {d.a32_tx, d.a32_ty, d.a32_tz, d.a32_dg, d.a32_dinv};
}
template <typename T> const T *aih2(const DevLevel &d);
template <> const double *aih2<double>(const DevLevel &d) { return d.ih2_64; }
template <> const float *aih2<float>(const DevLevel &d) { return d.ih2_32; }
template <typename T> const T *ah2(const DevLevel &d);
template <> const double *ah2<double>(const DevLevel &d) { return d.h2_64; }
template <> const float *ah2<float>(const DevLevel &d) { return d.h2_32; }

template <int MODE, typename T>
void exchange_T(mg_forest *F, DevLevel &d, T *G) {
    Prof p(F, P_ADJ, 2);
    if (d.nsegs && F->cfg.interface_flux)
        k_et_segs_flux<MODE, T><<<grid_for(static_cast<int64_t>(d.nsegs) << (2 * (d.g.lg - 1))), kThreads, 0, F->st>>>(
            G, acoef<T>(d), aih2<T>(d), d.segs, d.nsegs, d.g);
    if (d.nfaces)
        k_et_faces<T><<<grid_for(static_cast<int64_t>(d.nfaces) << (2 * d.g.lg)), kThreads, 0, F->st>>>(G, d.faces,
                                                                                                        d.nfaces, d.g);
    if (d.nsegs && !F->cfg.interface_flux)
        k_et_segs_mean<T><<<grid_for(static_cast<int64_t>(d.nsegs) << (2 * (d.g.lg - 1))), kThreads, 0, F->st>>>(
            G, d.segs, d.nsegs, d.g);
}

// out = A^T x on level l; x must have zero ghosts; out's ghost positions are left holding ghost adjoints.
template <int MODE, typename T>
void apply_T(mg_forest *F, DevLevel &d, const T *x, T *out) {
    if constexpr (sizeof(T) == 8) {
        apply64(F, d, x, out);
    } else {
        Prof p(F, P_ADJ, 1);
        k_apply_nat<T, MODE><<<grid_for(d.cells()), kThreads, 0, F->st>>>(x, acoef<T>(d), aih2<T>(d), d.g, out);
    }
    {
        Prof p(F, P_ADJ, 1);
        k_at_ghosts<MODE, T><<<grid_for(static_cast<int64_t>(d.g.nb) * 6 << (2 * d.g.lg)), kThreads, 0, F->st>>>(
            x, out, acoef<T>(d), aih2<T>(d), d.g);
    }
    exchange_T<MODE, T>(F, d, out);
}

template <int MODE, typename T>
void smooth_T(mg_forest *F, DevLevel &d, int iters) {
    const APools<T> a = apools<T>(d);
    for (int i = 0; i < iters; ++i)
        for (int colour = 1; colour >= 0; --colour) {
            {
                Prof p(F, P_ADJ, 1);
                k_adj_colour<MODE, T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(a.ub, a.fb, a.z, acoef<T>(d),
                                                                                    ah2<T>(d), d.g, colour);
            }
            apply_T<MODE, T>(F, d, a.z, a.tmp);
            Prof p(F, P_ADJ, 1);
            k_axpy<T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(a.ub, a.tmp, T(-1), d.g);
        }
}

// fbar = M_l^T ubar (level l's pools ub in, fb out), in precision T; the coarsest level's dense inverse is FP64.
template <int MODE, typename T>
void vcycle_T(mg_forest *F, int l) {
    DevLevel &d = F->L[l];
    const APools<T> a = apools<T>(d);
    const int last = static_cast<int>(F->L.size()) - 1;
    if (l == last) {
        Prof p(F, P_ADJ, 1);
        k_coarse_solve<T><<<(F->Nc * 32 + kThreads - 1) / kThreads, kThreads, 0, F->st>>>(
            a.fb, a.ub, F->AinvT, F->cmap, F->uprob, F->ustart, F->moff, F->Nc);
        return;
    }
    cudaMemsetAsync(a.fb, 0, d.pool_elems() * sizeof(T), F->st);
    smooth_T<MODE, T>(F, d, F->cfg.nu2);
    DevLevel &c = F->L[l + 1];
    const APools<T> ac = apools<T>(c);
    cudaMemsetAsync(ac.ub, 0, c.pool_elems() * sizeof(T), F->st);
    {
        Prof p(F, P_ADJ, 1);
        k_prolong_T<T><<<grid_for(c.cells()), kThreads, 0, F->st>>>(a.ub, d.g, ac.ub, d.xfer, c.g);
    }
    exchange_T<MODE, T>(F, c, ac.ub);
    vcycle_T<MODE, T>(F, l + 1);
    {
        Prof p(F, P_ADJ, 2);
        k_restrict_T<T><<<grid_for(c.cells()), kThreads, 0, F->st>>>(ac.fb, c.g, a.z, d.xfer, d.g);
        k_axpy<T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(a.fb, a.z, T(1), d.g);
    }
    apply_T<MODE, T>(F, d, a.z, a.tmp);
    {
        Prof p(F, P_ADJ, 1);
        k_axpy<T><<<grid_for(d.cells()), kThreads, 0, F->st>>>(a.ub, a.tmp, T(-1), d.g);
    }
    smooth_T<MODE, T>(F, d, F->cfg.nu1);
}

mg_status ensure_adjoint_pools(mg_forest *F) {
    MG_TRY(ensure_scratch64(F));
    MG_TRY(ensure_fp64_coefficients(F));
    if (F->a_g) return MG_OK;
    const bool fp32 = F->cfg.precision == 1;
    for (DevLevel &d : F->L) {
        const int64_t bytes = d.pool_elems() * static_cast<int64_t>(sizeof(double));
        void *p;
        MG_TRY(forest_alloc(F, &p, bytes));
        d.a_ub = static_cast<double *>(p);
        MG_TRY(forest_alloc(F, &p, bytes));
        d.a_fb = static_cast<double *>(p);
        MG_TRY(forest_alloc(F, &p, bytes));
        d.a_z = static_cast<double *>(p);
        MG_TRY(forest_alloc(F, &p, bytes));
        d.a_tmp = static_cast<double *>(p);
        if (!fp32) continue;
        // FP32 transposed cycles (forests with FP32 forward cycles): natural-layout FP32 pools and coefficients
        const int64_t b32 = d.pool_elems() * static_cast<int64_t>(sizeof(float));
        float **pools[] = {&d.a32_ub, &d.a32_fb, &d.a32_z, &d.a32_tmp};
        for (float **q : pools) {
            MG_TRY(forest_alloc(F, &p, b32));
            *q = static_cast<float *>(p);
        }
        if (F->cfg.coeff) {
            float **coefs[] = {&d.a32_tx, &d.a32_ty, &d.a32_tz, &d.a32_dg, &d.a32_dinv};
            for (float **q : coefs) {
                MG_TRY(forest_alloc(F, &p, b32));
                *q = static_cast<float *>(p);
            }
        }
    }
    const int64_t bytes0 = F->L[0].pool_elems() * static_cast<int64_t>(sizeof(double));
    void *p;
    MG_TRY(forest_alloc(F, &p, bytes0));
    F->a_lam = static_cast<double *>(p);
    MG_TRY(forest_alloc(F, &p, bytes0));
    F->a_g = static_cast<double *>(p);
    return MG_OK;
}

// The FP32 copies of the FP64 coefficients (rebuilt by every adjoint solve: mg_set_rhs may have changed k).
mg_status round_coefficients32(mg_forest *F) {
    if (!F->cfg.coeff) return MG_OK;
    for (DevLevel &d : F->L) {
        const int64_t cnt = d.pool_elems();
        const double *src[] = {d.tx, d.ty, d.tz, d.dg, d.dinv};
        float *dst[] = {d.a32_tx, d.a32_ty, d.a32_tz, d.a32_dg, d.a32_dinv};
        for (int i = 0; i < 5; ++i) k_round32<<<grid_for(cnt), kThreads, 0, F->st>>>(src[i], dst[i], cnt);
    }
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

mg_status read_sum(mg_forest *F, int grid, double *out) {
    k_sum_partials<<<1, kThreads, 0, F->st>>>(F->partial, grid, F->sums);
    MG_CUDA(cudaMemcpyAsync(F->pinned, F->sums, sizeof(double), cudaMemcpyDeviceToHost, F->st));
    MG_CUDA(cudaStreamSynchronize(F->st));
    *out = F->pinned[0];
    return MG_OK;
}

// The transposed operator and cycle are written for the quadratic coarse-to-fine scheme, red-black Gauss-Seidel, the
// dense coarsest solve and homogeneous boundary data (the k-gradient of a boundary term would need g).
mg_status adjoint_supported(const mg_forest *F) {
    if (F->cfg.c2f_variant != 0 || F->cfg.smoother != 0 || F->cfg.coarse_iters != 0 || F->cfg.prolongation != 0) {
        set_error("the adjoint needs c2f_variant 0, the Gauss-Seidel smoother, the dense coarsest solve and the "
                  "face-neighbour linear prolongation");
        return MG_ERR_INVALID_ARG;
    }
    if (F->gb) {
        set_error("the adjoint needs homogeneous boundary data (mg_set_boundary(forest, NULL))");
        return MG_ERR_STATE;
    }
    return MG_OK;
}

template <int MODE>
mg_status adjoint_solve(mg_forest *F, const double *u_dev, const double *dLdu_dev, double *lambda_dev,
                        double *dLdk_dev, double rtol, int max_cycles) {
    MG_TRY(ensure_adjoint_pools(F));
    DevLevel &d = F->L[0];
    const int grid = grid_for(d.cells());
    MG_CUDA(cudaMemsetAsync(F->a_lam, 0, d.pool_elems() * sizeof(double), F->st));
    k_pack<double><<<grid, kThreads, 0, F->st>>>(F->a_g, dLdu_dev, d.g, F->leaf_off);
    k_norm64<<<grid, kThreads, 0, F->st>>>(F->a_g, d.vol_64, d.g, F->partial);
    double gg = 0.0;
    MG_TRY(read_sum(F, grid, &gg));
    const double gn = std::sqrt(gg);
    double rel = gn > 0.0 ? 1.0 : 0.0;
    int it = 0;
    // Defect correction lambda += M^T (g - A^T lambda): the residual and the update in FP64; the transposed cycle
    // M^T in FP64, or, on forests with FP32 forward cycles, in FP32 on the residual scaled by a power of two near
    // 1 / ||r|| (the forward solve's mixed precision, transposed)
    const bool fp32 = F->cfg.precision == 1;
    if (fp32) MG_TRY(round_coefficients32(F));
    for (; gn > 0.0; ++it) {
        apply_T<MODE, double>(F, d, F->a_lam, d.a_tmp);
        k_sub_norm<<<grid, kThreads, 0, F->st>>>(F->a_g, d.a_tmp, d.a_ub, d.vol_64, d.g, F->partial);
        double rr = 0.0;
        MG_TRY(read_sum(F, grid, &rr));
        rel = std::sqrt(rr) / gn;
        if (!std::isfinite(rel) || rel <= rtol || it >= max_cycles) break;
        if (fp32) {
            const double sc = pow2_near(1.0 / std::sqrt(rr));
            k_scaled32<<<grid, kThreads, 0, F->st>>>(d.a_ub, d.a32_ub, sc, d.g);
            vcycle_T<MODE, float>(F, 0);
            k_add_from32<<<grid, kThreads, 0, F->st>>>(F->a_lam, d.a32_fb, 1.0 / sc, d.g);
        } else {
            vcycle_T<MODE, double>(F, 0);
            k_axpy<double><<<grid, kThreads, 0, F->st>>>(F->a_lam, d.a_fb, 1.0, d.g);
        }
    }
    k_unpack<double><<<grid, kThreads, 0, F->st>>>(lambda_dev, F->a_lam, d.g, F->leaf_off);
    MG_CUDA(cudaGetLastError());
    if (dLdk_dev && F->cfg.coeff) {
        // forward ghosts of u, then the face terms, the ghost-k maps and (conservative variant) the coarse rows
        MG_CUDA(cudaMemsetAsync(F->s64a, 0, d.pool_elems() * sizeof(double), F->st));
        k_pack<double><<<grid, kThreads, 0, F->st>>>(F->s64a, u_dev, d.g, F->leaf_off);
        exchange_any64(F, d, F->s64a);
        MG_CUDA(cudaMemsetAsync(F->s64b, 0, d.pool_elems() * sizeof(double), F->st));
        MG_CUDA(cudaMemsetAsync(d.a_tmp, 0, d.pool_elems() * sizeof(double), F->st));
        k_gradk_faces<<<grid, kThreads, 0, F->st>>>(F->s64a, F->a_lam, d.k64, d.ih2_64, d.fkind,
                                                     F->cfg.interface_flux, d.g, F->s64b, d.a_tmp);
        k_gradk_merge<<<grid, kThreads, 0, F->st>>>(F->s64b, d.a_tmp, d.g);
        if (d.nfaces)
            k_gradk_ghost_faces<<<grid_for(static_cast<int64_t>(d.nfaces) << (2 * d.g.lg)), kThreads, 0, F->st>>>(
                F->s64b, d.a_tmp, d.faces, d.nfaces, d.g);
        if (d.nsegs) {
            const int gs = grid_for(static_cast<int64_t>(d.nsegs) << (2 * (d.g.lg - 1)));
            if (F->cfg.interface_flux)
                k_gradk_flux_rows<<<gs, kThreads, 0, F->st>>>(F->s64b, F->s64a, F->a_lam, d.k64, d.ih2_64, d.segs,
                                                              d.nsegs, d.g);
            else
                k_gradk_ghost_segs<<<gs, kThreads, 0, F->st>>>(F->s64b, d.a_tmp, d.segs, d.nsegs, d.g);
        }
        k_unpack<double><<<grid, kThreads, 0, F->st>>>(dLdk_dev, F->s64b, d.g, F->leaf_off);
    }
    MG_CUDA(cudaStreamSynchronize(F->st));
    if (!std::isfinite(rel) || rel > rtol) {
        set_error("adjoint: relative residual " + fmt_e(rel) + " above rtol after " + std::to_string(it) +
                  " cycles");
        return MG_ERR_NOT_CONVERGED;
    }
    return MG_OK;
}

}  // namespace
}  // namespace octmg

using namespace octmg;

extern "C" mg_status mg_apply_transpose(mg_forest *F, const double *y_dev, double *ATy_dev) {
    if (!F || !y_dev || !ATy_dev) {
        set_error("null argument");
        return MG_ERR_INVALID_ARG;
    }
    if (F->cfg.coeff && !F->rhs_set) {
        set_error("mg_set_rhs (k) has not been called");
        return MG_ERR_STATE;
    }
    MG_TRY(adjoint_supported(F));
    MG_TRY(ensure_adjoint_pools(F));
    DevLevel &d = F->L[0];
    MG_CUDA(cudaMemsetAsync(d.a_z, 0, d.pool_elems() * sizeof(double), F->st));
    k_pack<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(d.a_z, y_dev, d.g, F->leaf_off);
    if (F->cfg.coeff)
        apply_T<1>(F, d, d.a_z, d.a_tmp);
    else
        apply_T<0>(F, d, d.a_z, d.a_tmp);
    k_unpack<double><<<grid_for(d.cells()), kThreads, 0, F->st>>>(ATy_dev, d.a_tmp, d.g, F->leaf_off);
    MG_CUDA(cudaStreamSynchronize(F->st));
    return MG_OK;
}

extern "C" mg_status mg_adjoint_solve(mg_forest *F, const double *u_dev, const double *dLdu_dev, double *lambda_dev,
                                      double *dLdk_dev, double rtol, int32_t max_cycles) {
    if (!F || !dLdu_dev || !lambda_dev || (dLdk_dev && !u_dev) || max_cycles < 0 || !(rtol >= 0.0)) {
        set_error("bad argument");
        return MG_ERR_INVALID_ARG;
    }
    MG_TRY(check_ready(F));
    MG_TRY(adjoint_supported(F));
    if (F->cfg.coeff) return adjoint_solve<1>(F, u_dev, dLdu_dev, lambda_dev, dLdk_dev, rtol, max_cycles);
    return adjoint_solve<0>(F, u_dev, dLdu_dev, lambda_dev, dLdk_dev, rtol, max_cycles);
}
