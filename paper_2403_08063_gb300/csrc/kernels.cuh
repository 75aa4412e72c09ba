// Device kernels of the octree-block multigrid (arXiv 2403.08063), written for sm_103a.
//
// Storage: every block of a level is a padded (n+2)^3 array (padded coordinate = interior + 1), one ghost layer
// per face (Sec. 3.3: one layer suffices for the quadratic C2F / linear F2C schemes); FP64 pools keep it x-fastest,
// FP32 pools split it by colour (see Lay below).  The blocks of a level are contiguous with one stride `bs`
// (elements) for both precisions: the larger of the two block sizes, rounded up to 64 elements.
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
#include <type_traits>
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

// Coefficient modes: 0 constant (-Laplace); 1 FP64 scaled face coefficients T / h^2 (natural layout); 2 FP32 1/k per
// cell, faces by harmonic means on the fly (colour-split); 3 FP32 halved face coefficients T / 2 per cell for its
// lower x, y and z faces (colour-split; the face-averaged coarse levels of FP32 cycles).
struct Coef {       // coefficient arrays of one level (unused members are null)
    const double *tx, *ty, *tz, *dg, *dinv;  // MODE 1
    const float *kap;                        // MODE 2
    const float *ax, *ay, *az;               // MODE 3
};

// Problems of a multi-problem level that have met their tolerance in a batched solve: their blocks are skipped by
// every kernel of the defect-correction step, so each problem stops where it converged (`done` null: none).
struct Skip {
    const int32_t *bprob;  // problem of each block of the level
    const uint8_t *done;   // per problem
    __device__ bool operator()(int64_t b) const { return done && done[bprob[b]]; }
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

// Padded coordinates of the cell at `depth` from face (axis, side) with tangential interior coordinates (i1, i2).
__device__ inline void face_xyz(int axis, int side, int depth, int i1, int i2, int n, int &X, int &Y, int &Z) {
    const int a = side ? (n + 1 - depth) : depth;
    const int t1 = axis == 0 ? 1 : 0;
    const int t2 = axis == 2 ? 1 : 2;
    int c[3];
    c[axis] = a;
    c[t1] = 1 + i1;
    c[t2] = 1 + i2;
    X = c[0];
    Y = c[1];
    Z = c[2];
}

// Storage of a padded cell (X, Y, Z) of block b.
//   FP64 pools: natural order, block b at b * bs, x fastest.
//   FP32 pools: colour-split ("red-black ordered"): a block is two halves holding the cells with X + Y + Z even
//   (half 0) and odd (half 1); inside a half, row (Y, Z) holds the (n+2)/2 cells of that parity at X / 2, with no
//   padding between rows.  A colour half-sweep then reads the other colour's half and writes its own with unit
//   stride.  Every half and block starts on a 16-byte boundary (P^2 is a multiple of 4); rows and planes in general
//   do not, so bulk copies of row runs are widened to 16-byte bounds (k_smooth32t).
// Row length of one half in the FP32 split layout: the (n+2)/2 cells of a parity.
__host__ __device__ constexpr int half_row(int P) { return P >> 1; }

// Block stride of a level's pools, in elements: one stride for both precisions, the natural FP64 block or the FP32
// split block (the same size), rounded to 64 elements, so every block and FP32 half starts on a 16-byte boundary and
// a bulk copy widened to 16-byte bounds at the end of the last block stays inside the pool.
__host__ __device__ constexpr int64_t block_stride(int P) {
    const int64_t nat = static_cast<int64_t>(P) * P * P, split = 2 * static_cast<int64_t>(P) * P * half_row(P);
    return ((nat > split ? nat : split) + 63) / 64 * 64;
}

template <typename T> struct Lay;
template <> struct Lay<double> {
    __device__ static int64_t at(const LevelGeom &g, int64_t b, int X, int Y, int Z) {
        return b * g.bs + off3(X, Y, Z, g.P);
    }
};
template <> struct Lay<float> {
    __host__ __device__ static int64_t at(const LevelGeom &g, int64_t b, int X, int Y, int Z) {
        const int P = g.P, hp = half_row(g.P);
        const int64_t half = static_cast<int64_t>(P) * P * hp;
        return b * g.bs + ((X + Y + Z) & 1) * half + (static_cast<int64_t>(Z) * P + Y) * hp + (X >> 1);
    }
};
template <typename T>
__device__ inline int64_t fidx(const LevelGeom &g, int64_t b, int axis, int side, int depth, int i1, int i2) {
    int X, Y, Z;
    face_xyz(axis, side, depth, i1, i2, g.n, X, Y, Z);
    return Lay<T>::at(g, b, X, Y, Z);
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
// Variant v of the scheme: 0 the quadratic rule above; 1 first order (linear along the normal through the current
// cell and the next one inward; along an orthogonal axis through the current cell and the neighbour on the target's
// side, the other neighbour when that one is outside the coarse block's interior); 2 constant (the covering coarse
// cell).  The paper names the lower orders (Table err_analysis) without describing them; these are readings.
//   v = 1 normal (5, -1, 0) / 4; orthogonal case 0: (1, 3, 0) / 4 and (0, 3, 1) / 4, case 1: (5, -1, 0) / 4 and
//   (3, 1, 0) / 4, case 2: (0, 1, 3) / 4 and (0, -1, 5) / 4.   v = 2: weight 1 on the current cell.
static __constant__ double c_wn[3][3] = {{45.0 / 32, -18.0 / 32, 5.0 / 32}, {1.25, -0.25, 0.0}, {1.0, 0.0, 0.0}};
static __constant__ double c_wt[3][3][2][3] = {
    {{{5.0 / 32, 30.0 / 32, -3.0 / 32}, {-3.0 / 32, 30.0 / 32, 5.0 / 32}},
     {{45.0 / 32, -18.0 / 32, 5.0 / 32}, {21.0 / 32, 14.0 / 32, -3.0 / 32}},
     {{-3.0 / 32, 14.0 / 32, 21.0 / 32}, {5.0 / 32, -18.0 / 32, 45.0 / 32}}},
    {{{0.25, 0.75, 0.0}, {0.0, 0.75, 0.25}}, {{1.25, -0.25, 0.0}, {0.75, 0.25, 0.0}},
     {{0.0, 0.25, 0.75}, {0.0, -0.25, 1.25}}},
    {{{0.0, 1.0, 0.0}, {0.0, 1.0, 0.0}}, {{1.0, 0.0, 0.0}, {1.0, 0.0, 0.0}}, {{0.0, 0.0, 1.0}, {0.0, 0.0, 1.0}}}};
static __constant__ int c_base[3][3] = {{-1, 0, 1}, {0, 1, 2}, {-2, -1, 0}};
static __constant__ float c_wn_f[3][3] = {{45.0f / 32, -18.0f / 32, 5.0f / 32}, {1.25f, -0.25f, 0.0f}, {1.0f, 0.0f, 0.0f}};
static __constant__ float c_wt_f[3][3][2][3] = {
    {{{5.0f / 32, 30.0f / 32, -3.0f / 32}, {-3.0f / 32, 30.0f / 32, 5.0f / 32}},
     {{45.0f / 32, -18.0f / 32, 5.0f / 32}, {21.0f / 32, 14.0f / 32, -3.0f / 32}},
     {{-3.0f / 32, 14.0f / 32, 21.0f / 32}, {5.0f / 32, -18.0f / 32, 45.0f / 32}}},
    {{{0.25f, 0.75f, 0.0f}, {0.0f, 0.75f, 0.25f}}, {{1.25f, -0.25f, 0.0f}, {0.75f, 0.25f, 0.0f}},
     {{0.0f, 0.25f, 0.75f}, {0.0f, -0.25f, 1.25f}}},
    {{{0.0f, 1.0f, 0.0f}, {0.0f, 1.0f, 0.0f}}, {{1.0f, 0.0f, 0.0f}, {1.0f, 0.0f, 0.0f}},
     {{0.0f, 0.0f, 1.0f}, {0.0f, 0.0f, 1.0f}}}};

template <typename T> __device__ inline T w_normal(int v, int a);
template <> __device__ inline double w_normal<double>(int v, int a) { return c_wn[v][a]; }
template <> __device__ inline float w_normal<float>(int v, int a) { return c_wn_f[v][a]; }
template <typename T> __device__ inline T w_tang(int v, int c, int al, int b);
template <> __device__ inline double w_tang<double>(int v, int c, int al, int b) { return c_wt[v][c][al][b]; }
template <> __device__ inline float w_tang<float>(int v, int c, int al, int b) { return c_wt_f[v][c][al][b]; }

// Global load of data that other CTAs of the same launch may have written earlier (CG = true: through L2 only,
// as in the persistent tail kernel, whose phases are separated by grid barriers), or a plain load.
template <bool CG, typename T>
__device__ __forceinline__ T ldv(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// Read-only-for-this-launch data (f of a level), or written by an earlier phase of a persistent launch (CG = true).
template <bool CG, typename T>
__device__ __forceinline__ T ldr(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}

__device__ inline float frcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// t / 6 for the constant-coefficient FP32 smoothers.  Multiplying by the binary32 value of 1/6, which is 3.0e-8
// (relative) too large, biases every update the same way, and the bias accumulates over the sweeps of a cycle
// (the FP32 V-cycle landed 17x further from the FP64 cycle than a plain FP32 evaluation).  Splitting 1/6 into a
// head and a tail that sum to it within 2^-48 and rounding once in an FMA gives t / 6 to within about half an ulp
// with no bias.
__device__ __forceinline__ float div6(float t) {
    constexpr float hi = 1.0f / 6.0f;
    constexpr float lo = static_cast<float>(1.0 / 6.0 - static_cast<double>(1.0f / 6.0f));
    return fmaf(t, hi, t * lo);
}

// Two lanes of frcp and div6 for the paired FP32 instructions (each component as the scalar function).
__device__ __forceinline__ float2 frcp2(float2 x) { return float2{frcp(x.x), frcp(x.y)}; }
__device__ __forceinline__ float2 div6x2(float2 t) {
    constexpr float hi = 1.0f / 6.0f;
    constexpr float lo = static_cast<float>(1.0 / 6.0 - static_cast<double>(1.0f / 6.0f));
    return __ffma2_rn(t, float2{hi, hi}, __fmul2_rn(t, float2{lo, lo}));
}

// Conversions between binary64 and binary32 with an exact power-of-two scale, written on the IEEE 754 bit fields
// (1 sign bit; 11 / 8 exponent bits with bias 1023 / 127; 52 / 23 fraction bits) so that they run on the integer
// pipes: the hardware conversion instructions between the two formats issue on the FP64 pipe, the bottleneck of
// the FP64 residual on this GPU.  Results below the binary32 normal range flush to a signed zero (binary32
// subnormals are not produced or read); the scale exponent is |sexp| <= 126.
// round_to_nearest_even(r * 2^sexp) as binary32
__device__ __forceinline__ float f64_to_f32_pow2(double r, int sexp) {
    const uint64_t bits = static_cast<uint64_t>(__double_as_longlong(r));
    const uint32_t sign = static_cast<uint32_t>(bits >> 32) & 0x80000000u;
    const int e = static_cast<int>((bits >> 52) & 0x7ff) - 1023 + 127 + sexp;  // binary32 biased exponent
    const uint32_t m = static_cast<uint32_t>(bits >> 29) & 0x7fffffu;          // the 23 kept fraction bits
    const uint32_t rest = static_cast<uint32_t>(bits) & 0x1fffffffu;           // the 29 dropped ones
    const uint32_t up = (rest > 0x10000000u) || (rest == 0x10000000u && (m & 1u));
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(((sign | (static_cast<uint32_t>(e) << 23)) | m) + up);  // a carry rounds up the exponent
}
// x * 2^pexp as binary64 (exact)
__device__ __forceinline__ double f32_to_f64_pow2(float x, int pexp) {
    const uint32_t bits = __float_as_uint(x);
    const uint64_t sign = static_cast<uint64_t>(bits & 0x80000000u) << 32;
    const int e = static_cast<int>((bits >> 23) & 0xff);
    if (e == 0) return __longlong_as_double(static_cast<long long>(sign));
    const uint64_t ed = e == 255 ? 0x7ffull : static_cast<uint64_t>(e - 127 + 1023 + pexp);
    return __longlong_as_double(static_cast<long long>(sign | (ed << 52) | (static_cast<uint64_t>(bits & 0x7fffffu) << 29)));
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
    if (MODE == 3) {
        const float *a = axis == 0 ? c.ax : (axis == 1 ? c.ay : c.az);
        return T(2.0f * a[loc]);
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
// gb (FP64 finest level only, may be null): 2 g on the domain-boundary faces, (b * 6 + face) * n^2 + i2 n + i1, so the
// reflection ghost is 2 g - u_i (inhomogeneous Dirichlet data, Sec. 5 Eq. 2); c2f: the coarse-to-fine variant.
template <typename T, bool KIND_K, bool CG = false>
__device__ __forceinline__ void exchange_faces_body(T *__restrict__ u, const FaceItem *__restrict__ items, int nitems,
                                                    LevelGeom g, Skip skip, int64_t t0, int64_t ts, int c2f = 0,
                                                    const T *__restrict__ gb = nullptr) {
    const int n = g.n, lg = g.lg, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lg);
    for (int64_t t = t0; t < total; t += ts) {
        const int it = static_cast<int>(t >> (2 * lg));
        const int r = static_cast<int>(t) & ((1 << (2 * lg)) - 1);
        const int i1 = r & (n - 1), i2 = r >> lg;
        const FaceItem F = items[it];
        if (skip(F.blk)) continue;
        T val;
        if (F.kind == FK_BND) {
            const T in = ldv<CG>(u + fidx<T>(g, F.blk, F.axis, F.side, 1, i1, i2));
            val = KIND_K ? in : (gb ? gb[(static_cast<int64_t>(F.blk) * 6 + 2 * F.axis + F.side) * n * n + i2 * n + i1] - in
                                     : -in);
        } else if (F.kind == FK_SAME) {
            val = ldv<CG>(u + fidx<T>(g, F.nbr, F.axis, 1 - F.side, 1, i1, i2));
        } else {
            const int yc = F.seg1 * h + (i1 >> 1), zc = F.seg2 * h + (i2 >> 1);
            if (KIND_K) {
                val = ldv<CG>(u + fidx<T>(g, F.nbr, F.axis, 1 - F.side, 1, yc, zc));
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
                        T e = w_normal<T>(c2f, 0) * ldv<CG>(u + fidx<T>(g, F.nbr, F.axis, 1 - F.side, 1, y, z));
                        e = fma(w_normal<T>(c2f, 1), ldv<CG>(u + fidx<T>(g, F.nbr, F.axis, 1 - F.side, 2, y, z)), e);
                        e = fma(w_normal<T>(c2f, 2), ldv<CG>(u + fidx<T>(g, F.nbr, F.axis, 1 - F.side, 3, y, z)), e);
                        accb = fma(w_tang<T>(c2f, cy, a1, b), e, accb);
                    }
                    acc = fma(w_tang<T>(c2f, cz, a2, c), accb, acc);
                }
                val = acc;
            }
        }
        u[fidx<T>(g, F.blk, F.axis, F.side, 0, i1, i2)] = val;
    }
}

// Every block face's ghost layer of a level, one thread per ghost cell: same-level copy (Sec. 3.1), quadratic
// coarse-to-fine extrapolation (Sec. 3.3.2) and the Dirichlet reflection at the domain boundary (Sec. 5, Eq. 2).
template <typename T, bool KIND_K>
static __global__ void k_exchange_faces(T *__restrict__ u, const FaceItem *__restrict__ items, int nitems, LevelGeom g,
                                        Skip skip = Skip{}, int c2f = 0, const T *__restrict__ gb = nullptr) {
    exchange_faces_body<T, KIND_K>(u, items, nitems, g, skip, blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x,
                                   static_cast<int64_t>(gridDim.x) * blockDim.x, c2f, gb);
}

// Coarse-to-fine ghosts of refinement interfaces only (Sec. 3.3.2), one CTA per fine block face, with the
// intermediate results shared between neighbouring coarse cells: the normal-direction extrapolation (the 1D step
// through the current coarse cell and the two inward) of every coarse cell of the segment and of its one-cell
// tangential border is computed once into shared memory, and each coarse cell's four fine ghosts are the
// tangential interpolation of 3 x 3 of those values.  Sec. 8 of the paper proposes this reuse of intermediate
// extrapolation results for neighbouring cells (a ring buffer on CPUs, shared memory on GPUs); it takes 3 loads per
// intermediate value, about 3.4 per coarse cell, instead of 27 per fine ghost.  Same operations in the same order as
// exchange_faces_body, so the same bits.  Dynamic shared memory: (n/2 + 2)^2 values of T.
template <typename T>
static __global__ void k_exchange_c2f_smem(T *__restrict__ u, const FaceItem *__restrict__ items, LevelGeom g,
                                           Skip skip, int c2f) {
    extern __shared__ __align__(16) unsigned char c2f_smem[];
    T *E = reinterpret_cast<T *>(c2f_smem);
    const FaceItem F = items[blockIdx.x];
    if (skip(F.blk)) return;  // uniform over the CTA, before the barrier
    const int n = g.n, h = n >> 1;
    // coarse cells [lo1, lo1 + w1) x [lo2, lo2 + w2) of the coarse face: the segment and the neighbours its
    // stencils reach (remapped bases stay inside the coarse block)
    const int lo1 = max(0, F.seg1 * h - 1), w1 = min(n - 1, F.seg1 * h + h) - lo1 + 1;
    const int lo2 = max(0, F.seg2 * h - 1), w2 = min(n - 1, F.seg2 * h + h) - lo2 + 1;
    for (int q = threadIdx.x; q < w1 * w2; q += blockDim.x) {
        const int y = lo1 + q % w1, z = lo2 + q / w1;
        T v = w_normal<T>(c2f, 0) * u[fidx<T>(g, F.nbr, F.axis, 1 - F.side, 1, y, z)];
        v = fma(w_normal<T>(c2f, 1), u[fidx<T>(g, F.nbr, F.axis, 1 - F.side, 2, y, z)], v);
        E[q] = fma(w_normal<T>(c2f, 2), u[fidx<T>(g, F.nbr, F.axis, 1 - F.side, 3, y, z)], v);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < h * h; q += blockDim.x) {
        const int ycl = q % h, zcl = q / h;
        const int yc = F.seg1 * h + ycl, zc = F.seg2 * h + zcl;
        const int cy = yc == 0 ? 1 : (yc == n - 1 ? 2 : 0);
        const int cz = zc == 0 ? 1 : (zc == n - 1 ? 2 : 0);
        T e[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int b = 0; b < 3; ++b)
                e[c][b] = E[(zc + c_base[cz][c] - lo2) * w1 + (yc + c_base[cy][b] - lo1)];
#pragma unroll
        for (int a2 = 0; a2 < 2; ++a2)
#pragma unroll
            for (int a1 = 0; a1 < 2; ++a1) {
                T acc = T(0);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    T accb = T(0);
#pragma unroll
                    for (int b = 0; b < 3; ++b) accb = fma(w_tang<T>(c2f, cy, a1, b), e[c][b], accb);
                    acc = fma(w_tang<T>(c2f, cz, a2, c), accb, acc);
                }
                u[fidx<T>(g, F.blk, F.axis, F.side, 0, 2 * ycl + a1, 2 * zcl + a2)] = acc;
            }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Ghost exchange, part 2: coarse ghost segments next to finer neighbours.
// FLUX = false: F2C mean of the 2x2x2 fine inner cells overlapping each coarse ghost cell (Sec. 3.3.1).
// FLUX = true:  conservative coarse ghost G with T_C (u_C - G) = 1/2 sum_j T_j (g_j - u_j) over the four fine
//               sub-faces j, g_j the fine ghosts (C2F, part 1 must have run), u_j the first fine layer.  With the
//               1/h^2-scaled coefficients of MODE 1, T_j / (2 T_C) = T~_j / (8 T~_C) since h_C = 2 h_j.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE, bool FLUX, bool CG = false>
__device__ __forceinline__ void exchange_segs_body(T *__restrict__ u, Coef cf, const SegItem *__restrict__ items,
                                                   int nitems, LevelGeom g, Skip skip, int64_t t0, int64_t ts) {
    const int n = g.n, lgh = g.lg - 1, h = n >> 1;
    const int64_t total = static_cast<int64_t>(nitems) << (2 * lgh);
    for (int64_t t = t0; t < total; t += ts) {
        const int it = static_cast<int>(t >> (2 * lgh));
        const int r = static_cast<int>(t) & ((1 << (2 * lgh)) - 1);
        const int p = r & (h - 1), q = r >> lgh;
        const SegItem S = items[it];
        if (skip(S.coarse)) continue;
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
                    for (int a = 0; a < 2; ++a) s += ldv<CG>(u + fidx<T>(g, S.fine, S.axis, fs, d, 2 * p + a, 2 * q + b));
            val = T(0.125) * s;
        } else {
            const int64_t gC = fidx<T>(g, S.coarse, S.axis, S.side, 1, yc, zc);
            const int64_t g0c = fidx<T>(g, S.coarse, S.axis, S.side, 0, yc, zc);
            const T uC = ldv<CG>(u + gC);
            T flux = T(0);
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int64_t g0 = fidx<T>(g, S.fine, S.axis, fs, 0, 2 * p + a, 2 * q + b);
                    const int64_t g1 = fidx<T>(g, S.fine, S.axis, fs, 1, 2 * p + a, 2 * q + b);
                    const T Tj = face_coef<T, MODE>(cf, fs ? g0 : g1, fs ? g1 : g0, S.axis);
                    flux = fma(Tj, ldv<CG>(u + g0) - ldv<CG>(u + g1), flux);
                }
            const T Tc = face_coef<T, MODE>(cf, S.side ? g0c : gC, S.side ? gC : g0c, S.axis);
            val = uC - flux / (T(MODE == 1 ? 8 : 2) * Tc);
        }
        u[fidx<T>(g, S.coarse, S.axis, S.side, 0, yc, zc)] = val;
    }
}

// Fine-to-coarse ghosts (Sec. 3.3.1: mean of the 2 x 2 x 2 fine cells over a coarse ghost), or with FLUX the
// conservative coarse ghost whose flux is the sum of the four fine sub-face fluxes (this library's reading).
template <typename T, int MODE, bool FLUX>
static __global__ void k_exchange_segs(T *__restrict__ u, Coef cf, const SegItem *__restrict__ items, int nitems,
                                       LevelGeom g, Skip skip = Skip{}) {
    exchange_segs_body<T, MODE, FLUX>(u, cf, items, nitems, g, skip,
                                      blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x,
                                      static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// ------------------------------------------------------------------------------------------------------------
// Red-black Gauss-Seidel half-sweep (the smoother of the problem statement; Sec. 5 smooths with damped Jacobi) of
// one colour ((x+y+z) mod 2 of the block-local interior index; red = 0):
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
                                LevelGeom g, int colour, const int32_t *__restrict__ nbr6, Skip skip = Skip{},
                                const T *__restrict__ gb = nullptr) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg - 1);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int j = static_cast<int>(t & ((n >> 1) - 1));
        const int y = static_cast<int>((t >> (lg - 1)) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg - 1)) & (n - 1));
        const int64_t b = t >> (3 * lg - 1);
        if (skip(b)) continue;
        const int x = 2 * j + ((y + z + colour) & 1);
        T val;
        if constexpr (sizeof(T) == 4) {
            // colour-split: this colour's cells have padded parity s = colour ^ 1; in row (Y, Z) the cell X = 2m + o
            // (o = (s + Y + Z) & 1) sits at m of half s, its x-neighbours at m - 1 + o and m + o of half s ^ 1, its
            // y- and z-neighbours at m in the adjacent rows of half s ^ 1
            const int hp = half_row(P);
            const int64_t half = static_cast<int64_t>(P) * P * hp;
            const int s = colour ^ 1;
            const int Y = y + 1, Z = z + 1;
            const int o = (s + Y + Z) & 1;
            const int m = (x + 1) >> 1;
            const int64_t row = (static_cast<int64_t>(Z) * P + Y) * hp;
            const int64_t own = b * g.bs + s * half + row + m;
            const int64_t oth = b * g.bs + (s ^ 1) * half + row;
            const int64_t ixm = oth + m - 1 + o, ixp = ixm + 1, iym = oth - hp + m, iyp = oth + hp + m;
            const int64_t izm = oth - static_cast<int64_t>(P) * hp + m, izp = oth + static_cast<int64_t>(P) * hp + m;
            if constexpr (MODE == 0) {
                const float S = ((u[ixm] + u[ixp]) + (u[iym] + u[iyp])) + (u[izm] + u[izp]);
                val = T(div6(fmaf(float(h2[b]), float(f[own]), S)));
            } else {
                const float *kap = cf.kap;
                const float k0 = kap[own];
                const float a0 = frcp(k0 + kap[ixm]), a1 = frcp(k0 + kap[ixp]);
                const float b0 = frcp(k0 + kap[iym]), b1 = frcp(k0 + kap[iyp]);
                const float c0 = frcp(k0 + kap[izm]), c1 = frcp(k0 + kap[izp]);
                float sacc = a0 * u[ixm];
                sacc = fmaf(a1, u[ixp], sacc);
                sacc = fmaf(b0, u[iym], sacc);
                sacc = fmaf(b1, u[iyp], sacc);
                sacc = fmaf(c0, u[izm], sacc);
                sacc = fmaf(c1, u[izp], sacc);
                const float D = ((a0 + a1) + (b0 + b1)) + (c0 + c1);
                val = T(fmaf(float(h2[b]), float(f[own]), 2.0f * sacc) * frcp(2.0f * D));
            }
            u[own] = val;
        } else {
            const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
            if constexpr (MODE == 1) {
                val = sten1(u, cf, gi, P, f[gi]) * cf.dinv[gi];
            } else {
                val = fma(h2[b], f[gi], sten0<T>(u, gi, P)) * T(1.0 / 6.0);
            }
            u[gi] = val;
        }
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
                        u[fidx<T>(g, nb, axis, 1 - side, 0, i1, i2)] = val;
                    else if (nb == -1)  // reflection, with the boundary data 2 g where given (gb: finest level)
                        u[fidx<T>(g, b, axis, side, 0, i1, i2)] =
                            gb ? gb[(b * 6 + 2 * axis + side) * static_cast<int64_t>(n) * n + i2 * n + i1] - val : -val;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------------------
// Damped Jacobi sweep (the paper's smoother and coarsest solver, Sec. 5), FP64, ghosts as left by the last exchange:
//     uo_i = (1 - omega) u_i + omega (h^2 f_i + sum_f T_f u_f) / sum_f T_f
// for every cell of the level at once, into the second pool uo (interior only; its ghosts need an exchange).
// ------------------------------------------------------------------------------------------------------------
template <int MODE>
static __global__ void k_jacobi64(const double *__restrict__ u, double *__restrict__ uo, const double *__restrict__ f,
                                  Coef cf, const double *__restrict__ h2, LevelGeom g, double omega,
                                  Skip skip = Skip{}) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        if (skip(b)) continue;
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        double nw;
        if constexpr (MODE == 1)
            nw = sten1(u, cf, gi, P, f[gi]) * cf.dinv[gi];
        else
            nw = fma(h2[b], f[gi], sten0<double>(u, gi, P)) * (1.0 / 6.0);
        uo[gi] = fma(omega, nw - u[gi], u[gi]);
    }
}

// ------------------------------------------------------------------------------------------------------------
// FP32 half-sweep on colour-split blocks with the block edge n = 2^LG fixed at compile time, so that every
// neighbour of a cell is an immediate offset from a few row pointers and all in-block offsets are 32-bit.
//
// Thread (b, j, y, z-group) updates the ZC cells x = 2j + c_z, z = z0 .. z0 + ZC - 1 of one z-column, where
// c_z = (y + z + colour) & 1.  With H = half_row(P) and row r_z = ((z+1) P + y+1) H of either half, such a cell sits
// at r_z + j + c_z of its colour's half.  Of the other half it reads r_z + j and r_z + j + 1 (its x-neighbours,
// whatever c_z), r_z -/+ H + j + c_z (y) and r_(z-/+1) + j + c_z (z).  Because c_(z+-1) = 1 - c_z, the z-neighbours
// of a column cell are x-neighbour pairs of the adjacent column cells, so the column loads the pairs of its ZC
// rows, one value in each of the two rows beyond, and the y-neighbours: 4 ZC + 2 values of u and of kappa instead
// of 6 ZC.  All loads of the column are issued before any store (the other half is not written by the sweep, but
// the compiler cannot prove it), which keeps 10 ZC + 4 independent loads per thread in flight.
//
// Write-through as in k_smooth: a cell on a block face stores its new value into the same-level neighbour's ghost
// that mirrors it (same half, offset +-n along the axis, i.e. +-n/2, +-n H or +-n P H elements), or -value into
// its own reflection ghost (the other half, at the neighbour position it read).  Mirrored ghosts belong to the
// colour being updated, which this half-sweep never reads; a reflection ghost is read only by the cell that writes
// it, before the write.  x faces concern one lane of a row (j = 0 with c = 0, j = n/2 - 1 with c = 1) and take a
// short path of their own; y and z faces are uniform over a row.
// ------------------------------------------------------------------------------------------------------------
template <int MODE, int LG, int ZC, bool CG = false>
__device__ __forceinline__ void smooth32_column(float *__restrict__ u, const float *__restrict__ f,
                                                const float *__restrict__ kap, const float *__restrict__ h2,
                                                int64_t bs, int colour, const int32_t *__restrict__ nbr6,
                                                Skip skip, int64_t t, const float *__restrict__ ax = nullptr,
                                                const float *__restrict__ ay = nullptr,
                                                const float *__restrict__ az = nullptr) {
    constexpr int n = 1 << LG, NH = n / 2, P = n + 2, HP = half_row(P), PL = P * HP, HALF = P * PL;
    constexpr int LZ = ZC == 1 ? 0 : (ZC == 2 ? 1 : (ZC == 4 ? 2 : 3));
    static_assert((1 << LZ) == ZC && ZC <= n, "column length");
    constexpr int SH = 3 * LG - 1 - LZ;  // log2(columns per block)
    const int r = static_cast<int>(t) & ((1 << SH) - 1);
    const int64_t b = t >> SH;
    if (skip(b)) return;
    const int j = r & (NH - 1);
    const int y = (r >> (LG - 1)) & (n - 1);
    const int z0 = (r >> (2 * LG - 1)) << LZ;
    const int s = colour ^ 1;  // padded parity of this colour's cells
    const int c0 = (y + z0 + colour) & 1;
    const int row0 = ((z0 + 1) * P + (y + 1)) * HP + j;  // r_z0 + j, inside a half
    const int io = (s ^ 1) * HALF + row0;                 // other half at r_z0 + j
    const int ioc = io + c0;
    const int iw = s * HALF + row0 + c0;                  // own half, cell z0 (odd dz: -/+ 1)
    const int64_t base = b * bs;
    float *ub = u + base;
    const float *fb = f + base, *kb = kap + base;
    // ---- loads -------------------------------------------------------------------------------------
    float xr0[ZC], xr1[ZC], ym[ZC], yp[ZC], fv[ZC];
    float kx0[ZC], kx1[ZC], kym[ZC], kyp[ZC], k0[ZC];
    float kzlo = 0.f, kzhi = 0.f;
    constexpr int odd = (ZC - 1) & 1;  // c of the last cell is c0 ^ odd
    const float zlo = ldv<CG>(ub + (ioc - PL));
    const float zhi = ldv<CG>(ub + ((odd ? io + 1 - c0 : ioc) + ZC * PL));
#pragma unroll
    for (int dz = 0; dz < ZC; ++dz) {
        xr0[dz] = ldv<CG>(ub + (io + dz * PL));
        xr1[dz] = ldv<CG>(ub + (io + dz * PL + 1));
        const int ic = (dz & 1) ? io + 1 - c0 : ioc;  // other half at r_z + j + c_z
        ym[dz] = ldv<CG>(ub + (ic + dz * PL - HP));
        yp[dz] = ldv<CG>(ub + (ic + dz * PL + HP));
        fv[dz] = ldr<CG>(fb + ((dz & 1) ? iw + 1 - 2 * c0 : iw) + dz * PL);
    }
    if constexpr (MODE == 2) {
        kzlo = __ldg(kb + ioc - PL);
        kzhi = __ldg(kb + (odd ? io + 1 - c0 : ioc) + ZC * PL);
#pragma unroll
        for (int dz = 0; dz < ZC; ++dz) {
            kx0[dz] = __ldg(kb + io + dz * PL);
            kx1[dz] = __ldg(kb + io + dz * PL + 1);
            const int ic = (dz & 1) ? io + 1 - c0 : ioc;
            kym[dz] = __ldg(kb + ic + dz * PL - HP);
            kyp[dz] = __ldg(kb + ic + dz * PL + HP);
            k0[dz] = __ldg(kb + ((dz & 1) ? iw + 1 - 2 * c0 : iw) + dz * PL);
        }
    }
    // MODE 3: the stored halved face coefficients, a cell's lower faces at the cell, its upper ones at the upper
    // neighbour (other half: x+ at the second of the x pair, y+ at the next row, z+ at the cell above)
    float fx0[ZC], fx1[ZC], fy0[ZC], fy1[ZC], fz0[ZC], fz1[ZC];
    if constexpr (MODE == 3) {
#pragma unroll
        for (int dz = 0; dz < ZC; ++dz) {
            const int own = ((dz & 1) ? iw + 1 - 2 * c0 : iw) + dz * PL;
            const int ic = (dz & 1) ? io + 1 - c0 : ioc;
            fx0[dz] = __ldg(ax + base + own);
            fx1[dz] = __ldg(ax + base + io + dz * PL + 1);
            fy0[dz] = __ldg(ay + base + own);
            fy1[dz] = __ldg(ay + base + ic + dz * PL + HP);
            fz0[dz] = __ldg(az + base + own);
            fz1[dz] = __ldg(az + base + io + (dz + 1) * PL + (c0 ^ (dz & 1)));
        }
    }
    const float hb = __ldg(h2 + b), hh = 0.5f * hb;  // T_f = 2 / (kap_i + kap_f): its 2 cancels against h^2 / 2
    // ---- updates -----------------------------------------------------------------------------------
    float val[ZC];
#pragma unroll
    for (int dz = 0; dz < ZC; ++dz) {
        const int c = c0 ^ (dz & 1);
        const float zm = dz == 0 ? zlo : (c ? xr1[dz - 1] : xr0[dz - 1]);
        const float zp = dz == ZC - 1 ? zhi : (c ? xr1[dz + 1] : xr0[dz + 1]);
        if constexpr (MODE == 2 || MODE == 3) {
            float a0, a1, b0, b1, e0, e1;
            if constexpr (MODE == 2) {
                const float kzm = dz == 0 ? kzlo : (c ? kx1[dz - 1] : kx0[dz - 1]);
                const float kzp = dz == ZC - 1 ? kzhi : (c ? kx1[dz + 1] : kx0[dz + 1]);
                const float kc = k0[dz];
                a0 = frcp(kc + kx0[dz]);
                a1 = frcp(kc + kx1[dz]);
                b0 = frcp(kc + kym[dz]);
                b1 = frcp(kc + kyp[dz]);
                e0 = frcp(kc + kzm);
                e1 = frcp(kc + kzp);
            } else {
                a0 = fx0[dz];
                a1 = fx1[dz];
                b0 = fy0[dz];
                b1 = fy1[dz];
                e0 = fz0[dz];
                e1 = fz1[dz];
            }
            float sacc = a0 * xr0[dz];
            sacc = fmaf(a1, xr1[dz], sacc);
            sacc = fmaf(b0, ym[dz], sacc);
            sacc = fmaf(b1, yp[dz], sacc);
            sacc = fmaf(e0, zm, sacc);
            sacc = fmaf(e1, zp, sacc);
            const float D = ((a0 + a1) + (b0 + b1)) + (e0 + e1);
            val[dz] = fmaf(hh, fv[dz], sacc) * frcp(D);
        } else {
            const float S = ((xr0[dz] + xr1[dz]) + (ym[dz] + yp[dz])) + (zm + zp);
            val[dz] = div6(fmaf(hb, fv[dz], S));
        }
    }
#pragma unroll
    for (int dz = 0; dz < ZC; ++dz) ub[((dz & 1) ? iw + 1 - 2 * c0 : iw) + dz * PL] = val[dz];
    // ---- write-through -----------------------------------------------------------------------------
    if (!nbr6) return;
    if (j == 0 || j == NH - 1) {  // x faces: the first and last lane of a row, side 0 / 1, the cells with c == side
        const int side = j == 0 ? 0 : 1;
        const int nbv = nbr6[b * 6 + side];
#pragma unroll
        for (int dz = 0; dz < ZC; ++dz) {
            const int c = c0 ^ (dz & 1);
            if (c != side) continue;
            const int q = row0 + dz * PL + c;  // the cell inside its half
            if (nbv >= 0) u[nbv * bs + s * HALF + q + (side ? -NH : NH)] = val[dz];
            else if (nbv == -1) ub[(s ^ 1) * HALF + q] = -val[dz];
        }
    }
    if (y == 0 || y == n - 1 || z0 == 0 || z0 + ZC == n) {
#pragma unroll
        for (int dz = 0; dz < ZC; ++dz) {
            const int c = c0 ^ (dz & 1);
            const int q = row0 + dz * PL + c;
            const int z = z0 + dz;
#pragma unroll
            for (int axis = 1; axis < 3; ++axis) {
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if ((axis == 1 ? y : z) != (side ? n - 1 : 0)) continue;
                    const int Dm = axis == 1 ? n * HP : n * PL, E = axis == 1 ? HP : PL;
                    const int nbv = nbr6[b * 6 + 2 * axis + side];
                    if (nbv >= 0) u[nbv * bs + s * HALF + q + (side ? -Dm : Dm)] = val[dz];
                    else if (nbv == -1) ub[(s ^ 1) * HALF + q + (side ? E : -E)] = -val[dz];
                }
            }
        }
    }
}

// FP32 red-black Gauss-Seidel half-sweep on colour-split blocks of edge 2^LG, one column per thread over `total`
// columns (the update of k_smooth, Sec. 5 operator).
template <int MODE, int LG, int ZC>
static __global__ void __launch_bounds__(512) k_smooth32(float *__restrict__ u, const float *__restrict__ f,
                                                         const float *__restrict__ kap, const float *__restrict__ h2,
                                                         int64_t total, int64_t bs, int colour,
                                                         const int32_t *__restrict__ nbr6, Skip skip,
                                                         const float *__restrict__ ax, const float *__restrict__ ay,
                                                         const float *__restrict__ az) {
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t < total) smooth32_column<MODE, LG, ZC>(u, f, kap, h2, bs, colour, nbr6, skip, t, ax, ay, az);
}

// ------------------------------------------------------------------------------------------------------------
// Shared-memory staging with the bulk-copy (TMA) engine: mbarrier helpers.  One thread arms a barrier with the
// byte count of the copies it issues; every consumer polls the barrier's phase with a bounded wait.
// ------------------------------------------------------------------------------------------------------------
__device__ inline uint32_t smem_u32(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void mbar_arm(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// plain arrival (release) of one thread on `bar`
__device__ inline void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// global -> shared bulk copy completing on `bar`; both addresses 16-byte aligned, bytes a multiple of 16
__device__ inline void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// One potentially blocking probe of phase `parity`: the thread is suspended in hardware (issuing nothing) until the
// phase completes or about 20 us pass.
__device__ inline bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return done != 0;
}
// Waits for phase `parity` of `bar` to complete; gives up after 2^14 probes (a fraction of a second) and returns
// false.
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int it = 0; it < (1 << 14); ++it)
        if (mbar_try(bar, parity)) return true;
    return false;
}

// ------------------------------------------------------------------------------------------------------------
// Copy plan of the staged half-sweep below (k_smooth32t), shared by the kernel's producer thread, the launch code
// (dynamic shared-memory size) and the host-side enumerator that checks every copy against the bulk-copy rules.
//
// Shared memory, in floats from the start: RO = D + 2 other-half slots of NA so floats, then RW = D + 1 own-half
// slots of NA sw floats, then 2 G + 2 mbarriers (G = D + 1).  NA arrays per half: 1 (constant k: u; f), 2 (1/k: u,
// kappa; f, kappa) or 4 (stored halved face coefficients: u, ax, ay, az; f, ax, ay, az), each NA-th part of a slot
// one array's plane segment.  A plane segment of len floats starting at float off of its half is copied from
// off & ~3 (the 16-byte boundary at or below it), (off & 3) + len floats rounded up to a multiple of 4, so it lands
// off & 3 floats into its slot.
// ------------------------------------------------------------------------------------------------------------
struct S32tPlan {
    int P, H, NA, RO, RW, G;  // padded edge, half-row length, staged arrays per half, ring sizes, group barriers
    int lo, lw, so, sw;       // other / own segment lengths and slot strides (floats)
};
// staged arrays per half of coefficient mode 0, 2 or 3
__host__ __device__ constexpr int s32t_arrays(int mode) { return mode == 3 ? 4 : (mode == 2 ? 2 : 1); }
__host__ __device__ __forceinline__ S32tPlan s32t_plan(int lg, int na, int TY, int D) {
    S32tPlan p;
    p.P = (1 << lg) + 2;
    p.H = half_row(p.P);
    p.NA = na;
    p.RO = 2 + D;
    p.RW = 1 + D;
    p.G = 1 + D;
    p.lo = (TY + 2) * p.H;
    p.lw = TY * p.H;
    p.so = (p.lo + 6) & ~3;  // room for the widening to 16-byte bounds
    p.sw = (p.lw + 6) & ~3;
    return p;
}
__host__ __device__ __forceinline__ int s32t_other_slot(const S32tPlan &p, int i) { return i * p.NA * p.so; }
__host__ __device__ __forceinline__ int s32t_own_slot(const S32tPlan &p, int i) {
    return p.NA * p.RO * p.so + i * p.NA * p.sw;
}
__host__ __device__ __forceinline__ int s32t_bar_floats(const S32tPlan &p) { return p.NA * (p.RO * p.so + p.RW * p.sw); }
__host__ __device__ __forceinline__ size_t s32t_smem_bytes(const S32tPlan &p) {
    return static_cast<size_t>(4) * s32t_bar_floats(p) + static_cast<size_t>(8) * (2 * p.G + 2);
}
// start (floats, within a half) of the other-half segment of padded plane Zp (rows y0 - 1 .. y0 + TY) and of the
// own-half one (rows y0 .. y0 + TY - 1)
__host__ __device__ __forceinline__ int s32t_off_other(const S32tPlan &p, int Zp, int y0) { return (Zp * p.P + y0) * p.H; }
__host__ __device__ __forceinline__ int s32t_off_own(const S32tPlan &p, int Zp, int y0) { return (Zp * p.P + y0 + 1) * p.H; }
__host__ __device__ __forceinline__ uint32_t s32t_bytes(int off, int len) {
    return static_cast<uint32_t>(((off & 3) + len + 3) & ~3) * 4;
}
// Array numbers of the a-th staged array of the other and of the own half: 0 other-half u, 1 other-half kappa or
// ax, 2 own-half f, 3 own-half kappa or ax, 4 / 5 other-half ay / az, 6 / 7 own-half ay / az.
__host__ __device__ __forceinline__ int s32t_other_array(int a) { return a < 2 ? a : a + 2; }
__host__ __device__ __forceinline__ int s32t_own_array(int a) { return a < 2 ? a + 2 : a + 4; }
// The copies of one CTA.  sink.arm(bar, bytes) arms barrier `bar` (0: the first planes; 1 + g % G: group g) with
// the bytes that will complete it; sink.copy(dst, array, src, lead, bytes, bar) copies `bytes` from float `src` of
// `array` (numbered as above) to shared float `dst`, the wanted segment starting `lead` floats into the copy.
// First: other-half padded planes z0 and z0 + 1 (planes z0 - 1 and z0) into other slots 0 and 1.
#pragma nv_exec_check_disable
template <class Sink>
__host__ __device__ __forceinline__ void s32t_issue_first(const S32tPlan &p, int z0, int y0, Sink &&sink) {
    const int o0 = s32t_off_other(p, z0, y0), o1 = s32t_off_other(p, z0 + 1, y0);
    const uint32_t b0 = s32t_bytes(o0, p.lo), b1 = s32t_bytes(o1, p.lo);
    sink.arm(0, p.NA * (b0 + b1));
    for (int io = 0; io < 2; ++io) {
        const int off = io ? o1 : o0;
        const uint32_t bb = io ? b1 : b0;
        const int d = s32t_other_slot(p, io);
        for (int a = 0; a < p.NA; ++a) sink.copy(d + a * p.so, s32t_other_array(a), off & ~3, off & 3, bb, 0);
    }
}
// Group g: other-half padded plane z0 + g + 2 (plane z0 + g + 1) into other slot (g + 2) % RO, own-half padded
// plane z0 + g + 1 (plane z0 + g) into own slot g % RW.
#pragma nv_exec_check_disable
template <class Sink>
__host__ __device__ __forceinline__ void s32t_issue_group(const S32tPlan &p, int z0, int y0, int g, Sink &&sink) {
    const int bi = 1 + g % p.G;
    const int oo = s32t_off_other(p, z0 + g + 2, y0), ow = s32t_off_own(p, z0 + 1 + g, y0);
    const uint32_t bo = s32t_bytes(oo, p.lo), bw = s32t_bytes(ow, p.lw);
    sink.arm(bi, p.NA * (bo + bw));
    const int d0 = s32t_other_slot(p, (g + 2) % p.RO), d1 = s32t_own_slot(p, g % p.RW);
    for (int a = 0; a < p.NA; ++a) sink.copy(d0 + a * p.so, s32t_other_array(a), oo & ~3, oo & 3, bo, bi);
    for (int a = 0; a < p.NA; ++a) sink.copy(d1 + a * p.sw, s32t_own_array(a), ow & ~3, ow & 3, bw, bi);
}
// The kernel's sink: arms the CTA's mbarriers and issues the bulk copies.
struct S32tDeviceSink {
    float *smem;
    const float *src[8];  // the block's halves of the arrays, numbered as above (null where not staged)
    uint64_t *bar;
    __device__ __forceinline__ void arm(int bi, uint32_t bytes) const { mbar_arm(&bar[bi], bytes); }
    __device__ __forceinline__ void copy(int dst, int array, int off, int, uint32_t bytes, int bi) const {
        bulk_load(smem + dst, src[array] + off, bytes, &bar[bi]);
    }
};

// ------------------------------------------------------------------------------------------------------------
// FP32 half-sweep with the other colour's planes staged in shared memory by bulk copies (block edge n = 2^LG,
// colour-split pools with H = half_row(P)).
//
// A CTA owns block b, interior rows y0 .. y0 + TY - 1 and planes z0 .. z0 + TZ - 1 and marches in z.  Thread (j, yl)
// updates the cells at position j + C of rows y0 + yl + i TW (i < R, TW = TY / R) in every plane, where
// C = (y + z + colour) & 1.  TY, TW and z0 are even, so C is the same for all rows of a thread, and lanes are mapped
// to rows so that it is the same for every lane of a warp: a warp covers one row (n >= 64) or two rows two apart
// (n = 32).  Each plane then runs one of two bodies with C a compile-time constant, without per-cell selects.
//
// Per plane z the CTA needs, of the other half, rows y0 - 1 .. y0 + TY of planes z - 1, z, z + 1 (u, and kappa for
// variable k) and, of its own half, rows y0 .. y0 + TY - 1 of plane z (f, and kappa).  Each plane segment is one
// contiguous run of (TY + 2) H or TY H floats, fetched by one bulk copy.  The other half's planes z0 - 1 and z0 come
// first, on barrier 0; after that, group g = {other plane z0 + g + 1, own plane z0 + g} completes on one of D + 1
// "full" group barriers, so each plane costs one wait.  Groups run D + 1 planes ahead of the plane being updated, in
// rings of D + 2 (other half) and D + 1 (own half) slots.  The copies are issued by one thread of an extra producer
// warp (the CTA's last): group g reuses the slots of group g - D - 1, and the producer issues it once every consumer
// warp has arrived on that group's "empty" barrier (lane 0, after the warp's last read of the slots); group D reuses
// the slot of plane z0 - 1 and waits for every warp to have moved that plane into registers.  Consumer warps are
// never synchronised with each other: a warp runs ahead until it needs a group that has not landed.
//
// Per cell the thread reads from shared memory its x-neighbour pair of plane z + 1 (positions j, j + 1 of row yl + 1;
// the pair of plane z was read one plane earlier and gives the x-neighbours now, that of plane z - 1 the z-minus
// neighbour at position C), its y-neighbours (rows yl and yl + 2 at j + C) and its own f and kappa: 4 + 4 + 2 shared
// loads instead of 14.  New values go straight to global memory (the own half is not staged).  Write-through of
// block-face cells as in k_smooth32, with the target of every face this thread can touch resolved before the
// march: the x face of lanes j = 0 (side 0, cells with C = 0) and j = n/2 - 1 (side 1, C = 1), the y face of the
// thread's row y = 0 or n - 1, and the z faces of planes 0 and n - 1 (uniform over the CTA).  No staged value is
// written during the sweep except reflection ghosts, which only the writing cell reads, before it writes.
//
// Every wait is bounded.  A consumer warp whose wait runs out (its lanes agree by a vote) sets *err and stops; the
// producer stops when an empty barrier is not reached in time, sets *err, and before it exits waits, again bounded,
// for the copies it issued, so no copy lands in released shared memory.
// ------------------------------------------------------------------------------------------------------------
template <int MODE, int LG, int R>
static __global__ void __launch_bounds__(544) k_smooth32t(float *__restrict__ u, const float *__restrict__ f,
                                                          const float *__restrict__ kap, const float *__restrict__ h2,
                                                          int64_t bs, int colour, const int32_t *__restrict__ nbr6,
                                                          int TY, int TZ, int D, int *__restrict__ err, Skip skip,
                                                          const float *__restrict__ ax, const float *__restrict__ ay,
                                                          const float *__restrict__ az) {
    static_assert(MODE == 0 || MODE == 2 || MODE == 3, "coefficient modes 0, 2, 3");
    constexpr int n = 1 << LG, NH = n / 2, P = n + 2, H = half_row(P), PL = P * H, HALF = P * PL;
    constexpr int NA = s32t_arrays(MODE);  // staged arrays per half
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const S32tPlan plan = s32t_plan(LG, NA, TY, D);
    const int RO = plan.RO, RW = plan.RW, G = plan.G;
    const int so = plan.so, sw = plan.sw;
    // other-half slot i: u at ou + i NA so, then kappa (MODE 2) or ax, ay, az (MODE 3) so floats apart; own-half
    // slot i: f at wf + i NA sw, then kappa or ax, ay, az sw floats apart
    float *ou = reinterpret_cast<float *>(smem_raw);
    float *wf = ou + s32t_own_slot(plan, 0);
    // full barriers: bar[0] planes z0 - 1, z0; bar[1 + g % G] group g.  Empty barriers (all consumer warps are done
    // with the slots): ebar[g % G] group g, ibar planes z0 - 1, z0 moved into registers
    uint64_t *bar = reinterpret_cast<uint64_t *>(ou + s32t_bar_floats(plan));
    uint64_t *ebar = bar + 1 + G, *ibar = ebar + G;

    // the second colour walks the tiles in reverse: it starts where the first colour's launch ended, on the blocks
    // whose u and 1/k that launch left in L2 (the updates of one colour are independent, so the order changes nothing)
    const unsigned bid = colour ? gridDim.x - 1 - blockIdx.x : blockIdx.x;
    const int nty = n / TY;
    const int ty = static_cast<int>(bid % nty);
    const int64_t rest = bid / nty;
    const int tz = static_cast<int>(rest % (n / TZ));
    const int64_t b = rest / (n / TZ);
    if (skip(b)) return;  // uniform over the CTA, before any barrier
    const int y0 = ty * TY, z0 = tz * TZ;
    const int s = colour ^ 1;
    const int tid = threadIdx.x;
    const int TW = TY / R;
    const int j = tid & (NH - 1);
    int yl0 = tid >> (LG - 1);
    if constexpr (NH < 32) yl0 = (yl0 & ~3) | ((yl0 & 1) << 1) | ((yl0 >> 1) & 1);  // a warp's two rows: same parity
    const int64_t base = b * bs;
    // the block's halves of the staged arrays, numbered as in s32t_other_array / s32t_own_array
    const float *c1 = MODE == 3 ? ax : kap;
    const int64_t ho = base + (s ^ 1) * HALF, hw = base + s * HALF;

    const auto off_o = [&](int Zp) { return s32t_off_other(plan, Zp, y0); };
    const auto off_w = [&](int Zp) { return s32t_off_own(plan, Zp, y0); };
    // the producer's copies, as planned by s32t_issue_first / s32t_issue_group
    const S32tDeviceSink sink{ou,
                              {u + ho, MODE ? c1 + ho : nullptr, f + hw, MODE ? c1 + hw : nullptr,
                               MODE == 3 ? ay + ho : nullptr, MODE == 3 ? az + ho : nullptr,
                               MODE == 3 ? ay + hw : nullptr, MODE == 3 ? az + hw : nullptr},
                              bar};
    const auto issue_first = [&]() { s32t_issue_first(plan, z0, y0, sink); };
    const auto issue_group = [&](int g) { s32t_issue_group(plan, z0, y0, g, sink); };
    const int nthc = blockDim.x - 32, ncw = nthc >> 5;  // consumer threads and warps; the last warp produces
    if (tid == 0) {
        for (int i = 0; i < 1 + G; ++i) mbar_init(&bar[i], 1);
        for (int i = 0; i < G + 1; ++i) mbar_init(&ebar[i], ncw);
        mbar_init_fence();
    }
    __syncthreads();
    if (tid >= nthc) {
        if (tid == nthc) {
            // group g reuses the slots of group g - G (other half: the plane that was `oc` at plane g - G); group
            // G - 1 the slot of plane z0 - 1
            issue_first();
            int g = 0;
            for (; g < G - 1 && g < TZ; ++g) issue_group(g);
            bool ok = true;
            while (g < TZ) {
                ok = g == G - 1 ? mbar_wait(ibar, 0) : mbar_wait(&ebar[(g - G) % G], ((g - G) / G) & 1);
                if (!ok) break;
                issue_group(g++);
            }
            if (!ok) atomicOr(err, 1);
            // the copies still in flight land before the CTA's shared memory can be released
            mbar_wait(&bar[0], 0);
            for (int q = g > G ? g - G : 0; q < g; ++q) mbar_wait(&bar[1 + q % G], (q / G) & 1);
        }
        return;
    }
    const float hb = __ldg(h2 + b), hh = 0.5f * hb;

    // write-through targets, as pointers p with the target of the cell at index q (in its half) at p[q]
    float *us = u + base + s * HALF;
    float *xw = nullptr, *yw = nullptr, *zlo = nullptr, *zhi = nullptr;
    float xsg = 1.f, ysg = 1.f, zlsg = 1.f, zhsg = 1.f;
    const int xs = j == 0 ? 0 : 1;  // x face side of lanes j = 0 and j = n/2 - 1
    int yr = -1;                    // which of the thread's rows lies on a y face
    if (nbr6) {
        const auto target = [&](int q6, int nb_off, int refl_off, float *&p, float &sg) {
            const int nbv = __ldg(nbr6 + b * 6 + q6);
            if (nbv >= 0) p = u + nbv * bs + s * HALF + nb_off;
            else if (nbv == -1) { p = u + base + (s ^ 1) * HALF + refl_off; sg = -1.f; }
        };
        if (j == 0 || j == NH - 1) target(xs, xs ? -NH : NH, 0, xw, xsg);
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
            const int y = y0 + yl0 + rr * TW;
            if (y == 0) { target(2, n * H, -H, yw, ysg); yr = rr; }
            if (y == n - 1) { target(3, -n * H, H, yw, ysg); yr = rr; }
        }
        if (!yw) yr = -1;
        if (z0 == 0) target(4, n * PL, -PL, zlo, zlsg);
        if (z0 + TZ == n) target(5, -n * PL, PL, zhi, zhsg);
    }

    int bad = __any_sync(0xffffffffu, !mbar_wait(&bar[0], 0));
    const int cpar = (yl0 + colour) & 1;  // C of plane z0 (y0, TW and z0 are even)
    const int ro0 = (yl0 + 1) * H + j, rstep = TW * H;  // row yl + 1 of an other-half slot, position j
    const int qo0 = ((z0 + 1) * P + y0 + yl0 + 1) * H + j, qstep = TW * H;  // the cell at plane z0, C = 0
    float pc[R][2], qc[R][2], zmu[R], zmk[R];  // x-neighbour pair of the current plane, z-minus neighbour (u, kappa)
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
        const int ro = ro0 + rr * rstep;
        const int e0 = off_o(z0) & 3, e1 = off_o(z0 + 1) & 3;  // slot offsets of planes z0 - 1 and z0
        zmu[rr] = ou[e0 + ro + cpar];
        pc[rr][0] = ou[NA * so + e1 + ro];
        pc[rr][1] = ou[NA * so + e1 + ro + 1];
        if constexpr (MODE == 2) {
            zmk[rr] = ou[so + e0 + ro + cpar];
            qc[rr][0] = ou[NA * so + so + e1 + ro];
            qc[rr][1] = ou[NA * so + so + e1 + ro + 1];
        } else {
            zmk[rr] = qc[rr][0] = qc[rr][1] = 0.f;
        }
    }
    // Slot 0 (plane z0 - 1) is refilled by a bulk copy once every warp has arrived on ibar, but its values are only
    // used at the first plane, so nothing forces these loads to have read shared memory by the time of the arrival:
    // without this fence the copy was seen to overwrite the slot under them (the z-minus 1/k of a warp's rows came
    // from plane z0 + D + 1, mostly when other kernels shared the SMs).  The proxy fence orders this thread's
    // generic-proxy reads of the slot before the async-proxy writes that follow the arrival.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(ibar);
    // ring positions: other-half slots of planes z + 1 and z, own-half slot and group barrier of plane z
    int on_s = 2 % RO, oc_s = 1, w_s = 0, g_s = 0, g_ph = 0;
    if (!bad) {
        for (int k = 0; k < TZ; ++k) {
            bad = __any_sync(0xffffffffu, !mbar_wait(&bar[1 + g_s], g_ph));
            if (bad) break;
            const float *on = ou + on_s * NA * so + (off_o(z0 + k + 2) & 3);
            const float *oc = ou + oc_s * NA * so + (off_o(z0 + k + 1) & 3);
            const float *fw = wf + w_s * NA * sw + (off_w(z0 + k + 1) & 3);
            const float *kn = on + so, *kc = oc + so, *kw = fw + sw;
            const int z = z0 + k;
            float *zw = z == 0 ? zlo : (z == n - 1 ? zhi : nullptr);
            const float zsg = z == 0 ? zlsg : zhsg;
            const int qz = qo0 + k * PL;
            const auto plane = [&](auto Cc) {
                constexpr int C = decltype(Cc)::value;
                float pn0[R], pn1[R], val[R];
                [[maybe_unused]] float qn0[R], qn1[R];  // kappa pair of plane z + 1 (MODE 2)
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const int ro = ro0 + rr * rstep;
                    pn0[rr] = on[ro];
                    pn1[rr] = on[ro + 1];
                    if constexpr (MODE == 2) {
                        qn0[rr] = kn[ro];
                        qn1[rr] = kn[ro + 1];
                    }
                }
                // rows in pairs on the paired FP32 instructions (each component rounds as the scalar operation, in
                // the same order as the column smoother), an odd last row alone
#pragma unroll
                for (int rr = 0; rr + 1 < R; rr += 2) {
                    const int ra = ro0 + rr * rstep, rb = ra + rstep;
                    const float2 ym{oc[ra - H + C], oc[rb - H + C]}, yp{oc[ra + H + C], oc[rb + H + C]};
                    const float2 fv{fw[ra - H + C], fw[rb - H + C]};
                    const float2 x0{pc[rr][0], pc[rr + 1][0]}, x1{pc[rr][1], pc[rr + 1][1]};
                    const float2 zm{zmu[rr], zmu[rr + 1]};
                    const float2 zp = C ? float2{pn1[rr], pn1[rr + 1]} : float2{pn0[rr], pn0[rr + 1]};
                    float2 v;
                    if constexpr (MODE == 2) {
                        const float2 kym{kc[ra - H + C], kc[rb - H + C]}, kyp{kc[ra + H + C], kc[rb + H + C]};
                        const float2 k0{kw[ra - H + C], kw[rb - H + C]};
                        const float2 kzp = C ? float2{qn1[rr], qn1[rr + 1]} : float2{qn0[rr], qn0[rr + 1]};
                        const float2 a0 = frcp2(__fadd2_rn(k0, float2{qc[rr][0], qc[rr + 1][0]}));
                        const float2 a1 = frcp2(__fadd2_rn(k0, float2{qc[rr][1], qc[rr + 1][1]}));
                        const float2 b0 = frcp2(__fadd2_rn(k0, kym)), b1 = frcp2(__fadd2_rn(k0, kyp));
                        const float2 e0 = frcp2(__fadd2_rn(k0, float2{zmk[rr], zmk[rr + 1]}));
                        const float2 e1 = frcp2(__fadd2_rn(k0, kzp));
                        float2 sacc = __fmul2_rn(a0, x0);
                        sacc = __ffma2_rn(a1, x1, sacc);
                        sacc = __ffma2_rn(b0, ym, sacc);
                        sacc = __ffma2_rn(b1, yp, sacc);
                        sacc = __ffma2_rn(e0, zm, sacc);
                        sacc = __ffma2_rn(e1, zp, sacc);
                        const float2 Dn =
                            __fadd2_rn(__fadd2_rn(__fadd2_rn(a0, a1), __fadd2_rn(b0, b1)), __fadd2_rn(e0, e1));
                        v = __fmul2_rn(__ffma2_rn(float2{hh, hh}, fv, sacc), frcp2(Dn));
                    } else if constexpr (MODE == 3) {
                        // stored halved faces: the lower ones at the cell (own slot), the upper ones at the x+ and
                        // y+ neighbours of this plane and the z+ neighbour of the next (other slots)
                        const int wa = ra - H + C, wb = rb - H + C;
                        const float2 a0{fw[sw + wa], fw[sw + wb]}, b0{fw[2 * sw + wa], fw[2 * sw + wb]};
                        const float2 e0{fw[3 * sw + wa], fw[3 * sw + wb]};
                        const float2 a1{oc[so + ra + 1], oc[so + rb + 1]};
                        const float2 b1{oc[2 * so + ra + H + C], oc[2 * so + rb + H + C]};
                        const float2 e1{on[3 * so + ra + C], on[3 * so + rb + C]};
                        float2 sacc = __fmul2_rn(a0, x0);
                        sacc = __ffma2_rn(a1, x1, sacc);
                        sacc = __ffma2_rn(b0, ym, sacc);
                        sacc = __ffma2_rn(b1, yp, sacc);
                        sacc = __ffma2_rn(e0, zm, sacc);
                        sacc = __ffma2_rn(e1, zp, sacc);
                        const float2 Dn =
                            __fadd2_rn(__fadd2_rn(__fadd2_rn(a0, a1), __fadd2_rn(b0, b1)), __fadd2_rn(e0, e1));
                        v = __fmul2_rn(__ffma2_rn(float2{hh, hh}, fv, sacc), frcp2(Dn));
                    } else {
                        const float2 S = __fadd2_rn(__fadd2_rn(__fadd2_rn(x0, x1), __fadd2_rn(ym, yp)), __fadd2_rn(zm, zp));
                        v = div6x2(__ffma2_rn(float2{hb, hb}, fv, S));
                    }
                    val[rr] = v.x;
                    val[rr + 1] = v.y;
                }
                if constexpr (R & 1) {
                    constexpr int rr = R - 1;
                    const int ro = ro0 + rr * rstep;
                    const float ym = oc[ro - H + C], yp = oc[ro + H + C];
                    const float fv = fw[ro - H + C];
                    const float zp = C ? pn1[rr] : pn0[rr];
                    if constexpr (MODE == 2) {
                        const float kym = kc[ro - H + C], kyp = kc[ro + H + C];
                        const float k0 = kw[ro - H + C];
                        const float kzp = C ? qn1[rr] : qn0[rr];
                        const float a0 = frcp(k0 + qc[rr][0]), a1 = frcp(k0 + qc[rr][1]);
                        const float b0 = frcp(k0 + kym), b1 = frcp(k0 + kyp);
                        const float e0 = frcp(k0 + zmk[rr]), e1 = frcp(k0 + kzp);
                        float sacc = a0 * pc[rr][0];
                        sacc = fmaf(a1, pc[rr][1], sacc);
                        sacc = fmaf(b0, ym, sacc);
                        sacc = fmaf(b1, yp, sacc);
                        sacc = fmaf(e0, zmu[rr], sacc);
                        sacc = fmaf(e1, zp, sacc);
                        const float Dn = ((a0 + a1) + (b0 + b1)) + (e0 + e1);
                        val[rr] = fmaf(hh, fv, sacc) * frcp(Dn);
                    } else if constexpr (MODE == 3) {
                        const int w = ro - H + C;
                        const float a0 = fw[sw + w], a1 = oc[so + ro + 1];
                        const float b0 = fw[2 * sw + w], b1 = oc[2 * so + ro + H + C];
                        const float e0 = fw[3 * sw + w], e1 = on[3 * so + ro + C];
                        float sacc = a0 * pc[rr][0];
                        sacc = fmaf(a1, pc[rr][1], sacc);
                        sacc = fmaf(b0, ym, sacc);
                        sacc = fmaf(b1, yp, sacc);
                        sacc = fmaf(e0, zmu[rr], sacc);
                        sacc = fmaf(e1, zp, sacc);
                        const float Dn = ((a0 + a1) + (b0 + b1)) + (e0 + e1);
                        val[rr] = fmaf(hh, fv, sacc) * frcp(Dn);
                    } else {
                        const float S = ((pc[rr][0] + pc[rr][1]) + (ym + yp)) + (zmu[rr] + zp);
                        val[rr] = div6(fmaf(hb, fv, S));
                    }
                }
#pragma unroll
                for (int rr = 0; rr < R; ++rr) {
                    const int q = qz + rr * qstep + C;
                    us[q] = val[rr];
                    if (xs == C && xw) xw[q] = xsg * val[rr];
                    if (yr == rr) yw[q] = ysg * val[rr];
                    if (zw) zw[q] = zsg * val[rr];
                    zmu[rr] = pc[rr][1 - C];
                    pc[rr][0] = pn0[rr];
                    pc[rr][1] = pn1[rr];
                    if constexpr (MODE == 2) {
                        zmk[rr] = qc[rr][1 - C];
                        qc[rr][0] = qn0[rr];
                        qc[rr][1] = qn1[rr];
                    }
                }
            };
            if ((cpar + k) & 1) plane(std::integral_constant<int, 1>{});
            else plane(std::integral_constant<int, 0>{});
            // this warp is done with the slots of group k and other-half plane z: group k + G may refill them.  Every
            // value read from those slots fed an update stored above, and the release arrival orders the stores (and
            // so the reads they needed) before the refill; the first planes' slot 0 is the case that needs a fence
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(&ebar[g_s]);
            oc_s = on_s;
            if (++on_s == RO) on_s = 0;
            if (++w_s == RW) w_s = 0;
            if (++g_s == G) { g_s = 0; g_ph ^= 1; }
        }
    }
    if (bad && (tid & 31) == 0) atomicOr(err, 1);
}

// Point-form residual at padded cell (X, Y, Z) of block b, any layout (used by the FP32 kernels).
template <typename T, int MODE, bool CG = false>
__device__ inline T residual_xyz(const T *__restrict__ u, const T *__restrict__ f, const Coef &cf,
                                 const LevelGeom &g, int64_t b, int X, int Y, int Z, T ih2) {
    const int64_t i0 = Lay<T>::at(g, b, X, Y, Z);
    const int64_t nb[6] = {Lay<T>::at(g, b, X - 1, Y, Z), Lay<T>::at(g, b, X + 1, Y, Z),
                           Lay<T>::at(g, b, X, Y - 1, Z), Lay<T>::at(g, b, X, Y + 1, Z),
                           Lay<T>::at(g, b, X, Y, Z - 1), Lay<T>::at(g, b, X, Y, Z + 1)};
    const T u0 = ldv<CG>(u + i0);
    if constexpr (MODE == 0) {
        const T S = ((ldv<CG>(u + nb[0]) + ldv<CG>(u + nb[1])) + (ldv<CG>(u + nb[2]) + ldv<CG>(u + nb[3]))) +
                    (ldv<CG>(u + nb[4]) + ldv<CG>(u + nb[5]));
        return fma(fma(T(-6), u0, S), ih2, ldv<CG>(f + i0));
    } else {
        float S = 0.0f, D = 0.0f;
        if constexpr (MODE == 3) {  // stored halved face coefficients: lower faces at the cell, upper at the neighbour
            const float a6[6] = {cf.ax[i0], cf.ax[nb[1]], cf.ay[i0], cf.ay[nb[3]], cf.az[i0], cf.az[nb[5]]};
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                S = fmaf(a6[q], float(ldv<CG>(u + nb[q])), S);
                D += a6[q];
            }
        } else {
            const float k0 = cf.kap[i0];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float a = frcp(k0 + cf.kap[nb[q]]);
                S = fmaf(a, float(ldv<CG>(u + nb[q])), S);
                D += a;
            }
        }
        return T(fmaf(2.0f * fmaf(-D, float(u0), S), float(ih2), float(ldv<CG>(f + i0))));
    }
}

// ------------------------------------------------------------------------------------------------------------
// Residual of the fine level restricted to the next level (mean of the 8 children), written as the coarse
// right-hand side; the coarse solution's interior is zeroed (coarse-grid correction starts from 0).
// One thread per coarse cell.  ih2f: 1/h^2 per fine block.
// ------------------------------------------------------------------------------------------------------------
template <typename T, int MODE, bool CG = false>
__device__ __forceinline__ void residual_restrict_body(const T *__restrict__ u, const T *__restrict__ f, Coef cf,
                                                       const T *__restrict__ ih2f, LevelGeom gf, T *__restrict__ fc,
                                                       T *__restrict__ uc, const XferItem *__restrict__ xf,
                                                       LevelGeom gc, Skip skip, int64_t t0, int64_t ts) {
    const int lgc = gc.lg, nc = gc.n;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    for (int64_t t = t0; t < total; t += ts) {
        const int X = static_cast<int>(t & (nc - 1));
        const int Y = static_cast<int>((t >> lgc) & (nc - 1));
        const int Z = static_cast<int>((t >> (2 * lgc)) & (nc - 1));
        const int64_t B = t >> (3 * lgc);
        if (skip(B)) continue;
        const XferItem xi = xf[B];
        const int64_t gcell = Lay<T>::at(gc, B, X + 1, Y + 1, Z + 1);
        uc[gcell] = T(0);
        const auto res = [&](int64_t bb, int xx, int yy, int zz, T ih2) {
            if constexpr (sizeof(T) == 4)
                return residual_xyz<T, MODE, CG>(u, f, cf, gf, bb, xx, yy, zz, ih2);
            else
                return residual_at<T, MODE>(u, f, cf, bb * gf.bs + off3(xx, yy, zz, gf.P), gf.P, ih2);
        };
        if (xi.kind == XF_COPY) {
            const int64_t b = xi.src[0];
            fc[gcell] = res(b, X + 1, Y + 1, Z + 1, ih2f[b]);
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
                for (int a = 0; a < 2; ++a) s += res(b, x0 + a + 1, y0 + bb + 1, z0 + c + 1, ih2);
        fc[gcell] = T(0.125) * s;
    }
}

// Residual r = f - A u (Sec. 5, Eq. 1) restricted 8:1 to the coarse right-hand side (mean of the 8 children, the
// block-local coarsening of Sec. 5), coarse correction zeroed.
template <typename T, int MODE>
static __global__ void k_residual_restrict(const T *__restrict__ u, const T *__restrict__ f, Coef cf,
                                           const T *__restrict__ ih2f, LevelGeom gf, T *__restrict__ fc,
                                           T *__restrict__ uc, const XferItem *__restrict__ xf, LevelGeom gc,
                                           Skip skip = Skip{}) {
    residual_restrict_body<T, MODE>(u, f, cf, ih2f, gf, fc, uc, xf, gc, skip,
                                    blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x,
                                    static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// ------------------------------------------------------------------------------------------------------------
// FP32 residual + restriction for a level whose blocks all halve (fine edge n = 2^LG, coarse n/2), colour-split
// pools on both sides.  One thread per coarse cell (X, Y, Z): its 8 children are the fine padded cells
// (2X + i, 2Y + j, 2Z + k), i, j, k in {1, 2}, and the 32 distinct values of u (and of kappa) their 7-point stencils
// touch lie in the 4^3 box i, j, k in {0..3} without its edges.  In the split layout box cell (i, j, k) sits at
//     ((i + j + k) & 1) * HALF + (k P + j) H + (i >> 1),   H = half_row(P),
// from the box's corner offset ((2Z P + 2Y) H + X), so every load is an immediate offset from one pointer; the
// interior faces of the box are shared by two children and their coefficients are evaluated once.
// ------------------------------------------------------------------------------------------------------------
template <int LG>
struct Box32 {
    static constexpr int n = 1 << LG, P = n + 2, HP = half_row(P), HALF = P * P * HP;
    __device__ static constexpr int off(int i, int j, int k) {
        return ((i + j + k) & 1) * HALF + (k * P + j) * HP + (i >> 1);
    }
};

// The sum of the 8 children's residuals from the box values (U, and K for MODE 2, AX / AY / AZ for MODE 3, as
// loaded by residual_restrict32_body or staged by k_residual_restrict32t) and f of child (i, j, k) from fv(i, j, k),
// children in (k, j, i) order, so both kernels give the same bits.
template <int MODE, class FV>
__device__ __forceinline__ float rr32_sum(const float (&U)[4][4][4], const float (&K)[4][4][4],
                                          const float (&AX)[3][3][4], const float (&AY)[3][4][3],
                                          const float (&AZ)[4][3][3], float ih2, FV &&fv_at) {
    float sum = 0.0f;
#pragma unroll
    for (int k = 1; k < 3; ++k)
#pragma unroll
        for (int j = 1; j < 3; ++j)
#pragma unroll
            for (int i = 1; i < 3; ++i) {
                const float u0 = U[k][j][i];
                const float fv = fv_at(i, j, k);
                const float nbu[6] = {U[k][j][i - 1], U[k][j][i + 1], U[k][j - 1][i],
                                      U[k][j + 1][i], U[k - 1][j][i], U[k + 1][j][i]};
                if constexpr (MODE == 0) {
                    const float S = ((nbu[0] + nbu[1]) + (nbu[2] + nbu[3])) + (nbu[4] + nbu[5]);
                    sum += fmaf(fmaf(-6.0f, u0, S), ih2, fv);
                } else if constexpr (MODE == 3) {
                    const float a6[6] = {AX[k][j][i], AX[k][j][i + 1], AY[k][j][i],
                                         AY[k][j + 1][i], AZ[k][j][i], AZ[k + 1][j][i]};
                    float S = 0.0f, D = 0.0f;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        S = fmaf(a6[q], nbu[q], S);
                        D += a6[q];
                    }
                    sum += fmaf(2.0f * fmaf(-D, u0, S), ih2, fv);
                } else {
                    const float k0 = K[k][j][i];
                    const float nbk[6] = {K[k][j][i - 1], K[k][j][i + 1], K[k][j - 1][i],
                                          K[k][j + 1][i], K[k - 1][j][i], K[k + 1][j][i]};
                    float S = 0.0f, D = 0.0f;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        // operands in a fixed order per face (the lower neighbour first), so the two children
                        // of an interior face evaluate the same expression and it is computed once; the sum
                        // is the same either way
                        const float a = (q & 1) ? frcp(k0 + nbk[q]) : frcp(nbk[q] + k0);
                        S = fmaf(a, nbu[q], S);
                        D += a;
                    }
                    sum += fmaf(2.0f * fmaf(-D, u0, S), ih2, fv);
                }
            }
    return sum;
}

// The coarse right-hand side (1/8 of the children's residual sum) and a zero coarse correction, with its face
// ghosts, at coarse cell (X, Y, Z) of coarse block B (coarse edge nc, colour-split pool).
template <int LG>
__device__ __forceinline__ void rr32_store(float *__restrict__ fc, float *__restrict__ uc, int64_t B, int64_t bsc,
                                           int X, int Y, int Z, float sum) {
    constexpr int nc = (1 << LG) / 2, Pc = nc + 2, HPc = half_row(Pc), HALFc = Pc * Pc * HPc;
    const int Xc = X + 1, Yc = Y + 1, Zc = Z + 1;
    const auto at = [&](int xx, int yy, int zz) {
        return B * bsc + ((xx + yy + zz) & 1) * HALFc + (zz * Pc + yy) * HPc + (xx >> 1);
    };
    const int64_t gc = at(Xc, Yc, Zc);
    fc[gc] = 0.125f * sum;
    uc[gc] = 0.0f;
    // the coarse correction starts from zero: its face ghosts are zero too, so the level needs no exchange
    // before its first half-sweep
    if (X == 0) uc[at(0, Yc, Zc)] = 0.0f;
    if (X == nc - 1) uc[at(nc + 1, Yc, Zc)] = 0.0f;
    if (Y == 0) uc[at(Xc, 0, Zc)] = 0.0f;
    if (Y == nc - 1) uc[at(Xc, nc + 1, Zc)] = 0.0f;
    if (Z == 0) uc[at(Xc, Yc, 0)] = 0.0f;
    if (Z == nc - 1) uc[at(Xc, Yc, nc + 1)] = 0.0f;
}

template <int MODE, int LG, bool CG = false>
__device__ __forceinline__ void residual_restrict32_body(
        const float *__restrict__ u, const float *__restrict__ f, const float *__restrict__ kap,
        const float *__restrict__ ih2f, int64_t bsf, float *__restrict__ fc, float *__restrict__ uc,
        const XferItem *__restrict__ xf, int32_t nbc, int64_t bsc, Skip skip, int64_t t0, int64_t ts,
        const float *__restrict__ ax = nullptr, const float *__restrict__ ay = nullptr,
        const float *__restrict__ az = nullptr) {
    using Bx = Box32<LG>;
    constexpr int nc = (1 << LG) / 2, LC = LG - 1;
    const int64_t total = static_cast<int64_t>(nbc) << (3 * LC);
    for (int64_t t = t0; t < total; t += ts) {
        const int r = static_cast<int>(t) & ((1 << (3 * LC)) - 1);
        const int64_t B = t >> (3 * LC);
        if (skip(B)) continue;  // the coarse level's problem ids
        const int X = r & (nc - 1), Y = (r >> LC) & (nc - 1), Z = r >> (2 * LC);
        const int64_t b = xf[B].src[0];
        const int64_t corner = b * bsf + (2 * Z * Bx::P + 2 * Y) * Bx::HP + X;
        const float *ub = u + corner;
        float U[4][4][4], K[4][4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int out = (i == 0 || i == 3) + (j == 0 || j == 3) + (k == 0 || k == 3);
                    if (out > 1) continue;
                    U[k][j][i] = ldv<CG>(ub + Bx::off(i, j, k));
                    if constexpr (MODE == 2) K[k][j][i] = __ldg(kap + corner + Bx::off(i, j, k));
                }
        // MODE 3: the children's halved face coefficients, a face stored at the cell on its upper side
        float AX[3][3][4], AY[3][4][3], AZ[4][3][3];
        if constexpr (MODE == 3) {
#pragma unroll
            for (int k = 1; k < 3; ++k)
#pragma unroll
                for (int j = 1; j < 3; ++j)
#pragma unroll
                    for (int i = 1; i < 4; ++i) {
                        AX[k][j][i] = __ldg(ax + corner + Bx::off(i, j, k));
                        AY[k][i][j] = __ldg(ay + corner + Bx::off(j, i, k));
                        AZ[i][k][j] = __ldg(az + corner + Bx::off(j, k, i));
                    }
        }
        const float ih2 = __ldg(ih2f + b);
        const float sum = rr32_sum<MODE>(U, K, AX, AY, AZ, ih2, [&](int i, int j, int k) {
            return ldr<CG>(f + corner + Bx::off(i, j, k));
        });
        rr32_store<LG>(fc, uc, B, bsc, X, Y, Z, sum);
    }
}

template <int MODE, int LG>
static __global__ void __launch_bounds__(256) k_residual_restrict32(
        const float *__restrict__ u, const float *__restrict__ f, const float *__restrict__ kap,
        const float *__restrict__ ih2f, int64_t bsf, float *__restrict__ fc, float *__restrict__ uc,
        const XferItem *__restrict__ xf, int32_t nbc, int64_t bsc, Skip skip, const float *__restrict__ ax,
        const float *__restrict__ ay, const float *__restrict__ az) {
    residual_restrict32_body<MODE, LG>(u, f, kap, ih2f, bsf, fc, uc, xf, nbc, bsc, skip,
                                       blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x,
                                       static_cast<int64_t>(gridDim.x) * blockDim.x, ax, ay, az);
}

// ------------------------------------------------------------------------------------------------------------
// Copy plan of the staged residual + restriction below (k_residual_restrict32t), shared by the kernel's producer
// thread, the launch code and the host-side enumerator that checks every copy against the bulk-copy rules.
//
// A CTA owns fine block b, interior rows y0 .. y0 + TY - 1 and planes z0 .. z0 + TZ - 1 (TY, TZ, y0, z0 even): the
// coarse cells of TY / 2 coarse rows and TZ / 2 coarse planes.  It stages the fine padded planes z0 .. z0 + TZ + 1
// (q = 0 .. TZ + 1 relative to z0), one by one, into a ring of RS = 4 + 2 D plane slots.  A slot holds, of both
// halves, the segment of padded rows y0 .. y0 + TY + 1 of each of the NU arrays the residual reads around a cell (u;
// u and kappa; u, ax, ay, az) and, for q = 1 .. TZ, the segment of rows y0 + 1 .. y0 + TY of f; each widened to
// 16-byte bounds as in the staged smoother (a segment never ends past its half: the half length is a multiple of 4
// floats).  Coarse plane step g reads planes 2g .. 2g + 3 and then releases planes 2g and 2g + 1; plane q reuses the
// slot of plane q - RS once that plane is released, and the planes a step reads are RS-consecutive or fewer, so they
// sit in distinct slots.  Shared memory: RS slots of ss floats, then RS "full" and RS "empty" mbarriers.
// ------------------------------------------------------------------------------------------------------------
struct R32tPlan {
    int P, H, NU, RS, TZ;
    int lo, lw, so, sw, ss;  // segment lengths, segment strides and the slot stride (floats)
};
__host__ __device__ __forceinline__ R32tPlan r32t_plan(int lg, int mode, int TY, int TZ, int D) {
    R32tPlan p;
    p.P = (1 << lg) + 2;
    p.H = half_row(p.P);
    p.NU = mode == 3 ? 4 : (mode == 2 ? 2 : 1);
    p.RS = 4 + 2 * D;
    p.TZ = TZ;
    p.lo = (TY + 2) * p.H;
    p.lw = TY * p.H;
    p.so = (p.lo + 6) & ~3;
    p.sw = (p.lw + 6) & ~3;
    p.ss = 2 * p.NU * p.so + 2 * p.sw;
    return p;
}
__host__ __device__ __forceinline__ size_t r32t_smem_bytes(const R32tPlan &p) {
    return static_cast<size_t>(4) * p.RS * p.ss + static_cast<size_t>(8) * 2 * p.RS;
}
// start (floats, within a half) of padded plane Zp's segment of the stencil arrays and of f
__host__ __device__ __forceinline__ int r32t_off_lo(const R32tPlan &p, int Zp, int y0) { return (Zp * p.P + y0) * p.H; }
__host__ __device__ __forceinline__ int r32t_off_f(const R32tPlan &p, int Zp, int y0) { return (Zp * p.P + y0 + 1) * p.H; }
// shared float offset, within its slot, of array a's (a = NU: f's) segment of half h
__host__ __device__ __forceinline__ int r32t_seg(const R32tPlan &p, int a, int h) {
    return a < p.NU ? (2 * a + h) * p.so : 2 * p.NU * p.so + h * p.sw;
}
// The copies of plane q of one CTA: sink.arm(slot, bytes) arms the slot's full barrier with the bytes that complete
// it; sink.copy(dst, array, half, src, lead, bytes, slot) copies `bytes` from float `src` of half `half` of `array`
// (0 .. NU - 1: u, then kappa or ax, ay, az; NU: f) to shared float `dst`, the wanted segment `lead` floats in.
#pragma nv_exec_check_disable
template <class Sink>
__host__ __device__ __forceinline__ void r32t_issue_plane(const R32tPlan &p, int z0, int y0, int q, Sink &&sink) {
    const int slot = q % p.RS, base = slot * p.ss;
    const int ol = r32t_off_lo(p, z0 + q, y0), of = r32t_off_f(p, z0 + q, y0);
    const uint32_t bl = s32t_bytes(ol, p.lo), bf = s32t_bytes(of, p.lw);
    const bool withf = q >= 1 && q <= p.TZ;
    sink.arm(slot, 2 * p.NU * bl + (withf ? 2 * bf : 0));
    for (int a = 0; a < p.NU; ++a)
        for (int h = 0; h < 2; ++h) sink.copy(base + r32t_seg(p, a, h), a, h, ol & ~3, ol & 3, bl, slot);
    if (withf)
        for (int h = 0; h < 2; ++h) sink.copy(base + r32t_seg(p, p.NU, h), p.NU, h, of & ~3, of & 3, bf, slot);
}
struct R32tDeviceSink {
    float *smem;
    const float *src[5][2];  // [plan array (u, kappa or ax, ay, az, then f)][half] of the block
    uint64_t *full;
    __device__ __forceinline__ void arm(int slot, uint32_t bytes) const { mbar_arm(&full[slot], bytes); }
    __device__ __forceinline__ void copy(int dst, int array, int half, int off, int, uint32_t bytes, int slot) const {
        bulk_load(smem + dst, src[array][half] + off, bytes, &full[slot]);
    }
};

// FP32 residual + restriction of a halving level (fine edge 2^LG) with the fine planes staged in shared memory by
// bulk copies (plan above): consumer thread (X, Yl) owns coarse cell (X, y0 / 2 + Yl) of every coarse plane of the
// tile and reads its box of u (and kappa / face coefficients) and f from the staged planes, with the arithmetic of
// residual_restrict32_body (rr32_sum, rr32_store), so the results are bit-identical to k_residual_restrict32.
// Warps of one coarse row each (nc >= 32); the CTA's last warp produces.  The tile is compiled in ({8, 32, 1}, the
// one restrict32t_shape launches); a launch with another tile sets bit 4 of *err and returns before any barrier is
// initialised.  Every wait is bounded: a consumer warp whose wait runs out sets bit 4 of *err and stops; the producer
// stops when a slot is not released in time, sets the bit and waits, again bounded, for the copies it issued before
// it exits.
template <int MODE, int LG>
static __global__ void __launch_bounds__(544) k_residual_restrict32t(
        const float *__restrict__ u, const float *__restrict__ f, const float *__restrict__ kap,
        const float *__restrict__ ih2f, int64_t bsf, float *__restrict__ fc, float *__restrict__ uc,
        const XferItem *__restrict__ xf, int32_t nbc, int64_t bsc, Skip skip, const float *__restrict__ ax,
        const float *__restrict__ ay, const float *__restrict__ az, int TYr, int TZr, int Dr, int *__restrict__ err) {
    // the tile the launch code uses, as constants: ring slots, segment offsets and plane strides fold into immediates
    constexpr int TY = 8, TZ = 32, D = 1;
    if (TYr != TY || TZr != TZ || Dr != D) {
        if (threadIdx.x == 0) atomicOr(err, 4);
        return;
    }
    constexpr int n = 1 << LG, nc = n / 2, P = n + 2, H = half_row(P), HALF = P * P * H;
    static_assert(nc >= 32, "a warp per coarse row");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const R32tPlan plan = r32t_plan(LG, MODE, TY, TZ, D);
    const int RS = plan.RS, ss = plan.ss;
    float *sm = reinterpret_cast<float *>(smem_raw);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + RS * ss), *empty = full + RS;
    const int nty = n / TY, ntz = n / TZ;
    const int ty = static_cast<int>(blockIdx.x % nty);
    const int tz = static_cast<int>((blockIdx.x / nty) % ntz);
    const int64_t B = blockIdx.x / (nty * ntz);
    if (B >= nbc || skip(B)) return;  // uniform over the CTA, before any barrier
    const int64_t b = xf[B].src[0];
    const int y0 = ty * TY, z0 = tz * TZ;
    const int tid = threadIdx.x, nthc = blockDim.x - 32, ncw = nthc >> 5;
    if (tid == 0) {
        for (int i = 0; i < RS; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], ncw);
        }
        mbar_init_fence();
    }
    __syncthreads();
    if (tid >= nthc) {
        if (tid == nthc) {
            const int64_t h0 = b * bsf, h1 = h0 + HALF;
            // the plan's arrays: u, then kappa (MODE 2) or ax, ay, az (MODE 3), then f
            constexpr int NU = MODE == 3 ? 4 : (MODE == 2 ? 2 : 1);
            const float *arr[5] = {u, MODE == 3 ? ax : kap, ay, az, f};
            if constexpr (NU < 4) arr[NU] = f;
            R32tDeviceSink sink{sm, {}, full};
#pragma unroll
            for (int a = 0; a <= NU; ++a) {
                sink.src[a][0] = arr[a] + h0;
                sink.src[a][1] = arr[a] + h1;
            }
            const int NP = TZ + 2;
            bool ok = true;
            int q = 0;
            for (; q < NP; ++q) {
                if (q >= RS && !mbar_wait(&empty[q % RS], ((q / RS) - 1) & 1)) {
                    ok = false;
                    break;
                }
                r32t_issue_plane(plan, z0, y0, q, sink);
            }
            if (!ok) atomicOr(err, 4);
            // the copies still in flight land before the CTA's shared memory can be released
            for (int r = q > RS ? q - RS : 0; r < q; ++r) mbar_wait(&full[r % RS], (r / RS) & 1);
        }
        return;
    }
    const int X = tid & (nc - 1), Yl = tid >> (LG - 1);
    const float ih2 = __ldg(ih2f + b);
    int bad = 0;
    for (int g = 0; g < TZ / 2; ++g) {
        for (int q = g ? 2 * g + 2 : 0; q <= 2 * g + 3; ++q)
            bad |= __any_sync(0xffffffffu, !mbar_wait(&full[q % RS], (q / RS) & 1));
        if (bad) break;
        // box cell (i, j, k) of array a: plane q = 2g + k, half (i + j + k) & 1, slot row 2 Yl + j, position X + i / 2
        const auto at = [&](int a, int i, int j, int k) {
            const int q = 2 * g + k;
            return sm[(q % RS) * ss + r32t_seg(plan, a, (i + j + k) & 1) + (r32t_off_lo(plan, z0 + q, y0) & 3) +
                      (2 * Yl + j) * H + X + (i >> 1)];
        };
        float U[4][4][4], K[4][4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int out = (i == 0 || i == 3) + (j == 0 || j == 3) + (k == 0 || k == 3);
                    if (out > 1) continue;
                    U[k][j][i] = at(0, i, j, k);
                    if constexpr (MODE == 2) K[k][j][i] = at(1, i, j, k);
                }
        float AX[3][3][4], AY[3][4][3], AZ[4][3][3];
        if constexpr (MODE == 3) {
#pragma unroll
            for (int k = 1; k < 3; ++k)
#pragma unroll
                for (int j = 1; j < 3; ++j)
#pragma unroll
                    for (int i = 1; i < 4; ++i) {
                        AX[k][j][i] = at(1, i, j, k);
                        AY[k][i][j] = at(2, j, i, k);
                        AZ[i][k][j] = at(3, j, k, i);
                    }
        }
        const float sum = rr32_sum<MODE>(U, K, AX, AY, AZ, ih2, [&](int i, int j, int k) {
            const int q = 2 * g + k;
            return sm[(q % RS) * ss + r32t_seg(plan, plan.NU, (i + j + k) & 1) + (r32t_off_f(plan, z0 + q, y0) & 3) +
                      (2 * Yl + j - 1) * H + X + (i >> 1)];
        });
        rr32_store<LG>(fc, uc, B, bsc, X, y0 / 2 + Yl, z0 / 2 + g, sum);
        // planes 2g and 2g + 1 are done: every value read from them fed the store above
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if ((tid & 31) == 0) {
            mbar_arrive(&empty[(2 * g) % RS]);
            mbar_arrive(&empty[(2 * g + 1) % RS]);
        }
    }
    if (bad && (tid & 31) == 0) atomicOr(err, 4);
}

// The 8 children (2X + a, 2Y + b, 2Z + c), a, b, c in {1, 2}, of coarse cell (X, Y, Z) in fine block b of a halving
// level (fine edge 2^LG) take the values val[c][b][a].  With nbr6 (the fine level's face table, as in k_smooth) every
// child on a block face also writes its new value through to the same-level neighbour's mirroring ghost, or the
// reflected value to its own boundary ghost, so that afterwards only refinement-interface ghosts need an exchange.
template <int LG>
__device__ __forceinline__ void prolong32_put(float *__restrict__ uf, int64_t bsf, int64_t b, int X, int Y, int Z,
                                              const float (&val)[2][2][2], const int32_t *__restrict__ nbr6) {
    using Bx = Box32<LG>;
    constexpr int nc = (1 << LG) / 2;
    const int corner = (2 * Z * Bx::P + 2 * Y) * Bx::HP + X;  // in-block offset of the box corner
    float *ub = uf + b * bsf + corner;
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int a = 0; a < 2; ++a) ub[Bx::off(a + 1, bb + 1, c + 1)] = val[c][bb][a];
    if (!nbr6) return;
    constexpr int n = Bx::n, H = Bx::HP, PL = Bx::P * Bx::HP, HALF = Bx::HALF;
    // x faces: one lane per coarse row (X = 0: children a = 0, X = nc - 1: children a = 1)
    if (X == 0 || X == nc - 1) {
        const int a = X == 0 ? 0 : 1;
        const int nbv = nbr6[b * 6 + a];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const int hs = (a + bb + c + 1) & 1;  // half of the child (its padded coordinate sum's parity)
                const int q = corner + Bx::off(a + 1, bb + 1, c + 1) - hs * HALF;  // offset inside its half
                if (nbv >= 0) uf[nbv * bsf + hs * HALF + q + (a ? -n / 2 : n / 2)] = val[c][bb][a];
                else if (nbv == -1) uf[b * bsf + (hs ^ 1) * HALF + q] = -val[c][bb][a];
            }
    }
    // y and z faces: whole coarse rows
    if (Y == 0 || Y == nc - 1 || Z == 0 || Z == nc - 1) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    const int hs = (a + bb + c + 1) & 1;
                    const int q = corner + Bx::off(a + 1, bb + 1, c + 1) - hs * HALF;
                    const int cc[3] = {0, 2 * Y + bb, 2 * Z + c};
#pragma unroll
                    for (int axis = 1; axis < 3; ++axis) {
#pragma unroll
                        for (int side = 0; side < 2; ++side) {
                            if (cc[axis] != (side ? n - 1 : 0)) continue;
                            const int Dm = axis == 1 ? n * H : n * PL, E = axis == 1 ? H : PL;
                            const int nbv = nbr6[b * 6 + 2 * axis + side];
                            if (nbv >= 0) uf[nbv * bsf + hs * HALF + q + (side ? -Dm : Dm)] = val[c][bb][a];
                            else if (nbv == -1) uf[b * bsf + (hs ^ 1) * HALF + q + (side ? E : -E)] = -val[c][bb][a];
                        }
                    }
                }
    }
}

// FP32 prolongation + correction for a level whose blocks all halve (fine edge 2^LG): one thread per coarse cell
// adds 1/4 (e_C + e_{C+sx} + e_{C+sy} + e_{C+sz}) to its 8 children, fine offsets as in Box32, and writes them
// through to the face ghosts (prolong32_put).
template <int LG, bool CG = false>
__device__ __forceinline__ void prolong32_body(float *__restrict__ uf, int64_t bsf, const float *__restrict__ ec,
                                               const XferItem *__restrict__ xf, int32_t nbc, int64_t bsc,
                                               const int32_t *__restrict__ nbr6, Skip skip, int64_t t0, int64_t ts) {
    using Bx = Box32<LG>;
    constexpr int nc = (1 << LG) / 2, LC = LG - 1, Pc = nc + 2, HPc = half_row(Pc), PLc = Pc * HPc, HALFc = Pc * PLc;
    const int64_t total = static_cast<int64_t>(nbc) << (3 * LC);
    for (int64_t t = t0; t < total; t += ts) {
        const int r = static_cast<int>(t) & ((1 << (3 * LC)) - 1);
        const int64_t B = t >> (3 * LC);
        if (skip(B)) continue;
        const int X = r & (nc - 1), Y = (r >> LC) & (nc - 1), Z = r >> (2 * LC);
        const int Xc = X + 1, Yc = Y + 1, Zc = Z + 1;
        const int pc = (Xc + Yc + Zc) & 1;
        const int row = (Zc * Pc + Yc) * HPc;
        const float *own = ec + B * bsc + pc * HALFc + row;
        const float *oth = ec + B * bsc + (pc ^ 1) * HALFc + row;
        const float e0 = ldv<CG>(own + (Xc >> 1));
        const float exm = ldv<CG>(oth + ((Xc - 1) >> 1)), exp_ = ldv<CG>(oth + ((Xc + 1) >> 1));
        const float eym = ldv<CG>(oth + ((Xc >> 1) - HPc)), eyp = ldv<CG>(oth + ((Xc >> 1) + HPc));
        const float ezm = ldv<CG>(oth + ((Xc >> 1) - PLc)), ezp = ldv<CG>(oth + ((Xc >> 1) + PLc));
        const float ex[2] = {exm, exp_}, ey[2] = {eym, eyp}, ez[2] = {ezm, ezp};
        const int64_t b = xf[B].src[0];
        const float *ub = uf + b * bsf + (2 * Z * Bx::P + 2 * Y) * Bx::HP + X;
        float val[2][2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a)
                    val[c][bb][a] = ldv<CG>(ub + Bx::off(a + 1, bb + 1, c + 1)) +
                                    0.25f * ((e0 + ex[a]) + (ey[bb] + ez[c]));
        prolong32_put<LG>(uf, bsf, b, X, Y, Z, val, nbr6);
    }
}

template <int LG>
static __global__ void __launch_bounds__(256) k_prolong32(float *__restrict__ uf, int64_t bsf,
                                                          const float *__restrict__ ec,
                                                          const XferItem *__restrict__ xf, int32_t nbc, int64_t bsc,
                                                          const int32_t *__restrict__ nbr6, Skip skip) {
    prolong32_body<LG>(uf, bsf, ec, xf, nbc, bsc, nbr6, skip,
                       blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x,
                       static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// The same prolongation with one thread per segment of ZC coarse cells of a z-column (X fastest across threads, then
// Y, then the segment, then the block).  The thread loads the segment's coarse values once (the column's ZC + 2 and
// the four lateral neighbours per cell) and the next cell's 8 children before it stores this cell's: loads touch
// interior cells only, stores touch other interior cells and ghosts, so the early loads read the values the cell-by-cell
// order would.  Each child takes the expression of prolong32_body, so the results are bit-identical to it.
template <int LG, int ZC>
static __global__ void __launch_bounds__(256) k_prolong32z(float *__restrict__ uf, int64_t bsf,
                                                           const float *__restrict__ ec,
                                                           const XferItem *__restrict__ xf, int32_t nbc, int64_t bsc,
                                                           const int32_t *__restrict__ nbr6, Skip skip) {
    using Bx = Box32<LG>;
    constexpr int nc = (1 << LG) / 2, LC = LG - 1, Pc = nc + 2, HPc = half_row(Pc), PLc = Pc * HPc, HALFc = Pc * PLc;
    static_assert(nc % ZC == 0 && (ZC & (ZC - 1)) == 0, "ZC: a power of two dividing the coarse edge");
    constexpr int LS = LC - (ZC == 1 ? 0 : ZC == 2 ? 1 : ZC == 4 ? 2 : 3);  // log2 of the segments per column
    static_assert(ZC <= 8, "ZC up to 8");
    const int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (t >= (static_cast<int64_t>(nbc) << (2 * LC + LS))) return;
    const int X = static_cast<int>(t) & (nc - 1), Y = static_cast<int>(t >> LC) & (nc - 1);
    const int seg = static_cast<int>(t >> (2 * LC)) & ((1 << LS) - 1);
    const int64_t B = t >> (2 * LC + LS);
    if (skip(B)) return;
    const int Z0 = seg * ZC, Xc = X + 1, Yc = Y + 1;
    const float *eb = ec + B * bsc;
    // coarse padded cell (xc, yc, zc) in the split layout
    const auto E = [&](int xc, int yc, int zc) {
        return eb[((xc + yc + zc) & 1) * HALFc + (zc * Pc + yc) * HPc + (xc >> 1)];
    };
    float col[ZC + 2], exm[ZC], exp_[ZC], eym[ZC], eyp[ZC];
#pragma unroll
    for (int z = 0; z < ZC + 2; ++z) col[z] = E(Xc, Yc, Z0 + z);  // padded z = Z0 .. Z0 + ZC + 1
#pragma unroll
    for (int z = 0; z < ZC; ++z) {
        const int Zc = Z0 + z + 1;
        exm[z] = E(Xc - 1, Yc, Zc);
        exp_[z] = E(Xc + 1, Yc, Zc);
        eym[z] = E(Xc, Yc - 1, Zc);
        eyp[z] = E(Xc, Yc + 1, Zc);
    }
    const int64_t b = xf[B].src[0];
    const float *ub = uf + b * bsf + (2 * Z0 * Bx::P + 2 * Y) * Bx::HP + X;
    constexpr int ZSTEP = 2 * Bx::P * Bx::HP;  // two fine planes
    float cur[2][2][2];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int a = 0; a < 2; ++a) cur[c][bb][a] = ub[Bx::off(a + 1, bb + 1, c + 1)];
#pragma unroll
    for (int z = 0; z < ZC; ++z) {
        float nxt[2][2][2];
        if (z + 1 < ZC) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int a = 0; a < 2; ++a) nxt[c][bb][a] = ub[(z + 1) * ZSTEP + Bx::off(a + 1, bb + 1, c + 1)];
        }
        const float e0 = col[z + 1];
        const float ex[2] = {exm[z], exp_[z]}, ey[2] = {eym[z], eyp[z]}, ez[2] = {col[z], col[z + 2]};
        float val[2][2][2];
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                for (int a = 0; a < 2; ++a) val[c][bb][a] = cur[c][bb][a] + 0.25f * ((e0 + ex[a]) + (ey[bb] + ez[c]));
        prolong32_put<LG>(uf, bsf, b, X, Y, Z0 + z, val, nbr6);
        if (z + 1 < ZC) {
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int a = 0; a < 2; ++a) cur[c][bb][a] = nxt[c][bb][a];
        }
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
// Edge (corners = false) or corner (corners = true) ghosts of a level, after its face exchange (the trilinear
// prolongation reads them): the cells of the same-level block across the edge or corner where there is one (nbr >= 0),
// else linear extrapolation along each of the item's ghost axes from the two ghosts next to it on that axis (face
// ghosts for an edge, edge ghosts for a corner), averaged over the axes -- exact for trilinear data.  Edges: one
// thread per ghost cell along the edge (n per item); corners: one thread per item.  Corners run after the edges.
template <typename T>
static __global__ void k_exchange_diag(T *__restrict__ u, const DiagItem *__restrict__ items, int nitems, LevelGeom g,
                                       bool corners, Skip skip) {
    const int n = g.n;
    const int64_t total = corners ? static_cast<int64_t>(nitems) : static_cast<int64_t>(nitems) * n;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const DiagItem D = items[corners ? t : t / n];
        if (skip(D.blk)) continue;
        int nax = 3, ax[3] = {0, 1, 2}, sg[3];
        int X[3];
        if (corners) {
            for (int a = 0; a < 3; ++a) sg[a] = (D.code >> a) & 1;
        } else {
            const int q = D.code >> 2;
            nax = 2;
            ax[0] = q == 2 ? 1 : 0;
            ax[1] = q == 0 ? 1 : 2;
            const int third = 3 - ax[0] - ax[1];
            sg[0] = D.code & 1;
            sg[1] = (D.code >> 1) & 1;
            X[third] = static_cast<int>(t % n) + 1;
        }
        for (int i = 0; i < nax; ++i) X[ax[i]] = sg[i] ? n + 1 : 0;
        const int64_t dst = Lay<T>::at(g, D.blk, X[0], X[1], X[2]);
        if (D.nbr >= 0) {
            int S[3] = {X[0], X[1], X[2]};
            for (int i = 0; i < nax; ++i) S[ax[i]] = sg[i] ? 1 : n;  // the neighbour's cells next to it
            u[dst] = u[Lay<T>::at(g, D.nbr, S[0], S[1], S[2])];
            continue;
        }
        T acc = T(0);
        for (int i = 0; i < nax; ++i) {
            int A[3] = {X[0], X[1], X[2]}, B2[3] = {X[0], X[1], X[2]};
            A[ax[i]] = sg[i] ? n : 1;       // first interior layer next to the ghost on that axis
            B2[ax[i]] = sg[i] ? n - 1 : 2;  // second
            acc = acc + (T(2) * u[Lay<T>::at(g, D.blk, A[0], A[1], A[2])] - u[Lay<T>::at(g, D.blk, B2[0], B2[1], B2[2])]);
        }
        u[dst] = acc / T(nax);
    }
}

// Trilinear prolongation and correction, u_f += P e_c with P the 8-point tensor-product interpolation: a fine cell
// takes (3/4)^(3-d) (1/4)^d of each of the 8 coarse cells that are d = 0 .. 3 steps (one per axis) from its coarse
// cell towards it, edge and corner ghosts of e_c included (k_exchange_diag); carried-over blocks are injected.  One
// thread per coarse cell, its 8 children (halved block or merged octet) written.  No ghost is written through.
template <typename T>
static __global__ void k_prolong_tri(T *__restrict__ uf, LevelGeom gf, const T *__restrict__ ec,
                                     const XferItem *__restrict__ xf, LevelGeom gc, Skip skip) {
    const int lgc = gc.lg, nc = gc.n;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int X = static_cast<int>(t & (nc - 1));
        const int Y = static_cast<int>((t >> lgc) & (nc - 1));
        const int Z = static_cast<int>((t >> (2 * lgc)) & (nc - 1));
        const int64_t B = t >> (3 * lgc);
        if (skip(B)) continue;
        const XferItem xi = xf[B];
        if (xi.kind == XF_COPY) {
            const int64_t gi = Lay<T>::at(gf, xi.src[0], X + 1, Y + 1, Z + 1);
            uf[gi] = uf[gi] + ec[Lay<T>::at(gc, B, X + 1, Y + 1, Z + 1)];
            continue;
        }
        T e[3][3][3];  // e[dz + 1][dy + 1][dx + 1]: the coarse cell and its 26 neighbours (ghosts included)
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx)
                    e[dz + 1][dy + 1][dx + 1] = ec[Lay<T>::at(gc, B, X + 1 + dx, Y + 1 + dy, Z + 1 + dz)];
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
                    T acc = T(0);
#pragma unroll
                    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                            for (int dx = 0; dx < 2; ++dx) {
                                const int d = dx + dy + dz;
                                const T w = T(d == 0 ? 27.0 / 64.0 : (d == 1 ? 9.0 / 64.0 : (d == 2 ? 3.0 / 64.0 : 1.0 / 64.0)));
                                acc = acc + w * e[1 + (c ? dz : -dz)][1 + (bb ? dy : -dy)][1 + (a ? dx : -dx)];
                            }
                    const int64_t gi = Lay<T>::at(gf, b, x0 + a + 1, y0 + bb + 1, z0 + c + 1);
                    uf[gi] = uf[gi] + acc;
                }
    }
}

template <typename T, bool CG = false>
__device__ __forceinline__ void prolong_body(T *__restrict__ uf, LevelGeom gf, const T *__restrict__ ec,
                                             const XferItem *__restrict__ xf, LevelGeom gc, Skip skip, int64_t t0,
                                             int64_t ts) {
    const int lgc = gc.lg, nc = gc.n;
    const int64_t total = static_cast<int64_t>(gc.nb) << (3 * lgc);
    for (int64_t t = t0; t < total; t += ts) {
        const int X = static_cast<int>(t & (nc - 1));
        const int Y = static_cast<int>((t >> lgc) & (nc - 1));
        const int Z = static_cast<int>((t >> (2 * lgc)) & (nc - 1));
        const int64_t B = t >> (3 * lgc);
        if (skip(B)) continue;
        const XferItem xi = xf[B];
        const T e0 = ldv<CG>(ec + Lay<T>::at(gc, B, X + 1, Y + 1, Z + 1));
        if (xi.kind == XF_COPY) {
            {
                const int64_t gi = Lay<T>::at(gf, xi.src[0], X + 1, Y + 1, Z + 1);
                uf[gi] = ldv<CG>(uf + gi) + e0;
            }
            continue;
        }
        const T ex[2] = {ldv<CG>(ec + Lay<T>::at(gc, B, X, Y + 1, Z + 1)), ldv<CG>(ec + Lay<T>::at(gc, B, X + 2, Y + 1, Z + 1))};
        const T ey[2] = {ldv<CG>(ec + Lay<T>::at(gc, B, X + 1, Y, Z + 1)), ldv<CG>(ec + Lay<T>::at(gc, B, X + 1, Y + 2, Z + 1))};
        const T ez[2] = {ldv<CG>(ec + Lay<T>::at(gc, B, X + 1, Y + 1, Z)), ldv<CG>(ec + Lay<T>::at(gc, B, X + 1, Y + 1, Z + 2))};
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
                for (int a = 0; a < 2; ++a)
                {
                    const int64_t gi = Lay<T>::at(gf, b, x0 + a + 1, y0 + bb + 1, z0 + c + 1);
                    uf[gi] = ldv<CG>(uf + gi) + T(0.25) * ((e0 + ex[a]) + (ey[bb] + ez[c]));
                }
    }
}

// Prolongation and correction u_f += P e_c, P the face-neighbour linear cell-centred interpolation (the paper
// inherits its transfers and does not state them; this is the library's reading).
template <typename T>
static __global__ void k_prolong(T *__restrict__ uf, LevelGeom gf, const T *__restrict__ ec,
                                 const XferItem *__restrict__ xf, LevelGeom gc, Skip skip = Skip{}) {
    prolong_body<T>(uf, gf, ec, xf, gc, skip, blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x,
                    static_cast<int64_t>(gridDim.x) * blockDim.x);
}

// ------------------------------------------------------------------------------------------------------------
// Coarsest level: u = A_c^{-1} f with the dense FP64 inverse of every problem (block-diagonal: the unknowns of
// problem p are cmap[ustart[p] .. ustart[p+1]), its inverse is the row-major N_p x N_p matrix at Ainv + moff[p]).
// One warp per unknown; f gathered from the padded pool through cmap.
// ------------------------------------------------------------------------------------------------------------
template <typename T, bool CG = false>
__device__ __forceinline__ void coarse_solve_row(T *__restrict__ u, const T *__restrict__ f,
                                                 const double *__restrict__ Ainv, const int64_t *__restrict__ cmap,
                                                 const int32_t *__restrict__ uprob, const int64_t *__restrict__ ustart,
                                                 const int64_t *__restrict__ moff, const uint8_t *__restrict__ done,
                                                 int row_i, int lane) {
    const int p = uprob[row_i];
    if (done && done[p]) return;
    const int64_t base = ustart[p];
    const int Np = static_cast<int>(ustart[p + 1] - base);
    const double *row = Ainv + moff[p] + static_cast<int64_t>(row_i - base) * Np;
    double s = 0.0;
    for (int j = lane; j < Np; j += 32) s = fma(row[j], static_cast<double>(ldv<CG>(f + cmap[base + j])), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) u[cmap[row_i]] = T(s);
}

// Coarsest-level solve u = A^-1 f by the dense FP64 inverse, one warp per row (this library's direct coarsest
// solver; Sec. 5's is damped Jacobi, run by the Jacobi kernels when coarse_iters > 0).
template <typename T>
static __global__ void k_coarse_solve(T *__restrict__ u, const T *__restrict__ f, const double *__restrict__ Ainv,
                                      const int64_t *__restrict__ cmap, const int32_t *__restrict__ uprob,
                                      const int64_t *__restrict__ ustart, const int64_t *__restrict__ moff, int N,
                                      const uint8_t *__restrict__ done = nullptr) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= N) return;
    coarse_solve_row<T>(u, f, Ainv, cmap, uprob, ustart, moff, done, warp, threadIdx.x & 31);
}

// ------------------------------------------------------------------------------------------------------------
// FP64 residual over the finest level, r = f - A u (Sec. 5, Eq. 1), written as FP32 r * scale_p (scale_p a power of two per
// problem, so the scaling is exact), with the FP32 correction field zeroed, and per-block sums of h^3 (r scale_p)^2.
// Grid: nb * cpb CTAs, CTA (b, c) covers the c-th of cpb contiguous chunks of block b and writes its partial sum to
// bpart[b cpb + c] (cleared before the launch, so 0 for a skipped block), which k_problem_sums adds up in a fixed
// order, so the norm is the same from run to run.  The squared norm is accumulated in FP32 per thread (it decides convergence and is reported to
// ~1e-6 relative) and in FP64 across threads.  out / zero_out may be null.  ZU: u is known to be zero (a zero
// initial guess), so r = f without reading u or the operator.
// ------------------------------------------------------------------------------------------------------------
template <int MODE, bool ZU = false>
static __global__ void __launch_bounds__(kThreads, 5) k_residual_norm(const double *__restrict__ u, const double *__restrict__ f, Coef cf,
                                       const double *__restrict__ ih2, const float *__restrict__ vol, LevelGeom g,
                                       int cpb, float *__restrict__ out, const float *__restrict__ pscale,
                                       const int32_t *__restrict__ bprob, double *__restrict__ bpart,
                                       float *__restrict__ zero_out, Skip skip = Skip{}) {
    const int lg = g.lg, n = g.n, P = g.P;
    const int64_t b = blockIdx.x / cpb;
    if (skip(b)) return;  // the whole CTA: its partial stays 0
    const int chunk = blockIdx.x - static_cast<int>(b * cpb);
    const int per = (1 << (3 * lg)) / cpb;
    const int sexp = static_cast<int>((__float_as_uint(pscale[bprob[b]]) >> 23) & 0xff) - 127;  // scale = 2^sexp
    const double ihb = MODE == 1 ? 0.0 : ih2[b];
    float acc = 0.0f;
    // the zero-guess form is a stream (f in, r and the zeroed correction out): four cells in flight per thread
#pragma unroll(ZU ? 4 : 1)
    for (int c = chunk * per + threadIdx.x; c < (chunk + 1) * per; c += blockDim.x) {
        const int x = c & (n - 1), y = (c >> lg) & (n - 1), z = c >> (2 * lg);
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, P);
        const double r = ZU ? f[gi] : residual_at<double, MODE>(u, f, cf, gi, P, ihb);  // ZU: u = 0, r = f
        const float rs = f64_to_f32_pow2(r, sexp);
        const int64_t gs = Lay<float>::at(g, b, x + 1, y + 1, z + 1);  // FP32 pools are colour-split
        if (out) out[gs] = rs;
        if (zero_out) {
            zero_out[gs] = 0.0f;
            // and the face ghosts next to it, so that every ghost of the zeroed correction is current
            if (x == 0) zero_out[Lay<float>::at(g, b, 0, y + 1, z + 1)] = 0.0f;
            if (x == n - 1) zero_out[Lay<float>::at(g, b, n + 1, y + 1, z + 1)] = 0.0f;
            if (y == 0) zero_out[Lay<float>::at(g, b, x + 1, 0, z + 1)] = 0.0f;
            if (y == n - 1) zero_out[Lay<float>::at(g, b, x + 1, n + 1, z + 1)] = 0.0f;
            if (z == 0) zero_out[Lay<float>::at(g, b, x + 1, y + 1, 0)] = 0.0f;
            if (z == n - 1) zero_out[Lay<float>::at(g, b, x + 1, y + 1, n + 1)] = 0.0f;
        }
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
        bpart[blockIdx.x] = s;
    }
}

// Per-CTA partial sums of h^3 x^2 over the interior of an FP64 field (same grid shape and partials as
// k_residual_norm).
static __global__ void k_block_norm64(const double *__restrict__ x, const double *__restrict__ vol, LevelGeom g,
                                      int cpb, double *__restrict__ bpart) {
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
        bpart[blockIdx.x] = s;
    }
}

// Per-problem sums of the per-CTA partials (cpb per block, blocks of problem p listed in pblk[pstart[p] ..
// pstart[p+1])): one CTA of 1024 threads per problem, thread t adding partials t, t + 1024, ... of the problem's list
// (block-major), then a fixed tree, so the sum does not depend on the order in which the partials were written.
constexpr int kSumThreads = 1024;
static __global__ void __launch_bounds__(kSumThreads) k_problem_sums(const double *__restrict__ bpart, int cpb,
                                                                     const int32_t *__restrict__ pstart,
                                                                     const int32_t *__restrict__ pblk, int np,
                                                                     double *__restrict__ psum) {
    const int p = blockIdx.x;
    if (p >= np) return;
    const int first = pstart[p], nblk = pstart[p + 1] - first;
    // (block, chunk) of list entry t, advanced by kSumThreads entries per step without a division
    const int step_b = kSumThreads / cpb, step_c = kSumThreads % cpb;
    int bq = threadIdx.x / cpb, c = threadIdx.x % cpb;
    double s = 0.0;
#pragma unroll 4
    for (; bq < nblk; bq += step_b) {
        s += bpart[static_cast<int64_t>(pblk[first + bq]) * cpb + c];
        c += step_c;
        if (c >= cpb) {
            c -= cpb;
            ++bq;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double sm[kSumThreads / 32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kSumThreads / 32; ++w) t += sm[w];
        psum[p] = t;
    }
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
                              const int64_t *__restrict__ off = nullptr, int *__restrict__ nonzero = nullptr) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
    bool any = false;
#pragma unroll 4  // several cells' loads in flight per thread
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        const int64_t src = off ? off[b] + (t & ((int64_t(1) << (3 * lg)) - 1)) : t;
        const double v = user[src];
        any = any || v != 0.0;
        pool[b * g.bs + off3(x + 1, y + 1, z + 1, g.P)] = T(v);
    }
    if (nonzero && __ballot_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) atomicOr(nonzero, 1);
}

template <typename T>
static __global__ void k_unpack(double *__restrict__ user, const T *__restrict__ pool, LevelGeom g,
                                const int64_t *__restrict__ off = nullptr) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
#pragma unroll 4  // several cells' loads in flight per thread
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

// u64 += e32 / scale_p over the interior (mixed-precision defect correction update, an extension the paper does not
// have; pinv = 1 / scale_p per problem)
static __global__ void k_update_mixed(double *__restrict__ u, const float *__restrict__ e,
                                      const double *__restrict__ pinv, const int32_t *__restrict__ bprob,
                                      LevelGeom g, Skip skip = Skip{}) {
    const int lg = g.lg, n = g.n;
    const int64_t total = static_cast<int64_t>(g.nb) << (3 * lg);
#pragma unroll 4  // several cells' loads in flight per thread
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int x = static_cast<int>(t & (n - 1));
        const int y = static_cast<int>((t >> lg) & (n - 1));
        const int z = static_cast<int>((t >> (2 * lg)) & (n - 1));
        const int64_t b = t >> (3 * lg);
        if (skip(b)) continue;
        const int64_t gi = b * g.bs + off3(x + 1, y + 1, z + 1, g.P);
        const int pexp = static_cast<int>((static_cast<uint64_t>(__double_as_longlong(pinv[bprob[b]])) >> 52) & 0x7ff) - 1023;
        u[gi] += f32_to_f64_pow2(e[Lay<float>::at(g, b, x + 1, y + 1, z + 1)], pexp);  // pinv = 2^pexp: exact
    }
}

// Face coefficients of a level from k with ghosts (variable coefficients: future work in Sec. 8; harmonic-mean
// reading): MODE 1 arrays (harmonic mean times the block's 1/h^2) and
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
        const bool wx = tx && X >= 1 && inY && inZ, wy = ty && Y >= 1 && inX && inZ, wz = tz && Z >= 1 && inX && inY;
        if (wx || wy || wz) {
            // harmonic means 2 k_a k_c / (k_a + k_c) of the three lower faces with one FP64 division: the reciprocals
            // of the three sums from the reciprocal of their product (batch inversion), unless the product leaves
            // the normal range, then one division each
            const double ka = wx ? k[gi - 1] : kc, kb = wy ? k[gi - P] : kc;
            const double kd = wz ? k[gi - static_cast<int64_t>(P) * P] : kc;
            const double sa = ka + kc, sb = kb + kc, sd = kd + kc, sab = sa * sb, prod = sab * sd;
            double ra, rb, rd;
            if (isfinite(prod) && prod > 2.2250738585072014e-308) {
                const double ip = 1.0 / prod, iab = ip * sd;
                ra = iab * sb;
                rb = iab * sa;
                rd = ip * sab;
            } else {
                ra = 1.0 / sa;
                rb = 1.0 / sb;
                rd = 1.0 / sd;
            }
            if (wx) tx[gi] = 2.0 * ka * kc * ra * s;
            if (wy) ty[gi] = 2.0 * kb * kc * rb * s;
            if (wz) tz[gi] = 2.0 * kd * kc * rd * s;
        }
        const bool face_or_interior = (inX && inY) || (inX && inZ) || (inY && inZ);
        // 1/k for the FP32 cycles: FP32 accuracy suffices (binary32 conversion on exponent bits, FP32 division)
        if (kap && face_or_interior && kc > 0.0) kap[Lay<float>::at(g, b, X, Y, Z)] = 1.0f / f64_to_f32_pow2(kc, 0);
    }
}

// Face coefficients of a coarse level averaged from the finer level's (face-averaged coarse coefficients): every
// coarse face is covered by 2 x 2 faces of the finer level and takes their mean; the stored T / h^2 scales by
// h_f^2 / h_c^2 = 1/4, so the coarse value is the sum of the four over 16 (halved blocks and merged octets; carried-over
// blocks keep theirs).  Inside a merged octet the face between two children is held by both (their values differ where
// it was a refinement interface, or lay between a carried-over and a merged block, on the finer level): the merged
// block takes the mean of the two sides' eight values, so that each face inside a block has one coefficient.  One
// thread per face position of every coarse block and axis: along the axis the lower face
// of cell a (a = 0 .. n-1) and the block's upper face (a = n, stored at the ghost position), the two other
// coordinates 0 .. n-1.  An operator-aware coarsening the paper does not discuss; its reading is this library's.
static __global__ void k_average_faces64(const double *__restrict__ tfx, const double *__restrict__ tfy,
                                         const double *__restrict__ tfz, LevelGeom gf, double *__restrict__ tcx,
                                         double *__restrict__ tcy, double *__restrict__ tcz,
                                         const XferItem *__restrict__ xf, LevelGeom gc) {
    const int nc = gc.n, nf = gf.n;
    const int64_t per = static_cast<int64_t>(nc + 1) * nc * nc;
    const int64_t total = static_cast<int64_t>(gc.nb) * 3 * per;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t B = t / (3 * per);
        const int64_t r = t - B * 3 * per;
        const int axis = static_cast<int>(r / per);
        const int q = static_cast<int>(r - axis * per);
        const int a = q % (nc + 1), t1 = (q / (nc + 1)) % nc, t2 = q / ((nc + 1) * nc);
        const int o1 = axis == 0 ? 1 : 0, o2 = axis == 2 ? 1 : 2;  // the other two axes, increasing
        int C[3];
        C[axis] = a + 1;
        C[o1] = t1 + 1;
        C[o2] = t2 + 1;
        const double *src = axis == 0 ? tfx : (axis == 1 ? tfy : tfz);
        double *dst = axis == 0 ? tcx : (axis == 1 ? tcy : tcz);
        const XferItem xi = xf[B];
        const int64_t gcell = B * gc.bs + off3(C[0], C[1], C[2], gc.P);
        if (xi.kind == XF_COPY) {
            dst[gcell] = src[xi.src[0] * gf.bs + off3(C[0], C[1], C[2], gf.P)];
            continue;
        }
        // a merged octet's face between two children: each child holds its own value of it (the lower child at its
        // upper ghost position, the upper child at its first cell), and the merged block takes the mean of both
        const bool shared = xi.kind == XF_MERGE && 2 * a == nf;
        double s = 0.0;
        for (int e2 = 0; e2 < 2; ++e2)
            for (int e1 = 0; e1 < 2; ++e1) {
                int F[3];  // finer interior coordinates of the cell on the face's upper side (2 n_c: the upper face)
                F[axis] = 2 * a;
                F[o1] = 2 * t1 + e1;
                F[o2] = 2 * t2 + e2;
                if (xi.kind == XF_HALVE) {
                    s += src[xi.src[0] * gf.bs + off3(F[0] + 1, F[1] + 1, F[2] + 1, gf.P)];
                    continue;
                }
                // merged octet: children of edge nf (= nc) assembled into a 2 nf block
                int oc[3], L[3];
                for (int d = 0; d < 3; ++d) {
                    oc[d] = F[d] >= nf ? 1 : 0;
                    L[d] = F[d] - oc[d] * nf + 1;
                }
                s += src[xi.src[oc[0] + 2 * oc[1] + 4 * oc[2]] * gf.bs + off3(L[0], L[1], L[2], gf.P)];
                if (shared) {
                    oc[axis] = 0;
                    L[axis] = nf + 1;
                    s += src[xi.src[oc[0] + 2 * oc[1] + 4 * oc[2]] * gf.bs + off3(L[0], L[1], L[2], gf.P)];
                }
            }
        dst[gcell] = (shared ? 0.03125 : 0.0625) * s;
    }
}

// FP32 halved face coefficients T / 2 = (T / h^2) h^2 / 2 of a face-averaged coarse level, from its FP64 scaled ones,
// in the colour-split layout of the FP32 pools (a cell's lower x, y and z faces at the cell, the block's upper faces
// at the ghost positions), for the FP32 cycles' coefficient mode 3.
static __global__ void k_face_half32(const double *__restrict__ tx, const double *__restrict__ ty,
                                     const double *__restrict__ tz, const double *__restrict__ h2, LevelGeom g,
                                     float *__restrict__ ax, float *__restrict__ ay, float *__restrict__ az) {
    const int P = g.P, n = g.n;
    const int64_t per = static_cast<int64_t>(P) * P * P;
    const int64_t total = static_cast<int64_t>(g.nb) * per;
    for (int64_t t = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int64_t b = t / per;
        const int r = static_cast<int>(t - b * per);
        const int X = r % P, Y = (r / P) % P, Z = r / (P * P);
        const bool inY = Y >= 1 && Y <= n, inZ = Z >= 1 && Z <= n, inX = X >= 1 && X <= n;
        const int64_t gi = b * g.bs + r, gs = Lay<float>::at(g, b, X, Y, Z);
        const double s = 0.5 * h2[b];
        if (X >= 1 && inY && inZ) ax[gs] = static_cast<float>(tx[gi] * s);
        if (Y >= 1 && inX && inZ) ay[gs] = static_cast<float>(ty[gi] * s);
        if (Z >= 1 && inX && inY) az[gs] = static_cast<float>(tz[gi] * s);
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
// Unit entry m of every problem with more than m coarsest unknowns, and entry m - 1 cleared again (the interior is
// otherwise zero; the exchange rewrites every ghost from it).
static __global__ void k_set_units(double *__restrict__ u, const int64_t *__restrict__ cmap,
                                   const int64_t *__restrict__ ustart, int np, int m) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    if (m > 0 && ustart[p] + m - 1 < ustart[p + 1]) u[cmap[ustart[p] + m - 1]] = 0.0;
    if (ustart[p] + m < ustart[p + 1]) u[cmap[ustart[p] + m]] = 1.0;
}
// Gauss-Jordan inversion of every problem's coarsest block (row-major N_p x N_p at moff[p]) on the device, in place
// with partial pivoting, one column c per step (two launches), reading one buffer and writing the other:
//   pivot: q = the row r >= c with the largest |a[r][c]| (the first on ties), v = 1 / a[q][c];
//   step:  rows c and q exchanged, then  a'[c][j] = a[c][j] v (j != c), a'[c][c] = v,
//          a'[r][j] = a[r][j] - a[r][c] a'[c][j] (r != c, j != c), a'[r][c] = -a[r][c] v.
// After N steps the buffer holds (P A)^{-1} = A^{-1} P^T for the row exchanges P; A^{-1} follows by exchanging the
// columns back in reverse order.  Problems with fewer unknowns than c copy their block through.
// One warp per problem; a zero (or non-finite) pivot sets *bad.
static __global__ void k_gj_pivot(const double *__restrict__ A, const int64_t *__restrict__ moff,
                                  const int64_t *__restrict__ ustart, int np, int c, int32_t *__restrict__ piv,
                                  double *__restrict__ pinv, int maxN, int *__restrict__ bad) {
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (p >= np) return;
    const int N = static_cast<int>(ustart[p + 1] - ustart[p]);
    if (c >= N) return;
    const double *a = A + moff[p];
    double best = -1.0;
    int row = N;
    for (int r = c + lane; r < N; r += 32) {
        const double v = fabs(a[static_cast<int64_t>(r) * N + c]);
        if (v > best) { best = v; row = r; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int orow = __shfl_xor_sync(0xffffffffu, row, o);
        if (ob > best || (ob == best && orow < row)) { best = ob; row = orow; }
    }
    if (lane == 0) {
        if (!(best > 0.0) || !isfinite(best) || row >= N) {
            atomicOr(bad, 1);
            row = c;
        }
        piv[static_cast<int64_t>(p) * maxN + c] = row;
        pinv[p] = 1.0 / a[static_cast<int64_t>(row) * N + c];
    }
}
static __global__ void k_gj_step(const double *__restrict__ A, double *__restrict__ B, const int64_t *__restrict__ moff,
                                 const int64_t *__restrict__ ustart, int c, const int32_t *__restrict__ piv,
                                 const double *__restrict__ pinv, int maxN) {
    const int p = blockIdx.y;
    const int N = static_cast<int>(ustart[p + 1] - ustart[p]);
    const int64_t NN = static_cast<int64_t>(N) * N;
    const double *a = A + moff[p];
    double *b = B + moff[p];
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < NN;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        if (c >= N) {
            b[e] = a[e];
            continue;
        }
        const int r = static_cast<int>(e / N), j = static_cast<int>(e - static_cast<int64_t>(r) * N);
        const int q = piv[static_cast<int64_t>(p) * maxN + c];
        const double v = pinv[p];
        const int sr = r == c ? q : (r == q ? c : r);  // row r of the exchanged matrix
        const double *arow = a + static_cast<int64_t>(sr) * N, *prow = a + static_cast<int64_t>(q) * N;
        double out;
        if (r == c) {
            out = j == c ? v : prow[j] * v;
        } else {
            const double fr = arow[c];
            out = j == c ? -fr * v : fma(-fr, prow[j] * v, arow[j]);
        }
        b[e] = out;
    }
}
// A^{-1} from the eliminated buffer R: the column exchanges undone (src = composed inverse permutation per problem,
// src[k] the column of R that becomes column k), written to X; and its transpose to R afterwards (k_gj_transpose).
static __global__ void k_gj_unpermute(const double *__restrict__ R, double *__restrict__ X,
                                      const int64_t *__restrict__ moff, const int64_t *__restrict__ ustart,
                                      const int32_t *__restrict__ src, int maxN) {
    const int p = blockIdx.y;
    const int N = static_cast<int>(ustart[p + 1] - ustart[p]);
    const int64_t NN = static_cast<int64_t>(N) * N;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < NN;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / N), k = static_cast<int>(e - static_cast<int64_t>(r) * N);
        X[moff[p] + e] = R[moff[p] + static_cast<int64_t>(r) * N + src[static_cast<int64_t>(p) * maxN + k]];
    }
}
static __global__ void k_gj_transpose(const double *__restrict__ X, double *__restrict__ T,
                                      const int64_t *__restrict__ moff, const int64_t *__restrict__ ustart) {
    const int p = blockIdx.y;
    const int N = static_cast<int>(ustart[p + 1] - ustart[p]);
    const int64_t NN = static_cast<int64_t>(N) * N;
    for (int64_t e = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; e < NN;
         e += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int r = static_cast<int>(e / N), k = static_cast<int>(e - static_cast<int64_t>(r) * N);
        T[moff[p] + static_cast<int64_t>(k) * N + r] = X[moff[p] + e];
    }
}
// The inverse column permutation of every problem from its pivot rows (one thread per problem): exchanges undone in
// reverse order, src[k] = the eliminated column that holds column k of A^{-1}.
static __global__ void k_gj_perm(const int32_t *__restrict__ piv, const int64_t *__restrict__ ustart, int np,
                                 int32_t *__restrict__ src, int maxN) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const int N = static_cast<int>(ustart[p + 1] - ustart[p]);
    int32_t *s = src + static_cast<int64_t>(p) * maxN;
    const int32_t *pv = piv + static_cast<int64_t>(p) * maxN;
    for (int k = 0; k < N; ++k) s[k] = k;
    for (int c = N - 1; c >= 0; --c) {
        const int q = pv[c], t = s[c];
        s[c] = s[q];
        s[q] = t;
    }
}
// Colour probe of a coarsest level without refinement interfaces (its operator couples a cell only with its six face
// neighbours, across block faces through same-level ghosts): u = 1 on every unknown of colour C (global cell
// coordinates mod 3 per axis, 27 colours), 0 elsewhere.  Then row i of A u is A[i, m] for the one unknown m of colour
// C among i and its six neighbours (nbu: their unknown indices, -1 outside the domain), or 0.
static __global__ void k_set_colour(double *__restrict__ u, const int64_t *__restrict__ cmap,
                                    const int8_t *__restrict__ col, int N, int C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) u[cmap[i]] = col[i] == C ? 1.0 : 0.0;
}
static __global__ void k_gather_colour(const double *__restrict__ r, const int64_t *__restrict__ cmap,
                                       const int32_t *__restrict__ uprob, const int64_t *__restrict__ ustart,
                                       const int64_t *__restrict__ moff, const int8_t *__restrict__ col,
                                       const int32_t *__restrict__ nbu, int N, double *__restrict__ A, int C) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int p = uprob[i];
    const int64_t base = ustart[p], Np = ustart[p + 1] - base;
#pragma unroll
    for (int q = 0; q < 7; ++q) {
        const int m = nbu[static_cast<int64_t>(i) * 7 + q];
        if (m >= 0 && col[m] == C) {
            A[moff[p] + (i - base) * Np + (m - base)] = r[cmap[i]];
            return;
        }
    }
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
