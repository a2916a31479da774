// dtn_device.cuh -- device-side building blocks of the walk-on-spheres /
// local-BIE path: counter RNG, distance to the boundary, Dirichlet data, and
// the whole-sphere Green's function of the patch ball.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dtn {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxL = 16;                 // highest spherical-harmonic degree
constexpr int kMaxSmemBoxes = 1024;       // obstacle boxes staged in shared memory

// ------------------------------------------------------------------ RNG
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// products (multipliers D2511F53, CD9E8D57) and xors with the key, the key
// advancing by the Weyl increments 9E3779B9, BB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product per multiplier gives both halves
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same generator with the ten round keys (k0 + r 9E3779B9, k1 + r BB67AE85)
// given: from kernel parameters they are constant-bank operands of the xors.
__device__ __forceinline__ uint4 philox4x32_10_rk(uint4 c, const uint32_t *rk0, const uint32_t *rk1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ rk1[r],
                       (uint32_t)p0);
    }
    return c;
}

// Uniforms in (0,1), never 0 or 1: an odd integer times a power of two.
__device__ __forceinline__ double u01_53(uint32_t hi, uint32_t lo) {
    const unsigned long long v = ((unsigned long long)hi << 21) | (unsigned long long)(lo >> 11);
    return __ull2double_rn(v | 1ull) * 0x1p-53;
}

// ------------------------------------------------------------------ geometry
enum GeomKind : int { kBall = 0, kBox = 1, kBoxMinusBoxes = 2, kHalfSpace = 3, kDiskExterior = 4, kBallExterior = 5 };

// regions whose walks can leave for infinity (through the truncation sphere)
__host__ __device__ constexpr bool unbounded(int gk) { return gk == 3 || gk == 4 || gk == 5; }

struct DGeom {
    int kind;
    double c[3], R;          // ball
    double lo[3], hi[3];     // outer box
    float c_f[3], R_f, lo_f[3], hi_f[3];   // the same, rounded to FP32 on the host
    double trunc;            // unbounded regions: truncation radius
    float trunc_f;
    int nb;                  // obstacle boxes
    const double *boxes;     // nb x 6
    const float *boxes_f;    // nb x 6
    // obstacle lookup grid over the outer box: per cell, the boxes within the
    // listing distance (CSR) and a lower bound of the distance from the cell to
    // every box not listed
    int gn[3];
    double glo[3], cell;
    float glo_f[3], inv_cell_f;
    const int *cstart;
    const int *citems;
    const float *ccap;
};

template <typename T> struct Vec3 { T x, y, z; };

// A parameter in the walk's precision: FP32 walks read the host-rounded copy
// (a double-to-float conversion on the device would run on the FP64 pipe).
template <typename T> __device__ __forceinline__ T pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// Distance from x to the boundary, the radius of the largest empty sphere
// used by one walk step.  For the box-minus-boxes region the obstacle part
// only looks at the boxes listed for x's grid cell and caps the result at the
// cell's bound for all others, which is a valid (never larger) radius and
// exact whenever it is below the bound.  `sb` are the boxes staged in shared
// memory (kind 2, T = float) or nullptr.
template <typename T>
__device__ __forceinline__ T box_interior_dist(const DGeom &g, T x, T y, T z) {
    T d = x - pick<T>(g.lo[0], g.lo_f[0]);
    d = fmin(d, pick<T>(g.hi[0], g.hi_f[0]) - x);
    d = fmin(d, y - pick<T>(g.lo[1], g.lo_f[1]));
    d = fmin(d, pick<T>(g.hi[1], g.hi_f[1]) - y);
    d = fmin(d, z - pick<T>(g.lo[2], g.lo_f[2]));
    d = fmin(d, pick<T>(g.hi[2], g.hi_f[2]) - z);
    return d;
}

template <typename T>
__device__ __forceinline__ T box_exterior_dist(const T *b, T x, T y, T z) {
    const T ex = fmax(fmax(b[0] - x, (T)0), x - b[3]);
    const T ey = fmax(fmax(b[1] - y, (T)0), y - b[4]);
    const T ez = fmax(fmax(b[2] - z, (T)0), z - b[5]);
    return sqrt(ex * ex + ey * ey + ez * ez);
}

// Grid cell of a point (FP32 index arithmetic: a point near a cell face may be
// filed in the neighbouring cell, whose candidate list is built with a margin
// that covers this).
template <typename T>
__device__ __forceinline__ int grid_cell(const DGeom &g, T x, T y, T z) {
    int ix = (int)floorf(((float)x - g.glo_f[0]) * g.inv_cell_f);
    int iy = (int)floorf(((float)y - g.glo_f[1]) * g.inv_cell_f);
    int iz = (int)floorf(((float)z - g.glo_f[2]) * g.inv_cell_f);
    ix = min(max(ix, 0), g.gn[0] - 1);
    iy = min(max(iy, 0), g.gn[1] - 1);
    iz = min(max(iz, 0), g.gn[2] - 1);
    return (iz * g.gn[1] + iy) * g.gn[0] + ix;
}

template <typename T, int GK>
__device__ __forceinline__ T geo_dist(const DGeom &g, const T *sb, T x, T y, T z) {
    if (GK == kBall || GK == kBallExterior) {
        const T dx = x - pick<T>(g.c[0], g.c_f[0]), dy = y - pick<T>(g.c[1], g.c_f[1]),
                dz = z - pick<T>(g.c[2], g.c_f[2]);
        T r;
        if constexpr (sizeof(T) == 4) {
            // SFU reciprocal square root: |x| to a few FP32 ulps
            // the 1e-30 keeps r2 > 0 at the centre (below half an ulp of any other r2)
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-30f)));
            r = r2 * rsqrtf(r2);
        } else {
            r = sqrt(dx * dx + dy * dy + dz * dz);
        }
        return GK == kBall ? pick<T>(g.R, g.R_f) - r : r - pick<T>(g.R, g.R_f);
    } else if (GK == kHalfSpace) {
        return z - pick<T>(g.c[2], g.c_f[2]);
    } else if (GK == kDiskExterior) {
        const T dx = x - pick<T>(g.c[0], g.c_f[0]), dy = y - pick<T>(g.c[1], g.c_f[1]),
                dz = z - pick<T>(g.c[2], g.c_f[2]);
        const T b = pick<T>(g.R, g.R_f);
        const T r = sqrt(dx * dx + dy * dy);
        if (r <= b) return fabs(dz);
        return sqrt((r - b) * (r - b) + dz * dz);
    } else if (GK == kBox) {
        return box_interior_dist<T>(g, x, y, z);
    } else {
        T d = box_interior_dist<T>(g, x, y, z);
        const int c = grid_cell<T>(g, x, y, z);
        d = fmin(d, (T)g.ccap[c]);
        const int e = g.cstart[c + 1];
        for (int i = g.cstart[c]; i < e; ++i) {
            const int b = g.citems[i];
            const T *bb;
            T tmp[6];
            if (sb) {
                bb = sb + 6 * b;
            } else {
#pragma unroll
                for (int k = 0; k < 6; ++k) tmp[k] = (T)g.boxes[6 * b + k];
                bb = tmp;
            }
            d = fmin(d, box_exterior_dist<T>(bb, x, y, z));
        }
        return d;
    }
}

// Unbounded regions: outside the truncation sphere a walk has gone to infinity.
template <typename T>
__device__ __forceinline__ bool geo_escaped(const DGeom &g, T x, T y, T z) {
    const T dx = x - pick<T>(g.c[0], g.c_f[0]), dy = y - pick<T>(g.c[1], g.c_f[1]), dz = z - pick<T>(g.c[2], g.c_f[2]);
    const T R = pick<T>(g.trunc, g.trunc_f);
    return dx * dx + dy * dy + dz * dz > R * R;
}

// Nearest boundary point (the absorption point whose data are scored), exact
// over the same candidates; ties take the lowest face index, the outer box
// before obstacles, and obstacles in index order.
template <typename T>
__device__ T geo_nearest(const DGeom &g, const T *sb, T x, T y, T z, T &nx, T &ny, T &nz) {
    if (g.kind == kHalfSpace) {
        nx = x;
        ny = y;
        nz = pick<T>(g.c[2], g.c_f[2]);
        return z - nz;
    }
    if (g.kind == kDiskExterior) {
        const T cx = pick<T>(g.c[0], g.c_f[0]), cy = pick<T>(g.c[1], g.c_f[1]), cz = pick<T>(g.c[2], g.c_f[2]);
        const T b = pick<T>(g.R, g.R_f);
        const T dx = x - cx, dy = y - cy, dz = z - cz;
        const T r = sqrt(dx * dx + dy * dy);
        nz = cz;
        if (r <= b) {
            nx = x;
            ny = y;
            return fabs(dz);
        }
        nx = cx + b * dx / r;
        ny = cy + b * dy / r;
        return sqrt((r - b) * (r - b) + dz * dz);
    }
    if (g.kind == kBall || g.kind == kBallExterior) {
        const T cx = pick<T>(g.c[0], g.c_f[0]), cy = pick<T>(g.c[1], g.c_f[1]), cz = pick<T>(g.c[2], g.c_f[2]);
        const T R = pick<T>(g.R, g.R_f);
        const T dx = x - cx, dy = y - cy, dz = z - cz;
        const T r2 = dx * dx + dy * dy + dz * dz;
        T r, s;
        if constexpr (sizeof(T) == 4) {
            const float ir = r2 > 0.f ? rsqrtf(r2) : 0.f;   // SFU, a few ulps
            r = r2 * ir;
            s = R * ir;
        } else {
            r = sqrt(r2);
            s = r > (T)0 ? R / r : (T)0;
        }
        if (r > (T)0) {
            nx = cx + s * dx; ny = cy + s * dy; nz = cz + s * dz;
        } else {
            nx = cx; ny = cy; nz = cz + R;
        }
        return g.kind == kBall ? R - r : r - R;
    }
    const T xs[3] = {x, y, z};
    T best = (T)INFINITY;
    int bf = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int ax = f >> 1;
        const T d = (f & 1) ? pick<T>(g.hi[ax], g.hi_f[ax]) - xs[ax] : xs[ax] - pick<T>(g.lo[ax], g.lo_f[ax]);
        if (d < best) { best = d; bf = f; }
    }
    T p[3] = {x, y, z};
    p[bf >> 1] = (bf & 1) ? pick<T>(g.hi[bf >> 1], g.hi_f[bf >> 1]) : pick<T>(g.lo[bf >> 1], g.lo_f[bf >> 1]);
    if (g.kind == kBoxMinusBoxes) {
        const int c = grid_cell<T>(g, x, y, z);
        const int e = g.cstart[c + 1];
        for (int i = g.cstart[c]; i < e; ++i) {
            const int b = g.citems[i];
            T bb[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) bb[k] = sb ? sb[6 * b + k] : (T)g.boxes[6 * b + k];
            const T d = box_exterior_dist<T>(bb, x, y, z);
            if (d < best) {
                best = d;
#pragma unroll
                for (int k = 0; k < 3; ++k) p[k] = fmin(fmax(xs[k], bb[k]), bb[k + 3]);
            }
        }
    }
    nx = p[0]; ny = p[1]; nz = p[2];
    return best;
}

// ------------------------------------------------------------------ data
enum DataKind : int { kPointSource = 0, kHarmonicSH = 1, kConstant = 2 };

// normalised associated-Legendre recurrence coefficients, filled at load time:
// A[l][m] = sqrt((4l^2-1)/(l^2-m^2)), B[l][m] = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
// D[m] = sqrt((2m+1)/(2m))
// Pairs (l, m), 0 <= m <= l <= kMaxL, in m-major order: pair (l, m) sits at
// sh_pair(l, m).
constexpr int kShPairs = (kMaxL + 1) * (kMaxL + 2) / 2;
__host__ __device__ constexpr int sh_pair(int l, int m) { return m * (kMaxL + 1) - m * (m - 1) / 2 + (l - m); }

struct ShTables {
    double A[kMaxL + 1][kMaxL + 1], B[kMaxL + 1][kMaxL + 1], D[kMaxL + 1];
    float Af[kMaxL + 1][kMaxL + 1], Bf[kMaxL + 1][kMaxL + 1], Df[kMaxL + 1];
    // scaled solid-harmonic recurrence (FP32): beta[sh_pair(l, m)] = B_lm / A_{l-1,m}
    // for l >= m + 2, else 0
    float beta[kShPairs];
};

struct DData {
    int kind;
    double x0[3], strength;
    int lmax;
    const double *clm;      // (lmax+1)^2
    const float *clm_f;
    double ctr[3], inv_scale;
    double constant;
    const ShTables *sh;     // device copy of the recurrence tables
    // FP32 copies rounded on the host; q_f = strength / (4 pi)
    float x0_f[3], q_f, ctr_f[3], inv_scale_f, constant_f;
    // FP32 coefficients in pair order times the recurrence scale alpha_lm:
    // cart[sh_pair(l, m)] = alpha_lm (c_{l,m}, c_{l,-m}) (c_{l,-0} = 0, zero beyond lmax)
    const float2 *cart;
};

// The recurrence coefficients live in constant memory: every index (l, m) is the
// same across a warp, so reads are broadcasts with no load latency.  Each
// translation unit has its own copy (no relocatable device code), filled by its
// upload function at table set-up.
static __constant__ ShTables c_sh;

static inline cudaError_t upload_sh_tables_here(const ShTables &t) {
    return cudaMemcpyToSymbol(c_sh, &t, sizeof(t));
}

template <typename T> __device__ __forceinline__ T sh_A(const ShTables *, int l, int m);
template <> __device__ __forceinline__ double sh_A<double>(const ShTables *, int l, int m) { return c_sh.A[l][m]; }
template <> __device__ __forceinline__ float sh_A<float>(const ShTables *, int l, int m) { return c_sh.Af[l][m]; }
template <typename T> __device__ __forceinline__ T sh_B(const ShTables *, int l, int m);
template <> __device__ __forceinline__ double sh_B<double>(const ShTables *, int l, int m) { return c_sh.B[l][m]; }
template <> __device__ __forceinline__ float sh_B<float>(const ShTables *, int l, int m) { return c_sh.Bf[l][m]; }
template <typename T> __device__ __forceinline__ T sh_D(const ShTables *, int m);
template <> __device__ __forceinline__ double sh_D<double>(const ShTables *, int m) { return c_sh.D[m]; }
template <> __device__ __forceinline__ float sh_D<float>(const ShTables *, int m) { return c_sh.Df[m]; }
template <typename T> __device__ __forceinline__ T clm_at(const DData &d, int i);
template <> __device__ __forceinline__ double clm_at<double>(const DData &d, int i) { return d.clm[i]; }
template <> __device__ __forceinline__ float clm_at<float>(const DData &d, int i) { return d.clm_f[i]; }

// sum c_lm rho^l Y_lm(direction) with orthonormal real harmonics (no
// Condon-Shortley phase), by the normalised Legendre recurrences in m and l
// and the angle-addition recurrence for cos(m phi), sin(m phi).
template <typename T>
__device__ T harmonic_eval(const DData &d, T x, T y, T z) {
    const T is = pick<T>(d.inv_scale, d.inv_scale_f);
    x = (x - pick<T>(d.ctr[0], d.ctr_f[0])) * is;
    y = (y - pick<T>(d.ctr[1], d.ctr_f[1])) * is;
    z = (z - pick<T>(d.ctr[2], d.ctr_f[2])) * is;
    const T rxy2 = x * x + y * y;
    const T r = sqrt(rxy2 + z * z);
    const T y00 = (T)0.28209479177387814;  // 1/sqrt(4 pi)
    if (r == (T)0) return clm_at<T>(d, 0) * y00;
    const T rxy = sqrt(rxy2);
    const T ct = z / r, st = rxy / r;
    const T cp = rxy > (T)0 ? x / rxy : (T)1, sp = rxy > (T)0 ? y / rxy : (T)0;
    const T sqrt2 = (T)1.4142135623730951;
    T acc = (T)0;
    T pmm = y00, cm = (T)1, sm = (T)0, rm = (T)1;
    for (int m = 0; m <= d.lmax; ++m) {
        if (m > 0) {
            pmm *= sh_D<T>(d.sh, m) * st;
            const T c2 = cm * cp - sm * sp;
            sm = sm * cp + cm * sp;
            cm = c2;
            rm *= r;
        }
        T p1 = pmm, p2 = (T)0, rl = rm;
        for (int l = m; l <= d.lmax; ++l) {
            if (l > m) {
                const T p = sh_A<T>(d.sh, l, m) * (ct * p1 - sh_B<T>(d.sh, l, m) * p2);
                p2 = p1;
                p1 = p;
                rl *= r;
            }
            const int base = l * l + l;
            if (m == 0) {
                acc += clm_at<T>(d, base) * rl * p1;
            } else {
                acc += sqrt2 * rl * p1 * (clm_at<T>(d, base + m) * cm + clm_at<T>(d, base - m) * sm);
            }
        }
    }
    return acc;
}

// The same sum in FP32 without square roots or divisions, by the solid
// harmonics r^l Ybar_lm: with (C_m + i S_m) = (x + i y)^m and
// T_lm = r^(l-m) Pbar_lm(cos theta) / sin^m theta, a polynomial in z and r^2,
//   T_mm = pmm_m,  T_lm = A_lm (z T_{l-1,m} - B_lm r^2 T_{l-2,m}),
//   g = sum_m sum_l T_lm (c_{l,m} C_m + c_{l,-m} S_m).
// The recurrence runs scaled: T_lm = alpha_lm Q_lm with alpha_mm = pmm_m and
// alpha_lm = A_lm alpha_{l-1,m}, so Q_mm = 1 and
//   Q_lm = z Q_{l-1,m} - beta_lm r^2 Q_{l-2,m},  beta_lm = B_lm / A_{l-1,m},
// and the pair table holds alpha_lm (c_{l,m}, c_{l,-m}) (three operations per
// term for the recurrence instead of four, none for the diagonal).
// `cs` is that table (shared memory), x, y, z already centred and scaled.
__device__ __forceinline__ float harmonic_cart(const float2 *cs, int lmax, float x, float y, float z) {
    const float r2 = x * x + y * y + z * z;
    float C = 1.f, S = 0.f, acc = 0.f;
    for (int m = 0; m <= lmax; ++m) {
        if (m > 0) {
            const float c2 = C * x - S * y;
            S = fmaf(S, x, C * y);
            C = c2;
        }
        int k = sh_pair(m, m);
        float q2 = 0.f, q1 = 1.f;
        float2 c = cs[k];
        float ac = c.x, as = c.y;
        for (int l = m + 1; l <= lmax; ++l) {
            ++k;
            const float q = fmaf(z, q1, -c_sh.beta[k] * r2 * q2);
            q2 = q1;
            q1 = q;
            c = cs[k];
            ac = fmaf(c.x, q, ac);
            as = fmaf(c.y, q, as);
        }
        acc = fmaf(ac, C, fmaf(as, S, acc));
    }
    return acc;
}

// The same with the degree fixed at compile time (coefficients beyond the
// data's lmax are zero in the pair table): every loop unrolls, so the
// recurrence constants are immediate constant-bank operands.
template <int L>
__device__ __forceinline__ float harmonic_cart_fixed(const float2 *cs, float x, float y, float z) {
    const float r2 = x * x + y * y + z * z;
    float C = 1.f, S = 0.f, acc = 0.f;
#pragma unroll
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            const float c2 = C * x - S * y;
            S = fmaf(S, x, C * y);
            C = c2;
        }
        float q2 = 0.f, q1 = 1.f;
        float2 c = cs[sh_pair(m, m)];
        float ac = c.x, as = c.y;
#pragma unroll
        for (int l = m + 1; l <= L; ++l) {
            const float q = fmaf(z, q1, -c_sh.beta[sh_pair(l, m)] * r2 * q2);
            q2 = q1;
            q1 = q;
            c = cs[sh_pair(l, m)];
            ac = fmaf(c.x, q, ac);
            as = fmaf(c.y, q, as);
        }
        acc = fmaf(ac, C, fmaf(as, S, acc));
    }
    return acc;
}

template <typename T>
__device__ __forceinline__ T dirichlet_eval(const DData &d, T x, T y, T z) {
    if (d.kind == kPointSource) {
        const T dx = x - pick<T>(d.x0[0], d.x0_f[0]), dy = y - pick<T>(d.x0[1], d.x0_f[1]),
                dz = z - pick<T>(d.x0[2], d.x0_f[2]);
        return pick<T>(d.strength / (4.0 * kPi), d.q_f) / sqrt(dx * dx + dy * dy + dz * dz);
    } else if (d.kind == kHarmonicSH) {
        return harmonic_eval<T>(d, x, y, z);
    }
    return pick<T>(d.constant, d.constant_f);
}

// ------------------------------------------------------------------ Green's functions
// Whole-sphere Dirichlet Green's function of B(c, a), local coordinates X = x - c,
// Y = y - c: free-space term minus the Kelvin image of charge a/|Y| at a^2 Y/|Y|^2,
//   G = (1/4pi) [ 1/|X - Y| - a / sqrt(Q) ],
//   Q = |X|^2|Y|^2 - 2a^2 X.Y + a^4 = (a^2 - |X||Y|)^2 + a^2 |X||Y| |Xh - Yh|^2,
// the second form (no cancellation near the rim) with Xh, Yh unit vectors.
template <typename T>
__device__ __forceinline__ T image_q(T a2, const T *X, T xn, const T *Y) {
    const T yn = sqrt(Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2]);
    const T p = xn * yn;
    const T t = a2 - p;
    if (xn == (T)0 || yn == (T)0) return t * t;
    // |X|Y| - Y|X||^2 / (|X||Y|) = |X||Y| |Xh - Yh|^2
    const T ux = X[0] * yn - Y[0] * xn, uy = X[1] * yn - Y[1] * xn, uz = X[2] * yn - Y[2] * xn;
    return t * t + a2 * (ux * ux + uy * uy + uz * uz) / p;
}

template <typename T>
__device__ __forceinline__ T green_ball(T a, const T *X, T xn, const T *Y) {
    const T dx = X[0] - Y[0], dy = X[1] - Y[1], dz = X[2] - Y[2];
    const T r = sqrt(dx * dx + dy * dy + dz * dz);
    const T Q = image_q<T>(a * a, X, xn, Y);
    return ((T)1 / r - a / sqrt(Q)) * (T)(0.25 / kPi);
}

// n_y . grad_Y G = (1/4pi) [ n.(X-Y)/|X-Y|^3 + a n.(|X|^2 Y - a^2 X) / Q^{3/2} ]
template <typename T>
__device__ __forceinline__ T green_ball_dny(T a, const T *X, T xn, const T *Y, const T *ny) {
    const T dx = X[0] - Y[0], dy = X[1] - Y[1], dz = X[2] - Y[2];
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T r = sqrt(r2);
    const T a2 = a * a;
    const T Q = image_q<T>(a2, X, xn, Y);
    const T sQ = sqrt(Q);
    const T xx = xn * xn;
    const T t1 = (ny[0] * dx + ny[1] * dy + ny[2] * dz) / (r2 * r);
    const T t2 = a * (xx * (ny[0] * Y[0] + ny[1] * Y[1] + ny[2] * Y[2]) -
                      a2 * (ny[0] * X[0] + ny[1] * X[1] + ny[2] * X[2])) / (Q * sQ);
    return (t1 + t2) * (T)(0.25 / kPi);
}

// d2G/dn_x dn_y of the whole-sphere Dirichlet Green's function of B(c, a), local
// coordinates, unit normals nx at X and ny at Y (the kernel of Eq. bw53, bw59):
//   (1/4pi) [ nx.ny/r^3 - 3 (D.nx)(D.ny)/r^5 + a ( (2 (X.nx)(Y.ny) - a^2 nx.ny) Q^-3/2
//             - 3 (|X|^2 Y.ny - a^2 X.ny)(|Y|^2 X.nx - a^2 Y.nx) Q^-5/2 ) ],  D = X - Y
__device__ __forceinline__ double green_ball_dnn(double a, const double *X, const double *nx, const double *Y,
                                                 const double *ny) {
    const double D[3] = {X[0] - Y[0], X[1] - Y[1], X[2] - Y[2]};
    const double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2], r = sqrt(r2);
    const double Dnx = D[0] * nx[0] + D[1] * nx[1] + D[2] * nx[2];
    const double Dny = D[0] * ny[0] + D[1] * ny[1] + D[2] * ny[2];
    const double nn = nx[0] * ny[0] + nx[1] * ny[1] + nx[2] * ny[2];
    const double XX = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    const double YY = Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2];
    const double XY = X[0] * Y[0] + X[1] * Y[1] + X[2] * Y[2];
    const double Xnx = X[0] * nx[0] + X[1] * nx[1] + X[2] * nx[2];
    const double Yny = Y[0] * ny[0] + Y[1] * ny[1] + Y[2] * ny[2];
    const double Xny = X[0] * ny[0] + X[1] * ny[1] + X[2] * ny[2];
    const double Ynx = Y[0] * nx[0] + Y[1] * nx[1] + Y[2] * nx[2];
    const double a2 = a * a;
    const double Q = XX * YY - 2.0 * a2 * XY + a2 * a2;
    const double sq = sqrt(Q);
    const double fr = nn / (r2 * r) - 3.0 * Dnx * Dny / (r2 * r2 * r);
    const double im = a * ((2.0 * Xnx * Yny - a2 * nn) / (Q * sq) -
                           3.0 * (XX * Yny - a2 * Xny) * (YY * Xnx - a2 * Ynx) / (Q * Q * sq));
    return (fr + im) / (4.0 * kPi);
}

// Poisson kernel of the ball, -dG/dn_y on |Y| = a: (a^2 - |X|^2) / (4 pi a |X - Y|^3)
template <typename T>
__device__ __forceinline__ T poisson_ball(T a, const T *X, const T *Y) {
    const T dx = X[0] - Y[0], dy = X[1] - Y[1], dz = X[2] - Y[2];
    const T r2 = dx * dx + dy * dy + dz * dz;
    const T xx = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    return (a * a - xx) / ((T)(4.0 * kPi) * a * r2 * sqrt(r2));
}

// ------------------------------------------------------------------ patches
enum PatchKind : int { kDisk = 0, kCap = 1, kWrapped = 2 };

// Local frame of a patch: n = outward normal of D at c; t1 = normalised
// projection of the coordinate axis least aligned with n (lowest index on
// ties); t2 = n x t1.
struct PatchFrame {
    double c[3], n[3], t1[3], t2[3];
    double a, R, theta_max, umax;
    int kind, status;
    double blo[3], bhi[3];   // wrapped patch: the obstacle box
    int npiece;              // wrapped patch: pieces (kMaxPieces per patch in the pieces array)
};

// A piece of a wrapped patch (the ball about a point of an obstacle face meets
// further faces of that box): a face rectangle cut by the ball's slice of the
// face plane, in polar coordinates about P (the point of the rectangle nearest
// the slice centre cf): rho <= rho_max(phi), phi in [sub[0], sub[nsub]], the
// angle cut where rho_max changes from one rectangle side or the circle to
// another.  Panels: rings in u = rho / rho_max, cnt[j] sectors in sub-range j.
constexpr int kMaxPieces = 6, kMaxSub = 16;
struct Piece {
    double P[2], cf[2], rlo[2], rhi[2], rf, fv;
    double Pl[3], Ul[3], Vl[3], nl[3];   // in the patch frame: P, the in-plane axes, the normal
    double sub[kMaxSub + 1];
    // what bounds a sub-range: the circle (stype 0), or a rectangle side (stype
    // 1) at distance sdist from P along the direction of angle svn
    double svn[kMaxSub], sdist[kMaxSub];
    double en[kMaxSub][3], et[kMaxSub][3];   // side-bounded: e(svn), e(svn + pi/2) in the patch frame, times sdist
    int stype[kMaxSub];
    int centred;   // P is the slice centre (rho_max = rf on circle-bounded sub-ranges)
    int ax, side, ua, va, onlo[2], onhi[2], nsub;
    int cnt[kMaxSub];
};

// rho_max(phi): from P along (cos phi, sin phi) to the circle, or to a
// rectangle side if nearer (the sides through P bound no ray of the range)
__device__ __forceinline__ double piece_rho(const Piece &q, double ph) {
    double e0, e1;
    sincos(ph, &e1, &e0);
    const double w0 = q.P[0] - q.cf[0], w1 = q.P[1] - q.cf[1];
    const double we = w0 * e0 + w1 * e1, ww = w0 * w0 + w1 * w1;
    double r = -we + sqrt(fmax(0.0, we * we - ww + q.rf * q.rf));
    if (e0 > 0.0 && !q.onhi[0]) r = fmin(r, (q.rhi[0] - q.P[0]) / e0);
    if (e0 < 0.0 && !q.onlo[0]) r = fmin(r, (q.rlo[0] - q.P[0]) / e0);
    if (e1 > 0.0 && !q.onhi[1]) r = fmin(r, (q.rhi[1] - q.P[1]) / e1);
    if (e1 < 0.0 && !q.onlo[1]) r = fmin(r, (q.rlo[1] - q.P[1]) / e1);
    return r;
}

// point of a piece at (u, v) = (rho / rho_max, phi), in the patch frame:
// Y = Pl + u rho_max(v) (cos v Ul + sin v Vl), its normal, J = u rho_max(v)^2
template <typename T>
__device__ __forceinline__ void wrapped_point(const Piece &q, T u, T v, T *Y, T *nl, T &J) {
    const double r = piece_rho(q, (double)v);
    double sv, cv;
    sincos((double)v, &sv, &cv);
    const double ur = (double)u * r;
    for (int d = 0; d < 3; ++d) {
        Y[d] = (T)(q.Pl[d] + ur * (cv * q.Ul[d] + sv * q.Vl[d]));
        nl[d] = (T)q.nl[d];
    }
    J = (T)((double)u * r * r);
}

// The quadrature parameters of a panel of sub-range j: (u, v) on a sub-range
// bounded by the circle (rho_max constant there), (u, t) with t = tan(v -
// svn) on one bounded by a rectangle side, where the point P + u sdist (e_n +
// t e_t) is bilinear in (u, t) (J = sdist^2 u): the same panel, but the
// integrands stay smooth however close the side's pole angle svn +- pi/2
// comes to the sub-range.
template <typename T>
__device__ __forceinline__ void wrapped_point_q(const Piece &q, int j, T u, T w, T *Y, T *nl, T &J) {
    if (q.stype[j] == 0) {
        if (!q.centred) {
            wrapped_point<T>(q, u, w, Y, nl, J);
            return;
        }
        double sv, cv;
        sincos((double)w, &sv, &cv);
        const double ur = (double)u * q.rf;
        for (int d = 0; d < 3; ++d) {
            Y[d] = (T)(q.Pl[d] + ur * (cv * q.Ul[d] + sv * q.Vl[d]));
            nl[d] = (T)q.nl[d];
        }
        J = (T)((double)u * q.rf * q.rf);
        return;
    }
    const double ud = (double)u, wt = (double)w;
    for (int d = 0; d < 3; ++d) {
        Y[d] = (T)(q.Pl[d] + ud * (q.en[j][d] + wt * q.et[j][d]));
        nl[d] = (T)q.nl[d];
    }
    J = (T)(q.sdist[j] * q.sdist[j] * ud);
}

// the direction of a wrapped panel's quadrature line at parameter w (the point
// is Pl + u B, the Jacobian u Jf): separable in (u, w)
__device__ __forceinline__ void wrapped_line(const Piece &q, int j, double w, double *B, double &Jf) {
    if (q.stype[j] == 0) {
        const double r = q.centred ? q.rf : piece_rho(q, w);
        double sv, cv;
        sincos(w, &sv, &cv);
        for (int d = 0; d < 3; ++d) B[d] = r * (cv * q.Ul[d] + sv * q.Vl[d]);
        Jf = r * r;
    } else {
        for (int d = 0; d < 3; ++d) B[d] = q.en[j][d] + w * q.et[j][d];
        Jf = q.sdist[j] * q.sdist[j];
    }
}

// point of the patch at parameters (u, v), local coordinates (t1, t2, n),
// its local unit normal and the area Jacobian.  Disk: Y = u (cos v, sin v, 0),
// J = u.  Cap (boundary sphere of radius R through c, centre c - R n):
// Y = (R sin u cos v, R sin u sin v, -2R sin^2(u/2)), J = R^2 sin u.
template <typename T>
__device__ __forceinline__ void patch_point(int kind, T R, T u, T v, T *Y, T *nl, T &J) {
    T sv, cv;
    sincos(v, &sv, &cv);
    if (kind == kDisk) {
        Y[0] = u * cv; Y[1] = u * sv; Y[2] = (T)0;
        nl[0] = (T)0; nl[1] = (T)0; nl[2] = (T)1;
        J = u;
    } else {
        T su, cu;
        sincos(u, &su, &cu);
        const T sh = sin((T)0.5 * u);
        Y[0] = R * su * cv; Y[1] = R * su * sv; Y[2] = (T)-2 * R * sh * sh;
        nl[0] = su * cv; nl[1] = su * sv; nl[2] = cu;
        J = R * R * su;
    }
}

}  // namespace dtn
