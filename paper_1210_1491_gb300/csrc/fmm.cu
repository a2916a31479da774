// fmm.cu -- fast multipole evaluation of the integral representation Eq. bw03
// (Sec. 6: once the patches have their Neumann data, the potential anywhere is
// one application of the fast multipole method of Greengard and Rokhlin to the
// panel sources).
//
// Sources.  Panel p is a charge c_p = area_p q_p / 4pi and a dipole
// d_p = -area_p g_p n_p / 4pi at its collocation point y_p, so that
//   u(t) = sum_p [ c_p / |t - y_p| + d_p.(t - y_p) / |t - y_p|^3 ],
// the panel-midpoint sum of the direct kernels in potential.cu.
//
// Expansions.  Complex solid harmonics
//   R_n^m(x) = r^n P_n^m(cos th) e^{i m ph} / (n+m)!,
//   S_n^m(x) = (n-m)! P_n^m(cos th) e^{i m ph} / r^{n+1},
// P_n^m without the Condon-Shortley phase and A_n^{-m} = (-1)^m conj(A_n^m), so
// that 1/|x - y| = sum_{n,|m|<=n} S_n^m(x) conj(R_n^m(y)) for |y| < |x|.  The
// fields are real, so every expansion obeys the same symmetry and only m >= 0
// is stored ((P+1)(P+2)/2 coefficients, index n(n+1)/2 + m).  With centres c
// (multipole) and z (local) the operators follow from the addition theorems
// R_n^m(a + b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b) and
//   S_n^m(a + b) = sum_{k,l} (-1)^k conj(R_k^l(b)) S_{n+k}^{m+l}(a):
//   P2M  M_n^m = sum_p conj(c_p R_n^m(v) + d_p.grad R_n^m(v)),  v = y_p - c,
//        grad: (dx + i dy)/2 R_{n-1}^{m-1} - (dx - i dy)/2 R_{n-1}^{m+1} + dz R_{n-1}^m
//   M2M  M'_n^m = sum_{k,l} conj(R_k^l(c - c')) M_{n-k}^{m-l}
//   M2L  L_n^m = (-1)^{n+m} sum_{j,k} S_{j+n}^{k-m}(z - c) M_j^k
//   L2L  L'_k^l = sum_{n>=k,m} L_n^m R_{n-k}^{m-l}(z' - z)
//   L2P  u(t) = sum_{n,m} R_n^m(t - z) L_n^m
// Each expansion is stored scaled by its cell's half-width h (M / h^n, L h^n),
// which keeps every FP32 coefficient of order one.
//
// Trees and traversal.  Sources and targets get separate adaptive octrees over
// one bounding cube: points sorted by 63-bit Morton keys, a cell split while it
// holds more than the leaf size (cells in level order, the children of a cell
// contiguous).  A dual-tree traversal, level-synchronous on the GPU, sorts every
// (target cell, source cell) pair into an M2L pair when (r_T + r_S) < theta |z - c|
// (r the radius about the cell centre of a ball holding the cell's points: exact
// for leaves, bounded through the children above), a P2P pair when both are
// leaves, and otherwise splits the larger cell.  Each target point then receives every source exactly once,
// through one M2L (plus the L2L chain below it) or one P2P pair.
//
// Precision: expansions and pair terms in FP32, centre differences in FP64,
// per-target sums in FP64 (the source and target offsets of a P2P pair are
// taken from the target leaf's centre, so their difference keeps its digits).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kFmmMaxOrder = 16;
constexpr int kMortonBits = 21;
constexpr int kNcMax = (kFmmMaxOrder + 1) * (kFmmMaxOrder + 2) / 2;               // 153
constexpr int kNsMax = (2 * kFmmMaxOrder + 1) * (2 * kFmmMaxOrder + 2) / 2;       // 561
constexpr int kOwnMax = (kNcMax + 31) / 32;                                        // outputs per lane
constexpr int kCellWarps = 4;                                                      // warps per CTA
constexpr int kBboxBlocks = 256;

struct FCell {
    double c[3];            // centre
    double r;               // radius about c of a ball holding the cell's points
    uint64_t key;           // Morton prefix, 3 bits per level
    int32_t start, count;   // points [start, start + count) in Morton order
    int32_t child, nchild;  // first child (next level, contiguous); -1 for a leaf
    int32_t level, pad;
};

__host__ __device__ inline int tri(int n, int m) { return n * (n + 1) / 2 + m; }

__device__ inline float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a += b c
__device__ inline void cmac(float2 &a, float2 b, float2 c) {
    a.x = fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(b.y, c.x, a.y));
}
// a += s c, s real
__device__ inline void rmac(float2 &a, float s, float2 c) {
    a.x = fmaf(s, c.x, a.x);
    a.y = fmaf(s, c.y, a.y);
}
// a += conj(b) c
__device__ inline void cmac_cb(float2 &a, float2 b, float2 c) {
    a.x = fmaf(b.x, c.x, fmaf(b.y, c.y, a.x));
    a.y = fmaf(b.x, c.y, fmaf(-b.y, c.x, a.y));
}

// (n, m) of the stored coefficient idx = n(n+1)/2 + m
__device__ inline void tri_nm(int idx, int &n, int &m) {
    n = (int)((sqrtf(8.0f * idx + 1.0f) - 1.0f) * 0.5f);
    while (tri(n + 1, 0) <= idx) ++n;
    while (tri(n, 0) > idx) --n;
    m = idx - tri(n, 0);
}

// Column m (R_m^m .. R_P^m) of the regular harmonics at v, into tab[tri(n, m)]:
//   R_m^m = (x + i y)^m / (2^m m!),  R_{m+1}^m = z R_m^m,
//   R_n^m = ((2n-1) z R_{n-1}^m - r^2 R_{n-2}^m) / ((n+m)(n-m)).
__device__ inline void regular_column(float2 *tab, int m, int P, float x, float y, float z) {
    const float r2 = fmaf(x, x, fmaf(y, y, z * z));
    float2 rmm = make_float2(1.0f, 0.0f);
    for (int k = 1; k <= m; ++k) rmm = cscale(cmul(rmm, make_float2(x, y)), 0.5f / (float)k);
    if (m > P) return;
    tab[tri(m, m)] = rmm;
    float2 a = make_float2(0.0f, 0.0f), b = rmm;
    for (int n = m + 1; n <= P; ++n) {
        const float inv = 1.0f / (float)((n + m) * (n - m));
        const float2 c = make_float2(((2 * n - 1) * z * b.x - r2 * a.x) * inv, ((2 * n - 1) * z * b.y - r2 * a.y) * inv);
        tab[tri(n, m)] = c;
        a = b;
        b = c;
    }
}

// Column m (S_m^m .. S_N^m) of the singular harmonics at v:
//   S_0^0 = 1/r,  S_m^m = (2m-1) (x + i y) / r^2 S_{m-1}^{m-1},  S_{m+1}^m = (2m+1) z / r^2 S_m^m,
//   S_n^m = ((2n-1) z S_{n-1}^m - (n+m-1)(n-m-1) S_{n-2}^m) / r^2.
__device__ inline void singular_column(float2 *tab, int m, int N, float x, float y, float z) {
    const float r2 = fmaf(x, x, fmaf(y, y, z * z));
    const float ir2 = 1.0f / r2;
    float2 smm = make_float2(rsqrtf(r2), 0.0f);
    for (int k = 1; k <= m; ++k) smm = cscale(cmul(smm, make_float2(x, y)), (float)(2 * k - 1) * ir2);
    tab[tri(m, m)] = smm;
    float2 a = make_float2(0.0f, 0.0f), b = smm;
    for (int n = m + 1; n <= N; ++n) {
        const float f = (float)((n + m - 1) * (n - m - 1));
        const float2 c = make_float2(((2 * n - 1) * z * b.x - f * a.x) * ir2, ((2 * n - 1) * z * b.y - f * a.y) * ir2);
        tab[tri(n, m)] = c;
        a = b;
        b = c;
    }
}

// A_n^m for any |m| <= n from the stored m >= 0 half
__device__ inline float2 sym_get(const float2 *tab, int n, int m) {
    if (m >= 0) return tab[tri(n, m)];
    const float2 v = tab[tri(n, -m)];
    return ((-m) & 1) ? make_float2(-v.x, v.y) : make_float2(v.x, -v.y);
}

// ------------------------------------------------------------------ tree build

// Bounding box partials per block; an index outside [0, n_total) sets *bad and
// is skipped (it is never dereferenced).
__global__ void fmm_bbox_kernel(int64_t n, const double *__restrict__ x, const int64_t *__restrict__ index,
                                int64_t n_total, double *__restrict__ part, int *__restrict__ bad) {
    __shared__ double red[6][256];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = index ? index[i] : i;
        if (p < 0 || p >= n_total) {
            atomicOr(bad, 1);
            continue;
        }
        for (int a = 0; a < 3; ++a) {
            const double v = x[3 * p + a];
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    }
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = lo[a];
        red[3 + a][threadIdx.x] = hi[a];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int a = 0; a < 3; ++a) {
                red[a][threadIdx.x] = fmin(red[a][threadIdx.x], red[a][threadIdx.x + o]);
                red[3 + a][threadIdx.x] = fmax(red[3 + a][threadIdx.x], red[3 + a][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

__device__ inline uint64_t spread21(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ inline uint32_t quantise(double v, double lo, double scale) {
    const double q = floor((v - lo) * scale);
    return (uint32_t)fmin(fmax(q, 0.0), (double)((1u << kMortonBits) - 1));
}

// key = interleaved (x, y, z) bits, x most significant; val = the point's id
__global__ void fmm_morton_kernel(int64_t n, const double *__restrict__ x, const int64_t *__restrict__ index,
                                  double lx, double ly, double lz, double scale, uint64_t *__restrict__ key,
                                  int32_t *__restrict__ val) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = index ? index[i] : i;
    key[i] = spread21(quantise(x[3 * p], lx, scale)) << 2 | spread21(quantise(x[3 * p + 1], ly, scale)) << 1 |
             spread21(quantise(x[3 * p + 2], lz, scale));
    val[i] = (int32_t)p;
}

// One thread per (cell of this level, octant): the run of the cell's points
// whose next Morton digit is the octant (points are sorted, so within a cell
// the digit is non-decreasing).
__global__ void fmm_split_kernel(const FCell *__restrict__ cells, int64_t c0, int64_t nc,
                                 const uint64_t *__restrict__ keys, int ncrit, int max_level,
                                 int32_t *__restrict__ flag, int32_t *__restrict__ lo, int32_t *__restrict__ hi) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 8 * nc) return;
    const FCell &cell = cells[c0 + i / 8];
    const int d = (int)(i % 8);
    if (cell.count <= ncrit || cell.level >= max_level) {
        flag[i] = 0;
        return;
    }
    const int shift = 3 * (kMortonBits - cell.level - 1);
    const int s0 = cell.start, s1 = cell.start + cell.count;
    auto lower = [&](int dd) {
        int a = s0, b = s1;
        while (a < b) {
            const int mid = (a + b) >> 1;
            if ((int)((keys[mid] >> shift) & 7u) < dd) a = mid + 1;
            else b = mid;
        }
        return a;
    };
    const int l = lower(d), h = (d == 7) ? s1 : lower(d + 1);
    flag[i] = h > l ? 1 : 0;
    lo[i] = l;
    hi[i] = h;
}

__global__ void fmm_emit_kernel(FCell *__restrict__ cells, int64_t c0, int64_t nc, int64_t c_next,
                                const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                                const int32_t *__restrict__ lo, const int32_t *__restrict__ hi, double h_child) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 8 * nc) return;
    const int64_t p = c0 + i / 8;
    const int d = (int)(i % 8);
    if (d == 0) {
        int cnt = 0;
        for (int k = 0; k < 8; ++k) cnt += flag[i + k];
        cells[p].child = cnt ? (int32_t)(c_next + pos[i]) : -1;
        cells[p].nchild = cnt;
    }
    if (!flag[i]) return;
    FCell ch;
    ch.c[0] = cells[p].c[0] + ((d & 4) ? h_child : -h_child);
    ch.c[1] = cells[p].c[1] + ((d & 2) ? h_child : -h_child);
    ch.c[2] = cells[p].c[2] + ((d & 1) ? h_child : -h_child);
    ch.key = cells[p].key << 3 | (uint64_t)d;
    ch.start = lo[i];
    ch.count = hi[i] - lo[i];
    ch.child = -1;
    ch.nchild = 0;
    ch.level = cells[p].level + 1;
    ch.pad = 0;
    ch.r = 0.0;
    cells[c_next + pos[i]] = ch;
}

// sources in Morton order: FP64 position, (dipole, charge) as float4
__global__ void fmm_source_kernel(int64_t n, const int32_t *__restrict__ val, const double *__restrict__ xyz,
                                  const double *__restrict__ nrm, const double *__restrict__ area,
                                  const double *__restrict__ q, const double *__restrict__ g,
                                  double *__restrict__ spos, float4 *__restrict__ sdat) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t p = val[i];
    const double inv4pi = 0.25 / kPi;
    const double c = area[p] * q[p] * inv4pi, dd = -area[p] * g[p] * inv4pi;
    spos[3 * i] = xyz[3 * p];
    spos[3 * i + 1] = xyz[3 * p + 1];
    spos[3 * i + 2] = xyz[3 * p + 2];
    sdat[i] = make_float4((float)(dd * nrm[3 * p]), (float)(dd * nrm[3 * p + 1]), (float)(dd * nrm[3 * p + 2]),
                          (float)c);
}

// Cell radii, one level at a time from the deepest, a warp per cell: a leaf
// takes the largest distance of its points from its centre (FP64, points
// through the optional id list), a split cell max over children of
// |c_child - c| + r_child.
__global__ void fmm_radius_kernel(FCell *__restrict__ cells, int64_t c0, int64_t ncell,
                                  const double *__restrict__ x, const int32_t *__restrict__ ids) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= ncell) return;
    FCell &C = cells[c0 + i];
    double r = 0.0;
    if (C.child < 0) {
        double r2 = 0.0;
        for (int k = C.start + lane; k < C.start + C.count; k += 32) {
            const int64_t p = ids ? ids[k] : k;
            const double dx = x[3 * p] - C.c[0], dy = x[3 * p + 1] - C.c[1], dz = x[3 * p + 2] - C.c[2];
            r2 = fmax(r2, dx * dx + dy * dy + dz * dz);
        }
        r = sqrt(r2);
    } else if (lane < C.nchild) {
        const FCell &D = cells[C.child + lane];
        const double dx = D.c[0] - C.c[0], dy = D.c[1] - C.c[1], dz = D.c[2] - C.c[2];
        r = sqrt(dx * dx + dy * dy + dz * dz) + D.r;
    }
    for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) C.r = r;
}

// ------------------------------------------------------------------ upward pass

struct FmmShared {
    float2 tab[kNsMax];   // R or S table
    float2 exp[kNcMax];   // a staged expansion
};

// P2M: one warp per source leaf; the warp builds each source's regular table
// (lane m computes column m) and every lane accumulates the coefficients it owns.
// Also writes each source's FP32 offset from its leaf centre with its charge
// (srel), the form the leaf-pair sums read.
__global__ void __launch_bounds__(32 * kCellWarps) fmm_p2m_kernel(
    const FCell *__restrict__ cells, int64_t ncell, const double *__restrict__ spos,
    const float4 *__restrict__ sdat, double half_w0, int P, float2 *__restrict__ M, float4 *__restrict__ srel) {
    __shared__ FmmShared sh[kCellWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ci = blockIdx.x * (int64_t)kCellWarps + wid;
    if (ci >= ncell) return;
    const FCell cell = cells[ci];
    if (cell.child >= 0) return;
    const int nc = tri(P + 1, 0);
    const double ihd = ldexp(1.0 / half_w0, cell.level);   // 1/h, a power-of-two scaling of 1/half_w0
    const float ih = (float)ihd;
    float2 acc[kOwnMax];
    int on[kOwnMax], om[kOwnMax];
#pragma unroll
    for (int r = 0; r < kOwnMax; ++r) {
        acc[r] = make_float2(0.0f, 0.0f);
        const int idx = lane + 32 * r;
        if (idx < nc) tri_nm(idx, on[r], om[r]);
        else on[r] = om[r] = 0;
    }
    float2 *tab = sh[wid].tab;
    for (int s = cell.start + lane; s < cell.start + cell.count; s += 32)
        srel[s] = make_float4((float)(spos[3 * s] - cell.c[0]), (float)(spos[3 * s + 1] - cell.c[1]),
                              (float)(spos[3 * s + 2] - cell.c[2]), sdat[s].w);
    // G sources per pass: lane group g = lane / (P+1) builds source g's table, lane m = lane % (P+1) its column
    const int G = min(32 / (P + 1), kNsMax / nc);
    const int grp = lane / (P + 1), col = lane % (P + 1);
    for (int s0 = cell.start; s0 < cell.start + cell.count; s0 += G) {
        const int ng = min(G, cell.start + cell.count - s0);
        __syncwarp();
        if (grp < ng) {
            const int s = s0 + grp;
            const float vx = (float)((spos[3 * s] - cell.c[0]) * ihd), vy = (float)((spos[3 * s + 1] - cell.c[1]) * ihd),
                        vz = (float)((spos[3 * s + 2] - cell.c[2]) * ihd);
            regular_column(tab + grp * nc, col, P, vx, vy, vz);
        }
        __syncwarp();
        for (int g = 0; g < ng; ++g) {
            const float2 *tg = tab + g * nc;
            const float4 sd = sdat[s0 + g];
            const float dx = sd.x * ih, dy = sd.y * ih, dz = sd.z * ih, c = sd.w;
            const float2 dp = make_float2(0.5f * dx, 0.5f * dy);    // (dx + i dy) / 2
            const float2 dm = make_float2(0.5f * dx, -0.5f * dy);   // (dx - i dy) / 2
#pragma unroll
            for (int r = 0; r < kOwnMax; ++r) {
                if (lane + 32 * r >= nc) break;
                const int n = on[r], m = om[r];
                float2 t = cscale(tg[tri(n, m)], c);
                if (n >= 1) {
                    // R_{n-1}^{m-1} (m = 0: -conj(R_{n-1}^1)), R_{n-1}^{m+1}, R_{n-1}^m
                    float2 rm1 = make_float2(0.0f, 0.0f);
                    if (m >= 1) rm1 = tg[tri(n - 1, m - 1)];
                    else if (n - 1 >= 1) { const float2 v = tg[tri(n - 1, 1)]; rm1 = make_float2(-v.x, v.y); }
                    cmac(t, dp, rm1);
                    if (m + 1 <= n - 1) { const float2 v = tg[tri(n - 1, m + 1)]; cmac(t, make_float2(-dm.x, -dm.y), v); }
                    if (m <= n - 1) { const float2 v = tg[tri(n - 1, m)]; t.x = fmaf(dz, v.x, t.x); t.y = fmaf(dz, v.y, t.y); }
                }
                acc[r] = cadd(acc[r], cconj(t));
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kOwnMax; ++r)
        if (lane + 32 * r < nc) M[ci * nc + lane + 32 * r] = acc[r];
}

// M2M for the split cells of one level: M'_n^m = sum conj(R_k^l(d)) 2^{-(n-k)} M_{n-k}^{m-l},
// d = (child centre - parent centre) / h_parent.
__global__ void __launch_bounds__(32 * kCellWarps) fmm_m2m_kernel(
    const FCell *__restrict__ cells, int64_t c0, int64_t ncell, double half_w0, int P, float2 *__restrict__ M) {
    __shared__ FmmShared sh[kCellWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ci = c0 + blockIdx.x * (int64_t)kCellWarps + wid;
    if (ci >= c0 + ncell) return;
    const FCell cell = cells[ci];
    if (cell.child < 0) return;
    const int nc = tri(P + 1, 0);
    const double ihd = ldexp(1.0 / half_w0, cell.level);
    float2 acc[kOwnMax];
    int on[kOwnMax], om[kOwnMax];
#pragma unroll
    for (int r = 0; r < kOwnMax; ++r) {
        acc[r] = make_float2(0.0f, 0.0f);
        const int idx = lane + 32 * r;
        if (idx < nc) tri_nm(idx, on[r], om[r]);
        else on[r] = om[r] = 0;
    }
    float2 *tab = sh[wid].tab, *ex = sh[wid].exp;
    for (int k = 0; k < cell.nchild; ++k) {
        const int64_t cc = cell.child + k;
        const float dx = (float)((cells[cc].c[0] - cell.c[0]) * ihd), dy = (float)((cells[cc].c[1] - cell.c[1]) * ihd),
                    dz = (float)((cells[cc].c[2] - cell.c[2]) * ihd);
        __syncwarp();
        if (lane <= P) regular_column(tab, lane, P, dx, dy, dz);
        for (int e = lane; e < nc; e += 32) ex[e] = M[cc * nc + e];
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kOwnMax; ++r) {
            if (lane + 32 * r >= nc) break;
            const int n = on[r], m = om[r];
            float2 s = make_float2(0.0f, 0.0f);
            for (int kk = 0; kk <= n; ++kk) {
                const int nn = n - kk;
                const float sc = ldexpf(1.0f, -nn);
                const int l0 = max(-kk, m - nn), l1 = min(kk, m + nn);
                for (int l = l0; l <= l1; ++l) {
                    const float2 rv = sym_get(tab, kk, l);
                    const float2 mv = sym_get(ex, nn, m - l);
                    cmac_cb(s, cscale(rv, sc), mv);
                }
            }
            acc[r] = cadd(acc[r], s);
        }
    }
#pragma unroll
    for (int r = 0; r < kOwnMax; ++r)
        if (lane + 32 * r < nc) M[ci * nc + lane + 32 * r] = acc[r];
}

// ------------------------------------------------------------------ traversal

struct DttCounters {
    unsigned long long next, m2l, p2p, p2p_terms, overflow;
};

// One thread per frontier pair; appends are aggregated per warp (one atomic per
// list per warp, offsets by warp prefix sums).
__global__ void fmm_dtt_kernel(const int2 *__restrict__ front, int64_t nf, const FCell *__restrict__ tc,
                               const FCell *__restrict__ sc, double theta2, int2 *__restrict__ next,
                               int64_t cap_next, uint64_t *__restrict__ m2l, int64_t cap_m2l,
                               uint64_t *__restrict__ p2p, int64_t cap_p2p, DttCounters *__restrict__ cnt) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < nf;
    int2 pr = make_int2(0, 0);
    int kind = -1;   // 0 M2L, 1 P2P, 2 split
    int first = 0, nch = 0;
    bool split_t = false;
    unsigned long long terms = 0;
    if (valid) {
        pr = front[i];
        const FCell &T = tc[pr.x];
        const FCell &S = sc[pr.y];
        const double rt = T.r, rs = S.r;
        const double dx = T.c[0] - S.c[0], dy = T.c[1] - S.c[1], dz = T.c[2] - S.c[2];
        const double d2 = dx * dx + dy * dy + dz * dz;
        const bool tleaf = T.child < 0, sleaf = S.child < 0;
        if ((rt + rs) * (rt + rs) < theta2 * d2) {
            kind = 0;
        } else if (tleaf && sleaf) {
            kind = 1;
            terms = (unsigned long long)T.count * (unsigned long long)S.count;
        } else {
            kind = 2;
            split_t = sleaf || (!tleaf && rt >= rs);
            first = split_t ? T.child : S.child;
            nch = split_t ? T.nchild : S.nchild;
        }
    }
    const uint64_t key = (uint64_t)(uint32_t)pr.x << 32 | (uint32_t)pr.y;
    // M2L and P2P: one slot each
    for (int k = 0; k < 2; ++k) {
        const unsigned mask = __ballot_sync(0xffffffffu, kind == k);
        if (!mask) continue;
        const int leader = __ffs(mask) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(k == 0 ? &cnt->m2l : &cnt->p2p, (unsigned long long)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (kind == k) {
            const int64_t slot = (int64_t)base + __popc(mask & ((1u << lane) - 1u));
            if (slot < (k == 0 ? cap_m2l : cap_p2p)) (k == 0 ? m2l : p2p)[slot] = key;
            else cnt->overflow = 1;
        }
    }
    // P2P pair terms (statistics)
    unsigned long long tsum = terms;
    for (int o = 16; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
    if (lane == 0 && tsum) atomicAdd(&cnt->p2p_terms, tsum);
    // splits: nch slots each, warp prefix sum
    int incl = nch;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&cnt->next, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (nch) {
            const int64_t at = (int64_t)base + incl - nch;
            if (at + nch <= cap_next) {
                for (int c = 0; c < nch; ++c)
                    next[at + c] = split_t ? make_int2(first + c, pr.y) : make_int2(pr.x, first + c);
            } else {
                cnt->overflow = 1;
            }
        }
    }
}

// CSR offsets of a list of (target << 32 | source) keys sorted ascending
__global__ void fmm_csr_kernel(int64_t ncell, const uint64_t *__restrict__ keys, int64_t n, int64_t *__restrict__ off) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t > ncell) return;
    const uint64_t want = (uint64_t)t << 32;
    int64_t a = 0, b = n;
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (keys[mid] < want) a = mid + 1;
        else b = mid;
    }
    off[t] = a;
}

// ------------------------------------------------------------------ downward pass

// M2L: one warp per target cell, over its sorted source list.  With phi the
// azimuth of v = (z - c)/rho, S_N^l(v) = e^{i l phi} s_N^l where s are the
// singular harmonics at (|v_xy|, 0, v_z), which are real; so
//   L_n^m += (-1)^{n+m} (h_T/rho)^n / rho e^{-i m phi}
//            sum_j sum_{k=-j}^{j} s_{j+n}^{k-m} (h_S/rho)^j M_j^k e^{i k phi},
// rho = max(h_T, h_S): a real table times the turned coefficients (half the
// multiply-adds of the complex sum).  For each source the warp writes s to
// degree 2P and the turned, scaled coefficients as full tables (orders -N..N at
// index N^2 + N + l, the negative orders from the symmetries), contiguous in k.
// A lane owns three outputs (n, m0), (n, m0+1), (n, m0+2): walking k upwards,
// the s value loaded for (n, m0) at k serves (n, m0+1) at k+1 and (n, m0+2) at
// k+2, so each step loads one s value and one (broadcast) M value for three
// real-by-complex products.  Outputs past m = n are computed on in-bounds
// padding and dropped.  L is zeroed before the launch; cells without pairs are
// skipped.
constexpr int kM2lBlock = 3;
constexpr int kM2lTasksMax = 2;   // rounds of 32 lanes: sum_n ceil((n+1)/3) <= 64 for P <= 16
constexpr int kSPad = 2;          // entries before the S table (k - m0 - 2 >= -2 - N)

struct M2lShared {
    float s[kSPad + (2 * kFmmMaxOrder + 1) * (2 * kFmmMaxOrder + 1)];
    float2 m[(kFmmMaxOrder + 1) * (kFmmMaxOrder + 1)];
};

// task t -> (n, m0): n ascending, m0 = 0, 3, 6, ... <= n; false past the last
__device__ inline bool m2l_task(int t, int P, int &n, int &m0) {
    for (n = 0; n <= P; ++n) {
        const int c = (n + kM2lBlock) / kM2lBlock;
        if (t < c) {
            m0 = kM2lBlock * t;
            return true;
        }
        t -= c;
    }
    return false;
}

// The geometry of each accepted pair, once per pair (the M2L kernel's lanes would
// otherwise each redo it, on GB300's narrow FP64 pipe): the translation z - c
// in units of the finer cell's half-width, that scale, and the two cells'
// level offsets from the finer level.
struct M2lGeo {
    float v[3], fr;
    int bt, bs;
};

__global__ void fmm_m2lgeo_kernel(int64_t n, const uint64_t *__restrict__ list, const FCell *__restrict__ tc,
                                  const FCell *__restrict__ sc, double half_w0, M2lGeo *__restrict__ geo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const uint64_t key = list[e];
    const FCell &T = tc[(int64_t)(key >> 32)];
    const FCell &Sc = sc[(int64_t)(uint32_t)(key & 0xffffffffu)];
    const int lt = T.level, ls = Sc.level;
    const int lr = min(lt, ls);
    const double irho = ldexp(1.0 / half_w0, lr);
    M2lGeo G;
    G.v[0] = (float)((T.c[0] - Sc.c[0]) * irho);
    G.v[1] = (float)((T.c[1] - Sc.c[1]) * irho);
    G.v[2] = (float)((T.c[2] - Sc.c[2]) * irho);
    G.fr = (float)irho;
    G.bt = lt - lr;
    G.bs = ls - lr;
    geo[e] = G;
}

// Persistent warps: each takes the next target cell from *queue (L is zeroed
// before the launch, so cells without M2L pairs are skipped).
// PT > 0: the order is the compile-time PT (the j and k loops unroll fully;
// instantiated for P = 8 and 10, where one round of lanes holds all outputs);
// PT = 0: the runtime order P.
template <int PT>
__global__ void __launch_bounds__(32 * kCellWarps) fmm_m2l_kernel(
    const FCell *__restrict__ tc, int64_t ntc, const FCell *__restrict__ sc, const int64_t *__restrict__ off,
    const uint64_t *__restrict__ list, const M2lGeo *__restrict__ geo, int P, const float2 *__restrict__ M,
    float2 *__restrict__ L, unsigned long long *__restrict__ queue) {
    if (PT > 0) P = PT;
    __shared__ M2lShared sh[kCellWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nc = tri(P + 1, 0);
    int tn[kM2lTasksMax], tm[kM2lTasksMax];
    bool tv[kM2lTasksMax];
#pragma unroll
    for (int r = 0; r < kM2lTasksMax; ++r) {
        tv[r] = m2l_task(lane + 32 * r, P, tn[r], tm[r]);
        if (!tv[r]) tn[r] = tm[r] = 0;
    }
    const bool round2 = __any_sync(0xffffffffu, tv[1]);
    float *S = sh[wid].s + kSPad;
    float2 *Mf = sh[wid].m;
    if (lane < kSPad) sh[wid].s[lane] = 0.0f;
    for (;;) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(queue, 1ull);
    const int64_t ti = (int64_t)__shfl_sync(0xffffffffu, qi, 0);
    if (ti >= ntc) break;
    const int64_t e0 = off[ti], e1 = off[ti + 1];
    if (e0 == e1) continue;
    float2 acc[kM2lTasksMax][kM2lBlock];
#pragma unroll
    for (int r = 0; r < kM2lTasksMax; ++r)
#pragma unroll
        for (int d = 0; d < kM2lBlock; ++d) acc[r][d] = make_float2(0.0f, 0.0f);
    for (int64_t e = e0; e < e1; ++e) {
        const int64_t si = (int64_t)(uint32_t)(list[e] & 0xffffffffu);
        const M2lGeo G = geo[e];
        const float vx = G.v[0], vy = G.v[1], vz = G.v[2];
        const int bt = G.bt, bs = G.bs;
        // azimuth of z - c taken out: S_N^l(v) = e^{i l phi} s_N^l with s the (real)
        // singular harmonics at (rho_xy, 0, vz); the source's coefficients are
        // turned by e^{i k phi} and each output by e^{-i m phi}
        const float rxy = sqrtf(fmaf(vx, vx, vy * vy));
        const float2 eph = rxy > 0.0f ? make_float2(vx / rxy, vy / rxy) : make_float2(1.0f, 0.0f);
        __syncwarp();
        for (int m = lane; m <= 2 * P; m += 32) {
            // column m of s, both signs of the order (s_N^{-m} = (-1)^m s_N^m)
            const float r2 = fmaf(rxy, rxy, vz * vz);
            const float ir2 = 1.0f / r2;
            float smm = rsqrtf(r2);
            for (int k = 1; k <= m; ++k) smm *= (float)(2 * k - 1) * rxy * ir2;
            const float sg = (m & 1) ? -1.0f : 1.0f;
            float a = 0.0f, b = smm;
            for (int n = m; n <= 2 * P; ++n) {
                if (n > m) {
                    const float c = ((2 * n - 1) * vz * b - (float)((n + m - 1) * (n - m - 1)) * a) * ir2;
                    a = b;
                    b = c;
                }
                S[n * n + n + m] = b;
                if (m) S[n * n + n - m] = sg * b;
            }
        }
        for (int q = lane; q < nc; q += 32) {
            int n, m;
            tri_nm(q, n, m);
            const float2 v = M[si * nc + q];
            float2 w = make_float2(ldexpf(v.x, -n * bs), ldexpf(v.y, -n * bs));
            for (int k = 0; k < m; ++k) w = cmul(w, eph);
            const float sg = (m & 1) ? -1.0f : 1.0f;
            Mf[n * n + n + m] = w;
            if (m) Mf[n * n + n - m] = make_float2(sg * w.x, -sg * w.y);
        }
        __syncwarp();
        const float fr = G.fr;
#pragma unroll
        for (int r = 0; r < kM2lTasksMax; ++r) {
            if (r == 1 && !round2) break;
            const int n = tn[r], m0 = tm[r];
            float2 p0 = make_float2(0.0f, 0.0f), p1 = p0, p2 = p0;
            if constexpr (PT > 0) {
#pragma unroll
                for (int j = 0; j <= PT; ++j) {
                    const float2 *mr = Mf + j * j + j;
                    const int N = j + n;
                    const float *sr = S + N * N + N - m0;
                    float w1 = sr[-j - 1], w2 = sr[-j - 2];
#pragma unroll
                    for (int k = -j; k <= j; ++k) {
                        const float2 mv = mr[k];
                        const float v = sr[k];
                        rmac(p0, v, mv);
                        rmac(p1, w1, mv);
                        rmac(p2, w2, mv);
                        w2 = w1;
                        w1 = v;
                    }
                }
            } else
            for (int j = 0; j <= P; ++j) {
                const float2 *mr = Mf + j * j + j;
                const int N = j + n;
                const float *sr = S + N * N + N - m0;   // s_N^{k - m0} at sr[k]
                float w1 = sr[-j - 1], w2 = sr[-j - 2];
                int k = -j;
                for (; k + 2 <= j; k += 3) {   // three steps with the window rotated in registers
                    const float2 m0v = mr[k], m1v = mr[k + 1], m2v = mr[k + 2];
                    const float v0 = sr[k], v1 = sr[k + 1], v2 = sr[k + 2];
                    rmac(p0, v0, m0v);
                    rmac(p1, w1, m0v);
                    rmac(p2, w2, m0v);
                    rmac(p0, v1, m1v);
                    rmac(p1, v0, m1v);
                    rmac(p2, w1, m1v);
                    rmac(p0, v2, m2v);
                    rmac(p1, v1, m2v);
                    rmac(p2, v0, m2v);
                    w2 = v1;
                    w1 = v2;
                }
                for (; k <= j; ++k) {
                    const float2 mv = mr[k];
                    const float v = sr[k];
                    rmac(p0, v, mv);
                    rmac(p1, w1, mv);
                    rmac(p2, w2, mv);
                    w2 = w1;
                    w1 = v;
                }
            }
            const float2 pr[kM2lBlock] = {p0, p1, p2};
            // e^{-i m phi} for m = m0, m0 + 1, m0 + 2
            float2 em = make_float2(1.0f, 0.0f);
            const float2 ec = cconj(eph);
            for (int k = 0; k < m0; ++k) em = cmul(em, ec);
#pragma unroll
            for (int d = 0; d < kM2lBlock; ++d) {
                const int m = m0 + d;
                const float f = ldexpf(((n + m) & 1) ? -fr : fr, -n * bt);
                const float2 t = cmul(pr[d], em);
                acc[r][d] = make_float2(fmaf(f, t.x, acc[r][d].x), fmaf(f, t.y, acc[r][d].y));
                em = cmul(em, ec);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kM2lTasksMax; ++r) {
        if (!tv[r]) continue;
#pragma unroll
        for (int d = 0; d < kM2lBlock; ++d)
            if (tm[r] + d <= tn[r]) L[ti * nc + tri(tn[r], tm[r] + d)] = acc[r][d];
    }
    }
}

// L2L for the cells of one level (parent complete): L'_k^l += 2^-k sum_{n>=k,m} L_n^m R_{n-k}^{m-l}(d),
// d = (child centre - parent centre) / h_parent.  The root has no parent.
__global__ void __launch_bounds__(32 * kCellWarps) fmm_l2l_kernel(
    const FCell *__restrict__ tc, int64_t c0, int64_t ncell, const int32_t *__restrict__ parent, double half_w0,
    int P, float2 *__restrict__ L) {
    __shared__ FmmShared sh[kCellWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ci = c0 + blockIdx.x * (int64_t)kCellWarps + wid;
    if (ci >= c0 + ncell) return;
    const int64_t pi = parent[ci];
    const FCell &C = tc[ci];
    const FCell &Pp = tc[pi];
    const int nc = tri(P + 1, 0);
    const double ihd = ldexp(1.0 / half_w0, Pp.level);
    const float dx = (float)((C.c[0] - Pp.c[0]) * ihd), dy = (float)((C.c[1] - Pp.c[1]) * ihd),
                dz = (float)((C.c[2] - Pp.c[2]) * ihd);
    float2 *tab = sh[wid].tab, *ex = sh[wid].exp;
    if (lane <= P) regular_column(tab, lane, P, dx, dy, dz);
    for (int q = lane; q < nc; q += 32) ex[q] = L[pi * nc + q];
    __syncwarp();
    for (int q = lane; q < nc; q += 32) {
        int k, l;
        tri_nm(q, k, l);
        float2 s = make_float2(0.0f, 0.0f);
        for (int n = k; n <= P; ++n) {
            const int d = n - k;
            const int m0 = max(-n, l - d), m1 = min(n, l + d);
            for (int m = m0; m <= m1; ++m) cmac(s, sym_get(ex, n, m), sym_get(tab, d, m - l));
        }
        const float sc = ldexpf(1.0f, -k);
        L[ci * nc + q] = make_float2(fmaf(sc, s.x, L[ci * nc + q].x), fmaf(sc, s.y, L[ci * nc + q].y));
    }
}

__global__ void fmm_parent_kernel(const FCell *__restrict__ tc, int64_t ncell, int32_t *__restrict__ parent) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    if (i == 0) parent[0] = -1;
    const FCell &c = tc[i];
    for (int k = 0; k < c.nchild; ++k) parent[c.child + k] = (int32_t)i;
}

// Target leaves: persistent warps take cells from *queue and skip non-leaves.
// Per leaf, first L2P, a lane per target, by the
// regular recurrence at (t - z)/h with the leaf's local expansion in shared
// memory.  Then the direct sum over the leaf's source leaves: the warp takes the
// source leaves 32 at a time (their counts, a warp prefix sum and the FP32
// offsets c_S - z from FP64 centres), stages their sources in chunks of
// kP2pChunk as FP32 offsets from the target leaf's centre, and a target's terms
// are split over lpt lanes (the largest power of two with lpt x targets <= 32),
// combined by shuffles at the end.  FP32 chunk sums, FP64 per target.
constexpr int kP2pChunk = 128;

struct LeafShared {
    float2 l[kNcMax];
    float4 a[kP2pChunk], b[kP2pChunk];
    int pre[33], start[32];
    float dc[32][3];
    float far[64];
};

__global__ void __launch_bounds__(32 * kCellWarps) fmm_leaf_kernel(
    const FCell *__restrict__ tc, int64_t ntc, const FCell *__restrict__ sc, const int64_t *__restrict__ off,
    const uint64_t *__restrict__ list, const int32_t *__restrict__ tval, const double *__restrict__ targets,
    const float4 *__restrict__ srel, const float4 *__restrict__ sdat, double half_w0, int P,
    const float2 *__restrict__ L, double *__restrict__ out, unsigned long long *__restrict__ queue) {
    __shared__ LeafShared sh[kCellWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    LeafShared &S = sh[wid];
    const int nc = tri(P + 1, 0);
    for (;;) {
    unsigned long long qi = 0;
    if (lane == 0) qi = atomicAdd(queue, 1ull);
    const int64_t ti = (int64_t)__shfl_sync(0xffffffffu, qi, 0);
    if (ti >= ntc) break;
    const FCell T = tc[ti];
    if (T.child >= 0) continue;
    __syncwarp();
    for (int q = lane; q < nc; q += 32) S.l[q] = L[ti * nc + q];
    __syncwarp();
    const double ihd = ldexp(1.0 / half_w0, T.level);
    const int64_t e0 = off[ti], e1 = off[ti + 1];
    for (int tb = T.start; tb < T.start + T.count; tb += 64) {
        const int nt = min(64, T.start + T.count - tb);
        __syncwarp();
        // L2P, a lane per target (two rounds of lanes for more than 32 targets)
        for (int tt = lane; tt < nt; tt += 32) {
            const int32_t id = tval[tb + tt];
            const float x = (float)((targets[3 * id] - T.c[0]) * ihd), y = (float)((targets[3 * id + 1] - T.c[1]) * ihd),
                        z = (float)((targets[3 * id + 2] - T.c[2]) * ihd);
            const float r2 = fmaf(x, x, fmaf(y, y, z * z));
            float far = 0.0f;
            float2 rmm = make_float2(1.0f, 0.0f);
            for (int m = 0; m <= P; ++m) {
                if (m > 0) rmm = cscale(cmul(rmm, make_float2(x, y)), 0.5f / (float)m);
                float2 a = make_float2(0.0f, 0.0f), b = rmm;
                float part = b.x * S.l[tri(m, m)].x - b.y * S.l[tri(m, m)].y;
                for (int n = m + 1; n <= P; ++n) {
                    const float inv = 1.0f / (float)((n + m) * (n - m));
                    const float2 c = make_float2(((2 * n - 1) * z * b.x - r2 * a.x) * inv,
                                                 ((2 * n - 1) * z * b.y - r2 * a.y) * inv);
                    const float2 lv = S.l[tri(n, m)];
                    part = fmaf(c.x, lv.x, fmaf(-c.y, lv.y, part));
                    a = b;
                    b = c;
                }
                far = fmaf(m ? 2.0f : 1.0f, part, far);
            }
            S.far[tt] = far;
        }
        // near field: more than 32 targets, two per lane (targets lane and
        // lane + 32, one staged source serving both); else lanes (target tt,
        // slice) with lpt lanes per target
        const bool two = nt > 32;
        int lpt = 1;
        if (!two)
            while (lpt * 2 * nt <= 32) lpt *= 2;
        const int tt = two ? lane : lane / lpt, slice = two ? 0 : lane % lpt;
        const bool tvalid = tt < nt, tvalid1 = two && lane + 32 < nt;
        const int32_t id = tval[tb + (tvalid ? tt : 0)];
        const int32_t id1 = tval[tb + (tvalid1 ? lane + 32 : 0)];
        const float ox = (float)(targets[3 * id] - T.c[0]), oy = (float)(targets[3 * id + 1] - T.c[1]),
                    oz = (float)(targets[3 * id + 2] - T.c[2]);
        const float qx = (float)(targets[3 * id1] - T.c[0]), qy = (float)(targets[3 * id1 + 1] - T.c[1]),
                    qz = (float)(targets[3 * id1 + 2] - T.c[2]);
        double acc = 0.0, acc1 = 0.0;
        for (int64_t g0 = e0; g0 < e1; g0 += 32) {
            const int ng = (int)min((int64_t)32, e1 - g0);
            int cntv = 0;
            __syncwarp();
            if (lane < ng) {
                const FCell &C = sc[(uint32_t)(list[g0 + lane] & 0xffffffffu)];
                cntv = C.count;
                S.start[lane] = C.start;
                S.dc[lane][0] = (float)(C.c[0] - T.c[0]);
                S.dc[lane][1] = (float)(C.c[1] - T.c[1]);
                S.dc[lane][2] = (float)(C.c[2] - T.c[2]);
            }
            int incl = cntv;
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            S.pre[lane + 1] = incl;
            if (lane == 0) S.pre[0] = 0;
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            for (int cb = 0; cb < total; cb += kP2pChunk) {
                const int cn = min(kP2pChunk, total - cb);
                __syncwarp();
                for (int i = lane; i < cn; i += 32) {
                    const int gidx = cb + i;
                    int lo = 0, hi = ng;   // pair p with pre[p] <= gidx < pre[p+1]
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (S.pre[mid] <= gidx) lo = mid;
                        else hi = mid;
                    }
                    const int src = S.start[lo] + gidx - S.pre[lo];
                    const float4 a = srel[src];
                    S.a[i] = make_float4(a.x + S.dc[lo][0], a.y + S.dc[lo][1], a.z + S.dc[lo][2], a.w);
                    S.b[i] = sdat[src];
                }
                __syncwarp();
                float part0 = 0.0f, part1 = 0.0f;
                if (two) {
                    for (int k = 0; k < cn; ++k) {
                        const float4 pa = S.a[k], pb = S.b[k];
                        const float dx = ox - pa.x, dy = oy - pa.y, dz = oz - pa.z;
                        const float ex2 = qx - pa.x, ey2 = qy - pa.y, ez2 = qz - pa.z;
                        const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                        const float rj = rsqrtf(fmaf(ex2, ex2, fmaf(ey2, ey2, ez2 * ez2)));
                        const float dn = fmaf(dx, pb.x, fmaf(dy, pb.y, dz * pb.z));
                        const float en = fmaf(ex2, pb.x, fmaf(ey2, pb.y, ez2 * pb.z));
                        part0 += ri * fmaf(dn, ri * ri, pa.w);
                        part1 += rj * fmaf(en, rj * rj, pa.w);
                    }
                    acc += (double)part0;
                    acc1 += (double)part1;
                } else {
                    int k = slice;
                    for (; k + lpt < cn; k += 2 * lpt) {
                        const float4 pa = S.a[k], pb = S.b[k], qa = S.a[k + lpt], qb = S.b[k + lpt];
                        const float dx = ox - pa.x, dy = oy - pa.y, dz = oz - pa.z;
                        const float ex2 = ox - qa.x, ey2 = oy - qa.y, ez2 = oz - qa.z;
                        const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                        const float rj = rsqrtf(fmaf(ex2, ex2, fmaf(ey2, ey2, ez2 * ez2)));
                        const float dn = fmaf(dx, pb.x, fmaf(dy, pb.y, dz * pb.z));
                        const float en = fmaf(ex2, qb.x, fmaf(ey2, qb.y, ez2 * qb.z));
                        part0 += ri * fmaf(dn, ri * ri, pa.w);
                        part1 += rj * fmaf(en, rj * rj, qa.w);
                    }
                    if (k < cn) {
                        const float4 pa = S.a[k], pb = S.b[k];
                        const float dx = ox - pa.x, dy = oy - pa.y, dz = oz - pa.z;
                        const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                        const float dn = fmaf(dx, pb.x, fmaf(dy, pb.y, dz * pb.z));
                        part0 += ri * fmaf(dn, ri * ri, pa.w);
                    }
                    acc += (double)part0 + (double)part1;
                }
            }
        }
        for (int o = 1; o < lpt; o <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __syncwarp();
        if (tvalid && slice == 0) out[id] = acc + (double)S.far[tt];
        if (tvalid1) out[id1] = acc1 + (double)S.far[lane + 32];
    }
    }
}

__global__ void fmm_zero_kernel(int64_t n, double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = 0.0;
}

inline int64_t nblk(int64_t n, int t) { return (n + t - 1) / t; }

}  // namespace

// ------------------------------------------------------------------ host side

struct FmmWorkspace {
    DevBuf part, kin, kout, vin, sval, tval, flag, pos, lo, hi, cub, scell, tcell, tparent;
    DevBuf spos, sdat, srel, M, L, front, next, m2l, m2l_s, p2p, p2p_s, m2l_off, p2p_off, cnt, gtmp, queue, m2lgeo;
    DttCounters *host_cnt = nullptr;   // pinned
    int64_t cap_front = 0, cap_m2l = 0, cap_p2p = 0;
    int64_t grid_m2l = 0, grid_leaf = 0;   // persistent grids (resident CTAs x SMs)
};

void fmm_release(dtn_geometry *g) {
    FmmWorkspace *w = static_cast<FmmWorkspace *>(g->fmm_ws);
    if (!w) return;
    DevBuf *bufs[] = {&w->part, &w->kin, &w->kout, &w->vin, &w->sval, &w->tval, &w->flag, &w->pos, &w->lo,
                      &w->hi, &w->cub, &w->scell, &w->tcell, &w->tparent, &w->spos, &w->sdat, &w->srel, &w->M, &w->L,
                      &w->front, &w->next, &w->m2l, &w->m2l_s, &w->p2p, &w->p2p_s, &w->m2l_off, &w->p2p_off,
                      &w->cnt, &w->gtmp, &w->queue, &w->m2lgeo};
    for (DevBuf *b : bufs) b->release();
    if (w->host_cnt) cudaFreeHost(w->host_cnt);
    delete w;
    g->fmm_ws = nullptr;
}

namespace {

#define FMM_TRY(x)                                   \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

// grow a buffer keeping its first `keep` bytes (stream-ordered copy)
cudaError_t grow_keep(DevBuf &b, size_t need, size_t keep, cudaStream_t s) {
    if (need <= b.bytes && b.p) return cudaSuccess;
    void *np = nullptr;
    const size_t want = std::max(need, b.bytes * 3 / 2);
    FMM_TRY(cudaMalloc(&np, want));
    if (b.p && keep) FMM_TRY(cudaMemcpyAsync(np, b.p, keep, cudaMemcpyDeviceToDevice, s));
    FMM_TRY(cudaStreamSynchronize(s));
    b.release();
    b.p = np;
    b.bytes = want;
    return cudaSuccess;
}

struct TreeInfo {
    std::vector<int64_t> level_off;   // cells of level l: [level_off[l], level_off[l+1])
    int64_t ncell = 0, nleaf = 0;
};

// Sorts the points by Morton key and builds the cells level by level.
cudaError_t build_tree(FmmWorkspace &w, DevBuf &cells, DevBuf &val_out, int64_t n, const double *x,
                       const int64_t *index, const double lo[3], double width, int ncrit, int max_level,
                       TreeInfo &ti, cudaStream_t s) {
    const double scale = std::ldexp(1.0, kMortonBits) / width;
    FMM_TRY(w.kin.reserve(n * 8));
    FMM_TRY(w.kout.reserve(n * 8));
    FMM_TRY(w.vin.reserve(n * 4));
    FMM_TRY(val_out.reserve(n * 4));
    fmm_morton_kernel<<<nblk(n, 256), 256, 0, s>>>(n, x, index, lo[0], lo[1], lo[2], scale, w.kin.as<uint64_t>(),
                                                    w.vin.as<int32_t>());
    FMM_TRY(cudaGetLastError());
    size_t tb = 0;
    FMM_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tb, w.kin.as<uint64_t>(), w.kout.as<uint64_t>(),
                                            w.vin.as<int32_t>(), val_out.as<int32_t>(), (int)n, 0, 3 * kMortonBits, s));
    FMM_TRY(w.cub.reserve(tb));
    FMM_TRY(cub::DeviceRadixSort::SortPairs(w.cub.p, tb, w.kin.as<uint64_t>(), w.kout.as<uint64_t>(),
                                            w.vin.as<int32_t>(), val_out.as<int32_t>(), (int)n, 0, 3 * kMortonBits, s));
    const uint64_t *keys = w.kout.as<uint64_t>();
    // root
    FCell root{};
    root.c[0] = lo[0] + 0.5 * width;
    root.c[1] = lo[1] + 0.5 * width;
    root.c[2] = lo[2] + 0.5 * width;
    root.key = 0;
    root.start = 0;
    root.count = (int32_t)n;
    root.child = -1;
    root.nchild = 0;
    root.level = 0;
    FMM_TRY(grow_keep(cells, sizeof(FCell) * 1024, 0, s));
    FMM_TRY(cudaMemcpyAsync(cells.p, &root, sizeof(FCell), cudaMemcpyHostToDevice, s));
    ti.level_off.assign({0, 1});
    for (int l = 0; l < max_level; ++l) {
        const int64_t c0 = ti.level_off[l], nc = ti.level_off[l + 1] - c0;
        if (nc == 0) break;
        FMM_TRY(w.flag.reserve(8 * nc * 4));
        FMM_TRY(w.pos.reserve(8 * nc * 4));
        FMM_TRY(w.lo.reserve(8 * nc * 4));
        FMM_TRY(w.hi.reserve(8 * nc * 4));
        fmm_split_kernel<<<nblk(8 * nc, 256), 256, 0, s>>>(cells.as<FCell>(), c0, nc, keys, ncrit, max_level,
                                                            w.flag.as<int32_t>(), w.lo.as<int32_t>(),
                                                            w.hi.as<int32_t>());
        FMM_TRY(cudaGetLastError());
        size_t sb = 0;
        FMM_TRY(cub::DeviceScan::ExclusiveSum(nullptr, sb, w.flag.as<int32_t>(), w.pos.as<int32_t>(), (int)(8 * nc), s));
        FMM_TRY(w.cub.reserve(std::max(sb, w.cub.bytes)));
        FMM_TRY(cub::DeviceScan::ExclusiveSum(w.cub.p, sb, w.flag.as<int32_t>(), w.pos.as<int32_t>(), (int)(8 * nc), s));
        int32_t tail[2];
        FMM_TRY(cudaMemcpyAsync(&tail[0], w.pos.as<int32_t>() + 8 * nc - 1, 4, cudaMemcpyDeviceToHost, s));
        FMM_TRY(cudaMemcpyAsync(&tail[1], w.flag.as<int32_t>() + 8 * nc - 1, 4, cudaMemcpyDeviceToHost, s));
        FMM_TRY(cudaStreamSynchronize(s));
        const int64_t total = (int64_t)tail[0] + tail[1];
        const int64_t c_next = c0 + nc;
        FMM_TRY(grow_keep(cells, sizeof(FCell) * (c_next + std::max<int64_t>(total, 1)), sizeof(FCell) * c_next, s));
        const double h_child = std::ldexp(width, -(l + 2));
        fmm_emit_kernel<<<nblk(8 * nc, 256), 256, 0, s>>>(cells.as<FCell>(), c0, nc, c_next, w.flag.as<int32_t>(),
                                                           w.pos.as<int32_t>(), w.lo.as<int32_t>(),
                                                           w.hi.as<int32_t>(), h_child);
        FMM_TRY(cudaGetLastError());
        if (total == 0) break;
        ti.level_off.push_back(c_next + total);
    }
    ti.ncell = ti.level_off.back();
    return cudaSuccess;
}

}  // namespace

cudaError_t fmm_evaluate(dtn_geometry *g, int64_t np, int64_t np_total, const double *xyz, const double *nrm,
                         const double *area, const double *q, const double *gv, const int64_t *index, int64_t nt,
                         const double *t, double *out, const dtn_fmm_opts &o, dtn_fmm_stats *st, bool *bad_index,
                         cudaStream_t s) {
    *bad_index = false;
    if (!g->fmm_ws) g->fmm_ws = new FmmWorkspace();
    FmmWorkspace &w = *static_cast<FmmWorkspace *>(g->fmm_ws);
    if (!w.host_cnt) FMM_TRY(cudaMallocHost((void **)&w.host_cnt, sizeof(DttCounters)));
    dtn_fmm_stats stats{};
    if (np == 0) {
        fmm_zero_kernel<<<nblk(nt, 256), 256, 0, s>>>(nt, out);
        FMM_TRY(cudaGetLastError());
        if (st) *st = stats;
        return cudaSuccess;
    }
    // bounding cube of sources and targets
    const size_t part_bytes = 2 * kBboxBlocks * 6 * sizeof(double);
    FMM_TRY(w.part.reserve(part_bytes + 16));
    int *d_bad = reinterpret_cast<int *>(w.part.as<char>() + part_bytes);
    FMM_TRY(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    fmm_bbox_kernel<<<kBboxBlocks, 256, 0, s>>>(np, xyz, index, np_total, w.part.as<double>(), d_bad);
    fmm_bbox_kernel<<<kBboxBlocks, 256, 0, s>>>(nt, t, nullptr, nt, w.part.as<double>() + kBboxBlocks * 6, d_bad);
    FMM_TRY(cudaGetLastError());
    std::vector<double> part(2 * kBboxBlocks * 6 + 2);
    FMM_TRY(cudaMemcpyAsync(part.data(), w.part.p, part_bytes + 16, cudaMemcpyDeviceToHost, s));
    FMM_TRY(cudaStreamSynchronize(s));
    if (*reinterpret_cast<const int *>(part.data() + 2 * kBboxBlocks * 6)) {
        *bad_index = true;
        return cudaSuccess;
    }
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < 2 * kBboxBlocks; ++b)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], part[6 * b + a]);
            hi[a] = std::max(hi[a], part[6 * b + 3 + a]);
        }
    double width = 0.0;
    for (int a = 0; a < 3; ++a) width = std::max(width, hi[a] - lo[a]);
    if (!std::isfinite(width)) return cudaErrorInvalidValue;
    width = width * (1.0 + 1e-9) + 1e-300;
    for (int a = 0; a < 3; ++a) lo[a] -= 0.5 * (width - (hi[a] - lo[a]));   // centre the cube on the box
    const double half_w0 = 0.5 * width;

    // trees
    TreeInfo st_s, st_t;
    FMM_TRY(build_tree(w, w.scell, w.sval, np, xyz, index, lo, width, o.leaf_sources, o.max_level, st_s, s));
    FMM_TRY(w.spos.reserve(np * 24));
    FMM_TRY(w.sdat.reserve(np * 16));
    fmm_source_kernel<<<nblk(np, 256), 256, 0, s>>>(np, w.sval.as<int32_t>(), xyz, nrm, area, q, gv,
                                                     w.spos.as<double>(), w.sdat.as<float4>());
    FMM_TRY(cudaGetLastError());
    FMM_TRY(build_tree(w, w.tcell, w.tval, nt, t, nullptr, lo, width, o.leaf_targets, o.max_level, st_t, s));
    for (int l = (int)st_s.level_off.size() - 2; l >= 0; --l) {
        const int64_t c0 = st_s.level_off[l], n = st_s.level_off[l + 1] - c0;
        fmm_radius_kernel<<<nblk(32 * n, 128), 128, 0, s>>>(w.scell.as<FCell>(), c0, n, w.spos.as<double>(), nullptr);
    }
    for (int l = (int)st_t.level_off.size() - 2; l >= 0; --l) {
        const int64_t c0 = st_t.level_off[l], n = st_t.level_off[l + 1] - c0;
        fmm_radius_kernel<<<nblk(32 * n, 128), 128, 0, s>>>(w.tcell.as<FCell>(), c0, n, t, w.tval.as<int32_t>());
    }
    FMM_TRY(cudaGetLastError());
    const int64_t nsc = st_s.ncell, ntc = st_t.ncell;
    const int P = o.order, nc = tri(P + 1, 0);

    // upward pass
    FMM_TRY(w.M.reserve(nsc * nc * sizeof(float2)));
    FMM_TRY(w.srel.reserve(np * 16));
    fmm_p2m_kernel<<<nblk(nsc, kCellWarps), 32 * kCellWarps, 0, s>>>(w.scell.as<FCell>(), nsc, w.spos.as<double>(),
                                                                     w.sdat.as<float4>(), half_w0, P,
                                                                     w.M.as<float2>(), w.srel.as<float4>());
    FMM_TRY(cudaGetLastError());
    for (int l = (int)st_s.level_off.size() - 2; l >= 0; --l) {
        const int64_t c0 = st_s.level_off[l], n = st_s.level_off[l + 1] - c0;
        fmm_m2m_kernel<<<nblk(n, kCellWarps), 32 * kCellWarps, 0, s>>>(w.scell.as<FCell>(), c0, n, half_w0, P,
                                                                       w.M.as<float2>());
        FMM_TRY(cudaGetLastError());
    }

    // dual-tree traversal
    // list capacities from the tree sizes (grown and the traversal restarted on overflow)
    w.cap_front = std::max(w.cap_front, 32 * (nsc + ntc) + 4096);
    w.cap_m2l = std::max(w.cap_m2l, 256 * ntc + 4096);
    w.cap_p2p = std::max(w.cap_p2p, 64 * ntc + 4096);
    int64_t n_m2l = 0, n_p2p = 0;
    int passes = 0, restarts = 0;
    for (;;) {
        FMM_TRY(w.front.reserve(w.cap_front * sizeof(int2)));
        FMM_TRY(w.next.reserve(w.cap_front * sizeof(int2)));
        FMM_TRY(w.m2l.reserve(w.cap_m2l * 8));
        FMM_TRY(w.p2p.reserve(w.cap_p2p * 8));
        FMM_TRY(w.cnt.reserve(sizeof(DttCounters)));
        FMM_TRY(cudaMemsetAsync(w.cnt.p, 0, sizeof(DttCounters), s));
        const int2 root = make_int2(0, 0);
        FMM_TRY(cudaMemcpyAsync(w.front.p, &root, sizeof(int2), cudaMemcpyHostToDevice, s));
        int64_t nf = 1;
        bool overflow = false;
        passes = 0;
        while (nf > 0) {
            FMM_TRY(cudaMemsetAsync(w.cnt.p, 0, sizeof(unsigned long long), s));   // next = 0
            fmm_dtt_kernel<<<nblk(nf, 256), 256, 0, s>>>(
                w.front.as<int2>(), nf, w.tcell.as<FCell>(), w.scell.as<FCell>(), o.theta * o.theta,
                w.next.as<int2>(), w.cap_front, w.m2l.as<uint64_t>(), w.cap_m2l, w.p2p.as<uint64_t>(), w.cap_p2p,
                w.cnt.as<DttCounters>());
            FMM_TRY(cudaGetLastError());
            FMM_TRY(cudaMemcpyAsync(w.host_cnt, w.cnt.p, sizeof(DttCounters), cudaMemcpyDeviceToHost, s));
            FMM_TRY(cudaStreamSynchronize(s));
            ++passes;
            const DttCounters c = *w.host_cnt;
            if (c.overflow) {
                overflow = true;
                if ((int64_t)c.next > w.cap_front) w.cap_front = 2 * (int64_t)c.next;
                if ((int64_t)c.m2l >= w.cap_m2l) w.cap_m2l = 2 * (int64_t)c.m2l;
                if ((int64_t)c.p2p >= w.cap_p2p) w.cap_p2p = 2 * (int64_t)c.p2p;
                break;
            }
            std::swap(w.front, w.next);
            nf = (int64_t)c.next;
            n_m2l = (int64_t)c.m2l;
            n_p2p = (int64_t)c.p2p;
            stats.p2p_terms = (int64_t)c.p2p_terms;
        }
        if (!overflow) break;
        ++restarts;
    }
    // sort both lists by target and build their offsets
    FMM_TRY(w.m2l_s.reserve(std::max<int64_t>(n_m2l, 1) * 8));
    FMM_TRY(w.p2p_s.reserve(std::max<int64_t>(n_p2p, 1) * 8));
    {
        size_t tb1 = 0, tb2 = 0;
        FMM_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb1, w.m2l.as<uint64_t>(), w.m2l_s.as<uint64_t>(), (int)n_m2l, 0, 64, s));
        FMM_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb2, w.p2p.as<uint64_t>(), w.p2p_s.as<uint64_t>(), (int)n_p2p, 0, 64, s));
        FMM_TRY(w.cub.reserve(std::max(std::max(tb1, tb2), w.cub.bytes)));
        size_t tb = w.cub.bytes;
        FMM_TRY(cub::DeviceRadixSort::SortKeys(w.cub.p, tb, w.m2l.as<uint64_t>(), w.m2l_s.as<uint64_t>(), (int)n_m2l, 0, 64, s));
        tb = w.cub.bytes;
        FMM_TRY(cub::DeviceRadixSort::SortKeys(w.cub.p, tb, w.p2p.as<uint64_t>(), w.p2p_s.as<uint64_t>(), (int)n_p2p, 0, 64, s));
    }
    FMM_TRY(w.m2l_off.reserve((ntc + 1) * 8));
    FMM_TRY(w.p2p_off.reserve((ntc + 1) * 8));
    fmm_csr_kernel<<<nblk(ntc + 1, 256), 256, 0, s>>>(ntc, w.m2l_s.as<uint64_t>(), n_m2l, w.m2l_off.as<int64_t>());
    FMM_TRY(w.m2lgeo.reserve(std::max<int64_t>(n_m2l, 1) * sizeof(M2lGeo)));
    if (n_m2l > 0)
        fmm_m2lgeo_kernel<<<nblk(n_m2l, 256), 256, 0, s>>>(n_m2l, w.m2l_s.as<uint64_t>(), w.tcell.as<FCell>(),
                                                           w.scell.as<FCell>(), half_w0, w.m2lgeo.as<M2lGeo>());
    fmm_csr_kernel<<<nblk(ntc + 1, 256), 256, 0, s>>>(ntc, w.p2p_s.as<uint64_t>(), n_p2p, w.p2p_off.as<int64_t>());
    FMM_TRY(cudaGetLastError());

    // downward pass
    FMM_TRY(w.L.reserve(ntc * nc * sizeof(float2)));
    FMM_TRY(w.queue.reserve(2 * sizeof(unsigned long long)));
    unsigned long long *queue = w.queue.as<unsigned long long>();
    FMM_TRY(cudaMemsetAsync(queue, 0, 2 * sizeof(unsigned long long), s));
    FMM_TRY(cudaMemsetAsync(w.L.p, 0, ntc * nc * sizeof(float2), s));
    if (w.grid_m2l == 0) {
        int per_sm = 0;
        FMM_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fmm_m2l_kernel<0>, 32 * kCellWarps, 0));
        w.grid_m2l = std::max(1, per_sm) * g->num_sms;
        FMM_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fmm_leaf_kernel, 32 * kCellWarps, 0));
        w.grid_leaf = std::max(1, per_sm) * g->num_sms;
    }
    {
        const int grid = (int)std::min<int64_t>(w.grid_m2l, nblk(ntc, kCellWarps));
        auto kern = P == 8 ? fmm_m2l_kernel<8> : P == 10 ? fmm_m2l_kernel<10> : fmm_m2l_kernel<0>;
        kern<<<grid, 32 * kCellWarps, 0, s>>>(w.tcell.as<FCell>(), ntc, w.scell.as<FCell>(), w.m2l_off.as<int64_t>(),
                                              w.m2l_s.as<uint64_t>(), w.m2lgeo.as<M2lGeo>(), P, w.M.as<float2>(),
                                              w.L.as<float2>(), queue);
    }
    FMM_TRY(cudaGetLastError());
    FMM_TRY(w.tparent.reserve(ntc * 4));
    fmm_parent_kernel<<<nblk(ntc, 256), 256, 0, s>>>(w.tcell.as<FCell>(), ntc, w.tparent.as<int32_t>());
    FMM_TRY(cudaGetLastError());
    for (size_t l = 1; l + 1 < st_t.level_off.size(); ++l) {
        const int64_t c0 = st_t.level_off[l], n = st_t.level_off[l + 1] - c0;
        fmm_l2l_kernel<<<nblk(n, kCellWarps), 32 * kCellWarps, 0, s>>>(w.tcell.as<FCell>(), c0, n,
                                                                       w.tparent.as<int32_t>(), half_w0, P,
                                                                       w.L.as<float2>());
        FMM_TRY(cudaGetLastError());
    }
    fmm_leaf_kernel<<<(int)std::min<int64_t>(w.grid_leaf, nblk(ntc, kCellWarps)), 32 * kCellWarps, 0, s>>>(
        w.tcell.as<FCell>(), ntc, w.scell.as<FCell>(), w.p2p_off.as<int64_t>(), w.p2p_s.as<uint64_t>(),
        w.tval.as<int32_t>(), t, w.srel.as<float4>(), w.sdat.as<float4>(), half_w0, P, w.L.as<float2>(), out,
        queue + 1);
    FMM_TRY(cudaGetLastError());

    if (st) {
        stats.source_cells = nsc;
        stats.target_cells = ntc;
        stats.source_levels = (int32_t)st_s.level_off.size() - 1;
        stats.target_levels = (int32_t)st_t.level_off.size() - 1;
        stats.m2l_pairs = n_m2l;
        stats.p2p_pairs = n_p2p;
        stats.traversal_passes = passes;
        stats.restarts = restarts;
        *st = stats;
    }
    return cudaSuccess;
}

}  // namespace dtn

extern "C" dtn_status dtn_eval_potential_fmm(dtn_geometry *g, int64_t np, const double *xyz, const double *nrm,
                                             const double *area, const double *q, const double *gv,
                                             const int64_t *index, const int64_t *n_index, int64_t nt,
                                             const double *t, double *out, const dtn_fmm_opts *o,
                                             dtn_fmm_stats *st, void *stream) {
    using namespace dtn;
    if (!g || !o || np < 0 || nt < 0) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (o->order < 1 || o->order > kFmmMaxOrder || !(o->theta > 0.0 && o->theta < 1.0) || o->leaf_sources < 1 ||
        o->leaf_sources > 4096 || o->leaf_targets < 1 || o->leaf_targets > 4096 || o->max_level < 1 ||
        o->max_level > kMortonBits)
        return DTN_E_INVALID_ARG;
    if (np >= (int64_t)1 << 31 || nt >= (int64_t)1 << 31) return DTN_E_INVALID_ARG;
    if (st) *st = dtn_fmm_stats{};
    if (nt == 0) return DTN_OK;
    if (!t || !out || (np > 0 && (!xyz || !nrm || !area || !q))) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    int64_t n = np;
    if (index && n_index) {
        if ((e = cudaMemcpyAsync(&n, n_index, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return to_status(e);
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return to_status(e);
        if (n < 0 || n > np) return DTN_E_INVALID_ARG;
    }
    if (!gv && n > 0) {
        if (!g->has_data) return DTN_E_INVALID_ARG;
        if (!g->fmm_ws) g->fmm_ws = new FmmWorkspace();
        FmmWorkspace &w = *static_cast<FmmWorkspace *>(g->fmm_ws);
        if ((e = w.gtmp.reserve(np * sizeof(double))) != cudaSuccess) return to_status(e);
        if ((e = launch_dirichlet(g, np, xyz, w.gtmp.as<double>(), s)) != cudaSuccess) return to_status(e);
        gv = w.gtmp.as<double>();
    }
    bool bad = false;
    e = fmm_evaluate(g, n, np, xyz, nrm, area, q, gv, index, nt, t, out, *o, st, &bad, s);
    if (e == cudaSuccess && bad) return DTN_E_INVALID_ARG;
    return to_status(e);
}
