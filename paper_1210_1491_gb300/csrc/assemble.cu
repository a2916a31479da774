// assemble.cu -- collocation matrix and right side of the first-kind local BIE
// (Eq. bw49-bw51) on piecewise-constant panels, one CTA per collocation row:
//
//   A_ij = int_{panel j} G(x_i, y) ds_y                       (single layer, Eq. bw50)
//   b_i  = int_S dG/dn_y(x_i, y) (g(y) - g(x_i)) ds_y
//          - sum_k W_k P(x_i, y_k) (U_k - g(x_i))
//
// with G the whole-sphere Dirichlet Green's function of the patch ball and P its
// Poisson kernel.  b is Eq. bw51 with the constant solution subtracted (the
// identity 1/2 + p.v. int_S dG/dn_y + int_Gamma dG/dn_y = 0 times g(x_i)), the
// regularisation Sec. 3 applies to its single-point formula (Eq. bw61-bw68).
// On a plane through the ball centre dG/dn_y vanishes, so disk patches have
// no S term.
//
// Quadrature (per entry, in the panel's (u, v) parameters):
//   self panel   : four triangles from the collocation point, each through the
//                  Duffy map (the local polar transform of Sec. 5.2), FP64;
//   other panels : tensor Gauss-Legendre whose order follows the ratio r of the
//                  distance from the singular points (x_i and its Kelvin image)
//                  to the panel centre over the panel radius; below r = 2 the
//                  parameter box is split into four, recursively.  Mixed
//                  precision evaluates panels with r >= 2 in FP32 and keeps the
//                  split (near-singular) cases and the rim image term in FP64.
#include <cmath>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kAsmThreads = 128;
constexpr int kMaxDepth = 10;
constexpr int kStack = 40;
constexpr int kMaxRule = 20;   // highest Gauss order the rules below use
// fixed double-layer rules of the right side (mixed precision): per panel an
// 8x8 Gauss rule (64 points) and the same rule on its four quarters (256)
constexpr int kPreCoarse = 64, kPrePerPanel = 320, kPreN = 8;

template <typename T>
struct Ctx {
    int kind;
    T a, R;
    T X[3], xn;
    T Xs[3];
    bool img;
    bool needD;
    bool data32;   // evaluate g in FP32 for the (bounded) double-layer integrand
    bool needA;    // accumulate the single-layer entry
    T gx;
    T c[3], t1[3], t2[3], n[3];
    const DData *dat;
};

template <typename T>
__device__ __forceinline__ void eval_point(const Ctx<T> &c, T u, T v, T w, T &sa, T &sd) {
    T Y[3], nl[3], J;
    patch_point<T>(c.kind, c.R, u, v, Y, nl, J);
    const T wj = w * J;
    if (c.needA) sa += wj * green_ball<T>(c.a, c.X, c.xn, Y);
    if (c.needD) {
        const T yx = c.c[0] + Y[0] * c.t1[0] + Y[1] * c.t2[0] + Y[2] * c.n[0];
        const T yy = c.c[1] + Y[0] * c.t1[1] + Y[1] * c.t2[1] + Y[2] * c.n[1];
        const T yz = c.c[2] + Y[0] * c.t1[2] + Y[1] * c.t2[2] + Y[2] * c.n[2];
        const T gy = c.data32 ? (T)dirichlet_eval<float>(*c.dat, (float)yx, (float)yy, (float)yz)
                              : dirichlet_eval<T>(*c.dat, yx, yy, yz);
        sd += wj * green_ball_dny<T>(c.a, c.X, c.xn, Y, nl) * (gy - c.gx);
    }
}

// parameter region: rectangle (u0, du, v0, dv) or Duffy triangle
// (S_u, S_v, E1_u, E1_v, E2_u, E2_v) mapped from (xi, eta) in [0,1]^2
struct Region {
    bool tri;
    double p[6];
    double det;
};

template <typename T>
__device__ __forceinline__ void map_uv(const Region &R, T xi, T eta, T &u, T &v, T &jac) {
    if (!R.tri) {
        u = (T)R.p[0] + xi * (T)R.p[1];
        v = (T)R.p[2] + eta * (T)R.p[3];
        jac = (T)(R.p[1] * R.p[3]);
    } else {
        u = (T)R.p[0] + xi * ((T)R.p[2] + eta * (T)R.p[4]);
        v = (T)R.p[1] + xi * ((T)R.p[3] + eta * (T)R.p[5]);
        jac = xi * (T)R.det;
    }
}

template <typename T>
__device__ void gauss_square(const Ctx<T> &c, const Region &R, T x0, T x1, T e0, T e1, int n,
                             const double *__restrict__ glx, const double *__restrict__ glw, T &sa, T &sd) {
    const double *gx = glx + n * (n - 1) / 2, *gw = glw + n * (n - 1) / 2;
    const T hx = (T)0.5 * (x1 - x0), mx = (T)0.5 * (x0 + x1);
    const T he = (T)0.5 * (e1 - e0), me = (T)0.5 * (e0 + e1);
    for (int i = 0; i < n; ++i) {
        const T xi = mx + hx * (T)gx[i];
        const T wi = (T)gw[i] * hx * he;
        for (int j = 0; j < n; ++j) {
            const T eta = me + he * (T)gx[j];
            T u, v, jac;
            map_uv<T>(R, xi, eta, u, v, jac);
            eval_point<T>(c, u, v, wi * (T)gw[j] * jac, sa, sd);
        }
    }
}

// The same rule on a rectangle of the parameter box.  The map is separable, so
// the sines and cosines of u and of v are taken once per Gauss line.
template <typename T>
__device__ void gauss_rect(const Ctx<T> &c, const Region &R, T x0, T x1, T e0, T e1, int n,
                           const double *__restrict__ glx, const double *__restrict__ glw, T &sa, T &sd,
                           const float *__restrict__ gpre = nullptr) {
    const double *gx = glx + n * (n - 1) / 2, *gw = glw + n * (n - 1) / 2;
    const T hx = (T)0.5 * (x1 - x0), mx = (T)0.5 * (x0 + x1);
    const T he = (T)0.5 * (e1 - e0), me = (T)0.5 * (e0 + e1);
    const T du = (T)R.p[1], dv = (T)R.p[3];
    const T jac = du * dv;
    T cvs[kMaxRule], svs[kMaxRule];
    for (int j = 0; j < n; ++j) {
        const T v = (T)R.p[2] + (me + he * (T)gx[j]) * dv;
        sincos(v, &svs[j], &cvs[j]);
    }
    for (int i = 0; i < n; ++i) {
        const T u = (T)R.p[0] + (mx + hx * (T)gx[i]) * du;
        const T wi = (T)gw[i] * hx * he * jac;
        T ru, rz, nu, nz, J;
        if (c.kind == kDisk) {
            ru = u; rz = (T)0; nu = (T)0; nz = (T)1; J = u;
        } else {
            T su, cu;
            sincos(u, &su, &cu);
            const T sh = sin((T)0.5 * u);
            ru = c.R * su; rz = (T)-2 * c.R * sh * sh; nu = su; nz = cu; J = c.R * c.R * su;
        }
        for (int j = 0; j < n; ++j) {
            const T Y[3] = {ru * cvs[j], ru * svs[j], rz};
            const T wj = wi * (T)gw[j] * J;
            if (c.needA) sa += wj * green_ball<T>(c.a, c.X, c.xn, Y);
            if (c.needD) {
                const T nl[3] = {nu * cvs[j], nu * svs[j], nz};
                T gy;
                if (gpre) {
                    gy = (T)gpre[i * n + j];   // data precomputed at this rule's points
                } else {
                    const T yx = c.c[0] + Y[0] * c.t1[0] + Y[1] * c.t2[0] + Y[2] * c.n[0];
                    const T yy = c.c[1] + Y[0] * c.t1[1] + Y[1] * c.t2[1] + Y[2] * c.n[1];
                    const T yz = c.c[2] + Y[0] * c.t1[2] + Y[1] * c.t2[2] + Y[2] * c.n[2];
                    gy = c.data32 ? (T)dirichlet_eval<float>(*c.dat, (float)yx, (float)yy, (float)yz)
                                  : dirichlet_eval<T>(*c.dat, yx, yy, yz);
                }
                sd += wj * green_ball_dny<T>(c.a, c.X, c.xn, Y, nl) * (gy - c.gx);
            }
        }
    }
}

// Gauss order from the distance ratio r (0: split further).  FP64 orders aim at
// 1e-15 relative for a singularity next to the middle of a panel edge, FP32
// orders at 1e-8.
__device__ __forceinline__ int order64(double r) {
    if (r >= 20.0) return 5;
    if (r >= 10.0) return 6;
    if (r >= 5.0) return 9;
    if (r >= 3.0) return 12;
    if (r >= 2.0) return 20;
    return 0;
}
__device__ __forceinline__ int order32(double r) {
    if (r >= 20.0) return 3;
    if (r >= 10.0) return 4;
    if (r >= 5.0) return 5;
    if (r >= 3.0) return 7;
    if (r >= 2.0) return 11;
    return 0;
}

// distance ratio of a sub-square: min distance from the singular points to the
// square's physical centre over the largest centre-to-(corner or edge midpoint)
// distance
// (also returns the physical lengths of the square's two mid-lines, lx along
// xi and le along eta, which decide where to split)
template <typename T>
__device__ T square_ratio(const Ctx<T> &c, const Region &R, T x0, T x1, T e0, T e1, bool withX, T &lx, T &le) {
    T uc, vc, jac, Yc[3], nl[3], J;
    map_uv<T>(R, (T)0.5 * (x0 + x1), (T)0.5 * (e0 + e1), uc, vc, jac);
    patch_point<T>(c.kind, c.R, uc, vc, Yc, nl, J);
    T rad = (T)0;
    T P[3][3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            if (a == 1 && b == 1) {
                P[1][1][0] = Yc[0]; P[1][1][1] = Yc[1]; P[1][1][2] = Yc[2];
                continue;
            }
            T u, v, Y[3];
            map_uv<T>(R, x0 + (T)0.5 * a * (x1 - x0), e0 + (T)0.5 * b * (e1 - e0), u, v, jac);
            patch_point<T>(c.kind, c.R, u, v, Y, nl, J);
            P[a][b][0] = Y[0]; P[a][b][1] = Y[1]; P[a][b][2] = Y[2];
            const T d2 = (Y[0] - Yc[0]) * (Y[0] - Yc[0]) + (Y[1] - Yc[1]) * (Y[1] - Yc[1]) +
                         (Y[2] - Yc[2]) * (Y[2] - Yc[2]);
            rad = fmax(rad, sqrt(d2));
        }
    lx = (T)0;
    le = (T)0;
    for (int k = 0; k < 2; ++k) {
        T dx = (T)0, de = (T)0;
        for (int d = 0; d < 3; ++d) {
            dx += (P[k + 1][1][d] - P[k][1][d]) * (P[k + 1][1][d] - P[k][1][d]);
            de += (P[1][k + 1][d] - P[1][k][d]) * (P[1][k + 1][d] - P[1][k][d]);
        }
        lx += sqrt(dx);
        le += sqrt(de);
    }
    T dmin = (T)INFINITY;
    if (withX) {
        const T d2 = (c.X[0] - Yc[0]) * (c.X[0] - Yc[0]) + (c.X[1] - Yc[1]) * (c.X[1] - Yc[1]) +
                     (c.X[2] - Yc[2]) * (c.X[2] - Yc[2]);
        dmin = sqrt(d2);
    }
    if (c.img) {
        const T d2 = (c.Xs[0] - Yc[0]) * (c.Xs[0] - Yc[0]) + (c.Xs[1] - Yc[1]) * (c.Xs[1] - Yc[1]) +
                     (c.Xs[2] - Yc[2]) * (c.Xs[2] - Yc[2]);
        dmin = fmin(dmin, sqrt(d2));
    }
    return rad > (T)0 ? dmin / rad : (T)INFINITY;
}

template <typename T>
__device__ void integrate_region(const Ctx<T> &c, const Region &R, bool withX, int min_order,
                                 const double *__restrict__ glx, const double *__restrict__ glw, T &sa, T &sd) {
    struct Sq { T x0, x1, e0, e1; int depth; };
    Sq stack[kStack];
    int sp = 0;
    stack[sp++] = Sq{(T)0, (T)1, (T)0, (T)1, 0};
    while (sp > 0) {
        const Sq q = stack[--sp];
        T lx, le;
        const T r = square_ratio<T>(c, R, q.x0, q.x1, q.e0, q.e1, withX, lx, le);
        int n = sizeof(T) == 8 ? order64((double)r) : order32((double)r);
        if (n == 0 && q.depth < kMaxDepth && sp + 4 <= kStack) {
            // split the long direction only while the square is more than 2:1
            const T xm = (T)0.5 * (q.x0 + q.x1), em = (T)0.5 * (q.e0 + q.e1);
            if (lx > (T)2 * le) {
                stack[sp++] = Sq{q.x0, xm, q.e0, q.e1, q.depth + 1};
                stack[sp++] = Sq{xm, q.x1, q.e0, q.e1, q.depth + 1};
            } else if (le > (T)2 * lx) {
                stack[sp++] = Sq{q.x0, q.x1, q.e0, em, q.depth + 1};
                stack[sp++] = Sq{q.x0, q.x1, em, q.e1, q.depth + 1};
            } else {
                stack[sp++] = Sq{q.x0, xm, q.e0, em, q.depth + 1};
                stack[sp++] = Sq{xm, q.x1, q.e0, em, q.depth + 1};
                stack[sp++] = Sq{q.x0, xm, em, q.e1, q.depth + 1};
                stack[sp++] = Sq{xm, q.x1, em, q.e1, q.depth + 1};
            }
            continue;
        }
        if (n == 0) n = sizeof(T) == 8 ? 20 : 11;
        if (n < min_order) n = min_order;
        if (R.tri) gauss_square<T>(c, R, q.x0, q.x1, q.e0, q.e1, n, glx, glw, sa, sd);
        else gauss_rect<T>(c, R, q.x0, q.x1, q.e0, q.e1, n, glx, glw, sa, sd);
    }
}

template <typename T>
__device__ void make_ctx(Ctx<T> &c, const PatchFrame &f, const double *X, double gx, const DData *dat) {
    c.kind = f.kind;
    c.a = (T)f.a;
    c.R = (T)f.R;
    for (int d = 0; d < 3; ++d) {
        c.X[d] = (T)X[d];
        c.c[d] = (T)f.c[d]; c.t1[d] = (T)f.t1[d]; c.t2[d] = (T)f.t2[d]; c.n[d] = (T)f.n[d];
    }
    const double xx = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
    c.xn = (T)sqrt(xx);
    c.img = xx > 0.0;
    if (c.img)
        for (int d = 0; d < 3; ++d) c.Xs[d] = (T)(f.a * f.a * X[d] / xx);
    c.needD = (f.kind == kCap);
    c.data32 = false;
    c.needA = true;
    c.gx = (T)gx;
    c.dat = dat;
}

struct AsmDev {
    const PatchFrame *frames;
    const int64_t *panel_off, *gamma_off, *mat_off;
    const int64_t *grows_off, *rep, *gmat_off;
    int64_t n_groups;
    const double *panel_loc, *panel_prm, *panel_aux, *panel_g;
    const double *gamma_loc, *gamma_w, *U;
    double *A, *b;
    DData dat;
    int64_t n_patches;
    int prec;
    int mode;
    const double *glx, *glw;
    const float *gpre;    // mode 2: data at the fixed per-panel rules
};

// self panel: triangles from the collocation point (uc, vc) to each side, each
// side cut into m pieces so that every Duffy triangle's far edge is no longer
// than its height (the angular factor of the transformed integrand then stays
// smooth for thin panels)
template <typename T>
__device__ void self_panel(const Ctx<T> &c, const PatchFrame &f, const double *prm, int min_order,
                           const double *glx, const double *glw, T &sa, T &sd) {
    const double S[2] = {prm[4], prm[5]};
    const double cu[5] = {prm[0], prm[1], prm[1], prm[0], prm[0]};
    const double cv[5] = {prm[2], prm[2], prm[3], prm[3], prm[2]};
    double PS[3], nl[3], J;
    patch_point<double>(f.kind, f.R, S[0], S[1], PS, nl, J);
    for (int e = 0; e < 4; ++e) {
        double PA[3], PB[3];
        patch_point<double>(f.kind, f.R, cu[e], cv[e], PA, nl, J);
        patch_point<double>(f.kind, f.R, cu[e + 1], cv[e + 1], PB, nl, J);
        const double ab[3] = {PB[0] - PA[0], PB[1] - PA[1], PB[2] - PA[2]};
        const double as[3] = {PS[0] - PA[0], PS[1] - PA[1], PS[2] - PA[2]};
        const double cr[3] = {ab[1] * as[2] - ab[2] * as[1], ab[2] * as[0] - ab[0] * as[2], ab[0] * as[1] - ab[1] * as[0]};
        const double L = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
        const double h = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / fmax(L, 1e-300);
        const int m = (int)fmin(64.0, fmax(1.0, ceil(L / fmax(h, 1e-300))));
        for (int k = 0; k < m; ++k) {
            const double ua = cu[e] + (cu[e + 1] - cu[e]) * k / m, va = cv[e] + (cv[e + 1] - cv[e]) * k / m;
            const double ub = cu[e] + (cu[e + 1] - cu[e]) * (k + 1) / m;
            const double vb = cv[e] + (cv[e + 1] - cv[e]) * (k + 1) / m;
            Region R;
            R.tri = true;
            R.p[0] = S[0]; R.p[1] = S[1];
            R.p[2] = ua - S[0]; R.p[3] = va - S[1];
            R.p[4] = ub - ua; R.p[5] = vb - va;
            R.det = fabs(R.p[2] * R.p[5] - R.p[3] * R.p[4]);
            if (R.det == 0.0) continue;
            integrate_region<T>(c, R, false, min_order, glx, glw, sa, sd);
        }
    }
}

// distance ratio of panel j (its bounding sphere) to the singular points of row X
__device__ __forceinline__ double panel_ratio(const Ctx<double> &c, const double *X, const double *ax) {
    double dmin = sqrt((X[0] - ax[0]) * (X[0] - ax[0]) + (X[1] - ax[1]) * (X[1] - ax[1]) + (X[2] - ax[2]) * (X[2] - ax[2]));
    if (c.img) {
        const double d2 = (c.Xs[0] - ax[0]) * (c.Xs[0] - ax[0]) + (c.Xs[1] - ax[1]) * (c.Xs[1] - ax[1]) +
                          (c.Xs[2] - ax[2]) * (c.Xs[2] - ax[2]);
        dmin = fmin(dmin, sqrt(d2));
    }
    return dmin / ax[3];
}

__global__ void __launch_bounds__(kAsmThreads) assemble_kernel(AsmDev P) {
    int64_t p, row;
    int n, i;
    double *Arow = nullptr;
    if (P.mode == 1) {
        const int64_t grp = find_group(P.grows_off, P.n_groups, (int64_t)blockIdx.x);
        i = (int)(blockIdx.x - P.grows_off[grp]);
        p = P.rep[grp];
        n = (int)(P.grows_off[grp + 1] - P.grows_off[grp]);
        row = P.panel_off[p] + i;
        Arow = P.A + P.gmat_off[grp] + (int64_t)i * n;
    } else {
        row = blockIdx.x;
        p = find_group(P.panel_off, P.n_patches, row);
        n = (int)(P.panel_off[p + 1] - P.panel_off[p]);
        i = (int)(row - P.panel_off[p]);
        if (P.mode == 0) Arow = P.A + P.mat_off[p] + (int64_t)i * n;
    }
    const PatchFrame f = P.frames[p];
    const int64_t poff = P.panel_off[p];
    __shared__ double red[2][kAsmThreads / 32];
    if (P.mode != 1 && f.status != DTN_OK) {
        if (Arow)
            for (int j = threadIdx.x; j < n; j += blockDim.x) Arow[j] = (i == j) ? 1.0 : 0.0;
        if (threadIdx.x == 0) P.b[row] = 0.0;
        return;
    }
    const double X[3] = {P.panel_loc[3 * row], P.panel_loc[3 * row + 1], P.panel_loc[3 * row + 2]};
    const double gx = P.panel_g[row];
    Ctx<double> c64;
    make_ctx<double>(c64, f, X, gx, &P.dat);
    c64.data32 = (P.prec == DTN_PREC_MIXED);
    if (P.mode == 1) c64.needD = false;
    Ctx<float> c32;
    make_ctx<float>(c32, f, X, gx, &P.dat);
    c32.data32 = true;
    if (P.mode == 2) c32.needA = false;
    double dsum = 0.0;
    const bool doD = (P.mode != 1) && (f.kind == kCap);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int64_t pj = poff + j;
        const double *prm = P.panel_prm + 6 * pj;
        if (P.mode == 2) {
            // double layer only: the integrand (g(y) - g(x_i)) dG/dn_y is bounded,
            // so fixed 8x8 rules with the data precomputed per patch (whole panel
            // when the panel is far, its four quarters when near) and a Duffy rule
            // on the self panel, all FP32
            if (!doD) break;
            float a32 = 0.f, d32 = 0.f;
            if (j == i) {
                self_panel<float>(c32, f, prm, 6, P.glx, P.glw, a32, d32);
            } else {
                const double r = panel_ratio(c64, X, P.panel_aux + 4 * pj);
                Region R;
                R.tri = false;
                R.p[0] = prm[0]; R.p[1] = prm[1] - prm[0]; R.p[2] = prm[2]; R.p[3] = prm[3] - prm[2];
                R.det = 0.0;
                const float *gp = P.gpre + pj * kPrePerPanel;
                if (r >= 2.0) {
                    gauss_rect<float>(c32, R, 0.f, 1.f, 0.f, 1.f, kPreN, P.glx, P.glw, a32, d32, gp);
                } else {
                    for (int s = 0; s < 4; ++s) {
                        const float x0 = 0.5f * (s & 1), e0 = 0.5f * (s >> 1);
                        gauss_rect<float>(c32, R, x0, x0 + 0.5f, e0, e0 + 0.5f, kPreN, P.glx, P.glw, a32, d32,
                                          gp + kPreCoarse + kPreCoarse * s);
                    }
                }
            }
            dsum += (double)d32;
            continue;
        }
        double sa = 0.0, sd = 0.0;
        if (j == i) {
            self_panel<double>(c64, f, prm, 16, P.glx, P.glw, sa, sd);
        } else {
            const double r = panel_ratio(c64, X, P.panel_aux + 4 * pj);
            Region R;
            R.tri = false;
            R.p[0] = prm[0]; R.p[1] = prm[1] - prm[0]; R.p[2] = prm[2]; R.p[3] = prm[3] - prm[2];
            R.det = 0.0;
            if (r >= 2.0) {
                if (P.mode == 0 && P.prec == DTN_PREC_MIXED) {
                    float a32 = 0.f, d32 = 0.f;
                    gauss_rect<float>(c32, R, 0.f, 1.f, 0.f, 1.f, order32(r), P.glx, P.glw, a32, d32);
                    sa = a32; sd = d32;
                } else {
                    gauss_rect<double>(c64, R, 0.0, 1.0, 0.0, 1.0, order64(r), P.glx, P.glw, sa, sd);
                }
            } else {
                integrate_region<double>(c64, R, true, 0, P.glx, P.glw, sa, sd);
            }
        }
        Arow[j] = sa;
        dsum += sd;
    }
    if (P.mode == 1) return;
    // Gamma term: sum_k W_k P(x_i, y_k) (U_k - g(x_i)), FP64
    const int64_t goff = P.gamma_off[p];
    const int nk = (int)(P.gamma_off[p + 1] - goff);
    double gsum = 0.0;
    for (int k = threadIdx.x; k < nk; k += blockDim.x) {
        const int64_t gk = goff + k;
        const double Y[3] = {P.gamma_loc[3 * gk], P.gamma_loc[3 * gk + 1], P.gamma_loc[3 * gk + 2]};
        gsum += P.gamma_w[gk] * poisson_ball<double>(f.a, X, Y) * (P.U[gk] - gx);
    }
    double v0 = dsum, v1 = gsum;
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { red[0][w] = v0; red[1][w] = v1; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < kAsmThreads / 32; ++k) { s0 += red[0][k]; s1 += red[1][k]; }
        P.b[row] = s0 - s1;
    }
}

// Data g at the fixed per-panel rules of the double-layer term (cap patches):
// points 0..63 the 8x8 Gauss rule on the panel, points 64..319 the same rule on
// each quarter of the panel (quarter s = 2 e + x of the parameter box).  One
// thread per point; the row kernels read these values instead of evaluating
// the harmonic data again for every collocation row.
__global__ void panel_gpre_kernel(DData dat, int64_t n_patches, int64_t total, const int64_t *__restrict__ panel_off,
                                  const PatchFrame *__restrict__ frames, const double *__restrict__ panel_prm,
                                  const double *__restrict__ glx, float *__restrict__ out) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int64_t pj = idx / kPrePerPanel;
    const int q = (int)(idx - pj * kPrePerPanel);
    const int64_t p = find_group(panel_off, n_patches, pj);
    const PatchFrame &f = frames[p];
    const double *prm = panel_prm + 6 * pj;
    double x0 = 0.0, x1 = 1.0, e0 = 0.0, e1 = 1.0;
    int k = q;
    if (q >= kPreCoarse) {
        const int s = (q - kPreCoarse) / kPreCoarse;
        k = (q - kPreCoarse) % kPreCoarse;
        x0 = 0.5 * (s & 1); x1 = x0 + 0.5;
        e0 = 0.5 * (s >> 1); e1 = e0 + 0.5;
    }
    const int i = k / kPreN, j = k % kPreN;
    const double *gx = glx + kPreN * (kPreN - 1) / 2;
    const double u = prm[0] + (0.5 * (x0 + x1) + 0.5 * (x1 - x0) * gx[i]) * (prm[1] - prm[0]);
    const double v = prm[2] + (0.5 * (e0 + e1) + 0.5 * (e1 - e0) * gx[j]) * (prm[3] - prm[2]);
    double Y[3], nl[3], J;
    patch_point<double>(f.kind, f.R, u, v, Y, nl, J);
    const double y0 = f.c[0] + Y[0] * f.t1[0] + Y[1] * f.t2[0] + Y[2] * f.n[0];
    const double y1 = f.c[1] + Y[0] * f.t1[1] + Y[1] * f.t2[1] + Y[2] * f.n[1];
    const double y2 = f.c[2] + Y[0] * f.t1[2] + Y[1] * f.t2[2] + Y[2] * f.n[2];
    out[idx] = dirichlet_eval<float>(dat, (float)y0, (float)y1, (float)y2);
}

__global__ void expand_kernel(int64_t n_patches, const int64_t *__restrict__ mat_off,
                              const int64_t *__restrict__ group_of, const int64_t *__restrict__ gmat_off,
                              const double *__restrict__ gA, double *__restrict__ A) {
    const int64_t p = blockIdx.y;
    if (p >= n_patches) return;
    const int64_t len = mat_off[p + 1] - mat_off[p];
    const double *src = gA + gmat_off[group_of[p]];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < len; k += (int64_t)gridDim.x * blockDim.x)
        A[mat_off[p] + k] = src[k];
}

}  // namespace

cudaError_t launch_assemble(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D, int prec, int mode,
                            const double *panel_loc, const double *panel_prm, const double *panel_aux,
                            const double *panel_g, const double *gamma_loc, const double *gamma_w,
                            const double *U, double *A, double *b, float *gpre, cudaStream_t s) {
    const int64_t rows = (mode == 1) ? L.grows_total : L.panels_total;
    if (rows == 0) return cudaSuccess;
    AsmDev P;
    P.frames = D.frames;
    P.panel_off = D.panel_off;
    P.gamma_off = D.gamma_off;
    P.mat_off = D.mat_off;
    P.grows_off = D.grows_off;
    P.rep = D.rep;
    P.gmat_off = D.gmat_off;
    P.n_groups = L.n_groups;
    P.panel_loc = panel_loc;
    P.panel_prm = panel_prm;
    P.panel_aux = panel_aux;
    P.panel_g = panel_g;
    P.gamma_loc = gamma_loc;
    P.gamma_w = gamma_w;
    P.U = U;
    P.A = A;
    P.b = b;
    P.dat = g->dd;
    P.n_patches = L.n_patches;
    P.prec = prec;
    P.mode = mode;
    P.glx = gl_x_dev();
    P.glw = gl_w_dev();
    P.gpre = gpre;
    if (mode == 2 && g->dg.kind == kBall) {
        // data at the fixed double-layer rules, once per patch
        const int64_t total = L.panels_total * kPrePerPanel;
        const int T = 256;
        panel_gpre_kernel<<<(unsigned)((total + T - 1) / T), T, 0, s>>>(g->dd, L.n_patches, total, D.panel_off,
                                                                        D.frames, panel_prm, P.glx, gpre);
    }
    assemble_kernel<<<(unsigned)rows, kAsmThreads, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t upload_sh_assemble(const ShTables &t) { return upload_sh_tables_here(t); }

cudaError_t launch_expand_matrices(const BatchLayout &L, const DevLayout &D, const double *gA, double *A,
                                   cudaStream_t s) {
    if (L.n_patches == 0) return cudaSuccess;
    expand_kernel<<<dim3(8, (unsigned)L.n_patches), 256, 0, s>>>(L.n_patches, D.mat_off, D.group_of, D.gmat_off, gA, A);
    return cudaGetLastError();
}

}  // namespace dtn
