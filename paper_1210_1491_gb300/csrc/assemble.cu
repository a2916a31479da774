// assemble.cu -- collocation matrix and right side of the first-kind local BIE
// (Eq. bw49-bw51) on piecewise-constant panels:
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
//                  parameter box is split, recursively.
//
// FP64 mode assembles A and b per patch (one CTA per row).  Mixed precision
// uses that A and b are linear in the patch data with coefficients that depend
// only on the patch shape: per shape group one FP64 matrix A, and one weight
// row per collocation point,
//   b_i = sum_q w_iq (s_q - c) - (g(x_i) - c) sum_q w_iq,
// whose samples s are the data at the 8 x 8 Gauss points of every panel (cap
// patches) followed by the walk estimates U_k, c a per-patch constant.  The
// double-layer weights are product rules, w_iq = int dG/dn_y(x_i, y) l_q(y) ds_y
// with l_q the panel's tensor Lagrange basis on those points (the 8 x 8 rule
// itself on far panels); the walk weights are -W_k P(x_i, y_k).  All right
// sides of a group are then one FP32 product (FP64 sums across k-tiles), the
// row sums of W taken in the same pass.
#include <cmath>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kAsmThreads = 128;
constexpr int kMaxDepth = 10;
constexpr int kStack = 40;
constexpr int kMaxRule = 20;   // highest Gauss order the rules below use
constexpr int kWtThreads = 128;
constexpr double kFarRatio = 5.0;   // right-side weights: the plain 8 x 8 rule from here on
constexpr int kSelfOrderW = 12;     // Duffy order of the self-panel product rules

template <typename T>
struct Ctx {
    int kind;
    T a, R;
    T X[3], xn;
    T Xs[3];
    bool img;
    bool needD;
    bool needA;    // accumulate the single-layer entry
    T gx;
    T c[3], t1[3], t2[3], n[3];
    const DData *dat;
    // second kind (Eq. bw55-bw59): A accumulates dG/dn_x, D the regularised
    // right-side integrand K (g - l) + dG/dn_x a.n_y, l(Y) = gx + ga.(Y - X)
    bool sk;
    T nx[3], ga[3];
    const Piece *pc;   // wrapped patch: the piece of the panel being integrated ...
    int sub;           // ... and its sub-range (the panel's quadrature parameters)
};

// point of the panel's quadrature parameters for any patch kind
template <typename T>
__device__ __forceinline__ void ctx_point(const Ctx<T> &c, T u, T v, T *Y, T *nl, T &J) {
    if (c.kind == kWrapped) wrapped_point_q<T>(*c.pc, c.sub, u, v, Y, nl, J);
    else patch_point<T>(c.kind, c.R, u, v, Y, nl, J);
}

// the piece and sub-range of a wrapped patch's panel (panel_piece = piece * kMaxSub + sub)
template <typename T>
__device__ __forceinline__ void ctx_panel(Ctx<T> &c, const Piece *pcs, int32_t code) {
    if (!pcs) return;
    c.pc = pcs + code / kMaxSub;
    c.sub = code % kMaxSub;
}

// One quadrature point of the second-kind integrands (FP64 only).
__device__ __forceinline__ void sk_point(const Ctx<double> &c, const double *Y, const double *nl, double wj,
                                         double &sa, double &sd) {
    const double yn = sqrt(Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2]);
    // dG/dn_x(X, Y) = n_x . grad_X G(X, Y) = n_x . (grad_y G)(Y, X): G is symmetric
    const double dnx = green_ball_dny<double>(c.a, Y, yn, c.X, c.nx);
    if (c.needA) sa += wj * dnx;
    if (c.needD) {
        const double yx = c.c[0] + Y[0] * c.t1[0] + Y[1] * c.t2[0] + Y[2] * c.n[0];
        const double yy = c.c[1] + Y[0] * c.t1[1] + Y[1] * c.t2[1] + Y[2] * c.n[1];
        const double yz = c.c[2] + Y[0] * c.t1[2] + Y[1] * c.t2[2] + Y[2] * c.n[2];
        const double l = c.gx + c.ga[0] * (Y[0] - c.X[0]) + c.ga[1] * (Y[1] - c.X[1]) + c.ga[2] * (Y[2] - c.X[2]);
        const double an = c.ga[0] * nl[0] + c.ga[1] * nl[1] + c.ga[2] * nl[2];
        sd += wj * (green_ball_dnn(c.a, c.X, c.nx, Y, nl) * (dirichlet_eval<double>(*c.dat, yx, yy, yz) - l) +
                    dnx * an);
    }
}
template <typename T>
__device__ __forceinline__ void sk_point(const Ctx<T> &, const T *, const T *, T, T &, T &) {}

template <typename T>
__device__ __forceinline__ void eval_point(const Ctx<T> &c, T u, T v, T w, T &sa, T &sd) {
    T Y[3], nl[3], J;
    ctx_point<T>(c, u, v, Y, nl, J);
    const T wj = w * J;
    if (c.sk) {
        sk_point(c, Y, nl, wj, sa, sd);
        return;
    }
    if (c.needA) sa += wj * green_ball<T>(c.a, c.X, c.xn, Y);
    if (c.needD) {
        const T yx = c.c[0] + Y[0] * c.t1[0] + Y[1] * c.t2[0] + Y[2] * c.n[0];
        const T yy = c.c[1] + Y[0] * c.t1[1] + Y[1] * c.t2[1] + Y[2] * c.n[1];
        const T yz = c.c[2] + Y[0] * c.t1[2] + Y[1] * c.t2[2] + Y[2] * c.n[2];
        const T gy = dirichlet_eval<T>(*c.dat, yx, yy, yz);
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

// Tensor Gauss rule of order n on a rectangle of the parameter box.  The map is
// separable, so the sines and cosines of u and of v are taken once per Gauss line.
template <typename T>
__device__ void gauss_rect(const Ctx<T> &c, const Region &R, T x0, T x1, T e0, T e1, int n,
                           const double *__restrict__ glx, const double *__restrict__ glw, T &sa, T &sd) {
    const double *gx = glx + n * (n - 1) / 2, *gw = glw + n * (n - 1) / 2;
    const T hx = (T)0.5 * (x1 - x0), mx = (T)0.5 * (x0 + x1);
    const T he = (T)0.5 * (e1 - e0), me = (T)0.5 * (e0 + e1);
    const T du = (T)R.p[1], dv = (T)R.p[3];
    const T jac = du * dv;
    if (c.kind == kWrapped) {
        // piece of a wrapped patch: Y = Pl + u B(w), J = u Jf(w), the lines in w
        // taken once each
        T Bs[kMaxRule][3], Jfs[kMaxRule];
        for (int j = 0; j < n; ++j) {
            double B[3], Jf;
            wrapped_line(*c.pc, c.sub, (double)((T)R.p[2] + (me + he * (T)gx[j]) * dv), B, Jf);
            for (int d = 0; d < 3; ++d) Bs[j][d] = (T)B[d];
            Jfs[j] = (T)Jf;
        }
        const T nl[3] = {(T)c.pc->nl[0], (T)c.pc->nl[1], (T)c.pc->nl[2]};
        const T Pl[3] = {(T)c.pc->Pl[0], (T)c.pc->Pl[1], (T)c.pc->Pl[2]};
        for (int i = 0; i < n; ++i) {
            const T u = (T)R.p[0] + (mx + hx * (T)gx[i]) * du;
            const T wi = (T)gw[i] * hx * he * jac;
            for (int j = 0; j < n; ++j) {
                const T Y[3] = {Pl[0] + u * Bs[j][0], Pl[1] + u * Bs[j][1], Pl[2] + u * Bs[j][2]};
                const T wj = wi * (T)gw[j] * u * Jfs[j];
                if (c.needA) sa += wj * green_ball<T>(c.a, c.X, c.xn, Y);
                if (c.needD) {
                    const T yx = c.c[0] + Y[0] * c.t1[0] + Y[1] * c.t2[0] + Y[2] * c.n[0];
                    const T yy = c.c[1] + Y[0] * c.t1[1] + Y[1] * c.t2[1] + Y[2] * c.n[1];
                    const T yz = c.c[2] + Y[0] * c.t1[2] + Y[1] * c.t2[2] + Y[2] * c.n[2];
                    const T gy = dirichlet_eval<T>(*c.dat, yx, yy, yz);
                    sd += wj * green_ball_dny<T>(c.a, c.X, c.xn, Y, nl) * (gy - c.gx);
                }
            }
        }
        return;
    }
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
            if (c.sk) {
                const T nl[3] = {nu * cvs[j], nu * svs[j], nz};
                sk_point(c, Y, nl, wj, sa, sd);
                continue;
            }
            if (c.needA) sa += wj * green_ball<T>(c.a, c.X, c.xn, Y);
            if (c.needD) {
                const T nl[3] = {nu * cvs[j], nu * svs[j], nz};
                const T yx = c.c[0] + Y[0] * c.t1[0] + Y[1] * c.t2[0] + Y[2] * c.n[0];
                const T yy = c.c[1] + Y[0] * c.t1[1] + Y[1] * c.t2[1] + Y[2] * c.n[1];
                const T yz = c.c[2] + Y[0] * c.t1[2] + Y[1] * c.t2[2] + Y[2] * c.n[2];
                const T gy = dirichlet_eval<T>(*c.dat, yx, yy, yz);
                sd += wj * green_ball_dny<T>(c.a, c.X, c.xn, Y, nl) * (gy - c.gx);
            }
        }
    }
}

// Gauss order from the distance ratio r (0: split further), aiming at 1e-15
// relative for a singularity next to the middle of a panel edge.
__device__ __forceinline__ int order64(double r) {
    if (r >= 20.0) return 5;
    if (r >= 10.0) return 6;
    if (r >= 5.0) return 9;
    if (r >= 3.0) return 12;
    if (r >= 2.0) return 20;
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
    ctx_point<T>(c, uc, vc, Yc, nl, J);
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
            ctx_point<T>(c, u, v, Y, nl, J);
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

// Adaptive cover of a region's unit parameter square: sub-squares whose ratio
// asks for more than the highest order are split (the long direction only
// while the square is more than 2:1); fn(x0, x1, e0, e1, n) integrates each
// accepted sub-square with Gauss order n.
template <typename T, typename Fn>
__device__ void adaptive_squares(const Ctx<T> &c, const Region &R, bool withX, int min_order, Fn &&fn) {
    struct Sq { T x0, x1, e0, e1; int depth; };
    Sq stack[kStack];
    int sp = 0;
    stack[sp++] = Sq{(T)0, (T)1, (T)0, (T)1, 0};
    while (sp > 0) {
        const Sq q = stack[--sp];
        T lx, le;
        const T r = square_ratio<T>(c, R, q.x0, q.x1, q.e0, q.e1, withX, lx, le);
        int n = order64((double)r);
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
        if (n == 0) n = kMaxRule;
        if (n < min_order) n = min_order;
        fn(q.x0, q.x1, q.e0, q.e1, n);
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
    // dG/dn_y vanishes on a plane through c: the S integral of the right side
    // is needed on caps and on a wrapped patch's other faces
    c.needD = (f.kind == kCap || f.kind == kWrapped);
    c.needA = true;
    c.gx = (T)gx;
    c.dat = dat;
    c.sk = false;
    c.pc = nullptr;
    c.sub = 0;
}

struct PanelStatic32;

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
    int mode;   // 0 matrix and right side per patch, 1 matrix per shape group, 2 right side only
    int sk;     // second-kind system (1/2 I - D) q = b instead of Eq. bw49-bw51
    int only_wrapped;   // mode 2: the rows of wrapped patches only (the others are left untouched)
    const int64_t *group_of;   // mode 2: a wrapped patch's group (its matrix in A, gmat_off)
    const PanelStatic32 *pstat;   // mixed-precision wrapped pass: per-panel FP32 maps
    const double *glx, *glw;
    const Piece *pieces;        // n_patches x kMaxPieces, or nullptr
    const int32_t *panel_piece; // per panel
};

// self panel: triangles from the collocation point (uc, vc) to each side, each
// side cut into m pieces so that every Duffy triangle's far edge is no longer
// than its height (the angular factor of the transformed integrand then stays
// smooth for thin panels)
// (fn(R) integrates over one triangle R)
template <typename Fn>
__device__ void self_triangles(const Ctx<double> &c, const double *prm, Fn &&fn) {
    const double S[2] = {prm[4], prm[5]};
    const double cu[5] = {prm[0], prm[1], prm[1], prm[0], prm[0]};
    const double cv[5] = {prm[2], prm[2], prm[3], prm[3], prm[2]};
    double PS[3], nl[3], J;
    ctx_point<double>(c, S[0], S[1], PS, nl, J);
    for (int e = 0; e < 4; ++e) {
        double PA[3], PB[3];
        ctx_point<double>(c, cu[e], cv[e], PA, nl, J);
        ctx_point<double>(c, cu[e + 1], cv[e + 1], PB, nl, J);
        const double ab[3] = {PB[0] - PA[0], PB[1] - PA[1], PB[2] - PA[2]};
        const double as[3] = {PS[0] - PA[0], PS[1] - PA[1], PS[2] - PA[2]};
        const double cr[3] = {ab[1] * as[2] - ab[2] * as[1], ab[2] * as[0] - ab[0] * as[2], ab[0] * as[1] - ab[1] * as[0]};
        const double L = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
        const double h = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / fmax(L, 1e-300);
        int m = (int)fmin(64.0, fmax(1.0, ceil(L / fmax(h, 1e-300))));
        // a side that maps to one point (the polar origin of a ring-0 panel):
        // the triangle is a sliver whose angular factor still varies across the
        // side's parameter range; four pieces
        const double sa = sqrt(as[0] * as[0] + as[1] * as[1] + as[2] * as[2]);
        if (L <= 1e-9 * sa) m = 4;
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
            fn(R);
        }
    }
}


// Self panel of a wrapped patch, whose panels can be long and thin (a sector of
// a strip along a box edge): the parameter box is cut at the singular point
// into four quadrants, and a quadrant whose physical sides differ by more than
// 2:1 is cut along its long side at lengths l, 2l, 4l, ... from the point (l the
// short side), so that every piece is about as long as its distance from the
// point.  The piece at the point takes two Duffy triangles from it, their far
// sides cut as in self_triangles (fn(R, false, 16)); the others the adaptive
// cover with the point as a singular point (fn(R, true, 0)).
template <typename Fn>
__device__ void self_regions(const Ctx<double> &c, const double *prm, Fn &&fn) {
    const double us = prm[4], ws = prm[5];
    const double ucs[2] = {prm[0], prm[1]}, wcs[2] = {prm[2], prm[3]};
    double X[3], nl[3], J;
    ctx_point<double>(c, us, ws, X, nl, J);
    auto dist = [](const double *A, const double *B) {
        return sqrt((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]));
    };
    for (int qu = 0; qu < 2; ++qu)
        for (int qw = 0; qw < 2; ++qw) {
            const double uC = ucs[qu], wC = wcs[qw];
            if (uC == us || wC == ws) continue;
            double Pa[3], Pm[3], Pb[3];
            ctx_point<double>(c, uC, ws, Pa, nl, J);
            ctx_point<double>(c, us, ws + 0.5 * (wC - ws), Pm, nl, J);
            ctx_point<double>(c, us, wC, Pb, nl, J);
            const double lu = dist(Pa, X), lw = dist(Pm, X) + dist(Pb, Pm);
            // graded direction (1: u, 2: w) and the first cut as a fraction
            int along = 0;
            double f0 = 1.0;
            if (lw > 2.0 * lu) { along = 2; f0 = lu / lw; }
            else if (lu > 2.0 * lw) { along = 1; f0 = lw / lu; }
            f0 = fmax(f0, 1.0 / 1048576.0);
            double fa = 0.0, fb = f0;
            for (int k = 0;; ++k) {
                double a1 = uC, b1 = wC, a0 = us, b0 = ws;
                if (along == 1) { a0 = us + fa * (uC - us); a1 = us + fb * (uC - us); }
                if (along == 2) { b0 = ws + fa * (wC - ws); b1 = ws + fb * (wC - ws); }
                if (k == 0) {
                    // Duffy triangles (S, (a1, ws), (a1, b1)) and (S, (a1, b1), (us, b1)),
                    // each far side cut into pieces no longer than the triangle's
                    // height (four if it maps to one point)
                    const double ta[2][2] = {{a1, ws}, {a1, b1}}, tb[2][2] = {{a1, b1}, {us, b1}};
                    for (int t = 0; t < 2; ++t) {
                        double PA[3], PB[3];
                        ctx_point<double>(c, ta[t][0], ta[t][1], PA, nl, J);
                        ctx_point<double>(c, tb[t][0], tb[t][1], PB, nl, J);
                        const double ab[3] = {PB[0] - PA[0], PB[1] - PA[1], PB[2] - PA[2]};
                        const double as[3] = {X[0] - PA[0], X[1] - PA[1], X[2] - PA[2]};
                        const double cr[3] = {ab[1] * as[2] - ab[2] * as[1], ab[2] * as[0] - ab[0] * as[2],
                                              ab[0] * as[1] - ab[1] * as[0]};
                        const double L = sqrt(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
                        const double h = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / fmax(L, 1e-300);
                        int m = (int)fmin(64.0, fmax(1.0, ceil(L / fmax(h, 1e-300))));
                        if (L <= 1e-9 * sqrt(as[0] * as[0] + as[1] * as[1] + as[2] * as[2])) m = 4;
                        for (int e = 0; e < m; ++e) {
                            const double Au = ta[t][0] + (tb[t][0] - ta[t][0]) * e / m;
                            const double Aw = ta[t][1] + (tb[t][1] - ta[t][1]) * e / m;
                            const double Bu = ta[t][0] + (tb[t][0] - ta[t][0]) * (e + 1) / m;
                            const double Bw = ta[t][1] + (tb[t][1] - ta[t][1]) * (e + 1) / m;
                            Region R;
                            R.tri = true;
                            R.p[0] = us; R.p[1] = ws;
                            R.p[2] = Au - us; R.p[3] = Aw - ws;
                            R.p[4] = Bu - Au; R.p[5] = Bw - Aw;
                            R.det = fabs(R.p[2] * R.p[5] - R.p[3] * R.p[4]);
                            if (R.det > 0.0) fn(R, false, 16);
                        }
                    }
                } else {
                    Region R;
                    R.tri = false;
                    R.p[0] = fmin(a0, a1); R.p[1] = fabs(a1 - a0);
                    R.p[2] = fmin(b0, b1); R.p[3] = fabs(b1 - b0);
                    R.det = 0.0;
                    fn(R, true, 0);
                }
                if (along == 0 || fb >= 1.0) break;
                fa = fb;
                fb = fmin(1.0, 2.0 * fb);
            }
        }
}

// ---------------------------------------------------------------------------
// Mixed precision on wrapped patches: FP32 rules in offset form.
//
// A wrapped patch lies anywhere in the box and the data of a distant source
// vary little over it, so points formed from coordinates, and g(y) - g(x),
// would lose most of FP32's digits.  Instead every point is the offset of its
// quadrature parameters (du, dw) from the panel centre C = (uc, wc), pushed
// through the sub-range's map: on a side-bounded sub-range B(w) = e_n + w e_t
// (so B(w) - B(wc) = dw e_t); on a circle-bounded one B(v) = rho(v) e(v) with
// e(v) - e(vc) = 2 sin(dv/2) e'(vc + dv/2) and, when P is off the slice centre,
// rho(v) - rho(vc) = (p - pc) (-1 + (p + pc) / (sqrt D + sqrt Dc)), p = (P -
// cf).e, D = p^2 - |P - cf|^2 + rf^2.  The point's offset from C is du B(w) +
// uc (B(w) - B(wc)); C's offsets from X and from its Kelvin image X*, and the
// data's e = x - x0, are formed in FP64 once per (row, panel).  |Y - X|, |Y -
// X*| and the data difference -q d.(2e + d) / (|e + d| |e| (|e + d| + |e|))
// then keep FP32's relative accuracy, down to the collocation point itself
// (the self panel's centre), where the Duffy factor removes 1/r as in FP64.
// Adaptive-cover decisions are taken on the same FP32 offsets.  Other data
// than a point source are differenced in FP64.

struct Off32 {
    int type;                          // 1: rectangle side, 0: circle about P, 2: circle, P off centre
    float uc, wc;
    float eg[3], tg[3], js;            // side: B(w) = eg + w tg (global axes), Jacobian factor js
    float Ug[3], Vg[3], rf;            // circle: e(v) = cos v Ug + sin v Vg
    float w2[2], ww, pc, sDc, rhoc;    // off-centre circle
    float Dc[3], Ds[3];                // C - X, C - X* (global axes)
    float k1, k2, gi, g0;              // G = (1/r - gi/rs - g0)/4pi, dG/dn_y = (k1/r^3 + k2/rs^3)/4pi
    bool img;
};

struct Row32 {
    double xg[3], gx;                  // x (global) and g(x)
    float e[3], ne, qf;                // point source: e = x - x0, |e|, q/4pi
    bool point, needA, needD;
    const DData *dat;
};

__device__ void row32_setup(const Ctx<double> &c, Row32 &R) {
    for (int d = 0; d < 3; ++d) R.xg[d] = c.c[d] + c.X[0] * c.t1[d] + c.X[1] * c.t2[d] + c.X[2] * c.n[d];
    R.gx = c.gx;
    R.dat = c.dat;
    const int dk = c.dat->kind;
    R.point = (dk == kPointSource);
    R.needA = c.needA;
    R.needD = c.needD && dk != kConstant;
    R.qf = c.dat->q_f;
    double sq = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double ed = R.point ? R.xg[d] - c.dat->x0[d] : 0.0;
        sq += ed * ed;
        R.e[d] = (float)ed;
    }
    R.ne = (float)sqrt(sq);
}

// Per wrapped panel, once per call (`wrapped_static_kernel`): its map about its
// centre C in FP32, C in global axes (FP64, from the ball centre), and its
// bounding sphere's centre as an FP32 offset from C.
struct PanelStatic32 {
    double Ycg[3];
    float uc, wc;
    float eg[3], tg[3], js;
    float Ug[3], Vg[3], rf;
    float w2[2], ww, pc, sDc, rhoc;
    float Ao[3], arad;
    int type, piece;
};

// local (t1, t2, n) to global axes, one expression wherever it is used, so
// that the same local point gives the same global offsets bit for bit
__device__ __forceinline__ void to_global(const PatchFrame &f, const double *v, double *g) {
    for (int d = 0; d < 3; ++d) g[d] = v[0] * f.t1[d] + v[1] * f.t2[d] + v[2] * f.n[d];
}

__device__ void panel_static32(const PatchFrame &f, const Piece &q, int k, int j, const double *prm, const double *Yc,
                               const double *aux, PanelStatic32 &S) {
    S.piece = k;
    to_global(f, Yc, S.Ycg);
    const double uc = prm[4], wc = prm[5];
    S.uc = (float)uc;
    S.wc = (float)wc;
    S.type = q.stype[j] ? 1 : (q.centred ? 0 : 2);
    double g[3];
    to_global(f, q.en[j], g);
    for (int d = 0; d < 3; ++d) S.eg[d] = (float)g[d];
    to_global(f, q.et[j], g);
    for (int d = 0; d < 3; ++d) S.tg[d] = (float)g[d];
    to_global(f, q.Ul, g);
    for (int d = 0; d < 3; ++d) S.Ug[d] = (float)g[d];
    to_global(f, q.Vl, g);
    for (int d = 0; d < 3; ++d) S.Vg[d] = (float)g[d];
    S.js = (float)(q.sdist[j] * q.sdist[j]);
    S.rf = (float)q.rf;
    if (S.type == 2) {
        const double w0 = q.P[0] - q.cf[0], w1 = q.P[1] - q.cf[1];
        double sv, cv;
        sincos(wc, &sv, &cv);
        const double pc = w0 * cv + w1 * sv, ww = w0 * w0 + w1 * w1;
        const double sDc = sqrt(fmax(0.0, pc * pc - ww + q.rf * q.rf));
        S.w2[0] = (float)w0; S.w2[1] = (float)w1;
        S.ww = (float)ww; S.pc = (float)pc; S.sDc = (float)sDc; S.rhoc = (float)(-pc + sDc);
    } else {
        S.w2[0] = S.w2[1] = S.ww = S.pc = S.sDc = 0.f;
        S.rhoc = S.rf;
    }
    const double ao[3] = {aux[0] - Yc[0], aux[1] - Yc[1], aux[2] - Yc[2]};
    to_global(f, ao, g);
    for (int d = 0; d < 3; ++d) S.Ao[d] = (float)g[d];
    S.arad = (float)aux[3];
}

// Per row (shared memory): X and its Kelvin image in global axes, and the
// normal-derivative constants of each piece
struct RowStatic32 {
    double Xg[3], Xsg[3];
    float k1[kMaxPieces], k2[kMaxPieces], gi, g0;
    int img;
};

__device__ void row_static32(const Ctx<double> &c, const PatchFrame &f, const Piece *pcs, RowStatic32 &R) {
    to_global(f, c.X, R.Xg);
    const double zero[3] = {0.0, 0.0, 0.0};
    to_global(f, c.img ? c.Xs : zero, R.Xsg);
    const double xx = c.xn * c.xn;
    for (int k = 0; k < f.npiece && k < kMaxPieces; ++k) {
        const Piece &q = pcs[k];
        double nyX = 0.0, nyP = 0.0, nyXP = 0.0;
        for (int d = 0; d < 3; ++d) {
            nyX += q.nl[d] * c.X[d];
            nyP += q.nl[d] * q.Pl[d];
            nyXP += q.nl[d] * (c.X[d] - q.Pl[d]);
        }
        R.k1[k] = (float)nyXP;
        R.k2[k] = c.img ? (float)(c.a * (xx * nyP - c.a * c.a * nyX) / (xx * c.xn)) : 0.f;
    }
    R.img = c.img;
    R.gi = c.img ? (float)(c.a / c.xn) : 0.f;
    R.g0 = c.img ? 0.f : (float)(1.0 / c.a);
}

// the panel's map about C and C's offsets from X and X*: the FP64 work of a
// (row, panel) pair is six subtractions
__device__ __forceinline__ void off32_make(const PanelStatic32 &S, const RowStatic32 &R, Off32 &O) {
    O.type = S.type;
    O.uc = S.uc;
    O.wc = S.wc;
    for (int d = 0; d < 3; ++d) {
        O.eg[d] = S.eg[d]; O.tg[d] = S.tg[d]; O.Ug[d] = S.Ug[d]; O.Vg[d] = S.Vg[d];
        O.Dc[d] = (float)(S.Ycg[d] - R.Xg[d]);
        O.Ds[d] = R.img ? (float)(S.Ycg[d] - R.Xsg[d]) : 0.f;
    }
    O.js = S.js; O.rf = S.rf;
    O.w2[0] = S.w2[0]; O.w2[1] = S.w2[1];
    O.ww = S.ww; O.pc = S.pc; O.sDc = S.sDc; O.rhoc = S.rhoc;
    O.k1 = R.k1[S.piece]; O.k2 = R.k2[S.piece];
    O.gi = R.gi; O.g0 = R.g0;
    O.img = R.img != 0;
}

// distance ratio of the panel (its bounding sphere) to X and X*, in FP32
__device__ __forceinline__ float ratio_panel32(const PanelStatic32 &S, const Off32 &O) {
    const float ax = O.Dc[0] + S.Ao[0], ay = O.Dc[1] + S.Ao[1], az = O.Dc[2] + S.Ao[2];
    float d2 = ax * ax + ay * ay + az * az;
    if (O.img) {
        const float bx = O.Ds[0] + S.Ao[0], by = O.Ds[1] + S.Ao[1], bz = O.Ds[2] + S.Ao[2];
        d2 = fminf(d2, bx * bx + by * by + bz * bz);
    }
    return sqrtf(d2) / S.arad;
}

__global__ void wrapped_static_kernel(int64_t n_patches, int64_t total, const int64_t *__restrict__ panel_off,
                                      const PatchFrame *__restrict__ frames, const Piece *__restrict__ pieces,
                                      const int32_t *__restrict__ panel_piece, const double *__restrict__ prm,
                                      const double *__restrict__ loc, const double *__restrict__ aux,
                                      PanelStatic32 *__restrict__ out) {
    const int64_t gidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gidx >= total) return;
    const int64_t p = find_group(panel_off, n_patches, gidx);
    const PatchFrame &f = frames[p];
    if (f.kind != kWrapped || f.status != DTN_OK) return;
    const int code = panel_piece[gidx];
    const int k = code / kMaxSub, j = code - k * kMaxSub;
    panel_static32(f, pieces[p * kMaxPieces + k], k, j, prm + 6 * gidx, loc + 3 * gidx, aux + 4 * gidx, out[gidx]);
}

// line dw of the map: B(wc + dw), uc (B(wc + dw) - B(wc)) (global axes), Jacobian factor
// (not inlined: one copy of the sine and cosine code keeps the kernel within the
// instruction cache, whose misses otherwise stalled it most)
__device__ __noinline__ void line32(const Off32 &O, float dw, float *Bg, float *dBg, float &Jf) {
    if (O.type == 1) {
        const float w = O.wc + dw;
        for (int d = 0; d < 3; ++d) {
            Bg[d] = fmaf(w, O.tg[d], O.eg[d]);
            dBg[d] = O.uc * (dw * O.tg[d]);
        }
        Jf = O.js;
        return;
    }
    float sv, cv, sm, cm;
    sincosf(O.wc + dw, &sv, &cv);
    sincosf(O.wc + 0.5f * dw, &sm, &cm);
    const float h = 2.f * sinf(0.5f * dw);
    const float de0 = -h * sm, de1 = h * cm;   // e(v) - e(vc) in (U, V)
    float rho = O.rf, drho = 0.f;
    if (O.type == 2) {
        const float pv = O.w2[0] * cv + O.w2[1] * sv;
        const float dp = O.w2[0] * de0 + O.w2[1] * de1;
        const float sD = sqrtf(fmaxf(0.f, pv * pv - O.ww + O.rf * O.rf));
        rho = -pv + sD;
        drho = dp * (-1.f + __fdividef(pv + O.pc, sD + O.sDc));
    }
    for (int d = 0; d < 3; ++d) {
        const float e = cv * O.Ug[d] + sv * O.Vg[d];
        Bg[d] = rho * e;
        dBg[d] = O.uc * (drho * e + O.rhoc * (de0 * O.Ug[d] + de1 * O.Vg[d]));
    }
    Jf = rho * rho;
}

// the point at offsets (du, dw) from C: its offset from C (global axes) and u Jf
__device__ __forceinline__ void pos32(const Off32 &O, float du, float dw, float *o, float &J) {
    float Bg[3], dBg[3], Jf;
    line32(O, dw, Bg, dBg, Jf);
    for (int d = 0; d < 3; ++d) o[d] = fmaf(du, Bg[d], dBg[d]);
    J = (O.uc + du) * Jf;
}

// one point by its offset o from C, weight w (Gauss weights, Jacobians)
__device__ __forceinline__ void eval32(const Off32 &O, const Row32 &R, const float *o, float w, float &la,
                                       float &ld) {
    const float dx = o[0] + O.Dc[0], dy = o[1] + O.Dc[1], dz = o[2] + O.Dc[2];
    const float ir = rsqrtf(dx * dx + dy * dy + dz * dz);
    float irs = 0.f;
    if (O.img) {
        const float sx = o[0] + O.Ds[0], sy = o[1] + O.Ds[1], sz = o[2] + O.Ds[2];
        irs = rsqrtf(sx * sx + sy * sy + sz * sz);
    }
    if (R.needA) la += w * (ir - O.gi * irs - O.g0);
    if (R.needD) {
        float dg;
        if (R.point) {
            const float px = R.e[0] + dx, py = R.e[1] + dy, pz = R.e[2] + dz;
            const float rp = sqrtf(px * px + py * py + pz * pz);
            const float num = dx * (R.e[0] + px) + dy * (R.e[1] + py) + dz * (R.e[2] + pz);
            dg = -R.qf * __fdividef(num, rp * R.ne * (rp + R.ne));
        } else {
            dg = (float)(dirichlet_eval<double>(*R.dat, R.xg[0] + (double)dx, R.xg[1] + (double)dy,
                                               R.xg[2] + (double)dz) - R.gx);
        }
        ld += w * (O.k1 * ir * ir * ir + O.k2 * irs * irs * irs) * dg;
    }
}

// A region in offsets from C: a box (du = a0 + x da, dw = b0 + e db) or a
// Duffy triangle from C (du = x (E1u + e E2u), dw = x (E1w + e E2w), Jacobian x det)
struct Reg32 {
    bool tri;
    float a0, da, b0, db;
    float E1[2], E2[2], det;
};

__device__ __forceinline__ void map32(const Reg32 &R, float x, float e, float &du, float &dw, float &jac) {
    if (!R.tri) {
        du = fmaf(x, R.da, R.a0);
        dw = fmaf(e, R.db, R.b0);
        jac = R.da * R.db;
    } else {
        du = x * fmaf(e, R.E2[0], R.E1[0]);
        dw = x * fmaf(e, R.E2[1], R.E1[1]);
        jac = x * R.det;
    }
}

// Gauss order per direction of the FP32 rules at distance ratio r (0: split):
// about two thirds of order64's points per direction, ~1e-10, below FP32 rounding
__device__ __forceinline__ int order32r(float r) {
    if (r >= 20.f) return 4;
    if (r >= 10.f) return 4;
    if (r >= 5.f) return 6;
    if (r >= 3.f) return 8;
    if (r >= 2.f) return 14;
    return 0;
}

// the adaptive cover of order64/adaptive_squares on FP32 offsets, taken by a
// whole warp: the square's nine points (corners, edge midpoints, centre) are
// placed by lanes 0-8, one each, and shared by shuffles, so that every lane
// takes the same decision on the same values
__device__ float ratio32(const Off32 &O, const Reg32 &R, float x0, float x1, float e0, float e1, bool withX, int lane,
                         float &lx, float &le) {
    float P[3][3][3], mine[3] = {0.f, 0.f, 0.f};
    if (lane < 9) {
        const int a = lane / 3, b = lane - 3 * (lane / 3);
        float J, du, dw, jac;
        map32(R, x0 + 0.5f * a * (x1 - x0), e0 + 0.5f * b * (e1 - e0), du, dw, jac);
        pos32(O, du, dw, mine, J);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
        for (int d = 0; d < 3; ++d) P[k / 3][k % 3][d] = __shfl_sync(0xffffffffu, mine[d], k);
    const float *Yc = P[1][1];
    float rad2 = 0.f;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const float d0 = P[a][b][0] - Yc[0], d1 = P[a][b][1] - Yc[1], d2 = P[a][b][2] - Yc[2];
            rad2 = fmaxf(rad2, d0 * d0 + d1 * d1 + d2 * d2);
        }
    lx = 0.f;
    le = 0.f;
    for (int k = 0; k < 2; ++k) {
        float dx = 0.f, de = 0.f;
        for (int d = 0; d < 3; ++d) {
            dx += (P[k + 1][1][d] - P[k][1][d]) * (P[k + 1][1][d] - P[k][1][d]);
            de += (P[1][k + 1][d] - P[1][k][d]) * (P[1][k + 1][d] - P[1][k][d]);
        }
        lx += sqrtf(dx);
        le += sqrtf(de);
    }
    float dmin2 = INFINITY;
    if (withX) {
        const float x = Yc[0] + O.Dc[0], y = Yc[1] + O.Dc[1], z = Yc[2] + O.Dc[2];
        dmin2 = x * x + y * y + z * z;
    }
    if (O.img) {
        const float x = Yc[0] + O.Ds[0], y = Yc[1] + O.Ds[1], z = Yc[2] + O.Ds[2];
        dmin2 = fminf(dmin2, x * x + y * y + z * z);
    }
    return rad2 > 0.f ? sqrtf(dmin2 / rad2) : INFINITY;
}

// (called by whole warps: the cover's measures are shared by shuffles)
template <typename Fn>
__device__ void adaptive32(const Off32 &O, const Reg32 &R, bool withX, int min_order, int lane, Fn &&fn) {
    struct Sq { float x0, x1, e0, e1; int depth; };
    Sq stack[kStack];
    int sp = 0;
    stack[sp++] = Sq{0.f, 1.f, 0.f, 1.f, 0};
    while (sp > 0) {
        const Sq q = stack[--sp];
        float lx, le;
        const float r = ratio32(O, R, q.x0, q.x1, q.e0, q.e1, withX, lane, lx, le);
        int n = order32r(r);
        if (n == 0 && q.depth < kMaxDepth && sp + 4 <= kStack) {
            const float xm = 0.5f * (q.x0 + q.x1), em = 0.5f * (q.e0 + q.e1);
            if (lx > 2.f * le) {
                stack[sp++] = Sq{q.x0, xm, q.e0, q.e1, q.depth + 1};
                stack[sp++] = Sq{xm, q.x1, q.e0, q.e1, q.depth + 1};
            } else if (le > 2.f * lx) {
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
        if (n == 0) n = 14;
        if (n < min_order) n = min_order;
        fn(q.x0, q.x1, q.e0, q.e1, n);
    }
}

// FP32 Gauss tables: nodes (1 + x)/2 and weights w/2 on [0, 1], order n at n(n-1)/2
struct Gauss32 {
    float t[kMaxRule * (kMaxRule + 1) / 2], w[kMaxRule * (kMaxRule + 1) / 2];
};

// one accepted square of a region, its points dealt to the lanes of a warp;
// each lane adds its part, times 1/4pi, to sa and sd.  On a box the map's
// line (dw) depends on the point's second index alone: lane j maps line j once
// and the points take its values by shuffles (the same values pos32 forms).
__device__ void square32_warp(const Off32 &O, const Row32 &Rw, const Reg32 &R, float x0, float x1, float e0, float e1,
                              int n, const Gauss32 &G, int lane, double &sa, double &sd) {
    const float *t = G.t + n * (n - 1) / 2, *w = G.w + n * (n - 1) / 2;
    const float hx = x1 - x0, he = e1 - e0;
    float la = 0.f, ld = 0.f;
    if (!R.tri && n <= 32) {
        const unsigned FULL = 0xffffffffu;
        float Bl[3] = {0.f, 0.f, 0.f}, dBl[3] = {0.f, 0.f, 0.f}, Jl = 0.f;
        if (lane < n) line32(O, fmaf(fmaf(he, t[lane], e0), R.db, R.b0), Bl, dBl, Jl);
        const float jac = R.da * R.db;
        for (int k0 = 0; k0 < n * n; k0 += 32) {
            const int k = k0 + lane;
            const bool ok = k < n * n;
            const int i = ok ? k / n : 0, j = ok ? k - (k / n) * n : 0;
            float Bg[3], dBg[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                Bg[d] = __shfl_sync(FULL, Bl[d], j);
                dBg[d] = __shfl_sync(FULL, dBl[d], j);
            }
            const float Jf = __shfl_sync(FULL, Jl, j);
            if (ok) {
                const float du = fmaf(fmaf(hx, t[i], x0), R.da, R.a0);
                const float o[3] = {fmaf(du, Bg[0], dBg[0]), fmaf(du, Bg[1], dBg[1]), fmaf(du, Bg[2], dBg[2])};
                const float J = (O.uc + du) * Jf;
                eval32(O, Rw, o, w[i] * w[j] * hx * he * jac * J, la, ld);
            }
        }
        sa += (double)la * (0.25 / kPi);
        sd += (double)ld * (0.25 / kPi);
        return;
    }
    for (int k = lane; k < n * n; k += 32) {
        const int i = k / n, j = k - i * n;
        float du, dw, jac, o[3], J;
        map32(R, fmaf(hx, t[i], x0), fmaf(he, t[j], e0), du, dw, jac);
        pos32(O, du, dw, o, J);
        eval32(O, Rw, o, w[i] * w[j] * hx * he * jac * J, la, ld);
    }
    sa += (double)la * (0.25 / kPi);
    sd += (double)ld * (0.25 / kPi);
}

// a whole far panel by one thread: the tensor rule of order n on the box
// du in [a0, a0 + da], dw in [b0, b0 + db] (offsets of the panel's parameter box
// from C: on a side-bounded sub-range C is not the box's midpoint in w), lines
// once each
__device__ void far_panel32(const Off32 &O, const Row32 &Rw, float a0, float da, float b0, float db, int n,
                            const Gauss32 &G, double &sa, double &sd) {
    const float *t = G.t + n * (n - 1) / 2, *w = G.w + n * (n - 1) / 2;
    float la = 0.f, ld = 0.f;
    for (int j = 0; j < n; ++j) {
        float Bg[3], dBg[3], Jf;
        line32(O, fmaf(db, t[j], b0), Bg, dBg, Jf);
        float li = 0.f, lj = 0.f;
        for (int i = 0; i < n; ++i) {
            const float du = fmaf(da, t[i], a0);
            const float o[3] = {fmaf(du, Bg[0], dBg[0]), fmaf(du, Bg[1], dBg[1]), fmaf(du, Bg[2], dBg[2])};
            eval32(O, Rw, o, w[i] * (O.uc + du), li, lj);
        }
        la += w[j] * Jf * li;
        ld += w[j] * Jf * lj;
    }
    const float jac = da * db;
    sa += (double)(la * jac) * (0.25 / kPi);
    sd += (double)(ld * jac) * (0.25 / kPi);
}

// self_regions on FP32 offsets from the collocation point (the panel centre C
// of the Off32 map), for the mixed-precision pass: the same quadrants, graded
// pieces and Duffy triangles, measured on pos32 (a side that maps to one point
// is recognised at 1e-5 of its distance, above FP32 rounding of the offsets).
template <typename Fn>
__device__ void self_regions32(const Off32 &O, const double *prm, Fn &&fn) {
    const double ucs[2] = {prm[0], prm[1]}, wcs[2] = {prm[2], prm[3]};
    auto len = [](const float *A, const float *B) {
        return sqrtf((A[0] - B[0]) * (A[0] - B[0]) + (A[1] - B[1]) * (A[1] - B[1]) + (A[2] - B[2]) * (A[2] - B[2]));
    };
    const float Z[3] = {0.f, 0.f, 0.f};
    float J;
#pragma unroll 1
    for (int qd = 0; qd < 4; ++qd) {
        const float Du = (float)(ucs[qd >> 1] - prm[4]), Dw = (float)(wcs[qd & 1] - prm[5]);
        if (Du == 0.f || Dw == 0.f) continue;
        float Pa[3], Pm[3], Pb[3];
        pos32(O, Du, 0.f, Pa, J);
        pos32(O, 0.f, 0.5f * Dw, Pm, J);
        pos32(O, 0.f, Dw, Pb, J);
        const float lu = len(Pa, Z), lw = len(Pm, Z) + len(Pb, Pm);
        int along = 0;
        float f0 = 1.f;
        if (lw > 2.f * lu) { along = 2; f0 = lu / lw; }
        else if (lu > 2.f * lw) { along = 1; f0 = lw / lu; }
        f0 = fmaxf(f0, 1.f / 1048576.f);
        float fa = 0.f, fb = f0;
        for (int k = 0;; ++k) {
            float a1 = Du, b1 = Dw, a0 = 0.f, b0 = 0.f;
            if (along == 1) { a0 = fa * Du; a1 = fb * Du; }
            if (along == 2) { b0 = fa * Dw; b1 = fb * Dw; }
            if (k == 0) {
                // Duffy triangles (C, (a1, 0), (a1, b1)) and (C, (a1, b1), (0, b1)), far
                // sides cut to the triangle's height (four pieces on a degenerate side)
                const float ta[2][2] = {{a1, 0.f}, {a1, b1}}, tb[2][2] = {{a1, b1}, {0.f, b1}};
#pragma unroll 1
                for (int t = 0; t < 2; ++t) {
                    float PA[3], PB[3];
                    pos32(O, ta[t][0], ta[t][1], PA, J);
                    pos32(O, tb[t][0], tb[t][1], PB, J);
                    const float ab[3] = {PB[0] - PA[0], PB[1] - PA[1], PB[2] - PA[2]};
                    const float as[3] = {-PA[0], -PA[1], -PA[2]};
                    const float cr[3] = {ab[1] * as[2] - ab[2] * as[1], ab[2] * as[0] - ab[0] * as[2],
                                         ab[0] * as[1] - ab[1] * as[0]};
                    const float L = sqrtf(ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2]);
                    const float h = sqrtf(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]) / fmaxf(L, 1e-30f);
                    int m = (int)fminf(64.f, fmaxf(1.f, ceilf(L / fmaxf(h, 1e-30f))));
                    if (L <= 1e-5f * sqrtf(as[0] * as[0] + as[1] * as[1] + as[2] * as[2])) m = 4;
                    for (int e = 0; e < m; ++e) {
                        const float Au = ta[t][0] + (tb[t][0] - ta[t][0]) * e / m;
                        const float Aw = ta[t][1] + (tb[t][1] - ta[t][1]) * e / m;
                        const float Bu = ta[t][0] + (tb[t][0] - ta[t][0]) * (e + 1) / m;
                        const float Bw = ta[t][1] + (tb[t][1] - ta[t][1]) * (e + 1) / m;
                        Reg32 R;
                        R.tri = true;
                        R.a0 = R.da = R.b0 = R.db = 0.f;
                        R.E1[0] = Au; R.E1[1] = Aw;
                        R.E2[0] = Bu - Au; R.E2[1] = Bw - Aw;
                        R.det = fabsf(R.E1[0] * R.E2[1] - R.E1[1] * R.E2[0]);
                        if (R.det > 0.f) fn(R, false, 10);
                    }
                }
            } else {
                Reg32 R;
                R.tri = false;
                R.a0 = fminf(a0, a1); R.da = fabsf(a1 - a0);
                R.b0 = fminf(b0, b1); R.db = fabsf(b1 - b0);
                R.E1[0] = R.E1[1] = R.E2[0] = R.E2[1] = R.det = 0.f;
                fn(R, true, 0);
            }
            if (along == 0 || fb >= 1.f) break;
            fa = fb;
            fb = fminf(1.f, 2.f * fb);
        }
    }
}

// The Gauss rule of order nq on one sub-square of a region, its points dealt
// to the lanes of a warp in turn (each lane sums its own points).
__device__ __forceinline__ void coop_gauss(const Ctx<double> &c, const Region &R, double x0, double x1, double e0,
                                           double e1, int nq, const double *__restrict__ glx,
                                           const double *__restrict__ glw, int lane, double &sa, double &sd) {
    const double *gx = glx + nq * (nq - 1) / 2, *gw = glw + nq * (nq - 1) / 2;
    const double hx = 0.5 * (x1 - x0), mx = 0.5 * (x0 + x1);
    const double he = 0.5 * (e1 - e0), me = 0.5 * (e0 + e1);
    for (int q = lane; q < nq * nq; q += 32) {
        const int qi = q / nq, qj = q - qi * nq;
        double u, v, jac;
        map_uv<double>(R, mx + hx * gx[qi], me + he * gx[qj], u, v, jac);
        eval_point<double>(c, u, v, gw[qi] * gw[qj] * hx * he * jac, sa, sd);
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

// SK: the second-kind system (a separate instance, so the first-kind code
// carries none of its branches).
// W32: the mixed-precision pass over wrapped patches (FP32 rules in offset
// form), a separate instance so that the FP64 code keeps its registers.
template <bool SK, bool W32>
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
    if (P.only_wrapped && f.kind != kWrapped) return;
    // a wrapped patch is a group of its own: its matrix rows and right side are
    // assembled together by the mode-2 pass, into its group matrix
    if (P.mode == 1 && f.kind == kWrapped) return;
    if (P.mode == 2 && P.A) Arow = P.A + P.gmat_off[P.group_of[p]] + (int64_t)i * n;
    const Piece *pcs = (f.kind == kWrapped) ? P.pieces + p * kMaxPieces : nullptr;
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
    if (P.mode == 1) c64.needD = false;
    if (P.mode == 2) c64.needA = (Arow != nullptr);
    // mixed precision on a wrapped patch (a matrix of its own): every panel by
    // FP32 rules in offset form (Off32), with FP32 adaptive covers
    const bool far32 = W32;   // (the W32 pass runs over wrapped patches only)
    __shared__ int near_list[1024];
    __shared__ int near_count;
    __shared__ double self_part[2][kAsmThreads / 32];
    __shared__ Gauss32 g32;
    __shared__ RowStatic32 rs32;
    Row32 rw;
    if (W32) {
        for (int k = threadIdx.x; k < kMaxRule * (kMaxRule + 1) / 2; k += blockDim.x) {
            g32.t[k] = (float)(0.5 + 0.5 * P.glx[k]);
            g32.w[k] = (float)(0.5 * P.glw[k]);
        }
        if (threadIdx.x == 0) row_static32(c64, f, pcs, rs32);
        row32_setup(c64, rw);
    }
    __shared__ double sk_grad[2];
    double e1[3] = {0.0, 0.0, 0.0}, e2[3] = {0.0, 0.0, 0.0};
    if (SK) {
        // normal at the collocation point and unit tangents along u and v there
        const double uc = P.panel_prm[6 * row + 4], vc = P.panel_prm[6 * row + 5];
        double Yc[3], nl[3], J;
        patch_point<double>(f.kind, f.R, uc, vc, Yc, nl, J);
        double su, cu, sv, cv;
        sincos(uc, &su, &cu);
        sincos(vc, &sv, &cv);
        if (f.kind == kDisk) { e1[0] = cv; e1[1] = sv; e1[2] = 0.0; }
        else { e1[0] = cu * cv; e1[1] = cu * sv; e1[2] = -su; }
        e2[0] = -sv; e2[1] = cv; e2[2] = 0.0;
        c64.sk = true;
        c64.needA = (P.mode != 2);
        c64.needD = (P.mode != 1);
        for (int d = 0; d < 3; ++d) c64.nx[d] = nl[d];
        if (threadIdx.x < 2) {
            // tangential derivative of the data by central differences, h = 1e-5 a
            const double h = 1e-5 * f.a;
            const double *e = threadIdx.x == 0 ? e1 : e2;
            double gp[3], gm[3];
            for (int d = 0; d < 3; ++d) {
                const double lp[3] = {X[0] + h * e[0], X[1] + h * e[1], X[2] + h * e[2]};
                const double lm[3] = {X[0] - h * e[0], X[1] - h * e[1], X[2] - h * e[2]};
                gp[d] = f.c[d] + lp[0] * f.t1[d] + lp[1] * f.t2[d] + lp[2] * f.n[d];
                gm[d] = f.c[d] + lm[0] * f.t1[d] + lm[1] * f.t2[d] + lm[2] * f.n[d];
            }
            sk_grad[threadIdx.x] = (dirichlet_eval<double>(P.dat, gp[0], gp[1], gp[2]) -
                                    dirichlet_eval<double>(P.dat, gm[0], gm[1], gm[2])) / (2.0 * h);
        }
    }
    if (threadIdx.x == 0) near_count = 0;
    __syncthreads();
    if (SK)
        for (int d = 0; d < 3; ++d) c64.ga[d] = sk_grad[0] * e1[d] + sk_grad[1] * e2[d];
    const double dsign = SK ? -1.0 : 1.0;   // second kind: A = 1/2 I - D
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double dsum = 0.0;
    // far panels (r >= 2): one thread each, separable Gauss rule.  The near
    // panels are listed in panel order (ballots and a prefix over the warps),
    // so that the warps sum their right-side parts in the same order on every
    // run.
    __shared__ int warp_near[kAsmThreads / 32];
    for (int j0 = 0; j0 < n; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        const bool mine = j < n && j != i;
        Off32 O;
        float r32 = 0.f;
        if (W32 && mine) {
            const PanelStatic32 &S = P.pstat[poff + j];
            off32_make(S, rs32, O);
            r32 = ratio_panel32(S, O);
        }
        const bool near = mine && (W32 ? r32 < 2.f : panel_ratio(c64, X, P.panel_aux + 4 * (poff + j)) < 2.0);
        const unsigned bal = __ballot_sync(0xffffffffu, near);
        if (lane == 0) warp_near[warp] = __popc(bal);
        __syncthreads();
        int base = near_count;
        for (int w = 0; w < warp; ++w) base += warp_near[w];
        if (near) near_list[base + __popc(bal & ((1u << lane) - 1u))] = j;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 0; w < kAsmThreads / 32; ++w) near_count += warp_near[w];
        __syncthreads();
        if (!mine || near) continue;
        const int64_t pj = poff + j;
        const double r = W32 ? (double)r32 : panel_ratio(c64, X, P.panel_aux + 4 * pj);
        const double *prm = P.panel_prm + 6 * pj;
        Region R;
        R.tri = false;
        R.p[0] = prm[0]; R.p[1] = prm[1] - prm[0]; R.p[2] = prm[2]; R.p[3] = prm[3] - prm[2];
        R.det = 0.0;
        double sa = 0.0, sd = 0.0;
        if (far32) {
            far_panel32(O, rw, (float)(prm[0] - prm[4]), (float)(prm[1] - prm[0]), (float)(prm[2] - prm[5]),
                        (float)(prm[3] - prm[2]), order32r((float)r), g32, sa, sd);
        } else {
            ctx_panel(c64, pcs, P.panel_piece[pj]);
            gauss_rect<double>(c64, R, 0.0, 1.0, 0.0, 1.0, order64(r), P.glx, P.glw, sa, sd);
        }
        if (Arow) Arow[j] = dsign * sa;
        dsum += sd;
    }
    // self panel: its Duffy triangles dealt to the warps in turn, the points of
    // each accepted sub-square to the lanes; sums in a fixed order
    {
        double sa = 0.0, sd = 0.0;
        int tri = 0;
        ctx_panel(c64, pcs, P.panel_piece[row]);
        auto region = [&](const Region &R, bool withX, int min_order) {
            if ((tri++ % (kAsmThreads / 32)) != warp) return;
            adaptive_squares<double>(c64, R, withX, min_order, [&](double x0, double x1, double e0, double e1, int nq) {
                coop_gauss(c64, R, x0, x1, e0, e1, nq, P.glx, P.glw, lane, sa, sd);
            });
        };
        if (far32) {
            // mixed precision: the graded regions, in offsets from the collocation
            // point (the panel centre), by the FP32 rules and covers
            const double *prm = P.panel_prm + 6 * row;
            Off32 O;
            off32_make(P.pstat[row], rs32, O);
            self_regions32(O, prm, [&](const Reg32 &Q, bool withX, int min_order) {
                if ((tri++ % (kAsmThreads / 32)) != warp) return;
                adaptive32(O, Q, withX, min_order, lane, [&](float x0, float x1, float e0, float e1, int n) {
                    square32_warp(O, rw, Q, x0, x1, e0, e1, n, g32, lane, sa, sd);
                });
            });
        } else if (f.kind == kWrapped) {
            self_regions(c64, P.panel_prm + 6 * row, region);
        } else {
            self_triangles(c64, P.panel_prm + 6 * row, [&](const Region &R) { region(R, false, 16); });
        }
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sd += __shfl_xor_sync(0xffffffffu, sd, o);
        }
        if (lane == 0) {
            self_part[0][warp] = sa;
            self_part[1][warp] = sd;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sd = 0.0;
        for (int w = 0; w < kAsmThreads / 32; ++w) {
            sa += self_part[0][w];
            sd += self_part[1][w];
        }
        if (Arow) Arow[i] = SK ? 0.5 - sa : sa;
        dsum += sd;
    }
    // near panels (r < 2): one warp each, adaptive cover, points over the lanes
    const int nn = near_count;
    for (int k = warp; k < nn; k += kAsmThreads / 32) {
        const int j = near_list[k];
        const double *prm = P.panel_prm + 6 * (poff + j);
        Region R;
        R.tri = false;
        R.p[0] = prm[0]; R.p[1] = prm[1] - prm[0]; R.p[2] = prm[2]; R.p[3] = prm[3] - prm[2];
        R.det = 0.0;
        double sa = 0.0, sd = 0.0;
        ctx_panel(c64, pcs, P.panel_piece[poff + j]);
        if (far32) {
            // mixed precision on a wrapped patch: the FP32 cover in offsets from the panel centre
            Off32 O;
            off32_make(P.pstat[poff + j], rs32, O);
            Reg32 Q;
            Q.tri = false;
            Q.a0 = (float)(prm[0] - prm[4]); Q.da = (float)(prm[1] - prm[0]);
            Q.b0 = (float)(prm[2] - prm[5]); Q.db = (float)(prm[3] - prm[2]);
            Q.E1[0] = Q.E1[1] = Q.E2[0] = Q.E2[1] = Q.det = 0.f;
            adaptive32(O, Q, true, 0, lane, [&](float x0, float x1, float e0, float e1, int n) {
                square32_warp(O, rw, Q, x0, x1, e0, e1, n, g32, lane, sa, sd);
            });
        } else {
            adaptive_squares<double>(c64, R, true, 0, [&](double x0, double x1, double e0, double e1, int nq) {
                coop_gauss(c64, R, x0, x1, e0, e1, nq, P.glx, P.glw, lane, sa, sd);
            });
        }
        for (int o = 16; o > 0; o >>= 1) {
            sa += __shfl_xor_sync(0xffffffffu, sa, o);
            sd += __shfl_xor_sync(0xffffffffu, sd, o);
        }
        if (lane == 0) {
            if (Arow) Arow[j] = dsign * sa;
            dsum += sd;
        }
    }
    if (P.mode == 1) return;
    // Gamma term: sum_k W_k P(x_i, y_k) (U_k - g(x_i)), FP64
    const int64_t goff = P.gamma_off[p];
    const int nk = (int)(P.gamma_off[p + 1] - goff);
    double gsum = 0.0;
    if (W32) {
        // mixed precision: FP32 terms W_k (U_k - g(x)) / |x - y_k|^3 from FP64
        // differences, summed per thread in FP32, times the row's
        // (a^2 - |x|^2) / (4 pi a)
        const double xx = X[0] * X[0] + X[1] * X[1] + X[2] * X[2];
        const float cp = (float)((f.a * f.a - xx) / (4.0 * kPi * f.a));
        float gs = 0.f;
        for (int k = threadIdx.x; k < nk; k += blockDim.x) {
            const int64_t gk = goff + k;
            const float dx = (float)(X[0] - P.gamma_loc[3 * gk]), dy = (float)(X[1] - P.gamma_loc[3 * gk + 1]),
                        dz = (float)(X[2] - P.gamma_loc[3 * gk + 2]);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            gs += (float)P.gamma_w[gk] * (float)(P.U[gk] - gx) / (r2 * sqrtf(r2));
        }
        gsum = (double)(gs * cp);
    }
    for (int k = threadIdx.x; k < nk && !W32; k += blockDim.x) {
        const int64_t gk = goff + k;
        const double Y[3] = {P.gamma_loc[3 * gk], P.gamma_loc[3 * gk + 1], P.gamma_loc[3 * gk + 2]};
        if (SK) {
            // second kind: sum_k W_k K(x_i, y_k) (U_k - l(y_k)), K = d2G/dn_x dn_y, n_y = Y / a
            const double ny[3] = {Y[0] / f.a, Y[1] / f.a, Y[2] / f.a};
            const double l = gx + c64.ga[0] * (Y[0] - X[0]) + c64.ga[1] * (Y[1] - X[1]) + c64.ga[2] * (Y[2] - X[2]);
            gsum += P.gamma_w[gk] * green_ball_dnn(f.a, X, c64.nx, Y, ny) * (P.U[gk] - l);
        } else {
            gsum += P.gamma_w[gk] * poisson_ball<double>(f.a, X, Y) * (P.U[gk] - gx);
        }
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
        P.b[row] = SK ? -s0 - s1 : s0 - s1;
    }
}

// ---------------------------------------------------------------------------
// Mixed precision right sides (one weight row per collocation point of each
// shape group, then one product per group).

// Lagrange basis on the 8 Gauss-Legendre points of the unit interval
struct Basis8 {
    double s[kSampleN], w[kSampleN], inv[kSampleN];
};

__device__ __forceinline__ void basis_all(const Basis8 &B, double t, double *l) {
    double pre[kSampleN], acc = 1.0;
#pragma unroll
    for (int m = 0; m < kSampleN; ++m) {
        pre[m] = acc;
        acc *= (t - B.s[m]);
    }
    double suf = 1.0;
#pragma unroll
    for (int m = kSampleN - 1; m >= 0; --m) {
        l[m] = pre[m] * suf * B.inv[m];
        suf *= (t - B.s[m]);
    }
}

struct WtDev {
    const PatchFrame *frames;
    const int64_t *panel_off, *gamma_off, *wrows_off, *wrep, *kcols, *gw_off;
    int64_t n_wgroups;
    const double *panel_loc, *panel_prm, *panel_aux, *gamma_loc, *gamma_w;
    float *gw;
    const double *glx, *glw;
};

// Row `grow` of the weight groups: its group, local row, representative patch
// and weight row.
struct WtRow {
    int64_t grp, p, poff;
    int i, n, m;
    int64_t dcols, kc;
    float *W;
    double X[3];
};

__device__ __forceinline__ WtRow wt_row(const WtDev &P, int64_t grow) {
    WtRow r;
    r.grp = find_group(P.wrows_off, P.n_wgroups, grow);
    r.i = (int)(grow - P.wrows_off[r.grp]);
    r.p = P.wrep[r.grp];
    r.n = (int)(P.wrows_off[r.grp + 1] - P.wrows_off[r.grp]);
    r.kc = P.kcols[r.grp];
    const int64_t goff = P.gamma_off[r.p];
    r.m = (int)(P.gamma_off[r.p + 1] - goff);
    r.dcols = r.kc - r.m;
    r.W = P.gw + P.gw_off[r.grp] + (int64_t)r.i * r.kc;
    r.poff = P.panel_off[r.p];
    const int64_t row = r.poff + r.i;
    for (int d = 0; d < 3; ++d) r.X[d] = P.panel_loc[3 * row + d];
    return r;
}

__device__ __forceinline__ void basis8_init(Basis8 &B, const double *glx, const double *glw) {
    const double *gx = glx + kSampleN * (kSampleN - 1) / 2, *gw = glw + kSampleN * (kSampleN - 1) / 2;
    for (int a = 0; a < kSampleN; ++a) {
        B.s[a] = 0.5 * (1.0 + gx[a]);
        B.w[a] = 0.5 * gw[a];
    }
    for (int a = 0; a < kSampleN; ++a) {
        double d = 1.0;
        for (int q = 0; q < kSampleN; ++q)
            if (q != a) d *= (B.s[a] - B.s[q]);
        B.inv[a] = 1.0 / d;
    }
}

// Double-layer weights of the far panels (r >= 5, not the row's own), one
// thread per (row, panel, a): the 8 x 8 rule itself (the interpolatory rule on
// its own points), so w_(a,b) = w_a w_b |box| J dG/dn_y at point (a, b).
// Grid (rows, task blocks).  FP64, stored FP32.
__global__ void __launch_bounds__(kWtThreads) rhs_far_weights_kernel(WtDev P) {
    const WtRow r = wt_row(P, blockIdx.x);
    const int t = blockIdx.y * blockDim.x + threadIdx.x;
    __shared__ Basis8 B;
    if (threadIdx.x == 0) basis8_init(B, P.glx, P.glw);
    __syncthreads();
    if (r.kc == 0 || r.dcols == 0 || t >= r.n * kSampleN) return;   // (no columns: a wrapped patch's row)
    const int j = t / kSampleN, a = t - j * kSampleN;
    if (j == r.i) return;
    const PatchFrame f = P.frames[r.p];
    Ctx<double> c;
    make_ctx<double>(c, f, r.X, 0.0, nullptr);
    const int64_t pj = r.poff + j;
    if (panel_ratio(c, r.X, P.panel_aux + 4 * pj) < kFarRatio) return;   // near: rhs_near_weights_kernel
    const double *prm = P.panel_prm + 6 * pj;
    const double u0 = prm[0], du = prm[1] - prm[0], v0 = prm[2], dv = prm[3] - prm[2];
    const double ua = u0 + B.s[a] * du;
    float *dst = r.W + (int64_t)j * kSamplesPerPanel + a * kSampleN;
#pragma unroll
    for (int b = 0; b < kSampleN; ++b) {
        double Y[3], nl[3], J;
        patch_point<double>(f.kind, f.R, ua, v0 + B.s[b] * dv, Y, nl, J);
        dst[b] = (float)(B.w[a] * B.w[b] * du * dv * J * green_ball_dny<double>(c.a, c.X, c.xn, Y, nl));
    }
}

constexpr int kNearWarps = 8;

// Warp-cooperative product rule over one accepted sub-square: the lanes take
// its points in turn; each point's k = weight * J * dG/dn_y times the 8 basis
// values in u, and the 8 basis values in v, go through shared memory, and lane
// l accumulates the weights (a, b) = (l / 4, 2 (l % 4) + {0, 1}).  Every point
// is evaluated once for all 64 weights; the summation order is fixed.
struct ProdBuf {
    double ku[32][kSampleN], lv[32][kSampleN];
};

__device__ __forceinline__ void coop_square(const Ctx<double> &c, const PatchFrame &f, const Basis8 &B,
                                            const Region &R, double u0, double du, double v0, double dv,
                                            double x0, double x1, double e0, double e1, int nq, const double *glx,
                                            const double *glw, ProdBuf &pb, int lane, double &acc0, double &acc1) {
    const double *gx = glx + nq * (nq - 1) / 2, *gw = glw + nq * (nq - 1) / 2;
    const double hx = 0.5 * (x1 - x0), mx = 0.5 * (x0 + x1);
    const double he = 0.5 * (e1 - e0), me = 0.5 * (e0 + e1);
    const int npts = nq * nq;
    const int a = lane >> 2, b0 = (lane & 3) * 2;
    for (int base = 0; base < npts; base += 32) {
        const int q = base + lane;
        if (q < npts) {
            const int qi = q / nq, qj = q - qi * nq;
            double u, v, jac, Y[3], nl[3], J;
            map_uv<double>(R, mx + hx * gx[qi], me + he * gx[qj], u, v, jac);
            patch_point<double>(f.kind, f.R, u, v, Y, nl, J);
            const double k = gw[qi] * gw[qj] * hx * he * jac * J * green_ball_dny<double>(c.a, c.X, c.xn, Y, nl);
            double lu[kSampleN];
            basis_all(B, (u - u0) / du, lu);
            basis_all(B, (v - v0) / dv, pb.lv[lane]);
#pragma unroll
            for (int m = 0; m < kSampleN; ++m) pb.ku[lane][m] = k * lu[m];
        } else {
#pragma unroll
            for (int m = 0; m < kSampleN; ++m) {
                pb.ku[lane][m] = 0.0;
                pb.lv[lane][m] = 0.0;
            }
        }
        __syncwarp();
        const int cnt = min(32, npts - base);
        for (int s = 0; s < cnt; ++s) {
            const double ka = pb.ku[s][a];
            acc0 = fma(ka, pb.lv[s][b0], acc0);
            acc1 = fma(ka, pb.lv[s][b0 + 1], acc1);
        }
        __syncwarp();
    }
}

// Double-layer weights of the row's own panel and of its near panels (r < 5),
// one CTA of 8 warps per row.  Own panel: the Duffy triangles (adaptive cover,
// order >= 12) are dealt to the warps in turn and the warps' sums added in warp
// order; near panels: one warp per panel, adaptive cover with order >= 8.
__global__ void __launch_bounds__(32 * kNearWarps) rhs_near_weights_kernel(WtDev P) {
    const WtRow r = wt_row(P, blockIdx.x);
    __shared__ Basis8 B;
    __shared__ ProdBuf pbuf[kNearWarps];
    __shared__ double part[kNearWarps][kSamplesPerPanel];
    __shared__ int near_list[1024];
    __shared__ int near_count;
    if (threadIdx.x == 0) {
        basis8_init(B, P.glx, P.glw);
        near_count = 0;
    }
    __syncthreads();
    if (r.kc == 0 || r.dcols == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PatchFrame f = P.frames[r.p];
    Ctx<double> c;
    make_ctx<double>(c, f, r.X, 0.0, nullptr);
    // near panels of this row: the row's CTAs (gridDim.y) take the panels j with
    // j mod gridDim.y = blockIdx.y; the own panel is the first CTA's
    for (int j = threadIdx.x; j < r.n; j += blockDim.x)
        if (j != r.i && (j % (int)gridDim.y) == (int)blockIdx.y &&
            panel_ratio(c, r.X, P.panel_aux + 4 * (r.poff + j)) < kFarRatio)
            near_list[atomicAdd(&near_count, 1)] = j;
    // own panel
    if (blockIdx.y == 0) {
        const double *prm = P.panel_prm + 6 * (r.poff + r.i);
        const double u0 = prm[0], du = prm[1] - prm[0], v0 = prm[2], dv = prm[3] - prm[2];
        double acc0 = 0.0, acc1 = 0.0;
        int tri = 0;
        self_triangles(c, prm, [&](const Region &R) {
            if ((tri++ % kNearWarps) != warp) return;
            adaptive_squares<double>(c, R, false, kSelfOrderW, [&](double x0, double x1, double e0, double e1, int nq) {
                coop_square(c, f, B, R, u0, du, v0, dv, x0, x1, e0, e1, nq, P.glx, P.glw, pbuf[warp], lane, acc0,
                            acc1);
            });
        });
        const int o = (lane >> 2) * kSampleN + (lane & 3) * 2;
        part[warp][o] = acc0;
        part[warp][o + 1] = acc1;
    }
    __syncthreads();
    if (blockIdx.y == 0 && threadIdx.x < kSamplesPerPanel) {
        double t = 0.0;
        for (int w = 0; w < kNearWarps; ++w) t += part[w][threadIdx.x];
        r.W[(int64_t)r.i * kSamplesPerPanel + threadIdx.x] = (float)t;
    }
    // near panels, one warp each
    const int nn = near_count;
    for (int k = warp; k < nn; k += kNearWarps) {
        const int j = near_list[k];
        const double *prm = P.panel_prm + 6 * (r.poff + j);
        const double u0 = prm[0], du = prm[1] - prm[0], v0 = prm[2], dv = prm[3] - prm[2];
        Region R;
        R.tri = false;
        R.p[0] = u0; R.p[1] = du; R.p[2] = v0; R.p[3] = dv;
        R.det = 0.0;
        double acc0 = 0.0, acc1 = 0.0;
        adaptive_squares<double>(c, R, true, kSampleN, [&](double x0, double x1, double e0, double e1, int nq) {
            coop_square(c, f, B, R, u0, du, v0, dv, x0, x1, e0, e1, nq, P.glx, P.glw, pbuf[warp], lane, acc0, acc1);
        });
        float *dst = r.W + (int64_t)j * kSamplesPerPanel + (lane >> 2) * kSampleN + (lane & 3) * 2;
        dst[0] = (float)acc0;
        dst[1] = (float)acc1;
    }
}

// Walk-term weights -W_k P(x_i, y_k): grid (rows, node blocks).
__global__ void __launch_bounds__(kWtThreads) rhs_walk_weights_kernel(WtDev P) {
    const WtRow r = wt_row(P, blockIdx.x);
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    if (r.kc == 0 || k >= r.m) return;   // no columns: a wrapped patch's row (its right side is assembled directly)
    const double a = P.frames[r.p].a;
    const int64_t gk = P.gamma_off[r.p] + k;
    const double Y[3] = {P.gamma_loc[3 * gk], P.gamma_loc[3 * gk + 1], P.gamma_loc[3 * gk + 2]};
    r.W[r.dcols + k] = (float)(-P.gamma_w[gk] * poisson_ball<double>(a, r.X, Y));
}

// Per-patch sample vectors: the data at the 8 x 8 Gauss points of every panel
// (FP32 evaluation) and the walk estimates, each minus c = g at the first
// collocation point, stored FP32.  One thread per sample.
// Per-patch sample vectors: the data at the 8 x 8 Gauss points of every panel
// and the walk estimates, less c = g at the patch's first collocation point.
// The members of a weight group are congruent, so a sample's point in the patch
// frame is the same for all of them: a thread places its sample once (FP64
// trigonometry) and then, for a chunk of the group's patches, only rotates it
// into each patch's frame and evaluates the data (grid: samples x member chunks
// x weight groups).  The values are those of placing it per patch, bit for bit.
__global__ void rhs_samples_kernel(DData dat, const int64_t *__restrict__ wrep, const int64_t *__restrict__ mem_off,
                                   const int64_t *__restrict__ members, int chunk, int64_t gbase,
                                   const int64_t *__restrict__ vec_off, const int64_t *__restrict__ panel_off,
                                   const int64_t *__restrict__ gamma_off, const PatchFrame *__restrict__ frames,
                                   const double *__restrict__ panel_prm, const double *__restrict__ panel_g,
                                   const double *__restrict__ U, const double *__restrict__ glx,
                                   float *__restrict__ vec) {
    const int64_t grp = gbase + blockIdx.z;
    const int64_t rep = wrep[grp];
    const int64_t kc = vec_off[rep + 1] - vec_off[rep];
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= kc) return;
    const int64_t m = gamma_off[rep + 1] - gamma_off[rep];
    const int64_t dcols = kc - m;
    const int64_t k0 = mem_off[grp] + (int64_t)blockIdx.y * chunk;
    const int64_t k1 = min(mem_off[grp + 1], k0 + chunk);
    if (k0 >= k1) return;
    if (q < dcols) {
        const int64_t j = q / kSamplesPerPanel;
        const int a = (int)(q - j * kSamplesPerPanel) / kSampleN, b = (int)(q % kSampleN);
        const double *gx = glx + kSampleN * (kSampleN - 1) / 2;
        const double *prm = panel_prm + 6 * (panel_off[rep] + j);
        const double u = prm[0] + 0.5 * (1.0 + gx[a]) * (prm[1] - prm[0]);
        const double v = prm[2] + 0.5 * (1.0 + gx[b]) * (prm[3] - prm[2]);
        const PatchFrame &fr = frames[rep];
        double Y[3], nl[3], J;
        patch_point<double>(fr.kind, fr.R, u, v, Y, nl, J);
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t p = members[k];
            const PatchFrame &f = frames[p];
            const double y0 = f.c[0] + Y[0] * f.t1[0] + Y[1] * f.t2[0] + Y[2] * f.n[0];
            const double y1 = f.c[1] + Y[0] * f.t1[1] + Y[1] * f.t2[1] + Y[2] * f.n[1];
            const double y2 = f.c[2] + Y[0] * f.t1[2] + Y[1] * f.t2[2] + Y[2] * f.n[2];
            const double val = (double)dirichlet_eval<float>(dat, (float)y0, (float)y1, (float)y2) -
                               panel_g[panel_off[p]];
            vec[vec_off[p] + q] = (float)val;
        }
    } else {
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t p = members[k];
            vec[vec_off[p] + q] = (float)(U[gamma_off[p] + (q - dcols)] - panel_g[panel_off[p]]);
        }
    }
}

constexpr int kGemmM = 32, kGemmK = 32, kGemmThreads = 256;

struct RhsDev {
    const PatchFrame *frames;
    const int64_t *panel_off, *wrows_off, *kcols, *gw_off, *vec_off, *members, *mem_off, *tile_off;
    int64_t n_wgroups;
    int row_tiles;
    const float *gw, *vec;
    const double *panel_g;
    double *b;
};

// b = W s - (g(x_i) - c) rowsum(W) for a tile of 32 rows x 32 patches of one
// weight group.  FP32 products summed over each k-tile of 32, the tile sums added in
// FP64; every b entry sums in the same order whatever the batch holds.
__global__ void __launch_bounds__(kGemmThreads) rhs_product_kernel(RhsDev P) {
    const int64_t tile = blockIdx.x / P.row_tiles;
    const int rt = (int)(blockIdx.x - tile * P.row_tiles);
    const int64_t grp = find_group(P.tile_off, P.n_wgroups, tile);
    const int n = (int)(P.wrows_off[grp + 1] - P.wrows_off[grp]);
    const int row0 = rt * kGemmM;
    if (row0 >= n) return;
    const int64_t kc = P.kcols[grp];
    if (kc == 0) return;   // a wrapped patch's group: its right side is assembled directly
    const float *W = P.gw + P.gw_off[grp];
    const int64_t m0 = P.mem_off[grp] + (tile - P.tile_off[grp]) * kRhsTileN;
    const int mcount = (int)min((int64_t)kRhsTileN, P.mem_off[grp + 1] - m0);
    __shared__ float Ws[kGemmK][kGemmM + 1];
    __shared__ float Vs[kGemmK][kRhsTileN + 1];
    __shared__ int64_t vbase[kRhsTileN];
    if (threadIdx.x < kRhsTileN)
        vbase[threadIdx.x] = (int)threadIdx.x < mcount ? P.vec_off[P.members[m0 + threadIdx.x]] : -1;
    __syncthreads();
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    double rsum[2] = {0.0, 0.0};   // row sums of W, in the same summation order
    for (int64_t k0 = 0; k0 < kc; k0 += kGemmK) {
#pragma unroll
        for (int e = 0; e < (kGemmM * kGemmK) / kGemmThreads; ++e) {
            const int idx = threadIdx.x + kGemmThreads * e;
            const int r = idx >> 5, kk = idx & 31;
            const int64_t k = k0 + kk;
            Ws[kk][r] = (row0 + r < n && k < kc) ? W[(int64_t)(row0 + r) * kc + k] : 0.f;
            Vs[kk][r] = (vbase[r] >= 0 && k < kc) ? P.vec[vbase[r] + k] : 0.f;
        }
        __syncthreads();
        float s00 = 0.f, s01 = 0.f, s10 = 0.f, s11 = 0.f, r0 = 0.f, r1 = 0.f;
#pragma unroll
        for (int kk = 0; kk < kGemmK; ++kk) {
            const float a0 = Ws[kk][2 * ty], a1 = Ws[kk][2 * ty + 1];
            const float b0 = Vs[kk][2 * tx], b1 = Vs[kk][2 * tx + 1];
            s00 = fmaf(a0, b0, s00);
            s01 = fmaf(a0, b1, s01);
            s10 = fmaf(a1, b0, s10);
            s11 = fmaf(a1, b1, s11);
            r0 += a0;
            r1 += a1;
        }
        acc[0][0] += (double)s00;
        acc[0][1] += (double)s01;
        acc[1][0] += (double)s10;
        acc[1][1] += (double)s11;
        rsum[0] += (double)r0;
        rsum[1] += (double)r1;
        __syncthreads();
    }
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            const int row = row0 + 2 * ty + rr, col = 2 * tx + cc;
            if (row >= n || col >= mcount) continue;
            const int64_t p = P.members[m0 + col];
            const int64_t off = P.panel_off[p];
            P.b[off + row] = (P.frames[p].status == DTN_OK)
                                 ? acc[rr][cc] - (P.panel_g[off + row] - P.panel_g[off]) * rsum[rr]
                                 : 0.0;
        }
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
                            const double *U, double *A, double *b, cudaStream_t s, int sk, int only_wrapped,
                            void *pstat) {
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
    P.sk = sk;
    P.only_wrapped = only_wrapped;
    P.group_of = D.group_of;
    P.pstat = (const PanelStatic32 *)pstat;
    P.glx = gl_x_dev();
    P.glw = gl_w_dev();
    P.pieces = D.pieces;
    P.panel_piece = g->ws.panel_piece.as<int32_t>();
    const dim3 grid((unsigned)rows);
    if (sk) assemble_kernel<true, false><<<grid, kAsmThreads, 0, s>>>(P);
    else if (mode == 2 && only_wrapped && prec == DTN_PREC_MIXED) {
        if (!pstat) return cudaErrorInvalidValue;
        wrapped_static_kernel<<<(unsigned)((L.panels_total + 255) / 256), 256, 0, s>>>(
            L.n_patches, L.panels_total, D.panel_off, D.frames, D.pieces, P.panel_piece, panel_prm, panel_loc,
            panel_aux, (PanelStatic32 *)pstat);
        assemble_kernel<false, true><<<(unsigned)rows, kAsmThreads, 0, s>>>(P);
    }
    else assemble_kernel<false, false><<<grid, kAsmThreads, 0, s>>>(P);
    return cudaGetLastError();
}

size_t wrapped_static_bytes(int64_t panels) { return (size_t)panels * sizeof(PanelStatic32); }

cudaError_t launch_rhs_shared(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                              const double *panel_loc, const double *panel_prm, const double *panel_aux,
                              const double *panel_g, const double *gamma_loc, const double *gamma_w,
                              const double *U, float *gw, float *vec, double *b, cudaStream_t s) {
    if (L.wrows_total == 0) return cudaSuccess;
    WtDev Wd;
    Wd.frames = D.frames;
    Wd.panel_off = D.panel_off;
    Wd.gamma_off = D.gamma_off;
    Wd.wrows_off = D.wrows_off;
    Wd.wrep = D.wrep;
    Wd.kcols = D.kcols;
    Wd.gw_off = D.gw_off;
    Wd.n_wgroups = L.n_wgroups;
    Wd.panel_loc = panel_loc;
    Wd.panel_prm = panel_prm;
    Wd.panel_aux = panel_aux;
    Wd.gamma_loc = gamma_loc;
    Wd.gamma_w = gamma_w;
    Wd.gw = gw;
    Wd.glx = gl_x_dev();
    Wd.glw = gl_w_dev();
    const unsigned rows = (unsigned)L.wrows_total;
    if (g->dg.kind == kBall || g->dg.kind == kBallExterior) {
        const unsigned tb = (unsigned)((L.max_wgroup_rows * kSampleN + kWtThreads - 1) / kWtThreads);
        rhs_far_weights_kernel<<<dim3(rows, tb), kWtThreads, 0, s>>>(Wd);
        // four CTAs per row: the FP64 quadrature of one weight group's rows spread
        // over every SM (a single group has as few as 128 rows)
        rhs_near_weights_kernel<<<dim3(rows, 4), 32 * kNearWarps, 0, s>>>(Wd);
    }
    rhs_walk_weights_kernel<<<dim3(rows, (unsigned)((L.max_nodes + kWtThreads - 1) / kWtThreads)), kWtThreads, 0, s>>>(Wd);
    const int T = 256;
    // (a batch of wrapped patches only has weight rows without columns: their
    // right sides are assembled directly, and there are no samples)
    if (L.vec_total > 0) {
        int64_t max_kc = 0, max_mem = 0;
        for (int64_t k = 0; k < L.n_wgroups; ++k) {
            max_kc = std::max(max_kc, L.kcols[k]);
            max_mem = std::max(max_mem, L.mem_off[k + 1] - L.mem_off[k]);
        }
        const int chunk = (int)std::max<int64_t>(16, (max_mem + 65534) / 65535);
        for (int64_t g0 = 0; g0 < L.n_wgroups; g0 += 65535) {   // grid z holds at most 65535 groups
            const dim3 grid((unsigned)((max_kc + T - 1) / T), (unsigned)((max_mem + chunk - 1) / chunk),
                            (unsigned)std::min<int64_t>(65535, L.n_wgroups - g0));
            rhs_samples_kernel<<<grid, T, 0, s>>>(g->dd, D.wrep, D.mem_off, D.members, chunk, g0, D.vec_off,
                                                  D.panel_off, D.gamma_off, D.frames, panel_prm, panel_g, U, Wd.glx,
                                                  vec);
        }
    }
    RhsDev R;
    R.frames = D.frames;
    R.panel_off = D.panel_off;
    R.wrows_off = D.wrows_off;
    R.kcols = D.kcols;
    R.gw_off = D.gw_off;
    R.vec_off = D.vec_off;
    R.members = D.members;
    R.mem_off = D.mem_off;
    R.tile_off = D.tile_off;
    R.n_wgroups = L.n_wgroups;
    R.row_tiles = (L.max_wgroup_rows + kGemmM - 1) / kGemmM;
    R.gw = gw;
    R.vec = vec;
    R.panel_g = panel_g;
    R.b = b;
    rhs_product_kernel<<<(unsigned)(L.tiles_total * R.row_tiles), kGemmThreads, 0, s>>>(R);
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
