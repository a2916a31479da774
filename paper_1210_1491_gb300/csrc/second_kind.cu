// second_kind.cu -- Neumann data of flat (disk) patches by the second-kind local
// BIE (Eq. bw55-bw59).  For x and y in the plane of the patch, which passes
// through the ball centre, dG/dn_x vanishes (X.n = Y.n = (X - Y).n = 0 in both
// terms of the whole-sphere Green's function), so the double-layer operator D
// is zero and Eq. bw55 reads q = 2b: no linear system.  b is regularised with
// the constant solution (u = 1, q = 0), so at each collocation point
//
//   q_i = - 2 sum_k W_k K(x_i, y_k) (U_k - g(x_i)) - 2 p.v. int_S K(x_i, y) (g(y) - g(x_i)) ds_y,
//
// K = d2G/dn_x dn_y, on S equal to (1/4pi)(1/rho^3 - a^3 Q^-3/2).  In the S
// integral the linear Taylor term t = grad g(x_i).(y - x_i) is taken out: its
// free-space part is exact (p.v. int_S (y - x)/rho^3 ds = - oint of nu / rho over
// the rim, the divergence theorem in the plane), the rest goes through polar
// Gauss rules about x_i.  One CTA per collocation row, FP64, fixed summation
// order.
#include <cmath>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kSkThreads = 128;

struct SkDev {
    const PatchFrame *frames;
    const int64_t *panel_off, *gamma_off;
    int64_t n_patches;
    const double *panel_loc, *panel_g, *gamma_loc, *gamma_w, *U;
    const double *panel_prm;
    DData dat;
    int ng2;
    const double *glx, *glw;
    double *q, *b;
    int32_t *iters, *status;
    double *resid;
};

__device__ __forceinline__ void to_global(const PatchFrame &f, const double *L, double *y) {
    for (int d = 0; d < 3; ++d) y[d] = f.c[d] + L[0] * f.t1[d] + L[1] * f.t2[d] + L[2] * f.n[d];
}

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kSkThreads / 32; ++w) t += red[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kSkThreads) second_kind_kernel(SkDev P) {
    const int64_t row = blockIdx.x;
    const int64_t p = find_group(P.panel_off, P.n_patches, row);
    const int64_t i = row - P.panel_off[p];
    const PatchFrame f = P.frames[p];
    __shared__ double red[kSkThreads / 32];
    __shared__ double grad[2];
    if (i == 0 && threadIdx.x == 0) {
        if (P.iters) P.iters[p] = 0;
        if (P.resid) P.resid[p] = 0.0;
        if (P.status) P.status[p] = f.status;
    }
    if (f.status != DTN_OK) {
        if (threadIdx.x == 0) {
            P.q[row] = 0.0;
            if (P.b) P.b[row] = 0.0;
        }
        return;
    }
    const double a = f.a;
    const double X[3] = {P.panel_loc[3 * row], P.panel_loc[3 * row + 1], 0.0};
    const double gxi = P.panel_g[row];
    const double ez[3] = {0.0, 0.0, 1.0};
    if (threadIdx.x < 2) {
        // tangential gradient of the data by central differences, h = 1e-5 a
        const double h = 1e-5 * a;
        double Lp[3] = {X[0], X[1], 0.0}, Lm[3] = {X[0], X[1], 0.0}, yp[3], ym[3];
        Lp[threadIdx.x] += h;
        Lm[threadIdx.x] -= h;
        to_global(f, Lp, yp);
        to_global(f, Lm, ym);
        grad[threadIdx.x] = (dirichlet_eval<double>(P.dat, yp[0], yp[1], yp[2]) -
                             dirichlet_eval<double>(P.dat, ym[0], ym[1], ym[2])) / (2.0 * h);
    }
    // hemisphere term
    const int64_t goff = P.gamma_off[p];
    const int m = (int)(P.gamma_off[p + 1] - goff);
    double sg = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int64_t gk = goff + k;
        const double Y[3] = {P.gamma_loc[3 * gk], P.gamma_loc[3 * gk + 1], P.gamma_loc[3 * gk + 2]};
        const double ny[3] = {Y[0] / a, Y[1] / a, Y[2] / a};
        sg += P.gamma_w[gk] * green_ball_dnn(a, X, ez, Y, ny) * (P.U[gk] - gxi);
    }
    __syncthreads();
    const double g0 = grad[0], g1 = grad[1];
    const int n2 = P.ng2;
    const double *gx = P.glx + n2 * (n2 - 1) / 2, *gw = P.glw + n2 * (n2 - 1) / 2;
    const double xx = X[0] * X[0] + X[1] * X[1];
    double ss = 0.0;
    // polar rules about x_i: angle j, radius l in [0, rho_max(angle)]
    for (int k = threadIdx.x; k < n2 * n2; k += blockDim.x) {
        const int j = k / n2, l = k - j * n2;
        double se, ce;
        sincos(kPi * (gx[j] + 1.0), &se, &ce);
        const double xe = X[0] * ce + X[1] * se;
        const double rmax = -xe + sqrt(xe * xe + a * a - xx);
        const double rho = 0.5 * rmax * (gx[l] + 1.0), w = kPi * gw[j] * 0.5 * rmax * gw[l];
        const double L[3] = {X[0] + rho * ce, X[1] + rho * se, 0.0};
        double y[3];
        to_global(f, L, y);
        const double t = rho * (g0 * ce + g1 * se);
        const double YY = L[0] * L[0] + L[1] * L[1], XY = X[0] * L[0] + X[1] * L[1];
        const double Q = xx * YY - 2.0 * a * a * XY + a * a * a * a;
        const double img = a * a * a / (Q * sqrt(Q));
        ss += w * rho * ((dirichlet_eval<double>(P.dat, y[0], y[1], y[2]) - gxi - t) * (1.0 / (rho * rho * rho) - img) -
                         t * img);
    }
    // p.v. int_S (y - x)/rho^3 ds = - oint nu / rho dl over the rim
    for (int j = threadIdx.x; j < n2; j += blockDim.x) {
        double sn, cn;
        sincos(kPi * (gx[j] + 1.0), &sn, &cn);
        const double w = kPi * gw[j] * a;
        const double dy0 = a * cn - X[0], dy1 = a * sn - X[1];
        const double rr = sqrt(dy0 * dy0 + dy1 * dy1);
        ss -= w * (g0 * cn + g1 * sn) / rr;
    }
    sg = block_sum(sg, red);
    ss = block_sum(ss, red);
    if (threadIdx.x == 0) {
        const double bb = -sg - ss / (4.0 * kPi);
        P.q[row] = 2.0 * bb;
        if (P.b) P.b[row] = bb;
    }
}

// Right side of the second-kind system on a cap patch (R27), one CTA per row:
//   b_i = - sum_k W_k K(x_i, y_k) (U_k - l_i(y_k))
//         - int_S [ K(x_i, y) (g(y) - l_i(y)) + dG/dn_x(x_i, y) a_i.n_y ] ds_y
// with the S integral in geodesic polar coordinates (sigma, phi) about x_i on the
// sphere of the cap (centre o = (0, 0, -R) in the patch frame, signed R), the
// cap's edge at sigma_max(phi) from spherical trigonometry, ring_order Gauss
// points in each variable; the integrand is bounded there (O(1/r) against the
// Jacobian R^2 sin sigma).  FP64, fixed summation order.
__global__ void __launch_bounds__(kSkThreads) second_kind_cap_rhs_kernel(SkDev P) {
    const int64_t row = blockIdx.x;
    const int64_t p = find_group(P.panel_off, P.n_patches, row);
    const PatchFrame f = P.frames[p];
    __shared__ double red[kSkThreads / 32];
    __shared__ double grad[2];
    if (f.status != DTN_OK) {
        if (threadIdx.x == 0) P.b[row] = 0.0;
        return;
    }
    const double a = f.a, R = f.R;
    const double X[3] = {P.panel_loc[3 * row], P.panel_loc[3 * row + 1], P.panel_loc[3 * row + 2]};
    const double gxi = P.panel_g[row];
    const double uc = P.panel_prm[6 * row + 4], vc = P.panel_prm[6 * row + 5];
    double su, cu, sv, cv;
    sincos(uc, &su, &cu);
    sincos(vc, &sv, &cv);
    const double nx[3] = {su * cv, su * sv, cu};          // outward normal at x_i = (X - o)/R
    const double e1[3] = {cu * cv, cu * sv, -su}, e2[3] = {-sv, cv, 0.0};
    if (threadIdx.x < 2) {
        // tangential derivative of the data by central differences, h = 1e-5 a
        const double h = 1e-5 * a;
        const double *e = threadIdx.x == 0 ? e1 : e2;
        double Lp[3], Lm[3], yp[3], ym[3];
        for (int d = 0; d < 3; ++d) { Lp[d] = X[d] + h * e[d]; Lm[d] = X[d] - h * e[d]; }
        to_global(f, Lp, yp);
        to_global(f, Lm, ym);
        grad[threadIdx.x] = (dirichlet_eval<double>(P.dat, yp[0], yp[1], yp[2]) -
                             dirichlet_eval<double>(P.dat, ym[0], ym[1], ym[2])) / (2.0 * h);
    }
    __syncthreads();
    const double ga[3] = {grad[0] * e1[0] + grad[1] * e2[0], grad[0] * e1[1] + grad[1] * e2[1],
                          grad[0] * e1[2] + grad[1] * e2[2]};
    // hemisphere term
    const int64_t goff = P.gamma_off[p];
    const int m = (int)(P.gamma_off[p + 1] - goff);
    double sg = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int64_t gk = goff + k;
        const double Y[3] = {P.gamma_loc[3 * gk], P.gamma_loc[3 * gk + 1], P.gamma_loc[3 * gk + 2]};
        const double ny[3] = {Y[0] / a, Y[1] / a, Y[2] / a};
        const double l = gxi + ga[0] * (Y[0] - X[0]) + ga[1] * (Y[1] - X[1]) + ga[2] * (Y[2] - X[2]);
        sg += P.gamma_w[gk] * green_ball_dnn(a, X, nx, Y, ny) * (P.U[gk] - l);
    }
    // geodesic polar frame about x_i: p = (X - o)/R, f1 = p x e_y normalised, f2 = p x f1
    const double pz = nx[2];
    double f1[3] = {-nx[2], 0.0, nx[0]};                  // p x (0, 1, 0)
    const double f1n = sqrt(f1[0] * f1[0] + f1[2] * f1[2]);
    f1[0] /= f1n; f1[2] /= f1n;
    const double f2[3] = {nx[1] * f1[2] - nx[2] * f1[1], nx[2] * f1[0] - nx[0] * f1[2], nx[0] * f1[1] - nx[1] * f1[0]};
    const double cmax = cos(f.umax);
    const int n2 = P.ng2;
    const double *gx = P.glx + n2 * (n2 - 1) / 2, *gw = P.glw + n2 * (n2 - 1) / 2;
    double ss = 0.0;
    for (int k = threadIdx.x; k < n2 * n2; k += blockDim.x) {
        const int j = k / n2, l = k - j * n2;
        double sp, cp;
        sincos(kPi * (gx[j] + 1.0), &sp, &cp);
        const double d[3] = {cp * f1[0] + sp * f2[0], cp * f1[1] + sp * f2[1], cp * f1[2] + sp * f2[2]};
        const double C0 = sqrt(pz * pz + d[2] * d[2]);
        const double smax = atan2(d[2], pz) + acos(fmin(1.0, cmax / C0));
        const double sgm = 0.5 * smax * (gx[l] + 1.0);
        const double w = kPi * gw[j] * 0.5 * smax * gw[l];
        double ss_, cs_;
        sincos(sgm, &ss_, &cs_);
        const double ny[3] = {cs_ * nx[0] + ss_ * d[0], cs_ * nx[1] + ss_ * d[1], cs_ * nx[2] + ss_ * d[2]};
        const double Y[3] = {R * ny[0], R * ny[1], R * ny[2] - R};   // o + R ny, o = (0, 0, -R)
        double y[3];
        to_global(f, Y, y);
        const double l0 = gxi + ga[0] * (Y[0] - X[0]) + ga[1] * (Y[1] - X[1]) + ga[2] * (Y[2] - X[2]);
        const double an = ga[0] * ny[0] + ga[1] * ny[1] + ga[2] * ny[2];
        const double yn = sqrt(Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2]);
        const double dnx = green_ball_dny<double>(a, Y, yn, X, nx);   // dG/dn_x(X, Y), G symmetric
        ss += w * R * R * ss_ *
              (green_ball_dnn(a, X, nx, Y, ny) * (dirichlet_eval<double>(P.dat, y[0], y[1], y[2]) - l0) + dnx * an);
    }
    sg = block_sum(sg, red);
    ss = block_sum(ss, red);
    if (threadIdx.x == 0) P.b[row] = -sg - ss;
}

}  // namespace

cudaError_t launch_second_kind(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                               const double *panel_loc, const double *panel_g, const double *gamma_loc,
                               const double *gamma_w, const double *U, int ng2, double *q, double *b,
                               int32_t *iters, double *resid, int32_t *status, cudaStream_t s) {
    if (L.panels_total == 0) return cudaSuccess;
    SkDev P;
    P.frames = D.frames;
    P.panel_off = D.panel_off;
    P.gamma_off = D.gamma_off;
    P.n_patches = L.n_patches;
    P.panel_loc = panel_loc;
    P.panel_g = panel_g;
    P.gamma_loc = gamma_loc;
    P.gamma_w = gamma_w;
    P.U = U;
    P.dat = g->dd;
    P.ng2 = ng2;
    P.glx = gl_x_dev();
    P.glw = gl_w_dev();
    P.q = q;
    P.b = b;
    P.iters = iters;
    P.status = status;
    P.resid = resid;
    second_kind_kernel<<<(unsigned)L.panels_total, kSkThreads, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace dtn

namespace dtn {

cudaError_t launch_second_kind_cap_rhs(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                                       const double *panel_loc, const double *panel_prm, const double *panel_g,
                                       const double *gamma_loc, const double *gamma_w, const double *U, int ng,
                                       double *b, cudaStream_t s) {
    if (L.panels_total == 0) return cudaSuccess;
    SkDev P{};
    P.frames = D.frames;
    P.panel_off = D.panel_off;
    P.gamma_off = D.gamma_off;
    P.n_patches = L.n_patches;
    P.panel_loc = panel_loc;
    P.panel_prm = panel_prm;
    P.panel_g = panel_g;
    P.gamma_loc = gamma_loc;
    P.gamma_w = gamma_w;
    P.U = U;
    P.dat = g->dd;
    P.ng2 = ng;
    P.glx = gl_x_dev();
    P.glw = gl_w_dev();
    P.b = b;
    second_kind_cap_rhs_kernel<<<(unsigned)L.panels_total, kSkThreads, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace dtn

namespace dtn {
cudaError_t upload_sh_second_kind(const ShTables &t) { return upload_sh_tables_here(t); }
}  // namespace dtn
