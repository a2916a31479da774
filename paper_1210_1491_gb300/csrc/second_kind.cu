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
