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
    // the second-kind rows are written for disk patches: a wrapped patch is not supported
    const int st = (f.status == DTN_OK && f.kind != kDisk) ? DTN_E_UNSUPPORTED : f.status;
    if (i == 0 && threadIdx.x == 0) {
        if (P.iters) P.iters[p] = 0;
        if (P.resid) P.resid[p] = 0.0;
        if (P.status) P.status[p] = st;
    }
    if (st != DTN_OK) {
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

// ---------------------------------------------------------------------------
// Second kind on caps, mixed precision, as one product per patch shape.  In the
// patch frame the polar points about x_i, the kernels at them and the
// hemisphere nodes are the same for every patch of a weight group; only the
// data differ.  With g interpolated on each panel from its 8 x 8 Gauss samples
// (tensor Lagrange basis, the sample layout of the first-kind right sides) and
// l_i built from the interpolant itself (its value and tangential gradient at
// x_i, linear in the self panel's samples), g - l_i is O(|y - x_i|^2) for the
// interpolated data exactly, and the row of the polar-rule right side is
//   b_i = sum_s W_is g_s + sum_k W_i,k U_k,
//   W_is = - sum_q w_q K_q L_s(y_q) + cg_i L_s(x_i) + cv_i . grad_S L_s(x_i),
//   W_i,k = - W_k K(x_i, y_k),
//   cg_i = sum_q w_q K_q + sum_k W_k K_ik,
//   cv_i = sum_q w_q [K_q (Y_q - X_i) - dG/dn_x(x_i, y_q) n_q] + sum_k W_k K_ik (Y_k - X_i),
// (w_q the polar weights with R^2 sin sigma, K = d2G/dn_x dn_y, the L_s(x_i)
// terms on the self panel's samples only).  Weights and samples are FP64: next
// to x_i the weights are large and cancel.

constexpr int kSkWThreads = 128;
constexpr int kSkSamp = 8;           // samples per panel direction (the first kind's 8 x 8)

struct SkwDev {
    const PatchFrame *frames;
    const int64_t *panel_off, *gamma_off, *wrows_off, *wrep, *kcols, *gw_off, *vec_off, *members, *mem_off;
    int64_t n_wgroups, n_patches;
    const int32_t *nr, *ns;
    const double *panel_loc, *panel_prm, *gamma_loc, *gamma_w, *U;
    DData dat;
    int ng;
    const double *glx, *glw;
    double *W, *vec, *b;
};

// Lagrange basis on the 8 Gauss-Legendre points of [0, 1] at t
__device__ __forceinline__ void lagrange8(const double *s, const double *inv, double t, double *l) {
    for (int a = 0; a < kSkSamp; ++a) {
        double v = inv[a];
        for (int q = 0; q < kSkSamp; ++q)
            if (q != a) v *= (t - s[q]);
        l[a] = v;
    }
}

// Derivative of the same basis at t
__device__ __forceinline__ void lagrange8_d(const double *s, const double *inv, double t, double *l) {
    for (int a = 0; a < kSkSamp; ++a) {
        double sum = 0.0;
        for (int r = 0; r < kSkSamp; ++r) {
            if (r == a) continue;
            double v = 1.0;
            for (int q = 0; q < kSkSamp; ++q)
                if (q != a && q != r) v *= (t - s[q]);
            sum += v;
        }
        l[a] = inv[a] * sum;
    }
}

// One weight row per CTA.  Pass 1: the polar points (kernel weight, panel,
// local parameters) into shared memory, with the row constants.  Pass 2: thread
// t owns panels t, t + 128, ... and adds the points of its panels in index order
// to that panel's 64 weights (a fixed summation order).
__global__ void __launch_bounds__(kSkWThreads) sk_weights_kernel(SkwDev P) {
    extern __shared__ double sh[];
    const int64_t grow = blockIdx.x;
    const int64_t grp = find_group(P.wrows_off, P.n_wgroups, grow);
    const int i = (int)(grow - P.wrows_off[grp]);
    const int64_t p = P.wrep[grp];
    const PatchFrame f = P.frames[p];
    const int nr = P.nr[p], ns = P.ns[p], np = nr * ns;
    const int64_t kc = P.kcols[grp];
    const int64_t goff = P.gamma_off[p];
    const int m = (int)(P.gamma_off[p + 1] - goff);
    double *Wrow = P.W + P.gw_off[grp] + (int64_t)i * kc;
    const int nq = P.ng * P.ng;
    double *qk = sh;                 // w_q K_q per point
    int *qpan = (int *)(sh + nq);    // panel of the point
    double *qxi = sh + nq + (nq + 1) / 2, *qet = qxi + nq;
    __shared__ double red[4][kSkWThreads / 32];
    __shared__ double s8[kSkSamp], inv8[kSkSamp];
    if (threadIdx.x == 0) {
        const double *gx = P.glx + kSkSamp * (kSkSamp - 1) / 2;
        for (int a = 0; a < kSkSamp; ++a) s8[a] = 0.5 * (1.0 + gx[a]);
        for (int a = 0; a < kSkSamp; ++a) {
            double d = 1.0;
            for (int q = 0; q < kSkSamp; ++q)
                if (q != a) d *= (s8[a] - s8[q]);
            inv8[a] = 1.0 / d;
        }
    }
    const int64_t row = P.panel_off[p] + i;
    const double a = f.a, R = f.R;
    const double X[3] = {P.panel_loc[3 * row], P.panel_loc[3 * row + 1], P.panel_loc[3 * row + 2]};
    const double uc = P.panel_prm[6 * row + 4], vc = P.panel_prm[6 * row + 5];
    double su, cu, sv, cv;
    sincos(uc, &su, &cu);
    sincos(vc, &sv, &cv);
    const double nx[3] = {su * cv, su * sv, cu};
    const double pz = nx[2];
    double f1[3] = {-nx[2], 0.0, nx[0]};
    const double f1n = sqrt(f1[0] * f1[0] + f1[2] * f1[2]);
    f1[0] /= f1n; f1[2] /= f1n;
    const double f2[3] = {nx[1] * f1[2] - nx[2] * f1[1], nx[2] * f1[0] - nx[0] * f1[2], nx[0] * f1[1] - nx[1] * f1[0]};
    const double cmax = cos(f.umax), du = f.umax / nr, dv = 2.0 * kPi / ns;
    const double *gx = P.glx + P.ng * (P.ng - 1) / 2, *gw = P.glw + P.ng * (P.ng - 1) / 2;
    double cg = 0.0, cv0 = 0.0, cv1 = 0.0, cv2 = 0.0;
    for (int k = threadIdx.x; k < nq; k += blockDim.x) {
        const int j = k / P.ng, l = k - j * P.ng;
        double sp, cp;
        sincos(kPi * (gx[j] + 1.0), &sp, &cp);
        const double d[3] = {cp * f1[0] + sp * f2[0], cp * f1[1] + sp * f2[1], cp * f1[2] + sp * f2[2]};
        const double C0 = sqrt(pz * pz + d[2] * d[2]);
        const double smax = atan2(d[2], pz) + acos(fmin(1.0, cmax / C0));
        const double sgm = 0.5 * smax * (gx[l] + 1.0);
        double ss_, cs_;
        sincos(sgm, &ss_, &cs_);
        const double w = kPi * gw[j] * 0.5 * smax * gw[l] * R * R * ss_;
        const double ny[3] = {cs_ * nx[0] + ss_ * d[0], cs_ * nx[1] + ss_ * d[1], cs_ * nx[2] + ss_ * d[2]};
        const double Y[3] = {R * ny[0], R * ny[1], R * ny[2] - R};
        const double yn = sqrt(Y[0] * Y[0] + Y[1] * Y[1] + Y[2] * Y[2]);
        const double wk = w * green_ball_dnn(a, X, nx, Y, ny);
        const double wd = w * green_ball_dny<double>(a, Y, yn, X, nx);
        cg += wk;
        cv0 += wk * (Y[0] - X[0]) - wd * ny[0];
        cv1 += wk * (Y[1] - X[1]) - wd * ny[1];
        cv2 += wk * (Y[2] - X[2]) - wd * ny[2];
        // panel of the point and its parameters in the panel's box
        const double u = acos(fmin(1.0, fmax(-1.0, ny[2])));
        double v = atan2(ny[1], ny[0]);
        if (v < 0.0) v += 2.0 * kPi;
        const int ri = min(nr - 1, max(0, (int)floor(u / du)));
        const int si = min(ns - 1, max(0, (int)floor(v / dv)));
        qk[k] = -wk;
        qpan[k] = ri * ns + si;
        qxi[k] = (u - ri * du) / du;
        qet[k] = (v - si * dv) / dv;
    }
    // hemisphere nodes: W_i,k = - W_k K_ik, and their part of the row constants
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        const int64_t gk = goff + k;
        const double Y[3] = {P.gamma_loc[3 * gk], P.gamma_loc[3 * gk + 1], P.gamma_loc[3 * gk + 2]};
        const double ny[3] = {Y[0] / a, Y[1] / a, Y[2] / a};
        const double v = P.gamma_w[gk] * green_ball_dnn(a, X, nx, Y, ny);
        Wrow[(int64_t)(kSkSamp * kSkSamp) * np + k] = -v;
        cg += v;
        cv0 += v * (Y[0] - X[0]);
        cv1 += v * (Y[1] - X[1]);
        cv2 += v * (Y[2] - X[2]);
    }
    __syncthreads();
    // panel weights, thread-owned panels, points in index order
    for (int pan = threadIdx.x; pan < np; pan += blockDim.x) {
        double acc[kSkSamp * kSkSamp];
        for (int e = 0; e < kSkSamp * kSkSamp; ++e) acc[e] = 0.0;
        for (int k = 0; k < nq; ++k) {
            if (qpan[k] != pan) continue;
            double lu[kSkSamp], lv[kSkSamp];
            lagrange8(s8, inv8, qxi[k], lu);
            lagrange8(s8, inv8, qet[k], lv);
            for (int a8 = 0; a8 < kSkSamp; ++a8) {
                const double t = qk[k] * lu[a8];
                for (int b8 = 0; b8 < kSkSamp; ++b8) acc[a8 * kSkSamp + b8] += t * lv[b8];
            }
        }
        for (int e = 0; e < kSkSamp * kSkSamp; ++e) Wrow[(int64_t)pan * (kSkSamp * kSkSamp) + e] = acc[e];
    }
    // row constants (fixed-order block sums), then l_i from the interpolant:
    // cg_i L_s(x_i) + cv_i . grad_S L_s(x_i) on the self panel's 64 samples,
    // grad_S = e_u (d/du) / R + e_v (d/dv) / (R sin u)
    double v4[4] = {cg, cv0, cv1, cv2};
    for (int c = 0; c < 4; ++c)
        for (int o = 16; o > 0; o >>= 1) v4[c] += __shfl_xor_sync(0xffffffffu, v4[c], o);
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 4; ++c) red[c][threadIdx.x >> 5] = v4[c];
    __syncthreads();
    if (threadIdx.x == 0) {
        double t4[4];
        for (int c = 0; c < 4; ++c) {
            t4[c] = 0.0;
            for (int w8 = 0; w8 < kSkWThreads / 32; ++w8) t4[c] += red[c][w8];
        }
        const double *prm = P.panel_prm + 6 * row;
        const double xi = (uc - prm[0]) / (prm[1] - prm[0]), et = (vc - prm[2]) / (prm[3] - prm[2]);
        double lu[kSkSamp], lv[kSkSamp], du_[kSkSamp], dv_[kSkSamp];
        lagrange8(s8, inv8, xi, lu);
        lagrange8(s8, inv8, et, lv);
        lagrange8_d(s8, inv8, xi, du_);
        lagrange8_d(s8, inv8, et, dv_);
        const double e1[3] = {cu * cv, cu * sv, -su}, e2[3] = {-sv, cv, 0.0};
        const double c1 = (t4[1] * e1[0] + t4[2] * e1[1] + t4[3] * e1[2]) / (R * (prm[1] - prm[0]));
        const double c2 = (t4[1] * e2[0] + t4[2] * e2[1] + t4[3] * e2[2]) / (R * su * (prm[3] - prm[2]));
        double *Ws = Wrow + (int64_t)i * (kSkSamp * kSkSamp);
        for (int a8 = 0; a8 < kSkSamp; ++a8)
            for (int b8 = 0; b8 < kSkSamp; ++b8)
                Ws[a8 * kSkSamp + b8] += t4[0] * lu[a8] * lv[b8] + c1 * du_[a8] * lv[b8] + c2 * lu[a8] * dv_[b8];
    }
}

// Per patch: the FP64 data samples at each panel's 8 x 8 Gauss points and the
// hemisphere values (the first kind's sample layout, unshifted), one thread per
// entry.
__global__ void sk_samples_kernel(SkwDev P, int64_t total) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= total) return;
    const int64_t p = find_group(P.vec_off, P.n_patches, e);
    const int64_t c = e - P.vec_off[p];
    const PatchFrame f = P.frames[p];
    const int np = P.nr[p] * P.ns[p];
    if (c >= (int64_t)(kSkSamp * kSkSamp) * np) {
        P.vec[e] = P.U[P.gamma_off[p] + (c - (int64_t)(kSkSamp * kSkSamp) * np)];
        return;
    }
    const int pan = (int)(c / (kSkSamp * kSkSamp)), ab = (int)(c - (int64_t)pan * (kSkSamp * kSkSamp));
    const double *gx = P.glx + kSkSamp * (kSkSamp - 1) / 2;
    const double *prm = P.panel_prm + 6 * (P.panel_off[p] + pan);
    const double u = prm[0] + 0.5 * (1.0 + gx[ab / kSkSamp]) * (prm[1] - prm[0]);
    const double v = prm[2] + 0.5 * (1.0 + gx[ab % kSkSamp]) * (prm[3] - prm[2]);
    double Y[3], nl[3], J;
    patch_point<double>(f.kind, f.R, u, v, Y, nl, J);
    double y[3];
    to_global(f, Y, y);
    P.vec[e] = dirichlet_eval<double>(P.dat, y[0], y[1], y[2]);
}

// b_i = sum_c W_ic vec_c for every row of every patch: one CTA per (patch,
// block of 32 rows), a warp per row in turn, lanes over the columns,
// fixed-order sums.
constexpr int kSkRowsPerCta = 32;

__global__ void __launch_bounds__(kSkWThreads) sk_product_kernel(SkwDev P) {
    const int64_t idx = blockIdx.x;   // member index
    const int64_t grp = find_group(P.mem_off, P.n_wgroups, idx);
    const int64_t p = P.members[idx];
    const PatchFrame f = P.frames[p];
    const int n = (int)(P.wrows_off[grp + 1] - P.wrows_off[grp]);
    const int64_t kc = P.kcols[grp];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double *vec = P.vec + P.vec_off[p];
    for (int i = blockIdx.y * kSkRowsPerCta + warp; i < min(n, (int)(blockIdx.y + 1) * kSkRowsPerCta);
         i += kSkWThreads / 32) {
        const int64_t row = P.panel_off[p] + i;
        if (f.status != DTN_OK) {
            if (lane == 0) P.b[row] = 0.0;
            continue;
        }
        const double *Wr = P.W + P.gw_off[grp] + (int64_t)i * kc;
        double s = 0.0;
        for (int64_t c = lane; c < kc; c += 32) s = fma(Wr[c], vec[c], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) P.b[row] = s;
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

namespace dtn {
cudaError_t upload_sh_second_kind(const ShTables &t) { return upload_sh_tables_here(t); }
}  // namespace dtn

namespace dtn {

// Second kind on caps, mixed precision: group weights (once per weight group),
// FP64 samples per patch, then the product.  W: wrows x kcols doubles per group
// (gw_off), vec: FP64 samples (vec_off).
cudaError_t launch_second_kind_cap_rhs_shared(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                                              const double *panel_loc, const double *panel_prm,
                                              const double *gamma_loc, const double *gamma_w, const double *U,
                                              int ng, double *W, double *vec, double *b, cudaStream_t s) {
    if (L.panels_total == 0 || L.wrows_total == 0) return cudaSuccess;
    SkwDev P{};
    P.frames = D.frames;
    P.panel_off = D.panel_off;
    P.gamma_off = D.gamma_off;
    P.wrows_off = D.wrows_off;
    P.wrep = D.wrep;
    P.kcols = D.kcols;
    P.gw_off = D.gw_off;
    P.vec_off = D.vec_off;
    P.members = D.members;
    P.mem_off = D.mem_off;
    P.n_wgroups = L.n_wgroups;
    P.n_patches = L.n_patches;
    P.nr = D.nr;
    P.ns = D.ns;
    P.panel_loc = panel_loc;
    P.panel_prm = panel_prm;
    P.gamma_loc = gamma_loc;
    P.gamma_w = gamma_w;
    P.U = U;
    P.dat = g->dd;
    P.ng = ng;
    P.glx = gl_x_dev();
    P.glw = gl_w_dev();
    P.W = W;
    P.vec = vec;
    P.b = b;
    const int nq = ng * ng;
    const size_t smem = (size_t)nq * 8 + (size_t)((nq + 1) / 2) * 8 + 2 * (size_t)nq * 8;
    // the largest ring order's table, set once (outside any stream capture that follows)
    static bool smem_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!smem_set[dev]) {
        const size_t smax = (size_t)kMaxGauss * kMaxGauss * 8 * 4;
        if ((e = cudaFuncSetAttribute(sk_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax)) !=
            cudaSuccess)
            return e;
        smem_set[dev] = true;
    }
    sk_weights_kernel<<<(unsigned)L.wrows_total, kSkWThreads, smem, s>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    sk_samples_kernel<<<(unsigned)((L.vec_total + 255) / 256), 256, 0, s>>>(P, L.vec_total);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((unsigned)L.n_patches, (unsigned)((L.max_wgroup_rows + kSkRowsPerCta - 1) / kSkRowsPerCta));
    sk_product_kernel<<<grid, kSkWThreads, 0, s>>>(P);
    return cudaGetLastError();
}

}  // namespace dtn
