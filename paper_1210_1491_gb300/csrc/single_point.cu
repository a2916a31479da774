// single_point.cu -- Neumann data at single points of a flat boundary piece by
// the BIE-WOS formula of Sec. 4.1 (Eq. bw64):
//
//   q(x) = Sigma1' + Sigma2',
//   Sigma1' = - sum_ij W_ij (3 cos th_i / (2 pi a^3)) (U_ij - g(x))      (Eq. bw83)
//   Sigma2' = -(1/2pi) int_{S_a minus disk(x, delta)} (1/rho^3 - 1/a^3) (g(y) - g(x)) ds_y
//                                                                   (Eq. bw68, bw82)
//
// with the hemisphere Gauss nodes th_i = (pi/4)(xi_i + 1), ph_j = pi (xi_j + 1)
// (Eq. bw85) and their area weights W_ij, U_ij the walk estimates there
// (Eq. bw87), and Sigma2' by an ng2 x ng2 Gauss rule in polar coordinates about
// x over delta <= rho <= a.  The walks are the persistent walk kernel's; these
// kernels place the nodes and form the two sums.
#include <cmath>

#include "dtn_internal.h"

namespace dtn {

namespace {

// one thread per (point, node): node position and its Sigma1' weight
// W_ij 3 cos th / (2 pi a^3), node index i * ng1 + j
__global__ void sp_nodes_kernel(int64_t total, int ng1, const PatchFrame *__restrict__ frames,
                                const double *__restrict__ glx, const double *__restrict__ glw,
                                double *__restrict__ y, double *__restrict__ wk) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int nn = ng1 * ng1;
    const int64_t p = idx / nn;
    const int k = (int)(idx - p * nn), i = k / ng1, j = k - i * ng1;
    const PatchFrame &f = frames[p];
    const double *gx = glx + ng1 * (ng1 - 1) / 2, *gw = glw + ng1 * (ng1 - 1) / 2;
    const double th = 0.25 * kPi * (gx[i] + 1.0), ph = kPi * (gx[j] + 1.0);
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    const double L[3] = {f.a * st * cp, f.a * st * sp, -f.a * ct};
    for (int d = 0; d < 3; ++d) y[3 * idx + d] = f.c[d] + L[0] * f.t1[d] + L[1] * f.t2[d] + L[2] * f.n[d];
    const double W = gw[i] * gw[j] * 0.25 * kPi * kPi * f.a * f.a * st;
    wk[idx] = W * 3.0 * ct / (2.0 * kPi * f.a * f.a * f.a);
}

constexpr int kSpThreads = 128;

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kSpThreads / 32; ++w) t += red[w];   // same order in every thread
    __syncthreads();
    return t;
}

// one CTA per point: the two sums, FP64, fixed summation order
__global__ void __launch_bounds__(kSpThreads) sp_sigma_kernel(DData dat, int64_t n, int ng1, int ng2, double delta,
                                                              const PatchFrame *__restrict__ frames,
                                                              const double *__restrict__ wk,
                                                              const double *__restrict__ U,
                                                              const double *__restrict__ SE,
                                                              const double *__restrict__ glx,
                                                              const double *__restrict__ glw, double *sigma1,
                                                              double *sigma2, double *q, double *se, int32_t *status) {
    const int64_t p = blockIdx.x;
    __shared__ double red[kSpThreads / 32];
    const PatchFrame f = frames[p];
    const bool ok = (f.status == DTN_OK) && (f.kind == kDisk);
    const double gxv = dirichlet_eval<double>(dat, f.c[0], f.c[1], f.c[2]);
    const int nn = ng1 * ng1;
    double s1 = 0.0, v1 = 0.0;
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
        const int64_t idx = p * nn + k;
        const double w = wk[idx];
        s1 -= w * (U[idx] - gxv);
        v1 += w * w * SE[idx] * SE[idx];
    }
    const double *gx = glx + ng2 * (ng2 - 1) / 2, *gw = glw + ng2 * (ng2 - 1) / 2;
    const double a = f.a;
    double s2 = 0.0;
    for (int k = threadIdx.x; k < ng2 * ng2; k += blockDim.x) {
        const int i = k / ng2, j = k - i * ng2;
        const double rho = delta + 0.5 * (a - delta) * (gx[i] + 1.0);
        const double wr = 0.5 * (a - delta) * gw[i] * kPi * gw[j];
        double sa, ca;
        sincos(kPi * (gx[j] + 1.0), &sa, &ca);
        double y[3];
        for (int d = 0; d < 3; ++d) y[d] = f.c[d] + rho * ca * f.t1[d] + rho * sa * f.t2[d];
        s2 += wr * rho * (1.0 / (rho * rho * rho) - 1.0 / (a * a * a)) *
              (dirichlet_eval<double>(dat, y[0], y[1], y[2]) - gxv);
    }
    s1 = block_sum(s1, red);
    v1 = block_sum(v1, red);
    s2 = block_sum(s2, red) * (-1.0 / (2.0 * kPi));
    if (threadIdx.x == 0) {
        if (!ok) s1 = s2 = v1 = 0.0;
        if (sigma1) sigma1[p] = s1;
        if (sigma2) sigma2[p] = s2;
        q[p] = s1 + s2;
        if (se) se[p] = sqrt(v1);
        if (status) status[p] = ok ? DTN_OK : (f.status == DTN_OK ? DTN_E_UNSUPPORTED : f.status);
    }
}

}  // namespace

cudaError_t launch_sp_nodes(int64_t n, int ng1, const PatchFrame *frames, double *y, double *wk, cudaStream_t s) {
    const int64_t total = n * ng1 * ng1;
    if (total == 0) return cudaSuccess;
    const int T = 128;
    sp_nodes_kernel<<<(unsigned)((total + T - 1) / T), T, 0, s>>>(total, ng1, frames, gl_x_dev(), gl_w_dev(), y, wk);
    return cudaGetLastError();
}

cudaError_t launch_sp_sigma(const dtn_geometry *g, int64_t n, int ng1, int ng2, double delta, const PatchFrame *frames,
                            const double *wk, const double *U, const double *SE, double *sigma1, double *sigma2,
                            double *q, double *se, int32_t *status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    sp_sigma_kernel<<<(unsigned)n, kSpThreads, 0, s>>>(g->dd, n, ng1, ng2, delta, frames, wk, U, SE, gl_x_dev(),
                                                       gl_w_dev(), sigma1, sigma2, q, se, status);
    return cudaGetLastError();
}

}  // namespace dtn

namespace dtn {
cudaError_t upload_sh_single_point(const ShTables &t) { return upload_sh_tables_here(t); }
}  // namespace dtn
