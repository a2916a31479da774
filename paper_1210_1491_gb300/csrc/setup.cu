// setup.cu -- patch setup on the device: local frame of each patch, the
// hemisphere Gauss nodes of Gamma (Eq. bw85 on theta in [0, theta_max]) and
// the panels of S with their collocation points (Sec. 5.2 collocation).
#include <cmath>
#include <mutex>

#include "dtn_internal.h"

namespace dtn {

namespace {
// Gauss-Legendre and spherical-harmonic tables, one copy per device (uploaded
// with that device current, together with every unit's __constant__ copy)
constexpr int kMaxTableDevices = 64;
std::mutex g_tab_mu;
bool g_tab_ready[kMaxTableDevices] = {false};
double *g_glx[kMaxTableDevices] = {nullptr}, *g_glw[kMaxTableDevices] = {nullptr};
ShTables *g_sh[kMaxTableDevices] = {nullptr};

int current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxTableDevices) return -1;
    return dev;
}
}  // namespace

// Gauss-Legendre by Newton iteration on P_n from its three-term recurrence,
// starting from the asymptotic guess cos(pi (i - 1/4) / (n + 1/2)).
void gauss_legendre_host(int n, double *x, double *w) {
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double pp = 1.0;
        for (int it = 0; it < 64; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int k = 0; k < n; ++k) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * k + 1.0) * z * p2 - k * p3) / (k + 1.0);
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            const double z1 = z;
            z = z1 - p1 / pp;
            if (std::fabs(z - z1) <= 1e-16) {
                p1 = 1.0; p2 = 0.0;
                for (int k = 0; k < n; ++k) {
                    const double p3 = p2;
                    p2 = p1;
                    p1 = ((2.0 * k + 1.0) * z * p2 - k * p3) / (k + 1.0);
                }
                pp = n * (z * p1 - p2) / (z * z - 1.0);
                break;
            }
        }
        const double wt = 2.0 / ((1.0 - z * z) * pp * pp);
        x[i] = -z; x[n - 1 - i] = z;
        w[i] = wt; w[n - 1 - i] = wt;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

cudaError_t ensure_tables() {
    const int dev = current_device();
    if (dev < 0) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (g_tab_ready[dev]) return cudaSuccess;
    const int total = kMaxGauss * (kMaxGauss + 1) / 2;
    std::vector<double> hx(total), hw(total);
    for (int n = 1; n <= kMaxGauss; ++n) gauss_legendre_host(n, &hx[n * (n - 1) / 2], &hw[n * (n - 1) / 2]);
    cudaError_t e = cudaMalloc(&g_glx[dev], total * sizeof(double));
    if (e != cudaSuccess) return e;
    e = cudaMalloc(&g_glw[dev], total * sizeof(double));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(g_glx[dev], hx.data(), total * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(g_glw[dev], hw.data(), total * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    ShTables t{};
    for (int l = 0; l <= kMaxL; ++l) {
        for (int m = 0; m <= l; ++m) {
            double A = 0.0, B = 0.0;
            if (l > m) {
                A = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                const double lm1 = l - 1.0;
                B = std::sqrt(std::max(0.0, (lm1 * lm1 - (double)m * m) / (4.0 * lm1 * lm1 - 1.0)));
            }
            t.A[l][m] = A; t.B[l][m] = B;
            t.Af[l][m] = (float)A; t.Bf[l][m] = (float)B;
        }
    }
    for (int m = 1; m <= kMaxL; ++m) {
        t.D[m] = std::sqrt((2.0 * m + 1.0) / (2.0 * m));
        t.Df[m] = (float)t.D[m];
    }
    for (int m = 0; m <= kMaxL; ++m)
        for (int l = m + 2; l <= kMaxL; ++l) t.beta[sh_pair(l, m)] = (float)(t.B[l][m] / t.A[l - 1][m]);
    e = cudaMalloc(&g_sh[dev], sizeof(ShTables));
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(g_sh[dev], &t, sizeof(t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    if ((e = upload_sh_tables_here(t)) != cudaSuccess) return e;
    if ((e = upload_sh_wos(t)) != cudaSuccess) return e;
    if ((e = upload_sh_assemble(t)) != cudaSuccess) return e;
    if ((e = upload_sh_second_kind(t)) != cudaSuccess) return e;
    if ((e = upload_sh_single_point(t)) != cudaSuccess) return e;
    g_tab_ready[dev] = true;
    return cudaSuccess;
}

// the tables of the current device (every launch goes to the current device,
// which the entry points check is the geometry's)
const double *gl_x_dev() {
    const int d = current_device();
    return d < 0 ? nullptr : g_glx[d];
}
const double *gl_w_dev() {
    const int d = current_device();
    return d < 0 ? nullptr : g_glw[d];
}
const ShTables *sh_tables_dev() {
    const int d = current_device();
    return d < 0 ? nullptr : g_sh[d];
}

namespace {

__device__ void frame_from_normal(PatchFrame &f) {
    int ax = 0;
    for (int i = 1; i < 3; ++i)
        if (fabs(f.n[i]) < fabs(f.n[ax])) ax = i;
    double t[3] = {-f.n[ax] * f.n[0], -f.n[ax] * f.n[1], -f.n[ax] * f.n[2]};
    t[ax] += 1.0;
    const double tn = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
    for (int i = 0; i < 3; ++i) f.t1[i] = t[i] / tn;
    f.t2[0] = f.n[1] * f.t1[2] - f.n[2] * f.t1[1];
    f.t2[1] = f.n[2] * f.t1[0] - f.n[0] * f.t1[2];
    f.t2[2] = f.n[0] * f.t1[1] - f.n[1] * f.t1[0];
}

// One thread per patch: which boundary piece the centre lies on, the frame,
// the polar range of the hemisphere and the radial range of the panels.
// Status DTN_E_UNSUPPORTED when the ball meets more than that one smooth piece
// (a plane face, or the sphere of a ball region).
__global__ void patch_frame_kernel(DGeom g, int64_t n, const double *__restrict__ centers,
                                   const double *__restrict__ radius, PatchFrame *__restrict__ out) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    PatchFrame f;
    const double c[3] = {centers[3 * p], centers[3 * p + 1], centers[3 * p + 2]};
    const double a = radius[p];
    for (int i = 0; i < 3; ++i) f.c[i] = c[i];
    f.a = a;
    f.status = DTN_OK;
    f.R = 0.0;
    if (!(a > 0.0)) f.status = DTN_E_INVALID_ARG;
    if (g.kind == kHalfSpace || g.kind == kDiskExterior) {
        // the plane z = c_z (half space: the region above it; thin disk: its top
        // face, with the ball's slice of the plane inside the disk)
        if (!(fabs(c[2] - g.c[2]) <= 1e-9 * fmax(1.0, fabs(g.c[2])))) f.status = DTN_E_UNSUPPORTED;
        if (g.kind == kDiskExterior && !(sqrt((c[0] - g.c[0]) * (c[0] - g.c[0]) + (c[1] - g.c[1]) * (c[1] - g.c[1])) + a < g.R))
            f.status = DTN_E_UNSUPPORTED;
        f.n[0] = 0.0; f.n[1] = 0.0; f.n[2] = -1.0;
        f.kind = kDisk;
        f.theta_max = 0.5 * kPi;
        f.umax = a;
    } else if (g.kind == kBallExterior) {
        // outside a sphere: the region's outward normal points into the sphere,
        // whose centre lies at c + R n; the cap takes the signed radius -R
        const double v[3] = {c[0] - g.c[0], c[1] - g.c[1], c[2] - g.c[2]};
        const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(fabs(r - g.R) <= 1e-9 * g.R) || !(a < 2.0 * g.R)) f.status = DTN_E_UNSUPPORTED;
        const double rr = r > 0.0 ? r : 1.0;
        for (int i = 0; i < 3; ++i) f.n[i] = -v[i] / rr;
        f.kind = kCap;
        f.R = -g.R;
        f.theta_max = kPi - acos(fmin(1.0, a / (2.0 * g.R)));
        f.umax = 2.0 * asin(fmin(1.0, a / (2.0 * g.R)));
    } else if (g.kind == kBall) {
        const double v[3] = {c[0] - g.c[0], c[1] - g.c[1], c[2] - g.c[2]};
        const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(fabs(r - g.R) <= 1e-9 * g.R) || !(a < 2.0 * g.R)) f.status = DTN_E_UNSUPPORTED;
        const double rr = r > 0.0 ? r : 1.0;
        for (int i = 0; i < 3; ++i) f.n[i] = v[i] / rr;
        f.kind = kCap;
        f.R = g.R;
        f.theta_max = acos(a / (2.0 * g.R));
        f.umax = 2.0 * asin(fmin(1.0, a / (2.0 * g.R)));
    } else {
        double best = INFINITY;
        int bw = -1, bf = 0;
        for (int fc = 0; fc < 6; ++fc) {
            const int ax = fc >> 1;
            const double d = fabs((fc & 1) ? g.hi[ax] - c[ax] : c[ax] - g.lo[ax]);
            if (d < best) { best = d; bw = -1; bf = fc; }
        }
        if (g.kind == kBoxMinusBoxes) {
            for (int b = 0; b < g.nb; ++b) {
                const double *lo = g.boxes + 6 * b, *hi = lo + 3;
                for (int fc = 0; fc < 6; ++fc) {
                    const int ax = fc >> 1;
                    const double d = fabs((fc & 1) ? c[ax] - hi[ax] : c[ax] - lo[ax]);
                    bool in = true;
                    for (int i = 0; i < 3; ++i)
                        if (i != ax && (c[i] < lo[i] || c[i] > hi[i])) in = false;
                    if (in && d < best) { best = d; bw = b; bf = fc; }
                }
            }
        }
        const int ax = bf >> 1, side = bf & 1;
        f.n[0] = f.n[1] = f.n[2] = 0.0;
        f.n[ax] = (bw < 0) ? (side ? 1.0 : -1.0) : (side ? -1.0 : 1.0);
        f.kind = kDisk;
        f.theta_max = 0.5 * kPi;
        f.umax = a;
        double scale = fmax(fmax(g.hi[0] - g.lo[0], g.hi[1] - g.lo[1]), g.hi[2] - g.lo[2]);
        if (!(best <= 1e-9 * scale)) f.status = DTN_E_UNSUPPORTED;
        // the ball may meet this face only
        for (int fc = 0; fc < 6; ++fc) {
            if (bw < 0 && fc == bf) continue;
            const int fx = fc >> 1;
            const double d = (fc & 1) ? g.hi[fx] - c[fx] : c[fx] - g.lo[fx];
            if (d <= a) f.status = DTN_E_UNSUPPORTED;
        }
        if (bw >= 0) {
            const double *lo = g.boxes + 6 * bw, *hi = lo + 3;
            for (int i = 0; i < 3; ++i)
                if (i != ax && (c[i] - lo[i] <= a || hi[i] - c[i] <= a)) f.status = DTN_E_UNSUPPORTED;
            if (hi[ax] - lo[ax] <= a) f.status = DTN_E_UNSUPPORTED;
        }
        if (g.kind == kBoxMinusBoxes) {
            for (int b = 0; b < g.nb; ++b) {
                if (b == bw) continue;
                const double *bb = g.boxes + 6 * b;
                double s = 0.0;
                for (int i = 0; i < 3; ++i) {
                    const double t = fmax(fmax(bb[i] - c[i], 0.0), c[i] - bb[i + 3]);
                    s += t * t;
                }
                if (sqrt(s) <= a) f.status = DTN_E_UNSUPPORTED;
            }
        }
    }
    frame_from_normal(f);
    out[p] = f;
}

__global__ void gamma_nodes_kernel(int64_t n_patches, int64_t total, const int64_t *__restrict__ off,
                                   const int32_t *__restrict__ nt, const int32_t *__restrict__ nph,
                                   const PatchFrame *__restrict__ frames, const double *__restrict__ glx,
                                   const double *__restrict__ glw, double *__restrict__ xyz,
                                   double *__restrict__ w, double *__restrict__ loc) {
    const int64_t gidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gidx >= total) return;
    const int64_t p = find_group(off, n_patches, gidx);
    const int k = (int)(gidx - off[p]);
    const int n1 = nt[p], n2 = nph[p];
    const int i = k / n2, j = k % n2;
    const PatchFrame &f = frames[p];
    const double xi = glx[n1 * (n1 - 1) / 2 + i], wi = glw[n1 * (n1 - 1) / 2 + i];
    const double xj = glx[n2 * (n2 - 1) / 2 + j], wj = glw[n2 * (n2 - 1) / 2 + j];
    const double th = 0.5 * f.theta_max * (xi + 1.0);
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincospi(xj + 1.0, &sp, &cp);
    const double L[3] = {f.a * st * cp, f.a * st * sp, -f.a * ct};
    if (loc) { loc[3 * gidx] = L[0]; loc[3 * gidx + 1] = L[1]; loc[3 * gidx + 2] = L[2]; }
    if (xyz)
        for (int d = 0; d < 3; ++d) xyz[3 * gidx + d] = f.c[d] + L[0] * f.t1[d] + L[1] * f.t2[d] + L[2] * f.n[d];
    if (w) w[gidx] = wi * wj * 0.5 * f.theta_max * kPi * f.a * f.a * st;
}

// Panels: ring r, sector s of the patch parameter box.  Collocation point:
// the area centroid of a disk panel, or the radial projection of the area
// centroid of a cap panel onto the sphere.
__global__ void panels_kernel(DData dat, int64_t n_patches, int64_t total, const int64_t *__restrict__ off,
                              const int32_t *__restrict__ nr, const int32_t *__restrict__ ns,
                              const PatchFrame *__restrict__ frames, double *__restrict__ colloc,
                              double *__restrict__ normals, double *__restrict__ areas,
                              double *__restrict__ loc, double *__restrict__ prm,
                              double *__restrict__ aux, double *__restrict__ gval) {
    const int64_t gidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gidx >= total) return;
    const int64_t p = find_group(off, n_patches, gidx);
    const int k = (int)(gidx - off[p]);
    const int r = k / ns[p], s = k % ns[p];
    const PatchFrame &f = frames[p];
    const double du = f.umax / nr[p], dv = 2.0 * kPi / ns[p];
    const double u0 = r * du, u1 = (r + 1) * du, v0 = s * dv, v1 = (s + 1) * dv;
    const double vc = 0.5 * (v0 + v1);
    const double sinc = sin(0.5 * dv) / (0.5 * dv);
    double uc, area;
    if (f.kind == kDisk) {
        uc = (2.0 / 3.0) * (u1 * u1 * u1 - u0 * u0 * u0) / (u1 * u1 - u0 * u0) * sinc;
        area = 0.5 * (u1 * u1 - u0 * u0) * dv;
    } else {
        const double Is = 0.5 * ((u1 - sin(u1) * cos(u1)) - (u0 - sin(u0) * cos(u0)));
        const double Ic = 0.5 * (sin(u1) * sin(u1) - sin(u0) * sin(u0));
        uc = atan2(Is * sinc, Ic);
        area = f.R * f.R * (cos(u0) - cos(u1)) * dv;
    }
    double Y[3], nl[3], J;
    patch_point<double>(f.kind, f.R, uc, vc, Y, nl, J);
    double x[3], nn[3];
    for (int d = 0; d < 3; ++d) {
        x[d] = f.c[d] + Y[0] * f.t1[d] + Y[1] * f.t2[d] + Y[2] * f.n[d];
        nn[d] = nl[0] * f.t1[d] + nl[1] * f.t2[d] + nl[2] * f.n[d];
    }
    if (colloc) for (int d = 0; d < 3; ++d) colloc[3 * gidx + d] = x[d];
    if (normals) for (int d = 0; d < 3; ++d) normals[3 * gidx + d] = nn[d];
    if (areas) areas[gidx] = area;
    for (int d = 0; d < 3; ++d) loc[3 * gidx + d] = Y[d];
    double *q = prm + 6 * gidx;
    q[0] = u0; q[1] = u1; q[2] = v0; q[3] = v1; q[4] = uc; q[5] = vc;
    // physical centre (parameter midpoint) and bounding radius over corners and edge midpoints
    double Yc[3], nc[3], Jc;
    patch_point<double>(f.kind, f.R, 0.5 * (u0 + u1), vc, Yc, nc, Jc);
    double rad = 0.0;
    for (int cu = 0; cu < 3; ++cu)
        for (int cv = 0; cv < 3; ++cv) {
            double Yq[3], nq[3], Jq;
            patch_point<double>(f.kind, f.R, u0 + 0.5 * cu * (u1 - u0), v0 + 0.5 * cv * (v1 - v0), Yq, nq, Jq);
            const double dd = sqrt((Yq[0] - Yc[0]) * (Yq[0] - Yc[0]) + (Yq[1] - Yc[1]) * (Yq[1] - Yc[1]) +
                                   (Yq[2] - Yc[2]) * (Yq[2] - Yc[2]));
            rad = fmax(rad, dd);
        }
    aux[4 * gidx] = Yc[0]; aux[4 * gidx + 1] = Yc[1]; aux[4 * gidx + 2] = Yc[2];
    aux[4 * gidx + 3] = rad;
    const double gv = dirichlet_eval<double>(dat, x[0], x[1], x[2]);
    gval[gidx] = gv;
}

}  // namespace

cudaError_t launch_patch_frames(const dtn_geometry *g, int64_t n, const double *centers, const double *radius,
                                PatchFrame *frames, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int T = 128;
    patch_frame_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(g->dg, n, centers, radius, frames);
    return cudaGetLastError();
}

cudaError_t launch_patch_setup(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                               const double *centers, double *gamma_xyz,
                               double *gamma_w, double *gamma_loc, double *colloc, double *normals,
                               double *areas, double *panel_loc, double *panel_prm, double *panel_aux,
                               double *panel_g, cudaStream_t s) {
    const int T = 128;
    const int64_t n = L.n_patches;
    patch_frame_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(g->dg, n, centers, D.radius, D.frames);
    if (L.gamma_total > 0)
        gamma_nodes_kernel<<<(unsigned)((L.gamma_total + T - 1) / T), T, 0, s>>>(
            n, L.gamma_total, D.gamma_off, D.nt, D.nph, D.frames, gl_x_dev(), gl_w_dev(), gamma_xyz,
            gamma_w, gamma_loc);
    if (L.panels_total > 0)
        panels_kernel<<<(unsigned)((L.panels_total + T - 1) / T), T, 0, s>>>(
            g->dd, n, L.panels_total, D.panel_off, D.nr, D.ns, D.frames, colloc, normals, areas,
            panel_loc, panel_prm, panel_aux, panel_g);
    return cudaGetLastError();
}

}  // namespace dtn
