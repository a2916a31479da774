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

// The piece of box face fc (axis fc/2, the lo face for even fc) inside the
// ball B(c, a); false if the ball misses the closed face rectangle.  The angle
// range of the rays from P into the rectangle is cut at the directions of the
// rectangle's corners inside the slice circle and of the circle's crossings
// with the rectangle sides (cuts closer than 1e-12 merged).
__device__ bool make_piece(const double *lo, const double *hi, int fc, const double c[3], double a, Piece &q) {
    q.ax = fc >> 1;
    q.side = fc & 1;
    q.fv = q.side ? hi[q.ax] : lo[q.ax];
    const double d = c[q.ax] - q.fv;
    if (!(fabs(d) < a)) return false;
    q.ua = (q.ax == 0) ? 1 : 0;
    q.va = (q.ax == 2) ? 1 : 2;
    const int ax2[2] = {q.ua, q.va};
    for (int k = 0; k < 2; ++k) {
        q.rlo[k] = lo[ax2[k]];
        q.rhi[k] = hi[ax2[k]];
        q.cf[k] = c[ax2[k]];
        q.P[k] = fmin(fmax(q.cf[k], q.rlo[k]), q.rhi[k]);
    }
    q.rf = sqrt(a * a - d * d);
    // a polar origin closer than rf/4 to a rectangle side moves onto it (onto
    // the corner when near two) if it stays well inside the disk: otherwise the
    // rings of the thin strip between it and the side are sliver panels
    for (int k = 0; k < 2; ++k) {
        const double dl = q.P[k] - q.rlo[k], dh = q.rhi[k] - q.P[k];
        if (fmin(dl, dh) < 0.25 * q.rf) {
            const double t = dl <= dh ? q.rlo[k] : q.rhi[k];
            const double e0 = (k == 0 ? t : q.P[0]) - q.cf[0], e1 = (k == 1 ? t : q.P[1]) - q.cf[1];
            if (hypot(e0, e1) < 0.9 * q.rf) q.P[k] = t;
        }
    }
    for (int k = 0; k < 2; ++k) {
        q.onlo[k] = (q.P[k] == q.rlo[k]);
        q.onhi[k] = (q.P[k] == q.rhi[k]);
    }
    if (!(hypot(q.P[0] - q.cf[0], q.P[1] - q.cf[1]) < q.rf)) return false;
    // angle range: halved by each rectangle side through P
    double ph0 = 0.0, ph1 = 2.0 * kPi;
    const bool l0 = q.onlo[0], h0 = q.onhi[0], l1 = q.onlo[1], h1 = q.onhi[1];
    if (l0 && l1) { ph0 = 0.0; ph1 = 0.5 * kPi; }
    else if (h0 && l1) { ph0 = 0.5 * kPi; ph1 = kPi; }
    else if (h0 && h1) { ph0 = kPi; ph1 = 1.5 * kPi; }
    else if (l0 && h1) { ph0 = 1.5 * kPi; ph1 = 2.0 * kPi; }
    else if (l0) { ph0 = -0.5 * kPi; ph1 = 0.5 * kPi; }
    else if (h0) { ph0 = 0.5 * kPi; ph1 = 1.5 * kPi; }
    else if (l1) { ph0 = 0.0; ph1 = kPi; }
    else if (h1) { ph0 = kPi; ph1 = 2.0 * kPi; }
    double pts[12][2];
    int np = 0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const double Q0 = i ? q.rhi[0] : q.rlo[0], Q1 = j ? q.rhi[1] : q.rlo[1];
            if (hypot(Q0 - q.cf[0], Q1 - q.cf[1]) < q.rf) { pts[np][0] = Q0; pts[np][1] = Q1; ++np; }
        }
    for (int k = 0; k < 2; ++k) {
        const int o = 1 - k;
        for (int sd = 0; sd < 2; ++sd) {
            const double uk = sd ? q.rhi[k] : q.rlo[k];
            const double h2 = q.rf * q.rf - (uk - q.cf[k]) * (uk - q.cf[k]);
            if (!(h2 > 0.0)) continue;
            const double hh = sqrt(h2);
            for (int sg = -1; sg <= 1; sg += 2) {
                const double vo = q.cf[o] + sg * hh;
                if (vo > q.rlo[o] && vo < q.rhi[o]) { pts[np][k] = uk; pts[np][o] = vo; ++np; }
            }
        }
    }
    double cut[12];
    int nc = 0;
    for (int i = 0; i < np; ++i) {
        const double dx = pts[i][0] - q.P[0], dy = pts[i][1] - q.P[1];
        if (hypot(dx, dy) < 1e-12 * q.rf) continue;
        double ang = atan2(dy, dx);
        while (ang < ph0) ang += 2.0 * kPi;
        while (ang >= ph0 + 2.0 * kPi) ang -= 2.0 * kPi;
        if (ang > ph0 + 1e-12 && ang < ph1 - 1e-12) {
            int j = nc++;   // insertion sort
            while (j > 0 && cut[j - 1] > ang) { cut[j] = cut[j - 1]; --j; }
            cut[j] = ang;
        }
    }
    q.sub[0] = ph0;
    q.nsub = 0;
    for (int i = 0; i < nc; ++i)
        if (cut[i] - q.sub[q.nsub] > 1e-12 && q.nsub < kMaxSub) q.sub[++q.nsub] = cut[i];
    if (ph1 - q.sub[q.nsub] > 1e-12 && q.nsub < kMaxSub) q.sub[++q.nsub] = ph1;
    else q.sub[q.nsub] = ph1;
    // what bounds each sub-range (at its middle angle): the circle or a side
    for (int j = 0; j < q.nsub; ++j) {
        const double vm = 0.5 * (q.sub[j] + q.sub[j + 1]);
        double e[2];
        sincos(vm, &e[1], &e[0]);
        const double w0 = q.P[0] - q.cf[0], w1 = q.P[1] - q.cf[1];
        const double we = w0 * e[0] + w1 * e[1];
        double best = -we + sqrt(fmax(0.0, we * we - (w0 * w0 + w1 * w1) + q.rf * q.rf));
        q.stype[j] = 0;
        q.svn[j] = 0.0;
        q.sdist[j] = 0.0;
        for (int k = 0; k < 2; ++k) {
            // the side u_k = rhi (normal angle 0 or pi/2) or u_k = rlo (pi or 3pi/2)
            if (e[k] > 0.0 && !q.onhi[k]) {
                const double t = (q.rhi[k] - q.P[k]) / e[k];
                if (t < best) { best = t; q.stype[j] = 1; q.svn[j] = k ? 0.5 * kPi : 0.0; q.sdist[j] = q.rhi[k] - q.P[k]; }
            }
            if (e[k] < 0.0 && !q.onlo[k]) {
                const double t = (q.rlo[k] - q.P[k]) / e[k];
                if (t < best) { best = t; q.stype[j] = 1; q.svn[j] = k ? 1.5 * kPi : kPi; q.sdist[j] = q.P[k] - q.rlo[k]; }
            }
        }
        // keep v - svn in (-pi, pi] for the tangent
        if (q.stype[j])
            while (q.svn[j] - vm > kPi) q.svn[j] -= 2.0 * kPi;
        if (q.stype[j])
            while (vm - q.svn[j] > kPi) q.svn[j] += 2.0 * kPi;
    }
    return true;
}

// int_{v0}^{v1} rho_max(v)^2 dv by the 32-point Gauss rule
__device__ double rho2_integral(const Piece &q, double v0, double v1, const double *glx, const double *glw) {
    const double *gx = glx + 32 * 31 / 2, *gw = glw + 32 * 31 / 2;
    const double h = 0.5 * (v1 - v0), m = 0.5 * (v0 + v1);
    double s = 0.0;
    for (int i = 0; i < 32; ++i) {
        const double r = piece_rho(q, m + h * gx[i]);
        s += gw[i] * h * r * r;
    }
    return s;
}

// One thread per patch: which boundary piece the centre lies on, the frame,
// the polar range of the hemisphere and the radial range of the panels.
// Status DTN_E_UNSUPPORTED when the ball meets more than that one smooth piece
// (a plane face, or the sphere of a ball region), except on an obstacle box
// whose further faces it meets (a wrapped patch, with `pieces` and `ns`
// given): there the ball must reach no other conductor and the box must be at
// least a thick along n (else Gamma is not star-shaped about the pole); the
// pieces are built and the patch's ns sectors shared among their sub-ranges,
// one each, then one at a time to the sub-range with the largest area per
// sector (a larger ratio wins only by more than 1e-12 relative; lowest index
// otherwise).
__global__ void patch_frame_kernel(DGeom g, int64_t n, const double *__restrict__ centers,
                                   const double *__restrict__ radius, PatchFrame *__restrict__ out,
                                   Piece *__restrict__ pieces, const int32_t *__restrict__ nsec,
                                   const int32_t *__restrict__ nring,
                                   const double *__restrict__ glx, const double *__restrict__ glw) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    PatchFrame f;
    const double c[3] = {centers[3 * p], centers[3 * p + 1], centers[3 * p + 2]};
    const double a = radius[p];
    for (int i = 0; i < 3; ++i) { f.c[i] = c[i]; f.blo[i] = 0.0; f.bhi[i] = 0.0; }
    f.a = a;
    f.status = DTN_OK;
    f.R = 0.0;
    f.npiece = 0;
    bool wrap = false;
    int wbox = -1, wface = 0;
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
                if (i != ax && (c[i] - lo[i] <= a || hi[i] - c[i] <= a)) wrap = true;
            if (hi[ax] - lo[ax] <= a) wrap = true;
            if (wrap) {
                // Gamma is star-shaped about the pole iff the box is at least a
                // thick along n: the arc from the pole enters the box once and
                // stays in it through theta = pi
                if (hi[ax] - lo[ax] < a || !pieces || !nsec || !nring) f.status = DTN_E_UNSUPPORTED;
                wbox = bw;
                wface = bf;
                for (int i = 0; i < 3; ++i) { f.blo[i] = lo[i]; f.bhi[i] = hi[i]; }
                f.kind = kWrapped;
                f.theta_max = 0.0;
                f.umax = 0.0;
            }
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
    if (f.kind == kWrapped && f.status == DTN_OK) {
        const double *lo = g.boxes + 6 * wbox, *hi = lo + 3;
        Piece *pc = pieces + p * kMaxPieces;
        int np = 0;
        for (int k = 0; k < 6; ++k) {
            // the face containing c first, then the others in face order
            const int fc = (k == 0) ? wface : (k <= wface ? k - 1 : k);
            Piece q;
            if (!make_piece(lo, hi, fc, c, a, q)) continue;
            // the piece's origin, in-plane axes and normal (into the box) in the frame
            double Pg[3], Ug[3] = {0.0, 0.0, 0.0}, Vg[3] = {0.0, 0.0, 0.0}, Ng[3] = {0.0, 0.0, 0.0};
            Pg[q.ax] = q.fv;
            Pg[q.ua] = q.P[0];
            Pg[q.va] = q.P[1];
            Ug[q.ua] = 1.0;
            Vg[q.va] = 1.0;
            Ng[q.ax] = q.side ? -1.0 : 1.0;
            for (int d = 0; d < 3; ++d) {
                const double *e = d == 0 ? f.t1 : (d == 1 ? f.t2 : f.n);
                q.Pl[d] = (Pg[0] - c[0]) * e[0] + (Pg[1] - c[1]) * e[1] + (Pg[2] - c[2]) * e[2];
                q.Ul[d] = Ug[0] * e[0] + Ug[1] * e[1] + Ug[2] * e[2];
                q.Vl[d] = Vg[0] * e[0] + Vg[1] * e[1] + Vg[2] * e[2];
                q.nl[d] = Ng[0] * e[0] + Ng[1] * e[1] + Ng[2] * e[2];
            }
            for (int j = 0; j < kMaxSub; ++j) q.cnt[j] = 0;
            q.centred = (q.P[0] == q.cf[0] && q.P[1] == q.cf[1]);
            for (int j = 0; j < q.nsub; ++j) {
                double sn, cn;
                sincos(q.svn[j], &sn, &cn);
                for (int d = 0; d < 3; ++d) {
                    q.en[j][d] = q.sdist[j] * (cn * q.Ul[d] + sn * q.Vl[d]);
                    q.et[j][d] = q.sdist[j] * (-sn * q.Ul[d] + cn * q.Vl[d]);
                }
            }
            pc[np++] = q;
        }
        f.npiece = np;
        // the sectors: one per sub-range of area at least area(S) / (nr^2 ns)
        // (smaller ones, below the layout's resolution, get none and are left
        // out of S), the rest by the largest area per sector
        const int ns = nsec[p], nrg = nring[p];
        double area[kMaxPieces][kMaxSub], As = 0.0;
        for (int k = 0; k < np; ++k)
            for (int j = 0; j < pc[k].nsub; ++j) {
                area[k][j] = 0.5 * rho2_integral(pc[k], pc[k].sub[j], pc[k].sub[j + 1], glx, glw);
                As += area[k][j];
            }
        const double thr = As / ((double)nrg * nrg * ns);
        int used = 0, fk = -1, fj = -1;
        for (int k = 0; k < np; ++k)
            for (int j = 0; j < pc[k].nsub; ++j) {
                pc[k].cnt[j] = area[k][j] >= thr ? 1 : 0;
                used += pc[k].cnt[j];
                if (pc[k].cnt[j] && fk < 0) { fk = k; fj = j; }
            }
        if (ns < used || fk < 0) {
            f.status = DTN_E_UNSUPPORTED;
        } else {
            for (int extra = ns - used; extra > 0; --extra) {
                int bk = fk, bj = fj;
                for (int k = 0; k < np; ++k)
                    for (int j = 0; j < pc[k].nsub; ++j)
                        if (pc[k].cnt[j] && (k > fk || (k == fk && j > fj)) &&
                            area[k][j] / pc[k].cnt[j] > area[bk][bj] / pc[bk].cnt[bj] * (1.0 + 1e-12)) { bk = k; bj = j; }
                pc[bk].cnt[bj] += 1;
            }
        }
    }
    out[p] = f;
}

// Polar range of the hemisphere at azimuth ph on a wrapped patch: the arc
// c + a (sin th e - cos th n), e = cos ph t1 + sin ph t2, leaves the region
// where it enters the box.  For th in [pi/2, pi] it stays on the box's side of
// the face plane and moves monotonically toward c along each in-plane axis k:
// it is inside the box's k range once sin th <= s_k, s_k the distance from c
// to the box side in the direction of e_k over a |e_k|; so theta_max =
// pi - asin(min(1, s_k)).
__device__ double theta_max_wrapped(const PatchFrame &f, double ph) {
    double sp, cp;
    sincos(ph, &sp, &cp);
    double m = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double ek = cp * f.t1[k] + sp * f.t2[k];
        if (ek > 0.0) m = fmin(m, (f.bhi[k] - f.c[k]) / (f.a * ek));
        else if (ek < 0.0) m = fmin(m, (f.c[k] - f.blo[k]) / (f.a * -ek));
    }
    return kPi - asin(fmax(m, 0.0));
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
    // wrapped patches: the polar range of this azimuth
    const double tmax = (f.kind == kWrapped) ? theta_max_wrapped(f, kPi * (xj + 1.0)) : f.theta_max;
    const double th = 0.5 * tmax * (xi + 1.0);
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincospi(xj + 1.0, &sp, &cp);
    const double L[3] = {f.a * st * cp, f.a * st * sp, -f.a * ct};
    if (loc) { loc[3 * gidx] = L[0]; loc[3 * gidx + 1] = L[1]; loc[3 * gidx + 2] = L[2]; }
    if (xyz)
        for (int d = 0; d < 3; ++d) xyz[3 * gidx + d] = f.c[d] + L[0] * f.t1[d] + L[1] * f.t2[d] + L[2] * f.n[d];
    if (w) w[gidx] = wi * wj * 0.5 * tmax * kPi * f.a * f.a * st;
}

// Panels: ring r, sector s of the patch parameter box.  Collocation point:
// the area centroid of a disk panel, or the radial projection of the area
// centroid of a cap panel onto the sphere.
// the point of panel parameters (u, v) in the patch frame, any patch kind
__device__ __forceinline__ void frame_point(const PatchFrame &f, const Piece *pc, double u, double v, double *Y,
                                            double *nl, double &J) {
    if (f.kind == kWrapped) wrapped_point<double>(*pc, u, v, Y, nl, J);
    else patch_point<double>(f.kind, f.R, u, v, Y, nl, J);
}

// Wrapped patch: panel (ring r, sector s): the sector's sub-range by the
// pieces' sector counts, rings even in u = rho / rho_max, collocation at the
// parameter midpoint; area = (u1^2 - u0^2)/2 int rho_max^2 dv.
__device__ void wrapped_panel(const PatchFrame &f, const Piece *pieces, int nr, int r, int s, const double *glx,
                              const double *glw, int &piece, int &sub, double &u0, double &u1, double &v0, double &v1,
                              double &uc, double &vc, double &area) {
    int k = 0, j = 0, m = s;
    for (k = 0; k < f.npiece; ++k) {
        for (j = 0; j < pieces[k].nsub; ++j) {
            if (m < pieces[k].cnt[j]) break;
            m -= pieces[k].cnt[j];
        }
        if (j < pieces[k].nsub) break;
    }
    const Piece &q = pieces[k];
    const double a0 = q.sub[j], a1 = q.sub[j + 1];
    const int cnt = q.cnt[j];
    piece = k;
    sub = j;
    v0 = a0 + (a1 - a0) * m / cnt;
    v1 = a0 + (a1 - a0) * (m + 1) / cnt;
    vc = 0.5 * (v0 + v1);
    u0 = (double)r / nr;
    u1 = (double)(r + 1) / nr;
    uc = 0.5 * (u0 + u1);
    area = 0.5 * (u1 * u1 - u0 * u0) * rho2_integral(q, v0, v1, glx, glw);
}

__global__ void panels_kernel(DData dat, int64_t n_patches, int64_t total, const int64_t *__restrict__ off,
                              const int32_t *__restrict__ nr, const int32_t *__restrict__ ns,
                              const PatchFrame *__restrict__ frames, const Piece *__restrict__ pieces,
                              const double *__restrict__ glx, const double *__restrict__ glw,
                              double *__restrict__ colloc,
                              double *__restrict__ normals, double *__restrict__ areas,
                              double *__restrict__ loc, double *__restrict__ prm,
                              double *__restrict__ aux, double *__restrict__ gval, int32_t *__restrict__ ppiece) {
    const int64_t gidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gidx >= total) return;
    const int64_t p = find_group(off, n_patches, gidx);
    const int k = (int)(gidx - off[p]);
    const int r = k / ns[p], s = k % ns[p];
    const PatchFrame &f = frames[p];
    if (f.kind == kWrapped) {
        const Piece *pcs = pieces + p * kMaxPieces;
        int piece = 0, sub = 0;
        double u0 = 0.0, u1 = 1.0, v0 = 0.0, v1 = 1.0, uc = 0.5, vc = 0.5, area = 0.0;
        if (f.status == DTN_OK)
            wrapped_panel(f, pcs, nr[p], r, s, glx, glw, piece, sub, u0, u1, v0, v1, uc, vc, area);
        const Piece *pc = pcs + piece;
        // quadrature parameters: t = tan(v - svn) on a side-bounded sub-range
        double w0 = v0, w1 = v1, wc = vc;
        if (f.status == DTN_OK && pc->stype[sub]) {
            w0 = tan(v0 - pc->svn[sub]);
            w1 = tan(v1 - pc->svn[sub]);
            wc = tan(vc - pc->svn[sub]);
        }
        double Y[3] = {0.0, 0.0, 0.0}, nl[3] = {0.0, 0.0, 1.0}, J = 0.0;
        if (f.status == DTN_OK) wrapped_point_q<double>(*pc, sub, uc, wc, Y, nl, J);
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
        q[0] = u0; q[1] = u1; q[2] = w0; q[3] = w1; q[4] = uc; q[5] = wc;
        ppiece[gidx] = piece * kMaxSub + sub;
        double rad = 0.0;
        if (f.status == DTN_OK)
            for (int cu = 0; cu < 3; ++cu)
                for (int cv = 0; cv < 3; ++cv) {
                    double Yq[3], nq[3], Jq;
                    wrapped_point_q<double>(*pc, sub, u0 + 0.5 * cu * (u1 - u0), w0 + 0.5 * cv * (w1 - w0), Yq, nq,
                                            Jq);
                    rad = fmax(rad, sqrt((Yq[0] - Y[0]) * (Yq[0] - Y[0]) + (Yq[1] - Y[1]) * (Yq[1] - Y[1]) +
                                         (Yq[2] - Y[2]) * (Yq[2] - Y[2])));
                }
        aux[4 * gidx] = Y[0]; aux[4 * gidx + 1] = Y[1]; aux[4 * gidx + 2] = Y[2];
        aux[4 * gidx + 3] = rad;
        gval[gidx] = dirichlet_eval<double>(dat, x[0], x[1], x[2]);
        return;
    }
    if (ppiece) ppiece[gidx] = 0;
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

// frames only (no pieces: a wrapped patch is reported unsupported)
cudaError_t launch_patch_frames(const dtn_geometry *g, int64_t n, const double *centers, const double *radius,
                                PatchFrame *frames, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int T = 128;
    patch_frame_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(g->dg, n, centers, radius, frames, nullptr, nullptr,
                                                                 nullptr, gl_x_dev(), gl_w_dev());
    return cudaGetLastError();
}

cudaError_t launch_patch_setup(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                               const double *centers, double *gamma_xyz,
                               double *gamma_w, double *gamma_loc, double *colloc, double *normals,
                               double *areas, double *panel_loc, double *panel_prm, double *panel_aux,
                               double *panel_g, int32_t *panel_piece, cudaStream_t s) {
    const int T = 128;
    const int64_t n = L.n_patches;
    patch_frame_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(g->dg, n, centers, D.radius, D.frames, D.pieces,
                                                                 D.ns, D.nr, gl_x_dev(), gl_w_dev());
    if (L.gamma_total > 0)
        gamma_nodes_kernel<<<(unsigned)((L.gamma_total + T - 1) / T), T, 0, s>>>(
            n, L.gamma_total, D.gamma_off, D.nt, D.nph, D.frames, gl_x_dev(), gl_w_dev(), gamma_xyz,
            gamma_w, gamma_loc);
    if (L.panels_total > 0)
        panels_kernel<<<(unsigned)((L.panels_total + T - 1) / T), T, 0, s>>>(
            g->dd, n, L.panels_total, D.panel_off, D.nr, D.ns, D.frames, D.pieces, gl_x_dev(), gl_w_dev(), colloc,
            normals, areas, panel_loc, panel_prm, panel_aux, panel_g, panel_piece);
    return cudaGetLastError();
}

}  // namespace dtn
