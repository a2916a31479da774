// lu.cu -- collocation solve A q = b for every patch of a batch, one CTA per
// patch.  LU with partial pivoting (pivot = first row of largest |a|), the
// factors held in shared memory when they fit (rows padded by one element so
// column reads do not collide in banks) and in a global scratch otherwise.
//
// FP64 mode: FP64 factors, one solve.  Mixed mode: FP32 factors, then
// iterative refinement r = b - A q with A and q in FP64, q += LU^{-1} r, until
// |r|_inf <= tol |b|_inf or the sweep limit; the first-kind system of Eq. bw49
// is ill conditioned for large panel counts (Sec. 4), so the FP32 factors only
// precondition and the FP64 residual sets the accuracy.
#include <cmath>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kLuThreads = 256;

struct LuDev {
    const PatchFrame *frames;
    const int64_t *panel_off, *mat_off;
    const double *A, *b;
    double *q;
    void *scratch;         // global factor storage when not in shared memory
    int in_smem;
    int max_iters;
    double tol;
    int32_t *iters;
    double *resid;
    int32_t *status;
};

// block-wide argmax of |v| (first index on ties)
__device__ __forceinline__ void argmax_update(double &bv, int &bi, double v, int i) {
    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

template <typename F>
__device__ void lu_solve_vec(const F *M, int ld, int n, const int *piv, double *x, int lane) {
    // x holds the right side on entry and the solution on exit (warp 0 only)
    for (int k = 0; k < n; ++k) {
        const int pk = piv[k];
        if (pk != k) {
            if (lane == 0) { const double t = x[k]; x[k] = x[pk]; x[pk] = t; }
            __syncwarp();
        }
    }
    // forward: unit lower triangle, F arithmetic on F-rounded values
    for (int k = 0; k < n; ++k) {
        const F xk = (F)x[k];
        for (int i = k + 1 + lane; i < n; i += 32) x[i] = (double)((F)x[i] - M[(int64_t)i * ld + k] * xk);
        __syncwarp();
    }
    for (int k = n - 1; k >= 0; --k) {
        if (lane == 0) x[k] = (double)((F)x[k] / M[(int64_t)k * ld + k]);
        __syncwarp();
        const F xk = (F)x[k];
        for (int i = lane; i < k; i += 32) x[i] = (double)((F)x[i] - M[(int64_t)i * ld + k] * xk);
        __syncwarp();
    }
}

template <typename F>
__global__ void __launch_bounds__(kLuThreads) lu_kernel(LuDev P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t p = blockIdx.x;
    const int64_t off = P.panel_off[p];
    const int n = (int)(P.panel_off[p + 1] - off);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kLuThreads / 32;
    const int ld = n + 1;
    double *q = P.q + off;
    const double *b = P.b + off;
    const double *A = P.A + P.mat_off[p];
    if (P.frames[p].status != DTN_OK) {
        for (int i = tid; i < n; i += kLuThreads) q[i] = 0.0;
        if (tid == 0) {
            if (P.status) P.status[p] = P.frames[p].status;
            if (P.iters) P.iters[p] = 0;
            if (P.resid) P.resid[p] = 0.0;
        }
        return;
    }
    // shared layout: [vec x (n doubles)][vec r (n doubles)][piv (n ints)][red][factors?]
    double *x = (double *)smem;
    double *r = x + n;
    int *piv = (int *)(r + n);
    double *redv = (double *)(piv + ((n + 1) & ~1));
    int *redi = (int *)(redv + nw);
    F *M;
    if (P.in_smem) {
        size_t o = (size_t)(2 * n) * sizeof(double) + (size_t)((n + 1) & ~1) * sizeof(int) + nw * (sizeof(double) + sizeof(int));
        o = (o + 15) & ~(size_t)15;
        M = (F *)(smem + o);
    } else {
        M = (F *)P.scratch + (int64_t)(P.mat_off[p] + off) ;  // n*(n+1) per patch fits in mat_off + off
    }
    for (int64_t idx = tid; idx < (int64_t)n * n; idx += kLuThreads) {
        const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
        M[(int64_t)i * ld + j] = (F)A[idx];
    }
    __shared__ int singular;
    if (tid == 0) singular = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        double bv = -1.0;
        int bi = n;
        for (int i = k + tid; i < n; i += kLuThreads) argmax_update(bv, bi, fabs((double)M[(int64_t)i * ld + k]), i);
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            argmax_update(bv, bi, ov, oi);
        }
        if (lane == 0) { redv[warp] = bv; redi[warp] = bi; }
        __syncthreads();
        if (tid == 0) {
            double v = -1.0;
            int ii = n;
            for (int w = 0; w < nw; ++w) argmax_update(v, ii, redv[w], redi[w]);
            piv[k] = ii;
            if (!(v > 0.0)) singular = 1;
        }
        __syncthreads();
        if (singular) break;
        const int pk = piv[k];
        if (pk != k)
            for (int j = tid; j < n; j += kLuThreads) {
                const F t = M[(int64_t)k * ld + j];
                M[(int64_t)k * ld + j] = M[(int64_t)pk * ld + j];
                M[(int64_t)pk * ld + j] = t;
            }
        __syncthreads();
        const F inv = (F)1 / M[(int64_t)k * ld + k];
        for (int i = k + 1 + tid; i < n; i += kLuThreads) M[(int64_t)i * ld + k] *= inv;
        __syncthreads();
        for (int i = k + 1 + warp; i < n; i += nw) {
            const F l = M[(int64_t)i * ld + k];
            for (int j = k + 1 + lane; j < n; j += 32) M[(int64_t)i * ld + j] -= l * M[(int64_t)k * ld + j];
        }
        __syncthreads();
    }
    if (singular) {
        for (int i = tid; i < n; i += kLuThreads) q[i] = 0.0;
        if (tid == 0) {
            if (P.status) P.status[p] = DTN_E_NOT_CONVERGED;
            if (P.iters) P.iters[p] = 0;
            if (P.resid) P.resid[p] = INFINITY;
        }
        return;
    }
    // q = LU^{-1} b
    for (int i = tid; i < n; i += kLuThreads) { x[i] = b[i]; r[i] = 0.0; }
    __syncthreads();
    if (warp == 0) lu_solve_vec<F>(M, ld, n, piv, x, lane);
    __syncthreads();
    // residual sweeps
    __shared__ double s_rn, s_bn;
    int it = 0;
    for (;; ++it) {
        // r = b - A x (FP64), one warp per row
        for (int i = warp; i < n; i += nw) {
            double s = 0.0;
            for (int j = lane; j < n; j += 32) s += A[(int64_t)i * n + j] * x[j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) r[i] = b[i] - s;
        }
        __syncthreads();
        if (tid == 0) {
            double rn = 0.0, bn = 0.0;
            for (int i = 0; i < n; ++i) { rn = fmax(rn, fabs(r[i])); bn = fmax(bn, fabs(b[i])); }
            s_rn = rn; s_bn = bn;
        }
        __syncthreads();
        const double rn = s_rn, bn = s_bn;
        if (rn <= P.tol * bn || it >= P.max_iters) break;
        if (warp == 0) lu_solve_vec<F>(M, ld, n, piv, r, lane);
        __syncthreads();
        for (int i = tid; i < n; i += kLuThreads) x[i] += r[i];
        __syncthreads();
    }
    for (int i = tid; i < n; i += kLuThreads) q[i] = x[i];
    if (tid == 0) {
        const double rel = s_bn > 0.0 ? s_rn / s_bn : 0.0;
        if (P.iters) P.iters[p] = it;
        if (P.resid) P.resid[p] = rel;
        if (P.status) P.status[p] = (rel <= P.tol || P.max_iters == 0) ? DTN_OK : DTN_E_NOT_CONVERGED;
    }
}

size_t lu_head_bytes(int n) {
    const int nw = kLuThreads / 32;
    size_t head = (size_t)(2 * n) * sizeof(double) + (size_t)((n + 1) & ~1) * sizeof(int) + nw * (sizeof(double) + sizeof(int));
    return (head + 15) & ~(size_t)15;
}

constexpr size_t kLuSmemLimit = 220 * 1024;

}  // namespace

size_t lu_scratch_bytes(const BatchLayout &L, int prec) {
    const int n = L.max_panels;
    const size_t fsz = prec == DTN_PREC_MIXED ? sizeof(float) : sizeof(double);
    if (lu_head_bytes(n) + (size_t)n * (n + 1) * fsz <= kLuSmemLimit) return 0;
    return (size_t)(L.matrix_total + L.panels_total) * fsz;
}

cudaError_t launch_lu_solve(dtn_geometry *g, const BatchLayout &L, const DevLayout &D, int prec,
                            const double *A, const double *b, double *q, int max_iters, double tol,
                            int32_t *iters, double *resid, int32_t *status, cudaStream_t s) {
    if (L.n_patches == 0) return cudaSuccess;
    cudaError_t e;
    const int n = L.max_panels;
    const bool fp32 = (prec == DTN_PREC_MIXED);
    const size_t fsz = fp32 ? sizeof(float) : sizeof(double);
    const size_t head = lu_head_bytes(n);
    const size_t fac = (size_t)n * (n + 1) * fsz;
    const size_t limit = kLuSmemLimit;
    LuDev P;
    P.frames = D.frames;
    P.panel_off = D.panel_off;
    P.mat_off = D.mat_off;
    P.A = A;
    P.b = b;
    P.q = q;
    P.max_iters = fp32 ? max_iters : 0;
    P.tol = tol;
    P.iters = iters;
    P.resid = resid;
    P.status = status;
    size_t smem = head;
    if (head + fac <= limit) {
        P.in_smem = 1;
        P.scratch = nullptr;
        smem = head + fac;
    } else {
        P.in_smem = 0;
        // factor storage n*(n+1) per patch: offsets mat_off[p] + panel_off[p] cover it
        DevBuf &buf = fp32 ? g->ws.lu32 : g->ws.lu64;
        if ((e = buf.reserve(lu_scratch_bytes(L, prec))) != cudaSuccess) return e;
        P.scratch = buf.p;
    }
    void *fn = fp32 ? (void *)lu_kernel<float> : (void *)lu_kernel<double>;
    if (smem > 48 * 1024)
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
    void *args[] = {&P};
    return cudaLaunchKernel(fn, dim3((unsigned)L.n_patches), dim3(kLuThreads), args, smem, s);
}

}  // namespace dtn
