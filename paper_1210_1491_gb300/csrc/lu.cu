// lu.cu -- collocation solve A q = b (Eq. bw49 discretised).  LU with partial
// pivoting (pivot = first row of largest |a|); factors held in shared memory
// when they fit (rows padded by one element so column reads do not collide in
// banks) and in a global scratch otherwise.
//
// FP64 path: one CTA per patch factors the patch's own FP64 matrix and solves.
// Shared path (mixed precision): the matrix of Eq. bw50 depends only on the
// patch shape, so one CTA per shape group computes FP32 factors of the group's
// FP64 matrix, then one CTA per patch solves with those factors and refines
// r = b - A q with A and q in FP64 until |r|_inf <= tol |b|_inf or the sweep
// limit.  The first-kind system is ill conditioned for large panel counts
// (Sec. 4), so the FP32 factors only precondition and the FP64 residual sets
// the accuracy.
#include <cmath>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kLuThreads = 256;
constexpr int kNw = kLuThreads / 32;
constexpr size_t kLuSmemLimit = 220 * 1024;

__host__ __device__ inline size_t lu_head_bytes(int n) {
    size_t head = (size_t)(2 * n) * sizeof(double) + (size_t)((n + 1) & ~1) * sizeof(int) + kNw * (sizeof(double) + sizeof(int));
    return (head + 15) & ~(size_t)15;
}

// block-wide argmax of |v| (first index on ties)
__device__ __forceinline__ void argmax_update(double &bv, int &bi, double v, int i) {
    if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

// In-place LU with partial pivoting of the n x n matrix M (leading dimension
// ld), all threads of the CTA.  piv[k] = row swapped with row k.  Returns
// nonzero if a pivot column is exactly zero.
template <typename F>
__device__ int lu_factor(F *M, int ld, int n, int *piv, double *redv, int *redi) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
            for (int w = 0; w < kNw; ++w) argmax_update(v, ii, redv[w], redi[w]);
            piv[k] = ii;
            if (!(v > 0.0)) singular = 1;
        }
        __syncthreads();
        if (singular) return 1;
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
        for (int i = k + 1 + warp; i < n; i += kNw) {
            const F l = M[(int64_t)i * ld + k];
            for (int j = k + 1 + lane; j < n; j += 32) M[(int64_t)i * ld + j] -= l * M[(int64_t)k * ld + j];
        }
        __syncthreads();
    }
    return 0;
}

// x <- (LU)^{-1} P x with F arithmetic (one warp)
template <typename F>
__device__ void lu_solve_vec(const F *M, int ld, int n, const int *piv, double *x, int lane) {
    for (int k = 0; k < n; ++k) {
        const int pk = piv[k];
        if (pk != k) {
            if (lane == 0) { const double t = x[k]; x[k] = x[pk]; x[pk] = t; }
            __syncwarp();
        }
    }
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

// Solve with factors M, then refine against the FP64 matrix A (n x n, row-major).
template <typename F>
__device__ void solve_refine(const F *M, int ld, int n, const int *piv, const double *A, const double *b, double *q,
                             double *x, double *r, int max_iters, double tol, int32_t *iters, double *resid,
                             int32_t *status) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < n; i += kLuThreads) { x[i] = b[i]; r[i] = 0.0; }
    __syncthreads();
    if (warp == 0) lu_solve_vec<F>(M, ld, n, piv, x, lane);
    __syncthreads();
    __shared__ double s_rn, s_bn;
    int it = 0;
    for (;; ++it) {
        for (int i = warp; i < n; i += kNw) {
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
        if (rn <= tol * bn || it >= max_iters) break;
        if (warp == 0) lu_solve_vec<F>(M, ld, n, piv, r, lane);
        __syncthreads();
        for (int i = tid; i < n; i += kLuThreads) x[i] += r[i];
        __syncthreads();
    }
    for (int i = tid; i < n; i += kLuThreads) q[i] = x[i];
    if (tid == 0) {
        const double rel = s_bn > 0.0 ? s_rn / s_bn : 0.0;
        if (iters) *iters = it;
        if (resid) *resid = rel;
        if (status) *status = (rel <= tol || max_iters == 0) ? DTN_OK : DTN_E_NOT_CONVERGED;
    }
}

__device__ void fail_patch(int n, double *q, int32_t *iters, double *resid, int32_t *status, int code, double res) {
    for (int i = threadIdx.x; i < n; i += kLuThreads) q[i] = 0.0;
    if (threadIdx.x == 0) {
        if (status) *status = code;
        if (iters) *iters = 0;
        if (resid) *resid = res;
    }
}

struct LuDev {
    const PatchFrame *frames;
    const int64_t *panel_off, *mat_off;
    const int64_t *group_of, *grows_off, *gmat_off, *gfac_off;
    const double *A, *b;
    double *q;
    void *scratch;     // factor storage (per patch, or per group on the shared path)
    int *piv;          // shared path: pivots, n per group at grows_off
    int in_smem;
    int max_iters;
    double tol;
    int32_t *iters;
    double *resid;
    int32_t *status;
};

// FP64 path: factor and solve one patch per CTA
template <typename F>
__global__ void __launch_bounds__(kLuThreads) lu_kernel(LuDev P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t p = blockIdx.x;
    const int64_t off = P.panel_off[p];
    const int n = (int)(P.panel_off[p + 1] - off);
    const int ld = n + 1;
    double *q = P.q + off;
    int32_t *it = P.iters ? P.iters + p : nullptr, *st = P.status ? P.status + p : nullptr;
    double *rs = P.resid ? P.resid + p : nullptr;
    if (P.frames[p].status != DTN_OK) {
        fail_patch(n, q, it, rs, st, P.frames[p].status, 0.0);
        return;
    }
    double *x = (double *)smem, *r = x + n;
    int *piv = (int *)(r + n);
    double *redv = (double *)(piv + ((n + 1) & ~1));
    int *redi = (int *)(redv + kNw);
    F *M = P.in_smem ? (F *)(smem + lu_head_bytes(n)) : (F *)P.scratch + (P.mat_off[p] + off);
    const double *A = P.A + P.mat_off[p];
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += kLuThreads) {
        const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
        M[(int64_t)i * ld + j] = (F)A[idx];
    }
    __syncthreads();
    if (lu_factor<F>(M, ld, n, piv, redv, redi)) {
        fail_patch(n, q, it, rs, st, DTN_E_NOT_CONVERGED, INFINITY);
        return;
    }
    solve_refine<F>(M, ld, n, piv, A, P.b + off, q, x, r, P.max_iters, P.tol, it, rs, st);
}

// shared path, step 1: FP32 factors of each group matrix (one CTA per group)
__global__ void __launch_bounds__(kLuThreads) lu_group_factor_kernel(LuDev P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t grp = blockIdx.x;
    const int n = (int)(P.grows_off[grp + 1] - P.grows_off[grp]);
    const int ld = n + 1;
    int *piv_s = (int *)smem;
    double *redv = (double *)(piv_s + ((n + 1) & ~1));
    int *redi = (int *)(redv + kNw);
    float *G = (float *)P.scratch + P.gfac_off[grp];
    float *M = P.in_smem ? (float *)(smem + lu_head_bytes(n)) : G;
    const double *A = P.A + P.gmat_off[grp];
    for (int64_t idx = threadIdx.x; idx < (int64_t)n * n; idx += kLuThreads) {
        const int i = (int)(idx / n), j = (int)(idx - (int64_t)i * n);
        M[(int64_t)i * ld + j] = (float)A[idx];
    }
    __syncthreads();
    const int bad = lu_factor<float>(M, ld, n, piv_s, redv, redi);
    __syncthreads();
    int *piv = P.piv + P.grows_off[grp];
    for (int k = threadIdx.x; k < n; k += kLuThreads) piv[k] = bad ? -1 : piv_s[k];
    if (P.in_smem)
        for (int64_t idx = threadIdx.x; idx < (int64_t)n * ld; idx += kLuThreads) G[idx] = M[idx];
}

// shared path, step 2: one CTA per patch solves with its group's factors
__global__ void __launch_bounds__(kLuThreads) lu_group_solve_kernel(LuDev P) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t p = blockIdx.x;
    const int64_t off = P.panel_off[p];
    const int n = (int)(P.panel_off[p + 1] - off);
    const int ld = n + 1;
    const int64_t grp = P.group_of[p];
    double *q = P.q + off;
    int32_t *it = P.iters ? P.iters + p : nullptr, *st = P.status ? P.status + p : nullptr;
    double *rs = P.resid ? P.resid + p : nullptr;
    if (P.frames[p].status != DTN_OK) {
        fail_patch(n, q, it, rs, st, P.frames[p].status, 0.0);
        return;
    }
    double *x = (double *)smem, *r = x + n;
    int *piv = (int *)(r + n);
    const int *gp = P.piv + P.grows_off[grp];
    for (int k = threadIdx.x; k < n; k += kLuThreads) piv[k] = gp[k];
    const float *G = (const float *)P.scratch + P.gfac_off[grp];
    const float *M = G;
    if (P.in_smem) {
        float *Ms = (float *)(smem + lu_head_bytes(n));
        for (int64_t idx = threadIdx.x; idx < (int64_t)n * ld; idx += kLuThreads) Ms[idx] = G[idx];
        M = Ms;
    }
    __syncthreads();
    if (piv[0] < 0) {
        fail_patch(n, q, it, rs, st, DTN_E_NOT_CONVERGED, INFINITY);
        return;
    }
    solve_refine<float>(M, ld, n, piv, P.A + P.gmat_off[grp], P.b + off, q, x, r, P.max_iters, P.tol, it, rs, st);
}

}  // namespace

size_t lu_scratch_bytes(const BatchLayout &L, int prec) {
    const int n = L.max_panels;
    const size_t fsz = prec == DTN_PREC_MIXED ? sizeof(float) : sizeof(double);
    if (lu_head_bytes(n) + (size_t)n * (n + 1) * fsz <= kLuSmemLimit) return 0;
    return (size_t)(L.matrix_total + L.panels_total) * fsz;
}

size_t lu_shared_scratch_bytes(const BatchLayout &L) { return (size_t)L.gfac_total * sizeof(float) + 64; }

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
    LuDev P{};
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
    if (head + fac <= kLuSmemLimit) {
        P.in_smem = 1;
        smem = head + fac;
    } else {
        DevBuf &buf = fp32 ? g->ws.lu32 : g->ws.lu64;
        if ((e = buf.reserve(lu_scratch_bytes(L, prec), s)) != cudaSuccess) return e;
        P.scratch = buf.p;
    }
    void *fn = fp32 ? (void *)lu_kernel<float> : (void *)lu_kernel<double>;
    if (smem > 48 * 1024)
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
    void *args[] = {&P};
    return cudaLaunchKernel(fn, dim3((unsigned)L.n_patches), dim3(kLuThreads), args, smem, s);
}

cudaError_t launch_lu_shared(dtn_geometry *g, const BatchLayout &L, const DevLayout &D, const double *gA,
                             const double *b, double *q, int max_iters, double tol, int32_t *iters, double *resid,
                             int32_t *status, cudaStream_t s) {
    if (L.n_patches == 0) return cudaSuccess;
    cudaError_t e;
    const int n = L.max_panels;
    const size_t head = lu_head_bytes(n);
    const size_t fac = (size_t)n * (n + 1) * sizeof(float);
    LuDev P{};
    P.frames = D.frames;
    P.panel_off = D.panel_off;
    P.mat_off = D.mat_off;
    P.group_of = D.group_of;
    P.grows_off = D.grows_off;
    P.gmat_off = D.gmat_off;
    P.gfac_off = D.gfac_off;
    P.A = gA;
    P.b = b;
    P.q = q;
    P.scratch = g->ws.gfac.p;
    P.piv = g->ws.gpiv.as<int>();
    P.max_iters = max_iters;
    P.tol = tol;
    P.iters = iters;
    P.resid = resid;
    P.status = status;
    P.in_smem = (head + fac <= kLuSmemLimit) ? 1 : 0;
    const size_t smem = P.in_smem ? head + fac : head;
    const void *fns[2] = {(const void *)lu_group_factor_kernel, (const void *)lu_group_solve_kernel};
    if (smem > 48 * 1024)
        for (const void *fn : fns)
            if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
                return e;
    void *args[] = {&P};
    if ((e = cudaLaunchKernel(fns[0], dim3((unsigned)L.n_groups), dim3(kLuThreads), args, smem, s)) != cudaSuccess)
        return e;
    return cudaLaunchKernel(fns[1], dim3((unsigned)L.n_patches), dim3(kLuThreads), args, smem, s);
}

}  // namespace dtn
