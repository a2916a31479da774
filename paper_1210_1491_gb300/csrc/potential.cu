// potential.cu -- integral representation Eq. bw03 with the free-space Green's
// function Eq. bw05, panel-midpoint rule:
//   u(t) = sum_p [ aq_p / |t - y_p| - ag_p n_p.(t - y_p) / |t - y_p|^3 ],
//   aq_p = area_p q_p / 4pi,  ag_p = area_p g_p / 4pi,
// and the panel gather of the overlapping-patch cover (Sec. 6).
//
// N-body layout: a CTA stages tiles of panels in shared memory and each thread
// sums one target over the tile.  Mixed precision keeps panel positions as
// FP32 offsets from an FP64 tile origin (so differences of nearby points keep
// their digits whatever the coordinates' magnitude), evaluates pair terms in
// FP32, sums a tile in FP32 and adds tile sums in FP64.
#include <algorithm>
#include <cmath>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kPotThreads = 256;
constexpr int kTile = 256;

__global__ void __launch_bounds__(kPotThreads) potential_mixed_kernel(
    int64_t np_host, const int64_t *__restrict__ index, const int64_t *__restrict__ n_index,
    const double *__restrict__ xyz, const double *__restrict__ nrm,
    const double *__restrict__ area, const double *__restrict__ q, const double *__restrict__ g,
    int64_t nt, const double *__restrict__ t, double *__restrict__ out) {
    // a panel as two float4 (offset from the tile origin with area q / 4pi, normal
    // with area g / 4pi): two shared-memory loads per pair term
    __shared__ float4 s_pa[kTile], s_pb[kTile];
    __shared__ double s_org[3];
    const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = it < nt;
    const double tx = valid ? t[3 * it] : 0.0, ty = valid ? t[3 * it + 1] : 0.0, tz = valid ? t[3 * it + 2] : 0.0;
    double acc = 0.0;
    const float inv4pi = (float)(0.25 / kPi);
    // split y of gridDim.y takes tiles [y0, y1) of the panel list
    const int64_t np = n_index ? *n_index : np_host;
    const int64_t ntiles = (np + kTile - 1) / kTile, per = (ntiles + gridDim.y - 1) / gridDim.y;
    const int64_t pend = min(np, (blockIdx.y + 1) * per * kTile);
    for (int64_t base = blockIdx.y * per * kTile; base < pend; base += kTile) {
        const int cnt = (int)min((int64_t)kTile, pend - base);
        __syncthreads();
        if (threadIdx.x == 0) {
            const int64_t p0 = index ? index[base] : base;
            s_org[0] = xyz[3 * p0]; s_org[1] = xyz[3 * p0 + 1]; s_org[2] = xyz[3 * p0 + 2];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int64_t pp = index ? index[base + k] : base + k;
            s_pa[k] = make_float4((float)(xyz[3 * pp] - s_org[0]), (float)(xyz[3 * pp + 1] - s_org[1]),
                                  (float)(xyz[3 * pp + 2] - s_org[2]), (float)(area[pp] * q[pp]) * inv4pi);
            s_pb[k] = make_float4((float)nrm[3 * pp], (float)nrm[3 * pp + 1], (float)nrm[3 * pp + 2],
                                  (float)(area[pp] * g[pp]) * inv4pi);
        }
        __syncthreads();
        const float ox = (float)(tx - s_org[0]), oy = (float)(ty - s_org[1]), oz = (float)(tz - s_org[2]);
        float s = 0.0f;
#pragma unroll 4
        for (int k = 0; k < cnt; ++k) {
            const float4 pa = s_pa[k], pb = s_pb[k];
            const float dx = ox - pa.x, dy = oy - pa.y, dz = oz - pa.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrtf(r2);
            const float dn = fmaf(dx, pb.x, fmaf(dy, pb.y, dz * pb.z));
            s += ri * fmaf(-pb.w * dn, ri * ri, pa.w);
        }
        acc += (double)s;
    }
    if (valid) out[blockIdx.y * nt + it] = acc;
}

__global__ void __launch_bounds__(kPotThreads) potential_fp64_kernel(
    int64_t np_host, const int64_t *__restrict__ index, const int64_t *__restrict__ n_index,
    const double *__restrict__ xyz, const double *__restrict__ nrm,
    const double *__restrict__ area, const double *__restrict__ q, const double *__restrict__ g,
    int64_t nt, const double *__restrict__ t, double *__restrict__ out) {
    __shared__ double sx[kTile], sy[kTile], sz[kTile], snx[kTile], sny[kTile], snz[kTile], saq[kTile], sag[kTile];
    const int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = it < nt;
    const double tx = valid ? t[3 * it] : 0.0, ty = valid ? t[3 * it + 1] : 0.0, tz = valid ? t[3 * it + 2] : 0.0;
    double acc = 0.0;
    const double inv4pi = 0.25 / kPi;
    const int64_t np = n_index ? *n_index : np_host;
    const int64_t ntiles = (np + kTile - 1) / kTile, per = (ntiles + gridDim.y - 1) / gridDim.y;
    const int64_t pend = min(np, (blockIdx.y + 1) * per * kTile);
    for (int64_t base = blockIdx.y * per * kTile; base < pend; base += kTile) {
        const int cnt = (int)min((int64_t)kTile, pend - base);
        __syncthreads();
        for (int k = threadIdx.x; k < cnt; k += blockDim.x) {
            const int64_t pp = index ? index[base + k] : base + k;
            sx[k] = xyz[3 * pp]; sy[k] = xyz[3 * pp + 1]; sz[k] = xyz[3 * pp + 2];
            snx[k] = nrm[3 * pp]; sny[k] = nrm[3 * pp + 1]; snz[k] = nrm[3 * pp + 2];
            saq[k] = area[pp] * q[pp] * inv4pi;
            sag[k] = area[pp] * g[pp] * inv4pi;
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const double dx = tx - sx[k], dy = ty - sy[k], dz = tz - sz[k];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double r = sqrt(r2);
            const double dn = dx * snx[k] + dy * sny[k] + dz * snz[k];
            acc += saq[k] / r - sag[k] * dn / (r2 * r);
        }
    }
    if (valid) out[blockIdx.y * nt + it] = acc;
}

// out[i] = sum over the splits of part[y nt + i], in split order
__global__ void potential_reduce_kernel(int64_t nt, int ns, const double *__restrict__ part, double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double s = 0.0;
    for (int y = 0; y < ns; ++y) s += part[y * nt + i];
    out[i] = s;
}

// ---------------------------------------------------------------- panel gather

constexpr int kGatherThreads = 256;

__global__ void __launch_bounds__(kGatherThreads) owner_kernel(int64_t np, const double *__restrict__ x,
                                                             const int64_t *__restrict__ owner, int64_t nc,
                                                             const double *__restrict__ cent,
                                                             uint8_t *__restrict__ keep) {
    // Two passes over the centres (staged in shared memory): the FP32 minimum of
    // the squared distances, then the FP64 decision (lowest index on ties) among
    // the centres whose FP32 squared distance is within twice the FP32 error
    // bound of that minimum, so the FP64 minimum is always a candidate.  Bound:
    // each FP32 difference is off by at most dl = 4 u M (u = 2^-24, M the size
    // of the coordinates involved), so a squared distance d^2 by at most
    // 2 sqrt(3) d dl + 3 dl^2 + 4 u d^2.
    __shared__ double sc[3 * kGatherThreads];
    __shared__ float sf[3 * kGatherThreads];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = i < np;
    const double px = valid ? x[3 * i] : 0.0, py = valid ? x[3 * i + 1] : 0.0, pz = valid ? x[3 * i + 2] : 0.0;
    const float fx = (float)px, fy = (float)py, fz = (float)pz;
    float fbest = INFINITY;
    for (int64_t base = 0; base < nc; base += kGatherThreads) {
        const int cnt = (int)min((int64_t)kGatherThreads, nc - base);
        __syncthreads();
        for (int k = threadIdx.x; k < 3 * cnt; k += blockDim.x) sf[k] = (float)cent[3 * base + k];
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const float dx = fx - sf[3 * k], dy = fy - sf[3 * k + 1], dz = fz - sf[3 * k + 2];
            fbest = fminf(fbest, dx * dx + dy * dy + dz * dz);
        }
    }
    const float D = sqrtf(fbest);
    const float M = fmaxf(fmaxf(fabsf(fx), fabsf(fy)), fabsf(fz)) + 2.0f * D;
    const float dl = 4.0f * 0x1p-24f * M;
    const float thr = fbest + 2.0f * (3.5f * D * dl + 3.0f * dl * dl + 4.0f * 0x1p-24f * fbest) + 1e-30f;
    double best = INFINITY;
    int64_t bi = -1;
    for (int64_t base = 0; base < nc; base += kGatherThreads) {
        const int cnt = (int)min((int64_t)kGatherThreads, nc - base);
        __syncthreads();
        for (int k = threadIdx.x; k < 3 * cnt; k += blockDim.x) {
            const double c = cent[3 * base + k];
            sc[k] = c;
            sf[k] = (float)c;
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const float dx = fx - sf[3 * k], dy = fy - sf[3 * k + 1], dz = fz - sf[3 * k + 2];
            if (dx * dx + dy * dy + dz * dz <= thr) {
                const double ex = px - sc[3 * k], ey = py - sc[3 * k + 1], ez = pz - sc[3 * k + 2];
                const double d2 = ex * ex + ey * ey + ez * ez;
                if (d2 < best) { best = d2; bi = base + k; }
            }
        }
    }
    if (valid) keep[i] = (bi == owner[i]) ? 1 : 0;
}

__global__ void block_count_kernel(int64_t n, const uint8_t *__restrict__ keep, int64_t *__restrict__ bsum) {
    __shared__ int64_t red[kGatherThreads / 32];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int v = (i < n) ? keep[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int k = 0; k < kGatherThreads / 32; ++k) s += red[k];
        bsum[blockIdx.x] = s;
    }
}

// exclusive scan of block counts (one CTA, sequential over chunks of 1024)
__global__ void scan_blocks_kernel(int64_t nb, int64_t *__restrict__ bsum, int64_t *__restrict__ total) {
    __shared__ int64_t carry;
    __shared__ int64_t buf[1024];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += 1024) {
        const int64_t i = base + threadIdx.x;
        buf[threadIdx.x] = (i < nb) ? bsum[i] : 0;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t v = (threadIdx.x >= o) ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += v;
            __syncthreads();
        }
        const int64_t incl = buf[threadIdx.x];
        const int64_t excl = incl - ((i < nb) ? bsum[i] : 0);
        __syncthreads();
        if (i < nb) bsum[i] = carry + excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void scatter_kernel(int64_t n, const uint8_t *__restrict__ keep, const int64_t *__restrict__ boff,
                               int64_t *__restrict__ kept) {
    __shared__ int wsum[kGatherThreads / 32];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int v = (i < n) ? keep[i] : 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned m = __ballot_sync(0xffffffffu, v);
    const int before = __popc(m & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int wb = 0;
    for (int k = 0; k < w; ++k) wb += wsum[k];
    if (v) kept[boff[blockIdx.x] + wb + before] = i;
}

}  // namespace

cudaError_t launch_potential(int64_t np, const int64_t *index, const int64_t *n_index, const double *xyz,
                             const double *nrm, const double *area, const double *q, const double *g, int64_t nt,
                             const double *t, double *out, int prec, int num_sms, cudaStream_t s) {
    if (nt == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((nt + kPotThreads - 1) / kPotThreads);
    // split the panel list across CTAs when the targets alone fill less than the
    // GPU (8 resident CTAs of 256 threads per SM); partial sums reduced in split order
    const int64_t want = (int64_t)num_sms * 8;
    int ns = (int)std::min<int64_t>(8, std::max<int64_t>(1, want / std::max<unsigned>(blocks, 1u)));
    ns = (int)std::min<int64_t>(ns, std::max<int64_t>(1, (np + kTile - 1) / kTile));
    double *part = out;
    cudaError_t e;
    if (ns > 1 && (e = cudaMallocAsync((void **)&part, (size_t)ns * nt * sizeof(double), s)) != cudaSuccess)
        return e;
    const dim3 grid(blocks, (unsigned)ns);
    if (prec == DTN_PREC_MIXED)
        potential_mixed_kernel<<<grid, kPotThreads, 0, s>>>(np, index, n_index, xyz, nrm, area, q, g, nt, t, part);
    else
        potential_fp64_kernel<<<grid, kPotThreads, 0, s>>>(np, index, n_index, xyz, nrm, area, q, g, nt, t, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ns > 1) {
        potential_reduce_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(nt, ns, part, out);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = cudaFreeAsync(part, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_gather(int64_t np, const double *x, const int64_t *owner, int64_t nc, const double *cent,
                          uint8_t *keep, int64_t *kept, int64_t *n_kept, cudaStream_t s) {
    if (np == 0) return cudaMemsetAsync(n_kept, 0, sizeof(int64_t), s);
    const int64_t nb = (np + kGatherThreads - 1) / kGatherThreads;
    int64_t *bsum = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&bsum, nb * sizeof(int64_t), s);
    if (e != cudaSuccess) return e;
    owner_kernel<<<(unsigned)nb, kGatherThreads, 0, s>>>(np, x, owner, nc, cent, keep);
    block_count_kernel<<<(unsigned)nb, kGatherThreads, 0, s>>>(np, keep, bsum);
    scan_blocks_kernel<<<1, 1024, 0, s>>>(nb, bsum, n_kept);
    scatter_kernel<<<(unsigned)nb, kGatherThreads, 0, s>>>(np, keep, bsum, kept);
    e = cudaGetLastError();
    cudaFreeAsync(bsum, s);
    return e;
}

}  // namespace dtn
