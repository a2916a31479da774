// wos.cu -- walk on spheres (Sec. 2) with an epsilon shell, estimator Eq. bw87.
//
// Persistent kernel, one walk per lane.  Work is a list of chunks (a chunk =
// up to `chunk` consecutive walks of one node); a warp takes a chunk from a
// global counter and hands its walks to idle lanes, so a lane whose walk ends
// starts the next walk without waiting for the rest of the warp (compaction of
// finished walks).  A lane keeps walking while fewer than `refill` lanes of its
// warp are idle; then absorbed walks are scored together (their data are
// evaluated in one pass, not one divergent lane at a time) and idle lanes are
// refilled.
//
// Scores are accumulated as 64-bit fixed-point integers (score * 2^F) per warp
// and node, together with the number of walks scored; steps and escapes per
// lane and node; all flushed by integer atomics when the node changes, so sums
// do not depend on scheduling: the estimates are bitwise reproducible.  A
// node's walks cut at max_steps are those neither scored nor escaped.
//
// Random numbers: Philox4x32-10 keyed by the seed.  FP64 walks draw one block
// per jump, counter (walk, j, point, patch), 53-bit uniforms from words (0,1)
// and (2,3).  FP32 walks draw one block per three jumps, counter
// (walk, j / 3, point, patch): the block's six 21-bit fields (the top 21 bits
// of each word, then the low 11 bits of words 0 and 2 with the low 10 bits of
// words 1 and 3 above them) give the uniforms (2f + 1) 2^-22 of jump j % 3
// from fields (2 (j % 3), 2 (j % 3) + 1); each loop iteration of an FP32 walk
// makes three jumps from one block.
#include <cmath>
#include <type_traits>

#include "dtn_internal.h"

namespace dtn {

namespace {

constexpr int kWosThreads = 128;

struct WosDev {
    DGeom g;
    DData dat;
    const double *y;
    const int64_t *node_off;
    const int64_t *walks;
    const uint32_t *pid;
    const uint32_t *point_id;
    const int64_t *chunk_off;
    const int32_t *cpn;
    int64_t n_groups, total_chunks;
    int32_t chunk;
    int32_t refill;
    unsigned long long *counter;
    unsigned long long *s1, *s2, *st;
    unsigned int *done;    // per node: walks that ended by absorption or escape
    int lgM1, lgM2;        // ceil(log2) of the score bound and of its square
    double eps;
    float eps_f;           // eps rounded to FP32 on the host (FP32 walks)
    uint32_t max_steps;
    uint32_t blk_fast;     // FP32 walks: blocks of three jumps below this index cannot reach max_steps
    uint32_t rk0[10], rk1[10];   // Philox round keys from the seed
};

// the round keys of Philox4x32-10 for a 64-bit seed
inline void philox_round_keys(uint64_t seed, uint32_t *rk0, uint32_t *rk1) {
    uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFull), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk0[r] = k0;
        rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Fixed-point exponent of a node's sums: |sum over W walks| <= W * bound < 2^61,
// so F = 61 - ceil(log2 W) - ceil(log2 bound).  It depends only on the node's own
// walk count, never on the rest of the batch.
__host__ __device__ __forceinline__ int fixed_exponent(int64_t walks, int lgM) {
    int lw = 0;
    while (lw < 63 && ((int64_t)1 << lw) < walks) ++lw;
    int e = 61 - lw - lgM;
    return e < -1000 ? -1000 : (e > 1000 ? 1000 : e);
}

__device__ __forceinline__ double pow2(int e) {
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Per-lane step and escape counts of the node the lane works on, flushed with
// integer atomics when the lane moves to another node.  Absorbed walks are
// counted where they are scored; a node's walks cut at max_steps are the rest.
struct LaneAcc {
    int node = -1;   // node ids are 32-bit in the kernel
    unsigned long long st = 0;
    unsigned int esc = 0;

    __device__ __forceinline__ void flush(const WosDev &P) {
        if (node >= 0) {
            atomicAdd(P.st + node, st);
            if (esc) atomicAdd(P.done + node, esc);
        }
        st = 0;
        esc = 0;
    }
};

// Fixed-point score terms round(s 2^F1) and round(s^2 2^F2).  FP32 scores:
// s = M 2^e with the 24-bit significand M, so s 2^F and s^2 2^F = M^2 2^(2e+F)
// are formed exactly from integers (M, or M^2 < 2^48) and shifts, and round to
// the same integers as the FP64 products would (ties to even).  Integer only:
// conversions to or from 64-bit types would run on the FP64 pipe.
__device__ __forceinline__ long long fixed_term(float s, int F) {
    const uint32_t u = __float_as_uint(s), bits = u & 0x7fffffffu;
    const int E = (int)(bits >> 23);
    const uint32_t M = E ? ((bits & 0x7fffffu) | 0x800000u) : (bits & 0x7fffffu);   // < 2^24
    const int sh = (E ? E : 1) - 150 + F;
    // right shift by k with ties to even (k = 25 already leaves less than 1/2), or
    // left shift by l (M 2^l = |s| 2^F < 2^61 by the choice of F; the cap only
    // keeps the shift defined)
    const int k = min(max(-sh, 0), 25), l = min(max(sh, 0), 62);
    const uint32_t q = M >> k, rem = M & ((1u << k) - 1u), half = (1u << k) >> 1;
    const uint32_t up = (k > 0 && (rem > half || (rem == half && (q & 1u)))) ? 1u : 0u;
    const long long v = (long long)((unsigned long long)(q + up) << l);
    return (u >> 31) ? -v : v;
}
__device__ __forceinline__ long long fixed_term(double s, int F) { return __double2ll_rn(s * pow2(F)); }

__device__ __forceinline__ long long fixed_square(float s, int F) {
    const uint32_t bits = __float_as_uint(s) & 0x7fffffffu;
    const int E = (int)(bits >> 23);
    const unsigned long long M = E ? ((bits & 0x7fffffu) | 0x800000u) : (bits & 0x7fffffu);
    const unsigned long long M2 = M * M;   // < 2^48
    if (M2 == 0ull) return 0;
    const int sh = 2 * ((E ? E : 1) - 150) + F;
    if (sh >= 0) return (long long)(M2 << (sh < 15 ? sh : 15));   // < 2^61 by the choice of F
    const int k = -sh;
    if (k > 48) return 0;   // below 1/2
    const unsigned long long q = M2 >> k, rem = M2 & ((1ull << k) - 1ull), half = 1ull << (k - 1);
    return (long long)(q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull));
}
__device__ __forceinline__ long long fixed_square(double s, int F) { return __double2ll_rn(s * s * pow2(F)); }

// Data at a boundary point for the score: FP32 harmonic data by the solid
// harmonic recurrences with the coefficients staged in shared memory.
template <typename T>
__device__ __forceinline__ T walk_data(const DData &d, const float2 *cs, T x, T y, T z) {
    if constexpr (sizeof(T) == 4) {
        if (d.kind == kHarmonicSH) {
            const float is = d.inv_scale_f;
            const float xs = (x - d.ctr_f[0]) * is, ys = (y - d.ctr_f[1]) * is, zs = (z - d.ctr_f[2]) * is;
            if (d.lmax <= 4) return harmonic_cart_fixed<4>(cs, xs, ys, zs);
            if (d.lmax <= 8) return harmonic_cart_fixed<8>(cs, xs, ys, zs);
            return harmonic_cart(cs, d.lmax, xs, ys, zs);
        }
    }
    return dirichlet_eval<T>(d, x, y, z);
}

// Absorbed walks wait in a per-warp ring of absorption points until 32 are
// there; then every lane scores one (projection onto the boundary and the
// data), so the scoring never runs with idle lanes.
constexpr int kQueue = 64;
template <typename T>
struct ScoreQueue {
    T x[kQueue], y[kQueue], z[kQueue];
    int node[kQueue];
    short f1[kQueue], f2[kQueue];
};

// Warp-uniform running score sums of one node, flushed with atomics when a
// batch brings another node.
struct WarpScore {
    int node = -1;
    long long a1 = 0, a2 = 0;
    unsigned int n = 0;   // walks scored
};

template <typename T, int GK>
__device__ __forceinline__ void score_batch(const WosDev &P, const T *sb, const float2 *cs, ScoreQueue<T> &Q,
                                            int &qhead, int &qcount, int cnt, int lane, WarpScore &ws) {
    const unsigned FULL = 0xffffffffu;
    int node = -1;
    long long v1 = 0, v2 = 0;
    if (lane < cnt) {
        const int e = (qhead + lane) & (kQueue - 1);
        T nx, ny, nz;
        geo_nearest<T>(P.g, sb, Q.x[e], Q.y[e], Q.z[e], nx, ny, nz);
        const T sc = walk_data<T>(P.dat, cs, nx, ny, nz);
        node = Q.node[e];
        v1 = fixed_term(sc, (int)Q.f1[e]);
        v2 = fixed_square(sc, (int)Q.f2[e]);
    }
    __syncwarp();
    unsigned rem = __ballot_sync(FULL, lane < cnt);
    while (rem) {
        const int nd = __shfl_sync(FULL, node, __ffs(rem) - 1);
        const bool in = (lane < cnt) && node == nd;
        long long s1 = in ? v1 : 0, s2 = in ? v2 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(FULL, s1, o);
            s2 += __shfl_xor_sync(FULL, s2, o);
        }
        const unsigned inm = __ballot_sync(FULL, in);
        rem &= ~inm;
        if (nd != ws.node) {
            if (ws.node >= 0 && lane == 0) {
                atomicAdd(P.s1 + ws.node, (unsigned long long)ws.a1);
                atomicAdd(P.s2 + ws.node, (unsigned long long)ws.a2);
                atomicAdd(P.done + ws.node, ws.n);
            }
            ws.node = nd;
            ws.a1 = 0;
            ws.a2 = 0;
            ws.n = 0;
        }
        ws.a1 += s1;
        ws.a2 += s2;
        ws.n += __popc(inm);
    }
    qhead = (qhead + cnt) & (kQueue - 1);
    qcount -= cnt;
    __syncwarp();   // the slots just read may be written by the next pushes
}

// one jump of the walk from x by d in the direction drawn from uniforms (u1, u2):
// z uniform in (-1, 1), azimuth uniform over a full turn
// FP32 walks: uniforms u = (2f + 1) 2^-22 from 21-bit fields, held as v = 1 + u
// built in the significand (4f + 2 < 2^23: an integer add, no conversion);
// z = 1 - 2 u1 = 3 - 2 v1 exactly; the azimuth 2 pi (u2 - 1/2) = 2 pi v2 - 3 pi,
// in (-pi, pi) up to one rounding (a constant shift of the angle), by the SFU
// sine/cosine; s = sqrt(1 - z^2) by the SFU reciprocal square root
// (1 - z^2 >= 2^-20 > 0 for these uniforms).  d = 0 leaves x unchanged.
// The six 21-bit fields of one Philox block: the top 21 bits of each word, then
// the low 11 bits of words 0 and 2 with the low 10 bits of words 1 and 3 above
// them (126 of the block's 128 bits, each used once).
__device__ __forceinline__ void fields21(const uint4 &w, uint32_t f[6]) {
    f[0] = w.x >> 11;
    f[1] = w.y >> 11;
    f[2] = w.z >> 11;
    f[3] = w.w >> 11;
    f[4] = (w.x & 0x7ffu) | ((w.y & 0x3ffu) << 11);
    f[5] = (w.z & 0x7ffu) | ((w.w & 0x3ffu) << 11);
}

// v = 1 + u for the uniform u = (2f + 1) 2^-22 of a 21-bit field f: the
// significand of 1.0 plus 4f + 2 units of 2^-23 (exact, no conversion)
__device__ __forceinline__ float one_plus_u21(uint32_t f) { return __uint_as_float(0x3F800002u + 4u * f); }

// The pieces of the jump direction from two fields: z = 1 - 2 u1 = 3 - 2 v1
// (exact), s = sqrt(1 - z^2), and the sine and cosine of the azimuth
// 2 pi (u2 - 1/2) = 2 pi v2 - 3 pi
__device__ __forceinline__ void direction21(uint32_t f1, uint32_t f2, float &zz, float &s, float &sn, float &cs) {
    constexpr float kTwoPi = 6.2831853071795865f, kAz0 = 1.5f * kTwoPi;
    const float v1 = one_plus_u21(f1), v2 = one_plus_u21(f2);
    zz = fmaf(-2.0f, v1, 3.0f);
    const float t = fmaf(-zz, zz, 1.0f);   // 1 - z^2, one rounding
    s = t * rsqrtf(t);
    __sincosf(fmaf(kTwoPi, v2, -kAz0), &sn, &cs);
}

__device__ __forceinline__ void jump(float &x, float &y, float &z, float d, uint32_t f1, uint32_t f2) {
    float zz, s, sn, cs;
    direction21(f1, f2, zz, s, sn, cs);
    x = fmaf(d * s, cs, x);
    y = fmaf(d * s, sn, y);
    z = fmaf(d, zz, z);
}

__device__ __forceinline__ void jump(double &x, double &y, double &z, double d, uint4 w) {
    const double u1 = u01_53(w.x, w.y), u2 = u01_53(w.z, w.w);
    const double zz = 1.0 - 2.0 * u1;
    const double s = sqrt(fmax(0.0, 1.0 - zz * zz));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    x += d * s * cs;
    y += d * s * sn;
    z += d * zz;
}

// Ball regions, FP32, position relative to the centre: distance to the sphere
// and the escape test of the exterior region
template <int GK>
__device__ __forceinline__ float ball_dist_rel(const DGeom &g, float x, float y, float z) {
    // the 1e-30 keeps r2 > 0 at the centre (below half an ulp of any other r2)
    const float r2 = fmaf(x, x, fmaf(y, y, fmaf(z, z, 1e-30f)));
    const float r = r2 * rsqrtf(r2);   // SFU reciprocal square root: |x| to a few FP32 ulps
    return GK == kBall ? g.R_f - r : r - g.R_f;
}
__device__ __forceinline__ bool ball_escaped_rel(const DGeom &g, float x, float y, float z) {
    return x * x + y * y + z * z > g.trunc_f * g.trunc_f;
}

template <typename T, int GK>
__global__ void __launch_bounds__(kWosThreads, 7) wos_kernel(WosDev P) {
    extern __shared__ float s_boxes[];
    __shared__ ScoreQueue<T> s_queue[kWosThreads / 32];
    __shared__ float2 s_cs[kShPairs];
    const float *sb = nullptr;
    if (GK == kBoxMinusBoxes && std::is_same<T, float>::value && P.g.nb <= kMaxSmemBoxes) {
        for (int i = threadIdx.x; i < 6 * P.g.nb; i += blockDim.x) s_boxes[i] = P.g.boxes_f[i];
        sb = s_boxes;
    }
    if (std::is_same<T, float>::value && P.dat.kind == kHarmonicSH)
        for (int i = threadIdx.x; i < kShPairs; i += blockDim.x) s_cs[i] = P.dat.cart[i];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // FP32 walks take the host-rounded copy: a double-to-float conversion here
    // would run on the FP64 pipe, and the compiler may redo it inside the loop
    const T eps = pick<T>(P.eps, P.eps_f);
    ScoreQueue<T> &Q = s_queue[threadIdx.x >> 5];
    // FP32 walks in a ball region keep positions relative to the centre: the
    // distance then needs no subtraction; absorption points get the centre back
    // when they are queued for scoring
    constexpr bool kRel = std::is_same<T, float>::value && (GK == kBall || GK == kBallExterior);
    const T ox = kRel ? pick<T>(P.g.c[0], P.g.c_f[0]) : (T)0, oy = kRel ? pick<T>(P.g.c[1], P.g.c_f[1]) : (T)0,
            oz = kRel ? pick<T>(P.g.c[2], P.g.c_f[2]) : (T)0;
    int qhead = 0, qcount = 0;   // warp-uniform
    WarpScore ws;

    // warp-uniform chunk state
    int cnode = -1;
    uint32_t cnext = 0, cend = 0;   // walk indices of the node (at most 2^32 - 1 walks)
    uint32_t cpid = 0, cpt = 0;
    int cf1 = 0, cf2 = 0;          // fixed-point exponents of the node's sums
    T cx = 0, cy = 0, cz = 0;
    bool no_more = false;

    // lane state
    bool active = false, pending = false;
    T x = 0, y = 0, z = 0;
    uint32_t walk = 0, step = 0, ppid = 0, ppt = 0;
    int f1 = 0, f2 = 0;
    LaneAcc acc;

    for (;;) {
        // absorbed walks go to the queue with their absorption point; full
        // batches of 32 are scored at once
        const unsigned pm = __ballot_sync(FULL, pending);
        if (pm) {
            if (pending) {
                const int e = (qhead + qcount + __popc(pm & lt_mask)) & (kQueue - 1);
                Q.x[e] = x + ox;
                Q.y[e] = y + oy;
                Q.z[e] = z + oz;
                Q.node[e] = acc.node;
                Q.f1[e] = (short)f1;
                Q.f2[e] = (short)f2;
                pending = false;
            }
            qcount += __popc(pm);
            __syncwarp();
            if (qcount >= 32) score_batch<T, GK>(P, (const T *)sb, s_cs, Q, qhead, qcount, 32, lane, ws);
        }
        // hand out walks to idle lanes
        unsigned idle = __ballot_sync(FULL, !active);
        while (idle != 0u && !no_more) {
            if (cnext >= cend) {
                unsigned long long c = 0;
                if (lane == 0) c = atomicAdd(P.counter, 1ull);
                c = __shfl_sync(FULL, c, 0);
                if (c >= (unsigned long long)P.total_chunks) {
                    no_more = true;
                    break;
                }
                const int64_t grp = find_group(P.chunk_off, P.n_groups, (int64_t)c);
                const int64_t local = (int64_t)c - P.chunk_off[grp];
                const int64_t cp = P.cpn[grp];
                const int64_t k = local / cp, j = local - k * cp;
                cnode = (int)(P.node_off[grp] + k);
                cnext = (uint32_t)(j * P.chunk);
                cend = (uint32_t)min(P.walks[grp], (j + 1) * (int64_t)P.chunk);
                cpid = P.pid[grp];
                cf1 = fixed_exponent(P.walks[grp], P.lgM1);
                cf2 = fixed_exponent(P.walks[grp], P.lgM2);
                cpt = P.point_id ? P.point_id[cnode] : (uint32_t)k;
                const double *yc = P.y + 3 * (int64_t)cnode;
                cx = (T)(yc[0] - (kRel ? P.g.c[0] : 0.0));
                cy = (T)(yc[1] - (kRel ? P.g.c[1] : 0.0));
                cz = (T)(yc[2] - (kRel ? P.g.c[2] : 0.0));
            }
            const int nidle = __popc(idle);
            const int take = (int)min((uint32_t)nidle, cend - cnext);
            const int rank = __popc(idle & lt_mask);
            if (!active && rank < take) {
                acc.st += step;   // the length of the lane's previous walk (0 before the first)
                if (acc.node != cnode) {
                    acc.flush(P);
                    acc.node = cnode;
                }
                walk = cnext + (uint32_t)rank;
                step = 0;
                ppid = cpid;
                ppt = cpt;
                f1 = cf1;
                f2 = cf2;
                x = cx;
                y = cy;
                z = cz;
                active = true;
            }
            cnext += (uint32_t)take;
            if (take == nidle) {   // every idle lane has a walk
                idle = 0u;
                break;
            }
            idle = __ballot_sync(FULL, !active);
        }
        if (idle == FULL) break;   // no lane active and no walk left
        const int thresh = no_more ? 32 : P.refill;
        for (;;) {
            if constexpr (std::is_same<T, float>::value) {
                // three jumps from one Philox block; idle lanes run it too and
                // jump by 0, so the block needs no branch around it
                const uint4 w = philox4x32_10_rk(make_uint4(walk, step / 3u, ppt, ppid), P.rk0, P.rk1);
                uint32_t f[6];
                fields21(w, f);
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    if (unbounded(GK) && active && (kRel ? ball_escaped_rel(P.g, x, y, z) : geo_escaped<T>(P.g, x, y, z))) {
                        active = false;   // gone to infinity: scores 0
                        acc.esc += 1u;
                    }
                    // branch-free step: every lane evaluates; the lanes that do not
                    // go on jump by 0 (the lanes stay converged through the block)
                    const T d = kRel ? ball_dist_rel<GK>(P.g, x, y, z) : geo_dist<T, GK>(P.g, (const T *)sb, x, y, z);
                    const uint32_t st1 = step + 1u;
                    const bool absorbed = active && d <= eps;
                    // a walk neither absorbed nor going on is cut at max_steps
                    const bool go = active && !absorbed && st1 < P.max_steps;
                    jump(x, y, z, go ? d : (T)0, f[2 * h], f[2 * h + 1]);
                    step = active ? st1 : step;   // a finished walk's length stays until refill
                    pending = pending || absorbed;
                    active = go;
                }
            } else if (active) {
                if (unbounded(GK) && geo_escaped<T>(P.g, x, y, z)) {
                    active = false;   // gone to infinity: scores 0
                    acc.esc += 1u;
                } else {
                    const T d = geo_dist<T, GK>(P.g, (const T *)sb, x, y, z);
                    ++step;
                    if (d <= eps) {
                        pending = true;
                        active = false;
                    } else if (step >= P.max_steps) {
                        active = false;   // cut
                    } else {
                        const uint4 w = philox4x32_10_rk(make_uint4(walk, step - 1, ppt, ppid), P.rk0, P.rk1);
                        jump(x, y, z, d, w);
                    }
                }
            }
            if (__popc(__ballot_sync(FULL, !active)) >= thresh) break;
        }
    }
    acc.st += step;   // the lane's last walk
    acc.flush(P);
    // the last absorbed walks (fewer than 32)
    {
        const unsigned pm = __ballot_sync(FULL, pending);
        if (pending) {
            const int e = (qhead + qcount + __popc(pm & lt_mask)) & (kQueue - 1);
            Q.x[e] = x + ox;
            Q.y[e] = y + oy;
            Q.z[e] = z + oz;
            Q.node[e] = acc.node;
            Q.f1[e] = (short)f1;
            Q.f2[e] = (short)f2;
        }
        qcount += __popc(pm);
        __syncwarp();
        while (qcount > 0) score_batch<T, GK>(P, (const T *)sb, s_cs, Q, qhead, qcount, min(qcount, 32), lane, ws);
    }
    if (ws.node >= 0 && lane == 0) {
        atomicAdd(P.s1 + ws.node, (unsigned long long)ws.a1);
        atomicAdd(P.s2 + ws.node, (unsigned long long)ws.a2);
        atomicAdd(P.done + ws.node, ws.n);
    }
}

// FP32 walks in the bounded regions (ball, box, box minus boxes): the same
// walks as wos_kernel<float, GK>, bit for bit, with the bookkeeping of a jump
// moved from predicates, selects and integer counters (the int/logic pipe,
// which throttles issue in this kernel) to FP32 arithmetic on the FMA pipe.
// A walk carries af = 1 while it goes on and 0 once it has ended: a jump first
// counts the distance evaluation (lst += af), then af *= sat((d - eps) 1e30),
// which is exactly 1 for d > eps and 0 for d <= eps (d - eps rounds to the sign
// of the difference, and any nonzero difference of these normal floats times
// 1e30 saturates), and the walk moves by d af.  The Philox counter is the
// block index itself.  The max_steps cap is tested once per block: a block in
// which no lane can reach it runs the arithmetic above; one that can (rare)
// runs the exact per-jump test.  An ended walk is absorbed unless it was cut.
// MINB: resident blocks per SM the registers are budgeted for (8: 64 registers,
// no spills; 9: 56 registers, a few spilled values of the refill rounds).
template <int GK, int MINB>
__global__ void __launch_bounds__(kWosThreads, MINB) wos_kernel_f32(WosDev P) {
    extern __shared__ float s_boxes[];
    __shared__ ScoreQueue<float> s_queue[kWosThreads / 32];
    __shared__ float2 s_cs[kShPairs];
    const float *sb = nullptr;
    if (GK == kBoxMinusBoxes && P.g.nb <= kMaxSmemBoxes) {
        for (int i = threadIdx.x; i < 6 * P.g.nb; i += blockDim.x) s_boxes[i] = P.g.boxes_f[i];
        sb = s_boxes;
    }
    if (P.dat.kind == kHarmonicSH)
        for (int i = threadIdx.x; i < kShPairs; i += blockDim.x) s_cs[i] = P.dat.cart[i];
    __syncthreads();
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    const float eps = P.eps_f;
    ScoreQueue<float> &Q = s_queue[threadIdx.x >> 5];
    constexpr bool kRel = (GK == kBall);
    const float ox = kRel ? P.g.c_f[0] : 0.f, oy = kRel ? P.g.c_f[1] : 0.f, oz = kRel ? P.g.c_f[2] : 0.f;
    int qhead = 0, qcount = 0;   // warp-uniform
    WarpScore ws;

    // warp-uniform chunk state
    int cnode = -1;
    uint32_t cnext = 0, cend = 0;
    uint32_t cpid = 0, cpt = 0;
    int cf1 = 0, cf2 = 0;
    float cx = 0.f, cy = 0.f, cz = 0.f;
    bool no_more = false;

    // lane state
    bool hw = false;     // the lane holds a walk whose end has not been handled
    bool cut = false;    // that walk was cut at max_steps
    float af = 0.f;      // 1 while the walk goes on, 0 once it has ended
    float lst = 0.f;     // distance evaluations of the walk (exact below 2^24)
    float x = 0.f, y = 0.f, z = 0.f;
    uint32_t walk = 0, blk = 0, ppid = 0, ppt = 0;
    int f1 = 0, f2 = 0;
    LaneAcc acc;

    for (;;) {
        // ended walks: absorbed ones go to the queue with their absorption
        // point, cut ones are only released
        const bool ended = hw && af == 0.f;
        const bool pend = ended && !cut;
        const unsigned pm = __ballot_sync(FULL, pend);
        if (pm) {
            if (pend) {
                const int e = (qhead + qcount + __popc(pm & lt_mask)) & (kQueue - 1);
                Q.x[e] = x + ox;
                Q.y[e] = y + oy;
                Q.z[e] = z + oz;
                Q.node[e] = acc.node;
                Q.f1[e] = (short)f1;
                Q.f2[e] = (short)f2;
            }
            qcount += __popc(pm);
            __syncwarp();
            if (qcount >= 32) score_batch<float, GK>(P, sb, s_cs, Q, qhead, qcount, 32, lane, ws);
        }
        if (ended) {
            hw = false;
            cut = false;
        }
        // hand out walks to idle lanes
        unsigned idle = __ballot_sync(FULL, !hw);
        while (idle != 0u && !no_more) {
            if (cnext >= cend) {
                unsigned long long c = 0;
                if (lane == 0) c = atomicAdd(P.counter, 1ull);
                c = __shfl_sync(FULL, c, 0);
                if (c >= (unsigned long long)P.total_chunks) {
                    no_more = true;
                    break;
                }
                const int64_t grp = find_group(P.chunk_off, P.n_groups, (int64_t)c);
                const int64_t local = (int64_t)c - P.chunk_off[grp];
                const int64_t cp = P.cpn[grp];
                const int64_t k = local / cp, j = local - k * cp;
                cnode = (int)(P.node_off[grp] + k);
                cnext = (uint32_t)(j * P.chunk);
                cend = (uint32_t)min(P.walks[grp], (j + 1) * (int64_t)P.chunk);
                cpid = P.pid[grp];
                cf1 = fixed_exponent(P.walks[grp], P.lgM1);
                cf2 = fixed_exponent(P.walks[grp], P.lgM2);
                cpt = P.point_id ? P.point_id[cnode] : (uint32_t)k;
                const double *yc = P.y + 3 * (int64_t)cnode;
                cx = (float)(yc[0] - (kRel ? P.g.c[0] : 0.0));
                cy = (float)(yc[1] - (kRel ? P.g.c[1] : 0.0));
                cz = (float)(yc[2] - (kRel ? P.g.c[2] : 0.0));
            }
            const int nidle = __popc(idle);
            const int take = (int)min((uint32_t)nidle, cend - cnext);
            const int rank = __popc(idle & lt_mask);
            if (!hw && rank < take) {
                acc.st += (uint32_t)lst;   // the length of the lane's previous walk (0 before the first)
                if (acc.node != cnode) {
                    acc.flush(P);
                    acc.node = cnode;
                }
                walk = cnext + (uint32_t)rank;
                blk = 0;
                lst = 0.f;
                ppid = cpid;
                ppt = cpt;
                f1 = cf1;
                f2 = cf2;
                x = cx;
                y = cy;
                z = cz;
                af = 1.f;
                hw = true;
            }
            cnext += (uint32_t)take;
            if (take == nidle) {   // every idle lane has a walk
                idle = 0u;
                break;
            }
            idle = __ballot_sync(FULL, !hw);
        }
        if (idle == FULL) break;   // no lane holds a walk and no walk is left
        const int thresh = no_more ? 32 : P.refill;
        for (;;) {
            // three jumps from one Philox block; lanes without a walk run it too
            // and move by 0
            const uint4 w = philox4x32_10_rk(make_uint4(walk, blk, ppt, ppid), P.rk0, P.rk1);
            uint32_t f[6];
            fields21(w, f);
            if (!__any_sync(FULL, hw && blk >= P.blk_fast)) {
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    const float d = kRel ? ball_dist_rel<GK>(P.g, x, y, z) : geo_dist<float, GK>(P.g, sb, x, y, z);
                    lst += af;
                    af *= __saturatef((d - eps) * 1e30f);
                    jump(x, y, z, d * af, f[2 * h], f[2 * h + 1]);
                }
            } else {
                // a lane may reach max_steps in this block: the exact test
#pragma unroll
                for (int h = 0; h < 3; ++h) {
                    const float d = kRel ? ball_dist_rel<GK>(P.g, x, y, z) : geo_dist<float, GK>(P.g, sb, x, y, z);
                    const bool active = af != 0.f;
                    const bool absorbed = active && d <= eps;
                    const bool go = active && !absorbed && 3u * blk + (uint32_t)h + 1u < P.max_steps;
                    cut = cut || (active && !absorbed && !go);
                    lst += af;
                    af = go ? 1.f : 0.f;
                    jump(x, y, z, go ? d : 0.f, f[2 * h], f[2 * h + 1]);
                }
            }
            ++blk;
            if (__popc(__ballot_sync(FULL, af == 0.f)) >= thresh) break;
        }
    }
    acc.st += (uint32_t)lst;   // the lane's last walk
    acc.flush(P);
    // the last absorbed walks (fewer than 32)
    {
        const bool pend = hw && af == 0.f && !cut;
        const unsigned pm = __ballot_sync(FULL, pend);
        if (pend) {
            const int e = (qhead + qcount + __popc(pm & lt_mask)) & (kQueue - 1);
            Q.x[e] = x + ox;
            Q.y[e] = y + oy;
            Q.z[e] = z + oz;
            Q.node[e] = acc.node;
            Q.f1[e] = (short)f1;
            Q.f2[e] = (short)f2;
        }
        qcount += __popc(pm);
        __syncwarp();
        while (qcount > 0) score_batch<float, GK>(P, sb, s_cs, Q, qhead, qcount, min(qcount, 32), lane, ws);
    }
    if (ws.node >= 0 && lane == 0) {
        atomicAdd(P.s1 + ws.node, (unsigned long long)ws.a1);
        atomicAdd(P.s2 + ws.node, (unsigned long long)ws.a2);
        atomicAdd(P.done + ws.node, ws.n);
    }
}

__global__ void wos_finalize_kernel(int64_t n_nodes, int64_t n_groups, const int64_t *__restrict__ node_off,
                                    const int64_t *__restrict__ walks, const unsigned long long *__restrict__ s1,
                                    const unsigned long long *__restrict__ s2,
                                    const unsigned long long *__restrict__ st,
                                    const unsigned int *__restrict__ done, int lgM1, int lgM2,
                                    double *__restrict__ mean, double *__restrict__ se,
                                    uint64_t *__restrict__ steps, uint32_t *__restrict__ capped,
                                    int32_t *__restrict__ group_capped) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    const int64_t grp = find_group(node_off, n_groups, i);
    const double N = (double)done[i];   // walks not cut at max_steps
    const double inv1 = pow2(-fixed_exponent(walks[grp], lgM1));
    const double inv2 = pow2(-fixed_exponent(walks[grp], lgM2));
    // a node with no walk left has no estimate (NaN); with one, no standard
    // error (+inf)
    const double m1 = N > 0.0 ? (double)(long long)s1[i] * inv1 / N : __longlong_as_double(0x7ff8000000000000ll);
    const double e2 = (double)(long long)s2[i] * inv2;
    const double var = N > 1.0 ? fmax((e2 - N * m1 * m1) / (N * (N - 1.0)), 0.0) : __longlong_as_double(0x7ff0000000000000ll);
    mean[i] = m1;
    if (se) se[i] = sqrt(var);
    if (steps) steps[i] = st[i];
    const uint32_t cut = (uint32_t)(walks[grp] - (int64_t)done[i]);
    if (capped) capped[i] = cut;
    if (group_capped && cut) group_capped[grp] = 1;   // every writer stores 1
}

// DTN_E_WALK_CAP for the solved patches that had walks cut at max_steps (it
// replaces DTN_E_NOT_CONVERGED: a node without walks makes the system NaN)
__global__ void walk_cap_status_kernel(int64_t n, const int32_t *__restrict__ group_capped,
                                       int32_t *__restrict__ status) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n && group_capped[p] && (status[p] == DTN_OK || status[p] == DTN_E_NOT_CONVERGED))
        status[p] = DTN_E_WALK_CAP;
}

// FP32 walks in bounded regions take wos_kernel_f32 while the float step count
// of a walk stays exact (max_steps <= 2^24), budgeted for 9 resident blocks
// per SM when 9 or more are asked for, else for 8
template <int GK>
void *wos_kernel_f32_ptr(int bps) {
    return bps >= 9 ? (void *)wos_kernel_f32<GK, 9> : (void *)wos_kernel_f32<GK, 8>;
}

template <typename T>
void *wos_kernel_ptr(int gk, uint64_t max_steps, int bps) {
    if (std::is_same<T, float>::value && max_steps <= (1ull << 24)) {
        if (gk == kBall) return wos_kernel_f32_ptr<kBall>(bps);
        if (gk == kBox) return wos_kernel_f32_ptr<kBox>(bps);
        if (gk == kBoxMinusBoxes) return wos_kernel_f32_ptr<kBoxMinusBoxes>(bps);
    }
    if (gk == kBall) return (void *)wos_kernel<T, kBall>;
    if (gk == kBox) return (void *)wos_kernel<T, kBox>;
    if (gk == kHalfSpace) return (void *)wos_kernel<T, kHalfSpace>;
    if (gk == kDiskExterior) return (void *)wos_kernel<T, kDiskExterior>;
    if (gk == kBallExterior) return (void *)wos_kernel<T, kBallExterior>;
    return (void *)wos_kernel<T, kBoxMinusBoxes>;
}

}  // namespace

// Accumulator bytes of a walk launch over `nodes` nodes: s1, s2, st (u64) and
// done (u32) per node, after a 64-byte slot for the work counter.
size_t wos_scratch_bytes(int64_t nodes) {
    return (size_t)nodes * (3 * sizeof(unsigned long long) + sizeof(unsigned int)) + 64;
}

// The walk launch with its accumulators in the geometry's workspace.
cudaError_t launch_wos(dtn_geometry *g, const WosLaunch &w, cudaStream_t s) {
    if (w.total_nodes == 0) return cudaSuccess;
    cudaError_t e = g->ws.acc.reserve(wos_scratch_bytes(w.total_nodes), s);
    if (e != cudaSuccess) return e;
    return launch_wos_into(g, w, g->ws.acc.p, s);
}

// The walk launch with the accumulators and the work counter in `acc` (at least
// wos_scratch_bytes(nodes) bytes, 256-byte aligned, device): walks, then the
// estimates of Eq. bw87.
cudaError_t launch_wos_into(dtn_geometry *g, const WosLaunch &w, void *acc, cudaStream_t s) {
    if (w.total_nodes == 0) return cudaSuccess;
    if (w.total_nodes > 0x7fffffffll) return cudaErrorInvalidValue;   // node ids are 32-bit in the kernel
    cudaError_t e;
    const size_t n = (size_t)w.total_nodes;
    const size_t bytes = wos_scratch_bytes(w.total_nodes);
    char *base = (char *)acc;
    unsigned long long *counter = (unsigned long long *)base;
    unsigned long long *s1 = (unsigned long long *)(base + 64);
    unsigned long long *s2 = s1 + n, *st = s2 + n;
    unsigned int *done = (unsigned int *)(st + n);
    if ((e = cudaMemsetAsync(base, 0, bytes, s)) != cudaSuccess) return e;
    if (w.group_capped && (e = cudaMemsetAsync(w.group_capped, 0, (size_t)w.n_groups * sizeof(int32_t), s)) != cudaSuccess)
        return e;
    // fixed-point scales follow the bound on |g| (per node walk count on the device)
    const double M = g->score_bound > 0 ? g->score_bound : 1.0;
    const int lgM1 = (int)std::ceil(std::log2(M)), lgM2 = (int)std::ceil(std::log2(M * M));
    WosDev P;
    P.g = g->dg;
    P.dat = g->dd;
    P.y = w.y;
    P.node_off = w.node_off;
    P.walks = w.walks;
    P.pid = w.pid;
    P.point_id = w.point_id;
    P.chunk_off = w.chunk_off;
    P.cpn = w.cpn;
    P.n_groups = w.n_groups;
    P.total_chunks = w.total_chunks;
    P.chunk = w.chunk;
    P.refill = w.refill > 0 ? std::min(w.refill, 32) : 8;
    P.counter = counter;
    P.s1 = s1; P.s2 = s2; P.st = st; P.done = done;
    P.lgM1 = lgM1;
    P.lgM2 = lgM2;
    P.eps = w.eps;
    P.eps_f = (float)w.eps;
    P.max_steps = (uint32_t)std::min<uint64_t>(w.max_steps, 0xFFFFFFFFull);
    // a block of jumps 3 blk + 1 .. 3 blk + 3 can reach max_steps once 3 blk + 3 >= max_steps
    P.blk_fast = P.max_steps >= 3u ? (P.max_steps - 1u) / 3u : 0u;
    philox_round_keys(w.seed, P.rk0, P.rk1);
    const int gk = g->dg.kind;
    const bool fp32 = (w.prec == DTN_PREC_MIXED);
    void *fn = fp32 ? wos_kernel_ptr<float>(gk, P.max_steps, w.blocks_per_sm)
                    : wos_kernel_ptr<double>(gk, P.max_steps, w.blocks_per_sm);
    const size_t smem = (gk == kBoxMinusBoxes && fp32 && g->dg.nb <= kMaxSmemBoxes) ? 6 * sizeof(float) * g->dg.nb : 0;
    if (smem > 48 * 1024) {
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
    }
    int resident = 1;
    // persistent grid: never more blocks per SM than can be resident at once
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fn, kWosThreads, smem)) != cudaSuccess)
        return e;
    resident = std::max(resident, 1);
    const int bps = w.blocks_per_sm > 0 ? std::min(w.blocks_per_sm, resident) : resident;
    int64_t blocks = (int64_t)g->num_sms * bps;
    // no more warps than chunks
    const int64_t max_blocks = (w.total_chunks + (kWosThreads / 32) - 1) / (kWosThreads / 32);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    void *args[] = {&P};
    if ((e = cudaLaunchKernel(fn, dim3((unsigned)blocks), dim3(kWosThreads), args, smem, s)) != cudaSuccess)
        return e;
    const int T = 256;
    wos_finalize_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(
        w.total_nodes, w.n_groups, w.node_off, w.walks, s1, s2, st, done, lgM1, lgM2, w.mean, w.se, w.steps, w.capped,
        w.group_capped);
    return cudaGetLastError();
}

int wos_resident_blocks(const dtn_geometry *g, int prec) {
    const int gk = g->dg.kind;
    const bool fp32 = (prec == DTN_PREC_MIXED);
    void *fn = fp32 ? wos_kernel_ptr<float>(gk, 1000000, 0) : wos_kernel_ptr<double>(gk, 1000000, 0);
    const size_t smem = (gk == kBoxMinusBoxes && fp32 && g->dg.nb <= kMaxSmemBoxes) ? 6 * sizeof(float) * g->dg.nb : 0;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int resident = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, fn, kWosThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(resident, 1);
}

cudaError_t launch_walk_cap_status(int64_t n, const int32_t *group_capped, int32_t *status, cudaStream_t s) {
    if (n == 0 || !status || !group_capped) return cudaSuccess;
    const int T = 256;
    walk_cap_status_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(n, group_capped, status);
    return cudaGetLastError();
}

cudaError_t upload_sh_wos(const ShTables &t) { return upload_sh_tables_here(t); }

// ---------------------------------------------------------------- small checks

namespace {

__global__ void philox_kernel(int64_t n, const uint32_t *__restrict__ ctr, uint32_t k0, uint32_t k1,
                              uint32_t *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 r = philox4x32_10(c, k0, k1);
    out[4 * i] = r.x; out[4 * i + 1] = r.y; out[4 * i + 2] = r.z; out[4 * i + 3] = r.w;
}

// The draws of FP32 walks for n Philox blocks: the six fields, their uniforms
// (v - 1, exact) and the unit directions of the block's three jumps (the jump
// of a walk at the origin by d = 1), by the walk kernel's own functions.
__global__ void fields21_kernel(int64_t n, const uint32_t *__restrict__ ctr, uint32_t k0, uint32_t k1,
                                uint32_t *__restrict__ fields, float *__restrict__ uni, float *__restrict__ dir) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 w = philox4x32_10(c, k0, k1);
    uint32_t f[6];
    fields21(w, f);
    for (int k = 0; k < 6; ++k) {
        if (fields) fields[6 * i + k] = f[k];
        if (uni) uni[6 * i + k] = one_plus_u21(f[k]) - 1.0f;
    }
    if (dir)
        for (int h = 0; h < 3; ++h) {
            float x = 0.f, y = 0.f, z = 0.f;
            jump(x, y, z, 1.0f, f[2 * h], f[2 * h + 1]);
            dir[9 * i + 3 * h] = x;
            dir[9 * i + 3 * h + 1] = y;
            dir[9 * i + 3 * h + 2] = z;
        }
}

template <typename T>
__global__ void distance_kernel(DGeom g, int64_t n, const double *__restrict__ x, double *__restrict__ d,
                                double *__restrict__ nb) {
    extern __shared__ float s_boxes[];
    const float *sb = nullptr;
    if (std::is_same<T, float>::value && g.kind == kBoxMinusBoxes && g.nb <= kMaxSmemBoxes) {
        for (int i = threadIdx.x; i < 6 * g.nb; i += blockDim.x) s_boxes[i] = g.boxes_f[i];
        __syncthreads();
        sb = s_boxes;
    }
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T px = (T)x[3 * i], py = (T)x[3 * i + 1], pz = (T)x[3 * i + 2];
    T dist;
    if (g.kind == kBall) dist = geo_dist<T, kBall>(g, (const T *)sb, px, py, pz);
    else if (g.kind == kBox) dist = geo_dist<T, kBox>(g, (const T *)sb, px, py, pz);
    else if (g.kind == kHalfSpace) dist = geo_dist<T, kHalfSpace>(g, (const T *)sb, px, py, pz);
    else if (g.kind == kDiskExterior) dist = geo_dist<T, kDiskExterior>(g, (const T *)sb, px, py, pz);
    else if (g.kind == kBallExterior) dist = geo_dist<T, kBallExterior>(g, (const T *)sb, px, py, pz);
    else dist = geo_dist<T, kBoxMinusBoxes>(g, (const T *)sb, px, py, pz);
    if (d) d[i] = (double)dist;
    if (nb) {
        T ax, ay, az;
        geo_nearest<T>(g, (const T *)sb, px, py, pz, ax, ay, az);
        nb[3 * i] = ax; nb[3 * i + 1] = ay; nb[3 * i + 2] = az;
    }
}

__global__ void dirichlet_kernel(DData dat, int64_t n, const double *__restrict__ x, double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = dirichlet_eval<double>(dat, x[3 * i], x[3 * i + 1], x[3 * i + 2]);
}

}  // namespace

cudaError_t launch_philox(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int T = 256;
    philox_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(n, ctr, (uint32_t)(seed & 0xFFFFFFFFull),
                                                            (uint32_t)(seed >> 32), out);
    return cudaGetLastError();
}

cudaError_t launch_fields21(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *fields, float *uni, float *dir,
                            cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int T = 256;
    fields21_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(n, ctr, (uint32_t)(seed & 0xFFFFFFFFull),
                                                              (uint32_t)(seed >> 32), fields, uni, dir);
    return cudaGetLastError();
}

cudaError_t launch_distance(const dtn_geometry *g, int64_t n, const double *x, double *d, double *nearest,
                            int prec, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int T = 128;
    const unsigned blocks = (unsigned)((n + T - 1) / T);
    if (prec == DTN_PREC_MIXED) {
        const size_t smem = (g->dg.kind == kBoxMinusBoxes && g->dg.nb <= kMaxSmemBoxes) ? 6 * sizeof(float) * g->dg.nb : 0;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute((void *)distance_kernel<float>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        distance_kernel<float><<<blocks, T, smem, s>>>(g->dg, n, x, d, nearest);
    } else {
        distance_kernel<double><<<blocks, T, 0, s>>>(g->dg, n, x, d, nearest);
    }
    return cudaGetLastError();
}

cudaError_t launch_dirichlet(const dtn_geometry *g, int64_t n, const double *x, double *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int T = 128;
    dirichlet_kernel<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(g->dd, n, x, out);
    return cudaGetLastError();
}

}  // namespace dtn
