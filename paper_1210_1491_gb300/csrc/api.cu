// api.cu -- the C ABI of include/dtn.h: geometry objects, Dirichlet data, the
// BIE-WOS batch solve (Sec. 4), potential evaluation (Eq. bw03) and the small
// checking entry points.  Host code only orchestrates; every numerical step
// runs in the kernels of setup.cu, wos.cu, assemble.cu, lu.cu, potential.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "dtn_internal.h"

namespace dtn {

namespace {
std::atomic<int32_t> g_last_cuda_error{0};
}

void set_cuda_error(cudaError_t e) { g_last_cuda_error.store((int32_t)e); }

bool wrong_device(const dtn_geometry *g) {
    int dev = -1;
    return cudaGetDevice(&dev) != cudaSuccess || dev != g->device;
}

cudaError_t DevBuf::reserve(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    if (p) {
        cudaError_t e = cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (e != cudaSuccess) return e;
    }
    const size_t want = std::max<size_t>(n, 256);
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        p = nullptr;
        return e;
    }
    bytes = want;
    pooled = false;
    return cudaSuccess;
}

cudaError_t DevBuf::reserve(size_t n, cudaStream_t s) {
    if (n <= bytes && p) return cudaSuccess;
    const size_t want = std::max<size_t>({n, bytes + bytes / 2, 256});
    if (p) {
        cudaError_t e = pooled ? cudaFreeAsync(p, s) : cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMallocAsync(&p, want, s);
    if (e != cudaSuccess) {
        p = nullptr;
        return e;
    }
    bytes = want;
    pooled = true;
    return cudaSuccess;
}

void DevBuf::release() {
    if (p) {
        if (pooled) {
            // stream-ordered memory: free it once nothing on the device can use it
            cudaDeviceSynchronize();
            cudaFreeAsync(p, nullptr);
            cudaStreamSynchronize(nullptr);
        } else {
            cudaFree(p);
        }
    }
    p = nullptr;
    bytes = 0;
    pooled = false;
}

dtn_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return DTN_OK;
    set_cuda_error(e);
    cudaGetLastError();   // do not leave a non-sticky error for the caller's next CUDA call
    return e == cudaErrorMemoryAllocation ? DTN_E_OUT_OF_MEMORY : DTN_E_CUDA;
}

namespace {

// Lower bound of the distance between two axis-aligned boxes.
double box_box_dist(const double *alo, const double *ahi, const double *blo, const double *bhi) {
    double s = 0.0;
    for (int i = 0; i < 3; ++i) {
        const double t = std::max({0.0, blo[i] - ahi[i], alo[i] - bhi[i]});
        s += t * t;
    }
    return std::sqrt(s);
}

// Obstacle lookup grid: every cell lists the boxes whose distance to the cell
// (grown by a small margin, so that a point filed in a neighbouring cell by
// rounding is still covered) is at most `listing`, and stores the smallest
// distance to any box it does not list.
void build_grid(GeometryHost &h) {
    const dtn_geometry_desc &d = h.desc;
    const double ext[3] = {d.hi[0] - d.lo[0], d.hi[1] - d.lo[1], d.hi[2] - d.lo[2]};
    double cell = d.cell_size > 0 ? d.cell_size : std::max({ext[0], ext[1], ext[2]}) / 64.0;
    for (int i = 0; i < 3; ++i) {
        h.gn[i] = std::max(1, (int)std::ceil(ext[i] / cell));
        h.glo[i] = d.lo[i];
    }
    h.cell = cell;
    const double listing = 2.0 * cell, margin = 1e-3 * cell;
    const int64_t nc = (int64_t)h.gn[0] * h.gn[1] * h.gn[2];
    h.cstart.assign(nc + 1, 0);
    h.citems.clear();
    h.ccap.assign(nc, 0.f);
    const int nb = d.n_boxes;
    for (int64_t c = 0; c < nc; ++c) {
        const int ix = (int)(c % h.gn[0]), iy = (int)((c / h.gn[0]) % h.gn[1]), iz = (int)(c / ((int64_t)h.gn[0] * h.gn[1]));
        const double lo[3] = {h.glo[0] + ix * cell - margin, h.glo[1] + iy * cell - margin, h.glo[2] + iz * cell - margin};
        const double hi[3] = {lo[0] + cell + 2 * margin, lo[1] + cell + 2 * margin, lo[2] + cell + 2 * margin};
        double cap = 1e30;
        for (int b = 0; b < nb; ++b) {
            const double *bl = &h.boxes[6 * b], *bh = bl + 3;
            const double dd = box_box_dist(lo, hi, bl, bh);
            if (dd <= listing) h.citems.push_back(b);
            else cap = std::min(cap, dd);
        }
        // FP32 cap rounded down so it never exceeds the true bound
        float cf = (float)cap;
        if ((double)cf > cap) cf = std::nextafter(cf, 0.0f);
        h.ccap[c] = cf;
        h.cstart[c + 1] = (int)h.citems.size();
    }
}

double point_boundary_distance(const dtn_geometry_desc &d, const double *x) {
    if (d.kind == DTN_GEOM_HALF_SPACE) return std::fabs(x[2] - d.center[2]);
    if (d.kind == DTN_GEOM_DISK_EXTERIOR) {
        const double r = std::hypot(x[0] - d.center[0], x[1] - d.center[1]), z = x[2] - d.center[2];
        return r <= d.radius ? std::fabs(z) : std::hypot(r - d.radius, z);
    }
    if (d.kind == DTN_GEOM_BALL_INTERIOR || d.kind == DTN_GEOM_BALL_EXTERIOR) {
        const double r = std::sqrt((x[0] - d.center[0]) * (x[0] - d.center[0]) + (x[1] - d.center[1]) * (x[1] - d.center[1]) +
                                   (x[2] - d.center[2]) * (x[2] - d.center[2]));
        return std::fabs(d.radius - r);
    }
    auto box_surface = [](const double *lo, const double *hi, const double *p) {
        bool inside = true;
        double s = 0.0, m = 1e300;
        for (int i = 0; i < 3; ++i) {
            const double t = std::max({0.0, lo[i] - p[i], p[i] - hi[i]});
            s += t * t;
            if (p[i] < lo[i] || p[i] > hi[i]) inside = false;
            m = std::min({m, p[i] - lo[i], hi[i] - p[i]});
        }
        return inside ? m : std::sqrt(s);
    };
    double dist = box_surface(d.lo, d.hi, x);
    if (d.kind == DTN_GEOM_BOX_MINUS_BOXES)
        for (int b = 0; b < d.n_boxes; ++b) dist = std::min(dist, box_surface(d.boxes + 6 * b, d.boxes + 6 * b + 3, x));
    return dist;
}

// |g| bound on the boundary, for the fixed-point scale of the walk sums
double score_bound(const dtn_geometry_desc &gd, const dtn_dirichlet_desc &dd) {
    if (dd.kind == DTN_DATA_POINT_SOURCE) {
        const double dist = point_boundary_distance(gd, dd.x0);
        return std::fabs(dd.strength) / (4.0 * kPi * std::max(dist, 1e-12));
    }
    if (dd.kind == DTN_DATA_HARMONIC_SH) {
        // farthest boundary point from the data centre
        double rmax = 0.0;
        if (gd.kind == DTN_GEOM_BALL_INTERIOR || gd.kind == DTN_GEOM_HALF_SPACE ||
            gd.kind == DTN_GEOM_DISK_EXTERIOR || gd.kind == DTN_GEOM_BALL_EXTERIOR) {
            // (unbounded regions: the scored points lie within the truncation sphere)
            rmax = (gd.kind == DTN_GEOM_BALL_INTERIOR ? gd.radius : gd.truncation) + std::sqrt((gd.center[0] - dd.center[0]) * (gd.center[0] - dd.center[0]) +
                                         (gd.center[1] - dd.center[1]) * (gd.center[1] - dd.center[1]) +
                                         (gd.center[2] - dd.center[2]) * (gd.center[2] - dd.center[2]));
        } else {
            for (int c = 0; c < 8; ++c) {
                double s = 0.0;
                for (int i = 0; i < 3; ++i) {
                    const double v = ((c >> i) & 1 ? gd.hi[i] : gd.lo[i]) - dd.center[i];
                    s += v * v;
                }
                rmax = std::max(rmax, std::sqrt(s));
            }
        }
        const double rho = rmax / dd.scale;
        double tot = 0.0, rl = 1.0;
        for (int l = 0; l <= dd.lmax; ++l) {
            double cs = 0.0;
            for (int m = -l; m <= l; ++m) cs += std::fabs(dd.clm[l * l + l + m]);
            tot += rl * cs * std::sqrt((2.0 * l + 1.0) / (4.0 * kPi));
            rl *= rho;
        }
        return tot;
    }
    return std::fabs(dd.constant);
}

// Batch layout: per-patch offsets, shape groups (one matrix per region kind,
// a, rings, sectors) and weight groups (also node orders).  A wrapped patch
// (wrapped[p] != 0) is congruent to no other: it gets groups of its own, and
// its weight group no columns (its right side is assembled directly).
dtn_status build_layout(const dtn_patch_batch *b, BatchLayout &L, bool cap, const uint8_t *wrapped = nullptr) {
    const int64_t n = b->n_patches;
    L.n_patches = n;
    L.gamma_off.assign(n + 1, 0);
    L.panel_off.assign(n + 1, 0);
    L.mat_off.assign(n + 1, 0);
    L.nt.resize(n); L.nph.resize(n); L.nr.resize(n); L.ns.resize(n);
    L.walks.resize(n); L.pid.resize(n); L.radius.assign(n, 0.0);
    L.group_of.assign(n, 0);
    L.rep.clear();
    L.max_panels = 0; L.max_nodes = 0; L.max_walks = 0;
    std::map<std::tuple<uint64_t, int32_t, int32_t, int64_t>, int64_t> groups;
    std::map<std::tuple<uint64_t, int32_t, int32_t, int32_t, int32_t, int64_t>, int64_t> wgroups;
    L.wrapped.assign(n, 0);
    L.wgroup_of.assign(n, 0);
    L.wrep.clear();
    for (int64_t p = 0; p < n; ++p) {
        const int32_t nt = b->n_theta[p], nph = b->n_phi[p], nr = b->n_rings[p], ns = b->n_sectors[p];
        if (nt < 1 || nt > kMaxGauss || nph < 1 || nph > kMaxGauss || nr < 1 || ns < 1 || (int64_t)nr * ns > 1024)
            return DTN_E_INVALID_ARG;
        const int32_t np = nr * ns, P = nt * nph;
        L.nt[p] = nt; L.nph[p] = nph; L.nr[p] = nr; L.ns[p] = ns;
        if (b->radius) {
            const double a = b->radius[p];
            if (!(a > 0.0) || !std::isfinite(a)) return DTN_E_INVALID_ARG;
            L.radius[p] = a;
        }
        uint64_t abits;
        std::memcpy(&abits, &L.radius[p], sizeof(abits));
        const int64_t uniq = (wrapped && wrapped[p]) ? p : -1;
        L.wrapped[p] = (uniq >= 0) ? 1 : 0;
        auto key = std::make_tuple(abits, nr, ns, uniq);
        auto it = groups.find(key);
        if (it == groups.end()) {
            it = groups.emplace(key, (int64_t)L.rep.size()).first;
            L.rep.push_back(p);
        }
        L.group_of[p] = it->second;
        auto wkey = std::make_tuple(abits, nr, ns, nt, nph, uniq);
        auto wit = wgroups.find(wkey);
        if (wit == wgroups.end()) {
            wit = wgroups.emplace(wkey, (int64_t)L.wrep.size()).first;
            L.wrep.push_back(p);
        }
        L.wgroup_of[p] = wit->second;
        L.walks[p] = b->walks_per_point ? b->walks_per_point[p] : 0;
        L.pid[p] = b->patch_ids ? b->patch_ids[p] : (uint32_t)(b->patch_id_base + (uint32_t)p);
        L.gamma_off[p + 1] = L.gamma_off[p] + P;
        L.panel_off[p + 1] = L.panel_off[p] + np;
        L.mat_off[p + 1] = L.mat_off[p] + (int64_t)np * np;
        L.max_panels = std::max(L.max_panels, np);
        L.max_nodes = std::max(L.max_nodes, P);
        L.max_walks = std::max(L.max_walks, L.walks[p]);
    }
    L.gamma_total = L.gamma_off[n];
    L.panels_total = L.panel_off[n];
    L.matrix_total = L.mat_off[n];
    L.n_groups = (int64_t)L.rep.size();
    L.grows_off.assign(L.n_groups + 1, 0);
    L.gmat_off.assign(L.n_groups + 1, 0);
    L.gfac_off.assign(L.n_groups + 1, 0);
    for (int64_t k = 0; k < L.n_groups; ++k) {
        const int64_t np = (int64_t)L.nr[L.rep[k]] * L.ns[L.rep[k]];
        L.grows_off[k + 1] = L.grows_off[k] + np;
        L.gmat_off[k + 1] = L.gmat_off[k] + np * np;
        L.gfac_off[k + 1] = L.gfac_off[k] + np * (np + 1);
    }
    L.grows_total = L.grows_off[L.n_groups];
    L.gmat_total = L.gmat_off[L.n_groups];
    L.gfac_total = L.gfac_off[L.n_groups];
    // right-side weights (per weight group) and sample vectors (per patch)
    const int64_t nw = (int64_t)L.wrep.size();
    L.n_wgroups = nw;
    L.wrows_off.assign(nw + 1, 0);
    L.kcols.assign(nw, 0);
    L.gw_off.assign(nw + 1, 0);
    L.mem_off.assign(nw + 1, 0);
    L.tile_off.assign(nw + 1, 0);
    L.max_wgroup_rows = 0;
    for (int64_t k = 0; k < nw; ++k) {
        const int64_t r = L.wrep[k];
        const int64_t np = (int64_t)L.nr[r] * L.ns[r];
        L.wrows_off[k + 1] = L.wrows_off[k] + np;
        L.kcols[k] = L.wrapped[r] ? 0 : (cap ? (int64_t)kSamplesPerPanel * np : 0) + (int64_t)L.nt[r] * L.nph[r];
        L.gw_off[k + 1] = L.gw_off[k] + np * L.kcols[k];
        L.max_wgroup_rows = std::max<int32_t>(L.max_wgroup_rows, (int32_t)np);
    }
    L.wrows_total = L.wrows_off[nw];
    L.gw_total = L.gw_off[nw];
    L.vec_off.assign(n + 1, 0);
    std::vector<int64_t> count(nw, 0);
    for (int64_t p = 0; p < n; ++p) {
        L.vec_off[p + 1] = L.vec_off[p] + L.kcols[L.wgroup_of[p]];
        ++count[L.wgroup_of[p]];
    }
    L.vec_total = L.vec_off[n];
    for (int64_t k = 0; k < nw; ++k) {
        L.mem_off[k + 1] = L.mem_off[k] + count[k];
        L.tile_off[k + 1] = L.tile_off[k] + (count[k] + kRhsTileN - 1) / kRhsTileN;
    }
    L.tiles_total = L.tile_off[nw];
    L.members.assign(n, 0);
    std::vector<int64_t> fill(L.mem_off.begin(), L.mem_off.end() - 1);
    for (int64_t p = 0; p < n; ++p) L.members[fill[L.wgroup_of[p]]++] = p;
    return DTN_OK;
}

// Packs the layout arrays (plus chunk bookkeeping of the walks) into one device
// buffer.  Pageable-memory copies are staged by the runtime before return.
cudaError_t upload_layout(dtn_geometry *g, const BatchLayout &L, int32_t chunk, DevLayout &D,
                          int64_t &total_chunks, cudaStream_t s) {
    const int64_t n = L.n_patches;
    std::vector<int64_t> chunk_off(n + 1, 0);
    std::vector<int32_t> cpn(n, 1);
    for (int64_t p = 0; p < n; ++p) {
        const int64_t c = (L.walks[p] + chunk - 1) / chunk;
        cpn[p] = (int32_t)std::max<int64_t>(c, 1);
        const int64_t nodes = L.gamma_off[p + 1] - L.gamma_off[p];
        chunk_off[p + 1] = chunk_off[p] + (L.walks[p] > 0 ? nodes * cpn[p] : 0);
    }
    total_chunks = chunk_off[n];
    // byte layout: 5 int64 arrays (n+1 or n), 5 int32 arrays (n), pid (n), frames (n)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    const size_t o_goff = off; off = al(off + (n + 1) * 8);
    const size_t o_poff = off; off = al(off + (n + 1) * 8);
    const size_t o_moff = off; off = al(off + (n + 1) * 8);
    const size_t o_walk = off; off = al(off + n * 8);
    const size_t o_coff = off; off = al(off + (n + 1) * 8);
    const size_t o_nt = off; off = al(off + n * 4);
    const size_t o_nph = off; off = al(off + n * 4);
    const size_t o_nr = off; off = al(off + n * 4);
    const size_t o_ns = off; off = al(off + n * 4);
    const size_t o_cpn = off; off = al(off + n * 4);
    const size_t o_pid = off; off = al(off + n * 4);
    const size_t o_rad = off; off = al(off + n * 8);
    const int64_t ng = L.n_groups;
    const size_t o_gof = off; off = al(off + n * 8);
    const size_t o_rep = off; off = al(off + ng * 8);
    const size_t o_grow = off; off = al(off + (ng + 1) * 8);
    const size_t o_gmat = off; off = al(off + (ng + 1) * 8);
    const size_t o_gfac = off; off = al(off + (ng + 1) * 8);
    const int64_t nw = L.n_wgroups;
    const size_t o_wrep = off; off = al(off + nw * 8);
    const size_t o_wrow = off; off = al(off + (nw + 1) * 8);
    const size_t o_kc = off; off = al(off + nw * 8);
    const size_t o_gwo = off; off = al(off + (nw + 1) * 8);
    const size_t o_vec = off; off = al(off + (n + 1) * 8);
    const size_t o_mem = off; off = al(off + n * 8);
    const size_t o_mof = off; off = al(off + (nw + 1) * 8);
    const size_t o_tof = off; off = al(off + (nw + 1) * 8);
    const size_t host_bytes = off;
    const size_t o_fr = off; off = al(off + n * sizeof(PatchFrame));
    // pieces of wrapped patches (obstacle regions only)
    const bool wrapped_possible = (g->dg.kind == kBoxMinusBoxes);
    const size_t o_pc = off; off = al(off + (wrapped_possible ? n * kMaxPieces * sizeof(Piece) : 0));
    cudaError_t e = g->ws.layout.reserve(off, s);
    if (e != cudaSuccess) return e;
    std::vector<unsigned char> h(host_bytes, 0);
    std::memcpy(&h[o_goff], L.gamma_off.data(), (n + 1) * 8);
    std::memcpy(&h[o_poff], L.panel_off.data(), (n + 1) * 8);
    std::memcpy(&h[o_moff], L.mat_off.data(), (n + 1) * 8);
    std::memcpy(&h[o_walk], L.walks.data(), n * 8);
    std::memcpy(&h[o_coff], chunk_off.data(), (n + 1) * 8);
    std::memcpy(&h[o_nt], L.nt.data(), n * 4);
    std::memcpy(&h[o_nph], L.nph.data(), n * 4);
    std::memcpy(&h[o_nr], L.nr.data(), n * 4);
    std::memcpy(&h[o_ns], L.ns.data(), n * 4);
    std::memcpy(&h[o_cpn], cpn.data(), n * 4);
    std::memcpy(&h[o_pid], L.pid.data(), n * 4);
    std::memcpy(&h[o_rad], L.radius.data(), n * 8);
    std::memcpy(&h[o_gof], L.group_of.data(), n * 8);
    std::memcpy(&h[o_rep], L.rep.data(), ng * 8);
    std::memcpy(&h[o_grow], L.grows_off.data(), (ng + 1) * 8);
    std::memcpy(&h[o_gmat], L.gmat_off.data(), (ng + 1) * 8);
    std::memcpy(&h[o_gfac], L.gfac_off.data(), (ng + 1) * 8);
    std::memcpy(&h[o_wrep], L.wrep.data(), nw * 8);
    std::memcpy(&h[o_wrow], L.wrows_off.data(), (nw + 1) * 8);
    std::memcpy(&h[o_kc], L.kcols.data(), nw * 8);
    std::memcpy(&h[o_gwo], L.gw_off.data(), (nw + 1) * 8);
    std::memcpy(&h[o_vec], L.vec_off.data(), (n + 1) * 8);
    std::memcpy(&h[o_mem], L.members.data(), n * 8);
    std::memcpy(&h[o_mof], L.mem_off.data(), (nw + 1) * 8);
    std::memcpy(&h[o_tof], L.tile_off.data(), (nw + 1) * 8);
    char *base = g->ws.layout.as<char>();
    e = cudaMemcpyAsync(base, h.data(), host_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    D.gamma_off = (int64_t *)(base + o_goff);
    D.panel_off = (int64_t *)(base + o_poff);
    D.mat_off = (int64_t *)(base + o_moff);
    D.walks = (int64_t *)(base + o_walk);
    D.chunk_off = (int64_t *)(base + o_coff);
    D.nt = (int32_t *)(base + o_nt);
    D.nph = (int32_t *)(base + o_nph);
    D.nr = (int32_t *)(base + o_nr);
    D.ns = (int32_t *)(base + o_ns);
    D.cpn = (int32_t *)(base + o_cpn);
    D.pid = (uint32_t *)(base + o_pid);
    D.radius = (double *)(base + o_rad);
    D.group_of = (int64_t *)(base + o_gof);
    D.rep = (int64_t *)(base + o_rep);
    D.grows_off = (int64_t *)(base + o_grow);
    D.gmat_off = (int64_t *)(base + o_gmat);
    D.gfac_off = (int64_t *)(base + o_gfac);
    D.wrep = (int64_t *)(base + o_wrep);
    D.wrows_off = (int64_t *)(base + o_wrow);
    D.kcols = (int64_t *)(base + o_kc);
    D.gw_off = (int64_t *)(base + o_gwo);
    D.vec_off = (int64_t *)(base + o_vec);
    D.members = (int64_t *)(base + o_mem);
    D.mem_off = (int64_t *)(base + o_mof);
    D.tile_off = (int64_t *)(base + o_tof);
    D.frames = (PatchFrame *)(base + o_fr);
    D.pieces = wrapped_possible ? (Piece *)(base + o_pc) : nullptr;
    return cudaSuccess;
}

}  // namespace

// Device bytes a dtn_solve_patches call on this batch reserves in a fresh
// geometry workspace (the buffers the call grows; an upper bound for a batch
// merged from several queries, whose shape groups are shared).
size_t solve_workspace_bytes(const dtn_patch_batch *b, const dtn_solve_opts *o, bool caps) {
    BatchLayout L;
    if (build_layout(b, L, caps) != DTN_OK) return 0;
    const size_t G = (size_t)L.gamma_total, Pn = (size_t)L.panels_total, n = (size_t)L.n_patches;
    size_t t = 40 * 256 + n * (200 + sizeof(PatchFrame)) + (size_t)(L.n_groups + L.n_wgroups) * 64;   // layout
    t += G * (3 + 1 + 3 + 1) * 8 + Pn * (3 + 6 + 4 + 1 + 1) * 8 + n * 4;   // nodes, panels, flags
    if (!o->u_provided) t += wos_scratch_bytes(L.gamma_total);
    if (o->prec == DTN_PREC_MIXED) {
        const size_t w = o->bie_kind == 1 ? 8 : 4;
        t += (size_t)L.gmat_total * 8 + lu_shared_scratch_bytes(L) + (size_t)L.grows_total * 4 +
             (size_t)(L.gw_total + L.vec_total) * w;
        if (!caps && o->bie_kind == 0) t += wrapped_static_bytes(L.panels_total);   // wrapped patches (box regions)
    } else {
        t += (size_t)L.matrix_total * 8 + lu_scratch_bytes(L, o->prec);
    }
    return t;
}

// Device bytes the geometry's workspaces hold now.
size_t workspace_bytes(const dtn_geometry *g) {
    const Workspace &W = g->ws;
    const DevBuf *bufs[] = {&W.layout, &W.gamma_loc, &W.gamma_w, &W.gamma_xyz, &W.panel_loc, &W.panel_prm,
                            &W.panel_aux, &W.panel_g, &W.mat, &W.lu32, &W.lu64, &W.rhs, &W.acc, &W.counter,
                            &W.se_tmp, &W.tune, &W.gmat, &W.gfac, &W.gpiv, &W.gw, &W.vec, &W.sp, &W.capflag,
                            &W.panel_piece, &W.kinds, &W.pstat};
    size_t t = 0;
    for (const DevBuf *d : bufs) t += d->bytes;
    return t;
}

namespace {

// Walk-kernel launch parameters: explicit opts fields win; fields left at 0 come
// from the autotuner's cache for (device name, region kind, precision), else
// from defaults (chunk 256, all resident blocks, refill at 8 idle lanes).
std::mutex g_tune_mu;
std::map<std::tuple<std::string, int, int>, dtn_tuning> g_tune;

struct WalkParams {
    int32_t chunk, bps, refill;
};

WalkParams walk_params(const dtn_geometry *g, const dtn_solve_opts *o) {
    WalkParams w{256, 0, 8};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(std::make_tuple(std::string(g->dev_name), g->dg.kind, o->prec));
        if (it != g_tune.end()) w = WalkParams{it->second.walk_chunk, it->second.wos_blocks_per_sm, it->second.wos_refill};
    }
    if (o->walk_chunk > 0) w.chunk = o->walk_chunk;
    if (o->wos_blocks_per_sm > 0) w.bps = o->wos_blocks_per_sm;
    if (o->wos_refill > 0) w.refill = o->wos_refill;
    return w;
}

cudaError_t enqueue_solve(dtn_geometry *g, const BatchLayout &L, const DevLayout &D, const dtn_solve_opts *o,
                          const WalkParams &wp, int64_t total_chunks, const dtn_patch_batch *b, dtn_patch_result *r,
                          double *gxyz, double *gw, double *pg, double *A, double *rhs, bool rec, cudaStream_t s);

}  // namespace
}  // namespace dtn

using namespace dtn;

extern "C" {

const char *dtn_status_string(dtn_status s) {
    switch (s) {
        case DTN_OK: return "ok";
        case DTN_E_INVALID_ARG: return "invalid argument";
        case DTN_E_OUT_OF_MEMORY: return "out of device memory";
        case DTN_E_CUDA: return "CUDA runtime error";
        case DTN_E_NOT_CONVERGED: return "refinement did not converge";
        case DTN_E_TIMEOUT: return "timed out";
        case DTN_E_UNSUPPORTED: return "unsupported patch or geometry";
        case DTN_E_WALK_CAP: return "walks cut at max_steps";
    }
    return "unknown status";
}

int32_t dtn_last_cuda_error(void) { return g_last_cuda_error.load(); }

dtn_status dtn_create_geometry(const dtn_geometry_desc *desc, dtn_geometry **out) {
    if (!desc || !out) return DTN_E_INVALID_ARG;
    *out = nullptr;
    const dtn_geometry_desc &d = *desc;
    if (d.kind == DTN_GEOM_BALL_INTERIOR) {
        if (!(d.radius > 0)) return DTN_E_INVALID_ARG;
    } else if (d.kind == DTN_GEOM_HALF_SPACE) {
        if (!(d.truncation > 0)) return DTN_E_INVALID_ARG;
    } else if (d.kind == DTN_GEOM_DISK_EXTERIOR || d.kind == DTN_GEOM_BALL_EXTERIOR) {
        if (!(d.radius > 0) || !(d.truncation > d.radius)) return DTN_E_INVALID_ARG;
    } else if (d.kind == DTN_GEOM_BOX_INTERIOR || d.kind == DTN_GEOM_BOX_MINUS_BOXES) {
        for (int i = 0; i < 3; ++i)
            if (!(d.hi[i] > d.lo[i])) return DTN_E_INVALID_ARG;
        if (d.kind == DTN_GEOM_BOX_MINUS_BOXES) {
            if (d.n_boxes < 0 || (d.n_boxes > 0 && !d.boxes)) return DTN_E_INVALID_ARG;
            for (int b = 0; b < d.n_boxes; ++b)
                for (int i = 0; i < 3; ++i) {
                    const double lo = d.boxes[6 * b + i], hi = d.boxes[6 * b + 3 + i];
                    if (!(hi > lo) || lo < d.lo[i] || hi > d.hi[i]) return DTN_E_INVALID_ARG;
                }
        }
    } else {
        return DTN_E_INVALID_ARG;
    }
    cudaError_t e = ensure_tables();
    if (e != cudaSuccess) return to_status(e);
    dtn_geometry *g = new dtn_geometry();
    g->host.desc = d;
    const int nb = d.kind == DTN_GEOM_BOX_MINUS_BOXES ? d.n_boxes : 0;
    g->host.boxes.assign(d.boxes ? d.boxes : nullptr, d.boxes ? d.boxes + 6 * nb : nullptr);
    g->host.desc.boxes = g->host.boxes.data();
    g->host.desc.n_boxes = nb;
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, g->device) == cudaSuccess)
            std::strncpy(g->dev_name, prop.name, sizeof(g->dev_name) - 1);
    }
    DGeom &dg = g->dg;
    std::memset(&dg, 0, sizeof(dg));
    dg.kind = d.kind;
    for (int i = 0; i < 3; ++i) {
        dg.c[i] = d.center[i];
        dg.lo[i] = d.lo[i];
        dg.hi[i] = d.hi[i];
    }
    dg.R = d.radius;
    for (int i = 0; i < 3; ++i) {
        dg.c_f[i] = (float)dg.c[i];
        dg.lo_f[i] = (float)dg.lo[i];
        dg.hi_f[i] = (float)dg.hi[i];
    }
    dg.R_f = (float)dg.R;
    dg.trunc = d.truncation;
    dg.trunc_f = (float)d.truncation;
    dg.nb = nb;
    dg.gn[0] = dg.gn[1] = dg.gn[2] = 1;
    dg.cell = 1.0;
    dg.inv_cell_f = 1.0f;
    if (d.kind == DTN_GEOM_BOX_MINUS_BOXES) {
        build_grid(g->host);
        std::vector<float> bf(g->host.boxes.begin(), g->host.boxes.end());
        const size_t nbx = std::max<size_t>(g->host.boxes.size(), 1);
        if ((e = g->d_boxes.reserve(nbx * sizeof(double))) != cudaSuccess ||
            (e = g->d_boxes_f.reserve(nbx * sizeof(float))) != cudaSuccess ||
            (e = g->d_cstart.reserve(g->host.cstart.size() * sizeof(int))) != cudaSuccess ||
            (e = g->d_citems.reserve(std::max<size_t>(g->host.citems.size(), 1) * sizeof(int))) != cudaSuccess ||
            (e = g->d_ccap.reserve(g->host.ccap.size() * sizeof(float))) != cudaSuccess) {
            delete g;
            return to_status(e);
        }
        cudaMemcpy(g->d_boxes.p, g->host.boxes.data(), g->host.boxes.size() * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(g->d_boxes_f.p, bf.data(), bf.size() * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(g->d_cstart.p, g->host.cstart.data(), g->host.cstart.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (!g->host.citems.empty())
            cudaMemcpy(g->d_citems.p, g->host.citems.data(), g->host.citems.size() * sizeof(int), cudaMemcpyHostToDevice);
        e = cudaMemcpy(g->d_ccap.p, g->host.ccap.data(), g->host.ccap.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            delete g;
            return to_status(e);
        }
        dg.boxes = g->d_boxes.as<double>();
        dg.boxes_f = g->d_boxes_f.as<float>();
        dg.cstart = g->d_cstart.as<int>();
        dg.citems = g->d_citems.as<int>();
        dg.ccap = g->d_ccap.as<float>();
        for (int i = 0; i < 3; ++i) {
            dg.gn[i] = g->host.gn[i];
            dg.glo[i] = g->host.glo[i];
            dg.glo_f[i] = (float)g->host.glo[i];
        }
        dg.cell = g->host.cell;
        dg.inv_cell_f = (float)(1.0 / g->host.cell);
    }
    std::memset(&g->dd, 0, sizeof(g->dd));
    g->dd.kind = DTN_DATA_CONSTANT;
    g->dd.inv_scale = 1.0;
    g->dd.inv_scale_f = 1.0f;
    g->dd.sh = sh_tables_dev();
    *out = g;
    return DTN_OK;
}

dtn_status dtn_destroy_geometry(dtn_geometry *g) {
    if (!g) return DTN_E_INVALID_ARG;
    cudaDeviceSynchronize();
    DevBuf *bufs[] = {&g->d_boxes, &g->d_boxes_f, &g->d_cstart, &g->d_citems, &g->d_ccap, &g->d_clm, &g->d_clm_f,
                      &g->d_clm_cart,
                      &g->ws.layout, &g->ws.gamma_loc, &g->ws.gamma_w, &g->ws.gamma_xyz, &g->ws.panel_loc,
                      &g->ws.panel_prm, &g->ws.panel_aux, &g->ws.panel_g, &g->ws.mat, &g->ws.lu32, &g->ws.lu64,
                      &g->ws.rhs, &g->ws.acc, &g->ws.counter, &g->ws.se_tmp, &g->ws.tune, &g->ws.gmat,
                      &g->ws.gfac, &g->ws.gpiv, &g->ws.gw, &g->ws.vec, &g->ws.sp, &g->ws.capflag,
                      &g->ws.panel_piece, &g->ws.kinds, &g->ws.pstat};
    for (DevBuf *b : bufs) b->release();
    fmm_release(g);
    for (int k = 0; k < 5; ++k)
        if (g->stage_ev[k]) cudaEventDestroy(g->stage_ev[k]);
    if (g->graph_exec) cudaGraphExecDestroy(g->graph_exec);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
    return DTN_OK;
}

dtn_status dtn_release_workspace(dtn_geometry *g) {
    if (!g) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    cudaDeviceSynchronize();
    Workspace &W = g->ws;
    DevBuf *bufs[] = {&W.layout, &W.gamma_loc, &W.gamma_w, &W.gamma_xyz, &W.panel_loc, &W.panel_prm, &W.panel_aux,
                      &W.panel_g, &W.mat, &W.lu32, &W.lu64, &W.rhs, &W.acc, &W.counter, &W.se_tmp, &W.tune,
                      &W.gmat, &W.gfac, &W.gpiv, &W.gw, &W.vec, &W.sp, &W.capflag, &W.panel_piece, &W.kinds,
                      &W.pstat};
    for (DevBuf *b : bufs) b->release();
    if (g->graph_exec) {   // a captured graph holds the old pointers
        cudaGraphExecDestroy(g->graph_exec);
        g->graph_exec = nullptr;
        g->graph_key.clear();
    }
    return DTN_OK;
}

dtn_status dtn_set_dirichlet(dtn_geometry *g, const dtn_dirichlet_desc *d) {
    if (!g || !d) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    DData &dd = g->dd;
    if (d->kind == DTN_DATA_HARMONIC_SH) {
        if (d->lmax < 0 || d->lmax > kMaxL || !d->clm || !(d->scale > 0)) return DTN_E_INVALID_ARG;
        const int nc = (d->lmax + 1) * (d->lmax + 1);
        std::vector<float> cf(d->clm, d->clm + nc);
        cudaError_t e;
        if ((e = g->d_clm.reserve(nc * sizeof(double))) != cudaSuccess) return to_status(e);
        if ((e = g->d_clm_f.reserve(nc * sizeof(float))) != cudaSuccess) return to_status(e);
        cudaDeviceSynchronize();
        if ((e = cudaMemcpy(g->d_clm.p, d->clm, nc * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
            return to_status(e);
        if ((e = cudaMemcpy(g->d_clm_f.p, cf.data(), nc * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
            return to_status(e);
        // FP32 pair table of the walk scoring: coefficients times the scale alpha_lm
        // of the recurrence T_lm = alpha_lm Q_lm (see harmonic_cart), formed in FP64
        // and rounded once
        std::vector<float2> cart(kShPairs, make_float2(0.f, 0.f));
        double pmm = 0.28209479177387814;   // Y00 = 1 / sqrt(4 pi)
        for (int m = 0; m <= d->lmax; ++m) {
            if (m > 0) pmm *= std::sqrt((2.0 * m + 1.0) / (2.0 * m));
            double alpha = m > 0 ? std::sqrt(2.0) * pmm : pmm;
            for (int l = m; l <= d->lmax; ++l) {
                if (l > m) alpha *= std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                cart[sh_pair(l, m)] = make_float2((float)(alpha * d->clm[l * l + l + m]),
                                                  m > 0 ? (float)(alpha * d->clm[l * l + l - m]) : 0.f);
            }
        }
        if ((e = g->d_clm_cart.reserve(kShPairs * sizeof(float2))) != cudaSuccess) return to_status(e);
        if ((e = cudaMemcpy(g->d_clm_cart.p, cart.data(), kShPairs * sizeof(float2), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return to_status(e);
        dd.clm = g->d_clm.as<double>();
        dd.clm_f = g->d_clm_f.as<float>();
        dd.cart = g->d_clm_cart.as<float2>();
        dd.lmax = d->lmax;
    } else if (d->kind != DTN_DATA_POINT_SOURCE && d->kind != DTN_DATA_CONSTANT) {
        return DTN_E_INVALID_ARG;
    }
    dd.kind = d->kind;
    for (int i = 0; i < 3; ++i) {
        dd.x0[i] = d->x0[i];
        dd.ctr[i] = d->center[i];
    }
    dd.strength = d->strength;
    dd.inv_scale = d->kind == DTN_DATA_HARMONIC_SH ? 1.0 / d->scale : 1.0;
    dd.constant = d->constant;
    for (int i = 0; i < 3; ++i) {
        dd.x0_f[i] = (float)dd.x0[i];
        dd.ctr_f[i] = (float)dd.ctr[i];
    }
    dd.q_f = (float)(dd.strength / (4.0 * kPi));
    dd.inv_scale_f = (float)dd.inv_scale;
    dd.constant_f = (float)dd.constant;
    dd.sh = sh_tables_dev();
    g->score_bound = std::max(score_bound(g->host.desc, *d), 1e-300);
    g->data_version += 1;
    g->host.data = *d;
    if (d->kind == DTN_DATA_HARMONIC_SH) {
        g->host.clm.assign(d->clm, d->clm + (d->lmax + 1) * (d->lmax + 1));
        g->host.data.clm = g->host.clm.data();
    } else {
        g->host.clm.clear();
        g->host.data.clm = nullptr;
    }
    g->has_data = true;
    return DTN_OK;
}

dtn_status dtn_query_patch_sizes(const dtn_patch_batch *b, int64_t *panels_total, int64_t *gamma_total,
                                 int64_t *matrix_total) {
    if (!b || b->n_patches < 0) return DTN_E_INVALID_ARG;
    if (b->n_patches > 0 && (!b->n_theta || !b->n_phi || !b->n_rings || !b->n_sectors)) return DTN_E_INVALID_ARG;
    BatchLayout L;
    dtn_status st = build_layout(b, L, false);
    if (st != DTN_OK) return st;
    if (panels_total) *panels_total = L.panels_total;
    if (gamma_total) *gamma_total = L.gamma_total;
    if (matrix_total) *matrix_total = L.matrix_total;
    return DTN_OK;
}

dtn_status dtn_solve_patches(dtn_geometry *g, const dtn_patch_batch *b, const dtn_solve_opts *o,
                             dtn_patch_result *r, void *stream) {
    if (!g || !b || !o || !r) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (b->n_patches < 0) return DTN_E_INVALID_ARG;
    if (b->n_patches == 0) return DTN_OK;
    if (!b->centers || !b->radius || !b->n_theta || !b->n_phi || !b->n_rings || !b->n_sectors) return DTN_E_INVALID_ARG;
    if (!r->u_gamma_mean || !r->neumann) return DTN_E_INVALID_ARG;
    if (o->prec != DTN_PREC_FP64 && o->prec != DTN_PREC_MIXED) return DTN_E_INVALID_ARG;
    if (o->bie_kind != 0 && o->bie_kind != 1) return DTN_E_INVALID_ARG;
    if (o->ring_order < 0 || o->ring_order > kMaxGauss) return DTN_E_INVALID_ARG;
    // the second-kind rows are written for flat patches (the double layer vanishes there)

    if (!o->u_provided) {
        if (!b->walks_per_point || !(o->epsilon > 0)) return DTN_E_INVALID_ARG;
        for (int64_t p = 0; p < b->n_patches; ++p)
            if (b->walks_per_point[p] < 2 || b->walks_per_point[p] > 0xFFFFFFFFll) return DTN_E_INVALID_ARG;
    }
    if (!g->has_data) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    cudaStream_t s = (cudaStream_t)stream;
    BatchLayout L;
    // Mixed precision shares one matrix among congruent patches; on an obstacle
    // region a wrapped patch (the ball meets several faces of a box) is
    // congruent to no other.  Which patches wrap is read back from a frames
    // pass on the device before the batch is grouped (this synchronises s).
    std::vector<uint8_t> wrapped;
    if (g->dg.kind == kBoxMinusBoxes && o->prec == DTN_PREC_MIXED && o->bie_kind == 0) {
        const int64_t n = b->n_patches;
        for (int64_t p = 0; p < n; ++p)
            if (!(b->radius[p] > 0.0)) return DTN_E_INVALID_ARG;
        cudaError_t e;
        const size_t fbytes = ((size_t)n * sizeof(PatchFrame) + 255) & ~(size_t)255;
        if ((e = g->ws.kinds.reserve(fbytes + (size_t)n * sizeof(double), s)) != cudaSuccess) return to_status(e);
        PatchFrame *fr = g->ws.kinds.as<PatchFrame>();
        double *rad = (double *)(g->ws.kinds.as<char>() + fbytes);
        std::vector<int32_t> kinds(n);
        if ((e = cudaMemcpyAsync(rad, b->radius, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s)) !=
                cudaSuccess ||
            (e = launch_patch_frames(g, n, b->centers, rad, fr, s)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(kinds.data(), sizeof(int32_t), &fr->kind, sizeof(PatchFrame), sizeof(int32_t),
                                   (size_t)n, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return to_status(e);
        wrapped.resize(n);
        for (int64_t p = 0; p < n; ++p) wrapped[p] = (kinds[p] == kWrapped) ? 1 : 0;
    }
    dtn_status st = build_layout(b, L, g->dg.kind == kBall || g->dg.kind == kBallExterior,
                                 wrapped.empty() ? nullptr : wrapped.data());
    if (st != DTN_OK) return st;
    const WalkParams wp = walk_params(g, o);
    const int32_t chunk = wp.chunk;
    DevLayout D;
    int64_t total_chunks = 0;
    cudaError_t e = upload_layout(g, L, chunk, D, total_chunks, s);
    if (e != cudaSuccess) return to_status(e);
    Workspace &W = g->ws;
    const size_t G = (size_t)L.gamma_total, Pn = (size_t)L.panels_total;
    if ((e = W.gamma_loc.reserve(G * 3 * 8, s)) != cudaSuccess || (e = W.gamma_w.reserve(G * 8, s)) != cudaSuccess ||
        (e = W.gamma_xyz.reserve(G * 3 * 8, s)) != cudaSuccess ||
        (e = W.panel_loc.reserve(Pn * 3 * 8, s)) != cudaSuccess ||
        (e = W.panel_prm.reserve(Pn * 6 * 8, s)) != cudaSuccess ||
        (e = W.panel_aux.reserve(Pn * 4 * 8, s)) != cudaSuccess || (e = W.panel_g.reserve(Pn * 8, s)) != cudaSuccess ||
        (e = W.rhs.reserve(Pn * 8, s)) != cudaSuccess || (e = W.se_tmp.reserve(G * 8, s)) != cudaSuccess ||
        (e = W.capflag.reserve((size_t)L.n_patches * sizeof(int32_t), s)) != cudaSuccess ||
        (e = W.panel_piece.reserve(Pn * sizeof(int32_t), s)) != cudaSuccess ||
        (!o->u_provided && (e = W.acc.reserve(wos_scratch_bytes(L.gamma_total), s)) != cudaSuccess))
        return to_status(e);
    const bool shared = (o->prec == DTN_PREC_MIXED);
    if (shared) {
        if ((e = W.gmat.reserve((size_t)L.gmat_total * 8, s)) != cudaSuccess ||
            (e = W.gfac.reserve(lu_shared_scratch_bytes(L), s)) != cudaSuccess ||
            (e = W.gpiv.reserve((size_t)L.grows_total * 4, s)) != cudaSuccess ||
            (e = W.gw.reserve((size_t)L.gw_total * (o->bie_kind == 1 ? sizeof(double) : sizeof(float)), s)) !=
                cudaSuccess ||
            (e = W.vec.reserve((size_t)L.vec_total * (o->bie_kind == 1 ? sizeof(double) : sizeof(float)), s)) !=
                cudaSuccess)
            return to_status(e);
        if (std::find(L.wrapped.begin(), L.wrapped.end(), 1) != L.wrapped.end() &&
            (e = W.pstat.reserve(wrapped_static_bytes(L.panels_total), s)) != cudaSuccess)
            return to_status(e);

    } else {
        if (!r->matrix && (e = W.mat.reserve((size_t)L.matrix_total * 8, s)) != cudaSuccess) return to_status(e);
        const size_t lus = lu_scratch_bytes(L, o->prec);
        if (lus && (e = W.lu64.reserve(lus, s)) != cudaSuccess) return to_status(e);
    }
    double *gxyz = r->gamma_xyz ? r->gamma_xyz : W.gamma_xyz.as<double>();
    double *gw = r->gamma_w ? r->gamma_w : W.gamma_w.as<double>();
    double *pg = r->dirichlet ? r->dirichlet : W.panel_g.as<double>();
    double *A = r->matrix ? r->matrix : W.mat.as<double>();
    double *rhs = r->rhs ? r->rhs : W.rhs.as<double>();
    const bool rec = o->record_stages != 0;
    if (rec) {
        for (int k = 0; k < 5; ++k)
            if (!g->stage_ev[k] && (e = cudaEventCreate(&g->stage_ev[k])) != cudaSuccess) return to_status(e);
        g->stages_recorded = true;
    }
    if (o->graph_capture) {
        // every buffer the device part touches is reserved above, before capture,
        // so the captured graph allocates nothing and its pointers stay valid
        // while the key (shapes, pointers, options, data version) repeats
        if ((e = W.acc.reserve(wos_scratch_bytes(L.gamma_total), s)) != cudaSuccess) return to_status(e);
        std::vector<unsigned char> key;
        auto put = [&key](const void *p, size_t n) {
            const unsigned char *c = (const unsigned char *)p;
            key.insert(key.end(), c, c + n);
        };
        put(L.nt.data(), L.nt.size() * 4); put(L.nph.data(), L.nph.size() * 4);
        put(L.nr.data(), L.nr.size() * 4); put(L.ns.data(), L.ns.size() * 4);
        put(L.walks.data(), L.walks.size() * 8); put(L.pid.data(), L.pid.size() * 4);
        put(L.radius.data(), L.radius.size() * 8);
        put(L.wrapped.data(), L.wrapped.size());
        put(&wp, sizeof(wp)); put(o, sizeof(*o)); put(&b->centers, sizeof(void *));
        put(r, sizeof(*r)); put(&g->data_version, sizeof(g->data_version));
        const DevBuf *bufs[] = {&W.layout, &W.gamma_loc, &W.gamma_w, &W.gamma_xyz, &W.panel_loc, &W.panel_prm,
                                &W.panel_aux, &W.panel_g, &W.mat, &W.lu32, &W.lu64, &W.rhs, &W.acc, &W.se_tmp,
                                &W.gmat, &W.gfac, &W.gpiv, &W.gw, &W.vec, &W.capflag, &W.panel_piece, &W.pstat};
        for (const DevBuf *d : bufs) put(&d->p, sizeof(void *));
        if (!(g->graph_exec && key == g->graph_key)) {
            if (g->graph_exec) {
                cudaGraphExecDestroy(g->graph_exec);
                g->graph_exec = nullptr;
            }
            // capture on a private stream (the legacy default stream cannot be
            // captured); the graph is then launched on the caller's stream
            if (!g->cap_stream && (e = cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
                return to_status(e);
            if ((e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
                return to_status(e);
            // (stage events are not recorded inside the graph: the whole replay is
            // timed instead, see below)
            cudaError_t ce = enqueue_solve(g, L, D, o, wp, total_chunks, b, r, gxyz, gw, pg, A, rhs, false,
                                           g->cap_stream);
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(g->cap_stream, &graph);
            if (ce != cudaSuccess) e = ce;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&g->graph_exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                g->graph_exec = nullptr;
                return to_status(e);
            }
            g->graph_key.swap(key);
        }
        // a replay is timed as a whole: stage 0 spans the graph, stages 1-3 are empty
        if (rec && (e = cudaEventRecord(g->stage_ev[0], s)) != cudaSuccess) return to_status(e);
        e = cudaGraphLaunch(g->graph_exec, s);
        if (e == cudaSuccess && rec) {
            e = cudaEventRecord(g->stage_ev[1], s);
            for (int k = 2; k < 5 && e == cudaSuccess; ++k) e = cudaEventRecord(g->stage_ev[k], s);
        }
        return to_status(e);
    }
    return to_status(enqueue_solve(g, L, D, o, wp, total_chunks, b, r, gxyz, gw, pg, A, rhs, rec, s));
}

}  // extern "C"

namespace dtn {
namespace {

// The device part of a batch solve: setup, walks, assembly, solve, enqueued on s.
cudaError_t enqueue_solve(dtn_geometry *g, const BatchLayout &L, const DevLayout &D, const dtn_solve_opts *o,
                          const WalkParams &wp, int64_t total_chunks, const dtn_patch_batch *b, dtn_patch_result *r,
                          double *gxyz, double *gw, double *pg, double *A, double *rhs, bool rec, cudaStream_t s) {
    Workspace &W = g->ws;
    cudaError_t e;
    const int32_t chunk = wp.chunk;
    auto mark = [&](int k) -> cudaError_t { return rec ? cudaEventRecord(g->stage_ev[k], s) : cudaSuccess; };
    if ((e = mark(0)) != cudaSuccess) return e;
    // 1. patch setup
    e = launch_patch_setup(g, L, D, b->centers, gxyz, gw, W.gamma_loc.as<double>(), r->colloc_xyz,
                           r->normals, r->areas, W.panel_loc.as<double>(), W.panel_prm.as<double>(),
                           W.panel_aux.as<double>(), pg, W.panel_piece.as<int32_t>(), s);
    if (e != cudaSuccess) return e;
    if ((e = mark(1)) != cudaSuccess) return e;
    // 2. walks at the hemisphere nodes (step 1 of the BIE-WOS algorithm)
    if (!o->u_provided) {
        WosLaunch w{};
        w.n_groups = L.n_patches;
        w.node_off = D.gamma_off;
        w.walks = D.walks;
        w.pid = D.pid;
        w.point_id = nullptr;
        w.chunk_off = D.chunk_off;
        w.cpn = D.cpn;
        w.total_chunks = total_chunks;
        w.total_nodes = L.gamma_total;
        w.chunk = chunk;
        w.max_walks = L.max_walks;
        w.y = gxyz;
        w.prec = o->prec;
        w.eps = o->epsilon;
        w.max_steps = o->max_steps ? o->max_steps : 1000000ull;
        w.seed = o->seed;
        w.blocks_per_sm = wp.bps;
        w.refill = wp.refill;
        w.mean = r->u_gamma_mean;
        w.se = r->u_gamma_se ? r->u_gamma_se : W.se_tmp.as<double>();
        w.steps = r->gamma_steps;
        w.capped = r->gamma_capped;
        w.group_capped = W.capflag.as<int32_t>();
        if ((e = launch_wos(g, w, s)) != cudaSuccess) return e;
    }
    // after the solve: DTN_E_WALK_CAP where a patch had walks cut and no other error
    auto walk_cap = [&]() -> cudaError_t {
        return o->u_provided ? cudaSuccess
                             : launch_walk_cap_status(L.n_patches, W.capflag.as<int32_t>(), r->patch_status, s);
    };
    if ((e = mark(2)) != cudaSuccess) return e;
    const bool caps = (g->dg.kind == kBall || g->dg.kind == kBallExterior);
    // 3-4. second kind (Eq. bw55-bw59) on disk patches: q = 2b row by row, no system
    if (o->bie_kind == 1 && !caps) {
        e = launch_second_kind(g, L, D, W.panel_loc.as<double>(), pg, W.gamma_loc.as<double>(), gw, r->u_gamma_mean,
                               o->ring_order > 0 ? o->ring_order : 20, r->neumann, r->rhs, r->refine_iters,
                               r->residual, r->patch_status, s);
        if (e == cudaSuccess) e = walk_cap();
        if (e == cudaSuccess) e = mark(3);
        if (e == cudaSuccess) e = mark(4);
        return e;
    }
    // 3. assembly of Eq. bw49-bw51 (step 2)
    const double *pl = W.panel_loc.as<double>(), *pp = W.panel_prm.as<double>(), *pa = W.panel_aux.as<double>();
    const bool shared = (o->prec == DTN_PREC_MIXED);
    if (o->bie_kind == 1) {
        // second kind on cap patches: (1/2 I - D) q = b.  Mixed precision: D per
        // shape group (FP64 rules), the right sides by the geodesic polar rule
        // about each collocation point folded into FP64 weights per weight group
        // and one FP64 product per patch, FP32 group factors with FP64
        // refinement; FP64: matrix and right side per patch with the panel rules.
        if (shared) {
            e = launch_assemble(g, L, D, o->prec, 1, pl, pp, pa, pg, W.gamma_loc.as<double>(), gw, r->u_gamma_mean,
                                W.gmat.as<double>(), rhs, s, 1);
            if (e == cudaSuccess)
                e = launch_second_kind_cap_rhs_shared(g, L, D, pl, pp, W.gamma_loc.as<double>(), gw,
                                                      r->u_gamma_mean, o->ring_order > 0 ? o->ring_order : 32,
                                                      W.gw.as<double>(), W.vec.as<double>(), rhs, s);
            if (e == cudaSuccess && r->matrix) e = launch_expand_matrices(L, D, W.gmat.as<double>(), r->matrix, s);
        } else {
            e = launch_assemble(g, L, D, o->prec, 0, pl, pp, pa, pg, W.gamma_loc.as<double>(), gw, r->u_gamma_mean, A,
                                rhs, s, 1);
        }
    } else if (shared) {
        // one matrix and one set of right-side weights per patch shape, FP64
        // rules; the right sides of all patches of a shape as one product
        double *gA = W.gmat.as<double>();
        e = launch_assemble(g, L, D, o->prec, 1, pl, pp, pa, pg, W.gamma_loc.as<double>(), gw, r->u_gamma_mean,
                            gA, rhs, s);
        if (e == cudaSuccess)
            e = launch_rhs_shared(g, L, D, pl, pp, pa, pg, W.gamma_loc.as<double>(), gw, r->u_gamma_mean,
                                  W.gw.as<float>(), W.vec.as<float>(), rhs, s);
        // wrapped patches (groups of their own): matrix rows and right sides by
        // the panel rules, row by row
        if (e == cudaSuccess && std::find(L.wrapped.begin(), L.wrapped.end(), 1) != L.wrapped.end())
            e = launch_assemble(g, L, D, o->prec, 2, pl, pp, pa, pg, W.gamma_loc.as<double>(), gw, r->u_gamma_mean,
                                gA, rhs, s, 0, 1, W.pstat.p);
        if (e == cudaSuccess && r->matrix) e = launch_expand_matrices(L, D, gA, r->matrix, s);
    } else {
        e = launch_assemble(g, L, D, o->prec, 0, pl, pp, pa, pg, W.gamma_loc.as<double>(), gw, r->u_gamma_mean, A,
                            rhs, s);
    }
    if (e != cudaSuccess) return e;
    if ((e = mark(3)) != cudaSuccess) return e;
    // 4. collocation solve
    const int iters = o->max_refine_iters > 0 ? o->max_refine_iters : 10;
    const double tol = o->refine_tol > 0 ? o->refine_tol : 1e-12;
    if (shared)
        e = launch_lu_shared(g, L, D, W.gmat.as<double>(), rhs, r->neumann, iters, tol, r->refine_iters, r->residual,
                             r->patch_status, s);
    else
        e = launch_lu_solve(g, L, D, o->prec, A, rhs, r->neumann, iters, tol, r->refine_iters, r->residual,
                            r->patch_status, s);
    if (e == cudaSuccess) e = walk_cap();
    if (e == cudaSuccess) e = mark(4);
    return e;
}

}  // namespace
}  // namespace dtn

extern "C" {

dtn_status dtn_autotune_walks(dtn_geometry *g, const dtn_patch_batch *b, const dtn_solve_opts *o, dtn_tuning *out,
                              void *stream) {
    if (!g || !b || !o || b->n_patches < 1 || !b->centers || !b->radius || !b->walks_per_point) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (!b->n_theta || !b->n_phi || !b->n_rings || !b->n_sectors || !(o->epsilon > 0)) return DTN_E_INVALID_ARG;
    if (o->prec != DTN_PREC_FP64 && o->prec != DTN_PREC_MIXED) return DTN_E_INVALID_ARG;
    if (!g->has_data) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    cudaStream_t s = (cudaStream_t)stream;
    // sample: the first patches (enough work for several waves of chunks, so the
    // tail of the launch does not decide), walks capped
    const int64_t n = std::min<int64_t>(b->n_patches, 96);
    std::vector<int64_t> walks(n);
    for (int64_t p = 0; p < n; ++p) walks[p] = std::max<int64_t>(2, std::min<int64_t>(b->walks_per_point[p], 4096));
    dtn_patch_batch sb = *b;
    sb.n_patches = n;
    sb.walks_per_point = walks.data();
    BatchLayout L;
    dtn_status st = build_layout(&sb, L, g->dg.kind == kBall || g->dg.kind == kBallExterior);
    if (st != DTN_OK) return st;
    DevLayout D;
    int64_t total_chunks = 0;
    cudaError_t e = upload_layout(g, L, 256, D, total_chunks, s);
    if (e != cudaSuccess) return to_status(e);
    Workspace &W = g->ws;
    const size_t G = (size_t)L.gamma_total, Pn = (size_t)L.panels_total;
    if ((e = W.gamma_loc.reserve(G * 3 * 8)) != cudaSuccess || (e = W.gamma_w.reserve(G * 8)) != cudaSuccess ||
        (e = W.gamma_xyz.reserve(G * 3 * 8)) != cudaSuccess || (e = W.panel_loc.reserve(Pn * 3 * 8)) != cudaSuccess ||
        (e = W.panel_prm.reserve(Pn * 6 * 8)) != cudaSuccess || (e = W.panel_aux.reserve(Pn * 4 * 8)) != cudaSuccess ||
        (e = W.panel_g.reserve(Pn * 8)) != cudaSuccess || (e = W.tune.reserve(G * 8 * 3)) != cudaSuccess ||
        (e = W.panel_piece.reserve(Pn * sizeof(int32_t))) != cudaSuccess)
        return to_status(e);
    e = launch_patch_setup(g, L, D, b->centers, W.gamma_xyz.as<double>(), W.gamma_w.as<double>(),
                           W.gamma_loc.as<double>(), nullptr, nullptr, nullptr, W.panel_loc.as<double>(),
                           W.panel_prm.as<double>(), W.panel_aux.as<double>(), W.panel_g.as<double>(),
                           W.panel_piece.as<int32_t>(), s);
    if (e != cudaSuccess) return to_status(e);
    double *mean = W.tune.as<double>(), *se = mean + G;
    uint64_t *steps = (uint64_t *)(se + G);
    cudaEvent_t e0, e1;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess) return to_status(e);
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) { cudaEventDestroy(e0); return to_status(e); }
    dtn_tuning best{256, 0, 8, 1e30f};
    uint64_t total_steps = 0;
    const int chunks[4] = {64, 128, 256, 512}, bpss[5] = {5, 6, 7, 8, 9}, refills[4] = {4, 8, 12, 16};
    for (int ci = 0; ci < 4 && e == cudaSuccess; ++ci) {
        if ((e = upload_layout(g, L, chunks[ci], D, total_chunks, s)) != cudaSuccess) break;
        for (int bi = 0; bi < 5 && e == cudaSuccess; ++bi)
            for (int ri = 0; ri < 4 && e == cudaSuccess; ++ri) {
                WosLaunch w{};
                w.n_groups = L.n_patches;
                w.node_off = D.gamma_off;
                w.walks = D.walks;
                w.pid = D.pid;
                w.chunk_off = D.chunk_off;
                w.cpn = D.cpn;
                w.total_chunks = total_chunks;
                w.total_nodes = L.gamma_total;
                w.chunk = chunks[ci];
                w.max_walks = L.max_walks;
                w.y = W.gamma_xyz.as<double>();
                w.prec = o->prec;
                w.eps = o->epsilon;
                w.max_steps = o->max_steps ? o->max_steps : 1000000ull;
                w.seed = o->seed;
                w.blocks_per_sm = bpss[bi];
                w.refill = refills[ri];
                w.mean = mean;
                w.se = se;
                w.steps = steps;
                float ms = 1e30f;
                for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the faster of two runs
                    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
                    if ((e = launch_wos(g, w, s)) != cudaSuccess) break;
                    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
                    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
                    float t = 0.f;
                    cudaEventElapsedTime(&t, e0, e1);
                    ms = std::min(ms, t);
                }
                if (e != cudaSuccess) break;
                if (total_steps == 0) {
                    std::vector<uint64_t> hs(G);
                    if ((e = cudaMemcpy(hs.data(), steps, G * 8, cudaMemcpyDeviceToHost)) != cudaSuccess) break;
                    for (uint64_t v : hs) total_steps += v;
                }
                const float ns = (float)(ms * 1e6 / (double)std::max<uint64_t>(total_steps, 1));
                if (ns < best.ns_per_walk_step) best = dtn_tuning{chunks[ci], bpss[bi], refills[ri], ns};
            }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return to_status(e);
    {
        std::lock_guard<std::mutex> tl(g_tune_mu);
        g_tune[std::make_tuple(std::string(g->dev_name), g->dg.kind, o->prec)] = best;
    }
    if (out) *out = best;
    return DTN_OK;
}

dtn_status dtn_stage_times(dtn_geometry *g, float ms[4]) {
    if (!g || !ms || !g->stages_recorded) return DTN_E_INVALID_ARG;
    cudaError_t e = cudaEventSynchronize(g->stage_ev[4]);
    if (e != cudaSuccess) return to_status(e);
    for (int k = 0; k < 4; ++k)
        if ((e = cudaEventElapsedTime(&ms[k], g->stage_ev[k], g->stage_ev[k + 1])) != cudaSuccess) return to_status(e);
    return DTN_OK;
}

dtn_status dtn_eval_potential(const dtn_geometry *g, int64_t np, const double *xyz, const double *nrm,
                              const double *area, const double *q, const double *gv, const int64_t *index,
                              const int64_t *n_index, int64_t nt, const double *t, double *out, int32_t prec,
                              void *stream) {
    if (!g || np < 0 || nt < 0) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (nt == 0) return DTN_OK;
    if (!t || !out || (np > 0 && (!xyz || !nrm || !area || !q))) return DTN_E_INVALID_ARG;
    if (prec != DTN_PREC_FP64 && prec != DTN_PREC_MIXED) return DTN_E_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    double *tmp = nullptr;
    if (!gv && np > 0) {
        if (!g->has_data) return DTN_E_INVALID_ARG;
        if ((e = cudaMallocAsync((void **)&tmp, np * sizeof(double), s)) != cudaSuccess) return to_status(e);
        if ((e = launch_dirichlet(g, np, xyz, tmp, s)) != cudaSuccess) return to_status(e);
        gv = tmp;
    }
    e = launch_potential(np, index, n_index, xyz, nrm, area, q, gv, nt, t, out, prec, g->num_sms, s);
    if (tmp) cudaFreeAsync(tmp, s);
    return to_status(e);
}

dtn_status dtn_gather_owned(int64_t np, const double *x, const int64_t *owner, int64_t nc, const double *cent,
                            uint8_t *keep, int64_t *kept, int64_t *n_kept, void *stream) {
    if (np < 0 || nc < 0 || !n_kept) return DTN_E_INVALID_ARG;
    if (np > 0 && (!x || !owner || !keep || !kept || nc == 0 || !cent)) return DTN_E_INVALID_ARG;
    return to_status(launch_gather(np, x, owner, nc, cent, keep, kept, n_kept, (cudaStream_t)stream));
}

dtn_status dtn_wos_points(const dtn_geometry *gc, int64_t n, const double *y, const uint32_t *point_ids,
                          const uint32_t *patch_ids, const int64_t *walks, const dtn_solve_opts *o, double *mean,
                          double *se, uint64_t *steps, uint32_t *capped, void *stream) {
    dtn_geometry *g = const_cast<dtn_geometry *>(gc);
    if (!g || n < 0 || !o) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (n == 0) return DTN_OK;
    if (!y || !point_ids || !patch_ids || !walks || !mean || !(o->epsilon > 0)) return DTN_E_INVALID_ARG;
    if (o->prec != DTN_PREC_FP64 && o->prec != DTN_PREC_MIXED) return DTN_E_INVALID_ARG;
    if (!g->has_data) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    cudaStream_t s = (cudaStream_t)stream;
    int64_t maxw = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (walks[i] < 2 || walks[i] > 0xFFFFFFFFll) return DTN_E_INVALID_ARG;
        maxw = std::max(maxw, walks[i]);
    }
    const WalkParams wp = walk_params(g, o);
    const int32_t chunk = wp.chunk;
    std::vector<int64_t> node_off(n + 1), chunk_off(n + 1, 0);
    std::vector<int32_t> cpn(n);
    for (int64_t i = 0; i <= n; ++i) node_off[i] = i;
    for (int64_t i = 0; i < n; ++i) {
        cpn[i] = (int32_t)((walks[i] + chunk - 1) / chunk);
        chunk_off[i + 1] = chunk_off[i] + cpn[i];
    }
    // device staging: node_off, chunk_off, walks, cpn
    const size_t bytes = (size_t)(3 * (n + 1)) * 8 + (size_t)n * 4 + 64;
    cudaError_t e = g->ws.counter.reserve(bytes);
    if (e != cudaSuccess) return to_status(e);
    char *base = g->ws.counter.as<char>();
    int64_t *d_node = (int64_t *)base, *d_chunk = d_node + (n + 1), *d_walks = d_chunk + (n + 1);
    int32_t *d_cpn = (int32_t *)(d_walks + (n + 1));
    if ((e = cudaMemcpyAsync(d_node, node_off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_chunk, chunk_off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_walks, walks, n * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_cpn, cpn.data(), n * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return to_status(e);
    WosLaunch w{};
    w.n_groups = n;
    w.node_off = d_node;
    w.walks = d_walks;
    w.pid = patch_ids;
    w.point_id = point_ids;
    w.chunk_off = d_chunk;
    w.cpn = d_cpn;
    w.total_chunks = chunk_off[n];
    w.total_nodes = n;
    w.chunk = chunk;
    w.max_walks = maxw;
    w.y = y;
    w.prec = o->prec;
    w.eps = o->epsilon;
    w.max_steps = o->max_steps ? o->max_steps : 1000000ull;
    w.seed = o->seed;
    w.blocks_per_sm = wp.bps;
    w.refill = wp.refill;
    w.mean = mean;
    if (!se) {
        if ((e = g->ws.se_tmp.reserve(n * 8)) != cudaSuccess) return to_status(e);
        se = g->ws.se_tmp.as<double>();
    }
    w.se = se;
    w.steps = steps;
    w.capped = capped;
    e = launch_wos(g, w, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging vectors go out of scope
    return to_status(e);
}

dtn_status dtn_single_point_neumann(dtn_geometry *g, int64_t n, const double *x, double a, int32_t ng1, int32_t ng2,
                                    double delta, const int64_t *walks, uint32_t patch_id_base,
                                    const dtn_solve_opts *o, double *sigma1, double *sigma2, double *q, double *se,
                                    int32_t *status, double *U, void *stream) {
    if (!g || n < 0 || !o) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (n == 0) return DTN_OK;
    if (!x || !walks || !q || !(a > 0) || !(delta >= 0) || !(delta < a)) return DTN_E_INVALID_ARG;
    if (ng1 < 1 || ng1 > kMaxGauss || ng2 < 1 || ng2 > kMaxGauss || !(o->epsilon > 0)) return DTN_E_INVALID_ARG;
    if (o->prec != DTN_PREC_FP64 && o->prec != DTN_PREC_MIXED) return DTN_E_INVALID_ARG;
    if (!g->has_data) return DTN_E_INVALID_ARG;
    int64_t maxw = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (walks[i] < 2 || walks[i] > 0xFFFFFFFFll) return DTN_E_INVALID_ARG;
        maxw = std::max(maxw, walks[i]);
    }
    std::lock_guard<std::mutex> lk(g->mu);
    cudaStream_t s = (cudaStream_t)stream;
    const WalkParams wp = walk_params(g, o);
    const int32_t chunk = wp.chunk;
    const int64_t nn = (int64_t)ng1 * ng1, nodes = n * nn;
    // walk layout: one group per point, its ng1^2 nodes
    std::vector<int64_t> node_off(n + 1), chunk_off(n + 1, 0), wv(walks, walks + n);
    std::vector<int32_t> cpn(n);
    std::vector<uint32_t> pid(n);
    std::vector<double> rad(n, a);
    for (int64_t i = 0; i <= n; ++i) node_off[i] = i * nn;
    for (int64_t i = 0; i < n; ++i) {
        cpn[i] = (int32_t)((walks[i] + chunk - 1) / chunk);
        chunk_off[i + 1] = chunk_off[i] + nn * cpn[i];
        pid[i] = patch_id_base + (uint32_t)i;
    }
    auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
    size_t off = 0;
    const size_t o_node = off; off = al(off + (n + 1) * 8);
    const size_t o_chunk = off; off = al(off + (n + 1) * 8);
    const size_t o_walk = off; off = al(off + n * 8);
    const size_t o_cpn = off; off = al(off + n * 4);
    const size_t o_pid = off; off = al(off + n * 4);
    const size_t o_rad = off; off = al(off + n * 8);
    const size_t host_bytes = off;
    const size_t o_fr = off; off = al(off + n * sizeof(PatchFrame));
    // pieces of wrapped patches (obstacle regions only)
    const bool wrapped_possible = (g->dg.kind == kBoxMinusBoxes);
    const size_t o_pc = off; off = al(off + (wrapped_possible ? n * kMaxPieces * sizeof(Piece) : 0));
    const size_t o_y = off; off = al(off + nodes * 24);
    const size_t o_wk = off; off = al(off + nodes * 8);
    const size_t o_U = off; off = al(off + nodes * 8);
    const size_t o_SE = off; off = al(off + nodes * 8);
    cudaError_t e = g->ws.sp.reserve(off);
    if (e != cudaSuccess) return to_status(e);
    std::vector<unsigned char> h(host_bytes, 0);
    std::memcpy(&h[o_node], node_off.data(), (n + 1) * 8);
    std::memcpy(&h[o_chunk], chunk_off.data(), (n + 1) * 8);
    std::memcpy(&h[o_walk], wv.data(), n * 8);
    std::memcpy(&h[o_cpn], cpn.data(), n * 4);
    std::memcpy(&h[o_pid], pid.data(), n * 4);
    std::memcpy(&h[o_rad], rad.data(), n * 8);
    char *base = g->ws.sp.as<char>();
    if ((e = cudaMemcpyAsync(base, h.data(), host_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return to_status(e);
    PatchFrame *frames = (PatchFrame *)(base + o_fr);
    double *y = (double *)(base + o_y), *wk = (double *)(base + o_wk);
    double *Ud = U ? U : (double *)(base + o_U);
    double *SEd = (double *)(base + o_SE);
    if ((e = launch_patch_frames(g, n, x, (const double *)(base + o_rad), frames, s)) != cudaSuccess ||
        (e = launch_sp_nodes(n, ng1, frames, y, wk, s)) != cudaSuccess)
        return to_status(e);
    WosLaunch w{};
    w.n_groups = n;
    w.node_off = (const int64_t *)(base + o_node);
    w.walks = (const int64_t *)(base + o_walk);
    w.pid = (const uint32_t *)(base + o_pid);
    w.point_id = nullptr;   // node index within the point
    w.chunk_off = (const int64_t *)(base + o_chunk);
    w.cpn = (const int32_t *)(base + o_cpn);
    w.total_chunks = chunk_off[n];
    w.total_nodes = nodes;
    w.chunk = chunk;
    w.max_walks = maxw;
    w.y = y;
    w.prec = o->prec;
    w.eps = o->epsilon;
    w.max_steps = o->max_steps ? o->max_steps : 1000000ull;
    w.seed = o->seed;
    w.blocks_per_sm = wp.bps;
    w.refill = wp.refill;
    w.mean = Ud;
    w.se = SEd;
    w.steps = nullptr;
    w.capped = nullptr;
    if ((e = launch_wos(g, w, s)) != cudaSuccess) return to_status(e);
    return to_status(launch_sp_sigma(g, n, ng1, ng2, delta, frames, wk, Ud, SEd, sigma1, sigma2, q, se, status, s));
}

dtn_status dtn_distance(const dtn_geometry *g, int64_t n, const double *x, double *d, double *nearest, int32_t prec,
                        void *stream) {
    if (!g || n < 0 || (n > 0 && !x)) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (prec != DTN_PREC_FP64 && prec != DTN_PREC_MIXED) return DTN_E_INVALID_ARG;
    return to_status(launch_distance(g, n, x, d, nearest, prec, (cudaStream_t)stream));
}

dtn_status dtn_philox4x32_10(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out, void *stream) {
    if (n < 0 || (n > 0 && (!ctr || !out))) return DTN_E_INVALID_ARG;
    return to_status(launch_philox(n, ctr, seed, out, (cudaStream_t)stream));
}

dtn_status dtn_philox_fields21(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *fields, float *uniforms,
                               float *directions, void *stream) {
    if (n < 0 || (n > 0 && !ctr)) return DTN_E_INVALID_ARG;
    if (n > 0 && !fields && !uniforms && !directions) return DTN_E_INVALID_ARG;
    return to_status(launch_fields21(n, ctr, seed, fields, uniforms, directions, (cudaStream_t)stream));
}

dtn_status dtn_eval_dirichlet(const dtn_geometry *g, int64_t n, const double *x, double *out, void *stream) {
    if (!g || n < 0 || (n > 0 && (!x || !out))) return DTN_E_INVALID_ARG;
    if (wrong_device(g)) return DTN_E_INVALID_ARG;
    if (!g->has_data) return DTN_E_INVALID_ARG;
    return to_status(launch_dirichlet(g, n, x, out, (cudaStream_t)stream));
}

}  // extern "C"
