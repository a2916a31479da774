// dtn_internal.h -- host-side structures shared by the translation units of
// the library (geometry object, per-call batch layout, kernel launchers).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <vector>

#include "../../include/dtn.h"
#include "dtn_device.cuh"

namespace dtn {

// A device buffer that only grows; freed with the geometry object.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool pooled = false;   // allocated stream-ordered (cudaMallocAsync)
    // grow to at least n bytes (contents are not kept): cudaFree + cudaMalloc,
    // which may synchronise the device
    cudaError_t reserve(size_t n);
    // grow stream-ordered on s (cudaFreeAsync + cudaMallocAsync: no device-wide
    // synchronisation), to at least 1.5x the old size, so that a workload whose
    // sizes vary settles at a high-water mark and then allocates nothing
    cudaError_t reserve(size_t n, cudaStream_t s);
    void release();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// Per-call layout of a batch on the device (offsets are prefix sums over
// patches in batch order).
struct BatchLayout {
    int64_t n_patches = 0;
    int64_t gamma_total = 0, panels_total = 0, matrix_total = 0;
    int32_t max_panels = 0, max_nodes = 0;
    int64_t max_walks = 0;
    std::vector<int64_t> gamma_off, panel_off, mat_off;   // n+1
    std::vector<uint8_t> wrapped;                         // n: a wrapped patch (groups of its own)
    std::vector<int32_t> nt, nph, nr, ns;                 // n
    std::vector<int64_t> walks;                           // n
    std::vector<uint32_t> pid;                            // n
    std::vector<double> radius;                           // n
    // shape groups (patches with equal radius, rings and sectors): the matrix of
    // Eq. bw50 in the patch frame is the same for all members
    int64_t n_groups = 0;
    std::vector<int64_t> group_of;                        // n
    std::vector<int64_t> rep;                             // n_groups: first member
    std::vector<int64_t> grows_off, gmat_off, gfac_off;   // n_groups + 1
    int64_t grows_total = 0, gmat_total = 0, gfac_total = 0;
    // weight groups (shape and node orders): the weights that map the data and
    // the walk estimates to the right side of Eq. bw51 are the same for all
    // members; rows x kcols FP32, kcols = 64 per panel (8 x 8 data samples,
    // cap patches only) + hemisphere nodes
    int64_t n_wgroups = 0;
    std::vector<int64_t> wgroup_of, wrep;                 // n, n_wgroups
    std::vector<int64_t> wrows_off;                       // n_wgroups + 1
    int64_t wrows_total = 0;
    std::vector<int64_t> kcols, gw_off;                   // n_wgroups, n_wgroups + 1
    int64_t gw_total = 0;
    std::vector<int64_t> vec_off;                         // n + 1: per-patch sample vectors
    int64_t vec_total = 0;
    std::vector<int64_t> members, mem_off, tile_off;      // n, n_wgroups + 1, n_wgroups + 1
    int64_t tiles_total = 0;
    int32_t max_wgroup_rows = 0;
};

// panel samples of the data in the right-side weights (8 x 8 Gauss points)
constexpr int kSampleN = 8, kSamplesPerPanel = kSampleN * kSampleN;
// patches per column tile of the right-side product
constexpr int kRhsTileN = 32;

// Device copies of one layout (kept in the geometry workspace).
struct DevLayout {
    int64_t *gamma_off, *panel_off, *mat_off, *walks, *chunk_off;
    int32_t *nt, *nph, *nr, *ns, *cpn;
    uint32_t *pid;
    double *radius;
    int64_t *group_of, *rep, *grows_off, *gmat_off, *gfac_off;
    int64_t *wrep, *wrows_off, *kcols, *gw_off, *vec_off, *members, *mem_off, *tile_off;
    PatchFrame *frames;
    Piece *pieces;          // n_patches x kMaxPieces (box-minus-boxes regions), else nullptr
};

struct Workspace {
    DevBuf layout;          // DevLayout arrays
    DevBuf gamma_loc;       // gamma_total x 3 (local node coordinates)
    DevBuf gamma_w;         // gamma_total
    DevBuf gamma_xyz;       // gamma_total x 3
    DevBuf panel_loc;       // panels_total x 3 (local collocation coordinates)
    DevBuf panel_prm;       // panels_total x 4 (u0, u1, v0, v1) + (uc, vc)
    DevBuf panel_aux;       // panels_total x 4: local centre xyz + bounding radius
    DevBuf panel_g;         // panels_total
    DevBuf mat;             // matrix_total doubles (assembled A)
    DevBuf lu32;            // matrix_total floats (LU factors when not in shared memory)
    DevBuf lu64;            // matrix_total doubles (FP64 LU when not in shared memory)
    DevBuf rhs;             // panels_total
    DevBuf acc;             // WOS accumulators: 3 x u64 + u32 per node
    DevBuf counter;         // work counter(s)
    DevBuf se_tmp;          // gamma_total (standard errors when not requested)
    DevBuf tune;            // autotuner outputs (means, steps)
    DevBuf gmat;            // shared matrices, one per shape group (FP64)
    DevBuf gfac;            // shared FP32 factors, n(n+1) per group
    DevBuf gpiv;            // shared pivots, n per group
    DevBuf gw;              // right-side weights per weight group (FP32)
    DevBuf vec;             // per-patch samples (data at panel points, walk estimates), FP32
    DevBuf sp;              // single-point method: frames, nodes, weights, estimates, walk layout
    DevBuf capflag;         // n_patches int32: 1 where a walk of the patch was cut at max_steps
    DevBuf panel_piece;     // panels_total int32: the piece of a wrapped patch's panel
    DevBuf kinds;           // n_patches frames + kinds of the classification pre-pass (mixed, wires)
    DevBuf pstat;           // panels_total per-panel FP32 maps (mixed precision, wrapped patches)
};

struct GeometryHost {
    dtn_geometry_desc desc{};
    std::vector<double> boxes;
    // obstacle grid (host copy)
    int gn[3] = {1, 1, 1};
    double glo[3] = {0, 0, 0}, cell = 1.0;
    std::vector<int> cstart, citems;
    std::vector<float> ccap;
    // last Dirichlet data set (for cloning geometry objects)
    dtn_dirichlet_desc data{};
    std::vector<double> clm;
};

}  // namespace dtn

struct dtn_geometry {
    dtn::GeometryHost host;
    dtn::DGeom dg{};
    dtn::DData dd{};
    bool has_data = false;
    double score_bound = 1.0;          // bound on |g| over the boundary
    dtn::DevBuf d_boxes, d_boxes_f, d_cstart, d_citems, d_ccap, d_clm, d_clm_f, d_clm_cart;
    dtn::Workspace ws;
    int device = 0;
    int num_sms = 0;
    char dev_name[256] = {0};
    uint64_t data_version = 0;                // bumped by every dtn_set_dirichlet
    cudaGraphExec_t graph_exec = nullptr;     // last captured solve (graph_capture)
    void *fmm_ws = nullptr;                   // fast multipole workspace (fmm.cu)
    cudaStream_t cap_stream = nullptr;        // private stream used for capture
    std::vector<unsigned char> graph_key;
    cudaEvent_t stage_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    bool stages_recorded = false;
    std::mutex mu;
};

namespace dtn {

// error bookkeeping
void set_cuda_error(cudaError_t e);
#define DTN_CUDA(call)                                        \
    do {                                                      \
        cudaError_t _e = (call);                              \
        if (_e != cudaSuccess) {                              \
            ::dtn::set_cuda_error(_e);                        \
            return _e == cudaErrorMemoryAllocation ? DTN_E_OUT_OF_MEMORY : DTN_E_CUDA; \
        }                                                     \
    } while (0)

// Gauss-Legendre tables on the device: orders 1..kMaxGauss, order n at offset
// n(n-1)/2, nodes ascending on [-1, 1].
constexpr int kMaxGauss = 64;
cudaError_t ensure_tables();
// 1 when the current device is not the geometry's (the entry points then return
// DTN_E_INVALID_ARG: every launch goes to the current device)
bool wrong_device(const dtn_geometry *g);
// workspace bytes a solve of this batch reserves, and what a geometry holds now
size_t solve_workspace_bytes(const dtn_patch_batch *b, const dtn_solve_opts *o, bool caps);
size_t workspace_bytes(const dtn_geometry *g);
const double *gl_x_dev();
const double *gl_w_dev();
const ShTables *sh_tables_dev();
// per-unit constant-memory copies of the harmonic recurrence tables
cudaError_t upload_sh_wos(const ShTables &t);
cudaError_t upload_sh_assemble(const ShTables &t);
cudaError_t upload_sh_second_kind(const ShTables &t);
cudaError_t upload_sh_single_point(const ShTables &t);
void gauss_legendre_host(int n, double *x, double *w);

// launchers (each enqueues on `s`)
cudaError_t launch_patch_setup(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                               const double *centers, double *gamma_xyz,
                               double *gamma_w, double *gamma_loc, double *colloc, double *normals,
                               double *areas, double *panel_loc, double *panel_prm, double *panel_aux,
                               double *panel_g, int32_t *panel_piece, cudaStream_t s);

cudaError_t launch_patch_frames(const dtn_geometry *g, int64_t n, const double *centers, const double *radius,
                                PatchFrame *frames, cudaStream_t s);

// single-point method (Sec. 4.1): hemisphere nodes with their Sigma1' weights,
// then the two sums per point
cudaError_t launch_sp_nodes(int64_t n, int ng1, const PatchFrame *frames, double *y, double *wk, cudaStream_t s);
cudaError_t launch_sp_sigma(const dtn_geometry *g, int64_t n, int ng1, int ng2, double delta, const PatchFrame *frames,
                            const double *wk, const double *U, const double *SE, double *sigma1, double *sigma2,
                            double *q, double *se, int32_t *status, cudaStream_t s);

struct WosLaunch {
    int64_t n_groups;
    const int64_t *node_off;     // n_groups + 1
    const int64_t *walks;        // per group
    const uint32_t *pid;         // per group (RNG patch id)
    const uint32_t *point_id;    // per node or nullptr (then node - node_off[group])
    const int64_t *chunk_off;    // n_groups + 1
    const int32_t *cpn;          // chunks per node, per group
    int64_t total_chunks;
    int64_t total_nodes;
    int32_t chunk;
    int64_t max_walks;
    const double *y;             // nodes x 3
    int prec;
    double eps;
    uint64_t max_steps, seed;
    int blocks_per_sm;
    int refill;
    // outputs
    double *mean, *se;
    uint64_t *steps;
    uint32_t *capped;
    int32_t *group_capped;       // per group or nullptr: set to 1 where a walk was cut (cleared first)
};
cudaError_t launch_wos(dtn_geometry *g, const WosLaunch &w, cudaStream_t s);
size_t wos_scratch_bytes(int64_t nodes);
cudaError_t launch_wos_into(dtn_geometry *g, const WosLaunch &w, void *acc, cudaStream_t s);
cudaError_t launch_walk_cap_status(int64_t n, const int32_t *group_capped, int32_t *status, cudaStream_t s);
// resident 128-thread walk blocks per SM of the walk kernel for this geometry and precision
int wos_resident_blocks(const dtn_geometry *g, int prec);

// mode 0: per patch, A and b (FP64 rules, or FP32 far field in mixed precision);
// mode 1: A of each shape group's representative (FP64 rules) into A + gmat_off
cudaError_t launch_assemble(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                            int prec, int mode, const double *panel_loc, const double *panel_prm,
                            const double *panel_aux, const double *panel_g, const double *gamma_loc,
                            const double *gamma_w, const double *U, double *A, double *b, cudaStream_t s,
                            int sk = 0, int only_wrapped = 0, void *pstat = nullptr);
// bytes of the per-panel FP32 maps of the mixed-precision wrapped pass
size_t wrapped_static_bytes(int64_t panels);

// mixed precision right sides: FP64 weights per shape group (product rules of
// the double layer against the panel interpolants of the data, and the walk
// term), the per-patch sample vectors, then one product per group
cudaError_t launch_rhs_shared(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                              const double *panel_loc, const double *panel_prm, const double *panel_aux,
                              const double *panel_g, const double *gamma_loc, const double *gamma_w,
                              const double *U, float *gw, float *vec, double *b, cudaStream_t s);

// second-kind local BIE on disk patches (Eq. bw55-bw59): q = 2b per collocation row
cudaError_t launch_second_kind(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                               const double *panel_loc, const double *panel_g, const double *gamma_loc,
                               const double *gamma_w, const double *U, int ng2, double *q, double *b,
                               int32_t *iters, double *resid, int32_t *status, cudaStream_t s);
cudaError_t launch_second_kind_cap_rhs_shared(const dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                                              const double *panel_loc, const double *panel_prm,
                                              const double *gamma_loc, const double *gamma_w, const double *U,
                                              int ng, double *W, double *vec, double *b, cudaStream_t s);

// copies each patch's group matrix into its own block (mat_off) for checking
cudaError_t launch_expand_matrices(const BatchLayout &L, const DevLayout &D, const double *gA,
                                   double *A, cudaStream_t s);

// bytes of global factor scratch the LU launch needs (0 when the factors fit in
// shared memory)
size_t lu_scratch_bytes(const BatchLayout &L, int prec);

cudaError_t launch_lu_solve(dtn_geometry *g, const BatchLayout &L, const DevLayout &D, int prec,
                            const double *A, const double *b, double *q, int max_iters, double tol,
                            int32_t *iters, double *resid, int32_t *status, cudaStream_t s);

// shared-matrix path: FP32 factors of every group matrix, then one solve with
// FP64-residual refinement per patch against its group's matrix and factors
cudaError_t launch_lu_shared(dtn_geometry *g, const BatchLayout &L, const DevLayout &D,
                             const double *gA, const double *b, double *q, int max_iters, double tol,
                             int32_t *iters, double *resid, int32_t *status, cudaStream_t s);
size_t lu_shared_scratch_bytes(const BatchLayout &L);

cudaError_t launch_potential(int64_t np, const int64_t *index, const int64_t *n_index, const double *xyz,
                             const double *nrm, const double *area, const double *q, const double *g,
                             int64_t nt, const double *t, double *out, int prec, int num_sms,
                             cudaStream_t s);

cudaError_t launch_gather(int64_t np, const double *x, const int64_t *owner, int64_t nc,
                          const double *cent, uint8_t *keep, int64_t *kept, int64_t *n_kept,
                          cudaStream_t s);

cudaError_t launch_fields21(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *fields, float *uni, float *dir,
                            cudaStream_t s);
cudaError_t launch_philox(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out,
                          cudaStream_t s);
cudaError_t launch_distance(const dtn_geometry *g, int64_t n, const double *x, double *d,
                            double *nearest, int prec, cudaStream_t s);
cudaError_t launch_dirichlet(const dtn_geometry *g, int64_t n, const double *x, double *out,
                             cudaStream_t s);

// fast multipole evaluation (fmm.cu)
cudaError_t fmm_evaluate(dtn_geometry *g, int64_t np, int64_t np_total, const double *xyz, const double *nrm,
                         const double *area, const double *q, const double *gv, const int64_t *index, int64_t nt,
                         const double *t, double *out, const dtn_fmm_opts &o, dtn_fmm_stats *st, bool *bad_index,
                         cudaStream_t s);
void fmm_release(dtn_geometry *g);
dtn_status to_status(cudaError_t e);

__host__ __device__ inline int64_t find_group(const int64_t *off, int64_t n, int64_t idx) {
    // largest p in [0, n) with off[p] <= idx
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace dtn
