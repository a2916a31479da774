/*
 * dtn.h -- C ABI of the GB300 (sm_103a) local-BIE / walk-on-spheres
 * Dirichlet-to-Neumann library (method of Yan, Cai and Zeng, arXiv 1210.1491).
 *
 * Problem (Sec. 2, Eq. bw01-bw05): the Laplace equation holds in a region D with
 * Dirichlet data g on its boundary.  For each patch S = boundary of D inside a
 * ball B(c, a) centred at a boundary point c, the library returns the Neumann
 * data q = du/dn (n = outward normal of D) on S (Sec. 4, BIE-WOS algorithm):
 *   step 1: walk-on-spheres estimates U_k of u at the Gauss nodes y_k of the
 *           hemisphere Gamma = dB inside D (Sec. 2, Eq. bw87, Eq. bw85);
 *   step 2: collocation solve of the first-kind local BIE (Eq. bw49-bw51) built
 *           on the whole-sphere Dirichlet Green's function of B (one Kelvin image).
 * The potential anywhere then follows from the integral representation Eq. bw03.
 *
 * Conventions for every call:
 *   - Pointers marked "device" are CUDA device pointers (for instance the data
 *     pointers of torch tensors on cuda:0); "host" pointers are ordinary memory.
 *     The caller owns every pointer it passes; host descriptors and host arrays
 *     are copied before the call returns.  The library owns the geometry object,
 *     its device copies and its workspaces.
 *   - Calls taking a `stream` (a cudaStream_t passed as void*, NULL = default
 *     stream) are asynchronous: argument errors are returned synchronously
 *     before anything is enqueued; conditions found on the device (unsupported
 *     patch, capped walks, refinement that did not converge) are written to the
 *     per-patch status array and counters, which the caller reads after a
 *     stream synchronisation.  No call aborts, traps or prints.
 *   - A geometry object may be used from several threads only if the caller
 *     serialises the calls on it.
 *   - Arrays of 3-vectors are row-major (x, y, z) per row; matrices row-major.
 *
 * Error behaviour: every call returns a dtn_status; DTN_E_CUDA means a CUDA
 * runtime call failed (dtn_last_cuda_error() gives its code).
 */
#ifndef DTN_H
#define DTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque, library-owned geometry object (region, data, device workspaces). */
typedef struct dtn_geometry dtn_geometry;

typedef enum {
    DTN_OK = 0,
    DTN_E_INVALID_ARG = 1,
    DTN_E_OUT_OF_MEMORY = 2,
    DTN_E_CUDA = 3,
    DTN_E_NOT_CONVERGED = 4,
    DTN_E_TIMEOUT = 5,
    DTN_E_UNSUPPORTED = 6,
    DTN_E_WALK_CAP = 7
} dtn_status;

/* Region kinds (the solution domain D; walks run inside it). */
typedef enum {
    DTN_GEOM_BALL_INTERIOR = 0,    /* |x - center| < radius */
    DTN_GEOM_BOX_INTERIOR = 1,     /* lo < x < hi */
    DTN_GEOM_BOX_MINUS_BOXES = 2,  /* outer box minus the closed obstacle boxes */
    /* unbounded regions (Sec. 4.1.3): a walk that leaves the truncation sphere of
       radius `truncation` about `center` has gone to infinity and scores 0 */
    DTN_GEOM_HALF_SPACE = 3,       /* z > center[2] */
    DTN_GEOM_DISK_EXTERIOR = 4,    /* space outside the thin disk of radius `radius`
                                      about `center` in the plane z = center[2] */
    DTN_GEOM_BALL_EXTERIOR = 5     /* |x - center| > radius */
} dtn_geom_kind;

typedef struct {
    int32_t kind;                  /* dtn_geom_kind */
    double center[3];              /* ball; half space: a point of the plane; disk */
    double radius;                 /* ball; disk */
    double lo[3], hi[3];           /* outer box */
    int32_t n_boxes;               /* obstacle boxes, disjoint, inside the outer box */
    const double *boxes;           /* host, n_boxes x 6 (lo xyz, hi xyz), copied */
    double cell_size;              /* obstacle lookup grid cell edge; <= 0 picks one */
    double truncation;             /* unbounded regions: truncation radius (> radius) */
} dtn_geometry_desc;

/* Dirichlet data g on the boundary (Eq. bw01).  Each kind is the trace of a
 * function harmonic in D, so exact Neumann data exist for testing. */
typedef enum {
    DTN_DATA_POINT_SOURCE = 0,     /* g = strength / (4 pi |x - x0|), x0 outside D */
    DTN_DATA_HARMONIC_SH = 1,      /* g = sum c_lm rho^l Y_lm(dir), rho = |x-center|/scale,
                                      real orthonormal Y_lm, no Condon-Shortley phase */
    DTN_DATA_CONSTANT = 2          /* g = constant */
} dtn_data_kind;

typedef struct {
    int32_t kind;                  /* dtn_data_kind */
    double x0[3];
    double strength;
    int32_t lmax;                  /* <= 16 */
    const double *clm;             /* host, (lmax+1)^2 coefficients, index l*l + l + m, copied */
    double center[3];
    double scale;
    double constant;
} dtn_dirichlet_desc;

typedef enum {
    DTN_PREC_FP64 = 0,   /* FP64 walks, FP64 assembly, FP64 LU (the plain path) */
    DTN_PREC_MIXED = 1   /* FP32 walks with FP64 sums; patches of one shape share one
                            FP64-rule matrix, their right sides by FP32 weights and products
                            summed in FP64; a wrapped patch (its own shape) by FP32 rules in
                            offset form, FP32 hemisphere terms from FP64 differences; FP32 LU
                            with FP64-residual iterative refinement */
} dtn_precision;

typedef struct {
    int32_t prec;               /* dtn_precision */
    double epsilon;             /* absorption shell width (Sec. 2); > 0 */
    uint64_t seed;              /* Philox key = (seed low 32 bits, seed high 32 bits) */
    uint64_t max_steps;         /* distance evaluations per walk before it is cut (0 = 1e6) */
    int32_t max_refine_iters;   /* mixed precision: refinement sweeps (0 = 10) */
    double refine_tol;          /* stop when |r|_inf <= refine_tol |b|_inf (0 = 1e-12) */
    int32_t u_provided;         /* 1: skip the walks and read U_k from result->u_gamma_mean */
    int32_t walk_chunk;         /* walks per warp work item (0 = tuned) */
    int32_t wos_blocks_per_sm;  /* resident 128-thread walk blocks per SM (0 = tuned) */
    int32_t graph_capture;      /* 1: replay the device part as a CUDA graph when the shapes of
                                   the previous call repeat */
    int32_t record_stages;      /* 1: record CUDA events between the stages of the call on its
                                   stream (read them with dtn_stage_times) */
    int32_t wos_refill;         /* idle lanes of a warp before it refills them (0 = tuned) */
    int32_t bie_kind;           /* 0: first-kind local BIE (Eq. bw49-bw51, collocation solve);
                                   1: second-kind local BIE (Eq. bw55-bw59).  Disk patches: the
                                   double-layer operator vanishes and q = 2b row by row.  Cap
                                   patches: (1/2 I - D) q = b with D_ij the integral of dG/dn_x
                                   over panel j, the finite part of b regularised by the harmonic
                                   l = g(x) + grad_S g(x).(y - x).  DTN_PREC_FP64: D and b by the
                                   panel rules per patch.  DTN_PREC_MIXED: D per patch shape, b by
                                   a geodesic polar rule about each collocation point over the
                                   data interpolated on the panels (FP64 weights per patch shape,
                                   one FP64 product per patch), FP32 factors with FP64
                                   refinement */
    int32_t ring_order;         /* second kind: Gauss order of the polar rules on S
                                   (0 = 20 on disks, 32 on caps) */
} dtn_solve_opts;

/* Launch parameters of the walk kernel chosen by dtn_autotune_walks. */
typedef struct {
    int32_t walk_chunk;
    int32_t wos_blocks_per_sm;
    int32_t wos_refill;
    float ns_per_walk_step;     /* measured device time per walk-step of the best choice */
} dtn_tuning;

/* A batch of patches.  Patch p has a ball of radius radius[p] about centers[p]
 * (a point of the boundary), n_theta[p] x n_phi[p] hemisphere Gauss nodes
 * (Eq. bw85, theta in [0, theta_max]), n_rings[p] x n_sectors[p] panels on S
 * and walks_per_point[p] walks per node.  Node k = i*n_phi + j (i polar, j
 * azimuthal); panel index = ring*n_sectors + sector.  The walks of node k of
 * patch p use Philox counters (walk, step, k, patch id). */
typedef struct {
    int64_t n_patches;
    const double *centers;          /* device, n_patches x 3 */
    const double *radius;           /* host, n_patches (a patch-shape parameter, like the
                                       ring and sector counts) */
    const int32_t *n_theta;         /* host, n_patches, 1..64 */
    const int32_t *n_phi;           /* host, n_patches, 1..64 */
    const int32_t *n_rings;         /* host, n_patches, >= 1 */
    const int32_t *n_sectors;       /* host, n_patches, >= 1; rings*sectors <= 1024 */
    const int64_t *walks_per_point; /* host, n_patches, >= 2 (ignored with u_provided) */
    uint32_t patch_id_base;         /* RNG patch id of patch p = base + p ... */
    const uint32_t *patch_ids;      /* ... unless this host array (n_patches) is given */
} dtn_patch_batch;

/* Outputs (all device; offsets of patch p are the prefix sums of the per-patch
 * node and panel counts in batch order).  NULL marks an output not wanted,
 * except where "required" is stated. */
typedef struct {
    double *gamma_xyz;       /* gamma_total x 3, hemisphere node positions */
    double *gamma_w;         /* gamma_total, node weights (area element of Eq. bw83) */
    double *u_gamma_mean;    /* gamma_total, required: U_k (written; read when u_provided).
                                A node whose walks were all cut at max_steps has no
                                estimate: NaN (its patch gets DTN_E_WALK_CAP) */
    double *u_gamma_se;      /* gamma_total, standard error of U_k (+inf when fewer than two
                                of the node's walks were kept) */
    uint64_t *gamma_steps;   /* gamma_total, walk-steps (distance evaluations) per node */
    uint32_t *gamma_capped;  /* gamma_total, walks cut at max_steps (excluded from U_k) */
    double *colloc_xyz;      /* panels_total x 3, collocation points */
    double *normals;         /* panels_total x 3, outward normals of D there */
    double *areas;           /* panels_total */
    double *dirichlet;       /* panels_total, g at the collocation points */
    double *neumann;         /* panels_total, required: q = du/dn */
    double *matrix;          /* sum n_p^2: assembled A (row-major per patch), for checking */
    double *rhs;             /* panels_total: assembled b, for checking */
    int32_t *refine_iters;   /* n_patches */
    double *residual;        /* n_patches, final |b - A q|_inf / |b|_inf */
    int32_t *patch_status;   /* n_patches, dtn_status per patch: DTN_E_UNSUPPORTED (no solve),
                                else DTN_E_WALK_CAP (walks of the patch were cut at max_steps),
                                else DTN_E_NOT_CONVERGED, else DTN_OK */
} dtn_patch_result;

/* Creates a geometry object (device copies of the region, obstacle lookup
 * grid).  Errors: DTN_E_INVALID_ARG for a malformed description (radius <= 0,
 * lo >= hi, obstacle outside the outer box), DTN_E_CUDA / DTN_E_OUT_OF_MEMORY. */
dtn_status dtn_create_geometry(const dtn_geometry_desc *desc, dtn_geometry **out);

/* Releases the geometry object and every device buffer it owns (synchronises). */
dtn_status dtn_destroy_geometry(dtn_geometry *geom);

/* Frees the device workspaces the geometry's calls have grown (they grow again,
 * stream-ordered, on the next call) and drops a captured solve graph.
 * Synchronises the device.  The calls that grow a workspace do so with
 * cudaMallocAsync on their stream, by at least half its size each time, and
 * keep it: a workload of recurring sizes settles at a high-water mark and then
 * allocates nothing. */
dtn_status dtn_release_workspace(dtn_geometry *geom);

/* Sets the Dirichlet data g of Eq. bw01 (copied to the device). */
dtn_status dtn_set_dirichlet(dtn_geometry *geom, const dtn_dirichlet_desc *data);

/* Totals of a batch: panels_total = sum rings*sectors, gamma_total = sum
 * n_theta*n_phi, matrix_total = sum (rings*sectors)^2 (host, synchronous). */
dtn_status dtn_query_patch_sizes(const dtn_patch_batch *batch, int64_t *panels_total,
                                 int64_t *gamma_total, int64_t *matrix_total);

/* BIE-WOS algorithm (Sec. 4) for every patch of the batch: patch setup,
 * walks (Sec. 2, Eq. bw87), assembly of Eq. bw49-bw51 and the collocation
 * solve.  Asynchronous on `stream`.  The matrix A of Eq. bw50 depends only on
 * the patch shape (region kind, a, sphere radius, rings, sectors) expressed in
 * the patch frame; in DTN_PREC_MIXED the patches of one shape share one FP64
 * A (assembled with the FP64 rules) and one FP32 factorisation, and each patch
 * gets its own right side and FP64-residual refinement.  DTN_PREC_FP64 (the
 * plain path) assembles and factors every patch separately.  Per-patch failures land in patch_status
 * (DTN_E_UNSUPPORTED: the centre is not on the boundary; or the ball meets a
 * second smooth piece, except further faces of the obstacle box the centre
 * lies on (a wrapped patch), which is then unsupported if the ball also reaches
 * another conductor or the outer box, if the box is thinner than a along the
 * face normal, or if its face pieces need more sectors than n_sectors holds;
 * DTN_E_NOT_CONVERGED: refinement stopped above refine_tol; DTN_E_WALK_CAP:
 * some walks were cut at max_steps). */
dtn_status dtn_solve_patches(dtn_geometry *geom, const dtn_patch_batch *batch,
                             const dtn_solve_opts *opts, dtn_patch_result *result, void *stream);

/* Integral representation Eq. bw03 with the free-space G of Eq. bw05 and the
 * panel-midpoint rule over n_panels panels:
 *   u(t) = sum_p area_p [ q_p / (4 pi |t - y_p|) - g_p n_p.(t - y_p) / (4 pi |t - y_p|^3) ].
 * All arrays device.  dirichlet may be NULL (then g is evaluated from the
 * data set on geom).  If panel_index (device int64) is given, the sum runs
 * over panels panel_index[0 .. m) of the arrays, m = *n_index (device int64,
 * for instance the count written by dtn_gather_owned) or n_panels when n_index
 * is NULL; otherwise over panels 0 .. n_panels.  prec: DTN_PREC_FP64 (FP64
 * pairs) or DTN_PREC_MIXED (FP32 pair terms, FP64 per-target accumulation).
 * Asynchronous. */
dtn_status dtn_eval_potential(const dtn_geometry *geom, int64_t n_panels, const double *xyz,
                              const double *normals, const double *areas, const double *neumann,
                              const double *dirichlet, const int64_t *panel_index,
                              const int64_t *n_index, int64_t n_targets, const double *targets,
                              double *u_out, int32_t prec, void *stream);

/* Options of the fast multipole evaluation (dtn_eval_potential_fmm). */
typedef struct {
    int32_t order;          /* expansion order P, 1 .. 16 */
    int32_t leaf_sources;   /* a source cell holding more panels is split, 1 .. 4096 */
    int32_t leaf_targets;   /* a target cell holding more targets is split, 1 .. 4096 */
    int32_t max_level;      /* deepest octree level, 1 .. 21 */
    double theta;           /* acceptance (r_T + r_S) < theta |z - c|, r the cells' point radii; (0, 1) */
} dtn_fmm_opts;

/* What one evaluation did (counts; written when the pointer is not NULL). */
typedef struct {
    int64_t source_cells, target_cells;   /* octree cells, all levels */
    int64_t m2l_pairs, p2p_pairs;         /* accepted cell pairs and leaf pairs */
    int64_t p2p_terms;                    /* direct pair terms (sum of leaf-pair products) */
    int32_t source_levels, target_levels; /* levels including the root */
    int32_t traversal_passes;             /* level-synchronous traversal passes */
    int32_t restarts;                     /* traversals restarted after a list grew */
} dtn_fmm_stats;

/* The same sum as dtn_eval_potential (Eq. bw03 with the free-space G of
 * Eq. bw05, panel-midpoint rule) by the fast multipole method of Greengard and
 * Rokhlin, the evaluation Sec. 6 names for the potential after the patch
 * solves.  Panel p is a charge area_p q_p / 4pi and a dipole
 * -area_p g_p n_p / 4pi at its collocation point.  Sources and targets get
 * adaptive octrees over one bounding cube; a dual-tree traversal sends each
 * (target cell, source cell) pair with (r_T + r_S) < theta |z - c| (z and c the
 * cell centres, r the radii of balls about them that hold the cells' points)
 * through multipole-to-local
 * translation with expansions of order P in solid harmonics, and leaf pairs
 * that fail the test through the direct pair sum.  The far-field error of a
 * pair falls like theta^(P+1).  Expansions and pair terms are FP32, centre
 * differences and per-target sums FP64.
 *   Arrays as in dtn_eval_potential (device; dirichlet may be NULL: g from the
 *   data set on geom; panel_index / n_index select panels the same way, and
 *   panel_index must hold at least that many entries).  An index outside
 *   [0, n_panels) is found on the device before any panel is read and gives
 *   DTN_E_INVALID_ARG.
 *   n_panels and n_targets below 2^31.  A target that coincides with a panel
 *   point gets an infinite value, as in the direct sum.
 *   opts: required; stats: may be NULL.
 * Synchronises `stream` (the octrees and the traversal are built level by
 * level with host-side counts); the result is complete when the call returns
 * DTN_OK.  The workspace is owned by geom and reused; calls on one geom must
 * be serialised.  Errors: DTN_E_INVALID_ARG for options out of range or
 * missing arrays, DTN_E_CUDA / DTN_E_OUT_OF_MEMORY. */
dtn_status dtn_eval_potential_fmm(dtn_geometry *geom, int64_t n_panels, const double *xyz,
                                  const double *normals, const double *areas, const double *neumann,
                                  const double *dirichlet, const int64_t *panel_index,
                                  const int64_t *n_index, int64_t n_targets, const double *targets,
                                  double *u_out, const dtn_fmm_opts *opts, dtn_fmm_stats *stats,
                                  void *stream);

/* Panel gather for the overlapping-patch cover (Sec. 6: the boundary is covered
 * by overlapping patches S_i): panel i (of patch owner[i]) is kept iff the
 * patch centre nearest to its collocation point (FP64 distances, lowest index
 * on ties) is owner[i]'s.  Writes keep[i] (0/1) and the kept panels' indices,
 * in input order, to kept_index; *n_kept (device int64) receives their count.
 * Asynchronous. */
dtn_status dtn_gather_owned(int64_t n_panels, const double *colloc_xyz, const int64_t *owner,
                            int64_t n_centers, const double *centers, uint8_t *keep,
                            int64_t *kept_index, int64_t *n_kept, void *stream);

/* Walk-on-spheres estimates (Sec. 2, Eq. bw87) at arbitrary points of D:
 * n points y (device n x 3), each with its RNG point id and patch id (device
 * u32 arrays) and walk count (host int64 array, each in [2, 2^32)).  Outputs
 * (device, n): mean, standard error (may be NULL), walk-steps per point (may
 * be NULL), capped walks (may be NULL).  Uses opts->prec, epsilon, seed,
 * max_steps, walk_chunk, wos_blocks_per_sm.  Returns after the stream has
 * finished the walks (it synchronises `stream`). */
dtn_status dtn_wos_points(const dtn_geometry *geom, int64_t n, const double *y,
                          const uint32_t *point_ids, const uint32_t *patch_ids,
                          const int64_t *walks, const dtn_solve_opts *opts, double *mean,
                          double *se, uint64_t *steps, uint32_t *capped, void *stream);

/* Neumann data at single points of a flat boundary piece by the BIE-WOS formula
 * of Sec. 4.1, Eq. bw64: q(x) = Sigma1' + Sigma2', where
 *   Sigma1' = - sum_ij W_ij (3 cos th_i / (2 pi a^3)) (U_ij - g(x))   (Eq. bw65, bw83)
 * over the ng1 x ng1 Gauss nodes th_i = (pi/4)(xi_i + 1), ph_j = pi (xi_j + 1)
 * of the hemisphere of radius a about x (Eq. bw85), U_ij the walk estimates
 * there (Eq. bw87, walks[i] walks per node), and
 *   Sigma2' = -(1/2pi) int (1/rho^3 - 1/a^3) (g(y) - g(x)) ds_y      (Eq. bw68, bw82)
 * over the annulus delta <= rho <= a of the plane about x, by the ng2 x ng2
 * Gauss rule in (rho, angle).  The error of leaving out the disk of radius
 * delta is O(delta) (Eq. bw81).
 *   x: device n x 3 points, each on a plane face (box, box minus boxes, half
 *      space; thin disk: its top face z = center[2], the side z > center[2], with
 *      the ball's slice of the plane inside the disk) with the ball of radius a
 *      meeting that face only; q = ∂u/∂n with n the outward normal of D.
 *   walks: host int64 n, each in [2, 2^32); RNG point id = node index i*ng1 + j,
 *      patch id = patch_id_base + point index (as dtn_wos_points).
 *   ng1, ng2 in [1, 64]; 0 <= delta < a.
 *   Outputs, device, n values each: q (required); sigma1, sigma2, se (standard
 *      error of Sigma1'), status (DTN_OK, or DTN_E_UNSUPPORTED when x is not on
 *      a supported flat piece, then q = 0) may be NULL; U (n x ng1^2 node
 *      estimates) may be NULL.
 *   Uses opts->prec, epsilon, seed, max_steps and the walk launch fields.
 *   Asynchronous on `stream`; argument errors are returned before any work. */
dtn_status dtn_single_point_neumann(dtn_geometry *geom, int64_t n, const double *x, double a, int32_t ng1,
                                    int32_t ng2, double delta, const int64_t *walks, uint32_t patch_id_base,
                                    const dtn_solve_opts *opts, double *sigma1, double *sigma2, double *q,
                                    double *se, int32_t *status, double *U, void *stream);

/* dtn_wos_points for callers that cannot allocate device memory.  (The paper
 * has no counterpart; this is a deployment variant.)  Some callers must not
 * call cudaMalloc: a serving loop that cannot afford the device-wide
 * synchronisation an allocation or a free may cause, or a host that owns all
 * device memory through its own pool and cannot let a library take memory
 * (or fail for lack of it) in the middle of a request.  This entry point
 * allocates nothing: its scratch (walk accumulators, work counter, per-point
 * tables) is one file-scope device array of about 4 MB that every GPU loading
 * the library keeps until the process exits.
 *   - n must be at most 65536 points; larger n returns DTN_E_INVALID_ARG
 *     before any device work.  Arguments and outputs as in dtn_wos_points
 *     (walks is a host array); se may be NULL.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture on the device.
 *   - Every call uses the same array and leaves its contents behind; each call
 *     clears the parts that must start at zero.  Calls whose work overlaps on
 *     the GPU race on the array: serialise them (one stream, or events).
 *   - The device current at the call must be the geometry's device
 *     (DTN_E_INVALID_ARG otherwise).
 *   - Asynchronous on `stream`; the host array walks is copied before
 *     return and may be reused at once. */
dtn_status dtn_wos_points_noalloc(const dtn_geometry *geom, int64_t n, const double *y,
                                  const uint32_t *point_ids, const uint32_t *patch_ids,
                                  const int64_t *walks, const dtn_solve_opts *opts, double *mean,
                                  double *se, uint64_t *steps, uint32_t *capped, void *stream);

/* Distance to the boundary and nearest boundary point (the WOS sphere radius,
 * Sec. 2) at n device points; d and nearest are device outputs (n, n x 3).
 * prec selects FP64 or the FP32 arithmetic the mixed walks use. */
dtn_status dtn_distance(const dtn_geometry *geom, int64_t n, const double *x, double *d,
                        double *nearest, int32_t prec, void *stream);

/* Philox4x32-10 (Salmon et al., SC'11) on n device counters (n x 4 u32) with
 * key (seed lo32, seed hi32): out (device, n x 4 u32).  The walk kernels use
 * the same generator; this entry point exposes it for bit-exact checking. */
dtn_status dtn_philox4x32_10(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *out,
                             void *stream);

/* The draws of the FP32 (DTN_PREC_MIXED) walks for n Philox blocks, computed
 * by the walk kernel's own device functions, for bit-exact checking.  Walk
 * jump j uses the block with counter (walk, j / 3, point, patch) and its
 * fields 2m and 2m + 1, m = j mod 3 (the walk on spheres of Sec. 2 draws a
 * uniform direction per jump; the generator is not in the paper).
 *   ctr: device, n x 4 u32 counters; key = (seed lo32, seed hi32).
 *   fields: device, n x 6 u32 (may be NULL): the 21-bit fields, the top 21 bits
 *     of each word, then (w0 & 0x7ff) | (w1 & 0x3ff) << 11 and the same of w2, w3.
 *   uniforms: device, n x 6 float (may be NULL): u = (2 f + 1) 2^-22, exact.
 *   directions: device, n x 3 x 3 float (may be NULL): per jump m the unit
 *     vector (s cos ph, s sin ph, z), z = 1 - 2 u_{2m}, s = sqrt(1 - z^2),
 *     ph = 2 pi (u_{2m+1} - 1/2), with the walk kernel's FP32 sine, cosine and
 *     square root (a few 1e-7 from the exact values).
 * At least one output must be given.  Asynchronous; DTN_E_INVALID_ARG for
 * n < 0 or missing arrays. */
dtn_status dtn_philox_fields21(int64_t n, const uint32_t *ctr, uint64_t seed, uint32_t *fields,
                               float *uniforms, float *directions, void *stream);

/* Dirichlet data g at n device points (FP64). */
dtn_status dtn_eval_dirichlet(const dtn_geometry *geom, int64_t n, const double *x, double *g,
                              void *stream);

/* Autotuner (not in the paper): times the walk kernel on a sample of the batch
 * (its first 96 patches at most, at most 4096 walks per node) for every combination of
 * walk chunk {64, 128, 256, 512}, resident 128-thread blocks per SM
 * {5, 6, 7, 8, 9} (each capped at the occupancy limit) and refill threshold
 * {4, 8, 12, 16}, and keeps the fastest per
 * (device name, region kind, precision) in a process-wide cache that
 * dtn_solve_patches and dtn_wos_points consult for every opts field left at 0.
 * Synchronises `stream`.  *out (may be NULL) receives the choice. */
dtn_status dtn_autotune_walks(dtn_geometry *geom, const dtn_patch_batch *batch,
                              const dtn_solve_opts *opts, dtn_tuning *out, void *stream);

/* Device time in milliseconds of the stages of the last dtn_solve_patches call
 * on geom made with record_stages = 1: ms[0] patch setup, ms[1] walks and their
 * estimates, ms[2] assembly, ms[3] LU and refinement.  A call replayed as a
 * CUDA graph (graph_capture) is timed as a whole in ms[0], with ms[1..3] = 0.
 * Waits for that call's last event.  DTN_E_INVALID_ARG if no call recorded
 * stages. */
dtn_status dtn_stage_times(dtn_geometry *geom, float ms[4]);

/* Human-readable name of a status code (static storage). */
const char *dtn_status_string(dtn_status s);

/* The last failing CUDA runtime error code seen by this library (0 if none). */
int32_t dtn_last_cuda_error(void);

/* ---------------------------------------------------------------- serving */
/* Continuous-batching request server (not in the paper: a serving layer over
 * dtn_solve_patches, which relies on the independence of the patch solves,
 * Sec. 6).  Queries are sets of patches with their own walk budgets.  A worker
 * thread merges queued queries into batches and runs each batch on one of
 * max_inflight slots (a stream and a private copy of the geometry's
 * workspace); queries that arrive while batches run are admitted as slots and
 * device memory free up, so batches of different requests overlap on the
 * device.  Results depend only on the query (its patch ids fix every random
 * number), so a query gives the same answer alone or in a mix.
 * Admission by device memory: the budget is the free device memory at
 * creation (cudaMemGetInfo) less a reserve of max(1 GiB, 5% of the device),
 * or memory_budget if that is smaller.  A batch starts only if the slots'
 * workspaces (what each holds now, and for the starting batch the workspace
 * its solve reserves) stay within the budget; idle slots give theirs back when
 * a batch would not fit otherwise, and a query that cannot fit in an empty
 * server finishes with DTN_E_OUT_OF_MEMORY.  Slot workspaces grow
 * stream-ordered and are kept, so a steady stream of similar queries neither
 * frees nor allocates. */
typedef struct dtn_server dtn_server;

typedef struct {
    int32_t max_inflight;        /* concurrent batches (streams), >= 1 */
    int64_t max_batch_patches;   /* patches merged into one launch */
    int64_t memory_budget;       /* upper limit in bytes of the budget above (0: none) */
    dtn_solve_opts opts;         /* solve options for every query */
    int32_t split_sms;           /* 1: when opts.wos_blocks_per_sm is 0, each slot's walk launch
                                    takes 1/max_inflight of the resident walk blocks per SM, so the
                                    walks of several slots run side by side; 0: every walk launch
                                    may fill the GPU (batches then overlap at kernel boundaries) */
} dtn_server_config;

/* Counters of a server (dtn_server_stats). */
typedef struct {
    int64_t budget_bytes;        /* admission budget */
    int64_t device_free_bytes;   /* free device memory at creation */
    int64_t held_bytes;          /* slot workspaces now (and batches in flight) */
    int64_t peak_held_bytes;     /* the most the ledger has held */
    int64_t batches;             /* finished batches */
    int64_t queries;             /* finished queries (any status) */
    int64_t rejected;            /* queries that could not fit the budget */
    int32_t max_concurrent;      /* most batches in flight on the device at one time */
    double busy_ms;              /* device time with at least one batch in flight */
    double overlap_ms;           /* device time with two or more batches in flight */
} dtn_server_info;

/* One query: host arrays, copied at submission.  Node/panel layout as in
 * dtn_patch_batch. */
typedef struct {
    int64_t n_patches;
    const double *centers;          /* host n x 3 */
    const double *radius;           /* host n */
    const int32_t *n_theta, *n_phi, *n_rings, *n_sectors; /* host n */
    const int64_t *walks_per_point; /* host n */
    const uint32_t *patch_ids;      /* host n: RNG patch ids */
} dtn_query;

dtn_status dtn_server_create(dtn_geometry *geom, const dtn_server_config *cfg, dtn_server **out);
/* Enqueues a query; *ticket identifies it.  Never blocks on the GPU. */
dtn_status dtn_server_submit(dtn_server *srv, const dtn_query *q, int64_t *ticket);
/* Non-blocking: *done = 1 once the query has finished; then latency_s (may be
 * NULL) gets submit-to-completion seconds and the call returns the query's
 * status: DTN_OK, or the first non-OK patch status of its patches
 * (DTN_E_UNSUPPORTED, DTN_E_WALK_CAP, DTN_E_NOT_CONVERGED), or DTN_E_CUDA /
 * DTN_E_OUT_OF_MEMORY when the query did not run.  Unless the query did not
 * run, neumann (host, its panels_total; may be NULL), u_mean (host, its
 * gamma_total; may be NULL) and patch_status (host, its n_patches; may be
 * NULL) receive its results.  DTN_OK with *done = 0 while it runs. */
dtn_status dtn_server_poll(dtn_server *srv, int64_t ticket, int32_t *done, double *neumann,
                           double *u_mean, double *latency_s, int32_t *patch_status);
/* Blocks until every submitted query has completed; returns DTN_E_CUDA if a
 * batch failed on the device, else DTN_OK. */
dtn_status dtn_server_drain(dtn_server *srv);
/* Counters and device intervals of the finished batches (CUDA events recorded
 * on the slot streams around each batch). */
dtn_status dtn_server_stats(dtn_server *srv, dtn_server_info *out);
dtn_status dtn_server_destroy(dtn_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* DTN_H */
