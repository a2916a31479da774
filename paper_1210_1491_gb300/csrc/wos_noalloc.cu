// wos_noalloc.cu -- dtn_wos_points_noalloc: the walk-on-spheres estimates of
// dtn_wos_points for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: serving loops whose latency budget has
// no room for the device-wide synchronisation an allocation (or a free) can
// cause, and hosts that own all device memory through a pool of their own and
// must not see a library take memory behind their back (or fail for lack of
// it halfway through a request).  This entry point takes its scratch (the walk
// accumulators, the work counter and the per-point offset tables) from one
// file-scope device array of fixed size instead of allocating it.
//
// The array holds kNoAllocMaxPoints points' worth of scratch (a few MB); every
// GPU that loads this library keeps it until the process exits.  Its device
// address is looked up once per device with cudaGetSymbolAddress; host code
// never passes the array's own name to a kernel, because on the host that
// name is only a stand-in, not a device address.
#include <cstring>
#include <mutex>
#include <vector>

#include "dtn_internal.h"

namespace {

constexpr int64_t kNoAllocMaxPoints = 65536;
constexpr int kMaxDevices = 64;

// scratch layout (bytes from the start, each part 256-byte aligned):
//   walk accumulators and counter   wos_scratch_bytes(n)
//   node offsets    (n + 1) x int64
//   chunk offsets   (n + 1) x int64
//   walks           n x int64
//   chunks per node n x int32
//   standard errors n x double (used when the caller passes se = NULL)
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kAccBytes = align256((size_t)kNoAllocMaxPoints * (3 * 8 + 4) + 64);
constexpr size_t kScratchBytes = kAccBytes + align256((kNoAllocMaxPoints + 1) * 8) * 2 +
                                 align256(kNoAllocMaxPoints * 8) + align256(kNoAllocMaxPoints * 4) +
                                 align256(kNoAllocMaxPoints * 8);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
cudaError_t scratch_on_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

using dtn::to_status;

extern "C" dtn_status dtn_wos_points_noalloc(const dtn_geometry *gc, int64_t n, const double *y,
                                             const uint32_t *point_ids, const uint32_t *patch_ids,
                                             const int64_t *walks, const dtn_solve_opts *o, double *mean,
                                             double *se, uint64_t *steps, uint32_t *capped, void *stream) {
    using namespace dtn;
    dtn_geometry *g = const_cast<dtn_geometry *>(gc);
    if (!g || n < 0 || !o) return DTN_E_INVALID_ARG;
    if (n > kNoAllocMaxPoints) return DTN_E_INVALID_ARG;
    if (n == 0) return DTN_OK;
    if (!y || !point_ids || !patch_ids || !walks || !mean || !(o->epsilon > 0)) return DTN_E_INVALID_ARG;
    if (o->prec != DTN_PREC_FP64 && o->prec != DTN_PREC_MIXED) return DTN_E_INVALID_ARG;
    if (!g->has_data) return DTN_E_INVALID_ARG;
    int64_t maxw = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (walks[i] < 2 || walks[i] > 0xFFFFFFFFll) return DTN_E_INVALID_ARG;
        maxw = std::max(maxw, walks[i]);
    }
    // the geometry's device copies and the scratch address must be of one device
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return to_status(e);
    if (dev != g->device) return DTN_E_INVALID_ARG;
    void *scratch = nullptr;
    if ((e = scratch_on_current_device(&scratch)) != cudaSuccess) return to_status(e);
    const int32_t chunk = o->walk_chunk > 0 ? o->walk_chunk : 256;
    // private copy of the walk counts, so that every host array the copies
    // below read is pageable memory of this call
    std::vector<int64_t> wv(walks, walks + n);
    std::vector<int64_t> node_off(n + 1), chunk_off(n + 1, 0);
    std::vector<int32_t> cpn(n);
    for (int64_t i = 0; i <= n; ++i) node_off[i] = i;
    for (int64_t i = 0; i < n; ++i) {
        cpn[i] = (int32_t)((walks[i] + chunk - 1) / chunk);
        chunk_off[i + 1] = chunk_off[i] + cpn[i];
    }
    char *base = (char *)scratch;
    void *acc = base;
    int64_t *d_node = (int64_t *)(base + kAccBytes);
    int64_t *d_chunk = (int64_t *)((char *)d_node + align256((kNoAllocMaxPoints + 1) * 8));
    int64_t *d_walks = (int64_t *)((char *)d_chunk + align256((kNoAllocMaxPoints + 1) * 8));
    int32_t *d_cpn = (int32_t *)((char *)d_walks + align256(kNoAllocMaxPoints * 8));
    double *d_se = (double *)((char *)d_cpn + align256(kNoAllocMaxPoints * 4));
    cudaStream_t s = (cudaStream_t)stream;
    // pageable host-to-device copies are staged before cudaMemcpyAsync returns,
    // so the host vectors may go out of scope afterwards
    if ((e = cudaMemcpyAsync(d_node, node_off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_chunk, chunk_off.data(), (n + 1) * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_walks, wv.data(), n * 8, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
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
    w.blocks_per_sm = o->wos_blocks_per_sm;
    w.refill = o->wos_refill;
    w.mean = mean;
    w.se = se ? se : d_se;
    w.steps = steps;
    w.capped = capped;
    return to_status(launch_wos_into(g, w, acc, s));
}
