// noalloc.cu -- splat_bin_sort without a caller-supplied workspace.
//
// Some callers cannot allocate device memory when they need to sort: for
// example a renderer plugin whose host application has already reserved the
// whole GPU memory budget for itself, or a frame loop that must never reach
// cudaMalloc / cudaFree because those calls can synchronise the whole device
// and stall the frame.  For them this entry point takes its scratch from a
// fixed array compiled into the library instead of from a workspace argument.
//
// The array below is a file-scope device variable: every GPU that loads this
// part of the library keeps its kSplatNoallocScratchBytes until the process
// exits.  Every call shares it, so calls whose work overlaps on the GPU
// (different streams, or different host threads without ordering) race on it.
// Its contents persist from the previous call; the sort clears every part it
// relies on starting at zero.
#include <mutex>

#include "splat_internal.cuh"

namespace splat {

cudaError_t launch_bin_sort(const splat_proj&, const ViewBatch&, const splat_bins&, int32_t*, void*, const LaunchCtx&);
size_t bin_sort_workspace(int64_t n_rows, int64_t capacity, int V, const int* TX, const int* TY, int tile_sort);

constexpr size_t kSplatNoallocScratchBytes = SPLAT_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kSplatNoallocScratchBytes];

// Host-side device address of g_noalloc_scratch, looked up once per device.  In
// host code the name g_noalloc_scratch is only a host-side stand-in for the
// symbol; kernels must get the address returned by cudaGetSymbolAddress.
static void* g_scratch_ptr[64];
static std::mutex g_scratch_mutex;

static void* scratch_for_current_device(cudaError_t* err)
{
    int dev = 0;
    *err = cudaGetDevice(&dev);
    if (*err != cudaSuccess || dev < 0 || dev >= 64) {
        if (*err == cudaSuccess) *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        g_scratch_ptr[dev] = p;
    }
    return g_scratch_ptr[dev];
}

}  // namespace splat

using namespace splat;

extern "C" splat_status splat_bin_sort_noalloc(const splat_proj* proj, const splat_view* views, int V,
                                               splat_bins* bins, int32_t* status, void* stream)
{
    // the argument checks of splat_bin_sort, so both entry points reject the same calls
    if (!host_valid_views(views, V) || !host_valid_proj(proj, V) || !host_valid_bins(bins) || !status)
        return SPLAT_ERR_INVALID_ARG;
    int TX[SPLAT_MAX_VIEWS], TY[SPLAT_MAX_VIEWS];
    for (int v = 0; v < V; ++v) {
        TX[v] = (views[v].W + kTile - 1) / kTile;
        TY[v] = (views[v].H + kTile - 1) / kTile;
    }
    const LaunchCtx ctx = launch_ctx(stream);  // the library-wide tuning (splat_set_*)
    const size_t need = bin_sort_workspace(proj->n * V, bins->capacity, V, TX, TY, ctx.tile_sort);
    if (need > kSplatNoallocScratchBytes) return SPLAT_ERR_CAPACITY;  // larger than the fixed scratch
    cudaError_t err;
    void* scratch = scratch_for_current_device(&err);
    if (!scratch) return SPLAT_ERR_CUDA;
    // views -> kernel parameters, as in splat_bin_sort
    ViewBatch vb{};
    vb.V = V;
    int tiles = 0;
    int64_t pix = 0;
    for (int v = 0; v < V; ++v) {
        ViewParams& p = vb.v[v];
        p.W = views[v].W;
        p.H = views[v].H;
        p.TX = TX[v];
        p.TY = TY[v];
        p.tile_base = tiles;
        p.pix_base = pix;
        tiles += TX[v] * TY[v];
        pix += (int64_t)views[v].W * views[v].H;
    }
    vb.total_tiles = tiles;
    return launch_bin_sort(*proj, vb, *bins, status, scratch, ctx) == cudaSuccess ? SPLAT_OK : SPLAT_ERR_CUDA;
}
